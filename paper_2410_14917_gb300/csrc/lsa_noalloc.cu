// lsa_phiv_noalloc: the phi-product entry point for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: plugins that run inside a host
// application which owns all device memory through its own pool allocator,
// and latency-critical code that must not allocate or free after start-up
// (cudaMalloc/cudaFree can synchronise the whole device).  For them the
// workspace of lsa_phiv lives in a fixed, file-scope device array of
// LSA_STATIC_WORKSPACE_BYTES that the library carries; every GPU that loads
// the library holds it until the process exits.
//
// In host code `g_lsa_static_work` names only a host-side stand-in, never the
// device memory, so the device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached.  The entry point
// itself then calls the regular lsa_phiv with that address as its workspace,
// with no event creation and no allocation of any kind.  The cached address
// belongs to the device's current context: after cudaDeviceReset (or a release
// and re-creation of the primary context) the library's module is loaded
// again and the cache must not be used, so a process that resets a device
// must not call this entry point afterwards.
#include <atomic>

#include "lsa_internal.cuh"

namespace {

constexpr size_t kStaticBytes = (size_t)LSA_STATIC_WORKSPACE_BYTES;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_lsa_static_work[kStaticBytes];

// device address of g_lsa_static_work, per device (first calls from several
// host threads may all look it up; they store the same value)
std::atomic<void*> g_static_addr[kMaxDevices];

}  // namespace

extern "C" lsa_status lsa_phiv_noalloc(const lsa_op* op, const double* v, double h, int p, int m,
                                       double tol, int variant, int precision, double* y,
                                       lsa_stats* stats, void* stream) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return LSA_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return LSA_ERR_ARG;
  void* work = g_static_addr[dev].load(std::memory_order_acquire);
  if (!work) {                        // first call on this device: look the array up
    if (cudaGetSymbolAddress(&work, g_lsa_static_work) != cudaSuccess || !work)
      return LSA_ERR_CUDA;
    g_static_addr[dev].store(work, std::memory_order_release);
  }
  const long long N = lsa_op_dof(op);
  if (N < 1 || m < 1) return LSA_ERR_ARG;
  const int m_used = (m > N) ? (int)N : m;
  const size_t need = lsa_workspace_bytes(op, m_used, p, precision);
  if (need == 0) return LSA_ERR_ARG;
  if (need > kStaticBytes) return LSA_ERR_WORKSPACE;   // beyond the fixed maximum
  lsa_status st = lsa_phiv(op, v, h, p, m, tol, variant, precision, y, work, kStaticBytes,
                           nullptr, stream);
  if (st != LSA_OK) return st;
  if (stats) return lsa_read_stats(work, stats, stream);
  return LSA_OK;
}
