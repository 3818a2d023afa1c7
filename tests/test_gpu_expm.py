"""S5: phi_k(h H) e_1 from the GPU's augmented-matrix exponential against the
oracle (Taylor scaling and squaring, checked itself against scipy)."""
import numpy as np
import pytest

from oracle import krylov as OK

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def hessenberg(m, scale, seed):
    rng = np.random.default_rng(seed)
    H = np.triu(rng.standard_normal((m, m)), -1) * scale / np.sqrt(m)
    H[np.arange(1, m), np.arange(m - 1)] = np.abs(H[np.arange(1, m), np.arange(m - 1)]) + 0.1
    return H


@pytest.mark.parametrize("m,scale,h,p", [(1, 1.0, 0.5, 0), (5, 2.0, 1.0, 1), (30, 4.0, 1.0, 3),
                                         (64, 10.0, 1.0, 2), (40, 30.0, 0.4, 1), (64, 1.0, 0.0, 8),
                                         (17, 100.0, 1.0, 4)])
def test_expm_phi_matches_oracle(m, scale, h, p):
    import paper_2410_14917_gb300 as lsa

    H = hessenberg(m, scale, seed=m * 7 + p)
    C = lsa.expm_phi(torch.from_numpy(H).cuda(), m, h, p).cpu().numpy()
    ref = OK.small_phi_coeffs(H, h, p)
    for k in range(p + 2):
        err = np.abs(C[k] - ref[k]).max() / max(np.abs(ref[k]).max(), 1e-300)
        assert err < 5e-12, (k, err)
