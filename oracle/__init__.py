"""CPU oracle for the Krylov phi-product path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, float64 NumPy/SciPy restatement of what the paper's method
computes, used to check the CUDA path.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the product (``paper_2410_14917_gb300``) never does, and this package never
imports the product.  The two share no code: the oracle builds its operators as
sparse matrices from Kronecker products, the CUDA path applies stencils.

Modules (each function cites the passage of the paper it follows):
  operators  sparse matrices of the three synthetic stencil operators
  phi        scalar phi_k functions (Sect. 2, Eqs. 5-6)
  expm       small dense exponential by Taylor scaling and squaring
  exact      O-exact: dense augmented exponential (Sect. 2.1, Eq. 7), FFT and
             diagonal closed forms
  arnoldi    MGS (Alg. 1), classical CGS2 (textbook, Sect. 2.3), hybrid
             low-synchronisation Arnoldi (Alg. 4 with Algs. 5, 6, 7)
  krylov     O-Krylov: phi_k(hA)v by Krylov projection (Sect. 2.2, Eq. 13,
             with the phi augmentation of Sect. 2.1)
  lincomb    sum_j tau^j phi_j(tau A) b_j by Krylov projection of the
             augmented operator (Sect. 2.1, Eqs. 7-9) in equal sub-steps
  adjoint    gradients of a phi_1 loss (Krylov and dense Frechet forms)
  integrators  SRERK3, EPI4 and EPI5 (Sect. 4) on phi linear combinations

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against a closed form, a library routine, brute force or a worked example of
the paper.  The loss-of-orthogonality level of each Gram-Schmidt variant, for
which the paper states no bound, is pinned to the textbook laws instead:
driven as a Gram-Schmidt QR of a matrix of condition number kappa, MGS and the
hybrid corrections stay within 2 eps kappa (Bjorck's law for MGS; the paper
states the hybrids match MGS accuracy) and CGS2 within 10 n eps ("twice is
enough").
"""
