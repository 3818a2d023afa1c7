"""The CPU oracle against facts it does not compute itself (closed forms,
library routines, brute force, the paper's worked example).  No GPU."""
import pytest

from tests import pins

VARIANTS = ["mgs", "cgs2", "hcwy", "hncwy", "hgsmgs"]


def test_phi_at_zero():
    # phi_k(0) = 1/k!  (Eq. 6 at z = 0)
    assert pins.pin_phi_at_zero() < 1e-15


def test_phi_matches_integral_definition():
    assert pins.pin_phi_quadrature() < 1e-12


def test_expm_matches_scipy():
    assert pins.pin_expm_vs_scipy() < 1e-13


def test_expm_nilpotent_and_diagonal():
    assert pins.pin_expm_nilpotent_shift() < 1e-15
    assert pins.pin_expm_diagonal() < 1e-14


def test_advdiff_operator_fourier_symbol():
    assert pins.pin_advdiff_fourier() < 1e-10


def test_adr_operator_fourier_symbol():
    assert pins.pin_adr_fourier() < 1e-10


def test_grayscott_operator_is_jacobian_of_rhs():
    assert pins.pin_grayscott_jacobian() < 1e-8


def test_t3_worked_example():
    assert pins.pin_t3_worked_example() < 1e-15


def test_cwy_projector_identity():
    assert pins.pin_cwy_projector_identity() < 1e-13


def test_gsmgs_equals_two_gauss_seidel_sweeps():
    assert pins.pin_gsmgs_two_sweeps() < 1e-13


def test_norm_estimate_exact_for_orthonormal_basis():
    assert pins.pin_norm_estimate_orthonormal() < 1e-12


def test_mgs_basis_is_q_of_krylov_matrix():
    assert pins.pin_mgs_vs_qr() < 1e-10


def test_variants_equal_mgs():
    assert pins.pin_variants_equal_mgs() < 1e-11


def test_orthogonality_follows_textbook_laws():
    # MGS and the hybrid corrections within 2 eps kappa(X), CGS2 within 10 n eps
    assert pins.pin_orthogonality_laws() <= 1.0


@pytest.mark.parametrize("variant", VARIANTS)
def test_arnoldi_relation(variant):
    assert pins.pin_arnoldi_relation(variant) < 1e-14


@pytest.mark.parametrize("variant", ["mgs", "hcwy"])
def test_krylov_matches_dense_augmented_exponential(variant):
    assert pins.pin_krylov_vs_dense(variant) < 1e-12


def test_krylov_grayscott_matches_dense():
    assert pins.pin_krylov_grayscott_vs_dense() < 1e-11


@pytest.mark.parametrize("variant", VARIANTS)
def test_krylov_matches_fft_on_advdiff_64(variant):
    assert pins.pin_krylov_vs_fft_config1(variant) < 1e-12


def test_krylov_matches_fft_on_adr3d():
    assert pins.pin_krylov_vs_fft_adr() < 1e-11


@pytest.mark.parametrize("variant", VARIANTS)
def test_diagonal_operator_breakdown_exact(variant):
    assert pins.pin_diagonal_breakdown(variant) < 1e-12


@pytest.mark.parametrize("variant", VARIANTS)
def test_zero_operator(variant):
    assert pins.pin_zero_operator(variant) < 1e-15


@pytest.mark.parametrize("variant", VARIANTS)
def test_h_zero(variant):
    assert pins.pin_h_zero(variant) < 1e-14


def test_sync_counts():
    assert pins.pin_sync_counts() == 0


def test_iocgs_symmetric_operator_is_lanczos():
    assert pins.pin_iocgs_symmetric_is_lanczos() < 1e-9


def test_iocgs_defining_properties():
    assert pins.pin_iocgs_defining_properties() < 1e-12
