"""Pins of the oracle's gradients of 1/2 ||phi_1(hA(theta))v - y_t||^2 (the
adjoint workload): against dense exponentials and Frechet derivatives of exp
(tiny grid) and against central differences of the loss (step 1e-6)."""
from tests import pins


def test_adjoint_krylov_matches_dense_frechet():
    assert pins.pin_adjoint_vs_dense() < 1e-9


def test_adjoint_dF_closed_form_matches_frechet():
    assert pins.pin_adjoint_dF_closed_form() < 1e-12


def test_adjoint_matches_central_differences():
    assert pins.pin_adjoint_finite_differences() < 1e-5
