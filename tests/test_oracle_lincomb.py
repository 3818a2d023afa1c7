"""Pins of the oracle's phi-function linear combinations (Sect. 2.1, Eqs. 7-9)
and their equal sub-steps: closed forms for a diagonal operator, the forced
ODE the combination solves, dense exponentials of the augmented matrix, and
the single-vector case of the plain phi products."""
from tests import pins


def test_lincomb_diagonal_closed_form():
    assert pins.pin_lincomb_diagonal() < 1e-12


def test_lincomb_solves_forced_ode():
    assert pins.pin_lincomb_solves_forced_ode() < 1e-9


def test_lincomb_substeps_match_dense_augmented_exponential():
    assert pins.pin_lincomb_substeps_vs_dense() < 1e-11


def test_lincomb_single_vector_is_a_phi_product():
    assert pins.pin_lincomb_single_vector() < 1e-11


def test_lincomb_adaptive_substeps_meet_the_tolerance():
    err_over_tol, nsteps, converged = pins.pin_lincomb_adaptive()
    assert converged and nsteps > 1
    assert err_over_tol < 10.0


def test_lincomb_adaptive_dimension_grows_and_shrinks():
    """Adaptive sub-step size and Krylov dimension (this build's rule): a start
    far below the needed dimension is raised, one far above it is lowered,
    both meet the tolerance against the dense augmented exponential, and the
    modeled cost beats the fixed-m controller from the same start."""
    r = pins.pin_lincomb_adaptive_m()
    lo, hi = r[4], r[40]
    assert lo["converged"] and hi["converged"]
    assert lo["err"] < 10.0 and hi["err"] < 10.0
    assert lo["largest"] >= 10                # raised from 4
    assert hi["last"] <= 20                   # lowered from 40
    assert lo["cost_ratio"] < 0.5 and hi["cost_ratio"] < 1.0
