"""Pins of the oracle's exponential integrators (Sect. 4): exactness on a
linear system (the remainder vanishes) and the convergence order each method
is named for, observed against a tight implicit reference solution."""
from tests import pins


def test_integrators_exact_on_linear_systems():
    assert pins.pin_integrators_linear_exact() < 1e-12


def test_integrator_orders():
    orders = pins.integrator_orders()
    assert orders["srerk3"] > 2.8          # named third order
    assert orders["epi4"] > 3.8
    assert orders["epi5"] > 4.8
