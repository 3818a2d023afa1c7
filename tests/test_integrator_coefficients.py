"""The integrators' coefficients, in the oracle and in the product, equal the
values Sect. 4 prints (tests/golden/integrator_coefficients.json); the two
copies are written independently, so this also checks they agree."""
import json
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "integrator_coefficients.json")


def golden():
    with open(GOLDEN) as f:
        g = json.load(f)
    mats = {k: np.array([[float(Fraction(x)) for x in row] for row in g[k]]) for k in ("epi4", "epi5")}
    return mats, {k: float(Fraction(v)) for k, v in g["srerk3"].items()}


def test_oracle_coefficients_are_the_printed_ones():
    from oracle import integrators as OI

    mats, _ = golden()
    for order in (4, 5):
        assert np.array_equal(OI.EPI_ALPHA[order], mats[f"epi{order}"])


def test_product_coefficients_are_the_printed_ones():
    import ast

    # read the product module's table as text (no import: the module loads the CUDA library)
    src = open(os.path.join(os.path.dirname(GOLDEN), "..", "..", "paper_2410_14917_gb300",
                            "integrators.py")).read()
    tree = ast.parse(src)
    table = next(node.value for node in ast.walk(tree)
                 if isinstance(node, ast.Assign) and any(getattr(t, "id", "") == "EPI_ALPHA" for t in node.targets))
    alpha = eval(compile(ast.Expression(table), "integrators.py", "eval"))
    mats, s3 = golden()
    for order in (4, 5):
        assert np.array_equal(np.array(alpha[order]), mats[f"epi{order}"])
    assert "0.75 * h" in src and "(32.0 / 9.0) * h" in src
    assert s3["c1"] == 0.75 and s3["phi3_weight"] == 32.0 / 9.0
