"""The usage example of the README runs as written (the documented calls
exist with the documented arguments and return what the example reads)."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_example_runs():
    text = open(os.path.join(ROOT, "README.md")).read()
    code = text.split("```python\n", 1)[1].split("```", 1)[0]
    ns = {}
    exec(compile(code, "README.md", "exec"), ns)
    out, bnd, r = ns["out"], ns["bnd"], ns["r"]
    cost = out["cost"].cpu().numpy()
    assert np.all(out["status"].cpu().numpy() == 0) and np.all(cost > 0)
    assert np.all(bnd["lower"].cpu().numpy() <= cost) and np.all(cost <= bnd["upper"].cpu().numpy())
    assert np.isfinite(float(ns["energy"][-1])) and r["status"] == 0 and r["cost"] > 0
    ns["ctx"].close()
