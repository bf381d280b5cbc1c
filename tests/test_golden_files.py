"""The stored full-size oracle solves (tests/golden/config2_oracle.json and the solution fields in
config2_oracle_fields.npz) are complete and self-consistent: every instance has its fields, of the
workload's size, finite, and the source f reproduces the summaries written beside it."""
import json
import os

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(__file__), "golden")


def _load():
    path = os.path.join(HERE, "config2_oracle.json")
    if not os.path.exists(path):
        pytest.skip("golden oracle solve not generated")
    with open(path) as fh:
        g = json.load(fh)
    fpath = os.path.join(HERE, g.get("fields", "config2_oracle_fields.npz"))
    if not os.path.exists(fpath):
        pytest.skip("golden oracle fields not generated")
    return g, dict(np.load(fpath))


def test_golden_fields_complete_and_consistent():
    g, arr = _load()
    N = 255 * 255
    assert len(g["instances"]) == 2
    for k, inst in enumerate(g["instances"]):
        assert inst["converged"] and inst["relres_est"] <= 1e-10
        assert inst["v_levels"] == [1, 128, 256]
        for name in ("f", "v1", "vmid", "vS"):
            a = arr["%s_%d" % (name, k)]
            assert a.shape == (N,) and a.dtype == np.float64 and np.isfinite(a).all()
        f = arr["f_%d" % k]
        assert np.linalg.norm(f) == pytest.approx(inst["f_norm2"], rel=1e-14)
        assert f.sum() == pytest.approx(inst["f_sum"], rel=1e-13)
        assert f[N // 2] == inst["f_center"]
        # the residual history decreases to the stop and ends at the estimate
        h = inst["history"]
        assert h[0] == 1.0 and h[-1] == pytest.approx(inst["relres_est"], rel=1e-5)
