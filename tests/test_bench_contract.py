"""The benchmark's reference arm (the FP64 oracle on the host cores) prints one JSON line
with the keys the benchmark contract fixes; it needs no GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.slow
def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "points/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


class _FakeHandle:
    """The two exported arrays pass_rooflines reads (level offsets, operator offsets)."""

    def export(self, what):
        import numpy as np
        if what == "LEVEL_BASE":
            return np.array([0, 1, 9, 73, 585, 4681], dtype=np.int64)
        if what == "OP_OFF":
            return np.arange(4682, dtype=np.int64) * 100
        raise KeyError(what)


def _passes(nrhs, precision):
    sys.path.insert(0, ROOT)
    import bench
    st = {"kappa": 4, "op_entries": 468100, "n_pivots": 1000, "n": 5000, "m2l_pairs": 10 ** 6,
          "m2l_evals": 5 * 10 ** 5, "p2p_pairs": 2 * 10 ** 6}
    out = bench.pass_rooflines(_FakeHandle(), st, [0.0, 1.0, 1.0, 1.0, 1.0, 4.0], 152, 2070.0, {}, nrhs, precision)
    return {p["pass"]: p for p in out}


def test_pass_work_counts_whole_product():
    """The work of every pass is summed over the product's passes of right-hand sides,
    the same way as the pass times it is divided by."""
    p = _passes(1, "fp32")
    assert p["m2l"]["work"] == 5 * 10 ** 5 and p["l2p_p2p"]["work"] == 2 * 10 ** 6
    assert p["p2m_m2m"]["work"] == 8 * (468100 + 6000)
    p = _passes(9, "fp32")      # two passes of four, then one right-hand side
    assert p["m2l"]["work"] == 2 * 10 ** 6 + 5 * 10 ** 5
    assert p["l2p_p2p"]["work"] == 3 * 2 * 10 ** 6
    assert p["p2m_m2m"]["work"] == 8 * (3 * 468100 + 9 * 6000)
    assert p["l2l"]["work"] == 8 * (3 * 58500 + 2 * 9 * 1000)   # non-leaf operators: cells before the leaf level
    p = _passes(64, "tf32x3")   # one tensor-core pass, operators in eight groups of eight
    assert p["m2l"]["work"] == 2.0 * 3 * 10 ** 6 * 64 and p["m2l"]["bound"] == "tensor"
    assert p["l2p_p2p"]["work"] == 16 * 2 * 10 ** 6
    assert p["p2m_m2m"]["work"] == 8 * (8 * 468100 + 64 * 6000)
