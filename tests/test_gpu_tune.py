"""The full batch tuner on the GPU: it picks a launch choice by timing the
batch, stores it in the cache file, and a second process applies the stored
choice without timing (spmesl_batch_tune_cached)."""
from __future__ import annotations

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, {root!r})
import paper_2203_15031_gb300 as sp, synth
probs = [synth.make_problem(k, p, n, s, dtype=np.float32)
         for k, p, n, s in (("er", 300, 120, 3), ("hub_scaled", 257, 90, 3), ("ar1", 150, 60, 1))]
inputs = [(torch.from_numpy(pr.X).cuda(), pr.lambda0) for pr in probs]
bt = sp.Batch(inputs, kind="X", precision="mixed", tol=1e-6, maxit=1000, use_graph=True)
choice = bt.tune(cache={path!r})
bt.run()
statuses, _ = bt.result()
print(json.dumps({{"choice": choice, "statuses": statuses}}))
"""


def _run(path):
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, path=path)],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])


def test_second_process_reuses_the_cached_choice(tmp_path):
    path = str(tmp_path / "tune.json")
    first = _run(path)
    assert first["choice"]["from_cache"] == 0 and first["choice"]["ms"] > 0
    assert all(s == 0 for s in first["statuses"])
    assert os.path.exists(path)
    second = _run(path)
    assert second["choice"]["from_cache"] == 1
    for k in ("warps_per_block", "handover", "heavy_min_p", "heavy_heat"):
        assert second["choice"][k] == first["choice"][k]
    assert all(s == 0 for s in second["statuses"])
