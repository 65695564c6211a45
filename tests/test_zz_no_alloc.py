"""spmesl_fit_noalloc: the fit for callers that cannot allocate device memory
(a plugin whose host application owns all device memory, real-time code that
forbids allocation after start-up).  Its scratch is the library's own fixed
device array, so its results must equal spmesl_fit's on the same input bit
for bit, call after call, and a call after the first must not change the
device memory in use.  Kept in a file of its own that pytest collects last."""
from __future__ import annotations

import gc

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2203_15031_gb300 as sp  # noqa: E402

DEV = torch.device("cuda", 0)
MAX_P = {sp.FP32: 2351, sp.MIXED: 2351, sp.FP64: 1664}   # the 64 MiB scratch's limits


def _free_device_bytes() -> int:
    free, _ = torch.cuda.mem_get_info(DEV)        # cudaMemGetInfo
    return int(free)


def _with_workspace(S, lam, tol, prec):
    p = S.shape[0]
    opts = sp.spmesl_default_opts()
    opts.precision = prec
    T = torch.empty((p, p), dtype=torch.float64, device=DEV)
    sg = torch.empty(p, dtype=torch.float64, device=DEV)
    nb = sp.spmesl_fit_workspace_bytes(p, prec)
    keep, ws = sp._workspace(nb, DEV)
    st = sp.Stats()
    assert sp.spmesl_fit(S, 0, p, lam, tol, 1000, opts, T, sg, st, ws, nb) == sp.SPMESL_OK
    del keep
    return T.cpu().numpy(), sg.cpu().numpy()


def _without_allocation(S, lam, tol, prec, T=None, sg=None):
    p = S.shape[0]
    opts = sp.spmesl_default_opts()
    opts.precision = prec
    T = torch.empty((p, p), dtype=torch.float64, device=DEV) if T is None else T
    sg = torch.empty(p, dtype=torch.float64, device=DEV) if sg is None else sg
    st = sp.Stats()
    rc = sp.spmesl_fit_noalloc(S, 0, p, lam, tol, 1000, opts, T, sg, st)
    assert rc == sp.SPMESL_OK, sp.spmesl_status_string(rc)
    assert st.lambda0 == lam
    return T.cpu().numpy(), sg.cpu().numpy()


@pytest.mark.parametrize("kind,p,n,seed,prec,tol", [
    ("er", 300, 120, 3, sp.FP32, 1e-6),
    ("hub_scaled", 400, 150, 5, sp.MIXED, 1e-6),
    ("ar1", 100, 50, 0, sp.FP64, 1e-8),
])
def test_noalloc_equals_workspace_fit_on_consecutive_calls(kind, p, n, seed, prec, tol):
    dt = np.float64 if prec == sp.FP64 else np.float32
    prob = synth.make_problem(kind, p, n, seed, dtype=dt)
    S = sp.gram(torch.from_numpy(prob.X).to(DEV), precision=prec)
    Tw, sw = _with_workspace(S, prob.lambda0, tol, prec)
    for _ in range(2):               # two calls in a row on the shared scratch
        Tn, sn = _without_allocation(S, prob.lambda0, tol, prec)
        assert np.array_equal(Tn, Tw) and np.array_equal(sn, sw)


def test_noalloc_allocates_nothing_after_the_first_call():
    prob = synth.make_problem("er", 500, 200, 9, dtype=np.float32)
    S = sp.gram(torch.from_numpy(prob.X).to(DEV), precision=sp.FP32)
    T = torch.empty((500, 500), dtype=torch.float64, device=DEV)
    sg = torch.empty(500, dtype=torch.float64, device=DEV)
    _without_allocation(S, prob.lambda0, 1e-6, sp.FP32, T, sg)      # first call: set-up
    # tensors left by earlier tests are collected first, and no collection may
    # free any while the two calls run
    gc.collect()
    torch.cuda.synchronize()
    gc.disable()
    try:
        torch_before, free_before = torch.cuda.memory_allocated(DEV), _free_device_bytes()
        for _ in range(2):
            _without_allocation(S, prob.lambda0, 1e-6, sp.FP32, T, sg)
        torch.cuda.synchronize()
        torch_after, free_after = torch.cuda.memory_allocated(DEV), _free_device_bytes()
    finally:
        gc.enable()
    assert torch_after == torch_before
    assert free_after == free_before


def test_noalloc_size_limits():
    # the largest p the scratch holds runs (FP32), one more is refused
    p = MAX_P[sp.FP32]
    prob = synth.make_problem("ar1", p, 60, 1, dtype=np.float32)
    S = sp.gram(torch.from_numpy(prob.X).to(DEV), precision=sp.FP32)
    _without_allocation(S, prob.lambda0, 1e-6, sp.FP32)
    fake = 1 << 20           # never dereferenced: the size check comes first
    opts = sp.spmesl_default_opts()
    for prec, limit in MAX_P.items():
        opts.precision = prec
        assert sp.spmesl_fit_noalloc(fake, 0, limit + 1, 0.1, 1e-6, 10, opts, fake, fake,
                                     None) == sp.SPMESL_ENOMEM
