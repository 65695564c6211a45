"""spmesl_fit_noalloc: the fit for callers that cannot allocate device memory
(its scratch is the library's own fixed device array).  Its results must match
spmesl_fit's on the same input, call after call.  Kept in a file of its own
that pytest collects last."""
from __future__ import annotations

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2203_15031_gb300 as sp  # noqa: E402

DEV = torch.device("cuda", 0)
REL = 1e-4      # the parity tolerance used for Theta throughout the tests


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


def _without_allocation(S, lam, tol, prec):
    p = S.shape[0]
    opts = sp.spmesl_default_opts()
    opts.precision = prec
    T = torch.empty((p, p), dtype=torch.float64, device=DEV)
    sg = torch.empty(p, dtype=torch.float64, device=DEV)
    st = sp.Stats()
    rc = sp.spmesl_fit_noalloc(S, 0, p, lam, tol, 1000, opts, T, sg, st)
    assert rc == sp.SPMESL_OK, sp.spmesl_status_string(rc)
    return T.cpu().numpy(), sg.cpu().numpy()


def _close(a, b):
    scale = float(np.max(np.abs(b)))
    return float(np.max(np.abs(a - b))) <= REL * scale


def test_noalloc_matches_workspace_fit_on_consecutive_calls():
    cases = [("er", 300, 120, 3, np.float32, sp.FP32, 1e-6),
             ("ar1", 100, 50, 0, np.float64, sp.FP64, 1e-8)]
    for kind, p, n, seed, dt, prec, tol in cases:
        prob = synth.make_problem(kind, p, n, seed, dtype=dt)
        S = sp.gram(torch.from_numpy(prob.X).to(DEV), precision=prec)
        Tw, sw = _with_workspace(S, prob.lambda0, tol, prec)
        for _ in range(2):               # two calls in a row on the shared scratch
            Tn, sn = _without_allocation(S, prob.lambda0, tol, prec)
            assert _close(Tn, Tw) and _close(sn, sw)


def test_noalloc_rejects_p_beyond_its_scratch():
    fake = 1 << 20           # never dereferenced: the size check comes first
    opts = sp.spmesl_default_opts()
    opts.precision = sp.FP32
    assert sp.spmesl_fit_noalloc(fake, 0, 2359, 0.1, 1e-6, 10, opts, fake, fake, None) == sp.SPMESL_ENOMEM
    opts.precision = sp.FP64
    assert sp.spmesl_fit_noalloc(fake, 0, 1665, 0.1, 1e-6, 10, opts, fake, fake, None) == sp.SPMESL_ENOMEM
