"""Serving context (continuous batching) through the C ABI: results equal to
the same fit alone, overlapping work, admission under the memory budget,
per-request errors."""
from __future__ import annotations

import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2203_15031_gb300 as sp  # noqa: E402

DEV = torch.device("cuda", 0)
GB = 1 << 30


def _wait(srv, ticket, timeout=60.0):
    t0 = time.time()
    while True:
        r = srv.poll(ticket)
        if r is not None:
            return r
        if time.time() - t0 > timeout:
            raise TimeoutError(ticket)
        time.sleep(0.0002)


def _requests(specs):
    probs = [synth.make_problem(s["kind"], s["p"], s["n"], s["seed"], dtype=np.float32)
             for s in specs]
    return probs, [torch.from_numpy(pr.X).to(DEV) for pr in probs]


SPECS = [dict(kind="er", p=120, n=60, seed=1), dict(kind="ar1", p=400, n=100, seed=2),
         dict(kind="hub_scaled", p=250, n=80, seed=3), dict(kind="er", p=600, n=150, seed=4),
         dict(kind="ar1", p=90, n=40, seed=5), dict(kind="er", p=333, n=90, seed=6),
         dict(kind="hub_scaled", p=700, n=175, seed=7), dict(kind="ar1", p=50, n=30, seed=8)]


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_same_result_alone_and_in_the_mix(prec):
    probs, Xs = _requests(SPECS)
    srv = sp.Server(8 * GB, max_slots=64, precision=prec)
    alone = []
    for pr, X in zip(probs, Xs):
        st, T, sg, info = _wait(srv, srv.submit(X, pr.lambda0))
        assert st == sp.SPMESL_OK and info["batch_size"] == 1
        alone.append((T.clone(), sg.clone()))
    tickets = [srv.submit(X, pr.lambda0) for pr, X in zip(probs, Xs)]   # arrive together
    for k, t in enumerate(tickets):
        st, T, sg, info = _wait(srv, t)
        assert st == sp.SPMESL_OK
        assert torch.equal(T, alone[k][0]) and torch.equal(sg, alone[k][1]), k
        # and equal to the plain single-fit path
        S = sp.gram(Xs[k], precision=prec)
        T1, s1, _ = sp.fit(S, probs[k].lambda0, tol=1e-6, precision=prec)
        assert torch.equal(T, T1) and torch.equal(sg, s1)
    srv.close()


def test_later_small_request_overlaps_and_finishes_first():
    """A small request submitted while a large one is on the GPU runs in its
    own batch at once and completes before the large one (completion times
    from the submit clock plus each request's measured latency)."""
    big = synth.make_problem("er", 4000, 1000, 11, dtype=np.float32)
    small = synth.make_problem("ar1", 80, 40, 12, dtype=np.float32)
    Xb = torch.from_numpy(big.X).to(DEV)
    Xs = torch.from_numpy(small.X).to(DEV)
    srv = sp.Server(16 * GB, max_slots=16)
    _wait(srv, srv.submit(Xb, big.lambda0))            # warm the context up
    overlapped = 0
    for _ in range(3):
        tb = srv.submit(Xb, big.lambda0)
        t_big = time.perf_counter()
        while srv.query()["running"] == 0:              # the big one is admitted
            time.sleep(0.00005)
        ts = srv.submit(Xs, small.lambda0)
        t_small = time.perf_counter()
        rs, rb = _wait(srv, ts), _wait(srv, tb)
        assert rs[0] == sp.SPMESL_OK and rb[0] == sp.SPMESL_OK
        assert rs[3]["batch_size"] == 1 and rb[3]["batch_size"] == 1
        done_small = t_small + rs[3]["ms_total"] / 1e3
        done_big = t_big + rb[3]["ms_total"] / 1e3
        overlapped += done_small < done_big
    assert overlapped >= 1
    srv.close()


def test_admission_stays_within_budget():
    probs, Xs = _requests([dict(kind="er", p=1500, n=300, seed=20 + k) for k in range(6)])
    budget = 60 << 20            # room for about two of these fits at a time
    srv = sp.Server(budget, max_slots=64)
    tickets = [srv.submit(X, pr.lambda0) for pr, X in zip(probs, Xs)]
    seen_queue = False
    pending = set(tickets)
    t0 = time.time()
    while pending and time.time() - t0 < 120:
        q = srv.query()
        assert q["bytes_in_use"] <= budget
        seen_queue |= q["queued"] > 0
        for t in list(pending):
            r = srv.poll(t)
            if r is not None:
                assert r[0] == sp.SPMESL_OK
                pending.discard(t)
        time.sleep(0.0002)
    assert not pending and seen_queue
    srv.close()


def test_request_errors():
    srv = sp.Server(1 << 20, max_slots=4)        # 1 MiB budget
    X = torch.from_numpy(synth.make_problem("er", 600, 100, 3, dtype=np.float32).X).to(DEV)
    with pytest.raises(sp.SpmeslError) as e:
        srv.submit(X, 0.2)                       # needs more than the whole budget
    assert e.value.status == sp.SPMESL_ENOMEM
    with pytest.raises(sp.SpmeslError) as e:
        srv.poll(12345)
    assert e.value.status == sp.SPMESL_ENOTFOUND
    srv.close()
    srv = sp.Server(4 * GB, max_slots=16)
    good = synth.make_problem("ar1", 100, 50, 4, dtype=np.float32)
    Xg = torch.from_numpy(good.X).to(DEV)
    Xbad = Xg.clone()
    Xbad[2, 3] = float("nan")
    t1 = srv.submit(Xg, good.lambda0)
    t2 = srv.submit(Xbad, good.lambda0)
    t3 = srv.submit(Xg, good.lambda0)
    assert _wait(srv, t2)[0] == sp.SPMESL_ENONFINITE
    r1, r3 = _wait(srv, t1), _wait(srv, t3)
    assert r1[0] == sp.SPMESL_OK and r3[0] == sp.SPMESL_OK and torch.equal(r1[1], r3[1])
    srv.close()
