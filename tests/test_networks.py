"""The estimation study's networks (Section 4.2) and its measures, on the CPU:
the edge counts the paper prints for p = 500 (Table 4), the structure of each
generator, and the measures on cases worked out by hand."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import synth


def _edges(T):
    iu = np.triu_indices(T.shape[0], 1)
    return int(np.count_nonzero(T[iu]))


def _check_precision(T):
    assert np.array_equal(T, T.T)
    assert np.allclose(np.diag(T), 1.0)
    assert np.linalg.eigvalsh(T)[0] > 0.0


def test_ar_networks_edge_counts_and_values():
    p = 500
    T1 = synth.theta_ar1_paper(p)
    T4 = synth.theta_ar4(p)
    # |E| printed in Table 4 for p = 500
    assert _edges(T1) == 499 and _edges(T4) == 1990
    _check_precision(T1)
    _check_precision(T4)
    assert T1[10, 11] == 0.48 and T1[10, 12] == 0.0
    for d in range(1, 5):
        assert T4[100, 100 + d] == pytest.approx(0.6 ** d, rel=0, abs=1e-15)
    assert T4[100, 105] == 0.0


def test_scale_free_subnetworks_are_trees():
    p = 500
    T = synth.theta_scale_free(p, np.random.default_rng(4))
    _check_precision(T)
    assert _edges(T) == 495                      # Table 4: |E| = 495
    for s in range(0, p, 100):                   # block diagonal, one tree per block
        B = T[s:s + 100, s:s + 100]
        assert _edges(B) == 99
        off = np.ones((p, p), dtype=bool)
        off[s:s + 100, s:s + 100] = False
        assert not np.any(T[s:s + 100][:, off[s]])
    # a tree: connected with 99 edges (BFS over the block)
    A = T[:100, :100] != 0.0
    seen, todo = {0}, [0]
    while todo:
        v = todo.pop()
        for u in np.flatnonzero(A[v]):
            if int(u) not in seen:
                seen.add(int(u))
                todo.append(int(u))
    assert len(seen) == 100


def test_hub_subnetworks():
    p = 500
    T = synth.theta_hub_peng(p, np.random.default_rng(5))
    _check_precision(T)
    # Table 4 prints |E| = 551 for one draw; ten hubs and one or two hub links
    # per non-hub node give about 110 edges per 100 nodes
    assert 500 <= _edges(T) <= 600
    for s in range(0, p, 100):
        deg = np.count_nonzero(T[s:s + 100, s:s + 100], axis=1) - 1
        hubs = np.argsort(-deg)[:10]
        rest = np.setdiff1d(np.arange(100), hubs)
        assert deg[rest].min() >= 1 and deg[rest].max() <= 2
        assert deg[hubs].min() >= 9            # every hub gets 9 first links


def test_measures_by_hand():
    a, b, c, d = 0.3, -0.2, 0.25, 0.1
    true = np.array([[1, a, 0], [a, 1, b], [0, b, 1]], dtype=float)
    est = np.array([[1, c, d], [c, 1, 0], [d, 0, 1]], dtype=float)
    m = oracle.support_metrics(est, true)
    # (0,1): both nonzero; (0,2): estimated only; (1,2): true only
    assert (m["tp"], m["fp"], m["tn"], m["fn"]) == (1, 1, 0, 1)
    assert m["sen"] == 0.5 and m["spe"] == 0.0 and m["fdr"] == 0.5
    assert m["misr"] == pytest.approx(2.0 / 3.0)
    assert m["mcc"] == pytest.approx(-0.5)
    assert m["frobenius"] == pytest.approx(math.sqrt(2 * (a - c) ** 2 + 2 * d ** 2 + 2 * b ** 2))
    assert m["n_edges_hat"] == 2 and m["n_edges_true"] == 2


def test_measures_limits():
    T = synth.theta_ar1_paper(20)
    m = oracle.support_metrics(T, T)
    assert m["sen"] == 1.0 and m["spe"] == 1.0 and m["fdr"] == 0.0 and m["misr"] == 0.0
    assert m["mcc"] == 1.0 and m["frobenius"] == 0.0
    z = oracle.support_metrics(np.eye(20), T)
    assert z["sen"] == 0.0 and z["spe"] == 1.0
    assert math.isnan(z["fdr"]) and math.isnan(z["mcc"])
    assert z["misr"] == pytest.approx(19 / 190)


def test_measures_match_a_vectorised_count():
    """oracle.support_metrics (plain loops) against the same measures counted
    with whole-array operations, on random sparse pairs."""
    rng = np.random.default_rng(9)
    for p in (5, 40, 123):
        A = np.where(rng.random((p, p)) < 0.15, rng.standard_normal((p, p)), 0.0)
        B = np.where(rng.random((p, p)) < 0.15, rng.standard_normal((p, p)), 0.0)
        A[:3] = B[:3]
        m = oracle.support_metrics(A, B)
        iu = np.triu_indices(p, 1)
        e, t = A[iu] != 0, B[iu] != 0
        tp, fp = int(np.sum(e & t)), int(np.sum(e & ~t))
        tn, fn = int(np.sum(~e & ~t)), int(np.sum(~e & t))
        assert (m["tp"], m["fp"], m["tn"], m["fn"]) == (tp, fp, tn, fn)
        assert m["frobenius"] == pytest.approx(np.linalg.norm(A - B), rel=1e-12)
        assert m["mcc"] == pytest.approx(
            (tp * tn - fp * fn) / math.sqrt((tp + fp) * (tp + fn) * (tn + fp) * (tn + fn)), rel=1e-12)
