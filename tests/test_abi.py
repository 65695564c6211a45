"""The C-ABI library builds for sm_103a, loads and exports every symbol that
include/*.h declares; host-only entry points behave (no GPU needed)."""
from __future__ import annotations

import ctypes
import glob
import json
import math
import os
import re

import pytest

import paper_2203_15031_gb300 as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(spmesl_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    path = sp.build()
    h = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(h, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    for n in declared_functions():
        assert hasattr(sp, n), n


def test_defaults_version_status_strings():
    o = sp.spmesl_default_opts()
    assert o.precision == sp.FP32 and o.standardize == 1 and o.center == 0
    assert o.inner_rule == sp.INNER_COLUMN
    assert sp.spmesl_version() >= 10000
    assert "invalid" in sp.spmesl_status_string(sp.SPMESL_EINVAL)
    assert sp.spmesl_status_string(0) == "ok"


def test_host_penalty_levels_match_paper_example():
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "lambda_p1000_n100.json")))
    p, n, tol = g["p"], g["n"], g["abs_tol"]
    assert abs(sp.spmesl_lambda(sp.LAMBDA_UB, n, p) - g["lambda_ub"]) < tol
    assert abs(sp.spmesl_lambda(sp.LAMBDA_PB, n, p) - g["lambda_pb"]) < tol
    assert abs(sp.spmesl_lambda(sp.LAMBDA_UNIV_PM1, n, p) - g["lambda_univ_pm1"]) < tol
    assert abs(sp.spmesl_lambda(sp.LAMBDA_UNIV, 50, 100) - math.sqrt(2 * math.log(100) / 50)) < 1e-15
    assert math.isnan(sp.spmesl_lambda(sp.LAMBDA_GIVEN, n, p))


def test_workspace_sizes():
    for prec, s in ((sp.FP64, 8), (sp.FP32, 4)):
        nb = sp.spmesl_fit_workspace_bytes(2000, prec)
        assert nb >= 3 * 2000 * 2016 * s
        assert sp.spmesl_solve_workspace_bytes(200, 2000, prec) > nb
    assert sp.spmesl_fit_workspace_bytes(1, sp.FP32) == 0
    assert sp.spmesl_max_p(sp.FP32) >= 10000
    assert sp.spmesl_max_p(sp.FP64) >= 5000


def test_invalid_arguments_rejected_on_host():
    # no device work is enqueued on these paths: validation comes first
    st = sp.Stats()
    o = sp.spmesl_default_opts()
    fake = 1 << 20        # never dereferenced
    assert sp.spmesl_fit(None, 10, 5, 0.1, 1e-6, 10, o, fake, fake, None, fake, 1 << 30, 0) == sp.SPMESL_EINVAL
    assert sp.spmesl_fit(fake, 10, 1, 0.1, 1e-6, 10, o, fake, fake, None, fake, 1 << 30, 0) == sp.SPMESL_EINVAL
    assert sp.spmesl_fit(fake, 10, 5, -0.1, 1e-6, 10, o, fake, fake, None, fake, 1 << 30, 0) == sp.SPMESL_EINVAL
    assert sp.spmesl_fit(fake, 10, 5, 0.1, 0.0, 10, o, fake, fake, None, fake, 1 << 30, 0) == sp.SPMESL_EINVAL
    assert sp.spmesl_fit(fake, 10, 5, 0.1, 1e-6, 0, o, fake, fake, None, fake, 1 << 30, 0) == sp.SPMESL_EINVAL
    assert sp.spmesl_fit(fake, 10, 5, 0.1, 1e-6, 10, o, fake, fake, None, fake, 16, 0) == sp.SPMESL_EINVAL
    assert sp.spmesl_fit(fake + 8, 10, 5, 0.1, 1e-6, 10, o, fake, fake, None, fake + 8, 1 << 30, 0) == sp.SPMESL_EINVAL
    big = sp.spmesl_max_p(sp.FP32) + 32
    assert sp.spmesl_fit(fake, 10, big, 0.1, 1e-6, 10, o, fake, fake, None, fake, 1 << 40, 0) == sp.SPMESL_EINVAL
    o.inner_rule = 7
    assert sp.spmesl_fit(fake, 10, 5, 0.1, 1e-6, 10, o, fake, fake, None, fake, 1 << 30, 0) == sp.SPMESL_EINVAL
    o = sp.spmesl_default_opts()
    o.lambda_rule = sp.LAMBDA_UNIV
    assert sp.spmesl_fit(fake, 0, 5, 0.0, 1e-6, 10, o, fake, fake, None, fake, 1 << 30, 0) == sp.SPMESL_EINVAL
    assert sp.spmesl_gram(fake, 0, 5, 5, sp.FP32, 0, fake, 5, fake, 1 << 20, 0) == sp.SPMESL_EINVAL
    assert sp.spmesl_gram(fake, 4, 5, 3, sp.FP32, 0, fake, 5, fake, 1 << 20, 0) == sp.SPMESL_EINVAL
    assert sp.spmesl_gram(fake, 4, 5, 5, 9, 0, fake, 5, fake, 1 << 20, 0) == sp.SPMESL_EINVAL


def _al(x):
    return (x + 255) // 256 * 256


def test_residual_workspace_layout_and_limits():
    """spmesl_fit_residual_workspace_bytes: the control block, six p-vectors,
    W (ldn x ldp), Wt (p x ldn) and the coefficients (p x ldp), each 256-byte
    aligned, with ldn = roundup(n, 32) and ldp = roundup(p, 32)."""
    for prec, s in ((sp.FP32, 4), (sp.FP64, 8), (sp.MIXED, 4)):
        for n, p in ((200, 2000), (37, 131), (1, 2), (16384, 64)):
            ldn, ldp = (n + 31) // 32 * 32, (p + 31) // 32 * 32
            want = (256 + 2 * _al(p * 8) + _al(p * 4) + 2 * _al(p * 8) + _al(p * s)
                    + _al(ldn * ldp * s) + _al(p * ldn * s) + _al(p * ldp * s))
            assert sp.spmesl_fit_residual_workspace_bytes(n, p, prec) == want, (prec, n, p)
    # no p x p covariance: well below the Gram + fit workspaces of the covariance form
    res = sp.spmesl_fit_residual_workspace_bytes(200, 2000, sp.FP32)
    cov = sp.spmesl_gram_workspace_bytes(200, 2000, sp.FP32) + sp.spmesl_fit_workspace_bytes(2000, sp.FP32)
    assert 3 * res < cov + 4 * 2000 * 2000
    for n, p in ((0, 10), (16385, 10), (10, 1), (-1, 10)):
        assert sp.spmesl_fit_residual_workspace_bytes(n, p, sp.FP32) == 0
    assert sp.spmesl_fit_residual_workspace_bytes(10, 10, 7) == 0


def test_residual_invalid_arguments_rejected_on_host():
    o = sp.spmesl_default_opts()
    fake = 1 << 20        # never dereferenced: validation comes first
    nb = sp.spmesl_fit_residual_workspace_bytes(30, 50, sp.FP32)
    ws = 1 << 24          # 256-byte aligned address, never dereferenced
    ok_args = (fake, 30, 50, 50, 0.2, 1e-6, 100, o, fake, fake, None, ws, nb, 0)

    def call(**kw):
        a = list(ok_args)
        names = ["X", "n", "p", "ldx", "lam", "tol", "maxit", "opts", "T", "sig", "st", "ws", "nb",
                 "stream"]
        for k, v in kw.items():
            a[names.index(k)] = v
        return sp.spmesl_fit_residual(*a)

    assert call(X=None) == sp.SPMESL_EINVAL
    assert call(n=0) == sp.SPMESL_EINVAL
    assert call(n=16385) == sp.SPMESL_EINVAL
    assert call(p=1, ldx=1) == sp.SPMESL_EINVAL
    assert call(ldx=49) == sp.SPMESL_EINVAL
    assert call(lam=-0.2) == sp.SPMESL_EINVAL
    assert call(tol=0.0) == sp.SPMESL_EINVAL
    assert call(maxit=0) == sp.SPMESL_EINVAL
    assert call(ws=ws + 16) == sp.SPMESL_EINVAL          # misaligned workspace
    assert call(nb=nb - 1) == sp.SPMESL_EINVAL           # short workspace
    joint = sp.spmesl_default_opts()
    joint.inner_rule = sp.INNER_JOINT
    assert call(opts=joint) == sp.SPMESL_EINVAL
    bad_prec = sp.spmesl_default_opts()
    bad_prec.precision = 9
    assert call(opts=bad_prec) == sp.SPMESL_EINVAL


def test_every_entry_point_cites_its_passage():
    """Each function's comment block in include/spmesl.h (the text since the
    previous declaration) cites the paper's passage for the operation, or
    states that the paper has no counterpart."""
    cite = re.compile(r"Section|Eqs?\.|Algorithm|Proposition|Table|Theorem|"
                      r"no passage of the paper|paper has no|not in the paper|has no serving")
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        decl = re.compile(r"^(?:spmesl_status|size_t|int|double|void|const char\*)\s+(spmesl_\w+)\s*\(",
                          re.M)
        prev, last = 0, ""
        for m in decl.finditer(text):
            block = text[prev:m.start()]
            if not block.strip():         # declared right after another: shares its comment
                block = last
            assert cite.search(block), m.group(1)
            prev, last = text.index(";", m.end()) + 1, block


def test_noalloc_limits_match_the_fit_workspace():
    """The allocation-free fit's documented limits are the largest p whose fit
    workspace fits its 64 MiB scratch (include/spmesl.h)."""
    cap = 64 << 20
    for prec, limit in ((sp.FP32, 2351), (sp.MIXED, 2351), (sp.FP64, 1664)):
        assert sp.spmesl_fit_workspace_bytes(limit, prec) <= cap
        assert sp.spmesl_fit_workspace_bytes(limit + 1, prec) > cap


def test_aligned_views_layout():
    """Batch keeps every fit's Theta and sigma as views of one buffer each
    (one copy moves a batch's results): every view starts on a 256-byte
    boundary, has its own shape, and no two views overlap."""
    import torch
    shapes = [(3, 3), (50, 50), (1,), (7,), (129, 129), (2, 2)]
    for dtype in (torch.float64, torch.float32):
        buf, views = sp.aligned_views(shapes, dtype, "cpu")
        es = buf.element_size()
        spans = []
        for sh, v in zip(shapes, views):
            assert tuple(v.shape) == sh and v.is_contiguous() and v.dtype == dtype
            off = (v.data_ptr() - buf.data_ptr())
            assert off % 256 == 0
            spans.append((off, off + v.numel() * es))
            assert off + v.numel() * es <= buf.numel() * es
        spans.sort()
        assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))
        # writing through a view lands in the buffer, at the view's place
        buf.zero_()
        views[1].fill_(2.0)
        o = (views[1].data_ptr() - buf.data_ptr()) // es
        assert float(buf.sum()) == 2.0 * 50 * 50 and float(buf[o:o + 2500].sum()) == 5000.0
