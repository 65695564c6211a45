"""The batch tuner's persistent cache (host code, no GPU): keying by class of
batch, storage and reuse, invalidation by library version, malformed files."""
from __future__ import annotations

import json
import os

import pytest

import paper_2203_15031_gb300 as sp



def _choice(w=8, h=32, mp=4096, hh=32, ms=3.5):
    c = sp.TuneChoice()
    c.warps_per_block, c.handover, c.heavy_min_p, c.heavy_heat, c.ms = w, h, mp, hh, ms
    return c


def test_key_buckets_what_the_choice_depends_on():
    k = sp.spmesl_tune_key(sp.MIXED, 1, 152, 256, 1995, 215.3)
    assert k == "prec=2|std=1|sms=152|pmax=2^11|nmean=2^8|fits=2^8"
    # same class: p, n and count within the same power-of-two buckets
    assert sp.spmesl_tune_key(sp.MIXED, 1, 152, 200, 1100, 130.0) == k
    # another class for each component
    others = [sp.spmesl_tune_key(sp.FP32, 1, 152, 256, 1995, 215.3),
              sp.spmesl_tune_key(sp.MIXED, 0, 152, 256, 1995, 215.3),
              sp.spmesl_tune_key(sp.MIXED, 1, 148, 256, 1995, 215.3),
              sp.spmesl_tune_key(sp.MIXED, 1, 152, 257, 1995, 215.3),
              sp.spmesl_tune_key(sp.MIXED, 1, 152, 256, 2049, 215.3),
              sp.spmesl_tune_key(sp.MIXED, 1, 152, 256, 1995, 257.0)]
    assert len(set(others)) == len(others) and k not in others
    with pytest.raises(sp.SpmeslError):
        sp.spmesl_tune_key(sp.MIXED, 1, 0, 256, 1995, 215.3)


def test_store_and_lookup_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    k1 = sp.spmesl_tune_key(sp.MIXED, 1, 152, 256, 1995, 215.3)
    k2 = sp.spmesl_tune_key(sp.FP32, 1, 152, 10, 2000, 200.0)
    rc, _ = sp.spmesl_tune_cache_lookup(path, k1)
    assert rc == sp.SPMESL_ENOTFOUND                      # no file yet
    assert sp.spmesl_tune_cache_store(path, k1, _choice(4, 32, 4096, 32, 3.25)) == sp.SPMESL_OK
    assert sp.spmesl_tune_cache_store(path, k2, _choice(8, 64, -1, 32, 0.5)) == sp.SPMESL_OK
    rc, c = sp.spmesl_tune_cache_lookup(path, k1)
    assert rc == sp.SPMESL_OK and c.from_cache == 1
    assert (c.warps_per_block, c.handover, c.heavy_min_p, c.heavy_heat) == (4, 32, 4096, 32)
    assert c.ms == pytest.approx(3.25)
    rc, c = sp.spmesl_tune_cache_lookup(path, k2)
    assert rc == sp.SPMESL_OK and (c.warps_per_block, c.handover, c.heavy_min_p) == (8, 64, -1)
    # replacing an entry keeps the others; the file is valid JSON
    assert sp.spmesl_tune_cache_store(path, k1, _choice(8, 32, 1024, 32, 3.0)) == sp.SPMESL_OK
    d = json.load(open(path))
    assert d["spmesl_tune_cache"] == 1 and set(d["entries"]) == {k1, k2}
    assert d["entries"][k1]["heavy_min_p"] == 1024
    assert not os.path.exists(path + ".tmp")


def test_entries_of_another_version_are_not_used(tmp_path):
    path = str(tmp_path / "tune.json")
    k = sp.spmesl_tune_key(sp.MIXED, 1, 152, 256, 1995, 215.3)
    assert sp.spmesl_tune_cache_store(path, k, _choice()) == sp.SPMESL_OK
    d = json.load(open(path))
    d["entries"][k]["version"] = "10000/1"                # written by another library version
    json.dump(d, open(path, "w"))
    rc, _ = sp.spmesl_tune_cache_lookup(path, k)
    assert rc == sp.SPMESL_ENOTFOUND
    # storing again replaces it with this version's entry
    assert sp.spmesl_tune_cache_store(path, k, _choice(4)) == sp.SPMESL_OK
    rc, c = sp.spmesl_tune_cache_lookup(path, k)
    assert rc == sp.SPMESL_OK and c.warps_per_block == 4


def test_malformed_files_and_bad_keys(tmp_path):
    path = str(tmp_path / "tune.json")
    k = sp.spmesl_tune_key(sp.FP64, 1, 152, 3, 100, 50.0)
    for text in ("", "not json", '{"spmesl_tune_cache":1,"entries":{"', '{"other":1}'):
        open(path, "w").write(text)
        rc, _ = sp.spmesl_tune_cache_lookup(path, k)
        assert rc == sp.SPMESL_ENOTFOUND
    assert sp.spmesl_tune_cache_store(path, 'bad"key', _choice()) == sp.SPMESL_EINVAL
    # a malformed file is replaced by a valid one on the next store
    assert sp.spmesl_tune_cache_store(path, k, _choice()) == sp.SPMESL_OK
    assert sp.spmesl_tune_cache_lookup(path, k)[0] == sp.SPMESL_OK
    assert sp.spmesl_tune_cache_store(str(tmp_path / "no" / "dir.json"), k, _choice()) == \
        sp.SPMESL_EINVAL
