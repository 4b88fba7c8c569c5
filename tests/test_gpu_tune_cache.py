"""Tuner cache (environment variable DEMAG_TUNE_CACHE).

A tuned plan's choices (p, leaf size, M2L launch shape) are appended to the
file under a key that hashes the mesh, the options and the device; a second
plan of the same mesh and options is built from them without timing and is the
same plan (identical statistics, bit-identical results).  A different theta or
a moved node is another key; lines that do not parse or hold values out of
range are skipped, the last valid line of a key wins, and a file that cannot
be written leaves a warning but not a failure.
"""
import pytest
import torch

from paper_1606_00247_gb300 import inputs

pytestmark = pytest.mark.gpu

KW = dict(p=8, leaf_size=32, max_batch=128, near_mode=1, precision="bf16x3", autotune=3)
SAME = ("p", "leaf_size", "m2l_kps", "m2l_ring_bytes", "m2l_targets_per_cta", "n_cells", "n_m2l", "n_near_tiles")


def _plan(nodes, tets, **kw):
    from paper_1606_00247_gb300.api import Plan

    return Plan(nodes, tets, **kw)


def _entries(path):
    return [ln.split() for ln in path.read_text().splitlines() if ln.strip()]


def test_tuned_choices_are_cached_and_reused(tmp_path, monkeypatch):
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("DEMAG_TUNE_CACHE", str(path))
    nodes, tets = inputs.sphere(h=0.13)
    M = inputs.gaussian_unit_m(nodes.shape[0], batch=128, seed=97)
    a = _plan(nodes, tets, **KW)
    sa = a.stats()
    assert sa["tune_source"] == 1 and sa["n_m2l_ops"] > 0
    (e,) = _entries(path)
    assert e[:2] == ["demag-tune", "1"] and len(e[2]) == 16
    assert [int(v) for v in e[3:]] == [sa["p"], sa["leaf_size"], sa["m2l_targets_per_cta"], sa["m2l_kps"],
                                       sa["m2l_ring_bytes"]]
    b = _plan(nodes, tets, **KW)
    sb = b.stats()
    assert sb["tune_source"] == 2
    assert all(sa[k] == sb[k] for k in SAME), {k: (sa[k], sb[k]) for k in SAME}
    assert len(_entries(path)) == 1  # a hit appends nothing
    ua, Ha = a.eval(M)
    ub, Hb = b.eval(M)
    assert torch.equal(ua, ub) and torch.equal(Ha, Hb)

    # another theta, or one node moved, is another key: tuned again and appended
    c = _plan(nodes, tets, **dict(KW, theta=0.45))
    assert c.stats()["tune_source"] == 1 and len(_entries(path)) == 2
    moved = nodes.copy()
    moved[0, 0] += 1e-9
    d = _plan(moved, tets, **KW)
    assert d.stats()["tune_source"] == 1 and len(_entries(path)) == 3
    for pl in (a, b, c, d):
        pl.close()


def test_cache_lines_are_validated_and_the_last_valid_one_wins(tmp_path, monkeypatch):
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("DEMAG_TUNE_CACHE", str(path))
    nodes, tets = inputs.sphere(h=0.2)
    kw = dict(p=6, leaf_size=32, max_batch=2, near_mode=1, precision="fp32", autotune=6)
    a = _plan(nodes, tets, **kw)
    sa = a.stats()
    assert sa["tune_source"] == 1
    (e,) = _entries(path)
    key = e[2]
    p_other = 4 if sa["p"] != 4 else 6
    leaf_other = 16 if sa["leaf_size"] != 16 else 64
    with open(path, "a") as f:
        f.write("not a cache line\n")
        f.write(f"demag-tune 1 {key} {p_other} 0 1 0 0\n")  # leaf 0: out of range, skipped
        f.write(f"demag-tune 2 {key} {p_other} {leaf_other} 1 0 0\n")  # another format version, skipped
        f.write(f"demag-tune 1 {key} {p_other} {leaf_other} 1 0 0\n")  # the last valid line of the key
    b = _plan(nodes, tets, **kw)
    sb = b.stats()
    assert sb["tune_source"] == 2 and (sb["p"], sb["leaf_size"]) == (p_other, leaf_other)
    M = inputs.gaussian_unit_m(nodes.shape[0], batch=2, seed=98)
    ub, Hb = b.eval(M)
    uc, Hc = _plan(nodes, tets, **dict(kw, p=p_other, leaf_size=leaf_other, autotune=0)).eval(M)
    assert torch.equal(ub, uc) and torch.equal(Hb, Hc)


def test_no_tuning_no_cache_and_unwritable_cache(tmp_path, monkeypatch):
    from paper_1606_00247_gb300 import _lib

    nodes, tets = inputs.sphere(h=0.2)
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("DEMAG_TUNE_CACHE", str(path))
    pl = _plan(nodes, tets, p=6, leaf_size=32, max_batch=2, near_mode=1, precision="fp32")
    assert pl.stats()["tune_source"] == 0 and not path.exists()
    monkeypatch.setenv("DEMAG_TUNE_CACHE", str(tmp_path))  # a directory: cannot be opened for appending
    pt = _plan(nodes, tets, p=6, leaf_size=32, max_batch=2, near_mode=1, precision="fp32", autotune=2)
    assert pt.stats()["tune_source"] == 1
    assert "tuner cache" in _lib.demag_last_error()
