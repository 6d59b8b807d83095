"""The oracle addresses particles by 64-bit offsets: a group whose members
sit above index 2^31 / 3 (the 1.07B-particle workload has them) gives the
same hierarchy, moments and r_dyn as the same particles at small indices.
The large arrays are zero-filled lazily, so only the pages the group uses
are touched.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1110_4372_gb300 import synth

BASE = 716_000_000  # 3 * BASE > 2^31 - 1


def _big_zeros(n):
    try:
        return np.zeros((n, 3), np.float32)
    except MemoryError:
        pytest.skip("no address space for a lazily zeroed array of this size")


def test_group_above_2_31_over_3():
    rng = np.random.default_rng(7)
    k = 600
    box = 100.0
    pos_s = np.empty((k, 3), np.float32)
    vel_s = np.empty((k, 3), np.float32)
    # two offset blobs in phase space: a hierarchy with children
    for half, (c, v) in enumerate([((50.0, 50.0, 50.0), (0.0, 0.0, 0.0)), ((50.6, 50.0, 50.0), (300.0, 0.0, 0.0))]):
        sl = slice(half * k // 2, (half + 1) * k // 2)
        pos_s[sl] = synth.wrap(np.asarray(c) + rng.normal(0.0, 0.15, (k // 2, 3)), box)
        vel_s[sl] = (np.asarray(v) + rng.normal(0.0, 40.0, (k // 2, 3))).astype(np.float32)
    n_big = BASE + k + 8
    pos_b, vel_b = _big_zeros(n_big), _big_zeros(n_big)
    pos_b[BASE:BASE + k] = pos_s
    vel_b[BASE:BASE + k] = vel_s
    mem_s = np.arange(k, dtype=np.int32)
    mem_b = (BASE + mem_s).astype(np.int32)

    ms, mb = oracle.moments(pos_s, vel_s, mem_s, box), oracle.moments(pos_b, vel_b, mem_b, box)
    for key in ("sigx", "sigv"):
        assert ms[key] == mb[key]
    assert np.array_equal(ms["xbar"], mb["xbar"]) and np.array_equal(ms["vbar"], mb["vbar"])
    assert oracle.rdyn2(pos_s, mem_s, box, ms["xbar"], 360.0, 1.0) == \
        oracle.rdyn2(pos_b, mem_b, box, mb["xbar"], 360.0, 1.0)

    ts = oracle.refine(pos_s, vel_s, box, mem_s, np.array([0, k]))
    tb = oracle.refine(pos_b, vel_b, box, mem_b, np.array([0, k]))
    assert ts.n_nodes == tb.n_nodes > 1
    for key in ("parent", "level", "count", "nchild", "tie"):
        assert np.array_equal(getattr(ts, key), getattr(tb, key)), key
    for key in ("lnk", "sigx", "sigv", "xbar", "vbar"):
        assert np.array_equal(getattr(ts, key), getattr(tb, key)), key
    assert np.array_equal(ts.minidx + BASE, tb.minidx)
    assert np.array_equal(ts.members + BASE, tb.members)
    ts.free()
    tb.free()
