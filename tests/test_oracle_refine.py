"""Pins of the oracle's phase-space hierarchy (Sec. 3.2, Eq. 1): hand-worked
cases, an independent nearest-neighbour routine (scipy's k-d tree), the
exact-fraction invariant, exact invariances and the co-spatial merger idea of
Sec. 2.2 / Fig. 2.  CPU only."""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from paper_1110_4372_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


def tree_signature(t):
    """Node set keyed by (level, smallest member), value = sorted members."""
    return {(int(t.level[i]), int(t.minidx[i])): tuple(sorted(t.node_members(i).tolist()))
            for i in range(t.n_nodes)}


@pytest.mark.parametrize("case", load("hand_moments.json")["cases"], ids=lambda c: c["name"])
def test_hand_moments(case):
    pos = np.array(case["pos"], np.float32)
    vel = np.array(case["vel"], np.float32)
    m = oracle.moments(pos, vel, np.arange(len(pos)), case["box"])
    assert m["sigx"] == pytest.approx(case["sigx"], rel=1e-15)
    assert m["sigv"] == pytest.approx(case["sigv"], rel=1e-15)
    assert np.allclose(m["xbar"], case["xbar"], rtol=0, atol=1e-14)
    assert np.allclose(m["vbar"], case["vbar"], rtol=0, atol=1e-14)


def test_hand_hierarchy():
    g = load("hand_hierarchy.json")
    pos = np.array(g["pos"], np.float32)
    vel = np.array(g["vel"], np.float32)
    n = len(pos)
    t = oracle.refine(pos, vel, g["box"], np.arange(n, dtype=np.int32), np.array([0, n]), g["f"], g["min_n"])
    got = {tuple(sorted(t.node_members(i).tolist())): i for i in range(t.n_nodes)}
    assert len(got) == len(g["expect"]["nodes"])
    for e in g["expect"]["nodes"]:
        i = got[tuple(e["members"])]
        assert t.level[i] == e["level"]
        assert (t.nchild[i] == 0) == e["leaf"]
        assert t.lnk[i] * t.sigx[i] == pytest.approx(e["lnk_times_sigx"], rel=1e-12)
        assert t.sigv[i] == 0.0


def _norm_coords(pos, vel, mem, box):
    """Unwrapped, dispersion-normalised 6D coordinates (numpy, two-pass)."""
    p = pos[mem].astype(np.float64)
    v = vel[mem].astype(np.float64)
    ref = p[np.argmin(mem)]
    d = p - ref
    d -= box * np.round(d / box)
    dx = d - d.mean(0)
    dv = v - v.mean(0)
    sx = math.sqrt((dx * dx).sum() / len(mem))
    sv = math.sqrt((dv * dv).sum() / len(mem))
    return np.hstack([d / sx, v / sv])


@pytest.mark.parametrize("n", [12, 100, 700, 2500])
def test_nn_distances_vs_scipy(n):
    c = synth.generate("c1", seed=20 + n)
    lab, l, _ = oracle.fof3d(c.pos, c.box)
    # a real group plus random background members to vary the shape
    g = np.bincount(lab).argmax()
    mem = np.flatnonzero(lab == g)
    rng = np.random.default_rng(n)
    if len(mem) < n:
        extra = rng.choice(np.setdiff1d(np.arange(c.n), mem), n - len(mem), replace=False)
        # keep them near the group so the unwrapped extent stays below box/2
        mem = np.concatenate([mem, extra])
        pos = c.pos.copy()
        centre = pos[mem[0]]
        pos[extra] = np.mod(centre + (pos[extra] - centre) * 0.2, c.box).astype(np.float32)
    else:
        pos = c.pos
        mem = mem[:n]
    mem = np.sort(mem).astype(np.int32)
    dnn2, l2, _ = oracle.node_dnn(pos, c.vel, mem, c.box, 0.7)
    u = _norm_coords(pos, c.vel, mem, c.box)
    dd, _ = cKDTree(u).query(u, k=2)
    assert np.allclose(np.sqrt(dnn2), dd[:, 1], rtol=1e-9, atol=0)
    k = math.ceil(0.7 * len(mem))
    assert l2 == pytest.approx(np.sort(dd[:, 1])[k - 1] ** 2, rel=1e-9)


def test_kd_path_equals_brute_path():
    c = synth.generate("c1")
    lab, l, _ = oracle.fof3d(c.pos, c.box)
    mem, off = oracle.groups_from_labels(lab, 10)
    a = oracle.refine(c.pos, c.vel, c.box, mem, off, kd_threshold=1 << 30)
    b = oracle.refine(c.pos, c.vel, c.box, mem, off, kd_threshold=16)
    assert tree_signature(a) == tree_signature(b)
    sa = {(int(a.level[i]), int(a.minidx[i])): a.lnk[i] for i in range(a.n_nodes)}
    for i in range(b.n_nodes):
        assert b.lnk[i] == pytest.approx(sa[(int(b.level[i]), int(b.minidx[i]))], rel=1e-12)


@pytest.fixture(scope="module")
def c1_tree():
    c = synth.generate("c1")
    lab, l, _ = oracle.fof3d(c.pos, c.box)
    mem, off = oracle.groups_from_labels(lab, 10)
    t = oracle.refine(c.pos, c.vel, c.box, mem, off)
    return c, lab, mem, off, t


def test_exact_fraction_invariant(c1_tree):
    """Sec. 3.2: the linking length links a fraction f -- with k = ceil(f n),
    at least k members have their nearest neighbour within l and fewer than
    k strictly inside it (nearest neighbours from scipy's k-d tree)."""
    c, _, _, _, t = c1_tree
    for i in range(t.n_nodes):
        mem = t.node_members(i)
        u = _norm_coords(c.pos, c.vel, mem, c.box)
        dd, _ = cKDTree(u).query(u, k=2)
        dnn = dd[:, 1]
        k = math.ceil(0.7 * len(mem))
        lnk = t.lnk[i]
        assert np.count_nonzero(dnn <= lnk * (1 + 1e-9)) >= k
        assert np.count_nonzero(dnn < lnk * (1 - 1e-9)) < k


def test_structure(c1_tree):
    c, lab, mem, off, t = c1_tree
    # roots are exactly the 3D groups with >= min_n members
    roots = np.flatnonzero(t.parent < 0)
    assert len(roots) == len(off) - 1
    for i in range(t.n_nodes):
        p = t.parent[i]
        if p >= 0:
            assert t.level[i] == t.level[p] + 1
            assert 10 <= t.count[i] < t.count[p]
            assert t.first[p] <= t.first[i] and t.first[i] + t.count[i] <= t.first[p] + t.count[p]
        # children's particles sit at the front of the parent's range
    for i in range(t.n_nodes):
        kids = np.flatnonzero(t.parent == i)
        assert len(kids) == t.nchild[i]
        if len(kids):
            span = t.count[kids].sum()
            cover = np.sort(np.concatenate([t.node_members(k) for k in kids]))
            assert np.array_equal(cover, np.sort(t.members[t.first[i]:t.first[i] + span]))
    # members of the same child are linked in 6D at the parent's length, and
    # no child has a friend outside it (components, Sec. 3.2)
    for i in range(min(t.n_nodes, 40)):
        kids = np.flatnonzero(t.parent == i)
        memi = t.node_members(i)
        u = _norm_coords(c.pos, c.vel, memi, c.box)
        tree = cKDTree(u)
        pairs = tree.query_pairs(t.lnk[i] * (1 + 1e-9), output_type="ndarray")
        which = np.full(len(memi), -1)
        for kk, k in enumerate(kids):
            which[np.isin(memi, t.node_members(k))] = kk
        for a, b in pairs:
            if which[a] >= 0 or which[b] >= 0:
                assert which[a] == which[b]


def test_scale_and_boost_invariance():
    """Eq. 1 normalises by the group's own dispersions: doubling all
    velocities, doubling positions with the box, boosting every velocity by
    the same vector or permuting axes leaves every partition unchanged
    (inputs chosen so the transformed float32 values are exact)."""
    c = synth.generate("c1")
    q = 1.0 / 256
    vel = (np.round(c.vel / q) * q).astype(np.float32)
    pos = c.pos
    lab, l, _ = oracle.fof3d(pos, c.box)
    mem, off = oracle.groups_from_labels(lab, 10)
    base = tree_signature(oracle.refine(pos, vel, c.box, mem, off))
    assert tree_signature(oracle.refine(pos, vel * 2, c.box, mem, off)) == base
    assert tree_signature(oracle.refine(pos * 2, vel, c.box * 2, mem, off)) == base
    boost = np.array([512.0, -1000.0, 37.5], np.float32)
    assert tree_signature(oracle.refine(pos, vel + boost, c.box, mem, off)) == base
    perm = [2, 0, 1]
    assert tree_signature(oracle.refine(pos[:, perm].copy(), vel[:, perm].copy(), c.box, mem, off)) == base
    assert tree_signature(oracle.refine(pos, -vel, c.box, mem, off)) == base


def test_particle_order_invariance():
    n = 4000
    c = synth.generate("c1", seed=33, n=n, box=10.0 * (n / 32768) ** (1 / 3), n_halos=5)
    lab, l, _ = oracle.fof3d(c.pos, c.box)
    mem, off = oracle.groups_from_labels(lab, 10)
    t0 = oracle.refine(c.pos, c.vel, c.box, mem, off)
    perm = np.random.default_rng(2).permutation(n)
    inv = np.argsort(perm)
    lab1, _, _ = oracle.fof3d(c.pos[perm], c.box, l=l)
    mem1, off1 = oracle.groups_from_labels(lab1, 10)
    t1 = oracle.refine(c.pos[perm], c.vel[perm], c.box, mem1, off1)
    s0 = {(lv, tuple(sorted(m))) for (lv, _), m in tree_signature(t0).items()}
    s1 = {(lv, tuple(sorted(perm[list(m)].tolist()))) for (lv, _), m in tree_signature(t1).items()}
    assert s0 == s1
    assert inv is not None


def test_cospatial_blobs_split_in_6d():
    """Sec. 2.2 and Fig. 2: two halos at the same place moving apart are one
    group in position space but separate in phase space."""
    rng = np.random.default_rng(11)
    box = 20.0
    n1 = n2 = 600
    p1, v1 = synth.blob(rng, n1, [10, 10, 10], [0, 0, 0], 0.08, 40.0)
    p2, v2 = synth.blob(rng, n2, [10, 10, 10], [240, 0, 0], 0.08, 40.0)
    pos = synth.wrap(np.vstack([p1, p2]), box)
    vel = np.vstack([v1, v2]).astype(np.float32)
    lab, l, _ = oracle.fof3d(pos, box, l=0.05)
    sizes = np.bincount(lab)
    assert sizes.max() >= 0.95 * (n1 + n2)  # one 3D group
    mem, off = oracle.groups_from_labels(lab, 10)
    t = oracle.refine(pos, vel, box, mem, off)
    # the root splits into subgroups that each hold one blob, and both blobs
    # carry seeds; every seed is pure
    kids = np.flatnonzero(t.parent == 0)
    frac = [np.mean(t.node_members(k) < n1) for k in kids]
    assert max(frac) >= 0.95 and min(frac) <= 0.05
    leaves = [i for i in range(t.n_nodes) if t.nchild[i] == 0]
    lfrac = [np.mean(t.node_members(i) < n1) for i in leaves]
    assert all(f >= 0.95 or f <= 0.05 for f in lfrac)
    assert any(f >= 0.95 for f in lfrac) and any(f <= 0.05 for f in lfrac)
    # without the velocity separation the same positions give no such split
    vel0 = np.vstack([v1, v2 - np.array([240.0, 0, 0])]).astype(np.float32)
    t0 = oracle.refine(pos, vel0, box, mem, off)
    kids0 = np.flatnonzero(t0.parent == 0)
    frac0 = [np.mean(t0.node_members(k) < n1) for k in kids0]
    assert all(0.2 < f < 0.8 for f in frac0 if t0.count[kids0[0]] > 100)


def test_degenerate_identical_points():
    pos = np.tile(np.array([[1, 2, 3]], np.float32), (25, 1))
    vel = np.tile(np.array([[4, 5, 6]], np.float32), (25, 1))
    t = oracle.refine(pos, vel, 10.0, np.arange(25, dtype=np.int32), np.array([0, 25]))
    assert t.n_nodes == 1 and t.nchild[0] == 0 and t.lnk[0] == 0.0
    assert t.sigx[0] == 0.0 and t.sigv[0] == 0.0


def test_small_groups_not_refined():
    pos = np.random.default_rng(0).random((9, 3)).astype(np.float32)
    vel = np.zeros((9, 3), np.float32)
    t = oracle.refine(pos, vel, 10.0, np.arange(9, dtype=np.int32), np.array([0, 9]))
    assert t.n_nodes == 0


def test_f_sweep_monotone_seeds(c1_tree):
    """Sec. 3.2 / 4.5: a larger f keeps more particles per level, finding at
    least as many seeds (qualitative; reported on the same input)."""
    c, lab, mem, off, _ = c1_tree
    counts = []
    for f in (0.5, 0.7, 0.9):
        t = oracle.refine(c.pos, c.vel, c.box, mem, off, f=f)
        counts.append(int((t.nchild == 0).sum()))
    assert counts[0] <= counts[2]
