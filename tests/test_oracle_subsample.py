"""Pins of the oracle's sampled linking length (Sec. 3.2: above 10,000
members the nearest-neighbour distances of a random 10,000-member subset set
the linking length).  The subset of a node is its s members with the
smallest SplitMix64 keys; these tests pin the generator to its published
outputs, the subset to uniformity, and the linking length to an independent
nearest-neighbour routine (scipy's k-d tree) and to the sampling error of a
quantile.  CPU only."""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from paper_1110_4372_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
F = 0.7


def test_splitmix64_published_outputs():
    with open(os.path.join(GOLD, "splitmix64.json")) as fh:
        g = json.load(fh)
    for s in g["streams"]:
        want = [int(v, 0) for v in s["outputs"]]
        # particle i draws the (i+1)-th output of the stream
        assert [oracle.sample_key(s["seed"], i) for i in range(len(want))] == want
        assert oracle.sample_keys(s["seed"], 0, len(want)).tolist() == want


def test_keys_distinct_and_spread():
    k = oracle.sample_keys(20261203, 0, 1 << 21)
    assert len(np.unique(k)) == len(k)  # the finaliser is a bijection
    top = (k >> np.uint64(56)).astype(np.int64)
    h = np.bincount(top, minlength=256)
    e = len(k) / 256
    chi2 = float(((h - e) ** 2 / e).sum())
    assert chi2 < 255 + 8 * math.sqrt(2 * 255)  # 255 degrees of freedom, 8 sigma


def test_subset_inclusion_is_uniform():
    """The s smallest keys of a fixed member set select every member with
    probability s/n over seeds."""
    n, s, seeds = 300, 60, 1500
    mem = (np.arange(n) * 7 + 3).astype(np.int64)
    hits = np.zeros(n, np.int64)
    for seed in range(seeds):
        keys = np.array([oracle.sample_key(seed, int(i)) for i in mem], np.uint64)
        hits[np.argsort(keys)[:s]] += 1
    p = s / n
    sd = math.sqrt(seeds * p * (1 - p))
    assert np.all(np.abs(hits - seeds * p) < 6 * sd)


def _node():
    """One 6000-member node: a host blob with two smaller blobs offset in
    position and velocity."""
    rng = np.random.default_rng(1110)
    box = 20.0
    parts = [synth.blob(rng, 5000, [10, 10, 10], [0, 0, 0], 0.3, 300.0),
             synth.blob(rng, 500, [10.4, 10, 10], [250, 0, 0], 0.05, 60.0),
             synth.blob(rng, 500, [10, 9.7, 10], [0, -200, 0], 0.05, 60.0)]
    pos = synth.wrap(np.vstack([p for p, _ in parts]), box)
    vel = np.vstack([v for _, v in parts]).astype(np.float32)
    n = len(pos)
    return pos, vel, box, np.arange(n, dtype=np.int32), np.array([0, n])


def _norm_coords(pos, vel, mem, box):
    p = pos[mem].astype(np.float64)
    v = vel[mem].astype(np.float64)
    d = p - p[np.argmin(mem)]
    d -= box * np.round(d / box)
    dx = d - d.mean(0)
    dv = v - v.mean(0)
    sx = math.sqrt((dx * dx).sum() / len(mem))
    sv = math.sqrt((dv * dv).sum() / len(mem))
    return np.hstack([d / sx, v / sv])


def _exact_dnn(pos, vel, mem, box):
    u = _norm_coords(pos, vel, mem, box)
    dd, _ = cKDTree(u).query(u, k=2)
    return dd[:, 1]


@pytest.fixture(scope="module")
def node():
    return _node()


def test_sampled_length_is_the_subset_quantile(node):
    pos, vel, box, mem, off = node
    s, seed = 1500, 77
    t = oracle.refine(pos, vel, box, mem, off, sub_n=s, sub_seed=seed)
    for i in range(t.n_nodes):
        m = t.node_members(i)
        dnn = _exact_dnn(pos, vel, m, box)  # neighbours among all members
        if len(m) > s:
            keys = oracle.sample_keys(seed, 0, len(pos))[m]
            sub = np.argsort(keys)[:s]
            want = np.sort(dnn[sub])[math.ceil(F * s) - 1]
        else:
            want = np.sort(dnn)[math.ceil(F * len(m)) - 1]
        assert t.lnk[i] == pytest.approx(want, rel=1e-9), f"node {i} ({len(m)} members)"
    assert t.count[0] > s and np.count_nonzero(t.count > s) >= 2  # root and a child sampled


def test_subset_at_least_node_size_is_exact(node):
    pos, vel, box, mem, off = node
    a = oracle.refine(pos, vel, box, mem, off)
    for s in (len(mem), 10 * len(mem)):
        b = oracle.refine(pos, vel, box, mem, off, sub_n=s, sub_seed=5)
        assert b.n_nodes == a.n_nodes
        assert np.array_equal(b.members, a.members)
        assert np.array_equal(b.lnk, a.lnk)


def test_sampled_length_within_quantile_error(node):
    """The subset's k-th value sits, among all members' exact values, at a
    rank within the sampling error of the f-quantile (hypergeometric: sd =
    n sqrt(f(1-f)/s (1-s/n))), and different seeds draw different subsets."""
    pos, vel, box, mem, off = node
    n = len(mem)
    dnn = np.sort(_exact_dnn(pos, vel, mem, box))
    exact = dnn[math.ceil(F * n) - 1]
    s = 1500
    sd = n * math.sqrt(F * (1 - F) / s * (1 - s / n))
    seen = set()
    for seed in range(6):
        t = oracle.refine(pos, vel, box, mem, off, sub_n=s, sub_seed=seed)
        l = t.lnk[0]
        rank = np.searchsorted(dnn, l * (1 + 1e-12), side="right")
        assert abs(rank - F * n) < 6 * sd + 1
        assert abs(l / exact - 1) < 0.1
        seen.add(float(l))
    assert len(seen) > 1


def test_sampled_tree_children_are_components(node):
    """The subset only sets l: the links are still every pair within l, so
    no pair within a node's l joins two different children or a child and
    the rest (Sec. 3.2)."""
    pos, vel, box, mem, off = node
    t = oracle.refine(pos, vel, box, mem, off, sub_n=1500, sub_seed=3)
    for i in range(t.n_nodes):
        if t.count[i] <= 1500:
            continue
        kids = np.flatnonzero(t.parent == i)
        m = t.node_members(i)
        u = _norm_coords(pos, vel, m, box)
        pairs = cKDTree(u).query_pairs(t.lnk[i] * (1 + 1e-9), output_type="ndarray")
        which = np.full(len(m), -1)
        for kk, k in enumerate(kids):
            which[np.isin(m, t.node_members(k))] = kk
        cross = (which[pairs[:, 0]] != which[pairs[:, 1]]) & ((which[pairs[:, 0]] >= 0) | (which[pairs[:, 1]] >= 0))
        assert not cross.any()
