"""Pins of the oracle's accelerated 3D FOF (Sec. 3.1): a particle with more
than 16 neighbours within l joins everything within 2l, and its neighbours
skip their own search.  Visiting particles in index order, the result has a
closed form that involves no skipping: with "centres" the dense particles
(more than 16 neighbours) that have no earlier centre within l -- the
index-greedy maximal independent set of the dense particles -- the groups are
the connected components of the plain FOF graph plus an edge from every
centre to every particle within 2l of it.  (A skipped particle lies within l
of a centre, so each of its FOF edges ends within 2l of that centre.)  The
tests compare the oracle with that closed form computed by brute force, check
the paper's statement that the groups are unions of plain FOF groups, and
work small cases by hand.  CPU only."""
import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

import oracle
from paper_1110_4372_gb300 import synth


def _d2(pos, box):
    p = np.asarray(pos, np.float64)
    d = p[:, None, :] - p[None, :, :]
    d -= box * np.round(d / box)
    return (d * d).sum(-1)


def _components(n, i, j):
    g = coo_matrix((np.ones(len(i)), (i, j)), shape=(n, n))
    nc, lab = connected_components(g, directed=False)
    mins = np.full(nc, n)
    np.minimum.at(mins, lab, np.arange(n))
    return mins[lab].astype(np.int32)


def closed_form(pos, box, l, dense_n=16):
    n = len(pos)
    d2 = _d2(pos, box)
    near = d2 <= l * l
    np.fill_diagonal(near, False)
    dense = near.sum(1) > dense_n
    centre = np.zeros(n, bool)
    for c in np.flatnonzero(dense):  # increasing index
        if not (near[c] & centre).any():
            centre[c] = True
    i, j = np.nonzero(np.triu(near, 1))
    ci, cj = np.nonzero((d2 <= (2 * l) ** 2) & centre[:, None])
    return _components(n, np.concatenate([i, ci]), np.concatenate([j, cj])), int(centre.sum())


def _is_union_of(coarse, fine):
    """Every group of `fine` lies inside one group of `coarse`."""
    for g in np.unique(fine):
        if len(np.unique(coarse[fine == g])) != 1:
            return False
    return True


@pytest.mark.parametrize("seed", [4, 5, 6])
def test_clustered_vs_closed_form(seed):
    n = 2500
    box = 10.0 * (n / 32768) ** (1 / 3)
    c = synth.generate("c1", seed=seed, n=n, box=box, n_halos=6)
    lab, l, nc = oracle.fof3d_accel(c.pos, c.box, 0.28)
    ref, nref = closed_form(c.pos, c.box, l)
    assert np.array_equal(lab, ref)
    assert nc == nref and nc > 0
    plain, _, _ = oracle.fof3d(c.pos, c.box, l=l)
    assert _is_union_of(lab, plain)


@pytest.mark.parametrize("dense_n", [0, 3, 8, 16])
def test_uniform_dense_vs_closed_form(dense_n):
    c = synth.uniform(1500, 10.0, 30 + dense_n)
    l = oracle.linking_length(1500, 10.0, 0.9)
    lab, _, nc = oracle.fof3d_accel(c.pos, c.box, l=l, dense_n=dense_n)
    ref, nref = closed_form(c.pos, c.box, l, dense_n)
    assert np.array_equal(lab, ref) and nc == nref


def test_sparse_equals_plain():
    """No particle with more than 16 neighbours: plain FOF exactly."""
    c = synth.uniform(3000, 10.0, 7)
    l = oracle.linking_length(3000, 10.0, 0.28)
    lab, _, nc = oracle.fof3d_accel(c.pos, c.box, l=l)
    plain, _, _ = oracle.fof3d(c.pos, c.box, l=l)
    assert nc == 0 and np.array_equal(lab, plain)


def test_huge_threshold_equals_plain():
    n = 2000
    box = 10.0 * (n / 32768) ** (1 / 3)
    c = synth.generate("c1", seed=9, n=n, box=box, n_halos=6)
    lab, l, nc = oracle.fof3d_accel(c.pos, c.box, 0.28, dense_n=n)
    plain, _, _ = oracle.fof3d(c.pos, c.box, l=l)
    assert nc == 0 and np.array_equal(lab, plain)


def _clump(k, centre, radius, rng):
    """k points within `radius` of centre, the first exactly at it."""
    v = rng.standard_normal((k, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    r = radius * rng.random(k)[:, None]
    p = centre + v * r
    p[0] = centre
    return p


@pytest.mark.parametrize("k,sat,joined", [(18, 1.5, True), (18, 2.5, False), (17, 1.5, False)])
def test_hand_clump_and_satellite(k, sat, joined):
    """Particle 0 has k-1 neighbours in a tight clump: with more than 16 it
    searches 2l, so a satellite at 1.5 l joins; at 2.5 l it stays alone; with
    exactly 16 neighbours there is no 2l search."""
    rng = np.random.default_rng(k)
    l, box = 1.0, 20.0
    pos = np.vstack([_clump(k, np.array([10.0, 10, 10]), 0.05, rng), [[10.0 + sat, 10, 10]]])
    pos = synth.wrap(pos, box)
    lab, _, nc = oracle.fof3d_accel(pos, box, l=l)
    plain, _, _ = oracle.fof3d(pos, box, l=l)
    assert plain[-1] == k  # alone in plain FOF
    assert (lab[-1] == 0) == joined
    assert nc == (1 if k - 1 > 16 else 0)


def test_hand_skip_depends_on_order():
    """A dense particle inside the first centre's l-ball is skipped, so its
    own 2l ball (which would reach a far satellite) is never searched -- but
    if it is visited first it becomes the centre and the satellite joins."""
    rng = np.random.default_rng(2)
    l, box = 1.0, 20.0
    clump = _clump(18, np.array([10.0, 10, 10]), 0.05, rng)  # particle 0 at the centre
    k = np.array([[10.9, 10, 10]])     # within l of the whole clump: dense
    t = np.array([[12.7, 10, 10]])     # 1.8 l from k, 2.7 l from particle 0
    first = synth.wrap(np.vstack([clump, k, t]), box)
    lab, _, nc = oracle.fof3d_accel(first, box, l=l)
    assert nc == 1 and lab[18] == 0 and lab[19] == 19
    second = synth.wrap(np.vstack([k, clump, t]), box)
    lab2, _, nc2 = oracle.fof3d_accel(second, box, l=l)
    assert nc2 == 1 and np.all(lab2 == 0)
    for p, lb in ((first, lab), (second, lab2)):
        assert np.array_equal(lb, closed_form(p, box, l)[0])


def test_across_the_periodic_boundary():
    """The 2l search wraps around the box like the plain one."""
    rng = np.random.default_rng(3)
    l, box = 1.0, 20.0
    pos = np.vstack([_clump(18, np.array([0.2, 10, 10]), 0.05, rng), [[box - 1.3, 10, 10]]])
    pos = synth.wrap(pos, box)
    lab, _, nc = oracle.fof3d_accel(pos, box, l=l)
    assert nc == 1 and lab[-1] == 0


def test_empty_single_and_threshold_zero():
    lab, _, nc = oracle.fof3d_accel(np.zeros((0, 3), np.float32), 10.0, l=1.0)
    assert len(lab) == 0 and nc == 0
    lab, _, nc = oracle.fof3d_accel(np.array([[1, 2, 3]], np.float32), 10.0, l=1.0)
    assert list(lab) == [0] and nc == 0
    # with dense_n = 0 any particle with a neighbour is dense: particle 0 (one
    # neighbour at 0.5) joins particle 2, 1.2 away across the face, at 2l = 1.2
    p = np.array([[1.0, 1, 1], [1.5, 1, 1], [9.75, 1, 1]], np.float32)
    lab, _, nc = oracle.fof3d_accel(p, 10.0, l=0.65, dense_n=0)
    assert list(lab) == [0, 0, 0] and nc == 1
    assert np.array_equal(lab, closed_form(p, 10.0, 0.65, 0)[0])
    plain, _, _ = oracle.fof3d(p, 10.0, l=0.65)
    assert list(plain) == [0, 0, 2]
