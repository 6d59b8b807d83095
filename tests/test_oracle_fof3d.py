"""Pins of the oracle's 3D friends-of-friends (Sec. 3.1) against brute force,
closed forms and exact invariances.  CPU only."""
import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

import oracle
from paper_1110_4372_gb300 import synth


def brute_labels(pos, box, l):
    """All pairs at periodic distance <= l; components by scipy; label =
    smallest member index."""
    p = np.asarray(pos, np.float64)
    n = len(p)
    d = p[:, None, :] - p[None, :, :]
    d -= box * np.round(d / box)
    d2 = (d * d).sum(-1)
    i, j = np.nonzero(np.triu(d2 <= l * l, 1))
    g = coo_matrix((np.ones(len(i)), (i, j)), shape=(n, n))
    nc, lab = connected_components(g, directed=False)
    mins = np.full(nc, n)
    np.minimum.at(mins, lab, np.arange(n))
    return mins[lab].astype(np.int32)


def brute_tieband(pos, box, l):
    p = np.asarray(pos, np.float64)
    d = p[:, None, :] - p[None, :, :]
    d -= box * np.round(d / box)
    dist = np.sqrt((d * d).sum(-1))
    iu = np.triu_indices(len(p), 1)
    return int(np.count_nonzero(np.abs(dist[iu] - l) <= 1e-6 * l))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_uniform_vs_brute(seed):
    c = synth.uniform(1500, 10.0, seed)
    l = oracle.linking_length(1500, 10.0, 0.6)  # dense enough for large groups
    lab, _, _ = oracle.fof3d(c.pos, c.box, l=l)
    ref = brute_labels(c.pos, c.box, l)
    assert np.array_equal(lab, ref)
    assert len(np.unique(lab)) < 1400  # non-trivial grouping


@pytest.mark.parametrize("seed", [4, 5])
def test_clustered_vs_brute(seed):
    n = 2000
    box = 10.0 * (n / 32768) ** (1 / 3)
    c = synth.generate("c1", seed=seed, n=n, box=box, n_halos=6)
    lab, l, _ = oracle.fof3d(c.pos, c.box, 0.28)
    assert np.array_equal(lab, brute_labels(c.pos, c.box, l))
    assert np.bincount(lab).max() >= 20


def test_periodic_faces_edges_corners():
    box = 10.0
    l = 0.5
    eps = np.float32(0.1)
    far = np.float32(box) - np.float32(0.15)
    pts = []
    # straddling a face, an edge and a corner: each pair is 0.25 apart per
    # crossed axis through the boundary
    pts += [[eps, 5, 5], [far, 5, 5]]
    pts += [[eps, eps, 3], [far, far, 3]]
    pts += [[eps, eps, eps], [far, far, far]]
    # a pair that is close only in the direct (non-periodic) sense is far apart
    pts += [[4.0, 8.0, 8.0], [4.6, 8.0, 8.0]]
    pos = np.array(pts, np.float32)
    lab, _, _ = oracle.fof3d(pos, box, l=l)
    assert lab[1] == 0 and lab[3] == 2 and lab[5] == 4
    assert lab[7] == 7 and lab[6] == 6
    assert np.array_equal(lab, brute_labels(pos, box, l))


def test_lattice_closed_form():
    a, m = 1.0, 8
    g = (np.arange(m) + 0.5) * a
    pos = np.array(np.meshgrid(g, g, g, indexing="ij"), np.float32).reshape(3, -1).T.copy()
    box = m * a
    lab, _, _ = oracle.fof3d(pos, box, l=a * (1 + 1e-3))
    assert np.all(lab == 0)
    lab, _, _ = oracle.fof3d(pos, box, l=a * (1 - 1e-3))
    assert np.array_equal(lab, np.arange(len(pos)))
    # diagonal neighbours need sqrt(2) a
    lab, _, _ = oracle.fof3d(pos[::2].copy(), box, l=a * (1 - 1e-3))
    assert len(np.unique(lab)) == len(pos[::2])


def test_translation_exact():
    rng = np.random.default_rng(7)
    box = 8.0
    q = 2.0 ** -10
    pos = (rng.integers(0, int(box / q), size=(1200, 3)) * q).astype(np.float32)
    l = 0.55
    lab0, _, _ = oracle.fof3d(pos, box, l=l)
    for shift in ([3 * q, 0, 0], [box / 2, box / 4, 1000 * q], [7.5, 7.75, 0.25]):
        p2 = np.mod(pos.astype(np.float64) + np.array(shift), box).astype(np.float32)
        lab, _, _ = oracle.fof3d(p2, box, l=l)
        assert np.array_equal(lab, lab0)


def test_permutation_invariance():
    c = synth.generate("c1", seed=9, n=3000, box=10.0 * (3000 / 32768) ** (1 / 3), n_halos=8)
    lab0, l, _ = oracle.fof3d(c.pos, c.box)
    perm = np.random.default_rng(1).permutation(c.n)
    lab1, _, _ = oracle.fof3d(c.pos[perm], c.box, l=l)
    # same partition: particle perm[a] and perm[b] share a group iff a, b do
    back = perm[lab1]  # smallest new index -> old particle id
    # canonicalise old-id labels by component minimum
    mins = {}
    for a in range(c.n):
        mins.setdefault(back[a], []).append(perm[a])
    canon = np.empty(c.n, np.int64)
    for k, v in mins.items():
        canon[np.array(v)] = min(v)
    assert np.array_equal(canon, lab0)


def test_tieband_count():
    box, l = 10.0, 0.5
    pos = np.array([[1, 1, 1], [1 + l * (1 + 4e-7), 1, 1],
                    [3, 3, 3], [3, 3 + l * (1 - 4e-7), 3],
                    [6, 6, 6], [6, 6, 6 + l * (1 + 5e-6)],
                    [8, 8, 8], [8.3, 8, 8]], np.float32)
    assert oracle.fof3d_tieband(pos, box, l) == brute_tieband(pos, box, l) == 2
    _, _, tie = oracle.fof3d(pos, box, l=l)
    assert tie == 1  # only the linked one of the two (the other is beyond l)


def test_grid_component_and_neighbours():
    c = synth.generate("c1")
    lab, l, _ = oracle.fof3d(c.pos, c.box)
    grid = oracle.Grid(c.pos, c.box, l)
    sizes = np.bincount(lab)
    big = np.argsort(sizes)[::-1][:5]
    for g in big:
        comp = grid.component(int(g))
        assert np.array_equal(comp, np.flatnonzero(lab == g))
    rng = np.random.default_rng(3)
    p = c.pos.astype(np.float64)
    for i in rng.integers(0, c.n, 20):
        nb = grid.neighbours(int(i))
        d = p - p[i]
        d -= c.box * np.round(d / c.box)
        ref = np.flatnonzero(((d * d).sum(1) <= l * l) & (np.arange(c.n) != i))
        assert np.array_equal(nb, ref)


def test_empty_and_single():
    lab, _, tie = oracle.fof3d(np.zeros((0, 3), np.float32), 10.0, l=0.1)
    assert lab.shape == (0,) and tie == 0
    lab, _, _ = oracle.fof3d(np.array([[1, 2, 3]], np.float32), 10.0, l=0.1)
    assert lab.tolist() == [0]


def test_random_small_boxes_vs_brute():
    """Property check: random tiny catalogues (clumps and a background, any
    box side and linking length the grid accepts) give the brute-force
    partition."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=60, deadline=None, derandomize=True)
    @hyp.given(seed=st.integers(0, 2 ** 32 - 1), n=st.integers(1, 300), box=st.floats(1.0, 50.0),
               rel=st.floats(0.02, 0.3), clumps=st.integers(0, 4))
    def check(seed, n, box, rel, clumps):
        rng = np.random.default_rng(seed)
        p = rng.random((n, 3)) * box
        for c in range(clumps):
            k = rng.integers(0, n + 1)
            p[:k] = rng.random(3) * box + rng.normal(0.0, rel * box * 0.2, (k, 3))
        p = synth.wrap(p, box)
        box32 = float(np.float32(box))
        l = rel * box32
        lab, _, _ = oracle.fof3d(p, box32, l=l)
        assert np.array_equal(lab, brute_labels(p, box32, l))

    check()
