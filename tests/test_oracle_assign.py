"""Pins of the oracle's seed merge (Eq. 2), r_dyn,vir (Eq. 4) and
hierarchical assignment (Sec. 3.3, Eq. 3).  CPU only."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1110_4372_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
SEEDS = json.load(open(os.path.join(GOLD, "hand_seeds.json")))


@pytest.mark.parametrize("case", SEEDS["merge_cases"], ids=range(len(SEEDS["merge_cases"])))
def test_merge_distance_hand(case):
    D = oracle.merge_distance(case["a"], case["b"], case["box"])
    assert D == pytest.approx(case["D"], rel=1e-12, abs=1e-12)
    assert (D < 10 * np.sqrt(2)) == case["merge"]
    # symmetric in its arguments
    assert oracle.merge_distance(case["b"], case["a"], case["box"]) == pytest.approx(D, rel=1e-15, abs=1e-15)


@pytest.mark.parametrize("case", SEEDS["rdyn_cases"], ids=range(len(SEEDS["rdyn_cases"])))
def test_rdyn_hand(case):
    pos = np.array(case["pos"], np.float32)
    r2 = oracle.rdyn2(pos, np.arange(len(pos)), case["box"], case["xbar"], case["delta_vir"], case["nbar"])
    assert r2 == pytest.approx(case["rdyn2"], rel=1e-12)


def test_hand_hierarchy_assignment():
    g = json.load(open(os.path.join(GOLD, "hand_hierarchy.json")))
    pos = np.array(g["pos"], np.float32)
    vel = np.array(g["vel"], np.float32)
    n = len(pos)
    t = oracle.refine(pos, vel, g["box"], np.arange(n, dtype=np.int32), np.array([0, n]), g["f"], g["min_n"])
    nbar = n / g["box"] ** 3
    hid, halos = oracle.assign(t, n, g["box"], g["delta_vir"], nbar)
    assert hid.tolist() == g["expect"]["halo_id"]
    rho = 4.0 / 3.0 * np.pi * g["delta_vir"] * nbar
    for k, v in g["expect"]["rdyn2_times_rho_term"].items():
        h = list(halos.id).index(int(k))
        assert halos.rdyn2[h] * rho == pytest.approx(v, rel=1e-12)


def test_two_identical_seeds_merge_far_ones_do_not():
    """Two copies of the same compact blob at one place merge (D = 0); the
    same two blobs 20 sqrt 2 uncertainties apart in position do not."""
    rng = np.random.default_rng(5)
    box = 50.0
    p, v = synth.blob(rng, 40, [25, 25, 25], [0, 0, 0], 0.01, 5.0)
    pos = synth.wrap(np.vstack([p, p]), box)
    vel = np.vstack([v, v]).astype(np.float32)
    # each blob alone: one seed; both: duplicates link at l = 0 ...
    m = oracle.moments(pos[:40], vel[:40], np.arange(40), box)
    a = dict(n=40, minidx=0, xbar=m["xbar"], vbar=m["vbar"], sigx=m["sigx"], sigv=m["sigv"])
    b = dict(a, minidx=40)
    assert oracle.merge_distance(a, b, box) == 0.0
    mu = m["sigx"] / np.sqrt(40)
    b2 = dict(a, minidx=40, xbar=m["xbar"] + np.array([20 * np.sqrt(2) * mu, 0, 0]))
    assert oracle.merge_distance(a, b2, box) == pytest.approx(20 * np.sqrt(2), rel=1e-12)


@pytest.fixture(scope="module")
def c1_all():
    c = synth.generate("c1")
    r = oracle.run_all(c.pos, c.vel, c.box)
    return c, r


def test_every_grouped_particle_assigned(c1_all):
    c, r = c1_all
    hid = r["halo_id"]
    grouped = np.zeros(c.n, bool)
    grouped[r["members"]] = True
    assert np.all(hid[grouped] >= 0)
    assert np.all(hid[~grouped] == -1)
    # a halo id is the smallest index of its seeds' members and never crosses
    # a 3D group
    lab = r["labels"]
    for h in np.unique(hid[hid >= 0]):
        assert len(np.unique(lab[hid == h])) == 1
    assert set(np.unique(hid[hid >= 0]).tolist()) <= set(r["halos"].id.tolist())


def test_single_seed_parent_takes_all(c1_all):
    """Sec. 3.3: a parent whose seeds form a single halo gives all its
    particles to that halo."""
    c, r = c1_all
    t, hid, halos = r["tree"], r["halo_id"], r["halos"]
    leaf_h = halos.leaf_halo
    checked = 0
    for i in range(t.n_nodes):
        span = (t.first[i], t.first[i] + t.count[i])
        under = [j for j in range(t.n_nodes) if t.nchild[j] == 0 and span[0] <= t.first[j] < span[1]]
        hs = {int(leaf_h[j]) for j in under}
        if len(hs) == 1:
            assert np.all(hid[t.node_members(i)] == hs.pop())
            checked += 1
    assert checked > 10


def test_multi_seed_argmin(c1_all):
    """Members of a multi-seed node that lie outside its children go to the
    halo with the smallest Eq. 3 distance among the node's seeds."""
    c, r = c1_all
    t, hid, halos = r["tree"], r["halo_id"], r["halos"]
    hidx = {int(h): k for k, h in enumerate(halos.id)}
    seen = 0
    for i in range(t.n_nodes):
        if t.nchild[i] == 0:
            continue
        span = (t.first[i], t.first[i] + t.count[i])
        under = [j for j in range(t.n_nodes) if t.nchild[j] == 0 and span[0] <= t.first[j] < span[1]]
        hs = sorted({int(halos.leaf_halo[j]) for j in under})
        if len(hs) < 2:
            continue
        kids = np.flatnonzero(t.parent == i)
        tail = t.members[t.first[i] + t.count[kids].sum(): span[1]]
        for p in tail:
            d2 = []
            for h in hs:
                k = hidx[h]
                dx = halos.xbar[k] - c.pos[p].astype(np.float64)
                dx -= c.box * np.round(dx / c.box)
                dv = halos.vbar[k] - c.vel[p].astype(np.float64)
                d2.append((dx @ dx) / halos.rdyn2[k] + (dv @ dv) / halos.sigv[k] ** 2)
            assert hid[p] == hs[int(np.argmin(d2))]
            seen += 1
    assert seen > 0
