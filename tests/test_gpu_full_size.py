"""Parity at the benchmark's full size (134M particles, and 1.07B with
RS_TEST_C5=1; the same calls the benchmark times), on sampled outputs the
oracle can compute one by one:

* 3D groups: the member set of the group of sampled particles, found by the
  oracle's breadth-first search over the whole box, equals the CUDA label
  set (both directions: every oracle member has the label, and the group has
  no other member);
* hierarchy and assignment: sampled groups -- a spread of sizes up to 60k
  members plus the largest group of at most LARGE_MAX members (a few hundred
  thousand, the multi-level big-node path) -- are refined and assigned by
  the oracle from its own member lists; node sets per (level, smallest
  member), child and tie-band counts and every halo id must match exactly,
  with sigma, centre and linking length within 1e-6 relative.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1110_4372_gb300 import synth

from gpu_util import compare_trees, oracle_tree_dict

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

N_PARTICLES = 24        # random particles whose 3D group is checked
N_GROUPS = 12           # sampled groups refined and assigned by the oracle
MAX_GROUP = 60000
LARGE_MIN, LARGE_MAX = 200_000, 450_000


@pytest.fixture(scope="module", params=["c3", "c5"])
def full(request):
    """The 134M-particle workload; the 1.07B-particle one (c5) only when
    RS_TEST_C5=1, since generating it and the oracle's grid over it take
    about a quarter of an hour on the host."""
    if request.param == "c5" and os.environ.get("RS_TEST_C5") != "1":
        pytest.skip("the 1.07B-particle case runs with RS_TEST_C5=1")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1110_4372_gb300 import rsgpu
    cat = synth.generate(request.param)
    ctx = rsgpu.Context()
    pos = torch.from_numpy(cat.pos).cuda()
    vel = torch.from_numpy(cat.vel).cuda()
    p = rsgpu.params()
    labels, _, _ = rsgpu.rs_fof3d(ctx, pos, cat.box, p.b)
    perm, offsets = rsgpu.rs_group_sort(ctx, labels, p.min_n)
    tree = rsgpu.rs_refine6d(ctx, pos, vel, cat.box, perm, offsets, p.f, p.min_n)
    hid, nh = rsgpu.rs_assign(ctx, tree, pos, vel, cat.box, p)
    nd = {k: v.cpu().numpy() for k, v in tree.nodes().items()}
    out = dict(cat=cat, labels=labels.cpu().numpy(), hid=hid.cpu().numpy(), nodes=nd,
               members=tree.members().cpu().numpy(), l=oracle.linking_length(cat.n, cat.box, p.b))
    del pos, vel
    torch.cuda.empty_cache()
    out["grid"] = oracle.Grid(cat.pos, cat.box, out["l"])
    return out


def _gpu_nodes_of(full, group_members):
    """GPU nodes (as the dict of gpu_util) whose members lie in the group."""
    nd, mem = full["nodes"], full["members"]
    inside = np.zeros(full["cat"].n, bool)
    inside[group_members] = True
    out = {}
    keys = {}
    for i in np.flatnonzero(inside[nd["minidx"]]):
        keys[i] = (int(nd["level"][i]), int(nd["minidx"][i]))
    for i, key in keys.items():
        m = mem[nd["first"][i]:nd["first"][i] + nd["count"][i]]
        p = int(nd["parent"][i])
        out[key] = dict(members=tuple(np.sort(m).tolist()), lnk=nd["lnk"][i], sigx=nd["sigx"][i], sigv=nd["sigv"][i],
                        xbar=nd["xbar"][i], vbar=nd["vbar"][i], tie=int(nd["tie"][i]), nchild=int(nd["nchild"][i]),
                        parent_key=keys.get(p) if p >= 0 else None)
    return out


def test_fof_groups_of_sampled_particles(full):
    rng = np.random.default_rng(20261202)
    cat, labels, grid = full["cat"], full["labels"], full["grid"]
    seeds = list(rng.integers(0, cat.n, N_PARTICLES))
    # and three of the largest groups below 200k members (the oracle's search
    # is quadratic inside dense cores)
    sizes = np.bincount(labels)
    big = [g for g in np.argsort(sizes)[::-1][:2000] if sizes[g] <= 200_000][:3]
    seeds += [int(g) for g in big]
    for s in seeds:
        comp = grid.component(int(s))
        lab = labels[s]
        assert np.all(labels[comp] == lab), f"particle {s}: oracle group member with another label"
        assert sizes[lab] == len(comp), f"particle {s}: label set {sizes[lab]} vs oracle group {len(comp)}"
        assert lab == comp.min()


def _check_group(full, g):
    cat, labels, grid = full["cat"], full["labels"], full["grid"]
    nbar = cat.n / cat.box ** 3
    members = grid.component(int(g))  # the oracle's own member list
    assert len(members) == np.count_nonzero(labels == labels[g])
    t = oracle.refine(cat.pos, cat.vel, cat.box, members.astype(np.int32), np.array([0, len(members)]))
    hid_o, _ = oracle.assign(t, cat.n, cat.box, 360.0, nbar)
    gd = _gpu_nodes_of(full, members)
    od = oracle_tree_dict(t)
    matched, _ = compare_trees(gd, od, cat.box)
    assert np.array_equal(full["hid"][members], hid_o[members]), f"group {g}: halo ids differ"
    n_nodes = t.n_nodes
    t.free()
    return matched, n_nodes


def test_hierarchy_and_assignment_of_sampled_groups(full):
    rng = np.random.default_rng(11104373)
    labels = full["labels"]
    sizes = np.bincount(labels)
    candidates = np.flatnonzero((sizes >= 10) & (sizes <= MAX_GROUP))
    # spread the sample over group sizes: a third from the largest eligible
    by_size = candidates[np.argsort(sizes[candidates])]
    pick = list(rng.choice(by_size[: len(by_size) * 2 // 3], N_GROUPS - N_GROUPS // 3, replace=False))
    pick += list(by_size[-(N_GROUPS // 3):])
    checked = 0
    for g in pick:
        matched, n_nodes = _check_group(full, g)
        assert matched == n_nodes
        checked += matched
    assert checked > N_GROUPS


def test_hierarchy_of_a_large_group(full):
    """The largest group of at most LARGE_MAX members (at least LARGE_MIN):
    several big-node levels (k-d order, sampled bracket, box hierarchy)
    before the subtree kernels take over."""
    sizes = np.bincount(full["labels"])
    ok = np.flatnonzero((sizes >= LARGE_MIN) & (sizes <= LARGE_MAX))
    assert len(ok), "the 134M workload has a group in the size range"
    g = int(ok[np.argmax(sizes[ok])])
    matched, n_nodes = _check_group(full, g)
    assert matched == n_nodes > 20
