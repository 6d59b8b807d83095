"""Parity of the CUDA path (through the C ABI) with the float64 oracle.

Bar: 3D labels, group CSR, node member sets, child counts, tie-band counts
and halo ids equal the oracle's exactly, with no excused node; sigma_x,
sigma_v and linking lengths within 1e-6 relative; centres within 1e-6
sigma; the halo table (Sec. 3.3: centre, bulk velocity, sigma_v, r_dyn,vir)
within 1e-6 relative or 1e-6 sigma."""
import numpy as np
import pytest

import oracle
from paper_1110_4372_gb300 import synth

from gpu_util import (compare_halo_tables, compare_trees, cuda_inputs, gpu_tree_dict, oracle_tree_dict,
                      run_gpu_path, run_oracle_path)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rs():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1110_4372_gb300 import rsgpu
    return rsgpu


@pytest.fixture(scope="module")
def ctx(rs):
    return rs.Context()


def _small(seed, n=4000, halos=10, nmax=4000, sub=0):
    box = 10.0 * (n / 32768) ** (1 / 3)
    return synth.generate("c1", seed=seed, n=n, box=box, n_halos=halos)


# ---------------------------------------------------------------------------
# 3D friends-of-friends
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("stride", [3, 4])
def test_fof3d_c1_exact(rs, ctx, stride):
    c = synth.generate("c1")
    pos, _ = cuda_inputs(c, stride)
    lab, ng, nt = rs.rs_fof3d(ctx, pos, c.box, 0.28, want_groups=True, want_tieband=True)
    ref, l, _ = oracle.fof3d(c.pos, c.box, 0.28)
    assert np.array_equal(lab.cpu().numpy(), ref)
    assert ng == len(np.unique(ref))
    assert nt == oracle.fof3d_tieband(c.pos, c.box, l)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_fof3d_uniform_dense(rs, ctx, seed):
    c = synth.uniform(6000, 10.0, seed)
    pos, _ = cuda_inputs(c)
    for b in (0.2, 0.6, 0.9):
        lab, _, _ = rs.rs_fof3d(ctx, pos, c.box, b)
        ref, _, _ = oracle.fof3d(c.pos, c.box, b)
        assert np.array_equal(lab.cpu().numpy(), ref), b


def test_fof3d_periodic_faces(rs, ctx):
    rng = np.random.default_rng(5)
    box = 10.0
    n = 3000
    # particles crowded against every face, edge and corner
    p = rng.random((n, 3)) * 0.3
    flip = rng.random((n, 3)) < 0.5
    p = np.where(flip, box - p, p)
    c = synth.Catalogue(pos=synth.wrap(p, box), vel=np.zeros((n, 3), np.float32), box=box,
                        truth=np.zeros(n, np.int32), comp_parent=np.zeros(0, np.int32), comp_n=np.zeros(0))
    pos, _ = cuda_inputs(c)
    for b in (0.1, 0.3):
        lab, _, _ = rs.rs_fof3d(ctx, pos, box, b)
        ref, _, _ = oracle.fof3d(c.pos, box, b)
        assert np.array_equal(lab.cpu().numpy(), ref), b


def test_fof3d_lattice_closed_form(rs, ctx):
    m = 16
    g = (np.arange(m) + 0.5).astype(np.float32)
    pos = np.array(np.meshgrid(g, g, g, indexing="ij"), np.float32).reshape(3, -1).T.copy()
    box = float(m)
    # l = b * spacing; spacing = 1 here
    t = torch.from_numpy(pos).cuda()
    lab, _, _ = rs.rs_fof3d(ctx, t, box, 1.0 + 1e-3)
    assert np.all(lab.cpu().numpy() == 0)
    lab, _, _ = rs.rs_fof3d(ctx, t, box, 1.0 - 1e-3)
    assert np.array_equal(lab.cpu().numpy(), np.arange(len(pos)))


def test_fof3d_empty_and_tiny(rs, ctx):
    lab, ng, _ = rs.rs_fof3d(ctx, torch.zeros((0, 3), device="cuda"), 10.0, 0.28, want_groups=True)
    assert lab.numel() == 0 and ng == 0


def test_fof3d_bad_args(rs, ctx):
    pos = torch.rand((100, 3), device="cuda") * 10
    with pytest.raises(rs.RsError):
        rs.rs_fof3d(ctx, pos, -1.0, 0.28)
    with pytest.raises(rs.RsError):
        rs.rs_fof3d(ctx, pos, 10.0, 0.0)


def test_fof3d_narrow_box_without_grid_is_rejected(rs, ctx):
    """box/l = 7.5: no grid of 4k cells per side has cells between l/2 and
    l/sqrt(3), so the call fails instead of missing friends three cells
    apart."""
    n = 64
    box = 10.0
    b = box / 7.5 / n ** (1 / 3)  # l = box / 7.5
    pos = torch.from_numpy(synth.wrap(np.random.default_rng(75).random((n, 3)) * box, box)).cuda()
    with pytest.raises(rs.RsError):
        rs.rs_fof3d(ctx, pos, box, b)
    b_ok = box / 9.0 / n ** (1 / 3)  # box/l = 9 has one
    lab, _, _ = rs.rs_fof3d(ctx, pos, box, b_ok)
    ref, _, _ = oracle.fof3d(pos.cpu().numpy(), box, b_ok)
    assert np.array_equal(lab.cpu().numpy(), ref)


# ---------------------------------------------------------------------------
# accelerated 3D FOF (Sec. 3.1)
# ---------------------------------------------------------------------------
def _accel_check(rs, ctx, pos_np, box, b, dense_n=16):
    pos = torch.from_numpy(np.ascontiguousarray(pos_np, np.float32)).cuda()
    lab, ng, nc = rs.rs_fof3d_accel(ctx, pos, box, b, dense_n)
    ref, _, nref = oracle.fof3d_accel(pos_np, box, b, dense_n=dense_n)
    lab = lab.cpu().numpy()
    assert np.array_equal(lab, ref)
    assert nc == nref and ng == len(np.unique(ref))
    return lab, nc


def test_fof3d_accel_c1_and_small(rs, ctx):
    for c in (synth.generate("c1"), _small(11), _small(12)):
        lab, nc = _accel_check(rs, ctx, c.pos, c.box, 0.28)
        plain, _, _ = oracle.fof3d(c.pos, c.box, 0.28)
        for g in np.unique(plain)[:2000]:  # groups are unions of plain groups
            assert len(np.unique(lab[plain == g])) == 1
        assert nc > 0


@pytest.mark.parametrize("dense_n", [0, 3, 16])
def test_fof3d_accel_dense_uniform(rs, ctx, dense_n):
    c = synth.uniform(6000, 10.0, 40 + dense_n)
    _accel_check(rs, ctx, c.pos, c.box, 0.9, dense_n)


def test_fof3d_accel_hand_order(rs, ctx):
    """A dense particle skipped inside the first centre's ball does not join
    its far satellite; visited first, it does."""
    rng = np.random.default_rng(2)
    box, n = 20.0, 20
    b = 1.0 * n ** (1 / 3) / box  # l = 1
    v = rng.standard_normal((18, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    clump = np.array([10.0, 10, 10]) + v * 0.05 * rng.random(18)[:, None]
    clump[0] = [10.0, 10, 10]
    k, t = np.array([[10.9, 10, 10]]), np.array([[12.7, 10, 10]])
    first = synth.wrap(np.vstack([clump, k, t]), box)
    lab, nc = _accel_check(rs, ctx, first, box, b)
    assert nc == 1 and lab[18] == 0 and lab[19] == 19
    second = synth.wrap(np.vstack([k, clump, t]), box)
    lab2, nc2 = _accel_check(rs, ctx, second, box, b)
    assert nc2 == 1 and np.all(lab2 == 0)


def test_fof3d_accel_bad_args(rs, ctx):
    pos = torch.from_numpy(synth.wrap(np.random.default_rng(76).random((100, 3)) * 10, 10.0)).cuda()
    with pytest.raises(rs.RsError):
        rs.rs_fof3d_accel(ctx, pos, 10.0, 0.28, -1)
    lab, ng, nc = rs.rs_fof3d_accel(ctx, torch.zeros((0, 3), device="cuda"), 10.0, 0.28)
    assert lab.numel() == 0 and ng == 0 and nc == 0


# ---------------------------------------------------------------------------
# group CSR
# ---------------------------------------------------------------------------
def test_group_sort_c1(rs, ctx):
    c = synth.generate("c1")
    pos, _ = cuda_inputs(c)
    lab, _, _ = rs.rs_fof3d(ctx, pos, c.box, 0.28)
    perm, off = rs.rs_group_sort(ctx, lab, 10)
    ref_lab, _, _ = oracle.fof3d(c.pos, c.box, 0.28)
    m, o = oracle.groups_from_labels(ref_lab, 10)
    assert np.array_equal(perm.cpu().numpy(), m)
    assert np.array_equal(off.cpu().numpy(), o)


# ---------------------------------------------------------------------------
# hierarchy and assignment
# ---------------------------------------------------------------------------
def _check_all(rs, ctx, cat, stride=3, f=0.7, min_n=10, sub_n=0, sub_seed=0):
    g = run_gpu_path(ctx, rs, cat, stride=stride, f=f, min_n=min_n, sub_n=sub_n, sub_seed=sub_seed)
    o = run_oracle_path(cat, f=f, min_n=min_n, sub_n=sub_n, sub_seed=sub_seed)
    assert np.array_equal(g["labels"], o["labels"])
    assert g["tie3"] == oracle.fof3d_tieband(cat.pos, cat.box, o["l"])
    assert np.array_equal(g["perm"], o["members"]) and np.array_equal(g["offsets"], o["offsets"])
    gd, od = gpu_tree_dict(g["tree"]), oracle_tree_dict(o["tree"])
    matched, tie_nodes = compare_trees(gd, od, cat.box)
    info = g["tree"].info()
    assert info.n_nodes == o["tree"].n_nodes == matched
    assert info.n_tieband == int(o["tree"].tie.sum())
    assert np.array_equal(g["halo_id"], o["halo_id"])
    assert g["n_halos"] == len(o["halos"].id)
    compare_halo_tables(g["halo_table"], o["tree"], o["halos"], cat.pos, cat.vel, cat.box)
    # rs_assign (the call rs_find_halos makes) gives the ids of rs_assign_ex
    pos, vel = cuda_inputs(cat, stride)
    hid, nh = rs.rs_assign(ctx, g["tree"], pos, vel, cat.box, rs.params(f=f, min_n=min_n))
    assert np.array_equal(hid.cpu().numpy(), g["halo_id"]) and nh == g["n_halos"]
    return matched, tie_nodes, info


def test_refine_assign_c1(rs, ctx):
    matched, tie_nodes, info = _check_all(rs, ctx, synth.generate("c1"))
    assert matched > 50 and info.n_seeds > 30


@pytest.mark.parametrize("seed", [11, 12])
def test_refine_assign_small_catalogues(rs, ctx, seed):
    _check_all(rs, ctx, _small(seed))


def test_refine_stride4_and_f_values(rs, ctx):
    c = _small(21)
    _check_all(rs, ctx, c, stride=4)
    _check_all(rs, ctx, c, f=0.5)
    _check_all(rs, ctx, c, f=0.9, min_n=20)


def _big_catalogue():
    rng = np.random.default_rng(3)
    box = 20.0
    parts, vels = [], []
    for k, n in enumerate((6000, 2500, 1500)):
        centre = rng.random(3) * 14 + 3
        p, v = synth.blob(rng, n, centre, rng.standard_normal(3) * 100, 0.15, 60.0)
        parts.append(p)
        vels.append(v)
        # a co-spatial clump moving differently inside the first blob
        if k == 0:
            p2, v2 = synth.blob(rng, 800, centre, [300.0, 0, 0], 0.05, 30.0)
            parts.append(p2)
            vels.append(v2)
    pos = synth.wrap(np.vstack(parts), box)
    vel = np.vstack(vels).astype(np.float32)
    n = len(pos)
    perm = rng.permutation(n)
    return synth.Catalogue(pos=pos[perm].copy(), vel=vel[perm].copy(), box=box, truth=np.zeros(n, np.int32),
                           comp_parent=np.zeros(0, np.int32), comp_n=np.zeros(0))


def test_refine_big_node_path(rs, ctx):
    """Groups above 1024 members take the multi-CTA level path; their
    children below it finish in the one-CTA subtree kernel."""
    matched, tie_nodes, info = _check_all(rs, ctx, _big_catalogue())
    assert info.n_levels >= 3


@pytest.mark.parametrize("sub_n,seed", [(1024, 0), (2048, 7), (4096, 2 ** 63 + 5)])
def test_refine_sampled_subsets(rs, ctx, sub_n, seed):
    """Sec. 3.2 subset linking lengths: nodes above sub_n members take l from
    the nearest-neighbour distances of their sub_n smallest-key members."""
    c = _big_catalogue()
    matched, tie_nodes, info = _check_all(rs, ctx, c, sub_n=sub_n, sub_seed=seed)
    sizes = np.bincount(oracle.fof3d(c.pos, c.box)[0])
    assert sizes.max() > sub_n  # at least the largest root is sampled
    assert matched >= 5


def test_refine_sampled_covering_subset_is_exact(rs, ctx):
    """A subset at least as large as every node is the exact linking length:
    the same tree bit for bit."""
    c = _big_catalogue()
    a = run_gpu_path(ctx, rs, c, assign=False)
    b = run_gpu_path(ctx, rs, c, assign=False, sub_n=len(c.pos), sub_seed=9)
    da, db = gpu_tree_dict(a["tree"]), gpu_tree_dict(b["tree"])
    assert da.keys() == db.keys()
    for k in da:
        assert da[k]["members"] == db[k]["members"] and da[k]["lnk"] == db[k]["lnk"]


def test_refine_sampled_bad_subset_size(rs, ctx):
    c = _small(11)
    pos, vel = cuda_inputs(c)
    labels, _, _ = rs.rs_fof3d(ctx, pos, c.box, 0.28)
    perm, offsets = rs.rs_group_sort(ctx, labels, 10)
    for bad in (1, 1023, -5):
        with pytest.raises(RuntimeError):
            rs.rs_refine6d_sampled(ctx, pos, vel, c.box, perm, offsets, 0.7, 10, bad, 0)


def test_refine_group_across_box_corner(rs, ctx):
    rng = np.random.default_rng(8)
    box = 10.0
    p, v = synth.blob(rng, 3000, [0.0, 0.0, 0.0], [0, 0, 0], 0.2, 50.0)
    p2, v2 = synth.blob(rng, 400, [0.05, 9.95, 0.0], [200, 0, 0], 0.05, 20.0)
    pos = synth.wrap(np.vstack([p, p2]), box)
    vel = np.vstack([v, v2]).astype(np.float32)
    n = len(pos)
    c = synth.Catalogue(pos=pos, vel=vel, box=box, truth=np.zeros(n, np.int32), comp_parent=np.zeros(0, np.int32),
                        comp_n=np.zeros(0))
    _check_all(rs, ctx, c)


def test_refine_duplicates(rs, ctx):
    """Identical points: zero linking lengths and zero dispersions."""
    rng = np.random.default_rng(4)
    box = 10.0
    base = rng.random((40, 3)) * 0.05 + 5.0
    pos = synth.wrap(np.repeat(base, 30, axis=0), box)
    vel = np.repeat(rng.standard_normal((40, 3)) * 10, 30, axis=0).astype(np.float32)
    n = len(pos)
    c = synth.Catalogue(pos=pos, vel=vel, box=box, truth=np.zeros(n, np.int32), comp_parent=np.zeros(0, np.int32),
                        comp_n=np.zeros(0))
    _check_all(rs, ctx, c)


def test_level_labels(rs, ctx):
    c = synth.generate("c1")
    g = run_gpu_path(ctx, rs, c, assign=False)
    o = run_oracle_path(c, assign=False)
    t = g["tree"]
    for level in range(t.info().n_levels):
        assert np.array_equal(t.level_labels(level).cpu().numpy(), o["tree"].level_labels(level, c.n))


def test_find_halos_host_and_device(rs, ctx):
    c = _small(31)
    o = run_oracle_path(c)
    pos, vel = cuda_inputs(c)
    lab = torch.empty(c.n, dtype=torch.int32, device="cuda")
    hid, _, st = rs.rs_find_halos(ctx, pos, vel, c.box, fof_labels=lab)
    assert np.array_equal(hid.cpu().numpy(), o["halo_id"])
    assert np.array_equal(lab.cpu().numpy(), o["labels"])
    hp = torch.from_numpy(c.pos).pin_memory()
    vp = torch.from_numpy(c.vel).pin_memory()
    lab_h = torch.full((c.n,), -5, dtype=torch.int32).pin_memory()
    hid2, _, st2 = rs.rs_find_halos(ctx, hp, vp, c.box, fof_labels=lab_h)
    assert not hid2.is_cuda
    assert np.array_equal(hid2.numpy(), o["halo_id"])
    assert np.array_equal(lab_h.numpy(), o["labels"])  # copied back while the refinement ran
    assert st2["n_halos"] == len(o["halos"].id) == st["n_halos"]
    # repeated host-buffer calls reuse the second stream and its events
    for _ in range(2):
        hid3, _, _ = rs.rs_find_halos(ctx, hp, vp, c.box)
        assert np.array_equal(hid3.numpy(), o["halo_id"])


def test_empty_inputs(rs, ctx):
    z = torch.zeros((0, 3), device="cuda")
    hid, _, st = rs.rs_find_halos(ctx, z, z, 10.0)
    assert hid.numel() == 0 and st["n_halos"] == 0
    # a catalogue with no group of min_n members
    c = synth.uniform(500, 10.0, 3)
    g = run_gpu_path(ctx, rs, c)
    assert g["tree"].info().n_nodes == 0 and np.all(g["halo_id"] == -1)


def test_deterministic_repeat(rs, ctx):
    c = _small(41)
    a = run_gpu_path(ctx, rs, c)
    b = run_gpu_path(ctx, rs, c)
    assert np.array_equal(a["halo_id"], b["halo_id"])
    assert gpu_tree_dict(a["tree"]).keys() == gpu_tree_dict(b["tree"]).keys()


@pytest.mark.slow
def test_full_path_c2(rs, ctx):
    matched, tie_nodes, info = _check_all(rs, ctx, synth.generate("c2"))
    assert matched == info.n_nodes > 5000


@pytest.mark.slow
def test_fof3d_accel_c2(rs, ctx):
    c = synth.generate("c2")
    lab, nc = _accel_check(rs, ctx, c.pos, c.box, 0.28)
    print(f"c2 accelerated FOF: {nc} centres, {len(np.unique(lab))} groups")


@pytest.mark.slow
def test_full_path_c2_subset_10000(rs, ctx):
    """The paper's setting: groups above 10,000 particles take their linking
    length from a random 10,000-particle subset (Sec. 3.2)."""
    matched, tie_nodes, info = _check_all(rs, ctx, synth.generate("c2"), sub_n=10000, sub_seed=11104372)
    assert matched == info.n_nodes > 5000


@pytest.mark.slow
def test_batching_stress_groups_c4s(rs, ctx):
    """The independent-group batching workload (small case of its recipe:
    NFW hosts with co-spatial, velocity-offset subhalos, Sec. 2.2 / Fig. 2),
    first 400 groups given straight to rs_refine6d as group offsets (no 3D
    FOF): the node tree equals the oracle's exactly, and so do the seed
    merge and assignment at the recipe's density."""
    g = synth.groups("c4s", first=0, count=400)
    pos = torch.from_numpy(g.pos).cuda()
    vel = torch.from_numpy(g.vel).cuda()
    perm = torch.arange(g.n, dtype=torch.int32, device="cuda")
    off = torch.from_numpy(g.offsets).cuda()
    tree = rs.rs_refine6d(ctx, pos, vel, g.box, perm, off)
    t = oracle.refine(g.pos, g.vel, g.box, np.arange(g.n, dtype=np.int32), g.offsets)
    matched, _ = compare_trees(gpu_tree_dict(tree), oracle_tree_dict(t), g.box)
    assert matched == t.n_nodes == tree.info().n_nodes > 400
    assert tree.info().n_tieband == int(t.tie.sum())
    hid, nh = rs.rs_assign(ctx, tree, pos, vel, g.box, rs.params(nbar=synth.GROUP_NBAR))
    hid_o, halos = oracle.assign(t, g.n, g.box, 360.0, synth.GROUP_NBAR)
    assert np.array_equal(hid.cpu().numpy(), hid_o) and nh == len(halos.id)


OTHER_TUNING = dict(link_blocks_per_sm=4, nn_blocks_per_sm=7, kd_levels=1, bracket_min=2048, mid_max=128,
                    tiny_max=16, small_ctas_per_sm=1, mid_ctas_per_sm=4, tiny_ctas_per_sm=12, fof_link_ctas_per_sm=8)


def test_launch_choices_change_no_result(rs):
    """Every launch choice of rs_tuning changes which CTA or warp does which
    work, never a result: the whole path under choices different from the
    defaults still matches the oracle exactly."""
    ctx2 = rs.Context()
    t = rs.rs_set_tuning(ctx2, **OTHER_TUNING)
    assert t == dict(rs.rs_tuning_default(), **OTHER_TUNING) == rs.rs_get_tuning(ctx2)
    for cat in (_big_catalogue(), synth.generate("c1")):
        _check_all(rs, ctx2, cat)
    ctx2.close()


def test_tuning_rejects_out_of_range(rs, ctx):
    before = rs.rs_get_tuning(ctx)
    for bad in (dict(link_blocks_per_sm=3), dict(kd_levels=4), dict(mid_max=300), dict(tiny_max=33),
                dict(bracket_min=100), dict(fof_link_ctas_per_sm=0)):
        with pytest.raises(rs.RsError):
            rs.rs_set_tuning(ctx, **bad)
    assert rs.rs_get_tuning(ctx) == before


def test_bracket_fallback_redoes_only_failed_nodes_exactly(rs, monkeypatch):
    """Big nodes (above 4096 members) search within a sampled bracket of
    the linking length; a node whose bracket does not hold is searched again
    without it.  With the injected fault RS_FAULT=bracket every bracketed
    node of odd rank takes that path while the others keep their bracketed
    values: the tree still equals the oracle's exactly."""
    rng = np.random.default_rng(9)
    box = 40.0
    parts, vels = [], []
    for c in range(5):
        centre = rng.random(3) * 30 + 5
        p, v = synth.blob(rng, 5000 + 300 * c, centre, rng.standard_normal(3) * 100, 0.2, 80.0)
        parts.append(p)
        vels.append(v)
    pos = synth.wrap(np.vstack(parts), box)
    vel = np.vstack(vels).astype(np.float32)
    n = len(pos)
    cat = synth.Catalogue(pos=pos, vel=vel, box=box, truth=np.zeros(n, np.int32),
                          comp_parent=np.zeros(0, np.int32), comp_n=np.zeros(0))
    monkeypatch.setenv("RS_FAULT", "bracket")
    ctx2 = rs.Context()
    _check_all(rs, ctx2, cat)
    p, v = cuda_inputs(cat)
    _, _, st = rs.rs_find_halos(ctx2, p, v, cat.box)
    assert st["n_fallback_levels"] >= 1
    monkeypatch.delenv("RS_FAULT")
    _, _, st = rs.rs_find_halos(ctx2, p, v, cat.box)
    assert st["n_fallback_levels"] == 0


@pytest.mark.parametrize("n,pinned", [(4001, True), (4002, False), (4003, True)])
def test_find_halos_host_buffers_odd_sizes(rs, ctx, n, pinned):
    """Host-buffer calls copy pinned positions with a kernel (16-byte words
    and a 4-byte tail, here n % 4 != 0) and pageable ones with a plain copy;
    both give the oracle's halo ids and labels."""
    c = synth.generate("c1", seed=n, n=n, box=10.0 * (n / 32768) ** (1 / 3), n_halos=12)
    o = run_oracle_path(c)
    hp, hv = torch.from_numpy(c.pos), torch.from_numpy(c.vel)
    lab = torch.full((c.n,), -3, dtype=torch.int32)
    if pinned:
        hp, hv, lab = hp.pin_memory(), hv.pin_memory(), lab.pin_memory()
    hid, _, _ = rs.rs_find_halos(ctx, hp, hv, c.box, fof_labels=lab)
    assert np.array_equal(hid.numpy(), o["halo_id"])
    assert np.array_equal(lab.numpy(), o["labels"])
