"""Parity of the halo-property calls with the oracle: rs_halo_props (Sec.
3.5.1 centres, Sec. 3.4 hosts) and rs_unbind (Sec. 3.4, App. B) through the
C ABI.  Centre nodes, hosts, assigned counts and set sizes must equal the
oracle's; bound flags may differ only for particles whose energy is within
rounding of zero; the tree potential of a set above 4096 members must lie
within theta of the oracle's direct sum."""
import numpy as np
import pytest

import oracle
from paper_1110_4372_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rs():
    assert torch.cuda.is_available()
    from paper_1110_4372_gb300 import rsgpu
    return rsgpu


def _small(seed, n=6000, halos=12):
    return synth.generate("c1", seed=seed, n=n, box=10.0 * (n / 32768) ** (1 / 3), n_halos=halos)


def _run(rs, cat):
    ctx = rs.Context()
    pos = torch.from_numpy(cat.pos).cuda()
    vel = torch.from_numpy(cat.vel).cuda()
    p = rs.params()
    labels, _, _ = rs.rs_fof3d(ctx, pos, cat.box, p.b)
    perm, off = rs.rs_group_sort(ctx, labels, p.min_n)
    tree = rs.rs_refine6d(ctx, pos, vel, cat.box, perm, off, p.f, p.min_n)
    hid, halos = rs.rs_assign_ex(ctx, tree, pos, vel, cat.box, p)
    hp = rs.rs_halo_props(ctx, tree, halos, hid)
    gm = oracle.particle_gm(cat.n / cat.box ** 3)
    ub = rs.rs_unbind(ctx, tree, halos, hid, hp["host"], pos, vel, gm)
    nodes = {k: v.cpu().numpy() for k, v in tree.nodes().items()}
    return dict(hid=hid.cpu().numpy(), arr={k: v.cpu().numpy() for k, v in halos.arrays().items()},
                hp={k: v.cpu().numpy() for k, v in hp.items()}, ub={k: v.cpu().numpy() for k, v in ub.items()},
                nodes=nodes, gm=gm)


@pytest.mark.parametrize("which", ["c1", "s31"])
def test_halo_props_and_unbind_match_oracle(rs, which):
    cat = synth.generate("c1") if which == "c1" else _small(int(which[1:]))
    g = _run(rs, cat)
    o = oracle.run_all(cat.pos, cat.vel, cat.box)
    assert np.array_equal(g["hid"], o["halo_id"])
    ohp = oracle.halo_props(o["tree"], o["halo_id"], o["halos"])
    # match halos by id
    gi = np.argsort(g["arr"]["id"])
    oi = np.argsort(o["halos"].id)
    assert np.array_equal(g["arr"]["id"][gi], o["halos"].id[oi])
    nd = g["nodes"]
    g_lv = nd["level"][g["hp"]["centre_node"][gi]]
    g_mi = nd["minidx"][g["hp"]["centre_node"][gi]]
    assert np.array_equal(g_lv, ohp["level"][oi]) and np.array_equal(g_mi, ohp["minidx"][oi])
    assert np.allclose(g["hp"]["xc"][gi], ohp["xc"][oi], rtol=0, atol=1e-6 * cat.box)
    assert np.array_equal(g["hp"]["n_assigned"][gi], ohp["n_assigned"][oi])
    assert np.array_equal(g["hp"]["host"][gi], ohp["host"][oi])
    ub = oracle.unbind(o["tree"], o["halo_id"], ohp["host"], g["gm"])
    assert np.array_equal(g["ub"]["n_part"][gi], ub["n_part"][oi])
    assert np.allclose(g["ub"]["vbulk"][gi], ub["vbulk"][oi], rtol=1e-9, atol=1e-9)
    diff = np.abs(g["ub"]["n_bound"][gi] - ub["n_bound"][oi])
    assert diff.max() <= 2  # particles at |E| within float32 rounding of zero
    assert np.mean(g["ub"]["bound_own"] == ub["bound_own"]) > 0.9999


def _one_big_halo(n=20000, seed=7):
    rng = np.random.default_rng(seed)
    box = 30.0
    p, v = synth.blob(rng, n, [15, 15, 15], [0, 0, 0], 0.4, 150.0)
    bg = rng.random((4000, 3)) * box
    pos = synth.wrap(np.vstack([p, bg]), box)
    vel = np.vstack([v, rng.standard_normal((4000, 3)) * 20]).astype(np.float32)
    return synth.Catalogue(pos=pos, vel=vel, box=box, truth=np.zeros(len(pos), np.int32),
                           comp_parent=np.zeros(0, np.int32), comp_n=np.zeros(0))


@pytest.mark.parametrize("theta", [0.04])
def test_unbind_tree_within_theta(rs, theta):
    """Sets above 4096 members use the tree: every potential within theta of
    the oracle's direct sum (App. B: each accepted box errs by at most theta
    relative, and all terms have one sign)."""
    cat = _one_big_halo()
    ctx = rs.Context()
    pos = torch.from_numpy(cat.pos).cuda()
    vel = torch.from_numpy(cat.vel).cuda()
    p = rs.params()
    labels, _, _ = rs.rs_fof3d(ctx, pos, cat.box, p.b)
    perm, off = rs.rs_group_sort(ctx, labels, p.min_n)
    tree = rs.rs_refine6d(ctx, pos, vel, cat.box, perm, off, p.f, p.min_n)
    hid, halos = rs.rs_assign_ex(ctx, tree, pos, vel, cat.box, p)
    hp = rs.rs_halo_props(ctx, tree, halos, hid)
    gm = oracle.particle_gm(len(cat.pos) / cat.box ** 3)
    ub = rs.rs_unbind(ctx, tree, halos, hid, hp["host"], pos, vel, gm, 0.0, theta)
    hid = hid.cpu().numpy()
    host = hp["host"].cpu().numpy()
    ids = halos.arrays()["id"].cpu().numpy()
    phi = ub["phi_own"].cpu().numpy()
    big = int(np.argmax(ub["n_part"].cpu().numpy()))
    assert ub["n_part"][big] > 4096
    # the biggest halo's own particles against the direct sum over its set
    members = [np.flatnonzero(hid == ids[big])] + [np.flatnonzero(hid == ids[s]) for s in range(len(ids))
                                                   if host[s] == ids[big]]
    mem = np.concatenate(members)
    flags, phi_o, _ = oracle.unbind_set(cat.pos, cat.vel, cat.box, mem, gm)
    own = hid[mem] == ids[big]
    rel = np.abs(phi[mem[own]] - phi_o[own]) / np.abs(phi_o[own])
    assert rel.max() <= max(theta, 1e-5) * 1.001
    # flags agree away from |E| <= theta |phi|
    v = cat.vel[mem[own]].astype(np.float64) - ub["vbulk"][big].cpu().numpy()
    e = 0.5 * (v * v).sum(1) + phi_o[own]
    clear = np.abs(e) > max(theta, 1e-5) * np.abs(phi_o[own]) * 1.01
    g = ub["bound_own"].cpu().numpy()[mem[own]].astype(bool)
    assert np.array_equal(g[clear], flags[own][clear])
