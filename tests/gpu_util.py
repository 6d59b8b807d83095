"""Helpers shared by the GPU parity tests: run the CUDA path through the C
ABI binding and compare it with the oracle in canonical form."""
import numpy as np
import torch

import oracle


def cuda_inputs(cat, stride=3):
    pos = torch.from_numpy(cat.pos).cuda()
    vel = torch.from_numpy(cat.vel).cuda()
    if stride == 4:
        pos = torch.nn.functional.pad(pos, (0, 1)).contiguous()
        vel = torch.nn.functional.pad(vel, (0, 1)).contiguous()
    return pos, vel


def gpu_tree_dict(tree):
    nd = {k: v.cpu().numpy() for k, v in tree.nodes().items()}
    mem = tree.members().cpu().numpy()
    out = {}
    for i in range(len(nd["level"])):
        key = (int(nd["level"][i]), int(nd["minidx"][i]))
        m = mem[nd["first"][i]:nd["first"][i] + nd["count"][i]]
        out[key] = dict(members=tuple(np.sort(m).tolist()), lnk=nd["lnk"][i], sigx=nd["sigx"][i],
                        sigv=nd["sigv"][i], xbar=nd["xbar"][i], vbar=nd["vbar"][i], tie=int(nd["tie"][i]),
                        parent=int(nd["parent"][i]), nchild=int(nd["nchild"][i]))
    # parent keys
    keys = list(out.keys())
    idx_key = {}
    for i in range(len(nd["level"])):
        idx_key[i] = (int(nd["level"][i]), int(nd["minidx"][i]))
    for i in range(len(nd["level"])):
        p = int(nd["parent"][i])
        out[idx_key[i]]["parent_key"] = idx_key[p] if p >= 0 else None
    return out


def oracle_tree_dict(t):
    out = {}
    for i in range(t.n_nodes):
        key = (int(t.level[i]), int(t.minidx[i]))
        p = int(t.parent[i])
        out[key] = dict(members=tuple(np.sort(t.node_members(i)).tolist()), lnk=t.lnk[i], sigx=t.sigx[i],
                        sigv=t.sigv[i], xbar=t.xbar[i], vbar=t.vbar[i], tie=int(t.tie[i]),
                        parent_key=(int(t.level[p]), int(t.minidx[p])) if p >= 0 else None,
                        nchild=int(t.nchild[i]))
    return out


def compare_trees(g, o, box, rel=1e-6):
    """Node sets must match exactly: the same (level, smallest member) keys
    with the same member sets.  The float64 recheck of every float32
    decision inside its error band makes the GPU's partitions those of the
    float64 definition, tie-band pairs included, so no difference is
    excused.  sigma_x, sigma_v and the linking length must agree within rel
    (relative), centres within rel sigma (minimum image for positions), and
    child counts exactly.  Returns (n_matched, n_tie_nodes): the matched
    node count and how many of them hold tie-band pairs (reported, since a
    tie-band pair is where float32 alone would have gone wrong)."""
    only_g = sorted(set(g) - set(o))
    only_o = sorted(set(o) - set(g))
    assert not only_g and not only_o, (f"node keys differ: {len(only_g)} only on the GPU (e.g. {only_g[:3]}), "
                                       f"{len(only_o)} only in the oracle (e.g. {only_o[:3]})")
    bad = [k for k in g if g[k]["members"] != o[k]["members"]]
    assert not bad, f"{len(bad)} node(s) with different member sets, e.g. {sorted(bad)[:5]}"
    tie_nodes = 0
    for k in g:
        a, b = g[k], o[k]
        assert a["sigx"] == b["sigx"] or abs(a["sigx"] - b["sigx"]) <= rel * b["sigx"], (k, a["sigx"], b["sigx"])
        assert a["sigv"] == b["sigv"] or abs(a["sigv"] - b["sigv"]) <= rel * b["sigv"], (k, a["sigv"], b["sigv"])
        assert a["lnk"] == b["lnk"] or abs(a["lnk"] - b["lnk"]) <= rel * b["lnk"], (k, a["lnk"], b["lnk"])
        dx = a["xbar"] - b["xbar"]
        dx -= box * np.round(dx / box)
        assert np.linalg.norm(dx) <= rel * max(b["sigx"], 1e-300) + 1e-12, (k, a["xbar"], b["xbar"])
        assert np.linalg.norm(a["vbar"] - b["vbar"]) <= rel * max(b["sigv"], 1e-300) + 1e-9, (k, a["vbar"],
                                                                                           b["vbar"])
        assert a["nchild"] == b["nchild"], k
        assert a["parent_key"] == b["parent_key"], k
        assert a["tie"] == b["tie"], (k, a["tie"], b["tie"])
        tie_nodes += b["tie"] > 0
    return len(g), tie_nodes


def halo_seed_members(t, halos):
    """Per oracle halo (in the order of oracle.assign's Halos), the particle
    indices of its seeds' members: the members of the leaves whose
    leaf_halo (a halo id) is that halo's id."""
    slot = {int(h): k for k, h in enumerate(halos.id)}
    out = [[] for _ in range(len(halos.id))]
    for i in np.flatnonzero(t.nchild == 0):
        h = int(halos.leaf_halo[i])
        if h >= 0:
            out[slot[h]].append(t.node_members(i))
    return [np.concatenate(m) if m else np.zeros(0, np.int32) for m in out]


def compare_halo_tables(g_arr, o_tree, o_halos, pos, vel, box, rel=1e-6):
    """The GPU halo table (rs_halos_export) against the oracle's Halos, halo
    by halo after matching ids: sigma_v and r_dyn,vir^2 within rel
    (relative); the centre within rel sigma_x and the bulk velocity within
    rel sigma_v, sigma_x and sigma_v being the 3D dispersions of the halo's
    seeds' members (Sec. 3.3), computed by the oracle."""
    import oracle
    gi = np.argsort(g_arr["id"], kind="stable")
    oi = np.argsort(o_halos.id, kind="stable")
    assert np.array_equal(g_arr["id"][gi], o_halos.id[oi]), "halo ids differ"
    sv_g, sv_o = g_arr["sigv"][gi], o_halos.sigv[oi]
    assert np.all(np.abs(sv_g - sv_o) <= rel * sv_o), "sigma_v differs"
    rd_g, rd_o = g_arr["rdyn2"][gi], o_halos.rdyn2[oi]
    assert np.all((rd_g == rd_o) | (np.abs(rd_g - rd_o) <= rel * rd_o)), "r_dyn,vir^2 differs"
    mem = halo_seed_members(o_tree, o_halos)
    for a, b in zip(gi, oi):
        m = oracle.moments(pos, vel, mem[b], box)
        dx = g_arr["xbar"][a] - o_halos.xbar[b]
        dx -= box * np.round(dx / box)
        assert np.linalg.norm(dx) <= rel * m["sigx"] + 1e-12, ("centre", int(o_halos.id[b]))
        dv = g_arr["vbar"][a] - o_halos.vbar[b]
        assert np.linalg.norm(dv) <= rel * m["sigv"] + 1e-9, ("bulk velocity", int(o_halos.id[b]))
    return len(gi)


def run_gpu_path(ctx, rs, cat, stride=3, f=0.7, min_n=10, b=0.28, assign=True, sub_n=0, sub_seed=0):
    pos, vel = cuda_inputs(cat, stride)
    labels, ng, nt = rs.rs_fof3d(ctx, pos, cat.box, b, want_groups=True, want_tieband=True)
    perm, offsets = rs.rs_group_sort(ctx, labels, min_n)
    if sub_n:
        tree = rs.rs_refine6d_sampled(ctx, pos, vel, cat.box, perm, offsets, f, min_n, sub_n, sub_seed)
    else:
        tree = rs.rs_refine6d(ctx, pos, vel, cat.box, perm, offsets, f, min_n)
    out = dict(labels=labels.cpu().numpy(), n_groups=ng, tie3=nt, perm=perm.cpu().numpy(),
               offsets=offsets.cpu().numpy(), tree=tree)
    if assign:
        hid, halos = rs.rs_assign_ex(ctx, tree, pos, vel, cat.box, rs.params(b=b, f=f, min_n=min_n))
        out.update(halo_id=hid.cpu().numpy(), n_halos=halos.n,
                   halo_table={k: v.cpu().numpy() for k, v in halos.arrays().items()})
    return out


def run_oracle_path(cat, f=0.7, min_n=10, b=0.28, assign=True, sub_n=0, sub_seed=0):
    return oracle.run_all(cat.pos, cat.vel, cat.box, b=b, f=f, min_n=min_n, assign_too=assign, sub_n=sub_n,
                          sub_seed=sub_seed)
