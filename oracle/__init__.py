"""float64 CPU oracle for the ROCKSTAR hot path -- TEST INFRASTRUCTURE.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``rs_oracle.c`` (plain C,
float64, no code shared with the CUDA library) through ctypes and adds the
few host-side steps the definitions need (the linking length of Sec. 3.1 and
grouping particles by label).

Every oracle function follows a passage of Behroozi, Wechsler & Wu,
arXiv:1110.4372:

* :func:`linking_length`, :func:`fof3d`, :class:`Grid` -- Sec. 3.1;
* :func:`refine`, :func:`node_dnn` -- Sec. 3.2 and Eq. 1;
* :func:`assign` -- Sec. 3.3, Eqs. 2-4.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rs_oracle.c")
_LIB = os.path.join(_HERE, "librsoracle.so")
_lib = None

TIE_REL = 1e-6


def build(force: bool = False) -> str:
    """Compile rs_oracle.c into oracle/librsoracle.so (no fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    P = C.c_void_p
    i64, i32, f64 = C.c_int64, C.c_int32, C.c_double
    lib.or_version.restype = i64
    lib.or_fof3d.argtypes = [P, i64, f64, f64, P, P]
    lib.or_fof3d_accel.argtypes = [P, i64, f64, f64, i64, P, P]
    lib.or_fof3d_accel.restype = C.c_int
    lib.or_fof3d.restype = C.c_int
    lib.or_fof3d_tieband.argtypes = [P, i64, f64, f64]
    lib.or_fof3d_tieband.restype = i64
    lib.or_grid_build.argtypes = [P, i64, f64, f64]
    lib.or_grid_build.restype = P
    lib.or_grid_free.argtypes = [P]
    lib.or_grid_component.argtypes = [P, i64, P, i64]
    lib.or_grid_component.restype = i64
    lib.or_grid_neighbours.argtypes = [P, i64, P, i64]
    lib.or_grid_neighbours.restype = i64
    lib.or_set_kd_threshold.argtypes = [C.c_int]
    lib.or_refine.argtypes = [P, P, i64, f64, P, P, i64, f64, i32, C.POINTER(C.c_int)]
    lib.or_refine.restype = P
    lib.or_refine_sampled.argtypes = [P, P, i64, f64, P, P, i64, f64, i32, i64, C.c_uint64, C.POINTER(C.c_int)]
    lib.or_refine_sampled.restype = P
    lib.or_sample_key.argtypes = [C.c_uint64, i64]
    lib.or_sample_key.restype = C.c_uint64
    lib.or_sample_keys.argtypes = [C.c_uint64, i64, i64, P]
    lib.or_tree_n_nodes.argtypes = [P]
    lib.or_tree_n_nodes.restype = i64
    lib.or_tree_n_members.argtypes = [P]
    lib.or_tree_n_members.restype = i64
    lib.or_tree_export.argtypes = [P] * 14
    lib.or_tree_members.argtypes = [P, P]
    lib.or_tree_free.argtypes = [P]
    lib.or_assign.argtypes = [P, f64, f64, f64, P, P]
    lib.or_assign.restype = C.c_int
    lib.or_halos_export.argtypes = [P] * 8
    lib.or_leaf_halo.argtypes = [P, P]
    lib.or_halo_props.argtypes = [P, P, P, P, P, P, P]
    lib.or_halo_props.restype = C.c_int
    lib.or_unbind.argtypes = [P, P, P, f64, f64, P, P, P, P]
    lib.or_unbind.restype = C.c_int
    lib.or_unbind_set.argtypes = [P, P, f64, P, i64, f64, f64, P, P, P]
    lib.or_unbind_set.restype = i64
    lib.or_node_dnn.argtypes = [P, P, P, i64, f64, f64, P, P]
    lib.or_node_dnn.restype = f64
    lib.merge_distance.argtypes = [i64, i32, P, P, f64, f64, i64, i32, P, P, f64, f64, f64]
    lib.merge_distance.restype = f64
    lib.rdyn2_of.argtypes = [P, P, i64, f64, P, f64, f64]
    lib.rdyn2_of.restype = f64
    lib.or_moments.argtypes = [P, P, P, i64, f64, P]
    lib.or_moments.restype = C.c_int
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32).reshape(-1, 3)


def linking_length(n: int, box: float, b: float = 0.28) -> float:
    """Sec. 3.1: the linking length is b times the mean interparticle
    distance, taken as the cube root of the mean volume per particle."""
    return float(b * np.cbrt(box * box * box / float(n)))


def fof3d(pos, box: float, b: float = 0.28, l: float | None = None):
    """Sec. 3.1: periodic 3D friends-of-friends.  Returns (labels, l, tie)
    where labels[i] is the smallest particle index of i's group and tie the
    number of pairs with |d - l| <= 1e-6 l among those linked."""
    pos = _f32(pos)
    n = pos.shape[0]
    if l is None:
        l = linking_length(n, box, b) if n > 0 else 0.0
    labels = np.empty(n, np.int32)
    tie = C.c_int64(0)
    st = _load().or_fof3d(_ptr(pos), n, float(box), float(l), _ptr(labels), C.byref(tie))
    if st:
        raise RuntimeError(f"or_fof3d failed with status {st}")
    return labels, l, int(tie.value)


def fof3d_accel(pos, box: float, b: float = 0.28, l: float | None = None, dense_n: int = 16):
    """Sec. 3.1, the accelerated variant: particles in index order; one with
    more than dense_n neighbours within l joins everything within 2l and its
    neighbours skip their own search.  Returns (labels, l, n_centres), labels
    being the smallest particle index of each group and n_centres the number
    of particles that searched 2l."""
    pos = _f32(pos)
    n = pos.shape[0]
    if l is None:
        l = linking_length(n, box, b) if n > 0 else 0.0
    labels = np.empty(n, np.int32)
    nc = C.c_int64(0)
    st = _load().or_fof3d_accel(_ptr(pos), n, float(box), float(l), int(dense_n), _ptr(labels), C.byref(nc))
    if st:
        raise RuntimeError(f"or_fof3d_accel failed with status {st}")
    return labels, l, int(nc.value)


def fof3d_tieband(pos, box: float, l: float) -> int:
    """Number of pairs whose periodic distance is within 1e-6 l of l."""
    pos = _f32(pos)
    return int(_load().or_fof3d_tieband(_ptr(pos), pos.shape[0], float(box), float(l)))


class Grid:
    """The 3D friendship graph of one catalogue, queried one particle or one
    group at a time (for checks at sizes where a full oracle pass is slow)."""

    def __init__(self, pos, box: float, l: float):
        self.pos = _f32(pos)
        self.n = self.pos.shape[0]
        self._h = _load().or_grid_build(_ptr(self.pos), self.n, float(box), float(l))
        if not self._h:
            raise MemoryError("or_grid_build failed")

    def component(self, seed: int, cap: int | None = None) -> np.ndarray:
        cap = self.n if cap is None else cap
        out = np.empty(cap, np.int32)
        k = _load().or_grid_component(self._h, int(seed), _ptr(out), cap)
        if k < 0:
            raise ValueError("component larger than cap")
        return out[:k].copy()

    def neighbours(self, i: int, cap: int = 1 << 20) -> np.ndarray:
        out = np.empty(cap, np.int32)
        k = _load().or_grid_neighbours(self._h, int(i), _ptr(out), cap)
        if k < 0:
            raise ValueError("more neighbours than cap")
        return out[:k].copy()

    def close(self):
        if self._h:
            _load().or_grid_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def groups_from_labels(labels: np.ndarray, min_n: int):
    """Members of every group with at least min_n particles, groups ordered
    by their label (smallest member index), members ascending.
    Returns (members int32, offsets int64)."""
    labels = np.asarray(labels)
    order = np.argsort(labels, kind="stable").astype(np.int64)
    sl = labels[order]
    if sl.size == 0:
        return np.zeros(0, np.int32), np.zeros(1, np.int64)
    starts = np.flatnonzero(np.r_[True, sl[1:] != sl[:-1]])
    ends = np.r_[starts[1:], sl.size]
    keep = (ends - starts) >= min_n
    parts = [order[s:e] for s, e in zip(starts[keep], ends[keep])]
    counts = (ends - starts)[keep]
    members = np.concatenate(parts).astype(np.int32) if parts else np.zeros(0, np.int32)
    offsets = np.zeros(len(parts) + 1, np.int64)
    offsets[1:] = np.cumsum(counts)
    return members, offsets


@dataclasses.dataclass
class Tree:
    """Oracle hierarchy.  Node arrays are indexed by node; members[first :
    first + count] are a node's particles with its children's particles at the
    front of the range (nested intervals)."""
    parent: np.ndarray
    level: np.ndarray
    first: np.ndarray
    count: np.ndarray
    minidx: np.ndarray
    group: np.ndarray
    nchild: np.ndarray
    lnk: np.ndarray
    xbar: np.ndarray
    vbar: np.ndarray
    sigx: np.ndarray
    sigv: np.ndarray
    tie: np.ndarray
    members: np.ndarray
    handle: object = None

    @property
    def n_nodes(self):
        return int(self.parent.shape[0])

    def node_members(self, i: int) -> np.ndarray:
        return self.members[self.first[i]:self.first[i] + self.count[i]]

    def level_labels(self, level: int, n_total: int) -> np.ndarray:
        """Per particle: smallest member index of the level-`level` node that
        holds it, or -1."""
        out = np.full(n_total, -1, np.int32)
        for i in np.flatnonzero(self.level == level):
            out[self.node_members(i)] = self.minidx[i]
        return out

    def free(self):
        if self.handle is not None:
            _load().or_tree_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sample_key(seed: int, i: int) -> int:
    """Sec. 3.2 subset draws: the SplitMix64 key of particle i (the (i+1)-th
    output of the stream whose state starts at `seed`)."""
    return int(_load().or_sample_key(int(seed) & (2 ** 64 - 1), int(i)))


def sample_keys(seed: int, first: int, count: int) -> np.ndarray:
    """:func:`sample_key` of particles first .. first+count-1 (uint64)."""
    out = np.empty(count, np.uint64)
    _load().or_sample_keys(int(seed) & (2 ** 64 - 1), int(first), int(count), _ptr(out))
    return out


def refine(pos, vel, box: float, members, offsets, f: float = 0.7, min_n: int = 10,
           kd_threshold: int = 1024, sub_n: int = 0, sub_seed: int = 0) -> Tree:
    """Sec. 3.2: phase-space FOF hierarchy of every group (members/offsets
    as returned by :func:`groups_from_labels`).  With sub_n > 0, a node of
    more than sub_n members takes its linking length from the nearest-
    neighbour distances of the sub_n members with the smallest
    :func:`sample_key` values (the paper's random 10,000-member subset)."""
    lib = _load()
    pos = _f32(pos)
    vel = _f32(vel)
    members = np.ascontiguousarray(members, np.int32)
    offsets = np.ascontiguousarray(offsets, np.int64)
    lib.or_set_kd_threshold(int(kd_threshold))
    st = C.c_int(0)
    h = lib.or_refine_sampled(_ptr(pos), _ptr(vel), pos.shape[0], float(box), _ptr(members), _ptr(offsets),
                              offsets.shape[0] - 1, float(f), int(min_n), int(sub_n),
                              int(sub_seed) & (2 ** 64 - 1), C.byref(st))
    if not h:
        raise RuntimeError(f"or_refine failed with status {st.value}")
    if st.value:
        lib.or_tree_free(h)
        raise RuntimeError(f"or_refine failed with status {st.value}")
    m = lib.or_tree_n_nodes(h)
    arr = dict(parent=np.empty(m, np.int32), level=np.empty(m, np.int32), first=np.empty(m, np.int64),
               count=np.empty(m, np.int64), minidx=np.empty(m, np.int32), group=np.empty(m, np.int32),
               nchild=np.empty(m, np.int32), lnk=np.empty(m), xbar=np.empty((m, 3)), vbar=np.empty((m, 3)),
               sigx=np.empty(m), sigv=np.empty(m), tie=np.empty(m, np.int64))
    lib.or_tree_export(h, *[_ptr(arr[k]) for k in ("parent", "level", "first", "count", "minidx", "group",
                                                   "nchild", "lnk", "xbar", "vbar", "sigx", "sigv", "tie")])
    mem = np.empty(lib.or_tree_n_members(h), np.int32)
    lib.or_tree_members(h, _ptr(mem))
    t = Tree(members=mem, handle=h, **arr)
    t._pos, t._vel = pos, vel  # keep the inputs alive for assign()
    return t


@dataclasses.dataclass
class Halos:
    id: np.ndarray
    ncore: np.ndarray
    nseeds: np.ndarray
    xbar: np.ndarray
    vbar: np.ndarray
    sigv: np.ndarray
    rdyn2: np.ndarray
    leaf_halo: np.ndarray


def assign(tree: Tree, n_total: int, box: float, delta_vir: float = 360.0, nbar: float | None = None,
           merge_thresh: float = 10.0 * np.sqrt(2.0)):
    """Sec. 3.3: seed merge (Eq. 2), r_dyn,vir (Eq. 4) and hierarchical
    assignment (Eq. 3).  Returns (halo_id per particle, Halos)."""
    lib = _load()
    if nbar is None:
        nbar = n_total / box ** 3
    hid = np.empty(n_total, np.int32)
    nh = C.c_int64(0)
    st = lib.or_assign(tree.handle, float(delta_vir), float(nbar), float(merge_thresh), _ptr(hid), C.byref(nh))
    if st:
        raise RuntimeError(f"or_assign failed with status {st}")
    h = int(nh.value)
    out = dict(id=np.empty(h, np.int32), ncore=np.empty(h, np.int64), nseeds=np.empty(h, np.int32),
               xbar=np.empty((h, 3)), vbar=np.empty((h, 3)), sigv=np.empty(h), rdyn2=np.empty(h))
    lib.or_halos_export(tree.handle, *[_ptr(out[k]) for k in ("id", "ncore", "nseeds", "xbar", "vbar", "sigv",
                                                              "rdyn2")])
    leaf = np.empty(tree.n_nodes, np.int32)
    lib.or_leaf_halo(tree.handle, _ptr(leaf))
    return hid, Halos(leaf_halo=leaf, **out)


# G in Mpc (km/s)^2 / Msun and the critical density in h^2 Msun / Mpc^3
G_MPC_KMS2_MSUN = 4.30091e-9
RHO_CRIT_H2 = 2.77536627e11


def particle_gm(nbar: float, omega_m: float = 0.27) -> float:
    """G times the particle mass, in (km/s)^2 Mpc/h, for a catalogue whose
    particles sample the matter density Omega_m rho_crit at nbar particles
    per (Mpc/h)^3 (reading; Omega_m = 0.27 is the Bolshoi cosmology of
    Sec. 4.1)."""
    return G_MPC_KMS2_MSUN * omega_m * RHO_CRIT_H2 / nbar


def halo_props(tree: Tree, halo_id, halos: "Halos"):
    """Sec. 3.5.1 centres and the Sec. 3.4 host relation, per halo in the
    order of :func:`assign`'s Halos: centre node (index into the tree), its
    level and smallest member, centre xc and velocity vc, assigned particle
    count and host id (-1 for a host halo)."""
    lib = _load()
    H = len(halos.id)
    halo_id = np.ascontiguousarray(halo_id, np.int32)
    out = dict(node=np.empty(H, np.int32), xc=np.empty((H, 3)), vc=np.empty((H, 3)),
               n_assigned=np.empty(H, np.int64), host=np.empty(H, np.int32))
    st = lib.or_halo_props(tree.handle, _ptr(halo_id), _ptr(out["node"]), _ptr(out["xc"]), _ptr(out["vc"]),
                           _ptr(out["n_assigned"]), _ptr(out["host"]))
    if st:
        raise RuntimeError(f"or_halo_props failed with status {st}")
    out["level"] = tree.level[out["node"]] if H else np.empty(0, np.int32)
    out["minidx"] = tree.minidx[out["node"]] if H else np.empty(0, np.int32)
    return out


def unbind(tree: Tree, halo_id, host, gm: float, eps: float = 0.0):
    """Sec. 3.4 / App. B single-pass unbinding with the exact potential.
    Per halo: n_part (its particles and its substructure's), n_bound, vbulk;
    per particle: bound_own (1/0 against its own halo's set, -1 outside every
    halo)."""
    lib = _load()
    H = len(host)
    halo_id = np.ascontiguousarray(halo_id, np.int32)
    host = np.ascontiguousarray(host, np.int32)
    out = dict(n_part=np.empty(H, np.int64), n_bound=np.empty(H, np.int64), vbulk=np.empty((H, 3)),
               bound_own=np.empty(len(halo_id), np.int8))
    st = lib.or_unbind(tree.handle, _ptr(halo_id), _ptr(host), float(gm), float(eps), _ptr(out["n_part"]),
                       _ptr(out["n_bound"]), _ptr(out["vbulk"]), _ptr(out["bound_own"]))
    if st:
        raise RuntimeError(f"or_unbind failed with status {st}")
    return out


def unbind_set(pos, vel, box: float, mem, gm: float, eps: float = 0.0):
    """The bound test on one particle set (App. B with the exact potential):
    returns (flags, phi per member, bulk velocity)."""
    pos = _f32(pos)
    vel = _f32(vel)
    mem = np.ascontiguousarray(mem, np.int32)
    n = mem.shape[0]
    flags = np.empty(n, np.int8)
    phi = np.empty(n)
    vb = np.empty(3)
    _load().or_unbind_set(_ptr(pos), _ptr(vel), float(box), _ptr(mem), n, float(gm), float(eps), _ptr(vb),
                          _ptr(phi), _ptr(flags))
    return flags.astype(bool), phi, vb


def node_dnn(pos, vel, mem, box: float, f: float = 0.7):
    """Brute-force nearest-neighbour distances (squared, Eq. 1) of one member
    list, its linking length squared, and its moments (sigx, sigv, xbar,
    vbar) -- Sec. 3.2."""
    pos = _f32(pos)
    vel = _f32(vel)
    mem = np.ascontiguousarray(mem, np.int32)
    dnn2 = np.empty(mem.shape[0])
    sig = np.empty(8)
    l2 = _load().or_node_dnn(_ptr(pos), _ptr(vel), _ptr(mem), mem.shape[0], float(box), float(f), _ptr(dnn2),
                             _ptr(sig))
    return dnn2, l2, dict(sigx=sig[0], sigv=sig[1], xbar=sig[2:5].copy(), vbar=sig[5:8].copy())


def run_all(pos, vel, box: float, b: float = 0.28, f: float = 0.7, min_n: int = 10, assign_too: bool = True,
            sub_n: int = 0, sub_seed: int = 0):
    """The whole path on one catalogue: 3D FOF, refinement (with subset
    linking lengths above sub_n members when sub_n > 0), assignment."""
    labels, l, tie3 = fof3d(pos, box, b)
    members, offsets = groups_from_labels(labels, min_n)
    tree = refine(pos, vel, box, members, offsets, f, min_n, sub_n=sub_n, sub_seed=sub_seed)
    out = dict(labels=labels, l=l, tie3=tie3, members=members, offsets=offsets, tree=tree)
    if assign_too:
        hid, halos = assign(tree, np.asarray(pos).reshape(-1, 3).shape[0], box)
        out.update(halo_id=hid, halos=halos)
    return out


def moments(pos, vel, mem, box: float):
    """Sec. 3.2: centre, bulk velocity and the 3D dispersions sigma_x, sigma_v
    of one member list (periodic unwrap about its smallest-index member)."""
    pos = _f32(pos)
    vel = _f32(vel)
    mem = np.ascontiguousarray(mem, np.int32)
    out = np.empty(8)
    st = _load().or_moments(_ptr(pos), _ptr(vel), _ptr(mem), mem.shape[0], float(box), _ptr(out))
    if st:
        raise ValueError(f"or_moments failed with status {st}")
    return dict(sigx=out[0], sigv=out[1], xbar=out[2:5].copy(), vbar=out[5:8].copy())


def merge_distance(a: dict, b: dict, box: float) -> float:
    """Eq. 2 separation of two seeds given as dicts with n, minidx, xbar,
    vbar, sigx, sigv."""
    xa, va = np.ascontiguousarray(a["xbar"], float), np.ascontiguousarray(a["vbar"], float)
    xb, vb = np.ascontiguousarray(b["xbar"], float), np.ascontiguousarray(b["vbar"], float)
    return float(_load().merge_distance(int(a["n"]), int(a["minidx"]), _ptr(xa), _ptr(va), float(a["sigx"]),
                                        float(a["sigv"]), int(b["n"]), int(b["minidx"]), _ptr(xb), _ptr(vb),
                                        float(b["sigx"]), float(b["sigv"]), float(box)))


def rdyn2(pos, mem, box: float, xbar, delta_vir: float, nbar: float) -> float:
    """Eq. 4: r_dyn,vir squared of a member list about centre xbar."""
    pos = _f32(pos)
    mem = np.ascontiguousarray(mem, np.int32)
    xb = np.ascontiguousarray(xbar, float)
    return float(_load().rdyn2_of(_ptr(pos), _ptr(mem), mem.shape[0], float(box), _ptr(xb), float(delta_vir),
                                  float(nbar)))
