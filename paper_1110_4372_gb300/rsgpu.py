"""Thin ctypes binding of librsgpu.so (include/rsgpu.h).

Every function here has the name of the C entry point it calls and only
marshals arguments: torch tensors in, ``data_ptr()`` and sizes out, the
current torch CUDA stream as the context's stream.  All computation runs in
the library's CUDA kernels.  Importing this module loads the library and
fails loudly if it is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librsgpu.so")

RS_OK = 0
STATUS_NAMES = {0: "RS_OK", 1: "RS_ERR_INVALID_ARG", 2: "RS_ERR_CUDA", 3: "RS_ERR_OOM", 4: "RS_ERR_TIMEOUT",
                5: "RS_ERR_TOO_LARGE", 6: "RS_ERR_INTERNAL", 7: "RS_ERR_EXTENT"}


class RsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class rs_params(C.Structure):
    _fields_ = [("b", C.c_double), ("f", C.c_double), ("min_n", C.c_int32), ("delta_vir", C.c_double),
                ("nbar", C.c_double), ("merge_thresh", C.c_double), ("nn_subset", C.c_int64),
                ("nn_seed", C.c_uint64)]


class rs_tuning(C.Structure):
    _fields_ = [(k, C.c_int32) for k in ("link_blocks_per_sm", "nn_blocks_per_sm", "kd_levels", "bracket_min",
                                         "mid_max", "tiny_max", "small_ctas_per_sm", "mid_ctas_per_sm",
                                         "tiny_ctas_per_sm", "fof_link_ctas_per_sm")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class rs_stats(C.Structure):
    _fields_ = [("n_fof_groups", C.c_int64), ("n_members", C.c_int64), ("n_nodes", C.c_int64),
                ("n_levels", C.c_int32), ("n_seeds", C.c_int64), ("n_halos", C.c_int64),
                ("n_tieband6d", C.c_int64), ("sum_level_members", C.c_int64),
                ("sum_big_level_members", C.c_int64), ("n_fallback_levels", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _declare(lib):
    P, i32, i64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "rs_params_default": (None, [C.POINTER(rs_params)]),
        "rs_create": (C.c_int, [C.POINTER(P), P]),
        "rs_destroy": (None, [P]),
        "rs_set_stream": (C.c_int, [P, P]),
        "rs_status_string": (C.c_char_p, [C.c_int]),
        "rs_last_error": (C.c_char_p, [P]),
        "rs_linking_length": (f64, [i64, f64, f64]),
        "rs_selftest_wait": (C.c_int, [P, i32, i64]),
        "rs_fof3d": (C.c_int, [P, P, i32, i64, f64, f64, P, P, P]),
        "rs_fof3d_accel": (C.c_int, [P, P, i32, i64, f64, f64, i32, P, P, P]),
        "rs_group_sort": (C.c_int, [P, P, i64, i32, P, P, i64, C.POINTER(i64), C.POINTER(i64)]),
        "rs_refine6d": (C.c_int, [P, P, P, i32, i64, f64, P, P, i64, f64, i32, C.POINTER(P)]),
        "rs_refine6d_sampled": (C.c_int, [P, P, P, i32, i64, f64, P, P, i64, f64, i32, i64, C.c_uint64,
                                          C.POINTER(P)]),
        "rs_tree_info": (C.c_int, [P, C.POINTER(i64), C.POINTER(i32), C.POINTER(i64), C.POINTER(i64),
                                   C.POINTER(i64)]),
        "rs_tree_nodes": (C.c_int, [P, P] + [P] * 12),
        "rs_tree_members": (C.c_int, [P, P, P]),
        "rs_tree_level_labels": (C.c_int, [P, P, i32, i64, P]),
        "rs_tree_free": (None, [P]),
        "rs_assign": (C.c_int, [P, P, P, P, i32, i64, f64, C.POINTER(rs_params), P, C.POINTER(i64)]),
        "rs_assign_ex": (C.c_int, [P, P, P, P, i32, i64, f64, C.POINTER(rs_params), P, C.POINTER(i64),
                                   C.POINTER(P)]),
        "rs_halos_free": (None, [P]),
        "rs_halos_count": (i64, [P]),
        "rs_halos_export": (C.c_int, [P, P, P, P, P, P, P]),
        "rs_halo_props": (C.c_int, [P, P, P, P, i64, P, P, P, P, P]),
        "rs_unbind": (C.c_int, [P, P, P, P, P, P, P, i32, i64, f64, f64, f64, P, P, P, P, P]),
        "rs_find_halos": (C.c_int, [P, P, P, i32, i64, f64, C.POINTER(rs_params), P, P, C.POINTER(rs_stats),
                                    i32]),
        "rs_profile_enable": (C.c_int, [P, i32]),
        "rs_profile_reset": (None, [P]),
        "rs_profile_count": (i32, [P]),
        "rs_profile_read": (C.c_int, [P, i32, C.POINTER(C.c_char_p), C.POINTER(i64), C.POINTER(f64)]),
        "rs_launch_count": (i64, [P]),
        "rs_workspace_bytes": (i64, [P]),
        "rs_tuning_default": (None, [C.POINTER(rs_tuning)]),
        "rs_set_tuning": (C.c_int, [P, C.POINTER(rs_tuning)]),
        "rs_get_tuning": (C.c_int, [P, C.POINTER(rs_tuning)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1110_4372_gb300.build.build()")
        _lib = _declare(C.CDLL(LIB_PATH))
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if t.numel() == 0:
            return None
        return C.c_void_p(t.data_ptr())
    return t


def _stride_of(t: torch.Tensor) -> int:
    if t.dim() != 2 or t.shape[1] not in (3, 4) or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("positions/velocities must be contiguous float32 tensors of shape (n, 3) or (n, 4)")
    return int(t.shape[1])


class Context:
    """An rs_ctx bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, stream: torch.cuda.Stream | None = None):
        self._h = C.c_void_p()
        s = (stream or torch.cuda.current_stream()).cuda_stream
        st = lib().rs_create(C.byref(self._h), C.c_void_p(s))
        if st != RS_OK:
            raise RsError(st, "rs_create failed")

    @property
    def handle(self):
        return self._h

    def check(self, st: int):
        if st != RS_OK:
            raise RsError(st, lib().rs_last_error(self._h).decode(errors="replace"))

    def set_stream(self, stream: torch.cuda.Stream):
        self.check(lib().rs_set_stream(self._h, C.c_void_p(stream.cuda_stream)))

    def close(self):
        if self._h:
            lib().rs_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def params(**kw) -> rs_params:
    p = rs_params()
    lib().rs_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def rs_selftest_wait(ctx: Context, set_flag: bool, limit: int = 20000) -> None:
    """Failure-detection self-test: a bounded device wait on a flag nothing
    sets (set_flag False) raises RsError with RS_ERR_TIMEOUT; the context
    stays usable."""
    ctx.check(lib().rs_selftest_wait(ctx.handle, 1 if set_flag else 0, int(limit)))


def rs_linking_length(n: int, box: float, b: float = 0.28) -> float:
    return float(lib().rs_linking_length(int(n), float(box), float(b)))


def rs_fof3d(ctx: Context, pos: torch.Tensor, box: float, b: float = 0.28, labels: torch.Tensor | None = None,
             want_groups: bool = False, want_tieband: bool = False):
    """Sec. 3.1.  Returns (labels, n_groups or None, n_tieband or None)."""
    n = pos.shape[0]
    if labels is None:
        labels = torch.empty(n, dtype=torch.int32, device=pos.device)
    ng, nt = C.c_int64(0), C.c_int64(0)
    ctx.check(lib().rs_fof3d(ctx.handle, _ptr(pos), _stride_of(pos), n, float(box), float(b), _ptr(labels),
                             C.byref(ng) if want_groups else None, C.byref(nt) if want_tieband else None))
    return labels, (ng.value if want_groups else None), (nt.value if want_tieband else None)


def rs_fof3d_accel(ctx: Context, pos: torch.Tensor, box: float, b: float = 0.28, dense_n: int = 16,
                   labels: torch.Tensor | None = None):
    """Sec. 3.1, the accelerated variant.  Returns (labels, n_groups,
    n_centres)."""
    n = pos.shape[0]
    if labels is None:
        labels = torch.empty(n, dtype=torch.int32, device=pos.device)
    ng, nc = C.c_int64(0), C.c_int64(0)
    ctx.check(lib().rs_fof3d_accel(ctx.handle, _ptr(pos), _stride_of(pos), n, float(box), float(b), int(dense_n),
                                   _ptr(labels), C.byref(ng), C.byref(nc)))
    return labels, ng.value, nc.value


def rs_group_sort(ctx: Context, labels: torch.Tensor, min_n: int = 10):
    """App. A work units.  Returns (perm[:n_members], offsets[:n_groups+1])."""
    n = labels.shape[0]
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=labels.device)
    cap = n // max(min_n, 1) + 2
    offsets = torch.empty(cap, dtype=torch.int64, device=labels.device)
    ng, nm = C.c_int64(0), C.c_int64(0)
    ctx.check(lib().rs_group_sort(ctx.handle, _ptr(labels), n, int(min_n), _ptr(perm), _ptr(offsets), cap,
                                  C.byref(ng), C.byref(nm)))
    return perm[:nm.value], offsets[:ng.value + 1]


@dataclasses.dataclass
class TreeInfo:
    n_nodes: int
    n_levels: int
    n_seeds: int
    n_tieband: int
    n_members: int


class Tree:
    """Library-owned hierarchy (rs_tree)."""

    def __init__(self, ctx: Context, handle: C.c_void_p, n_total: int, device):
        self.ctx = ctx
        self._h = handle
        self.n_total = n_total
        self.device = device

    def info(self) -> TreeInfo:
        a, c, d, e = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        b = C.c_int32()
        self.ctx.check(lib().rs_tree_info(self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(d), C.byref(e)))
        return TreeInfo(a.value, b.value, c.value, d.value, e.value)

    def nodes(self) -> dict:
        m = self.info().n_nodes
        dev = self.device
        i32 = lambda k=1: torch.empty(m * k, dtype=torch.int32, device=dev)
        i64 = lambda: torch.empty(m, dtype=torch.int64, device=dev)
        f64 = lambda k=1: torch.empty(m * k, dtype=torch.float64, device=dev)
        out = dict(parent=i32(), level=i32(), first=i64(), count=i64(), minidx=i32(), nchild=i32(), lnk=f64(),
                   xbar=f64(3), vbar=f64(3), sigx=f64(), sigv=f64(), tie=i64())
        if m:
            self.ctx.check(lib().rs_tree_nodes(self.ctx.handle, self._h, *[_ptr(out[k]) for k in (
                "parent", "level", "first", "count", "minidx", "nchild", "lnk", "xbar", "vbar", "sigx", "sigv",
                "tie")]))
        out["xbar"] = out["xbar"].view(m, 3)
        out["vbar"] = out["vbar"].view(m, 3)
        return out

    def members(self) -> torch.Tensor:
        m = self.info().n_members
        t = torch.empty(m, dtype=torch.int32, device=self.device)
        self.ctx.check(lib().rs_tree_members(self.ctx.handle, self._h, _ptr(t)))
        return t

    def level_labels(self, level: int) -> torch.Tensor:
        t = torch.empty(self.n_total, dtype=torch.int32, device=self.device)
        self.ctx.check(lib().rs_tree_level_labels(self.ctx.handle, self._h, int(level), self.n_total, _ptr(t)))
        return t

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h:
            lib().rs_tree_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def rs_refine6d(ctx: Context, pos: torch.Tensor, vel: torch.Tensor, box: float, perm: torch.Tensor,
                offsets: torch.Tensor, f: float = 0.7, min_n: int = 10) -> Tree:
    """Sec. 3.2."""
    return rs_refine6d_sampled(ctx, pos, vel, box, perm, offsets, f, min_n, 0, 0)


def rs_refine6d_sampled(ctx: Context, pos: torch.Tensor, vel: torch.Tensor, box: float, perm: torch.Tensor,
                        offsets: torch.Tensor, f: float = 0.7, min_n: int = 10, subset_n: int = 10000,
                        subset_seed: int = 0) -> Tree:
    """Sec. 3.2 with the linking length of nodes above subset_n members taken
    from a random subset_n-member subset (subset_n = 0: every member)."""
    stride = _stride_of(pos)
    if _stride_of(vel) != stride:
        raise ValueError("pos and vel must have the same stride")
    h = C.c_void_p()
    ng = offsets.shape[0] - 1
    ctx.check(lib().rs_refine6d_sampled(ctx.handle, _ptr(pos), _ptr(vel), stride, pos.shape[0], float(box),
                                        _ptr(perm), C.c_void_p(offsets.data_ptr()), ng, float(f), int(min_n),
                                        int(subset_n), int(subset_seed) & (2 ** 64 - 1), C.byref(h)))
    return Tree(ctx, h, pos.shape[0], pos.device)


def rs_assign(ctx: Context, tree: Tree, pos: torch.Tensor, vel: torch.Tensor, box: float,
              p: rs_params | None = None, halo_id: torch.Tensor | None = None):
    """Sec. 3.3.  Returns (halo_id, n_halos)."""
    p = p or params()
    n = pos.shape[0]
    if halo_id is None:
        halo_id = torch.empty(n, dtype=torch.int32, device=pos.device)
    nh = C.c_int64(0)
    ctx.check(lib().rs_assign(ctx.handle, tree.handle, _ptr(pos), _ptr(vel), _stride_of(pos), n, float(box),
                              C.byref(p), _ptr(halo_id), C.byref(nh)))
    return halo_id, nh.value


def particle_gm(nbar: float, omega_m: float = 0.27) -> float:
    """G times the particle mass in (km/s)^2 Mpc/h for particles sampling the
    matter density Omega_m rho_crit at nbar per (Mpc/h)^3 (G = 4.30091e-9
    Mpc (km/s)^2 / Msun, rho_crit = 2.77536627e11 h^2 Msun / Mpc^3)."""
    return 4.30091e-9 * omega_m * 2.77536627e11 / nbar


class Halos:
    """Library-owned per-halo table from :func:`rs_assign_ex`."""

    def __init__(self, ctx: Context, handle: C.c_void_p, device):
        self.ctx, self._h, self.device = ctx, handle, device
        self.n = int(lib().rs_halos_count(handle))

    @property
    def handle(self):
        return self._h

    def arrays(self) -> dict:
        """id, xbar, vbar, sigv, rdyn2 as device tensors (the table's order)."""
        H = self.n
        out = dict(id=torch.empty(H, dtype=torch.int32, device=self.device),
                   xbar=torch.empty((H, 3), dtype=torch.float64, device=self.device),
                   vbar=torch.empty((H, 3), dtype=torch.float64, device=self.device),
                   sigv=torch.empty(H, dtype=torch.float64, device=self.device),
                   rdyn2=torch.empty(H, dtype=torch.float64, device=self.device))
        if H:
            self.ctx.check(lib().rs_halos_export(self.ctx.handle, self._h, *[_ptr(out[k]) for k in
                                                                          ("id", "xbar", "vbar", "sigv", "rdyn2")]))
        return out

    def __del__(self):
        try:
            if self._h:
                lib().rs_halos_free(self._h)
                self._h = None
        except Exception:
            pass


def rs_assign_ex(ctx: Context, tree: Tree, pos: torch.Tensor, vel: torch.Tensor, box: float,
                 p: rs_params | None = None):
    """Sec. 3.3 with the per-halo table.  Returns (halo_id, Halos)."""
    p = p or params()
    n = pos.shape[0]
    halo_id = torch.empty(n, dtype=torch.int32, device=pos.device)
    nh = C.c_int64(0)
    h = C.c_void_p()
    ctx.check(lib().rs_assign_ex(ctx.handle, tree.handle, _ptr(pos), _ptr(vel), _stride_of(pos), n, float(box),
                                 C.byref(p), _ptr(halo_id), C.byref(nh), C.byref(h)))
    return halo_id, Halos(ctx, h, pos.device)


def rs_halo_props(ctx: Context, tree: Tree, halos: Halos, halo_id: torch.Tensor) -> dict:
    """Sec. 3.5.1 centres and the Sec. 3.4 host relation, per halo in the
    table's order: centre_node, xc, vc, n_assigned, host (device tensors)."""
    H, dev = halos.n, halo_id.device
    out = dict(centre_node=torch.empty(H, dtype=torch.int32, device=dev),
               xc=torch.empty((H, 3), dtype=torch.float64, device=dev),
               vc=torch.empty((H, 3), dtype=torch.float64, device=dev),
               n_assigned=torch.empty(H, dtype=torch.int64, device=dev),
               host=torch.empty(H, dtype=torch.int32, device=dev))
    ctx.check(lib().rs_halo_props(ctx.handle, tree.handle, halos.handle, _ptr(halo_id), halo_id.shape[0],
                                  *[_ptr(out[k]) for k in ("centre_node", "xc", "vc", "n_assigned", "host")]))
    return out


def rs_unbind(ctx: Context, tree: Tree, halos: Halos, halo_id: torch.Tensor, host: torch.Tensor, pos: torch.Tensor,
              vel: torch.Tensor, gm: float, eps: float = 0.0, theta: float = 0.04) -> dict:
    """Sec. 3.4 / App. B single-pass unbinding (theta = 0: direct sums; else
    the tree for sets above 4096 members): n_part, n_bound, vbulk per halo,
    bound_own and phi_own per particle (device tensors)."""
    H, dev, n = halos.n, pos.device, pos.shape[0]
    out = dict(n_part=torch.empty(H, dtype=torch.int64, device=dev),
               n_bound=torch.empty(H, dtype=torch.int64, device=dev),
               vbulk=torch.empty((H, 3), dtype=torch.float64, device=dev),
               bound_own=torch.empty(n, dtype=torch.int8, device=dev),
               phi_own=torch.full((n,), float("nan"), dtype=torch.float64, device=dev))
    ctx.check(lib().rs_unbind(ctx.handle, tree.handle, halos.handle, _ptr(halo_id), _ptr(host), _ptr(pos),
                              _ptr(vel), _stride_of(pos), n, float(gm), float(eps), float(theta),
                              *[_ptr(out[k]) for k in ("n_part", "n_bound", "vbulk", "bound_own", "phi_own")]))
    return out


def rs_find_halos(ctx: Context, pos: torch.Tensor, vel: torch.Tensor, box: float, p: rs_params | None = None,
                  fof_labels: torch.Tensor | None = None, halo_id: torch.Tensor | None = None):
    """The whole path.  pos/vel may be CUDA tensors (device buffers) or CPU
    tensors (host buffers; pinned memory copies fastest); the outputs live on
    the same side.  Returns (halo_id, fof_labels or None, stats dict)."""
    p = p or params()
    n = pos.shape[0]
    host = not pos.is_cuda
    dev = pos.device
    if halo_id is None:
        halo_id = torch.empty(n, dtype=torch.int32, device=dev, pin_memory=host and torch.cuda.is_available())
    st = rs_stats()
    ctx.check(lib().rs_find_halos(ctx.handle, _ptr(pos), _ptr(vel), _stride_of(pos), n, float(box), C.byref(p),
                                  _ptr(fof_labels), _ptr(halo_id), C.byref(st), 1 if host else 0))
    return halo_id, fof_labels, st.as_dict()


def rs_profile_enable(ctx: Context, on: bool = True):
    ctx.check(lib().rs_profile_enable(ctx.handle, 1 if on else 0))


def rs_profile_reset(ctx: Context):
    lib().rs_profile_reset(ctx.handle)


def rs_profile_read(ctx: Context) -> dict:
    """{kernel name: (launches, total device ms)}."""
    out = {}
    for i in range(lib().rs_profile_count(ctx.handle)):
        name, n, ms = C.c_char_p(), C.c_int64(), C.c_double()
        ctx.check(lib().rs_profile_read(ctx.handle, i, C.byref(name), C.byref(n), C.byref(ms)))
        if n.value:
            out[name.value.decode()] = (n.value, ms.value)
    return out


def rs_launch_count(ctx: Context) -> int:
    return int(lib().rs_launch_count(ctx.handle))


def rs_tuning_default() -> dict:
    t = rs_tuning()
    lib().rs_tuning_default(C.byref(t))
    return t.as_dict()


def rs_get_tuning(ctx: Context) -> dict:
    t = rs_tuning()
    ctx.check(lib().rs_get_tuning(ctx.handle, C.byref(t)))
    return t.as_dict()


def rs_set_tuning(ctx: Context, **fields) -> dict:
    """Sets the named launch choices (the rest keep their current values);
    returns the context's whole tuning."""
    t = rs_tuning()
    ctx.check(lib().rs_get_tuning(ctx.handle, C.byref(t)))
    for k, v in fields.items():
        if k not in t.as_dict():
            raise KeyError(k)
        setattr(t, k, int(v))
    ctx.check(lib().rs_set_tuning(ctx.handle, C.byref(t)))
    return t.as_dict()


TUNING_FILE = os.path.join(_HERE, "tuning_gb300.json")


def apply_tuning(ctx: Context, path: str = TUNING_FILE) -> dict:
    """Applies the "tuned" table of a tuner record (tune.py --out; by default
    the record of the GB300 run shipped with the package, whose table the
    library's defaults already equal) to the context."""
    import json
    with open(path) as fh:
        return rs_set_tuning(ctx, **json.load(fh)["tuned"])


def rs_workspace_bytes(ctx: Context) -> int:
    return int(lib().rs_workspace_bytes(ctx.handle))


def mean_spacing(n: int, box: float) -> float:
    return box / math.cbrt(n)
