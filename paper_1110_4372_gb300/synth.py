"""Seeded synthetic particle catalogues for the halo-finding path.

A catalogue is a periodic box of side ``box`` (Mpc/h) holding a uniform
background plus NFW halos, with float32 positions in [0, box) and float32
velocities in km/s, shuffled into random order. The halo content follows the
workloads the ROCKSTAR paper runs on (cosmological boxes at z = 0, Sec. 4.1,
Table 1), at the sizes of the benchmark configurations:

* halo particle counts n from dN/dn ~ n^-1.9 on [nmin, nmax] (inverse CDF);
* NFW radial profile with enclosed-mass shape m(x) = ln(1+x) - x/(1+x)
  (the same f(x) as Eq. 9 of the paper), concentration c ~ U[5, 15], virial
  radius R from an overdensity of 360 times the background (Sec. 3.3);
* isotropic directions; Maxwellian internal velocities with a per-axis
  dispersion 300 km/s * (n / 4000)^(1/3); host bulk velocity N(0, 300) per axis;
* optional subhalos (1-8 per host, each 1-10% of the host's particles, carved
  out of it, at r/R ~ U[0.1, 1], bulk offset N(0, 0.5 sigma_host) per axis) and
  sub-subhalos (2 per subhalo of >= 2000 particles, same rules);
* background: uniform positions, velocities N(0, 20 km/s) per axis; it holds
  whatever the halos leave of the requested particle count.

This module only draws inputs. It contains no step of the halo finder, and both
the CUDA path and the oracle receive the arrays it returns.
"""
from __future__ import annotations

import dataclasses
import numpy as np

BASE_SEED = 11104372

# name -> (particles, box side in Mpc/h, host halos, nmin, nmax, subhalo depth)
CONFIGS = {
    "c1": dict(n=32768, box=10.0, n_halos=40, nmin=20, nmax=4000, sub_levels=0),
    "c2": dict(n=2097152, box=40.0, n_halos=2500, nmin=20, nmax=200_000, sub_levels=1),
    "c3": dict(n=134217728, box=160.0, n_halos=150_000, nmin=20, nmax=1_000_000, sub_levels=2),
    "c5": dict(n=1073741824, box=320.0, n_halos=1_200_000, nmin=20, nmax=1_000_000, sub_levels=2),
    # the 134M-particle workload at one eighth of its volume (same density,
    # same mass function and hierarchy): a profiling-size case
    "c3q": dict(n=16777216, box=80.0, n_halos=18_750, nmin=20, nmax=1_000_000, sub_levels=2),
}
CONFIG_INDEX = {"c1": 1, "c2": 2, "c3": 3, "c5": 5, "c3q": 6}

DELTA_VIR = 360.0          # overdensity used for the generated halos' radii
N_C_LEVELS = 256           # concentration drawn from 256 equally spaced values in [5, 15]
N_U_GRID = 4096            # inverse-CDF table resolution (in sqrt(u))


@dataclasses.dataclass
class Catalogue:
    pos: np.ndarray        # (N, 3) float32 in [0, box)
    vel: np.ndarray        # (N, 3) float32, km/s
    box: float
    truth: np.ndarray      # (N,) int32 generating component id, -1 = background
    comp_parent: np.ndarray  # (n_comp,) int32 parent component, -1 for hosts
    comp_n: np.ndarray     # (n_comp,) int64 particles drawn for each component
    comp_center: np.ndarray | None = None  # (n_comp, 3) float64 generating centre (not wrapped)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _m_nfw(x):
    return np.log1p(x) - x / (1.0 + x)


def _inverse_cdf_table():
    """x(c_level, s) with s = sqrt(u): radius in units of r_s such that the
    NFW mass inside x is a fraction u of the mass inside c."""
    cs = np.linspace(5.0, 15.0, N_C_LEVELS)
    s = np.linspace(0.0, 1.0, N_U_GRID + 1)
    table = np.empty((N_C_LEVELS, N_U_GRID + 1))
    xs = np.concatenate([[0.0], np.geomspace(1e-7, 1.0, 20000)])
    for j, c in enumerate(cs):
        xg = xs * c
        frac = _m_nfw(xg) / _m_nfw(c)
        table[j] = np.interp(s * s, frac, xg)
    return cs, table


def _power_law_counts(rng, k, nmin, nmax, slope=1.9):
    a = nmin ** (1.0 - slope)
    b = (nmax + 1.0) ** (1.0 - slope)
    u = rng.random(k)
    x = (a - u * (a - b)) ** (1.0 / (1.0 - slope))
    return np.clip(np.floor(x).astype(np.int64), nmin, nmax)


def _sigma1d(n):
    return 300.0 * (np.asarray(n, dtype=np.float64) / 4000.0) ** (1.0 / 3.0)


def _virial_radius(n, nbar):
    return (3.0 * np.asarray(n, dtype=np.float64) / (4.0 * np.pi * DELTA_VIR * nbar)) ** (1.0 / 3.0)


def _isotropic(rng, k):
    d = rng.standard_normal((k, 3))
    nrm = np.linalg.norm(d, axis=1, keepdims=True)
    nrm[nrm == 0] = 1.0
    return d / nrm


def _components(rng, cfg, nbar):
    """Component table: hosts, then subhalos, then sub-subhalos."""
    box = cfg["box"]
    nh = cfg["n_halos"]
    host_n = _power_law_counts(rng, nh, cfg["nmin"], cfg["nmax"])
    comp_n = [host_n.copy()]
    comp_parent = [np.full(nh, -1, np.int64)]
    comp_center = [rng.random((nh, 3)) * box]
    comp_bulk = [rng.standard_normal((nh, 3)) * 300.0]
    comp_mass = [host_n.astype(np.float64)]         # particle count before carving
    level_start = [0]
    total = nh
    for depth in range(cfg["sub_levels"]):
        par_first = level_start[-1]
        par_n_orig = comp_mass[-1]
        n_par = par_n_orig.shape[0]
        if depth == 0:
            k_per = rng.integers(1, 9, size=n_par)            # 1-8 subhalos per host
        else:
            k_per = np.where(par_n_orig >= 2000, 2, 0)         # 2 per subhalo of >= 2000
        parent_local = np.repeat(np.arange(n_par), k_per)
        frac = rng.uniform(0.01, 0.10, size=parent_local.shape[0])
        sub_n = np.floor(frac * par_n_orig[parent_local]).astype(np.int64)
        keep = sub_n >= 10
        parent_local = parent_local[keep]
        sub_n = sub_n[keep]
        k = sub_n.shape[0]
        par_R = _virial_radius(par_n_orig, nbar)[parent_local]
        par_sig = _sigma1d(par_n_orig)[parent_local]
        r = rng.uniform(0.1, 1.0, size=k) * par_R
        centers_par = comp_center[-1][parent_local]
        center = centers_par + _isotropic(rng, k) * r[:, None]
        bulk = comp_bulk[-1][parent_local] + rng.standard_normal((k, 3)) * (0.5 * par_sig)[:, None]
        # carve the subhalos' particles out of their parents
        carve = np.bincount(parent_local, weights=sub_n, minlength=n_par).astype(np.int64)
        comp_n[-1] = comp_n[-1] - carve
        level_start.append(total)
        comp_n.append(sub_n)
        comp_parent.append(parent_local + par_first)
        comp_center.append(center)
        comp_bulk.append(bulk)
        comp_mass.append(sub_n.astype(np.float64))
        total += k
    return (np.concatenate(comp_n), np.concatenate(comp_parent),
            np.concatenate(comp_center), np.concatenate(comp_bulk),
            np.concatenate(comp_mass))


def _wrap32(x64, box):
    x = np.mod(x64, box).astype(np.float32)
    x[x >= np.float32(box)] = np.float32(0.0)
    x[x < 0] = np.float32(0.0)
    return x


def generate(name: str = "c1", *, seed: int | None = None, n: int | None = None,
             box: float | None = None, n_halos: int | None = None,
             chunk: int = 1 << 23) -> Catalogue:
    """Draw the catalogue of configuration ``name`` (c1, c2, c3, c5).

    ``seed`` defaults to 11104372 + the configuration's index. ``n``, ``box``
    and ``n_halos`` override the configuration (keeping the mean density
    fixed is the caller's business)."""
    cfg = dict(CONFIGS[name])
    if n is not None:
        cfg["n"] = int(n)
    if box is not None:
        cfg["box"] = float(box)
    if n_halos is not None:
        cfg["n_halos"] = int(n_halos)
    if seed is None:
        seed = BASE_SEED + CONFIG_INDEX[name]
    rng = np.random.Generator(np.random.PCG64(seed))
    N = cfg["n"]
    L = float(np.float32(cfg["box"]))  # the box side is a float32 value
    nbar = N / L ** 3
    comp_n, comp_parent, comp_center, comp_bulk, comp_mass = _components(rng, cfg, nbar)
    n_halo_particles = int(comp_n.sum())
    if n_halo_particles > N:
        raise ValueError(f"halos need {n_halo_particles} particles, only {N} requested")
    cs, table = _inverse_cdf_table()
    n_comp = comp_n.shape[0]
    c_level = rng.integers(0, N_C_LEVELS, size=n_comp)
    R = _virial_radius(comp_mass, nbar)
    sig = _sigma1d(comp_mass)

    pos = np.empty((N, 3), np.float32)
    vel = np.empty((N, 3), np.float32)
    truth = np.empty(N, np.int32)
    ends = np.cumsum(comp_n)
    starts = ends - comp_n
    # halo particles, in chunks of whole components
    c0 = 0
    while c0 < n_comp:
        c1 = int(np.searchsorted(ends, starts[c0] + chunk, side="right"))
        c1 = max(c1, c0 + 1)
        ids = np.repeat(np.arange(c0, c1), comp_n[c0:c1])
        k = ids.shape[0]
        p0 = int(starts[c0])
        s = np.sqrt(rng.random(k)) * N_U_GRID
        i0 = np.minimum(s.astype(np.int64), N_U_GRID - 1)
        w = s - i0
        lev = c_level[ids]
        x = table[lev, i0] * (1.0 - w) + table[lev, i0 + 1] * w
        r = R[ids] * x / cs[lev]
        p = comp_center[ids] + _isotropic(rng, k) * r[:, None]
        v = comp_bulk[ids] + rng.standard_normal((k, 3)) * sig[ids][:, None]
        pos[p0:p0 + k] = _wrap32(p, L)
        vel[p0:p0 + k] = v.astype(np.float32)
        truth[p0:p0 + k] = ids.astype(np.int32)
        c0 = c1
    # background
    p0 = n_halo_particles
    while p0 < N:
        k = min(chunk, N - p0)
        pos[p0:p0 + k] = _wrap32(rng.random((k, 3)) * L, L)
        vel[p0:p0 + k] = (rng.standard_normal((k, 3)) * 20.0).astype(np.float32)
        truth[p0:p0 + k] = -1
        p0 += k
    perm = rng.permutation(N)
    pos = pos[perm]
    vel = vel[perm]
    truth = truth[perm]
    return Catalogue(pos=np.ascontiguousarray(pos), vel=np.ascontiguousarray(vel), box=L,
                     truth=truth, comp_parent=comp_parent.astype(np.int32),
                     comp_n=comp_n, comp_center=comp_center)


# Independent 6D groups for the batching stress workload: sizes log-uniform
# on [nmin, nmax]; each group an NFW host with 0-max_subs co-spatial subhalos
# (same centre, each 1-10% of the host's particles, bulk velocity offset by
# U[1, 3] sigma_host in an isotropic direction).  Radii and dispersions use
# the density of the benchmark boxes (32^3 particles per 10 Mpc/h cube).
GROUP_CONFIGS = {
    "c4": dict(n_groups=200_000, nmin=20, nmax=500_000, max_subs=12),
    "c4s": dict(n_groups=2_000, nmin=20, nmax=20_000, max_subs=12),  # small case of the same recipe
}
GROUP_NBAR = 32768 / 10.0 ** 3
GROUP_BOX = 1000.0


@dataclasses.dataclass
class GroupCatalogue:
    pos: np.ndarray          # (N, 3) float32 in [0, box), groups back to back
    vel: np.ndarray          # (N, 3) float32, km/s
    box: float
    offsets: np.ndarray      # (n_groups + 1,) int64: group g is rows offsets[g]:offsets[g+1]
    truth: np.ndarray        # (N,) int32: 0 for the host, k for the group's k-th subhalo

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _group_rng_and_size(g, cfg, seed):
    """Group g's substream and its particle count, the substream's first draw."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, g])))
    n = int(np.exp(rng.uniform(np.log(cfg["nmin"]), np.log(cfg["nmax"] + 1.0))))
    return rng, min(max(n, cfg["nmin"]), cfg["nmax"])


def _group(g, cfg, seed, cs, table):
    """One group from its own substream (so groups can be drawn in any chunks)."""
    rng, n = _group_rng_and_size(g, cfg, seed)
    k = int(rng.integers(0, cfg["max_subs"] + 1))
    sub_n = np.floor(rng.uniform(0.01, 0.10, size=k) * n).astype(np.int64)
    sub_n = sub_n[sub_n >= 10]
    host_n = n - int(sub_n.sum())
    counts = np.concatenate([[host_n], sub_n]).astype(np.int64)
    masses = np.concatenate([[n], sub_n]).astype(np.float64)
    centre = rng.random(3) * GROUP_BOX
    sig_host = _sigma1d(n)
    bulk = np.zeros((len(counts), 3))
    bulk[0] = rng.standard_normal(3) * 300.0
    if len(sub_n):
        dv = _isotropic(rng, len(sub_n)) * (rng.uniform(1.0, 3.0, size=len(sub_n)) * sig_host)[:, None]
        bulk[1:] = bulk[0] + dv
    R = _virial_radius(masses, GROUP_NBAR)
    sig = _sigma1d(masses)
    lev = rng.integers(0, N_C_LEVELS, size=len(counts))
    ids = np.repeat(np.arange(len(counts)), counts)
    m = ids.shape[0]
    sq = np.sqrt(rng.random(m)) * N_U_GRID
    i0 = np.minimum(sq.astype(np.int64), N_U_GRID - 1)
    w = sq - i0
    L = lev[ids]
    x = table[L, i0] * (1.0 - w) + table[L, i0 + 1] * w
    r = R[ids] * x / cs[L]
    p = centre + _isotropic(rng, m) * r[:, None]
    v = bulk[ids] + rng.standard_normal((m, 3)) * sig[ids][:, None]
    perm = rng.permutation(m)
    return p[perm], v[perm], ids[perm].astype(np.int32)


def groups(name: str = "c4s", *, first: int = 0, count: int | None = None,
           seed: int | None = None) -> GroupCatalogue:
    """Groups first .. first+count-1 of the independent-group workload
    ``name`` (all of them by default); any slice equals the same rows of the
    whole draw, so the workload can be streamed in chunks of whole groups."""
    cfg = GROUP_CONFIGS[name]
    if seed is None:
        seed = BASE_SEED + 4
    if count is None:
        count = cfg["n_groups"] - first
    cs, table = _inverse_cdf_table()
    L = float(np.float32(GROUP_BOX))
    parts = [_group(g, cfg, seed, cs, table) for g in range(first, first + count)]
    sizes = np.array([len(q[0]) for q in parts], np.int64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    if count == 0:
        e = np.zeros((0, 3), np.float32)
        return GroupCatalogue(pos=e, vel=e.copy(), box=L, offsets=offsets, truth=np.zeros(0, np.int32))
    pos = _wrap32(np.concatenate([q[0] for q in parts]), L)
    vel = np.concatenate([q[1] for q in parts]).astype(np.float32)
    truth = np.concatenate([q[2] for q in parts])
    return GroupCatalogue(pos=np.ascontiguousarray(pos), vel=np.ascontiguousarray(vel), box=L, offsets=offsets,
                          truth=truth)


def group_sizes(name: str = "c4s", *, first: int = 0, count: int | None = None,
                seed: int | None = None) -> np.ndarray:
    """Particle counts of groups first .. first+count-1 of the workload
    ``name``, without drawing the particles (int64)."""
    cfg = GROUP_CONFIGS[name]
    if seed is None:
        seed = BASE_SEED + 4
    if count is None:
        count = cfg["n_groups"] - first
    return np.array([_group_rng_and_size(g, cfg, seed)[1] for g in range(first, first + count)], np.int64)


def uniform(n: int, box: float, seed: int, vel_sigma: float = 20.0) -> Catalogue:
    """Plain uniform box (no halos), for edge cases and small tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    box = float(np.float32(box))
    pos = _wrap32(rng.random((n, 3)) * box, box)
    vel = (rng.standard_normal((n, 3)) * vel_sigma).astype(np.float32)
    return Catalogue(pos=pos, vel=vel, box=box, truth=np.full(n, -1, np.int32),
                     comp_parent=np.zeros(0, np.int32), comp_n=np.zeros(0, np.int64))


def blob(rng, n, center, bulk, sig_x, sig_v):
    """Isotropic Gaussian blob in 6D (float64 arrays, not wrapped)."""
    p = np.asarray(center, np.float64) + rng.standard_normal((n, 3)) * sig_x
    v = np.asarray(bulk, np.float64) + rng.standard_normal((n, 3)) * sig_v
    return p, v


def wrap(pos64, box):
    """Wrap float64 positions into float32 [0, box)."""
    return _wrap32(np.asarray(pos64, np.float64), box)
