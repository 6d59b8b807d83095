"""The seeded generator: determinism, ranges and the requested structure."""
import numpy as np

from paper_1110_4372_gb300 import synth


def test_deterministic_and_in_range():
    a = synth.generate("c1")
    b = synth.generate("c1")
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.vel, b.vel)
    assert a.pos.dtype == np.float32 and a.pos.shape == (32768, 3)
    assert a.pos.min() >= 0 and a.pos.max() < a.box
    c = synth.generate("c1", seed=123)
    assert not np.array_equal(a.pos, c.pos)


def test_halo_counts_follow_config():
    c = synth.generate("c2")
    hosts = np.flatnonzero(c.comp_parent < 0)
    assert len(hosts) == 2500
    subs = np.flatnonzero(c.comp_parent >= 0)
    assert 0 < len(subs) <= 8 * 2500  # 1-8 per host, minus those under 10 particles
    assert c.comp_n[subs].min() >= 10
    assert (c.truth >= 0).sum() == c.comp_n.sum()


def test_independent_groups_recipe_and_chunks():
    """The batching-stress groups: sizes log-uniform in range, 0-12
    co-spatial subhalos moving at 1-3 sigma_host, and any chunk of groups
    equal to the same rows of the whole draw."""
    whole = synth.groups("c4s", count=300)
    sizes = np.diff(whole.offsets)
    assert sizes.min() >= 20 and sizes.max() <= 20_000
    # log-uniform: about half the groups below the geometric midpoint
    mid = np.sqrt(20 * 20_000)
    assert 0.4 < np.mean(sizes < mid) < 0.6
    assert whole.pos.min() >= 0 and whole.pos.max() < whole.box
    part = synth.groups("c4s", first=100, count=50)
    a, b = whole.offsets[100], whole.offsets[150]
    assert np.array_equal(part.pos, whole.pos[a:b]) and np.array_equal(part.vel, whole.vel[a:b])
    assert np.array_equal(part.offsets, whole.offsets[100:151] - a)
    n_subs = [len(np.unique(whole.truth[whole.offsets[g]:whole.offsets[g + 1]])) - 1 for g in range(300)]
    assert min(n_subs) >= 0 and max(n_subs) <= 12 and np.mean(n_subs) > 2
    # a subhalo shares the host's centre; its bulk velocity is offset by 1-3 sigma_host
    checked = 0
    for g in range(300):
        s0, s1 = whole.offsets[g], whole.offsets[g + 1]
        t = whole.truth[s0:s1]
        if t.max() == 0 or sizes[g] < 5000:
            continue
        p, v = whole.pos[s0:s1].astype(np.float64), whole.vel[s0:s1].astype(np.float64)
        host_c = np.median(p[t == 0], axis=0)
        sig = 300.0 * (sizes[g] / 4000.0) ** (1 / 3)
        for k in np.unique(t[t > 0]):
            sel = t == k
            if sel.sum() < 200:
                continue
            assert np.linalg.norm(np.median(p[sel], axis=0) - host_c) < 0.5 * np.abs(p[t == 0] - host_c).max()
            dv = np.linalg.norm(v[sel].mean(0) - v[t == 0].mean(0)) / sig
            assert 0.7 < dv < 3.3
            checked += 1
    assert checked >= 3


def test_group_sizes_without_drawing_particles():
    """The size-only draw equals the sizes of the drawn groups (the streamed
    batching benchmark plans its chunks from it)."""
    g = synth.groups("c4s", first=17, count=9)
    assert np.array_equal(synth.group_sizes("c4s", first=17, count=9), np.diff(g.offsets))
    s = synth.group_sizes("c4", first=0, count=2000)
    assert s.min() >= 20 and s.max() <= 500_000


def test_recipe_mass_function_nfw_profile_and_velocities():
    """The catalogue recipe: host counts follow dN/dn ∝ n^-1.9 (the
    discretised inverse CDF), a host's particles follow the NFW enclosed
    mass of a concentration in [5, 15] inside its virial radius, and halo
    and background velocities have the stated dispersions."""
    rng = np.random.Generator(np.random.PCG64(5))
    nmin, nmax = 20, 200_000
    n = synth._power_law_counts(rng, 200_000, nmin, nmax)
    a = 1.0 - 1.9
    for m in (20, 25, 40, 100, 1000, 20_000):
        cdf = (nmin ** a - (m + 1.0) ** a) / (nmin ** a - (nmax + 1.0) ** a)
        assert abs(np.mean(n <= m) - cdf) < 0.005, m

    c = synth.generate("c2")
    hosts = np.flatnonzero(c.comp_parent < 0)
    orig = c.comp_n.astype(np.float64).copy()
    np.add.at(orig, c.comp_parent[c.comp_parent >= 0], c.comp_n[c.comp_parent >= 0])
    nbar = c.n / c.box ** 3
    m_nfw = lambda x: np.log1p(x) - x / (1.0 + x)  # noqa: E731
    checked = 0
    for h in hosts[np.argsort(c.comp_n[hosts])[::-1][:5]]:
        sel = c.truth == h
        d = c.pos[sel].astype(np.float64) - c.comp_center[h]
        d -= c.box * np.round(d / c.box)
        q = np.linalg.norm(d, axis=1) / (3.0 * orig[h] / (4.0 * np.pi * 360.0 * nbar)) ** (1.0 / 3.0)
        assert q.max() <= 1.0 + 1e-4
        for r in (0.1, 0.3, 0.6):
            emp = np.mean(q <= r)
            lo, hi = m_nfw(5 * r) / m_nfw(5.0), m_nfw(15 * r) / m_nfw(15.0)
            tol = 4.0 / np.sqrt(sel.sum())
            assert lo - tol <= emp <= hi + tol, (h, r, emp, lo, hi)
        sig = np.std(c.vel[sel].astype(np.float64), axis=0)
        assert np.all(np.abs(sig / (300.0 * (orig[h] / 4000.0) ** (1.0 / 3.0)) - 1.0) < 6.0 / np.sqrt(sel.sum()) + 0.01)
        checked += 1
    assert checked == 5
    bg = c.truth < 0
    assert abs(np.std(c.vel[bg].astype(np.float64)) / 20.0 - 1.0) < 0.01
