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
