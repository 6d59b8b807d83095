"""Failure detection without a GPU fault: a bounded device wait on a flag
that nothing sets runs out, the synchronising call reports RS_ERR_TIMEOUT
from the device status word, and the same context then runs the path
correctly.  Nothing traps, faults or hangs."""
import numpy as np
import pytest

import oracle
from paper_1110_4372_gb300 import synth

from gpu_util import cuda_inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RS_ERR_TIMEOUT = 4


def test_bounded_wait_times_out_and_the_context_survives():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1110_4372_gb300 import rsgpu
    ctx = rsgpu.Context()
    with pytest.raises(rsgpu.RsError) as e:
        rsgpu.rs_selftest_wait(ctx, False, 20000)
    assert e.value.status == RS_ERR_TIMEOUT
    rsgpu.rs_selftest_wait(ctx, True, 20000)  # the flag is set: no timeout, status clear
    c = synth.generate("c1")
    pos, _ = cuda_inputs(c)
    lab, _, _ = rsgpu.rs_fof3d(ctx, pos, c.box, 0.28)
    ref, _, _ = oracle.fof3d(c.pos, c.box, 0.28)
    assert np.array_equal(lab.cpu().numpy(), ref)


# ---- host-side fault injection (RS_FAULT=<site>) and corrupt inputs ----
RS_ERR_INVALID_ARG, RS_ERR_OOM = 1, 3


@pytest.fixture()
def fault(monkeypatch):
    """Sets RS_FAULT for one test; the library reads it at each fault site,
    so clearing it restores normal operation in the same process."""
    def set_fault(site):
        if site:
            monkeypatch.setenv("RS_FAULT", site)
        else:
            monkeypatch.delenv("RS_FAULT", raising=False)
    yield set_fault
    monkeypatch.delenv("RS_FAULT", raising=False)


def _c1_checked(rsgpu, ctx, c):
    pos, vel = cuda_inputs(c)
    hid, _, _ = rsgpu.rs_find_halos(ctx, pos, vel, c.box)
    o = oracle.run_all(c.pos, c.vel, c.box)
    assert np.array_equal(hid.cpu().numpy(), o["halo_id"])


def test_injected_allocation_failure(fault):
    """Every workspace allocation fails: a fresh context reports RS_ERR_OOM
    with the injected message; without the fault the same context works."""
    from paper_1110_4372_gb300 import rsgpu
    c = synth.generate("c1")
    ctx = rsgpu.Context()
    fault("alloc")
    pos, vel = cuda_inputs(c)
    with pytest.raises(rsgpu.RsError) as e:
        rsgpu.rs_fof3d(ctx, pos, c.box, 0.28, want_groups=True)
    assert e.value.status == RS_ERR_OOM and "RS_FAULT=alloc" in str(e.value)
    fault(None)
    _c1_checked(rsgpu, ctx, c)


def test_injected_timeout_bound(fault):
    """The 3D FOF label pass runs with a bound of one step per find: its
    bounded loops run out, the synchronising call reports RS_ERR_TIMEOUT, and
    the context then runs the whole path correctly."""
    from paper_1110_4372_gb300 import rsgpu
    c = synth.generate("c1")
    ctx = rsgpu.Context()
    pos, vel = cuda_inputs(c)
    fault("timeout1")
    with pytest.raises(rsgpu.RsError) as e:
        rsgpu.rs_fof3d(ctx, pos, c.box, 0.28, want_groups=True)
    assert e.value.status == RS_ERR_TIMEOUT
    with pytest.raises(rsgpu.RsError) as e:
        rsgpu.rs_find_halos(ctx, pos, vel, c.box)
    assert e.value.status == RS_ERR_TIMEOUT
    fault(None)
    _c1_checked(rsgpu, ctx, c)


def test_injected_corrupt_group_offsets(fault):
    """rs_find_halos passes a decreasing group boundary to the refinement,
    whose argument check reports RS_ERR_INVALID_ARG."""
    from paper_1110_4372_gb300 import rsgpu
    c = synth.generate("c1")
    ctx = rsgpu.Context()
    pos, vel = cuda_inputs(c)
    fault("offsets")
    with pytest.raises(rsgpu.RsError) as e:
        rsgpu.rs_find_halos(ctx, pos, vel, c.box)
    assert e.value.status == RS_ERR_INVALID_ARG
    fault(None)
    _c1_checked(rsgpu, ctx, c)


def test_corrupt_offsets_and_members_are_rejected():
    """Decreasing offsets, offsets beyond n and member indices outside
    [0, n) passed to rs_refine6d give RS_ERR_INVALID_ARG (the member check
    runs on the device; every load it guards is clamped into range), and the
    context stays usable."""
    from paper_1110_4372_gb300 import rsgpu
    c = synth.generate("c1")
    ctx = rsgpu.Context()
    pos, vel = cuda_inputs(c)
    labels, _, _ = rsgpu.rs_fof3d(ctx, pos, c.box, 0.28)
    perm, off = rsgpu.rs_group_sort(ctx, labels, 10)
    assert off.numel() > 3
    bad = off.clone()
    bad[2] = bad[1] - 1
    with pytest.raises(rsgpu.RsError) as e:
        rsgpu.rs_refine6d(ctx, pos, vel, c.box, perm, bad)
    assert e.value.status == RS_ERR_INVALID_ARG
    big = off.clone()
    big[-1] = c.n + 5
    with pytest.raises(rsgpu.RsError) as e:
        rsgpu.rs_refine6d(ctx, pos, vel, c.box, perm, big)
    assert e.value.status == RS_ERR_INVALID_ARG
    wild = perm.clone()
    wild[3] = c.n + 7
    wild[5] = -2
    with pytest.raises(rsgpu.RsError) as e:
        rsgpu.rs_refine6d(ctx, pos, vel, c.box, wild, off)
    assert e.value.status == RS_ERR_INVALID_ARG
    _c1_checked(rsgpu, ctx, c)
