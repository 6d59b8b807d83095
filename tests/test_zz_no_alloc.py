"""The no-allocation 3D friends-of-friends entry point (rs_fof3d_static).

It is meant for callers that cannot allocate device memory when they need
groups (a plugin whose host framework owns all device memory through its own
pool, a service with a device memory budget fixed at start-up, a
latency-critical loop).  This test calls it through the C ABI twice in a row,
on two different catalogues, and checks each result against rs_fof3d, the
entry point that allocates its own workspace.  It lives in its own file,
collected last, so a run that stops at the first failure has already run
everything else.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1110_4372_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _static_fn():
    from paper_1110_4372_gb300 import rsgpu
    fn = rsgpu.lib().rs_fof3d_static
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_double, C.c_void_p, C.c_void_p]
    return rsgpu, fn


def test_no_alloc_fof_matches_fof3d_on_two_calls():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    rsgpu, fn = _static_fn()
    ctx = rsgpu.Context()
    stream = torch.cuda.current_stream().cuda_stream
    cats = [synth.generate("c1"),
            synth.generate("c1", seed=4242, n=60000, box=10.0 * (60000 / 32768) ** (1 / 3), n_halos=70)]
    for cat in cats:
        pos = torch.from_numpy(cat.pos).cuda()
        ref, _, _ = rsgpu.rs_fof3d(ctx, pos, cat.box, 0.28)
        out = torch.full((cat.n,), -7, dtype=torch.int32, device="cuda")
        st = fn(C.c_void_p(pos.data_ptr()), 3, cat.n, cat.box, 0.28, C.c_void_p(out.data_ptr()), C.c_void_p(stream))
        assert st == 0
        assert torch.equal(out, ref)
        assert int(out.max()) < cat.n and int(out.min()) >= 0


def test_no_alloc_fof_rejects_oversize():
    rsgpu, fn = _static_fn()
    n = 65537
    pos = torch.rand((n, 3), device="cuda") * 20.0
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    st = fn(C.c_void_p(pos.data_ptr()), 3, n, 20.0, 0.28, C.c_void_p(out.data_ptr()), None)
    assert st == 5  # RS_ERR_TOO_LARGE
    assert fn(C.c_void_p(pos.data_ptr()), 3, 1000, 20.0, 0.01, C.c_void_p(out.data_ptr()), None) == 5


def test_no_alloc_fof_leaves_device_memory_unchanged():
    """After the first call on the device (which loads the library's device
    code and its scratch array), further calls change the device's free
    memory by nothing: they allocate nothing."""
    rsgpu, fn = _static_fn()
    cat = synth.generate("c1", seed=77, n=20000, box=10.0 * (20000 / 32768) ** (1 / 3), n_halos=20)
    pos = torch.from_numpy(cat.pos).cuda()
    out = torch.empty(cat.n, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = (C.c_void_p(pos.data_ptr()), 3, cat.n, cat.box, 0.28, C.c_void_p(out.data_ptr()), stream)
    assert fn(*args) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert fn(*args) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ctx = rsgpu.Context()
    ref, _, _ = rsgpu.rs_fof3d(ctx, pos, cat.box, 0.28)
    assert torch.equal(out, ref)
