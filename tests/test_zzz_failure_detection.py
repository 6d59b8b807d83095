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
