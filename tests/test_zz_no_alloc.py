"""bp_residual_noalloc against bp_residual.

The no-allocation variant serves callers that cannot let the library
allocate device memory during the call (a thread that does not own the
context's allocator, or a run whose device memory is fully committed).  On a
fresh context it must run before anything has allocated the residual's
scratch, leave the allocator untouched, and give the same residual as the
allocating entry point -- also on a second call, whose static scratch still
holds the first call's values.  This file is collected last so that a failure
here comes after every other test.
"""
import numpy as np
import pytest

from paper_2208_08038_gb300 import synth

pytestmark = pytest.mark.gpu


def _context():
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from _common import gpu_from_workload
    wl = synth.ionized_crystal_2d(n=(256, 64), span=(2.0, 6.0), steps=10, a0=0.3)
    return gpu_from_workload(wl, deposit_mode=1)[0]


def test_noalloc_residual_matches_allocating_entry_point():
    import torch
    assert torch.cuda.is_available()
    ctx = _context()  # fresh: bp_residual has never run on it
    for call in range(2):
        ctx.step(3)
        ctx.sync()
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        peak_before = torch.cuda.max_memory_allocated()
        got = ctx.residual_noalloc()
        torch.cuda.synchronize()
        # the context allocates only through torch's caching allocator: no
        # block was taken, not even a transient one
        assert torch.cuda.memory_allocated() == before, call
        assert torch.cuda.max_memory_allocated() == peak_before, call
        ref = ctx.residual()
        scale = np.abs(ref).max()
        assert scale > 0
        # the same FP64 sums; only the order of the FP64 atomic adds differs
        assert np.abs(got - ref).max() <= 1e-12 * scale, call
    ctx.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_2208_08038_gb300 import binding as B
    ctx = B.Context(2, (4096, 2048), (0.2, 0.2), 0.1, (1, 0))
    with pytest.raises(B.BPError) as e:
        ctx.residual_noalloc()
    assert e.value.code == B.BP_ERR_ARG
    ctx.close()
