"""The allocation-free non-finite count, called through the C ABI, against the context's
existing finite check (fdtd_check_finite) on consecutive calls.

The allocation-free entry point exists for callers that cannot allocate device memory (their
memory is owned by a caching allocator or a fixed budget); it shares one file-scope scratch
array between calls, so consecutive calls must not see each other's counts.  This file is
collected last so that a run stopping at the first failure has run every other test first."""
import numpy as np
import pytest
import torch

from paper_2609_30039_gb300 import build as B
from paper_2609_30039_gb300 import fdtd
from paper_2609_30039_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    B.build()
    fdtd.load()
    sc = W.cpml_blocks(n=24, d=4, n_steps=30, block=4, region=(6, 18), wavelengths=(8.0, 10.0))
    sc.sources[0].wave = W.gaussian_pulse(30, wavelength=10.0, periods=1.0, delay=3.0)
    c = fdtd.Context([sc], dtype="f32")
    c.step(30)
    torch.cuda.synchronize()
    yield c
    c.close()


def _existing_says_finite(c):
    try:
        fdtd.fdtd_check_finite(c.ctx)
        return True
    except fdtd.FdtdError as e:
        assert e.status == fdtd.FDTD_ENONFINITE
        return False


def _noalloc_counts(c):
    stream = c.stream.cuda_stream
    total = 0
    for p in range(c.part_count(0)):
        t = c.part(0, p)
        if t.numel():
            total += fdtd.fdtd_count_nonfinite_noalloc(t.data_ptr(), t.numel(), fdtd.FDTD_F32, stream)
    return total


def test_noalloc_count_agrees_with_existing_check_on_consecutive_calls(ctx):
    # call 1: the finite state
    assert _existing_says_finite(ctx)
    assert _noalloc_counts(ctx) == 0
    # call 2: plant NaN / Inf values on the host side of the state and count them
    ez = ctx.part(0, 2).clone()
    idx = torch.tensor([3, 777, 5000, 9999, 13000], device=ez.device)
    ez[idx[:3]] = float("nan")
    ez[idx[3:]] = float("inf") * torch.tensor([1.0, -1.0], device=ez.device)
    ctx.set_part(0, 2, ez)
    assert not _existing_says_finite(ctx)
    assert _noalloc_counts(ctx) == 5 == int((~torch.isfinite(ez)).sum())
    # call 3: restore a finite state; the shared scratch must not carry the previous count
    ez[idx] = 0.0
    ctx.set_part(0, 2, ez)
    assert _existing_says_finite(ctx)
    assert _noalloc_counts(ctx) == 0


def test_noalloc_fp64_and_limits():
    B.build()
    fdtd.load()
    x = torch.zeros(1 << 20, dtype=torch.float64, device="cuda")
    x[12345] = float("nan")
    s = torch.cuda.current_stream().cuda_stream
    assert fdtd.fdtd_count_nonfinite_noalloc(x.data_ptr(), x.numel(), fdtd.FDTD_F64, s) == 1
    assert fdtd.fdtd_count_nonfinite_noalloc(x.data_ptr(), 0, fdtd.FDTD_F64, s) == 0
    with pytest.raises(fdtd.FdtdError) as e:
        fdtd.fdtd_count_nonfinite_noalloc(x.data_ptr(), 33554432 + 1, fdtd.FDTD_F64, s)
    assert e.value.status == fdtd.FDTD_EINVAL
