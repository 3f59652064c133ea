"""Failure detection of the device-side waits, exercised without hanging or faulting the GPU.

The persistent step kernel (launch modes 1-3) meets at grid-wide barriers whose waits are bounded.
fdtd_set_wait_limit shortens the bound and, as a test hook, makes every barrier wait for one block
more than the launch has: no barrier can complete, so every block gives up after the short bound,
records the sticky error word and returns.  The host must then see FDTD_ETIMEOUT, the context must
be poisoned (FDTD_ESTATE afterwards), later persistent launches must do nothing, and the GPU must
stay usable for a fresh context.
"""
import numpy as np
import pytest
import torch

from paper_2609_30039_gb300 import build as B
from paper_2609_30039_gb300 import fdtd
from paper_2609_30039_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    fdtd.load()


def _scene():
    sc = W.cpml_blocks(n=24, d=4, n_steps=700, block=4, region=(6, 18), wavelengths=(8.0, 10.0))
    sc.sources[0].wave = W.gaussian_pulse(700, wavelength=10.0, periods=1.0, delay=3.0)
    return sc


@pytest.mark.parametrize("n_steps", [8, 600])   # one persistent launch; two (the second must do nothing)
def test_barrier_wait_runs_out_reports_timeout_and_poisons(n_steps):
    ctx = fdtd.Context([_scene()], dtype="f32")
    fdtd.fdtd_set_launch_mode(ctx.ctx, 1)
    fdtd.fdtd_set_wait_limit(ctx.ctx, 4096, 1)   # ~0.3 ms per wait; no barrier can complete
    ctx.step(n_steps)
    with pytest.raises(fdtd.FdtdError) as e:
        ctx.synchronize(timeout_ms=120000)
    assert e.value.status == fdtd.FDTD_ETIMEOUT, fdtd.fdtd_last_error(ctx.ctx)
    assert "barrier" in fdtd.fdtd_last_error(ctx.ctx)
    with pytest.raises(fdtd.FdtdError) as e:
        ctx.step(1)
    assert e.value.status == fdtd.FDTD_ESTATE
    ctx.close()
    torch.cuda.synchronize()   # the CUDA context itself is intact


def test_short_limit_without_the_hook_still_steps_correctly():
    """A short (but sufficient) wait bound changes nothing: persistent steps stay bitwise equal to
    the per-cell steps, and the sticky word stays clear."""
    sc = _scene()
    out = []
    for mode, limit in ((4, None), (1, 1 << 22)):
        ctx = fdtd.Context([sc], dtype="f32")
        fdtd.fdtd_set_launch_mode(ctx.ctx, mode)
        if limit:
            fdtd.fdtd_set_wait_limit(ctx.ctx, limit, 0)
        ctx.step(64)
        ctx.synchronize()
        out.append(np.concatenate([ctx.field(0, c).cpu().numpy().ravel() for c in range(6)]))
        ctx.close()
    assert np.array_equal(out[0], out[1])


def test_wait_limit_arguments_are_checked():
    ctx = fdtd.Context([_scene()], dtype="f32")
    for polls, extra in ((0, 0), (10, 2), (10, -1)):
        with pytest.raises(fdtd.FdtdError) as e:
            fdtd.fdtd_set_wait_limit(ctx.ctx, polls, extra)
        assert e.value.status == fdtd.FDTD_EINVAL
    ctx.close()
