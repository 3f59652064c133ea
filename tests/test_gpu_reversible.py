"""Reversible reconstruction on the GPU (Sec. 3.2): backward steps of Eq. (yee) for lossless
nondispersive domains, against the FP64 oracle, and the checkpoint-free gradient against the
oracle's replayed one."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import gradient_replay
from paper_2609_30039_gb300 import adjoint as ADJ
from paper_2609_30039_gb300 import fdtd
from paper_2609_30039_gb300 import workloads as W
from tests.oracle_adapter import oracle_from_scene
from tests.test_gpu_parity import _gpu_loss, _oracle_objective, compare_state, rel

pytestmark = pytest.mark.gpu


def lossless_scene(steps=60, aniso=True, design=True):
    """Periodic in x, PEC in y and z, no CPML, no poles: blocky anisotropic eps, an Ez sheet and
    an Hx patch source, a DFT plane of Ex and a design box."""
    nx, ny, nz = 20, 16, 18
    rng = np.random.default_rng(26090)
    inv = [1.0 / np.repeat(np.repeat(np.repeat(rng.uniform(1.0, 5.0, size=(nz // 3, ny // 4, nx // 4)), 3, 0), 4, 1),
                           4, 2) for _ in range(3 if aniso else 1)]
    srcs = [W.Source(W.EZ, (0, 1, 4), (nx, ny, 5), W.gaussian_pulse(steps, wavelength=8.0, periods=1.0, delay=3.0)),
            W.Source(W.HX, (3, 5, 9), (6, 8, 10), W.gaussian_pulse(steps, wavelength=6.0, periods=1.0, delay=2.0))]
    mons = [W.Monitor((0, 1, 13), (nx, ny, 14), (W.EX, W.EZ), W.omegas_for((7.0, 8.0)))]
    sc = W.Scene(shape=(nx, ny, nz), n_steps=steps, cpml=(0,) * 6, inv_eps=inv, sources=srcs, monitors=mons,
                 periodic=(1, 0, 0), name="lossless")
    if design:
        sc.design = ((0, 3, 7), (6, 11, 11))    # straddles the periodic seam x = 0
    return sc


def test_backward_steps_match_oracle_fp64():
    sc = lossless_scene(design=False)
    o = oracle_from_scene(sc)
    o.step(40)
    o.step_backward(15)
    ctx = fdtd.Context([sc], dtype="f64")
    ctx.step(40)
    fdtd.fdtd_step_backward(ctx.ctx, 15)
    assert ctx.step_count == 25
    compare_state(ctx, o, sc, tol=1e-12)
    # and the reconstruction is the forward state of step 25
    o2 = oracle_from_scene(sc)
    o2.step(25)
    compare_state(ctx, o2, sc, tol=1e-11)


def test_reversible_gradient_matches_replayed_oracle_gradient():
    sc = lossless_scene()
    o = oracle_from_scene(sc)
    J_ref = gradient_replay(o, sc.n_steps, _oracle_objective)
    g_ref = np.stack([o.grad(a) for a in range(3)])
    ctx = fdtd.Context([sc], dtype="f64")
    (J, _), grads, stats = ADJ.ReversibleAdjoint(ctx).run(sc.n_steps, _gpu_loss)
    assert abs(J - J_ref) <= 1e-12 * abs(J_ref)
    g = grads[0].cpu().numpy().reshape(g_ref.shape)
    assert rel(g, g_ref) < 1e-10, rel(g, g_ref)
    assert stats["backward_steps"] == sc.n_steps
    # FP32: the reversible and the checkpointed gradient agree to FP32 rounding
    c32 = fdtd.Context([sc], dtype="f32")
    (_, _), g_rev, _ = ADJ.ReversibleAdjoint(c32).run(sc.n_steps, _gpu_loss)
    g_rev = g_rev[0].cpu().numpy().copy()
    c32b = fdtd.Context([sc], dtype="f32")
    (_, _), g_chk, _ = ADJ.DesignAdjoint(c32b, slots=8).run(sc.n_steps, _gpu_loss)
    g_chk = g_chk[0].cpu().numpy()
    assert rel(g_rev, g_chk) < 1e-4, rel(g_rev, g_chk)
    assert rel(g_rev.reshape(g_ref.shape), g_ref) < 1e-4


def test_backward_steps_refuse_lossy_domains_and_step_zero():
    sc = small = W.cpml_blocks(n=24, d=4, n_steps=10, block=4, region=(6, 18), wavelengths=(9.0, 10.0, 11.0))
    ctx = fdtd.Context([small], dtype="f32")
    ctx.step(3)
    with pytest.raises(fdtd.FdtdError) as e:
        fdtd.fdtd_step_backward(ctx.ctx, 1)
    assert e.value.status == fdtd.FDTD_EINVAL
    c2 = fdtd.Context([lossless_scene(design=False)], dtype="f32")
    c2.step(2)
    with pytest.raises(fdtd.FdtdError) as e:
        fdtd.fdtd_step_backward(c2.ctx, 3)
    assert e.value.status == fdtd.FDTD_ESTATE
