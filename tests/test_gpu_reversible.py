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


# ---- absorbing-face variant (Sec. 3.2): interior reconstruction with a recorded interface --------
def cpml_scene(steps=60, design=True):
    """CPML (4 cells) on every face, vacuum absorber, blocky anisotropic eps inside, an Ez sheet and a
    DFT plane inside, a design box inside: the interior reversal's workload."""
    nx, ny, nz, d = 20, 18, 24, 4
    rng = np.random.default_rng(26091)
    inv = []
    for _ in range(3):
        a = np.ones((nz, ny, nx))
        blk = rng.uniform(1.0, 5.0, size=(4, 3, 3))
        a[d:nz - d, d:ny - d, d:nx - d] = 1.0 / np.repeat(np.repeat(np.repeat(blk, 4, 0), 4, 1), 4, 2)[:nz - 2 * d,
                                                                                                     :ny - 2 * d,
                                                                                                     :nx - 2 * d]
        inv.append(a)
    srcs = [W.Source(W.EZ, (d, d, 7), (nx - d, ny - d, 8), W.gaussian_pulse(steps, wavelength=8.0, periods=1.0,
                                                                               delay=3.0))]
    mons = [W.Monitor((d, d, 16), (nx - d, ny - d, 17), (W.EX, W.EZ), W.omegas_for((7.0, 8.0)))]
    sc = W.Scene(shape=(nx, ny, nz), n_steps=steps, cpml=(d,) * 6, kappa_max=3.0, alpha_max=0.05, inv_eps=inv,
                 sources=srcs, monitors=mons, name="cpml_reversible")
    if design:
        sc.design = ((6, 6, 10), (14, 12, 14))
    return sc


def _interior(sc):
    nx, ny, nz = sc.shape
    m = np.zeros((nz, ny, nx), dtype=bool)
    lo = [sc.cpml[2 * q] for q in range(3)]
    hi = [sc.shape[q] - sc.cpml[2 * q + 1] for q in range(3)]
    m[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = True
    return m


def test_interior_backward_steps_with_the_interface_record_match_the_oracle_fp64():
    sc = cpml_scene(steps=40, design=False)
    inner = _interior(sc)
    o = oracle_from_scene(sc)
    states = [o.fields()]
    for _ in range(40):
        o.step(1)
        states.append(o.fields())
    for n in reversed(range(25, 40)):
        o.step_backward_interior(states[n + 1][:3], states[n][3:])
    ctx = fdtd.Context([sc], dtype="f64")
    fdtd.fdtd_record_interface(ctx.ctx, 40)
    ctx.step(40)
    fdtd.fdtd_step_backward(ctx.ctx, 15)
    assert ctx.step_count == 25
    g = np.concatenate([ctx.field(0, c).cpu().numpy()[inner] for c in range(6)])
    r = np.concatenate([f[inner] for f in o.fields()])
    f25 = np.concatenate([f[inner] for f in states[25]])
    assert rel(g, r) <= 1e-12, rel(g, r)
    assert rel(g, f25) <= 1e-11, rel(g, f25)
    # beyond the record's reach: refused
    with pytest.raises(fdtd.FdtdError) as e:
        fdtd.fdtd_step_backward(ctx.ctx, 26)
    assert e.value.status == fdtd.FDTD_ESTATE
    ctx.close()


def test_reversible_gradient_with_absorbing_faces_matches_the_replayed_oracle_gradient():
    sc = cpml_scene()
    o = oracle_from_scene(sc)
    J_ref = gradient_replay(o, sc.n_steps, _oracle_objective)
    g_ref = np.stack([o.grad(a) for a in range(3)])
    ctx = fdtd.Context([sc], dtype="f64")
    (J, _), grads, stats = ADJ.ReversibleAdjoint(ctx).run(sc.n_steps, _gpu_loss)
    assert abs(J - J_ref) <= 1e-12 * abs(J_ref)
    g = grads[0].cpu().numpy().reshape(g_ref.shape)
    print(f"\nreversible (recorded interface) FP64 gradient vs oracle: {rel(g, g_ref):.3e}")
    assert rel(g, g_ref) < 1e-10, rel(g, g_ref)
    ctx.close()
    c32 = fdtd.Context([sc], dtype="f32")
    (_, _), g_rev, _ = ADJ.ReversibleAdjoint(c32).run(sc.n_steps, _gpu_loss)
    g_rev = g_rev[0].cpu().numpy().copy()
    c32b = fdtd.Context([sc], dtype="f32")
    (_, _), g_chk, _ = ADJ.DesignAdjoint(c32b, slots=8).run(sc.n_steps, _gpu_loss)
    g_chk = g_chk[0].cpu().numpy()
    print(f"reversible vs checkpointed FP32 gradient: {rel(g_rev, g_chk):.3e}")
    assert rel(g_rev, g_chk) < 1e-4, rel(g_rev, g_chk)
