"""Pole-parameter gradients on the GPU (Sec. 3.1: Drude and Lorentz pole parameters differentiate
through the transposed dispersion update), through the C ABI, against the FP64 oracle (whose own
pole gradients are pinned by central differences)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import gradient_replay
from paper_2609_30039_gb300 import adjoint as ADJ
from paper_2609_30039_gb300 import fdtd
from paper_2609_30039_gb300 import workloads as W
from tests.oracle_adapter import oracle_from_scene
from tests.test_gpu_parity import _design_scene, _gpu_loss, _oracle_objective, rel

pytestmark = pytest.mark.gpu


def _oracle_pole_grad(sc):
    o = oracle_from_scene(sc)
    J = gradient_replay(o, sc.n_steps, _oracle_objective)
    return J, o.pole_grad(), np.stack([o.grad(a) for a in range(3)]) if sc.design is not None else None


@pytest.mark.parametrize("slots", [4, 70])
def test_pole_grads_fp64_match_oracle(slots):
    sc = _design_scene(True)
    J_ref, pg_ref, g_ref = _oracle_pole_grad(sc)
    ctx = fdtd.Context([sc], dtype="f64")
    adj = ADJ.DesignAdjoint(ctx, slots=slots, pole_grads=True)
    (J, _), grads, _ = adj.run(sc.n_steps, _gpu_loss)
    assert abs(J - J_ref) <= 1e-12 * abs(J_ref)
    pg = adj.pole_grads[0]
    assert pg.shape == (2, 3) and pg[1, 0] == 0.0
    assert np.max(np.abs(pg - pg_ref)) <= 1e-10 * np.max(np.abs(pg_ref)), (pg, pg_ref)
    # the material cotangent is unchanged by collecting the pole cotangents
    assert rel(grads[0].cpu().numpy().reshape(g_ref.shape), g_ref) < 1e-10


def test_pole_grads_fp32_close_to_oracle_and_leave_eps_gradient_bitwise():
    sc = _design_scene(True)
    _, pg_ref, _ = _oracle_pole_grad(sc)
    out = {}
    for on in (False, True):
        ctx = fdtd.Context([sc], dtype="f32")
        adj = ADJ.DesignAdjoint(ctx, slots=8, pole_grads=on)
        (_, _), grads, _ = adj.run(sc.n_steps, _gpu_loss)
        out[on] = (grads[0].clone(), adj.pole_grads.get(0))
        ctx.close()
    assert torch.equal(out[False][0], out[True][0])
    pg = out[True][1]
    assert np.max(np.abs(pg - pg_ref)) <= 1e-4 * np.max(np.abs(pg_ref)), (pg, pg_ref)


def test_pole_grads_of_two_batched_domains():
    # two dispersive domains of different shapes and poles in one context: each domain's pole
    # cotangents are its own (J is the sum of the per-domain objectives)
    scs = W.lorentz_batch(n_domains=2, sizes=(20, 24), d=4, n_steps=80)
    for sc in scs:
        sc.sources[0].wave = W.gaussian_pulse(80, 8.0, periods=1, delay=3)
        sc.monitors[0].omegas = W.omegas_for((7.0, 9.0))
    ctx = fdtd.Context(scs, dtype="f64")
    adj = ADJ.DesignAdjoint(ctx, slots=10, pole_grads=True)

    def loss(specs):
        J = sum(float((F.abs() ** 2).sum()) for F in specs)
        return J, [torch.view_as_real(2.0 * F).contiguous() for F in specs]

    adj.run(80, loss)
    for d, sc in enumerate(scs):
        _, pg_ref, _ = _oracle_pole_grad(sc)
        pg = adj.pole_grads[d]
        assert np.max(np.abs(pg - pg_ref)) <= 1e-10 * np.max(np.abs(pg_ref)), (d, pg, pg_ref)


def test_pole_grads_rejected_where_undefined():
    # pole box reaching into the CPML slabs, a domain without poles, reading without collecting
    sc = W.random_state_scene(shape=(12, 10, 14), d=2, n_poles=2, aniso=False)
    ctx = fdtd.Context([sc], dtype="f32")
    with pytest.raises(fdtd.FdtdError) as e:
        fdtd.fdtd_set_pole_grad(ctx.ctx, 0, 1)
    assert e.value.status == fdtd.FDTD_EINVAL
    sc2 = _design_scene(False)
    ctx2 = fdtd.Context([sc2], dtype="f32")
    with pytest.raises(fdtd.FdtdError):
        fdtd.fdtd_set_pole_grad(ctx2.ctx, 0, 1)
    sc3 = _design_scene(True)
    ctx3 = fdtd.Context([sc3], dtype="f32")
    with pytest.raises(fdtd.FdtdError):
        fdtd.fdtd_pole_grad(ctx3.ctx, 0, 2)
