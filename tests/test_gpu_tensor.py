"""Symmetric node tensors (Sec. 2.3) on the GPU through the C ABI, against the FP64 oracle on the
same seeded inputs:
  * forward fields, CPML memories and spectra (FP64 <= 1e-12, FP32 <= 1e-4 relative L2), on grids
    whose extents leave ragged tiles, with and without a periodic axis, and in a batch beside a
    diagonal domain;
  * transposed steps: the adjoint state against the oracle's (FP64 <= 1e-12) and the dot-product
    identity (<= 1e-10);
  * the node-tensor cotangent of a design box against the oracle's replayed gradient (FP64 <= 1e-10,
    FP32 <= 1e-4);
  * the admission rule decides as the oracle's statement of it does; the calls a tensor domain does
    not support are refused.
"""
import numpy as np
import pytest
import torch

from oracle.oracle import gradient_replay, tensor_rejected
from paper_2609_30039_gb300 import adjoint as ADJ
from paper_2609_30039_gb300 import build as B
from paper_2609_30039_gb300 import fdtd
from paper_2609_30039_gb300 import workloads as W
from tests.oracle_adapter import oracle_from_scene
from tests.test_gpu_parity import _oracle_vec_from_parts, _random_parts, _set_parts, compare_state, gpu_parts, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    fdtd.load()


def _admitted(rng, shape, lo=1.0, hi=4.0):
    nx, ny, nz = shape
    n = nx * ny * nz
    Q, _ = np.linalg.qr(rng.standard_normal((n, 3, 3)))
    lam = rng.uniform(lo, hi, (n, 3))
    eps = np.einsum("nij,nj,nkj->nik", Q, lam, Q)
    return W.inv_tensor6(eps).reshape(6, nz, ny, nx)


def tensor_scene(shape=(37, 21, 19), steps=60, periodic=(0, 0, 0), design=None, seed=21):
    """Rotated random tensors inside; in the CPML slabs (x faces unless x is periodic, z faces) the
    diagonal eps = (1.2, 2, 4), whose x and z eigenvalues are the extreme ones; PEC y faces."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    cx = 0 if periodic[0] else 3
    sc = W.Scene(shape=shape, n_steps=steps, cpml=(cx, cx, 0, 0, 4, 4), kappa_max=3.0, alpha_max=0.05,
                 periodic=periodic)
    t = _admitted(rng, shape)
    slab = np.zeros((nz, ny, nx), dtype=bool)
    slab[:4], slab[nz - 4:] = True, True
    if cx:
        slab[:, :, :cx], slab[:, :, nx - cx:] = True, True
    d = W.inv_tensor6(W.principal_eps((1.2, 2.0, 4.0)))
    for q in range(6):
        t[q][slab] = d[q]
    sc.tensor = t
    wave = W.gaussian_pulse(steps, 7.0, periods=1, delay=3)
    sc.sources = [W.Source(W.EX, (nx // 6, ny // 4, nz // 2 - 1), (nx // 3, ny // 2, nz // 2), wave),
                  W.Source(W.EZ, (nx // 2, ny // 2, nz // 2 + 1), (nx // 2 + 1, ny // 2 + 1, nz // 2 + 2), -wave)]
    sc.monitors = [W.Monitor((3, 1, nz - 6), (nx - 3, ny, nz - 5), (0, 1, 2, 3, 4, 5), W.omegas_for((6.0, 8.0)))]
    sc.design = design
    assert not tensor_rejected(t, shape, sc.cpml).any()
    return sc


@pytest.mark.parametrize("dtype,periodic,tol", [
    ("f64", (0, 0, 0), 1e-12), ("f64", (1, 0, 0), 1e-12), ("f32", (0, 0, 0), 1e-4)])
def test_tensor_fields_and_spectra_match_the_oracle(dtype, periodic, tol):
    sc = tensor_scene(periodic=periodic)
    ctx = fdtd.Context([sc], dtype=dtype)
    assert fdtd.fdtd_get_launch_mode(ctx.ctx) == 4
    ctx.step(sc.n_steps)
    o = oracle_from_scene(sc)
    o.step(sc.n_steps)
    errs = compare_state(ctx, o, sc, tol=tol)
    e = rel(ctx.dft(0).cpu().numpy(), o.dft(0))
    print(f"\n{dtype} periodic={periodic}: state {max(errs.values()):.2e}, spectra {e:.2e}")
    assert e <= tol, e
    ctx.close()


def test_tensor_domain_in_a_batch_beside_a_diagonal_domain_fp64():
    a = tensor_scene(shape=(20, 13, 17), steps=40)
    b = W.random_state_scene(shape=(11, 9, 14), d=2, n_poles=0, aniso=False)
    b.n_steps = 40
    b.sources = [W.Source(W.EY, (4, 3, 6), (6, 5, 7), W.gaussian_pulse(40, 6.0, periods=1, delay=3))]
    ctx = fdtd.Context([a, b], dtype="f64")
    ctx.step(40)
    for d, sc in enumerate((a, b)):
        o = oracle_from_scene(sc)
        o.step(40)
        compare_state(ctx, o, sc, d=d, tol=1e-12)
    ctx.close()


def test_isotropic_node_tensor_is_the_diagonal_update_with_edge_means_fp64():
    sc = tensor_scene(shape=(19, 11, 16), steps=50)
    nx, ny, nz = sc.shape
    s = 1.0 / np.random.default_rng(3).uniform(1.0, 5.0, (nz, ny, nx))
    # vacuum within one node of the CPML slabs: there the edge means stay isotropic, which the
    # diagonal domain's own admission rule needs
    keep = np.zeros_like(s, dtype=bool)
    keep[5:nz - 5, :, 4:nx - 4] = True
    s[~keep] = 1.0
    sc.tensor = np.stack([s, s, s, 0 * s, 0 * s, 0 * s])
    edge = []
    for a in range(3):
        ax = 2 - a
        m = 0.5 * (s + np.roll(s, -1, axis=ax))
        sl = [slice(None)] * 3
        sl[ax] = -1
        m[tuple(sl)] = s[tuple(sl)]
        edge.append(m)
    ref = W.Scene(**{**sc.__dict__, "tensor": None, "inv_eps": edge})
    c1 = fdtd.Context([sc], dtype="f64")
    c2 = fdtd.Context([ref], dtype="f64")
    c1.step(50)
    c2.step(50)
    for c in range(6):
        x, y = c1.part(0, c).cpu().numpy(), c2.part(0, c).cpu().numpy()
        assert rel(x, y) <= 1e-13, c
    c1.close()
    c2.close()


def test_tensor_transposed_steps_match_the_oracle_fp64():
    sc = tensor_scene(shape=(21, 13, 17), steps=0)
    sc.sources, sc.monitors = [], []
    ctx = fdtd.Context([sc], dtype="f64")
    o = oracle_from_scene(sc, with_sources=False, with_monitors=False)
    rng = np.random.default_rng(11)
    x = _random_parts(ctx, sc, rng)
    y = _random_parts(ctx, sc, rng)
    n = 6
    _set_parts(ctx, x, 0)
    ctx.step(n)
    fx = gpu_parts(ctx, 0, 0)
    fdtd.fdtd_adjoint_begin(ctx.ctx)
    _set_parts(ctx, y, 1)
    fdtd.fdtd_step_adjoint(ctx.ctx, n)
    fty = gpu_parts(ctx, 0, 1)
    lhs = sum(float(a @ b) for a, b in zip(fx, y))
    rhs = sum(float(a @ b) for a, b in zip(x, fty))
    scale = np.sqrt(sum(float(a @ a) for a in fx) * sum(float(b @ b) for b in y))
    print(f"\ntensor dot-product identity: {abs(lhs - rhs) / scale:.2e}")
    assert abs(lhs - rhs) <= 1e-10 * scale, (lhs, rhs)
    o.adj_reset()
    o.set_state(_oracle_vec_from_parts(o, sc, ctx, y), adjoint=True)
    for m in reversed(range(n)):
        o.adjoint_step(m)
    compare_state(ctx, o, sc, which=1)
    ref = o.get_state(adjoint=True)
    got = _oracle_vec_from_parts(o, sc, ctx, fty)
    keep = np.zeros_like(ref, dtype=bool)
    keep[:6 * o.n] = True   # psi cotangents outside the slabs are no GPU state
    assert rel(got[keep], ref[keep]) < 1e-12
    ctx.close()


def _oracle_objective(o):
    F = o.dft(0)
    return float((np.abs(F) ** 2).sum()), {0: 2.0 * F}


def _gpu_loss(specs):
    F = specs[0]
    return float((F.abs() ** 2).sum()), [torch.view_as_real(2.0 * F).contiguous()]


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_node_tensor_gradient_matches_the_oracle(dtype, tol):
    box = ((8, 3, 6), (17, 9, 11))   # nodes outside the CPML slabs, across tile edges
    sc = tensor_scene(shape=(29, 13, 17), steps=50, design=box)
    o = oracle_from_scene(sc)
    J_ref = gradient_replay(o, sc.n_steps, _oracle_objective)
    g_ref = np.stack([o.grad(q) for q in range(6)])
    ctx = fdtd.Context([sc], dtype=dtype)
    (J, _), grads, _ = ADJ.DesignAdjoint(ctx, slots=5).run(sc.n_steps, _gpu_loss)
    g = grads[0].cpu().numpy().reshape(g_ref.shape)
    err = rel(g, g_ref)
    print(f"\n{dtype} node-tensor gradient vs oracle: {err:.2e} (J {abs(J - J_ref) / abs(J_ref):.1e})")
    assert abs(J - J_ref) <= (1e-12 if dtype == "f64" else 1e-5) * abs(J_ref)
    assert err <= tol, err
    # off-diagonal components carry a real share of the gradient
    assert np.linalg.norm(g_ref[3:]) > 0.05 * np.linalg.norm(g_ref[:3])
    ctx.close()


def test_admission_decisions_follow_the_rule():
    base = tensor_scene(shape=(12, 9, 16), steps=0)
    nx, ny, nz = base.shape
    rot = W.inv_tensor6(W.principal_eps((1.5, 3.0, 5.0), W.rotation(0, 0.4)))
    cases = {
        "admitted": None,
        "rotated_in_z_face": ((1, 4, 5), rot),                                # z not a principal axis
        "intermediate_in_x_face": ((4, 1, 5), W.inv_tensor6(W.principal_eps((2.0, 1.2, 4.0)))),
        "rotated_inside": ((7, 4, 8), rot),                                   # allowed inside
        "eps_below_one": ((7, 4, 8), W.inv_tensor6(W.principal_eps((0.7, 2.0, 2.0)))),
        "not_positive": ((7, 4, 8), -W.inv_tensor6(np.eye(3))),
    }
    for name, change in cases.items():
        t = base.tensor.copy()
        if change is not None:
            (k, j, i), v = change
            t[:, k, j, i] = v
        want = bool(tensor_rejected(t, base.shape, base.cpml).any())
        sc = W.Scene(**{**base.__dict__, "tensor": None})
        ctx = fdtd.Context([sc], dtype="f32")
        comps = [torch.from_numpy(np.ascontiguousarray(t[q], dtype=np.float32)).cuda() for q in range(6)]
        try:
            fdtd.fdtd_set_tensor(ctx.ctx, 0, comps)
            got = False
        except fdtd.FdtdError as e:
            assert e.status == fdtd.FDTD_ETENSOR, (name, e)
            got = True
        assert got == want, name
        if got:
            ctx.step(3)   # the domain is left on its diagonal eps^-1 and still steps
        ctx.close()


def test_tensor_domain_refuses_what_it_does_not_support():
    sc = tensor_scene(shape=(12, 9, 16), steps=4)
    ctx = fdtd.Context([sc], dtype="f32")
    for call in (lambda: fdtd.fdtd_set_launch_mode(ctx.ctx, 0),
                 lambda: fdtd.fdtd_autotune(ctx.ctx, 8),
                 lambda: fdtd.fdtd_step_backward(ctx.ctx, 1),
                 lambda: fdtd.fdtd_enable_energy(ctx.ctx, 8),
                 lambda: fdtd.fdtd_time_half_steps(ctx.ctx, 0, 2)):
        with pytest.raises(fdtd.FdtdError) as e:
            call()
        assert e.value.status == fdtd.FDTD_EINVAL
    # back to the diagonal eps^-1: the other modes are open again
    fdtd.fdtd_set_tensor(ctx.ctx, 0, None)
    fdtd.fdtd_set_launch_mode(ctx.ctx, 0)
    ctx.close()
    poles = W.random_state_scene(shape=(10, 9, 8), d=2, n_poles=1, aniso=False)
    ctx = fdtd.Context([poles], dtype="f32")
    comps = [torch.from_numpy(np.ascontiguousarray(tensor_scene(shape=(10, 9, 8), steps=0).tensor[q],
                                                   dtype=np.float32)).cuda() for q in range(6)]
    with pytest.raises(fdtd.FdtdError) as e:
        fdtd.fdtd_set_tensor(ctx.ctx, 0, comps)
    assert e.value.status == fdtd.FDTD_EINVAL
    ctx.close()
