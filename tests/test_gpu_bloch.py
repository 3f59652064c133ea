"""Bloch-periodic faces on the GPU (Sec. 2.2; transposed with conjugate seam factors, Sec. 3.1),
through the C ABI, against the FP64 Bloch oracle (oracle/bloch.py) on the same seeded states:
  * the complex fields after 200 steps at nonzero x and y phases (FP64 <= 1e-12 relative L2);
  * the transposed steps are the adjoint of the steps under <u, v> = sum conj(u) v (FP64 dot
    product <= 1e-10);
  * at zero phase the real parts step bit for bit like the real periodic path and the imaginary
    parts stay zero;
  * the calls that a Bloch domain does not support are refused.
"""
import math

import numpy as np
import pytest
import torch

from oracle.bloch import BlochOracle
from paper_2609_30039_gb300 import build as B
from paper_2609_30039_gb300 import fdtd
from paper_2609_30039_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPE = (12, 10, 9)
KX, KY = 0.37, -0.23   # wavenumbers per cell: phases k N per period


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    fdtd.load()


def _cell(seed=7, shape=SHAPE):
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    ie = [1.0 / rng.uniform(1.0, 4.0, size=(nz, ny, nx)) for _ in range(3)]
    sc = W.Scene(shape=shape, n_steps=0, cpml=(0,) * 6, inv_eps=ie, periodic=(1, 1, 0), name="bloch_cell")
    return sc, ie, rng


def _ctx(sc, dtype, phase=(KX * SHAPE[0], KY * SHAPE[1])):
    ctx = fdtd.Context([sc], dtype=dtype)
    fdtd.fdtd_set_bloch(ctx.ctx, 0, phase)
    return ctx


def _pec(shape):
    nx, ny, nz = shape
    m = [np.zeros((nz, ny, nx), dtype=bool) for _ in range(3)]
    m[0][0] = True   # tangential E on z = 0
    m[1][0] = True
    return m


def _random_state(rng, shape):
    n = int(np.prod(shape))
    x = rng.standard_normal(6 * n) + 1j * rng.standard_normal(6 * n)
    pec = _pec(shape)
    for a in range(3):
        x[a * n:(a + 1) * n][pec[a].ravel()] = 0.0
    return x


def _set_state(ctx, x, which=0):
    n = x.size // 6
    imag0 = ctx.part_count(0) - 6
    for c in range(6):
        v = x[c * n:(c + 1) * n]
        ctx.set_part(0, c, torch.from_numpy(np.ascontiguousarray(v.real)), which=which)
        ctx.set_part(0, imag0 + c, torch.from_numpy(np.ascontiguousarray(v.imag)), which=which)


def _get_state(ctx, which=0):
    imag0 = ctx.part_count(0) - 6
    re = [ctx.part(0, c, which).cpu().numpy().astype(np.float64) for c in range(6)]
    im = [ctx.part(0, imag0 + c, which).cpu().numpy().astype(np.float64) for c in range(6)]
    return np.concatenate([r + 1j * m for r, m in zip(re, im)])


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-4)])
def test_bloch_fields_after_200_steps_match_the_oracle(dtype, tol):
    sc, ie, rng = _cell()
    x = _random_state(rng, SHAPE)
    bo = BlochOracle(SHAPE, W.COURANT, kx=KX, ky=KY, inv_eps=ie)
    bo.set_state(x)
    bo.step(200)
    ctx = _ctx(sc, dtype)
    assert ctx.part_count(0) == 24
    _set_state(ctx, x)
    ctx.step(200)
    err = _rel(_get_state(ctx), bo.state())
    print(f"\n{dtype} Bloch fields after 200 steps vs oracle: {err:.3e}")
    assert err <= tol, err
    ctx.close()


def test_bloch_transposed_steps_are_the_adjoint_with_conjugate_seams():
    sc, ie, rng = _cell(seed=11)
    n_steps = 4
    x = _random_state(rng, SHAPE)
    y = _random_state(rng, SHAPE)
    ctx = _ctx(sc, "f64")
    _set_state(ctx, x)
    ctx.step(n_steps)
    Ax = _get_state(ctx)
    _set_state(ctx, y, which=1)
    fdtd.fdtd_set_adjoint_step_count(ctx.ctx, n_steps)
    fdtd.fdtd_step_adjoint(ctx.ctx, n_steps)
    Aty = _get_state(ctx, which=1)
    lhs, rhs = np.vdot(y, Ax), np.vdot(Aty, x)
    err = abs(lhs - rhs) / (np.linalg.norm(Ax) * np.linalg.norm(y))
    print(f"\nBloch dot-product identity: |<y,Ax> - <A^H y,x>| / (|Ax||y|) = {err:.3e}")
    assert err <= 1e-10, err
    # the oracle's transposed step gives the same adjoint state
    bo = BlochOracle(SHAPE, W.COURANT, kx=KX, ky=KY, inv_eps=ie)
    bo.set_state(y)
    bo.adjoint_step(n_steps)
    assert _rel(Aty, bo.state()) <= 1e-12
    ctx.close()


def test_bloch_at_zero_phase_steps_like_the_real_periodic_path():
    sc, ie, rng = _cell(seed=3)
    n = int(np.prod(SHAPE))
    x = _random_state(rng, SHAPE).real.copy()
    ctx_b = _ctx(sc, "f64", phase=(0.0, 0.0))
    ctx_r = fdtd.Context([sc], dtype="f64")
    for c in range(6):
        t = torch.from_numpy(np.ascontiguousarray(x[c * n:(c + 1) * n]))
        ctx_b.set_part(0, c, t)
        ctx_r.set_part(0, c, t)
    ctx_b.step(50)
    ctx_r.step(50)
    for c in range(6):
        assert torch.equal(ctx_b.part(0, c), ctx_r.part(0, c)), c
        assert float(ctx_b.part(0, 18 + c).abs().max()) == 0.0
    ctx_b.close()
    ctx_r.close()


def test_bloch_refuses_what_it_does_not_support():
    sc, ie, _ = _cell()
    ctx = fdtd.Context([sc], dtype="f64")
    with pytest.raises(fdtd.FdtdError) as e:   # a phase on a non-periodic axis
        fdtd.fdtd_set_periodic(ctx.ctx, 0, (1, 0, 0))
        fdtd.fdtd_set_bloch(ctx.ctx, 0, (0.1, 0.2))
    assert e.value.status == fdtd.FDTD_EINVAL
    fdtd.fdtd_set_periodic(ctx.ctx, 0, (1, 1, 0))
    fdtd.fdtd_set_bloch(ctx.ctx, 0, (0.1, 0.2))
    for call in (lambda: fdtd.fdtd_set_launch_mode(ctx.ctx, 0),
                 lambda: fdtd.fdtd_add_dft_monitor(ctx.ctx, 0, (0, 0, 3), (12, 10, 4), 1, np.array([0.2])),
                 lambda: fdtd.fdtd_step_backward(ctx.ctx, 1)):
        with pytest.raises(fdtd.FdtdError) as e:
            call()
        assert e.value.status == fdtd.FDTD_EINVAL
    ctx.close()
    cp = W.Scene(shape=(12, 10, 16), n_steps=0, cpml=(0, 0, 0, 0, 4, 4), periodic=(1, 1, 0))
    ctx = fdtd.Context([cp], dtype="f64")
    with pytest.raises(fdtd.FdtdError) as e:   # CPML slabs
        fdtd.fdtd_set_bloch(ctx.ctx, 0, (0.1, 0.2))
    assert e.value.status == fdtd.FDTD_EINVAL
    ctx.close()
