"""Host-streamed slabs (Sec. 4.2) on the GPU through the C ABI.  A streamed context keeps the state
in pinned host memory and steps z-slabs with halos in device workspaces; its owned planes must
hold exactly what the resident context computes (fields, CPML memories, pole states, spectra),
which the FP64 oracle also pins directly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.flux import plane_flux_z
from paper_2609_30039_gb300 import fdtd
from paper_2609_30039_gb300 import workloads as W
from tests.oracle_adapter import oracle_from_scene
from tests.test_gpu_parity import _random_parts, _set_parts, compare_state, rel

pytestmark = pytest.mark.gpu


def _rich_scene(shape=(21, 17, 40), steps=37):
    """CPML on every face, a diagonal tensor, a Lorentz and a Drude pole in a box that crosses
    several slabs, sources in a CPML-adjacent, a middle and a top plane, and monitors that span
    slab edges."""
    sc = W.random_state_scene(shape=shape, d=4, n_poles=2, aniso=True)
    sc.poles = ((W.LORENTZ, 1.3, 0.2, 0.03), (W.DRUDE, 0.0, 0.3, 0.05))
    sc.n_steps = steps
    nx, ny, nz = shape
    wave = W.gaussian_pulse(steps, 8.0, periods=1, delay=3)
    sc.sources = [W.Source(W.EY, (10, 8, 5), (12, 9, 6), wave),
                  W.Source(W.HZ, (6, 6, nz // 2), (7, 11, nz // 2 + 1), 0.5 * wave),
                  W.Source(W.EX, (9, 9, nz - 6), (10, 10, nz - 5), -wave)]
    sc.monitors = [W.Monitor((2, 3, 5), (19, 14, nz - 7), (0, 1, 2, 3, 4, 5), W.omegas_for((7.0, 9.0, 11.0))),
                   W.Monitor((8, 8, nz - 9), (9, 9, nz - 8), (W.EZ,), W.omegas_for((10.0,)))]
    return sc


def _parts(ctx):
    return [ctx.part(0, p).clone() for p in range(ctx.part_count(0))]


def _assert_same(a, b):
    assert len(a) == len(b)
    for p, (x, y) in enumerate(zip(a, b)):
        assert torch.equal(x, y), f"part {p} differs"


@pytest.mark.parametrize("slab,halo,steps,dtype", [
    (8, 3, 37, "f32"),    # five slabs, batches of 3 with a ragged last batch
    (8, 8, 20, "f32"),    # halo = slab
    (5, 1, 9, "f32"),     # one step per batch, eight slabs
    (13, 4, 30, "f32"),   # last slab of one plane
    (64, 16, 25, "f32"),  # one slab holds the domain
    (8, 3, 37, "f64"),
])
def test_streamed_equals_resident_bitwise(slab, halo, steps, dtype):
    sc = _rich_scene(steps=steps)
    res = fdtd.Context([sc], dtype=dtype)
    st = fdtd.Context([sc], dtype=dtype, streamed=(slab, halo))
    # start both from the same nonzero state: CPML memories and pole states evolve too
    x = _random_parts(res, sc, np.random.default_rng(5))
    _set_parts(res, x, 0)
    _set_parts(st, x, 0)
    res.step(steps // 2)
    res.step(steps - steps // 2)
    st.step(steps // 2)
    st.step(steps - steps // 2)
    assert fdtd.fdtd_step_count(st.ctx) == steps
    _assert_same(_parts(res), _parts(st))
    for k in range(len(sc.monitors)):
        assert torch.equal(res.dft(k), st.dft(k))


def test_streamed_fp64_matches_oracle():
    sc = _rich_scene(steps=60)
    ctx = fdtd.Context([sc], dtype="f64", streamed=(7, 4))
    ctx.step(sc.n_steps)
    o = oracle_from_scene(sc)
    o.step(sc.n_steps)
    compare_state(ctx, o, sc, tol=1e-12)
    for k in range(len(sc.monitors)):
        assert rel(ctx.dft(k).cpu().numpy(), o.dft(k)) < 1e-12


def test_streamed_periodic_cell_flux_equals_resident():
    sc = W.slab_cell(n_steps=600)
    nf = len(sc.monitors[0].omegas)
    res = fdtd.Context([sc], dtype="f32")
    st = fdtd.Context([sc], dtype="f32", streamed=(40, 12))
    res.step(sc.n_steps)
    st.step(sc.n_steps)
    _assert_same(_parts(res), _parts(st))
    for k in range(2):
        a = fdtd.fdtd_dft_flux(res.ctx, res.monitors[k][0], nf)
        b = fdtd.fdtd_dft_flux(st.ctx, st.monitors[k][0], nf)
        assert np.array_equal(a, b)
        assert np.allclose(b, plane_flux_z(st.dft(k).cpu().numpy(), (0, 1, 3, 4)), rtol=1e-12, atol=0)


def test_streamed_reset_and_dft_reset_repeat_the_run():
    sc = _rich_scene(steps=24)
    ctx = fdtd.Context([sc], dtype="f32", streamed=(8, 4))
    ctx.step(24)
    first = _parts(ctx) + [ctx.dft(0).clone()]
    fdtd.fdtd_reset(ctx.ctx)
    fdtd.fdtd_dft_reset(ctx.ctx)
    assert all(int(torch.count_nonzero(p)) == 0 for p in _parts(ctx))
    ctx.step(24)
    _assert_same(first, _parts(ctx) + [ctx.dft(0).clone()])


def test_streamed_context_rejects_what_it_does_not_hold():
    sc = _rich_scene(steps=8)
    ctx = fdtd.Context([sc], dtype="f32", streamed=(8, 4))
    for call in (lambda: fdtd.fdtd_state_save(ctx.ctx, 0, 0),
                 lambda: fdtd.fdtd_set_launch_mode(ctx.ctx, 0),
                 lambda: fdtd.fdtd_step_backward(ctx.ctx, 1)):
        with pytest.raises(fdtd.FdtdError) as e:
            call()
        assert e.value.status == fdtd.FDTD_EINVAL
    # the adjoint state exists after fdtd_adjoint_begin, and a transposed sweep needs the forward
    # checkpoints of its batches
    for call in (lambda: ctx.part(0, 0, which=1), lambda: fdtd.fdtd_step_adjoint(ctx.ctx, 0)):
        with pytest.raises(fdtd.FdtdError) as e:
            call()
        assert e.value.status == fdtd.FDTD_ESTATE
    ctx.step(4)
    fdtd.fdtd_adjoint_begin(ctx.ctx)
    with pytest.raises(fdtd.FdtdError) as e:
        fdtd.fdtd_step_adjoint(ctx.ctx, 2)
    assert e.value.status == fdtd.FDTD_ESTATE
    fdtd.fdtd_set_launch_mode(ctx.ctx, 4)
    # materials on the device, a halo wider than the slab, no halo
    with pytest.raises(fdtd.FdtdError):
        fdtd.Context([sc], dtype="f32", streamed=(4, 5))
    with pytest.raises(fdtd.FdtdError):
        fdtd.Context([sc], dtype="f32", streamed=(4, 0))
    dev = fdtd.Context([sc], dtype="f32")
    with pytest.raises(fdtd.FdtdError) as e:
        fdtd.fdtd_create_streamed(fdtd.fdtd_grid(*sc.shape, 1.0, sc.courant, 0.0, fdtd.FDTD_F32), fdtd.fdtd_cpml(),
                                  dev._material_struct(sc, dev.inv_eps[0]), 8, 4)
    assert e.value.status == fdtd.FDTD_EINVAL


def test_streamed_device_footprint_is_the_windows():
    # 96 x 96 x 512 FP32 with CPML: the resident context holds fields, adjoint fields, CPML memories
    # of the whole domain; the streamed one three windows of 32 + 2 * 8 planes
    sc = W.cpml_blocks(n=96, d=8, n_steps=10, block=8, region=(20, 76), wavelengths=(10.0,))
    sc.shape = (96, 96, 512)
    sc.inv_eps = [np.ones((512, 96, 96))]
    sc.sources = [W.Source(W.EZ, (48, 48, 100), (49, 49, 101), W.gaussian_pulse(10, 10.0))]
    sc.monitors = []
    torch.cuda.synchronize()
    f0 = torch.cuda.mem_get_info()[0]
    st = fdtd.Context([sc], dtype="f32", streamed=(32, 8))
    torch.cuda.synchronize()
    used_st = f0 - torch.cuda.mem_get_info()[0]
    st.close()
    torch.cuda.synchronize()
    f1 = torch.cuda.mem_get_info()[0]
    res = fdtd.Context([sc], dtype="f32")
    torch.cuda.synchronize()
    used_res = f1 - torch.cuda.mem_get_info()[0]
    res.close()
    assert used_st < 0.3 * used_res, (used_st, used_res)


# ---- the streamed transposed sweep (Sec. 4.2: it runs the slab tiling in reverse) ----------------
def _adjoint_scene(steps):
    sc = _rich_scene(steps=steps)
    sc.design = ((6, 5, 8), (15, 12, 30))   # outside the CPML slabs, across several slab edges
    return sc


def _loss(specs):
    F = specs[0]
    return float((F.abs() ** 2).sum()), [torch.view_as_real(2.0 * F).contiguous()] + [None] * (len(specs) - 1)


@pytest.mark.parametrize("slab,halo,steps,dtype", [
    (8, 3, 37, "f32"),    # five slabs, batches of 3 with a ragged last batch
    (9, 6, 20, "f64"),
    (64, 16, 25, "f32"),  # one slab holds the domain
])
def test_streamed_transposed_sweep_equals_the_resident_one(slab, halo, steps, dtype):
    from paper_2609_30039_gb300 import adjoint as ADJ
    sc = _adjoint_scene(steps)
    res = fdtd.Context([sc], dtype=dtype)
    (J_r, _), g_r, _ = ADJ.DesignAdjoint(res, slots=6).run(sc.n_steps, _loss)
    adj_r = [res.part(0, p, which=1).clone() for p in range(res.part_count(0))]
    st = fdtd.Context([sc], dtype=dtype, streamed=(slab, halo))
    (J_s, _), g_s, _ = ADJ.StreamedAdjoint(st).run(sc.n_steps, _loss)
    adj_s = [st.part(0, p, which=1).clone() for p in range(st.part_count(0))]
    assert J_s == J_r
    assert float(g_r[0].abs().max()) > 0.0
    # the owned planes of every window hold what the resident sweep computes, bit for bit: the
    # adjoint state at step 0 and the material cotangent (each cell sums its steps in the same order)
    for p, (x, y) in enumerate(zip(adj_s, adj_r)):
        assert torch.equal(x.cpu(), y.cpu()), f"adjoint part {p} differs: {float((x.cpu() - y.cpu()).abs().max())}"
    assert torch.equal(g_s[0], g_r[0]), float((g_s[0] - g_r[0]).abs().max())
    res.close()
    st.close()


def test_streamed_gradient_matches_the_oracle_fp64():
    from oracle.oracle import gradient_replay
    from paper_2609_30039_gb300 import adjoint as ADJ
    sc = _adjoint_scene(24)
    o = oracle_from_scene(sc)

    def obj(orc):
        F = orc.dft(0)
        return float((np.abs(F) ** 2).sum()), {0: 2.0 * F}

    J_ref = gradient_replay(o, sc.n_steps, obj)
    g_ref = np.stack([o.grad(a) for a in range(3)])
    st = fdtd.Context([sc], dtype="f64", streamed=(8, 3))
    (J, _), g, _ = ADJ.StreamedAdjoint(st).run(sc.n_steps, _loss)
    assert abs(J - J_ref) <= 1e-12 * abs(J_ref)
    err = rel(g[0].cpu().numpy().reshape(g_ref.shape), g_ref)
    print(f"\nstreamed FP64 gradient vs oracle: {err:.3e}")
    assert err < 1e-10, err
    st.close()


def test_streamed_gradient_repeats_with_the_kept_checkpoint_buffers():
    from paper_2609_30039_gb300 import adjoint as ADJ
    sc = _adjoint_scene(20)
    st = fdtd.Context([sc], dtype="f32", streamed=(8, 3))
    runner = ADJ.StreamedAdjoint(st)
    (J1, _), g, _ = runner.run(sc.n_steps, _loss)
    g1 = g[0].clone()
    # a second run from step 0 reuses the pinned buffers of the first and gives the same result
    fdtd.fdtd_reset(st.ctx)
    fdtd.fdtd_dft_reset(st.ctx)
    (J2, _), g, _ = runner.run(sc.n_steps, _loss)
    assert J2 == J1
    assert torch.equal(g[0], g1)
    with pytest.raises(fdtd.FdtdError) as e:
        fdtd.fdtd_stream_checkpoints(st.ctx, 3)
    assert e.value.status == fdtd.FDTD_EINVAL
    runner.release()
    st.close()
