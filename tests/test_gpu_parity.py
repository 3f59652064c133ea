"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances: FP64 GPU vs oracle <= 1e-12 relative L2 on fields (rounding order and FMA
contraction differ, nothing else); FP32 <= 1e-4 relative L2 on DFT spectra; adjoint FP64
dot-product identity <= 1e-10; FP64 gradient vs the oracle's discrete adjoint <= 1e-10.
"""
import numpy as np
import pytest
import torch

from oracle.oracle import gradient_replay
from paper_2609_30039_gb300 import adjoint as ADJ
from paper_2609_30039_gb300 import build as B
from paper_2609_30039_gb300 import fdtd
from paper_2609_30039_gb300 import workloads as W
from tests.oracle_adapter import oracle_from_scene, pec_mask_E

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    fdtd.load()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def slab_index(N, lo, hi):
    return np.r_[0:lo, N - hi:N]


def psi_from_oracle(o, sc, magnetic, a, s):
    """Oracle full-grid psi restricted to the cells the GPU stores (slabs of the derivative axis)."""
    ax = (a + 1 + s) % 3
    lo, hi = sc.cpml[2 * ax], sc.cpml[2 * ax + 1]
    full = o.psi(magnetic, a, s)
    return np.take(full, slab_index(sc.shape[ax], lo, hi), axis=2 - ax)


def gpu_parts(ctx, d=0, which=0):
    return [ctx.part(d, p, which).cpu().numpy() for p in range(ctx.part_count(d))]


def _group_errors(pairs):
    """Error of each array normalised by the norm of its whole group (a component that is zero by
    symmetry holds only rounding noise on both sides; its own relative error is meaningless)."""
    tot = np.sqrt(sum(float(np.sum(np.asarray(r) ** 2)) for _, _, r in pairs)) or 1.0
    return {k: float(np.linalg.norm(np.asarray(g) - np.asarray(r)) / tot) for k, g, r in pairs}


def compare_state(ctx, o, sc, d=0, tol=1e-12, which=0):
    """Fields, CPML memories and pole states of domain d against the oracle (relative L2 over
    each group: the six fields, the CPML memories, the pole states)."""
    parts = gpu_parts(ctx, d, which)
    nx, ny, nz = sc.shape
    get_f = (o.adj_field if which else o.field)
    errs = _group_errors([(f"F{c}", parts[c].reshape(nz, ny, nx), get_f(c)) for c in range(6)])
    if not which:
        ps = []
        for mag in (0, 1):
            for a in range(3):
                for s in range(2):
                    p = 6 + 6 * mag + 2 * a + s
                    if parts[p].size:
                        ref = psi_from_oracle(o, sc, mag, a, s)
                        ps.append((f"psi{mag}{a}{s}", parts[p].reshape(ref.shape), ref))
        if ps:
            errs.update(_group_errors(ps))
        if o.npole:
            lo, hi = fdtd.fdtd_ade_box(ctx.ctx, d)
            xs = []
            for a in range(3):
                for p in range(o.npole):
                    for w in range(2):
                        g = parts[18 + 2 * (a * o.npole + p) + w].reshape(hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0])
                        ref = o.pole_state(a, p, w)[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
                        xs.append((f"x{a}{p}{w}", g, ref))
            errs.update(_group_errors(xs))
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, bad
    return errs


def small_blocks(n=40, d=6, steps=300, lam=10.0):
    sc = W.cpml_blocks(n=n, d=d, n_steps=steps, block=4, region=(n // 4, n - n // 4),
                       wavelengths=(0.9 * lam, lam, 1.1 * lam))
    sc.sources[0].wave = W.gaussian_pulse(steps, wavelength=lam, periods=1.0, delay=3.0)
    return sc


# ----------------------------------------------------------------------------- forward
def test_pec_vacuum_fp64_fields_and_energy():
    sc = W.pec_vacuum(32, 200)
    ctx = fdtd.Context([sc], dtype="f64")
    ctx.step(sc.n_steps)
    o = oracle_from_scene(sc)
    o.step(sc.n_steps)
    compare_state(ctx, o, sc)
    e_gpu = ctx.energy(0, sc.n_steps)
    assert rel(e_gpu, o.energy()) < 1e-12


def test_cpml_blocks_fp64_state_and_dft():
    sc = small_blocks(40, 6, 300)
    ctx = fdtd.Context([sc], dtype="f64")
    ctx.step(sc.n_steps)
    o = oracle_from_scene(sc)
    o.step(sc.n_steps)
    compare_state(ctx, o, sc)
    assert rel(ctx.dft(0).cpu().numpy(), o.dft(0)) < 1e-12


def test_cpml_blocks_fp32_dft_within_1e4():
    sc = small_blocks(48, 8, 1500, lam=12.0)
    ctx = fdtd.Context([sc], dtype="f32")
    ctx.step(sc.n_steps)
    o = oracle_from_scene(sc)
    o.step(sc.n_steps)
    err = rel(ctx.dft(0).cpu().numpy(), o.dft(0))
    assert err < 1e-4, err


@pytest.mark.parametrize("poles", [
    ((W.LORENTZ, 1.3, 0.2, 0.03), (W.LORENTZ, 0.6, 0.11, 0.01)),
    ((W.DRUDE, 0.0, 0.3, 0.05),),
])
def test_dispersive_anisotropic_fp64(poles):
    sc = W.random_state_scene(shape=(37, 29, 21), d=4, n_poles=len(poles), aniso=True)
    sc.poles = poles
    sc.n_steps = 150
    c = (12, 14, 10)
    sc.sources = [W.Source(W.EY, c, (c[0] + 1, c[1] + 1, c[2] + 1), W.gaussian_pulse(150, 10.0, periods=1, delay=3))]
    sc.monitors = [W.Monitor((5, 5, 9), (30, 24, 12), (0, 1, 2, 3, 4, 5), W.omegas_for((9.0, 11.0)))]
    ctx = fdtd.Context([sc], dtype="f64")
    ctx.step(sc.n_steps)
    o = oracle_from_scene(sc)
    o.step(sc.n_steps)
    compare_state(ctx, o, sc)
    assert rel(ctx.dft(0).cpu().numpy(), o.dft(0)) < 1e-12


def _tiny_batch(n=3, steps=200):
    scs = W.lorentz_batch(n_domains=n, sizes=(24, 32, 40), d=4, n_steps=steps)
    for sc in scs:
        sc.sources[0].wave = W.gaussian_pulse(steps, 10.0, periods=1, delay=3)
    return scs


def test_batch_uneven_domains_fp64_vs_oracle():
    scs = _tiny_batch(3, 200)
    ctx = fdtd.Context(scs, dtype="f64")
    ctx.step(200)
    for d, sc in enumerate(scs):
        o = oracle_from_scene(sc)
        o.step(200)
        compare_state(ctx, o, sc, d=d)
        assert rel(ctx.dft(d).cpu().numpy(), o.dft(0)) < 1e-12


def test_batch_bitwise_equal_to_single_runs_fp32():
    scs = _tiny_batch(4, 120)
    batch = fdtd.Context(scs, dtype="f32")
    batch.step(120)
    for d, sc in enumerate(scs):
        one = fdtd.Context([sc], dtype="f32")
        one.step(120)
        for p in range(one.part_count(0)):
            assert torch.equal(batch.part(d, p), one.part(0, p)), (d, p)
        assert torch.equal(batch.dft(d), one.dft(0))
        one.close()


# ----------------------------------------------------------------------------- adjoint
def _random_parts(ctx, sc, rng, d=0):
    pec = pec_mask_E(sc.shape)
    parts = []
    for p in range(ctx.part_count(d)):
        n = fdtd.fdtd_part_size(ctx.ctx, d, p)
        v = rng.standard_normal(n)
        if p < 3:
            v = v.reshape(sc.shape[::-1])
            v[pec[p]] = 0.0
            v = v.reshape(-1)
        parts.append(v)
    return parts


def _set_parts(ctx, parts, which, d=0):
    for p, v in enumerate(parts):
        if v.size:
            ctx.set_part(d, p, torch.from_numpy(v), which=which)


@pytest.mark.parametrize("nsteps", [1, 10])
def test_adjoint_dot_product_fp64(nsteps):
    sc = W.random_state_scene(shape=(13, 11, 9), d=2, n_poles=2, aniso=True)
    ctx = fdtd.Context([sc], dtype="f64")
    rng = np.random.default_rng(42 + nsteps)
    x = _random_parts(ctx, sc, rng)
    y = _random_parts(ctx, sc, rng)
    _set_parts(ctx, x, 0)
    ctx.step(nsteps)
    fx = gpu_parts(ctx, 0, 0)
    fdtd.fdtd_adjoint_begin(ctx.ctx)
    _set_parts(ctx, y, 1)
    fdtd.fdtd_step_adjoint(ctx.ctx, nsteps)
    fty = gpu_parts(ctx, 0, 1)
    lhs = sum(float(a @ b) for a, b in zip(fx, y))
    rhs = sum(float(a @ b) for a, b in zip(x, fty))
    scale = np.sqrt(sum(float(a @ a) for a in fx) * sum(float(b @ b) for b in y))
    assert abs(lhs - rhs) <= 1e-10 * scale, (lhs, rhs)


def _oracle_vec_from_parts(o, sc, ctx, parts):
    """Full-grid oracle state vector from GPU parts (slab/box parts placed, zero elsewhere)."""
    nx, ny, nz = sc.shape
    n = nx * ny * nz
    vec = np.zeros(o.state_len)
    for c in range(6):
        vec[c * n:(c + 1) * n] = parts[c]
    for mag in (0, 1):
        for a in range(3):
            for s in range(2):
                p = 6 + 6 * mag + 2 * a + s
                if not parts[p].size:
                    continue
                ax = (a + 1 + s) % 3
                full = np.zeros((nz, ny, nx))
                shp = list(full.shape)
                shp[2 - ax] = sc.cpml[2 * ax] + sc.cpml[2 * ax + 1]
                idx = slab_index(sc.shape[ax], sc.cpml[2 * ax], sc.cpml[2 * ax + 1])
                sl = [slice(None)] * 3
                sl[2 - ax] = idx
                full[tuple(sl)] = parts[p].reshape(shp)
                k = 6 + 6 * mag + 2 * a + s
                vec[k * n:(k + 1) * n] = full.reshape(-1)
    if o.npole:
        lo, hi = fdtd.fdtd_ade_box(ctx.ctx, 0)
        for a in range(3):
            for p in range(o.npole):
                for w in range(2):
                    full = np.zeros((nz, ny, nx))
                    full[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = parts[18 + 2 * (a * o.npole + p) + w].reshape(
                        hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0])
                    k = 18 + 2 * (a * o.npole + p) + w
                    vec[k * n:(k + 1) * n] = full.reshape(-1)
    return vec


def test_adjoint_state_matches_oracle_fp64():
    sc = W.random_state_scene(shape=(13, 11, 9), d=2, n_poles=2, aniso=True)
    ctx = fdtd.Context([sc], dtype="f64")
    o = oracle_from_scene(sc, with_sources=False, with_monitors=False)
    rng = np.random.default_rng(7)
    y = _random_parts(ctx, sc, rng)
    ctx.step(6)
    fdtd.fdtd_adjoint_begin(ctx.ctx)
    _set_parts(ctx, y, 1)
    fdtd.fdtd_step_adjoint(ctx.ctx, 6)
    o.adj_reset()
    o.set_state(_oracle_vec_from_parts(o, sc, ctx, y), adjoint=True)
    for m in reversed(range(6)):
        o.adjoint_step(m)
    compare_state(ctx, o, sc, which=1)
    ref = o.get_state(adjoint=True)
    got = _oracle_vec_from_parts(o, sc, ctx, gpu_parts(ctx, 0, 1))
    # psi cotangents outside the slabs and pole cotangents outside the box are not GPU state
    n = int(np.prod(sc.shape))
    keep = np.zeros_like(ref, dtype=bool)
    keep[:6 * n] = True
    keep[18 * n:] = True
    assert rel(got[keep], ref[keep]) < 1e-12


def _design_scene(dispersive, n=18, steps=70):
    sc = W.adjoint_design(n=n, d=3, n_steps=steps)
    sc.sources[0].wave = W.gaussian_pulse(steps, wavelength=8.0, periods=1.0, delay=3.0)
    sc.monitors[0].omegas = W.omegas_for((7.0, 8.0, 9.0))
    if dispersive:
        (lx, ly, lz), (hx, hy, hz) = sc.design
        mask = np.zeros(sc.shape[::-1], dtype=np.uint8)
        mask[lz:hz, ly:hy, lx:hx] = 1
        sc.pole_mask = mask
        sc.poles = ((W.LORENTZ, 1.2, 0.5, 0.05), (W.DRUDE, 0.0, 0.3, 0.1))
    return sc


def _oracle_objective(o):
    F = o.dft(0)
    return float((np.abs(F) ** 2).sum()), {0: 2.0 * F}


def _gpu_loss(specs):
    F = specs[0]
    return float((F.abs() ** 2).sum()), [torch.view_as_real(2.0 * F).contiguous()]


@pytest.mark.parametrize("dispersive", [False, True])
@pytest.mark.parametrize("slots", [4, 70])
def test_gradient_matches_oracle_fp64(dispersive, slots):
    sc = _design_scene(dispersive)
    o = oracle_from_scene(sc)
    J_ref = gradient_replay(o, sc.n_steps, _oracle_objective)
    g_ref = np.stack([o.grad(a) for a in range(3)])
    ctx = fdtd.Context([sc], dtype="f64")
    runner = ADJ.DesignAdjoint(ctx, slots=slots)
    (J, _), grads, stats = runner.run(sc.n_steps, _gpu_loss)
    assert abs(J - J_ref) <= 1e-12 * abs(J_ref)
    g = grads[0].cpu().numpy().reshape(g_ref.shape)
    assert rel(g, g_ref) < 1e-10, rel(g, g_ref)
    assert stats["adjoint_steps"] == sc.n_steps


def test_native_schedule_executor_matches_per_action_calls():
    # the same schedule run action by action through the ABI and by fdtd_run_schedule: same bits
    sc = _design_scene(True)
    out = []
    for native in (False, True):
        ctx = fdtd.Context([sc], dtype="f32")
        runner = ADJ.DesignAdjoint(ctx, slots=6, pole_grads=True)
        if native:
            (J, _), grads, _ = runner.run(sc.n_steps, _gpu_loss)
        else:
            c = ctx.ctx
            for a in ADJ.schedule(sc.n_steps, 6):
                if a[0] == "save":
                    fdtd.fdtd_state_save(c, a[1], fdtd.FDTD_CODEC_NATIVE)
                elif a[0] == "restore":
                    fdtd.fdtd_state_restore(c, a[1])
                elif a[0] == "advance":
                    fdtd.fdtd_step_forward(c, a[1])
                elif a[0] == "adjoint":
                    fdtd.fdtd_step_adjoint(c, 1)
                else:
                    specs = [ctx.dft(k) for k in range(len(ctx.monitors))]
                    J, cots = _gpu_loss(specs)
                    keep = [ct.contiguous() for ct in cots]
                    fdtd.fdtd_set_adjoint_source(c, ctx.monitors[0][0], keep[0].data_ptr())
                    fdtd.fdtd_adjoint_begin(c)
                    fdtd.fdtd_dft_enable(c, 0)
            fdtd.fdtd_dft_enable(c, 1)
            ctx.synchronize()
            grads = runner.grads
            runner.pole_grads = {0: fdtd.fdtd_pole_grad(c, 0, 2)}
        out.append((J, grads[0].clone(), runner.pole_grads[0].copy()))
        ctx.close()
    assert out[0][0] == out[1][0]
    assert torch.equal(out[0][1], out[1][1])
    # the pole cotangents are FP64 atomic sums over warps, whose order varies between runs
    assert np.max(np.abs(out[0][2] - out[1][2])) <= 1e-12 * np.max(np.abs(out[0][2]))


def test_gradient_fp32_close_to_oracle():
    sc = _design_scene(False)
    o = oracle_from_scene(sc)
    gradient_replay(o, sc.n_steps, _oracle_objective)
    g_ref = np.stack([o.grad(a) for a in range(3)])
    ctx = fdtd.Context([sc], dtype="f32")
    (J, _), grads, _ = ADJ.DesignAdjoint(ctx, slots=8).run(sc.n_steps, _gpu_loss)
    g = grads[0].cpu().numpy().reshape(g_ref.shape)
    assert rel(g, g_ref) < 1e-4, rel(g, g_ref)


def test_autograd_function_matches_driver():
    sc = _design_scene(False)
    ctx = fdtd.Context([sc], dtype="f64")
    (J, _), grads, _ = ADJ.DesignAdjoint(ctx, slots=6).run(sc.n_steps, _gpu_loss)
    g_ref = grads[0].clone()
    ctx2 = fdtd.Context([sc], dtype="f64")
    runner = ADJ.Runner(ctx2, slots=6)
    (lx, ly, lz), (hx, hy, hz) = sc.design
    box = torch.stack([t[lz:hz, ly:hy, lx:hx] for t in ctx2.inv_eps[0]]).clone().requires_grad_(True)
    specs = ADJ.spectra(box, runner, sc.n_steps)
    loss = (specs[0].abs() ** 2).sum()
    loss.backward()
    assert abs(loss.item() - J) <= 1e-12 * abs(J)
    assert rel(box.grad.reshape(-1).cpu().numpy(), g_ref.cpu().numpy()) < 1e-12


# ----------------------------------------------------------------------------- checkpoints
def test_snapshot_native_roundtrip_bitwise_and_bf16_bound():
    sc = small_blocks(40, 6, 200)
    ctx = fdtd.Context([sc], dtype="f32")
    ctx.step(80)
    fdtd.fdtd_state_save(ctx.ctx, 0, fdtd.FDTD_CODEC_NATIVE)
    fdtd.fdtd_state_save(ctx.ctx, 1, fdtd.FDTD_CODEC_BF16)
    saved = [ctx.part(0, p).clone() for p in range(ctx.part_count(0))]
    ctx.step(60)
    after = [ctx.part(0, p).clone() for p in range(ctx.part_count(0))]
    fdtd.fdtd_state_restore(ctx.ctx, 0)
    assert ctx.step_count == 80
    ctx.step(60)
    for p in range(ctx.part_count(0)):
        assert torch.equal(ctx.part(0, p), after[p])
    fdtd.fdtd_state_restore(ctx.ctx, 1)
    nx, ny, nz = sc.shape
    for c in range(6):
        got = ctx.part(0, c).view(nz, ny, nx)
        ref = saved[c].view(nz, ny, nx)
        s = ref.abs().amax(dim=(1, 2), keepdim=True)
        assert torch.all((got - ref).abs() <= s * 2.0 ** -8 + 1e-30)


def test_bf16_snapshot_every_part_anisotropic_poles():
    # CPML memories and pole states too: each restored value within 2^-8 of its slab's max |x|
    sc = W.large_adjoint(n=48, d=4, n_steps=200, margin=2)
    ctx = fdtd.Context([sc], dtype="f32")
    ctx.step(150)
    saved = [ctx.part(0, p).clone() for p in range(ctx.part_count(0))]
    fdtd.fdtd_state_save(ctx.ctx, 3, fdtd.FDTD_CODEC_BF16)
    ctx.step(7)
    fdtd.fdtd_state_restore(ctx.ctx, 3)
    for p in range(ctx.part_count(0)):
        got, ref = ctx.part(0, p), saved[p]
        if not ref.numel():
            continue
        assert torch.isfinite(got).all(), p
        bound = ref.abs().max() * 2.0 ** -8 + 1e-30
        assert (got - ref).abs().max() <= bound, (p, float((got - ref).abs().max()), float(bound))


def test_bf16_snapshot_on_a_grid_with_odd_extents():
    """Parts of odd size (33 x 35 x 37 fields, odd CPML slab arrays): each part's scales follow its
    codes at the next 4-byte boundary, so save and restore work and stay within the BF16 bound."""
    sc = W.cpml_blocks(n=33, d=5, n_steps=120, block=3, region=(9, 24), wavelengths=(8.0, 10.0))
    sc.shape = (33, 35, 37)
    inv = np.ones((37, 35, 33))
    inv[9:24, 9:24, 9:24] = sc.inv_eps[0][9:24, 9:24, 9:24]
    sc.inv_eps = [inv]
    sc.sources[0] = W.Source(W.EZ, (10, 5, 5), (11, 30, 32), W.gaussian_pulse(120, wavelength=10.0, periods=1.0,
                                                                               delay=3.0))
    sc.monitors = [W.Monitor((0, 0, 18), (33, 35, 19), (0, 1, 2), sc.monitors[0].omegas)]
    ctx = fdtd.Context([sc], dtype="f32")
    ctx.step(70)
    sizes = [fdtd.fdtd_part_size(ctx.ctx, 0, p) for p in range(ctx.part_count(0))]
    assert any(n % 2 for n in sizes if n)
    saved = [ctx.part(0, p).clone() for p in range(ctx.part_count(0))]
    fdtd.fdtd_state_save(ctx.ctx, 5, fdtd.FDTD_CODEC_BF16)
    ctx.step(9)
    fdtd.fdtd_state_restore(ctx.ctx, 5)
    assert ctx.step_count == 70
    for p in range(ctx.part_count(0)):
        got, ref = ctx.part(0, p), saved[p]
        if not ref.numel():
            continue
        assert torch.isfinite(got).all(), p
        assert (got - ref).abs().max() <= ref.abs().max() * 2.0 ** -8 + 1e-30, p


# ----------------------------------------------------------------------------- errors
def _grid(nx=16, courant=W.COURANT, dtype=fdtd.FDTD_F32):
    return fdtd.fdtd_grid(nx, nx, nx, 1.0, courant, 0.0, dtype)


def _mat(ie, mask=None, poles=()):
    m = fdtd.fdtd_material()
    for a in range(3):
        m.inv_eps[a] = ie[a].data_ptr()
    m.n_poles = len(poles)
    m.poles = None
    m.pole_mask = mask.data_ptr() if mask is not None else None
    return m


def test_cfl_and_invalid_arguments_rejected():
    ie = torch.ones(16 ** 3, device="cuda")
    cp = fdtd.fdtd_cpml()
    with pytest.raises(fdtd.FdtdError) as e:
        fdtd.fdtd_create([_grid(courant=0.6)], [cp], [_mat([ie] * 3)])
    assert e.value.status == fdtd.FDTD_ECFL
    cp2 = fdtd.fdtd_cpml()
    cp2.cells[0] = 15
    cp2.kappa_max = 1.0
    with pytest.raises(fdtd.FdtdError) as e:
        fdtd.fdtd_create([_grid()], [cp2], [_mat([ie] * 3)])
    assert e.value.status == fdtd.FDTD_EINVAL


def test_tensor_admission_rule_in_cpml():
    n = 16
    cp = fdtd.fdtd_cpml()
    for f in range(6):
        cp.cells[f] = 3
    cp.m, cp.kappa_max, cp.alpha_max, cp.sigma_max = 3.0, 2.0, 0.05, -1.0
    # eps_xx = 2 between eps_yy = 1 and eps_zz = 3 in an x-face: rejected
    bad = [torch.full((n ** 3,), 1 / v, device="cuda") for v in (2.0, 1.0, 3.0)]
    with pytest.raises(fdtd.FdtdError) as e:
        fdtd.fdtd_create([_grid(n)], [cp], [_mat(bad)])
    assert e.value.status == fdtd.FDTD_ETENSOR
    # normal eigenvalue extreme on every face (eps_xx = eps_yy = eps_zz ordering not strict): admitted
    ok = [torch.full((n ** 3,), 1 / v, device="cuda") for v in (2.0, 2.0, 3.0)]
    ctx = fdtd.fdtd_create([_grid(n)], [cp], [_mat(ok)])
    fdtd.fdtd_destroy(ctx)


def test_nonfinite_detection_and_adjoint_state_rules():
    sc = _design_scene(False)
    ctx = fdtd.Context([sc], dtype="f32")
    runner = ADJ.DesignAdjoint(ctx, slots=4)
    ctx.step(4)
    fdtd.fdtd_state_save(ctx.ctx, 0, fdtd.FDTD_CODEC_NATIVE)
    ctx.step(1)
    fdtd.fdtd_adjoint_begin(ctx.ctx)            # adjoint index 5
    with pytest.raises(fdtd.FdtdError) as e:
        fdtd.fdtd_step_adjoint(ctx.ctx, 1)      # transposing step 4 needs u^4, u^5 is held
    assert e.value.status == fdtd.FDTD_ESTATE
    fdtd.fdtd_state_restore(ctx.ctx, 0)
    fdtd.fdtd_step_adjoint(ctx.ctx, 1)          # u^4 held: allowed
    with pytest.raises(fdtd.FdtdError) as e:
        fdtd.fdtd_step_adjoint(ctx.ctx, 1)      # needs u^3
    assert e.value.status == fdtd.FDTD_ESTATE
    fdtd.fdtd_check_finite(ctx.ctx)
    f = ctx.part(0, 2)
    f[123] = float("nan")
    ctx.set_part(0, 2, f)
    with pytest.raises(fdtd.FdtdError) as e:
        fdtd.fdtd_check_finite(ctx.ctx)
    assert e.value.status == fdtd.FDTD_ENONFINITE
    del runner


@pytest.mark.parametrize("which,dtype", [("blocks", "f32"), ("batch", "f32"), ("blocks", "f64"), ("rows42", "f32")])
def test_tile_and_per_cell_launch_modes_bitwise_equal(which, dtype):
    # both launch modes (tile launches over all domains, per-cell launches per domain) run the
    # same arithmetic per cell, so the states and spectra must agree bit for bit (42-cell rows: a
    # row width that is no multiple of a warp)
    if which == "blocks":
        scs = [small_blocks(40, 6, 150)]
    elif which == "rows42":
        scs = [small_blocks(42, 6, 150)]
    else:
        scs = _tiny_batch(3, 150)
    outs = []
    for mode in fdtd.MODES:
        ctx = fdtd.Context(scs, dtype=dtype)
        fdtd.fdtd_set_launch_mode(ctx.ctx, mode)
        ctx.step(70)
        ctx.step(80)   # two calls: the device step counter carries across launches
        assert ctx.step_count == 150
        outs.append(([ctx.part(d, p).clone() for d in range(len(scs)) for p in range(ctx.part_count(d))],
                     [ctx.dft(k).clone() for k in range(len(ctx.monitors))]))
        ctx.close()
    for other in outs[1:]:
        for a, b in zip(outs[0][0], other[0]):
            assert torch.equal(a, b)
        for a, b in zip(outs[0][1], other[1]):
            assert torch.equal(a, b)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_monitor_ring_fold_matches_per_step_dft(dtype):
    # the per-cell mode stores monitor samples during a batch of steps and folds them into the DFT
    # once per batch; a second monitor in the same domain turns the rings off (one DFT launch per
    # half-step): the shared monitor's spectra must agree bit for bit, over batches of 32 steps
    # (graphs) and of 1 to 31 (eager remainders)
    sc = small_blocks(40, 6, 150)
    sc2 = small_blocks(40, 6, 150)
    sc2.monitors.append(W.Monitor((4, 4, 4), (12, 12, 5), (W.EX, W.HZ), sc2.monitors[0].omegas))
    specs = []
    for s, prof in ((sc, False), (sc2, False), (sc, True)):
        ctx = fdtd.Context([s], dtype=dtype)
        fdtd.fdtd_set_launch_mode(ctx.ctx, 4)
        if prof:
            # per-launch profiling steps without graphs: eager batches of at most 32 steps
            fdtd.fdtd_profile_begin(ctx.ctx, 4096)
        for n in (70, 1, 31, 48):
            ctx.step(n)
        if prof:
            fdtd.fdtd_profile_end(ctx.ctx)
        specs.append(ctx.dft(0).clone())
        if s is sc and not prof:
            # the fold of one batch can be timed on its own; the per-step form has no rings
            assert fdtd.fdtd_time_half_steps(ctx.ctx, 5, 2) > 0
        elif s is sc2:
            with pytest.raises(fdtd.FdtdError):
                fdtd.fdtd_time_half_steps(ctx.ctx, 5, 2)
        ctx.close()
    assert torch.equal(specs[0], specs[1])
    assert torch.equal(specs[0], specs[2])
    assert float(specs[0].abs().max()) > 0


def test_bf16_snapshot_denormal_slab_stays_finite():
    # a slab whose largest value is an FP32 denormal (the leading edge of a wave far from the
    # source) must round-trip without NaN
    sc = small_blocks(24, 4, 10)
    ctx = fdtd.Context([sc], dtype="f32")
    nx, ny, nz = sc.shape
    ez = torch.zeros(nz, ny, nx, device="cuda")
    ez[5, 3, 7] = 1e-40
    ez[5, 3, 8] = -3e-41
    ez[9, 2, 2] = 0.75
    ctx.set_part(0, 2, ez.view(-1))
    fdtd.fdtd_state_save(ctx.ctx, 0, fdtd.FDTD_CODEC_BF16)
    ctx.set_part(0, 2, torch.zeros_like(ez).view(-1))
    fdtd.fdtd_state_restore(ctx.ctx, 0)
    got = ctx.part(0, 2).view(nz, ny, nx)
    assert torch.isfinite(got).all()
    assert abs(float(got[9, 2, 2]) - 0.75) <= 0.75 * 2.0 ** -8
    assert float(got[5, 3, 7]) > 0 and float(got[5, 3, 8]) < 0
    assert float(got.abs().sum()) - 0.75 < 1e-3


def test_autotune_keeps_state_and_spectra():
    sc = small_blocks(40, 6, 120)
    ref = fdtd.Context([sc], dtype="f32")
    ref.step(60)
    ctx = fdtd.Context([sc], dtype="f32")
    ctx.step(30)
    ms = fdtd.fdtd_autotune(ctx.ctx, 12)
    assert [m > 0 for m in ms] == [q in fdtd.MODES for q in range(fdtd.LAUNCH_MODES)]
    assert fdtd.fdtd_get_launch_mode(ctx.ctx) in fdtd.MODES
    assert ctx.step_count == 30
    ctx.step(30)
    for p in range(ctx.part_count(0)):
        assert torch.equal(ctx.part(0, p), ref.part(0, p))
    assert torch.equal(ctx.dft(0), ref.dft(0))


@pytest.mark.parametrize("mode", [0, 4])
def test_new_material_after_graph_capture(mode):
    # graphs captured before a material change must not keep the old eps^-1 arrays
    sc = small_blocks(40, 6, 80)
    ctx = fdtd.Context([sc], dtype="f32")
    fdtd.fdtd_set_launch_mode(ctx.ctx, mode)
    ctx.step(64)                                   # two graph replays captured with the old material
    inv = torch.from_numpy(np.ascontiguousarray(sc.inv_eps3()[0])).to(device=ctx.device, dtype=torch.float32) * 0.5
    ctx.set_inv_eps(0, [inv, inv, inv])
    fdtd.fdtd_reset(ctx.ctx)
    fdtd.fdtd_dft_reset(ctx.ctx)
    ctx.step(64)
    ref = fdtd.Context([sc], dtype="f32")
    fdtd.fdtd_set_launch_mode(ref.ctx, mode)
    ref.set_inv_eps(0, [inv.clone(), inv.clone(), inv.clone()])
    ref.step(64)
    for p in range(ctx.part_count(0)):
        assert torch.equal(ctx.part(0, p), ref.part(0, p))
    assert torch.equal(ctx.dft(0), ref.dft(0))
