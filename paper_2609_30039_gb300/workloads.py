"""Seeded synthetic workloads (inputs only).

This module holds none of the method's arithmetic: it draws permittivity maps, pole
parameters, design densities and source waveforms with numpy's PCG64 generator and
describes sources, monitors and design boxes.  Both the CUDA path (through the C-ABI
binding) and the FP64 oracle consume the same `Scene` objects, so no random number is
ever generated twice.

The five workloads are synthetic stand-ins for the paper's scenes (which are not
available): grids, CPML depths, material ranges, source types and monitor layouts follow
the benchmark descriptions; everything is reduced units (c = eps0 = mu0 = 1, dx = 1,
dt = S = Courant number).  A `scale` argument builds geometrically similar smaller
replicas for tests.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

COURANT = 0.99 / math.sqrt(3.0)
SEED0 = 2609030039
LORENTZ, DRUDE = 0, 1
EX, EY, EZ, HX, HY, HZ = range(6)


@dataclasses.dataclass
class Source:
    comp: int
    lo: Tuple[int, int, int]
    hi: Tuple[int, int, int]
    wave: np.ndarray            # wave[n] is added at forward step n (E: time n+1, H: n+3/2)


@dataclasses.dataclass
class Monitor:
    lo: Tuple[int, int, int]
    hi: Tuple[int, int, int]
    comps: Tuple[int, ...]
    omegas: np.ndarray          # rad / step


@dataclasses.dataclass
class Scene:
    shape: Tuple[int, int, int]                 # (nx, ny, nz)
    n_steps: int
    courant: float = COURANT
    cpml: Tuple[int, ...] = (0, 0, 0, 0, 0, 0)  # cells on -x,+x,-y,+y,-z,+z (0 = PEC face)
    cpml_m: float = 3.0
    kappa_max: float = 1.0
    alpha_max: float = 0.0
    sigma_max: float = -1.0                     # < 0: 0.8 (m + 1)
    inv_eps: Optional[Sequence[np.ndarray]] = None   # 1 (isotropic) or 3 arrays (nz, ny, nx), float64
    poles: Tuple[Tuple[int, float, float, float], ...] = ()   # (kind, deps, omega_dt, gamma_dt)
    pole_mask: Optional[np.ndarray] = None      # uint8 (nz, ny, nx)
    sources: List[Source] = dataclasses.field(default_factory=list)
    monitors: List[Monitor] = dataclasses.field(default_factory=list)
    design: Optional[Tuple[Tuple[int, int, int], Tuple[int, int, int]]] = None
    rho: Optional[np.ndarray] = None            # design densities
    energy: bool = False
    name: str = ""
    periodic: Tuple[int, int, int] = (0, 0, 0)   # periodic x / y (z must be 0)
    # symmetric eps^-1 tensor per grid node (Sec. 2.3 node assembly), shape (6, nz, ny, nx), components
    # xx, yy, zz, xy, xz, yz; replaces inv_eps in the E update (no poles)
    tensor: Optional[np.ndarray] = None

    @property
    def cells(self) -> int:
        return int(np.prod(self.shape))

    def inv_eps3(self):
        if self.inv_eps is None:
            one = np.ones(self.shape[::-1])
            return [one, one, one]
        if len(self.inv_eps) == 1:
            return [self.inv_eps[0]] * 3
        return list(self.inv_eps)


# ------------------------------------------------------------------ waveforms
def gaussian_derivative(n_steps: int, t0: float = 30.0, spread: float = 10.0) -> np.ndarray:
    """g(t) = -((t-t0)/s) exp(-(t-t0)^2 / (2 s^2)), sampled at t = n+1 (time of E^{n+1})."""
    t = np.arange(n_steps, dtype=np.float64) + 1.0
    u = (t - t0) / spread
    return -u * np.exp(-0.5 * u * u)


def gaussian_pulse(n_steps: int, wavelength: float = 20.0, courant: float = COURANT,
                   periods: float = 2.0, delay: float = 4.0) -> np.ndarray:
    """sin(w0 (t-t0)) exp(-(t-t0)^2/(2 tau^2)); w0 = 2 pi S / lambda, tau = periods * lambda / S,
    t0 = delay * tau; sampled at t = n+1."""
    w0 = 2.0 * math.pi * courant / wavelength
    tau = periods * wavelength / courant
    t0 = delay * tau
    t = np.arange(n_steps, dtype=np.float64) + 1.0
    return np.sin(w0 * (t - t0)) * np.exp(-0.5 * ((t - t0) / tau) ** 2)


def rotation(axis: int, angle: float) -> np.ndarray:
    """Rotation matrix about coordinate axis 0, 1 or 2 by angle (radians)."""
    c, s = math.cos(angle), math.sin(angle)
    b, d = (axis + 1) % 3, (axis + 2) % 3
    R = np.eye(3)
    R[b, b], R[b, d], R[d, b], R[d, d] = c, -s, s, c
    return R


def inv_tensor6(eps: np.ndarray) -> np.ndarray:
    """The six components (xx, yy, zz, xy, xz, yz) of eps^-1 for a symmetric 3 x 3 eps, or for an
    array of them with the matrix axes last."""
    inv = np.linalg.inv(np.asarray(eps, dtype=np.float64))
    return np.stack([inv[..., 0, 0], inv[..., 1, 1], inv[..., 2, 2], inv[..., 0, 1], inv[..., 0, 2], inv[..., 1, 2]])


def principal_eps(principal, R=None) -> np.ndarray:
    """eps = R diag(principal) R^T (principal axes rotated by R)."""
    D = np.diag(np.asarray(principal, dtype=np.float64))
    return D if R is None else R @ D @ R.T


def omegas_for(wavelengths, courant: float = COURANT) -> np.ndarray:
    return np.array([2.0 * math.pi * courant / lam for lam in wavelengths], dtype=np.float64)


def _rng(index: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED0 + index + 1000 * salt))


# ------------------------------------------------------------------ workloads
def pec_vacuum(n: int = 32, n_steps: int = 200) -> Scene:
    """Plain FP64 vacuum in a PEC box, Gaussian-derivative Ez point source at the centre."""
    c = n // 2
    return Scene(shape=(n, n, n), n_steps=n_steps, name=f"pec_vacuum_{n}^3",
                 sources=[Source(EZ, (c, c, c), (c + 1, c + 1, c + 1), gaussian_derivative(n_steps))],
                 energy=True)


def cpml_blocks(n: int = 128, d: int = 10, n_steps: int = 2000, block: int = 8, seed_index: int = 1,
                region: Optional[Tuple[int, int]] = None, wavelengths=(18.0, 20.0, 22.0)) -> Scene:
    """CPML box with a central cube of blocky random eps_r in [1, 12]; Ez soft sheet source
    (Gaussian pulse, centre wavelength 20 cells); DFT of all six components on the z mid-plane."""
    rng = _rng(seed_index)
    lo, hi = region if region is not None else (n // 4, n - n // 4)
    inv = np.ones((n, n, n))
    nb = -(-(hi - lo) // block)
    blocks = rng.uniform(1.0, 12.0, size=(nb, nb, nb))
    eps = np.repeat(np.repeat(np.repeat(blocks, block, 0), block, 1), block, 2)[: hi - lo, : hi - lo, : hi - lo]
    inv[lo:hi, lo:hi, lo:hi] = 1.0 / eps
    xs = d + 5
    src = Source(EZ, (xs, d, d), (xs + 1, n - d, n - d), gaussian_pulse(n_steps))
    mon = Monitor((0, 0, n // 2), (n, n, n // 2 + 1), (EX, EY, EZ, HX, HY, HZ), omegas_for(wavelengths))
    return Scene(shape=(n, n, n), n_steps=n_steps, cpml=(d,) * 6, kappa_max=5.0, alpha_max=0.05,
                 inv_eps=[inv], sources=[src], monitors=[mon], name=f"cpml_blocks_{n}^3")


def tensor_blocks(n: int = 256, d: int = 10, n_steps: int = 200, block: int = 8, seed_index: int = 6,
                  wavelengths=(18.0, 20.0, 22.0)) -> Scene:
    """The cpml_blocks box with anisotropic blocks (Sec. 2.3 tensors at the nodes): every 8^3 block of
    the central cube holds eps with principal values uniform in [1, 4] (indices up to 2, like the
    birefringent media of the paper's validation) along random principal axes; vacuum elsewhere,
    so every CPML node holds the identity (admitted)."""
    rng = _rng(seed_index)
    sc = cpml_blocks(n=n, d=d, n_steps=n_steps, block=block, seed_index=seed_index, wavelengths=wavelengths)
    lo, hi = n // 4, n - n // 4
    nb = -(-(hi - lo) // block)
    Q, _ = np.linalg.qr(rng.standard_normal((nb ** 3, 3, 3)))
    lam = rng.uniform(1.0, 4.0, size=(nb ** 3, 3))
    blocks = inv_tensor6(np.einsum("nij,nj,nkj->nik", Q, lam, Q)).reshape(6, nb, nb, nb)
    t = np.zeros((6, n, n, n))
    t[0] = t[1] = t[2] = 1.0
    for q in range(6):
        big = np.repeat(np.repeat(np.repeat(blocks[q], block, 0), block, 1), block, 2)
        t[q, lo:hi, lo:hi, lo:hi] = big[: hi - lo, : hi - lo, : hi - lo]
    sc.inv_eps = None
    sc.tensor = t
    sc.name = f"tensor_blocks_{n}^3"
    return sc


def density_to_eps(rho: np.ndarray) -> np.ndarray:
    """Design map eps_r = 1 + 11 sigmoid(8 (rho - 0.5)) (the workload's material producer)."""
    return 1.0 + 11.0 / (1.0 + np.exp(-8.0 * (rho - 0.5)))


def adjoint_design(n: int = 256, d: int = 12, n_steps: int = 3000, seed_index: int = 2,
                   wavelengths=(18.0, 20.0, 22.0)) -> Scene:
    """Adjoint workload: design box (x,y in [n/4, 3n/4), z in [7n/16, 9n/16)) of per-cell random
    densities, Ex soft sheet, objective = sum |F_Ex|^2 over a 16x16 patch of the plane z = 200/256 n."""
    rng = _rng(seed_index)
    q = n // 4
    zlo, zhi = (7 * n) // 16, (9 * n) // 16
    design = ((q, q, zlo), (n - q, n - q, zhi))
    rho = rng.uniform(0.0, 1.0, size=(zhi - zlo, n - 2 * q, n - 2 * q))
    inv = np.ones((n, n, n))
    inv[zlo:zhi, q:n - q, q:n - q] = 1.0 / density_to_eps(rho)
    zs = d + max(1, (8 * n) // 256)
    src = Source(EX, (d, d, zs), (n - d, n - d, zs + 1), gaussian_pulse(n_steps))
    zt = (200 * n) // 256
    c, hw = n // 2, max(1, n // 32)
    mon = Monitor((c - hw, c - hw, zt), (c + hw, c + hw, zt + 1), (EX,), omegas_for(wavelengths))
    return Scene(shape=(n, n, n), n_steps=n_steps, cpml=(d,) * 6, kappa_max=5.0, alpha_max=0.05,
                 inv_eps=[inv], sources=[src], monitors=[mon], design=design, rho=rho,
                 name=f"adjoint_design_{n}^3")


def lorentz_batch(n_domains: int = 64, sizes=(48, 56, 64, 72, 80, 88, 96), d: int = 8,
                  n_steps: int = 1500, seed_index: int = 3) -> List[Scene]:
    """Independent domains of uneven size, 2-pole Lorentz (eps_inf = 2) in a random half-space
    outside the CPML, a point Ez source and a point DFT monitor per domain."""
    rng = _rng(seed_index)
    scenes = []
    for b in range(n_domains):
        nx, ny, nz = (int(v) for v in rng.choice(sizes, size=3))
        poles = tuple((LORENTZ, float(rng.uniform(0.5, 3.0)), float(rng.uniform(0.05, 0.3)),
                       float(rng.uniform(0.001, 0.02))) for _ in range(2))
        axis = int(rng.integers(0, 3))
        ext = (nx, ny, nz)[axis]
        cut = int(rng.integers(ext // 3, 2 * ext // 3 + 1))
        mask = np.zeros((nz, ny, nx), dtype=np.uint8)
        sl = [slice(d, nz - d), slice(d, ny - d), slice(d, nx - d)]
        ax_np = 2 - axis
        sl[ax_np] = slice(max(cut, d), (nz, ny, nx)[ax_np] - d)
        mask[tuple(sl)] = 1
        inv = np.ones((nz, ny, nx))
        inv[mask == 1] = 0.5
        p = [int(rng.integers(d + 2, v - d - 2)) for v in (nx, ny, nz)]
        src = Source(EZ, tuple(p), tuple(v + 1 for v in p), gaussian_pulse(n_steps))
        mp = [int(rng.integers(d + 2, v - d - 2)) for v in (nx, ny, nz)]
        mon = Monitor(tuple(mp), tuple(v + 1 for v in mp), (EZ, HX), omegas_for((18.0, 20.0, 22.0)))
        scenes.append(Scene(shape=(nx, ny, nz), n_steps=n_steps, cpml=(d,) * 6, kappa_max=5.0,
                            alpha_max=0.05, inv_eps=[inv], poles=poles, pole_mask=mask,
                            sources=[src], monitors=[mon], name=f"lorentz_domain_{b}"))
    return scenes


def large_adjoint(n: int = 640, d: int = 16, n_steps: int = 4000, seed_index: int = 4, block: int = 4,
                  layer=None, margin: int = 4) -> Scene:
    """Diagonal anisotropic eps (xx, yy, zz each U[1, 6] per 4^3 block) in the interior (CPML and a
    4-cell margin stay vacuum), 2-pole Lorentz design layer (512 x 512 x 64 at n = 640) whose
    eps_inf,a = 1 + (eps_block,a - 1) sigmoid(8 (rho(x,y) - 0.5)); Ey sheet; DFT of Ey on a far
    plane at 2 frequencies."""
    rng = _rng(seed_index)
    lo, hi = d + margin, n - d - margin
    m = hi - lo
    nb = -(-m // block)
    inv = []
    blocks_a = []
    for a in range(3):
        blk = rng.uniform(1.0, 6.0, size=(nb, nb, nb))
        blocks_a.append(blk)
        e = np.repeat(np.repeat(np.repeat(blk, block, 0), block, 1), block, 2)[:m, :m, :m]
        arr = np.ones((n, n, n))
        arr[lo:hi, lo:hi, lo:hi] = 1.0 / e
        inv.append(arr)
    if layer is None:
        w = (512 * n) // 640
        t = (64 * n) // 640
        z0 = (288 * n) // 640
        x0 = (n - w) // 2
        layer = ((x0, x0, z0), (x0 + w, x0 + w, z0 + t))
    (lx, ly, lz), (hx, hy, hz) = layer
    rho = rng.uniform(0.0, 1.0, size=(hy - ly, hx - lx))
    sig = 1.0 / (1.0 + np.exp(-8.0 * (rho - 0.5)))
    for a in range(3):
        cur = 1.0 / inv[a][lz:hz, ly:hy, lx:hx]
        inv[a][lz:hz, ly:hy, lx:hx] = 1.0 / (1.0 + (cur - 1.0) * sig[None, :, :])
    poles = tuple((LORENTZ, float(rng.uniform(0.5, 3.0)), float(rng.uniform(0.05, 0.3)),
                   float(rng.uniform(0.001, 0.02))) for _ in range(2))
    mask = np.zeros((n, n, n), dtype=np.uint8)
    mask[lz:hz, ly:hy, lx:hx] = 1
    zs = d + 8
    src = Source(EY, (d, d, zs), (n - d, n - d, zs + 1), gaussian_pulse(n_steps))
    zf = (600 * n) // 640
    mon = Monitor((lx, ly, zf), (hx, hy, zf + 1), (EY,), omegas_for((19.0, 21.0)))
    return Scene(shape=(n, n, n), n_steps=n_steps, cpml=(d,) * 6, kappa_max=5.0, alpha_max=0.05,
                 inv_eps=inv, poles=poles, pole_mask=mask, sources=[src], monitors=[mon],
                 design=layer, rho=rho, name=f"large_adjoint_{n}^3")


def random_state_scene(shape=(9, 8, 7), d: int = 2, n_poles: int = 2, aniso: bool = True,
                       seed_index: int = 11, periodic: bool = False) -> Scene:
    """Tiny grid with CPML on every face (periodic: x and y periodic, CPML on the z faces only),
    anisotropic eps and a dispersive box: the operator under the dot-product (transpose) tests."""
    rng = _rng(seed_index)
    nx, ny, nz = shape
    inv = [1.0 / rng.uniform(1.0, 4.0, size=(nz, ny, nx)) for _ in range(3 if aniso else 1)]
    if aniso and d > 0:
        # inside the absorbing slabs the tensor must pass the admission rule: keep it isotropic
        slab = np.zeros((nz, ny, nx), dtype=bool)
        slab[:d], slab[nz - d:] = True, True
        if not periodic:
            slab[:, :d], slab[:, ny - d:], slab[:, :, :d], slab[:, :, nx - d:] = (True,) * 4
        for a in (1, 2):
            inv[a][slab] = inv[0][slab]
    poles = tuple((LORENTZ, float(rng.uniform(0.5, 3.0)), float(rng.uniform(0.05, 0.3)),
                   float(rng.uniform(0.01, 0.05))) for _ in range(n_poles))
    mask = np.zeros((nz, ny, nx), dtype=np.uint8)
    mask[nz // 3: nz - 1, 1: ny - 2, nx // 2: nx] = 1 if n_poles else 0
    cpml = (0, 0, 0, 0, d, d) if periodic else (d,) * 6
    return Scene(shape=shape, n_steps=10, cpml=cpml, kappa_max=3.0, alpha_max=0.05,
                 inv_eps=inv, poles=poles, pole_mask=mask, name="random_state",
                 periodic=(1, 1, 0) if periodic else (0, 0, 0))


def lossless_design(n: int = 256, n_steps: int = 2000, seed_index: int = 13,
                    wavelengths=(18.0, 20.0, 22.0)) -> Scene:
    """Lossless nondispersive n^3 box for the reversible gradient: periodic in x, PEC in y and z
    (no CPML), eps_r ~ U[1, 6] in 8^3 blocks, an Ez sheet at z = n/8, a design box against the
    x = 0 seam (x in [0, n/8), y in [3n/8, 5n/8), z in [7n/16, 9n/16)) and an Ex DFT patch."""
    rng = _rng(seed_index)
    b = 8
    eps = rng.uniform(1.0, 6.0, size=(n // b, n // b, n // b))
    inv = 1.0 / np.repeat(np.repeat(np.repeat(eps, b, 0), b, 1), b, 2)
    zs = n // 8
    src = Source(EZ, (0, 1, zs), (n, n, zs + 1), gaussian_pulse(n_steps))
    zt = (3 * n) // 4
    c, hw = n // 2, max(1, n // 32)
    mon = Monitor((c - hw, c - hw, zt), (c + hw, c + hw, zt + 1), (EX,), omegas_for(wavelengths))
    design = ((0, (3 * n) // 8, (7 * n) // 16), (n // 8, (5 * n) // 8, (9 * n) // 16))
    return Scene(shape=(n, n, n), n_steps=n_steps, cpml=(0,) * 6, inv_eps=[inv], sources=[src], monitors=[mon],
                 design=design, periodic=(1, 0, 0), name=f"lossless_design_{n}^3")


def periodic_cell(shape=(24, 20, 48), d: int = 8, n_steps: int = 300, layer=(18, 30), block: int = 4,
                  seed_index: int = 12, wavelengths=(9.0, 10.0, 11.0)) -> Scene:
    """Periodic unit cell (x and y periodic, CPML on both z faces): eps_r ~ U[1, 6] per block of
    block^2 columns in the layer z in [layer), an Ex sheet below it, a two-plane flux monitor
    (Ex, Ey, Hx, Hy) above it and a plane monitor of all six components inside it."""
    rng = _rng(seed_index)
    nx, ny, nz = shape
    inv = np.ones((nz, ny, nx))
    bx, by = -(-nx // block), -(-ny // block)
    eps = rng.uniform(1.0, 6.0, size=(by, bx))
    inv[layer[0]:layer[1]] = 1.0 / np.repeat(np.repeat(eps, block, 0), block, 1)[:ny, :nx]
    zs, zt = d + 2, layer[1] + 4
    src = Source(EX, (0, 0, zs), (nx, ny, zs + 1), gaussian_pulse(n_steps, wavelength=wavelengths[1], periods=1.0,
                                                                    delay=3.0))
    om = omegas_for(wavelengths)
    flux = Monitor((0, 0, zt), (nx, ny, zt + 2), (EX, EY, HX, HY), om)
    plane = Monitor((0, 0, (layer[0] + layer[1]) // 2), (nx, ny, (layer[0] + layer[1]) // 2 + 1), (0, 1, 2, 3, 4, 5),
                    om)
    return Scene(shape=shape, n_steps=n_steps, cpml=(0, 0, 0, 0, d, d), kappa_max=3.0, alpha_max=0.05,
                 inv_eps=[inv], sources=[src], monitors=[flux, plane], periodic=(1, 1, 0), name="periodic_cell")


def slab_cell(n_index: float = 1.5, thickness: int = 20, nz: int = 260, d: int = 16, n_steps: int = 3000,
              wavelengths=(30.0, 40.0, 50.0, 60.0), with_slab: bool = True) -> Scene:
    """Normal incidence on a lossless slab: a 2 x 2 periodic cell (a plane wave), CPML on both z
    faces, an Ex sheet, a reflection flux monitor between sheet and slab and a transmission flux
    monitor beyond it (the reference run is the same cell with with_slab=False)."""
    z1, zs, zr, zt = 140, d + 10, 60, 200
    inv = np.ones((nz, 2, 2))
    if with_slab:
        inv[z1:z1 + thickness] = 1.0 / n_index ** 2
    om = omegas_for(wavelengths)
    src = Source(EX, (0, 0, zs), (2, 2, zs + 1), gaussian_pulse(n_steps, wavelength=40.0, periods=1.0, delay=3.0))
    mons = [Monitor((0, 0, zr), (2, 2, zr + 2), (EX, EY, HX, HY), om),
            Monitor((0, 0, zt), (2, 2, zt + 2), (EX, EY, HX, HY), om)]
    return Scene(shape=(2, 2, nz), n_steps=n_steps, cpml=(0, 0, 0, 0, d, d), kappa_max=1.0, alpha_max=0.0,
                 inv_eps=[inv], sources=[src], monitors=mons, periodic=(1, 1, 0), name="slab_cell")


def random_state(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.standard_normal(n)
