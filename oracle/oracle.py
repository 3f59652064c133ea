"""FP64 CPU oracle of the Yee/CPML/ADE step and its discrete adjoint (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; the product path never imports it.  The arithmetic lives
in ``fdtd_oracle.c`` (plain C, full-grid FP64 arrays, one thread unless a team is asked for);
this module only compiles it with gcc, marshals arguments and exposes numpy views.

Paper passages followed (arxiv 2609.30039): Sec. 2.1 Eq. (yee) and the half-step time
bookkeeping; Sec. 2.2 CPML and PEC; Sec. 2.3 diagonal permittivity and trapezoidal
Drude/Lorentz poles, symmetric node tensors with the node assembly and their admission rule; Sec. 2.4 plane DFT monitors; Sec. 3.1 Eq. (adjoint) and the CPML /
pole transposes; Sec. 3.2 checkpoint replay (here a plain two-level store-all replay) and the
reversible reconstruction (backward steps of Eq. (yee)).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdtd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: -O3, ISO C99 (so no multiply-add contraction: every
    operation rounds on its own, on x86 and Arm alike), portable (no -march flags), with OpenMP
    for the optional cell-loop team (see Oracle.set_threads); without libgomp it builds serial."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O3", "-fPIC", "-shared", "-std=c99", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        vp = C.c_void_p
        sig = {
            "oracle_create": (vp, [C.c_int, C.c_int, C.c_int, C.c_double, _ip, _ip, C.c_double, C.c_double,
                                   C.c_double, C.c_double]),
            "oracle_destroy": (None, [vp]),
            "oracle_set_material": (None, [vp, _dp, _dp, _dp, C.c_int, _ip, _dp, _dp, _dp,
                                           C.POINTER(C.c_ubyte)]),
            "oracle_add_source": (C.c_int, [vp, C.c_int, _ip, _ip, _dp, C.c_int]),
            "oracle_add_dft_box": (C.c_int, [vp, _ip, _ip, C.c_uint, C.c_int, _dp]),
            "oracle_enable_energy": (None, [vp, C.c_long]),
            "oracle_step": (None, [vp, C.c_int]),
            "oracle_set_threads": (None, [vp, C.c_int]),
            "oracle_step_backward": (C.c_int, [vp, C.c_int]),
            "oracle_step_backward_interior": (C.c_int, [vp, _dp, _dp, _dp, _dp, _dp, _dp]),
            "oracle_field": (_dp, [vp, C.c_int]),
            "oracle_psi": (_dp, [vp, C.c_int, C.c_int, C.c_int]),
            "oracle_pole": (_dp, [vp, C.c_int, C.c_int, C.c_int]),
            "oracle_dft": (_dp, [vp, C.c_int]),
            "oracle_dft_len": (C.c_long, [vp, C.c_int]),
            "oracle_energy": (_dp, [vp]),
            "oracle_step_count": (C.c_long, [vp]),
            "oracle_set_step": (None, [vp, C.c_long]),
            "oracle_coef": (_dp, [vp, C.c_int, C.c_int, C.c_int]),
            "oracle_pole_coef": (None, [vp, C.c_int, _dp, _dp]),
            "oracle_state_len": (C.c_long, [vp]),
            "oracle_state_get": (None, [vp, _dp, C.c_int]),
            "oracle_state_set": (None, [vp, _dp, C.c_int]),
            "oracle_dft_reset": (None, [vp]),
            "oracle_set_adjoint_source": (None, [vp, C.c_int, _dp]),
            "oracle_set_design": (C.c_int, [vp, _ip, _ip]),
            "oracle_grad": (_dp, [vp, C.c_int]),
            "oracle_adj_field": (_dp, [vp, C.c_int]),
            "oracle_adj_reset": (None, [vp]),
            "oracle_adjoint_step": (None, [vp, C.c_long]),
            "oracle_pole_grad": (None, [vp, _dp]),
            "oracle_pole_coef_grad": (None, [vp, _dp]),
            "oracle_set_tensor": (C.c_int, [vp, _dp]),
            "oracle_tensor_apply": (C.c_int, [vp, _dp, _dp, _dp, _dp, _dp, _dp]),
            "oracle_tensor_D": (_dp, [vp, C.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(seq):
    arr = (C.c_int * len(seq))(*[int(v) for v in seq])
    return C.cast(arr, _ip), arr


LORENTZ, DRUDE = 0, 1


class Oracle:
    """One FP64 domain.  Arrays are (nz, ny, nx) numpy views, x fastest."""

    def __init__(self, shape, courant, periodic=(0, 0, 0), cpml=(0, 0, 0, 0, 0, 0), m=3.0,
                 kappa_max=1.0, alpha_max=0.0, sigma_max=-1.0):
        self.lib = _load()
        nx, ny, nz = (int(v) for v in shape)
        self.shape = (nx, ny, nz)
        self.courant = float(courant)
        pp, self._pp = _i(periodic)
        cp, self._cp = _i(cpml)
        self.h = self.lib.oracle_create(nx, ny, nz, float(courant), pp, cp, float(m), float(kappa_max),
                                        float(alpha_max), float(sigma_max))
        self.n = nx * ny * nz
        self.npole = 0
        self._mons = []

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.oracle_destroy(h)
            self.h = None

    # -- set-up -----------------------------------------------------------------------
    def set_material(self, inv_eps, poles=(), mask=None):
        """inv_eps: array (nz,ny,nx) (isotropic) or sequence of three such arrays.
        poles: sequence of (kind, deps, omega_dt, gamma_dt); kind LORENTZ or DRUDE."""
        if isinstance(inv_eps, np.ndarray) and inv_eps.ndim == 3:
            ie = [inv_eps] * 3
        else:
            ie = list(inv_eps)
        ie = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in ie]
        for a in ie:
            assert a.size == self.n
        npole = len(poles)
        kinds = np.array([p[0] for p in poles] or [0], dtype=np.int32)
        deps = np.array([p[1] for p in poles] or [0.0], dtype=np.float64)
        w = np.array([p[2] for p in poles] or [0.0], dtype=np.float64)
        g = np.array([p[3] for p in poles] or [0.0], dtype=np.float64)
        mk = None
        if mask is not None:
            mk = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
            assert mk.size == self.n
        self._keep = (ie, kinds, deps, w, g, mk)
        self.lib.oracle_set_material(self.h, _d(ie[0]), _d(ie[1]), _d(ie[2]), npole,
                                     kinds.ctypes.data_as(_ip), _d(deps), _d(w), _d(g),
                                     mk.ctypes.data_as(C.POINTER(C.c_ubyte)) if mk is not None else None)
        self.npole = npole

    def set_tensor(self, t6):
        """Tensor mode (Sec. 2.3): t6 = the six components (xx, yy, zz, xy, xz, yz) of eps^-1 at
        every grid node, shape (6, nz, ny, nx); the E update then applies the node assembly
        S_t = D^{-1/2} (1/8 sum R^T eps^-1 R) D^{-1/2} to the curl.  None switches it off.  Not
        with poles or an energy record."""
        if t6 is None:
            self.lib.oracle_set_tensor(self.h, None)
            self.tensor = False
            return
        t = np.ascontiguousarray(t6, dtype=np.float64).reshape(-1)
        assert t.size == 6 * self.n
        if self.lib.oracle_set_tensor(self.h, _d(t)) != 0:
            raise ValueError("tensor mode excludes poles and the energy record")
        self.tensor = True

    def tensor_apply(self, v):
        """S_t applied to three E-component arrays (tensor mode)."""
        nx, ny, nz = self.shape
        vin = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in v]
        out = [np.zeros(self.n) for _ in range(3)]
        r = self.lib.oracle_tensor_apply(self.h, *[_d(a) for a in vin], *[_d(a) for a in out])
        assert r == 0
        return [a.reshape(nz, ny, nx) for a in out]

    def tensor_D(self, a):
        """The diagonal of D = 1/8 sum R^T R on the edges of E component a (tensor mode)."""
        nx, ny, nz = self.shape
        return self._view(self.lib.oracle_tensor_D(self.h, int(a))).reshape(nz, ny, nx).copy()

    def add_source(self, comp, lo, hi, wave):
        wave = np.ascontiguousarray(wave, dtype=np.float64)
        lp, _a = _i(lo)
        hp, _b = _i(hi)
        r = self.lib.oracle_add_source(self.h, int(comp), lp, hp, _d(wave), int(wave.size))
        assert r >= 0
        return r

    def add_dft_box(self, lo, hi, comps, omegas):
        """DFT monitor over the half-open box [lo, hi) of cells (Sec. 2.4)."""
        mask = 0
        for c in comps:
            mask |= 1 << int(c)
        om = np.ascontiguousarray(omegas, dtype=np.float64)
        lp, _a = _i(lo)
        hp, _b = _i(hi)
        r = self.lib.oracle_add_dft_box(self.h, lp, hp, mask, int(om.size), _d(om))
        assert r >= 0
        ncomp = bin(mask).count("1")
        ext = tuple(int(h) - int(l) for l, h in zip(lo, hi))
        self._mons.append((ncomp, om.size, ext[2], ext[1], ext[0]))
        return r

    def add_dft_plane(self, axis, index, comps, omegas):
        lo = [0, 0, 0]
        hi = list(self.shape)
        lo[axis], hi[axis] = int(index), int(index) + 1
        return self.add_dft_box(lo, hi, comps, omegas)

    def enable_energy(self, cap):
        self.lib.oracle_enable_energy(self.h, int(cap))
        self._ecap = int(cap)

    # -- stepping and access ----------------------------------------------------------
    def step(self, n=1):
        self.lib.oracle_step(self.h, int(n))

    def set_threads(self, n):
        """OpenMP team size of the forward step's cell loops (1 = serial, the default).  Every
        cell's arithmetic is the same for any team size, so results are identical bit for bit."""
        self.lib.oracle_set_threads(self.h, int(n))

    def step_backward(self, n=1):
        """Undoes n forward steps by stepping Eq. (yee) backward (lossless, nondispersive
        domains only: no CPML layers, no poles; Sec. 3.2 reversible reconstruction)."""
        r = self.lib.oracle_step_backward(self.h, int(n))
        if r != 0:
            raise ValueError("backward stepping needs a domain without CPML layers and without poles")

    def step_backward_interior(self, rec_e, rec_h):
        """Undoes the last forward step on the interior (cells whose own node lies in no CPML slab),
        the absorbing-face variant of the reversible reconstruction (Sec. 3.2): rec_e = (Ex, Ey, Ez)
        of E^{n+1} and rec_h = (Hx, Hy, Hz) of H^{n+1/2}, full-grid arrays recorded by the forward
        run, of which only the nodes outside the interior are read."""
        e = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in rec_e]
        h = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in rec_h]
        for a in e + h:
            assert a.size == self.n
        r = self.lib.oracle_step_backward_interior(self.h, *[_d(a) for a in e + h])
        if r != 0:
            raise ValueError("interior backward steps need a domain without poles and a step count >= 1")

    @property
    def step_count(self):
        return int(self.lib.oracle_step_count(self.h))

    def _view(self, ptr, n=None):
        n = self.n if n is None else n
        return np.ctypeslib.as_array(ptr, shape=(n,))

    def field(self, comp):
        nx, ny, nz = self.shape
        return self._view(self.lib.oracle_field(self.h, int(comp))).reshape(nz, ny, nx)

    def fields(self):
        return [self.field(c).copy() for c in range(6)]

    def psi(self, magnetic, comp, which):
        nx, ny, nz = self.shape
        return self._view(self.lib.oracle_psi(self.h, int(magnetic), int(comp), int(which))).reshape(nz, ny, nx)

    def pole_state(self, comp, pole, which):
        nx, ny, nz = self.shape
        return self._view(self.lib.oracle_pole(self.h, int(comp), int(pole), int(which))).reshape(nz, ny, nx)

    def dft(self, mon):
        """Complex spectra, shape (ncomp, nfreq, bz, by, bx)."""
        shp = self._mons[mon]
        raw = self._view(self.lib.oracle_dft(self.h, int(mon)), int(self.lib.oracle_dft_len(self.h, int(mon))))
        return (raw[0::2] + 1j * raw[1::2]).reshape(shp)

    def energy(self):
        return self._view(self.lib.oracle_energy(self.h), self._ecap)[: self.step_count].copy()

    def coef(self, magnetic, axis, which):
        n = self.shape[axis]
        return self._view(self.lib.oracle_coef(self.h, int(magnetic), int(axis), int(which)), n).copy()

    def pole_coef(self, p):
        M = np.zeros(4)
        g = np.zeros(2)
        self.lib.oracle_pole_coef(self.h, int(p), _d(M), _d(g))
        return M.reshape(2, 2), g

    # -- whole-state vectors -----------------------------------------------------------
    @property
    def state_len(self):
        return int(self.lib.oracle_state_len(self.h))

    def get_state(self, adjoint=False):
        buf = np.zeros(self.state_len)
        self.lib.oracle_state_get(self.h, _d(buf), int(adjoint))
        return buf

    def set_state(self, buf, adjoint=False, step=None):
        buf = np.ascontiguousarray(buf, dtype=np.float64)
        assert buf.size == self.state_len
        self.lib.oracle_state_set(self.h, _d(buf), int(adjoint))
        if step is not None:
            self.lib.oracle_set_step(self.h, int(step))

    def set_step(self, s):
        self.lib.oracle_set_step(self.h, int(s))

    def dft_reset(self):
        self.lib.oracle_dft_reset(self.h)

    # -- adjoint --------------------------------------------------------------------------
    def set_design(self, lo, hi):
        lp, _a = _i(lo)
        hp, _b = _i(hi)
        self.lib.oracle_set_design(self.h, lp, hp)
        self._design = (tuple(lo), tuple(hi))

    def grad(self, comp):
        """dJ/d eps^-1 over the design box: comp 0..2 the diagonal components of the cells; in
        tensor mode 0..5 the node components xx, yy, zz, xy, xz, yz (an off-diagonal one counts
        once, as one symmetric parameter)."""
        lo, hi = self._design
        n = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])
        return self._view(self.lib.oracle_grad(self.h, int(comp)), n).reshape(
            hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0]).copy()

    def set_adjoint_source(self, mon, cot):
        """cot: complex array shaped like dft(mon) = dJ/dRe F + i dJ/dIm F."""
        if cot is None:
            self.lib.oracle_set_adjoint_source(self.h, int(mon), None)
            return
        cot = np.asarray(cot, dtype=np.complex128).reshape(-1)
        raw = np.empty(2 * cot.size)
        raw[0::2] = cot.real
        raw[1::2] = cot.imag
        self.lib.oracle_set_adjoint_source(self.h, int(mon), _d(raw))

    def adj_reset(self):
        self.lib.oracle_adj_reset(self.h)

    def adj_field(self, comp):
        nx, ny, nz = self.shape
        return self._view(self.lib.oracle_adj_field(self.h, int(comp))).reshape(nz, ny, nx)

    def adjoint_step(self, m):
        """Adjoint of forward step m; the held forward state must be u^m."""
        self.lib.oracle_adjoint_step(self.h, int(m))

    def pole_grad(self):
        """d J / d(deps, omega_dt, gamma_dt) of each pole, (n_poles, 3), accumulated by the
        adjoint steps since adj_reset (Sec. 3.1: pole parameters through the transposed
        dispersion update)."""
        n = self.npole
        out = np.zeros(3 * max(n, 1))
        self.lib.oracle_pole_grad(self.h, _d(out))
        return out[: 3 * n].reshape(n, 3)

    def pole_coef_grad(self):
        """Cotangents of (M00, M01, M10, M11, g0, g1) of each pole, (n_poles, 6)."""
        n = self.npole
        out = np.zeros(6 * max(n, 1))
        self.lib.oracle_pole_coef_grad(self.h, _d(out))
        return out[: 6 * n].reshape(n, 6)


TENSOR_TOL = 1e-6


def tensor_rejected(t6, shape, cpml):
    """The admission rule of Sec. 2.3, node by node: eps^-1 (components xx, yy, zz, xy, xz, yz,
    shape (6, nz, ny, nx)) must be symmetric positive definite with every eigenvalue of eps at or
    above one (eigenvalues of eps^-1 in (0, 1], up to a relative TENSOR_TOL), and inside the CPML
    slab of an axis q (node coordinate < lo_q or >= N_q - hi_q; cpml = (xlo, xhi, ylo, yhi, zlo,
    zhi)) the face normal e_q must be a principal axis (the off-diagonal entries of row q are zero
    up to TENSOR_TOL times the largest diagonal entry) whose eigenvalue is not strictly between the
    other two.  Returns a boolean (nz, ny, nx) array, True where the node is rejected."""
    nx, ny, nz = shape
    t = np.asarray(t6, dtype=np.float64).reshape(6, nz, ny, nx)
    idx = [[0, 3, 4], [3, 1, 5], [4, 5, 2]]
    M = np.stack([np.stack([t[idx[a][b]] for b in range(3)], axis=-1) for a in range(3)], axis=-2)
    lam = np.linalg.eigvalsh(M)
    bad = (lam[..., 0] <= 0.0) | (lam[..., 2] > 1.0 + TENSOR_TOL)
    coords = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pos = [coords[2], coords[1], coords[0]]
    scale = np.max(np.abs(np.stack([t[0], t[1], t[2]])), axis=0)
    for q in range(3):
        lo, hi = cpml[2 * q], cpml[2 * q + 1]
        if lo == 0 and hi == 0:
            continue
        n = shape[q]
        inslab = (pos[q] < lo) | (pos[q] >= n - hi)
        b, c = (q + 1) % 3, (q + 2) % 3
        off = np.maximum(np.abs(M[..., q, b]), np.abs(M[..., q, c])) > TENSOR_TOL * scale
        sub = np.stack([np.stack([M[..., b, b], M[..., b, c]], -1), np.stack([M[..., c, b], M[..., c, c]], -1)], -2)
        mu = np.linalg.eigvalsh(sub)
        tol = TENSOR_TOL * (np.abs(mu[..., 0]) + np.abs(mu[..., 1]))
        inter = (M[..., q, q] - mu[..., 0] > tol) & (mu[..., 1] - M[..., q, q] > tol)
        bad |= inslab & (off | inter)
    return bad


def gradient_replay(orc: Oracle, n_steps: int, objective, segment: int = 0):
    """Run n_steps forward from the held state, evaluate objective(orc) -> (J, {mon: cot}),
    then sweep the adjoint back to step 0 with a two-level replay (checkpoint every
    `segment` steps, store every state of one segment at a time; Sec. 3.2).
    Returns J; the gradient is left in orc.grad(...).  The replays re-accumulate the
    DFT monitors, so read spectra inside `objective`, not afterwards."""
    seg = segment or max(1, int(np.ceil(np.sqrt(n_steps))))
    s0 = orc.step_count
    ckpt = {}
    for n in range(n_steps):
        if n % seg == 0:
            ckpt[n] = orc.get_state()
        orc.step(1)
    J, cots = objective(orc)
    for mon, cot in cots.items():
        orc.set_adjoint_source(mon, cot)
    orc.adj_reset()
    final_state = orc.get_state()
    starts = sorted(ckpt)
    for st in reversed(starts):
        end = min(st + seg, n_steps)
        orc.set_state(ckpt[st], step=s0 + st)
        states = []
        for n in range(st, end):
            states.append(orc.get_state())
            orc.step(1)
        for n in range(end - 1, st - 1, -1):
            orc.set_state(states[n - st], step=s0 + n)
            orc.adjoint_step(s0 + n)
    orc.set_state(final_state, step=s0 + n_steps)
    return J
