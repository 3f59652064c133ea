"""FP64 oracle of the Yee step with Bloch-periodic x / y faces (complex fields), and its transpose.

TEST INFRASTRUCTURE ONLY: nothing in the product path imports this module.

Sec. 2.2 pairs periodic faces with a fixed Bloch phase: a field continued across the seam of
axis q is multiplied by the phase p_q = exp(i k_q N_q), i.e. f(x + N_q) = p_q f(x).  So the fields
are complex.  The difference operators of Eq. (yee) then wrap as
  backward (E update): f(-1) = f(N - 1) / p,    forward (H update): f(N) = f(0) p.
The z faces are PEC (tangential E held at 0 on z = 0, nodes at z = N absent); no CPML, no poles.
Units and Yee positions are those of the main oracle (c = eps0 = mu0 = 1, h = 1, dt = S).

The transposed step (Sec. 3.1: Bloch boundaries are transposed with conjugate seam factors)
is the adjoint under <u, v> = sum conj(u) v.  The backward difference reads across its seam with
the factor 1/p; its adjoint is minus the forward difference, which reads across the seam with
p = conj(1/p) (|p| = 1), and vice versa.  Plain numpy, whole-array operations in the order of
Eq. (yee).
"""
import numpy as np


class BlochOracle:
    def __init__(self, shape, courant, kx=0.0, ky=0.0, inv_eps=None):
        """shape (nx, ny, nz); kx, ky: Bloch wavenumbers per cell (phase per period k N);
        inv_eps: None (vacuum), one (nz, ny, nx) array (isotropic) or three."""
        self.nx, self.ny, self.nz = (int(v) for v in shape)
        self.S = float(courant)
        self.px = np.exp(1j * kx * self.nx)
        self.py = np.exp(1j * ky * self.ny)
        shp = (self.nz, self.ny, self.nx)
        if inv_eps is None:
            ie = [np.ones(shp)] * 3
        elif isinstance(inv_eps, np.ndarray):
            ie = [inv_eps] * 3
        else:
            ie = list(inv_eps)
        self.ie = [np.asarray(a, dtype=np.float64) for a in ie]
        self.E = [np.zeros(shp, dtype=np.complex128) for _ in range(3)]
        self.H = [np.zeros(shp, dtype=np.complex128) for _ in range(3)]
        # PEC: tangential E on z = 0 (Ex, Ey)
        self.pec = [np.zeros(shp, dtype=bool) for _ in range(3)]
        self.pec[0][0] = True
        self.pec[1][0] = True

    # -- difference operators (axis 0 = x, 1 = y, 2 = z of the (z, y, x) arrays) ----------------
    def _back(self, f, axis):
        """f(r) - f(r - e_axis); across a Bloch seam f(-1) = f(N-1) / p; below z = 0: 0."""
        if axis == 2:
            g = np.zeros_like(f)
            g[1:] = f[:-1]
            return f - g
        ax = 2 - axis
        p = self.px if axis == 0 else self.py
        g = np.roll(f, 1, axis=ax)
        idx = [slice(None)] * 3
        idx[ax] = 0
        g[tuple(idx)] = g[tuple(idx)] / p
        return f - g

    def _fwd(self, f, axis):
        """f(r + e_axis) - f(r); across a Bloch seam f(N) = f(0) p; beyond z = N-1: 0."""
        if axis == 2:
            g = np.zeros_like(f)
            g[:-1] = f[1:]
            return g - f
        ax = 2 - axis
        p = self.px if axis == 0 else self.py
        g = np.roll(f, -1, axis=ax)
        idx = [slice(None)] * 3
        idx[ax] = -1
        g[tuple(idx)] = g[tuple(idx)] * p
        return g - f

    # adjoints under sum conj(u) v: (back)^H = -fwd and (fwd)^H = -back, with the same p (the
    # seam factor of the adjoint, p or 1/p, is the conjugate of the original's, 1/p or p)
    def _back_adj(self, f, axis):
        return -self._fwd(f, axis)

    def _fwd_adj(self, f, axis):
        return -self._back(f, axis)

    # -- Eq. (yee) ----------------------------------------------------------------------------
    def curl_H(self):
        """C^- H: backward differences (the E update's curl)."""
        d = self._back
        Hx, Hy, Hz = self.H
        return [d(Hz, 1) - d(Hy, 2), d(Hx, 2) - d(Hz, 0), d(Hy, 0) - d(Hx, 1)]

    def curl_E(self):
        """C^+ E: forward differences (the H update's curl)."""
        f = self._fwd
        Ex, Ey, Ez = self.E
        return [f(Ez, 1) - f(Ey, 2), f(Ex, 2) - f(Ez, 0), f(Ey, 0) - f(Ex, 1)]

    def step(self, n=1):
        for _ in range(n):
            c = self.curl_H()
            for a in range(3):
                self.E[a] = np.where(self.pec[a], 0.0, self.E[a] + self.S * self.ie[a] * c[a])
            c = self.curl_E()
            for a in range(3):
                self.H[a] = self.H[a] - self.S * c[a]

    def adjoint_step(self, n=1):
        """Transpose of `step` on (Ebar, Hbar) held in E, H: the H update first (reverse order)."""
        for _ in range(n):
            # H' = H - S C^+ E'  ->  Ebar' += -S (C^+)^H Hbar ; Hbar passes through
            Hx, Hy, Hz = self.H
            fa = self._fwd_adj
            # (C^+)^H Hbar, one E component at a time
            ct = [np.zeros_like(Hx) for _ in range(3)]
            # H_x row: f(Ez, y) - f(Ey, z); H_y row: f(Ex, z) - f(Ez, x); H_z row: f(Ey, x) - f(Ex, y)
            ct[2] += fa(Hx, 1)
            ct[1] -= fa(Hx, 2)
            ct[0] += fa(Hy, 2)
            ct[2] -= fa(Hy, 0)
            ct[1] += fa(Hz, 0)
            ct[0] -= fa(Hz, 1)
            Eb = [self.E[a] - self.S * ct[a] for a in range(3)]
            # E' = mask (E + S ie C^- H)  ->  with w = mask Eb: Ebar = w, Hbar += S (C^-)^H (ie w)
            w = [np.where(self.pec[a], 0.0, Eb[a]) for a in range(3)]
            v = [self.S * self.ie[a] * w[a] for a in range(3)]
            ba = self._back_adj
            ch = [np.zeros_like(Hx) for _ in range(3)]
            # E_x row: b(Hz, y) - b(Hy, z); E_y row: b(Hx, z) - b(Hz, x); E_z row: b(Hy, x) - b(Hx, y)
            ch[2] += ba(v[0], 1)
            ch[1] -= ba(v[0], 2)
            ch[0] += ba(v[1], 2)
            ch[2] -= ba(v[1], 0)
            ch[1] += ba(v[2], 0)
            ch[0] -= ba(v[2], 1)
            self.E = w
            self.H = [self.H[a] + ch[a] for a in range(3)]

    def electric_energy(self):
        """sum eps |E|^2 (the electric part of the discrete energy)."""
        return sum(float(np.sum(np.abs(self.E[a]) ** 2 / self.ie[a])) for a in range(3))

    def state(self):
        return np.concatenate([x.reshape(-1) for x in self.E + self.H])

    def set_state(self, v):
        n = self.nx * self.ny * self.nz
        shp = (self.nz, self.ny, self.nx)
        parts = [v[k * n:(k + 1) * n].reshape(shp).astype(np.complex128) for k in range(6)]
        self.E = parts[:3]
        self.H = parts[3:]
