"""Net Poynting flux through a z-plane from plane-monitor spectra (oracle side).

TEST INFRASTRUCTURE ONLY (imported by ``tests/`` like the rest of ``oracle/``).  Plain numpy,
written from the definition (Sec. 2.4: plane monitors form the signed Poynting flux from
Yee-interpolated spectra): for time-harmonic fields the mean flux along +z is
    P(w) = 1/2 Re sum_cells [ Ex(w) Hy(w)^* - Ey(w) Hx(w)^* ]
(reduced units: c = eps0 = mu0 = 1, cell area 1).  On the Yee lattice Hy(i+1/2, j, k+1/2) and
Hx(i, j+1/2, k+1/2) sit on the plane z = k + 1/2, halfway between the Ex (Ey) nodes of planes k
and k+1; averaging those two E planes puts each product at one point, with no interpolation in
x or y.  The spectra use each component's own sample times (E at t = n+1, H at t = n+3/2), so
the half-step between them is already in their phases.
"""
import numpy as np


def plane_flux_z(spec, comps):
    """spec: complex array (ncomp, nf, 2, by, bx) of a monitor box two z-planes thick (planes
    k and k+1) recording at least Ex, Ey, Hx, Hy; comps: the recorded component indices in
    order (0..5 = Ex..Hz).  Returns P(w) through z = k + 1/2, shape (nf,)."""
    comps = list(comps)
    if spec.shape[2] != 2:
        raise ValueError("the monitor must span exactly two z-planes")
    ex = spec[comps.index(0)]
    ey = spec[comps.index(1)]
    hx = spec[comps.index(3)]
    hy = spec[comps.index(4)]
    ex_mid = 0.5 * (ex[:, 0] + ex[:, 1])
    ey_mid = 0.5 * (ey[:, 0] + ey[:, 1])
    return 0.5 * np.real(np.sum(ex_mid * np.conj(hy[:, 0]) - ey_mid * np.conj(hx[:, 0]), axis=(1, 2)))


def slab_transmission(n, thickness, wavelength, courant=None):
    """Normal-incidence power transmission of a lossless slab of index n and the given
    thickness (cells) in vacuum: the two-interface (Fabry-Perot) closed form
        T = 1 / (1 + F sin^2(delta)),  F = 4 R / (1 - R)^2,  R = ((n - 1) / (n + 1))^2,
    with delta the one-way phase through the slab.  With courant given, delta uses the Yee
    lattice's own wavenumber in the slab, sin(k/2) = (n / S) sin(w / 2) with w = 2 pi S / lambda
    the phase advance per time step (Sec. 2.1: the dispersion relation of the Yee scheme), instead of the continuum
    n * 2 pi / lambda."""
    R = ((n - 1.0) / (n + 1.0)) ** 2
    F = 4.0 * R / (1.0 - R) ** 2
    if courant is None:
        k = n * 2.0 * np.pi / np.asarray(wavelength, dtype=float)
    else:
        w = 2.0 * np.pi * courant / np.asarray(wavelength, dtype=float)
        k = 2.0 * np.arcsin(n / courant * np.sin(w / 2.0))
    delta = k * thickness
    return 1.0 / (1.0 + F * np.sin(delta) ** 2)


def lattice_transmission(inv_eps_z, omega_dt, courant, reflection=False):
    """Exact power transmission (and, with reflection=True, reflection) of a layered medium on
    the 1-D Yee lattice at normal incidence,
    by a frequency-domain solve of the same difference equations (no time stepping).

    inv_eps_z[z]: eps^-1 at the E nodes z = 0 .. L-1 (vacuum on both sides beyond them);
    omega_dt: phase advance per time step.  With E^n = e_z exp(-i W n), H^(n+1/2) =
    h_(z+1/2) exp(-i W (n+1/2)) and s = sin(W/2) / S, the H and E updates of Eq. (yee) read
        2 i s h_(z+1/2) = e_(z+1) - e_z,       2 i s e_z = inv_eps_z (h_(z+1/2) - h_(z-1/2)).
    Starting from a unit transmitted wave e_z = exp(i k0 z) beyond the layers (sin(k0/2) = s),
    the two relations are marched to the incident side, where e = A exp(i k0 z) +
    B exp(-i k0 z) is split into its incident part A and reflected part B; T = 1 / |A|^2 and
    R = |B / A|^2."""
    ie = np.asarray(inv_eps_z, dtype=float)
    L = ie.size
    out, refl = [], []
    for W in np.atleast_1d(omega_dt):
        s = np.sin(W / 2.0) / courant
        k0 = 2.0 * np.arcsin(s)
        # transmitted side: nodes z >= L are vacuum; e_L, h_(L-1/2) from the outgoing wave
        e_next = np.exp(1j * k0 * L)                       # e_(z+1) with z = L-1
        h = np.exp(1j * k0 * (L - 0.5))                    # h_(L-1/2) (vacuum impedance 1)
        e_nodes = {}
        for z in range(L - 1, -3, -1):                     # march to two vacuum nodes z = -1, -2
            e_z = e_next - 2j * s * h                      # from the H relation at z + 1/2
            iez = ie[z] if 0 <= z < L else 1.0
            h = h - 2j * s * e_z / iez                     # h_(z-1/2) from the E relation at z
            e_nodes[z] = e_z
            e_next = e_z
        e1, e2 = e_nodes[-1], e_nodes[-2]
        # e_z = A exp(i k0 z) + B exp(-i k0 z) at z = -1, -2
        M = np.array([[np.exp(-1j * k0), np.exp(1j * k0)], [np.exp(-2j * k0), np.exp(2j * k0)]])
        A, B = np.linalg.solve(M, np.array([e1, e2]))
        out.append(1.0 / abs(A) ** 2)
        refl.append(abs(B / A) ** 2)
    if reflection:
        return np.array(out), np.array(refl)
    return np.array(out)
