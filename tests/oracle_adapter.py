"""Builds an FP64 oracle domain from a workload Scene (test-side glue only)."""
import numpy as np

from oracle.oracle import Oracle


def oracle_from_scene(sc, with_sources=True, with_monitors=True, periodic=None):
    if periodic is None:
        periodic = getattr(sc, "periodic", (0, 0, 0))
    o = Oracle(sc.shape, sc.courant, periodic=periodic, cpml=sc.cpml, m=sc.cpml_m,
               kappa_max=sc.kappa_max, alpha_max=sc.alpha_max, sigma_max=sc.sigma_max)
    o.set_material(sc.inv_eps3(), poles=sc.poles, mask=sc.pole_mask)
    if with_sources:
        for s in sc.sources:
            o.add_source(s.comp, s.lo, s.hi, s.wave)
    if with_monitors:
        for m in sc.monitors:
            o.add_dft_box(m.lo, m.hi, m.comps, m.omegas)
    if sc.design is not None:
        o.set_design(*sc.design)
    if sc.energy:
        o.enable_energy(sc.n_steps + 8)
    return o


def pec_mask_E(shape, periodic=(0, 0, 0)):
    """Boolean masks (nz,ny,nx) of PEC-held E nodes per component: E_a at coordinate 0 of a
    non-periodic axis q != a."""
    nx, ny, nz = shape
    masks = []
    for a in range(3):
        m = np.zeros((nz, ny, nx), dtype=bool)
        for q in range(3):
            if q == a or periodic[q]:
                continue
            sl = [slice(None)] * 3
            sl[2 - q] = 0
            m[tuple(sl)] = True
        masks.append(m)
    return masks
