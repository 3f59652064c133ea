"""Builds an FP64 oracle domain from a workload Scene (test-side glue only)."""
import numpy as np

from oracle.oracle import Oracle


def oracle_from_scene(sc, with_sources=True, with_monitors=True, periodic=None):
    if periodic is None:
        periodic = getattr(sc, "periodic", (0, 0, 0))
    o = Oracle(sc.shape, sc.courant, periodic=periodic, cpml=sc.cpml, m=sc.cpml_m,
               kappa_max=sc.kappa_max, alpha_max=sc.alpha_max, sigma_max=sc.sigma_max)
    o.set_material(sc.inv_eps3(), poles=sc.poles, mask=sc.pole_mask)
    if getattr(sc, "tensor", None) is not None:
        o.set_tensor(sc.tensor)
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


def oracle_spectra(sc, threads=1):
    """Runs a Scene's whole forward solve in the oracle and returns the spectra of its monitors
    (a list, in the scene's monitor order).  Module-level so a spawn process pool can call it."""
    o = oracle_from_scene(sc)
    o.set_threads(threads)
    o.step(sc.n_steps)
    return [o.dft(k).copy() for k in range(len(sc.monitors))]


def oracle_spectra_many(scenes, processes=None):
    """oracle_spectra of many independent scenes, one single-threaded oracle per worker of a
    spawn pool (safe after CUDA was initialised in this process)."""
    import multiprocessing as mp
    import os
    procs = processes or max(1, min(len(scenes), os.cpu_count() or 1))
    if procs == 1:
        return [oracle_spectra(sc) for sc in scenes]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(oracle_spectra, scenes, chunksize=1)
