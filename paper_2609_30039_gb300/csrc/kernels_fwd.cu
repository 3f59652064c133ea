// Forward half-steps of the Yee leapfrog (arxiv 2609.30039, Sec. 2.1 Eq. (yee)) with the CPML
// memories of Sec. 2.2, the trapezoidal Drude/Lorentz update and diagonal eps^-1 of Sec. 2.3,
// soft sources and running DFT monitors of Sec. 2.4.
//
// Work decomposition: a tile is 32 x 8 columns of one domain; each thread owns a column (i, j)
// and marches k over the tile's z range, so consecutive planes of the same column stay in L1
// and every warp reads 32 consecutive floats (128 B) of each array.  Soft sources, the FP64
// DFT accumulation and the device step counter are fused into the two field kernels (per-tile
// flags mark the tiles that hold source or monitor cells), so a forward step is two kernels per
// tile class and a CUDA graph of them replays without host work.
#include "fdtd_internal.cuh"

namespace gbfdtd {

// Fused multiply-add with one rounding, spelled out where several kernels must agree bit for bit.
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }

// CPML coefficients of one node along one axis: y = D/kappa + psi, psi <- b psi + c D.
template <typename T>
struct Cpml1 {
    int s;        // slab index, -1 outside the slabs
    T b, c, k;
};

template <typename T>
__device__ __forceinline__ Cpml1<T> cpml_at(const Dom<T>& d, const T* coef, int q, int x) {
    Cpml1<T> r;
    r.s = d.ns[q] ? slab_of(x, d.dlo[q], d.dhi[q], d.n[q]) : -1;
    r.b = T(1);
    r.c = T(0);
    r.k = T(1);
    if (r.s >= 0) {
        const int N = d.n[q];
        r.b = coef[x];
        r.c = coef[N + x];
        r.k = coef[2 * N + x];
    }
    return r;
}

// In-slab CPML correction of one derivative: psi <- b psi + c D first, then y = D/kappa + psi
// (c D rounded, then two fused multiply-adds).

template <typename T>
__device__ __forceinline__ T cpml_rec(T b, T c, T kinv, T* psi, T D) {
    const T cd = c * D;
    const T ps = fma_t(b, *psi, cd);
    *psi = ps;
    return fma_t(kinv, D, ps);
}

template <typename T>
__device__ __forceinline__ T cpml_apply(const Cpml1<T>& q, T* psi, T D) {
    return cpml_rec(q.b, q.c, q.k, psi, D);
}

// Trapezoidal pole update of one E component (Sec. 2.3):
// (eps_inf + G) E^{n+1} = (eps_inf + G) E^n + Delta,
// Delta = S curl + sum_p (P_p - (M_p x_p)_P - 2 g_p E^n);  x_p <- M_p x_p + g_p (E^{n+1} + E^n).
// (Multiply-adds are written as explicit fused operations so every kernel rounds alike.)
template <typename T>
__device__ __forceinline__ T ade_update(const Dom<T>& d, int a, long long bo, T e0, T ie, T scurl) {
    T delta = scurl;
    T* base = d.ade + (long long)a * d.npole * 2 * d.bcell + bo;
    for (int p = 0; p < d.npole; ++p) {
        const T P = base[(2 * p) * d.bcell], Q = base[(2 * p + 1) * d.bcell];
        const T mp = fma_t(d.M00[p], P, d.M01[p] * Q);
        delta = delta + fma_t(-T(2) * d.g0[p], e0, P - mp);
    }
    const T e1 = fma_t(ie / fma_t(ie, d.G, T(1)), delta, e0);
    const T es = e1 + e0;
    for (int p = 0; p < d.npole; ++p) {
        T* pp = base + (2 * p) * d.bcell;
        T* pq = base + (2 * p + 1) * d.bcell;
        const T P = *pp, Q = *pq;
        *pp = fma_t(d.g0[p], es, fma_t(d.M00[p], P, d.M01[p] * Q));
        *pq = fma_t(d.g1[p], es, fma_t(d.M10[p], P, d.M11[p] * Q));
    }
    return e1;
}

template <typename T>
__device__ __forceinline__ T src_add(const Dom<T>& d, const Src* __restrict__ srcs, int comp, int i, int j, int k,
                                     int step) {
    return src_add_t<T>(d, srcs, comp, i, j, k, step);
}

// Running DFT (Sec. 2.4), F += f exp(i w t) accumulated in FP64, of one work item: up to 256
// consecutive cells of one monitor (one per thread), for the recorded components of one kind
// (0: E at t = n+1, 1: H at t = n+3/2).  It runs beside the field updates, never on their
// critical path: the E part of step n while H is updated, the H part while E of step n+1 is (each
// only reads the field the other half-step leaves alone).  A cell's accumulators are updated in
// batches of four, loads before stores, one memory round trip per batch.
template <typename T>
__device__ __forceinline__ void dft_item(const Dom<T>* __restrict__ doms, const Mon* __restrict__ mons,
                                         const DftItem& it, int kind, int step) {
    const Mon& m = mons[it.mon];
    const long long cell = it.begin + threadIdx.y * kTileX + threadIdx.x;
    if (cell >= it.end) return;
    const int i = m.lo[0] + (int)(cell % m.bx);
    const int j = m.lo[1] + (int)((cell / m.bx) % m.by);
    const int k = m.lo[2] + (int)(cell / ((long long)m.bx * m.by)) - it.kz0;
    const Dom<T>& d = doms[it.dom];
    const long long id = cidx(d.n, i, j, k);
    const double2* ph = m.phase + ((long long)step * 2 + kind) * m.nf;
    const int nf = m.nf;
    int ci = 0;
    for (int c = 0; c < 6; ++c) {
        if (!((m.mask >> c) & 1u)) continue;
        if (c / 3 == kind) {
            const double v = (double)d.F[c][id];
            double2* acc = m.acc + (long long)ci * nf * m.ncell + cell;
            for (int f0 = 0; f0 < nf; f0 += 4) {
                double2 x[4], p[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int f = f0 + q < nf ? f0 + q : f0;
                    x[q] = acc[(long long)f * m.ncell];
                    p[q] = ph[f];
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (f0 + q >= nf) break;
                    x[q].x = fma_t(v, p[q].x, x[q].x);
                    x[q].y = fma_t(v, p[q].y, x[q].y);
                    acc[(long long)(f0 + q) * m.ncell] = x[q];
                }
            }
        }
        ++ci;
    }
}

// Per-half-step DFT launch: one block per work item; the step is *d_base + offset (the first
// step of the launched batch plus this launch's position in it, so a captured graph replays).
template <typename T>
__global__ void __launch_bounds__(kTileX* kTileY)
    k_dft(const Dom<T>* __restrict__ doms, const Mon* __restrict__ mons, const DftItem* __restrict__ items, int kind,
          const int* __restrict__ d_base, int offset) {
    dft_item(doms, mons, items[blockIdx.x], kind, *d_base + offset);
}

// DFT of a batch of cnt steps from the monitor rings (per-cell mode): block (x, y) takes work item
// x for the monitor's y-th component (one thread per monitor cell), so the FP64 work of a batch
// spreads over items x components blocks; each accumulator takes the samples of steps base,
// base + 1, ... in order with the fused multiply-adds of dft_item, so it ends bit for bit where cnt
// per-step launches of each kind would leave it, with one accumulator load and store per batch
// instead of per step.
template <typename T>
__global__ void __launch_bounds__(kTileX* kTileY)
    k_dft_ring(const Mon* __restrict__ mons, const DftItem* __restrict__ items, const int* __restrict__ d_base,
               int cnt) {
    const DftItem& it = items[blockIdx.x];
    const Mon& m = mons[it.mon];
    const int ci = blockIdx.y;
    const long long cell = it.begin + threadIdx.y * kTileX + threadIdx.x;
    if (ci >= m.ncomp || cell >= it.end) return;
    const int base = *d_base, nf = m.nf;
    const long long slot = (long long)m.ncomp * m.ncell;
    {
        const int kind = m.comps[ci] >= 3 ? 1 : 0;
        const T* r = (const T*)m.ring + (long long)ci * m.ncell + cell;
        double2* acc = m.acc + (long long)ci * nf * m.ncell + cell;
        for (int f0 = 0; f0 < nf; f0 += 4) {
            double2 x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = acc[(long long)(f0 + q < nf ? f0 + q : f0) * m.ncell];
            for (int t = 0; t < cnt; ++t) {
                const double v = (double)r[t * slot];
                const double2* ph = m.phase + ((long long)(base + t) * 2 + kind) * nf + f0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (f0 + q >= nf) break;
                    const double2 p = ph[q];
                    x[q].x = fma_t(v, p.x, x[q].x);
                    x[q].y = fma_t(v, p.y, x[q].y);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (f0 + q >= nf) break;
                acc[(long long)(f0 + q) * m.ncell] = x[q];
            }
        }
    }
}

// Monitor samples: plane kg (global; block-uniform in the per-cell kernels) crosses the domain's
// monitor box and the step stores samples, then cell (i, j) lies in the box; the sample of a
// component goes to slot a.offset of its ring at sample_off.
template <typename T>
__device__ __forceinline__ bool in_sample_plane(const CellArgs<T>& c, const StepArgs& a, int kg) {
    return (unsigned)(kg - c.slo[2]) < (unsigned)(c.shi[2] - c.slo[2]) && a.ring;
}
template <typename T>
__device__ __forceinline__ bool in_sample_rect(const CellArgs<T>& c, int i, int j) {
    return (unsigned)(i - c.slo[0]) < (unsigned)(c.shi[0] - c.slo[0]) &&
           (unsigned)(j - c.slo[1]) < (unsigned)(c.shi[1] - c.slo[1]);
}
template <typename T>
__device__ __forceinline__ long long sample_off(const CellArgs<T>& c, const StepArgs& a, int i, int j, int kg) {
    return (long long)a.offset * c.sstride +
           ((long long)(kg - c.slo[2]) * (c.shi[1] - c.slo[1]) + (j - c.slo[1])) * (c.shi[0] - c.slo[0]) +
           (i - c.slo[0]);
}

__global__ void k_copy_int(const int* __restrict__ src, int* __restrict__ dst) { *dst = *src; }

__global__ void k_set_int(int* __restrict__ dst, int v) { *dst = v; }

// Blocks per SM the per-launch kernels are compiled for.  Interior tiles run the plain register
// path at full occupancy (8 blocks of 256 threads in FP32, at most 32 registers): the warps in
// flight are what keeps enough loads outstanding to approach the DRAM bandwidth.
#ifndef GBFDTD_INT_BLOCKS_F32
#define GBFDTD_INT_BLOCKS_F32 8
#endif
template <typename T>
constexpr int min_blocks(bool general) {
    return general ? (sizeof(T) == 4 ? 4 : 2) : (sizeof(T) == 4 ? GBFDTD_INT_BLOCKS_F32 : 4);
}

// E half-step (Eq. (yee) first half) of a tile.  kGen = false: the tile touches no CPML slab,
// PEC plane, domain edge or dispersive cell, so none of that code is compiled in.  Every load of
// a plane is issued before any store of it; H_x, H_y of plane k-1 stay in registers.
template <typename T, bool kGen, bool kAniso>
__device__ __forceinline__ void tile_e(const Dom<T>* __restrict__ doms, const Tile& t, T S, const StepArgs& a,
                                       int step) {
    const Dom<T>& d = doms[t.dom];
    const int nx = d.n[0], ny = d.n[1];
    int i, j;
    tile_coords(t, i, j);
    if (i < 0 || j < 0) return;
    const bool fsrc = t.flags & kTileSrcE;
    const long long nxy = (long long)nx * ny;
    T* Ex = d.F[0];
    T* Ey = d.F[1];
    T* Ez = d.F[2];
    const T* Hx = d.F[3];
    const T* Hy = d.F[4];
    const T* Hz = d.F[5];
    const T* ie0 = d.ie[0];
    const T* ie1 = d.ie[1];
    const T* ie2 = d.ie[2];
    Cpml1<T> cx, cy;
    bool pi = false, pj = false;              // PEC plane at this column's x / y
    bool hasx = true, hasy = true;            // the -x / -y neighbour exists (wraps if periodic)
    long long oxm = -1, oym = -(long long)nx;
    if (kGen) {
        cx = cpml_at(d, d.cE[0], 0, i);
        cy = cpml_at(d, d.cE[1], 1, j);
        pi = i == 0 && !d.per[0];
        pj = j == 0 && !d.per[1];
        oxm = nb_minus(i, nx, 1, d.per[0], &hasx);
        oym = nb_minus(j, ny, nx, d.per[1], &hasy);
    }
    long long id = (long long)t.z0 * nxy + (long long)j * nx + i;
    T hxz = T(0), hyz = T(0);
    if (!kGen || t.z0 > 0) {
        hxz = Hx[id - nxy];
        hyz = Hy[id - nxy];
    }
    for (int k = t.z0; k < t.z1; ++k, id += nxy) {
        const T hx = Hx[id], hy = Hy[id], hz = Hz[id];
        const T hz_ym = (!kGen || hasy) ? Hz[id + oym] : T(0);
        const T hx_ym = (!kGen || hasy) ? Hx[id + oym] : T(0);
        const T hz_xm = (!kGen || hasx) ? Hz[id + oxm] : T(0);
        const T hy_xm = (!kGen || hasx) ? Hy[id + oxm] : T(0);
        T ex = Ex[id], ey = Ey[id], ez = Ez[id];
        const T iex = ie0[id];
        const T iey = kAniso ? ie1[id] : iex;
        const T iez = kAniso ? ie2[id] : iex;
        T yx1 = hz - hz_ym, yx2 = hy - hyz;  // Ex: dHz/dy, dHy/dz
        T yy1 = hx - hxz, yy2 = hz - hz_xm;  // Ey: dHx/dz, dHz/dx
        T yz1 = hy - hy_xm, yz2 = hx - hx_ym;  // Ez: dHy/dx, dHx/dy
        hxz = hx;
        hyz = hy;
        if (kGen) {
            const bool pk = k == 0;
            const bool px = pj || pk, py = pi || pk, pz = pi || pj;  // PEC-held components
            const Cpml1<T> cz = cpml_at(d, d.cE[2], 2, k);
            if (cz.s >= 0) {
                const long long o = ((long long)cz.s * ny + j) * nx + i;
                if (!px) yx2 = cpml_apply(cz, d.psiE[0][1] + o, yx2);
                if (!py) yy1 = cpml_apply(cz, d.psiE[1][0] + o, yy1);
            }
            if (cx.s >= 0) {
                const long long o = ((long long)k * ny + j) * d.ns[0] + cx.s;
                if (!py) yy2 = cpml_apply(cx, d.psiE[1][1] + o, yy2);
                if (!pz) yz1 = cpml_apply(cx, d.psiE[2][0] + o, yz1);
            }
            if (cy.s >= 0) {
                const long long o = ((long long)k * d.ns[1] + cy.s) * nx + i;
                if (!px) yx1 = cpml_apply(cy, d.psiE[0][0] + o, yx1);
                if (!pz) yz2 = cpml_apply(cy, d.psiE[2][1] + o, yz2);
            }
            const bool disp = d.npole > 0 && i >= d.blo[0] && i < d.bhi[0] && j >= d.blo[1] && j < d.bhi[1] &&
                              k >= d.blo[2] && k < d.bhi[2] && d.mask[id];
            if (disp) {
                const long long bo = ade_off(d, i, j, k);
                if (!px) ex = ade_update(d, 0, bo, ex, iex, S * (yx1 - yx2));
                if (!py) ey = ade_update(d, 1, bo, ey, iey, S * (yy1 - yy2));
                if (!pz) ez = ade_update(d, 2, bo, ez, iez, S * (yz1 - yz2));
            } else {
                if (!px) ex = fma_t(S * iex, (yx1 - yx2), ex);
                if (!py) ey = fma_t(S * iey, (yy1 - yy2), ey);
                if (!pz) ez = fma_t(S * iez, (yz1 - yz2), ez);
            }
            // a PEC-held component keeps its (zero) value and receives no source
        } else {
            ex = fma_t(S * iex, (yx1 - yx2), ex);
            ey = fma_t(S * iey, (yy1 - yy2), ey);
            ez = fma_t(S * iez, (yz1 - yz2), ez);
        }
        if (fsrc) {
            ex += src_add(d, a.srcs, 0, i, j, k, step);
            ey += src_add(d, a.srcs, 1, i, j, k, step);
            ez += src_add(d, a.srcs, 2, i, j, k, step);
        }
        if (kGen) {
            const bool pk = k == 0;
            if (!(pj || pk)) Ex[id] = ex;
            if (!(pi || pk)) Ey[id] = ey;
            if (!(pi || pj)) Ez[id] = ez;
        } else {
            Ex[id] = ex;
            Ey[id] = ey;
            Ez[id] = ez;
        }
    }
}

template <typename T, bool kGen, bool kAniso>
__global__ void __launch_bounds__(kTileX* kTileY, min_blocks<T>(kGen))
    k_e_update(const Dom<T>* __restrict__ doms, const Tile* __restrict__ tiles, T S, const StepArgs a) {
    tile_e<T, kGen, kAniso>(doms, tiles[blockIdx.x], S, a, *a.d_step);
}

// H half-step (Eq. (yee) second half) of a tile; E_x, E_y of plane k+1 are carried to the next
// plane in registers.  kEnergy adds W_{n+1} = 1/2 sum eps |E|^2 + 1/2 sum H^{n+1/2} H^{n+3/2}.
template <typename T, bool kGen, bool kEnergy>
__device__ __forceinline__ void tile_h(const Dom<T>* __restrict__ doms, const Tile& t, T S, const StepArgs& a,
                                       int step) {
    const Dom<T>& d = doms[t.dom];
    const int nx = d.n[0], ny = d.n[1], nz = d.n[2];
    int i, j;
    tile_coords(t, i, j);
    const bool fsrc = t.flags & kTileSrcH;
    double w = 0.0;
    if (i >= 0 && j >= 0) {
        const long long nxy = (long long)nx * ny;
        const T* Ex = d.F[0];
        const T* Ey = d.F[1];
        const T* Ez = d.F[2];
        T* Hx = d.F[3];
        T* Hy = d.F[4];
        T* Hz = d.F[5];
        Cpml1<T> cx, cy;
        bool xe = true, ye = true;  // the +x / +y neighbour node exists (wraps if periodic)
        long long oxp = 1, oyp = nx;
        if (kGen) {
            cx = cpml_at(d, d.cH[0], 0, i);
            cy = cpml_at(d, d.cH[1], 1, j);
            oxp = nb_plus(i, nx, 1, d.per[0], &xe);
            oyp = nb_plus(j, ny, nx, d.per[1], &ye);
        }
        long long id = (long long)t.z0 * nxy + (long long)j * nx + i;
        T exk = Ex[id], eyk = Ey[id];
        for (int k = t.z0; k < t.z1; ++k, id += nxy) {
            const bool ze = !kGen || k + 1 < nz;
            const T exn = ze ? Ex[id + nxy] : T(0);
            const T eyn = ze ? Ey[id + nxy] : T(0);
            const T ez = Ez[id];
            const T ez_yp = ye ? Ez[id + oyp] : T(0);
            const T ez_xp = xe ? Ez[id + oxp] : T(0);
            const T ey_xp = xe ? Ey[id + oxp] : T(0);
            const T ex_yp = ye ? Ex[id + oyp] : T(0);
            const T hx = Hx[id], hy = Hy[id], hz = Hz[id];
            T yx1 = ez_yp - ez, yx2 = eyn - eyk;  // Hx: dEz/dy, dEy/dz
            T yy1 = exn - exk, yy2 = ez_xp - ez;  // Hy: dEx/dz, dEz/dx
            T yz1 = ey_xp - eyk, yz2 = ex_yp - exk;  // Hz: dEy/dx, dEx/dy
            if (kGen) {
                const Cpml1<T> cz = cpml_at(d, d.cH[2], 2, k);
                if (cz.s >= 0) {
                    const long long o = ((long long)cz.s * ny + j) * nx + i;
                    yx2 = cpml_apply(cz, d.psiH[0][1] + o, yx2);
                    yy1 = cpml_apply(cz, d.psiH[1][0] + o, yy1);
                }
                if (cx.s >= 0) {
                    const long long o = ((long long)k * ny + j) * d.ns[0] + cx.s;
                    yy2 = cpml_apply(cx, d.psiH[1][1] + o, yy2);
                    yz1 = cpml_apply(cx, d.psiH[2][0] + o, yz1);
                }
                if (cy.s >= 0) {
                    const long long o = ((long long)k * d.ns[1] + cy.s) * nx + i;
                    yx1 = cpml_apply(cy, d.psiH[0][0] + o, yx1);
                    yz2 = cpml_apply(cy, d.psiH[2][1] + o, yz2);
                }
            }
            T hx1 = fma_t(-S, (yx1 - yx2), hx);
            T hy1 = fma_t(-S, (yy1 - yy2), hy);
            T hz1 = fma_t(-S, (yz1 - yz2), hz);
            if (fsrc) {
                hx1 += src_add(d, a.srcs, 3, i, j, k, step);
                hy1 += src_add(d, a.srcs, 4, i, j, k, step);
                hz1 += src_add(d, a.srcs, 5, i, j, k, step);
            }
            Hx[id] = hx1;
            Hy[id] = hy1;
            Hz[id] = hz1;
            if (kEnergy) {
                w += 0.5 * ((double)hx * hx1 + (double)hy * hy1 + (double)hz * hz1);
                w += 0.5 * ((double)exk * exk / (double)d.ie[0][id] + (double)eyk * eyk / (double)d.ie[1][id] +
                            (double)ez * ez / (double)d.ie[2][id]);
            }
            exk = exn;
            eyk = eyn;
        }
    }
    if (kEnergy) {
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if ((threadIdx.x & 31) == 0 && d.energy && step < d.energy_cap) atomicAdd(d.energy + step, w);
    }
}

template <typename T, bool kGen, bool kEnergy>
__global__ void __launch_bounds__(kTileX* kTileY, min_blocks<T>(kGen))
    k_h_update(const Dom<T>* __restrict__ doms, const Tile* __restrict__ tiles, T S, const StepArgs a,
               unsigned advance_blocks) {
    const int step = *a.d_step;
    tile_h<T, kGen, kEnergy>(doms, tiles[blockIdx.x], S, a, step);
    if (advance_blocks) {
        // the H launches of a step (general and interior, possibly running concurrently) hold
        // advance_blocks blocks together; the last of them to finish advances the device step
        // counter (every block has read it)
        __syncthreads();
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            __threadfence();
            const unsigned done = atomicAdd(a.d_ticket, 1u);
            if (done == advance_blocks - 1) {
                *a.d_ticket = 0u;
                *a.d_step = step + 1;
                __threadfence();
            }
        }
    }
}

// ---- per-cell streaming kernels -------------------------------------------------------------
// One thread per cell, every cell of a domain in one launch (grid: x chunks, y chunks, z planes,
// so no index division): no z-march, no tile classes.  All loads of a thread are independent
// (the z-1 / z+1 neighbour comes from L2 instead of a carried register) and the domain's
// pointers arrive as a kernel parameter, so the first loads issue at once; with 32 registers and
// full occupancy the SMs keep many loads in flight.  CPML, PEC and pole work is decided per cell
// (warps diverge only where a slab edge or a pole boundary crosses them).  Arithmetic per cell is
// the same as in tile_e / tile_h.
#ifndef GBFDTD_CELL_BLOCKS_F32
#define GBFDTD_CELL_BLOCKS_F32 8
#endif
// FP32: full occupancy (32 registers) except with poles (their update needs more registers)
template <typename T, bool kPoles = false>
constexpr int cell_blocks() {
    return sizeof(T) == 4 ? (kPoles ? 6 : GBFDTD_CELL_BLOCKS_F32) : 4;
}

template <typename T>
__device__ __forceinline__ T cpml_cell(const T* coef, int N, int x, T* psi, T D) {
    return cpml_rec(coef[x], coef[N + x], coef[2 * N + x], psi, D);
}

// kBack: the backward step of the reversible reconstruction (Sec. 3.2) for a lossless domain,
// E^n = (E^{n+1} - s^n) - S eps^-1 curl H^{n+1/2}, called with S negated (no CPML, no poles).
// kCurl: the first half of a tensor domain's E update (Sec. 2.3): the CPML-corrected curl of every
// non-PEC edge into c.cur (the memories advance as usual); launch_tensor_apply then applies S_t.
template <typename T, bool kAniso, bool kPoles, bool kPer, bool kBack, bool kCurl>
__device__ __forceinline__ void e_cell_body(const CellArgs<T>& c, const Dom<T>* __restrict__ doms, T S,
                                            const StepArgs& a, int i, int j, int k) {
    const int nx = c.n[0], ny = c.n[1];
    const int kg = k + c.kz0;   // global plane (CPML z profile, sources)
    if (i >= nx || j >= ny) return;
    const long long nxy = (long long)nx * ny;
    const long long id = ((long long)k * ny + j) * nx + i;
    // -1 neighbours (wrapping on a periodic axis); a PEC plane holds tangential E at coordinate 0
    bool hx_, hy_, hz_;
    const long long ox = nb_minus(i, nx, 1, kPer && c.per[0], &hx_);
    const long long oy = nb_minus(j, ny, nx, kPer && c.per[1], &hy_);
    const long long oz = nb_minus(k, c.n[2], nxy, 0, &hz_);
    const T* Hx = c.F[3];
    const T* Hy = c.F[4];
    const T* Hz = c.F[5];
    const T hx = Hx[id], hy = Hy[id], hz = Hz[id];
    T yx1 = hz - (hy_ ? Hz[id + oy] : T(0)), yx2 = hy - (hz_ ? Hy[id + oz] : T(0));  // Ex: dHz/dy, dHy/dz
    T yy1 = hx - (hz_ ? Hx[id + oz] : T(0)), yy2 = hz - (hx_ ? Hz[id + ox] : T(0));  // Ey: dHx/dz, dHz/dx
    T yz1 = hy - (hx_ ? Hy[id + ox] : T(0)), yz2 = hx - (hy_ ? Hx[id + oy] : T(0));  // Ez: dHy/dx, dHx/dy
    T ex = c.F[0][id], ey = c.F[1][id], ez = c.F[2][id];
    const T iex = c.ie[0][id];
    const T iey = kAniso ? c.ie[1][id] : iex;
    const T iez = kAniso ? c.ie[2][id] : iex;
    const bool pi = i == 0 && !(kPer && c.per[0]), pj = j == 0 && !(kPer && c.per[1]), pk = k == 0;
    const bool px = pj || pk, py = pi || pk, pz = pi || pj;   // PEC-held
    if (kBack) {
        if (i < c.alo[0] || i >= c.ahi[0] || j < c.alo[1] || j >= c.ahi[1] || k < c.alo[2] || k >= c.ahi[2]) return;
        T sx = T(0), sy = T(0), sz = T(0);
        if (i >= c.src_lo[0] && i < c.src_hi[0] && j >= c.src_lo[1] && j < c.src_hi[1] && kg >= c.src_lo[2] &&
            kg < c.src_hi[2]) {
            const int step = *a.d_base + a.offset;
            sx = src_add_t<T>(c, a.srcs, 0, i, j, kg, step);
            sy = src_add_t<T>(c, a.srcs, 1, i, j, kg, step);
            sz = src_add_t<T>(c, a.srcs, 2, i, j, kg, step);
        }
        if (!px) c.F[0][id] = fma_t(S * iex, (yx1 - yx2), ex - sx);
        if (!py) c.F[1][id] = fma_t(S * iey, (yy1 - yy2), ey - sy);
        if (!pz) c.F[2][id] = fma_t(S * iez, (yz1 - yz2), ez - sz);
        return;
    }
    // in-slab CPML corrections (the coefficients are read per derivative: loading them once per axis
    // measured slower here, unlike in k_h_cell)
    if (c.ns[2]) {
        const int sl = slab_of(kg, c.dlo[2], c.dhi[2], c.nzg);
        if (sl >= 0) {
            const long long o = ((long long)sl * ny + j) * nx + i;
            if (!px) yx2 = cpml_cell(c.coef[2], c.nzg, kg, c.psi[0][1] + o, yx2);
            if (!py) yy1 = cpml_cell(c.coef[2], c.nzg, kg, c.psi[1][0] + o, yy1);
        }
    }
    if (c.ns[0]) {
        const int sl = slab_of(i, c.dlo[0], c.dhi[0], nx);
        if (sl >= 0) {
            const long long o = ((long long)k * ny + j) * c.ns[0] + sl;
            if (!py) yy2 = cpml_cell(c.coef[0], nx, i, c.psi[1][1] + o, yy2);
            if (!pz) yz1 = cpml_cell(c.coef[0], nx, i, c.psi[2][0] + o, yz1);
        }
    }
    if (c.ns[1]) {
        const int sl = slab_of(j, c.dlo[1], c.dhi[1], ny);
        if (sl >= 0) {
            const long long o = ((long long)k * c.ns[1] + sl) * nx + i;
            if (!px) yx1 = cpml_cell(c.coef[1], ny, j, c.psi[0][0] + o, yx1);
            if (!pz) yz2 = cpml_cell(c.coef[1], ny, j, c.psi[2][1] + o, yz2);
        }
    }
    if (kCurl) {
        if (!px) c.cur[0][id] = yx1 - yx2;
        if (!py) c.cur[1][id] = yy1 - yy2;
        if (!pz) c.cur[2][id] = yz1 - yz2;
        return;
    }
    bool disp = false;
    if (kPoles) {
        const Dom<T>& d = doms[c.dom];
        disp = d.npole > 0 && in_ade_box(d, i, j, k) && d.mask[id];
        if (disp) {
            const long long bo = ade_off(d, i, j, k);
            if (!px) ex = ade_update(d, 0, bo, ex, iex, S * (yx1 - yx2));
            if (!py) ey = ade_update(d, 1, bo, ey, iey, S * (yy1 - yy2));
            if (!pz) ez = ade_update(d, 2, bo, ez, iez, S * (yz1 - yz2));
        }
    }
    if (!disp) {
        if (!px) ex = fma_t(S * iex, (yx1 - yx2), ex);
        if (!py) ey = fma_t(S * iey, (yy1 - yy2), ey);
        if (!pz) ez = fma_t(S * iez, (yz1 - yz2), ez);
    }
    if (i >= c.src_lo[0] && i < c.src_hi[0] && j >= c.src_lo[1] && j < c.src_hi[1] && kg >= c.src_lo[2] &&
        kg < c.src_hi[2]) {
        const int step = *a.d_base + a.offset;
        ex += src_add_t<T>(c, a.srcs, 0, i, j, kg, step);
        ey += src_add_t<T>(c, a.srcs, 1, i, j, kg, step);
        ez += src_add_t<T>(c, a.srcs, 2, i, j, kg, step);
    }
    if (!px) c.F[0][id] = ex;
    if (!py) c.F[1][id] = ey;
    if (!pz) c.F[2][id] = ez;
    if (in_sample_plane(c, a, kg) && in_sample_rect(c, i, j)) {
        // the DFT sample of E^{n+1} (a PEC-held component keeps its value)
        const long long o = sample_off(c, a, i, j, kg);
        if (c.smp[0]) c.smp[0][o] = ex;
        if (c.smp[1]) c.smp[1][o] = ey;
        if (c.smp[2]) c.smp[2][o] = ez;
    }
}

// Block (bx, by, bz) of a domain's per-cell grid: blocks of 32 x 8 threads cover 16 x 16 cells of a
// z-plane, a warp 16 x 2 cells (two aligned half-rows): a row's x slabs fill two of its warps.
__device__ __forceinline__ void cell_of(int bx, int by, int& i, int& j) {
    i = bx * 16 + (threadIdx.x & 15);
    j = by * 16 + threadIdx.y * 2 + (threadIdx.x >> 4);
}

template <typename T, bool kAniso, bool kPoles, bool kPer, bool kBack = false, bool kCurl = false>
__global__ void __launch_bounds__(kTileX* kTileY, cell_blocks<T, kPoles>())
    k_e_cell(const CellArgs<T> c, const Dom<T>* __restrict__ doms, T S, const StepArgs a) {
    int i, j;
    cell_of(blockIdx.x, blockIdx.y, i, j);
    e_cell_body<T, kAniso, kPoles, kPer, kBack, kCurl>(c, doms, S, a, i, j, blockIdx.z);
}

// Domain of block b of a multi-domain launch: the last d with bbeg[d] <= b (bbeg: prefix sums of the
// domains' block counts); its argument block is copied into shared memory once per block.
template <typename T>
__device__ __forceinline__ int multi_cell(const CellArgs<T>* __restrict__ args, const int* __restrict__ bbeg, int ndom,
                                          CellArgs<T>& sc, int& i, int& j, int& k) {
    const int b = blockIdx.x;
    int lo = 0, hi = ndom - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bbeg[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const int tid = threadIdx.y * kTileX + threadIdx.x;
    const int* src = (const int*)(args + lo);
    int* dst = (int*)&sc;
    for (int w = tid; w < (int)(sizeof(CellArgs<T>) / sizeof(int)); w += kTileX * kTileY) dst[w] = src[w];
    __syncthreads();
    const int local = b - bbeg[lo];
    const int gx = (sc.n[0] + 15) >> 4, gy = (sc.n[1] + 15) >> 4;
    cell_of(local % gx, (local / gx) % gy, i, j);
    k = local / (gx * gy);
    return lo;
}

// Every domain of a batch in one launch (per-cell launch mode with several domains): the same body as
// k_e_cell, the domain's operands read from its argument block.
template <typename T, bool kAniso, bool kPoles, bool kPer>
__global__ void __launch_bounds__(kTileX* kTileY, cell_blocks<T, kPoles>())
    k_e_cells(const CellArgs<T>* __restrict__ args, const int* __restrict__ bbeg, int ndom,
              const Dom<T>* __restrict__ doms, T S, const StepArgs a) {
    __shared__ CellArgs<T> sc;
    int i, j, k;
    multi_cell(args, bbeg, ndom, sc, i, j, k);
    e_cell_body<T, kAniso, kPoles, kPer, false, false>(sc, doms, S, a, i, j, k);
}


// kBack: backward H step, H^{n+1/2} = (H^{n+3/2} - m^n) + S curl E^{n+1}, called with S negated.
template <typename T, bool kPer, bool kBack>
__device__ __forceinline__ void h_cell_body(const CellArgs<T>& c, T S, const StepArgs& a, int i, int j, int k) {
    const int nx = c.n[0], ny = c.n[1], nz = c.n[2];
    const int kg = k + c.kz0;   // global plane (CPML z profile, sources)
    if (i < nx && j < ny) {
        const long long nxy = (long long)nx * ny;
        const long long id = ((long long)k * ny + j) * nx + i;
        const T* Ex = c.F[0];
        const T* Ey = c.F[1];
        const T* Ez = c.F[2];
        bool xe, ye, ze;   // the + neighbour exists (wraps on a periodic axis)
        const long long ox = nb_plus(i, nx, 1, kPer && c.per[0], &xe);
        const long long oy = nb_plus(j, ny, nx, kPer && c.per[1], &ye);
        const long long oz = nb_plus(k, nz, nxy, 0, &ze);
        const T exk = Ex[id], eyk = Ey[id], ez = Ez[id];
        T yx1 = (ye ? Ez[id + oy] : T(0)) - ez, yx2 = (ze ? Ey[id + oz] : T(0)) - eyk;   // Hx: dEz/dy, dEy/dz
        T yy1 = (ze ? Ex[id + oz] : T(0)) - exk, yy2 = (xe ? Ez[id + ox] : T(0)) - ez;   // Hy: dEx/dz, dEz/dx
        T yz1 = (xe ? Ey[id + ox] : T(0)) - eyk, yz2 = (ye ? Ex[id + oy] : T(0)) - exk;  // Hz: dEy/dx, dEx/dy
        const T hx = c.F[3][id], hy = c.F[4][id], hz = c.F[5][id];
        if (kBack) {
            if (i < c.alo[0] || i >= c.ahi[0] || j < c.alo[1] || j >= c.ahi[1] || k < c.alo[2] || k >= c.ahi[2]) return;
            T mx = T(0), my = T(0), mz = T(0);
            if (i >= c.src_lo[0] && i < c.src_hi[0] && j >= c.src_lo[1] && j < c.src_hi[1] && kg >= c.src_lo[2] &&
                kg < c.src_hi[2]) {
                const int step = *a.d_base + a.offset;
                mx = src_add_t<T>(c, a.srcs, 3, i, j, kg, step);
                my = src_add_t<T>(c, a.srcs, 4, i, j, kg, step);
                mz = src_add_t<T>(c, a.srcs, 5, i, j, kg, step);
            }
            c.F[3][id] = fma_t(-S, (yx1 - yx2), hx - mx);
            c.F[4][id] = fma_t(-S, (yy1 - yy2), hy - my);
            c.F[5][id] = fma_t(-S, (yz1 - yz2), hz - mz);
            return;
        }
        // in-slab CPML corrections; each axis' coefficients are loaded once for its two derivatives
        if (c.ns[2]) {
            const int sl = slab_of(kg, c.dlo[2], c.dhi[2], c.nzg);
            if (sl >= 0) {
                const long long o = ((long long)sl * ny + j) * nx + i;
                const T b = c.coef[2][kg], cc = c.coef[2][c.nzg + kg], kk = c.coef[2][2 * c.nzg + kg];
                yx2 = cpml_rec(b, cc, kk, c.psi[0][1] + o, yx2);
                yy1 = cpml_rec(b, cc, kk, c.psi[1][0] + o, yy1);
            }
        }
        if (c.ns[0]) {
            const int sl = slab_of(i, c.dlo[0], c.dhi[0], nx);
            if (sl >= 0) {
                const long long o = ((long long)k * ny + j) * c.ns[0] + sl;
                const T b = c.coef[0][i], cc = c.coef[0][nx + i], kk = c.coef[0][2 * nx + i];
                yy2 = cpml_rec(b, cc, kk, c.psi[1][1] + o, yy2);
                yz1 = cpml_rec(b, cc, kk, c.psi[2][0] + o, yz1);
            }
        }
        if (c.ns[1]) {
            const int sl = slab_of(j, c.dlo[1], c.dhi[1], ny);
            if (sl >= 0) {
                const long long o = ((long long)k * c.ns[1] + sl) * nx + i;
                const T b = c.coef[1][j], cc = c.coef[1][ny + j], kk = c.coef[1][2 * ny + j];
                yx1 = cpml_rec(b, cc, kk, c.psi[0][0] + o, yx1);
                yz2 = cpml_rec(b, cc, kk, c.psi[2][1] + o, yz2);
            }
        }
        T hx1 = fma_t(-S, (yx1 - yx2), hx);
        T hy1 = fma_t(-S, (yy1 - yy2), hy);
        T hz1 = fma_t(-S, (yz1 - yz2), hz);
        if (i >= c.src_lo[0] && i < c.src_hi[0] && j >= c.src_lo[1] && j < c.src_hi[1] && kg >= c.src_lo[2] &&
            kg < c.src_hi[2]) {
            const int step = *a.d_base + a.offset;
            hx1 += src_add_t<T>(c, a.srcs, 3, i, j, kg, step);
            hy1 += src_add_t<T>(c, a.srcs, 4, i, j, kg, step);
            hz1 += src_add_t<T>(c, a.srcs, 5, i, j, kg, step);
        }
        c.F[3][id] = hx1;
        c.F[4][id] = hy1;
        c.F[5][id] = hz1;
        if (in_sample_plane(c, a, kg) && in_sample_rect(c, i, j)) {
            // the DFT sample of H^{n+3/2}
            const long long o = sample_off(c, a, i, j, kg);
            if (c.smp[3]) c.smp[3][o] = hx1;
            if (c.smp[4]) c.smp[4][o] = hy1;
            if (c.smp[5]) c.smp[5][o] = hz1;
        }
    }
}

template <typename T, bool kPer, bool kBack = false>
__global__ void __launch_bounds__(kTileX* kTileY, cell_blocks<T>()) k_h_cell(const CellArgs<T> c, T S, const StepArgs a) {
    int i, j;
    cell_of(blockIdx.x, blockIdx.y, i, j);
    h_cell_body<T, kPer, kBack>(c, S, a, i, j, blockIdx.z);
}

template <typename T, bool kPer>
__global__ void __launch_bounds__(kTileX* kTileY, cell_blocks<T>())
    k_h_cells(const CellArgs<T>* __restrict__ args, const int* __restrict__ bbeg, int ndom, T S, const StepArgs a) {
    __shared__ CellArgs<T> sc;
    int i, j, k;
    multi_cell(args, bbeg, ndom, sc, i, j, k);
    h_cell_body<T, kPer, false>(sc, S, a, i, j, k);
}


// grid: (x chunks of kTileX, y chunks of kTileY, z planes)
inline dim3 cell_grid(const int* n) {
    return dim3((unsigned)((n[0] + 15) / 16), (unsigned)((n[1] + 15) / 16), (unsigned)n[2]);
}

template <typename T, bool kPer>
static void launch_e_cell_t(const Launch& L, const CellArgs<T>& c, const Dom<T>* doms, T S, const StepArgs& a,
                            int aniso, int poles) {
    const dim3 g = cell_grid(c.n), b(kTileX, kTileY);
    if (poles)
        (aniso ? k_e_cell<T, true, true, kPer> : k_e_cell<T, false, true, kPer>)<<<g, b, 0, L.stream>>>(c, doms, S, a);
    else
        (aniso ? k_e_cell<T, true, false, kPer> : k_e_cell<T, false, false, kPer>)<<<g, b, 0, L.stream>>>(c, doms, S,
                                                                                                         a);
}

template <typename T>
void launch_e_cell(const Launch& L, const CellArgs<T>& c, const Dom<T>* doms, T S, const StepArgs& a, int aniso,
                   int poles) {
    if (c.per[0] || c.per[1])
        launch_e_cell_t<T, true>(L, c, doms, S, a, aniso, poles);
    else
        launch_e_cell_t<T, false>(L, c, doms, S, a, aniso, poles);
    ++*L.counter;
}

template <typename T>
void launch_e_cells(const Launch& L, const CellArgs<T>* args, const int* bbeg, int ndom, int nblocks,
                    const Dom<T>* doms, T S, const StepArgs& a, int aniso, int poles, int per) {
    const dim3 b(kTileX, kTileY);
    if (per) {
        if (poles)
            (aniso ? k_e_cells<T, true, true, true> : k_e_cells<T, false, true, true>)<<<nblocks, b, 0, L.stream>>>(
                args, bbeg, ndom, doms, S, a);
        else
            (aniso ? k_e_cells<T, true, false, true> : k_e_cells<T, false, false, true>)<<<nblocks, b, 0, L.stream>>>(
                args, bbeg, ndom, doms, S, a);
    } else {
        if (poles)
            (aniso ? k_e_cells<T, true, true, false> : k_e_cells<T, false, true, false>)<<<nblocks, b, 0, L.stream>>>(
                args, bbeg, ndom, doms, S, a);
        else
            (aniso ? k_e_cells<T, true, false, false> : k_e_cells<T, false, false, false>)<<<nblocks, b, 0, L.stream>>>(
                args, bbeg, ndom, doms, S, a);
    }
    ++*L.counter;
}

template <typename T>
void launch_h_cells(const Launch& L, const CellArgs<T>* args, const int* bbeg, int ndom, int nblocks, T S,
                    const StepArgs& a, int per) {
    const dim3 b(kTileX, kTileY);
    if (per)
        k_h_cells<T, true><<<nblocks, b, 0, L.stream>>>(args, bbeg, ndom, S, a);
    else
        k_h_cells<T, false><<<nblocks, b, 0, L.stream>>>(args, bbeg, ndom, S, a);
    ++*L.counter;
}

template <typename T>
void launch_e_curl(const Launch& L, const CellArgs<T>& c) {
    const dim3 g = cell_grid(c.n), b(kTileX, kTileY);
    if (c.per[0] || c.per[1])
        k_e_cell<T, false, false, true, false, true><<<g, b, 0, L.stream>>>(c, nullptr, T(0), StepArgs{});
    else
        k_e_cell<T, false, false, false, false, true><<<g, b, 0, L.stream>>>(c, nullptr, T(0), StepArgs{});
    ++*L.counter;
}

// Backward step of a lossless domain: the H kernel first (it reads E^{n+1}), then the E kernel.
template <typename T>
void launch_back_cell(const Launch& L, const CellArgs<T>& ce, const CellArgs<T>& ch, T S, const StepArgs& a,
                      int aniso) {
    const dim3 g = cell_grid(ce.n), b(kTileX, kTileY);
    const bool per = ce.per[0] || ce.per[1];
    if (per)
        k_h_cell<T, true, true><<<g, b, 0, L.stream>>>(ch, -S, a);
    else
        k_h_cell<T, false, true><<<g, b, 0, L.stream>>>(ch, -S, a);
    if (aniso)
        (per ? k_e_cell<T, true, false, true, true> : k_e_cell<T, true, false, false, true>)<<<g, b, 0, L.stream>>>(
            ce, nullptr, -S, a);
    else
        (per ? k_e_cell<T, false, false, true, true> : k_e_cell<T, false, false, false, true>)<<<g, b, 0, L.stream>>>(
            ce, nullptr, -S, a);
    *L.counter += 2;
}

template <typename T>
void launch_back_h(const Launch& L, const CellArgs<T>& ch, T S, const StepArgs& a) {
    const dim3 g = cell_grid(ch.n), b(kTileX, kTileY);
    if (ch.per[0] || ch.per[1])
        k_h_cell<T, true, true><<<g, b, 0, L.stream>>>(ch, -S, a);
    else
        k_h_cell<T, false, true><<<g, b, 0, L.stream>>>(ch, -S, a);
    ++*L.counter;
}

template <typename T>
void launch_back_e(const Launch& L, const CellArgs<T>& ce, T S, const StepArgs& a, int aniso) {
    const dim3 g = cell_grid(ce.n), b(kTileX, kTileY);
    const bool per = ce.per[0] || ce.per[1];
    if (aniso)
        (per ? k_e_cell<T, true, false, true, true> : k_e_cell<T, true, false, false, true>)<<<g, b, 0, L.stream>>>(
            ce, nullptr, -S, a);
    else
        (per ? k_e_cell<T, false, false, true, true> : k_e_cell<T, false, false, false, true>)<<<g, b, 0, L.stream>>>(
            ce, nullptr, -S, a);
    ++*L.counter;
}

// Interface planes <-> record slot (see IfaceArgs): blockIdx.y picks the plane, threads run over
// its three components x cells.
template <typename T>
__global__ void __launch_bounds__(256) k_iface(const int n0, const int n1, const int n2, const IfaceArgs ia,
                                               T* __restrict__ rec, const int* __restrict__ d_base, int bias, int kinds,
                                               int to_rec, T* Ex, T* Ey, T* Ez, T* Hx, T* Hy, T* Hz) {
    if (blockIdx.y >= (unsigned)ia.np) return;
    const IfacePlane pl = ia.p[blockIdx.y];
    if (!((kinds >> pl.kind) & 1)) return;   // kind 0 = H (bit 0), 1 = E (bit 1)
    const long long s = (long long)(d_base ? *d_base : 0) + bias - ia.t0;
    if (s < 0 || s > ia.cap) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * pl.cells) return;
    const int comp = (int)(t / pl.cells);
    const long long cell = t - (long long)comp * pl.cells;
    // plane cell -> (i, j, k): the two other axes in increasing order, the first one fastest
    int c[3];
    const int nn[3] = {n0, n1, n2};
    const int a0 = pl.q == 0 ? 1 : 0, a1 = pl.q == 2 ? 1 : 2;
    c[pl.q] = pl.x;
    c[a0] = (int)(cell % nn[a0]);
    c[a1] = (int)(cell / nn[a0]);
    const long long id = ((long long)c[2] * n1 + c[1]) * n0 + c[0];
    T* fields[6] = {Ex, Ey, Ez, Hx, Hy, Hz};
    T* f = fields[(pl.kind == 0 ? 3 : 0) + comp];
    T* r = rec + s * ia.slot + pl.off + t;
    if (to_rec)
        *r = f[id];
    else
        f[id] = *r;
}

template <typename T>
void launch_iface(const Launch& L, T* const* F, const int* n, const IfaceArgs& ia, T* rec, const int* d_base, int bias,
                  int kinds, int to_rec) {
    if (ia.np <= 0) return;
    long long most = 0;
    for (int q = 0; q < ia.np; ++q) most = most > 3 * ia.p[q].cells ? most : 3 * ia.p[q].cells;
    const dim3 g((unsigned)((most + 255) / 256), (unsigned)ia.np);
    k_iface<T><<<g, 256, 0, L.stream>>>(n[0], n[1], n[2], ia, rec, d_base, bias, kinds, to_rec, F[0], F[1], F[2], F[3],
                                         F[4], F[5]);
    ++*L.counter;
}

template <typename T>
void launch_h_cell(const Launch& L, const CellArgs<T>& c, T S, const StepArgs& a) {
    const dim3 g = cell_grid(c.n), b(kTileX, kTileY);
    if (c.per[0] || c.per[1])
        k_h_cell<T, true><<<g, b, 0, L.stream>>>(c, S, a);
    else
        k_h_cell<T, false><<<g, b, 0, L.stream>>>(c, S, a);
    ++*L.counter;
}

__global__ void k_advance(int* d_step, int delta) { *d_step += delta; }

// ---- host launchers --------------------------------------------------------------------------
template <typename T>
void launch_e_update(const Launch& L, const Dom<T>* doms, const Tile* tiles, int ntiles, T S, const StepArgs& a,
                     int general, int aniso) {
    if (ntiles <= 0) return;
    const dim3 b(kTileX, kTileY);
    if (general)
        k_e_update<T, true, true><<<ntiles, b, 0, L.stream>>>(doms, tiles, S, a);
    else
        (aniso ? k_e_update<T, false, true> : k_e_update<T, false, false>)<<<ntiles, b, 0, L.stream>>>(doms, tiles, S,
                                                                                                     a);
    ++*L.counter;
}

template <typename T>
void launch_h_update(const Launch& L, const Dom<T>* doms, const Tile* tiles, int ntiles, T S, const StepArgs& a,
                     int general, int energy, unsigned advance) {
    if (ntiles <= 0) return;
    const dim3 b(kTileX, kTileY);
    if (general)
        (energy ? k_h_update<T, true, true> : k_h_update<T, true, false>)<<<ntiles, b, 0, L.stream>>>(doms, tiles, S, a,
                                                                                                    advance);
    else
        (energy ? k_h_update<T, false, true> : k_h_update<T, false, false>)<<<ntiles, b, 0, L.stream>>>(
            doms, tiles, S, a, advance);
    ++*L.counter;
}

template <typename T>
void launch_dft(const Launch& L, const Dom<T>* doms, const Mon* mons, const DftItem* items, int nitems, int kind,
                const int* d_base, int offset) {
    if (nitems <= 0) return;
    k_dft<T><<<nitems, dim3(kTileX, kTileY), 0, L.stream>>>(doms, mons, items, kind, d_base, offset);
    ++*L.counter;
}

template <typename T>
void launch_dft_ring(const Launch& L, const Mon* mons, const DftItem* items, int nitems, const int* d_base, int cnt) {
    if (nitems <= 0 || cnt <= 0) return;
    // one grid row per component slot (6 at most; rows past a monitor's components return at once)
    k_dft_ring<T><<<dim3(nitems, 6), dim3(kTileX, kTileY), 0, L.stream>>>(mons, items, d_base, cnt);
    ++*L.counter;
}

void launch_copy_int(const Launch& L, const int* src, int* dst) {
    k_copy_int<<<1, 1, 0, L.stream>>>(src, dst);
    ++*L.counter;
}

void launch_set_int(const Launch& L, int* dst, int v) {
    k_set_int<<<1, 1, 0, L.stream>>>(dst, v);
    ++*L.counter;
}

void launch_advance(const Launch& L, int* d_step, int delta) {
    k_advance<<<1, 1, 0, L.stream>>>(d_step, delta);
    ++*L.counter;
}

#define GBFDTD_INST(T)                                                                                           \
    template void launch_e_update<T>(const Launch&, const Dom<T>*, const Tile*, int, T, const StepArgs&, int, int); \
    template void launch_h_update<T>(const Launch&, const Dom<T>*, const Tile*, int, T, const StepArgs&, int, int,  \
                                     unsigned);
GBFDTD_INST(float)
GBFDTD_INST(double)
#undef GBFDTD_INST
template void launch_dft<float>(const Launch&, const Dom<float>*, const Mon*, const DftItem*, int, int, const int*,
                                int);
template void launch_dft<double>(const Launch&, const Dom<double>*, const Mon*, const DftItem*, int, int, const int*,
                                 int);
template void launch_dft_ring<float>(const Launch&, const Mon*, const DftItem*, int, const int*, int);
template void launch_dft_ring<double>(const Launch&, const Mon*, const DftItem*, int, const int*, int);
template void launch_e_cell<float>(const Launch&, const CellArgs<float>&, const Dom<float>*, float, const StepArgs&,
                                   int, int);
template void launch_e_cell<double>(const Launch&, const CellArgs<double>&, const Dom<double>*, double,
                                    const StepArgs&, int, int);
template void launch_back_cell<float>(const Launch&, const CellArgs<float>&, const CellArgs<float>&, float,
                                      const StepArgs&, int);
template void launch_back_cell<double>(const Launch&, const CellArgs<double>&, const CellArgs<double>&, double,
                                       const StepArgs&, int);
template void launch_back_h<float>(const Launch&, const CellArgs<float>&, float, const StepArgs&);
template void launch_back_h<double>(const Launch&, const CellArgs<double>&, double, const StepArgs&);
template void launch_back_e<float>(const Launch&, const CellArgs<float>&, float, const StepArgs&, int);
template void launch_back_e<double>(const Launch&, const CellArgs<double>&, double, const StepArgs&, int);
template void launch_iface<float>(const Launch&, float* const*, const int*, const IfaceArgs&, float*, const int*, int,
                                  int, int);
template void launch_iface<double>(const Launch&, double* const*, const int*, const IfaceArgs&, double*, const int*,
                                   int, int, int);
template void launch_e_cells<float>(const Launch&, const CellArgs<float>*, const int*, int, int, const Dom<float>*,
                                    float, const StepArgs&, int, int, int);
template void launch_e_cells<double>(const Launch&, const CellArgs<double>*, const int*, int, int,
                                     const Dom<double>*, double, const StepArgs&, int, int, int);
template void launch_h_cells<float>(const Launch&, const CellArgs<float>*, const int*, int, int, float,
                                    const StepArgs&, int);
template void launch_h_cells<double>(const Launch&, const CellArgs<double>*, const int*, int, int, double,
                                     const StepArgs&, int);
template void launch_e_curl<float>(const Launch&, const CellArgs<float>&);
template void launch_e_curl<double>(const Launch&, const CellArgs<double>&);
template void launch_h_cell<float>(const Launch&, const CellArgs<float>&, float, const StepArgs&);
template void launch_h_cell<double>(const Launch&, const CellArgs<double>&, double, const StepArgs&);

}  // namespace gbfdtd
