// Forward half-steps of the Yee leapfrog (arxiv 2609.30039, Sec. 2.1 Eq. (yee)) with the CPML
// memories of Sec. 2.2, the trapezoidal Drude/Lorentz update and diagonal eps^-1 of Sec. 2.3,
// soft sources and running DFT monitors of Sec. 2.4.
//
// Work decomposition: a tile is 32 x 4 columns of one domain; each thread owns a column (i, j)
// and marches k over the tile's z range, so consecutive planes of the same column stay in L1
// and every warp reads 32 consecutive floats (128 B) of each array.
#include "fdtd_internal.cuh"

namespace gbfdtd {

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

// In-slab CPML correction of one derivative: psi updated first, then y = D/kappa + psi.
template <typename T>
__device__ __forceinline__ T cpml_apply(const Cpml1<T>& q, T* psi, T D) {
    const T ps = q.b * (*psi) + q.c * D;
    *psi = ps;
    return q.k * D + ps;
}

// Trapezoidal pole update of one E component (Sec. 2.3):
// (eps_inf + G) E^{n+1} = (eps_inf + G) E^n + Delta,
// Delta = S curl + sum_p (P_p - (M_p x_p)_P - 2 g_p E^n);  x_p <- M_p x_p + g_p (E^{n+1} + E^n).
template <typename T>
__device__ __forceinline__ T ade_update(const Dom<T>& d, int a, long long bo, T e0, T ie, T scurl) {
    T delta = scurl;
    T* base = d.ade + (long long)a * d.npole * 2 * d.bcell + bo;
    for (int p = 0; p < d.npole; ++p) {
        const T P = base[(2 * p) * d.bcell], Q = base[(2 * p + 1) * d.bcell];
        delta += P - (d.M00[p] * P + d.M01[p] * Q) - T(2) * d.g0[p] * e0;
    }
    const T e1 = e0 + ie / (T(1) + ie * d.G) * delta;
    const T es = e1 + e0;
    for (int p = 0; p < d.npole; ++p) {
        T* pp = base + (2 * p) * d.bcell;
        T* pq = base + (2 * p + 1) * d.bcell;
        const T P = *pp, Q = *pq;
        *pp = d.M00[p] * P + d.M01[p] * Q + d.g0[p] * es;
        *pq = d.M10[p] * P + d.M11[p] * Q + d.g1[p] * es;
    }
    return e1;
}

// E half-step (Eq. (yee) first half) of a tile.  kGen = false: the tile touches no CPML slab,
// PEC plane, domain edge or dispersive cell, so none of that code is compiled in.  Every load of
// a plane is issued before any store of it; H_x, H_y of plane k-1 stay in registers.
template <typename T, bool kGen, bool kAniso>
__global__ void __launch_bounds__(kTileX* kTileY) k_e_update(const Dom<T>* __restrict__ doms,
                                                             const Tile* __restrict__ tiles, T S) {
    const Tile t = tiles[blockIdx.x];
    const Dom<T>& d = doms[t.dom];
    const int nx = d.n[0], ny = d.n[1];
    const int i = t.x0 + threadIdx.x, j = t.y0 + threadIdx.y;
    if (i >= nx || j >= ny) return;
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
    bool pi = false, pj = false;
    if (kGen) {
        cx = cpml_at(d, d.cE[0], 0, i);
        cy = cpml_at(d, d.cE[1], 1, j);
        pi = i == 0;
        pj = j == 0;
    }
    long long id = (long long)t.z0 * nxy + (long long)j * nx + i;
    T hxz = T(0), hyz = T(0);
    if (!kGen || t.z0 > 0) {
        hxz = Hx[id - nxy];
        hyz = Hy[id - nxy];
    }
    for (int k = t.z0; k < t.z1; ++k, id += nxy) {
        const T hx = Hx[id], hy = Hy[id], hz = Hz[id];
        const T hz_ym = (!kGen || !pj) ? Hz[id - nx] : T(0);
        const T hx_ym = (!kGen || !pj) ? Hx[id - nx] : T(0);
        const T hz_xm = (!kGen || !pi) ? Hz[id - 1] : T(0);
        const T hy_xm = (!kGen || !pi) ? Hy[id - 1] : T(0);
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
                if (!px) ex += S * iex * (yx1 - yx2);
                if (!py) ey += S * iey * (yy1 - yy2);
                if (!pz) ez += S * iez * (yz1 - yz2);
            }
            if (!px) Ex[id] = ex;
            if (!py) Ey[id] = ey;
            if (!pz) Ez[id] = ez;
        } else {
            Ex[id] = ex + S * iex * (yx1 - yx2);
            Ey[id] = ey + S * iey * (yy1 - yy2);
            Ez[id] = ez + S * iez * (yz1 - yz2);
        }
    }
}

// H half-step (Eq. (yee) second half) of a tile; E_x, E_y of plane k+1 are carried to the next
// plane in registers.  kEnergy adds W_{n+1} = 1/2 sum eps |E|^2 + 1/2 sum H^{n+1/2} H^{n+3/2}.
template <typename T, bool kGen, bool kEnergy>
__global__ void __launch_bounds__(kTileX* kTileY) k_h_update(const Dom<T>* __restrict__ doms,
                                                             const Tile* __restrict__ tiles, T S,
                                                             const int* __restrict__ d_step) {
    const Tile t = tiles[blockIdx.x];
    const Dom<T>& d = doms[t.dom];
    const int nx = d.n[0], ny = d.n[1], nz = d.n[2];
    const int i = t.x0 + threadIdx.x, j = t.y0 + threadIdx.y;
    double w = 0.0;
    if (i < nx && j < ny) {
        const long long nxy = (long long)nx * ny;
        const T* Ex = d.F[0];
        const T* Ey = d.F[1];
        const T* Ez = d.F[2];
        T* Hx = d.F[3];
        T* Hy = d.F[4];
        T* Hz = d.F[5];
        Cpml1<T> cx, cy;
        bool xe = true, ye = true;  // the +x / +y neighbour node exists
        if (kGen) {
            cx = cpml_at(d, d.cH[0], 0, i);
            cy = cpml_at(d, d.cH[1], 1, j);
            xe = i + 1 < nx;
            ye = j + 1 < ny;
        }
        long long id = (long long)t.z0 * nxy + (long long)j * nx + i;
        T exk = Ex[id], eyk = Ey[id];
        for (int k = t.z0; k < t.z1; ++k, id += nxy) {
            const bool ze = !kGen || k + 1 < nz;
            const T exn = ze ? Ex[id + nxy] : T(0);
            const T eyn = ze ? Ey[id + nxy] : T(0);
            const T ez = Ez[id];
            const T ez_yp = ye ? Ez[id + nx] : T(0);
            const T ez_xp = xe ? Ez[id + 1] : T(0);
            const T ey_xp = xe ? Ey[id + 1] : T(0);
            const T ex_yp = ye ? Ex[id + nx] : T(0);
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
            const T hx1 = hx - S * (yx1 - yx2);
            const T hy1 = hy - S * (yy1 - yy2);
            const T hz1 = hz - S * (yz1 - yz2);
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
        const int step = *d_step;
        if ((threadIdx.x & 31) == 0 && d.energy && step < d.energy_cap) atomicAdd(d.energy + step, w);
    }
}

template <typename T>
__global__ void k_sources(const Dom<T>* __restrict__ doms, const Src* __restrict__ srcs, int nsrc, long long ncells,
                          const int* __restrict__ d_step) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= ncells) return;
    int s = 0;
    while (s + 1 < nsrc && srcs[s + 1].begin <= t) ++s;
    const Src& sr = srcs[s];
    const int step = *d_step;
    if (step >= sr.n) return;
    const long long l = t - sr.begin;
    const int i = sr.lo[0] + (int)(l % sr.bx);
    const int j = sr.lo[1] + (int)((l / sr.bx) % sr.by);
    const int k = sr.lo[2] + (int)(l / ((long long)sr.bx * sr.by));
    const Dom<T>& d = doms[sr.dom];
    d.F[sr.comp][cidx(d.n, i, j, k)] += (T)sr.wave[step];
}

// Running DFT (Sec. 2.4): F += f(t) exp(i w t), FP64 accumulation of the field value.
template <typename T>
__global__ void k_dft(const Dom<T>* __restrict__ doms, const Mon* __restrict__ mons, const int* __restrict__ entries,
                      int nentries, long long nthreads, const long long* __restrict__ entry_begin,
                      const int* __restrict__ d_step, int kind) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nthreads) return;
    int e = 0;
    while (e + 1 < nentries && entry_begin[e + 1] <= t) ++e;
    const int mi = entries[2 * e], ci = entries[2 * e + 1];
    const Mon& m = mons[mi];
    const long long cell = t - entry_begin[e];
    const int i = m.lo[0] + (int)(cell % m.bx);
    const int j = m.lo[1] + (int)((cell / m.bx) % m.by);
    const int k = m.lo[2] + (int)(cell / ((long long)m.bx * m.by));
    const Dom<T>& d = doms[m.dom];
    const double v = (double)d.F[m.comps[ci]][cidx(d.n, i, j, k)];
    const int step = *d_step;
    const double2* ph = m.phase + ((long long)step * 2 + kind) * m.nf;
    double2* acc = m.acc + (long long)ci * m.nf * m.ncell + cell;
    for (int f = 0; f < m.nf; ++f) {
        const double2 p = ph[f];
        double2 a = acc[(long long)f * m.ncell];
        a.x += v * p.x;
        a.y += v * p.y;
        acc[(long long)f * m.ncell] = a;
    }
}

__global__ void k_advance(int* d_step, int delta) { *d_step += delta; }

// ---- host launchers --------------------------------------------------------------------------
template <typename T>
void launch_e_update(const Launch& L, const Dom<T>* doms, const Tile* tiles, int ntiles, T S, int general, int aniso) {
    if (ntiles <= 0) return;
    const dim3 b(kTileX, kTileY);
    if (general)
        k_e_update<T, true, true><<<ntiles, b, 0, L.stream>>>(doms, tiles, S);
    else if (aniso)
        k_e_update<T, false, true><<<ntiles, b, 0, L.stream>>>(doms, tiles, S);
    else
        k_e_update<T, false, false><<<ntiles, b, 0, L.stream>>>(doms, tiles, S);
    ++*L.counter;
}

template <typename T>
void launch_h_update(const Launch& L, const Dom<T>* doms, const Tile* tiles, int ntiles, T S, const int* d_step,
                     int general, int energy) {
    if (ntiles <= 0) return;
    const dim3 b(kTileX, kTileY);
    if (general) {
        if (energy)
            k_h_update<T, true, true><<<ntiles, b, 0, L.stream>>>(doms, tiles, S, d_step);
        else
            k_h_update<T, true, false><<<ntiles, b, 0, L.stream>>>(doms, tiles, S, d_step);
    } else {
        if (energy)
            k_h_update<T, false, true><<<ntiles, b, 0, L.stream>>>(doms, tiles, S, d_step);
        else
            k_h_update<T, false, false><<<ntiles, b, 0, L.stream>>>(doms, tiles, S, d_step);
    }
    ++*L.counter;
}

template <typename T>
void launch_sources(const Launch& L, const Dom<T>* doms, const Src* srcs, int nsrc, long long ncells,
                    const int* d_step) {
    if (nsrc <= 0 || ncells <= 0) return;
    const int bs = 256;
    k_sources<T><<<(unsigned)((ncells + bs - 1) / bs), bs, 0, L.stream>>>(doms, srcs, nsrc, ncells, d_step);
    ++*L.counter;
}

template <typename T>
void launch_dft(const Launch& L, const Dom<T>* doms, const Mon* mons, const int* entries, int nentries,
                long long nthreads, const long long* entry_begin, const int* d_step, int kind) {
    if (nentries <= 0 || nthreads <= 0) return;
    const int bs = 256;
    k_dft<T><<<(unsigned)((nthreads + bs - 1) / bs), bs, 0, L.stream>>>(doms, mons, entries, nentries, nthreads,
                                                                        entry_begin, d_step, kind);
    ++*L.counter;
}

void launch_advance(const Launch& L, int* d_step, int delta) {
    k_advance<<<1, 1, 0, L.stream>>>(d_step, delta);
    ++*L.counter;
}

#define GBFDTD_INST(T)                                                                                           \
    template void launch_e_update<T>(const Launch&, const Dom<T>*, const Tile*, int, T, int, int);               \
    template void launch_h_update<T>(const Launch&, const Dom<T>*, const Tile*, int, T, const int*, int, int);   \
    template void launch_sources<T>(const Launch&, const Dom<T>*, const Src*, int, long long, const int*);       \
    template void launch_dft<T>(const Launch&, const Dom<T>*, const Mon*, const int*, int, long long,            \
                                const long long*, const int*, int);
GBFDTD_INST(float)
GBFDTD_INST(double)
#undef GBFDTD_INST

}  // namespace gbfdtd
