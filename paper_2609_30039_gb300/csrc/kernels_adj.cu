// Transposed (discrete-adjoint) half-steps, arxiv 2609.30039 Sec. 3.1, Eq. (adjoint).
//
// Every forward update has a transpose kernel of the same locality, in a general form (CPML,
// PEC, poles: k_adj_e_gen / k_adj_h_gen) and an interior form (k_adj_e_int / k_adj_h_int):
//   * k_adj_e*  (one thread per E column, like the forward E update) applies the transpose of
//     the forward H update (Ebar += gathered backward differences of the H cotangent, the
//     opposite-direction differences of Sec. 3.1), injects dJ/dE of the monitors, and
//     transposes the E update's own-cell part (poles, eps^-1, material cotangent);
//   * k_adj_h*  (one thread per H column) applies the transpose of the forward E update
//     (Hbar += gathered forward differences) and the H-side CPML recursion.
// CPML transpose (Sec. 3.1): psibar_mem = psibar + ybar, Dbar = ybar/kappa + c psibar_mem,
// psibar_old = b psibar_mem.  Pole transpose: the 2x2 trapezoidal system applied to the
// cotangents with M^T.
//
// Gather form needs the cotangent of every neighbour's derivative D while its owner is still
// updating psibar.  So that no kernel reads a value another thread of the same launch writes,
// the E-side own-cell part of transposed step m is deferred to the next k_adj_e* (m-1):
// after k_adj_e*(m) the E array holds F = S/(eps_inf + G) * Etilde_bar (the cotangent of the
// curl, which k_adj_h needs at neighbours), and the pole/psi cotangents still hold their step
// m+1 values.  k_adj_e*(m-1) (or k_adj_flush) first completes step m for its own cell:
//   Ebar^m   = (eps_inf - G)/S * F + sum_p g_p . xbar_p
//   xbar_p^m = M_p^T xbar_p + ((1 - M00_p) / S, -M01_p / S) F
//   psibar_E^m = b (psibar_E + (+F | -F))
// The H side needs no deferral: psibar_H of step m is finished by k_adj_h*(m) after
// k_adj_e*(m) has read it.
#include "fdtd_internal.cuh"

namespace gbfdtd {

// Completes the deferred own-cell transpose of an E update for component a; returns Ebar.
template <typename T>
__device__ __forceinline__ T e_deferred(const Dom<T>& d, int a, int i, int j, int k, long long id, bool disp,
                                        T F, T S) {
    const int c[3] = {i, j, k};
    const T ie = d.ie[a][id];
    T eb;
    if (disp) {
        eb = (T(1) / ie - d.G) / S * F;
        const long long bo = ade_off(d, i, j, k);
        for (int p = 0; p < d.npole; ++p) {
            T* pp = d.aade + ((long long)(a * d.npole + p) * 2 + 0) * d.bcell + bo;
            T* pq = d.aade + ((long long)(a * d.npole + p) * 2 + 1) * d.bcell + bo;
            const T xp = *pp, xq = *pq;
            eb += d.g0[p] * xp + d.g1[p] * xq;
            *pp = d.M00[p] * xp + d.M10[p] * xq + (T(1) - d.M00[p]) / S * F;
            *pq = d.M01[p] * xp + d.M11[p] * xq - d.M01[p] / S * F;
        }
    } else {
        eb = F / (S * ie);
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int ax = (a + 1 + s) % 3;
        if (d.ns[ax] == 0) continue;
        const int x = c[ax];
        const int sl = slab_of(x, d.dlo[ax], d.dhi[ax], d.n[ax]);
        if (sl < 0) continue;
        T* p = d.apsiE[a][s] + slab_off(d.n, d.ns, ax, i, j, k, sl);
        *p = d.cE[ax][x] * (*p + (s == 0 ? F : -F));
    }
    return eb;
}

template <typename T>
__device__ __forceinline__ double inject_at(const Dom<T>& d, const Mon* __restrict__ mons, int comp, int i, int j,
                                            int k, long long pidx) {
    // dJ/df(t) = Re(conj(cot) exp(i w t)), pidx = (step * 2 + kind) of the phase table
    double acc = 0.0;
    for (int mm = 0; mm < d.nmon; ++mm) {
        const Mon& m = mons[d.mon[mm]];
        if (!m.cot || !((m.mask >> comp) & 1u)) continue;
        if (i < m.lo[0] || i >= m.hi[0] || j < m.lo[1] || j >= m.hi[1] || k < m.lo[2] || k >= m.hi[2]) continue;
        int ci = 0;
        for (int c2 = 0; c2 < comp; ++c2) ci += (m.mask >> c2) & 1u;
        const long long cell = ((long long)(k - m.lo[2]) * m.by + (j - m.lo[1])) * m.bx + (i - m.lo[0]);
        const double2* ph = m.phase + pidx * m.nf;
        const double2* ct = m.cot + (long long)ci * m.nf * m.ncell + cell;
        for (int f = 0; f < m.nf; ++f) {
            const double2 c = ct[(long long)f * m.ncell];
            const double2 p = ph[f];
            acc += c.x * p.x + c.y * p.y;
        }
    }
    return acc;
}

// ---- general tiles, hoisted form -------------------------------------------------------------
// Column constants (CPML coefficients along x and y at this column and its -1 / +1 neighbour)
// are computed once per thread; along z once per plane.  Per plane every load precedes every
// store.  The cotangent terms of the z-derivatives are carried from plane to plane.

template <typename T>
struct CpmlC {   // coefficients of one node: slab index (-1 outside), b, c, 1/kappa
    int s;
    T b, c, k;
};

template <typename T>
__device__ __forceinline__ CpmlC<T> cpml_c(const Dom<T>& d, const T* coef, int q, int x) {
    CpmlC<T> r;
    r.s = (d.ns[q] && x >= 0 && x < d.n[q]) ? slab_of(x, d.dlo[q], d.dhi[q], d.n[q]) : -1;
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

// Dbar of a derivative whose ybar is yb, at a node with coefficients cc and memory cotangent ps.
template <typename T>
__device__ __forceinline__ T dbar_c(const CpmlC<T>& cc, T yb, T ps) {
    return cc.s >= 0 ? cc.k * yb + cc.c * (ps + yb) : yb;
}

// Offsets of a cell inside the slab arrays of each axis.
template <typename T>
__device__ __forceinline__ long long off_x(const Dom<T>& d, int s, int j, int k) {
    return ((long long)k * d.n[1] + j) * d.ns[0] + s;
}
template <typename T>
__device__ __forceinline__ long long off_y(const Dom<T>& d, int s, int i, int k) {
    return ((long long)k * d.ns[1] + s) * d.n[0] + i;
}
template <typename T>
__device__ __forceinline__ long long off_z(const Dom<T>& d, int s, int i, int j) {
    return ((long long)s * d.n[1] + j) * d.n[0] + i;
}

// Transposed E step of column (i, j) over planes [z0, z1) in general form (CPML, PEC, poles,
// periodic wrap); `flags` tells whether monitor injection can apply.  pacc (or nullptr): this
// thread's sums of the pole-coefficient cotangents [pole][M00, M01, M10, M11, g0, g1].
template <typename T>
__device__ __forceinline__ void adj_e_column(const Dom<T>& d, const Mon* __restrict__ mons, int i, int j, int z0,
                                             int z1, int flags, T S, int m, int pending, double* pacc) {
    const int nx = d.n[0], ny = d.n[1];
    const long long nxy = (long long)nx * ny;
    T* A0 = d.A[0];
    T* A1 = d.A[1];
    T* A2 = d.A[2];
    const T* B0 = d.A[3];
    const T* B1 = d.A[4];
    const T* B2 = d.A[5];
    // E-node coefficients (deferred psibar_E), H-node coefficients at this column and the -1 one
    const CpmlC<T> xE = cpml_c(d, d.cE[0], 0, i), yE = cpml_c(d, d.cE[1], 1, j);
    const CpmlC<T> xH = cpml_c(d, d.cH[0], 0, i), xHm = cpml_c(d, d.cH[0], 0, i - 1);
    const CpmlC<T> yH = cpml_c(d, d.cH[1], 1, j), yHm = cpml_c(d, d.cH[1], 1, j - 1);
    const bool pi = i == 0 && !d.per[0], pj = j == 0 && !d.per[1];   // PEC plane at this column
    bool hasx, hasy;                                                   // -x / -y neighbour exists
    const long long oxm = nb_minus(i, nx, 1, d.per[0], &hasx);
    const long long oym = nb_minus(j, ny, nx, d.per[1], &hasy);
    const bool gcol = d.design && i >= d.glo[0] && i < d.ghi[0] && j >= d.glo[1] && j < d.ghi[1];
    const bool mon = d.nmon && (flags & kTileMonE);
    long long id = (long long)z0 * nxy + (long long)j * nx + i;
    // z-derivative terms of H_y (s = 0) and H_x (s = 1) at plane k-1
    T tyz_m = T(0), txz_m = T(0);
    if (z0 > 0) {
        const CpmlC<T> zH = cpml_c(d, d.cH[2], 2, z0 - 1);
        const long long o = zH.s >= 0 ? off_z(d, zH.s, i, j) : 0;
        tyz_m = dbar_c(zH, -S * B1[id - nxy], zH.s >= 0 ? d.apsiH[1][0][o] : T(0));
        txz_m = dbar_c(zH, S * B0[id - nxy], zH.s >= 0 ? d.apsiH[0][1][o] : T(0));
    }
    for (int k = z0; k < z1; ++k, id += nxy) {
        const bool pk = k == 0;
        const bool px = pj || pk, py = pi || pk, pz = pi || pj;
        const CpmlC<T> zE = cpml_c(d, d.cE[2], 2, k), zH = cpml_c(d, d.cH[2], 2, k);
        // loads of the plane
        const T f0 = A0[id], f1 = A1[id], f2 = A2[id];
        const T b0 = B0[id], b1 = B1[id], b2 = B2[id];
        const T b2_xm = hasx ? B2[id + oxm] : T(0), b1_xm = hasx ? B1[id + oxm] : T(0);
        const T b2_ym = hasy ? B2[id + oym] : T(0), b0_ym = hasy ? B0[id + oym] : T(0);
        const long long oz = zH.s >= 0 ? off_z(d, zH.s, i, j) : 0;
        const T p10 = zH.s >= 0 ? d.apsiH[1][0][oz] : T(0);   // H_y, d/dz
        const T p01 = zH.s >= 0 ? d.apsiH[0][1][oz] : T(0);   // H_x, d/dz
        const T p20 = xH.s >= 0 ? d.apsiH[2][0][off_x(d, xH.s, j, k)] : T(0);                 // H_z, d/dx
        const T p20m = (hasx && xHm.s >= 0) ? d.apsiH[2][0][off_x(d, xHm.s, j, k)] : T(0);
        const T p11 = xH.s >= 0 ? d.apsiH[1][1][off_x(d, xH.s, j, k)] : T(0);                 // H_y, d/dx
        const T p11m = (hasx && xHm.s >= 0) ? d.apsiH[1][1][off_x(d, xHm.s, j, k)] : T(0);
        const T p21 = yH.s >= 0 ? d.apsiH[2][1][off_y(d, yH.s, i, k)] : T(0);                 // H_z, d/dy
        const T p21m = (hasy && yHm.s >= 0) ? d.apsiH[2][1][off_y(d, yHm.s, i, k)] : T(0);
        const T p00 = yH.s >= 0 ? d.apsiH[0][0][off_y(d, yH.s, i, k)] : T(0);                 // H_x, d/dy
        const T p00m = (hasy && yHm.s >= 0) ? d.apsiH[0][0][off_y(d, yHm.s, i, k)] : T(0);
        // derivative cotangents of the H update: s = 0 has ybar = -S Hbar, s = 1 has +S Hbar
        const T tyz = dbar_c(zH, -S * b1, p10), txz = dbar_c(zH, S * b0, p01);
        const T tzx = dbar_c(xH, -S * b2, p20), tzx_m = hasx ? dbar_c(xHm, -S * b2_xm, p20m) : T(0);
        const T tyx = dbar_c(xH, S * b1, p11), tyx_m = hasx ? dbar_c(xHm, S * b1_xm, p11m) : T(0);
        const T tzy = dbar_c(yH, S * b2, p21), tzy_m = hasy ? dbar_c(yHm, S * b2_ym, p21m) : T(0);
        const T txy = dbar_c(yH, -S * b0, p00), txy_m = hasy ? dbar_c(yHm, -S * b0_ym, p00m) : T(0);
        const bool dcell = d.npole > 0 && i >= d.blo[0] && i < d.bhi[0] && j >= d.blo[1] && j < d.bhi[1] &&
                           k >= d.blo[2] && k < d.bhi[2] && d.mask[id];
        const bool gcell = gcol && k >= d.glo[2] && k < d.ghi[2];
        const T fin[3] = {f0, f1, f2};
        const T gat[3] = {(tyz_m - tyz) + (tzy_m - tzy), (tzx_m - tzx) + (txz_m - txz), (txy_m - txy) + (tyx_m - tyx)};
        const bool pec[3] = {px, py, pz};
        // own-cell CPML nodes of E_a's two derivatives (s = 0 along (a+1)%3, s = 1 along (a+2)%3)
        const CpmlC<T>* ec[3][2] = {{&yE, &zE}, {&zE, &xE}, {&xE, &yE}};
        T fout[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (pec[a]) {
                fout[a] = T(0);
                continue;
            }
            const T ie = d.ie[a][id];
            const T F = fin[a];
            T eb;
            if (pending) {
                // complete the own-cell transpose of step m+1
                if (dcell) {
                    eb = (T(1) / ie - d.G) / S * F;
                    const long long bo = ade_off(d, i, j, k);
                    for (int p = 0; p < d.npole; ++p) {
                        T* pp = d.aade + ((long long)(a * d.npole + p) * 2 + 0) * d.bcell + bo;
                        T* pq = d.aade + ((long long)(a * d.npole + p) * 2 + 1) * d.bcell + bo;
                        const T xp = *pp, xq = *pq;
                        eb += d.g0[p] * xp + d.g1[p] * xq;
                        *pp = d.M00[p] * xp + d.M10[p] * xq + (T(1) - d.M00[p]) / S * F;
                        *pq = d.M01[p] * xp + d.M11[p] * xq - d.M01[p] / S * F;
                    }
                } else {
                    eb = F / (S * ie);
                }
#pragma unroll
                for (int s2 = 0; s2 < 2; ++s2) {
                    const CpmlC<T>& cc = *ec[a][s2];
                    if (cc.s < 0) continue;
                    const int ax = (a + 1 + s2) % 3;
                    const long long o = ax == 0 ? off_x(d, cc.s, j, k) : (ax == 1 ? off_y(d, cc.s, i, k) : off_z(d, cc.s, i, j));
                    T* pp = d.apsiE[a][s2] + o;
                    *pp = cc.b * (*pp + (s2 == 0 ? F : -F));
                }
            } else {
                eb = F;
            }
            eb += gat[a];
            if (mon) eb += (T)inject_at(d, mons, a, i, j, k, (long long)m * 2 + 0);
            T et = eb;
            T gdisp = T(0);
            if (dcell) {
                const long long bo = ade_off(d, i, j, k);
                for (int p = 0; p < d.npole; ++p) {
                    const T xp = d.aade[((long long)(a * d.npole + p) * 2 + 0) * d.bcell + bo];
                    const T xq = d.aade[((long long)(a * d.npole + p) * 2 + 1) * d.bcell + bo];
                    et += d.g0[p] * xp + d.g1[p] * xq;
                }
                gdisp = d.G;
            }
            const bool pcell = pacc && dcell;
            if (gcell || pcell) {
                const int b = (a + 1) % 3, q = (a + 2) % 3;
                // -1 neighbours along b and q (this component is not PEC-held, so they exist,
                // wrapping on a periodic axis); the cell lies outside the CPML slabs, so the
                // forward update used the plain curl
                const long long om[3] = {oxm, oym, -nxy};
                const T* Hq = d.F[3 + q];
                const T* Hb = d.F[3 + b];
                const T curl = (Hq[id] - Hq[id + om[b]]) - (Hb[id] - Hb[id + om[q]]);
                double delta = (double)(S * curl);
                const T e0 = d.F[a][id];
                const long long bo = dcell ? ade_off(d, i, j, k) : 0;
                if (dcell) {
                    for (int p = 0; p < d.npole; ++p) {
                        const T P = d.ade[((long long)(a * d.npole + p) * 2 + 0) * d.bcell + bo];
                        const T Q = d.ade[((long long)(a * d.npole + p) * 2 + 1) * d.bcell + bo];
                        delta += (double)(P - (d.M00[p] * P + d.M01[p] * Q) - T(2) * d.g0[p] * e0);
                    }
                }
                // E^{m+1} = E^m + rho delta with rho = eps^-1 / (1 + eps^-1 G)
                const double r = 1.0 / (1.0 + (double)ie * (double)gdisp);
                if (gcell) {
                    const long long gi = ((long long)(k - d.glo[2]) * (d.ghi[1] - d.glo[1]) + (j - d.glo[1])) *
                                             (d.ghi[0] - d.glo[0]) + (i - d.glo[0]);
                    const long long gn =
                        (long long)(d.ghi[0] - d.glo[0]) * (d.ghi[1] - d.glo[1]) * (d.ghi[2] - d.glo[2]);
                    d.grad[a * gn + gi] += (double)et * delta * r * r;
                }
                if (pcell) {
                    // x_p^{m+1} = M_p x_p^m + g_p es with es = E^m + E^{m+1}; E^{m+1} depends on
                    // M00, M01 (through delta) and on g0 (through delta and G): with et the total
                    // cotangent of E^{m+1} and u = xbar_P - rho et,
                    //   M00 += u P, M01 += u Q, M10 += xbar_Q P, M11 += xbar_Q Q,
                    //   g0 += u es,  g1 += xbar_Q es
                    const double rho = (double)ie * r;
                    const double es = 2.0 * (double)e0 + rho * delta;
                    const double etr = (double)et * rho;
                    for (int p = 0; p < d.npole; ++p) {
                        const long long o0 = ((long long)(a * d.npole + p) * 2 + 0) * d.bcell + bo;
                        const long long o1 = o0 + d.bcell;
                        const double P = (double)d.ade[o0], Q = (double)d.ade[o1];
                        const double xq = (double)d.aade[o1];
                        const double u = (double)d.aade[o0] - etr;
                        double* pa = pacc + 6 * p;
                        pa[0] += u * P;
                        pa[1] += u * Q;
                        pa[2] += xq * P;
                        pa[3] += xq * Q;
                        pa[4] += u * es;
                        pa[5] += xq * es;
                    }
                }
            }
            fout[a] = S * ie / (T(1) + ie * gdisp) * et;
        }
        A0[id] = fout[0];
        A1[id] = fout[1];
        A2[id] = fout[2];
        tyz_m = tyz;
        txz_m = txz;
    }
}

// kPG: also sums the pole-coefficient cotangents of domains that collect them (Sec. 3.1: pole
// parameters through the transposed dispersion update): per thread over its column, then one
// warp sum and one FP64 atomic per warp and coefficient into the domain's accumulator.
template <typename T, bool kPG>
__global__ void __launch_bounds__(kTileX* kTileY, sizeof(T) == 4 ? 3 : 2)
    k_adj_e_gen(const Dom<T>* __restrict__ doms, const Mon* __restrict__ mons, const Tile* __restrict__ tiles, T S,
                int m, int pending) {
    const Tile t = tiles[blockIdx.x];
    int i, j;
    tile_coords(t, i, j);
    const Dom<T>& d = doms[t.dom];
    if (!kPG) {
        if (i < 0 || j < 0) return;
        adj_e_column(d, mons, i, j, t.z0, t.z1, t.flags, S, m, pending, (double*)nullptr);
        return;
    }
    // every lane of a warp reaches the shuffles below (the domain, hence np, is the block's)
    const int np = d.pgc ? d.npole : 0;
    double acc[kMaxPole * 6];
    for (int q = 0; q < np * 6; ++q) acc[q] = 0.0;
    if (i >= 0 && j >= 0) adj_e_column(d, mons, i, j, t.z0, t.z1, t.flags, S, m, pending, np ? acc : nullptr);
    for (int q = 0; q < np * 6; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(d.pgc + q, v);
    }
}

// Transposed H step of column (i, j) over planes [z0, z1) in general form.
template <typename T>
__device__ __forceinline__ void adj_h_column(const Dom<T>& d, const Mon* __restrict__ mons, int i, int j, int z0,
                                             int z1, int flags, T S, int m) {
    const int nx = d.n[0], ny = d.n[1], nz = d.n[2];
    const long long nxy = (long long)nx * ny;
    const T* A0 = d.A[0];
    const T* A1 = d.A[1];
    const T* A2 = d.A[2];
    T* B0 = d.A[3];
    T* B1 = d.A[4];
    T* B2 = d.A[5];
    bool xe, ye;   // the +x / +y neighbour exists (wraps on a periodic axis)
    const long long oxp = nb_plus(i, nx, 1, d.per[0], &xe);
    const long long oyp = nb_plus(j, ny, nx, d.per[1], &ye);
    const bool pi = i == 0 && !d.per[0], pj = j == 0 && !d.per[1];   // PEC plane at this column
    // H-node coefficients (own psibar_H); E-node coefficients at this column and the +1 one
    const CpmlC<T> xH = cpml_c(d, d.cH[0], 0, i), yH = cpml_c(d, d.cH[1], 1, j);
    const CpmlC<T> xE = cpml_c(d, d.cE[0], 0, i), xEp = cpml_c(d, d.cE[0], 0, i + 1);
    const CpmlC<T> yE = cpml_c(d, d.cE[1], 1, j), yEp = cpml_c(d, d.cE[1], 1, j + 1);
    const bool mon = d.nmon && m >= 1 && (flags & kTileMonH);
    long long id = (long long)z0 * nxy + (long long)j * nx + i;
    // z-derivative terms of E_y (s = 0) and E_x (s = 1) at plane k (carried to the next plane)
    auto zterms = [&](int k, long long idk, T& ty, T& tx) {
        if (k >= nz) {
            ty = T(0);
            tx = T(0);
            return;
        }
        const CpmlC<T> zE = cpml_c(d, d.cE[2], 2, k);
        const long long o = zE.s >= 0 ? off_z(d, zE.s, i, j) : 0;
        // E_y is PEC-held where i == 0 or k == 0; E_x where j == 0 or k == 0
        ty = (pi || k == 0) ? T(0) : dbar_c(zE, A1[idk], zE.s >= 0 ? d.apsiE[1][0][o] : T(0));
        tx = (pj || k == 0) ? T(0) : dbar_c(zE, -A0[idk], zE.s >= 0 ? d.apsiE[0][1][o] : T(0));
    };
    T tyz_k, txz_k;
    zterms(z0, id, tyz_k, txz_k);
    for (int k = z0; k < z1; ++k, id += nxy) {
        T tyz_n, txz_n;
        zterms(k + 1, id + nxy, tyz_n, txz_n);
        const bool pk = k == 0;
        const CpmlC<T> zH = cpml_c(d, d.cH[2], 2, k);
        const T b0 = B0[id], b1 = B1[id], b2 = B2[id];
        const T f0 = A0[id], f1 = A1[id], f2 = A2[id];
        const T f2_xp = xe ? A2[id + oxp] : T(0), f1_xp = xe ? A1[id + oxp] : T(0);
        const T f2_yp = ye ? A2[id + oyp] : T(0), f0_yp = ye ? A0[id + oyp] : T(0);
        // E-derivative cotangents: E_e's s = 0 has ybar = +F, s = 1 has ybar = -F; PEC nodes give 0
        // H_x gathers E_y s=0 (z) and E_z s=1 (y); H_y gathers E_z s=0 (x) and E_x s=1 (z);
        // H_z gathers E_x s=0 (y) and E_y s=1 (x)
        // (a +1 neighbour reached by wrapping lies at coordinate 0 of a periodic axis: no PEC)
        const T tzy = (pi || pj) ? T(0)
                                 : dbar_c(yE, -f2, yE.s >= 0 ? d.apsiE[2][1][off_y(d, yE.s, i, k)] : T(0));
        const T tzy_p = (!ye || pi) ? T(0)
                                    : dbar_c(yEp, -f2_yp, yEp.s >= 0 ? d.apsiE[2][1][off_y(d, yEp.s, i, k)] : T(0));
        const T tzx = (pi || pj) ? T(0)
                                 : dbar_c(xE, f2, xE.s >= 0 ? d.apsiE[2][0][off_x(d, xE.s, j, k)] : T(0));
        const T tzx_p = (!xe || pj) ? T(0)
                                    : dbar_c(xEp, f2_xp, xEp.s >= 0 ? d.apsiE[2][0][off_x(d, xEp.s, j, k)] : T(0));
        const T txy = (pk || pj) ? T(0)
                                 : dbar_c(yE, f0, yE.s >= 0 ? d.apsiE[0][0][off_y(d, yE.s, i, k)] : T(0));
        const T txy_p = (!ye || pk) ? T(0)
                                    : dbar_c(yEp, f0_yp, yEp.s >= 0 ? d.apsiE[0][0][off_y(d, yEp.s, i, k)] : T(0));
        const T tyx = (pk || pi) ? T(0)
                                     : dbar_c(xE, -f1, xE.s >= 0 ? d.apsiE[1][1][off_x(d, xE.s, j, k)] : T(0));
        const T tyx_p = (!xe || pk) ? T(0)
                                    : dbar_c(xEp, -f1_xp, xEp.s >= 0 ? d.apsiE[1][1][off_x(d, xEp.s, j, k)] : T(0));
        (void)f1;
        T h0 = b0 + (tyz_k - tyz_n) + (tzy - tzy_p);
        T h1 = b1 + (tzx - tzx_p) + (txz_k - txz_n);
        T h2 = b2 + (txy - txy_p) + (tyx - tyx_p);
        // finish the H-side CPML transpose of step m (k_adj_e(m) has read psibar_H)
        if (yH.s >= 0) {
            T* p = d.apsiH[0][0] + off_y(d, yH.s, i, k);
            *p = yH.b * (*p - S * b0);
            T* q = d.apsiH[2][1] + off_y(d, yH.s, i, k);
            *q = yH.b * (*q + S * b2);
        }
        if (zH.s >= 0) {
            T* p = d.apsiH[0][1] + off_z(d, zH.s, i, j);
            *p = zH.b * (*p + S * b0);
            T* q = d.apsiH[1][0] + off_z(d, zH.s, i, j);
            *q = zH.b * (*q - S * b1);
        }
        if (xH.s >= 0) {
            T* p = d.apsiH[1][1] + off_x(d, xH.s, j, k);
            *p = xH.b * (*p + S * b1);
            T* q = d.apsiH[2][0] + off_x(d, xH.s, j, k);
            *q = xH.b * (*q - S * b2);
        }
        if (mon) {
            h0 += (T)inject_at(d, mons, 3, i, j, k, (long long)(m - 1) * 2 + 1);
            h1 += (T)inject_at(d, mons, 4, i, j, k, (long long)(m - 1) * 2 + 1);
            h2 += (T)inject_at(d, mons, 5, i, j, k, (long long)(m - 1) * 2 + 1);
        }
        B0[id] = h0;
        B1[id] = h1;
        B2[id] = h2;
        tyz_k = tyz_n;
        txz_k = txz_n;
    }
}

template <typename T>
__global__ void __launch_bounds__(kTileX* kTileY, sizeof(T) == 4 ? 3 : 2)
    k_adj_h_gen(const Dom<T>* __restrict__ doms, const Mon* __restrict__ mons, const Tile* __restrict__ tiles, T S,
                int m) {
    const Tile t = tiles[blockIdx.x];
    int i, j;
    tile_coords(t, i, j);
    if (i < 0 || j < 0) return;
    adj_h_column(doms[t.dom], mons, i, j, t.z0, t.z1, t.flags, S, m);
}

// Interior fast paths of the two transposed kernels: tiles that touch no CPML slab, PEC plane,
// domain edge or pole cell.  Without CPML the derivative cotangents reduce to -S Hbar / +S Hbar
// and +F / -F, so k_adj_e_int is the forward E update with Ebar -= S C^- Hbar and
// k_adj_h_int is Hbar += C^+ F.  Loads of a plane are issued before its stores; the z-1
// (z+1) neighbours are carried in registers.  The design-box gradient and the monitor
// injection keep their per-cell checks.
// Interior transposed kernels: bounded so that 4 (FP32) / 3 (FP64) blocks of 256 threads fit an
// SM; left unbounded they take ~140 registers (one block per SM) and starve the memory system.
#ifndef GBFDTD_ADJ_INT_BLOCKS_F32
#define GBFDTD_ADJ_INT_BLOCKS_F32 4
#endif
template <typename T>
constexpr int adj_int_blocks() {
    return sizeof(T) == 4 ? GBFDTD_ADJ_INT_BLOCKS_F32 : 3;
}

template <typename T, bool kAniso>
__global__ void __launch_bounds__(kTileX* kTileY, adj_int_blocks<T>()) k_adj_e_int(const Dom<T>* __restrict__ doms,
                                                              const Mon* __restrict__ mons,
                                                              const Tile* __restrict__ tiles, T S, int m,
                                                              int pending) {
    const Tile t = tiles[blockIdx.x];
    const Dom<T>& d = doms[t.dom];
    const int nx = d.n[0], ny = d.n[1];
    int i, j;
    tile_coords(t, i, j);
    if (i < 0 || j < 0) return;
    const long long nxy = (long long)nx * ny;
    T* Fx = d.A[0];
    T* Fy = d.A[1];
    T* Fz = d.A[2];
    const T* Bx = d.A[3];
    const T* By = d.A[4];
    const T* Bz = d.A[5];
    const T* ie0 = d.ie[0];
    const T* ie1 = d.ie[1];
    const T* ie2 = d.ie[2];
    const bool gcol = d.design && i >= d.glo[0] && i < d.ghi[0] && j >= d.glo[1] && j < d.ghi[1];
    long long id = (long long)t.z0 * nxy + (long long)j * nx + i;
    T bxz = Bx[id - nxy], byz = By[id - nxy];
    for (int k = t.z0; k < t.z1; ++k, id += nxy) {
        const T bx = Bx[id], by = By[id], bz = Bz[id];
        const T bz_ym = Bz[id - nx], bx_ym = Bx[id - nx];
        const T bz_xm = Bz[id - 1], by_xm = By[id - 1];
        const T fx = Fx[id], fy = Fy[id], fz = Fz[id];
        const T iex = ie0[id];
        const T iey = kAniso ? ie1[id] : iex;
        const T iez = kAniso ? ie2[id] : iex;
        // deferred own-cell transpose of step m+1 (non-dispersive: Ebar = F / (S eps^-1))
        T ex = pending ? fx / (S * iex) : fx;
        T ey = pending ? fy / (S * iey) : fy;
        T ez = pending ? fz / (S * iez) : fz;
        // transpose of the H update: Ebar -= S C^- Hbar
        ex += S * ((by - byz) - (bz - bz_ym));
        ey += S * ((bz - bz_xm) - (bx - bxz));
        ez += S * ((bx - bx_ym) - (by - by_xm));
        bxz = bx;
        byz = by;
        if (d.nmon && (t.flags & kTileMonE)) {
            ex += (T)inject_at(d, mons, 0, i, j, k, (long long)m * 2 + 0);
            ey += (T)inject_at(d, mons, 1, i, j, k, (long long)m * 2 + 0);
            ez += (T)inject_at(d, mons, 2, i, j, k, (long long)m * 2 + 0);
        }
        if (gcol && k >= d.glo[2] && k < d.ghi[2]) {
            // d E^{m+1} / d(eps^-1) = S curl(H^{m+1/2}) of the forward state u^m
            const T* Hx = d.F[3];
            const T* Hy = d.F[4];
            const T* Hz = d.F[5];
            const T cx = (Hz[id] - Hz[id - nx]) - (Hy[id] - Hy[id - nxy]);
            const T cy = (Hx[id] - Hx[id - nxy]) - (Hz[id] - Hz[id - 1]);
            const T cz = (Hy[id] - Hy[id - 1]) - (Hx[id] - Hx[id - nx]);
            const long long gi = ((long long)(k - d.glo[2]) * (d.ghi[1] - d.glo[1]) + (j - d.glo[1])) *
                                     (d.ghi[0] - d.glo[0]) + (i - d.glo[0]);
            const long long gn = (long long)(d.ghi[0] - d.glo[0]) * (d.ghi[1] - d.glo[1]) * (d.ghi[2] - d.glo[2]);
            d.grad[gi] += (double)ex * (double)(S * cx);
            d.grad[gn + gi] += (double)ey * (double)(S * cy);
            d.grad[2 * gn + gi] += (double)ez * (double)(S * cz);
        }
        Fx[id] = S * iex * ex;
        Fy[id] = S * iey * ey;
        Fz[id] = S * iez * ez;
    }
}

template <typename T>
__global__ void __launch_bounds__(kTileX* kTileY, adj_int_blocks<T>()) k_adj_h_int(const Dom<T>* __restrict__ doms,
                                                              const Mon* __restrict__ mons,
                                                              const Tile* __restrict__ tiles, T S, int m) {
    const Tile t = tiles[blockIdx.x];
    const Dom<T>& d = doms[t.dom];
    const int nx = d.n[0], ny = d.n[1];
    int i, j;
    tile_coords(t, i, j);
    if (i < 0 || j < 0) return;
    const long long nxy = (long long)nx * ny;
    const T* Fx = d.A[0];
    const T* Fy = d.A[1];
    const T* Fz = d.A[2];
    T* Bx = d.A[3];
    T* By = d.A[4];
    T* Bz = d.A[5];
    long long id = (long long)t.z0 * nxy + (long long)j * nx + i;
    T fxk = Fx[id], fyk = Fy[id];
    for (int k = t.z0; k < t.z1; ++k, id += nxy) {
        const T fxn = Fx[id + nxy], fyn = Fy[id + nxy];
        const T fz = Fz[id];
        const T fz_yp = Fz[id + nx], fz_xp = Fz[id + 1];
        const T fy_xp = Fy[id + 1], fx_yp = Fx[id + nx];
        T bx = Bx[id], by = By[id], bz = Bz[id];
        // transpose of the E update: Hbar += C^+ F
        bx += (fz_yp - fz) - (fyn - fyk);
        by += (fxn - fxk) - (fz_xp - fz);
        bz += (fy_xp - fyk) - (fx_yp - fxk);
        if (d.nmon && m >= 1 && (t.flags & kTileMonH)) {
            bx += (T)inject_at(d, mons, 3, i, j, k, (long long)(m - 1) * 2 + 1);
            by += (T)inject_at(d, mons, 4, i, j, k, (long long)(m - 1) * 2 + 1);
            bz += (T)inject_at(d, mons, 5, i, j, k, (long long)(m - 1) * 2 + 1);
        }
        Bx[id] = bx;
        By[id] = by;
        Bz[id] = bz;
        fxk = fxn;
        fyk = fyn;
    }
}

template <typename T>
__global__ void __launch_bounds__(kTileX* kTileY) k_adj_flush(const Dom<T>* __restrict__ doms,
                                                              const Tile* __restrict__ tiles, T S) {
    const Tile t = tiles[blockIdx.x];
    const Dom<T>& d = doms[t.dom];
    int i, j;
    tile_coords(t, i, j);
    if (i < 0 || j < 0) return;
    for (int k = t.z0; k < t.z1; ++k) {
        const int c[3] = {i, j, k};
        const long long id = cidx(d.n, i, j, k);
        const bool dcell = d.npole > 0 && d.mask[id] && in_ade_box(d, i, j, k);
        for (int a = 0; a < 3; ++a) {
            const int b = (a + 1) % 3, q = (a + 2) % 3;
            if ((c[b] == 0 && !d.per[b]) || (c[q] == 0 && !d.per[q])) continue;   // PEC-held
            d.A[a][id] = e_deferred(d, a, i, j, k, id, dcell, d.A[a][id], S);
        }
    }
}

// Standalone injection of dJ/df(t) into the adjoint fields (used to start a sweep).
template <typename T>
__global__ void k_inject(const Dom<T>* __restrict__ doms, const Mon* __restrict__ mons,
                         const int* __restrict__ entries, int nentries, long long nthreads,
                         const long long* __restrict__ entry_begin, int step, int kind) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nthreads) return;
    int e = 0;
    while (e + 1 < nentries && entry_begin[e + 1] <= t) ++e;
    const int mi = entries[2 * e], ci = entries[2 * e + 1];
    const Mon& m = mons[mi];
    if (!m.cot) return;
    const long long cell = t - entry_begin[e];
    const int i = m.lo[0] + (int)(cell % m.bx);
    const int j = m.lo[1] + (int)((cell / m.bx) % m.by);
    const int k = m.lo[2] + (int)(cell / ((long long)m.bx * m.by));
    const Dom<T>& d = doms[m.dom];
    const double2* ph = m.phase + ((long long)step * 2 + kind) * m.nf;
    const double2* ct = m.cot + (long long)ci * m.nf * m.ncell + cell;
    double acc = 0.0;
    for (int f = 0; f < m.nf; ++f) {
        const double2 c = ct[(long long)f * m.ncell];
        acc += c.x * ph[f].x + c.y * ph[f].y;
    }
    d.A[m.comps[ci]][cidx(d.n, i, j, k)] += (T)acc;
}

// Injection values of one half-step over a box of cells (see launch_inject_box): the sum over the
// domain's monitors of inject_at, rounded to T once, exactly the value the per-cell kernels add.
template <typename T>
__global__ void k_inject_box(const Dom<T>* __restrict__ dom, const Mon* __restrict__ mons, int3 lo, int3 hi,
                             long long pidx_e, long long pidx_h, T* __restrict__ inj) {
    const long long bx = hi.x - lo.x, by = hi.y - lo.y, vol = bx * by * (hi.z - lo.z);
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= vol) return;
    const int i = lo.x + (int)(t % bx), j = lo.y + (int)((t / bx) % by), k = lo.z + (int)(t / (bx * by));
    for (int c = 0; c < 3; ++c) inj[c * vol + t] = (T)inject_at(*dom, mons, c, i, j, k, pidx_e);
    if (pidx_h >= 0)
        for (int c = 3; c < 6; ++c) inj[c * vol + t] = (T)inject_at(*dom, mons, c, i, j, k, pidx_h);
}

// ---- per-cell transposed kernels -------------------------------------------------------------------
// One thread per cell over the forward per-cell grid (x chunks of 32, y chunks of 8, z planes), so a
// warp reads 128 contiguous bytes per array and every load of a thread is independent (the -1 / +1
// neighbours come from L1 / L2).  The domain's operands arrive by value.  The algebra is that of
// adj_e_column / adj_h_column: a gathered derivative cotangent is Dbar = ybar outside the CPML slabs
// and ybar / kappa + c (psibar + ybar) in them, so a cell whose gather meets no slab node takes the
// short form (differences of the cotangent fields scaled by S), decided per cell: warps diverge
// only where a slab edge crosses them.  Poles, the material cotangent and monitor injection are
// compiled in only where a domain needs them; pole-parameter cotangents keep the tile kernels.
#ifndef GBFDTD_ADJ_CELL_BLOCKS_F32
#define GBFDTD_ADJ_CELL_BLOCKS_F32 8
#endif
template <typename T, bool kHeavy>
constexpr int adj_cell_blocks() {
    return sizeof(T) == 4 ? (kHeavy ? 4 : GBFDTD_ADJ_CELL_BLOCKS_F32) : 3;
}

// Offset of cell (i, j, k) in the slab array of axis q at slab index s, written so that the part
// depending only on the block's plane k (block-uniform) is computed in 64 bits once and the in-plane
// part in 32 bits.
__device__ __forceinline__ int slab_off_c(const int* n, const int* ns, int q, int i, int j, int k, int s) {
    if (q == 0) return k * (n[1] * ns[0]) + (j * ns[0] + s);
    if (q == 1) return k * (ns[1] * n[0]) + (s * n[0] + i);
    return s * (n[0] * n[1]) + (j * n[0] + i);
}

// Dbar of a derivative at node (i, j, k) whose coordinate along axis q is x and slab index sl
// (-1 outside the slabs): coef is the axis' CPML row [b | c | 1/kappa], psi its memory cotangents.
template <typename T>
__device__ __forceinline__ T dbar_node(const T* coef, int N, const T* psi, const int* n, const int* ns, int q, int i,
                                       int j, int k, int x, int sl, T yb) {
    if (sl < 0) return yb;
    const T ps = psi[slab_off_c(n, ns, q, i, j, k, sl)];
    return coef[2 * N + x] * yb + coef[N + x] * (ps + yb);
}

__device__ __forceinline__ bool in_box3(const int* lo, const int* hi, int i, int j, int k) {
    return i >= lo[0] && i < hi[0] && j >= lo[1] && j < hi[1] && k >= lo[2] && k < hi[2];
}

// Offset of cell (i, j, k) inside the box [lo, hi), x fastest.
__device__ __forceinline__ long long box_cell(const int* lo, const int* hi, int i, int j, int k) {
    return ((long long)(k - lo[2]) * (hi[1] - lo[1]) + (j - lo[1])) * (hi[0] - lo[0]) + (i - lo[0]);
}

// 1 / x: a correctly rounded reciprocal in FP32 (a multiply by it replaces the IEEE division of
// the deferred own-cell part), the exact quotient in FP64.
__device__ __forceinline__ float recip_t(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip_t(double x) { return 1.0 / x; }

// Slab index of coordinate x along an axis with CPML depths (lo, hi) over N nodes, or -1; an axis
// without CPML (ns = 0) has none.
__device__ __forceinline__ int slab_or_none(int x, int lo, int hi, int N, int ns) {
    return ns ? slab_of(x, lo, hi, N) : -1;
}

// One E component a of the transposed E step at cell (i, j, k) (offset id of the whole array):
// completes the deferred own-cell transpose of step m+1 (pending), adds the gathered cotangent gat
// and the monitor injection, accumulates the material (and pole-coefficient) cotangents, and
// returns the new lagged value S eps^-1 / (1 + eps^-1 G) Ebar.  om: offsets to the -1 neighbours.
// kTen (a tensor domain, Sec. 2.3): Ebar of step m+1 is kept in c.Eb (the pending part only advances
// the psibar_E with F, the curl cotangent the apply kernel left in the E array) and the return value
// is Ebar itself, which the caller stores into c.Eb.
template <typename T, int a, bool kPoles, bool kGrad, bool kMon, bool kPG, bool kTen = false>
__device__ __forceinline__ T adj_e_comp(const AdjCellArgs<T>& c, const Dom<T>* __restrict__ doms,
                                        const Mon* __restrict__ mons, int i, int j, int k, long long id, T F, T ie,
                                        T gat, T S, int m, int pending, bool disp, long long bo, const int* sl,
                                        const long long* om, double* pacc) {
    constexpr int q0 = (a + 1) % 3, q1 = (a + 2) % 3;
    const int x[3] = {i, j, k + c.kz0};   // coefficient rows are indexed by global coordinates
    T eb;
    if (pending) {
        if (kTen) {
            eb = c.Eb[a][id];
        } else if (kPoles && disp) {
            const Dom<T>& d = doms[c.dom];
            eb = (T(1) / ie - d.G) / S * F;
            for (int p = 0; p < d.npole; ++p) {
                T* pp = d.aade + ((long long)(a * d.npole + p) * 2 + 0) * d.bcell + bo;
                T* pq = pp + d.bcell;
                const T xp = *pp, xq = *pq;
                eb += d.g0[p] * xp + d.g1[p] * xq;
                *pp = d.M00[p] * xp + d.M10[p] * xq + (T(1) - d.M00[p]) / S * F;
                *pq = d.M01[p] * xp + d.M11[p] * xq - d.M01[p] / S * F;
            }
        } else {
            eb = F * recip_t(S * ie);
        }
        // own psibar_E of E_a's two derivatives: s = 0 along q0 (ybar = +F), s = 1 along q1 (-F)
        if (sl[q0] >= 0) {
            T* p = c.apsiE[a][0] + slab_off_c(c.n, c.ns, q0, i, j, k, sl[q0]);
            *p = c.cE[q0][x[q0]] * (*p + F);
        }
        if (sl[q1] >= 0) {
            T* p = c.apsiE[a][1] + slab_off_c(c.n, c.ns, q1, i, j, k, sl[q1]);
            *p = c.cE[q1][x[q1]] * (*p - F);
        }
    } else {
        eb = F;
    }
    eb += gat;
    if (kMon && in_box3(c.mlo, c.mhi, i, j, k + c.kz0)) eb += c.inj[a * c.mvol + box_cell(c.mlo, c.mhi, i, j, k + c.kz0)];
    T et = eb, gdisp = T(0);
    if (kPoles && disp) {
        const Dom<T>& d = doms[c.dom];
        for (int p = 0; p < d.npole; ++p) {
            const T* pp = d.aade + ((long long)(a * d.npole + p) * 2 + 0) * d.bcell + bo;
            et += d.g0[p] * pp[0] + d.g1[p] * pp[d.bcell];
        }
        gdisp = d.G;
    }
    const bool gcell = kGrad && in_box3(c.glo, c.ghi, i, j, k);
    const bool pcell = kPG && disp;
    if (gcell || pcell) {
        // d E^{m+1} / d(eps^-1): S curl(H^{m+1/2}) of the forward state u^m (plus the pole terms);
        // the design and pole boxes lie outside the CPML slabs, so the forward update used the
        // plain curl
        const T* Hq = c.F[3 + q1];
        const T* Hb = c.F[3 + q0];
        const T curl = (Hq[id] - Hq[id + om[q0]]) - (Hb[id] - Hb[id + om[q1]]);
        double delta = (double)(S * curl);
        const T e0 = c.F[a][id];
        if (kPoles && disp) {
            const Dom<T>& d = doms[c.dom];
            for (int p = 0; p < d.npole; ++p) {
                const T P = d.ade[((long long)(a * d.npole + p) * 2 + 0) * d.bcell + bo];
                const T Q = d.ade[((long long)(a * d.npole + p) * 2 + 1) * d.bcell + bo];
                delta += (double)(P - (d.M00[p] * P + d.M01[p] * Q) - T(2) * d.g0[p] * e0);
            }
        }
        const double r = 1.0 / (1.0 + (double)ie * (double)gdisp);
        if (gcell) {
            const long long gi = ((long long)(k + c.kz0 - c.gzg) * (c.ghi[1] - c.glo[1]) + (j - c.glo[1])) *
                                     (c.ghi[0] - c.glo[0]) + (i - c.glo[0]);
            c.grad[a * c.gvol + gi] += (double)et * delta * r * r;
        }
        if (pcell) {
            // pole-coefficient cotangents (the algebra of adj_e_column): with u = xbar_P - rho et,
            //   M00 += u P, M01 += u Q, M10 += xbar_Q P, M11 += xbar_Q Q, g0 += u es, g1 += xbar_Q es
            const Dom<T>& d = doms[c.dom];
            const double rho = (double)ie * r;
            const double es = 2.0 * (double)e0 + rho * delta;
            const double etr = (double)et * rho;
            for (int p = 0; p < d.npole; ++p) {
                const long long o0 = ((long long)(a * d.npole + p) * 2 + 0) * d.bcell + bo;
                const long long o1 = o0 + d.bcell;
                const double P = (double)d.ade[o0], Q = (double)d.ade[o1];
                const double xq = (double)d.aade[o1];
                const double u = (double)d.aade[o0] - etr;
                double* pa = pacc + 6 * p;
                pa[0] += u * P;
                pa[1] += u * Q;
                pa[2] += xq * P;
                pa[3] += xq * Q;
                pa[4] += u * es;
                pa[5] += xq * es;
            }
        }
    }
    if (kTen) return et;
    if (kPoles && disp) return S * ie / (T(1) + ie * gdisp) * et;
    return S * ie * et;
}

// kPG (with kPoles): also sums the pole-coefficient cotangents of the domain (Sec. 3.1: pole parameters
// through the transposed dispersion update): per thread, then one warp sum, a block sum in shared
// memory and one FP64 atomic per block and coefficient into the domain's accumulator.
template <typename T, bool kPoles, bool kGrad, bool kMon, bool kPG, bool kTen>
__device__ __forceinline__ void adj_e_cell_body(const AdjCellArgs<T>& c, const Dom<T>* __restrict__ doms,
                                                const Mon* __restrict__ mons, T S, int m, int pending, double* pacc) {
    const int nx = c.n[0], ny = c.n[1], nz = c.n[2];
    // a warp covers 16 x 2 cells (two half-rows of 64 / 128 aligned bytes): a row's x slabs fill two
    // of its warps instead of half of them
    const int i = blockIdx.x * 16 + (threadIdx.x & 15), j = blockIdx.y * 16 + threadIdx.y * 2 + (threadIdx.x >> 4);
    const int k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const int kg = k + c.kz0;   // global plane (CPML z profile, monitors, plain ranges)
    const long long nxy = (long long)nx * ny;
    const long long pl = (long long)k * nxy;   // first cell of this z-plane (block-uniform)
    const int ij = j * nx + i;                  // offset inside the plane
    // -1 neighbours (wrapping on a periodic axis); in-plane offsets in 32 bits
    const bool hx_ = i > 0 || c.per[0], hy_ = j > 0 || c.per[1], hz_ = k > 0;
    const int ox = i > 0 ? -1 : nx - 1, oy = j > 0 ? -nx : (ny - 1) * nx;
    pdl_wait();
    pdl_trigger();
    const T* Bx = c.A[3] + pl;
    const T* By = c.A[4] + pl;
    const T* Bz = c.A[5] + pl;
    const T bx = Bx[ij], by = By[ij], bz = Bz[ij];
    const T by_zm = hz_ ? (By - nxy)[ij] : T(0), bx_zm = hz_ ? (Bx - nxy)[ij] : T(0);
    const T bz_ym = hy_ ? Bz[ij + oy] : T(0), bx_ym = hy_ ? Bx[ij + oy] : T(0);
    const T bz_xm = hx_ ? Bz[ij + ox] : T(0), by_xm = hx_ ? By[ij + ox] : T(0);
    const T f0 = (c.A[0] + pl)[ij], f1 = (c.A[1] + pl)[ij], f2 = (c.A[2] + pl)[ij];
    const bool aniso = c.ie[1] != c.ie[0];
    const T ie0 = kTen ? T(1) : (c.ie[0] + pl)[ij];
    const T ie1 = kTen ? T(1) : (aniso ? (c.ie[1] + pl)[ij] : ie0);
    const T ie2 = kTen ? T(1) : (aniso ? (c.ie[2] + pl)[ij] : ie0);
    // where the new E cotangents go: the lagged form into the E array, a tensor domain's Ebar into Eb
    T* const E0 = kTen ? c.Eb[0] : c.A[0];
    T* const E1 = kTen ? c.Eb[1] : c.A[1];
    T* const E2 = kTen ? c.Eb[2] : c.A[2];
    const bool pi = i == 0 && !c.per[0], pj = j == 0 && !c.per[1], pk = k == 0;
    const long long id = pl + ij;
    const long long om[3] = {ox, oy, -nxy};
    bool disp = false;
    long long bo = 0;
    if (kPoles) {
        const Dom<T>& d = doms[c.dom];
        disp = d.npole > 0 && in_ade_box(d, i, j, k) && d.mask[pl + ij];
        if (disp) bo = ade_off(d, i, j, k);
    }
    // a warp (one x row of one plane) whose cells all gather no slab node takes the plain form: the
    // derivative cotangents are S times differences of the H cotangent, and no psibar is touched
    const unsigned am = __activemask();
    const bool plain = (unsigned)(i - c.elo[0]) < (unsigned)(c.ehi[0] - c.elo[0]) &&
                       (unsigned)(j - c.elo[1]) < (unsigned)(c.ehi[1] - c.elo[1]) &&
                       (unsigned)(kg - c.elo[2]) < (unsigned)(c.ehi[2] - c.elo[2]);
    if (__all_sync(am, plain)) {
        const int none[3] = {-1, -1, -1};
        const T g0 = S * ((by - by_zm) - (bz - bz_ym));
        const T g1 = S * ((bz - bz_xm) - (bx - bx_zm));
        const T g2 = S * ((bx - bx_ym) - (by - by_xm));
        if (!(pj || pk))
            (E0 + pl)[ij] = adj_e_comp<T, 0, kPoles, kGrad, kMon, kPG, kTen>(c, doms, mons, i, j, k, id, f0, ie0, g0, S,
                                                                          m, pending, disp, bo, none, om, pacc);
        if (!(pi || pk))
            (E1 + pl)[ij] = adj_e_comp<T, 1, kPoles, kGrad, kMon, kPG, kTen>(c, doms, mons, i, j, k, id, f1, ie1, g1, S,
                                                                          m, pending, disp, bo, none, om, pacc);
        if (!(pi || pj))
            (E2 + pl)[ij] = adj_e_comp<T, 2, kPoles, kGrad, kMon, kPG, kTen>(c, doms, mons, i, j, k, id, f2, ie2, g2, S,
                                                                          m, pending, disp, bo, none, om, pacc);
        return;
    }
    // slab index of this node along each axis (-1: outside the slabs); the -1 node lies in a slab
    // only where this node is the first one past the low slab
    const int sl[3] = {slab_or_none(i, c.dlo[0], c.dhi[0], nx, c.ns[0]), slab_or_none(j, c.dlo[1], c.dhi[1], ny, c.ns[1]),
                       slab_or_none(kg, c.dlo[2], c.dhi[2], c.nzg, c.ns[2])};
    // per axis, decided for the whole warp: a warp with any lane near a slab of that axis takes the
    // general form, whose per-lane slab checks give the plain values elsewhere
    const bool px_plain = __all_sync(am, sl[0] < 0 && !(i > 0 && i == c.dlo[0]));
    const bool py_plain = __all_sync(am, sl[1] < 0 && !(j > 0 && j == c.dlo[1]));
    const bool pz_plain = __all_sync(am, sl[2] < 0 && !(k > 0 && kg == c.dlo[2]));
    // gathered transposes of the H update's derivatives: the q-derivative of H_c has ybar = -S Hbar_c
    // for s = 0 of H_c and +S Hbar_c for s = 1; E_a gathers its two curl terms at this node and at
    // -1.  Per axis, without a slab node among the two the Dbar are the ybar themselves.
    T g0, g1, g2;
    // z: H_y (s = 0) into E_x, H_x (s = 1) into E_y
    if (pz_plain) {
        g0 = S * (by - by_zm);
        g1 = -(S * (bx - bx_zm));
    } else {
        const int szm = k > 0 ? slab_or_none(kg - 1, c.dlo[2], c.dhi[2], c.nzg, c.ns[2]) : -1;
        const T tyz = dbar_node(c.cH[2], c.nzg, c.apsiH[1][0], c.n, c.ns, 2, i, j, k, kg, sl[2], -S * by);
        const T tyz_m = hz_ ? dbar_node(c.cH[2], c.nzg, c.apsiH[1][0], c.n, c.ns, 2, i, j, k - 1, kg - 1, szm, -S * by_zm) : T(0);
        const T txz = dbar_node(c.cH[2], c.nzg, c.apsiH[0][1], c.n, c.ns, 2, i, j, k, kg, sl[2], S * bx);
        const T txz_m = hz_ ? dbar_node(c.cH[2], c.nzg, c.apsiH[0][1], c.n, c.ns, 2, i, j, k - 1, kg - 1, szm, S * bx_zm) : T(0);
        g0 = tyz_m - tyz;
        g1 = txz_m - txz;
    }
    // y: H_z (s = 1) into E_x, H_x (s = 0) into E_z
    if (py_plain) {
        g0 -= S * (bz - bz_ym);
        g2 = S * (bx - bx_ym);
    } else {
        const int sym = j > 0 ? slab_or_none(j - 1, c.dlo[1], c.dhi[1], ny, c.ns[1]) : -1;
        const T tzy = dbar_node(c.cH[1], c.n[1], c.apsiH[2][1], c.n, c.ns, 1, i, j, k, j, sl[1], S * bz);
        const T tzy_m = hy_ ? dbar_node(c.cH[1], c.n[1], c.apsiH[2][1], c.n, c.ns, 1, i, j - 1, k, j - 1, sym, S * bz_ym) : T(0);
        const T txy = dbar_node(c.cH[1], c.n[1], c.apsiH[0][0], c.n, c.ns, 1, i, j, k, j, sl[1], -S * bx);
        const T txy_m = hy_ ? dbar_node(c.cH[1], c.n[1], c.apsiH[0][0], c.n, c.ns, 1, i, j - 1, k, j - 1, sym, -S * bx_ym) : T(0);
        g0 += tzy_m - tzy;
        g2 = txy_m - txy;
    }
    // x: H_z (s = 0) into E_y, H_y (s = 1) into E_z
    if (px_plain) {
        g1 += S * (bz - bz_xm);
        g2 -= S * (by - by_xm);
    } else {
        const int sxm = i > 0 ? slab_or_none(i - 1, c.dlo[0], c.dhi[0], nx, c.ns[0]) : -1;
        const T tzx = dbar_node(c.cH[0], c.n[0], c.apsiH[2][0], c.n, c.ns, 0, i, j, k, i, sl[0], -S * bz);
        const T tzx_m = hx_ ? dbar_node(c.cH[0], c.n[0], c.apsiH[2][0], c.n, c.ns, 0, i - 1, j, k, i - 1, sxm, -S * bz_xm) : T(0);
        const T tyx = dbar_node(c.cH[0], c.n[0], c.apsiH[1][1], c.n, c.ns, 0, i, j, k, i, sl[0], S * by);
        const T tyx_m = hx_ ? dbar_node(c.cH[0], c.n[0], c.apsiH[1][1], c.n, c.ns, 0, i - 1, j, k, i - 1, sxm, S * by_xm) : T(0);
        g1 += tzx_m - tzx;
        g2 += tyx_m - tyx;
    }
    // tangential E on a PEC plane (coordinate 0 of a non-periodic axis other than its own) is held
    if (!(pj || pk))
        (E0 + pl)[ij] = adj_e_comp<T, 0, kPoles, kGrad, kMon, kPG, kTen>(c, doms, mons, i, j, k, id, f0, ie0, g0, S, m,
                                                                      pending, disp, bo, sl, om, pacc);
    if (!(pi || pk))
        (E1 + pl)[ij] = adj_e_comp<T, 1, kPoles, kGrad, kMon, kPG, kTen>(c, doms, mons, i, j, k, id, f1, ie1, g1, S, m,
                                                                      pending, disp, bo, sl, om, pacc);
    if (!(pi || pj))
        (E2 + pl)[ij] = adj_e_comp<T, 2, kPoles, kGrad, kMon, kPG, kTen>(c, doms, mons, i, j, k, id, f2, ie2, g2, S, m,
                                                                      pending, disp, bo, sl, om, pacc);
}

template <typename T, bool kPoles, bool kGrad, bool kMon, bool kPG, bool kTen = false>
__global__ void __launch_bounds__(kTileX* kTileY, adj_cell_blocks<T, kPoles || kGrad>())
    k_adj_e_cell(const AdjCellArgs<T> c, const Dom<T>* __restrict__ doms, const Mon* __restrict__ mons, T S, int m,
                 int pending) {
    if (!kPG) {
        adj_e_cell_body<T, kPoles, kGrad, kMon, false, kTen>(c, doms, mons, S, m, pending, nullptr);
        return;
    }
    const Dom<T>& d = doms[c.dom];
    const int np = d.pgc ? d.npole : 0;
    // a block of 16 x 16 cells of one plane that meets no pole-box cell has no pole-coefficient
    // cotangent to add (a block-uniform test): it runs the plain body and skips the reductions
    {
        const int i0 = blockIdx.x * 16, j0 = blockIdx.y * 16, k = blockIdx.z;
        const bool meets = np > 0 && i0 < d.bhi[0] && i0 + 16 > d.blo[0] && j0 < d.bhi[1] && j0 + 16 > d.blo[1] &&
                           k >= d.blo[2] && k < d.bhi[2];
        if (!meets) {
            adj_e_cell_body<T, kPoles, kGrad, kMon, false, kTen>(c, doms, mons, S, m, pending, nullptr);
            return;
        }
    }
    // every thread of the block reaches the reductions below (the domain, hence np, is the launch's)
    double acc[kMaxPole * 6];
    for (int q = 0; q < np * 6; ++q) acc[q] = 0.0;
    adj_e_cell_body<T, kPoles, kGrad, kMon, true, false>(c, doms, mons, S, m, pending, acc);
    __shared__ double red[kTileX * kTileY / 32];
    const int tid = threadIdx.y * kTileX + threadIdx.x;
    for (int q = 0; q < np * 6; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) red[tid >> 5] = v;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < kTileX * kTileY / 32; ++w) t += red[w];
            if (t != 0.0) atomicAdd(d.pgc + q, t);
        }
        __syncthreads();
    }
}

template <typename T, bool kMon>
__global__ void __launch_bounds__(kTileX* kTileY, adj_cell_blocks<T, false>())
    k_adj_h_cell(const AdjCellArgs<T> c, const Dom<T>* __restrict__ doms, const Mon* __restrict__ mons, T S, int m) {
    const int nx = c.n[0], ny = c.n[1], nz = c.n[2];
    const int i = blockIdx.x * 16 + (threadIdx.x & 15), j = blockIdx.y * 16 + threadIdx.y * 2 + (threadIdx.x >> 4);
    const int k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const int kg = k + c.kz0;   // global plane (CPML z profile, monitors, plain ranges)
    const long long nxy = (long long)nx * ny;
    const long long pl = (long long)k * nxy;   // first cell of this z-plane (block-uniform)
    const int ij = j * nx + i;
    // +1 neighbours (wrapping on a periodic axis)
    const bool xe = i + 1 < nx || c.per[0], ye = j + 1 < ny || c.per[1], ze = k + 1 < nz;
    const int ox = i + 1 < nx ? 1 : -(nx - 1), oy = j + 1 < ny ? nx : -(ny - 1) * nx;
    pdl_wait();
    pdl_trigger();
    const T* Fx = c.A[0] + pl;
    const T* Fy = c.A[1] + pl;
    const T* Fz = c.A[2] + pl;
    const T fx = Fx[ij], fy = Fy[ij], fz = Fz[ij];
    const T fy_zp = ze ? (Fy + nxy)[ij] : T(0), fx_zp = ze ? (Fx + nxy)[ij] : T(0);
    const T fz_yp = ye ? Fz[ij + oy] : T(0), fx_yp = ye ? Fx[ij + oy] : T(0);
    const T fz_xp = xe ? Fz[ij + ox] : T(0), fy_xp = xe ? Fy[ij + ox] : T(0);
    T* B0 = c.A[3] + pl;
    T* B1 = c.A[4] + pl;
    T* B2 = c.A[5] + pl;
    const T b0 = B0[ij], b1 = B1[ij], b2 = B2[ij];
    // a warp whose cells all gather no slab node and no PEC-held node takes the plain form
    const unsigned am = __activemask();
    const bool plain = (unsigned)(i - c.hlo[0]) < (unsigned)(c.hhi[0] - c.hlo[0]) &&
                       (unsigned)(j - c.hlo[1]) < (unsigned)(c.hhi[1] - c.hlo[1]) &&
                       (unsigned)(kg - c.hlo[2]) < (unsigned)(c.hhi[2] - c.hlo[2]) && k > 0;
    if (__all_sync(am, plain)) {
        T h0 = b0 + (fy - fy_zp) + (fz_yp - fz);
        T h1 = b1 + (fz - fz_xp) + (fx_zp - fx);
        T h2 = b2 + (fx - fx_yp) + (fy_xp - fy);
        if (kMon && m >= 1 && in_box3(c.mlo, c.mhi, i, j, kg)) {
            const long long bo = box_cell(c.mlo, c.mhi, i, j, kg);
            h0 += c.inj[bo];
            h1 += c.inj[c.mvol + bo];
            h2 += c.inj[2 * c.mvol + bo];
        }
        B0[ij] = h0;
        B1[ij] = h1;
        B2[ij] = h2;
        return;
    }
    const bool pi = i == 0 && !c.per[0], pj = j == 0 && !c.per[1], pk = k == 0;
    const bool edge = pi || pj || pk;
    // slab index of this node along each axis; the +1 node lies in a slab only where this node is
    // the last one before the high slab
    const int sx = slab_or_none(i, c.dlo[0], c.dhi[0], nx, c.ns[0]);
    const int sy = slab_or_none(j, c.dlo[1], c.dhi[1], ny, c.ns[1]);
    const int sz = slab_or_none(kg, c.dlo[2], c.dhi[2], c.nzg, c.ns[2]);
    // per axis, decided for the whole warp (see k_adj_e_cell)
    const bool px_plain = __all_sync(am, !edge && sx < 0 && !(c.dhi[0] > 0 && i + 1 == nx - c.dhi[0]));
    const bool py_plain = __all_sync(am, !edge && sy < 0 && !(c.dhi[1] > 0 && j + 1 == ny - c.dhi[1]));
    const bool pz_plain = __all_sync(am, !edge && sz < 0 && !(c.dhi[2] > 0 && kg + 1 == c.nzg - c.dhi[2]));
    // transposes of the E update's derivatives: E_e's s = 0 derivative has ybar = +F_e, s = 1 has
    // -F_e; H_c gathers them at this node and at +1.  PEC-held E nodes carry no cotangent (a +1 node
    // reached by wrapping is no PEC node).  Per axis, away from PEC planes and without a slab node
    // among the two, the Dbar are the ybar themselves.
    T h0 = b0, h1 = b1, h2 = b2;
    // z: E_y (s = 0) into H_x, E_x (s = 1) into H_y
    if (pz_plain) {
        h0 += fy - fy_zp;
        h1 += fx_zp - fx;
    } else {
        const int szp = k + 1 < nz ? slab_or_none(kg + 1, c.dlo[2], c.dhi[2], c.nzg, c.ns[2]) : -1;
        const T tyz_k = (pi || pk) ? T(0) : dbar_node(c.cE[2], c.nzg, c.apsiE[1][0], c.n, c.ns, 2, i, j, k, kg, sz, fy);
        const T tyz_n = (!ze || pi) ? T(0) : dbar_node(c.cE[2], c.nzg, c.apsiE[1][0], c.n, c.ns, 2, i, j, k + 1, kg + 1, szp, fy_zp);
        const T txz_k = (pj || pk) ? T(0) : dbar_node(c.cE[2], c.nzg, c.apsiE[0][1], c.n, c.ns, 2, i, j, k, kg, sz, -fx);
        const T txz_n = (!ze || pj) ? T(0) : dbar_node(c.cE[2], c.nzg, c.apsiE[0][1], c.n, c.ns, 2, i, j, k + 1, kg + 1, szp, -fx_zp);
        h0 += tyz_k - tyz_n;
        h1 += txz_k - txz_n;
    }
    // y: E_z (s = 1) into H_x, E_x (s = 0) into H_z
    if (py_plain) {
        h0 += fz_yp - fz;
        h2 += fx - fx_yp;
    } else {
        const int syp = j + 1 < ny ? slab_or_none(j + 1, c.dlo[1], c.dhi[1], ny, c.ns[1]) : -1;
        const T tzy = (pi || pj) ? T(0) : dbar_node(c.cE[1], c.n[1], c.apsiE[2][1], c.n, c.ns, 1, i, j, k, j, sy, -fz);
        const T tzy_p = (!ye || pi) ? T(0) : dbar_node(c.cE[1], c.n[1], c.apsiE[2][1], c.n, c.ns, 1, i, j + 1, k, j + 1, syp, -fz_yp);
        const T txy = (pk || pj) ? T(0) : dbar_node(c.cE[1], c.n[1], c.apsiE[0][0], c.n, c.ns, 1, i, j, k, j, sy, fx);
        const T txy_p = (!ye || pk) ? T(0) : dbar_node(c.cE[1], c.n[1], c.apsiE[0][0], c.n, c.ns, 1, i, j + 1, k, j + 1, syp, fx_yp);
        h0 += tzy - tzy_p;
        h2 += txy - txy_p;
    }
    // x: E_z (s = 0) into H_y, E_y (s = 1) into H_z
    if (px_plain) {
        h1 += fz - fz_xp;
        h2 += fy_xp - fy;
    } else {
        const int sxp = i + 1 < nx ? slab_or_none(i + 1, c.dlo[0], c.dhi[0], nx, c.ns[0]) : -1;
        const T tzx = (pi || pj) ? T(0) : dbar_node(c.cE[0], c.n[0], c.apsiE[2][0], c.n, c.ns, 0, i, j, k, i, sx, fz);
        const T tzx_p = (!xe || pj) ? T(0) : dbar_node(c.cE[0], c.n[0], c.apsiE[2][0], c.n, c.ns, 0, i + 1, j, k, i + 1, sxp, fz_xp);
        const T tyx = (pk || pi) ? T(0) : dbar_node(c.cE[0], c.n[0], c.apsiE[1][1], c.n, c.ns, 0, i, j, k, i, sx, -fy);
        const T tyx_p = (!xe || pk) ? T(0) : dbar_node(c.cE[0], c.n[0], c.apsiE[1][1], c.n, c.ns, 0, i + 1, j, k, i + 1, sxp, -fy_xp);
        h1 += tzx - tzx_p;
        h2 += tyx - tyx_p;
    }
    // finish the H-side CPML transpose of step m (the E-side launch has read psibar_H)
    if (sy >= 0) {
        const int o = slab_off_c(c.n, c.ns, 1, i, j, k, sy);
        const T b = c.cH[1][j];
        c.apsiH[0][0][o] = b * (c.apsiH[0][0][o] - S * b0);
        c.apsiH[2][1][o] = b * (c.apsiH[2][1][o] + S * b2);
    }
    if (sz >= 0) {
        const int o = slab_off_c(c.n, c.ns, 2, i, j, k, sz);
        const T b = c.cH[2][kg];
        c.apsiH[0][1][o] = b * (c.apsiH[0][1][o] + S * b0);
        c.apsiH[1][0][o] = b * (c.apsiH[1][0][o] - S * b1);
    }
    if (sx >= 0) {
        const int o = slab_off_c(c.n, c.ns, 0, i, j, k, sx);
        const T b = c.cH[0][i];
        c.apsiH[1][1][o] = b * (c.apsiH[1][1][o] + S * b1);
        c.apsiH[2][0][o] = b * (c.apsiH[2][0][o] - S * b2);
    }
    if (kMon && m >= 1 && in_box3(c.mlo, c.mhi, i, j, kg)) {
        const long long bo = box_cell(c.mlo, c.mhi, i, j, kg);
        h0 += c.inj[bo];
        h1 += c.inj[c.mvol + bo];
        h2 += c.inj[2 * c.mvol + bo];
    }
    B0[ij] = h0;
    B1[ij] = h1;
    B2[ij] = h2;
}

// Completes a pending transposed step cell by cell (the algebra of e_deferred): for every E
// component not held by a PEC plane, Ebar = F / (S eps^-1) (or the pole form in dispersive cells,
// which also advances the pole cotangents) and the own psibar_E of its two derivatives.
template <typename T, bool kPoles, bool kTen = false>
__global__ void __launch_bounds__(kTileX* kTileY) k_adj_flush_cell(const AdjCellArgs<T> c,
                                                                   const Dom<T>* __restrict__ doms, T S) {
    const int nx = c.n[0], ny = c.n[1];
    const int i = blockIdx.x * kTileX + threadIdx.x, j = blockIdx.y * kTileY + threadIdx.y, k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const int kg = k + c.kz0;
    const long long id = ((long long)k * ny + j) * nx + i;
    const int sl[3] = {slab_or_none(i, c.dlo[0], c.dhi[0], nx, c.ns[0]), slab_or_none(j, c.dlo[1], c.dhi[1], ny, c.ns[1]),
                       slab_or_none(kg, c.dlo[2], c.dhi[2], c.nzg, c.ns[2])};
    const int x[3] = {i, j, kg};
    bool disp = false;
    long long bo = 0;
    if (kPoles) {
        const Dom<T>& d = doms[c.dom];
        disp = d.npole > 0 && in_ade_box(d, i, j, k) && d.mask[id];
        if (disp) bo = ade_off(d, i, j, k);
    }
    const bool pi = i == 0 && !c.per[0], pj = j == 0 && !c.per[1], pk = k == 0;
    const bool pec[3] = {pj || pk, pi || pk, pi || pj};
    for (int a = 0; a < 3; ++a) {
        if (pec[a]) continue;
        const T ie = kTen ? T(1) : c.ie[a][id];
        const T F = c.A[a][id];
        T eb;
        if (kTen) {
            eb = c.Eb[a][id];
        } else if (kPoles && disp) {
            const Dom<T>& d = doms[c.dom];
            eb = (T(1) / ie - d.G) / S * F;
            for (int p = 0; p < d.npole; ++p) {
                T* pp = d.aade + ((long long)(a * d.npole + p) * 2 + 0) * d.bcell + bo;
                T* pq = pp + d.bcell;
                const T xp = *pp, xq = *pq;
                eb += d.g0[p] * xp + d.g1[p] * xq;
                *pp = d.M00[p] * xp + d.M10[p] * xq + (T(1) - d.M00[p]) / S * F;
                *pq = d.M01[p] * xp + d.M11[p] * xq - d.M01[p] / S * F;
            }
        } else {
            eb = F * recip_t(S * ie);
        }
        for (int s2 = 0; s2 < 2; ++s2) {
            const int ax = (a + 1 + s2) % 3;
            if (sl[ax] < 0) continue;
            T* p = c.apsiE[a][s2] + slab_off_c(c.n, c.ns, ax, i, j, k, sl[ax]);
            *p = c.cE[ax][x[ax]] * (*p + (s2 == 0 ? F : -F));
        }
        c.A[a][id] = eb;
    }
}

template <typename T>
void launch_adj_flush_cell(const Launch& L, const AdjCellArgs<T>& c, const Dom<T>* doms, T S, int poles,
                           int tensor) {
    const dim3 g((unsigned)((c.n[0] + kTileX - 1) / kTileX), (unsigned)((c.n[1] + kTileY - 1) / kTileY),
                 (unsigned)c.n[2]);
    if (tensor)
        k_adj_flush_cell<T, false, true><<<g, dim3(kTileX, kTileY), 0, L.stream>>>(c, doms, S);
    else if (poles)
        k_adj_flush_cell<T, true><<<g, dim3(kTileX, kTileY), 0, L.stream>>>(c, doms, S);
    else
        k_adj_flush_cell<T, false><<<g, dim3(kTileX, kTileY), 0, L.stream>>>(c, doms, S);
    ++*L.counter;
}

// blocks of 32 x 8 threads covering 16 x 16 cells of a plane (warps of 16 x 2 cells)
inline dim3 adj_cell_grid(const int* n) {
    return dim3((unsigned)((n[0] + 15) / 16), (unsigned)((n[1] + 15) / 16), (unsigned)n[2]);
}

template <typename T>
void launch_adj_e_cell(const Launch& L, const AdjCellArgs<T>& c, const Dom<T>* doms, const Mon* mons, T S, int m,
                       int pending, int poles, int mon, int pole_grad, int tensor) {
    const dim3 g = adj_cell_grid(c.n), b(kTileX, kTileY);
    if (tensor) {
        // a tensor domain has no poles; its material cotangent comes from launch_tensor_grad
        if (mon)
            launch_k(L, k_adj_e_cell<T, false, false, true, false, true>, g, b, c, doms, mons, S, m, pending);
        else
            launch_k(L, k_adj_e_cell<T, false, false, false, false, true>, g, b, c, doms, mons, S, m, pending);
        ++*L.counter;
        return;
    }
    const bool grad = c.grad != nullptr;
    const int key = (poles && pole_grad ? 8 : 0) | (poles ? 4 : 0) | (grad ? 2 : 0) | (mon ? 1 : 0);
    switch (key) {
        case 0: launch_k(L, k_adj_e_cell<T, false, false, false, false>, g, b, c, doms, mons, S, m, pending); break;
        case 1: launch_k(L, k_adj_e_cell<T, false, false, true, false>, g, b, c, doms, mons, S, m, pending); break;
        case 2: launch_k(L, k_adj_e_cell<T, false, true, false, false>, g, b, c, doms, mons, S, m, pending); break;
        case 3: launch_k(L, k_adj_e_cell<T, false, true, true, false>, g, b, c, doms, mons, S, m, pending); break;
        case 4: launch_k(L, k_adj_e_cell<T, true, false, false, false>, g, b, c, doms, mons, S, m, pending); break;
        case 5: launch_k(L, k_adj_e_cell<T, true, false, true, false>, g, b, c, doms, mons, S, m, pending); break;
        case 6: launch_k(L, k_adj_e_cell<T, true, true, false, false>, g, b, c, doms, mons, S, m, pending); break;
        case 7: launch_k(L, k_adj_e_cell<T, true, true, true, false>, g, b, c, doms, mons, S, m, pending); break;
        case 12: launch_k(L, k_adj_e_cell<T, true, false, false, true>, g, b, c, doms, mons, S, m, pending); break;
        case 13: launch_k(L, k_adj_e_cell<T, true, false, true, true>, g, b, c, doms, mons, S, m, pending); break;
        case 14: launch_k(L, k_adj_e_cell<T, true, true, false, true>, g, b, c, doms, mons, S, m, pending); break;
        default: launch_k(L, k_adj_e_cell<T, true, true, true, true>, g, b, c, doms, mons, S, m, pending); break;
    }
    ++*L.counter;
}

template <typename T>
void launch_adj_h_cell(const Launch& L, const AdjCellArgs<T>& c, const Dom<T>* doms, const Mon* mons, T S, int m,
                       int mon) {
    const dim3 g = adj_cell_grid(c.n), b(kTileX, kTileY);
    if (mon)
        launch_k(L, k_adj_h_cell<T, true>, g, b, c, doms, mons, S, m);
    else
        launch_k(L, k_adj_h_cell<T, false>, g, b, c, doms, mons, S, m);
    ++*L.counter;
}

template <typename T>
void launch_adj_e(const Launch& L, const Dom<T>* doms, const Mon* mons, const Tile* tiles, int ntiles, T S, int m,
                  int pending, int general, int aniso, int pole_grad) {
    if (ntiles <= 0) return;
    const dim3 b(kTileX, kTileY);
    if (general && pole_grad)
        k_adj_e_gen<T, true><<<ntiles, b, 0, L.stream>>>(doms, mons, tiles, S, m, pending);
    else if (general)
        k_adj_e_gen<T, false><<<ntiles, b, 0, L.stream>>>(doms, mons, tiles, S, m, pending);
    else if (aniso)
        k_adj_e_int<T, true><<<ntiles, b, 0, L.stream>>>(doms, mons, tiles, S, m, pending);
    else
        k_adj_e_int<T, false><<<ntiles, b, 0, L.stream>>>(doms, mons, tiles, S, m, pending);
    ++*L.counter;
}

template <typename T>
void launch_adj_h(const Launch& L, const Dom<T>* doms, const Mon* mons, const Tile* tiles, int ntiles, T S, int m,
                  int general) {
    if (ntiles <= 0) return;
    const dim3 b(kTileX, kTileY);
    if (general)
        k_adj_h_gen<T><<<ntiles, b, 0, L.stream>>>(doms, mons, tiles, S, m);
    else
        k_adj_h_int<T><<<ntiles, b, 0, L.stream>>>(doms, mons, tiles, S, m);
    ++*L.counter;
}

template <typename T>
void launch_adj_flush(const Launch& L, const Dom<T>* doms, const Tile* tiles, int ntiles, T S) {
    if (ntiles <= 0) return;
    k_adj_flush<T><<<ntiles, dim3(kTileX, kTileY), 0, L.stream>>>(doms, tiles, S);
    ++*L.counter;
}

template <typename T>
void launch_inject_box(const Launch& L, const Dom<T>* dom, const Mon* mons, const int* lo, const int* hi,
                       long long pidx_e, long long pidx_h, T* inj) {
    const long long vol = (long long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
    if (vol <= 0) return;
    const int bs = 256;
    k_inject_box<T><<<(unsigned)((vol + bs - 1) / bs), bs, 0, L.stream>>>(dom, mons, make_int3(lo[0], lo[1], lo[2]),
                                                                           make_int3(hi[0], hi[1], hi[2]), pidx_e,
                                                                           pidx_h, inj);
    ++*L.counter;
}

template <typename T>
void launch_inject(const Launch& L, const Dom<T>* doms, const Mon* mons, const int* entries, int nentries,
                   long long nthreads, const long long* entry_begin, int step, int kind) {
    if (nentries <= 0 || nthreads <= 0) return;
    const int bs = 256;
    k_inject<T><<<(unsigned)((nthreads + bs - 1) / bs), bs, 0, L.stream>>>(doms, mons, entries, nentries, nthreads,
                                                                           entry_begin, step, kind);
    ++*L.counter;
}

#define GBFDTD_INST(T)                                                                                          \
    template void launch_adj_e<T>(const Launch&, const Dom<T>*, const Mon*, const Tile*, int, T, int, int, int, \
                                  int, int);                                                                    \
    template void launch_adj_h<T>(const Launch&, const Dom<T>*, const Mon*, const Tile*, int, T, int, int);     \
    template void launch_adj_flush<T>(const Launch&, const Dom<T>*, const Tile*, int, T);                       \
    template void launch_inject<T>(const Launch&, const Dom<T>*, const Mon*, const int*, int, long long,        \
                                   const long long*, int, int);                                                 \
    template void launch_inject_box<T>(const Launch&, const Dom<T>*, const Mon*, const int*, const int*,         \
                                       long long, long long, T*);                                               \
    template void launch_adj_e_cell<T>(const Launch&, const AdjCellArgs<T>&, const Dom<T>*, const Mon*, T, int,  \
                                       int, int, int, int, int);                                                \
    template void launch_adj_h_cell<T>(const Launch&, const AdjCellArgs<T>&, const Dom<T>*, const Mon*, T, int,  \
                                       int);                                                                    \
    template void launch_adj_flush_cell<T>(const Launch&, const AdjCellArgs<T>&, const Dom<T>*, T, int, int);
GBFDTD_INST(float)
GBFDTD_INST(double)
#undef GBFDTD_INST

}  // namespace gbfdtd
