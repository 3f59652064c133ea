// Bloch-periodic lateral faces (arxiv 2609.30039, Sec. 2.2: periodic pairs with a fixed Bloch
// phase; Sec. 3.1: Bloch boundaries are transposed with conjugate seam factors).
//
// A field continued across the seam of a Bloch axis q picks up the phase p_q = exp(i phi_q):
// f(x + N_q) = p_q f(x).  The fields are complex, held as two real arrays per component (the
// domain's ordinary field array is the real part, a second array the imaginary part).  Every
// coefficient of Eq. (yee) is real, so the update acts on both parts alike; only a neighbour reached
// across a seam mixes them: the backward differences of the E update read f(-1) = f(N - 1) / p =
// f(N - 1) conj(p), the forward differences of the H update f(N) = f(0) p.  The transposed step is
// the adjoint under <u, v> = sum conj(u) v: the transpose of a forward difference is minus the
// backward difference with the conjugate seam factor and vice versa, so the transposed E side
// (which gathers backward differences of Hbar) reads across the seam with conj(p) and the
// transposed H side (forward differences of the lagged E cotangent) with p -- the same factors as the
// forward kernels.  The lagged form of the transposed E side is that of kernels_adj.cu (after the
// E-side launch of step m the E array holds F = S eps^-1 Ebar-tilde).
//
// Scope: Bloch domains have no CPML slabs and no poles (PEC z faces), soft sources add their real
// waveform to the real part, and they carry no DFT monitor or design box; one thread per cell
// over the grid of the per-cell kernels.
#include "fdtd_internal.cuh"

namespace gbfdtd {

namespace {

__device__ __forceinline__ float fma_b(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_b(double a, double b, double c) { return __fma_rn(a, b, c); }

// (re, im) of array pair (r, m) at offset o, times (wr, wi) when `seam` (a wrapped neighbour).
template <typename T>
__device__ __forceinline__ void ld_seam(const T* r, const T* m, long long o, bool seam, T wr, T wi, T& vr, T& vi) {
    const T a = r[o], b = m[o];
    if (seam) {
        vr = a * wr - b * wi;
        vi = a * wi + b * wr;
    } else {
        vr = a;
        vi = b;
    }
}

// -1 neighbour along an axis of N nodes (stride st) at coordinate x: offset, whether it exists, and
// whether it is reached across a Bloch seam (periodic axis, x = 0)
__device__ __forceinline__ long long nbm(int x, int N, long long st, int per, bool& ex, bool& seam) {
    seam = x == 0 && per;
    ex = x > 0 || per;
    return x > 0 ? -st : (long long)(N - 1) * st;
}
__device__ __forceinline__ long long nbp(int x, int N, long long st, int per, bool& ex, bool& seam) {
    seam = x + 1 == N && per;
    ex = x + 1 < N || per;
    return x + 1 < N ? st : -(long long)(N - 1) * st;
}

}  // namespace

// E half-step of a Bloch domain (forward): E += S eps^-1 C^-(H), backward differences, seam factor
// conj(p) on a wrapped -1 neighbour; tangential E on z = 0 (and on coordinate 0 of a non-periodic
// lateral axis) is held.
template <typename T>
__global__ void __launch_bounds__(kTileX* kTileY, 6) k_e_bloch(const BlochArgs<T> b, T S, const StepArgs a) {
    const CellArgs<T>& c = b.c;
    const int nx = c.n[0], ny = c.n[1], nz = c.n[2];
    const int i = blockIdx.x * kTileX + threadIdx.x, j = blockIdx.y * kTileY + threadIdx.y, k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const long long nxy = (long long)nx * ny;
    const long long id = ((long long)k * ny + j) * nx + i;
    bool hx_, hy_, sx_, sy_;
    const long long ox = nbm(i, nx, 1, c.per[0], hx_, sx_);
    const long long oy = nbm(j, ny, nx, c.per[1], hy_, sy_);
    const bool hz_ = k > 0;
    const T cxr = b.pr[0], cxi = -b.pi[0], cyr = b.pr[1], cyi = -b.pi[1];   // conj(p_x), conj(p_y)
    const T* HR[3] = {c.F[3], c.F[4], c.F[5]};
    const T* HI[3] = {b.FI[3], b.FI[4], b.FI[5]};
    T hr[3], hi[3];
    for (int q = 0; q < 3; ++q) {
        hr[q] = HR[q][id];
        hi[q] = HI[q][id];
    }
    T zr = T(0), zi = T(0);
    // Ex: dHz/dy - dHy/dz ; Ey: dHx/dz - dHz/dx ; Ez: dHy/dx - dHx/dy
    T ny_r = zr, ny_i = zi, nzy_r = zr, nzy_i = zi;   // Hz(j-1), Hx(j-1)
    T nxz_r = zr, nxz_i = zi, nyx_r = zr, nyx_i = zi; // Hz(i-1), Hy(i-1)
    T nyz_r = zr, nyz_i = zi, nxz2_r = zr, nxz2_i = zi; // Hy(k-1), Hx(k-1)
    if (hy_) {
        ld_seam(HR[2], HI[2], id + oy, sy_, cyr, cyi, ny_r, ny_i);
        ld_seam(HR[0], HI[0], id + oy, sy_, cyr, cyi, nzy_r, nzy_i);
    }
    if (hx_) {
        ld_seam(HR[2], HI[2], id + ox, sx_, cxr, cxi, nxz_r, nxz_i);
        ld_seam(HR[1], HI[1], id + ox, sx_, cxr, cxi, nyx_r, nyx_i);
    }
    if (hz_) {
        nyz_r = HR[1][id - nxy];
        nyz_i = HI[1][id - nxy];
        nxz2_r = HR[0][id - nxy];
        nxz2_i = HI[0][id - nxy];
    }
    const T cur_r[3] = {(hr[2] - ny_r) - (hr[1] - nyz_r), (hr[0] - nxz2_r) - (hr[2] - nxz_r),
                        (hr[1] - nyx_r) - (hr[0] - nzy_r)};
    const T cur_i[3] = {(hi[2] - ny_i) - (hi[1] - nyz_i), (hi[0] - nxz2_i) - (hi[2] - nxz_i),
                        (hi[1] - nyx_i) - (hi[0] - nzy_i)};
    const bool pi = i == 0 && !c.per[0], pj = j == 0 && !c.per[1], pk = k == 0;
    const bool pec[3] = {pj || pk, pi || pk, pi || pj};
    const bool src = i >= c.src_lo[0] && i < c.src_hi[0] && j >= c.src_lo[1] && j < c.src_hi[1] &&
                     k >= c.src_lo[2] && k < c.src_hi[2];
    const int step = src ? *a.d_base + a.offset : 0;
    for (int q = 0; q < 3; ++q) {
        if (pec[q]) continue;
        const T ie = c.ie[q][id];
        T er = fma_b(S * ie, cur_r[q], c.F[q][id]);
        const T ei = fma_b(S * ie, cur_i[q], b.FI[q][id]);
        if (src) er += src_add_t<T>(c, a.srcs, q, i, j, k, step);
        c.F[q][id] = er;
        b.FI[q][id] = ei;
    }
}

// H half-step of a Bloch domain (forward): H -= S C^+(E), forward differences, seam factor p on a
// wrapped +1 neighbour; nodes beyond z = N - 1 are absent.
template <typename T>
__global__ void __launch_bounds__(kTileX* kTileY, 6) k_h_bloch(const BlochArgs<T> b, T S, const StepArgs a) {
    const CellArgs<T>& c = b.c;
    const int nx = c.n[0], ny = c.n[1], nz = c.n[2];
    const int i = blockIdx.x * kTileX + threadIdx.x, j = blockIdx.y * kTileY + threadIdx.y, k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const long long nxy = (long long)nx * ny;
    const long long id = ((long long)k * ny + j) * nx + i;
    bool xe, ye, sx_, sy_;
    const long long ox = nbp(i, nx, 1, c.per[0], xe, sx_);
    const long long oy = nbp(j, ny, nx, c.per[1], ye, sy_);
    const bool ze = k + 1 < nz;
    const T pxr = b.pr[0], pxi = b.pi[0], pyr = b.pr[1], pyi = b.pi[1];
    const T* ER[3] = {c.F[0], c.F[1], c.F[2]};
    const T* EI[3] = {b.FI[0], b.FI[1], b.FI[2]};
    T er[3], ei[3];
    for (int q = 0; q < 3; ++q) {
        er[q] = ER[q][id];
        ei[q] = EI[q][id];
    }
    T zy_r = 0, zy_i = 0, xy_r = 0, xy_i = 0;   // Ez(j+1), Ex(j+1)
    T zx_r = 0, zx_i = 0, yx_r = 0, yx_i = 0;   // Ez(i+1), Ey(i+1)
    T yz_r = 0, yz_i = 0, xz_r = 0, xz_i = 0;   // Ey(k+1), Ex(k+1)
    if (ye) {
        ld_seam(ER[2], EI[2], id + oy, sy_, pyr, pyi, zy_r, zy_i);
        ld_seam(ER[0], EI[0], id + oy, sy_, pyr, pyi, xy_r, xy_i);
    }
    if (xe) {
        ld_seam(ER[2], EI[2], id + ox, sx_, pxr, pxi, zx_r, zx_i);
        ld_seam(ER[1], EI[1], id + ox, sx_, pxr, pxi, yx_r, yx_i);
    }
    if (ze) {
        yz_r = ER[1][id + nxy];
        yz_i = EI[1][id + nxy];
        xz_r = ER[0][id + nxy];
        xz_i = EI[0][id + nxy];
    }
    // Hx: dEz/dy - dEy/dz ; Hy: dEx/dz - dEz/dx ; Hz: dEy/dx - dEx/dy
    const T cur_r[3] = {(zy_r - er[2]) - (yz_r - er[1]), (xz_r - er[0]) - (zx_r - er[2]), (yx_r - er[1]) - (xy_r - er[0])};
    const T cur_i[3] = {(zy_i - ei[2]) - (yz_i - ei[1]), (xz_i - ei[0]) - (zx_i - ei[2]), (yx_i - ei[1]) - (xy_i - ei[0])};
    const bool src = i >= c.src_lo[0] && i < c.src_hi[0] && j >= c.src_lo[1] && j < c.src_hi[1] &&
                     k >= c.src_lo[2] && k < c.src_hi[2];
    const int step = src ? *a.d_base + a.offset : 0;
    for (int q = 0; q < 3; ++q) {
        T hr = fma_b(-S, cur_r[q], c.F[3 + q][id]);
        const T hi = fma_b(-S, cur_i[q], b.FI[3 + q][id]);
        if (src) hr += src_add_t<T>(c, a.srcs, 3 + q, i, j, k, step);
        c.F[3 + q][id] = hr;
        b.FI[3 + q][id] = hi;
    }
}

// Transposed E half-step of a Bloch domain (the lagged form of kernels_adj.cu): completes the
// deferred own-cell part of step m+1 (pending: Ebar = F / (S eps^-1)), adds S times the backward
// differences of Hbar (seam factor conj(p)) and stores F = S eps^-1 Ebar-tilde, real and imaginary.
template <typename T>
__global__ void __launch_bounds__(kTileX* kTileY, 6) k_adj_e_bloch(const AdjBlochArgs<T> b, T S, int pending) {
    const AdjCellArgs<T>& c = b.c;
    const int nx = c.n[0], ny = c.n[1];
    const int i = blockIdx.x * kTileX + threadIdx.x, j = blockIdx.y * kTileY + threadIdx.y, k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const long long nxy = (long long)nx * ny;
    const long long id = ((long long)k * ny + j) * nx + i;
    bool hx_, hy_, sx_, sy_;
    const long long ox = nbm(i, nx, 1, c.per[0], hx_, sx_);
    const long long oy = nbm(j, ny, nx, c.per[1], hy_, sy_);
    const bool hz_ = k > 0;
    const T cxr = b.pr[0], cxi = -b.pi[0], cyr = b.pr[1], cyi = -b.pi[1];
    const T* BR[3] = {c.A[3], c.A[4], c.A[5]};
    const T* BI[3] = {b.AI[3], b.AI[4], b.AI[5]};
    T br[3], bi[3];
    for (int q = 0; q < 3; ++q) {
        br[q] = BR[q][id];
        bi[q] = BI[q][id];
    }
    T bz_ym_r = 0, bz_ym_i = 0, bx_ym_r = 0, bx_ym_i = 0;
    T bz_xm_r = 0, bz_xm_i = 0, by_xm_r = 0, by_xm_i = 0;
    T by_zm_r = 0, by_zm_i = 0, bx_zm_r = 0, bx_zm_i = 0;
    if (hy_) {
        ld_seam(BR[2], BI[2], id + oy, sy_, cyr, cyi, bz_ym_r, bz_ym_i);
        ld_seam(BR[0], BI[0], id + oy, sy_, cyr, cyi, bx_ym_r, bx_ym_i);
    }
    if (hx_) {
        ld_seam(BR[2], BI[2], id + ox, sx_, cxr, cxi, bz_xm_r, bz_xm_i);
        ld_seam(BR[1], BI[1], id + ox, sx_, cxr, cxi, by_xm_r, by_xm_i);
    }
    if (hz_) {
        by_zm_r = BR[1][id - nxy];
        by_zm_i = BI[1][id - nxy];
        bx_zm_r = BR[0][id - nxy];
        bx_zm_i = BI[0][id - nxy];
    }
    const T g_r[3] = {S * ((br[1] - by_zm_r) - (br[2] - bz_ym_r)), S * ((br[2] - bz_xm_r) - (br[0] - bx_zm_r)),
                      S * ((br[0] - bx_ym_r) - (br[1] - by_xm_r))};
    const T g_i[3] = {S * ((bi[1] - by_zm_i) - (bi[2] - bz_ym_i)), S * ((bi[2] - bz_xm_i) - (bi[0] - bx_zm_i)),
                      S * ((bi[0] - bx_ym_i) - (bi[1] - by_xm_i))};
    const bool pi = i == 0 && !c.per[0], pj = j == 0 && !c.per[1], pk = k == 0;
    const bool pec[3] = {pj || pk, pi || pk, pi || pj};
    for (int q = 0; q < 3; ++q) {
        if (pec[q]) continue;
        const T ie = c.ie[q][id];
        T fr = c.A[q][id], fi = b.AI[q][id];
        if (pending) {
            fr = fr / (S * ie);
            fi = fi / (S * ie);
        }
        c.A[q][id] = S * ie * (fr + g_r[q]);
        b.AI[q][id] = S * ie * (fi + g_i[q]);
    }
}

// Transposed H half-step of a Bloch domain: Hbar += the forward differences of the lagged E
// cotangent F (seam factor p), real and imaginary.
template <typename T>
__global__ void __launch_bounds__(kTileX* kTileY, 6) k_adj_h_bloch(const AdjBlochArgs<T> b) {
    const AdjCellArgs<T>& c = b.c;
    const int nx = c.n[0], ny = c.n[1], nz = c.n[2];
    const int i = blockIdx.x * kTileX + threadIdx.x, j = blockIdx.y * kTileY + threadIdx.y, k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const long long nxy = (long long)nx * ny;
    const long long id = ((long long)k * ny + j) * nx + i;
    bool xe, ye, sx_, sy_;
    const long long ox = nbp(i, nx, 1, c.per[0], xe, sx_);
    const long long oy = nbp(j, ny, nx, c.per[1], ye, sy_);
    const bool ze = k + 1 < nz;
    const T pxr = b.pr[0], pxi = b.pi[0], pyr = b.pr[1], pyi = b.pi[1];
    const T* FR[3] = {c.A[0], c.A[1], c.A[2]};
    const T* FI[3] = {b.AI[0], b.AI[1], b.AI[2]};
    // a PEC-held E node carries no cotangent: tangential E on coordinate 0 of a non-periodic axis
    // (z always; a +1 node reached by wrapping is no PEC node)
    const bool pi = i == 0 && !c.per[0], pj = j == 0 && !c.per[1], pk = k == 0;
    const bool pec[3] = {pj || pk, pi || pk, pi || pj};
    T fr[3], fi[3];
    for (int q = 0; q < 3; ++q) {
        fr[q] = pec[q] ? T(0) : FR[q][id];
        fi[q] = pec[q] ? T(0) : FI[q][id];
    }
    T fz_yp_r = 0, fz_yp_i = 0, fx_yp_r = 0, fx_yp_i = 0;
    T fz_xp_r = 0, fz_xp_i = 0, fy_xp_r = 0, fy_xp_i = 0;
    T fy_zp_r = 0, fy_zp_i = 0, fx_zp_r = 0, fx_zp_i = 0;
    // +1 neighbours; E_z(j+1) is held where i is a PEC plane, E_x(j+1) where k is, and so on
    if (ye) {
        if (!pi) ld_seam(FR[2], FI[2], id + oy, sy_, pyr, pyi, fz_yp_r, fz_yp_i);
        if (!pk) ld_seam(FR[0], FI[0], id + oy, sy_, pyr, pyi, fx_yp_r, fx_yp_i);
    }
    if (xe) {
        if (!pj) ld_seam(FR[2], FI[2], id + ox, sx_, pxr, pxi, fz_xp_r, fz_xp_i);
        if (!pk) ld_seam(FR[1], FI[1], id + ox, sx_, pxr, pxi, fy_xp_r, fy_xp_i);
    }
    if (ze) {
        if (!pi) {
            fy_zp_r = FR[1][id + nxy];
            fy_zp_i = FI[1][id + nxy];
        }
        if (!pj) {
            fx_zp_r = FR[0][id + nxy];
            fx_zp_i = FI[0][id + nxy];
        }
    }
    T* BR[3] = {c.A[3], c.A[4], c.A[5]};
    T* BI[3] = {b.AI[3], b.AI[4], b.AI[5]};
    const T d_r[3] = {(fr[1] - fy_zp_r) + (fz_yp_r - fr[2]), (fr[2] - fz_xp_r) + (fx_zp_r - fr[0]),
                      (fr[0] - fx_yp_r) + (fy_xp_r - fr[1])};
    const T d_i[3] = {(fi[1] - fy_zp_i) + (fz_yp_i - fi[2]), (fi[2] - fz_xp_i) + (fx_zp_i - fi[0]),
                      (fi[0] - fx_yp_i) + (fy_xp_i - fi[1])};
    for (int q = 0; q < 3; ++q) {
        BR[q][id] = BR[q][id] + d_r[q];
        BI[q][id] = BI[q][id] + d_i[q];
    }
}

// Completes a pending transposed step of the imaginary E part of a Bloch domain: Ebar = F / (S eps^-1)
// (the real part goes through the general flush with every other domain).
template <typename T>
__global__ void __launch_bounds__(kTileX* kTileY) k_adj_flush_bloch(const AdjBlochArgs<T> b, T S) {
    const AdjCellArgs<T>& c = b.c;
    const int nx = c.n[0], ny = c.n[1];
    const int i = blockIdx.x * kTileX + threadIdx.x, j = blockIdx.y * kTileY + threadIdx.y, k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const long long id = ((long long)k * ny + j) * nx + i;
    const bool pi = i == 0 && !c.per[0], pj = j == 0 && !c.per[1], pk = k == 0;
    const bool pec[3] = {pj || pk, pi || pk, pi || pj};
    for (int q = 0; q < 3; ++q)
        if (!pec[q]) b.AI[q][id] = b.AI[q][id] / (S * c.ie[q][id]);
}

static dim3 bloch_grid(const int* n) {
    return dim3((unsigned)((n[0] + kTileX - 1) / kTileX), (unsigned)((n[1] + kTileY - 1) / kTileY), (unsigned)n[2]);
}

template <typename T>
void launch_e_bloch(const Launch& L, const BlochArgs<T>& b, T S, const StepArgs& a) {
    k_e_bloch<T><<<bloch_grid(b.c.n), dim3(kTileX, kTileY), 0, L.stream>>>(b, S, a);
    ++*L.counter;
}
template <typename T>
void launch_h_bloch(const Launch& L, const BlochArgs<T>& b, T S, const StepArgs& a) {
    k_h_bloch<T><<<bloch_grid(b.c.n), dim3(kTileX, kTileY), 0, L.stream>>>(b, S, a);
    ++*L.counter;
}
template <typename T>
void launch_adj_e_bloch(const Launch& L, const AdjBlochArgs<T>& b, T S, int pending) {
    k_adj_e_bloch<T><<<bloch_grid(b.c.n), dim3(kTileX, kTileY), 0, L.stream>>>(b, S, pending);
    ++*L.counter;
}
template <typename T>
void launch_adj_h_bloch(const Launch& L, const AdjBlochArgs<T>& b) {
    k_adj_h_bloch<T><<<bloch_grid(b.c.n), dim3(kTileX, kTileY), 0, L.stream>>>(b);
    ++*L.counter;
}
template <typename T>
void launch_adj_flush_bloch(const Launch& L, const AdjBlochArgs<T>& b, T S) {
    k_adj_flush_bloch<T><<<bloch_grid(b.c.n), dim3(kTileX, kTileY), 0, L.stream>>>(b, S);
    ++*L.counter;
}

#define GBFDTD_INST(T)                                                                         \
    template void launch_e_bloch<T>(const Launch&, const BlochArgs<T>&, T, const StepArgs&);   \
    template void launch_h_bloch<T>(const Launch&, const BlochArgs<T>&, T, const StepArgs&);   \
    template void launch_adj_e_bloch<T>(const Launch&, const AdjBlochArgs<T>&, T, int);        \
    template void launch_adj_h_bloch<T>(const Launch&, const AdjBlochArgs<T>&);                \
    template void launch_adj_flush_bloch<T>(const Launch&, const AdjBlochArgs<T>&, T);
GBFDTD_INST(float)
GBFDTD_INST(double)
#undef GBFDTD_INST

}  // namespace gbfdtd
