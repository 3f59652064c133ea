// Symmetric permittivity tensors at the grid nodes, arxiv 2609.30039 Sec. 2.3.
//
// A tensor domain carries eps^-1 (symmetric positive definite, every eigenvalue of eps at least one)
// at every grid node n and applies it to the curl through the node assembly
//   S_t = D^{-1/2} (1/8 sum_n sum_c R_{n,c}^T eps^-1_n R_{n,c}) D^{-1/2},
// where R_{n,c} picks, for each of the 2^3 choices c, one E edge per axis next to node n (the edge
// along q with coordinate n_q - 1 + c_q), and D is the same sum with the identity tensor.  Counting
// the choices gives the per-edge form used here: for the a-edge e between nodes n0 = e's own node
// and n1 = n0 + e_a,
//   (S_t v)_e = r_e sum_{n in {n0, n1}} [ 1/2 eps^-1_n,aa r_e v_e
//                                          + 1/4 sum_{b != a} eps^-1_n,ab P_b(n) ],
//   P_b(n) = sum of r_f v_f over the two b-edges f next to n,
// with r = D^{-1/2}: D_e = 1/2 per end node, so r = 1, or sqrt(2) on an edge whose node n1 lies
// beyond a non-periodic high face.  PEC-held edges are no unknowns: read as zero, never written.
// S_t is symmetric, so the transposed E update applies the same operator to Ebar.  The cotangent of
// eps^-1_n follows from d(S_t)/d(eps^-1_n): with U_a = sum r Ebar and W_a = sum r C over n's two
// a-edges, d/d xx += S/2 sum r^2 Ebar C over the x-edges, d/d xy += S/4 (U_x W_y + U_y W_x).
#include "fdtd_internal.cuh"

namespace gbfdtd {
namespace {

// Component index of eps^-1_{ab} in the (xx, yy, zz, xy, xz, yz) order.
__host__ __device__ constexpr int tc(int a, int b) { return a == b ? a : (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5)); }

// D^{-1/2} of the q-edge with coordinate x.
template <typename T>
__device__ __forceinline__ T rinv(const int* n, const int* per, int q, int x) {
    return (x + 1 < n[q] || per[q]) ? T(1) : T(1.41421356237309504880);
}

// P_b(node): r-weighted sum of the operand over the two b-edges next to node (x, y, z); zero when
// the node lies on a PEC plane of those edges (a coordinate other than b is 0 on a non-periodic
// axis).  The edge below the node (coordinate x_b - 1) is absent at a non-periodic low face and
// wraps on a periodic axis; it always has both end nodes, so its r is 1.
template <typename T>
__device__ __forceinline__ T pair_sum(const TensorArgs<T>& a, int b, int x, int y, int z) {
    const int p[3] = {x, y, z};
    for (int q = 0; q < 3; ++q)
        if (q != b && p[q] == 0 && !a.per[q]) return T(0);
    const long long nx = a.n[0], nxy = nx * a.n[1];
    const long long id = (long long)z * nxy + (long long)y * nx + x;
    const long long stride = b == 0 ? 1 : (b == 1 ? nx : nxy);
    T s = rinv<T>(a.n, a.per, b, p[b]) * a.v[b][id];
    if (p[b] > 0)
        s += a.v[b][id - stride];
    else if (a.per[b])
        s += a.v[b][id + (long long)(a.n[b] - 1) * stride];
    return s;
}

// (S_t v) on the a-edge of cell (i, j, k), S included; `own` holds this node's six components and
// s0 its three pair sums.
template <typename T, int a>
__device__ __forceinline__ T apply_edge(const TensorArgs<T>& ta, int i, int j, int k, const T* own, const T* s0, T S) {
    constexpr int b = (a + 1) % 3, c = (a + 2) % 3;
    const int p[3] = {i, j, k};
    const long long nx = ta.n[0], nxy = nx * ta.n[1];
    const long long id = (long long)k * nxy + (long long)j * nx + i;
    const T r = rinv<T>(ta.n, ta.per, a, p[a]);
    const T rv = r * ta.v[a][id];
    T acc = T(0.5) * own[a] * rv + T(0.25) * (own[tc(a, b)] * s0[b] + own[tc(a, c)] * s0[c]);
    int q[3] = {i, j, k};
    q[a] += 1;
    bool has1 = q[a] < ta.n[a];
    if (!has1 && ta.per[a]) {
        q[a] = 0;
        has1 = true;
    }
    if (has1) {
        const long long id1 = (long long)q[2] * nxy + (long long)q[1] * nx + q[0];
        acc += T(0.5) * ta.t[a][id1] * rv +
               T(0.25) * (ta.t[tc(a, b)][id1] * pair_sum(ta, b, q[0], q[1], q[2]) +
                          ta.t[tc(a, c)][id1] * pair_sum(ta, c, q[0], q[1], q[2]));
    }
    return S * r * acc;
}

// One thread per cell (the forward per-cell grid).  kFwd: E += S S_t C and the soft sources (the
// second half of a tensor domain's E update); else the transposed form, out = S S_t Ebar (zero on
// PEC-held edges).
template <typename T, bool kFwd>
__global__ void __launch_bounds__(kTileX* kTileY) k_tensor_apply(const TensorArgs<T> ta, const CellArgs<T> c, T S,
                                                                 const StepArgs sa) {
    const int nx = ta.n[0], ny = ta.n[1];
    const int i = blockIdx.x * kTileX + threadIdx.x, j = blockIdx.y * kTileY + threadIdx.y, k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const long long id = ((long long)k * ny + j) * nx + i;
    T own[6];
    for (int q = 0; q < 6; ++q) own[q] = ta.t[q][id];
    const T s0[3] = {pair_sum(ta, 0, i, j, k), pair_sum(ta, 1, i, j, k), pair_sum(ta, 2, i, j, k)};
    const bool pi = i == 0 && !ta.per[0], pj = j == 0 && !ta.per[1], pk = k == 0 && !ta.per[2];
    const bool pec[3] = {pj || pk, pi || pk, pi || pj};
    T val[3];
    val[0] = pec[0] ? T(0) : apply_edge<T, 0>(ta, i, j, k, own, s0, S);
    val[1] = pec[1] ? T(0) : apply_edge<T, 1>(ta, i, j, k, own, s0, S);
    val[2] = pec[2] ? T(0) : apply_edge<T, 2>(ta, i, j, k, own, s0, S);
    if (!kFwd) {
        for (int a = 0; a < 3; ++a) ta.out[a][id] = val[a];
        return;
    }
    T e[3];
    for (int a = 0; a < 3; ++a) e[a] = pec[a] ? T(0) : ta.out[a][id] + val[a];
    // soft sources are added after the update (Eq. (yee))
    if (i >= c.src_lo[0] && i < c.src_hi[0] && j >= c.src_lo[1] && j < c.src_hi[1] && k >= c.src_lo[2] &&
        k < c.src_hi[2]) {
        const int step = *sa.d_base + sa.offset;
        for (int a = 0; a < 3; ++a) e[a] += src_add_t<T>(c, sa.srcs, a, i, j, k, step);
    }
    for (int a = 0; a < 3; ++a)
        if (!pec[a]) ta.out[a][id] = e[a];
}

// Plain curl of the E update on the a-edge at (x, y, z) from the H arrays (the design box lies
// outside the CPML slabs); the -1 neighbour is zero beyond a non-periodic low face and wraps on a
// periodic axis, as in the forward kernel.
template <typename T>
__device__ __forceinline__ T plain_curl(const TensorGradArgs<T>& g, int a, int x, int y, int z) {
    const int p[3] = {x, y, z};
    const long long nx = g.n[0], nxy = nx * g.n[1];
    const long long id = (long long)z * nxy + (long long)y * nx + x;
    auto minus = [&](const T* H, int q) -> T {
        const long long stride = q == 0 ? 1 : (q == 1 ? nx : nxy);
        if (p[q] > 0) return H[id - stride];
        if (g.per[q]) return H[id + (long long)(g.n[q] - 1) * stride];
        return T(0);
    };
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    // curl_a = dH_c/dx_b - dH_b/dx_c
    const T* Hc = g.H[c];
    const T* Hb = g.H[b];
    return (Hc[id] - minus(Hc, b)) - (Hb[id] - minus(Hb, c));
}

template <typename T>
__global__ void __launch_bounds__(kTileX* kTileY) k_tensor_grad(const TensorArgs<T> ta, const TensorGradArgs<T> g,
                                                                T S) {
    const int bx = g.ghi[0] - g.glo[0], by = g.ghi[1] - g.glo[1];
    const int li = blockIdx.x * kTileX + threadIdx.x, lj = blockIdx.y * kTileY + threadIdx.y, lk = blockIdx.z;
    if (li >= bx || lj >= by) return;
    const int p[3] = {g.glo[0] + li, g.glo[1] + lj, g.glo[2] + lk};
    const long long nx = g.n[0], nxy = nx * g.n[1];
    double U[3], W[3], Dg[3];
    for (int a = 0; a < 3; ++a) {
        U[a] = W[a] = Dg[a] = 0.0;
        bool pec = false;
        for (int q = 0; q < 3; ++q) pec = pec || (q != a && p[q] == 0 && !g.per[q]);
        if (pec) continue;
        for (int side = 0; side < 2; ++side) {
            int e[3] = {p[0], p[1], p[2]};
            if (side == 0) {
                if (e[a] > 0)
                    e[a] -= 1;
                else if (g.per[a])
                    e[a] = g.n[a] - 1;
                else
                    continue;
            }
            const long long id = (long long)e[2] * nxy + (long long)e[1] * nx + e[0];
            const double r = (double)rinv<T>(g.n, g.per, a, e[a]);
            const double eb = r * (double)g.Eb[a][id];
            const double cu = r * (double)plain_curl(g, a, e[0], e[1], e[2]);
            U[a] += eb;
            W[a] += cu;
            Dg[a] += eb * cu;
        }
    }
    const long long gi = ((long long)lk * by + lj) * bx + li;
    const double s = (double)S;
    for (int a = 0; a < 3; ++a) g.grad[a * g.gvol + gi] += 0.5 * s * Dg[a];
    g.grad[3 * g.gvol + gi] += 0.25 * s * (U[0] * W[1] + U[1] * W[0]);
    g.grad[4 * g.gvol + gi] += 0.25 * s * (U[0] * W[2] + U[2] * W[0]);
    g.grad[5 * g.gvol + gi] += 0.25 * s * (U[1] * W[2] + U[2] * W[1]);
}

struct SlabDesc {
    int dlo[3], dhi[3], ns[3];
};

// Sec. 2.3 admission, node by node, in FP64 with a relative tolerance of 1e-6: eps^-1 positive
// definite (leading minors) with I - eps^-1 positive semidefinite (every principal minor), i.e. every
// eigenvalue of eps at least one; inside the CPML slab of axis q the normal e_q is a principal axis
// (row q off the diagonal is zero) whose eigenvalue is not strictly between the two of the
// tangential block.
template <typename T>
__global__ void k_tensor_admission(const TensorArgs<T> ta, SlabDesc sd, unsigned long long* bad) {
    const long long ncell = (long long)ta.n[0] * ta.n[1] * ta.n[2];
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= ncell) return;
    const int p[3] = {(int)(t % ta.n[0]), (int)((t / ta.n[0]) % ta.n[1]), (int)(t / ((long long)ta.n[0] * ta.n[1]))};
    double M[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) M[a][b] = (double)ta.t[tc(a, b)][t];
    const double tol = 1e-6;
    const double xx = M[0][0], yy = M[1][1], zz = M[2][2], xy = M[0][1], xz = M[0][2], yz = M[1][2];
    const double det = xx * (yy * zz - yz * yz) - xy * (xy * zz - yz * xz) + xz * (xy * yz - yy * xz);
    bool ok = xx > 0.0 && xx * yy - xy * xy > 0.0 && det > 0.0;
    const double a1 = 1.0 - xx, b1 = 1.0 - yy, c1 = 1.0 - zz;
    ok = ok && a1 >= -tol && b1 >= -tol && c1 >= -tol;
    ok = ok && a1 * b1 - xy * xy >= -tol && a1 * c1 - xz * xz >= -tol && b1 * c1 - yz * yz >= -tol;
    ok = ok && a1 * b1 * c1 - a1 * yz * yz - b1 * xz * xz - c1 * xy * xy - 2.0 * xy * xz * yz >= -tol;
    const double scale = fmax(fabs(xx), fmax(fabs(yy), fabs(zz)));
    for (int q = 0; q < 3 && ok; ++q) {
        if (sd.ns[q] == 0 || slab_of(p[q], sd.dlo[q], sd.dhi[q], ta.n[q]) < 0) continue;
        const int b = (q + 1) % 3, c = (q + 2) % 3;
        if (fmax(fabs(M[q][b]), fabs(M[q][c])) > tol * scale) {
            ok = false;
            break;
        }
        const double m = 0.5 * (M[b][b] + M[c][c]), h = 0.5 * (M[b][b] - M[c][c]);
        const double d = sqrt(h * h + M[b][c] * M[b][c]);
        const double lo = m - d, hi = m + d, tl = tol * (fabs(lo) + fabs(hi));
        if (M[q][q] - lo > tl && hi - M[q][q] > tl) ok = false;
    }
    if (!ok) atomicAdd(bad, 1ull);
}

inline dim3 cells_grid(const int* n) {
    return dim3((unsigned)((n[0] + kTileX - 1) / kTileX), (unsigned)((n[1] + kTileY - 1) / kTileY), (unsigned)n[2]);
}

}  // namespace

template <typename T>
void launch_tensor_apply(const Launch& L, const TensorArgs<T>& t, const CellArgs<T>& c, T S, const StepArgs& a,
                         int fwd) {
    const dim3 g = cells_grid(t.n), b(kTileX, kTileY);
    if (fwd)
        k_tensor_apply<T, true><<<g, b, 0, L.stream>>>(t, c, S, a);
    else
        k_tensor_apply<T, false><<<g, b, 0, L.stream>>>(t, c, S, a);
    ++*L.counter;
}

template <typename T>
void launch_tensor_grad(const Launch& L, const TensorArgs<T>& t, const TensorGradArgs<T>& g, T S) {
    const int bn[3] = {g.ghi[0] - g.glo[0], g.ghi[1] - g.glo[1], g.ghi[2] - g.glo[2]};
    if (bn[0] <= 0 || bn[1] <= 0 || bn[2] <= 0 || !g.grad) return;
    k_tensor_grad<T><<<cells_grid(bn), dim3(kTileX, kTileY), 0, L.stream>>>(t, g, S);
    ++*L.counter;
}

template <typename T>
void launch_tensor_admission(const Launch& L, const TensorArgs<T>& t, const int* dlo, const int* dhi, const int* ns,
                             unsigned long long* d_bad) {
    SlabDesc sd;
    for (int q = 0; q < 3; ++q) {
        sd.dlo[q] = dlo[q];
        sd.dhi[q] = dhi[q];
        sd.ns[q] = ns[q];
    }
    const long long n = (long long)t.n[0] * t.n[1] * t.n[2];
    const int bs = 256;
    k_tensor_admission<T><<<(unsigned)((n + bs - 1) / bs), bs, 0, L.stream>>>(t, sd, d_bad);
    ++*L.counter;
}

#define GBFDTD_INST(T)                                                                                        \
    template void launch_tensor_apply<T>(const Launch&, const TensorArgs<T>&, const CellArgs<T>&, T,          \
                                         const StepArgs&, int);                                               \
    template void launch_tensor_grad<T>(const Launch&, const TensorArgs<T>&, const TensorGradArgs<T>&, T);    \
    template void launch_tensor_admission<T>(const Launch&, const TensorArgs<T>&, const int*, const int*,     \
                                             const int*, unsigned long long*);
GBFDTD_INST(float)
GBFDTD_INST(double)
#undef GBFDTD_INST

}  // namespace gbfdtd
