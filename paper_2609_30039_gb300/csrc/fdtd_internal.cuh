// Internal device-side types of the gbfdtd library (not part of the ABI).
//
// Layout in HBM (per domain, dtype T = float | double):
//   F[0..5]   forward fields Ex..Hz, full grid (nz, ny, nx), x fastest
//   A[0..5]   adjoint fields (lagged form during a sweep, see kernels_adj.cu)
//   psiE[a][s], psiH[a][s]  CPML memories, only over the two slabs of the derivative's axis
//   ade       pole states [3][npole][2 (P,Q)][ADE box cells]   (bounding box of the pole mask)
//   cE[q], cH[q]  CPML coefficients along axis q: [b(N) | c(N) | 1/kappa(N)], E at integer
//                 nodes, H at half nodes (Sec. 2.2)
// All descriptors live in device memory and are read through the read-only path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "fdtd.h"

namespace gbfdtd {

constexpr int kMaxPole = 16;
constexpr int kMaxMonPerDom = 8;
constexpr int kMaxSrcPerDom = 8;
constexpr int kTileX = 32;    // block shape (threads): one warp per row of a 32-wide tile
constexpr int kTileY = 8;
// Interior tiles may be wider than a warp (same 256 threads, kIntX x kIntY columns): rows of
// kIntX consecutive x give the DRAM longer contiguous runs per array and plane.
#ifndef GBFDTD_INT_X
#define GBFDTD_INT_X 32
#endif
constexpr int kIntX = GBFDTD_INT_X;
constexpr int kIntY = kTileX * kTileY / kIntX;

template <typename T>
struct Dom {
    int n[3];                  // nx, ny, nz
    long long ncell;
    T* F[6];
    T* A[6];
    const T* ie[3];            // 1/eps per E component (borrowed)
    const uint8_t* mask;       // pole mask (borrowed) or nullptr
    int dlo[3], dhi[3], ns[3]; // CPML depth per axis (low, high), ns = dlo + dhi
    int per[3];                // 1: periodic axis (x, y only): neighbours wrap, no PEC plane
    T* psiE[3][2];
    T* psiH[3][2];
    T* apsiE[3][2];
    T* apsiH[3][2];
    const T* cE[3];
    const T* cH[3];
    int blo[3], bhi[3];        // pole-state box
    long long bcell;
    T* ade;
    T* aade;
    int npole;
    T M00[kMaxPole], M01[kMaxPole], M10[kMaxPole], M11[kMaxPole], g0[kMaxPole], g1[kMaxPole];
    T G;                       // sum_p g0[p]
    int design;                // 1 if a design box is set
    int glo[3], ghi[3];
    double* grad;              // [3][design cells]
    double* pgc;               // pole-coefficient cotangents [npole][6] or nullptr (not collected)
    int nmon;                  // monitors of this domain
    int mon[kMaxMonPerDom];
    int nsrc;                  // soft sources of this domain
    int src[kMaxSrcPerDom];
    double* energy;            // per-step energy or nullptr
    int energy_cap;
};

// A running DFT monitor (Sec. 2.4).  acc / cot: [ncomp][nf][ncell] double2.
// phase: [cap][2 (E: t=n+1, H: t=n+3/2)][nf] double2 = exp(i w t).
struct Mon {
    int dom;
    int lo[3], hi[3];
    int bx, by;
    long long ncell;
    int nf;
    int ncomp;
    int comps[6];
    unsigned mask;
    double2* acc;
    const double2* cot;
    const double2* phase;
    int cap;
    // per-cell mode: field samples of one launched batch of steps, [step of the batch][ncomp][ncell]
    // in the field type, written by the update kernels and folded into acc once per batch
    void* ring;
};

// A DFT work item: cells [begin, min(begin + 256, end)) of monitor `mon` (one thread per cell),
// read from domain descriptor `dom` whose plane k holds global plane k + kz0 (a host-streamed slab;
// resident items have dom = the monitor's domain, kz0 = 0).
struct DftItem {
    int mon;
    int begin;
    int end;
    int dom;
    int kz0;
};

struct Src {
    int dom, comp;
    int lo[3], hi[3];
    int bx, by;
    long long ncell, begin;    // begin: offset of this source in the flattened cell list
    const double* wave;
    int n;
};

// One tile of work: kTileX x kTileY columns of a domain marched over [z0, z1).
enum : int {
    kTileSrcE = 1,   // holds a cell of an electric soft source
    kTileSrcH = 2,   // ... of a magnetic soft source
    kTileMonE = 4,   // holds a cell of a monitor recording an E component (objective injection)
    kTileMonH = 8,   // ... an H component
    kTileGeneral = 16 // needs the CPML / PEC / pole code path (the transposed tile kernels)
};

// Columns of a tile: lane tx maps to x in [xs[0], xs[1]) then [xs[2], xs[3]) (two segments let
// one warp cover both opposite CPML slabs), thread row ty to y likewise with ys; at most
// kTileX x kTileY columns.  z runs over [z0, z1).
struct Tile {
    int dom;
    int xs[4];
    int ys[4];
    int z0, z1;
    int flags;
    int x0, y0;   // first column (for flag tests)
    int lw;       // log2 of the row width in threads (5: 32 x 8 tiles; interior tiles: log2 kIntX)
};

// Coordinate of lane `l` of a two-segment range, or -1 past its end.
__host__ __device__ inline int seg_coord(const int* s, int l) {
    const int n1 = s[1] - s[0];
    if (l < n1) return s[0] + l;
    const int x = s[2] + (l - n1);
    return x < s[3] ? x : -1;
}

// Column (i, j) of this thread in tile t (-1 where the thread has no column): thread number
// tid = threadIdx.y * kTileX + threadIdx.x, lane tid mod 2^lw along x, row tid / 2^lw along y.
__device__ __forceinline__ void tile_coords(const Tile& t, int& i, int& j) {
    const int tid = threadIdx.y * kTileX + threadIdx.x;
    i = seg_coord(t.xs, tid & ((1 << t.lw) - 1));
    j = seg_coord(t.ys, tid >> t.lw);
}

// Offset from cell (x along axis q, element stride st) to its -1 / +1 neighbour along q, or 0
// with *exists = false where the neighbour is absent (beyond a PEC wall or the domain edge); on a
// periodic axis the neighbour wraps around.
__host__ __device__ inline long long nb_minus(int x, int N, long long st, int per, bool* exists) {
    if (x > 0) {
        *exists = true;
        return -st;
    }
    *exists = per != 0;
    return per ? (long long)(N - 1) * st : 0;
}
__host__ __device__ inline long long nb_plus(int x, int N, long long st, int per, bool* exists) {
    if (x + 1 < N) {
        *exists = true;
        return st;
    }
    *exists = per != 0;
    return per ? -(long long)(N - 1) * st : 0;
}

__host__ __device__ inline long long cidx(const int* n, int i, int j, int k) {
    return ((long long)k * n[1] + j) * n[0] + i;
}

// Slab index of coordinate x along an axis with CPML depths (lo, hi) over N nodes, or -1.
__host__ __device__ inline int slab_of(int x, int lo, int hi, int N) {
    if (x < lo) return x;
    if (x >= N - hi) return lo + (x - (N - hi));
    return -1;
}

// Offset inside the slab array of axis q for cell (i,j,k) with slab index s.
__host__ __device__ inline long long slab_off(const int* n, const int* ns, int q, int i, int j, int k, int s) {
    if (q == 0) return ((long long)k * n[1] + j) * ns[0] + s;
    if (q == 1) return ((long long)k * ns[1] + s) * n[0] + i;
    return ((long long)s * n[1] + j) * n[0] + i;
}

// Soft source increments of component `comp` at a cell (Eq. (yee): added after the update); D is a
// domain descriptor or per-cell argument block listing the domain's sources.
template <typename T, typename D>
__device__ __forceinline__ T src_add_t(const D& d, const Src* __restrict__ srcs, int comp, int i, int j, int k,
                                       int step) {
    T add = T(0);
    for (int s = 0; s < d.nsrc; ++s) {
        const Src& sr = srcs[d.src[s]];
        if (sr.comp != comp || step >= sr.n) continue;
        if (i < sr.lo[0] || i >= sr.hi[0] || j < sr.lo[1] || j >= sr.hi[1] || k < sr.lo[2] || k >= sr.hi[2]) continue;
        add += (T)sr.wave[step];
    }
    return add;
}

template <typename T>
__device__ inline bool in_ade_box(const Dom<T>& d, int i, int j, int k) {
    return i >= d.blo[0] && i < d.bhi[0] && j >= d.blo[1] && j < d.bhi[1] && k >= d.blo[2] && k < d.bhi[2];
}

template <typename T>
__device__ inline long long ade_off(const Dom<T>& d, int i, int j, int k) {
    return ((long long)(k - d.blo[2]) * (d.bhi[1] - d.blo[1]) + (j - d.blo[1])) * (d.bhi[0] - d.blo[0]) + (i - d.blo[0]);
}

// ---- launch helpers (host) -------------------------------------------------------------
struct Launch {
    cudaStream_t stream;
    long long* counter;   // launches enqueued
    // programmatic dependent launch: the kernel may start while the previous kernel of the stream
    // finishes (only kernels that call pdl_wait before reading what an earlier kernel writes)
    bool pdl = false;
};

// Programmatic dependent launch (sm_90+): pdl_wait returns once the grids this one depends on have
// completed and their writes are visible (at once for a kernel launched without the attribute);
// pdl_trigger lets the next kernel of the stream start launching once every block of this grid has
// issued it or exited.  A kernel launched with the attribute calls pdl_wait before it reads anything
// an earlier kernel writes (argument blocks uploaded by copies may come first) and pdl_trigger after
// it, so a dependent launch begins only after this grid's prerequisites, hence every earlier kernel
// of the stream, have completed, and its waiting blocks only hold SM slots.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch kernel k on L.stream, with the programmatic-serialization attribute when L.pdl is set.
template <typename... KArgs, typename... Args>
inline void launch_k(const Launch& L, void (*k)(KArgs...), dim3 g, dim3 b, Args&&... args) {
    if (!L.pdl) {
        k<<<g, b, 0, L.stream>>>(std::forward<Args>(args)...);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = L.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

// Forward kernels (kernels_fwd.cu)
// Step context shared by the fused forward kernels: sources, monitors, the device step counter
// and the grid-completion ticket that advances it.
struct StepArgs {
    const Src* srcs;
    const Mon* mons;
    int* d_step;
    unsigned* d_ticket;
    int dft_on;
    const int* d_base;          // per-cell mode: first step of the launched batch ...
    int offset;                 // ... and this step's position in it (step = *d_base + offset)
    int ring = 0;               // per-cell mode: the updates store monitor samples into slot offset
};

template <typename T>
void launch_e_update(const Launch& L, const Dom<T>* doms, const Tile* tiles, int ntiles, T S, const StepArgs& a,
                     int general, int aniso);
// advance: total blocks of the step's H launches that count towards advancing the step counter
// (0: this launch does not advance it)
template <typename T>
void launch_h_update(const Launch& L, const Dom<T>* doms, const Tile* tiles, int ntiles, T S, const StepArgs& a,
                     int general, int energy, unsigned advance);
void launch_advance(const Launch& L, int* d_step, int delta);
// DFT of one kind (0: E, 1: H) for every monitor work item, at step *d_base + offset.
template <typename T>
void launch_dft(const Launch& L, const Dom<T>* doms, const Mon* mons, const DftItem* items, int nitems, int kind,
                const int* d_base, int offset);
// Folds the samples of steps *d_base .. *d_base + cnt - 1 in every monitor's ring into its DFT
// accumulators, in step order with the per-step kernel's FP64 fused multiply-adds (bit for bit the
// accumulators cnt launches of launch_dft of each kind would leave).
template <typename T>
void launch_dft_ring(const Launch& L, const Mon* mons, const DftItem* items, int nitems, const int* d_base, int cnt);
void launch_copy_int(const Launch& L, const int* src, int* dst);
void launch_set_int(const Launch& L, int* dst, int v);
// One domain's operands for the per-cell kernels, passed by value (kernel parameter space) so
// the first field loads need no descriptor load before them.  psi / coef: the CPML memories and
// coefficient rows of the half-step (E or H).
template <typename T>
struct CellArgs {
    T* F[6];
    const T* ie[3];
    T* psi[3][2];
    const T* coef[3];
    int n[3], dlo[3], dhi[3], ns[3];
    int per[3];
    int nsrc;
    int src[kMaxSrcPerDom];
    int src_lo[3], src_hi[3];   // bounding box of this half-step's sources (empty: lo = hi = 0)
    int dom;
    // z window of a host-streamed slab: local plane k is global plane k + kz0 of a domain of nzg
    // planes (the CPML z profile, its memory index and the source boxes use global planes); a
    // resident domain has kz0 = 0, nzg = n[2]
    int kz0, nzg;
    // cells [alo, ahi) the backward step updates (the whole domain, or the interior of a domain
    // with absorbing faces, see launch_iface)
    int alo[3], ahi[3];
    // curl output of the E side of a tensor domain (launch_e_curl), else unused
    T* cur[3];
    // monitor samples (StepArgs::ring): the box [slo, shi) of the domain's monitor, and for each
    // field component in it the ring plane of slot 0 (nullptr: not monitored); slot s starts
    // s * sstride values further
    T* smp[6];
    int slo[3], shi[3];
    long long sstride;
};

// Interface planes of the absorbing-face reversible reconstruction (Sec. 3.2): the H nodes on the
// plane just below each low face of the interior and the E nodes on the plane just above each high
// face (the interior is the box of cells whose own node lies in no CPML slab).  One plane: axis q,
// coordinate x along q, kind 0 = H (three components), 1 = E; its 3 * cells values start at `off`
// inside a record slot.
struct IfacePlane {
    int q, x, kind;
    long long cells, off;
};
struct IfaceArgs {
    IfacePlane p[6];
    int np;
    long long slot;   // values per slot
    int cap;          // last slot index
    int t0;           // step count of slot 0
};
// Copies the planes of `kinds` (bit 0: H, bit 1: E) of every IfacePlane between the fields F and
// record slot s = (d_base ? *d_base : 0) + bias - t0 (to_rec: fields -> record; else record ->
// fields).  Slots outside [0, cap] are skipped.
template <typename T>
void launch_iface(const Launch& L, T* const* F, const int* n, const IfaceArgs& ia, T* rec, const int* d_base, int bias,
                  int kinds, int to_rec);
// The two halves of a backward step (reversible reconstruction) of one domain, each over the box
// [alo, ahi) of its argument block; the step undone is *a.d_base + a.offset.
template <typename T>
void launch_back_h(const Launch& L, const CellArgs<T>& ch, T S, const StepArgs& a);
template <typename T>
void launch_back_e(const Launch& L, const CellArgs<T>& ce, T S, const StepArgs& a, int aniso);

// One domain's operands for the per-cell transposed kernels, passed by value: the adjoint fields,
// the forward fields (material cotangent), eps^-1, the adjoint CPML memories of both half-steps
// and the coefficient rows of both node kinds, the design box and its gradient buffer.
template <typename T>
struct AdjCellArgs {
    T* A[6];
    const T* F[6];
    const T* ie[3];
    T* apsiE[3][2];
    T* apsiH[3][2];
    const T* cE[3];
    const T* cH[3];
    int n[3], dlo[3], dhi[3], ns[3];
    int per[3];
    int dom;
    int glo[3], ghi[3];   // design box (empty: lo = hi = 0)
    double* grad;         // [3][design cells] or nullptr
    int mlo[3], mhi[3];   // bounding box of the domain's monitor cells that carry adjoint sources
    // coordinates [elo, ehi) / [hlo, hhi) per axis where the E-side (H-side) gather meets no slab
    // node (and, H side, no PEC-held node): a cell inside on all three axes takes the plain form
    int elo[3], ehi[3], hlo[3], hhi[3];
    // z window of a host-streamed slab (see CellArgs): local plane k is global plane k + kz0 of a
    // domain of nzg planes (CPML z profile, plain ranges, monitors); resident: kz0 = 0, nzg = n[2].
    // The design box [glo, ghi) is given in local planes; its gradient buffer is indexed as the
    // whole box, whose first global plane is gzg and whose cell count is gvol.
    int kz0, nzg, gzg;
    long long gvol;
    // tensor domain (Sec. 2.3 node assembly): the E cotangent Ebar (the E array then carries the
    // curl cotangent S S_t Ebar between the E and H launches), else nullptr
    T* Eb[3];
    // objective injection over the monitor box [mlo, mhi) (global coordinates): [3][mvol] values of
    // this half-step's components (launch_inject_box), or nullptr without monitors
    const T* inj;
    long long mvol;
};

// Operands of the node-assembled tensor operator S_t = D^{-1/2} (1/8 sum R^T eps^-1 R) D^{-1/2}
// (Sec. 2.3) of one domain: eps^-1 at the nodes (xx, yy, zz, xy, xz, yz; node (i, j, k) at offset
// (k ny + j) nx + i), the E-edge operand v and the output.
template <typename T>
struct TensorArgs {
    const T* t[6];
    const T* v[3];
    T* out[3];
    int n[3], per[3];
};

// Node-tensor cotangent over a design box of nodes: the E cotangent Ebar^{m+1}, the forward H of
// u^m (whose plain curl is the curl the update used), and the FP64 gradient [6][box nodes].
template <typename T>
struct TensorGradArgs {
    const T* Eb[3];
    const T* H[3];
    int n[3], per[3];
    int glo[3], ghi[3];
    long long gvol;
    double* grad;
};

// A Bloch domain's operands (Sec. 2.2): the per-cell arguments of its real parts plus the
// imaginary field arrays and the seam phases p_q = pr[q] + i pi[q] of the x and y faces.
template <typename T>
struct BlochArgs {
    CellArgs<T> c;
    T* FI[6];
    T pr[2], pi[2];
};
template <typename T>
struct AdjBlochArgs {
    AdjCellArgs<T> c;
    T* AI[6];
    T pr[2], pi[2];
};
// Forward and transposed half-steps of a Bloch domain and the completion of a pending transposed
// step of its imaginary E part (kernels_bloch.cu).
template <typename T>
void launch_e_bloch(const Launch& L, const BlochArgs<T>& b, T S, const StepArgs& a);
template <typename T>
void launch_h_bloch(const Launch& L, const BlochArgs<T>& b, T S, const StepArgs& a);
template <typename T>
void launch_adj_e_bloch(const Launch& L, const AdjBlochArgs<T>& b, T S, int pending);
template <typename T>
void launch_adj_h_bloch(const Launch& L, const AdjBlochArgs<T>& b);
template <typename T>
void launch_adj_flush_bloch(const Launch& L, const AdjBlochArgs<T>& b, T S);

// One thread per cell over all cells of one domain (per-cell streaming launch mode).
template <typename T>
void launch_e_cell(const Launch& L, const CellArgs<T>& c, const Dom<T>* doms, T S, const StepArgs& a, int aniso,
                   int poles);
template <typename T>
void launch_h_cell(const Launch& L, const CellArgs<T>& c, T S, const StepArgs& a);
// The per-cell updates of every domain of a batch in one launch each: args holds one argument block
// per domain (device memory), bbeg the prefix sums of the domains' block counts (ceil(nx / 16)
// ceil(ny / 16) nz each; ndom + 1 entries, nblocks = bbeg[ndom]).  The same arithmetic per cell as
// launch_e_cell / launch_h_cell.  aniso / poles / per: some domain is anisotropic, dispersive,
// periodic.
template <typename T>
void launch_e_cells(const Launch& L, const CellArgs<T>* args, const int* bbeg, int ndom, int nblocks,
                    const Dom<T>* doms, T S, const StepArgs& a, int aniso, int poles, int per);
template <typename T>
void launch_h_cells(const Launch& L, const CellArgs<T>* args, const int* bbeg, int ndom, int nblocks, T S,
                    const StepArgs& a, int per);
// Curl of the E update of a tensor domain (CPML memories advanced, no E update, no sources) into
// c.cur; PEC-held edges are not written.
template <typename T>
void launch_e_curl(const Launch& L, const CellArgs<T>& c);
// Tensor operator (kernels_tensor.cu), one thread per cell, every non-PEC E edge: forward (fwd = 1)
// out += S S_t v plus the soft sources of c (the E update of a tensor domain, out = E, v = its curl);
// transposed (fwd = 0) out = S S_t v, zero on PEC-held edges (the curl cotangent from Ebar).
template <typename T>
void launch_tensor_apply(const Launch& L, const TensorArgs<T>& t, const CellArgs<T>& c, T S, const StepArgs& a,
                         int fwd);
// d J / d eps^-1 of every node of the design box, += over one transposed step.
template <typename T>
void launch_tensor_grad(const Launch& L, const TensorArgs<T>& t, const TensorGradArgs<T>& g, T S);
// Counts the nodes the Sec. 2.3 admission rule rejects into *d_bad.
template <typename T>
void launch_tensor_admission(const Launch& L, const TensorArgs<T>& t, const int* dlo, const int* dhi, const int* ns,
                             unsigned long long* d_bad);
// One backward step (reversible reconstruction) of a lossless domain: ce / ch hold the E / H
// half-step's sources; the step index is *a.d_base + a.offset.
template <typename T>
void launch_back_cell(const Launch& L, const CellArgs<T>& ce, const CellArgs<T>& ch, T S, const StepArgs& a,
                      int aniso);

// Adjoint kernels (kernels_adj.cu)
template <typename T>
void launch_adj_e(const Launch& L, const Dom<T>* doms, const Mon* mons, const Tile* tiles, int ntiles, T S, int m,
                  int pending, int general, int aniso,
                  int pole_grad);
template <typename T>
void launch_adj_h(const Launch& L, const Dom<T>* doms, const Mon* mons, const Tile* tiles, int ntiles, T S, int m,
                  int general);
template <typename T>
void launch_adj_flush(const Launch& L, const Dom<T>* doms, const Tile* tiles, int ntiles, T S);
// Per-cell transposed half-steps of one domain (one thread per cell, the forward per-cell grid).
// poles: the domain has a pole box; mon: some monitor of the domain carries an adjoint source;
// pole_grad: the domain collects pole-coefficient cotangents; tensor: the domain is a tensor domain
// (Ebar lives in c.Eb, no poles, the material cotangent comes from launch_tensor_grad).
template <typename T>
void launch_adj_e_cell(const Launch& L, const AdjCellArgs<T>& c, const Dom<T>* doms, const Mon* mons, T S, int m,
                       int pending, int poles, int mon, int pole_grad, int tensor);
template <typename T>
void launch_adj_h_cell(const Launch& L, const AdjCellArgs<T>& c, const Dom<T>* doms, const Mon* mons, T S, int m,
                       int mon);
// Completes a pending transposed step (the deferred own-cell part of the E side) for every cell of
// one domain or window, per cell; poles: the descriptor doms[c.dom] holds the pole box; tensor: Ebar
// comes from c.Eb.
template <typename T>
void launch_adj_flush_cell(const Launch& L, const AdjCellArgs<T>& c, const Dom<T>* doms, T S, int poles,
                           int tensor);
template <typename T>
void launch_inject(const Launch& L, const Dom<T>* doms, const Mon* mons, const int* entries, int nentries,
                   long long nthreads, const long long* entry_begin, int step, int kind);
// The objective injection of one transposed step m for every cell of the box [lo, hi) of the
// domain *dom: inj[c][box cell, x fastest] = dJ/df of component c, for the E components (c < 3)
// at phase index pidx_e = 2 m (the E-DFT of step m) and for the H components (c >= 3) at pidx_h =
// 2 (m - 1) + 1 (the H-DFT of step m - 1; skipped for pidx_h < 0), summed over the domain's
// monitors in FP64 and rounded to T once, as the per-cell transposed kernels add it.
template <typename T>
void launch_inject_box(const Launch& L, const Dom<T>* dom, const Mon* mons, const int* lo, const int* hi,
                       long long pidx_e, long long pidx_h, T* inj);

// Auxiliary kernels (kernels_aux.cu)
// Flux through the H plane of a two-plane monitor; slots: accumulator slots of Ex, Ey, Hx, Hy.
void launch_flux(const Launch& L, const Mon* mon, int nf, const int* slots, double* out);
template <typename T>
void launch_admission(const Launch& L, const Dom<T>* d_dom, const Dom<T>& h_dom, unsigned long long* d_bad);
void launch_mask_box(const Launch& L, const uint8_t* mask, int nx, int ny, int nz, int* d_box);
template <typename T>
void launch_nonfinite(const Launch& L, const T* p, long long n, unsigned long long* d_bad);
// One state part of a native snapshot: the live array, its byte offset in the slot, its size.
struct SnapSeg {
    char* state;
    long long off;
    long long bytes;
};
// Copies every segment live -> slot (to_slot) or slot -> live in one launch (gridDim.y = nseg <=
// 65535); max_bytes: the largest segment.
void launch_snapshot_copy(const Launch& L, const SnapSeg* segs, int nseg, long long max_bytes, void* slot,
                          int to_slot);
template <typename T>
void launch_bf16_encode(const Launch& L, const T* src, long long nplanes, long long plane, uint16_t* dst,
                        float* scales);
template <typename T>
void launch_bf16_decode(const Launch& L, const uint16_t* src, const float* scales, long long nplanes,
                        long long plane, T* dst);

}  // namespace gbfdtd
