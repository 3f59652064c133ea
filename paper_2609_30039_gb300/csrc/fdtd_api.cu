// C-ABI of the gbfdtd library (declared in include/fdtd.h): context, memory plan, device
// descriptors, forward stepping, adjoint sweep bookkeeping, snapshots.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "fdtd_internal.cuh"

using namespace gbfdtd;

// Forward steps per captured CUDA graph, and per launched batch of the per-cell mode (the monitor
// rings hold one batch of samples).
constexpr int kGraphSteps = 32;
// Device bytes the monitor rings of a context may take; beyond, the DFT runs per step.
constexpr long long kRingMaxBytes = 512ll << 20;

namespace {

struct DomainHost {
    int n[3] = {0, 0, 0};
    long long ncell = 0;
    int dlo[3] = {0, 0, 0}, dhi[3] = {0, 0, 0}, ns[3] = {0, 0, 0};
    fdtd_cpml cpml{};
    const void* ie[3] = {nullptr, nullptr, nullptr};
    const uint8_t* mask = nullptr;
    int npole = 0;
    fdtd_pole poles[kMaxPole];
    int blo[3] = {0, 0, 0}, bhi[3] = {0, 0, 0};
    long long bcell = 0;
    void* F[6] = {};
    void* A[6] = {};
    void* psiE[3][2] = {};
    void* psiH[3][2] = {};
    void* apsiE[3][2] = {};
    void* apsiH[3][2] = {};
    void* cE[3] = {};
    void* cH[3] = {};
    void* ade = nullptr;
    void* aade = nullptr;
    double* energy = nullptr;
    int energy_cap = 0;
    int design = 0;
    int glo[3] = {0, 0, 0}, ghi[3] = {0, 0, 0};
    double* grad = nullptr;
    std::vector<int> mons;
    std::vector<int> srcs;
    int per[3] = {0, 0, 0};        // periodic axes (x, y)
    double* pgc = nullptr;         // pole-coefficient cotangents [npole][6] (device, owned)
    int pgc_on = 0;                // collected by the transposed steps
    // Bloch-periodic faces (Sec. 2.2): complex fields, the imaginary parts of the forward and
    // adjoint fields in FI / AI, phase per period of the x and y seams
    int bloch = 0;
    double bphase[2] = {0.0, 0.0};
    void* FI[6] = {};
    void* AI[6] = {};
    // interface record of the absorbing-face reversible reconstruction (Sec. 3.2), or nullptr
    void* rec = nullptr;
    IfaceArgs ia{};
    // symmetric node tensors (Sec. 2.3): eps^-1 xx yy zz xy xz yz at the nodes, the curl of the E
    // update and the E cotangent of the transposed sweep (device, owned)
    int tensor = 0;
    void* tn[6] = {};
    void* tcur[3] = {};
    void* teb[3] = {};
    // objective injection of one transposed step over the box of the monitors that carry adjoint
    // sources ([6][box cells]: E of step m, H of step m - 1; device, owned; grown with the box)
    void* inj = nullptr;
    long long inj_cap = 0;
};

struct MonHost {
    Mon m{};
    std::vector<double> omega;
};

struct SrcHost {
    Src s{};
    double* wave = nullptr;
};

struct Slot {
    void* buf = nullptr;
    size_t bytes = 0;
    int codec = 0;
    long long step = 0;
};

}  // namespace

struct fdtd_ctx {
    int dtype = FDTD_F32;
    size_t esz = 4;
    double S = 0;
    cudaStream_t stream = nullptr;
    std::vector<DomainHost> doms;
    void* d_doms = nullptr;
    std::vector<Tile> tiles;        // every tile (transposed kernels)
    std::vector<Tile> tiles_gen;    // tiles touching CPML, PEC planes, domain edges or poles
    std::vector<Tile> tiles_int;    // all other tiles
    Tile* d_tiles = nullptr;
    Tile* d_tiles_gen = nullptr;
    Tile* d_tiles_int = nullptr;
    int aniso = 0;
    std::vector<MonHost> mons;
    Mon* d_mons = nullptr;
    int* d_entries[2] = {nullptr, nullptr};
    long long* d_entry_begin[2] = {nullptr, nullptr};
    int nentries[2] = {0, 0};
    long long nthreads[2] = {0, 0};
    std::vector<SrcHost> srcs;
    Src* d_srcs = nullptr;          // every source of every domain
    int* d_step = nullptr;
    unsigned* d_ticket = nullptr;   // completion ticket of the last H launch of a step
    int cell_mode = 1;              // per-half-step launches of the per-cell streaming kernels
    // per-cell mode with several domains: one launch per half-step over all of them, from argument
    // blocks in device memory (E side, H side) and the prefix sums of the domains' block counts
    void* d_cargs[2] = {nullptr, nullptr};
    int* d_bbeg = nullptr;
    int multi_blocks = 0;
    int cargs_dirty = 1;
    int h_step_tmp = 0;
    long long step = 0;
    long long adj_step = 0;
    int adj_pending = 0;
    int dft_enabled = 1;
    int ring_on = 0;   // monitor rings in use (per-cell mode: DFT once per batch, see ensure_ring)
    int energy_on = 0;
    int phase_cap = 0;
    long long launches = 0;
    std::string err;
    int poisoned = 0;
    std::map<int, Slot> slots;
    unsigned long long* d_flag = nullptr;
    int* d_box = nullptr;
    std::vector<void*> owned;   // every device allocation of the context
    // CUDA graphs of kGraphSteps forward steps, keyed by (dft enabled, energy on)
    cudaStream_t cap_stream = nullptr;
    cudaStream_t aux_stream = nullptr;   // interior launches of the per-half-step mode
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaStream_t dft_stream = nullptr;   // DFT launches of the per-half-step mode
    cudaEvent_t ev_e = nullptr, ev_h = nullptr, ev_de = nullptr, ev_dh = nullptr;
    DftItem* d_dft_items = nullptr;      // 256-cell work items of every monitor
    int n_dft_items = 0;
    int* d_base = nullptr;               // first step of the batch being launched (DFT phases)
    cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    long long graph_launches[2][2] = {{0, 0}, {0, 0}};
    int use_graphs = 1;
    SnapSeg* d_snapsegs = nullptr;   // the state parts of a native snapshot (one copy launch)
    int n_snapsegs = 0;
    long long snap_max = 0;
    // host streaming (Sec. 4.2): the one domain's fields, CPML memories, pole state and materials
    // live in pinned host memory; each batch of up to sk steps runs z-slab by z-slab (sw owned
    // planes plus sk halo planes on each side) in a ring of three device workspaces
    int streamed = 0;
    int sw = 0, sk = 0;
    std::vector<void*> host_owned;            // pinned host allocations of the context
    struct Workspace {
        void* F[6] = {};
        void* ie[3] = {};
        void* psiE[3][2] = {};
        void* psiH[3][2] = {};
        void* ade = nullptr;
        void* mask = nullptr;
    } ws[3];
    cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr;
    cudaEvent_t ws_done[3] = {}, ws_free[3] = {};
    std::vector<cudaEvent_t> ev_in, ev_out;   // per slab: its window copied in / its planes copied out
    void* d_sdoms = nullptr;                  // one descriptor per slab (workspace pointers, local box)
    DftItem* d_sitems = nullptr;              // DFT items of the owned planes of every slab
    std::vector<int> sitem_begin, sitem_count;
    int stream_dirty = 1;
    // streamed transposed sweep (Sec. 4.2: it runs the slab tiling in reverse): forward checkpoints
    // at batch starts (step -> pinned buffer of every forward part, taken every sk steps from
    // ck_t0), the adjoint state in two pinned host sets (the batch end is read, the batch start
    // written), a device adjoint window and the kb replayed forward windows of a batch
    int ck_on = 0;
    long long ck_t0 = 0;
    std::map<long long, void*> ck;
    std::vector<void*> ck_pool;               // pinned checkpoint buffers kept for the next run
    Workspace hadj[2];
    int hadj_cur = 0;
    int hadj_ready = 0;
    Workspace aws;
    std::vector<Workspace> rws;
    void* d_adoms = nullptr;                  // descriptors (slab s, replay j) of the transposed windows
    // instrumentation
    int prof_on = 0;
    int prof_used = 0;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_kind;
};

namespace {

fdtd_status fail(fdtd_ctx* c, fdtd_status st, const std::string& msg) {
    if (c) {
        c->err = msg;
        if (st == FDTD_ECUDA) c->poisoned = 1;
    }
    return st;
}

#define CK(ctx, call)                                                                              \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail((ctx), FDTD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
    } while (0)

#define CKL(ctx)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = cudaGetLastError();                                                       \
        if (e_ != cudaSuccess) return fail((ctx), FDTD_ECUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
    } while (0)

#define GUARD(ctx)                                                                                 \
    do {                                                                                           \
        if (!(ctx)) return FDTD_EINVAL;                                                            \
        if ((ctx)->poisoned) return fail((ctx), FDTD_ESTATE, "context poisoned by an earlier CUDA error"); \
    } while (0)

#define NOT_STREAMED(ctx)                                                                          \
    do {                                                                                           \
        if ((ctx)->streamed) return fail((ctx), FDTD_EINVAL, "not available on a host-streamed context"); \
    } while (0)

fdtd_status dmalloc(fdtd_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return FDTD_OK;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(c, FDTD_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    if (e != cudaSuccess) return fail(c, FDTD_ECUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    c->owned.push_back(*p);
    CK(c, cudaMemsetAsync(*p, 0, bytes, c->stream));
    return FDTD_OK;
}

// Pinned host allocation (host-streamed contexts), zero-filled, owned by the context.
fdtd_status hmalloc(fdtd_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return FDTD_OK;
    cudaError_t e = cudaHostAlloc(p, bytes, cudaHostAllocDefault);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(c, FDTD_ENOMEM, "cudaHostAlloc of " + std::to_string(bytes) + " bytes failed");
    }
    if (e != cudaSuccess) return fail(c, FDTD_ECUDA, std::string("cudaHostAlloc: ") + cudaGetErrorString(e));
    c->host_owned.push_back(*p);
    std::memset(*p, 0, bytes);
    return FDTD_OK;
}

void dfree(fdtd_ctx* c, void* p) {
    if (!p) return;
    for (auto it = c->owned.begin(); it != c->owned.end(); ++it)
        if (*it == p) {
            c->owned.erase(it);
            break;
        }
    cudaFree(p);
}

Launch L(fdtd_ctx* c) { return Launch{c->stream, &c->launches}; }

// CPML profile (Sec. 2.2, reading stated in include/fdtd.h): rows [b | c | 1/kappa] at
// integer (E derivative) or half-integer (H derivative) nodes.
void cpml_table(const fdtd_cpml& p, int q, int N, double S, bool half, std::vector<double>& out) {
    out.assign(3 * (size_t)N, 0.0);
    const int dlo = p.cells[2 * q], dhi = p.cells[2 * q + 1];
    const double smax = p.sigma_max < 0 ? 0.8 * (p.m + 1.0) : p.sigma_max;
    for (int j = 0; j < N; ++j) {
        const double x = j + (half ? 0.5 : 0.0);
        double rho = -1.0, d = 1.0;
        if (dlo > 0 && x < dlo) {
            rho = dlo - x;
            d = dlo;
        } else if (dhi > 0 && x > N - dhi) {
            rho = x - (N - dhi);
            d = dhi;
        }
        double b = 1.0, cc = 0.0, kinv = 1.0;
        if (rho >= 0.0) {
            if (rho > d) rho = d;
            const double r = std::pow(rho / d, p.m);
            const double sigma = smax * r;
            const double kappa = 1.0 + (p.kappa_max - 1.0) * r;
            const double alpha = p.alpha_max * (1.0 - rho / d);
            b = std::exp(-(sigma / kappa + alpha) * S);
            cc = sigma > 0.0 ? sigma * (b - 1.0) / (sigma * kappa + kappa * kappa * alpha) : 0.0;
            kinv = 1.0 / kappa;
        }
        out[j] = b;
        out[N + j] = cc;
        out[2 * N + j] = kinv;
    }
}

// Trapezoidal pole update (Sec. 2.3), closed form of (I - A/2)^-1 (I + A/2) with
// A = [[0, 1], [-a0, -g]]:  M = [[1 + g/2 - a0/4, 1], [-a0, 1 - g/2 - a0/4]] / det,
// det = 1 + g/2 + a0/4;  x-increment vector (b1/(4 det), b1/(2 det)).
void pole_coef(const fdtd_pole& p, double M[4], double g[2]) {
    const double w2 = p.omega_dt * p.omega_dt;
    const double a0 = p.kind == FDTD_LORENTZ ? w2 : 0.0;
    const double b1 = p.kind == FDTD_LORENTZ ? p.delta_eps * w2 : w2;
    const double gm = p.gamma_dt;
    const double det = 1.0 + 0.5 * gm + 0.25 * a0;
    M[0] = (1.0 + 0.5 * gm - 0.25 * a0) / det;
    M[1] = 1.0 / det;
    M[2] = -a0 / det;
    M[3] = (1.0 - 0.5 * gm - 0.25 * a0) / det;
    g[0] = b1 / (4.0 * det);
    g[1] = b1 / (2.0 * det);
}

// Derivatives of the pole coefficients (M00, M01, M10, M11, g0, g1) of pole_coef with respect to
// parameter `wrt` (0 delta_eps, 1 omega_dt, 2 gamma_dt): the same closed form evaluated on dual
// numbers (value, derivative).
struct Dual {
    double v, d;
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
inline Dual cst(double x) { return {x, 0.0}; }

void pole_coef_deriv(const fdtd_pole& p, int wrt, double dc[6]) {
    const Dual de = {p.delta_eps, wrt == 0 ? 1.0 : 0.0};
    const Dual w = {p.omega_dt, wrt == 1 ? 1.0 : 0.0};
    const Dual gm = {p.gamma_dt, wrt == 2 ? 1.0 : 0.0};
    const bool lor = p.kind == FDTD_LORENTZ;
    const Dual w2 = w * w;
    const Dual a0 = lor ? w2 : cst(0.0);
    const Dual b1 = lor ? de * w2 : w2;
    const Dual det = cst(1.0) + cst(0.5) * gm + cst(0.25) * a0;
    const Dual c[6] = {(cst(1.0) + cst(0.5) * gm - cst(0.25) * a0) / det,
                       cst(1.0) / det,
                       (cst(0.0) - a0) / det,
                       (cst(1.0) - cst(0.5) * gm - cst(0.25) * a0) / det,
                       b1 / (cst(4.0) * det),
                       b1 / (cst(2.0) * det)};
    for (int q = 0; q < 6; ++q) dc[q] = c[q].d;
}

long long part_size(const DomainHost& d, int part) {
    if (part < 6 || part >= 18 + 6 * d.npole) return d.ncell;   // fields (real, then a Bloch domain's imaginary)
    if (part < 18) {
        const int a = ((part - 6) % 6) / 2, s = (part - 6) % 2;
        const int ax = (a + 1 + s) % 3;
        return d.ncell / d.n[ax] * d.ns[ax];
    }
    return d.bcell;
}

int part_count(const DomainHost& d) { return 18 + 6 * d.npole + (d.bloch ? 6 : 0); }

void* part_ptr(const DomainHost& d, int which, int part, size_t esz) {
    if (part < 6) return which ? d.A[part] : d.F[part];
    if (part >= 18 + 6 * d.npole) return which ? d.AI[part - 18 - 6 * d.npole] : d.FI[part - 18 - 6 * d.npole];
    if (part < 12) {
        const int a = (part - 6) / 2, s = (part - 6) % 2;
        return which ? d.apsiE[a][s] : d.psiE[a][s];
    }
    if (part < 18) {
        const int a = (part - 12) / 2, s = (part - 12) % 2;
        return which ? d.apsiH[a][s] : d.psiH[a][s];
    }
    char* base = (char*)(which ? d.aade : d.ade);
    if (!base) return nullptr;
    return base + (size_t)(part - 18) * d.bcell * esz;
}

// Outermost extent of a part's array (slabs of the BF16 codec).
long long part_planes(const DomainHost& d, int part) {
    if (part < 6 || part >= 18 + 6 * d.npole) return d.n[2];
    if (part < 18) {
        const int a = ((part - 6) % 6) / 2, s = (part - 6) % 2;
        const int ax = (a + 1 + s) % 3;
        return ax == 2 ? d.ns[2] : d.n[2];
    }
    return d.bhi[2] - d.blo[2];
}

template <typename T>
void fill_dom(const fdtd_ctx* c, const DomainHost& h, Dom<T>& d) {
    std::memset(&d, 0, sizeof(d));
    for (int q = 0; q < 3; ++q) {
        d.n[q] = h.n[q];
        d.dlo[q] = h.dlo[q];
        d.dhi[q] = h.dhi[q];
        d.ns[q] = h.ns[q];
        d.per[q] = h.per[q];
        d.blo[q] = h.blo[q];
        d.bhi[q] = h.bhi[q];
        d.glo[q] = h.glo[q];
        d.ghi[q] = h.ghi[q];
        d.ie[q] = (const T*)h.ie[q];
        d.cE[q] = (const T*)h.cE[q];
        d.cH[q] = (const T*)h.cH[q];
    }
    d.ncell = h.ncell;
    for (int f = 0; f < 6; ++f) {
        d.F[f] = (T*)h.F[f];
        d.A[f] = (T*)h.A[f];
    }
    for (int a = 0; a < 3; ++a)
        for (int s = 0; s < 2; ++s) {
            d.psiE[a][s] = (T*)h.psiE[a][s];
            d.psiH[a][s] = (T*)h.psiH[a][s];
            d.apsiE[a][s] = (T*)h.apsiE[a][s];
            d.apsiH[a][s] = (T*)h.apsiH[a][s];
        }
    d.mask = h.mask;
    d.pgc = h.pgc_on ? h.pgc : nullptr;
    d.bcell = h.bcell;
    d.ade = (T*)h.ade;
    d.aade = (T*)h.aade;
    d.npole = h.npole;
    double G = 0.0;
    for (int p = 0; p < h.npole; ++p) {
        double M[4], g[2];
        pole_coef(h.poles[p], M, g);
        d.M00[p] = (T)M[0];
        d.M01[p] = (T)M[1];
        d.M10[p] = (T)M[2];
        d.M11[p] = (T)M[3];
        d.g0[p] = (T)g[0];
        d.g1[p] = (T)g[1];
        G += g[0];
    }
    d.G = (T)G;
    d.design = h.design;
    d.grad = h.grad;
    d.nmon = (int)h.mons.size();
    for (int i = 0; i < d.nmon; ++i) d.mon[i] = h.mons[i];
    d.nsrc = (int)h.srcs.size();
    for (int i = 0; i < d.nsrc; ++i) d.src[i] = h.srcs[i];
    d.energy = c->energy_on ? h.energy : nullptr;
    d.energy_cap = h.energy_cap;
}

template <typename T>
fdtd_status sync_doms_t(fdtd_ctx* c) {
    std::vector<Dom<T>> hd(c->doms.size());
    for (size_t i = 0; i < c->doms.size(); ++i) fill_dom<T>(c, c->doms[i], hd[i]);
    CK(c, cudaMemcpyAsync(c->d_doms, hd.data(), sizeof(Dom<T>) * hd.size(), cudaMemcpyHostToDevice, c->stream));
    return FDTD_OK;
}

void drop_graphs(fdtd_ctx* c);

fdtd_status sync_doms(fdtd_ctx* c) {
    // captured graphs of the per-cell mode hold the domains' pointers as kernel parameters:
    // any descriptor change (materials, sources, monitors, design) invalidates them
    drop_graphs(c);
    c->stream_dirty = 1;
    c->cargs_dirty = 1;
    return c->dtype == FDTD_F32 ? sync_doms_t<float>(c) : sync_doms_t<double>(c);
}

fdtd_status ensure_phase(fdtd_ctx* c, long long need, bool* changed = nullptr) {
    if (changed) *changed = false;
    if (need <= c->phase_cap) return FDTD_OK;
    if (changed) *changed = true;
    long long cap = c->phase_cap ? c->phase_cap : 1024;
    while (cap < need) cap *= 2;
    for (auto& mh : c->mons) {
        const int nf = mh.m.nf;
        std::vector<double> tab((size_t)cap * 2 * nf * 2);
        for (long long n = 0; n < cap; ++n)
            for (int kind = 0; kind < 2; ++kind) {
                const double t = (double)n + (kind ? 1.5 : 1.0);
                for (int f = 0; f < nf; ++f) {
                    const size_t o = (((size_t)n * 2 + kind) * nf + f) * 2;
                    tab[o] = std::cos(mh.omega[f] * t);
                    tab[o + 1] = std::sin(mh.omega[f] * t);
                }
            }
        void* p = nullptr;
        fdtd_status st = dmalloc(c, &p, tab.size() * sizeof(double));
        if (st != FDTD_OK) return st;
        CK(c, cudaMemcpyAsync(p, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        if (mh.m.phase) {
            CK(c, cudaStreamSynchronize(c->stream));
            dfree(c, (void*)mh.m.phase);
        }
        mh.m.phase = (const double2*)p;
        mh.m.cap = (int)cap;
    }
    c->phase_cap = (int)cap;
    return FDTD_OK;
}

void drop_graphs(fdtd_ctx* c);

fdtd_status sync_mons(fdtd_ctx* c) {
    drop_graphs(c);
    c->stream_dirty = 1;
    if (c->d_mons) {
        CK(c, cudaStreamSynchronize(c->stream));
        dfree(c, c->d_mons);
        c->d_mons = nullptr;
    }
    for (int kind = 0; kind < 2; ++kind) {
        if (c->d_entries[kind]) dfree(c, c->d_entries[kind]);
        if (c->d_entry_begin[kind]) dfree(c, c->d_entry_begin[kind]);
        c->d_entries[kind] = nullptr;
        c->d_entry_begin[kind] = nullptr;
        c->nentries[kind] = 0;
        c->nthreads[kind] = 0;
    }
    if (c->d_dft_items) dfree(c, c->d_dft_items);
    c->d_dft_items = nullptr;
    c->n_dft_items = 0;
    if (c->mons.empty()) return FDTD_OK;
    std::vector<Mon> hm;
    for (auto& m : c->mons) hm.push_back(m.m);
    {
        std::vector<DftItem> items;
        for (size_t mi = 0; mi < c->mons.size(); ++mi)
            for (long long b = 0; b < c->mons[mi].m.ncell; b += kTileX * kTileY) items.push_back({(int)mi, (int)b, (int)std::min<long long>(b + kTileX * kTileY, c->mons[mi].m.ncell),
                                 c->mons[mi].m.dom, 0});
        fdtd_status st = dmalloc(c, (void**)&c->d_dft_items, sizeof(DftItem) * items.size());
        if (st != FDTD_OK) return st;
        CK(c, cudaMemcpyAsync(c->d_dft_items, items.data(), sizeof(DftItem) * items.size(), cudaMemcpyHostToDevice,
                              c->stream));
        c->n_dft_items = (int)items.size();
    }
    fdtd_status st = dmalloc(c, (void**)&c->d_mons, sizeof(Mon) * hm.size());
    if (st != FDTD_OK) return st;
    CK(c, cudaMemcpyAsync(c->d_mons, hm.data(), sizeof(Mon) * hm.size(), cudaMemcpyHostToDevice, c->stream));
    for (int kind = 0; kind < 2; ++kind) {
        std::vector<int> ent;
        std::vector<long long> beg;
        long long tot = 0;
        for (size_t mi = 0; mi < c->mons.size(); ++mi) {
            const Mon& m = c->mons[mi].m;
            for (int ci = 0; ci < m.ncomp; ++ci) {
                if ((m.comps[ci] >= 3) != (kind == 1)) continue;
                ent.push_back((int)mi);
                ent.push_back(ci);
                beg.push_back(tot);
                tot += m.ncell;
            }
        }
        if (ent.empty()) continue;
        st = dmalloc(c, (void**)&c->d_entries[kind], ent.size() * sizeof(int));
        if (st != FDTD_OK) return st;
        st = dmalloc(c, (void**)&c->d_entry_begin[kind], beg.size() * sizeof(long long));
        if (st != FDTD_OK) return st;
        CK(c, cudaMemcpyAsync(c->d_entries[kind], ent.data(), ent.size() * sizeof(int), cudaMemcpyHostToDevice,
                              c->stream));
        CK(c, cudaMemcpyAsync(c->d_entry_begin[kind], beg.data(), beg.size() * sizeof(long long),
                              cudaMemcpyHostToDevice, c->stream));
        c->nentries[kind] = (int)beg.size();
        c->nthreads[kind] = tot;
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return FDTD_OK;
}

fdtd_status upload_tiles(fdtd_ctx* c);

fdtd_status sync_srcs(fdtd_ctx* c) {
    CK(c, cudaStreamSynchronize(c->stream));
    drop_graphs(c);
    if (c->d_srcs) dfree(c, c->d_srcs);
    c->d_srcs = nullptr;
    for (auto& d : c->doms) d.srcs.clear();
    if (!c->srcs.empty()) {
        std::vector<Src> hs;
        for (size_t k = 0; k < c->srcs.size(); ++k) {
            hs.push_back(c->srcs[k].s);
            c->doms[c->srcs[k].s.dom].srcs.push_back((int)k);
        }
        fdtd_status st = dmalloc(c, (void**)&c->d_srcs, sizeof(Src) * hs.size());
        if (st != FDTD_OK) return st;
        CK(c, cudaMemcpyAsync(c->d_srcs, hs.data(), sizeof(Src) * hs.size(), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    fdtd_status st = upload_tiles(c);
    if (st != FDTD_OK) return st;
    return sync_doms(c);
}

bool valid_dom(const fdtd_ctx* c, int d) { return d >= 0 && d < (int)c->doms.size(); }

bool any_bloch(const fdtd_ctx* c) {
    for (const auto& d : c->doms)
        if (d.bloch) return true;
    return false;
}

bool any_tensor(const fdtd_ctx* c) {
    for (const auto& d : c->doms)
        if (d.tensor) return true;
    return false;
}

#define NOT_TENSOR(ctx, what)                                                                      \
    do {                                                                                           \
        if (any_tensor(ctx)) return fail((ctx), FDTD_EINVAL, std::string(what) + " is not available with tensor domains"); \
    } while (0)

#define NOT_BLOCH(ctx, what)                                                                       \
    do {                                                                                           \
        if (any_bloch(ctx)) return fail((ctx), FDTD_EINVAL, std::string(what) + " is not available with Bloch domains"); \
    } while (0)

bool valid_box(const DomainHost& d, const int32_t lo[3], const int32_t hi[3]) {
    for (int q = 0; q < 3; ++q)
        if (lo[q] < 0 || hi[q] > d.n[q] || lo[q] >= hi[q]) return false;
    return true;
}

fdtd_status check_material(fdtd_ctx* c, const fdtd_material& m) {
    for (int a = 0; a < 3; ++a)
        if (!m.inv_eps[a]) return fail(c, FDTD_EINVAL, "inv_eps pointer is NULL");
    if (m.n_poles < 0 || m.n_poles > kMaxPole) return fail(c, FDTD_EINVAL, "n_poles must be in [0, 16]");
    if (m.n_poles > 0 && (!m.poles || !m.pole_mask)) return fail(c, FDTD_EINVAL, "poles need a table and a mask");
    for (int p = 0; p < m.n_poles; ++p) {
        const fdtd_pole& q = m.poles[p];
        if ((q.kind != FDTD_LORENTZ && q.kind != FDTD_DRUDE) || !(q.gamma_dt >= 0) || !(q.omega_dt >= 0) ||
            !std::isfinite(q.delta_eps))
            return fail(c, FDTD_EINVAL, "invalid pole parameters");
    }
    return FDTD_OK;
}

template <typename T>
fdtd_status admission_t(fdtd_ctx* c, int di) {
    Dom<T> hd;
    fill_dom<T>(c, c->doms[di], hd);
    Dom<T>* dd = nullptr;
    fdtd_status st = dmalloc(c, (void**)&dd, sizeof(Dom<T>));
    if (st != FDTD_OK) return st;
    CK(c, cudaMemcpyAsync(dd, &hd, sizeof(Dom<T>), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemsetAsync(c->d_flag, 0, sizeof(unsigned long long), c->stream));
    launch_admission<T>(L(c), dd, hd, c->d_flag);
    CKL(c);
    unsigned long long bad = 0;
    CK(c, cudaMemcpyAsync(&bad, c->d_flag, sizeof(bad), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    dfree(c, dd);
    if (bad)
        return fail(c, FDTD_ETENSOR,
                    "domain " + std::to_string(di) + ": " + std::to_string(bad) +
                        " CPML cells hold a permittivity whose face-normal eigenvalue is the intermediate one");
    return FDTD_OK;
}

fdtd_status admission(fdtd_ctx* c, int di) {
    const DomainHost& d = c->doms[di];
    if (d.ie[0] == d.ie[1] && d.ie[1] == d.ie[2]) return FDTD_OK;  // isotropic: always admitted
    if (d.ns[0] + d.ns[1] + d.ns[2] == 0) return FDTD_OK;
    return c->dtype == FDTD_F32 ? admission_t<float>(c, di) : admission_t<double>(c, di);
}

fdtd_status mask_box(fdtd_ctx* c, const uint8_t* mask, const int n[3], int lo[3], int hi[3]) {
    int init[6] = {n[0], n[1], n[2], 0, 0, 0};
    CK(c, cudaMemcpyAsync(c->d_box, init, sizeof(init), cudaMemcpyHostToDevice, c->stream));
    launch_mask_box(L(c), mask, n[0], n[1], n[2], c->d_box);
    CKL(c);
    int out[6];
    CK(c, cudaMemcpyAsync(out, c->d_box, sizeof(out), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (out[3] == 0) {
        for (int q = 0; q < 3; ++q) lo[q] = hi[q] = 0;
    } else {
        for (int q = 0; q < 3; ++q) {
            lo[q] = out[q];
            hi[q] = out[3 + q];
        }
    }
    return FDTD_OK;
}

// Tiles of kTileX x kTileY columns and a z chunk chosen so that the grid holds several blocks
// per SM.  Each domain is split into an interior box and the boundary shell around it; the
// interior box holds every cell whose update and transpose need no CPML, PEC or domain-edge
// code: per axis [d_lo + 1, N - max(1, d_hi)) (d_lo + 1 keeps the -1 neighbour out of the low
// H slab, whose CPML terms the transposed H update carries to E; 1 when there is no CPML).
// Interior tiles meeting the pole box join the general class.  The shell is cut into six
// disjoint boxes (z-low, z-high, y-low, y-high, x-low, x-high) of general tiles.
// Packs a list of disjoint [lo, hi) ranges, in order, into chunks of at most w coordinates that
// span at most two ranges each: {s0, s1, s2, s3} as in Tile::xs.
static std::vector<std::array<int, 4>> pack_ranges(const std::vector<std::pair<int, int>>& rs, int w) {
    std::vector<std::array<int, 4>> out;
    std::vector<std::pair<int, int>> cur;
    int used = 0;
    auto flush = [&]() {
        if (cur.empty()) return;
        std::array<int, 4> a;
        a[0] = cur[0].first;
        a[1] = cur[0].second;
        a[2] = cur.size() > 1 ? cur[1].first : cur[0].second;
        a[3] = cur.size() > 1 ? cur[1].second : cur[0].second;
        out.push_back(a);
        cur.clear();
        used = 0;
    };
    for (auto r : rs) {
        int lo = r.first;
        while (lo < r.second) {
            if (cur.size() == 2 || used == w) flush();
            const int take = std::min(w - used, r.second - lo);
            cur.push_back({lo, lo + take});
            used += take;
            lo += take;
        }
    }
    flush();
    return out;
}

void build_tiles(fdtd_ctx* c) {
    c->tiles.clear();
    c->tiles_gen.clear();
    c->tiles_int.clear();
    long long zsum = 0;
    for (const auto& d : c->doms)
        zsum += (long long)((d.n[0] + kTileX - 1) / kTileX) * ((d.n[1] + kTileY - 1) / kTileY) * d.n[2];
#ifndef GBFDTD_TILES_PER_SM
#define GBFDTD_TILES_PER_SM 8
#endif
#ifndef GBFDTD_ZCHUNK_MIN
#define GBFDTD_ZCHUNK_MIN 4
#endif
    int zc = (int)(zsum / (152 * GBFDTD_TILES_PER_SM));
    zc = zc < GBFDTD_ZCHUNK_MIN ? GBFDTD_ZCHUNK_MIN : (zc > 32 ? 32 : zc);
    for (int di = 0; di < (int)c->doms.size(); ++di) {
        const DomainHost& d = c->doms[di];
        int a[3], b[3];
        bool has_int = true;
        for (int q = 0; q < 3; ++q) {
            a[q] = d.dlo[q] > 0 ? d.dlo[q] + 1 : 1;
            b[q] = d.n[q] - (d.dhi[q] > 1 ? d.dhi[q] : 1);
            if (a[q] >= b[q]) has_int = false;
        }
        // xr / yr: column ranges; zr: z ranges; interior decides the class
        auto emit = [&](const std::vector<std::pair<int, int>>& xr, const std::vector<std::pair<int, int>>& yr,
                        const std::vector<std::pair<int, int>>& zr, bool interior) {
            const int tw = interior ? kIntX : kTileX;
            const auto xt = pack_ranges(xr, tw);
            const auto yt = pack_ranges(yr, kTileX * kTileY / tw);
            int lw = 0;
            while ((1 << lw) < tw) ++lw;
            for (auto z : zr)
                for (int z0 = z.first; z0 < z.second; z0 += zc)
                    for (const auto& ys : yt)
                        for (const auto& xs : xt) {
                            Tile t;
                            t.dom = di;
                            for (int k = 0; k < 4; ++k) {
                                t.xs[k] = xs[k];
                                t.ys[k] = ys[k];
                            }
                            t.x0 = xs[0];
                            t.y0 = ys[0];
                            t.z0 = z0;
                            t.z1 = z0 + zc < z.second ? z0 + zc : z.second;
                            t.flags = 0;
                            t.lw = lw;
                            bool inner = interior;
                            if (inner && d.npole > 0 && d.bcell > 0) {
                                const int tl[3] = {xs[0], ys[0], t.z0}, th[3] = {xs[1], ys[1], t.z1};
                                bool meet = true;
                                for (int q = 0; q < 3; ++q)
                                    if (th[q] <= d.blo[q] || tl[q] >= d.bhi[q]) meet = false;
                                if (meet) inner = false;
                            }
                            c->tiles.push_back(t);
                            (inner ? c->tiles_int : c->tiles_gen).push_back(t);
                        }
        };
        typedef std::vector<std::pair<int, int>> R;
        const int N[3] = {d.n[0], d.n[1], d.n[2]};
        if (!has_int) {
            emit(R{{0, N[0]}}, R{{0, N[1]}}, R{{0, N[2]}}, false);
            continue;
        }
        // z slabs (full xy), y slabs (both sides in one tile row range), x slabs (both sides per warp)
        emit(R{{0, N[0]}}, R{{0, N[1]}}, R{{0, a[2]}, {b[2], N[2]}}, false);
        emit(R{{0, N[0]}}, R{{0, a[1]}, {b[1], N[1]}}, R{{a[2], b[2]}}, false);
        emit(R{{0, a[0]}, {b[0], N[0]}}, R{{a[1], b[1]}}, R{{a[2], b[2]}}, false);
        emit(R{{a[0], b[0]}}, R{{a[1], b[1]}}, R{{a[2], b[2]}}, true);
    }
}

// Per-tile flags: which tiles hold cells of a soft source or of a DFT monitor (of E or H).
void tile_flags(fdtd_ctx* c, Tile& t) {
    const DomainHost& d = c->doms[t.dom];
    // a two-segment tile is tested against the hull of its columns (flags may over-select)
    const int lo[3] = {t.xs[0], t.ys[0], t.z0};
    const int hi[3] = {t.xs[3] > t.xs[1] ? t.xs[3] : t.xs[1], t.ys[3] > t.ys[1] ? t.ys[3] : t.ys[1], t.z1};
    auto meets = [&](const int* blo, const int* bhi) {
        for (int q = 0; q < 3; ++q)
            if (hi[q] <= blo[q] || lo[q] >= bhi[q]) return false;
        return true;
    };
    t.flags = 0;
    for (int k : d.srcs) {
        const Src& s = c->srcs[k].s;
        if (meets(s.lo, s.hi)) t.flags |= s.comp < 3 ? kTileSrcE : kTileSrcH;
    }
    for (int k : d.mons) {
        const Mon& m = c->mons[k].m;
        if (!meets(m.lo, m.hi)) continue;
        if (m.mask & 7u) t.flags |= kTileMonE;
        if (m.mask & 56u) t.flags |= kTileMonH;
    }
}

fdtd_status upload_tiles(fdtd_ctx* c) {
    drop_graphs(c);
    CK(c, cudaStreamSynchronize(c->stream));
    std::vector<Tile>* lists[3] = {&c->tiles, &c->tiles_gen, &c->tiles_int};
    Tile** dst[3] = {&c->d_tiles, &c->d_tiles_gen, &c->d_tiles_int};
    for (int li = 0; li < 3; ++li) {
        for (auto& t : *lists[li]) tile_flags(c, t);
        const std::vector<Tile>& up = *lists[li];
        if (up.empty()) continue;
        if (!*dst[li]) {
            fdtd_status st = dmalloc(c, (void**)dst[li], sizeof(Tile) * up.size());
            if (st != FDTD_OK) return st;
        }
        CK(c, cudaMemcpyAsync(*dst[li], up.data(), sizeof(Tile) * up.size(), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return FDTD_OK;
}

// Event pair around one launch when profiling (two records on the stream, no work changed).
struct Prof {
    fdtd_ctx* c;
    bool on;
    Prof(fdtd_ctx* cc, int kind) : c(cc), on(false) {
        if (!c->prof_on || c->prof_used + 2 > (int)c->prof_ev.size()) return;
        on = true;
        c->prof_kind[c->prof_used / 2] = kind;
        cudaEventRecord(c->prof_ev[c->prof_used], c->stream);
    }
    ~Prof() {
        if (!on) return;
        cudaEventRecord(c->prof_ev[c->prof_used + 1], c->stream);
        c->prof_used += 2;
    }
};

// Per-cell kernel arguments of domain di for the E (e_side) or H half-step.
template <typename T>
CellArgs<T> make_cell_args(const fdtd_ctx* c, int di, bool e_side) {
    const DomainHost& h = c->doms[di];
    CellArgs<T> ca;
    std::memset(&ca, 0, sizeof(ca));
    for (int f = 0; f < 6; ++f) ca.F[f] = (T*)h.F[f];
    for (int q = 0; q < 3; ++q) {
        ca.ie[q] = (const T*)h.ie[q];
        ca.coef[q] = (const T*)(e_side ? h.cE[q] : h.cH[q]);
        ca.n[q] = h.n[q];
        ca.dlo[q] = h.dlo[q];
        ca.dhi[q] = h.dhi[q];
        ca.ns[q] = h.ns[q];
        ca.per[q] = h.per[q];
        for (int s2 = 0; s2 < 2; ++s2) ca.psi[q][s2] = (T*)(e_side ? h.psiE[q][s2] : h.psiH[q][s2]);
    }
    ca.nsrc = (int)h.srcs.size();
    for (int q = 0; q < ca.nsrc && q < kMaxSrcPerDom; ++q) ca.src[q] = h.srcs[q];
    // bounding box of this half-step's sources (cells outside it skip the source loop)
    bool any = false;
    for (int q = 0; q < ca.nsrc && q < kMaxSrcPerDom; ++q) {
        const Src& sr = c->srcs[h.srcs[q]].s;
        if ((sr.comp < 3) != e_side) continue;
        for (int ax = 0; ax < 3; ++ax) {
            ca.src_lo[ax] = any ? std::min(ca.src_lo[ax], sr.lo[ax]) : sr.lo[ax];
            ca.src_hi[ax] = any ? std::max(ca.src_hi[ax], sr.hi[ax]) : sr.hi[ax];
        }
        any = true;
    }
    ca.dom = di;
    ca.kz0 = 0;
    ca.nzg = h.n[2];
    for (int q = 0; q < 3; ++q) {
        ca.alo[q] = 0;
        ca.ahi[q] = h.n[q];
        ca.cur[q] = (T*)h.tcur[q];
    }
    // the ring of the domain's monitor: component f's plane of slot 0 (E side E, H side H only)
    if (c->ring_on && h.mons.size() == 1) {
        const Mon& m = c->mons[h.mons[0]].m;
        for (int q = 0; q < 3; ++q) {
            ca.slo[q] = m.lo[q];
            ca.shi[q] = m.hi[q];
        }
        ca.sstride = (long long)m.ncomp * m.ncell;
        for (int ci = 0; ci < m.ncomp; ++ci)
            if ((m.comps[ci] < 3) == e_side) ca.smp[m.comps[ci]] = (T*)m.ring + (long long)ci * m.ncell;
    }
    return ca;
}

// Whether the per-cell mode folds the DFT once per batch from monitor rings: a resident context
// whose monitors sit one per domain in domains the per-cell update kernels step (no tensor domain),
// within kRingMaxBytes of rings.
bool ring_wanted(const fdtd_ctx* c) {
    if (c->streamed || c->mons.empty()) return false;
    for (const DomainHost& h : c->doms)
        if (h.mons.size() > 1 || (!h.mons.empty() && (h.tensor || h.bloch))) return false;
    const long long esize = c->dtype == FDTD_F32 ? 4 : 8;
    long long bytes = 0;
    for (const MonHost& mh : c->mons) bytes += (long long)kGraphSteps * mh.m.ncomp * mh.m.ncell * esize;
    return bytes <= kRingMaxBytes;
}


// Brings the rings in line with the configuration (outside graph capture): allocates a missing ring,
// and drops the captured graphs and argument blocks when the rings come into or out of use.
fdtd_status ensure_ring(fdtd_ctx* c) {
    int want = ring_wanted(c) ? 1 : 0;
    const long long esize = c->dtype == FDTD_F32 ? 4 : 8;
    bool alloc = false;
    if (want)
        for (MonHost& mh : c->mons)
            if (!mh.m.ring) {
                fdtd_status st = dmalloc(c, &mh.m.ring, (size_t)(kGraphSteps * mh.m.ncomp * mh.m.ncell * esize));
                if (st == FDTD_ENOMEM) {   // no room for a ring: the DFT runs per half-step instead
                    want = 0;
                    break;
                }
                if (st != FDTD_OK) return st;
                alloc = true;
            }
    if (want == c->ring_on && !alloc) return FDTD_OK;
    c->ring_on = want;
    if (alloc) {
        fdtd_status st = sync_mons(c);   // the device monitor records carry the ring pointers
        if (st != FDTD_OK) return st;
    }
    drop_graphs(c);
    c->cargs_dirty = 1;
    return FDTD_OK;
}

// Whether the per-cell mode runs every domain in one launch per half-step: several domains, none
// of them a Bloch or tensor domain or one with an interface record.
bool multi_cells(const fdtd_ctx* c) {
    if (c->doms.size() < 2 || c->streamed) return false;
    for (const DomainHost& h : c->doms)
        if (h.bloch || h.tensor || h.rec) return false;
    return true;
}

// Uploads the argument blocks of every domain and the block prefix sums (outside graph capture).
template <typename T>
fdtd_status sync_cell_args_t(fdtd_ctx* c) {
    const int nd = (int)c->doms.size();
    std::vector<CellArgs<T>> ae(nd), ah(nd);
    std::vector<int> beg(nd + 1, 0);
    for (int di = 0; di < nd; ++di) {
        ae[di] = make_cell_args<T>(c, di, true);
        ah[di] = make_cell_args<T>(c, di, false);
        const DomainHost& h = c->doms[di];
        beg[di + 1] = beg[di] + ((h.n[0] + 15) / 16) * ((h.n[1] + 15) / 16) * h.n[2];
    }
    for (int s2 = 0; s2 < 2; ++s2) {
        if (!c->d_cargs[s2]) {
            fdtd_status st = dmalloc(c, &c->d_cargs[s2], sizeof(CellArgs<T>) * nd);
            if (st != FDTD_OK) return st;
        }
        CK(c, cudaMemcpyAsync(c->d_cargs[s2], s2 ? ah.data() : ae.data(), sizeof(CellArgs<T>) * nd,
                              cudaMemcpyHostToDevice, c->stream));
    }
    if (!c->d_bbeg) {
        fdtd_status st = dmalloc(c, (void**)&c->d_bbeg, sizeof(int) * (nd + 1));
        if (st != FDTD_OK) return st;
    }
    CK(c, cudaMemcpyAsync(c->d_bbeg, beg.data(), sizeof(int) * (nd + 1), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));   // the host vectors go out of scope
    c->multi_blocks = beg[nd];
    c->cargs_dirty = 0;
    return FDTD_OK;
}

fdtd_status sync_cell_args(fdtd_ctx* c) {
    if (!c->cell_mode || !c->cargs_dirty || !multi_cells(c)) return FDTD_OK;
    return c->dtype == FDTD_F32 ? sync_cell_args_t<float>(c) : sync_cell_args_t<double>(c);
}

// Tensor-operator operands of domain di: operand v, output out (three E-edge arrays each).
template <typename T>
TensorArgs<T> tensor_args(const fdtd_ctx* c, int di, void* const* v, void* const* out) {
    const DomainHost& h = c->doms[di];
    TensorArgs<T> t;
    std::memset(&t, 0, sizeof(t));
    for (int q = 0; q < 6; ++q) t.t[q] = (const T*)h.tn[q];
    for (int a = 0; a < 3; ++a) {
        t.v[a] = (const T*)v[a];
        t.out[a] = (T*)out[a];
        t.n[a] = h.n[a];
        t.per[a] = h.per[a];
    }
    return t;
}

// The interface planes of a domain with absorbing faces (see IfacePlane) and their offsets in a slot.
IfaceArgs iface_args(const DomainHost& h, int cap, long long t0) {
    IfaceArgs ia{};
    long long off = 0;
    auto add = [&](int q, int x, int kind) {
        const long long cells = h.ncell / h.n[q];
        ia.p[ia.np++] = IfacePlane{q, x, kind, cells, off};
        off += 3 * cells;
    };
    for (int q = 0; q < 3; ++q)
        if (h.dlo[q] > 0) add(q, h.dlo[q] - 1, 0);   // H just below the interior's low face
    for (int q = 0; q < 3; ++q)
        if (h.dhi[q] > 0) add(q, h.n[q] - h.dhi[q], 1);   // E just above its high face
    ia.slot = off;
    ia.cap = cap;
    ia.t0 = (int)t0;
    return ia;
}

bool has_cpml(const DomainHost& h) { return h.ns[0] || h.ns[1] || h.ns[2]; }

// One forward step as per-half-step launches on stream st.  offset: position of this step in the
// launched batch of at most kGraphSteps steps (its DFT phase index is *d_base + offset, its monitor
// ring slot offset); first / last: first and last step of the batch (no wait on DFT work of an
// earlier batch; the DFT stream is joined back at the end; the rings are folded after the last).
template <typename T>
void step_once(fdtd_ctx* c, cudaStream_t st, int offset, bool first, bool last) {
    const Launch l{st, &c->launches};
    const Dom<T>* dd = (const Dom<T>*)c->d_doms;
    StepArgs a;
    a.srcs = c->d_srcs;
    a.mons = c->d_mons;
    a.d_step = c->d_step;
    a.d_ticket = c->d_ticket;
    a.dft_on = c->dft_enabled;
    a.d_base = c->d_base;
    a.offset = offset;
    const int ng = (int)c->tiles_gen.size(), ni = (int)c->tiles_int.size();
    // The general and interior launches of a half-step touch disjoint cells: they run
    // concurrently (interior on the auxiliary stream, forked and joined with events, also inside
    // a graph capture) so the high-occupancy interior blocks fill the SMs around the general
    // ones.  Under per-launch profiling they run one after the other on st.
    const bool fork = c->aux_stream && !c->prof_on && ng > 0 && ni > 0;
    const Launch la{fork ? c->aux_stream : st, &c->launches};
    // per-cell mode (no energy record): the kernels take their step from the batch base, and
    // the step counter advances once, after the batch's last step
    const bool cell = c->cell_mode && !c->energy_on;
    // With monitor rings the per-cell updates store the monitor samples and one launch after the
    // batch's last step folds them into the DFT.  Otherwise the DFT of E (step n) runs on its own
    // stream beside the H update, the DFT of H beside the next E update; a half-step waits only for
    // the DFT of the field it overwrites.
    const bool ring = cell && c->ring_on && c->dft_enabled && c->n_dft_items > 0;
    a.ring = ring ? 1 : 0;
    const int nd = (c->dft_enabled && !ring) ? c->n_dft_items : 0;
    const bool dstream = nd > 0 && !c->prof_on;
    const Launch ld{dstream ? c->dft_stream : st, &c->launches};
    const unsigned adv = (unsigned)(ng + ni);
    auto fork_int = [&]() {
        if (!fork) return;
        cudaEventRecord(c->ev_fork, st);
        cudaStreamWaitEvent(c->aux_stream, c->ev_fork, 0);
    };
    auto join_int = [&]() {
        if (!fork) return;
        cudaEventRecord(c->ev_join, c->aux_stream);
        cudaStreamWaitEvent(st, c->ev_join, 0);
    };
    if ((nd > 0 || cell) && first) launch_copy_int(l, c->d_step, c->d_base);
    if (dstream && !first) cudaStreamWaitEvent(st, c->ev_de, 0);   // DFT of E^n done before E changes
    auto cell_args = [&](int di, bool e_side) { return make_cell_args<T>(c, di, e_side); };
    auto bloch_args = [&](int di, bool e_side) {
        const DomainHost& h = c->doms[di];
        BlochArgs<T> b;
        b.c = make_cell_args<T>(c, di, e_side);
        for (int f = 0; f < 6; ++f) b.FI[f] = (T*)h.FI[f];
        for (int q = 0; q < 2; ++q) {
            b.pr[q] = (T)std::cos(h.bphase[q]);
            b.pi[q] = (T)std::sin(h.bphase[q]);
        }
        return b;
    };
    // one launch per half-step over every domain of a batch (per-cell mode)
    const bool multi = cell && multi_cells(c) && !c->cargs_dirty;
    int any_poles = 0, any_per = 0;
    if (multi)
        for (const DomainHost& h : c->doms) {
            any_poles |= h.npole > 0 && h.bcell > 0;
            any_per |= h.per[0] | h.per[1];
        }
    if (multi) {
        Prof p(c, FDTD_KERNEL_E);
        launch_e_cells<T>(l, (const CellArgs<T>*)c->d_cargs[0], c->d_bbeg, (int)c->doms.size(), c->multi_blocks, dd,
                          (T)c->S, a, c->aniso, any_poles, any_per);
    } else if (cell) {
        Prof p(c, FDTD_KERNEL_E);
        for (int di = 0; di < (int)c->doms.size(); ++di) {
            const DomainHost& h = c->doms[di];
            if (h.bloch) {
                launch_e_bloch<T>(l, bloch_args(di, true), (T)c->S, a);
            } else if (h.tensor) {
                // the curl (CPML memories advanced), then E += S S_t curl and the sources
                const CellArgs<T> ce = cell_args(di, true);
                launch_e_curl<T>(l, ce);
                launch_tensor_apply<T>(l, tensor_args<T>(c, di, h.tcur, h.F), ce, (T)c->S, a, 1);
            } else {
                launch_e_cell<T>(l, cell_args(di, true), dd, (T)c->S, a, c->aniso, h.npole > 0 && h.bcell > 0);
            }
        }
    } else {
        fork_int();
        {
            Prof p(c, FDTD_KERNEL_E);
            launch_e_update<T>(l, dd, c->d_tiles_gen, ng, (T)c->S, a, 1, 1);
        }
        {
            Prof p(c, FDTD_KERNEL_E);
            launch_e_update<T>(la, dd, c->d_tiles_int, ni, (T)c->S, a, 0, c->aniso);
        }
        join_int();
    }
    if (nd > 0) {
        if (dstream) {
            cudaEventRecord(c->ev_e, st);
            cudaStreamWaitEvent(c->dft_stream, c->ev_e, 0);
        }
        {
            Prof p(c, FDTD_KERNEL_DFT);
            launch_dft<T>(ld, dd, c->d_mons, c->d_dft_items, nd, 0, c->d_base, offset);
        }
        if (dstream) cudaEventRecord(c->ev_de, c->dft_stream);
    }
    if (dstream && !first) cudaStreamWaitEvent(st, c->ev_dh, 0);   // DFT of H^{n-1/2} done
    if (cell) {
        if (multi) {
            Prof p(c, FDTD_KERNEL_H);
            launch_h_cells<T>(l, (const CellArgs<T>*)c->d_cargs[1], c->d_bbeg, (int)c->doms.size(), c->multi_blocks,
                              (T)c->S, a, any_per);
        } else {
            Prof p(c, FDTD_KERNEL_H);
            for (int di = 0; di < (int)c->doms.size(); ++di) {
                if (c->doms[di].bloch)
                    launch_h_bloch<T>(l, bloch_args(di, false), (T)c->S, a);
                else
                    launch_h_cell<T>(l, cell_args(di, false), (T)c->S, a);
            }
        }
        // interface record of the reversible reconstruction: E^{n+1}, H^{n+3/2} into slot n + 1 - t0
        for (const DomainHost& h : c->doms)
            if (h.rec) launch_iface<T>(l, (T* const*)h.F, h.n, h.ia, (T*)h.rec, c->d_base, offset + 1, 3, 1);
        if (last && ring) {
            Prof p(c, FDTD_KERNEL_DFT);
            launch_dft_ring<T>(l, c->d_mons, c->d_dft_items, c->n_dft_items, c->d_base, offset + 1);
        }
        if (last) launch_advance(l, c->d_step, offset + 1);
    } else {
        fork_int();
        {
            Prof p(c, FDTD_KERNEL_H);
            launch_h_update<T>(l, dd, c->d_tiles_gen, ng, (T)c->S, a, 1, c->energy_on, adv);
        }
        {
            Prof p(c, FDTD_KERNEL_H);
            launch_h_update<T>(la, dd, c->d_tiles_int, ni, (T)c->S, a, 0, c->energy_on, adv);
        }
        join_int();
    }
    if (nd > 0) {
        if (dstream) {
            cudaEventRecord(c->ev_h, st);
            cudaStreamWaitEvent(c->dft_stream, c->ev_h, 0);
        }
        {
            Prof p(c, FDTD_KERNEL_DFT);
            launch_dft<T>(ld, dd, c->d_mons, c->d_dft_items, nd, 1, c->d_base, offset);
        }
        if (dstream) cudaEventRecord(c->ev_dh, c->dft_stream);
        if (dstream && last) cudaStreamWaitEvent(st, c->ev_dh, 0);
    }
}

// ---- host streaming (Sec. 4.2) ------------------------------------------------------------------
// The one domain is cut into z-slabs of sw owned planes.  A batch of kb <= sk steps advances every
// slab in turn: its window (owned planes plus up to sk planes on each side) is copied from the
// host state into a device workspace, stepped kb times with the resident per-cell kernels (the
// global plane offset picks the CPML z profile and the sources), and its owned planes are copied
// back.  Each step spoils one more plane at each cut edge of the window (a cut edge is stepped as
// if it were a PEC / open end), so after kb <= sk steps the owned planes hold exactly the values
// the resident stepper computes.  z is the slowest axis of every per-cell array, so a window is one
// contiguous range per array.
struct SlabWin {
    int zs, ze;     // owned planes [zs, ze)
    int wlo, whi;   // window [wlo, whi)
    int zb0, zb1;   // window part of the pole-state box
};

SlabWin slab_win(const fdtd_ctx* c, int s) {
    const DomainHost& h = c->doms[0];
    const int nz = h.n[2];
    SlabWin w;
    w.zs = s * c->sw;
    w.ze = std::min(nz, w.zs + c->sw);
    w.wlo = std::max(0, w.zs - c->sk);
    w.whi = std::min(nz, w.ze + c->sk);
    w.zb0 = std::max(w.wlo, h.blo[2]);
    w.zb1 = std::min(w.whi, h.bhi[2]);
    if (h.npole == 0 || h.bcell == 0 || w.zb1 <= w.zb0) w.zb0 = w.zb1 = 0;
    return w;
}

int slab_count(const fdtd_ctx* c) { return (c->doms[0].n[2] + c->sw - 1) / c->sw; }

// Elements per z-plane of CPML memory (a, s) (axis (a + 1 + s) % 3; 0 when that axis has none);
// the z-axis memories are indexed by CPML plane, not by grid plane.
long long psi_plane(const DomainHost& h, int a, int s) {
    const int ax = (a + 1 + s) % 3;
    if (h.ns[ax] == 0) return 0;
    if (ax == 0) return (long long)h.n[1] * h.ns[0];
    if (ax == 1) return (long long)h.ns[1] * h.n[0];
    return (long long)h.n[0] * h.n[1];
}

// First E component whose eps^-1 array is the same as that of component a.
int ie_first(const DomainHost& h, int a) {
    for (int b = 0; b < a; ++b)
        if (h.ie[b] == h.ie[a]) return b;
    return a;
}

// Descriptor of slab s's window in its workspace (local z extent and pole box).
template <typename T>
Dom<T> slab_dom(const fdtd_ctx* c, int s) {
    const DomainHost& h = c->doms[0];
    const long long nxy = (long long)h.n[0] * h.n[1];
    const SlabWin w = slab_win(c, s);
    const fdtd_ctx::Workspace& ws = c->ws[s % 3];
    Dom<T> d;
    fill_dom<T>(c, h, d);
    d.n[2] = w.whi - w.wlo;
    d.ncell = nxy * d.n[2];
    for (int f = 0; f < 6; ++f) {
        d.F[f] = (T*)ws.F[f];
        d.A[f] = nullptr;
    }
    for (int a = 0; a < 3; ++a) {
        d.ie[a] = (const T*)ws.ie[ie_first(h, a)];   // distinct arrays, distinct windows
        for (int s2 = 0; s2 < 2; ++s2) {
            d.psiE[a][s2] = (T*)ws.psiE[a][s2];
            d.psiH[a][s2] = (T*)ws.psiH[a][s2];
            d.apsiE[a][s2] = d.apsiH[a][s2] = nullptr;
        }
    }
    d.mask = (const uint8_t*)ws.mask;
    d.aade = nullptr;
    d.ade = (T*)ws.ade;
    d.grad = nullptr;
    d.design = 0;
    d.energy = nullptr;
    if (w.zb1 > w.zb0) {
        d.blo[2] = w.zb0 - w.wlo;
        d.bhi[2] = w.zb1 - w.wlo;
        d.bcell = (long long)(h.bhi[0] - h.blo[0]) * (h.bhi[1] - h.blo[1]) * (w.zb1 - w.zb0);
    } else {
        for (int q = 0; q < 3; ++q) d.blo[q] = d.bhi[q] = 0;
        d.bcell = 0;
    }
    return d;
}

// Per-slab descriptors (workspace pointers, local pole box) and the DFT items of its owned planes.
template <typename T>
fdtd_status stream_prepare(fdtd_ctx* c) {
    if (!c->stream_dirty) return FDTD_OK;
    CK(c, cudaStreamSynchronize(c->stream));
    const DomainHost& h = c->doms[0];
    {
        const size_t fb = (size_t)std::min(h.n[2], c->sw + 2 * c->sk) * h.n[0] * h.n[1] * c->esz;
        for (int r = 0; r < 3; ++r)
            for (int a = 0; a < 3; ++a)
                if (ie_first(h, a) == a && !c->ws[r].ie[a]) {
                    fdtd_status st = dmalloc(c, &c->ws[r].ie[a], fb);
                    if (st != FDTD_OK) return st;
                }
    }
    const int nsl = slab_count(c);
    std::vector<Dom<T>> hd(nsl);
    std::vector<DftItem> items;
    c->sitem_begin.assign(nsl, 0);
    c->sitem_count.assign(nsl, 0);
    for (int s = 0; s < nsl; ++s) {
        const SlabWin w = slab_win(c, s);
        hd[s] = slab_dom<T>(c, s);
        // DFT: monitor cells of the owned planes (cells are numbered x fastest, z slowest)
        c->sitem_begin[s] = (int)items.size();
        for (size_t mi = 0; mi < c->mons.size(); ++mi) {
            const Mon& m = c->mons[mi].m;
            const int za = std::max(w.zs, m.lo[2]), zb = std::min(w.ze, m.hi[2]);
            if (zb <= za) continue;
            const long long per = (long long)m.bx * m.by;
            const long long c0 = (za - m.lo[2]) * per, c1 = (zb - m.lo[2]) * per;
            for (long long b = c0; b < c1; b += kTileX * kTileY)
                items.push_back({(int)mi, (int)b, (int)std::min<long long>(b + kTileX * kTileY, c1), s, w.wlo});
        }
        c->sitem_count[s] = (int)items.size() - c->sitem_begin[s];
    }
    if (!c->d_sdoms) {
        fdtd_status st = dmalloc(c, &c->d_sdoms, sizeof(Dom<T>) * nsl);
        if (st != FDTD_OK) return st;
    }
    CK(c, cudaMemcpyAsync(c->d_sdoms, hd.data(), sizeof(Dom<T>) * nsl, cudaMemcpyHostToDevice, c->stream));
    if (c->d_sitems) dfree(c, c->d_sitems);
    c->d_sitems = nullptr;
    if (!items.empty()) {
        fdtd_status st = dmalloc(c, (void**)&c->d_sitems, sizeof(DftItem) * items.size());
        if (st != FDTD_OK) return st;
        CK(c, cudaMemcpyAsync(c->d_sitems, items.data(), sizeof(DftItem) * items.size(), cudaMemcpyHostToDevice,
                              c->stream));
    }
    CK(c, cudaStreamSynchronize(c->stream));
    c->stream_dirty = 0;
    return FDTD_OK;
}

// CPML memory (a, s) of the E (e = 0) or H (e = 1) update in a set of home arrays.
void* home_psi(const fdtd_ctx::Workspace& hs, int e, int a, int s) { return e ? hs.psiH[a][s] : hs.psiE[a][s]; }

// Copies the global planes [lo, hi) of a state (fields, CPML memories, pole states) between a set of
// arrays in host layout (home: whole domain) and a device window (dev: planes [w.wlo, w.whi)), and,
// with `materials`, the eps^-1 and pole-mask planes host -> device.
fdtd_status window_copy(fdtd_ctx* c, const SlabWin& w, const fdtd_ctx::Workspace& home, const fdtd_ctx::Workspace& dev,
                        int lo, int hi, bool to_dev, bool materials, cudaStream_t st) {
    const DomainHost& h = c->doms[0];
    const fdtd_ctx::Workspace& ws = dev;
    const size_t esz = c->esz;
    const long long nxy = (long long)h.n[0] * h.n[1];
    const int nz = h.n[2];
    const cudaMemcpyKind kind = to_dev ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
    // planes [lo, hi) of an array of `per` elements per plane; the workspace holds the window
    auto planes = [&](void* home, void* dev, long long per, size_t el) -> cudaError_t {
        if (per == 0 || hi <= lo) return cudaSuccess;
        char* hp = (char*)home + (size_t)lo * per * el;
        char* dp = (char*)dev + (size_t)(lo - w.wlo) * per * el;
        const size_t bytes = (size_t)(hi - lo) * per * el;
        return to_dev ? cudaMemcpyAsync(dp, hp, bytes, kind, st) : cudaMemcpyAsync(hp, dp, bytes, kind, st);
    };
    for (int f = 0; f < 6; ++f)
        if (home.F[f] && ws.F[f]) CK(c, planes(home.F[f], ws.F[f], nxy, esz));
    if (to_dev && materials) {
        for (int a = 0; a < 3; ++a)
            if (ie_first(h, a) == a) CK(c, planes(const_cast<void*>(h.ie[a]), ws.ie[a], nxy, esz));
        if (h.npole > 0 && h.mask) CK(c, planes(const_cast<uint8_t*>(h.mask), ws.mask, nxy, 1));
    }
    for (int a = 0; a < 3; ++a)
        for (int s = 0; s < 2; ++s) {
            const long long per = psi_plane(h, a, s);
            if (per == 0 || !home.psiE[a][s] || !ws.psiE[a][s]) continue;
            void* hpsi[2] = {home_psi(home, 0, a, s), home_psi(home, 1, a, s)};
            void* dpsi[2] = {ws.psiE[a][s], ws.psiH[a][s]};
            if ((a + 1 + s) % 3 != 2) {
                for (int e = 0; e < 2; ++e) CK(c, planes(hpsi[e], dpsi[e], per, esz));
                continue;
            }
            // z memories: CPML planes [0, dlo) are grid planes [0, dlo), planes [dlo, ns) are grid
            // planes [nz - dhi, nz); the workspace keeps the whole array at the same offsets
            const int dlo = h.dlo[2], dhi = h.dhi[2];
            const int r0[2] = {lo, std::max(lo, nz - dhi)}, r1[2] = {std::min(hi, dlo), hi};
            for (int part = 0; part < 2; ++part) {
                if (r1[part] <= r0[part]) continue;
                const long long p0 = part == 0 ? r0[0] : dlo + (r0[1] - (nz - dhi));
                const size_t off = (size_t)p0 * per * esz, bytes = (size_t)(r1[part] - r0[part]) * per * esz;
                for (int e = 0; e < 2; ++e) {
                    char* hp = (char*)hpsi[e] + off;
                    char* dp = (char*)dpsi[e] + off;
                    CK(c, to_dev ? cudaMemcpyAsync(dp, hp, bytes, kind, st) : cudaMemcpyAsync(hp, dp, bytes, kind, st));
                }
            }
        }
    // pole state: chunks [component][pole][P / Q] of the box, z slowest inside a chunk
    if (w.zb1 > w.zb0 && home.ade && ws.ade) {
        const long long bxy = (long long)(h.bhi[0] - h.blo[0]) * (h.bhi[1] - h.blo[1]);
        const long long lb = bxy * (w.zb1 - w.zb0);
        const int z0 = std::max(lo, w.zb0), z1 = std::min(hi, w.zb1);
        if (z1 > z0) {
            const size_t bytes = (size_t)(z1 - z0) * bxy * esz;
            for (int q = 0; q < 6 * h.npole; ++q) {
                char* hp = (char*)home.ade + ((size_t)q * h.bcell + (size_t)(z0 - h.blo[2]) * bxy) * esz;
                char* dp = (char*)ws.ade + ((size_t)q * lb + (size_t)(z0 - w.zb0) * bxy) * esz;
                CK(c, to_dev ? cudaMemcpyAsync(dp, hp, bytes, kind, st) : cudaMemcpyAsync(hp, dp, bytes, kind, st));
            }
        }
    }
    return FDTD_OK;
}

// The domain's own host state as a set of home arrays.
fdtd_ctx::Workspace host_state(const DomainHost& h) {
    fdtd_ctx::Workspace hs;
    for (int f = 0; f < 6; ++f) hs.F[f] = h.F[f];
    for (int a = 0; a < 3; ++a)
        for (int s2 = 0; s2 < 2; ++s2) {
            hs.psiE[a][s2] = h.psiE[a][s2];
            hs.psiH[a][s2] = h.psiH[a][s2];
        }
    hs.ade = h.ade;
    return hs;
}

// Copies window or owned planes between the host state and workspace r (to_dev: host -> device
// of the window, materials included; otherwise device -> host of the owned planes).
fdtd_status stream_copy(fdtd_ctx* c, const SlabWin& w, int r, bool to_dev, cudaStream_t st) {
    return window_copy(c, w, host_state(c->doms[0]), c->ws[r], to_dev ? w.wlo : w.zs, to_dev ? w.whi : w.ze, to_dev,
                       true, st);
}

template <typename T>
CellArgs<T> stream_cell_args(const fdtd_ctx* c, int s, bool e_side) {
    const SlabWin w = slab_win(c, s);
    const fdtd_ctx::Workspace& ws = c->ws[s % 3];
    const DomainHost& h = c->doms[0];
    CellArgs<T> ca = make_cell_args<T>(c, 0, e_side);
    for (int f = 0; f < 6; ++f) ca.F[f] = (T*)ws.F[f];
    for (int a = 0; a < 3; ++a) {
        ca.ie[a] = (const T*)ws.ie[ie_first(h, a)];
        for (int s2 = 0; s2 < 2; ++s2) ca.psi[a][s2] = (T*)(e_side ? ws.psiE[a][s2] : ws.psiH[a][s2]);
    }
    ca.n[2] = w.whi - w.wlo;
    ca.kz0 = w.wlo;
    ca.nzg = h.n[2];
    ca.dom = s;
    return ca;
}

// Bytes of the whole forward state of the streamed domain (every part).
size_t state_bytes(const fdtd_ctx* c) {
    size_t b = 0;
    const DomainHost& h = c->doms[0];
    for (int p = 0; p < part_count(h); ++p) b += (size_t)part_size(h, p) * c->esz;
    return b;
}

// The pinned host buffer of the checkpoint of step `now` (taken from the kept buffers, else
// allocated).
fdtd_status ck_alloc(fdtd_ctx* c, long long now) {
    void*& buf = c->ck[now];
    if (buf) return FDTD_OK;
    if (!c->ck_pool.empty()) {
        buf = c->ck_pool.back();
        c->ck_pool.pop_back();
        return FDTD_OK;
    }
    cudaError_t e = cudaHostAlloc(&buf, state_bytes(c), cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->ck.erase(now);
        return fail(c, FDTD_ENOMEM, "pinned host checkpoint allocation failed");
    }
    return FDTD_OK;
}

// Keeps the host forward state (held at step `now`) as the checkpoint of that step, in pinned host
// memory, once every copy of the previous batch has landed.
fdtd_status ck_save(fdtd_ctx* c, long long now) {
    CK(c, cudaStreamSynchronize(c->stream));
    CK(c, cudaStreamSynchronize(c->d2h_stream));
    fdtd_status st = ck_alloc(c, now);
    if (st != FDTD_OK) return st;
    void* buf = c->ck[now];
    const DomainHost& h = c->doms[0];
    size_t off = 0;
    for (int p = 0; p < part_count(h); ++p) {
        const size_t b = (size_t)part_size(h, p) * c->esz;
        if (b) std::memcpy((char*)buf + off, part_ptr(h, 0, p, c->esz), b);
        off += b;
    }
    return FDTD_OK;
}

// A checkpoint buffer seen as a set of home arrays (parts in id order, so the pole parts form one
// contiguous block).
fdtd_ctx::Workspace ck_view(const fdtd_ctx* c, void* buf) {
    const DomainHost& h = c->doms[0];
    fdtd_ctx::Workspace v;
    size_t off = 0;
    for (int p = 0; p < part_count(h); ++p) {
        char* at = (char*)buf + off;
        const long long n = part_size(h, p);
        if (p < 6) v.F[p] = at;
        else if (p < 12) v.psiE[(p - 6) / 2][(p - 6) % 2] = n ? at : nullptr;
        else if (p < 18) v.psiH[(p - 12) / 2][(p - 12) % 2] = n ? at : nullptr;
        else if (p == 18) v.ade = at;
        off += (size_t)n * c->esz;
    }
    return v;
}

// n_steps forward steps of a host-streamed context, in batches of at most sk steps.
template <typename T>
fdtd_status stream_forward(fdtd_ctx* c, int n_steps) {
    fdtd_status st = stream_prepare<T>(c);
    if (st != FDTD_OK) return st;
    const DomainHost& h = c->doms[0];
    const int nsl = slab_count(c);
    const Launch l{c->stream, &c->launches};
    const Dom<T>* sd = (const Dom<T>*)c->d_sdoms;
    StepArgs a;
    a.srcs = c->d_srcs;
    a.mons = c->d_mons;
    a.d_step = c->d_step;
    a.d_ticket = c->d_ticket;
    a.dft_on = c->dft_enabled;
    a.d_base = c->d_base;
    a.offset = 0;
    // the host state may have been written on the caller's stream (set_part, reset)
    CK(c, cudaEventRecord(c->ev_fork, c->stream));
    CK(c, cudaStreamWaitEvent(c->h2d_stream, c->ev_fork, 0));
    auto copy_in = [&](int s) -> fdtd_status {
        const int r = s % 3;
        // the workspace is free once its last slab has been copied out; the window's host planes
        // hold the batch's start state once the previous batch copied out slab s + 1 (in order
        // after slabs s - 1 and s)
        CK(c, cudaStreamWaitEvent(c->h2d_stream, c->ws_free[r], 0));
        CK(c, cudaStreamWaitEvent(c->h2d_stream, c->ev_out[std::min(s + 1, nsl - 1)], 0));
        fdtd_status e = stream_copy(c, slab_win(c, s), r, true, c->h2d_stream);
        if (e != FDTD_OK) return e;
        CK(c, cudaEventRecord(c->ev_in[s], c->h2d_stream));
        return FDTD_OK;
    };
    int left = n_steps;
    long long ck_next = -1;   // the checkpoint this batch's copy-outs also write (its end step), or -1
    while (left > 0) {
        int kb = std::min(left, c->sk);
        const long long ck_written = ck_next;
        ck_next = -1;
        if (c->ck_on) {
            // batches aligned to the checkpoint grid; the state at every batch start on it is kept:
            // the first one copied from the host state, later ones written by the previous batch
            const long long now = c->step + (n_steps - left), rel = now - c->ck_t0;
            if (rel >= 0) {
                kb = (int)std::min<long long>(left, c->sk - rel % c->sk);
                if (rel % c->sk == 0 && now != ck_written) {
                    st = ck_save(c, now);
                    if (st != FDTD_OK) return st;
                }
                if (left > kb) {
                    st = ck_alloc(c, now + kb);
                    if (st != FDTD_OK) return st;
                    ck_next = now + kb;
                }
            }
        }
        st = copy_in(0);
        if (st != FDTD_OK) return st;
        for (int s = 0; s < nsl; ++s) {
            const int r = s % 3;
            // the next window is read before this slab's owned planes are written back
            if (s + 1 < nsl) {
                st = copy_in(s + 1);
                if (st != FDTD_OK) return st;
            }
            CK(c, cudaStreamWaitEvent(c->stream, c->ev_in[s], 0));
            if (s == 0) launch_copy_int(l, c->d_step, c->d_base);
            const CellArgs<T> ce = stream_cell_args<T>(c, s, true), ch = stream_cell_args<T>(c, s, false);
            const SlabWin w = slab_win(c, s);
            const int poles = h.npole > 0 && w.zb1 > w.zb0;
            const int nd = c->dft_enabled ? c->sitem_count[s] : 0;
            const DftItem* items = c->d_sitems ? c->d_sitems + c->sitem_begin[s] : nullptr;
            for (int o = 0; o < kb; ++o) {
                a.offset = o;
                launch_e_cell<T>(l, ce, sd, (T)c->S, a, c->aniso, poles);
                if (nd > 0) launch_dft<T>(l, sd, c->d_mons, items, nd, 0, c->d_base, o);
                launch_h_cell<T>(l, ch, (T)c->S, a);
                if (nd > 0) launch_dft<T>(l, sd, c->d_mons, items, nd, 1, c->d_base, o);
            }
            if (s == nsl - 1) launch_advance(l, c->d_step, kb);
            CK(c, cudaEventRecord(c->ws_done[r], c->stream));
            CK(c, cudaStreamWaitEvent(c->d2h_stream, c->ws_done[r], 0));
            if (s + 1 < nsl) CK(c, cudaStreamWaitEvent(c->d2h_stream, c->ev_in[s + 1], 0));
            st = stream_copy(c, w, r, false, c->d2h_stream);
            if (st != FDTD_OK) return st;
            if (ck_next >= 0) {
                // the owned planes at the batch end are also the next checkpoint's
                st = window_copy(c, w, ck_view(c, c->ck[ck_next]), c->ws[r], w.zs, w.ze, false, false, c->d2h_stream);
                if (st != FDTD_OK) return st;
            }
            CK(c, cudaEventRecord(c->ev_out[s], c->d2h_stream));
            CK(c, cudaEventRecord(c->ws_free[r], c->d2h_stream));
        }
        left -= kb;
    }
    // later work on the caller's stream sees the final host state
    CK(c, cudaStreamWaitEvent(c->stream, c->ev_out[nsl - 1], 0));
    CKL(c);
    return FDTD_OK;
}

// Per-cell transposed-kernel arguments of domain di.
template <typename T>
AdjCellArgs<T> make_adj_args(const fdtd_ctx* c, int di, int* mon) {
    const DomainHost& h = c->doms[di];
    AdjCellArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    for (int f = 0; f < 6; ++f) {
        a.A[f] = (T*)h.A[f];
        a.F[f] = (const T*)h.F[f];
    }
    for (int q = 0; q < 3; ++q) {
        a.ie[q] = (const T*)h.ie[q];
        a.cE[q] = (const T*)h.cE[q];
        a.cH[q] = (const T*)h.cH[q];
        a.n[q] = h.n[q];
        a.dlo[q] = h.dlo[q];
        a.dhi[q] = h.dhi[q];
        a.ns[q] = h.ns[q];
        a.per[q] = h.per[q];
        for (int s2 = 0; s2 < 2; ++s2) {
            a.apsiE[q][s2] = (T*)h.apsiE[q][s2];
            a.apsiH[q][s2] = (T*)h.apsiH[q][s2];
        }
    }
    for (int q = 0; q < 3; ++q) {
        // E side gathers this node and -1: plain past the low slab's last node + 1 and before the
        // high slab; H side gathers this node and +1 and must avoid PEC-held nodes (coordinate 0 of
        // a non-periodic axis)
        const int N = h.n[q], lo = h.ns[q] ? h.dlo[q] : 0, hi = h.ns[q] ? h.dhi[q] : 0;
        a.elo[q] = lo > 0 ? lo + 1 : 0;
        a.ehi[q] = N - hi;
        a.hlo[q] = std::max(lo, h.per[q] ? 0 : 1);
        a.hhi[q] = N - hi - (hi > 0 ? 1 : 0);
    }
    a.dom = di;
    a.kz0 = 0;
    a.nzg = h.n[2];
    for (int q = 0; q < 3; ++q) a.Eb[q] = (T*)h.teb[q];
    if (h.design && h.grad) {
        for (int q = 0; q < 3; ++q) {
            a.glo[q] = h.glo[q];
            a.ghi[q] = h.ghi[q];
        }
        a.grad = h.grad;
        a.gzg = h.glo[2];
        a.gvol = (long long)(h.ghi[0] - h.glo[0]) * (h.ghi[1] - h.glo[1]) * (h.ghi[2] - h.glo[2]);
    }
    // bounding box of the monitor cells that carry an adjoint source, and its injection scratch
    *mon = 0;
    for (int mi : h.mons) {
        const Mon& m = c->mons[mi].m;
        if (!m.cot) continue;
        for (int q = 0; q < 3; ++q) {
            a.mlo[q] = *mon ? std::min(a.mlo[q], m.lo[q]) : m.lo[q];
            a.mhi[q] = *mon ? std::max(a.mhi[q], m.hi[q]) : m.hi[q];
        }
        *mon = 1;
    }
    if (*mon) {
        a.mvol = (long long)(a.mhi[0] - a.mlo[0]) * (a.mhi[1] - a.mlo[1]) * (a.mhi[2] - a.mlo[2]);
        a.inj = (const T*)h.inj;
    }
    return a;
}

// Transposed-kernel arguments of a Bloch domain (its real-part arguments a).
template <typename T>
AdjBlochArgs<T> make_adj_bloch(const fdtd_ctx* c, int di, const AdjCellArgs<T>& a) {
    const DomainHost& h = c->doms[di];
    AdjBlochArgs<T> b;
    b.c = a;
    for (int f = 0; f < 6; ++f) b.AI[f] = (T*)h.AI[f];
    for (int q = 0; q < 2; ++q) {
        b.pr[q] = (T)std::cos(h.bphase[q]);
        b.pi[q] = (T)std::sin(h.bphase[q]);
    }
    return b;
}

// Sizes every domain's injection scratch for the box of its monitors that carry adjoint sources
// (before transposed steps are launched: the launches themselves cannot fail).
fdtd_status prepare_inj(fdtd_ctx* c) {
    for (DomainHost& h : c->doms) {
        bool any = false;
        int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int mi : h.mons) {
            const Mon& m = c->mons[mi].m;
            if (!m.cot) continue;
            for (int q = 0; q < 3; ++q) {
                lo[q] = any ? std::min(lo[q], m.lo[q]) : m.lo[q];
                hi[q] = any ? std::max(hi[q], m.hi[q]) : m.hi[q];
            }
            any = true;
        }
        if (!any) continue;
        const long long need = 6ll * (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
        if (need <= h.inj_cap) continue;
        if (h.inj) {
            CK(c, cudaStreamSynchronize(c->stream));
            dfree(c, h.inj);
            h.inj = nullptr;
            h.inj_cap = 0;
        }
        fdtd_status st = dmalloc(c, &h.inj, (size_t)need * c->esz);
        if (st != FDTD_OK) return st;
        h.inj_cap = need;
    }
    return FDTD_OK;
}

template <typename T>
void adj_once(fdtd_ctx* c, int m) {
    const Launch l = L(c);
    const Dom<T>* dd = (const Dom<T>*)c->d_doms;
    int pgrad = 0;   // some domain collects pole-coefficient cotangents
    for (const auto& h : c->doms) pgrad |= h.pgc_on;
    if (c->cell_mode) {
        // per-cell launch mode: one launch per domain and half-step, E side first (the H side
        // reads the lagged E cotangent it leaves).  The per-cell transposed kernels are launched
        // programmatically (they start while the kernel before them finishes; not under per-launch
        // profiling): these eager launches otherwise leave the GPU idle between half-steps.
        Launch lp = l;
        lp.pdl = !c->prof_on;
        std::vector<AdjCellArgs<T>> args(c->doms.size());
        std::vector<int> mon(c->doms.size(), 0);
        for (int di = 0; di < (int)c->doms.size(); ++di) args[di] = make_adj_args<T>(c, di, &mon[di]);
        // the E-DFT cotangents of step m and the H-DFT ones of step m - 1 over each monitor box, one
        // launch per domain; the H-side launches read the second half of the scratch
        for (int di = 0; di < (int)c->doms.size(); ++di)
            if (mon[di])
                launch_inject_box<T>(l, dd + di, c->d_mons, args[di].mlo, args[di].mhi, 2ll * m,
                                     m >= 1 ? 2ll * (m - 1) + 1 : -1ll, (T*)c->doms[di].inj);
        {
            Prof p(c, FDTD_KERNEL_ADJ_E);
            for (int di = 0; di < (int)c->doms.size(); ++di) {
                const DomainHost& h = c->doms[di];
                if (h.bloch) {
                    launch_adj_e_bloch<T>(l, make_adj_bloch<T>(c, di, args[di]), (T)c->S, c->adj_pending);
                } else if (h.tensor) {
                    // Ebar^{m+1} into Eb, the node-tensor cotangent, then the curl cotangent S S_t Ebar
                    // into the E array for the H side
                    launch_adj_e_cell<T>(l, args[di], dd, c->d_mons, (T)c->S, m, c->adj_pending, 0, mon[di], 0, 1);
                    if (h.design && h.grad) {
                        TensorGradArgs<T> g;
                        std::memset(&g, 0, sizeof(g));
                        for (int q = 0; q < 3; ++q) {
                            g.Eb[q] = (const T*)h.teb[q];
                            g.H[q] = (const T*)h.F[3 + q];
                            g.n[q] = h.n[q];
                            g.per[q] = h.per[q];
                            g.glo[q] = h.glo[q];
                            g.ghi[q] = h.ghi[q];
                        }
                        g.gvol = (long long)(h.ghi[0] - h.glo[0]) * (h.ghi[1] - h.glo[1]) * (h.ghi[2] - h.glo[2]);
                        g.grad = h.grad;
                        launch_tensor_grad<T>(l, tensor_args<T>(c, di, h.teb, h.A), g, (T)c->S);
                    }
                    CellArgs<T> none;
                    std::memset(&none, 0, sizeof(none));
                    launch_tensor_apply<T>(l, tensor_args<T>(c, di, h.teb, h.A), none, (T)c->S, StepArgs{}, 0);
                } else {
                    launch_adj_e_cell<T>(lp, args[di], dd, c->d_mons, (T)c->S, m, c->adj_pending,
                                         h.npole > 0 && h.bcell > 0, mon[di], h.pgc_on, 0);
                }
            }
        }
        for (int di = 0; di < (int)c->doms.size(); ++di)
            if (mon[di]) args[di].inj += 3 * args[di].mvol;
        {
            Prof p(c, FDTD_KERNEL_ADJ_H);
            for (int di = 0; di < (int)c->doms.size(); ++di) {
                if (c->doms[di].bloch)
                    launch_adj_h_bloch<T>(l, make_adj_bloch<T>(c, di, args[di]));
                else
                    launch_adj_h_cell<T>(lp, args[di], dd, c->d_mons, (T)c->S, m, mon[di]);
            }
        }
        return;
    }
    const int ng = (int)c->tiles_gen.size(), ni = (int)c->tiles_int.size();
    // as in step_once: the interior launches run on the auxiliary stream next to the general ones
    const bool fork = c->aux_stream && !c->prof_on && ng > 0 && ni > 0;
    const Launch la{fork ? c->aux_stream : c->stream, &c->launches};
    auto fork_here = [&]() {
        if (!fork) return;
        cudaEventRecord(c->ev_fork, c->stream);
        cudaStreamWaitEvent(c->aux_stream, c->ev_fork, 0);
    };
    auto join_here = [&]() {
        if (!fork) return;
        cudaEventRecord(c->ev_join, c->aux_stream);
        cudaStreamWaitEvent(c->stream, c->ev_join, 0);
    };
    fork_here();
    {
        Prof p(c, FDTD_KERNEL_ADJ_E);
        launch_adj_e<T>(la, dd, c->d_mons, c->d_tiles_int, ni, (T)c->S, m, c->adj_pending, 0, c->aniso, 0);
    }
    {
        Prof p(c, FDTD_KERNEL_ADJ_E);
        launch_adj_e<T>(l, dd, c->d_mons, c->d_tiles_gen, ng, (T)c->S, m, c->adj_pending, 1, 1, pgrad);
    }
    join_here();
    fork_here();
    {
        Prof p(c, FDTD_KERNEL_ADJ_H);
        launch_adj_h<T>(la, dd, c->d_mons, c->d_tiles_int, ni, (T)c->S, m, 0);
    }
    {
        Prof p(c, FDTD_KERNEL_ADJ_H);
        launch_adj_h<T>(l, dd, c->d_mons, c->d_tiles_gen, ng, (T)c->S, m, 1);
    }
    join_here();
}

// ---- host-streamed transposed sweep (Sec. 4.2) -------------------------------------------------
// The transposed sweep runs the slab tiling in reverse.  Batches of kb <= sk steps (aligned to the
// forward checkpoints) run last to first; for each slab its window replays the batch's forward steps
// from the checkpoint at the batch start (keeping every replayed window state: the transposed step m
// reads u^m for the material cotangent), then takes the kb transposed steps from the adjoint state
// at the batch end (monitor cotangents injected over the whole window), completes the last one to
// the natural form and writes its owned planes back; only owned design cells add to the material
// cotangent.  A cut edge of a window acts as a PEC / open end and spoils one more plane per step, so
// the owned planes come out exactly as the resident sweep computes them.  The adjoint state lives in
// two pinned host sets (read at the batch end, written at the batch start).

// Host adjoint sets, the device adjoint window, the replay windows and their descriptors.
template <typename T>
fdtd_status stream_adj_prepare(fdtd_ctx* c) {
    if (c->hadj_ready) return FDTD_OK;
    CK(c, cudaStreamSynchronize(c->stream));
    const DomainHost& h = c->doms[0];
    const long long nxy = (long long)h.n[0] * h.n[1];
    const int nw = std::min(h.n[2], c->sw + 2 * c->sk);
    for (int b = 0; b < 2; ++b) {
        fdtd_ctx::Workspace& hs = c->hadj[b];
        for (int f = 0; f < 6; ++f)
            if (hmalloc(c, &hs.F[f], (size_t)h.ncell * c->esz) != FDTD_OK) return FDTD_ENOMEM;
        for (int a = 0; a < 3; ++a)
            for (int s2 = 0; s2 < 2; ++s2) {
                const long long n = part_size(h, 6 + 2 * a + s2);
                if (n == 0) continue;
                if (hmalloc(c, &hs.psiE[a][s2], (size_t)n * c->esz) != FDTD_OK ||
                    hmalloc(c, &hs.psiH[a][s2], (size_t)n * c->esz) != FDTD_OK)
                    return FDTD_ENOMEM;
            }
        if (h.npole > 0 && h.bcell > 0 && hmalloc(c, &hs.ade, (size_t)6 * h.npole * h.bcell * c->esz) != FDTD_OK)
            return FDTD_ENOMEM;
    }
    const size_t fb = (size_t)nw * nxy * c->esz;
    const size_t ab = (h.npole > 0 && h.bcell > 0)
                          ? 6 * (size_t)h.npole * (h.bhi[0] - h.blo[0]) * (h.bhi[1] - h.blo[1]) *
                                std::min(h.bhi[2] - h.blo[2], nw) * c->esz
                          : 0;
    for (int f = 0; f < 6; ++f)
        if (dmalloc(c, &c->aws.F[f], fb) != FDTD_OK) return FDTD_ENOMEM;
    for (int a = 0; a < 3; ++a)
        for (int s2 = 0; s2 < 2; ++s2) {
            const long long per = psi_plane(h, a, s2);
            if (per == 0) continue;
            const size_t sb = (size_t)per * ((a + 1 + s2) % 3 == 2 ? h.ns[2] : nw) * c->esz;
            if (dmalloc(c, &c->aws.psiE[a][s2], sb) || dmalloc(c, &c->aws.psiH[a][s2], sb)) return FDTD_ENOMEM;
        }
    if (ab && dmalloc(c, &c->aws.ade, ab) != FDTD_OK) return FDTD_ENOMEM;
    c->rws.assign(c->sk, fdtd_ctx::Workspace());
    for (auto& rw : c->rws) {
        for (int f = 0; f < 6; ++f)
            if (dmalloc(c, &rw.F[f], fb) != FDTD_OK) return FDTD_ENOMEM;
        if (ab && dmalloc(c, &rw.ade, ab) != FDTD_OK) return FDTD_ENOMEM;
    }
    // descriptor (s, j): slab s's window with the replayed forward state j and the adjoint window
    const int nsl = slab_count(c);
    std::vector<Dom<T>> hd((size_t)nsl * c->sk);
    for (int s2 = 0; s2 < nsl; ++s2)
        for (int j = 0; j < c->sk; ++j) {
            Dom<T> d = slab_dom<T>(c, s2);
            for (int f = 0; f < 6; ++f) {
                d.F[f] = (T*)c->rws[j].F[f];
                d.A[f] = (T*)c->aws.F[f];
            }
            for (int a = 0; a < 3; ++a)
                for (int q = 0; q < 2; ++q) {
                    d.apsiE[a][q] = (T*)c->aws.psiE[a][q];
                    d.apsiH[a][q] = (T*)c->aws.psiH[a][q];
                }
            d.ade = (T*)c->rws[j].ade;
            d.aade = (T*)c->aws.ade;
            hd[(size_t)s2 * c->sk + j] = d;
        }
    if (dmalloc(c, &c->d_adoms, sizeof(Dom<T>) * hd.size()) != FDTD_OK) return FDTD_ENOMEM;
    CK(c, cudaMemcpy(c->d_adoms, hd.data(), sizeof(Dom<T>) * hd.size(), cudaMemcpyHostToDevice));
    c->hadj_ready = 1;
    return FDTD_OK;
}

// The domain's adjoint parts point at host set b (part access, the injection at the sweep start).
fdtd_status stream_adj_bind(fdtd_ctx* c, int b) {
    DomainHost& h = c->doms[0];
    for (int f = 0; f < 6; ++f) h.A[f] = c->hadj[b].F[f];
    for (int a = 0; a < 3; ++a)
        for (int s2 = 0; s2 < 2; ++s2) {
            h.apsiE[a][s2] = c->hadj[b].psiE[a][s2];
            h.apsiH[a][s2] = c->hadj[b].psiH[a][s2];
        }
    h.aade = c->hadj[b].ade;
    c->hadj_cur = b;
    return sync_doms(c);
}

// Transposed-kernel arguments of slab s's window with replayed forward state j.
template <typename T>
AdjCellArgs<T> window_adj_args(const fdtd_ctx* c, int s, int j, int* mon) {
    const DomainHost& h = c->doms[0];
    const SlabWin w = slab_win(c, s);
    const fdtd_ctx::Workspace& ws = c->ws[s % 3];
    AdjCellArgs<T> a = make_adj_args<T>(c, 0, mon);
    for (int f = 0; f < 6; ++f) {
        a.A[f] = (T*)c->aws.F[f];
        a.F[f] = (const T*)c->rws[j].F[f];
    }
    for (int q = 0; q < 3; ++q) {
        a.ie[q] = (const T*)ws.ie[ie_first(h, q)];
        for (int s2 = 0; s2 < 2; ++s2) {
            a.apsiE[q][s2] = (T*)c->aws.psiE[q][s2];
            a.apsiH[q][s2] = (T*)c->aws.psiH[q][s2];
        }
    }
    a.n[2] = w.whi - w.wlo;
    a.kz0 = w.wlo;
    a.nzg = h.n[2];
    a.dom = s * c->sk + j;
    if (a.grad) {
        // only owned design cells add to the material cotangent
        const int z0 = std::max(h.glo[2], w.zs), z1 = std::min(h.ghi[2], w.ze);
        if (z1 > z0) {
            a.glo[2] = z0 - w.wlo;
            a.ghi[2] = z1 - w.wlo;
        } else {
            a.grad = nullptr;
            for (int q = 0; q < 3; ++q) a.glo[q] = a.ghi[q] = 0;
        }
    }
    return a;
}

template <typename T>
fdtd_status stream_adjoint(fdtd_ctx* c, int n_steps) {
    fdtd_status st = stream_prepare<T>(c);
    if (st != FDTD_OK) return st;
    st = stream_adj_prepare<T>(c);
    if (st != FDTD_OK) return st;
    const DomainHost& h = c->doms[0];
    const int nsl = slab_count(c);
    const Launch l{c->stream, &c->launches};
    const Dom<T>* sd = (const Dom<T>*)c->d_sdoms;
    const Dom<T>* ad = (const Dom<T>*)c->d_adoms;
    const long long nxy = (long long)h.n[0] * h.n[1];
    StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.srcs = c->d_srcs;
    a.mons = c->d_mons;
    a.d_step = c->d_step;
    a.d_ticket = c->d_ticket;
    a.d_base = c->d_base;
    int left = n_steps;
    while (left > 0) {
        const long long te = c->adj_step;
        const long long tb = c->ck_t0 + ((te - 1 - c->ck_t0) / c->sk) * c->sk;
        const int kb = (int)(te - tb);
        auto it = c->ck.find(tb);
        if (te <= c->ck_t0 || kb > left || it == c->ck.end())
            return fail(c, FDTD_ESTATE, "a streamed transposed batch needs the forward checkpoint of step " +
                                            std::to_string(tb) + " and all of its " + std::to_string(kb) + " steps");
        const fdtd_ctx::Workspace ckv = ck_view(c, it->second);
        const int cur = c->hadj_cur, nxt = 1 - cur;
        for (int s2 = 0; s2 < nsl; ++s2) {
            const int r = s2 % 3;
            const SlabWin w = slab_win(c, s2);
            const size_t wb = (size_t)(w.whi - w.wlo) * nxy * c->esz;
            const size_t ab = (w.zb1 > w.zb0) ? 6 * (size_t)h.npole * (h.bhi[0] - h.blo[0]) * (h.bhi[1] - h.blo[1]) *
                                                    (w.zb1 - w.zb0) * c->esz
                                              : 0;
            const int poles = h.npole > 0 && w.zb1 > w.zb0;
            // forward window at the batch start, then its replay (the step index of the sources is
            // the global one: the batch base tb plus the position in the batch)
            st = window_copy(c, w, ckv, c->ws[r], w.wlo, w.whi, true, true, c->stream);
            if (st != FDTD_OK) return st;
            launch_set_int(l, c->d_base, (int)tb);
            const CellArgs<T> ce = stream_cell_args<T>(c, s2, true), ch = stream_cell_args<T>(c, s2, false);
            for (int j = 0; j < kb; ++j) {
                for (int f = 0; f < 6; ++f)
                    CK(c, cudaMemcpyAsync(c->rws[j].F[f], c->ws[r].F[f], wb, cudaMemcpyDeviceToDevice, c->stream));
                if (ab) CK(c, cudaMemcpyAsync(c->rws[j].ade, c->ws[r].ade, ab, cudaMemcpyDeviceToDevice, c->stream));
                if (j + 1 == kb) break;
                a.offset = j;
                launch_e_cell<T>(l, ce, sd, (T)c->S, a, c->aniso, poles);
                launch_h_cell<T>(l, ch, (T)c->S, a);
            }
            // adjoint window at the batch end, kb transposed steps, natural form, owned planes out
            st = window_copy(c, w, c->hadj[cur], c->aws, w.wlo, w.whi, true, false, c->stream);
            if (st != FDTD_OK) return st;
            AdjCellArgs<T> aa;
            for (int j = kb - 1; j >= 0; --j) {
                int mon = 0;
                aa = window_adj_args<T>(c, s2, j, &mon);
                if (mon)
                    launch_inject_box<T>(l, (const Dom<T>*)c->d_doms, c->d_mons, aa.mlo, aa.mhi, 2ll * (tb + j),
                                         tb + j >= 1 ? 2ll * (tb + j - 1) + 1 : -1ll, (T*)h.inj);
                launch_adj_e_cell<T>(l, aa, ad, c->d_mons, (T)c->S, (int)(tb + j), j < kb - 1 ? 1 : 0, poles, mon, 0,
                                     0);
                if (mon) aa.inj += 3 * aa.mvol;
                launch_adj_h_cell<T>(l, aa, ad, c->d_mons, (T)c->S, (int)(tb + j), mon);
            }
            launch_adj_flush_cell<T>(l, aa, ad, (T)c->S, poles, 0);
            st = window_copy(c, w, c->hadj[nxt], c->aws, w.zs, w.ze, false, false, c->stream);
            if (st != FDTD_OK) return st;
        }
        CK(c, cudaStreamSynchronize(c->stream));
        st = stream_adj_bind(c, nxt);
        if (st != FDTD_OK) return st;
        c->adj_step = tb;
        left -= kb;
    }
    CKL(c);
    return FDTD_OK;
}


void drop_graphs(fdtd_ctx* c) {
    bool any = false;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) any = any || c->graph[a][b];
    if (any) cudaStreamSynchronize(c->stream);   // no replay of a graph in flight when it goes
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            if (c->graph[a][b]) {
                cudaGraphExecDestroy(c->graph[a][b]);
                c->graph[a][b] = nullptr;
            }
}

// Captures kGraphSteps forward steps on a private stream (the step index, source amplitudes
// and DFT phases are read from device memory, so one graph serves every replay).
fdtd_status build_graph(fdtd_ctx* c) {
    const int a = c->dft_enabled, b = c->energy_on;
    if (c->graph[a][b]) return FDTD_OK;
    if (!c->cap_stream) CK(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    const long long l0 = c->launches;
    CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int s = 0; s < kGraphSteps; ++s) {
        if (c->dtype == FDTD_F32)
            step_once<float>(c, c->cap_stream, s, s == 0, s == kGraphSteps - 1);
        else
            step_once<double>(c, c->cap_stream, s, s == 0, s == kGraphSteps - 1);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    const long long captured = c->launches - l0;   // kernel launches of one replay
    c->launches = l0;
    if (e != cudaSuccess) return fail(c, FDTD_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->graph[a][b], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph[a][b] = nullptr;
        return fail(c, FDTD_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    c->graph_launches[a][b] = captured;
    return FDTD_OK;
}

fdtd_status flush_adjoint(fdtd_ctx* c) {
    if (!c->adj_pending) return FDTD_OK;
    if (c->cell_mode) {
        // the per-cell form, with the arithmetic of the per-cell transposed kernels
        for (int di = 0; di < (int)c->doms.size(); ++di) {
            int mon = 0;
            const DomainHost& h = c->doms[di];
            const int poles = h.npole > 0 && h.bcell > 0;
            if (c->dtype == FDTD_F32)
                launch_adj_flush_cell<float>(L(c), make_adj_args<float>(c, di, &mon), (const Dom<float>*)c->d_doms,
                                             (float)c->S, poles, h.tensor);
            else
                launch_adj_flush_cell<double>(L(c), make_adj_args<double>(c, di, &mon), (const Dom<double>*)c->d_doms,
                                              c->S, poles, h.tensor);
        }
    } else if (c->dtype == FDTD_F32) {
        launch_adj_flush<float>(L(c), (const Dom<float>*)c->d_doms, c->d_tiles, (int)c->tiles.size(), (float)c->S);
    } else {
        launch_adj_flush<double>(L(c), (const Dom<double>*)c->d_doms, c->d_tiles, (int)c->tiles.size(), c->S);
    }
    for (int di = 0; di < (int)c->doms.size(); ++di) {
        if (!c->doms[di].bloch) continue;   // the imaginary E part of a Bloch domain
        int mon = 0;
        if (c->dtype == FDTD_F32)
            launch_adj_flush_bloch<float>(L(c), make_adj_bloch<float>(c, di, make_adj_args<float>(c, di, &mon)),
                                          (float)c->S);
        else
            launch_adj_flush_bloch<double>(L(c), make_adj_bloch<double>(c, di, make_adj_args<double>(c, di, &mon)),
                                           c->S);
    }
    CKL(c);
    c->adj_pending = 0;
    return FDTD_OK;
}

fdtd_status set_device_step(fdtd_ctx* c, long long s) {
    c->h_step_tmp = (int)s;
    CK(c, cudaMemcpyAsync(c->d_step, &c->h_step_tmp, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return FDTD_OK;
}

// Layout of one part in a BF16 snapshot: n bf16 codes, then (from the next 4-byte boundary, so
// that parts of odd size keep their scales aligned) one FP32 scale per plane.
size_t bf16_scale_off(long long n) { return ((size_t)n * 2 + 3) & ~(size_t)3; }
size_t bf16_part_bytes(long long n, long long planes) { return bf16_scale_off(n) + (size_t)planes * 4; }

size_t snapshot_bytes(const fdtd_ctx* c, int codec) {
    size_t tot = 0;
    for (const auto& d : c->doms)
        for (int p = 0; p < part_count(d); ++p) {
            const long long n = part_size(d, p);
            if (n == 0) continue;
            const size_t b = codec == FDTD_CODEC_BF16 ? bf16_part_bytes(n, part_planes(d, p)) : (size_t)n * c->esz;
            tot += (b + 255) & ~(size_t)255;
        }
    return tot;
}

// True when every array of a material is in pinned (page-locked) host memory.
bool host_material(const fdtd_material& m) {
    auto pinned = [](const void* p) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return at.type == cudaMemoryTypeHost;
    };
    for (int a = 0; a < 3; ++a)
        if (!pinned(m.inv_eps[a])) return false;
    return m.n_poles == 0 || pinned(m.pole_mask);
}

// Device workspaces, copy streams and events of a host-streamed context.
fdtd_status stream_alloc(fdtd_ctx* c) {
    const DomainHost& d = c->doms[0];
    const long long nxy = (long long)d.n[0] * d.n[1];
    const int nw = std::min(d.n[2], c->sw + 2 * c->sk);
    const size_t fb = (size_t)nw * nxy * c->esz;
    for (int r = 0; r < 3; ++r) {
        fdtd_ctx::Workspace& w = c->ws[r];
        for (int f = 0; f < 6; ++f)
            if (dmalloc(c, &w.F[f], fb) != FDTD_OK) return FDTD_ENOMEM;
        // one eps^-1 window per distinct array (an isotropic medium needs one; a later material
        // with more distinct arrays gets the others in stream_prepare)
        for (int a = 0; a < 3; ++a)
            if (ie_first(d, a) == a && dmalloc(c, &w.ie[a], fb) != FDTD_OK) return FDTD_ENOMEM;
        for (int a = 0; a < 3; ++a)
            for (int s = 0; s < 2; ++s) {
                const long long per = psi_plane(d, a, s);
                const size_t sb = (size_t)per * ((a + 1 + s) % 3 == 2 ? d.ns[2] : nw) * c->esz;
                if (dmalloc(c, &w.psiE[a][s], sb) || dmalloc(c, &w.psiH[a][s], sb)) return FDTD_ENOMEM;
            }
        if (d.npole > 0 && d.bcell > 0) {
            if (dmalloc(c, &w.mask, (size_t)nw * nxy) != FDTD_OK) return FDTD_ENOMEM;
            const size_t ab = 6 * (size_t)d.npole * (d.bhi[0] - d.blo[0]) * (d.bhi[1] - d.blo[1]) *
                              std::min(d.bhi[2] - d.blo[2], nw) * c->esz;
            if (dmalloc(c, &w.ade, ab) != FDTD_OK) return FDTD_ENOMEM;
        }
    }
    CK(c, cudaStreamCreateWithFlags(&c->h2d_stream, cudaStreamNonBlocking));
    CK(c, cudaStreamCreateWithFlags(&c->d2h_stream, cudaStreamNonBlocking));
    for (int r = 0; r < 3; ++r) {
        CK(c, cudaEventCreateWithFlags(&c->ws_done[r], cudaEventDisableTiming));
        CK(c, cudaEventCreateWithFlags(&c->ws_free[r], cudaEventDisableTiming));
    }
    const int nsl = slab_count(c);
    c->ev_in.assign(nsl, nullptr);
    c->ev_out.assign(nsl, nullptr);
    for (int s = 0; s < nsl; ++s) {
        CK(c, cudaEventCreateWithFlags(&c->ev_in[s], cudaEventDisableTiming));
        CK(c, cudaEventCreateWithFlags(&c->ev_out[s], cudaEventDisableTiming));
    }
    return FDTD_OK;
}

}  // namespace

namespace {

template <typename T>
void time_launches_t(fdtd_ctx* c, cudaStream_t st, int which, int n, long long* counter) {
    const Launch l{st, counter};
    const Dom<T>* dd = (const Dom<T>*)c->d_doms;
    StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.srcs = c->d_srcs;
    a.mons = c->d_mons;
    a.d_step = c->d_step;
    a.d_ticket = c->d_ticket;
    a.dft_on = c->dft_enabled;
    a.d_base = c->d_base;
    a.offset = 0;
    // the updates store their monitor samples as in a step (into slot 0)
    a.ring = c->ring_on && c->dft_enabled && c->n_dft_items > 0 ? 1 : 0;
    for (int r = 0; r < n; ++r) {
        if (which == 0) {
            for (int di = 0; di < (int)c->doms.size(); ++di) {
                const DomainHost& h = c->doms[di];
                launch_e_cell<T>(l, make_cell_args<T>(c, di, true), dd, (T)c->S, a, c->aniso, h.npole > 0 && h.bcell > 0);
            }
        } else if (which == 1) {
            for (int di = 0; di < (int)c->doms.size(); ++di) launch_h_cell<T>(l, make_cell_args<T>(c, di, false), (T)c->S, a);
        } else if (which == 2) {
            launch_dft<T>(l, dd, c->d_mons, c->d_dft_items, c->n_dft_items, 0, c->d_base, 0);
        } else if (which == 5) {
            launch_dft_ring<T>(l, c->d_mons, c->d_dft_items, c->n_dft_items, c->d_base, kGraphSteps);
        } else {
            // transposed half-steps at adjoint index m = step count (no pending deferral)
            for (int di = 0; di < (int)c->doms.size(); ++di) {
                const DomainHost& h = c->doms[di];
                int mon = 0;
                const AdjCellArgs<T> aa = make_adj_args<T>(c, di, &mon);
                const int m = (int)std::max(0ll, c->adj_step - 1);
                if (which == 3)
                    launch_adj_e_cell<T>(l, aa, dd, c->d_mons, (T)c->S, m, 1, h.npole > 0 && h.bcell > 0, mon, h.pgc_on,
                                         0);
                else
                    launch_adj_h_cell<T>(l, aa, dd, c->d_mons, (T)c->S, m, mon);
            }
        }
    }
}

}  // namespace

extern "C" {

const char* fdtd_version(void) { return "gbfdtd 0.1 (sm_103a)"; }

static thread_local std::string g_create_err;

const char* fdtd_last_error(const fdtd_ctx* ctx) {
    if (!ctx) return g_create_err.c_str();
    return ctx->err.c_str();
}

static fdtd_status create_impl(int32_t n_domains, const fdtd_grid* grids, const fdtd_cpml* cpml,
                               const fdtd_material* materials, void* stream, fdtd_ctx** out, int streamed, int sw,
                               int sk) {
    if (!out || n_domains < 1 || !grids || !cpml || !materials) return FDTD_EINVAL;
    *out = nullptr;
    fdtd_ctx* c = new fdtd_ctx();
    c->stream = (cudaStream_t)stream;
    c->streamed = streamed;
    c->sw = sw;
    c->sk = sk;
    c->dtype = grids[0].dtype;
    g_create_err.clear();
    auto bail = [&](fdtd_status st) {
        g_create_err = c->err.empty() ? std::string("fdtd_create failed with status ") + std::to_string((int)st) : c->err;
        c->poisoned = 0;
        fdtd_destroy(c);
        return st;
    };
    if (c->dtype != FDTD_F32 && c->dtype != FDTD_F64) return bail(FDTD_EINVAL);
    c->esz = c->dtype == FDTD_F32 ? 4 : 8;
    c->S = grids[0].courant;
    for (int di = 0; di < n_domains; ++di) {
        const fdtd_grid& g = grids[di];
        if (g.dtype != c->dtype || g.courant != c->S) return bail(FDTD_EINVAL);
        if (g.nx < 2 || g.ny < 2 || g.nz < 2 || !(g.dx > 0) || !(g.courant > 0)) return bail(FDTD_EINVAL);
        if ((long long)g.nx * g.ny * g.nz >= (1ll << 40) || g.nx > 65535 || g.ny > 65535) return bail(FDTD_EINVAL);
        if (g.dt != 0.0 && std::fabs(g.dt - g.courant * g.dx) > 1e-12 * g.courant * g.dx) return bail(FDTD_EINVAL);
        if (g.courant * std::sqrt(3.0) > 0.99 * (1.0 + 1e-12)) return bail(FDTD_ECFL);
        const fdtd_cpml& p = cpml[di];
        for (int q = 0; q < 3; ++q) {
            const int n = q == 0 ? g.nx : (q == 1 ? g.ny : g.nz);
            if (p.cells[2 * q] < 0 || p.cells[2 * q + 1] < 0 || p.cells[2 * q] + p.cells[2 * q + 1] > n - 2)
                return bail(FDTD_EINVAL);
        }
        // the per-cell kernels index within a z-plane and within a CPML memory array in 32 bits
        const long long nn[3] = {g.nx, g.ny, g.nz};
        bool fits = nn[0] * nn[1] < (1ll << 31);
        for (int q = 0; q < 3; ++q)
            fits = fits && (long long)(p.cells[2 * q] + p.cells[2 * q + 1]) * nn[(q + 1) % 3] * nn[(q + 2) % 3] < (1ll << 31);
        if (!fits) {
            c->err = "a z-plane or a CPML memory array holds 2^31 or more cells";
            return bail(FDTD_EINVAL);
        }
        if ((p.cells[0] | p.cells[1] | p.cells[2] | p.cells[3] | p.cells[4] | p.cells[5]) &&
            (!(p.m >= 0) || !(p.kappa_max >= 1) || !(p.alpha_max >= 0)))
            return bail(FDTD_EINVAL);
        if (check_material(c, materials[di]) != FDTD_OK) return bail(FDTD_EINVAL);
        if (streamed && !host_material(materials[di])) {
            c->err = "a host-streamed context needs its eps^-1 arrays and pole mask in pinned host memory";
            return bail(FDTD_EINVAL);
        }
    }
    // scratch
    cudaError_t e = cudaMalloc((void**)&c->d_flag, 64);
    if (e != cudaSuccess) return bail(FDTD_ECUDA);
    c->owned.push_back(c->d_flag);
    e = cudaMalloc((void**)&c->d_box, 64);
    if (e != cudaSuccess) return bail(FDTD_ECUDA);
    c->owned.push_back(c->d_box);
    e = cudaMalloc((void**)&c->d_step, 64);
    if (e != cudaSuccess) return bail(FDTD_ECUDA);
    c->owned.push_back(c->d_step);
    if (cudaMemsetAsync(c->d_step, 0, 64, c->stream) != cudaSuccess) return bail(FDTD_ECUDA);
    e = cudaMalloc((void**)&c->d_ticket, 64);
    if (e != cudaSuccess) return bail(FDTD_ECUDA);
    c->owned.push_back(c->d_ticket);
    if (cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->dft_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_e, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_h, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_de, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_dh, cudaEventDisableTiming) != cudaSuccess)
        return bail(FDTD_ECUDA);
    e = cudaMalloc((void**)&c->d_base, 64);
    if (e != cudaSuccess) return bail(FDTD_ECUDA);
    c->owned.push_back(c->d_base);
    if (cudaMemsetAsync(c->d_ticket, 0, 64, c->stream) != cudaSuccess) return bail(FDTD_ECUDA);

    // domain geometry, pole boxes and the memory plan
    c->doms.resize(n_domains);
    size_t plan = 0;
    for (int di = 0; di < n_domains; ++di) {
        DomainHost& d = c->doms[di];
        const fdtd_grid& g = grids[di];
        d.n[0] = g.nx;
        d.n[1] = g.ny;
        d.n[2] = g.nz;
        d.ncell = (long long)g.nx * g.ny * g.nz;
        d.cpml = cpml[di];
        for (int q = 0; q < 3; ++q) {
            d.dlo[q] = cpml[di].cells[2 * q];
            d.dhi[q] = cpml[di].cells[2 * q + 1];
            d.ns[q] = d.dlo[q] + d.dhi[q];
        }
        const fdtd_material& m = materials[di];
        for (int a = 0; a < 3; ++a) d.ie[a] = m.inv_eps[a];
        d.npole = m.n_poles;
        for (int p = 0; p < m.n_poles; ++p) d.poles[p] = m.poles[p];
        d.mask = m.n_poles > 0 ? m.pole_mask : nullptr;
        if (d.mask) {
            fdtd_status st = mask_box(c, d.mask, d.n, d.blo, d.bhi);
            if (st != FDTD_OK) return bail(st);
        }
        d.bcell = (long long)(d.bhi[0] - d.blo[0]) * (d.bhi[1] - d.blo[1]) * (d.bhi[2] - d.blo[2]);
        if (d.bcell == 0) {
            d.npole = 0;
            d.mask = nullptr;
        }
        if (streamed) {
            // three workspaces of one window each (fields, eps^-1, CPML memories, mask, pole state)
            const long long nxy = (long long)d.n[0] * d.n[1];
            const int nw = std::min(d.n[2], sw + 2 * sk);
            const int nie = d.ie[0] == d.ie[1] && d.ie[1] == d.ie[2] ? 1 : 3;
            size_t ws = (size_t)nw * nxy * ((6 + nie) * c->esz + (d.npole > 0 ? 1 : 0));
            ws += 4 * ((size_t)nw * d.n[1] * d.ns[0] + (size_t)nw * d.ns[1] * d.n[0] + (size_t)d.ns[2] * nxy) * c->esz;
            if (d.bcell > 0)
                ws += 6 * (size_t)d.npole * (d.bhi[0] - d.blo[0]) * (d.bhi[1] - d.blo[1]) *
                      std::min(d.bhi[2] - d.blo[2], nw) * c->esz;
            plan += 3 * ws;
            for (int q = 0; q < 3; ++q) plan += 6 * d.n[q] * c->esz;
            continue;
        }
        plan += 12 * (size_t)d.ncell * c->esz;
        for (int q = 0; q < 3; ++q) plan += 8 * (size_t)(d.ncell / d.n[q]) * d.ns[q] * c->esz + 6 * d.n[q] * c->esz;
        plan += 2 * 6 * (size_t)d.npole * d.bcell * c->esz;
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return bail(FDTD_ECUDA);
    if (plan + (64ull << 20) > free_b) {
        c->err = "memory plan " + std::to_string(plan) + " B exceeds free device memory " + std::to_string(free_b) + " B";
        return bail(FDTD_ENOMEM);
    }
    for (int di = 0; di < n_domains; ++di) {
        DomainHost& d = c->doms[di];
        const size_t fb = (size_t)d.ncell * c->esz;
        if (streamed) {
            // the state lives in pinned host memory; no adjoint arrays
            for (int f = 0; f < 6; ++f)
                if (hmalloc(c, &d.F[f], fb) != FDTD_OK) return bail(FDTD_ENOMEM);
            for (int a = 0; a < 3; ++a)
                for (int s = 0; s < 2; ++s) {
                    const int ax = (a + 1 + s) % 3;
                    const size_t sb = (size_t)(d.ncell / d.n[ax]) * d.ns[ax] * c->esz;
                    if (hmalloc(c, &d.psiE[a][s], sb) || hmalloc(c, &d.psiH[a][s], sb)) return bail(FDTD_ENOMEM);
                }
        }
        for (int f = 0; f < 6 && !streamed; ++f) {
            if (dmalloc(c, &d.F[f], fb) != FDTD_OK) return bail(FDTD_ENOMEM);
            if (dmalloc(c, &d.A[f], fb) != FDTD_OK) return bail(FDTD_ENOMEM);
        }
        for (int a = 0; a < 3 && !streamed; ++a)
            for (int s = 0; s < 2; ++s) {
                const int ax = (a + 1 + s) % 3;
                const size_t sb = (size_t)(d.ncell / d.n[ax]) * d.ns[ax] * c->esz;
                if (dmalloc(c, &d.psiE[a][s], sb) || dmalloc(c, &d.psiH[a][s], sb) || dmalloc(c, &d.apsiE[a][s], sb) ||
                    dmalloc(c, &d.apsiH[a][s], sb))
                    return bail(FDTD_ENOMEM);
            }
        for (int q = 0; q < 3; ++q) {
            std::vector<double> te, th;
            cpml_table(d.cpml, q, d.n[q], c->S, false, te);
            cpml_table(d.cpml, q, d.n[q], c->S, true, th);
            const size_t tb = te.size() * c->esz;
            if (dmalloc(c, &d.cE[q], tb) || dmalloc(c, &d.cH[q], tb)) return bail(FDTD_ENOMEM);
            std::vector<float> fe(te.begin(), te.end()), fh(th.begin(), th.end());
            const void* se = c->dtype == FDTD_F32 ? (const void*)fe.data() : (const void*)te.data();
            const void* sh = c->dtype == FDTD_F32 ? (const void*)fh.data() : (const void*)th.data();
            if (cudaMemcpyAsync(d.cE[q], se, tb, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
                cudaMemcpyAsync(d.cH[q], sh, tb, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
                cudaStreamSynchronize(c->stream) != cudaSuccess)
                return bail(FDTD_ECUDA);
        }
        const size_t ab = 6 * (size_t)d.npole * d.bcell * c->esz;
        if (streamed) {
            if (hmalloc(c, &d.ade, ab)) return bail(FDTD_ENOMEM);
        } else if (dmalloc(c, &d.ade, ab) || dmalloc(c, &d.aade, ab)) {
            return bail(FDTD_ENOMEM);
        }
    }
    if (streamed) {
        fdtd_status st = stream_alloc(c);
        if (st != FDTD_OK) return bail(st);
    }
    const size_t domb = (c->dtype == FDTD_F32 ? sizeof(Dom<float>) : sizeof(Dom<double>)) * n_domains;
    if (dmalloc(c, &c->d_doms, domb) != FDTD_OK) return bail(FDTD_ENOMEM);
    build_tiles(c);
    for (int di = 0; di < n_domains; ++di) {
        const DomainHost& d = c->doms[di];
        if (d.ie[0] != d.ie[1] || d.ie[1] != d.ie[2]) c->aniso = 1;
    }
    if (upload_tiles(c) != FDTD_OK) return bail(FDTD_ECUDA);
    if (sync_doms(c) != FDTD_OK) return bail(FDTD_ECUDA);
    for (int di = 0; di < n_domains; ++di) {
        fdtd_status st = admission(c, di);
        if (st != FDTD_OK) return bail(st);
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(FDTD_ECUDA);
    *out = c;
    return FDTD_OK;
}

fdtd_status fdtd_create(int32_t n_domains, const fdtd_grid* grids, const fdtd_cpml* cpml,
                        const fdtd_material* materials, void* stream, fdtd_ctx** out) {
    return create_impl(n_domains, grids, cpml, materials, stream, out, 0, 0, 0);
}

fdtd_status fdtd_create_streamed(const fdtd_grid* grid, const fdtd_cpml* cpml, const fdtd_material* material,
                                 int32_t slab, int32_t halo, void* stream, fdtd_ctx** out) {
    if (!out) return FDTD_EINVAL;
    *out = nullptr;
    g_create_err.clear();
    if (halo < 1 || slab < halo) {
        g_create_err = "host streaming needs halo >= 1 and slab >= halo";
        return FDTD_EINVAL;
    }
    return create_impl(1, grid, cpml, material, stream, out, 1, slab, halo);
}

static void prof_release(fdtd_ctx* ctx);

fdtd_status fdtd_destroy(fdtd_ctx* ctx) {
    if (!ctx) return FDTD_OK;
    cudaStreamSynchronize(ctx->stream);
    prof_release(ctx);
    drop_graphs(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->dft_stream) cudaStreamDestroy(ctx->dft_stream);
    for (cudaEvent_t e : {ctx->ev_e, ctx->ev_h, ctx->ev_de, ctx->ev_dh})
        if (e) cudaEventDestroy(e);
    for (cudaStream_t st : {ctx->h2d_stream, ctx->d2h_stream})
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
    for (int r = 0; r < 3; ++r)
        for (cudaEvent_t e : {ctx->ws_done[r], ctx->ws_free[r]})
            if (e) cudaEventDestroy(e);
    for (auto* v : {&ctx->ev_in, &ctx->ev_out})
        for (cudaEvent_t e : *v)
            if (e) cudaEventDestroy(e);
    for (void* p : ctx->owned) cudaFree(p);
    for (void* p : ctx->host_owned) cudaFreeHost(p);
    for (auto& kv : ctx->ck) cudaFreeHost(kv.second);
    for (void* p : ctx->ck_pool) cudaFreeHost(p);
    for (auto& s : ctx->slots) cudaFree(s.second.buf);
    delete ctx;
    return FDTD_OK;
}

fdtd_status fdtd_dft_flux(fdtd_ctx* ctx, int32_t monitor, double* flux_host, int32_t n_freq) {
    GUARD(ctx);
    if (monitor < 0 || monitor >= (int)ctx->mons.size() || !flux_host)
        return fail(ctx, FDTD_EINVAL, "bad monitor or output");
    const Mon& m = ctx->mons[monitor].m;
    if (n_freq != m.nf) return fail(ctx, FDTD_EINVAL, "n_freq differs from the monitor's frequency count");
    if (m.hi[2] - m.lo[2] != 2) return fail(ctx, FDTD_EINVAL, "a flux monitor spans exactly two z-planes");
    int slots[4] = {-1, -1, -1, -1};
    const int want[4] = {0, 1, 3, 4};   // Ex, Ey, Hx, Hy
    for (int ci = 0; ci < m.ncomp; ++ci)
        for (int q = 0; q < 4; ++q)
            if (m.comps[ci] == want[q]) slots[q] = ci;
    for (int q = 0; q < 4; ++q)
        if (slots[q] < 0) return fail(ctx, FDTD_EINVAL, "a flux monitor records Ex, Ey, Hx and Hy");
    double* d_out = nullptr;
    fdtd_status st = dmalloc(ctx, (void**)&d_out, sizeof(double) * m.nf);
    if (st != FDTD_OK) return st;
    launch_flux(L(ctx), ctx->d_mons + monitor, m.nf, slots, d_out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(flux_host, d_out, sizeof(double) * m.nf, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, d_out);
    if (e != cudaSuccess) return fail(ctx, FDTD_ECUDA, std::string("flux: ") + cudaGetErrorString(e));
    return FDTD_OK;
}

fdtd_status fdtd_set_periodic(fdtd_ctx* ctx, int32_t domain, const int32_t periodic[3]) {
    GUARD(ctx);
    if (!valid_dom(ctx, domain) || !periodic) return fail(ctx, FDTD_EINVAL, "bad domain or periodic flags");
    DomainHost& d = ctx->doms[domain];
    if (periodic[2]) return fail(ctx, FDTD_EINVAL, "z cannot be periodic (x and y only)");
    for (int q = 0; q < 2; ++q)
        if (periodic[q] && (d.dlo[q] || d.dhi[q] || d.n[q] < 2))
            return fail(ctx, FDTD_EINVAL, "a periodic axis needs no CPML on its faces and at least 2 cells");
    for (int q = 0; q < 3; ++q) d.per[q] = periodic[q] ? 1 : 0;
    return sync_doms(ctx);
}

fdtd_status fdtd_set_tensor(fdtd_ctx* ctx, int32_t domain, const void* const inv_eps[6]) {
    GUARD(ctx);
    NOT_STREAMED(ctx);
    if (!valid_dom(ctx, domain)) return fail(ctx, FDTD_EINVAL, "bad domain");
    DomainHost& d = ctx->doms[domain];
    // a design box's buffer holds [3][cells] for the diagonal eps^-1 and [6][nodes] for tensors: a
    // change between the two removes the box, so that no launch writes past a buffer of the other form
    auto drop_design = [&]() -> fdtd_status {
        if (!d.design) return FDTD_OK;
        d.design = 0;
        d.grad = nullptr;
        return sync_doms(ctx);
    };
    if (!inv_eps) {
        if (d.tensor) {
            drop_graphs(ctx);   // captured steps change
            fdtd_status st = drop_design();
            if (st != FDTD_OK) return st;
        }
        d.tensor = 0;
        return FDTD_OK;
    }
    for (int q = 0; q < 6; ++q)
        if (!inv_eps[q]) return fail(ctx, FDTD_EINVAL, "a tensor needs its six component arrays");
    if (d.bloch || d.npole > 0) return fail(ctx, FDTD_EINVAL, "a tensor domain has no poles and no Bloch phase");
    if (ctx->energy_on || d.rec)
        return fail(ctx, FDTD_EINVAL, "tensor domains take no energy record and no interface record");
    const size_t bytes = (size_t)d.ncell * ctx->esz;
    fdtd_status st = FDTD_OK;
    if (!d.tn[0]) {
        for (int q = 0; q < 6 && st == FDTD_OK; ++q) st = dmalloc(ctx, &d.tn[q], bytes);
        for (int q = 0; q < 3 && st == FDTD_OK; ++q) st = dmalloc(ctx, &d.tcur[q], bytes);
        for (int q = 0; q < 3 && st == FDTD_OK; ++q) st = dmalloc(ctx, &d.teb[q], bytes);
        if (st != FDTD_OK) return st;
    }
    drop_graphs(ctx);   // captured steps change
    st = drop_design();
    if (st != FDTD_OK) return st;
    d.tensor = 0;
    for (int q = 0; q < 6; ++q) CK(ctx, cudaMemcpyAsync(d.tn[q], inv_eps[q], bytes, cudaMemcpyDefault, ctx->stream));
    // the admission rule, node by node
    CK(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(unsigned long long), ctx->stream));
    if (ctx->dtype == FDTD_F32)
        launch_tensor_admission<float>(L(ctx), tensor_args<float>(ctx, domain, d.tcur, d.tcur), d.dlo, d.dhi, d.ns,
                                       ctx->d_flag);
    else
        launch_tensor_admission<double>(L(ctx), tensor_args<double>(ctx, domain, d.tcur, d.tcur), d.dlo, d.dhi, d.ns,
                                        ctx->d_flag);
    CKL(ctx);
    unsigned long long bad = 0;
    CK(ctx, cudaMemcpyAsync(&bad, ctx->d_flag, sizeof(bad), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (bad)
        return fail(ctx, FDTD_ETENSOR,
                    "domain " + std::to_string(domain) + ": " + std::to_string(bad) +
                        " nodes hold a tensor the admission rule rejects (eps below one, not positive definite, or "
                        "inside a CPML face whose normal is no principal axis or has the intermediate eigenvalue)");
    ctx->cell_mode = 1;
    d.tensor = 1;
    return FDTD_OK;
}

fdtd_status fdtd_set_bloch(fdtd_ctx* ctx, int32_t domain, const double phase[2]) {
    GUARD(ctx);
    NOT_STREAMED(ctx);
    if (!ctx->cell_mode || ctx->energy_on)
        return fail(ctx, FDTD_EINVAL, "Bloch domains step in launch mode 4 without an energy record");
    if (!valid_dom(ctx, domain) || !phase || !std::isfinite(phase[0]) || !std::isfinite(phase[1]))
        return fail(ctx, FDTD_EINVAL, "bad domain or phase");
    DomainHost& d = ctx->doms[domain];
    for (int q = 0; q < 2; ++q)
        if (phase[q] != 0.0 && !d.per[q])
            return fail(ctx, FDTD_EINVAL, "a Bloch phase needs a periodic axis (fdtd_set_periodic first)");
    if (d.ns[0] || d.ns[1] || d.ns[2] || d.npole > 0 || !d.mons.empty() || d.design || d.tensor)
        return fail(ctx, FDTD_EINVAL, "a Bloch domain has no CPML slabs, poles, DFT monitors, design box or tensors");
    if (!d.bloch) {
        // the state gains six parts: snapshots and the snapshot part table start afresh
        fdtd_status st = fdtd_snapshots_free(ctx);
        if (st != FDTD_OK) return st;
        if (ctx->d_snapsegs) {
            dfree(ctx, ctx->d_snapsegs);
            ctx->d_snapsegs = nullptr;
            ctx->n_snapsegs = 0;
        }
        for (int f = 0; f < 6; ++f) {
            st = dmalloc(ctx, &d.FI[f], (size_t)d.ncell * ctx->esz);
            if (st == FDTD_OK) st = dmalloc(ctx, &d.AI[f], (size_t)d.ncell * ctx->esz);
            if (st != FDTD_OK) return st;
        }
        d.bloch = 1;
    }
    d.bphase[0] = phase[0];
    d.bphase[1] = phase[1];
    drop_graphs(ctx);   // captured launches hold the kernels and phases of the old configuration
    return FDTD_OK;
}

fdtd_status fdtd_set_material(fdtd_ctx* ctx, int32_t domain, const fdtd_material* m) {
    GUARD(ctx);
    if (!valid_dom(ctx, domain) || !m) return fail(ctx, FDTD_EINVAL, "bad domain or material");
    fdtd_status st = check_material(ctx, *m);
    if (st != FDTD_OK) return st;
    if (ctx->streamed && !host_material(*m))
        return fail(ctx, FDTD_EINVAL, "a host-streamed context needs its materials in pinned host memory");
    DomainHost& d = ctx->doms[domain];
    if (m->n_poles != d.npole) return fail(ctx, FDTD_EINVAL, "the pole count cannot change after create");
    if (d.npole > 0) {
        int lo[3], hi[3];
        st = mask_box(ctx, m->pole_mask, d.n, lo, hi);
        if (st != FDTD_OK) return st;
        for (int q = 0; q < 3; ++q)
            if (hi[q] > lo[q] && (lo[q] < d.blo[q] || hi[q] > d.bhi[q]))
                return fail(ctx, FDTD_EINVAL, "dispersive cells outside the pole-state box chosen at create");
    }
    const void* old[3] = {d.ie[0], d.ie[1], d.ie[2]};
    const uint8_t* oldm = d.mask;
    fdtd_pole oldp[kMaxPole];
    std::memcpy(oldp, d.poles, sizeof(oldp));
    for (int a = 0; a < 3; ++a) d.ie[a] = m->inv_eps[a];
    for (int p = 0; p < m->n_poles; ++p) d.poles[p] = m->poles[p];
    if (d.npole > 0) d.mask = m->pole_mask;
    if (d.ie[0] != d.ie[1] || d.ie[1] != d.ie[2]) ctx->aniso = 1;
    st = admission(ctx, domain);
    if (st != FDTD_OK) {
        for (int a = 0; a < 3; ++a) d.ie[a] = old[a];
        d.mask = oldm;
        std::memcpy(d.poles, oldp, sizeof(oldp));
        return st;
    }
    return sync_doms(ctx);
}

fdtd_status fdtd_add_source(fdtd_ctx* ctx, int32_t domain, int32_t component, const int32_t lo[3],
                            const int32_t hi[3], const double* waveform, int32_t n_steps, int32_t* source_id) {
    GUARD(ctx);
    if (!valid_dom(ctx, domain) || component < 0 || component > 5 || !lo || !hi || n_steps < 0 ||
        (n_steps > 0 && !waveform))
        return fail(ctx, FDTD_EINVAL, "bad source arguments");
    const DomainHost& d = ctx->doms[domain];
    if (!valid_box(d, lo, hi)) return fail(ctx, FDTD_EINVAL, "source box outside the domain");
    if ((int)d.srcs.size() >= kMaxSrcPerDom) return fail(ctx, FDTD_EINVAL, "at most 8 sources per domain");
    if (component < 3)
        for (int q = 0; q < 3; ++q)
            if (q != component && lo[q] == 0 && !d.per[q])
                return fail(ctx, FDTD_EINVAL, "an electric source box must not include PEC-held nodes (coordinate 0)");
    for (auto& s : ctx->srcs) {
        if (s.s.dom != domain || s.s.comp != component) continue;
        bool overlap = true;
        for (int q = 0; q < 3; ++q)
            if (hi[q] <= s.s.lo[q] || lo[q] >= s.s.hi[q]) overlap = false;
        if (overlap) return fail(ctx, FDTD_EINVAL, "source boxes of one component must not overlap");
    }
    SrcHost sh;
    sh.s.dom = domain;
    sh.s.comp = component;
    for (int q = 0; q < 3; ++q) {
        sh.s.lo[q] = lo[q];
        sh.s.hi[q] = hi[q];
    }
    sh.s.bx = hi[0] - lo[0];
    sh.s.by = hi[1] - lo[1];
    sh.s.ncell = (long long)sh.s.bx * sh.s.by * (hi[2] - lo[2]);
    sh.s.n = n_steps;
    fdtd_status st = dmalloc(ctx, (void**)&sh.wave, sizeof(double) * (n_steps > 0 ? n_steps : 1));
    if (st != FDTD_OK) return st;
    if (n_steps > 0) {
        CK(ctx, cudaMemcpyAsync(sh.wave, waveform, sizeof(double) * n_steps, cudaMemcpyHostToDevice, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
    }
    sh.s.wave = sh.wave;
    ctx->srcs.push_back(sh);
    if (source_id) *source_id = (int)ctx->srcs.size() - 1;
    return sync_srcs(ctx);
}

fdtd_status fdtd_add_dft_monitor(fdtd_ctx* ctx, int32_t domain, const int32_t lo[3], const int32_t hi[3],
                                 uint32_t component_mask, int32_t n_freq, const double* omega_dt,
                                 int32_t* monitor_id) {
    GUARD(ctx);
    if (!valid_dom(ctx, domain) || !lo || !hi || n_freq < 1 || !omega_dt || (component_mask & ~63u) ||
        component_mask == 0)
        return fail(ctx, FDTD_EINVAL, "bad monitor arguments");
    DomainHost& d = ctx->doms[domain];
    if (d.bloch) return fail(ctx, FDTD_EINVAL, "a Bloch domain carries no DFT monitor");
    if (!valid_box(d, lo, hi)) return fail(ctx, FDTD_EINVAL, "monitor box outside the domain");
    if ((int)d.mons.size() >= kMaxMonPerDom) return fail(ctx, FDTD_EINVAL, "at most 8 monitors per domain");
    MonHost mh;
    Mon& m = mh.m;
    m.dom = domain;
    for (int q = 0; q < 3; ++q) {
        m.lo[q] = lo[q];
        m.hi[q] = hi[q];
    }
    m.bx = hi[0] - lo[0];
    m.by = hi[1] - lo[1];
    m.ncell = (long long)m.bx * m.by * (hi[2] - lo[2]);
    m.nf = n_freq;
    m.mask = component_mask;
    m.ncomp = 0;
    for (int cc = 0; cc < 6; ++cc)
        if (component_mask & (1u << cc)) m.comps[m.ncomp++] = cc;
    mh.omega.assign(omega_dt, omega_dt + n_freq);
    fdtd_status st = dmalloc(ctx, (void**)&m.acc, sizeof(double2) * m.ncomp * n_freq * m.ncell);
    if (st != FDTD_OK) return st;
    ctx->mons.push_back(mh);
    const int id = (int)ctx->mons.size() - 1;
    d.mons.push_back(id);
    // (re)build phase tables for every monitor at the current capacity
    const int cap = ctx->phase_cap;
    ctx->phase_cap = 0;
    for (auto& x : ctx->mons)
        if (x.m.phase) {
            CK(ctx, cudaStreamSynchronize(ctx->stream));
            dfree(ctx, (void*)x.m.phase);
            x.m.phase = nullptr;
        }
    st = ensure_phase(ctx, cap > 0 ? cap : 1024);
    if (st != FDTD_OK) return st;
    if (monitor_id) *monitor_id = id;
    st = sync_mons(ctx);
    if (st != FDTD_OK) return st;
    st = upload_tiles(ctx);
    if (st != FDTD_OK) return st;
    return sync_doms(ctx);
}

fdtd_status fdtd_dft_size(fdtd_ctx* ctx, int32_t monitor_id, int64_t* n) {
    GUARD(ctx);
    if (monitor_id < 0 || monitor_id >= (int)ctx->mons.size() || !n) return fail(ctx, FDTD_EINVAL, "bad monitor id");
    const Mon& m = ctx->mons[monitor_id].m;
    *n = (int64_t)m.ncomp * m.nf * m.ncell;
    return FDTD_OK;
}

fdtd_status fdtd_dft_read(fdtd_ctx* ctx, int32_t monitor_id, void* dst, size_t bytes, int32_t dst_on_device) {
    GUARD(ctx);
    int64_t n = 0;
    fdtd_status st = fdtd_dft_size(ctx, monitor_id, &n);
    if (st != FDTD_OK) return st;
    if (!dst || bytes < (size_t)n * 16) return fail(ctx, FDTD_EINVAL, "destination too small");
    const Mon& m = ctx->mons[monitor_id].m;
    CK(ctx, cudaMemcpyAsync(dst, m.acc, (size_t)n * 16, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            ctx->stream));
    if (!dst_on_device) CK(ctx, cudaStreamSynchronize(ctx->stream));
    return FDTD_OK;
}

fdtd_status fdtd_dft_reset(fdtd_ctx* ctx) {
    GUARD(ctx);
    for (auto& mh : ctx->mons)
        CK(ctx, cudaMemsetAsync(mh.m.acc, 0, sizeof(double2) * mh.m.ncomp * mh.m.nf * mh.m.ncell, ctx->stream));
    return FDTD_OK;
}

fdtd_status fdtd_dft_enable(fdtd_ctx* ctx, int32_t enabled) {
    GUARD(ctx);
    ctx->dft_enabled = enabled ? 1 : 0;
    return FDTD_OK;
}

fdtd_status fdtd_enable_energy(fdtd_ctx* ctx, int32_t capacity) {
    GUARD(ctx);
    NOT_STREAMED(ctx);
    NOT_BLOCH(ctx, "the energy record");
    NOT_TENSOR(ctx, "the energy record");
    if (capacity < 1) return fail(ctx, FDTD_EINVAL, "capacity must be >= 1");
    for (auto& d : ctx->doms) {
        if (d.energy) dfree(ctx, d.energy);
        fdtd_status st = dmalloc(ctx, (void**)&d.energy, sizeof(double) * capacity);
        if (st != FDTD_OK) return st;
        d.energy_cap = capacity;
    }
    ctx->energy_on = 1;
    drop_graphs(ctx);
    return sync_doms(ctx);
}

fdtd_status fdtd_energy_read(fdtd_ctx* ctx, int32_t domain, double* host_dst, int32_t n) {
    GUARD(ctx);
    if (!valid_dom(ctx, domain) || !host_dst || n < 0) return fail(ctx, FDTD_EINVAL, "bad arguments");
    const DomainHost& d = ctx->doms[domain];
    if (!d.energy || n > d.energy_cap) return fail(ctx, FDTD_ESTATE, "energy not enabled or n > capacity");
    CK(ctx, cudaMemcpyAsync(host_dst, d.energy, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return FDTD_OK;
}

fdtd_status fdtd_step_forward(fdtd_ctx* ctx, int32_t n_steps) {
    GUARD(ctx);
    if (n_steps < 0) return fail(ctx, FDTD_EINVAL, "n_steps < 0");
    if (any_bloch(ctx) && (!ctx->cell_mode || ctx->energy_on))
        return fail(ctx, FDTD_EINVAL, "Bloch domains step in launch mode 4 without an energy record");
    if (ctx->step + n_steps >= (1ll << 30)) return fail(ctx, FDTD_EINVAL, "step count overflow");
    if (!ctx->mons.empty()) {
        bool changed = false;
        fdtd_status st = ensure_phase(ctx, ctx->step + n_steps + 2, &changed);
        if (st != FDTD_OK) return st;
        if (changed) {
            st = sync_mons(ctx);
            if (st != FDTD_OK) return st;
        }
    }
    if (ctx->streamed) {
        fdtd_status st = ctx->dtype == FDTD_F32 ? stream_forward<float>(ctx, n_steps) : stream_forward<double>(ctx, n_steps);
        if (st != FDTD_OK) return st;
        ctx->step += n_steps;
        return FDTD_OK;
    }
    int left = n_steps;
    {
        fdtd_status st = ensure_ring(ctx);   // monitor rings, before the argument blocks and any capture
        if (st != FDTD_OK) return st;
        st = sync_cell_args(ctx);   // a batch's argument blocks, before any capture
        if (st != FDTD_OK) return st;
    }
    if (ctx->use_graphs && !ctx->prof_on && left >= kGraphSteps) {
        fdtd_status st = build_graph(ctx);
        if (st != FDTD_OK) return st;
        cudaGraphExec_t ge = ctx->graph[ctx->dft_enabled][ctx->energy_on];
        while (left >= kGraphSteps) {
            CK(ctx, cudaGraphLaunch(ge, ctx->stream));
            ctx->launches += ctx->graph_launches[ctx->dft_enabled][ctx->energy_on];
            left -= kGraphSteps;
        }
    }
    // the rest in eager batches of at most kGraphSteps steps (a monitor ring holds one batch)
    for (int b0 = 0; b0 < left; b0 += kGraphSteps) {
        const int nb = std::min(kGraphSteps, left - b0);
        for (int s = 0; s < nb; ++s) {
            if (ctx->dtype == FDTD_F32)
                step_once<float>(ctx, ctx->stream, s, s == 0, s == nb - 1);
            else
                step_once<double>(ctx, ctx->stream, s, s == 0, s == nb - 1);
        }
    }
    CKL(ctx);
    ctx->step += n_steps;
    return FDTD_OK;
}

fdtd_status fdtd_stream_checkpoints(fdtd_ctx* ctx, int32_t enabled) {
    GUARD(ctx);
    if (!ctx->streamed) return fail(ctx, FDTD_EINVAL, "forward checkpoints in host memory belong to a streamed context");
    if (enabled < 0 || enabled > 2) return fail(ctx, FDTD_EINVAL, "enabled must be 0, 1 or 2");
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->d2h_stream));
    for (auto& kv : ctx->ck) ctx->ck_pool.push_back(kv.second);
    ctx->ck.clear();
    if (enabled == 0) {
        for (void* p : ctx->ck_pool) cudaFreeHost(p);
        ctx->ck_pool.clear();
    }
    ctx->ck_on = enabled == 1;
    ctx->ck_t0 = ctx->step;
    return FDTD_OK;
}

fdtd_status fdtd_record_interface(fdtd_ctx* ctx, int32_t capacity) {
    GUARD(ctx);
    NOT_STREAMED(ctx);
    NOT_BLOCH(ctx, "the interface record");
    NOT_TENSOR(ctx, "the interface record");
    if (capacity < 0) return fail(ctx, FDTD_EINVAL, "capacity must be >= 0");
    if (capacity > 0 && (!ctx->cell_mode || ctx->energy_on))
        return fail(ctx, FDTD_EINVAL, "the interface record runs in launch mode 4 without an energy record");
    drop_graphs(ctx);   // captured forward steps change (they record, or stop recording)
    for (auto& d : ctx->doms) {
        if (d.rec) {
            dfree(ctx, d.rec);
            d.rec = nullptr;
        }
        if (capacity == 0 || !has_cpml(d)) continue;
        d.ia = iface_args(d, capacity, ctx->step);
        fdtd_status st = dmalloc(ctx, &d.rec, (size_t)(capacity + 1) * d.ia.slot * ctx->esz);
        if (st != FDTD_OK) return st;
        // slot 0: the interface of the held state u^{t0}
        if (ctx->dtype == FDTD_F32)
            launch_iface<float>(L(ctx), (float* const*)d.F, d.n, d.ia, (float*)d.rec, nullptr, (int)ctx->step, 3, 1);
        else
            launch_iface<double>(L(ctx), (double* const*)d.F, d.n, d.ia, (double*)d.rec, nullptr, (int)ctx->step, 3, 1);
        CKL(ctx);
    }
    return FDTD_OK;
}

fdtd_status fdtd_step_backward(fdtd_ctx* ctx, int32_t n_steps) {
    GUARD(ctx);
    NOT_STREAMED(ctx);
    NOT_BLOCH(ctx, "the backward step");
    NOT_TENSOR(ctx, "the backward step");
    if (n_steps < 0) return fail(ctx, FDTD_EINVAL, "n_steps must be >= 0");
    for (const auto& d : ctx->doms) {
        if (d.npole > 0) return fail(ctx, FDTD_EINVAL, "backward steps need nondispersive domains (no poles)");
        if (has_cpml(d) && !d.rec)
            return fail(ctx, FDTD_EINVAL, "a domain with CPML faces steps backward only with an interface record "
                                          "(fdtd_record_interface before the forward steps)");
        if (d.rec && (ctx->step - n_steps < d.ia.t0 || ctx->step - d.ia.t0 > d.ia.cap))
            return fail(ctx, FDTD_ESTATE, "the interface record does not cover these steps");
        if (d.ie[0] == nullptr) return fail(ctx, FDTD_EINVAL, "no material");
    }
    if (!ctx->cell_mode) return fail(ctx, FDTD_EINVAL, "backward steps run in launch mode 4");
    if (n_steps > ctx->step) return fail(ctx, FDTD_ESTATE, "cannot step back past step 0");
    if (n_steps == 0) return FDTD_OK;
    const Launch l = L(ctx);
    StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.srcs = ctx->d_srcs;
    a.mons = ctx->d_mons;
    a.d_step = ctx->d_step;
    a.d_ticket = ctx->d_ticket;
    a.d_base = ctx->d_base;
    launch_copy_int(l, ctx->d_step, ctx->d_base);
    for (int q = 0; q < n_steps; ++q) {
        a.offset = -1 - q;   // undoes forward step n = step - 1 - q
        for (int di = 0; di < (int)ctx->doms.size(); ++di) {
            const DomainHost& d = ctx->doms[di];
            if (!d.rec) {
                if (ctx->dtype == FDTD_F32)
                    launch_back_cell<float>(l, make_cell_args<float>(ctx, di, true),
                                            make_cell_args<float>(ctx, di, false), (float)ctx->S, a, ctx->aniso);
                else
                    launch_back_cell<double>(l, make_cell_args<double>(ctx, di, true),
                                             make_cell_args<double>(ctx, di, false), ctx->S, a, ctx->aniso);
                continue;
            }
            // absorbing faces: the interior steps back, its interface planes come from the record
            // (E^{n+1} from slot n + 1 - t0 before the H half, H^{n+1/2} from slot n - t0 before E)
            auto back = [&](auto zero) {
                using T = decltype(zero);
                CellArgs<T> ce = make_cell_args<T>(ctx, di, true), ch = make_cell_args<T>(ctx, di, false);
                for (int ax = 0; ax < 3; ++ax) {
                    ce.alo[ax] = ch.alo[ax] = d.dlo[ax];
                    ce.ahi[ax] = ch.ahi[ax] = d.n[ax] - d.dhi[ax];
                }
                launch_iface<T>(l, (T* const*)d.F, d.n, d.ia, (T*)d.rec, ctx->d_base, a.offset + 1, 2, 0);
                launch_back_h<T>(l, ch, (T)ctx->S, a);
                launch_iface<T>(l, (T* const*)d.F, d.n, d.ia, (T*)d.rec, ctx->d_base, a.offset, 1, 0);
                launch_back_e<T>(l, ce, (T)ctx->S, a, ctx->aniso);
            };
            if (ctx->dtype == FDTD_F32)
                back(0.0f);
            else
                back(0.0);
        }
    }
    launch_advance(l, ctx->d_step, -n_steps);
    CKL(ctx);
    ctx->step -= n_steps;
    return FDTD_OK;
}

fdtd_status fdtd_set_launch_mode(fdtd_ctx* ctx, int32_t mode) {
    GUARD(ctx);
    if (ctx->streamed && mode != 4) return fail(ctx, FDTD_EINVAL, "a host-streamed context steps per cell (mode 4)");
    if (mode != 0 && mode != 4) return fail(ctx, FDTD_EINVAL, "launch mode must be 0 or 4");
    if (mode != 4 && any_bloch(ctx)) return fail(ctx, FDTD_EINVAL, "Bloch domains step in launch mode 4");
    if (mode != 4 && any_tensor(ctx)) return fail(ctx, FDTD_EINVAL, "tensor domains step in launch mode 4");
    for (const auto& d : ctx->doms)
        if (mode != 4 && d.rec) return fail(ctx, FDTD_EINVAL, "an interface record runs in launch mode 4");
    if (mode != ctx->cell_mode * 4) drop_graphs(ctx);   // graphs hold the launches of one mode
    ctx->cell_mode = mode == 4;
    return FDTD_OK;
}

fdtd_status fdtd_get_launch_mode(fdtd_ctx* ctx, int32_t* mode) {
    GUARD(ctx);
    if (!mode) return FDTD_EINVAL;
    *mode = ctx->cell_mode ? 4 : 0;
    return FDTD_OK;
}

// Times launch modes 0 and 4 for n_steps on the live state (saved to a private snapshot first and
// restored after each trial) and keeps the faster.
static fdtd_status save_slot(fdtd_ctx* ctx, int32_t slot, int32_t codec);
static fdtd_status restore_slot(fdtd_ctx* ctx, int32_t slot);

fdtd_status fdtd_autotune(fdtd_ctx* ctx, int32_t n_steps, double* ms_per_mode) {
    GUARD(ctx);
    NOT_STREAMED(ctx);
    NOT_BLOCH(ctx, "autotuning (Bloch domains step in launch mode 4)");
    NOT_TENSOR(ctx, "autotuning (tensor domains step in launch mode 4)");
    if (n_steps < 1) return fail(ctx, FDTD_EINVAL, "n_steps must be >= 1");
    const int slot = 1 << 30;   // private slot id (public ids are below 2^30)
    const int energy = ctx->energy_on;
    const long long step0 = ctx->step;
    ctx->energy_on = 0;
    fdtd_status st = FDTD_OK;
    double best = 1e30;
    int best_mode = 4;
    if (ms_per_mode)
        for (int q = 0; q < FDTD_LAUNCH_MODES; ++q) ms_per_mode[q] = -1.0;
    // the trials run with DFT recording as configured (its cost shapes the ranking); the monitor
    // accumulators are copied aside first and put back after every trial
    std::vector<std::pair<void*, size_t>> saved;
    auto put_back = [&]() -> fdtd_status {
        for (size_t q = 0; q < saved.size(); ++q)
            CK(ctx, cudaMemcpyAsync(ctx->mons[q].m.acc, saved[q].first, saved[q].second, cudaMemcpyDeviceToDevice,
                                    ctx->stream));
        return FDTD_OK;
    };
    for (auto& mh : ctx->mons) {
        const size_t bytes = (size_t)mh.m.ncomp * mh.m.nf * mh.m.ncell * sizeof(double2);
        void* p = nullptr;
        if (st == FDTD_OK) st = dmalloc(ctx, &p, bytes);
        if (st == FDTD_OK)
            if (cudaMemcpyAsync(p, mh.m.acc, bytes, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
                st = fail(ctx, FDTD_ECUDA, "saving the DFT accumulators failed");
        saved.push_back({p, bytes});
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == FDTD_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = fail(ctx, FDTD_ECUDA, "cudaEventCreate failed");
    if (st == FDTD_OK) st = save_slot(ctx, slot, FDTD_CODEC_NATIVE);
    for (int mode : {0, 4}) {
        if (st != FDTD_OK) break;
        fdtd_set_launch_mode(ctx, mode);
        // warm-up: graph capture, caches
        st = fdtd_step_forward(ctx, n_steps < kGraphSteps ? n_steps : kGraphSteps);
        if (st == FDTD_OK) st = restore_slot(ctx, slot);
        if (st != FDTD_OK) break;
        cudaEventRecord(e0, ctx->stream);
        st = fdtd_step_forward(ctx, n_steps);
        cudaEventRecord(e1, ctx->stream);
        if (st != FDTD_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = fail(ctx, FDTD_ECUDA, "autotune event synchronisation failed");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms_per_mode) ms_per_mode[mode] = ms;
        if (ms < best) {
            best = ms;
            best_mode = mode;
        }
        st = restore_slot(ctx, slot);
    }
    if (st == FDTD_OK) st = put_back();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(ctx->stream);
    for (auto& sv : saved) dfree(ctx, sv.first);
    auto it = ctx->slots.find(slot);
    if (it != ctx->slots.end()) {
        cudaFree(it->second.buf);
        ctx->slots.erase(it);
    }
    ctx->energy_on = energy;
    ctx->step = step0;
    if (st != FDTD_OK) return st;
    st = set_device_step(ctx, step0);
    if (st != FDTD_OK) return st;
    return fdtd_set_launch_mode(ctx, best_mode);
}

fdtd_status fdtd_step_count(fdtd_ctx* ctx, int64_t* n) {
    GUARD(ctx);
    if (!n) return FDTD_EINVAL;
    *n = ctx->step;
    return FDTD_OK;
}

fdtd_status fdtd_set_step_count(fdtd_ctx* ctx, int64_t n) {
    GUARD(ctx);
    if (n < 0 || n >= (1ll << 30)) return fail(ctx, FDTD_EINVAL, "bad step count");
    ctx->step = n;
    return set_device_step(ctx, n);
}

fdtd_status fdtd_reset(fdtd_ctx* ctx) {
    GUARD(ctx);
    if (ctx->streamed) {
        // host state: cleared by the host once the streams are idle
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->d2h_stream));
        const DomainHost& d = ctx->doms[0];
        for (int p = 0; p < part_count(d); ++p) {
            void* ptr = part_ptr(d, 0, p, ctx->esz);
            const long long n = part_size(d, p);
            if (ptr && n) std::memset(ptr, 0, (size_t)n * ctx->esz);
        }
        ctx->step = 0;
        return set_device_step(ctx, 0);
    }
    for (auto& d : ctx->doms)
        for (int p = 0; p < part_count(d); ++p) {
            void* ptr = part_ptr(d, 0, p, ctx->esz);
            const long long n = part_size(d, p);
            if (ptr && n) CK(ctx, cudaMemsetAsync(ptr, 0, (size_t)n * ctx->esz, ctx->stream));
        }
    ctx->step = 0;
    return set_device_step(ctx, 0);
}

fdtd_status fdtd_part_count(fdtd_ctx* ctx, int32_t domain, int32_t* n_parts) {
    GUARD(ctx);
    if (!valid_dom(ctx, domain) || !n_parts) return fail(ctx, FDTD_EINVAL, "bad domain");
    *n_parts = part_count(ctx->doms[domain]);
    return FDTD_OK;
}

fdtd_status fdtd_part_size(fdtd_ctx* ctx, int32_t domain, int32_t part, int64_t* n_values) {
    GUARD(ctx);
    if (!valid_dom(ctx, domain) || !n_values) return fail(ctx, FDTD_EINVAL, "bad domain");
    const DomainHost& d = ctx->doms[domain];
    if (part < 0 || part >= part_count(d)) return fail(ctx, FDTD_EINVAL, "bad part id");
    *n_values = part_size(d, part);
    return FDTD_OK;
}

fdtd_status fdtd_get_part(fdtd_ctx* ctx, int32_t domain, int32_t which, int32_t part, void* dst) {
    GUARD(ctx);
    if (!valid_dom(ctx, domain) || (which != 0 && which != 1) || !dst) return fail(ctx, FDTD_EINVAL, "bad arguments");
    const DomainHost& d = ctx->doms[domain];
    if (part < 0 || part >= part_count(d)) return fail(ctx, FDTD_EINVAL, "bad part id");
    if (which == 1 && ctx->streamed && !ctx->hadj_ready)
        return fail(ctx, FDTD_ESTATE, "a host-streamed context has an adjoint state after fdtd_adjoint_begin");
    if (which == 1 && !ctx->streamed) {
        fdtd_status st = flush_adjoint(ctx);
        if (st != FDTD_OK) return st;
    }
    const long long n = part_size(d, part);
    if (n == 0) return FDTD_OK;
    CK(ctx, cudaMemcpyAsync(dst, part_ptr(d, which, part, ctx->esz), (size_t)n * ctx->esz, cudaMemcpyDefault,
                            ctx->stream));
    return FDTD_OK;
}

fdtd_status fdtd_set_part(fdtd_ctx* ctx, int32_t domain, int32_t which, int32_t part, const void* src) {
    GUARD(ctx);
    if (!valid_dom(ctx, domain) || (which != 0 && which != 1) || !src) return fail(ctx, FDTD_EINVAL, "bad arguments");
    const DomainHost& d = ctx->doms[domain];
    if (part < 0 || part >= part_count(d)) return fail(ctx, FDTD_EINVAL, "bad part id");
    if (which == 1 && ctx->streamed && !ctx->hadj_ready)
        return fail(ctx, FDTD_ESTATE, "a host-streamed context has an adjoint state after fdtd_adjoint_begin");
    if (which == 1 && !ctx->streamed) {
        fdtd_status st = flush_adjoint(ctx);
        if (st != FDTD_OK) return st;
    }
    const long long n = part_size(d, part);
    if (n == 0) return FDTD_OK;
    CK(ctx, cudaMemcpyAsync(part_ptr(d, which, part, ctx->esz), src, (size_t)n * ctx->esz, cudaMemcpyDefault,
                            ctx->stream));
    return FDTD_OK;
}

fdtd_status fdtd_ade_box(fdtd_ctx* ctx, int32_t domain, int32_t lo[3], int32_t hi[3]) {
    GUARD(ctx);
    if (!valid_dom(ctx, domain) || !lo || !hi) return fail(ctx, FDTD_EINVAL, "bad arguments");
    for (int q = 0; q < 3; ++q) {
        lo[q] = ctx->doms[domain].blo[q];
        hi[q] = ctx->doms[domain].bhi[q];
    }
    return FDTD_OK;
}

fdtd_status fdtd_snapshot_bytes(fdtd_ctx* ctx, int32_t codec, int64_t* bytes) {
    GUARD(ctx);
    NOT_STREAMED(ctx);
    if (!bytes || (codec != FDTD_CODEC_NATIVE && codec != FDTD_CODEC_BF16)) return fail(ctx, FDTD_EINVAL, "bad codec");
    *bytes = (int64_t)snapshot_bytes(ctx, codec);
    return FDTD_OK;
}

// Segment table of a native snapshot (built once: part arrays and sizes are fixed at create).
static fdtd_status snap_segments(fdtd_ctx* ctx) {
    if (ctx->d_snapsegs) return FDTD_OK;
    std::vector<SnapSeg> segs;
    long long off = 0;
    for (const auto& d : ctx->doms)
        for (int part = 0; part < part_count(d); ++part) {
            const long long n = part_size(d, part);
            if (n == 0) continue;
            const long long b = n * (long long)ctx->esz;
            segs.push_back({(char*)part_ptr(d, 0, part, ctx->esz), off, b});
            ctx->snap_max = std::max(ctx->snap_max, b);
            off += (b + 255) & ~255ll;
        }
    if (segs.size() > 65535) return fail(ctx, FDTD_EINVAL, "too many state parts for one snapshot launch");
    if (segs.empty()) return FDTD_OK;
    fdtd_status st = dmalloc(ctx, (void**)&ctx->d_snapsegs, sizeof(SnapSeg) * segs.size());
    if (st != FDTD_OK) return st;
    CK(ctx, cudaMemcpyAsync(ctx->d_snapsegs, segs.data(), sizeof(SnapSeg) * segs.size(), cudaMemcpyHostToDevice,
                            ctx->stream));
    ctx->n_snapsegs = (int)segs.size();
    return FDTD_OK;
}

static fdtd_status save_slot(fdtd_ctx* ctx, int32_t slot, int32_t codec) {
    const size_t need = snapshot_bytes(ctx, codec);
    Slot& s = ctx->slots[slot];
    if (s.bytes < need) {
        if (s.buf) {
            CK(ctx, cudaStreamSynchronize(ctx->stream));
            cudaFree(s.buf);
            s.buf = nullptr;
            s.bytes = 0;
        }
        cudaError_t e = cudaMalloc(&s.buf, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->slots.erase(slot);
            return fail(ctx, FDTD_ENOMEM, "snapshot slot allocation failed");
        }
        s.bytes = need;
    }
    s.codec = codec;
    s.step = ctx->step;
    char* p = (char*)s.buf;
    const Launch l = L(ctx);
    if (codec == FDTD_CODEC_NATIVE) {
        fdtd_status st = snap_segments(ctx);
        if (st != FDTD_OK) return st;
        launch_snapshot_copy(l, ctx->d_snapsegs, ctx->n_snapsegs, ctx->snap_max, s.buf, 1);
        CKL(ctx);
        return FDTD_OK;
    }
    for (const auto& d : ctx->doms)
        for (int part = 0; part < part_count(d); ++part) {
            const long long n = part_size(d, part);
            if (n == 0) continue;
            const void* src = part_ptr(d, 0, part, ctx->esz);
            const long long np = part_planes(d, part);
            const size_t b = bf16_part_bytes(n, np);
            uint16_t* q = (uint16_t*)p;
            float* sc = (float*)(p + bf16_scale_off(n));
            if (ctx->dtype == FDTD_F32)
                launch_bf16_encode<float>(l, (const float*)src, np, n / np, q, sc);
            else
                launch_bf16_encode<double>(l, (const double*)src, np, n / np, q, sc);
            CKL(ctx);
            p += (b + 255) & ~(size_t)255;
        }
    return FDTD_OK;
}

static fdtd_status restore_slot(fdtd_ctx* ctx, int32_t slot) {
    auto it = ctx->slots.find(slot);
    if (it == ctx->slots.end() || !it->second.buf) return fail(ctx, FDTD_ESTATE, "empty snapshot slot");
    const Slot& s = it->second;
    const char* p = (const char*)s.buf;
    const Launch l = L(ctx);
    if (s.codec == FDTD_CODEC_NATIVE) {
        fdtd_status st = snap_segments(ctx);
        if (st != FDTD_OK) return st;
        launch_snapshot_copy(l, ctx->d_snapsegs, ctx->n_snapsegs, ctx->snap_max, s.buf, 0);
        CKL(ctx);
        ctx->step = s.step;
        return set_device_step(ctx, s.step);
    }
    for (const auto& d : ctx->doms)
        for (int part = 0; part < part_count(d); ++part) {
            const long long n = part_size(d, part);
            if (n == 0) continue;
            void* dst = part_ptr(d, 0, part, ctx->esz);
            const long long np = part_planes(d, part);
            const size_t b = bf16_part_bytes(n, np);
            const uint16_t* q = (const uint16_t*)p;
            const float* sc = (const float*)(p + bf16_scale_off(n));
            if (ctx->dtype == FDTD_F32)
                launch_bf16_decode<float>(l, q, sc, np, n / np, (float*)dst);
            else
                launch_bf16_decode<double>(l, q, sc, np, n / np, (double*)dst);
            CKL(ctx);
            p += (b + 255) & ~(size_t)255;
        }
    ctx->step = s.step;
    return set_device_step(ctx, s.step);
}

fdtd_status fdtd_state_save(fdtd_ctx* ctx, int32_t slot, int32_t codec) {
    GUARD(ctx);
    NOT_STREAMED(ctx);
    if (slot < 0 || slot >= (1 << 30) || (codec != FDTD_CODEC_NATIVE && codec != FDTD_CODEC_BF16))
        return fail(ctx, FDTD_EINVAL, "bad slot or codec");
    return save_slot(ctx, slot, codec);
}

fdtd_status fdtd_state_restore(fdtd_ctx* ctx, int32_t slot) {
    GUARD(ctx);
    NOT_STREAMED(ctx);
    if (slot < 0 || slot >= (1 << 30)) return fail(ctx, FDTD_EINVAL, "bad slot");
    return restore_slot(ctx, slot);
}

fdtd_status fdtd_snapshots_free(fdtd_ctx* ctx) {
    GUARD(ctx);
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (auto& s : ctx->slots) cudaFree(s.second.buf);
    ctx->slots.clear();
    return FDTD_OK;
}

fdtd_status fdtd_set_design(fdtd_ctx* ctx, int32_t domain, const int32_t lo[3], const int32_t hi[3], double* grad) {
    GUARD(ctx);
    if (!valid_dom(ctx, domain)) return fail(ctx, FDTD_EINVAL, "bad domain");
    DomainHost& d = ctx->doms[domain];
    if (d.bloch && grad) return fail(ctx, FDTD_EINVAL, "a Bloch domain carries no design box");
    if (!grad) {
        d.design = 0;
        d.grad = nullptr;
        return sync_doms(ctx);
    }
    if (!lo || !hi || !valid_box(d, lo, hi)) return fail(ctx, FDTD_EINVAL, "design box outside the domain");
    for (int q = 0; q < 3; ++q)
        if (lo[q] < d.dlo[q] || hi[q] > d.n[q] - d.dhi[q])
            return fail(ctx, FDTD_EINVAL, "design box must lie outside the CPML slabs");
    d.design = 1;
    d.grad = grad;
    for (int q = 0; q < 3; ++q) {
        d.glo[q] = lo[q];
        d.ghi[q] = hi[q];
    }
    return sync_doms(ctx);
}

fdtd_status fdtd_set_pole_grad(fdtd_ctx* ctx, int32_t domain, int32_t enabled) {
    GUARD(ctx);
    NOT_STREAMED(ctx);
    if (!valid_dom(ctx, domain)) return fail(ctx, FDTD_EINVAL, "bad domain");
    DomainHost& d = ctx->doms[domain];
    if (!enabled) {
        d.pgc_on = 0;
        return sync_doms(ctx);
    }
    if (d.npole == 0 || d.bcell == 0) return fail(ctx, FDTD_EINVAL, "the domain has no dispersive cell");
    for (int q = 0; q < 3; ++q)
        if (d.blo[q] < d.dlo[q] || d.bhi[q] > d.n[q] - d.dhi[q])
            return fail(ctx, FDTD_EINVAL, "pole-parameter gradients need the pole-state box outside the CPML slabs");
    if (!d.pgc) {
        fdtd_status st = dmalloc(ctx, (void**)&d.pgc, sizeof(double) * 6 * kMaxPole);
        if (st != FDTD_OK) return st;
    }
    CK(ctx, cudaMemsetAsync(d.pgc, 0, sizeof(double) * 6 * kMaxPole, ctx->stream));
    d.pgc_on = 1;
    return sync_doms(ctx);
}

fdtd_status fdtd_pole_grad(fdtd_ctx* ctx, int32_t domain, double* host_out) {
    GUARD(ctx);
    NOT_STREAMED(ctx);
    if (!valid_dom(ctx, domain) || !host_out) return fail(ctx, FDTD_EINVAL, "bad arguments");
    const DomainHost& d = ctx->doms[domain];
    if (!d.pgc_on) return fail(ctx, FDTD_EINVAL, "pole-parameter gradients are not collected for this domain");
    double pgc[6 * kMaxPole];
    CK(ctx, cudaMemcpyAsync(pgc, d.pgc, sizeof(pgc), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (int p = 0; p < d.npole; ++p)
        for (int t = 0; t < 3; ++t) {
            double dc[6];
            pole_coef_deriv(d.poles[p], t, dc);
            double acc = 0.0;
            for (int q = 0; q < 6; ++q) acc += pgc[6 * p + q] * dc[q];
            host_out[3 * p + t] = acc;
        }
    return FDTD_OK;
}

fdtd_status fdtd_set_adjoint_source(fdtd_ctx* ctx, int32_t monitor_id, const void* cot) {
    GUARD(ctx);
    if (monitor_id < 0 || monitor_id >= (int)ctx->mons.size()) return fail(ctx, FDTD_EINVAL, "bad monitor id");
    ctx->mons[monitor_id].m.cot = (const double2*)cot;
    return sync_mons(ctx);
}

fdtd_status fdtd_adjoint_begin(fdtd_ctx* ctx) {
    GUARD(ctx);
    if (ctx->streamed) {
        // the adjoint state lives in pinned host memory: set 0 of the two host sets, zeroed
        fdtd_status st = ctx->dtype == FDTD_F32 ? stream_adj_prepare<float>(ctx) : stream_adj_prepare<double>(ctx);
        if (st != FDTD_OK) return st;
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        st = stream_adj_bind(ctx, 0);
        if (st != FDTD_OK) return st;
        const DomainHost& d = ctx->doms[0];
        for (int p = 0; p < part_count(d); ++p) {
            void* ptr = part_ptr(d, 1, p, ctx->esz);
            const long long n = part_size(d, p);
            if (ptr && n) std::memset(ptr, 0, (size_t)n * ctx->esz);
        }
    } else {
        for (auto& d : ctx->doms)
            for (int p = 0; p < part_count(d); ++p) {
                void* ptr = part_ptr(d, 1, p, ctx->esz);
                const long long n = part_size(d, p);
                if (ptr && n) CK(ctx, cudaMemsetAsync(ptr, 0, (size_t)n * ctx->esz, ctx->stream));
            }
    }
    for (auto& d : ctx->doms)
        if (d.pgc_on) CK(ctx, cudaMemsetAsync(d.pgc, 0, sizeof(double) * 6 * kMaxPole, ctx->stream));
    ctx->adj_step = ctx->step;
    ctx->adj_pending = 0;
    if (ctx->step >= 1 && ctx->nentries[1] > 0) {
        bool changed = false;
        fdtd_status st = ensure_phase(ctx, ctx->step + 2, &changed);
        if (st != FDTD_OK) return st;
        if (changed) {
            st = sync_mons(ctx);
            if (st != FDTD_OK) return st;
        }
        if (ctx->dtype == FDTD_F32)
            launch_inject<float>(L(ctx), (const Dom<float>*)ctx->d_doms, ctx->d_mons, ctx->d_entries[1],
                                 ctx->nentries[1], ctx->nthreads[1], ctx->d_entry_begin[1], (int)ctx->step - 1, 1);
        else
            launch_inject<double>(L(ctx), (const Dom<double>*)ctx->d_doms, ctx->d_mons, ctx->d_entries[1],
                                  ctx->nentries[1], ctx->nthreads[1], ctx->d_entry_begin[1], (int)ctx->step - 1, 1);
        CKL(ctx);
    }
    return FDTD_OK;
}

fdtd_status fdtd_step_adjoint(fdtd_ctx* ctx, int32_t n_steps) {
    GUARD(ctx);
    if (n_steps < 0 || n_steps > ctx->adj_step) return fail(ctx, FDTD_EINVAL, "n_steps out of range");
    if (ctx->streamed) {
        if (!ctx->hadj_ready || !ctx->ck_on)
            return fail(ctx, FDTD_ESTATE, "a streamed transposed sweep needs forward checkpoints "
                                          "(fdtd_stream_checkpoints) and fdtd_adjoint_begin");
        if (!ctx->mons.empty()) {
            fdtd_status st = ensure_phase(ctx, ctx->adj_step + 2, nullptr);
            if (st != FDTD_OK) return st;
            st = sync_mons(ctx);
            if (st != FDTD_OK) return st;
        }
        fdtd_status st = prepare_inj(ctx);
        if (st != FDTD_OK) return st;
        return ctx->dtype == FDTD_F32 ? stream_adjoint<float>(ctx, n_steps) : stream_adjoint<double>(ctx, n_steps);
    }
    bool design = false;
    for (auto& d : ctx->doms) design = design || d.design;
    if (design && n_steps > 0 && (n_steps != 1 || ctx->step != ctx->adj_step - 1))
        return fail(ctx, FDTD_ESTATE,
                    "with a design box each adjoint step m needs the forward state u^m (step count " +
                        std::to_string(ctx->step) + ", adjoint index " + std::to_string(ctx->adj_step) + ")");
    if (!ctx->mons.empty()) {
        bool changed = false;
        fdtd_status st = ensure_phase(ctx, ctx->adj_step + 2, &changed);
        if (st != FDTD_OK) return st;
        if (changed) {
            st = sync_mons(ctx);
            if (st != FDTD_OK) return st;
        }
    }
    {
        fdtd_status st = prepare_inj(ctx);
        if (st != FDTD_OK) return st;
    }
    for (int s = 0; s < n_steps; ++s) {
        const int m = (int)ctx->adj_step - 1;
        if (ctx->dtype == FDTD_F32)
            adj_once<float>(ctx, m);
        else
            adj_once<double>(ctx, m);
        ctx->adj_pending = 1;
        ctx->adj_step = m;
    }
    CKL(ctx);
    return FDTD_OK;
}

fdtd_status fdtd_run_schedule(fdtd_ctx* ctx, const int32_t* actions, int32_t n_actions, int32_t codec,
                              int32_t* executed) {
    GUARD(ctx);
    if (!actions || n_actions < 0 || !executed) return fail(ctx, FDTD_EINVAL, "bad arguments");
    *executed = 0;
    for (int32_t i = 0; i < n_actions; ++i) {
        const int32_t kind = actions[2 * i], arg = actions[2 * i + 1];
        fdtd_status st;
        switch (kind) {
            case FDTD_ACT_SAVE: st = fdtd_state_save(ctx, arg, codec); break;
            case FDTD_ACT_RESTORE: st = fdtd_state_restore(ctx, arg); break;
            case FDTD_ACT_ADVANCE: st = fdtd_step_forward(ctx, arg); break;
            case FDTD_ACT_ADJOINT: st = fdtd_step_adjoint(ctx, arg); break;
            case FDTD_ACT_STOP: *executed = i + 1; return FDTD_OK;
            default: return fail(ctx, FDTD_EINVAL, "unknown schedule action " + std::to_string(kind));
        }
        if (st != FDTD_OK) return st;
        *executed = i + 1;
    }
    return FDTD_OK;
}

fdtd_status fdtd_adjoint_step_count(fdtd_ctx* ctx, int64_t* a) {
    GUARD(ctx);
    if (!a) return FDTD_EINVAL;
    *a = ctx->adj_step;
    return FDTD_OK;
}

fdtd_status fdtd_set_adjoint_step_count(fdtd_ctx* ctx, int64_t a) {
    GUARD(ctx);
    if (a < 0 || a >= (1ll << 30)) return fail(ctx, FDTD_EINVAL, "bad adjoint index");
    fdtd_status st = flush_adjoint(ctx);
    if (st != FDTD_OK) return st;
    ctx->adj_step = a;
    return FDTD_OK;
}

fdtd_status fdtd_check_finite(fdtd_ctx* ctx) {
    GUARD(ctx);
    CK(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(unsigned long long), ctx->stream));
    for (auto& d : ctx->doms)
        for (int p = 0; p < part_count(d); ++p) {
            const void* ptr = part_ptr(d, 0, p, ctx->esz);
            const long long n = part_size(d, p);
            if (!ptr || !n) continue;
            if (ctx->dtype == FDTD_F32)
                launch_nonfinite<float>(L(ctx), (const float*)ptr, n, ctx->d_flag);
            else
                launch_nonfinite<double>(L(ctx), (const double*)ptr, n, ctx->d_flag);
        }
    CKL(ctx);
    unsigned long long bad = 0;
    CK(ctx, cudaMemcpyAsync(&bad, ctx->d_flag, sizeof(bad), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (bad) return fail(ctx, FDTD_ENONFINITE, "non-finite values in the forward state");
    return FDTD_OK;
}

fdtd_status fdtd_synchronize(fdtd_ctx* ctx, int32_t timeout_ms) {
    GUARD(ctx);
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(ctx->stream);
        if (e == cudaSuccess) return FDTD_OK;
        if (e != cudaErrorNotReady) return fail(ctx, FDTD_ECUDA, std::string("stream: ") + cudaGetErrorString(e));
        const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
        if (ms.count() >= timeout_ms) return fail(ctx, FDTD_ETIMEOUT, "stream not finished within the timeout");
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

fdtd_status fdtd_launch_count(fdtd_ctx* ctx, int64_t* n) {
    if (!ctx || !n) return FDTD_EINVAL;
    *n = ctx->launches;
    return FDTD_OK;
}

fdtd_status fdtd_time_half_steps(fdtd_ctx* ctx, int32_t which, int32_t n_launches, double* ms_per_launch) {
    GUARD(ctx);
    NOT_STREAMED(ctx);
    if (!ms_per_launch || which < 0 || which > 5 || n_launches < 1 || n_launches > 4096)
        return fail(ctx, FDTD_EINVAL, "bad arguments");
    *ms_per_launch = 0.0;
    if (!ctx->cell_mode || ctx->energy_on)
        return fail(ctx, FDTD_EINVAL, "per-cell launch mode (4) without an energy record only");
    NOT_BLOCH(ctx, "kernel timing");
    NOT_TENSOR(ctx, "kernel timing");
    if (which == 2 && ctx->n_dft_items == 0) return fail(ctx, FDTD_EINVAL, "no DFT monitor");
    if (which <= 2 || which == 5) {
        fdtd_status st = ensure_ring(ctx);
        if (st != FDTD_OK) return st;
    }
    if (which == 5) {
        if (!ctx->ring_on || ctx->n_dft_items == 0)
            return fail(ctx, FDTD_EINVAL, "no monitor ring (the DFT runs per step in this configuration)");
        bool changed = false;   // phases of the kGraphSteps steps the fold reads
        fdtd_status st = ensure_phase(ctx, ctx->step + kGraphSteps + 2, &changed);
        if (st != FDTD_OK) return st;
        if (changed) {
            st = sync_mons(ctx);
            if (st != FDTD_OK) return st;
        }
    }
    if (which >= 3) {
        fdtd_status st = prepare_inj(ctx);   // the transposed kernels read the injection scratch
        if (st != FDTD_OK) return st;
    }
    if (!ctx->cap_stream) CK(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    launch_copy_int(L(ctx), ctx->d_step, ctx->d_base);   // phases / sources of the current step
    CKL(ctx);
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    long long dummy = 0;
    CK(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    if (ctx->dtype == FDTD_F32)
        time_launches_t<float>(ctx, ctx->cap_stream, which, n_launches, &dummy);
    else
        time_launches_t<double>(ctx, ctx->cap_stream, which, n_launches, &dummy);
    cudaGraph_t g = nullptr;
    CK(ctx, cudaStreamEndCapture(ctx->cap_stream, &g));
    cudaGraphExec_t ge = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    CK(ctx, e);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, ctx->stream);   // warm-up replay
    if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaGraphExecDestroy(ge);
    CK(ctx, e);
    ctx->launches += 2ll * n_launches * ((which == 2 || which == 5) ? 1 : (long long)ctx->doms.size());
    if (which >= 3) ctx->adj_pending = 1;   // the adjoint arrays now hold the lagged form
    *ms_per_launch = (double)ms / n_launches;
    return FDTD_OK;
}

static void prof_release(fdtd_ctx* ctx) {
    for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
    ctx->prof_ev.clear();
    ctx->prof_kind.clear();
    ctx->prof_on = 0;
    ctx->prof_used = 0;
}

fdtd_status fdtd_profile_begin(fdtd_ctx* ctx, int32_t max_launches) {
    GUARD(ctx);
    NOT_STREAMED(ctx);
    if (max_launches < 1) return fail(ctx, FDTD_EINVAL, "max_launches must be >= 1");
    prof_release(ctx);
    ctx->prof_ev.resize(2 * (size_t)max_launches);
    ctx->prof_kind.assign(max_launches, 0);
    for (auto& e : ctx->prof_ev) {
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) {
            e = nullptr;
            prof_release(ctx);
            return fail(ctx, FDTD_ECUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(r));
        }
    }
    ctx->prof_on = 1;
    return FDTD_OK;
}

fdtd_status fdtd_profile_end(fdtd_ctx* ctx, double* ms, int64_t* launches) {
    GUARD(ctx);
    if (!ms || !launches) return fail(ctx, FDTD_EINVAL, "NULL output");
    for (int k = 0; k < FDTD_KERNEL_CLASSES; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i + 1 < ctx->prof_used; i += 2) {
        float t = 0.f;
        CK(ctx, cudaEventElapsedTime(&t, ctx->prof_ev[i], ctx->prof_ev[i + 1]));
        const int k = ctx->prof_kind[i / 2];
        ms[k] += t;
        launches[k] += 1;
    }
    prof_release(ctx);
    return FDTD_OK;
}

}  // extern "C"
