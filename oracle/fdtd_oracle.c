/*
 * FP64 CPU oracle of the 3-D Yee FDTD step and its discrete adjoint.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or helper with the CUDA
 * library: every coefficient below is derived here from the paper's text.
 *
 * Plain, slow, full-grid arrays, written so that each line can be checked
 * against the paper by eye.  Single-threaded by default; oracle_set_threads(n)
 * lets an OpenMP team share the k-planes of the E and H phases and the cells of
 * the DFT accumulation, where every cell reads only values no other cell of the
 * same loop writes, so each cell's arithmetic (and hence every result, bit for
 * bit) is the same for any thread count.  The energy sum and the adjoint
 * (scatter form) always run on one thread.
 *   - Eq. (yee)   (Sec. 2.1): E^{n+1} = E^n + S eps^{-1} C^-(H^{n+1/2}) + s^{n+1},
 *                             H^{n+3/2} = H^{n+1/2} - S C^+(E^{n+1}) + m^{n+3/2};
 *                 soft sources are added after the update; fields start at 0,
 *                 E is sampled at (n+1) dt and H at (n+3/2) dt.
 *   - Sec. 2.2    CPML (Roden-Gedney): one memory variable per transverse
 *                 derivative in each absorbing face, polynomial kappa/sigma/alpha
 *                 profiles; PEC holds tangential E at zero on the boundary node;
 *                 periodic pairs wrap the difference operators (oracle-only).
 *   - Sec. 2.3    real permittivity per Yee E position (diagonal), Drude/Lorentz
 *                 poles integrated with the trapezoidal ADE; or (tensor mode, no
 *                 poles) a symmetric eps^{-1} tensor per grid node applied to the
 *                 curl through the node assembly S = D^{-1/2} (1/8 sum R^T eps^-1 R) D^{-1/2}.
 *   - Sec. 2.4    DFT monitors over a box of cells (plane, patch or point) with the
 *                 half-step magnetic phase.
 *   - Sec. 3.1, Eq. (adjoint): reverse recursion, transposed curls, the CPML
 *                 transpose  psibar_mem = psibar + ybar, Dbar = ybar/kappa + c psibar_mem,
 *                 psibar_old = b psibar_mem, and the transposed 2x2 pole system;
 *                 material cotangent w.r.t. eps^{-1}; pole-parameter cotangents
 *                 (d J / d(deps, w, gamma) of each pole) through the transposed
 *                 dispersion update.
 *
 * Readings where the paper is silent (all listed with their reasons in the
 * design notes of the repository):
 *   units c = eps0 = mu0 = 1, h = 1, dt = S; Yee positions Ex(i+1/2,j,k),
 *   Ey(i,j+1/2,k), Ez(i,j,k+1/2), Hx(i,j+1/2,k+1/2), Hy(i+1/2,j,k+1/2),
 *   Hz(i+1/2,j+1/2,k); PEC walls at coordinate 0 and N of a non-periodic axis;
 *   CPML sigma(rho) = sigma_max (rho/d)^m, kappa = 1 + (kappa_max-1)(rho/d)^m,
 *   alpha = alpha_max (1 - rho/d), b = exp(-(sigma/kappa + alpha) S),
 *   c = sigma (b-1) / (sigma kappa + kappa^2 alpha)  (c = 0 when sigma = 0);
 *   ADE per pole in per-step time: dP/dt = Q, dQ/dt = -gamma Q - a0 P + b1 E,
 *   Lorentz a0 = w0^2, b1 = deps w0^2; Drude a0 = 0, b1 = wp^2; trapezoidal
 *   rule on x = (P,Q), D = eps_inf E + sum_p P_p, dD/dt = curl H.
 *   DFT: F(w) = sum_n f(t_n) exp(+i w t_n), no dt factor.
 *
 * Index of a cell: idx = (k*ny + j)*nx + i (x fastest).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#define MAXP 16
#define MAXSRC 64
#define MAXMON 16

typedef struct {
    int comp;            /* 0..2 = Ex..Ez, 3..5 = Hx..Hz */
    int lo[3], hi[3];    /* half-open box */
    double *wave;        /* wave[n] is added at forward step n (time n+1 for E, n+3/2 for H) */
    int n;
} osrc_t;

typedef struct {
    int lo[3], hi[3];    /* half-open box of cells (a plane, a patch of a plane, a point) */
    unsigned mask;       /* bit c set: component c (0..5) recorded */
    int ncomp, comps[6];
    int nf;
    double *omega;       /* rad / step */
    long ncell;          /* box cells, x fastest */
    double *acc;         /* [ncomp][nf][ncell] complex (re, im) */
    double *cot;         /* adjoint source, same layout, or NULL */
} omon_t;

typedef struct oracle {
    int N[3];
    long ncell;
    double S;
    int periodic[3];
    int cpml[6];
    double m, kappa_max, alpha_max, sigma_max;
    /* CPML coefficients per axis: E-derivatives at integer nodes, H-derivatives at half nodes */
    double *eb[3], *ec[3], *ek[3];
    double *hb[3], *hc[3], *hk[3];
    /* materials */
    double *inv_eps[3];
    int npole;
    double a0[MAXP], b1[MAXP], gam[MAXP];
    int pkind[MAXP]; double pdeps[MAXP], pw[MAXP];   /* the pole parameters as given */
    double M[MAXP][2][2], g[MAXP][2];   /* x^{n+1} = M x^n + g (E^{n+1} + E^n) */
    /* cotangents of (M00, M01, M10, M11, g0, g1) of each pole, summed over the
     * dispersive cells, components and adjoint steps since the last adj_reset */
    double pgc[MAXP][6];
    unsigned char *mask;
    /* forward state */
    double *F[6];                 /* Ex Ey Ez Hx Hy Hz */
    double *psiE[3][2], *psiH[3][2];
    double *P[3][MAXP], *Q[3][MAXP];
    long step;
    /* sources, monitors, energy */
    int nsrc; osrc_t src[MAXSRC];
    int nmon; omon_t mon[MAXMON];
    int energy_on; long energy_cap; double *energy;
    /* adjoint state (natural cotangents) */
    double *A[6];
    double *apsiE[3][2], *apsiH[3][2];
    double *aP[3][MAXP], *aQ[3][MAXP];
    int design_on; int dlo[3], dhi[3]; long dcell; double *grad[6];
    /* tensor mode (Sec. 2.3): eps^-1 per node, components xx yy zz xy xz yz; D per E edge */
    int tensor_on; double *tinv[6]; double *tD[3]; double *tscr[3], *tacc[3];
    /* scratch */
    double *tmpE[3], *curl[3], *tmpH[3];
    int threads;                  /* OpenMP team size of the cell loops (1: serial) */
} oracle_t;

static long IDX(const oracle_t *o, int i, int j, int k) { return ((long)k * o->N[1] + j) * o->N[0] + i; }

static double *zalloc(long n) { return (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

/* Value of array a at integer coordinates c (may be one outside the grid):
 * wraps on a periodic axis, else returns 0 (no node beyond a PEC wall). */
static double at(const oracle_t *o, const double *a, int c0, int c1, int c2) {
    int c[3] = {c0, c1, c2};
    for (int q = 0; q < 3; ++q) {
        if (c[q] < 0) { if (o->periodic[q]) c[q] += o->N[q]; else return 0.0; }
        if (c[q] >= o->N[q]) { if (o->periodic[q]) c[q] -= o->N[q]; else return 0.0; }
    }
    return a[IDX(o, c[0], c[1], c[2])];
}
/* Scatter-add into array a at c (wrap / drop like at()). */
static void add_at(const oracle_t *o, double *a, int c0, int c1, int c2, double v) {
    int c[3] = {c0, c1, c2};
    for (int q = 0; q < 3; ++q) {
        if (c[q] < 0) { if (o->periodic[q]) c[q] += o->N[q]; else return; }
        if (c[q] >= o->N[q]) { if (o->periodic[q]) c[q] -= o->N[q]; else return; }
    }
    a[IDX(o, c[0], c[1], c[2])] += v;
}

/* CPML profile at coordinate x (cells) along axis q.  Outside the layer the
 * derivative is the plain difference: b = 1, c = 0, 1/kappa = 1. */
static void cpml_coef(const oracle_t *o, int q, double x, double *b, double *c, double *kinv) {
    int dlo = o->cpml[2 * q], dhi = o->cpml[2 * q + 1];
    double Nq = (double)o->N[q];
    double rho = -1.0, d = 1.0;
    if (dlo > 0 && x < (double)dlo) { rho = (double)dlo - x; d = (double)dlo; }
    else if (dhi > 0 && x > Nq - (double)dhi) { rho = x - (Nq - (double)dhi); d = (double)dhi; }
    if (rho < 0.0) { *b = 1.0; *c = 0.0; *kinv = 1.0; return; }
    if (rho > d) rho = d;
    double smax = o->sigma_max < 0.0 ? 0.8 * (o->m + 1.0) : o->sigma_max;
    double r = pow(rho / d, o->m);
    double sigma = smax * r;
    double kappa = 1.0 + (o->kappa_max - 1.0) * r;
    double alpha = o->alpha_max * (1.0 - rho / d);
    double bb = exp(-(sigma / kappa + alpha) * o->S);
    double cc = 0.0;
    if (sigma > 0.0) cc = sigma * (bb - 1.0) / (sigma * kappa + kappa * kappa * alpha);
    *b = bb; *c = cc; *kinv = 1.0 / kappa;
}

oracle_t *oracle_create(int nx, int ny, int nz, double S, const int *periodic, const int *cpml,
                        double m, double kappa_max, double alpha_max, double sigma_max) {
    oracle_t *o = (oracle_t *)calloc(1, sizeof(oracle_t));
    o->N[0] = nx; o->N[1] = ny; o->N[2] = nz;
    o->ncell = (long)nx * ny * nz;
    o->S = S;
    o->threads = 1;
    for (int q = 0; q < 3; ++q) o->periodic[q] = periodic ? periodic[q] : 0;
    for (int f = 0; f < 6; ++f) o->cpml[f] = cpml ? cpml[f] : 0;
    o->m = m; o->kappa_max = kappa_max; o->alpha_max = alpha_max; o->sigma_max = sigma_max;
    for (int q = 0; q < 3; ++q) {
        int n = o->N[q];
        o->eb[q] = zalloc(n); o->ec[q] = zalloc(n); o->ek[q] = zalloc(n);
        o->hb[q] = zalloc(n); o->hc[q] = zalloc(n); o->hk[q] = zalloc(n);
        for (int j = 0; j < n; ++j) {
            cpml_coef(o, q, (double)j, &o->eb[q][j], &o->ec[q][j], &o->ek[q][j]);
            cpml_coef(o, q, (double)j + 0.5, &o->hb[q][j], &o->hc[q][j], &o->hk[q][j]);
        }
    }
    for (int a = 0; a < 3; ++a) {
        o->inv_eps[a] = zalloc(o->ncell);
        for (long c = 0; c < o->ncell; ++c) o->inv_eps[a][c] = 1.0;
    }
    o->mask = (unsigned char *)calloc((size_t)o->ncell, 1);
    for (int f = 0; f < 6; ++f) { o->F[f] = zalloc(o->ncell); o->A[f] = zalloc(o->ncell); }
    for (int a = 0; a < 3; ++a)
        for (int s = 0; s < 2; ++s) {
            o->psiE[a][s] = zalloc(o->ncell); o->psiH[a][s] = zalloc(o->ncell);
            o->apsiE[a][s] = zalloc(o->ncell); o->apsiH[a][s] = zalloc(o->ncell);
        }
    for (int a = 0; a < 3; ++a) {
        o->tmpE[a] = zalloc(o->ncell); o->curl[a] = zalloc(o->ncell); o->tmpH[a] = zalloc(o->ncell);
    }
    return o;
}

void oracle_destroy(oracle_t *o) {
    if (!o) return;
    for (int q = 0; q < 3; ++q) {
        free(o->eb[q]); free(o->ec[q]); free(o->ek[q]); free(o->hb[q]); free(o->hc[q]); free(o->hk[q]);
        free(o->inv_eps[q]); free(o->tmpE[q]); free(o->curl[q]); free(o->tmpH[q]); free(o->grad[q]);
        free(o->grad[3 + q]); free(o->tinv[q]); free(o->tinv[3 + q]); free(o->tD[q]); free(o->tscr[q]); free(o->tacc[q]);
        for (int s = 0; s < 2; ++s) { free(o->psiE[q][s]); free(o->psiH[q][s]); free(o->apsiE[q][s]); free(o->apsiH[q][s]); }
        for (int p = 0; p < o->npole; ++p) { free(o->P[q][p]); free(o->Q[q][p]); free(o->aP[q][p]); free(o->aQ[q][p]); }
    }
    for (int f = 0; f < 6; ++f) { free(o->F[f]); free(o->A[f]); }
    free(o->mask);
    for (int s = 0; s < o->nsrc; ++s) free(o->src[s].wave);
    for (int s = 0; s < o->nmon; ++s) { free(o->mon[s].omega); free(o->mon[s].acc); free(o->mon[s].cot); }
    free(o->energy);
    free(o);
}

/* 2x2 helpers for the trapezoidal pole update (Sec. 2.3, Okoniewski's ADE). */
static void mat2_inv(const double A[2][2], double R[2][2]) {
    double det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    R[0][0] = A[1][1] / det; R[0][1] = -A[0][1] / det;
    R[1][0] = -A[1][0] / det; R[1][1] = A[0][0] / det;
}
static void mat2_mul(const double A[2][2], const double B[2][2], double R[2][2]) {
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) R[r][c] = A[r][0] * B[0][c] + A[r][1] * B[1][c];
}

/* kinds: 0 = Lorentz (deps, w0, gamma), 1 = Drude (unused, wp, gamma).
 * Each pole p: x' = A x + bvec E with A = [[0,1],[-a0,-gamma]], bvec = (0,b1).
 * Trapezoidal: (I - A/2) x^{n+1} = (I + A/2) x^n + (bvec/2)(E^{n+1} + E^n). */
void oracle_set_material(oracle_t *o, const double *iex, const double *iey, const double *iez,
                         int npole, const int *kind, const double *deps, const double *w,
                         const double *gamma, const unsigned char *mask) {
    const double *ie[3] = {iex, iey, iez};
    for (int a = 0; a < 3; ++a)
        if (ie[a]) memcpy(o->inv_eps[a], ie[a], sizeof(double) * (size_t)o->ncell);
    for (int a = 0; a < 3; ++a)
        for (int p = 0; p < o->npole; ++p) { free(o->P[a][p]); free(o->Q[a][p]); free(o->aP[a][p]); free(o->aQ[a][p]); }
    o->npole = npole;
    for (int p = 0; p < npole; ++p) {
        o->pkind[p] = kind[p]; o->pdeps[p] = deps[p]; o->pw[p] = w[p];
        if (kind[p] == 0) { o->a0[p] = w[p] * w[p]; o->b1[p] = deps[p] * w[p] * w[p]; }
        else { o->a0[p] = 0.0; o->b1[p] = w[p] * w[p]; }
        o->gam[p] = gamma[p];
        double A[2][2] = {{0.0, 1.0}, {-o->a0[p], -o->gam[p]}};
        double Im[2][2], Ip[2][2], Iminv[2][2];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) {
                double id = (r == c) ? 1.0 : 0.0;
                Im[r][c] = id - 0.5 * A[r][c];
                Ip[r][c] = id + 0.5 * A[r][c];
            }
        mat2_inv(Im, Iminv);
        mat2_mul(Iminv, Ip, o->M[p]);
        /* g = (I - A/2)^{-1} bvec / 2 */
        o->g[p][0] = Iminv[0][1] * o->b1[p] * 0.5;
        o->g[p][1] = Iminv[1][1] * o->b1[p] * 0.5;
        for (int a = 0; a < 3; ++a) {
            o->P[a][p] = zalloc(o->ncell); o->Q[a][p] = zalloc(o->ncell);
            o->aP[a][p] = zalloc(o->ncell); o->aQ[a][p] = zalloc(o->ncell);
        }
    }
    if (mask) memcpy(o->mask, mask, (size_t)o->ncell);
    else memset(o->mask, 0, (size_t)o->ncell);
}

int oracle_add_source(oracle_t *o, int comp, const int *lo, const int *hi, const double *wave, int n) {
    if (o->nsrc >= MAXSRC) return -1;
    osrc_t *s = &o->src[o->nsrc];
    s->comp = comp;
    for (int q = 0; q < 3; ++q) { s->lo[q] = lo[q]; s->hi[q] = hi[q]; }
    s->wave = zalloc(n); memcpy(s->wave, wave, sizeof(double) * (size_t)n); s->n = n;
    return o->nsrc++;
}

int oracle_add_dft_box(oracle_t *o, const int *lo, const int *hi, unsigned mask, int nf, const double *omega) {
    if (o->nmon >= MAXMON) return -1;
    omon_t *m = &o->mon[o->nmon];
    for (int q = 0; q < 3; ++q) { m->lo[q] = lo[q]; m->hi[q] = hi[q]; }
    m->mask = mask; m->nf = nf;
    m->ncomp = 0;
    for (int c = 0; c < 6; ++c) if (mask & (1u << c)) m->comps[m->ncomp++] = c;
    m->omega = zalloc(nf); memcpy(m->omega, omega, sizeof(double) * (size_t)nf);
    m->ncell = (long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
    m->acc = zalloc(2L * m->ncomp * nf * m->ncell);
    m->cot = NULL;
    return o->nmon++;
}

void oracle_enable_energy(oracle_t *o, long cap) {
    if (o->tensor_on) return;   /* the energy below is the diagonal one */
    free(o->energy);
    o->energy = zalloc(cap); o->energy_cap = cap; o->energy_on = 1;
}

/* Grid cell of the c-th cell of monitor box m (x fastest). */
static void mon_cell(const omon_t *m, long c, int *i, int *j, int *k) {
    long bx = m->hi[0] - m->lo[0], by = m->hi[1] - m->lo[1];
    *i = m->lo[0] + (int)(c % bx);
    *j = m->lo[1] + (int)((c / bx) % by);
    *k = m->lo[2] + (int)(c / (bx * by));
}

/* Accumulate F += f(t) exp(i w t) for the components of one field kind. */
static void dft_accumulate(oracle_t *o, int magnetic, double t) {
    for (int s = 0; s < o->nmon; ++s) {
        omon_t *m = &o->mon[s];
        for (int ci = 0; ci < m->ncomp; ++ci) {
            int comp = m->comps[ci];
            if ((comp >= 3) != magnetic) continue;
            for (int f = 0; f < m->nf; ++f) {
                double cr = cos(m->omega[f] * t), si = sin(m->omega[f] * t);
                double *acc = m->acc + 2L * ((long)ci * m->nf + f) * m->ncell;
#pragma omp parallel for num_threads(o->threads) if (o->threads > 1 && m->ncell >= 4096)
                for (long c = 0; c < m->ncell; ++c) {
                    int i, j, k; mon_cell(m, c, &i, &j, &k);
                    double v = o->F[comp][IDX(o, i, j, k)];
                    acc[2 * c] += v * cr;
                    acc[2 * c + 1] += v * si;
                }
            }
        }
    }
}

static int is_pec_E(const oracle_t *o, int a, const int c[3]) {
    for (int q = 0; q < 3; ++q)
        if (q != a && !o->periodic[q] && c[q] == 0) return 1;
    return 0;
}

/* ---------------- symmetric tensors at the nodes, Sec. 2.3 ----------------
 * Grid node n = (i, j, k) carries eps^-1_n (symmetric, 3 x 3).  For a choice c in {0,1}^3,
 * R_{n,c} picks one E edge per axis next to the node: along axis q the edge whose coordinate is
 * n_q - 1 + c_q (the E_q array index; it wraps on a periodic axis and is absent below 0 on a
 * non-periodic one), the other two coordinates those of the node.  The assembly is
 *   A = 1/8 sum_n sum_c R_{n,c}^T eps^-1_n R_{n,c},   D = 1/8 sum_n sum_c R_{n,c}^T R_{n,c},
 * D diagonal (the same sum with the identity tensor), and the E update applies
 *   S_t = D^{-1/2} A D^{-1/2}
 * to the curl: E^{n+1} = E^n + S S_t C.  PEC-held edges are not unknowns: the operator reads them
 * as zero and leaves them alone.  With eps^-1 <= I at every node, A <= D, so ||S_t|| <= 1 and the
 * vacuum time step stays admissible. */
static int tcomp(int u, int v) {
    if (u == v) return u;
    if (u + v == 1) return 3;   /* xy */
    if (u + v == 2) return 4;   /* xz */
    return 5;                   /* yz */
}

/* Coordinate along axis q of the edge that choice bit cq picks at node coordinate x, or -1. */
static int edge_coord(const oracle_t *o, int q, int x, int cq) {
    int e = x - 1 + cq;
    if (e < 0) { if (!o->periodic[q]) return -1; e += o->N[q]; }
    return e;
}

/* Edge ids (or -1) of choice c at node (i, j, k), per axis. */
static void node_edges(const oracle_t *o, int i, int j, int k, int c, long id[3]) {
    const int n[3] = {i, j, k};
    for (int a = 0; a < 3; ++a) {
        int e[3] = {i, j, k};
        e[a] = edge_coord(o, a, n[a], (c >> a) & 1);
        id[a] = -1;
        if (e[a] < 0 || is_pec_E(o, a, e)) continue;
        id[a] = IDX(o, e[0], e[1], e[2]);
    }
}

/* out = S_t in (full arrays of the three E components). */
static void tensor_apply(oracle_t *o, double *const in[3], double *const out[3]) {
    const int nx = o->N[0], ny = o->N[1], nz = o->N[2];
    for (int a = 0; a < 3; ++a) memset(o->tacc[a], 0, sizeof(double) * (size_t)o->ncell);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long n = IDX(o, i, j, k);
                for (int c = 0; c < 8; ++c) {
                    long id[3];
                    node_edges(o, i, j, k, c, id);
                    double v[3], u[3];
                    for (int a = 0; a < 3; ++a) v[a] = id[a] >= 0 ? in[a][id[a]] / sqrt(o->tD[a][id[a]]) : 0.0;
                    for (int a = 0; a < 3; ++a) {
                        u[a] = 0.0;
                        for (int b = 0; b < 3; ++b) u[a] += o->tinv[tcomp(a, b)][n] * v[b];
                    }
                    for (int a = 0; a < 3; ++a)
                        if (id[a] >= 0) o->tacc[a][id[a]] += u[a] / 8.0;
                }
            }
    for (int a = 0; a < 3; ++a)
        for (long e = 0; e < o->ncell; ++e) out[a][e] = o->tD[a][e] > 0.0 ? o->tacc[a][e] / sqrt(o->tD[a][e]) : 0.0;
}

/* Tensor mode on (t6 = six full node arrays xx yy zz xy xz yz) or off (t6 = NULL).
 * -1 with poles or an energy record (neither is defined here for tensors). */
int oracle_set_tensor(oracle_t *o, const double *t6) {
    if (!t6) { o->tensor_on = 0; return 0; }
    if (o->npole > 0 || o->energy_on) return -1;
    const int nx = o->N[0], ny = o->N[1], nz = o->N[2];
    for (int q = 0; q < 6; ++q) {
        if (!o->tinv[q]) o->tinv[q] = zalloc(o->ncell);
        memcpy(o->tinv[q], t6 + (long)q * o->ncell, sizeof(double) * (size_t)o->ncell);
    }
    for (int a = 0; a < 3; ++a) {
        if (!o->tD[a]) { o->tD[a] = zalloc(o->ncell); o->tscr[a] = zalloc(o->ncell); o->tacc[a] = zalloc(o->ncell); }
        memset(o->tD[a], 0, sizeof(double) * (size_t)o->ncell);
    }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                for (int c = 0; c < 8; ++c) {
                    long id[3];
                    node_edges(o, i, j, k, c, id);
                    for (int a = 0; a < 3; ++a)
                        if (id[a] >= 0) o->tD[a][id[a]] += 1.0 / 8.0;
                }
    o->tensor_on = 1;
    return 0;
}

/* The assembled operator on three arrays (in tensor mode; -1 otherwise). */
int oracle_tensor_apply(oracle_t *o, const double *inx, const double *iny, const double *inz, double *outx,
                        double *outy, double *outz) {
    if (!o->tensor_on) return -1;
    double *in[3] = {(double *)inx, (double *)iny, (double *)inz}, *out[3] = {outx, outy, outz};
    tensor_apply(o, in, out);
    return 0;
}

/* The diagonal D of the assembly for E component a (tensor mode; NULL otherwise). */
double *oracle_tensor_D(oracle_t *o, int a) { return o->tensor_on ? o->tD[a] : NULL; }

/* E-phase of Eq. (yee): reads E, H, psiE, P, Q; writes Enew (pre-source), psiE_out,
 * P/Q outputs and the CPML-corrected curl.  Output arrays may alias inputs
 * because every cell reads only its own E/psi/P/Q and the (unchanged) H. */
static void e_phase(oracle_t *o, double *const Eout[3], double *const psiout[3][2],
                    double *const Pout[3][MAXP], double *const Qout[3][MAXP]) {
    const int nx = o->N[0], ny = o->N[1], nz = o->N[2];
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, cax = (a + 2) % 3;
        const double *Hc = o->F[3 + cax], *Hb = o->F[3 + b];
#pragma omp parallel for num_threads(o->threads) if (o->threads > 1)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    int c[3] = {i, j, k};
                    long id = IDX(o, i, j, k);
                    if (is_pec_E(o, a, c)) {
                        Eout[a][id] = o->F[a][id];
                        o->curl[a][id] = 0.0;
                        continue;
                    }
                    int cb[3] = {i, j, k}; cb[b] -= 1;
                    int cc[3] = {i, j, k}; cc[cax] -= 1;
                    double d1 = Hc[id] - at(o, Hc, cb[0], cb[1], cb[2]);   /* dHc/dx_b */
                    double d2 = Hb[id] - at(o, Hb, cc[0], cc[1], cc[2]);   /* dHb/dx_c */
                    int pb = c[b], pc = c[cax];
                    double ps1 = o->eb[b][pb] * o->psiE[a][0][id] + o->ec[b][pb] * d1;
                    double ps2 = o->eb[cax][pc] * o->psiE[a][1][id] + o->ec[cax][pc] * d2;
                    double y1 = o->ek[b][pb] * d1 + ps1;
                    double y2 = o->ek[cax][pc] * d2 + ps2;
                    double cu = y1 - y2;
                    psiout[a][0][id] = ps1;
                    psiout[a][1][id] = ps2;
                    o->curl[a][id] = cu;
                    double E = o->F[a][id];
                    if (o->tensor_on) {
                        Eout[a][id] = E;   /* updated below, once every curl is known */
                    } else if (o->npole > 0 && o->mask[id]) {
                        double eps = 1.0 / o->inv_eps[a][id];
                        double G = 0.0, num = eps * E + o->S * cu;
                        for (int p = 0; p < o->npole; ++p) {
                            double Pp = o->P[a][p][id], Qp = o->Q[a][p][id];
                            double MxP = o->M[p][0][0] * Pp + o->M[p][0][1] * Qp;
                            num += Pp - MxP - o->g[p][0] * E;
                            G += o->g[p][0];
                        }
                        double En = num / (eps + G);
                        for (int p = 0; p < o->npole; ++p) {
                            double Pp = o->P[a][p][id], Qp = o->Q[a][p][id];
                            double Pn = o->M[p][0][0] * Pp + o->M[p][0][1] * Qp + o->g[p][0] * (En + E);
                            double Qn = o->M[p][1][0] * Pp + o->M[p][1][1] * Qp + o->g[p][1] * (En + E);
                            Pout[a][p][id] = Pn; Qout[a][p][id] = Qn;
                        }
                        Eout[a][id] = En;
                    } else {
                        Eout[a][id] = E + o->S * o->inv_eps[a][id] * cu;
                        for (int p = 0; p < o->npole; ++p) {
                            Pout[a][p][id] = o->P[a][p][id]; Qout[a][p][id] = o->Q[a][p][id];
                        }
                    }
                }
    }
    if (o->tensor_on) {
        /* E^{n+1} = E^n + S S_t C over the whole curl field */
        tensor_apply(o, o->curl, o->tscr);
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) {
                        int c[3] = {i, j, k};
                        if (is_pec_E(o, a, c)) continue;
                        long id = IDX(o, i, j, k);
                        Eout[a][id] = o->F[a][id] + o->S * o->tscr[a][id];
                    }
    }
}

static void add_sources(oracle_t *o, int magnetic, long n) {
    for (int s = 0; s < o->nsrc; ++s) {
        osrc_t *sr = &o->src[s];
        if ((sr->comp >= 3) != magnetic) continue;
        if (n >= sr->n) continue;
        double v = sr->wave[n];
        for (int k = sr->lo[2]; k < sr->hi[2]; ++k)
            for (int j = sr->lo[1]; j < sr->hi[1]; ++j)
                for (int i = sr->lo[0]; i < sr->hi[0]; ++i) o->F[sr->comp][IDX(o, i, j, k)] += v;
    }
}

/* H-phase of Eq. (yee): H -= S * curl(E) with CPML at half-integer nodes. */
static void h_phase(oracle_t *o) {
    const int nx = o->N[0], ny = o->N[1], nz = o->N[2];
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, cax = (a + 2) % 3;
        const double *Ec = o->F[cax], *Eb = o->F[b];
        double *H = o->F[3 + a];
#pragma omp parallel for num_threads(o->threads) if (o->threads > 1)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    int c[3] = {i, j, k};
                    long id = IDX(o, i, j, k);
                    int cb[3] = {i, j, k}; cb[b] += 1;
                    int cc[3] = {i, j, k}; cc[cax] += 1;
                    double d1 = at(o, Ec, cb[0], cb[1], cb[2]) - Ec[id];   /* dEc/dx_b */
                    double d2 = at(o, Eb, cc[0], cc[1], cc[2]) - Eb[id];   /* dEb/dx_c */
                    int pb = c[b], pc = c[cax];
                    double ps1 = o->hb[b][pb] * o->psiH[a][0][id] + o->hc[b][pb] * d1;
                    double ps2 = o->hb[cax][pc] * o->psiH[a][1][id] + o->hc[cax][pc] * d2;
                    o->psiH[a][0][id] = ps1;
                    o->psiH[a][1][id] = ps2;
                    double y1 = o->hk[b][pb] * d1 + ps1;
                    double y2 = o->hk[cax][pc] * d2 + ps2;
                    o->tmpH[a][id] = H[id];
                    H[id] = H[id] - o->S * (y1 - y2);
                }
    }
}

static void record_energy(oracle_t *o) {
    /* W_{n+1} = 1/2 sum eps |E^{n+1}|^2 + 1/2 sum H^{n+1/2} . H^{n+3/2} */
    double w = 0.0;
    for (int a = 0; a < 3; ++a)
        for (long c = 0; c < o->ncell; ++c) {
            w += 0.5 * o->F[a][c] * o->F[a][c] / o->inv_eps[a][c];
            w += 0.5 * o->tmpH[a][c] * o->F[3 + a][c];
        }
    if (o->step < o->energy_cap) o->energy[o->step] = w;
}

/* One forward step n -> n+1 in the order of Eq. (yee) and Sec. 2.1. */
static void step_once(oracle_t *o) {
    long n = o->step;
    double *Eout[3] = {o->F[0], o->F[1], o->F[2]};
    e_phase(o, Eout, o->psiE, o->P, o->Q);
    add_sources(o, 0, n);
    dft_accumulate(o, 0, (double)(n + 1));
    h_phase(o);
    add_sources(o, 1, n);
    dft_accumulate(o, 1, (double)n + 1.5);
    if (o->energy_on) record_energy(o);
    o->step = n + 1;
}

void oracle_step(oracle_t *o, int n) { for (int s = 0; s < n; ++s) step_once(o); }

/* Team size of the cell loops of the forward step (values < 1 mean 1).  Results do not
 * depend on it. */
void oracle_set_threads(oracle_t *o, int n) { o->threads = n < 1 ? 1 : n; }

/* Reversible reconstruction (Sec. 3.2: lossless nondispersive problems step Eq. (yee)
 * backward): one backward step u^{n+1} -> u^n undoes the forward step n in reverse order,
 *   H^{n+1/2} = (H^{n+3/2} - m^n) + S curl E^{n+1},
 *   E^n       = (E^{n+1} - s^n) - S eps^-1 curl H^{n+1/2},
 * with the plain differences of Eq. (yee) (no CPML memory, no pole state: the caller must
 * hold a domain without CPML layers and without poles; returns -1 otherwise).  DFT monitors
 * and energies are not touched.  PEC-held E nodes stay as they are. */
static void sub_sources(oracle_t *o, int magnetic, long n) {
    for (int s = 0; s < o->nsrc; ++s) {
        osrc_t *sr = &o->src[s];
        if ((sr->comp >= 3) != magnetic) continue;
        if (n >= sr->n) continue;
        double v = sr->wave[n];
        for (int k = sr->lo[2]; k < sr->hi[2]; ++k)
            for (int j = sr->lo[1]; j < sr->hi[1]; ++j)
                for (int i = sr->lo[0]; i < sr->hi[0]; ++i) o->F[sr->comp][IDX(o, i, j, k)] -= v;
    }
}

int oracle_step_backward(oracle_t *o, int n) {
    for (int q = 0; q < 3; ++q)
        if (o->cpml[2 * q] || o->cpml[2 * q + 1]) return -1;
    if (o->npole > 0 || o->tensor_on) return -1;
    const int nx = o->N[0], ny = o->N[1], nz = o->N[2];
    for (int s = 0; s < n && o->step > 0; ++s) {
        const long m = o->step - 1;
        /* H: every H node reads E^{n+1} only, so the whole H update can be done in place */
        sub_sources(o, 1, m);
        for (int a = 0; a < 3; ++a) {
            int b = (a + 1) % 3, cax = (a + 2) % 3;
            const double *Ec = o->F[cax], *Eb = o->F[b];
            double *H = o->F[3 + a];
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) {
                        long id = IDX(o, i, j, k);
                        int cb[3] = {i, j, k}; cb[b] += 1;
                        int cc[3] = {i, j, k}; cc[cax] += 1;
                        double d1 = at(o, Ec, cb[0], cb[1], cb[2]) - Ec[id];   /* dEc/dx_b */
                        double d2 = at(o, Eb, cc[0], cc[1], cc[2]) - Eb[id];   /* dEb/dx_c */
                        H[id] = H[id] + o->S * (d1 - d2);
                    }
        }
        /* E: reads the reconstructed H only */
        sub_sources(o, 0, m);
        for (int a = 0; a < 3; ++a) {
            int b = (a + 1) % 3, cax = (a + 2) % 3;
            const double *Hc = o->F[3 + cax], *Hb = o->F[3 + b];
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) {
                        int c[3] = {i, j, k};
                        long id = IDX(o, i, j, k);
                        if (is_pec_E(o, a, c)) continue;
                        int cb[3] = {i, j, k}; cb[b] -= 1;
                        int cc[3] = {i, j, k}; cc[cax] -= 1;
                        double d1 = Hc[id] - at(o, Hc, cb[0], cb[1], cb[2]);   /* dHc/dx_b */
                        double d2 = Hb[id] - at(o, Hb, cc[0], cc[1], cc[2]);   /* dHb/dx_c */
                        o->F[a][id] = o->F[a][id] - o->S * o->inv_eps[a][id] * (d1 - d2);
                    }
        }
        o->step = m;
    }
    return 0;
}

/* Absorbing-face variant of the reversible reconstruction (Sec. 3.2: the fields at the interface
 * between interior and absorber are recorded so that the interior reconstruction stays lossless).
 * The interior is the set of cells whose own node lies in no CPML slab along any axis; its E and H
 * updates use no memory variable, so they can be undone exactly like a lossless domain's.  One
 * backward step undoes forward step n = step - 1 on the interior only, in reverse order:
 *   every E node outside the interior takes E^{n+1} from the record rec_e (three full-grid arrays;
 *   only nodes outside the interior are read), then the interior H nodes
 *   H^{n+1/2} = (H^{n+3/2} - m^n) + S curl E^{n+1};
 *   every H node outside the interior takes H^{n+1/2} from rec_h, then the interior E nodes
 *   E^n = (E^{n+1} - s^n) - S eps^-1 curl H^{n+1/2}.
 * Cells outside the interior end up holding the recorded values (their memories and the absorber
 * state are not reconstructed).  Poles: -1 (dispersion is not reversible). */
static int in_interior(const oracle_t *o, int i, int j, int k) {
    const int c[3] = {i, j, k};
    for (int q = 0; q < 3; ++q) {
        const int lo = o->cpml[2 * q], hi = o->cpml[2 * q + 1];
        if (c[q] < lo || c[q] >= o->N[q] - hi) return 0;
    }
    return 1;
}

int oracle_step_backward_interior(oracle_t *o, const double *rex, const double *rey, const double *rez,
                                  const double *rhx, const double *rhy, const double *rhz) {
    if (o->npole > 0 || o->tensor_on || o->step < 1) return -1;
    const int nx = o->N[0], ny = o->N[1], nz = o->N[2];
    const double *re[3] = {rex, rey, rez}, *rh[3] = {rhx, rhy, rhz};
    const long m = o->step - 1;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                if (!in_interior(o, i, j, k))
                    for (int a = 0; a < 3; ++a) o->F[a][IDX(o, i, j, k)] = re[a][IDX(o, i, j, k)];
    sub_sources(o, 1, m);
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, cax = (a + 2) % 3;
        const double *Ec = o->F[cax], *Eb = o->F[b];
        double *H = o->F[3 + a];
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    if (!in_interior(o, i, j, k)) continue;
                    long id = IDX(o, i, j, k);
                    int cb[3] = {i, j, k}; cb[b] += 1;
                    int cc[3] = {i, j, k}; cc[cax] += 1;
                    double d1 = at(o, Ec, cb[0], cb[1], cb[2]) - Ec[id];   /* dEc/dx_b */
                    double d2 = at(o, Eb, cc[0], cc[1], cc[2]) - Eb[id];   /* dEb/dx_c */
                    H[id] = H[id] + o->S * (d1 - d2);
                }
    }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                if (!in_interior(o, i, j, k))
                    for (int a = 0; a < 3; ++a) o->F[3 + a][IDX(o, i, j, k)] = rh[a][IDX(o, i, j, k)];
    sub_sources(o, 0, m);
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, cax = (a + 2) % 3;
        const double *Hc = o->F[3 + cax], *Hb = o->F[3 + b];
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    int c[3] = {i, j, k};
                    if (!in_interior(o, i, j, k) || is_pec_E(o, a, c)) continue;
                    long id = IDX(o, i, j, k);
                    int cb[3] = {i, j, k}; cb[b] -= 1;
                    int cc[3] = {i, j, k}; cc[cax] -= 1;
                    double d1 = Hc[id] - at(o, Hc, cb[0], cb[1], cb[2]);   /* dHc/dx_b */
                    double d2 = Hb[id] - at(o, Hb, cc[0], cc[1], cc[2]);   /* dHb/dx_c */
                    o->F[a][id] = o->F[a][id] - o->S * o->inv_eps[a][id] * (d1 - d2);
                }
    }
    o->step = m;
    return 0;
}

/* ---------------- access ---------------- */
double *oracle_field(oracle_t *o, int comp) { return o->F[comp]; }
double *oracle_psi(oracle_t *o, int magnetic, int comp, int which) {
    return magnetic ? o->psiH[comp][which] : o->psiE[comp][which];
}
double *oracle_pole(oracle_t *o, int comp, int pole, int which) { return which ? o->Q[comp][pole] : o->P[comp][pole]; }
double *oracle_dft(oracle_t *o, int mon) { return o->mon[mon].acc; }
long oracle_dft_len(oracle_t *o, int mon) { return 2L * o->mon[mon].ncomp * o->mon[mon].nf * o->mon[mon].ncell; }
double *oracle_energy(oracle_t *o) { return o->energy; }
long oracle_step_count(oracle_t *o) { return o->step; }
void oracle_set_step(oracle_t *o, long s) { o->step = s; }
double *oracle_coef(oracle_t *o, int magnetic, int axis, int which) {
    if (magnetic) return which == 0 ? o->hb[axis] : (which == 1 ? o->hc[axis] : o->hk[axis]);
    return which == 0 ? o->eb[axis] : (which == 1 ? o->ec[axis] : o->ek[axis]);
}
void oracle_pole_coef(oracle_t *o, int p, double *M4, double *g2) {
    M4[0] = o->M[p][0][0]; M4[1] = o->M[p][0][1]; M4[2] = o->M[p][1][0]; M4[3] = o->M[p][1][1];
    g2[0] = o->g[p][0]; g2[1] = o->g[p][1];
}

/* Whole forward state (E, H, psiE, psiH, P, Q) as one vector. */
long oracle_state_len(oracle_t *o) { return o->ncell * (6 + 12 + 6L * o->npole); }
static void state_ptrs(oracle_t *o, double **v, int adj) {
    int n = 0;
    for (int f = 0; f < 6; ++f) v[n++] = adj ? o->A[f] : o->F[f];
    for (int a = 0; a < 3; ++a) for (int s = 0; s < 2; ++s) v[n++] = adj ? o->apsiE[a][s] : o->psiE[a][s];
    for (int a = 0; a < 3; ++a) for (int s = 0; s < 2; ++s) v[n++] = adj ? o->apsiH[a][s] : o->psiH[a][s];
    for (int a = 0; a < 3; ++a) for (int p = 0; p < o->npole; ++p) {
        v[n++] = adj ? o->aP[a][p] : o->P[a][p];
        v[n++] = adj ? o->aQ[a][p] : o->Q[a][p];
    }
}
void oracle_state_get(oracle_t *o, double *buf, int adj) {
    double *v[18 + 6 * MAXP];
    state_ptrs(o, v, adj);
    int nv = 18 + 6 * o->npole;
    for (int s = 0; s < nv; ++s) memcpy(buf + (long)s * o->ncell, v[s], sizeof(double) * (size_t)o->ncell);
}
void oracle_state_set(oracle_t *o, const double *buf, int adj) {
    double *v[18 + 6 * MAXP];
    state_ptrs(o, v, adj);
    int nv = 18 + 6 * o->npole;
    for (int s = 0; s < nv; ++s) memcpy(v[s], buf + (long)s * o->ncell, sizeof(double) * (size_t)o->ncell);
}
void oracle_dft_reset(oracle_t *o) {
    for (int s = 0; s < o->nmon; ++s) memset(o->mon[s].acc, 0, sizeof(double) * (size_t)oracle_dft_len(o, s));
}

/* ---------------- discrete adjoint, Sec. 3.1 / Eq. (adjoint) ----------------
 * Scatter form: every forward assignment y = sum_i c_i x_i becomes
 * xbar_i += c_i ybar, visited in reverse statement order.  State cotangents
 * are the natural ones (of E^n, H^{n+1/2}, psi, P, Q after step n).  PEC
 * nodes are not state: their cotangent is held at zero. */
void oracle_set_adjoint_source(oracle_t *o, int mon, const double *cot) {
    omon_t *m = &o->mon[mon];
    long len = oracle_dft_len(o, mon);
    free(m->cot);
    m->cot = NULL;
    if (!cot) return;
    m->cot = zalloc(len);
    memcpy(m->cot, cot, sizeof(double) * (size_t)len);
}

int oracle_set_design(oracle_t *o, const int *lo, const int *hi) {
    for (int q = 0; q < 3; ++q) { o->dlo[q] = lo[q]; o->dhi[q] = hi[q]; }
    o->dcell = (long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
    for (int a = 0; a < 6; ++a) { free(o->grad[a]); o->grad[a] = zalloc(o->dcell); }
    o->design_on = 1;
    return 0;
}
double *oracle_grad(oracle_t *o, int comp) { return o->grad[comp]; }
double *oracle_adj_field(oracle_t *o, int comp) { return o->A[comp]; }

void oracle_adj_reset(oracle_t *o) {
    double *v[18 + 6 * MAXP];
    state_ptrs(o, v, 1);
    int nv = 18 + 6 * o->npole;
    for (int s = 0; s < nv; ++s) memset(v[s], 0, sizeof(double) * (size_t)o->ncell);
    if (o->design_on) for (int a = 0; a < 6; ++a) memset(o->grad[a], 0, sizeof(double) * (size_t)o->dcell);
    memset(o->pgc, 0, sizeof(o->pgc));
}

/* d J / d(deps, w, gamma) of each pole (out[3p + 0..2]; a Drude pole has no deps) from the
 * coefficient cotangents, by differentiating the trapezoidal construction: with
 * B = I - A/2, M = B^-1 (I + A/2) and g = B^-1 bvec / 2,
 *   dM = B^-1 (dA/2) (M + I),   dg = B^-1 (dA/2) g + B^-1 dbvec / 2,
 * A = [[0, 1], [-a0, -gamma]], bvec = (0, b1); Lorentz a0 = w^2, b1 = deps w^2; Drude a0 = 0,
 * b1 = w^2. */
void oracle_pole_grad(oracle_t *o, double *out) {
    for (int p = 0; p < o->npole; ++p) {
        double A[2][2] = {{0.0, 1.0}, {-o->a0[p], -o->gam[p]}};
        double B[2][2], Binv[2][2];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) B[r][c] = (r == c ? 1.0 : 0.0) - 0.5 * A[r][c];
        mat2_inv(B, Binv);
        const int lor = o->pkind[p] == 0;
        const double w = o->pw[p], de = o->pdeps[p];
        /* (d a0, d b1, d gamma) per parameter */
        const double dpar[3][3] = {{0.0, lor ? w * w : 0.0, 0.0},
                                   {lor ? 2.0 * w : 0.0, lor ? 2.0 * de * w : 2.0 * w, 0.0},
                                   {0.0, 0.0, 1.0}};
        for (int t = 0; t < 3; ++t) {
            double dA[2][2] = {{0.0, 0.0}, {-dpar[t][0], -dpar[t][2]}};
            double hdA[2][2], MI[2][2], T1[2][2], dM[2][2];
            for (int r = 0; r < 2; ++r)
                for (int c = 0; c < 2; ++c) { hdA[r][c] = 0.5 * dA[r][c]; MI[r][c] = o->M[p][r][c] + (r == c ? 1.0 : 0.0); }
            mat2_mul(hdA, MI, T1);
            mat2_mul(Binv, T1, dM);
            /* dg = B^-1 (hdA g + dbvec / 2) */
            double v0 = hdA[0][0] * o->g[p][0] + hdA[0][1] * o->g[p][1];
            double v1 = hdA[1][0] * o->g[p][0] + hdA[1][1] * o->g[p][1] + 0.5 * dpar[t][1];
            double dg0 = Binv[0][0] * v0 + Binv[0][1] * v1;
            double dg1 = Binv[1][0] * v0 + Binv[1][1] * v1;
            out[3 * p + t] = o->pgc[p][0] * dM[0][0] + o->pgc[p][1] * dM[0][1] + o->pgc[p][2] * dM[1][0] +
                             o->pgc[p][3] * dM[1][1] + o->pgc[p][4] * dg0 + o->pgc[p][5] * dg1;
        }
    }
}

/* The coefficient cotangents themselves: out[6p + 0..5] for (M00, M01, M10, M11, g0, g1). */
void oracle_pole_coef_grad(oracle_t *o, double *out) {
    for (int p = 0; p < o->npole; ++p)
        for (int q = 0; q < 6; ++q) out[6 * p + q] = o->pgc[p][q];
}

/* dJ/df(t) = Re(conj(Fbar) exp(i w t)) for the components of one kind. */
static void inject(oracle_t *o, int magnetic, double t) {
    for (int s = 0; s < o->nmon; ++s) {
        omon_t *m = &o->mon[s];
        if (!m->cot) continue;
        for (int ci = 0; ci < m->ncomp; ++ci) {
            int comp = m->comps[ci];
            if ((comp >= 3) != magnetic) continue;
            for (int f = 0; f < m->nf; ++f) {
                double cr = cos(m->omega[f] * t), si = sin(m->omega[f] * t);
                const double *cot = m->cot + 2L * ((long)ci * m->nf + f) * m->ncell;
                for (long c = 0; c < m->ncell; ++c) {
                    int i, j, k; mon_cell(m, c, &i, &j, &k);
                    o->A[comp][IDX(o, i, j, k)] += cot[2 * c] * cr + cot[2 * c + 1] * si;
                }
            }
        }
    }
}

/* Adjoint of forward step m (u^m -> u^{m+1}).  The forward state held by the
 * oracle must be u^m: it is read only for the material cotangent. */
void oracle_adjoint_step(oracle_t *o, long m) {
    const int nx = o->N[0], ny = o->N[1], nz = o->N[2];
    /* Forward values of step m needed by the material cotangent: pre-source
     * E^{m+1} and the curl, recomputed from u^m without touching the state. */
    if (o->design_on || o->npole > 0) {
        double *Pt[3][MAXP], *Qt[3][MAXP], *pst[3][2];
        for (int a = 0; a < 3; ++a) {
            for (int p = 0; p < o->npole; ++p) { Pt[a][p] = zalloc(o->ncell); Qt[a][p] = zalloc(o->ncell); }
            pst[a][0] = zalloc(o->ncell); pst[a][1] = zalloc(o->ncell);
        }
        e_phase(o, o->tmpE, pst, Pt, Qt);
        for (int a = 0; a < 3; ++a) {
            for (int p = 0; p < o->npole; ++p) { free(Pt[a][p]); free(Qt[a][p]); }
            free(pst[a][0]); free(pst[a][1]);
        }
    }
    /* reverse of: DFT-H at t = m + 3/2 */
    inject(o, 1, (double)m + 1.5);
    /* reverse of the H-phase: H_a -= S (y1 - y2), psi = b psi + c d, y = d/kappa + psi */
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, cax = (a + 2) % 3;
        double *Ac = o->A[cax], *Ab = o->A[b];
        const double *Ha = o->A[3 + a];
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    int c[3] = {i, j, k};
                    long id = IDX(o, i, j, k);
                    int pb = c[b], pc = c[cax];
                    double yb1 = -o->S * Ha[id];
                    double yb2 = o->S * Ha[id];
                    double pm1 = o->apsiH[a][0][id] + yb1;
                    double pm2 = o->apsiH[a][1][id] + yb2;
                    double db1 = o->hk[b][pb] * yb1 + o->hc[b][pb] * pm1;
                    double db2 = o->hk[cax][pc] * yb2 + o->hc[cax][pc] * pm2;
                    o->apsiH[a][0][id] = o->hb[b][pb] * pm1;
                    o->apsiH[a][1][id] = o->hb[cax][pc] * pm2;
                    int cb[3] = {i, j, k}; cb[b] += 1;
                    int cc[3] = {i, j, k}; cc[cax] += 1;
                    add_at(o, Ac, cb[0], cb[1], cb[2], db1);
                    Ac[id] -= db1;
                    add_at(o, Ab, cc[0], cc[1], cc[2], db2);
                    Ab[id] -= db2;
                }
    }
    /* reverse of: DFT-E at t = m + 1 */
    inject(o, 0, (double)(m + 1));
    if (o->tensor_on) {
        /* E^{m+1} = E^m + S S_t C: Cbar = S S_t^T Ebar = S S_t Ebar (S_t is symmetric), and
         * d/d eps^-1_n[u][v] of Ebar^T S S_t C is S/8 sum_c (R_c D^-1/2 Ebar)_u (R_c D^-1/2 C)_v,
         * summed over [u][v] and [v][u] for an off-diagonal component */
        tensor_apply(o, o->A, o->tscr);
        if (o->design_on)
            for (int k = o->dlo[2]; k < o->dhi[2]; ++k)
                for (int j = o->dlo[1]; j < o->dhi[1]; ++j)
                    for (int i = o->dlo[0]; i < o->dhi[0]; ++i) {
                        long did = ((long)(k - o->dlo[2]) * (o->dhi[1] - o->dlo[1]) + (j - o->dlo[1])) *
                                       (o->dhi[0] - o->dlo[0]) + (i - o->dlo[0]);
                        for (int c = 0; c < 8; ++c) {
                            long id[3];
                            node_edges(o, i, j, k, c, id);
                            double wb[3], wc[3];
                            for (int a = 0; a < 3; ++a) {
                                double r = id[a] >= 0 ? 1.0 / sqrt(o->tD[a][id[a]]) : 0.0;
                                wb[a] = id[a] >= 0 ? r * o->A[a][id[a]] : 0.0;
                                wc[a] = id[a] >= 0 ? r * o->curl[a][id[a]] : 0.0;
                            }
                            for (int u = 0; u < 3; ++u)
                                for (int v = u; v < 3; ++v) {
                                    double t = u == v ? wb[u] * wc[u] : wb[u] * wc[v] + wb[v] * wc[u];
                                    o->grad[tcomp(u, v)][did] += o->S * t / 8.0;
                                }
                        }
                    }
    }
    /* reverse of the E-phase */
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, cax = (a + 2) % 3;
        double *Hc = o->A[3 + cax], *Hb = o->A[3 + b];
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    int c[3] = {i, j, k};
                    long id = IDX(o, i, j, k);
                    if (is_pec_E(o, a, c)) { o->A[a][id] = 0.0; continue; }
                    double Etb = o->A[a][id];        /* cotangent of pre-source E^{m+1} */
                    double Eold_b = 0.0, curl_b;
                    int indesign = o->design_on && i >= o->dlo[0] && i < o->dhi[0] && j >= o->dlo[1] &&
                                   j < o->dhi[1] && k >= o->dlo[2] && k < o->dhi[2];
                    long did = indesign ? ((long)(k - o->dlo[2]) * (o->dhi[1] - o->dlo[1]) + (j - o->dlo[1])) *
                                              (o->dhi[0] - o->dlo[0]) + (i - o->dlo[0]) : 0;
                    if (o->npole > 0 && o->mask[id]) {
                        double eps = 1.0 / o->inv_eps[a][id];
                        double G = 0.0;
                        for (int p = 0; p < o->npole; ++p) G += o->g[p][0];
                        double den = eps + G;
                        /* pole-parameter cotangents: Et depends on M00, M01 and g0 (through
                         * num and den), x^{m+1} on all six coefficients; Etot is the total
                         * cotangent of Et (its own plus the path through x^{m+1}) */
                        {
                            double Etot = Etb;
                            for (int p = 0; p < o->npole; ++p)
                                Etot += o->g[p][0] * o->aP[a][p][id] + o->g[p][1] * o->aQ[a][p][id];
                            double Eold = o->F[a][id], Et = o->tmpE[a][id], es = Et + Eold;
                            for (int p = 0; p < o->npole; ++p) {
                                double Pp = o->P[a][p][id], Qp = o->Q[a][p][id];
                                double xbP = o->aP[a][p][id], xbQ = o->aQ[a][p][id];
                                o->pgc[p][0] += xbP * Pp - Etot * Pp / den;
                                o->pgc[p][1] += xbP * Qp - Etot * Qp / den;
                                o->pgc[p][2] += xbQ * Pp;
                                o->pgc[p][3] += xbQ * Qp;
                                o->pgc[p][4] += xbP * es - Etot * es / den;
                                o->pgc[p][5] += xbQ * es;
                            }
                        }
                        /* x_p^{m+1} = M_p x_p^m + g_p (Et + E^m) */
                        for (int p = 0; p < o->npole; ++p) {
                            double xbP = o->aP[a][p][id], xbQ = o->aQ[a][p][id];
                            double gx = o->g[p][0] * xbP + o->g[p][1] * xbQ;
                            Etb += gx;
                            Eold_b += gx;
                            o->aP[a][p][id] = o->M[p][0][0] * xbP + o->M[p][1][0] * xbQ;
                            o->aQ[a][p][id] = o->M[p][0][1] * xbP + o->M[p][1][1] * xbQ;
                        }
                        /* Et = (eps E + sum_p (P - (M x)_P - g_P E) + S curl) / (eps + G) */
                        Eold_b += Etb * (eps - G) / den;
                        for (int p = 0; p < o->npole; ++p) {
                            o->aP[a][p][id] += Etb * (1.0 - o->M[p][0][0]) / den;
                            o->aQ[a][p][id] += Etb * (-o->M[p][0][1]) / den;
                        }
                        curl_b = Etb * o->S / den;
                        if (indesign) {
                            double Eold = o->F[a][id], Et = o->tmpE[a][id];
                            double eps_b = Etb * (Eold - Et) / den;
                            o->grad[a][did] += -eps * eps * eps_b;
                        }
                    } else if (o->tensor_on) {
                        Eold_b = Etb;
                        curl_b = o->S * o->tscr[a][id];
                    } else {
                        /* Et = E + S inv_eps curl */
                        Eold_b = Etb;
                        curl_b = Etb * o->S * o->inv_eps[a][id];
                        if (indesign) o->grad[a][did] += Etb * o->S * o->curl[a][id];
                    }
                    /* curl = y1 - y2 ; psi = b psi + c d ; y = d/kappa + psi */
                    int pb = c[b], pc = c[cax];
                    double yb1 = curl_b, yb2 = -curl_b;
                    double pm1 = o->apsiE[a][0][id] + yb1;
                    double pm2 = o->apsiE[a][1][id] + yb2;
                    double db1 = o->ek[b][pb] * yb1 + o->ec[b][pb] * pm1;
                    double db2 = o->ek[cax][pc] * yb2 + o->ec[cax][pc] * pm2;
                    o->apsiE[a][0][id] = o->eb[b][pb] * pm1;
                    o->apsiE[a][1][id] = o->eb[cax][pc] * pm2;
                    /* d1 = Hc(r) - Hc(r - e_b), d2 = Hb(r) - Hb(r - e_c) */
                    int cb[3] = {i, j, k}; cb[b] -= 1;
                    int cc[3] = {i, j, k}; cc[cax] -= 1;
                    Hc[id] += db1;
                    add_at(o, Hc, cb[0], cb[1], cb[2], -db1);
                    Hb[id] += db2;
                    add_at(o, Hb, cc[0], cc[1], cc[2], -db2);
                    o->A[a][id] = Eold_b;
                }
    }
}
