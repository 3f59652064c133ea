/*
 * gbfdtd — GB300-native differentiable FDTD hot path (C ABI).
 *
 * The method is the differentiable FDTD scheme of arxiv 2609.30039 (TorchFDTD):
 *   Sec. 2.1, Eq. (yee): E^{n+1} = E^n + S eps^{-1} C^-(H^{n+1/2}) + s^{n+1},
 *                        H^{n+3/2} = H^{n+1/2} - S C^+(E^{n+1}) + m^{n+3/2};
 *   Sec. 2.2: CPML memories per transverse derivative in absorbing faces, PEC faces;
 *   Sec. 2.3: permittivity per Yee E position (diagonal), up to 16 Drude/Lorentz poles
 *             integrated with the trapezoidal ADE, tensor admission rule inside a face;
 *   Sec. 2.4: soft point/sheet sources, running DFT monitors with the half-step phase;
 *   Sec. 3.1, Eq. (adjoint): transposed kernel of every update and the material
 *             cotangent d(objective)/d(eps^-1);
 *   Sec. 3.2: checkpoint snapshots for replay;
 *   Sec. 4.1: several independent structures advanced by one launch;
 *   Sec. 4.2: host-streamed slabs (state in host memory, stepped slab by slab with halos).
 *
 * Conventions (all entry points):
 *   - Reduced units: lengths in cells, c = eps0 = mu0 = 1; only the Courant number
 *     S = c dt / dx enters the update.  Arrays of cells are (nz, ny, nx) with x fastest:
 *     idx = (k*ny + j)*nx + i.  Yee positions: Ex(i+1/2,j,k), Ey(i,j+1/2,k), Ez(i,j,k+1/2),
 *     Hx(i,j+1/2,k+1/2), Hy(i+1/2,j,k+1/2), Hz(i+1/2,j+1/2,k).  The outer boundary of
 *     every domain is PEC: tangential E on the planes of coordinate 0 is held at zero and
 *     nodes at coordinate N do not exist.
 *   - Component ids: 0..2 = Ex, Ey, Ez; 3..5 = Hx, Hy, Hz.
 *   - Every function returns an fdtd_status; nothing throws across the ABI.  On error the
 *     context keeps a message (fdtd_last_error).  After FDTD_ECUDA the context is poisoned:
 *     every later call except fdtd_destroy / fdtd_last_error returns FDTD_ESTATE.  No kernel of
 *     the library spins on a flag of another block or kernel; the only device-side wait is the
 *     griddepcontrol wait of the programmatically launched transposed kernels, which the hardware
 *     ends when the kernels launched before them on the stream complete, so none can run out.
 *   - All device work is enqueued on the stream given to fdtd_create (a cudaStream_t passed
 *     as void*; NULL = legacy default stream).  Calls are asynchronous unless stated.
 *     A context is not thread-safe.
 *   - "device" pointers are CUDA global memory; "borrowed" means the caller keeps it alive
 *     for as long as the context may use it; "copied" means the library copies it before
 *     returning.
 *   - Time indexing: fields start at zero (step count 0).  Forward step n (n = 0, 1, ...)
 *     maps u^n -> u^{n+1}; its electric samples belong to time (n+1) dt and its magnetic
 *     samples to (n+3/2) dt (Sec. 2.1).
 */
#ifndef GBFDTD_FDTD_H
#define GBFDTD_FDTD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FDTD_OK = 0,
    FDTD_EINVAL = 1,     /* bad argument (sizes, ids, boxes, NULL pointers) */
    FDTD_ECFL = 2,       /* Courant number violates Eq. (cfl): S sqrt(3) > 0.99 */
    FDTD_ETENSOR = 3,    /* a CPML cell holds a permittivity rejected by the Sec. 2.3 admission rule */
    FDTD_ENOMEM = 4,     /* the memory plan exceeds free device memory (nothing allocated) */
    FDTD_ECUDA = 5,      /* a CUDA call failed; the context is poisoned */
    FDTD_ESTATE = 6,     /* call not valid in the current state (see each function) */
    FDTD_ENONFINITE = 7, /* NaN/Inf found by fdtd_check_finite */
    FDTD_ETIMEOUT = 8    /* a bounded host wait ran out (fdtd_synchronize) */
} fdtd_status;

enum { FDTD_F32 = 0, FDTD_F64 = 1 };          /* storage and arithmetic type of fields */
enum { FDTD_LORENTZ = 0, FDTD_DRUDE = 1 };
enum { FDTD_CODEC_NATIVE = 0, FDTD_CODEC_BF16 = 1 };   /* snapshot codecs */

typedef struct fdtd_ctx fdtd_ctx;

/* One domain's grid (Sec. 2.1).  dx > 0 and dt only serve the consistency check
 * dt == courant * dx (dt = 0: derived).  All domains of a context share courant and dtype. */
typedef struct {
    int32_t nx, ny, nz;   /* cells per axis, each >= 2 */
    double dx;
    double courant;       /* S; Eq. (cfl): 0 < S <= 0.99 / sqrt(3) */
    double dt;
    int32_t dtype;        /* FDTD_F32 | FDTD_F64 */
} fdtd_grid;

/* CPML of one domain (Sec. 2.2, Roden-Gedney).  cells[f] = depth d of face f in
 * (-x,+x,-y,+y,-z,+z); 0 = bare PEC face.  At depth rho (cells, measured at the node of the
 * derivative: integer for E updates, half-integer for H updates):
 *   sigma = sigma_max (rho/d)^m, kappa = 1 + (kappa_max - 1)(rho/d)^m, alpha = alpha_max (1 - rho/d),
 *   b = exp(-(sigma/kappa + alpha) S), c = sigma (b - 1)/(sigma kappa + kappa^2 alpha) (0 if sigma = 0);
 *   psi <- b psi + c D,  y = D / kappa + psi.  sigma_max < 0 selects 0.8 (m + 1). */
typedef struct {
    int32_t cells[6];
    double m, kappa_max, alpha_max, sigma_max;
} fdtd_cpml;

/* One pole (Sec. 2.3).  Per step: dP/dt = Q, dQ/dt = -gamma Q - a0 P + b1 E with
 * Lorentz a0 = omega^2, b1 = delta_eps omega^2; Drude a0 = 0, b1 = omega^2 (omega = wp dt). */
typedef struct {
    int32_t kind;         /* FDTD_LORENTZ | FDTD_DRUDE */
    double delta_eps;     /* Lorentz strength (unused for Drude) */
    double omega_dt;      /* rad/step */
    double gamma_dt;      /* damping per step, >= 0 */
} fdtd_pole;

/* Materials of one domain (Sec. 2.3).  inv_eps[a]: device, borrowed, dtype of the grid,
 * nz*ny*nx values of 1/eps (1/eps_inf in dispersive cells) at the Yee position of E_a; the
 * same pointer three times declares an isotropic medium.  Values must be > 0.
 * pole_mask: device, borrowed, nz*ny*nx bytes, nonzero = this domain's poles act on all three
 * E components of the cell; NULL = no dispersion.  poles: host, copied, n_poles <= 16. */
typedef struct {
    const void* inv_eps[3];
    int32_t n_poles;
    const fdtd_pole* poles;
    const uint8_t* pole_mask;
} fdtd_material;

/* Creates a context owning all internal device state (fields, CPML memories, pole states,
 * adjoint state, monitors, snapshots) for n_domains independent domains (Sec. 4.1); arrays
 * grids/cpml/materials have n_domains entries.  Checks Eq. (cfl) (FDTD_ECFL), the tensor
 * admission rule in every CPML cell (FDTD_ETENSOR: with a diagonal tensor the face normal is
 * a principal axis; the normal eigenvalue must not lie strictly between the other two), and
 * the memory plan against cudaMemGetInfo before allocating (FDTD_ENOMEM).  Grid limits
 * (FDTD_EINVAL): 2 <= nx, ny <= 65535, nz >= 2, fewer than 2^40 cells, fewer than 2^31 cells per
 * z-plane and per CPML memory array (slab depth times the two other extents).  Synchronises the
 * stream.  *out is set only on FDTD_OK. */
fdtd_status fdtd_create(int32_t n_domains, const fdtd_grid* grids, const fdtd_cpml* cpml,
                        const fdtd_material* materials, void* stream, fdtd_ctx** out);

/* Creates a host-streamed context of one domain (Sec. 4.2).  The fields, CPML memories and pole
 * states live in pinned host memory owned by the context; material->inv_eps[a] and
 * material->pole_mask must be pinned host memory (cudaHostAlloc / cudaHostRegister; borrowed,
 * same layout as in fdtd_create).  The domain is cut along z (the slowest axis) into slabs of
 * `slab` owned planes.  fdtd_step_forward advances in batches of at most `halo` steps: each slab's
 * window (its planes plus up to `halo` planes on each side) is copied into one of three device
 * workspaces, stepped by the per-cell kernels, and its owned planes are copied back, with the
 * copies of neighbouring slabs overlapping the stepping on two copy streams.  The owned planes then
 * hold exactly the values that a resident context (fdtd_create) computes, bit for bit.  The device
 * holds the three windows of min(nz, slab + 2 halo) planes plus the monitors, not the domain.
 * Requires 1 <= halo <= slab (FDTD_EINVAL).  Supported on a streamed context: stepping, sources,
 * DFT monitors and flux, periodic x / y, materials (pinned host), get/set of state parts (the copy
 * may involve device or host memory), reset, step counters, fdtd_check_finite, and the streamed
 * transposed sweep (fdtd_stream_checkpoints, then fdtd_adjoint_begin / fdtd_step_adjoint with
 * adjoint sources and a design box as on a resident context).  Not supported (FDTD_EINVAL):
 * snapshots, energy records, the backward step, pole-parameter gradients, autotuning, profiling,
 * and launch modes other than 4. */
fdtd_status fdtd_create_streamed(const fdtd_grid* grid, const fdtd_cpml* cpml, const fdtd_material* material,
                                 int32_t slab, int32_t halo, void* stream, fdtd_ctx** out);

/* Forward checkpoints of a host-streamed context (Sec. 4.2; the transposed sweep runs the slab
 * tiling in reverse).  enabled = 1: from the held step t0 on, fdtd_step_forward runs its batches
 * aligned to t0 + j * halo and keeps the whole forward state at every such batch start in pinned
 * host memory owned by the context (existing checkpoints are dropped, their buffers reused); each
 * batch writes the next checkpoint with the copies of its owned planes.  enabled = 0 stops taking
 * checkpoints and frees every checkpoint buffer; enabled = 2 stops taking them but keeps the
 * buffers for the next enabled = 1 (a gradient loop then pins its host memory once); other values:
 * FDTD_EINVAL.  fdtd_destroy frees them in any case.  The
 * transposed sweep of a streamed context -- fdtd_adjoint_begin, then fdtd_step_adjoint -- then runs
 * the batches last to first: per slab its window replays the batch from the checkpoint on the device
 * (keeping each replayed window state, kb <= halo of them), takes the transposed steps from the
 * adjoint state at the batch end (monitor cotangents injected over the whole window), completes them
 * and writes its owned planes back; only owned design cells add to the material cotangent.  The
 * owned planes then hold what the resident sweep computes (bit for bit in the adjoint state; the
 * material cotangent to rounding order, each window summing its own steps first).  The adjoint
 * state lives in two pinned host sets owned by the context (parts with which = 1 read the current
 * one, always in natural form); fdtd_step_adjoint takes whole batches (FDTD_ESTATE otherwise).
 * Device memory of the sweep: the adjoint window and halo replayed forward windows (fields and pole
 * states of min(nz, slab + 2 halo) planes) besides the three stepping workspaces.  FDTD_EINVAL on a
 * resident context. */
fdtd_status fdtd_stream_checkpoints(fdtd_ctx* ctx, int32_t enabled);

/* Frees everything the context owns.  NULL-safe.  Synchronises the stream. */
fdtd_status fdtd_destroy(fdtd_ctx* ctx);

/* Message of the last error on this context ("" if none); static text when ctx == NULL. */
const char* fdtd_last_error(const fdtd_ctx* ctx);

/* Library version string (static). */
const char* fdtd_version(void);

/* Rebinds domain `domain`'s material (same rules as in fdtd_create; the pole count and the
 * set of dispersive cells must not grow beyond the box chosen at create: FDTD_EINVAL). */
fdtd_status fdtd_set_material(fdtd_ctx* ctx, int32_t domain, const fdtd_material* material);

/* Net Poynting flux along +z (Sec. 2.4: plane monitors form the signed Poynting flux from
 * Yee-interpolated spectra) through the plane z = k + 1/2 of a monitor spanning the two z-planes
 * [k, k+2): P(w) = 1/2 Re sum over the monitor's x-y cells of
 *   (Ex(k) + Ex(k+1))/2 conj(Hy(k)) - (Ey(k) + Ey(k+1))/2 conj(Hx(k)),
 * which puts each product at one Yee point (Hy and Hx live on z = k + 1/2).  Spectra carry
 * their own sample times (E: t = n+1, H: t = n+3/2), so the magnetic half step is already in
 * their phases.  The monitor must record Ex, Ey, Hx and Hy (FDTD_EINVAL otherwise).
 * flux_host: n_freq doubles (host); n_freq must equal the monitor's frequency count (FDTD_EINVAL
 * otherwise, nothing written).  Synchronises. */
fdtd_status fdtd_dft_flux(fdtd_ctx* ctx, int32_t monitor, double* flux_host, int32_t n_freq);

/* Periodic boundaries (Sec. 2.2: periodic/Bloch lateral boundaries, here with zero Bloch
 * phase) on the x and/or y axis of one domain: the neighbour beyond the last node is the first
 * one and vice versa, and the coordinate-0 plane of that axis is no PEC wall.  periodic[3] are
 * flags for x, y, z; z must be 0, and a periodic axis must have no CPML cells on either face and
 * at least 2 cells (FDTD_EINVAL otherwise).  Applies to the forward and transposed steps in every
 * launch mode. */
fdtd_status fdtd_set_periodic(fdtd_ctx* ctx, int32_t domain, const int32_t periodic[3]);

/* Bloch-periodic faces (Sec. 2.2: periodic pairs with a fixed Bloch phase; Sec. 3.1: transposed
 * with conjugate seam factors).  phase[q] = k_q N_q (radians) for the x and y axes: a field continued
 * across the seam of axis q picks up p_q = exp(i phase[q]), f(x + N_q) = p_q f(x), so the E update's
 * backward differences read f(-1) = conj(p) f(N - 1) and the H update's forward differences
 * f(N) = p f(0).  The domain's fields become complex: the field parts 0..5 hold the real parts and
 * six more parts (ids 18 + 6 n_poles + c, c = 0..5, i.e. 18..23) the imaginary parts, forward
 * (which = 0) and adjoint (which = 1; the adjoint is taken under <u, v> = sum conj(u) v).  A nonzero
 * phase needs that axis periodic (fdtd_set_periodic first).  Scope: the domain has no CPML slabs
 * (PEC z faces), no poles, no DFT monitor and no design box; soft sources add their (real) waveform
 * to the real part; the context steps in launch mode 4 without an energy record, and autotuning, the
 * backward step and kernel timing are not available.  FDTD_EINVAL otherwise.  The first call on a
 * domain allocates the imaginary parts (zero) and frees every snapshot slot; later calls only
 * change the phases.  Forward and transposed steps then run the Bloch kernels for this domain. */
fdtd_status fdtd_set_bloch(fdtd_ctx* ctx, int32_t domain, const double phase[2]);

/* Symmetric permittivity tensors at the grid nodes (Sec. 2.3).  inv_eps[6]: the components xx, yy,
 * zz, xy, xz, yz of eps^-1 at every node (node (i, j, k) at offset (k ny + j) nx + i, the context's
 * dtype; device or host memory, copied into memory the context owns).  The domain's E update then
 * applies the node assembly S_t = D^{-1/2} (1/8 sum_n sum_c R_{n,c}^T eps^-1_n R_{n,c}) D^{-1/2} to
 * the CPML-corrected curl, E += S S_t curl, where R_{n,c} picks one E edge per axis next to node n
 * (the q-edge of coordinate n_q - 1 + c_q, for the 2^3 choices c) and D is the same sum with the
 * identity tensor (1 on an edge with two end nodes, 1/2 on one whose upper node lies beyond a
 * non-periodic high face); the diagonal eps^-1 of fdtd_create is no longer read.  The transposed
 * steps apply S_t to Ebar (it is symmetric), and a design box (fdtd_set_design) then collects
 * d J / d eps^-1 of its nodes, six components per node.  Admission rule (FDTD_ETENSOR, the domain is
 * then left without tensors): every node positive definite with each eigenvalue of eps at least one
 * (relative tolerance 1e-6), and at a node inside the CPML slab of an axis q, e_q is a principal axis
 * (eps^-1_qb = eps^-1_qc = 0 up to 1e-6 of the largest diagonal entry) whose eigenvalue is not
 * strictly between the two others.  Scope: no poles, no Bloch phase, no energy record, no interface
 * record, resident contexts (FDTD_EINVAL otherwise); the context switches to launch mode 4, and
 * other launch modes, autotuning, the backward step and kernel timing are refused while a domain
 * holds tensors.  inv_eps = NULL returns the domain to its diagonal eps^-1.  Every call removes the
 * domain's design box (its gradient buffer has the other layout): set the box afterwards. */
fdtd_status fdtd_set_tensor(fdtd_ctx* ctx, int32_t domain, const void* const inv_eps[6]);

/* Soft source (Sec. 2.4, Eq. (yee) s and m): after the update of `component` in forward
 * step n, every cell of the half-open box [lo, hi) gets += waveform[n] (no effect for
 * n >= n_steps).  waveform: host, copied, FP64.  *source_id may be NULL.  An electric source
 * box may not hold PEC-held nodes (coordinate 0 of a non-periodic axis other than the
 * component's own: FDTD_EINVAL), so mark periodic axes before adding a source on their seam. */
fdtd_status fdtd_add_source(fdtd_ctx* ctx, int32_t domain, int32_t component, const int32_t lo[3],
                            const int32_t hi[3], const double* waveform, int32_t n_steps,
                            int32_t* source_id);

/* Running DFT monitor over the half-open box [lo, hi) (a plane, a patch or a point; Sec. 2.4):
 * F_c(f, cell) += field_c(cell) * exp(+i omega_dt[f] t) with t = n+1 for E components and
 * t = n+3/2 for H components in forward step n.  Accumulators are complex FP64, layout
 * [ncomp][n_freq][box cells (x fastest)], components in increasing id among component_mask
 * (bit c = component c).  omega_dt: host, copied.  *monitor_id receives the id.
 * In launch mode 4 without an energy record, a resident context whose monitors sit at most one per
 * domain (and in no tensor domain) keeps a device ring of one batch (32 steps) of samples per
 * monitor (32 * ncomp * box cells field values, at most 512 MiB for all monitors): the update
 * kernels store the samples and one launch per batch adds them to the accumulators in step order,
 * bit for bit the values per-step accumulation gives.  Otherwise (or when a ring does not fit in
 * device memory) the DFT runs per half-step. */
fdtd_status fdtd_add_dft_monitor(fdtd_ctx* ctx, int32_t domain, const int32_t lo[3], const int32_t hi[3],
                                 uint32_t component_mask, int32_t n_freq, const double* omega_dt,
                                 int32_t* monitor_id);

/* Number of complex FP64 values of a monitor (ncomp * n_freq * box cells). */
fdtd_status fdtd_dft_size(fdtd_ctx* ctx, int32_t monitor_id, int64_t* n_complex);

/* Copies a monitor's accumulators (interleaved re, im doubles) to dst (bytes >= 16 * size).
 * dst_on_device = 0: host memory, the call synchronises the stream. */
fdtd_status fdtd_dft_read(fdtd_ctx* ctx, int32_t monitor_id, void* dst, size_t bytes, int32_t dst_on_device);

/* Zeroes every DFT accumulator. */
fdtd_status fdtd_dft_reset(fdtd_ctx* ctx);

/* enabled = 0 freezes every DFT accumulator during fdtd_step_forward (used while replaying
 * forward segments of the adjoint, Sec. 3.2); 1 (default) accumulates. */
fdtd_status fdtd_dft_enable(fdtd_ctx* ctx, int32_t enabled);

/* Records the discrete energy W_{n+1} = 1/2 sum eps |E^{n+1}|^2 + 1/2 sum H^{n+1/2} . H^{n+3/2}
 * of every domain at every forward step n < capacity (FP64, per domain). */
fdtd_status fdtd_enable_energy(fdtd_ctx* ctx, int32_t capacity);

/* Copies n per-step energies of one domain to host memory (synchronises). */
fdtd_status fdtd_energy_read(fdtd_ctx* ctx, int32_t domain, double* host_dst, int32_t n);

/* Advances every domain by n_steps forward steps (Eq. (yee): E update with CPML, poles and
 * eps^-1; E sources; E DFT; H update with CPML; H sources; H DFT; energy).  Asynchronous.
 * How the steps are launched is set by fdtd_set_launch_mode (default: per-cell kernels replayed
 * as CUDA graphs of 32 steps). */
fdtd_status fdtd_step_forward(fdtd_ctx* ctx, int32_t n_steps);

/* Reversible reconstruction (Sec. 3.2: for lossless nondispersive problems the forward fields
 * are rebuilt by stepping Eq. (yee) backward instead of replaying from checkpoints): undoes the
 * last n_steps forward steps, each in reverse order,
 *   H^{n+1/2} = (H^{n+3/2} - m^n) + S curl E^{n+1},  E^n = (E^{n+1} - s^n) - S eps^-1 curl H^{n+1/2}.
 * Domains must have no poles (FDTD_EINVAL).  A domain without CPML faces steps back whole.  A
 * domain with CPML faces (the absorbing-face variant of Sec. 3.2) steps back its interior only --
 * the cells whose own node lies in no CPML slab, whose updates use no memory variable -- with the
 * fields at the interface between interior and absorber taken from the record of the forward run
 * (fdtd_record_interface, which must cover these steps: FDTD_ESTATE otherwise); its absorber cells
 * are left holding the recorded interface planes and otherwise whatever they held.  Launch mode 4
 * only.  FDTD_ESTATE when n_steps exceeds the held step count.  DFT accumulators and energies are
 * not touched; the step count decreases by n_steps.  In floating point the reconstruction differs
 * from the forward states by accumulated rounding.  Asynchronous. */
fdtd_status fdtd_step_backward(fdtd_ctx* ctx, int32_t n_steps);

/* Interface record of the absorbing-face reversible reconstruction (Sec. 3.2: the fields at the
 * interface between interior and absorber are recorded so that the interior reconstruction stays
 * lossless).  For every domain with CPML faces: allocates a device record of capacity + 1 slots
 * (each slot: the three H components on the plane just below each low CPML face of the interior
 * and the three E components on the plane just above each high one, full planes) and records the
 * held state as slot 0; every later forward step n (up to t0 + capacity - 1, t0 = the step count
 * now) records E^{n+1} and H^{n+3/2} into slot n + 1 - t0 (the record is captured into the
 * forward graphs).  capacity = 0 frees the records.  Launch mode 4 without an energy record
 * (FDTD_EINVAL otherwise); FDTD_ENOMEM if the record does not fit. */
fdtd_status fdtd_record_interface(fdtd_ctx* ctx, int32_t capacity);

/* Launch modes (no counterpart in the paper; they change scheduling, not arithmetic):
 * mode 0: per-half-step launches over one tile work list of every domain (interior and shell
 * tiles on two streams), replayed as CUDA graphs; the path of the energy record.
 * Mode 4 (default): per-half-step launches (CUDA graphs) of per-cell kernels, one thread per cell;
 * with several domains one launch per half-step covers every cell of every domain (with an energy
 * record it runs the mode-0 code).  Both compute the same values bitwise.
 * Modes 1-3 (persistent multi-step kernels with grid barriers) are not available: FDTD_EINVAL,
 * as for any other value. */
#define FDTD_LAUNCH_MODES 5
fdtd_status fdtd_set_launch_mode(fdtd_ctx* ctx, int32_t mode);
fdtd_status fdtd_get_launch_mode(fdtd_ctx* ctx, int32_t* mode);

/* Autotuner (no counterpart in the paper): times launch modes 0 and 4 for n_steps forward steps
 * on the current state, with DFT recording as configured and energy recording off, and keeps the
 * faster.  The state, step count, DFT accumulators and energies are left as they were (state
 * and accumulators are copied aside and restored after every trial).  ms_per_mode
 * (FDTD_LAUNCH_MODES entries indexed by mode, may be NULL) receives the measured milliseconds
 * of modes 0 and 4 and -1 for the others.  Needs device
 * memory for one native snapshot plus the accumulators (FDTD_ENOMEM otherwise).  Synchronises
 * the stream. */
fdtd_status fdtd_autotune(fdtd_ctx* ctx, int32_t n_steps, double* ms_per_mode);

/* Number of forward steps the held state has taken (u^n: returns n). */
fdtd_status fdtd_step_count(fdtd_ctx* ctx, int64_t* n);

/* Zeroes the forward state (fields, CPML memories, pole states) and sets the step count to 0.
 * DFT accumulators and energies are left alone (see fdtd_dft_reset). */
fdtd_status fdtd_reset(fdtd_ctx* ctx);

/* ---- state access (tests, checkpoints held by the caller) ----
 * A domain's state is a list of parts:
 *   part 0..5            field Ex..Hz, nz*ny*nx values;
 *   part 6 + 2a + s      E CPML memory psi of E_a for its s-th curl derivative
 *                        (s = 0: along axis (a+1)%3, s = 1: along (a+2)%3);
 *   part 12 + 2a + s     the same for H_a;
 *   part 18 + 2(a*P + p) + w   pole state (w = 0: P, 1: Q) of pole p for E_a (P = n_poles).
 * A CPML part of axis q holds the cells whose q-coordinate lies in [0, d_lo) U [N_q - d_hi, N_q)
 * (the slabs of the two q faces), in (z, y, x) order with x fastest, the q extent replaced by
 * d_lo + d_hi; it is empty if the axis has no CPML.  A pole part holds the cells of the box
 * reported by fdtd_ade_box.  Values are in the dtype of the grid.
 * which = 0: forward state; which = 1: adjoint state in natural form (the cotangent of the
 * forward part of the same id; reading it completes any pending transposition first).
 * dst / src: device or pinned host memory of part_size values (copied on the context's stream). */
fdtd_status fdtd_part_count(fdtd_ctx* ctx, int32_t domain, int32_t* n_parts);
fdtd_status fdtd_part_size(fdtd_ctx* ctx, int32_t domain, int32_t part, int64_t* n_values);
fdtd_status fdtd_get_part(fdtd_ctx* ctx, int32_t domain, int32_t which, int32_t part, void* dst);
fdtd_status fdtd_set_part(fdtd_ctx* ctx, int32_t domain, int32_t which, int32_t part, const void* src);
/* Box [lo, hi) of the pole states of a domain (empty box if it has no dispersive cell). */
fdtd_status fdtd_ade_box(fdtd_ctx* ctx, int32_t domain, int32_t lo[3], int32_t hi[3]);
/* Sets the forward step count (after the caller wrote a state with fdtd_set_part). */
fdtd_status fdtd_set_step_count(fdtd_ctx* ctx, int64_t n);

/* ---- checkpoints (Sec. 3.2) ----
 * Saves the whole forward state of every domain and its step count into slot `slot` (device
 * memory owned by the context, allocated on first use of the slot; FDTD_ENOMEM if it does not
 * fit).  codec FDTD_CODEC_NATIVE copies values exactly; FDTD_CODEC_BF16 stores bf16(x / s)
 * with one FP32 scale s = max|x| per (part, outermost index) slab (a z-plane for field parts),
 * s = 0 for an all-zero slab.  restore dequantises into the live state. */
fdtd_status fdtd_state_save(fdtd_ctx* ctx, int32_t slot, int32_t codec);
fdtd_status fdtd_state_restore(fdtd_ctx* ctx, int32_t slot);
/* Native executor of a checkpoint-replay schedule (Sec. 3.2).  actions holds n_actions pairs
 * (kind, arg): FDTD_ACT_SAVE (fdtd_state_save of slot arg with `codec`), FDTD_ACT_RESTORE (slot
 * arg), FDTD_ACT_ADVANCE (arg forward steps), FDTD_ACT_ADJOINT (arg transposed steps),
 * FDTD_ACT_STOP (return, so that the caller evaluates its objective, registers adjoint sources and
 * calls fdtd_adjoint_begin before resuming after it).  *executed = actions consumed, the STOP
 * included.  Stops at the first failing action and returns its status (*executed counts the
 * actions before it).  Host memory: actions (read only). */
#define FDTD_ACT_SAVE 0
#define FDTD_ACT_RESTORE 1
#define FDTD_ACT_ADVANCE 2
#define FDTD_ACT_ADJOINT 3
#define FDTD_ACT_STOP 4
fdtd_status fdtd_run_schedule(fdtd_ctx* ctx, const int32_t* actions, int32_t n_actions, int32_t codec,
                              int32_t* executed);
/* Device bytes one snapshot of this context takes with a codec. */
fdtd_status fdtd_snapshot_bytes(fdtd_ctx* ctx, int32_t codec, int64_t* bytes);
/* Frees every snapshot slot. */
fdtd_status fdtd_snapshots_free(fdtd_ctx* ctx);

/* ---- discrete adjoint (Sec. 3.1, Eq. (adjoint)) ----
 * Design box of a domain: the material cotangent d J / d(eps^-1_a) of every cell of [lo, hi)
 * is accumulated (+=) into grad_device (FP64, borrowed, layout [3][box cells, x fastest]) by
 * every adjoint step.  In a tensor domain (fdtd_set_tensor) the box is one of nodes and the layout
 * [6][box nodes], components xx, yy, zz, xy, xz, yz (an off-diagonal component is one symmetric
 * parameter).  The box must lie outside the CPML slabs.  grad_device = NULL removes it. */
fdtd_status fdtd_set_design(fdtd_ctx* ctx, int32_t domain, const int32_t lo[3], const int32_t hi[3],
                            double* grad_device);

/* Pole-parameter gradients (Sec. 3.1: Drude and Lorentz pole parameters differentiate through the
 * transposed dispersion update).  enabled != 0: every later transposed step sums, over the domain's
 * dispersive cells and E components, the cotangents of each pole's trapezoidal coefficients
 * (M00, M01, M10, M11, g0, g1; FP64 device accumulator owned by the context, zeroed here and by
 * fdtd_adjoint_begin).  Needs poles and a pole-state box outside the CPML slabs (FDTD_EINVAL).
 * enabled = 0 stops collecting. */
fdtd_status fdtd_set_pole_grad(fdtd_ctx* ctx, int32_t domain, int32_t enabled);
/* d J / d(delta_eps, omega_dt, gamma_dt) of each pole of the domain, host_out[3 p + 0..2]
 * (n_poles * 3 doubles; a Drude pole's delta_eps entry is 0), from the coefficient cotangents
 * collected since fdtd_adjoint_begin and the exact derivatives of the coefficients' closed form.
 * Synchronises the stream.  FDTD_EINVAL if the domain does not collect them. */
fdtd_status fdtd_pole_grad(fdtd_ctx* ctx, int32_t domain, double* host_out);

/* Adjoint source of a monitor: cot_device (borrowed, complex FP64 interleaved, the monitor's
 * layout) holds dJ/dRe F + i dJ/dIm F.  The adjoint injects dJ/df(t) = Re(conj(cot) exp(i w t))
 * at the monitor cells.  NULL clears it. */
fdtd_status fdtd_set_adjoint_source(fdtd_ctx* ctx, int32_t monitor_id, const void* cot_device);

/* Starts an adjoint sweep at the current forward step count N: zeroes the adjoint state
 * (cotangent of u^N) and injects the magnetic samples of time N + 1/2. */
fdtd_status fdtd_adjoint_begin(fdtd_ctx* ctx);

/* Transposes n_steps forward steps, m = A-1, A-2, ... where A is the index of the current
 * adjoint state (N after fdtd_adjoint_begin).  When any design box is set, each transposed
 * step m needs the forward state u^m (for the material cotangent): then n_steps must be 1 and
 * the forward step count must equal m (FDTD_ESTATE otherwise); the caller re-creates u^m by
 * checkpoint replay.  Without a design box any n_steps <= A is allowed. */
fdtd_status fdtd_step_adjoint(fdtd_ctx* ctx, int32_t n_steps);

/* Index A of the current adjoint state (the cotangent held is that of u^A). */
fdtd_status fdtd_adjoint_step_count(fdtd_ctx* ctx, int64_t* a);

/* Replaces the adjoint state's step index (after the caller wrote a natural adjoint state
 * with fdtd_set_part, which = 1). */
fdtd_status fdtd_set_adjoint_step_count(fdtd_ctx* ctx, int64_t a);

/* ---- health ---- */
/* Scans the forward state of every domain for NaN/Inf; returns FDTD_ENONFINITE if any
 * (synchronises). */
fdtd_status fdtd_check_finite(fdtd_ctx* ctx);

/* Synchronises the context's stream, polling at most timeout_ms milliseconds
 * (FDTD_ETIMEOUT if the work has not finished by then; the work itself is not cancelled, and the
 * context stays usable).  A CUDA error reported by the stream poisons the context (FDTD_ECUDA). */
fdtd_status fdtd_synchronize(fdtd_ctx* ctx, int32_t timeout_ms);

/* Number of kernel launches this context has enqueued since creation (instrumentation). */
fdtd_status fdtd_launch_count(fdtd_ctx* ctx, int64_t* n);

/* ---- allocation-free health check (no counterpart in the paper) ----
 * Counts the NaN / Inf values among n values of one device array (dtype FDTD_F32 | FDTD_F64,
 * e.g. a state part read with fdtd_get_part) into *count (host).  Unlike fdtd_check_finite it
 * needs no context and allocates nothing: it is for callers that cannot call cudaMalloc, such
 * as code whose device memory is owned by a framework's caching allocator or a fixed budget,
 * where an extra allocation may fail or (cudaMalloc synchronises the device) stall other work.
 * Its scratch is a file-scope device array of 2048 per-block counts plus one total (16 KiB),
 * which every GPU that loads the library holds until the process exits.  Limit: n <= 33554432
 * values (2048 blocks x 256 threads x 64 values); larger n returns FDTD_EINVAL before any GPU
 * work.  Every call looks up that array's device address on the current device
 * (cudaGetSymbolAddress), so the address stays right after the device's context was reset; the
 * first call on a device also loads the library's device code there and should come before any
 * stream capture on that device.  Work is
 * enqueued on `stream` (NULL = legacy default stream) and the call synchronises it.  All calls
 * share the one scratch array and every call rewrites the slots it reads, so consecutive calls
 * are independent, but calls that overlap on the GPU (different streams or threads at once)
 * race and may return wrong counts.  Errors: FDTD_EINVAL (NULL count, negative or too large n,
 * bad dtype, NULL data with n > 0), FDTD_ECUDA (a CUDA call failed). */
fdtd_status fdtd_count_nonfinite_noalloc(const void* data_device, int64_t n, int32_t dtype, void* stream,
                                         int64_t* count);

/* ---- instrumentation: per-kernel device time with CUDA events on the context's stream ----
 * Kernel classes: */
enum {
    FDTD_KERNEL_E = 0,        /* E update (Eq. (yee) first half, CPML, poles) */
    FDTD_KERNEL_H = 1,        /* H update (second half, CPML, energy) */
    FDTD_KERNEL_SOURCE = 2,   /* soft sources */
    FDTD_KERNEL_DFT = 3,      /* running DFT monitors */
    FDTD_KERNEL_STEP = 4,     /* device step counter */
    FDTD_KERNEL_ADJ_E = 5,    /* transposed step, E side */
    FDTD_KERNEL_ADJ_H = 6,    /* transposed step, H side */
    FDTD_KERNEL_CLASSES = 8   /* (class 7 is unused) */
};
/* Starts recording an event pair around every kernel launch (at most max_launches launches,
 * later ones are not timed).  Adds two event records per launch to the stream. */
fdtd_status fdtd_profile_begin(fdtd_ctx* ctx, int32_t max_launches);
/* Stops recording, synchronises, and writes per class (FDTD_KERNEL_CLASSES entries each) the
 * summed device milliseconds and the number of timed launches. */
fdtd_status fdtd_profile_end(fdtd_ctx* ctx, double* ms_per_class, int64_t* launches_per_class);

/* FP64 arithmetic-rate probe (instrumentation; no counterpart in the paper): runs independent
 * FP64 fused multiply-add chains on every SM (a few milliseconds, best of five timed runs after a
 * warm-up, CUDA events on `stream`, NULL = legacy default stream; it allocates and frees one small
 * device buffer) and writes the measured FP64 instruction rate (*fma_per_s, FMA instructions per
 * second; 2 flops each) and the best run's duration.  The FP64 path's roof is
 * min(HBM bandwidth / bytes, this rate / FP64 instructions) per cell-step.  Synchronises. */
fdtd_status fdtd_measure_fp64_rate(void* stream, double* fma_per_s, double* best_ms);

/* Device time of one kernel class running back to back (instrumentation; no counterpart in the
 * paper): captures n_launches (1..4096) launches of the E update (which = 0), the H update (1), the
 * DFT of E (2), the transposed E half-step (3), the transposed H half-step (4) or the fold of one
 * 32-step batch of monitor-ring samples into the DFT (5; FDTD_EINVAL without monitor rings) -- the
 * per-cell kernels of every domain, as one step launches them -- into a CUDA graph, replays it once to warm
 * up and once between two CUDA events on the context's stream, and writes the milliseconds per
 * launch.  Only the graph is bracketed, so nothing sits between the timed launches.  The launches
 * act on the live state (forward or adjoint fields, CPML memories, pole states, DFT accumulators or
 * the design gradient change as if the half-step ran 2 n_launches times at the current step index):
 * reset or restore the state afterwards (fdtd_adjoint_begin for the adjoint state).  Per-cell launch
 * mode (4) without an energy record only, and which = 2 needs a monitor (FDTD_EINVAL otherwise).
 * Synchronises. */
fdtd_status fdtd_time_half_steps(fdtd_ctx* ctx, int32_t which, int32_t n_launches, double* ms_per_launch);

#ifdef __cplusplus
}
#endif
#endif /* GBFDTD_FDTD_H */
