/*
 * metad.h -- C ABI of the GB300 (sm_103a) metadynamics bias path.
 *
 * One context holds one periodic system: its neighbour list, collective
 * variables (CVs), deposited hills and bias grid, all resident on one GPU.
 * Each MD step the caller hands over positions and receives bias forces to
 * add to its own forces, following the paper's biased potential
 *     U_b = U_0 + V_b                                      (Methods, Eq. 1)
 *     V_b(s) = sum_tau w_tau exp(-(s - s_tau)^2 / 2 sigma^2)  (Eqs. 2-3)
 * and its interface, which extracts the MD data every step and returns the
 * bias-driven forces (Section "Frameworks of GPU-MetaD", Fig. 1).
 *
 * Conventions (all entry points):
 *   * Units: Angstrom, kJ/mol, kJ/mol/Angstrom.
 *   * Positions: device float32 [N][4] = x, y, z, species id as a float
 *     (0.0 or 1.0), in the caller's atom order, inside the orthorhombic box
 *     [0, L) per axis (coordinates outside are wrapped: x - L floor(x/L) in
 *     FP64, rounded to float32, a result equal to L becomes 0).
 *   * Forces: device float32 [N][3] in the caller's atom order.
 *   * Ownership: the caller owns every pointer it passes and keeps device
 *     buffers alive until the context's stream has passed the call; the
 *     library owns all internal state and copies nothing out except through
 *     the explicit host outputs below.
 *   * Streams: work is enqueued on params.stream (a cudaStream_t; NULL makes
 *     the context create its own).  Calls with host outputs synchronise that
 *     stream; calls without them are asynchronous.
 *   * Errors: every call returns a metad_status and never throws.  Device-side
 *     errors (neighbour-list overflow, non-finite positions) are recorded in a
 *     device word and reported by the next synchronising call; after any error
 *     the context returns METAD_ERR_STATE until it is destroyed.
 *   * Call order per frame: build_neighbors -> cv_forward -> bias_eval ->
 *     bias_forces (-> deposit_hill).  A call out of order returns
 *     METAD_ERR_STATE without touching the context.
 */
#ifndef METAD_H
#define METAD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct metad_ctx metad_ctx;

typedef enum {
    METAD_OK = 0,
    METAD_ERR_INVALID = 1,  /* bad argument, size or parameter */
    METAD_ERR_OOM = 2,      /* device or host allocation failed */
    METAD_ERR_CUDA = 3,     /* a CUDA runtime call failed */
    METAD_ERR_CAPACITY = 4, /* neighbour list or hill list capacity exceeded */
    METAD_ERR_TIMEOUT = 5,  /* a bounded device wait gave up */
    METAD_ERR_STATE = 6     /* call out of order, or context already failed */
} metad_status;

/* Parameters of one context.  Fill with metad_params_default, then edit. */
typedef struct {
    int32_t n_atoms;        /* N >= 1 */
    int32_t n_cv;           /* 1: coordination number; 2: CN and averaged Q6
                               (torsion / nearest-distance families: 1 or 2
                               CVs of the family) */
    double box[3];          /* orthorhombic box lengths, each >= 2 rc (> 0 for
                               the torsion and nearest-distance families) */
    double rc;              /* neighbour cutoff (3.5) */
    double r0;              /* switch length (2.5) */
    int32_t sw_n, sw_m;     /* rational switch exponents (6, 12) */
    int32_t stretch;        /* 1: switch shifted and scaled to vanish at rc */
    int32_t cn_pairs;       /* 1: CN counts unlike-species pairs only; 0: all */
    double sigma[2];        /* hill widths per CV */
    double w0;              /* initial hill height, kJ/mol */
    double biasfactor;      /* well-tempered gamma > 1; +infinity gives plain
                               metadynamics (every height w0) */
    double temperature;     /* K */
    double kB;              /* kJ/mol/K (0.0083144626) */
    int32_t grid_on;        /* 1: bicubic Hermite bias grid (n_cv == 2 only;
                               not for torsions) */
    int32_t grid_n[2];      /* nodes per axis, both ends included (>= 2) */
    int32_t hill_capacity;  /* maximum live hills */
    double grid_lo[2];
    double grid_hi[2];
    int32_t precision;      /* 0: FP32 pair arithmetic, FP64 reductions and
                               hills; 1: FP64 throughout */
    int32_t max_neighbors;  /* per-atom capacity of the neighbour list (0: 64;
                               rounded up to a multiple of 4) */
    int32_t device;         /* CUDA device ordinal */
    int32_t step_graph;     /* 1: metad_step replays a captured CUDA graph of
                               its kernels, one per combination of flags and
                               hill count (up to 16 kept, least recently used
                               replaced; not while profiling); new position
                               and force buffers are patched into a captured
                               graph, not recaptured.  0 (default): direct
                               launches */
    void *stream;           /* cudaStream_t, or NULL */
    double skin;            /* Verlet skin in Angstrom (1.0): the cell order and
                               the rc + skin candidate list are rebuilt only
                               when an atom has moved more than skin/2 since
                               the last rebuild; 0 rebuilds every step.  The
                               exact rc list is recomputed every step. */
    int32_t cv_kind;        /* METAD_CV_COORDINATION (default), METAD_CV_TORSION
                               or METAD_CV_NEAREST (below) */
    int32_t reserved0;      /* 0 */
    double softmin_beta;    /* METAD_CV_NEAREST: 0 (default) = the exact nearest
                               distance; > 0 = its soft minimum with this beta
                               (1/Angstrom), see metad_set_cv_atoms */
    int32_t lattice_cvs;    /* 1: the three box lengths are CVs too, after the
                               per-atom ones: s = (s1 [, s2], L_x, L_y, L_z),
                               D = n_cv + 3 CVs, D-dimensional hills (the GaN
                               NPT runs bias the coordination number with the
                               triaxial lattice parameters, Section "B4-B1
                               phase transition in Large-scale systems").
                               Coordination family only; no grid.  Implies
                               virial. */
    int32_t virial;         /* 1: bias_forces also sums the bias virial and the
                               box gradient (metad_box_gradient) */
    double sigma_lattice[3];/* hill widths of the lattice CVs, Angstrom */
} metad_params;

/* CV families (metad_params.cv_kind).
 *
 * METAD_CV_COORDINATION: s1 = mean coordination number, s2 = mean locally
 *   averaged Q6, over the rc neighbour list (the paper's GaN runs, Section
 *   "B4-B1 phase transition in Large-scale systems").
 * METAD_CV_TORSION: n_cv torsion (dihedral) angles of atom quadruplets, the
 *   backbone Phi / Psi of the paper's alanine-dipeptide runs (Section
 *   "Alanine dipeptide torsion").  IUPAC sign, values in [-pi, pi], bond
 *   vectors by the minimum image; collinear atoms give 0 and no force.  The
 *   CVs are periodic: every hill sees s_d - c_kd wrapped into [-pi, pi]
 *   (nearest image).  No grid.
 * METAD_CV_NEAREST: n_cv distances, each from a reference atom to the
 *   nearest atom of one candidate group (minimum image), the surface-oxygen
 *   to nearest-hydrogen CV of the paper's rutile runs (Section "Water
 *   dissociation on rutile (110) surface").  The nearest candidate is the
 *   argmin of the FP64 squared distance (first in list order on a tie); with
 *   softmin_beta > 0 the CV is instead the soft minimum
 *     s = r_min - (1/beta) log sum_j exp(-beta (r_j - r_min)).
 *
 * The torsion and nearest-distance families use no neighbour list: rc, r0,
 * the switch, skin and max_neighbors are ignored, each box length need only
 * be positive, and the atoms come from metad_set_cv_atoms, which must be
 * called before the first cv_forward.  Bond and distance vectors are exact
 * FP64 differences of the float32 positions; a torsion's angle and gradient
 * then run in FP32 (precision 0) or FP64 (precision 1); the nearest distance
 * is FP64 in both.  Hills and forces are as for every family. */
enum { METAD_CV_COORDINATION = 0, METAD_CV_TORSION = 1, METAD_CV_NEAREST = 2 };

/* Defaults of the paper's GaN-style workloads: rc 3.5, r0 2.5, n 6, m 12,
 * stretched switch, unlike-pair CN, two CVs, sigma (0.05, 0.02), w0 1,
 * gamma 10, T 300 K, no grid, 65,536 hills, FP32 pairs, skin 1 A. */
void metad_params_default(metad_params *p);

/* Create a context for one system.  Validates p (METAD_ERR_INVALID), allocates
 * all device state up front (METAD_ERR_OOM).  *out is NULL on failure. */
metad_status metad_create(const metad_params *p, metad_ctx **out);

/* Release everything the context owns.  Safe on NULL. */
metad_status metad_destroy(metad_ctx *ctx);

/* Step a1-a3: wrap, cell binning and the full neighbour list
 * {j : r_ij^2 < rc^2}, minimum image, strict inequality, decided exactly as
 * the FP64 definition.  The paper is silent on neighbour lists: its CVs sum
 * over neighbours within a cutoff (Section "B4-B1 phase transition in
 * Large-scale systems", coordination number), and the list itself is this
 * library's infrastructure for them.  pos_dev: device float32 [N][4] (see
 * conventions), read on the context stream. */
metad_status metad_build_neighbors(metad_ctx *ctx, const float *pos_dev);

/* Steps a4-a5: per-atom CVs and their FP64 means.
 *   s1 = (1/N) sum_i CN_i,  CN_i = sum_j s(r_ij)   (unlike pairs by default)
 *   s2 = (1/N) sum_i qbar6_i (locally averaged Steinhardt Q6, n_cv == 2)
 * The coordination number is the CV of the paper's GaN runs (Section "B4-B1
 * phase transition in Large-scale systems": the Ga-N coordination, 4 in B4
 * and 6 in B1; the paper prints no switching function, read here as the
 * stretched rational switch (1 - x^n)/(1 - x^m), x = r/r0).  The averaged Q6
 * is the second CV of the benchmark workloads (the paper does not use it):
 * q_m(i) = sum_j w_ij Y_6m(r_ij) / W_i with w_ij the switch,
 * qbar_m(i) = (q_m(i) + sum_j w_ij q_m(j)) / (1 + W_i),
 * qbar6 = sqrt(4 pi / 13 sum_m |qbar_m|^2).
 * cv_host (NULL or double[n_cv]) receives s and synchronises.
 * per_atom_dev (NULL or device double [n_cv][N], caller order) receives CN_i
 * and qbar6_i. */
metad_status metad_cv_forward(metad_ctx *ctx, double *cv_host, double *per_atom_dev);

/* Step a6: V(s) = grid(s) + sum_k w_k exp(-sum_d (s_d - c_kd)^2 / 2 sigma_d^2)
 * and dV/ds in FP64 (Eqs. 2-3, a per-dimension sigma).  s_host NULL uses the
 * CVs of the last cv_forward (on the device, no synchronisation); otherwise
 * double[n_cv].  V_host / dVds_host (NULL or double / double[n_cv]) receive
 * the result and synchronise. */
metad_status metad_bias_eval(metad_ctx *ctx, const double *s_host, double *V_host, double *dVds_host);

/* Steps a7-a8: bias forces F = -dV_b/dr = -sum_d (dV/ds_d) ds_d/dr, the
 * force of the bias term of U_b = U_0 + V_b (Methods, Eq. 1), by the chain
 * rule through the CVs; the paper obtains it by automatic differentiation of
 * the CVs and bias (Section "Frameworks of GPU-MetaD"), here a hand-written
 * adjoint.  Written in the caller's atom order, times `scale` (1.0 for plain
 * forces).
 * accumulate 0: forces_dev = F; 1: forces_dev += F.  Deterministic: no
 * floating-point atomics. */
metad_status metad_bias_forces(metad_ctx *ctx, float *forces_dev, int32_t accumulate, double scale);

/* Atoms of the torsion and nearest-distance CVs, caller indices (host int32):
 *   METAD_CV_TORSION: count = 4 n_cv, quadruplets (a, b, c, d) in CV order;
 *   METAD_CV_NEAREST: count = n_cv + M, the n_cv reference atoms, then the
 *     M >= 1 candidate atoms shared by every CV.
 * Copied to the device (stream-ordered); may be called again between steps.
 * Errors: METAD_ERR_INVALID (NULL, wrong count, an index outside [0, N), an
 * atom repeated within a quadruplet or in the candidate group, a reference
 * atom that is also a candidate, a context of the coordination family). */
metad_status metad_set_cv_atoms(metad_ctx *ctx, const int32_t *atoms_host, int32_t count);

/* Number of CVs D the hills see: n_cv, plus 3 with lattice_cvs.  Every CV
 * vector a call takes or returns (cv_host, s_host, dVds_host, centres) has
 * D entries per point; hill centres are [K][D]. */

/* NPT: the orthorhombic box of the next steps (host double[3]; each length
 * >= 2 rc, > 0 for the torsion and nearest-distance families).  Positions
 * passed afterwards must lie in (or are wrapped into) the new box.  The cell
 * grid follows the box (never more cells than at creation).  The Verlet rows
 * are kept while every atom's move since the last rebuild stays within
 * (skin - |L - L_rebuild|) / 2, else rebuilt (decided on the device).
 * Captured step graphs are dropped.  Asynchronous unless the number of cells
 * changes.
 * Errors: METAD_ERR_INVALID (NULL, a length out of range). */
metad_status metad_set_box(metad_ctx *ctx, const double *box_host);

/* The derivative a barostat needs, from the last bias_forces: for each box
 * length, at fixed fractional coordinates (positions scaling with the box),
 *     dV/dL_a = dV/ds_{L_a} [lattice CVs] + (1/L_a) sum_pairs (dV/dd_ij)_a (d_ij)_a
 * (every per-atom CV depends on the positions only through the pair
 * displacements d_ij, which scale with the box), times the scale that
 * bias_forces was given.  dVdL_host: double[3].  Synchronises.
 * Errors: METAD_ERR_INVALID (NULL, a context without virial or lattice_cvs),
 * METAD_ERR_STATE (no bias_forces since creation). */
metad_status metad_box_gradient(metad_ctx *ctx, double *dVdL_host);

/* Step a9: deposit one hill at c (center_host double[n_cv], or NULL for the
 * last CVs) with the well-tempered height
 *   w = w0 exp(-V(c) / (kB T (gamma - 1)))
 * (the rule the paper names for its rutile runs; V includes the grid and
 * every earlier hill).  height_host (NULL or double) synchronises.
 * METAD_ERR_CAPACITY when the live list is full. */
metad_status metad_deposit_hill(metad_ctx *ctx, const double *center_host, double *height_host);

/* Deposit K hills one after another at centers_host (double[K][n_cv]), each
 * with its well-tempered height from the bias of all earlier ones; heights
 * (NULL or double[K]) receives them and synchronises. */
metad_status metad_deposit_hills(metad_ctx *ctx, const double *centers_host, int32_t K, double *heights_host);

/* Replace the live hills by K given hills (centers double[K][n_cv], heights
 * double[K], host memory). */
metad_status metad_load_hills(metad_ctx *ctx, const double *centers_host, const double *heights_host, int32_t K);

/* Copy the live hills out: *K receives the count; centers/heights (NULL or
 * room for cap hills) receive up to cap of them.  Synchronises. */
metad_status metad_get_hills(metad_ctx *ctx, double *centers_host, double *heights_host, int32_t cap, int32_t *K);

/* Fold every live hill into the bias grid (node values V, dV/ds1, dV/ds2,
 * d2V/ds1ds2 as exact FP64 sums) and empty the live list.  Needs grid_on. */
metad_status metad_fold_hills(metad_ctx *ctx);

/* Copy the grid nodes out: double [grid_n0][grid_n1][4].  Synchronises. */
metad_status metad_get_grid(metad_ctx *ctx, double *grid_host);

/* The last neighbour list as unordered pairs (i < j, caller indices,
 * ascending): *P receives the count, pairs_host (NULL or int64[cap][2])
 * up to cap pairs.  Synchronises. */
metad_status metad_export_neighbors(metad_ctx *ctx, int64_t *pairs_host, int64_t cap, int64_t *P);

/* One whole step a1-a8 (+ a9 when deposit != 0) without any host
 * synchronisation: build_neighbors, cv_forward, bias_eval, bias_forces. */
metad_status metad_step(metad_ctx *ctx, const float *pos_dev, float *forces_dev, int32_t accumulate,
                        int32_t deposit);

/* One whole step from HOST buffers, for callers whose positions live in host
 * memory: copies pos_host (float32 [N][4]) to a context-owned device buffer,
 * runs metad_step, copies the forces back to forces_host (float32 [N][3];
 * with accumulate 1 its incoming values are uploaded and added to) and the
 * CVs / bias to cv_host / V_host (NULL to skip).  Synchronises.  Page-locked
 * host memory makes the copies asynchronous DMA.  The device staging buffers
 * are allocated on the first call. */
metad_status metad_step_host(metad_ctx *ctx, const float *pos_host, float *forces_host, int32_t accumulate,
                             int32_t deposit, double *cv_host, double *V_host);

/* Stage profiling.  Between begin and end, every kernel stage this context
 * launches is bracketed by CUDA events on its stream (at most max_records
 * stages are recorded).  end synchronises and writes, per stage index
 * 0..METAD_NUM_STAGES-1 (names from metad_stage_name), the summed device
 * milliseconds and the number of records (either pointer may be NULL). */
#define METAD_NUM_STAGES 11
metad_status metad_profile_begin(metad_ctx *ctx, int32_t max_records);
metad_status metad_profile_end(metad_ctx *ctx, double *ms_per_stage, int32_t *records_per_stage);
const char *metad_stage_name(int32_t stage);

/* Statistics of the last neighbour list: total entries of the full list
 * (twice the unordered pair count) and the largest per-atom count.
 * Synchronises. */
metad_status metad_neighbor_stats(metad_ctx *ctx, int64_t *entries, int32_t *max_per_atom);

/* Number of cell-order / Verlet-list rebuilds since creation (the first
 * build_neighbors always rebuilds).  Synchronises. */
metad_status metad_rebuild_count(metad_ctx *ctx, int64_t *count);

/* Device bytes a context with these parameters allocates at creation (the
 * sum of its requests; the allocator may round each up).  No GPU needed.
 * Errors: those of metad_create's parameter checks. */
metad_status metad_estimate_bytes(const metad_params *params, int64_t *bytes);

/* Device bytes this context has requested so far (creation plus the
 * buffers allocated on first use by export and host-buffer steps). */
int64_t metad_device_bytes(const metad_ctx *ctx);

/* Turn the CUDA-graph replay of metad_step on (1) or off (0) after creation
 * (params.step_graph sets it at creation).  Errors: METAD_ERR_INVALID. */
metad_status metad_set_step_graph(metad_ctx *ctx, int32_t on);

/* Number of kernels this context has launched since creation. */
int64_t metad_launch_count(const metad_ctx *ctx);

/* Bias V(s) and dV/ds from caller-held hills, allocating nothing.
 *
 * (No counterpart in the paper: this serves callers that cannot allocate
 * device memory where they need the bias -- an MD engine whose step runs on
 * its own stream while other work is in flight, where cudaMalloc/cudaFree
 * could synchronise the device and stall it; code bound to a fixed memory
 * budget or pool; code that must not create a metad_ctx, which allocates.)
 *
 * Computes the hill sum of metad_bias_eval on a context without a grid and
 * without periodic CVs:
 *   out_dev[0] = sum_k w_k exp(-sum_d (s_d - c_kd)^2 / 2 sigma_d^2)
 *   out_dev[1 + d] = dV/ds_d
 * s_dev: device double[n_cv]; centers_dev: device double[K][n_cv];
 * heights_dev: device double[K]; sigma_host: host double[n_cv];
 * out_dev: device double[3] (out_dev[2] = 0 when n_cv == 1).  Work is
 * enqueued on `stream` of `device` and the call returns without waiting;
 * the caller's current device is restored before returning.
 *
 * Scratch: a fixed array inside the library (about 12 KB on every GPU that
 * loads it, held until the process exits) that holds one partial sum per
 * block of 256 hills, so K may be at most 131,072: larger K returns
 * METAD_ERR_CAPACITY.  The first call on a device looks up that array's
 * device address; make the first call before any stream capture.  That
 * address is cached for the life of the process: after a cudaDeviceReset of
 * the device, do not call this entry point again.  Each call clears the
 * completion counter it needs; calls that overlap on the GPU (concurrent
 * streams) share the array and race, so order them.
 *
 * Intended for CVs without a period (the coordination family, nearest
 * distances): s - c is taken as is, with no wrap to the nearest image, so a
 * torsion context's periodic hills need metad_bias_eval instead.
 * Errors: METAD_ERR_INVALID (NULL pointers, n_cv not 1 or 2, K < 0,
 * sigma <= 0), METAD_ERR_CUDA (a runtime call failed). */
metad_status metad_bias_eval_noalloc(const double *s_dev, int32_t n_cv, const double *centers_dev,
                                     const double *heights_dev, int32_t K, const double *sigma_host,
                                     double *out_dev, int32_t device, void *stream);

/* Measured FP32 multiply-add throughput of a device, in TFLOP/s: the
 * denominator of the FP32 roofline fraction the benchmark reports for its
 * ALU-bound kernels.  (No counterpart in the paper: a measurement helper.)
 * Every thread of a grid of 8 x 256-thread blocks per SM runs 8 independent
 * fmaf chains of `iters` steps; `repeats` launches are timed with CUDA events
 * after one untimed launch.  Allocates a small buffer, synchronises, and
 * restores the caller's current device.
 * Errors: METAD_ERR_INVALID (NULL, iters or repeats < 1), METAD_ERR_CUDA. */
metad_status metad_probe_fp32_peak(int32_t device, int32_t iters, int32_t repeats, double *tflops_host);

/* Accuracy probe of the kernels' FP32 reciprocal square root and reciprocal
 * (the SFU estimate refined by one Newton-Raphson step with an exactly formed
 * residual) beside CUDA's correctly rounded intrinsics, for a test.  (No
 * counterpart in the paper.)  out_dev[i] = f(v_dev[i]) for i < n, with f by
 * `which`: 0 the kernels' 1/sqrt, 1 __frsqrt_rn, 2 the kernels' 1/v,
 * 3 __frcp_rn.  Device arrays of n floats, owned by the caller; launched on
 * `stream` (NULL: the default stream), asynchronous.
 * Errors: METAD_ERR_INVALID (NULL array, n < 0, which outside 0..3),
 * METAD_ERR_CUDA (launch failure). */
metad_status metad_probe_recip(const float *v_dev, float *out_dev, int64_t n, int32_t which, void *stream);

/* Copy the last CVs, bias and bias gradient to the host (any may be NULL).
 * Synchronises and reports any pending device error. */
metad_status metad_read_results(metad_ctx *ctx, double *cv_host, double *V_host, double *dVds_host);

/* Wait for the context's stream and report any pending device error. */
metad_status metad_sync(metad_ctx *ctx);

/* The stream the context enqueues on (cudaStream_t). */
void *metad_stream(metad_ctx *ctx);

/* Live hill count as tracked on the host (no synchronisation). */
int32_t metad_hill_count(const metad_ctx *ctx);

/* Static text for a status code. */
const char *metad_status_string(metad_status s);

/* Text of the last error recorded on this context (never NULL). */
const char *metad_last_error(const metad_ctx *ctx);

/* ------------------------------------------------------------------ batches
 * Many independent systems stepped together: each stage of the step
 * (gather, rebuild chain, CVs, bias, adjoint and forces, deposit) is ONE
 * kernel launch whose grid is the concatenation of every system's own grid,
 * instead of one launch per stage per system.  (No counterpart in the
 * paper, which runs one system per process; it serves many small walkers or
 * replicas on one GPU, where per-system launches leave the GPU idle.)
 *
 * A batch refers to existing contexts; it owns none of them.  Every context
 * must be on the same device and stream, with the same n_cv and precision.
 * Each system keeps its own neighbour state, hills, grid and reductions, so
 * with the default tile (0) a batched step gives every system the same bits
 * as metad_step on that context alone.  Destroy the batch before its
 * contexts; per-context calls may be interleaved with batched steps (same
 * stream, so they are ordered). */
typedef struct metad_batch metad_batch;

/* ctxs: host array of n >= 1 context pointers.  Allocates the descriptor
 * tables (device) and a small pinned ring (host).
 * Errors: METAD_ERR_INVALID (NULL, n < 1, contexts that differ in device,
 * stream, n_cv or precision, a failed context), METAD_ERR_OOM. */
metad_status metad_batch_create(metad_ctx *const *ctxs, int32_t n, metad_batch **out);

metad_status metad_batch_destroy(metad_batch *batch);

/* Tile setting of the per-atom kernels: at most `blocks_per_system` blocks
 * per system for each of them (0 = the single-context grid); the blocks
 * then walk the system's atoms grid-stride.  It changes no result: those
 * kernels carry no reduction, and the pass holding the CV sums keeps its
 * own grid, fixed by N.
 * Errors: METAD_ERR_INVALID (negative). */
metad_status metad_batch_set_tile(metad_batch *batch, int32_t blocks_per_system);

/* One full step (metad_step: neighbours, CVs, bias, forces, then an optional
 * deposit) for every active system of the batch.
 * pos_dev: host array of n device pointers, float32 [N_k][4] each;
 * forces_dev: host array of n device pointers, float32 [N_k][3] each, written
 * (accumulate = 0) or added to (accumulate = 1);
 * deposit: host int32[n] (1 = deposit a hill at that system's CVs after its
 * forces) or NULL for none;
 * active: host int32[n] (0 = leave system k out of this step; its pointers
 * may then be NULL) or NULL for all.  Asynchronous; stream-ordered.
 * Errors: METAD_ERR_INVALID (NULL pointers), METAD_ERR_STATE (a context has
 * failed), METAD_ERR_CAPACITY (a deposit into a full hill list),
 * METAD_ERR_CUDA. */
metad_status metad_batch_step(metad_batch *batch, const float *const *pos_dev, float *const *forces_dev,
                              int32_t accumulate, const int32_t *deposit, const int32_t *active);

/* CVs (host double [n][2], s2 = 0 when n_cv == 1) and biases (host double
 * [n]) of the last batched step; either may be NULL.  Synchronises and
 * reports the first device error of any system (that context then fails). */
metad_status metad_batch_read(metad_batch *batch, double *cv_host, double *V_host);

/* Asynchronous form of metad_batch_read: enqueues the copy of, per system,
 * {s1, s2, V, device error word} (double [n][4]) into out_host (page-locked
 * memory for a true asynchronous copy) and returns.  The values are valid
 * once the batch's stream has passed this call; a non-zero error word means
 * that system's context has failed (its next call reports it). */
metad_status metad_batch_collect(metad_batch *batch, double *out_host);

/* Kernels launched by batched steps since creation. */
int64_t metad_batch_launch_count(const metad_batch *batch);

/* Text of the last error recorded on this batch (never NULL). */
const char *metad_batch_last_error(const metad_batch *batch);

/* -------------------------------------------------------------- free energy
 * Analysis passes (not per step; each call allocates a device buffer for
 * its own use and synchronises).  The grid is regular: n[d] bins over
 * [lo[d], hi[d]) per CV (n[1], lo[1], hi[1] unused when n_cv == 1), laid
 * out row-major with the first CV slowest; F_host is double [n0 (x n1)].
 *
 * metad_fes_grid: the well-tempered sum-of-hills estimate at the bin centres
 * s_d = lo_d + (i_d + 1/2)(hi_d - lo_d)/n_d,
 *     F(s) = -(gamma / (gamma - 1)) V(s),  gamma = params.biasfactor,
 * with V this context's bias (live hills + grid), shifted so the minimum
 * over the grid is 0 (Methods: the bias fills the FES; the well-tempered
 * limit is read here as the standard one, the paper prints no formula).
 *
 * metad_fes_reweight: Eqs. 4-5 on the grid's histogram: for T samples
 * (samples_host: double [T][n_cv] CV values; V_host: double [T] the bias at
 * each, as a biased run records them),
 *     P_b = sum_{t in b} exp(beta V_t) / sum_{t inside the grid} exp(beta V_t),
 *     F_b = -(1/beta) log P_b,  beta = 1 / (params.kB params.temperature),
 * shifted to minimum 0 over the non-empty bins; empty bins are +inf.  Every
 * sum runs in sample order (bit-reproducible).
 * Errors: METAD_ERR_INVALID (NULL pointers, n < 1, hi <= lo, more than 2^24
 * bins, T < 1), METAD_ERR_OOM / METAD_ERR_CUDA. */
metad_status metad_fes_grid(metad_ctx *ctx, const double *lo, const double *hi, const int32_t *n, double *F_host);

/* CVs of a stored trajectory (offline analysis, no bias or forces; the
 * paper's trajectory-analysis module aligns CV outputs with the MD frames,
 * Section "Frameworks of GPU-MetaD").  frames_dev: device float32 [T][N][4]
 * (N = params.n_atoms), frame t at frames_dev + 4 N t; cv_host: double
 * [T][2] (s2 = 0 when n_cv == 1).  Runs build_neighbors and cv_forward per
 * frame (the neighbour list carries over between frames as in a run) and
 * copies all CVs back once; synchronises.
 * Errors: METAD_ERR_INVALID (NULL, T < 1), those of the per-frame calls. */
metad_status metad_cv_trajectory(metad_ctx *ctx, const float *frames_dev, int64_t T, double *cv_host);
metad_status metad_fes_reweight(metad_ctx *ctx, const double *samples_host, const double *V_host, int64_t T,
                                const double *lo, const double *hi, const int32_t *n, double *F_host);

#ifdef __cplusplus
}
#endif

#endif /* METAD_H */
