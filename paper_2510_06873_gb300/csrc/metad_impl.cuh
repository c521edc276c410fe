// Internal declarations of the sm_103a metadynamics bias path.
//
// One `Sys` value describes one system: geometry, switch constants and the
// device pointers of all its per-atom state.  Kernels take it by value; the
// batched kernels take a device array of them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace metad {

constexpr int kNY = 13;          // real Y_6^m, m = -6..6
constexpr int kBlockAtoms = 128; // threads per block of the per-atom kernels
constexpr int kBlockBias = 256;  // threads per block of the hill kernels
constexpr int kMaxBiasBlocks = 304;  // two per SM
constexpr int kHillsPerBlock = 256;  // hill kernel: blocks of kBlockBias threads take this many hills each
constexpr int kMaxCv = 5;        // CN, Q6 and the three lattice parameters

enum ErrBits : int {
    kErrCapacity = 1,   // an atom had more neighbours than max_nb
    kErrNonFinite = 2,  // a position was NaN or infinite
    kErrHills = 4,      // live hill list overflow
    kErrInternal = 8,   // a launch shape the buffers were not sized for
};

// Slots of the per-system FP64 scalar block `scal` (D = ncv + 3 lattice CVs
// at most kMaxCv; each vector slot holds kMaxCv entries).
enum Scal : int {
    kS0 = 0, kS1 = 1,            // CVs s1, s2 (then the lattice CVs, if any)
    kV = 5, kDV0 = 6, kDV1 = 7,  // bias and its gradient at the CVs
    kDepV = 11, kDepDV0 = 12,    // bias and gradient at the last deposit centre
    kDepW = 17,                  // height of the last deposited hill
    kDepC0 = 18,                 // the last deposit centre (or a caller's CV point)
    kVir0 = 23,                  // bias virial sum_pairs (dV/dd)_a d_a, a = x, y, z
    kBoxG0 = 26,                 // dV/dL_a at fixed fractional coordinates
    kNumScal = 32
};

// CV families (the metad_params.cv_kind values).
enum CvKind : int { kKindCoord = 0, kKindTorsion = 1, kKindNearest = 2 };

struct Sys {
    int n;          // atoms
    int ncv;        // 1 or 2
    int kind;       // CvKind
    int cn_unlike;  // CN mask
    int max_nb;     // ELL capacity per atom
    // box
    double L[3];
    float Lhi[3], Llo[3], halfL[3];
    float Lin[3];          // the largest float below L: x < L  <=>  x <= Lin
    // cells (edge >= rc, Morton-ranked)
    int nc[3];
    int ncell;
    float inv_h[3];
    // neighbour predicate: r^2 < rc^2 decided in FP64 inside the guard band
    double rc2;
    float rc2_lo, rc2_hi;
    // switch
    int sw_n, sw_m, stretch;
    float sw_nf;                 // sw_n and N as floating point: an int
    double sw_nd;                // conversion in a per-pair loop runs on
    float n_f;                   // the slow FP64 pipe of this part
    double n_d;
    double r0, rc;
    float inv_r0_hi, inv_r0_lo;  // 1/r0 as a float pair
    float a_hi, a_lo;            // 1/(1 - s_raw(rc)) (1 when not stretched)
    float k_hi, k_lo;            // s_raw(rc)/(1 - s_raw(rc)) (0 when not stretched)
    double a_d, k_d, inv_r0_d;
    // per-atom state, sorted order (cells ranked tile by tile) unless noted
    const float4 *pos_in;  // caller order
    float4 *pos_s;
    int *perm;             // sorted -> caller
    int *ucell, *uslot;    // caller order: cell and slot within it
    int *cell_count;       // [ncell]
    int *cell_start;       // [ncell + 1]
    int *scan_part;        // block partial sums of the cell scan
    const int *rank_of_xyz;  // cell (x, y, z) -> rank
    // tiles of up to 3 x 3 x 3 cells, one thread block each (tiles.cuh)
    int tiles;             // tiles of the current cell grid
    const int *tile_xyz;   // [tiles] tile coordinates x | y << 10 | z << 20, Morton order
    void *tile_tab;        // [tiles] staging tables, written by each rebuild
    int stage_cap;         // staged atoms a tile keeps in shared memory
    int fp64;              // records in FP64 (precision 1)
    // neighbour rows in quad-major order ([k / 4][n][4]: four entries of an
    // atom side by side, quads of consecutive atoms side by side); entries
    // are tile-local atom indices
    unsigned short *elist; // [max_nb / 4][n][4]: r < rc exactly, in Verlet-row order
    int *nn;               // [n]
    // Verlet rows (cutoff rc + skin at the reference positions)
    float4 *pos_ref;       // sorted positions at the last rebuild
    unsigned short *vlist; // [max_vnb / 4][n][4]
    int *vnn;              // [n]
    int max_vnb;
    int *flag;             // 1: rebuild the cell order and Verlet list this step
    float disp_thr2;       // (skin / 2)^2 with margin: rebuild above it
    float skin_eff;        // skin with margin
    float *Lref;           // [3] the box at the last rebuild (float)
    float rv2;             // (rc + skin)^2 with margin: Verlet cutoff
    int always_rebuild;    // skin == 0
    unsigned long long *rebuilds;  // number of rebuilds done
    // per-atom records [n][16] in the pair precision:
    //   rq: q_m (0..12), W (13), CN (14)
    //   rb: b_m (0..12), beta (13), qbar6 (14)
    //   rh: h_m (0..12), gamma (13)
    // 4-vectors [n][4]: fc = FC (the CN force sum, which needs no dV/ds) and
    // wc its virial sum (with the virial only); and per exact entry, in the
    // rows' quad-major order, the switch weight w_ij (wl) and the two halves
    // of the cross term c_ij = b_i.q_j + b_j.q_i: e_ij = b_i.q_j (eq) and
    // d_ij = q_i.b_j (dq)
    void *rq, *rb, *rh;
    void *fc, *wc;
    void *wl, *eq, *dq;
    double *part;          // per-block FP64 partial sums, slots of part_stride
    int part_stride;
    unsigned *ticket;      // completion counters of the last-block reductions
    double *scal;          // kNumScal doubles
    int *err;
    // hills and grid
    double *hc;            // [cap][hstride]
    double *hw;            // [cap]
    int hill_cap;
    double sigma[kMaxCv];  // per CV (the lattice CVs last)
    double inv2v[kMaxCv];  // 0.5 / sigma^2 per CV
    int D;                 // CVs the hills see: ncv (+ 3 lattice parameters)
    int hstride;           // doubles per hill centre: max(D, 2)
    int lattice;           // 1: the box lengths are CVs ncv .. ncv + 2
    int virial;            // 1: the force pass also sums the bias virial
    double w0, kbdt;
    int grid_on;
    int gn[2];
    double glo[2], ghi[2], gh[2];
    double *grid;          // [gn0][gn1][4]
    // per-step arguments, set on the copy of the descriptor a launch takes
    int K;                 // live hills
    const double *bias_x;  // CV point of the hill kernel
    double *bias_out;      // V, dV/ds1, dV/ds2 of the hill kernel
    int deposit;           // hill kernel: 1 = append a hill at bias_x
    float *F_out;          // caller's forces [n][3]
    int accumulate;        // 1: F_out += force, 0: F_out = force
    double fscale;         // forces are scaled by this
    // torsion and nearest-distance families (no neighbour list)
    double period[kMaxCv];      // 0, or the period of a periodic CV (2 pi for a torsion)
    double inv_period[kMaxCv];  // 1 / period (0 when not periodic)
    const int *cv_atoms;   // torsion: [ncv][4]; nearest: [ncv] references, then n_cand candidates
    const int *cand_slot;  // nearest: [n] position of each atom in the candidate group, or -1
    int n_cand;
    double sm_beta;        // nearest: 0 = exact, > 0 = soft minimum
    double *gcv;           // [ncv][16] per-CV gradient terms of the last CV pass
};

// The difference s - c a hill sees along CV d: wrapped into [-P/2, P/2]
// (nearest image) for a periodic CV, x - P rint(x / P), with x / P taken as
// x * (1 / P) (no division per hill; the two can pick different images only
// within an ulp of a half period, where both images are equally near).
__device__ __forceinline__ double hill_diff(const Sys &s, int d, double x)
{
    const double P = s.period[d];
    if (P > 0.0) x -= P * rint(x * s.inv_period[d]);
    return x;
}

// A coordinate wrapped into [0, L): x - L floor(x / L) in FP64, rounded to
// float32; a result that rounds up to L becomes 0.  The in-box test is the
// FP32 comparison with Lin (exact: x < L iff x <= Lin for a float x), so a
// wrapped input costs no FP64 instruction (their pipe is narrow here).
__device__ __forceinline__ float wrap_coord(float x, float Lin, double L)
{
    if (x >= 0.0f && x <= Lin) return x;
    double xd = (double)x;
    double w = xd - L * floor(xd / L);
    float f = (float)w;
    if ((double)f >= L) f = 0.0f;
    return f;
}

// Where a block works: block b of a grid of nb blocks of its system.  A
// single-system launch is that grid; a batched launch concatenates the grids
// of all its systems.
struct Blk {
    int b, nb;
};

__device__ __forceinline__ Blk own_blk() { return Blk{(int)blockIdx.x, (int)gridDim.x}; }

// A batched launch: block x belongs to system k with pre[k] <= x < pre[k + 1]
// (systems with no block in this launch have pre[k] == pre[k + 1]).
struct BatchView {
    const Sys *sys;  // device [nsys]
    const int *pre;  // device [nsys + 1], this launch's row
    int nsys;
};

__device__ __forceinline__ int batch_system(const BatchView &v, Blk &k)
{
    const int x = (int)blockIdx.x;
    int lo = 0, hi = v.nsys - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(v.pre + mid) <= x) lo = mid;
        else hi = mid - 1;
    }
    const int p0 = __ldg(v.pre + lo);
    k.b = x - p0;
    k.nb = __ldg(v.pre + lo + 1) - p0;
    return lo;
}

// Grids of a step, one row of block counts per launch kind.
enum GridKind : int {
    GK_ATOM256 = 0,    // one thread per atom, 256 per block
    GK_ATOM256_CAP,    // rebuild: binning and scatter
    GK_SCAN_TILES,     // rebuild: cell scan
    GK_CELL128_CAP,    // rebuild: cell sort
    GK_ONE,            // one block per system
    GK_TILES,          // one block per tile; a batch tile setting caps it
    GK_TILES_CAP,      // rebuild: Verlet rows (tiles, grid capped)
    GK_TILES_SUM,      // one block per tile (the pass holding the CV sums: never capped)
    GK_HILLS,          // hill kernel, evaluation
    GK_DEPOSIT,        // hill kernel, deposit (systems that deposit)
    kGridKinds
};

// Block count of one system for a grid kind (host side; shared by the
// single-system launches and the batch tables).  persist_cap > 0 caps the
// tile grids that carry no sum (a batch tile setting), 0 keeps the default.
int grid_blocks(const Sys &s, int kind, int persist_cap);

// The per-atom passes of a step on spatial tiles (k_cv.cu).
enum Pass : int {
    kPassFwd = 0,   // exact rows (+ CV forward with flag): a3-a4
    kPassAvg,       // Q6 average and the CV sums: a5
    kPassAdj,       // adjoint: a7
    kPassForce,     // forces: a8
    kPassForceCn,   // forces without a Q6 CV
    kNumPasses
};
constexpr int kMaxTileSmem = 224 * 1024;  // dynamic shared memory limit of a pass
// Staged atoms per tile kept in shared memory (a tile with its one-cell
// shell holds about 1,000 atoms at the workloads' densities): in FP32 two
// blocks of every pass fit on an SM.
constexpr int kStageCapF32 = 1216;
constexpr int kStageCapF64 = 1216;
int tile_smem(const Sys &s, int pass);   // dynamic shared memory of a pass
int pass_blocks(const Sys &s, int pass); // single-system grid of a pass
void launch_tile_pass(const Sys &s, int pass, int flag, cudaStream_t st);
void launch_batch_pass(const BatchView &v, int total, int pass, int fp64, int flag, int vir, int smem,
                       cudaStream_t st);

// Batched stage launches (one launch each over every system of the view).
void launch_batch_gather(const BatchView &v, int total, cudaStream_t st);
void launch_batch_rebuild(const BatchView *rows, const int *totals, int verlet_smem, cudaStream_t st);
void launch_batch_bias(const BatchView &v, int total, int deposit, cudaStream_t st);
void launch_batch_collect(const BatchView &v, double *out, cudaStream_t st);

// Launch entry points (stream-ordered, no host synchronisation).
void launch_gather_check(const Sys &s, cudaStream_t st);
void launch_rebuild(const Sys &s, cudaStream_t st);  // kernels early-exit unless *flag
void launch_bias(const Sys &s, int K, const double *s_dev, double *out_dev, int deposit, cudaStream_t st);
void configure_kernels();
void launch_grid_fold(const Sys &s, int K, cudaStream_t st);
void launch_nn_stats(const Sys &s, unsigned long long *sum, int *mx, cudaStream_t st);
void launch_export_pairs(const Sys &s, long long *pairs, int *count, cudaStream_t st);
void launch_per_atom_out(const Sys &s, int fp64, double *out, cudaStream_t st);
void set_ylm_constants(cudaStream_t st);
// Torsion and nearest-distance families: the CV pass (one block per system)
// and the force pass (one thread per atom).
void launch_gcv_forward(const Sys &s, int fp64, cudaStream_t st);
void launch_gcv_forces(const Sys &s, float *F, int accumulate, double scale, cudaStream_t st);
void launch_batch_gcv(const BatchView &one, int one_total, int fp64, cudaStream_t st);
void launch_batch_gcv_forces(const BatchView &atoms, int atom_total, cudaStream_t st);
// The whole small-system step in one launch (CVs, hills, deposit, forces),
// for systems of at most kFuseAtoms atoms.
constexpr int kFuseAtoms = 32768;
void launch_gcv_step(const Sys &s, int K, float *F, int accumulate, int deposit, int fp64, cudaStream_t st);
void launch_batch_gcv_step(const BatchView &hills, int hill_total, int fp64, cudaStream_t st);

int bias_blocks(int K);

// Free-energy passes (k_fes.cu): F at the bin centres of a regular grid from
// the hills (and grid), and F reweighted from biased samples.  V, F:
// device [prod n]; scratch: device [1 + prod n].
void launch_fes_points(const Sys &s, int K, const double *lo, const double *hi, const int *n, double *V, double *F,
                       double fac, cudaStream_t st);
void launch_fes_reweight(const double *S, const double *V, long long T, int ncv, const double *lo, const double *hi,
                         const int *n, double beta, double *scratch, double *F, cudaStream_t st);

// ----------------------------------------------------------------- device math
__device__ __forceinline__ float mi_f(float d, float halfL, float Lhi, float Llo)
{
    // one periodic shift, L carried as a float pair so the shift adds no
    // systematic error
    if (d > halfL) d = (d - Lhi) - Llo;
    else if (d < -halfL) d = (d + Lhi) + Llo;
    return d;
}

__device__ __forceinline__ double mi_d(double d, double L)
{
    if (d > 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
    return d;
}

template <typename real>
struct Vec3 {
    real x, y, z;
};

// Displacement r_j - r_i, minimum image, in the pair precision.
template <typename real>
__device__ __forceinline__ Vec3<real> displacement(const Sys &s, float4 pi, float4 pj);

// One axis of the minimum-image displacement xj - xi in float32.  Across the
// periodic boundary xj - xi is about +-L and would round at ulp(L) (7.6e-6 A
// for a 230 A box, a 1e-5 relative error in the switch of that pair); instead
// the coordinate near L is shifted first (x - L_hi is exact by Sterbenz), so
// only the small remainder is rounded.  The two directions of a pair give
// exactly opposite results.
__device__ __forceinline__ float mi_axis(float xj, float xi, float halfL, float Lhi, float Llo)
{
    const float d = xj - xi;
    if (d > halfL) return ((xj - Lhi) - xi) - Llo;   // xj near L
    if (d < -halfL) return (xj - (xi - Lhi)) + Llo;  // xi near L
    return d;
}

template <>
__device__ __forceinline__ Vec3<float> displacement<float>(const Sys &s, float4 pi, float4 pj)
{
    Vec3<float> d;
    d.x = mi_axis(pj.x, pi.x, s.halfL[0], s.Lhi[0], s.Llo[0]);
    d.y = mi_axis(pj.y, pi.y, s.halfL[1], s.Lhi[1], s.Llo[1]);
    d.z = mi_axis(pj.z, pi.z, s.halfL[2], s.Lhi[2], s.Llo[2]);
    return d;
}

template <>
__device__ __forceinline__ Vec3<double> displacement<double>(const Sys &s, float4 pi, float4 pj)
{
    Vec3<double> d;
    d.x = mi_d((double)pj.x - (double)pi.x, s.L[0]);
    d.y = mi_d((double)pj.y - (double)pi.y, s.L[1]);
    d.z = mi_d((double)pj.z - (double)pi.z, s.L[2]);
    return d;
}

// 1/sqrt(v) and 1/v with IEEE rounding.  (The SFU estimate refined by one
// Newton step is cheaper, but its rounding is not centred: over many pairs it
// shifted the averaged Q6 by about -2e-7 relative, which the bias gradient
// amplifies past the 1e-5 tolerance.)
template <typename real>
__device__ __forceinline__ real rsqrt_r(real v);
template <>
__device__ __forceinline__ float rsqrt_r<float>(float v) { return __frcp_rn(__fsqrt_rn(v)); }
template <>
__device__ __forceinline__ double rsqrt_r<double>(double v) { return 1.0 / sqrt(v); }

template <typename real>
__device__ __forceinline__ real recip_r(real v);
template <>
__device__ __forceinline__ float recip_r<float>(float v) { return __frcp_rn(v); }
template <>
__device__ __forceinline__ double recip_r<double>(double v) { return 1.0 / v; }

// Rational switch s_raw = (1 - x^n)/(1 - x^m), x = r/r0.  For integer n, m
// it equals S_n(x)/S_m(x) with S_k = 1 + x + ... + x^(k-1): sums of positive
// terms, so no cancellation near x = 1 (where float32 would lose 1e-4 of its
// precision) and no removable singularity.  m == 2n reduces to 1/(1 + x^n).
// Returns w and dw/dr (stretched: shifted and scaled to vanish at rc).
template <typename real>
__device__ __forceinline__ void switch_eval(const Sys &s, real r, real &w, real &dw);

template <typename real>
__device__ __forceinline__ real ipow(real x, int n)
{
    real v = real(1);
    real b = x;
    while (n > 0) {
        if (n & 1) v *= b;
        b *= b;
        n >>= 1;
    }
    return v;
}

// S_k(x) and S_k'(x) by Horner.
template <typename real>
__device__ __forceinline__ void geom_sum(real x, int k, real &S, real &dS)
{
    S = real(0);
    dS = real(0);
    for (int t = k - 1; t >= 0; --t) {
        dS = dS * x + S;
        S = S * x + real(1);
    }
}

template <typename real>
__device__ __forceinline__ real sw_n_real(const Sys &s);
template <>
__device__ __forceinline__ float sw_n_real<float>(const Sys &s) { return s.sw_nf; }
template <>
__device__ __forceinline__ double sw_n_real<double>(const Sys &s) { return s.sw_nd; }

template <typename real>
__device__ __forceinline__ real n_real(const Sys &s);
template <>
__device__ __forceinline__ float n_real<float>(const Sys &s) { return s.n_f; }
template <>
__device__ __forceinline__ double n_real<double>(const Sys &s) { return s.n_d; }

template <typename real>
__device__ __forceinline__ void switch_raw(const Sys &s, real x, real &f, real &dfdx)
{
    const int n = s.sw_n, m = s.sw_m;
    if (m == 2 * n) {
        real xn1;
        if (n == 6) {  // the common 6-12 switch: x^5 without the power loop
            const real x2 = x * x;
            xn1 = x2 * x2 * x;
        } else {
            xn1 = ipow<real>(x, n - 1);
        }
        real xn = xn1 * x;
        real inv = recip_r<real>(real(1) + xn);
        f = inv;
        dfdx = -sw_n_real<real>(s) * xn1 * inv * inv;
        return;
    }
    real Sn, dSn, Sm, dSm;
    geom_sum<real>(x, n, Sn, dSn);
    geom_sum<real>(x, m, Sm, dSm);
    const real inv = recip_r<real>(Sm);
    f = Sn * inv;
    dfdx = (dSn * Sm - Sn * dSm) * inv * inv;
}

template <>
__device__ __forceinline__ void switch_eval<float>(const Sys &s, float r, float &w, float &dw)
{
    float x = fmaf(r, s.inv_r0_hi, r * s.inv_r0_lo);
    float f, dfdx;
    switch_raw<float>(s, x, f, dfdx);
    // (f - s_c) / (1 - s_c) = f*a - k with a, k carried as float pairs
    w = (fmaf(f, s.a_hi, f * s.a_lo) - s.k_hi) - s.k_lo;
    dw = dfdx * s.a_hi * s.inv_r0_hi;
}

template <>
__device__ __forceinline__ void switch_eval<double>(const Sys &s, double r, double &w, double &dw)
{
    double x = r * s.inv_r0_d;
    double f, dfdx;
    switch_raw<double>(s, x, f, dfdx);
    w = f * s.a_d - s.k_d;
    dw = dfdx * s.a_d * s.inv_r0_d;
}



__device__ __forceinline__ void set_err(const Sys &s, int bits) { atomicOr(s.err, bits); }

// ------------------------------------------------------------------ bias grid
__device__ __forceinline__ void hermite(double t, double A[2], double B[2], double dA[2], double dB[2])
{
    const double t2 = t * t, t3 = t2 * t;
    A[0] = 2.0 * t3 - 3.0 * t2 + 1.0;
    A[1] = 3.0 * t2 - 2.0 * t3;
    B[0] = t3 - 2.0 * t2 + t;
    B[1] = t3 - t2;
    dA[0] = 6.0 * (t2 - t);
    dA[1] = 6.0 * (t - t2);
    dB[0] = 3.0 * t2 - 4.0 * t + 1.0;
    dB[1] = 3.0 * t2 - 2.0 * t;
}

// Bicubic Hermite patch of the node grid; zero outside [lo, hi].
__device__ __forceinline__ void grid_value(const Sys &s, double x0, double x1, double &V, double &g0, double &g1)
{
    V = g0 = g1 = 0.0;
    if (!s.grid_on) return;
    const double x[2] = {x0, x1};
    int c[2];
    double t[2];
    for (int a = 0; a < 2; ++a) {
        if (!(x[a] >= s.glo[a] && x[a] <= s.ghi[a])) return;
        int k = (int)floor((x[a] - s.glo[a]) / s.gh[a]);
        k = k < 0 ? 0 : (k > s.gn[a] - 2 ? s.gn[a] - 2 : k);
        c[a] = k;
        t[a] = (x[a] - (s.glo[a] + k * s.gh[a])) / s.gh[a];
    }
    double A0[2], B0[2], dA0[2], dB0[2], A1[2], B1[2], dA1[2], dB1[2];
    hermite(t[0], A0, B0, dA0, dB0);
    hermite(t[1], A1, B1, dA1, dB1);
    const double h0 = s.gh[0], h1 = s.gh[1];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const double *nd = s.grid + ((size_t)(c[0] + a) * s.gn[1] + (c[1] + b)) * 4;
            const double f = nd[0], fx = h0 * nd[1], fy = h1 * nd[2], fxy = h0 * h1 * nd[3];
            V += A0[a] * A1[b] * f + B0[a] * A1[b] * fx + A0[a] * B1[b] * fy + B0[a] * B1[b] * fxy;
            g0 += dA0[a] * A1[b] * f + dB0[a] * A1[b] * fx + dA0[a] * B1[b] * fy + dB0[a] * B1[b] * fxy;
            g1 += A0[a] * dA1[b] * f + B0[a] * dA1[b] * fx + A0[a] * dB1[b] * fy + B0[a] * dB1[b] * fxy;
        }
    g0 /= h0;
    g1 /= h1;
}


// Exact FP64 pair test: r^2 = (dx*dx + dy*dy) + dz*dz < rc^2 on the
// minimum-image displacement, no contraction.  Kept out of line and given
// plain values (no reference to the kernel's descriptor): it runs only for
// candidates inside the guard band, and inlined the compiler may evaluate
// it for every candidate under a predicate, on the slow FP64 pipe.
static __device__ __noinline__ bool pair_exact_fp64(float4 pi, float4 pj, double L0, double L1, double L2, double rc2)
{
    double dx = mi_d(__dadd_rn((double)pj.x, -(double)pi.x), L0);
    double dy = mi_d(__dadd_rn((double)pj.y, -(double)pi.y), L1);
    double dz = mi_d(__dadd_rn((double)pj.z, -(double)pi.z), L2);
    double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    r2 = __dadd_rn(r2, __dmul_rn(dz, dz));
    return r2 < rc2;
}

__device__ __forceinline__ bool pair_exact(const Sys &s, float4 pi, float4 pj)
{
    return pair_exact_fp64(pi, pj, s.L[0], s.L[1], s.L[2], s.rc2);
}

// displacement<float> for code where the whole warp is converged: the plain
// difference, and the boundary fix only when some lane of the warp needs it
// (a vote), instead of both fixes evaluated for every pair.  The same bits:
// mi_axis returns the plain difference exactly when |d| <= L/2.
__device__ __forceinline__ Vec3<float> displacement_warp(const Sys &s, float4 pi, float4 pj)
{
    Vec3<float> d{pj.x - pi.x, pj.y - pi.y, pj.z - pi.z};
    const bool wrap = fabsf(d.x) > s.halfL[0] || fabsf(d.y) > s.halfL[1] || fabsf(d.z) > s.halfL[2];
    if (__any_sync(0xffffffffu, wrap)) d = displacement<float>(s, pi, pj);
    return d;
}

// The float32 estimate decides every candidate outside a relative guard band
// of 3e-5 around rc^2; inside it the FP64 definition decides.  d is the
// float32 displacement of the pair.
__device__ __forceinline__ bool pair_in(const Sys &s, float4 pi, float4 pj, const Vec3<float> &d)
{
    float r2 = fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z));
    if (r2 < s.rc2_lo) return true;
    if (r2 > s.rc2_hi) return false;
    return pair_exact(s, pi, pj);
}

}  // namespace metad
