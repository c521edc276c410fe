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
    // per-atom state, sorted (Morton) order unless noted
    const float4 *pos_in;  // caller order
    float4 *pos_s;
    int *perm;             // sorted -> caller
    int *scell;            // cell of each sorted atom
    int *ucell, *uslot;    // caller order: cell and slot within it
    int *cell_count;       // [ncell]
    int *cell_start;       // [ncell + 1]
    int *scan_part;        // block partial sums of the cell scan
    const int *rank_of_xyz;  // cell (x, y, z) -> Morton rank
    const int *xyz_of_rank;  // Morton rank -> packed x | y << 10 | z << 20
    int *nbr;              // [n][max_nb] sorted indices, row per atom: r < rc exactly;
                           // entries j > i first (nh of them), then j < i
    int *nn;               // [n]
    int *nh;               // [n] entries with j > i
    void *wl;              // JW<real> [n][max_nb]: neighbour and switch weight of each entry
    void *pairF;           // real [n][max_nb][4]: G_ij in i's entry of j, -G_ji in the others
    void *cross;           // real [n][max_nb]: b_j.q_i of each exact entry (two CVs)
    void *geo;             // real [n][max_nb][4]: r_j - r_i (minimum image) and the CN mask
                           // of each exact entry, written by the exact filter
    // Verlet list (cutoff rc + skin, built at the reference positions)
    float4 *pos_ref;       // sorted positions at the last rebuild
    int *vnbr;             // [n][max_vnb]; with mirror slots an entry j > i carries, above bit 23,
                           // i's position in j's Verlet row (set once per rebuild by the filter)
    int *vnn;              // [n]
    int *vnh;              // [n] Verlet entries with j > i (stored first)
    int max_vnb;
    // mirror slots: where the pair force of i's entry j > i goes in j's row,
    // without searching j's row in the force pass
    int mirror;                // 1: in use (n < 2^23, rows of at most 255 entries)
    unsigned short *vround;    // [n][vround_stride]: per filter round r (Verlet entries 8r .. 8r + 7),
                               // the exact entries before it | the round's exact bits << 8
    int vround_stride;
    int *rows_fresh;           // 1 from a rebuild until the CV pass after the next filter
    int *flag;             // 1: rebuild the cell order and Verlet list this step
    float disp_thr2;       // (skin / 2)^2 with margin: rebuild above it
    float skin_eff;        // skin with margin
    float *Lref;           // [3] the box at the last rebuild (float)
    float rv2;             // (rc + skin)^2 with margin: Verlet cutoff
    int always_rebuild;    // skin == 0
    unsigned long long *rebuilds;  // number of rebuilds done
    void *cn, *W, *qb6;    // real-typed per-atom scalars
    void *q, *b, *h;       // real-typed per-atom records [n][16]: q_m; b_m, beta; h_m, gamma
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
    GK_GROUPS_CAP,     // rebuild: Verlet rows
    GK_ONE,            // one block per system
    GK_GROUPS,         // one block per 16 atoms (lane-group kernels); a batch tile caps it
    GK_CV,             // the Q6 pass with the CV sums: persistent, by N only
    GK_ATOM32,         // one block per 32 atoms (four-lane adjoint); a batch tile caps it
    GK_ATOM128,        // one block per 128 atoms (pair-parallel force); a batch tile caps it
    GK_SUM,            // the CV sums: blocks by N only
    GK_HILLS,          // hill kernel, evaluation
    GK_DEPOSIT,        // hill kernel, deposit (systems that deposit)
    kGridKinds
};

// Block count of one system for a grid kind (host side; shared by the
// single-system launches and the batch tables).  persist_cap > 0 caps the
// lane-group grids (a batch tile setting), 0 keeps the default.
int grid_blocks(const Sys &s, int kind, int persist_cap);

// Batched stage launches (one launch each over every system of the view).
void launch_batch_gather(const BatchView &v, int total, cudaStream_t st);
void launch_batch_rebuild(const BatchView *rows, const int *totals, cudaStream_t st);
void launch_batch_cv(const BatchView &groups, int group_total, const BatchView &cv, int cv_total,
                     const BatchView &sums, int sum_total, int fp64, int ncv, cudaStream_t st);
void launch_cv_sum(const Sys &s, int fp64, cudaStream_t st);
void launch_batch_bias(const BatchView &v, int total, int deposit, cudaStream_t st);
// part 0: adjoint, pair forces and gather; 1: the adjoint only; 2: the rest
void launch_batch_force(const BatchView &groups, int group_total, const BatchView &adj, int adj_total,
                        const BatchView &pairs, int pair_total, int fp64, int ncv, int virial, cudaStream_t st,
                        int part = 0);
void launch_batch_collect(const BatchView &v, double *out, cudaStream_t st);

// Launch entry points (stream-ordered, no host synchronisation).
void launch_gather_check(const Sys &s, cudaStream_t st);
void launch_rebuild(const Sys &s, cudaStream_t st);  // kernels early-exit unless *flag
void launch_filter(const Sys &s, int fp64, cudaStream_t st);
void launch_cv_fwd(const Sys &s, int fp64, int fused_filter, cudaStream_t st);
void launch_cv_avg(const Sys &s, int fp64, cudaStream_t st);
void launch_bias(const Sys &s, int K, const double *s_dev, double *out_dev, int deposit, cudaStream_t st);
void launch_adjoint(const Sys &s, int fp64, cudaStream_t st);
void launch_force_pairs(const Sys &s, int fp64, double scale, cudaStream_t st);  // + virial if s.virial
void launch_force_gather(const Sys &s, int fp64, float *F, int accumulate, cudaStream_t st);
void configure_kernels();
void launch_grid_fold(const Sys &s, int K, cudaStream_t st);
void launch_nn_stats(const Sys &s, unsigned long long *sum, int *mx, cudaStream_t st);
// Kernels whose only argument is the descriptor, per file (step graphs patch
// their I/O buffers in place).
bool sys_kernel_neighbors(const void *func);
bool sys_kernel_cv(const void *func);
bool sys_kernel_bias(const void *func);
bool sys_kernel_gcv(const void *func);
void launch_export_pairs(const Sys &s, int fp64, long long *pairs, int *count, cudaStream_t st);
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

// 1/sqrt(v) and 1/v in FP32, branch-free: the SFU estimate y refined by one
// Newton-Raphson step whose residual is formed without losing the product's
// rounding error (Markstein's scheme; the exact error of v*y recovered by an
// FMA, as in Dekker's two-product).  The step's result is y (1 + r/2) (resp.
// y (1 + r)) rounded once, within a few units of 2^-44 of the exact value:
// correctly rounded except next to a rounding tie, and with no rounding
// bias.  (An estimate refined with a rounded residual rounds with a bias:
// over many pairs it shifted the averaged Q6 by about -2e-7 relative, which
// the bias gradient amplifies past the 1e-5 tolerance.)  Positive normal
// arguments only (squared pair distances, switch denominators >= 1).
__device__ __forceinline__ float rsqrt_newton(float v)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
    const float p = v * y;
    const float pe = fmaf(v, y, -p);                  // v y = p + pe exactly
    const float r = fmaf(-pe, y, fmaf(-p, y, 1.0f));  // 1 - v y^2
    return fmaf(0.5f * y, r, y);
}
__device__ __forceinline__ float recip_newton(float v)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
    const float r = fmaf(-v, y, 1.0f);  // 1 - v y, one rounding of a quantity of order 2^-22
    return fmaf(y, r, y);
}

template <typename real>
__device__ __forceinline__ real rsqrt_r(real v);
template <>
__device__ __forceinline__ float rsqrt_r<float>(float v) { return rsqrt_newton(v); }
template <>
__device__ __forceinline__ double rsqrt_r<double>(double v) { return 1.0 / sqrt(v); }

template <typename real>
__device__ __forceinline__ real recip_r(real v);
template <>
__device__ __forceinline__ float recip_r<float>(float v) { return recip_newton(v); }
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


// ------------------------------------------------------------ lane groups
// Per-atom kernels give one atom a group of kG lanes; lane l handles the
// atom's neighbours l, l + kG, ... so all its neighbour loads are in flight
// together.
constexpr int kG = 8;
constexpr int kAtomsPerBlock = kBlockAtoms / kG;

// Grid of every lane-group kernel; the FP64 partial-sum slots are sized from
// it, so launches and allocations can never disagree.
__host__ __device__ inline int group_grid(int n) { return (n + kAtomsPerBlock - 1) / kAtomsPerBlock; }

// Without a Q6 pass the CN sum runs in its own kernel: kSumThreads threads
// per block, one block per kSumAtoms atoms (at most kMaxBiasBlocks blocks).
constexpr int kSumThreads = 256;
constexpr int kSumAtoms = 2048;
__host__ __device__ inline int sum_blocks(int n)
{
    const int b = (n + kSumAtoms - 1) / kSumAtoms;
    return b < 1 ? 1 : (b > kMaxBiasBlocks ? kMaxBiasBlocks : b);
}

// Persistent grids (the CV kernels, and the capped rebuild kernels) have at
// most kPersistBlocks blocks, walking their work grid-stride.
constexpr int kPersistBlocks = 152 * 16;

// The it-th work item (atom group or chunk) of block b of nb: items b,
// b + nb, b + 2 nb, ...  The items of one sweep form one compact window of
// the Morton order, so the records they gather stay in L2.  (Mapping the
// blocks that share an SM to consecutive items, for L1 reuse, measured
// slower: the gather kernels lost more to L2 misses than they won in L1.)
__device__ __forceinline__ int work_item(Blk k, int it) { return k.b + it * k.nb; }

__host__ __device__ inline int persist_grid(int n)
{
    const int g = group_grid(n);
    return g < kPersistBlocks ? g : kPersistBlocks;
}

struct AtomLane {
    int i;    // atom (sorted index), may be >= n for idle groups
    int l;    // lane within the group
    bool ok;  // i < n
};

__device__ __forceinline__ AtomLane atom_lane_at(const Sys &s, int blk)
{
    AtomLane a;
    a.i = blk * kAtomsPerBlock + (threadIdx.x / kG);
    a.l = threadIdx.x & (kG - 1);
    a.ok = a.i < s.n;
    return a;
}


__device__ __forceinline__ unsigned group_mask_bits(unsigned ballot)
{
    const int base = (threadIdx.x & 31) & ~(kG - 1);
    return (ballot >> base) & ((1u << kG) - 1u);
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

// pair_in for code where the whole warp is converged: the FP64 decision runs
// only when some lane of the warp has a candidate inside the guard band (a
// vote), as a warp-uniform branch.  The same decisions as pair_in.
__device__ __forceinline__ bool pair_in_warp(const Sys &s, bool valid, float4 pi, float4 pj, const Vec3<float> &d)
{
    const float r2 = fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z));
    bool in = valid && r2 < s.rc2_lo;
    const bool band = valid && r2 >= s.rc2_lo && r2 <= s.rc2_hi;
    if (__any_sync(0xffffffffu, band)) {
        if (band) in = pair_exact(s, pi, pj);
    }
    return in;
}

// The geometry of an exact entry, cached by the filter so the CV and force
// passes read one contiguous record per entry instead of gathering the
// neighbour's position again: r_j - r_i, and in the fourth slot a tag
// (carried through float registers unchanged): the bits of j, the CN mask in
// bit 31, and with mirror slots, for an entry j > i, i's position in j's
// Verlet row in bits 23..30.  The force pass reads it for the last time
// (kLast: an evict-first load, so the stream does not push the gathered
// per-atom records out of L2).
constexpr unsigned kCnBit = 0x80000000u;
constexpr int kMirrorShift = 23;
constexpr unsigned kMirrorJ = (1u << kMirrorShift) - 1u;

__device__ __forceinline__ unsigned make_tag(const Sys &s, int j, float4 pi, float4 pj, unsigned vm)
{
    return (unsigned)j | (vm << kMirrorShift) | ((!s.cn_unlike || pj.w != pi.w) ? kCnBit : 0u);
}

template <typename real>
__device__ __forceinline__ void store_geo(const Sys &s, size_t slot, const Vec3<float> &df, float4 pi, float4 pj,
                                          int j, unsigned vm);
template <>
__device__ __forceinline__ void store_geo<float>(const Sys &s, size_t slot, const Vec3<float> &df, float4 pi,
                                                 float4 pj, int j, unsigned vm)
{
    const unsigned tag = make_tag(s, j, pi, pj, vm);
    reinterpret_cast<float4 *>(s.geo)[slot] = make_float4(df.x, df.y, df.z, __uint_as_float(tag));
}
template <>
__device__ __forceinline__ void store_geo<double>(const Sys &s, size_t slot, const Vec3<float> &, float4 pi,
                                                  float4 pj, int j, unsigned vm)
{
    const Vec3<double> d = displacement<double>(s, pi, pj);
    const unsigned tag = make_tag(s, j, pi, pj, vm);
    double2 *g = reinterpret_cast<double2 *>(s.geo) + 2 * slot;
    g[0] = make_double2(d.x, d.y);
    g[1] = make_double2(d.z, __longlong_as_double((long long)tag));
}

// j, the CN mask and the mirror position (0 without mirror slots) of a tag.
__device__ __forceinline__ void untag(const Sys &s, unsigned tag, int &j, bool &cn, unsigned &vm)
{
    j = (int)(tag & (s.mirror ? kMirrorJ : ~kCnBit));
    cn = (tag & kCnBit) != 0u;
    vm = s.mirror ? (tag & ~kCnBit) >> kMirrorShift : 0u;
}

template <typename real, bool kLast = false>
__device__ __forceinline__ void load_geo(const Sys &s, size_t slot, Vec3<real> &d, bool &cn, int &j, unsigned &vm);
template <>
__device__ __forceinline__ void load_geo<float, false>(const Sys &s, size_t slot, Vec3<float> &d, bool &cn, int &j,
                                                       unsigned &vm)
{
    const float4 g = reinterpret_cast<const float4 *>(s.geo)[slot];
    d.x = g.x;
    d.y = g.y;
    d.z = g.z;
    untag(s, __float_as_uint(g.w), j, cn, vm);
}
template <>
__device__ __forceinline__ void load_geo<float, true>(const Sys &s, size_t slot, Vec3<float> &d, bool &cn, int &j,
                                                      unsigned &vm)
{
    const float4 g = __ldcs(reinterpret_cast<const float4 *>(s.geo) + slot);
    d.x = g.x;
    d.y = g.y;
    d.z = g.z;
    untag(s, __float_as_uint(g.w), j, cn, vm);
}
template <>
__device__ __forceinline__ void load_geo<double, true>(const Sys &s, size_t slot, Vec3<double> &d, bool &cn, int &j,
                                                       unsigned &vm)
{
    const double2 *g = reinterpret_cast<const double2 *>(s.geo) + 2 * slot;
    const double2 a = __ldcs(g), b = __ldcs(g + 1);
    d.x = a.x;
    d.y = a.y;
    d.z = b.x;
    untag(s, (unsigned)__double_as_longlong(b.y), j, cn, vm);
}
template <>
__device__ __forceinline__ void load_geo<double, false>(const Sys &s, size_t slot, Vec3<double> &d, bool &cn, int &j,
                                                        unsigned &vm)
{
    const double2 *g = reinterpret_cast<const double2 *>(s.geo) + 2 * slot;
    const double2 a = g[0], b = g[1];
    d.x = a.x;
    d.y = a.y;
    d.z = b.x;
    untag(s, (unsigned)__double_as_longlong(b.y), j, cn, vm);
}

// i's position in the j < i part of j's Verlet row (rows are symmetric: the
// Verlet predicate is), four entries per load.  Run by the filter of the
// first step on new rows only; the later steps read the stored result.  The
// part searched holds plain indices (only entries j > i carry a position).
__device__ __forceinline__ unsigned mirror_position(const Sys &s, int j, int i)
{
    const int *rj = s.vnbr + (size_t)j * s.max_vnb;
    const int lo = s.vnh[j], hi = s.vnn[j];
    for (int b = lo & ~3; b < hi; b += 4) {
        const int4 v = *reinterpret_cast<const int4 *>(rj + b);
        if (v.x == i && b >= lo) return (unsigned)b;
        if (v.y == i && b + 1 >= lo && b + 1 < hi) return (unsigned)(b + 1);
        if (v.z == i && b + 2 >= lo && b + 2 < hi) return (unsigned)(b + 2);
        if (v.w == i && b + 3 >= lo && b + 3 < hi) return (unsigned)(b + 3);
    }
    set_err(s, kErrInternal);  // rows not symmetric: never expected
    return 0u;
}

// One exact entry for the gather passes: the neighbour and the switch
// weight side by side, read with one load.
template <typename real>
struct alignas(2 * sizeof(real)) JW {
    int j;
    real w;
};

template <typename real>
__device__ __forceinline__ int filter_row(const Sys &s, const AtomLane &a)
{
    const int vn = a.ok ? s.vnn[a.i] : 0;
    const int vh = a.ok ? s.vnh[a.i] : 0;
    const float4 pi = a.ok ? s.pos_s[a.i] : make_float4(0.f, 0.f, 0.f, 0.f);
    int *vrow = s.vnbr + (size_t)(a.ok ? a.i : 0) * s.max_vnb;
    int *row = s.nbr + (size_t)(a.ok ? a.i : 0) * s.max_nb;
    unsigned short *vround = s.vround + (s.mirror ? (size_t)(a.ok ? a.i : 0) * s.vround_stride : 0);
    // mirror slots: each Verlet entry j > i carries i's position in j's
    // Verlet row in its high bits (searched once on new rows, kept there for
    // the steps after, read with the entry), and each round records the exact
    // entries before it and its exact bits
    if (s.mirror && *s.rows_fresh) {
        for (int k = a.l; k < vh; k += kG) {
            const int j = vrow[k] & (int)kMirrorJ;
            vrow[k] = j | (int)(mirror_position(s, j, a.i) << kMirrorShift);
        }
        __syncwarp();
    }
    const unsigned lt = (1u << a.l) - 1u;
    const unsigned jmask = s.mirror ? kMirrorJ : 0xffffffffu;
    int cnt = 0, nh = 0;
    unsigned short rec = 0;  // lane r keeps round r's record (rounds below kG)
    // one pass: the Verlet row already has its j > i part first, so accepted
    // entries come out in the same order; nh counts those from that part
    const int vmax = __reduce_max_sync(0xffffffffu, vn);
    for (int base = 0; base < vmax; base += kG) {
        const int k = base + a.l;
        const bool valid = k < vn;
        const unsigned raw = valid ? (unsigned)vrow[k] : 0u;
        const int j = (int)(raw & jmask);
        const unsigned vm = (s.mirror && k < vh) ? raw >> kMirrorShift : 0u;
        const float4 pj = valid ? s.pos_s[j] : pi;
        const Vec3<float> d = displacement_warp(s, pi, pj);  // every lane: a warp vote inside
        const bool in = pair_in_warp(s, valid, pi, pj, d);
        const unsigned gm = group_mask_bits(__ballot_sync(0xffffffffu, in));
        const int below = min(max(vh - base, 0), kG);  // lanes of this round in the j > i part
        const int at = cnt + __popc(gm & lt);
        if (s.mirror) {  // only rounds that reach the j < i part are ever looked up
            const unsigned short r = (unsigned short)(min(cnt, 255) | (gm << 8));
            const int round = base / kG;
            if (round < kG) {
                if (a.l == round) rec = r;
            } else if (a.l == 0 && base < vn && base + kG > vh) {
                vround[round] = r;
            }
        }
        if (in && at < s.max_nb) {
            if (!s.mirror) row[at] = j;  // with mirror slots the exact entries' j live in their tags
            store_geo<real>(s, (size_t)a.i * s.max_nb + at, d, pi, pj, j, vm);
        }
        cnt += __popc(gm);
        nh += __popc(gm & ((1u << below) - 1u));
    }
    if (s.mirror && a.ok) {
        const int base = a.l * kG;
        if (base < vn && base + kG > vh) vround[a.l] = rec;
    }
    if (a.ok && a.l == 0) {
        if (cnt > s.max_nb) set_err(s, kErrCapacity);
        s.nn[a.i] = min(cnt, s.max_nb);
        s.nh[a.i] = min(nh, s.max_nb);
    }
    __syncwarp();
    return min(cnt, s.max_nb);
}

}  // namespace metad
