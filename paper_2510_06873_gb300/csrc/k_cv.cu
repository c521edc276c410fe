// Steps a4-a5 (CV forward) and a7-a8 (adjoint and bias forces).
//
// Per-atom definitions (sorted order i; N(i) the full neighbour list):
//   w_ij = s(r_ij)                 rational switch, stretched to vanish at rc
//   CN_i = sum_j w_ij [unlike]     s1 = (1/N) sum_i CN_i
//   W_i  = sum_j w_ij              q_m(i) = sum_j w_ij Y_m(rhat_ij) / W_i
//   qb_m(i) = (q_m(i) + sum_j w_ij q_m(j)) / (1 + W_i)
//   qb6(i)  = sqrt(4 pi / 13 sum_m qb_m(i)^2)     s2 = (1/N) sum_i qb6(i)
// (computed with unnormalised harmonics and weights K_m, see below)
// Adjoint (reverse mode, the paper's autograd written by hand):
//   b_m(i) = K_m qb_m(i) / (N qb6(i) (1 + W_i))                ds2/dA_m(i)
//   g_m(k) = b_m(k) + sum_i w_ik b_m(i)                        ds2/dq_m(k)
//   h_m(k) = g_m(k) / W_k                                      ds2/dQ_m(k)
//   gam_k  = h(k).q(k) + b(k).qb(k)                            -ds2/dW_k
//   per pair (i, j), d = r_j - r_i:
//     ds2/dw = (h_i + h_j).Y - gam_i - gam_j + b(i).q(j) + b(j).q(i)
//     ds2/dd = ds2/dw w'(r) d/r + w sum_m (h_m(i)+h_m(j)) dY_m/dd
//     ds1/dd = (2/N) w'(r) d/r [unlike]
//   F_i = sum_{j in N(i)} (V1 ds1/dd + V2 ds2/dd)
// The CV passes walk full rows (each atom gathers its own sums); the force
// evaluates each unordered pair once and gathers per atom in a fixed order:
// no floating-point atomics, bit-reproducible.
#include "metad_impl.cuh"

namespace metad {

// Real Y_6^m on the unit sphere, unnormalised: the pole-free associated-
// Legendre parts P_m(z) = d^m P_6 / dz^m (dyadic coefficients from the
// recurrence, exact in float32) times C_m, S_m, the real and imaginary parts
// of (x + i y)^m.  The normalisation enters only through the weights
//   K_0 = 1,  K_m = 2 (6-m)!/(6+m)!   (m > 0),
// with qbar6^2 = sum_m K_m (unnormalised qbar_m)^2 (the 4 pi / 13 of the
// Steinhardt definition cancels against the Y_6^m norms).  K_m is carried as
// a float pair so no rounded constant biases the CV.
// Layout: Y[0] m = 0; Y[2m-1] = P_m C_m; Y[2m] = P_m S_m, m = 1..6.
struct YlmConst {
    float pf[7][4];   // P_m(z) coefficients over z^2 powers (highest first)
    float dpf[7][4];  // dP_m/dz likewise
    double pd[7][4];
    double dpd[7][4];
    float kf_hi[kNY], kf_lo[kNY];  // K per Y slot
    double kd[kNY];
};
__constant__ YlmConst c_ylm;

template <typename real>
__device__ __forceinline__ real ylm_c(int m, int k);
template <>
__device__ __forceinline__ float ylm_c<float>(int m, int k) { return c_ylm.pf[m][k]; }
template <>
__device__ __forceinline__ double ylm_c<double>(int m, int k) { return c_ylm.pd[m][k]; }
template <typename real>
__device__ __forceinline__ real ylm_dc(int m, int k);
template <>
__device__ __forceinline__ float ylm_dc<float>(int m, int k) { return c_ylm.dpf[m][k]; }
template <>
__device__ __forceinline__ double ylm_dc<double>(int m, int k) { return c_ylm.dpd[m][k]; }

// P_m(z): degree 6 - m with the parity of 6 - m.
template <typename real>
__device__ __forceinline__ void legendre_parts(real z, real P[7])
{
#define C_(m, k) ylm_c<real>(m, k)
    real z2 = z * z;
    P[0] = ((C_(0, 0) * z2 + C_(0, 1)) * z2 + C_(0, 2)) * z2 + C_(0, 3);
    P[1] = z * ((C_(1, 0) * z2 + C_(1, 1)) * z2 + C_(1, 2));
    P[2] = (C_(2, 0) * z2 + C_(2, 1)) * z2 + C_(2, 2);
    P[3] = z * (C_(3, 0) * z2 + C_(3, 1));
    P[4] = C_(4, 0) * z2 + C_(4, 1);
    P[5] = z * C_(5, 0);
    P[6] = C_(6, 0);
#undef C_
}

template <typename real>
__device__ __forceinline__ void legendre_dparts(real z, real D[7])
{
#define C_(m, k) ylm_dc<real>(m, k)
    real z2 = z * z;
    D[0] = z * ((C_(0, 0) * z2 + C_(0, 1)) * z2 + C_(0, 2));
    D[1] = (C_(1, 0) * z2 + C_(1, 1)) * z2 + C_(1, 2);
    D[2] = z * (C_(2, 0) * z2 + C_(2, 1));
    D[3] = C_(3, 0) * z2 + C_(3, 1);
    D[4] = z * C_(4, 0);
    D[5] = C_(5, 0);
    D[6] = real(0);
#undef C_
}

template <typename real>
__device__ __forceinline__ void cs_powers(real x, real y, real C[7], real S[7])
{
    // (x + iy)^m; the first power written out (x 1 - y 0 is not folded to x
    // under IEEE rules: y 0 is not 0 for every y)
    C[0] = real(1);
    S[0] = real(0);
    C[1] = x;
    S[1] = y;
#pragma unroll
    for (int m = 2; m <= 6; ++m) {
        C[m] = x * C[m - 1] - y * S[m - 1];
        S[m] = x * S[m - 1] + y * C[m - 1];
    }
}

// v_k += w Y_k(u) for the 13 harmonics, w applied to the seven Legendre
// parts (seven products before the thirteen accumulations, where forming
// the harmonics first takes twelve).
template <typename real>
__device__ __forceinline__ void ylm13_acc(real x, real y, real z, real w, real v[kNY])
{
    real P[7], C[7], S[7];
    legendre_parts<real>(z, P);
    cs_powers<real>(x, y, C, S);
    v[0] += w * P[0];
#pragma unroll
    for (int m = 1; m <= 6; ++m) {
        const real wp = w * P[m];
        v[2 * m - 1] += wp * C[m];
        v[2 * m] += wp * S[m];
    }
}

// Y_k(u) and g = (I - u u^T) grad(sum_k c_k Y_k) / r.
template <typename real>
__device__ __forceinline__ void ylm13_grad(real x, real y, real z, real inv_r, const real c[kNY], real Y[kNY],
                                           real g[3])
{
    real P[7], D[7], C[7], S[7];
    legendre_parts<real>(z, P);
    legendre_dparts<real>(z, D);
    cs_powers<real>(x, y, C, S);
    Y[0] = P[0];
    real gx = real(0), gy = real(0), gz = c[0] * D[0];
#pragma unroll
    for (int m = 1; m <= 6; ++m) {
        real cc = c[2 * m - 1], cs = c[2 * m];
        Y[2 * m - 1] = P[m] * C[m];
        Y[2 * m] = P[m] * S[m];
        real pm = P[m] * real(m);
        gx += pm * (cc * C[m - 1] + cs * S[m - 1]);
        gy += pm * (cs * C[m - 1] - cc * S[m - 1]);
        gz += D[m] * (cc * C[m] + cs * S[m]);
    }
    real ug = x * gx + y * gy + z * gz;
    g[0] = (gx - ug * x) * inv_r;
    g[1] = (gy - ug * y) * inv_r;
    g[2] = (gz - ug * z) * inv_r;
}

// sum_k h_k Y_k(u) and g = (I - u u^T) grad(sum_k h_k Y_k) / r in one loop,
// without materialising the harmonics (fewer live registers in the pair pass).
template <typename real>
__device__ __forceinline__ real ylm13_dot_grad(real x, real y, real z, real inv_r, const real h[kNY], real g[3])
{
    real P[7], D[7], C[7], S[7];
    legendre_parts<real>(z, P);
    legendre_dparts<real>(z, D);
    cs_powers<real>(x, y, C, S);
    real t = h[0] * P[0];
    real gx = real(0), gy = real(0), gz = h[0] * D[0];
#pragma unroll
    for (int m = 1; m <= 6; ++m) {
        const real hc = h[2 * m - 1], hs = h[2 * m];
        t += hc * (P[m] * C[m]) + hs * (P[m] * S[m]);
        const real pm = P[m] * real(m);
        gx += pm * (hc * C[m - 1] + hs * S[m - 1]);
        gy += pm * (hs * C[m - 1] - hc * S[m - 1]);
        gz += D[m] * (hc * C[m] + hs * S[m]);
    }
    const real ug = x * gx + y * gy + z * gz;
    g[0] = (gx - ug * x) * inv_r;
    g[1] = (gy - ug * y) * inv_r;
    g[2] = (gz - ug * z) * inv_r;
    return t;
}

// sum_k K_k a_k^2 with K as a float pair (FP32) or exact (FP64).
template <typename real>
__device__ __forceinline__ real weighted_sq(const real a[kNY]);
template <>
__device__ __forceinline__ float weighted_sq<float>(const float a[kNY])
{
    float hi = 0.0f, lo = 0.0f;
#pragma unroll
    for (int m = 0; m < kNY; ++m) {
        float a2 = a[m] * a[m];
        hi = fmaf(c_ylm.kf_hi[m], a2, hi);
        lo = fmaf(c_ylm.kf_lo[m], a2, lo);
    }
    return hi + lo;
}
template <>
__device__ __forceinline__ double weighted_sq<double>(const double a[kNY])
{
    double s = 0.0;
#pragma unroll
    for (int m = 0; m < kNY; ++m) s += c_ylm.kd[m] * a[m] * a[m];
    return s;
}
template <typename real>
__device__ __forceinline__ real weighted_term(int m, real a);
template <>
__device__ __forceinline__ float weighted_term<float>(int m, float a)
{
    const float a2 = a * a;
    return fmaf(c_ylm.kf_lo[m], a2, c_ylm.kf_hi[m] * a2);
}
template <>
__device__ __forceinline__ double weighted_term<double>(int m, double a) { return c_ylm.kd[m] * a * a; }

template <typename real>
__device__ __forceinline__ real kweight(int m);
template <>
__device__ __forceinline__ float kweight<float>(int m) { return c_ylm.kf_hi[m]; }
template <>
__device__ __forceinline__ double kweight<double>(int m) { return c_ylm.kd[m]; }

// 16-wide per-atom records (13 used): one 64 B (FP32) or 128 B (FP64) row
// per atom, so a neighbour's record is two sectors, not thirteen.
constexpr int kRec = 16;

template <typename real>
__device__ __forceinline__ void load_rec(const real *base, int i, real v[kRec]);
template <>
__device__ __forceinline__ void load_rec<float>(const float *base, int i, float v[kRec])
{
    const float4 *p = reinterpret_cast<const float4 *>(base + (size_t)i * kRec);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float4 t = p[k];
        v[4 * k] = t.x;
        v[4 * k + 1] = t.y;
        v[4 * k + 2] = t.z;
        v[4 * k + 3] = t.w;
    }
}
template <>
__device__ __forceinline__ void load_rec<double>(const double *base, int i, double v[kRec])
{
    const double2 *p = reinterpret_cast<const double2 *>(base + (size_t)i * kRec);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        double2 t = p[k];
        v[2 * k] = t.x;
        v[2 * k + 1] = t.y;
    }
}
template <typename real>
__device__ __forceinline__ void store_rec(real *base, int i, const real v[kRec]);
template <>
__device__ __forceinline__ void store_rec<float>(float *base, int i, const float v[kRec])
{
    float4 *p = reinterpret_cast<float4 *>(base + (size_t)i * kRec);
#pragma unroll
    for (int k = 0; k < 4; ++k) p[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}
template <>
__device__ __forceinline__ void store_rec<double>(double *base, int i, const double v[kRec])
{
    double2 *p = reinterpret_cast<double2 *>(base + (size_t)i * kRec);
#pragma unroll
    for (int k = 0; k < 8; ++k) p[k] = make_double2(v[2 * k], v[2 * k + 1]);
}

namespace {

template <typename real>
__device__ __forceinline__ real *R(void *p) { return reinterpret_cast<real *>(p); }

// Fixed-order FP64 block sum (result valid in thread 0).
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    __syncthreads();
    return t;
}

// Displacement (cached by the exact filter), 1/r, switch weight and its
// derivative of one exact entry, with its neighbour, CN mask and mirror
// position.
template <typename real, bool kLast = false>
__device__ __forceinline__ void cached_geometry(const Sys &s, size_t slot, Vec3<real> &d, real &inv_r, real &w,
                                                real &dw, bool &cn, int &j, unsigned &vm)
{
    load_geo<real, kLast>(s, slot, d, cn, j, vm);
    real r2 = d.x * d.x + d.y * d.y + d.z * d.z;
    inv_r = rsqrt_r<real>(r2);
    switch_eval<real>(s, r2 * inv_r, w, dw);
}

// Butterfly reduce-scatter of 16 values over the kG lanes of a group:
// afterwards lane l holds the group sums of values 2l and 2l + 1 in v[0], v[1].
template <typename real>
__device__ __forceinline__ void reduce_scatter16(real v[kRec], int l)
{
    int len = kRec;
#pragma unroll
    for (int o = kG / 2; o >= 1; o >>= 1) {
        len >>= 1;
        const bool upper = (l & o) != 0;
#pragma unroll
        for (int t = 0; t < kRec / 2; ++t) {
            if (t < len) {
                real a = v[t], b = v[t + len];
                real send = upper ? a : b;
                real keep = upper ? b : a;
                v[t] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
    }
}

// Sum over the kG lanes of a group, result in every lane.
template <typename real>
__device__ __forceinline__ real group_sum(real v)
{
#pragma unroll
    for (int o = kG / 2; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename real>
__device__ __forceinline__ real group_get(real v, int src_lane)
{
    const int base = (threadIdx.x & 31) & ~(kG - 1);
    return __shfl_sync(0xffffffffu, v, base + src_lane);
}

template <typename real>
__device__ __forceinline__ void store_pair(real *base, int i, int l, real a, real b);
template <>
__device__ __forceinline__ void store_pair<float>(float *base, int i, int l, float a, float b)
{
    reinterpret_cast<float2 *>(base + (size_t)i * kRec)[l] = make_float2(a, b);
}
template <>
__device__ __forceinline__ void store_pair<double>(double *base, int i, int l, double a, double b)
{
    reinterpret_cast<double2 *>(base + (size_t)i * kRec)[l] = make_double2(a, b);
}

// Components (2l, 2l + 1) of record i: the kG lanes of a group together read
// the whole 64 B (FP32) row with one coalesced access.
template <typename real>
__device__ __forceinline__ void load_pair(const real *base, int i, int l, real &a, real &b);
template <>
__device__ __forceinline__ void load_pair<float>(const float *base, int i, int l, float &a, float &b)
{
    const float2 t = reinterpret_cast<const float2 *>(base + (size_t)i * kRec)[l];
    a = t.x;
    b = t.y;
}
template <>
__device__ __forceinline__ void load_pair<double>(const double *base, int i, int l, double &a, double &b)
{
    const double2 t = reinterpret_cast<const double2 *>(base + (size_t)i * kRec)[l];
    a = t.x;
    b = t.y;
}

__device__ __forceinline__ const int *nbr_row(const Sys &s, int i) { return s.nbr + (size_t)i * s.max_nb; }

// a4: CN_i, W_i and q_m(i) = sum_j w_ij Y_m(rhat_ij) / W_i.
// With kFilter the exact row is first compacted from the Verlet row.
template <typename real, bool kFilter>
__device__ __forceinline__ double cv_fwd_group(const Sys &s, const AtomLane a)
{
    int nn_f = 0;
    if (kFilter) nn_f = filter_row<real>(s, a);
    real v[kRec];  // 0..12: sum w Y_m ; 13: W ; 14: CN
#pragma unroll
    for (int m = 0; m < kRec; ++m) v[m] = real(0);
    if (a.ok) {
        const int nn = kFilter ? nn_f : s.nn[a.i];
        JW<real> *jwrow = reinterpret_cast<JW<real> *>(s.wl) + (size_t)a.i * s.max_nb;
        for (int k = a.l; k < nn; k += kG) {
            Vec3<real> d;
            real inv_r, w, dw;
            bool cn;
            int j;
            unsigned vm;
            cached_geometry<real>(s, (size_t)a.i * s.max_nb + k, d, inv_r, w, dw, cn, j, vm);
            jwrow[k] = JW<real>{j, w};
            if (cn) v[14] += w;
            v[13] += w;
            if (s.ncv == 2) ylm13_acc<real>(d.x * inv_r, d.y * inv_r, d.z * inv_r, w, v);
        }
    }
    reduce_scatter16<real>(v, a.l);
    // lane 6 holds (13: W, ...) in v[1]; lane 7 holds (14: CN, 15) in v[0]
    const real W = group_get<real>(v[1], 6);
    double cn_out = 0.0;
    if (a.ok) {
        if (a.l == 7) {
            R<real>(s.cn)[a.i] = v[0];
            cn_out = (double)v[0];
        }
        if (a.l == 6) R<real>(s.W)[a.i] = W;
        if (s.ncv == 2) {
            const real inv_W = W > real(0) ? real(1) / W : real(0);
            real q0 = v[0] * inv_W, q1 = v[1] * inv_W;
            if (a.l == 6) q1 = real(0);
            if (a.l == 7) q0 = q1 = real(0);
            store_pair<real>(R<real>(s.q), a.i, a.l, q0, q1);
        }
    }
    return cn_out;
}

template <typename real, bool kFilter>
__device__ __forceinline__ void cv_fwd(const Sys &s, Blk k)
{
    const int groups = group_grid(s.n);
    for (int it = 0, g; (g = work_item(k, it)) < groups; ++it) cv_fwd_group<real, kFilter>(s, atom_lane_at(s, g));
}

template <typename real, bool kFilter>
__global__ void __launch_bounds__(kBlockAtoms, 12) k_cv_fwd(Sys s) { cv_fwd<real, kFilter>(s, own_blk()); }

template <typename real>
__global__ void __launch_bounds__(kBlockAtoms, 12) kb_cv_fwd(BatchView v)
{
    Blk k;
    const Sys &s = v.sys[batch_system(v, k)];
    cv_fwd<real, true>(s, k);
}

// Per-thread running sum of a per-atom CV.  With FP32 records it is a
// compensated pair (Knuth's TwoSum: s + c holds the sum with only c's own
// rounding), so no FP64 instruction runs per atom (their pipe is narrow on
// this part); it enters the FP64 block and grid sums once per thread.
template <typename real>
struct RunSum;
template <>
struct RunSum<float> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float t = s + x;
        const float bp = t - s;
        c += (s - (t - bp)) + (x - bp);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
template <>
struct RunSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};

// Warp tree over RunSum values (lane 0 ends with the warp's sum): FP32
// pairs combine by TwoSum on s and a plain sum of the c terms.
__device__ __forceinline__ void warp_sum(RunSum<float> &v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float os = __shfl_down_sync(0xffffffffu, v.s, o);
        const float oc = __shfl_down_sync(0xffffffffu, v.c, o);
        const float t = v.s + os;
        const float bp = t - v.s;
        v.c += oc + ((v.s - (t - bp)) + (os - bp));
        v.s = t;
    }
}
__device__ __forceinline__ void warp_sum(RunSum<double> &v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v.s += __shfl_down_sync(0xffffffffu, v.s, o);
}

// Row entries k and k + 1 (k even, so k + 1 lies inside the row's capacity,
// a multiple of four entries; the caller uses the second only below the row
// length).  FP32 entries share one 16 B word (rows start on 32 B): one load,
// and for a lane group reading the same entries one L1 wavefront where two
// 8 B loads take two.  (Four entries in one 32 B load measured slower in
// the Q6 pass: 242 against 158 us at 1M atoms, its registers 32 -> 42.)
template <typename real>
__device__ __forceinline__ void load_jw2(const JW<real> *row, int k, JW<real> &e0, JW<real> &e1)
{
    e0 = row[k];
    e1 = row[k + 1];
}
template <>
__device__ __forceinline__ void load_jw2<float>(const JW<float> *row, int k, JW<float> &e0, JW<float> &e1)
{
    const int4 v = *reinterpret_cast<const int4 *>(row + k);
    e0 = JW<float>{v.x, __int_as_float(v.y)};
    e1 = JW<float>{v.z, __int_as_float(v.w)};
}

// a5: qbar_m(i), qbar6(i), s2.  Record b: b_m(i) = K_m qbar_m(i) / (N qbar6
// (1 + W_i)) (slots 0..12) and beta_i = b(i).qbar(i) (slot 13).
template <typename real>
__device__ __forceinline__ void cv_avg_group(const Sys &s, const AtomLane a, RunSum<real> &cn_sum,
                                             RunSum<real> &q6_sum)
{
    // lane l owns components 2l, 2l + 1 and walks every neighbour of the atom
    const real *q = R<real>(s.q);
    real a0 = real(0), a1 = real(0);
    if (a.ok) {
        const int nn = s.nn[a.i];
        const JW<real> *jwrow = reinterpret_cast<const JW<real> *>(s.wl) + (size_t)a.i * s.max_nb;
#pragma unroll 2
        for (int k = 0; k < nn; k += 2) {
            JW<real> e0, e1;
            load_jw2<real>(jwrow, k, e0, e1);
            const bool two = k + 1 < nn;
            real x0, x1, y0 = real(0), y1 = real(0);
            load_pair<real>(q, e0.j, a.l, x0, x1);
            if (two) load_pair<real>(q, e1.j, a.l, y0, y1);
            a0 += e0.w * x0;
            a1 += e0.w * x1;
            if (two) {
                a0 += e1.w * y0;
                a1 += e1.w * y1;
            }
        }
    }
    real qb0 = real(0), qb1 = real(0), sq = real(0), inv_D = real(0);
    if (a.ok) {
        inv_D = real(1) / (real(1) + R<real>(s.W)[a.i]);
        real o0, o1;
        load_pair<real>(q, a.i, a.l, o0, o1);
        const int m0 = 2 * a.l, m1 = 2 * a.l + 1;
        if (m0 < kNY) qb0 = (o0 + a0) * inv_D;
        if (m1 < kNY) qb1 = (o1 + a1) * inv_D;
        if (m0 < kNY) sq += weighted_term<real>(m0, qb0);
        if (m1 < kNY) sq += weighted_term<real>(m1, qb1);
    }
    sq = group_sum<real>(sq);
    const real qb6 = sqrt(sq);
    const real ci = qb6 > real(0) ? inv_D / (n_real<real>(s) * qb6) : real(0);
    const int m0 = 2 * a.l, m1 = 2 * a.l + 1;
    real b0 = m0 < kNY ? ci * kweight<real>(m0) * qb0 : real(0);
    real b1 = m1 < kNY ? ci * kweight<real>(m1) * qb1 : real(0);
    const real beta = group_sum<real>(b0 * qb0 + b1 * qb1);
    if (a.ok) {
        if (a.l == 6) b1 = beta;  // slot 13
        store_pair<real>(R<real>(s.b), a.i, a.l, b0, b1);
        if (a.l == 0) {
            R<real>(s.qb6)[a.i] = qb6;
            cn_sum.add(R<real>(s.cn)[a.i]);
            q6_sum.add(qb6);
        }
    }
}

// Block sums c, q -> part[b], part[part_stride + b]; the last block to finish
// adds them (thread t takes blocks t, t + blockDim, ... in order, then a
// fixed tree): s1 = C / N, s2 = Q / N.  A fixed association for a given grid.
__device__ void last_block_cv(const Sys &s, Blk k, double c, double q)
{
    __shared__ double sh[32];
    __shared__ bool am_last;
    if (k.nb > s.part_stride) {  // never with the grids used; refuse rather than overrun
        if (k.b == 0 && threadIdx.x == 0) set_err(s, kErrInternal);
        return;
    }
    c = block_sum(c, sh);
    q = block_sum(q, sh);
    double *pc = s.part, *pq = s.part + s.part_stride;
    if (threadIdx.x == 0) {
        pc[k.b] = c;
        pq[k.b] = q;
        __threadfence();
        am_last = atomicAdd(&s.ticket[0], 1u) == (unsigned)k.nb - 1u;
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double C = 0.0, Q = 0.0;
    for (int b = threadIdx.x; b < k.nb; b += blockDim.x) {
        C += __ldcg(pc + b);
        Q += __ldcg(pq + b);
    }
    C = block_sum(C, sh);
    Q = block_sum(Q, sh);
    if (threadIdx.x == 0) {
        s.scal[kS0] = C / s.n;
        if (s.ncv == 2) s.scal[kS1] = Q / s.n;
        else if (!s.lattice) s.scal[kS1] = 0.0;
        if (s.lattice)  // the triaxial lattice parameters follow the per-atom CVs
            for (int a = 0; a < 3; ++a) s.scal[kS0 + s.ncv + a] = s.L[a];
        s.ticket[0] = 0u;
    }
}

// a5 with the CV sums: persistent (the block partials are few).
// The filter of the last kernel saw the rows' mirror positions stored.
__device__ __forceinline__ void rows_used(const Sys &s, Blk k)
{
    if (k.b == 0 && threadIdx.x == 0 && s.mirror) *s.rows_fresh = 0;
}

template <typename real>
__device__ __forceinline__ void cv_avg(const Sys &s, Blk k)
{
    rows_used(s, k);
    RunSum<real> c, q;
    const int groups = group_grid(s.n);
    for (int it = 0, g; (g = work_item(k, it)) < groups; ++it) cv_avg_group<real>(s, atom_lane_at(s, g), c, q);
    last_block_cv(s, k, c.value(), q.value());
}

// The CV sum when there is no Q6 pass (n_cv == 1): thread t of block b sums
// the CN of atoms b kSumThreads + t, + blocks kSumThreads, ... in order
// (a compensated FP32 pair with FP32 records).
template <typename real>
__device__ __forceinline__ void cv_sum(const Sys &s, Blk k)
{
    rows_used(s, k);
    RunSum<real> c;
    const real *cn = R<real>(s.cn);
    for (int i = k.b * blockDim.x + threadIdx.x; i < s.n; i += k.nb * blockDim.x) c.add(cn[i]);
    last_block_cv(s, k, c.value(), 0.0);
}

template <typename real>
__global__ void __launch_bounds__(kSumThreads) k_cv_sum(Sys s) { cv_sum<real>(s, own_blk()); }

template <typename real>
__global__ void __launch_bounds__(kSumThreads) kb_cv_sum(BatchView v)
{
    Blk k;
    const Sys &s = v.sys[batch_system(v, k)];
    cv_sum<real>(s, k);
}

template <typename real>
__global__ void __launch_bounds__(kBlockAtoms) k_cv_avg(Sys s) { cv_avg<real>(s, own_blk()); }

template <typename real>
__global__ void __launch_bounds__(kBlockAtoms) kb_cv_avg(BatchView v)
{
    Blk k;
    const Sys &s = v.sys[batch_system(v, k)];
    cv_avg<real>(s, k);
}

// a7: g_m(k) = b_m(k) + sum_i w_ik b_m(i) ; h = g / W ; record h holds h_m
// (0..12) and gamma_k = h(k).q(k) + beta_k (slot 13).
// a7 with four lanes per atom, four record components per lane (one 16 B
// load of each neighbour record per lane): a warp has eight atoms' gathers in
// flight.  (Measured faster than eight lanes of two components here; the Q6
// average keeps eight lanes, where four cost it occupancy.)
constexpr int kG4 = 4;
constexpr int kAtoms4 = kBlockAtoms / kG4;

template <typename real>
__device__ __forceinline__ void load4(const real *base, int i, int l, real v[4]);
template <>
__device__ __forceinline__ void load4<float>(const float *base, int i, int l, float v[4])
{
    const float4 t = reinterpret_cast<const float4 *>(base + (size_t)i * kRec)[l];
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
}
template <>
__device__ __forceinline__ void load4<double>(const double *base, int i, int l, double v[4])
{
    const double2 *p = reinterpret_cast<const double2 *>(base + (size_t)i * kRec) + 2 * l;
    const double2 a = p[0], b = p[1];
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}
template <typename real>
__device__ __forceinline__ void store4(real *base, int i, int l, const real v[4]);
template <>
__device__ __forceinline__ void store4<float>(float *base, int i, int l, const float v[4])
{
    reinterpret_cast<float4 *>(base + (size_t)i * kRec)[l] = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void store4<double>(double *base, int i, int l, const double v[4])
{
    double2 *p = reinterpret_cast<double2 *>(base + (size_t)i * kRec) + 2 * l;
    p[0] = make_double2(v[0], v[1]);
    p[1] = make_double2(v[2], v[3]);
}

template <typename real>
__device__ __forceinline__ real group4_sum(real v)
{
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v;
}

// Reduce-scatter of four values over the four lanes of this thread's group:
// lane l returns the group sum of v[l].  The shuffle masks name the group
// alone, so groups of one warp may run different trip counts.
template <typename real>
__device__ __forceinline__ real group4_reduce_scatter(const real v[4], int l)
{
    const unsigned mask = 0xfu << (threadIdx.x & 28);
    const bool hi2 = (l & 2) != 0, hi1 = (l & 1) != 0;
    // lanes 2, 3 keep values 2, 3 and send 0, 1; lanes 0, 1 the reverse
    const real a0 = (hi2 ? v[2] : v[0]) + __shfl_xor_sync(mask, hi2 ? v[0] : v[2], 2);
    const real a1 = (hi2 ? v[3] : v[1]) + __shfl_xor_sync(mask, hi2 ? v[1] : v[3], 2);
    // odd lanes keep the second of their pair, even lanes the first
    return (hi1 ? a1 : a0) + __shfl_xor_sync(mask, hi1 ? a0 : a1, 1);
}

template <typename real>
__device__ __forceinline__ void adjoint_group(const Sys &s, int g)
{
    // lane l owns components 4l .. 4l + 3; record b holds b_m (0..12), beta (13)
    const int i = g * kAtoms4 + (threadIdx.x / kG4), l = threadIdx.x & (kG4 - 1);
    const bool ok = i < s.n;
    const real *bb = R<real>(s.b);
    real acc[4] = {real(0), real(0), real(0), real(0)};
    real o[4] = {real(0), real(0), real(0), real(0)}, q[4] = {real(0), real(0), real(0), real(0)};
    if (ok) {
        load4<real>(bb, i, l, o);
        load4<real>(R<real>(s.q), i, l, q);
        const int nn = s.nn[i];
        const JW<real> *jwrow = reinterpret_cast<const JW<real> *>(s.wl) + (size_t)i * s.max_nb;
        // with each gathered b_j also the half b_j.q_i of the pair's cross
        // term b_i.q_j + b_j.q_i in ds2/dw (a8), stored per entry: the force
        // pass adds the halves of entry ij and its mirror ji.  Entries go
        // four at a time; a reduce-scatter over the group leaves entry
        // k0 + l's sum in lane l, so the group stores 16 contiguous bytes.
        real *crow = R<real>(s.cross) + (size_t)i * s.max_nb;
        for (int k0 = 0; k0 < nn; k0 += 4) {
            JW<real> e4[4];
            load_jw2<real>(jwrow, k0, e4[0], e4[1]);
            load_jw2<real>(jwrow, k0 + 2, e4[2], e4[3]);
            real p[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                p[u] = real(0);
                if (k0 + u < nn) {
                    const JW<real> e = e4[u];
                    const real w = e.w;
                    real x[4];
                    load4<real>(bb, e.j, l, x);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        acc[c] += w * x[c];
                        if (4 * l + c < kNY) p[u] += x[c] * q[c];
                    }
                }
            }
            const real t = group4_reduce_scatter<real>(p, l);
            if (k0 + l < nn) crow[k0 + l] = t;
        }
    }
    real h[4] = {real(0), real(0), real(0), real(0)};
    real alpha = real(0), beta = real(0);
    if (ok) {
        const real W = R<real>(s.W)[i];
        const real inv_W = W > real(0) ? real(1) / W : real(0);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int m = 4 * l + c;
            if (m < kNY) {
                h[c] = (o[c] + acc[c]) * inv_W;
                alpha += h[c] * q[c];
            }
            if (m == 13) beta = o[c];
        }
    }
    alpha = group4_sum<real>(alpha);
    beta = group4_sum<real>(beta);
    if (ok) {
        if (l == 3) h[1] = alpha + beta;  // slot 13: gamma = h.q + b.qbar
        store4<real>(R<real>(s.h), i, l, h);
    }
}

template <typename real>
__device__ __forceinline__ void adjoint(const Sys &s, Blk k)
{
    const int groups = (s.n + kAtoms4 - 1) / kAtoms4;
    for (int it = 0, g; (g = work_item(k, it)) < groups; ++it) adjoint_group<real>(s, g);
}

// Resident blocks per SM the adjoint is compiled for: 12 in FP32 (40
// registers, no spill; measured 163 against 183 us at 1M atoms with the
// default 47 registers and 10 blocks), unconstrained in FP64.
template <typename real>
constexpr int kAdjointBlocks = sizeof(real) == 4 ? 12 : 0;

template <typename real>
__global__ void __launch_bounds__(kBlockAtoms, kAdjointBlocks<real>) k_adjoint(Sys s) { adjoint<real>(s, own_blk()); }

template <typename real>
__global__ void __launch_bounds__(kBlockAtoms, kAdjointBlocks<real>) kb_adjoint(BatchView v)
{
    Blk k;
    const Sys &s = v.sys[batch_system(v, k)];
    adjoint<real>(s, k);
}

// a8, pass 1: for every unordered pair, from the row of its lower index i
// (entries k < nh_i, j > i), G_ij = V1 ds1/dd + V2 ds2/dd at d = r_j - r_i,
// stored in the pair's slot.  Each pair is evaluated once.
//   ds2/dw = (h_i + h_j).Y - gamma_i - gamma_j + b_i.q_j + b_j.q_i
//   ds2/dd = ds2/dw w' d/r + w sum_m (h_i + h_j)_m dY_m/dd
//   ds1/dd = (2/N) w' d/r [unlike]
// The pair slots are a stream (written once, read once by pass 2): stored
// and loaded evict-first, so they leave the gathered records in L2.
template <typename real>
__device__ __forceinline__ void store_pair_force(real *slot, real fx, real fy, real fz);
template <>
__device__ __forceinline__ void store_pair_force<float>(float *slot, float fx, float fy, float fz)
{
    __stcs(reinterpret_cast<float4 *>(slot), make_float4(fx, fy, fz, 0.0f));
}
template <>
__device__ __forceinline__ void store_pair_force<double>(double *slot, double fx, double fy, double fz)
{
    __stcs(reinterpret_cast<double2 *>(slot), make_double2(fx, fy));
    __stcs(reinterpret_cast<double2 *>(slot) + 1, make_double2(fz, 0.0));
}

// Pair-parallel: the half-row entries (k < nh_i) of a chunk of kPairChunk
// atoms are numbered in atom order and thread t of the block evaluates
// entries t, t + blockDim, ...: every lane has a pair while the chunk lasts,
// whatever the spread of the atoms' half-row lengths.
//
// G_ij goes to the slot of entry k in i's row and -G_ij to the slot of i in
// the j < i part of j's row (rows are symmetric: the neighbour predicate is),
// so pass 2 sums each atom's own slots in row order.
constexpr int kPairChunk = 32;

template <typename real, bool kVir>
__device__ __forceinline__ void pair_force(const Sys &s, int i, int k, real cn_fac, real V2, RunSum<real> &vx,
                                           RunSum<real> &vy, RunSum<real> &vz)
{
    Vec3<real> d;
    real inv_r, w, dw;
    bool cn;
    int j;
    unsigned vm;
    cached_geometry<real, true>(s, (size_t)i * s.max_nb + k, d, inv_r, w, dw, cn, j, vm);
    // the slot of i in j's exact row: with mirror slots, the exact entries
    // of j's Verlet row before i's position vm there (one 2 B load);
    // otherwise a search of the j < i part [nh_j, nn_j) of j's row, four
    // entries per load
    int kk = -1;
    if (s.mirror) {
        const unsigned e = s.vround[(size_t)j * s.vround_stride + (vm >> 3)];
        kk = (int)(e & 0xffu) + __popc((e >> 8) & ((1u << (vm & 7u)) - 1u));
    } else {
        const int nhj = s.nh[j], nnj = s.nn[j];
        const int *rj = nbr_row(s, j);
        for (int b = nhj & ~3; b < nnj && kk < 0; b += 4) {
            const int4 v = *reinterpret_cast<const int4 *>(rj + b);
            if (v.x == i && b >= nhj) kk = b;
            else if (v.y == i && b + 1 >= nhj && b + 1 < nnj) kk = b + 1;
            else if (v.z == i && b + 2 >= nhj && b + 2 < nnj) kk = b + 2;
            else if (v.w == i && b + 3 >= nhj && b + 3 < nnj) kk = b + 3;
        }
    }
    if (kk < 0 || kk >= s.max_nb) {
        set_err(s, kErrInternal);  // rows not symmetric: never expected
        return;
    }
    const real ux = d.x * inv_r, uy = d.y * inv_r, uz = d.z * inv_r;
    real radial = cn ? cn_fac * dw : real(0);
    real fx = real(0), fy = real(0), fz = real(0);
    if (s.ncv == 2) {
        const real *hh = R<real>(s.h), *cc = R<real>(s.cross);
        // cross term b_i.q_j + b_j.q_i: the halves the adjoint pass stored
        // in entry ij (b_j.q_i) and in its mirror ji (b_i.q_j)
        real t = cc[(size_t)i * s.max_nb + k] + cc[(size_t)j * s.max_nb + kk];
        real hi[kRec], hj[kRec];
        load_rec<real>(hh, i, hi);
        load_rec<real>(hh, j, hj);
        t -= hi[13] + hj[13];
        real hs[kNY];
#pragma unroll
        for (int m = 0; m < kNY; ++m) hs[m] = hi[m] + hj[m];
        // (h_i + h_j).Y and its transverse gradient; the w Y term's gradient
        // is w times it
        real gY[3];
        t += ylm13_dot_grad<real>(ux, uy, uz, inv_r, hs, gY);
        radial += V2 * t * dw;
        const real vw = V2 * w;
        fx = vw * gY[0];
        fy = vw * gY[1];
        fz = vw * gY[2];
    }
    fx += radial * ux;
    fy += radial * uy;
    fz += radial * uz;
    if (kVir) {  // (dV/dd)_a d_a of this pair
        vx.add(fx * d.x);
        vy.add(fy * d.y);
        vz.add(fz * d.z);
    }
    real *pf = R<real>(s.pairF);
    store_pair_force<real>(pf + ((size_t)i * s.max_nb + k) * 4, fx, fy, fz);
    store_pair_force<real>(pf + ((size_t)j * s.max_nb + kk) * 4, -fx, -fy, -fz);
}

// The bias virial W_a = sum_pairs (dV/dd)_a d_a, which a barostat needs: it
// gives dV/dL_a at fixed fractional coordinates as W_a / L_a, plus dV/ds of
// a lattice CV.  Per-thread compensated sums, a warp tree, FP64 block
// partials in slot 1 of `part` (free once the CV sums are taken), and the
// last block to finish adds them in block order.
template <typename real>
__device__ void virial_finish(const Sys &s, Blk k, RunSum<real> &vx, RunSum<real> &vy, RunSum<real> &vz)
{
    constexpr int kW = kBlockAtoms / 32;
    __shared__ double sh[3][kW];
    __shared__ bool am_last;
    if (3 * k.nb > s.part_stride) {  // never with the grids used; refuse rather than overrun
        if (k.b == 0 && threadIdx.x == 0) set_err(s, kErrInternal);
        return;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    warp_sum(vx);
    warp_sum(vy);
    warp_sum(vz);
    if (lane == 0) {
        sh[0][wid] = vx.value();
        sh[1][wid] = vy.value();
        sh[2][wid] = vz.value();
    }
    __syncthreads();
    double *part = s.part + s.part_stride;
    if (threadIdx.x == 0) {
        for (int a = 0; a < 3; ++a) {
            double t = 0.0;
            for (int w = 0; w < kW; ++w) t += sh[a][w];
            part[3 * k.b + a] = t;
        }
        __threadfence();
        am_last = atomicAdd(&s.ticket[3], 1u) == (unsigned)k.nb - 1u;
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    // thread t adds partials t, t + blockDim, ... in order into four
    // interleaved accumulators (a short FP64 chain), combined in order
    double acc[3][4] = {};
    for (int b0 = threadIdx.x; b0 < k.nb; b0 += 4 * blockDim.x) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int b = b0 + r * blockDim.x;
            if (b < k.nb) {
#pragma unroll
                for (int a = 0; a < 3; ++a) acc[a][r] += __ldcg(part + 3 * b + a);
            }
        }
    }
    double v[3];
    for (int a = 0; a < 3; ++a) {
        v[a] = (acc[a][0] + acc[a][1]) + (acc[a][2] + acc[a][3]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[a] += __shfl_down_sync(0xffffffffu, v[a], o);
    }
    __syncthreads();
    if (lane == 0)
        for (int a = 0; a < 3; ++a) sh[a][wid] = v[a];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int a = 0; a < 3; ++a) {
            double t = 0.0;
            for (int w = 0; w < kW; ++w) t += sh[a][w];
            s.scal[kVir0 + a] = t;
            s.scal[kBoxG0 + a] = (s.lattice ? s.fscale * s.scal[kDV0 + s.ncv + a] : 0.0) + t / s.L[a];
        }
        s.ticket[3] = 0u;
    }
}

template <typename real, bool kVir>
__device__ __forceinline__ void force_pairs(const Sys &s, Blk k)
{
    // the chain-rule factors of the two CVs, once per block: an FP64 chain is
    // long and its pipe narrow on this part, so no thread repeats it
    __shared__ real fac[2];
    if (threadIdx.x == 0) {
        fac[0] = (real)(s.scal[kDV0] * s.fscale * 2.0 / s.n);
        fac[1] = s.ncv == 2 ? (real)(s.scal[kDV1] * s.fscale) : real(0);
    }
    __syncthreads();
    const real cn_fac = fac[0], V2 = fac[1];
    // each warp takes its own chunk of 32 atoms (a block of kBlockAtoms/32
    // warps is one work item, one per 128 atoms of the grid): no barrier
    constexpr int kWarps = kBlockAtoms / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int items = (s.n + kPairChunk * kWarps - 1) / (kPairChunk * kWarps);
    RunSum<real> vx, vy, vz;
    for (int it = 0, g; (g = work_item(k, it)) < items; ++it) {
        const int i0 = (g * kWarps + warp) * kPairChunk;
        if (i0 >= s.n) continue;  // warp-uniform
        // inclusive prefix of the half-row lengths, one lane per atom
        int off = i0 + lane < s.n ? s.nh[i0 + lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, off, o);
            if (lane >= o) off += y;
        }
        const int T = __shfl_sync(0xffffffffu, off, 31);
        for (int p0 = 0; p0 < T; p0 += 32) {
            const int p = p0 + lane;
            // the atom of entry p: the first a whose inclusive prefix exceeds p
            int lo = 0, hi = 31;
#pragma unroll
            for (int step = 0; step < 5; ++step) {
                const int mid = (lo + hi) >> 1;
                if (__shfl_sync(0xffffffffu, off, mid) > p) hi = mid;
                else lo = mid + 1;
            }
            const int prev = __shfl_sync(0xffffffffu, off, lo > 0 ? lo - 1 : 0);  // every lane shuffles
            const int start = lo > 0 ? prev : 0;
            if (p < T) pair_force<real, kVir>(s, i0 + lo, p - start, cn_fac, V2, vx, vy, vz);
        }
    }
    if (kVir) virial_finish<real>(s, k, vx, vy, vz);
}

template <typename real, bool kVir = false>
__global__ void __launch_bounds__(kBlockAtoms) k_force_pairs(Sys s) { force_pairs<real, kVir>(s, own_blk()); }

template <typename real, bool kVir = false>
__global__ void __launch_bounds__(kBlockAtoms) kb_force_pairs(BatchView v)
{
    Blk k;
    const Sys &s = v.sys[batch_system(v, k)];
    force_pairs<real, kVir>(s, k);
}

template <typename real>
__device__ __forceinline__ void load_pair_force(const real *slot, real &fx, real &fy, real &fz);
template <>
__device__ __forceinline__ void load_pair_force<float>(const float *slot, float &fx, float &fy, float &fz)
{
    const float4 t = __ldcs(reinterpret_cast<const float4 *>(slot));
    fx = t.x;
    fy = t.y;
    fz = t.z;
}
template <>
__device__ __forceinline__ void load_pair_force<double>(const double *slot, double &fx, double &fy, double &fz)
{
    const double2 a = __ldcs(reinterpret_cast<const double2 *>(slot));
    const double2 b = __ldcs(reinterpret_cast<const double2 *>(slot) + 1);
    fx = a.x;
    fy = a.y;
    fz = b.x;
}

// a8, pass 2: F_i = sum_{j > i} G_ij - sum_{j < i} G_ji: the slots of i's
// row hold exactly those terms (pass 1 wrote both ends of every pair), summed
// in row order per lane and a fixed shuffle tree across lanes: deterministic,
// no atomics, and contiguous reads.
template <typename real>
__device__ __forceinline__ void force_gather_group(const Sys &s, const AtomLane a, float *F, int accumulate)
{
    real fx = real(0), fy = real(0), fz = real(0);
    if (a.ok) {
        const int nn = s.nn[a.i];
        const real *pf = R<real>(s.pairF) + (size_t)a.i * s.max_nb * 4;
        for (int k = a.l; k < nn; k += kG) {
            real gx, gy, gz;
            load_pair_force<real>(pf + 4 * (size_t)k, gx, gy, gz);
            fx += gx;
            fy += gy;
            fz += gz;
        }
    }
    fx = group_sum<real>(fx);
    fy = group_sum<real>(fy);
    fz = group_sum<real>(fz);
    if (a.ok && a.l == 0) {
        float *o = F + 3 * (size_t)s.perm[a.i];
        if (accumulate) {
            o[0] += (float)fx;
            o[1] += (float)fy;
            o[2] += (float)fz;
        } else {
            o[0] = (float)fx;
            o[1] = (float)fy;
            o[2] = (float)fz;
        }
    }
}

template <typename real>
__device__ __forceinline__ void force_gather(const Sys &s, Blk k)
{
    const int groups = group_grid(s.n);
    for (int it = 0, g; (g = work_item(k, it)) < groups; ++it)
        force_gather_group<real>(s, atom_lane_at(s, g), s.F_out, s.accumulate);
}

template <typename real>
__global__ void __launch_bounds__(kBlockAtoms) k_force_gather(Sys s) { force_gather<real>(s, own_blk()); }

template <typename real>
__global__ void __launch_bounds__(kBlockAtoms) kb_force_gather(BatchView v)
{
    Blk k;
    const Sys &s = v.sys[batch_system(v, k)];
    force_gather<real>(s, k);
}

template <typename real>
__global__ void k_per_atom_out(Sys s, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const int u = s.perm[i];
    out[u] = (double)R<real>(s.cn)[i];
    if (s.ncv == 2) out[(size_t)s.n + u] = (double)R<real>(s.qb6)[i];
}


}  // namespace

void launch_cv_fwd(const Sys &s, int fp64, int fused_filter, cudaStream_t st)
{
    const int nb = group_grid(s.n);
    if (fp64) {
        if (fused_filter)
            k_cv_fwd<double, true><<<nb, kBlockAtoms, 0, st>>>(s);
        else
            k_cv_fwd<double, false><<<nb, kBlockAtoms, 0, st>>>(s);
    } else {
        if (fused_filter)
            k_cv_fwd<float, true><<<nb, kBlockAtoms, 0, st>>>(s);
        else
            k_cv_fwd<float, false><<<nb, kBlockAtoms, 0, st>>>(s);
    }
}

void launch_cv_avg(const Sys &s, int fp64, cudaStream_t st)
{
    if (fp64)
        k_cv_avg<double><<<grid_blocks(s, GK_CV, 0), kBlockAtoms, 0, st>>>(s);
    else
        k_cv_avg<float><<<grid_blocks(s, GK_CV, 0), kBlockAtoms, 0, st>>>(s);
}

void launch_cv_sum(const Sys &s, int fp64, cudaStream_t st)
{
    if (fp64)
        k_cv_sum<double><<<grid_blocks(s, GK_SUM, 0), kSumThreads, 0, st>>>(s);
    else
        k_cv_sum<float><<<grid_blocks(s, GK_SUM, 0), kSumThreads, 0, st>>>(s);
}

void launch_adjoint(const Sys &s, int fp64, cudaStream_t st)
{
    if (fp64)
        k_adjoint<double><<<grid_blocks(s, GK_ATOM32, 0), kBlockAtoms, 0, st>>>(s);
    else
        k_adjoint<float><<<grid_blocks(s, GK_ATOM32, 0), kBlockAtoms, 0, st>>>(s);
}

void launch_force_pairs(const Sys &s, int fp64, double scale, cudaStream_t st)
{
    Sys t = s;
    t.fscale = scale;
    const int nb = grid_blocks(s, GK_ATOM128, 0);
    if (fp64) {
        if (s.virial) k_force_pairs<double, true><<<nb, kBlockAtoms, 0, st>>>(t);
        else k_force_pairs<double><<<nb, kBlockAtoms, 0, st>>>(t);
    } else {
        if (s.virial) k_force_pairs<float, true><<<nb, kBlockAtoms, 0, st>>>(t);
        else k_force_pairs<float><<<nb, kBlockAtoms, 0, st>>>(t);
    }
}

void launch_force_gather(const Sys &s, int fp64, float *F, int accumulate, cudaStream_t st)
{
    Sys t = s;
    t.F_out = F;
    t.accumulate = accumulate;
    if (fp64)
        k_force_gather<double><<<group_grid(s.n), kBlockAtoms, 0, st>>>(t);
    else
        k_force_gather<float><<<group_grid(s.n), kBlockAtoms, 0, st>>>(t);
}

void launch_batch_cv(const BatchView &groups, int group_total, const BatchView &cv, int cv_total,
                     const BatchView &sums, int sum_total, int fp64, int ncv, cudaStream_t st)
{
    if (group_total <= 0) return;
    if (fp64) {
        kb_cv_fwd<double><<<group_total, kBlockAtoms, 0, st>>>(groups);
        if (ncv == 2)
            kb_cv_avg<double><<<cv_total, kBlockAtoms, 0, st>>>(cv);
        else
            kb_cv_sum<double><<<sum_total, kSumThreads, 0, st>>>(sums);
    } else {
        kb_cv_fwd<float><<<group_total, kBlockAtoms, 0, st>>>(groups);
        if (ncv == 2)
            kb_cv_avg<float><<<cv_total, kBlockAtoms, 0, st>>>(cv);
        else
            kb_cv_sum<float><<<sum_total, kSumThreads, 0, st>>>(sums);
    }
}

void launch_batch_force(const BatchView &groups, int group_total, const BatchView &adj, int adj_total,
                        const BatchView &pairs, int pair_total, int fp64, int ncv, int virial, cudaStream_t st,
                        int part)
{
    if (group_total <= 0) return;
    const bool adjoint = part != 2 && ncv == 2, forces = part != 1;
    if (fp64) {
        if (adjoint) kb_adjoint<double><<<adj_total, kBlockAtoms, 0, st>>>(adj);
        if (!forces) return;
        if (virial) kb_force_pairs<double, true><<<pair_total, kBlockAtoms, 0, st>>>(pairs);
        else kb_force_pairs<double><<<pair_total, kBlockAtoms, 0, st>>>(pairs);
        kb_force_gather<double><<<group_total, kBlockAtoms, 0, st>>>(groups);
    } else {
        if (adjoint) kb_adjoint<float><<<adj_total, kBlockAtoms, 0, st>>>(adj);
        if (!forces) return;
        if (virial) kb_force_pairs<float, true><<<pair_total, kBlockAtoms, 0, st>>>(pairs);
        else kb_force_pairs<float><<<pair_total, kBlockAtoms, 0, st>>>(pairs);
        kb_force_gather<float><<<group_total, kBlockAtoms, 0, st>>>(groups);
    }
}

// The gather kernels without shared memory prefer the SM's unified storage
// as L1.  (Kernels with even a small static shared array, the pair pass's
// two chain-rule factors among them, are left to the driver: a minimal
// shared carve-out caps how many of their blocks fit, 7 where the pair
// pass's registers allow 9.)
void configure_kernels()
{
    const int l1 = cudaSharedmemCarveoutMaxL1;
    cudaFuncSetAttribute(k_adjoint<float>, cudaFuncAttributePreferredSharedMemoryCarveout, l1);
    cudaFuncSetAttribute(k_force_gather<float>, cudaFuncAttributePreferredSharedMemoryCarveout, l1);
    cudaFuncSetAttribute(kb_adjoint<float>, cudaFuncAttributePreferredSharedMemoryCarveout, l1);
    cudaFuncSetAttribute(kb_force_gather<float>, cudaFuncAttributePreferredSharedMemoryCarveout, l1);
    cudaGetLastError();
}

void launch_per_atom_out(const Sys &s, int fp64, double *out, cudaStream_t st)
{
    if (fp64)
        k_per_atom_out<double><<<(s.n + 255) / 256, 256, 0, st>>>(s, out);
    else
        k_per_atom_out<float><<<(s.n + 255) / 256, 256, 0, st>>>(s, out);
}

// Polynomial parts from the associated-Legendre recurrence on coefficient
// arrays (pole-free, unnormalised):
//   P_m^m = (2m-1)!!,  P_{m+1}^m = (2m+1) z P_m^m,
//   P_l^m = ((2l-1) z P_{l-1}^m - (l+m-1) P_{l-2}^m) / (l-m);
// every coefficient is a dyadic rational, exact in float32.  Weights
// K_0 = 1, K_m = 2 (6-m)!/(6+m)!.
void set_ylm_constants(cudaStream_t st)
{
    YlmConst h{};
    const int l = 6;
    for (int m = 0; m <= l; ++m) {
        double prev2[8] = {0}, prev1[8] = {0}, cur[8] = {0};
        double dfact = 1.0;
        for (int k = 1; k <= 2 * m - 1; k += 2) dfact *= k;
        prev1[0] = dfact;
        if (m == l) {
            for (int p = 0; p < 8; ++p) cur[p] = prev1[p];
        } else {
            for (int p = 0; p < 7; ++p) cur[p + 1] = (2 * m + 1) * prev1[p];
            for (int ll = m + 2; ll <= l; ++ll) {
                for (int p = 0; p < 8; ++p) { prev2[p] = prev1[p]; prev1[p] = cur[p]; cur[p] = 0.0; }
                for (int p = 0; p < 7; ++p) cur[p + 1] += (2 * ll - 1) * prev1[p];
                for (int p = 0; p < 8; ++p) cur[p] -= (ll + m - 1) * prev2[p];
                for (int p = 0; p < 8; ++p) cur[p] /= (ll - m);
            }
        }
        const int deg = l - m;
        int t = 0;
        for (int p = deg; p >= 0; p -= 2, ++t) {
            h.pd[m][t] = cur[p];
            h.pf[m][t] = (float)cur[p];
        }
        t = 0;
        for (int p = deg; p >= 1; p -= 2, ++t) {
            h.dpd[m][t] = cur[p] * p;
            h.dpf[m][t] = (float)(cur[p] * p);
        }
        double fr = 1.0;  // (l-m)!/(l+m)!
        for (int k = l - m + 1; k <= l + m; ++k) fr /= k;
        const double K = m > 0 ? 2.0 * fr : 1.0;
        const int slots[2] = {m == 0 ? 0 : 2 * m - 1, m == 0 ? 0 : 2 * m};
        for (int q = 0; q < (m == 0 ? 1 : 2); ++q) {
            h.kd[slots[q]] = K;
            h.kf_hi[slots[q]] = (float)K;
            h.kf_lo[slots[q]] = (float)(K - (double)(float)K);
        }
    }
    cudaMemcpyToSymbolAsync(c_ylm, &h, sizeof(h), 0, cudaMemcpyHostToDevice, st);
}


// The kernels of this file whose only argument is the system descriptor
// (a captured step's nodes of these can take new I/O buffers in place).
bool sys_kernel_cv(const void *func)
{
    static const void *const kernels[] = {
        (const void *)k_cv_fwd<float, true>,
        (const void *)k_cv_fwd<float, false>,
        (const void *)k_cv_fwd<double, true>,
        (const void *)k_cv_fwd<double, false>,
        (const void *)k_cv_avg<float>,
        (const void *)k_cv_avg<double>,
        (const void *)k_cv_sum<float>,
        (const void *)k_cv_sum<double>,
        (const void *)k_adjoint<float>,
        (const void *)k_adjoint<double>,
        (const void *)k_force_pairs<float, false>,
        (const void *)k_force_pairs<float, true>,
        (const void *)k_force_pairs<double, false>,
        (const void *)k_force_pairs<double, true>,
        (const void *)k_force_gather<float>,
        (const void *)k_force_gather<double>,
    };
    for (const void *k : kernels)
        if (k == func) return true;
    return false;
}

}  // namespace metad
