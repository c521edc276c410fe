// Steps a3-a8 on spatial tiles: the exact neighbour rows with the CV
// forward pass (a3-a4), the local Q6 average with the CV sums (a5), the
// adjoint (a7) and the bias forces (a8).  One block per tile of cells; the
// tile's atoms and its one-cell shell are staged in shared memory
// (tiles.cuh), and every neighbour read of a pass comes from there.
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
// Force on atom i from its own row, every directed entry (no pair slots and
// no scatter; deterministic, no atomics), d = r_j - r_i, v_ij = w'(r) d / r:
//   F_i = V1 (2/N) sum_j [unlike] v_ij
//       + V2 sum_j { [(h_i + h_j).Y - gam_i - gam_j] v_ij + w grad_d((h_i + h_j).Y)
//                    + [b_i.q_j + b_j.q_i] v_ij }
// (V_d = dV/ds_d; F_i = sum_j dV/dd_ij).  The sums that need no dV/ds are
// taken by the passes that hold their records:
//   FC_i = sum_j [unlike] v_ij                     forward pass
//   FB_i = sum_m b_m(i) sum_j q_m(j) v_ij          Q6 pass (before b_i is known)
//        + sum_j (q_i.b_j) v_ij                    adjoint pass
// and the force pass adds V1 (2/N) FC_i + V2 FB_i to its own sum.
#include "tiles.cuh"

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

// This file is compiled without multiply-add contraction (-fmad=false):
// every fused multiply-add below is written out (fma_r), so the rounding of
// every expression is the one the source states, identical in every kernel
// that inlines it (single-system and batched launches, staged and unstaged
// tiles give the same bits).
template <typename real>
__device__ __forceinline__ real fma_r(real a, real b, real c);
template <>
__device__ __forceinline__ float fma_r<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <>
__device__ __forceinline__ double fma_r<double>(double a, double b, double c) { return fma(a, b, c); }

// P_m(z): degree 6 - m with the parity of 6 - m (Horner in z^2).
template <typename real>
__device__ __forceinline__ void legendre_parts(real z, real P[7])
{
#define C_(m, k) ylm_c<real>(m, k)
    const real z2 = z * z;
    P[0] = fma_r(fma_r(fma_r(C_(0, 0), z2, C_(0, 1)), z2, C_(0, 2)), z2, C_(0, 3));
    P[1] = z * fma_r(fma_r(C_(1, 0), z2, C_(1, 1)), z2, C_(1, 2));
    P[2] = fma_r(fma_r(C_(2, 0), z2, C_(2, 1)), z2, C_(2, 2));
    P[3] = z * fma_r(C_(3, 0), z2, C_(3, 1));
    P[4] = fma_r(C_(4, 0), z2, C_(4, 1));
    P[5] = z * C_(5, 0);
    P[6] = C_(6, 0);
#undef C_
}

template <typename real>
__device__ __forceinline__ void legendre_dparts(real z, real D[7])
{
#define C_(m, k) ylm_dc<real>(m, k)
    const real z2 = z * z;
    D[0] = z * fma_r(fma_r(C_(0, 0), z2, C_(0, 1)), z2, C_(0, 2));
    D[1] = fma_r(fma_r(C_(1, 0), z2, C_(1, 1)), z2, C_(1, 2));
    D[2] = z * fma_r(C_(2, 0), z2, C_(2, 1));
    D[3] = fma_r(C_(3, 0), z2, C_(3, 1));
    D[4] = z * C_(4, 0);
    D[5] = C_(5, 0);
    D[6] = real(0);
#undef C_
}

// C_m + i S_m = (x + i y)^m.
template <typename real>
__device__ __forceinline__ void cs_powers(real x, real y, real C[7], real S[7])
{
    C[0] = real(1);
    S[0] = real(0);
    C[1] = x;
    S[1] = y;
#pragma unroll
    for (int m = 2; m <= 6; ++m) {
        C[m] = fma_r(x, C[m - 1], -(y * S[m - 1]));
        S[m] = fma_r(x, S[m - 1], y * C[m - 1]);
    }
}

template <typename real>
__device__ __forceinline__ void ylm13(real x, real y, real z, real Y[kNY])
{
    real P[7], C[7], S[7];
    legendre_parts<real>(z, P);
    cs_powers<real>(x, y, C, S);
    Y[0] = P[0];
#pragma unroll
    for (int m = 1; m <= 6; ++m) {
        Y[2 * m - 1] = P[m] * C[m];
        Y[2 * m] = P[m] * S[m];
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
        const real cc = c[2 * m - 1], cs = c[2 * m];
        Y[2 * m - 1] = P[m] * C[m];
        Y[2 * m] = P[m] * S[m];
        const real pm = P[m] * real(m);
        gx = fma_r(pm, fma_r(cc, C[m - 1], cs * S[m - 1]), gx);
        gy = fma_r(pm, fma_r(cs, C[m - 1], -(cc * S[m - 1])), gy);
        gz = fma_r(D[m], fma_r(cc, C[m], cs * S[m]), gz);
    }
    const real ug = fma_r(x, gx, fma_r(y, gy, z * gz));
    g[0] = fma_r(-ug, x, gx) * inv_r;
    g[1] = fma_r(-ug, y, gy) * inv_r;
    g[2] = fma_r(-ug, z, gz) * inv_r;
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

namespace {

template <typename real>
__device__ __forceinline__ real *R(void *p) { return reinterpret_cast<real *>(p); }

// Four consecutive reals (16-byte aligned), and a store of four.
template <typename real>
__device__ __forceinline__ void ld4(const real *p, real x[4]);
template <>
__device__ __forceinline__ void ld4<float>(const float *p, float x[4])
{
    const float4 t = *reinterpret_cast<const float4 *>(p);
    x[0] = t.x;
    x[1] = t.y;
    x[2] = t.z;
    x[3] = t.w;
}
template <>
__device__ __forceinline__ void ld4<double>(const double *p, double x[4])
{
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    x[0] = a.x;
    x[1] = a.y;
    x[2] = b.x;
    x[3] = b.y;
}
template <typename real>
__device__ __forceinline__ void st4(real *p, real a, real b, real c, real d);
template <>
__device__ __forceinline__ void st4<float>(float *p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
template <>
__device__ __forceinline__ void st4<double>(double *p, double a, double b, double c, double d)
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2 *>(p)[1] = make_double2(c, d);
}

// Component c (0..3, not a compile-time constant) of a 4-array in registers,
// by selection (no local-memory indexing).
template <typename real>
__device__ __forceinline__ real quad_pick(const real v[4], int c)
{
    return c == 0 ? v[0] : (c == 1 ? v[1] : (c == 2 ? v[2] : v[3]));
}

// Displacement r_j - r_i in the pair precision.  The float32 form takes a
// warp vote: every lane of the warp must call it.
template <typename real>
__device__ __forceinline__ Vec3<real> pair_disp(const Sys &s, float4 pi, float4 pj);
template <>
__device__ __forceinline__ Vec3<float> pair_disp<float>(const Sys &s, float4 pi, float4 pj)
{
    return displacement_warp(s, pi, pj);
}
template <>
__device__ __forceinline__ Vec3<double> pair_disp<double>(const Sys &s, float4 pi, float4 pj)
{
    return displacement<double>(s, pi, pj);
}

// 1/r, the switch weight and its derivative of one displacement.
template <typename real>
__device__ __forceinline__ void pair_switch(const Sys &s, const Vec3<real> &d, real &inv_r, real &w, real &dw)
{
    const real r2 = fma_r(d.x, d.x, fma_r(d.y, d.y, d.z * d.z));
    inv_r = rsqrt_r<real>(r2);
    switch_eval<real>(s, r2 * inv_r, w, dw);
}

// The same quantities with the hardware's approximate reciprocal square root
// and reciprocal (relative error ~1e-7, not correctly rounded): for the force
// pass, whose results are derivatives (the CV values, whose rounding must be
// unbiased, use pair_switch).  FP64 keeps the exact form.
template <typename real>
__device__ __forceinline__ void pair_switch_fast(const Sys &s, const Vec3<real> &d, real &inv_r, real &w, real &dw);
template <>
__device__ __forceinline__ void pair_switch_fast<double>(const Sys &s, const Vec3<double> &d, double &inv_r, double &w,
                                                         double &dw)
{
    pair_switch<double>(s, d, inv_r, w, dw);
}
template <>
__device__ __forceinline__ void pair_switch_fast<float>(const Sys &s, const Vec3<float> &d, float &inv_r, float &w,
                                                        float &dw)
{
    const float r2 = fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z));
    inv_r = rsqrtf(r2);
    const float x = (r2 * inv_r) * s.inv_r0_hi;
    float f, dfdx;
    if (s.sw_m == 2 * s.sw_n) {
        const float xn1 = s.sw_n == 6 ? (x * x) * (x * x) * x : ipow<float>(x, s.sw_n - 1);
        const float inv = __fdividef(1.0f, fmaf(xn1, x, 1.0f));
        f = inv;
        dfdx = -s.sw_nf * xn1 * inv * inv;
    } else {
        float Sn, dSn, Sm, dSm;
        geom_sum<float>(x, s.sw_n, Sn, dSn);
        geom_sum<float>(x, s.sw_m, Sm, dSm);
        const float inv = __fdividef(1.0f, Sm);
        f = Sn * inv;
        dfdx = (dSn * Sm - Sn * dSm) * inv * inv;
    }
    w = fmaf(f, s.a_hi, -s.k_hi);
    dw = dfdx * s.a_hi * s.inv_r0_hi;
}

// Where a pass reads the tile's atoms: shared memory, or, for a tile larger
// than the staging capacity, global memory through the same local indices
// (the same values, so the same bits).
template <typename real, bool kStaged>
struct Src {
    const TileTable &T;
    const float4 *spos;  // staged positions
    const real *srec;    // staged record components 0..11
    const real *spair;   // staged record components 12..13
    const float4 *gpos;  // sorted positions (global)
    const real *grec;    // records [n][16] (global)

    __device__ __forceinline__ float4 pos(int a) const { return kStaged ? spos[a] : gpos[tile_global(T, a)]; }
    // record components 4l .. 4l + 3 (l < 3), or component 12 then zeros (l == 3)
    __device__ __forceinline__ void quad(int a, int l, real x[4]) const
    {
        if (kStaged) {
            if (l < 3) {
                ld4<real>(srec + (size_t)a * kRecQ + 4 * l, x);
            } else {
                x[0] = spair[2 * (size_t)a];
                x[1] = x[2] = x[3] = real(0);
            }
        } else {
            const real *r = grec + (size_t)tile_global(T, a) * 16;
            if (l < 3) {
                ld4<real>(r + 4 * l, x);
            } else {
                x[0] = r[12];
                x[1] = x[2] = x[3] = real(0);
            }
        }
    }
    // record component 13
    __device__ __forceinline__ real c13(int a) const
    {
        return kStaged ? spair[2 * (size_t)a + 1] : grec[(size_t)tile_global(T, a) * 16 + 13];
    }
    // record components 0..13
    __device__ __forceinline__ void all(int a, real x[14]) const
    {
        const real *r = kStaged ? srec + (size_t)a * kRecQ : grec + (size_t)tile_global(T, a) * 16;
        ld4<real>(r, x);
        ld4<real>(r + 4, x + 4);
        ld4<real>(r + 8, x + 8);
        if (kStaged) {
            x[12] = spair[2 * (size_t)a];
            x[13] = spair[2 * (size_t)a + 1];
        } else {
            x[12] = r[12];
            x[13] = r[13];
        }
    }
};

// Per-thread running sum of a per-atom value.  With FP32 records it is a
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

// The bias virial W_a = sum_pairs (dV/dd)_a d_a, which a barostat needs: it
// gives dV/dL_a at fixed fractional coordinates as W_a / L_a, plus dV/ds of
// a lattice CV.  Per-thread compensated sums, a warp tree, FP64 block
// partials in slot 1 of `part` (free once the CV sums are taken), and the
// last block to finish adds them in block order.
template <typename real>
__device__ void virial_finish(const Sys &s, Blk k, RunSum<real> &vx, RunSum<real> &vy, RunSum<real> &vz)
{
    constexpr int kW = kTileThreads / 32;
    __shared__ double sh[3][kW];
    __shared__ bool am_last;
    if (3 * k.nb > s.part_stride) {  // never with the grids used; refuse rather than overrun
        if (k.b == 0 && threadIdx.x == 0) set_err(s, kErrInternal);
        return;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double v3[3] = {vx.value(), vy.value(), vz.value()};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v3[a] += __shfl_down_sync(0xffffffffu, v3[a], o);
    if (lane == 0)
        for (int a = 0; a < 3; ++a) sh[a][wid] = v3[a];
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

template <typename real>
__device__ __forceinline__ real group4_sum(real v)
{
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v;
}

constexpr int kGroups4 = kTileThreads / 4;  // atoms a block's 4-lane groups take at once

// Per-entry scalars in quad-major order, like the rows: entries 4q .. 4q + 3
// of atom i are four reals at [q][i].
template <typename real>
__device__ __forceinline__ real *quad_real(void *base, size_t n, int q, int i)
{
    return reinterpret_cast<real *>(base) + (((size_t)q * n + i) << 2);
}


// ------------------------------------------------------------------ a3-a4
// The exact rows of the tile's atoms from their Verlet rows (r^2 < rc^2,
// decided as the FP64 definition), kept in shared memory (slist, a column
// per thread) and stored as the step's neighbour rows; then (kCompute) CN_i,
// W_i, q_m(i) and FC_i.  One thread per atom; the rows are read four
// entries (one 8-byte quad) at a time, the next quad loaded before the
// current one is used.
template <typename real, bool kStaged, bool kCompute, bool kVir>
__device__ __forceinline__ void fwd_tile(const Sys &s, const TileTable &T, const Src<real, kStaged> &src,
                                         unsigned short *slist, RunSum<real> &cn_sum)
{
    const size_t N = (size_t)s.n;
    const int lane = threadIdx.x & 31;
    const ushort4 none = make_ushort4(0, 0, 0, 0);
    for (int a0 = threadIdx.x & ~31; a0 < T.n_own; a0 += kTileThreads) {
        const int a = a0 + lane;
        const bool ok = a < T.n_own;
        const int i = T.atom0 + (ok ? a : 0);
        const float4 pi = ok ? src.pos(a) : make_float4(0.f, 0.f, 0.f, 0.f);
        const int vn = ok ? s.vnn[i] : 0;
        const int qmax = __reduce_max_sync(0xffffffffu, (vn + 3) >> 2);
        int cnt = 0;
        ushort4 nxt = vn > 0 ? quad_at(s.vlist, N, 0, i) : none;
        for (int q = 0; q < qmax; ++q) {
            const ushort4 cur = nxt;
            if (q + 1 < qmax) nxt = 4 * (q + 1) < vn ? quad_at(s.vlist, N, q + 1, i) : none;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                int jl = quad_get(cur, c);
                const bool valid = 4 * q + c < vn && jl < T.total;  // rows hold staged atoms only
                jl = valid ? jl : 0;
                const float4 pj = valid ? src.pos(jl) : pi;
                const Vec3<float> d = displacement_warp(s, pi, pj);  // every lane: a warp vote inside
                if (valid && pair_in(s, pi, pj, d)) {
                    if (cnt < s.max_nb) slist[cnt * kTileThreads + threadIdx.x] = (unsigned short)jl;
                    ++cnt;
                }
            }
        }
        const int nn = min(cnt, s.max_nb);
        if (ok) {
            if (cnt > s.max_nb) set_err(s, kErrCapacity);
            s.nn[i] = nn;
            // the exact row, quad by quad (threads of a warp own consecutive
            // atoms: each quad row is one contiguous store per warp)
            for (int q = 0; 4 * q < nn; ++q) {
                const unsigned short *col = slist + 4 * q * kTileThreads + threadIdx.x;
                const int m = nn - 4 * q;  // entries of this quad in the row (the rest are 0)
                quad_ref(s.elist, N, q, i) =
                    make_ushort4(col[0], m > 1 ? col[kTileThreads] : 0, m > 2 ? col[2 * kTileThreads] : 0,
                                 m > 3 ? col[3 * kTileThreads] : 0);
            }
        }
        if (!kCompute) continue;
        const int nmax = __reduce_max_sync(0xffffffffu, nn);
        real Q[kNY];
#pragma unroll
        for (int m = 0; m < kNY; ++m) Q[m] = real(0);
        real W = real(0), CN = real(0);
        real f3[3] = {real(0), real(0), real(0)}, w3[3] = {real(0), real(0), real(0)};
        for (int k0 = 0; k0 < nmax; k0 += 4) {
            // a quad of entries, unrolled and predicated (an entry past the
            // row is evaluated at a dummy displacement and not added)
            real wq[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int k = k0 + c;
                const bool valid = k < nn;
                const int jl = valid ? (int)slist[k * kTileThreads + threadIdx.x] : 0;
                const float4 pj = valid ? src.pos(jl) : pi;
                Vec3<real> d = pair_disp<real>(s, pi, pj);
                if (!valid) {
                    d.x = real(s.r0);
                    d.y = d.z = real(0);
                }
                real inv_r, w, dw;
                pair_switch<real>(s, d, inv_r, w, dw);
                w = valid ? w : real(0);
                wq[c] = w;
                W += w;
                const bool cn = valid && (!s.cn_unlike || pj.w != pi.w);
                CN += cn ? w : real(0);
                const real f = cn ? dw * inv_r : real(0);
                f3[0] = fma_r(f, d.x, f3[0]);
                f3[1] = fma_r(f, d.y, f3[1]);
                f3[2] = fma_r(f, d.z, f3[2]);
                if (kVir) {
                    w3[0] = fma_r(f * d.x, d.x, w3[0]);
                    w3[1] = fma_r(f * d.y, d.y, w3[1]);
                    w3[2] = fma_r(f * d.z, d.z, w3[2]);
                }
                if (s.ncv == 2) {
                    real Y[kNY];
                    ylm13<real>(d.x * inv_r, d.y * inv_r, d.z * inv_r, Y);
#pragma unroll
                    for (int m = 0; m < kNY; ++m) Q[m] = fma_r(w, Y[m], Q[m]);
                }
            }
            // the quad's weights, for the passes that need w_ij without the
            // geometry (entries past the row are 0)
            if (s.ncv == 2 && k0 < nn) st4<real>(quad_real<real>(s.wl, N, k0 >> 2, i), wq[0], wq[1], wq[2], wq[3]);
        }
        if (!ok) continue;
        real *rq = R<real>(s.rq) + (size_t)i * 16;
        real q12 = real(0);
        if (s.ncv == 2) {
            const real inv_W = W > real(0) ? real(1) / W : real(0);
            st4<real>(rq, Q[0] * inv_W, Q[1] * inv_W, Q[2] * inv_W, Q[3] * inv_W);
            st4<real>(rq + 4, Q[4] * inv_W, Q[5] * inv_W, Q[6] * inv_W, Q[7] * inv_W);
            st4<real>(rq + 8, Q[8] * inv_W, Q[9] * inv_W, Q[10] * inv_W, Q[11] * inv_W);
            q12 = Q[12] * inv_W;
        }
        st4<real>(rq + 12, q12, W, CN, real(0));
        st4<real>(R<real>(s.fc) + 4 * (size_t)i, f3[0], f3[1], f3[2], real(0));
        if (kVir) st4<real>(R<real>(s.wc) + 4 * (size_t)i, w3[0], w3[1], w3[2], real(0));
        cn_sum.add(CN);
    }
}

// Where the Q6 and adjoint passes read an own atom's row quads and weights:
// the tile's staged copy, or global memory.
template <typename real, bool kStaged>
struct RowSrc {
    const OwnRows<real> &o;
    const unsigned short *elist;
    void *wl;
    size_t n;
    int atom0;
    __device__ __forceinline__ ushort4 jq(int a, int q) const
    {
        return kStaged ? o.jq[o.qoff[a] + q] : quad_at(elist, n, q, atom0 + a);
    }
    __device__ __forceinline__ void w(int a, int q, real x[4]) const
    {
        ld4<real>(kStaged ? o.wq + 4 * (o.qoff[a] + q) : quad_real<real>(wl, n, q, atom0 + a), x);
    }
};

// ------------------------------------------------------------------ a5
// qbar_m(i), qbar6(i), the CV sums, record b (b_m(i) in 0..12, beta_i =
// b(i).qbar(i) in 13, qbar6 in 14), and per entry e_ij = b_i.q_j (the half
// of the cross term b_i.q_j + b_j.q_i this pass can form).  One thread per
// atom: each neighbour's 13 q components from shared memory, the entry's
// weight w_ij from the forward pass (no geometry here), rows a quad at a
// time.
template <typename real, bool kStaged>
__device__ __forceinline__ void avg_tile(const Sys &s, const TileTable &T, const Src<real, kStaged> &src,
                                         const RowSrc<real, kStaged> &rows, RunSum<real> &cn_sum,
                                         RunSum<real> &q6_sum)
{
    const size_t N = (size_t)s.n;
    for (int a = threadIdx.x; a < T.n_own; a += kTileThreads) {
        const int i = T.atom0 + a;
        const int nn = s.nn[i];
        real A[kNY];
#pragma unroll
        for (int m = 0; m < kNY; ++m) A[m] = real(0);
        for (int q = 0; 4 * q < nn; ++q) {
            const ushort4 jq = rows.jq(a, q);
            real wq[4];
            rows.w(a, q, wq);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (4 * q + e < nn) {
                    real x[14];
                    src.all(quad_get(jq, e), x);
#pragma unroll
                    for (int m = 0; m < kNY; ++m) A[m] = fma_r(wq[e], x[m], A[m]);
                }
            }
        }
        real qo[16];
        const real *rq = R<real>(s.rq) + (size_t)i * 16;
#pragma unroll
        for (int u = 0; u < 4; ++u) ld4<real>(rq + 4 * u, qo + 4 * u);
        const real W = qo[13], CN = qo[14];
        const real inv_D = real(1) / (real(1) + W);
        real qb[kNY], sq = real(0);
#pragma unroll
        for (int m = 0; m < kNY; ++m) {
            qb[m] = (qo[m] + A[m]) * inv_D;
            sq += weighted_term<real>(m, qb[m]);
        }
        const real qb6 = sqrt(sq);
        const real ci = qb6 > real(0) ? inv_D / (n_real<real>(s) * qb6) : real(0);
        real b[kNY], beta = real(0);
#pragma unroll
        for (int m = 0; m < kNY; ++m) {
            b[m] = ci * kweight<real>(m) * qb[m];
            beta = fma_r(b[m], qb[m], beta);
        }
        // e_ij = b_i.q_j for every entry, a quad at a time
        for (int q = 0; 4 * q < nn; ++q) {
            const ushort4 jq = rows.jq(a, q);
            real eo[4] = {real(0), real(0), real(0), real(0)};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (4 * q + e < nn) {
                    real x[14];
                    src.all(quad_get(jq, e), x);
                    real p = b[0] * x[0];
#pragma unroll
                    for (int m = 1; m < kNY; ++m) p = fma_r(b[m], x[m], p);
                    eo[e] = p;
                }
            }
            st4<real>(quad_real<real>(s.eq, N, q, i), eo[0], eo[1], eo[2], eo[3]);
        }
        real *rb = R<real>(s.rb) + (size_t)i * 16;
        st4<real>(rb, b[0], b[1], b[2], b[3]);
        st4<real>(rb + 4, b[4], b[5], b[6], b[7]);
        st4<real>(rb + 8, b[8], b[9], b[10], b[11]);
        st4<real>(rb + 12, b[12], beta, qb6, real(0));
        cn_sum.add(CN);
        q6_sum.add(qb6);
    }
}

// ------------------------------------------------------------------ a7
// g_m(k) = b_m(k) + sum_i w_ik b_m(i), h = g / W, record h (h_m in 0..12,
// gamma_k = h(k).q(k) + beta_k in 13), and per entry the other half of the
// cross term, d_ki = q_k.b_i.  One thread per atom as in the Q6 pass.
template <typename real, bool kStaged>
__device__ __forceinline__ void adj_tile(const Sys &s, const TileTable &T, const Src<real, kStaged> &src,
                                         const RowSrc<real, kStaged> &rows)
{
    const size_t N = (size_t)s.n;
    for (int a = threadIdx.x; a < T.n_own; a += kTileThreads) {
        const int i = T.atom0 + a;
        const int nn = s.nn[i];
        real qi[16];
        const real *rq = R<real>(s.rq) + (size_t)i * 16;
#pragma unroll
        for (int u = 0; u < 4; ++u) ld4<real>(rq + 4 * u, qi + 4 * u);
        real acc[kNY];
#pragma unroll
        for (int m = 0; m < kNY; ++m) acc[m] = real(0);
        for (int q = 0; 4 * q < nn; ++q) {
            const ushort4 jq = rows.jq(a, q);
            real wq[4], dout[4] = {real(0), real(0), real(0), real(0)};
            rows.w(a, q, wq);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (4 * q + e < nn) {
                    real x[14];
                    src.all(quad_get(jq, e), x);
                    real p = qi[0] * x[0];
#pragma unroll
                    for (int m = 0; m < kNY; ++m) {
                        acc[m] = fma_r(wq[e], x[m], acc[m]);
                        if (m > 0) p = fma_r(qi[m], x[m], p);
                    }
                    dout[e] = p;
                }
            }
            st4<real>(quad_real<real>(s.dq, N, q, i), dout[0], dout[1], dout[2], dout[3]);
        }
        real bo[14];
        src.all(a, bo);
        const real W = qi[13];
        const real inv_W = W > real(0) ? real(1) / W : real(0);
        real h[kNY], alpha = real(0);
#pragma unroll
        for (int m = 0; m < kNY; ++m) {
            h[m] = (bo[m] + acc[m]) * inv_W;
            alpha = fma_r(h[m], qi[m], alpha);
        }
        real *rh = R<real>(s.rh) + (size_t)i * 16;
        st4<real>(rh, h[0], h[1], h[2], h[3]);
        st4<real>(rh + 4, h[4], h[5], h[6], h[7]);
        st4<real>(rh + 8, h[8], h[9], h[10], h[11]);
        st4<real>(rh + 12, h[12], alpha + bo[13], real(0), real(0));
    }
}

// ------------------------------------------------------------------ a8
// F_i = V1 (2/N) FC_i + V2 sum_j { [(h_i + h_j).Y - gam_i - gam_j + c_ij]
// v_ij + w grad_d((h_i + h_j).Y) }, written in the caller's order.  One
// thread per atom; the neighbour's h record (14 components) and position
// come from shared memory, the row and its cross terms a quad at a time
// (the next quad loaded ahead).  With kVir each thread also sums the bias
// virial of its atom's entries (every pair appears in both rows: half of
// it).
template <typename real, bool kStaged, bool kVir>
__device__ __forceinline__ void force_tile(const Sys &s, const TileTable &T, const Src<real, kStaged> &src,
                                           real cn_fac, real V2, RunSum<real> vir[3])
{
    const size_t N = (size_t)s.n;
    const int lane = threadIdx.x & 31;
    const ushort4 none = make_ushort4(0, 0, 0, 0);
    for (int a0 = threadIdx.x & ~31; a0 < T.n_own; a0 += kTileThreads) {
        const int a = a0 + lane;
        const bool ok = a < T.n_own;
        const int i = T.atom0 + (ok ? a : 0);
        const float4 pi = ok ? src.pos(a) : make_float4(0.f, 0.f, 0.f, 0.f);
        real hi[14];
        src.all(ok ? a : 0, hi);
        const int nn = ok ? s.nn[i] : 0;
        const int qmax = __reduce_max_sync(0xffffffffu, (nn + 3) >> 2);
        real F[3] = {real(0), real(0), real(0)}, Wv[3] = {real(0), real(0), real(0)};
        ushort4 nxt = nn > 0 ? quad_at(s.elist, N, 0, i) : none;
        for (int q = 0; q < qmax; ++q) {
            const ushort4 cur = nxt;
            if (q + 1 < qmax) nxt = 4 * (q + 1) < nn ? quad_at(s.elist, N, q + 1, i) : none;
            real cq[4] = {real(0), real(0), real(0), real(0)};
            if (4 * q < nn) {  // the cross terms c = b_i.q_j + b_j.q_i of the quad
                real dq[4];
                ld4<real>(quad_real<real>(s.eq, N, q, i), cq);
                ld4<real>(quad_real<real>(s.dq, N, q, i), dq);
#pragma unroll
                for (int c = 0; c < 4; ++c) cq[c] += dq[c];
            }
            // the quad's four entries, unrolled and predicated (an entry past
            // the row is evaluated at a dummy displacement and not added)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const bool valid = 4 * q + c < nn;
                const int jl = valid ? quad_get(cur, c) : 0;
                const float4 pj = valid ? src.pos(jl) : pi;
                Vec3<real> d = pair_disp<real>(s, pi, pj);
                if (!valid) {
                    d.x = real(s.r0);
                    d.y = d.z = real(0);
                }
                real inv_r, w, dw;
                pair_switch_fast<real>(s, d, inv_r, w, dw);
                real hj[14];
                src.all(jl, hj);
                const real ux = d.x * inv_r, uy = d.y * inv_r, uz = d.z * inv_r;
                real hs[kNY], cvec[kNY];
#pragma unroll
                for (int m = 0; m < kNY; ++m) {
                    hs[m] = hi[m] + hj[m];
                    cvec[m] = w * hs[m];
                }
                real Y[kNY], gY[3];
                ylm13_grad<real>(ux, uy, uz, inv_r, cvec, Y, gY);
                real t = cq[c] - (hi[13] + hj[13]);
#pragma unroll
                for (int m = 0; m < kNY; ++m) t = fma_r(hs[m], Y[m], t);
                const real radial = valid ? V2 * t * dw : real(0);
                const real V2v = valid ? V2 : real(0);
                const real G[3] = {fma_r(radial, ux, V2v * gY[0]), fma_r(radial, uy, V2v * gY[1]),
                                   fma_r(radial, uz, V2v * gY[2])};
                F[0] += G[0];
                F[1] += G[1];
                F[2] += G[2];
                if (kVir) {
                    Wv[0] = fma_r(G[0], d.x, Wv[0]);
                    Wv[1] = fma_r(G[1], d.y, Wv[1]);
                    Wv[2] = fma_r(G[2], d.z, Wv[2]);
                }
            }
        }
        if (!ok) continue;
        real fc[4];
        ld4<real>(R<real>(s.fc) + 4 * (size_t)i, fc);
        float *o = s.F_out + 3 * (size_t)s.perm[i];
        real Ft[3];
#pragma unroll
        for (int z = 0; z < 3; ++z) Ft[z] = fma_r(cn_fac, fc[z], F[z]);
        if (s.accumulate) {
            o[0] += (float)Ft[0];
            o[1] += (float)Ft[1];
            o[2] += (float)Ft[2];
        } else {
            o[0] = (float)Ft[0];
            o[1] = (float)Ft[1];
            o[2] = (float)Ft[2];
        }
        if (kVir) {
            real wc[4];
            ld4<real>(R<real>(s.wc) + 4 * (size_t)i, wc);
#pragma unroll
            for (int z = 0; z < 3; ++z) vir[z].add(real(0.5) * fma_r(cn_fac, wc[z], Wv[z]));
        }
    }
}

// The chain-rule factors of the two CVs, once per block: an FP64 chain is
// long and its pipe narrow on this part, so no thread repeats it.
template <typename real>
__device__ __forceinline__ void force_factors(const Sys &s, real &cn_fac, real &V2)
{
    __shared__ real fac[2];
    if (threadIdx.x == 0) {
        fac[0] = (real)(s.scal[kDV0] * s.fscale * 2.0 / s.n);
        fac[1] = s.ncv == 2 ? (real)(s.scal[kDV1] * s.fscale) : real(0);
    }
    __syncthreads();
    cn_fac = fac[0];
    V2 = fac[1];
}

// ------------------------------------------------------------------ blocks
// Each block walks tiles b, b + nb, ...; per tile: the staging table, the
// staged atoms (when they fit), the pass, a barrier before the next tile.

// Shared-memory layout of a staged pass: with positions, [cap] float4 then
// the records; without, the records alone.
template <typename real>
__device__ __forceinline__ void stage_pointers(const Sys &s, bool with_pos, float4 *&spos, real *&srec, real *&spair)
{
    spos = with_pos ? reinterpret_cast<float4 *>(tile_dyn) : nullptr;
    srec = reinterpret_cast<real *>(tile_dyn + (with_pos ? (size_t)s.stage_cap * 16 : 0));
    spair = srec + (size_t)s.stage_cap * kRecQ;
}

template <typename real, bool kCompute, bool kVir>
__device__ __forceinline__ void fwd_block(const Sys &s, Blk k)
{
    __shared__ __align__(16) TileTable T;
    float4 *spos = reinterpret_cast<float4 *>(tile_dyn);
    unsigned short *slist = reinterpret_cast<unsigned short *>(tile_dyn + (size_t)s.stage_cap * 16);
    RunSum<real> cn;
    for (int t = k.b; t < s.tiles; t += k.nb) {
        tile_load(s, t, T);
        if (T.total <= s.stage_cap) {
            stage_tile<real>(T, s.pos_s, nullptr, spos, nullptr, nullptr);
            const Src<real, true> src{T, spos, nullptr, nullptr, s.pos_s, nullptr};
            fwd_tile<real, true, kCompute, kVir>(s, T, src, slist, cn);
        } else {
            const Src<real, false> src{T, nullptr, nullptr, nullptr, s.pos_s, nullptr};
            fwd_tile<real, false, kCompute, kVir>(s, T, src, slist, cn);
        }
        __syncthreads();
    }
    // without a Q6 pass this pass holds the CV sum (its grid: one block per tile)
    if (kCompute && s.ncv == 1) last_block_cv(s, k, cn.value(), 0.0);
}

// The Q6 and adjoint passes: records and the own rows staged (both must
// fit), else both read from global memory.
template <typename real, bool kAvg>
__device__ __forceinline__ void records_block(const Sys &s, Blk k)
{
    __shared__ __align__(16) TileTable T;
    float4 *spos;
    real *srec, *spair;
    stage_pointers<real>(s, false, spos, srec, spair);
    const OwnRows<real> o = own_rows_at<real>(reinterpret_cast<unsigned char *>(spair + (size_t)s.stage_cap * 2));
    const real *rec = R<real>(kAvg ? s.rq : s.rb);
    const size_t N = (size_t)s.n;
    RunSum<real> cn, q6;
    for (int t = k.b; t < s.tiles; t += k.nb) {
        tile_load(s, t, T);
        if (T.total <= s.stage_cap && stage_own_rows<real>(s, T, o)) {
            stage_tile<real>(T, nullptr, rec, nullptr, srec, spair);  // waits for the rows' copies too
            const Src<real, true> src{T, nullptr, srec, spair, s.pos_s, rec};
            const RowSrc<real, true> rows{o, s.elist, s.wl, N, T.atom0};
            if (kAvg) avg_tile<real, true>(s, T, src, rows, cn, q6);
            else adj_tile<real, true>(s, T, src, rows);
        } else {
            const Src<real, false> src{T, nullptr, nullptr, nullptr, s.pos_s, rec};
            const RowSrc<real, false> rows{o, s.elist, s.wl, N, T.atom0};
            if (kAvg) avg_tile<real, false>(s, T, src, rows, cn, q6);
            else adj_tile<real, false>(s, T, src, rows);
        }
        __syncthreads();
    }
    if (kAvg) last_block_cv(s, k, cn.value(), q6.value());
}

template <typename real, bool kVir>
__device__ __forceinline__ void force_block(const Sys &s, Blk k)
{
    __shared__ __align__(16) TileTable T;
    float4 *spos;
    real *srec, *spair;
    stage_pointers<real>(s, true, spos, srec, spair);
    real cn_fac, V2;
    force_factors<real>(s, cn_fac, V2);
    const real *rh = R<real>(s.rh);
    RunSum<real> vir[3];
    for (int t = k.b; t < s.tiles; t += k.nb) {
        tile_load(s, t, T);
        if (T.total <= s.stage_cap) {
            stage_tile<real>(T, s.pos_s, rh, spos, srec, spair);
            const Src<real, true> src{T, spos, srec, spair, s.pos_s, rh};
            force_tile<real, true, kVir>(s, T, src, cn_fac, V2, vir);
        } else {
            const Src<real, false> src{T, nullptr, nullptr, nullptr, s.pos_s, rh};
            force_tile<real, false, kVir>(s, T, src, cn_fac, V2, vir);
        }
        __syncthreads();
    }
    if (kVir) virial_finish<real>(s, k, vir[0], vir[1], vir[2]);
}

// n_cv == 1: F_i = V1 (2/N) FC_i, one thread per atom (sorted order).
template <typename real, bool kVir>
__device__ __forceinline__ void force_cn(const Sys &s, Blk k)
{
    real cn_fac, V2;
    force_factors<real>(s, cn_fac, V2);
    RunSum<real> vir[3];
    for (int i = k.b * kTileThreads + threadIdx.x; i < s.n; i += k.nb * kTileThreads) {
        real fc[4];
        ld4<real>(R<real>(s.fc) + 4 * (size_t)i, fc);
        float *o = s.F_out + 3 * (size_t)s.perm[i];
        if (s.accumulate) {
            o[0] += (float)(cn_fac * fc[0]);
            o[1] += (float)(cn_fac * fc[1]);
            o[2] += (float)(cn_fac * fc[2]);
        } else {
            o[0] = (float)(cn_fac * fc[0]);
            o[1] = (float)(cn_fac * fc[1]);
            o[2] = (float)(cn_fac * fc[2]);
        }
        if (kVir) {
            real wc[4];
            ld4<real>(R<real>(s.wc) + 4 * (size_t)i, wc);
#pragma unroll
            for (int z = 0; z < 3; ++z) vir[z].add(real(0.5) * cn_fac * wc[z]);
        }
    }
    if (kVir) virial_finish<real>(s, k, vir[0], vir[1], vir[2]);
}

// ------------------------------------------------------------------ kernels
// Single-system launches: one block per tile (the passes holding a sum keep
// that grid; the others may be capped by a batch tile setting and walk
// their tiles grid-stride).  Batched launches: a block finds its system and
// its block index within that system's grid.
#define METAD_TILE_KERNELS(NAME, BODY, MINB)                                                              \
    template <typename real, bool kA, bool kB>                                                           \
    __global__ void __launch_bounds__(kTileThreads, MINB) k_##NAME(Sys s) { BODY<real, kA, kB>(s, own_blk()); } \
    template <typename real, bool kA, bool kB>                                                           \
    __global__ void __launch_bounds__(kTileThreads, MINB) kb_##NAME(BatchView v)                          \
    {                                                                                                    \
        Blk k;                                                                                           \
        const Sys &s = v.sys[batch_system(v, k)];                                                        \
        BODY<real, kA, kB>(s, k);                                                                        \
    }

template <typename real, bool kCompute, bool kVir>
__device__ __forceinline__ void fwd_body(const Sys &s, Blk k) { fwd_block<real, kCompute, kVir>(s, k); }
template <typename real, bool kUnusedA, bool kUnusedB>
__device__ __forceinline__ void avg_body(const Sys &s, Blk k) { records_block<real, true>(s, k); }
template <typename real, bool kUnusedA, bool kUnusedB>
__device__ __forceinline__ void adj_body(const Sys &s, Blk k) { records_block<real, false>(s, k); }
template <typename real, bool kVir, bool kUnused>
__device__ __forceinline__ void force_body(const Sys &s, Blk k) { force_block<real, kVir>(s, k); }
template <typename real, bool kVir, bool kUnused>
__device__ __forceinline__ void force_cn_body(const Sys &s, Blk k) { force_cn<real, kVir>(s, k); }

METAD_TILE_KERNELS(tile_fwd, fwd_body, 2)
METAD_TILE_KERNELS(tile_avg, avg_body, 2)
METAD_TILE_KERNELS(tile_adj, adj_body, 2)
METAD_TILE_KERNELS(tile_force, force_body, 2)
METAD_TILE_KERNELS(force_cn, force_cn_body, 1)
#undef METAD_TILE_KERNELS

template <typename real>
__global__ void k_per_atom_out(Sys s, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const int u = s.perm[i];
    out[u] = (double)R<real>(s.rq)[(size_t)i * 16 + 14];
    if (s.ncv == 2) out[(size_t)s.n + u] = (double)R<real>(s.rb)[(size_t)i * 16 + 14];
}

}  // namespace

// ------------------------------------------------------------------ host side
namespace {

// The kernel of a pass: precision, flag (forward pass: with the CV math),
// virial, single-system or batched.
template <typename real>
const void *pass_kernel(int pass, bool flag, bool vir, bool batched)
{
#define METAD_PICK(K, A, B) (batched ? (const void *)kb_##K<real, A, B> : (const void *)k_##K<real, A, B>)
    switch (pass) {
    case kPassFwd:
        if (!flag) return METAD_PICK(tile_fwd, false, false);
        return vir ? METAD_PICK(tile_fwd, true, true) : METAD_PICK(tile_fwd, true, false);
    case kPassAvg: return METAD_PICK(tile_avg, false, false);
    case kPassAdj: return METAD_PICK(tile_adj, false, false);
    case kPassForce: return vir ? METAD_PICK(tile_force, true, false) : METAD_PICK(tile_force, false, false);
    case kPassForceCn: return vir ? METAD_PICK(force_cn, true, false) : METAD_PICK(force_cn, false, false);
    }
#undef METAD_PICK
    return nullptr;
}

const void *pick(int pass, int fp64, bool flag, bool vir, bool batched)
{
    return fp64 ? pass_kernel<double>(pass, flag, vir, batched) : pass_kernel<float>(pass, flag, vir, batched);
}

}  // namespace

int tile_smem(const Sys &s, int pass)
{
    const int rs = s.fp64 ? 8 : 4;
    switch (pass) {
    case kPassFwd: return s.stage_cap * 16 + s.max_nb * kTileThreads * 2;
    case kPassForceCn: return 0;
    case kPassForce: return s.stage_cap * (16 + (kRecQ + 2) * rs);
    default: return s.stage_cap * (kRecQ + 2) * rs + own_rows_bytes(rs);  // records and own rows
    }
}

int pass_blocks(const Sys &s, int pass)
{
    if (pass == kPassForceCn) {
        const int g = (s.n + kTileThreads - 1) / kTileThreads;
        return g < 1 ? 1 : g;
    }
    return s.tiles;
}

void launch_tile_pass(const Sys &s, int pass, int flag, cudaStream_t st)
{
    const void *k = pick(pass, s.fp64, flag != 0, s.virial != 0, false);
    void *args[] = {const_cast<Sys *>(&s)};
    cudaLaunchKernel(k, dim3((unsigned)pass_blocks(s, pass)), dim3(kTileThreads), args, (size_t)tile_smem(s, pass),
                     st);
}

void launch_batch_pass(const BatchView &v, int total, int pass, int fp64, int flag, int vir, int smem,
                       cudaStream_t st)
{
    if (total <= 0) return;
    const void *k = pick(pass, fp64, flag != 0, vir != 0, true);
    void *args[] = {const_cast<BatchView *>(&v)};
    cudaLaunchKernel(k, dim3((unsigned)total), dim3(kTileThreads), args, (size_t)smem, st);
}

// Dynamic shared memory limits of the tile passes (their staging capacity
// needs more than the default 48 KB).
void configure_kernels()
{
    for (int fp64 = 0; fp64 < 2; ++fp64)
        for (int pass = 0; pass < kNumPasses; ++pass)
            for (int flag = 0; flag < 2; ++flag)
                for (int vir = 0; vir < 2; ++vir)
                    for (int batched = 0; batched < 2; ++batched) {
                        const void *k = pick(pass, fp64, flag != 0, vir != 0, batched != 0);
                        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxTileSmem);
                        // all of the SM's unified storage as shared memory, so
                        // two blocks of a staged pass fit on an SM
                        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                             cudaSharedmemCarveoutMaxShared);
                    }
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


}  // namespace metad

