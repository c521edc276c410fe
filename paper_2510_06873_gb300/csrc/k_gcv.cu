// Steps a4-a8 for the small-system CV families, which need no neighbour list:
//
//   torsion angles (the backbone Phi / Psi of the alanine-dipeptide runs,
//   Section "Alanine dipeptide torsion"), and
//   the distance from a reference atom to the nearest atom of a group (the
//   surface-oxygen to nearest-hydrogen CV of the rutile runs, Section "Water
//   dissociation on rutile (110) surface"), exact or as a soft minimum.
//
// Each system's CVs take one block (k_gcv_forward): its threads split the
// candidate group and reduce in a fixed tree, so the result does not depend
// on scheduling, and it leaves the gradient terms of every CV in s.gcv.
// The force pass (k_gcv_forces) gives one thread to each atom in the
// caller's order; it writes every atom (0 for atoms on no CV), adding the
// terms of each CV it belongs to in CV order: deterministic, no atomics.
// Positions are float32; bond and distance vectors are exact FP64
// differences.  The nearest-distance CV stays FP64 throughout (its nearest
// candidate is decided on the FP64 squared distance, as the definition);
// a torsion's angle and gradient run in FP32 (precision 0) or FP64
// (precision 1).  The file is compiled without multiply-add contraction, so
// squared distances round exactly as their plain definition.
#include <float.h>
#include <limits.h>

#include "hills.cuh"

namespace metad {

namespace {

constexpr int kGcvThreads = 256;

__device__ __forceinline__ double min_image(double d, double L)
{
    if (d > 0.5 * L)
        d -= L;
    else if (d < -0.5 * L)
        d += L;
    return d;
}

// Caller atom i, wrapped into the box, in FP64; flags a non-finite input.
__device__ __forceinline__ void atom_pos(const Sys &s, int i, double p[3], bool &bad)
{
    const float4 q = __ldg(s.pos_in + i);
    bad |= !(isfinite(q.x) && isfinite(q.y) && isfinite(q.z));
    p[0] = (double)wrap_coord(isfinite(q.x) ? q.x : 0.0f, s.Lin[0], s.L[0]);
    p[1] = (double)wrap_coord(isfinite(q.y) ? q.y : 0.0f, s.Lin[1], s.L[1]);
    p[2] = (double)wrap_coord(isfinite(q.z) ? q.z : 0.0f, s.Lin[2], s.L[2]);
}

// Minimum-image displacement r_j - r_i.
__device__ __forceinline__ void disp(const Sys &s, const double pi[3], const double pj[3], double d[3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = min_image(pj[k] - pi[k], s.L[k]);
}

template <typename real>
__device__ __forceinline__ real dot3(const real a[3], const real b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

template <typename real>
__device__ __forceinline__ void cross3(const real a[3], const real b[3], real c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ double sq_dist(const double d[3])
{
    const double xy = d[0] * d[0] + d[1] * d[1];
    return xy + d[2] * d[2];
}

__device__ __forceinline__ float real_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double real_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float real_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double real_atan2(double y, double x) { return atan2(y, x); }

// Torsion d of the system: with bonds b1 = r_b - r_a, b2 = r_c - r_b,
// b3 = r_d - r_c, the angle is atan2(y, x) where
//   x = (b1 x b2) . (b2 x b3) = (b1.b2)(b2.b3) - (b1.b3)(b2.b2)
//   y = |b2| b1 . (b2 x b3),
// and its gradient follows from d(atan2) = (x dy - y dx) / (x^2 + y^2) with
//   dx/db1 = (b2.b3) b2 - (b2.b2) b3
//   dx/db2 = (b2.b3) b1 + (b1.b2) b3 - 2 (b1.b3) b2
//   dx/db3 = (b1.b2) b2 - (b2.b2) b1
//   dy/db1 = |b2| (b2 x b3),  dy/db3 = |b2| (b1 x b2),
//   dy/db2 = |b2| (b3 x b1) + (b1 . (b2 x b3)) b2 / |b2|.
// Collinear atoms (x = y = 0): angle 0, no gradient.  The bonds are exact
// FP64 differences of the float32 positions (minimum image); the rest runs
// in `real` (float: a dependent FP64 chain is long on this part, and the
// angle of float32 positions needs no more).
template <typename real>
__device__ void torsion(const Sys &s, int d, bool &bad, double *xo, double *go)
{
    const int *q = s.cv_atoms + 4 * d;
    double ra[3], rb[3], rc[3], rd[3], e1[3], e2[3], e3[3];
    atom_pos(s, q[0], ra, bad);
    atom_pos(s, q[1], rb, bad);
    atom_pos(s, q[2], rc, bad);
    atom_pos(s, q[3], rd, bad);
    disp(s, ra, rb, e1);
    disp(s, rb, rc, e2);
    disp(s, rc, rd, e3);
    real b1[3], b2[3], b3[3];
    for (int k = 0; k < 3; ++k) {
        b1[k] = (real)e1[k];
        b2[k] = (real)e2[k];
        b3[k] = (real)e3[k];
    }
    real n1[3], n2[3], n3[3];
    cross3(b1, b2, n1);
    cross3(b2, b3, n2);
    cross3(b3, b1, n3);
    const real m2 = dot3(b2, b2), m = real_sqrt(m2);
    const real x = dot3(n1, n2);
    const real T = dot3(b1, n2);
    const real y = m * T;
    const real D = x * x + y * y;
    double *g = go + 16 * d;
    if (D == (real)0 || m == (real)0) {
        xo[d] = 0.0;
        for (int k = 0; k < 12; ++k) g[k] = 0.0;
        return;
    }
    xo[d] = (double)real_atan2(y, x);
    const real b12 = dot3(b1, b2), b23 = dot3(b2, b3), b13 = dot3(b1, b3);
    const real invD = (real)1 / D, inv_m = (real)1 / m;
    const real cx = x * invD, cy = y * invD;  // dphi = cx dy - cy dx
    const real tm = T * inv_m;
    for (int k = 0; k < 3; ++k) {
        const real dx1 = b23 * b2[k] - m2 * b3[k];
        const real dx2 = b23 * b1[k] + b12 * b3[k] - (real)2 * b13 * b2[k];
        const real dx3 = b12 * b2[k] - m2 * b1[k];
        const real dy1 = m * n2[k];
        const real dy2 = m * n3[k] + tm * b2[k];
        const real dy3 = m * n1[k];
        const real p1 = cx * dy1 - cy * dx1;  // dphi/db1
        const real p2 = cx * dy2 - cy * dx2;
        const real p3 = cx * dy3 - cy * dx3;
        g[k] = (double)(-p1);           // r_a
        g[3 + k] = (double)(p1 - p2);   // r_b
        g[6 + k] = (double)(p2 - p3);   // r_c
        g[9 + k] = (double)p3;          // r_d
    }
}

// Block reductions over the kGcvThreads threads in a fixed tree.
__device__ __forceinline__ void block_argmin(double &v, int &arg, double *shv, int *sha)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, v, o);
        const int oa = __shfl_down_sync(0xffffffffu, arg, o);
        if (ov < v || (ov == v && oa < arg)) { v = ov; arg = oa; }
    }
    if (lane == 0) { shv[wid] = v; sha[wid] = arg; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kGcvThreads / 32; ++w)
            if (shv[w] < v || (shv[w] == v && sha[w] < arg)) { v = shv[w]; arg = sha[w]; }
        shv[0] = v;
        sha[0] = arg;
    }
    __syncthreads();
    v = shv[0];
    arg = sha[0];
    __syncthreads();
}

// Four sums at once; the totals land in thread 0 only.
__device__ __forceinline__ void block_sum4(double v[4], double (*sh)[kGcvThreads / 32])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) sh[k][wid] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double t = 0.0;
            for (int w = 0; w < kGcvThreads / 32; ++w) t += sh[k][w];
            v[k] = t;
        }
    __syncthreads();
}

// Soft-minimum weight numerator exp(-beta (r - r_min)) of one candidate;
// the forward and force passes share it, so they round alike.
__device__ __forceinline__ double soft_weight(const Sys &s, double r, double rmin)
{
    return exp(-s.sm_beta * (r - rmin));
}

// Nearest-distance CV d (all threads of the block): go[16 d] holds the
// nearest slot, r_min, the soft-minimum normaliser Z and d s/d r_ref.
__device__ void nearest(const Sys &s, int d, bool &bad, double *xo, double *go)
{
    __shared__ double shv[kGcvThreads / 32];
    __shared__ int sha[kGcvThreads / 32];
    const int o = s.cv_atoms[d];
    const int *cand = s.cv_atoms + s.ncv;
    double po[3];
    atom_pos(s, o, po, bad);
    double best = DBL_MAX;
    int arg = INT_MAX;
    for (int m = threadIdx.x; m < s.n_cand; m += kGcvThreads) {
        double pj[3], dv[3];
        atom_pos(s, cand[m], pj, bad);
        disp(s, po, pj, dv);
        const double r2 = sq_dist(dv);
        if (r2 < best) { best = r2; arg = m; }
    }
    block_argmin(best, arg, shv, sha);
    const double rmin = sqrt(best);
    double *g = go + 16 * d;
    if (s.sm_beta <= 0.0) {
        if (threadIdx.x == 0) {
            double pj[3], dv[3];
            atom_pos(s, cand[arg], pj, bad);
            disp(s, po, pj, dv);
            xo[d] = rmin;
            g[0] = (double)arg;
            g[1] = rmin;
            g[2] = 1.0;
            for (int k = 0; k < 3; ++k) g[3 + k] = rmin > 0.0 ? -dv[k] / rmin : 0.0;
        }
        return;
    }
    __shared__ double sh4[4][kGcvThreads / 32];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};  // Z and sum_j e_j u_j
    for (int m = threadIdx.x; m < s.n_cand; m += kGcvThreads) {
        double pj[3], dv[3];
        atom_pos(s, cand[m], pj, bad);
        disp(s, po, pj, dv);
        const double r = sqrt(sq_dist(dv));
        const double e = soft_weight(s, r, rmin);
        acc[0] += e;
        if (r > 0.0) {
            acc[1] += e * (dv[0] / r);
            acc[2] += e * (dv[1] / r);
            acc[3] += e * (dv[2] / r);
        }
    }
    block_sum4(acc, sh4);
    if (threadIdx.x == 0) {
        const double Z = acc[0];
        xo[d] = rmin - log(Z) / s.sm_beta;
        g[0] = (double)arg;
        g[1] = rmin;
        g[2] = Z;
        g[3] = -acc[1] / Z;
        g[4] = -acc[2] / Z;
        g[5] = -acc[3] / Z;
    }
}

// The CVs into xo[d] and their gradient terms into go[16 d ...] (shared or
// global memory).
template <typename real>
__device__ void gcv_eval(const Sys &s, double *xo, double *go)
{
    bool bad = false;
    if (s.kind == kKindTorsion) {
        if (threadIdx.x < s.ncv) torsion<real>(s, threadIdx.x, bad, xo, go);
    } else {
        for (int d = 0; d < s.ncv; ++d) nearest(s, d, bad, xo, go);
    }
    if (bad) atomicOr(s.err, kErrNonFinite);
}

template <typename real>
__device__ void gcv_forward(const Sys &s)
{
    gcv_eval<real>(s, s.scal + kS0, s.gcv);
    if (threadIdx.x == 0 && s.ncv == 1) s.scal[kS1] = 0.0;
}

// F_i = (accumulate ? F_i : 0) - scale sum_d dV/ds_d ds_d/dr_i, with the
// gradient terms gterms of the CV pass.
__device__ void gcv_forces(const Sys &s, Blk blk, const double *gterms)
{
    const int *cand = s.cv_atoms + s.ncv;
    for (int i = blk.b * kGcvThreads + threadIdx.x; i < s.n; i += blk.nb * kGcvThreads) {
        double f[3] = {0.0, 0.0, 0.0};
        for (int d = 0; d < s.ncv; ++d) {
            const double dv = s.scal[kDV0 + d];
            const double *g = gterms + 16 * d;
            if (s.kind == kKindTorsion) {
                for (int q = 0; q < 4; ++q)
                    if (s.cv_atoms[4 * d + q] == i)
                        for (int k = 0; k < 3; ++k) f[k] -= dv * g[3 * q + k];
                continue;
            }
            if (s.cv_atoms[d] == i)
                for (int k = 0; k < 3; ++k) f[k] -= dv * g[3 + k];
            const int m = s.cand_slot[i];
            if (m < 0) continue;
            const bool exact = s.sm_beta <= 0.0;
            if (exact && m != (int)g[0]) continue;
            bool bad = false;
            double po[3], pj[3], dd[3];
            atom_pos(s, s.cv_atoms[d], po, bad);
            atom_pos(s, cand[m], pj, bad);
            disp(s, po, pj, dd);
            const double r = sqrt(sq_dist(dd));
            if (!(r > 0.0)) continue;
            const double w = exact ? 1.0 : soft_weight(s, r, g[1]) / g[2];
            for (int k = 0; k < 3; ++k) f[k] -= dv * (w * (dd[k] / r));
        }
        float *out = s.F_out + 3 * (size_t)i;
        for (int k = 0; k < 3; ++k) {
            const float v = (float)(s.fscale * f[k]);
            out[k] = s.accumulate ? out[k] + v : v;
        }
    }
}

template <typename real>
__global__ void __launch_bounds__(kGcvThreads) k_gcv_forward(Sys s) { gcv_forward<real>(s); }

__global__ void __launch_bounds__(kGcvThreads) k_gcv_forces(Sys s) { gcv_forces(s, own_blk(), s.gcv); }

// The whole step in one launch (systems of up to kFuseAtoms atoms): every
// block evaluates the CVs (a few atoms, or one pass over the candidates)
// into shared memory and sums its share of the hills there; block 0
// publishes the CVs; the last block to finish the hill sum (which also
// deposits, if asked) writes every atom's force from its own copy of the
// CV gradient terms.  The same arithmetic as the three-kernel path, so the
// same bits.
template <typename real>
__device__ void gcv_step(const Sys &s, Blk blk)
{
    __shared__ double xs[kMaxCv];
    __shared__ double gs[16 * 2];
    if (threadIdx.x < kMaxCv) xs[threadIdx.x] = 0.0;
    if (threadIdx.x < 16 * 2) gs[threadIdx.x] = 0.0;
    __syncthreads();
    gcv_eval<real>(s, xs, gs);
    __syncthreads();
    if (blk.b == 0) {
        if (threadIdx.x < kMaxCv) s.scal[kS0 + threadIdx.x] = xs[threadIdx.x];
        if (threadIdx.x < 16 * s.ncv) s.gcv[threadIdx.x] = gs[threadIdx.x];
    }
    if (!hill_sum(s, blk, xs, s.scal + kV, s.deposit)) return;
    __syncthreads();  // thread 0 of this block wrote dV/ds
    gcv_forces(s, Blk{0, 1}, gs);
}

template <typename real>
__global__ void __launch_bounds__(kGcvThreads) k_gcv_step(Sys s) { gcv_step<real>(s, own_blk()); }

template <typename real>
__global__ void __launch_bounds__(kGcvThreads) kb_gcv_step(BatchView v)
{
    Blk k;
    const Sys &s = v.sys[batch_system(v, k)];
    gcv_step<real>(s, k);
}

template <typename real>
__global__ void __launch_bounds__(kGcvThreads) kb_gcv_forward(BatchView v)
{
    Blk k;
    const Sys &s = v.sys[batch_system(v, k)];
    gcv_forward<real>(s);
}

__global__ void __launch_bounds__(kGcvThreads) kb_gcv_forces(BatchView v)
{
    Blk k;
    const Sys &s = v.sys[batch_system(v, k)];
    gcv_forces(s, k, s.gcv);
}

}  // namespace

void launch_gcv_forward(const Sys &s, int fp64, cudaStream_t st)
{
    if (fp64)
        k_gcv_forward<double><<<1, kGcvThreads, 0, st>>>(s);
    else
        k_gcv_forward<float><<<1, kGcvThreads, 0, st>>>(s);
}

void launch_gcv_forces(const Sys &s, float *F, int accumulate, double scale, cudaStream_t st)
{
    Sys t = s;
    t.F_out = F;
    t.accumulate = accumulate;
    t.fscale = scale;
    k_gcv_forces<<<grid_blocks(t, GK_ATOM256, 0), kGcvThreads, 0, st>>>(t);
}

void launch_batch_gcv(const BatchView &one, int one_total, int fp64, cudaStream_t st)
{
    if (one_total <= 0) return;
    if (fp64)
        kb_gcv_forward<double><<<one_total, kGcvThreads, 0, st>>>(one);
    else
        kb_gcv_forward<float><<<one_total, kGcvThreads, 0, st>>>(one);
}

void launch_batch_gcv_forces(const BatchView &atoms, int atom_total, cudaStream_t st)
{
    if (atom_total > 0) kb_gcv_forces<<<atom_total, kGcvThreads, 0, st>>>(atoms);
}

void launch_gcv_step(const Sys &s, int K, float *F, int accumulate, int deposit, int fp64, cudaStream_t st)
{
    Sys t = s;
    t.K = K;
    t.F_out = F;
    t.accumulate = accumulate;
    t.fscale = 1.0;
    t.deposit = deposit;
    const int nb = bias_blocks(K);
    if (fp64)
        k_gcv_step<double><<<nb, kGcvThreads, 0, st>>>(t);
    else
        k_gcv_step<float><<<nb, kGcvThreads, 0, st>>>(t);
}

void launch_batch_gcv_step(const BatchView &hills, int hill_total, int fp64, cudaStream_t st)
{
    if (hill_total <= 0) return;
    if (fp64)
        kb_gcv_step<double><<<hill_total, kGcvThreads, 0, st>>>(hills);
    else
        kb_gcv_step<float><<<hill_total, kGcvThreads, 0, st>>>(hills);
}


// The kernels of this file whose only argument is the system descriptor
// (a captured step's nodes of these can take new I/O buffers in place).
bool sys_kernel_gcv(const void *func)
{
    static const void *const kernels[] = {
        (const void *)k_gcv_forward<float>,
        (const void *)k_gcv_forward<double>,
        (const void *)k_gcv_forces,
        (const void *)k_gcv_step<float>,
        (const void *)k_gcv_step<double>,
    };
    for (const void *k : kernels)
        if (k == func) return true;
    return false;
}

}  // namespace metad
