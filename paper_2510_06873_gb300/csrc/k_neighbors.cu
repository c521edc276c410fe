// Steps a1-a3: ingest, Morton-ranked cell order, Verlet list and the exact
// neighbour list.
//
// Each step:
//   k_gather_check  positions in cell order (wrapped), and a flag when any
//                   atom moved more than skin/2 since the last rebuild
//   rebuild chain   (early exit unless flagged) counting sort of the atoms
//                   into Morton-ranked cells of edge >= rc + skin, stable by
//                   caller index, and the Verlet list r < rc + skin
//   filter          exact rows {j : r_ij^2 < rc^2} from the Verlet rows
//                   (fused into the CV kernel, or k_filter on its own)
// The exact rows are the FP64 definition bit for bit: while no atom has moved
// more than skin/2, every pair now inside rc was inside rc + skin at the
// rebuild, and the float32 estimate only decides outside a guard band.
#include "metad_impl.cuh"

namespace metad {

namespace {

__device__ __forceinline__ float4 load_wrapped(const Sys &s, int u, bool &bad)
{
    float4 p = s.pos_in[u];
    bad = !(isfinite(p.x) && isfinite(p.y) && isfinite(p.z));
    if (bad) {
        p.x = p.y = p.z = 0.0f;
        return p;
    }
    p.x = wrap_coord(p.x, s.Lin[0], s.L[0]);
    p.y = wrap_coord(p.y, s.Lin[1], s.L[1]);
    p.z = wrap_coord(p.z, s.Lin[2], s.L[2]);
    return p;
}

__device__ __forceinline__ int cell_axis(float x, float inv_h, int nc)
{
    int c = (int)floorf(x * inv_h);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// Current positions in the cell order of the last rebuild, and the rebuild
// test.  Before the first rebuild the flag is already set.  The Verlet rows
// hold every pair within rc + skin at the last rebuild; a pair's
// displacement has since changed by at most |dr_i| + |dr_j| + |L - L_ref|
// (the last term for pairs across the box faces when the box changed), so
// the rows stay valid while every |dr| <= (skin - |L - L_ref|) / 2.
__device__ __forceinline__ void gather_check(const Sys &s, Blk k)
{
    const int t = k.b * blockDim.x + threadIdx.x;
    bool move = false;
    float thr2 = s.disp_thr2;
    {
        const float ex = s.Lhi[0] - __ldg(s.Lref), ey = s.Lhi[1] - __ldg(s.Lref + 1), ez = s.Lhi[2] - __ldg(s.Lref + 2);
        const float dL2 = ex * ex + ey * ey + ez * ez;
        if (dL2 > 0.0f) {
            const float half = 0.5f * (s.skin_eff - sqrtf(dL2));
            thr2 = half > 0.0f ? half * half : -1.0f;
        }
    }
    if (t < s.n) {
        bool bad;
        float4 p = load_wrapped(s, s.perm[t], bad);
        if (bad) set_err(s, kErrNonFinite);
        s.pos_s[t] = p;
        const float4 r = s.pos_ref[t];
        float dx = mi_f(p.x - r.x, s.halfL[0], s.Lhi[0], s.Llo[0]);
        float dy = mi_f(p.y - r.y, s.halfL[1], s.Lhi[1], s.Llo[1]);
        float dz = mi_f(p.z - r.z, s.halfL[2], s.Lhi[2], s.Llo[2]);
        move = !(dx * dx + dy * dy + dz * dz <= thr2) || p.w != r.w;
    }
    if (__any_sync(0xffffffffu, move) && (threadIdx.x & 31) == 0) atomicOr(s.flag, 1);
}

// Programmatic dependent launch along the rebuild chain.  A kernel of the
// chain lets the next one be scheduled once all its own blocks have started
// (so the next launch overlaps its run instead of following it), and waits
// for the previous kernel to complete, its memory visible, before it reads
// anything.  A step without a rebuild then pays little more than the
// blocks' early exits.  (Without a programmatic launch the wait returns at
// once: the previous kernel has completed.)
__device__ __forceinline__ void chain_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void chain_enter()
{
    chain_next();
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__global__ void k_gather_check(Sys s)
{
    chain_next();
    gather_check(s, own_blk());
}

__device__ __forceinline__ void bin_one(const Sys &s, int u)
{
    bool bad;
    float4 p = load_wrapped(s, u, bad);
    int cx = cell_axis(p.x, s.inv_h[0], s.nc[0]);
    int cy = cell_axis(p.y, s.inv_h[1], s.nc[1]);
    int cz = cell_axis(p.z, s.inv_h[2], s.nc[2]);
    int c = s.rank_of_xyz[(cz * s.nc[1] + cy) * s.nc[0] + cx];
    s.ucell[u] = c;
    s.uslot[u] = atomicAdd(&s.cell_count[c], 1);
}

__device__ __forceinline__ void bin_count(const Sys &s, Blk k)
{
    if (!*s.flag) return;
    for (int u = k.b * blockDim.x + threadIdx.x; u < s.n; u += k.nb * blockDim.x) bin_one(s, u);
}

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_sums, int &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = warp_sums[lane];
        int t = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_sums[lane] = t - w;
        if (lane == 31) warp_sums[32] = t;
    }
    __syncthreads();
    total = warp_sums[32];
    int r = warp_sums[wid] + x - v;
    __syncthreads();
    return r;
}

__device__ __forceinline__ void scan_reduce(const Sys &s, Blk k)
{
    if (!*s.flag) return;
    __shared__ int ws[33];
    int base = k.b * kScanTile + threadIdx.x * kScanItems;
    int v = 0;
#pragma unroll
    for (int t = 0; t < kScanItems; ++t)
        if (base + t < s.ncell) v += s.cell_count[base + t];
    int total;
    block_exclusive_scan(v, ws, total);
    if (threadIdx.x == 0) s.scan_part[k.b] = total;
}

__device__ __forceinline__ void scan_down(const Sys &s, Blk k)
{
    if (!*s.flag) return;
    __shared__ int ws[33];
    __shared__ int prefix;
    if (threadIdx.x < 32) {
        int acc = 0;
        for (int b = threadIdx.x; b < k.b; b += 32) acc += s.scan_part[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) prefix = acc;
    }
    __syncthreads();
    int base = k.b * kScanTile + threadIdx.x * kScanItems;
    int c[kScanItems];
    int v = 0;
    // the counters' last reader: they are left zero for the next rebuild
    // (zero from creation on, so no pass of their own clears them)
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        c[t] = 0;
        if (base + t < s.ncell) {
            c[t] = s.cell_count[base + t];
            s.cell_count[base + t] = 0;
        }
        v += c[t];
    }
    int total;
    int ex = block_exclusive_scan(v, ws, total) + prefix;
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        if (base + t < s.ncell) s.cell_start[base + t] = ex;
        ex += c[t];
    }
    if (base <= s.ncell - 1 && s.ncell - 1 < base + kScanItems) s.cell_start[s.ncell] = s.n;
}

__device__ __forceinline__ void bin_scatter(const Sys &s, Blk k)
{
    if (!*s.flag) return;
    for (int u = k.b * blockDim.x + threadIdx.x; u < s.n; u += k.nb * blockDim.x)
        s.perm[s.cell_start[s.ucell[u]] + s.uslot[u]] = u;
}

// One thread per cell: order the cell's atoms by caller index (the atomic
// slots above are not deterministic), gather their wrapped positions and
// keep them as the reference of the new Verlet list.
__device__ __forceinline__ void sort_gather_cell(const Sys &s, int c)
{
    int a = s.cell_start[c], e = s.cell_start[c + 1];
    for (int t = a + 1; t < e; ++t) {
        int v = s.perm[t];
        int k = t - 1;
        while (k >= a && s.perm[k] > v) {
            s.perm[k + 1] = s.perm[k];
            --k;
        }
        s.perm[k + 1] = v;
    }
    for (int t = a; t < e; ++t) {
        bool bad;
        float4 p = load_wrapped(s, s.perm[t], bad);
        s.pos_s[t] = p;
        s.pos_ref[t] = p;
        s.scell[t] = c;
    }
}

__device__ __forceinline__ void cell_sort_gather(const Sys &s, Blk k)
{
    if (!*s.flag) return;
    for (int c = k.b * blockDim.x + threadIdx.x; c < s.ncell; c += k.nb * blockDim.x) sort_gather_cell(s, c);
}

__device__ __forceinline__ int wrap_cell(int c, int nc)
{
    c += (c < 0) ? nc : 0;
    c -= (c >= nc) ? nc : 0;
    return c;
}

// Stencil offsets along one axis: -1, 0, 1 with three or more cells (each
// distinct cell once with fewer).
__device__ __forceinline__ int axis_span(int nc) { return nc >= 3 ? 3 : nc; }
__device__ __forceinline__ int axis_off(int nc, int idx) { return nc >= 3 ? idx - 1 : idx; }

// Verlet rows {j : r_ij^2 < (rc + skin)^2 (1 + 1e-4)} over the 27 cells
// around each atom's own (each distinct cell once): entries with j > i
// first, then j < i, each part in stencil-cell order (x fastest), atoms in
// cell order.  Atoms are sorted by cell rank, so a cell ranked above the
// atom's own holds only j > i and one ranked below only j < i.
//
// One warp per cell A at a time.  The candidates of A's atoms are the same
// list: the part-0 cells (rank >= A's) then the part-1 cells (rank <= A's),
// each in stencil order, A itself in both.  The warp stages that list in
// shared memory with coalesced loads (position, index, stencil cell), then
// sweeps its 32 lanes over it for each atom of A in turn, compacting the
// accepted entries with a ballot: the row comes out in its final order, with
// no per-lane cell search and no divergence between lanes.  A list longer
// than the buffer is staged and swept in chunks, per atom.
//
// Displacements: with three or more cells along every axis each stencil cell
// is a distinct cell at one periodic image, and d = (r_j - r_i) + shift with
// the cell's image shift (0 or +-L per axis): no minimum-image test per
// candidate, and since both roundings are sign-symmetric the two directions
// of a pair give exactly opposite vectors, so the rows stay symmetric.  With
// fewer cells along an axis, the minimum image per candidate.  The 1e-4
// margin on the cutoff covers the rounding of either form.
constexpr int kStencil = 27;
constexpr int kVerletWarps = kBlockAtoms / 32;
constexpr int kCandBuf = 256;  // staged candidates per warp

struct VerletWarpSmem {
    float4 pos[kCandBuf];      // candidate position, index bits in w
    unsigned char q[kCandBuf]; // candidate's stencil cell
    float4 shift[kStencil];    // image shift of each stencil cell
};

// Copy the candidates [k0, k0 + len) of the list into the buffer: lane q
// copies its stencil cell's segments (in part 0 at o0, in part 1 at o1; -1
// when not in it), so the warp's loads are all independent of one another.
__device__ __forceinline__ void verlet_stage(const Sys &s, VerletWarpSmem &w, int st, int n, int o0, int o1, int k0,
                                             int len, int lane)
{
#pragma unroll
    for (int part = 0; part < 2; ++part) {
        const int o = part == 0 ? o0 : o1;
        if (o < 0) continue;
        const int lo = max(o, k0), hi = min(o + n, k0 + len);
#pragma unroll 4
        for (int t = lo; t < hi; ++t) {
            const int j = st + (t - o);
            float4 pj = s.pos_s[j];
            pj.w = __int_as_float(j);
            w.pos[t - k0] = pj;
            w.q[t - k0] = (unsigned char)lane;
        }
    }
    __syncwarp();
}

// Sweep atom i over the staged candidates [t0, t1) of the buffer, all in one
// part (kUp: part 0, j > i; else part 1, j < i), appending to its row.
// kShift: some stencil cell of this one is a periodic image (a cell on the
// box faces); interior cells need no shift.
template <bool kImages, bool kShift, bool kUp>
__device__ __forceinline__ bool verlet_test(const Sys &s, const VerletWarpSmem &w, int i, float4 pi, int t, int t1,
                                            int &j)
{
    // branch-free: the buffer position is clamped in bounds and the test
    // masked by t < t1
    const int tc = min(t, kCandBuf - 1);
    const float4 cp = w.pos[tc];
    j = __float_as_int(cp.w);
    Vec3<float> d;
    if (!kImages) {
        d = displacement<float>(s, pi, cp);
    } else if (kShift) {
        // past the staged length w.q is stale: keep the index in the table
        const float4 h = w.shift[min((int)w.q[tc], kStencil - 1)];
        d.x = (cp.x - pi.x) + h.x;
        d.y = (cp.y - pi.y) + h.y;
        d.z = (cp.z - pi.z) + h.z;
    } else {
        d.x = cp.x - pi.x;
        d.y = cp.y - pi.y;
        d.z = cp.z - pi.z;
    }
    return t < t1 && (kUp ? j > i : j < i) && fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z)) < s.rv2;
}

// Sweep atom i over the staged candidates [t0, t1) of the buffer, all in one
// part (kUp: part 0, j > i; else part 1, j < i), appending to its row, two
// rounds of 32 per iteration.  kShift: some stencil cell of this one is a
// periodic image (a cell on the box faces); interior cells need no shift.
template <bool kImages, bool kShift, bool kUp>
__device__ __forceinline__ void verlet_sweep(const Sys &s, const VerletWarpSmem &w, int i, float4 pi, int t0, int t1,
                                             int lane, int *vrow, int &total)
{
    const unsigned lt = (1u << lane) - 1u;
    for (int r = t0; r < t1; r += 64) {
        int ja, jb;
        const bool ina = verlet_test<kImages, kShift, kUp>(s, w, i, pi, r + lane, t1, ja);
        const bool inb = verlet_test<kImages, kShift, kUp>(s, w, i, pi, r + 32 + lane, t1, jb);
        const unsigned ba = __ballot_sync(0xffffffffu, ina), bb = __ballot_sync(0xffffffffu, inb);
        const int ata = total + __popc(ba & lt);
        const int atb = total + __popc(ba) + __popc(bb & lt);
        if (ina && ata < s.max_vnb) vrow[ata] = ja;
        if (inb && atb < s.max_vnb) vrow[atb] = jb;
        total += __popc(ba) + __popc(bb);
    }
}

template <bool kImages, bool kShift>
__device__ __forceinline__ void verlet_sweeps(const Sys &s, const VerletWarpSmem &w, int i, float4 pi, int k0, int len,
                                              int T0, int lane, int *vrow, int &total, int &up)
{
    const int split = min(max(T0 - k0, 0), len);  // buffer positions below it are part 0
    verlet_sweep<kImages, kShift, true>(s, w, i, pi, 0, split, lane, vrow, total);
    if (k0 < T0) up = total;
    verlet_sweep<kImages, kShift, false>(s, w, i, pi, split, len, lane, vrow, total);
}

template <bool kImages>
__device__ __forceinline__ void verlet_cell(const Sys &s, VerletWarpSmem &w, int c, int lane)
{
    const int a0 = s.cell_start[c], na = s.cell_start[c + 1] - a0;
    if (na == 0) return;
    const int xyz = s.xyz_of_rank[c];
    const int cx = xyz & 1023, cy = (xyz >> 10) & 1023, cz = xyz >> 20;
    // with images every axis spans three cells: constant divisions below
    const int sx = kImages ? 3 : axis_span(s.nc[0]), sy = kImages ? 3 : axis_span(s.nc[1]),
              sz = kImages ? 3 : axis_span(s.nc[2]);
    const int nq = sx * sy * sz;
    // a cell on the box faces has stencil cells at a periodic image
    const bool shifted = cx == 0 || cy == 0 || cz == 0 || cx == s.nc[0] - 1 || cy == s.nc[1] - 1 || cz == s.nc[2] - 1;
    // the stencil: lane q < nq looks up cell q (x fastest) and its segments
    int n0 = 0, n1 = 0, st = 0, n = 0;  // lane q's cell: first atom, atoms, its part-0 / part-1 lengths
    if (lane < nq) {
        const int ex = lane % sx, ey = (lane / sx) % sy, ez = lane / (sx * sy);
        const int x = cx + axis_off(s.nc[0], ex), y = cy + axis_off(s.nc[1], ey), z = cz + axis_off(s.nc[2], ez);
        const int cq = s.rank_of_xyz[(wrap_cell(z, s.nc[2]) * s.nc[1] + wrap_cell(y, s.nc[1])) * s.nc[0] +
                                     wrap_cell(x, s.nc[0])];
        st = s.cell_start[cq];
        n = s.cell_start[cq + 1] - st;
        if (kImages && shifted)  // only a cell on the box faces reads the shifts
            w.shift[lane] = make_float4(x < 0 ? -s.Lhi[0] : (x >= s.nc[0] ? s.Lhi[0] : 0.0f),
                                        y < 0 ? -s.Lhi[1] : (y >= s.nc[1] ? s.Lhi[1] : 0.0f),
                                        z < 0 ? -s.Lhi[2] : (z >= s.nc[2] ? s.Lhi[2] : 0.0f), 0.0f);
        n0 = cq >= c ? n : 0;
        n1 = cq <= c ? n : 0;
    }
    // exclusive scans of the segment lengths over the stencil (lanes)
    int i0 = n0, i1 = n1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y0 = __shfl_up_sync(0xffffffffu, i0, o), y1 = __shfl_up_sync(0xffffffffu, i1, o);
        if (lane >= o) {
            i0 += y0;
            i1 += y1;
        }
    }
    const int T0 = __shfl_sync(0xffffffffu, i0, 31), T1 = __shfl_sync(0xffffffffu, i1, 31);
    // lane q's segments in the list (-1: not in that part); lanes past the
    // stencil have none
    const int o0 = n0 > 0 ? i0 - n0 : -1, o1 = n1 > 0 ? T0 + i1 - n1 : -1;
    const int T = T0 + T1;
    const bool one_chunk = T <= kCandBuf;
    if (one_chunk) verlet_stage(s, w, st, n, o0, o1, 0, T, lane);
    for (int ia = 0; ia < na; ++ia) {
        const int i = a0 + ia;
        const float4 pi = s.pos_s[i];
        int *vrow = s.vnbr + (size_t)i * s.max_vnb;
        int total = 0, up = 0;
        for (int k0 = 0; k0 < T; k0 += kCandBuf) {
            const int len = min(kCandBuf, T - k0);
            if (!one_chunk) verlet_stage(s, w, st, n, o0, o1, k0, len, lane);
            if (shifted) verlet_sweeps<kImages, true>(s, w, i, pi, k0, len, T0, lane, vrow, total, up);
            else verlet_sweeps<kImages, false>(s, w, i, pi, k0, len, T0, lane, vrow, total, up);
            if (!one_chunk) __syncwarp();  // the chunk is read before the next is staged
        }
        if (lane == 0) {
            if (total > s.max_vnb) set_err(s, kErrCapacity);
            s.vnn[i] = min(total, s.max_vnb);
            s.vnh[i] = min(up, s.max_vnb);
        }
    }
    __syncwarp();  // the tables are read before the next cell overwrites them
}

// End of a rebuild, run once by the last Verlet block to finish: the rows'
// box becomes the reference, the rows are marked new, and the flag is
// cleared for the next step (kept set when the skin is zero, so every step
// rebuilds).
__device__ __forceinline__ void finish_rebuild(const Sys &s, Blk k)
{
    __shared__ bool am_last;
    __syncthreads();
    if (threadIdx.x == 0) am_last = atomicAdd(&s.ticket[4], 1u) == (unsigned)k.nb - 1u;
    __syncthreads();
    if (!am_last || threadIdx.x != 0) return;
    s.ticket[4] = 0u;
    *s.rebuilds += 1ull;
    for (int a = 0; a < 3; ++a) s.Lref[a] = s.Lhi[a];
    if (s.mirror) *s.rows_fresh = 1;  // the next filter finds the mirror positions
    *s.flag = s.always_rebuild ? 1 : 0;
}

// Grid-stride over cells, one warp per cell, so an idle launch (no rebuild)
// retires at once.
__device__ __forceinline__ void verlet(const Sys &s, Blk k)
{
    if (!*s.flag) return;
    __shared__ VerletWarpSmem sh[kVerletWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool images = s.nc[0] >= 3 && s.nc[1] >= 3 && s.nc[2] >= 3;
    const int warps = k.nb * kVerletWarps;
    for (int c = k.b * kVerletWarps + wid; c < s.ncell; c += warps) {
        if (images) verlet_cell<true>(s, sh[wid], c, lane);
        else verlet_cell<false>(s, sh[wid], c, lane);
    }
    finish_rebuild(s, k);
}

// Exact rows from the Verlet rows, when the CV kernel does not fuse it.
template <typename real>
__global__ void __launch_bounds__(kBlockAtoms) k_filter(Sys s)
{
    const int groups = group_grid(s.n);
    for (int blk = blockIdx.x; blk < groups; blk += gridDim.x) filter_row<real>(s, atom_lane_at(s, blk));
}


// Single-system kernels of the rebuild chain.
__global__ void k_bin_count(Sys s)
{
    chain_enter();
    bin_count(s, own_blk());
}
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(Sys s)
{
    chain_enter();
    scan_reduce(s, own_blk());
}
__global__ void __launch_bounds__(kScanThreads) k_scan_down(Sys s)
{
    chain_enter();
    scan_down(s, own_blk());
}
__global__ void k_bin_scatter(Sys s)
{
    chain_enter();
    bin_scatter(s, own_blk());
}
__global__ void k_cell_sort_gather(Sys s)
{
    chain_enter();
    cell_sort_gather(s, own_blk());
}
__global__ void __launch_bounds__(kBlockAtoms) k_verlet(Sys s)
{
    chain_enter();
    verlet(s, own_blk());
}

// The same kernels over every system of a batch.
__global__ void kb_gather_check(BatchView v)
{
    chain_next();
    Blk k;
    const Sys &s = v.sys[batch_system(v, k)];
    gather_check(s, k);
}
__global__ void kb_bin_count(BatchView v)
{
    chain_enter();
    Blk k;
    const Sys &s = v.sys[batch_system(v, k)];
    bin_count(s, k);
}
__global__ void __launch_bounds__(kScanThreads) kb_scan_reduce(BatchView v)
{
    chain_enter();
    Blk k;
    const Sys &s = v.sys[batch_system(v, k)];
    scan_reduce(s, k);
}
__global__ void __launch_bounds__(kScanThreads) kb_scan_down(BatchView v)
{
    chain_enter();
    Blk k;
    const Sys &s = v.sys[batch_system(v, k)];
    scan_down(s, k);
}
__global__ void kb_bin_scatter(BatchView v)
{
    chain_enter();
    Blk k;
    const Sys &s = v.sys[batch_system(v, k)];
    bin_scatter(s, k);
}
__global__ void kb_cell_sort_gather(BatchView v)
{
    chain_enter();
    Blk k;
    const Sys &s = v.sys[batch_system(v, k)];
    cell_sort_gather(s, k);
}
__global__ void __launch_bounds__(kBlockAtoms) kb_verlet(BatchView v)
{
    chain_enter();
    Blk k;
    const Sys &s = v.sys[batch_system(v, k)];
    verlet(s, k);
}

// Pairs (i < j) in caller indices, for export: one thread per sorted atom,
// entries with caller(i) < caller(j) appended through one counter.  Each
// exact entry's j is read from its geometry tag (the exact rows of indices
// are kept only without mirror slots).
template <typename real>
__global__ void k_export_pairs(Sys s, long long *pairs, int *count)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    int ui = s.perm[i];
    for (int k = 0; k < s.nn[i]; ++k) {
        Vec3<real> d;
        bool cn;
        int j;
        unsigned vm;
        load_geo<real>(s, (size_t)i * s.max_nb + k, d, cn, j, vm);
        int uj = s.perm[j];
        if (ui < uj) {
            int slot = atomicAdd(count, 1);
            pairs[2 * (size_t)slot] = ui;
            pairs[2 * (size_t)slot + 1] = uj;
        }
    }
}

// Sum and maximum of the per-atom neighbour counts.
__global__ void k_nn_stats(Sys s, unsigned long long *sum, int *mx)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int v = i < s.n ? s.nn[i] : 0;
    int m = v;
    unsigned long long t = (unsigned long long)v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t += __shfl_xor_sync(0xffffffffu, t, o);
        m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(sum, t);
        atomicMax(mx, m);
    }
}

}  // namespace

// Grids of the rebuild chain are capped (grid-stride loops inside) so that
// the common no-rebuild step pays a few microseconds of launches.
constexpr int kRebuildGrid = 152 * 8;

inline int capped(int blocks) { return blocks < kRebuildGrid ? (blocks < 1 ? 1 : blocks) : kRebuildGrid; }

int grid_blocks(const Sys &s, int kind, int persist_cap)
{
    if (s.kind != kKindCoord) {  // no neighbour list: a CV block, an atom grid, hills
        switch (kind) {
        case GK_ONE: return 1;
        case GK_ATOM256: return (s.n + 255) / 256;
        case GK_HILLS: return bias_blocks(s.K);
        case GK_DEPOSIT: return s.deposit ? bias_blocks(s.K) : 0;
        }
        return 0;
    }
    switch (kind) {
    case GK_ATOM256: return (s.n + 255) / 256;
    case GK_ATOM256_CAP: return capped((s.n + 255) / 256);
    case GK_SCAN_TILES: return (s.ncell + kScanTile - 1) / kScanTile;
    case GK_CELL128_CAP: return capped((s.ncell + 127) / 128);
    case GK_GROUPS_CAP: return persist_grid(s.n);  // Verlet rows: up to 16 blocks per SM
    case GK_ONE: return 1;
    case GK_GROUPS: {
        const int g = group_grid(s.n);
        return persist_cap > 0 && persist_cap < g ? persist_cap : g;
    }
    case GK_CV: return persist_grid(s.n);  // not tiled: its grid fixes the CV sums' order
    case GK_ATOM32: {
        const int g = (s.n + 31) / 32;
        return persist_cap > 0 && persist_cap < g ? persist_cap : g;
    }
    case GK_ATOM128: {
        const int g = (s.n + 127) / 128;
        return persist_cap > 0 && persist_cap < g ? persist_cap : g;
    }
    case GK_SUM: return sum_blocks(s.n);
    case GK_HILLS: return bias_blocks(s.K);
    case GK_DEPOSIT: return s.deposit ? bias_blocks(s.K) : 0;
    }
    return 0;
}

void launch_gather_check(const Sys &s, cudaStream_t st)
{
    k_gather_check<<<grid_blocks(s, GK_ATOM256, 0), 256, 0, st>>>(s);
}

// A kernel of the rebuild chain, launched so it may be scheduled while the
// previous kernel of the stream still runs (it waits for it on the device).
template <typename Arg>
void chained(void (*kern)(Arg), int grid, int block, cudaStream_t st, const Arg &arg)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, arg);
    if (e == cudaErrorNotSupported || e == cudaErrorInvalidValue) {
        // a stream that refuses the attribute gets a plain launch (the
        // device-side wait is then already satisfied); the refusal is this
        // launch's own error, cleared before the retry.  Any other launch
        // error stays pending for the caller's check.
        cudaGetLastError();
        cfg.numAttrs = 0;
        cudaLaunchKernelEx(&cfg, kern, arg);
    }
}

void launch_rebuild(const Sys &s, cudaStream_t st)
{
    chained(k_bin_count, grid_blocks(s, GK_ATOM256_CAP, 0), 256, st, s);
    chained(k_scan_reduce, grid_blocks(s, GK_SCAN_TILES, 0), kScanThreads, st, s);
    chained(k_scan_down, grid_blocks(s, GK_SCAN_TILES, 0), kScanThreads, st, s);
    chained(k_bin_scatter, grid_blocks(s, GK_ATOM256_CAP, 0), 256, st, s);
    chained(k_cell_sort_gather, grid_blocks(s, GK_CELL128_CAP, 0), 128, st, s);
    chained(k_verlet, grid_blocks(s, GK_GROUPS_CAP, 0), kBlockAtoms, st, s);
}

void launch_batch_gather(const BatchView &v, int total, cudaStream_t st)
{
    if (total > 0) kb_gather_check<<<total, 256, 0, st>>>(v);
}

void launch_batch_rebuild(const BatchView *rows, const int *totals, cudaStream_t st)
{
    chained(kb_bin_count, totals[GK_ATOM256_CAP], 256, st, rows[GK_ATOM256_CAP]);
    chained(kb_scan_reduce, totals[GK_SCAN_TILES], kScanThreads, st, rows[GK_SCAN_TILES]);
    chained(kb_scan_down, totals[GK_SCAN_TILES], kScanThreads, st, rows[GK_SCAN_TILES]);
    chained(kb_bin_scatter, totals[GK_ATOM256_CAP], 256, st, rows[GK_ATOM256_CAP]);
    chained(kb_cell_sort_gather, totals[GK_CELL128_CAP], 128, st, rows[GK_CELL128_CAP]);
    chained(kb_verlet, totals[GK_GROUPS_CAP], kBlockAtoms, st, rows[GK_GROUPS_CAP]);
}

void launch_filter(const Sys &s, int fp64, cudaStream_t st)
{
    if (fp64)
        k_filter<double><<<group_grid(s.n), kBlockAtoms, 0, st>>>(s);
    else
        k_filter<float><<<group_grid(s.n), kBlockAtoms, 0, st>>>(s);
}

void launch_nn_stats(const Sys &s, unsigned long long *sum, int *mx, cudaStream_t st)
{
    cudaMemsetAsync(sum, 0, sizeof(unsigned long long), st);
    cudaMemsetAsync(mx, 0, sizeof(int), st);
    k_nn_stats<<<(s.n + 255) / 256, 256, 0, st>>>(s, sum, mx);
}

void launch_export_pairs(const Sys &s, int fp64, long long *pairs, int *count, cudaStream_t st)
{
    cudaMemsetAsync(count, 0, sizeof(int), st);
    if (fp64)
        k_export_pairs<double><<<(s.n + 255) / 256, 256, 0, st>>>(s, pairs, count);
    else
        k_export_pairs<float><<<(s.n + 255) / 256, 256, 0, st>>>(s, pairs, count);
}


// The kernels of this file whose only argument is the system descriptor
// (a captured step's nodes of these can take new I/O buffers in place).
bool sys_kernel_neighbors(const void *func)
{
    static const void *const kernels[] = {
        (const void *)k_gather_check,
        (const void *)k_bin_count,
        (const void *)k_scan_reduce,
        (const void *)k_scan_down,
        (const void *)k_bin_scatter,
        (const void *)k_cell_sort_gather,
        (const void *)k_verlet,
        (const void *)k_filter<float>,
        (const void *)k_filter<double>,
    };
    for (const void *k : kernels)
        if (k == func) return true;
    return false;
}

}  // namespace metad
