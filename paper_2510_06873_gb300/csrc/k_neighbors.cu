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

// Verlet row of atom i: {j : r_ij^2 < (rc + skin)^2 (1 + 1e-4)} over the
// 27 surrounding cells (each distinct cell once), entries with j > i first,
// then j < i, each part in stencil-cell order (x fastest), atoms in cell
// order.  One thread per atom, one pass over the cells: atoms are sorted by
// cell rank, so j > i is the part test, and the j > i entries fill the row
// from the front while the j < i ones fill it from the back; the back part is
// then reversed in place and moved down behind the front part.
// kImages (three or more cells along every axis): each stencil cell is a
// distinct cell at one periodic image, so the displacement is
// (r_j - r_i) + shift with the cell's image shift (0 or +-L per axis), and no
// minimum-image test per candidate.  Both roundings are sign-symmetric, so
// the pair's two directions give exactly opposite vectors and the rows stay
// symmetric.  Otherwise the minimum image per candidate.  The 1e-4 margin on
// the cutoff covers the rounding of either form (ulp(L) across the faces).
template <bool kImages>
__device__ __forceinline__ void verlet_row(const Sys &s, int i)
{
    const float4 pi = s.pos_s[i];
    const int own = s.scell[i];
    const int xyz = s.xyz_of_rank[own];
    const int cx = xyz & 1023, cy = (xyz >> 10) & 1023, cz = xyz >> 20;
    const int sx = axis_span(s.nc[0]), sy = axis_span(s.nc[1]), sz = axis_span(s.nc[2]);
    const int cap = s.max_vnb;
    int *vrow = s.vnbr + (size_t)i * cap;
    int up = 0, dn = 0;  // entries kept with j > i (front), j < i (back)
    bool over = false;   // more entries than the row holds
    for (int oz = 0; oz < sz; ++oz) {
        const int z = cz + axis_off(s.nc[2], oz);
        const float hz = z < 0 ? -s.Lhi[2] : (z >= s.nc[2] ? s.Lhi[2] : 0.0f);
        const int zr = wrap_cell(z, s.nc[2]) * s.nc[1];
        for (int oy = 0; oy < sy; ++oy) {
            const int y = cy + axis_off(s.nc[1], oy);
            const float hy = y < 0 ? -s.Lhi[1] : (y >= s.nc[1] ? s.Lhi[1] : 0.0f);
            const int yr = (zr + wrap_cell(y, s.nc[1])) * s.nc[0];
            for (int ox = 0; ox < sx; ++ox) {
                const int x = cx + axis_off(s.nc[0], ox);
                const float hx = x < 0 ? -s.Lhi[0] : (x >= s.nc[0] ? s.Lhi[0] : 0.0f);
                const int c = s.rank_of_xyz[yr + wrap_cell(x, s.nc[0])];
                const int a = s.cell_start[c], e = s.cell_start[c + 1];
#pragma unroll 4
                for (int j = a; j < e; ++j) {
                    const float4 pj = s.pos_s[j];
                    Vec3<float> d;
                    if (kImages) {
                        d.x = (pj.x - pi.x) + hx;
                        d.y = (pj.y - pi.y) + hy;
                        d.z = (pj.z - pi.z) + hz;
                    } else {
                        d = displacement<float>(s, pi, pj);
                    }
                    if (j != i && fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z)) < s.rv2) {
                        const bool fw = j > i;
                        if (up + dn < cap) {
                            vrow[fw ? up : cap - 1 - dn] = j;
                            up += fw ? 1 : 0;
                            dn += fw ? 0 : 1;
                        } else {
                            over = true;
                        }
                    }
                }
            }
        }
    }
    // the back part [cap - dn, cap) holds its first-found entry last: reverse
    // it in place, then move it down behind the front part (a copy to lower
    // addresses in increasing order never overwrites an unread entry)
    for (int t = 0; t < dn / 2; ++t) {
        const int u = vrow[cap - 1 - t], v = vrow[cap - dn + t];
        vrow[cap - 1 - t] = v;
        vrow[cap - dn + t] = u;
    }
    if (up + dn < cap)
        for (int t = 0; t < dn; ++t) vrow[up + t] = vrow[cap - dn + t];
    if (over) set_err(s, kErrCapacity);
    s.vnn[i] = up + dn;
    s.vnh[i] = up;
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

// Grid-stride over tiles of blockDim atoms, so an idle launch (no rebuild)
// retires at once.
__device__ __forceinline__ void verlet(const Sys &s, Blk k)
{
    if (!*s.flag) return;
    const bool images = s.nc[0] >= 3 && s.nc[1] >= 3 && s.nc[2] >= 3;
    const int tiles = (s.n + (int)blockDim.x - 1) / (int)blockDim.x;
    for (int it = 0, blk; (blk = work_item(k, it)) < tiles; ++it) {
        const int i = blk * (int)blockDim.x + (int)threadIdx.x;
        if (i < s.n) {
            if (images) verlet_row<true>(s, i);
            else verlet_row<false>(s, i);
        }
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
// entries with caller(i) < caller(j) appended through one counter.
__global__ void k_export_pairs(Sys s, long long *pairs, int *count)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    int ui = s.perm[i];
    for (int k = 0; k < s.nn[i]; ++k) {
        int uj = s.perm[s.nbr[(size_t)i * s.max_nb + k]];
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

void launch_export_pairs(const Sys &s, long long *pairs, int *count, cudaStream_t st)
{
    cudaMemsetAsync(count, 0, sizeof(int), st);
    k_export_pairs<<<(s.n + 255) / 256, 256, 0, st>>>(s, pairs, count);
}

}  // namespace metad
