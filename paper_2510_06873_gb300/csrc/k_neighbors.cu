// Steps a1-a3: ingest, tile-ranked cell order, Verlet rows, and the export
// of the exact neighbour rows.
//
// Each step:
//   k_gather_check  positions in cell order (wrapped), and a flag when any
//                   atom moved more than skin/2 since the last rebuild
//   rebuild chain   (early exit unless flagged) counting sort of the atoms
//                   into cells of edge >= rc + skin, ranked tile by tile,
//                   stable by caller index, and the Verlet rows
//                   r < rc + skin, one block per tile of cells
// The exact rows {j : r_ij^2 < rc^2} are filtered from the Verlet rows by
// the forward pass (k_cv.cu).  They are the FP64 definition bit for bit:
// while no atom has moved more than skin/2, every pair now inside rc was
// inside rc + skin at the rebuild, and the float32 estimate only decides
// outside a guard band.
#include "tiles.cuh"

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
    }
}

__device__ __forceinline__ void cell_sort_gather(const Sys &s, Blk k)
{
    if (!*s.flag) return;
    for (int c = k.b * blockDim.x + threadIdx.x; c < s.ncell; c += k.nb * blockDim.x) sort_gather_cell(s, c);
}

// End of a rebuild, run once by the last Verlet block to finish: the rows'
// box becomes the reference and the flag is cleared for the next step (kept
// set when the skin is zero, so every step rebuilds).
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
    *s.flag = s.always_rebuild ? 1 : 0;
}

// The staged-list entries along one axis that the stencil of list entry e
// touches: its cell coordinate -1, 0, +1 (periodic), each distinct cell
// once (fewer than three cells on an axis repeat coordinates).
__device__ __forceinline__ void stencil_axis(const TileTable &T, int axis, int e, int nc, int out[3], int &m)
{
    m = 0;
    const int c = T.c[axis][e];
    for (int d = -1; d <= 1; ++d) {
        const int cc = (c + d + nc) % nc;
        int j = 0;
        while (j < T.n[axis] - 1 && T.c[axis][j] != cc) ++j;  // the list holds every neighbour cell
        bool dup = false;
        for (int q = 0; q < m; ++q) dup = dup || out[q] == j;
        if (!dup) out[m++] = j;
    }
}

// Verlet rows {j : r_ij^2 < (rc + skin)^2 (1 + 1e-4)} of the tile's atoms at
// the reference positions, over the 27 surrounding cells (each distinct
// cell once): entries in stencil order (offsets z, y, x), atoms in cell
// order, stored as tile-local indices.  One thread per atom.
template <bool kStaged>
__device__ __forceinline__ void verlet_tile(const Sys &s, const TileTable &T, const float4 *spos)
{
    const size_t N = (size_t)s.n;
    for (int a = threadIdx.x; a < T.n_own; a += kTileThreads) {
        const int i = T.atom0 + a;
        const float4 pi = kStaged ? spos[a] : s.pos_ref[i];
        int lo = 0, hi = T.nown_cells - 1;  // own cell of a
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (T.lstart[mid] <= a) lo = mid;
            else hi = mid - 1;
        }
        const int ix = lo % T.ext[0], iy = (lo / T.ext[0]) % T.ext[1], iz = lo / (T.ext[0] * T.ext[1]);
        int sx[3], sy[3], sz[3], nx, ny, nz;
        stencil_axis(T, 0, ix, s.nc[0], sx, nx);
        stencil_axis(T, 1, iy, s.nc[1], sy, ny);
        stencil_axis(T, 2, iz, s.nc[2], sz, nz);
        int cnt = 0;
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const int c = T.map[(sz[z] * T.n[1] + sy[y]) * T.n[0] + sx[x]];
                    const int e = T.lstart[c + 1];
                    for (int b = T.lstart[c]; b < e; ++b) {
                        const float4 pj = kStaged ? spos[b] : s.pos_ref[tile_global(T, b)];
                        const Vec3<float> d = displacement<float>(s, pi, pj);
                        if (b != a && fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z)) < s.rv2) {
                            if (cnt < s.max_vnb) entry_ref(s.vlist, N, cnt, i) = (unsigned short)b;
                            ++cnt;
                        }
                    }
                }
        if (cnt > s.max_vnb) set_err(s, kErrCapacity);
        s.vnn[i] = min(cnt, s.max_vnb);
    }
}

// Verlet rows of the tiles b, b + nb, ... (reference positions staged in
// shared memory when they fit), then the end of the rebuild.
__device__ __forceinline__ void verlet(const Sys &s, Blk k)
{
    if (!*s.flag) return;
    __shared__ __align__(16) TileTable T;
    float4 *spos = reinterpret_cast<float4 *>(tile_dyn);
    for (int t = k.b; t < s.tiles; t += k.nb) {
        tile_build(s, t, T);
        tile_store(s, t, T);  // the passes load it until the next rebuild
        if (T.total > 65535) {  // local indices are 16-bit: empty rows, and an error
            if (threadIdx.x == 0) set_err(s, kErrCapacity);
            for (int a = threadIdx.x; a < T.n_own; a += kTileThreads) s.vnn[T.atom0 + a] = 0;
        } else if (T.total <= s.stage_cap) {
            stage_tile<float>(T, s.pos_ref, nullptr, spos, nullptr, nullptr);
            verlet_tile<true>(s, T, spos);
        } else {
            verlet_tile<false>(s, T, spos);
        }
        __syncthreads();
    }
    finish_rebuild(s, k);
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
__global__ void __launch_bounds__(kTileThreads) k_verlet(Sys s)
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
__global__ void __launch_bounds__(kTileThreads) kb_verlet(BatchView v)
{
    chain_enter();
    Blk k;
    const Sys &s = v.sys[batch_system(v, k)];
    verlet(s, k);
}

// Pairs (i < j) in caller indices, for export: one block per tile, one
// thread per owned atom, entries with caller(i) < caller(j) appended through
// one counter.
__global__ void __launch_bounds__(kTileThreads) k_export_pairs(Sys s, long long *pairs, int *count)
{
    __shared__ __align__(16) TileTable T;
    const size_t N = (size_t)s.n;
    for (int t = blockIdx.x; t < s.tiles; t += gridDim.x) {
        tile_load(s, t, T);
        for (int a = threadIdx.x; a < T.n_own; a += kTileThreads) {
            const int i = T.atom0 + a;
            const int ui = s.perm[i];
            for (int k = 0; k < s.nn[i]; ++k) {
                const int uj = s.perm[tile_global(T, (int)entry_ref(s.elist, N, k, i))];
                if (ui < uj) {
                    const int slot = atomicAdd(count, 1);
                    pairs[2 * (size_t)slot] = ui;
                    pairs[2 * (size_t)slot + 1] = uj;
                }
            }
        }
        __syncthreads();
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
    case GK_ONE: return 1;
    case GK_TILES: return persist_cap > 0 && persist_cap < s.tiles ? persist_cap : s.tiles;
    case GK_TILES_SUM: return s.tiles;
    case GK_TILES_CAP: return capped(s.tiles);
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
void chained(void (*kern)(Arg), int grid, int block, cudaStream_t st, const Arg &arg, size_t smem = 0)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
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
    chained(k_verlet, capped(s.tiles), kTileThreads, st, s, (size_t)s.stage_cap * 16);
}

void launch_batch_gather(const BatchView &v, int total, cudaStream_t st)
{
    if (total > 0) kb_gather_check<<<total, 256, 0, st>>>(v);
}

void launch_batch_rebuild(const BatchView *rows, const int *totals, int verlet_smem, cudaStream_t st)
{
    chained(kb_bin_count, totals[GK_ATOM256_CAP], 256, st, rows[GK_ATOM256_CAP]);
    chained(kb_scan_reduce, totals[GK_SCAN_TILES], kScanThreads, st, rows[GK_SCAN_TILES]);
    chained(kb_scan_down, totals[GK_SCAN_TILES], kScanThreads, st, rows[GK_SCAN_TILES]);
    chained(kb_bin_scatter, totals[GK_ATOM256_CAP], 256, st, rows[GK_ATOM256_CAP]);
    chained(kb_cell_sort_gather, totals[GK_CELL128_CAP], 128, st, rows[GK_CELL128_CAP]);
    chained(kb_verlet, totals[GK_TILES_CAP], kTileThreads, st, rows[GK_TILES_CAP], (size_t)verlet_smem);
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
    k_export_pairs<<<s.tiles > 0 ? s.tiles : 1, kTileThreads, 0, st>>>(s, pairs, count);
}

}  // namespace metad
