// Spatial tiles of the per-step passes.
//
// The cells (edge >= rc + skin) are grouped into tiles of up to
// kTileCells^3 cells; one thread block works on one tile.  Cells are ranked
// tile by tile (tiles in Morton order, cells within a tile in z, y, x
// order), so the atoms a tile owns are one contiguous range of the sorted
// order.  A block stages, in shared memory, every atom of its tile and of the
// one-cell shell around it: each neighbour of an owned atom is there (the
// Verlet rows and the exact rows are built from cells of edge >= rc + skin).
//
// Local atom index: the staged cells in a fixed order (the tile's own cells
// first, in rank order, then the shell), atoms in cell order.  Local
// a < n_own is sorted atom atom0 + a; the neighbour lists store local
// indices (16 bits), valid while the cell order stays (until the next
// rebuild).  A tile whose staged atoms do not fit the shared-memory
// capacity reads them from global memory through the same indices (the
// same values, so the same bits).
#pragma once

#include "metad_impl.cuh"

namespace metad {

constexpr int kTileCells = 3;                // tile edge in cells
constexpr int kTileSpan = kTileCells + 2;    // staged cells per axis at most
constexpr int kMaxStagedCells = 128;         // >= kTileSpan^3 = 125
constexpr int kTileThreads = 256;            // threads per block of the tile passes
static_assert(kTileSpan * kTileSpan * kTileSpan <= kMaxStagedCells, "staged cells");
static_assert(kTileThreads >= kMaxStagedCells, "one thread per staged cell");

// Tiles per axis of a system with nc cells per axis.
__host__ __device__ inline int tiles_axis(int nc) { return (nc + kTileCells - 1) / kTileCells; }

// The staging table of one tile (shared memory).
struct TileTable {
    int ncell;       // staged cells
    int nown_cells;  // the tile's own cells (the first ncell entries)
    int n_own;       // atoms the tile owns: local 0 .. n_own - 1
    int total;       // staged atoms
    int atom0;       // sorted index of local atom 0
    int n[3];        // per axis: staged cell coordinates
    int ext[3];      // per axis: the tile's own cells
    int c[3][kTileSpan];                  // per axis: cell coordinate of each list entry
    unsigned char map[kMaxStagedCells];   // (iz n1 + iy) n0 + ix -> staged cell
    int gstart[kMaxStagedCells];          // sorted index of each staged cell's first atom
    int lstart[kMaxStagedCells + 1];      // local index of each staged cell's first atom
};

// Build the table of tile t (every thread of the block takes part; ends
// with a barrier).  Per axis the list is the own cells, then the cell below
// and the cell above (periodic), each distinct cell once: with fewer than
// kTileCells + 2 cells on an axis the shell wraps onto cells already listed.
__device__ __forceinline__ void tile_build(const Sys &s, int t, TileTable &T)
{
    __shared__ int scan_w[kMaxStagedCells / 32];
    __shared__ int halo_w[kMaxStagedCells / 32];
    if (threadIdx.x == 0) {
        const int p = s.tile_xyz[t];
        const int tc[3] = {p & 1023, (p >> 10) & 1023, p >> 20};
        for (int a = 0; a < 3; ++a) {
            const int nc = s.nc[a];
            const int c0 = tc[a] * kTileCells;
            const int e = min(kTileCells, nc - c0);
            int m = 0;
            for (int k = 0; k < e; ++k) T.c[a][m++] = c0 + k;
            const int lo = (c0 - 1 + nc) % nc, hi = (c0 + e) % nc;
            bool dup = false;
            for (int k = 0; k < m; ++k) dup = dup || T.c[a][k] == lo;
            if (!dup) T.c[a][m++] = lo;
            dup = false;
            for (int k = 0; k < m; ++k) dup = dup || T.c[a][k] == hi;
            if (!dup) T.c[a][m++] = hi;
            T.n[a] = m;
            T.ext[a] = e;
        }
        T.ncell = T.n[0] * T.n[1] * T.n[2];
        T.nown_cells = T.ext[0] * T.ext[1] * T.ext[2];
    }
    __syncthreads();
    const int q = threadIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int start = 0, cnt = 0, pos = 0;
    bool halo = false;
    if (q < T.ncell) {
        const int ix = q % T.n[0], iy = (q / T.n[0]) % T.n[1], iz = q / (T.n[0] * T.n[1]);
        const bool own = ix < T.ext[0] && iy < T.ext[1] && iz < T.ext[2];
        halo = !own;
        const int cell = s.rank_of_xyz[(T.c[2][iz] * s.nc[1] + T.c[1][iy]) * s.nc[0] + T.c[0][ix]];
        start = s.cell_start[cell];
        cnt = s.cell_start[cell + 1] - start;
        pos = (iz * T.ext[1] + iy) * T.ext[0] + ix;
    }
    // shell cells follow the own cells in q order
    const unsigned hb = __ballot_sync(0xffffffffu, halo);
    if (lane == 0 && w < kMaxStagedCells / 32) halo_w[w] = __popc(hb);
    __syncthreads();
    if (q < T.ncell) {
        if (halo) {
            int before = T.nown_cells;
            for (int k = 0; k < w; ++k) before += halo_w[k];
            pos = before + __popc(hb & ((1u << lane) - 1u));
        }
        T.map[q] = (unsigned char)pos;
        T.gstart[pos] = start;
        T.lstart[pos + 1] = cnt;  // counts, scanned below
    }
    __syncthreads();
    // inclusive scan of the counts in staged order
    int v = (q < T.ncell) ? T.lstart[q + 1] : 0;
    if (q < kMaxStagedCells) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) scan_w[w] = v;
    }
    __syncthreads();
    if (q < T.ncell) {
        int off = 0;
        for (int k = 0; k < w; ++k) off += scan_w[k];
        T.lstart[q + 1] = v + off;
    }
    if (q == 0) {
        T.lstart[0] = 0;
        T.atom0 = T.gstart[0];
    }
    __syncthreads();
    if (q == 0) {
        T.n_own = T.lstart[T.nown_cells];
        T.total = T.lstart[T.ncell];
    }
    __syncthreads();
}

// A tile's table as stored in global memory by the rebuild (it depends only
// on the cell order, fixed until the next rebuild): 80 16-byte words per
// tile.  Every pass loads its tile's table with one coalesced copy.
constexpr int kTileTableWords = 80;
static_assert(sizeof(TileTable) <= 16 * kTileTableWords, "tile table size");

__device__ __forceinline__ void tile_store(const Sys &s, int t, const TileTable &T)
{
    const int4 *src = reinterpret_cast<const int4 *>(&T);
    int4 *dst = reinterpret_cast<int4 *>(s.tile_tab) + (size_t)t * kTileTableWords;
    for (int u = threadIdx.x; u < (int)(sizeof(TileTable) + 15) / 16; u += blockDim.x) dst[u] = src[u];
}

// Load the table of tile t into shared memory (every thread of the block;
// ends with a barrier).  T must be 16-byte aligned.
__device__ __forceinline__ void tile_load(const Sys &s, int t, TileTable &T)
{
    const int4 *src = reinterpret_cast<const int4 *>(s.tile_tab) + (size_t)t * kTileTableWords;
    int4 *dst = reinterpret_cast<int4 *>(&T);
    for (int u = threadIdx.x; u < (int)(sizeof(TileTable) + 15) / 16; u += blockDim.x) dst[u] = src[u];
    __syncthreads();
}

// Neighbour rows in quad-major order: entries 4q .. 4q + 3 of atom i are one
// ushort4 at [q][i], so the threads of a warp (consecutive atoms) read a
// quad row as one contiguous 256-byte access, and a thread gets four
// entries per load.
__device__ __forceinline__ ushort4 quad_at(const unsigned short *base, size_t n, int q, int i)
{
    return reinterpret_cast<const ushort4 *>(base)[(size_t)q * n + i];
}
__device__ __forceinline__ ushort4 &quad_ref(unsigned short *base, size_t n, int q, int i)
{
    return reinterpret_cast<ushort4 *>(base)[(size_t)q * n + i];
}
__device__ __forceinline__ int quad_get(ushort4 e, int c)
{
    return c == 0 ? e.x : (c == 1 ? e.y : (c == 2 ? e.z : e.w));
}
// Entry k of atom i.
__device__ __forceinline__ unsigned short &entry_ref(unsigned short *base, size_t n, int k, int i)
{
    return base[(((size_t)(k >> 2) * n + i) << 2) + (k & 3)];
}

// Staged cell holding local atom a (a < total).
__device__ __forceinline__ int tile_cell_of(const TileTable &T, int a)
{
    int lo = 0, hi = T.ncell - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.lstart[mid] <= a) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Sorted index of local atom a.
__device__ __forceinline__ int tile_global(const TileTable &T, int a)
{
    if (a < T.n_own) return T.atom0 + a;
    const int c = tile_cell_of(T, a);
    return T.gstart[c] + (a - T.lstart[c]);
}

// ------------------------------------------------------------ staging
// Asynchronous global -> shared copies (no register round trip); the block
// waits for all of its own with stage_wait.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void stage_wait()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
}

// Dynamic shared memory of the tile kernels.
extern __shared__ __align__(16) unsigned char tile_dyn[];

// Per-atom records: 16 reals per atom in global memory; staged as
// components 0..11 (rec, 12 reals per atom) and 12..13 (pair, 2 per atom).
constexpr int kRecQ = 12;

// Stage the tile's atoms: positions (from `pos`, sorted order, unless
// nullptr) and, unless rec is nullptr, components 0..13 of the records.
// Each warp copies whole cells, a cell's atoms in groups of lanes (one lane
// per 16-byte unit).
template <typename real>
__device__ __forceinline__ void stage_tile(const TileTable &T, const float4 *pos, const real *rec, float4 *spos,
                                           real *srec, real *spair)
{
    // units per atom: the position, the 16-byte pieces of components 0..11,
    // and components 12..13 (8 bytes in FP32, 16 in FP64)
    constexpr int kQuads = kRecQ * sizeof(real) / 16;
    const int P = pos ? 1 : 0;
    const int U = P + (rec ? 1 + kQuads : 0);
    const int per = 32 / U;  // atoms per warp pass
    const int lane = threadIdx.x & 31;
    const int k = lane / U, u = lane - k * U;
    for (int c = threadIdx.x >> 5; c < T.ncell; c += kTileThreads / 32) {
        const int g0 = T.gstart[c], l0 = T.lstart[c], cnt = T.lstart[c + 1] - l0;
        for (int b = k; b < cnt && k < per; b += per) {
            const int g = g0 + b, l = l0 + b;
            if (u < P) {
                cp_async16(spos + l, pos + g);
            } else if (u - P < kQuads) {
                const int v = u - P;
                cp_async16(srec + (size_t)l * kRecQ + v * (16 / sizeof(real)),
                           rec + (size_t)g * 16 + v * (16 / sizeof(real)));
            } else if (sizeof(real) == 4) {
                cp_async8(spair + 2 * (size_t)l, rec + (size_t)g * 16 + kRecQ);
            } else {
                cp_async16(spair + 2 * (size_t)l, rec + (size_t)g * 16 + kRecQ);
            }
        }
    }
    stage_wait();
}

// The tile's own rows packed per atom in shared memory (the passes that
// read them once per entry and need no positions): quad offsets of the own
// atoms (a block scan of ceil(nn / 4)), the row quads and, per entry, the
// switch weight from the forward pass.
constexpr int kOwnCap = 512;    // own atoms of a tile whose rows are staged
constexpr int kQuadCap = 1536;  // row quads of a tile staged
__host__ __device__ constexpr int own_rows_bytes(int real_bytes)
{
    return ((kOwnCap + 1) * 4 + 15) / 16 * 16 + kQuadCap * (8 + 4 * real_bytes);
}

template <typename real>
struct OwnRows {
    int *qoff;    // [n_own + 1]
    ushort4 *jq;  // [quads]
    real *wq;     // [quads][4]
};

template <typename real>
__device__ __forceinline__ OwnRows<real> own_rows_at(unsigned char *base)
{
    OwnRows<real> o;
    o.qoff = reinterpret_cast<int *>(base);
    o.jq = reinterpret_cast<ushort4 *>(base + ((kOwnCap + 1) * 4 + 15) / 16 * 16);
    o.wq = reinterpret_cast<real *>(o.jq + kQuadCap);
    return o;
}

// Stage the own rows and weights (cp.async, waited for by the next
// stage_wait).  Returns false, the same in every thread, when they do not
// fit (the pass then reads them from global memory).
template <typename real>
__device__ __forceinline__ bool stage_own_rows(const Sys &s, const TileTable &T, const OwnRows<real> &o)
{
    __shared__ int warp_sum[kTileThreads / 32];
    __shared__ int qmax_sh;
    if (T.n_own > kOwnCap) return false;
    const size_t N = (size_t)s.n;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // each thread owns atoms 2t and 2t + 1 (kOwnCap = 2 kTileThreads)
    const int a0 = 2 * threadIdx.x, a1 = a0 + 1;
    const int q0 = a0 < T.n_own ? (s.nn[T.atom0 + a0] + 3) >> 2 : 0;
    const int q1 = a1 < T.n_own ? (s.nn[T.atom0 + a1] + 3) >> 2 : 0;
    int v = q0 + q1, incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    const int qm = __reduce_max_sync(0xffffffffu, max(q0, q1));
    if (lane == 31) warp_sum[w] = incl;
    if (threadIdx.x == 0) qmax_sh = 0;
    __syncthreads();
    if (lane == 0) atomicMax(&qmax_sh, qm);
    int before = 0;
    for (int k = 0; k < w; ++k) before += warp_sum[k];
    const int ex = before + incl - v;
    if (a0 <= T.n_own) o.qoff[a0] = ex;
    if (a1 <= T.n_own) o.qoff[a1] = ex + q0;
    __syncthreads();
    const int total = o.qoff[T.n_own];
    if (total > kQuadCap) return false;
    const int qmax = qmax_sh;
    // copy quad q of every own atom (quad rows are contiguous in the atoms)
    for (int item = threadIdx.x; item < qmax * T.n_own; item += kTileThreads) {
        const int q = item / T.n_own, a = item - q * T.n_own;
        const int base = o.qoff[a];
        if (q < o.qoff[a + 1] - base) {
            const int slot = base + q;
            const size_t src = (size_t)q * N + T.atom0 + a;
            cp_async8(o.jq + slot, reinterpret_cast<const ushort4 *>(s.elist) + src);
            const real *wsrc = reinterpret_cast<const real *>(s.wl) + 4 * src;
            cp_async16(o.wq + 4 * slot, wsrc);
            if (sizeof(real) == 8) cp_async16(o.wq + 4 * slot + 2, wsrc + 2);
        }
    }
    return true;
}

}  // namespace metad
