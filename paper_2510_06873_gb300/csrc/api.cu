// C ABI of the metadynamics bias path (declared in include/metad.h).
//
// A context owns every device buffer of one system, allocated once at
// creation; the per-step calls only enqueue kernels on the context stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "metad.h"
#include "metad_impl.cuh"

using metad::Sys;

struct metad_ctx {
    metad_params p{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // metad_step runs the hill kernel on a side stream, concurrently with the
    // adjoint (which does not need dV/ds), joined before the pair forces
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    Sys sys{};
    int fp64 = 0;
    int K = 0;
    bool have_nbr = false, have_cv = false, have_bias = false;
    bool atoms_set = false;       // torsion / nearest-distance: metad_set_cv_atoms done
    bool forces_done = false;     // a bias_forces ran since the last box or CV change
    int nc_created[3] = {1, 1, 1};  // cells per axis at creation (the allocation)
    int ncell_alloc = 1;
    bool filter_pending = false;  // exact rows not yet compacted from the Verlet rows
    bool failed = false;
    std::string last_error;
    std::vector<void *> allocs;
    double *stage = nullptr;      // hill centres staged for deposit_hills
    long long *pairs = nullptr;   // export buffer (allocated on first export)
    int *pair_count = nullptr;
    int64_t pairs_cap = 0;
    double *host_pinned = nullptr;
    int *err_pinned = nullptr;
    // host-buffer step staging (allocated on first metad_step_host)
    float *pos_stage = nullptr;
    float *force_stage = nullptr;
    // stage profiling with CUDA events on the context stream
    bool prof_on = false;
    int prof_cap = 0, prof_used = 0;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_stage;
    int64_t launches = 0;
    int64_t device_bytes = 0;  // requested by cudaMalloc for this context
    // metad_step as captured CUDA graphs, each valid for the flags and hill
    // count it was captured with; a few are kept (least recently used
    // replaced).  When every kernel node takes only the descriptor, a graph
    // serves any position and force buffers: their pointers are patched into
    // the nodes' descriptors before a replay (otherwise the buffers are part
    // of the key).
    struct StepNode {
        cudaGraphNode_t node;
        metad::Sys sys;  // the node's argument as last set
    };
    struct StepGraph {
        cudaGraphExec_t exec = nullptr;
        cudaGraph_t graph = nullptr;  // kept while its nodes can be patched
        std::vector<StepNode> nodes;
        bool patchable = false;
        const float *pos = nullptr;
        float *forces = nullptr;
        int accumulate = -1;
        int deposit = -1;
        int K = -1;
        int64_t kernels = 0;
        int64_t last_use = 0;
    };
    static constexpr int kGraphs = 16;
    StepGraph graphs[kGraphs];
    int64_t graph_clock = 0;
};

namespace {

// Release a captured step (its executable graph and, if kept, the graph).
void drop_graph(metad_ctx::StepGraph &g)
{
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g.exec = nullptr;
    g.graph = nullptr;
    g.nodes.clear();
    g.patchable = false;
}

// The captured kernel nodes that take only the descriptor; false when some
// kernel node takes other arguments (its buffers cannot be patched).
bool collect_step_nodes(cudaGraph_t graph, std::vector<metad_ctx::StepNode> &out)
{
    size_t count = 0;
    if (cudaGraphGetNodes(graph, nullptr, &count) != cudaSuccess) return false;
    std::vector<cudaGraphNode_t> nodes(count);
    if (count && cudaGraphGetNodes(graph, nodes.data(), &count) != cudaSuccess) return false;
    out.clear();
    for (cudaGraphNode_t n : nodes) {
        cudaGraphNodeType type;
        if (cudaGraphNodeGetType(n, &type) != cudaSuccess) return false;
        if (type != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp = {};
        if (cudaGraphKernelNodeGetParams(n, &kp) != cudaSuccess || !kp.kernelParams) return false;
        if (!(metad::sys_kernel_neighbors(kp.func) || metad::sys_kernel_cv(kp.func) ||
              metad::sys_kernel_bias(kp.func) || metad::sys_kernel_gcv(kp.func)))
            return false;
        out.push_back({n, *static_cast<const metad::Sys *>(kp.kernelParams[0])});
    }
    return true;
}

// Point a patchable captured step at new position and force buffers: every
// descriptor that held the old ones gets the new ones.
cudaError_t patch_step_buffers(metad_ctx::StepGraph &g, const float *pos, float *forces)
{
    for (auto &sn : g.nodes) {
        metad::Sys t = sn.sys;
        if (t.pos_in == reinterpret_cast<const float4 *>(g.pos)) t.pos_in = reinterpret_cast<const float4 *>(pos);
        if (t.F_out == g.forces) t.F_out = forces;
        cudaKernelNodeParams kp = {};
        cudaError_t e = cudaGraphKernelNodeGetParams(sn.node, &kp);
        if (e != cudaSuccess) return e;
        void *args[1] = {&t};
        kp.kernelParams = args;
        kp.extra = nullptr;
        if ((e = cudaGraphExecKernelNodeSetParams(g.exec, sn.node, &kp)) != cudaSuccess) return e;
        sn.sys = t;
    }
    g.pos = pos;
    g.forces = forces;
    return cudaSuccess;
}

metad_status fail(metad_ctx *c, metad_status s, const std::string &msg)
{
    if (c) {
        c->last_error = msg;
        if (s == METAD_ERR_CUDA || s == METAD_ERR_CAPACITY || s == METAD_ERR_TIMEOUT) c->failed = true;
    }
    return s;
}

metad_status cuda_check(metad_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return METAD_OK;
    return fail(c, METAD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

metad_status launched(metad_ctx *c, const char *what) { return cuda_check(c, cudaGetLastError(), what); }

enum Stage {
    ST_BIN,
    ST_NBR,
    ST_CV_FWD,
    ST_CV_AVG,
    ST_CV_SUM,
    ST_BIAS,
    ST_ADJ,
    ST_FORCE,
    ST_FGATHER,
    ST_DEPOSIT,
    ST_OTHER,
    ST_COUNT
};
// "gather": positions into cell order + rebuild test; "neighbors": the
// conditional rebuild chain (and a stand-alone exact filter); "cv_fwd" holds
// the fused exact filter.
const char *kStageNames[ST_COUNT] = {"gather",      "neighbors",    "cv_fwd",  "cv_avg", "cv_sum", "bias", "adjoint",
                                     "force_pairs", "force_gather", "deposit", "other"};

// Brackets the kernels of one stage with CUDA events while profiling is on,
// and counts the kernels launched.
struct StageScope {
    metad_ctx *c;
    cudaStream_t st;
    int idx = -1;
    StageScope(metad_ctx *ctx, int stage, int kernels, cudaStream_t on = nullptr) : c(ctx), st(on ? on : ctx->stream)
    {
        c->launches += kernels;
        if (c->prof_on && c->prof_used < c->prof_cap) {
            idx = c->prof_used++;
            c->prof_stage[idx] = stage;
            cudaEventRecord(c->prof_ev[2 * idx], st);
        }
    }
    ~StageScope()
    {
        if (idx >= 0) cudaEventRecord(c->prof_ev[2 * idx + 1], st);
    }
};

template <typename T>
metad_status dalloc(metad_ctx *c, T **ptr, size_t count)
{
    void *p = nullptr;
    size_t bytes = sizeof(T) * (count > 0 ? count : 1);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, METAD_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    c->allocs.push_back(p);
    c->device_bytes += (int64_t)bytes;
    *ptr = static_cast<T *>(p);
    return METAD_OK;
}

// s_raw(x) = S_n(x) / S_m(x), S_k = 1 + x + ... + x^(k-1) (the device form).
double switch_raw_host(double x, int n, int m)
{
    double sn = 0.0, sm = 0.0;
    for (int t = n - 1; t >= 0; --t) sn = sn * x + 1.0;
    for (int t = m - 1; t >= 0; --t) sm = sm * x + 1.0;
    return sn / sm;
}

void split(double v, float &hi, float &lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

uint32_t spread3(uint32_t v)
{
    uint32_t r = 0;
    for (int b = 0; b < 10; ++b) r |= ((v >> b) & 1u) << (3 * b);
    return r;
}

metad_status check_usable(metad_ctx *c)
{
    if (!c) return METAD_ERR_INVALID;
    if (c->failed) return METAD_ERR_STATE;
    cudaError_t e = cudaSetDevice(c->p.device);
    if (e != cudaSuccess) return cuda_check(c, e, "cudaSetDevice");
    return METAD_OK;
}

metad_status error_word_status(metad_ctx *c, int e);

// Wait for the stream and turn a recorded device error into a status.
metad_status sync_and_check(metad_ctx *c)
{
    metad_status s = cuda_check(c, cudaMemcpyAsync(c->err_pinned, c->sys.err, sizeof(int), cudaMemcpyDeviceToHost,
                                                   c->stream), "error word copy");
    if (s != METAD_OK) return s;
    s = cuda_check(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    if (s != METAD_OK) return s;
    return error_word_status(c, *c->err_pinned);
}

// Turn a device error word into a status (the context fails on any bit).
metad_status error_word_status(metad_ctx *c, int e)
{
    if (e) c->failed = true;
    if (e & metad::kErrNonFinite) return fail(c, METAD_ERR_INVALID, "non-finite position");
    if (e & metad::kErrCapacity)
        return fail(c, METAD_ERR_CAPACITY, "an atom has more neighbours than max_neighbors");
    if (e & metad::kErrHills) return fail(c, METAD_ERR_CAPACITY, "hill list full");
    if (e) return fail(c, METAD_ERR_CUDA, "internal launch-shape check failed (error word " + std::to_string(e) + ")");
    return METAD_OK;
}

metad_status validate(const metad_params *p, std::string &why)
{
    if (!p) { why = "params is NULL"; return METAD_ERR_INVALID; }
    if (p->n_atoms < 1) { why = "n_atoms < 1"; return METAD_ERR_INVALID; }
    if (p->n_cv != 1 && p->n_cv != 2) { why = "n_cv must be 1 or 2"; return METAD_ERR_INVALID; }
    if (p->cv_kind != METAD_CV_COORDINATION && p->cv_kind != METAD_CV_TORSION && p->cv_kind != METAD_CV_NEAREST) {
        why = "unknown cv_kind";
        return METAD_ERR_INVALID;
    }
    if (p->cv_kind != METAD_CV_COORDINATION) {
        for (int a = 0; a < 3; ++a)
            if (!(p->box[a] > 0.0) || !std::isfinite(p->box[a])) {
                why = "every box length must be positive";
                return METAD_ERR_INVALID;
            }
        if (p->n_atoms < (p->cv_kind == METAD_CV_TORSION ? 4 : 2)) { why = "too few atoms"; return METAD_ERR_INVALID; }
        if (p->cv_kind == METAD_CV_TORSION && p->grid_on) { why = "no grid for torsions"; return METAD_ERR_INVALID; }
        if (!(p->softmin_beta >= 0.0) || !std::isfinite(p->softmin_beta)) {
            why = "softmin_beta must be >= 0";
            return METAD_ERR_INVALID;
        }
    } else {
        if (!(p->rc > 0) || !(p->r0 > 0)) { why = "rc and r0 must be positive"; return METAD_ERR_INVALID; }
        for (int a = 0; a < 3; ++a)
            if (!(p->box[a] >= 2.0 * p->rc) || !std::isfinite(p->box[a])) {
                why = "every box length must be >= 2 rc";
                return METAD_ERR_INVALID;
            }
        if (p->sw_n < 1 || p->sw_m < 1 || p->sw_n == p->sw_m) { why = "switch exponents"; return METAD_ERR_INVALID; }
    }
    for (int d = 0; d < p->n_cv; ++d)
        if (!(p->sigma[d] > 0)) { why = "sigma must be positive"; return METAD_ERR_INVALID; }
    if (!(p->biasfactor > 1.0) || !(p->temperature > 0) || !(p->kB > 0)) {
        why = "well-tempered parameters";
        return METAD_ERR_INVALID;
    }
    if (p->hill_capacity < 1) { why = "hill_capacity < 1"; return METAD_ERR_INVALID; }
    if (p->grid_on) {
        if (p->n_cv != 2) { why = "the grid needs n_cv == 2"; return METAD_ERR_INVALID; }
        for (int a = 0; a < 2; ++a)
            if (p->grid_n[a] < 2 || !(p->grid_hi[a] > p->grid_lo[a])) {
                why = "grid shape";
                return METAD_ERR_INVALID;
            }
    }
    if (p->precision != 0 && p->precision != 1) { why = "precision must be 0 or 1"; return METAD_ERR_INVALID; }
    if (p->lattice_cvs != 0 && p->lattice_cvs != 1) { why = "lattice_cvs must be 0 or 1"; return METAD_ERR_INVALID; }
    if (p->virial != 0 && p->virial != 1) { why = "virial must be 0 or 1"; return METAD_ERR_INVALID; }
    if ((p->lattice_cvs || p->virial) && p->cv_kind != METAD_CV_COORDINATION) {
        why = "lattice CVs and the virial need the coordination family";
        return METAD_ERR_INVALID;
    }
    if (p->lattice_cvs) {
        if (p->grid_on) { why = "no grid with lattice CVs"; return METAD_ERR_INVALID; }
        for (int a = 0; a < 3; ++a)
            if (!(p->sigma_lattice[a] > 0)) { why = "sigma_lattice must be positive"; return METAD_ERR_INVALID; }
    }
    if (p->max_neighbors < 0) { why = "max_neighbors < 0"; return METAD_ERR_INVALID; }
    if (!(p->skin >= 0.0) || !std::isfinite(p->skin)) { why = "skin must be >= 0"; return METAD_ERR_INVALID; }
    return METAD_OK;
}

constexpr double kTwoPi = 6.283185307179586476925286766559;  // the period of a torsion angle

// CVs the hills see: the per-atom CVs, then the three box lengths when they
// are CVs too.
int cv_dims(const metad_params &p) { return p.n_cv + (p.lattice_cvs ? 3 : 0); }

// Host-side geometry and constants of a context's system (no allocation).
metad_status setup_system(metad_ctx *c)
{
    Sys &y = c->sys;
    const int n = c->p.n_atoms;
    y.n = n;
    y.ncv = c->p.n_cv;
    y.kind = c->p.cv_kind;
    y.period[0] = y.period[1] = c->p.cv_kind == METAD_CV_TORSION ? kTwoPi : 0.0;
    y.inv_period[0] = y.inv_period[1] = c->p.cv_kind == METAD_CV_TORSION ? 1.0 / kTwoPi : 0.0;
    y.sm_beta = c->p.softmin_beta;
    y.cn_unlike = c->p.cn_pairs ? 1 : 0;
    y.max_nb = c->p.max_neighbors;
    for (int a = 0; a < 3; ++a) {
        const double L = c->p.box[a];
        y.L[a] = L;
        split(L, y.Lhi[a], y.Llo[a]);
        y.halfL[a] = (float)(0.5 * L);
        float lin = (float)L;
        if ((double)lin >= L) lin = std::nextafter(lin, 0.0f);
        y.Lin[a] = lin;
        // cell edge >= (rc + skin)(1 + 1e-4): float32 cell assignment can
        // never split a Verlet pair across non-adjacent cells
        int nc = (int)std::floor(L / ((c->p.rc + c->p.skin) * (1.0 + 1e-4)));
        if (nc < 1) nc = 1;
        if (nc > 1023) {
            if (c->p.cv_kind != METAD_CV_COORDINATION) nc = 1;  // no cells
            else return METAD_ERR_INVALID;
        }
        y.nc[a] = nc;
        y.inv_h[a] = (float)(nc / L);
    }
    y.ncell = y.nc[0] * y.nc[1] * y.nc[2];
    y.rc = c->p.rc;
    y.rc2 = c->p.rc * c->p.rc;
    y.rc2_lo = (float)(y.rc2 * (1.0 - 3e-5));
    y.rc2_hi = (float)(y.rc2 * (1.0 + 3e-5));
    {
        const double rv = c->p.rc + c->p.skin;
        y.rv2 = (float)(rv * rv * (1.0 + 1e-4));
        const double half = 0.5 * c->p.skin * (1.0 - 1e-3);
        y.disp_thr2 = (float)(half * half);
        y.skin_eff = (float)(c->p.skin * (1.0 - 1e-3));
        y.always_rebuild = c->p.skin > 0.0 ? 0 : 1;
        const double grow = std::pow(rv / c->p.rc, 3.0);
        y.max_vnb = ((int)std::ceil(y.max_nb * grow) + 7) / 8 * 8;
        // mirror slots put i's Verlet position (8 bits) beside j (23 bits)
        // in an entry's tag, and count exact entries in a byte
        y.mirror = (n < (1 << metad::kMirrorShift) && y.max_vnb <= 256 && y.max_nb <= 255) ? 1 : 0;
        y.vround_stride = y.max_vnb / 8;  // one u16 per 8 Verlet entries, rows packed
    }
    y.sw_n = c->p.sw_n;
    y.sw_m = c->p.sw_m;
    y.sw_nf = (float)c->p.sw_n;
    y.sw_nd = (double)c->p.sw_n;
    y.n_f = (float)n;
    y.n_d = (double)n;
    y.stretch = c->p.stretch;
    y.r0 = c->p.r0;
    y.inv_r0_d = 1.0 / c->p.r0;
    split(y.inv_r0_d, y.inv_r0_hi, y.inv_r0_lo);
    const double sc = c->p.stretch ? switch_raw_host(c->p.rc / c->p.r0, c->p.sw_n, c->p.sw_m) : 0.0;
    y.a_d = 1.0 / (1.0 - sc);
    y.k_d = sc * y.a_d;
    split(y.a_d, y.a_hi, y.a_lo);
    split(y.k_d, y.k_hi, y.k_lo);
    y.hill_cap = c->p.hill_capacity;
    y.lattice = c->p.lattice_cvs;
    y.virial = c->p.virial || c->p.lattice_cvs;
    y.D = cv_dims(c->p);
    y.hstride = std::max(y.D, 2);
    for (int d = 0; d < metad::kMaxCv; ++d) y.sigma[d] = 1.0;
    y.sigma[0] = c->p.sigma[0];
    if (c->p.n_cv == 2) y.sigma[1] = c->p.sigma[1];
    if (c->p.lattice_cvs)
        for (int a = 0; a < 3; ++a) y.sigma[c->p.n_cv + a] = c->p.sigma_lattice[a];
    for (int d = 0; d < metad::kMaxCv; ++d) y.inv2v[d] = 0.5 / (y.sigma[d] * y.sigma[d]);
    y.w0 = c->p.w0;
    y.kbdt = c->p.kB * c->p.temperature * (c->p.biasfactor - 1.0);
    y.grid_on = c->p.grid_on;
    for (int a = 0; a < 2; ++a) {
        y.gn[a] = c->p.grid_on ? c->p.grid_n[a] : 2;
        y.glo[a] = c->p.grid_lo[a];
        y.ghi[a] = c->p.grid_hi[a];
        y.gh[a] = c->p.grid_on ? (y.ghi[a] - y.glo[a]) / (y.gn[a] - 1) : 1.0;
    }
    // one FP64 partial per block of the per-atom kernels (slot 0: CN, 1: Q6),
    // three per block of the hill kernel (slot 2), the neighbour statistics
    // (slot 3)
    y.part_stride = std::max(metad::group_grid(n), metad::kMaxBiasBlocks * (metad::kMaxCv + 1));
    return METAD_OK;
}

// Morton ranks of the cells (sort cell coordinates by interleaved bits) and
// their inverse, uploaded to the rank tables (sized for the cells at
// creation; a box change never asks for more).
metad_status upload_cell_ranks(metad_ctx *c)
{
    const Sys &y = c->sys;
    std::vector<std::pair<uint32_t, int>> key(y.ncell);
    for (int z = 0; z < y.nc[2]; ++z)
        for (int yy = 0; yy < y.nc[1]; ++yy)
            for (int x = 0; x < y.nc[0]; ++x) {
                int id = (z * y.nc[1] + yy) * y.nc[0] + x;
                key[id] = {spread3(x) | (spread3(yy) << 1) | (spread3(z) << 2), id};
            }
    std::sort(key.begin(), key.end());
    std::vector<int> r(y.ncell), xr(y.ncell);
    for (int k = 0; k < y.ncell; ++k) {
        int id = key[k].second;
        int x = id % y.nc[0], yy = (id / y.nc[0]) % y.nc[1], z = id / (y.nc[0] * y.nc[1]);
        r[id] = k;
        xr[k] = x | (yy << 10) | (z << 20);
    }
    metad_status s;
    if ((s = cuda_check(c, cudaMemcpy(const_cast<int *>(y.rank_of_xyz), r.data(), sizeof(int) * y.ncell,
                                      cudaMemcpyHostToDevice), "rank upload")) ||
        (s = cuda_check(c, cudaMemcpy(const_cast<int *>(y.xyz_of_rank), xr.data(), sizeof(int) * y.ncell,
                                      cudaMemcpyHostToDevice), "rank upload")))
        return s;
    return METAD_OK;
}

// Caller centres [K][D] -> the device layout [K][hstride] (zero padded).
std::vector<double> pack_centres(const metad_ctx *c, const double *centers, int K)
{
    const int hs = c->sys.hstride, D = c->sys.D;
    std::vector<double> out((size_t)hs * K, 0.0);
    for (int k = 0; k < K; ++k)
        for (int d = 0; d < D; ++d) out[(size_t)hs * k + d] = centers[(size_t)D * k + d];
    return out;
}

struct Buffers {
    int *rank_xyz = nullptr, *xyz_rank = nullptr;
    char *rb = nullptr, *wlb = nullptr, *pfb = nullptr, *geob = nullptr, *crossb = nullptr;
};

// Every device buffer of a context in one list: alloc(&ptr, count) allocates
// count elements for ptr (or, for the size estimate, only counts them).
template <class Alloc>
metad_status state_buffers(metad_ctx *c, Buffers &b, Alloc &&alloc)
{
    Sys &y = c->sys;
    const int n = c->p.n_atoms;
    const size_t rs = c->fp64 ? sizeof(double) : sizeof(float);
    const size_t nq = c->p.n_cv == 2 ? (size_t)16 * n : 16;
    metad_status s;
    if (c->p.cv_kind != METAD_CV_COORDINATION) {
        // no neighbour list: CV atoms, gradient terms, reductions and hills
        int *atoms = nullptr, *slot = nullptr;
        if ((s = alloc(&atoms, 4 * (size_t)2 + n)) || (s = alloc(&slot, n)) || (s = alloc(&y.gcv, 32)) ||
            (s = alloc(&y.part, (size_t)y.part_stride * 4)) || (s = alloc(&y.ticket, 8)) ||
            (s = alloc(&y.scal, metad::kNumScal)) || (s = alloc(&y.err, 1)) ||
            (s = alloc(&y.hc, (size_t)y.hstride * ((size_t)y.hill_cap + 1))) ||
            (s = alloc(&y.hw, (size_t)y.hill_cap + 1)) ||
            (s = alloc(&c->stage, (size_t)y.hstride * ((size_t)y.hill_cap + 1))) ||
            (s = alloc(&y.grid, (size_t)y.gn[0] * y.gn[1] * 4)))
            return s;
        y.cv_atoms = atoms;
        y.cand_slot = slot;
        return METAD_OK;
    }
    if ((s = alloc(&y.pos_s, n)) || (s = alloc(&y.perm, n)) || (s = alloc(&y.scell, n)) ||
        (s = alloc(&y.ucell, n)) || (s = alloc(&y.uslot, n)) || (s = alloc(&y.cell_count, y.ncell)) ||
        (s = alloc(&y.cell_start, (size_t)y.ncell + 1)) || (s = alloc(&y.scan_part, y.ncell / 4096 + 2)) ||
        (s = alloc(&b.rank_xyz, y.ncell)) || (s = alloc(&b.xyz_rank, y.ncell)) ||
        (s = alloc(&y.nbr, (size_t)y.max_nb * n)) || (s = alloc(&y.nn, n)) || (s = alloc(&y.nh, n)) ||
        (s = alloc(&y.vnh, n)) || (s = alloc(&b.wlb, 2 * rs * (size_t)y.max_nb * n)) ||
        (s = alloc(&b.pfb, rs * 4 * (size_t)y.max_nb * n)) || (s = alloc(&b.geob, rs * 4 * (size_t)y.max_nb * n)) ||
        (s = alloc(&b.crossb, c->p.n_cv == 2 ? rs * (size_t)y.max_nb * n : 1)) ||
        (s = alloc(&y.pos_ref, n)) ||
        (s = alloc(&y.vnbr, (size_t)y.max_vnb * n)) || (s = alloc(&y.vnn, n)) || (s = alloc(&y.flag, 1)) ||
        (s = alloc(&y.vround, y.mirror ? (size_t)y.vround_stride * n : 1)) || (s = alloc(&y.rows_fresh, 1)) ||
        (s = alloc(&y.rebuilds, 1)) || (s = alloc(&y.Lref, 4)) || (s = alloc(&b.rb, rs * (nq * 3 + (size_t)n * 4 + 64))) ||
        (s = alloc(&y.part, (size_t)y.part_stride * 4)) || (s = alloc(&y.ticket, 8)) ||
        (s = alloc(&y.scal, metad::kNumScal)) || (s = alloc(&y.err, 1)) ||
        (s = alloc(&y.hc, (size_t)y.hstride * ((size_t)y.hill_cap + 1))) ||
        (s = alloc(&y.hw, (size_t)y.hill_cap + 1)) ||
        (s = alloc(&c->stage, (size_t)y.hstride * ((size_t)y.hill_cap + 1))) ||
        (s = alloc(&y.grid, (size_t)y.gn[0] * y.gn[1] * 4)))
        return s;
    return METAD_OK;
}

}  // namespace

extern "C" {

// The row capacity a context uses: 0 asks for 64; rows hold a multiple of
// four entries, so rows of 8 B (j, w) entries start on 32 B and every even
// entry begins a 16 B pair that lies inside its row (the Q6 and adjoint
// passes read entries two per load; the pair search reads four).
static int32_t row_capacity(int32_t max_neighbors)
{
    const int32_t m = max_neighbors == 0 ? 64 : max_neighbors;
    return (m + 3) / 4 * 4;
}

metad_status metad_estimate_bytes(const metad_params *p, int64_t *bytes)
{
    if (!bytes) return METAD_ERR_INVALID;
    *bytes = 0;
    std::string why;
    metad_status v = validate(p, why);
    if (v != METAD_OK) return v;
    metad_ctx c;
    c.p = *p;
    c.p.max_neighbors = row_capacity(c.p.max_neighbors);
    c.fp64 = c.p.precision == 1;
    if ((v = setup_system(&c))) return v;
    Buffers bf;
    int64_t total = 0;
    state_buffers(&c, bf, [&total](auto **ptr, size_t count) {
        total += (int64_t)(sizeof(**ptr) * (count > 0 ? count : 1));
        return METAD_OK;
    });
    *bytes = total;
    return METAD_OK;
}

int64_t metad_device_bytes(const metad_ctx *c) { return c ? c->device_bytes : 0; }

metad_status metad_set_step_graph(metad_ctx *c, int32_t on)
{
    if (!c) return METAD_ERR_INVALID;
    c->p.step_graph = on ? 1 : 0;
    return METAD_OK;
}

void metad_params_default(metad_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->n_atoms = 1;
    p->n_cv = 2;
    p->box[0] = p->box[1] = p->box[2] = 10.0;
    p->rc = 3.5;
    p->r0 = 2.5;
    p->sw_n = 6;
    p->sw_m = 12;
    p->stretch = 1;
    p->cn_pairs = 1;
    p->sigma[0] = 0.05;
    p->sigma[1] = 0.02;
    for (int a = 0; a < 3; ++a) p->sigma_lattice[a] = 0.1;
    p->w0 = 1.0;
    p->biasfactor = 10.0;
    p->temperature = 300.0;
    p->kB = 0.0083144626;
    p->grid_on = 0;
    p->grid_n[0] = p->grid_n[1] = 200;
    p->hill_capacity = 65536;
    p->precision = 0;
    p->max_neighbors = 64;
    p->device = 0;
    p->stream = nullptr;
    p->skin = 1.0;
}

const char *metad_status_string(metad_status s)
{
    switch (s) {
    case METAD_OK: return "ok";
    case METAD_ERR_INVALID: return "invalid argument";
    case METAD_ERR_OOM: return "out of memory";
    case METAD_ERR_CUDA: return "CUDA error";
    case METAD_ERR_CAPACITY: return "capacity exceeded";
    case METAD_ERR_TIMEOUT: return "device wait timed out";
    case METAD_ERR_STATE: return "call out of order or context failed";
    }
    return "unknown status";
}

const char *metad_last_error(const metad_ctx *c) { return c ? c->last_error.c_str() : "null context"; }

int32_t metad_hill_count(const metad_ctx *c) { return c ? c->K : 0; }

void *metad_stream(metad_ctx *c) { return c ? (void *)c->stream : nullptr; }

metad_status metad_destroy(metad_ctx *c)
{
    if (!c) return METAD_OK;
    cudaSetDevice(c->p.device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    for (void *ptr : c->allocs) cudaFree(ptr);
    if (c->host_pinned) cudaFreeHost(c->host_pinned);
    if (c->err_pinned) cudaFreeHost(c->err_pinned);
    for (auto &g : c->graphs) drop_graph(g);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    cudaGetLastError();
    delete c;
    return METAD_OK;
}

metad_status metad_create(const metad_params *p, metad_ctx **out)
{
    if (!out) return METAD_ERR_INVALID;
    *out = nullptr;
    std::string why;
    metad_status v = validate(p, why);
    if (v != METAD_OK) return v;
    metad_ctx *c = new (std::nothrow) metad_ctx();
    if (!c) return METAD_ERR_OOM;
    c->p = *p;
    c->p.max_neighbors = row_capacity(c->p.max_neighbors);
    c->fp64 = c->p.precision == 1;
    metad_status s = cuda_check(c, cudaSetDevice(c->p.device), "cudaSetDevice");
    if (s != METAD_OK) { metad_destroy(c); return s; }
    if (c->p.stream) {
        c->stream = (cudaStream_t)c->p.stream;
    } else {
        s = cuda_check(c, cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "cudaStreamCreate");
        if (s != METAD_OK) { metad_destroy(c); return s; }
        c->own_stream = true;
    }
    if ((s = setup_system(c))) {
        metad_destroy(c);
        return s;
    }
    int prio_low = 0, prio_high = 0;  // the side stream outranks the adjoint's blocks
    cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    if ((s = cuda_check(c, cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_high), "side stream")) ||
        (s = cuda_check(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "event")) ||
        (s = cuda_check(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "event"))) {
        metad_destroy(c);
        return s;
    }
    Sys &y = c->sys;
    const int n = c->p.n_atoms;
    const size_t rs = c->fp64 ? sizeof(double) : sizeof(float);
    const size_t nq = c->p.n_cv == 2 ? (size_t)16 * n : 16;
    Buffers bf;
    if ((s = state_buffers(c, bf, [c](auto **ptr, size_t count) { return dalloc(c, ptr, count); }))) {
        metad_destroy(c);
        return s;
    }
    if (c->p.cv_kind != METAD_CV_COORDINATION) {
        if (cudaMallocHost(&c->host_pinned, 64 * sizeof(double)) != cudaSuccess ||
            cudaMallocHost(&c->err_pinned, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            metad_destroy(c);
            return METAD_ERR_OOM;
        }
        cudaMemsetAsync(y.ticket, 0, 8 * sizeof(unsigned), c->stream);
        cudaMemsetAsync(y.scal, 0, metad::kNumScal * sizeof(double), c->stream);
        cudaMemsetAsync(y.err, 0, sizeof(int), c->stream);
        cudaMemsetAsync(y.gcv, 0, 32 * sizeof(double), c->stream);
        cudaMemsetAsync(y.grid, 0, sizeof(double) * (size_t)y.gn[0] * y.gn[1] * 4, c->stream);
        cudaMemsetAsync(const_cast<int *>(y.cand_slot), 0xff, sizeof(int) * (size_t)n, c->stream);  // -1
        s = cuda_check(c, cudaStreamSynchronize(c->stream), "create");
        if (s != METAD_OK) { metad_destroy(c); return s; }
        *out = c;
        return METAD_OK;
    }
    int *rank_xyz = bf.rank_xyz, *xyz_rank = bf.xyz_rank;
    char *rb = bf.rb, *wlb = bf.wlb, *pfb = bf.pfb;
    // records first (16-element rows stay 64 / 128 B aligned), scalars after
    y.q = rb;
    y.b = rb + rs * nq;
    y.h = rb + rs * 2 * nq;
    y.cn = rb + rs * 3 * nq;
    y.W = rb + rs * (3 * nq + n);
    y.qb6 = rb + rs * (3 * nq + 2 * (size_t)n);
    y.wl = wlb;
    y.pairF = pfb;
    y.cross = bf.crossb;
    y.geo = bf.geob;
    y.rank_of_xyz = rank_xyz;
    y.xyz_of_rank = xyz_rank;
    for (int a = 0; a < 3; ++a) c->nc_created[a] = y.nc[a];
    c->ncell_alloc = y.ncell;
    if ((s = upload_cell_ranks(c))) {
        metad_destroy(c);
        return s;
    }
    if (cudaMallocHost(&c->host_pinned, 64 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->err_pinned, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        metad_destroy(c);
        return METAD_ERR_OOM;
    }
    cudaMemsetAsync(y.ticket, 0, 8 * sizeof(unsigned), c->stream);
    cudaMemsetAsync(y.scal, 0, metad::kNumScal * sizeof(double), c->stream);
    cudaMemsetAsync(y.err, 0, sizeof(int), c->stream);
    cudaMemsetAsync(y.grid, 0, sizeof(double) * (size_t)y.gn[0] * y.gn[1] * 4, c->stream);
    cudaMemsetAsync(y.nn, 0, sizeof(int) * (size_t)n, c->stream);
    // the cell counters start at zero; every rebuild's scan leaves them zero
    cudaMemsetAsync(y.cell_count, 0, sizeof(int) * (size_t)c->ncell_alloc, c->stream);
    cudaMemsetAsync(y.nh, 0, sizeof(int) * (size_t)n, c->stream);
    cudaMemsetAsync(y.vnh, 0, sizeof(int) * (size_t)n, c->stream);
    cudaMemsetAsync(y.vnn, 0, sizeof(int) * (size_t)n, c->stream);
    cudaMemsetAsync(y.rebuilds, 0, sizeof(unsigned long long), c->stream);
    cudaMemsetAsync(y.rows_fresh, 0, sizeof(int), c->stream);
    {
        const float Lr[4] = {y.Lhi[0], y.Lhi[1], y.Lhi[2], 0.0f};
        if ((s = cuda_check(c, cudaMemcpy(y.Lref, Lr, sizeof(Lr), cudaMemcpyHostToDevice), "box upload"))) {
            metad_destroy(c);
            return s;
        }
    }
    cudaMemsetAsync(y.pos_ref, 0, sizeof(float4) * (size_t)n, c->stream);
    {
        // identity order until the first rebuild, which the set flag forces
        std::vector<int> iota(n);
        for (int k = 0; k < n; ++k) iota[k] = k;
        const int one = 1;
        if ((s = cuda_check(c, cudaMemcpy(y.perm, iota.data(), sizeof(int) * n, cudaMemcpyHostToDevice), "perm")) ||
            (s = cuda_check(c, cudaMemcpy(y.flag, &one, sizeof(int), cudaMemcpyHostToDevice), "flag"))) {
            metad_destroy(c);
            return s;
        }
    }
    metad::set_ylm_constants(c->stream);
    metad::configure_kernels();
    s = cuda_check(c, cudaStreamSynchronize(c->stream), "create");
    if (s != METAD_OK) { metad_destroy(c); return s; }
    *out = c;
    return METAD_OK;
}

metad_status metad_build_neighbors(metad_ctx *c, const float *pos_dev)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (!pos_dev) return fail(c, METAD_ERR_INVALID, "pos_dev is NULL");
    c->sys.pos_in = reinterpret_cast<const float4 *>(pos_dev);
    if (c->p.cv_kind != METAD_CV_COORDINATION) {  // no list: the positions are read by the CV pass
        c->have_nbr = true;
        c->have_cv = c->have_bias = false;
        return METAD_OK;
    }
    {
        StageScope t(c, ST_BIN, 1);
        metad::launch_gather_check(c->sys, c->stream);
    }
    {
        StageScope t(c, ST_NBR, 6);
        metad::launch_rebuild(c->sys, c->stream);
    }
    s = launched(c, "build_neighbors");
    if (s) return s;
    c->have_nbr = true;
    c->filter_pending = true;
    c->have_cv = c->have_bias = false;
    return METAD_OK;
}

metad_status metad_cv_forward(metad_ctx *c, double *cv_host, double *per_atom_dev)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (!c->have_nbr) return fail(c, METAD_ERR_STATE, "cv_forward before build_neighbors");
    if (c->p.cv_kind != METAD_CV_COORDINATION) {
        if (per_atom_dev) return fail(c, METAD_ERR_INVALID, "no per-atom CVs for this CV family");
        if (!c->atoms_set) return fail(c, METAD_ERR_STATE, "cv_forward before set_cv_atoms");
        StageScope t(c, ST_CV_FWD, 1);
        metad::launch_gcv_forward(c->sys, c->fp64, c->stream);
    } else {
    {
        StageScope t(c, ST_CV_FWD, 1);
        metad::launch_cv_fwd(c->sys, c->fp64, c->filter_pending ? 1 : 0, c->stream);
        c->filter_pending = false;
    }
    if (c->p.n_cv == 2) {
        StageScope t(c, ST_CV_AVG, 1);  // with the CV sums
        metad::launch_cv_avg(c->sys, c->fp64, c->stream);
    } else {
        StageScope t(c, ST_CV_SUM, 1);
        metad::launch_cv_sum(c->sys, c->fp64, c->stream);
    }
    if (per_atom_dev) {
        StageScope t(c, ST_OTHER, 1);
        metad::launch_per_atom_out(c->sys, c->fp64, per_atom_dev, c->stream);
    }
    }
    s = launched(c, "cv_forward");
    if (s) return s;
    c->have_cv = true;
    c->have_bias = false;
    if (cv_host) {
        s = cuda_check(c, cudaMemcpyAsync(c->host_pinned, c->sys.scal + metad::kS0, metad::kMaxCv * sizeof(double),
                                          cudaMemcpyDeviceToHost, c->stream), "cv copy");
        if (s) return s;
        if ((s = sync_and_check(c))) return s;
        for (int d = 0; d < c->sys.D; ++d) cv_host[d] = c->host_pinned[d];
    }
    return METAD_OK;
}

metad_status metad_bias_eval(metad_ctx *c, const double *s_host, double *V_host, double *dVds_host)
{
    metad_status s = check_usable(c);
    if (s) return s;
    const double *x = c->sys.scal + metad::kS0;
    if (s_host) {
        double tmp[metad::kMaxCv] = {};
        for (int d = 0; d < c->sys.D; ++d) tmp[d] = s_host[d];
        // a user-given CV point: evaluate into the deposit slots so the step's
        // own CVs stay untouched
        s = cuda_check(c, cudaMemcpyAsync(c->sys.scal + metad::kDepC0, tmp, sizeof(tmp), cudaMemcpyHostToDevice,
                                          c->stream), "s upload");
        if (s) return s;
        x = c->sys.scal + metad::kDepC0;
    } else if (!c->have_cv) {
        return fail(c, METAD_ERR_STATE, "bias_eval(NULL) before cv_forward");
    }
    {
        StageScope t(c, ST_BIAS, 1);
        metad::launch_bias(c->sys, c->K, x, c->sys.scal + metad::kV, 0, c->stream);
    }
    s = launched(c, "bias_eval");
    if (s) return s;
    c->have_bias = !s_host ? true : false;
    if (V_host || dVds_host) {
        s = cuda_check(c, cudaMemcpyAsync(c->host_pinned, c->sys.scal + metad::kV, (1 + metad::kMaxCv) * sizeof(double),
                                          cudaMemcpyDeviceToHost, c->stream), "bias copy");
        if (s) return s;
        if ((s = sync_and_check(c))) return s;
        if (V_host) *V_host = c->host_pinned[0];
        if (dVds_host)
            for (int d = 0; d < c->sys.D; ++d) dVds_host[d] = c->host_pinned[1 + d];
    }
    return METAD_OK;
}

metad_status metad_bias_forces(metad_ctx *c, float *forces_dev, int32_t accumulate, double scale)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (!forces_dev) return fail(c, METAD_ERR_INVALID, "forces_dev is NULL");
    if (!c->have_bias || !c->have_cv) return fail(c, METAD_ERR_STATE, "bias_forces before bias_eval");
    if (c->p.cv_kind != METAD_CV_COORDINATION) {
        {
            StageScope t(c, ST_FORCE, 1);
            metad::launch_gcv_forces(c->sys, forces_dev, accumulate ? 1 : 0, scale, c->stream);
        }
        return launched(c, "bias_forces");
    }
    c->forces_done = true;
    if (c->p.n_cv == 2) {
        StageScope t(c, ST_ADJ, 1);
        metad::launch_adjoint(c->sys, c->fp64, c->stream);
    }
    {
        StageScope t(c, ST_FORCE, 1);
        metad::launch_force_pairs(c->sys, c->fp64, scale, c->stream);
    }
    {
        StageScope t(c, ST_FGATHER, 1);
        metad::launch_force_gather(c->sys, c->fp64, forces_dev, accumulate ? 1 : 0, c->stream);
    }
    return launched(c, "bias_forces");
}

metad_status metad_set_cv_atoms(metad_ctx *c, const int32_t *atoms_host, int32_t count)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (c->p.cv_kind == METAD_CV_COORDINATION) return fail(c, METAD_ERR_INVALID, "the coordination CVs take no atoms");
    if (!atoms_host) return fail(c, METAD_ERR_INVALID, "atoms is NULL");
    const int n = c->p.n_atoms, ncv = c->p.n_cv;
    for (int k = 0; k < count; ++k)
        if (atoms_host[k] < 0 || atoms_host[k] >= n) return fail(c, METAD_ERR_INVALID, "atom index out of range");
    std::vector<int> slot(n, -1);
    if (c->p.cv_kind == METAD_CV_TORSION) {
        if (count != 4 * ncv) return fail(c, METAD_ERR_INVALID, "a torsion takes 4 atoms");
        for (int d = 0; d < ncv; ++d)
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < a; ++b)
                    if (atoms_host[4 * d + a] == atoms_host[4 * d + b])
                        return fail(c, METAD_ERR_INVALID, "an atom repeated within a torsion");
    } else {
        if (count < ncv + 1) return fail(c, METAD_ERR_INVALID, "no candidate atoms");
        for (int m = 0; m < count - ncv; ++m) {
            const int j = atoms_host[ncv + m];
            if (slot[j] >= 0) return fail(c, METAD_ERR_INVALID, "a candidate repeated");
            slot[j] = m;
        }
        for (int d = 0; d < ncv; ++d)
            if (slot[atoms_host[d]] >= 0) return fail(c, METAD_ERR_INVALID, "a reference atom is also a candidate");
        c->sys.n_cand = count - ncv;
    }
    // the buffers are sized for 8 + N entries; stream-ordered after earlier steps
    if ((s = cuda_check(c, cudaMemcpyAsync(const_cast<int *>(c->sys.cv_atoms), atoms_host, sizeof(int) * count,
                                           cudaMemcpyHostToDevice, c->stream), "atom upload")) ||
        (s = cuda_check(c, cudaMemcpyAsync(const_cast<int *>(c->sys.cand_slot), slot.data(), sizeof(int) * n,
                                           cudaMemcpyHostToDevice, c->stream), "slot upload")) ||
        (s = sync_and_check(c)))
        return s;
    c->atoms_set = true;
    c->have_cv = c->have_bias = false;
    for (auto &g : c->graphs) drop_graph(g);  // captured steps hold the old descriptor
    return METAD_OK;
}

metad_status metad_set_box(metad_ctx *c, const double *box_host)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (!box_host) return fail(c, METAD_ERR_INVALID, "box is NULL");
    if (c->p.cv_kind != METAD_CV_COORDINATION) {
        for (int a = 0; a < 3; ++a)
            if (!(box_host[a] > 0.0) || !std::isfinite(box_host[a])) return fail(c, METAD_ERR_INVALID, "box");
    } else {
        for (int a = 0; a < 3; ++a)
            if (!(box_host[a] >= 2.0 * c->p.rc) || !std::isfinite(box_host[a]))
                return fail(c, METAD_ERR_INVALID, "every box length must be >= 2 rc");
    }
    Sys &y = c->sys;
    const int nc_before[3] = {y.nc[0], y.nc[1], y.nc[2]};
    const metad_params old = c->p;
    for (int a = 0; a < 3; ++a) c->p.box[a] = box_host[a];
    if ((s = setup_system(c))) {
        c->p = old;
        setup_system(c);
        return fail(c, s, "box");
    }
    if (c->p.cv_kind == METAD_CV_COORDINATION) {
        // cells no smaller than rc + skin, no more than allocated
        if (y.ncell > c->ncell_alloc) {
            for (int a = 0; a < 3; ++a) y.nc[a] = std::min(y.nc[a], c->nc_created[a]);
            y.ncell = y.nc[0] * y.nc[1] * y.nc[2];
            for (int a = 0; a < 3; ++a) y.inv_h[a] = (float)(y.nc[a] / c->p.box[a]);
        }
        if (y.nc[0] != nc_before[0] || y.nc[1] != nc_before[1] || y.nc[2] != nc_before[2]) {
            // new cell ranks: wait for steps in flight that read the old ones
            if ((s = cuda_check(c, cudaStreamSynchronize(c->stream), "set_box")) || (s = upload_cell_ranks(c)))
                return s;
        }
        // the Verlet rows stay while the atoms' moves and the box change fit in
        // the skin (tested on the device at the next step)
        c->have_nbr = false;
    }
    c->have_cv = c->have_bias = false;
    for (auto &g : c->graphs) drop_graph(g);  // captured steps hold the old box
    return METAD_OK;
}

metad_status metad_box_gradient(metad_ctx *c, double *dVdL_host)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (!dVdL_host) return fail(c, METAD_ERR_INVALID, "output is NULL");
    if (!c->sys.virial) return fail(c, METAD_ERR_INVALID, "needs params.virial or params.lattice_cvs");
    if (!c->forces_done) return fail(c, METAD_ERR_STATE, "box_gradient before bias_forces");
    if ((s = cuda_check(c, cudaMemcpyAsync(c->host_pinned, c->sys.scal + metad::kBoxG0, 3 * sizeof(double),
                                           cudaMemcpyDeviceToHost, c->stream), "box gradient copy")) ||
        (s = sync_and_check(c)))
        return s;
    for (int a = 0; a < 3; ++a) dVdL_host[a] = c->host_pinned[a];
    return METAD_OK;
}

metad_status metad_deposit_hill(metad_ctx *c, const double *center_host, double *height_host)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (c->K >= c->p.hill_capacity) return fail(c, METAD_ERR_CAPACITY, "hill list full");
    const double *x = c->sys.scal + metad::kS0;
    if (center_host) {
        double tmp[metad::kMaxCv] = {};
        for (int d = 0; d < c->sys.D; ++d) tmp[d] = center_host[d];
        s = cuda_check(c, cudaMemcpyAsync(c->sys.scal + metad::kDepC0, tmp, sizeof(tmp), cudaMemcpyHostToDevice,
                                          c->stream), "centre upload");
        if (s) return s;
        x = c->sys.scal + metad::kDepC0;
    } else if (!c->have_cv) {
        return fail(c, METAD_ERR_STATE, "deposit_hill(NULL) before cv_forward");
    }
    {
        StageScope t(c, ST_DEPOSIT, 1);
        metad::launch_bias(c->sys, c->K, x, c->sys.scal + metad::kDepV, 1, c->stream);
    }
    s = launched(c, "deposit_hill");
    if (s) return s;
    c->K += 1;
    if (height_host) {
        s = cuda_check(c, cudaMemcpyAsync(c->host_pinned, c->sys.scal + metad::kDepW, sizeof(double),
                                          cudaMemcpyDeviceToHost, c->stream), "height copy");
        if (s) return s;
        if ((s = sync_and_check(c))) return s;
        *height_host = c->host_pinned[0];
    }
    return METAD_OK;
}

metad_status metad_deposit_hills(metad_ctx *c, const double *centers_host, int32_t K, double *heights_host)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (K < 0 || (K > 0 && !centers_host)) return fail(c, METAD_ERR_INVALID, "bad hill arguments");
    if ((int64_t)c->K + K > c->p.hill_capacity) return fail(c, METAD_ERR_CAPACITY, "hill list full");
    if (K == 0) return METAD_OK;
    const std::vector<double> tmp = pack_centres(c, centers_host, K);
    s = cuda_check(c, cudaMemcpyAsync(c->stage, tmp.data(), sizeof(double) * tmp.size(), cudaMemcpyHostToDevice,
                                      c->stream), "centre upload");
    if (s) return s;
    const int k0 = c->K;
    for (int k = 0; k < K; ++k) {
        StageScope t(c, ST_DEPOSIT, 1);
        metad::launch_bias(c->sys, c->K, c->stage + (size_t)c->sys.hstride * k, c->sys.scal + metad::kDepV, 1,
                           c->stream);
        c->K += 1;
    }
    s = launched(c, "deposit_hills");
    if (s) return s;
    if (heights_host) {
        s = cuda_check(c, cudaMemcpyAsync(heights_host, c->sys.hw + k0, sizeof(double) * K, cudaMemcpyDeviceToHost,
                                          c->stream), "heights copy");
        if (s) return s;
        return sync_and_check(c);
    }
    return METAD_OK;
}

metad_status metad_load_hills(metad_ctx *c, const double *centers_host, const double *heights_host, int32_t K)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (K < 0 || (K > 0 && (!centers_host || !heights_host))) return fail(c, METAD_ERR_INVALID, "bad hills");
    if (K > c->p.hill_capacity) return fail(c, METAD_ERR_CAPACITY, "hill list full");
    const std::vector<double> tmp = pack_centres(c, centers_host, K);
    if (K > 0) {
        if ((s = cuda_check(c, cudaMemcpyAsync(c->sys.hc, tmp.data(), sizeof(double) * tmp.size(),
                                               cudaMemcpyHostToDevice, c->stream), "hill upload")))
            return s;
        if ((s = cuda_check(c, cudaMemcpyAsync(c->sys.hw, heights_host, sizeof(double) * K, cudaMemcpyHostToDevice,
                                               c->stream), "hill upload")))
            return s;
    }
    c->K = K;
    return cuda_check(c, cudaStreamSynchronize(c->stream), "load_hills");
}

metad_status metad_get_hills(metad_ctx *c, double *centers_host, double *heights_host, int32_t cap, int32_t *K)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (K) *K = c->K;
    const int m = std::min(cap, c->K);
    if (m <= 0) return sync_and_check(c);
    const int hs = c->sys.hstride, D = c->sys.D;
    std::vector<double> tmp((size_t)hs * m);
    if (centers_host &&
        (s = cuda_check(c, cudaMemcpyAsync(tmp.data(), c->sys.hc, sizeof(double) * tmp.size(), cudaMemcpyDeviceToHost,
                                           c->stream), "hill copy")))
        return s;
    if (heights_host &&
        (s = cuda_check(c, cudaMemcpyAsync(heights_host, c->sys.hw, sizeof(double) * m, cudaMemcpyDeviceToHost,
                                           c->stream), "hill copy")))
        return s;
    if ((s = sync_and_check(c))) return s;
    if (centers_host)
        for (int k = 0; k < m; ++k)
            for (int d = 0; d < D; ++d) centers_host[(size_t)D * k + d] = tmp[(size_t)hs * k + d];
    return METAD_OK;
}

metad_status metad_fold_hills(metad_ctx *c)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (!c->p.grid_on) return fail(c, METAD_ERR_INVALID, "fold_hills needs grid_on");
    if (c->K > 0) {
        StageScope t(c, ST_OTHER, 1);
        metad::launch_grid_fold(c->sys, c->K, c->stream);
    }
    s = launched(c, "fold_hills");
    if (s) return s;
    c->K = 0;
    c->have_bias = false;
    return METAD_OK;
}

metad_status metad_get_grid(metad_ctx *c, double *grid_host)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (!c->p.grid_on || !grid_host) return fail(c, METAD_ERR_INVALID, "no grid");
    s = cuda_check(c, cudaMemcpyAsync(grid_host, c->sys.grid, sizeof(double) * c->sys.gn[0] * c->sys.gn[1] * 4,
                                      cudaMemcpyDeviceToHost, c->stream), "grid copy");
    if (s) return s;
    return sync_and_check(c);
}

metad_status metad_export_neighbors(metad_ctx *c, int64_t *pairs_host, int64_t cap, int64_t *P)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (c->p.cv_kind != METAD_CV_COORDINATION) return fail(c, METAD_ERR_INVALID, "no neighbour list");
    if (!c->have_nbr) return fail(c, METAD_ERR_STATE, "export before build_neighbors");
    const int64_t need = (int64_t)c->sys.n * c->sys.max_nb / 2 + 1;
    if (c->pairs_cap < need) {
        if ((s = dalloc(c, &c->pairs, 2 * (size_t)need)) || (s = dalloc(c, &c->pair_count, 1))) return s;
        c->pairs_cap = need;
    }
    if (c->filter_pending) {
        StageScope t(c, ST_NBR, 1);
        metad::launch_filter(c->sys, c->fp64, c->stream);
        c->filter_pending = false;
    }
    {
        StageScope t(c, ST_OTHER, 1);
        metad::launch_export_pairs(c->sys, c->fp64, c->pairs, c->pair_count, c->stream);
    }
    if ((s = launched(c, "export"))) return s;
    int cnt = 0;
    if ((s = cuda_check(c, cudaMemcpyAsync(&cnt, c->pair_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
                        "count copy")))
        return s;
    if ((s = sync_and_check(c))) return s;
    if (P) *P = cnt;
    if (!pairs_host || cap <= 0) return METAD_OK;
    std::vector<long long> tmp(2 * (size_t)cnt);
    if (cnt > 0 &&
        (s = cuda_check(c, cudaMemcpy(tmp.data(), c->pairs, sizeof(long long) * 2 * cnt, cudaMemcpyDeviceToHost),
                        "pair copy")))
        return s;
    std::vector<std::pair<long long, long long>> v(cnt);
    for (int k = 0; k < cnt; ++k) v[k] = {tmp[2 * k], tmp[2 * k + 1]};
    std::sort(v.begin(), v.end());
    const int64_t m = std::min<int64_t>(cap, cnt);
    for (int64_t k = 0; k < m; ++k) {
        pairs_host[2 * k] = v[k].first;
        pairs_host[2 * k + 1] = v[k].second;
    }
    return METAD_OK;
}

namespace {

// The torsion and nearest-distance families' whole step as one launch
// (systems of at most kFuseAtoms atoms): CVs, bias, deposit and forces.
metad_status gcv_step_fused(metad_ctx *c, const float *pos_dev, float *forces_dev, int32_t accumulate,
                            int32_t deposit)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (!pos_dev || !forces_dev) return fail(c, METAD_ERR_INVALID, "NULL buffer");
    if (!c->atoms_set) return fail(c, METAD_ERR_STATE, "step before set_cv_atoms");
    if (deposit && c->K >= c->p.hill_capacity) return fail(c, METAD_ERR_CAPACITY, "hill list full");
    c->sys.pos_in = reinterpret_cast<const float4 *>(pos_dev);
    {
        StageScope t(c, ST_CV_FWD, 1);
        metad::launch_gcv_step(c->sys, c->K, forces_dev, accumulate ? 1 : 0, deposit ? 1 : 0, c->fp64, c->stream);
    }
    if ((s = launched(c, "step"))) return s;
    c->have_nbr = c->have_cv = c->have_bias = true;
    if (deposit) c->K += 1;
    return METAD_OK;
}

// The coordination family's step with the hill kernel on the side stream,
// concurrent with the adjoint pass: the adjoint needs only the CV pass's
// records, and the pair forces (which need dV/ds) wait for the join.  The
// same kernels and arguments as the sequential calls, so the same bits.
metad_status step_overlapped(metad_ctx *c, const float *pos_dev, float *forces_dev, int32_t accumulate,
                             int32_t deposit)
{
    metad_status s;
    if ((s = metad_build_neighbors(c, pos_dev))) return s;
    if ((s = metad_cv_forward(c, nullptr, nullptr))) return s;
    if (!forces_dev) return fail(c, METAD_ERR_INVALID, "forces_dev is NULL");
    if ((s = cuda_check(c, cudaEventRecord(c->ev_fork, c->stream), "fork")) ||
        (s = cuda_check(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0), "fork")))
        return s;
    {
        StageScope t(c, ST_BIAS, 1, c->side);
        metad::launch_bias(c->sys, c->K, c->sys.scal + metad::kS0, c->sys.scal + metad::kV, 0, c->side);
    }
    if ((s = cuda_check(c, cudaEventRecord(c->ev_join, c->side), "join"))) return s;
    if (c->p.n_cv == 2) {
        StageScope t(c, ST_ADJ, 1);
        metad::launch_adjoint(c->sys, c->fp64, c->stream);
    }
    if ((s = cuda_check(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0), "join"))) return s;
    {
        StageScope t(c, ST_FORCE, 1);
        metad::launch_force_pairs(c->sys, c->fp64, 1.0, c->stream);
    }
    {
        StageScope t(c, ST_FGATHER, 1);
        metad::launch_force_gather(c->sys, c->fp64, forces_dev, accumulate ? 1 : 0, c->stream);
    }
    if ((s = launched(c, "step"))) return s;
    c->have_bias = true;
    c->forces_done = true;
    if (deposit && (s = metad_deposit_hill(c, nullptr, nullptr))) return s;
    return METAD_OK;
}

metad_status step_direct(metad_ctx *c, const float *pos_dev, float *forces_dev, int32_t accumulate, int32_t deposit)
{
    metad_status s;
    if (c && !c->failed && c->p.cv_kind != METAD_CV_COORDINATION && c->p.n_atoms <= metad::kFuseAtoms)
        return gcv_step_fused(c, pos_dev, forces_dev, accumulate, deposit);
    if (c && !c->failed && c->p.cv_kind == METAD_CV_COORDINATION)
        return step_overlapped(c, pos_dev, forces_dev, accumulate, deposit);
    if ((s = metad_build_neighbors(c, pos_dev))) return s;
    if ((s = metad_cv_forward(c, nullptr, nullptr))) return s;
    if ((s = metad_bias_eval(c, nullptr, nullptr, nullptr))) return s;
    if ((s = metad_bias_forces(c, forces_dev, accumulate, 1.0))) return s;
    if (deposit && (s = metad_deposit_hill(c, nullptr, nullptr))) return s;
    return METAD_OK;
}

// The step's kernels take the hill count and the buffers as launch
// arguments, so a captured graph is valid only for the values it was
// captured with; anything else triggers a new capture.  The rebuild
// decision is taken on the device, so one graph serves every step.
metad_status step_graph(metad_ctx *c, const float *pos_dev, float *forces_dev, int32_t accumulate, int32_t deposit)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (!pos_dev || !forces_dev) return fail(c, METAD_ERR_INVALID, "NULL buffer");
    if (deposit && c->K >= c->p.hill_capacity) return fail(c, METAD_ERR_CAPACITY, "hill list full");
    const int acc = accumulate ? 1 : 0, dep = deposit ? 1 : 0;
    metad_ctx::StepGraph *hit = nullptr, *lru = &c->graphs[0];
    bool exact = false;  // a graph captured with these very buffers
    for (auto &x : c->graphs) {
        if (x.exec && x.accumulate == acc && x.deposit == dep && x.K == c->K) {
            if (x.pos == pos_dev && x.forces == forces_dev) {
                hit = &x;
                exact = true;
            } else if (x.patchable && !exact && !hit) {
                hit = &x;  // any buffers, patched in below
            }
        }
        if (!x.exec || (lru->exec && x.last_use < lru->last_use)) lru = &x;
    }
    metad_ctx::StepGraph &g = hit ? *hit : *lru;
    g.last_use = ++c->graph_clock;
    if (hit && !exact) {
        if ((s = cuda_check(c, patch_step_buffers(g, pos_dev, forces_dev), "graph buffers"))) return s;
    }
    if (!hit) {
        drop_graph(g);
        const int K0 = c->K;
        const int64_t l0 = c->launches;
        if ((s = cuda_check(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "capture")))
            return s;
        metad_status st = step_direct(c, pos_dev, forces_dev, accumulate, deposit);  // records, and moves the
                                                                                  // host state one step on
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        if (st) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if ((s = cuda_check(c, e, "end capture"))) return s;
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        if (e == cudaSuccess && collect_step_nodes(graph, g.nodes)) {
            g.graph = graph;  // kept: its nodes take new buffers in place
            g.patchable = true;
        } else {
            g.nodes.clear();
            cudaGraphDestroy(graph);
        }
        if ((s = cuda_check(c, e, "graph instantiate"))) return s;
        g.pos = pos_dev;
        g.forces = forces_dev;
        g.accumulate = acc;
        g.deposit = dep;
        g.K = K0;
        g.kernels = c->launches - l0;
        c->launches = l0;
    } else {
        // the host state a direct step would leave
        c->sys.pos_in = reinterpret_cast<const float4 *>(pos_dev);
        c->have_nbr = c->have_cv = c->have_bias = true;
        c->forces_done = c->p.cv_kind == METAD_CV_COORDINATION;
        c->filter_pending = false;
        if (deposit) c->K += 1;
    }
    c->launches += g.kernels;
    return cuda_check(c, cudaGraphLaunch(g.exec, c->stream), "graph launch");
}

}  // namespace

metad_status metad_step(metad_ctx *c, const float *pos_dev, float *forces_dev, int32_t accumulate, int32_t deposit)
{
    if (c && c->p.step_graph && !c->prof_on) return step_graph(c, pos_dev, forces_dev, accumulate, deposit);
    return step_direct(c, pos_dev, forces_dev, accumulate, deposit);
}

metad_status metad_step_host(metad_ctx *c, const float *pos_host, float *forces_host, int32_t accumulate,
                             int32_t deposit, double *cv_host, double *V_host)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (!pos_host || !forces_host) return fail(c, METAD_ERR_INVALID, "NULL host buffer");
    const size_t n = (size_t)c->p.n_atoms;
    if (!c->pos_stage) {
        if ((s = dalloc(c, &c->pos_stage, 4 * n)) || (s = dalloc(c, &c->force_stage, 3 * n))) return s;
    }
    if ((s = cuda_check(c, cudaMemcpyAsync(c->pos_stage, pos_host, sizeof(float) * 4 * n, cudaMemcpyHostToDevice,
                                           c->stream), "position upload")))
        return s;
    if (accumulate &&
        (s = cuda_check(c, cudaMemcpyAsync(c->force_stage, forces_host, sizeof(float) * 3 * n,
                                           cudaMemcpyHostToDevice, c->stream), "force upload")))
        return s;
    if ((s = metad_step(c, c->pos_stage, c->force_stage, accumulate, deposit))) return s;
    if ((s = cuda_check(c, cudaMemcpyAsync(forces_host, c->force_stage, sizeof(float) * 3 * n,
                                           cudaMemcpyDeviceToHost, c->stream), "force download")))
        return s;
    if ((s = cuda_check(c, cudaMemcpyAsync(c->host_pinned, c->sys.scal, metad::kNumScal * sizeof(double),
                                           cudaMemcpyDeviceToHost, c->stream), "result copy")))
        return s;
    if ((s = sync_and_check(c))) return s;
    if (cv_host)
        for (int d = 0; d < c->sys.D; ++d) cv_host[d] = c->host_pinned[metad::kS0 + d];
    if (V_host) *V_host = c->host_pinned[metad::kV];
    return METAD_OK;
}

metad_status metad_profile_begin(metad_ctx *c, int32_t max_records)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (max_records < 1) return fail(c, METAD_ERR_INVALID, "max_records < 1");
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    c->prof_ev.assign(2 * (size_t)max_records, nullptr);
    c->prof_stage.assign(max_records, 0);
    for (auto &e : c->prof_ev)
        if ((s = cuda_check(c, cudaEventCreate(&e), "cudaEventCreate"))) return s;
    c->prof_cap = max_records;
    c->prof_used = 0;
    c->prof_on = true;
    return METAD_OK;
}

metad_status metad_profile_end(metad_ctx *c, double *ms_per_stage, int32_t *records_per_stage)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (!c->prof_on) return fail(c, METAD_ERR_STATE, "profiling was not started");
    c->prof_on = false;
    if ((s = sync_and_check(c))) return s;
    for (int k = 0; k < ST_COUNT; ++k) {
        if (ms_per_stage) ms_per_stage[k] = 0.0;
        if (records_per_stage) records_per_stage[k] = 0;
    }
    for (int r = 0; r < c->prof_used; ++r) {
        float ms = 0.0f;
        if ((s = cuda_check(c, cudaEventElapsedTime(&ms, c->prof_ev[2 * r], c->prof_ev[2 * r + 1]), "elapsed")))
            return s;
        if (ms_per_stage) ms_per_stage[c->prof_stage[r]] += ms;
        if (records_per_stage) records_per_stage[c->prof_stage[r]] += 1;
    }
    c->prof_used = 0;
    return METAD_OK;
}

const char *metad_stage_name(int32_t stage) { return (stage >= 0 && stage < ST_COUNT) ? kStageNames[stage] : "?"; }

int64_t metad_launch_count(const metad_ctx *c) { return c ? c->launches : 0; }

metad_status metad_rebuild_count(metad_ctx *c, int64_t *count)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (c->p.cv_kind != METAD_CV_COORDINATION) return fail(c, METAD_ERR_INVALID, "no neighbour list");
    unsigned long long v = 0;
    if ((s = cuda_check(c, cudaMemcpyAsync(&v, c->sys.rebuilds, sizeof(v), cudaMemcpyDeviceToHost, c->stream),
                        "rebuild count")))
        return s;
    if ((s = sync_and_check(c))) return s;
    if (count) *count = (int64_t)v;
    return METAD_OK;
}

metad_status metad_neighbor_stats(metad_ctx *c, int64_t *entries, int32_t *max_per_atom)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (c->p.cv_kind != METAD_CV_COORDINATION) return fail(c, METAD_ERR_INVALID, "no neighbour list");
    if (!c->have_nbr) return fail(c, METAD_ERR_STATE, "neighbor_stats before build_neighbors");
    unsigned long long *sum = reinterpret_cast<unsigned long long *>(c->sys.part + 3 * (size_t)c->sys.part_stride);
    int *mx = reinterpret_cast<int *>(sum + 1);
    if (c->filter_pending) {
        StageScope t(c, ST_NBR, 1);
        metad::launch_filter(c->sys, c->fp64, c->stream);
        c->filter_pending = false;
    }
    {
        StageScope t(c, ST_OTHER, 1);
        metad::launch_nn_stats(c->sys, sum, mx, c->stream);
    }
    if ((s = launched(c, "neighbor_stats"))) return s;
    unsigned long long hs[2] = {0, 0};
    if ((s = cuda_check(c, cudaMemcpyAsync(hs, sum, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                           c->stream), "stats copy")))
        return s;
    if ((s = sync_and_check(c))) return s;
    if (entries) *entries = (int64_t)hs[0];
    if (max_per_atom) *max_per_atom = (int32_t)(hs[1] & 0xffffffffu);
    return METAD_OK;
}

metad_status metad_read_results(metad_ctx *c, double *cv_host, double *V_host, double *dVds_host)
{
    metad_status s = check_usable(c);
    if (s) return s;
    s = cuda_check(c, cudaMemcpyAsync(c->host_pinned, c->sys.scal, metad::kNumScal * sizeof(double),
                                      cudaMemcpyDeviceToHost, c->stream), "result copy");
    if (s) return s;
    if ((s = sync_and_check(c))) return s;
    for (int d = 0; d < c->sys.D; ++d) {
        if (cv_host) cv_host[d] = c->host_pinned[metad::kS0 + d];
        if (dVds_host) dVds_host[d] = c->host_pinned[metad::kDV0 + d];
    }
    if (V_host) *V_host = c->host_pinned[metad::kV];
    return METAD_OK;
}

metad_status metad_sync(metad_ctx *c)
{
    metad_status s = check_usable(c);
    if (s) return s;
    return sync_and_check(c);
}

}  // extern "C"

// ------------------------------------------------------------------ batches

struct metad_batch {
    std::vector<metad_ctx *> ctx;
    int n = 0;
    cudaStream_t stream = nullptr;
    int device = 0, fp64 = 0, ncv = 2, kind = 0;
    int persist_cap = 0;
    // device: descriptors [n], then the block prefix rows [kGridKinds][n + 1]
    char *dev = nullptr;
    size_t sys_bytes = 0, table_bytes = 0;
    double *dout = nullptr;  // [n][4] collected results
    // pinned host ring of descriptor tables: slot k is rewritten only after
    // the copy that last read it has run
    static constexpr int kRing = 4;
    char *host[kRing] = {};
    cudaEvent_t ev[kRing] = {};
    int slot = 0;
    double *hout = nullptr;
    cudaStream_t side = nullptr;  // the hill kernel, concurrent with the adjoint
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int64_t launches = 0;
    bool stepped = false;  // the device table holds the last step's descriptors
    std::string last_error;
};

namespace {

metad_status batch_fail(metad_batch *b, metad_status s, const std::string &msg)
{
    if (b) b->last_error = msg;
    return s;
}

}  // namespace

extern "C" {

metad_status metad_batch_destroy(metad_batch *b)
{
    if (!b) return METAD_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (int k = 0; k < metad_batch::kRing; ++k) {
        if (b->ev[k]) cudaEventDestroy(b->ev[k]);
        if (b->host[k]) cudaFreeHost(b->host[k]);
    }
    if (b->hout) cudaFreeHost(b->hout);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->dev) cudaFree(b->dev);
    if (b->dout) cudaFree(b->dout);
    cudaGetLastError();
    delete b;
    return METAD_OK;
}

metad_status metad_batch_create(metad_ctx *const *ctxs, int32_t n, metad_batch **out)
{
    if (!out) return METAD_ERR_INVALID;
    *out = nullptr;
    if (!ctxs || n < 1) return METAD_ERR_INVALID;
    for (int k = 0; k < n; ++k) {
        const metad_ctx *c = ctxs[k];
        if (!c || c->failed) return METAD_ERR_INVALID;
        if (c->p.device != ctxs[0]->p.device || c->stream != ctxs[0]->stream || c->p.n_cv != ctxs[0]->p.n_cv ||
            c->fp64 != ctxs[0]->fp64 || c->p.cv_kind != ctxs[0]->p.cv_kind ||
            c->sys.virial != ctxs[0]->sys.virial)
            return METAD_ERR_INVALID;
    }
    metad_batch *b = new (std::nothrow) metad_batch();
    if (!b) return METAD_ERR_OOM;
    b->ctx.assign(ctxs, ctxs + n);
    b->n = n;
    b->stream = ctxs[0]->stream;
    b->device = ctxs[0]->p.device;
    b->fp64 = ctxs[0]->fp64;
    b->ncv = ctxs[0]->p.n_cv;
    b->kind = ctxs[0]->p.cv_kind;
    if (cudaSetDevice(b->device) != cudaSuccess) {
        metad_batch_destroy(b);
        return METAD_ERR_CUDA;
    }
    b->sys_bytes = (sizeof(Sys) * (size_t)n + 255) / 256 * 256;
    b->table_bytes = b->sys_bytes + sizeof(int) * (size_t)metad::kGridKinds * (n + 1);
    bool ok = cudaMalloc(&b->dev, b->table_bytes) == cudaSuccess &&
              cudaMalloc(&b->dout, sizeof(double) * 4 * (size_t)n) == cudaSuccess &&
              cudaMallocHost(&b->hout, sizeof(double) * 4 * (size_t)n) == cudaSuccess;
    for (int k = 0; ok && k < metad_batch::kRing; ++k)
        ok = cudaMallocHost(&b->host[k], b->table_bytes) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->ev[k], cudaEventDisableTiming) == cudaSuccess;
    int prio_low = 0, prio_high = 0;  // the side stream outranks the adjoint's blocks
    cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    ok = ok && cudaStreamCreateWithPriority(&b->side, cudaStreamNonBlocking, prio_high) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        metad_batch_destroy(b);
        return METAD_ERR_OOM;
    }
    *out = b;
    return METAD_OK;
}

metad_status metad_batch_set_tile(metad_batch *b, int32_t blocks_per_system)
{
    if (!b || blocks_per_system < 0) return METAD_ERR_INVALID;
    b->persist_cap = blocks_per_system;
    return METAD_OK;
}

metad_status metad_batch_step(metad_batch *b, const float *const *pos_dev, float *const *forces_dev,
                              int32_t accumulate, const int32_t *deposit, const int32_t *active)
{
    if (!b || !pos_dev || !forces_dev) return METAD_ERR_INVALID;
    const int n = b->n;
    bool any_deposit = false, any_active = false;
    for (int k = 0; k < n; ++k) {
        if (active && !active[k]) continue;
        any_active = true;
        metad_ctx *c = b->ctx[k];
        if (c->failed) return batch_fail(b, METAD_ERR_STATE, "system " + std::to_string(k) + " has failed");
        if (!pos_dev[k] || !forces_dev[k]) return batch_fail(b, METAD_ERR_INVALID, "NULL buffer");
        if (b->kind != METAD_CV_COORDINATION && !c->atoms_set)
            return batch_fail(b, METAD_ERR_STATE, "system " + std::to_string(k) + " has no CV atoms");
        if (deposit && deposit[k]) {
            if (c->K >= c->p.hill_capacity)
                return batch_fail(b, METAD_ERR_CAPACITY, "hill list of system " + std::to_string(k) + " full");
            any_deposit = true;
        }
    }
    if (!any_active) return METAD_OK;
    if (cudaSetDevice(b->device) != cudaSuccess) return batch_fail(b, METAD_ERR_CUDA, "cudaSetDevice");
    const int slot = b->slot;
    b->slot = (slot + 1) % metad_batch::kRing;
    if (cudaEventSynchronize(b->ev[slot]) != cudaSuccess) return batch_fail(b, METAD_ERR_CUDA, "ring event");
    Sys *hs = reinterpret_cast<Sys *>(b->host[slot]);
    int *pre = reinterpret_cast<int *>(b->host[slot] + b->sys_bytes);
    int totals[metad::kGridKinds];
    for (int g = 0; g < metad::kGridKinds; ++g) pre[g * (n + 1)] = 0;
    for (int k = 0; k < n; ++k) {
        metad_ctx *c = b->ctx[k];
        const bool on = !active || active[k];
        if (on) c->sys.pos_in = reinterpret_cast<const float4 *>(pos_dev[k]);
        Sys y = c->sys;
        y.K = c->K;
        y.deposit = on && deposit && deposit[k] ? 1 : 0;
        y.F_out = on ? forces_dev[k] : nullptr;
        y.accumulate = accumulate ? 1 : 0;
        y.fscale = 1.0;
        hs[k] = y;
        for (int g = 0; g < metad::kGridKinds; ++g)
            pre[g * (n + 1) + k + 1] = pre[g * (n + 1) + k] + (on ? metad::grid_blocks(y, g, b->persist_cap) : 0);
    }
    for (int g = 0; g < metad::kGridKinds; ++g) totals[g] = pre[g * (n + 1) + n];
    if (cudaMemcpyAsync(b->dev, b->host[slot], b->table_bytes, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaEventRecord(b->ev[slot], b->stream) != cudaSuccess)
        return batch_fail(b, METAD_ERR_CUDA, "descriptor upload");
    const Sys *dsys = reinterpret_cast<const Sys *>(b->dev);
    const int *dpre = reinterpret_cast<const int *>(b->dev + b->sys_bytes);
    metad::BatchView rows[metad::kGridKinds];
    for (int g = 0; g < metad::kGridKinds; ++g) rows[g] = metad::BatchView{dsys, dpre + g * (n + 1), n};
    if (b->kind != METAD_CV_COORDINATION) {
        bool fuse = true;
        for (int k = 0; k < n; ++k) fuse = fuse && b->ctx[k]->p.n_atoms <= metad::kFuseAtoms;
        if (fuse) {  // one launch: CVs, hills, deposits and forces
            metad::launch_batch_gcv_step(rows[metad::GK_HILLS], totals[metad::GK_HILLS], b->fp64, b->stream);
            b->launches += 1;
        } else {
            metad::launch_batch_gcv(rows[metad::GK_ONE], totals[metad::GK_ONE], b->fp64, b->stream);
            metad::launch_batch_bias(rows[metad::GK_HILLS], totals[metad::GK_HILLS], 0, b->stream);
            metad::launch_batch_gcv_forces(rows[metad::GK_ATOM256], totals[metad::GK_ATOM256], b->stream);
            if (any_deposit)
                metad::launch_batch_bias(rows[metad::GK_DEPOSIT], totals[metad::GK_DEPOSIT], 1, b->stream);
            b->launches += 3 + (any_deposit ? 1 : 0);
        }
    } else {
    metad::launch_batch_gather(rows[metad::GK_ATOM256], totals[metad::GK_ATOM256], b->stream);
    metad::launch_batch_rebuild(rows, totals, b->stream);
    metad::launch_batch_cv(rows[metad::GK_GROUPS], totals[metad::GK_GROUPS], rows[metad::GK_CV], totals[metad::GK_CV],
                           rows[metad::GK_SUM], totals[metad::GK_SUM], b->fp64, b->ncv, b->stream);
    // the hill kernel on the side stream, concurrent with the adjoint
    cudaEventRecord(b->ev_fork, b->stream);
    cudaStreamWaitEvent(b->side, b->ev_fork, 0);
    metad::launch_batch_bias(rows[metad::GK_HILLS], totals[metad::GK_HILLS], 0, b->side);
    cudaEventRecord(b->ev_join, b->side);
    metad::launch_batch_force(rows[metad::GK_GROUPS], totals[metad::GK_GROUPS], rows[metad::GK_ATOM32],
                              totals[metad::GK_ATOM32], rows[metad::GK_ATOM128], totals[metad::GK_ATOM128], b->fp64,
                              b->ncv, b->ctx[0]->sys.virial, b->stream, 1);
    cudaStreamWaitEvent(b->stream, b->ev_join, 0);
    metad::launch_batch_force(rows[metad::GK_GROUPS], totals[metad::GK_GROUPS], rows[metad::GK_ATOM32],
                              totals[metad::GK_ATOM32], rows[metad::GK_ATOM128], totals[metad::GK_ATOM128], b->fp64,
                              b->ncv, b->ctx[0]->sys.virial, b->stream, 2);
    if (any_deposit) metad::launch_batch_bias(rows[metad::GK_DEPOSIT], totals[metad::GK_DEPOSIT], 1, b->stream);
    b->launches += 1 + 6 + 2 + 1 + (b->ncv == 2 ? 3 : 2) + (any_deposit ? 1 : 0);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        for (metad_ctx *c : b->ctx) c->failed = true;
        return batch_fail(b, METAD_ERR_CUDA, std::string("batched launch: ") + cudaGetErrorString(e));
    }
    for (int k = 0; k < n; ++k) {
        if (active && !active[k]) continue;
        metad_ctx *c = b->ctx[k];
        c->have_nbr = c->have_cv = c->have_bias = true;
        c->forces_done = b->kind == METAD_CV_COORDINATION;
        c->filter_pending = false;
        if (deposit && deposit[k]) c->K += 1;
    }
    b->stepped = true;
    return METAD_OK;
}

metad_status metad_batch_read(metad_batch *b, double *cv_host, double *V_host)
{
    if (!b) return METAD_ERR_INVALID;
    if (!b->stepped) return batch_fail(b, METAD_ERR_STATE, "batch_read before batch_step");
    if (cudaSetDevice(b->device) != cudaSuccess) return batch_fail(b, METAD_ERR_CUDA, "cudaSetDevice");
    const metad::BatchView v{reinterpret_cast<const Sys *>(b->dev), nullptr, b->n};
    metad::launch_batch_collect(v, b->dout, b->stream);
    b->launches += 1;
    if (cudaMemcpyAsync(b->hout, b->dout, sizeof(double) * 4 * (size_t)b->n, cudaMemcpyDeviceToHost, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return batch_fail(b, METAD_ERR_CUDA, "batch read");
    metad_status first = METAD_OK;
    for (int k = 0; k < b->n; ++k) {
        const int e = (int)b->hout[4 * k + 3];
        if (e) {
            metad_status s = error_word_status(b->ctx[k], e);
            if (first == METAD_OK) {
                first = s;
                b->last_error = "system " + std::to_string(k) + ": " + b->ctx[k]->last_error;
            }
        }
        if (cv_host) {
            cv_host[2 * k] = b->hout[4 * k];
            cv_host[2 * k + 1] = b->ncv == 2 ? b->hout[4 * k + 1] : 0.0;
        }
        if (V_host) V_host[k] = b->hout[4 * k + 2];
    }
    return first;
}

metad_status metad_batch_collect(metad_batch *b, double *out_host)
{
    if (!b || !out_host) return METAD_ERR_INVALID;
    if (!b->stepped) return batch_fail(b, METAD_ERR_STATE, "batch_collect before batch_step");
    if (cudaSetDevice(b->device) != cudaSuccess) return batch_fail(b, METAD_ERR_CUDA, "cudaSetDevice");
    const metad::BatchView v{reinterpret_cast<const Sys *>(b->dev), nullptr, b->n};
    metad::launch_batch_collect(v, b->dout, b->stream);
    b->launches += 1;
    if (cudaMemcpyAsync(out_host, b->dout, sizeof(double) * 4 * (size_t)b->n, cudaMemcpyDeviceToHost, b->stream) !=
        cudaSuccess)
        return batch_fail(b, METAD_ERR_CUDA, "batch collect");
    return METAD_OK;
}

int64_t metad_batch_launch_count(const metad_batch *b) { return b ? b->launches : 0; }

const char *metad_batch_last_error(const metad_batch *b) { return b ? b->last_error.c_str() : "null batch"; }


// ------------------------------------------------------------------ free energy

namespace {

metad_status fes_grid_args(metad_ctx *c, const double *lo, const double *hi, const int32_t *n, int64_t &bins)
{
    if (!lo || !hi || !n) return fail(c, METAD_ERR_INVALID, "NULL grid argument");
    if (c->sys.D > 2) return fail(c, METAD_ERR_INVALID, "free-energy grids take one or two CVs");
    bins = 1;
    for (int d = 0; d < c->p.n_cv; ++d) {
        if (n[d] < 1 || !(hi[d] > lo[d])) return fail(c, METAD_ERR_INVALID, "grid shape");
        bins *= n[d];
    }
    if (bins > (1 << 24)) return fail(c, METAD_ERR_INVALID, "more than 2^24 grid points");
    return METAD_OK;
}

// A device buffer that lives for one call.
struct Scratch {
    void *p = nullptr;
    ~Scratch()
    {
        if (p) cudaFree(p);
    }
};

}  // namespace

metad_status metad_fes_grid(metad_ctx *c, const double *lo, const double *hi, const int32_t *n, double *F_host)
{
    metad_status s = check_usable(c);
    if (s) return s;
    int64_t bins = 0;
    if ((s = fes_grid_args(c, lo, hi, n, bins))) return s;
    if (!F_host) return fail(c, METAD_ERR_INVALID, "F_host is NULL");
    Scratch buf;
    if ((s = cuda_check(c, cudaMalloc(&buf.p, sizeof(double) * 2 * bins), "fes buffer"))) return s;
    double *V = static_cast<double *>(buf.p), *F = V + bins;
    const int nn[2] = {n[0], c->p.n_cv == 2 ? n[1] : 1};
    const double fac = std::isinf(c->p.biasfactor) ? 1.0 : c->p.biasfactor / (c->p.biasfactor - 1.0);
    metad::launch_fes_points(c->sys, c->K, lo, hi, nn, V, F, fac, c->stream);
    c->launches += 2;
    if ((s = launched(c, "fes_grid"))) return s;
    if ((s = cuda_check(c, cudaMemcpyAsync(F_host, F, sizeof(double) * bins, cudaMemcpyDeviceToHost, c->stream),
                        "fes copy")))
        return s;
    return sync_and_check(c);
}

metad_status metad_fes_reweight(metad_ctx *c, const double *samples_host, const double *V_host, int64_t T,
                                const double *lo, const double *hi, const int32_t *n, double *F_host)
{
    metad_status s = check_usable(c);
    if (s) return s;
    int64_t bins = 0;
    if ((s = fes_grid_args(c, lo, hi, n, bins))) return s;
    if (T < 1 || !samples_host || !V_host || !F_host) return fail(c, METAD_ERR_INVALID, "bad samples");
    const int ncv = c->p.n_cv;
    Scratch buf;
    const size_t doubles = (size_t)T * (ncv + 1) + 1 + 2 * (size_t)bins;
    if ((s = cuda_check(c, cudaMalloc(&buf.p, sizeof(double) * doubles), "reweight buffer"))) return s;
    double *S = static_cast<double *>(buf.p), *V = S + (size_t)T * ncv, *scratch = V + T, *F = scratch + 1 + bins;
    if ((s = cuda_check(c, cudaMemcpyAsync(S, samples_host, sizeof(double) * T * ncv, cudaMemcpyHostToDevice,
                                           c->stream), "sample upload")) ||
        (s = cuda_check(c, cudaMemcpyAsync(V, V_host, sizeof(double) * T, cudaMemcpyHostToDevice, c->stream),
                        "bias upload")))
        return s;
    const int nn[2] = {n[0], ncv == 2 ? n[1] : 1};
    const double beta = 1.0 / (c->p.kB * c->p.temperature);
    metad::launch_fes_reweight(S, V, T, ncv, lo, hi, nn, beta, scratch, F, c->stream);
    c->launches += 3;
    if ((s = launched(c, "fes_reweight"))) return s;
    if ((s = cuda_check(c, cudaMemcpyAsync(F_host, F, sizeof(double) * bins, cudaMemcpyDeviceToHost, c->stream),
                        "fes copy")))
        return s;
    return sync_and_check(c);
}

metad_status metad_cv_trajectory(metad_ctx *c, const float *frames_dev, int64_t T, double *cv_host)
{
    metad_status s = check_usable(c);
    if (s) return s;
    if (!frames_dev || !cv_host || T < 1) return fail(c, METAD_ERR_INVALID, "bad trajectory arguments");
    Scratch buf;
    if ((s = cuda_check(c, cudaMalloc(&buf.p, sizeof(double) * 2 * T), "trajectory buffer"))) return s;
    double *out = static_cast<double *>(buf.p);
    const size_t stride = 4 * (size_t)c->p.n_atoms;
    for (int64_t t = 0; t < T; ++t) {
        if ((s = metad_build_neighbors(c, frames_dev + stride * t))) return s;
        if ((s = metad_cv_forward(c, nullptr, nullptr))) return s;
        if ((s = cuda_check(c, cudaMemcpyAsync(out + 2 * t, c->sys.scal + metad::kS0, 2 * sizeof(double),
                                               cudaMemcpyDeviceToDevice, c->stream), "cv copy")))
            return s;
    }
    if ((s = cuda_check(c, cudaMemcpyAsync(cv_host, out, sizeof(double) * 2 * T, cudaMemcpyDeviceToHost, c->stream),
                        "trajectory copy")))
        return s;
    if ((s = sync_and_check(c))) return s;
    if (c->p.n_cv == 1)
        for (int64_t t = 0; t < T; ++t) cv_host[2 * t + 1] = 0.0;
    return METAD_OK;
}

}  // extern "C"
