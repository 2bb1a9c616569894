// sw_engine.cu -- host side of the C ABI declared in include/swgpu.h:
// lattice contexts, device buffers, the per-call sweep schedule and its CUDA
// graphs.  Every step of a sweep runs in the kernels of sw_device.cuh.
#include "swgpu.h"
#include "sw_device.cuh"
#include "sw_internal.h"
#include "sw_launch.cuh"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

using namespace swg;

// ---- the kernel launches (declared in sw_launch.cuh)
namespace swg {

// Raises the tile kernels' dynamic shared-memory limit.  The attribute is
// per device, so it is set once for every device, while that device is
// current; one mutex guards the record for all callers.
constexpr int PREP_MAX_DEVICES = 64;
template <int TH>
cudaError_t tile_prepare()
{
    static std::mutex mu;
    static bool done[PREP_MAX_DEVICES] = {};
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= PREP_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return cudaSuccess;
    const void *fn[2] = {(const void *)k_tile<TH, 0>, (const void *)k_tile<TH, FEAT_TILE>};
    for (int f = 0; f < 2 && err == cudaSuccess; ++f)
        err = cudaFuncSetAttribute(fn[f], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem<TH>(true));
    if (err == cudaSuccess) done[dev] = true;
    return err;
}

template <int TH>
void launch_tile(const SweepArgs &a, bool pcc, int feat, cudaStream_t st)
{
    const size_t smem = tile_smem<TH>(pcc);
    if (pcc || (feat & FEAT_TILE))
        k_tile<TH, FEAT_TILE><<<a.n_tiles, TileCfg<TH>::NT, smem, st>>>(a);
    else
        k_tile<TH, 0><<<a.n_tiles, TileCfg<TH>::NT, smem, st>>>(a);
}

// The merge of launch group j: unions across tile edges, one round of
// pointer jumping, every node's resolved root and new spin; then for PCC
// lattices the span test and the feedback.
template <int TH, bool W>
void launch_merge_w(const SweepArgs &a, bool pcc, int n_reps, cudaStream_t st)
{
    constexpr int S = Slots<TH>::S;
    constexpr int MT = MergeCfg<TH>::MT;
    const int64_t nu = (int64_t)a.n_tiles * (TH + TW);
    const int64_t nn = (int64_t)a.n_tiles * S;
    const unsigned bu = (unsigned)((nu + MERGE_THREADS - 1) / MERGE_THREADS);
    const unsigned bn = (unsigned)((nn + MERGE_THREADS - 1) / MERGE_THREADS);
    const unsigned tiles = (unsigned)a.n_tiles;
    if (W) k_wind_init<TH><<<tiles, MT, 0, st>>>(a);
    k_merge_union<TH, W><<<tiles, MT, 0, st>>>(a);
    k_merge_jump<TH, W><<<tiles, MT, 0, st>>>(a);
    k_merge_resolve<TH, W><<<tiles, MT, 0, st>>>(a);
    if (pcc) {   // reads the compressed forest; the spins do not depend on it
        k_pcc_candidates<TH><<<bu, MERGE_THREADS, 0, st>>>(a);
        k_pcc_cover<TH><<<bn, MERGE_THREADS, 0, st>>>(a);
        k_pcc_decide<TH><<<dim3(PCC_DECIDE_BLOCKS, n_reps), 256, 0, st>>>(a, n_reps);
    }
}

template <int TH>
void launch_merge(const SweepArgs &a, bool pcc, int feat, int n_reps, cudaStream_t st)
{
    if (feat & FEAT_WIND)
        launch_merge_w<TH, true>(a, pcc, n_reps, st);
    else
        launch_merge_w<TH, false>(a, pcc, n_reps, st);
}

cudaError_t enqueue_tile(int TH, const SweepArgs &a, bool pcc, int feat, cudaStream_t st)
{
    switch (TH) {
    case 32: launch_tile<32>(a, pcc, feat, st); break;
    case 64: launch_tile<64>(a, pcc, feat, st); break;
    case 96: launch_tile<96>(a, pcc, feat, st); break;
    default: launch_tile<128>(a, pcc, feat, st); break;
    }
    return cudaGetLastError();
}

cudaError_t enqueue_merge(int TH, const SweepArgs &a, bool pcc, int feat, int n_reps, cudaStream_t st)
{
    switch (TH) {
    case 32: launch_merge<32>(a, pcc, feat, n_reps, st); break;
    case 64: launch_merge<64>(a, pcc, feat, n_reps, st); break;
    case 96: launch_merge<96>(a, pcc, feat, n_reps, st); break;
    default: launch_merge<128>(a, pcc, feat, n_reps, st); break;
    }
    return cudaGetLastError();
}

// One launch group: the tile kernel of launch j, then the merge of sweep j.
cudaError_t enqueue_launch_th(int TH, const SweepArgs &a, bool pcc, int feat, int n_reps, cudaStream_t st)
{
    cudaError_t e = enqueue_tile(TH, a, pcc, feat, st);
    if (e != cudaSuccess) return e;
    return enqueue_merge(TH, a, pcc, feat, n_reps, st);
}

cudaError_t prepare_th(int TH)
{
    switch (TH) {
    case 32: return tile_prepare<32>();
    case 64: return tile_prepare<64>();
    case 96: return tile_prepare<96>();
    default: return tile_prepare<128>();
    }
}

cudaError_t enqueue_hot_start(uint8_t *spin, int64_t N, uint64_t seed, cudaStream_t st)
{
    k_hot_start<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(spin, N, (uint32_t)seed, (uint32_t)(seed >> 32));
    return cudaGetLastError();
}

cudaError_t enqueue_job_init(uint8_t *spin, int64_t N, uint64_t seed, void *obs, int64_t obs_bytes, uint64_t *thr_dev,
                             uint64_t thr, cudaStream_t st)
{
    const int64_t n_obs = obs_bytes / 8;
    const int64_t n = std::max(N, n_obs);
    k_job_init<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(spin, N, (uint32_t)seed, (uint32_t)(seed >> 32),
                                                            static_cast<unsigned long long *>(obs), n_obs, thr_dev,
                                                            thr);
    return cudaGetLastError();
}

}  // namespace swg

namespace {

constexpr int MAX_CHUNK = 512;   // launches per captured graph

#define SW_CUDA(call)                                             \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return sw_cuda_fail(e_, __LINE__); \
    } while (0)

thread_local cudaError_t last_cuda_error = cudaSuccess;
thread_local int last_cuda_line = 0;
thread_local char last_cuda_text[160];

int sw_cuda_fail(cudaError_t e, int line = 0)
{
    last_cuda_error = e;
    last_cuda_line = line;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return SW_ERR_NOMEM;
    }
    return SW_ERR_CUDA;
}

// Tile height used for an L x L lattice: a SW_FLAG_TILE_* flag, else the
// smallest height that covers short lattices, else 96 (three CTAs fit on an
// SM, against two for 128).
int pick_tile_height(int L, uint32_t flags)
{
    if (flags & SW_FLAG_TILE_32) return 32;
    if (flags & SW_FLAG_TILE_64) return 64;
    if (flags & SW_FLAG_TILE_96) return 96;
    if (flags & SW_FLAG_TILE_128) return 128;
    if (L <= 32) return 32;
    if (L <= 64) return 64;
    if (L <= 128) return 128;
    return 96;
}

std::atomic<int> g_alloc_skip{0}, g_alloc_failures{0};   // sw_debug_fail_allocations

template <typename T>
cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    if (sw_inject_alloc_failure()) return cudaErrorMemoryAllocation;
    return cudaMalloc((void **)p, count * sizeof(T));
}

}  // namespace

bool sw_inject_alloc_failure()
{
    if (g_alloc_failures.load() <= 0) return false;
    int s = g_alloc_skip.load();
    while (s > 0)
        if (g_alloc_skip.compare_exchange_weak(s, s - 1)) return false;   // this one still succeeds
    int n = g_alloc_failures.load();
    while (n > 0)
        if (g_alloc_failures.compare_exchange_weak(n, n - 1)) return true;
    return false;
}

std::mutex &sw_capture_mutex()
{
    static std::mutex m;
    return m;
}

struct sw_ctx {
    int dev = 0;
    int32_t L = 0;
    int TH = 128;
    int tiles_x = 0, tiles_y = 0, n_tiles = 0, S = 0;
    uint64_t seed = 0;
    bool pcc = false;
    bool open = false;
    bool wind = false;
    uint64_t sweep = 0;
    uint64_t thr = 0;
    bool swept = false;

    cudaStream_t stream = nullptr;      // where work is queued
    cudaStream_t own_stream = nullptr;  // the library's default stream
    cudaStream_t cap_stream = nullptr;  // graph capture

    uint8_t *spin = nullptr;
    int32_t *label = nullptr;
    uint16_t *code = nullptr;
    uint32_t *bondbits = nullptr;
    uint32_t *cross = nullptr;
    int32_t *npar = nullptr, *nkey = nullptr;
    uint32_t *nfinal = nullptr;
    uint64_t *thr_dev = nullptr;
    Replica *rep_dev = nullptr;
    int32_t *tile_rep = nullptr;
    int32_t *jbase = nullptr;
    uint8_t *bond_bytes = nullptr;
    // PCC scratch
    uint32_t *pmask = nullptr;
    int32_t *cid = nullptr, *cand = nullptr, *ncand = nullptr;
    uint32_t *cov = nullptr;
    // cluster sizes (SW_FLAG_CSIZE)
    int32_t *psize = nullptr, *csize = nullptr;
    // topological rule (SW_FLAG_WIND)
    unsigned long long *nlink = nullptr;
    // a q-state Potts lattice (sw_create_potts): spin, label and bond_bytes
    // hold its state, the tile scratch above its tiles' codes and nodes, and
    // nstate its representatives' new states
    bool is_potts = false;
    uint8_t *nstate = nullptr;
    int4 *wlink = nullptr;   // a Potts lattice's node links under the topological rule
    PottsDev pd{};
    int64_t nsites = 0;   // L^d

    DevObs *obs = nullptr;
    int64_t obs_cap = 0, obs_head = 0, obs_tail = 0;

    Replica rep{};
    std::map<int, cudaGraphExec_t> graphs;

    // opt-in per-kernel timing (launches without graphs)
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;      // events owned by the context
    std::vector<cudaEvent_t> ev_marks;     // per launch group: tile start, tile end, merge end
    size_t ev_used = 0;
    int64_t prof_groups = 0;
    double prof_tile_ms = 0.0, prof_merge_ms = 0.0;
};

namespace {

void ctx_free(sw_ctx *c)
{
    if (!c) return;
    std::lock_guard<std::mutex> lk(sw_capture_mutex());
    cudaSetDevice(c->dev);
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    c->ev_pool.clear();
    void *ptrs[] = {c->spin, c->label, c->code, c->bondbits, c->cross, c->npar, c->nkey,
                    c->nfinal, c->thr_dev, c->rep_dev, c->tile_rep, c->jbase, c->bond_bytes, c->obs,
                    c->pmask, c->cid, c->cand, c->ncand, c->cov, c->psize, c->csize, c->nlink, c->nstate, c->wlink};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

SweepArgs args_of(const sw_ctx *c)
{
    SweepArgs a{};
    a.reps = c->rep_dev;
    a.tile_rep = c->tile_rep;
    a.n_tiles = c->n_tiles;
    a.j = 0;
    a.jbase = c->jbase;
    return a;
}

int ctx_create(sw_ctx **out, int32_t L, uint64_t thr, uint64_t seed, bool pcc, uint32_t flags)
{
    if (!out) return SW_ERR_ARG;
    *out = nullptr;
    if (L < 2 || L > 32768) return SW_ERR_ARG;
    cudaGetLastError();   // a stale error of an unrelated earlier call is not ours
    sw_ctx *c = new (std::nothrow) sw_ctx();
    if (!c) return SW_ERR_NOMEM;
    int rc = SW_OK;
    std::unique_lock<std::mutex> lk(sw_capture_mutex());
    auto fail = [&](cudaError_t e) {
        rc = sw_cuda_fail(e, __LINE__);
        lk.unlock();
        ctx_free(c);
        return rc;
    };
    cudaError_t e = cudaGetDevice(&c->dev);
    if (e != cudaSuccess) return fail(e);
    c->L = L;
    c->nsites = (int64_t)L * L;
    c->TH = pick_tile_height(L, flags);
    c->S = slots_of(c->TH);
    c->tiles_x = (L + TW - 1) / TW;
    c->tiles_y = (L + c->TH - 1) / c->TH;
    c->n_tiles = c->tiles_x * c->tiles_y;
    c->seed = seed;
    c->pcc = pcc;
    c->open = (flags & SW_FLAG_OPEN) != 0;
    c->wind = (flags & SW_FLAG_WIND) != 0;
    c->thr = thr;
    const size_t N = (size_t)L * L;
    const size_t nt = (size_t)c->n_tiles;
    if ((e = prepare_th(c->TH)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
    c->stream = c->own_stream;
    if ((e = dalloc(&c->spin, N)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->label, N)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->code, nt * c->TH * TW)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->bondbits, nt * c->TH * 2 * TWW)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->cross, nt * CROSS_WORDS)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->npar, nt * c->S)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->nkey, nt * c->S)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->nfinal, nt * c->S)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->thr_dev, 1)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->rep_dev, 1)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->tile_rep, nt)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->jbase, 1)) != cudaSuccess) return fail(e);
    if ((e = cudaMemsetAsync(c->tile_rep, 0, nt * sizeof(int32_t), c->stream)) != cudaSuccess) return fail(e);
    if (pcc) {
        const size_t ncov = (size_t)L * (c->tiles_x + c->tiles_y) * 4;
        if ((e = dalloc(&c->pmask, nt * c->S * 8)) != cudaSuccess) return fail(e);
        if ((e = dalloc(&c->cid, nt * c->S * 2)) != cudaSuccess) return fail(e);
        if ((e = dalloc(&c->cand, (size_t)2 * L)) != cudaSuccess) return fail(e);
        if ((e = dalloc(&c->ncand, 3)) != cudaSuccess) return fail(e);
        if ((e = dalloc(&c->cov, ncov)) != cudaSuccess) return fail(e);
        if ((e = cudaMemsetAsync(c->cid, 0, nt * c->S * 2 * sizeof(int32_t), c->stream)) != cudaSuccess) return fail(e);
        if ((e = cudaMemsetAsync(c->ncand, 0, 3 * sizeof(int32_t), c->stream)) != cudaSuccess) return fail(e);
        if ((e = cudaMemsetAsync(c->cov, 0, ncov * sizeof(uint32_t), c->stream)) != cudaSuccess) return fail(e);
    }
    if (flags & SW_FLAG_CSIZE) {
        if ((e = dalloc(&c->psize, nt * c->S)) != cudaSuccess) return fail(e);
        if ((e = dalloc(&c->csize, nt * c->S)) != cudaSuccess) return fail(e);
    }
    if (c->wind && (e = dalloc(&c->nlink, nt * c->S)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(c->thr_dev, &c->thr, sizeof(uint64_t), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
        return fail(e);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    k_hot_start<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>(c->spin, (int64_t)N, k0, k1);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    Replica &R = c->rep;
    R.L = L;
    R.tiles_x = c->tiles_x;
    R.tiles_y = c->tiles_y;
    R.tile_base = 0;
    R.key0 = k0;
    R.key1 = k1;
    R.nsweeps = 0;
    R.flags = (pcc ? RF_PCC : 0) | (c->open ? RF_OPEN : 0) | (c->psize ? RF_CSIZE : 0) | (c->wind ? RF_WIND : 0);
    R.sweep0 = 0;
    R.thr = thr;
    R.thr_dev = c->thr_dev;
    R.spin = c->spin;
    R.label = c->label;
    R.bond = nullptr;
    R.obs = nullptr;
    R.jstart = 0;
    R.code = c->code;
    R.bondbits = c->bondbits;
    R.cross = c->cross;
    R.npar = c->npar;
    R.nkey = c->nkey;
    R.nfinal = c->nfinal;
    R.pmask = c->pmask;
    R.cid = c->cid;
    R.cand = c->cand;
    R.ncand = c->ncand;
    R.cov = c->cov;
    R.psize = c->psize;
    R.csize = c->csize;
    R.nlink = c->nlink;
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return fail(e);
    lk.unlock();
    *out = c;
    return SW_OK;
}

// Tile-kernel features this lattice needs (FEAT_*).
int ctx_features(const sw_ctx *c)
{
    return (c->psize ? FEAT_CSIZE : 0) | (c->open ? FEAT_OPEN : 0) | (c->wind ? FEAT_WIND : 0);
}

// An NVTX range for tracing tools (free when none is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

int ensure_obs(sw_ctx *c, int64_t n)
{
    if (c->obs_head == c->obs_tail) c->obs_head = c->obs_tail = 0;
    if (c->obs_tail + n <= c->obs_cap) return SW_OK;
    const int64_t pending = c->obs_tail - c->obs_head;
    int64_t cap = c->obs_cap ? c->obs_cap : 64;
    while (cap < pending + n) cap *= 2;
    DevObs *nb = nullptr;
    std::lock_guard<std::mutex> lk(sw_capture_mutex());
    SW_CUDA(dalloc(&nb, (size_t)cap));
    if (pending > 0) {
        cudaError_t e = cudaMemcpyAsync(nb, c->obs + c->obs_head, pending * sizeof(DevObs),
                                        cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) {
            cudaFree(nb);
            return sw_cuda_fail(e);
        }
    }
    SW_CUDA(cudaStreamSynchronize(c->stream));
    if (c->obs) cudaFree(c->obs);
    c->obs = nb;
    c->obs_cap = cap;
    c->obs_head = 0;
    c->obs_tail = pending;
    return SW_OK;
}

// Graph of `m` launch groups j = 0..m-1 (offset by *jbase at run time).
int graph_for(sw_ctx *c, int m, cudaGraphExec_t *out)
{
    auto it = c->graphs.find(m);
    if (it != c->graphs.end()) {
        *out = it->second;
        return SW_OK;
    }
    cudaGraph_t g = nullptr;
    std::lock_guard<std::mutex> lk(sw_capture_mutex());
    SW_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    SweepArgs a = args_of(c);
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < m && e == cudaSuccess; ++j) {
        a.j = j;
        e = enqueue_launch_th(c->TH, a, c->pcc, ctx_features(c), 1, c->cap_stream);
    }
    cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return sw_cuda_fail(e != cudaSuccess ? e : e2);
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return sw_cuda_fail(e);
    c->graphs[m] = ex;
    *out = ex;
    return SW_OK;
}

cudaError_t next_event(sw_ctx *c, cudaEvent_t *ev)
{
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        c->ev_pool.push_back(e);
    }
    *ev = c->ev_pool[c->ev_used++];
    return cudaSuccess;
}

// Profiling mode: the same launch groups, enqueued one by one, the tile
// kernel and the three merge kernels of every group bracketed by events.
int enqueue_profiled(sw_ctx *c, int32_t n)
{
    int32_t zero = 0;
    SW_CUDA(cudaMemcpyAsync(c->jbase, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    SweepArgs a = args_of(c);
    for (int j = 0; j <= n; ++j) {
        cudaEvent_t e0, e1, e2;
        SW_CUDA(next_event(c, &e0));
        SW_CUDA(next_event(c, &e1));
        SW_CUDA(next_event(c, &e2));
        a.j = j;
        SW_CUDA(cudaEventRecord(e0, c->stream));
        SW_CUDA(enqueue_tile(c->TH, a, c->pcc, ctx_features(c), c->stream));
        SW_CUDA(cudaEventRecord(e1, c->stream));
        if (j < n) SW_CUDA(enqueue_merge(c->TH, a, c->pcc, ctx_features(c), 1, c->stream));
        SW_CUDA(cudaEventRecord(e2, c->stream));
        c->ev_marks.push_back(e0);
        c->ev_marks.push_back(e1);
        c->ev_marks.push_back(e2);
    }
    return SW_OK;
}

int run_sweeps(sw_ctx *c, int32_t n)
{
    if (n < 0) return SW_ERR_ARG;
    if (n == 0) return SW_OK;
    NvtxRange range(c->is_potts ? "sw_sweep (Potts)" : c->pcc ? "pcc_step" : "sw_sweep");
    SW_CUDA(cudaSetDevice(c->dev));
    cudaGetLastError();   // a stale error of an unrelated earlier call is not ours
    int rc = ensure_obs(c, n);
    if (rc != SW_OK) return rc;
    if (c->is_potts) {
        DevObs *obs = c->obs + c->obs_tail;
        SW_CUDA(cudaMemsetAsync(obs, 0, (size_t)n * sizeof(DevObs), c->stream));
        if (c->profiling) {
            // events around the tile kernel and the merge of every launch group
            for (int j = 0; j <= n; ++j) {
                cudaEvent_t e0, e1, e2;
                SW_CUDA(next_event(c, &e0));
                SW_CUDA(next_event(c, &e1));
                SW_CUDA(next_event(c, &e2));
                SW_CUDA(cudaEventRecord(e0, c->stream));
                SW_CUDA(potts_enqueue_tile(c->pd, j, n, c->sweep, obs, c->stream));
                SW_CUDA(cudaEventRecord(e1, c->stream));
                if (j < n) SW_CUDA(potts_enqueue_merge(c->pd, j, c->sweep, obs, c->stream));
                SW_CUDA(cudaEventRecord(e2, c->stream));
                c->ev_marks.push_back(e0);
                c->ev_marks.push_back(e1);
                c->ev_marks.push_back(e2);
            }
        } else {
            SW_CUDA(potts_enqueue_sweeps(c->pd, n, c->sweep, obs, c->stream));
        }
        c->obs_tail += n;
        c->sweep += (uint64_t)n;
        c->swept = true;
        return SW_OK;
    }
    Replica &R = c->rep;
    R.sweep0 = c->sweep;
    R.nsweeps = n;
    R.thr = c->thr;
    R.obs = c->obs + c->obs_tail;
    SW_CUDA(cudaMemcpyAsync(c->rep_dev, &R, sizeof(Replica), cudaMemcpyHostToDevice, c->stream));
    SW_CUDA(cudaMemsetAsync(R.obs, 0, (size_t)n * sizeof(DevObs), c->stream));
    if (c->profiling) {
        rc = enqueue_profiled(c, n);
        if (rc != SW_OK) return rc;
        c->obs_tail += n;
        c->sweep += (uint64_t)n;
        c->swept = true;
        return SW_OK;
    }
    // n + 1 tile launches (j = 0..n), in graph chunks of at most MAX_CHUNK
    int64_t done = 0;
    const int64_t total = (int64_t)n + 1;
    while (done < total) {
        const int m = (int)std::min<int64_t>(MAX_CHUNK, total - done);
        int32_t jb = (int32_t)done;
        SW_CUDA(cudaMemcpyAsync(c->jbase, &jb, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
        cudaGraphExec_t ex = nullptr;
        rc = graph_for(c, m, &ex);
        if (rc == SW_OK) {
            SW_CUDA(cudaGraphLaunch(ex, c->stream));
        } else {
            // capture refused (e.g. invalidated by another thread): the same
            // launch groups, enqueued directly
            cudaGetLastError();
            SweepArgs a = args_of(c);
            for (int j = 0; j < m; ++j) {
                a.j = j;
                SW_CUDA(enqueue_launch_th(c->TH, a, c->pcc, ctx_features(c), 1, c->stream));
            }
        }
        done += m;
    }
    c->obs_tail += n;
    c->sweep += (uint64_t)n;
    c->swept = true;
    return SW_OK;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

const char *sw_strerror(int code)
{
    switch (code) {
    case SW_OK: return "ok";
    case SW_PENDING: return "pending";
    case SW_ERR_ARG: return "invalid argument";
    case SW_ERR_NOMEM: return "out of memory";
    case SW_ERR_CUDA: return "CUDA error";
    case SW_ERR_TIMEOUT: return "device wait timed out";
    case SW_ERR_STATE: return "invalid state for this call";
    default: return "unknown status";
    }
}

const char *sw_last_error_detail(void)
{
    if (last_cuda_error == cudaSuccess) return "";
    std::snprintf(last_cuda_text, sizeof(last_cuda_text), "%s (sw_engine.cu:%d)",
                  cudaGetErrorString(last_cuda_error), last_cuda_line);
    return last_cuda_text;
}

int sw_threshold(double J, double T, uint64_t *out)
{
    if (!out || !(J >= 0.0) || !(T > 0.0)) return SW_ERR_ARG;
    // Sec. I step 1: P = 1 - exp(-2J/T), held as floor(P * 2^32) in [0, 2^32].
    const double P = 1.0 - std::exp(-2.0 * J / T);
    if (!(P > 0.0))
        *out = 0;
    else if (P >= 1.0)
        *out = (uint64_t)1 << 32;
    else
        *out = (uint64_t)std::floor(std::ldexp(P, 32));
    return SW_OK;
}

int sw_threshold_p_internal(double p, uint64_t *out)
{
    if (!(p >= 0.0) || !(p <= 1.0)) return SW_ERR_ARG;
    if (p == 0.0)
        *out = 0;
    else if (p == 1.0)
        *out = (uint64_t)1 << 32;
    else
        *out = (uint64_t)std::floor(std::ldexp(p, 32));
    return SW_OK;
}

int sw_create(sw_ctx **out, int32_t L, double J, double T, uint64_t seed, uint32_t flags)
{
    if (out) *out = nullptr;
    uint64_t thr = 0;
    int rc = sw_threshold(J, T, &thr);
    if (rc != SW_OK) return rc;
    return ctx_create(out, L, thr, seed, false, flags);
}

int sw_create_p(sw_ctx **out, int32_t L, double p, uint64_t seed, uint32_t flags)
{
    if (out) *out = nullptr;
    uint64_t thr = 0;
    int rc = sw_threshold_p_internal(p, &thr);
    if (rc != SW_OK) return rc;
    return ctx_create(out, L, thr, seed, false, flags);
}

int pcc_create(sw_ctx **out, int32_t L, uint64_t seed, uint32_t flags)
{
    if (out) *out = nullptr;
    return ctx_create(out, L, (uint64_t)1 << 31, seed, true, flags);   // p = 1/2
}

}  // extern "C"

namespace {

// A q-state Potts lattice (plain at threshold thr, or PCC from thr with the
// feedback on the device): the body of sw_create_potts and pcc_create_potts.
int potts_create(sw_ctx **out, int32_t dim, int32_t L, int32_t q, uint64_t thr, uint64_t seed, uint32_t flags,
                 bool pcc)
{
    if (!out) return SW_ERR_ARG;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || L < 2 || q < 2 || q > 256 ||
        (flags & ~(SW_FLAG_CSIZE | SW_FLAG_OPEN | SW_FLAG_WIND)) != 0)
        return SW_ERR_ARG;
    const int64_t N = dim == 2 ? (int64_t)L * L : (int64_t)L * L * L;
    if (N > ((int64_t)1 << 30)) return SW_ERR_ARG;
    cudaGetLastError();
    sw_ctx *c = new (std::nothrow) sw_ctx();
    if (!c) return SW_ERR_NOMEM;
    int rc = SW_OK;
    std::unique_lock<std::mutex> lk(sw_capture_mutex());
    auto fail = [&](cudaError_t e) {
        rc = sw_cuda_fail(e, __LINE__);
        lk.unlock();
        ctx_free(c);
        return rc;
    };
    cudaError_t e = cudaGetDevice(&c->dev);
    if (e != cudaSuccess) return fail(e);
    c->is_potts = true;
    c->L = L;
    c->nsites = N;
    c->seed = seed;
    c->thr = thr;
    c->pcc = pcc;
    c->open = (flags & SW_FLAG_OPEN) != 0;
    c->wind = (flags & SW_FLAG_WIND) != 0;
    if ((e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
    c->stream = c->own_stream;
    PottsGeometry g{};
    potts_geometry(dim, L, &g);
    const size_t nt = (size_t)g.ntiles, S = (size_t)g.slots;
    if ((e = dalloc(&c->spin, (size_t)N)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->label, (size_t)N)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->bond_bytes, (size_t)N)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->jbase, 1)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->code, nt * (size_t)g.sites_per_tile)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->cross, nt * (size_t)g.cross_words)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->npar, nt * S)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->nkey, nt * S)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->nfinal, nt * S)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&c->nstate, nt * S)) != cudaSuccess) return fail(e);
    if (flags & SW_FLAG_CSIZE) {
        if ((e = dalloc(&c->psize, nt * S)) != cudaSuccess) return fail(e);
        if ((e = dalloc(&c->csize, nt * S)) != cudaSuccess) return fail(e);
    }
    if (c->wind && (e = dalloc(&c->wlink, nt * S)) != cudaSuccess) return fail(e);
    PottsDev &p = c->pd;
    p.dim = dim;
    p.L = L;
    p.q = q;
    p.flags = (pcc ? RF_PCC : 0) | (c->open ? RF_OPEN : 0) | ((flags & SW_FLAG_CSIZE) ? RF_CSIZE : 0) |
              (c->wind ? RF_WIND : 0);
    p.ntx = g.ntx;
    p.nty = g.nty;
    p.ntz = g.ntz;
    p.ntiles = g.ntiles;
    p.N = N;
    p.thr = thr;
    p.seed = seed;
    p.spin = c->spin;
    p.bond = c->bond_bytes;
    p.label = c->label;
    p.code = c->code;
    p.cross = c->cross;
    p.npar = c->npar;
    p.nkey = c->nkey;
    p.nfinal = c->nfinal;
    p.nstate = c->nstate;
    p.psize = c->psize;
    p.csize = c->csize;
    p.wlink = c->wlink;
    if (pcc) {
        // per node and axis the candidate ids of roots; per axis the
        // candidates of the face (F = L^(dim-1) sites), their counts and
        // coverage (W words each); per node its piece's coordinates
        const size_t F = dim == 2 ? (size_t)L : (size_t)L * L, W = ((size_t)L + 31) / 32;
        if ((e = dalloc(&c->thr_dev, 1)) != cudaSuccess) return fail(e);
        if ((e = dalloc(&c->cid, nt * S * (size_t)dim)) != cudaSuccess) return fail(e);
        if ((e = dalloc(&c->pmask, nt * S * (size_t)g.pmask_words)) != cudaSuccess) return fail(e);
        if ((e = dalloc(&c->cand, (size_t)dim * F)) != cudaSuccess) return fail(e);
        if ((e = dalloc(&c->ncand, 4)) != cudaSuccess) return fail(e);
        if ((e = dalloc(&c->cov, (size_t)dim * F * W)) != cudaSuccess) return fail(e);
        if ((e = cudaMemsetAsync(c->cid, 0, nt * S * (size_t)dim * sizeof(int32_t), c->stream)) != cudaSuccess)
            return fail(e);
        if ((e = cudaMemsetAsync(c->ncand, 0, 4 * sizeof(int32_t), c->stream)) != cudaSuccess) return fail(e);
        if ((e = cudaMemsetAsync(c->cov, 0, (size_t)dim * F * W * sizeof(uint32_t), c->stream)) != cudaSuccess)
            return fail(e);
        if ((e = cudaMemcpyAsync(c->thr_dev, &c->thr, sizeof(uint64_t), cudaMemcpyHostToDevice, c->stream)) !=
            cudaSuccess)
            return fail(e);
        p.thr_dev = c->thr_dev;
        p.pmask = c->pmask;
        p.cid = c->cid;
        p.cand = c->cand;
        p.ncand = c->ncand;
        p.cov = c->cov;
    }
    if ((e = potts_enqueue_hot_start(p, c->stream)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return fail(e);
    lk.unlock();
    *out = c;
    return SW_OK;
}

}  // namespace

extern "C" {

int sw_create_potts(sw_ctx **out, int32_t dim, int32_t L, int32_t q, double J, double T, uint64_t seed,
                    uint32_t flags)
{
    if (!out) return SW_ERR_ARG;
    *out = nullptr;
    // P = 1 - exp(-J/T): the Ising threshold at J/2 (the same double)
    uint64_t thr = 0;
    int rc = sw_threshold(0.5 * J, T, &thr);
    if (rc != SW_OK) return rc;
    return potts_create(out, dim, L, q, thr, seed, flags, false);
}

int pcc_create_potts(sw_ctx **out, int32_t dim, int32_t L, int32_t q, uint64_t seed, uint32_t flags)
{
    return potts_create(out, dim, L, q, (uint64_t)1 << 31, seed, flags, true);   // p = 1/2
}

int sw_destroy(sw_ctx *ctx)
{
    if (!ctx) return SW_OK;
    cudaSetDevice(ctx->dev);
    cudaStreamSynchronize(ctx->stream);
    ctx_free(ctx);
    return SW_OK;
}

int sw_set_stream(sw_ctx *ctx, void *stream)
{
    if (!ctx) return SW_ERR_ARG;
    ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
    return SW_OK;
}

int sw_sweep(sw_ctx *ctx, int32_t nsweeps)
{
    if (!ctx) return SW_ERR_ARG;
    return run_sweeps(ctx, nsweeps);
}

int pcc_step(sw_ctx *ctx, int32_t nsweeps)
{
    if (!ctx) return SW_ERR_ARG;
    if (!ctx->pcc) return SW_ERR_STATE;
    return run_sweeps(ctx, nsweeps);
}

int sw_observables(sw_ctx *ctx, sw_obs *out, int32_t max, int32_t *n_written)
{
    if (!ctx || max < 0 || (max > 0 && !out) || !n_written) return SW_ERR_ARG;
    *n_written = 0;
    SW_CUDA(cudaSetDevice(ctx->dev));
    const int64_t pending = ctx->obs_tail - ctx->obs_head;
    const int64_t n = std::min<int64_t>(pending, max);
    if (n > 0) {
        SW_CUDA(cudaMemcpyAsync(out, ctx->obs + ctx->obs_head, (size_t)n * sizeof(sw_obs),
                                cudaMemcpyDeviceToHost, ctx->stream));
    }
    SW_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->obs_head += n;
    *n_written = (int32_t)n;
    return SW_OK;
}

int sw_get_spins(sw_ctx *ctx, uint8_t *host_out)
{
    if (!ctx || !host_out) return SW_ERR_ARG;
    SW_CUDA(cudaSetDevice(ctx->dev));
    SW_CUDA(cudaMemcpyAsync(host_out, ctx->spin, (size_t)ctx->nsites, cudaMemcpyDeviceToHost, ctx->stream));
    SW_CUDA(cudaStreamSynchronize(ctx->stream));
    return SW_OK;
}

int sw_set_spins(sw_ctx *ctx, const uint8_t *host_in)
{
    if (!ctx || !host_in) return SW_ERR_ARG;
    const size_t N = (size_t)ctx->nsites;
    SW_CUDA(cudaSetDevice(ctx->dev));
    // Stage in a buffer that is free between calls (the site codes, or a
    // Potts lattice's bond bytes; at least N bytes), check every byte on the
    // device, and only then replace the spins.
    uint8_t *stage = ctx->is_potts ? ctx->bond_bytes : reinterpret_cast<uint8_t *>(ctx->code);
    int32_t *bad = ctx->jbase;   // scratch word, rewritten by every sweep call
    SW_CUDA(cudaMemcpyAsync(stage, host_in, N, cudaMemcpyHostToDevice, ctx->stream));
    SW_CUDA(cudaMemsetAsync(bad, 0, sizeof(int32_t), ctx->stream));
    if (ctx->is_potts) {
        SW_CUDA(potts_enqueue_check(stage, (int64_t)N, ctx->pd.q, bad, ctx->stream));
    } else {
        k_check_spins<<<(unsigned)std::min<size_t>((N + 4095) / 4096, 4096), 256, 0, ctx->stream>>>(stage, (int64_t)N,
                                                                                                   bad);
    }
    SW_CUDA(cudaGetLastError());
    int32_t hbad = 0;
    SW_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    SW_CUDA(cudaStreamSynchronize(ctx->stream));
    if (hbad) return SW_ERR_ARG;
    SW_CUDA(cudaMemcpyAsync(ctx->spin, stage, N, cudaMemcpyDeviceToDevice, ctx->stream));
    SW_CUDA(cudaStreamSynchronize(ctx->stream));
    return SW_OK;
}

int sw_profile(sw_ctx *ctx, int32_t enable)
{
    if (!ctx) return SW_ERR_ARG;
    ctx->profiling = enable != 0;
    return SW_OK;
}

int sw_profile_read(sw_ctx *ctx, sw_kernel_stats *out)
{
    if (!ctx || !out) return SW_ERR_ARG;
    SW_CUDA(cudaSetDevice(ctx->dev));
    SW_CUDA(cudaStreamSynchronize(ctx->stream));
    for (size_t i = 0; i + 2 < ctx->ev_marks.size(); i += 3) {
        float t = 0.f, m = 0.f;
        SW_CUDA(cudaEventElapsedTime(&t, ctx->ev_marks[i], ctx->ev_marks[i + 1]));
        SW_CUDA(cudaEventElapsedTime(&m, ctx->ev_marks[i + 1], ctx->ev_marks[i + 2]));
        ctx->prof_tile_ms += t;
        ctx->prof_merge_ms += m;
        ctx->prof_groups += 1;
    }
    ctx->ev_marks.clear();
    ctx->ev_used = 0;
    out->tile_launches = ctx->prof_groups;
    out->tile_ms = ctx->prof_tile_ms;
    out->merge_groups = ctx->prof_groups;
    out->merge_ms = ctx->prof_merge_ms;
    out->tile_sites = ctx->is_potts ? ctx->nsites : (int64_t)ctx->L * ctx->L;
    out->tile_height = ctx->is_potts ? 0 : ctx->TH;
    ctx->prof_groups = 0;
    ctx->prof_tile_ms = ctx->prof_merge_ms = 0.0;
    return SW_OK;
}

int sw_get_labels(sw_ctx *ctx, int32_t *host_out)
{
    if (!ctx || !host_out) return SW_ERR_ARG;
    if (!ctx->swept) return SW_ERR_STATE;
    SW_CUDA(cudaSetDevice(ctx->dev));
    SW_CUDA(cudaMemcpyAsync(host_out, ctx->label, (size_t)ctx->nsites * sizeof(int32_t), cudaMemcpyDeviceToHost,
                            ctx->stream));
    SW_CUDA(cudaStreamSynchronize(ctx->stream));
    return SW_OK;
}

int sw_get_bonds(sw_ctx *ctx, uint8_t *host_out)
{
    if (!ctx || !host_out) return SW_ERR_ARG;
    if (!ctx->swept) return SW_ERR_STATE;
    SW_CUDA(cudaSetDevice(ctx->dev));
    const size_t N = (size_t)ctx->nsites;
    if (ctx->is_potts) {   // the bond bytes of the last sweep, as they are
        SW_CUDA(cudaMemcpyAsync(host_out, ctx->bond_bytes, N, cudaMemcpyDeviceToHost, ctx->stream));
        SW_CUDA(cudaStreamSynchronize(ctx->stream));
        return SW_OK;
    }
    if (!ctx->bond_bytes) {
        std::lock_guard<std::mutex> lk(sw_capture_mutex());
        SW_CUDA(dalloc(&ctx->bond_bytes, N));
    }
    const unsigned blocks = (unsigned)((N + 255) / 256);
    switch (ctx->TH) {
    case 32: k_bond_bytes<32><<<blocks, 256, 0, ctx->stream>>>(ctx->bondbits, ctx->L, ctx->tiles_x, ctx->bond_bytes); break;
    case 64: k_bond_bytes<64><<<blocks, 256, 0, ctx->stream>>>(ctx->bondbits, ctx->L, ctx->tiles_x, ctx->bond_bytes); break;
    case 96: k_bond_bytes<96><<<blocks, 256, 0, ctx->stream>>>(ctx->bondbits, ctx->L, ctx->tiles_x, ctx->bond_bytes); break;
    default: k_bond_bytes<128><<<blocks, 256, 0, ctx->stream>>>(ctx->bondbits, ctx->L, ctx->tiles_x, ctx->bond_bytes); break;
    }
    SW_CUDA(cudaGetLastError());
    SW_CUDA(cudaMemcpyAsync(host_out, ctx->bond_bytes, N, cudaMemcpyDeviceToHost, ctx->stream));
    SW_CUDA(cudaStreamSynchronize(ctx->stream));
    return SW_OK;
}

int sw_get_state(sw_ctx *ctx, sw_state *out)
{
    if (!ctx || !out) return SW_ERR_ARG;
    SW_CUDA(cudaSetDevice(ctx->dev));
    uint64_t thr = ctx->thr;
    if (ctx->pcc) {
        SW_CUDA(cudaMemcpyAsync(&thr, ctx->thr_dev, sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
        SW_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    out->L = ctx->L;
    out->pcc = ctx->pcc ? 1 : 0;
    out->seed = ctx->seed;
    out->sweep = ctx->sweep;
    out->threshold = thr;
    out->open = ctx->open ? 1 : 0;
    out->tile_h = ctx->is_potts ? 0 : ctx->TH;
    out->dim = ctx->is_potts ? ctx->pd.dim : 2;
    out->q = ctx->is_potts ? ctx->pd.q : 2;
    return SW_OK;
}

int sw_sync(sw_ctx *ctx)
{
    if (!ctx) return SW_ERR_ARG;
    SW_CUDA(cudaSetDevice(ctx->dev));
    SW_CUDA(cudaStreamSynchronize(ctx->stream));
    return SW_OK;
}

// ---- checkpoint / resume: a header, then the spins (one byte a site)
namespace {
constexpr uint64_t CKPT_MAGIC = 0x3130504b43575353ull;   // "SSWCKP01"
struct CkptHeader {
    uint64_t magic;
    int32_t L, dim, q, kind;   // kind bits: 1 PCC, 2 open, 4 winding
    uint64_t seed, sweep, threshold, nsites;
};
int ctx_kind(const sw_ctx *c) { return (c->pcc ? 1 : 0) | (c->open ? 2 : 0) | (c->wind ? 4 : 0); }
}  // namespace

int sw_checkpoint_bytes(sw_ctx *ctx, uint64_t *bytes)
{
    if (!ctx || !bytes) return SW_ERR_ARG;
    *bytes = sizeof(CkptHeader) + (uint64_t)ctx->nsites;
    return SW_OK;
}

int sw_save(sw_ctx *ctx, void *host_buf, uint64_t bytes)
{
    if (!ctx || !host_buf || bytes < sizeof(CkptHeader) + (uint64_t)ctx->nsites) return SW_ERR_ARG;
    sw_state st{};
    int rc = sw_get_state(ctx, &st);   // waits for the queued sweeps
    if (rc != SW_OK) return rc;
    CkptHeader h{};
    h.magic = CKPT_MAGIC;
    h.L = ctx->L;
    h.dim = st.dim;
    h.q = st.q;
    h.kind = ctx_kind(ctx);
    h.seed = ctx->seed;
    h.sweep = ctx->sweep;
    h.threshold = st.threshold;
    h.nsites = (uint64_t)ctx->nsites;
    std::memcpy(host_buf, &h, sizeof(h));
    return sw_get_spins(ctx, static_cast<uint8_t *>(host_buf) + sizeof(h));
}

int sw_load(sw_ctx *ctx, const void *host_buf, uint64_t bytes)
{
    if (!ctx || !host_buf || bytes < sizeof(CkptHeader)) return SW_ERR_ARG;
    CkptHeader h;
    std::memcpy(&h, host_buf, sizeof(h));
    const int dim = ctx->is_potts ? ctx->pd.dim : 2, q = ctx->is_potts ? ctx->pd.q : 2;
    if (h.magic != CKPT_MAGIC || h.L != ctx->L || h.dim != dim || h.q != q || h.kind != ctx_kind(ctx) ||
        h.nsites != (uint64_t)ctx->nsites || bytes < sizeof(h) + h.nsites || h.threshold > ((uint64_t)1 << 32))
        return SW_ERR_ARG;
    int rc = sw_set_spins(ctx, static_cast<const uint8_t *>(host_buf) + sizeof(h));   // checks every state
    if (rc != SW_OK) return rc;
    ctx->seed = h.seed;
    ctx->sweep = h.sweep;
    ctx->thr = h.threshold;
    ctx->rep.key0 = (uint32_t)h.seed;
    ctx->rep.key1 = (uint32_t)(h.seed >> 32);
    ctx->pd.seed = h.seed;
    ctx->pd.thr = h.threshold;
    if (ctx->pcc) {
        SW_CUDA(cudaMemcpyAsync(ctx->thr_dev, &h.threshold, sizeof(uint64_t), cudaMemcpyHostToDevice, ctx->stream));
        SW_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    ctx->swept = false;   // labels and bonds come back with the next sweep
    return SW_OK;
}

int sw_bench_philox(int64_t nblocks, uint64_t seed, uint32_t *out_dev, void *stream)
{
    if (!out_dev || nblocks < 0 || nblocks > ((int64_t)1 << 32)) return SW_ERR_ARG;
    if ((uintptr_t)out_dev & 3u) return SW_ERR_ARG;
    cudaGetLastError();
    int dev = 0, sms = 0;
    SW_CUDA(cudaGetDevice(&dev));
    SW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t want = (nblocks + 255) / 256;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
    k_philox_rate<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(nblocks, (uint32_t)seed,
                                                                       (uint32_t)(seed >> 32), out_dev);
    SW_CUDA(cudaGetLastError());
    return SW_OK;
}

int sw_bench_l2(const void *src_dev, void *dst_dev, int64_t bytes, int32_t reps, void *stream)
{
    if (!src_dev || !dst_dev || bytes <= 0 || (bytes & 15) || reps < 1) return SW_ERR_ARG;
    if (((uintptr_t)src_dev & 15u) || ((uintptr_t)dst_dev & 15u)) return SW_ERR_ARG;
    const uintptr_t a0 = (uintptr_t)src_dev, b0 = (uintptr_t)dst_dev, nb = (uintptr_t)bytes;
    if (a0 < b0 + nb && b0 < a0 + nb) return SW_ERR_ARG;
    cudaGetLastError();
    int dev = 0, sms = 0;
    SW_CUDA(cudaGetDevice(&dev));
    SW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t n = bytes / 16;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8));
    k_l2_rate<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const uint4 *>(src_dev),
                                                                   static_cast<uint4 *>(dst_dev), n, reps);
    SW_CUDA(cudaGetLastError());
    return SW_OK;
}

int sw_debug_fail_allocations(int32_t skip, int32_t n)
{
    if (skip < 0 || n < 0) return SW_ERR_ARG;
    g_alloc_failures.store(0);
    g_alloc_skip.store(skip);
    g_alloc_failures.store(n);
    return SW_OK;
}

}  // extern "C"
