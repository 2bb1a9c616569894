// sw_server.cu -- batched and served runs (the sw_server / sw_batch_* part of
// include/swgpu.h).
//
// Many independent lattices share every kernel launch: a "lane" (one per
// tile height) keeps a fixed-capacity tile table over all its admitted
// lattices and one captured CUDA graph of GROUPS_PER_STEP launch groups.
// A worker thread loops: admit queued jobs while their device bytes fit the
// budget (stream-ordered allocations, hot start on the device), run one step
// of every busy lane, retire the lattices whose last sweep has finished
// (copy their observables, spins and labels out, free their memory).  New
// jobs therefore join at sweep boundaries while others are mid-run.  Each
// lattice keeps its own scratch, counters and launch offset (jstart), so a
// job's results do not depend on what else runs beside it.
#include "swgpu.h"
#include "sw_device.cuh"
#include "sw_internal.h"
#include "sw_launch.cuh"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

using namespace swg;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int GROUPS_PER_STEP = 16;   // launch groups between admissions
// Lanes: one per tile height (32, 64, 96, 128) for plain lattices and one
// per height for lattices that need a kernel feature (PCC, open boundaries,
// cluster sizes, the topological rule), so plain lattices keep the plain
// kernels whatever else is being served.
constexpr int N_LANES = 8;
constexpr int32_t SERVER_MAX_L = 4096;

int lane_of_th(int th) { return th == 32 ? 0 : th == 64 ? 1 : th == 96 ? 2 : 3; }
int th_of_lane(int l) { return (l & 3) == 0 ? 32 : (l & 3) == 1 ? 64 : (l & 3) == 2 ? 96 : 128; }

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Job {
    uint64_t id = 0;
    sw_job spec{};
    uint64_t thr = 0;
    bool pcc = false;
    int TH = 128, tiles_x = 0, tiles_y = 0, n_tiles = 0, S = 0;
    size_t bytes = 0;
    Clock::time_point t_submit, t_admit;
    // device state: every buffer is carved from one block
    void *block = nullptr;
    uint8_t *spin = nullptr;
    int32_t *label = nullptr;
    uint16_t *code = nullptr;
    uint32_t *bondbits = nullptr, *cross = nullptr, *nfinal = nullptr, *pmask = nullptr, *cov = nullptr;
    int32_t *npar = nullptr, *nkey = nullptr, *cid = nullptr, *cand = nullptr, *ncand = nullptr;
    uint64_t *thr_dev = nullptr;
    DevObs *obs = nullptr;
    int32_t *psize = nullptr, *csize = nullptr;   // SW_FLAG_CSIZE
    unsigned long long *nlink = nullptr;          // SW_FLAG_WIND
    // placement
    int lane = -1, slot = -1, tile_base = -1;
    int32_t jstart = 0;
};

// Byte offsets of a job's buffers inside its one device block, each on a
// 256-byte boundary; PCC scratch last, in one range that starts zeroed.
struct JobLayout {
    size_t spin, label, code, bondbits, cross, npar, nkey, nfinal, thr, obs, psize, csize, nlink;
    size_t pmask, cid, cand, ncand, cov, pcc_end, total;
};

JobLayout job_layout(int L, int TH, int nsweeps, bool pcc, bool csize, bool wind)
{
    const size_t N = (size_t)L * L;
    const size_t tx = (L + TW - 1) / TW, ty = (L + TH - 1) / TH, nt = tx * ty;
    const size_t S = (size_t)slots_of(TH);
    JobLayout o{};
    size_t at = 0;
    auto take = [&at](size_t bytes) {
        const size_t here = at;
        at += round256(std::max<size_t>(bytes, 1));
        return here;
    };
    o.spin = take(N);
    o.label = take(4 * N);
    o.code = take(nt * TH * TW * 2);
    o.bondbits = take(nt * TH * 2 * TWW * 4);
    o.cross = take(nt * CROSS_WORDS * 4);
    o.npar = take(nt * S * 4);
    o.nkey = take(nt * S * 4);
    o.nfinal = take(nt * S * 4);
    o.thr = take(8);
    o.obs = take((size_t)nsweeps * sizeof(DevObs));
    o.psize = o.csize = at;
    if (csize) {
        o.psize = take(nt * S * 4);
        o.csize = take(nt * S * 4);
    }
    o.nlink = wind ? take(nt * S * 8) : at;
    o.pmask = o.cid = o.cand = o.ncand = o.cov = o.pcc_end = at;
    if (pcc) {
        o.pmask = take(nt * S * 8 * 4);
        o.cid = take(nt * S * 2 * 4);
        o.cand = take(2 * (size_t)L * 4);
        o.ncand = take(3 * 4);
        o.cov = take((size_t)L * (tx + ty) * 4 * 4);
        o.pcc_end = at;
    }
    o.total = at;
    return o;
}

size_t job_bytes(int L, int TH, int nsweeps, bool pcc, uint32_t flags)
{
    return job_layout(L, TH, nsweeps, pcc, (flags & SW_FLAG_CSIZE) != 0, (flags & SW_FLAG_WIND) != 0).total;
}

struct Lane {
    int TH = 128;
    int cap_tiles = 0, cap_reps = 0;
    cudaStream_t stream = nullptr;
    Replica *reps_dev = nullptr;
    int32_t *tile_rep_dev = nullptr;
    int32_t *jbase_dev = nullptr;
    std::vector<Replica> reps_host;
    std::vector<int32_t> tile_rep_host;
    std::vector<Job *> slot_job;
    std::vector<int> free_slots;   // unused slots (a stack)
    int tail = 0;                  // every tile from here on is free
    cudaGraphExec_t graph = nullptr;
    bool graph_pcc = false;
    int graph_feat = 0;         // FEAT_* of the captured tile kernel
    bool dirty = true;       // tables changed since the last upload
    bool recapture = true;   // capacity or mode changed since the last capture
    int active = 0;
};

}  // namespace

struct sw_server {
    int dev = 0;
    size_t budget = 0, used = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> pending;
    std::map<uint64_t, sw_result> finished;
    std::map<uint64_t, int> known;   // id -> 0 queued/running
    uint64_t next_id = 1;
    bool stop = false;
    int32_t launch_index = 0;
    Lane lanes[N_LANES];
    std::vector<Job *> running;
    std::thread worker;
    sw_server_stats stats{};
    int worker_error = SW_OK;
    DevObs *stage = nullptr;   // pinned staging for retired jobs' observables
    size_t stage_cap = 0;
};

namespace {

void free_job_device(Job *j, cudaStream_t st)
{
    if (j->block) cudaFreeAsync(j->block, st);
    j->block = nullptr;
}

// Device state of a newly admitted job: one stream-ordered block for all its
// buffers, zeroed PCC scratch, and one kernel for the hot start, the
// observables and the threshold.
cudaError_t job_alloc(Job *j, cudaStream_t st)
{
    const size_t N = (size_t)j->spec.L * j->spec.L;
    const bool csz = (j->spec.flags & SW_FLAG_CSIZE) != 0;
    const bool wnd = (j->spec.flags & SW_FLAG_WIND) != 0;
    const JobLayout o = job_layout(j->spec.L, j->TH, j->spec.nsweeps, j->pcc, csz, wnd);
    cudaError_t e = sw_inject_alloc_failure() ? cudaErrorMemoryAllocation : cudaMallocAsync(&j->block, o.total, st);
    if (e != cudaSuccess) {
        j->block = nullptr;
        return e;
    }
    unsigned char *b = static_cast<unsigned char *>(j->block);
    j->spin = b + o.spin;
    j->label = reinterpret_cast<int32_t *>(b + o.label);
    j->code = reinterpret_cast<uint16_t *>(b + o.code);
    j->bondbits = reinterpret_cast<uint32_t *>(b + o.bondbits);
    j->cross = reinterpret_cast<uint32_t *>(b + o.cross);
    j->npar = reinterpret_cast<int32_t *>(b + o.npar);
    j->nkey = reinterpret_cast<int32_t *>(b + o.nkey);
    j->nfinal = reinterpret_cast<uint32_t *>(b + o.nfinal);
    j->thr_dev = reinterpret_cast<uint64_t *>(b + o.thr);
    j->obs = reinterpret_cast<DevObs *>(b + o.obs);
    if (csz) {
        j->psize = reinterpret_cast<int32_t *>(b + o.psize);
        j->csize = reinterpret_cast<int32_t *>(b + o.csize);
    }
    if (wnd) j->nlink = reinterpret_cast<unsigned long long *>(b + o.nlink);
    if (j->pcc) {
        j->pmask = reinterpret_cast<uint32_t *>(b + o.pmask);
        j->cid = reinterpret_cast<int32_t *>(b + o.cid);
        j->cand = reinterpret_cast<int32_t *>(b + o.cand);
        j->ncand = reinterpret_cast<int32_t *>(b + o.ncand);
        j->cov = reinterpret_cast<uint32_t *>(b + o.cov);
        if ((e = cudaMemsetAsync(b + o.pmask, 0, o.pcc_end - o.pmask, st)) != cudaSuccess) return e;
    }
    return enqueue_job_init(j->spin, (int64_t)N, j->spec.seed, j->obs, (int64_t)j->spec.nsweeps * sizeof(DevObs),
                            j->thr_dev, j->thr, st);
}

Replica replica_of(const Job *j)
{
    Replica R{};
    R.L = j->spec.L;
    R.tiles_x = j->tiles_x;
    R.tiles_y = j->tiles_y;
    R.tile_base = j->tile_base;
    R.key0 = (uint32_t)j->spec.seed;
    R.key1 = (uint32_t)(j->spec.seed >> 32);
    R.nsweeps = j->spec.nsweeps;
    R.flags = (j->pcc ? RF_PCC : 0) | ((j->spec.flags & SW_FLAG_OPEN) ? RF_OPEN : 0) |
              ((j->spec.flags & SW_FLAG_CSIZE) ? RF_CSIZE : 0) | ((j->spec.flags & SW_FLAG_WIND) ? RF_WIND : 0);
    R.sweep0 = 0;
    R.thr = j->thr;
    R.thr_dev = j->thr_dev;
    R.spin = j->spin;
    R.label = j->label;
    R.bond = nullptr;
    R.obs = j->obs;
    R.jstart = j->jstart;
    R.code = j->code;
    R.bondbits = j->bondbits;
    R.cross = j->cross;
    R.npar = j->npar;
    R.nkey = j->nkey;
    R.nfinal = j->nfinal;
    R.pmask = j->pmask;
    R.cid = j->cid;
    R.cand = j->cand;
    R.ncand = j->ncand;
    R.cov = j->cov;
    R.psize = j->psize;
    R.csize = j->csize;
    R.nlink = j->nlink;
    return R;
}

// Grow a lane's tables to hold at least `tiles` tiles and `reps` lattices.
cudaError_t lane_reserve(Lane &ln, int tiles, int reps)
{
    std::lock_guard<std::mutex> lk(sw_capture_mutex());
    if (tiles > ln.cap_tiles) {
        int cap = std::max(ln.cap_tiles * 2, 256);
        while (cap < tiles) cap *= 2;
        int32_t *d = nullptr;
        cudaError_t e = cudaMalloc(&d, (size_t)cap * sizeof(int32_t));
        if (e != cudaSuccess) return e;
        if (ln.tile_rep_dev) cudaFree(ln.tile_rep_dev);
        ln.tile_rep_dev = d;
        ln.tile_rep_host.resize(cap, -1);
        ln.cap_tiles = cap;
        ln.dirty = ln.recapture = true;
    }
    if (reps > ln.cap_reps) {
        int cap = std::max(ln.cap_reps * 2, 64);
        while (cap < reps) cap *= 2;
        Replica *d = nullptr;
        cudaError_t e = cudaMalloc(&d, (size_t)cap * sizeof(Replica));
        if (e != cudaSuccess) return e;
        if (ln.reps_dev) cudaFree(ln.reps_dev);
        ln.reps_dev = d;
        Replica empty{};
        ln.reps_host.resize(cap, empty);
        ln.slot_job.resize(cap, nullptr);
        for (int i = cap - 1; i >= ln.cap_reps; --i) ln.free_slots.push_back(i);
        ln.cap_reps = cap;
        ln.dirty = ln.recapture = true;
    }
    return cudaSuccess;
}

// `n` free tiles in a row in the lane's table: after the last used tile when
// they fit there, else the first run of free tiles, else new capacity.
int lane_place_tiles(Lane &ln, int n)
{
    int start = -1;
    if (ln.tail + n <= ln.cap_tiles) {
        start = ln.tail;
    } else {
        int run = 0;
        for (int i = 0; i < ln.tail && start < 0; ++i) {
            run = ln.tile_rep_host[i] < 0 ? run + 1 : 0;
            if (run == n) start = i - n + 1;
        }
        if (start < 0) {
            start = ln.tail;
            if (lane_reserve(ln, start + n, ln.cap_reps) != cudaSuccess) return -1;
        }
    }
    ln.tail = std::max(ln.tail, start + n);
    return start;
}

int lane_free_slot(Lane &ln)
{
    if (ln.free_slots.empty() && lane_reserve(ln, ln.cap_tiles, ln.cap_reps + 1) != cudaSuccess) return -1;
    const int s = ln.free_slots.back();
    ln.free_slots.pop_back();
    return s;
}

// Gives a retired lattice's tiles and slot back.
void lane_release(Lane &ln, Job *j)
{
    for (int i = 0; i < j->n_tiles; ++i) ln.tile_rep_host[j->tile_base + i] = -1;
    while (ln.tail > 0 && ln.tile_rep_host[ln.tail - 1] < 0) --ln.tail;
    ln.slot_job[j->slot] = nullptr;
    ln.reps_host[j->slot] = Replica{};
    ln.free_slots.push_back(j->slot);
    ln.active -= 1;
    ln.dirty = true;
}

SweepArgs lane_args(Lane &ln)
{
    SweepArgs a{};
    a.reps = ln.reps_dev;
    a.tile_rep = ln.tile_rep_dev;
    a.n_tiles = ln.cap_tiles;
    a.j = 0;
    a.jbase = ln.jbase_dev;
    return a;
}

cudaError_t lane_capture(Lane &ln, cudaStream_t cap_stream, bool pcc, int feat)
{
    if (ln.graph) {
        cudaGraphExecDestroy(ln.graph);
        ln.graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    std::lock_guard<std::mutex> lk(sw_capture_mutex());
    cudaError_t e = cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    SweepArgs a = lane_args(ln);
    for (int j = 0; j < GROUPS_PER_STEP && e == cudaSuccess; ++j) {
        a.j = j;
        e = enqueue_launch_th(ln.TH, a, pcc, feat, ln.cap_reps, cap_stream);
    }
    cudaError_t e2 = cudaStreamEndCapture(cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e != cudaSuccess ? e : e2;
    }
    e = cudaGraphInstantiate(&ln.graph, g, 0);
    cudaGraphDestroy(g);
    ln.graph_pcc = pcc;
    ln.graph_feat = feat;
    ln.recapture = false;
    return e;
}

double secs(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double>(b - a).count();
}

// Copy finished jobs' outputs to their callers, summarise them and free
// them: every job's observables go through one pinned staging buffer, with
// one wait per lane instead of one per job.
void retire_all(sw_server *s, const std::vector<Job *> &done)
{
    size_t need = 0;
    for (Job *j : done) need += (size_t)j->spec.nsweeps + 1;   // + one record for the threshold
    DevObs *stage = s->stage;
    std::vector<DevObs> heap;
    if (need > s->stage_cap) {
        std::lock_guard<std::mutex> lk(sw_capture_mutex());
        if (s->stage) cudaFreeHost(s->stage);
        s->stage = nullptr;
        s->stage_cap = 0;
        const size_t cap = std::max(need, (size_t)2 * s->stage_cap + 4096);
        if (cudaMallocHost(&s->stage, cap * sizeof(DevObs)) == cudaSuccess) {
            s->stage_cap = cap;
        } else {
            cudaGetLastError();
            s->stage = nullptr;
        }
        stage = s->stage;
    }
    if (!stage) {   // no pinned memory: plain host memory (the copies then wait)
        heap.resize(need);
        stage = heap.data();
    }
    std::vector<size_t> at(done.size());
    std::vector<cudaError_t> err(done.size(), cudaSuccess);
    bool used[N_LANES] = {};
    size_t off = 0;
    for (size_t i = 0; i < done.size(); ++i) {
        Job *j = done[i];
        const cudaStream_t st = s->lanes[j->lane].stream;
        used[j->lane] = true;
        at[i] = off;
        const size_t nobs = (size_t)j->spec.nsweeps, N = (size_t)j->spec.L * j->spec.L;
        cudaError_t e = cudaMemcpyAsync(stage + off, j->obs, nobs * sizeof(DevObs), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && j->pcc)
            e = cudaMemcpyAsync(stage + off + nobs, j->thr_dev, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && j->spec.spins_out)
            e = cudaMemcpyAsync(j->spec.spins_out, j->spin, N, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && j->spec.labels_out)
            e = cudaMemcpyAsync(j->spec.labels_out, j->label, N * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        err[i] = e;
        off += nobs + 1;
    }
    cudaError_t lane_err[N_LANES] = {};
    for (int l = 0; l < N_LANES; ++l)
        if (used[l]) lane_err[l] = cudaStreamSynchronize(s->lanes[l].stream);
    std::vector<sw_result> res(done.size());
    const auto now = Clock::now();
    for (size_t i = 0; i < done.size(); ++i) {
        Job *j = done[i];
        Lane &ln = s->lanes[j->lane];
        const size_t nobs = (size_t)j->spec.nsweeps;
        const DevObs *obs = stage + at[i];
        sw_result &r = res[i];
        std::memset(&r, 0, sizeof(r));
        r.status = (err[i] == cudaSuccess && lane_err[j->lane] == cudaSuccess) ? SW_OK : SW_ERR_CUDA;
        r.L = j->spec.L;
        r.nsweeps = j->spec.nsweeps;
        r.tile_h = j->TH;
        r.threshold = j->thr;
        if (j->pcc) std::memcpy(&r.threshold, obs + nobs, sizeof(uint64_t));
        for (size_t k = 0; k < nobs; ++k) {
            r.sum_bond_sum += (int64_t)obs[k].bond_sum;
            r.sum_abs_mag += std::llabs((long long)obs[k].mag);
            r.sum_nclusters += (int64_t)obs[k].nclusters;
        }
        if (j->spec.obs_out) std::memcpy(j->spec.obs_out, obs, nobs * sizeof(DevObs));
        r.queued_s = secs(j->t_submit, j->t_admit);
        r.run_s = secs(j->t_admit, now);
        lane_release(ln, j);
        free_job_device(j, ln.stream);
    }
    // the frees complete before the budget counts the bytes as available
    for (int l = 0; l < N_LANES; ++l)
        if (used[l]) cudaStreamSynchronize(s->lanes[l].stream);
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t i = 0; i < done.size(); ++i) {
        Job *j = done[i];
        s->used -= j->bytes;
        s->finished[j->id] = res[i];
        s->stats.finished += 1;
        s->stats.site_updates += (int64_t)j->spec.L * j->spec.L * j->spec.nsweeps;
        delete j;
    }
    s->cv_done.notify_all();
}

void worker_main(sw_server *s)
{
    cudaSetDevice(s->dev);
    cudaStream_t cap_stream = nullptr;
    cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking);
    for (;;) {
        // ---- admit queued jobs that fit (in submission order, skipping ones that do not fit yet)
        std::vector<Job *> admit;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop) break;
            if (s->running.empty() && s->pending.empty()) {
                s->cv_work.wait(lk, [s] { return s->stop || !s->pending.empty(); });
                if (s->stop) break;
            }
            for (auto it = s->pending.begin(); it != s->pending.end();) {
                if (s->used + (*it)->bytes <= s->budget) {
                    s->used += (*it)->bytes;
                    admit.push_back(*it);
                    it = s->pending.erase(it);
                } else {
                    ++it;
                }
            }
            s->stats.pending = (int64_t)s->pending.size();
        }
        for (Job *j : admit) {
            j->lane = lane_of_th(j->TH) + ((j->pcc || j->spec.flags) ? 4 : 0);
            Lane &ln = s->lanes[j->lane];
            j->t_admit = Clock::now();
            j->jstart = s->launch_index;
            int rc = SW_OK;
            if (job_alloc(j, ln.stream) != cudaSuccess) rc = SW_ERR_NOMEM;
            if (rc == SW_OK) {
                j->slot = lane_free_slot(ln);
                j->tile_base = j->slot >= 0 ? lane_place_tiles(ln, j->n_tiles) : -1;
                if (j->slot >= 0 && j->tile_base < 0) ln.free_slots.push_back(j->slot);
                if (j->slot < 0 || j->tile_base < 0) rc = SW_ERR_NOMEM;
            }
            if (rc != SW_OK) {
                cudaGetLastError();
                free_job_device(j, ln.stream);
                cudaStreamSynchronize(ln.stream);
                sw_result res{};
                res.status = rc;
                res.L = j->spec.L;
                res.nsweeps = j->spec.nsweeps;
                std::lock_guard<std::mutex> lk(s->mu);
                s->used -= j->bytes;
                s->finished[j->id] = res;
                s->stats.finished += 1;
                s->cv_done.notify_all();
                delete j;
                continue;
            }
            for (int i = 0; i < j->n_tiles; ++i) ln.tile_rep_host[j->tile_base + i] = j->slot;
            ln.slot_job[j->slot] = j;
            ln.reps_host[j->slot] = replica_of(j);
            ln.active += 1;
            ln.dirty = true;
            s->running.push_back(j);
            std::lock_guard<std::mutex> lk(s->mu);
            s->stats.admitted += 1;
        }
        // ---- one step of every busy lane
        nvtxRangePushA("server step");
        bool any = false;
        for (Lane &ln : s->lanes) {
            if (ln.active == 0) continue;
            any = true;
            bool pcc = false;
            int feat = 0;
            for (Job *j : ln.slot_job) {
                if (!j) continue;
                pcc = pcc || j->pcc;
                feat |= (j->psize ? FEAT_CSIZE : 0) | ((j->spec.flags & SW_FLAG_OPEN) ? FEAT_OPEN : 0) |
                        (j->nlink ? FEAT_WIND : 0);
            }
            if (pcc != ln.graph_pcc || feat != ln.graph_feat) ln.recapture = true;
            if (ln.dirty) {
                cudaMemcpyAsync(ln.tile_rep_dev, ln.tile_rep_host.data(), (size_t)ln.cap_tiles * sizeof(int32_t),
                                cudaMemcpyHostToDevice, ln.stream);
                cudaMemcpyAsync(ln.reps_dev, ln.reps_host.data(), (size_t)ln.cap_reps * sizeof(Replica),
                                cudaMemcpyHostToDevice, ln.stream);
                ln.dirty = false;
            }
            if (ln.recapture || !ln.graph) {
                if (lane_capture(ln, cap_stream, pcc, feat) != cudaSuccess) {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->worker_error = SW_ERR_CUDA;
                }
            }
            const int32_t jb = s->launch_index;
            cudaMemcpyAsync(ln.jbase_dev, &jb, sizeof(int32_t), cudaMemcpyHostToDevice, ln.stream);
            if (ln.graph) cudaGraphLaunch(ln.graph, ln.stream);
        }
        if (!any) {
            nvtxRangePop();
            continue;
        }
        s->launch_index += GROUPS_PER_STEP;
        for (Lane &ln : s->lanes)
            if (ln.active) cudaStreamSynchronize(ln.stream);
        nvtxRangePop();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stats.launches += GROUPS_PER_STEP;
        }
        // ---- retire lattices whose last launch (jstart + nsweeps) has run
        std::vector<Job *> done;
        for (auto it = s->running.begin(); it != s->running.end();) {
            if ((int64_t)(*it)->jstart + (*it)->spec.nsweeps < (int64_t)s->launch_index) {
                done.push_back(*it);
                it = s->running.erase(it);
            } else {
                ++it;
            }
        }
        if (!done.empty()) retire_all(s, done);
    }
    cudaStreamDestroy(cap_stream);
}

}  // namespace

// ====================================================================== ABI
extern "C" {

int sw_server_create(sw_server **out, size_t device_bytes, uint32_t flags)
{
    (void)flags;
    if (!out) return SW_ERR_ARG;
    *out = nullptr;
    sw_server *s = new (std::nothrow) sw_server();
    if (!s) return SW_ERR_NOMEM;
    if (cudaGetDevice(&s->dev) != cudaSuccess) {
        delete s;
        return SW_ERR_CUDA;
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete s;
        return SW_ERR_CUDA;
    }
    s->budget = device_bytes ? device_bytes : (size_t)(0.8 * (double)free_b);
    s->stats.bytes_budget = s->budget;
    // keep freed blocks in the stream-ordered pool instead of returning them
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, s->dev) == cudaSuccess) {
        uint64_t thresh = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thresh);
    }
    for (int l = 0; l < N_LANES; ++l) {
        Lane &ln = s->lanes[l];
        ln.TH = th_of_lane(l);
        if (prepare_th(ln.TH) != cudaSuccess || cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc(&ln.jbase_dev, sizeof(int32_t)) != cudaSuccess || lane_reserve(ln, 256, 64) != cudaSuccess) {
            sw_server_destroy(s);
            return SW_ERR_CUDA;
        }
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return SW_OK;
}

int sw_server_destroy(sw_server *s)
{
    if (!s) return SW_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->dev);
    for (Job *j : s->running) {
        free_job_device(j, s->lanes[j->lane].stream);
        delete j;
    }
    for (Job *j : s->pending) delete j;
    for (Lane &ln : s->lanes) {
        if (ln.stream) cudaStreamSynchronize(ln.stream);
        if (ln.graph) cudaGraphExecDestroy(ln.graph);
        if (ln.reps_dev) cudaFree(ln.reps_dev);
        if (ln.tile_rep_dev) cudaFree(ln.tile_rep_dev);
        if (ln.jbase_dev) cudaFree(ln.jbase_dev);
        if (ln.stream) cudaStreamDestroy(ln.stream);
    }
    if (s->stage) cudaFreeHost(s->stage);
    delete s;
    return SW_OK;
}

int sw_batch_submit(sw_server *s, const sw_job *jobs, int32_t n, uint64_t *ids_out)
{
    if (!s || n < 0 || (n > 0 && (!jobs || !ids_out))) return SW_ERR_ARG;
    std::vector<Job *> made;
    made.reserve((size_t)n);
    int rc = SW_OK;
    for (int32_t i = 0; i < n && rc == SW_OK; ++i) {
        const sw_job &q = jobs[i];
        Job *j = new (std::nothrow) Job();
        if (!j) {
            rc = SW_ERR_NOMEM;
            break;
        }
        made.push_back(j);
        j->spec = q;
        if (q.L < 2 || q.L > SERVER_MAX_L || q.nsweeps < 1 || (q.flags & ~(SW_FLAG_OPEN | SW_FLAG_CSIZE | SW_FLAG_WIND)) != 0 ||
            (q.tile_h != 0 && q.tile_h != 32 && q.tile_h != 64 && q.tile_h != 96 && q.tile_h != 128)) {
            rc = SW_ERR_ARG;
            break;
        }
        if (q.kind == SW_JOB_SW)
            rc = sw_threshold(q.J, q.T, &j->thr);
        else if (q.kind == SW_JOB_SWP)
            rc = sw_threshold_p_internal(q.p, &j->thr);
        else if (q.kind == SW_JOB_PCC)
            j->thr = (uint64_t)1 << 31;
        else
            rc = SW_ERR_ARG;
        if (rc != SW_OK) break;
        j->pcc = q.kind == SW_JOB_PCC;
        if (q.tile_h) {
            j->TH = q.tile_h;
        } else {
            int32_t th = 0;
            rc = sw_autotune(q.L, q.kind == SW_JOB_SW ? q.T : 2.269185, &th);
            if (rc != SW_OK) break;
            j->TH = th;
        }
        j->tiles_x = (q.L + TW - 1) / TW;
        j->tiles_y = (q.L + j->TH - 1) / j->TH;
        j->n_tiles = j->tiles_x * j->tiles_y;
        j->S = slots_of(j->TH);
        j->bytes = job_bytes(q.L, j->TH, q.nsweeps, j->pcc, q.flags);
        if (j->bytes > s->budget) rc = SW_ERR_NOMEM;
    }
    if (rc != SW_OK) {
        for (Job *j : made) delete j;
        return rc;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const auto now = Clock::now();
        for (int32_t i = 0; i < n; ++i) {
            Job *j = made[(size_t)i];
            j->id = s->next_id++;
            j->t_submit = now;
            ids_out[i] = j->id;
            s->known[j->id] = 0;
            s->pending.push_back(j);
        }
        s->stats.submitted += n;
        s->stats.pending = (int64_t)s->pending.size();
    }
    s->cv_work.notify_all();
    return SW_OK;
}

int sw_batch_poll(sw_server *s, uint64_t id, sw_result *out)
{
    if (!s || !out) return SW_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto f = s->finished.find(id);
    if (f != s->finished.end()) {
        *out = f->second;
        s->finished.erase(f);
        s->known.erase(id);
        return SW_OK;
    }
    return s->known.count(id) ? SW_PENDING : SW_ERR_ARG;
}

int sw_batch_wait_all(sw_server *s, double timeout_s)
{
    if (!s) return SW_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto done = [s] { return s->stats.finished >= s->stats.submitted || s->worker_error != SW_OK; };
    if (timeout_s > 0) {
        if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) return SW_ERR_TIMEOUT;
    } else {
        s->cv_done.wait(lk, done);
    }
    return s->worker_error;
}

}  // extern "C"

namespace {

// Seconds per site update of tile height th on a batch of lattices of side
// Lb (about 2^23 sites together, 20 sweeps) run through a private server:
// the throughput that batched and served runs see, where a single small
// lattice would leave most of the GPU idle and time latency instead.  The
// faster of two runs (the first one also captures the lane's graph).
double batch_cost(int Lb, double T, int th)
{
    sw_server *srv = nullptr;
    if (sw_server_create(&srv, 0, 0) != SW_OK) return 0.0;
    const int m = std::max(2, (1 << 23) / (Lb * Lb));
    const int nsw = 20;
    std::vector<sw_job> jobs((size_t)m);
    for (int r = 0; r < m; ++r) {
        sw_job &q = jobs[(size_t)r];
        std::memset(&q, 0, sizeof(q));
        q.L = Lb;
        q.kind = SW_JOB_SW;
        q.J = 1.0;
        q.T = T;
        q.seed = 12345 + (uint64_t)r;
        q.nsweeps = nsw;
        q.tile_h = th;
    }
    std::vector<uint64_t> ids((size_t)m);
    double best = 0.0;
    for (int rep = 0; rep < 2; ++rep) {
        const auto t0 = Clock::now();
        if (sw_batch_submit(srv, jobs.data(), m, ids.data()) != SW_OK || sw_batch_wait_all(srv, 120.0) != SW_OK) {
            best = 0.0;
            break;
        }
        const double dt = secs(t0, Clock::now());
        if (rep == 0 || dt < best) best = dt;
        sw_result r;
        for (uint64_t id : ids) sw_batch_poll(srv, id, &r);
    }
    sw_server_destroy(srv);
    return best / ((double)m * Lb * Lb * nsw);
}

}  // namespace

extern "C" {

// Autotuner: per (L_b, temperature regime), with L_b = L rounded up to a power
// of two, time every tile height that fits and keep the fastest.  Up to
// 2048 x 2048 sites the candidates run as a batch of L_b x L_b lattices
// through the server (batched and served runs share the GPU among many
// lattices, so throughput is what counts); larger lattices fill the GPU on
// their own and are timed alone.  Any height gives the same results.
int sw_autotune(int32_t L, double T, int32_t *tile_h_out)
{
    if (!tile_h_out || L < 2 || !(T > 0.0)) return SW_ERR_ARG;
    static std::mutex mu;
    static std::map<std::pair<int, int>, int> cache;
    int Lb = 32;
    while (Lb < L && Lb < 32768) Lb *= 2;
    if (Lb > L && L > 4096) Lb = L;
    const int regime = T < 2.15 ? 0 : (T < 2.4 ? 1 : 2);   // ordered, critical, disordered
    const std::pair<int, int> key(Lb, regime);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *tile_h_out = it->second;
        return SW_OK;
    }
    const double Trep = regime == 0 ? 2.0 : (regime == 1 ? 2.269185 : 3.0);
    const int heights[4] = {32, 64, 96, 128};
    const uint32_t flags[4] = {SW_FLAG_TILE_32, SW_FLAG_TILE_64, SW_FLAG_TILE_96, SW_FLAG_TILE_128};
    const double target = 4e7;   // site updates timed per candidate
    const int n = (int)std::min(200.0, std::max(4.0, target / ((double)Lb * Lb)));
    int best = Lb <= 32 ? 32 : (Lb <= 64 ? 64 : 128);
    double best_t = 1e300;
    const bool batch = (int64_t)Lb * Lb <= ((int64_t)1 << 22);
    if (Lb <= 32) {   // one candidate: nothing to time
        cache[key] = 32;
        *tile_h_out = 32;
        return SW_OK;
    }
    for (int c = 0; c < 4; ++c) {
        if (heights[c] > std::max(32, Lb)) continue;
        if (batch) {
            const double cost = batch_cost(Lb, Trep, heights[c]);
            if (cost > 0.0 && cost < best_t) {
                best_t = cost;
                best = heights[c];
            }
            continue;
        }
        sw_ctx *ctx = nullptr;
        if (sw_create(&ctx, Lb, 1.0, Trep, 12345, flags[c]) != SW_OK) continue;
        // direct launches with events around every kernel (no graph capture,
        // which another thread's allocations could disturb)
        sw_profile(ctx, 1);
        sw_kernel_stats st{};
        int rc = sw_sweep(ctx, 3);
        if (rc == SW_OK) rc = sw_profile_read(ctx, &st);
        if (rc == SW_OK) rc = sw_sweep(ctx, n);
        if (rc == SW_OK) rc = sw_profile_read(ctx, &st);
        sw_destroy(ctx);
        const double dt = st.tile_ms + st.merge_ms;
        if (rc == SW_OK && dt > 0 && dt < best_t) {
            best_t = dt;
            best = heights[c];
        }
    }
    cache[key] = best;
    *tile_h_out = best;
    return SW_OK;
}

int sw_server_get_stats(sw_server *s, sw_server_stats *out)
{
    if (!s || !out) return SW_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->active = s->stats.admitted - s->stats.finished;
    out->bytes_in_use = s->used;
    out->bytes_budget = s->budget;
    return SW_OK;
}

}  // extern "C"
