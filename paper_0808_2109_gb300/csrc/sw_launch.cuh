// sw_launch.cuh -- how the host enqueues the kernels of sw_device.cuh: one
// launch group = the tile kernel of launch j, then the merge of sweep j.
// Shared by the single-lattice engine and the batch server.
#pragma once

#include "sw_device.cuh"

#include <cuda_runtime.h>

namespace swg {

constexpr int MERGE_THREADS = 256;

// Defined once, in sw_engine.cu: every kernel template is instantiated in
// that translation unit only, so each kernel has a single module copy (and
// the shared-memory attribute set by prepare_th applies to the copy that
// runs).
__attribute__((visibility("hidden"))) cudaError_t prepare_th(int TH);
// feat: FEAT_* bits of the tile-kernel variant to launch (the union of what
// the launch's lattices need)
__attribute__((visibility("hidden"))) cudaError_t enqueue_tile(int TH, const SweepArgs &a, bool pcc, int feat,
                                                               cudaStream_t st);
__attribute__((visibility("hidden"))) cudaError_t enqueue_merge(int TH, const SweepArgs &a, bool pcc, int feat,
                                                                int n_reps, cudaStream_t st);
__attribute__((visibility("hidden"))) cudaError_t enqueue_launch_th(int TH, const SweepArgs &a, bool pcc, int feat,
                                                                    int n_reps, cudaStream_t st);
__attribute__((visibility("hidden"))) cudaError_t enqueue_hot_start(uint8_t *spin, int64_t N, uint64_t seed,
                                                                    cudaStream_t st);
__attribute__((visibility("hidden"))) cudaError_t enqueue_job_init(uint8_t *spin, int64_t N, uint64_t seed, void *obs,
                                                                   int64_t obs_bytes, uint64_t *thr_dev, uint64_t thr,
                                                                   cudaStream_t st);

inline int slots_of(int TH) { return 2 * TW + 2 * TH; }

// A q-state Potts lattice on the periodic d-dimensional torus (sw_potts.cu):
// N = L^d sites; size is null unless cluster sizes are summed.
struct PottsDev {
    int32_t dim, L, q;
    int64_t N;
    uint64_t thr, seed;
    uint8_t *spin, *bond;
    int32_t *label, *size;
    int32_t open;              // open boundaries: no link leaves the lattice
    // PCC (null otherwise): the threshold lives on the device and follows the
    // feedback; per axis a < dim, candidate ids of roots (cid + a N, id + 2),
    // the candidates (cand + a F, F = L^(dim-1) face sites), their counts
    // (ncand[a]; ncand[3] counts finished decision blocks) and coverage
    // (cov + a F W, W = ceil(L / 32) words per candidate)
    uint64_t *thr_dev;
    int32_t *cid, *cand, *ncand;
    uint32_t *cov;
};
__attribute__((visibility("hidden"))) cudaError_t potts_enqueue_hot_start(const PottsDev &p, cudaStream_t st);
__attribute__((visibility("hidden"))) cudaError_t potts_enqueue_sweep(const PottsDev &p, uint64_t sweep, DevObs *obs,
                                                                      cudaStream_t st);
__attribute__((visibility("hidden"))) cudaError_t potts_enqueue_check(const uint8_t *s, int64_t n, int q, int32_t *bad,
                                                                      cudaStream_t st);

}  // namespace swg
