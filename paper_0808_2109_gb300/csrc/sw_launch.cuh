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

// A q-state Potts lattice on the d-dimensional lattice (sw_potts.cu): N =
// L^d sites cut into tiles (128 x 64 in 2D, 32 x 16 x 16 in 3D) of which the
// kernels keep per-tile scratch as the 2D Ising path does: a 2-byte code per
// site, crossing-bond bits and the face nodes' forest (parent, key, final,
// the new state of a representative), and with RF_CSIZE the sizes of the
// pieces and clusters at their nodes.
struct PottsDev {
    int32_t dim, L, q, flags;          // flags: RF_OPEN | RF_CSIZE | RF_PCC | RF_WIND
    int32_t ntx, nty, ntz, ntiles;     // tiles along x, y, z (1 in 2D)
    int64_t N;
    uint64_t thr, seed;
    uint8_t *spin, *bond;              // N states (read by launch 0, written by the last), N bond bytes
    int32_t *label;                    // N labels of the last sweep
    uint16_t *code;                    // ntiles * sites-per-tile
    uint32_t *cross;                   // ntiles * cross words
    int32_t *npar, *nkey;              // ntiles * slots
    uint32_t *nfinal;                  // ntiles * slots: a representative's cluster root
    uint8_t *nstate;                   // ntiles * slots: a representative's new state
    int32_t *psize, *csize;            // ntiles * slots (RF_CSIZE only)
    int4 *wlink;                       // RF_WIND: ntiles * slots node links {parent, dx, dy, dz}
    // PCC (null otherwise): the threshold lives on the device and follows the
    // feedback; per node and axis a < dim, a root's candidate id (cid, id + 2),
    // per border piece its occupied coordinates (pmask), per axis the
    // candidates (cand + a F, F = L^(dim-1) face sites), their counts
    // (ncand[a]; ncand[3] counts finished decision blocks) and coverage
    // (cov + a F W, W = ceil(L / 32) words per candidate)
    uint64_t *thr_dev;
    uint32_t *pmask;
    int32_t *cid, *cand, *ncand;
    uint32_t *cov;
};

// Tile counts and per-tile sizes of a Potts lattice's scratch.
struct PottsGeometry {
    int32_t ntx, nty, ntz, ntiles;
    int32_t sites_per_tile, slots, cross_words, pmask_words;
};
__attribute__((visibility("hidden"))) void potts_geometry(int dim, int L, PottsGeometry *g);
__attribute__((visibility("hidden"))) cudaError_t potts_enqueue_hot_start(const PottsDev &p, cudaStream_t st);
// Launch j (0 .. nsweeps) of a call: the tile kernel, then (j < nsweeps) the merge of sweep j.
__attribute__((visibility("hidden"))) cudaError_t potts_enqueue_tile(const PottsDev &p, int j, int nsweeps,
                                                                     uint64_t sweep0, DevObs *obs, cudaStream_t st);
__attribute__((visibility("hidden"))) cudaError_t potts_enqueue_merge(const PottsDev &p, int j, uint64_t sweep0,
                                                                      DevObs *obs, cudaStream_t st);
// One call of nsweeps sweeps (observables into obs[0 .. nsweeps-1]).
__attribute__((visibility("hidden"))) cudaError_t potts_enqueue_sweeps(const PottsDev &p, int nsweeps,
                                                                       uint64_t sweep0, DevObs *obs,
                                                                       cudaStream_t st);
__attribute__((visibility("hidden"))) cudaError_t potts_enqueue_check(const uint8_t *s, int64_t n, int q, int32_t *bad,
                                                                      cudaStream_t st);

}  // namespace swg
