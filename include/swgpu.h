/*
 * swgpu.h -- C ABI of the GB300 (sm_103a) Swendsen-Wang / PCC library.
 *
 * Paper: S. Lin and B. Zheng, "Two Parallel Swendsen-Wang Cluster Algorithms
 * Using Message-Passing Paradigm" (arXiv:0808.2109).  The problem statement
 * is the paper's: an L x L periodic Ising lattice H = -J sum sigma_i sigma_j,
 * temperature T (or a bond probability p), swept by the Swendsen-Wang update
 * of Sec. I (steps 1-4); PCC (Sec. I, Sec. III) tunes p by percolation
 * feedback.
 *
 * Conventions shared by every call
 *   - Every call returns SW_OK (0) or a negative SW_ERR_* code; nothing
 *     throws across the ABI.  sw_strerror() names a code.
 *   - The library owns all device memory it allocates.  Host buffers passed
 *     in are owned by the caller and are only read or written during the
 *     call.
 *   - Site index i = y*L + x (row-major).  Site i owns link d=0 to
 *     (x+1 mod L, y) and link d=1 to (x, y+1 mod L).  Spins are uint8 s in
 *     {0,1} with sigma = 2s-1.  Labels are int32 roots: the minimum site
 *     index of the cluster.  Bond bytes: bit0 = right link, bit1 = down link.
 *   - Random numbers: Philox4x32-10, key = (seed mod 2^32, seed >> 32),
 *     counter = (index word, sweep mod 2^32, sweep >> 32, stream) with
 *     streams INIT=0 (hot start, bit i mod 128 of block i/128), BOND=1
 *     (word l mod 4 of block l/4 for link l = 2i+d) and SPIN=2 (bit r mod 128
 *     of block r/128 for a cluster with root r).  Sweep k counts the sweeps
 *     since the lattice was created (k = 0 first).
 *   - The bond threshold t = floor(P * 2^32) (an integer in [0, 2^32]) is
 *     computed once on the host in IEEE double; a link between equal spins
 *     is bonded iff its 32-bit word u < t.
 *   - The GPU path supports 2 <= L <= 32768.
 *   - Work is queued on the context's stream (default: a stream the library
 *     creates); calls that return host data synchronise that stream.
 *   - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef SWGPU_H
#define SWGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define SW_OK 0
#define SW_PENDING 1          /* sw_batch_poll: the job has not finished yet  */
#define SW_ERR_ARG (-1)       /* an argument is out of range or NULL          */
#define SW_ERR_NOMEM (-2)     /* device or host memory could not be obtained  */
#define SW_ERR_CUDA (-3)      /* a CUDA runtime call or kernel launch failed   */
#define SW_ERR_TIMEOUT (-4)   /* a bounded device-side wait ran out            */
#define SW_ERR_STATE (-5)     /* the call does not fit the object's state      */

/* Creation flags.  A tile-height flag fixes the rows per 128-site-wide tile
 * (results do not depend on it; it trades shared memory against the number
 * of border nodes); without one the library picks from L. */
#define SW_FLAG_NONE 0u
#define SW_FLAG_TILE_32 (1u << 8)
#define SW_FLAG_TILE_64 (1u << 9)
#define SW_FLAG_TILE_128 (1u << 10)
#define SW_FLAG_TILE_96 (1u << 11)
/* Open (free) boundaries instead of periodic ones (Sec. III treats both):
 * the right link of column L-1 and the down link of row L-1 do not exist --
 * they never bond and add nothing to bond_sum -- and the PCC span test is
 * the open-boundary one (a cluster touches both opposite borders). */
#define SW_FLAG_OPEN (1u << 12)
/* Also sum |C|^2 over every sweep's clusters into sw_obs.csize2 (two more
 * int32 per border node of device memory).  Each cluster takes an independent
 * fair sign, so the mean of csize2 is <M^2>: the cluster ("improved")
 * estimator of the susceptibility, with a smaller variance than M^2. */
#define SW_FLAG_CSIZE (1u << 13)
/* Topological rule (Sec. III): spans_x / spans_y report, every sweep,
 * whether some cluster winds around the box in x / y (holds a closed path of
 * bonds whose net displacement is a non-zero multiple of L), and a PCC
 * lattice feeds back on that instead of the extension rule.  One more 8-byte
 * word per border node of device memory. */
#define SW_FLAG_WIND (1u << 14)

typedef struct sw_ctx sw_ctx; /* opaque; owned by the library */

/* Observables of one sweep, all taken after the cluster flip of Sec. I
 * step 3 (a reading: the paper does not say when it measures). */
typedef struct {
    int64_t bond_sum;   /* sum over the links (2N periodic, 2L(L-1) open) of
                           sigma_i sigma_j; E = -J bond_sum                    */
    int64_t mag;        /* sum of sigma_i                                      */
    int64_t nclusters;  /* clusters built in this sweep (Sec. I step 2)        */
    int64_t nbonds;     /* bonded links in this sweep (Sec. I step 1)          */
    int32_t spans_x;    /* PCC: a cluster occupies all L columns (Sec. III);
                           open boundaries: it touches columns 0 and L-1,
                           which is the same for clusters without wrap links */
    int32_t spans_y;    /* PCC: the same for rows                              */
    uint64_t threshold; /* bond threshold t used in this sweep                 */
    int64_t csize2;     /* SW_FLAG_CSIZE: sum over this sweep's clusters of
                           |C|^2; 0 without the flag                          */
} sw_obs;

/* Snapshot of a lattice's scalar state (the spins are read separately). */
typedef struct {
    int32_t L;
    int32_t pcc;        /* 1 for a PCC lattice                               */
    uint64_t seed;
    uint64_t sweep;     /* sweeps done since creation = index of the next one */
    uint64_t threshold; /* threshold the next sweep will use                 */
    int32_t open;       /* 1 for open boundaries (SW_FLAG_OPEN)              */
    int32_t tile_h;     /* rows per tile (0 for a Potts lattice)             */
    int32_t dim;        /* 2, or 3 for a 3D Potts lattice                    */
    int32_t q;          /* states per site (2 for the Ising lattices)        */
} sw_state;

/* Name of a status code (static string). */
const char *sw_strerror(int code);

/* The CUDA runtime's description of the last CUDA failure the library saw
 * on the calling thread ("" if none); diagnostic text for SW_ERR_CUDA and
 * SW_ERR_NOMEM. */
const char *sw_last_error_detail(void);

/* Bond threshold of Sec. I step 1: t = floor((1 - exp(-2J/T)) * 2^32).
 * J >= 0 and T > 0 (T may be +inf); else SW_ERR_ARG. */
int sw_threshold(double J, double T, uint64_t *out);

/* Create an L x L lattice with coupling J >= 0 at temperature T > 0
 * (Sec. I: P = 1 - exp(-2J/T)), hot start from `seed` (every spin an
 * independent fair bit of the INIT stream).  *out receives the context.
 * Errors: SW_ERR_ARG (L outside [2, 32768], J < 0, T <= 0, out NULL),
 * SW_ERR_NOMEM, SW_ERR_CUDA.  On error *out is set to NULL. */
int sw_create(sw_ctx **out, int32_t L, double J, double T, uint64_t seed, uint32_t flags);

/* As sw_create, with the bond probability p in [0, 1] given directly. */
int sw_create_p(sw_ctx **out, int32_t L, double p, uint64_t seed, uint32_t flags);

/* Create a PCC lattice (the probability-changing cluster method the paper
 * parallelises in Sec. III): threshold starts at 2^31 (p = 1/2); after sweep
 * k it moves by delta_k = 2^(32 - min(8 + floor(k/1000), 20)) threshold
 * units, down if some cluster of that sweep spans the lattice in x or y by
 * the extension rule under periodic boundaries, up otherwise, clamped to
 * [0, 2^32].  Errors as sw_create. */
int pcc_create(sw_ctx **out, int32_t L, uint64_t seed, uint32_t flags);

/* A q-state Potts lattice (2 <= q <= 256) on the periodic d-dimensional
 * torus, d = 2 or 3, L^d <= 2^30 sites: the cluster update of Sec. I with
 * equal states bonding (H = -J sum delta(s_i, s_j), P = 1 - exp(-J/T); q = 2
 * is Ising at J/2) on the d-dimensional lattice the paper states its method
 * for (Sec. II), on the tiled design of the 2D Ising path (2D tiles of 128 x
 * 64 sites, 3D tiles of 32 x 16 x 16).  Sites i = x + L y (+ L^2 z); link l = d i + dir (dir 0: +x, 1: +y, 2: +z)
 * draws word (l mod 4) of Philox(l/4, k, BOND); a cluster with root r takes
 * state floor(w q / 2^32), w = word (r mod 4) of Philox(r/4, k, stream 3);
 * the hot start is the same of word (i mod 4) of Philox(i/4, 0, INIT).
 * Observables: bond_sum = sum over links of (2 delta - 1), mag = sum over
 * sites of (q [s_i = 0] - 1).  flags: SW_FLAG_CSIZE, SW_FLAG_OPEN (open
 * boundaries: the last coordinate along a direction has no + link, which
 * neither bonds nor enters bond_sum) and SW_FLAG_WIND (the topological rule
 * of Sec. III reported every sweep: spans_x = some cluster winds around the
 * box along x, spans_y = along y, or in 3D along y or z), or 0.  The other
 * calls take the context as usual (spins, labels and bond bytes have L^d
 * entries, bond bit dir; sw_profile times its tile kernel and merge); pcc_step
 * on a lattice not made by pcc_create_potts answers SW_ERR_STATE.  Errors:
 * SW_ERR_ARG, SW_ERR_NOMEM, SW_ERR_CUDA. */
int sw_create_potts(sw_ctx **out, int32_t dim, int32_t L, int32_t q, double J, double T, uint64_t seed,
                    uint32_t flags);

/* A PCC lattice on the Potts path (Sec. III, whose percolation criteria hold
 * in any dimension): as sw_create_potts, with the bond threshold starting at
 * 2^31 and moved after every sweep by the feedback of pcc_create (down by
 * delta_k if some cluster spans some axis, up otherwise).  A cluster spans
 * axis a when it occupies all L hyperplanes perpendicular to a (the
 * extension rule; under open boundaries, touching both faces).  Per sweep
 * spans_x reports the x axis and spans_y the y axis, or in 3D the y or the z
 * axis.  With SW_FLAG_WIND the criterion is the topological rule instead
 * (some cluster winds around the box along some axis).  flags: SW_FLAG_CSIZE,
 * SW_FLAG_OPEN, SW_FLAG_WIND or 0.  Errors as sw_create_potts. */
int pcc_create_potts(sw_ctx **out, int32_t dim, int32_t L, int32_t q, uint64_t seed, uint32_t flags);

/* Release the context and all its device memory.  NULL is accepted. */
int sw_destroy(sw_ctx *ctx);

/* Queue the context's work on `stream` (a cudaStream_t; NULL = the library's
 * own stream).  The caller keeps ownership of the stream. */
int sw_set_stream(sw_ctx *ctx, void *stream);

/* Run `nsweeps` >= 0 Swendsen-Wang sweeps (Sec. I steps 1-4).  Asynchronous
 * on the context's stream.  Afterwards the device holds the new spins, the
 * labels and bonds of the last sweep, and one sw_obs per sweep pending for
 * sw_observables.  On a PCC context this is the same as pcc_step.
 * Errors: SW_ERR_ARG (nsweeps < 0), SW_ERR_NOMEM, SW_ERR_CUDA. */
int sw_sweep(sw_ctx *ctx, int32_t nsweeps);

/* Run `nsweeps` PCC sweeps: each is a Swendsen-Wang sweep, the span test of
 * Sec. III on its clusters, and the threshold feedback.  Errors as sw_sweep,
 * plus SW_ERR_STATE when ctx was not made by pcc_create. */
int pcc_step(sw_ctx *ctx, int32_t nsweeps);

/* Copy the observables of the sweeps run since the last call (oldest first)
 * into the caller's out[max]; *n_written receives how many.  Entries that do
 * not fit stay pending for the next call.  Synchronises the stream. */
int sw_observables(sw_ctx *ctx, sw_obs *out, int32_t max, int32_t *n_written);

/* Copy the L*L spins (uint8 0/1) to host_out.  Synchronises the stream. */
int sw_get_spins(sw_ctx *ctx, uint8_t *host_out);

/* Replace the L*L spins by host_in (each byte must be 0 or 1, else
 * SW_ERR_ARG).  The sweep counter and threshold are unchanged.
 * Synchronises the stream. */
int sw_set_spins(sw_ctx *ctx, const uint8_t *host_in);

/* Copy the L*L labels of the last sweep (root = minimum site index of each
 * cluster, Sec. II.B steps 4-6) to host_out.  SW_ERR_STATE before the first
 * sweep.  Synchronises the stream. */
int sw_get_labels(sw_ctx *ctx, int32_t *host_out);

/* Copy the L*L bond bytes of the last sweep to host_out.  SW_ERR_STATE
 * before the first sweep.  Synchronises the stream. */
int sw_get_bonds(sw_ctx *ctx, uint8_t *host_out);

/* Scalar state of the lattice. */
int sw_get_state(sw_ctx *ctx, sw_state *out);

/* Wait for all work queued on the context's stream. */
int sw_sync(sw_ctx *ctx);

/* Device time of the kernels of the sweeps run since the last read, from
 * CUDA events recorded around them.  (Measurement support: the paper's
 * per-step timings, Sec. II.C, have no other counterpart here.) */
typedef struct {
    int64_t tile_launches; /* launches of the tile kernel                   */
    double tile_ms;        /* their summed device time                      */
    int64_t merge_groups;  /* launch groups (a group = the three merge kernels) */
    double merge_ms;       /* summed device time of the merge groups         */
    int64_t tile_sites;    /* L*L (a Potts lattice: L^d)                     */
    int32_t tile_height;   /* rows per tile (tiles are 128 sites wide); 0 on a
                              Potts lattice, whose tiles are 128 x 64 (2D) or
                              32 x 16 x 16 (3D)                              */
} sw_kernel_stats;

/* enable != 0: later sweeps are launched one kernel at a time (not as CUDA
 * graphs) with events around every kernel; 0 restores graph launches. */
int sw_profile(sw_ctx *ctx, int32_t enable);

/* Synchronise, return the accumulated kernel times and reset them. */
int sw_profile_read(sw_ctx *ctx, sw_kernel_stats *out);

/* ---------------------------------------------------- checkpoint / resume
 * (The paper has no counterpart.)  A lattice's state is its spins, seed,
 * sweep counter and threshold (plus its kind: PCC, open boundaries, the
 * topological rule, d and q); labels and bonds are rebuilt by the next
 * sweep.  Because every random number is a counter-based Philox draw, a chain
 * saved after n sweeps and resumed for m more equals a straight run of n + m
 * sweeps bit for bit. */

/* Size in bytes of a checkpoint of this lattice (a header and L^d bytes). */
int sw_checkpoint_bytes(sw_ctx *ctx, uint64_t *bytes);

/* Write the state into the caller's host buffer (at least
 * sw_checkpoint_bytes); waits for the sweeps queued on the context. */
int sw_save(sw_ctx *ctx, void *host_buf, uint64_t bytes);

/* Replace the context's state by a saved one.  The context must be of the same
 * kind, L, d and q (its seed may differ: the saved seed is taken); else
 * SW_ERR_ARG, as for a corrupt buffer or out-of-range states.  sw_get_labels
 * and sw_get_bonds answer SW_ERR_STATE until the next sweep. */
int sw_load(sw_ctx *ctx, const void *host_buf, uint64_t bytes);

/* Integer ceiling of the bond step (measurement support).  Sec. II's cost
 * model charges every sweep a per-site bond-activating time tau_site; here
 * that work is Philox4x32-10 draws, so their rate bounds the sweep.  Draws
 * the BOND-stream blocks with counters 0 .. nblocks-1 (sweep 0, key = seed)
 * on a grid that fills the GPU, four blocks in flight per thread, and xors
 * every word into *out_dev (a caller-owned 4-byte-aligned device word; the
 * call does not clear it).  Asynchronous on `stream` (a cudaStream_t, NULL:
 * the legacy default stream); time it with events on that stream to get
 * blocks per second.  0 <= nblocks <= 2^32, else SW_ERR_ARG; a NULL or
 * misaligned out_dev: SW_ERR_ARG. */
int sw_bench_philox(int64_t nblocks, uint64_t seed, uint32_t *out_dev, void *stream);

/* L2 copy ceiling (measurement support for the lattices whose state fits
 * the L2 cache, Sec. II.C's smaller L).  reps passes of dst = src ^ pass over
 * `bytes` bytes of caller-owned device memory, loads and stores cached in L2
 * only; with src and dst together smaller than L2, every pass after the
 * first runs out of L2.  Time it with events on `stream`: 2 * bytes * reps /
 * time is the copy bandwidth.  Both buffers 16-byte aligned, not
 * overlapping, bytes > 0 and a multiple of 16, reps >= 1; else SW_ERR_ARG. */
int sw_bench_l2(const void *src_dev, void *dst_dev, int64_t bytes, int32_t reps, void *stream);

/* Fault injection for tests (host side; the paper has no counterpart): of
 * the library's next device allocations, the first `skip` proceed and the n
 * after them report out-of-memory without allocating, so callers see
 * SW_ERR_NOMEM (contexts) or a job result with that status (servers).
 * n = 0 switches it off. */
int sw_debug_fail_allocations(int32_t skip, int32_t n);

/* ------------------------------------------------- batched and served runs
 * Many independent lattices on one GPU at once (the paper's decompositions
 * spread ONE lattice over processors, Sec. II; here independent lattices
 * share the device).  A server owns a worker thread that admits submitted
 * jobs while their device memory fits its budget, runs every admitted
 * lattice in the same kernel launches (one tile table over all of them,
 * captured as CUDA graphs), lets new jobs join at sweep boundaries and
 * copies finished jobs out.  A job's results equal those of the same
 * lattice run alone with sw_create/pcc_create and sw_sweep. */
typedef struct sw_server sw_server;

#define SW_JOB_SW 0   /* plain SW at (J, T)                  */
#define SW_JOB_SWP 1  /* plain SW at bond probability p      */
#define SW_JOB_PCC 2  /* PCC lattice (threshold starts at 2^31) */

typedef struct {
    int32_t L;          /* 2 <= L <= 4096                                      */
    int32_t kind;       /* SW_JOB_*                                            */
    double J, T, p;     /* J, T for SW_JOB_SW; p for SW_JOB_SWP                */
    uint64_t seed;
    int32_t nsweeps;    /* >= 1                                                */
    int32_t tile_h;     /* 0 = autotuned, else 32, 64, 96 or 128               */
    sw_obs *obs_out;    /* optional: nsweeps entries, written before completion */
    uint8_t *spins_out; /* optional: L*L final spins                            */
    int32_t *labels_out;/* optional: L*L labels of the last sweep               */
    uint32_t flags;     /* SW_FLAG_OPEN | SW_FLAG_CSIZE | SW_FLAG_WIND, or 0
                           (tile heights go in tile_h)                          */
} sw_job;
/* The caller owns obs_out/spins_out/labels_out; they must stay valid until
 * sw_batch_poll reports the job finished. */

typedef struct {
    int32_t status;         /* SW_OK, or the error that ended the job             */
    int32_t L, nsweeps, tile_h;
    uint64_t threshold;     /* threshold after the last sweep (PCC: fed back)     */
    int64_t sum_bond_sum;   /* sums over the sweeps of the sw_obs fields          */
    int64_t sum_abs_mag;
    int64_t sum_nclusters;
    double queued_s;        /* submit -> admitted                                 */
    double run_s;           /* admitted -> finished                               */
} sw_result;

typedef struct {
    int64_t submitted, admitted, finished, pending, active;
    int64_t site_updates;   /* L*L*nsweeps summed over finished jobs              */
    size_t bytes_in_use, bytes_budget;
    int64_t launches;       /* launch groups run by the worker                    */
} sw_server_stats;

/* Create a server on the current device with a budget of device bytes for
 * lattice state (0 = 80% of the free memory).  Errors: SW_ERR_NOMEM,
 * SW_ERR_CUDA. */
int sw_server_create(sw_server **out, size_t device_bytes, uint32_t flags);

/* Stop the worker (jobs not finished are dropped) and free everything. */
int sw_server_destroy(sw_server *srv);

/* Queue n jobs; ids_out[n] receives their ids.  A job that can never run
 * (bad arguments, or larger than the whole budget) makes the call return
 * SW_ERR_ARG / SW_ERR_NOMEM with nothing queued. */
int sw_batch_submit(sw_server *srv, const sw_job *jobs, int32_t n, uint64_t *ids_out);

/* SW_PENDING while job `id` waits or runs; SW_OK once finished, with *out
 * filled (the job is then forgotten); SW_ERR_ARG for an unknown id. */
int sw_batch_poll(sw_server *srv, uint64_t id, sw_result *out);

/* Block until every submitted job has finished (or timeout_s > 0 passes:
 * SW_ERR_TIMEOUT). */
int sw_batch_wait_all(sw_server *srv, double timeout_s);

int sw_server_get_stats(sw_server *srv, sw_server_stats *out);

/* ------------------------------------------------- sweep without allocation
 * The paper has no counterpart to this call.  It exists for callers that may
 * not, or cannot, allocate device memory: a framework or memory pool that
 * owns all device memory and forbids foreign cudaMalloc, code running from an
 * allocator hook or a host callback, or a real-time loop where cudaMalloc's
 * implicit device synchronisation and latency are not acceptable.  It runs
 * ONE Swendsen-Wang sweep k of an L x L lattice on caller-owned DEVICE
 * buffers, and all its scratch memory sits in one fixed-size array inside
 * the library (2,755,328 bytes = 2.63 MiB, reserved on every GPU that loads
 * the library until the process exits), so it calls no cudaMalloc or
 * cudaFree.
 *   spin_in   L*L spins (0/1) before the sweep
 *   spin_out  L*L spins after the sweep; equal to spin_in, or not
 *             overlapping it at all; 8-byte aligned
 *   labels_out L*L labels of the sweep (cluster roots, minimum site index);
 *             16-byte aligned
 *   obs_out   one sw_obs of the sweep (the call zeroes it first); 8-byte
 *             aligned
 *   threshold the bond threshold t in [0, 2^32] (see sw_threshold)
 *   seed, sweep  the Philox key and the sweep index k of the sweep
 *   stream    a cudaStream_t (NULL: the legacy default stream); the call is
 *             asynchronous on it
 * Buffers from cudaMalloc (256-byte aligned) meet every alignment above; a
 * view at an offset into one may not.  Results equal sw_sweep on a lattice
 * with the same spins, seed, threshold and sweep index.  Errors, all
 * returned before anything is enqueued: SW_ERR_ARG for L above
 * SW_STATIC_MAX_L (or below 2), a threshold above 2^32, a NULL buffer, a
 * misaligned buffer, or spin buffers that overlap without being equal.  The
 * one array is shared by every call: calls that overlap on the GPU (other
 * streams, other threads) race; run them one after another.  The first call
 * on a device sets the array up for that device (looks up its device address
 * and raises a kernel's shared-memory limit while the device is current):
 * make it before any stream capture starts. */
#define SW_STATIC_MAX_L 1024
int sw_sweep_static(const uint8_t *spin_in, uint8_t *spin_out, int32_t *labels_out, sw_obs *obs_out,
                    int32_t L, uint64_t threshold, uint64_t seed, uint64_t sweep, void *stream);

/* Autotuner: the fastest tile height for an L x L lattice at temperature T
 * on this GPU, timed on a short run and cached per (L, T bucket). */
int sw_autotune(int32_t L, double T, int32_t *tile_h_out);

#ifdef __cplusplus
}
#endif

#endif /* SWGPU_H */
