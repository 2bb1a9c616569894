// sw_noalloc.cu -- sw_sweep_static: one Swendsen-Wang sweep on caller-owned
// device buffers, with every piece of scratch memory in a fixed array that
// is part of the loaded library, so the call allocates nothing.
//
// Who needs this: callers that may not, or cannot, call cudaMalloc -- a
// framework or memory pool that owns all device memory and forbids foreign
// allocations, code running from an allocator hook or a host callback, or a
// real-time loop where cudaMalloc's implicit device synchronisation and
// latency are not acceptable.
//
// Every other buffer the sweep touches (site codes, bond bits, border
// nodes) is fully rewritten by each sweep before it is read, so only the
// lattice descriptor, the tile table and the caller's observables are set up
// (zeroed where they accumulate) at the start of every call.
//
// Costs and rules:
//   - SW_STATIC_MAX_L x SW_STATIC_MAX_L is the largest lattice; the array
//     (SCRATCH_BYTES below: 2,755,328 bytes, 2.63 MiB) stays reserved on
//     every GPU that loads the library until the process exits.
//   - All calls share the one array: two calls that overlap on the GPU (on
//     different streams, or from different threads) race and corrupt each
//     other.  Serialise them.
//   - The first call on a device looks the array's device address up
//     (cudaGetSymbolAddress) and raises the tile kernel's shared-memory limit
//     on that device; make that first call before any stream capture begins.
//   - The kernels store spins 8 bytes, labels 16 bytes and observables 8
//     bytes at a time: spin_out must be 8-byte, labels_out 16-byte and
//     obs_out 8-byte aligned (buffers from cudaMalloc are 256-byte aligned).
#include "swgpu.h"
#include "sw_device.cuh"
#include "sw_internal.h"
#include "sw_launch.cuh"

#include <cuda_runtime.h>

#include <mutex>

using namespace swg;

namespace {

constexpr int TH_STATIC = 128;
constexpr int MAX_TILES_STATIC = (SW_STATIC_MAX_L / TW) * (SW_STATIC_MAX_L / TH_STATIC);
constexpr int S_STATIC = 2 * TW + 2 * TH_STATIC;

// Layout of the scratch array (byte offsets, each 256-byte aligned).
constexpr size_t al(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t OFF_REP = 0;
constexpr size_t OFF_TILE_REP = OFF_REP + al(sizeof(Replica));
constexpr size_t OFF_JBASE = OFF_TILE_REP + al(MAX_TILES_STATIC * sizeof(int32_t));
constexpr size_t OFF_CODE = OFF_JBASE + al(sizeof(int32_t));
constexpr size_t OFF_BONDBITS = OFF_CODE + al((size_t)MAX_TILES_STATIC * TH_STATIC * TW * sizeof(uint16_t));
constexpr size_t OFF_CROSS = OFF_BONDBITS + al((size_t)MAX_TILES_STATIC * TH_STATIC * 2 * TWW * sizeof(uint32_t));
constexpr size_t OFF_NPAR = OFF_CROSS + al((size_t)MAX_TILES_STATIC * CROSS_WORDS * sizeof(uint32_t));
constexpr size_t OFF_NKEY = OFF_NPAR + al((size_t)MAX_TILES_STATIC * S_STATIC * sizeof(int32_t));
constexpr size_t OFF_NFINAL = OFF_NKEY + al((size_t)MAX_TILES_STATIC * S_STATIC * sizeof(int32_t));
constexpr size_t SCRATCH_BYTES = OFF_NFINAL + al((size_t)MAX_TILES_STATIC * S_STATIC * sizeof(uint32_t));
static_assert(SCRATCH_BYTES == 2755328, "the size quoted in the comments and the header");

// The scratch memory itself: file scope, fixed size, no allocation.
static __device__ __align__(256) unsigned char g_static_scratch[SCRATCH_BYTES];

// Per-device address of g_static_scratch (host code cannot use the symbol
// itself as a device address).
constexpr int MAX_DEVICES = 64;
unsigned char *g_scratch_dev[MAX_DEVICES] = {nullptr};
std::mutex g_setup_mu;

// Writes the lattice descriptor and tile table into the scratch array and
// zeroes the caller's observables (everything that must start at zero).
__global__ void k_static_setup(unsigned char *scratch, Replica R, int n_tiles, DevObs *obs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        *reinterpret_cast<Replica *>(scratch + OFF_REP) = R;
        *reinterpret_cast<int32_t *>(scratch + OFF_JBASE) = 0;
        DevObs z{};
        *obs = z;
    }
    int32_t *tile_rep = reinterpret_cast<int32_t *>(scratch + OFF_TILE_REP);
    for (int g = i; g < MAX_TILES_STATIC; g += gridDim.x * blockDim.x) tile_rep[g] = g < n_tiles ? 0 : -1;
}

int setup_device(int dev, unsigned char **out)
{
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (dev < 0 || dev >= MAX_DEVICES) return SW_ERR_ARG;
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return SW_ERR_CUDA;
        if (prepare_th(TH_STATIC) != cudaSuccess) return SW_ERR_CUDA;
        g_scratch_dev[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_dev[dev];
    return SW_OK;
}

}  // namespace

extern "C" int sw_sweep_static(const uint8_t *spin_in, uint8_t *spin_out, int32_t *labels_out, sw_obs *obs_out,
                               int32_t L, uint64_t threshold, uint64_t seed, uint64_t sweep, void *stream)
{
    if (!spin_in || !spin_out || !labels_out || !obs_out) return SW_ERR_ARG;
    if (L < 2 || L > SW_STATIC_MAX_L) return SW_ERR_ARG;
    if (threshold > ((uint64_t)1 << 32)) return SW_ERR_ARG;
    // the widths of the kernels' stores (a misaligned one would fault on the GPU)
    if (((uintptr_t)spin_out & 7u) || ((uintptr_t)labels_out & 15u) || ((uintptr_t)obs_out & 7u))
        return SW_ERR_ARG;
    // spin_in is copied to spin_out first: the two must be the same buffer
    // or not overlap at all
    const uintptr_t n_bytes = (uintptr_t)L * (uintptr_t)L;
    const uintptr_t a0 = (uintptr_t)spin_in, b0 = (uintptr_t)spin_out;
    if (a0 != b0 && a0 < b0 + n_bytes && b0 < a0 + n_bytes) return SW_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SW_ERR_CUDA;
    unsigned char *scratch = nullptr;
    int rc = setup_device(dev, &scratch);
    if (rc != SW_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaGetLastError();

    const int tiles_x = (L + TW - 1) / TW, tiles_y = (L + TH_STATIC - 1) / TH_STATIC;
    Replica R{};
    R.L = L;
    R.tiles_x = tiles_x;
    R.tiles_y = tiles_y;
    R.tile_base = 0;
    R.key0 = (uint32_t)seed;
    R.key1 = (uint32_t)(seed >> 32);
    R.nsweeps = 1;
    R.flags = 0;
    R.sweep0 = sweep;
    R.thr = threshold;
    R.thr_dev = nullptr;
    // the tile kernel reads the spins at its first launch and writes the new
    // spins and the labels at its second
    R.spin = spin_out;
    R.label = labels_out;
    R.obs = reinterpret_cast<DevObs *>(obs_out);
    R.jstart = 0;
    R.code = reinterpret_cast<uint16_t *>(scratch + OFF_CODE);
    R.bondbits = reinterpret_cast<uint32_t *>(scratch + OFF_BONDBITS);
    R.cross = reinterpret_cast<uint32_t *>(scratch + OFF_CROSS);
    R.npar = reinterpret_cast<int32_t *>(scratch + OFF_NPAR);
    R.nkey = reinterpret_cast<int32_t *>(scratch + OFF_NKEY);
    R.nfinal = reinterpret_cast<uint32_t *>(scratch + OFF_NFINAL);

    if (spin_in != spin_out &&
        cudaMemcpyAsync(spin_out, spin_in, (size_t)L * L, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return SW_ERR_CUDA;
    k_static_setup<<<(MAX_TILES_STATIC + 255) / 256, 256, 0, st>>>(scratch, R, tiles_x * tiles_y,
                                                                    reinterpret_cast<DevObs *>(obs_out));
    if (cudaGetLastError() != cudaSuccess) return SW_ERR_CUDA;

    SweepArgs a{};
    a.reps = reinterpret_cast<const Replica *>(scratch + OFF_REP);
    a.tile_rep = reinterpret_cast<const int32_t *>(scratch + OFF_TILE_REP);
    a.n_tiles = tiles_x * tiles_y;
    a.jbase = reinterpret_cast<const int32_t *>(scratch + OFF_JBASE);
    a.j = 0;   // start the sweep (bonds, tile labels, border nodes) ...
    if (enqueue_launch_th(TH_STATIC, a, false, 0, 1, st) != cudaSuccess) return SW_ERR_CUDA;
    a.j = 1;   // ... and finish it (cluster flip, spins, labels, observables)
    if (enqueue_tile(TH_STATIC, a, false, 0, st) != cudaSuccess) return SW_ERR_CUDA;
    return SW_OK;
}
