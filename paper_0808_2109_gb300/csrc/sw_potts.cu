// sw_potts.cu -- the q-state Potts model on periodic 2D and 3D lattices
// (sw_create_potts in include/swgpu.h): the cluster update of Sec. I with
// "equal spins" read as "equal states", on the d-dimensional lattice the
// paper states its method for (Sec. II).
//
// A site-level path, one thread per site: bonds, unions in a global
// union-find (the smaller index wins, so roots are cluster minima), a
// flattening pass, the new states, and the sums.  The tiled 2D Ising kernels
// keep spins as single bits and do not carry over to q states or a third
// dimension; this path trades their speed for generality.
//
// Conventions (both sides implement them; the CPU oracle is the reference):
//   - N = L^d sites, i = x + L*y (+ L*L*z); site i owns link dir = 0 (+x),
//     1 (+y), 2 (+z) with index l = d*i + dir; bond byte bit dir.
//   - A link between equal states bonds iff word (l mod 4) of Philox(l/4, k,
//     BOND) < t, t = floor((1 - exp(-J/T)) 2^32).
//   - A cluster with root r takes state floor(w q / 2^32), w = word (r mod 4)
//     of Philox(r/4, k, QSPIN); the hot start is the same function of word
//     (i mod 4) of Philox(i/4, 0, INIT).
//   - bond_sum = sum over links of (2 delta - 1), mag = sum over sites of
//     (q [s_i = 0] - 1).
#include "swgpu.h"
#include "sw_device.cuh"
#include "sw_internal.h"
#include "sw_launch.cuh"

#include <cuda_runtime.h>

#include <algorithm>

using namespace swg;

namespace {

constexpr uint32_t STREAM_QSPIN = 3;
constexpr int PT = 256;   // threads per block

__device__ __forceinline__ uint8_t potts_state(uint32_t w, int q)
{
    return (uint8_t)(((uint64_t)w * (uint32_t)q) >> 32);
}

__device__ __forceinline__ int64_t nd_neighbour(const PottsDev &p, int64_t i, int dir)
{
    const int64_t L = p.L;
    int64_t x = i % L, y = (i / L) % L, z = i / (L * L);
    if (dir == 0)
        x = x + 1 == L ? 0 : x + 1;
    else if (dir == 1)
        y = y + 1 == L ? 0 : y + 1;
    else
        z = z + 1 == L ? 0 : z + 1;
    return p.dim == 2 ? y * L + x : (z * L + y) * L + x;
}

__device__ __forceinline__ int pfind(int32_t *lab, int x)
{
    int p = gload(lab + x);
    while (p != x) {
        const int gp = gload(lab + p);
        if (gp != p) *(volatile int32_t *)(lab + x) = gp;   // halving: an ancestor
        x = gp;
        p = gload(lab + x);
    }
    return x;
}

// Hang the larger root under the smaller (roots end as cluster minima).
__device__ __forceinline__ void punite(int32_t *lab, int a, int b)
{
    for (;;) {
        a = pfind(lab, a);
        b = pfind(lab, b);
        if (a == b) return;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(lab + b, b, a) == b) return;
    }
}

__global__ void k_potts_hot_start(const PottsDev p)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    const U4 r = philox4x32_10((uint32_t)(i >> 2), 0u, 0u, STREAM_INIT, (uint32_t)p.seed, (uint32_t)(p.seed >> 32));
    p.spin[i] = potts_state(u4_word(r, (int)(i & 3)), p.q);
}

// Every site its own cluster; cluster sizes zeroed.
__global__ void k_potts_reset(const PottsDev p)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    p.label[i] = (int32_t)i;
    if (p.size) p.size[i] = 0;
}

// Bonds of site i's own links (Sec. I step 1) and their unions (step 2).
__global__ void k_potts_bonds(const PottsDev p, uint64_t k)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    const uint32_t klo = (uint32_t)k, khi = (uint32_t)(k >> 32);
    const uint32_t k0 = (uint32_t)p.seed, k1 = (uint32_t)(p.seed >> 32);
    const uint8_t s = p.spin[i];
    const int64_t l0 = (int64_t)p.dim * i;
    // the site's links fall in one or two Philox blocks
    const int64_t m0 = l0 >> 2, m1 = (l0 + p.dim - 1) >> 2;
    const U4 r0 = philox4x32_10((uint32_t)m0, klo, khi, STREAM_BOND, k0, k1);
    U4 r1 = r0;
    if (m1 != m0) r1 = philox4x32_10((uint32_t)m1, klo, khi, STREAM_BOND, k0, k1);
    uint8_t b = 0;
    for (int dir = 0; dir < p.dim; ++dir) {
        const int64_t l = l0 + dir;
        const uint32_t u = u4_word((l >> 2) == m0 ? r0 : r1, (int)(l & 3));
        const int64_t j = nd_neighbour(p, i, dir);
        if (p.spin[j] == s && (uint64_t)u < p.thr) {
            b |= (uint8_t)(1u << dir);
            punite(p.label, (int)i, (int)j);
        }
    }
    p.bond[i] = b;
}

// Every site's label becomes its root: the cluster minimum.
__global__ void k_potts_flatten(const PottsDev p)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int x = (int)i, nx = gload(p.label + x);
    while (nx != x) {
        x = nx;
        nx = gload(p.label + x);
    }
    p.label[i] = x;
    if (p.size) atomicAdd(p.size + x, 1);
}

// New states (Sec. I step 3) and the cluster count.
__global__ void k_potts_assign(const PottsDev p, uint64_t k, DevObs *obs)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int root = 0;
    if (i < p.N) {
        const int64_t r = p.label[i];
        const U4 w = philox4x32_10((uint32_t)(r >> 2), (uint32_t)k, (uint32_t)(k >> 32), STREAM_QSPIN,
                                   (uint32_t)p.seed, (uint32_t)(p.seed >> 32));
        p.spin[i] = potts_state(u4_word(w, (int)(r & 3)), p.q);
        root = r == i;
    }
    const int n = __syncthreads_count(root);
    if (threadIdx.x == 0 && n) atomicAdd(&obs->nclusters, (unsigned long long)n);
    if (i == 0) obs->threshold = p.thr;
}

// Sums of the new states: bond_sum, mag, the bond count and sum |C|^2.
__global__ void k_potts_measure(const PottsDev p, DevObs *obs)
{
    __shared__ long long red[PT / 32][4];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    long long v[4] = {0, 0, 0, 0};
    if (i < p.N) {
        const uint8_t s = p.spin[i];
        for (int dir = 0; dir < p.dim; ++dir) v[0] += p.spin[nd_neighbour(p, i, dir)] == s ? 1 : -1;
        v[1] = s == 0 ? p.q - 1 : -1;
        v[2] = __popc((uint32_t)p.bond[i]);
        if (p.size) {
            const long long c = p.size[i];
            v[3] = c * c;
        }
    }
    unsigned long long *const dst[4] = {&obs->bond_sum, &obs->mag, &obs->nbonds, &obs->csize2};
    block_sum_atomic<PT, 4>(v, dst, red);
}

// Sets *bad if any of the n states is >= q.
__global__ void k_potts_check(const uint8_t *s, int64_t n, int q, int32_t *bad)
{
    int found = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        found |= s[i] >= q;
    if (__syncthreads_or(found) && threadIdx.x == 0) atomicOr(bad, 1);
}

unsigned blocks_of(int64_t n) { return (unsigned)((n + PT - 1) / PT); }

}  // namespace

namespace swg {

cudaError_t potts_enqueue_hot_start(const PottsDev &p, cudaStream_t st)
{
    k_potts_hot_start<<<blocks_of(p.N), PT, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t potts_enqueue_sweep(const PottsDev &p, uint64_t sweep, DevObs *obs, cudaStream_t st)
{
    const unsigned nb = blocks_of(p.N);
    k_potts_reset<<<nb, PT, 0, st>>>(p);
    k_potts_bonds<<<nb, PT, 0, st>>>(p, sweep);
    k_potts_flatten<<<nb, PT, 0, st>>>(p);
    k_potts_assign<<<nb, PT, 0, st>>>(p, sweep, obs);
    k_potts_measure<<<nb, PT, 0, st>>>(p, obs);
    return cudaGetLastError();
}

cudaError_t potts_enqueue_check(const uint8_t *s, int64_t n, int q, int32_t *bad, cudaStream_t st)
{
    const unsigned nb = (unsigned)std::min<int64_t>((n + 4095) / 4096, 4096);
    k_potts_check<<<nb > 0 ? nb : 1, PT, 0, st>>>(s, n, q, bad);
    return cudaGetLastError();
}

}  // namespace swg
