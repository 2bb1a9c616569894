// sw_potts.cu -- the q-state Potts model on periodic 2D and 3D lattices
// (sw_create_potts in include/swgpu.h): the cluster update of Sec. I with
// "equal spins" read as "equal states", on the d-dimensional lattice the
// paper states its method for (Sec. II).
//
// Per sweep, four kernels, the first two over bricks of sites (32 x 32 in 2D,
// 8 x 8 x 8 in 3D):
//   1. k_potts_local: the brick's states (with a halo on the + side) in shared
//      memory, its bonds, and a shared-memory union-find over the bonds inside
//      the brick; every site's label becomes its piece's minimum site;
//   2. k_potts_cross: the bonds that leave a brick unite pieces in a global
//      union-find over those labels (the smaller index wins, so roots are
//      cluster minima);
//   3. k_potts_resolve: every label becomes its cluster's root, piece sizes
//      move to the roots, every site takes its cluster's new state, and the
//      clusters are counted;
//   4. k_potts_measure: the sums.
// The tiled 2D Ising kernels keep spins as single bits and do not carry over
// to q states or a third dimension.
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
constexpr int POTTS_BY2 = 16;   // rows of a 2D brick (16 measured best of 8, 16 and 32)

__device__ __forceinline__ uint8_t potts_state(uint32_t w, int q)
{
    return (uint8_t)(((uint64_t)w * (uint32_t)q) >> 32);
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

// Sites of a brick, one thread each, and its shared states with a halo of
// one site on the + side of every axis.
template <int DIM>
struct Brick {
    static constexpr int BX = DIM == 2 ? 32 : 8, BY = DIM == 2 ? POTTS_BY2 : 8, BZ = DIM == 2 ? 1 : 8;
    static constexpr int NT = BX * BY * BZ;
    static constexpr int HX = BX + 1, HY = BY + 1, HZ = DIM == 2 ? 1 : BZ + 1;
};

// Bonds of every site's own links (Sec. I step 1); unions of the bonds inside
// the brick (step 2) in shared memory, larger root under smaller (local order
// is global order inside a brick, so a piece's root is its minimum site).
// Every site's label: its piece's minimum site; with cluster sizes, each piece
// root's size holds the piece's site count and every other size is zero.
template <int DIM>
__global__ void __launch_bounds__(Brick<DIM>::NT) k_potts_local(const PottsDev p, uint64_t k)
{
    using B = Brick<DIM>;
    __shared__ uint8_t st[B::HZ][B::HY][B::HX];
    __shared__ int par[B::NT];
    __shared__ int cnt[B::NT];
    __shared__ __align__(16) uint32_t uw[DIM * B::NT];   // the BOND words of the brick's links
    const int L = p.L;
    const int x0 = blockIdx.x * B::BX, y0 = blockIdx.y * B::BY, z0 = blockIdx.z * B::BZ;
    const uint32_t uL = (uint32_t)L;
    // past the lattice's last site the halo wraps (a lattice narrower than a
    // brick wraps more than once)
    auto wrap = [L](int g) { return (uint32_t)(g < L ? g : g % L); };
    if (DIM == 2) {
        // a warp per halo row: lane x loads site x0 + x, lane 0 also the
        // halo column's site
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const uint32_t gx = wrap(x0 + lane), gh = wrap(x0 + B::BX);
        for (int hy = warp; hy < B::HY; hy += B::NT / 32) {
            const uint8_t *row = p.spin + (size_t)uL * wrap(y0 + hy);
            st[0][hy][lane] = row[gx];
            if (lane == 0) st[0][hy][B::BX] = row[gh];
        }
    } else if ((L & 7) == 0) {
        // L a multiple of 8: each halo row's 8 brick sites are one aligned
        // 8-byte load (x0 is a multiple of 8, so is every row start); thread
        // t < 81 loads row (t mod 9, t / 9) and its halo site
        if (threadIdx.x < B::HY * B::HZ) {
            const int hy = threadIdx.x % B::HY, hz = threadIdx.x / B::HY;
            const size_t row = (size_t)uL * (wrap(y0 + hy) + (size_t)uL * wrap(z0 + hz));
            const uint2 v = *reinterpret_cast<const uint2 *>(p.spin + row + (uint32_t)x0);
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                st[hz][hy][x] = (uint8_t)(v.x >> (8 * x));
                st[hz][hy][4 + x] = (uint8_t)(v.y >> (8 * x));
            }
            st[hz][hy][B::BX] = p.spin[row + wrap(x0 + B::BX)];
        }
    } else {
        for (int q = threadIdx.x; q < B::HX * B::HY * B::HZ; q += B::NT) {
            const int hx = q % B::HX, hy = (q / B::HX) % B::HY, hz = q / (B::HX * B::HY);
            const uint32_t gx = wrap(x0 + hx), gy = wrap(y0 + hy), gz = wrap(z0 + hz);
            st[hz][hy][hx] = p.spin[gx + uL * (gy + uL * gz)];
        }
    }
    const int t = threadIdx.x;
    const int lx = t % B::BX, ly = (t / B::BX) % B::BY, lz = t / (B::BX * B::BY);
    const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
    const bool valid = gx < L && gy < L && (DIM == 2 || gz < L);
    const uint32_t i = (uint32_t)gx + uL * ((uint32_t)gy + uL * (uint32_t)gz);   // N <= 2^30
    par[t] = t;
    if (p.size) cnt[t] = 0;
    const uint32_t klo = (uint32_t)k, khi = (uint32_t)(k >> 32);
    const uint32_t k0 = (uint32_t)p.seed, k1 = (uint32_t)(p.seed >> 32);
    const uint64_t thr = p.thr_dev ? *p.thr_dev : p.thr;
    if (DIM == 2 && (L & 1) == 0) {
        // even L: a 2D brick row of 32 sites starts on an even site, so its
        // 64 links are exactly the 16 Philox blocks from (site index) / 2;
        // thread t < 16 BY draws block t & 15 of row t >> 4 (words of sites
        // past the lattice's edge are drawn but never read)
        if (t < 16 * B::BY) {
            const int row = t >> 4, jb = t & 15;
            if (y0 + row < L) {
                const uint32_t i0 = (uint32_t)x0 + uL * (uint32_t)(y0 + row);
                const U4 r = philox4x32_10((i0 >> 1) + (uint32_t)jb, klo, khi, STREAM_BOND, k0, k1);
                *reinterpret_cast<uint4 *>(&uw[64 * row + 4 * jb]) = make_uint4(r.x, r.y, r.z, r.w);
            }
        }
    } else if (DIM == 3 && (L & 3) == 0) {
        // L a multiple of 4: a 3D brick row of 8 sites starts on a site i0
        // that is a multiple of 4, so its 24 links are exactly the 6 Philox
        // blocks from 3 i0 / 4; thread t < 384 draws block t mod 6 of row t / 6
        if (t < 6 * B::BY * B::BZ) {
            const int row = t / 6, jb = t % 6;
            const int ry = row % B::BY, rz = row / B::BY;
            if (y0 + ry < L && z0 + rz < L) {
                const uint32_t i0 = (uint32_t)x0 + uL * ((uint32_t)(y0 + ry) + uL * (uint32_t)(z0 + rz));
                const U4 r = philox4x32_10(3u * (i0 >> 2) + (uint32_t)jb, klo, khi, STREAM_BOND, k0, k1);
                *reinterpret_cast<uint4 *>(&uw[24 * row + 4 * jb]) = make_uint4(r.x, r.y, r.z, r.w);
            }
        }
    } else {
        // a brick row's BX sites own DIM * BX consecutive links, which span
        // RB - 1 or RB Philox blocks; each block is drawn once, by one thread
        // (words of sites past the lattice's edge are drawn but never read)
        constexpr int RL = DIM * B::BX, RB = RL / 4 + 1, NR = B::BY * B::BZ;
        for (int q = t; q < NR * RB; q += B::NT) {
            const int row = q / RB, jb = q % RB;
            const int ry = row % B::BY, rz = row / B::BY;
            if (y0 + ry >= L || (DIM == 3 && z0 + rz >= L)) continue;
            const uint32_t i0 = (uint32_t)x0 + uL * ((uint32_t)(y0 + ry) + uL * (uint32_t)(z0 + rz));
            const uint32_t la = (uint32_t)DIM * i0, ma = la >> 2, mb = (la + RL - 1) >> 2;
            if ((uint32_t)jb > mb - ma) continue;
            const U4 r = philox4x32_10(ma + (uint32_t)jb, klo, khi, STREAM_BOND, k0, k1);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const uint32_t l = 4u * (ma + (uint32_t)jb) + (uint32_t)w;
                if (l >= la && l < la + RL) uw[RL * row + (l - la)] = u4_word(r, w);
            }
        }
    }
    __syncthreads();
    uint8_t bits = 0;
    if (valid) {
        const uint8_t s = st[lz][ly][lx];
#pragma unroll
        for (int dir = 0; dir < DIM; ++dir) {
            const uint32_t u = uw[DIM * t + dir];   // link DIM * i + dir
            const uint8_t ns = dir == 0 ? st[lz][ly][lx + 1] : dir == 1 ? st[lz][ly + 1][lx] : st[lz + 1][ly][lx];
            const int c = dir == 0 ? gx : dir == 1 ? gy : gz;   // under open boundaries the last one links out
            if (ns == s && (uint64_t)u < thr && !(p.open && c + 1 == L)) bits |= (uint8_t)(1u << dir);
        }
        p.bond[i] = bits;
    }
    // bonds whose far end is in the brick (not across the lattice's edge)
    const bool bx = (bits & 1) && lx + 1 < B::BX && gx + 1 < L;
    const bool by = (bits & 2) && ly + 1 < B::BY && gy + 1 < L;
    int head = t;   // the site whose root is this site's root
    if constexpr (DIM == 2) {
        // A warp is one 32-site row of the brick.  The union-find runs on
        // run heads (the leftmost site of a maximal chain of x bonds), so the
        // x bonds need no unions; a down bond is a contact between the run
        // above and the run below, skipped when the down bond to its left
        // already joins the same two runs.
        __shared__ uint32_t heads_of[B::BY];
        const uint32_t hbits = __ballot_sync(0xFFFFFFFFu, bx);
        const uint32_t vbits = __ballot_sync(0xFFFFFFFFu, by);
        const uint32_t heads = run_heads(hbits);
        if (lx == 0) heads_of[ly] = heads;
        head = head_of(heads, B::BX * ly, lx);
        __syncthreads();
        const uint32_t below = ly + 1 < B::BY ? heads_of[ly + 1] : 0xFFFFFFFFu;
        const uint32_t u = vbits & (~(vbits << 1) | heads | below);
        if ((u >> lx) & 1u) sunite(par, head, head_of(below, B::BX * (ly + 1), lx));
    } else {
        // 3D: a warp holds four 8-site rows of one layer (lane = x + 8 (y mod
        // 4)).  The union-find runs on the heads of x runs inside those rows;
        // a y or z bond is a contact between the run of its site and the run
        // of the site it reaches (the next row: in the same warp or the next
        // one; the next layer: two warps on), skipped when the bond of the
        // same direction to its left joins the same two runs.
        static_assert(B::BX == 8 && B::BY == 8, "3D bricks of 8 x 8 x 8 sites");
        __shared__ uint32_t heads_of[B::NT / 32];
        const bool bz = (bits & 4) && lz + 1 < B::BZ && gz + 1 < L;
        const int lane = t & 31, warp = t >> 5;
        const uint32_t hbits = __ballot_sync(0xFFFFFFFFu, bx);
        const uint32_t ybits = __ballot_sync(0xFFFFFFFFu, by);
        const uint32_t zbits = __ballot_sync(0xFFFFFFFFu, bz);
        const uint32_t heads = run_heads(hbits);   // bit x = 0 of every row is set: no bond crosses lx = 7
        if (lane == 0) heads_of[warp] = heads;
        head = head_of(heads, 32 * warp, lane);
        __syncthreads();
        const bool left = lx > 0;   // the site to the left is in the same row
        if (by) {
            const int tw = (lane < 24) ? warp : warp + 1, tl = (lane + 8) & 31;   // the site t + 8
            const uint32_t th_ = heads_of[tw];
            const bool own_head = (heads >> lane) & 1u, tgt_head = (th_ >> tl) & 1u;
            if (!(left && ((ybits >> (lane - 1)) & 1u) && !own_head && !tgt_head))
                sunite(par, head, head_of(th_, 32 * tw, tl));
        }
        if (bz) {
            const int tw = warp + 2;   // the site t + 64, same lane
            const uint32_t th_ = heads_of[tw];
            const bool own_head = (heads >> lane) & 1u, tgt_head = (th_ >> lane) & 1u;
            if (!(left && ((zbits >> (lane - 1)) & 1u) && !own_head && !tgt_head))
                sunite(par, head, head_of(th_, 32 * tw, lane));
        }
    }
    __syncthreads();
    if (valid) {
        const int r = sroot(par, head);
        const int rx = r % B::BX, ry = (r / B::BX) % B::BY, rz = r / (B::BX * B::BY);
        p.label[i] = (int32_t)((uint32_t)(x0 + rx) + uL * ((uint32_t)(y0 + ry) + uL * (uint32_t)(z0 + rz)));
        if (p.size) atomicAdd(&cnt[r], 1);
    }
    if (p.size) {
        __syncthreads();
        if (valid) p.size[i] = par[t] == t ? cnt[t] : 0;
    }
}

// Bonds that leave their brick (Sec. I step 2 across bricks): unite the two
// ends' pieces in the global forest of labels.  One block per brick, one
// thread per site of its + faces (the brick's last valid column, row and
// layer, which also hold the lattice's wrapping links).
template <int DIM>
struct Faces {
    static constexpr int FS = DIM == 2 ? 32 : 64;   // sites of one face
    static constexpr int NT = DIM * FS;
};

template <int DIM>
__global__ void __launch_bounds__(Faces<DIM>::NT) k_potts_cross(const PottsDev p)
{
    using B = Brick<DIM>;
    constexpr int FS = Faces<DIM>::FS;
    const int L = p.L;
    const uint32_t uL = (uint32_t)L;
    const int x0 = blockIdx.x * B::BX, y0 = blockIdx.y * B::BY, z0 = blockIdx.z * B::BZ;
    const int f = threadIdx.x / FS, r = threadIdx.x % FS;   // f: the face's axis
    const int a = DIM == 2 ? r : r % 8, b = DIM == 2 ? 0 : r / 8;
    if (DIM == 2 && f == 0 && a >= B::BY) return;   // the x face is BY sites long
    int gx, gy, gz;
    if (f == 0) {
        gx = min(x0 + B::BX, L) - 1;
        gy = y0 + a;
        gz = z0 + b;
    } else if (f == 1) {
        gx = x0 + a;
        gy = min(y0 + B::BY, L) - 1;
        gz = z0 + b;
    } else {
        gx = x0 + a;
        gy = y0 + b;
        gz = min(z0 + B::BZ, L) - 1;
    }
    if (gx >= L || gy >= L || (DIM == 3 && gz >= L)) return;
    const uint32_t i = (uint32_t)gx + uL * ((uint32_t)gy + uL * (uint32_t)gz);
    if (!((p.bond[i] >> f) & 1u)) return;   // (open boundaries: no bond leaves the lattice)
    uint32_t j;
    if (f == 0)
        j = i - (uint32_t)gx + (gx + 1 == L ? 0u : (uint32_t)gx + 1u);
    else if (f == 1)
        j = gy + 1 == L ? i - (uint32_t)gy * uL : i + uL;
    else
        j = gz + 1 == L ? i - (uint32_t)gz * uL * uL : i + uL * uL;
    punite(p.label, (int)i, (int)j);
}

// The per-site passes below stride over the lattice with a bounded grid, so
// each block adds its sums to the observables once.
constexpr unsigned MAX_BLOCKS = 4096;

// Every site's label becomes its root, the cluster minimum (every write moves
// a label to an ancestor, so concurrent walks stay on their paths), and the
// site takes its cluster's new state (Sec. I step 3); cluster roots are
// counted.  A piece root that is not a cluster root hands its size to the
// cluster root.
__global__ void k_potts_resolve(const PottsDev p, uint64_t k, DevObs *obs)
{
    int roots = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.N; i += (int64_t)gridDim.x * blockDim.x) {
        const int first = gload(p.label + i);   // the piece's root, or an ancestor of it
        int x = first, nx = gload(p.label + x);
        while (nx != x) {
            x = nx;
            nx = gload(p.label + x);
        }
        // the other sites of the piece then stop one step later
        if (x != first) *(volatile int32_t *)(p.label + first) = x;
        if (p.size && x != (int)i) {
            const int s = p.size[i];
            if (s > 0) {
                atomicAdd(p.size + x, s);
                p.size[i] = 0;
            }
        }
        p.label[i] = x;
        const U4 w = philox4x32_10((uint32_t)x >> 2, (uint32_t)k, (uint32_t)(k >> 32), STREAM_QSPIN,
                                   (uint32_t)p.seed, (uint32_t)(p.seed >> 32));
        p.spin[i] = potts_state(u4_word(w, x & 3), p.q);
        roots += x == (int)i;
    }
    roots = __reduce_add_sync(0xFFFFFFFFu, roots);
    __shared__ int red[PT / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = roots;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long n = 0;
        for (int w = 0; w < PT / 32; ++w) n += red[w];
        if (n) atomicAdd(&obs->nclusters, (unsigned long long)n);
        if (blockIdx.x == 0) obs->threshold = p.thr_dev ? *p.thr_dev : p.thr;
    }
}

// Sums of the new states: bond_sum, mag, the bond count and sum |C|^2.  A
// warp takes one lattice row (L sites along x) at a time, so neighbours are
// found without dividing site indices.
__global__ void k_potts_measure(const PottsDev p, DevObs *obs)
{
    __shared__ long long red[PT / 32][4];
    long long v[4] = {0, 0, 0, 0};
    const uint32_t uL = (uint32_t)p.L;
    const uint32_t rows = (uint32_t)(p.N / p.L);   // row R = y + L z
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t R = w0; R < rows; R += nw) {
        const uint32_t y = R % uL, z = R / uL;
        const uint32_t Ry = y + 1 == uL ? R - y : R + 1;                     // row at y + 1
        const uint32_t Rz = p.dim == 3 ? (z + 1 == uL ? R - z * uL : R + uL) : 0u;   // row at z + 1
        const uint8_t *row = p.spin + (size_t)R * uL;
        const uint8_t *row_y = p.spin + (size_t)Ry * uL;
        const uint8_t *row_z = p.spin + (size_t)Rz * uL;
        for (uint32_t x = lane; x < uL; x += 32) {
            const uint8_t s = row[x];
            // each link that exists (open boundaries drop those leaving the lattice)
            if (!(p.open && x + 1 == uL)) v[0] += row[x + 1 == uL ? 0u : x + 1] == s ? 1 : -1;
            if (!(p.open && y + 1 == uL)) v[0] += row_y[x] == s ? 1 : -1;
            if (p.dim == 3 && !(p.open && z + 1 == uL)) v[0] += row_z[x] == s ? 1 : -1;
            v[1] += s == 0 ? p.q - 1 : -1;
            const size_t i = (size_t)R * uL + x;
            v[2] += __popc((uint32_t)p.bond[i]);
            if (p.size) {
                const long long c = p.size[i];
                v[3] += c * c;
            }
        }
    }
    unsigned long long *const dst[4] = {&obs->bond_sum, &obs->mag, &obs->nbonds, &obs->csize2};
    block_sum_atomic<PT, 4>(v, dst, red);
}

// ------------------------------------------------------------- Potts PCC
// The extension rule in d dimensions (Sec. III): a cluster spans axis a iff it
// occupies all L hyperplanes perpendicular to a.  Such a cluster holds a site
// of the hyperplane a = 0, so the roots found there are the candidates; every
// site then marks its coordinate along a in its root's coverage (when the root
// is a candidate), and a candidate spans iff its coverage is full.  Labels are
// cluster roots by now (k_potts_resolve).

// Coordinate of site i along axis a, and the site of face a = 0 with index f
// (the other coordinates in order).
__device__ __forceinline__ uint32_t coord_of(uint32_t i, uint32_t L, int a)
{
    return a == 0 ? i % L : a == 1 ? (i / L) % L : i / (L * L);
}
__device__ __forceinline__ uint32_t face_site(uint32_t f, uint32_t L, int a)
{
    const uint32_t u = f % L, v = f / L;   // v = 0 in 2D
    return a == 0 ? L * u + L * L * v : a == 1 ? u + L * L * v : u + L * v;
}

// Step 1: candidate ids for the roots on each axis's face a = 0.
__global__ void k_potts_pcc_cand(const PottsDev p, int64_t F)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= F * p.dim) return;
    const int a = (int)(q / F);
    const uint32_t f = (uint32_t)(q % F);
    const int32_t r = p.label[face_site(f, (uint32_t)p.L, a)];
    int32_t *c = p.cid + (size_t)a * p.N + r;
    if (atomicCAS(c, 0, 1) == 0) {
        const int id = atomicAdd(p.ncand + a, 1);   // < F: at most one per face site
        p.cand[(size_t)a * F + id] = r;
        *(volatile int32_t *)c = id + 2;
    }
}

// Step 2: every site marks its coordinates in its root's coverage, for each
// axis whose candidate the root is.  A warp of 32 consecutive sites of one row
// (L a multiple of 32) shares its y and z and one word of x: one atomic per
// root and axis.
__global__ void k_potts_pcc_cover(const PottsDev p, int64_t F)
{
    const uint32_t L = (uint32_t)p.L, W = (L + 31) / 32;
    const bool rows = (L & 31u) == 0;
    const int lane = threadIdx.x & 31;
    for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; i0 < p.N;
         i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + lane;
        const bool ok = i < p.N;
        const int32_t r = ok ? p.label[i] : -1;
        for (int a = 0; a < p.dim; ++a) {
            const int32_t c = ok ? p.cid[(size_t)a * p.N + r] : 0;
            const uint32_t x = ok ? coord_of((uint32_t)i, L, a) : 0u;
            uint32_t *cov = p.cov + (size_t)a * F * W;
            if (rows) {
                const unsigned grp = __match_any_sync(0xFFFFFFFFu, c);
                if (c >= 2 && lane == __ffs(grp) - 1) {
                    // the group's bits: x along the row (lane = x mod 32), else one coordinate
                    const uint32_t bits = a == 0 ? grp : 1u << (x & 31);
                    atomicOr(cov + (size_t)(c - 2) * W + (x >> 5), bits);
                }
            } else if (c >= 2) {
                atomicOr(cov + (size_t)(c - 2) * W + (x >> 5), 1u << (x & 31));
            }
        }
    }
}

// Step 3 (PCC_DECIDE blocks): each block checks a contiguous range of every
// axis's candidates, clears their scratch and ORs its flags into the sweep's
// spans_x (axis x) / spans_y (axis y, and z in 3D); the last block to finish
// (a counter, after a fence: no block waits) applies the feedback to the
// threshold -- down by delta_k if some cluster spans, up otherwise, clamped
// to [0, 2^32] -- and resets the counts.
constexpr int POTTS_PCC_DECIDE = 16;
__global__ void k_potts_pcc_decide(const PottsDev p, int64_t F, uint64_t k, DevObs *obs)
{
    const uint32_t L = (uint32_t)p.L, W = (L + 31) / 32;
    int sx = 0, sy = 0;
    for (int a = 0; a < p.dim; ++a) {
        const int n = p.ncand[a];
        const int chunk = (n + gridDim.x - 1) / gridDim.x;
        const int c0 = blockIdx.x * chunk, c1 = min(n, c0 + chunk);
        uint32_t *cov = p.cov + (size_t)a * F * W;
        int s = 0;
        for (int id = c0 + threadIdx.x; id < c1; id += blockDim.x) {
            bool full = true;
            for (uint32_t w = 0; w < W && full; ++w) {
                const uint32_t m = w + 1 < W || (L & 31u) == 0 ? 0xFFFFFFFFu : (1u << (L & 31u)) - 1u;
                full = (cov[(size_t)id * W + w] & m) == m;
            }
            s |= full;
            p.cid[(size_t)a * p.N + p.cand[(size_t)a * F + id]] = 0;
        }
        s = __syncthreads_or(s);   // also: every check of this range has read its coverage
        for (int64_t q = (int64_t)c0 * W + threadIdx.x; q < (int64_t)c1 * W; q += blockDim.x) cov[q] = 0u;
        if (a == 0) sx |= s; else sy |= s;
    }
    if (threadIdx.x != 0) return;
    if (sx) atomicOr(&obs->spans_x, 1);
    if (sy) atomicOr(&obs->spans_y, 1);
    __threadfence();
    if (atomicAdd(p.ncand + 3, 1) != (int)gridDim.x - 1) return;
    __threadfence();   // the last block: every other block's flags are visible
    const int fx = *(volatile int32_t *)&obs->spans_x, fy = *(volatile int32_t *)&obs->spans_y;
    const uint64_t e = 8 + k / 1000;
    const uint64_t delta = (uint64_t)1 << (32 - (e < 20 ? e : 20));
    const uint64_t top = (uint64_t)1 << 32;
    const uint64_t t = *p.thr_dev;
    *p.thr_dev = (fx || fy) ? (t > delta ? t - delta : 0) : (t + delta < top ? t + delta : top);
    for (int a = 0; a < 4; ++a) p.ncand[a] = 0;
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
    // one block per brick (2D: L <= 2^15, so at most 1024 bricks along an
    // axis; 3D: L <= 2^10, at most 128)
    if (p.dim == 2) {
        using B = Brick<2>;
        const dim3 g((unsigned)((p.L + B::BX - 1) / B::BX), (unsigned)((p.L + B::BY - 1) / B::BY), 1u);
        k_potts_local<2><<<g, B::NT, 0, st>>>(p, sweep);
        k_potts_cross<2><<<g, Faces<2>::NT, 0, st>>>(p);
    } else {
        using B = Brick<3>;
        const unsigned nb3 = (unsigned)((p.L + B::BX - 1) / B::BX);
        const dim3 g(nb3, nb3, nb3);
        k_potts_local<3><<<g, B::NT, 0, st>>>(p, sweep);
        k_potts_cross<3><<<g, Faces<3>::NT, 0, st>>>(p);
    }
    const unsigned ns = std::min(nb, MAX_BLOCKS);
    k_potts_resolve<<<ns, PT, 0, st>>>(p, sweep, obs);
    if (p.thr_dev) {   // PCC: the span test on the cluster roots, then the feedback
        const int64_t F = p.dim == 2 ? (int64_t)p.L : (int64_t)p.L * p.L;
        k_potts_pcc_cand<<<(unsigned)((F * p.dim + PT - 1) / PT), PT, 0, st>>>(p, F);
        k_potts_pcc_cover<<<ns, PT, 0, st>>>(p, F);
        k_potts_pcc_decide<<<POTTS_PCC_DECIDE, PT, 0, st>>>(p, F, sweep, obs);
    }
    k_potts_measure<<<ns, PT, 0, st>>>(p, obs);
    return cudaGetLastError();
}

cudaError_t potts_enqueue_check(const uint8_t *s, int64_t n, int q, int32_t *bad, cudaStream_t st)
{
    const unsigned nb = (unsigned)std::min<int64_t>((n + 4095) / 4096, 4096);
    k_potts_check<<<nb > 0 ? nb : 1, PT, 0, st>>>(s, n, q, bad);
    return cudaGetLastError();
}

}  // namespace swg
