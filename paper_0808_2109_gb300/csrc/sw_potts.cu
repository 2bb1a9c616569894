// sw_potts.cu -- the q-state Potts model on 2D and 3D lattices
// (sw_create_potts, pcc_create_potts in include/swgpu.h): the cluster update
// of Sec. I with "equal spins" read as "equal states", on the d-dimensional
// lattice the paper states its method for (Sec. II), split as the 2D Ising
// sweep of sw_device.cuh is (Sec. II.A's slaves and master inside one GPU):
//
//   k_ptile   one CTA per tile (128 x 64 sites in 2D, 32 x 16 x 16 in 3D).
//             It finishes sweep k-1 (each site's 2-byte tile-local cluster
//             code, the border clusters' new states from the merged node
//             table, the halo from the neighbours' tables, the observables)
//             and starts sweep k on those states, which stay in shared
//             memory: Philox bonds between equal states, a shared-memory
//             union-find over the bonds inside the tile, the new state of
//             every cluster that ends inside the tile, one node per site of
//             each tile face, and the site codes.
//   k_pmerge_union / k_pmerge_resolve (with k_pwind_init / k_pwind_jump under
//             the topological rule)
//             the master's step 2: a union-find over the face nodes joined by
//             the bonds that leave a tile (the wrapping links included),
//             smaller key (cluster minimum) wins; then every representative
//             node gets its cluster's root and new state.
//   k_ppcc_candidates / k_ppcc_cover / k_ppcc_decide
//             PCC (Sec. III): the extension rule per axis on the merged
//             clusters, and the feedback on the threshold.
//
// Conventions (both sides implement them; the CPU oracle is the reference):
//   - N = L^d sites, i = x + L*y (+ L*L*z); site i owns link dir = 0 (+x),
//     1 (+y), 2 (+z) with index l = d*i + dir; bond byte bit dir.  Under open
//     boundaries the + link of the last coordinate along an axis does not
//     exist.
//   - A link between equal states bonds iff word (l mod 4) of Philox(l/4, k,
//     BOND) < t, t = floor((1 - exp(-J/T)) 2^32).
//   - A cluster with root r (its minimum site) takes state floor(w q / 2^32),
//     w = word (r mod 4) of Philox(r/4, k, QSPIN); the hot start is the same
//     function of word (i mod 4) of Philox(i/4, 0, INIT).
//   - bond_sum = sum over links of (2 delta - 1), mag = sum over sites of
//     (q [s_i = 0] - 1).
#include "swgpu.h"
#include "sw_device.cuh"
#include "sw_internal.h"
#include "sw_launch.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <mutex>

using namespace swg;

namespace {

constexpr uint32_t STREAM_QSPIN = 3;
constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr int PT = 256;   // threads of the per-site helper kernels

__device__ __forceinline__ uint8_t potts_state(uint32_t w, int q)
{
    return (uint8_t)(((uint64_t)w * (uint32_t)q) >> 32);
}

// New state of the cluster whose root is global site r in sweep k.
__device__ __forceinline__ uint8_t cluster_state(uint32_t r, uint32_t klo, uint32_t khi, uint32_t k0, uint32_t k1,
                                                 int q)
{
    const U4 u = philox4x32_10(r >> 2, klo, khi, STREAM_QSPIN, k0, k1);
    return potts_state(u4_word(u, (int)(r & 3u)), q);
}

// ------------------------------------------------------------ tile geometry
// A tile is TX x TY (x TZ) sites; its rows (y, z) are row index r = y + TY z,
// each of TWW 32-site words.  One thread per word: NT = 256 threads.
// Face nodes: for each axis a, a "-" face (local coordinate a = 0) and a "+"
// face (the tile's last valid coordinate along a), each of Fa slots indexed
// by the site's other coordinates (axis 0: y + TY z; axis 1: x + TX z; axis
// 2: x + TX y).  Slot layout: [x-, x+, y-, y+, z-, z+].
template <int DIM>
struct PG {
    static constexpr int TX = DIM == 2 ? 128 : 32;
    static constexpr int TY = DIM == 2 ? 64 : 16;
    static constexpr int TZ = DIM == 2 ? 1 : 16;
    static constexpr int TWW = TX / 32;
    static constexpr int NR = TY * TZ;          // rows
    static constexpr int NT = NR * TWW;         // threads
    static constexpr int NW = NT / 32;          // warps
    static constexpr int NS = TX * TY * TZ;     // sites
    static constexpr int PW = TX + 1;           // forest row pitch (rows on distinct banks)
    static constexpr int RS = TX + 4;           // state row pitch in bytes (the halo column, padded)
    static constexpr int HY = TY + 1, HZ = DIM == 2 ? 1 : TZ + 1;
    static constexpr int F0 = TY * TZ, F1 = TX * TZ, F2 = DIM == 3 ? TX * TY : 0;
    static constexpr int FT = F0 + F1 + F2;     // + face sites: crossing links, and halo sites
    static constexpr int S = 2 * FT;            // node slots
    static constexpr int CW = FT / 32;          // crossing-bit words
    static constexpr int PMW = DIM == 2 ? 6 : 2;   // PCC coverage words of a piece
    static constexpr int NQ = NS / 8 / NT;      // 8-site groups per thread
    static constexpr int SPT = (S + NT - 1) / NT;  // node slots per thread
    static_assert(NT == 256 && NQ == 4, "tile launch shape");
    static_assert(F0 % 32 == 0 && F1 % 32 == 0 && F2 % 32 == 0, "faces of whole words");
    static_assert(S <= 0x7FFF, "slots fit the code");
};

template <int DIM>
__device__ __forceinline__ int face_off(int a, int side)
{
    using G = PG<DIM>;
    return (a == 0 ? 0 : a == 1 ? 2 * G::F0 : 2 * G::F0 + 2 * G::F1) +
           side * (a == 0 ? G::F0 : a == 1 ? G::F1 : G::F2);
}

// The local site of slot s (false past the tile's valid sites).
template <int DIM>
__device__ __forceinline__ bool slot_xyz(int s, const int (&e)[3], int &x, int &y, int &z)
{
    using G = PG<DIM>;
    if (s < 2 * G::F0) {
        const int side = s >= G::F0, f = s - side * G::F0;
        x = side ? e[0] - 1 : 0;
        y = f % G::TY;
        z = f / G::TY;
    } else if (s < 2 * G::F0 + 2 * G::F1) {
        const int s2 = s - 2 * G::F0, side = s2 >= G::F1, f = s2 - side * G::F1;
        y = side ? e[1] - 1 : 0;
        x = f % G::TX;
        z = f / G::TX;
    } else {
        const int s2 = s - 2 * G::F0 - 2 * G::F1, side = s2 >= G::F2, f = s2 - side * G::F2;
        z = side ? e[2] - 1 : 0;
        x = f % G::TX;
        y = f / G::TX;
    }
    return x < e[0] && y < e[1] && z < e[2];
}

// A slot on a "-" face: the halo of the neighbour on that side reads its final.
template <int DIM>
__device__ __forceinline__ bool minus_slot(int s)
{
    using G = PG<DIM>;
    return s < G::F0 || (s >= 2 * G::F0 && s < 2 * G::F0 + G::F1) ||
           (DIM == 3 && s >= 2 * G::F0 + 2 * G::F1 && s < 2 * G::F0 + 2 * G::F1 + G::F2);
}

struct PTile {
    int c[3];      // tile coordinates
    int o[3];      // origin (sites)
    int e[3];      // extent (valid sites; 1 along z in 2D)
    int nb[3];     // tile index of the + neighbour along each axis (periodic)
    uint32_t gbase;   // global index of local site (0, 0, 0)
};

template <int DIM>
__device__ __forceinline__ PTile ptile_of(const PottsDev &p, int lt)
{
    using G = PG<DIM>;
    PTile t;
    const int n[3] = {p.ntx, p.nty, p.ntz};
    const int T[3] = {G::TX, G::TY, G::TZ};
    t.c[0] = lt % p.ntx;
    t.c[1] = (lt / p.ntx) % p.nty;
    t.c[2] = lt / (p.ntx * p.nty);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        t.o[a] = t.c[a] * T[a];
        t.e[a] = a < DIM ? min(T[a], p.L - t.o[a]) : 1;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int cc[3] = {t.c[0], t.c[1], t.c[2]};
        cc[a] = (cc[a] + 1) % n[a];
        t.nb[a] = cc[0] + n[0] * (cc[1] + n[1] * cc[2]);
    }
    const uint32_t uL = (uint32_t)p.L;
    t.gbase = (uint32_t)t.o[0] + uL * ((uint32_t)t.o[1] + uL * (uint32_t)t.o[2]);
    return t;
}

// ------------------------------------------------- 3D tile union-find
// Connected components of the bonds inside a 32 x 16 x 16 tile (X: +x bonds,
// whose link leaving the tile's last column is ignored; Y, Z: +y / +z bonds,
// ignored in the tile's last row / layer).  The forest lives on run heads (a
// run = maximal chain of x bonds in a row; its head is its leftmost site):
//   1. warp w holds the rows y = 4 (w mod 4) + (lane mod 4), z = 8 (w / 4) +
//      lane / 4; lane = row unites its runs with those of the next row along
//      y and along z inside the warp, skipping a bond when the bond of the
//      same direction to its left joins the same two runs;
//   2. the y and z bonds between the warps' row blocks, one thread per link,
//      with the same skip rule.
// Links hang the larger root under the smaller, so roots are piece minima in
// local row-major order, which is global order.
__device__ void tile_label3(volatile int *par, const uint32_t (*X)[1], const uint32_t (*Y)[1],
                            const uint32_t (*Z)[1], int tw, int th, int td)
{
    using G = PG<3>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int yy = lane & 3, zz = lane >> 2;
    const int y = 4 * (warp & 3) + yy, z = 8 * (warp >> 2) + zz;
    const int r = y + G::TY * z;
    const bool ok = y < th && z < td;
    const uint32_t vx = valid_mask(0, tw - 1);
    const uint32_t heads = run_heads(ok ? X[r][0] & vx : 0u);
    const uint32_t hy = __shfl_down_sync(FULL, heads, 1);   // row (y + 1, z) when yy < 3
    const uint32_t hz = __shfl_down_sync(FULL, heads, 4);   // row (y, z + 1) when zz < 7
    const int base = r * G::PW;
    if (ok) {
#pragma unroll
        for (int x = 0; x < 32; ++x) par[base + x] = base + x;
    }
    __syncwarp();
    const uint32_t vy = (ok && yy < 3 && y + 1 < th) ? Y[r][0] : 0u;
    const uint32_t vz = (ok && zz < 7 && z + 1 < td) ? Z[r][0] : 0u;
    const uint32_t uy = vy & (~(vy << 1) | heads | hy);
    const uint32_t uz = vz & (~(vz << 1) | heads | hz);
    int pa = -1, pb = -1, pr = 0;
    for (uint32_t b = uy; b; b &= b - 1) {
        const int x = __ffs(b) - 1;
        const int ha = head_of(heads, base, x), hb = head_of(hy, base + G::PW, x);
        pr = sunite_root(par, ha == pa ? pr : ha, hb == pb ? pr : hb);
        pa = ha;
        pb = hb;
    }
    pa = pb = -1;
    for (uint32_t b = uz; b; b &= b - 1) {
        const int x = __ffs(b) - 1;
        const int ha = head_of(heads, base, x), hb = head_of(hz, base + G::TY * G::PW, x);
        pr = sunite_root(par, ha == pa ? pr : ha, hb == pb ? pr : hb);
        pa = ha;
        pb = hb;
    }
    __syncthreads();
    // y bonds from rows y = 3, 7, 11 (every z), z bonds from layer z = 7 (every y)
    constexpr int NYB = 3 * G::TZ * 32, NZB = G::TY * 32;
    for (int q = threadIdx.x; q < NYB + NZB; q += G::NT) {
        int A, B, x;
        uint32_t bw;
        if (q < NYB) {
            const int bnd = q / (G::TZ * 32), rem = q % (G::TZ * 32);
            const int zq = rem >> 5, yq = 4 * bnd + 3;
            x = rem & 31;
            if (yq + 1 >= th || zq >= td) continue;
            A = yq + G::TY * zq;
            B = A + 1;
            bw = Y[A][0];
        } else {
            const int rem = q - NYB, yq = rem >> 5;
            x = rem & 31;
            if (8 >= td || yq >= th) continue;
            A = yq + G::TY * 7;
            B = A + G::TY;
            bw = Z[A][0];
        }
        if (!((bw >> x) & 1u)) continue;
        const uint32_t hA = run_heads(X[A][0] & vx), hB = run_heads(X[B][0] & vx);
        if (x > 0 && ((bw >> (x - 1)) & 1u) && !((hA >> x) & 1u) && !((hB >> x) & 1u)) continue;
        sunite(par, head_of(hA, A * G::PW, x), head_of(hB, B * G::PW, x));
    }
    __syncthreads();
}

// ------------------------------------------------------------ shared layout
// The states are dead once the bonds are drawn and the forest is not written
// before the labelling, so the two share memory: five CTAs fit an SM (48
// registers a thread), which runs the kernel 5% faster than four.
template <int DIM>
struct PSmem {
    using G = PG<DIM>;
    union {
        int par[G::NR * G::PW];             // from the labelling on: union-find forest over run heads
        struct {
            uint8_t fst[G::S];              // finish half: new states of the tile's pieces, by slot
            uint8_t st[G::HZ][G::HY][G::RS];   // states; row TY, layer TZ and column tw: + halo
            alignas(16) uint16_t code[G::NS];  // finish half: the tile's site codes
        } s;
    } f;
    uint8_t qs[G::NR][G::TX];               // each site's state drawn from the QSPIN stream
    uint32_t bx[G::NR][G::TWW];             // +x bonds (bit x of word c: site 32 c + x)
    uint32_t by[G::NR][G::TWW];             // +y bonds
    uint32_t bz[DIM == 3 ? G::NR : 1][G::TWW];   // +z bonds
    long long red[G::NW][4];                // the reduction that ends each half
    uint32_t pm[G::S][G::PMW];              // PCC: coordinates each border piece occupies
};

static_assert(sizeof(PSmem<2>::f) == sizeof(int) * PG<2>::NR * PG<2>::PW, "the finish half fits the forest's space");
static_assert(sizeof(PSmem<3>::f) == sizeof(int) * PG<3>::NR * PG<3>::PW, "the finish half fits the forest's space");

template <int DIM>
constexpr size_t ptile_smem(bool pcc)
{
    return pcc ? sizeof(PSmem<DIM>) : offsetof(PSmem<DIM>, pm);
}

// bytes 0 .. n-1 of a word (n in [0, 4])
__device__ __forceinline__ uint32_t byte_mask(int n)
{
    return n >= 4 ? 0xFFFFFFFFu : (n <= 0 ? 0u : (1u << (8 * n)) - 1u);
}

// ----------------------------------------------------------------- k_ptile
// Launch j finishes sweep j-1 (j >= 1) and starts sweep j (j < nsweeps).
// F: FEAT_* bits compiled in (0: periodic plain lattices only).
template <int DIM, int F>
__global__ void __launch_bounds__(PG<DIM>::NT, 5)
    k_ptile(const PottsDev p, int j, int nsweeps, uint64_t sweep0, DevObs *obs)
{
    using G = PG<DIM>;
    constexpr int NT = G::NT, NW = G::NW, S = G::S, TWW = G::TWW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PSmem<DIM> &sm = *reinterpret_cast<PSmem<DIM> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lt = blockIdx.x;
    if (lt >= p.ntiles) return;
    const bool fin = j >= 1, start = j < nsweeps;
    const PTile t = ptile_of<DIM>(p, lt);
    const int tw = t.e[0], th = t.e[1], td = t.e[2];
    const uint32_t uL = (uint32_t)p.L;
    const int q = p.q;
    const bool open = (F & FEAT_OPEN) && (p.flags & RF_OPEN);
    const bool open_x = open && t.c[0] == p.ntx - 1;
    const bool open_y = open && t.c[1] == p.nty - 1;
    const bool open_z = DIM == 3 && open && t.c[2] == p.ntz - 1;
    const bool csz = (F & FEAT_CSIZE) && (p.flags & RF_CSIZE);
    const bool pcc = (F & FEAT_PCC) && (p.flags & RF_PCC);
    uint16_t *code = p.code + (size_t)lt * G::NS;
    const size_t nbase = (size_t)lt * S;
    const uint32_t k0 = (uint32_t)p.seed, k1 = (uint32_t)(p.seed >> 32);
    // global index of a local site, and of a forest index
    auto gidx = [&](int x, int y, int z) { return t.gbase + (uint32_t)x + uL * ((uint32_t)y + uL * (uint32_t)z); };
    auto gfor = [&](int fi) {
        const int r = fi / G::PW;
        return gidx(fi - r * G::PW, r % G::TY, r / G::TY);
    };
    // local site of 8-site group idx (row-major order), false past the valid rows
    auto group = [&](int idx, int &x, int &y, int &z) {
        const int li = 8 * idx, r = li / G::TX;
        x = li - r * G::TX;
        y = r % G::TY;
        z = r / G::TY;
        return y < th && z < td;
    };
    // intra-tile x bonds of word (r, c): the link leaving the tile's last column is ignored
    auto ih = [&](int r, int c) { return sm.bx[r][c] & valid_mask(c, tw - 1); };

    if (fin) {
        // ---- finish sweep j-1: every site's new state
        const bool last = j == nsweeps;
        // the tile's codes, 8 sites per 16-byte asynchronous copy straight
        // into shared memory (the forest's space, free until the labelling)
        const uint4 *code4 = reinterpret_cast<const uint4 *>(code);
        uint4 *scode4 = reinterpret_cast<uint4 *>(sm.f.s.code);
#pragma unroll
        for (int qq = 0; qq < G::NQ; ++qq) {
            int x, y, z;
            const int idx = tid + qq * NT;
            if (group(idx, x, y, z)) cp_async16(scode4 + idx, code4 + idx);
        }
        {
            const uint32_t *ns4 = reinterpret_cast<const uint32_t *>(p.nstate + nbase);
            uint32_t *fs4 = reinterpret_cast<uint32_t *>(sm.f.s.fst);
            for (int w = tid; w < S / 4; w += NT) fs4[w] = ns4[w];
        }
        // the + halo: new states of the neighbours' "-" face sites (the merge
        // gives every "-" face slot its cluster's state)
        constexpr int HPT = (G::FT + NT - 1) / NT;
        uint32_t hs[HPT];
        int hnode[HPT], hpos[HPT];
#pragma unroll
        for (int qq = 0; qq < HPT; ++qq) {
            const int h = tid + qq * NT;
            hpos[qq] = -1;
            hnode[qq] = 0;
            if (h < G::F0) {
                const int y = h % G::TY, z = h / G::TY;
                if (y < th && z < td) {
                    hnode[qq] = t.nb[0] * S + face_off<DIM>(0, 0) + h;
                    hpos[qq] = (z * G::HY + y) * G::RS + tw;
                }
            } else if (h < G::F0 + G::F1) {
                const int f = h - G::F0, x = f % G::TX, z = f / G::TX;
                if (x < tw && z < td) {
                    hnode[qq] = t.nb[1] * S + face_off<DIM>(1, 0) + f;
                    hpos[qq] = (z * G::HY + th) * G::RS + x;
                }
            } else if (h < G::FT) {
                const int f = h - G::F0 - G::F1, x = f % G::TX, y = f / G::TX;
                if (x < tw && y < th) {
                    hnode[qq] = t.nb[2] * S + face_off<DIM>(2, 0) + f;
                    hpos[qq] = (td * G::HY + y) * G::RS + x;
                }
            }
            hs[qq] = hpos[qq] >= 0 ? p.nstate[hnode[qq]] : 0u;
        }
        cp_async_wait_all();
        __syncthreads();
        uint8_t *st = &sm.f.s.st[0][0][0];
#pragma unroll
        for (int qq = 0; qq < G::NQ; ++qq) {
            int x, y, z;
            const int idx = tid + qq * NT;
            if (!group(idx, x, y, z)) continue;
            const uint4 cq = scode4[idx];
            const uint32_t wv[4] = {cq.x, cq.y, cq.z, cq.w};
            uint32_t lo = 0u, hi = 0u;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint32_t u = (wv[e >> 1] >> (16 * (e & 1))) & 0xFFFFu;
                const uint32_t s = (u & CODE_BORDER) ? sm.f.s.fst[u & 0x7FFFu] : (u & 0xFFu);
                if (e < 4) lo |= s << (8 * e);
                else hi |= s << (8 * (e - 4));
            }
            const int nval = min(8, tw - x);
            uint8_t *row = st + (z * G::HY + y) * G::RS + x;
            if (nval == 8) {
                reinterpret_cast<uint32_t *>(row)[0] = lo;
                reinterpret_cast<uint32_t *>(row)[1] = hi;
            } else {
                for (int e = 0; e < nval; ++e) row[e] = (uint8_t)((e < 4 ? lo >> (8 * e) : hi >> (8 * (e - 4))) & 0xFFu);
            }
            if (last) {
                const uint32_t gi0 = gidx(x, y, z);
                if (nval == 8 && (gi0 & 7u) == 0) {
                    *reinterpret_cast<uint2 *>(p.spin + gi0) = make_uint2(lo, hi);
                } else {
                    for (int e = 0; e < nval; ++e)
                        p.spin[gi0 + e] = (uint8_t)((e < 4 ? lo >> (8 * e) : hi >> (8 * (e - 4))) & 0xFFu);
                }
                // border sites' labels: their cluster's root (the interior
                // clusters' were written when the sweep started)
                for (int e = 0; e < nval; ++e) {
                    const uint32_t u = (wv[e >> 1] >> (16 * (e & 1))) & 0xFFFFu;
                    if (u & CODE_BORDER) p.label[gi0 + e] = (int32_t)(p.nfinal[nbase + (u & 0x7FFFu)] & ROOT_MASK);
                }
            }
        }
#pragma unroll
        for (int qq = 0; qq < HPT; ++qq) {
            if (hpos[qq] >= 0) st[hpos[qq]] = (uint8_t)hs[qq];
        }
        __syncthreads();
        // observables of sweep j-1: every link that exists, every site
        long long bs = 0, mag = 0;
        for (int w = tid; w < G::NR * TWW; w += NT) {
            const int r = w / TWW, c = w % TWW;
            const int y = r % G::TY, z = r / G::TY;
            if (y >= th || z >= td) continue;
            const uint8_t *row = st + (z * G::HY + y) * G::RS;
            const uint8_t *rowy = row + G::RS;
            const uint8_t *rowz = row + G::HY * G::RS;
            const bool dy = !(open_y && y == th - 1), dz = DIM == 3 && !(open_z && z == td - 1);
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int x = 32 * c + 4 * m;
                const int nv = min(4, tw - x);
                if (nv <= 0) break;
                const uint32_t cur = *reinterpret_cast<const uint32_t *>(row + x);
                const uint32_t nxt = *reinterpret_cast<const uint32_t *>(row + x + 4);
                const uint32_t right = __funnelshift_r(cur, nxt, 8);
                const uint32_t vm = byte_mask(nv);
                const int nr = min(4, tw - x - (open_x ? 1 : 0));
                bs += 2 * (__popc(__vcmpeq4(cur, right) & byte_mask(nr)) >> 3) - max(nr, 0);
                if (dy) {
                    const uint32_t down = *reinterpret_cast<const uint32_t *>(rowy + x);
                    bs += 2 * (__popc(__vcmpeq4(cur, down) & vm) >> 3) - nv;
                }
                if (dz) {
                    const uint32_t back = *reinterpret_cast<const uint32_t *>(rowz + x);
                    bs += 2 * (__popc(__vcmpeq4(cur, back) & vm) >> 3) - nv;
                }
                mag += (long long)q * (__popc(__vcmpeq4(cur, 0u) & vm) >> 3) - nv;
            }
        }
        // clusters that touch a tile face: their sizes were summed at their
        // root nodes by the merge; each root node is in exactly one tile
        long long c2 = 0;
        if (csz)
            for (int s = tid; s < S; s += NT) {
                const long long c = p.csize[nbase + s];
                c2 += c * c;
            }
        long long v[4] = {bs, mag, c2, 0};
        DevObs *o = obs + (j - 1);
        unsigned long long *const dst[4] = {&o->bond_sum, &o->mag, &o->csize2, nullptr};
        block_sum_atomic<NT, 4>(v, dst, sm.red);
        __syncthreads();
    }

    if (!start) return;

    // ---- start sweep j
    const uint64_t k = sweep0 + (uint64_t)j;
    const uint64_t thr = p.thr_dev ? *p.thr_dev : p.thr;
    const uint32_t klo = (uint32_t)k, khi = (uint32_t)(k >> 32);
    if (!fin) {
        // first sweep of the call: states and + halos from global memory
        const int hrows = (th + 1) * (DIM == 3 ? td + 1 : 1);
        for (int rw = warp; rw < hrows; rw += NW) {
            const int hy = rw % (th + 1), hz = rw / (th + 1);
            const uint32_t gy = (uint32_t)((t.o[1] + hy) % p.L), gz = DIM == 3 ? (uint32_t)((t.o[2] + hz) % p.L) : 0u;
            const uint8_t *grow = p.spin + (size_t)uL * (gy + (size_t)uL * gz);
            for (int x = lane; x <= tw; x += 32) {
                int gx = t.o[0] + x;
                if (gx >= p.L) gx -= p.L;
                sm.f.s.st[hz][hy][x] = grow[gx];
            }
        }
        __syncthreads();
    }
    if (pcc)
        for (int w = tid; w < S * G::PMW; w += NT) (&sm.pm[0][0])[w] = 0u;
    if (lt == 0 && tid == 0) {
        obs[j].threshold = thr;
        obs[j].spans_x = 0;
        obs[j].spans_y = 0;
    }

    // Step 1 (Sec. I): bonds between equal states.
    const bool any_bond = thr != 0;
    const uint32_t tm1 = (uint32_t)(thr - 1);
    // every row starts a QSPIN block (4 divides L): the bond draws also fill qs
    const bool qsm = any_bond && (uL & 3u) == 0;
    // row (y, z) from its random bond bits (rx, ry, rz: bit x of word c set
    // iff the link's Philox word is below the threshold)
    auto store_row = [&](int y, int z, const uint32_t (&rx)[TWW], const uint32_t (&ry)[TWW],
                         const uint32_t (&rz)[TWW]) {
        const int r = y + G::TY * z;
        const bool dy = !(open_y && y == th - 1), dz = !(open_z && z == td - 1);
#pragma unroll
        for (int c = 0; c < TWW; ++c) {
            const int x = 32 * c + lane;
            const uint8_t s = sm.f.s.st[z][y][x];
            const uint32_t ex = __ballot_sync(FULL, s == sm.f.s.st[z][y][x + 1]);
            const uint32_t ey = __ballot_sync(FULL, s == sm.f.s.st[z][y + 1][x]);
            uint32_t ez = 0u;
            if (DIM == 3) ez = __ballot_sync(FULL, s == sm.f.s.st[DIM == 3 ? z + 1 : z][y][x]);
            const uint32_t vm = valid_mask(c, tw);
            const uint32_t vr = open_x ? valid_mask(c, tw - 1) : vm;
            if (lane == c) {
                sm.bx[r][c] = rx[c] & ex & vr;
                sm.by[r][c] = dy ? ry[c] & ey & vm : 0u;
                if (DIM == 3) sm.bz[DIM == 3 ? r : 0][c] = dz ? rz[c] & ez & vm : 0u;
            }
        }
    };
    if constexpr (DIM == 2) {
        // link l = 2i + d: sites 2m and 2m + 1 share Philox block m
        // aligned row: lane l drew the blocks of sites (2l, 2l+1) (r0) and
        // (64+2l, 65+2l) (r1); lane x of each 32-site word takes its two bits
        // by shuffle
        auto draws_aligned = [&](const U4 &r0, const U4 &r1, uint32_t (&rh)[TWW], uint32_t (&rv)[TWW]) {
            const uint32_t nib0 = (below(r0.x, tm1) ? 1u : 0u) | (below(r0.y, tm1) ? 2u : 0u) |
                                  (below(r0.z, tm1) ? 4u : 0u) | (below(r0.w, tm1) ? 8u : 0u);
            const uint32_t nib1 = (below(r1.x, tm1) ? 1u : 0u) | (below(r1.y, tm1) ? 2u : 0u) |
                                  (below(r1.z, tm1) ? 4u : 0u) | (below(r1.w, tm1) ? 8u : 0u);
#pragma unroll
            for (int c = 0; c < TWW; ++c) {
                const uint32_t n = __shfl_sync(FULL, c < 2 ? nib0 : nib1, 16 * (c & 1) + (lane >> 1)) >>
                                   (2 * (lane & 1));
                rh[c] = __ballot_sync(FULL, n & 1u);
                rv[c] = __ballot_sync(FULL, n & 2u);
            }
        };
        uint32_t rz[TWW] = {};
        if (any_bond && (uL & 1u) == 0) {
            for (int y = warp; y < th; y += 2 * NW) {
                const int y2 = y + NW;
                const uint32_t b0 = ((t.gbase + (uint32_t)y * uL) >> 1) + lane;
                const uint32_t b2 = ((t.gbase + (uint32_t)y2 * uL) >> 1) + lane;
                const U4 r0 = philox4x32_10(b0, klo, khi, STREAM_BOND, k0, k1);
                const U4 r1 = philox4x32_10(b0 + 32, klo, khi, STREAM_BOND, k0, k1);
                const U4 r2 = philox4x32_10(b2, klo, khi, STREAM_BOND, k0, k1);
                const U4 r3 = philox4x32_10(b2 + 32, klo, khi, STREAM_BOND, k0, k1);
                if (qsm) {
                    // lane l: the QSPIN block of sites 4l .. 4l + 3 of each row
                    const U4 s0 = philox4x32_10(((t.gbase + (uint32_t)y * uL) >> 2) + lane, klo, khi, STREAM_QSPIN, k0, k1);
                    const U4 s2 = philox4x32_10(((t.gbase + (uint32_t)y2 * uL) >> 2) + lane, klo, khi, STREAM_QSPIN, k0, k1);
                    *reinterpret_cast<uint32_t *>(&sm.qs[y][4 * lane]) =
                        (uint32_t)potts_state(s0.x, q) | ((uint32_t)potts_state(s0.y, q) << 8) |
                        ((uint32_t)potts_state(s0.z, q) << 16) | ((uint32_t)potts_state(s0.w, q) << 24);
                    if (y2 < th)
                        *reinterpret_cast<uint32_t *>(&sm.qs[y2][4 * lane]) =
                            (uint32_t)potts_state(s2.x, q) | ((uint32_t)potts_state(s2.y, q) << 8) |
                            ((uint32_t)potts_state(s2.z, q) << 16) | ((uint32_t)potts_state(s2.w, q) << 24);
                }
                uint32_t rh[TWW], rv[TWW], rh2[TWW], rv2[TWW];
                draws_aligned(r0, r1, rh, rv);
                draws_aligned(r2, r3, rh2, rv2);
                store_row(y, 0, rh, rv, rz);
                if (y2 < th) store_row(y2, 0, rh2, rv2, rz);
            }
        } else {
            for (int y = warp; y < th; y += NW) {
                const uint32_t G0 = t.gbase + (uint32_t)y * uL;
                uint32_t rh[TWW], rv[TWW];
#pragma unroll
                for (int c = 0; c < TWW; ++c) {
                    rh[c] = rv[c] = 0u;
                    if (any_bond) {
                        // odd L: a row may start on an odd site; every site draws its block
                        const uint32_t gi = G0 + 32 * c + lane;
                        const U4 r = philox4x32_10(gi >> 1, klo, khi, STREAM_BOND, k0, k1);
                        const bool odd = gi & 1u;
                        rh[c] = __ballot_sync(FULL, below(odd ? r.z : r.x, tm1));
                        rv[c] = __ballot_sync(FULL, below(odd ? r.w : r.y, tm1));
                    }
                }
                store_row(y, 0, rh, rv, rz);
            }
        }
    } else {
        // link l = 3i + d.  When 4 divides L every row starts on a multiple
        // of 4, so its 96 links are exactly the 24 Philox blocks from 3 i0 / 4:
        // lane b < 24 draws block b, and lane x takes bits 3x + d of the row's
        // link string from four ballots (one per word of a block)
        const int nrows = th * td;
        auto bits_of = [&](const uint32_t (&B)[4], int l) { return (B[l & 3] >> (l >> 2)) & 1u; };
        auto row_aligned = [&](const U4 &u, int r, uint32_t (&rx)[1], uint32_t (&ry)[1], uint32_t (&rz)[1]) {
            const bool act = lane < 24;
            if (!act && r >= 0)   // lanes 24..31 drew the row's QSPIN blocks: four sites' states each
                *reinterpret_cast<uint32_t *>(&sm.qs[r][4 * (lane - 24)]) =
                    (uint32_t)potts_state(u.x, q) | ((uint32_t)potts_state(u.y, q) << 8) |
                    ((uint32_t)potts_state(u.z, q) << 16) | ((uint32_t)potts_state(u.w, q) << 24);
            uint32_t B[4];
            B[0] = __ballot_sync(FULL, act && below(u.x, tm1));
            B[1] = __ballot_sync(FULL, act && below(u.y, tm1));
            B[2] = __ballot_sync(FULL, act && below(u.z, tm1));
            B[3] = __ballot_sync(FULL, act && below(u.w, tm1));
            const int l = 3 * lane;
            rx[0] = __ballot_sync(FULL, bits_of(B, l));
            ry[0] = __ballot_sync(FULL, bits_of(B, l + 1));
            rz[0] = __ballot_sync(FULL, bits_of(B, l + 2));
        };
        if (any_bond && (uL & 3u) == 0) {
            for (int rw = warp; rw < nrows; rw += 2 * NW) {
                const int rw2 = rw + NW;
                const int y = rw % th, z = rw / th, y2 = rw2 % th, z2 = rw2 / th;
                // lane b < 24: BOND block b of the row; lane 24 + b: QSPIN block b
                const uint32_t i0 = gidx(0, y, z), i2 = gidx(0, y2, z2);
                const bool bl = lane < 24;
                const uint32_t st_ = bl ? STREAM_BOND : STREAM_QSPIN;
                const uint32_t c0 = bl ? 3u * (i0 >> 2) + (uint32_t)lane : (i0 >> 2) + (uint32_t)(lane - 24);
                const uint32_t c2 = bl ? 3u * (i2 >> 2) + (uint32_t)lane : (i2 >> 2) + (uint32_t)(lane - 24);
                const U4 u0 = philox4x32_10(c0, klo, khi, st_, k0, k1);
                const U4 u2 = philox4x32_10(c2, klo, khi, st_, k0, k1);
                uint32_t rx[1], ry[1], rz[1], rx2[1], ry2[1], rz2[1];
                row_aligned(u0, y + G::TY * z, rx, ry, rz);
                row_aligned(u2, rw2 < nrows ? y2 + G::TY * z2 : -1, rx2, ry2, rz2);
                store_row(y, z, rx, ry, rz);
                if (rw2 < nrows) store_row(y2, z2, rx2, ry2, rz2);
            }
        } else {
            for (int rw = warp; rw < nrows; rw += NW) {
                const int y = rw % th, z = rw / th;
                uint32_t rx[1] = {0u}, ry[1] = {0u}, rz[1] = {0u};
                if (any_bond) {
                    // each site's three links span one or two blocks
                    const uint32_t l0 = 3u * gidx(lane, y, z);
                    const uint32_t m0 = l0 >> 2, m1 = (l0 + 2u) >> 2;
                    const U4 u0 = philox4x32_10(m0, klo, khi, STREAM_BOND, k0, k1);
                    U4 u1 = u0;
                    if (m1 != m0) u1 = philox4x32_10(m1, klo, khi, STREAM_BOND, k0, k1);
                    bool bit[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const uint32_t l = l0 + (uint32_t)d;
                        bit[d] = below(u4_word((l >> 2) == m0 ? u0 : u1, (int)(l & 3u)), tm1);
                    }
                    rx[0] = __ballot_sync(FULL, bit[0]);
                    ry[0] = __ballot_sync(FULL, bit[1]);
                    rz[0] = __ballot_sync(FULL, bit[2]);
                }
                store_row(y, z, rx, ry, rz);
            }
        }
    }
    __syncthreads();

    long long nb = 0;
    for (int w = tid; w < G::NR * TWW; w += NT) {
        const int r = w / TWW, c = w % TWW;
        const int y = r % G::TY, z = r / G::TY;
        if (y >= th || z >= td) continue;
        nb += __popc(sm.bx[r][c]) + __popc(sm.by[r][c]) + (DIM == 3 ? __popc(sm.bz[DIM == 3 ? r : 0][c]) : 0);
    }
    // crossing bonds, bit f of face a at word (f / 32) of that face's block:
    // x face f = r (the row), y face f = x + TX z, z face f = x + TX y
    {
        uint32_t *cross = p.cross + (size_t)lt * G::CW;
        for (int qq = warp; qq < G::F0 / 32; qq += NW) {
            const int r = 32 * qq + lane, y = r % G::TY, z = r / G::TY;
            const int bit = (y < th && z < td) ? (sm.bx[r][(tw - 1) >> 5] >> ((tw - 1) & 31)) & 1 : 0;
            const uint32_t word = __ballot_sync(FULL, bit);
            if (lane == 0) cross[qq] = word;
        }
        for (int w = tid; w < G::F1 / 32; w += NT) {
            const int c = w % TWW, z = w / TWW;
            cross[G::F0 / 32 + w] = z < td ? sm.by[(th - 1) + G::TY * z][c] : 0u;
        }
        if (DIM == 3)
            for (int w = tid; w < G::F2 / 32; w += NT) {
                const int c = w % TWW, y = w / TWW;
                cross[(G::F0 + G::F1) / 32 + w] = y < th ? sm.bz[DIM == 3 ? y + G::TY * (td - 1) : 0][c] : 0u;
            }
    }
    const bool last_start = j == nsweeps - 1;
    if (last_start) {
        // the last sweep of the call keeps its bond bytes
        for (int rw = warp; rw < th * td; rw += NW) {
            const int y = rw % th, z = rw / th, r = y + G::TY * z;
            const uint32_t g0 = gidx(0, y, z);
#pragma unroll
            for (int c = 0; c < TWW; ++c) {
                const int x = 32 * c + lane;
                if (x >= tw) break;
                uint32_t b = ((sm.bx[r][c] >> lane) & 1u) | (((sm.by[r][c] >> lane) & 1u) << 1);
                if (DIM == 3) b |= ((sm.bz[DIM == 3 ? r : 0][c] >> lane) & 1u) << 2;
                p.bond[g0 + (uint32_t)x] = (uint8_t)b;
            }
        }
    }

    // Step 2 inside the tile
    if constexpr (DIM == 2)
        tile_label<64>(sm.f.par, sm.bx, sm.by, th, tw);
    else
        tile_label3(sm.f.par, sm.bx, sm.by, sm.bz, tw, th, td);

    // One node per face site: key = global index of the piece's local root,
    // parent = the piece's first face slot (the representative).
    int rs[G::SPT];
#pragma unroll
    for (int qq = 0; qq < G::SPT; ++qq) {
        const int s = tid + qq * NT;
        int x, y, z;
        rs[qq] = -1;
        if (s < S && slot_xyz<DIM>(s, t.e, x, y, z)) {
            const int r = y + G::TY * z, c = x >> 5;
            rs[qq] = sroot(sm.f.par, head_of(run_heads(ih(r, c)), r * G::PW + 32 * c, x & 31));
        }
    }
    __syncthreads();
#pragma unroll
    for (int qq = 0; qq < G::SPT; ++qq)
        if (rs[qq] >= 0) atomicMin((int *)&sm.f.par[rs[qq]], (int)(INFO_BORDER | (uint32_t)(tid + qq * NT)));
    __syncthreads();
#pragma unroll
    for (int qq = 0; qq < G::SPT; ++qq) {
        const int s = tid + qq * NT;
        if (s >= S) break;
        const size_t node = nbase + s;
        if (rs[qq] >= 0) {
            const int rep = sm.f.par[rs[qq]] & 0x7FFF;
            p.npar[node] = (int32_t)(nbase + rep);
            p.nkey[node] = (int32_t)(gfor(rs[qq]) | (rep == s ? KEY_REP : 0u));
        } else {
            p.npar[node] = (int32_t)node;
            p.nkey[node] = (int32_t)KEY_NONE;
        }
        if (csz) p.csize[node] = 0;   // the merge adds piece sizes at root nodes
    }
    // Every run head learns its root; every interior root gets its record:
    // its cluster's new state (Sec. I step 3, drawn here), and is counted.
    // A walk stops at a root, a border record or an interior record; each
    // thread writes only its own heads, so concurrent walks see ancestors.
    long long ncl_interior = 0;
    const int nrows = th * td;
    for (int w = tid; w < nrows * TWW; w += NT) {
        const int rr = w % nrows, c = w / nrows;   // a warp covers consecutive rows
        const int y = rr % th, z = rr / th, r = y + G::TY * z;
        const int base = r * G::PW + 32 * c;
        for (uint32_t bits = run_heads(ih(r, c)); bits; bits &= bits - 1) {
            const int hx = __ffs(bits) - 1;
            const int hd = base + hx;
            int x = hd, pp = sm.f.par[x];
            while (pp != x && pp >= 0 && (uint32_t)pp < INFO_INTERIOR) {
                x = pp;
                pp = sm.f.par[x];
            }
            if (x != hd) {
                sm.f.par[hd] = x;
            } else if (pp == hd && 32 * c + hx < tw) {
                const uint8_t s = qsm ? sm.qs[r][32 * c + hx] : cluster_state(gidx(32 * c + hx, y, z), klo, khi, k0, k1, q);
                sm.f.par[hd] = (int)(INFO_INTERIOR | (uint32_t)s);
                ++ncl_interior;
            }
        }
    }
    __syncthreads();
    if (csz) {
        // cluster sizes: every run adds its length to bits 16-30 of its root's
        // record (a piece or cluster holds at most 8192 sites); the codes
        // below read bits 0-15 only
        for (int w = tid; w < nrows * TWW; w += NT) {
            const int rr = w % nrows, c = w / nrows;
            const int y = rr % th, z = rr / th, r = y + G::TY * z;
            const int base = r * G::PW + 32 * c;
            const int vw = min(32, tw - 32 * c);
            for (uint32_t bits = run_heads(ih(r, c)); bits;) {
                const int hx = __ffs(bits) - 1;
                bits &= bits - 1;
                if (hx >= vw) break;
                const int nx = bits ? __ffs(bits) - 1 : 32;
                const int v = sm.f.par[base + hx];
                const int root = (v < 0 || (uint32_t)v >= INFO_INTERIOR) ? base + hx : v;
                atomicAdd((int *)&sm.f.par[root], (min(nx, vw) - hx) << 16);
            }
        }
        __syncthreads();
    }
    // Every site's 2-byte code (the low half of its root's record): border
    // pieces by representative slot, interior clusters by new state.
    uint4 *code4 = reinterpret_cast<uint4 *>(code);
#pragma unroll
    for (int qq = 0; qq < G::NQ; ++qq) {
        int xb, y, z;
        const int idx = tid + qq * NT;
        if (!group(idx, xb, y, z)) continue;
        const int r = y + G::TY * z, c = xb >> 5;
        const uint32_t heads = run_heads(ih(r, c));
        const int base = r * G::PW + 32 * c;
        const uint32_t gi0 = gidx(xb, y, z);
        uint32_t wv[4] = {0u, 0u, 0u, 0u};
        int slot = -1;   // PCC: border piece of the sites gathered in cols
        uint32_t cols = 0u;
        int info = 0, root = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int x = xb + e;
            if (x >= tw) break;
            if (e == 0 || ((heads >> (x & 31)) & 1u)) {
                const int hd = e == 0 ? head_of(heads, base, x & 31) : base + (x & 31);
                const int v = sm.f.par[hd];
                if ((uint32_t)v >= INFO_INTERIOR) {   // records: negative or >= INFO_INTERIOR
                    info = v;
                    root = hd;
                } else {
                    info = sm.f.par[v];
                    root = v;
                }
            }
            wv[e >> 1] |= ((uint32_t)info & 0xFFFFu) << (16 * (e & 1));
            if (last_start && info >= 0) p.label[gi0 + e] = (int32_t)gfor(root);
            if (pcc && info < 0) {
                const int sl = info & 0x7FFF;
                if (sl != slot) {
                    if (slot >= 0) {
                        if (DIM == 2) {
                            atomicOr(&sm.pm[slot][c], cols);
                            atomicOr(&sm.pm[slot][4 + (y >> 5)], 1u << (y & 31));
                        } else {
                            atomicOr(&sm.pm[slot][0], cols);
                            atomicOr(&sm.pm[slot][1], (1u << y) | (1u << (16 + z)));
                        }
                    }
                    slot = sl;
                    cols = 0u;
                }
                cols |= 1u << (x & 31);
            }
        }
        if (slot >= 0) {
            if (DIM == 2) {
                atomicOr(&sm.pm[slot][c], cols);
                atomicOr(&sm.pm[slot][4 + (y >> 5)], 1u << (y & 31));
            } else {
                atomicOr(&sm.pm[slot][0], cols);
                atomicOr(&sm.pm[slot][1], (1u << y) | (1u << (16 + z)));
            }
        }
        code4[idx] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
    }
    if (pcc) {
        __syncthreads();
        for (int w = tid; w < S * G::PMW; w += NT) p.pmask[nbase * G::PMW + w] = (&sm.pm[0][0])[w];
    }
    long long c2 = 0;
    if (csz) {
        // every root: an interior cluster adds its |C|^2; a border piece hands
        // its size to its representative node for the merge
        for (int w = tid; w < nrows * TWW; w += NT) {
            const int rr = w % nrows, c = w / nrows;
            const int y = rr % th, z = rr / th, r = y + G::TY * z;
            const int base = r * G::PW + 32 * c;
            const int vw = min(32, tw - 32 * c);
            for (uint32_t bits = run_heads(ih(r, c)) & valid_mask(0, vw); bits; bits &= bits - 1) {
                const int v = sm.f.par[base + __ffs(bits) - 1];
                if (v < 0) {   // piece size: bits 16-30 (bit 31 is the border flag)
                    p.psize[nbase + (v & 0x7FFF)] = (int32_t)(((uint32_t)v >> 16) & 0x7FFFu);
                } else if ((uint32_t)v >= INFO_INTERIOR) {   // bits 16-29 (bit 30 is the flag)
                    const long long size = ((uint32_t)v >> 16) & 0x3FFFu;
                    c2 += size * size;
                }
            }
        }
    }
    long long v4[4] = {nb, ncl_interior, c2, 0};
    DevObs *o = obs + j;
    unsigned long long *const dst[4] = {&o->nbonds, &o->nclusters, &o->csize2, nullptr};
    block_sum_atomic<NT, 4>(v4, dst, sm.red);
}

// ------------------------------------------------ topological rule (RF_WIND)
// A cluster percolates when it winds around the box (Sec. III): some closed
// path of its bonds has a non-zero net displacement.  Every node carries its
// parent and its unwrapped displacement from that parent, one 16-byte word
// changed by 16-byte compare-and-swap so that the four move together; a root
// links to itself with displacement 0.  The displacements are exact: a set's
// nodes lift to a connected set of at most N sites, so they stay below 2^30.
struct alignas(16) WLink {
    int32_t parent, dx, dy, dz;
};

__device__ __forceinline__ WLink wl_read(WLink *w)
{
    const WLink z{0, 0, 0, 0};
    return atomicCAS(w, z, z);   // an atomic 16-byte read (rewrites an equal word)
}

// Root of x with pos(x) - pos(root); the walk halves the path (x's link is
// moved to its grandparent with the summed displacement: a failed swap means
// another walk moved it first).
__device__ __forceinline__ int wfind3(WLink *wl, int x, int &ox, int &oy, int &oz)
{
    ox = oy = oz = 0;
    WLink w = wl_read(wl + x);
    while (w.parent != x) {
        const WLink g = wl_read(wl + w.parent);
        if (g.parent != w.parent) {
            const WLink nw{g.parent, w.dx + g.dx, w.dy + g.dy, w.dz + g.dz};
            atomicCAS(wl + x, w, nw);
            ox += nw.dx;
            oy += nw.dy;
            oz += nw.dz;
            x = g.parent;
            w = wl_read(wl + x);
        } else {
            ox += w.dx;
            oy += w.dy;
            oz += w.dz;
            x = w.parent;
            w = g;
        }
    }
    return x;
}

// The link from node a to node b steps +1 along axis ax.  Roots of the same
// set: the cycle it closes has net displacement pos(a) + e_ax - pos(b) through
// the tree, non-zero exactly when it winds (recorded per axis).  Else the root
// of larger key hangs under the other with its displacement from it.
__device__ __forceinline__ void wunite3(WLink *wl, const int32_t *key, int a, int b, int ax, DevObs *o)
{
    for (;;) {
        int oax, oay, oaz, obx, oby, obz;
        const int ra = wfind3(wl, a, oax, oay, oaz);
        const int rb = wfind3(wl, b, obx, oby, obz);
        // pos(rb) - pos(ra) = (pos(a) - off_a ... ) through the link: off_a + e_ax - off_b
        const int cx = oax + (ax == 0) - obx, cy = oay + (ax == 1) - oby, cz = oaz + (ax == 2) - obz;
        if (ra == rb) {
            if (cx) atomicOr(&o->spans_x, 1);
            if (cy || cz) atomicOr(&o->spans_y, 1);   // y, or in 3D y or z
            return;
        }
        const bool a_lo = (uint32_t)key[ra] < (uint32_t)key[rb];
        const int lo = a_lo ? ra : rb, hi = a_lo ? rb : ra;
        const WLink root{hi, 0, 0, 0};
        const WLink nl = a_lo ? WLink{lo, cx, cy, cz} : WLink{lo, -cx, -cy, -cz};
        const WLink old = atomicCAS(wl + hi, root, nl);
        if (old.parent == hi && old.dx == 0 && old.dy == 0 && old.dz == 0) return;
    }
}

// ------------------------------------------------------------------ merge
template <int DIM>
struct PMC {
    static constexpr int MT = DIM == 2 ? 96 : 512;                  // threads per block (measured best)
    static constexpr int EPT = (PG<DIM>::FT + MT - 1) / MT;        // crossing links per thread
    static constexpr int NPT = PG<DIM>::S / MT;                    // slots per thread
    static_assert(PG<DIM>::S % MT == 0, "merge launch shape");
};

// Master step 2 of Sec. II.A on the face nodes: link e of a tile joins slot
// f of its + face along axis a to slot f of the - face of the next tile
// along a (e = f, F0 + f, F0 + F1 + f for a = 0, 1, 2); union by key, the
// finds of all of a thread's links advancing in lock step.  (A per-block
// shared-memory forest that filters links joining pieces already joined, as
// the Ising merge has, made the 3D merge slower: its pieces are small and
// seldom meet twice.)
template <int DIM, bool W>
__global__ void __launch_bounds__(PMC<DIM>::MT) k_pmerge_union(const PottsDev p, int j, DevObs *obs)
{
    using G = PG<DIM>;
    using MC = PMC<DIM>;
    constexpr int S = G::S;
    const int lt = blockIdx.x;
    const PTile t = ptile_of<DIM>(p, lt);
    const uint32_t *cross = p.cross + (size_t)lt * G::CW;
    int na[MC::EPT], nb[MC::EPT], ax[MC::EPT], nt[MC::EPT];
#pragma unroll
    for (int qq = 0; qq < MC::EPT; ++qq) {
        const int e = threadIdx.x + qq * MC::MT;
        na[qq] = -1;
        ax[qq] = 0;
        nt[qq] = 0;
        if (e < G::FT && ((cross[e >> 5] >> (e & 31)) & 1u)) {
            const int a = e < G::F0 ? 0 : e < G::F0 + G::F1 ? 1 : 2;
            const int f = e - (a == 0 ? 0 : a == 1 ? G::F0 : G::F0 + G::F1);
            nt[qq] = a == 0 ? t.nb[0] : a == 1 ? t.nb[1] : t.nb[2];
            na[qq] = lt * S + face_off<DIM>(a, 1) + f;
            nb[qq] = nt[qq] * S + face_off<DIM>(a, 0) + f;
            ax[qq] = a;
        }
    }
    if (W && (p.flags & RF_WIND)) {
        WLink *wl = reinterpret_cast<WLink *>(p.wlink);
#pragma unroll
        for (int qq = 0; qq < MC::EPT; ++qq)
            if (na[qq] >= 0) wunite3(wl, p.nkey, na[qq], nb[qq], ax[qq], obs + j);
        return;
    }
    int pa[MC::EPT], pb[MC::EPT], ka[MC::EPT], kb[MC::EPT];
#pragma unroll
    for (int qq = 0; qq < MC::EPT; ++qq) {
        if (na[qq] < 0) continue;
        pa[qq] = gload(p.npar + na[qq]);
        pb[qq] = gload(p.npar + nb[qq]);
        ka[qq] = p.nkey[na[qq]];
        kb[qq] = p.nkey[nb[qq]];
    }
    bool live[MC::EPT];
#pragma unroll
    for (int qq = 0; qq < MC::EPT; ++qq) live[qq] = na[qq] >= 0;
    // First try, one compare-and-swap: hang the larger-key one of the two
    // pieces' representatives under the other.  Every parent carries a smaller
    // key than its children, so a root of key k holds no node of smaller key:
    // if that representative is still a root, the two sets differ and the
    // link joins them (its new parent need not be a root).
#pragma unroll
    for (int qq = 0; qq < MC::EPT; ++qq) {
        if (!live[qq]) continue;
        const bool ra = ((uint32_t)ka[qq] & KEY_REP) != 0u, rb = ((uint32_t)kb[qq] & KEY_REP) != 0u;
        const int u = ra ? na[qq] : pa[qq], v = rb ? nb[qq] : pb[qq];
        if (u == v) {
            live[qq] = false;
            continue;
        }
        const bool u_hi = ((uint32_t)ka[qq] & KEY_MASK) > ((uint32_t)kb[qq] & KEY_MASK);
        const int hi = u_hi ? u : v, lo = u_hi ? v : u;
        // a representative whose parent was read as another node is no root
        const bool inner = u_hi ? (ra && pa[qq] != na[qq]) : (rb && pb[qq] != nb[qq]);
        if (!inner && atomicCAS(p.npar + hi, hi, lo) == hi) live[qq] = false;
    }
    // the remaining unions in lock step (path splitting on the way up; the
    // larger key's root is hung under the smaller by compare-and-swap)
    int xa[MC::EPT], xb[MC::EPT], sa[MC::EPT], sb[MC::EPT];
#pragma unroll
    for (int qq = 0; qq < MC::EPT; ++qq) {
        xa[qq] = na[qq];
        xb[qq] = nb[qq];
        sa[qq] = sb[qq] = -1;
    }
    for (;;) {
        bool more = false;
#pragma unroll
        for (int qq = 0; qq < MC::EPT; ++qq) {
            if (!live[qq]) continue;
            const bool ra = pa[qq] == xa[qq], rb = pb[qq] == xb[qq];
            if (!ra || !rb) {
                // path splitting rewrites representatives only: a slot that
                // is not one keeps its own representative as its parent
                if (!ra) {
                    if (sa[qq] >= 0) *(volatile int32_t *)(p.npar + sa[qq]) = pa[qq];
                    sa[qq] = ((uint32_t)ka[qq] & KEY_REP) ? xa[qq] : -1;
                    xa[qq] = pa[qq];
                }
                if (!rb) {
                    if (sb[qq] >= 0) *(volatile int32_t *)(p.npar + sb[qq]) = pb[qq];
                    sb[qq] = ((uint32_t)kb[qq] & KEY_REP) ? xb[qq] : -1;
                    xb[qq] = pb[qq];
                }
                more = true;
            } else if (xa[qq] == xb[qq]) {
                live[qq] = false;
            } else {
                const bool a_lo = ka[qq] < kb[qq];
                const int lo = a_lo ? xa[qq] : xb[qq], hi = a_lo ? xb[qq] : xa[qq];
                if (atomicCAS(p.npar + hi, hi, lo) == hi) live[qq] = false;
                else more = true;
            }
        }
        if (!more) break;
#pragma unroll
        for (int qq = 0; qq < MC::EPT; ++qq) {
            if (!live[qq]) continue;
            pa[qq] = gload(p.npar + xa[qq]);
            pb[qq] = gload(p.npar + xb[qq]);
            ka[qq] = p.nkey[xa[qq]];
            kb[qq] = p.nkey[xb[qq]];
        }
    }
}

// Topological rule: every node's link before the unions -- its parent from
// the tile kernel (its piece's representative, or itself) and its
// displacement from it, both sites of one tile.
template <int DIM>
__global__ void __launch_bounds__(PMC<DIM>::MT) k_pwind_init(const PottsDev p)
{
    using G = PG<DIM>;
    using MC = PMC<DIM>;
    const int lt = blockIdx.x, base = lt * G::S;
    const PTile t = ptile_of<DIM>(p, lt);
    WLink *wl = reinterpret_cast<WLink *>(p.wlink);
#pragma unroll
    for (int qq = 0; qq < MC::NPT; ++qq) {
        const int s = threadIdx.x + qq * MC::MT, n = base + s;
        const int rep = p.npar[n];
        WLink w{n, 0, 0, 0};
        int x, y, z, xr, yr, zr;
        if ((uint32_t)p.nkey[n] != KEY_NONE && rep != n && slot_xyz<DIM>(s, t.e, x, y, z) &&
            slot_xyz<DIM>(rep - base, t.e, xr, yr, zr))
            w = WLink{rep, x - xr, y - yr, z - zr};
        wl[n] = w;
    }
}

// Topological rule: one round of pointer jumping on the representatives'
// links (the wind unions hang roots under roots, so the walks grow longer
// than on the plain path, which has no such round).
template <int DIM>
__global__ void __launch_bounds__(PMC<DIM>::MT) k_pwind_jump(const PottsDev p)
{
    using MC = PMC<DIM>;
    const int base = blockIdx.x * PG<DIM>::S;
    WLink *wl = reinterpret_cast<WLink *>(p.wlink);
#pragma unroll
    for (int qq = 0; qq < MC::NPT; ++qq) {
        const int n = base + threadIdx.x + qq * MC::MT;
        const uint32_t key = (uint32_t)p.nkey[n];
        if (key == KEY_NONE || !(key & KEY_REP)) continue;
        const WLink w = wl_read(wl + n);
        if (w.parent == n) continue;
        const WLink g = wl_read(wl + w.parent);
        if (g.parent != w.parent) atomicCAS(wl + n, w, WLink{g.parent, w.dx + g.dx, w.dy + g.dy, w.dz + g.dz});
    }
}

// Every representative walks to its root r (key: the cluster's minimum site)
// and stores the cluster's root and new state (Sec. I step 3); under PCC it
// also points every node of its walk at r.  A "-" face slot that is not a
// representative then takes its representative's state (its parent, in the
// same tile: the unions rewrite representatives only) for the neighbour's
// halo.  Counts the clusters that touch a tile face (one root node each).
template <int DIM, bool W>
__global__ void __launch_bounds__(PMC<DIM>::MT) k_pmerge_resolve(const PottsDev p, int j, uint64_t sweep0,
                                                                 DevObs *obs)
{
    using MC = PMC<DIM>;
    const int base = blockIdx.x * PG<DIM>::S;
    // under the topological rule the forest lives in the node links (their
    // first word is the parent); npar keeps each node's representative
    const bool wind = W && (p.flags & RF_WIND);
    const int32_t *wpar = reinterpret_cast<const int32_t *>(p.wlink);
    auto parent = [&](int x) { return wind ? gload(wpar + 4 * (size_t)x) : gload(p.npar + x); };
    uint32_t key[MC::NPT];
    int r[MC::NPT], pr[MC::NPT], rep[MC::NPT];
#pragma unroll
    for (int qq = 0; qq < MC::NPT; ++qq) key[qq] = (uint32_t)p.nkey[base + threadIdx.x + qq * MC::MT];
#pragma unroll
    for (int qq = 0; qq < MC::NPT; ++qq) {
        r[qq] = base + threadIdx.x + qq * MC::MT;
        rep[qq] = gload(p.npar + r[qq]);
        pr[qq] = wind ? parent(r[qq]) : rep[qq];
    }
    auto is_rep = [](uint32_t kk) { return kk != KEY_NONE && (kk & KEY_REP); };
    __shared__ uint8_t rst[PG<DIM>::S];   // the new state of each representative slot
    for (;;) {
        bool more = false;
#pragma unroll
        for (int qq = 0; qq < MC::NPT; ++qq)
            if (is_rep(key[qq]) && pr[qq] != r[qq]) {
                r[qq] = pr[qq];
                more = true;
            }
        if (!more) break;
#pragma unroll
        for (int qq = 0; qq < MC::NPT; ++qq)
            if (is_rep(key[qq])) pr[qq] = parent(r[qq]);
    }
    const uint64_t k = sweep0 + (uint64_t)j;
    const uint32_t klo = (uint32_t)k, khi = (uint32_t)(k >> 32);
    const uint32_t k0 = (uint32_t)p.seed, k1 = (uint32_t)(p.seed >> 32);
    const bool pcc = (p.flags & RF_PCC) != 0 && !wind;   // the extension rule's candidates read npar
    int nroots = 0;
#pragma unroll
    for (int qq = 0; qq < MC::NPT; ++qq) {
        const int s = threadIdx.x + qq * MC::MT, n = base + s;
        if (is_rep(key[qq])) {
            if (pcc) {
                // the PCC kernels read a representative's root from its parent
                for (int x = n; x != r[qq];) {
                    const int nx = gload(p.npar + x);
                    *(volatile int32_t *)(p.npar + x) = r[qq];
                    x = nx;
                }
            }
            nroots += r[qq] == n;
            if (p.flags & RF_CSIZE) atomicAdd(p.csize + r[qq], p.psize[n]);
            const uint32_t rkey = (uint32_t)p.nkey[r[qq]] & KEY_MASK;
            const uint8_t st = cluster_state(rkey, klo, khi, k0, k1, p.q);
            p.nstate[n] = st;
            rst[s] = st;
            p.nfinal[n] = rkey;
        }
    }
    __syncthreads();
    // a "-" face slot that is not a representative (whose parent is still its
    // own representative in this tile) takes its cluster's new state too: the
    // neighbour's halo reads it with one load
#pragma unroll
    for (int qq = 0; qq < MC::NPT; ++qq) {
        const int s = threadIdx.x + qq * MC::MT;
        if (!is_rep(key[qq]) && key[qq] != KEY_NONE && minus_slot<DIM>(s)) p.nstate[base + s] = rst[rep[qq] - base];
    }
    const int wb = threadIdx.x & ~31;
    const unsigned wm = MC::MT - wb >= 32 ? 0xFFFFFFFFu : (1u << (MC::MT - wb)) - 1u;
    nroots = __reduce_add_sync(wm, nroots);
    if ((threadIdx.x & 31) == 0 && nroots) atomicAdd(&obs[j].nclusters, (unsigned long long)nroots);
}

// ------------------------------------------------------------------- PCC
// The extension rule in d dimensions (Sec. III): a cluster spans axis a iff
// it occupies all L hyperplanes perpendicular to a.  Such a cluster holds a
// site of the hyperplane a = 0, on the - face of a tile of tile coordinate 0
// along a: those nodes' roots are the candidates (cid of the root node, per
// axis: id + 2).  Every border piece then ORs the coordinates it occupies
// along a into its candidate root's coverage (L bits), and a candidate spans
// iff its coverage is full.  Interior clusters touch no face and span nothing.
template <int DIM>
__global__ void k_ppcc_candidates(const PottsDev p, int64_t F)
{
    using G = PG<DIM>;
    constexpr int S = G::S;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)p.ntiles * G::FT) return;
    const int lt = (int)(idx / G::FT), e = (int)(idx % G::FT);
    const int a = e < G::F0 ? 0 : e < G::F0 + G::F1 ? 1 : 2;
    const int f = e - (a == 0 ? 0 : a == 1 ? G::F0 : G::F0 + G::F1);
    const PTile t = ptile_of<DIM>(p, lt);
    if (t.c[a] != 0) return;
    const int node = lt * S + face_off<DIM>(a, 0) + f;
    const uint32_t key = (uint32_t)p.nkey[node];
    if (key == KEY_NONE) return;
    int r = gload(p.npar + node);
    if (!(key & KEY_REP)) r = gload(p.npar + r);   // via a representative
    int32_t *c = p.cid + (size_t)r * DIM + a;
    if (atomicCAS(c, 0, 1) == 0) {
        const int id = atomicAdd(p.ncand + a, 1);   // < F: at most one per face site
        p.cand[(size_t)a * F + id] = r;
        *(volatile int32_t *)c = id + 2;
    }
}

template <int DIM>
__global__ void k_ppcc_cover(const PottsDev p)
{
    using G = PG<DIM>;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (int64_t)p.ntiles * G::S) return;
    const uint32_t key = (uint32_t)p.nkey[n];
    if (key == KEY_NONE || !(key & KEY_REP)) return;
    uint32_t m[G::PMW];
    uint32_t any = 0u;
#pragma unroll
    for (int w = 0; w < G::PMW; ++w) any |= (m[w] = p.pmask[(size_t)n * G::PMW + w]);
    if (!any) return;
    const int r = gload(p.npar + n);
    const PTile t = ptile_of<DIM>(p, (int)(n / G::S));
    const uint32_t W = ((uint32_t)p.L + 31u) / 32u;
    const int64_t F = DIM == 2 ? (int64_t)p.L : (int64_t)p.L * p.L;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const int c = p.cid[(size_t)r * DIM + a];
        if (c < 2) continue;
        uint32_t *cov = p.cov + ((size_t)a * F + (size_t)(c - 2)) * W + (size_t)(t.o[a] >> 5);
        if (DIM == 2) {
            if (a == 0) {
#pragma unroll
                for (int w = 0; w < 4; ++w)
                    if (m[w]) atomicOr(cov + w, m[w]);
            } else {
#pragma unroll
                for (int w = 0; w < 2; ++w)
                    if (m[4 + w]) atomicOr(cov + w, m[4 + w]);
            }
        } else {
            // 32-site x words; 16-site y and z halves at an origin that is a
            // multiple of 16
            const uint32_t bits = a == 0 ? m[0] : a == 1 ? (m[1] & 0xFFFFu) : (m[1] >> 16);
            if (bits) atomicOr(cov, a == 0 ? bits : bits << (t.o[a] & 31));
        }
    }
}

// PPCC_DECIDE blocks: each checks a contiguous range of every axis's
// candidates, clears their scratch and ORs its flags into the sweep's
// spans_x (axis x) / spans_y (axis y, and z in 3D); the last block to finish
// (a counter after a fence: no block waits) applies the feedback -- down by
// delta_k if some cluster spans, up otherwise, delta_k = 2^(32 - min(8 +
// floor(k / 1000), 20)), clamped to [0, 2^32] -- and resets the counts.
constexpr int PPCC_DECIDE = 16;
__global__ void k_ppcc_decide(const PottsDev p, int64_t F, int j, uint64_t sweep0, DevObs *obs)
{
    const uint32_t L = (uint32_t)p.L, W = (L + 31) / 32;
    DevObs *o = obs + j;
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
            p.cid[(size_t)p.cand[(size_t)a * F + id] * p.dim + a] = 0;
        }
        s = __syncthreads_or(s);   // also: every check of this range has read its coverage
        for (int64_t qq = (int64_t)c0 * W + threadIdx.x; qq < (int64_t)c1 * W; qq += blockDim.x) cov[qq] = 0u;
        if (a == 0) sx |= s;
        else sy |= s;
    }
    if (threadIdx.x != 0) return;
    if (sx) atomicOr(&o->spans_x, 1);
    if (sy) atomicOr(&o->spans_y, 1);
    __threadfence();
    if (atomicAdd(p.ncand + 3, 1) != (int)gridDim.x - 1) return;
    __threadfence();   // the last block: every other block's flags are visible
    const int fx = *(volatile int32_t *)&o->spans_x, fy = *(volatile int32_t *)&o->spans_y;
    const uint64_t k = sweep0 + (uint64_t)j;
    const uint64_t e = 8 + k / 1000;
    const uint64_t delta = (uint64_t)1 << (32 - (e < 20 ? e : 20));
    const uint64_t top = (uint64_t)1 << 32;
    const uint64_t tt = *p.thr_dev;
    *p.thr_dev = (fx || fy) ? (tt > delta ? tt - delta : 0) : (tt + delta < top ? tt + delta : top);
    for (int a = 0; a < 4; ++a) p.ncand[a] = 0;
}

// ------------------------------------------------------------ small kernels
__global__ void k_potts_hot_start(const PottsDev p)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    const U4 r = philox4x32_10((uint32_t)(i >> 2), 0u, 0u, STREAM_INIT, (uint32_t)p.seed, (uint32_t)(p.seed >> 32));
    p.spin[i] = potts_state(u4_word(r, (int)(i & 3)), p.q);
}

// Sets *bad if any of the n states is >= q.
__global__ void k_potts_check(const uint8_t *s, int64_t n, int q, int32_t *bad)
{
    int found = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        found |= s[i] >= q;
    if (__syncthreads_or(found) && threadIdx.x == 0) atomicOr(bad, 1);
}

// The tile kernels' dynamic shared-memory limit, raised once per device.
constexpr int PREP_DEVICES = 64;
cudaError_t potts_prepare()
{
    static std::mutex mu;
    static bool done[PREP_DEVICES] = {};
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= PREP_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return cudaSuccess;
    const void *fn[4] = {(const void *)k_ptile<2, 0>, (const void *)k_ptile<2, FEAT_TILE>,
                         (const void *)k_ptile<3, 0>, (const void *)k_ptile<3, FEAT_TILE>};
    const int bytes[4] = {(int)ptile_smem<2>(true), (int)ptile_smem<2>(true), (int)ptile_smem<3>(true),
                          (int)ptile_smem<3>(true)};
    for (int f = 0; f < 4 && err == cudaSuccess; ++f)
        err = cudaFuncSetAttribute(fn[f], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes[f]);
    if (err == cudaSuccess) done[dev] = true;
    return err;
}

template <int DIM>
void launch_tile(const PottsDev &p, int j, int nsweeps, uint64_t sweep0, DevObs *obs, cudaStream_t st)
{
    using G = PG<DIM>;
    const bool pcc = (p.flags & RF_PCC) != 0;
    const bool feat = (p.flags & (RF_PCC | RF_OPEN | RF_CSIZE)) != 0;
    const unsigned tiles = (unsigned)p.ntiles;
    const size_t smem = ptile_smem<DIM>(pcc);
    if (feat)
        k_ptile<DIM, FEAT_TILE><<<tiles, G::NT, smem, st>>>(p, j, nsweeps, sweep0, obs);
    else
        k_ptile<DIM, 0><<<tiles, G::NT, smem, st>>>(p, j, nsweeps, sweep0, obs);
}

template <int DIM>
void launch_merge(const PottsDev &p, int j, uint64_t sweep0, DevObs *obs, cudaStream_t st)
{
    using G = PG<DIM>;
    const bool pcc = (p.flags & RF_PCC) != 0;
    const unsigned tiles = (unsigned)p.ntiles;
    const bool wind = (p.flags & RF_WIND) != 0;
    if (wind) {
        k_pwind_init<DIM><<<tiles, PMC<DIM>::MT, 0, st>>>(p);
        k_pmerge_union<DIM, true><<<tiles, PMC<DIM>::MT, 0, st>>>(p, j, obs);
        k_pwind_jump<DIM><<<tiles, PMC<DIM>::MT, 0, st>>>(p);
        k_pmerge_resolve<DIM, true><<<tiles, PMC<DIM>::MT, 0, st>>>(p, j, sweep0, obs);
    } else {
        // no pointer-jumping round: after the unions' single-swap links the
        // walks are short, and the round cost more than it saved (3D 2.99 ->
        // 2.94 ms a sweep without it)
        k_pmerge_union<DIM, false><<<tiles, PMC<DIM>::MT, 0, st>>>(p, j, obs);
        k_pmerge_resolve<DIM, false><<<tiles, PMC<DIM>::MT, 0, st>>>(p, j, sweep0, obs);
    }
    if (pcc && wind) {
        // the flags are the windings the unions recorded: the feedback only
        const int64_t F = DIM == 2 ? (int64_t)p.L : (int64_t)p.L * p.L;
        k_ppcc_decide<<<PPCC_DECIDE, PT, 0, st>>>(p, F, j, sweep0, obs);
    } else if (pcc) {
        const int64_t F = DIM == 2 ? (int64_t)p.L : (int64_t)p.L * p.L;
        const int64_t nc = (int64_t)p.ntiles * G::FT, nn = (int64_t)p.ntiles * G::S;
        k_ppcc_candidates<DIM><<<(unsigned)((nc + PT - 1) / PT), PT, 0, st>>>(p, F);
        k_ppcc_cover<DIM><<<(unsigned)((nn + PT - 1) / PT), PT, 0, st>>>(p);
        k_ppcc_decide<<<PPCC_DECIDE, PT, 0, st>>>(p, F, j, sweep0, obs);
    }
}

}  // namespace

namespace swg {

void potts_geometry(int dim, int L, PottsGeometry *g)
{
    const int tx = dim == 2 ? PG<2>::TX : PG<3>::TX, ty = dim == 2 ? PG<2>::TY : PG<3>::TY;
    const int tz = dim == 2 ? PG<2>::TZ : PG<3>::TZ;
    g->ntx = (L + tx - 1) / tx;
    g->nty = (L + ty - 1) / ty;
    g->ntz = dim == 2 ? 1 : (L + tz - 1) / tz;
    g->ntiles = g->ntx * g->nty * g->ntz;
    g->sites_per_tile = dim == 2 ? PG<2>::NS : PG<3>::NS;
    g->slots = dim == 2 ? PG<2>::S : PG<3>::S;
    g->cross_words = dim == 2 ? PG<2>::CW : PG<3>::CW;
    g->pmask_words = dim == 2 ? PG<2>::PMW : PG<3>::PMW;
}

cudaError_t potts_enqueue_hot_start(const PottsDev &p, cudaStream_t st)
{
    cudaError_t e = potts_prepare();
    if (e != cudaSuccess) return e;
    k_potts_hot_start<<<(unsigned)((p.N + PT - 1) / PT), PT, 0, st>>>(p);
    return cudaGetLastError();
}

// Launch j of a call of nsweeps sweeps: the tile kernel (finishing sweep
// j-1, starting sweep j) ...
cudaError_t potts_enqueue_tile(const PottsDev &p, int j, int nsweeps, uint64_t sweep0, DevObs *obs, cudaStream_t st)
{
    cudaError_t e = potts_prepare();
    if (e != cudaSuccess) return e;
    if (p.dim == 2) launch_tile<2>(p, j, nsweeps, sweep0, obs, st);
    else launch_tile<3>(p, j, nsweeps, sweep0, obs, st);
    return cudaGetLastError();
}

// ... and, for j < nsweeps, the merge of sweep j.
cudaError_t potts_enqueue_merge(const PottsDev &p, int j, uint64_t sweep0, DevObs *obs, cudaStream_t st)
{
    if (p.dim == 2) launch_merge<2>(p, j, sweep0, obs, st);
    else launch_merge<3>(p, j, sweep0, obs, st);
    return cudaGetLastError();
}

// The launches of one call of nsweeps sweeps: tile kernel j = 0 .. nsweeps,
// each but the last followed by the merge of sweep j.
cudaError_t potts_enqueue_sweeps(const PottsDev &p, int nsweeps, uint64_t sweep0, DevObs *obs, cudaStream_t st)
{
    for (int j = 0; j <= nsweeps; ++j) {
        cudaError_t e = potts_enqueue_tile(p, j, nsweeps, sweep0, obs, st);
        if (e == cudaSuccess && j < nsweeps) e = potts_enqueue_merge(p, j, sweep0, obs, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t potts_enqueue_check(const uint8_t *s, int64_t n, int q, int32_t *bad, cudaStream_t st)
{
    const unsigned nb = (unsigned)std::min<int64_t>((n + 4095) / 4096, 4096);
    k_potts_check<<<nb > 0 ? nb : 1, PT, 0, st>>>(s, n, q, bad);
    return cudaGetLastError();
}

}  // namespace swg
