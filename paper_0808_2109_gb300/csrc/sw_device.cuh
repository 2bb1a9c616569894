// sw_device.cuh -- device code of the Swendsen-Wang / PCC sweep for sm_103a.
//
// One sweep (Lin & Zheng, arXiv:0808.2109, Sec. I steps 1-4) is split the way
// the paper's master-slave model splits it (Sec. II.A), but inside one GPU:
//
//   k_tile   one CTA per TH x 128 tile ("slave domain").  It finishes sweep
//            k-1 (reads each site's 2-byte tile-local cluster code, resolves
//            border clusters through the merged node table, writes the new
//            spins into shared memory, reduces the observables) and, in the
//            same launch, starts sweep k on those spins: Philox bonds, a
//            shared-memory union-find over the bonds inside the tile, the new
//            spin of every cluster that does not touch the tile border, and
//            one "node" per border site (the master's "new lattice").
//   k_merge_union / k_merge_jump / k_merge_resolve
//            the master's step 2 (Sec. II.A): union-find over the border
//            nodes joined by the bonds that cross tile edges, including the
//            periodic wrap; the root of a global cluster is the minimum site
//            index (the DPM rule "the smaller label wins", Sec. II.B step 5);
//            then each node gets its cluster's root and new spin.
//
// Between launches only the 2-byte code per site and the node table cross
// the SM boundary; spins stay in shared memory from one sweep to the next.
#pragma once

#include <cstddef>
#include <cstdint>

namespace swg {

constexpr int TW = 128;           // tile width in sites (4 words of 32 sites)
constexpr int TWW = TW / 32;      // words per tile row
constexpr int PW = TW + 1;        // padded row of the shared forest (rows fall on distinct banks)
constexpr int CROSS_WORDS = 8;    // per tile: 4 words right-edge bits, 4 words bottom-edge bits

// 30-bit global roots: the GPU path supports N = L*L <= 2^30.
constexpr uint32_t ROOT_MASK = 0x3FFFFFFFu;
constexpr uint32_t FINAL_SPIN = 0x40000000u;
// A node key is a 30-bit site index (bits 0-29) plus KEY_REP; an edge slot
// past the tile's sites holds KEY_NONE, outside that range, so it differs
// from every real key up to site 2^30 - 1 (the corner of an L = 32768 lattice).
constexpr uint32_t KEY_NONE = 0x80000000u;
constexpr uint32_t KEY_REP = 0x40000000u;    // the node represents its piece
constexpr uint32_t KEY_MASK = 0x3FFFFFFFu;

// 2-byte tile-local cluster code of a site, written when a sweep starts and
// read when it finishes.
constexpr uint16_t CODE_BORDER = 0x8000u;   // bits 0-9: the piece's node slot
constexpr uint16_t CODE_SPIN = 0x4000u;     // interior: the cluster's new spin
constexpr uint16_t CODE_ROOT = 0x3FFFu;     // interior: tile-local root index

// Philox streams (counter word 3).
constexpr uint32_t STREAM_INIT = 0u, STREAM_BOND = 1u, STREAM_SPIN = 2u;

// Replica flags.
constexpr int32_t RF_PCC = 1;
constexpr int32_t RF_OPEN = 2;   // open boundaries: the links leaving the lattice do not exist
constexpr int32_t RF_CSIZE = 4;  // also sum |C|^2 over the clusters (psize, csize below)
constexpr int32_t RF_WIND = 8;   // topological rule: spans = a cluster winds around the box (nlink)

// Per-sweep observables as the device accumulates them (layout of sw_obs).
struct DevObs {
    unsigned long long bond_sum, mag, nclusters, nbonds;
    int32_t spans_x, spans_y;
    unsigned long long threshold;
    unsigned long long csize2;
};
static_assert(sizeof(DevObs) == 56, "DevObs must match sw_obs");

// One lattice of a launch.  A single sw_sweep call is a batch of one.
struct Replica {
    int32_t L;
    int32_t tiles_x, tiles_y;
    int32_t tile_base;      // first global tile index of this lattice
    uint32_t key0, key1;    // Philox key = (seed lo, seed hi)
    int32_t nsweeps;        // sweeps of this call
    int32_t flags;          // RF_*
    uint64_t sweep0;        // sweep index started by launch j = 0
    uint64_t thr;           // bond threshold (plain SW)
    uint64_t *thr_dev;      // PCC: the threshold lives on the device
    uint8_t *spin;          // L*L spins (read at j = 0, written at j = nsweeps)
    int32_t *label;         // L*L labels of the last sweep (written at j = nsweeps)
    uint8_t *bond;          // unused by the kernels (host bookkeeping)
    DevObs *obs;            // nsweeps entries
    int32_t jstart;         // launch index of this lattice's first launch
    // per-lattice scratch, indexed by the lattice's own tiles (lt) and nodes (lt * S + slot)
    uint16_t *code;         // tiles * TH * TW site codes
    uint32_t *bondbits;     // tiles * TH * 8 words (last sweep of a call only)
    uint32_t *cross;        // tiles * CROSS_WORDS
    int32_t *npar;          // tiles * S node parents
    int32_t *nkey;          // tiles * S node keys (global root candidates)
    uint32_t *nfinal;       // tiles * S resolved (root | spin << 30)
    // PCC scratch (Sec. III): spanning candidates and their coverage (null otherwise)
    uint32_t *pmask;        // tiles * S * 8: a piece's column mask (4 words), row mask (4 words)
    int32_t *cid;           // tiles * S * 2: candidate id + 2 of a root node (x, y), 0 = none
    int32_t *cand;          // [2][L] candidate roots (x, then y)
    int32_t *ncand;         // [3]: candidate counts (x, y), decide blocks finished
    uint32_t *cov;
    // cluster sizes (RF_CSIZE): sites of each border piece at its
    // representative node, and of each cluster at its root node
    int32_t *psize, *csize;
    // topological rule (RF_WIND): per node, parent (low 32 bits) and the
    // node's unwrapped displacement from its parent (high 32 bits, see
    // wind_off) -- one 64-bit word, so both change together
    unsigned long long *nlink;          // [L][tiles_x][4] column coverage, then [L][tiles_y][4] row coverage
};

// A launch: every tile of every lattice in the tile table (entries of -1
// are idle CTAs, so a batch can keep a fixed grid while lattices come and go).
struct SweepArgs {
    const Replica *reps;
    const int32_t *tile_rep;    // lattice of each global tile, or -1
    int32_t n_tiles;
    int32_t j;                  // launch index within a graph chunk
    const int32_t *jbase;       // chunk offset: launch index = j + *jbase
};

// Launch index of a lattice: finishes its sweep j-1 and starts its sweep j.
__device__ __forceinline__ int lattice_launch(const SweepArgs &a, const Replica &R)
{
    return a.j + *a.jbase - R.jstart;
}

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications, the high halves xored with the other counter
// words and the key, the key advanced by the Weyl constants between rounds.
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

// The method's blocks: counter = (word, sweep lo, sweep hi, stream).
__device__ __forceinline__ U4 stream_block(const Replica &R, uint64_t word, uint64_t sweep,
                                           uint32_t stream)
{
    return philox4x32_10((uint32_t)word, (uint32_t)sweep, (uint32_t)(sweep >> 32), stream,
                         R.key0, R.key1);
}

__device__ __forceinline__ uint32_t u4_word(const U4 &v, int i)
{
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// u < t for a threshold t in [1, 2^32], given t - 1 (t = 0 is handled by the
// caller: no link bonds)
__device__ __forceinline__ bool below(uint32_t u, uint32_t t_minus_1)
{
    return u <= t_minus_1;
}

// Mask of the valid sites (x < tw) in word c of a tile row.
__device__ __forceinline__ uint32_t valid_mask(int c, int tw)
{
    const int n = tw - 32 * c;
    return n >= 32 ? 0xFFFFFFFFu : (n <= 0 ? 0u : ((1u << n) - 1u));
}

// Resolved final (root | spin << 30) of an edge slot: a representative holds
// its cluster's, and so does every top or left slot (the ones a neighbour
// reads for its halo).  Only nfinal is read: the tile kernel that reads a
// neighbour's finals rewrites that neighbour's npar and nkey concurrently.

// ------------------------------------------------------------ tile geometry
struct Tile {
    int g, lt, tx, ty, x0, y0, tw, th, g_right, g_down;   // lt, g_right, g_down: the lattice's own tiles
};

__device__ __forceinline__ Tile tile_of(const Replica &R, int g, int TH)
{
    Tile t;
    t.g = g;
    t.lt = g - R.tile_base;
    t.tx = t.lt % R.tiles_x;
    t.ty = t.lt / R.tiles_x;
    t.x0 = t.tx * TW;
    t.y0 = t.ty * TH;
    t.tw = min(TW, R.L - t.x0);
    t.th = min(TH, R.L - t.y0);
    t.g_right = t.ty * R.tiles_x + (t.tx + 1) % R.tiles_x;        // local tile indices
    t.g_down = ((t.ty + 1) % R.tiles_y) * R.tiles_x + t.tx;
    return t;
}

// Node slots of a tile: [0,TW) top row, [TW,2TW) bottom row, [2TW,2TW+TH)
// left column, [2TW+TH, 2TW+2TH) right column.
template <int TH>
struct Slots {
    static constexpr int S = 2 * TW + 2 * TH;
    static constexpr int TOP = 0, BOTTOM = TW, LEFT = 2 * TW, RIGHT = 2 * TW + TH;
};

template <int TH>
__device__ __forceinline__ bool slot_site(int s, int tw, int th, int &site)
{
    using SL = Slots<TH>;
    int x, y;
    if (s < SL::BOTTOM) {
        x = s;
        y = 0;
        if (x >= tw) return false;
    } else if (s < SL::LEFT) {
        x = s - SL::BOTTOM;
        y = th - 1;
        if (x >= tw) return false;
    } else if (s < SL::RIGHT) {
        x = 0;
        y = s - SL::LEFT;
        if (y >= th) return false;
    } else {
        x = tw - 1;
        y = s - SL::RIGHT;
        if (y >= th) return false;
    }
    site = y * TW + x;
    return true;
}

// ----------------------------------------------- shared-memory union-find
// Links always hang the larger root under the smaller index, so every root
// is the minimum local index of its piece, and tile-local row-major order is
// the global order: the local root is the piece's minimum global site.
__device__ __forceinline__ int sfind(volatile int *par, int x)
{
    int p = par[x];
    while (p != x) {
        const int gp = par[p];
        if (gp != p) par[x] = gp;  // path halving: only ever an ancestor
        x = gp;
        p = par[x];
    }
    return x;
}

// As sunite, returning the root of the united set.
__device__ __forceinline__ int sunite_root(volatile int *par, int a, int b)
{
    for (;;) {
        a = sfind(par, a);
        b = sfind(par, b);
        if (a == b) return a;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS((int *)&par[b], b, a) == b) return a;
    }
}

__device__ __forceinline__ void sunite(volatile int *par, int a, int b)
{
    for (;;) {
        a = sfind(par, a);
        b = sfind(par, b);
        if (a == b) return;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS((int *)&par[b], b, a) == b) return;
    }
}

// As sunite, reporting whether this call linked two sets (false: a and b
// were already in one set).
__device__ __forceinline__ bool sunite_linked(volatile int *par, int a, int b)
{
    for (;;) {
        a = sfind(par, a);
        b = sfind(par, b);
        if (a == b) return false;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS((int *)&par[b], b, a) == b) return true;
    }
}

// Threads of a tile CTA: one warp per 32 x 32 sub-tile.
template <int TH>
struct TileCfg {
    static constexpr int NT = 4 * TH;           // threads per CTA
    static constexpr int NW = NT / 32;          // warps = sub-tiles
    static constexpr int SUBY = TH / 32;        // sub-tile rows
    // CTAs per SM the register allocation must leave room for: as many as
    // the shared memory allows (32 rows: eleven CTAs; 64 rows: six; 96 rows:
    // four; 128 rows: three), which caps a thread at 40 registers.  The
    // kernel is latency-bound in its union-find, so resident warps pay: three
    // 128-row CTAs per SM run 19% faster than two.
    static constexpr int MINB = TH == 32 ? 11 : TH == 64 ? 6 : TH == 96 ? 4 : 3;
};

// Root of x without writing (a forest no thread is changing any more).
__device__ __forceinline__ int sroot(const volatile int *par, int x)
{
    int p = par[x];
    while (p != x) {
        x = p;
        p = par[x];
    }
    return x;
}

// Packed per-root record written over a root's own forest entry once the
// tile is labelled: INFO_BORDER | 0x8000 | slot for a piece that touches the
// tile border (slot = its representative node), INFO_INTERIOR | spin << 14 |
// local index for a cluster that ends inside the tile.  The low 16 bits are
// the site code.  Forest indices stay below INFO_INTERIOR.
constexpr uint32_t INFO_BORDER = 0x80008000u;
constexpr uint32_t INFO_INTERIOR = 0x40000000u;

// Run heads of a 32-site row word inside one sub-tile: bit x is set iff
// x == 0 or the link (x-1, x) is not a bond (bit 31 of h, the link leaving
// the sub-tile, is ignored).
__device__ __forceinline__ uint32_t run_heads(uint32_t h)
{
    return ~((h & 0x7FFFFFFFu) << 1);
}

// Local index of the head of the run that holds bit x of a row word whose
// first site has local index base.
__device__ __forceinline__ int head_of(uint32_t heads, int base, int x)
{
    return base + 31 - __clz(heads & (0xFFFFFFFFu >> (31 - x)));
}

// Connected components of the intra-tile bonds (H: right links, whose link
// leaving the tile's last column is ignored; V: down links, ignored in the
// tile's last row).  The tile is cut into 32 x 32 sub-tiles, one per warp,
// and the forest lives on run heads only (a run = maximal chain of right
// bonds inside one sub-tile row; its head is its leftmost site):
//   1. lane r of a warp owns row r of its sub-tile: it unites the runs of its
//      row with the runs below at every down bond, skipping a bond when the
//      bond to its left already joins the same two runs;
//   2. unions across the sub-tile boundaries inside the tile.
// Links always hang the larger root under the smaller, so par[x] < x unless x
// is a root and every root is the minimum local index of its piece; local
// row-major order is the global order, so the root is the piece's minimum
// site.  Forest indices are padded, y * PW + x, which keeps row-major order
// and puts the rows of a column on distinct shared-memory banks.
template <int TH>
__device__ void tile_label(volatile int *par, const uint32_t (*Hb)[TWW], const uint32_t (*Vb)[TWW],
                           int th, int tw)
{
    constexpr int NT = TileCfg<TH>::NT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sx = warp & (TWW - 1), sy = warp / TWW;
    // the intra-tile bonds: the tile's last column has no right link inside,
    // its last row no down link inside
    auto H = [&](int y, int c) { return Hb[y][c] & valid_mask(c, tw - 1); };
    auto V = [&](int y, int c) { return y < th - 1 ? Vb[y][c] : 0u; };

    // ---- 1. inside each sub-tile, lane = row
    {
        const int y = 32 * sy + lane;
        const bool row_ok = y < th;
        const uint32_t heads = run_heads(row_ok ? H(y, sx) : 0u);
        const uint32_t heads_below = __shfl_down_sync(0xFFFFFFFFu, heads, 1);
        const uint32_t v = (row_ok && lane < 31) ? V(y, sx) : 0u;
        const uint32_t u = v & (~(v << 1) | heads | heads_below);
        const int base = y * PW + 32 * sx;
        if (row_ok) {   // every site of the row its own root (only run heads are used)
#pragma unroll
            for (int x = 0; x < 32; ++x) par[base + x] = base + x;
        }
        __syncwarp();
        // consecutive contacts often share a run above or below: their
        // finds start at the last union's root (an ancestor of that run's
        // head), not at the head
        int prev_a = -1, prev_b = -1, prev_r = 0;
        for (uint32_t b = u; b; b &= b - 1) {
            const int x = __ffs(b) - 1;
            const int ha = head_of(heads, base, x), hb = head_of(heads_below, base + PW, x);
            prev_r = sunite_root(par, ha == prev_a ? prev_r : ha, hb == prev_b ? prev_r : hb);
            prev_a = ha;
            prev_b = hb;
        }
    }
    __syncthreads();

    // ---- 2. links across sub-tile boundaries: vertical boundaries between
    //         sub-tile columns, horizontal ones between sub-tile rows
    {
        constexpr int NV = (TWW - 1) * TH;
        constexpr int NH = (TH / 32 - 1) * TW;
        for (int q = threadIdx.x; q < NV + NH; q += NT) {
            int a, b;
            if (q < NV) {
                const int bnd = q / TH + 1, y = q % TH;     // link (32 bnd - 1, y) - (32 bnd, y)
                if (y >= th || !((H(y, bnd - 1) >> 31) & 1u)) continue;
                // skip when the row above already joins the same two sites
                // through down links inside the sub-tiles (united in phase 1;
                // at a sub-tile row edge those down links are phase-2 links
                // themselves and could justify each other in a cycle)
                if ((y & 31) != 0 && ((H(y - 1, bnd - 1) >> 31) & 1u) &&
                    ((V(y - 1, bnd - 1) >> 31) & 1u) && (V(y - 1, bnd) & 1u))
                    continue;
                a = head_of(run_heads(H(y, bnd - 1)), y * PW + 32 * (bnd - 1), 31);
                b = y * PW + 32 * bnd;   // column 0 of a sub-tile row is always a head
            } else {
                const int r = q - NV;
                const int bnd = r / TW + 1, x = r % TW;     // link (x, 32 bnd - 1) - (x, 32 bnd)
                const int y = 32 * bnd - 1;
                if (y + 1 >= th || !((V(y, x >> 5) >> (x & 31)) & 1u)) continue;
                // skip when the column to the left already joins the same two
                // sites through right links inside the sub-tiles
                if ((x & 31) != 0 && ((V(y, (x - 1) >> 5) >> ((x - 1) & 31)) & 1u) &&
                    ((H(y, (x - 1) >> 5) >> ((x - 1) & 31)) & 1u) &&
                    ((H(y + 1, (x - 1) >> 5) >> ((x - 1) & 31)) & 1u))
                    continue;
                const int c = x >> 5;
                a = head_of(run_heads(H(y, c)), y * PW + 32 * c, x & 31);
                b = head_of(run_heads(H(y + 1, c)), (y + 1) * PW + 32 * c, x & 31);
            }
            sunite(par, a, b);
        }
    }
    __syncthreads();
}

// ------------------------------------------------ global-memory union-find
__device__ __forceinline__ int gload(const int32_t *p)
{
    return *(const volatile int32_t *)p;
}

__device__ __forceinline__ int gfind(int32_t *par, int x)
{
    int p = gload(par + x);
    while (p != x) {
        const int gp = gload(par + p);
        if (gp != p) *(volatile int32_t *)(par + x) = gp;
        x = gp;
        p = gload(par + x);
    }
    return x;
}

// Union of the node forest ordered by key: the root with the larger key is
// hung under the root with the smaller one.  Keys are the global indices of
// the pieces' local roots, distinct between pieces and equal only inside one
// piece (whose non-representative nodes are never roots), so keys fall
// strictly along every chain of root links (no cycle can form) and each
// set's root carries the set's minimum key: the global cluster root.
__device__ __forceinline__ void gunite_by_key(int32_t *par, const int32_t *key, int a, int b)
{
    for (;;) {
        a = gfind(par, a);
        b = gfind(par, b);
        if (a == b) return;
        if (key[a] > key[b]) {
            const int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(par + b, b, a) == b) return;
    }
}

// --------------------------------------------------------- block reductions
template <int NT, int K>
__device__ __forceinline__ void block_sum_atomic(long long (&v)[K], unsigned long long *const dst[K],
                                                 long long (*red)[K])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < K; ++q) {
        long long x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
        if (lane == 0) red[warp][q] = x;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            long long x = lane < NT / 32 ? red[lane][q] : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
            if (lane == 0 && dst[q] && x != 0) atomicAdd(dst[q], (unsigned long long)x);
        }
    }
}

// 16 bytes from global to shared memory without passing through registers
// (completed by cp_async_wait_all before a barrier)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ------------------------------------------------------------ shared layout
template <int TH>
struct TileSmem {
    int par[TH * PW];               // union-find forest over run heads (padded rows); in the
                                    // finish half, the tile's site codes (TH * TW * 2 bytes)
    uint32_t sp[TH + 1][TWW];       // spins as bits, row TH = halo row; in a tile narrower
                                    // than TW, bit tw of a row = the halo column
    uint32_t spx[TH / 32];          // halo column of a full-width tile: bit y = row y
    uint32_t bh[TH][TWW];           // right-link bonds (bit x: link (x,y)-(x+1,y))
    uint32_t bv[TH][TWW];           // down-link bonds
    union {                         // never live at the same time:
        uint32_t finfo[Slots<TH>::S];        // finish half: finals of the tile's own nodes
        uint32_t spb[TH][TWW];               // start half: SPIN-stream bit of each site
        long long red[TileCfg<TH>::NW][4];   // the reduction that ends each half
    } u;
    uint32_t pm[Slots<TH>::S][8];   // PCC: per border piece, columns and rows it occupies
};

// Dynamic shared memory of a tile launch: the piece masks only when a PCC
// lattice takes part.
template <int TH>
constexpr size_t tile_smem(bool pcc)
{
    return pcc ? sizeof(TileSmem<TH>) : offsetof(TileSmem<TH>, pm);
}

// ----------------------------------------------------------------- k_tile
// Optional features, compiled in only where a launch has a lattice that
// needs them, so the plain kernels carry none of their code.  The tile kernel
// comes in two variants, plain (F = 0) and with every tile feature (F =
// FEAT_TILE, each feature then checked per lattice); the merge kernels with
// and without FEAT_WIND.
constexpr int FEAT_CSIZE = 1;   // cluster sizes (RF_CSIZE)
constexpr int FEAT_OPEN = 2;    // open boundaries (RF_OPEN)
constexpr int FEAT_WIND = 4;    // topological rule (RF_WIND; merge kernels only)
constexpr int FEAT_PCC = 8;     // PCC piece masks (RF_PCC)
constexpr int FEAT_TILE = FEAT_CSIZE | FEAT_OPEN | FEAT_PCC;

template <int TH, int F>
__global__ void __launch_bounds__(TileCfg<TH>::NT, TileCfg<TH>::MINB) k_tile(const SweepArgs a)
{
    using SL = Slots<TH>;
    constexpr int S = SL::S;
    constexpr int NT = TileCfg<TH>::NT;
    constexpr int NW = TileCfg<TH>::NW;
    constexpr int SPT = (S + NT - 1) / NT;   // node slots per thread
    constexpr int NQ = TH * TW / 8 / NT;     // 8-site groups per thread
    static_assert(NQ * 8 * NT == TH * TW, "tile sites must split into 8-site groups");
    static_assert(TH * TWW == NT, "one 32-site word of the tile per thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem<TH> &sm = *reinterpret_cast<TileSmem<TH> *>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;

    const int g = blockIdx.x;
    if (g >= a.n_tiles) return;
    const int ri = a.tile_rep[g];
    if (ri < 0) return;
    const Replica &R = a.reps[ri];
    const int j = lattice_launch(a, R);   // finishes sweep j-1, starts sweep j
    if (j < 0) return;
    const bool fin = j >= 1 && j <= R.nsweeps;
    const bool start = j < R.nsweeps;
    if (!fin && !start) return;
    const Tile t = tile_of(R, g, TH);
    const int L = R.L;
    // open boundaries: the last tile column has no right link in its last
    // column, the last tile row no down link in its last row
    const bool open_r = (F & FEAT_OPEN) && (R.flags & RF_OPEN) && t.tx == R.tiles_x - 1;
    const bool open_b = (F & FEAT_OPEN) && (R.flags & RF_OPEN) && t.ty == R.tiles_y - 1;
    // site indices fit in 32 bits (N <= 2^30)
    const uint32_t uL = (uint32_t)L;
    const uint32_t gbase = (uint32_t)t.y0 * uL + (uint32_t)t.x0;   // global index of local site 0
    uint16_t *code = R.code + (size_t)t.lt * TH * TW;
    // the intra-tile right bonds of word (y, c): the tile's last column links out
    auto ih_of = [&](int y, int c) { return sm.bh[y][c] & valid_mask(c, t.tw - 1); };
    // the spin word right of word (y, c), of which only bit 0 is used: the next
    // word of the row, or the halo column of a full-width tile
    auto right_of = [&](int y, int c) { return c + 1 < TWW ? sm.sp[y][c + 1] : sm.spx[y >> 5] >> (y & 31); };
    // sets the halo-column spin of row y (the spin right of the tile's last column)
    auto set_halo = [&](int y) {
        if (t.tw == TW)
            atomicOr(&sm.spx[y >> 5], 1u << (y & 31));
        else
            sm.sp[y][t.tw >> 5] |= 1u << (t.tw & 31);
    };

    if (fin) {
        // ---- finish sweep k-1: resolve every site's cluster and flip it
        const int jf = j - 1;
        const bool last = j == R.nsweeps;
        // the tile's codes, 8 sites per 16-byte asynchronous copy straight
        // into shared memory (the forest's space, unused until the labelling)
        const uint4 *code4 = reinterpret_cast<const uint4 *>(code);
        uint4 *scode4 = reinterpret_cast<uint4 *>(sm.par);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int idx = tid + q * NT;
            if ((idx * 8) / TW < t.th) cp_async16(scode4 + idx, code4 + idx);
        }
        for (int s = tid; s < S; s += NT) sm.u.finfo[s] = R.nfinal[(size_t)t.lt * S + s];
        // the halos' finals (new spins of the top row of the tile below and of
        // the left column of the tile to the right), issued with the codes
        uint32_t fb = 0u, fr = 0u;
        if (warp < TWW && 32 * warp + lane < t.tw) fb = R.nfinal[(size_t)t.g_down * S + SL::TOP + 32 * warp + lane];
        if (tid < t.th) fr = R.nfinal[(size_t)t.g_right * S + SL::LEFT + tid];
        for (int w = tid; w < TH / 32; w += NT) sm.spx[w] = 0u;
        cp_async_wait_all();
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int idx = tid + q * NT;
            const int y = (idx * 8) / TW, xb = (idx * 8) % TW;
            if (y >= t.th) continue;
            const uint4 cq = scode4[idx];
            const uint32_t wv[4] = {cq.x, cq.y, cq.z, cq.w};
            uint32_t bits = 0;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint32_t u = (wv[e >> 1] >> (16 * (e & 1))) & 0xFFFFu;
                const uint32_t spin =
                    (u & CODE_BORDER) ? (sm.u.finfo[u & 0x3FFu] >> 30) & 1u : (u >> 14) & 1u;
                bits |= spin << e;
            }
            bits &= (1u << min(8, max(0, t.tw - xb))) - 1u;   // sites past tw are not spins
            reinterpret_cast<uint8_t *>(&sm.sp[y][0])[xb >> 3] = (uint8_t)bits;
            if (last) {
                const uint32_t gi0 = gbase + (uint32_t)y * uL + (uint32_t)xb;
                uint32_t roots[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const uint32_t u = (wv[e >> 1] >> (16 * (e & 1))) & 0xFFFFu;
                    const uint32_t lr = u & CODE_ROOT;
                    roots[e] = (u & CODE_BORDER) ? sm.u.finfo[u & 0x3FFu] & ROOT_MASK
                                                 : gbase + (lr / TW) * uL + (lr % TW);
                }
                const int nval = min(8, t.tw - xb);
                if (nval == 8 && (gi0 & 7u) == 0) {
                    // spread the 8 spin bits to 8 bytes
                    const uint32_t lo = ((bits & 0xFu) * 0x00204081u) & 0x01010101u;
                    const uint32_t hi = (((bits >> 4) & 0xFu) * 0x00204081u) & 0x01010101u;
                    *reinterpret_cast<uint2 *>(R.spin + gi0) = make_uint2(lo, hi);
                    int4 *lp = reinterpret_cast<int4 *>(R.label + gi0);
                    lp[0] = make_int4((int)roots[0], (int)roots[1], (int)roots[2], (int)roots[3]);
                    lp[1] = make_int4((int)roots[4], (int)roots[5], (int)roots[6], (int)roots[7]);
                } else {
                    for (int e = 0; e < nval; ++e) {
                        R.spin[gi0 + e] = (uint8_t)((bits >> e) & 1u);
                        R.label[gi0 + e] = (int32_t)roots[e];
                    }
                }
            }
        }
        // bottom halo row: new spins of the top row of the tile below
        if (warp < TWW) {
            const uint32_t word = __ballot_sync(0xFFFFFFFFu, (fb & FINAL_SPIN) != 0u);
            if (lane == 0) sm.sp[t.th][warp] = word;
        }
        __syncthreads();
        // right halo column: new spins of the left column of the tile to the right
        if (fr & FINAL_SPIN) set_halo(tid);
        __syncthreads();
        long long bs = 0, mag = 0;
        for (int w = tid; w < t.th * TWW; w += NT) {
            const int y = w >> 2, c = w & 3;
            const uint32_t vm = valid_mask(c, t.tw);
            const uint32_t vr = open_r ? valid_mask(c, t.tw - 1) : vm;   // sites with a right link
            const uint32_t vd = (open_b && y == t.th - 1) ? 0u : vm;      // sites with a down link
            const uint32_t cur = sm.sp[y][c];
            const uint32_t right = (cur >> 1) | (right_of(y, c) << 31);
            const uint32_t down = sm.sp[y + 1][c];
            bs += __popc(vr) - 2 * __popc((cur ^ right) & vr) + __popc(vd) - 2 * __popc((cur ^ down) & vd);
            mag += 2 * __popc(cur & vm) - __popc(vm);
        }
        // clusters that touch a tile border: their sizes were summed at their
        // root nodes by the merge; each root node is in exactly one tile
        long long c2 = 0;
        if ((F & FEAT_CSIZE) && (R.flags & RF_CSIZE))
            for (int s = tid; s < S; s += NT) {
                const long long c = R.csize[(size_t)t.lt * S + s];
                c2 += c * c;
            }
        long long v[4] = {bs, mag, c2, 0};
        DevObs *o = R.obs + jf;
        unsigned long long *const dst[4] = {&o->bond_sum, &o->mag, &o->csize2, nullptr};
        block_sum_atomic<NT, 4>(v, dst, sm.u.red);
        __syncthreads();
    }

    if (!start) return;

    // ---- start sweep k
    const uint64_t k = R.sweep0 + (uint64_t)j;
    const uint64_t thr = (R.flags & RF_PCC) ? *R.thr_dev : R.thr;
    if (!fin) {
        // first sweep of the call: spins (and halos) from global memory
        for (int w = tid; w < TH / 32; w += NT) sm.spx[w] = 0u;
        for (int w = warp; w < (t.th + 1) * TWW; w += NW) {
            const int y = w >> 2, c = w & 3;
            const int x = 32 * c + lane;
            const uint32_t gy = (uint32_t)((t.y0 + y) % L);
            int spin = 0;
            if (x < t.tw) spin = R.spin[gy * uL + (uint32_t)(t.x0 + x)];
            const uint32_t word = __ballot_sync(0xFFFFFFFFu, spin);
            if (lane == 0) sm.sp[y][c] = word;
        }
        __syncthreads();
        for (int y = tid; y < t.th; y += NT) {
            const uint32_t gi = (uint32_t)(t.y0 + y) * uL + (uint32_t)((t.x0 + t.tw) % L);
            if (R.spin[gi]) set_halo(y);
        }
        __syncthreads();
    }
    const bool pcc = (F & FEAT_PCC) && (R.flags & RF_PCC) != 0;
    if (pcc)
        for (int q = tid; q < S * 8; q += NT) (&sm.pm[0][0])[q] = 0u;
    if (t.lt == 0 && tid == 0) {
        R.obs[j].threshold = thr;
        R.obs[j].spans_x = 0;
        R.obs[j].spans_y = 0;
    }

    // Step 1 (Sec. I): bonds.  Link l = 2i + d draws word (l mod 4) of
    // Philox(l/4, k, BOND), i.e. sites 2m and 2m+1 share block m.
    const uint32_t klo = (uint32_t)k, khi = (uint32_t)(k >> 32);
    const bool any_bond = thr != 0;               // t = 0: P = 0, nothing bonds
    const uint32_t tm1 = (uint32_t)(thr - 1);     // t in [1, 2^32] -> t - 1 fits 32 bits
    // the bonds of row y from its two horizontal-and-vertical draw words per
    // 32-site word (rh, rv): keep the links whose spins agree, store them
    // rows yA and yB at once: lane c < 4 takes word c of row yA, lane 4 + c
    // word c of row yB (skipped when yB is past the tile)
    auto store_rows = [&](int yA, const uint32_t (&rhA)[TWW], const uint32_t (&rvA)[TWW], int yB,
                          const uint32_t (&rhB)[TWW], const uint32_t (&rvB)[TWW]) {
        const bool second = lane >= TWW;
        const int y = second ? yB : yA;
        if (lane < 2 * TWW && y < t.th) {
            const int c = lane & (TWW - 1);
            const uint32_t rhc = second ? (c == 0 ? rhB[0] : c == 1 ? rhB[1] : c == 2 ? rhB[2] : rhB[3])
                                        : (c == 0 ? rhA[0] : c == 1 ? rhA[1] : c == 2 ? rhA[2] : rhA[3]);
            const uint32_t rvc = second ? (c == 0 ? rvB[0] : c == 1 ? rvB[1] : c == 2 ? rvB[2] : rvB[3])
                                        : (c == 0 ? rvA[0] : c == 1 ? rvA[1] : c == 2 ? rvA[2] : rvA[3]);
            const uint32_t vm = valid_mask(c, t.tw);
            const uint32_t vr = open_r ? valid_mask(c, t.tw - 1) : vm;
            const uint32_t vd = (open_b && y == t.th - 1) ? 0u : vm;
            const uint32_t cur = sm.sp[y][c];
            const uint32_t right = (cur >> 1) | (right_of(y, c) << 31);
            const uint32_t down = sm.sp[y + 1][c];
            const uint32_t h = rhc & ~(cur ^ right) & vr;
            const uint32_t v = rvc & ~(cur ^ down) & vd;
            sm.bh[y][c] = h;
            sm.bv[y][c] = v;
        }
    };
    auto store_row = [&](int y, const uint32_t (&rh)[TWW], const uint32_t (&rv)[TWW]) {
        store_rows(y, rh, rv, t.th, rh, rv);
    };
    // aligned row: lane l drew the blocks of sites (2l, 2l+1) (r0) and
    // (64+2l, 65+2l) (r1); lane x of each 32-site word fetches its two bits
    // by shuffle
    auto draws_aligned = [&](const U4 &r0, const U4 &r1, uint32_t (&rh)[TWW], uint32_t (&rv)[TWW]) {
        const uint32_t nib0 = (below(r0.x, tm1) ? 1u : 0u) | (below(r0.y, tm1) ? 2u : 0u) |
                              (below(r0.z, tm1) ? 4u : 0u) | (below(r0.w, tm1) ? 8u : 0u);
        const uint32_t nib1 = (below(r1.x, tm1) ? 1u : 0u) | (below(r1.y, tm1) ? 2u : 0u) |
                              (below(r1.z, tm1) ? 4u : 0u) | (below(r1.w, tm1) ? 8u : 0u);
#pragma unroll
        for (int q = 0; q < TWW; ++q) {
            const uint32_t n = __shfl_sync(0xFFFFFFFFu, q < 2 ? nib0 : nib1, 16 * (q & 1) + (lane >> 1)) >>
                               (2 * (lane & 1));
            rh[q] = __ballot_sync(0xFFFFFFFFu, n & 1u);
            rv[q] = __ballot_sync(0xFFFFFFFFu, n & 2u);
        }
    };
    if (any_bond && (uL & 1u) == 0) {
        // even L: every row starts on an even site; two rows per pass, four
        // independent Philox blocks in flight per lane
        for (int y = warp; y < t.th; y += 2 * NW) {
            const int y2 = y + NW;
            const uint32_t b0 = ((gbase + (uint32_t)y * uL) >> 1) + lane;
            const uint32_t b2 = ((gbase + (uint32_t)y2 * uL) >> 1) + lane;
            const U4 r0 = philox4x32_10(b0, klo, khi, STREAM_BOND, R.key0, R.key1);
            const U4 r1 = philox4x32_10(b0 + 32, klo, khi, STREAM_BOND, R.key0, R.key1);
            const U4 r2 = philox4x32_10(b2, klo, khi, STREAM_BOND, R.key0, R.key1);
            const U4 r3 = philox4x32_10(b2 + 32, klo, khi, STREAM_BOND, R.key0, R.key1);
            uint32_t rh[TWW], rv[TWW], rh2[TWW], rv2[TWW];
            draws_aligned(r0, r1, rh, rv);
            draws_aligned(r2, r3, rh2, rv2);
            store_rows(y, rh, rv, y2, rh2, rv2);
        }
    } else {
        for (int y = warp; y < t.th; y += NW) {
            const uint32_t G0 = gbase + (uint32_t)y * uL;
            uint32_t rh[TWW], rv[TWW];
            if (!any_bond) {
#pragma unroll
                for (int q = 0; q < TWW; ++q) rh[q] = rv[q] = 0u;
            } else if ((G0 & 1u) == 0) {
                const uint32_t b0 = (G0 >> 1) + lane;
                const U4 r0 = philox4x32_10(b0, klo, khi, STREAM_BOND, R.key0, R.key1);
                const U4 r1 = philox4x32_10(b0 + 32, klo, khi, STREAM_BOND, R.key0, R.key1);
                draws_aligned(r0, r1, rh, rv);
            } else {
                // odd row start (odd L): every site draws its own block
#pragma unroll
                for (int q = 0; q < TWW; ++q) {
                    const uint32_t gi = G0 + 32 * q + lane;
                    const U4 r = philox4x32_10(gi >> 1, klo, khi, STREAM_BOND, R.key0, R.key1);
                    const bool odd = gi & 1u;
                    rh[q] = __ballot_sync(0xFFFFFFFFu, below(odd ? r.z : r.x, tm1));
                    rv[q] = __ballot_sync(0xFFFFFFFFu, below(odd ? r.w : r.y, tm1));
                }
            }
            store_row(y, rh, rv);
        }
    }
    // The SPIN-stream bit of every site of the tile, for the clusters that end
    // inside it (Sec. I step 3: one new random spin per cluster): bit (g mod
    // 128) of Philox(g / 128, k, SPIN) for a site of global index g.  A row's
    // 128 sites span the two blocks from the one holding its first site; one
    // thread per row draws them and keeps the row's 128 bits.
    for (int y = tid; y < t.th; y += NT) {
        const uint32_t g0 = gbase + (uint32_t)y * uL;
        const uint32_t pos = g0 & 127u;
        const U4 r0 = philox4x32_10(g0 >> 7, klo, khi, STREAM_SPIN, R.key0, R.key1);
        U4 r1 = r0;
        if (pos) r1 = philox4x32_10((g0 >> 7) + 1, klo, khi, STREAM_SPIN, R.key0, R.key1);
        // the 8 words from the first one the row needs: words pos/32 .. pos/32 + 4
        uint32_t w[5];
        switch (pos >> 5) {
        case 0: w[0] = r0.x; w[1] = r0.y; w[2] = r0.z; w[3] = r0.w; w[4] = r1.x; break;
        case 1: w[0] = r0.y; w[1] = r0.z; w[2] = r0.w; w[3] = r1.x; w[4] = r1.y; break;
        case 2: w[0] = r0.z; w[1] = r0.w; w[2] = r1.x; w[3] = r1.y; w[4] = r1.z; break;
        default: w[0] = r0.w; w[1] = r1.x; w[2] = r1.y; w[3] = r1.z; w[4] = r1.w; break;
        }
#pragma unroll
        for (int c = 0; c < TWW; ++c) sm.u.spb[y][c] = __funnelshift_r(w[c], w[c + 1], pos & 31u);
    }
    __syncthreads();

    long long nb = 0;
    for (int w = tid; w < t.th * TWW; w += NT) {
        const int y = w >> 2, c = w & 3;
        nb += __popc(sm.bh[y][c]) + __popc(sm.bv[y][c]);
    }
    // crossing bonds: right edge (bit tw-1 of each row), bottom edge (row th-1)
    for (int q = warp; q <= TH / 32; q += NW) {
        if (q < TH / 32) {
            const int y = 32 * q + lane;
            const int bit = (y < t.th) ? (sm.bh[y][(t.tw - 1) >> 5] >> ((t.tw - 1) & 31)) & 1 : 0;
            const uint32_t word = __ballot_sync(0xFFFFFFFFu, bit);
            if (lane == 0) R.cross[(size_t)t.lt * CROSS_WORDS + q] = word;
        } else if (lane < TWW) {
            R.cross[(size_t)t.lt * CROSS_WORDS + TWW + lane] = sm.bv[t.th - 1][lane];
        }
    }
    if (j == R.nsweeps - 1) {
        // the last sweep of the call keeps its bonds for sw_get_bonds
        uint32_t *bb = R.bondbits + (size_t)t.lt * TH * 2 * TWW;
        for (int w = tid; w < t.th * TWW; w += NT) {
            const int y = w >> 2, c = w & 3;
            bb[y * 2 * TWW + c] = sm.bh[y][c];
            bb[y * 2 * TWW + TWW + c] = sm.bv[y][c];
        }
    }

    // Step 2 inside the tile (Hoshen-Kopelman's role in Sec. II.A slave step 1)
    tile_label<TH>(sm.par, sm.bh, sm.bv, t.th, t.tw);

    // One node per border site: key = global index of the piece's local root,
    // parent = the piece's first border slot (the representative).
    int rs[SPT];
#pragma unroll
    for (int q = 0; q < SPT; ++q) {
        const int s = tid + q * NT;
        int site;
        rs[q] = -1;
        if (s < S && slot_site<TH>(s, t.tw, t.th, site)) {
            const int sy = site / TW, c = (site % TW) >> 5;
            rs[q] = sroot(sm.par, head_of(run_heads(ih_of(sy, c)), sy * PW + 32 * c, site & 31));
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < SPT; ++q)
        if (rs[q] >= 0) atomicMin((int *)&sm.par[rs[q]], (int)(INFO_BORDER | (uint32_t)(tid + q * NT)));
    __syncthreads();
#pragma unroll
    for (int q = 0; q < SPT; ++q) {
        const int s = tid + q * NT;
        if (s >= S) break;
        const size_t node = (size_t)t.lt * S + s;
        if (rs[q] >= 0) {
            const int rep = sm.par[rs[q]] & 0x3FF;
            R.npar[node] = (int32_t)((size_t)t.lt * S + rep);
            R.nkey[node] = (int32_t)((gbase + (uint32_t)(rs[q] / PW) * uL + (uint32_t)(rs[q] % PW)) |
                                     (rep == s ? KEY_REP : 0u));
        } else {
            R.npar[node] = (int32_t)node;
            R.nkey[node] = (int32_t)KEY_NONE;
        }
        if ((F & FEAT_CSIZE) && (R.flags & RF_CSIZE)) R.csize[node] = 0;   // the merge adds piece sizes at root nodes
    }
    // Every run head learns its root; every interior root gets its record
    // (the cluster's new spin, Sec. I step 3, drawn here) and is counted.
    // A walk stops at a root, a border record or an interior record, and each
    // thread writes only its own heads, so concurrent walks see ancestors.
    long long ncl_interior = 0;
    for (int w = tid; w < t.th * TWW; w += NT) {
        const int y = w % t.th, c = w / t.th;   // a warp covers consecutive rows
        const int base = y * PW + 32 * c;
        for (uint32_t bits = run_heads(ih_of(y, c)); bits; bits &= bits - 1) {
            const int hx = __ffs(bits) - 1;
            const int hd = base + hx;
            int x = hd, p = sm.par[x];
            while (p != x && p >= 0 && (uint32_t)p < INFO_INTERIOR) {
                x = p;
                p = sm.par[x];
            }
            if (x != hd) {
                // the root's record itself where it is already there (codes
                // then need one load); the root otherwise.  Cluster sizes add
                // at roots, so the feature variant keeps root indices.
                sm.par[hd] = (!(F & FEAT_CSIZE) && (uint32_t)p >= INFO_INTERIOR && p != x) ? p : x;
            } else if (p == hd && 32 * c + hx < t.tw) {
                // an interior root inside the tile: its site's SPIN-stream bit
                const uint32_t spin = (sm.u.spb[y][c] >> hx) & 1u;
                sm.par[hd] = (int)(INFO_INTERIOR | (spin << 14) | (uint32_t)(y * TW + 32 * c + hx));
                ++ncl_interior;
            }
        }
    }
    __syncthreads();
    const bool csz = (F & FEAT_CSIZE) && (R.flags & RF_CSIZE) != 0;
    if (csz) {
        // cluster sizes: every run adds its length to bits 16-30 of its root's
        // record (a piece holds at most TW*TH = 2^14 sites, an interior
        // cluster at most (TW-2)(TH-2) < 2^14, so neither field overflows
        // into the record's flag bits); the codes below read bits 0-15 only
        for (int w = tid; w < t.th * TWW; w += NT) {
            const int y = w % t.th, c = w / t.th;
            const int base = y * PW + 32 * c;
            const int vw = min(32, t.tw - 32 * c);   // real sites in this word
            for (uint32_t bits = run_heads(ih_of(y, c)); bits;) {
                const int hx = __ffs(bits) - 1;
                bits &= bits - 1;
                if (hx >= vw) break;
                const int nx = bits ? __ffs(bits) - 1 : 32;
                const int v = sm.par[base + hx];
                const int root = (v < 0 || (uint32_t)v >= INFO_INTERIOR) ? base + hx : v;
                atomicAdd((int *)&sm.par[root], (min(nx, vw) - hx) << 16);
            }
        }
    }
    // Every site's 2-byte code (the low half of its root's record): border
    // pieces by node slot, interior clusters by local root and new spin.
    // 8 sites per 16-byte store.
    uint4 *code4 = reinterpret_cast<uint4 *>(code);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int idx = tid + q * NT;
        const int y = (idx * 8) / TW, xb = (idx * 8) % TW;
        if (y >= t.th) continue;
        uint32_t wv[4] = {0u, 0u, 0u, 0u};
        const int c = xb >> 5;
        const uint32_t heads = run_heads(ih_of(y, c));
        const int base = y * PW + 32 * c;
        int slot = -1;            // PCC: border piece of the sites gathered in cols
        uint32_t cols = 0u;
        int info = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int x = xb + e;
            if (x >= t.tw) break;
            // a site inside a run shares the run head's code: look up only
            // where a run starts (and for the group's first site)
            if (e == 0 || ((heads >> (x & 31)) & 1u)) {
                const int v = sm.par[e == 0 ? head_of(heads, base, x & 31) : base + (x & 31)];
                info = ((uint32_t)v >= INFO_INTERIOR) ? v : sm.par[v];   // records: negative or >= INFO_INTERIOR
            }
            wv[e >> 1] |= ((uint32_t)info & 0xFFFFu) << (16 * (e & 1));
            if (pcc && info < 0) {
                // the columns and rows each border piece occupies (only a
                // piece touching the border can belong to a spanning cluster)
                const int sl = info & 0x3FF;
                if (sl != slot) {
                    if (slot >= 0) {
                        atomicOr(&sm.pm[slot][c], cols);
                        atomicOr(&sm.pm[slot][4 + (y >> 5)], 1u << (y & 31));
                    }
                    slot = sl;
                    cols = 0u;
                }
                cols |= 1u << (x & 31);
            }
        }
        if (slot >= 0) {
            atomicOr(&sm.pm[slot][c], cols);
            atomicOr(&sm.pm[slot][4 + (y >> 5)], 1u << (y & 31));
        }
        code4[idx] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
    }
    if (pcc) {
        __syncthreads();
        for (int q = tid; q < S * 8; q += NT) R.pmask[(size_t)t.lt * S * 8 + q] = (&sm.pm[0][0])[q];
    }
    long long c2 = 0;
    if (csz) {
        // every root: an interior cluster adds its |C|^2; a border piece
        // hands its size to its representative node for the merge
        __syncthreads();
        for (int w = tid; w < t.th * TWW; w += NT) {
            const int y = w % t.th, c = w / t.th;
            const int base = y * PW + 32 * c;
            const int vw = min(32, t.tw - 32 * c);
            for (uint32_t bits = run_heads(ih_of(y, c)) & valid_mask(0, vw); bits; bits &= bits - 1) {
                const int v = sm.par[base + __ffs(bits) - 1];
                if (v < 0) {   // piece size: bits 16-30 (bit 31 is the border flag)
                    R.psize[(size_t)t.lt * S + (v & 0x3FF)] = (int32_t)(((uint32_t)v >> 16) & 0x7FFFu);
                } else if ((uint32_t)v >= INFO_INTERIOR) {   // bits 16-29 (bit 30 is the flag)
                    const long long size = ((uint32_t)v >> 16) & 0x3FFFu;
                    c2 += size * size;
                }
            }
        }
    }
    long long v4[4] = {nb, ncl_interior, c2, 0};
    DevObs *o = R.obs + j;
    unsigned long long *const dst[4] = {&o->nbonds, &o->nclusters, &o->csize2, nullptr};
    block_sum_atomic<NT, 4>(v4, dst, sm.u.red);
}

// ------------------------------------------------ union-find with offsets
// Topological rule (Sec. III): a cluster winds around the box when one of
// its cycles has a non-zero net displacement.  Nodes carry their unwrapped
// displacement from their parent; each component is held as a residue mod
// WIND_M, a prime above any lattice side.  A cycle's net displacement is
// (n_x L, n_y L) with |n| <= L, which is zero mod WIND_M only for n = 0.
constexpr uint32_t WIND_M = 65521u;

__device__ __forceinline__ uint32_t wind_off(int dx, int dy)
{
    int x = dx % (int)WIND_M, y = dy % (int)WIND_M;
    x += x < 0 ? (int)WIND_M : 0;
    y += y < 0 ? (int)WIND_M : 0;
    return (uint32_t)x | ((uint32_t)y << 16);
}

__device__ __forceinline__ uint32_t wind_add(uint32_t a, uint32_t b)
{
    uint32_t x = (a & 0xFFFFu) + (b & 0xFFFFu), y = (a >> 16) + (b >> 16);
    x -= x >= WIND_M ? WIND_M : 0u;
    y -= y >= WIND_M ? WIND_M : 0u;
    return x | (y << 16);
}

__device__ __forceinline__ uint32_t wind_neg(uint32_t a)
{
    const uint32_t x = a & 0xFFFFu, y = a >> 16;
    return (x ? WIND_M - x : 0u) | ((y ? WIND_M - y : 0u) << 16);
}

__device__ __forceinline__ unsigned long long wind_link(int parent, uint32_t off)
{
    return (unsigned long long)(uint32_t)parent | ((unsigned long long)off << 32);
}

__device__ __forceinline__ unsigned long long wload(const unsigned long long *p)
{
    return *(const volatile unsigned long long *)p;
}

// Root of x and x's displacement from it, halving the path on the way (a
// node's link only ever moves to an ancestor, with the summed displacement).
__device__ __forceinline__ int wfind(unsigned long long *lk, int x, uint32_t &off)
{
    off = 0u;
    unsigned long long v = wload(lk + x);
    int p = (int)(uint32_t)v;
    while (p != x) {
        const unsigned long long w = wload(lk + p);
        const int gp = (int)(uint32_t)w;
        if (gp != p) {
            const uint32_t o = wind_add((uint32_t)(v >> 32), (uint32_t)(w >> 32));
            *(volatile unsigned long long *)(lk + x) = wind_link(gp, o);
            off = wind_add(off, o);
            x = gp;
        } else {
            off = wind_add(off, (uint32_t)(v >> 32));
            x = p;
        }
        v = wload(lk + x);
        p = (int)(uint32_t)v;
    }
    return x;
}

// Union by key (as gunite_by_key) of the nodes a and b joined by a bond that
// moves by d from a to b.  If they already share a root, the bond closes a
// cycle: a non-zero displacement around it is a winding, recorded in the
// sweep's spans_x / spans_y.
__device__ __forceinline__ void wunite(unsigned long long *lk, const int32_t *key, int a, int b, uint32_t d,
                                       DevObs *o)
{
    for (;;) {
        uint32_t oa, ob;
        const int ra = wfind(lk, a, oa);
        const int rb = wfind(lk, b, ob);
        const uint32_t rel = wind_add(wind_add(oa, d), wind_neg(ob));   // U(rb) - U(ra)
        if (ra == rb) {
            if (rel & 0xFFFFu) atomicOr(&o->spans_x, 1);
            if (rel >> 16) atomicOr(&o->spans_y, 1);
            return;
        }
        int lo = ra, hi = rb;
        uint32_t off = rel;
        if ((uint32_t)key[ra] > (uint32_t)key[rb]) {
            lo = rb;
            hi = ra;
            off = wind_neg(rel);
        }
        const unsigned long long root = (unsigned long long)(uint32_t)hi;   // self link, offset 0
        if (atomicCAS(lk + hi, root, wind_link(lo, off)) == root) return;
    }
}

// ------------------------------------------------------------- merge phase
// Launch shape of the merge kernels: one block per tile (blockIdx.x = the
// tile's index in the tile table) of S/4 threads; thread i takes the slots
// i + q*S/4 (q < 4) and the crossing links i + q*S/4 (q < 2).  The tile's
// lattice, launch and range checks are read once per thread instead of once
// per node, and the loads of a thread's nodes are issued together.
template <int TH>
struct MergeCfg {
    static constexpr int S = Slots<TH>::S;
    static constexpr int MT = S / 4;                    // threads per block
    static constexpr int NPT = 4;                       // slots per thread
    static constexpr int EPT = (TH + TW + MT - 1) / MT; // crossing links per thread
    static_assert(S % 4 == 0 && EPT == 2, "merge launch shape");
};

// The lattice of tile g and its launch index, or null when the tile is idle
// or the lattice has no sweep in this launch (uniform across the block).
__device__ __forceinline__ const Replica *merge_lattice(const SweepArgs &a, int g, int &j)
{
    const int ri = a.tile_rep[g];
    if (ri < 0) return nullptr;
    const Replica *R = a.reps + ri;
    j = lattice_launch(a, *R);
    return (j < 0 || j >= R->nsweeps) ? nullptr : R;
}

// Master step 2 of Sec. II.A: only links between neighbouring domains are
// activated on the "new lattice" of border sites.  Link e < TH joins row e
// of the tile's right column to the left column of the tile to its right;
// link TH + x joins column x of its bottom row to the top row below it.
// W: compiled with the topological rule (lattices with RF_WIND unite their
// nodes with displacements in nlink); every kernel of the merge has it.
template <int TH, bool W>
__global__ void __launch_bounds__(MergeCfg<TH>::MT, 64 / ((MergeCfg<TH>::MT + 31) / 32)) k_merge_union(const SweepArgs a)
{
    using SL = Slots<TH>;
    using MC = MergeCfg<TH>;
    constexpr int S = SL::S;
    int j;
    const Replica *Rp = merge_lattice(a, blockIdx.x, j);
    if (!Rp) return;
    const Replica &R = *Rp;
    const Tile t = tile_of(R, blockIdx.x, TH);
    const uint32_t *cross = R.cross + (size_t)t.lt * CROSS_WORDS;
    int na[MC::EPT], nb[MC::EPT];
    bool prev[MC::EPT];   // the link before it along the edge is bonded too
#pragma unroll
    for (int q = 0; q < MC::EPT; ++q) {
        const int e = threadIdx.x + q * MC::MT;
        na[q] = -1;
        prev[q] = false;
        if (e < TH) {
            if (e < t.th && ((cross[e >> 5] >> (e & 31)) & 1u)) {
                na[q] = t.lt * S + SL::RIGHT + e;
                nb[q] = t.g_right * S + SL::LEFT + e;
                prev[q] = e > 0 && ((cross[(e - 1) >> 5] >> ((e - 1) & 31)) & 1u);
            }
        } else if (e < TH + TW) {
            const int x = e - TH;
            if (x < t.tw && ((cross[TWW + (x >> 5)] >> (x & 31)) & 1u)) {
                na[q] = t.lt * S + SL::BOTTOM + x;
                nb[q] = t.g_down * S + SL::TOP + x;
                prev[q] = x > 0 && ((cross[TWW + ((x - 1) >> 5)] >> ((x - 1) & 31)) & 1u);
            }
        }
    }
    if (W && (R.flags & RF_WIND)) {
        // A link whose two ends lie in the same two pieces as the bonded link
        // just before it along the edge joins nothing new (pieces are known
        // by their keys, which no union changes): skip it.
#pragma unroll
        for (int q = 0; q < MC::EPT; ++q) {
            if (!prev[q]) continue;
            const uint32_t ka = (uint32_t)R.nkey[na[q]] ^ (uint32_t)R.nkey[na[q] - 1];
            const uint32_t kb = (uint32_t)R.nkey[nb[q]] ^ (uint32_t)R.nkey[nb[q] - 1];
            if (((ka | kb) & KEY_MASK) == 0) na[q] = -1;
        }
#pragma unroll
        for (int q = 0; q < MC::EPT; ++q) {
            if (na[q] < 0) continue;
            // a right link moves by (+1, 0), a down link by (0, +1)
            const bool right = threadIdx.x + q * MC::MT < TH;
            wunite(R.nlink, R.nkey, na[q], nb[q], right ? wind_off(1, 0) : wind_off(0, 1), R.obs + j);
        }
        return;
    }
    // The block's links first meet in a small forest in shared memory over
    // the pieces they touch: the tile's own pieces (ids [0, S): a piece's
    // representative slot), the right neighbour's ([S, 2S)) and the lower
    // neighbour's ([2S, 3S)).  Only a link that joins two of those sets there
    // goes on to the global forest; every other link joins pieces that the
    // block's global unions connect already.  A slot's piece: its own slot
    // for a representative (whose parent other blocks may be relinking), else
    // its parent, which is its representative: no find ever passes through a
    // slot that is not a representative, and each such slot ends one link only.
    __shared__ int lp[3 * S];
    for (int i = threadIdx.x; i < 3 * S; i += MC::MT) lp[i] = i;
    int pa[MC::EPT], pb[MC::EPT], ka[MC::EPT], kb[MC::EPT];
#pragma unroll
    for (int q = 0; q < MC::EPT; ++q) {
        if (na[q] < 0) continue;
        pa[q] = gload(R.npar + na[q]);
        pb[q] = gload(R.npar + nb[q]);
        ka[q] = R.nkey[na[q]];
        kb[q] = R.nkey[nb[q]];
    }
    __syncthreads();
    bool live[MC::EPT];
#pragma unroll
    for (int q = 0; q < MC::EPT; ++q) {
        live[q] = false;
        if (na[q] < 0) continue;
        const bool right = threadIdx.x + q * MC::MT < TH;
        const int own = t.lt * S, nbr = (right ? t.g_right : t.g_down) * S;
        const int la = ((uint32_t)ka[q] & KEY_REP) ? na[q] - own : pa[q] - own;
        const int lb = (right ? S : 2 * S) + (((uint32_t)kb[q] & KEY_REP) ? nb[q] - nbr : pb[q] - nbr);
        live[q] = sunite_linked(lp, la, lb);
    }
    // First try, one compare-and-swap: hang the larger-key one of the two
    // pieces' representatives under the other.  Every parent carries a smaller
    // key than its children, so a root of key k holds no node of smaller key:
    // if that representative is still a root, the two sets differ and the
    // link joins them (its new parent need not be a root).
#pragma unroll
    for (int q = 0; q < MC::EPT; ++q) {
        if (!live[q]) continue;
        const bool ra = ((uint32_t)ka[q] & KEY_REP) != 0u, rb = ((uint32_t)kb[q] & KEY_REP) != 0u;
        const int u = ra ? na[q] : pa[q], v = rb ? nb[q] : pb[q];
        const bool u_hi = ((uint32_t)ka[q] & KEY_MASK) > ((uint32_t)kb[q] & KEY_MASK);
        const int hi = u_hi ? u : v, lo = u_hi ? v : u;
        const bool inner = u_hi ? (ra && pa[q] != na[q]) : (rb && pb[q] != nb[q]);
        if (!inner && atomicCAS(R.npar + hi, hi, lo) == hi) live[q] = false;
    }
    // The thread's remaining unions (gunite_by_key's steps) advance in lock
    // step, both finds of every link at once, so their L2 round trips
    // overlap: each pass climbs every find that is not at a root (path
    // splitting: the node it came from is pointed at the parent just read, an
    // ancestor), links two distinct roots by compare-and-swap, the larger key
    // under the smaller (a failed swap climbs on from the root that was
    // linked meanwhile), and loads the parent and key of every current node
    // for the next pass (the first pass uses the loads above).
    int xa[MC::EPT], xb[MC::EPT], sa[MC::EPT], sb[MC::EPT];
#pragma unroll
    for (int q = 0; q < MC::EPT; ++q) {
        xa[q] = na[q];
        xb[q] = nb[q];
        sa[q] = sb[q] = -1;
    }
    for (;;) {
        bool more = false;
#pragma unroll
        for (int q = 0; q < MC::EPT; ++q) {
            if (!live[q]) continue;
            const bool ra = pa[q] == xa[q], rb = pb[q] == xb[q];
            if (!ra || !rb) {
                // path splitting rewrites representatives only: a slot that
                // is not one keeps its own representative as its parent
                if (!ra) {
                    if (sa[q] >= 0) *(volatile int32_t *)(R.npar + sa[q]) = pa[q];
                    sa[q] = ((uint32_t)ka[q] & KEY_REP) ? xa[q] : -1;
                    xa[q] = pa[q];
                }
                if (!rb) {
                    if (sb[q] >= 0) *(volatile int32_t *)(R.npar + sb[q]) = pb[q];
                    sb[q] = ((uint32_t)kb[q] & KEY_REP) ? xb[q] : -1;
                    xb[q] = pb[q];
                }
                more = true;
            } else if (xa[q] == xb[q]) {
                live[q] = false;
            } else {
                const bool a_lo = ka[q] < kb[q];
                const int lo = a_lo ? xa[q] : xb[q], hi = a_lo ? xb[q] : xa[q];
                if (atomicCAS(R.npar + hi, hi, lo) == hi) live[q] = false;
                else more = true;
            }
        }
        if (!more) break;
#pragma unroll
        for (int q = 0; q < MC::EPT; ++q) {
            if (!live[q]) continue;
            pa[q] = gload(R.npar + xa[q]);
            pb[q] = gload(R.npar + xb[q]);
            ka[q] = R.nkey[xa[q]];
            kb[q] = R.nkey[xb[q]];
        }
    }
}

// Topological rule: every node's link before the unions -- its parent from
// the tile kernel (a piece's representative, or itself) and its displacement
// from it, both inside one tile.
template <int TH>
__global__ void __launch_bounds__(MergeCfg<TH>::MT) k_wind_init(const SweepArgs a)
{
    using MC = MergeCfg<TH>;
    int j;
    const Replica *Rp = merge_lattice(a, blockIdx.x, j);
    if (!Rp || !(Rp->flags & RF_WIND)) return;
    const Replica &R = *Rp;
    const Tile t = tile_of(R, blockIdx.x, TH);
    const int base = (blockIdx.x - R.tile_base) * MC::S;
#pragma unroll
    for (int q = 0; q < MC::NPT; ++q) {
        const int s = threadIdx.x + q * MC::MT, n = base + s;
        const int p = R.npar[n];
        uint32_t off = 0u;
        int site, rsite;
        if (p != n && slot_site<TH>(s, t.tw, t.th, site) && slot_site<TH>(p - base, t.tw, t.th, rsite))
            off = wind_off(site % TW - rsite % TW, site / TW - rsite / TW);
        R.nlink[n] = wind_link(p, off);
    }
}

// Pointer jumping over the representatives (every parent replaced by its
// grandparent, MERGE_JUMP_ROUNDS times) between the unions and the
// resolve: it cuts the depth of the chains that unions across many tiles
// leave behind.  The rounds run in one launch, so a round may read a parent
// that its own thread has already moved up; every value read is still an
// ancestor, and the resolve kernel walks to the root whatever depth is left.
// One round is best since the unions split their paths (L=16384, 64-row
// tiles, merge per sweep with 0 / 1 / 2 / 3 rounds: 0.31 / 0.28 / 0.29 / 0.34
// ms at T_c, 0.45 / 0.50 / 0.59 ms for 1 / 2 / 3 rounds at T = 2.0).
// Other slots keep their piece's representative as parent.
constexpr int MERGE_JUMP_ROUNDS = 1;
template <int TH, bool W>
__global__ void __launch_bounds__(MergeCfg<TH>::MT) k_merge_jump(const SweepArgs a)
{
    using MC = MergeCfg<TH>;
    int j;
    const Replica *Rp = merge_lattice(a, blockIdx.x, j);
    if (!Rp) return;
    const Replica &R = *Rp;
    const int base = (blockIdx.x - R.tile_base) * MC::S;   // the lattice's own nodes
    if (W && (R.flags & RF_WIND)) {
        for (int r = 0; r < MERGE_JUMP_ROUNDS; ++r) {
            unsigned long long v[MC::NPT], w[MC::NPT];
#pragma unroll
            for (int q = 0; q < MC::NPT; ++q)
                v[q] = ((uint32_t)R.nkey[base + threadIdx.x + q * MC::MT] & KEY_REP)
                           ? wload(R.nlink + base + threadIdx.x + q * MC::MT) : ~0ull;
#pragma unroll
            for (int q = 0; q < MC::NPT; ++q) w[q] = v[q] != ~0ull ? wload(R.nlink + (uint32_t)v[q]) : ~0ull;
#pragma unroll
            for (int q = 0; q < MC::NPT; ++q)
                if (v[q] != ~0ull && (uint32_t)w[q] != (uint32_t)v[q])
                    *(volatile unsigned long long *)(R.nlink + base + threadIdx.x + q * MC::MT) =
                        wind_link((int)(uint32_t)w[q], wind_add((uint32_t)(v[q] >> 32), (uint32_t)(w[q] >> 32)));
        }
        return;
    }
    uint32_t key[MC::NPT];
    int p[MC::NPT], gp[MC::NPT];
#pragma unroll
    for (int q = 0; q < MC::NPT; ++q) key[q] = (uint32_t)R.nkey[base + threadIdx.x + q * MC::MT];
#pragma unroll
    for (int q = 0; q < MC::NPT; ++q) {   // loaded with the key, not after it: one round trip less
        const int pq = gload(R.npar + base + threadIdx.x + q * MC::MT);
        p[q] = (key[q] & KEY_REP) ? pq : -1;
    }
    for (int r = 0; r < MERGE_JUMP_ROUNDS; ++r) {
#pragma unroll
        for (int q = 0; q < MC::NPT; ++q) gp[q] = p[q] >= 0 ? gload(R.npar + p[q]) : -1;
#pragma unroll
        for (int q = 0; q < MC::NPT; ++q) {
            if (gp[q] != p[q]) *(volatile int32_t *)(R.npar + base + threadIdx.x + q * MC::MT) = gp[q];
            p[q] = gp[q];
        }
    }
}

// Resolve every node once the unions are done: each representative walks to
// its root r (key: the cluster's minimum site index), for PCC lattices writes
// r over every node of the walk (full path compression: no union happens any
// more, so every node on it has root r) and stores the cluster's root and new spin,
// bit (root mod 128) of Philox(root/128, k, SPIN) (Sec. I step 3); a top or
// left slot that is not a representative then copies its representative's.
// Counts the clusters that touch a tile border (one root node each).
template <int TH, bool W>
__global__ void __launch_bounds__(MergeCfg<TH>::MT) k_merge_resolve(const SweepArgs a)
{
    using MC = MergeCfg<TH>;
    int j;
    const Replica *Rp = merge_lattice(a, blockIdx.x, j);
    if (!Rp) return;
    const Replica &R = *Rp;
    const int base = (blockIdx.x - R.tile_base) * MC::S;
    const bool wind = W && (R.flags & RF_WIND);   // the forest lives in nlink
    auto parent = [&](int x) { return wind ? (int)(uint32_t)wload(R.nlink + x) : gload(R.npar + x); };
    uint32_t key[MC::NPT];
    int r[MC::NPT], p[MC::NPT];
#pragma unroll
    for (int q = 0; q < MC::NPT; ++q) key[q] = (uint32_t)R.nkey[base + threadIdx.x + q * MC::MT];
#pragma unroll
    for (int q = 0; q < MC::NPT; ++q) {
        r[q] = base + threadIdx.x + q * MC::MT;
        // a representative walks its forest; any other slot keeps its parent
        // from the tile kernel (its representative) for the copy below
        p[q] = (wind && (key[q] & KEY_REP)) ? parent(r[q]) : gload(R.npar + r[q]);
    }
    // the walks of the thread's representatives advance in lock step
    for (;;) {
        bool more = false;
#pragma unroll
        for (int q = 0; q < MC::NPT; ++q) {
            if ((key[q] & KEY_REP) && p[q] != r[q]) {
                r[q] = p[q];
                more = true;
            }
        }
        if (!more) break;
#pragma unroll
        for (int q = 0; q < MC::NPT; ++q)
            if (key[q] & KEY_REP) p[q] = parent(r[q]);
    }
    __shared__ uint32_t rfin[MC::S];   // the finals of the representatives
    uint32_t rkey[MC::NPT];
#pragma unroll
    for (int q = 0; q < MC::NPT; ++q) rkey[q] = (key[q] & KEY_REP) ? (uint32_t)R.nkey[r[q]] & KEY_MASK : 0u;
    const uint64_t k = R.sweep0 + (uint64_t)j;
    int nroots = 0;
#pragma unroll
    for (int q = 0; q < MC::NPT; ++q) {
        const int n = base + threadIdx.x + q * MC::MT;
        if (key[q] & KEY_REP) {
            if (wind) {
                // displacement from the root along the walk, then every link
                // of the walk rewritten to the root with its own displacement
                uint32_t tot = 0u;
                for (int x = n; x != r[q];) {
                    const unsigned long long v = wload(R.nlink + x);
                    tot = wind_add(tot, (uint32_t)(v >> 32));
                    x = (int)(uint32_t)v;
                }
                for (int x = n; x != r[q];) {
                    const unsigned long long v = wload(R.nlink + x);
                    *(volatile unsigned long long *)(R.nlink + x) = wind_link(r[q], tot);
                    tot = wind_add(tot, wind_neg((uint32_t)(v >> 32)));
                    x = (int)(uint32_t)v;
                }
            } else if (R.flags & RF_PCC) {
                // the PCC kernels that follow read a representative's root
                // straight from its parent; no other kernel reads the forest
                // again before the next tile launch rewrites it
                for (int x = n; x != r[q];) {
                    const int nx = gload(R.npar + x);
                    *(volatile int32_t *)(R.npar + x) = r[q];
                    x = nx;
                }
            }
            nroots += r[q] == n;
            if (R.flags & RF_CSIZE) atomicAdd(R.csize + r[q], R.psize[n]);
            const U4 u = stream_block(R, rkey[q] >> 7, k, STREAM_SPIN);
            const int bit = rkey[q] & 127;
            const uint32_t spin = (u4_word(u, bit >> 5) >> (bit & 31)) & 1u;
            R.nfinal[n] = rkey[q] | (spin ? FINAL_SPIN : 0u);
            rfin[threadIdx.x + q * MC::MT] = R.nfinal[n];
        }
    }
    __syncthreads();
    // a top or left slot that is not a representative, whose final a
    // neighbour's tile kernel reads for its halo: its representative's (its
    // parent since the tile kernel, in this tile: the unions rewrite
    // representatives only); past the tile's sites, 0.  No kernel reads the
    // final of any other slot that is not a representative.
#pragma unroll
    for (int q = 0; q < MC::NPT; ++q) {
        const int s = threadIdx.x + q * MC::MT;
        if (!(key[q] & KEY_REP) && (s < Slots<TH>::BOTTOM || (s >= Slots<TH>::LEFT && s < Slots<TH>::RIGHT)))
            R.nfinal[base + s] = key[q] == KEY_NONE ? 0u : rfin[p[q] - base];
    }
    // every thread of the block gets here; the last warp may be partial
    const int wb = threadIdx.x & ~31;
    const unsigned wm = MC::MT - wb >= 32 ? 0xFFFFFFFFu : (1u << (MC::MT - wb)) - 1u;
    nroots = __reduce_add_sync(wm, nroots);
    if ((threadIdx.x & 31) == 0 && nroots) atomicAdd(&R.obs[j].nclusters, (unsigned long long)nroots);
}

// ------------------------------------------------------------------- PCC
// Extension rule under periodic boundaries (Sec. III): a cluster spans x
// iff its projection on the x axis, the range P_x(C), is all of [0, L-1],
// i.e. iff it occupies every column (likewise y and rows).  Each tile
// recorded, per border piece, the columns and rows it occupies; here the
// pieces of one global cluster are united (the paper's update of P_x on a
// merge) as bit sets per tile column (tile row).
//
// Step 1: candidates.  A cluster occupying every column holds a site of
// column 0, on the left edge of a tile of tile column 0; one occupying every
// row holds a site of row 0, on the top edge of a tile of tile row 0.  Those
// edge nodes' roots get compact candidate ids (cid = id + 2).
template <int TH>
__global__ void k_pcc_candidates(const SweepArgs a)
{
    using SL = Slots<TH>;
    constexpr int S = SL::S;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)a.n_tiles * (TH + TW)) return;
    const int g = (int)(idx / (TH + TW));
    const int e = (int)(idx % (TH + TW));
    const int ri = a.tile_rep[g];
    if (ri < 0) return;
    const Replica &R = a.reps[ri];
    const int j = lattice_launch(a, R);
    if (!(R.flags & RF_PCC) || (R.flags & RF_WIND) || j < 0 || j >= R.nsweeps) return;
    const Tile t = tile_of(R, g, TH);
    int axis, node;
    if (e < TH) {
        if (t.tx != 0 || e >= t.th) return;
        axis = 0;
        node = t.lt * S + SL::LEFT + e;
    } else {
        const int x = e - TH;
        if (t.ty != 0 || x >= t.tw) return;
        axis = 1;
        node = t.lt * S + SL::TOP + x;
    }
    int r = gload(R.npar + node);
    if (!((uint32_t)R.nkey[node] & KEY_REP)) r = gload(R.npar + r);   // via the representative
    int32_t *c = R.cid + (size_t)r * 2 + axis;
    if (atomicCAS(c, 0, 1) == 0) {
        const int id = atomicAdd(R.ncand + axis, 1);   // < L: at most one per edge site
        R.cand[axis * R.L + id] = r;
        *(volatile int32_t *)c = id + 2;
    }
}

// Step 2: every border piece ORs the columns (rows) it occupies into its
// candidate cluster's coverage of the piece's tile column (tile row).
template <int TH>
__global__ void k_pcc_cover(const SweepArgs a)
{
    constexpr int S = Slots<TH>::S;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (int64_t)a.n_tiles * S) return;
    const int g = (int)(n / S);
    const int ri = a.tile_rep[g];
    if (ri < 0) return;
    const Replica &R = a.reps[ri];
    const int j = lattice_launch(a, R);
    if (!(R.flags & RF_PCC) || (R.flags & RF_WIND) || j < 0 || j >= R.nsweeps) return;
    const int64_t nl = n - (int64_t)R.tile_base * S;   // the lattice's own node
    const uint4 *pm4 = reinterpret_cast<const uint4 *>(R.pmask + (size_t)nl * 8);
    const uint4 c4 = pm4[0], r4 = pm4[1];
    if (!(c4.x | c4.y | c4.z | c4.w | r4.x | r4.y | r4.z | r4.w)) return;
    const int r = gload(R.npar + nl);
    const Tile t = tile_of(R, g, TH);
    const int cx = R.cid[(size_t)r * 2 + 0], cy = R.cid[(size_t)r * 2 + 1];
    if (cx >= 2) {
        uint32_t *cov = R.cov + ((size_t)(cx - 2) * R.tiles_x + t.tx) * 4;
        const uint32_t w[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (w[q]) atomicOr(cov + q, w[q]);
    }
    if (cy >= 2) {
        uint32_t *cov = R.cov + (size_t)R.L * R.tiles_x * 4 + ((size_t)(cy - 2) * R.tiles_y + t.ty) * 4;
        const uint32_t w[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (w[q]) atomicOr(cov + q, w[q]);
    }
}

// Step 3 (PCC_DECIDE_BLOCKS blocks per lattice, blockIdx.y = the lattice): a
// candidate spans x iff its coverage of every tile column is that column's
// full mask (P_x(C) = [0, L-1]); y alike.  Each block checks its share of the
// candidates, clears their scratch and ORs what it found into the sweep's
// spans_x / spans_y; the lattice's last block to finish (a counter, ncand[2],
// taken after a fence: no block waits for another) applies the PCC feedback
// to the threshold for the next sweep -- down by delta_k if the clusters
// percolate, up otherwise, delta_k = 2^(32 - min(8 + floor(k/1000), 20)),
// clamped to [0, 2^32] -- and resets the counts.  Under the topological rule
// (RF_WIND) there are no candidates: the flags are the windings the unions
// recorded.
constexpr int PCC_DECIDE_BLOCKS = 8;
template <int TH>
__global__ void k_pcc_decide(const SweepArgs a, int n_reps)
{
    const int rr = blockIdx.y;
    if (rr >= n_reps) return;
    const Replica &R = a.reps[rr];
    if (R.L <= 0) return;                  // unused slot of a batch
    const int j = lattice_launch(a, R);
    if (!(R.flags & RF_PCC) || j < 0 || j >= R.nsweeps) return;
    const int nx = R.ncand[0], ny = R.ncand[1];
    uint32_t *covx = R.cov;
    uint32_t *covy = R.cov + (size_t)R.L * R.tiles_x * 4;
    // block b takes a contiguous range of each axis's candidates: checks stop
    // at the first tile column (row) a candidate does not cover, and the
    // range's coverage is cleared with coalesced stores afterwards
    const int cx = (nx + gridDim.x - 1) / gridDim.x, cy = (ny + gridDim.x - 1) / gridDim.x;
    const int x0 = blockIdx.x * cx, x1 = min(nx, x0 + cx);
    const int y0 = blockIdx.x * cy, y1 = min(ny, y0 + cy);
    int sx = 0, sy = 0;
    for (int id = x0 + threadIdx.x; id < x1; id += blockDim.x) {
        bool full = true;
        for (int tx = 0; tx < R.tiles_x && full; ++tx) {
            const int tw = min(TW, R.L - TW * tx);
            const uint32_t *cv = covx + ((size_t)id * R.tiles_x + tx) * 4;
            for (int q = 0; q < 4; ++q) {
                const uint32_t m = valid_mask(q, tw);
                full &= (cv[q] & m) == m;
            }
        }
        sx |= full;
        R.cid[(size_t)R.cand[id] * 2 + 0] = 0;
    }
    for (int id = y0 + threadIdx.x; id < y1; id += blockDim.x) {
        bool full = true;
        for (int ty = 0; ty < R.tiles_y && full; ++ty) {
            const int th = min(TH, R.L - TH * ty);
            const uint32_t *cv = covy + ((size_t)id * R.tiles_y + ty) * 4;
            for (int q = 0; q < 4; ++q) {
                const uint32_t m = valid_mask(q, th);
                full &= (cv[q] & m) == m;
            }
        }
        sy |= full;
        R.cid[(size_t)R.cand[R.L + id] * 2 + 1] = 0;
    }
    __syncthreads();   // every check of this block's range has read its coverage
    for (int64_t q = (int64_t)x0 * R.tiles_x * 4 + threadIdx.x; q < (int64_t)x1 * R.tiles_x * 4; q += blockDim.x)
        covx[q] = 0u;
    for (int64_t q = (int64_t)y0 * R.tiles_y * 4 + threadIdx.x; q < (int64_t)y1 * R.tiles_y * 4; q += blockDim.x)
        covy[q] = 0u;
    sx = __syncthreads_or(sx);
    sy = __syncthreads_or(sy);
    if (threadIdx.x != 0) return;
    DevObs &o = R.obs[j];
    if (sx) atomicOr(&o.spans_x, 1);
    if (sy) atomicOr(&o.spans_y, 1);
    __threadfence();
    if (atomicAdd(R.ncand + 2, 1) != (int)gridDim.x - 1) return;
    // the last block: every other block's flags are visible
    __threadfence();
    const int fx = *(volatile int32_t *)&o.spans_x, fy = *(volatile int32_t *)&o.spans_y;
    const uint64_t k = R.sweep0 + (uint64_t)j;
    const uint64_t e = 8 + k / 1000;
    const uint64_t delta = (uint64_t)1 << (32 - (e < 20 ? e : 20));
    const uint64_t top = (uint64_t)1 << 32;
    const uint64_t t = *R.thr_dev;
    *R.thr_dev = (fx || fy) ? (t > delta ? t - delta : 0) : (t + delta < top ? t + delta : top);
    R.ncand[0] = 0;
    R.ncand[1] = 0;
    R.ncand[2] = 0;
}

// ------------------------------------------------------------ small kernels
// Hot start: s_i = bit (i mod 128) of Philox(i/128, 0, INIT).
static __global__ void k_hot_start(uint8_t *spin, int64_t N, uint32_t key0, uint32_t key1)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const U4 r = philox4x32_10((uint32_t)(i >> 7), 0u, 0u, STREAM_INIT, key0, key1);
    const int bit = (int)(i & 127);
    spin[i] = (uint8_t)((u4_word(r, bit >> 5) >> (bit & 31)) & 1u);
}

// A served lattice's initial device state in one launch: the hot start, zero
// observables (n_obs 8-byte words) and the threshold word.
static __global__ void k_job_init(uint8_t *spin, int64_t N, uint32_t key0, uint32_t key1,
                                  unsigned long long *obs, int64_t n_obs, uint64_t *thr_dev, uint64_t thr)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        const U4 r = philox4x32_10((uint32_t)(i >> 7), 0u, 0u, STREAM_INIT, key0, key1);
        const int bit = (int)(i & 127);
        spin[i] = (uint8_t)((u4_word(r, bit >> 5) >> (bit & 31)) & 1u);
    }
    if (i < n_obs) obs[i] = 0ull;
    if (i == 0) *thr_dev = thr;
}

// Integer ceiling of the bond step: nblocks BOND-stream Philox blocks
// (counters 0 .. nblocks-1 of sweep 0), four in flight per thread as in the
// tile kernel's bond draws, all words xored together and into *out so that
// no draw can be dropped.  A grid-stride loop over a grid that fills the SMs.
static __global__ void __launch_bounds__(256) k_philox_rate(int64_t nblocks, uint32_t key0, uint32_t key1,
                                                            uint32_t *out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0u;
    for (; i + 3 * stride < nblocks; i += 4 * stride) {
        const U4 r0 = philox4x32_10((uint32_t)i, 0u, 0u, STREAM_BOND, key0, key1);
        const U4 r1 = philox4x32_10((uint32_t)(i + stride), 0u, 0u, STREAM_BOND, key0, key1);
        const U4 r2 = philox4x32_10((uint32_t)(i + 2 * stride), 0u, 0u, STREAM_BOND, key0, key1);
        const U4 r3 = philox4x32_10((uint32_t)(i + 3 * stride), 0u, 0u, STREAM_BOND, key0, key1);
        acc ^= r0.x ^ r0.y ^ r0.z ^ r0.w ^ r1.x ^ r1.y ^ r1.z ^ r1.w;
        acc ^= r2.x ^ r2.y ^ r2.z ^ r2.w ^ r3.x ^ r3.y ^ r3.z ^ r3.w;
    }
    for (; i < nblocks; i += stride) {
        const U4 r = philox4x32_10((uint32_t)i, 0u, 0u, STREAM_BOND, key0, key1);
        acc ^= r.x ^ r.y ^ r.z ^ r.w;
    }
    acc = __reduce_xor_sync(0xFFFFFFFFu, acc);
    if ((threadIdx.x & 31) == 0) atomicXor(out, acc);
}

// L2 copy ceiling: reps passes of dst[i] = src[i] ^ pass over n 16-byte
// words, loads and stores cached in L2 only (ld/st .cg), so a working set
// that fits L2 is read and written there after the first pass.
static __global__ void __launch_bounds__(256) k_l2_rate(const uint4 *src, uint4 *dst, int64_t n, int32_t reps)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int32_t r = 0; r < reps; ++r) {
        for (int64_t i = i0; i < n; i += stride) {
            uint4 v = __ldcg(src + i);
            v.x ^= (uint32_t)r;
            __stcg(dst + i, v);
        }
    }
}

// Sets *bad if any of the n bytes is not 0 or 1.
static __global__ void k_check_spins(const uint8_t *p, int64_t n, int32_t *bad)
{
    int found = 0;
    const int64_t n16 = n / 16;
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 v = q[i];
        found |= ((v.x | v.y | v.z | v.w) & 0xFEFEFEFEu) != 0u;
    }
    for (int64_t i = n16 * 16 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        found |= p[i] > 1;
    if (__syncthreads_or(found) && threadIdx.x == 0) atomicOr(bad, 1);
}

// Bond bits of the last sweep (tile-major words) -> row-major bond bytes.
template <int TH>
__global__ void k_bond_bytes(const uint32_t *bondbits, int L, int tiles_x, uint8_t *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)L * L) return;
    const int y = (int)(i / L), x = (int)(i % L);
    const int tx = x / TW, ty = y / TH, lx = x % TW, ly = y % TH;
    const size_t g = (size_t)ty * tiles_x + tx;
    const uint32_t *bb = bondbits + g * TH * 2 * TWW + (size_t)ly * 2 * TWW;
    const uint32_t h = (bb[lx >> 5] >> (lx & 31)) & 1u;
    const uint32_t v = (bb[TWW + (lx >> 5)] >> (lx & 31)) & 1u;
    out[i] = (uint8_t)(h | (v << 1));
}

}  // namespace swg
