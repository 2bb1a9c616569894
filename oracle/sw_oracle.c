/*
 * sw_oracle.c -- plain, single-threaded CPU oracle of one Swendsen-Wang sweep
 * of the periodic 2D Ising model and of the PCC feedback built on it.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the package smoke check and
 * the benchmark's CPU-baseline leg, never by the product path.  It shares no
 * code with the CUDA path.
 *
 * Every function states what the method computes in the most direct way
 * available; nothing here is blocked, fused or reordered for speed.
 *
 * Paper: S. Lin and B. Zheng, "Two Parallel Swendsen-Wang Cluster Algorithms
 * Using Message-Passing Paradigm" (arXiv:0808.2109):
 *   Sec. I, steps 1-4      -- the Swendsen-Wang update (bond, cluster, flip);
 *   Sec. II.A slave step 1 -- Hoshen-Kopelman cluster counting;
 *   Sec. II.B steps 4-6    -- the smaller label wins: root = minimum index;
 *   Sec. III               -- extension rule, range operator under PBC;
 *   Sec. I (PCC, cited)    -- feedback on the bond probability.
 */
#include "sw_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon et al., SC'11, Sec. 3: the Philox S-box is two
 * 32x32->64 multiplications whose high halves are xored with the other two
 * counter words and the key; the key is bumped by a Weyl sequence between
 * rounds).
 * ---------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0;
    c[1] = n1;
    c[2] = n2;
    c[3] = n3;
}

void swo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k[0] += PHILOX_W0;
            k[1] += PHILOX_W1;
        }
        philox_round(c, k);
    }
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
    out[3] = c[3];
}

void swo_philox_batch(int64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    for (int64_t i = 0; i < n; i++)
        swo_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

/* One Philox block of the method's streams: counter (word, k lo, k hi, stream). */
static void stream_block(uint64_t seed, uint64_t word, uint64_t sweep, uint32_t stream,
                         uint32_t out[4])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)word, (uint32_t)sweep, (uint32_t)(sweep >> 32), stream};
    swo_philox4x32_10(ctr, key, out);
}

/* Bit b (0..127) of a 128-bit block: bit (b mod 32) of word floor(b/32). */
static int block_bit(const uint32_t w[4], uint64_t b)
{
    return (int)((w[b / 32] >> (b % 32)) & 1u);
}

/* ------------------------------------------------------------------------
 * Bond probability (Sec. I step 1): P = 1 - exp(-2J/T), held as the integer
 * threshold t = floor(P * 2^32); a link with uniform 32-bit word u is
 * activated iff u < t.  P = 0 never bonds and P = 1 (t = 2^32) always does.
 * ---------------------------------------------------------------------- */
uint64_t swo_threshold_p(double p)
{
    if (!(p > 0.0))
        return 0;
    if (p >= 1.0)
        return (uint64_t)1 << 32;
    return (uint64_t)floor(ldexp(p, 32));
}

uint64_t swo_threshold_T(double J, double T)
{
    double P = 1.0 - exp(-2.0 * J / T);
    return swo_threshold_p(P);
}

/* ------------------------------------------------------------------------
 * Hot start: every spin an independent fair bit of the INIT stream.
 * ---------------------------------------------------------------------- */
void swo_hot_start(int32_t L, uint64_t seed, uint8_t *spin)
{
    uint64_t N = (uint64_t)L * (uint64_t)L;
    for (uint64_t i = 0; i < N; i++) {
        uint32_t w[4];
        stream_block(seed, i / 128, 0, SWO_STREAM_INIT, w);
        spin[i] = (uint8_t)block_bit(w, i % 128);
    }
}

/* Neighbour of site i across its link d (periodic). */
static uint64_t neighbour(int32_t L, uint64_t i, int d)
{
    uint64_t x = i % (uint64_t)L, y = i / (uint64_t)L;
    if (d == 0)
        return y * (uint64_t)L + (x + 1) % (uint64_t)L;
    return ((y + 1) % (uint64_t)L) * (uint64_t)L + x;
}

/* Does link d of site i exist?  Under periodic boundaries every link does;
 * under open boundaries (Sec. III) the right link of the last column and the
 * down link of the last row leave the lattice and do not exist. */
static int link_exists(int32_t L, uint64_t i, int d, int32_t open)
{
    if (!open)
        return 1;
    uint64_t x = i % (uint64_t)L, y = i / (uint64_t)L;
    return d == 0 ? x + 1 < (uint64_t)L : y + 1 < (uint64_t)L;
}

/* ------------------------------------------------------------------------
 * Step 1 (Sec. I; also DPM step 1 of Sec. II.B): traverse every link; a link
 * between equal spins becomes a bond with probability P.  Link l = 2i + d
 * draws word (l mod 4) of Philox(floor(l/4), k, BOND).
 * ---------------------------------------------------------------------- */
int64_t swo_bonds(int32_t L, uint64_t seed, uint64_t sweep, uint64_t thr,
                  const uint8_t *spin, uint8_t *bond, int32_t open)
{
    uint64_t N = (uint64_t)L * (uint64_t)L;
    int64_t nb = 0;
    for (uint64_t i = 0; i < N; i++) {
        uint8_t b = 0;
        for (int d = 0; d < 2; d++) {
            if (!link_exists(L, i, d, open))
                continue;
            uint64_t j = neighbour(L, i, d);
            uint64_t l = 2 * i + (uint64_t)d;
            uint32_t w[4];
            stream_block(seed, l / 4, sweep, SWO_STREAM_BOND, w);
            if (spin[i] == spin[j] && (uint64_t)w[l % 4] < thr) {
                b |= (uint8_t)(1u << d);
                nb++;
            }
        }
        bond[i] = b;
    }
    return nb;
}

/* ------------------------------------------------------------------------
 * Step 2 (Sec. I): two spins are in one cluster iff a path of bonds joins
 * them.  Hoshen-Kopelman (Sec. II.A slave step 1): a raster scan in which
 * each site looks back at its left and upper neighbour and records label
 * equivalences in a union-find forest; the periodic wrap links are joined
 * after the scan.  Unions always hang the larger root under the smaller, so
 * every root is the minimum site index of its cluster: the smaller label
 * wins, as in the DPM label exchange (Sec. II.B steps 4-6).
 * ---------------------------------------------------------------------- */
static int32_t uf_find(int32_t *parent, int32_t a)
{
    int32_t r = a;
    while (parent[r] != r)
        r = parent[r];
    while (parent[a] != r) { /* path compression: does not change any root */
        int32_t next = parent[a];
        parent[a] = r;
        a = next;
    }
    return r;
}

static void uf_unite(int32_t *parent, int32_t a, int32_t b)
{
    int32_t ra = uf_find(parent, a), rb = uf_find(parent, b);
    if (ra < rb)
        parent[rb] = ra;
    else if (rb < ra)
        parent[ra] = rb;
}

int64_t swo_label(int32_t L, const uint8_t *bond, int32_t *label)
{
    int64_t N = (int64_t)L * (int64_t)L;
    for (int64_t i = 0; i < N; i++)
        label[i] = (int32_t)i;
    /* raster scan over the links that do not wrap */
    for (int64_t y = 0; y < L; y++) {
        for (int64_t x = 0; x < L; x++) {
            int64_t i = y * L + x;
            if (x > 0 && (bond[i - 1] & 1u))
                uf_unite(label, (int32_t)(i - 1), (int32_t)i);
            if (y > 0 && (bond[i - L] & 2u))
                uf_unite(label, (int32_t)(i - L), (int32_t)i);
        }
    }
    /* periodic wrap links: right edge -> column 0, bottom edge -> row 0 */
    for (int64_t y = 0; y < L; y++) {
        int64_t i = y * L + (L - 1);
        if (bond[i] & 1u)
            uf_unite(label, (int32_t)i, (int32_t)(y * L));
    }
    for (int64_t x = 0; x < L; x++) {
        int64_t i = (int64_t)(L - 1) * L + x;
        if (bond[i] & 2u)
            uf_unite(label, (int32_t)i, (int32_t)x);
    }
    int64_t nclusters = 0;
    for (int64_t i = 0; i < N; i++) {
        label[i] = uf_find(label, (int32_t)i);
        if (label[i] == i)
            nclusters++;
    }
    return nclusters;
}

void swo_count_clusters_batch(int32_t L, int64_t nsets, const uint8_t *bonds, int64_t *counts)
{
    int64_t N = (int64_t)L * (int64_t)L;
    int32_t *label = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    if (!label) {
        for (int64_t s = 0; s < nsets; s++)
            counts[s] = -1;
        return;
    }
    for (int64_t s = 0; s < nsets; s++)
        counts[s] = swo_label(L, bonds + s * N, label);
    free(label);
}

/* ------------------------------------------------------------------------
 * Step 3 (Sec. I): every cluster gets one new random spin, shared by all of
 * its sites; the old spin is not used.  The bit is keyed by the cluster's
 * root r: bit (r mod 128) of Philox(floor(r/128), k, SPIN).
 * ---------------------------------------------------------------------- */
void swo_assign(int32_t L, uint64_t seed, uint64_t sweep, const int32_t *label, uint8_t *spin)
{
    uint64_t N = (uint64_t)L * (uint64_t)L;
    for (uint64_t i = 0; i < N; i++) {
        uint64_t r = (uint64_t)label[i];
        uint32_t w[4];
        stream_block(seed, r / 128, sweep, SWO_STREAM_SPIN, w);
        spin[i] = (uint8_t)block_bit(w, r % 128);
    }
}

/* Sum of |C|^2 over the clusters: count the sites of every root, then sum
 * the squares of the counts. */
int64_t swo_csize2(int32_t L, const int32_t *label)
{
    int64_t N = (int64_t)L * (int64_t)L;
    int64_t *count = (int64_t *)calloc((size_t)N, sizeof(int64_t));
    if (!count)
        return -1;
    for (int64_t i = 0; i < N; i++)
        count[label[i]]++;
    int64_t s = 0;
    for (int64_t r = 0; r < N; r++)
        s += count[r] * count[r];
    free(count);
    return s;
}

/* Energy E = -J * bond_sum with bond_sum = sum over links of sigma_i sigma_j
 * (the Hamiltonian of Sec. I), magnetisation M = sum of sigma_i. */
void swo_measure(int32_t L, const uint8_t *spin, int32_t open, int64_t *bond_sum, int64_t *mag)
{
    uint64_t N = (uint64_t)L * (uint64_t)L;
    int64_t bs = 0, m = 0;
    for (uint64_t i = 0; i < N; i++) {
        int64_t si = 2 * (int64_t)spin[i] - 1;
        m += si;
        for (int d = 0; d < 2; d++) {
            if (!link_exists(L, i, d, open))
                continue;
            int64_t sj = 2 * (int64_t)spin[neighbour(L, i, d)] - 1;
            bs += si * sj;
        }
    }
    *bond_sum = bs;
    *mag = m;
}

/* ------------------------------------------------------------------------
 * Extension rule under periodic boundaries (Sec. III): project every cluster
 * onto the x axis (and the y axis); it spans x iff its projection P_x(C) is
 * the whole range [0, L-1], i.e. iff it occupies every one of the L columns.
 * Each cluster's number of distinct columns is counted by scanning column by
 * column and stamping each root with the last column it was seen in.
 * ---------------------------------------------------------------------- */
static int32_t spans_axis(int32_t L, const int32_t *label, int32_t *stamp, int32_t *count,
                          int columns)
{
    int64_t N = (int64_t)L * (int64_t)L;
    for (int64_t i = 0; i < N; i++) {
        stamp[i] = -1;
        count[i] = 0;
    }
    int32_t spans = 0;
    for (int32_t a = 0; a < L; a++) {         /* the line: column a (or row a) */
        for (int32_t b = 0; b < L; b++) {     /* the sites along that line     */
            int64_t i = columns ? (int64_t)b * L + a : (int64_t)a * L + b;
            int32_t r = label[i];
            if (stamp[r] != a) {
                stamp[r] = a;
                count[r]++;
                if (count[r] == L)
                    spans = 1;
            }
        }
    }
    return spans;
}

int swo_spans(int32_t L, const int32_t *label, int32_t *spans_x, int32_t *spans_y)
{
    int64_t N = (int64_t)L * (int64_t)L;
    int32_t *stamp = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *count = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    if (!stamp || !count) {
        free(stamp);
        free(count);
        return -1;
    }
    *spans_x = spans_axis(L, label, stamp, count, 1);
    *spans_y = spans_axis(L, label, stamp, count, 0);
    free(stamp);
    free(count);
    return 0;
}

/* ------------------------------------------------------------------------
 * Topological rule (Sec. III): a cluster percolates in x if it winds around
 * the box in x, i.e. holds a closed path of bonds whose net displacement in
 * x is a non-zero multiple of L (likewise y).  Each cluster is explored
 * breadth first, giving every site an unwrapped position (its start at 0,
 * each bond moving by one lattice step); a bond that reaches an explored
 * site at a position other than the one it predicts closes a cycle whose
 * displacement is that difference.  Every cycle is a sum of such cycles, so
 * a winding cluster always shows one.
 * ---------------------------------------------------------------------- */
int swo_windings(int32_t L, const uint8_t *bond, int32_t *wraps_x, int32_t *wraps_y)
{
    int64_t N = (int64_t)L * (int64_t)L;
    int64_t *ux = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int64_t *uy = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    uint8_t *seen = (uint8_t *)calloc((size_t)N, 1);
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    if (!ux || !uy || !seen || !queue) {
        free(ux);
        free(uy);
        free(seen);
        free(queue);
        return -1;
    }
    *wraps_x = 0;
    *wraps_y = 0;
    for (int64_t s = 0; s < N; s++) {
        if (seen[s])
            continue;
        int64_t head = 0, tail = 0;
        seen[s] = 1;
        ux[s] = 0;
        uy[s] = 0;
        queue[tail++] = s;
        while (head < tail) {
            int64_t i = queue[head++];
            int64_t x = i % L, y = i / L;
            /* the four links at site i: its own right and down links, and the
             * right link of its left neighbour and the down link of the site
             * above (each a bond or not) */
            int64_t nb[4], dx[4], dy[4];
            int has[4];
            nb[0] = y * L + (x + 1) % L;       dx[0] = 1;  dy[0] = 0;  has[0] = bond[i] & 1;
            nb[1] = ((y + 1) % L) * L + x;     dx[1] = 0;  dy[1] = 1;  has[1] = (bond[i] >> 1) & 1;
            nb[2] = y * L + (x + L - 1) % L;   dx[2] = -1; dy[2] = 0;  has[2] = bond[nb[2]] & 1;
            nb[3] = ((y + L - 1) % L) * L + x; dx[3] = 0;  dy[3] = -1; has[3] = (bond[nb[3]] >> 1) & 1;
            for (int q = 0; q < 4; q++) {
                if (!has[q])
                    continue;
                int64_t j = nb[q], px = ux[i] + dx[q], py = uy[i] + dy[q];
                if (!seen[j]) {
                    seen[j] = 1;
                    ux[j] = px;
                    uy[j] = py;
                    queue[tail++] = j;
                } else {
                    if (ux[j] != px)
                        *wraps_x = 1;
                    if (uy[j] != py)
                        *wraps_y = 1;
                }
            }
        }
    }
    free(ux);
    free(uy);
    free(seen);
    free(queue);
    return 0;
}

/* ------------------------------------------------------------------------
 * Percolation under open boundaries (Sec. III): a cluster spans x iff it
 * holds a site of the leftmost column and a site of the rightmost column
 * (spans y: topmost and bottommost rows).
 * ---------------------------------------------------------------------- */
int swo_spans_open(int32_t L, const int32_t *label, int32_t *spans_x, int32_t *spans_y)
{
    int64_t N = (int64_t)L * (int64_t)L;
    uint8_t *mark = (uint8_t *)calloc((size_t)N, 1);
    if (!mark)
        return -1;
    /* bit 0: the root has a site in column 0; bit 1: in row 0 */
    for (int32_t b = 0; b < L; b++) {
        mark[label[(int64_t)b * L]] |= 1;
        mark[label[b]] |= 2;
    }
    *spans_x = 0;
    *spans_y = 0;
    for (int32_t b = 0; b < L; b++) {
        if (mark[label[(int64_t)b * L + (L - 1)]] & 1)
            *spans_x = 1;
        if (mark[label[(int64_t)(L - 1) * L + b]] & 2)
            *spans_y = 1;
    }
    free(mark);
    return 0;
}

/* ------------------------------------------------------------------------
 * PCC feedback (the probability-changing cluster method the paper builds
 * on, Sec. I and Sec. III): after sweep k lower p if the clusters of that
 * sweep percolate, raise it otherwise.  The step is 2^-8 in p for sweeps
 * 0..999 and halves every 1000 sweeps down to 2^-20; in threshold units
 * delta_k = 2^(32 - min(8 + floor(k/1000), 20)).  t stays in [0, 2^32].
 * ---------------------------------------------------------------------- */
uint64_t swo_pcc_delta(uint64_t sweep)
{
    uint64_t e = 8 + sweep / 1000;
    if (e > 20)
        e = 20;
    return (uint64_t)1 << (32 - e);
}

uint64_t swo_pcc_update(uint64_t thr, uint64_t sweep, int32_t flag)
{
    uint64_t d = swo_pcc_delta(sweep);
    uint64_t top = (uint64_t)1 << 32;
    if (flag)
        return thr > d ? thr - d : 0;
    return thr + d < top ? thr + d : top;
}

/* ------------------------------------------------------------------------
 * Whole sweeps, step by step in the paper's order (Sec. I steps 1-4).
 * ---------------------------------------------------------------------- */
int swo_run(int32_t L, uint64_t seed, uint64_t sweep0, int32_t nsweeps, int32_t pcc, int32_t open,
            int32_t csize, int32_t wind, uint64_t *thr, uint8_t *spin, int32_t *label, uint8_t *bond, swo_obs *obs)
{
    int64_t N = (int64_t)L * (int64_t)L;
    uint8_t *b = bond ? bond : (uint8_t *)malloc((size_t)N);
    if (!b)
        return -1;
    int rc = 0;
    for (int32_t n = 0; n < nsweeps; n++) {
        uint64_t k = sweep0 + (uint64_t)n;
        uint64_t t = *thr;
        swo_obs o;
        memset(&o, 0, sizeof(o));
        o.threshold = t;
        o.nbonds = swo_bonds(L, seed, k, t, spin, b, open); /* step 1 */
        o.nclusters = swo_label(L, b, label);            /* step 2 */
        if (csize) {
            o.csize2 = swo_csize2(L, label);
            if (o.csize2 < 0) {
                rc = -1;
                break;
            }
        }
        swo_assign(L, seed, k, label, spin);             /* step 3 */
        swo_measure(L, spin, open, &o.bond_sum, &o.mag);
        if (pcc || wind) {
            int src = wind   ? swo_windings(L, b, &o.spans_x, &o.spans_y)
                      : open ? swo_spans_open(L, label, &o.spans_x, &o.spans_y)
                             : swo_spans(L, label, &o.spans_x, &o.spans_y);
            if (src != 0) {
                rc = -1;
                break;
            }
            if (pcc)
                *thr = swo_pcc_update(t, k, o.spans_x || o.spans_y);
        }
        obs[n] = o;
    }
    if (!bond)
        free(b);
    return rc;
}

/* ========================================================================
 * q-state Potts model on the periodic d-dimensional lattice (d = 2 or 3).
 * The paper states the cluster update for general d (Sec. II); the Potts
 * form of SW replaces "equal spins" by "equal states" and a fair bit by a
 * uniform state.  Conventions (a reading: the paper fixes none of them):
 *   - N = L^d sites, i = x + L*y (+ L*L*z); site i owns link dir = 0 (+x),
 *     1 (+y), 2 (+z), link index l = d*i + dir.
 *   - H = -J sum over links of delta(s_i, s_j); a link between equal states
 *     bonds with P = 1 - exp(-J/T) (for q = 2 this is the Ising update with
 *     J_Ising = J/2), drawing word (l mod 4) of Philox(l/4, k, BOND).
 *   - A cluster with root r takes state floor(w*q / 2^32), w = word (r mod 4)
 *     of Philox(r/4, k, QSPIN); the hot start takes the same function of
 *     word (i mod 4) of Philox(i/4, 0, INIT).
 *   - bond_sum = sum over links of (2 delta - 1) (for q = 2: sum sigma sigma),
 *     mag = sum over sites of (q [s_i = 0] - 1).
 * ======================================================================== */
static uint64_t nd_neighbour(int32_t dim, int32_t L, uint64_t i, int dir)
{
    uint64_t l = (uint64_t)L, x = i % l, y = (i / l) % l, z = i / (l * l);
    if (dir == 0)
        x = (x + 1) % l;
    else if (dir == 1)
        y = (y + 1) % l;
    else
        z = (z + 1) % l;
    return dim == 2 ? y * l + x : (z * l + y) * l + x;
}

/* The link of site i in direction dir exists unless open boundaries cut it:
 * under open boundaries the last coordinate along dir has no + link. */
static int nd_link_exists(int32_t L, uint64_t i, int dir, int32_t open)
{
    if (!open)
        return 1;
    uint64_t l = (uint64_t)L, c = dir == 0 ? i % l : dir == 1 ? (i / l) % l : i / (l * l);
    return c + 1 < l;
}

static uint64_t nd_sites(int32_t dim, int32_t L)
{
    uint64_t n = (uint64_t)L * (uint64_t)L;
    return dim == 3 ? n * (uint64_t)L : n;
}

static uint8_t potts_state(uint32_t w, int32_t q)
{
    return (uint8_t)(((uint64_t)w * (uint64_t)q) >> 32);
}

uint64_t swo_threshold_potts(double J, double T)
{
    return swo_threshold_p(1.0 - exp(-J / T));
}

void swo_potts_hot_start(int32_t dim, int32_t L, int32_t q, uint64_t seed, uint8_t *spin)
{
    uint64_t N = nd_sites(dim, L);
    for (uint64_t i = 0; i < N; i++) {
        uint32_t w[4];
        stream_block(seed, i / 4, 0, SWO_STREAM_INIT, w);
        spin[i] = potts_state(w[i % 4], q);
    }
}

int64_t swo_potts_bonds(int32_t dim, int32_t L, uint64_t seed, uint64_t sweep, uint64_t thr,
                        const uint8_t *spin, uint8_t *bond)
{
    return swo_potts_bonds_open(dim, L, seed, sweep, thr, spin, bond, 0);
}

int64_t swo_potts_bonds_open(int32_t dim, int32_t L, uint64_t seed, uint64_t sweep, uint64_t thr,
                             const uint8_t *spin, uint8_t *bond, int32_t open)
{
    uint64_t N = nd_sites(dim, L);
    int64_t nb = 0;
    for (uint64_t i = 0; i < N; i++) {
        uint8_t b = 0;
        for (int dir = 0; dir < dim; dir++) {
            if (!nd_link_exists(L, i, dir, open))
                continue;
            uint64_t j = nd_neighbour(dim, L, i, dir);
            uint64_t l = (uint64_t)dim * i + (uint64_t)dir;
            uint32_t w[4];
            stream_block(seed, l / 4, sweep, SWO_STREAM_BOND, w);
            if (spin[i] == spin[j] && (uint64_t)w[l % 4] < thr) {
                b |= (uint8_t)(1u << dir);
                nb++;
            }
        }
        bond[i] = b;
    }
    return nb;
}

/* Clusters of a d-dimensional bond set: union of the ends of every bond,
 * the smaller root winning, then every site's root (its cluster minimum). */
int64_t swo_label_nd(int32_t dim, int32_t L, const uint8_t *bond, int32_t *label)
{
    uint64_t N = nd_sites(dim, L);
    for (uint64_t i = 0; i < N; i++)
        label[i] = (int32_t)i;
    for (uint64_t i = 0; i < N; i++)
        for (int dir = 0; dir < dim; dir++)
            if ((bond[i] >> dir) & 1u)
                uf_unite(label, (int32_t)i, (int32_t)nd_neighbour(dim, L, i, dir));
    int64_t nclusters = 0;
    for (uint64_t i = 0; i < N; i++) {
        label[i] = uf_find(label, (int32_t)i);
        if ((uint64_t)label[i] == i)
            nclusters++;
    }
    return nclusters;
}

void swo_count_clusters_nd(int32_t dim, int32_t L, int64_t nsets, const uint8_t *bonds, int64_t *counts)
{
    uint64_t N = nd_sites(dim, L);
    int32_t *label = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    for (int64_t s = 0; s < nsets; s++)
        counts[s] = label ? swo_label_nd(dim, L, bonds + s * (int64_t)N, label) : -1;
    free(label);
}

void swo_potts_assign(int32_t dim, int32_t L, int32_t q, uint64_t seed, uint64_t sweep,
                      const int32_t *label, uint8_t *spin)
{
    uint64_t N = nd_sites(dim, L);
    for (uint64_t i = 0; i < N; i++) {
        uint64_t r = (uint64_t)label[i];
        uint32_t w[4];
        stream_block(seed, r / 4, sweep, SWO_STREAM_QSPIN, w);
        spin[i] = potts_state(w[r % 4], q);
    }
}

void swo_potts_measure(int32_t dim, int32_t L, int32_t q, const uint8_t *spin, int64_t *bond_sum,
                       int64_t *mag)
{
    swo_potts_measure_open(dim, L, q, spin, 0, bond_sum, mag);
}

void swo_potts_measure_open(int32_t dim, int32_t L, int32_t q, const uint8_t *spin, int32_t open,
                            int64_t *bond_sum, int64_t *mag)
{
    uint64_t N = nd_sites(dim, L);
    int64_t bs = 0, m = 0;
    for (uint64_t i = 0; i < N; i++) {
        m += spin[i] == 0 ? q - 1 : -1;
        for (int dir = 0; dir < dim; dir++)
            if (nd_link_exists(L, i, dir, open))
                bs += spin[i] == spin[nd_neighbour(dim, L, i, dir)] ? 1 : -1;
    }
    *bond_sum = bs;
    *mag = m;
}

/* ------------------------------------------------------------------------
 * Extension rule on the d-dimensional lattice (Sec. III states it for any
 * dimension): a cluster spans axis a iff its projection on that axis is the
 * whole range [0, L-1], i.e. iff it occupies every one of the L hyperplanes
 * perpendicular to a.  Each root's number of distinct hyperplanes is counted
 * by scanning the hyperplanes in order and stamping each root with the last
 * one it was seen in (as swo_spans does for the rows and columns of d = 2).
 * Under open boundaries a cluster cannot wrap, so its projection is an
 * interval and occupying every hyperplane is touching both opposite faces.
 * ---------------------------------------------------------------------- */
int swo_spans_nd(int32_t dim, int32_t L, const int32_t *label, int32_t *spans)
{
    uint64_t N = nd_sites(dim, L), l = (uint64_t)L;
    int32_t *stamp = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *count = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    if (!stamp || !count) {
        free(stamp);
        free(count);
        return -1;
    }
    uint64_t inner = dim == 3 ? l * l : l;   /* sites of one hyperplane */
    for (int a = 0; a < dim; a++) {
        for (uint64_t i = 0; i < N; i++) {
            stamp[i] = -1;
            count[i] = 0;
        }
        spans[a] = 0;
        for (uint64_t c = 0; c < l; c++) {           /* the hyperplane: coordinate a = c */
            for (uint64_t u = 0; u < inner; u++) {   /* its sites */
                uint64_t v0 = u % l, v1 = u / l, x, y, z;
                if (a == 0) { x = c; y = v0; z = v1; }
                else if (a == 1) { x = v0; y = c; z = v1; }
                else { x = v0; y = v1; z = c; }
                uint64_t i = dim == 2 ? y * l + x : (z * l + y) * l + x;
                int32_t r = label[i];
                if (stamp[r] != (int32_t)c) {
                    stamp[r] = (int32_t)c;
                    if (++count[r] == L)
                        spans[a] = 1;
                }
            }
        }
    }
    free(stamp);
    free(count);
    return 0;
}

/* ------------------------------------------------------------------------
 * Topological rule in d dimensions (Sec. III: the winding criterion stated
 * for the periodic box of any dimension): a cluster winds around axis a iff
 * it holds a closed path of bonds whose net displacement along a is a
 * non-zero multiple of L.  As swo_windings does in 2D: every cluster is
 * explored breadth first from its lowest site, each site getting an
 * unwrapped position (each bond one lattice step, the periodic link included);
 * a bond reaching an explored site at a position other than the predicted one
 * closes a cycle with that displacement, and every cycle is a sum of such
 * cycles.  wraps[a] = 1 iff some cluster winds around axis a (a < dim).
 * ---------------------------------------------------------------------- */
int swo_windings_nd(int32_t dim, int32_t L, const uint8_t *bond, int32_t *wraps)
{
    uint64_t N = nd_sites(dim, L), l = (uint64_t)L;
    int64_t *u = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)N);
    uint8_t *seen = (uint8_t *)calloc((size_t)N, 1);
    uint64_t *queue = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    if (!u || !seen || !queue) {
        free(u);
        free(seen);
        free(queue);
        return -1;
    }
    for (int a = 0; a < 3; a++)
        wraps[a] = 0;
    uint64_t stride[3] = {1, l, l * l};
    for (uint64_t s = 0; s < N; s++) {
        if (seen[s])
            continue;
        uint64_t head = 0, tail = 0;
        seen[s] = 1;
        u[3 * s] = u[3 * s + 1] = u[3 * s + 2] = 0;
        queue[tail++] = s;
        while (head < tail) {
            uint64_t i = queue[head++];
            uint64_t c[3] = {i % l, (i / l) % l, dim == 3 ? i / (l * l) : 0};
            /* the 2 dim links at site i: its own + link along each axis, and
             * the + link of its - neighbour along each axis */
            for (int a = 0; a < dim; a++) {
                for (int side = 0; side < 2; side++) {
                    uint64_t j;
                    int has;
                    if (side == 0) {
                        j = c[a] + 1 == l ? i - c[a] * stride[a] : i + stride[a];
                        has = (bond[i] >> a) & 1;
                    } else {
                        j = c[a] == 0 ? i + (l - 1) * stride[a] : i - stride[a];
                        has = (bond[j] >> a) & 1;
                    }
                    if (!has)
                        continue;
                    int64_t p[3] = {u[3 * i], u[3 * i + 1], u[3 * i + 2]};
                    p[a] += side == 0 ? 1 : -1;
                    if (!seen[j]) {
                        seen[j] = 1;
                        u[3 * j] = p[0];
                        u[3 * j + 1] = p[1];
                        u[3 * j + 2] = p[2];
                        queue[tail++] = j;
                    } else {
                        for (int b = 0; b < 3; b++)
                            if (u[3 * j + b] != p[b])
                                wraps[b] = 1;
                    }
                }
            }
        }
    }
    free(u);
    free(seen);
    free(queue);
    return 0;
}

int swo_potts_run(int32_t dim, int32_t L, int32_t q, uint64_t seed, uint64_t sweep0, int32_t nsweeps,
                  int32_t csize, uint64_t thr, uint8_t *spin, int32_t *label, uint8_t *bond, swo_obs *obs)
{
    return swo_potts_run_pcc(dim, L, q, seed, sweep0, nsweeps, 0, 0, csize, &thr, spin, label, bond, obs);
}

int swo_potts_run_pcc(int32_t dim, int32_t L, int32_t q, uint64_t seed, uint64_t sweep0, int32_t nsweeps,
                      int32_t pcc, int32_t open, int32_t csize, uint64_t *thr_io, uint8_t *spin, int32_t *label,
                      uint8_t *bond, swo_obs *obs)
{
    return swo_potts_run_rules(dim, L, q, seed, sweep0, nsweeps, pcc, open, csize, 0, thr_io, spin, label, bond,
                               obs);
}

int swo_potts_run_rules(int32_t dim, int32_t L, int32_t q, uint64_t seed, uint64_t sweep0, int32_t nsweeps,
                        int32_t pcc, int32_t open, int32_t csize, int32_t wind, uint64_t *thr_io, uint8_t *spin,
                        int32_t *label, uint8_t *bond, swo_obs *obs)
{
    uint64_t thr = *thr_io;
    uint64_t N = nd_sites(dim, L);
    uint8_t *b = bond ? bond : (uint8_t *)malloc((size_t)N);
    if (!b)
        return -1;
    int rc = 0;
    for (int32_t n = 0; n < nsweeps; n++) {
        uint64_t k = sweep0 + (uint64_t)n;
        swo_obs o;
        memset(&o, 0, sizeof(o));
        o.threshold = thr;
        o.nbonds = swo_potts_bonds_open(dim, L, seed, k, thr, spin, b, open);
        o.nclusters = swo_label_nd(dim, L, b, label);
        if (wind) {   /* the topological rule, reported every sweep */
            int32_t w[3] = {0, 0, 0};
            if (swo_windings_nd(dim, L, b, w) != 0) {
                rc = -1;
                break;
            }
            o.spans_x = w[0];
            o.spans_y = w[1] | w[2];     /* y, or in 3D y or z */
        } else if (pcc) {
            int32_t sp[3] = {0, 0, 0};
            if (swo_spans_nd(dim, L, label, sp) != 0) {
                rc = -1;
                break;
            }
            o.spans_x = sp[0];
            o.spans_y = sp[1] | sp[2];   /* y, or in 3D y or z */
        }
        if (csize) {
            int64_t *count = (int64_t *)calloc((size_t)N, sizeof(int64_t));
            if (!count) {
                rc = -1;
                break;
            }
            for (uint64_t i = 0; i < N; i++)
                count[label[i]]++;
            for (uint64_t r = 0; r < N; r++)
                o.csize2 += count[r] * count[r];
            free(count);
        }
        swo_potts_assign(dim, L, q, seed, k, label, spin);
        swo_potts_measure_open(dim, L, q, spin, open, &o.bond_sum, &o.mag);
        obs[n] = o;
        if (pcc)
            thr = swo_pcc_update(thr, k, o.spans_x || o.spans_y);
    }
    *thr_io = thr;
    if (!bond)
        free(b);
    return rc;
}
