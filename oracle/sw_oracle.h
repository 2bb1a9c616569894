/*
 * sw_oracle.h -- CPU oracle for the Swendsen-Wang / PCC hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Paper: S. Lin and B. Zheng, "Two Parallel Swendsen-Wang Cluster Algorithms
 * Using Message-Passing Paradigm" (arXiv:0808.2109).
 *
 * Lattice conventions (a reading: the paper fixes none of them):
 *   - L x L periodic square lattice, site index i = y*L + x, row-major.
 *   - Site i owns link d=0 to (x+1 mod L, y) and d=1 to (x, y+1 mod L); the
 *     link index is l = 2*i + d, so there are 2*L*L links.  For L = 2 the two
 *     links between the same pair of sites are both counted.
 *   - Spins are stored as uint8 s in {0,1}; sigma = 2*s - 1.
 *   - Bond bytes: bit 0 = link d=0 (right) is bonded, bit 1 = link d=1 (down).
 *   - Labels: int32 root(i) = the minimum site index of i's cluster.
 *   - open != 0 selects open (free) boundaries: the right link of column L-1
 *     and the down link of row L-1 do not exist (no bond, no energy term).
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11).  Key = (seed mod 2^32, seed >> 32).
 * Counter = (index word, sweep mod 2^32, sweep >> 32, stream).
 */
#ifndef SW_ORACLE_H
#define SW_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SWO_STREAM_INIT 0u
#define SWO_STREAM_BOND 1u
#define SWO_STREAM_SPIN 2u
#define SWO_STREAM_QSPIN 3u   /* Potts cluster states */

/* Observables of one sweep (all taken after the cluster flip). */
typedef struct {
    int64_t bond_sum;   /* sum over all 2N links of sigma_i sigma_j          */
    int64_t mag;        /* sum of sigma_i                                    */
    int64_t nclusters;  /* number of clusters built in this sweep            */
    int64_t nbonds;     /* number of bonded links in this sweep              */
    int32_t spans_x;    /* PCC only: some cluster occupies all L columns     */
    int32_t spans_y;    /* PCC only: some cluster occupies all L rows        */
    uint64_t threshold; /* bond threshold used in this sweep                 */
    int64_t csize2;     /* sum over this sweep's clusters of |C|^2           */
} swo_obs;

/* Philox4x32-10 of one counter block. */
void swo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* n independent blocks: ctr[4n], key[2n] -> out[4n]. */
void swo_philox_batch(int64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out);

/* Bond threshold t = floor(P * 2^32), P = 1 - exp(-2J/T) (paper, Sec. I step 1). */
uint64_t swo_threshold_T(double J, double T);
/* Bond threshold for a given bond probability p in [0, 1]. */
uint64_t swo_threshold_p(double p);

/* Hot start: s_i = bit (i mod 128) of Philox(i/128, sweep 0, INIT). */
void swo_hot_start(int32_t L, uint64_t seed, uint8_t *spin);

/* Step 1: bond activation of sweep k.  Returns the number of bonds. */
int64_t swo_bonds(int32_t L, uint64_t seed, uint64_t sweep, uint64_t thr,
                  const uint8_t *spin, uint8_t *bond, int32_t open);

/* Step 2: clusters by Hoshen-Kopelman raster scan + union-find, labels are
 * the minimum site index of each cluster.  Returns the number of clusters. */
int64_t swo_label(int32_t L, const uint8_t *bond, int32_t *label);

/* Number of clusters of each of nsets bond sets bonds[nsets * L*L]. */
void swo_count_clusters_batch(int32_t L, int64_t nsets, const uint8_t *bonds, int64_t *counts);

/* Step 3: every cluster takes bit (root mod 128) of Philox(root/128, k, SPIN). */
void swo_assign(int32_t L, uint64_t seed, uint64_t sweep, const int32_t *label, uint8_t *spin);

/* Sum over the clusters of |C|^2, from the labels.  Each cluster takes an
 * independent fair sign, so its mean over the flip is M^2: the cluster
 * ("improved") estimator of the susceptibility. */
int64_t swo_csize2(int32_t L, const int32_t *label);

/* Energy and magnetisation sums of a spin field. */
void swo_measure(int32_t L, const uint8_t *spin, int32_t open, int64_t *bond_sum, int64_t *mag);

/* Extension rule under periodic boundaries (paper, Sec. III): spans_x is 1 iff
 * some cluster occupies all L columns, spans_y iff some cluster occupies all
 * L rows.  Returns 0, or -1 when memory is short. */
int swo_spans(int32_t L, const int32_t *label, int32_t *spans_x, int32_t *spans_y);

/* Percolation under open boundaries (paper, Sec. III): spans_x is 1 iff some
 * cluster touches both the leftmost and the rightmost column, spans_y iff
 * some cluster touches both the topmost and the bottommost row. */
int swo_spans_open(int32_t L, const int32_t *label, int32_t *spans_x, int32_t *spans_y);

/* Topological rule (paper, Sec. III): wraps_x is 1 iff some cluster of the
 * bond set winds around the box in x (holds a closed path of bonds whose net
 * x displacement is a non-zero multiple of L); wraps_y likewise.  Returns 0,
 * or -1 when memory is short. */
int swo_windings(int32_t L, const uint8_t *bond, int32_t *wraps_x, int32_t *wraps_y);

/* PCC feedback step size after sweep k, in threshold units. */
uint64_t swo_pcc_delta(uint64_t sweep);
/* PCC feedback: t -= delta if flag else t += delta, clamped to [0, 2^32]. */
uint64_t swo_pcc_update(uint64_t thr, uint64_t sweep, int32_t flag);

/* nsweeps full sweeps k = sweep0 .. sweep0+nsweeps-1 on spin[] in place.
 * *thr is the threshold of the first sweep; with pcc != 0 it is updated by
 * the feedback after every sweep (spans by swo_spans, or swo_spans_open when
 * open != 0).  csize != 0 fills obs[].csize2 (else it stays 0).  wind != 0
 * switches the span test to the topological rule (swo_windings) and reports
 * it every sweep, PCC or not.  label[] receives the labels of the last
 * sweep, bond[] (optional, may be NULL) its bonds, obs[nsweeps] the
 * per-sweep observables.  Returns 0, or -1 when memory is short. */
int swo_run(int32_t L, uint64_t seed, uint64_t sweep0, int32_t nsweeps, int32_t pcc, int32_t open,
            int32_t csize, int32_t wind, uint64_t *thr, uint8_t *spin, int32_t *label, uint8_t *bond, swo_obs *obs);

/* ---- q-state Potts model on the periodic d-dimensional lattice (d = 2, 3).
 * Site i = x + L*y (+ L*L*z), link l = d*i + dir (dir 0: +x, 1: +y, 2: +z),
 * bond bytes bit dir.  H = -J sum delta(s_i, s_j), bonds with P = 1 - exp(-J/T).
 * States: floor(w*q / 2^32) of a Philox word (hot start: word i mod 4 of
 * Philox(i/4, 0, INIT); cluster with root r: word r mod 4 of Philox(r/4, k,
 * QSPIN)).  bond_sum = sum over links of (2 delta - 1); mag = sum over sites of
 * (q [s_i = 0] - 1). */
uint64_t swo_threshold_potts(double J, double T);
void swo_potts_hot_start(int32_t dim, int32_t L, int32_t q, uint64_t seed, uint8_t *spin);
int64_t swo_potts_bonds(int32_t dim, int32_t L, uint64_t seed, uint64_t sweep, uint64_t thr,
                        const uint8_t *spin, uint8_t *bond);
int64_t swo_label_nd(int32_t dim, int32_t L, const uint8_t *bond, int32_t *label);
void swo_count_clusters_nd(int32_t dim, int32_t L, int64_t nsets, const uint8_t *bonds, int64_t *counts);
void swo_potts_assign(int32_t dim, int32_t L, int32_t q, uint64_t seed, uint64_t sweep,
                      const int32_t *label, uint8_t *spin);
void swo_potts_measure(int32_t dim, int32_t L, int32_t q, const uint8_t *spin, int64_t *bond_sum,
                       int64_t *mag);
/* open != 0: open boundaries (the last coordinate along a direction has no
 * + link; no bond, no energy term). */
int64_t swo_potts_bonds_open(int32_t dim, int32_t L, uint64_t seed, uint64_t sweep, uint64_t thr,
                             const uint8_t *spin, uint8_t *bond, int32_t open);
void swo_potts_measure_open(int32_t dim, int32_t L, int32_t q, const uint8_t *spin, int32_t open,
                            int64_t *bond_sum, int64_t *mag);
/* Extension rule in d = 2 or 3 dimensions (Sec. III): spans[a] = 1 iff some
 * cluster occupies all L hyperplanes perpendicular to axis a (a < dim).
 * Returns 0, or -1 when memory is short. */
int swo_spans_nd(int32_t dim, int32_t L, const int32_t *label, int32_t *spans);
/* As swo_potts_run, with open boundaries (open != 0) and the PCC feedback
 * (pcc != 0): *thr_io is the first sweep's threshold and, after each sweep,
 * moves by swo_pcc_update on (some cluster spans some axis); obs[].spans_x
 * reports the x axis, spans_y the y axis (in 3D: the y or the z axis).  On
 * return *thr_io holds the next sweep's threshold. */
int swo_potts_run_pcc(int32_t dim, int32_t L, int32_t q, uint64_t seed, uint64_t sweep0, int32_t nsweeps,
                      int32_t pcc, int32_t open, int32_t csize, uint64_t *thr_io, uint8_t *spin, int32_t *label,
                      uint8_t *bond, swo_obs *obs);
/* Topological rule in d = 2 or 3 dimensions (Sec. III): wraps[a] = 1 iff
 * some cluster of the bond set winds around the box along axis a (holds a
 * closed path of bonds whose net displacement along a is a non-zero multiple
 * of L), for a < dim; wraps[2] = 0 in 2D.  Returns 0, or -1 when memory is
 * short. */
int swo_windings_nd(int32_t dim, int32_t L, const uint8_t *bond, int32_t *wraps);
/* As swo_potts_run_pcc; wind != 0 switches the span test to the topological
 * rule (swo_windings_nd) and reports it every sweep, PCC or not (spans_x:
 * axis x; spans_y: axis y, in 3D y or z). */
int swo_potts_run_rules(int32_t dim, int32_t L, int32_t q, uint64_t seed, uint64_t sweep0, int32_t nsweeps,
                        int32_t pcc, int32_t open, int32_t csize, int32_t wind, uint64_t *thr_io, uint8_t *spin,
                        int32_t *label, uint8_t *bond, swo_obs *obs);
/* nsweeps sweeps at the fixed threshold thr (obs[].csize2 filled when csize). */
int swo_potts_run(int32_t dim, int32_t L, int32_t q, uint64_t seed, uint64_t sweep0, int32_t nsweeps,
                  int32_t csize, uint64_t thr, uint8_t *spin, int32_t *label, uint8_t *bond, swo_obs *obs);

#ifdef __cplusplus
}
#endif

#endif
