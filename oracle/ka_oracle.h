/*
 * ka_oracle.h -- serial CPU oracle for the multispin Kob-Andersen chain.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct
 * restatement of the method of Boccagna, "A Multispin Algorithm for the
 * Kob-Andersen Stochastic Dynamics on Regular Lattices" (arXiv 1710.05155),
 * with one byte per (site, replica).  Only the test suite, the package smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * State arrays are site-major: byte [i * Rs + rr] holds replica r0 + rr at
 * site i.  Every function returns 0 on success, 1 on invalid arguments,
 * 2 when memory runs out.
 */
#ifndef KA_ORACLE_H
#define KA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11). */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* 64-bit random gate word for word w of edge `bond` in class `cls` at sweep t
 * on a graph: half (w mod 2) of the block at counter (t, cls, bond, w / 2). */
uint64_t ora_gate_word(uint64_t seed, int64_t t, int64_t cls, int64_t bond, int64_t w);

/* The same on a periodic cubic lattice of side L, where `bond` is the base
 * site: bonds starting at pencil positions 4k + 2b and 4k + 2b + 1 (classes
 * 4g + 2b and 4g + 2b + 1) share the block at counter
 * (t, 4g + 2b, base site of the first, w), the first taking half 0. */
uint64_t ora_cubic_gate_word(uint64_t seed, int64_t t, int64_t cls, int64_t bond, int64_t w,
                             int L);

/* K = rho*N rounded half away from zero. */
int64_t ora_particles(double rho, int64_t N);

/* Neighbour table nbr[N][2d] of the periodic cubic lattice and its bond
 * classes.  Buffers: nbr N*2d, bu/bv/bid d*N, class_off nclass+1 where
 * nclass = 4 for d = 1 and 8d otherwise. */
int ora_cubic_tables(int d, int L, int32_t *nbr, int64_t *class_off,
                     int32_t *bu, int32_t *bv, int64_t *bid, int64_t *nclass);

/* Random z-regular simple graph on N vertices (configuration model with
 * whole-graph rejection).  nbr[N][z] sorted ascending per vertex. */
int ora_rrg_build(int64_t N, int z, uint64_t graph_seed, int64_t max_attempts,
                  int32_t *nbr, int64_t *attempts_out);

/* Edges (u < v) of a z-regular graph in lexicographic order, E = N*z/2. */
int ora_graph_edges(int64_t N, int z, const int32_t *nbr, int32_t *eu, int32_t *ev);

/* Greedy strong edge colouring in edge-id order; classes are the colours in
 * ascending order, edges inside a class in id order.  Buffers: class_off
 * (E+1 worst case), bu/bv/bid E. */
int ora_graph_classes(int64_t N, int z, const int32_t *nbr, int64_t *class_off,
                      int32_t *bu, int32_t *bv, int64_t *bid, int64_t *nclass);

/* Brute-force check: every class is a strong matching and the classes
 * together hold every edge of the graph exactly once.  Returns 0 if valid. */
int ora_check_schedule(int64_t N, int z, const int32_t *nbr, int64_t nclass,
                       const int64_t *class_off, const int32_t *bu, const int32_t *bv);

/* The Kob-Andersen exchange rule on one bond for one replica, given the
 * occupations of the z-1 other neighbours of i and of j. */
int ora_local_move(int z, int m, int ni, int nj, const uint8_t *others_i,
                   const uint8_t *others_j, int gate, int *ni_out, int *nj_out);

/* Initial state: exactly K particles per replica at the K sites of smallest
 * (key, site) where key comes from Philox; n0 = n, p = 1. */
int ora_init(int64_t N, int64_t r0, int64_t Rs, uint64_t seed, int64_t K,
             uint8_t *n, uint8_t *n0, uint8_t *p);

/* One class of bonds at sweep t.  cubic_L > 0 selects the cubic-lattice gate
 * stream (ora_cubic_gate_word with side cubic_L), 0 the graph stream. */
int ora_class_step(int64_t N, int z, const int32_t *nbr, int m, int64_t nb,
                   const int32_t *bu, const int32_t *bv, const int64_t *bid,
                   int64_t cls, int64_t t, uint64_t seed, int64_t r0, int64_t Rs,
                   int cubic_L, uint8_t *n, uint8_t *p);

/* nsweeps sweeps starting at sweep index t0 (all classes in order). */
int ora_sweeps(int64_t N, int z, const int32_t *nbr, int m, int64_t nclass,
               const int64_t *class_off, const int32_t *bu, const int32_t *bv,
               const int64_t *bid, uint64_t seed, int64_t r0, int64_t Rs, int cubic_L,
               int64_t t0, int64_t nsweeps, uint8_t *n, uint8_t *p);

/* Per replica: particles, overlap (n and n0), persist_occ (n0 and p),
 * persist_all (p).  counts[Rs][4]. */
void ora_observe(int64_t N, int64_t Rs, const uint8_t *n, const uint8_t *n0,
                 const uint8_t *p, int64_t *counts);

/* Four-point correlations on the periodic cubic lattice (section 2.2 g_4(r,t),
 * section 3.3 Phi(r,t)), by brute force over all ordered site pairs (i, j).
 * The displacement of a pair is taken with every component in [-L/2, L/2)
 * (one representative per class modulo L) and its shell is s = |delta|^2.
 * With q_i = n_i AND n0_i per replica and M_i = sum over replicas of q_i:
 *   phi[rr * (smax + 1) + s] = sum over pairs in shell s of q_i q_j (replica rr)
 *   psi[s]                   = sum over pairs in shell s of M_i M_j
 * for s = 0 .. smax; pairs in shells above smax are not counted. */
int ora_four_point(int d, int L, int64_t Rs, const uint8_t *n, const uint8_t *n0, int64_t smax,
                   int64_t *phi, int64_t *psi);

/* Layered random graph (section 5.2): M copies of the periodic cubic lattice
 * of side L in d dimensions (vertex a N + i is site i of copy a); for every
 * base bond (i, i + e_mu) the M links (copy a of i, copy a of j) are replaced
 * by (copy a of i, copy pi(a) of j), pi a uniform permutation of the copies
 * drawn independently per bond: Fisher-Yates from the top, step k drawing a
 * uniform integer in [0, k] by Lemire's method on the Philox words of counter
 * (i, 0xFFFFFFFD, mu << 16 | k, draw) keyed by the graph seed.  nbr[M N][2d]:
 * entry 2 mu is the neighbour across the up bond along mu, 2 mu + 1 across
 * the down bond.  Needs 1 <= d <= 4, L >= 3, 1 <= M < 65536. */
int ora_layered_graph(int d, int L, int M, uint64_t graph_seed, int32_t *nbr);

/* Random-sequential sweeps (section 3.2 with the time unit of section 2.1):
 * per word of 64 replicas and per sweep t, N attempts k = 0 .. N-1; attempt k
 * draws r uniform in [0, N z) (Lemire's method on the low 64 bits of the
 * Philox block at counter (t, 0xFFFFFFFC - draw, k, word), key = seed,
 * draw = 0, 1, ...), takes site i = r / z and its neighbour j in slot r mod z,
 * and exchanges n_i and n_j in every replica of the word where the rule
 * allows it (no gate; p cleared on both sites).  All replicas of a word share
 * the bond sequence.  Replicas r0 .. r0+Rs-1, r0 and Rs multiples of 64. */
int ora_sequential_sweeps(int64_t N, int z, const int32_t *nbr, int m, uint64_t seed, int64_t r0,
                          int64_t Rs, int64_t t0, int64_t nsweeps, uint8_t *n, uint8_t *p);

#ifdef __cplusplus
}
#endif
#endif
