/*
 * ka_oracle.c -- serial CPU oracle for the multispin Kob-Andersen chain.
 *
 * TEST INFRASTRUCTURE ONLY (see ka_oracle.h).  Written for a reader who
 * checks it against the paper by eye: one byte per (site, replica), the
 * steps in the paper's order, no blocking, no fusion, no bit tricks.
 *
 * What it follows:
 *   - the exchange rule: section 2.1 of the paper, rules (a)-(c).  A particle
 *     at i moves to the empty neighbour j iff i has at most m occupied
 *     neighbours (j is empty, so this counts N(i) without j) and j has at
 *     most m+1 occupied neighbours (i is occupied, so N(j) without i has at
 *     most m).  Both conditions read as "at most m among the z-1 other
 *     neighbours", which is symmetric in i and j.
 *   - conserved particle number and the flat stationary measure: sections
 *     2.1 and 2.2.
 *   - one bit per replica, the same bond attempted in all replicas:
 *     section 3.1 and the update of section 3.2 (Table 1), with an
 *     independent Bernoulli(1/2) gate per replica on every attempt.
 *   - observables: the overlap n_i(t) n_i(0) of section 2.2 summed over
 *     sites per replica, and a persistence count.
 *   - random regular graphs: the configuration model of section 2.1
 *     (Bollobas), with whole-graph rejection of self-loops and multi-edges.
 *
 * Philox4x32-10 follows Salmon, Moraes, Dror and Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11).  Lemire's bounded integer method
 * follows Lemire, "Fast random integer generation in an interval" (ACM
 * TOMACS 2019).
 */
#include "ka_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORA_OK 0
#define ORA_EINVAL 1
#define ORA_ENOMEM 2

/* Counter field c1 tags the stream: bond classes use ids below these. */
#define ORA_TAG_INIT 0xFFFFFFFFu
#define ORA_TAG_GRAPH 0xFFFFFFFEu
#define ORA_TAG_LAYER 0xFFFFFFFDu
#define ORA_TAG_SEQUENTIAL 0xFFFFFFFCu

/* ------------------------------------------------------------------ */
/* Philox4x32-10                                                       */
/* ------------------------------------------------------------------ */

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += weyl0;
            k1 += weyl1;
        }
        uint64_t prod0 = (uint64_t)mult0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)mult1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

static void ora_philox_seeded(uint64_t seed, uint32_t a, uint32_t b, uint32_t c, uint32_t d,
                              uint32_t out[4])
{
    uint32_t ctr[4] = {a, b, c, d};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    ora_philox4x32_10(ctr, key, out);
}

uint64_t ora_gate_word(uint64_t seed, int64_t t, int64_t cls, int64_t bond, int64_t w)
{
    /* graphs: one block per (sweep, class, edge, word pair), half w mod 2 */
    uint32_t o[4];
    ora_philox_seeded(seed, (uint32_t)t, (uint32_t)cls, (uint32_t)bond, (uint32_t)(w / 2), o);
    if (w % 2 == 0)
        return (uint64_t)o[0] | ((uint64_t)o[1] << 32);
    return (uint64_t)o[2] | ((uint64_t)o[3] << 32);
}

uint64_t ora_cubic_gate_word(uint64_t seed, int64_t t, int64_t cls, int64_t bond, int64_t w,
                             int L)
{
    /* cubic lattices: the bonds of classes 4g + 2b and 4g + 2b + 1 that start
     * at pencil positions 4k + 2b and 4k + 2b + 1 share one block, counter
     * (sweep, 4g + 2b, base site of the first of the two, word); the first
     * bond takes half 0, the second half 1 */
    int64_t mu = cls / 8, a = cls % 4;
    int64_t stride = 1;
    for (int64_t k = 0; k < mu; k++)
        stride *= L;
    int64_t first = bond - (a % 2) * stride;
    uint32_t o[4];
    ora_philox_seeded(seed, (uint32_t)t, (uint32_t)(cls - (cls % 2)), (uint32_t)first,
                      (uint32_t)w, o);
    if (a % 2 == 0)
        return (uint64_t)o[0] | ((uint64_t)o[1] << 32);
    return (uint64_t)o[2] | ((uint64_t)o[3] << 32);
}

int64_t ora_particles(double rho, int64_t N)
{
    double x = rho * (double)N;
    return (int64_t)floor(x + 0.5);
}

/* ------------------------------------------------------------------ */
/* Periodic cubic lattice                                              */
/* ------------------------------------------------------------------ */

static int64_t ora_ipow(int64_t b, int e)
{
    int64_t r = 1;
    for (int k = 0; k < e; k++)
        r *= b;
    return r;
}

static void ora_coords(int64_t i, int d, int L, int *x)
{
    for (int k = 0; k < d; k++) {
        x[k] = (int)(i % L);
        i /= L;
    }
}

static int64_t ora_index(const int *x, int d, int L)
{
    int64_t i = 0;
    for (int k = d - 1; k >= 0; k--)
        i = i * L + x[k];
    return i;
}

int ora_cubic_tables(int d, int L, int32_t *nbr, int64_t *class_off, int32_t *bu, int32_t *bv,
                     int64_t *bid, int64_t *nclass)
{
    if (d < 1 || d > 4 || L < 4 || L % 4 != 0)
        return ORA_EINVAL;
    int64_t N = ora_ipow(L, d);
    int z = 2 * d;
    int x[4], y[4];

    /* neighbours: +e_k then -e_k for k = 0..d-1, periodic */
    for (int64_t i = 0; i < N; i++) {
        ora_coords(i, d, L, x);
        for (int k = 0; k < d; k++) {
            memcpy(y, x, sizeof(x));
            y[k] = (x[k] + 1) % L;
            nbr[i * z + 2 * k] = (int32_t)ora_index(y, d, L);
            y[k] = (x[k] + L - 1) % L;
            nbr[i * z + 2 * k + 1] = (int32_t)ora_index(y, d, L);
        }
    }

    /* class c = (2*mu + p)*4 + a holds the bonds (x, x + e_mu) with
     * x_mu = a mod 4 and (sum of the other coordinates) = p mod 2.
     * In one dimension there are no other coordinates, so only p = 0. */
    int64_t nc = (d == 1) ? 4 : 8 * d;
    int64_t nb = 0;
    for (int64_t c = 0; c < nc; c++) {
        int mu = (int)(c / 8), par = (int)((c / 4) % 2), a = (int)(c % 4);
        class_off[c] = nb;
        for (int64_t i = 0; i < N; i++) {
            ora_coords(i, d, L, x);
            int perp = 0;
            for (int k = 0; k < d; k++)
                if (k != mu)
                    perp += x[k];
            if (x[mu] % 4 != a || perp % 2 != par)
                continue;
            memcpy(y, x, sizeof(x));
            y[mu] = (x[mu] + 1) % L;
            bu[nb] = (int32_t)i;
            bv[nb] = (int32_t)ora_index(y, d, L);
            bid[nb] = i;
            nb++;
        }
    }
    class_off[nc] = nb;
    *nclass = nc;
    return ORA_OK;
}

/* ------------------------------------------------------------------ */
/* Random regular graph: configuration model, whole-graph rejection    */
/* ------------------------------------------------------------------ */

/* Uniform integer in [0, range) from 64-bit Philox words (Lemire's
 * multiply-and-reject method).  Draw number `draw` of step k of attempt t
 * uses counter (t, TAG_GRAPH, k, draw). */
static uint64_t ora_graph_bounded(uint64_t gseed, uint32_t t, uint32_t k, uint64_t range)
{
    uint32_t draw = 0, o[4];
    ora_philox_seeded(gseed, t, ORA_TAG_GRAPH, k, draw, o);
    uint64_t x = (uint64_t)o[0] | ((uint64_t)o[1] << 32);
    unsigned __int128 prod = (unsigned __int128)x * range;
    uint64_t low = (uint64_t)prod;
    if (low < range) {
        uint64_t threshold = (0 - range) % range;
        while (low < threshold) {
            draw++;
            ora_philox_seeded(gseed, t, ORA_TAG_GRAPH, k, draw, o);
            x = (uint64_t)o[0] | ((uint64_t)o[1] << 32);
            prod = (unsigned __int128)x * range;
            low = (uint64_t)prod;
        }
    }
    return (uint64_t)(prod >> 64);
}

static int ora_cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int ora_rrg_build(int64_t N, int z, uint64_t graph_seed, int64_t max_attempts, int32_t *nbr,
                  int64_t *attempts_out)
{
    if (N < 2 || z < 1 || z >= N || (N * z) % 2 != 0 || N * z > 0xFFFFFFFFLL)
        return ORA_EINVAL;
    int64_t M = N * z; /* stubs; stub s belongs to vertex s / z */
    int64_t *perm = (int64_t *)malloc((size_t)M * sizeof(int64_t));
    int32_t *deg = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    if (!perm || !deg) {
        free(perm);
        free(deg);
        return ORA_ENOMEM;
    }
    for (int64_t t = 0; t < max_attempts; t++) {
        for (int64_t s = 0; s < M; s++)
            perm[s] = s;
        for (int64_t v = 0; v < N; v++)
            deg[v] = 0;
        int simple = 1;
        /* Fisher-Yates from the top; after step k, position k is final, so
         * the pair (2q, 2q+1) is final once step 2q has run (pair 0 after
         * step 1).  A self-loop or a repeated edge rejects the attempt. */
        for (int64_t k = M - 1; k >= 1 && simple; k--) {
            int64_t j = (int64_t)ora_graph_bounded(graph_seed, (uint32_t)t, (uint32_t)k,
                                                   (uint64_t)(k + 1));
            int64_t tmp = perm[k];
            perm[k] = perm[j];
            perm[j] = tmp;
            int64_t q = -1;
            if (k % 2 == 0)
                q = k / 2;
            else if (k == 1)
                q = 0;
            if (q < 0)
                continue;
            int64_t u = perm[2 * q] / z, v = perm[2 * q + 1] / z;
            if (u == v) {
                simple = 0;
                break;
            }
            for (int s = 0; s < deg[u]; s++)
                if (nbr[u * z + s] == v)
                    simple = 0;
            if (!simple)
                break;
            nbr[u * z + deg[u]++] = (int32_t)v;
            nbr[v * z + deg[v]++] = (int32_t)u;
        }
        if (simple) {
            for (int64_t v = 0; v < N; v++)
                qsort(nbr + v * z, (size_t)z, sizeof(int32_t), ora_cmp_i32);
            *attempts_out = t + 1;
            free(perm);
            free(deg);
            return ORA_OK;
        }
    }
    free(perm);
    free(deg);
    *attempts_out = max_attempts;
    return ORA_EINVAL;
}

int ora_graph_edges(int64_t N, int z, const int32_t *nbr, int32_t *eu, int32_t *ev)
{
    int64_t e = 0;
    /* vertices in order, neighbours sorted ascending: (u, v) with u < v come
     * out in lexicographic order */
    for (int64_t u = 0; u < N; u++) {
        int32_t sorted[16];
        if (z > 16)
            return ORA_EINVAL;
        memcpy(sorted, nbr + u * z, (size_t)z * sizeof(int32_t));
        qsort(sorted, (size_t)z, sizeof(int32_t), ora_cmp_i32);
        for (int s = 0; s < z; s++) {
            if (sorted[s] > u) {
                eu[e] = (int32_t)u;
                ev[e] = sorted[s];
                e++;
            }
        }
    }
    return (e == N * z / 2) ? ORA_OK : ORA_EINVAL;
}

/* id of edge {a, b} by binary search in the lexicographic edge list */
static int64_t ora_edge_id(int64_t E, const int32_t *eu, const int32_t *ev, int32_t a, int32_t b)
{
    int32_t u = a < b ? a : b, v = a < b ? b : a;
    int64_t lo = 0, hi = E - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (eu[mid] < u || (eu[mid] == u && ev[mid] < v))
            lo = mid + 1;
        else if (eu[mid] > u || (eu[mid] == u && ev[mid] > v))
            hi = mid - 1;
        else
            return mid;
    }
    return -1;
}

int ora_graph_classes(int64_t N, int z, const int32_t *nbr, int64_t *class_off, int32_t *bu,
                      int32_t *bv, int64_t *bid, int64_t *nclass)
{
    int64_t E = N * z / 2;
    int32_t *eu = (int32_t *)malloc((size_t)E * sizeof(int32_t));
    int32_t *ev = (int32_t *)malloc((size_t)E * sizeof(int32_t));
    int32_t *colour = (int32_t *)malloc((size_t)E * sizeof(int32_t));
    int64_t *inc = (int64_t *)malloc((size_t)N * z * sizeof(int64_t));
    if (!eu || !ev || !colour || !inc) {
        free(eu);
        free(ev);
        free(colour);
        free(inc);
        return ORA_ENOMEM;
    }
    int rc = ora_graph_edges(N, z, nbr, eu, ev);
    if (rc != ORA_OK)
        goto done;
    /* incident edge ids of every vertex */
    for (int64_t v = 0; v < N; v++)
        for (int s = 0; s < z; s++)
            inc[v * z + s] = ora_edge_id(E, eu, ev, (int32_t)v, nbr[v * z + s]);

    /* greedy: each edge in id order takes the smallest colour not used by an
     * already coloured edge that touches u, v, or any neighbour of u or v */
    int32_t ncol = 0;
    for (int64_t e = 0; e < E; e++) {
        char used[512];
        memset(used, 0, sizeof(used));
        int32_t verts[2 + 2 * 16];
        int nv = 0;
        verts[nv++] = eu[e];
        verts[nv++] = ev[e];
        for (int s = 0; s < z; s++) {
            verts[nv++] = nbr[(int64_t)eu[e] * z + s];
            verts[nv++] = nbr[(int64_t)ev[e] * z + s];
        }
        for (int a = 0; a < nv; a++) {
            for (int s = 0; s < z; s++) {
                int64_t f = inc[(int64_t)verts[a] * z + s];
                if (f < e)
                    used[colour[f]] = 1;
            }
        }
        int32_t c = 0;
        while (used[c])
            c++;
        colour[e] = c;
        if (c + 1 > ncol)
            ncol = c + 1;
    }
    /* classes: colours ascending, edges in id order inside a class */
    int64_t nb = 0;
    for (int32_t c = 0; c < ncol; c++) {
        class_off[c] = nb;
        for (int64_t e = 0; e < E; e++) {
            if (colour[e] != c)
                continue;
            bu[nb] = eu[e];
            bv[nb] = ev[e];
            bid[nb] = e;
            nb++;
        }
    }
    class_off[ncol] = nb;
    *nclass = ncol;
done:
    free(eu);
    free(ev);
    free(colour);
    free(inc);
    return rc;
}

int ora_check_schedule(int64_t N, int z, const int32_t *nbr, int64_t nclass,
                       const int64_t *class_off, const int32_t *bu, const int32_t *bv)
{
    int64_t E = N * z / 2;
    int64_t *owner = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    int32_t *eu = (int32_t *)malloc((size_t)E * sizeof(int32_t));
    int32_t *ev = (int32_t *)malloc((size_t)E * sizeof(int32_t));
    int32_t *seen = (int32_t *)calloc((size_t)E, sizeof(int32_t));
    int bad = 0;
    if (!owner || !eu || !ev || !seen) {
        bad = ORA_ENOMEM;
        goto out;
    }
    if (ora_graph_edges(N, z, nbr, eu, ev) != ORA_OK) {
        bad = 10;
        goto out;
    }
    if (class_off[nclass] != E) {
        bad = 11;
        goto out;
    }
    for (int64_t c = 0; c < nclass; c++) {
        for (int64_t v = 0; v < N; v++)
            owner[v] = -1;
        /* endpoints are distinct between bonds of a class */
        for (int64_t b = class_off[c]; b < class_off[c + 1]; b++) {
            if (owner[bu[b]] != -1 || owner[bv[b]] != -1) {
                bad = 12;
                goto out;
            }
            owner[bu[b]] = b;
            owner[bv[b]] = b;
        }
        /* no endpoint of one bond neighbours an endpoint of another */
        for (int64_t b = class_off[c]; b < class_off[c + 1]; b++) {
            int32_t ends[2] = {bu[b], bv[b]};
            for (int e = 0; e < 2; e++)
                for (int s = 0; s < z; s++) {
                    int64_t w = nbr[(int64_t)ends[e] * z + s];
                    if (owner[w] != -1 && owner[w] != b) {
                        bad = 13;
                        goto out;
                    }
                }
        }
        /* each bond is an edge of the graph, seen once over the sweep */
        for (int64_t b = class_off[c]; b < class_off[c + 1]; b++) {
            int64_t id = ora_edge_id(E, eu, ev, bu[b], bv[b]);
            if (id < 0 || seen[id]) {
                bad = 14;
                goto out;
            }
            seen[id] = 1;
        }
    }
out:
    free(owner);
    free(eu);
    free(ev);
    free(seen);
    return bad;
}

/* ------------------------------------------------------------------ */
/* Dynamics                                                            */
/* ------------------------------------------------------------------ */

/* Rules (a)-(c) of section 2.1 with the random gate.  ci and cj count the
 * occupied neighbours of i other than j, and of j other than i. */
static void ora_rule(int m, int ni, int nj, int ci, int cj, int gate, int *ni_out, int *nj_out)
{
    *ni_out = ni;
    *nj_out = nj;
    if (!gate)
        return;
    if (ni == nj)
        return; /* rule (a): the target site must be empty */
    /* source s (occupied) and destination d (empty) */
    int c_src = ni ? ci : cj;
    int c_dst = ni ? cj : ci;
    int rule_b = (c_src + 0) <= m;     /* N(src) counts d, which is empty */
    int rule_c = (c_dst + 1) <= m + 1; /* N(dst) counts src, which is occupied */
    if (rule_b && rule_c) {
        *ni_out = nj;
        *nj_out = ni;
    }
}

int ora_local_move(int z, int m, int ni, int nj, const uint8_t *others_i, const uint8_t *others_j,
                   int gate, int *ni_out, int *nj_out)
{
    if (z < 1 || m < 0)
        return ORA_EINVAL;
    int ci = 0, cj = 0;
    for (int k = 0; k < z - 1; k++) {
        ci += others_i[k] ? 1 : 0;
        cj += others_j[k] ? 1 : 0;
    }
    ora_rule(m, ni ? 1 : 0, nj ? 1 : 0, ci, cj, gate ? 1 : 0, ni_out, nj_out);
    return ORA_OK;
}

typedef struct {
    uint64_t key;
    int64_t site;
} ora_keyed;

static int ora_cmp_keyed(const void *a, const void *b)
{
    const ora_keyed *x = (const ora_keyed *)a, *y = (const ora_keyed *)b;
    if (x->key != y->key)
        return x->key < y->key ? -1 : 1;
    return (x->site > y->site) - (x->site < y->site);
}

int ora_init(int64_t N, int64_t r0, int64_t Rs, uint64_t seed, int64_t K, uint8_t *n, uint8_t *n0,
             uint8_t *p)
{
    if (N < 1 || Rs < 0 || r0 < 0 || K < 0 || K > N)
        return ORA_EINVAL;
    ora_keyed *keys = (ora_keyed *)malloc((size_t)N * sizeof(ora_keyed));
    if (!keys)
        return ORA_ENOMEM;
    for (int64_t rr = 0; rr < Rs; rr++) {
        int64_t r = r0 + rr;
        /* replicas 2k and 2k+1 take the two halves of one Philox block */
        for (int64_t i = 0; i < N; i++) {
            uint32_t o[4];
            ora_philox_seeded(seed, (uint32_t)(r / 2), ORA_TAG_INIT, (uint32_t)i, 0u, o);
            if (r % 2 == 0)
                keys[i].key = (uint64_t)o[0] | ((uint64_t)o[1] << 32);
            else
                keys[i].key = (uint64_t)o[2] | ((uint64_t)o[3] << 32);
            keys[i].site = i;
        }
        qsort(keys, (size_t)N, sizeof(ora_keyed), ora_cmp_keyed);
        for (int64_t i = 0; i < N; i++)
            n[i * Rs + rr] = 0;
        for (int64_t k = 0; k < K; k++)
            n[keys[k].site * Rs + rr] = 1;
        for (int64_t i = 0; i < N; i++) {
            n0[i * Rs + rr] = n[i * Rs + rr];
            p[i * Rs + rr] = 1;
        }
    }
    free(keys);
    return ORA_OK;
}

int ora_class_step(int64_t N, int z, const int32_t *nbr, int m, int64_t nb, const int32_t *bu,
                   const int32_t *bv, const int64_t *bid, int64_t cls, int64_t t, uint64_t seed,
                   int64_t r0, int64_t Rs, int cubic_L, uint8_t *n, uint8_t *p)
{
    if (Rs <= 0)
        return ORA_OK;
    (void)N;
    int64_t w_first = r0 / 64, w_last = (r0 + Rs - 1) / 64;
    int64_t nw = w_last - w_first + 1;
    uint64_t *gate = (uint64_t *)malloc((size_t)nw * sizeof(uint64_t));
    if (!gate)
        return ORA_ENOMEM;
    for (int64_t b = 0; b < nb; b++) {
        int64_t i = bu[b], j = bv[b];
        for (int64_t w = w_first; w <= w_last; w++)
            gate[w - w_first] = cubic_L > 0 ? ora_cubic_gate_word(seed, t, cls, bid[b], w, cubic_L)
                                            : ora_gate_word(seed, t, cls, bid[b], w);
        for (int64_t rr = 0; rr < Rs; rr++) {
            int64_t r = r0 + rr;
            int g = (int)((gate[r / 64 - w_first] >> (r % 64)) & 1u);
            int ni = n[i * Rs + rr], nj = n[j * Rs + rr];
            int ci = 0, cj = 0;
            for (int s = 0; s < z; s++) {
                int64_t k = nbr[i * z + s];
                if (k != j)
                    ci += n[k * Rs + rr];
                k = nbr[j * z + s];
                if (k != i)
                    cj += n[k * Rs + rr];
            }
            int ni2, nj2;
            ora_rule(m, ni, nj, ci, cj, g, &ni2, &nj2);
            if (ni2 != ni) {
                n[i * Rs + rr] = (uint8_t)ni2;
                n[j * Rs + rr] = (uint8_t)nj2;
                p[i * Rs + rr] = 0;
                p[j * Rs + rr] = 0;
            }
        }
    }
    free(gate);
    return ORA_OK;
}

int ora_sweeps(int64_t N, int z, const int32_t *nbr, int m, int64_t nclass,
               const int64_t *class_off, const int32_t *bu, const int32_t *bv, const int64_t *bid,
               uint64_t seed, int64_t r0, int64_t Rs, int cubic_L, int64_t t0, int64_t nsweeps,
               uint8_t *n, uint8_t *p)
{
    for (int64_t s = 0; s < nsweeps; s++) {
        for (int64_t c = 0; c < nclass; c++) {
            int64_t off = class_off[c];
            int rc = ora_class_step(N, z, nbr, m, class_off[c + 1] - off, bu + off, bv + off,
                                    bid + off, c, t0 + s, seed, r0, Rs, cubic_L, n, p);
            if (rc != ORA_OK)
                return rc;
        }
    }
    return ORA_OK;
}

void ora_observe(int64_t N, int64_t Rs, const uint8_t *n, const uint8_t *n0, const uint8_t *p,
                 int64_t *counts)
{
    for (int64_t rr = 0; rr < Rs; rr++) {
        int64_t particles = 0, overlap = 0, persist_occ = 0, persist_all = 0;
        for (int64_t i = 0; i < N; i++) {
            int a = n[i * Rs + rr], b = n0[i * Rs + rr], c = p[i * Rs + rr];
            particles += a;
            overlap += a & b;
            persist_occ += b & c;
            persist_all += c;
        }
        counts[rr * 4 + 0] = particles;
        counts[rr * 4 + 1] = overlap;
        counts[rr * 4 + 2] = persist_occ;
        counts[rr * 4 + 3] = persist_all;
    }
}

int ora_four_point(int d, int L, int64_t Rs, const uint8_t *n, const uint8_t *n0, int64_t smax,
                   int64_t *phi, int64_t *psi)
{
    if (d < 1 || d > 4 || L < 2 || L % 2 || Rs < 1 || smax < 0) return 1;
    int64_t N = 1;
    for (int k = 0; k < d; k++) N *= L;
    for (int64_t x = 0; x < Rs * (smax + 1); x++) phi[x] = 0;
    for (int64_t s = 0; s <= smax; s++) psi[s] = 0;
    int64_t *M = (int64_t *)calloc((size_t)N, sizeof(int64_t));
    if (!M) return 2;
    for (int64_t i = 0; i < N; i++)
        for (int64_t rr = 0; rr < Rs; rr++) M[i] += n[i * Rs + rr] & n0[i * Rs + rr];
    for (int64_t i = 0; i < N; i++) {
        for (int64_t j = 0; j < N; j++) {
            /* shell of the pair: squared norm of the representative displacement */
            int64_t s = 0, a = i, b = j;
            for (int k = 0; k < d; k++) {
                int64_t dx = (b % L) - (a % L);
                a /= L;
                b /= L;
                if (dx < -L / 2) dx += L;
                if (dx >= L / 2) dx -= L;
                s += dx * dx;
            }
            if (s > smax) continue;
            psi[s] += M[i] * M[j];
            for (int64_t rr = 0; rr < Rs; rr++)
                phi[rr * (smax + 1) + s] +=
                    (n[i * Rs + rr] & n0[i * Rs + rr]) & (n[j * Rs + rr] & n0[j * Rs + rr]);
        }
    }
    free(M);
    return 0;
}

/* Uniform integer in [0, range) by Lemire's method on the Philox words of
 * counter (c0, tag, c2, draw), draw = 0, 1, ... until accepted. */
static uint64_t ora_bounded_at(uint64_t gseed, uint32_t c0, uint32_t tag, uint32_t c2,
                               uint64_t range)
{
    uint32_t draw = 0, o[4];
    ora_philox_seeded(gseed, c0, tag, c2, draw, o);
    uint64_t x = (uint64_t)o[0] | ((uint64_t)o[1] << 32);
    unsigned __int128 prod = (unsigned __int128)x * range;
    uint64_t low = (uint64_t)prod;
    if (low < range) {
        uint64_t threshold = (0 - range) % range;
        while (low < threshold) {
            draw++;
            ora_philox_seeded(gseed, c0, tag, c2, draw, o);
            x = (uint64_t)o[0] | ((uint64_t)o[1] << 32);
            prod = (unsigned __int128)x * range;
            low = (uint64_t)prod;
        }
    }
    return (uint64_t)(prod >> 64);
}

int ora_layered_graph(int d, int L, int M, uint64_t graph_seed, int32_t *nbr)
{
    if (d < 1 || d > 4 || L < 3 || M < 1 || M >= 65536) return ORA_EINVAL;
    int64_t N = 1;
    for (int k = 0; k < d; k++) N *= L;
    const int z = 2 * d;
    if ((int64_t)M * N * z > 0x7FFFFFFFLL) return ORA_EINVAL;
    int32_t *perm = (int32_t *)malloc((size_t)M * sizeof(int32_t));
    if (!perm) return ORA_ENOMEM;
    for (int64_t i = 0; i < N; i++) {
        for (int mu = 0; mu < d; mu++) {
            /* the base bond (i, i + e_mu), periodic */
            int64_t stride = 1;
            for (int k = 0; k < mu; k++) stride *= L;
            const int64_t x = (i / stride) % L;
            const int64_t j = (x == L - 1) ? i - (int64_t)(L - 1) * stride : i + stride;
            /* a uniform permutation of the M layers, Fisher-Yates from the top */
            for (int a = 0; a < M; a++) perm[a] = a;
            for (int k = M - 1; k >= 1; k--) {
                const int r = (int)ora_bounded_at(graph_seed, (uint32_t)i, ORA_TAG_LAYER,
                                                  ((uint32_t)mu << 16) | (uint32_t)k,
                                                  (uint64_t)(k + 1));
                const int tmp = perm[k];
                perm[k] = perm[r];
                perm[r] = tmp;
            }
            /* copy a of i is linked to copy perm[a] of j */
            for (int a = 0; a < M; a++) {
                const int64_t u = (int64_t)a * N + i, v = (int64_t)perm[a] * N + j;
                nbr[u * z + 2 * mu] = (int32_t)v;
                nbr[v * z + 2 * mu + 1] = (int32_t)u;
            }
        }
    }
    free(perm);
    return 0;
}

/* Attempt k of sweep t of word w in the random-sequential mode: a uniform
 * integer in [0, N z) by Lemire's method on the low 64 bits of the Philox
 * block at counter (t, 0xFFFFFFFC - draw, k, w), draw = 0, 1, ... */
static uint64_t ora_sequential_draw(uint64_t seed, uint32_t t, uint32_t k, uint32_t w,
                                    uint64_t range)
{
    uint32_t draw = 0, o[4];
    ora_philox_seeded(seed, t, ORA_TAG_SEQUENTIAL - draw, k, w, o);
    uint64_t x = (uint64_t)o[0] | ((uint64_t)o[1] << 32);
    unsigned __int128 prod = (unsigned __int128)x * range;
    uint64_t low = (uint64_t)prod;
    if (low < range) {
        uint64_t threshold = (0 - range) % range;
        while (low < threshold) {
            draw++;
            ora_philox_seeded(seed, t, ORA_TAG_SEQUENTIAL - draw, k, w, o);
            x = (uint64_t)o[0] | ((uint64_t)o[1] << 32);
            prod = (unsigned __int128)x * range;
            low = (uint64_t)prod;
        }
    }
    return (uint64_t)(prod >> 64);
}

int ora_sequential_sweeps(int64_t N, int z, const int32_t *nbr, int m, uint64_t seed, int64_t r0,
                          int64_t Rs, int64_t t0, int64_t nsweeps, uint8_t *n, uint8_t *p)
{
    if (N < 1 || z < 1 || m < 0 || r0 < 0 || Rs < 0 || (r0 % 64) != 0 || (Rs % 64) != 0 ||
        N * z > 0xFFFFFFFFLL)
        return ORA_EINVAL;
    for (int64_t w = 0; w < Rs / 64; w++) {
        const int64_t word = r0 / 64 + w;
        for (int64_t t = t0; t < t0 + nsweeps; t++) {
            for (int64_t k = 0; k < N; k++) {
                /* the bond: site i and its neighbour in slot s, shared by the
                 * 64 replicas of the word (section 3.2) */
                const uint64_t r = ora_sequential_draw(seed, (uint32_t)t, (uint32_t)k,
                                                       (uint32_t)word, (uint64_t)(N * z));
                const int64_t i = (int64_t)(r / (uint64_t)z);
                const int64_t j = nbr[i * z + (int64_t)(r % (uint64_t)z)];
                for (int64_t b = 0; b < 64; b++) {
                    const int64_t rr = w * 64 + b;
                    int ni = n[i * Rs + rr], nj = n[j * Rs + rr];
                    int ci = 0, cj = 0;
                    for (int s = 0; s < z; s++) {
                        int64_t x = nbr[i * z + s];
                        if (x != j) ci += n[x * Rs + rr];
                        x = nbr[j * z + s];
                        if (x != i) cj += n[x * Rs + rr];
                    }
                    int ni2, nj2;
                    ora_rule(m, ni, nj, ci, cj, 1, &ni2, &nj2);
                    if (ni2 != ni) {
                        n[i * Rs + rr] = (uint8_t)ni2;
                        n[j * Rs + rr] = (uint8_t)nj2;
                        p[i * Rs + rr] = 0;
                        p[j * Rs + rr] = 0;
                    }
                }
            }
        }
    }
    return ORA_OK;
}
