/*
 * ka.h -- C ABI of the GB300 multispin Kob-Andersen library.
 *
 * The library runs the Kob-Andersen kinetically constrained lattice gas of
 * Boccagna, "A Multispin Algorithm for the Kob-Andersen Stochastic Dynamics
 * on Regular Lattices" (arXiv 1710.05155) with multispin coding (section 3.1):
 * the occupation of one site in R independent replicas is stored as R/64
 * uint64 words, one bit per replica.  Replica r lives in word r / 64, bit
 * r % 64.
 *
 * Dynamics (section 2.1, rules (a)-(c); section 3.2).  A sweep runs a fixed
 * sequence of bond classes.  Each class is a strong matching (no two bonds
 * share a site or are joined by an edge), so its bonds are independent.  On a
 * bond (i, j) every replica exchanges n_i and n_j iff
 *   - exactly one of i, j is occupied                          (rule (a)),
 *   - the occupied site has at most m occupied neighbours      (rule (b)),
 *   - the empty site has at most m + 1 occupied neighbours     (rule (c)),
 *   - the replica's random gate bit for this attempt is 1.
 * Equivalently: at most m of the z-1 other neighbours of i are occupied, and
 * at most m of the z-1 other neighbours of j.  An exchange clears the
 * persistence bit of both sites.
 *
 * Random gates.  Philox4x32-10 (Salmon et al., SC'11), key = (seed low 32,
 * seed high 32); a block at counter (c0, c1, c2, c3) has halves
 * half 0 = x0 | x1 << 32 and half 1 = x2 | x3 << 32.  The gate word that
 * replica word w of a bond uses at sweep t is:
 *   - graphs (random regular and caller graphs): half (w mod 2) of the block
 *     at counter (t, c, e, w / 2), c the bond's class and e its edge id;
 *   - cubic lattices: classes pair up as (4g + 2b, 4g + 2b + 1), b in {0, 1},
 *     g = 2 mu + p the group.  A bond of class c with base site i takes half
 *     (c mod 2) of the block at counter (t, c - (c mod 2), i - (c mod 2) L^mu,
 *     w): the bonds at pencil positions 4k + 2b and 4k + 2b + 1 of one pencil
 *     share the block keyed by the base site of the first, and every word w
 *     has its own block.
 *
 * Cubic schedule (d-dimensional periodic lattice, L % 4 == 0, site index
 * i = sum_k x_k L^k).  Class c = (2 mu + p) * 4 + a, for mu < d, p in {0, 1}
 * (only p = 0 when d = 1) and a < 4, holds the bonds (x, x + e_mu) with
 * x_mu = a mod 4 and sum_{nu != mu} x_nu = p mod 2.  Classes run in
 * ascending c.
 *
 * Graph schedule (random regular graphs and caller graphs).  Edges (u < v)
 * sorted lexicographically get ids 0..E-1; a greedy strong edge colouring in
 * id order gives the classes, run in ascending colour.
 *
 * Random regular graphs: configuration model (section 2.1, Bollobas); stubs
 * are shuffled by Fisher-Yates with Lemire's bounded integers from Philox
 * counter (attempt, 0xFFFFFFFE, k, draw) keyed by graph_seed, paired
 * (2q, 2q+1), and the whole attempt is rejected on any self-loop or
 * multi-edge.  This samples simple z-regular graphs uniformly.
 *
 * Initial state (section 3.1: draw a configuration at density rho at
 * random): K = round-half-away(rho N) particles per replica at the K sites
 * with the smallest (key, site), key = half (r mod 2) of the Philox block at
 * counter (r / 2, 0xFFFFFFFF, site, 0) keyed by seed.  n0 = n, p = all ones.
 *
 * Observables (section 2.2 overlap q_i = n_i(t) n_i(0); section 3.3 popcounts):
 * per replica, int64 [R][4] = { sum n, sum n & n0, sum n0 & p, sum p }.
 * C(t) = mean_r (overlap_r - N rho^2) / (N rho (1 - rho)) with rho = K / N.
 *
 * Errors.  Every entry point returns a ka_status; no exception crosses the
 * ABI.  Kernel faults surface as KA_ECUDA at the next call that synchronises
 * (ka_observe, ka_get_state, ka_sync, ka_destroy).  ka_last_error gives a
 * message.  A context is not thread-safe; distinct contexts are independent.
 * All device work of a context is issued on its stream, in call order.
 */
#ifndef KA_H
#define KA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KA_OK = 0,
    KA_EINVAL = 1,   /* bad argument or unsupported parameter set */
    KA_ENOMEM = 2,   /* device or host allocation failed, or buffer too small */
    KA_ECUDA = 3,    /* CUDA runtime or kernel error */
    KA_ETIMEOUT = 4, /* a bounded device wait ran out */
    KA_EBUSY = 5,    /* resource budget exhausted (admission refused) */
    KA_ESTATE = 6    /* call out of order (e.g. sweep before init) */
} ka_status;

typedef enum {
    KA_CUBIC = 0, /* periodic d-dimensional cubic lattice, z = 2d */
    KA_RRG = 1,   /* random z-regular graph built from graph_seed */
    KA_GRAPH = 2  /* caller-supplied simple z-regular graph (nbr) */
} ka_topology;

/* flags */
#define KA_FLAG_GENERIC 1 /* cubic lattices: use the edge-gather kernel, not the pencil kernel */

typedef struct {
    int32_t topo;        /* ka_topology */
    int32_t d;           /* cubic: 1 <= d <= 4 */
    int32_t L;           /* cubic: L >= 4, L % 4 == 0, L^d < 2^31 */
    int32_t z;           /* graphs: 1 <= z <= 8, z < N (cubic: ignored, z = 2d) */
    int64_t N;           /* graphs: number of vertices, N z even, N z < 2^32 (cubic: ignored) */
    int32_t m;           /* activation number, 0 <= m <= z - 1 (section 2.1) */
    int32_t replicas;    /* R, a positive multiple of 64 */
    uint64_t graph_seed; /* KA_RRG */
    const int32_t *nbr;  /* KA_GRAPH: host array [N][z], copied at create (rows kept in
                            ascending order); else NULL.  The rows must describe a simple
                            undirected graph: v in row u iff u in row v, no self-loop, no
                            repeated entry; ka_create returns KA_EINVAL otherwise */
    void *stream;        /* cudaStream_t for all work of the context; NULL = legacy default */
    int32_t device;      /* CUDA device ordinal */
    int32_t flags;       /* KA_FLAG_* */
} ka_params;

typedef struct ka_ctx ka_ctx;

typedef struct {
    int64_t N;          /* sites */
    int32_t z;          /* neighbours per site */
    int32_t m;          /* activation number */
    int32_t replicas;   /* R */
    int32_t words;      /* R / 64 */
    int64_t nclass;     /* bond classes per sweep */
    int64_t nbonds;     /* bonds per sweep = N z / 2 */
    int64_t sweep;      /* sweeps completed since init (or set_state) */
    int64_t K;          /* particles per replica at the last init (-1 if none) */
    uint64_t seed;      /* dynamics seed */
    int32_t kernel;     /* 0 = general cubic pencil kernel, 1 = edge-gather kernel,
                           3 = group kernels of three-dimensional lattices (d = 3,
                           L % 4 == 0, L <= 128: from two planes up, and for one
                           plane at the sides where they are measured faster) */
    int32_t rrg_attempts; /* configuration-model attempts (KA_RRG) */
    size_t device_bytes;  /* device memory the context uses */
    int32_t planes;       /* device state planes per array */
    int32_t plane_words;  /* words per site in one plane */
    int32_t planes_per_launch; /* planes one sweep launch covers (cubic group
                                  launches per class group and sweep:
                                  ceil(planes / planes_per_launch)) */
} ka_info_t;

/* Device bytes ka_create_in needs for these parameters. */
ka_status ka_required_bytes(const ka_params *params, size_t *bytes);

/* Create a context; the library allocates its device memory with cudaMalloc
 * and frees it in ka_destroy.  Builds the graph and its bond classes on the
 * host (KA_RRG, KA_GRAPH) and uploads them.  *out is NULL on failure. */
ka_status ka_create(const ka_params *params, ka_ctx **out);

/* As ka_create, but all device memory is carved from the caller's buffer
 * (at least ka_required_bytes, 256-byte aligned).  The caller keeps
 * ownership and must keep the buffer alive until ka_destroy. */
ka_status ka_create_in(const ka_params *params, void *device_buffer, size_t bytes, ka_ctx **out);

/* Initial state at density rho in [0, 1] with dynamics seed `seed`; resets
 * the sweep counter to 0.  Asynchronous on the context stream. */
ka_status ka_init(ka_ctx *ctx, uint64_t seed, double rho);

/* Run n >= 0 sweeps (every class once, in order).  Asynchronous.  The sweep
 * counter must stay below 2^32 (it is a Philox counter word). */
ka_status ka_sweep(ka_ctx *ctx, int64_t n);

/* n sweeps of the paper's random-sequential schedule (section 3.2) instead
 * of the class schedule: each attempt picks one bond, shared by the 64
 * replicas of a word, and exchanges the two sites in every replica where the
 * rule of section 2.1 allows it (no gate); N attempts make a sweep.  Attempt
 * k of sweep t of word w draws r uniform in [0, N z) by Lemire's method on
 * the low 64 bits of Philox4x32-10 at counter (t, 0xFFFFFFFC - draw, k, w),
 * key = the dynamics seed, draw = 0, 1, ... until accepted, and takes site
 * i = r / z and its neighbour in slot r mod z (on cubic lattices slot 2 mu is
 * the up and 2 mu + 1 the down neighbour along mu; on graphs the slots are
 * the neighbour row in ascending order, as ka_graph_tables returns it).  One warp per word runs
 * the chain, 32 attempts at a time, applying together the attempts that do
 * not touch each other's sites (the result is the in-order chain's), in
 * shared memory when the lattice has at most 10240 sites.  Advances the sweep
 * counter; no synchronisation.  KA_ESTATE before init, KA_EINVAL if
 * N z >= 2^32. */
ka_status ka_sweep_sequential(ka_ctx *ctx, int64_t n);

/* Observables of the current state into host int64 counts[R][4]; writes the
 * sweep counter to *sweep_out (may be NULL).  Synchronises the stream. */
ka_status ka_observe(ka_ctx *ctx, int64_t *sweep_out, int64_t *counts);

/* Observables into a device buffer int64 [R][4] (overwritten), no
 * synchronisation. */
ka_status ka_observe_device(ka_ctx *ctx, int64_t *counts_device);

/* Four-point correlations of a cubic lattice (section 2.2 g_4(r, t); section
 * 3.3 Phi(r, t)) between the current state and the initial one.  With
 * q_i = n_i AND n0_i per replica and M_i = the number of replicas with
 * q_i = 1, every ordered site pair (i, j) is counted once, in the shell
 * s = |delta|^2 of the representative of its displacement with every
 * component in [-L/2, L/2):
 *   phi[r * (smax + 1) + s] = sum over pairs in shell s of q_i q_j  (replica r)
 *   psi[s]                  = sum over pairs in shell s of M_i M_j
 * for s = 0 .. smax (shells without lattice vectors stay 0; pairs beyond
 * smax are not counted).  g_4 of shell s is (sum_r phi[r][s] / R - psi[s] /
 * R^2) / (N rho^2 (1 - rho)^2); summed over all shells it is chi_4.
 * phi: host int64 [R][smax + 1], required; psi: host int64 [smax + 1] or
 * NULL.  0 <= smax <= d (L/2)^2 and at most 65536 displacement vectors with
 * |delta|^2 <= smax, else KA_EINVAL; KA_EINVAL on graphs, KA_ESTATE before
 * init.  Uses stream-ordered scratch memory on the context's device,
 * released before return; synchronises the stream. */
ka_status ka_four_point(ka_ctx *ctx, int32_t smax, int64_t *phi, int64_t *psi);

/* Copy the state to host arrays in canonical layout [R/64][N] uint64 each
 * (word-plane major).  Any pointer may be NULL.  Synchronises. */
ka_status ka_get_state(ka_ctx *ctx, uint64_t *n, uint64_t *n0, uint64_t *p);

/* Load a state from host arrays in canonical layout; sets the sweep counter.
 * n, n0 and p are all required.  Synchronises. */
ka_status ka_set_state(ka_ctx *ctx, const uint64_t *n, const uint64_t *n0, const uint64_t *p,
                       int64_t sweep, uint64_t seed);

/* ka_set_state without the synchronisation: the copies (and, for V > 1, the
 * layout conversion) are queued on the context's stream and the call
 * returns.  The host arrays must stay valid and unchanged until that work
 * has run (ka_sync, or any later synchronising call on the context).  From
 * page-locked host memory the copies run asynchronously to the host and can
 * overlap other streams' kernels; from pageable memory the call may return
 * only once they are done.  Errors as ka_set_state; copy errors may also
 * surface at the next synchronising call. */
ka_status ka_set_state_async(ka_ctx *ctx, const uint64_t *n, const uint64_t *n0,
                             const uint64_t *p, int64_t sweep, uint64_t seed);

/* Wait for all work of the context; reports deferred kernel errors. */
ka_status ka_sync(ka_ctx *ctx);

/* Context description. */
ka_status ka_info(const ka_ctx *ctx, ka_info_t *out);

/* Host copies of the topology: nbr [N][z], class_off [nclass+1],
 * bu / bv / bid [nbonds] (bonds grouped by class, in class order).  Any
 * pointer may be NULL. */
ka_status ka_graph_tables(const ka_ctx *ctx, int32_t *nbr, int64_t *class_off, int32_t *bu,
                          int32_t *bv, int64_t *bid);

/* Host only (no device, no context): build the topology of `params` as
 * ka_create would and report its size; copy the tables into the non-NULL
 * buffers.  Capacities: nbr N*z, class_off nbonds+1 (the class count of a
 * random graph is known only after colouring), bu / bv / bid nbonds. */
ka_status ka_build_topology(const ka_params *params, int64_t *nclass, int64_t *nbonds,
                            int32_t *nbr,
                      int64_t *class_off, int32_t *bu, int32_t *bv, int64_t *bid);

/* Host only: neighbour rows nbr[M L^d][2d] (int32, caller-allocated) of the
 * layered random graph of section 5.2, to be run as a KA_GRAPH topology with
 * N = M L^d and z = 2d.  M copies of the periodic cubic lattice of side L in
 * d dimensions, vertex a L^d + i being site i of copy a; for every base bond
 * (i, i + e_mu) the M links between the copies of i and those of j = i + e_mu
 * are rewired by a uniform permutation pi of the copies, independent per
 * bond: copy a of i is linked to copy pi(a) of j.  pi is drawn by
 * Fisher-Yates from the top, step k taking a uniform integer in [0, k] by
 * Lemire's method on the low 64 bits of Philox4x32-10 at counter
 * (i, 0xFFFFFFFD, mu << 16 | k, draw), key = graph_seed, draw = 0, 1, ...
 * until accepted.  Entry 2 mu of a row is the neighbour across the up bond
 * along mu, entry 2 mu + 1 across the down bond.  M = 1 gives the lattice.
 * KA_EINVAL unless 1 <= d <= 4, L >= 3, 1 <= M < 65536, M L^d 2d < 2^31. */
ka_status ka_layered_graph(int32_t d, int32_t L, int32_t M, uint64_t graph_seed, int32_t *nbr);

/* Kernel timing for roofline reports.  When enabled, ka_sweep brackets
 * every sweep-kernel launch with CUDA events on the context stream (the
 * events sit between launches that would otherwise overlap their prologues,
 * so the times are those of launches run one after the other).
 * ka_profile_read synchronises and returns the summed kernel time (ms) and
 * the number of launches since the last read; ka_profile_read_dirs returns
 * the same split by bond direction: host arrays kernel_ms[4] and
 * launches[4], entry mu for the group launches of direction mu on cubic
 * lattices, entry 0 for every class launch on graphs.  Either read clears
 * all sums.  KA_EINVAL for a NULL context; KA_ECUDA if an event fails. */
ka_status ka_profile_enable(ka_ctx *ctx, int32_t enable);
ka_status ka_profile_read(ka_ctx *ctx, double *kernel_ms, int64_t *launches);
ka_status ka_profile_read_dirs(ka_ctx *ctx, double *kernel_ms, int64_t *launches);

/* Destroy a context (NULL is fine).  Synchronises; returns a deferred
 * kernel error if one is pending. */
ka_status ka_destroy(ka_ctx *ctx);

/* ------------------------------------------------------------------------
 * Batched and served execution
 *
 * A batch holds many independent jobs (each a context with its own
 * topology, density, seed, replica count and sweep target) resident on one
 * device, and advances them together: one kernel launch runs a bond-class
 * group of every three-dimensional job of the same side and m (the group
 * kernels, one table entry per job plane), or of every other small cubic
 * job of the same shape class (d, words per plane, m), and one launch runs
 * a colour class of every graph job of the same (words per plane, m).  A
 * cubic job whose groups have at least the batch's own-launch threshold of
 * tiles (ka_batch_tuning; ka_batch_autotune sets it) runs with its own
 * launches inside each round.  Each job's result is bit-identical to running it alone:
 * the random streams are keyed by the job's seed, sweep, class and site,
 * never by its position in the batch.  The paper has no batching; this is
 * the serving layer around its method.  A batch is not thread-safe: call its
 * functions from one host thread at a time (contexts for ka_batch_adopt may
 * be created and initialised on other threads).
 * ------------------------------------------------------------------------ */
typedef struct ka_batch ka_batch;

typedef struct {
    int64_t sweeps;        /* sweeps to run, >= 0 */
    int64_t observe_every; /* observe after every this many sweeps (>= 1), and at the end */
    uint64_t seed;         /* dynamics seed (ka_init) */
    double rho;            /* density (ka_init) */
} ka_job_spec;

#define KA_BATCH_GRAPH 1 /* capture each round in a CUDA graph and replay it */
#define KA_BATCH_PLAIN 2 /* run every job with its own launches (the unbatched reference) */

/* Create a batch on `device` whose jobs may use at most hbm_budget bytes of
 * device memory (contexts plus observation buffers).  All work is issued on
 * `stream` (cudaStream_t or NULL). */
ka_status ka_batch_create(int32_t device, void *stream, size_t hbm_budget, int32_t flags,
                          ka_batch **out);

/* Admit a job: allocates its context and observation buffer, builds its
 * topology, draws its initial state and records the sweep-0 observation.
 * KA_EBUSY (nothing allocated) when the job would exceed the budget. */
ka_status ka_batch_add(ka_batch *b, const ka_params *params, const ka_job_spec *spec,
                       int64_t *job_id);

/* Device bytes a job takes from a batch's budget: its context
 * (ka_required_bytes) plus its observation buffer of
 * (sweeps / observe_every + 2) * replicas * 4 int64. */
ka_status ka_job_bytes(const ka_params *params, const ka_job_spec *spec, size_t *bytes);

/* Admit a job whose context already exists, so that topologies and initial
 * states can be prepared on other host threads (each with its own stream)
 * while the batch runs.  ctx must come from ka_create (the batch takes
 * ownership and frees it on removal), be initialised (ka_init or
 * ka_set_state) and live on the batch's device.  spec->sweeps is the target
 * sweep count (absolute, >= the context's sweep); spec->seed and rho are not
 * used.  The context's stream is synchronised and replaced by the batch's,
 * and the first observation is recorded at the context's current sweep.
 * KA_EBUSY when over budget, KA_EINVAL for a context the batch cannot own;
 * on any error the context stays the caller's. */
ka_status ka_batch_adopt(ka_batch *b, ka_ctx *ctx, const ka_job_spec *spec, int64_t *job_id);

/* One round: advance every unfinished job by up to max_sweeps sweeps (a job
 * stops early at its next observation point or its target), then record
 * the due observations.  *sweeps_run = the round's length.  Synchronises. */
ka_status ka_batch_step(ka_batch *b, int64_t max_sweeps, int64_t *sweeps_run);

/* Tune the live batch by timing real rounds, in two stages: (1) which cubic
 * jobs run with their own launches -- the tile threshold (one wave of
 * tiles, half, a quarter, an eighth, or none on their own launches), at the
 * present round length; (2) the round length (4, 16, 64 sweeps) with the
 * chosen threshold.  Each candidate first runs warm-up rounds (tables; in
 * graph mode the capture), then one timed round; all these rounds do real
 * work.  The fastest of each stage is kept (ka_batch_tuning);
 * *best_round = the round length, may be NULL.  Results do not depend on
 * the tuning. */
ka_status ka_batch_autotune(ka_batch *b, int64_t *best_round);

/* The batch's present tuning: the round length ka_batch_step(b, 0, ...)
 * takes, and the tile threshold above which a cubic job runs with its own
 * launches inside each round instead of sharing the batched launches (in
 * tiles of eight one-word pencils; before autotuning: one wave of tiles,
 * twice the SM count).  Either pointer may be NULL. */
ka_status ka_batch_tuning(const ka_batch *b, int64_t *round_sweeps, int64_t *own_tiles);

/* Progress of a job. */
ka_status ka_batch_poll(const ka_batch *b, int64_t job_id, int64_t *sweep, int32_t *finished);

/* Observations of a job: *n_obs; if obs_sweeps / counts are non-NULL they
 * receive the sweep of each observation [n_obs] and the counts
 * [n_obs][R][4] (as ka_observe). */
ka_status ka_batch_observations(const ka_batch *b, int64_t job_id, int64_t *n_obs,
                                int64_t *obs_sweeps, int64_t *counts);

/* State of a job (its current sweep: ka_batch_poll) copied to host arrays in
 * the canonical layout of ka_get_state, [R/64][N] uint64 each; any pointer
 * may be NULL.  Synchronises the batch stream.  KA_EINVAL for an unknown
 * job; the status of ka_get_state otherwise (a deferred device error of the
 * job's launches included). */
ka_status ka_batch_state(ka_batch *b, int64_t job_id, uint64_t *n, uint64_t *n0, uint64_t *p);

/* Retire a job and free its memory (finished or not). */
ka_status ka_batch_remove(ka_batch *b, int64_t job_id);

/* Device bytes in use, jobs held, jobs still running. */
ka_status ka_batch_info(const ka_batch *b, size_t *used_bytes, int64_t *jobs, int64_t *active);

/* Free everything (NULL is fine). */
ka_status ka_batch_destroy(ka_batch *b);

/* Observables computed without allocating any memory.
 *
 * For callers that cannot call cudaMalloc -- code running where the device
 * heap is reserved or allocation is forbidden, such as inside another
 * framework's memory pool, a real-time loop, or a driver that has already
 * committed every byte -- this variant of ka_observe uses no memory of its
 * own: its per-replica accumulators live in a fixed array compiled into the
 * library (128 KiB, enough for 4096 replicas), which every GPU that loads
 * the library keeps until the process exits.  The paper has no counterpart;
 * it is a deployment convenience.
 *
 * n, n0, p: device arrays in the canonical layout [R/64][N] uint64 (the
 * layout of ka_get_state), read only.  counts: host int64 [R][4], written
 * as by ka_observe.  stream: cudaStream_t or NULL.  Synchronises the stream.
 * Returns KA_EINVAL when replicas is not a multiple of 64 or exceeds 4096,
 * or when stream belongs to another device than the current one (the array
 * used is the current device's).  The first call on a device looks up the
 * array's device address (with that device current, once, safely from any
 * host thread).  Every call copies the counts to the host and synchronises
 * the stream, so no call may be made while the stream is being captured.
 * All calls share the one array, which keeps the last call's contents (each
 * call clears it first), so calls that overlap on the GPU -- concurrent
 * streams or host threads -- race and must be serialised by the caller. */
ka_status ka_observe_static(const uint64_t *n, const uint64_t *n0, const uint64_t *p, int64_t N,
                            int32_t replicas, int64_t *counts, void *stream);

/* Message of the last failed call on this context (never NULL). */
const char *ka_last_error(const ka_ctx *ctx);

/* Human-readable name of a status code. */
const char *ka_status_name(ka_status s);

#ifdef __cplusplus
}
#endif
#endif
