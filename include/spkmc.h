/*
 * spkmc.h -- C ABI of the GB300 spkMC library (libspkmc.so).
 *
 * The library runs the synchronous parallel kinetic Monte Carlo (spkMC) cycle
 * of Martinez, Monasterio and Marian, arXiv:1005.4713, Sec. 3.1 (steps 1-6)
 * with the chessboard sublattice of Sec. 3.2, on periodic simple-cubic 3D
 * Ising lattices (Eq. 1) with Glauber rates (Eq. 3), on one CUDA GPU.
 *
 * Conventions shared by every entry point:
 *   - lattice edge L, domain edge d, nd = L/d domains per axis; L % (2d) == 0
 *     (nd even, so the 8 colours tile the lattice) and d in {2, 4, 8, 16};
 *   - site (X,Y,Z), global index g = X + L*(Y + L*Z) (x fastest); spins are
 *     exchanged with the host as int8 +1/-1 in that order;
 *   - domain (dx,dy,dz), index k = dx + nd*(dy + nd*dz); local site
 *     l = x + d*(y + d*z); sublattices of Sec. 3.2 step 4a
 *     (spkmc_params.sublattice): eight colours, colour = (dx&1) | (dy&1)<<1 |
 *     (dz&1)<<2, cycle t works on colour t % 8 (deterministic rotation, the
 *     default); or two colours, colour = (dx+dy+dz) & 1, cycle t works on
 *     the colour given by the top bit of Philox word 0 at counter (t, 0, 5, 0)
 *     (the paper's random choice);
 *   - class of a site = 7*[sigma = +1] + (number of up neighbours), 0..13;
 *     rate r = 1/(1 + exp(2 sigma (J S + H) / T)), S = sum of the 6
 *     neighbour spins, lambda = 1, k_B = 1 (Eq. 3 read as Glauber dynamics);
 *   - random numbers: Philox4x64-10 keyed by (seed, 0); counter (t, k, 1, 0)
 *     for the event of domain k in cycle t, (t, 0, 2, 0) for the clock,
 *     (g/256, 0, 3, 0) for the hot start;
 *   - every active domain's frequency line is padded with a null rate to a
 *     common R (Sec. 3.1 step 3): the exact R_max of the cycle (Sec. 3.1
 *     step 2), or one of the bounds of Sec. 3.2 step 4b (spkmc_params
 *     rmax_mode), which need no device-wide reduction before the events.
 *
 * Ownership: the library owns all device memory it allocates (through the
 * optional allocator callbacks of spkmc_config, else stream-ordered
 * cudaMallocAsync) and runs all work on the configured stream.  Host buffers
 * passed in belong to the caller and are not retained after the call returns.
 *
 * Errors: every int-returning entry point returns SPKMC_OK (0) or one of the
 * codes below; spkmc_last_error() gives a thread-local message.  A handle is
 * never left partially constructed: a failed create returns no handle.
 * Work is asynchronous on the stream: errors raised inside a kernel (a grid
 * barrier that timed out, an internal inconsistency) are reported by the next
 * entry point that synchronises (spkmc_synchronize, spkmc_observables,
 * spkmc_get_*), after which the handle refuses to run until spkmc_set_state.
 */
#ifndef SPKMC_H
#define SPKMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPKMC_OK 0
#define SPKMC_EINVAL 1    /* invalid argument (message says which) */
#define SPKMC_ENOMEM 2    /* device or host allocation failed */
#define SPKMC_ECUDA 3     /* a CUDA runtime call failed */
#define SPKMC_ETIMEOUT 4  /* a grid barrier gave up after its time limit */
#define SPKMC_EBUSY 5     /* no free slot, or the budget does not allow it */
#define SPKMC_EINTERNAL 6 /* the device found its class counts inconsistent */
#define SPKMC_EBOUND 7    /* an active domain's R_k exceeded the R_max bound */

#define SPKMC_INIT_HOT 0  /* uniform +-1 spins from Philox (g/256, 0, 3, 0) */
#define SPKMC_INIT_COLD 1 /* all spins +1 (the relaxation start of Sec. 6) */

/* The rate R every active domain's frequency line is padded to (Sec. 3.2,
 * step 4b).  With R above the exact R_max the events keep their relative
 * probabilities and only the null fraction grows.
 *   EXACT:      R = max over the cycle's active domains of R_k (Sec. 3.1
 *               step 2); one device-wide reduction per cycle before events.
 *   PRESCRIBED: R = R' = d^3 * max_c r_c * (1 + 2^-32), the maximum aggregate
 *               rate of a domain, with E_max = -2(6|J| + |H|) (the printed
 *               -|H| read as +|H|); no reduction at all.
 *   LEARNED:    R = min(R', (R_max(t-8) + m) * (1 + 2^-32)) once colour t%8
 *               has a recorded visit (R' before): R_max(t-8) is the exact
 *               maximum of the same colour at its previous visit, reduced in
 *               the background, and m = a + 12 b bounds how much a domain's
 *               R_k can grow between two visits (a = max_S |r(+1,S) -
 *               r(-1,S)| for the flipped site, b = max |r(s,S+2) - r(s,S)|
 *               for each of the 12 sites whose neighbour sum moves).  This is
 *               the self-learning bound of Sec. 3.2 with a tolerance that
 *               provably keeps R >= R_k.
 * The factor 1 + 2^-32 covers the rounding of the 14-term sum R_k.  Every
 * active domain checks R_k <= R; a violation stops the lattice with
 * SPKMC_EBOUND (it cannot happen unless the state was altered). */
#define SPKMC_RMAX_EXACT 0
#define SPKMC_RMAX_PRESCRIBED 1
#define SPKMC_RMAX_LEARNED 2

/* Sublattice scheme of Sec. 3.2 step 4a.  EIGHT_ROTATING: K/8 active domains
 * per cycle, colours in rotation; class counts are kept up to date flip by
 * flip.  TWO_RANDOM: K/2 active domains per cycle, colour drawn per cycle;
 * an inactive site can then see flips in up to three neighbouring domains
 * in one cycle, so the class counts of an active domain are recounted from
 * its spins at the start of its cycle instead (the linear frequency-line
 * evaluation of Sec. 3.1 step 1).  The LEARNED bound needs EIGHT_ROTATING
 * (it relies on one visit of every colour in any eight cycles). */
#define SPKMC_SUBLATTICE_8_ROTATING 0
#define SPKMC_SUBLATTICE_2_RANDOM 1

typedef struct spkmc_engine spkmc_t;
typedef struct spkmc_batch spkmc_batch_t;
typedef struct spkmc_graph spkmc_graph_t;

/* Allocator callbacks: alloc returns device memory of at least `bytes` bytes
 * usable on `stream` (NULL on failure); free releases it.  `ctx` is passed
 * through unchanged. */
typedef void *(*spkmc_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*spkmc_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);

/* Physics and start state of one lattice (Eq. 1, Eq. 3). */
typedef struct spkmc_params {
    int32_t L;                  /* lattice edge */
    int32_t domain_edge;        /* d in {2,4,8,16}; 0 = pick by a fixed rule */
    double J;                   /* coupling (finite) */
    double H;                   /* field (finite) */
    double T;                   /* temperature in J/k_B units (> 0, finite) */
    uint64_t seed;              /* Philox key word 0 */
    int32_t init;               /* SPKMC_INIT_HOT or SPKMC_INIT_COLD */
    int32_t rmax_mode;          /* SPKMC_RMAX_EXACT (default), _PRESCRIBED or _LEARNED */
    int64_t event_log_capacity; /* events kept (see spkmc_event); 0 = off */
    int32_t sublattice;         /* SPKMC_SUBLATTICE_8_ROTATING (default) or _2_RANDOM */
    int32_t reserved1;          /* 0 */
} spkmc_params;

/* Engine runtime: stream, allocator and launch geometry. */
typedef struct spkmc_config {
    void *stream;               /* cudaStream_t; NULL = a stream of the library's own */
    spkmc_alloc_fn alloc;       /* NULL = cudaMallocAsync on the stream */
    spkmc_free_fn free;
    void *alloc_ctx;
    int32_t device;             /* CUDA device ordinal; -1 = current device */
    int32_t ctas_per_sm;        /* persistent grid: CTAs per SM; 0 = occupancy limit */
    int32_t max_ctas;           /* cap on the grid; 0 = no cap */
    int32_t items_per_cta;      /* target active domains per CTA; 0 = 64 */
    int64_t barrier_timeout_ns; /* grid-barrier time limit; 0 = 2 s */
    int32_t debug_skip_arrival_cta; /* fault test: that CTA never arrives; -1 = off */
    int32_t reserved1;
} spkmc_config;

/* Observables (Eq. 1, Eq. 4, Eq. 7 moments and the Eq. 10 counters). */
typedef struct spkmc_obs {
    int64_t cycle;              /* cycles done */
    double clock;               /* sum of dt = -ln(xi)/R_max (Sec. 3.1 step 5) */
    int64_t M;                  /* sum of spins */
    int64_t B;                  /* sum over sites of sigma_i (sigma_{+x}+sigma_{+y}+sigma_{+z}) */
    double E;                   /* -J*B - H*M */
    double m;                   /* M / N */
    double m2;                  /* m^2 */
    double m4;                  /* m^4 */
    int64_t n_flip;             /* flip events so far */
    int64_t n_null;             /* null events so far */
    double sum_null_rate;       /* sum over cycles and active domains of R_max - R_k */
    uint64_t sum_null_rate_fx[2]; /* the same, exact: sum of floor((R_max-R_k) 2^64), lo, hi */
    int32_t L;
    int32_t domain_edge;
} spkmc_obs;

/* One event of one active domain in one cycle (debug and parity log). */
typedef struct spkmc_event {
    int64_t cycle;              /* lattice-local cycle t */
    int32_t domain;             /* k */
    int32_t cls;                /* chosen class 0..13, or -1 for the null event */
    int32_t site;               /* local site l of the flipped spin, or -1 */
    int32_t reserved;
} spkmc_event;

/* Checkpoint scalars; spins are saved with spkmc_get_spins. */
typedef struct spkmc_state {
    int64_t cycle;
    double clock;
    int64_t n_flip;
    int64_t n_null;
    uint64_t sum_null_rate_fx[2];
    double rmax_hist[8];        /* exact R_max of cycles cycle-8 .. cycle-1 (0 = not run);
                                   the history of the LEARNED bound */
} spkmc_state;

/* Sizes of a created lattice. */
typedef struct spkmc_info {
    int32_t L, domain_edge, nd, reserved;
    int64_t K;                  /* domains */
    int64_t K_act;              /* active domains (events) per cycle: K/8, or K/2 with two colours */
    int64_t device_bytes;       /* device memory held for this lattice */
    int32_t grid_ctas;          /* CTAs of the persistent launch */
    int32_t threads_per_cta;
} spkmc_info;

/* ---- defaults ---------------------------------------------------------- */
void spkmc_params_init(spkmc_params *p);   /* L=16, d=4, J=1, H=0, T=4.5115, seed=1, hot */
void spkmc_config_init(spkmc_config *c);   /* all defaults (NULL stream, own allocator) */

/* Host-side rate table r[14] of Eq. 3 (read as Glauber), class order above,
 * evaluated in FP64 with the C library's exp.  Returns EINVAL unless T > 0
 * and J, H, T are finite. */
int spkmc_rate_table(double J, double H, double T, double out[14]);

/* The bounds of Sec. 3.2 step 4b for domain edge d (host arithmetic, FP64,
 * from the rate table above): *prescribed = d^3 * max_c r_c * (1 + 2^-32) and
 * *margin = a + 12 b (see SPKMC_RMAX_LEARNED).  EINVAL as spkmc_rate_table,
 * or for d outside {2, 4, 8, 16} or NULL outputs. */
int spkmc_rmax_bounds(int32_t d, double J, double H, double T, double *prescribed, double *margin);

/* Domain edge used for L when domain_edge = 0: the largest d in {16,8,4,2}
 * with L % (2d) == 0, or 0 if none. */
int32_t spkmc_resolve_domain_edge(int32_t L);

/* Device bytes one lattice of these parameters holds (0 if invalid). */
int64_t spkmc_bytes_required(const spkmc_params *p);

/* ---- single lattice ---------------------------------------------------- */
/* Create a lattice with a hot start (Sec. 3.1, the system to be partitioned).
 * EINVAL unless L % (2d) == 0, d in {2,4,8,16} (or 0), T > 0 and all finite. */
int spkmc_create(int32_t L, int32_t domain_edge, double J, double H, double T,
                 uint64_t seed, spkmc_t **out);
/* Same with every parameter; cfg may be NULL for defaults. */
int spkmc_create_ex(const spkmc_params *p, const spkmc_config *cfg, spkmc_t **out);
/* Release everything; NULL-safe.  Synchronises the stream first. */
void spkmc_destroy(spkmc_t *h);
/* Enqueue ncycles spkMC cycles (Sec. 3.1 steps 1-6, one colour per cycle) as
 * one persistent cooperative launch; ncycles >= 0 (0 is a no-op). */
int spkmc_run_cycles(spkmc_t *h, int64_t ncycles);
/* Wait for the stream and report kernel-side errors (ETIMEOUT, EINTERNAL,
 * EBOUND). */
int spkmc_synchronize(spkmc_t *h);
/* Synchronise and read the observables (M and B are kept exact in the
 * lattice state; E, m, m^2, m^4 follow on the host). */
int spkmc_observables(spkmc_t *h, spkmc_obs *out);
/* The same observables, enqueued on the handle's stream without waiting: a
 * one-thread kernel writes them from the lattice state (the kernel keeps M
 * and B exact, so no lattice pass is needed) and a copy brings them to
 * host_out, which must stay valid and unread until spkmc_synchronize
 * returns; pinned host memory lets the copy overlap the next cycles.  The
 * values equal those of spkmc_observables at the same point of the stream
 * bit for bit.  Device errors are reported by the next synchronising call. */
int spkmc_observables_async(spkmc_t *h, spkmc_obs *host_out);
/* Run every * nrec cycles (Sec. 3.1 steps 1-6, as spkmc_run_cycles) in one
 * persistent launch and record the observables after every `every` cycles
 * into host_out[0 .. nrec), record r after cycle (r + 1) * every of the run.
 * Each record equals, bit for bit, what spkmc_observables would return had
 * the run stopped there: the kernel adds every CTA's counters of M, B, the
 * events and the null rates into the record at that cycle and the clock's
 * keeper writes the clock there once its step is known.  Enqueued on the
 * handle's stream without waiting, like spkmc_observables_async: host_out
 * (nrec records; pinned host memory lets the copy overlap later work) must
 * stay valid and unread until spkmc_synchronize returns.  EINVAL if every or
 * nrec is not positive, every * nrec exceeds 2^18 cycles or the lattice's
 * cycle budget, ENOMEM if the device buffers (nrec records of 64 and 128
 * bytes per slot, kept for later calls) cannot be allocated. */
int spkmc_run_recorded(spkmc_t *h, int64_t every, int32_t nrec, spkmc_obs *host_out);
/* A CUDA graph of `steps` steps of the lattice's stream work, each
 * cycles_per_step cycles (one persistent launch, as spkmc_run_cycles) and,
 * if host_obs is not NULL, the asynchronous observables into host_obs[i]
 * (pinned host memory of `steps` records, else EINVAL).  Replaying it with
 * spkmc_graph_launch does the same work as the calls it captured, with one
 * launch from the host; the graph refers to the handle and to host_obs.
 * Destroying the handle first releases the graph's replay: spkmc_graph_launch
 * then returns SPKMC_EINVAL, and spkmc_graph_destroy still frees the graph
 * handle.  steps * cycles_per_step must be even (each launch
 * bakes in the parity of the cycle it starts on).  ECUDA if the driver
 * refuses the capture. */
int spkmc_graph_create(spkmc_t *h, int64_t cycles_per_step, int32_t steps, spkmc_obs *host_obs,
                       spkmc_graph_t **out);
/* Enqueue one replay on the handle's stream (asynchronous, like
 * spkmc_run_cycles; errors surface at the next synchronising call). */
int spkmc_graph_launch(spkmc_graph_t *g);
/* Synchronise the stream and release the graph; NULL-safe. */
void spkmc_graph_destroy(spkmc_graph_t *g);
/* Copy spins to/from a host int8 buffer of n = L^3 entries in global order.
 * set_spins recomputes the ghost faces, class counts, M and B on the device
 * and clears the R_max history (it no longer describes the spins); restore a
 * checkpoint with set_spins first, then set_state. */
int spkmc_get_spins(spkmc_t *h, int8_t *host_buf, size_t n);
int spkmc_set_spins(spkmc_t *h, const int8_t *host_buf, size_t n);
/* The same spins packed one bit per site: bit (i mod 8) of byte i / 8 is site
 * i = x + L (y + L z) of the global order above, 1 for +1 and 0 for -1;
 * nbytes = L^3 / 8 (an eighth of the int8 transfer), else EINVAL.  set has
 * the effects of spkmc_set_spins.  For these and spkmc_get/set_spins, a
 * page-locked buffer mapped into the device's address space (cudaHostAlloc,
 * cudaHostRegister with mapping) is read or written in place by the
 * transposing kernel, with no device staging buffer; any other host memory
 * goes through one.  All four return once the buffer is no longer used. */
int spkmc_get_spins_packed(spkmc_t *h, uint8_t *host_bits, size_t nbytes);
int spkmc_set_spins_packed(spkmc_t *h, const uint8_t *host_bits, size_t nbytes);
/* Copy up to cap logged events (cycle-major, ascending k within a cycle);
 * n_out receives the number copied.  The log holds the first
 * event_log_capacity events after create, spkmc_clear_event_log or
 * spkmc_set_state (which restarts it at the restored cycle). */
int spkmc_get_event_log(spkmc_t *h, spkmc_event *buf, size_t cap, size_t *n_out);
/* Synchronise and empty the event log: it fills again from the current
 * cycle on. */
int spkmc_clear_event_log(spkmc_t *h);
/* Checkpoint scalars (with get/set_spins the state is complete: the random
 * numbers are counter-based, so a resumed run is bit-identical). */
int spkmc_get_state(spkmc_t *h, spkmc_state *out);
int spkmc_set_state(spkmc_t *h, const spkmc_state *in);
/* Maintained class counts, n = 14*K int32 in domain order. */
int spkmc_class_counts(spkmc_t *h, int32_t *host_counts, size_t n);
/* Recount every domain from the spins on the device and report how many
 * domains differ from the maintained counts (0 when consistent). */
int spkmc_check_counts(spkmc_t *h, int64_t *mismatched_domains);
/* Sizes of the lattice (resolved domain edge, K, K_act, device bytes) and
 * the launch shape; grid_ctas is that of the last launch, 0 before the first.
 * Does not synchronise. */
int spkmc_info_get(spkmc_t *h, spkmc_info *out);

/* ---- batched and served ensembles --------------------------------------- */
/* A batch holds up to `capacity` independent lattices (slots) that advance
 * together in one persistent launch over a flat table of their active
 * domains; each lattice keeps its own R_max, clock, cycle counter and
 * random streams, so its trajectory is bit-identical to a solo run. */
int spkmc_batch_create(int32_t capacity, const spkmc_config *cfg, spkmc_batch_t **out);
/* Release every slot and the batch; NULL-safe.  Synchronises the stream
 * first. */
void spkmc_batch_destroy(spkmc_batch_t *b);
/* Admit a lattice into a free slot with a budget of `cycles` cycles
 * (< 0: unlimited).  EBUSY when no slot is free. */
int spkmc_batch_admit(spkmc_batch_t *b, const spkmc_params *p, int64_t cycles, int32_t *slot);
/* Run up to `cycles` cycles; each lattice stops at its own budget. */
int spkmc_batch_run(spkmc_batch_t *b, int64_t cycles);
/* spkmc_run_recorded for every lattice of the batch in one launch:
 * host_out[slot * nrec + r] (capacity * nrec records) after cycle
 * (r + 1) * every of the run.  A lattice whose budget ends within the run
 * keeps its final observables in the records after its last cycle; the
 * records of slots that are not live are undefined. */
int spkmc_batch_run_recorded(spkmc_batch_t *b, int64_t every, int32_t nrec, spkmc_obs *host_out);
/* Synchronise and list slots whose budget is spent and that were not listed
 * before (at most cap); n receives the count. */
int spkmc_batch_poll(spkmc_batch_t *b, int32_t *done_slots, int32_t cap, int32_t *n);
/* Free a slot's device memory; the slot may be admitted again. */
int spkmc_batch_retire(spkmc_batch_t *b, int32_t slot);
/* Wait for the batch's stream and report kernel-side errors, as
 * spkmc_synchronize. */
int spkmc_batch_synchronize(spkmc_batch_t *b);
/* The single-lattice read-outs for one slot (spkmc_observables,
 * spkmc_get_spins, spkmc_get_event_log); EINVAL for a slot that is not
 * live. */
int spkmc_batch_observables(spkmc_batch_t *b, int32_t slot, spkmc_obs *out);
int spkmc_batch_get_spins(spkmc_batch_t *b, int32_t slot, int8_t *host_buf, size_t n);
int spkmc_batch_get_event_log(spkmc_batch_t *b, int32_t slot, spkmc_event *buf, size_t cap,
                              size_t *n_out);
/* Observables of every slot in one synchronising read: out[slot] for
 * slot < min(cap, capacity); slots that are not live get L = 0.  n_out
 * receives the number of entries written. */
int spkmc_batch_observables_all(spkmc_batch_t *b, spkmc_obs *out, int32_t cap, int32_t *n_out);
/* Number of admitted (not retired) slots and device bytes they hold. */
int spkmc_batch_usage(spkmc_batch_t *b, int32_t *live_slots, int64_t *device_bytes);

/* ---- no-allocation variant --------------------------------------------- */
/* Some callers cannot allocate device memory: code that runs inside a memory
 * pool or arena owned by someone else, code that must not touch the CUDA
 * allocator at all (real-time loops, or an allocator that is itself being
 * set up), or a host program that only lends its own buffers.  This entry
 * point runs spkMC cycles on such a caller's lattice without any allocation.
 * It has no counterpart in the paper: it is the same cycle as
 * spkmc_run_cycles, with all of its working memory taken from one
 * file-scope device array of SPKMC_NOALLOC_SCRATCH_BYTES bytes that every GPU
 * which loads the library holds until the process exits.
 *
 *   p          physics of the lattice (L, domain_edge, J, H, T, seed); init
 *              is ignored and event_log_capacity must be 0;
 *   dev_spins  device buffer of L^3 int8 +1/-1 in global order (input), which
 *              receives the spins after the cycles (output); on any error
 *              return it still holds its input, and state is unchanged;
 *   state      host struct: cycle, clock and counters before the call (input)
 *              and after it (output); start from all zeros;
 *   ncycles    cycles to run (>= 0);
 *   stream     cudaStream_t of the caller (NULL = legacy default stream).
 *
 * The lattice's blocks, counts, frequency lines and launch tables must fit
 * the array: EINVAL (with the size in the message) for larger lattices, e.g.
 * 256^3 with d = 16 fits and 512^3 does not.  The call returns after the
 * work has finished.  No cudaMalloc, cudaFree or other allocating routine is
 * called.  Every call looks up the array's device address
 * (cudaGetSymbolAddress) with the caller's current device, so the address
 * is right again after the device's primary context was reset; the first
 * call on a device also reads its SM count and the kernel's occupancy.  Make
 * that first call before any stream capture.  Every call shares the one array and it keeps
 * the last call's contents (the call clears what must start at zero): calls
 * that overlap on the GPU, from any thread or stream, race with each other
 * and must be serialised by the caller. */
#define SPKMC_NOALLOC_SCRATCH_BYTES (16u << 20)
int spkmc_run_cycles_noalloc(const spkmc_params *p, int8_t *dev_spins, spkmc_state *state,
                             int64_t ncycles, void *stream);

/* Thread-local description of the last error of this thread. */
const char *spkmc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SPKMC_H */
