/*
 * spkmc_oracle.c -- plain, slow CPU oracle for the synchronous parallel kinetic
 * Monte Carlo (spkMC) cycle on the periodic 3D Ising lattice
 * (Martinez, Monasterio, Marian, "Billion-atom synchronous parallel kinetic
 * Monte Carlo simulations of critical 3D Ising systems", arXiv:1005.4713).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check of the
 * package entry module and the CPU-baseline leg of the benchmark may load this
 * code.  The product (the CUDA library and its Python binding) never calls it
 * and shares no source with it.
 *
 * Everything is computed in IEEE double precision, compiled with
 * -ffp-contract=off so that no multiply-add is fused.  Each function names the
 * passage of the paper it follows.  The loops are written in the order of the
 * paper's algorithm (Sec. 3.1, steps 1-6, and Sec. 3.2, steps 4a/4b), with no
 * blocking, fusion or incremental bookkeeping: every cycle recounts every
 * active domain from the spins.
 *
 * Conventions fixed where the paper is silent (each is a reading, listed with
 * its reason in the design notes of the repository):
 *   - sites (X,Y,Z), global index g = X + L*(Y + L*Z), spin +1/-1;
 *   - domain edge d, nd = L/d domains per axis (nd even), domain index
 *     k = dx + nd*(dy + nd*dz), local site index l = x + d*(y + d*z);
 *   - eight colours (default): colour(k) = (dx&1) | (dy&1)<<1 | (dz&1)<<2 and
 *     cycle t activates colour t%8; two colours (the paper's own scheme):
 *     colour(k) = (dx+dy+dz)&1 and cycle t activates the colour given by the
 *     top bit of Philox word 0 at counter (t, 0, 5, 0);
 *   - u = number of up neighbours (0..6), S = 2u-6, class c = 7*[sigma=+1] + u;
 *   - Glauber rate r(sigma,S) = 1/(1+exp(2*sigma*(J*S+H)/T)) (lambda = 1);
 *   - Philox4x64-10 with key (seed, 0); counters (t, k, 1, 0) for the event of
 *     domain k in cycle t, (t, 0, 2, 0) for the clock of cycle t,
 *     (g/256, 0, 3, 0) for the hot start;
 *   - u01 = (w0 >> 11) * 2^-53 ; xi = (2*(w0 >> 12) + 1) * 2^-53 ;
 *   - event: first class c with target < cum_c (null if none), then the j-th
 *     site of that class in ascending l with j = floor(w1 * n_c / 2^64);
 *   - the frequency lines are padded to R, which is the exact R_max of the
 *     cycle (Sec. 3.1 step 2) or one of the two bounds of Sec. 3.2 step 4b:
 *     the prescribed maximum aggregate rate, or a bound learned from the
 *     recorded history of R_max (see oracle_rmax_bounds).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------- */
/* Philox4x64-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3" (SC'11).  Counter-based generator; the paper asks for     */
/* independent random streams per domain (Sec. 3.1, step 4).                  */
/* ------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2E7470EE14C6C93ULL
#define PHILOX_M1 0xCA5A826395121157ULL
#define PHILOX_W0 0x9E3779B97F4A7C15ULL
#define PHILOX_W1 0xBB67AE8584CAA73BULL

void oracle_philox(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                   uint64_t k0, uint64_t k1, uint64_t out[4])
{
    uint64_t c[4] = {c0, c1, c2, c3};
    for (int round = 0; round < 10; ++round) {
        u128 p0 = (u128)PHILOX_M0 * c[0];
        u128 p1 = (u128)PHILOX_M1 * c[2];
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c[1] ^ k0;
        uint64_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* ------------------------------------------------------------------------- */
/* Eq. 3 (Glauber rate), read as r = (lambda/2)[1 - sigma tanh(beta dE/2)]   */
/* with dE = 2 sigma (J S + H) the energy change of flipping sigma, which is  */
/* the same number as lambda / (1 + exp(beta dE)).  lambda = 1, k_B = 1.      */
/* Class c = 7*[sigma=+1] + u, S = 2u - 6.                                    */
/* ------------------------------------------------------------------------- */
void oracle_rates(double J, double H, double T, double r[14])
{
    for (int c = 0; c < 14; ++c) {
        double sigma = (c >= 7) ? 1.0 : -1.0;
        int u = c % 7;
        double S = (double)(2 * u - 6);
        double field = J * S;          /* local field J*S + H */
        field = field + H;
        double dE = 2.0 * sigma * field; /* exact: scaling by +-2 */
        double x = dE / T;
        r[c] = 1.0 / (1.0 + exp(x));
    }
}

/* ------------------------------------------------------------------------- */
/* Lattice helpers                                                            */
/* ------------------------------------------------------------------------- */
static inline int64_t gidx(int L, int X, int Y, int Z)
{
    return (int64_t)X + (int64_t)L * ((int64_t)Y + (int64_t)L * Z);
}

static inline int wrap(int a, int L) { return a < 0 ? a + L : (a >= L ? a - L : a); }

/* number of up neighbours of site (X,Y,Z) among its 6 periodic neighbours */
static int up_neighbours(int L, const int8_t *s, int X, int Y, int Z)
{
    int u = 0;
    u += s[gidx(L, wrap(X - 1, L), Y, Z)] > 0;
    u += s[gidx(L, wrap(X + 1, L), Y, Z)] > 0;
    u += s[gidx(L, X, wrap(Y - 1, L), Z)] > 0;
    u += s[gidx(L, X, wrap(Y + 1, L), Z)] > 0;
    u += s[gidx(L, X, Y, wrap(Z - 1, L))] > 0;
    u += s[gidx(L, X, Y, wrap(Z + 1, L))] > 0;
    return u;
}

static int site_class(int L, const int8_t *s, int X, int Y, int Z)
{
    int up = s[gidx(L, X, Y, Z)] > 0;
    return 7 * up + up_neighbours(L, s, X, Y, Z);
}

/* Initial state.  init = 0: hot start (uniform +-1 from Philox, counter
 * (g/256, 0, 3, 0), bit g%256 in word (g%256)/64); init = 1: all +1 (cold
 * start, as in the relaxation runs of Sec. 6). */
void oracle_init_spins(int L, uint64_t seed, int init, int8_t *s)
{
    int64_t N = (int64_t)L * L * L;
    uint64_t w[4] = {0, 0, 0, 0};
    for (int64_t g = 0; g < N; ++g) {
        if (init == 1) { s[g] = 1; continue; }
        if (g % 256 == 0) oracle_philox((uint64_t)(g / 256), 0, 3, 0, seed, 0, w);
        int b = (int)(g % 256);
        s[g] = ((w[b / 64] >> (b % 64)) & 1) ? 1 : -1;
    }
}

/* Eq. 1 and Eq. 4: M = sum sigma, and the bond sum
 * B = sum_i sigma_i (sigma_{i+x} + sigma_{i+y} + sigma_{i+z})  (periodic),
 * so that E = -J B - H M. */
void oracle_observables(int L, const int8_t *s, int64_t *M_out, int64_t *B_out)
{
    int64_t M = 0, B = 0;
    for (int Z = 0; Z < L; ++Z)
        for (int Y = 0; Y < L; ++Y)
            for (int X = 0; X < L; ++X) {
                int si = s[gidx(L, X, Y, Z)];
                M += si;
                B += si * (s[gidx(L, wrap(X + 1, L), Y, Z)] +
                           s[gidx(L, X, wrap(Y + 1, L), Z)] +
                           s[gidx(L, X, Y, wrap(Z + 1, L))]);
            }
    *M_out = M;
    *B_out = B;
}

/* Per-domain class counts n_c (14 per domain, domain order k), from scratch. */
void oracle_class_counts(int L, int d, const int8_t *s, int32_t *counts)
{
    int nd = L / d;
    int64_t K = (int64_t)nd * nd * nd;
    memset(counts, 0, sizeof(int32_t) * 14 * K);
    for (int Z = 0; Z < L; ++Z)
        for (int Y = 0; Y < L; ++Y)
            for (int X = 0; X < L; ++X) {
                int64_t k = (X / d) + (int64_t)nd * ((Y / d) + (int64_t)nd * (Z / d));
                counts[14 * k + site_class(L, s, X, Y, Z)] += 1;
            }
}

/* floor(x * 2^64) as an unsigned 128-bit integer (x >= 0).  Used to sum the
 * null rates r_0k of Eq. 10 order-independently. */
static inline u128 to_fixed64(double x)
{
    return (u128)ldexp(x, 64);
}

/* ------------------------------------------------------------------------- */
/* spkMC cycles, Sec. 3.1 steps 1-6 with the sublattice steps 4a/4b of       */
/* Sec. 3.2.  State in/out: spins s (global order), cycle t0, clock,         */
/* counters.  If events != NULL it receives, for each cycle and each active     */
/* domain in ascending k, the triple (k, class or -1, site l or -1).         */
/* nthreads > 1 spreads the independent per-domain work of steps 1 and 4     */
/* over OpenMP threads; the result does not depend on it.                   */
/* Returns 0, or -1 on invalid arguments.                                   */
/* ------------------------------------------------------------------------- */
/* ------------------------------------------------------------------------- */
/* Sec. 3.2, step 4b: bounds that replace the exact R_max.                    */
/*                                                                            */
/* Prescribed: the maximum aggregate rate of a domain of n_k = d^3 spins,     */
/* R' = lambda n_k exp(-dE)/(1+exp(-dE)) with dE = E_max/T and                */
/* E_max = -2(n_b|J| + |H|), n_b = 6 (the printed E_max carries -|H|; with    */
/* -|H| the bound fails for H != 0, so the field term is read as +|H|).       */
/* exp(-dE)/(1+exp(-dE)) is evaluated as 1/(1+exp(dE)), the same number.      */
/*                                                                            */
/* Learned: the exact R_max of colour c at its previous visit, eight cycles   */
/* earlier, plus the most the rate of a domain can grow between two visits.   */
/* The domain's own flip moves the flipped site's rate by at most             */
/* a = max_S |r(+1,S) - r(-1,S)| and the rates of its (at most 6) neighbours  */
/* in the domain, whose S moves by 2, by at most b = max |r(s,S+2) - r(s,S)|  */
/* each; each of the 6 face-neighbouring domains is visited once in between   */
/* and its flip moves the S of at most one site of the domain by 2.  Hence    */
/* R_max(t) <= R_max(t-8) + a + 12 b.  The learned R is the smaller of that   */
/* and the prescribed bound; before a colour has a recorded visit it is the   */
/* prescribed bound.                                                          */
/*                                                                            */
/* Both bounds are multiplied by (1 + 2^-32): the computed R_k is a rounded   */
/* sum of 14 products, so it may exceed the exact bound by a few ulp.         */
/* ------------------------------------------------------------------------- */
#define ORACLE_RMAX_EXACT 0
#define ORACLE_RMAX_PRESCRIBED 1
#define ORACLE_RMAX_LEARNED 2
#define ORACLE_BOUND_SLACK (1.0 + 0x1p-32)

void oracle_rmax_bounds(int d, double J, double H, double T, double *prescribed, double *margin)
{
    const double dE = (6.0 * fabs(J) + fabs(H)) * -2.0 / T;
    const double r_top = 1.0 / (1.0 + exp(dE));
    const double n_k = (double)d * d * d;
    *prescribed = (n_k * r_top) * ORACLE_BOUND_SLACK;
    double rate[14];
    oracle_rates(J, H, T, rate);
    double a = 0.0, b = 0.0; /* class c = 7 [sigma = +1] + u, S = 2u - 6 */
    for (int u = 0; u < 7; ++u)
        if (fabs(rate[7 + u] - rate[u]) > a) a = fabs(rate[7 + u] - rate[u]);
    for (int sg = 0; sg < 2; ++sg)
        for (int u = 0; u < 6; ++u)
            if (fabs(rate[7 * sg + u + 1] - rate[7 * sg + u]) > b) b = fabs(rate[7 * sg + u + 1] - rate[7 * sg + u]);
    *margin = a + 12.0 * b;
}

/* Sec. 3.2, step 4a: the sublattice of cycle t and its a-th domain, in
 * ascending domain index.  Eight colours: a deterministic rotation over the
 * 2x2x2 parity classes of (dx, dy, dz) (a = ix + h (iy + h iz), dx = 2 ix + cx,
 * ...).  Two colours: the chessboard (dx+dy+dz) mod 2, drawn at random each
 * cycle; in each (dy, dz) row of domains the active ones are every other dx. */
#define ORACLE_SUB_8_ROTATING 0
#define ORACLE_SUB_2_RANDOM 1

static int cycle_colour(int sublattice, int64_t t, uint64_t seed)
{
    if (sublattice == ORACLE_SUB_8_ROTATING) return (int)(t % 8);
    uint64_t w[4];
    oracle_philox((uint64_t)t, 0, 5, 0, seed, 0, w);
    return (int)(w[0] >> 63);
}

static void active_domain(int sublattice, int nd, int64_t a, int c, int *dx, int *dy, int *dz)
{
    const int h = nd / 2;
    if (sublattice == ORACLE_SUB_8_ROTATING) {
        *dx = 2 * (int)(a % h) + (c & 1);
        *dy = 2 * (int)((a / h) % h) + ((c >> 1) & 1);
        *dz = 2 * (int)(a / ((int64_t)h * h)) + ((c >> 2) & 1);
    } else {
        *dy = (int)((a / h) % nd);
        *dz = (int)(a / ((int64_t)h * nd));
        *dx = 2 * (int)(a % h) + ((*dy + *dz + c) & 1);
    }
}

/* rmax_hist[i] (in/out, may be NULL) is the exact R_max of cycle t0 - 8 + i,
 * 0 where that cycle was not run.  Returns -1 for invalid arguments and -2
 * if a bound of Sec. 3.2 is exceeded by an active domain (the tolerance
 * check of the self-learning bullet); the state is then left at that cycle. */
int oracle_spkmc_run(int L, int d, double J, double H, double T, uint64_t seed,
                     int8_t *s, int64_t t0, int64_t ncycles,
                     double *clock, int64_t *n_flip, int64_t *n_null,
                     uint64_t null_fx[2], int32_t *events, int nthreads,
                     int rmax_mode, double *rmax_hist, int sublattice)
{
    if (d < 2 || L <= 0 || L % (2 * d) != 0 || !(T > 0.0)) return -1;
    if (rmax_mode < ORACLE_RMAX_EXACT || rmax_mode > ORACLE_RMAX_LEARNED) return -1;
    if (sublattice != ORACLE_SUB_8_ROTATING && sublattice != ORACLE_SUB_2_RANDOM) return -1;
    /* the learned bound rests on the eight-colour rotation (one visit of
     * every colour in any eight cycles) */
    if (sublattice == ORACLE_SUB_2_RANDOM && rmax_mode == ORACLE_RMAX_LEARNED) return -1;
    double hist_local[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double *hist = rmax_hist ? rmax_hist : hist_local;
    double R_prescribed, R_margin;
    oracle_rmax_bounds(d, J, H, T, &R_prescribed, &R_margin);
    const int nd = L / d;
    const int h = nd / 2;
    const int64_t Kact = sublattice == ORACLE_SUB_8_ROTATING ? (int64_t)h * h * h : (int64_t)h * nd * nd;
    const int64_t nsite = (int64_t)d * d * d;

    double rate[14];
    oracle_rates(J, H, T, rate);

    int32_t *cnt = (int32_t *)malloc(sizeof(int32_t) * 14 * Kact);
    double *cum = (double *)malloc(sizeof(double) * 14 * Kact);
    int32_t *ev_cls = (int32_t *)malloc(sizeof(int32_t) * Kact);
    int32_t *ev_site = (int32_t *)malloc(sizeof(int32_t) * Kact);
    if (!cnt || !cum || !ev_cls || !ev_site) {
        free(cnt); free(cum); free(ev_cls); free(ev_site);
        return -1;
    }
    u128 acc = ((u128)null_fx[1] << 64) | null_fx[0];
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#else
    (void)nthreads;
#endif

    for (int64_t t = t0; t < t0 + ncycles; ++t) {
        /* Step 4a: the sublattice (colour) of this cycle. */
        const int c = cycle_colour(sublattice, t, seed);

        /* Step 1: frequency line of every active domain, R_k = sum_c n_c r_c,
         * summed in class order 0..13. */
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
        for (int64_t a = 0; a < Kact; ++a) {
            int dx, dy, dz;
            active_domain(sublattice, nd, a, c, &dx, &dy, &dz);
            int32_t *n = cnt + 14 * a;
            for (int q = 0; q < 14; ++q) n[q] = 0;
            for (int z = 0; z < d; ++z)
                for (int y = 0; y < d; ++y)
                    for (int x = 0; x < d; ++x)
                        n[site_class(L, s, dx * d + x, dy * d + y, dz * d + z)] += 1;
            double sum = 0.0;
            for (int q = 0; q < 14; ++q) {
                sum = sum + (double)n[q] * rate[q];
                cum[14 * a + q] = sum;
            }
        }

        /* Step 2: R_max = max_k R_k over the active domains (equality case). */
        double Rmax = 0.0;
        for (int64_t a = 0; a < Kact; ++a)
            if (cum[14 * a + 13] > Rmax) Rmax = cum[14 * a + 13];

        /* Step 4b: the rate R that the lines are padded to. */
        double R = Rmax;
        if (rmax_mode != ORACLE_RMAX_EXACT) {
            R = R_prescribed;
            if (rmax_mode == ORACLE_RMAX_LEARNED && hist[0] > 0.0) {
                const double learned = (hist[0] + R_margin) * ORACLE_BOUND_SLACK;
                if (learned < R) R = learned;
            }
        }
        if (R < Rmax) {
            free(cnt); free(cum); free(ev_cls); free(ev_site);
            null_fx[0] = (uint64_t)acc;
            null_fx[1] = (uint64_t)(acc >> 64);
            return -2;
        }
        for (int i = 0; i < 7; ++i) hist[i] = hist[i + 1];
        hist[7] = Rmax;

        /* Steps 3, 4 and 4b: null rate r_0k = R - R_k padded at the end of
         * each frequency line; one event per domain with p = r/R. */
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
        for (int64_t a = 0; a < Kact; ++a) {
            int dx, dy, dz;
            active_domain(sublattice, nd, a, c, &dx, &dy, &dz);
            int64_t k = dx + (int64_t)nd * (dy + (int64_t)nd * dz);
            uint64_t w[4];
            oracle_philox((uint64_t)t, (uint64_t)k, 1, 0, seed, 0, w);
            double u01 = (double)(w[0] >> 11) * 0x1p-53;
            double target = u01 * R;
            int chosen = -1;
            for (int q = 0; q < 14; ++q)
                if (target < cum[14 * a + q]) { chosen = q; break; }
            ev_cls[a] = chosen;
            ev_site[a] = -1;
            if (chosen < 0) continue;
            uint64_t nc = (uint64_t)cnt[14 * a + chosen];
            uint64_t j = (uint64_t)(((u128)w[1] * nc) >> 64);
            uint64_t seen = 0;
            for (int64_t l = 0; l < nsite && ev_site[a] < 0; ++l) {
                int x = (int)(l % d), y = (int)((l / d) % d), z = (int)(l / ((int64_t)d * d));
                if (site_class(L, s, dx * d + x, dy * d + y, dz * d + z) == chosen) {
                    if (seen == j) ev_site[a] = (int32_t)l;
                    ++seen;
                }
            }
        }

        /* Step 6: the chosen flips become visible to the neighbours. */
        int64_t flips = 0, nulls = 0;
        for (int64_t a = 0; a < Kact; ++a) {
            int dx, dy, dz;
            active_domain(sublattice, nd, a, c, &dx, &dy, &dz);
            int64_t k = dx + (int64_t)nd * (dy + (int64_t)nd * dz);
            if (events) {
                int32_t *e = events + 3 * ((t - t0) * Kact + a);
                e[0] = (int32_t)k; e[1] = ev_cls[a]; e[2] = ev_site[a];
            }
            /* Eq. 10 numerator: sum of null rates over the domains */
            acc += to_fixed64(R - cum[14 * a + 13]);
            if (ev_cls[a] < 0) { ++nulls; continue; }
            int l = ev_site[a];
            int x = l % d, y = (l / d) % d, z = l / (d * d);
            int64_t g = gidx(L, dx * d + x, dy * d + y, dz * d + z);
            s[g] = (int8_t)(-s[g]);
            ++flips;
        }

        /* Step 5: one global time increment dt = -ln(xi) / R. */
        uint64_t wc[4];
        oracle_philox((uint64_t)t, 0, 2, 0, seed, 0, wc);
        double xi = (double)(2 * (wc[0] >> 12) + 1) * 0x1p-53;
        double dt = -log(xi) / R;
        *clock = *clock + dt;
        *n_flip += flips;
        *n_null += nulls;
    }
    null_fx[0] = (uint64_t)acc;
    null_fx[1] = (uint64_t)(acc >> 64);
    free(cnt); free(cum); free(ev_cls); free(ev_site);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Serial BKL (rejection-free n-fold way, the serial reference of Sec. 4) on  */
/* a general Lx x Ly x Lz periodic lattice.  Each event: pick site i with     */
/* probability r_i / R_tot, flip it, advance time by -ln(xi)/R_tot.  Philox   */
/* counter (step, 0, 4, 0).  Time-weighted sums (weight = residence time of   */
/* the state before the event) are accumulated per batch of events:          */
/* out[b*6 + {0..5}] = {sum dt, sum E dt, sum E^2 dt, sum m^2 dt,            */
/* sum m^4 dt, sum |m| dt}.  An axis of length 2 lists the same partner in  */
/* both neighbour slots; the energy then counts that bond twice, which is    */
/* the energy whose flip cost is 2 sigma (J S + H).                          */
/* ------------------------------------------------------------------------- */
static int64_t gidx3(int Lx, int Ly, int X, int Y, int Z)
{
    return (int64_t)X + (int64_t)Lx * ((int64_t)Y + (int64_t)Ly * Z);
}

static void bkl_neighbours(int Lx, int Ly, int Lz, int64_t i, int64_t nb[6])
{
    int X = (int)(i % Lx), Y = (int)((i / Lx) % Ly), Z = (int)(i / ((int64_t)Lx * Ly));
    nb[0] = gidx3(Lx, Ly, wrap(X - 1, Lx), Y, Z);
    nb[1] = gidx3(Lx, Ly, wrap(X + 1, Lx), Y, Z);
    nb[2] = gidx3(Lx, Ly, X, wrap(Y - 1, Ly), Z);
    nb[3] = gidx3(Lx, Ly, X, wrap(Y + 1, Ly), Z);
    nb[4] = gidx3(Lx, Ly, X, Y, wrap(Z - 1, Lz));
    nb[5] = gidx3(Lx, Ly, X, Y, wrap(Z + 1, Lz));
}

static void bkl_energy(int Lx, int Ly, int Lz, const int8_t *s, double J, double H,
                       double *E, double *M)
{
    int64_t N = (int64_t)Lx * Ly * Lz;
    int64_t bonds = 0, mag = 0;
    for (int64_t i = 0; i < N; ++i) {
        int64_t nb[6];
        bkl_neighbours(Lx, Ly, Lz, i, nb);
        bonds += s[i] * (s[nb[1]] + s[nb[3]] + s[nb[5]]);
        mag += s[i];
    }
    *E = -J * (double)bonds - H * (double)mag;
    *M = (double)mag;
}

int oracle_bkl_run(int Lx, int Ly, int Lz, double J, double H, double T, uint64_t seed,
                   int8_t *s, int64_t nevents, int nbatches, double *out)
{
    if (Lx < 2 || Ly < 2 || Lz < 2 || nbatches < 1 || !(T > 0.0)) return -1;
    const int64_t N = (int64_t)Lx * Ly * Lz;
    double rate[14];
    oracle_rates(J, H, T, rate);
    double *r = (double *)malloc(sizeof(double) * N);
    if (!r) return -1;
    memset(out, 0, sizeof(double) * 6 * nbatches);
    const int64_t per_batch = nevents / nbatches;
    for (int64_t step = 0; step < per_batch * nbatches; ++step) {
        /* frequency line of the whole lattice */
        double Rtot = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            int64_t nb[6];
            bkl_neighbours(Lx, Ly, Lz, i, nb);
            int u = 0;
            for (int q = 0; q < 6; ++q) u += s[nb[q]] > 0;
            r[i] = rate[7 * (s[i] > 0) + u];
            Rtot = Rtot + r[i];
        }
        uint64_t w[4];
        oracle_philox((uint64_t)step, 0, 4, 0, seed, 0, w);
        double xi = (double)(2 * (w[1] >> 12) + 1) * 0x1p-53;
        double dt = -log(xi) / Rtot;
        double E, M;
        bkl_energy(Lx, Ly, Lz, s, J, H, &E, &M);
        double m = M / (double)N;
        double *o = out + 6 * (step / per_batch);
        o[0] += dt;
        o[1] += E * dt;
        o[2] += E * E * dt;
        o[3] += m * m * dt;
        o[4] += m * m * m * m * dt;
        o[5] += fabs(m) * dt;
        /* choose the event on the frequency line */
        double target = (double)(w[0] >> 11) * 0x1p-53 * Rtot;
        double run = 0.0;
        int64_t pick = N - 1;
        for (int64_t i = 0; i < N; ++i) {
            run = run + r[i];
            if (target < run) { pick = i; break; }
        }
        s[pick] = (int8_t)(-s[pick]);
    }
    free(r);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Serial BKL (the n-fold way, the serial reference of Sec. 4) with the sites  */
/* grouped by rate class, for relaxation runs on lattices too large for the   */
/* rescan above.  Each event, in the order of the frequency line of Sec. 3.1  */
/* applied to the whole lattice as a single domain with no null rate: R =     */
/* sum_c n_c r_c in class order; with Philox counter (e, 0, 6, 0), target =   */
/* u R (u = (w0 >> 11) 2^-53), the first class c with target < cum_c (the     */
/* last populated class if rounding leaves none); the j-th site of that class */
/* in ascending index, j = floor(w1 n_c / 2^64); dt = -ln(xi)/R with          */
/* xi = (2 (w2 >> 12) + 1) 2^-53.  The members of each class are kept in a    */
/* Fenwick tree over the site index (rank and select in O(log N)).  m at the  */
/* times times[0..ntimes-1] (ascending) is the magnetisation of the state at  */
/* that time.  sites (may be NULL) receives the flipped sites.                */
/* ------------------------------------------------------------------------- */
static void fen_add(int32_t *f, int64_t n, int64_t i, int32_t v)
{
    for (int64_t x = i + 1; x <= n; x += x & (-x)) f[x] += v;
}

/* index of the (j+1)-th member (0-based j < total) */
static int64_t fen_select(const int32_t *f, int64_t n, int64_t j)
{
    int64_t pos = 0, step = 1;
    while (step * 2 <= n) step *= 2;
    int64_t left = j + 1;
    for (; step > 0; step /= 2) {
        if (pos + step <= n && f[pos + step] < left) {
            pos += step;
            left -= f[pos];
        }
    }
    return pos; /* 0-based index */
}

int oracle_bkl_relax(int Lx, int Ly, int Lz, double J, double H, double T, uint64_t seed, int8_t *s,
                     int ntimes, const double *times, double *m_out, int64_t max_events,
                     int64_t *nevents_out, int32_t *sites)
{
    if (Lx < 2 || Ly < 2 || Lz < 2 || ntimes < 0 || !(T > 0.0)) return -1;
    const int64_t N = (int64_t)Lx * Ly * Lz;
    double rate[14];
    oracle_rates(J, H, T, rate);
    int32_t *fen = (int32_t *)calloc((size_t)(14 * (N + 1)), sizeof(int32_t));
    int8_t *cls = (int8_t *)malloc((size_t)N);
    if (!fen || !cls) {
        free(fen); free(cls);
        return -1;
    }
    int64_t n[14] = {0};
    int64_t M = 0;
    for (int64_t i = 0; i < N; ++i) {
        int64_t nb[6];
        bkl_neighbours(Lx, Ly, Lz, i, nb);
        int u = 0;
        for (int q = 0; q < 6; ++q) u += s[nb[q]] > 0;
        cls[i] = (int8_t)(7 * (s[i] > 0) + u);
        n[cls[i]] += 1;
        fen_add(fen + cls[i] * (N + 1), N, i, 1);
        M += s[i];
    }
    double t = 0.0;
    int g = 0;
    int64_t e = 0;
    for (; e < max_events && g < ntimes; ++e) {
        double cum[14], R = 0.0;
        for (int c = 0; c < 14; ++c) {
            R = R + (double)n[c] * rate[c];
            cum[c] = R;
        }
        uint64_t w[4];
        oracle_philox((uint64_t)e, 0, 6, 0, seed, 0, w);
        const double xi = (double)(2 * (w[2] >> 12) + 1) * 0x1p-53;
        const double dt = -log(xi) / R; /* +inf when every rate is 0 */
        /* the state holds until t + dt */
        while (g < ntimes && times[g] < t + dt) m_out[g++] = (double)M / (double)N;
        if (g >= ntimes) break;
        const double target = (double)(w[0] >> 11) * 0x1p-53 * R;
        int c = -1;
        for (int q = 0; q < 14; ++q)
            if (target < cum[q]) { c = q; break; }
        if (c < 0)
            for (int q = 13; q >= 0; --q)
                if (n[q] > 0) { c = q; break; }
        const uint64_t j = (uint64_t)(((u128)w[1] * (uint64_t)n[c]) >> 64);
        const int64_t i = fen_select(fen + c * (N + 1), N, (int64_t)j);
        if (sites) sites[e] = (int32_t)i;
        t = t + dt;
        /* the flip: site i changes spin, its neighbours change up count */
        const int8_t old = s[i];
        s[i] = (int8_t)(-old);
        M += 2 * s[i];
        int64_t nb[6];
        bkl_neighbours(Lx, Ly, Lz, i, nb);
        int64_t touch[7] = {i, nb[0], nb[1], nb[2], nb[3], nb[4], nb[5]};
        for (int a = 0; a < 7; ++a) {
            const int64_t x = touch[a];
            int dup = 0;
            for (int b = 0; b < a; ++b) dup |= touch[b] == x; /* an axis of length 2 lists a partner twice */
            if (dup) continue;
            int64_t nx[6];
            bkl_neighbours(Lx, Ly, Lz, x, nx);
            int u = 0;
            for (int q = 0; q < 6; ++q) u += s[nx[q]] > 0;
            const int8_t cn = (int8_t)(7 * (s[x] > 0) + u);
            if (cn != cls[x]) {
                n[cls[x]] -= 1;
                fen_add(fen + cls[x] * (N + 1), N, x, -1);
                cls[x] = cn;
                n[cn] += 1;
                fen_add(fen + cn * (N + 1), N, x, 1);
            }
        }
    }
    if (nevents_out) *nevents_out = e;
    free(fen);
    free(cls);
    return g; /* time points filled */
}

/* ------------------------------------------------------------------------- */
/* Exact Boltzmann averages by enumeration of all 2^N states of a small       */
/* Lx x Ly x Lz lattice (N <= 24), with the energy of Eq. 1 (bonds counted as */
/* in oracle_bkl_run).  out = {<E>, <E^2>, <m^2>, <m^4>, <|m|>, <m>}.         */
/* ------------------------------------------------------------------------- */
int oracle_enumerate(int Lx, int Ly, int Lz, double J, double H, double T, double out[6])
{
    const int64_t N = (int64_t)Lx * Ly * Lz;
    if (N > 24 || N < 1 || !(T > 0.0)) return -1;
    int8_t s[24];
    double Emin = 0.0;
    /* first pass: the ground-state energy, to keep the weights finite */
    for (uint64_t st = 0; st < (1ULL << N); ++st) {
        for (int64_t i = 0; i < N; ++i) s[i] = ((st >> i) & 1) ? 1 : -1;
        double E, M;
        bkl_energy(Lx, Ly, Lz, s, J, H, &E, &M);
        if (st == 0 || E < Emin) Emin = E;
    }
    double Z = 0, sE = 0, sE2 = 0, sm2 = 0, sm4 = 0, sam = 0, sm = 0;
    for (uint64_t st = 0; st < (1ULL << N); ++st) {
        for (int64_t i = 0; i < N; ++i) s[i] = ((st >> i) & 1) ? 1 : -1;
        double E, M;
        bkl_energy(Lx, Ly, Lz, s, J, H, &E, &M);
        double wgt = exp(-(E - Emin) / T);
        double m = M / (double)N;
        Z += wgt;
        sE += wgt * E;
        sE2 += wgt * E * E;
        sm2 += wgt * m * m;
        sm4 += wgt * m * m * m * m;
        sam += wgt * fabs(m);
        sm += wgt * m;
    }
    out[0] = sE / Z; out[1] = sE2 / Z; out[2] = sm2 / Z;
    out[3] = sm4 / Z; out[4] = sam / Z; out[5] = sm / Z;
    return 0;
}

int oracle_abi_version(void) { return 2; }
