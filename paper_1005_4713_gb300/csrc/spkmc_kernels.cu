// spkmc_kernels.cu -- sm_103a kernels of the spkMC cycle (arXiv:1005.4713,
// Sec. 3.1 steps 1-6 with the chessboard sublattice of Sec. 3.2).
//
// One persistent cooperative launch runs many cycles over the active domains
// of one or many lattices (a flat table of items, split evenly over the
// CTAs).  Per cycle:
//   staging             a CTA whose domains fit its staging area requests
//                       their blocks (bit-packed rows and one-site halo, 704
//                       bytes at d = 16) at once, one bulk copy each, from the
//                       upper warps; the copies land during steps 1-2;
//   recount             (two random colours only) the class counts of every
//                       active domain, recounted from its staged block;
//   phase A (step 1)    one lane per active domain reads its 14 class count
//                       words, looks up the products fl(n_c r_c) and sums the
//                       cumulative frequency line in FP64 in class order (no
//                       fused multiply-add); the line stays in registers, or
//                       goes to scratch for CTAs that stage in rounds; partial
//                       maxima go to shared memory, then one atomicMax per CTA
//                       and lattice;
//   grid barrier        (step 2: R_max is known everywhere) -- only when some
//                       lattice pads to the exact R_max; the bounds of
//                       Sec. 3.2 step 4b need none;
//   phase B (steps 3-6) one lane per domain finds its event on the line
//                       padded by the null rate R - R_k and splits the site's
//                       rank into a half of the domain and a rank there; one
//                       octet of lanes per domain classifies the chosen half
//                       with a bit-sliced adder and picks the site by popc, an
//                       octet scan, a binary search for the word and a bit
//                       search; one thread per domain flips the site, moves
//                       the class counts of the site and of its 6 neighbours
//                       and refreshes the neighbours' ghost faces;
//   end of cycle        (step 6: the flips are visible) -- not always the
//                       whole grid: after an even cycle a CTA waits for the
//                       CTAs sharing its rows of domains (row_wait); after an
//                       odd one nothing with the exact R_max (barrier 1 of
//                       the next cycle orders what must be ordered), and with
//                       the bounds the CTAs of its near domains (near_wait),
//                       with the whole grid every 8 cycles (see the loop).
// The clock (step 5) of a lattice is advanced by the last thread of the CTA
// that holds the lattice's first active domain: during the flip step of the
// cycle when the CTA stages its domains in one round, else one cycle behind.
#include "spkmc_device.cuh"

namespace spkmc {

namespace {

// ---------------------------------------------------------------------------
// Persistent cycle kernel
// ---------------------------------------------------------------------------
struct __align__(16) WorkItem {
    long long k;      // domain index
    int ls;           // local segment
    int a;            // active index within the lattice
    int cls;          // chosen class
    int j;            // rank of the site within the class
    int off;          // byte offset of the staged block
    int site;         // chosen local site (set by the classifier), -1 if none
    int half;         // half of the domain (z < d/2: 0) that holds the j-th site
    short dx, dy, dz, d;
};

struct CtaShared {
    long long seg_base[kMaxSegPerCta + 1];
    long long seg_t0[kMaxSegPerCta];
    long long seg_part[kMaxSegPerCta];
    unsigned long long seg_rmax[kMaxSegPerCta];
    unsigned long long seg_nflip[kMaxSegPerCta];
    unsigned long long seg_nnull[kMaxSegPerCta];
    unsigned long long seg_fxlo[kMaxSegPerCta];
    unsigned long long seg_fxhi[kMaxSegPerCta];
    unsigned long long seg_dM[kMaxSegPerCta];
    unsigned long long seg_dB[kMaxSegPerCta];
    int seg_colour[kMaxSegPerCta];    // colour of the running cycle (two-colour lattices)
    double seg_rbound[kMaxSegPerCta]; // R of the running cycle for lattices padded to a bound
    double seg_nlogxi[kMaxSegPerCta]; // -ln(xi) of the running cycle
    double seg_rnow[kMaxSegPerCta];   // R_max of the running cycle
    int seg_tick[kMaxSegPerCta];      // the clock of this lattice moves in this round
    int seg_slot[kMaxSegPerCta];
    LatticeDesc descc[kDescCached]; // descriptors of the CTA's first lattices
    unsigned long long mbar;
    int nsegc;
    int nwork;
    int bulk_bytes;
    int early_bytes; // bytes requested at the start of the cycle (one-round CTAs)
    int ok;
    int nb_lo, nb_hi; // CTAs whose items share a domain row with this CTA's (this one included)
    int nnear;        // CTAs of the near wait (below), in near[]; -1: every CTA
    short near[kMaxNear];
    WorkItem work[kThreads];
};

// Colour of cycle t of segment ls: t mod 8 (rotation), or the draw of the
// cycle for a two-colour lattice (made at the start of the cycle).
__device__ __forceinline__ int cycle_colour(const CtaShared &S, const LatticeDesc &Ld, int ls, long long t)
{
    return Ld.sub2 ? S.seg_colour[ls] : (int)(t & 7);
}

__device__ __forceinline__ int find_segment(const CtaShared &S, long long q)
{
    int lo = 0, hi = S.nsegc - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (S.seg_base[mid] <= q) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

static_assert(sizeof(LatticeDesc) % 8 == 0, "the descriptor is copied in 8-byte words");

// Descriptor of local segment ls: a shared-memory copy for the CTA's first
// kDescCached lattices (the fields are read in every phase, and the L1 copy
// of the global one does not survive the product-table lookups), else the
// global one.
__device__ __forceinline__ const LatticeDesc &seg_desc(const LaunchParams &P, const CtaShared &S, int ls)
{
    return ls < kDescCached ? S.descc[ls] : P.desc[S.seg_slot[ls]];
}

// Grid-wide barrier on a monotone arrival counter.  Waits at most
// timeout_ns (and a fixed number of polls); on timeout or when another CTA
// has raised an error it returns false and the caller leaves the kernel.
__device__ bool grid_barrier(const LaunchParams &P, CtaShared &S, unsigned &epoch)
{
    ++epoch;
    __syncthreads();
    if (gridDim.x == 1) return ld_volatile_int(P.err) == 0;
    if (threadIdx.x == 0) {
        int ok = 1;
        // the arrival is a release at GPU scope: with the CTA barrier above
        // it orders every write of the CTA before it; the polls are acquires
        if ((int)blockIdx.x != P.skip_cta) red_release_add_u32(P.bar, 1u);
        const unsigned target = epoch * gridDim.x;
        const long long t0 = global_timer_ns();
        unsigned polls = 0;
        while (ld_acquire_u32(P.bar) < target) {
            ++polls;
            if ((polls & 15u) == 0) {
                if (ld_volatile_int(P.err) != 0) {
                    ok = 0;
                    break;
                }
                if (global_timer_ns() - t0 > P.timeout_ns || polls > (1u << 28)) {
                    raise_error(P.err, SPKMC_ETIMEOUT);
                    ok = 0;
                    break;
                }
            }
            __nanosleep(32);
        }
        S.ok = ok;
    }
    __syncthreads();
    return *reinterpret_cast<volatile int *>(&S.ok) != 0;
}

// After an even cycle t (eight colours), colour t + 1 differs from colour t
// in the x parity bit alone: the active domains of cycle t + 1 in a row of
// domains (fixed dy, dz) are the x neighbours of those of cycle t in the same
// row.  Everything cycle t + 1 reads or moves that the flips of cycle t wrote
// -- the blocks and ghost faces it stages, the count lines of step 1, the
// rows two steps out along x that its flip step reads, the count lines of its
// x neighbours, which the flips of cycle t rewrote -- lies in the same row;
// its rows two steps out along y or z and its diagonal domains have colours
// t + 1 ^ 2, ^ 4, ^ 3, ^ 5 and ^ 6, which cycle t did not touch.  So a CTA
// need not wait for the whole grid, only for the CTAs whose items share a row
// with its own: it publishes the cycles it has finished (a release), then
// waits (acquires) until those CTAs have finished cycle g.  Each CTA's
// counter has a 128-byte line of its own (with neighbouring CTAs' counters in
// one line, the publishing and polling of 300 CTAs contended there and the
// waits cost more than the grid barrier they replace).  Bounded like the grid
// barrier; returns false on a timeout or another CTA's error.
__device__ bool row_wait(const LaunchParams &P, CtaShared &S, long long g)
{
    __syncthreads();
    if (threadIdx.x == 0 && (int)blockIdx.x != P.skip_cta)
        st_release_u32(&P.done[(long long)blockIdx.x * kDoneStride], (unsigned)(g + 1));
    int ok = 1;
    const int c = S.nb_lo + (int)threadIdx.x;
    if (c <= S.nb_hi && c != (int)blockIdx.x) {
        const long long t0 = global_timer_ns();
        unsigned polls = 0;
        while (ld_acquire_u32(&P.done[(long long)c * kDoneStride]) < (unsigned)(g + 1)) {
            ++polls;
            if ((polls & 15u) == 0) {
                if (ld_volatile_int(P.err) != 0) {
                    ok = 0;
                    break;
                }
                if (global_timer_ns() - t0 > P.timeout_ns || polls > (1u << 28)) {
                    raise_error(P.err, SPKMC_ETIMEOUT);
                    ok = 0;
                    break;
                }
            }
            __nanosleep(32);
        }
    }
    return __syncthreads_and(ok) != 0;
}

// After an odd cycle with the bounds of Sec. 3.2 step 4b (no barrier 1), a
// CTA waits for the CTAs holding the rows within one y step of its own rows,
// in its own plane and one z step either way (S.near), to have finished the
// cycle.  That orders the flip steps of colours one or two cycles apart that
// differ in two bits (they read and write domains diagonal to each other) and
// the y and z neighbours that the next colour stages and counts.  Bounded
// like the grid barrier; returns false on a timeout or another CTA's error.
__device__ bool near_wait(const LaunchParams &P, CtaShared &S, long long g)
{
    __syncthreads();
    if (threadIdx.x == 0 && (int)blockIdx.x != P.skip_cta)
        st_release_u32(&P.done[(long long)blockIdx.x * kDoneStride], (unsigned)(g + 1));
    int ok = 1;
    const int n = S.nnear < 0 ? (int)gridDim.x : S.nnear;
    for (int i = threadIdx.x; i < n && ok; i += blockDim.x) {
        const int c = S.nnear < 0 ? i : S.near[i];
        if (c == (int)blockIdx.x) continue;
        const long long t0 = global_timer_ns();
        unsigned polls = 0;
        while (ld_acquire_u32(&P.done[(long long)c * kDoneStride]) < (unsigned)(g + 1)) {
            ++polls;
            if ((polls & 15u) == 0) {
                if (ld_volatile_int(P.err) != 0) {
                    ok = 0;
                    break;
                }
                if (global_timer_ns() - t0 > P.timeout_ns || polls > (1u << 28)) {
                    raise_error(P.err, SPKMC_ETIMEOUT);
                    ok = 0;
                    break;
                }
            }
            __nanosleep(32);
        }
    }
    return __syncthreads_and(ok) != 0;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        unsigned long long o = __shfl_xor_sync(kFull, v, off);
        v = o > v ? o : v;
    }
    return v;
}

__device__ __forceinline__ void warp_sum_u128(unsigned long long &lo, unsigned long long &hi)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        unsigned long long ol = __shfl_xor_sync(kFull, lo, off);
        unsigned long long oh = __shfl_xor_sync(kFull, hi, off);
        unsigned long long nl = lo + ol;
        hi = hi + oh + (nl < lo ? 1ULL : 0ULL);
        lo = nl;
    }
}

// Segmented reductions over runs of consecutive lanes: a run starts at lane
// 0 and wherever the key differs from the previous lane's (lanes whose
// domains belong to one lattice).  After a scan the last lane of each run
// (run_last) holds the run's total; each run then needs one shared-memory
// update instead of one per lane.  Every lane of the warp takes part.
__device__ __forceinline__ bool run_head(int key)
{
    const int prev = __shfl_up_sync(kFull, key, 1);
    return (threadIdx.x & 31) == 0 || prev != key;
}

__device__ __forceinline__ bool run_last(int key)
{
    const int next = __shfl_down_sync(kFull, key, 1);
    return (threadIdx.x & 31) == 31 || next != key;
}

__device__ __forceinline__ void run_max_u64(bool head, unsigned long long &v)
{
    const int lane = threadIdx.x & 31;
    bool f = head;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long pv = __shfl_up_sync(kFull, v, off);
        const bool pf = __shfl_up_sync(kFull, f, off);
        if (lane >= off && !f) {
            v = pv > v ? pv : v;
            f = pf;
        }
    }
}

__device__ __forceinline__ void run_sum_u128(bool head, unsigned long long &lo, unsigned long long &hi)
{
    const int lane = threadIdx.x & 31;
    bool f = head;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long pl = __shfl_up_sync(kFull, lo, off), ph = __shfl_up_sync(kFull, hi, off);
        const bool pf = __shfl_up_sync(kFull, f, off);
        if (lane >= off && !f) {
            const unsigned long long nl = lo + pl;
            hi = hi + ph + (nl < lo ? 1ULL : 0ULL);
            lo = nl;
            f = pf;
        }
    }
}

__device__ __forceinline__ void run_sum3(bool head, int &a, int &b, int &c)
{
    const int lane = threadIdx.x & 31;
    bool f = head;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int pa = __shfl_up_sync(kFull, a, off), pb = __shfl_up_sync(kFull, b, off),
                  pc = __shfl_up_sync(kFull, c, off);
        const bool pf = __shfl_up_sync(kFull, f, off);
        if (lane >= off && !f) {
            a += pa;
            b += pb;
            c += pc;
            f = pf;
        }
    }
}

// --- shared-memory barrier (mbarrier) and bulk copies (TMA engine) ---------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *m, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *m, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *m, unsigned parity)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(smem_addr(m)), "r"(parity)
                 : "memory");
    return done != 0;
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes,
                                              unsigned long long *m)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(m))
                 : "memory");
}

// Wait for the bulk copies of one round.  The first limit raises an error
// (the copies must still land before the shared memory is released, so the
// wait goes on, bounded again); returns false if they never completed.
__device__ bool mbar_wait_bounded(const LaunchParams &P, unsigned long long *m, unsigned parity)
{
    if (mbar_try_wait(m, parity)) return true; // the usual case: the copies have landed
    const long long t0 = global_timer_ns();
    bool raised = false;
    for (unsigned polls = 0;; ++polls) {
        if (mbar_try_wait(m, parity)) return true;
        const long long dt = global_timer_ns() - t0;
        if (!raised && (dt > P.timeout_ns || polls > (1u << 26))) {
            raise_error(P.err, SPKMC_ETIMEOUT);
            raised = true;
        }
        if (dt > 4 * P.timeout_ns || polls > (1u << 28)) return false;
    }
}

// The frequency line of one active domain as phase B needs it.
struct Line {
    double cum[kClasses];  // cumulative rates, class order
    double u01;            // uniform draw for the event
    unsigned long long w1; // 64-bit draw for the site rank
};

// x * 2^-53 for an integer 0 <= x < 2^53, assembled from its bits (exact;
// the same value as the rounded conversion times 2^-53, with no FP64 work)
__device__ __forceinline__ double u53_times_2m53(unsigned long long x)
{
    if (x == 0) return 0.0;
    const int e = 63 - __clzll((long long)x); // top set bit, 0..52
    const unsigned long long mant = (x << (52 - e)) & ((1ULL << 52) - 1ULL);
    return __longlong_as_double((long long)(((unsigned long long)(1023 + e - 53) << 52) | mant));
}

// The class count words (total | lower-half count << 16) of the domain staged
// in the slot at byte offset `off`.
__device__ __forceinline__ uint32_t *slot_counts(unsigned char *stage, int off, int item_bytes)
{
    return reinterpret_cast<uint32_t *>(stage + off + item_bytes - kSlotCountBytes);
}

// Step 1: frequency line of every active domain of the CTA's item range.
// With `keep` (the CTA has at most one item per thread) the line of the
// thread's item stays in registers for phase B; otherwise it goes to scratch.
__device__ void phase_a(const LaunchParams &P, CtaShared &S, unsigned char *stage, long long g, long long lo,
                        long long hi, bool keep, Line &line)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (long long base = lo + warp * 32; base < hi; base += kThreads) {
        const long long q = base + lane;
        int ls = -1;
        unsigned long long rbits = 0;
        if (q < hi) {
            ls = find_segment(S, q);
            if (g < S.seg_part[ls]) {
                const LatticeDesc &Ld = seg_desc(P, S, ls);
                const long long a = q - S.seg_base[ls];
                const long long t = S.seg_t0[ls] + g;
                int dx, dy, dz;
                active_domain(Ld, a, cycle_colour(S, Ld, ls, t), dx, dy, dz);
                const long long k = domain_index(Ld.nd, dx, dy, dz);
                const int4 *cp = reinterpret_cast<const int4 *>(Ld.counts + k * kCountStride);
                const int4 n0 = __ldcg(cp), n1 = __ldcg(cp + 1), n2 = __ldcg(cp + 2),
                           n3 = __ldcg(cp + 3); // total | lower-half count << 16
                // the draw does not depend on the counts: compute it while they load
                unsigned long long w[4];
                philox4x64_10((unsigned long long)t, (unsigned long long)k, 1ULL, 0ULL, Ld.seed, 0ULL,
                              w);
                const double u01 = u53_times_2m53(w[0] >> 11);
                const uint32_t cw[kClasses] = {(uint32_t)n0.x, (uint32_t)n0.y, (uint32_t)n0.z, (uint32_t)n0.w,
                                               (uint32_t)n1.x, (uint32_t)n1.y, (uint32_t)n1.z, (uint32_t)n1.w,
                                               (uint32_t)n2.x, (uint32_t)n2.y, (uint32_t)n2.z, (uint32_t)n2.w,
                                               (uint32_t)n3.x, (uint32_t)n3.y};
                // the products fl(n_c r_c) come from the lattice's table (a
                // count is at most d^3; the clamp keeps the read in the table
                // whatever the words hold)
                const int tstride = Ld.d * Ld.d * Ld.d + 1;
                double prod[kClasses];
#pragma unroll
                for (int c = 0; c < kClasses; ++c)
                    prod[c] = __ldg(Ld.nrate + c * tstride + min(cw[c] & 0xFFFFu, (uint32_t)(tstride - 1)));
                double cum[kClasses];
                double acc = prod[0];
                cum[0] = acc;
#pragma unroll
                for (int c = 1; c < kClasses; ++c) {
                    acc = __dadd_rn(acc, prod[c]);
                    cum[c] = acc;
                }
                if (keep) {
#pragma unroll
                    for (int c = 0; c < kClasses; ++c) line.cum[c] = cum[c];
                    line.u01 = u01;
                    line.w1 = w[1];
                    // the count words go to the end of the domain's staging slot
                    // (the block copy fills only its front)
                    uint4 *tw = reinterpret_cast<uint4 *>(slot_counts(stage, (int)(q - lo) * P.item_bytes, P.item_bytes));
                    tw[0] = make_uint4(cw[0], cw[1], cw[2], cw[3]);
                    tw[1] = make_uint4(cw[4], cw[5], cw[6], cw[7]);
                    tw[2] = make_uint4(cw[8], cw[9], cw[10], cw[11]);
                    tw[3] = make_uint4(cw[12], cw[13], 0u, 0u);
                } else {
                    double2 *sp = reinterpret_cast<double2 *>(Ld.scratch + a * kScratchStride);
#pragma unroll
                    for (int c = 0; c < kClasses; c += 2) __stcg(sp + c / 2, make_double2(cum[c], cum[c + 1]));
                    __stcg(sp + 7, make_double2(u01, __longlong_as_double((long long)w[1])));
                    uint4 *np = reinterpret_cast<uint4 *>(sp + 8);
                    __stcg(np, make_uint4(cw[0], cw[1], cw[2], cw[3]));
                    __stcg(np + 1, make_uint4(cw[4], cw[5], cw[6], cw[7]));
                    __stcg(np + 2, make_uint4(cw[8], cw[9], cw[10], cw[11]));
                    __stcg(np + 3, make_uint4(cw[12], cw[13], 0u, 0u));
                }
                rbits = (unsigned long long)__double_as_longlong(acc);
            } else {
                ls = -1;
            }
        }
        const int ls0 = __shfl_sync(kFull, ls, 0);
        if (__all_sync(kFull, ls == ls0) && ls0 >= 0) {
            const unsigned long long m = warp_max_u64(rbits);
            if (lane == 0) atomicMax(&S.seg_rmax[ls0], m);
        } else { // lattices meet in this warp: one update per run of lanes
            const bool head = run_head(ls), last = run_last(ls);
            run_max_u64(head, rbits);
            if (last && ls >= 0) atomicMax(&S.seg_rmax[ls], rbits);
        }
    }
}

// -ln(xi) of the time step of lattice segment i in grid cycle g (step 5).
// Out of line, like clock_catch_up: one thread runs it, and inlined into the
// kernel its registers added spills on the paths every thread runs.
__device__ __noinline__ double neg_log_xi(const LaunchParams &P, const CtaShared &S, int i, long long g)
{
    const LatticeDesc &Ld = seg_desc(P, S, i);
    unsigned long long wc[4];
    philox4x64_10((unsigned long long)(S.seg_t0[i] + g), 0ULL, 2ULL, 0ULL, Ld.seed, 0ULL, wc);
    const double xi = __ull2double_rn(2ULL * (wc[0] >> 12) + 1ULL) * 0x1p-53;
    return -log(xi);
}

// Step 5 for the lattices whose clock this CTA keeps (those whose first
// active domain it holds), one cycle behind: the time increment of the cycle
// that ended (its R and -ln xi are known), then, with `draw`, the -ln xi of
// cycle g.  One thread; the clock advances in cycle order.
__device__ __noinline__ void clock_catch_up(const LaunchParams &P, CtaShared &S, long long g, long long lo,
                                               bool draw)
{
    for (int i = 0; i < S.nsegc; ++i) {
        if (S.seg_tick[i]) {
            S.seg_tick[i] = 0;
            LatticeState &st = P.state[S.seg_slot[i]];
            const double c = __dadd_rn(st.clock, __ddiv_rn(S.seg_nlogxi[i], S.seg_rnow[i]));
            st.clock = c;
            // the cycle whose step this was: g - 1, or the lattice's last at the end
            const long long ge = (draw ? g : S.seg_part[i]) - 1;
            if (P.rec_every > 0 && (ge + 1) % P.rec_every == 0 && (ge + 1) / P.rec_every <= P.rec_n)
                P.rec[(long long)S.seg_slot[i] * P.rec_n + (ge + 1) / P.rec_every - 1].clock = c;
        }
        if (draw && S.seg_base[i] >= lo && g < S.seg_part[i]) S.seg_nlogxi[i] = neg_log_xi(P, S, i, g);
    }
}

// Load plane z of a staged D = 16 block as 8 words of two rows (bit b of
// word p is site (b mod 16, 2p + b/16, z)), with the planes below and above
// (the z ghost faces at the ends).
__device__ __forceinline__ void load_plane16(const uint16_t *st, int z, uint32_t cur[8], uint32_t zm[8],
                                             uint32_t zp[8])
{
    const uint16_t *g = st + 256;
    const uint4 *pc = reinterpret_cast<const uint4 *>(st + 16 * z);
    const uint4 *pm = reinterpret_cast<const uint4 *>(z > 0 ? st + 16 * (z - 1) : g + 4 * 16);
    const uint4 *pp = reinterpret_cast<const uint4 *>(z < 15 ? st + 16 * (z + 1) : g + 5 * 16);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const uint4 c = pc[i], a = pm[i], b = pp[i];
        cur[4 * i] = c.x; cur[4 * i + 1] = c.y; cur[4 * i + 2] = c.z; cur[4 * i + 3] = c.w;
        zm[4 * i] = a.x; zm[4 * i + 1] = a.y; zm[4 * i + 2] = a.z; zm[4 * i + 3] = a.w;
        zp[4 * i] = b.x; zp[4 * i + 1] = b.y; zp[4 * i + 2] = b.z; zp[4 * i + 3] = b.w;
    }
}

// Spins and bit-sliced up counts (u = u0 + 2 u1 + 4 u2) of the 32 sites of
// word p of a D = 16 plane: the x neighbours by shifts with the x halo bits
// (hxm, hxp: bit y), the y neighbours from the adjacent words or the y halo
// words (below, above), the z neighbours from the planes around.
__device__ __forceinline__ RowPlanes pair_planes(const uint32_t cur[8], const uint32_t zm[8], const uint32_t zp[8],
                                                 uint32_t below, uint32_t above, uint32_t hxm, uint32_t hxp, int p)
{
    const int y = 2 * p;
    const uint32_t s = cur[p];
    const uint32_t xm = ((s << 1) & 0xFFFEFFFEu) | ((hxm >> y) & 1u) | (((hxm >> (y + 1)) & 1u) << 16);
    const uint32_t xp = ((s >> 1) & 0x7FFF7FFFu) | (((hxp >> y) & 1u) << 15) | (((hxp >> (y + 1)) & 1u) << 31);
    const uint32_t ym = (s << 16) | (p > 0 ? (cur[p - 1] >> 16) : below);
    const uint32_t yp = (s >> 16) | ((p < 7 ? (cur[p + 1] & 0xFFFFu) : above) << 16);
    const uint32_t e = zm[p], f = zp[p];
    const uint32_t s1 = xm ^ xp ^ ym, c1 = (xm & xp) | (ym & (xm ^ xp));
    const uint32_t s2 = yp ^ e ^ f, c2 = (yp & e) | (f & (yp ^ e));
    const uint32_t k2 = s1 & s2;
    RowPlanes q;
    q.s = s;
    q.u0 = s1 ^ s2;
    q.u1 = c1 ^ c2 ^ k2;
    q.u2 = (c1 & c2) | (k2 & (c1 ^ c2));
    return q;
}

// The sites of class w.cls in the half w.half of the domain (z < d/2 or
// z >= d/2) held by octet lane o (lanes q, q+4, ..., q+28 with q = lane % 4
// work on one domain; lane o takes the o-th eighth of the half's rows, in
// ascending local index): up to 8 words of class masks, and the local index
// of bit b of word i, base + i * stride + b + offset.  No collective: the
// four domains of a warp may have different edges.
struct ClassBits {
    uint32_t m[8];
    int nw, base, stride, offset;
};

template <int D>
__device__ __forceinline__ void class_bits(const WorkItem &w, const unsigned char *stage, int o, ClassBits &cb)
{
    const uint16_t *st = reinterpret_cast<const uint16_t *>(stage + w.off);
    const int sig = w.cls >= 7, us = w.cls - 7 * sig;
    if constexpr (D == 16) {
        // lane o holds the plane z = 8 half + o as 8 words of two 16-site
        // rows: bit b of word p is site 16 (16 z + 2p) + b
        const uint16_t *g = st + 256;
        const int z = 8 * w.half + o;
        uint32_t cur[8], zm[8], zp[8];
        load_plane16(st, z, cur, zm, zp);
        const uint32_t below = g[2 * 16 + z], above = g[3 * 16 + z];
        const uint32_t hxm = g[0 * 16 + z], hxp = g[1 * 16 + z];
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            const RowPlanes q = pair_planes(cur, zm, zp, below, above, hxm, hxp, p);
            uint32_t mm = sig ? q.s : ~q.s;
            mm &= (us & 1) ? q.u0 : ~q.u0;
            mm &= (us & 2) ? q.u1 : ~q.u1;
            mm &= (us & 4) ? q.u2 : ~q.u2;
            cb.m[p] = mm;
        }
        cb.nw = 8;
        cb.base = 256 * z;
        cb.stride = 32;
        cb.offset = 0;
    } else {
        constexpr int kHalfRows = D * D / 2;                     // rows y + D z with z in the half
        constexpr int kRpl = kHalfRows >= 8 ? kHalfRows / 8 : 1; // rows per octet lane, contiguous
        static_assert(kRpl <= 8, "at most 8 words per lane");
        const bool on = (kHalfRows >= 8) || (o < kHalfRows);
        const int rl = w.half * kHalfRows + o * kRpl; // first row of this lane
#pragma unroll
        for (int i = 0; i < 8; ++i) cb.m[i] = 0;
#pragma unroll
        for (int i = 0; i < kRpl; ++i) {
            const int r = rl + i;
            if (on) cb.m[i] = class_mask<D>(classify_row<D>(st, r % D, r / D), w.cls);
        }
        cb.nw = on ? kRpl : 0;
        cb.base = D * rl;
        cb.stride = D;
        cb.offset = -1; // bit x + 1 of a classified row is site x
    }
}

// Position of the n-th set bit (from 0, in ascending order) of a word that
// has more than n set bits: a binary search on bit counts of halves.
__device__ __forceinline__ int nth_set_bit(uint32_t b, int n)
{
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const int c = __popc(b & ((1u << w) - 1u));
        if (n >= c) {
            n -= c;
            b >>= w;
            pos += w;
        }
    }
    return pos;
}

// Rank the sites of class w.cls in the half w.half of the domain in
// ascending local index and return the w.j-th (-1 if the half has fewer),
// cooperatively in the octet that holds `lane`.  Every lane of the warp
// calls this together (one domain per octet, any mix of edges).
__device__ __forceinline__ int select_site(const WorkItem &w, const unsigned char *stage, int lane)
{
    const int o = lane >> 2;
    const unsigned grp = 0x11111111u << (lane & 3);
    ClassBits cb;
    switch (w.d) {
    case 2: class_bits<2>(w, stage, o, cb); break;
    case 4: class_bits<4>(w, stage, o, cb); break;
    case 8: class_bits<8>(w, stage, o, cb); break;
    default: class_bits<16>(w, stage, o, cb); break;
    }
    int pc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) pc[i] = __popc(cb.m[i]);
    const int s01 = pc[0] + pc[1], s23 = pc[2] + pc[3], s45 = pc[4] + pc[5], s67 = pc[6] + pc[7];
    const int s03 = s01 + s23;
    const int tot = s03 + s45 + s67;
    int incl = tot;
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, 4 * off);
        if (o >= off) incl += v;
    }
    const int excl = incl - tot;
    const bool mine = w.j >= excl && w.j < incl;
    const unsigned who = __ballot_sync(kFull, mine) & grp;
    int site = 0;
    if (mine) {
        // the word that holds the site, by a binary search on the bit
        // counts of the lane's halves, pairs and words; then one search in it
        int jj = w.j - excl;
        const bool h1 = jj >= s03;
        jj -= h1 ? s03 : 0;
        const int sp = h1 ? s45 : s01;
        const bool h2 = jj >= sp;
        jj -= h2 ? sp : 0;
        const int pf = h1 ? (h2 ? pc[6] : pc[4]) : (h2 ? pc[2] : pc[0]);
        const bool h3 = jj >= pf;
        jj -= h3 ? pf : 0;
        const uint32_t wa = h1 ? (h2 ? cb.m[6] : cb.m[4]) : (h2 ? cb.m[2] : cb.m[0]);
        const uint32_t wb = h1 ? (h2 ? cb.m[7] : cb.m[5]) : (h2 ? cb.m[3] : cb.m[1]);
        const int wi = (h1 ? 4 : 0) + (h2 ? 2 : 0) + (h3 ? 1 : 0);
        site = cb.base + wi * cb.stride + nth_set_bit(h3 ? wb : wa, jj) + cb.offset;
    }
    site = __shfl_sync(kFull, site, who ? __ffs(who) - 1 : lane);
    return who ? site : -1;
}

// Class counts of a set of sites: for each up count u, the sites of spin +1
// and of spin -1 among the bits `valid` of the planes, each counted as inc
// (1, plus 1 << 16 for sites in the lower half of the domain).
__device__ __forceinline__ void count_planes(const RowPlanes &q, uint32_t valid, uint32_t inc, uint32_t part[kClasses])
{
#pragma unroll
    for (int u = 0; u < 7; ++u) {
        uint32_t e = valid;
        e &= (u & 1) ? q.u0 : ~q.u0;
        e &= (u & 2) ? q.u1 : ~q.u1;
        e &= (u & 4) ? q.u2 : ~q.u2;
        part[7 + u] += (uint32_t)__popc(e & q.s) * inc;
        part[u] += (uint32_t)__popc(e & ~q.s) * inc;
    }
}

// Octet lane o's share of the class count words of a staged block (lane o
// takes the o-th eighth of the rows); no collective.
template <int D>
__device__ __forceinline__ void recount_part(const uint16_t *st, int o, uint32_t part[kClasses])
{
    if constexpr (D == 16) {
        const uint16_t *g = st + 256;
#pragma unroll
        for (int pl = 0; pl < 2; ++pl) {
            const int z = 2 * o + pl;
            uint32_t cur[8], zm[8], zp[8];
            load_plane16(st, z, cur, zm, zp);
            const uint32_t below = g[2 * 16 + z], above = g[3 * 16 + z];
            const uint32_t hxm = g[0 * 16 + z], hxp = g[1 * 16 + z];
            const uint32_t inc = 1u + ((z < 8 ? 1u : 0u) << 16);
#pragma unroll
            for (int p = 0; p < 8; ++p) count_planes(pair_planes(cur, zm, zp, below, above, hxm, hxp, p), ~0u, inc, part);
        }
    } else {
        constexpr int kRows = D * D;
        constexpr int kRpl = kRows >= 8 ? kRows / 8 : 1;
        constexpr uint32_t V = ((1u << D) - 1u) << 1;
        if (kRows >= 8 || o < kRows) {
#pragma unroll
            for (int i = 0; i < kRpl; ++i) {
                const int r = o * kRpl + i, z = r / D;
                const uint32_t inc = 1u + ((z < D / 2 ? 1u : 0u) << 16);
                count_planes(classify_row<D>(st, r % D, z), V, inc, part);
            }
        }
    }
}

// Two-colour lattices (Sec. 3.2 step 4a with two random colours) keep no
// class counts between visits: an inactive site can see flips in up to three
// neighbouring domains in one cycle, so moving its class flip by flip would
// need an order.  Their active domains are recounted here from the staged
// blocks (the linear frequency-line evaluation of Sec. 3.1 step 1) and the
// count words go back to global memory, where step 1 reads them.  A
// one-round CTA finds its blocks already requested for the whole cycle.
__device__ void phase_r(const LaunchParams &P, CtaShared &S, unsigned char *stage, long long g, long long lo,
                        long long hi, unsigned &mbar_phase, bool early)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, o = lane >> 2;
    __syncthreads();
    for (long long rbase = lo; rbase < hi; rbase += P.round_items) {
        const long long rend = rbase + P.round_items < hi ? rbase + P.round_items : hi;
        if (early) {
            if (S.early_bytes > 0) {
                if (threadIdx.x == 0 && !mbar_wait_bounded(P, &S.mbar, mbar_phase))
                    S.ok = 0; // copies never landed: leave without touching the area
                mbar_phase ^= 1u;
                __syncthreads();
                if (threadIdx.x == 0) S.early_bytes = 0; // phase B finds the blocks in place
                if (!*reinterpret_cast<volatile int *>(&S.ok)) return;
            }
        } else {
            if (threadIdx.x == 0) S.bulk_bytes = 0;
            __syncthreads();
            const long long q = rbase + threadIdx.x;
            const LatticeDesc *Ldp = nullptr;
            long long k = 0;
            int bytes = 0;
            if (q < rend) {
                const int ls = find_segment(S, q);
                const LatticeDesc &Ld = seg_desc(P, S, ls);
                if (Ld.sub2 && g < S.seg_part[ls]) {
                    int dx, dy, dz;
                    active_domain(Ld, q - S.seg_base[ls], cycle_colour(S, Ld, ls, S.seg_t0[ls] + g), dx, dy, dz);
                    k = domain_index(Ld.nd, dx, dy, dz);
                    Ldp = &Ld;
                    bytes = staged_bytes(Ld.d);
                }
            }
            const int wb = __reduce_add_sync(kFull, bytes);
            if (lane == 0 && wb) atomicAdd(&S.bulk_bytes, wb);
            __syncthreads();
            const int total = S.bulk_bytes;
            if (total > 0) {
                if (threadIdx.x == 0) mbar_expect_tx(&S.mbar, (unsigned)total);
                __syncthreads();
                if (Ldp) {
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                    bulk_copy_g2s(stage + (q - rbase) * P.item_bytes, Ldp->cells + k * block_words(Ldp->d), bytes,
                                  &S.mbar);
                }
                if (threadIdx.x == 0 && !mbar_wait_bounded(P, &S.mbar, mbar_phase)) S.ok = 0;
                mbar_phase ^= 1u;
                __syncthreads();
                if (!*reinterpret_cast<volatile int *>(&S.ok)) return;
            }
        }
        // the recount: 4 domains per warp, 8 lanes each
        for (long long base = rbase + warp * 4; base < rend; base += kWarps * 4) {
            const long long q = base + (lane & 3);
            const LatticeDesc *Ldp = nullptr;
            long long k = 0;
            if (q < rend) {
                const int ls = find_segment(S, q);
                const LatticeDesc &Ld = seg_desc(P, S, ls);
                if (Ld.sub2 && g < S.seg_part[ls]) {
                    int dx, dy, dz;
                    active_domain(Ld, q - S.seg_base[ls], cycle_colour(S, Ld, ls, S.seg_t0[ls] + g), dx, dy, dz);
                    k = domain_index(Ld.nd, dx, dy, dz);
                    Ldp = &Ld;
                }
            }
            uint32_t part[kClasses];
#pragma unroll
            for (int c = 0; c < kClasses; ++c) part[c] = 0;
            if (Ldp) {
                const uint16_t *st = reinterpret_cast<const uint16_t *>(stage + (q - rbase) * P.item_bytes);
                switch (Ldp->d) {
                case 2: recount_part<2>(st, o, part); break;
                case 4: recount_part<4>(st, o, part); break;
                case 8: recount_part<8>(st, o, part); break;
                default: recount_part<16>(st, o, part); break;
                }
            }
            // packed words add without carries (counts < 2^16): sum over the octet
#pragma unroll
            for (int c = 0; c < kClasses; ++c) {
                uint32_t v = part[c];
                v += __shfl_xor_sync(kFull, v, 4);
                v += __shfl_xor_sync(kFull, v, 8);
                v += __shfl_xor_sync(kFull, v, 16);
                part[c] = v;
            }
            if (Ldp && o < 4) {
                const uint32_t w0 = o == 0 ? part[0] : (o == 1 ? part[4] : (o == 2 ? part[8] : part[12]));
                const uint32_t w1 = o == 0 ? part[1] : (o == 1 ? part[5] : (o == 2 ? part[9] : part[13]));
                const uint32_t w2 = o == 0 ? part[2] : (o == 1 ? part[6] : (o == 2 ? part[10] : 0u));
                const uint32_t w3 = o == 0 ? part[3] : (o == 1 ? part[7] : (o == 2 ? part[11] : 0u));
                __stcg(reinterpret_cast<uint4 *>(Ldp->counts + k * kCountStride) + o, make_uint4(w0, w1, w2, w3));
            }
        }
        __syncthreads();
    }
}

// Global u16 load that is issued only when `pred` holds (no branch).
__device__ __forceinline__ uint32_t ldg_u16_if(const uint16_t *p, bool pred)
{
    unsigned short v = 0;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.cg.u16 %0, [%1];\n\t}"
        : "+h"(v)
        : "l"(p), "r"((unsigned)pred));
    return v;
}

struct FlipDelta {
    int dM, dB; // change of M and B
};

// Spin bit of local site (x, y, z) of a staged block when only coordinate
// A (and, if B >= 0, coordinate B) may lie outside [0, D), by one step;
// with both outside the result is not used.  The other coordinates are in
// the domain, so only the possible ghost faces are selected.
template <int D, int A, int B>
__device__ __forceinline__ uint32_t staged_bit(const uint16_t *blk, int x, int y, int z)
{
    const int c3[3] = {x, y, z};
    const bool ao = c3[A] < 0 || c3[A] >= D;
    const bool bo = B >= 0 && (c3[B < 0 ? 0 : B] < 0 || c3[B < 0 ? 0 : B] >= D);
    int idx = (y & (D - 1)) + D * (z & (D - 1));
    int bit = x & (D - 1);
    // ghost face of axis q (side by the sign of the coordinate): index by the
    // remaining coordinates as in the block layout
    auto ghost = [&](int q, bool below, int &gi, int &gb) {
        const int face = 2 * q + (below ? 0 : 1);
        gi = D * D + face * D + (q == 2 ? (y & (D - 1)) : (z & (D - 1)));
        gb = (q == 0 ? y : x) & (D - 1);
    };
    int gi, gb;
    ghost(A, c3[A] < 0, gi, gb);
    idx = ao ? gi : idx;
    bit = ao ? gb : bit;
    if (B >= 0) {
        ghost(B < 0 ? 0 : B, c3[B < 0 ? 0 : B] < 0, gi, gb);
        idx = bo ? gi : idx;
        bit = bo ? gb : bit;
    }
    return ((uint32_t)blk[idx] >> bit) & 1u;
}

// Flip the chosen site (step 6), move the class counts of the site and of its
// 6 neighbours (read from the pre-flip state) and refresh the ghost faces of
// the neighbour domains that see the site; one thread per domain.  The
// domain's own counts belong to this thread during phase B (no other active
// domain borders it) and are rewritten in place; counts of a neighbour domain
// can be moved by its two active neighbours along one axis and use atomics.  For a
// neighbour j outside the domain, the site two steps out and the neighbours
// of j beyond the staged ghost face come from global memory; those loads are
// all issued before any of them is used.
template <int D>
__device__ FlipDelta apply_flip(const LaunchParams &P, CtaShared &S, const WorkItem &w,
                                const unsigned char *stage, long long g)
{
    const LatticeDesc &Ld = seg_desc(P, S, w.ls);
    const uint16_t *st = reinterpret_cast<const uint16_t *>(stage + w.off);
    int32_t *cnt = Ld.counts;
    // the domain's own count words (staged with the block); no other thread
    // touches them this cycle
    int4 *own = reinterpret_cast<int4 *>(cnt + w.k * kCountStride);
    const int l = w.site;
    const int s3[3] = {l % D, (l / D) % D, (l / (D * D)) % D};
    const int sig = w.cls >= 7, us = w.cls - 7 * sig;
    const int delta = sig ? -1 : 1; // change of the neighbours' up count
    const int nd = Ld.nd;
    const int dc[3] = {w.dx, w.dy, w.dz};
    // A neighbour j outside the domain lies in the face neighbour kj across
    // direction dir; of its own neighbours, the halo face holds the lateral
    // ones inside the domain's extent, the global blocks hold the site two
    // steps out (in kj) and, along each lateral axis on which the site sits
    // at the domain's edge, the lateral one in the diagonal domain beyond.
    // Those reads are issued together (predicated) before any write.
    long long kj[6];
    uint32_t gv[6][3];
    int gbit[6][3];
    if constexpr (D < 16) {
        // small domains (most sites on a face): the same reads, addressed
        // from global coordinates, which measures faster there
        const int base3[3] = {w.dx * D, w.dy * D, w.dz * D};
#pragma unroll
        for (int dir = 0; dir < 6; ++dir) {
            const int ax = dir >> 1, step = (dir & 1) ? 1 : -1;
            int j3[3] = {s3[0], s3[1], s3[2]};
            j3[ax] += step;
            const bool out = j3[ax] < 0 || j3[ax] >= D;
            const bool need = out && !Ld.sub2;
            int t3[3] = {j3[0], j3[1], j3[2]};
            t3[ax] += step;
            gv[dir][0] = ldg_u16_if(row_of_site<D>(Ld, base3[0] + t3[0], base3[1] + t3[1], base3[2] + t3[2],
                                                   gbit[dir][0]),
                                    need);
#pragma unroll
            for (int bi = 0; bi < 2; ++bi) {
                const int b = (ax + 1 + bi) % 3;
                const int sg = s3[b] == 0 ? -1 : 1;
                const bool far = (s3[b] == 0) || (s3[b] == D - 1);
                int m3[3] = {j3[0], j3[1], j3[2]};
                m3[b] += sg;
                gv[dir][1 + bi] = ldg_u16_if(row_of_site<D>(Ld, base3[0] + m3[0], base3[1] + m3[1], base3[2] + m3[2],
                                                            gbit[dir][1 + bi]),
                                             need && far);
            }
            const int dd[3] = {j3[0] < 0 ? -1 : (j3[0] >= D ? 1 : 0), j3[1] < 0 ? -1 : (j3[1] >= D ? 1 : 0),
                               j3[2] < 0 ? -1 : (j3[2] >= D ? 1 : 0)};
            kj[dir] = domain_index(nd, wrap_coord(dc[0] + dd[0], nd), wrap_coord(dc[1] + dd[1], nd),
                                   wrap_coord(dc[2] + dd[2], nd));
        }
    } else {
#pragma unroll
    for (int dir = 0; dir < 6; ++dir) {
        const int ax = dir >> 1, step = (dir & 1) ? 1 : -1;
        const bool out = (step < 0) ? s3[ax] == 0 : s3[ax] == D - 1;
        int fc[3] = {dc[0], dc[1], dc[2]};
        fc[ax] = out ? wrap_coord(fc[ax] + step, nd) : fc[ax];
        kj[dir] = domain_index(nd, fc[0], fc[1], fc[2]); // w.k when inside
        const bool need = out && !Ld.sub2;               // no class moves with two colours
        int l3[3] = {s3[0], s3[1], s3[2]};               // j in its own domain
        l3[ax] = step < 0 ? D - 1 : 0;
        {
            int t3[3] = {l3[0], l3[1], l3[2]}; // two steps out, in kj
            t3[ax] = step < 0 ? D - 2 : 1;
            gv[dir][0] = ldg_u16_if(block_of<D>(Ld, kj[dir]) + t3[1] + D * t3[2], need);
            gbit[dir][0] = t3[0];
        }
#pragma unroll
        for (int bi = 0; bi < 2; ++bi) {
            const int b = (ax + 1 + bi) % 3;
            const int sg = s3[b] == 0 ? -1 : 1;            // the side that may leave the domain
            const bool far = (s3[b] == 0) || (s3[b] == D - 1);
            int gc[3] = {fc[0], fc[1], fc[2]};
            gc[b] = wrap_coord(gc[b] + sg, nd);
            int m3[3] = {l3[0], l3[1], l3[2]};
            m3[b] = sg < 0 ? D - 1 : 0;
            const long long kd = domain_index(nd, gc[0], gc[1], gc[2]);
            gv[dir][1 + bi] = ldg_u16_if(block_of<D>(Ld, kd) + m3[1] + D * m3[2], need && far);
            gbit[dir][1 + bi] = m3[0];
        }
    }
    }
    // The spins of the sites within two steps of the flipped site s, before
    // its flip, one bit each: bit 0 s, bit 1 + dir its neighbour across
    // direction dir, bit 7 + dir the site two steps out that way, bits 13 +
    // 4 pr + sg the diagonal sites s + sa e_a + sb e_b (pr: the axis pair
    // (a, b) = (0,1), (0,2), (1,2); sg: bit 0 sa > 0, bit 1 sb > 0).  A site
    // with one coordinate one step outside the domain is in a staged ghost
    // face; two steps out along one axis, or outside along two, it was
    // loaded from the neighbouring blocks above.  Each neighbour's up count
    // is then a popc of the ball under a fixed mask.
    uint32_t ball = ((uint32_t)st[s3[1] + D * s3[2]] >> s3[0]) & 1u;
#pragma unroll
    for (int dir = 0; dir < 6; ++dir) {
        const int ax = dir >> 1, step = (dir & 1) ? 1 : -1;
        int n3[3] = {s3[0], s3[1], s3[2]};
        n3[ax] += step;
        const uint32_t b1 = ax == 0 ? staged_bit<D, 0, -1>(st, n3[0], n3[1], n3[2])
                            : ax == 1 ? staged_bit<D, 1, -1>(st, n3[0], n3[1], n3[2])
                                      : staged_bit<D, 2, -1>(st, n3[0], n3[1], n3[2]);
        ball |= b1 << (1 + dir);
        n3[ax] += step;
        const bool two_out = n3[ax] < -1 || n3[ax] > D;
        const uint32_t s2 = ax == 0 ? staged_bit<D, 0, -1>(st, n3[0], n3[1], n3[2])
                            : ax == 1 ? staged_bit<D, 1, -1>(st, n3[0], n3[1], n3[2])
                                      : staged_bit<D, 2, -1>(st, n3[0], n3[1], n3[2]);
        const uint32_t b2 = two_out ? ((gv[dir][0] >> gbit[dir][0]) & 1u) : s2;
        ball |= b2 << (7 + dir);
    }
#pragma unroll
    for (int pr = 0; pr < 3; ++pr) {
        const int a = pr == 2 ? 1 : 0, b = pr == 0 ? 1 : 2;
        const int bi = (b - a + 2) % 3; // (a + 1 + bi) % 3 == b: the lateral index of b for direction a
#pragma unroll
        for (int sg = 0; sg < 4; ++sg) {
            const int sa = (sg & 1) ? 1 : -1, sb = (sg & 2) ? 1 : -1;
            int n3[3] = {s3[0], s3[1], s3[2]};
            n3[a] += sa;
            n3[b] += sb;
            const bool ao = n3[a] < 0 || n3[a] >= D, bo = n3[b] < 0 || n3[b] >= D;
            const int da = 2 * a + (sa > 0 ? 1 : 0);
            const uint32_t sv = pr == 0 ? staged_bit<D, 0, 1>(st, n3[0], n3[1], n3[2])
                                : pr == 1 ? staged_bit<D, 0, 2>(st, n3[0], n3[1], n3[2])
                                          : staged_bit<D, 1, 2>(st, n3[0], n3[1], n3[2]);
            const uint32_t v = (ao && bo) ? ((gv[da][1 + bi] >> gbit[da][1 + bi]) & 1u) : sv;
            ball |= v << (13 + 4 * pr + sg);
        }
    }
    int cold[6];
    bool outv[6];
#pragma unroll
    for (int dir = 0; dir < 6; ++dir) {
        const int ax = dir >> 1, sp = dir & 1, step = sp ? 1 : -1;
        // the neighbours of j = s + step e_ax: s, the site two steps out, and
        // the four diagonal sites s + step e_ax +- e_b
        uint32_t m = 1u | (1u << (7 + dir));
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (b == ax) continue;
            const int a0 = ax < b ? ax : b, b0 = ax < b ? b : ax;
            const int pr = (a0 == 0 && b0 == 1) ? 0 : (a0 == 0 ? 1 : 2);
#pragma unroll
            for (int sb = 0; sb < 2; ++sb) {
                const int sa_bit = ax < b ? sp : sb, sb_bit = ax < b ? sb : sp;
                m |= 1u << (13 + 4 * pr + sa_bit + 2 * sb_bit);
            }
        }
        cold[dir] = 7 * (int)((ball >> (1 + dir)) & 1u) + __popc(ball & m);
        const int jc = s3[ax] + step;
        outv[dir] = jc < 0 || jc >= D;
    }
    bool ok = true;
    if (!Ld.sub2) { // two-colour lattices recount at each visit instead
        // a class move of a site adds 1 to the total and, in the lower half
        // of its domain (z < D/2), 1 to bits 16-31 of the class word; the
        // moves of the domain's own words go to its staged copy (only this
        // thread touches the slot now), which is then written out
        int *tail = reinterpret_cast<int *>(slot_counts(const_cast<unsigned char *>(stage), w.off, P.item_bytes));
        const int inc_s = 1 + ((s3[2] < D / 2) << 16);
        tail[w.cls] -= inc_s;
        tail[7 * (1 - sig) + us] += inc_s;
#pragma unroll
        for (int dir = 0; dir < 6; ++dir) {
            const int cn = cold[dir] + delta;
            int j3z = s3[2] + (dir == 4 ? -1 : (dir == 5 ? 1 : 0));
            j3z = j3z < 0 ? D - 1 : (j3z >= D ? 0 : j3z); // z of the neighbour in its own domain
            const int inc = 1 + ((j3z < D / 2) << 16);
            if (cold[dir] >= 0 && cold[dir] < kClasses && cn >= 0 && cn < kClasses) {
                if (outv[dir]) {
                    atomicAdd(cnt + kj[dir] * kCountStride + cold[dir], -inc);
                    atomicAdd(cnt + kj[dir] * kCountStride + cn, inc);
                } else {
                    tail[cold[dir]] -= inc;
                    tail[cn] += inc;
                }
            } else {
                ok = false;
            }
        }
        const int4 *t4 = reinterpret_cast<const int4 *>(tail);
        const int4 v0 = t4[0], v1 = t4[1], v2 = t4[2], v3 = t4[3];
        __stcg(own, v0);
        __stcg(own + 1, v1);
        __stcg(own + 2, v2);
        __stcg(own + 3, make_int4(v3.x, v3.y, 0, 0));
    }
    if (!ok) raise_error(P.err, SPKMC_EINTERNAL);
    const int x = s3[0], y = s3[1], z = s3[2];
    // the flip, and the ghost faces of the neighbours that touch the site
    xor_u16(block_of<D>(Ld, w.k) + y + D * z, 1u << x);
    if (x == 0) xor_u16(block_of<D>(Ld, kj[0]) + D * D + 1 * D + z, 1u << y);
    if (x == D - 1) xor_u16(block_of<D>(Ld, kj[1]) + D * D + 0 * D + z, 1u << y);
    if (y == 0) xor_u16(block_of<D>(Ld, kj[2]) + D * D + 3 * D + z, 1u << x);
    if (y == D - 1) xor_u16(block_of<D>(Ld, kj[3]) + D * D + 2 * D + z, 1u << x);
    if (z == 0) xor_u16(block_of<D>(Ld, kj[4]) + D * D + 5 * D + y, 1u << x);
    if (z == D - 1) xor_u16(block_of<D>(Ld, kj[5]) + D * D + 4 * D + y, 1u << x);
    const long long t = S.seg_t0[w.ls] + g;
    if (Ld.log) {
        const long long idx = (t - Ld.log_t0) * Ld.Kact + w.a;
        if (idx >= 0 && idx < Ld.log_cap) {
            spkmc_event ev;
            ev.cycle = t;
            ev.domain = (int32_t)w.k;
            ev.cls = w.cls;
            ev.site = l;
            ev.reserved = 0;
            Ld.log[idx] = ev;
        }
    }
    // M and B move by -2 sigma and -2 sigma S (Eq. 1 and Eq. 4, S = 2u - 6)
    const int sgn = sig ? 1 : -1;
    FlipDelta f;
    f.dM = -2 * sgn;
    f.dB = -2 * sgn * (2 * us - 6);
    return f;
}

// Steps 3, 4/4b, 5 and 6 for the items [rbase, rbase + round_items) of the
// CTA's range.  With `early` (one-round CTA) the frequency lines come from
// registers and the blocks were requested at the start of the cycle.
__device__ __forceinline__ void phase_b_round(const LaunchParams &P, CtaShared &S, unsigned char *stage,
                                              long long g, long long lo, long long hi, long long rbase,
                                              unsigned &mbar_phase, bool early, const Line &line)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int R = P.round_items;
    {
        if (threadIdx.x == 0) {
            S.nwork = 0;
            S.bulk_bytes = 0;
        }
        __syncthreads();
        const long long q = rbase + threadIdx.x;
        int ls = -1, cls = -1, dx = 0, dy = 0, dz = 0, dval = 0;
        int jhalf = 0;
        uint4 cw4[4]; // count words of the item (rounds after the first: from scratch)
        long long a = 0, k = 0;
        unsigned long long fxlo = 0, fxhi = 0, jrank = 0;
        if (threadIdx.x < R && q < hi) {
            ls = find_segment(S, q);
            if (g < S.seg_part[ls]) {
                const int slot = S.seg_slot[ls];
                const LatticeDesc &Ld = seg_desc(P, S, ls);
                a = q - S.seg_base[ls];
                const long long t = S.seg_t0[ls] + g;
                // the rate R the lines are padded to (Sec. 3.1 step 2 or the
                // bounds of Sec. 3.2 step 4b)
                const double R = Ld.rmode == SPKMC_RMAX_EXACT
                                     ? __longlong_as_double((long long)__ldcg(&P.state[slot].rmax[t & (kRmaxRing - 1)]))
                                     : S.seg_rbound[ls];
                double cum[kClasses];
                double u01;
                unsigned long long w1;
                if (early) {
#pragma unroll
                    for (int c = 0; c < kClasses; ++c) cum[c] = line.cum[c];
                    u01 = line.u01;
                    w1 = line.w1;
                } else {
                    const double2 *sp = reinterpret_cast<const double2 *>(Ld.scratch + a * kScratchStride);
#pragma unroll
                    for (int c = 0; c < kClasses; c += 2) {
                        const double2 v = __ldcg(sp + c / 2);
                        cum[c] = v.x;
                        cum[c + 1] = v.y;
                    }
                    const double2 uw = __ldcg(sp + 7);
                    const uint4 *np = reinterpret_cast<const uint4 *>(sp + 8);
                    cw4[0] = __ldcg(np);
                    cw4[1] = __ldcg(np + 1);
                    cw4[2] = __ldcg(np + 2);
                    cw4[3] = __ldcg(np + 3);
                    u01 = uw.x;
                    w1 = (unsigned long long)__double_as_longlong(uw.y);
                }
                // the bound must cover the domain (tolerance check of Sec. 3.2)
                if (cum[kClasses - 1] > R) raise_error(P.err, SPKMC_EBOUND);
                // target on the frequency line padded to R (steps 3-4): the
                // first class whose cumulative rate exceeds it, else null.
                const double target = __dmul_rn(u01, R);
                const unsigned long long tb = (unsigned long long)__double_as_longlong(target);
#pragma unroll
                for (int c = kClasses - 1; c >= 0; --c)
                    if (tb < (unsigned long long)__double_as_longlong(cum[c])) cls = c;
                fixed64(__dadd_rn(R, -cum[kClasses - 1]), fxlo, fxhi);
                active_domain(Ld, a, cycle_colour(S, Ld, ls, t), dx, dy, dz);
                k = domain_index(Ld.nd, dx, dy, dz);
                dval = Ld.d;
                if (cls < 0) {
                    if (Ld.log) {
                        const long long idx = (t - Ld.log_t0) * Ld.Kact + a;
                        if (idx >= 0 && idx < Ld.log_cap) {
                            spkmc_event ev;
                            ev.cycle = t;
                            ev.domain = (int32_t)k;
                            ev.cls = -1;
                            ev.site = -1;
                            ev.reserved = 0;
                            Ld.log[idx] = ev;
                        }
                    }
                } else {
                    uint32_t word;
                    if (early) {
                        word = slot_counts(stage, (int)(q - lo) * P.item_bytes, P.item_bytes)[cls];
                    } else {
                        const uint32_t cw[16] = {cw4[0].x, cw4[0].y, cw4[0].z, cw4[0].w, cw4[1].x, cw4[1].y,
                                                 cw4[1].z, cw4[1].w, cw4[2].x, cw4[2].y, cw4[2].z, cw4[2].w,
                                                 cw4[3].x, cw4[3].y, cw4[3].z, cw4[3].w};
                        word = 0;
#pragma unroll
                        for (int c = 0; c < kClasses; ++c)
                            if (c == cls) word = cw[c];
                    }
                    // rank j of the site in its class (step 4), then the half of
                    // the domain that holds it and its rank there
                    const unsigned long long nc = word & 0xFFFFu, nlow = word >> 16;
                    jrank = __umul64hi(w1, nc);
                    if (jrank >= nlow) {
                        jhalf = 1;
                        jrank -= nlow;
                    }
                }
                if (a == 0) {
                    S.seg_rnow[ls] = R; // the clock moves once this cycle (step 5)
                    S.seg_tick[ls] = 1;
                    // slot of cycle t - 24, last read at t - 16: free for t + 8
                    P.state[slot].rmax[(t + 8) & (kRmaxRing - 1)] = 0ULL;
                }
            } else {
                ls = -1;
            }
        }
        // work list: warp-aggregated slots for the domains that flip
        const bool flips = ls >= 0 && cls >= 0;
        const unsigned bal = __ballot_sync(kFull, flips);
        const int bytes = __reduce_add_sync(kFull, flips ? staged_bytes(dval) : 0);
        int wbase = 0;
        if (lane == 0 && bal) {
            wbase = atomicAdd(&S.nwork, __popc(bal));
            atomicAdd(&S.bulk_bytes, bytes);
        }
        wbase = __shfl_sync(kFull, wbase, 0);
        if (flips) {
            const int idx = wbase + __popc(bal & ((1u << lane) - 1u));
            WorkItem wi;
            wi.k = k;
            wi.ls = ls;
            wi.a = (int)a;
            wi.cls = cls;
            wi.j = (int)jrank;
            wi.off = (early ? (int)(q - lo) : idx) * P.item_bytes;
            wi.site = -1;
            wi.dx = (short)dx;
            wi.dy = (short)dy;
            wi.dz = (short)dz;
            wi.d = (short)dval;
            wi.half = jhalf;
            S.work[idx] = wi;
            if (!early) {
                uint4 *tw = reinterpret_cast<uint4 *>(slot_counts(stage, wi.off, P.item_bytes));
                tw[0] = cw4[0];
                tw[1] = cw4[1];
                tw[2] = cw4[2];
                tw[3] = cw4[3];
            }
        }
        const int ls0 = __shfl_sync(kFull, ls, 0);
        const bool nul = ls >= 0 && cls < 0;
        if (__all_sync(kFull, ls == ls0) && ls0 >= 0) {
            warp_sum_u128(fxlo, fxhi);
            const unsigned nn = __popc(__ballot_sync(kFull, nul));
            if (lane == 0) {
                atomic_add_u128(&S.seg_fxlo[ls0], &S.seg_fxhi[ls0], fxlo, fxhi);
                if (nn) atomicAdd(&S.seg_nnull[ls0], (unsigned long long)nn);
            }
        } else { // lattices meet in this warp: one update per run of lanes
            const bool head = run_head(ls), last = run_last(ls);
            run_sum_u128(head, fxlo, fxhi);
            int nn = nul ? 1 : 0, z0 = 0, z1 = 0;
            run_sum3(head, nn, z0, z1);
            if (last && ls >= 0) {
                atomic_add_u128(&S.seg_fxlo[ls], &S.seg_fxhi[ls], fxlo, fxhi);
                if (nn) atomicAdd(&S.seg_nnull[ls], (unsigned long long)nn);
            }
        }
        __syncthreads();
        const int nwork = S.nwork;
        const int bulk = S.bulk_bytes;
        if (early) {
            // the blocks of all the CTA's domains were requested at the start
            // of the cycle; wait for them once
            if (S.early_bytes > 0) {
                if (threadIdx.x == 0 && !mbar_wait_bounded(P, &S.mbar, mbar_phase))
                    S.ok = 0; // copies never landed: leave without touching the area
                mbar_phase ^= 1u;
                __syncthreads();
                if (!*reinterpret_cast<volatile int *>(&S.ok)) return;
            }
            if (nwork == 0) {
                // step 5 of this cycle (see the flip step below)
                if (threadIdx.x == kThreads - 1) clock_catch_up(P, S, g + 1, lo, true);
                return;
            }
        } else {
            if (nwork == 0) return;
            // stage the blocks of every domain that flips in this round at once
            if (threadIdx.x == 0) mbar_expect_tx(&S.mbar, (unsigned)bulk);
            __syncthreads();
            if (threadIdx.x < nwork) {
                const WorkItem &w = S.work[threadIdx.x];
                const LatticeDesc &Ld = seg_desc(P, S, w.ls);
                asm volatile("fence.proxy.async.global;" ::: "memory");
                bulk_copy_g2s(stage + w.off, Ld.cells + w.k * block_words(w.d), staged_bytes(w.d), &S.mbar);
            }
            if (threadIdx.x == 0 && !mbar_wait_bounded(P, &S.mbar, mbar_phase))
                S.ok = 0; // copies never landed: leave without touching the area
            mbar_phase ^= 1u;
            __syncthreads();
            if (!*reinterpret_cast<volatile int *>(&S.ok)) return;
        }
        // The class counts of this CTA's domains of the next cycle into L2,
        // for lattices whose blocks exceed 64 MB (smaller ones stay in L2
        // anyway): step 1 of that cycle then finds them there, not behind
        // the block copies that start it.  The flips of this cycle move some
        // of those counts later, in L2.  Also in a launch's last cycle: the
        // next launch's first step 1 finds them in L2 too (a lattice that
        // never runs again only had a line prefetched).
        if (early) {
            const long long qn = lo + threadIdx.x;
            if (qn < hi) {
                const int lsn = find_segment(S, qn);
                const LatticeDesc &Ldn = seg_desc(P, S, lsn);
                if (!Ldn.sub2 && Ldn.K * staged_bytes(Ldn.d) > (64LL << 20)) {
                    int dx, dy, dz;
                    active_domain(Ldn, qn - S.seg_base[lsn], (int)((S.seg_t0[lsn] + g + 1) & 7), dx, dy, dz);
                    const int32_t *cp = Ldn.counts + domain_index(Ldn.nd, dx, dy, dz) * kCountStride;
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(cp));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(cp + 8));
                }
            }
        }
        // rank and pick the site: 4 domains per warp, 8 lanes each
        for (int base = warp * 4; base < nwork; base += kWarps * 4) {
            const int i = base + (lane & 3);
            const bool valid = i < nwork;
            const WorkItem &w = S.work[valid ? i : base];
            const int site = select_site(w, stage, lane);
            if (valid && lane < 4) {
                S.work[i].site = site;
                if (site < 0) raise_error(P.err, SPKMC_EINTERNAL);
            }
        }
        __syncthreads();
        // flips and class moves, one thread per domain
        int fls = -1, fdM = 0, fdB = 0;
        // step 5 of this cycle, and the draw of the next, on the last thread,
        // which has no domain here: the division and the logarithm run beside
        // the flips instead of beside step 1 of the next cycle, where they
        // could hold up the CTA barrier after step 1
        if (early && threadIdx.x == kThreads - 1) clock_catch_up(P, S, g + 1, lo, true);
        if (threadIdx.x < nwork) {
            const WorkItem w = S.work[threadIdx.x];
            if (w.site >= 0) {
                FlipDelta f;
                switch (w.d) {
                case 2: f = apply_flip<2>(P, S, w, stage, g); break;
                case 4: f = apply_flip<4>(P, S, w, stage, g); break;
                case 8: f = apply_flip<8>(P, S, w, stage, g); break;
                default: f = apply_flip<16>(P, S, w, stage, g); break;
                }
                fls = w.ls;
                fdM = f.dM;
                fdB = f.dB;
            }
        }
        // per-lattice flip counters, one shared-memory update per warp
        const int lsmax = __reduce_max_sync(kFull, fls);
        if (__all_sync(kFull, fls < 0 || fls == lsmax)) {
            const int nf = __popc(__ballot_sync(kFull, fls >= 0));
            const int sM = __reduce_add_sync(kFull, fdM), sB = __reduce_add_sync(kFull, fdB);
            if (lane == 0 && lsmax >= 0) {
                atomicAdd(&S.seg_nflip[lsmax], (unsigned long long)nf);
                atomicAdd(&S.seg_dM[lsmax], (unsigned long long)(long long)sM);
                atomicAdd(&S.seg_dB[lsmax], (unsigned long long)(long long)sB);
            }
        } else { // lattices meet in this warp: one update per run of lanes
            const bool head = run_head(fls), last = run_last(fls);
            int nf = fls >= 0 ? 1 : 0, sM = fdM, sB = fdB;
            run_sum3(head, nf, sM, sB);
            if (last && fls >= 0) {
                atomicAdd(&S.seg_nflip[fls], (unsigned long long)nf);
                atomicAdd(&S.seg_dM[fls], (unsigned long long)(long long)sM);
                atomicAdd(&S.seg_dB[fls], (unsigned long long)(long long)sB);
            }
        }
        __syncthreads();
    }
}

__device__ void phase_b(const LaunchParams &P, CtaShared &S, unsigned char *stage, long long g,
                        long long lo, long long hi, unsigned &mbar_phase, bool early, const Line &line)
{
    if (early) {
        if (lo < hi) phase_b_round(P, S, stage, g, lo, hi, lo, mbar_phase, true, line);
        return;
    }
    for (long long rbase = lo; rbase < hi; rbase += P.round_items) {
        phase_b_round(P, S, stage, g, lo, hi, rbase, mbar_phase, false, line);
        if (!*reinterpret_cast<volatile int *>(&S.ok)) return;
    }
}

__global__ void __launch_bounds__(kThreads, 2) spkmc_cycles_kernel(LaunchParams P)
{
    __shared__ CtaShared S;
    extern __shared__ __align__(128) unsigned char stage[];
    const long long G = gridDim.x;
    const long long lo = (P.Q * (long long)blockIdx.x) / G;
    const long long hi = (P.Q * ((long long)blockIdx.x + 1)) / G;

    if (threadIdx.x == 0) {
        // segments overlapping [lo, hi): the last one with base <= lo, onwards
        int first = 0, top = P.nseg - 1;
        while (first < top) {
            int mid = (first + top + 1) >> 1;
            if (P.seg[mid].base <= lo) first = mid;
            else top = mid - 1;
        }
        int n = 0, i = first;
        S.ok = 1;
        for (; i < P.nseg && P.seg[i].base < hi; ++i) {
            if (n == kMaxSegPerCta) {
                raise_error(P.err, SPKMC_EINTERNAL);
                S.ok = 0;
                break;
            }
            S.seg_base[n] = P.seg[i].base;
            S.seg_slot[n] = P.seg[i].slot;
            ++n;
        }
        S.seg_base[n] = (i < P.nseg) ? P.seg[i].base : P.Q;
        S.nsegc = n;
        mbar_init(&S.mbar, 1);
        // the CTAs whose items share a domain row (half items of one lattice,
        // fixed dy and dz) with this CTA's first and last items
        S.nb_lo = S.nb_hi = (int)blockIdx.x;
        // the CTA that holds item q
        auto owner = [&](long long q) {
            long long c = (q * G) / P.Q;
            while (c + 1 < G && (P.Q * (c + 1)) / G <= q) ++c;
            while (c > 0 && (P.Q * c) / G > q) --c;
            return (int)c;
        };
        if (P.done && S.ok && n > 0 && lo < hi) {
            auto row_edge = [&](long long q, bool end) {
                int j = 0;
                while (j + 1 < P.nseg && P.seg[j + 1].base <= q) ++j;
                const long long sb = P.seg[j].base, h = P.desc[P.seg[j].slot].half;
                const long long r0 = sb + ((q - sb) / h) * h;
                return end ? r0 + h - 1 : r0;
            };
            S.nb_lo = owner(row_edge(lo, false));
            S.nb_hi = owner(row_edge(hi - 1, true));
            if (S.nb_hi - S.nb_lo + 1 > kThreads) { // cannot happen with a segment table the host accepted
                raise_error(P.err, SPKMC_EINTERNAL);
                S.ok = 0;
            }
        }
        // The CTAs of the near wait (one lattice, the bounds of Sec. 3.2
        // step 4b; see the kernel loop): those holding, for a row of this
        // CTA's items at (ay, az), the rows ay - 1, ay, ay + 1 of the planes
        // az - 1, az, az + 1, each index wrapping.  A run of rows within one
        // plane (with the row that a y step wraps taken on its own) maps to a
        // run of whole rows in each image plane, whose owners are a
        // contiguous range of CTAs.
        S.nnear = 0;
        if (!P.exact_any && P.done && P.nseg == 1 && S.ok && lo < hi) {
            const long long h = P.desc[P.seg[0].slot].half;
            const long long r0 = lo / h, r1 = (hi - 1) / h;
            for (int dz = -1; dz <= 1 && S.nnear >= 0; ++dz) {
                for (int dy = -1; dy <= 1 && S.nnear >= 0; ++dy) {
                    for (long long r = r0; r <= r1 && S.nnear >= 0;) {
                        const long long ay = r % h, az = r / h;
                        long long e = (az + 1) * h - 1 < r1 ? (az + 1) * h - 1 : r1;
                        if ((dy < 0 && ay == 0) || (dy > 0 && ay == h - 1)) e = r;
                        else if (dy > 0 && e > az * h + h - 2) e = az * h + h - 2;
                        const long long first = ((ay + dy + h) % h + h * (((az + dz) % h + h) % h)) * h;
                        const int c0 = owner(first), c1 = owner(first + (e - r + 1) * h - 1);
                        for (int c = c0; c <= c1 && S.nnear >= 0; ++c) {
                            bool seen = false;
                            for (int k = 0; k < S.nnear; ++k) seen = seen || S.near[k] == c;
                            if (seen) continue;
                            if (S.nnear == kMaxNear) S.nnear = -1; // too many: wait for every CTA
                            else S.near[S.nnear++] = (short)c;
                        }
                        r = e + 1;
                    }
                }
            }
        }
    }
    __syncthreads();
    if (!S.ok) return; // the host sizes the grid so that this cannot happen
    {
        constexpr int kWords = (int)(sizeof(LatticeDesc) / 8);
        const int ncached = S.nsegc < kDescCached ? S.nsegc : kDescCached;
        for (int i = threadIdx.x; i < ncached * kWords; i += blockDim.x)
            reinterpret_cast<unsigned long long *>(&S.descc[i / kWords])[i % kWords] =
                reinterpret_cast<const unsigned long long *>(&P.desc[S.seg_slot[i / kWords]])[i % kWords];
    }
    for (int i = threadIdx.x; i < S.nsegc; i += blockDim.x) {
        const LatticeState &st = P.state[S.seg_slot[i]];
        const long long budget = st.budget;
        S.seg_t0[i] = st.t;
        S.seg_part[i] = budget < 0 ? P.ncycles : (budget < P.ncycles ? budget : P.ncycles);
        S.seg_rmax[i] = 0;
        S.seg_nflip[i] = 0;
        S.seg_nnull[i] = 0;
        S.seg_fxlo[i] = 0;
        S.seg_fxhi[i] = 0;
        S.seg_dM[i] = 0;
        S.seg_dB[i] = 0;
        S.seg_nlogxi[i] = 0.0;
        S.seg_rnow[i] = 0.0;
        S.seg_tick[i] = 0;
    }
    __syncthreads();
    if (ld_volatile_int(P.err) != 0) return;

    unsigned epoch = 0, mbar_phase = 0;
    // a CTA whose domains all fit the staging area requests their blocks at
    // the start of each cycle, so the copies overlap step 1 and the barrier
    // (an active domain's block does not change within its cycle)
    const bool early = hi - lo <= P.round_items;
    for (long long g = 0; g < P.ncycles; ++g) {
        Line line; // this cycle's frequency line of the thread's item (one-round CTAs)
        for (int i = kThreads - 1 - (int)threadIdx.x; i < S.nsegc; i += kThreads) {
            // the bound of Sec. 3.2 step 4b for lattices that use one (read
            // by the prepass, after step 1), from the last threads: the
            // learned bound waits for a memory round trip, and the first
            // warps hold the items of step 1
            const LatticeDesc &Ld = seg_desc(P, S, i);
            if (Ld.rmode != SPKMC_RMAX_EXACT && g < S.seg_part[i]) {
                double R = Ld.rbound;
                if (Ld.rmode == SPKMC_RMAX_LEARNED) {
                    // exact R_max of this colour's previous visit, cycle t - 8,
                    // final since the grid barrier that the bounds take at
                    // least every 8 cycles (see the kernel loop)
                    const long long t = S.seg_t0[i] + g;
                    const double h = __longlong_as_double(
                        (long long)__ldcg(&P.state[S.seg_slot[i]].rmax[(t - 8) & (kRmaxRing - 1)]));
                    if (h > 0.0) {
                        const double b = __dmul_rn(__dadd_rn(h, Ld.rmargin), kBoundSlack);
                        if (b < R) R = b;
                    }
                }
                S.seg_rbound[i] = R;
            }
        }
        if (P.sub2_any) {
            // Sec. 3.2 step 4a, two colours: the colour of this cycle
            for (int i = threadIdx.x; i < S.nsegc; i += blockDim.x) {
                const LatticeDesc &Ld = seg_desc(P, S, i);
                if (Ld.sub2 && g < S.seg_part[i]) {
                    unsigned long long w[4];
                    philox4x64_10((unsigned long long)(S.seg_t0[i] + g), 0ULL, 5ULL, 0ULL, Ld.seed, 0ULL, w);
                    S.seg_colour[i] = (int)(w[0] >> 63);
                }
            }
            __syncthreads();
        }
        if (early) {
            if (threadIdx.x == 0) {
                unsigned total = 0;
                for (int i = 0; i < S.nsegc; ++i) {
                    if (g >= S.seg_part[i]) continue;
                    const long long a0 = S.seg_base[i] > lo ? S.seg_base[i] : lo;
                    const long long a1 = S.seg_base[i + 1] < hi ? S.seg_base[i + 1] : hi;
                    total += (unsigned)(a1 - a0) * (unsigned)staged_bytes(seg_desc(P, S, i).d);
                }
                S.early_bytes = (int)total;
                if (total) mbar_expect_tx(&S.mbar, total);
            }
            // item i is requested by thread (i + 128) mod 256: with up to 128
            // items the upper warps issue the copies while the lower ones,
            // which hold the items in step 1, already load the count lines
            const long long q = lo + ((threadIdx.x + kThreads / 2) & (kThreads - 1));
            if (q < hi) {
                const int ls = find_segment(S, q);
                if (g < S.seg_part[ls]) {
                    const LatticeDesc &Ld = seg_desc(P, S, ls);
                    const long long t = S.seg_t0[ls] + g;
                    int dx, dy, dz;
                    active_domain(Ld, q - S.seg_base[ls], cycle_colour(S, Ld, ls, t), dx, dy, dz);
                    const long long k = domain_index(Ld.nd, dx, dy, dz);
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                    bulk_copy_g2s(stage + (q - lo) * P.item_bytes, Ld.cells + k * block_words(Ld.d),
                                  staged_bytes(Ld.d), &S.mbar);
                }
            }
        }
        if (P.sub2_any) {
            phase_r(P, S, stage, g, lo, hi, mbar_phase, early);
            if (!*reinterpret_cast<volatile int *>(&S.ok)) return;
        }
        // step 5 one cycle behind, on a thread that normally has no domain
        // in step 1 (a one-round CTA with domains took it during the last
        // flip step)
        if (threadIdx.x == kThreads - 1 && (!early || g == 0 || lo >= hi)) clock_catch_up(P, S, g, lo, true);
        phase_a(P, S, stage, g, lo, hi, early, line);
        __syncthreads();
        for (int i = threadIdx.x; i < S.nsegc; i += blockDim.x) {
            if (g < S.seg_part[i]) {
                const long long t = S.seg_t0[i] + g;
                atomicMax(&P.state[S.seg_slot[i]].rmax[t & (kRmaxRing - 1)], S.seg_rmax[i]);
            }
            S.seg_rmax[i] = 0;
        }
        // the exact R_max is needed before the events; the bounds are not
        // (their reductions are read eight cycles later)
        if (P.exact_any && !grid_barrier(P, S, epoch)) {
            // leaving on an error: the cycle's block copies must land first
            if (early && threadIdx.x == 0 && S.early_bytes > 0) mbar_wait_bounded(P, &S.mbar, mbar_phase);
            __syncthreads();
            return;
        }
        phase_b(P, S, stage, g, lo, hi, mbar_phase, early, line);
        if (!*reinterpret_cast<volatile int *>(&S.ok)) return;
        if (g + 1 < P.ncycles) {
            // After an odd cycle t, colour t + 1 shares no block, count or
            // ghost word with the flips of colour t (the colours differ in two
            // or three parity bits), so its staging and step 1 may start at
            // once.  The flip steps are another matter.  A flip reads the
            // spins of the domains diagonal to its own and moves the classes
            // of sites next to both, so the flip steps of two colours that
            // differ in two bits must not overlap: cycles t and t + 1 for
            // t = 1, 5 mod 8, and cycles t and t + 2 for t = 2, 3, 6, 7
            // mod 8 (their colours differ in the y and z bits).  With the
            // exact R_max, barrier 1 of cycle t + 1, which a CTA reaches only
            // after its flips of cycle t, orders both.  Without it (the
            // bounds of Sec. 3.2 step 4b), a CTA waits after an odd cycle for
            // the CTAs of its near domains (near_wait, one lattice) or for the
            // whole grid (several lattices), and the whole grid meets after
            // every 8th cycle of the launch, which the ring of exact R_max
            // maxima needs: the learned bound reads slot t - 8, which must be
            // final, and slot t + 8 is cleared at t, before any CTA writes it.
            // The row waits after even cycles order the rest
            // (tests/test_sync_schedule.py checks the schedule and the ring).
            const bool odd = P.parity0 >= 0 && (((long long)P.parity0 + g) & 1LL) == 1LL;
            const bool even = P.parity0 >= 0 && !odd;
            const bool skip = odd && P.exact_any;
            const bool grid8 = !P.exact_any && (g & 7LL) == 7LL;
            const bool near = odd && !P.exact_any && !grid8 && P.done && P.nseg == 1;
            if (skip) {
                __syncthreads();
            } else if (even && P.done && !grid8) {
                if (!row_wait(P, S, g)) return;
            } else if (near) {
                if (!near_wait(P, S, g)) return;
            } else if (!grid_barrier(P, S, epoch)) {
                return;
            }
        }
        if (P.rec_every > 0 && (g + 1) % P.rec_every == 0 && (g + 1) / P.rec_every <= P.rec_n) {
            // a recorded cycle: this CTA's counters so far join the record
            // (the clock joins it when it has caught up)
            __syncthreads();
            const long long r = (g + 1) / P.rec_every - 1;
            for (int i = threadIdx.x; i < S.nsegc; i += blockDim.x) {
                // (a lattice whose budget ended earlier adds its final counters)
                ObsRaw &o = P.rec[(long long)S.seg_slot[i] * P.rec_n + r];
                if (S.seg_nflip[i]) atomicAdd(&o.n_flip, S.seg_nflip[i]);
                if (S.seg_nnull[i]) atomicAdd(&o.n_null, S.seg_nnull[i]);
                if (S.seg_dM[i]) atomicAdd(reinterpret_cast<unsigned long long *>(&o.M), S.seg_dM[i]);
                if (S.seg_dB[i]) atomicAdd(reinterpret_cast<unsigned long long *>(&o.B), S.seg_dB[i]);
                atomic_add_u128(&o.null_fx_lo, &o.null_fx_hi, S.seg_fxlo[i], S.seg_fxhi[i]);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == kThreads - 1) {
        clock_catch_up(P, S, 0, lo, false); // the last cycle's step
        // records after the last cycle of a lattice whose budget ended
        // within the launch hold its final clock
        for (int i = 0; P.rec_every > 0 && i < S.nsegc; ++i) {
            if (S.seg_base[i] < lo) continue; // another CTA keeps this clock
            const double c = P.state[S.seg_slot[i]].clock;
            for (long long r = S.seg_part[i] / P.rec_every; r < P.rec_n; ++r)
                P.rec[(long long)S.seg_slot[i] * P.rec_n + r].clock = c;
        }
    }
    for (int i = threadIdx.x; i < S.nsegc; i += blockDim.x) {
        LatticeState &st = P.state[S.seg_slot[i]];
        if (S.seg_nflip[i]) atomicAdd(&st.n_flip, S.seg_nflip[i]);
        if (S.seg_nnull[i]) atomicAdd(&st.n_null, S.seg_nnull[i]);
        if (S.seg_dM[i]) atomicAdd(reinterpret_cast<unsigned long long *>(&st.M), S.seg_dM[i]);
        if (S.seg_dB[i]) atomicAdd(reinterpret_cast<unsigned long long *>(&st.B), S.seg_dB[i]);
        atomic_add_u128(&st.null_fx_lo, &st.null_fx_hi, S.seg_fxlo[i], S.seg_fxhi[i]);
        if (S.seg_base[i] >= lo) { // this CTA owns the lattice's first active domain
            st.t = S.seg_t0[i] + S.seg_part[i];
            if (st.budget >= 0) st.budget -= S.seg_part[i];
        }
    }
}

} // namespace

KernelShape cycle_kernel_shape()
{
    KernelShape s;
    s.threads = kThreads;
    s.smem_bytes = kStageBytes;
    return s;
}

int cycle_round_items(int d_max)
{
    const int per = kStageBytes / stage_slot_bytes(d_max);
    return per < kThreads ? per : kThreads;
}

int cycle_kernel_max_blocks_per_sm(int device)
{
    (void)device;
    if (cudaFuncSetAttribute(spkmc_cycles_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kStageBytes) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, spkmc_cycles_kernel, kThreads, kStageBytes) !=
        cudaSuccess)
        return 0;
    return n;
}

int launch_cycles(const LaunchParams &p, int grid, void *stream, bool cooperative)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kStageBytes;
    cfg.stream = (cudaStream_t)stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = cooperative ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return to_status(cudaLaunchKernelEx(&cfg, spkmc_cycles_kernel, p));
}

// The observables of one lattice from its sums (its state, or a record),
// with the operations (and the IEEE roundings) of the host-side read-out:
// E = -J B - H M, m = M / N, m^2, m^4, and the null-rate sum as
// hi + lo 2^-64.
template <typename Sums>
__device__ __forceinline__ spkmc_obs make_obs(const Sums &st, int L, int d, double J, double H)
{
    spkmc_obs o;
    const double N = (double)L * L * L;
    o.cycle = st.t;
    o.clock = st.clock;
    o.M = st.M;
    o.B = st.B;
    o.E = __dsub_rn(__dmul_rn(-J, (double)o.B), __dmul_rn(H, (double)o.M));
    o.m = __ddiv_rn((double)o.M, N);
    o.m2 = __dmul_rn(o.m, o.m);
    o.m4 = __dmul_rn(o.m2, o.m2);
    o.n_flip = (int64_t)st.n_flip;
    o.n_null = (int64_t)st.n_null;
    o.sum_null_rate_fx[0] = st.null_fx_lo;
    o.sum_null_rate_fx[1] = st.null_fx_hi;
    o.sum_null_rate = __dadd_rn(__ull2double_rn(st.null_fx_hi), __dmul_rn(__ull2double_rn(st.null_fx_lo), 0x1p-64));
    o.L = L;
    o.domain_edge = d;
    return o;
}

__global__ void obs_record_kernel(const LatticeState *st, int L, int d, double J, double H, spkmc_obs *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    *out = make_obs(*st, L, d, J, H);
}

int launch_obs_record(const LatticeState *st, int L, int d, double J, double H, spkmc_obs *out, void *stream)
{
    obs_record_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(st, L, d, J, H, out);
    return to_status(cudaGetLastError());
}

// Record r of lattice i: cycle t + min((r + 1) every, the cycles the
// lattice runs), the sums of the state; the clock is written by the launch
// (NaN until then), or is the state's if the lattice does not run.
__global__ void rec_init_kernel(const LatticeState *st, ObsRaw *rec, int nslots, int n, long long every,
                                long long total)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)nslots * n) return;
    const LatticeState &s = st[idx / n];
    const long long r = idx % n;
    const long long part = s.budget < 0 ? total : (s.budget < total ? s.budget : total);
    const long long done = (r + 1) * every < part ? (r + 1) * every : part;
    ObsRaw o;
    o.t = s.t + done;
    o.clock = part == 0 ? s.clock : __longlong_as_double(0x7FF8000000000000LL);
    o.n_flip = s.n_flip;
    o.n_null = s.n_null;
    o.null_fx_lo = s.null_fx_lo;
    o.null_fx_hi = s.null_fx_hi;
    o.M = s.M;
    o.B = s.B;
    rec[idx] = o;
}

__global__ void rec_series_kernel(const LatticeDesc *desc, const ObsRaw *rec, int nslots, int n, spkmc_obs *out)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)nslots * n) return;
    const LatticeDesc &D = desc[idx / n];
    out[idx] = make_obs(rec[idx], D.L, D.d, D.J, D.H);
}

int launch_rec_init(const LatticeState *st, ObsRaw *rec, int nslots, int n, long long every, long long total,
                    void *stream)
{
    const long long m = (long long)nslots * n;
    rec_init_kernel<<<(unsigned)((m + 127) / 128), 128, 0, (cudaStream_t)stream>>>(st, rec, nslots, n, every,
                                                                                    total);
    return to_status(cudaGetLastError());
}

int launch_rec_series(const LatticeDesc *desc, const ObsRaw *rec, int nslots, int n, spkmc_obs *out,
                      void *stream)
{
    const long long m = (long long)nslots * n;
    rec_series_kernel<<<(unsigned)((m + 127) / 128), 128, 0, (cudaStream_t)stream>>>(desc, rec, nslots, n, out);
    return to_status(cudaGetLastError());
}

} // namespace spkmc
