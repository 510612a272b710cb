// Internal types shared by the kernels (spkmc_kernels.cu) and the host
// runtime (spkmc_api.cu).  Device data layout of one lattice, for domain edge d:
//
//   cells   [K][d*d + 6*d] uint16, one contiguous block per domain:
//           rows[d*d]  bit x of slot (y + d*z) is 1 when spin (x,y,z) is +1;
//           ghosts[6][d]  copies of the neighbours' faces that touch the
//           domain (the one-site halo), kept current by the neighbours' flips:
//             0 gxm[z] bit y = spin (x=-1, y, z)   (x = d-1 face of the -x domain)
//             1 gxp[z] bit y = spin (x=d, y, z)    (x = 0 face of the +x domain)
//             2 gym[z] bit x = spin (x, y=-1, z)
//             3 gyp[z] bit x = spin (x, y=d, z)
//             4 gzm[y] bit x = spin (x, y, z=-1)
//             5 gzp[y] bit x = spin (x, y, z=d)
//           so a domain with its halo is 2d^2 + 12d bytes (704 for d = 16),
//           read by one bulk copy;
//   counts  [K][16]   uint32 per class c < 14: bits 0-15 the number of sites
//           of class c in the domain, bits 16-31 the number of those in its
//           lower half (z < d/2), so a class move of one site is a single
//           add of +-(1 + [z < d/2] << 16); words 14, 15 are zero;
//   scratch [K/8][24] 8-byte words: per active domain of the running cycle,
//           the cumulative frequency line cum[0..13], u01, w1 and the 14
//           count words;
//   nrate   [14][d^3 + 1] double: fl(n * r_c) for every count n a domain can
//           hold, computed on the host with the same IEEE product, so step 1
//           looks the products up instead of converting and multiplying.
#pragma once

#include <cstdint>

#include "../../include/spkmc.h"

namespace spkmc {

constexpr int kClasses = 14;
constexpr int kCountStride = 16;   // int32 per domain in counts
constexpr int kScratchStride = 24; // 8-byte words per active domain in scratch
constexpr int kMaxEdge = 16;
constexpr int kPadRow = kMaxEdge + 2;           // padded rows per axis
constexpr int kPadWords = kPadRow * kPadRow;    // words of one padded domain
constexpr int kMaxSegPerCta = 64;               // lattices one CTA may touch
constexpr int kMaxDoneCtas = 4096;              // CTAs of a launch that can use the row waits
constexpr int kMaxNear = 128;       // CTAs a near wait lists before it waits for every CTA
constexpr int kDoneStride = 32;                 // one counter per 128-byte line: CTAs publish and
                                                // poll without sharing a line

struct LatticeDesc {
    uint16_t *cells;
    int32_t *counts;
    double *scratch;
    const double *nrate; // fl(n r_c) at [c * (d^3 + 1) + n]
    spkmc_event *log;
    int64_t log_cap;
    int64_t log_t0;
    double rate[kClasses];
    double J, H;     // coupling and field, for the observables read-out
    double rbound;   // prescribed bound d^3 max r (1 + 2^-32) (Sec. 3.2 step 4b)
    double rmargin;  // growth of R_k between two visits of a colour, a + 12 b
    uint64_t seed;
    int32_t L, d, nd, half;
    int64_t K, Kact;
    int32_t rmode;   // SPKMC_RMAX_*
    int32_t sub2;    // two random colours (class counts recounted at each visit)
};

constexpr double kBoundSlack = 1.0 + 0x1p-32; // rounding cover of the R_max bounds
constexpr int kRmaxRing = 32;                 // exact R_max of cycle t in slot t % 32

// Per-lattice state written by the persistent kernel.
struct LatticeState {
    int64_t t;                      // cycles done
    double clock;
    unsigned long long n_flip;
    unsigned long long n_null;
    unsigned long long null_fx_lo;  // sum of floor(r_0k * 2^64), 128-bit
    unsigned long long null_fx_hi;
    int64_t budget;                 // cycles left; < 0 = unlimited
    unsigned long long rmax[kRmaxRing]; // exact R_max bit patterns of cycle t in slot t % 32:
                                        // written at t, read at t (exact) or t + 8
                                        // (learned), cleared at t + 24
    long long M;                    // sum of spins, kept exact flip by flip
    long long B;                    // forward bond sum, kept exact flip by flip
};

// One lattice's sums after a recorded cycle of a launch (the observables
// follow from them as from the state): the state at the launch's start plus
// every CTA's counters up to that cycle, and the clock once it has caught up.
struct ObsRaw {
    int64_t t;
    double clock;
    unsigned long long n_flip;
    unsigned long long n_null;
    unsigned long long null_fx_lo;
    unsigned long long null_fx_hi;
    long long M;
    long long B;
};

// One lattice's run of active domains in the flat work table.
struct Segment {
    int64_t base; // first flat item
    int32_t slot; // index into desc/state
    int32_t pad;
};

struct LaunchParams {
    const LatticeDesc *desc;
    LatticeState *state;
    const Segment *seg;   // nseg entries, sorted by base
    int32_t nseg;
    int32_t parity0;      // t % 2 shared by all running lattices at launch, -1 if mixed
    int64_t Q;            // total items
    int64_t ncycles;      // grid cycles of this launch
    unsigned *bar;        // grid-barrier arrival counter (zero at launch)
    unsigned *done;       // per CTA c at done[c * kDoneStride]: cycles it has finished in this launch
                          // (zero at launch), for the wait on the CTAs that share its rows after an
                          // even cycle; nullptr = none
    int *err;             // first error code raised on the device
    long long timeout_ns; // barrier time limit
    int skip_cta;         // debug: CTA that never arrives (-1 = none)
    int round_items;      // active domains per phase-B round (staging capacity)
    int item_bytes;       // staging bytes per domain (largest edge of the launch)
    int exact_any;        // some lattice pads to the exact R_max: reduce before the events
    int sub2_any;         // some lattice uses two random colours: draw colours, recount
    int rec_n;            // records per lattice (rec_every > 0)
    int64_t rec_every;    // record after every rec_every cycles of the launch; 0 = none
    ObsRaw *rec;          // [slot][rec_n] records
};

// u16 words and bytes of one domain block (rows and ghost faces).
__host__ __device__ constexpr int block_words(int d) { return d * d + 6 * d; }
__host__ __device__ constexpr int staged_bytes(int d) { return 2 * block_words(d); }
// Staging slot of one domain in shared memory: the block, then (in the last
// 64 bytes of the slot) the domain's 14 class count words of the cycle; the
// slot is an odd number of 16-byte units, so that consecutive slots start in
// different shared-memory banks.
__host__ __device__ constexpr int stage_slot_bytes(int d) { return (((staged_bytes(d) + 64) / 16) | 1) * 16; }
constexpr int kSlotCountBytes = 64; // count words at the end of each staging slot
constexpr int kStageBytes = 88 * 1024; // phase-B staging area per CTA

// Host-side launch helpers implemented in spkmc_kernels.cu.
struct KernelShape {
    int threads;
    int smem_bytes;
};
KernelShape cycle_kernel_shape();
int cycle_kernel_max_blocks_per_sm(int device);
int launch_cycles(const LaunchParams &p, int grid, void *stream, bool cooperative);
int launch_init_rows(const LatticeDesc &d, int init, void *stream);
int launch_pack_rows(const LatticeDesc &d, const int8_t *dev_spins, void *stream);
// With `gate` (a device int), the unpack writes nothing when *gate != 0 at
// the time it runs (an error raised by the launches before it).
int launch_unpack_rows(const LatticeDesc &d, int8_t *dev_spins, void *stream, const int *gate = nullptr);
// The same with one bit per site (bit i mod 8 of byte i / 8, 1 for +1).
int launch_pack_bits(const LatticeDesc &d, const uint8_t *dev_bits, void *stream);
int launch_unpack_bits(const LatticeDesc &d, uint8_t *dev_bits, void *stream);
// mode 0: rebuild every domain's ghost faces from its neighbours' rows;
// mode 1: compare and add the number of stale ghost words to *mismatch.
int launch_ghosts(const LatticeDesc &d, int mode, unsigned long long *mismatch, void *stream);
// mode 0: write counts; mode 1: compare with the stored counts and add the
// number of mismatching domains to *mismatch (device int64).
// With MB (mode 0), also M and B (device int64 pair, accumulated) in the same
// pass; the ghost faces must be current.
int launch_count_classes(const LatticeDesc &d, int mode, unsigned long long *mismatch, long long *MB,
                         void *stream);
// Ghost faces from the rows, then class counts (and, with MB, M and B) in one
// pass: one warp per domain.
int launch_refresh(const LatticeDesc &d, long long *MB, void *stream);
// M and B (device int64 pair, accumulated).
int launch_obs_record(const LatticeState *st, int L, int d, double J, double H, spkmc_obs *out, void *stream);
int launch_observables(const LatticeDesc &d, long long *MB, void *stream);
// Records of a launch of `total` cycles for nslots lattices (st[i], desc[i],
// rec[i * n + r]): before it, each record holds the state's sums and its
// cycle; after it, the observables of the filled records.
int launch_rec_init(const LatticeState *st, ObsRaw *rec, int nslots, int n, long long every, long long total,
                    void *stream);
int launch_rec_series(const LatticeDesc *desc, const ObsRaw *rec, int nslots, int n, spkmc_obs *out,
                      void *stream);
// Round size for a launch whose largest domain edge is d_max.
int cycle_round_items(int d_max);

} // namespace spkmc
