// spkmc_api.cu -- host runtime behind the C ABI declared in include/spkmc.h.
//
// A batch owns up to `capacity` lattices (slots).  Each slot holds its device
// arrays (domain blocks, counts, scratch, optional event log) and one entry
// of the device descriptor and state tables.  A run enqueues one persistent
// cooperative launch over the flat table of the running lattices' active
// domains (segments sorted by slot).  A single-lattice handle is a batch of
// capacity one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "spkmc_internal.h"
#include "spkmc_setup.h"

using namespace spkmc;

namespace {

thread_local std::string g_last_error = "no error";

// The grid-barrier counter (first 256 bytes) and the per-CTA counters of
// finished cycles for the row waits.
constexpr size_t kBarBytes = 256 + sizeof(unsigned) * kDoneStride * kMaxDoneCtas;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(SPKMC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// A launch helper's status as the calling entry point's: a CUDA error with its
// message, or the helper's own code (EINVAL for a layout it refuses).
int helper_fail(int rc, const char *what)
{
    return rc == SPKMC_ECUDA ? cuda_fail(cudaGetLastError(), what) : fail(rc, "%s refused the lattice", what);
}


#define CUDA_TRY(expr, what)                                                                       \
    do {                                                                                           \
        cudaError_t e_ = (expr);                                                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);                                         \
    } while (0)

bool valid_edge(int d)
{
    return d == 2 || d == 4 || d == 8 || d == 16;
}

// Rate table of Eq. 3 read as Glauber dynamics: r = 1/(1 + exp(2 sigma (J S + H)/T)),
// class c = 7*[sigma=+1] + u, S = 2u - 6; FP64 with the C library's exp and
// no contraction (the host compiler runs with -ffp-contract=off).
void host_rates(double J, double H, double T, double r[kClasses])
{
    for (int c = 0; c < kClasses; ++c) {
        const double sigma = c >= 7 ? 1.0 : -1.0;
        const double S = (double)(2 * (c % 7) - 6);
        double field = J * S;
        field = field + H;
        const double dE = 2.0 * sigma * field;
        const double x = dE / T;
        r[c] = 1.0 / (1.0 + std::exp(x));
    }
}

// Bounds of Sec. 3.2 step 4b from the rate table: the prescribed maximum
// aggregate rate d^3 max_c r_c and the growth margin a + 12 b of the learned
// bound (a: largest change of a flipped site's rate at fixed S; b: largest
// change of a rate when S moves by 2), see SPKMC_RMAX_LEARNED.
void host_bounds(int d, const double r[kClasses], double *prescribed, double *margin)
{
    double top = r[0];
    for (int c = 1; c < kClasses; ++c)
        if (r[c] > top) top = r[c];
    const double nk = (double)d * d * d;
    *prescribed = (nk * top) * kBoundSlack;
    double a = 0.0, b = 0.0;
    for (int u = 0; u < 7; ++u)
        if (std::fabs(r[7 + u] - r[u]) > a) a = std::fabs(r[7 + u] - r[u]);
    for (int sg = 0; sg < 2; ++sg)
        for (int u = 0; u < 6; ++u)
            if (std::fabs(r[7 * sg + u + 1] - r[7 * sg + u]) > b) b = std::fabs(r[7 * sg + u + 1] - r[7 * sg + u]);
    *margin = a + 12.0 * b;
}

void fill_physics(LatticeDesc &D, const spkmc_params *p, int d)
{
    host_rates(p->J, p->H, p->T, D.rate);
    host_bounds(d, D.rate, &D.rbound, &D.rmargin);
    D.rmode = p->rmax_mode;
    D.sub2 = p->sublattice == SPKMC_SUBLATTICE_2_RANDOM;
    D.J = p->J;
    D.H = p->H;
}

// R_max history of spkmc_state (cycles t-8 .. t-1) <-> the device ring.
void hist_to_ring(const double hist[8], long long t, unsigned long long ring[kRmaxRing])
{
    for (int i = 0; i < kRmaxRing; ++i) ring[i] = 0ULL;
    for (int i = 0; i < 8; ++i) {
        unsigned long long bits;
        std::memcpy(&bits, &hist[i], 8);
        ring[(t - 8 + i) & (kRmaxRing - 1)] = bits;
    }
}

void ring_to_hist(const unsigned long long ring[kRmaxRing], long long t, double hist[8])
{
    for (int i = 0; i < 8; ++i) std::memcpy(&hist[i], &ring[(t - 8 + i) & (kRmaxRing - 1)], 8);
}

int check_hist(const double hist[8])
{
    for (int i = 0; i < 8; ++i)
        if (!std::isfinite(hist[i]) || hist[i] < 0.0)
            return fail(SPKMC_EINVAL, "rmax_hist[%d] must be finite and >= 0", i);
    return SPKMC_OK;
}

int check_params(const spkmc_params *p, int *d_out)
{
    if (!p) return fail(SPKMC_EINVAL, "params is NULL");
    if (!std::isfinite(p->J) || !std::isfinite(p->H)) return fail(SPKMC_EINVAL, "J and H must be finite");
    if (!(p->T > 0.0) || !std::isfinite(p->T)) return fail(SPKMC_EINVAL, "T must be finite and > 0");
    if (p->L <= 0) return fail(SPKMC_EINVAL, "L must be positive (got %d)", p->L);
    int d = p->domain_edge;
    if (d == 0) d = spkmc_resolve_domain_edge(p->L);
    if (!valid_edge(d))
        return fail(SPKMC_EINVAL, "domain edge must be 2, 4, 8 or 16 (got %d for L=%d)",
                    p->domain_edge, p->L);
    if (p->L % (2 * d) != 0)
        return fail(SPKMC_EINVAL, "L %% (2d) must be 0 so the 8 colours tile the lattice (L=%d, d=%d)",
                    p->L, d);
    if (p->init != SPKMC_INIT_HOT && p->init != SPKMC_INIT_COLD)
        return fail(SPKMC_EINVAL, "init must be SPKMC_INIT_HOT or SPKMC_INIT_COLD");
    if (p->event_log_capacity < 0) return fail(SPKMC_EINVAL, "event_log_capacity must be >= 0");
    if (p->rmax_mode != SPKMC_RMAX_EXACT && p->rmax_mode != SPKMC_RMAX_PRESCRIBED &&
        p->rmax_mode != SPKMC_RMAX_LEARNED)
        return fail(SPKMC_EINVAL, "rmax_mode must be SPKMC_RMAX_EXACT, _PRESCRIBED or _LEARNED (got %d)",
                    p->rmax_mode);
    if (p->sublattice != SPKMC_SUBLATTICE_8_ROTATING && p->sublattice != SPKMC_SUBLATTICE_2_RANDOM)
        return fail(SPKMC_EINVAL, "sublattice must be SPKMC_SUBLATTICE_8_ROTATING or _2_RANDOM (got %d)",
                    p->sublattice);
    if (p->sublattice == SPKMC_SUBLATTICE_2_RANDOM && p->rmax_mode == SPKMC_RMAX_LEARNED)
        return fail(SPKMC_EINVAL, "the learned R_max bound needs the eight-colour rotation");
    const long long nd = p->L / d;
    if (nd * nd * nd > (1LL << 31) - 1) return fail(SPKMC_EINVAL, "too many domains (L/d)^3 for int32 ids");
    *d_out = d;
    return SPKMC_OK;
}

struct Sizes {
    long long K, Kact, cells_b, counts_b, scratch_b, log_b, nrate_b;
    long long total() const { return cells_b + counts_b + scratch_b + log_b + nrate_b; }
};

// The products fl(n r_c) of step 1 for n = 0 .. d^3, class-major (host FP64,
// no contraction: the same rounding as the device's __dmul_rn).
std::vector<double> host_nrate(int d, const double r[kClasses])
{
    const long long n1 = (long long)d * d * d + 1;
    std::vector<double> t((size_t)(kClasses * n1));
    for (int c = 0; c < kClasses; ++c)
        for (long long n = 0; n < n1; ++n) t[(size_t)(c * n1 + n)] = (double)n * r[c];
    return t;
}

Sizes sizes_of(int L, int d, long long log_cap, int sublattice)
{
    Sizes s;
    const long long nd = L / d;
    s.K = nd * nd * nd;
    s.Kact = sublattice == SPKMC_SUBLATTICE_2_RANDOM ? s.K / 2 : s.K / 8;
    auto up = [](long long b) { return (b + 255) & ~255LL; };
    s.cells_b = up(s.K * staged_bytes(d));
    s.counts_b = up(s.K * kCountStride * 4);
    s.scratch_b = up(s.Kact * kScratchStride * 8);
    s.log_b = up(log_cap * (long long)sizeof(spkmc_event));
    s.nrate_b = up(kClasses * ((long long)d * d * d + 1) * 8);
    return s;
}

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev)
    {
        if (dev < 0) return;
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            cudaSetDevice(dev);
            changed = true;
        }
    }
    ~DeviceGuard()
    {
        if (changed) cudaSetDevice(prev);
    }
};

} // namespace

struct Slot {
    bool live = false;
    bool done_reported = false;
    spkmc_params params{};
    int d = 0;
    Sizes sz{};
    LatticeDesc desc{};   // host copy of the device descriptor
    long long t = 0;      // host mirror of the cycle counter
    long long budget = -1;
    void *blocks[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    size_t block_bytes[5] = {0, 0, 0, 0, 0};
};

struct spkmc_batch {
    spkmc_config cfg{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int capacity = 0;
    std::vector<Slot> slots;
    LatticeDesc *d_desc = nullptr;
    LatticeState *d_state = nullptr;
    Segment *d_seg = nullptr;
    unsigned *d_bar = nullptr;
    int *d_err = nullptr;
    long long *d_MB = nullptr;
    spkmc_obs *d_obs = nullptr; // per-slot observables records for the asynchronous read-out
    ObsRaw *d_rec = nullptr;    // [slot][rec_cap] sums of a recorded run
    spkmc_obs *d_rec_obs = nullptr; // [rec_cap] their observables
    int rec_cap = 0;
    unsigned long long *d_mismatch = nullptr;
    // pinned host staging
    LatticeDesc *h_desc = nullptr;
    LatticeState *h_state = nullptr;
    Segment *h_seg = nullptr;
    int *h_err = nullptr;
    long long *h_MB = nullptr;
    int sm_count = 0;
    int max_blocks_per_sm = 0;
    int last_grid = 0;
    int sticky_error = SPKMC_OK;
    std::vector<Segment> uploaded_seg; // segment table currently on the device
    long long live_bytes = 0;
    // second stream and events of the layer-pipelined spin write (made on
    // first use)
    static constexpr int kWriteSlabs = 16;
    cudaStream_t aux = nullptr;
    cudaEvent_t ev[kWriteSlabs + 1] = {};

    void *dev_alloc(size_t bytes)
    {
        if (bytes == 0) bytes = 256;
        if (cfg.alloc) return cfg.alloc(bytes, (void *)stream, cfg.alloc_ctx);
        void *p = nullptr;
        if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void dev_free(void *p, size_t bytes)
    {
        if (!p) return;
        if (cfg.free) cfg.free(p, bytes, (void *)stream, cfg.alloc_ctx);
        else cudaFreeAsync(p, stream);
    }
};

struct spkmc_engine {
    spkmc_batch *b = nullptr;
    int slot = 0;
    std::vector<spkmc_graph *> graphs; // live graphs captured on this handle
};

struct spkmc_graph {
    spkmc_t *h = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long cycles_per_launch = 0;
};

namespace {

void free_slot_memory(spkmc_batch *b, Slot &s)
{
    for (int i = 0; i < 5; ++i) {
        b->dev_free(s.blocks[i], s.block_bytes[i]);
        s.blocks[i] = nullptr;
        s.block_bytes[i] = 0;
    }
}

void release_batch(spkmc_batch *b)
{
    if (!b) return;
    DeviceGuard g(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto &s : b->slots)
        if (s.live) free_slot_memory(b, s);
    cudaFree(b->d_desc);
    cudaFree(b->d_state);
    cudaFree(b->d_seg);
    cudaFree(b->d_bar);
    cudaFree(b->d_err);
    cudaFree(b->d_MB);
    cudaFree(b->d_obs);
    cudaFree(b->d_rec);
    cudaFree(b->d_rec_obs);
    cudaFree(b->d_mismatch);
    cudaFreeHost(b->h_desc);
    cudaFreeHost(b->h_state);
    cudaFreeHost(b->h_seg);
    cudaFreeHost(b->h_err);
    cudaFreeHost(b->h_MB);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->aux) {
        cudaStreamSynchronize(b->aux);
        cudaStreamDestroy(b->aux);
    }
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int batch_new(int capacity, const spkmc_config *cfg, spkmc_batch **out)
{
    if (!out) return fail(SPKMC_EINVAL, "out is NULL");
    *out = nullptr;
    if (capacity < 1) return fail(SPKMC_EINVAL, "capacity must be >= 1");
    spkmc_batch *b = new (std::nothrow) spkmc_batch();
    if (!b) return fail(SPKMC_ENOMEM, "host allocation failed");
    if (cfg) b->cfg = *cfg;
    else spkmc_config_init(&b->cfg);
    if (b->cfg.device >= 0) {
        b->device = b->cfg.device;
    } else if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return fail(SPKMC_ECUDA, "no CUDA device");
    }
    DeviceGuard g(b->device);
    auto bail = [&](int code) {
        release_batch(b);
        return code;
    };
    if (b->cfg.stream) {
        b->stream = (cudaStream_t)b->cfg.stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate"));
        b->own_stream = true;
    }
    b->capacity = capacity;
    b->slots.resize(capacity);
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&b->d_desc, sizeof(LatticeDesc) * capacity)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_state, sizeof(LatticeState) * capacity)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_seg, sizeof(Segment) * capacity)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_bar, kBarBytes)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_err, 256)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_MB, 256)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_obs, sizeof(spkmc_obs) * capacity)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_mismatch, 256)) != cudaSuccess ||
        (e = cudaMallocHost(&b->h_desc, sizeof(LatticeDesc) * capacity)) != cudaSuccess ||
        (e = cudaMallocHost(&b->h_state, sizeof(LatticeState) * capacity)) != cudaSuccess ||
        (e = cudaMallocHost(&b->h_seg, sizeof(Segment) * capacity)) != cudaSuccess ||
        (e = cudaMallocHost(&b->h_err, 256)) != cudaSuccess ||
        (e = cudaMallocHost(&b->h_MB, 256)) != cudaSuccess) {
        cudaGetLastError();
        return bail(e == cudaErrorMemoryAllocation ? fail(SPKMC_ENOMEM, "batch tables: out of memory")
                                                   : cuda_fail(e, "batch tables"));
    }
    std::memset(b->h_desc, 0, sizeof(LatticeDesc) * capacity);
    std::memset(b->h_state, 0, sizeof(LatticeState) * capacity);
    if ((e = cudaMemsetAsync(b->d_desc, 0, sizeof(LatticeDesc) * capacity, b->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(b->d_state, 0, sizeof(LatticeState) * capacity, b->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(b->d_err, 0, 256, b->stream)) != cudaSuccess)
        return bail(cuda_fail(e, "batch init"));
    if ((e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device)) !=
        cudaSuccess)
        return bail(cuda_fail(e, "device attributes"));
    b->max_blocks_per_sm = cycle_kernel_max_blocks_per_sm(b->device);
    if (b->max_blocks_per_sm < 1) return bail(fail(SPKMC_ECUDA, "cycle kernel cannot be resident"));
    *out = b;
    return SPKMC_OK;
}

// Report and latch a device-side error; ETIMEOUT / EINTERNAL make the batch
// refuse further runs.
int sync_and_check(spkmc_batch *b)
{
    if (b->sticky_error) return fail(b->sticky_error, "batch stopped after an earlier device error (%d)",
                                     b->sticky_error);
    CUDA_TRY(cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream),
             "read error flag");
    CUDA_TRY(cudaStreamSynchronize(b->stream), "stream synchronize");
    if (*b->h_err != 0) {
        b->sticky_error = *b->h_err;
        if (*b->h_err == SPKMC_ETIMEOUT)
            return fail(SPKMC_ETIMEOUT, "a grid barrier timed out on the device");
        if (*b->h_err == SPKMC_EBOUND)
            return fail(SPKMC_EBOUND, "an active domain's R_k exceeded the R_max bound");
        return fail(*b->h_err, "device reported inconsistent class counts");
    }
    return SPKMC_OK;
}

int upload_slot(spkmc_batch *b, int slot)
{
    b->h_desc[slot] = b->slots[slot].desc;
    CUDA_TRY(cudaMemcpyAsync(b->d_desc + slot, b->h_desc + slot, sizeof(LatticeDesc),
                             cudaMemcpyHostToDevice, b->stream),
             "upload descriptor");
    CUDA_TRY(cudaMemcpyAsync(b->d_state + slot, b->h_state + slot, sizeof(LatticeState),
                             cudaMemcpyHostToDevice, b->stream),
             "upload state");
    // the pinned staging entries are rewritten only after a synchronisation
    CUDA_TRY(cudaStreamSynchronize(b->stream), "stream synchronize");
    return SPKMC_OK;
}

// Ghost faces, class counts and the exact M and B of a slot from its rows,
// in one pass.
int refresh_derived(spkmc_batch *b, int slot)
{
    const LatticeDesc &d = b->slots[slot].desc;
    LatticeState *st = b->d_state + slot;
    CUDA_TRY(cudaMemsetAsync(&st->M, 0, 2 * sizeof(long long), b->stream), "clear M, B");
    if (launch_refresh(d, &st->M, b->stream) != SPKMC_OK)
        return cuda_fail(cudaGetLastError(), "ghost faces and class counts");
    return SPKMC_OK;
}

// Exact M and B of a slot, recomputed from the spins into its device state.
int recompute_MB(spkmc_batch *b, int slot)
{
    LatticeState *st = b->d_state + slot;
    CUDA_TRY(cudaMemsetAsync(&st->M, 0, 2 * sizeof(long long), b->stream), "clear M, B");
    if (launch_observables(b->slots[slot].desc, &st->M, b->stream) != SPKMC_OK)
        return cuda_fail(cudaGetLastError(), "observables kernel");
    return SPKMC_OK;
}

int admit(spkmc_batch *b, const spkmc_params *p, long long cycles, int slot_hint, int *slot_out)
{
    int d = 0;
    int rc = check_params(p, &d);
    if (rc) return rc;
    if (b->sticky_error) return fail(b->sticky_error, "batch stopped after an earlier device error");
    int slot = slot_hint;
    if (slot < 0) {
        for (int i = 0; i < b->capacity; ++i)
            if (!b->slots[i].live) {
                slot = i;
                break;
            }
    }
    if (slot < 0 || slot >= b->capacity || b->slots[slot].live) return fail(SPKMC_EBUSY, "no free slot");
    DeviceGuard g(b->device);
    CUDA_TRY(cudaStreamSynchronize(b->stream), "stream synchronize");
    Slot &s = b->slots[slot];
    s = Slot();
    s.params = *p;
    s.params.domain_edge = d;
    s.d = d;
    s.sz = sizes_of(p->L, d, p->event_log_capacity, p->sublattice);
    const long long bytes[5] = {s.sz.cells_b, s.sz.counts_b, s.sz.scratch_b, s.sz.log_b, s.sz.nrate_b};
    for (int i = 0; i < 5; ++i) {
        if (bytes[i] == 0) continue;
        s.blocks[i] = b->dev_alloc((size_t)bytes[i]);
        s.block_bytes[i] = (size_t)bytes[i];
        if (!s.blocks[i]) {
            free_slot_memory(b, s);
            cudaGetLastError();
            return fail(SPKMC_ENOMEM, "device allocation of %lld bytes failed", bytes[i]);
        }
    }
    LatticeDesc &D = s.desc;
    D.cells = (uint16_t *)s.blocks[0];
    D.counts = (int32_t *)s.blocks[1];
    D.scratch = (double *)s.blocks[2];
    D.log = p->event_log_capacity > 0 ? (spkmc_event *)s.blocks[3] : nullptr;
    D.log_cap = p->event_log_capacity;
    D.log_t0 = 0;
    fill_physics(D, p, d);
    D.nrate = (const double *)s.blocks[4];
    D.seed = p->seed;
    D.L = p->L;
    D.d = d;
    D.nd = p->L / d;
    D.half = D.nd / 2;
    D.K = s.sz.K;
    D.Kact = s.sz.Kact;
    {
        const std::vector<double> t = host_nrate(d, D.rate);
        const cudaError_t e = cudaMemcpyAsync(s.blocks[4], t.data(), t.size() * 8, cudaMemcpyHostToDevice,
                                              b->stream);
        if (e != cudaSuccess) {
            free_slot_memory(b, s);
            return cuda_fail(e, "upload rate products");
        }
    }
    std::memset(&b->h_state[slot], 0, sizeof(LatticeState));
    b->h_state[slot].budget = cycles;
    s.t = 0;
    s.budget = cycles;
    rc = upload_slot(b, slot);
    if (!rc) rc = launch_init_rows(D, p->init, b->stream);
    if (!rc) rc = refresh_derived(b, slot);
    if (rc) {
        free_slot_memory(b, s);
        s.live = false;
        return rc == SPKMC_ECUDA ? rc : fail(rc, "lattice initialisation failed");
    }
    s.live = true;
    b->live_bytes += s.sz.total();
    b->uploaded_seg.clear();
    *slot_out = slot;
    return SPKMC_OK;
}

// The flat table of the running lattices (those with cycles left), their
// total active domains Q and the shared cycle parity (-1 if mixed), uploaded
// to the device if it changed (which synchronises the stream first: the
// pinned staging copy is reused).
int segment_table(spkmc_batch *b, std::vector<Segment> &segs, long long &Q, int &parity)
{
    segs.clear();
    Q = 0;
    parity = -2;
    for (int i = 0; i < b->capacity; ++i) {
        Slot &s = b->slots[i];
        if (!s.live || s.budget == 0) continue;
        Segment sg;
        sg.base = Q;
        sg.slot = i;
        sg.pad = 0;
        segs.push_back(sg);
        Q += s.sz.Kact;
        const int par = (int)(s.t & 1);
        parity = parity == -2 ? par : (parity == par ? parity : -1);
    }
    const int nseg = (int)segs.size();
    if (nseg == 0) return SPKMC_OK;
    bool same = segs.size() == b->uploaded_seg.size();
    for (size_t i = 0; same && i < segs.size(); ++i)
        same = segs[i].base == b->uploaded_seg[i].base && segs[i].slot == b->uploaded_seg[i].slot;
    if (!same) {
        CUDA_TRY(cudaStreamSynchronize(b->stream), "stream synchronize"); // pinned staging reuse
        std::memcpy(b->h_seg, segs.data(), sizeof(Segment) * nseg);
        CUDA_TRY(cudaMemcpyAsync(b->d_seg, b->h_seg, sizeof(Segment) * nseg, cudaMemcpyHostToDevice, b->stream),
                 "upload segments");
        b->uploaded_seg = segs;
    }
    return SPKMC_OK;
}

constexpr long long kChunk = 1LL << 18; // cycles of one persistent launch at most

// Records of a run: after every `every` cycles of the launch, into
// rec[slot * n + r] (one launch: n * every <= kChunk).
struct RecReq {
    ObsRaw *rec;
    long long every;
    int n;
};

// One persistent launch (or several, in chunks) over the running lattices.
int run(spkmc_batch *b, long long cycles, const RecReq *rq = nullptr)
{
    if (cycles < 0) return fail(SPKMC_EINVAL, "ncycles must be >= 0");
    if (b->sticky_error) return fail(b->sticky_error, "batch stopped after an earlier device error");
    if (rq && cycles > kChunk) return fail(SPKMC_EINTERNAL, "a recorded run is one launch");
    DeviceGuard g(b->device);
    while (cycles > 0) {
        const long long n = std::min(cycles, kChunk);
        std::vector<Segment> segs;
        long long Q = 0;
        int parity = -2;
        int rc0 = segment_table(b, segs, Q, parity);
        if (rc0) return rc0;
        const int nseg = (int)segs.size();
        if (nseg == 0) return SPKMC_OK;
        // grid: enough CTAs for ~items_per_cta active domains each, within co-residency
        const int per_sm = b->cfg.ctas_per_sm > 0 ? std::min(b->cfg.ctas_per_sm, b->max_blocks_per_sm)
                                                  : b->max_blocks_per_sm;
        long long gmax = (long long)per_sm * b->sm_count;
        if (b->cfg.max_ctas > 0) gmax = std::min<long long>(gmax, b->cfg.max_ctas);
        const long long ipc = b->cfg.items_per_cta > 0 ? b->cfg.items_per_cta : 64;
        long long grid = std::max(1LL, std::min(gmax, (Q + ipc - 1) / ipc));
        // every CTA must see at most kMaxSegPerCta lattices
        for (;;) {
            int worst = 0;
            int si = 0;
            for (long long c = 0; c < grid; ++c) {
                const long long lo = Q * c / grid, hi = Q * (c + 1) / grid;
                while (si + 1 < nseg && segs[si + 1].base <= lo) ++si;
                int sj = si, cnt = 0;
                while (sj < nseg && segs[sj].base < hi) {
                    ++cnt;
                    ++sj;
                }
                worst = std::max(worst, cnt);
            }
            if (worst <= kMaxSegPerCta) break;
            if (grid >= gmax) return fail(SPKMC_EINVAL, "too many small lattices for one launch");
            grid = std::min(gmax, grid * 2);
        }
        CUDA_TRY(cudaMemsetAsync(b->d_bar, 0,
                                 256 + sizeof(unsigned) * kDoneStride * (size_t)std::min<long long>(grid, kMaxDoneCtas),
                                 b->stream),
                 "reset barrier");
        LaunchParams P{};
        P.desc = b->d_desc;
        P.state = b->d_state;
        P.seg = b->d_seg;
        P.nseg = nseg;
        P.parity0 = parity < 0 ? -1 : parity;
        P.Q = Q;
        P.ncycles = n;
        P.bar = b->d_bar;
        P.done = nullptr; // set below when the row waits apply
        P.err = b->d_err;
        P.timeout_ns = b->cfg.barrier_timeout_ns > 0 ? b->cfg.barrier_timeout_ns : 2000000000LL;
        P.skip_cta = b->cfg.debug_skip_arrival_cta;
        int dmax = 2;
        for (const Segment &sg : segs) dmax = std::max(dmax, b->slots[sg.slot].d);
        P.item_bytes = stage_slot_bytes(dmax);
        P.round_items = cycle_round_items(dmax);
        P.exact_any = 0;
        P.sub2_any = 0;
        for (const Segment &sg : segs) {
            P.exact_any |= b->slots[sg.slot].desc.rmode == SPKMC_RMAX_EXACT;
            P.sub2_any |= b->slots[sg.slot].desc.sub2;
        }
        // two random colours: consecutive cycles may use face-adjacent colours
        if (P.sub2_any) P.parity0 = -1;
        // eight colours with a shared t % 2: after an even cycle, wait only for
        // the CTAs that share rows
        if (P.parity0 >= 0 && !P.sub2_any && grid <= kMaxDoneCtas) P.done = b->d_bar + 64;
        if (rq) {
            P.rec = rq->rec;
            P.rec_every = rq->every;
            P.rec_n = rq->n;
        }
        int rc = launch_cycles(P, (int)grid, b->stream, grid > 1);
        if (rc) return cuda_fail(cudaGetLastError(), "persistent cycle launch");
        b->last_grid = (int)grid;
        for (int i = 0; i < nseg; ++i) {
            Slot &s = b->slots[segs[i].slot];
            const long long part = s.budget < 0 ? n : std::min(n, s.budget);
            s.t += part;
            if (s.budget >= 0) s.budget -= part;
        }
        cycles -= n;
    }
    return SPKMC_OK;
}

int slot_check(spkmc_batch *b, int slot)
{
    if (!b) return fail(SPKMC_EINVAL, "handle is NULL");
    if (slot < 0 || slot >= b->capacity || !b->slots[slot].live)
        return fail(SPKMC_EINVAL, "slot %d is not live", slot);
    return SPKMC_OK;
}

int read_state(spkmc_batch *b, int slot, LatticeState *st)
{
    CUDA_TRY(cudaMemcpyAsync(&b->h_state[slot], b->d_state + slot, sizeof(LatticeState),
                             cudaMemcpyDeviceToHost, b->stream),
             "read state");
    int rc = sync_and_check(b);
    if (rc) return rc;
    *st = b->h_state[slot];
    return SPKMC_OK;
}

int observables(spkmc_batch *b, int slot, spkmc_obs *out)
{
    int rc = slot_check(b, slot);
    if (rc) return rc;
    if (!out) return fail(SPKMC_EINVAL, "out is NULL");
    DeviceGuard g(b->device);
    const Slot &s = b->slots[slot];
    LatticeState st;
    if ((rc = read_state(b, slot, &st)) != SPKMC_OK) return rc;
    const double N = (double)s.params.L * s.params.L * s.params.L;
    std::memset(out, 0, sizeof(*out));
    out->cycle = st.t;
    out->clock = st.clock;
    out->M = st.M;
    out->B = st.B;
    out->E = -s.params.J * (double)out->B - s.params.H * (double)out->M;
    out->m = (double)out->M / N;
    out->m2 = out->m * out->m;
    out->m4 = out->m2 * out->m2;
    out->n_flip = (int64_t)st.n_flip;
    out->n_null = (int64_t)st.n_null;
    out->sum_null_rate_fx[0] = st.null_fx_lo;
    out->sum_null_rate_fx[1] = st.null_fx_hi;
    out->sum_null_rate = std::ldexp((double)st.null_fx_hi, 0) + std::ldexp((double)st.null_fx_lo, -64);
    out->L = s.params.L;
    out->domain_edge = s.d;
    return SPKMC_OK;
}

// Spins to the host: one int8 per site, or (packed) one bit per site.
// Device address of n bytes of page-locked host memory mapped into the
// current device's address space (cudaHostAlloc, or cudaHostRegister with
// mapping), or nullptr for any other memory: spins move between such a
// buffer and the rows in the transposing kernel itself, without a staging
// copy.  Both ends of the range must be mapped, at the same offset.
void *mapped_host(const void *host, size_t n)
{
    cudaPointerAttributes a{}, z{};
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess ||
        cudaPointerGetAttributes(&z, (const char *)host + (n - 1)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || z.type != cudaMemoryTypeHost || !a.devicePointer || !z.devicePointer ||
        (char *)z.devicePointer != (char *)a.devicePointer + (n - 1))
        return nullptr;
    return a.devicePointer;
}

int get_spins(spkmc_batch *b, int slot, void *host, size_t n, bool packed = false)
{
    int rc = slot_check(b, slot);
    if (rc) return rc;
    const Slot &s = b->slots[slot];
    const size_t sites = (size_t)s.params.L * s.params.L * s.params.L, N = packed ? sites / 8 : sites;
    if (!host || n != N)
        return fail(SPKMC_EINVAL, packed ? "host buffer must hold L^3 / 8 = %zu bytes" : "host buffer must hold L^3 = %zu int8", N);
    DeviceGuard g(b->device);
    if ((rc = sync_and_check(b)) != SPKMC_OK) return rc;
    if (void *direct = mapped_host(host, N)) {
        rc = packed ? launch_unpack_bits(s.desc, (uint8_t *)direct, b->stream)
                    : launch_unpack_rows(s.desc, (int8_t *)direct, b->stream);
        if (rc) return cuda_fail(cudaGetLastError(), "read spins");
        CUDA_TRY(cudaStreamSynchronize(b->stream), "read spins");
        return SPKMC_OK;
    }
    void *tmp = b->dev_alloc(N);
    if (!tmp) return fail(SPKMC_ENOMEM, "device allocation of %zu bytes failed", N);
    rc = packed ? launch_unpack_bits(s.desc, (uint8_t *)tmp, b->stream)
                : launch_unpack_rows(s.desc, (int8_t *)tmp, b->stream);
    cudaError_t e = rc ? cudaGetLastError()
                       : cudaMemcpyAsync(host, tmp, N, cudaMemcpyDeviceToHost, b->stream);
    cudaError_t e2 = cudaStreamSynchronize(b->stream);
    b->dev_free(tmp, N);
    if (e != cudaSuccess) return cuda_fail(e, "read spins");
    if (e2 != cudaSuccess) return cuda_fail(e2, "read spins");
    return SPKMC_OK;
}

// Rows from host-order spins at src (device-accessible) and the refresh of
// ghost faces, class counts and M, B.  Where the tiled pack applies and the
// lattice has at least 8 domain layers, the layers go in S = 8 or 16 slabs,
// packed on the batch stream in the order 0, S-1, 1, 2, ..., S-2, while a
// second stream refreshes each slab as soon as it and its two z neighbours
// (periodic) are in place: slab 0 after the third pack, slab j after the pack
// of slab j + 1, and slabs S-2 and S-1 after the last.  The transfer of the
// spins (a host-link-bound read when src is mapped host memory) thus
// overlaps most of the refresh (bound by integer arithmetic).
int write_rows(spkmc_batch *b, int slot, const void *src, bool packed)
{
    const LatticeDesc &d = b->slots[slot].desc;
    LatticeState *st = b->d_state + slot;
    const int S = d.nd >= spkmc_batch::kWriteSlabs ? spkmc_batch::kWriteSlabs : 8;
    if (d.nd < 8 || !pack_is_tiled(d, src, packed)) {
        const int rc = packed ? launch_pack_bits(d, (const uint8_t *)src, b->stream)
                              : launch_pack_rows(d, (const int8_t *)src, b->stream);
        if (rc) return helper_fail(rc, "write rows");
        return refresh_derived(b, slot);
    }
    if (!b->aux) { // all or nothing
        cudaStream_t aux = nullptr;
        cudaEvent_t ev[spkmc_batch::kWriteSlabs + 1] = {};
        cudaError_t e = cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking);
        for (int i = 0; e == cudaSuccess && i <= spkmc_batch::kWriteSlabs; ++i)
            e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (cudaEvent_t x : ev)
                if (x) cudaEventDestroy(x);
            if (aux) cudaStreamDestroy(aux);
            return cuda_fail(e, "create stream and events");
        }
        b->aux = aux;
        for (int i = 0; i <= spkmc_batch::kWriteSlabs; ++i) b->ev[i] = ev[i];
    }
    auto z = [&](int i) { return (int)((long long)d.nd * i / S); };
    CUDA_TRY(cudaMemsetAsync(&st->M, 0, 2 * sizeof(long long), b->stream), "clear M, B");
    for (int q = 0; q < S; ++q) {
        const int i = q == 0 ? 0 : (q == 1 ? S - 1 : q - 1); // the slab packed q-th
        // a few CTAs per SM: the refresh of earlier slabs shares the GPU
        int rc = launch_pack_layers(d, src, packed, z(i), z(i + 1), 4 * (b->sm_count > 0 ? b->sm_count : 152),
                                    b->stream);
        if (rc) return helper_fail(rc, "write rows");
        CUDA_TRY(cudaEventRecord(b->ev[q], b->stream), "record event");
        if (q >= 2) { // slab 0 (q = 2), else slab q - 2: its neighbours are packed
            CUDA_TRY(cudaStreamWaitEvent(b->aux, b->ev[q], 0), "wait event");
            const int j = q == 2 ? 0 : q - 2;
            if ((rc = launch_refresh_layers(d, &st->M, z(j), z(j + 1), b->aux)) != SPKMC_OK)
                return helper_fail(rc, "ghost faces and class counts");
        }
    }
    // slabs S-2 and S-1 (the aux stream has waited for the last pack)
    const int rc = launch_refresh_layers(d, &st->M, z(S - 2), z(S), b->aux);
    if (rc) return helper_fail(rc, "ghost faces and class counts");
    CUDA_TRY(cudaEventRecord(b->ev[spkmc_batch::kWriteSlabs], b->aux), "record event");
    CUDA_TRY(cudaStreamWaitEvent(b->stream, b->ev[spkmc_batch::kWriteSlabs], 0), "wait event");
    return SPKMC_OK;
}

int set_spins(spkmc_batch *b, int slot, const void *host, size_t n, bool packed = false)
{
    int rc = slot_check(b, slot);
    if (rc) return rc;
    const Slot &s = b->slots[slot];
    const size_t sites = (size_t)s.params.L * s.params.L * s.params.L, N = packed ? sites / 8 : sites;
    if (!host || n != N)
        return fail(SPKMC_EINVAL, packed ? "host buffer must hold L^3 / 8 = %zu bytes" : "host buffer must hold L^3 = %zu int8", N);
    DeviceGuard g(b->device);
    if ((rc = sync_and_check(b)) != SPKMC_OK) return rc;
    void *direct = mapped_host(host, N);
    void *tmp = direct ? nullptr : b->dev_alloc(N);
    if (!direct && !tmp) return fail(SPKMC_ENOMEM, "device allocation of %zu bytes failed", N);
    cudaError_t e = direct ? cudaSuccess : cudaMemcpyAsync(tmp, host, N, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) // the R_max history described the old spins
        e = cudaMemsetAsync(b->d_state[slot].rmax, 0, sizeof(b->d_state[slot].rmax), b->stream);
    if (e == cudaSuccess) {
        rc = write_rows(b, slot, direct ? direct : tmp, packed);
        if (rc) e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamSynchronize(b->stream);
    if (tmp) b->dev_free(tmp, N);
    if (e != cudaSuccess) return cuda_fail(e, "write spins");
    if (rc) return rc;
    if (e2 != cudaSuccess) return cuda_fail(e2, "write spins");
    return SPKMC_OK;
}

int get_event_log(spkmc_batch *b, int slot, spkmc_event *buf, size_t cap, size_t *n_out)
{
    int rc = slot_check(b, slot);
    if (rc) return rc;
    if (!n_out) return fail(SPKMC_EINVAL, "n_out is NULL");
    *n_out = 0;
    const Slot &s = b->slots[slot];
    DeviceGuard g(b->device);
    if ((rc = sync_and_check(b)) != SPKMC_OK) return rc;
    if (!s.desc.log) return SPKMC_OK;
    const long long logged = std::min<long long>(s.desc.log_cap, (s.t - s.desc.log_t0) * s.desc.Kact);
    const size_t n = (size_t)std::max<long long>(0, std::min<long long>(logged, (long long)cap));
    if (n == 0) return SPKMC_OK;
    if (!buf) return fail(SPKMC_EINVAL, "buf is NULL");
    CUDA_TRY(cudaMemcpyAsync(buf, s.desc.log, n * sizeof(spkmc_event), cudaMemcpyDeviceToHost, b->stream),
             "read event log");
    CUDA_TRY(cudaStreamSynchronize(b->stream), "stream synchronize");
    *n_out = n;
    return SPKMC_OK;
}

// Records of one lattice (slot >= 0) or of every slot (slot < 0) over a
// run of every * nrec cycles in one launch; host_out[i * nrec + r] for the
// i-th recorded slot.
int run_recorded(spkmc_batch *b, int slot, long long every, int nrec, spkmc_obs *host_out)
{
    if (!host_out) return fail(SPKMC_EINVAL, "host_out is NULL");
    if (every <= 0 || nrec <= 0) return fail(SPKMC_EINVAL, "every and nrec must be > 0");
    if (every > kChunk / nrec)
        return fail(SPKMC_EINVAL, "every * nrec must be <= %lld cycles (one launch)", kChunk);
    if (b->sticky_error) return fail(b->sticky_error, "batch stopped after an earlier device error");
    const long long total = every * (long long)nrec;
    if (slot >= 0 && b->slots[slot].budget >= 0 && b->slots[slot].budget < total)
        return fail(SPKMC_EINVAL, "the cycle budget is smaller than the run");
    DeviceGuard g(b->device);
    if (b->rec_cap < nrec) {
        CUDA_TRY(cudaStreamSynchronize(b->stream), "stream synchronize"); // the old buffers may be in use
        cudaFree(b->d_rec);
        cudaFree(b->d_rec_obs);
        b->d_rec = nullptr;
        b->d_rec_obs = nullptr;
        b->rec_cap = 0;
        const size_t m = (size_t)nrec * b->capacity;
        if (cudaMalloc(&b->d_rec, sizeof(ObsRaw) * m) != cudaSuccess ||
            cudaMalloc(&b->d_rec_obs, sizeof(spkmc_obs) * m) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(b->d_rec);
            b->d_rec = nullptr;
            return fail(SPKMC_ENOMEM, "record buffers of %d records per lattice", nrec);
        }
        b->rec_cap = nrec;
    }
    const int first = slot >= 0 ? slot : 0, nslots = slot >= 0 ? 1 : b->capacity;
    ObsRaw *rec = b->d_rec + (size_t)first * nrec;
    if (launch_rec_init(b->d_state + first, rec, nslots, nrec, every, total, b->stream) != SPKMC_OK)
        return cuda_fail(cudaGetLastError(), "record set-up");
    const RecReq rq{b->d_rec, every, nrec};
    int rc = run(b, total, &rq);
    if (rc) return rc;
    spkmc_obs *out = b->d_rec_obs + (size_t)first * nrec;
    if (launch_rec_series(b->d_desc + first, rec, nslots, nrec, out, b->stream) != SPKMC_OK)
        return cuda_fail(cudaGetLastError(), "record read-out");
    CUDA_TRY(cudaMemcpyAsync(host_out, out, sizeof(spkmc_obs) * (size_t)nslots * nrec, cudaMemcpyDeviceToHost,
                             b->stream),
             "records copy");
    return SPKMC_OK;
}

} // namespace

extern "C" {

void spkmc_params_init(spkmc_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->L = 16;
    p->domain_edge = 4;
    p->J = 1.0;
    p->H = 0.0;
    p->T = 4.5115;
    p->seed = 1;
    p->init = SPKMC_INIT_HOT;
}

void spkmc_config_init(spkmc_config *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->device = -1;
    c->debug_skip_arrival_cta = -1;
}

int spkmc_rate_table(double J, double H, double T, double out[14])
{
    if (!out) return fail(SPKMC_EINVAL, "out is NULL");
    if (!std::isfinite(J) || !std::isfinite(H) || !std::isfinite(T) || !(T > 0.0))
        return fail(SPKMC_EINVAL, "J, H, T must be finite and T > 0");
    host_rates(J, H, T, out);
    return SPKMC_OK;
}

int spkmc_rmax_bounds(int32_t d, double J, double H, double T, double *prescribed, double *margin)
{
    if (!prescribed || !margin) return fail(SPKMC_EINVAL, "outputs must not be NULL");
    if (!std::isfinite(J) || !std::isfinite(H) || !std::isfinite(T) || !(T > 0.0))
        return fail(SPKMC_EINVAL, "J, H, T must be finite and T > 0");
    if (!valid_edge(d)) return fail(SPKMC_EINVAL, "domain edge must be 2, 4, 8 or 16 (got %d)", d);
    double r[kClasses];
    host_rates(J, H, T, r);
    host_bounds(d, r, prescribed, margin);
    return SPKMC_OK;
}

int32_t spkmc_resolve_domain_edge(int32_t L)
{
    const int cand[4] = {16, 8, 4, 2};
    for (int d : cand)
        if (L > 0 && L % (2 * d) == 0) return d;
    return 0;
}

int64_t spkmc_bytes_required(const spkmc_params *p)
{
    int d = 0;
    if (check_params(p, &d) != SPKMC_OK) return 0;
    return sizes_of(p->L, d, p->event_log_capacity, p->sublattice).total();
}

int spkmc_create(int32_t L, int32_t domain_edge, double J, double H, double T, uint64_t seed,
                 spkmc_t **out)
{
    spkmc_params p;
    spkmc_params_init(&p);
    p.L = L;
    p.domain_edge = domain_edge;
    p.J = J;
    p.H = H;
    p.T = T;
    p.seed = seed;
    return spkmc_create_ex(&p, nullptr, out);
}

int spkmc_create_ex(const spkmc_params *p, const spkmc_config *cfg, spkmc_t **out)
{
    if (!out) return fail(SPKMC_EINVAL, "out is NULL");
    *out = nullptr;
    int d = 0;
    int rc = check_params(p, &d);
    if (rc) return rc;
    spkmc_batch *b = nullptr;
    if ((rc = batch_new(1, cfg, &b)) != SPKMC_OK) return rc;
    int slot = -1;
    if ((rc = admit(b, p, -1, 0, &slot)) != SPKMC_OK) {
        std::string msg = g_last_error;
        release_batch(b);
        g_last_error = msg;
        return rc;
    }
    spkmc_engine *h = new (std::nothrow) spkmc_engine();
    if (!h) {
        release_batch(b);
        return fail(SPKMC_ENOMEM, "host allocation failed");
    }
    h->b = b;
    h->slot = slot;
    *out = h;
    return SPKMC_OK;
}

void spkmc_destroy(spkmc_t *h)
{
    if (!h) return;
    if (!h->graphs.empty()) {
        // the graphs captured on this handle replay its device memory: once
        // their replays have finished, release their executables and leave
        // the graph handles orphaned (launch refuses, destroy frees them)
        DeviceGuard g(h->b->device);
        cudaStreamSynchronize(h->b->stream);
        for (spkmc_graph *gr : h->graphs) {
            cudaGraphExecDestroy(gr->exec);
            gr->exec = nullptr;
            gr->h = nullptr;
        }
        h->graphs.clear();
    }
    release_batch(h->b);
    delete h;
}

int spkmc_run_cycles(spkmc_t *h, int64_t ncycles)
{
    if (!h) return fail(SPKMC_EINVAL, "handle is NULL");
    return run(h->b, ncycles);
}

int spkmc_run_recorded(spkmc_t *h, int64_t every, int32_t nrec, spkmc_obs *host_out)
{
    if (!h) return fail(SPKMC_EINVAL, "handle is NULL");
    return run_recorded(h->b, h->slot, every, nrec, host_out);
}

int spkmc_synchronize(spkmc_t *h)
{
    if (!h) return fail(SPKMC_EINVAL, "handle is NULL");
    DeviceGuard g(h->b->device);
    return sync_and_check(h->b);
}

int spkmc_graph_create(spkmc_t *h, int64_t cycles_per_step, int32_t steps, spkmc_obs *host_obs,
                       spkmc_graph_t **out)
{
    if (!h || !out) return fail(SPKMC_EINVAL, "NULL argument");
    *out = nullptr;
    if (cycles_per_step <= 0 || steps <= 0) return fail(SPKMC_EINVAL, "cycles_per_step and steps must be > 0");
    if ((cycles_per_step * (long long)steps) % 2 != 0)
        return fail(SPKMC_EINVAL, "steps * cycles_per_step must be even (the launch bakes in the cycle parity)");
    spkmc_batch *b = h->b;
    DeviceGuard g(b->device);
    if (host_obs) {
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, host_obs) != cudaSuccess || pa.type != cudaMemoryTypeHost) {
            cudaGetLastError();
            return fail(SPKMC_EINVAL, "host_obs must be pinned (page-locked) host memory");
        }
    }
    int rc = sync_and_check(b);
    if (rc) return rc;
    std::vector<Segment> segs;
    long long Q = 0;
    int parity = -2;
    if ((rc = segment_table(b, segs, Q, parity)) != SPKMC_OK) return rc; // uploads outside the capture
    Slot &s = b->slots[h->slot];
    const long long t_saved = s.t, budget_saved = s.budget;
    CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    for (int i = 0; i < steps && rc == SPKMC_OK; ++i) {
        rc = run(b, cycles_per_step);
        if (rc == SPKMC_OK && host_obs) rc = spkmc_observables_async(h, host_obs + i);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->stream, &graph);
    s.t = t_saved; // nothing ran yet
    s.budget = budget_saved;
    if (rc != SPKMC_OK || ec != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (rc == SPKMC_OK) rc = cuda_fail(ec, "stream capture");
        cudaGetLastError();
        return rc;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return cuda_fail(ei, "graph instantiate");
    spkmc_graph_t *gr = new (std::nothrow) spkmc_graph_t;
    if (!gr) {
        cudaGraphExecDestroy(exec);
        return fail(SPKMC_ENOMEM, "graph handle");
    }
    gr->h = h;
    gr->exec = exec;
    gr->cycles_per_launch = cycles_per_step * (long long)steps;
    try {
        h->graphs.push_back(gr);
    } catch (...) {
        cudaGraphExecDestroy(exec);
        delete gr;
        return fail(SPKMC_ENOMEM, "graph list");
    }
    *out = gr;
    return SPKMC_OK;
}

int spkmc_graph_launch(spkmc_graph_t *gr)
{
    if (!gr) return fail(SPKMC_EINVAL, "graph is NULL");
    if (!gr->h) return fail(SPKMC_EINVAL, "the graph's lattice was destroyed");
    spkmc_batch *b = gr->h->b;
    if (b->sticky_error) return fail(b->sticky_error, "batch stopped after an earlier device error");
    DeviceGuard g(b->device);
    Slot &s = b->slots[gr->h->slot];
    if (s.budget >= 0 && s.budget < gr->cycles_per_launch)
        return fail(SPKMC_EINVAL, "the lattice's cycle budget is smaller than one graph launch");
    CUDA_TRY(cudaGraphLaunch(gr->exec, b->stream), "graph launch");
    s.t += gr->cycles_per_launch;
    if (s.budget >= 0) s.budget -= gr->cycles_per_launch;
    return SPKMC_OK;
}

void spkmc_graph_destroy(spkmc_graph_t *gr)
{
    if (!gr) return;
    if (gr->h) {
        DeviceGuard g(gr->h->b->device);
        cudaStreamSynchronize(gr->h->b->stream);
        cudaGraphExecDestroy(gr->exec);
        std::vector<spkmc_graph *> &v = gr->h->graphs;
        for (size_t i = 0; i < v.size(); ++i)
            if (v[i] == gr) {
                v.erase(v.begin() + (long)i);
                break;
            }
    } // else the handle was destroyed first and released the executable
    delete gr;
}

int spkmc_observables(spkmc_t *h, spkmc_obs *out)
{
    if (!h) return fail(SPKMC_EINVAL, "handle is NULL");
    return observables(h->b, h->slot, out);
}

int spkmc_observables_async(spkmc_t *h, spkmc_obs *host_out)
{
    if (!h || !host_out) return fail(SPKMC_EINVAL, "NULL argument");
    spkmc_batch *b = h->b;
    if (b->sticky_error) return fail(b->sticky_error, "batch stopped after an earlier device error");
    DeviceGuard g(b->device);
    const Slot &s = b->slots[h->slot];
    spkmc_obs *rec = b->d_obs + h->slot;
    if (launch_obs_record(b->d_state + h->slot, s.params.L, s.d, s.params.J, s.params.H, rec, b->stream) != SPKMC_OK)
        return cuda_fail(cudaGetLastError(), "observables record");
    CUDA_TRY(cudaMemcpyAsync(host_out, rec, sizeof(spkmc_obs), cudaMemcpyDeviceToHost, b->stream),
             "observables copy");
    return SPKMC_OK;
}

int spkmc_get_spins(spkmc_t *h, int8_t *host_buf, size_t n)
{
    if (!h) return fail(SPKMC_EINVAL, "handle is NULL");
    return get_spins(h->b, h->slot, host_buf, n);
}

int spkmc_set_spins(spkmc_t *h, const int8_t *host_buf, size_t n)
{
    if (!h) return fail(SPKMC_EINVAL, "handle is NULL");
    return set_spins(h->b, h->slot, host_buf, n);
}

int spkmc_get_spins_packed(spkmc_t *h, uint8_t *host_bits, size_t nbytes)
{
    if (!h) return fail(SPKMC_EINVAL, "handle is NULL");
    return get_spins(h->b, h->slot, host_bits, nbytes, true);
}

int spkmc_set_spins_packed(spkmc_t *h, const uint8_t *host_bits, size_t nbytes)
{
    if (!h) return fail(SPKMC_EINVAL, "handle is NULL");
    return set_spins(h->b, h->slot, host_bits, nbytes, true);
}

int spkmc_get_event_log(spkmc_t *h, spkmc_event *buf, size_t cap, size_t *n_out)
{
    if (!h) return fail(SPKMC_EINVAL, "handle is NULL");
    return get_event_log(h->b, h->slot, buf, cap, n_out);
}

int spkmc_clear_event_log(spkmc_t *h)
{
    if (!h) return fail(SPKMC_EINVAL, "handle is NULL");
    spkmc_batch *b = h->b;
    DeviceGuard g(b->device);
    int rc = sync_and_check(b);
    if (rc) return rc;
    Slot &s = b->slots[h->slot];
    s.desc.log_t0 = s.t;
    return upload_slot(b, h->slot);
}

int spkmc_get_state(spkmc_t *h, spkmc_state *out)
{
    if (!h || !out) return fail(SPKMC_EINVAL, "NULL argument");
    DeviceGuard g(h->b->device);
    LatticeState st;
    int rc = read_state(h->b, h->slot, &st);
    if (rc) return rc;
    out->cycle = st.t;
    out->clock = st.clock;
    out->n_flip = (int64_t)st.n_flip;
    out->n_null = (int64_t)st.n_null;
    out->sum_null_rate_fx[0] = st.null_fx_lo;
    out->sum_null_rate_fx[1] = st.null_fx_hi;
    ring_to_hist(st.rmax, st.t, out->rmax_hist);
    return SPKMC_OK;
}

int spkmc_set_state(spkmc_t *h, const spkmc_state *in)
{
    if (!h || !in) return fail(SPKMC_EINVAL, "NULL argument");
    if (in->cycle < 0 || in->n_flip < 0 || in->n_null < 0)
        return fail(SPKMC_EINVAL, "state counters must be >= 0");
    if (int rc0 = check_hist(in->rmax_hist)) return rc0;
    spkmc_batch *b = h->b;
    DeviceGuard g(b->device);
    CUDA_TRY(cudaStreamSynchronize(b->stream), "stream synchronize");
    LatticeState &st = b->h_state[h->slot];
    std::memset(&st, 0, sizeof(st));
    st.t = in->cycle;
    st.clock = in->clock;
    st.n_flip = (unsigned long long)in->n_flip;
    st.n_null = (unsigned long long)in->n_null;
    st.null_fx_lo = in->sum_null_rate_fx[0];
    st.null_fx_hi = in->sum_null_rate_fx[1];
    hist_to_ring(in->rmax_hist, in->cycle, st.rmax);
    Slot &s = b->slots[h->slot];
    st.budget = s.budget;
    s.t = in->cycle;
    s.desc.log_t0 = in->cycle;
    b->sticky_error = SPKMC_OK;
    CUDA_TRY(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream), "clear error flag");
    int rc = upload_slot(b, h->slot);
    if (!rc) rc = recompute_MB(b, h->slot);
    if (!rc) CUDA_TRY(cudaStreamSynchronize(b->stream), "stream synchronize");
    return rc;
}

int spkmc_class_counts(spkmc_t *h, int32_t *host_counts, size_t n)
{
    if (!h) return fail(SPKMC_EINVAL, "handle is NULL");
    spkmc_batch *b = h->b;
    const Slot &s = b->slots[h->slot];
    if (!host_counts || n != (size_t)(s.desc.K * kClasses))
        return fail(SPKMC_EINVAL, "buffer must hold 14*K = %lld int32", (long long)(s.desc.K * kClasses));
    DeviceGuard g(b->device);
    int rc = sync_and_check(b);
    if (rc) return rc;
    // two-colour lattices keep no class counts between visits: count now
    if (s.desc.sub2 && launch_count_classes(s.desc, 0, nullptr, nullptr, b->stream) != SPKMC_OK)
        return cuda_fail(cudaGetLastError(), "recount");
    std::vector<int32_t> tmp((size_t)(s.desc.K * kCountStride));
    CUDA_TRY(cudaMemcpyAsync(tmp.data(), s.desc.counts, tmp.size() * 4, cudaMemcpyDeviceToHost, b->stream),
             "read counts");
    CUDA_TRY(cudaStreamSynchronize(b->stream), "stream synchronize");
    // the device words carry the lower-half count in bits 16-31
    for (long long k = 0; k < s.desc.K; ++k)
        for (int c = 0; c < kClasses; ++c) host_counts[k * kClasses + c] = tmp[k * kCountStride + c] & 0xFFFF;
    return SPKMC_OK;
}

int spkmc_check_counts(spkmc_t *h, int64_t *mismatched)
{
    if (!h || !mismatched) return fail(SPKMC_EINVAL, "NULL argument");
    spkmc_batch *b = h->b;
    DeviceGuard g(b->device);
    int rc = sync_and_check(b);
    if (rc) return rc;
    CUDA_TRY(cudaMemsetAsync(b->d_mismatch, 0, 8, b->stream), "clear");
    CUDA_TRY(cudaMemsetAsync(b->d_MB, 0, 2 * sizeof(long long), b->stream), "clear");
    const LatticeDesc &D = b->slots[h->slot].desc;
    // two-colour lattices keep no class counts between visits: refresh them
    // (the ghost faces and M, B are still checked)
    if ((rc = launch_count_classes(D, D.sub2 ? 0 : 1, b->d_mismatch, nullptr, b->stream)) != SPKMC_OK)
        return cuda_fail(cudaGetLastError(), "recount");
    if ((rc = launch_ghosts(D, 1, b->d_mismatch, b->stream)) != SPKMC_OK)
        return cuda_fail(cudaGetLastError(), "ghost check");
    if ((rc = launch_observables(D, b->d_MB, b->stream)) != SPKMC_OK)
        return cuda_fail(cudaGetLastError(), "observables kernel");
    CUDA_TRY(cudaMemcpyAsync(b->h_MB, b->d_MB, 2 * sizeof(long long), cudaMemcpyDeviceToHost, b->stream),
             "read");
    CUDA_TRY(cudaMemcpyAsync(&b->h_MB[2], b->d_mismatch, 8, cudaMemcpyDeviceToHost, b->stream), "read");
    CUDA_TRY(cudaMemcpyAsync(&b->h_state[h->slot], b->d_state + h->slot, sizeof(LatticeState),
                             cudaMemcpyDeviceToHost, b->stream),
             "read state");
    CUDA_TRY(cudaStreamSynchronize(b->stream), "stream synchronize");
    const LatticeState &st = b->h_state[h->slot];
    *mismatched = b->h_MB[2] + ((b->h_MB[0] != st.M || b->h_MB[1] != st.B) ? 1 : 0);
    return SPKMC_OK;
}

int spkmc_info_get(spkmc_t *h, spkmc_info *out)
{
    if (!h || !out) return fail(SPKMC_EINVAL, "NULL argument");
    const Slot &s = h->b->slots[h->slot];
    std::memset(out, 0, sizeof(*out));
    out->L = s.params.L;
    out->domain_edge = s.d;
    out->nd = s.desc.nd;
    out->K = s.desc.K;
    out->K_act = s.desc.Kact;
    out->device_bytes = s.sz.total();
    out->grid_ctas = h->b->last_grid;
    out->threads_per_cta = cycle_kernel_shape().threads;
    return SPKMC_OK;
}

int spkmc_batch_create(int32_t capacity, const spkmc_config *cfg, spkmc_batch_t **out)
{
    return batch_new(capacity, cfg, out);
}

void spkmc_batch_destroy(spkmc_batch_t *b)
{
    release_batch(b);
}

int spkmc_batch_admit(spkmc_batch_t *b, const spkmc_params *p, int64_t cycles, int32_t *slot)
{
    if (!b || !slot) return fail(SPKMC_EINVAL, "NULL argument");
    int s = -1;
    int rc = admit(b, p, cycles, -1, &s);
    if (rc == SPKMC_OK) *slot = s;
    return rc;
}

int spkmc_batch_run(spkmc_batch_t *b, int64_t cycles)
{
    if (!b) return fail(SPKMC_EINVAL, "handle is NULL");
    return run(b, cycles);
}

int spkmc_batch_run_recorded(spkmc_batch_t *b, int64_t every, int32_t nrec, spkmc_obs *host_out)
{
    if (!b) return fail(SPKMC_EINVAL, "handle is NULL");
    return run_recorded(b, -1, every, nrec, host_out);
}

int spkmc_batch_poll(spkmc_batch_t *b, int32_t *done_slots, int32_t cap, int32_t *n)
{
    if (!b || !n || (cap > 0 && !done_slots)) return fail(SPKMC_EINVAL, "NULL argument");
    *n = 0;
    DeviceGuard g(b->device);
    int rc = sync_and_check(b);
    if (rc) return rc;
    for (int i = 0; i < b->capacity && *n < cap; ++i) {
        Slot &s = b->slots[i];
        if (s.live && s.budget == 0 && !s.done_reported) {
            s.done_reported = true;
            done_slots[(*n)++] = i;
        }
    }
    return SPKMC_OK;
}

int spkmc_batch_retire(spkmc_batch_t *b, int32_t slot)
{
    int rc = slot_check(b, slot);
    if (rc) return rc;
    DeviceGuard g(b->device);
    CUDA_TRY(cudaStreamSynchronize(b->stream), "stream synchronize");
    Slot &s = b->slots[slot];
    free_slot_memory(b, s);
    b->live_bytes -= s.sz.total();
    s = Slot();
    b->uploaded_seg.clear();
    return SPKMC_OK;
}

int spkmc_batch_synchronize(spkmc_batch_t *b)
{
    if (!b) return fail(SPKMC_EINVAL, "handle is NULL");
    DeviceGuard g(b->device);
    return sync_and_check(b);
}

int spkmc_batch_observables(spkmc_batch_t *b, int32_t slot, spkmc_obs *out)
{
    return observables(b, slot, out);
}

int spkmc_batch_get_spins(spkmc_batch_t *b, int32_t slot, int8_t *host_buf, size_t n)
{
    return get_spins(b, slot, host_buf, n);
}

int spkmc_batch_get_event_log(spkmc_batch_t *b, int32_t slot, spkmc_event *buf, size_t cap,
                              size_t *n_out)
{
    return get_event_log(b, slot, buf, cap, n_out);
}

int spkmc_batch_observables_all(spkmc_batch_t *b, spkmc_obs *out, int32_t cap, int32_t *n_out)
{
    if (!b || !n_out || (cap > 0 && !out)) return fail(SPKMC_EINVAL, "NULL argument");
    *n_out = 0;
    DeviceGuard g(b->device);
    const int n = std::min<int>(cap, b->capacity);
    if (n <= 0) return SPKMC_OK;
    CUDA_TRY(cudaMemcpyAsync(b->h_state, b->d_state, sizeof(LatticeState) * n, cudaMemcpyDeviceToHost, b->stream),
             "read states");
    int rc = sync_and_check(b);
    if (rc) return rc;
    for (int i = 0; i < n; ++i) {
        spkmc_obs &o = out[i];
        std::memset(&o, 0, sizeof(o));
        const Slot &s = b->slots[i];
        if (!s.live) continue;
        const LatticeState &st = b->h_state[i];
        const double N = (double)s.params.L * s.params.L * s.params.L;
        o.cycle = st.t;
        o.clock = st.clock;
        o.M = st.M;
        o.B = st.B;
        o.E = -s.params.J * (double)st.B - s.params.H * (double)st.M;
        o.m = (double)st.M / N;
        o.m2 = o.m * o.m;
        o.m4 = o.m2 * o.m2;
        o.n_flip = (int64_t)st.n_flip;
        o.n_null = (int64_t)st.n_null;
        o.sum_null_rate_fx[0] = st.null_fx_lo;
        o.sum_null_rate_fx[1] = st.null_fx_hi;
        o.sum_null_rate = (double)st.null_fx_hi + std::ldexp((double)st.null_fx_lo, -64);
        o.L = s.params.L;
        o.domain_edge = s.d;
    }
    *n_out = n;
    return SPKMC_OK;
}

int spkmc_batch_usage(spkmc_batch_t *b, int32_t *live_slots, int64_t *device_bytes)
{
    if (!b) return fail(SPKMC_EINVAL, "handle is NULL");
    int live = 0;
    for (const auto &s : b->slots) live += s.live ? 1 : 0;
    if (live_slots) *live_slots = live;
    if (device_bytes) *device_bytes = b->live_bytes;
    return SPKMC_OK;
}

const char *spkmc_last_error(void)
{
    return g_last_error.c_str();
}

} // extern "C"

// ---------------------------------------------------------------------------
// No-allocation variant: all working memory in one file-scope device array.
// ---------------------------------------------------------------------------
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SPKMC_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
int g_noalloc_blocks_per_sm[kNoallocMaxDevices] = {};
int g_noalloc_sms[kNoallocMaxDevices] = {};

// Device address of the array on the current device (a host-side use of
// the symbol itself is not a device address).  It is looked up on every
// call, so a device whose primary context was reset and created again gets
// the address in its new context; the device's SM count and the cycle
// kernel's occupancy are kept from the first call.
int noalloc_base(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(SPKMC_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) return cuda_fail(e, "cudaGetSymbolAddress of the no-allocation scratch");
    if (!g_noalloc_sms[dev]) {
        int sms = 0;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_fail(e, "device attributes");
        const int per = cycle_kernel_max_blocks_per_sm(dev);
        if (per < 1) return fail(SPKMC_ECUDA, "cycle kernel cannot be resident");
        g_noalloc_blocks_per_sm[dev] = per;
        g_noalloc_sms[dev] = sms;
    }
    *out = static_cast<unsigned char *>(ptr);
    return SPKMC_OK;
}

} // namespace

extern "C" int spkmc_run_cycles_noalloc(const spkmc_params *p, int8_t *dev_spins, spkmc_state *state,
                                        int64_t ncycles, void *stream)
{
    int d = 0;
    int rc = check_params(p, &d);
    if (rc) return rc;
    if (!dev_spins || !state) return fail(SPKMC_EINVAL, "dev_spins and state must not be NULL");
    if (ncycles < 0) return fail(SPKMC_EINVAL, "ncycles must be >= 0");
    if (p->event_log_capacity != 0) return fail(SPKMC_EINVAL, "the no-allocation variant keeps no event log");
    if (state->cycle < 0 || state->n_flip < 0 || state->n_null < 0)
        return fail(SPKMC_EINVAL, "state counters must be >= 0");
    if ((rc = check_hist(state->rmax_hist)) != SPKMC_OK) return rc;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    unsigned char *base = nullptr;
    if ((rc = noalloc_base(dev, &base)) != SPKMC_OK) return rc;

    // carve the array: tables first, then the lattice
    const Sizes sz = sizes_of(p->L, d, 0, p->sublattice);
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    size_t off = 0;
    LatticeDesc *d_desc = reinterpret_cast<LatticeDesc *>(base + off);
    off += up(sizeof(LatticeDesc));
    LatticeState *d_state = reinterpret_cast<LatticeState *>(base + off);
    off += up(sizeof(LatticeState));
    Segment *d_seg = reinterpret_cast<Segment *>(base + off);
    off += up(sizeof(Segment));
    unsigned *d_bar = reinterpret_cast<unsigned *>(base + off);
    off += up(kBarBytes);
    int *d_err = reinterpret_cast<int *>(base + off);
    off += 256;
    const size_t lattice_at = off;
    off += (size_t)sz.cells_b + (size_t)sz.counts_b + (size_t)sz.scratch_b + (size_t)sz.nrate_b;
    if (off > SPKMC_NOALLOC_SCRATCH_BYTES)
        return fail(SPKMC_EINVAL, "lattice L=%d d=%d needs %zu bytes of scratch, the no-allocation array has %u",
                    p->L, d, off, SPKMC_NOALLOC_SCRATCH_BYTES);

    LatticeDesc D{};
    D.cells = reinterpret_cast<uint16_t *>(base + lattice_at);
    D.counts = reinterpret_cast<int32_t *>(base + lattice_at + sz.cells_b);
    D.scratch = reinterpret_cast<double *>(base + lattice_at + sz.cells_b + sz.counts_b);
    D.nrate = reinterpret_cast<const double *>(base + lattice_at + sz.cells_b + sz.counts_b + sz.scratch_b);
    D.log = nullptr;
    D.log_cap = 0;
    D.log_t0 = 0;
    fill_physics(D, p, d);
    D.seed = p->seed;
    D.L = p->L;
    D.d = d;
    D.nd = p->L / d;
    D.half = D.nd / 2;
    D.K = sz.K;
    D.Kact = sz.Kact;
    LatticeState st{};
    st.t = state->cycle;
    st.clock = state->clock;
    st.n_flip = (unsigned long long)state->n_flip;
    st.n_null = (unsigned long long)state->n_null;
    st.null_fx_lo = state->sum_null_rate_fx[0];
    st.null_fx_hi = state->sum_null_rate_fx[1];
    hist_to_ring(state->rmax_hist, state->cycle, st.rmax);
    st.budget = -1; // M and B start at zero
    Segment seg{};
    seg.base = 0;
    seg.slot = 0;
    cudaStream_t s = (cudaStream_t)stream;

    // set-up: this call's tables (the array keeps the previous call's bytes)
    CUDA_TRY(cudaMemcpyAsync(d_desc, &D, sizeof(D), cudaMemcpyHostToDevice, s), "upload descriptor");
    CUDA_TRY(cudaMemcpyAsync(d_state, &st, sizeof(st), cudaMemcpyHostToDevice, s), "upload state");
    CUDA_TRY(cudaMemcpyAsync(d_seg, &seg, sizeof(seg), cudaMemcpyHostToDevice, s), "upload segment");
    const std::vector<double> nrate = host_nrate(d, D.rate);
    CUDA_TRY(cudaMemcpyAsync(const_cast<double *>(D.nrate), nrate.data(), nrate.size() * 8, cudaMemcpyHostToDevice, s),
             "upload rate products");
    CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), s), "clear error flag");
    if ((rc = launch_pack_rows(D, dev_spins, s)) != SPKMC_OK) return helper_fail(rc, "pack spins");
    if ((rc = launch_refresh(D, nullptr, s)) != SPKMC_OK) return helper_fail(rc, "ghost faces and class counts");

    // the cycles, in launches of at most 2^18 cycles, as spkmc_run_cycles
    const long long per_sm = g_noalloc_blocks_per_sm[dev];
    const long long gmax = per_sm * g_noalloc_sms[dev];
    long long grid = std::max(1LL, std::min(gmax, (sz.Kact + 63) / 64));
    long long left = ncycles, t = state->cycle;
    while (left > 0) {
        const long long n = std::min(left, 1LL << 18);
        CUDA_TRY(cudaMemsetAsync(d_bar, 0,
                                 256 + sizeof(unsigned) * kDoneStride * (size_t)std::min<long long>(grid, kMaxDoneCtas), s),
                 "reset barrier");
        LaunchParams P{};
        P.desc = d_desc;
        P.state = d_state;
        P.seg = d_seg;
        P.nseg = 1;
        P.parity0 = (int)(t & 1);
        P.Q = sz.Kact;
        P.ncycles = n;
        P.bar = d_bar;
        P.done = nullptr;
        P.err = d_err;
        P.timeout_ns = 2000000000LL;
        P.skip_cta = -1;
        P.item_bytes = stage_slot_bytes(d);
        P.round_items = cycle_round_items(d);
        P.exact_any = p->rmax_mode == SPKMC_RMAX_EXACT;
        P.sub2_any = D.sub2;
        if (D.sub2) P.parity0 = -1;
        if (P.parity0 >= 0 && !P.sub2_any && grid <= kMaxDoneCtas) P.done = d_bar + 64;
        if ((rc = launch_cycles(P, (int)grid, s, grid > 1)) != SPKMC_OK) return helper_fail(rc, "persistent cycle launch");
        left -= n;
        t += n;
    }
    // the unpack reads the error flag on the device and writes nothing after
    // a failed launch, so dev_spins keeps its input on every error return
    if ((rc = launch_unpack_rows(D, dev_spins, s, d_err)) != SPKMC_OK) return helper_fail(rc, "unpack spins");
    int err = 0;
    CUDA_TRY(cudaMemcpyAsync(&st, d_state, sizeof(st), cudaMemcpyDeviceToHost, s), "read state");
    CUDA_TRY(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s), "read error flag");
    CUDA_TRY(cudaStreamSynchronize(s), "stream synchronize");
    if (err == SPKMC_ETIMEOUT) return fail(SPKMC_ETIMEOUT, "a grid barrier timed out on the device");
    if (err == SPKMC_EBOUND) return fail(SPKMC_EBOUND, "an active domain's R_k exceeded the R_max bound");
    if (err != 0) return fail(err, "device reported inconsistent class counts");
    state->cycle = st.t;
    state->clock = st.clock;
    state->n_flip = (int64_t)st.n_flip;
    state->n_null = (int64_t)st.n_null;
    state->sum_null_rate_fx[0] = st.null_fx_lo;
    state->sum_null_rate_fx[1] = st.null_fx_hi;
    ring_to_hist(st.rmax, st.t, state->rmax_hist);
    return SPKMC_OK;
}
