// spkmc_setup_kernels.cu -- sm_103a kernels that set a lattice up and read
// it out, outside the cycle: the hot and cold start, the transfer of the
// spins between host order (one int8 or one bit per site) and the domain
// rows, the ghost faces, the 14 class counts of Sec. 3.1 step 1 and the
// exact M and B (Eq. 1, Eq. 4), built or checked.
#include "spkmc_device.cuh"
#include "spkmc_setup.h"

namespace spkmc {

namespace {

// ---------------------------------------------------------------------------
// Set-up and read-out kernels
// ---------------------------------------------------------------------------
template <int D>
__global__ void init_rows_kernel(LatticeDesc Ld, int init)
{
    const long long nrows = Ld.K * (D * D);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nrows;
         i += (long long)gridDim.x * blockDim.x) {
        const long long k = i / (D * D);
        const int r = (int)(i % (D * D));
        int dx, dy, dz;
        domain_coords(Ld, k, dx, dy, dz);
        uint32_t row = (1u << D) - 1u;
        if (init == SPKMC_INIT_HOT) {
            const long long X0 = (long long)dx * D, Y = (long long)dy * D + r % D,
                            Z = (long long)dz * D + r / D;
            const long long g0 = X0 + (long long)Ld.L * (Y + (long long)Ld.L * Z);
            unsigned long long w[4];
            philox4x64_10((unsigned long long)(g0 >> 8), 0ULL, 3ULL, 0ULL, Ld.seed, 0ULL, w);
            const int off = (int)(g0 & 255);
            row = (uint32_t)((w[off >> 6] >> (off & 63)) & ((1ULL << D) - 1ULL));
        }
        block_of<D>(Ld, k)[r] = (uint16_t)row;
    }
}

template <int D>
__device__ __forceinline__ long long first_site_of_row(const LatticeDesc &Ld, long long k, int r)
{
    int dx, dy, dz;
    domain_coords(Ld, k, dx, dy, dz);
    return (long long)dx * D +
           (long long)Ld.L * ((long long)dy * D + r % D + (long long)Ld.L * ((long long)dz * D + r / D));
}

template <int D>
__global__ void pack_rows_kernel(LatticeDesc Ld, const int8_t *s8)
{
    const long long nrows = Ld.K * (D * D);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nrows;
         i += (long long)gridDim.x * blockDim.x) {
        const long long k = i / (D * D);
        const int r = (int)(i % (D * D));
        const long long g0 = first_site_of_row<D>(Ld, k, r);
        uint32_t row = 0;
        for (int x = 0; x < D; ++x) row |= (s8[g0 + x] > 0 ? 1u : 0u) << x;
        block_of<D>(Ld, k)[r] = (uint16_t)row;
    }
}

template <int D>
__global__ void unpack_rows_kernel(LatticeDesc Ld, int8_t *s8, const int *gate)
{
    if (gate && ld_volatile_int(gate) != 0) return; // a failed run leaves the caller's spins as they were
    const long long nrows = Ld.K * (D * D);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nrows;
         i += (long long)gridDim.x * blockDim.x) {
        const long long k = i / (D * D);
        const int r = (int)(i % (D * D));
        const long long g0 = first_site_of_row<D>(Ld, k, r);
        const uint32_t row = block_of<D>(Ld, k)[r];
        for (int x = 0; x < D; ++x) s8[g0 + x] = ((row >> x) & 1u) ? int8_t(1) : int8_t(-1);
    }
}

// Transposition between domain rows and spins packed one bit per site in
// global order (bit i mod 8 of byte i / 8 is site i, 1 for +1), by tiles of
// up to 32 domains along x at one (dy, dz).  Their D*D rows r = y + D z cover
// D*D global line segments of 4 D bytes or fewer, which start on a byte
// when L % 8 == 0 (and on a word when L % 32 == 0); the segments sit in
// shared memory, one per row, at a stride of an odd number of words so that
// a warp on consecutive rows meets distinct banks.
constexpr int kTileDomains = 32;
template <int D>
__host__ __device__ constexpr int tile_line_stride() { return ((kTileDomains * D / 32) | 1) * 4; }

struct BitTile {
    int dx0, dy, dz, G, nb; // first domain, extent along x, segment bytes
    long long seg0;         // byte of row 0's segment
};

template <int D>
__device__ __forceinline__ BitTile bit_tile(const LatticeDesc &Ld, long long tile)
{
    const int nd = Ld.nd, ngx = (nd + kTileDomains - 1) / kTileDomains;
    BitTile T;
    const long long q = tile / ngx;
    T.dx0 = (int)(tile - q * ngx) * kTileDomains;
    T.dy = (int)(q % nd);
    T.dz = (int)(q / nd);
    T.G = min(kTileDomains, nd - T.dx0);
    T.nb = T.G * D / 8;
    const long long L = Ld.L;
    T.seg0 = (((long long)T.dz * D * L + (long long)T.dy * D) * L + (long long)T.dx0 * D) / 8;
    return T;
}

// byte offset of row r's segment from the tile's first
template <int D>
__device__ __forceinline__ long long seg_offset(long long L, int r)
{
    return ((long long)(r / D) * L + (r % D)) * (L / 8);
}

template <int D>
__global__ void __launch_bounds__(256) pack_bits_tiled_kernel(LatticeDesc Ld, const uint8_t *bits, long long t0,
                                                              long long t1)
{
    constexpr int S = tile_line_stride<D>();
    __shared__ __align__(16) uint8_t seg[D * D * S];
    const long long L = Ld.L;
    const bool wide = L % 32 == 0;
    for (long long tile = t0 + blockIdx.x; tile < t1; tile += gridDim.x) {
        const BitTile T = bit_tile<D>(Ld, tile);
        if (wide) {
            const int nw = T.nb / 4;
            for (int i = threadIdx.x; i < D * D * nw; i += blockDim.x) {
                const int r = i / nw, w = i - r * nw;
                *reinterpret_cast<uint32_t *>(seg + r * S + 4 * w) =
                    __ldcs(reinterpret_cast<const uint32_t *>(bits + T.seg0 + seg_offset<D>(L, r)) + w);
            }
        } else {
            for (int i = threadIdx.x; i < D * D * T.nb; i += blockDim.x) {
                const int r = i / T.nb, b = i - r * T.nb;
                seg[r * S + b] = bits[T.seg0 + seg_offset<D>(L, r) + b];
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < T.G * D * D; i += blockDim.x) {
            const int j = i / (D * D), r = i % (D * D);
            const uint8_t *ln = seg + r * S;
            uint32_t row;
            if constexpr (D == 16) row = ln[2 * j] | ((uint32_t)ln[2 * j + 1] << 8);
            else if constexpr (D == 8) row = ln[j];
            else row = (ln[(j * D) >> 3] >> ((j * D) & 7)) & ((1u << D) - 1u);
            block_of<D>(Ld, domain_index(Ld.nd, T.dx0 + j, T.dy, T.dz))[r] = (uint16_t)row;
        }
        __syncthreads();
    }
}

template <int D>
__global__ void __launch_bounds__(256) unpack_bits_tiled_kernel(LatticeDesc Ld, uint8_t *bits)
{
    constexpr int S = tile_line_stride<D>();
    __shared__ __align__(16) uint8_t seg[D * D * S];
    const long long L = Ld.L, ntiles = (long long)Ld.nd * Ld.nd * ((Ld.nd + kTileDomains - 1) / kTileDomains);
    const bool wide = L % 32 == 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const BitTile T = bit_tile<D>(Ld, tile);
        if constexpr (D >= 8) { // a row is whole bytes of its segment
            for (int i = threadIdx.x; i < T.G * D * D; i += blockDim.x) {
                const int j = i / (D * D), r = i % (D * D);
                const uint32_t row = block_of<D>(Ld, domain_index(Ld.nd, T.dx0 + j, T.dy, T.dz))[r];
                uint8_t *ln = seg + r * S;
                ln[(D / 8) * j] = (uint8_t)row;
                if constexpr (D == 16) ln[2 * j + 1] = (uint8_t)(row >> 8);
            }
        } else { // 8 / D rows of consecutive domains share a byte
            for (int i = threadIdx.x; i < D * D * T.nb; i += blockDim.x) {
                const int r = i / T.nb, b = i - r * T.nb;
                uint32_t v = 0;
#pragma unroll
                for (int m = 0; m < 8 / D; ++m)
                    v |= (uint32_t)block_of<D>(Ld, domain_index(Ld.nd, T.dx0 + b * (8 / D) + m, T.dy, T.dz))[r]
                         << (m * D);
                seg[r * S + b] = (uint8_t)v;
            }
        }
        __syncthreads();
        if (wide) {
            const int nw = T.nb / 4;
            for (int i = threadIdx.x; i < D * D * nw; i += blockDim.x) {
                const int r = i / nw, w = i - r * nw;
                __stcs(reinterpret_cast<uint32_t *>(bits + T.seg0 + seg_offset<D>(L, r)) + w,
                       *reinterpret_cast<const uint32_t *>(seg + r * S + 4 * w));
            }
        } else {
            for (int i = threadIdx.x; i < D * D * T.nb; i += blockDim.x) {
                const int r = i / T.nb, b = i - r * T.nb;
                bits[T.seg0 + seg_offset<D>(L, r) + b] = seg[r * S + b];
            }
        }
        __syncthreads();
    }
}

// The same tiles for one int8 per site (+1 or -1; a site is +1 where its
// byte is > 0).  A domain's row is D consecutive bytes of its global line, so
// the rows are formed or expanded in registers and shared memory holds the
// tile's rows, [domain][row] at a stride of an odd number of words.
template <int D>
__device__ __forceinline__ long long tile_site0(const LatticeDesc &Ld, const BitTile &T)
{
    const long long L = Ld.L;
    return ((long long)T.dz * D * L + (long long)T.dy * D) * L + (long long)T.dx0 * D;
}

template <int D>
__device__ __forceinline__ long long line_offset(long long L, int r)
{
    return ((long long)(r / D) * L + (r % D)) * L;
}

// 4 bits to 4 bytes of +1 (bit set) or -1
__device__ __forceinline__ uint32_t spins4(uint32_t b)
{
    const uint32_t w = ((b & 0xFu) * 0x00204081u) & 0x01010101u; // bit i to byte i
    return w | ((w ^ 0x01010101u) * 0xFFu);
}

template <int D>
__global__ void __launch_bounds__(256) pack_rows_tiled_kernel(LatticeDesc Ld, const int8_t *s8, long long t0,
                                                              long long t1)
{
    constexpr int S = D * D + 2;
    __shared__ __align__(16) uint16_t rows[kTileDomains * S];
    const long long L = Ld.L;
    for (long long tile = t0 + blockIdx.x; tile < t1; tile += gridDim.x) {
        const BitTile T = bit_tile<D>(Ld, tile);
        const long long site0 = tile_site0<D>(Ld, T);
        for (int i = threadIdx.x; i < D * D * T.G; i += blockDim.x) {
            const int r = i / T.G, j = i - r * T.G;
            const int8_t *src = s8 + site0 + line_offset<D>(L, r) + (long long)j * D;
            uint32_t row = 0;
            if constexpr (D == 16) { // 16-byte aligned: L, x0 and the buffer
                const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(src));
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int x = 0; x < 4; ++x) row |= (uint32_t)((int8_t)(w[q] >> (8 * x)) > 0) << (4 * q + x);
            } else {
#pragma unroll
                for (int x = 0; x < D; ++x) row |= (uint32_t)(src[x] > 0) << x;
            }
            rows[j * S + r] = (uint16_t)row;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < T.G * D * D; i += blockDim.x) {
            const int j = i / (D * D), r = i % (D * D);
            block_of<D>(Ld, domain_index(Ld.nd, T.dx0 + j, T.dy, T.dz))[r] = rows[j * S + r];
        }
        __syncthreads();
    }
}

template <int D>
__global__ void __launch_bounds__(256) unpack_rows_tiled_kernel(LatticeDesc Ld, int8_t *s8, const int *gate)
{
    if (gate && ld_volatile_int(gate) != 0) return; // a failed run leaves the caller's spins as they were
    constexpr int S = D * D + 2;
    __shared__ __align__(16) uint16_t rows[kTileDomains * S];
    const long long L = Ld.L, ntiles = (long long)Ld.nd * Ld.nd * ((Ld.nd + kTileDomains - 1) / kTileDomains);
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const BitTile T = bit_tile<D>(Ld, tile);
        const long long site0 = tile_site0<D>(Ld, T);
        for (int i = threadIdx.x; i < T.G * D * D; i += blockDim.x) {
            const int j = i / (D * D), r = i % (D * D);
            rows[j * S + r] = block_of<D>(Ld, domain_index(Ld.nd, T.dx0 + j, T.dy, T.dz))[r];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < D * D * T.G; i += blockDim.x) {
            const int r = i / T.G, j = i - r * T.G;
            int8_t *dst = s8 + site0 + line_offset<D>(L, r) + (long long)j * D;
            const uint32_t row = rows[j * S + r];
            if constexpr (D == 16) {
                __stcs(reinterpret_cast<uint4 *>(dst),
                       make_uint4(spins4(row), spins4(row >> 4), spins4(row >> 8), spins4(row >> 12)));
            } else {
#pragma unroll
                for (int x = 0; x < D; ++x) dst[x] = ((row >> x) & 1u) ? int8_t(1) : int8_t(-1);
            }
        }
        __syncthreads();
    }
}

// The same one thread per row or byte, for L % 8 != 0 (lines that do not
// start on a byte, possible for D < 8).
template <int D>
__global__ void pack_bits_kernel(LatticeDesc Ld, const uint8_t *bits)
{
    const long long nrows = Ld.K * (D * D);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nrows;
         i += (long long)gridDim.x * blockDim.x) {
        const long long k = i / (D * D);
        const int r = (int)(i % (D * D));
        const long long g0 = first_site_of_row<D>(Ld, k, r);
        uint32_t row = 0;
        if constexpr (D >= 8) { // L and x0 are multiples of 8: the row is D / 8 whole bytes
            row = bits[g0 >> 3];
            if constexpr (D == 16) row |= (uint32_t)bits[(g0 >> 3) + 1] << 8;
        } else {
            for (int x = 0; x < D; ++x) row |= (uint32_t)((bits[(g0 + x) >> 3] >> ((g0 + x) & 7)) & 1) << x;
        }
        block_of<D>(Ld, k)[r] = (uint16_t)row;
    }
}

// Global spins packed one bit per site from the rows: one thread per byte
// (8 consecutive sites in global order, which may span domains and lines).
template <int D>
__global__ void unpack_bits_kernel(LatticeDesc Ld, uint8_t *bits)
{
    const long long L = Ld.L, nbytes = L * L * L / 8;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nbytes;
         b += (long long)gridDim.x * blockDim.x) {
        const long long site = 8 * b;
        int X, Y, Z;
        if (L * L * L <= 0xFFFFFFFFLL) { // 32-bit divisions when the sites fit
            const unsigned sv = (unsigned)site, ul = (unsigned)L, q = sv / ul;
            X = (int)(sv - q * ul);
            Y = (int)(q % ul);
            Z = (int)(q / ul);
        } else {
            X = (int)(site % L);
            Y = (int)((site / L) % L);
            Z = (int)(site / (L * L));
        }
        if constexpr (D >= 8) { // L is a multiple of 8: the byte is 8 bits of one row
            const long long k = domain_index(Ld.nd, X / D, Y / D, Z / D);
            bits[b] = (uint8_t)(block_of<D>(Ld, k)[(Y % D) + D * (Z % D)] >> (X % D));
            continue;
        }
        uint32_t v = 0;
        for (int j = 0; j < 8; ++j) {
            const long long k = domain_index(Ld.nd, X / D, Y / D, Z / D);
            v |= (uint32_t)((block_of<D>(Ld, k)[(Y % D) + D * (Z % D)] >> (X % D)) & 1u) << j;
            if (++X == Ld.L) { // the next site in global order
                X = 0;
                if (++Y == Ld.L) {
                    Y = 0;
                    ++Z;
                }
            }
        }
        bits[b] = (uint8_t)v;
    }
}

// The ghost word (face f, index i) of domain k as the neighbours' rows define it.
template <int D>
__device__ __forceinline__ uint32_t ghost_word(const LatticeDesc &Ld, long long k, int f, int i)
{
    int dx, dy, dz;
    domain_coords(Ld, k, dx, dy, dz);
    const int nd = Ld.nd;
    uint32_t w = 0;
    if (f < 2) { // x faces: bit y of index z
        const long long kn = domain_index(nd, wrap_coord(dx + (f == 0 ? -1 : 1), nd), dy, dz);
        const int xb = f == 0 ? D - 1 : 0;
        const uint16_t *rows = block_of<D>(Ld, kn);
        for (int y = 0; y < D; ++y) w |= (((uint32_t)rows[y + D * i] >> xb) & 1u) << y;
    } else if (f < 4) { // y faces: row (y = d-1 or 0, z = i) of the y neighbour
        const long long kn = domain_index(nd, dx, wrap_coord(dy + (f == 2 ? -1 : 1), nd), dz);
        w = block_of<D>(Ld, kn)[(f == 2 ? D - 1 : 0) + D * i];
    } else { // z faces: row (y = i, z = d-1 or 0) of the z neighbour
        const long long kn = domain_index(nd, dx, dy, wrap_coord(dz + (f == 4 ? -1 : 1), nd));
        w = block_of<D>(Ld, kn)[i + D * (f == 4 ? D - 1 : 0)];
    }
    return w;
}

template <int D>
__global__ void ghosts_kernel(LatticeDesc Ld, int mode, unsigned long long *mismatch)
{
    const long long n = Ld.K * 6 * D;
    unsigned long long bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long k = i / (6 * D);
        const int f = (int)((i / D) % 6), idx = (int)(i % D);
        const uint32_t w = ghost_word<D>(Ld, k, f, idx);
        uint16_t *slot = block_of<D>(Ld, k) + D * D + f * D + idx;
        if (mode == 0) *slot = (uint16_t)w;
        else bad += (*slot != (uint16_t)w);
    }
    if (mode == 1 && bad) atomicAdd(mismatch, bad);
}

// Sites 0..D-1 of two row words in the classify_row layout (site x at bit
// x + 1), side by side: the first row at bits 0..D-1, the second at 16..16+D-1.
template <int D>
__device__ __forceinline__ uint32_t pair_bits(uint32_t a, uint32_t b)
{
    constexpr uint32_t M = (1u << D) - 1u;
    return ((a >> 1) & M) | (((b >> 1) & M) << 16);
}

// With MB (mode 0), M and B of Eq. 1 / Eq. 4 in the same pass: +x bonds
// inside each row and against the +x ghost, +y and +z bonds against the next
// row or the ghost faces.  With ghosts (mode 0), the warp first forms the
// domain's ghost faces from the neighbours' rows and writes them out, and
// classifies from a copy of the block in shared memory; otherwise the ghost
// faces must be current.
template <int D>
__global__ void __launch_bounds__(256, 5) count_classes_kernel(LatticeDesc Ld, int mode,
                                                            unsigned long long *mismatch, long long *MB, int ghosts,
                                                            long long k0, long long k1)
{
    __shared__ __align__(16) uint16_t staged[8][block_words(D)];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr uint32_t V = ((1u << D) - 1u) << 1;
    unsigned long long bad = 0;
    long long M = 0, B = 0;
    for (long long k = k0 + blockIdx.x * 8LL + warp; k < k1; k += gridDim.x * 8LL) {
        const uint16_t *blk = block_of<D>(Ld, k);
        if (ghosts) {
            uint16_t *own = block_of<D>(Ld, k), *sb = staged[warp];
            for (int i = lane; i < D * D / 2; i += 32)
                reinterpret_cast<uint32_t *>(sb)[i] = reinterpret_cast<const uint32_t *>(own)[i];
            for (int i = lane; i < 6 * D; i += 32) {
                const uint16_t w = (uint16_t)ghost_word<D>(Ld, k, i / D, i % D);
                own[D * D + i] = w;
                sb[D * D + i] = w;
            }
            __syncwarp();
            blk = sb;
        }
        const uint16_t *gh = blk + D * D;
        int cnt[kClasses];
#pragma unroll
        for (int c = 0; c < kClasses; ++c) cnt[c] = 0;
        int m = 0, b = 0;
        // rows (y, z) and (y + 1, z), y even, side by side in one word (sites
        // at bits 0..D-1 and 16..16+D-1), so that each mask is counted once
        // for both
        for (int q = lane; q < D * D / 2; q += 32) {
            const int r = 2 * q, y = r % D, z = r / D;
            const RowPlanes p0 = classify_row<D>(blk, y, z), p1 = classify_row<D>(blk, y + 1, z);
            const uint32_t s = pair_bits<D>(p0.s, p1.s);
            if (MB) { // bit x + 1 of p.s is spin x, x in [-1, D]
                const uint32_t yp1 = (uint32_t)(y + 1 < D - 1 ? blk[r + 2] : gh[3 * D + z]) << 1;
                const uint32_t zp0 = (uint32_t)(z < D - 1 ? blk[r + D] : gh[5 * D + y]) << 1;
                const uint32_t zp1 = (uint32_t)(z < D - 1 ? blk[r + 1 + D] : gh[5 * D + y + 1]) << 1;
                m += 2 * __popc(s) - 2 * D;
                b += 2 * __popc(pair_bits<D>(~(p0.s ^ (p0.s >> 1)), ~(p1.s ^ (p1.s >> 1)))) - 2 * D; // +x
                b += 2 * __popc(pair_bits<D>(~(p0.s ^ p1.s), ~(p1.s ^ yp1))) - 2 * D;                 // +y
                b += 2 * __popc(pair_bits<D>(~(p0.s ^ zp0), ~(p1.s ^ zp1))) - 2 * D;                // +z
            }
            const uint32_t u0 = pair_bits<D>(p0.u0, p1.u0), u1 = pair_bits<D>(p0.u1, p1.u1),
                           u2 = pair_bits<D>(p0.u2, p1.u2);
            const int inc = 1 + ((r < D * D / 2) ? (1 << 16) : 0); // lower half: z < D/2
#pragma unroll
            for (int u = 0; u < 7; ++u) {
                uint32_t e = (u & 1) ? u0 : ~u0;
                e &= (u & 2) ? u1 : ~u1;
                e &= (u & 4) ? u2 : ~u2;
                const int up = __popc(e & s), all = __popc(e & pair_bits<D>(~0u, ~0u));
                cnt[7 + u] += up * inc;
                cnt[u] += (all - up) * inc;
            }
        }
        int differs = 0;
#pragma unroll
        for (int c = 0; c < kClasses; ++c) {
            const int v = __reduce_add_sync(kFull, cnt[c]);
            if (lane == c) {
                if (mode == 0) Ld.counts[k * kCountStride + c] = v;
                else differs = Ld.counts[k * kCountStride + c] != v;
            }
        }
        if (mode == 0 && lane >= kClasses && lane < kCountStride) Ld.counts[k * kCountStride + lane] = 0;
        if (__any_sync(kFull, differs) && lane == 0) ++bad;
        if (MB) {
            M += __reduce_add_sync(kFull, m);
            B += __reduce_add_sync(kFull, b);
        }
        __syncwarp(); // the staged block is read before the next is written
    }
    if (mode == 1 && lane == 0 && bad) atomicAdd(mismatch, bad);
    if (MB && lane == 0 && (M || B)) {
        atomicAdd(reinterpret_cast<unsigned long long *>(MB), (unsigned long long)M);
        atomicAdd(reinterpret_cast<unsigned long long *>(MB + 1), (unsigned long long)B);
    }
}

// M and B of Eq. 1 / Eq. 4, one warp per domain: +x bonds inside each row
// and against the +x ghost, +y and +z bonds against the next row or the
// ghost faces.
template <int D>
__global__ void __launch_bounds__(256) observables_kernel(LatticeDesc Ld, long long *MB)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr uint32_t V = ((1u << D) - 1u) << 1;
    long long M = 0, B = 0;
    for (long long k = blockIdx.x * 8LL + warp; k < Ld.K; k += gridDim.x * 8LL) {
        const uint16_t *blk = block_of<D>(Ld, k);
        const uint16_t *gh = blk + D * D;
        int m = 0, b = 0;
        for (int r = lane; r < D * D; r += 32) {
            const int y = r % D, z = r / D;
            const uint32_t s = ((uint32_t)blk[r] << 1) | ((((uint32_t)gh[1 * D + z] >> y) & 1u) << (D + 1));
            const uint32_t yp = (uint32_t)(y < D - 1 ? blk[r + 1] : gh[3 * D + z]) << 1;
            const uint32_t zp = (uint32_t)(z < D - 1 ? blk[r + D] : gh[5 * D + y]) << 1;
            m += 2 * __popc(s & V) - D;
            b += 2 * __popc(~(s ^ (s >> 1)) & V) - D;
            b += 2 * __popc(~(s ^ yp) & V) - D;
            b += 2 * __popc(~(s ^ zp) & V) - D;
        }
        M += __reduce_add_sync(kFull, m);
        B += __reduce_add_sync(kFull, b);
    }
    if (lane == 0 && (M || B)) {
        atomicAdd(reinterpret_cast<unsigned long long *>(MB), (unsigned long long)M);
        atomicAdd(reinterpret_cast<unsigned long long *>(MB + 1), (unsigned long long)B);
    }
}

} // namespace

#define SPKMC_DISPATCH_D(dval, KERNEL, GRID, BLOCK, STREAM, ...)                                  \
    do {                                                                                          \
        switch (dval) {                                                                           \
        case 2: KERNEL<2><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;                        \
        case 4: KERNEL<4><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;                        \
        case 8: KERNEL<8><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;                        \
        case 16: KERNEL<16><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;                      \
        default: return SPKMC_EINVAL;                                                             \
        }                                                                                         \
    } while (0)

int launch_init_rows(const LatticeDesc &d, int init, void *stream)
{
    const int grid = simple_grid(d.K * d.d * d.d, 256);
    SPKMC_DISPATCH_D(d.d, init_rows_kernel, grid, 256, (cudaStream_t)stream, d, init);
    return to_status(cudaGetLastError());
}

// Tiles of domain layers [z0, z1) (tiles run with dz slowest), and the grid
// for them: at most `cap` CTAs.
inline void layer_tiles(const LatticeDesc &d, int z0, int z1, long long &t0, long long &t1)
{
    const long long per_layer = (long long)d.nd * ((d.nd + kTileDomains - 1) / kTileDomains);
    t0 = z0 * per_layer;
    t1 = z1 * per_layer;
}

inline int tile_grid(long long tiles, int cap)
{
    return (int)(tiles < cap ? (tiles > 0 ? tiles : 1) : cap);
}

bool pack_is_tiled(const LatticeDesc &d, const void *src, bool packed)
{
    return packed ? d.L % 8 == 0 : (d.d != 16 || ((uintptr_t)src & 15) == 0);
}

int launch_pack_layers(const LatticeDesc &d, const void *src, bool packed, int z0, int z1, int cap, void *stream)
{
    if (!pack_is_tiled(d, src, packed) || z0 < 0 || z1 > d.nd || z0 >= z1) return SPKMC_EINVAL;
    long long t0, t1;
    layer_tiles(d, z0, z1, t0, t1);
    const int grid = tile_grid(t1 - t0, cap);
    if (packed)
        SPKMC_DISPATCH_D(d.d, pack_bits_tiled_kernel, grid, 256, (cudaStream_t)stream, d, (const uint8_t *)src, t0,
                         t1);
    else
        SPKMC_DISPATCH_D(d.d, pack_rows_tiled_kernel, grid, 256, (cudaStream_t)stream, d, (const int8_t *)src, t0, t1);
    return to_status(cudaGetLastError());
}

int launch_pack_rows(const LatticeDesc &d, const int8_t *dev_spins, void *stream)
{
    if (pack_is_tiled(d, dev_spins, false)) // vector accesses at d = 16 need 16-byte alignment
        return launch_pack_layers(d, dev_spins, false, 0, d.nd, 2048, stream);
    const int grid = simple_grid(d.K * d.d * d.d, 256);
    SPKMC_DISPATCH_D(d.d, pack_rows_kernel, grid, 256, (cudaStream_t)stream, d, dev_spins);
    return to_status(cudaGetLastError());
}

int launch_unpack_rows(const LatticeDesc &d, int8_t *dev_spins, void *stream, const int *gate)
{
    if (d.d != 16 || ((uintptr_t)dev_spins & 15) == 0) { // vector accesses at d = 16
        const long long tiles = (long long)d.nd * d.nd * ((d.nd + kTileDomains - 1) / kTileDomains);
        SPKMC_DISPATCH_D(d.d, unpack_rows_tiled_kernel, (int)(tiles < 2048 ? tiles : 2048), 256, (cudaStream_t)stream, d,
                         dev_spins, gate);
        return to_status(cudaGetLastError());
    }
    const int grid = simple_grid(d.K * d.d * d.d, 256);
    SPKMC_DISPATCH_D(d.d, unpack_rows_kernel, grid, 256, (cudaStream_t)stream, d, dev_spins, gate);
    return to_status(cudaGetLastError());
}

int launch_pack_bits(const LatticeDesc &d, const uint8_t *dev_bits, void *stream)
{
    if (pack_is_tiled(d, dev_bits, true)) return launch_pack_layers(d, dev_bits, true, 0, d.nd, 2048, stream);
    const int grid = simple_grid(d.K * d.d * d.d, 256);
    SPKMC_DISPATCH_D(d.d, pack_bits_kernel, grid, 256, (cudaStream_t)stream, d, dev_bits);
    return to_status(cudaGetLastError());
}

int launch_unpack_bits(const LatticeDesc &d, uint8_t *dev_bits, void *stream)
{
    if (d.L % 8 == 0) {
        const long long tiles = (long long)d.nd * d.nd * ((d.nd + kTileDomains - 1) / kTileDomains);
        SPKMC_DISPATCH_D(d.d, unpack_bits_tiled_kernel, (int)(tiles < 2048 ? tiles : 2048), 256, (cudaStream_t)stream, d,
                         dev_bits);
        return to_status(cudaGetLastError());
    }
    const long long L = d.L;
    const int grid = simple_grid(L * L * L / 8, 256);
    SPKMC_DISPATCH_D(d.d, unpack_bits_kernel, grid, 256, (cudaStream_t)stream, d, dev_bits);
    return to_status(cudaGetLastError());
}

int launch_ghosts(const LatticeDesc &d, int mode, unsigned long long *mismatch, void *stream)
{
    const int grid = simple_grid(d.K * 6 * d.d, 256);
    SPKMC_DISPATCH_D(d.d, ghosts_kernel, grid, 256, (cudaStream_t)stream, d, mode, mismatch);
    return to_status(cudaGetLastError());
}

int launch_count_classes(const LatticeDesc &d, int mode, unsigned long long *mismatch, long long *MB, void *stream)
{
    const int grid = simple_grid(d.K, 8);
    SPKMC_DISPATCH_D(d.d, count_classes_kernel, grid, 256, (cudaStream_t)stream, d, mode, mismatch, MB, 0, 0LL, d.K);
    return to_status(cudaGetLastError());
}

int launch_refresh(const LatticeDesc &d, long long *MB, void *stream)
{
    return launch_refresh_layers(d, MB, 0, d.nd, stream);
}

int launch_refresh_layers(const LatticeDesc &d, long long *MB, int z0, int z1, void *stream)
{
    if (z0 < 0 || z1 > d.nd || z0 >= z1) return SPKMC_EINVAL;
    const long long layer = (long long)d.nd * d.nd, k0 = z0 * layer, k1 = z1 * layer;
    const int grid = simple_grid(k1 - k0, 8);
    SPKMC_DISPATCH_D(d.d, count_classes_kernel, grid, 256, (cudaStream_t)stream, d, 0, nullptr, MB, 1, k0, k1);
    return to_status(cudaGetLastError());
}

int launch_observables(const LatticeDesc &d, long long *MB, void *stream)
{
    const int grid = simple_grid(d.K, 8);
    SPKMC_DISPATCH_D(d.d, observables_kernel, grid, 256, (cudaStream_t)stream, d, MB);
    return to_status(cudaGetLastError());
}

} // namespace spkmc
