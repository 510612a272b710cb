// spkmc_device.cuh -- device helpers shared by the cycle kernel and the
// set-up kernels: Philox, memory-order primitives, domain geometry and the
// bit-sliced classification of a row (Sec. 3.1 step 1).  Internal linkage:
// each translation unit has its own copy.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "spkmc_internal.h"

namespace spkmc {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kDescCached = 4; // lattice descriptors a CTA keeps in shared memory

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), the counter-based
// generator that gives each domain its own stream (Sec. 3.1, step 4).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64_10(unsigned long long c0, unsigned long long c1,
                                              unsigned long long c2, unsigned long long c3,
                                              unsigned long long k0, unsigned long long k1,
                                              unsigned long long out[4])
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const unsigned long long m0 = 0xD2E7470EE14C6C93ULL, m1 = 0xCA5A826395121157ULL;
        unsigned long long hi0 = __umul64hi(m0, c0), lo0 = m0 * c0;
        unsigned long long hi1 = __umul64hi(m1, c2), lo1 = m1 * c2;
        unsigned long long n0 = hi1 ^ c1 ^ k0;
        unsigned long long n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B97F4A7C15ULL;
        k1 += 0xBB67AE8584CAA73BULL;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// ---------------------------------------------------------------------------
// Memory helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ long long global_timer_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_volatile_int(const int *p)
{
    return *reinterpret_cast<const volatile int *>(p);
}

// XOR into one 16-bit slot through the 32-bit word that holds it.
__device__ __forceinline__ void xor_u16(uint16_t *p, uint32_t bits)
{
    uintptr_t a = reinterpret_cast<uintptr_t>(p);
    uint32_t *w = reinterpret_cast<uint32_t *>(a & ~uintptr_t(3));
    atomicXor(w, bits << ((a & 2) ? 16 : 0));
}

__device__ __forceinline__ void raise_error(int *err, int code)
{
    atomicCAS(err, 0, code);
}

// floor(x * 2^64) for finite x >= 0 as a 128-bit integer (lo, hi).
__device__ __forceinline__ void fixed64(double x, unsigned long long &lo, unsigned long long &hi)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    int e = (int)((b >> 52) & 0x7ff);
    lo = 0;
    hi = 0;
    if (e == 0) return; // zero or subnormal: far below 2^-64
    unsigned long long m = (b & ((1ULL << 52) - 1)) | (1ULL << 52);
    int sh = e - 1011; // x * 2^64 = m * 2^(e - 1075 + 64)
    if (sh >= 64) {
        hi = m << (sh - 64);
    } else if (sh > 0) {
        lo = m << sh;
        hi = m >> (64 - sh);
    } else if (sh == 0) {
        lo = m;
    } else if (sh > -64) {
        lo = m >> (-sh);
    }
}

// 128-bit add into (lo, hi) held in memory, exact and order-independent.
__device__ __forceinline__ void atomic_add_u128(unsigned long long *lo_p, unsigned long long *hi_p,
                                                unsigned long long lo, unsigned long long hi)
{
    if (lo == 0 && hi == 0) return;
    unsigned long long old = atomicAdd(lo_p, lo);
    unsigned long long carry = (old + lo < old) ? 1ULL : 0ULL;
    if (hi + carry) atomicAdd(hi_p, hi + carry);
}

// ---------------------------------------------------------------------------
// Geometry
// ---------------------------------------------------------------------------
// The a-th active domain (ascending index) of the cycle's colour (Sec. 3.2
// step 4a).  Eight colours: the parity class `colour` of (dx, dy, dz).  Two
// colours: (dx + dy + dz) mod 2 = colour, every other dx along each
// (dy, dz) row.  a < K/2 < 2^30: 32-bit unsigned division is exact and much
// cheaper.
__device__ __forceinline__ void active_domain(const LatticeDesc &Ld, long long a, int colour, int &dx, int &dy,
                                              int &dz)
{
    const unsigned ua = (unsigned)a, h = (unsigned)Ld.half;
    const unsigned qx = ua / h;
    if (Ld.sub2) {
        const unsigned nd = (unsigned)Ld.nd, qz = qx / nd;
        dy = (int)(qx - qz * nd);
        dz = (int)qz;
        dx = 2 * (int)(ua - qx * h) + ((dy + dz + colour) & 1);
    } else {
        const unsigned qy = qx / h;
        dx = 2 * (int)(ua - qx * h) + (colour & 1);
        dy = 2 * (int)(qx - qy * h) + ((colour >> 1) & 1);
        dz = 2 * (int)qy + ((colour >> 2) & 1);
    }
}

__device__ __forceinline__ long long domain_index(int nd, int dx, int dy, int dz)
{
    return (long long)dx + (long long)nd * ((long long)dy + (long long)nd * dz);
}

__device__ __forceinline__ void domain_coords(const LatticeDesc &Ld, long long k, int &dx, int &dy, int &dz)
{
    // K = nd^3 < 2^32 for any lattice that fits a GPU: 32-bit divisions
    const unsigned kk = (unsigned)k, nd = (unsigned)Ld.nd, q = kk / nd;
    dx = (int)(kk - q * nd);
    dy = (int)(q % nd);
    dz = (int)(q / nd);
}

__device__ __forceinline__ int wrap_coord(int a, int n)
{
    return a < 0 ? a + n : (a >= n ? a - n : a);
}

template <int D>
__device__ __forceinline__ uint16_t *block_of(const LatticeDesc &Ld, long long k)
{
    return Ld.cells + k * block_words(D);
}

// Address of the row holding global site (X, Y, Z) (coordinates modulo L)
// and the site's bit in it.
template <int D>
__device__ __forceinline__ const uint16_t *row_of_site(const LatticeDesc &Ld, int X, int Y, int Z, int &bit)
{
    X = wrap_coord(X, Ld.L);
    Y = wrap_coord(Y, Ld.L);
    Z = wrap_coord(Z, Ld.L);
    const long long k = domain_index(Ld.nd, X / D, Y / D, Z / D);
    bit = X % D;
    return block_of<D>(Ld, k) + (Y % D) + D * (Z % D);
}

// Spin bit of local site (x, y, z) of a domain block (global or staged),
// with at most one coordinate one step outside [0, D) (read from the ghosts).
template <int D>
__device__ __forceinline__ int block_bit(const uint16_t *blk, int x, int y, int z)
{
    // word and bit chosen with selects, not branches (callers run divergent
    // sites side by side); a coordinate pair outside the halo reads a word of
    // the block (in bounds) and its value is not used
    const bool xo = x < 0 || x >= D, yo = y < 0 || y >= D, zo = z < 0 || z >= D;
    const int cz = z & (D - 1), cy = y & (D - 1);
    int idx = cy + D * cz;
    idx = zo ? D * D + (z < 0 ? 4 : 5) * D + cy : idx;
    idx = yo ? D * D + (y < 0 ? 2 : 3) * D + cz : idx;
    idx = xo ? D * D + (x < 0 ? 0 : 1) * D + cz : idx;
    const int b = (xo ? y : x) & 15;
    return (int)(((uint32_t)blk[idx] >> b) & 1u);
}

// Bit-sliced count of up neighbours for the D sites of row (y, z) of a
// domain block: bit x+1 of s is spin x (x in [-1, D], halo from the ghosts)
// and u = u0 + 2 u1 + 4 u2 per bit position.
struct RowPlanes {
    uint32_t s, u0, u1, u2;
};

template <int D>
__device__ __forceinline__ RowPlanes classify_row(const uint16_t *blk, int y, int z)
{
    const uint16_t *rows = blk, *g = blk + D * D;
    const int r = y + D * z;
    const uint32_t s = ((uint32_t)rows[r] << 1) | (((uint32_t)g[0 * D + z] >> y) & 1u) |
                       ((((uint32_t)g[1 * D + z] >> y) & 1u) << (D + 1));
    const uint32_t a = s << 1, b = s >> 1;
    const uint32_t c = (uint32_t)(y > 0 ? rows[r - 1] : g[2 * D + z]) << 1;
    const uint32_t d = (uint32_t)(y < D - 1 ? rows[r + 1] : g[3 * D + z]) << 1;
    const uint32_t e = (uint32_t)(z > 0 ? rows[r - D] : g[4 * D + y]) << 1;
    const uint32_t f = (uint32_t)(z < D - 1 ? rows[r + D] : g[5 * D + y]) << 1;
    const uint32_t s1 = a ^ b ^ c, c1 = (a & b) | (c & (a ^ b));
    const uint32_t s2 = d ^ e ^ f, c2 = (d & e) | (f & (d ^ e));
    const uint32_t k2 = s1 & s2;
    RowPlanes p;
    p.s = s;
    p.u0 = s1 ^ s2;
    p.u1 = c1 ^ c2 ^ k2;
    p.u2 = (c1 & c2) | (k2 & (c1 ^ c2));
    return p;
}

template <int D>
__device__ __forceinline__ uint32_t class_mask(const RowPlanes &p, int cls)
{
    constexpr uint32_t V = ((1u << D) - 1u) << 1;
    const int sig = cls >= 7, u = cls - 7 * sig;
    uint32_t m = V & (sig ? p.s : ~p.s);
    m &= (u & 1) ? p.u0 : ~p.u0;
    m &= (u & 2) ? p.u1 : ~p.u1;
    m &= (u & 4) ? p.u2 : ~p.u2;
    return m;
}

inline int to_status(cudaError_t e)
{
    return e == cudaSuccess ? SPKMC_OK : SPKMC_ECUDA;
}

inline int simple_grid(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535LL * 16) b = 65535LL * 16;
    return (int)b;
}

} // namespace

} // namespace spkmc
