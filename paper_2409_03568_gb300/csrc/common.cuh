// common.cuh -- device-side building blocks of libichee: word-size modular arithmetic on
// residues below 2^61 (RNS limbs of the CKKS modulus Q, Sec. 2.2), Philox4x32-10 and the
// samplers of Sec. 2.2.1 / 2.2.2, and the launch-argument structures shared by the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ichee {

typedef uint64_t u64;
typedef uint32_t u32;
typedef int64_t i64;

constexpr int kMaxPrimes = 8;          // ciphertext limbs
constexpr int kMaxModuli = kMaxPrimes + 1;  // plus the special prime P
constexpr int kMaxGaussBound = 31;

// --------------------------------------------------------------------------------------
// Modular arithmetic. Every modulus q is prime with q < 2^61, so 4q < 2^63 and the lazy
// ranges [0, 2q) and [0, 4q) of the NTT butterflies never overflow 64 bits.
// --------------------------------------------------------------------------------------

__device__ __forceinline__ u64 mulhi(u64 a, u64 b) { return __umul64hi(a, b); }

// Shoup product with a fixed multiplicand w < q and its companion wp = floor(w * 2^64 / q):
// returns x*w mod q in [0, 2q) for any 64-bit x.
__device__ __forceinline__ u64 shoup_lazy(u64 x, u64 w, u64 wp, u64 q)
{
    u64 hi = mulhi(x, wp);
    return x * w - hi * q;
}

__device__ __forceinline__ u64 shoup(u64 x, u64 w, u64 wp, u64 q)
{
    u64 r = shoup_lazy(x, w, wp, q);
    return r >= q ? r - q : r;
}

__device__ __forceinline__ u64 csub(u64 x, u64 q) { return x >= q ? x - q : x; }

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) { return csub(a + b, q); }

__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

// Barrett reduction of any 64-bit x with mu = floor(2^64 / q).
__device__ __forceinline__ u64 reduce64(u64 x, u64 q, u64 mu)
{
    u64 r = x - mulhi(x, mu) * q;
    return csub(r, q);
}

// Full product a*b mod q for a, b < q (Barrett on the 128-bit product with the 2-word
// constant m = floor(2^128 / q), m = m1*2^64 + m0).
__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, u64 q, u64 m0, u64 m1)
{
    u64 lo = a * b;
    u64 hi = mulhi(a, b);
    // x = hi*2^64 + lo. Estimate floor(x*m / 2^128) from the partial products that reach
    // the 2^64 and 2^128 places, dropping lo*m0 / 2^128 (< 1).
    u64 p1 = lo * m1, p1h = mulhi(lo, m1);
    u64 p2 = hi * m0, p2h = mulhi(hi, m0);
    u64 mid = p1 + p2;
    u64 carry = (mid < p1) ? 1 : 0;
    u64 qhat = hi * m1 + p1h + p2h + carry;
    // qhat >= floor(x/q) - 3, so x - qhat*q is in [0, 4q) and fits 64 bits (4q < 2^63)
    u64 r = lo - qhat * q;
    r = csub(r, 2 * q);
    r = csub(r, q);
    return r;
}

// Montgomery product a*b*2^{-64} mod q for a, b < q < 2^62, q odd, qinv = -q^{-1} mod 2^64
// (Montgomery, Math. Comp. 44, 1985): with m = (ab mod 2^64) * qinv mod 2^64, ab + mq is a
// multiple of 2^64 and (ab + mq) / 2^64 < 2q. The low words of ab and mq sum to 0 or 2^64, so
// the carry into the high word is (ab mod 2^64 != 0). Callers fold the factor 2^64 into a
// constant applied later.
__device__ __forceinline__ u64 mont_mul(u64 a, u64 b, u64 q, u64 qinv)
{
    const u64 lo = a * b;
    const u64 m = lo * qinv;
    const u64 t = mulhi(a, b) + mulhi(m, q) + (lo != 0 ? 1 : 0);
    return csub(t, q);
}

// --------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): key = per-call seed, counter =
// (block, stream, id lo, id hi). Every random draw of the library is a pure function of
// (seed, stream, ct id, coefficient), never of the launch shape.
// --------------------------------------------------------------------------------------

struct Words4 { u32 w[4]; };

__device__ __forceinline__ Words4 philox(u64 seed, u32 stream, u64 id, u32 block)
{
    u32 c0 = block, c1 = stream, c2 = (u32)id, c3 = (u32)(id >> 32);
    u32 k0 = (u32)seed, k1 = (u32)(seed >> 32);
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        u32 hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        u32 hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        u32 n0 = hi1 ^ c1 ^ k0;
        u32 n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    Words4 r;
    r.w[0] = c0; r.w[1] = c1; r.w[2] = c2; r.w[3] = c3;
    return r;
}

// Streams (which draw of a ciphertext a Philox block belongs to).
enum Stream : u32 {
    kStreamV = 0, kStreamE0 = 1, kStreamE1 = 2, kStreamRadixBits = 3, kStreamPool = 4,
    kStreamKeyS = 8, kStreamKeyE = 9, kStreamKeyA = 16
};

// Uniform ternary from one 32-bit word: floor(3w / 2^32) - 1.
__device__ __forceinline__ int ternary_of(u32 w) { return (int)(((u64)w * 3u) >> 32) - 1; }

// Discrete Gaussian from one 64-bit value: top bit sign, magnitude = number of table
// entries the low 63 bits reach (table strictly increasing, last entry 2^63).
struct CdtTable { u64 t[kMaxGaussBound + 1]; u32 bound; };

__device__ __forceinline__ int gauss_of(u64 u, const CdtTable& cdt)
{
    u64 r = u & 0x7FFFFFFFFFFFFFFFull;
    int mag = 0;
    for (u32 k = 0; k < cdt.bound; ++k) mag += (r >= cdt.t[k]) ? 1 : 0;
    return (u >> 63) ? -mag : mag;
}

// The same magnitude by a branch-free binary search: t holds the table's first kCdtSearch
// entries, those from `bound` on replaced by 2^63 (which no 63-bit value reaches), in memory
// that lanes may index independently (shared memory). Five probes count the entries the value
// reaches instead of one comparison per entry.
constexpr int kCdtSearch = 31;
static_assert(kMaxGaussBound <= kCdtSearch, "a 31-entry search covers every table");

__device__ __forceinline__ int gauss_of_sorted(u64 u, const u64* t)
{
    const u64 r = u & 0x7FFFFFFFFFFFFFFFull;
    int pos = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) pos += r >= t[pos + s - 1] ? s : 0;
    return (u >> 63) ? -pos : pos;
}

// Fill the search copy of the table (every thread of the block calls it).
__device__ __forceinline__ void cdt_for_search(const CdtTable& cdt, u64* t)
{
    for (int k = threadIdx.x; k < kCdtSearch; k += blockDim.x) t[k] = k < (int)cdt.bound ? cdt.t[k] : (1ull << 63);
}

// Residue of a small signed integer.
__device__ __forceinline__ u64 small_mod(int x, u64 q) { return x < 0 ? q - (u64)(-x) : (u64)x; }

// --------------------------------------------------------------------------------------
// Per-modulus constants and tables as the kernels see them.
// --------------------------------------------------------------------------------------

struct ModTables {
    const ulonglong2* tw;   // [N] (psi^{bitrev(k)}, Shoup companion): forward twiddles, bit-reversed order
    const ulonglong2* itw;  // [N] (psi^{-bitrev(k)}, Shoup companion): inverse twiddles
};

struct RnsArgs {
    int logn;
    int n_mod;                  // moduli described below
    u64 q[kMaxModuli];
    u64 mu[kMaxModuli];         // floor(2^64 / q)
    u64 m0[kMaxModuli], m1[kMaxModuli];  // floor(2^128 / q) as two words
    u64 qinv[kMaxModuli];       // -q^{-1} mod 2^64 (Montgomery)
    ModTables tab[kMaxModuli];
};

}  // namespace ichee
