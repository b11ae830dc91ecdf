// host_math.h -- host-side number theory for libichee's set-up: prime chain, roots of unity,
// twiddle tables with Shoup companions, the discrete-Gaussian table and CRT constants.
// Written for the CUDA library only (the CPU oracle has its own, separate code).
#pragma once
#include <cmath>
#include <cstdint>
#include <vector>

namespace ichee {
namespace host {

typedef unsigned __int128 u128;
typedef uint64_t u64;

inline u64 mulm(u64 a, u64 b, u64 m) { return (u64)((u128)a * b % m); }

inline u64 powm(u64 base, u64 exp, u64 m)
{
    u64 acc = 1 % m, b = base % m;
    for (; exp; exp >>= 1, b = mulm(b, b, m))
        if (exp & 1) acc = mulm(acc, b, m);
    return acc;
}

inline u64 invm(u64 a, u64 p) { return powm(a, p - 2, p); }  // p prime

// Strong-probable-prime test to the first twelve prime bases (exact below 2^64).
inline bool is_prime64(u64 n)
{
    if (n < 2) return false;
    const u64 small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (u64 p : small)
        if (n % p == 0) return n == p;
    u64 odd = n - 1;
    unsigned twos = 0;
    while (!(odd & 1)) { odd >>= 1; ++twos; }
    for (u64 a : small) {
        u64 x = powm(a, odd, n);
        bool witness = (x != 1 && x != n - 1);
        for (unsigned r = 1; witness && r < twos; ++r) {
            x = mulm(x, x, n);
            if (x == n - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

// Largest prime below 2^bits, congruent to 1 mod 2N, not in `taken`; 0 if none.
inline u64 chain_prime(unsigned bits, unsigned logn, const std::vector<u64>& taken)
{
    const u64 step = 2ull << logn;
    const u64 limit = 1ull << bits;
    u64 c = (limit - 1) - ((limit - 1) % step) + 1;
    if (c >= limit) c -= step;
    for (; c > (limit >> 1); c -= step) {
        bool used = false;
        for (u64 t : taken) used = used || (t == c);
        if (!used && is_prime64(c)) return c;
        if (c <= step) break;
    }
    return 0;
}

// A primitive 2N-th root of unity: psi = g^((q-1)/2N) for the first odd g >= 3 with
// psi^N = -1 (any such root gives the same negacyclic products).
inline u64 root_2n(u64 q, unsigned logn)
{
    const u64 n = 1ull << logn;
    for (u64 g = 3;; g += 2) {
        u64 psi = powm(g, (q - 1) / (2 * n), q);
        if (powm(psi, n, q) == q - 1) return psi;
    }
}

inline u64 shoup_of(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

inline unsigned bitrev(unsigned x, unsigned bits)
{
    unsigned r = 0;
    for (unsigned i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

// tw[k] = psi^{bitrev(k)}, itw[k] = psi^{-bitrev(k)} with Shoup companions, laid out as
// [tw | twp | itw | itwp], N words each.
inline std::vector<u64> twiddles(u64 q, unsigned logn)
{
    const unsigned n = 1u << logn;
    const u64 psi = root_2n(q, logn), psi_inv = invm(psi, q);
    std::vector<u64> pw(n), ipw(n);
    pw[0] = ipw[0] = 1;
    for (unsigned i = 1; i < n; ++i) { pw[i] = mulm(pw[i - 1], psi, q); ipw[i] = mulm(ipw[i - 1], psi_inv, q); }
    std::vector<u64> t(4 * (size_t)n);
    for (unsigned k = 0; k < n; ++k) {
        const unsigned e = bitrev(k, logn);
        t[k] = pw[e];
        t[n + k] = shoup_of(pw[e], q);
        t[2 * n + k] = ipw[e];
        t[3 * n + k] = shoup_of(ipw[e], q);
    }
    return t;
}

// Cumulative table of the folded discrete Gaussian on [0, bound]: weight 1 at 0 and
// 2 exp(-k^2 / (2 sigma^2)) beyond; entry k = floor(2^63 * CDF(k)) for k < bound, the last
// entry 2^63. Long double, partial sums in increasing k.
inline void gauss_cdt(double sigma, unsigned bound, u64* out)
{
    const long double denom = 2.0L * (long double)sigma * (long double)sigma;
    long double total = 1.0L;
    for (unsigned k = 1; k <= bound; ++k) total += 2.0L * expl(-(long double)((u64)k * k) / denom);
    long double run = 1.0L;
    for (unsigned k = 0; k < bound; ++k) {
        if (k > 0) run += 2.0L * expl(-(long double)((u64)k * k) / denom);
        out[k] = (u64)floorl(ldexpl(run / total, 63));
    }
    out[bound] = 1ull << 63;
}

// Residue of a signed 64-bit integer.
inline u64 signed_mod(int64_t v, u64 q)
{
    if (v >= 0) return (u64)v % q;
    const u64 mag = (u64)(-(v + 1)) + 1;  // |v| without overflow
    const u64 r = mag % q;
    return r == 0 ? 0 : q - r;
}

// Low three words of a * b for a 3-word a.
inline void mul3(const u64 a[3], u64 b, u64 out[3])
{
    u128 c = 0;
    for (int i = 0; i < 3; ++i) {
        c += (u128)a[i] * b;
        out[i] = (u64)c;
        c >>= 64;
    }
}

}  // namespace host
}  // namespace ichee
