/*
 * ckks_oracle.c -- plain CPU oracle for pixel-level CKKS with cached encryption
 * (Wang, Yang, Sun, Dai, Zhao, "Enabling Practical and Privacy-Preserving Image
 * Processing", arXiv 2409.03568; the method is called iCHEETAH there).
 *
 * TEST INFRASTRUCTURE. This file is the checker, not the product: only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline / reference leg may load it.
 * It shares no code, header, table or constant generator with the CUDA library.
 *
 * Style: scalar C, one residue at a time, 128-bit products reduced with the C `%`
 * operator, textbook algorithms in the order the paper states them.  Nothing is
 * blocked, fused or reordered for speed; the only parallelism is an OpenMP loop
 * over independent pixels (the paper's pixel-level encryption is per pixel, Sec. 3.1).
 *
 * Pins (tests/test_oracle_*.py) tie every function here to something other than
 * itself: schoolbook products, big-integer (non-RNS) CKKS, published Philox
 * known-answer vectors, closed-form noise bounds, the paper's worked radix example
 * (Sec. 3.3) and its MSE/PSNR table (Sec. 4.3.2).
 *
 * Where the paper is silent this file fixes one reading and states it next to the code:
 * the key / encryption sign convention, the constant-polynomial pixel encoding, the prime
 * chain (largest primes = 1 mod 2N below each bit size), Philox4x32-10 with counters
 * (block, stream, ciphertext id), the CDT Gaussian and ternary samplers, the signed-digit
 * form of the radix randomness, the pool index rule, centered rounding in rescale and
 * hybrid key switching with one special prime.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef uint64_t u64;
typedef uint32_t u32;
typedef int64_t i64;
typedef unsigned __int128 u128;
typedef __int128 i128;

#define ORC_MAX_LIMBS 16

/* ------------------------------------------------------------------------- */
/* Integer arithmetic modulo a word-size prime (Sec. 2.2: ring Z_Q[X]/(X^N+1),   */
/* Q a product of primes; every residue below is kept in [0, q)).              */
/* ------------------------------------------------------------------------- */

static u64 mod_add(u64 a, u64 b, u64 q) { u128 s = (u128)a + b; return (u64)(s % q); }
static u64 mod_sub(u64 a, u64 b, u64 q) { return a >= b ? a - b : (u64)(((u128)a + q) - b); }
static u64 mod_mul(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 mod_neg(u64 a, u64 q) { return a == 0 ? 0 : q - a; }
static u64 mod_pow(u64 b, u64 e, u64 q)
{
    u64 r = 1 % q;
    b %= q;
    while (e) {
        if (e & 1) r = mod_mul(r, b, q);
        b = mod_mul(b, b, q);
        e >>= 1;
    }
    return r;
}
static u64 mod_inv(u64 a, u64 q) { return mod_pow(a, q - 2, q); } /* q prime */
/* Residue of a signed integer. */
static u64 from_signed(i64 x, u64 q)
{
    i128 r = (i128)x % (i128)q;
    if (r < 0) r += q;
    return (u64)r;
}
/* Centered representative of a residue: (-q/2, q/2] (q odd, so no ties). */
static i64 centered(u64 a, u64 q) { return a > (q - 1) / 2 ? (i64)a - (i64)q : (i64)a; }

/* Deterministic Miller-Rabin for 64-bit n (the first 12 primes as bases suffice). */
int orc_is_prime(u64 n)
{
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    u64 d = n - 1;
    int r = 0;
    while ((d & 1) == 0) { d >>= 1; r++; }
    for (int i = 0; i < 12; i++) {
        u64 x = mod_pow(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int k = 1; k < r; k++) {
            x = mod_mul(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/*
 * Prime chain (Sec. 2.2 parameter table: N, Q, L; Sec. 4.2 uses one modulus Q
 * split into word-size primes).  For each requested bit size b, in order, take
 * the largest prime q < 2^b with q = 1 mod 2N that is not already taken.  The
 * special prime P (evaluation keys only) is chosen the same way from special_bits.
 * Returns 0 on success, -1 if a search runs out of candidates.
 */
int orc_gen_primes(u32 log_n, u32 n_primes, const u32 *bits, u32 special_bits,
                   u64 *q_out, u64 *p_out)
{
    u64 two_n = 2ull << log_n;
    u64 used[ORC_MAX_LIMBS + 1];
    int n_used = 0;
    for (u32 i = 0; i <= n_primes; i++) {
        u32 b = (i < n_primes) ? bits[i] : special_bits;
        if (i == n_primes && special_bits == 0) { *p_out = 0; break; }
        if (b < 2 || b > 62) return -1;
        u64 top = 1ull << b;
        u64 cand = ((top - 1) / two_n) * two_n + 1; /* largest 1 mod 2N below 2^b */
        if (cand >= top) cand -= two_n;
        u64 found = 0;
        while (cand > (top >> 1)) {
            int taken = 0;
            for (int k = 0; k < n_used; k++) taken |= (used[k] == cand);
            if (!taken && orc_is_prime(cand)) { found = cand; break; }
            if (cand < two_n) break;
            cand -= two_n;
        }
        if (!found) return -1;
        used[n_used++] = found;
        if (i < n_primes) q_out[i] = found; else *p_out = found;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Random source: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random   */
/* numbers: as easy as 1, 2, 3", SC'11).  The paper only says "random",         */
/* "discrete Gaussian" and "ternary" (Sec. 2.2.1, 2.2.2, 4.2); the counter      */
/* layout is a reading: key = seed, counter = (block, stream, id lo, id hi).    */
/* ------------------------------------------------------------------------- */

void orc_philox4x32_10(const u32 ctr_in[4], const u32 key_in[2], u32 out[4])
{
    u32 c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    u32 k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        u64 p0 = (u64)0xD2511F53u * c0;
        u64 p1 = (u64)0xCD9E8D57u * c2;
        u32 n0 = (u32)(p1 >> 32) ^ c1 ^ k0;
        u32 n1 = (u32)p1;
        u32 n2 = (u32)(p0 >> 32) ^ c3 ^ k1;
        u32 n3 = (u32)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_block(u64 seed, u32 stream, u64 id, u32 block, u32 out[4])
{
    u32 key[2] = {(u32)seed, (u32)(seed >> 32)};
    u32 ctr[4] = {block, stream, (u32)id, (u32)(id >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/*
 * Cumulative table for the discrete Gaussian (Sec. 2.2.1: error terms "sampled
 * from a discrete Gaussian distribution").  Folded distribution on |x| in
 * [0, bound]: weight 1 at 0 and 2*exp(-k^2 / (2 sigma^2)) at k >= 1.  T[k] is
 * floor(2^63 * F(k)) for k < bound and T[bound] = 2^63, computed in long double
 * with the partial sums taken in increasing k.
 */
void orc_cdt_table(double sigma, u32 bound, u64 *T)
{
    long double two_s2 = 2.0L * (long double)sigma * (long double)sigma;
    long double z = 1.0L;
    for (u32 k = 1; k <= bound; k++) z += 2.0L * expl(-(long double)((u64)k * k) / two_s2);
    long double acc = 1.0L;
    for (u32 k = 0; k < bound; k++) {
        if (k > 0) acc += 2.0L * expl(-(long double)((u64)k * k) / two_s2);
        T[k] = (u64)floorl(ldexpl(acc / z, 63));
    }
    T[bound] = 1ull << 63;
}

/* Uniform ternary {-1, 0, 1} (Sec. 4.2: s in {-1,0,1}^N; the encryption randomness
 * r of Sec. 2.2.2 is drawn the same way).  Coefficient i uses word i%4 of block i/4. */
void orc_sample_ternary(u64 seed, u32 stream, u64 id, u32 n, int8_t *out)
{
    for (u32 i = 0; i < n; i++) {
        u32 w[4];
        philox_block(seed, stream, id, i >> 2, w);
        u32 t = (u32)(((u64)w[i & 3] * 3u) >> 32);
        out[i] = (int8_t)((int)t - 1);
    }
}

/* Discrete Gaussian via the table above.  Coefficient i uses words 2(i%2) and
 * 2(i%2)+1 of block i/2 as one 64-bit value: top bit = sign, low 63 bits searched
 * in the table for the smallest k with value < T[k]. */
void orc_sample_gauss(u64 seed, u32 stream, u64 id, u32 n, const u64 *T, u32 bound, int8_t *out)
{
    for (u32 i = 0; i < n; i++) {
        u32 w[4];
        philox_block(seed, stream, id, i >> 1, w);
        u32 h = 2 * (i & 1);
        u64 u = (u64)w[h] | ((u64)w[h + 1] << 32);
        u64 r = u & ((1ull << 63) - 1);
        u32 mag = 0;
        while (mag < bound && r >= T[mag]) mag++;
        out[i] = (int8_t)((u >> 63) ? -(int)mag : (int)mag);
    }
}

/* Uniform residue mod q (Sec. 2.2.1: a uniformly random in R_q): the four words of
 * block i form a 128-bit x, and the residue is floor(x * q / 2^128). */
void orc_sample_uniform(u64 seed, u32 stream, u64 id, u32 n, u64 q, u64 *out)
{
    for (u32 i = 0; i < n; i++) {
        u32 w[4];
        philox_block(seed, stream, id, i, w);
        u64 lo = (u64)w[0] | ((u64)w[1] << 32);
        u64 hi = (u64)w[2] | ((u64)w[3] << 32);
        u128 carry = ((u128)lo * q) >> 64;
        u128 top = (u128)hi * q + carry;
        out[i] = (u64)(top >> 64);
    }
}

/* ------------------------------------------------------------------------- */
/* Negacyclic products in Z_q[X]/(X^N + 1) (Sec. 2.2).                          */
/* ------------------------------------------------------------------------- */

/* The definition: c_k = sum_{i+j=k} a_i b_j - sum_{i+j=k+N} a_i b_j. */
void orc_polymul_schoolbook(u32 n, u64 q, const u64 *a, const u64 *b, u64 *c)
{
    for (u32 k = 0; k < n; k++) {
        u64 acc = 0;
        for (u32 i = 0; i < n; i++) {
            if (i <= k) acc = mod_add(acc, mod_mul(a[i], b[k - i], q), q);
            else acc = mod_sub(acc, mod_mul(a[i], b[k + n - i], q), q);
        }
        c[k] = acc;
    }
}

/* A primitive 2N-th root of unity psi (psi^N = -1): psi = x^((q-1)/2N) for the
 * smallest x >= 2 that gives one. */
static u64 find_psi(u32 n, u64 q)
{
    for (u64 x = 2;; x++) {
        u64 psi = mod_pow(x, (q - 1) / (2ull * n), q);
        if (mod_pow(psi, n, q) == q - 1) return psi;
    }
}

/* Textbook iterative radix-2 cyclic transform of size n with root w (bit-reversal
 * permutation first, then log2(n) butterfly levels). */
static void dft_cyclic(u32 n, u64 q, u64 w, u64 *x)
{
    for (u32 i = 1, j = 0; i < n; i++) {
        u32 bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { u64 t = x[i]; x[i] = x[j]; x[j] = t; }
    }
    for (u32 len = 2; len <= n; len <<= 1) {
        u64 wl = mod_pow(w, n / len, q);
        for (u32 i = 0; i < n; i += len) {
            u64 wk = 1;
            for (u32 j = 0; j < len / 2; j++) {
                u64 u = x[i + j];
                u64 v = mod_mul(x[i + j + len / 2], wk, q);
                x[i + j] = mod_add(u, v, q);
                x[i + j + len / 2] = mod_sub(u, v, q);
                wk = mod_mul(wk, wl, q);
            }
        }
    }
}

/* Negacyclic product through the transform: twist by psi^i, cyclic transform with
 * omega = psi^2, pointwise product, inverse transform, scale by 1/N, untwist.
 * Pinned against orc_polymul_schoolbook for every prime at small N. */
void orc_polymul(u32 n, u64 q, const u64 *a, const u64 *b, u64 *c)
{
    u64 psi = find_psi(n, q);
    u64 psi_inv = mod_inv(psi, q);
    u64 omega = mod_mul(psi, psi, q);
    u64 omega_inv = mod_inv(omega, q);
    u64 n_inv = mod_inv(n % q, q);
    u64 *A = (u64 *)malloc(sizeof(u64) * n);
    u64 *B = (u64 *)malloc(sizeof(u64) * n);
    u64 pw = 1;
    for (u32 i = 0; i < n; i++) {
        A[i] = mod_mul(a[i] % q, pw, q);
        B[i] = mod_mul(b[i] % q, pw, q);
        pw = mod_mul(pw, psi, q);
    }
    dft_cyclic(n, q, omega, A);
    dft_cyclic(n, q, omega, B);
    for (u32 i = 0; i < n; i++) A[i] = mod_mul(A[i], B[i], q);
    dft_cyclic(n, q, omega_inv, A);
    pw = n_inv;
    for (u32 i = 0; i < n; i++) {
        c[i] = mod_mul(A[i], pw, q);
        pw = mod_mul(pw, psi_inv, q);
    }
    free(A);
    free(B);
}

/* Small signed polynomial (ternary or Gaussian) as residues mod q. */
static void small_to_residues(u32 n, const int8_t *x, u64 q, u64 *out)
{
    for (u32 i = 0; i < n; i++) out[i] = from_signed(x[i], q);
}

/* ------------------------------------------------------------------------- */
/* CKKS (Sec. 2.2.2, with the sign convention of the paper's library: the      */
/* printed KeyGen / Enc / Dec do not cancel as written -- r*a*(1 - s^2) stays). */
/*   pk = (pk0, pk1) = (-a*s + e, a)                                           */
/*   Enc(m) = (v*pk0 + e0 + m, v*pk1 + e1),  Dec(c) = c0 + c1*s                 */
/* Layouts: polynomial [n]; ciphertext [2][limbs][n] (coefficient domain).      */
/* ------------------------------------------------------------------------- */

enum { ST_V = 0, ST_E0 = 1, ST_E1 = 2, ST_RADIX_BITS = 3, ST_POOL = 4,
       ST_KEY_S = 8, ST_KEY_E = 9, ST_KEY_A = 16 };

/* KeyGen, Sec. 2.2.2 steps 1-2: s ternary; a uniform; e Gaussian; pk as above. */
int orc_keygen(u32 n, u32 L, const u64 *q, u64 seed, const u64 *T, u32 bound,
               int8_t *s_out, u64 *pk_out)
{
    int8_t *e = (int8_t *)malloc(n);
    u64 *a = (u64 *)malloc(sizeof(u64) * n);
    u64 *s = (u64 *)malloc(sizeof(u64) * n);
    u64 *as = (u64 *)malloc(sizeof(u64) * n);
    orc_sample_ternary(seed, ST_KEY_S, 0, n, s_out);
    orc_sample_gauss(seed, ST_KEY_E, 0, n, T, bound, e);
    for (u32 l = 0; l < L; l++) {
        orc_sample_uniform(seed, ST_KEY_A + l, 0, n, q[l], a);
        small_to_residues(n, s_out, q[l], s);
        orc_polymul(n, q[l], a, s, as);
        u64 *pk0 = pk_out + (size_t)(0 * L + l) * n;
        u64 *pk1 = pk_out + (size_t)(1 * L + l) * n;
        for (u32 i = 0; i < n; i++) {
            pk0[i] = mod_add(mod_neg(as[i], q[l]), from_signed(e[i], q[l]), q[l]);
            pk1[i] = a[i];
        }
    }
    free(e); free(a); free(s); free(as);
    return 0;
}

/*
 * Evaluation key for relinearisation (Sec. 2.2.3: Relin(ct, evk); Sec. 2.2.2
 * step 3).  The paper gives no construction; this oracle uses hybrid RNS key
 * switching with one special prime P and one digit per ciphertext prime.
 * Moduli m_0..m_{L-1} = q_0..q_{L-1}, m_L = P.  Digit j (ct id 1+j):
 *   evk_j = (-a_j*s + e_j + P*g_j*s^2, a_j) over Q*P,
 * where g_j = 1 mod q_j and 0 mod every other modulus.
 * Layout: evk[j][2][L+1][n].
 */
int orc_keygen_evk(u32 n, u32 L, const u64 *q, u64 P, u64 seed, const u64 *T, u32 bound,
                   const int8_t *s_small, u64 *evk_out)
{
    u64 m[ORC_MAX_LIMBS + 1];
    for (u32 i = 0; i < L; i++) m[i] = q[i];
    m[L] = P;
    int8_t *e = (int8_t *)malloc(n);
    u64 *a = (u64 *)malloc(sizeof(u64) * n);
    u64 *s = (u64 *)malloc(sizeof(u64) * n);
    u64 *as = (u64 *)malloc(sizeof(u64) * n);
    u64 *s2 = (u64 *)malloc(sizeof(u64) * n);
    for (u32 j = 0; j < L; j++) {
        u64 id = 1 + j;
        orc_sample_gauss(seed, ST_KEY_E, id, n, T, bound, e);
        for (u32 i = 0; i <= L; i++) {
            orc_sample_uniform(seed, ST_KEY_A + i, id, n, m[i], a);
            small_to_residues(n, s_small, m[i], s);
            orc_polymul(n, m[i], a, s, as);
            u64 *b0 = evk_out + ((size_t)(j * 2 + 0) * (L + 1) + i) * n;
            u64 *b1 = evk_out + ((size_t)(j * 2 + 1) * (L + 1) + i) * n;
            for (u32 k = 0; k < n; k++) {
                b0[k] = mod_add(mod_neg(as[k], m[i]), from_signed(e[k], m[i]), m[i]);
                b1[k] = a[k];
            }
            if (i == j) {
                orc_polymul(n, m[i], s, s, s2);
                u64 pm = P % m[i];
                for (u32 k = 0; k < n; k++) b0[k] = mod_add(b0[k], mod_mul(pm, s2[k], m[i]), m[i]);
            }
        }
    }
    free(e); free(a); free(s); free(as); free(s2);
    return 0;
}

/*
 * Encrypt one message (Sec. 2.2.2 "To encrypt a plaintext").  The message is the
 * encoded constant polynomial msg (a pixel fills every slot, so its
 * encoding is the constant round(Delta * p)).  v from stream 0, e0 from stream 1,
 * e1 from stream 2, all keyed by (seed, id).
 */
static void encrypt_one(u32 n, u32 L, const u64 *q, const u64 *pk, u64 seed, u64 id, i64 msg,
                        const u64 *T, u32 bound, u64 *out, int8_t *v, int8_t *e0, int8_t *e1,
                        u64 *vr, u64 *prod)
{
    orc_sample_ternary(seed, ST_V, id, n, v);
    orc_sample_gauss(seed, ST_E0, id, n, T, bound, e0);
    orc_sample_gauss(seed, ST_E1, id, n, T, bound, e1);
    for (u32 l = 0; l < L; l++) {
        const u64 *pk0 = pk + (size_t)(0 * L + l) * n;
        const u64 *pk1 = pk + (size_t)(1 * L + l) * n;
        u64 *c0 = out + (size_t)(0 * L + l) * n;
        u64 *c1 = out + (size_t)(1 * L + l) * n;
        small_to_residues(n, v, q[l], vr);
        orc_polymul(n, q[l], vr, pk0, prod);
        for (u32 i = 0; i < n; i++) c0[i] = mod_add(prod[i], from_signed(e0[i], q[l]), q[l]);
        c0[0] = mod_add(c0[0], from_signed(msg, q[l]), q[l]);
        orc_polymul(n, q[l], vr, pk1, prod);
        for (u32 i = 0; i < n; i++) c1[i] = mod_add(prod[i], from_signed(e1[i], q[l]), q[l]);
    }
}

/* Pixel-level encryption (Sec. 3.1): one ciphertext per message, independent
 * across messages.  out is [count][2][L][n]. */
int orc_encrypt_batch(u32 n, u32 L, const u64 *q, const u64 *pk, u64 seed, const u64 *ids,
                      const i64 *msgs, u64 count, const u64 *T, u32 bound, u64 *out)
{
#pragma omp parallel
    {
        int8_t *v = (int8_t *)malloc(n), *e0 = (int8_t *)malloc(n), *e1 = (int8_t *)malloc(n);
        u64 *vr = (u64 *)malloc(sizeof(u64) * n), *prod = (u64 *)malloc(sizeof(u64) * n);
#pragma omp for schedule(dynamic, 1)
        for (i64 k = 0; k < (i64)count; k++)
            encrypt_one(n, L, q, pk, seed, ids[k], msgs[k], T, bound,
                        out + (size_t)k * 2 * L * n, v, e0, e1, vr, prod);
        free(v); free(e0); free(e1); free(vr); free(prod);
    }
    return 0;
}

/* Number of threads an OpenMP region of this library uses. */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Homomorphic operations (Sec. 2.2.3), elementwise on [2][limbs][n].           */
/* ------------------------------------------------------------------------- */

/* ct_add: c = a (+) b; ct_sub: c = a (-) b; both polynomials, every limb. */
void orc_ct_add(u32 n, u32 limbs, const u64 *q, const u64 *a, const u64 *b, u64 *c)
{
    for (u32 p = 0; p < 2; p++)
        for (u32 l = 0; l < limbs; l++)
            for (u32 i = 0; i < n; i++) {
                size_t k = ((size_t)p * limbs + l) * n + i;
                c[k] = mod_add(a[k], b[k], q[l]);
            }
}

void orc_ct_sub(u32 n, u32 limbs, const u64 *q, const u64 *a, const u64 *b, u64 *c)
{
    for (u32 p = 0; p < 2; p++)
        for (u32 l = 0; l < limbs; l++)
            for (u32 i = 0; i < n; i++) {
                size_t k = ((size_t)p * limbs + l) * n + i;
                c[k] = mod_sub(a[k], b[k], q[l]);
            }
}

/* Multiply every coefficient by one signed integer constant (a constant
 * plaintext, Sec. 4.4 brightness / mean filter / watermark). */
void orc_ct_mul_int(u32 n, u32 limbs, const u64 *q, const u64 *a, i64 k, u64 *c)
{
    for (u32 p = 0; p < 2; p++)
        for (u32 l = 0; l < limbs; l++) {
            u64 kr = from_signed(k, q[l]);
            for (u32 i = 0; i < n; i++) {
                size_t x = ((size_t)p * limbs + l) * n + i;
                c[x] = mod_mul(a[x], kr, q[l]);
            }
        }
}

/* Add a signed integer constant to the message: coefficient 0 of c0 only. */
void orc_ct_add_int(u32 n, u32 limbs, const u64 *q, const u64 *a, i64 k, u64 *c)
{
    if (c != a) memcpy(c, a, sizeof(u64) * 2 * limbs * n);
    for (u32 l = 0; l < limbs; l++) c[(size_t)l * n] = mod_add(c[(size_t)l * n], from_signed(k, q[l]), q[l]);
}

/* Rescale (Sec. 2.2.3): divide by the last prime q_t with rounding and drop it.
 * c'_j = (c_j - [c_t]_centered) * q_t^{-1} mod q_j, [x]_centered in (-q_t/2, q_t/2]. */
void orc_rescale(u32 n, u32 limbs, const u64 *q, const u64 *a, u64 *c)
{
    u32 t = limbs - 1;
    for (u32 p = 0; p < 2; p++) {
        const u64 *last = a + ((size_t)p * limbs + t) * n;
        for (u32 j = 0; j < t; j++) {
            u64 qt_inv = mod_inv(q[t] % q[j], q[j]);
            const u64 *src = a + ((size_t)p * limbs + j) * n;
            u64 *dst = c + ((size_t)p * t + j) * n;
            for (u32 i = 0; i < n; i++) {
                u64 r = from_signed(centered(last[i], q[t]), q[j]);
                dst[i] = mod_mul(mod_sub(src[i], r, q[j]), qt_inv, q[j]);
            }
        }
    }
}

/* Ciphertext tensor of d with itself (Sec. 2.2.3 ct (x) ct): for decryption
 * c0 + c1*s the square is (d0*d0, 2*d0*d1, d1*d1) under (1, s, s^2).
 * out is [3][limbs][n]. */
void orc_ct_square(u32 n, u32 limbs, const u64 *q, const u64 *d, u64 *out)
{
    u64 *t = (u64 *)malloc(sizeof(u64) * n);
    for (u32 l = 0; l < limbs; l++) {
        const u64 *d0 = d + (size_t)(0 * limbs + l) * n;
        const u64 *d1 = d + (size_t)(1 * limbs + l) * n;
        orc_polymul(n, q[l], d0, d0, out + (size_t)(0 * limbs + l) * n);
        orc_polymul(n, q[l], d0, d1, t);
        for (u32 i = 0; i < n; i++) out[(size_t)(1 * limbs + l) * n + i] = mod_add(t[i], t[i], q[l]);
        orc_polymul(n, q[l], d1, d1, out + (size_t)(2 * limbs + l) * n);
    }
    free(t);
}

/*
 * Relinearisation (Sec. 2.2.3: ct_rel = Relin(ct_mul, evk)) by hybrid key
 * switching with the special prime P.
 * Input (d0, d1, d2) at `limbs` limbs, [3][limbs][n]; evk as from
 * orc_keygen_evk for L_full limbs.  For each digit j < limbs the centered
 * residue [d2]_{q_j} is lifted to every modulus q_0..q_{limbs-1}, P, multiplied
 * by evk_j, summed; the sum is divided by P with rounding (ModDown) and added
 * to (d0, d1).  out is [2][limbs][n].
 */
void orc_relin(u32 n, u32 limbs, u32 L_full, const u64 *q, u64 P, const u64 *evk,
               const u64 *d, u64 *out)
{
    u32 nm = limbs + 1;               /* moduli used: q_0..q_{limbs-1}, P */
    u64 *acc = (u64 *)calloc((size_t)2 * nm * n, sizeof(u64));
    u64 *dig = (u64 *)malloc(sizeof(u64) * n);
    u64 *prod = (u64 *)malloc(sizeof(u64) * n);
    const u64 *d2 = d + (size_t)2 * limbs * n;
    for (u32 j = 0; j < limbs; j++) {
        const u64 *dj = d2 + (size_t)j * n;
        for (u32 mi = 0; mi < nm; mi++) {
            u32 ei = (mi < limbs) ? mi : L_full;          /* index into evk's moduli */
            u64 mod = (mi < limbs) ? q[mi] : P;
            for (u32 i = 0; i < n; i++) dig[i] = from_signed(centered(dj[i], q[j]), mod);
            for (u32 b = 0; b < 2; b++) {
                const u64 *key = evk + ((size_t)(j * 2 + b) * (L_full + 1) + ei) * n;
                orc_polymul(n, mod, dig, key, prod);
                u64 *ac = acc + ((size_t)b * nm + mi) * n;
                for (u32 i = 0; i < n; i++) ac[i] = mod_add(ac[i], prod[i], mod);
            }
        }
    }
    for (u32 b = 0; b < 2; b++) {
        const u64 *accP = acc + ((size_t)b * nm + limbs) * n;
        for (u32 l = 0; l < limbs; l++) {
            u64 p_inv = mod_inv(P % q[l], q[l]);
            const u64 *ac = acc + ((size_t)b * nm + l) * n;
            const u64 *src = d + ((size_t)b * limbs + l) * n;
            u64 *dst = out + ((size_t)b * limbs + l) * n;
            for (u32 i = 0; i < n; i++) {
                u64 r = from_signed(centered(accP[i], P), q[l]);
                u64 ks = mod_mul(mod_sub(ac[i], r, q[l]), p_inv, q[l]);
                dst[i] = mod_add(src[i], ks, q[l]);
            }
        }
    }
    free(acc); free(dig); free(prod);
}

/* Decryption, coefficient 0 only (Sec. 2.2.2 "To decrypt"; a constant message is
 * decoded from coefficient 0).  By the definition of the negacyclic
 * product, (c1*s)_0 = c1_0 s_0 - sum_{j=1}^{N-1} c1_j s_{N-j}.  out[l] is the
 * residue of c0 + c1*s at coefficient 0 modulo q_l. */
void orc_decrypt_coef0(u32 n, u32 limbs, const u64 *q, const int8_t *s, const u64 *ct, u64 *out)
{
    for (u32 l = 0; l < limbs; l++) {
        const u64 *c0 = ct + (size_t)(0 * limbs + l) * n;
        const u64 *c1 = ct + (size_t)(1 * limbs + l) * n;
        u64 acc = mod_add(c0[0], mod_mul(c1[0], from_signed(s[0], q[l]), q[l]), q[l]);
        for (u32 j = 1; j < n; j++)
            acc = mod_sub(acc, mod_mul(c1[j], from_signed(s[n - j], q[l]), q[l]), q[l]);
        out[l] = acc;
    }
}

/* Full decryption polynomial c0 + c1*s (all coefficients), for noise checks. */
void orc_decrypt_poly(u32 n, u32 limbs, const u64 *q, const int8_t *s, const u64 *ct, u64 *out)
{
    u64 *sr = (u64 *)malloc(sizeof(u64) * n);
    u64 *prod = (u64 *)malloc(sizeof(u64) * n);
    for (u32 l = 0; l < limbs; l++) {
        small_to_residues(n, s, q[l], sr);
        orc_polymul(n, q[l], ct + (size_t)(1 * limbs + l) * n, sr, prod);
        for (u32 i = 0; i < n; i++)
            out[(size_t)l * n + i] = mod_add(ct[(size_t)(0 * limbs + l) * n + i], prod[i], q[l]);
    }
    free(sr); free(prod);
}

/* ------------------------------------------------------------------------- */
/* Cached encryption (Sec. 3.2) and randomness (Sec. 3.3).                      */
/* ------------------------------------------------------------------------- */

/* Radix randomness word of pixel `id` (stream 3, block 0, word 0): bit i says
 * whether step i of Sec. 3.3 is applied. */
u32 orc_radix_bits(u64 seed, u64 id)
{
    u32 w[4];
    philox_block(seed, ST_RADIX_BITS, id, 0, w);
    return w[0];
}

/* Pool index of pixel `id` (stream 4, block 0, word 0): floor(w * M / 2^32). */
u32 orc_pool_index(u64 seed, u64 id, u32 pool_size)
{
    u32 w[4];
    philox_block(seed, ST_POOL, id, 0, w);
    return (u32)(((u64)w[0] * pool_size) >> 32);
}

/*
 * Radix-based encryption of one pixel p, step by step as Sec. 3.2 and 3.3 state:
 *   c_p = sum over base-r digits d_k of d_k repeated homomorphic additions of
 *         radixes[k] = Enc(r^k);
 *   then for i = 1..n_pow-1, if bit i of the randomness word is set:
 *         Ctxt (+) radixes[i], then (-) radixes[i-1] r times.
 * radix_cts is [n_pow][2][limbs][n]; out is [2][limbs][n].
 */
void orc_radix_encrypt_sequential(u32 n, u32 limbs, const u64 *q, const u64 *radix_cts, u32 n_pow,
                                  u32 r, u32 p, int randomize, u32 bits, u64 *out)
{
    size_t ct_len = (size_t)2 * limbs * n;
    memset(out, 0, sizeof(u64) * ct_len);
    u32 rest = p;
    for (u32 k = 0; k < n_pow; k++) {
        u32 dk = rest % r;
        rest /= r;
        for (u32 t = 0; t < dk; t++) orc_ct_add(n, limbs, q, out, radix_cts + k * ct_len, out);
    }
    if (!randomize) return;
    for (u32 i = 1; i < n_pow; i++) {
        if (!((bits >> i) & 1u)) continue;
        orc_ct_add(n, limbs, q, out, radix_cts + i * ct_len, out);
        for (u32 t = 0; t < r; t++) orc_ct_sub(n, limbs, q, out, radix_cts + (i - 1) * ct_len, out);
    }
}

/* The same result written with signed digits d'_k = d_k + b_k - r*b_{k+1}
 * (b_0 = b_{n_pow} = 0) and one scalar multiply per cached ciphertext.  Kept in
 * the oracle only to pin the equivalence (tests compare it bit for bit with the
 * sequential form above). */
void orc_radix_encrypt_signed(u32 n, u32 limbs, const u64 *q, const u64 *radix_cts, u32 n_pow,
                              u32 r, u32 p, int randomize, u32 bits, u64 *out)
{
    size_t ct_len = (size_t)2 * limbs * n;
    u64 *tmp = (u64 *)malloc(sizeof(u64) * ct_len);
    memset(out, 0, sizeof(u64) * ct_len);
    u32 rest = p;
    for (u32 k = 0; k < n_pow; k++) {
        i64 dk = rest % r;
        rest /= r;
        i64 bk = (randomize && k >= 1) ? ((bits >> k) & 1u) : 0;
        i64 bk1 = (randomize && k + 1 < n_pow) ? ((bits >> (k + 1)) & 1u) : 0;
        i64 d = dk + bk - (i64)r * bk1;
        orc_ct_mul_int(n, limbs, q, radix_cts + k * ct_len, d, tmp);
        orc_ct_add(n, limbs, q, out, tmp, out);
    }
    free(tmp);
}

/*
 * Radix-cached encryption of a batch of pixels (Sec. 3.2 + 3.3), pixel ids
 * `ids`, randomness keyed by `seed`.  out is [count][2][limbs][n].
 */
int orc_radix_encrypt_batch(u32 n, u32 limbs, const u64 *q, const u64 *radix_cts, u32 n_pow, u32 r,
                            const uint8_t *pixels, const u64 *ids, u64 count, u64 seed, int randomize,
                            u64 *out)
{
    size_t ct_len = (size_t)2 * limbs * n;
#pragma omp parallel for schedule(dynamic, 4)
    for (i64 k = 0; k < (i64)count; k++) {
        u32 bits = randomize ? orc_radix_bits(seed, ids[k]) : 0;
        orc_radix_encrypt_sequential(n, limbs, q, radix_cts, n_pow, r, pixels[k], randomize, bits,
                                     out + (size_t)k * ct_len);
    }
    return 0;
}

/*
 * Scanning-based / full caching with the randomness pool (Sec. 3.2, 3.3):
 * c_final = c_p (+) c_z[idx].  lut[p] is the cache slot of value p or -1; a
 * pixel whose lut entry is -1 is skipped here (the caller encrypts it another
 * way) and its output left untouched.  pool_size 0 disables the pool.
 */
int orc_lookup_encrypt_batch(u32 n, u32 limbs, const u64 *q, const u64 *value_cts, const int32_t *lut,
                             const u64 *pool_cts, u32 pool_size, const uint8_t *pixels, const u64 *ids,
                             u64 count, u64 seed, u64 *out)
{
    size_t ct_len = (size_t)2 * limbs * n;
#pragma omp parallel for schedule(dynamic, 16)
    for (i64 k = 0; k < (i64)count; k++) {
        int32_t slot = lut[pixels[k]];
        if (slot < 0) continue;
        u64 *dst = out + (size_t)k * ct_len;
        const u64 *src = value_cts + (size_t)slot * ct_len;
        if (pool_size == 0) {
            memcpy(dst, src, sizeof(u64) * ct_len);
        } else {
            u32 z = orc_pool_index(seed, ids[k], pool_size);
            orc_ct_add(n, limbs, q, src, pool_cts + (size_t)z * ct_len, dst);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Image operations (Sec. 4.4) on an image of ciphertexts [h*w*c][2][limbs][n], */
/* pixel (y, x, ch) at index (y*w + x)*c + ch.                                  */
/* ------------------------------------------------------------------------- */

/* 3x3 mean filter (Sec. 4.4.1 formula with n = 3): sum of the 9 neighbours with
 * clamp-to-edge borders (the paper does not say how borders are treated), times the integer constant k9 (the
 * encoded 1/9), then rescale.  Output has limbs-1 limbs. */
int orc_meanfilter3(u32 n, u32 limbs, const u64 *q, const u64 *in, u32 h, u32 w, u32 ch,
                    i64 k9, u64 *out)
{
    size_t ct_len = (size_t)2 * limbs * n;
    size_t out_len = (size_t)2 * (limbs - 1) * n;
#pragma omp parallel
    {
        u64 *sum = (u64 *)malloc(sizeof(u64) * ct_len);
        u64 *prod = (u64 *)malloc(sizeof(u64) * ct_len);
#pragma omp for schedule(dynamic, 1)
        for (i64 pix = 0; pix < (i64)h * w; pix++) {
            i64 y = pix / w, x = pix % w;
            for (u32 c = 0; c < ch; c++) {
                memset(sum, 0, sizeof(u64) * ct_len);
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        i64 yy = y + dy, xx = x + dx;
                        if (yy < 0) yy = 0;
                        if (yy >= (i64)h) yy = h - 1;
                        if (xx < 0) xx = 0;
                        if (xx >= (i64)w) xx = w - 1;
                        orc_ct_add(n, limbs, q, sum, in + ((size_t)(yy * w + xx) * ch + c) * ct_len, sum);
                    }
                orc_ct_mul_int(n, limbs, q, sum, k9, prod);
                orc_rescale(n, limbs, q, prod, out + ((size_t)pix * ch + c) * out_len);
            }
        }
        free(sum); free(prod);
    }
    return 0;
}

/* Watermark blend alpha*I + (1-alpha)*W with W an encrypted pattern: both scaled by their
 * encoded integer constants, added, rescaled.  wm has c_w channels (1 or c). */
int orc_blend(u32 n, u32 limbs, const u64 *q, const u64 *img, const u64 *wm, u64 count, u32 ch,
              u32 ch_w, i64 ka, i64 kb, u64 *out)
{
    size_t ct_len = (size_t)2 * limbs * n;
    size_t out_len = (size_t)2 * (limbs - 1) * n;
#pragma omp parallel
    {
        u64 *t1 = (u64 *)malloc(sizeof(u64) * ct_len);
        u64 *t2 = (u64 *)malloc(sizeof(u64) * ct_len);
#pragma omp for schedule(dynamic, 4)
        for (i64 k = 0; k < (i64)count; k++) {
            u64 pix = (u64)k / ch, c = (u64)k % ch;
            u64 wk = pix * ch_w + (ch_w == 1 ? 0 : c);
            orc_ct_mul_int(n, limbs, q, img + (size_t)k * ct_len, ka, t1);
            orc_ct_mul_int(n, limbs, q, wm + (size_t)wk * ct_len, kb, t2);
            orc_ct_add(n, limbs, q, t1, t2, t1);
            orc_rescale(n, limbs, q, t1, out + (size_t)k * out_len);
        }
        free(t1); free(t2);
    }
    return 0;
}

/*
 * Image matching (Sec. 4.4.3; squared differences, since |x| is not
 * a CKKS operation): sum over all ciphertexts of (a_k - b_k)^2 as a degree-2
 * ciphertext, out is [3][limbs][n].  Relinearisation and rescale follow in the
 * caller (orc_relin, orc_rescale).
 */
int orc_sqdiff_sum(u32 n, u32 limbs, const u64 *q, const u64 *a, const u64 *b, u64 count, u64 *out)
{
    size_t ct_len = (size_t)2 * limbs * n;
    size_t t_len = (size_t)3 * limbs * n;
    int nt = orc_num_threads();
    u64 *partial = (u64 *)calloc((size_t)nt * t_len, sizeof(u64));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        u64 *d = (u64 *)malloc(sizeof(u64) * ct_len);
        u64 *t = (u64 *)malloc(sizeof(u64) * t_len);
        u64 *acc = partial + (size_t)tid * t_len;
#pragma omp for schedule(dynamic, 1)
        for (i64 k = 0; k < (i64)count; k++) {
            orc_ct_sub(n, limbs, q, a + (size_t)k * ct_len, b + (size_t)k * ct_len, d);
            orc_ct_square(n, limbs, q, d, t);
            for (u32 p = 0; p < 3; p++)
                for (u32 l = 0; l < limbs; l++)
                    for (u32 i = 0; i < n; i++) {
                        size_t x = ((size_t)p * limbs + l) * n + i;
                        acc[x] = mod_add(acc[x], t[x], q[l]);
                    }
        }
        free(d); free(t);
    }
    memset(out, 0, sizeof(u64) * t_len);
    for (int tid = 0; tid < nt; tid++)
        for (u32 p = 0; p < 3; p++)
            for (u32 l = 0; l < limbs; l++)
                for (u32 i = 0; i < n; i++) {
                    size_t x = ((size_t)p * limbs + l) * n + i;
                    out[x] = mod_add(out[x], partial[(size_t)tid * t_len + x], q[l]);
                }
    free(partial);
    return 0;
}
