// ntt.cuh -- block-wide negacyclic NTT / inverse NTT over one RNS limb, for the products in
// R_q = Z_q[X]/(X^N + 1) that CKKS encryption, key generation and ct x ct multiplication
// need (Sec. 2.2, 2.2.2, 2.2.3).
//
// Layout: N = 2^LOGN residues, one thread block of N/16 threads, every thread holding 16
// residues per polynomial in registers. The log2(N) butterfly stages run in passes of up to 4
// stages (a radix-16 step entirely in registers); between passes the block exchanges data
// through one shared-memory buffer of N words per polynomial, XOR-swizzled
// (x ^ ((x >> 4) & 15)) so that every pass reads and writes without bank conflicts.
// NP polynomials over the same modulus can be transformed in lockstep: each twiddle pair is
// loaded once for all of them and the block barriers are shared.
//
// Forward: Cooley-Tukey with the negacyclic twist merged into the twiddles, natural-order
// input, bit-reversed output; inputs in [0, q), outputs in [0, 4q) (Harvey's lazy bounds).
// Inverse: Gentleman-Sande, bit-reversed input in [0, 2q), natural-order output in [0, 2q),
// without the 1/N factor (callers fold 1/N into a constant operand).
// Twiddles: tw[k] = psi^{bitrev(k)}, itw[k] = psi^{-bitrev(k)}, psi a primitive 2N-th root,
// each stored next to its Shoup companion (one 16-byte load per twiddle).
#pragma once
#include "common.cuh"

namespace ichee {

__device__ __forceinline__ int swz(int x) { return x ^ ((x >> 4) & 15); }

template <int LOGN, int S0>
struct Pass {
    static constexpr int N = 1 << LOGN;
    static constexpr int T = N / 16;
    static constexpr int S = (LOGN - S0) < 4 ? (LOGN - S0) : 4;  // stages in this pass
    static constexpr int G = 16 >> S;                               // groups per thread
    static constexpr int LO = LOGN - S0 - S;                        // lowest varying index bit
};

template <int LOGN>
struct NttShape {
    static constexpr int N = 1 << LOGN;
    static constexpr int T = N / 16;
    static constexpr int LAST = ((LOGN - 1) / 4) * 4;  // first stage of the last pass
};

// Natural index of register e of thread tid in the pass starting at stage S0.
template <int LOGN, int S0>
__device__ __forceinline__ int elem_index(int tid, int e)
{
    using P = Pass<LOGN, S0>;
    const int g = e >> P::S, j = e & ((1 << P::S) - 1);
    const int gid = g * P::T + tid;
    const int l = gid & ((1 << P::LO) - 1);
    const int h = gid >> P::LO;
    return (h << (P::LO + P::S)) | (j << P::LO) | l;
}

template <int LOGN, int S0, int NP>
__device__ __forceinline__ void load_sm(const u64* sm, u64 (&r)[NP][16], int tid)
{
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int e = 0; e < 16; ++e) r[p][e] = sm[p * (1 << LOGN) + swz(elem_index<LOGN, S0>(tid, e))];
}

template <int LOGN, int S0, int NP>
__device__ __forceinline__ void store_sm(u64* sm, const u64 (&r)[NP][16], int tid)
{
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int e = 0; e < 16; ++e) sm[p * (1 << LOGN) + swz(elem_index<LOGN, S0>(tid, e))] = r[p][e];
}

// Forward stages S0 .. S0+S-1 on the registers. Stage s pairs x with x + N/2^{s+1} and uses
// twiddle index 2^s + (x >> (LOGN - s)). With TERNARY0 the first stage of pass 0 takes the
// odd operands as ternary residues {0, 1, q-1}, whose products with the twiddle are 0, W and
// q - W: no multiplication.
template <int LOGN, int S0, int NP, bool TERNARY0 = false>
__device__ __forceinline__ void fwd_regs(u64 (&r)[NP][16], int tid, const ulonglong2* __restrict__ tw, u64 q)
{
    using P = Pass<LOGN, S0>;
    const u64 q2 = 2 * q;
#pragma unroll
    for (int g = 0; g < P::G; ++g) {
        const int h = (g * P::T + tid) >> P::LO;
#pragma unroll
        for (int k = 0; k < P::S; ++k) {
            const int s = S0 + k;
            const int half = 1 << (P::S - 1 - k);
#pragma unroll
            for (int b = 0; b < (1 << k); ++b) {
                const int widx = (1 << s) + (h << k) + b;
                const ulonglong2 w2 = __ldg(tw + widx);
                const u64 W = w2.x, Wp = w2.y;
#pragma unroll
                for (int jj = b * 2 * half; jj < b * 2 * half + half; ++jj) {
                    const int i0 = g * (1 << P::S) + jj, i1 = i0 + half;
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        u64 X = r[p][i0];
                        u64 Tt;
                        if (TERNARY0 && S0 == 0 && k == 0) {
                            const u64 y = r[p][i1];
                            Tt = y == 0 ? 0 : (y == 1 ? W : q - W);
                        } else {
                            X = X >= q2 ? X - q2 : X;
                            Tt = shoup_lazy(r[p][i1], W, Wp, q);
                        }
                        r[p][i0] = X + Tt;
                        r[p][i1] = X - Tt + q2;
                    }
                }
            }
        }
    }
}

// Inverse stages S0+S-1 .. S0 (reverse order) on the registers.
template <int LOGN, int S0, int NP>
__device__ __forceinline__ void inv_regs(u64 (&r)[NP][16], int tid, const ulonglong2* __restrict__ itw, u64 q)
{
    using P = Pass<LOGN, S0>;
    const u64 q2 = 2 * q;
#pragma unroll
    for (int g = 0; g < P::G; ++g) {
        const int h = (g * P::T + tid) >> P::LO;
#pragma unroll
        for (int k = P::S - 1; k >= 0; --k) {
            const int s = S0 + k;
            const int half = 1 << (P::S - 1 - k);
#pragma unroll
            for (int b = 0; b < (1 << k); ++b) {
                const int widx = (1 << s) + (h << k) + b;
                const ulonglong2 w2 = __ldg(itw + widx);
                const u64 W = w2.x, Wp = w2.y;
#pragma unroll
                for (int jj = b * 2 * half; jj < b * 2 * half + half; ++jj) {
                    const int i0 = g * (1 << P::S) + jj, i1 = i0 + half;
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        const u64 X = r[p][i0], Y = r[p][i1];
                        u64 U = X + Y;
                        U = U >= q2 ? U - q2 : U;
                        r[p][i0] = U;
                        r[p][i1] = shoup_lazy(X - Y + q2, W, Wp, q);
                    }
                }
            }
        }
    }
}

// Forward passes after the first: on entry r holds the output of pass S0-4 (its layout), on
// exit the output of the last pass in the last pass's layout.
template <int LOGN, int S0, int NP>
__device__ __forceinline__ void fwd_rest(u64* sm, u64 (&r)[NP][16], int tid, const ulonglong2* __restrict__ tw, u64 q)
{
    if constexpr (S0 <= NttShape<LOGN>::LAST) {
        store_sm<LOGN, S0 - 4, NP>(sm, r, tid);
        __syncthreads();
        load_sm<LOGN, S0, NP>(sm, r, tid);
        fwd_regs<LOGN, S0, NP>(r, tid, tw, q);
        fwd_rest<LOGN, S0 + 4, NP>(sm, r, tid, tw, q);
    }
}

// Inverse passes S0, S0-4, ..., 0: on entry r holds bit-reversed data in the layout of pass
// S0 (no inverse stage applied yet), on exit natural-order data in the layout of pass 0.
template <int LOGN, int S0, int NP>
__device__ __forceinline__ void inv_rest(u64* sm, u64 (&r)[NP][16], int tid, const ulonglong2* __restrict__ itw, u64 q)
{
    inv_regs<LOGN, S0, NP>(r, tid, itw, q);
    if constexpr (S0 > 0) {
        store_sm<LOGN, S0, NP>(sm, r, tid);
        __syncthreads();
        load_sm<LOGN, S0 - 4, NP>(sm, r, tid);
        inv_rest<LOGN, S0 - 4, NP>(sm, r, tid, itw, q);
    }
}

// ---------------------------------------------------------------------------------------
// Full radix-16 passes with the pass position as a runtime value. The register indexing is
// the same as in the compile-time form (S = 4, one group per thread); only the index bits of
// the shared-memory and twiddle addresses depend on the pass. Every full pass of a transform
// runs through one copy of this code, which keeps a kernel that chains many transforms
// small enough for the instruction cache.
// ---------------------------------------------------------------------------------------

// Natural index of register e of thread tid in the full pass whose lowest varying index bit
// is lo (= LOGN - S0 - 4): (tid >> lo) << (lo + 4) | e << lo | (tid & (2^lo - 1)).
__device__ __forceinline__ int pass_base(int tid, int lo) { return ((tid >> lo) << (lo + 4)) | (tid & ((1 << lo) - 1)); }

template <int LOGN, int NP>
__device__ __forceinline__ void store_sm_rt(u64* sm, const u64 (&r)[NP][16], int tid, int lo)
{
    const int base = pass_base(tid, lo);
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int e = 0; e < 16; ++e) sm[p * (1 << LOGN) + swz(base | (e << lo))] = r[p][e];
}

template <int LOGN, int NP>
__device__ __forceinline__ void load_sm_rt(const u64* sm, u64 (&r)[NP][16], int tid, int lo)
{
    const int base = pass_base(tid, lo);
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int e = 0; e < 16; ++e) r[p][e] = sm[p * (1 << LOGN) + swz(base | (e << lo))];
}

// Forward stages S0 .. S0+3 (lo = LOGN - S0 - 4).
template <int NP>
__device__ __forceinline__ void fwd_regs_rt(u64 (&r)[NP][16], int tid, int S0, int lo, const ulonglong2* __restrict__ tw, u64 q)
{
    const u64 q2 = 2 * q;
    const int h = tid >> lo;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int half = 1 << (3 - k);
#pragma unroll
        for (int b = 0; b < (1 << k); ++b) {
            const int widx = (1 << (S0 + k)) + (h << k) + b;
            const ulonglong2 w2 = __ldg(tw + widx);
                const u64 W = w2.x, Wp = w2.y;
#pragma unroll
            for (int jj = b * 2 * half; jj < b * 2 * half + half; ++jj) {
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    u64 X = r[p][jj];
                    X = X >= q2 ? X - q2 : X;
                    const u64 Tt = shoup_lazy(r[p][jj + half], W, Wp, q);
                    r[p][jj] = X + Tt;
                    r[p][jj + half] = X - Tt + q2;
                }
            }
        }
    }
}

// Inverse stages S0+3 .. S0 (lo = LOGN - S0 - 4).
template <int NP>
__device__ __forceinline__ void inv_regs_rt(u64 (&r)[NP][16], int tid, int S0, int lo, const ulonglong2* __restrict__ itw, u64 q)
{
    const u64 q2 = 2 * q;
    const int h = tid >> lo;
#pragma unroll
    for (int k = 3; k >= 0; --k) {
        const int half = 1 << (3 - k);
#pragma unroll
        for (int b = 0; b < (1 << k); ++b) {
            const int widx = (1 << (S0 + k)) + (h << k) + b;
            const ulonglong2 w2 = __ldg(itw + widx);
                const u64 W = w2.x, Wp = w2.y;
#pragma unroll
            for (int jj = b * 2 * half; jj < b * 2 * half + half; ++jj) {
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const u64 X = r[p][jj], Y = r[p][jj + half];
                    u64 U = X + Y;
                    U = U >= q2 ? U - q2 : U;
                    r[p][jj] = U;
                    r[p][jj + half] = shoup_lazy(X - Y + q2, W, Wp, q);
                }
            }
        }
    }
}

// Whole forward transform of NP polynomials, input already in registers in the layout of
// pass 0 (values in [0, 4q); with TERNARY0, residues of a ternary polynomial); output in
// registers in the layout of the last pass. `sm` holds NP buffers of N words. The caller must
// make sure no thread still reads `sm` from an earlier use (a __syncthreads before the call).
// Passes: LOGN / 4 full radix-16 passes, then one pass of the remaining LOGN % 4 stages.
// COMPACT runs the full passes through one runtime loop (one copy of the pass code); otherwise
// every pass is unrolled with its position known at compile time, which needs fewer address
// instructions but about LOGN / 4 times the code.
template <int LOGN, int NP, bool TERNARY0 = false, bool COMPACT = false>
__device__ __forceinline__ void ntt_fwd_regs(u64* sm, u64 (&r)[NP][16], int tid, const ModTables& t, u64 q)
{
    if constexpr (!COMPACT) {
        fwd_regs<LOGN, 0, NP, TERNARY0>(r, tid, t.tw, q);
        fwd_rest<LOGN, 4, NP>(sm, r, tid, t.tw, q);
        return;
    }
    constexpr int NFULL = LOGN / 4, TAIL = LOGN % 4;
    int p0 = 0;
    if constexpr (TERNARY0) {
        fwd_regs<LOGN, 0, NP, true>(r, tid, t.tw, q);
        p0 = 1;
    }
#pragma unroll 1
    for (int p = p0; p < NFULL; ++p) {
        const int lo = LOGN - 4 * p - 4;
        if (p > 0) {
            store_sm_rt<LOGN, NP>(sm, r, tid, lo + 4);
            __syncthreads();
            load_sm_rt<LOGN, NP>(sm, r, tid, lo);
        }
        fwd_regs_rt<NP>(r, tid, 4 * p, lo, t.tw, q);
    }
    if constexpr (TAIL > 0) {
        store_sm_rt<LOGN, NP>(sm, r, tid, LOGN - 4 * NFULL);
        __syncthreads();
        load_sm<LOGN, 4 * NFULL, NP>(sm, r, tid);
        fwd_regs<LOGN, 4 * NFULL, NP>(r, tid, t.tw, q);
    }
}

// Whole inverse transform of NP polynomials, input in registers in the layout of the last
// pass (values in [0, 2q)); output in registers in the layout of pass 0, natural order, in
// [0, 2q).
template <int LOGN, int NP, bool COMPACT = false>
__device__ __forceinline__ void ntt_inv_regs(u64* sm, u64 (&r)[NP][16], int tid, const ModTables& t, u64 q)
{
    if constexpr (!COMPACT) {
        inv_rest<LOGN, NttShape<LOGN>::LAST, NP>(sm, r, tid, t.itw, q);
        return;
    }
    constexpr int NFULL = LOGN / 4, TAIL = LOGN % 4;
    if constexpr (TAIL > 0) {
        inv_regs<LOGN, 4 * NFULL, NP>(r, tid, t.itw, q);
        store_sm<LOGN, 4 * NFULL, NP>(sm, r, tid);
        __syncthreads();
        load_sm_rt<LOGN, NP>(sm, r, tid, LOGN - 4 * NFULL);
    }
#pragma unroll 1
    for (int p = NFULL - 1; p >= 0; --p) {
        const int lo = LOGN - 4 * p - 4;
        inv_regs_rt<NP>(r, tid, 4 * p, lo, t.itw, q);
        if (p > 0) {
            store_sm_rt<LOGN, NP>(sm, r, tid, lo);
            __syncthreads();
            load_sm_rt<LOGN, NP>(sm, r, tid, lo + 4);
        }
    }
}

}  // namespace ichee
