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
// Twiddles: tw[k] = psi^{bitrev(k)}, itw[k] = psi^{-bitrev(k)}, psi a primitive 2N-th root.
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
__device__ __forceinline__ void fwd_regs(u64 (&r)[NP][16], int tid, const u64* __restrict__ tw,
                                         const u64* __restrict__ twp, u64 q)
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
                const u64 W = __ldg(tw + widx), Wp = __ldg(twp + widx);
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
__device__ __forceinline__ void inv_regs(u64 (&r)[NP][16], int tid, const u64* __restrict__ itw,
                                         const u64* __restrict__ itwp, u64 q)
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
                const u64 W = __ldg(itw + widx), Wp = __ldg(itwp + widx);
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
__device__ __forceinline__ void fwd_rest(u64* sm, u64 (&r)[NP][16], int tid, const u64* __restrict__ tw,
                                         const u64* __restrict__ twp, u64 q)
{
    if constexpr (S0 <= NttShape<LOGN>::LAST) {
        store_sm<LOGN, S0 - 4, NP>(sm, r, tid);
        __syncthreads();
        load_sm<LOGN, S0, NP>(sm, r, tid);
        fwd_regs<LOGN, S0, NP>(r, tid, tw, twp, q);
        fwd_rest<LOGN, S0 + 4, NP>(sm, r, tid, tw, twp, q);
    }
}

// Inverse passes S0, S0-4, ..., 0: on entry r holds bit-reversed data in the layout of pass
// S0 (no inverse stage applied yet), on exit natural-order data in the layout of pass 0.
template <int LOGN, int S0, int NP>
__device__ __forceinline__ void inv_rest(u64* sm, u64 (&r)[NP][16], int tid, const u64* __restrict__ itw,
                                         const u64* __restrict__ itwp, u64 q)
{
    inv_regs<LOGN, S0, NP>(r, tid, itw, itwp, q);
    if constexpr (S0 > 0) {
        store_sm<LOGN, S0, NP>(sm, r, tid);
        __syncthreads();
        load_sm<LOGN, S0 - 4, NP>(sm, r, tid);
        inv_rest<LOGN, S0 - 4, NP>(sm, r, tid, itw, itwp, q);
    }
}

// Whole forward transform of NP polynomials, input already in registers in the layout of
// pass 0 (values in [0, 4q); with TERNARY0, residues of a ternary polynomial); output in
// registers in the layout of the last pass. `sm` holds NP buffers of N words. The caller must
// make sure no thread still reads `sm` from an earlier use (a __syncthreads before the call).
template <int LOGN, int NP, bool TERNARY0 = false>
__device__ __forceinline__ void ntt_fwd_regs(u64* sm, u64 (&r)[NP][16], int tid, const ModTables& t, u64 q)
{
    fwd_regs<LOGN, 0, NP, TERNARY0>(r, tid, t.tw, t.twp, q);
    fwd_rest<LOGN, 4, NP>(sm, r, tid, t.tw, t.twp, q);
}

// Whole inverse transform of NP polynomials, input in registers in the layout of the last
// pass (values in [0, 2q)); output in registers in the layout of pass 0, natural order, in
// [0, 2q).
template <int LOGN, int NP>
__device__ __forceinline__ void ntt_inv_regs(u64* sm, u64 (&r)[NP][16], int tid, const ModTables& t, u64 q)
{
    inv_rest<LOGN, NttShape<LOGN>::LAST, NP>(sm, r, tid, t.itw, t.itwp, q);
}

}  // namespace ichee
