// ntt.cuh -- block-wide negacyclic NTT / inverse NTT over one RNS limb, for the products in
// R_q = Z_q[X]/(X^N + 1) that CKKS encryption, key generation and ct x ct multiplication
// need (Sec. 2.2, 2.2.2, 2.2.3).
//
// Layout: N = 2^LOGN residues, one thread block of N/E threads, every thread holding E
// residues (E = 16 or 8) per polynomial in registers. The log2(N) butterfly stages run in
// passes of up to log2(E) stages (a radix-E step entirely in registers); between passes the
// block exchanges data through one shared-memory buffer of N words per polynomial,
// XOR-swizzled so that every pass reads and writes without bank conflicts (the host-compiled
// layout test checks every pass of N = 2^10 .. 2^14): x ^ ((x >> 4) & 15) for E = 16,
// x ^ ((x >> 2) & 7) ^ ((x >> 3) & 15) for E = 8. E = 8 halves the registers a polynomial
// takes, so twice the threads fit on an SM, at the price of one more exchange per transform.
// An exchange whose two layouts give every warp the same residues takes a warp barrier
// instead of a block barrier (the later passes of a transform). NP polynomials over the same
// modulus can be transformed in lockstep: each twiddle pair is loaded once for all of them and
// the barriers are shared.
//
// Between transforms on the same buffer: a forward transform's first exchange stores to its
// thread's pass-0 slots and its last exchange loads the thread's last-pass slots; an inverse
// does the reverse. So a forward after an inverse (or an inverse after a forward) overwrites
// only slots its own thread loaded last and needs no block barrier before it; two transforms
// of the same direction in a row do.
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

template <int E>
struct Radix {
    static_assert(E == 8 || E == 16, "8 or 16 residues per thread");
    static constexpr int LE = E == 16 ? 4 : 3;   // stages of a full pass
};

template <int E = 16>
__host__ __device__ constexpr int swz(int x)
{
    if constexpr (E == 16) return x ^ ((x >> 4) & 15);
    else return x ^ ((x >> 2) & 7) ^ ((x >> 3) & 15);
}

template <int LOGN, int S0, int E = 16>
struct Pass {
    static constexpr int LE = Radix<E>::LE;
    static constexpr int N = 1 << LOGN;
    static constexpr int T = N / E;
    static constexpr int S = (LOGN - S0) < LE ? (LOGN - S0) : LE;  // stages in this pass
    static constexpr int G = E >> S;                                 // groups per thread
    static constexpr int LO = LOGN - S0 - S;                         // lowest varying index bit
};

template <int LOGN, int E = 16>
struct NttShape {
    static constexpr int LE = Radix<E>::LE;
    static constexpr int N = 1 << LOGN;
    static constexpr int T = N / E;
    static constexpr int LAST = ((LOGN - 1) / LE) * LE;  // first stage of the last pass
};

__host__ __device__ constexpr int ilog2(int x) { return x > 1 ? 1 + ilog2(x >> 1) : 0; }

// Butterfly-group id of register group g of thread tid in a pass: a full pass has one group
// per thread; a partial last pass (fewer than LE stages, G > 1 groups per thread) keeps a
// warp's G x 32 groups adjacent (lane fastest, then g, then the warp), so that each warp holds
// the same 2^(LE+5) consecutive indices as in the full pass before it -- the exchange into the
// last pass stays inside the warp -- while a register's 32 lanes still touch consecutive
// butterflies (the coalescing and the bank pattern of global and shared accesses unchanged).
__host__ __device__ constexpr int pass_gid(int T, int G, int tid, int g, bool wt = true)
{
    return G > 1 && wt ? (((tid >> 5) << (5 + ilog2(G))) | (g << 5) | (tid & 31)) : g * T + tid;
}

// Natural index of register e of thread tid in the pass starting at stage S0 (values of the
// template parameters as arguments, for the compile-time checks below). WT = false keeps the
// groups of a partial last pass strided by the thread count (g * T + tid): the layout of the
// compact transform form.
__host__ __device__ constexpr int elem_index_of(int logn, int s0, int E, int tid, int e, bool wt = true)
{
    const int le = E == 16 ? 4 : 3;
    const int T = (1 << logn) / E;
    const int S = (logn - s0) < le ? (logn - s0) : le;
    const int G = E >> S, LO = logn - s0 - S;
    const int g = e >> S, j = e & ((1 << S) - 1);
    const int gid = pass_gid(T, G, tid, g, wt);
    return ((gid >> LO) << (LO + S)) | (j << LO) | (gid & ((1 << LO) - 1));
}

template <int LOGN, int S0, int E = 16, bool WT = true>
__device__ __forceinline__ int elem_index(int tid, int e) { return elem_index_of(LOGN, S0, E, tid, e, WT); }

// Whether the exchange between the layouts of the passes starting at SA and SB stays inside
// every warp: both layouts are bit permutations of (tid, e), so it does when the index bits
// driven by a warp's lane bits and the register bits are the same set in both, and every
// higher thread bit lands on the same index bit in both. Such an exchange needs only a warp
// barrier: a thread stores to the slots it loaded in the exchange before (the same layout),
// so no other warp's loads can be overtaken.
__host__ __device__ constexpr bool exchange_in_warp(int logn, int sa, int sb, int E)
{
    const int T = (1 << logn) / E;
    int va = 0, vb = 0;
    for (int i = 0; i < 5; ++i) {
        va |= elem_index_of(logn, sa, E, 1 << i, 0);
        vb |= elem_index_of(logn, sb, E, 1 << i, 0);
    }
    for (int k = 1; k < E; k <<= 1) {
        va |= elem_index_of(logn, sa, E, 0, k);
        vb |= elem_index_of(logn, sb, E, 0, k);
    }
    if (va != vb) return false;
    for (int i = 5; (1 << i) < T; ++i)
        if (elem_index_of(logn, sa, E, 1 << i, 0) != elem_index_of(logn, sb, E, 1 << i, 0)) return false;
    return true;
}

// Bit p set: the exchange between full passes p - 1 and p stays inside every warp (full passes
// have the same layout in both forms of the transform; the exchange is the same in the inverse
// direction).
__host__ __device__ constexpr unsigned full_exchanges_in_warp(int logn, int E)
{
    const int le = E == 16 ? 4 : 3;
    unsigned m = 0;
    for (int p = 1; p < logn / le; ++p)
        if (exchange_in_warp(logn, le * (p - 1), le * p, E)) m |= 1u << p;
    return m;
}

// The barrier of an exchange between two pass layouts.
template <bool IN_WARP>
__device__ __forceinline__ void exchange_barrier()
{
    if constexpr (IN_WARP) __syncwarp();
    else __syncthreads();
}

// Without the swizzle the split is additive: elem_index(tid, e) = elem_index(tid, 0) +
// elem_index(0, e) (disjoint bits), so global accesses take a per-thread base pointer and
// compile-time offsets.
template <int LOGN, int S0, int E = 16, bool WT = true>
__device__ __forceinline__ int elem_offset(int e) { return elem_index<LOGN, S0, E, WT>(0, e); }

// Shared-memory slot of register e of thread tid in the pass starting at S0. elem_index is a
// permutation of the bits of (tid, e) and the swizzle is linear over GF(2), so the slot is
// swz(elem_index(tid, 0)) ^ swz(elem_index(0, e)): a per-thread base XOR a compile-time
// constant, one instruction per access (checked for every pass of N = 2^10 .. 2^14).
template <int LOGN, int S0, int E = 16, bool WT = true>
__device__ __forceinline__ int slot_base(int tid) { return swz<E>(elem_index<LOGN, S0, E, WT>(tid, 0)); }

template <int LOGN, int S0, int E = 16, bool WT = true>
__device__ __forceinline__ int slot_of(int base, int e) { return base ^ swz<E>(elem_index<LOGN, S0, E, WT>(0, e)); }

template <int LOGN, int S0, int NP, int E = 16, bool WT = true>
__device__ __forceinline__ void load_sm(const u64* sm, u64 (&r)[NP][E], int tid)
{
    const int base = slot_base<LOGN, S0, E, WT>(tid);
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int e = 0; e < E; ++e) r[p][e] = sm[p * (1 << LOGN) + slot_of<LOGN, S0, E, WT>(base, e)];
}

template <int LOGN, int S0, int NP, int E = 16, bool WT = true>
__device__ __forceinline__ void store_sm(u64* sm, const u64 (&r)[NP][E], int tid)
{
    const int base = slot_base<LOGN, S0, E, WT>(tid);
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int e = 0; e < E; ++e) sm[p * (1 << LOGN) + slot_of<LOGN, S0, E, WT>(base, e)] = r[p][e];
}

// Forward stages S0 .. S0+S-1 on the registers. Stage s pairs x with x + N/2^{s+1} and uses
// twiddle index 2^s + (x >> (LOGN - s)). With TERNARY0 the first stage of pass 0 takes the
// odd operands as ternary residues {0, 1, q-1}, whose products with the twiddle are 0, W and
// q - W: no multiplication.
template <int LOGN, int S0, int NP, bool TERNARY0 = false, int E = 16, bool WT = true>
__device__ __forceinline__ void fwd_regs(u64 (&r)[NP][E], int tid, const ulonglong2* __restrict__ tw, u64 q)
{
    using P = Pass<LOGN, S0, E>;
    const u64 q2 = 2 * q;
#pragma unroll
    for (int g = 0; g < P::G; ++g) {
        const int h = pass_gid(P::T, P::G, tid, g, WT) >> P::LO;
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
template <int LOGN, int S0, int NP, int E = 16, bool WT = true>
__device__ __forceinline__ void inv_regs(u64 (&r)[NP][E], int tid, const ulonglong2* __restrict__ itw, u64 q)
{
    using P = Pass<LOGN, S0, E>;
    const u64 q2 = 2 * q;
#pragma unroll
    for (int g = 0; g < P::G; ++g) {
        const int h = pass_gid(P::T, P::G, tid, g, WT) >> P::LO;
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

// Forward passes after the first: on entry r holds the output of pass S0-LE (its layout), on
// exit the output of the last pass in the last pass's layout.
template <int LOGN, int S0, int NP, int E = 16>
__device__ __forceinline__ void fwd_rest(u64* sm, u64 (&r)[NP][E], int tid, const ulonglong2* __restrict__ tw, u64 q)
{
    constexpr int LE = Radix<E>::LE;
    if constexpr (S0 <= NttShape<LOGN, E>::LAST) {
        store_sm<LOGN, S0 - LE, NP, E>(sm, r, tid);
        exchange_barrier<exchange_in_warp(LOGN, S0 - LE, S0, E)>();
        load_sm<LOGN, S0, NP, E>(sm, r, tid);
        fwd_regs<LOGN, S0, NP, false, E>(r, tid, tw, q);
        fwd_rest<LOGN, S0 + LE, NP, E>(sm, r, tid, tw, q);
    }
}

// Inverse passes S0, S0-LE, ..., 0: on entry r holds bit-reversed data in the layout of pass
// S0 (no inverse stage applied yet), on exit natural-order data in the layout of pass 0.
template <int LOGN, int S0, int NP, int E = 16>
__device__ __forceinline__ void inv_rest(u64* sm, u64 (&r)[NP][E], int tid, const ulonglong2* __restrict__ itw, u64 q)
{
    constexpr int LE = Radix<E>::LE;
    inv_regs<LOGN, S0, NP, E>(r, tid, itw, q);
    if constexpr (S0 > 0) {
        store_sm<LOGN, S0, NP, E>(sm, r, tid);
        exchange_barrier<exchange_in_warp(LOGN, S0, S0 - LE, E)>();
        load_sm<LOGN, S0 - LE, NP, E>(sm, r, tid);
        inv_rest<LOGN, S0 - LE, NP, E>(sm, r, tid, itw, q);
    }
}

// ---------------------------------------------------------------------------------------
// Full passes with the pass position as a runtime value. The register indexing is the same as
// in the compile-time form (S = LE, one group per thread); only the index bits of the
// shared-memory and twiddle addresses depend on the pass. Every full pass of a transform runs
// through one copy of this code, which keeps a kernel that chains many transforms small
// enough for the instruction cache.
// ---------------------------------------------------------------------------------------

// Natural index of register e of thread tid in the full pass whose lowest varying index bit
// is lo (= LOGN - S0 - LE): (tid >> lo) << (lo + LE) | e << lo | (tid & (2^lo - 1)).
template <int LE>
__device__ __forceinline__ int pass_base(int tid, int lo) { return ((tid >> lo) << (lo + LE)) | (tid & ((1 << lo) - 1)); }

// As in the compile-time form, slot = swz(base) ^ swz(e << lo); with lo known only at run time
// the E offsets swz(e << lo) are XOR combinations of the LE basis values swz(2^k << lo).
template <int E = 16>
__device__ __forceinline__ void rt_offsets(int lo, int (&c)[E])
{
    constexpr int LE = Radix<E>::LE;
    int b[LE];
#pragma unroll
    for (int k = 0; k < LE; ++k) b[k] = swz<E>(1 << (k + lo));
#pragma unroll
    for (int e = 0; e < E; ++e) {
        int v = 0;
#pragma unroll
        for (int k = 0; k < LE; ++k)
            if (e & (1 << k)) v ^= b[k];
        c[e] = v;
    }
}

template <int LOGN, int NP, int E = 16>
__device__ __forceinline__ void store_sm_rt(u64* sm, const u64 (&r)[NP][E], int tid, int lo)
{
    const int base = swz<E>(pass_base<Radix<E>::LE>(tid, lo));
    int c[E];
    rt_offsets<E>(lo, c);
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int e = 0; e < E; ++e) sm[p * (1 << LOGN) + (base ^ c[e])] = r[p][e];
}

template <int LOGN, int NP, int E = 16>
__device__ __forceinline__ void load_sm_rt(const u64* sm, u64 (&r)[NP][E], int tid, int lo)
{
    const int base = swz<E>(pass_base<Radix<E>::LE>(tid, lo));
    int c[E];
    rt_offsets<E>(lo, c);
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int e = 0; e < E; ++e) r[p][e] = sm[p * (1 << LOGN) + (base ^ c[e])];
}

// Forward stages S0 .. S0+LE-1 (lo = LOGN - S0 - LE).
template <int NP, int E = 16>
__device__ __forceinline__ void fwd_regs_rt(u64 (&r)[NP][E], int tid, int S0, int lo, const ulonglong2* __restrict__ tw,
                                            u64 q)
{
    constexpr int LE = Radix<E>::LE;
    const u64 q2 = 2 * q;
    const int h = tid >> lo;
#pragma unroll
    for (int k = 0; k < LE; ++k) {
        const int half = 1 << (LE - 1 - k);
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

// Inverse stages S0+LE-1 .. S0 (lo = LOGN - S0 - LE).
template <int NP, int E = 16>
__device__ __forceinline__ void inv_regs_rt(u64 (&r)[NP][E], int tid, int S0, int lo, const ulonglong2* __restrict__ itw,
                                            u64 q)
{
    constexpr int LE = Radix<E>::LE;
    const u64 q2 = 2 * q;
    const int h = tid >> lo;
#pragma unroll
    for (int k = LE - 1; k >= 0; --k) {
        const int half = 1 << (LE - 1 - k);
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
// make sure no thread still reads `sm` from an earlier use other than an inverse transform's
// (a __syncthreads before the call; see the header comment).
// Passes: LOGN / LE full passes, then one pass of the remaining LOGN % LE stages.
// COMPACT runs the full passes through one runtime loop (one copy of the pass code); otherwise
// every pass is unrolled with its position known at compile time, which needs fewer address
// instructions but about LOGN / LE times the code. Both take a warp barrier for the exchanges
// that stay inside every warp (exchange_in_warp). The compact form, used by the per-pixel
// squared difference at N = 2^14 (where the unrolled passes spill), keeps the strided last-pass
// layout (WT = false; its callers index the last pass with it) and a block barrier into it:
// there the warp-adjacent layout took more registers (spills 8 -> 76 bytes) and time.
template <int LOGN, int NP, bool TERNARY0 = false, bool COMPACT = false, int E = 16>
__device__ __forceinline__ void ntt_fwd_regs(u64* sm, u64 (&r)[NP][E], int tid, const ModTables& t, u64 q)
{
    constexpr int LE = Radix<E>::LE;
    if constexpr (!COMPACT) {
        fwd_regs<LOGN, 0, NP, TERNARY0, E>(r, tid, t.tw, q);
        fwd_rest<LOGN, LE, NP, E>(sm, r, tid, t.tw, q);
        return;
    }
    constexpr int NFULL = LOGN / LE, TAIL = LOGN % LE;
    int p0 = 0;
    if constexpr (TERNARY0) {
        fwd_regs<LOGN, 0, NP, true, E>(r, tid, t.tw, q);
        p0 = 1;
    }
    constexpr unsigned in_warp = full_exchanges_in_warp(LOGN, E);
#pragma unroll 1
    for (int p = p0; p < NFULL; ++p) {
        const int lo = LOGN - LE * p - LE;
        if (p > 0) {
            store_sm_rt<LOGN, NP, E>(sm, r, tid, lo + LE);
            if ((in_warp >> p) & 1u) __syncwarp();   // uniform across the block
            else __syncthreads();
            load_sm_rt<LOGN, NP, E>(sm, r, tid, lo);
        }
        fwd_regs_rt<NP, E>(r, tid, LE * p, lo, t.tw, q);
    }
    if constexpr (TAIL > 0) {
        store_sm_rt<LOGN, NP, E>(sm, r, tid, LOGN - LE * NFULL);
        __syncthreads();
        load_sm<LOGN, LE * NFULL, NP, E, false>(sm, r, tid);
        fwd_regs<LOGN, LE * NFULL, NP, false, E, false>(r, tid, t.tw, q);
    }
}

// Whole inverse transform of NP polynomials, input in registers in the layout of the last
// pass (values in [0, 2q)); output in registers in the layout of pass 0, natural order, in
// [0, 2q).
template <int LOGN, int NP, bool COMPACT = false, int E = 16>
__device__ __forceinline__ void ntt_inv_regs(u64* sm, u64 (&r)[NP][E], int tid, const ModTables& t, u64 q)
{
    constexpr int LE = Radix<E>::LE;
    if constexpr (!COMPACT) {
        inv_rest<LOGN, NttShape<LOGN, E>::LAST, NP, E>(sm, r, tid, t.itw, q);
        return;
    }
    constexpr int NFULL = LOGN / LE, TAIL = LOGN % LE;
    if constexpr (TAIL > 0) {
        inv_regs<LOGN, LE * NFULL, NP, E, false>(r, tid, t.itw, q);
        store_sm<LOGN, LE * NFULL, NP, E, false>(sm, r, tid);
        __syncthreads();
        load_sm_rt<LOGN, NP, E>(sm, r, tid, LOGN - LE * NFULL);
    }
    constexpr unsigned in_warp = full_exchanges_in_warp(LOGN, E);
#pragma unroll 1
    for (int p = NFULL - 1; p >= 0; --p) {
        const int lo = LOGN - LE * p - LE;
        inv_regs_rt<NP, E>(r, tid, LE * p, lo, t.itw, q);
        if (p > 0) {
            store_sm_rt<LOGN, NP, E>(sm, r, tid, lo);
            if ((in_warp >> p) & 1u) __syncwarp();
            else __syncthreads();
            load_sm_rt<LOGN, NP, E>(sm, r, tid, lo + LE);
        }
    }
}

}  // namespace ichee
