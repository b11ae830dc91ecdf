// kernels_match.cu -- image matching (Sec. 4.4.3, as a squared L2 distance): the sum over all pixel
// ciphertexts of (a - b)^2 with ct x ct multiplication, then relinearisation with the
// evaluation key (Sec. 2.2.3; hybrid key switching with one special prime P).
#include "ops.h"
#include "ntt.cuh"

namespace ichee {

// One block per SM-sized share of the work: block j owns limb l = j % limbs and every
// (n_blocks/limbs)-th ciphertext. Per ciphertext it forms d = a - b for its limb, transforms
// d0 and d1, and accumulates (d0^2, 2 d0 d1, d1^2) position by position into its own slice of
// the scratch buffer (each position is owned by one thread, so no atomics are needed). The
// transform of d0 waits in a second shared-memory buffer (SMEM_D0) or, for the 2^14 ring whose
// buffers do not both fit, in the fourth scratch row; d1's waits in the transform buffer. Every
// thread parks and reads back only the slots of its own last-pass registers -- the slots it
// loaded in the transform's last exchange -- so no barrier follows the transform (2.69 -> 2.67
// ms); the barrier before each transform remains (its first exchange writes other slots).
template <int LOGN, bool SMEM_D0, int E>
__global__ void __launch_bounds__(NttShape<LOGN, E>::T, 1) k_sqdiff_accumulate(const __grid_constant__ SqDiffArgs a)
{
    constexpr int N = 1 << LOGN;
    constexpr int LAST = NttShape<LOGN, E>::LAST;
    extern __shared__ u64 buf[];
    u64* acc = a.partial + (size_t)blockIdx.x * 4 * N;
    u64* d0buf = SMEM_D0 ? buf + N : acc + 3 * N;
    const int tid = threadIdx.x;
    const int limbs = a.limbs;
    const int l = blockIdx.x % limbs;
    const u64 stride = a.n_blocks / limbs;
    const u64 start = blockIdx.x / limbs;
    const u64 q = a.rns.q[l];
    const u64 qinv = a.rns.qinv[l];
    const ModTables t = a.rns.tab[l];
    // In the last pass registers e and e + 1 (e even) hold positions x and x + 1 (its lowest
    // index bit is the stage bit), so the accumulators are read and written in 16-byte pairs.
#pragma unroll
    for (int e = 0; e < E; e += 2) {
        const int x = elem_index<LOGN, LAST, E>(tid, e);
        *reinterpret_cast<ulonglong2*>(acc + x) = make_ulonglong2(0, 0);
        *reinterpret_cast<ulonglong2*>(acc + N + x) = make_ulonglong2(0, 0);
        *reinterpret_cast<ulonglong2*>(acc + 2 * N + x) = make_ulonglong2(0, 0);
    }
    for (u64 k = start; k < a.n_ct; k += stride) {
        const u64* A = a.a + k * 2 * (u64)limbs * N;
        const u64* B = a.b + k * 2 * (u64)limbs * N;
#pragma unroll 1
        for (int pb = 0; pb < 2; ++pb) {
            const int x0 = elem_index<LOGN, 0, E>(tid, 0);   // first-pass layout: x0 + elem_offset(e)
            const u64* pa = A + ((u64)pb * limbs + l) * N + x0;
            const u64* pbb = B + ((u64)pb * limbs + l) * N + x0;
            u64 r[1][E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int x = elem_offset<LOGN, 0, E>(e);
                r[0][e] = sub_mod(__ldcs(pa + x), __ldcs(pbb + x), q);
            }
            // with both buffers in shared memory d0 is transformed in its parking buffer and d1 in
            // the other one: d1's transform then starts after d0's block-wide exchanges, which
            // every thread reaches only after its reads of the previous pixel, so it needs no
            // barrier of its own
            if (pb == 0 || !SMEM_D0) __syncthreads();
            ntt_fwd_regs<LOGN, 1, false, false, E>(SMEM_D0 && pb == 0 ? d0buf : buf, r, tid, t, q);
            u64* dst = pb == 0 ? d0buf : buf;
            const int sb = slot_base<LOGN, LAST, E>(tid);
            const int xl = elem_index<LOGN, LAST, E>(tid, 0);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int at = SMEM_D0 || pb ? slot_of<LOGN, LAST, E>(sb, e) : xl + elem_offset<LOGN, LAST, E>(e);
                dst[at] = csub(csub(r[0][e], 2 * q), q);
            }
        }
#pragma unroll   // unrolled: 2.62 -> 2.60 ms (the split kernel below keeps its loop: 2.45 -> 2.71 ms unrolled)
        for (int e = 0; e < E; e += 2) {
            const int x = elem_index<LOGN, LAST, E>(tid, e);
            ulonglong2* p0 = reinterpret_cast<ulonglong2*>(acc + x);
            ulonglong2* p1 = reinterpret_cast<ulonglong2*>(acc + N + x);
            ulonglong2* p2 = reinterpret_cast<ulonglong2*>(acc + 2 * N + x);
            ulonglong2 s0 = *p0, s1 = *p1, s2 = *p2;
            u64 t[2][3];
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const u64 d1 = buf[swz<E>(x + hh)];
                const u64 d0 = SMEM_D0 ? d0buf[swz<E>(x + hh)] : d0buf[x + hh];
                t[hh][0] = mont_mul(d0, d0, q, qinv);   // every term carries 2^{-64}, undone after the INTT
                const u64 c = mont_mul(d0, d1, q, qinv);
                t[hh][1] = add_mod(c, c, q);
                t[hh][2] = mont_mul(d1, d1, q, qinv);
            }
            s0 = make_ulonglong2(add_mod(s0.x, t[0][0], q), add_mod(s0.y, t[1][0], q));
            s1 = make_ulonglong2(add_mod(s1.x, t[0][1], q), add_mod(s1.y, t[1][1], q));
            s2 = make_ulonglong2(add_mod(s2.x, t[0][2], q), add_mod(s2.y, t[1][2], q));
            *p0 = s0;
            *p1 = s1;
            *p2 = s2;
        }
    }
}

// N = 2^14, split: the first stage of the forward transform pairs x with x + N/2 and leaves two
// independent 2^13-point transforms (outputs with the top index bit clear, and set). Block j
// takes limb j % limbs and half h = (j / limbs) % 2: it loads both halves of d = a - b, applies
// the first-stage butterfly for its half only (the product W d_hi is made by both halves'
// blocks: 1/14 more products), and runs the other 13 stages with the 2^13-point code -- 8
// residues per thread, 1024 threads, no spills -- and the half's twiddles:
// tw_h[2^s + g] = tw[(2 + h) 2^s + g]. Its tensor terms go to a [4][N/2] slice. The two
// blocks of a half pair read the same ciphertexts at about the same time (one HBM read, one
// L2 hit).
__global__ void __launch_bounds__(1024, 1) k_sqdiff_accumulate_split(const __grid_constant__ SqDiffArgs a)
{
    constexpr int LOGH = 13, NH = 1 << LOGH, N = 2 * NH, E = 8;
    constexpr int LAST = NttShape<LOGH, E>::LAST;
    extern __shared__ u64 buf[];
    u64* d0buf = buf + NH;
    const int tid = threadIdx.x;
    const int limbs = a.limbs;
    const int l = blockIdx.x % limbs;
    const int h = (blockIdx.x / limbs) & 1;
    const u64 stride = a.n_blocks / (2 * limbs);
    const u64 start = blockIdx.x / (2 * limbs);
    u64* acc = a.partial + (size_t)blockIdx.x * 4 * NH;
    const u64 q = a.rns.q[l];
    const u64 qinv = a.rns.qinv[l];
    const ModTables t = a.htab[h][l];
    const ulonglong2 w1 = a.rns.tab[l].tw[1];   // the first stage's twiddle and its companion
#pragma unroll
    for (int e = 0; e < E; e += 2) {
        const int x = elem_index<LOGH, LAST, E>(tid, e);
        *reinterpret_cast<ulonglong2*>(acc + x) = make_ulonglong2(0, 0);
        *reinterpret_cast<ulonglong2*>(acc + NH + x) = make_ulonglong2(0, 0);
        *reinterpret_cast<ulonglong2*>(acc + 2 * NH + x) = make_ulonglong2(0, 0);
    }
    for (u64 k = start; k < a.n_ct; k += stride) {
        const u64* A = a.a + k * 2 * (u64)limbs * N;
        const u64* B = a.b + k * 2 * (u64)limbs * N;
#pragma unroll 1
        for (int pb = 0; pb < 2; ++pb) {
            const int x0 = elem_index<LOGH, 0, E>(tid, 0);
            const u64* pa = A + ((u64)pb * limbs + l) * N + x0;
            const u64* pbb = B + ((u64)pb * limbs + l) * N + x0;
            u64 r[1][E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int x = elem_offset<LOGH, 0, E>(e);
                const u64 lo = sub_mod(pa[x], pbb[x], q);
                const u64 hi = sub_mod(pa[x + NH], pbb[x + NH], q);
                const u64 tt = shoup_lazy(hi, w1.x, w1.y, q);   // [0, 2q)
                r[0][e] = h ? lo + 2 * q - tt : lo + tt;         // [0, 3q)
            }
            if (pb == 0) __syncthreads();   // d0 in its parking buffer, d1 in the other (as above)
            ntt_fwd_regs<LOGH, 1, false, false, E>(pb == 0 ? d0buf : buf, r, tid, t, q);
            u64* dst = pb == 0 ? d0buf : buf;
            const int sb = slot_base<LOGH, LAST, E>(tid);
#pragma unroll
            for (int e = 0; e < E; ++e) dst[slot_of<LOGH, LAST, E>(sb, e)] = csub(csub(r[0][e], 2 * q), q);
        }
#pragma unroll 1
        for (int e = 0; e < E; e += 2) {
            const int x = elem_index<LOGH, LAST, E>(tid, e);
            ulonglong2* p0 = reinterpret_cast<ulonglong2*>(acc + x);
            ulonglong2* p1 = reinterpret_cast<ulonglong2*>(acc + NH + x);
            ulonglong2* p2 = reinterpret_cast<ulonglong2*>(acc + 2 * NH + x);
            ulonglong2 s0 = *p0, s1 = *p1, s2 = *p2;
            u64 tt[2][3];
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const u64 d1 = buf[swz<E>(x + hh)];
                const u64 d0 = d0buf[swz<E>(x + hh)];
                tt[hh][0] = mont_mul(d0, d0, q, qinv);   // every term carries 2^{-64}, undone after the INTT
                const u64 c = mont_mul(d0, d1, q, qinv);
                tt[hh][1] = add_mod(c, c, q);
                tt[hh][2] = mont_mul(d1, d1, q, qinv);
            }
            *p0 = make_ulonglong2(add_mod(s0.x, tt[0][0], q), add_mod(s0.y, tt[1][0], q));
            *p1 = make_ulonglong2(add_mod(s1.x, tt[0][1], q), add_mod(s1.y, tt[1][1], q));
            *p2 = make_ulonglong2(add_mod(s2.x, tt[0][2], q), add_mod(s2.y, tt[1][2], q));
        }
    }
}

// Residues per thread: 8 at N = 2^13 (1024 threads), else 16.
template <int LOGN>
static constexpr int kSqE = LOGN == 13 ? 8 : 16;

template <int LOGN>
static cudaError_t sqdiff_launch(const SqDiffArgs& a, cudaStream_t st)
{
    constexpr bool keep = LOGN <= 13;
    constexpr int E = kSqE<LOGN>;
    const size_t smem = (keep ? 2 : 1) * (sizeof(u64) << LOGN);
    cudaError_t e = cudaFuncSetAttribute(k_sqdiff_accumulate<LOGN, keep, E>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sqdiff_accumulate<LOGN, keep, E><<<a.n_blocks, NttShape<LOGN, E>::T, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sqdiff_accumulate(const SqDiffArgs& a, cudaStream_t st)
{
    if (a.n_blocks <= 0 || a.n_blocks % a.limbs != 0) return cudaErrorInvalidValue;
    if (sqdiff_split(a.rns.logn)) {
        if (a.n_blocks % (2 * a.limbs) != 0) return cudaErrorInvalidValue;
        const size_t smem = 2 * (sizeof(u64) << 13);
        cudaError_t e = cudaFuncSetAttribute(k_sqdiff_accumulate_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        k_sqdiff_accumulate_split<<<a.n_blocks, NttShape<13, 8>::T, smem, st>>>(a);
        return cudaGetLastError();
    }
    switch (a.rns.logn) {
    case 10: return sqdiff_launch<10>(a, st);
    case 11: return sqdiff_launch<11>(a, st);
    case 12: return sqdiff_launch<12>(a, st);
    case 13: return sqdiff_launch<13>(a, st);
    case 14: return sqdiff_launch<14>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

__global__ void k_sqdiff_reduce(RnsArgs rns, int limbs, const u64* partial, int n_blocks, u64* tensor, int add)
{
    const int n = 1 << rns.logn;
    const int pl = blockIdx.y;                 // p * limbs + l
    const int p = pl / limbs, l = pl % limbs;
    const u64 q = rns.q[l];
    const bool split = sqdiff_split(rns.logn);
    const int row = split ? n / 2 : n;         // slice row length
    const int step = split ? 2 * limbs : limbs;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        u64 s = add ? reduce64(tensor[(size_t)pl * n + x], q, rns.mu[l]) : 0;
        const int h = split ? x / row : 0, xx = split ? x % row : x;
        for (int j = l + h * limbs; j < n_blocks; j += step) s = add_mod(s, partial[((size_t)j * 4 + p) * row + xx], q);
        tensor[(size_t)pl * n + x] = s;
    }
}

cudaError_t launch_sqdiff_reduce(const RnsArgs& rns, int limbs, const u64* partial, int n_blocks, u64* tensor,
                                 bool add, cudaStream_t st)
{
    dim3 grid((1u << rns.logn) / 256, 3 * limbs);
    k_sqdiff_reduce<<<grid, 256, 0, st>>>(rns, limbs, partial, n_blocks, tensor, add ? 1 : 0);
    return cudaGetLastError();
}

// out[r][x] = in[r][x] mod q_{r % limbs} for any 64-bit input word (sums of accumulators).
__global__ void k_reduce_rows(RnsArgs rns, int limbs, const u64* in, u64* out)
{
    const int n = 1 << rns.logn;
    const int r = blockIdx.y, l = r % limbs;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
        out[(size_t)r * n + x] = reduce64(in[(size_t)r * n + x], rns.q[l], rns.mu[l]);
}

cudaError_t launch_reduce_rows(const RnsArgs& rns, int rows, int limbs, const u64* in, u64* out, cudaStream_t st)
{
    dim3 grid((1u << rns.logn) / 256, rows);
    k_reduce_rows<<<grid, 256, 0, st>>>(rns, limbs, in, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Per-pixel squared difference: out_k = Rescale(Relin((a_k - b_k) (x) (a_k - b_k))) for every
// ciphertext pair (the per-pixel form of Sec. 4.4.3; Relin by hybrid key switching, rescale
// with centered rounding). A persistent block takes one pixel at a time and runs the whole chain on it:
//   1. per limb l: d^ = NTT(a - b) for both polynomials; t0^ = d0^2, t1^ = 2 d0 d1 stay in the
//      NTT domain; t2 = INTT(d1^2) (N^{-1} folded into the product). The squares are
//      Montgomery products, so each carries 2^{-64}; the constants below carry 2^64. Digit l
//      of t2 lifted to its own modulus q_l is t2_l itself, whose transform d1^2 is at hand, so
//      the accumulators of modulus q_l start here: acc_b = (P N^{-1} 2^64) t_b^ + d1^2 evk^_l[b][l];
//   2. per modulus m (P first, then q_t, then q_0..q_{t-1}): acc_b += NTT([t2]_j lifted to m) *
//      evk^_j[b][m] for every digit j != m (all j for P), so INTT(acc_b) = P t_b + key-switched
//      part and (INTT(acc_b) - [acc_b mod P]) P^{-1} is the relinearised limb m;
//   3. the relinearised limb q_t is kept; every other limb is rescaled against it and stored.
// That is L^2 + 5L + 2 transforms per pixel (t2 is the only tensor limb inverse-transformed,
// and no digit is transformed back into its own modulus). They run in one loop over a per-pixel
// schedule (one word per transform, in shared memory) with one call site per direction, so the
// transform code with every pass unrolled appears twice and fits the instruction cache (four
// unrolled call sites did not; the compact pass loop in this schedule took 15.0 ms for 4096
// pixels at N = 2^13, the unrolled passes 12.6 ms, the compact loop at four call sites 13.9).
// A transform's first exchange stores to the slots of its thread in pass 0 (forward) or in the
// last pass (inverse), and its last exchange loads the slots of the other end, so a block
// barrier is needed only between two transforms of the same direction: after a forward, an
// inverse overwrites only slots its thread loaded last, and after an inverse a forward does.
// Every intermediate word is produced and consumed by the same thread (the transforms move
// data between threads only through their own shared buffer), so the block's scratch
// ([3 limbs + 2][N] words: t0^, t1^, t2 per limb, then the two P accumulators) is stored
// thread-major -- element e of thread tid at e * T + tid -- which makes every scratch access
// coalesced and needs no barrier of its own. The key-switching accumulators of modulus q_m
// build up in the t0^ / t1^ slots of limb m (the P accumulators in their own slots); keeping
// them in shared memory instead was slower, because the larger carve-out leaves too little
// L1 for the twiddle tables.
// ---------------------------------------------------------------------------------------
// Transform kinds of the per-pixel schedule.
constexpr u32 kFwdDiff = 0, kInvT2 = 1, kFwdDigit = 2, kInvAcc = 3;

template <int LOGN, int E>
__global__ void __launch_bounds__(NttShape<LOGN, E>::T) k_sqdiff_image(const __grid_constant__ SqImgArgs a)
{
    constexpr int N = 1 << LOGN;
    constexpr int T = NttShape<LOGN, E>::T;
    constexpr int LAST = NttShape<LOGN, E>::LAST;
    // transforms with every pass unrolled up to N = 2^13 (one call site per direction, so the
    // code fits the instruction cache), the compact pass loop at 2^14 (registers)
    constexpr bool CMP = LOGN >= 14;
    constexpr bool WT = !CMP;   // the last-pass layout of the unrolled form keeps a warp's groups adjacent
    extern __shared__ u64 sm[];
    u32* sched = reinterpret_cast<u32*>(sm + N);
    const int tid = threadIdx.x;
    const int limbs = a.limbs, L = a.L;
    const int t = limbs - 1;
    u64* S = a.scratch + (size_t)blockIdx.x * (3 * limbs + 2) * N + tid;   // thread-major slots
    u64* T0 = S;                          // [limbs] t0^, then the poly-0 accumulator / relinearised q_t limb
    u64* T1 = S + (size_t)limbs * N;      // [limbs] t1^, likewise for poly 1
    u64* T2 = S + (size_t)2 * limbs * N;  // [limbs] d1^, then t2 in the coefficient domain
    u64* AP = S + (size_t)3 * limbs * N;  // [2] accumulators modulo P, then their inverse transforms
    const u64 P = a.rns.q[L];
    const u64 halfP = (P - 1) / 2;
    // The transforms of one pixel in order, one word each: kind (bits 0-1), polynomial (2), limb
    // or digit (3-6), target modulus (7-10, 15 = P), barrier before the transform (11), first
    // term of the P accumulators (12). A barrier is needed only between two transforms of the
    // same direction (see above).
    if (tid == 0) {
        int n = 0;
        auto push = [&](u32 kind, u32 pb, u32 x, u32 mm, u32 bar, u32 first) {
            sched[n++] = kind | (pb << 2) | (x << 3) | (mm << 7) | (bar << 11) | (first << 12);
        };
        for (int l = 0; l < limbs; ++l) {
            push(kFwdDiff, 0, l, 0, 0, 0);
            push(kFwdDiff, 1, l, 0, 1, 0);
            push(kInvT2, 0, l, 0, 0, 0);
        }
        for (int step = 0; step <= limbs; ++step) {
            const int m = step == 0 ? -1 : (step == 1 ? t : step - 2);
            const u32 mm = m < 0 ? 15u : (u32)m;
            bool first = true;
            for (int j = 0; j < limbs; ++j) {
                if (j == m) continue;   // digit m's term went in with t_b^ in the first phase
                push(kFwdDigit, 0, j, mm, first ? 0 : 1, m < 0 && j == 0 ? 1 : 0);
                first = false;
            }
            push(kInvAcc, 0, 0, mm, 0, 0);
            push(kInvAcc, 1, 0, mm, 1, 0);
        }
    }
    __syncthreads();
    const int n_ops = limbs * limbs + 5 * limbs + 2;
    for (u64 k = blockIdx.x; k < a.n_ct; k += gridDim.x) {
        const u64* A = a.a + k * 2 * (u64)limbs * N;
        const u64* B = a.b + k * 2 * (u64)limbs * N;
        u64 r[1][E];
#pragma unroll 1
        for (int op = 0; op < n_ops; ++op) {
            const u32 code = sched[op];
            const u32 kind = code & 3u;
            const int pb = (int)((code >> 2) & 1u), x = (int)((code >> 3) & 15u);
            const int m = ((code >> 7) & 15u) == 15u ? -1 : (int)((code >> 7) & 15u);
            const int mod = kind == kFwdDiff || kind == kInvT2 ? x : (m < 0 ? L : m);
            const u64 q = a.rns.q[mod];
            if (kind == kFwdDiff || kind == kFwdDigit) {
                if (kind == kFwdDiff) {   // d = a - b, polynomial pb of limb x
                    const u64* pa = A + ((u64)pb * limbs + x) * N;
                    const u64* pq = B + ((u64)pb * limbs + x) * N;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int xi = elem_index<LOGN, 0, E>(tid, e);
                        r[0][e] = sub_mod(__ldcs(pa + xi), __ldcs(pq + xi), q);
                    }
                } else {                  // digit x of t2, centered, lifted to the modulus
                    const u64 mu = a.rns.mu[mod];
                    const u64 qj = a.rns.q[x];
                    const u64 half = (qj - 1) / 2;
                    const u64* t2 = T2 + (size_t)x * N;
                    if (qj <= q) {        // |digit| < q_j / 2 < q: no reduction
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            const u64 v = t2[e * T];
                            r[0][e] = v <= half ? v : q - (qj - v);
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            const u64 v = t2[e * T];
                            if (v <= half) {
                                r[0][e] = reduce64(v, q, mu);
                            } else {
                                const u64 mag = reduce64(qj - v, q, mu);
                                r[0][e] = mag == 0 ? 0 : q - mag;
                            }
                        }
                    }
                }
                if ((code >> 11) & 1u) __syncthreads();
                ntt_fwd_regs<LOGN, 1, false, CMP, E>(sm, r, tid, a.rns.tab[mod], q);
                if (kind == kFwdDiff) {
                    u64* dst = (pb == 0 ? T0 : T2) + (size_t)x * N;
#pragma unroll
                    for (int e = 0; e < E; ++e) dst[e * T] = csub(csub(r[0][e], 2 * q), q);
                } else {                  // acc_b(m) += NTT(digit) * evk^_x[b][m]
                    u64* acc0 = m < 0 ? AP : T0 + (size_t)m * N;
                    u64* acc1 = m < 0 ? AP + N : T1 + (size_t)m * N;
                    const bool init = (code >> 12) & 1u;
                    const u64* e0 = a.evk_hat + (((size_t)x * 2 + 0) * (L + 1) + mod) * N;
                    const u64* e0p = a.evk_hat_p + (((size_t)x * 2 + 0) * (L + 1) + mod) * N;
                    const u64* e1 = a.evk_hat + (((size_t)x * 2 + 1) * (L + 1) + mod) * N;
                    const u64* e1p = a.evk_hat_p + (((size_t)x * 2 + 1) * (L + 1) + mod) * N;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int xi = elem_index<LOGN, LAST, E, WT>(tid, e);
                        // the accumulators stay in [0, 2q): the inverse transform takes that range
                        const u64 d = csub(csub(r[0][e], 2 * q), q);
                        const u64 p0 = shoup_lazy(d, __ldg(e0 + xi), __ldg(e0p + xi), q);
                        const u64 p1 = shoup_lazy(d, __ldg(e1 + xi), __ldg(e1p + xi), q);
                        const u64 s0 = init ? 0 : acc0[e * T];
                        const u64 s1 = init ? 0 : acc1[e * T];
                        acc0[e * T] = csub(s0 + p0, 2 * q);
                        acc1[e * T] = csub(s1 + p1, 2 * q);
                    }
                }
            } else {
                if (kind == kInvT2) {     // the tensor of limb x; t2 = INTT(d1^2) next
                    u64* t0 = T0 + (size_t)x * N;
                    u64* t1 = T1 + (size_t)x * N;
                    const u64* t2 = T2 + (size_t)x * N;
                    const u64 qinv = a.rns.qinv[x];   // Montgomery products: 2^64 is folded into ninv, pn and r64
                    const u64* e0 = a.evk_hat + (((size_t)x * 2 + 0) * (L + 1) + x) * N;
                    const u64* e0p = a.evk_hat_p + (((size_t)x * 2 + 0) * (L + 1) + x) * N;
                    const u64* e1 = a.evk_hat + (((size_t)x * 2 + 1) * (L + 1) + x) * N;
                    const u64* e1p = a.evk_hat_p + (((size_t)x * 2 + 1) * (L + 1) + x) * N;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int xi = elem_index<LOGN, LAST, E, WT>(tid, e);
                        const u64 d0 = t0[e * T], d1 = t2[e * T];
                        const u64 m2 = mont_mul(d1, d1, q, qinv);
                        const u64 th = shoup(m2, a.r64[x], a.r64_p[x], q);   // d1^2, the transform of digit x
                        const u64 c = mont_mul(d0, d1, q, qinv);
                        t0[e * T] = csub(shoup_lazy(mont_mul(d0, d0, q, qinv), a.pn[x], a.pn_p[x], q) +
                                         shoup_lazy(th, __ldg(e0 + xi), __ldg(e0p + xi), q), 2 * q);
                        t1[e * T] = csub(shoup_lazy(add_mod(c, c, q), a.pn[x], a.pn_p[x], q) +
                                         shoup_lazy(th, __ldg(e1 + xi), __ldg(e1p + xi), q), 2 * q);
                        r[0][e] = shoup(m2, a.ninv[x], a.ninv_p[x], q);
                    }
                } else {
                    const u64* acc = (m < 0 ? AP + (size_t)pb * N : (pb == 0 ? T0 : T1) + (size_t)m * N);
#pragma unroll
                    for (int e = 0; e < E; ++e) r[0][e] = acc[e * T];
                }
                if ((code >> 11) & 1u) __syncthreads();
                ntt_inv_regs<LOGN, 1, CMP, E>(sm, r, tid, a.rns.tab[mod], q);
                if (kind == kInvT2) {
                    u64* t2 = T2 + (size_t)x * N;
#pragma unroll
                    for (int e = 0; e < E; ++e) t2[e * T] = csub(r[0][e], q);
                } else if (m < 0) {
                    u64* acc = AP + (size_t)pb * N;
#pragma unroll
                    for (int e = 0; e < E; ++e) acc[e * T] = csub(r[0][e], q);
                } else {
                    const u64 mu = a.rns.mu[mod];
                    u64* acc = (pb == 0 ? T0 : T1) + (size_t)m * N;
                    const u64* last = (pb == 0 ? T0 : T1) + (size_t)t * N;
                    u64* o = a.out + ((k * 2 + pb) * (u64)t + m) * N;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const u64 ap = AP[(size_t)pb * N + e * T];
                        u64 lp = reduce64(ap, q, mu);
                        if (ap > halfP) lp = add_mod(lp, a.neg_p_mod[m], q);   // (ap - P) mod q_m
                        const u64 md = shoup(sub_mod(csub(r[0][e], q), lp, q), a.p_inv[m], a.p_inv_p[m], q);
                        if (m == t) {
                            acc[e * T] = md;              // relinearised limb q_t, the rescale's divisor
                        } else {
                            const u64 ct = last[e * T];
                            const u64 u = shoup_lazy(md, a.qt_inv[m], a.qt_inv_p[m], q);
                            const u64 w = shoup_lazy(ct, a.qt_inv[m], a.qt_inv_p[m], q);
                            u64 v = csub(csub(u + 2 * q - w, 2 * q), q);
                            if (ct > a.half_qt) v = add_mod(v, 1, q);
                            __stcs(o + elem_index<LOGN, 0, E>(tid, e), v);
                        }
                    }
                }
            }
        }
    }
}

size_t sqdiff_image_scratch_words(int logn, int limbs) { return (size_t)(3 * limbs + 2) << logn; }

// Residues per thread: 8 up to N = 2^13 (twice the warps of the 16-residue layout hide the
// latency of the scratch and key loads), 16 at N = 2^14 (thread limit).
template <int LOGN>
static constexpr int kSqImgE = LOGN <= 13 ? 8 : 16;

template <int LOGN>
static size_t sqimg_smem() { return (sizeof(u64) << LOGN) + 128 * sizeof(u32); }   // + the schedule

template <int LOGN>
static cudaError_t sqimg_prepare(int* blocks_per_sm)
{
    auto kern = k_sqdiff_image<LOGN, kSqImgE<LOGN>>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sqimg_smem<LOGN>());
    if (e != cudaSuccess) return e;
    if (blocks_per_sm)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, NttShape<LOGN, kSqImgE<LOGN>>::T,
                                                          sqimg_smem<LOGN>());
    return e;
}

static cudaError_t sqimg_prepare_any(int logn, int* blocks_per_sm)
{
    switch (logn) {
    case 10: return sqimg_prepare<10>(blocks_per_sm);
    case 11: return sqimg_prepare<11>(blocks_per_sm);
    case 12: return sqimg_prepare<12>(blocks_per_sm);
    case 13: return sqimg_prepare<13>(blocks_per_sm);
    case 14: return sqimg_prepare<14>(blocks_per_sm);
    default: return cudaErrorInvalidValue;
    }
}

int sqdiff_image_grid(int logn, u64 n_ct, int num_sms)
{
    int per_sm = 0;
    if (sqimg_prepare_any(logn, &per_sm) != cudaSuccess || per_sm < 1) per_sm = 1;
    const u64 cap = (u64)num_sms * per_sm;
    return (int)(n_ct < cap ? n_ct : cap);
}

template <int LOGN>
static void sqimg_launch(const SqImgArgs& a, int grid, cudaStream_t st)
{
    k_sqdiff_image<LOGN, kSqImgE<LOGN>><<<grid, NttShape<LOGN, kSqImgE<LOGN>>::T, sqimg_smem<LOGN>(), st>>>(a);
}

cudaError_t launch_sqdiff_image(const SqImgArgs& a, int grid, cudaStream_t st)
{
    if (grid <= 0 || a.n_ct == 0) return cudaSuccess;
    cudaError_t e = sqimg_prepare_any(a.rns.logn, nullptr);
    if (e != cudaSuccess) return e;
    switch (a.rns.logn) {
    case 10: sqimg_launch<10>(a, grid, st); break;
    case 11: sqimg_launch<11>(a, grid, st); break;
    case 12: sqimg_launch<12>(a, grid, st); break;
    case 13: sqimg_launch<13>(a, grid, st); break;
    case 14: sqimg_launch<14>(a, grid, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Relinearisation by hybrid key switching with one special prime P, one digit per ciphertext
// prime, mod-down with centered rounding.
// ---------------------------------------------------------------------------------------

__global__ void k_relin_digits(const __grid_constant__ RelinArgs a, const u64* d2, u64* digits)
{
    const int n = 1 << a.rns.logn;
    const int nm = a.limbs + 1;
    const int jm = blockIdx.y;                 // j * nm + m
    const int j = jm / nm, m = jm % nm;
    const int mod = m < a.limbs ? m : a.L;     // index into the moduli (P at index L)
    const u64 qj = a.rns.q[j], qm = a.rns.q[mod];
    const u64 half = (qj - 1) / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const u64 v = d2[(size_t)j * n + i];
        u64 out;
        if (v <= half) {
            out = reduce64(v, qm, a.mu[mod]);
        } else {
            const u64 mag = reduce64(qj - v, qm, a.mu[mod]);
            out = mag == 0 ? 0 : qm - mag;
        }
        digits[(size_t)jm * n + i] = out;
    }
}

cudaError_t launch_relin_digits(const RelinArgs& a, const u64* d2, u64* digits, cudaStream_t st)
{
    dim3 grid((1u << a.rns.logn) / 256, a.limbs * (a.limbs + 1));
    k_relin_digits<<<grid, 256, 0, st>>>(a, d2, digits);
    return cudaGetLastError();
}

__global__ void k_relin_mac(const __grid_constant__ RelinArgs a, const u64* digits_hat, u64* acc)
{
    const int n = 1 << a.rns.logn;
    const int nm = a.limbs + 1;
    const int bm = blockIdx.y;                 // b * nm + m
    const int b = bm / nm, m = bm % nm;
    const int mod = m < a.limbs ? m : a.L;
    const u64 q = a.rns.q[mod];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        u64 s = 0;
        for (int j = 0; j < a.limbs; ++j) {
            const size_t ko = (((size_t)j * 2 + b) * (a.L + 1) + mod) * n + i;
            const u64 d = digits_hat[((size_t)j * nm + m) * n + i];
            s = add_mod(s, shoup(d, a.evk_hat[ko], a.evk_hat_p[ko], q), q);
        }
        acc[(size_t)bm * n + i] = s;
    }
}

cudaError_t launch_relin_mac(const RelinArgs& a, const u64* digits_hat, u64* acc, cudaStream_t st)
{
    dim3 grid((1u << a.rns.logn) / 256, 2 * (a.limbs + 1));
    k_relin_mac<<<grid, 256, 0, st>>>(a, digits_hat, acc);
    return cudaGetLastError();
}

__global__ void k_relin_moddown(const __grid_constant__ RelinArgs a, const u64* d01, const u64* acc, u64* out)
{
    const int n = 1 << a.rns.logn;
    const int nm = a.limbs + 1;
    const int bj = blockIdx.y;                 // b * limbs + j
    const int b = bj / a.limbs, j = bj % a.limbs;
    const u64 qj = a.rns.q[j];
    const u64 P = a.rns.q[a.L];
    const u64 halfP = (P - 1) / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const u64 ap = acc[((size_t)b * nm + a.limbs) * n + i];
        u64 r = reduce64(ap, qj, a.mu[j]);
        if (ap > halfP) r = add_mod(r, a.neg_p_mod[j], qj);   // (acc_P - P) mod q_j
        const u64 aj = acc[((size_t)b * nm + j) * n + i];
        const u64 ks = shoup(sub_mod(aj, r, qj), a.p_inv[j], a.p_inv_p[j], qj);
        out[(size_t)bj * n + i] = add_mod(d01[(size_t)bj * n + i], ks, qj);
    }
}

cudaError_t launch_relin_moddown(const RelinArgs& a, const u64* d01, const u64* acc, u64* out, cudaStream_t st)
{
    dim3 grid((1u << a.rns.logn) / 256, 2 * a.limbs);
    k_relin_moddown<<<grid, 256, 0, st>>>(a, d01, acc, out);
    return cudaGetLastError();
}

}  // namespace ichee
