// kernels_ops.cu -- ciphertext-wise image operations (Sec. 2.2.3, Sec. 4.4) and decryption
// (Sec. 2.2.2). Ciphertexts are [n_ct][2][limbs][N] residues in the coefficient domain.
#include "ops.h"
#include "bulk.cuh"
#include <cstring>

namespace ichee {

// ---------------------------------------------------------------------------------------
// Rescale by the last prime q_t of a ciphertext with t+1 limbs (Sec. 2.2.3, rounding to
// nearest):
//   c'_j = (c_j - [c_t]_centered) * q_t^{-1} mod q_j, [x]_centered in (-q_t/2, q_t/2].
// Since q_t * q_t^{-1} = 1 mod q_j this is c_j q_t^{-1} - c_t q_t^{-1} + [c_t > (q_t-1)/2]:
// two Shoup products (both accept any 64-bit operand, so c_t needs no reduction mod q_j).
// A constant K multiplied in before the rescale folds into the first product as
// K q_t^{-1} mod q_j.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ u64 rescale_fold(u64 prod_j, u64 ct, int j, const OpsArgs& a)
{
    // prod_j in [0, 2 q_j): the already scaled c_j q_t^{-1} (or sum K c_j q_t^{-1})
    const u64 qj = a.q[j];
    const u64 b = shoup_lazy(ct, a.qt_inv[j], a.qt_inv_p[j], qj);
    u64 v = csub(csub(prod_j + 2 * qj - b, 2 * qj), qj);
    return ct > a.half_qt ? add_mod(v, 1, qj) : v;
}

__device__ __forceinline__ u64 rescale_one(u64 cj, u64 ct, int j, const OpsArgs& a)
{
    return rescale_fold(shoup_lazy(cj, a.qt_inv[j], a.qt_inv_p[j], a.q[j]), ct, j, a);
}

// Fused multiply by K and rescale when K is one integer with 4K below every modulus
// (a.k0_same). Let S' = S_t - c q_t (S_t a sum of at most nine residues, below 9 q_t; S' below
// 4 q_t) and K S' = u q_t + m with m centered in (-q_t/2, q_t/2]. Then
//   (K S_j - m) q_t^{-1} = K q_t^{-1} (S_j - S') + u  (mod q_j),
// the rescale of K S, with one Shoup product per kept limb instead of two: the quotient u comes
// with the product on limb t (Shoup's quotient is exact up to one for any 64-bit operand), and
// u <= 4K < q_j.
struct RescaleQuot {
    u64 s;   // S_t reduced below 4 q_t
    u64 u;   // rounded quotient of K S' by q_t
};

__device__ __forceinline__ RescaleQuot rescale_quot(u64 st, const OpsArgs& a, int t)
{
    const u64 q = a.q[t];
    st = st >= 8 * q ? st - 8 * q : st;
    st = st >= 4 * q ? st - 4 * q : st;
    u64 hi = mulhi(st, a.k0p[t]);
    u64 r = st * a.k0[t] - hi * q;   // in [0, 2q): K S' = hi q + r
    if (r >= q) { r -= q; hi += 1; }
    return {st, hi + (r > a.half_qt ? 1 : 0)};
}

// Limb j < t of Rescale(K * S) from the unreduced sum S_j (below 9 q_j) and rescale_quot's
// result; mq[j] is a multiple of q_j of at least 4 q_t, and S_j + mq[j] - S' < 14 * 2^60.
__device__ __forceinline__ u64 rescale_quot_limb(u64 sj, const RescaleQuot& rq, int j, const OpsArgs& a)
{
    const u64 qj = a.q[j];
    u64 v = shoup_lazy(sj + a.mq[j] - rq.s, a.k0r[j], a.k0rp[j], qj) + rq.u;   // in [0, 3 q_j)
    v = v >= 2 * qj ? v - 2 * qj : v;
    return v >= qj ? v - qj : v;
}

// Elementwise add / sub of two images with the same shape (Sec. 2.2.3, Sec. 3.3).
__global__ void k_addsub(const __grid_constant__ OpsArgs a, int subtract)
{
    const int n = 1 << a.logn;
    const u64 total2 = a.n_ct * (u64)(2 * a.limbs) * (n / 2);
    const ulonglong2* x = reinterpret_cast<const ulonglong2*>(a.in0);
    const ulonglong2* y = reinterpret_cast<const ulonglong2*>(a.in1);
    ulonglong2* o = reinterpret_cast<ulonglong2*>(a.out);
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total2; i += (u64)gridDim.x * blockDim.x) {
        const int l = (int)((i / (n / 2)) % a.limbs);
        const u64 q = a.q[l];
        ulonglong2 u = __ldcs(x + i), v = __ldcs(y + i);
        if (subtract) { u.x = sub_mod(u.x, v.x, q); u.y = sub_mod(u.y, v.y, q); }
        else { u.x = add_mod(u.x, v.x, q); u.y = add_mod(u.y, v.y, q); }
        __stcs(o + i, u);
    }
}

// Plaintext constant add (brightness, Sec. 4.4.2; watermark pixel, Sec. 4.4.4): the encoded
// constant touches coefficient 0 of c0 only. The residue added to limb l of ciphertext k is
// kadd[k * limbs + l] (one constant per ciphertext) or k0[l] (one for all); only ciphertexts
// in [k_lo, k_hi) change. With in0 != out the whole image is
// copied first.
__global__ void k_ptadd_copy(const __grid_constant__ OpsArgs a)
{
    const int n = 1 << a.logn;
    const u64 total2 = a.n_ct * (u64)(2 * a.limbs) * (n / 2);
    const ulonglong2* x = reinterpret_cast<const ulonglong2*>(a.in0);
    ulonglong2* o = reinterpret_cast<ulonglong2*>(a.out);
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total2; i += (u64)gridDim.x * blockDim.x) {
        ulonglong2 u = __ldcs(x + i);
        const u64 row = i / (n / 2);               // (k * 2 + b) * limbs + l
        const u64 within = i % (n / 2);
        const int l = (int)(row % a.limbs);
        const u64 kb = row / a.limbs;
        const u64 k = kb / 2;
        if (within == 0 && (kb & 1) == 0 && k >= a.k_lo && k < a.k_hi)
            u.x = add_mod(u.x, a.kadd_per_ct ? a.kadd[k * a.limbs + l] : a.k0[l], a.q[l]);
        __stcs(o + i, u);
    }
}

__global__ void k_ptadd_inplace(const __grid_constant__ OpsArgs a)
{
    const int n = 1 << a.logn;
    const u64 cnt = (a.k_hi - a.k_lo) * (u64)a.limbs;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < cnt; i += (u64)gridDim.x * blockDim.x) {
        const u64 k = a.k_lo + i / a.limbs;
        const int l = (int)(i % a.limbs);
        u64* c = a.out + ((k * 2) * a.limbs + l) * (u64)n;
        *c = add_mod(*c, a.kadd_per_ct ? a.kadd[k * a.limbs + l] : a.k0[l], a.q[l]);
    }
}

// Plaintext constant multiply: every residue times the encoded constant (Shoup).
__global__ void k_ptmul(const __grid_constant__ OpsArgs a)
{
    const int n = 1 << a.logn;
    const u64 total2 = a.n_ct * (u64)(2 * a.limbs) * (n / 2);
    const ulonglong2* x = reinterpret_cast<const ulonglong2*>(a.in0);
    ulonglong2* o = reinterpret_cast<ulonglong2*>(a.out);
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total2; i += (u64)gridDim.x * blockDim.x) {
        const int l = (int)((i / (n / 2)) % a.limbs);
        const u64 q = a.q[l];
        ulonglong2 u = __ldcs(x + i);
        u.x = shoup(u.x, a.k0[l], a.k0p[l], q);
        u.y = shoup(u.y, a.k0[l], a.k0p[l], q);
        __stcs(o + i, u);
    }
}

// Rescale of a whole image: output has limbs-1 limbs. One thread per (ct, poly, coefficient
// pair), all limbs.
template <int LIMBS>
__global__ void k_rescale(const __grid_constant__ OpsArgs a)
{
    const int n = 1 << a.logn;
    const u64 total = a.n_ct * 2 * (u64)(n / 2);
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total; i += (u64)gridDim.x * blockDim.x) {
        const u64 kb = i / (n / 2);
        const int c = (int)(i % (n / 2));
        const ulonglong2* src = reinterpret_cast<const ulonglong2*>(a.in0 + kb * LIMBS * (u64)n) + c;
        ulonglong2* dst = reinterpret_cast<ulonglong2*>(a.out + kb * (LIMBS - 1) * (u64)n) + c;
        const ulonglong2 last = __ldcs(src + (LIMBS - 1) * (n / 2));
#pragma unroll
        for (int j = 0; j < LIMBS - 1; ++j) {
            ulonglong2 v = __ldcs(src + j * (n / 2));
            v.x = rescale_one(v.x, last.x, j, a);
            v.y = rescale_one(v.y, last.y, j, a);
            __stcs(dst + j * (n / 2), v);
        }
    }
}

// One output pair of the mean filter from the three column sums of its window (each the sum of
// three rows, unreduced): fused multiply by K9 and rescale, stored to o[j * half] per kept limb.
template <int LIMBS>
__device__ __forceinline__ void mf_store(const OpsArgs& a, const ulonglong2 (&cl)[LIMBS], const ulonglong2 (&cm)[LIMBS],
                                         const ulonglong2 (&cr)[LIMBS], ulonglong2* o, int half)
{
    const u64 qt = a.q[LIMBS - 1];
    const u64 sx = cl[LIMBS - 1].x + cm[LIMBS - 1].x + cr[LIMBS - 1].x;
    const u64 sy = cl[LIMBS - 1].y + cm[LIMBS - 1].y + cr[LIMBS - 1].y;
    if (a.k0_same) {
        const RescaleQuot rx = rescale_quot(sx, a, LIMBS - 1), ry = rescale_quot(sy, a, LIMBS - 1);
#pragma unroll
        for (int j = 0; j < LIMBS - 1; ++j) {
            ulonglong2 v;
            v.x = rescale_quot_limb(cl[j].x + cm[j].x + cr[j].x, rx, j, a);
            v.y = rescale_quot_limb(cl[j].y + cm[j].y + cr[j].y, ry, j, a);
            __stcs(o + j * half, v);
        }
    } else {
        const u64 tx = shoup(sx, a.k0[LIMBS - 1], a.k0p[LIMBS - 1], qt);
        const u64 ty = shoup(sy, a.k0[LIMBS - 1], a.k0p[LIMBS - 1], qt);
#pragma unroll
        for (int j = 0; j < LIMBS - 1; ++j) {
            const u64 qj = a.q[j];
            ulonglong2 v;
            v.x = rescale_fold(shoup_lazy(cl[j].x + cm[j].x + cr[j].x, a.k0r[j], a.k0rp[j], qj), tx, j, a);
            v.y = rescale_fold(shoup_lazy(cl[j].y + cm[j].y + cr[j].y, a.k0r[j], a.k0rp[j], qj), ty, j, a);
            __stcs(o + j * half, v);
        }
    }
}

// Fused 3x3 mean filter (Sec. 4.4.1; borders clamp to the edge): out(y,x) = Rescale(K9 * sum of the 9
// clamp-to-edge neighbours). One block per (row y, channel, poly, coefficient chunk); each
// thread owns one coefficient pair and walks the row left to right keeping the three column
// sums of the window in registers, so every input row is loaded once per output row. Residues
// are below 2^60, so the 9-term sums fit 64 bits unreduced and go straight into the Shoup
// products (K9 for the dropped limb, K9 q_t^{-1} for the kept ones).
// in0 holds the image's rows from row0 on, out0 its output rows from yout0 on (0 and 0 for a
// whole image); h is the height of the whole image (the clamping rows).
template <int LIMBS>
__device__ __forceinline__ void meanfilter_row(const OpsArgs& a, const u64* in0, u64* out0, int h, int w, int C, int y,
                                               int chunk, int b, int ch, int row0 = 0, int yout0 = 0)
{
    const int n = 1 << a.logn;
    const int c2 = chunk * blockDim.x + threadIdx.x;  // coefficient-pair index
    const u64 ct_len2 = (u64)2 * LIMBS * (n / 2);
    const u64 out_len2 = (u64)2 * (LIMBS - 1) * (n / 2);
    const ulonglong2* in = reinterpret_cast<const ulonglong2*>(in0) + (u64)b * LIMBS * (n / 2) + c2;
    ulonglong2* out = reinterpret_cast<ulonglong2*>(out0) + (u64)b * (LIMBS - 1) * (n / 2) + c2;
    const int ym = y > 0 ? y - 1 : 0, yp = y + 1 < h ? y + 1 : h - 1;
    const int half = n / 2;
    // the three input rows at column 0 and the output row at column 0; one column further is a
    // fixed stride of C ciphertexts (pointer adds, no per-column 64-bit products)
    const ulonglong2* r0 = in + ((u64)(ym - row0) * w * C + ch) * ct_len2;
    const ulonglong2* r1 = in + ((u64)(y - row0) * w * C + ch) * ct_len2;
    const ulonglong2* r2 = in + ((u64)(yp - row0) * w * C + ch) * ct_len2;
    const u64 in_step = (u64)C * ct_len2;
    ulonglong2* o = out + ((u64)(y - yout0) * w * C + ch) * out_len2;
    const u64 out_step = (u64)C * out_len2;

    ulonglong2 col[3][LIMBS];
    auto column = [&](int xx, ulonglong2 (&dst)[LIMBS]) {
        const u64 off = (u64)xx * in_step;
#pragma unroll
        for (int l = 0; l < LIMBS; ++l) {
            ulonglong2 v0 = __ldg(r0 + off + l * half);
            ulonglong2 v1 = __ldg(r1 + off + l * half);
            ulonglong2 v2 = __ldg(r2 + off + l * half);
            dst[l].x = v0.x + v1.x + v2.x;
            dst[l].y = v0.y + v1.y + v2.y;
        }
    };
    column(0, col[0]);  // x = -1 clamps to 0
#pragma unroll
    for (int l = 0; l < LIMBS; ++l) col[1][l] = col[0][l];
    column(w > 1 ? 1 : 0, col[2]);
    for (int x = 0; x < w; ++x, o += out_step) {
        mf_store<LIMBS>(a, col[0], col[1], col[2], o, half);
        if (x + 1 < w) {
#pragma unroll
            for (int l = 0; l < LIMBS; ++l) { col[0][l] = col[1][l]; col[1][l] = col[2][l]; }
            column(x + 2 < w ? x + 2 : w - 1, col[2]);
        }
    }
}

// Status word value written when a bounded wait of a kernel gives up.
constexpr int kStatusWaitTimeout = 0x5701;

// The same row walk with the input columns staged in shared memory by bulk copies: for each
// column of the row, one thread copies the three input rows' segments of every limb (T
// coefficient pairs, T x 16 bytes each) into one of two stages, two columns ahead of the
// threads that sum them, so the block keeps two columns of loads in flight without holding them
// in registers. `gc` counts the columns the block has consumed (stage = count mod 2, barrier
// phase = count / 2). Returns false, with every thread, if a wait gave up (the status word is
// set and the copies still in flight are waited for, within the bound).
constexpr int kMfStages = 2;

template <int LIMBS>
__device__ __forceinline__ bool meanfilter_row_staged(const OpsArgs& a, const u64* in0, u64* out0, int h, int w, int C,
                                                      int y, int chunk, int b, int ch, int row0, int yout0,
                                                      ulonglong2* stages, u64* bars, u32& gc)
{
    const int T = blockDim.x, tid = threadIdx.x;
    const int half = (1 << a.logn) / 2;
    const u64 ct_len2 = (u64)2 * LIMBS * half;
    const u64 out_len2 = (u64)2 * (LIMBS - 1) * half;
    const int ym = y > 0 ? y - 1 : 0, yp = y + 1 < h ? y + 1 : h - 1;
    const ulonglong2* in = reinterpret_cast<const ulonglong2*>(in0) + (u64)b * LIMBS * half + (u64)chunk * T;
    const ulonglong2* src[3] = {in + ((u64)(ym - row0) * w * C + ch) * ct_len2,
                                in + ((u64)(y - row0) * w * C + ch) * ct_len2,
                                in + ((u64)(yp - row0) * w * C + ch) * ct_len2};
    const u64 in_step = (u64)C * ct_len2;
    const u32 seg_bytes = (u32)T * 16u;
    const int stage_u2 = 3 * LIMBS * T;
    ulonglong2* o = reinterpret_cast<ulonglong2*>(out0) + (u64)b * (LIMBS - 1) * half + (u64)chunk * T + tid +
                    ((u64)(y - yout0) * w * C + ch) * out_len2;
    const u64 out_step = (u64)C * out_len2;

    auto issue = [&](int j) {   // one thread: column j into its stage
        const u32 k = gc + (u32)j;
        u64* bar = bars + (k % kMfStages);
        ulonglong2* dst = stages + (k % kMfStages) * stage_u2;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, 3u * LIMBS * seg_bytes);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int l = 0; l < LIMBS; ++l)
                bulk_g2s(dst + (r * LIMBS + l) * T, src[r] + (u64)j * in_step + (u64)l * half, seg_bytes, bar);
    };
    auto give_up = [&](int j) {   // every thread returns; thread 0 drains the copies issued
        if (tid == 0) {
            atomicExch(a.status, kStatusWaitTimeout);
            for (int jj = j; jj < w && jj < j + kMfStages; ++jj) {
                const u32 k = gc + (u32)jj;
                mbar_wait(bars + (k % kMfStages), (k / kMfStages) & 1u);
            }
        }
        return false;
    };
    // column j's three-row sums for this thread; then the stage is refilled with column j + 2
    auto take = [&](int j, ulonglong2 (&cs)[LIMBS]) -> bool {
        const u32 k = gc + (u32)j;
        const bool ok = mbar_wait(bars + (k % kMfStages), (k / kMfStages) & 1u);
        if (ok) {
            const ulonglong2* sp = stages + (k % kMfStages) * stage_u2 + tid;
#pragma unroll
            for (int l = 0; l < LIMBS; ++l) {
                const ulonglong2 v0 = sp[l * T], v1 = sp[(LIMBS + l) * T], v2 = sp[(2 * LIMBS + l) * T];
                cs[l] = make_ulonglong2(v0.x + v1.x + v2.x, v0.y + v1.y + v2.y);
            }
        }
        if (__syncthreads_or(ok ? 0 : 1)) return false;   // the stage is free again
        if (tid == 0 && j + kMfStages < w) issue(j + kMfStages);
        return true;
    };

    if (tid == 0) {
        issue(0);
        if (w > 1) issue(1);
    }
    ulonglong2 cl[LIMBS], cm[LIMBS], cr[LIMBS];
    if (!take(0, cm)) return give_up(0);
#pragma unroll
    for (int l = 0; l < LIMBS; ++l) cl[l] = cm[l];   // x = -1 clamps to 0
    if (w > 1) {
        if (!take(1, cr)) return give_up(1);
    } else {
#pragma unroll
        for (int l = 0; l < LIMBS; ++l) cr[l] = cm[l];
    }
    for (int x = 0; x < w; ++x, o += out_step) {
        mf_store<LIMBS>(a, cl, cm, cr, o, half);
#pragma unroll
        for (int l = 0; l < LIMBS; ++l) { cl[l] = cm[l]; cm[l] = cr[l]; }
        if (x + 2 < w && !take(x + 2, cr)) return give_up(x + 2);   // else column w-1 stays on the right
    }
    gc += (u32)w;
    return true;
}

// Shared memory of the staged mean filter: two barriers (padded to 128 bytes), two stages.
__host__ __device__ constexpr size_t mf_staged_smem(int limbs, int threads)
{
    return 128 + (size_t)kMfStages * 3 * limbs * threads * 16;
}

__device__ __forceinline__ void mf_staged_setup(unsigned char* smraw, u64*& bars, ulonglong2*& stages)
{
    bars = reinterpret_cast<u64*>(smraw);
    stages = reinterpret_cast<ulonglong2*>(smraw + 128);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMfStages; ++s) mbar_init(bars + s, 1);
        mbar_init_fence();
    }
    __syncthreads();
}

// Persistent grid over the items (row, chunk, poly, channel) of one image.
template <int LIMBS>
__global__ void __launch_bounds__(256) k_meanfilter3_staged(const __grid_constant__ OpsArgs a)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    u64* bars;
    ulonglong2* stages;
    mf_staged_setup(smraw, bars, stages);
    const int chunks = ((1 << a.logn) / 2) / blockDim.x;
    const u64 items = (u64)a.rows * chunks * 2 * a.c;
    u32 gc = 0;
    for (u64 g = blockIdx.x; g < items; g += gridDim.x) {
        u64 bid = g;
        const int y = a.y0 + (int)(bid % a.rows); bid /= a.rows;
        const int chunk = (int)(bid % chunks); bid /= chunks;
        const int b = (int)(bid % 2); bid /= 2;
        if (!meanfilter_row_staged<LIMBS>(a, a.in0, a.out, a.h, a.w, a.c, y, chunk, b, (int)bid, a.row0, a.y0, stages,
                                          bars, gc))
            return;
    }
}

// Ragged batch, same items as k_meanfilter3_batch.
template <int LIMBS>
__global__ void __launch_bounds__(512) k_meanfilter3_staged_batch(const __grid_constant__ OpsArgs a,
                                                                  const __grid_constant__ SegTable t)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    u64* bars;
    ulonglong2* stages;
    mf_staged_setup(smraw, bars, stages);
    const int chunks = ((1 << a.logn) / 2) / blockDim.x;
    const u64 total = t.start[t.n];
    u32 gc = 0;
    for (u64 g = blockIdx.x; g < total; g += gridDim.x) {
        const int s = seg_of(t, g);
        u64 i = g - t.start[s];
        const int h = (int)t.h[s];
        const int y = (int)(i % h); i /= h;
        const int chunk = (int)(i % chunks); i /= chunks;
        const int b = (int)(i % 2); i /= 2;
        if (!meanfilter_row_staged<LIMBS>(a, t.in0[s], t.out[s], h, (int)t.w[s], (int)t.c[s], y, chunk, b, (int)i, 0, 0,
                                          stages, bars, gc))
            return;
    }
}

// One block per (row y, coefficient chunk, poly, channel); registers bounded so that three
// blocks (up to three limbs) or two share an SM.
template <int LIMBS>
static constexpr int kMfMinBlocks = LIMBS <= 3 ? 3 : 2;

template <int LIMBS>
__global__ void __launch_bounds__(256, kMfMinBlocks<LIMBS>) k_meanfilter3(const __grid_constant__ OpsArgs a)
{
    const int chunks = ((1 << a.logn) / 2) / blockDim.x;
    u64 bid = blockIdx.x;
    const int y = a.y0 + (int)(bid % a.rows); bid /= a.rows;
    const int chunk = (int)(bid % chunks); bid /= chunks;
    const int b = (int)(bid % 2); bid /= 2;
    meanfilter_row<LIMBS>(a, a.in0, a.out, a.h, a.w, a.c, y, chunk, b, (int)bid, a.row0, a.y0);
}

// Largest block of the batched mean-filter kernels for a limb count: the column sums of more
// than three limbs need more than the 64 registers a thread gets at 1024 threads.
template <int LIMBS>
static constexpr int kMfMaxThreads = LIMBS <= 3 ? 1024 : 512;

// Ragged batch: segment s has h*chunks*2*c items, in the order of the single-image kernel.
// Launched with at most 512 threads (the tunable shapes).
template <int LIMBS>
__global__ void __launch_bounds__(kMfMaxThreads<LIMBS>) k_meanfilter3_batch(const __grid_constant__ OpsArgs a,
                                                            const __grid_constant__ SegTable t)
{
    const int chunks = ((1 << a.logn) / 2) / blockDim.x;
    const u64 total = t.start[t.n];
    for (u64 g = blockIdx.x; g < total; g += gridDim.x) {
        const int s = seg_of(t, g);
        u64 i = g - t.start[s];
        const int h = (int)t.h[s];
        const int rows = t.rows[s] ? (int)t.rows[s] : h;
        const int y = (int)t.y0[s] + (int)(i % rows); i /= rows;
        const int chunk = (int)(i % chunks); i /= chunks;
        const int b = (int)(i % 2); i /= 2;
        meanfilter_row<LIMBS>(a, t.in0[s], t.out[s], h, (int)t.w[s], (int)t.c[s], y, chunk, b, (int)i, (int)t.row0[s],
                              (int)t.y0[s]);
    }
}

// Fused radix encryption + 3x3 mean filter (Sec. 3.2, 3.3 and 4.4.1) for a ragged batch. Each
// item is a strip of columns of one image for one polynomial, channel and 32 coefficient
// pairs: lane = coefficient pair (coalesced 512-byte accesses), warp = column. Every warp walks
// its column from top to bottom, rebuilding each pixel's ciphertext once from the
// L2-resident cached multiples d * Enc(r^k) (signed digits with the pixel's randomness bits,
// and the pair table of the top two positions when the cache has one, as in the radix
// combine) and writing it as the encryption output. The vertical 3-sums come
// from two running sums in registers (S1 = row y, S2 = rows y-1 + y); the horizontal 3-sum from
// the neighbouring warps through shared memory (double-buffered: one barrier per row). The
// strip's first and last warps are halo columns (clamped at the image border) whose outputs
// belong to the neighbouring strips. Sums stay unreduced (at most 9 residues below 2^60) up to
// the fused multiply + rescale, as in the mean filter. Residues equal those of the radix
// combine followed by the mean filter.
template <int LIMBS>
__global__ void __launch_bounds__(kMfMaxThreads<LIMBS>) k_radix_meanfilter3_batch(const __grid_constant__ RadixArgs ra,
                                                                  const __grid_constant__ OpsArgs a,
                                                                  const __grid_constant__ SegTable t)
{
    extern __shared__ ulonglong2 vbuf[];   // [2][cols][LIMBS][32]: vertical sums of one row
    const int half = (1 << a.logn) / 2;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int cols = blockDim.x >> 5;
    const int pchunks = half / 32;
    const int width = 2 * ra.r + 1;
    const size_t ct_u2 = (size_t)2 * LIMBS * half;          // one ciphertext, in coefficient pairs
    const size_t out_u2 = (size_t)2 * (LIMBS - 1) * half;
    const ulonglong2* mult = reinterpret_cast<const ulonglong2*>(ra.mult);
    const u64 total = t.start[t.n];
    for (u64 g = blockIdx.x; g < total; g += gridDim.x) {
        const int s = seg_of(t, g);
        u64 i = g - t.start[s];
        const int h = (int)t.h[s], w = (int)t.w[s], C = (int)t.c[s];
        const int strips = (w + cols - 3) / (cols - 2);
        const int strip = (int)(i % strips); i /= strips;
        const int pc = (int)(i % pchunks); i /= pchunks;
        const int b = (int)(i % 2); i /= 2;
        const int ch = (int)i;
        const int xr = strip * (cols - 2) - 1 + wi;
        const int x = xr < 0 ? 0 : (xr >= w ? w - 1 : xr);
        const bool owned = wi >= 1 && wi <= cols - 2 && xr < w;
        const int c2 = pc * 32 + lane;
        const uint8_t* px = t.px[s];
        const u64 seed = t.seed[s];
        // this thread's coefficient pair in pixel (0, x) of each output; one row further is
        // a fixed stride (no per-row 64-bit products on the multiply pipe)
        const size_t row_px = (size_t)w * C;
        ulonglong2* enc = reinterpret_cast<ulonglong2*>(t.out[s]) + (size_t)b * LIMBS * half + c2 +
                          ((size_t)x * C + ch) * ct_u2;
        ulonglong2* flt = reinterpret_cast<ulonglong2*>(t.out2[s]) + (size_t)b * (LIMBS - 1) * half + c2 +
                          ((size_t)x * C + ch) * out_u2;
        const size_t enc_row = row_px * ct_u2, flt_row = row_px * out_u2;
        const ulonglong2* mult_b = mult + (size_t)b * LIMBS * half + c2;
        const ulonglong2* pair_b =
            ra.pair_w ? reinterpret_cast<const ulonglong2*>(ra.pair) + (size_t)b * LIMBS * half + c2 : nullptr;
        // digit codes of this column, 32 rows at a time: lane j holds row code_base + j, one
        // byte per cached power (signed digit + r)
        u64 code = 0;
        int code_base = -64;
        auto code_of = [&](int yy) -> u64 {
            if (yy >= code_base + 32) {   // warp-uniform
                code_base = yy;
                code = 0;
                const int yl = yy + lane;
                if (yl < h) {
                    const u64 k = ((u64)yl * w + x) * C + ch;
                    int p = px[k];
                    const u32 bits = ra.randomize ? philox(seed, kStreamRadixBits, k, 0).w[0] : 0u;
                    for (int kk = 0; kk < ra.n_pow; ++kk) {
                        const int dk = p % ra.r;
                        p /= ra.r;
                        const int bk = (ra.randomize && kk >= 1) ? (int)((bits >> kk) & 1u) : 0;
                        const int bk1 = (ra.randomize && kk + 1 < ra.n_pow) ? (int)((bits >> (kk + 1)) & 1u) : 0;
                        code |= (u64)(dk + bk - ra.r * bk1 + ra.r) << (8 * kk);
                    }
                }
            }
            return __shfl_sync(0xffffffffu, code, yy - code_base);
        };
        auto rebuild = [&](int yy, ulonglong2 (&v)[LIMBS]) {
            const u64 cd = code_of(yy);
#pragma unroll
            for (int l = 0; l < LIMBS; ++l) v[l] = make_ulonglong2(0, 0);
            auto add_ct = [&](const ulonglong2* src) {
                ulonglong2 m[LIMBS];
#pragma unroll
                for (int l = 0; l < LIMBS; ++l) m[l] = __ldg(src + (size_t)l * half);
#pragma unroll
                for (int l = 0; l < LIMBS; ++l) {
                    v[l].x = add_mod(v[l].x, m[l].x, a.q[l]);
                    v[l].y = add_mod(v[l].y, m[l].y, a.q[l]);
                }
            };
            const int separate = ra.pair_w ? ra.n_pow - 2 : ra.n_pow;
            for (int kk = 0; kk < separate; ++kk) {
                const int dr = (int)((cd >> (8 * kk)) & 0xffu);
                // (kk * width + dr) < 8 * 33 and ct_u2 <= 2^17: the offset fits 32 bits
                if (dr != ra.r) add_ct(mult_b + (u32)(kk * width + dr) * (u32)ct_u2);
            }
            if (ra.pair_w) {   // the top two positions from the pair table: (2r+1) * pair_w < 8 * 33 entries
                const int dr = (int)((cd >> (8 * separate)) & 0xffu);
                const int dt = (int)((cd >> (8 * separate + 8)) & 0xffu) - ra.r;
                if (dr != ra.r || dt != 0) add_ct(pair_b + (u32)(dr * ra.pair_w + dt) * (u32)ct_u2);
            }
        };
        auto store_enc = [&](int yy, const ulonglong2 (&v)[LIMBS]) {
            ulonglong2* o = enc + (size_t)yy * enc_row;
#pragma unroll
            for (int l = 0; l < LIMBS; ++l) __stcs(o + (size_t)l * half, v[l]);
        };
        ulonglong2 S1[LIMBS], S2[LIMBS], nv[LIMBS];
        rebuild(0, S1);
        if (owned) store_enc(0, S1);
#pragma unroll
        for (int l = 0; l < LIMBS; ++l) S2[l] = make_ulonglong2(S1[l].x + S1[l].x, S1[l].y + S1[l].y);  // row -1 = row 0
        const u64 qt = a.q[LIMBS - 1];
        for (int y = 0; y < h; ++y) {
            const int yn = y + 1 < h ? y + 1 : h - 1;
            rebuild(yn, nv);
            if (owned && y + 1 < h) store_enc(y + 1, nv);
            ulonglong2* vb = vbuf + ((size_t)(y & 1) * cols + wi) * LIMBS * 32 + lane;
#pragma unroll
            for (int l = 0; l < LIMBS; ++l) {
                vb[l * 32] = make_ulonglong2(S2[l].x + nv[l].x, S2[l].y + nv[l].y);
                S2[l] = make_ulonglong2(S1[l].x + nv[l].x, S1[l].y + nv[l].y);
                S1[l] = nv[l];
            }
            __syncthreads();
            if (owned) {
                const ulonglong2* vl = vb - LIMBS * 32;
                const ulonglong2* vr = vb + LIMBS * 32;
                const ulonglong2 ht0 = vl[(LIMBS - 1) * 32], ht1 = vb[(LIMBS - 1) * 32], ht2 = vr[(LIMBS - 1) * 32];
                ulonglong2* o = flt + (size_t)y * flt_row;
                if (a.k0_same) {
                    const RescaleQuot rx = rescale_quot(ht0.x + ht1.x + ht2.x, a, LIMBS - 1);
                    const RescaleQuot ry = rescale_quot(ht0.y + ht1.y + ht2.y, a, LIMBS - 1);
#pragma unroll
                    for (int j = 0; j < LIMBS - 1; ++j) {
                        const ulonglong2 h0 = vl[j * 32], h1 = vb[j * 32], h2 = vr[j * 32];
                        ulonglong2 v;
                        v.x = rescale_quot_limb(h0.x + h1.x + h2.x, rx, j, a);
                        v.y = rescale_quot_limb(h0.y + h1.y + h2.y, ry, j, a);
                        __stcs(o + (size_t)j * half, v);
                    }
                } else {
                    const u64 tx = shoup(ht0.x + ht1.x + ht2.x, a.k0[LIMBS - 1], a.k0p[LIMBS - 1], qt);
                    const u64 ty = shoup(ht0.y + ht1.y + ht2.y, a.k0[LIMBS - 1], a.k0p[LIMBS - 1], qt);
#pragma unroll
                    for (int j = 0; j < LIMBS - 1; ++j) {
                        const u64 qj = a.q[j];
                        const ulonglong2 h0 = vl[j * 32], h1 = vb[j * 32], h2 = vr[j * 32];
                        ulonglong2 v;
                        v.x = rescale_fold(shoup_lazy(h0.x + h1.x + h2.x, a.k0r[j], a.k0rp[j], qj), tx, j, a);
                        v.y = rescale_fold(shoup_lazy(h0.y + h1.y + h2.y, a.k0r[j], a.k0rp[j], qj), ty, j, a);
                        __stcs(o + (size_t)j * half, v);
                    }
                }
            }
        }
        __syncthreads();   // the next item rewrites both buffers
    }
}

// Fused watermark blend alpha*I + (1-alpha)*W, W an encrypted pattern: out = Rescale(Ka * I + Kb * W), W broadcast over
// channels when it has one channel. The kept limbs use Ka q_t^{-1}, Kb q_t^{-1}. One call
// handles coefficient pair c of polynomial b of one ciphertext.
template <int LIMBS>
__device__ __forceinline__ void blend_pair(const OpsArgs& a, const u64* ci, const u64* cw, u64* co, int b, int c)
{
    const int n = 1 << a.logn;
    const int t = LIMBS - 1;
    const ulonglong2* s0 = reinterpret_cast<const ulonglong2*>(ci + (u64)b * LIMBS * n) + c;
    const ulonglong2* s1 = reinterpret_cast<const ulonglong2*>(cw + (u64)b * LIMBS * n) + c;
    const u64 qt = a.q[t];
    const ulonglong2 ut = __ldcs(s0 + t * (n / 2)), wt = __ldg(s1 + t * (n / 2));
    // every limb's loads are issued before the first store: the compiler may not move a load
    // past a store that could alias it, and loads issued limb by limb between the stores left
    // too few bytes in flight (three limbs, 128x128x3: 0.77 -> 0.85 of copy bandwidth; four
    // limbs 0.76 -> 0.83; five limbs 0.73 -> 0.84)
    ulonglong2 uj[LIMBS - 1], vj[LIMBS - 1];
#pragma unroll
    for (int j = 0; j < LIMBS - 1; ++j) {
        uj[j] = __ldcs(s0 + j * (n / 2));
        vj[j] = __ldg(s1 + j * (n / 2));
    }
    if (a.k01_same) {
        // With Ka, Kb one integer each below every modulus, Ka I_t + Kb W_t = u q_t + m (m
        // centered) and limb j of the result is Ka q_t^{-1}(I_j - I_t) + Kb q_t^{-1}(W_j - W_t) + u:
        // two Shoup products per kept limb instead of three. u <= Ka + Kb < 2 q_j.
        ulonglong2* dst = reinterpret_cast<ulonglong2*>(co + (u64)b * (LIMBS - 1) * n) + c;
        auto quot = [&](u64 i_t, u64 w_t) -> u64 {
            u64 ha = mulhi(i_t, a.k0p[t]), hb = mulhi(w_t, a.k1p[t]);
            u64 r = (i_t * a.k0[t] - ha * qt) + (w_t * a.k1[t] - hb * qt);   // in [0, 4 q_t)
            u64 u = ha + hb;
            if (r >= 2 * qt) { r -= 2 * qt; u += 2; }
            if (r >= qt) { r -= qt; u += 1; }
            return u + (r > a.half_qt ? 1 : 0);
        };
        const u64 ux = quot(ut.x, wt.x), uy = quot(ut.y, wt.y);
#pragma unroll
        for (int j = 0; j < LIMBS - 1; ++j) {
            const u64 qj = a.q[j];
            const ulonglong2 u = uj[j], v = vj[j];
            auto limb = [&](u64 ij, u64 wj, u64 it, u64 wtt, u64 uu) -> u64 {
                uu = uu >= qj ? uu - qj : uu;
                u64 r = shoup_lazy(ij + a.mq[j] - it, a.k0r[j], a.k0rp[j], qj) +
                        shoup_lazy(wj + a.mq[j] - wtt, a.k1r[j], a.k1rp[j], qj) + uu;   // in [0, 5 q_j)
                r = r >= 4 * qj ? r - 4 * qj : r;
                r = r >= 2 * qj ? r - 2 * qj : r;
                return r >= qj ? r - qj : r;
            };
            ulonglong2 o;
            o.x = limb(u.x, v.x, ut.x, wt.x, ux);
            o.y = limb(u.y, v.y, ut.y, wt.y, uy);
            __stcs(dst + j * (n / 2), o);
        }
        return;
    }
    const u64 tx = add_mod(shoup(ut.x, a.k0[t], a.k0p[t], qt), shoup(wt.x, a.k1[t], a.k1p[t], qt), qt);
    const u64 ty = add_mod(shoup(ut.y, a.k0[t], a.k0p[t], qt), shoup(wt.y, a.k1[t], a.k1p[t], qt), qt);
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(co + (u64)b * (LIMBS - 1) * n) + c;
#pragma unroll
    for (int j = 0; j < LIMBS - 1; ++j) {
        const u64 qj = a.q[j];
        const ulonglong2 u = uj[j], v = vj[j];
        const u64 px = csub(shoup_lazy(u.x, a.k0r[j], a.k0rp[j], qj) + shoup_lazy(v.x, a.k1r[j], a.k1rp[j], qj), 2 * qj);
        const u64 py = csub(shoup_lazy(u.y, a.k0r[j], a.k0rp[j], qj) + shoup_lazy(v.y, a.k1r[j], a.k1rp[j], qj), 2 * qj);
        ulonglong2 o;
        o.x = rescale_fold(px, tx, j, a);
        o.y = rescale_fold(py, ty, j, a);
        __stcs(dst + j * (n / 2), o);
    }
}

// A block takes whole rows (ciphertext k, polynomial b): the pattern index of k (a division
// by the channel count) is worked out once per row, not once per coefficient pair.
template <int LIMBS>
__device__ __forceinline__ void blend_rows(const OpsArgs& a)
{
    const int n = 1 << a.logn;
    for (u64 kb = blockIdx.x; kb < 2 * a.n_ct; kb += gridDim.x) {
        const u64 k = kb >> 1;
        const int b = (int)(kb & 1);
        const u64 kw = (k / a.c) * a.c_w + (a.c_w == 1 ? 0 : k % a.c);
        const u64* ci = a.in0 + k * 2 * LIMBS * (u64)n;
        const u64* cw = a.in1 + kw * 2 * LIMBS * (u64)n;
        u64* co = a.out + k * 2 * (LIMBS - 1) * (u64)n;
        for (int c = threadIdx.x; c < n / 2; c += blockDim.x) blend_pair<LIMBS>(a, ci, cw, co, b, c);
    }
}

// Up to three limbs: no register bound (62 registers at three limbs).
template <int LIMBS>
__global__ void k_blend(const __grid_constant__ OpsArgs a)
{
    blend_rows<LIMBS>(a);
}

// Four limbs and more, 256 threads, compiled for three blocks per SM up to five limbs (80
// registers: the loads of every limb held at once, no spills at four limbs) and two above.
template <int LIMBS>
__global__ void __launch_bounds__(256, LIMBS <= 5 ? 3 : 2) k_blend_wide(const __grid_constant__ OpsArgs a)
{
    blend_rows<LIMBS>(a);
}

// Ragged batch: one block of kBlendBatchThreads per ciphertext; W of segment s has c1[s]
// channels. Compiled for three blocks per SM up to five limbs, as the single-image kernel.
constexpr int kBlendBatchThreads = 256;

template <int LIMBS>
__global__ void __launch_bounds__(kBlendBatchThreads, LIMBS <= 5 ? 3 : 2)
    k_blend_batch(const __grid_constant__ OpsArgs a, const __grid_constant__ SegTable t)
{
    const int n = 1 << a.logn;
    const u64 total = t.start[t.n];
    for (u64 g = blockIdx.x; g < total; g += gridDim.x) {
        const int s = seg_of(t, g);
        const u64 k = g - t.start[s];
        const u64 C = t.c[s], Cw = t.c1[s];
        const u64 kw = (k / C) * Cw + (Cw == 1 ? 0 : k % C);
        const u64* ci = t.in0[s] + k * 2 * LIMBS * (u64)n;
        const u64* cw = t.in1[s] + kw * 2 * LIMBS * (u64)n;
        u64* co = t.out[s] + k * 2 * (LIMBS - 1) * (u64)n;
        const int lh = a.logn - 1;   // n / 2 = 2^lh coefficient pairs per polynomial
        for (int i = threadIdx.x; i < n; i += blockDim.x) blend_pair<LIMBS>(a, ci, cw, co, i >> lh, i & ((1 << lh) - 1));
    }
}

// Plaintext add of a per-segment constant (brightness of each request), ciphertext copied:
// one block per ciphertext.
__global__ void __launch_bounds__(1024) k_ptadd_batch(const __grid_constant__ OpsArgs a,
                                                      const __grid_constant__ SegTable t)
{
    const int n = 1 << a.logn;
    const int limbs = a.limbs;
    const u64 total = t.start[t.n];
    for (u64 g = blockIdx.x; g < total; g += gridDim.x) {
        const int s = seg_of(t, g);
        const u64 k = g - t.start[s];
        if (t.in0[s] == t.out[s]) {   // in place: only coefficient 0 of c0 changes, per limb
            u64* c0 = t.out[s] + k * 2 * (u64)limbs * n;
            for (int l = threadIdx.x; l < limbs; l += blockDim.x) c0[(u64)l * n] = add_mod(c0[(u64)l * n], t.kadd[s][l], a.q[l]);
            continue;
        }
        const ulonglong2* src = reinterpret_cast<const ulonglong2*>(t.in0[s] + k * 2 * (u64)limbs * n);
        ulonglong2* dst = reinterpret_cast<ulonglong2*>(t.out[s] + k * 2 * (u64)limbs * n);
        for (int i = threadIdx.x; i < limbs * n; i += blockDim.x) {
            ulonglong2 v = __ldcs(src + i);
            const int row = i / (n / 2);                 // b * limbs + l
            if (i % (n / 2) == 0 && row < limbs) v.x = add_mod(v.x, t.kadd[s][row], a.q[row]);
            __stcs(dst + i, v);
        }
    }
}

// 192-bit two's-complement helpers for the CRT decode.
struct U192 { u64 w0, w1, w2; };

__device__ __forceinline__ void add192(U192& x, const U192& y)
{
    const u64 s0 = x.w0 + y.w0, c0 = s0 < x.w0;
    const u64 s1 = x.w1 + y.w1;
    u64 c1 = s1 < x.w1;
    const u64 s1c = s1 + c0;
    c1 += s1c < s1;
    x.w0 = s0; x.w1 = s1c; x.w2 = x.w2 + y.w2 + c1;
}

__device__ __forceinline__ void sub192(U192& x, const U192& y)
{
    const u64 d0 = x.w0 - y.w0, b0 = x.w0 < y.w0;
    const u64 d1 = x.w1 - y.w1;
    u64 b1 = x.w1 < y.w1;
    const u64 d1b = d1 - b0;
    b1 += d1 < b0;
    x.w0 = d0; x.w1 = d1b; x.w2 = x.w2 - y.w2 - b1;
}

// (y * W) mod 2^192 for a 64-bit y and a 3-word W
__device__ __forceinline__ U192 mul192(u64 y, const u64 (&w)[3])
{
    const u64 p0 = y * w[0], h0 = mulhi(y, w[0]);
    const u64 p1 = y * w[1], h1 = mulhi(y, w[1]);
    const u64 p2 = y * w[2];
    const u64 r1 = h0 + p1, c = r1 < h0;
    U192 r = {p0, r1, h1 + p2 + c};
    return r;
}

// ---------------------------------------------------------------------------------------
// Decryption of coefficient 0 (Sec. 2.2.2; the plaintext of a pixel is a constant polynomial)
// and exact CRT decoding (x held modulo 2^192, exact for |x| < 2^191).
// (c0 + c1*s)_0 = c0_0 + sum_j c1_j * srev_j with srev_0 = s_0, srev_j = -s_{N-j}; s is
// ternary, so the sum is signed additions only. One block per ciphertext.
// ---------------------------------------------------------------------------------------
// One block (whole warps, at most 32 of them) decrypts one ciphertext; `red` is the block's
// shared scratch. Ends with a barrier, so the caller may reuse `red` at once.
__device__ __forceinline__ void decrypt_ct(const DecArgs& a, const u64* ct, double scale, double* out,
                                           u64* residues, u64 (*red)[2][kMaxPrimes])
{
    const int n = 1 << a.logn;
    const int nl = a.crt.nl;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint16_t* s2 = reinterpret_cast<const uint16_t*>(a.srev);
    for (int l = 0; l < nl; ++l) {
        const u64 q = a.q[l], mu = a.crt.mu[l];
        const ulonglong2* c1 = reinterpret_cast<const ulonglong2*>(ct + ((u64)nl + l) * n);
        // residues are below 2^60: 8 of them plus a reduced partial sum fit 64 bits, so the
        // signed sums are reduced once per four coefficient pairs; the four loads of a round
        // are issued together to keep several requests in flight per thread
        u64 pos = 0, neg = 0;
        for (int j0 = threadIdx.x; j0 < n / 2; j0 += 4 * blockDim.x) {
            ulonglong2 v[4];
            uint16_t sg[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j2 = j0 + u * blockDim.x;
                v[u] = j2 < n / 2 ? __ldcs(c1 + j2) : make_ulonglong2(0, 0);
                sg[u] = j2 < n / 2 ? __ldg(s2 + j2) : (uint16_t)0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int s0 = (int8_t)(sg[u] & 0xff), s1 = (int8_t)(sg[u] >> 8);
                pos += (s0 > 0 ? v[u].x : 0) + (s1 > 0 ? v[u].y : 0);
                neg += (s0 < 0 ? v[u].x : 0) + (s1 < 0 ? v[u].y : 0);
            }
            pos = reduce64(pos, q, mu);
            neg = reduce64(neg, q, mu);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            pos = add_mod(pos, __shfl_down_sync(0xffffffffu, pos, off), q);
            neg = add_mod(neg, __shfl_down_sync(0xffffffffu, neg, off), q);
        }
        if (lane == 0) { red[warp][0][l] = pos; red[warp][1][l] = neg; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        u64 y[kMaxPrimes];
        double v = 0.0;
        for (int l = 0; l < nl; ++l) {
            const u64 q = a.q[l];
            u64 p = ct[(u64)l * n], m = 0;  // c0 coefficient 0
            for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) {
                p = add_mod(p, red[wi][0][l], q);
                m = add_mod(m, red[wi][1][l], q);
            }
            const u64 res = sub_mod(p, m, q);
            if (residues) residues[l] = res;
            y[l] = shoup(res, a.crt.inv[l], a.crt.invp[l], q);
            v += (double)y[l] * a.crt.qinv[l];
        }
        // x = sum_l y_l * (Q/q_l) - round(sum_l y_l/q_l) * Q, the centered CRT value, held
        // modulo 2^192 (exact for |x| < 2^191)
        const u64 kq = (u64)rint(v);
        U192 x = {0, 0, 0};
        for (int l = 0; l < nl; ++l) add192(x, mul192(y[l], a.crt.qiw[l]));
        sub192(x, mul192(kq, a.crt.qw));
        const bool negv = (x.w2 >> 63) != 0;
        if (negv) {
            U192 z = {0, 0, 0};
            sub192(z, x);
            x = z;
        }
        const double mag = (double)x.w2 * 0x1p128 + (double)x.w1 * 0x1p64 + (double)x.w0;
        const double val = mag / scale;
        *out = negv ? -val : val;
    }
    __syncthreads();
}

// Two register budgets: blocks of up to 256 threads at 8 resident blocks per SM (32 registers:
// twice the loads in flight of the unconstrained build, the shape for whole images), and
// blocks of up to 1024 threads for a handful of ciphertexts, where one block's bandwidth is
// what counts.
template <int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_decrypt(const __grid_constant__ DecArgs a)
{
    __shared__ u64 red[32][2][kMaxPrimes];
    const int nl = a.crt.nl;
    for (u64 k = blockIdx.x; k < a.n_ct; k += gridDim.x)
        decrypt_ct(a, a.ct + k * 2 * (u64)nl * (1u << a.logn), a.scale, a.out + k,
                   a.residues_out ? a.residues_out + k * nl : nullptr, red);
}

// Ragged batch: segment s decrypts in0[s] (at the level of `a`) into dout[s] with scale[s].
template <int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_decrypt_batch(const __grid_constant__ DecArgs a,
                                                              const __grid_constant__ SegTable t)
{
    __shared__ u64 red[32][2][kMaxPrimes];
    const int nl = a.crt.nl;
    const u64 total = t.start[t.n];
    for (u64 g = blockIdx.x; g < total; g += gridDim.x) {
        const int s = seg_of(t, g);
        const u64 k = g - t.start[s];
        decrypt_ct(a, t.in0[s] + k * 2 * (u64)nl * (1u << a.logn), t.scale[s], t.dout[s] + k, nullptr, red);
    }
}

// ---------------------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------------------
static unsigned grid_for(u64 work, int threads)
{
    u64 g = (work + threads - 1) / threads;
    const u64 cap = 152ull * 16;  // enough blocks to fill every SM several times over
    if (g > cap) g = cap;
    return (unsigned)(g == 0 ? 1 : g);
}

cudaError_t launch_addsub(const OpsArgs& a, bool subtract, cudaStream_t st)
{
    const u64 work = a.n_ct * (u64)(2 * a.limbs) * ((1u << a.logn) / 2);
    k_addsub<<<grid_for(work, 256), 256, 0, st>>>(a, subtract ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_ptadd(const OpsArgs& a, cudaStream_t st)
{
    if (a.out == a.in0) {
        const u64 work = (a.k_hi - a.k_lo) * (u64)a.limbs;
        if (work == 0) return cudaSuccess;
        k_ptadd_inplace<<<grid_for(work, 256), 256, 0, st>>>(a);
    } else {
        const u64 work = a.n_ct * (u64)(2 * a.limbs) * ((1u << a.logn) / 2);
        k_ptadd_copy<<<grid_for(work, 256), 256, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_ptmul(const OpsArgs& a, cudaStream_t st)
{
    const u64 work = a.n_ct * (u64)(2 * a.limbs) * ((1u << a.logn) / 2);
    k_ptmul<<<grid_for(work, 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

#define ICHEE_LIMB_SWITCH_T(KERNEL, GRID, BLOCK, ARGS, TABLE)                \
    switch (ARGS.limbs) {                                                     \
    case 2: KERNEL<2><<<GRID, BLOCK, 0, st>>>(ARGS, TABLE); break;            \
    case 3: KERNEL<3><<<GRID, BLOCK, 0, st>>>(ARGS, TABLE); break;            \
    case 4: KERNEL<4><<<GRID, BLOCK, 0, st>>>(ARGS, TABLE); break;            \
    case 5: KERNEL<5><<<GRID, BLOCK, 0, st>>>(ARGS, TABLE); break;            \
    case 6: KERNEL<6><<<GRID, BLOCK, 0, st>>>(ARGS, TABLE); break;            \
    case 7: KERNEL<7><<<GRID, BLOCK, 0, st>>>(ARGS, TABLE); break;            \
    case 8: KERNEL<8><<<GRID, BLOCK, 0, st>>>(ARGS, TABLE); break;            \
    default: return cudaErrorInvalidValue;                                    \
    }

#define ICHEE_LIMB_SWITCH(KERNEL, GRID, BLOCK, ARGS)                          \
    switch (ARGS.limbs) {                                                     \
    case 2: KERNEL<2><<<GRID, BLOCK, 0, st>>>(ARGS); break;                   \
    case 3: KERNEL<3><<<GRID, BLOCK, 0, st>>>(ARGS); break;                   \
    case 4: KERNEL<4><<<GRID, BLOCK, 0, st>>>(ARGS); break;                   \
    case 5: KERNEL<5><<<GRID, BLOCK, 0, st>>>(ARGS); break;                   \
    case 6: KERNEL<6><<<GRID, BLOCK, 0, st>>>(ARGS); break;                   \
    case 7: KERNEL<7><<<GRID, BLOCK, 0, st>>>(ARGS); break;                   \
    case 8: KERNEL<8><<<GRID, BLOCK, 0, st>>>(ARGS); break;                   \
    default: return cudaErrorInvalidValue;                                    \
    }

cudaError_t launch_rescale(const OpsArgs& a, cudaStream_t st)
{
    const u64 work = a.n_ct * 2 * (u64)((1u << a.logn) / 2);
    const unsigned g = grid_for(work, 256);
    ICHEE_LIMB_SWITCH(k_rescale, g, 256, a)
    return cudaGetLastError();
}

// Launch of a staged mean-filter kernel: persistent grid of the blocks that fit on the GPU
// (bounded by blocks_per_sm when it is set), dynamic shared memory for the two stages.
template <typename K, typename... Args>
static cudaError_t mf_staged_launch(K kern, int limbs, int threads, u64 items, int blocks_per_sm, int num_sms,
                                    cudaStream_t st, const Args&... args)
{
    const size_t smem = mf_staged_smem(limbs, threads);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int fit = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (fit < 1) return cudaErrorInvalidConfiguration;
    if (blocks_per_sm > 0 && blocks_per_sm < fit) fit = blocks_per_sm;
    const u64 cap = (u64)fit * num_sms;
    kern<<<(unsigned)(items < cap ? items : cap), threads, smem, st>>>(args...);
    return cudaGetLastError();
}

// Threads of a staged block: the requested count, halved while its two stages would not fit
// in 200 KB of shared memory.
static int mf_staged_threads(int limbs, int threads)
{
    while (threads > 128 && mf_staged_smem(limbs, threads) > 200 * 1024) threads /= 2;
    return threads;
}

cudaError_t launch_meanfilter3(const OpsArgs& a, bool staged, int num_sms, cudaStream_t st)
{
    const int n = 1 << a.logn;
    const int threads = 256;
    const int chunks = (n / 2) / threads;
    const u64 blocks = (u64)a.rows * chunks * 2 * a.c;
    if (blocks == 0) return cudaSuccess;
    if (staged) {
        switch (a.limbs) {
#define ICHEE_MF_STAGED_CASE(LB) \
    case LB: return mf_staged_launch(k_meanfilter3_staged<LB>, LB, threads, blocks, 0, num_sms, st, a);
            ICHEE_MF_STAGED_CASE(2) ICHEE_MF_STAGED_CASE(3) ICHEE_MF_STAGED_CASE(4) ICHEE_MF_STAGED_CASE(5)
            ICHEE_MF_STAGED_CASE(6) ICHEE_MF_STAGED_CASE(7) ICHEE_MF_STAGED_CASE(8)
#undef ICHEE_MF_STAGED_CASE
        default: return cudaErrorInvalidValue;
        }
    }
    if (a.limbs >= 5) {
        // five limbs and more through the batched kernel as a one-image batch (band included):
        // it filters at 0.81 of copy bandwidth against 0.72 for the single-image kernel with the
        // same launch shape, instruction count and traffic (fewer load stalls); at three limbs
        // the single-image kernel is the faster one (0.75 against 0.70), at four they are level
        SegTable t;
        std::memset(&t, 0, sizeof(t));
        t.n = 1;
        t.start[0] = 0;
        t.start[1] = blocks;
        t.in0[0] = a.in0;
        t.out[0] = a.out;
        t.h[0] = (uint32_t)a.h;
        t.w[0] = (uint32_t)a.w;
        t.c[0] = (uint32_t)a.c;
        t.y0[0] = (uint32_t)a.y0;
        t.rows[0] = (uint32_t)a.rows;
        t.row0[0] = (uint32_t)a.row0;
        return launch_meanfilter3_batch(a, t, LaunchShape{threads, 0}, false, num_sms, st);
    }
    ICHEE_LIMB_SWITCH(k_meanfilter3, (unsigned)blocks, threads, a)
    return cudaGetLastError();
}

cudaError_t launch_blend(const OpsArgs& a, cudaStream_t st)
{
    const unsigned g = grid_for(2 * a.n_ct, 1);   // rows (ciphertext, polynomial)
    switch (a.limbs) {
    case 2: k_blend<2><<<g, 256, 0, st>>>(a); break;
    case 3: k_blend<3><<<g, 256, 0, st>>>(a); break;
    case 4: k_blend_wide<4><<<g, 256, 0, st>>>(a); break;
    case 5: k_blend_wide<5><<<g, 256, 0, st>>>(a); break;
    case 6: k_blend_wide<6><<<g, 256, 0, st>>>(a); break;
    case 7: k_blend_wide<7><<<g, 256, 0, st>>>(a); break;
    case 8: k_blend_wide<8><<<g, 256, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

static unsigned persistent_grid(u64 total, LaunchShape ls, int num_sms)
{
    // blocks_per_sm = 0: one block per work item (no grid-stride loop), capped at 2^31 - 1
    const u64 cap = ls.blocks_per_sm > 0 ? (u64)num_sms * ls.blocks_per_sm : 0x7fffffffull;
    return (unsigned)(total < cap ? total : cap);
}

cudaError_t launch_meanfilter3_batch(const OpsArgs& a, const SegTable& t, LaunchShape ls, bool staged, int num_sms,
                                     cudaStream_t st)
{
    const u64 total = t.n > 0 ? t.start[t.n] : 0;
    if (total == 0) return cudaSuccess;
    if (staged) {
        // items were counted by the caller for ls.threads; the staged block keeps that count
        // unless its stages do not fit, so the caller counts with mf_batch_threads
        const int th = mf_staged_threads(a.limbs, ls.threads);
        if (th != ls.threads) return cudaErrorInvalidValue;
        switch (a.limbs) {
#define ICHEE_MF_STAGED_CASE(LB) \
    case LB: return mf_staged_launch(k_meanfilter3_staged_batch<LB>, LB, th, total, ls.blocks_per_sm, num_sms, st, a, t);
            ICHEE_MF_STAGED_CASE(2) ICHEE_MF_STAGED_CASE(3) ICHEE_MF_STAGED_CASE(4) ICHEE_MF_STAGED_CASE(5)
            ICHEE_MF_STAGED_CASE(6) ICHEE_MF_STAGED_CASE(7) ICHEE_MF_STAGED_CASE(8)
#undef ICHEE_MF_STAGED_CASE
        default: return cudaErrorInvalidValue;
        }
    }
    const unsigned g = persistent_grid(total, ls, num_sms);
    ICHEE_LIMB_SWITCH_T(k_meanfilter3_batch, g, ls.threads, a, t)
    return cudaGetLastError();
}

// Threads per block of the fused kernel for a launch shape: 32 x columns per strip (at least 4
// columns), at most 512 above three limbs (the kernel's register bound), halved until the two
// row buffers fit in shared memory.
int fused_threads(int limbs, int threads)
{
    const int cap = limbs <= 3 ? 1024 : 512;
    int th = threads < 128 ? 128 : (threads > cap ? cap : threads);
    while (th > 128 && (size_t)2 * (th / 32) * limbs * 32 * 16 > 200 * 1024) th /= 2;
    return th;
}

u64 fused_items(int logn, int limbs, int threads, u32 w, u32 c)
{
    const u64 cols = (u64)fused_threads(limbs, threads) / 32;
    const u64 strips = ((u64)w + cols - 3) / (cols - 2);
    return (u64)c * 2 * (((u64)1 << logn) / 2 / 32) * strips;
}

cudaError_t launch_radix_meanfilter3_batch(const RadixArgs& ra, const OpsArgs& a, const SegTable& t, LaunchShape ls,
                                           int num_sms, cudaStream_t st)
{
    const u64 total = t.n > 0 ? t.start[t.n] : 0;
    if (total == 0) return cudaSuccess;
    if ((1 << a.logn) / 2 < 32) return cudaErrorInvalidValue;
    const int th = fused_threads(a.limbs, ls.threads);
    const size_t smem = (size_t)2 * (th / 32) * a.limbs * 32 * sizeof(ulonglong2);
    const unsigned g = persistent_grid(total, ls, num_sms);
    cudaError_t e = cudaSuccess;
    switch (a.limbs) {
#define ICHEE_FUSED_CASE(LB)                                                                                   \
    case LB:                                                                                                   \
        e = cudaFuncSetAttribute(k_radix_meanfilter3_batch<LB>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                 (int)smem);                                                                   \
        if (e != cudaSuccess) return e;                                                                        \
        k_radix_meanfilter3_batch<LB><<<g, th, smem, st>>>(ra, a, t);                                          \
        break;
    ICHEE_FUSED_CASE(2)
    ICHEE_FUSED_CASE(3)
    ICHEE_FUSED_CASE(4)
    ICHEE_FUSED_CASE(5)
    ICHEE_FUSED_CASE(6)
    ICHEE_FUSED_CASE(7)
    ICHEE_FUSED_CASE(8)
#undef ICHEE_FUSED_CASE
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_blend_batch(const OpsArgs& a, const SegTable& t, LaunchShape ls, int num_sms, cudaStream_t st)
{
    const u64 total = t.n > 0 ? t.start[t.n] : 0;
    if (total == 0) return cudaSuccess;
    const unsigned g = persistent_grid(total, ls, num_sms);
    ICHEE_LIMB_SWITCH_T(k_blend_batch, g, kBlendBatchThreads, a, t)
    return cudaGetLastError();
}

cudaError_t launch_ptadd_batch(const OpsArgs& a, const SegTable& t, LaunchShape ls, int num_sms, cudaStream_t st)
{
    const u64 total = t.n > 0 ? t.start[t.n] : 0;
    if (total == 0) return cudaSuccess;
    k_ptadd_batch<<<persistent_grid(total, ls, num_sms), ls.threads, 0, st>>>(a, t);
    return cudaGetLastError();
}

cudaError_t launch_decrypt_batch(const DecArgs& a, const SegTable& t, LaunchShape ls, int num_sms, cudaStream_t st)
{
    const u64 total = t.n > 0 ? t.start[t.n] : 0;
    if (total == 0) return cudaSuccess;
    if (ls.threads <= 256) k_decrypt_batch<256, 8><<<persistent_grid(total, ls, num_sms), ls.threads, 0, st>>>(a, t);
    else k_decrypt_batch<1024, 1><<<persistent_grid(total, ls, num_sms), ls.threads, 0, st>>>(a, t);
    return cudaGetLastError();
}

cudaError_t launch_decrypt(const DecArgs& a, int threads, cudaStream_t st)
{
    if (a.n_ct == 0) return cudaSuccess;
    if (threads < 32 || threads > 1024 || threads % 32 != 0) return cudaErrorInvalidValue;
    unsigned grid = (unsigned)(a.n_ct < (1u << 30) ? a.n_ct : (1u << 30));
    if (a.n_ct < 64) threads = 1024;   // a few ciphertexts: one wide block each
    if (threads <= 256) k_decrypt<256, 8><<<grid, threads, 0, st>>>(a);
    else k_decrypt<1024, 1><<<grid, threads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ichee

namespace ichee {
int mf_batch_threads(int limbs, int threads, bool staged) { return staged ? mf_staged_threads(limbs, threads) : threads; }
}  // namespace ichee
