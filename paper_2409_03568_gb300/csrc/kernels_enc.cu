// kernels_enc.cu -- key generation helpers, fused fresh encryption (Sec. 2.2.2, 3.1) and the
// cached encryption kernels (radix combine and value lookup with the zero pool, Sec. 3.2, 3.3).
#include "internal.h"
#include "ntt.cuh"

namespace ichee {

// ---------------------------------------------------------------------------------------
// Samplers (Sec. 2.2.1 / 2.2.2). Coefficient i of a ternary polynomial uses word i%4 of
// Philox block i/4; of a Gaussian one, words 2(i%2), 2(i%2)+1 of block i/2; of a uniform
// one, the four words of block i as a 128-bit x giving floor(x*q / 2^128).
// ---------------------------------------------------------------------------------------

__global__ void k_sample_small(int8_t* out, int n, u64 seed, u32 stream_id, u64 id, int gaussian, CdtTable cdt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (gaussian) {
        Words4 w = philox(seed, stream_id, id, (u32)(i >> 1));
        int h = 2 * (i & 1);
        u64 u = (u64)w.w[h] | ((u64)w.w[h + 1] << 32);
        out[i] = (int8_t)gauss_of(u, cdt);
    } else {
        Words4 w = philox(seed, stream_id, id, (u32)(i >> 2));
        out[i] = (int8_t)ternary_of(w.w[i & 3]);
    }
}

__global__ void k_sample_uniform(u64* out, int n, u64 q, u64 seed, u32 stream_id, u64 id)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Words4 w = philox(seed, stream_id, id, (u32)i);
    u64 lo = (u64)w.w[0] | ((u64)w.w[1] << 32);
    u64 hi = (u64)w.w[2] | ((u64)w.w[3] << 32);
    // floor((hi*2^64 + lo) * q / 2^128) = floor((hi*q + floor(lo*q / 2^64)) / 2^64)
    u64 carry = mulhi(lo, q);
    u64 t_lo = hi * q;
    u64 t_hi = mulhi(hi, q);
    u64 s = t_lo + carry;
    t_hi += (s < t_lo) ? 1 : 0;
    out[i] = t_hi;
}

cudaError_t launch_sample_small(int8_t* out, int n, u64 seed, u32 stream_id, u64 id, int gaussian,
                                const CdtTable& cdt, cudaStream_t st)
{
    k_sample_small<<<(n + 255) / 256, 256, 0, st>>>(out, n, seed, stream_id, id, gaussian, cdt);
    return cudaGetLastError();
}

cudaError_t launch_sample_uniform(u64* out, int n, u64 q, u64 seed, u32 stream_id, u64 id, cudaStream_t st)
{
    k_sample_uniform<<<(n + 255) / 256, 256, 0, st>>>(out, n, q, seed, stream_id, id);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Batched transforms in global memory (set-up paths and key switching).
// ---------------------------------------------------------------------------------------

template <int LOGN>
__global__ void __launch_bounds__(NttShape<LOGN>::T) k_ntt_fwd(const __grid_constant__ RnsArgs rns, const __grid_constant__ PolyBatch b)
{
    extern __shared__ u64 sm[];
    const int tid = threadIdx.x;
    const int m = b.midx[blockIdx.x % b.nl];
    const u64 q = rns.q[m];
    u64* d = b.data + (size_t)blockIdx.x * (1 << LOGN);
    u64 r[1][16];
#pragma unroll
    for (int e = 0; e < 16; ++e) r[0][e] = d[elem_index<LOGN, 0>(tid, e)];
    ntt_fwd_regs<LOGN, 1>(sm, r, tid, rns.tab[m], q);
#pragma unroll
    for (int e = 0; e < 16; ++e) d[elem_index<LOGN, NttShape<LOGN>::LAST>(tid, e)] = csub(csub(r[0][e], 2 * q), q);
}

template <int LOGN>
__global__ void __launch_bounds__(NttShape<LOGN>::T) k_ntt_inv(const __grid_constant__ RnsArgs rns, const __grid_constant__ PolyBatch b)
{
    extern __shared__ u64 sm[];
    const int tid = threadIdx.x;
    const int m = b.midx[blockIdx.x % b.nl];
    const u64 q = rns.q[m];
    u64* d = b.data + (size_t)blockIdx.x * (1 << LOGN);
    u64 r[1][16];
#pragma unroll
    for (int e = 0; e < 16; ++e) r[0][e] = d[elem_index<LOGN, NttShape<LOGN>::LAST>(tid, e)];
    ntt_inv_regs<LOGN, 1>(sm, r, tid, rns.tab[m], q);
#pragma unroll
    for (int e = 0; e < 16; ++e) d[elem_index<LOGN, 0>(tid, e)] = csub(r[0][e], q);
}

template <int LOGN>
static cudaError_t ntt_launch(bool fwd, const RnsArgs& rns, const PolyBatch& b, cudaStream_t st)
{
    const int T = NttShape<LOGN>::T;
    const size_t smem = sizeof(u64) << LOGN;
    auto kern = fwd ? k_ntt_fwd<LOGN> : k_ntt_inv<LOGN>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<b.n_poly, T, smem, st>>>(rns, b);
    return cudaGetLastError();
}

static cudaError_t ntt_dispatch(bool fwd, const RnsArgs& rns, const PolyBatch& b, cudaStream_t st)
{
    if (b.n_poly <= 0) return cudaSuccess;
    switch (rns.logn) {
    case 10: return ntt_launch<10>(fwd, rns, b, st);
    case 11: return ntt_launch<11>(fwd, rns, b, st);
    case 12: return ntt_launch<12>(fwd, rns, b, st);
    case 13: return ntt_launch<13>(fwd, rns, b, st);
    case 14: return ntt_launch<14>(fwd, rns, b, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ntt_fwd(const RnsArgs& rns, const PolyBatch& b, cudaStream_t st) { return ntt_dispatch(true, rns, b, st); }
cudaError_t launch_ntt_inv(const RnsArgs& rns, const PolyBatch& b, cudaStream_t st) { return ntt_dispatch(false, rns, b, st); }

__global__ void k_pointwise_mul(RnsArgs rns, PolyBatch out, const u64* a, const u64* b, int b_period)
{
    const int n = 1 << rns.logn;
    const int p = blockIdx.y;
    const int m = out.midx[p % out.nl];
    const u64 q = rns.q[m];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        u64 x = a[(size_t)p * n + i];
        u64 y = b[(size_t)(p % b_period) * n + i];
        out.data[(size_t)p * n + i] = mul_mod(x, y, q, rns.m0[m], rns.m1[m]);
    }
}

cudaError_t launch_pointwise_mul(const RnsArgs& rns, const PolyBatch& out, const u64* a, const u64* b, int b_period,
                                 cudaStream_t st)
{
    dim3 grid((1u << rns.logn) / 256, out.n_poly);
    k_pointwise_mul<<<grid, 256, 0, st>>>(rns, out, a, b, b_period);
    return cudaGetLastError();
}

__global__ void k_scale_const(RnsArgs rns, PolyBatch b, const u64* cst)
{
    const int n = 1 << rns.logn;
    const int p = blockIdx.y;
    const int m = b.midx[p % b.nl];
    const u64 q = rns.q[m], c = cst[m];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        u64* x = b.data + (size_t)p * n + i;
        *x = mul_mod(*x, c, q, rns.m0[m], rns.m1[m]);
    }
}

cudaError_t launch_scale_const(const RnsArgs& rns, const PolyBatch& b, const u64* cst_per_mod, cudaStream_t st)
{
    dim3 grid((1u << rns.logn) / 256, b.n_poly);
    k_scale_const<<<grid, 256, 0, st>>>(rns, b, cst_per_mod);
    return cudaGetLastError();
}

// floor(w * 2^64 / q) by binary long division (w < q < 2^61)
__device__ u64 shoup_companion(u64 w, u64 q)
{
    u64 rem = w, quo = 0;
    for (int i = 0; i < 64; ++i) {
        rem <<= 1;
        quo <<= 1;
        if (rem >= q) { rem -= q; quo |= 1; }
    }
    return quo;
}

__global__ void k_shoup_companions(RnsArgs rns, PolyBatch b, u64* out)
{
    const int n = 1 << rns.logn;
    const int p = blockIdx.y;
    const u64 q = rns.q[b.midx[p % b.nl]];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[(size_t)p * n + i] = shoup_companion(b.data[(size_t)p * n + i], q);
}

cudaError_t launch_shoup_companions(const RnsArgs& rns, const PolyBatch& b, u64* out, cudaStream_t st)
{
    dim3 grid((1u << rns.logn) / 256, b.n_poly);
    k_shoup_companions<<<grid, 256, 0, st>>>(rns, b, out);
    return cudaGetLastError();
}

__global__ void k_small_to_mod(const int8_t* x, int n, u64 q, u64* out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = small_mod(x[i], q);
}

cudaError_t launch_small_to_mod(const int8_t* x, int n, u64 q, u64* out, cudaStream_t st)
{
    k_small_to_mod<<<(n + 255) / 256, 256, 0, st>>>(x, n, q, out);
    return cudaGetLastError();
}

__global__ void k_neg_add_small(const u64* x, const int8_t* e, int n, u64 q, u64* out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = add_mod(x[i] == 0 ? 0 : q - x[i], small_mod(e[i], q), q);
}

cudaError_t launch_neg_add_small(const u64* x, const int8_t* e, int n, u64 q, u64* out, cudaStream_t st)
{
    k_neg_add_small<<<(n + 255) / 256, 256, 0, st>>>(x, e, n, q, out);
    return cudaGetLastError();
}

__global__ void k_axpy_const(u64* out, const u64* x, const u64* y, u64 c, int n, u64 q, u64 m0, u64 m1)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = add_mod(x[i], mul_mod(c, y[i], q, m0, m1), q);
}

__global__ void k_interleave(const u64* a, const u64* b, u64 n, ulonglong2* pair)
{
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
        pair[i] = make_ulonglong2(a[i], b[i]);
}

cudaError_t launch_interleave(const u64* a, const u64* b, u64 n, ulonglong2* pair, cudaStream_t st)
{
    const u64 blocks = (n + 255) / 256;
    k_interleave<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(a, b, n, pair);
    return cudaGetLastError();
}

cudaError_t launch_axpy_const(u64* out, const u64* x, const u64* y, u64 c, int n, u64 q, u64 m0, u64 m1,
                              cudaStream_t st)
{
    k_axpy_const<<<(n + 255) / 256, 256, 0, st>>>(out, x, y, c, n, q, m0, m1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Fused fresh encryption (Sec. 2.2.2, with the library sign convention pk = (-a*s + e, a),
// since the printed formulas do not cancel): one thread block per ciphertext.
//   sample v (ternary), e0, e1 (Gaussian) once into shared memory (int8), then per limb l:
//   v^ = NTT(v); c_b = INTT(v^ . pk^_b) + e_b (+ Delta*p at coefficient 0 of c0)
// pk^_b already carries the 1/N of the inverse transform. With KEEP_VHAT the transform of v
// stays in registers for both products (3 transforms per limb); without it (N = 2^14,
// register budget) it is recomputed (4 per limb). The first forward stage multiplies by a
// ternary operand and needs no product.
// ---------------------------------------------------------------------------------------

// Shared memory of one encryption block: the transform buffers (N words each; two where both
// inverse transforms of a limb run in lockstep: N = 2^13, 8 residues per thread), v, e0, e1 as
// int8 (3N bytes; two sets up to N = 2^13, used by alternate ciphertexts of the block), then the
// search copy of the Gaussian table (32 words).
template <int LOGN>
static constexpr int kEncBufs = LOGN == 13 ? 2 : 1;

template <int LOGN>
static constexpr int kEncSampleSets = LOGN <= 13 ? 2 : 1;

template <int LOGN>
__device__ __forceinline__ u64* enc_cdt_smem(u64* smem)
{
    return smem + kEncBufs<LOGN> * (1 << LOGN) + ((3 * kEncSampleSets<LOGN>) << LOGN) / 8;
}

template <int LOGN>
static constexpr size_t kEncSmem = ((sizeof(u64) * kEncBufs<LOGN> + 3 * kEncSampleSets<LOGN>) << LOGN) + 32 * sizeof(u64);

// `it` counts the ciphertexts the block has encrypted before this one. With two sample sets the
// block draws this ciphertext's samples into set it % 2 while slower warps may still read the
// previous ciphertext's set in its last epilogue; the barrier after the sampling of the previous
// ciphertext ordered every read of this set (two ciphertexts back) before it. With one set a
// barrier must precede the sampling. The transform buffers need none (see the limb loop).
template <int LOGN, bool KEEP_VHAT, int E>
__device__ __forceinline__ void encrypt_ct(const EncArgs& a, int p, u64 seed, u64 id, u64* ct, u64* smem, int it)
{
    constexpr int N = 1 << LOGN;
    constexpr int T = NttShape<LOGN, E>::T;
    constexpr int LAST = NttShape<LOGN, E>::LAST;
    constexpr int NB = kEncBufs<LOGN>;
    int8_t* sv = reinterpret_cast<int8_t*>(smem + NB * N) + (kEncSampleSets<LOGN> == 2 ? (it & 1) * 3 * N : 0);
    int8_t* se0 = sv + N;
    int8_t* se1 = se0 + N;
    const u64* tcdt = enc_cdt_smem<LOGN>(smem);   // filled by the kernel before its first ciphertext
    const int tid = threadIdx.x;
    const int L = a.L;
    if constexpr (kEncSampleSets<LOGN> == 1) __syncthreads();   // the previous ciphertext's samples no longer read
    for (int b = tid; b < N / 4; b += T) {
        Words4 w = philox(seed, kStreamV, id, (u32)b);
        u32 packed = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) packed |= ((u32)(uint8_t)(int8_t)ternary_of(w.w[i])) << (8 * i);
        reinterpret_cast<u32*>(sv)[b] = packed;
    }
    for (int b = tid; b < N / 2; b += T) {
        Words4 w0 = philox(seed, kStreamE0, id, (u32)b);
        Words4 w1 = philox(seed, kStreamE1, id, (u32)b);
        int g00 = gauss_of_sorted((u64)w0.w[0] | ((u64)w0.w[1] << 32), tcdt);
        int g01 = gauss_of_sorted((u64)w0.w[2] | ((u64)w0.w[3] << 32), tcdt);
        int g10 = gauss_of_sorted((u64)w1.w[0] | ((u64)w1.w[1] << 32), tcdt);
        int g11 = gauss_of_sorted((u64)w1.w[2] | ((u64)w1.w[3] << 32), tcdt);
        reinterpret_cast<uint16_t*>(se0)[b] = (uint16_t)((uint8_t)g00 | ((uint16_t)(uint8_t)g01 << 8));
        reinterpret_cast<uint16_t*>(se1)[b] = (uint16_t)((uint8_t)g10 | ((uint16_t)(uint8_t)g11 << 8));
    }
    __syncthreads();

    const int x0 = elem_index<LOGN, 0, E>(tid, 0);       // first-pass layout: x0 + elem_offset(e)
    const int xl = elem_index<LOGN, LAST, E>(tid, 0);    // last-pass layout
    if constexpr (NB == 2 && KEEP_VHAT) {
        // per limb: v^ = NTT(v), both products v^ . pk^_b at once, then the two inverse
        // transforms in lockstep (one pass structure, barriers and twiddle loads shared). No
        // block barrier separates the transforms: a transform's first exchange stores to the
        // slots of the layout the previous one last loaded (pass 0 after an inverse, the last
        // pass after a forward), so every thread overwrites only slots it has read itself, and
        // the second buffer's last readers (the previous limb's inverse) are behind the forward
        // transform's block-wide exchanges (3.19 -> 3.10 ms).
        for (int l = 0; l < L; ++l) {
            const u64 q = a.rns.q[l];
            const ModTables t = a.rns.tab[l];
            u64 r[1][E];
#pragma unroll
            for (int e = 0; e < E; ++e) r[0][e] = small_mod(sv[x0 + elem_offset<LOGN, 0, E>(e)], q);
            ntt_fwd_regs<LOGN, 1, true, false, E>(smem, r, tid, t, q);
            u64 rr[2][E];
            const ulonglong2* pk0 = a.pk_pair + (size_t)l * N + xl;
            const ulonglong2* pk1 = a.pk_pair + ((size_t)L + l) * N + xl;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const ulonglong2 w0 = __ldg(pk0 + elem_offset<LOGN, LAST, E>(e));
                const ulonglong2 w1 = __ldg(pk1 + elem_offset<LOGN, LAST, E>(e));
                rr[0][e] = shoup_lazy(r[0][e], w0.x, w0.y, q);
                rr[1][e] = shoup_lazy(r[0][e], w1.x, w1.y, q);
            }
            ntt_inv_regs<LOGN, 2, false, E>(smem, rr, tid, t, q);
#pragma unroll
            for (int pb = 0; pb < 2; ++pb) {
                const int8_t* noise = (pb == 0 ? se0 : se1) + x0;
                u64* dst = ct + ((u64)pb * L + l) * N + x0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int x = elem_offset<LOGN, 0, E>(e);
                    u64 v = rr[pb][e] + (q + (u64)(i64)noise[x]);   // [q - 31, 3q + 31)
                    v = csub(csub(v, 2 * q), q);
                    if (pb == 0 && x == 0 && x0 == 0) v = add_mod(v, a.dm[l * 256 + p], q);   // coefficient 0
                    __stcs(dst + x, v);
                }
            }
        }
        return;
    }
    // one transform at a time: a block barrier is needed only between two inverse transforms
    // (with v^ kept, the second product's), as in the lockstep form above
    for (int l = 0; l < L; ++l) {
        const u64 q = a.rns.q[l];
        const ModTables t = a.rns.tab[l];
        u64 r[1][E];
        u64 vh[KEEP_VHAT ? E : 1];
        for (int pb = 0; pb < 2; ++pb) {
            if (KEEP_VHAT && pb == 1) {
#pragma unroll
                for (int e = 0; e < E; ++e) r[0][e] = vh[KEEP_VHAT ? e : 0];
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) r[0][e] = small_mod(sv[x0 + elem_offset<LOGN, 0, E>(e)], q);
                ntt_fwd_regs<LOGN, 1, true, false, E>(smem, r, tid, t, q);   // after an inverse: no barrier
                if constexpr (KEEP_VHAT) {
#pragma unroll
                    for (int e = 0; e < E; ++e) vh[e] = r[0][e];
                }
            }
            const ulonglong2* pk = a.pk_pair + ((size_t)pb * L + l) * N + xl;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const ulonglong2 w = __ldg(pk + elem_offset<LOGN, LAST, E>(e));
                r[0][e] = shoup_lazy(r[0][e], w.x, w.y, q);
            }
            if (KEEP_VHAT && pb == 1) __syncthreads();   // an inverse right after an inverse
            ntt_inv_regs<LOGN, 1, false, E>(smem, r, tid, t, q);
            const int8_t* noise = (pb == 0 ? se0 : se1) + x0;
            u64* dst = ct + ((u64)pb * L + l) * N + x0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int x = elem_offset<LOGN, 0, E>(e);
                u64 v = r[0][e] + (q + (u64)(i64)noise[x]);   // [q - 31, 3q + 31)
                v = csub(csub(v, 2 * q), q);
                if (pb == 0 && x == 0 && x0 == 0) v = add_mod(v, a.dm[l * 256 + p], q);   // coefficient 0
                __stcs(dst + x, v);
            }
        }
    }
}

template <int LOGN, bool KEEP_VHAT, int E>
__global__ void __launch_bounds__(NttShape<LOGN, E>::T, 1) k_encrypt_fresh(const __grid_constant__ EncArgs a)
{
    extern __shared__ u64 smem[];
    cdt_for_search(a.cdt, enc_cdt_smem<LOGN>(smem));
    __syncthreads();
    const u64 ct_len = (u64)2 * a.L << LOGN;
    int it = 0;
    // all pixels, or a listed subset (the misses of a value cache) shared evenly; one call site,
    // so the kernel holds one copy of the transform code
    const u64 n = a.idx != nullptr ? (u64)*a.n_idx : a.n_ct;
    for (u64 g = blockIdx.x; g < n; g += gridDim.x) {
        const u64 k = a.idx != nullptr ? (u64)a.idx[g] : g;
        const int p = a.pixels[k];
        if (a.skip_lut != nullptr && a.skip_lut[p] >= 0) continue;  // uniform across the block
        encrypt_ct<LOGN, KEEP_VHAT, E>(a, p, a.seed, a.id_base + k, a.out + k * ct_len, smem, it++);
    }
}

template <int LOGN, bool KEEP_VHAT, int E>
__global__ void __launch_bounds__(NttShape<LOGN, E>::T, 1) k_encrypt_fresh_batch(const __grid_constant__ EncArgs a,
                                                                              const __grid_constant__ SegTable t)
{
    extern __shared__ u64 smem[];
    cdt_for_search(a.cdt, enc_cdt_smem<LOGN>(smem));
    __syncthreads();
    const u64 ct_len = (u64)2 * a.L << LOGN;
    const u64 total = t.start[t.n];
    int it = 0;
    for (u64 g = blockIdx.x; g < total; g += gridDim.x) {
        const int s = seg_of(t, g);
        const u64 k = g - t.start[s];
        const int p = t.px[s][k];
        if (a.skip_lut != nullptr && a.skip_lut[p] >= 0) continue;
        encrypt_ct<LOGN, KEEP_VHAT, E>(a, p, t.seed[s], k, t.out[s] + k * ct_len, smem, it++);
    }
}

// Residues per thread of the encryption transforms: 8 at N = 2^13 (1024 threads, twice the
// warps per SM of the 16-residue layout), else 16.
template <int LOGN>
static constexpr int kEncE = LOGN == 13 ? 8 : 16;

template <int LOGN>
static cudaError_t enc_launch(const EncArgs& a, cudaStream_t st)
{
    constexpr bool keep = LOGN <= 13;
    constexpr int E = kEncE<LOGN>;
    const int T = NttShape<LOGN, E>::T;
    const size_t smem = kEncSmem<LOGN>;
    cudaError_t e = cudaFuncSetAttribute(k_encrypt_fresh<LOGN, keep, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    // persistent: one block per SM (the shared memory fits one), each walking its share of the
    // ciphertexts, so a block's sampling overlaps its previous ciphertext's epilogue (3.10 ->
    // 3.06 ms); a listed subset is shared the same way. With pixels to skip in-kernel the shares
    // would be uneven, so there every ciphertext is a block of its own (a static share of the
    // whole image: 2.40 -> 2.81 ms for the misses of the top-32 cache).
    const u64 cap = a.skip_lut == nullptr && a.num_sms > 0 ? (u64)a.num_sms : (u64)(1u << 30);
    const u64 grid = a.n_ct < cap ? a.n_ct : cap;
    k_encrypt_fresh<LOGN, keep, E><<<(unsigned)grid, T, smem, st>>>(a);
    return cudaGetLastError();
}

template <int LOGN>
static cudaError_t enc_batch_launch(const EncArgs& a, const SegTable& t, int num_sms, cudaStream_t st)
{
    constexpr bool keep = LOGN <= 13;
    constexpr int E = kEncE<LOGN>;
    const int T = NttShape<LOGN, E>::T;
    const size_t smem = kEncSmem<LOGN>;
    cudaError_t e = cudaFuncSetAttribute(k_encrypt_fresh_batch<LOGN, keep, E>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const u64 total = t.start[t.n];
    const u64 cap = (u64)num_sms * 4;   // persistent: a few resident blocks per SM
    const unsigned grid = (unsigned)(total < cap ? total : cap);
    k_encrypt_fresh_batch<LOGN, keep, E><<<grid, T, smem, st>>>(a, t);
    return cudaGetLastError();
}

cudaError_t launch_encrypt_fresh_batch(const EncArgs& a, const SegTable& t, int num_sms, cudaStream_t st)
{
    if (t.n <= 0 || t.start[t.n] == 0) return cudaSuccess;
    switch (a.rns.logn) {
    case 10: return enc_batch_launch<10>(a, t, num_sms, st);
    case 11: return enc_batch_launch<11>(a, t, num_sms, st);
    case 12: return enc_batch_launch<12>(a, t, num_sms, st);
    case 13: return enc_batch_launch<13>(a, t, num_sms, st);
    case 14: return enc_batch_launch<14>(a, t, num_sms, st);
    default: return cudaErrorInvalidValue;
    }
}

__global__ void k_miss_list(const uint8_t* px, u64 n, const int32_t* lut, u32* idx, u32* count)
{
    for (u64 k = blockIdx.x * (u64)blockDim.x + threadIdx.x; k < n; k += (u64)gridDim.x * blockDim.x)
        if (lut[px[k]] < 0) idx[atomicAdd(count, 1u)] = (u32)k;
}

cudaError_t launch_miss_list(const uint8_t* px, u64 n, const int32_t* lut, u32* idx, u32* count, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(u32), st);
    if (e != cudaSuccess || n == 0) return e;
    const u64 blocks = (n + 255) / 256;
    k_miss_list<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, st>>>(px, n, lut, idx, count);
    return cudaGetLastError();
}

cudaError_t launch_encrypt_fresh(const EncArgs& a, cudaStream_t st)
{
    if (a.n_ct == 0) return cudaSuccess;
    switch (a.rns.logn) {
    case 10: return enc_launch<10>(a, st);
    case 11: return enc_launch<11>(a, st);
    case 12: return enc_launch<12>(a, st);
    case 13: return enc_launch<13>(a, st);
    case 14: return enc_launch<14>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------------------
// Cached encryption.
// ---------------------------------------------------------------------------------------

// M[k][d + r] = d * Enc(r^k) mod q for d in [-r, r]: the multiples a radix combine can ask
// for. Repeated homomorphic addition of a ciphertext (Sec. 3.2) equals this scalar multiple
// residue for residue, so tabulating it once per cache changes no result.
__global__ void k_radix_multiples(const u64* cts, int n_pow, int r, RnsArgs rns, int L, u64* mult)
{
    const int n = 1 << rns.logn;
    const size_t ct_len = (size_t)2 * L * n;
    const int slot = blockIdx.y;            // kk * (2r+1) + (d + r)
    const int kk = slot / (2 * r + 1);
    const int d = slot % (2 * r + 1) - r;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < ct_len; i += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)((i / n) % L);
        const u64 q = rns.q[l];
        const u64 c = cts[kk * ct_len + i];
        mult[slot * ct_len + i] = mul_mod(c, small_mod(d, q), q, rns.m0[l], rns.m1[l]);
    }
}

cudaError_t launch_radix_multiples(const u64* radix_cts, int n_pow, int r, const RnsArgs& rns, int L, u64* mult,
                                       cudaStream_t st)
{
    dim3 grid(64, n_pow * (2 * r + 1));
    k_radix_multiples<<<grid, 256, 0, st>>>(radix_cts, n_pow, r, rns, L, mult);
    return cudaGetLastError();
}

// P[i][j] = M[n-2][i] + M[n-1][j + r] mod q (i = d + r for d in [-r, r], j in [0, pair_w)): the
// top two positions' multiples summed once per cache, so a combine reads one cached ciphertext
// for both. Modular addition is exact, so every output residue is unchanged.
__global__ void k_radix_pairs(const u64* mult, int n_pow, int r, int pair_w, RnsArgs rns, int L, u64* pair)
{
    const int n = 1 << rns.logn;
    const size_t ct_len = (size_t)2 * L * n;
    const int width = 2 * r + 1;
    const int slot = blockIdx.y;            // i * pair_w + j
    const int i = slot / pair_w, j = slot % pair_w;
    const u64* lo = mult + ((size_t)(n_pow - 2) * width + i) * ct_len;
    const u64* hi = mult + ((size_t)(n_pow - 1) * width + j + r) * ct_len;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < ct_len; e += (size_t)gridDim.x * blockDim.x)
        pair[slot * ct_len + e] = add_mod(lo[e], hi[e], rns.q[(e / n) % L]);
}

cudaError_t launch_radix_pairs(const u64* mult, int n_pow, int r, int pair_w, const RnsArgs& rns, int L, u64* pair,
                               cudaStream_t st)
{
    dim3 grid(64, (2 * r + 1) * pair_w);
    k_radix_pairs<<<grid, 256, 0, st>>>(mult, n_pow, r, pair_w, rns, L, pair);
    return cudaGetLastError();
}

// Radix combine: one block per ciphertext. Signed digits d'_k = d_k + b_k - r*b_{k+1} with b
// from bit k of the pixel's randomness word (stream 3); c = sum_k M[k][d'_k], residue-wise
// modular sums of cached rows (the top two positions' from the pair table when the cache has
// one), 16-byte loads, streaming 16-byte stores.
__device__ __forceinline__ void radix_ct(const RadixArgs& a, int p, u64 seed, u64 id, u64* ct)
{
    const int n = 1 << a.logn;
    const size_t ct_len = (size_t)2 * a.L * n;
    const int width = 2 * a.r + 1;
    u32 bits = 0;
    if (a.randomize) bits = philox(seed, kStreamRadixBits, id, 0).w[0];
    const u64* src[8];
    int ns = 0;
    int rest = p;
    int dig[8];
    for (int kk = 0; kk < a.n_pow; ++kk) {
        int dk = rest % a.r;
        rest /= a.r;
        int bk = (a.randomize && kk >= 1) ? (int)((bits >> kk) & 1u) : 0;
        int bk1 = (a.randomize && kk + 1 < a.n_pow) ? (int)((bits >> (kk + 1)) & 1u) : 0;
        dig[kk] = dk + bk - a.r * bk1;
    }
    const int separate = a.pair_w ? a.n_pow - 2 : a.n_pow;
    for (int kk = 0; kk < separate; ++kk)
        if (dig[kk] != 0) src[ns++] = a.mult + ((size_t)kk * width + (dig[kk] + a.r)) * ct_len;
    if (a.pair_w && (dig[separate] != 0 || dig[separate + 1] != 0))
        src[ns++] = a.pair + ((size_t)(dig[separate] + a.r) * a.pair_w + dig[separate + 1]) * ct_len;
    // Row by row (one modulus per row); four coefficient pairs per thread and round, their
    // loads issued together.
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(ct);
    const int half = n / 2;
    for (int row = 0; row < 2 * a.L; ++row) {
        const u64 q = a.q[row % a.L];
        const size_t base = (size_t)row * half;
        for (int i0 = threadIdx.x; i0 < half; i0 += 4 * blockDim.x) {
            ulonglong2 acc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = make_ulonglong2(0, 0);
            for (int s = 0; s < ns; ++s) {
                const ulonglong2* sp = reinterpret_cast<const ulonglong2*>(src[s]) + base;
                ulonglong2 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + u * blockDim.x;
                    v[u] = i < half ? __ldg(sp + i) : make_ulonglong2(0, 0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    acc[u].x = add_mod(acc[u].x, v[u].x, q);
                    acc[u].y = add_mod(acc[u].y, v[u].y, q);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + u * blockDim.x;
                if (i < half) __stcs(dst + base + i, acc[u]);
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_radix_combine(const __grid_constant__ RadixArgs a)
{
    const size_t ct_len = (size_t)2 * a.L << a.logn;
    for (u64 k = blockIdx.x; k < a.n_ct; k += gridDim.x) {
        const int p = a.pixels[k];
        if (a.skip_lut != nullptr && a.skip_lut[p] >= 0) continue;
        radix_ct(a, p, a.seed, a.id_base + k, a.out + k * ct_len);
    }
}

__global__ void __launch_bounds__(1024) k_radix_combine_batch(const __grid_constant__ RadixArgs a,
                                                              const __grid_constant__ SegTable t)
{
    const size_t ct_len = (size_t)2 * a.L << a.logn;
    const u64 total = t.start[t.n];
    for (u64 g = blockIdx.x; g < total; g += gridDim.x) {
        const int s = seg_of(t, g);
        const u64 k = g - t.start[s];
        const int p = t.px[s][k];
        if (a.skip_lut != nullptr && a.skip_lut[p] >= 0) continue;
        radix_ct(a, p, t.seed[s], k, t.out[s] + k * ct_len);
    }
}

cudaError_t launch_radix_combine(const RadixArgs& a, cudaStream_t st)
{
    if (a.n_ct == 0) return cudaSuccess;
    unsigned grid = (unsigned)(a.n_ct < (1u << 30) ? a.n_ct : (1u << 30));
    k_radix_combine<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// Value lookup with the randomness pool: c = C[lut[p]] (+) Z[idx], idx = floor(w*M / 2^32)
// from stream 4. Pixels whose value is not cached are left to another kernel.
// One row (polynomial b, limb l: row = b L + l) of one pixel's ciphertext. The work is
// ordered row-major -- row 0 of every pixel, then row 1, ... -- so that while a row is being
// written only that row of the cached ciphertexts and of the pool is read: 256 x N x 8 bytes
// (16 MB at N = 8192) plus the pool's, which stays in L2 even when the whole cache does not.
__device__ __forceinline__ void lookup_row(const LookupArgs& a, int slot, u64 seed, u64 id, u64* ct, int row)
{
    const int n = 1 << a.logn;
    const int half = n / 2;
    const size_t ct_len = (size_t)2 * a.L * n;
    const size_t base = (size_t)row * half;
    const ulonglong2* c = reinterpret_cast<const ulonglong2*>(a.value_cts + (size_t)slot * ct_len) + base;
    const ulonglong2* z = nullptr;
    if (a.pool_size > 0) {
        u32 w = philox(seed, kStreamPool, id, 0).w[0];
        u32 idx = (u32)(((u64)w * a.pool_size) >> 32);
        z = reinterpret_cast<const ulonglong2*>(a.pool + (size_t)idx * ct_len) + base;
    }
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(ct) + base;
    const u64 q = a.q[row % a.L];
    // four coefficient pairs per thread and round, their loads issued together
    for (int i0 = threadIdx.x; i0 < half; i0 += 4 * blockDim.x) {
        ulonglong2 v[4], w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * blockDim.x;
            v[u] = i < half ? __ldg(c + i) : make_ulonglong2(0, 0);
            w[u] = (i < half && z != nullptr) ? __ldg(z + i) : make_ulonglong2(0, 0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i >= half) continue;
            if (z != nullptr) {
                v[u].x = add_mod(v[u].x, w[u].x, q);
                v[u].y = add_mod(v[u].y, w[u].y, q);
            }
            __stcs(dst + i, v[u]);
        }
    }
}

// Work item g = row * n_ct + pixel.
__global__ void __launch_bounds__(256) k_lookup_combine(const __grid_constant__ LookupArgs a)
{
    const size_t ct_len = (size_t)2 * a.L << a.logn;
    const u64 items = a.n_ct * 2 * a.L;
    for (u64 g = blockIdx.x; g < items; g += gridDim.x) {
        const int row = (int)(g / a.n_ct);
        const u64 k = g % a.n_ct;
        const int slot = a.lut[a.pixels[k]];
        if (slot < 0) continue;
        lookup_row(a, slot, a.seed, a.id_base + k, a.out + k * ct_len, row);
    }
}

// Work item g = row * total + (pixel item of the batch), rows outermost across all segments.
__global__ void __launch_bounds__(1024) k_lookup_combine_batch(const __grid_constant__ LookupArgs a,
                                                               const __grid_constant__ SegTable t)
{
    const size_t ct_len = (size_t)2 * a.L << a.logn;
    const u64 total = t.start[t.n];
    const u64 items = total * 2 * a.L;
    for (u64 gg = blockIdx.x; gg < items; gg += gridDim.x) {
        const int row = (int)(gg / total);
        const u64 g = gg % total;
        const int s = seg_of(t, g);
        const u64 k = g - t.start[s];
        const int slot = a.lut[t.px[s][k]];
        if (slot < 0) continue;
        lookup_row(a, slot, t.seed[s], k, t.out[s] + k * ct_len, row);
    }
}

static unsigned persistent_grid(u64 total, LaunchShape ls, int num_sms)
{
    // blocks_per_sm = 0: one block per work item (no grid-stride loop), capped at 2^31 - 1
    const u64 cap = ls.blocks_per_sm > 0 ? (u64)num_sms * ls.blocks_per_sm : 0x7fffffffull;
    return (unsigned)(total < cap ? total : cap);
}

cudaError_t launch_radix_combine_batch(const RadixArgs& a, const SegTable& t, LaunchShape ls, int num_sms,
                                       cudaStream_t st)
{
    const u64 total = t.n > 0 ? t.start[t.n] : 0;
    if (total == 0) return cudaSuccess;
    k_radix_combine_batch<<<persistent_grid(total, ls, num_sms), ls.threads, 0, st>>>(a, t);
    return cudaGetLastError();
}

cudaError_t launch_lookup_combine_batch(const LookupArgs& a, const SegTable& t, LaunchShape ls, int num_sms,
                                        cudaStream_t st)
{
    const u64 total = t.n > 0 ? t.start[t.n] : 0;
    if (total == 0) return cudaSuccess;
    k_lookup_combine_batch<<<persistent_grid(total * 2 * a.L, ls, num_sms), ls.threads, 0, st>>>(a, t);
    return cudaGetLastError();
}

cudaError_t launch_lookup_combine(const LookupArgs& a, cudaStream_t st)
{
    if (a.n_ct == 0) return cudaSuccess;
    const u64 items = a.n_ct * 2 * a.L;
    unsigned grid = (unsigned)(items < (1u << 30) ? items : (1u << 30));
    k_lookup_combine<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

__global__ void k_histogram(const uint8_t* px, u64 n, u32* counts)
{
    __shared__ u32 h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
        atomicAdd(&h[px[i]], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&counts[i], h[i]);
}

cudaError_t launch_histogram(const uint8_t* pixels, u64 n, u32* counts, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    unsigned grid = (unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    k_histogram<<<grid, 256, 0, st>>>(pixels, n, counts);
    return cudaGetLastError();
}

}  // namespace ichee
