// kernels_match.cu -- image matching (Sec. 4.4.3, reading R12): the sum over all pixel
// ciphertexts of (a - b)^2 with ct x ct multiplication, then relinearisation with the
// evaluation key (Sec. 2.2.3, reading R11).
#include "ops.h"
#include "ntt.cuh"

namespace ichee {

// One block per SM-sized share of the work: block j owns limb l = j % limbs and every
// (n_blocks/limbs)-th ciphertext. Per ciphertext it forms d = a - b for its limb, transforms
// d0 and d1, and accumulates (d0^2, 2 d0 d1, d1^2) position by position into its own slice of
// the scratch buffer (each position is owned by one thread, so no atomics are needed). The
// transform of d0 waits in a second shared-memory buffer (SMEM_D0) or, for the 2^14 ring whose
// buffers do not both fit, in the fourth scratch row; d1's waits in the transform buffer.
template <int LOGN, bool SMEM_D0>
__global__ void __launch_bounds__(NttShape<LOGN>::T, 1) k_sqdiff_accumulate(const __grid_constant__ SqDiffArgs a)
{
    constexpr int N = 1 << LOGN;
    constexpr int LAST = NttShape<LOGN>::LAST;
    extern __shared__ u64 buf[];
    u64* acc = a.partial + (size_t)blockIdx.x * 4 * N;
    u64* d0buf = SMEM_D0 ? buf + N : acc + 3 * N;
    const int tid = threadIdx.x;
    const int limbs = a.limbs;
    const int l = blockIdx.x % limbs;
    const u64 stride = a.n_blocks / limbs;
    const u64 start = blockIdx.x / limbs;
    const u64 q = a.rns.q[l];
    const u64 m0 = a.rns.m0[l], m1 = a.rns.m1[l];
    const ModTables t = a.rns.tab[l];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int x = elem_index<LOGN, LAST>(tid, e);
        acc[x] = 0;
        acc[N + x] = 0;
        acc[2 * N + x] = 0;
    }
    for (u64 k = start; k < a.n_ct; k += stride) {
        const u64* A = a.a + k * 2 * (u64)limbs * N;
        const u64* B = a.b + k * 2 * (u64)limbs * N;
#pragma unroll 1
        for (int pb = 0; pb < 2; ++pb) {
            const u64* pa = A + ((u64)pb * limbs + l) * N;
            const u64* pbb = B + ((u64)pb * limbs + l) * N;
            u64 r[1][16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int x = elem_index<LOGN, 0>(tid, e);
                r[0][e] = sub_mod(__ldcs(pa + x), __ldcs(pbb + x), q);
            }
            __syncthreads();
            ntt_fwd_regs<LOGN, 1>(buf, r, tid, t, q);
            __syncthreads();
            u64* dst = pb == 0 ? d0buf : buf;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int x = elem_index<LOGN, LAST>(tid, e);
                dst[SMEM_D0 || pb ? swz(x) : x] = csub(csub(r[0][e], 2 * q), q);
            }
        }
#pragma unroll 1
        for (int e = 0; e < 16; ++e) {
            const int x = elem_index<LOGN, LAST>(tid, e);
            const u64 d1 = buf[swz(x)];
            const u64 d0 = SMEM_D0 ? d0buf[swz(x)] : d0buf[x];
            const u64 t0 = mul_mod(d0, d0, q, m0, m1);
            u64 t1 = mul_mod(d0, d1, q, m0, m1);
            t1 = add_mod(t1, t1, q);
            const u64 t2 = mul_mod(d1, d1, q, m0, m1);
            acc[x] = add_mod(acc[x], t0, q);
            acc[N + x] = add_mod(acc[N + x], t1, q);
            acc[2 * N + x] = add_mod(acc[2 * N + x], t2, q);
        }
    }
}

template <int LOGN>
static cudaError_t sqdiff_launch(const SqDiffArgs& a, cudaStream_t st)
{
    constexpr bool keep = LOGN <= 13;
    const size_t smem = (keep ? 2 : 1) * (sizeof(u64) << LOGN);
    cudaError_t e = cudaFuncSetAttribute(k_sqdiff_accumulate<LOGN, keep>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_sqdiff_accumulate<LOGN, keep><<<a.n_blocks, NttShape<LOGN>::T, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sqdiff_accumulate(const SqDiffArgs& a, cudaStream_t st)
{
    if (a.n_blocks <= 0 || a.n_blocks % a.limbs != 0) return cudaErrorInvalidValue;
    switch (a.rns.logn) {
    case 10: return sqdiff_launch<10>(a, st);
    case 11: return sqdiff_launch<11>(a, st);
    case 12: return sqdiff_launch<12>(a, st);
    case 13: return sqdiff_launch<13>(a, st);
    case 14: return sqdiff_launch<14>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

__global__ void k_sqdiff_reduce(RnsArgs rns, int limbs, const u64* partial, int n_blocks, u64* tensor)
{
    const int n = 1 << rns.logn;
    const int pl = blockIdx.y;                 // p * limbs + l
    const int p = pl / limbs, l = pl % limbs;
    const u64 q = rns.q[l];
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        u64 s = 0;
        for (int j = l; j < n_blocks; j += limbs) s = add_mod(s, partial[((size_t)j * 4 + p) * n + x], q);
        tensor[(size_t)pl * n + x] = s;
    }
}

cudaError_t launch_sqdiff_reduce(const RnsArgs& rns, int limbs, const u64* partial, int n_blocks, u64* tensor,
                                 cudaStream_t st)
{
    dim3 grid((1u << rns.logn) / 256, 3 * limbs);
    k_sqdiff_reduce<<<grid, 256, 0, st>>>(rns, limbs, partial, n_blocks, tensor);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Relinearisation by hybrid key switching with one special prime P (reading R11).
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
