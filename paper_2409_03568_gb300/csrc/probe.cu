// probe.cu -- integer throughput of the GPU, measured: the context the rooflines of the
// transform kernels need (their peak is derived from the SM count, clock and multiply-add rate;
// this measures the rate and what the library's butterfly reaches on its own). Not part of
// the method.
#include "api_internal.h"
#include "common.cuh"

namespace ichee {

// Eight independent chains of 32-bit multiply-adds per thread.
__global__ void __launch_bounds__(512) k_probe_imad(u32* out, int iters)
{
    u32 a[8];
    const u32 b = threadIdx.x | 1u, c = blockIdx.x;
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = threadIdx.x + i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = a[i] * b + c;
    }
    u32 acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= a[i];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// The library's forward butterfly (Harvey lazy reduction, Shoup product) on 16 residues held
// in registers: four radix-2 stages per iteration, 32 butterflies.
__global__ void __launch_bounds__(512) k_probe_butterfly(u64* out, u64 q, u64 w, u64 wp, int iters)
{
    u64 r[16];
    const u64 q2 = 2 * q;
#pragma unroll
    for (int i = 0; i < 16; ++i) r[i] = ((u64)threadIdx.x * 16 + i + blockIdx.x) % q;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int half = 1 << s;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                if (i & half) continue;
                u64 X = r[i];
                X = X >= q2 ? X - q2 : X;
                const u64 T = shoup_lazy(r[i + half], w + s, wp, q);
                r[i] = X + T;
                r[i + half] = X - T + q2;
            }
        }
    }
    u64 acc = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) acc ^= r[i];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace ichee

using namespace ichee;

extern "C" ichee_status ichee_probe_int_throughput(int device, double* imad_per_s, double* butterflies_per_s)
{
    if (!imad_per_s || !butterflies_per_s) return fail(ICHEE_EINVAL, "null argument");
    CK(cudaSetDevice(device));
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int threads = 512, blocks = sms * 4;
    void* out = nullptr;
    CK(cudaMalloc(&out, (size_t)blocks * threads * sizeof(u64)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const u64 q = 1152921504606830593ull;   // a 60-bit prime = 1 mod 2^14
    const u64 w = 123456789ull;
    const u64 wp = (u64)(((host::u128)w << 64) / q);
    cudaError_t err = cudaSuccess;
    float ms = 0.0f;
    k_probe_imad<<<blocks, threads>>>((u32*)out, 8);   // warm-up
    cudaEventRecord(e0);
    const int it_imad = 4000;
    k_probe_imad<<<blocks, threads>>>((u32*)out, it_imad);
    cudaEventRecord(e1);
    err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess) *imad_per_s = (double)blocks * threads * it_imad * 16 * 8 / (ms * 1e-3);
    if (err == cudaSuccess) {
        k_probe_butterfly<<<blocks, threads>>>((u64*)out, q, w, wp, 8);
        cudaEventRecord(e0);
        const int it_bfly = 1000;
        k_probe_butterfly<<<blocks, threads>>>((u64*)out, q, w, wp, it_bfly);
        cudaEventRecord(e1);
        err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess) *butterflies_per_s = (double)blocks * threads * it_bfly * 32 / (ms * 1e-3);
    }
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    CK(err);
    return ICHEE_OK;
}
