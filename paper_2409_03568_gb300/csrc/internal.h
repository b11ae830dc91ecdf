// internal.h -- argument structures and kernel launchers shared by the translation units of
// libichee (not part of the public C ABI, which is include/ichee.h).
#pragma once
#include "common.cuh"

namespace ichee {

constexpr int kMinLogN = 10;
constexpr int kMaxLogN = 14;

// Fresh public-key encryption of pixel values (Sec. 2.2.2, 3.1).
struct EncArgs {
    RnsArgs rns;               // moduli 0..L-1 = ciphertext primes
    int L;                     // limbs written
    u64 n_ct;                  // ciphertexts
    const uint8_t* pixels;     // [n_ct] device
    const u64* dm;             // [L][256] (Delta * p) mod q_l
    const ulonglong2* pk_pair; // [2][L][N] (NTT(pk_b) * N^{-1}, its Shoup companion), bit-reversed order
    const int32_t* skip_lut;   // optional [256]: skip pixel p when skip_lut[p] >= 0
    u64 seed;
    u64 id_base;               // ct id of ciphertext k is id_base + k
    CdtTable cdt;
    u64* out;                  // [n_ct][2][L][N]
    int num_sms;               // persistent grid of the single-image kernel: one block per SM
    const u32* idx;            // optional: encrypt only pixels idx[0 .. *n_idx) (device list)
    const u32* n_idx;
};

// idx[0 .. *count) = the pixels k < n whose value has no slot (lut[px[k]] < 0), in any order;
// *count is zeroed first. Everything on the stream.
cudaError_t launch_miss_list(const uint8_t* px, u64 n, const int32_t* lut, u32* idx, u32* count, cudaStream_t st);

// pair[i] = (a[i], b[i]) for i < n
cudaError_t launch_interleave(const u64* a, const u64* b, u64 n, ulonglong2* pair, cudaStream_t st);

// Radix-cached encryption: c = sum_k M[k][d'_k], M[k][d] = d * Enc(r^k) (Sec. 3.2, 3.3).
struct RadixArgs {
    u64 q[kMaxPrimes];
    int L, logn;
    u64 n_ct;
    const uint8_t* pixels;
    const u64* mult;           // [n_pow][2r+1][2][L][N]
    int r, n_pow, randomize;
    // optional (n_pow >= 3): sums of the top two positions' multiples,
    // pair[(d_{n-2} + r) * pair_w + d_{n-1}] = M[n-2][d_{n-2}] + M[n-1][d_{n-1}]; pair_w = 0 when absent
    const u64* pair;           // [2r+1][pair_w][2][L][N]
    int pair_w;
    const int32_t* skip_lut;   // optional, as in EncArgs
    u64 seed, id_base;
    u64* out;
};

// Scanning / full cached encryption with the zero pool (Sec. 3.2, 3.3).
struct LookupArgs {
    u64 q[kMaxPrimes];
    int L, logn;
    u64 n_ct;
    const uint8_t* pixels;
    const int32_t* lut;        // [256] slot or -1 (missing values are skipped)
    const u64* value_cts;      // [K][2][L][N]
    const u64* pool;           // [M][2][L][N]
    u32 pool_size;
    u64 seed, id_base;
    u64* out;
};

// A ragged batch: up to kMaxSegs images ("segments") in one launch. Work item g of the launch
// belongs to segment s with start[s] <= g < start[s + 1] and is item g - start[s] of it. The
// table travels as a kernel argument (no device memory, nothing to allocate).
constexpr int kMaxSegs = 64;
struct SegTable {
    int n;
    u64 start[kMaxSegs + 1];
    const uint8_t* px[kMaxSegs];      // pixel input (encryption)
    const u64* in0[kMaxSegs];         // ciphertext inputs
    const u64* in1[kMaxSegs];
    u64* out[kMaxSegs];               // ciphertext output
    u64* out2[kMaxSegs];              // second ciphertext output (fused encrypt + filter)
    double* dout[kMaxSegs];           // decoded output (decryption)
    u64 seed[kMaxSegs];
    uint32_t h[kMaxSegs], w[kMaxSegs], c[kMaxSegs], c1[kMaxSegs];
    // mean filter of a band: output rows y0 .. y0 + rows - 1 (rows = 0: the whole image), the
    // input holding the image's rows from row0 on
    uint32_t y0[kMaxSegs], rows[kMaxSegs], row0[kMaxSegs];
    double scale[kMaxSegs];
    u64 kadd[kMaxSegs][kMaxPrimes];   // per-segment plaintext constant residues
};

__device__ __forceinline__ int seg_of(const SegTable& t, u64 g)
{
    int lo = 0, hi = t.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.start[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Launch shape of a persistent batched kernel (chosen by the autotuner).
struct LaunchShape {
    int threads;       // per block
    int blocks_per_sm;
};

// Launchers (kernels_enc.cu). All launch on `stream` and return cudaGetLastError().
cudaError_t launch_sample_small(int8_t* out, int n, u64 seed, u32 stream_id, u64 id, int gaussian,
                                const CdtTable& cdt, cudaStream_t st);
cudaError_t launch_sample_uniform(u64* out, int n, u64 q, u64 seed, u32 stream_id, u64 id, cudaStream_t st);
// Batched transforms over polys [n_poly][N]; poly p uses modulus rns.q[midx[p % nl]].
struct PolyBatch {
    u64* data;
    int n_poly;
    int nl;
    int midx[kMaxModuli];
};
cudaError_t launch_ntt_fwd(const RnsArgs& rns, const PolyBatch& b, cudaStream_t st);
cudaError_t launch_ntt_inv(const RnsArgs& rns, const PolyBatch& b, cudaStream_t st);
// out[p][i] = a[p][i] * b[p % b_period][i] mod q  (b_period polys of b repeat), full residues
cudaError_t launch_pointwise_mul(const RnsArgs& rns, const PolyBatch& out, const u64* a, const u64* b,
                                 int b_period, cudaStream_t st);
// out[p][i] = out[p][i] * c_p mod q where c_p = cst[midx[p % nl]] (a per-modulus constant)
cudaError_t launch_scale_const(const RnsArgs& rns, const PolyBatch& b, const u64* cst_per_mod, cudaStream_t st);
// Shoup companions of [n_poly][N] residues
cudaError_t launch_shoup_companions(const RnsArgs& rns, const PolyBatch& b, u64* out, cudaStream_t st);
// Small signed int8 polynomial reduced into modulus rns.q[m]
cudaError_t launch_small_to_mod(const int8_t* x, int n, u64 q, u64* out, cudaStream_t st);
// out = -x + small(e) mod q (x full residues, e int8) for one poly
cudaError_t launch_neg_add_small(const u64* x, const int8_t* e, int n, u64 q, u64* out, cudaStream_t st);
// out = x + c*y mod q  (one poly)
cudaError_t launch_axpy_const(u64* out, const u64* x, const u64* y, u64 c, int n, u64 q, u64 m0, u64 m1,
                              cudaStream_t st);

cudaError_t launch_encrypt_fresh(const EncArgs& a, cudaStream_t st);
cudaError_t launch_radix_multiples(const u64* radix_cts, int n_pow, int r, const RnsArgs& rns, int L, u64* mult,
                                   cudaStream_t st);
cudaError_t launch_radix_pairs(const u64* mult, int n_pow, int r, int pair_w, const RnsArgs& rns, int L, u64* pair,
                               cudaStream_t st);
cudaError_t launch_radix_combine(const RadixArgs& a, cudaStream_t st);
cudaError_t launch_lookup_combine(const LookupArgs& a, cudaStream_t st);
cudaError_t launch_histogram(const uint8_t* pixels, u64 n, u32* counts /*[256], zeroed*/, cudaStream_t st);

// Batched encryption over a SegTable whose items are ciphertexts (px, out, seed per segment;
// ciphertext k of a segment has ct id k, as in a single-image call). The uniform fields of the
// argument structs (keys, cache tables, moduli) apply to every segment; their per-image fields
// (pixels, n_ct, seed, out) are ignored.
cudaError_t launch_encrypt_fresh_batch(const EncArgs& a, const SegTable& t, int num_sms, cudaStream_t st);
cudaError_t launch_radix_combine_batch(const RadixArgs& a, const SegTable& t, LaunchShape ls, int num_sms,
                                       cudaStream_t st);
cudaError_t launch_lookup_combine_batch(const LookupArgs& a, const SegTable& t, LaunchShape ls, int num_sms,
                                        cudaStream_t st);

}  // namespace ichee
