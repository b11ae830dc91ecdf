// ops.h -- argument structures and launchers of the image operations, decryption and the
// matching / relinearisation kernels (internal to libichee).
#pragma once
#include "internal.h"

namespace ichee {

struct OpsArgs {
    int logn;
    int limbs;                      // limbs of the input ciphertexts
    u64 n_ct;
    u64 q[kMaxPrimes], mu[kMaxPrimes];
    // plaintext constants per limb (Shoup pairs): k0 for the first operand, k1 for the second
    u64 k0[kMaxPrimes], k0p[kMaxPrimes], k1[kMaxPrimes], k1p[kMaxPrimes];
    // rescale by q_t, t = limbs - 1: q_t^{-1} mod q_j (Shoup), (-q_t) mod q_j, (q_t - 1) / 2
    u64 qt_inv[kMaxPrimes], qt_inv_p[kMaxPrimes], neg_qt_mod[kMaxPrimes], half_qt;
    // constants already multiplied by q_t^{-1} mod q_j (Shoup pairs), for fused multiply + rescale
    u64 k0r[kMaxPrimes], k0rp[kMaxPrimes], k1r[kMaxPrimes], k1rp[kMaxPrimes];
    // k0_same: k0 is one integer below every modulus (equal residues in every limb), which lets a
    // fused multiply + rescale take one product per kept limb; mq[j] = ceil(4 q_t / q_j) * q_j
    int k0_same;
    u64 mq[kMaxPrimes];
    // k01_same: k0 and k1 are both such integers and k0 + k1 < 2 q_j for every kept limb j
    int k01_same;
    // plaintext add to ciphertexts [k_lo, k_hi): kadd[k * limbs + l] if kadd_per_ct, else k0[l]
    const u64* kadd;
    int kadd_per_ct;
    u64 k_lo, k_hi;
    // image shape (mean filter), channels of the second operand (blend)
    int h, w, c, c_w;
    // mean filter over a band of rows: output rows [y0, y0 + rows) of the h-row image, in0
    // holding its rows from row0 on (0, h, 0 for the whole image)
    int y0, rows, row0;
    int* status;                    // device status word (bounded waits that give up)
    const u64* in0;
    const u64* in1;
    u64* out;
};

// Exact CRT for one level (nl limbs): x = sum_l y_l * (Q/q_l) - k*Q with
// y_l = r_l * (Q/q_l)^{-1} mod q_l and k = round(sum_l y_l / q_l).
struct CrtLevel {
    int nl;
    u64 inv[kMaxPrimes], invp[kMaxPrimes];
    u64 qiw[kMaxPrimes][3];        // (Q/q_l) mod 2^192
    u64 qw[3];                     // Q mod 2^192
    double qinv[kMaxPrimes];       // 1/q_l
    u64 mu[kMaxPrimes];            // floor(2^64 / q_l)
};

struct DecArgs {
    int logn;
    u64 n_ct;
    u64 q[kMaxPrimes];
    CrtLevel crt;
    const int8_t* srev;            // [N] s_0, -s_{N-1}, ..., -s_1
    const u64* ct;                 // [n_ct][2][nl][N]
    double scale;
    double* out;                   // [n_ct]
    u64* residues_out;             // optional [n_ct][nl]
};

cudaError_t launch_addsub(const OpsArgs& a, bool subtract, cudaStream_t st);
cudaError_t launch_ptadd(const OpsArgs& a, cudaStream_t st);
cudaError_t launch_ptmul(const OpsArgs& a, cudaStream_t st);
cudaError_t launch_rescale(const OpsArgs& a, cudaStream_t st);
// staged: the bulk-copy form (input columns staged in shared memory), else the register walk
cudaError_t launch_meanfilter3(const OpsArgs& a, bool staged, int num_sms, cudaStream_t st);
cudaError_t launch_blend(const OpsArgs& a, cudaStream_t st);
cudaError_t launch_decrypt(const DecArgs& a, int threads, cudaStream_t st);

// Ragged batches (SegTable items: ciphertexts, or mean-filter rows x chunks x polys x channels).
// All segments share the level, the scale class and the constants of `a`.
cudaError_t launch_meanfilter3_batch(const OpsArgs& a, const SegTable& t, LaunchShape ls, bool staged, int num_sms,
                                     cudaStream_t st);
// Threads per block the batched mean filter runs with for a requested count (the staged form
// halves it while its stages would not fit); items are counted with it.
int mf_batch_threads(int limbs, int threads, bool staged);
cudaError_t launch_blend_batch(const OpsArgs& a, const SegTable& t, LaunchShape ls, int num_sms, cudaStream_t st);
cudaError_t launch_ptadd_batch(const OpsArgs& a, const SegTable& t, LaunchShape ls, int num_sms, cudaStream_t st);
cudaError_t launch_decrypt_batch(const DecArgs& a, const SegTable& t, LaunchShape ls, int num_sms, cudaStream_t st);
// Fused radix encryption + 3x3 mean filter over a ragged batch: segment s has
// fused_items(logn, limbs, ls.threads, w, c) items (c * 2 * (N/64) strips of
// fused_threads(limbs, ls.threads) / 32 - 2 columns); it reads pixels px[s] (seed[s]) and writes
// the encryption to out[s] and the filtered image to out2[s].
int fused_threads(int limbs, int threads);
u64 fused_items(int logn, int limbs, int threads, u32 w, u32 c);
cudaError_t launch_radix_meanfilter3_batch(const RadixArgs& ra, const OpsArgs& a, const SegTable& t, LaunchShape ls,
                                           int num_sms, cudaStream_t st);

// Matching: sum over ciphertexts of (a - b)^2 as a degree-2 ciphertext in the NTT domain.
// At N = 2^14 the accumulation runs split: each polynomial as two 2^13-point halves after the
// transform's first stage (sqdiff_split(logn)), block j taking limb j % limbs and half
// (j / limbs) % 2, with twiddle tables per half (htab).
__host__ __device__ inline bool sqdiff_split(int logn) { return logn == 14; }
struct SqDiffArgs {
    RnsArgs rns;                   // moduli 0..limbs-1
    int limbs;
    u64 n_ct;
    const u64* a;
    const u64* b;
    u64* partial;                  // [n_blocks][4][N] (split: [n_blocks][4][N/2]) scratch
    int n_blocks;                  // a multiple of limbs (split: of 2 limbs)
    ModTables htab[2][kMaxPrimes]; // split: twiddles of the two half transforms
};
cudaError_t launch_sqdiff_accumulate(const SqDiffArgs& a, cudaStream_t st);
// tensor[p][l][x] = (add ? tensor[p][l][x] mod q_l : 0) + the sum over the blocks of limb l (and,
// split, of the half holding x) of their partial terms, mod q_l
cudaError_t launch_sqdiff_reduce(const RnsArgs& rns, int limbs, const u64* partial, int n_blocks, u64* tensor,
                                 bool add, cudaStream_t st);
// out[r][x] = in[r][x] mod q_{r % limbs}, rows of N words, any 64-bit input
cudaError_t launch_reduce_rows(const RnsArgs& rns, int rows, int limbs, const u64* in, u64* out, cudaStream_t st);

// Key switching of a degree-2 ciphertext (hybrid, one digit per ciphertext prime, one special
// prime P).
struct RelinArgs {
    RnsArgs rns;                   // moduli q_0..q_{L-1}, P at index L
    int L;                         // limbs of the key (full chain)
    int limbs;                     // limbs of the ciphertext (t + 1)
    const u64* evk_hat;            // [L][2][L+1][N] NTT domain
    const u64* evk_hat_p;          // Shoup companions
    u64 p_inv[kMaxPrimes], p_inv_p[kMaxPrimes];  // P^{-1} mod q_j (Shoup)
    u64 neg_p_mod[kMaxPrimes];     // (-P) mod q_j
    u64 mu[kMaxModuli];
};
// Per-pixel squared difference with relinearisation and rescale (one output ciphertext per
// input pair). Moduli: q_0..q_{limbs-1} of the ciphertexts, P at index L of rns.
struct SqImgArgs {
    RnsArgs rns;
    int L;                         // limbs of the key (full chain)
    int limbs;                     // limbs of the input ciphertexts (t + 1)
    u64 n_ct;
    const u64* a;                  // [n_ct][2][limbs][N]
    const u64* b;
    u64* out;                      // [n_ct][2][limbs-1][N]
    u64* scratch;                  // [gridDim.x][3 limbs + 2][N], private to each block
    const u64* evk_hat;            // [L][2][L+1][N] NTT domain, N^{-1} folded in
    const u64* evk_hat_p;
    u64 ninv[kMaxPrimes], ninv_p[kMaxPrimes];    // N^{-1} 2^64 mod q_j (Shoup; 2^64 undoes the tensor's Montgomery factor)
    u64 pn[kMaxPrimes], pn_p[kMaxPrimes];        // P N^{-1} 2^64 mod q_j (Shoup)
    u64 r64[kMaxPrimes], r64_p[kMaxPrimes];      // 2^64 mod q_j (Shoup): d1^2 out of the Montgomery form
    u64 p_inv[kMaxPrimes], p_inv_p[kMaxPrimes];  // P^{-1} mod q_j (Shoup)
    u64 neg_p_mod[kMaxPrimes];                   // (-P) mod q_j
    u64 qt_inv[kMaxPrimes], qt_inv_p[kMaxPrimes], half_qt;  // rescale by q_t, t = limbs - 1
};
// Words of per-block scratch, and the persistent grid for n_ct ciphertexts on this device.
size_t sqdiff_image_scratch_words(int logn, int limbs);
int sqdiff_image_grid(int logn, u64 n_ct, int num_sms);
cudaError_t launch_sqdiff_image(const SqImgArgs& a, int grid, cudaStream_t st);

// digits[j][m][N] = centered residue of d2 limb j lifted to modulus m (m = 0..limbs-1, then P)
cudaError_t launch_relin_digits(const RelinArgs& a, const u64* d2, u64* digits, cudaStream_t st);
// acc[b][m][N] = sum_j digits^[j][m] * evk^_j[b][m]
cudaError_t launch_relin_mac(const RelinArgs& a, const u64* digits_hat, u64* acc, cudaStream_t st);
// out_b[j] = d_b[j] + (acc_b[j] - [acc_b[P]]_centered) * P^{-1} mod q_j
cudaError_t launch_relin_moddown(const RelinArgs& a, const u64* d01, const u64* acc, u64* out, cudaStream_t st);

}  // namespace ichee
