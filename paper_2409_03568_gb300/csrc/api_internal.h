// api_internal.h -- library-internal definitions shared by the host translation units:
// context and cache objects, error reporting, and argument-building helpers.
#pragma once
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ichee.h"
#include "host_math.h"
#include "ops.h"

namespace ichee {

// Thread-local error message; returns `st`.
ichee_status fail(ichee_status st, const char* fmt, ...);

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t _e = (call);                                                           \
        if (_e != cudaSuccess)                                                             \
            return ::ichee::fail(_e == cudaErrorMemoryAllocation ? ICHEE_ENOMEM : ICHEE_ECUDA, "%s failed: %s", \
                                 #call, cudaGetErrorString(_e));                           \
    } while (0)

// NVTX range over a public entry point (shows up in Nsight / ncu timelines; a no-op without
// a tool attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace ichee

using ichee::u64;
using ichee::u32;
using ichee::RnsArgs;
using ichee::CdtTable;
using ichee::CrtLevel;
using ichee::LaunchShape;
using ichee::kMaxModuli;
using ichee::kMaxPrimes;

// Working buffer of a context: grows on demand, from cudaMalloc or from the allocator the
// caller installed (ichee_set_allocator). It remembers which allocator made its block, so the
// block goes back to the same one.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    ichee_free_fn freer = nullptr;
    void* freer_user = nullptr;
    cudaError_t ensure(size_t want, ichee_alloc_fn alloc, ichee_free_fn free_fn, void* user, cudaStream_t st)
    {
        if (want <= bytes) return cudaSuccess;
        release(st);
        if (alloc) {
            p = alloc(want, (void*)st, user);
            if (!p) return cudaErrorMemoryAllocation;
            freer = free_fn;
            freer_user = user;
        } else {
            cudaError_t e = cudaMalloc(&p, want);
            if (e != cudaSuccess) {
                p = nullptr;
                return e;
            }
        }
        bytes = want;
        return cudaSuccess;
    }
    void release(cudaStream_t st = nullptr)
    {
        if (p) {
            if (freer) freer(p, (void*)st, freer_user);
            else cudaFree(p);
        }
        p = nullptr;
        bytes = 0;
        freer = nullptr;
        freer_user = nullptr;
    }
};

struct ichee_ctx {
    ichee_params params;
    int device = 0;
    int logn = 0, n = 0, L = 0, nmod = 0;
    u64 q[kMaxModuli] = {};
    u64 P = 0;
    double delta = 0;
    RnsArgs rns;                 // all moduli (q_0..q_{L-1}, then P), device tables
    CdtTable cdt;
    u64* d_tables = nullptr;     // [nmod][2][N][2]: (twiddle, Shoup companion), forward then inverse
    u64* d_half_tw = nullptr;    // N = 2^14: [nmod][2][N/2][2] forward twiddles of the two half transforms
    ichee::ModTables half_tab[2][kMaxModuli] = {};
    u64* d_dm = nullptr;         // [L][256]
    u64* d_ninv = nullptr;       // [nmod] N^{-1} mod modulus, then [nmod] N^{-1} 2^64 (d_ninv_r)
    u64* d_ninv_r = nullptr;     // inside d_ninv: not freed separately
    CrtLevel crt[kMaxPrimes];    // index nl - 1
    bool have_pk = false, have_sk = false, have_evk = false;   // public key, secret key, evaluation key
    std::vector<int8_t> h_s;
    int8_t* d_s = nullptr;
    int8_t* d_srev = nullptr;
    u64* d_pk = nullptr;         // [2][L][N]
    u64* d_pk_hat = nullptr;
    u64* d_pk_hat_p = nullptr;
    ulonglong2* d_pk_pair = nullptr;   // (pk_hat, pk_hat_p) interleaved: the encryption kernel's operand
    u64* d_evk = nullptr;        // [L][2][L+1][N]
    u64* d_evk_hat = nullptr;
    u64* d_evk_hat_p = nullptr;
    DevBuf stage_in, stage_out, stage_res, scratch, kadd;
    ichee_alloc_fn user_alloc = nullptr;   // working-memory allocator (ichee_set_allocator), else cudaMalloc
    ichee_free_fn user_free = nullptr;
    void* user_alloc_ctx = nullptr;
    int* d_status = nullptr;
    int num_sms = 0;
    // launch shapes of the persistent batched kernels (defaults; ichee_autotune_batch refines)
    // one block per work item by default (the autotuner's choice for the 32-image batch)
    LaunchShape shape_radix = {256, 0}, shape_lookup = {256, 0}, shape_meanfilter = {256, 0};
    int mf_staged = 0;   // mean filter: 0 = register walk, 1 = bulk-copy staged form (ICHEE_TUNE_MF_STAGED)
    LaunchShape shape_blend = {256, 0}, shape_ptadd = {256, 0}, shape_decrypt = {256, 0};
    LaunchShape shape_fused = {1024, 1};
    int fused_schedule = 0;   // ichee_encrypt_meanfilter_batch: 0 = two batched kernels, 1 = fused kernel
};

struct ichee_cache {
    ichee_ctx* ctx = nullptr;
    ichee_cache_desc desc;
    std::vector<int> values;
    int32_t h_lut[256];
    int32_t* d_lut = nullptr;
    u64* d_values = nullptr;     // [K][2][L][N]
    u64* d_pool = nullptr;       // [M][2][L][N]
    int radix_base = 0, n_pow = 0, radix_randomize = 0;
    u64* d_radix = nullptr;      // [n_pow][2][L][N]
    u64* d_mult = nullptr;       // [n_pow][2r+1][2][L][N]
    u64* d_pair = nullptr;       // [2r+1][pair_w][2][L][N], top two positions summed (n_pow >= 3)
    int pair_w = 0;
};

constexpr u64 kIdPoolBase = 1ull << 32;
constexpr u64 kIdRadixBase = 1ull << 33;


namespace ichee {
// Ciphertexts of an h x w x c image; 0 if the image is empty or holds more than 2^40 of them (no
// device stores that many, and every size computed from the count then fits 64 bits).
inline u64 image_cts(uint32_t h, uint32_t w, uint32_t c)
{
    const u64 hw = (u64)h * w;
    if (hw == 0 || c == 0 || hw > (1ull << 40) / c) return 0;
    return hw * c;
}
size_t ct_words(const ichee_ctx* c, int limbs);
bool is_device_ptr(const void* p);
// Bytes from p to the end of the device allocation holding it; false if unknown.
bool device_bytes_left(const void* p, u64* left);
// EINVAL if [p, p + bytes) is known to run past the end of p's device allocation.
ichee_status check_span(const void* p, u64 bytes, const char* what);
RnsArgs rns_prefix(const ichee_ctx* c, int limbs);
PolyBatch batch(u64* data, int n_poly, int nl, const int* midx);
void encode_const(const ichee_ctx* c, double value, double scale, int limbs, u64* out);
EncArgs enc_args(const ichee_ctx* c, const uint8_t* d_pix, u64 n_ct, u64 seed, u64 id_base, u64* out);
RadixArgs radix_args(const ichee_ctx* c, const ichee_cache* k, const uint8_t* d_pix, u64 n_ct, u64 seed, u64* out);
LookupArgs lookup_args(const ichee_ctx* c, const ichee_cache* k, const uint8_t* d_pix, u64 n_ct, u64 seed, u64* out);
OpsArgs ops_base(const ichee_ctx* c, const ichee_ctimg_meta* m);
void set_rescale(const ichee_ctx* c, OpsArgs& a);
void set_k0(const ichee_ctx* c, OpsArgs& a, double v, double scale);
void set_k1(const ichee_ctx* c, OpsArgs& a, double v, double scale);
void fold_constants(const ichee_ctx* c, OpsArgs& a);
bool same_scale(double a, double b);
ichee_status check_img(const ichee_ctx* c, const uint64_t* d, const ichee_ctimg_meta* m, const char* what);
ichee_status check_out(const ichee_ctx* c, const uint64_t* d, u64 n_ct, int limbs, const char* what);
DecArgs dec_args(const ichee_ctx* c, int nl);
}  // namespace ichee
