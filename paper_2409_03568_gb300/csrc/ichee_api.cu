// ichee_api.cu -- the C ABI of libichee (include/ichee.h): argument checks, set-up, and the
// launch sequences of key generation, cache building, encryption, image operations and
// decryption. Every arithmetic step on ciphertexts runs in the kernels of kernels_*.cu.
#include <algorithm>
#include <cmath>
#include <string>

#include <cuda.h>

#include "api_internal.h"

using namespace ichee;
namespace hm = ichee::host;

// ---------------------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------------------
static thread_local char g_err[512] = "";

ichee_status ichee::fail(ichee_status st, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

extern "C" const char* ichee_last_error(void) { return g_err; }

// ---------------------------------------------------------------------------------------
// Context and cache
// ---------------------------------------------------------------------------------------
size_t ichee::ct_words(const ichee_ctx* c, int limbs) { return (size_t)2 * limbs * c->n; }

bool ichee::is_device_ptr(const void* p)
{
    if (p == nullptr) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// The driver's pointer-attribute query, looked up once through the runtime so that the library
// links no driver library. Of an address it gives the range of the allocation holding it: for
// cudaMalloc memory the allocation itself; for virtual-memory mappings (cuMemMap, as in pool
// allocators with expandable segments) the whole reserved address range, so a buffer that spans
// several mappings is never refused.
typedef CUresult (*PtrAttrsFn)(unsigned int n, CUpointer_attribute* attrs, void** data, CUdeviceptr p);

static PtrAttrsFn ptr_attrs_fn()
{
    static const PtrAttrsFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult qr = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuPointerGetAttributes", &f, 12000, cudaEnableDefault, &qr) != cudaSuccess ||
            qr != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<PtrAttrsFn>(f);
    }();
    return fn;
}

bool ichee::device_bytes_left(const void* p, u64* left)
{
    if (!is_device_ptr(p)) return false;
    const PtrAttrsFn fn = ptr_attrs_fn();
    if (!fn) return false;
    CUdeviceptr base = 0;
    size_t size = 0;
    CUpointer_attribute attrs[2] = {CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, CU_POINTER_ATTRIBUTE_RANGE_SIZE};
    void* data[2] = {&base, &size};
    if (fn(2, attrs, data, (CUdeviceptr)(uintptr_t)p) != CUDA_SUCCESS) return false;
    const u64 at = (u64)(uintptr_t)p;
    if (size == 0 || at < base || at - base >= size) return false;
    *left = size - (at - base);
    return true;
}

// Memory the query does not know (another process's, an unusual allocator's) is taken on trust.
ichee_status ichee::check_span(const void* p, u64 bytes, const char* what)
{
    u64 left = 0;
    if (bytes > 0 && device_bytes_left(p, &left) && bytes > left)
        return fail(ICHEE_EINVAL, "%s: needs %llu bytes but its allocation ends %llu bytes after the pointer", what,
                    (unsigned long long)bytes, (unsigned long long)left);
    return ICHEE_OK;
}

extern "C" ichee_status ichee_buffer_bytes_left(const void* p, size_t* bytes_left)
{
    if (!p || !bytes_left) return fail(ICHEE_EINVAL, "null argument");
    u64 left = 0;
    if (!device_bytes_left(p, &left)) return fail(ICHEE_EUNSUPPORTED, "extent of %p unknown", p);
    *bytes_left = (size_t)left;
    return ICHEE_OK;
}

RnsArgs ichee::rns_prefix(const ichee_ctx* c, int limbs)
{
    RnsArgs r = c->rns;
    r.n_mod = limbs;
    return r;
}

PolyBatch ichee::batch(u64* data, int n_poly, int nl, const int* midx)
{
    PolyBatch b;
    b.data = data;
    b.n_poly = n_poly;
    b.nl = nl;
    for (int i = 0; i < kMaxModuli; ++i) b.midx[i] = (i < nl) ? midx[i] : 0;
    return b;
}

static std::vector<int> iota_idx(int n)
{
    std::vector<int> v(n);
    for (int i = 0; i < n; ++i) v[i] = i;
    return v;
}

// Residue of llround(value * scale) in every limb.
void ichee::encode_const(const ichee_ctx* c, double value, double scale, int limbs, u64* out)
{
    const long long k = llround(value * scale);
    for (int l = 0; l < limbs; ++l) out[l] = hm::signed_mod(k, c->q[l]);
}

// ---------------------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------------------
extern "C" ichee_status ichee_ctx_create(const ichee_params* p, int device, ichee_ctx** out)
{
    if (!p || !out) return fail(ICHEE_EINVAL, "ichee_ctx_create: null argument");
    *out = nullptr;
    if (p->log_n < (u32)kMinLogN || p->log_n > (u32)kMaxLogN)
        return fail(ICHEE_EUNSUPPORTED, "log_n %u outside [%d, %d]", p->log_n, kMinLogN, kMaxLogN);
    if (p->n_primes < 1 || p->n_primes > ICHEE_MAX_PRIMES)
        return fail(ICHEE_EINVAL, "n_primes %u outside [1, %d]", p->n_primes, ICHEE_MAX_PRIMES);
    for (u32 i = 0; i < p->n_primes; ++i)
        if (p->prime_bits[i] < 20 || p->prime_bits[i] > 60)
            return fail(ICHEE_EINVAL, "prime_bits[%u] = %u outside [20, 60]", i, p->prime_bits[i]);
    if (p->special_bits != 0 && (p->special_bits < 30 || p->special_bits > 61))
        return fail(ICHEE_EINVAL, "special_bits %u outside {0} U [30, 61]", p->special_bits);
    if (p->log2_scale > 55) return fail(ICHEE_EINVAL, "log2_scale %u > 55", p->log2_scale);
    if (p->gauss_bound < 1 || p->gauss_bound > (u32)kMaxGaussBound)
        return fail(ICHEE_EINVAL, "gauss_bound %u outside [1, %d]", p->gauss_bound, kMaxGaussBound);
    if (!(p->sigma > 0.0) || !std::isfinite(p->sigma)) return fail(ICHEE_EINVAL, "sigma must be positive");

    ichee_ctx* c = new ichee_ctx();
    c->params = *p;
    c->device = device;
    c->logn = (int)p->log_n;
    c->n = 1 << c->logn;
    c->L = (int)p->n_primes;
    c->delta = std::ldexp(1.0, (int)p->log2_scale);
    std::vector<u64> taken;
    for (int i = 0; i < c->L; ++i) {
        u64 qi = hm::chain_prime(p->prime_bits[i], p->log_n, taken);
        if (!qi) { delete c; return fail(ICHEE_EUNSUPPORTED, "no %u-bit prime = 1 mod 2N left", p->prime_bits[i]); }
        taken.push_back(qi);
        c->q[i] = qi;
    }
    if (p->special_bits) {
        c->P = hm::chain_prime(p->special_bits, p->log_n, taken);
        if (!c->P) { delete c; return fail(ICHEE_EUNSUPPORTED, "no special prime"); }
        c->q[c->L] = c->P;
    }
    c->nmod = c->L + (c->P ? 1 : 0);

    auto cleanup = [&](ichee_status st) {
        ichee_ctx_destroy(c);
        return st;
    };
    if (cudaSetDevice(device) != cudaSuccess) return cleanup(fail(ICHEE_ECUDA, "cudaSetDevice(%d) failed", device));
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);

    // transform tables
    const size_t nwords = (size_t)c->nmod * 4 * c->n;
    if (cudaMalloc(&c->d_tables, nwords * 8) != cudaSuccess) return cleanup(fail(ICHEE_ENOMEM, "tables"));
    std::memset(&c->rns, 0, sizeof(c->rns));
    c->rns.logn = c->logn;
    c->rns.n_mod = c->nmod;
    std::vector<u64> ninv(c->nmod);
    for (int m = 0; m < c->nmod; ++m) {
        const u64 qm = c->q[m];
        const std::vector<u64> t = hm::twiddles(qm, (unsigned)c->logn);   // [tw | twp | itw | itwp]
        std::vector<u64> pairs(t.size());                                     // [(tw, twp)] then [(itw, itwp)]
        for (int d = 0; d < 2; ++d)
            for (int k = 0; k < c->n; ++k) {
                pairs[((size_t)d * c->n + k) * 2] = t[(size_t)(2 * d) * c->n + k];
                pairs[((size_t)d * c->n + k) * 2 + 1] = t[(size_t)(2 * d + 1) * c->n + k];
            }
        if (cudaMemcpy(c->d_tables + (size_t)m * 4 * c->n, pairs.data(), pairs.size() * 8, cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return cleanup(fail(ICHEE_ECUDA, "upload tables"));
        c->rns.q[m] = qm;
        c->rns.mu[m] = (u64)(((hm::u128)1 << 64) / qm);
        const hm::u128 big = ~(hm::u128)0 / qm;  // floor(2^128 / q): q is odd, so 2^128 - 1 gives the same
        c->rns.m0[m] = (u64)big;
        c->rns.m1[m] = (u64)(big >> 64);
        u64 inv = qm;                       // Newton iteration for q^{-1} mod 2^64 (q odd)
        for (int it = 0; it < 6; ++it) inv *= 2 - qm * inv;
        c->rns.qinv[m] = 0 - inv;
        const u64* base = c->d_tables + (size_t)m * 4 * c->n;
        c->rns.tab[m].tw = reinterpret_cast<const ulonglong2*>(base);
        c->rns.tab[m].itw = reinterpret_cast<const ulonglong2*>(base + 2 * (size_t)c->n);
        ninv[m] = hm::invm((u64)c->n % qm, qm);
        if (sqdiff_split(c->logn)) {   // twiddles of the two half transforms after the first stage
            const size_t nh = (size_t)c->n / 2;
            if (!c->d_half_tw && cudaMalloc(&c->d_half_tw, (size_t)c->nmod * 4 * nh * 8) != cudaSuccess)
                return cleanup(fail(ICHEE_ENOMEM, "half tables"));
            std::vector<u64> half(4 * nh, 0);
            for (int h = 0; h < 2; ++h)
                for (size_t k = 1; k < nh; ++k) {
                    size_t s2 = 1;
                    while (s2 * 2 <= k) s2 *= 2;
                    const size_t src = (2 + h) * s2 + (k - s2);
                    half[((size_t)h * nh + k) * 2] = t[src];
                    half[((size_t)h * nh + k) * 2 + 1] = t[(size_t)c->n + src];
                }
            u64* hb = c->d_half_tw + (size_t)m * 4 * nh;
            if (cudaMemcpy(hb, half.data(), half.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
                return cleanup(fail(ICHEE_ECUDA, "upload half tables"));
            for (int h = 0; h < 2; ++h) {
                c->half_tab[h][m].tw = reinterpret_cast<const ulonglong2*>(hb + (size_t)h * 2 * nh);
                c->half_tab[h][m].itw = nullptr;
            }
        }
    }
    if (cudaMalloc(&c->d_ninv, 16 * (size_t)c->nmod) != cudaSuccess) return cleanup(fail(ICHEE_ENOMEM, "ninv"));
    for (int m = 0; m < c->nmod; ++m)   // N^{-1} 2^64: undoes a Montgomery product's 2^{-64} as well
        ninv.push_back(hm::mulm(ninv[m], (u64)(((hm::u128)1 << 64) % c->q[m]), c->q[m]));
    cudaMemcpy(c->d_ninv, ninv.data(), 16 * (size_t)c->nmod, cudaMemcpyHostToDevice);
    c->d_ninv_r = c->d_ninv + c->nmod;

    // Delta * p mod q_l for p = 0..255
    std::vector<u64> dm((size_t)c->L * 256);
    const u64 dl = 1ull << p->log2_scale;
    for (int l = 0; l < c->L; ++l)
        for (int v = 0; v < 256; ++v) dm[(size_t)l * 256 + v] = (u64)((hm::u128)dl * (u64)v % c->q[l]);
    if (cudaMalloc(&c->d_dm, dm.size() * 8) != cudaSuccess) return cleanup(fail(ICHEE_ENOMEM, "dm"));
    cudaMemcpy(c->d_dm, dm.data(), dm.size() * 8, cudaMemcpyHostToDevice);

    // Gaussian table
    std::memset(&c->cdt, 0, sizeof(c->cdt));
    c->cdt.bound = p->gauss_bound;
    hm::gauss_cdt(p->sigma, p->gauss_bound, c->cdt.t);

    // CRT constants for every level
    for (int nl = 1; nl <= c->L; ++nl) {
        CrtLevel& cl = c->crt[nl - 1];
        std::memset(&cl, 0, sizeof(cl));
        cl.nl = nl;
        u64 Qw[3] = {1, 0, 0};
        for (int l = 0; l < nl; ++l) hm::mul3(Qw, c->q[l], Qw);
        std::memcpy(cl.qw, Qw, sizeof(Qw));
        for (int i = 0; i < nl; ++i) {
            u64 w3[3] = {1, 0, 0};
            u64 qi_mod = 1;
            for (int l = 0; l < nl; ++l)
                if (l != i) {
                    hm::mul3(w3, c->q[l], w3);
                    qi_mod = hm::mulm(qi_mod, c->q[l] % c->q[i], c->q[i]);
                }
            std::memcpy(cl.qiw[i], w3, sizeof(w3));
            cl.inv[i] = hm::invm(qi_mod, c->q[i]);
            cl.invp[i] = hm::shoup_of(cl.inv[i], c->q[i]);
            cl.qinv[i] = 1.0 / (double)c->q[i];
            cl.mu[i] = (u64)(((hm::u128)1 << 64) / c->q[i]);
        }
    }
    if (cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess) return cleanup(fail(ICHEE_ENOMEM, "status"));
    cudaMemset(c->d_status, 0, sizeof(int));
    if (cudaGetLastError() != cudaSuccess) return cleanup(fail(ICHEE_ECUDA, "context set-up"));
    *out = c;
    return ICHEE_OK;
}

extern "C" void ichee_ctx_destroy(ichee_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    void* ptrs[] = {c->d_tables, c->d_half_tw, c->d_dm, c->d_ninv, c->d_s, c->d_srev, c->d_pk, c->d_pk_hat, c->d_pk_hat_p, c->d_pk_pair,
                    c->d_evk, c->d_evk_hat, c->d_evk_hat_p, c->d_status};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    c->stage_in.release();
    c->stage_out.release();
    c->stage_res.release();
    c->scratch.release();
    c->kadd.release();
    delete c;
}

extern "C" ichee_status ichee_ctx_primes(const ichee_ctx* c, uint64_t* q_out, uint64_t* p_out)
{
    if (!c) return fail(ICHEE_EINVAL, "null context");
    if (q_out)
        for (int i = 0; i < c->L; ++i) q_out[i] = c->q[i];
    if (p_out) *p_out = c->P;
    return ICHEE_OK;
}

extern "C" ichee_status ichee_ct_bytes(const ichee_ctx* c, uint32_t level, size_t* bytes)
{
    if (!c || !bytes) return fail(ICHEE_EINVAL, "null argument");
    if ((int)level >= c->L) return fail(ICHEE_ELEVEL, "level %u >= %d", level, c->L);
    *bytes = ct_words(c, (int)level + 1) * 8;
    return ICHEE_OK;
}

// ---------------------------------------------------------------------------------------
// Key generation (Sec. 2.2.2: pk = (-a*s + e, a); evk for hybrid key switching with the
// special prime P, one digit per ciphertext prime)
// ---------------------------------------------------------------------------------------
// Key buffers of the context (allocated once, by keygen or the first import).
static cudaError_t alloc_key_buffers(ichee_ctx* c)
{
    const size_t polyb = (size_t)c->n * 8;
    cudaError_t e = cudaSuccess;
    if (!c->d_s) {
        if ((e = cudaMalloc(&c->d_s, c->n)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&c->d_srev, c->n)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&c->d_pk, 2 * c->L * polyb)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&c->d_pk_hat, 2 * c->L * polyb)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&c->d_pk_hat_p, 2 * c->L * polyb)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&c->d_pk_pair, 4 * c->L * polyb)) != cudaSuccess) return e;
    }
    return e;
}

extern "C" ichee_status ichee_keygen(ichee_ctx* c, uint64_t seed, uint32_t flags, void* stream)
{
    ichee::NvtxRange nvtx_range("ichee_keygen");
    if (!c) return fail(ICHEE_EINVAL, "null context");
    const bool want_evk = (flags & ICHEE_WITH_EVK) != 0;
    if (want_evk && !c->P) return fail(ICHEE_EINVAL, "evaluation key needs special_bits > 0");
    CK(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int n = c->n, L = c->L;
    const size_t polyb = (size_t)n * 8;
    CK(alloc_key_buffers(c));
    const int nm = L + 1;  // moduli of the evaluation key
    const size_t tmp_polys = want_evk ? (size_t)(3 * L * nm + 2 * nm) : (size_t)(3 * L);
    int8_t* d_e = nullptr;
    u64* tmp = nullptr;
    CK(cudaMalloc(&d_e, n));
    CK(cudaMalloc(&tmp, tmp_polys * polyb));
    auto done = [&](ichee_status s) {
        cudaStreamSynchronize(st);
        cudaFree(d_e);
        cudaFree(tmp);
        return s;
    };
#define KCK(call)                                                                           \
    do {                                                                                    \
        cudaError_t _e = (call);                                                            \
        if (_e != cudaSuccess) return done(fail(ICHEE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(_e))); \
    } while (0)

    // s ternary (stream 8), e Gaussian (stream 9), a_l uniform (stream 16 + l), ct id 0
    KCK(launch_sample_small(c->d_s, n, seed, kStreamKeyS, 0, 0, c->cdt, st));
    KCK(launch_sample_small(d_e, n, seed, kStreamKeyE, 0, 1, c->cdt, st));
    u64* pk0 = c->d_pk;
    u64* pk1 = c->d_pk + (size_t)L * n;
    for (int l = 0; l < L; ++l) KCK(launch_sample_uniform(pk1 + (size_t)l * n, n, c->q[l], seed, kStreamKeyA + l, 0, st));
    // a*s per limb through the transform
    u64* A = tmp;
    u64* S = tmp + (size_t)L * n;
    std::vector<int> id = iota_idx(kMaxModuli);
    KCK(cudaMemcpyAsync(A, pk1, (size_t)L * polyb, cudaMemcpyDeviceToDevice, st));
    for (int l = 0; l < L; ++l) KCK(launch_small_to_mod(c->d_s, n, c->q[l], S + (size_t)l * n, st));
    const RnsArgs rl = rns_prefix(c, L);
    KCK(launch_ntt_fwd(rl, batch(A, L, L, id.data()), st));
    KCK(launch_ntt_fwd(rl, batch(S, L, L, id.data()), st));
    KCK(launch_pointwise_mul(rl, batch(A, L, L, id.data()), A, S, L, st));
    KCK(launch_ntt_inv(rl, batch(A, L, L, id.data()), st));
    KCK(launch_scale_const(rl, batch(A, L, L, id.data()), c->d_ninv, st));
    for (int l = 0; l < L; ++l) KCK(launch_neg_add_small(A + (size_t)l * n, d_e, n, c->q[l], pk0 + (size_t)l * n, st));
    // pk^ = NTT(pk) * N^{-1} with Shoup companions (the encryption kernel's operands)
    KCK(cudaMemcpyAsync(c->d_pk_hat, c->d_pk, 2 * L * polyb, cudaMemcpyDeviceToDevice, st));
    KCK(launch_ntt_fwd(rl, batch(c->d_pk_hat, 2 * L, L, id.data()), st));
    KCK(launch_scale_const(rl, batch(c->d_pk_hat, 2 * L, L, id.data()), c->d_ninv, st));
    KCK(launch_shoup_companions(rl, batch(c->d_pk_hat, 2 * L, L, id.data()), c->d_pk_hat_p, st));
    KCK(launch_interleave(c->d_pk_hat, c->d_pk_hat_p, (u64)2 * L * c->n, c->d_pk_pair, st));

    // s on the host: export copy and the reversed-negated form used by decryption
    c->h_s.resize(n);
    KCK(cudaMemcpyAsync(c->h_s.data(), c->d_s, n, cudaMemcpyDeviceToHost, st));
    KCK(cudaStreamSynchronize(st));
    std::vector<int8_t> srev(n);
    srev[0] = c->h_s[0];
    for (int j = 1; j < n; ++j) srev[j] = (int8_t)(-c->h_s[n - j]);
    KCK(cudaMemcpyAsync(c->d_srev, srev.data(), n, cudaMemcpyHostToDevice, st));

    if (want_evk) {
        if (!c->d_evk) {
            KCK(cudaMalloc(&c->d_evk, (size_t)L * 2 * nm * polyb));
            KCK(cudaMalloc(&c->d_evk_hat, (size_t)L * 2 * nm * polyb));
            KCK(cudaMalloc(&c->d_evk_hat_p, (size_t)L * 2 * nm * polyb));
        }
        const RnsArgs rm = c->rns;  // all L+1 moduli
        u64* AE = tmp;                               // [L][nm][N] a_j,i
        u64* SM = tmp + (size_t)L * nm * n;          // [nm][N] s mod m_i, then NTT
        u64* S2 = SM + (size_t)nm * n;               // [nm][N] s^2
        for (int j = 0; j < L; ++j)
            for (int i = 0; i < nm; ++i) {
                u64* a_ji = c->d_evk + (((size_t)j * 2 + 1) * nm + i) * n;
                KCK(launch_sample_uniform(a_ji, n, c->q[i], seed, kStreamKeyA + i, 1 + j, st));
                KCK(cudaMemcpyAsync(AE + ((size_t)j * nm + i) * n, a_ji, polyb, cudaMemcpyDeviceToDevice, st));
            }
        for (int i = 0; i < nm; ++i) KCK(launch_small_to_mod(c->d_s, n, c->q[i], SM + (size_t)i * n, st));
        KCK(launch_ntt_fwd(rm, batch(AE, L * nm, nm, id.data()), st));
        KCK(launch_ntt_fwd(rm, batch(SM, nm, nm, id.data()), st));
        KCK(launch_pointwise_mul(rm, batch(AE, L * nm, nm, id.data()), AE, SM, nm, st));
        KCK(launch_pointwise_mul(rm, batch(S2, nm, nm, id.data()), SM, SM, nm, st));
        KCK(launch_ntt_inv(rm, batch(AE, L * nm, nm, id.data()), st));
        KCK(launch_ntt_inv(rm, batch(S2, nm, nm, id.data()), st));
        KCK(launch_scale_const(rm, batch(AE, L * nm, nm, id.data()), c->d_ninv, st));
        KCK(launch_scale_const(rm, batch(S2, nm, nm, id.data()), c->d_ninv, st));
        for (int j = 0; j < L; ++j) {
            KCK(launch_sample_small(d_e, n, seed, kStreamKeyE, 1 + j, 1, c->cdt, st));
            for (int i = 0; i < nm; ++i) {
                u64* b0 = c->d_evk + (((size_t)j * 2 + 0) * nm + i) * n;
                KCK(launch_neg_add_small(AE + ((size_t)j * nm + i) * n, d_e, n, c->q[i], b0, st));
                if (i == j) {
                    const u64 pm = c->P % c->q[j];
                    KCK(launch_axpy_const(b0, b0, S2 + (size_t)j * n, pm, n, c->q[j], c->rns.m0[j], c->rns.m1[j], st));
                }
            }
        }
        KCK(cudaMemcpyAsync(c->d_evk_hat, c->d_evk, (size_t)L * 2 * nm * polyb, cudaMemcpyDeviceToDevice, st));
        KCK(launch_ntt_fwd(rm, batch(c->d_evk_hat, L * 2 * nm, nm, id.data()), st));
        KCK(launch_scale_const(rm, batch(c->d_evk_hat, L * 2 * nm, nm, id.data()), c->d_ninv, st));
        KCK(launch_shoup_companions(rm, batch(c->d_evk_hat, L * 2 * nm, nm, id.data()), c->d_evk_hat_p, st));
        c->have_evk = true;
    }
#undef KCK
    c->have_pk = c->have_sk = true;
    return done(ICHEE_OK);
}

extern "C" ichee_status ichee_export_key(ichee_ctx* c, int which, void* host_out, size_t bytes, void* stream)
{
    if (!c || !host_out) return fail(ICHEE_EINVAL, "null argument");
    CK(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)c->n;
    if (which == 0) {
        if (!c->have_sk) return fail(ICHEE_EINVAL, "no secret key");
        if (bytes != n) return fail(ICHEE_EINVAL, "secret key is %zu bytes", n);
        std::memcpy(host_out, c->h_s.data(), n);
        return ICHEE_OK;
    }
    const void* src = nullptr;
    size_t want = 0;
    if (which == 1) {
        if (!c->have_pk) return fail(ICHEE_EINVAL, "no public key");
        src = c->d_pk;
        want = 2 * (size_t)c->L * n * 8;
    }
    else if (which == 2) {
        if (!c->have_evk) return fail(ICHEE_EINVAL, "no evaluation key");
        src = c->d_evk;
        want = (size_t)c->L * 2 * (c->L + 1) * n * 8;
    } else return fail(ICHEE_EINVAL, "unknown key %d", which);
    if (bytes != want) return fail(ICHEE_EINVAL, "key is %zu bytes, got %zu", want, bytes);
    CK(cudaMemcpyAsync(host_out, src, want, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return ICHEE_OK;
}

extern "C" ichee_status ichee_import_key(ichee_ctx* c, int which, const void* host_in, size_t bytes, void* stream)
{
    if (!c || !host_in) return fail(ICHEE_EINVAL, "null argument");
    CK(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int n = c->n, L = c->L, nm = L + 1;
    const size_t polyb = (size_t)n * 8;
    std::vector<int> id = iota_idx(kMaxModuli);
    CK(alloc_key_buffers(c));
    if (which == 0) {
        if (bytes != (size_t)n) return fail(ICHEE_EINVAL, "secret key is %d bytes, got %zu", n, bytes);
        const int8_t* s = static_cast<const int8_t*>(host_in);
        for (int j = 0; j < n; ++j)
            if (s[j] < -1 || s[j] > 1) return fail(ICHEE_EINVAL, "secret key coefficient %d is %d, not ternary", j, s[j]);
        c->h_s.assign(s, s + n);
        std::vector<int8_t> srev(n);
        srev[0] = s[0];
        for (int j = 1; j < n; ++j) srev[j] = (int8_t)(-s[n - j]);
        CK(cudaMemcpyAsync(c->d_s, s, n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(c->d_srev, srev.data(), n, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        c->have_sk = true;
        return ICHEE_OK;
    }
    if (which == 1) {
        if (bytes != 2 * (size_t)L * polyb) return fail(ICHEE_EINVAL, "public key is %zu bytes, got %zu", 2 * L * polyb, bytes);
        const u64* k = static_cast<const u64*>(host_in);
        for (int b = 0; b < 2; ++b)
            for (int l = 0; l < L; ++l)
                for (int j = 0; j < n; ++j)
                    if (k[((size_t)b * L + l) * n + j] >= c->q[l]) return fail(ICHEE_EINVAL, "public key residue out of range");
        const RnsArgs rl = rns_prefix(c, L);
        CK(cudaMemcpyAsync(c->d_pk, k, 2 * L * polyb, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(c->d_pk_hat, c->d_pk, 2 * L * polyb, cudaMemcpyDeviceToDevice, st));
        CK(launch_ntt_fwd(rl, batch(c->d_pk_hat, 2 * L, L, id.data()), st));
        CK(launch_scale_const(rl, batch(c->d_pk_hat, 2 * L, L, id.data()), c->d_ninv, st));
        CK(launch_shoup_companions(rl, batch(c->d_pk_hat, 2 * L, L, id.data()), c->d_pk_hat_p, st));
        CK(launch_interleave(c->d_pk_hat, c->d_pk_hat_p, (u64)2 * L * c->n, c->d_pk_pair, st));
        CK(cudaStreamSynchronize(st));
        c->have_pk = true;
        return ICHEE_OK;
    }
    if (which == 2) {
        if (!c->P) return fail(ICHEE_EINVAL, "evaluation key needs special_bits > 0");
        const size_t want = (size_t)L * 2 * nm * polyb;
        if (bytes != want) return fail(ICHEE_EINVAL, "evaluation key is %zu bytes, got %zu", want, bytes);
        const u64* k = static_cast<const u64*>(host_in);
        for (int j = 0; j < L; ++j)
            for (int b = 0; b < 2; ++b)
                for (int i = 0; i < nm; ++i)
                    for (int x = 0; x < n; ++x)
                        if (k[(((size_t)j * 2 + b) * nm + i) * n + x] >= c->q[i])
                            return fail(ICHEE_EINVAL, "evaluation key residue out of range");
        if (!c->d_evk) {
            CK(cudaMalloc(&c->d_evk, want));
            CK(cudaMalloc(&c->d_evk_hat, want));
            CK(cudaMalloc(&c->d_evk_hat_p, want));
        }
        const RnsArgs rm = c->rns;
        CK(cudaMemcpyAsync(c->d_evk, k, want, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(c->d_evk_hat, c->d_evk, want, cudaMemcpyDeviceToDevice, st));
        CK(launch_ntt_fwd(rm, batch(c->d_evk_hat, L * 2 * nm, nm, id.data()), st));
        CK(launch_scale_const(rm, batch(c->d_evk_hat, L * 2 * nm, nm, id.data()), c->d_ninv, st));
        CK(launch_shoup_companions(rm, batch(c->d_evk_hat, L * 2 * nm, nm, id.data()), c->d_evk_hat_p, st));
        CK(cudaStreamSynchronize(st));
        c->have_evk = true;
        return ICHEE_OK;
    }
    return fail(ICHEE_EINVAL, "unknown key %d", which);
}

// ---------------------------------------------------------------------------------------
// Encryption (Sec. 2.2.2, 3.1) and cached encryption (Sec. 3.2, 3.3)
// ---------------------------------------------------------------------------------------
EncArgs ichee::enc_args(const ichee_ctx* c, const uint8_t* d_pix, u64 n_ct, u64 seed, u64 id_base, u64* out)
{
    EncArgs a;
    std::memset(&a, 0, sizeof(a));
    a.rns = rns_prefix(c, c->L);
    a.L = c->L;
    a.n_ct = n_ct;
    a.pixels = d_pix;
    a.dm = c->d_dm;
    a.pk_pair = c->d_pk_pair;
    a.skip_lut = nullptr;
    a.seed = seed;
    a.id_base = id_base;
    a.cdt = c->cdt;
    a.out = out;
    a.num_sms = c->num_sms;
    return a;
}

RadixArgs ichee::radix_args(const ichee_ctx* c, const ichee_cache* k, const uint8_t* d_pix, u64 n_ct, u64 seed, u64* out)
{
    RadixArgs a;
    std::memset(&a, 0, sizeof(a));
    for (int l = 0; l < c->L; ++l) a.q[l] = c->q[l];
    a.L = c->L;
    a.logn = c->logn;
    a.n_ct = n_ct;
    a.pixels = d_pix;
    a.mult = k->d_mult;
    a.r = k->radix_base;
    a.n_pow = k->n_pow;
    a.randomize = k->radix_randomize;
    a.pair = k->d_pair;
    a.pair_w = k->pair_w;
    a.seed = seed;
    a.id_base = 0;
    a.out = out;
    return a;
}

LookupArgs ichee::lookup_args(const ichee_ctx* c, const ichee_cache* k, const uint8_t* d_pix, u64 n_ct, u64 seed,
                              u64* out)
{
    LookupArgs a;
    std::memset(&a, 0, sizeof(a));
    for (int l = 0; l < c->L; ++l) a.q[l] = c->q[l];
    a.L = c->L;
    a.logn = c->logn;
    a.n_ct = n_ct;
    a.pixels = d_pix;
    a.lut = k->d_lut;
    a.value_cts = k->d_values;
    a.pool = k->d_pool;
    a.pool_size = k->d_pool ? k->desc.pool_size : 0;
    a.seed = seed;
    a.id_base = 0;
    a.out = out;
    return a;
}

DecArgs ichee::dec_args(const ichee_ctx* c, int nl)
{
    DecArgs a;
    std::memset(&a, 0, sizeof(a));
    a.logn = c->logn;
    for (int l = 0; l < nl; ++l) a.q[l] = c->q[l];
    a.crt = c->crt[nl - 1];
    a.srev = c->d_srev;
    return a;
}

// Encrypt `count` pixel values held on the host into dst with ids id_base + k.
static ichee_status encrypt_values(ichee_ctx* c, const std::vector<uint8_t>& vals, u64 seed, u64 id_base, u64* dst,
                                   cudaStream_t st)
{
    if (vals.empty()) return ICHEE_OK;
    uint8_t* d_v = nullptr;
    CK(cudaMalloc(&d_v, vals.size()));
    cudaError_t e = cudaMemcpyAsync(d_v, vals.data(), vals.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_encrypt_fresh(enc_args(c, d_v, vals.size(), seed, id_base, dst), st);
    cudaStreamSynchronize(st);
    cudaFree(d_v);
    if (e != cudaSuccess) return fail(ICHEE_ECUDA, "cache encryption: %s", cudaGetErrorString(e));
    return ICHEE_OK;
}

// Largest pair table of a radix cache (bytes): beside the lowest positions' multiples it must
// stay resident in the 129 MB L2 while the combine streams its output.
constexpr size_t kRadixPairMaxBytes = size_t(48) << 20;

static ichee_status build_radix(ichee_ctx* c, ichee_cache* k, u32 base, u32 randomize, u64 seed, cudaStream_t st)
{
    int n_pow = 1;
    for (u32 p = base; p <= 255; p *= base) ++n_pow;
    k->radix_base = (int)base;
    k->n_pow = n_pow;
    k->radix_randomize = randomize ? 1 : 0;
    const size_t ctb = ct_words(c, c->L) * 8;
    CK(cudaMalloc(&k->d_radix, n_pow * ctb));
    CK(cudaMalloc(&k->d_mult, (size_t)n_pow * (2 * base + 1) * ctb));
    std::vector<uint8_t> pw(n_pow);
    u32 v = 1;
    for (int i = 0; i < n_pow; ++i, v *= base) pw[i] = (uint8_t)v;
    ichee_status s = encrypt_values(c, pw, seed, kIdRadixBase, k->d_radix, st);
    if (s != ICHEE_OK) return s;
    CK(launch_radix_multiples(k->d_radix, n_pow, (int)base, rns_prefix(c, c->L), c->L, k->d_mult, st));
    // With three or more positions, the top two are also tabulated as sums (one cached read for
    // both in every combine) while the table stays small enough to live in L2 beside the rest.
    // The top signed digit is d + b in [0, 255 / r^(n-1) + randomize].
    if (n_pow >= 3) {
        u32 top = 1;
        for (int i = 0; i < n_pow - 1; ++i) top *= base;
        const int pair_w = (int)(255 / top) + 1 + (randomize ? 1 : 0);
        const size_t bytes = (size_t)(2 * base + 1) * pair_w * ctb;
        if (bytes <= kRadixPairMaxBytes) {
            CK(cudaMalloc(&k->d_pair, bytes));
            k->pair_w = pair_w;
            CK(launch_radix_pairs(k->d_mult, n_pow, (int)base, pair_w, rns_prefix(c, c->L), c->L, k->d_pair, st));
        }
    }
    CK(cudaStreamSynchronize(st));
    return ICHEE_OK;
}

extern "C" ichee_status ichee_build_cache(ichee_ctx* c, const ichee_cache_desc* d, const uint8_t* scan, size_t n_scan,
                                          uint64_t seed, ichee_cache** out, void* stream)
{
    ichee::NvtxRange nvtx_range("ichee_build_cache");
    if (!c || !d || !out) return fail(ICHEE_EINVAL, "null argument");
    *out = nullptr;
    if (!c->have_pk) return fail(ICHEE_EINVAL, "ichee_build_cache: no public key");
    const bool needs_radix = d->kind == ICHEE_CACHE_RADIX || (d->kind == ICHEE_CACHE_FREQ && d->miss_policy == 1);
    if (needs_radix && (d->radix_base < 2 || d->radix_base > 16))
        return fail(ICHEE_EINVAL, "radix_base %u outside [2, 16]", d->radix_base);
    if (d->kind == ICHEE_CACHE_FREQ && (d->top_k < 1 || d->top_k > 256))
        return fail(ICHEE_EINVAL, "top_k %u outside [1, 256]", d->top_k);
    if (d->kind == ICHEE_CACHE_FREQ && d->miss_policy > 1) return fail(ICHEE_EINVAL, "miss_policy %u", d->miss_policy);
    if (d->kind != ICHEE_CACHE_RADIX && d->pool_size > 4096) return fail(ICHEE_EINVAL, "pool_size %u > 4096", d->pool_size);
    if (d->kind == ICHEE_CACHE_FREQ && (!scan || n_scan == 0)) return fail(ICHEE_EINVAL, "scanning cache needs pixels");
    if (d->kind > ICHEE_CACHE_FULL) return fail(ICHEE_EINVAL, "unknown cache kind");
    CK(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;

    ichee_cache* k = new ichee_cache();
    k->ctx = c;
    k->desc = *d;
    for (int i = 0; i < 256; ++i) k->h_lut[i] = -1;
    auto bail = [&](ichee_status s) {
        ichee_cache_free(k);
        return s;
    };
    const size_t ctb = ct_words(c, c->L) * 8;
    if (needs_radix) {
        ichee_status s = build_radix(c, k, d->radix_base, d->kind == ICHEE_CACHE_RADIX ? d->radix_randomize : 1, seed, st);
        if (s != ICHEE_OK) return bail(s);
    }
    if (d->kind != ICHEE_CACHE_RADIX) {
        if (d->kind == ICHEE_CACHE_FULL) {
            for (int v = 0; v < 256; ++v) k->values.push_back(v);
        } else {
            // scanning step: histogram on the device, top-k on the host (count desc, value asc)
            if (is_device_ptr(scan)) {
                ichee_status s = check_span(scan, n_scan, "scan pixels");
                if (s != ICHEE_OK) return bail(s);
            }
            const uint8_t* d_scan = scan;
            uint8_t* tmp = nullptr;
            u32* d_counts = nullptr;
            if (cudaMalloc(&d_counts, 256 * 4) != cudaSuccess) return bail(fail(ICHEE_ENOMEM, "histogram"));
            cudaMemsetAsync(d_counts, 0, 256 * 4, st);
            if (!is_device_ptr(scan)) {
                if (cudaMalloc(&tmp, n_scan) != cudaSuccess) { cudaFree(d_counts); return bail(fail(ICHEE_ENOMEM, "scan")); }
                cudaMemcpyAsync(tmp, scan, n_scan, cudaMemcpyHostToDevice, st);
                d_scan = tmp;
            }
            u32 counts[256];
            cudaError_t e = launch_histogram(d_scan, n_scan, d_counts, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(counts, d_counts, sizeof(counts), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            cudaFree(d_counts);
            if (tmp) cudaFree(tmp);
            if (e != cudaSuccess) return bail(fail(ICHEE_ECUDA, "histogram: %s", cudaGetErrorString(e)));
            std::vector<int> order;
            for (int v = 0; v < 256; ++v)
                if (counts[v]) order.push_back(v);
            std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return counts[a] > counts[b]; });
            if (order.size() > d->top_k) order.resize(d->top_k);
            k->values = order;
        }
        for (size_t j = 0; j < k->values.size(); ++j) k->h_lut[k->values[j]] = (int32_t)j;
        if (cudaMalloc(&k->d_values, std::max<size_t>(1, k->values.size()) * ctb) != cudaSuccess)
            return bail(fail(ICHEE_ENOMEM, "value cache"));
        std::vector<uint8_t> vals(k->values.begin(), k->values.end());
        ichee_status s = encrypt_values(c, vals, seed, 0, k->d_values, st);
        if (s != ICHEE_OK) return bail(s);
        if (d->pool_size) {
            if (cudaMalloc(&k->d_pool, (size_t)d->pool_size * ctb) != cudaSuccess) return bail(fail(ICHEE_ENOMEM, "pool"));
            std::vector<uint8_t> zeros(d->pool_size, 0);
            s = encrypt_values(c, zeros, seed, kIdPoolBase, k->d_pool, st);
            if (s != ICHEE_OK) return bail(s);
        }
    }
    if (cudaMalloc(&k->d_lut, sizeof(k->h_lut)) != cudaSuccess) return bail(fail(ICHEE_ENOMEM, "lut"));
    if (cudaMemcpy(k->d_lut, k->h_lut, sizeof(k->h_lut), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(fail(ICHEE_ECUDA, "lut upload"));
    *out = k;
    return ICHEE_OK;
}

extern "C" void ichee_cache_free(ichee_cache* k)
{
    if (!k) return;
    cudaSetDevice(k->ctx->device);
    cudaDeviceSynchronize();
    void* ptrs[] = {k->d_lut, k->d_values, k->d_pool, k->d_radix, k->d_mult, k->d_pair};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete k;
}

extern "C" ichee_status ichee_cache_info(const ichee_cache* k, uint32_t* n_values, uint8_t* values_out, uint32_t* pool)
{
    if (!k) return fail(ICHEE_EINVAL, "null cache");
    if (n_values) *n_values = (uint32_t)k->values.size();
    if (values_out)
        for (size_t j = 0; j < k->values.size(); ++j) values_out[j] = (uint8_t)k->values[j];
    if (pool) *pool = k->desc.kind == ICHEE_CACHE_RADIX ? 0 : k->desc.pool_size;
    return ICHEE_OK;
}

extern "C" ichee_status ichee_cache_export(const ichee_cache* k, int part, void* host_out, size_t bytes, void* stream)
{
    if (!k || !host_out) return fail(ICHEE_EINVAL, "null argument");
    const ichee_ctx* c = k->ctx;
    CK(cudaSetDevice(c->device));
    const size_t ctb = ct_words(c, c->L) * 8;
    const void* src = nullptr;
    size_t want = 0;
    if (part == 0) { src = k->d_values; want = k->values.size() * ctb; }
    else if (part == 1) { src = k->d_pool; want = (k->d_pool ? k->desc.pool_size : 0) * ctb; }
    else if (part == 2) { src = k->d_radix; want = (size_t)k->n_pow * ctb; }
    else return fail(ICHEE_EINVAL, "unknown part %d", part);
    if (bytes != want) return fail(ICHEE_EINVAL, "part is %zu bytes, got %zu", want, bytes);
    if (want == 0) return ICHEE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(host_out, src, want, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return ICHEE_OK;
}

// Pixels as a device pointer: staged through the context when they live on the host.
static ichee_status device_pixels(ichee_ctx* c, const uint8_t* px, u64 n, cudaStream_t st, const uint8_t** d_px)
{
    if (is_device_ptr(px)) {
        *d_px = px;
        return check_span(px, n, "pixels");
    }
    CK(c->stage_in.ensure(n, c->user_alloc, c->user_free, c->user_alloc_ctx, st));
    CK(cudaMemcpyAsync(c->stage_in.p, px, n, cudaMemcpyHostToDevice, st));
    *d_px = (const uint8_t*)c->stage_in.p;
    return ICHEE_OK;
}

// Pixels k = 0..n_ct-1 into ciphertexts with ct ids first_id + k (fresh, radix or lookup).
static ichee_status encrypt_impl(ichee_ctx* c, const ichee_cache* k, const uint8_t* pixels, u64 n_ct, u64 first_id,
                                 uint64_t seed, uint64_t* d_out, cudaStream_t st)
{
    if (!c->have_pk) return fail(ICHEE_EINVAL, "encryption needs the public key (ichee_keygen or ichee_import_key)");
    if (k && k->ctx != c) return fail(ICHEE_EMISMATCH, "cache belongs to another context");
    CK(cudaSetDevice(c->device));
    ichee_status s = check_out(c, d_out, n_ct, c->L, "ciphertext output");
    if (s != ICHEE_OK) return s;
    const uint8_t* d_px = nullptr;
    s = device_pixels(c, pixels, n_ct, st, &d_px);
    if (s != ICHEE_OK) return s;
    if (!k) {
        CK(launch_encrypt_fresh(enc_args(c, d_px, n_ct, seed, first_id, d_out), st));
    } else if (k->desc.kind == ICHEE_CACHE_RADIX) {
        RadixArgs r = radix_args(c, k, d_px, n_ct, seed, d_out);
        r.id_base = first_id;
        if (first_id == 0) {
            // a whole image runs the batched kernel as a one-image batch (same words; the 64x64
            // image at N = 8192: radix 16 0.319 -> 0.290 ms, radix 10 0.325 -> 0.297 ms)
            SegTable t;
            std::memset(&t, 0, sizeof(t));
            t.n = 1;
            t.start[1] = n_ct;
            t.px[0] = d_px;
            t.out[0] = d_out;
            t.seed[0] = seed;
            CK(launch_radix_combine_batch(r, t, c->shape_radix, c->num_sms, st));
        } else {
            CK(launch_radix_combine(r, st));
        }
    } else {
        LookupArgs a = lookup_args(c, k, d_px, n_ct, seed, d_out);
        a.id_base = first_id;
        CK(launch_lookup_combine(a, st));
        if (k->values.size() < 256) {  // values outside the cache
            if (k->desc.miss_policy == 0) {
                // the misses listed first (a pass over the pixels), then encrypted by the
                // persistent fresh kernel in even shares (2.39 -> 2.38 ms for the top-32 cache
                // of the 64x64 field, 72 % misses)
                EncArgs e = enc_args(c, d_px, n_ct, seed, first_id, d_out);
                if (n_ct < (u64(1) << 32)) {
                    CK(c->scratch.ensure(16 + n_ct * sizeof(u32), c->user_alloc, c->user_free, c->user_alloc_ctx, st));
                    u32* count = (u32*)c->scratch.p;
                    u32* idx = count + 4;
                    CK(launch_miss_list(d_px, n_ct, k->d_lut, idx, count, st));
                    e.idx = idx;
                    e.n_idx = count;
                } else {
                    e.skip_lut = k->d_lut;
                }
                CK(launch_encrypt_fresh(e, st));
            } else {
                RadixArgs r = radix_args(c, k, d_px, n_ct, seed, d_out);
                r.id_base = first_id;
                r.skip_lut = k->d_lut;
                CK(launch_radix_combine(r, st));
            }
        }
    }
    return ICHEE_OK;
}

extern "C" ichee_status ichee_encrypt_image(ichee_ctx* c, const ichee_cache* k, const uint8_t* pixels, uint32_t h,
                                            uint32_t w, uint32_t ch, uint64_t seed, uint64_t* d_out,
                                            ichee_ctimg_meta* meta, void* stream)
{
    ichee::NvtxRange nvtx_range("ichee_encrypt_image");
    if (!c || !pixels || !d_out || !meta) return fail(ICHEE_EINVAL, "null argument");
    const u64 n_ct = image_cts(h, w, ch);
    if (n_ct == 0) return fail(ICHEE_EINVAL, "empty or oversized image %ux%ux%u", h, w, ch);
    ichee_status s = encrypt_impl(c, k, pixels, n_ct, 0, seed, d_out, (cudaStream_t)stream);
    if (s != ICHEE_OK) return s;
    meta->h = h;
    meta->w = w;
    meta->c = ch;
    meta->level = (u32)(c->L - 1);
    meta->scale = c->delta;
    return ICHEE_OK;
}

extern "C" ichee_status ichee_encrypt_pixels(ichee_ctx* c, const ichee_cache* k, const uint8_t* pixels, uint64_t n,
                                             uint64_t first_id, uint64_t seed, uint64_t* d_out, void* stream)
{
    ichee::NvtxRange nvtx_range("ichee_encrypt_pixels");
    if (!c || !pixels || !d_out) return fail(ICHEE_EINVAL, "null argument");
    if (n == 0 || n > (1ull << 40)) return fail(ICHEE_EINVAL, "pixel count %llu outside [1, 2^40]", (unsigned long long)n);
    if (first_id > (1ull << 40)) return fail(ICHEE_EINVAL, "first ciphertext id beyond 2^40");
    return encrypt_impl(c, k, pixels, n, first_id, seed, d_out, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------------------
// Image operations
// ---------------------------------------------------------------------------------------
OpsArgs ichee::ops_base(const ichee_ctx* c, const ichee_ctimg_meta* m)
{
    OpsArgs a;
    std::memset(&a, 0, sizeof(a));
    a.logn = c->logn;
    a.limbs = (int)m->level + 1;
    a.n_ct = (u64)m->h * m->w * m->c;
    for (int l = 0; l < a.limbs; ++l) {
        a.q[l] = c->q[l];
        a.mu[l] = c->rns.mu[l];
    }
    a.h = (int)m->h;
    a.w = (int)m->w;
    a.c = (int)m->c;
    a.y0 = 0;
    a.rows = (int)m->h;
    a.row0 = 0;
    a.status = c->d_status;
    return a;
}

void ichee::set_rescale(const ichee_ctx* c, OpsArgs& a)
{
    const int t = a.limbs - 1;
    const u64 qt = c->q[t];
    a.half_qt = (qt - 1) / 2;
    for (int j = 0; j < t; ++j) {
        const u64 qj = c->q[j];
        a.qt_inv[j] = hm::invm(qt % qj, qj);
        a.qt_inv_p[j] = hm::shoup_of(a.qt_inv[j], qj);
        const u64 r = qt % qj;
        a.neg_qt_mod[j] = r == 0 ? 0 : qj - r;
    }
}

void ichee::set_k0(const ichee_ctx* c, OpsArgs& a, double v, double scale)
{
    encode_const(c, v, scale, a.limbs, a.k0);
    for (int l = 0; l < a.limbs; ++l) a.k0p[l] = hm::shoup_of(a.k0[l], c->q[l]);
}

void ichee::set_k1(const ichee_ctx* c, OpsArgs& a, double v, double scale)
{
    encode_const(c, v, scale, a.limbs, a.k1);
    for (int l = 0; l < a.limbs; ++l) a.k1p[l] = hm::shoup_of(a.k1[l], c->q[l]);
}

// Constants of a fused multiply + rescale: K * q_t^{-1} mod q_j for the kept limbs.
void ichee::fold_constants(const ichee_ctx* c, OpsArgs& a)
{
    const int t = a.limbs - 1;
    a.k0_same = 1;
    int k1_same = 1;
    for (int l = 1; l < a.limbs; ++l) {
        if (a.k0[l] != a.k0[0]) a.k0_same = 0;   // residues < q_l: equal ones are one integer below every q
        if (a.k1[l] != a.k1[0]) k1_same = 0;
    }
    a.k01_same = a.k0_same && k1_same;
    for (int j = 0; j < t; ++j) {
        if (a.k0[0] + a.k1[0] >= 2 * c->q[j]) a.k01_same = 0;
        if (a.k0[0] >= c->q[j] / 4) a.k0_same = 0;   // the mean filter's quotient reaches 4 K
    }
    for (int j = 0; j < t; ++j) {
        const u64 qj = c->q[j];
        a.k0r[j] = hm::mulm(a.k0[j], a.qt_inv[j], qj);
        a.k0rp[j] = hm::shoup_of(a.k0r[j], qj);
        a.k1r[j] = hm::mulm(a.k1[j], a.qt_inv[j], qj);
        a.k1rp[j] = hm::shoup_of(a.k1r[j], qj);
        a.mq[j] = (4 * c->q[t] + qj - 1) / qj * qj;
    }
}

bool ichee::same_scale(double a, double b) { return std::fabs(a - b) <= 1e-9 * std::fabs(a); }

ichee_status ichee::check_img(const ichee_ctx* c, const uint64_t* d, const ichee_ctimg_meta* m, const char* what)
{
    if (!d || !m) return fail(ICHEE_EINVAL, "%s: null operand", what);
    if ((int)m->level >= c->L) return fail(ICHEE_ELEVEL, "%s: level %u >= %d", what, m->level, c->L);
    if (image_cts(m->h, m->w, m->c) == 0) return fail(ICHEE_EINVAL, "%s: empty or oversized image", what);
    if (!(m->scale > 0.0)) return fail(ICHEE_ESCALE, "%s: scale must be positive", what);
    if (!is_device_ptr(d)) return fail(ICHEE_EINVAL, "%s: ciphertexts must be device memory", what);
    return check_span(d, (u64)m->h * m->w * m->c * ct_words(c, (int)m->level + 1) * 8, what);
}

ichee_status ichee::check_out(const ichee_ctx* c, const uint64_t* d, u64 n_ct, int limbs, const char* what)
{
    if (!d || !is_device_ptr(d)) return fail(ICHEE_EINVAL, "%s must be device memory", what);
    return check_span(d, n_ct * ct_words(c, limbs) * 8, what);
}

static ichee_status op_sqdiff(ichee_ctx* c, const uint64_t* d_a, const ichee_ctimg_meta* ma, const uint64_t* d_b,
                              uint64_t* d_out, ichee_ctimg_meta* mout, cudaStream_t st);
static ichee_status op_sqdiff_image(ichee_ctx* c, const uint64_t* d_a, const ichee_ctimg_meta* ma,
                                    const uint64_t* d_b, uint64_t* d_out, ichee_ctimg_meta* mout, cudaStream_t st);

extern "C" ichee_status ichee_eval(ichee_ctx* c, ichee_op op, const uint64_t* d_a, const ichee_ctimg_meta* ma,
                                   const uint64_t* d_b, const ichee_ctimg_meta* mb, const double* args, uint32_t n_args,
                                   uint64_t* d_out, ichee_ctimg_meta* mout, void* stream)
{
    ichee::NvtxRange nvtx_range("ichee_eval");
    if (!c || !mout) return fail(ICHEE_EINVAL, "null argument");
    CK(cudaSetDevice(c->device));
    ichee_status s = check_img(c, d_a, ma, "a");
    if (s != ICHEE_OK) return s;
    {
        // the output holds n_ct ciphertexts (one for the matching sum), one limb fewer after a rescale
        const bool drops = op == ICHEE_OP_RESCALE || op == ICHEE_OP_MEANFILTER3 || op == ICHEE_OP_BLEND ||
                           op == ICHEE_OP_SQDIFF_SUM || op == ICHEE_OP_SQDIFF;
        const u64 out_n = op == ICHEE_OP_SQDIFF_SUM ? 1 : (u64)ma->h * ma->w * ma->c;
        s = check_out(c, d_out, out_n, (int)ma->level + (drops ? 0 : 1), "output");
        if (s != ICHEE_OK) return s;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const bool binary = op == ICHEE_OP_ADD || op == ICHEE_OP_SUB || op == ICHEE_OP_BLEND || op == ICHEE_OP_SQDIFF_SUM ||
                        op == ICHEE_OP_SQDIFF;
    if (binary) {
        s = check_img(c, d_b, mb, "b");
        if (s != ICHEE_OK) return s;
        if (mb->level != ma->level) return fail(ICHEE_ELEVEL, "levels differ (%u vs %u)", ma->level, mb->level);
        if (!same_scale(ma->scale, mb->scale)) return fail(ICHEE_ESCALE, "scales differ (%g vs %g)", ma->scale, mb->scale);
        const bool bcast = op == ICHEE_OP_BLEND && mb->c == 1;
        if (mb->h != ma->h || mb->w != ma->w || (mb->c != ma->c && !bcast))
            return fail(ICHEE_EMISMATCH, "shapes differ");
    }
    const bool in_place_ok = op == ICHEE_OP_PTADD || op == ICHEE_OP_BRIGHTNESS || op == ICHEE_OP_WATERMARK_PIXEL;
    if (d_out == d_a && !in_place_ok) return fail(ICHEE_EINVAL, "this operation cannot run in place");
    OpsArgs a = ops_base(c, ma);
    a.in0 = d_a;
    a.in1 = d_b;
    a.out = d_out;
    ichee_ctimg_meta m = *ma;
    switch (op) {
    case ICHEE_OP_ADD:
    case ICHEE_OP_SUB:
        CK(launch_addsub(a, op == ICHEE_OP_SUB, st));
        break;
    case ICHEE_OP_PTADD:
    case ICHEE_OP_BRIGHTNESS:
    case ICHEE_OP_WATERMARK_PIXEL: {
        if (!args) return fail(ICHEE_EINVAL, "missing op_args");
        std::vector<u64> kadd;
        a.k_lo = 0;
        a.k_hi = a.n_ct;
        if (op == ICHEE_OP_WATERMARK_PIXEL) {
            if (n_args != 2) return fail(ICHEE_EINVAL, "watermark needs (x, index)");
            const double idx = args[1];
            if (!(idx >= 0) || idx >= (double)a.n_ct || idx != std::floor(idx))
                return fail(ICHEE_EINVAL, "watermark index %g outside the image", idx);
            a.k_lo = (u64)idx;
            a.k_hi = a.k_lo + 1;
            kadd.resize(a.limbs);
            encode_const(c, args[0], ma->scale, a.limbs, kadd.data());
        } else if (n_args == 1 || op == ICHEE_OP_BRIGHTNESS) {
            if (n_args != 1) return fail(ICHEE_EINVAL, "brightness needs one argument");
            kadd.resize(a.limbs);
            encode_const(c, args[0], ma->scale, a.limbs, kadd.data());
        } else if (n_args == a.n_ct) {
            kadd.resize((size_t)a.n_ct * a.limbs);
            for (u64 k = 0; k < a.n_ct; ++k) encode_const(c, args[k], ma->scale, a.limbs, kadd.data() + k * a.limbs);
            a.kadd_per_ct = 1;
        } else return fail(ICHEE_EINVAL, "ptadd needs 1 or n_ct arguments, got %u", n_args);
        if (a.kadd_per_ct) {
            CK(c->kadd.ensure(kadd.size() * 8, c->user_alloc, c->user_free, c->user_alloc_ctx, st));
            CK(cudaMemcpyAsync(c->kadd.p, kadd.data(), kadd.size() * 8, cudaMemcpyHostToDevice, st));
            a.kadd = (const u64*)c->kadd.p;
        } else {
            for (int l = 0; l < a.limbs; ++l) a.k0[l] = kadd[l];  // one constant: passed by value
        }
        CK(launch_ptadd(a, st));
        // a per-ciphertext table lives in a staging buffer the next call reuses
        if (a.kadd_per_ct) CK(cudaStreamSynchronize(st));
        break;
    }
    case ICHEE_OP_PTMUL:
        if (!args || n_args != 1) return fail(ICHEE_EINVAL, "ptmul needs one argument");
        set_k0(c, a, args[0], c->delta);
        CK(launch_ptmul(a, st));
        m.scale = ma->scale * c->delta;
        break;
    case ICHEE_OP_RESCALE:
        if (ma->level == 0) return fail(ICHEE_ELEVEL, "no limb left to drop");
        set_rescale(c, a);
        CK(launch_rescale(a, st));
        m.level = ma->level - 1;
        m.scale = ma->scale / (double)c->q[ma->level];
        break;
    case ICHEE_OP_MEANFILTER3:
        if (ma->level == 0) return fail(ICHEE_ELEVEL, "mean filter needs a limb to drop");
        if (c->n / 2 < 256) return fail(ICHEE_EUNSUPPORTED, "mean filter needs N >= 512");
        set_k0(c, a, 1.0 / 9.0, c->delta);
        set_rescale(c, a);
        fold_constants(c, a);
        CK(launch_meanfilter3(a, c->mf_staged != 0, c->num_sms, st));
        m.level = ma->level - 1;
        m.scale = ma->scale * c->delta / (double)c->q[ma->level];
        break;
    case ICHEE_OP_BLEND:
        if (!args || n_args != 1) return fail(ICHEE_EINVAL, "blend needs alpha");
        if (ma->level == 0) return fail(ICHEE_ELEVEL, "blend needs a limb to drop");
        set_k0(c, a, args[0], c->delta);
        set_k1(c, a, 1.0 - args[0], c->delta);
        set_rescale(c, a);
        fold_constants(c, a);
        a.c_w = (int)mb->c;
        CK(launch_blend(a, st));
        m.level = ma->level - 1;
        m.scale = ma->scale * c->delta / (double)c->q[ma->level];
        break;
    case ICHEE_OP_SQDIFF_SUM:
        return op_sqdiff(c, d_a, ma, d_b, d_out, mout, st);
    case ICHEE_OP_SQDIFF:
        if (d_out == d_b) return fail(ICHEE_EINVAL, "this operation cannot run in place");
        return op_sqdiff_image(c, d_a, ma, d_b, d_out, mout, st);
    default:
        return fail(ICHEE_EINVAL, "unknown op %d", (int)op);
    }
    *mout = m;
    return ICHEE_OK;
}

extern "C" ichee_status ichee_meanfilter_rows(ichee_ctx* c, const uint64_t* d_in, const ichee_ctimg_meta* m_img,
                                              uint32_t row0, uint32_t n_rows, uint32_t y0, uint32_t y1,
                                              uint64_t* d_out, ichee_ctimg_meta* mout, void* stream)
{
    ichee::NvtxRange nvtx_range("ichee_meanfilter_rows");
    if (!c || !d_in || !m_img || !mout) return fail(ICHEE_EINVAL, "null argument");
    CK(cudaSetDevice(c->device));
    if ((int)m_img->level >= c->L) return fail(ICHEE_ELEVEL, "level %u >= %d", m_img->level, c->L);
    if (m_img->level == 0) return fail(ICHEE_ELEVEL, "mean filter needs a limb to drop");
    if (image_cts(m_img->h, m_img->w, m_img->c) == 0) return fail(ICHEE_EINVAL, "empty or oversized image");
    if (!(m_img->scale > 0.0)) return fail(ICHEE_ESCALE, "scale must be positive");
    if (c->n / 2 < 256) return fail(ICHEE_EUNSUPPORTED, "mean filter needs N >= 512");
    if (!(y0 < y1 && y1 <= m_img->h)) return fail(ICHEE_EINVAL, "output rows [%u, %u) outside the %u-row image", y0, y1, m_img->h);
    const u32 need0 = y0 > 0 ? y0 - 1 : 0, need1 = y1 < m_img->h ? y1 + 1 : m_img->h;
    if (n_rows == 0 || row0 > need0 || (u64)row0 + n_rows < need1 || (u64)row0 + n_rows > m_img->h)
        return fail(ICHEE_EINVAL, "input rows [%u, %u) do not hold rows [%u, %u) the output needs", row0, row0 + n_rows,
                    need0, need1);
    const u64 row_cts = (u64)m_img->w * m_img->c;
    if (!is_device_ptr(d_in)) return fail(ICHEE_EINVAL, "input must be device memory");
    ichee_status s = check_span(d_in, (u64)n_rows * row_cts * ct_words(c, (int)m_img->level + 1) * 8, "input rows");
    if (s != ICHEE_OK) return s;
    s = check_out(c, d_out, (u64)(y1 - y0) * row_cts, (int)m_img->level, "output rows");
    if (s != ICHEE_OK) return s;
    OpsArgs a = ops_base(c, m_img);
    a.in0 = d_in;
    a.out = d_out;
    a.y0 = (int)y0;
    a.rows = (int)(y1 - y0);
    a.row0 = (int)row0;
    set_k0(c, a, 1.0 / 9.0, c->delta);
    set_rescale(c, a);
    fold_constants(c, a);
    CK(launch_meanfilter3(a, c->mf_staged != 0, c->num_sms, (cudaStream_t)stream));
    *mout = *m_img;
    mout->h = y1 - y0;
    mout->level = m_img->level - 1;
    mout->scale = m_img->scale * c->delta / (double)c->q[m_img->level];
    return ICHEE_OK;
}

// Matching (Sec. 4.4.3, as a squared L2 distance): T = sum_k (a_k - b_k)^2 in the NTT domain,
// INTT, relinearise, rescale. The steps are shared by ICHEE_OP_SQDIFF_SUM, the allocation-free
// entry point and the split form (ichee_sqdiff_accumulate / ichee_sqdiff_finish); they differ
// only in where the working memory comes from.

// Accumulating blocks of the first step: one per SM, rounded down to a multiple of the limbs
// (of twice the limbs in the split form), and the scratch words of one block's slice.
static int sqdiff_unit(const ichee_ctx* c, int limbs) { return sqdiff_split(c->logn) ? 2 * limbs : limbs; }

static int sqdiff_blocks(const ichee_ctx* c, int limbs)
{
    const int u = sqdiff_unit(c, limbs);
    const int nb = (c->num_sms / u) * u;
    return nb < u ? u : nb;
}

static size_t sqdiff_slice_words(const ichee_ctx* c) { return (size_t)(sqdiff_split(c->logn) ? 2 : 4) * c->n; }

// Words of the relinearisation working set: the tensor [3][limbs][N], the key-switching digits,
// the accumulators over Q*P and the relinearised pair.
static size_t relin_words(const ichee_ctx* c, int limbs)
{
    const size_t n = (size_t)c->n;
    return (size_t)3 * limbs * n + (size_t)limbs * (limbs + 1) * n + (size_t)2 * (limbs + 1) * n +
           (size_t)2 * limbs * n;
}

// tensor (= or +=) sum over the pixel pairs of (a - b) (x) (a - b), in the NTT domain (every term
// carries the Montgomery factor 2^-64); partial: n_blocks x 4N words of scratch.
static ichee_status sqdiff_partial_sum(ichee_ctx* c, const uint64_t* d_a, const ichee_ctimg_meta* ma,
                                       const uint64_t* d_b, u64* partial, int n_blocks, u64* tensor, bool add,
                                       cudaStream_t st)
{
    const int limbs = (int)ma->level + 1;
    SqDiffArgs sa;
    std::memset(&sa, 0, sizeof(sa));
    sa.rns = rns_prefix(c, limbs);
    sa.limbs = limbs;
    sa.n_ct = (u64)ma->h * ma->w * ma->c;
    sa.a = d_a;
    sa.b = d_b;
    sa.partial = partial;
    sa.n_blocks = n_blocks;
    for (int h = 0; h < 2; ++h)
        for (int l = 0; l < limbs; ++l) sa.htab[h][l] = c->half_tab[h][l];
    CK(launch_sqdiff_accumulate(sa, st));
    CK(launch_sqdiff_reduce(sa.rns, limbs, partial, n_blocks, tensor, add, st));
    return ICHEE_OK;
}

// tensor (reduced residues, NTT domain, overwritten) -> INTT -> relinearise -> rescale into
// d_out (one ciphertext at level - 1). work: relin_words - 3 limbs N words after the tensor.
static ichee_status sqdiff_relin_rescale(ichee_ctx* c, u64* tensor, const ichee_ctimg_meta* ma, u64* work,
                                         uint64_t* d_out, ichee_ctimg_meta* mout, cudaStream_t st)
{
    const int limbs = (int)ma->level + 1;
    const size_t n = (size_t)c->n;
    const int L = c->L;
    u64* digits = work;
    u64* acc = digits + (size_t)limbs * (limbs + 1) * n;
    u64* rel = acc + (size_t)2 * (limbs + 1) * n;
    int id[kMaxModuli];
    for (int m = 0; m < kMaxModuli; ++m) id[m] = m;
    CK(launch_ntt_inv(c->rns, batch(tensor, 3 * limbs, limbs, id), st));
    CK(launch_scale_const(c->rns, batch(tensor, 3 * limbs, limbs, id), c->d_ninv_r, st));

    RelinArgs ra;
    std::memset(&ra, 0, sizeof(ra));
    ra.rns = c->rns;
    ra.L = L;
    ra.limbs = limbs;
    ra.evk_hat = c->d_evk_hat;
    ra.evk_hat_p = c->d_evk_hat_p;
    for (int m = 0; m < c->nmod; ++m) ra.mu[m] = c->rns.mu[m];
    for (int j = 0; j < limbs; ++j) {
        ra.p_inv[j] = hm::invm(c->P % c->q[j], c->q[j]);
        ra.p_inv_p[j] = hm::shoup_of(ra.p_inv[j], c->q[j]);
        const u64 r = c->P % c->q[j];
        ra.neg_p_mod[j] = r == 0 ? 0 : c->q[j] - r;
    }
    int midx[kMaxModuli];
    for (int m = 0; m < limbs; ++m) midx[m] = m;
    midx[limbs] = L;
    CK(launch_relin_digits(ra, tensor + (size_t)2 * limbs * n, digits, st));
    CK(launch_ntt_fwd(c->rns, batch(digits, limbs * (limbs + 1), limbs + 1, midx), st));
    CK(launch_relin_mac(ra, digits, acc, st));
    CK(launch_ntt_inv(c->rns, batch(acc, 2 * (limbs + 1), limbs + 1, midx), st));
    CK(launch_relin_moddown(ra, tensor, acc, rel, st));

    ichee_ctimg_meta one = *ma;
    one.h = one.w = one.c = 1;
    OpsArgs a = ops_base(c, &one);
    a.in0 = rel;
    a.out = d_out;
    set_rescale(c, a);
    CK(launch_rescale(a, st));
    *mout = one;
    mout->level = ma->level - 1;
    mout->scale = ma->scale * ma->scale / (double)c->q[ma->level];
    return ICHEE_OK;
}

// The whole matching sum in one working block `base`: [tensor | relin work | partial slices].
static ichee_status sqdiff_in(ichee_ctx* c, const uint64_t* d_a, const ichee_ctimg_meta* ma, const uint64_t* d_b,
                              u64* base, int n_blocks, uint64_t* d_out, ichee_ctimg_meta* mout, cudaStream_t st)
{
    const int limbs = (int)ma->level + 1;
    u64* tensor = base;
    u64* work = tensor + (size_t)3 * limbs * c->n;
    u64* partial = base + relin_words(c, limbs);   // the accumulate kernel zeroes its own slices
    ichee_status s = sqdiff_partial_sum(c, d_a, ma, d_b, partial, n_blocks, tensor, false, st);
    if (s != ICHEE_OK) return s;
    return sqdiff_relin_rescale(c, tensor, ma, work, d_out, mout, st);
}

static ichee_status op_sqdiff(ichee_ctx* c, const uint64_t* d_a, const ichee_ctimg_meta* ma, const uint64_t* d_b,
                              uint64_t* d_out, ichee_ctimg_meta* mout, cudaStream_t st)
{
    if (!c->have_evk) return fail(ICHEE_EUNSUPPORTED, "matching needs the evaluation key (ICHEE_WITH_EVK)");
    if (ma->level == 0) return fail(ICHEE_ELEVEL, "matching needs a limb to drop");
    const int limbs = (int)ma->level + 1;
    const int n_blocks = sqdiff_blocks(c, limbs);
    const size_t words = relin_words(c, limbs) + (size_t)n_blocks * sqdiff_slice_words(c);
    CK(c->scratch.ensure(words * 8, c->user_alloc, c->user_free, c->user_alloc_ctx, st));
    return sqdiff_in(c, d_a, ma, d_b, (u64*)c->scratch.p, n_blocks, d_out, mout, st);
}

// Argument checks of the matching entry points outside ichee_eval.
static ichee_status check_match(ichee_ctx* c, const uint64_t* d_a, const ichee_ctimg_meta* ma, const uint64_t* d_b,
                                const ichee_ctimg_meta* mb)
{
    ichee_status s = check_img(c, d_a, ma, "a");
    if (s != ICHEE_OK) return s;
    s = check_img(c, d_b, mb, "b");
    if (s != ICHEE_OK) return s;
    if (mb->level != ma->level) return fail(ICHEE_ELEVEL, "levels differ (%u vs %u)", ma->level, mb->level);
    if (!same_scale(ma->scale, mb->scale)) return fail(ICHEE_ESCALE, "scales differ (%g vs %g)", ma->scale, mb->scale);
    if (mb->h != ma->h || mb->w != ma->w || mb->c != ma->c) return fail(ICHEE_EMISMATCH, "shapes differ");
    if (!c->have_evk) return fail(ICHEE_EUNSUPPORTED, "matching needs the evaluation key (ICHEE_WITH_EVK)");
    if (ma->level == 0) return fail(ICHEE_ELEVEL, "matching needs a limb to drop");
    return ICHEE_OK;
}

extern "C" ichee_status ichee_sqdiff_acc_words(const ichee_ctx* c, uint32_t level, size_t* words)
{
    if (!c || !words) return fail(ICHEE_EINVAL, "null argument");
    if ((int)level >= c->L) return fail(ICHEE_ELEVEL, "level %u >= %d", level, c->L);
    *words = (size_t)3 * (level + 1) * c->n;
    return ICHEE_OK;
}

extern "C" ichee_status ichee_sqdiff_accumulate(ichee_ctx* c, const uint64_t* d_a, const ichee_ctimg_meta* ma,
                                                const uint64_t* d_b, const ichee_ctimg_meta* mb, uint64_t* d_acc,
                                                int accumulate, void* stream)
{
    ichee::NvtxRange nvtx_range("ichee_sqdiff_accumulate");
    if (!c) return fail(ICHEE_EINVAL, "null context");
    CK(cudaSetDevice(c->device));
    ichee_status s = check_match(c, d_a, ma, d_b, mb);
    if (s != ICHEE_OK) return s;
    const int limbs = (int)ma->level + 1;
    const size_t acc_words = (size_t)3 * limbs * c->n;
    if (!d_acc || !is_device_ptr(d_acc)) return fail(ICHEE_EINVAL, "accumulator must be device memory");
    s = check_span(d_acc, acc_words * 8, "accumulator");
    if (s != ICHEE_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int n_blocks = sqdiff_blocks(c, limbs);
    CK(c->scratch.ensure((size_t)n_blocks * sqdiff_slice_words(c) * 8, c->user_alloc, c->user_free, c->user_alloc_ctx,
                         st));
    return sqdiff_partial_sum(c, d_a, ma, d_b, (u64*)c->scratch.p, n_blocks, d_acc, accumulate != 0, st);
}

extern "C" ichee_status ichee_sqdiff_finish(ichee_ctx* c, const uint64_t* d_acc, const ichee_ctimg_meta* m_in,
                                            uint64_t* d_out, ichee_ctimg_meta* mout, void* stream)
{
    ichee::NvtxRange nvtx_range("ichee_sqdiff_finish");
    if (!c || !m_in || !mout) return fail(ICHEE_EINVAL, "null argument");
    CK(cudaSetDevice(c->device));
    if (!c->have_evk) return fail(ICHEE_EUNSUPPORTED, "matching needs the evaluation key (ICHEE_WITH_EVK)");
    if ((int)m_in->level >= c->L) return fail(ICHEE_ELEVEL, "level %u >= %d", m_in->level, c->L);
    if (m_in->level == 0) return fail(ICHEE_ELEVEL, "matching needs a limb to drop");
    if (!(m_in->scale > 0.0)) return fail(ICHEE_ESCALE, "scale must be positive");
    const int limbs = (int)m_in->level + 1;
    const size_t acc_words = (size_t)3 * limbs * c->n;
    if (!d_acc || !is_device_ptr(d_acc)) return fail(ICHEE_EINVAL, "accumulator must be device memory");
    ichee_status s = check_span(d_acc, acc_words * 8, "accumulator");
    if (s != ICHEE_OK) return s;
    s = check_out(c, d_out, 1, limbs - 1, "output");
    if (s != ICHEE_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    CK(c->scratch.ensure(relin_words(c, limbs) * 8, c->user_alloc, c->user_free, c->user_alloc_ctx, st));
    u64* tensor = (u64*)c->scratch.p;
    CK(launch_reduce_rows(c->rns, 3 * limbs, limbs, d_acc, tensor, st));   // sums of accumulators, reduced
    return sqdiff_relin_rescale(c, tensor, m_in, tensor + acc_words, d_out, mout, st);
}

// Per-pixel squared difference (per-pixel form of Sec. 4.4.3): one persistent kernel; each
// block relinearises and rescales one pixel at a time in its own scratch.
static ichee_status op_sqdiff_image(ichee_ctx* c, const uint64_t* d_a, const ichee_ctimg_meta* ma,
                                    const uint64_t* d_b, uint64_t* d_out, ichee_ctimg_meta* mout, cudaStream_t st)
{
    if (!c->have_evk) return fail(ICHEE_EUNSUPPORTED, "squared difference needs the evaluation key (ICHEE_WITH_EVK)");
    if (ma->level == 0) return fail(ICHEE_ELEVEL, "squared difference needs a limb to drop");
    const int limbs = (int)ma->level + 1;
    const int t = limbs - 1;
    const u64 n_ct = (u64)ma->h * ma->w * ma->c;
    const int grid = sqdiff_image_grid(c->logn, n_ct, c->num_sms);
    CK(c->scratch.ensure((size_t)grid * sqdiff_image_scratch_words(c->logn, limbs) * 8, c->user_alloc, c->user_free, c->user_alloc_ctx, st));
    SqImgArgs a;
    std::memset(&a, 0, sizeof(a));
    a.rns = c->rns;
    a.L = c->L;
    a.limbs = limbs;
    a.n_ct = n_ct;
    a.a = d_a;
    a.b = d_b;
    a.out = d_out;
    a.scratch = (u64*)c->scratch.p;
    a.evk_hat = c->d_evk_hat;
    a.evk_hat_p = c->d_evk_hat_p;
    const u64 qt = c->q[t];
    a.half_qt = (qt - 1) / 2;
    for (int j = 0; j < limbs; ++j) {
        const u64 qj = c->q[j];
        const u64 r64 = (u64)(((hm::u128)1 << 64) % qj);   // undoes the tensor's Montgomery 2^{-64}
        a.ninv[j] = hm::mulm(hm::invm((u64)c->n % qj, qj), r64, qj);
        a.ninv_p[j] = hm::shoup_of(a.ninv[j], qj);
        a.pn[j] = hm::mulm(c->P % qj, a.ninv[j], qj);
        a.pn_p[j] = hm::shoup_of(a.pn[j], qj);
        a.r64[j] = r64;
        a.r64_p[j] = hm::shoup_of(r64, qj);
        a.p_inv[j] = hm::invm(c->P % qj, qj);
        a.p_inv_p[j] = hm::shoup_of(a.p_inv[j], qj);
        const u64 r = c->P % qj;
        a.neg_p_mod[j] = r == 0 ? 0 : qj - r;
        if (j < t) {
            a.qt_inv[j] = hm::invm(qt % qj, qj);
            a.qt_inv_p[j] = hm::shoup_of(a.qt_inv[j], qj);
        }
    }
    CK(launch_sqdiff_image(a, grid, st));
    *mout = *ma;
    mout->level = ma->level - 1;
    mout->scale = ma->scale * ma->scale / (double)qt;
    return ICHEE_OK;
}

extern "C" ichee_status ichee_set_allocator(ichee_ctx* c, ichee_alloc_fn alloc, ichee_free_fn free_fn, void* user)
{
    if (!c) return fail(ICHEE_EINVAL, "null context");
    if (alloc && !free_fn) return fail(ICHEE_EINVAL, "an allocator needs its free function");
    CK(cudaSetDevice(c->device));
    CK(cudaDeviceSynchronize());
    for (DevBuf* b : {&c->stage_in, &c->stage_out, &c->stage_res, &c->scratch, &c->kadd}) b->release();
    c->user_alloc = alloc;
    c->user_free = alloc ? free_fn : nullptr;
    c->user_alloc_ctx = alloc ? user : nullptr;
    return ICHEE_OK;
}

// ---------------------------------------------------------------------------------------
// Decryption
// ---------------------------------------------------------------------------------------
// Device address of page-locked host memory the GPU can write directly (null for pageable
// host memory or device memory).
static void* mapped_host_ptr(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// async_out: the output is device memory or page-locked host memory written by the kernel
// itself; nothing is staged and the call does not wait.
static ichee_status decrypt_impl(ichee_ctx* c, const uint64_t* d_ct, const ichee_ctimg_meta* m, double* out,
                                 uint64_t* residues, void* stream, bool async_out)
{
    if (!c || !out) return fail(ICHEE_EINVAL, "null argument");
    if (!c->have_sk) return fail(ICHEE_EINVAL, "no secret key");
    CK(cudaSetDevice(c->device));
    ichee_status s = check_img(c, d_ct, m, "ciphertexts");
    if (s != ICHEE_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const u64 n_ct = (u64)m->h * m->w * m->c;
    const int nl = (int)m->level + 1;
    const bool out_dev = is_device_ptr(out);
    const bool res_dev = residues == nullptr || is_device_ptr(residues);
    if (out_dev && (s = check_span(out, n_ct * 8, "output")) != ICHEE_OK) return s;
    if (residues && res_dev && (s = check_span(residues, n_ct * nl * 8, "residues")) != ICHEE_OK) return s;
    double* direct = out_dev ? out : nullptr;   // written by the kernel in place
    if (async_out && !out_dev) {
        direct = static_cast<double*>(mapped_host_ptr(out));
        if (!direct) return fail(ICHEE_EINVAL, "output must be device or page-locked host memory");
    }
    DecArgs a;
    std::memset(&a, 0, sizeof(a));
    a.logn = c->logn;
    a.n_ct = n_ct;
    for (int l = 0; l < nl; ++l) a.q[l] = c->q[l];
    a.crt = c->crt[nl - 1];
    a.srev = c->d_srev;
    a.ct = d_ct;
    a.scale = m->scale;
    if (direct) a.out = direct;
    else {
        CK(c->stage_out.ensure(n_ct * 8, c->user_alloc, c->user_free, c->user_alloc_ctx, st));
        a.out = (double*)c->stage_out.p;
    }
    if (residues) {
        if (res_dev) a.residues_out = residues;
        else {
            CK(c->stage_res.ensure(n_ct * nl * 8, c->user_alloc, c->user_free, c->user_alloc_ctx, st));
            a.residues_out = (u64*)c->stage_res.p;
        }
    }
    CK(launch_decrypt(a, c->shape_decrypt.threads, st));
    if (!direct) CK(cudaMemcpyAsync(out, a.out, n_ct * 8, cudaMemcpyDeviceToHost, st));
    if (residues && !res_dev) CK(cudaMemcpyAsync(residues, a.residues_out, n_ct * nl * 8, cudaMemcpyDeviceToHost, st));
    if (!direct || (residues && !res_dev)) CK(cudaStreamSynchronize(st));
    return ICHEE_OK;
}

extern "C" ichee_status ichee_decrypt_image(ichee_ctx* c, const uint64_t* d_ct, const ichee_ctimg_meta* m, double* out,
                                            void* stream)
{
    ichee::NvtxRange nvtx_range("ichee_decrypt_image");
    return decrypt_impl(c, d_ct, m, out, nullptr, stream, false);
}

extern "C" ichee_status ichee_decrypt_image_async(ichee_ctx* c, const uint64_t* d_ct, const ichee_ctimg_meta* m,
                                                  double* out, void* stream)
{
    ichee::NvtxRange nvtx_range("ichee_decrypt_image_async");
    return decrypt_impl(c, d_ct, m, out, nullptr, stream, true);
}

extern "C" ichee_status ichee_decrypt_residues(ichee_ctx* c, const uint64_t* d_ct, const ichee_ctimg_meta* m,
                                               double* out, uint64_t* residues, void* stream)
{
    if (!residues) return fail(ICHEE_EINVAL, "null residues");
    return decrypt_impl(c, d_ct, m, out, residues, stream, false);
}

extern "C" ichee_status ichee_stream_status(ichee_ctx* c, void* stream)
{
    if (!c) return fail(ICHEE_EINVAL, "null context");
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    CK(cudaGetLastError());
    int status = 0;
    CK(cudaMemcpy(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status != 0) {
        cudaMemset(c->d_status, 0, sizeof(int));
        return fail(ICHEE_ETIMEOUT, "device status word %d", status);
    }
    return ICHEE_OK;
}

// ---------------------------------------------------------------------------------------
// Matching without device allocation (ichee_sqdiff_sum_noalloc)
//
// For callers that cannot allocate device memory during their work: processes whose HBM is
// handed out by their own arena or a serving framework's pool, and latency-critical loops
// that must not risk the device-wide synchronisation cudaMalloc / cudaFree can cause. The
// scratch that ICHEE_OP_SQDIFF_SUM allocates lives here instead in one file-scope device
// array of ICHEE_NOALLOC_SCRATCH_BYTES, which every GPU that loads this library holds until
// the process exits. Host code cannot use the array's name as a device address; the address
// comes from cudaGetSymbolAddress, once per device, on that device's first call.
// ---------------------------------------------------------------------------------------
#include <mutex>

static __device__ __align__(256) uint64_t g_noalloc_scratch[ICHEE_NOALLOC_SCRATCH_BYTES / 8];

static std::mutex g_noalloc_mu;
static u64* g_noalloc_addr[64] = {};

// Device address of the scratch array for `device` (which must be current).
static ichee_status noalloc_scratch(int device, u64** out)
{
    if (device < 0 || device >= 64) return fail(ICHEE_EINVAL, "device %d out of range", device);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return fail(ICHEE_ECUDA, "cudaGetSymbolAddress(scratch) on device %d: %s", device, cudaGetErrorString(e));
        g_noalloc_addr[device] = (u64*)p;
    }
    *out = g_noalloc_addr[device];
    return ICHEE_OK;
}

extern "C" ichee_status ichee_sqdiff_sum_noalloc(ichee_ctx* c, const uint64_t* d_a, const ichee_ctimg_meta* ma,
                                                 const uint64_t* d_b, const ichee_ctimg_meta* mb, uint64_t* d_out,
                                                 ichee_ctimg_meta* mout, void* stream)
{
    if (!c || !mout) return fail(ICHEE_EINVAL, "null argument");
    CK(cudaSetDevice(c->device));
    ichee_status s = check_match(c, d_a, ma, d_b, mb);
    if (s != ICHEE_OK) return s;
    s = check_out(c, d_out, 1, (int)ma->level, "output");
    if (s != ICHEE_OK) return s;
    if (d_out == d_a || d_out == d_b) return fail(ICHEE_EINVAL, "this operation cannot run in place");
    const int limbs = (int)ma->level + 1;
    const size_t n = (size_t)c->n;
    // fixed part (tensor and relinearisation working set), then one slice per
    // accumulating block, as many blocks as fit (a multiple of limbs)
    const size_t fixed_w = relin_words(c, limbs);
    const size_t cap_w = ICHEE_NOALLOC_SCRATCH_BYTES / 8;
    const size_t slice_w = sqdiff_slice_words(c);
    const size_t fit = fixed_w < cap_w ? (cap_w - fixed_w) / slice_w : 0;
    const int unit = sqdiff_unit(c, limbs);
    int n_blocks = sqdiff_blocks(c, limbs);
    if ((size_t)n_blocks > fit) n_blocks = (int)((fit / unit) * unit);
    if (n_blocks < unit)
        return fail(ICHEE_EINVAL, "matching at N=%zu with %d limbs needs %zu bytes of scratch; the allocation-free "
                    "scratch holds %u bytes", n, limbs, (fixed_w + (size_t)unit * slice_w) * 8,
                    (unsigned)ICHEE_NOALLOC_SCRATCH_BYTES);
    u64* base = nullptr;
    s = noalloc_scratch(c->device, &base);
    if (s != ICHEE_OK) return s;
    return sqdiff_in(c, d_a, ma, d_b, base, n_blocks, d_out, mout, (cudaStream_t)stream);
}
