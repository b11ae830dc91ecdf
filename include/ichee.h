/*
 * ichee.h -- C ABI of libichee: pixel-level CKKS encryption of images with cached encryption
 * and ciphertext-wise image operations on one GB300 GPU (sm_103a), after Wang et al.,
 * "Enabling Practical and Privacy-Preserving Image Processing" (arXiv 2409.03568; the
 * method is called iCHEETAH there).
 *
 * Conventions for every entry point
 *  - Status: every call returns ICHEE_OK or an error code; argument, level, scale and shape
 *    checks happen before any launch. ichee_last_error() returns a thread-local message for
 *    the last failing call. No call aborts, traps or throws across the ABI.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the default stream). All GPU
 *    work is enqueued asynchronously on it; results are ready when the stream is.
 *  - Memory: ciphertext buffers are caller-owned DEVICE memory (size from ichee_ct_bytes).
 *    Every device buffer a call reads or writes is checked, before any launch, against the
 *    allocation that holds it (the driver's pointer attributes; for virtual-memory mappings the
 *    reserved address range): a buffer that ends before the bytes the call needs gives
 *    ICHEE_EINVAL. Memory the driver does not describe is trusted.
 *    Pixel inputs and decrypted outputs may be host or device memory; host buffers are staged
 *    through library-owned device memory. A decryption into host memory waits for its copy
 *    (ichee_decrypt_image_async does not). Host pixel input follows cudaMemcpyAsync: pageable
 *    memory may be reused when the call returns, page-locked memory once the stream has passed
 *    the call. The staging buffers belong to the context: calls that stage host buffers on
 *    different streams must be ordered between those streams by the caller.
 *    Library-owned state (keys, tables, caches) lives in opaque handles freed by the
 *    matching destroy/free call.
 *  - Layouts: one ciphertext = uint64[2][limbs][N] residues in the coefficient domain
 *    (polynomial b in {c0, c1}, limb l, coefficient i), each residue in [0, q_l). An image of
 *    h x w x c pixels is n_ct = h*w*c consecutive ciphertexts, pixel (y, x, ch) at index
 *    (y*w + x)*c + ch. Pixels are uint8 in the same order.
 *  - Determinism: outputs depend only on (params, key seed, cache seed, per-call seed, pixel
 *    values), never on launch shape or batch composition. Random draws come from
 *    Philox4x32-10 keyed by the seed, countered by (block, stream, ciphertext id).
 *  - Threads: one context may be used from one host thread at a time.
 *  - Streams: a context's working memory (below) is shared by its calls, so calls of one
 *    context that use it -- matching, the per-pixel squared difference, frequent-value
 *    encryption with fresh misses, host-buffer staging -- must be ordered on the device (one
 *    stream per context, or events between streams).
 */
#ifndef ICHEE_H
#define ICHEE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ICHEE_OK = 0,
    ICHEE_EINVAL = 1,        /* bad argument (null pointer, size, range, host pointer where device memory is needed) */
    ICHEE_ENOMEM = 2,        /* device or host allocation failed */
    ICHEE_ECUDA = 3,         /* a CUDA call failed; the message names it */
    ICHEE_ELEVEL = 4,        /* level mismatch or no limb left to drop */
    ICHEE_ESCALE = 5,        /* scale mismatch between operands */
    ICHEE_EMISMATCH = 6,     /* operands or cache belong to another context, or shapes differ */
    ICHEE_ETIMEOUT = 7,      /* a bounded device-side wait ran out (reported by ichee_stream_status) */
    ICHEE_EUNSUPPORTED = 8   /* parameters outside what the kernels implement */
} ichee_status;

#define ICHEE_MAX_PRIMES 8

/*
 * CKKS parameters (Sec. 2.2, parameter table: N, Q, L, Delta). N = 2^log_n with
 * 10 <= log_n <= 14. The ciphertext modulus Q is the product of n_primes primes
 * (1 <= n_primes <= 8): for each prime_bits[i] in order (20..60), the largest prime
 * q < 2^bits with q = 1 mod 2N not already taken. special_bits (0 = none, else 30..61) picks
 * the special prime P of the evaluation key the same way. The scale is Delta = 2^log2_scale
 * (log2_scale <= 55). sigma and gauss_bound (1..31) define the discrete Gaussian error.
 */
typedef struct {
    uint32_t log_n;
    uint32_t n_primes;
    uint32_t prime_bits[ICHEE_MAX_PRIMES];
    uint32_t special_bits;
    uint32_t log2_scale;
    double sigma;
    uint32_t gauss_bound;
} ichee_params;

/* Metadata of an image of ciphertexts: shape, level (limbs - 1) and the scale of the encoded
 * values (Delta for fresh encryptions; changed by plaintext multiply and rescale). */
typedef struct {
    uint32_t h, w, c;
    uint32_t level;
    double scale;
} ichee_ctimg_meta;

/* Caching strategies of Sec. 3.2. */
typedef enum {
    ICHEE_CACHE_RADIX = 0,   /* Enc(r^k) for every power r^k <= 255 */
    ICHEE_CACHE_FREQ = 1,    /* Enc(p) for the top_k most frequent values of a scanned image */
    ICHEE_CACHE_FULL = 2     /* Enc(p) for p = 0..255 */
} ichee_cache_kind;

/*
 * Cache description.
 *  radix_base      RADIX: base r (2..16). FREQ with miss_policy 1: base of the radix fallback.
 *  radix_randomize RADIX (and the FREQ radix fallback): 1 = apply the add/subtract randomness
 *                  of Sec. 3.3 (signed digits), 0 = plain sum of cached powers.
 *  top_k           FREQ: number of values cached (1..256; fewer if the scan has fewer values).
 *  pool_size       FREQ/FULL: encryptions of zero in the randomness pool of Sec. 3.3
 *                  (0 = none, else up to 4096).
 *  miss_policy     FREQ: a value outside the cache is encrypted fresh (0) or radix-encrypted (1).
 */
typedef struct {
    ichee_cache_kind kind;
    uint32_t radix_base;
    uint32_t radix_randomize;
    uint32_t top_k;
    uint32_t pool_size;
    uint32_t miss_policy;
} ichee_cache_desc;

/* Image operations (Sec. 2.2.3 and the case studies of Sec. 4.4). */
typedef enum {
    ICHEE_OP_ADD = 0,            /* a (+) b; same shape, level and scale */
    ICHEE_OP_SUB = 1,            /* a (-) b */
    ICHEE_OP_PTADD = 2,          /* a + v; args: v (one value), or n_ct values (one per ciphertext) */
    ICHEE_OP_PTMUL = 3,          /* a * v; args: v; v encoded as llround(v * Delta); scale *= Delta */
    ICHEE_OP_RESCALE = 4,        /* divide by the last prime with rounding; level - 1; scale /= q_last */
    ICHEE_OP_MEANFILTER3 = 5,    /* Sec. 4.4.1: 3x3 mean, clamp-to-edge borders, x 1/9, rescale */
    ICHEE_OP_BRIGHTNESS = 6,     /* Sec. 4.4.2: + beta on every pixel; args: beta */
    ICHEE_OP_BLEND = 7,          /* alpha * a + (1 - alpha) * b, rescaled; args: alpha; b has c or 1 channels */
    ICHEE_OP_WATERMARK_PIXEL = 8,/* Sec. 4.4.4: + x at one ciphertext; args: x, index */
    ICHEE_OP_SQDIFF_SUM = 9,     /* Sec. 4.4.3: sum over ciphertexts of (a - b)^2, relinearised
                                    with the evaluation key and rescaled; output one ciphertext */
    ICHEE_OP_SQDIFF = 10         /* per-pixel form of Sec. 4.4.3: (a_k - b_k)^2 for every ciphertext,
                                    each relinearised and rescaled; output an image of a's shape at
                                    level - 1, scale = scale^2 / q_level */
} ichee_op;

#define ICHEE_WITH_EVK 1u

typedef struct ichee_ctx ichee_ctx;
typedef struct ichee_cache ichee_cache;

/*
 * Create a context on CUDA device `device` (Sec. 2.2 parameter table): generates the prime
 * chain, transform tables and constant tables and uploads them. Keys are made by
 * ichee_keygen. *out receives a handle owned by the caller (ichee_ctx_destroy). Errors:
 * EINVAL (null pointer, parameter out of range), EUNSUPPORTED (no prime chain), ECUDA, ENOMEM.
 */
ichee_status ichee_ctx_create(const ichee_params* params, int device, ichee_ctx** out);

/* Free a context and everything it owns (NULL is a no-op). Caches built from it must be
 * freed first. Synchronises the device. */
void ichee_ctx_destroy(ichee_ctx* ctx);

/*
 * Report the context's primes: q_out[n_primes] receives q_0..q_{L-1} and *p_out the special
 * prime (0 if none). Either pointer may be NULL. Host memory.
 */
ichee_status ichee_ctx_primes(const ichee_ctx* ctx, uint64_t* q_out, uint64_t* p_out);

/*
 * Key generation (Sec. 2.2.2, KeyGen steps 1-3): secret s ternary, public key
 * pk = (-a*s + e, a), and with flags & ICHEE_WITH_EVK the evaluation key used by
 * ICHEE_OP_SQDIFF_SUM and ICHEE_OP_SQDIFF (hybrid key switching with the special prime; needs
 * special_bits > 0).
 * Deterministic in `seed`. Keys stay in the context (ichee_export_key / ichee_import_key move
 * them out and in). Enqueued on `stream`; the call waits for its own set-up copies. Errors:
 * EINVAL (evk without a special prime), ECUDA.
 */
ichee_status ichee_keygen(ichee_ctx* ctx, uint64_t seed, uint32_t flags, void* stream);

/*
 * Working-memory allocator. By default the library takes the device memory it needs during a
 * call (scratch of matching and of the per-pixel squared difference, the list of misses of a
 * frequent-value cache, staging of host buffers, per-ciphertext constant tables) from
 * cudaMalloc and keeps it for later calls. After
 * ichee_set_allocator those buffers come from alloc(bytes, stream, user), which must return
 * device memory of the context's device usable by work on `stream` (NULL: out of memory, the
 * call fails with ICHEE_ENOMEM), and go back through free_fn(ptr, stream, user), after which the
 * allocator may hand the memory out again only once the work already enqueued on that stream
 * has finished (a stream-ordered caching allocator such as PyTorch's qualifies). alloc = NULL
 * restores cudaMalloc. Buffers held from before are released first (the call synchronises the
 * device). Keys, tables and caches are not affected. Callbacks may be called from any library
 * call on the context, on the calling thread. Errors: EINVAL (free_fn missing).
 */
typedef void* (*ichee_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*ichee_free_fn)(void* ptr, void* stream, void* user);
ichee_status ichee_set_allocator(ichee_ctx* ctx, ichee_alloc_fn alloc, ichee_free_fn free_fn, void* user);

/*
 * Copy a key to host memory for inspection. which: 0 = secret key s as int8[N];
 * 1 = public key as uint64[2][L][N]; 2 = evaluation key as uint64[L][2][L+1][N]
 * (coefficient domain, limb L = the special prime). `bytes` must equal that size.
 * Synchronises `stream`. Errors: EINVAL (size, key absent).
 */
ichee_status ichee_export_key(ichee_ctx* ctx, int which, void* host_out, size_t bytes, void* stream);

/*
 * Load a key exported from a context with the same parameters (same `which` numbering and
 * layout as ichee_export_key), instead of or after ichee_keygen: for resuming from saved keys,
 * or for a context that holds only the public and evaluation keys (it encrypts and evaluates;
 * decryption there fails with EINVAL, as it has no secret key). The transformed forms the
 * kernels use are derived on `stream`; the call synchronises it. Errors: EINVAL (size, a
 * residue not below its modulus, a secret-key coefficient outside {-1, 0, 1}, no special prime
 * for the evaluation key), ENOMEM, ECUDA.
 */
ichee_status ichee_import_key(ichee_ctx* ctx, int which, const void* host_in, size_t bytes, void* stream);

/*
 * Build a cache (Sec. 3.2 radix / scanning / full caching, Sec. 3.3 randomness pool).
 * scan_pixels (host or device, n_scan bytes) is read for ICHEE_CACHE_FREQ only (may be NULL
 * otherwise). Cached ciphertexts are fresh encryptions keyed by `seed`: value slot j uses
 * ciphertext id j, pool zero m uses 2^32 + m, radix power k uses 2^33 + k. A radix cache also
 * tabulates d * Enc(r^k) for |d| <= r and, with three or more powers, the sums of the top two
 * powers' multiples when that table is at most 48 MB (one cached read for both digits; the
 * ciphertexts are the same). *out receives a handle (ichee_cache_free). Waits for
 * the histogram when scanning. Errors: EINVAL, ENOMEM, ECUDA.
 */
ichee_status ichee_build_cache(ichee_ctx* ctx, const ichee_cache_desc* desc, const uint8_t* scan_pixels,
                               size_t n_scan, uint64_t seed, ichee_cache** out, void* stream);

/* Free a cache (NULL is a no-op). Synchronises the device. */
void ichee_cache_free(ichee_cache* cache);

/*
 * Describe a cache: *n_values receives the number of cached values and values_out (may be
 * NULL, else 256 entries) the value of each slot; *pool receives the pool size.
 */
ichee_status ichee_cache_info(const ichee_cache* cache, uint32_t* n_values, uint8_t* values_out, uint32_t* pool);

/*
 * Copy cached ciphertexts to host memory. part 0 = value slots [K][2][L][N], 1 = pool
 * [M][2][L][N], 2 = radix powers [n_pow][2][L][N]. `bytes` must equal the size.
 */
ichee_status ichee_cache_export(const ichee_cache* cache, int part, void* host_out, size_t bytes, void* stream);

/* Bytes of one ciphertext at `level` (2 * (level+1) * N * 8). */
ichee_status ichee_ct_bytes(const ichee_ctx* ctx, uint32_t level, size_t* bytes_per_ct);

/*
 * Pixel-level encryption of an h x w x c uint8 image (Sec. 3.1): one ciphertext per pixel
 * value, encoded as the constant polynomial Delta * p. cache == NULL: fresh public-key
 * encryption (Sec. 2.2.2). Otherwise cached encryption (Sec. 3.2, 3.3) with the cache's
 * randomness; values a scanning cache lacks follow its miss_policy. Ciphertext k uses id k
 * and the randomness of `seed`. pixels: host or device, n_ct bytes. d_ct_out: device,
 * n_ct * ichee_ct_bytes(L-1). meta_out (host) receives the shape, level L-1 and scale Delta.
 * Errors: EINVAL (keys missing, sizes, non-device output), EMISMATCH (cache of another
 * context), ECUDA.
 */
ichee_status ichee_encrypt_image(ichee_ctx* ctx, const ichee_cache* cache, const uint8_t* pixels, uint32_t h,
                                 uint32_t w, uint32_t c, uint64_t seed, uint64_t* d_ct_out,
                                 ichee_ctimg_meta* meta_out, void* stream);

/*
 * Pixel-level encryption of a range of an image (Sec. 3.1), for images split into pieces: pixel
 * tiles streamed through limited memory, or pixel ranges on several GPUs. pixels (host or
 * device, n bytes) are the image's pixels first_id .. first_id + n - 1 in (y, x, channel)
 * order; d_ct_out (device, n ciphertexts at level L-1, scale Delta) receives exactly the
 * ciphertexts first_id .. first_id + n - 1 that ichee_encrypt_image makes for the whole image
 * with the same seed and cache (every random draw is keyed by the ciphertext's index in its
 * image). Errors: EINVAL (null, empty or n > 2^40, first_id > 2^40), EMISMATCH, ECUDA.
 */
ichee_status ichee_encrypt_pixels(ichee_ctx* ctx, const ichee_cache* cache, const uint8_t* pixels, uint64_t n,
                                  uint64_t first_id, uint64_t seed, uint64_t* d_ct_out, void* stream);

/*
 * Apply an image operation (see ichee_op). d_a / d_b / d_out are device ciphertext images
 * described by ma / mb / mout; d_b and mb are used by ADD, SUB, BLEND, SQDIFF_SUM and SQDIFF
 * only.
 * op_args holds the operation's real-valued arguments (host). d_out must not overlap the
 * inputs, except that PTADD, BRIGHTNESS and WATERMARK_PIXEL may run in place (d_out == d_a).
 * d_out holds h*w*c ciphertexts (one for SQDIFF_SUM) at level ma->level, or ma->level - 1 for
 * RESCALE, MEANFILTER3, BLEND, SQDIFF_SUM and SQDIFF (ichee_ct_bytes); a shorter allocation
 * gives EINVAL before any launch.
 * *mout receives the result's shape, level and scale. Errors: EINVAL, ELEVEL (no limb to
 * drop), ESCALE, EMISMATCH (shapes), EUNSUPPORTED (no evaluation key), ENOMEM, ECUDA.
 */
ichee_status ichee_eval(ichee_ctx* ctx, ichee_op op, const uint64_t* d_a, const ichee_ctimg_meta* ma,
                        const uint64_t* d_b, const ichee_ctimg_meta* mb, const double* op_args, uint32_t n_args,
                        uint64_t* d_out, ichee_ctimg_meta* mout, void* stream);

/*
 * Decrypt and decode (Sec. 2.2.2 decryption; a pixel is read from coefficient 0 of
 * c0 + c1*s): exact CRT of the residues to the centered integer, divided by meta->scale, one
 * double per ciphertext. out: host or device, n_ct doubles. Needs the secret key. Errors:
 * EINVAL (no secret key, arguments), ECUDA.
 */
ichee_status ichee_decrypt_image(ichee_ctx* ctx, const uint64_t* d_ct, const ichee_ctimg_meta* meta, double* out,
                                 void* stream);

/*
 * ichee_decrypt_image without waiting: out is device memory or page-locked host memory (from
 * cudaHostAlloc / cudaHostRegister, or a pinned tensor), which the decryption kernel writes
 * directly; the values are ready once `stream` is. Pageable host memory is refused (EINVAL).
 * Errors otherwise as ichee_decrypt_image.
 */
ichee_status ichee_decrypt_image_async(ichee_ctx* ctx, const uint64_t* d_ct, const ichee_ctimg_meta* meta,
                                       double* out, void* stream);

/*
 * Like ichee_decrypt_image, and also writes the residues of coefficient 0 of c0 + c1*s per
 * limb to residues_out (host or device, n_ct * (level+1) uint64).
 */
ichee_status ichee_decrypt_residues(ichee_ctx* ctx, const uint64_t* d_ct, const ichee_ctimg_meta* meta, double* out,
                                    uint64_t* residues_out, void* stream);

/* ------------------------------------------------------------------------------------------
 * Ragged batches. Many images of different shapes go through one launch of a persistent
 * kernel (per chunk of 64 images); every image gets exactly the ciphertexts and results the
 * single-image call would give it. Batched calls take host arrays of DEVICE pointers (one per
 * image), never allocate device memory and never synchronise, so a sequence of them can be
 * captured into a CUDA graph (ichee_graph_begin / ichee_graph_end).
 * ------------------------------------------------------------------------------------------ */

/* One image of a batch: shape and the seed of its encryption randomness. */
typedef struct {
    uint32_t h, w, c;
    uint64_t seed;
} ichee_image_desc;

/*
 * Pixel-level encryption of n_images images (Sec. 3.1; cache semantics as in
 * ichee_encrypt_image). pixels[i]: device, h*w*c bytes; d_ct_out[i]: device, h*w*c
 * ciphertexts at level L-1. Image i equals ichee_encrypt_image(..., images[i].seed, ...).
 * metas_out[i] (host) receives its metadata. Errors: EINVAL, EMISMATCH, ECUDA.
 */
ichee_status ichee_encrypt_batch(ichee_ctx* ctx, const ichee_cache* cache, const uint8_t* const* pixels,
                                 const ichee_image_desc* images, uint32_t n_images, uint64_t* const* d_ct_out,
                                 ichee_ctimg_meta* metas_out, void* stream);

/*
 * A batched image operation over n_images device images of one level and scale:
 * ICHEE_OP_MEANFILTER3 (Sec. 4.4.1), ICHEE_OP_BRIGHTNESS / ICHEE_OP_PTADD (Sec. 4.4.2; args:
 * one constant per image) and ICHEE_OP_BLEND (args: alpha; d_b[i] the pattern of image i with
 * c or 1 channels). Results equal the single-image ichee_eval per image. Outputs must not
 * alias inputs, except that brightness / plaintext add may run in place (d_out[i] == d_a[i]:
 * only coefficient 0 of c0 is rewritten). Other operations return ICHEE_EUNSUPPORTED.
 */
ichee_status ichee_eval_batch(ichee_ctx* ctx, ichee_op op, const uint64_t* const* d_a, const ichee_ctimg_meta* ma,
                              const uint64_t* const* d_b, const ichee_ctimg_meta* mb, const double* op_args,
                              uint32_t n_args, uint64_t* const* d_out, ichee_ctimg_meta* mout, uint32_t n_images,
                              void* stream);

/* Batched decryption (Sec. 2.2.2) of n_images device images of one level into device doubles
 * d_out[i] (h*w*c each), decoded with each image's scale. */
ichee_status ichee_decrypt_batch(ichee_ctx* ctx, const uint64_t* const* d_ct, const ichee_ctimg_meta* metas,
                                 double* const* d_out, uint32_t n_images, void* stream);

/*
 * Radix encryption + 3x3 mean filter of a ragged batch (Sec. 3.2, 3.3, 4.4.1). The fused
 * persistent kernel walks each image strip by strip from top to bottom, rebuilds every pixel's
 * ciphertext once from the radix cache, writes it, and forms the filter's sums in registers and
 * shared memory instead of reading the ciphertexts back from HBM. Which schedule runs -- this fused
 * kernel, or the batched encryption followed by the batched mean filter -- is the autotuner's
 * choice (two kernels until ichee_autotune_batch has timed both). Outputs are identical either
 * way, and to ichee_encrypt_batch followed by ichee_eval_batch(MEANFILTER3):
 * d_ct_out[i] (level L-1) and d_filtered_out[i] (level L-2), all device. Needs a radix cache
 * (else ICHEE_EUNSUPPORTED).
 */
ichee_status ichee_encrypt_meanfilter_batch(ichee_ctx* ctx, const ichee_cache* cache, const uint8_t* const* pixels,
                                            const ichee_image_desc* images, uint32_t n_images,
                                            uint64_t* const* d_ct_out, uint64_t* const* d_filtered_out,
                                            ichee_ctimg_meta* metas_ct, ichee_ctimg_meta* metas_filtered,
                                            void* stream);

/* Kernels whose launch shape the autotuner chooses. */
#define ICHEE_TUNE_RADIX 1u
#define ICHEE_TUNE_LOOKUP 2u
#define ICHEE_TUNE_MEANFILTER 3u
#define ICHEE_TUNE_FUSED 4u
#define ICHEE_TUNE_SCHEDULE 5u   /* ichee_tuned_shape: *threads = 1 if the fused kernel runs, 0 for two kernels */
#define ICHEE_TUNE_DECRYPT 6u    /* decryption, single-image and batched (one block per ciphertext) */
#define ICHEE_TUNE_MF_STAGED 7u  /* mean filter form: threads = 0 (default): each thread loads its input
                                    columns into registers; 1: columns staged in shared memory by bulk copies */

typedef struct {
    uint32_t kind;            /* ICHEE_TUNE_* */
    uint32_t threads;         /* threads per block */
    uint32_t blocks_per_sm;   /* persistent grid = blocks_per_sm x SM count; 0 = one block per work item */
    float ms;                 /* best of two timed runs */
} ichee_tune_entry;

/*
 * Autotuner for the batched encrypt-then-mean-filter pipeline: runs the batched encryption of
 * `cache` (fresh if NULL: nothing to tune), the fused radix pipeline (radix caches) and the
 * batched mean filter on the given batch with
 * every candidate launch shape (threads per block x resident blocks per SM), timed with CUDA
 * events on `stream`, and keeps the fastest shapes in the context for later batched calls.
 * d_ct and d_filtered receive valid outputs (the last run). report (host, *n_report entries,
 * may be NULL) receives every timing; *n_report is set to the number of timings. Synchronises
 * `stream`. Run it before capturing a graph that should use the tuned shapes.
 */
ichee_status ichee_autotune_batch(ichee_ctx* ctx, const ichee_cache* cache, const uint8_t* const* pixels,
                                  const ichee_image_desc* images, uint32_t n_images, uint64_t* const* d_ct,
                                  uint64_t* const* d_filtered, ichee_tune_entry* report, uint32_t* n_report,
                                  void* stream);

/* The launch shape the context currently uses for a kernel kind (ICHEE_TUNE_*). */
ichee_status ichee_tuned_shape(const ichee_ctx* ctx, uint32_t kind, uint32_t* threads, uint32_t* blocks_per_sm);

/*
 * Set the launch shape of a kernel kind (e.g. tuning results saved from an earlier run), or with
 * ICHEE_TUNE_SCHEDULE the encrypt + mean-filter schedule (threads = 1: fused kernel, 0: two
 * kernels; blocks_per_sm ignored). threads: 128, 256 or 512 (the fused kernel also 1024, decryption
 * 32 to 1024 in powers of two);
 * blocks_per_sm: 1..32 resident blocks per SM striding over the work, or 0 for one block per
 * work item. Results do not depend on shapes or schedule. Errors: EINVAL.
 */
ichee_status ichee_set_tuned_shape(ichee_ctx* ctx, uint32_t kind, uint32_t threads, uint32_t blocks_per_sm);

typedef struct ichee_graph ichee_graph;

/*
 * CUDA graphs of batched pipelines. ichee_graph_begin starts capturing `stream` (a
 * non-default stream; thread-local capture); the caller then issues batched calls on it;
 * ichee_graph_end stops the capture and instantiates the graph (*out, freed by
 * ichee_graph_destroy). ichee_graph_launch replays it on any stream: same buffers, same
 * inputs, bit-identical results. Only the batched entry points are meant for capture.
 */
ichee_status ichee_graph_begin(ichee_ctx* ctx, void* stream);
ichee_status ichee_graph_end(ichee_ctx* ctx, void* stream, ichee_graph** out);
ichee_status ichee_graph_launch(ichee_graph* graph, void* stream);
void ichee_graph_destroy(ichee_graph* graph);

/* ------------------------------------------------------------------------------------------
 * Serving: a continuous-batching request loop on one GPU. Requests arrive from any host thread
 * (ichee_server_submit) and run on a worker thread inside the library. The worker admits them
 * in arrival order while a device arena -- the HBM budget, reserved once at start -- has room
 * for their buffers (inputs, ciphertexts, results), and launches every admission round as
 * batched kernels per ring: encryption with the ring's cache, one launch per operation kind,
 * batched decryption, result copy. Rounds are stream-ordered per ring and never wait on the
 * host: requests that arrive while others are on the GPU are admitted as memory and slots
 * free up and join the next round. Keys and caches stay device-resident. Every result is
 * exactly what the single-request entry points give for the same seeds (alone or in a mix).
 * ------------------------------------------------------------------------------------------ */

#define ICHEE_REQ_ENCRYPT 0u     /* encrypt, decrypt: result = decoded pixels */
#define ICHEE_REQ_MEANFILTER 1u  /* encrypt, 3x3 mean filter, decrypt */
#define ICHEE_REQ_BRIGHTNESS 2u  /* encrypt, + arg on every pixel, decrypt */
#define ICHEE_REQ_WATERMARK 3u   /* encrypt image and pattern (pixels2, h x w x 1), blend with alpha = arg, decrypt */
#define ICHEE_REQ_MATCH 4u       /* encrypt both images, sum of squared differences (relinearised), decrypt */

typedef struct {
    uint32_t kind;            /* ICHEE_REQ_* */
    uint32_t ring;            /* index into the server's contexts */
    uint32_t h, w, c;
    uint64_t seed;            /* image encryption seed; the second image uses seed + 1 */
    const uint8_t* pixels;    /* host, h*w*c bytes; must stay valid until the request is done */
    const uint8_t* pixels2;   /* host: watermark pattern (h*w) or the image to match (h*w*c); else NULL */
    double arg;               /* brightness offset, or blend alpha */
    double* result;           /* host: h*w*c doubles (match: 1), written when the request is done */
    uint64_t* ct_out;         /* optional device buffer: receives the result's ciphertexts */
} ichee_request;

typedef struct {
    uint64_t ticket;
    int32_t status;           /* ichee_status of the request */
    uint32_t round_size;      /* requests admitted in the same round */
    double t_submit, t_admit, t_done;   /* seconds, monotonic clock */
} ichee_request_done;

typedef struct {
    uint64_t submitted, served, pixels, rounds, max_inflight, pending, inflight;
    uint64_t arena_bytes, arena_used_bytes, peak_arena_bytes;
} ichee_server_stats;

typedef struct ichee_server ichee_server;

/*
 * Start a server over n_rings contexts (keys made; matching needs the evaluation key) sharing
 * one device, each with its cache (NULL = fresh encryption). Reserves hbm_budget_bytes of
 * device memory and 512 MiB of pinned host staging; at most max_inflight requests (0 = 256)
 * are admitted at once. While the server runs, its worker thread uses the ring contexts and
 * caches: the caller must not use them itself until ichee_server_destroy has returned.
 * Requests whose buffers take more than 1/4 of the budget are served in row tiles, so a request
 * is refused only if one image row (with its halo rows) does not fit the whole budget.
 * Errors: EINVAL, EMISMATCH, ENOMEM, ECUDA.
 */
ichee_status ichee_server_create(ichee_ctx* const* rings, const ichee_cache* const* caches, uint32_t n_rings,
                                 size_t hbm_budget_bytes, uint32_t max_inflight, ichee_server** out);

/* Queue a request (copied; its buffers must stay valid until done). *ticket identifies it.
 * Errors: EINVAL (bad request, or one row of it larger than the budget), EUNSUPPORTED. Never
 * blocks on the GPU. */
ichee_status ichee_server_submit(ichee_server* server, const ichee_request* request, uint64_t* ticket);

/* Wait up to timeout_ms for a request; *out receives its timestamps and status. Returns
 * ICHEE_ETIMEOUT if it is not done yet (call again), else the request's own status. Each
 * ticket can be collected once. */
ichee_status ichee_server_wait(ichee_server* server, uint64_t ticket, uint32_t timeout_ms, ichee_request_done* out);

/* Counters: submitted, served, served pixels, admission rounds, peak concurrency, queue and
 * arena occupancy. A request larger than 1/4 of the budget is served as row tiles (pixel
 * ranges, mean-filter bands with halo rows, matching accumulated tile by tile, results as of
 * the whole request): pending counts requests none of whose tiles has been admitted,
 * max_inflight and inflight count admitted pieces (tiles or whole requests). */
ichee_status ichee_server_stats_get(ichee_server* server, ichee_server_stats* out);

/* Pause (hold != 0) or resume admission. While held, submitted requests queue and nothing new
 * starts; work already admitted finishes. On resume the worker admits everything that fits,
 * in arrival order (a burst arriving during a hold is batched as far as memory allows). */
ichee_status ichee_server_hold(ichee_server* server, int hold);

/* Finish every queued request, stop the worker and free the server (not the contexts). */
void ichee_server_destroy(ichee_server* server);

/*
 * Failure injection for tests (not part of the method), on the host only: the next
 * launch_errors admission rounds launch nothing and fail as a launch error would, and the next
 * query_errors round completions report a device error instead of reading the round's event.
 * Every request of such a round completes with ICHEE_ECUDA; the server keeps serving and
 * ichee_server_destroy returns. No GPU fault is involved. Errors: EINVAL.
 */
ichee_status ichee_server_inject_failure(ichee_server* server, uint32_t launch_errors, uint32_t query_errors);

/*
 * 3x3 mean filter (Sec. 4.4.1, the ICHEE_OP_MEANFILTER3 operation) of a band of rows, for images
 * split into pieces (row tiles streamed through limited memory, or row ranges on several GPUs).
 * m_img describes the whole image (h rows of w x c ciphertexts, level >= 1, scale); d_in (device)
 * holds its rows row0 .. row0 + n_rows - 1, which must include the rows the output needs
 * (y0 - 1 .. y1, clamped to the image). d_out (device, (y1 - y0) * w * c ciphertexts at level - 1)
 * receives output rows y0 .. y1 - 1, equal word for word to those rows of the whole-image
 * operation (borders clamp to the edge of the whole image, not of the band); *mout is their
 * metadata (h = y1 - y0). Errors: EINVAL (rows outside the image or not held, null, short or
 * non-device buffers), ELEVEL, ESCALE, EUNSUPPORTED (N < 512), ECUDA.
 */
ichee_status ichee_meanfilter_rows(ichee_ctx* ctx, const uint64_t* d_in, const ichee_ctimg_meta* m_img, uint32_t row0,
                                   uint32_t n_rows, uint32_t y0, uint32_t y1, uint64_t* d_out,
                                   ichee_ctimg_meta* mout, void* stream);

/*
 * Matching in pieces (Sec. 4.4.3): the sum over all pixel pairs of (a - b) (x) (a - b) is a sum,
 * so it can be formed tile by tile (images streamed through limited memory) or range by range
 * on several GPUs, and relinearised and rescaled once at the end.
 *
 * ichee_sqdiff_acc_words: *words = 3 * (level + 1) * N, the uint64 words of one accumulator.
 *
 * ichee_sqdiff_accumulate: d_acc (device, caller-owned, ichee_sqdiff_acc_words(ma->level)
 * words) receives the sum over the n pixel pairs of d_a, d_b (device images of the same shape,
 * level >= 1 and scale; evaluation key needed) -- overwriting it (accumulate = 0) or adding to the
 * accumulator it holds (accumulate != 0). The accumulator is an internal representation (the
 * transform domain of this library, residues below each prime): only ichee_sqdiff_accumulate and
 * ichee_sqdiff_finish of a context with the same parameters read it. The pixel ranges of the
 * pieces must together cover each pair once; their order does not matter (exact modular sums).
 * Working memory: the context's scratch (as ichee_eval).
 *
 * ichee_sqdiff_finish: relinearise and rescale an accumulator into d_out (device, one
 * ciphertext at level m_in->level - 1; *mout its metadata, shape 1x1x1). d_acc may also be the
 * element-wise uint64 sum, without reduction, of up to 8 accumulators (for example the
 * all-reduce of per-GPU accumulators): its words are reduced first. m_in gives the level and the
 * scale of the matched images (its shape is ignored). The result equals ichee_eval with
 * ICHEE_OP_SQDIFF_SUM over all the pairs, bit for bit.
 *
 * Errors: EINVAL (null or non-device buffers, short buffers), ELEVEL, ESCALE, EMISMATCH,
 * EUNSUPPORTED (no evaluation key), ENOMEM, ECUDA.
 */
ichee_status ichee_sqdiff_acc_words(const ichee_ctx* ctx, uint32_t level, size_t* words);
ichee_status ichee_sqdiff_accumulate(ichee_ctx* ctx, const uint64_t* d_a, const ichee_ctimg_meta* ma,
                                     const uint64_t* d_b, const ichee_ctimg_meta* mb, uint64_t* d_acc, int accumulate,
                                     void* stream);
ichee_status ichee_sqdiff_finish(ichee_ctx* ctx, const uint64_t* d_acc, const ichee_ctimg_meta* m_in,
                                 uint64_t* d_out, ichee_ctimg_meta* mout, void* stream);

/*
 * Matching (the ICHEE_OP_SQDIFF_SUM operation) for callers that cannot allocate device
 * memory: processes whose GPU memory is handed out by their own arena or pool, or loops that
 * must not risk the device-wide synchronisation cudaMalloc / cudaFree can cause. The paper
 * has no counterpart; this is an interface for such callers. Same arguments and result as
 * ichee_eval with ICHEE_OP_SQDIFF_SUM, and the same checks (d_out may not be d_a or d_b)
 * (d_a, d_b: device inputs; d_out: caller's device output of one ciphertext at level - 1;
 * *mout receives its metadata), but no call to
 * cudaMalloc, cudaFree or any other allocating routine: the working memory is one static
 * device array of ICHEE_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds until
 * the process exits. The first call on each device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call before any stream
 * capture. The address is kept for the life of the process, so a device reset
 * (cudaDeviceReset) after the first call is not supported. All calls share the array and it keeps the last call's contents (the kernels
 * overwrite or zero everything they read), so calls that overlap on the GPU -- on different
 * streams, or from different contexts on one device -- race: order them. A shape whose
 * working set exceeds the array fails with ICHEE_EINVAL and a message giving both sizes.
 */
#define ICHEE_NOALLOC_SCRATCH_BYTES (32u << 20)
ichee_status ichee_sqdiff_sum_noalloc(ichee_ctx* ctx, const uint64_t* d_a, const ichee_ctimg_meta* ma,
                                      const uint64_t* d_b, const ichee_ctimg_meta* mb, uint64_t* d_out,
                                      ichee_ctimg_meta* mout, void* stream);

/*
 * Measurement utility (not part of the method): integer throughput of CUDA device `device`,
 * the context of the rooflines of the transform kernels. Runs two register-only kernels for a
 * few tens of milliseconds: 32-bit multiply-adds (*imad_per_s, operations per second over the
 * whole GPU) and the library's forward butterfly with its Shoup product on 60-bit residues
 * (*butterflies_per_s). Synchronous; allocates and frees a small output buffer. Errors: EINVAL,
 * ECUDA.
 */
ichee_status ichee_probe_int_throughput(int device, double* imad_per_s, double* butterflies_per_s);

/*
 * Wait for `stream` and collect errors of work enqueued on it (CUDA launch or execution
 * errors, the context's device-side status word). Returns ICHEE_OK, ICHEE_ECUDA or
 * ICHEE_ETIMEOUT and clears the status word.
 */
ichee_status ichee_stream_status(ichee_ctx* ctx, void* stream);

/*
 * Bytes from `ptr` to the end of the device allocation that holds it (for a caching
 * allocator's block: to the end of its segment; for virtual-memory mappings: to the end of the
 * reserved address range), the bound the entry points check device buffers against.
 * Errors: EINVAL (null argument), EUNSUPPORTED (not device memory, or the driver does not
 * describe the allocation; calls then trust the buffer).
 */
ichee_status ichee_buffer_bytes_left(const void* ptr, size_t* bytes_left);

/* Message of the last failing call on this host thread ("" if none). */
const char* ichee_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ICHEE_H */
