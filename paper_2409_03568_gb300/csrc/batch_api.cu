// batch_api.cu -- ragged batches of images (many pixel-level ciphertext images per launch),
// the autotuner that picks the launch shapes of the persistent batched kernels, and CUDA-graph
// capture of batched pipelines (include/ichee.h, "Ragged batches").
//
// A batch of n images is cut into chunks of at most kMaxSegs images; each chunk is one launch
// of a persistent kernel whose SegTable (passed as a kernel argument) maps its work items to
// (image, item). Nothing here allocates device memory or synchronises the stream, so a batch
// call can be captured into a CUDA graph.
#include <algorithm>
#include <cmath>

#include "api_internal.h"

using namespace ichee;
namespace hm = ichee::host;

namespace {

u64 n_ct_of(const ichee_image_desc& d) { return image_cts(d.h, d.w, d.c); }

ichee_status check_desc(const ichee_image_desc* images, uint32_t n)
{
    if (!images || n == 0) return fail(ICHEE_EINVAL, "empty batch");
    for (uint32_t i = 0; i < n; ++i)
        if (n_ct_of(images[i]) == 0) return fail(ICHEE_EINVAL, "image %u is empty or oversized", i);
    return ICHEE_OK;
}

// Same level and scale for every image of a batched operation.
ichee_status check_metas(const ichee_ctx* c, const uint64_t* const* d, const ichee_ctimg_meta* m, uint32_t n,
                         const char* what)
{
    if (!d || !m || n == 0) return fail(ICHEE_EINVAL, "%s: empty batch", what);
    char name[64];
    for (uint32_t i = 0; i < n; ++i) {
        if (m[i].level != m[0].level) return fail(ICHEE_ELEVEL, "%s: image %u has another level", what, i);
        std::snprintf(name, sizeof(name), "%s, image %u", what, i);
        const ichee_status s = check_img(c, d[i], &m[i], name);
        if (s != ICHEE_OK) return s;
    }
    return ICHEE_OK;
}

// Pixels of every image: device memory of h*w*c bytes.
ichee_status check_pixels(const uint8_t* const* px, const ichee_image_desc* images, uint32_t n)
{
    char name[48];
    for (uint32_t i = 0; i < n; ++i) {
        if (!is_device_ptr(px[i])) return fail(ICHEE_EINVAL, "pixels of image %u must be device memory", i);
        std::snprintf(name, sizeof(name), "pixels of image %u", i);
        const ichee_status s = check_span(px[i], n_ct_of(images[i]), name);
        if (s != ICHEE_OK) return s;
    }
    return ICHEE_OK;
}

// Output images: device memory for h*w*c ciphertexts of `limbs` limbs each.
template <class Shape>
ichee_status check_outs(const ichee_ctx* c, uint64_t* const* out, const Shape* shapes, uint32_t n, int limbs,
                        const char* what)
{
    char name[64];
    for (uint32_t i = 0; i < n; ++i) {
        std::snprintf(name, sizeof(name), "%s, image %u", what, i);
        const ichee_status s = check_out(c, out[i], (u64)shapes[i].h * shapes[i].w * shapes[i].c, limbs, name);
        if (s != ICHEE_OK) return s;
    }
    return ICHEE_OK;
}

// Fill table segments [first, first + cnt) with `items(i)` work items each.
template <class F>
void fill_starts(SegTable& t, uint32_t first, int cnt, F items)
{
    t.n = cnt;
    t.start[0] = 0;
    for (int s = 0; s < cnt; ++s) t.start[s + 1] = t.start[s] + items(first + s);
}

ichee_status encrypt_chunked(ichee_ctx* c, const ichee_cache* k, const uint8_t* const* px,
                             const ichee_image_desc* images, uint32_t n, uint64_t* const* out, cudaStream_t st)
{
    for (uint32_t first = 0; first < n; first += kMaxSegs) {
        const int cnt = (int)std::min<uint32_t>(kMaxSegs, n - first);
        SegTable t;
        std::memset(&t, 0, sizeof(t));
        fill_starts(t, first, cnt, [&](uint32_t i) { return n_ct_of(images[i]); });
        for (int s = 0; s < cnt; ++s) {
            t.px[s] = px[first + s];
            t.out[s] = out[first + s];
            t.seed[s] = images[first + s].seed;
        }
        if (!k) {
            CK(launch_encrypt_fresh_batch(enc_args(c, nullptr, 0, 0, 0, nullptr), t, c->num_sms, st));
        } else if (k->desc.kind == ICHEE_CACHE_RADIX) {
            CK(launch_radix_combine_batch(radix_args(c, k, nullptr, 0, 0, nullptr), t, c->shape_radix, c->num_sms, st));
        } else {
            CK(launch_lookup_combine_batch(lookup_args(c, k, nullptr, 0, 0, nullptr), t, c->shape_lookup, c->num_sms, st));
            if (k->values.size() < 256) {
                if (k->desc.miss_policy == 0) {
                    EncArgs e = enc_args(c, nullptr, 0, 0, 0, nullptr);
                    e.skip_lut = k->d_lut;
                    CK(launch_encrypt_fresh_batch(e, t, c->num_sms, st));
                } else {
                    RadixArgs r = radix_args(c, k, nullptr, 0, 0, nullptr);
                    r.skip_lut = k->d_lut;
                    CK(launch_radix_combine_batch(r, t, c->shape_radix, c->num_sms, st));
                }
            }
        }
    }
    return ICHEE_OK;
}

ichee_status meanfilter_chunked(ichee_ctx* c, const uint64_t* const* a, const ichee_ctimg_meta* ma, uint64_t* const* out,
                                uint32_t n, LaunchShape ls, cudaStream_t st)
{
    OpsArgs base = ops_base(c, &ma[0]);
    set_k0(c, base, 1.0 / 9.0, c->delta);
    set_rescale(c, base);
    fold_constants(c, base);
    ls.threads = mf_batch_threads(base.limbs, ls.threads, c->mf_staged != 0);
    const int chunks = (c->n / 2) / ls.threads;
    for (uint32_t first = 0; first < n; first += kMaxSegs) {
        const int cnt = (int)std::min<uint32_t>(kMaxSegs, n - first);
        SegTable t;
        std::memset(&t, 0, sizeof(t));
        fill_starts(t, first, cnt, [&](uint32_t i) { return (u64)ma[i].h * chunks * 2 * ma[i].c; });
        for (int s = 0; s < cnt; ++s) {
            const uint32_t i = first + s;
            t.in0[s] = a[i];
            t.out[s] = out[i];
            t.h[s] = ma[i].h;
            t.w[s] = ma[i].w;
            t.c[s] = ma[i].c;
        }
        CK(launch_meanfilter3_batch(base, t, ls, c->mf_staged != 0, c->num_sms, st));
    }
    return ICHEE_OK;
}

ichee_status decrypt_chunked(ichee_ctx* c, const uint64_t* const* d_ct, const ichee_ctimg_meta* m, double* const* out,
                             uint32_t n, LaunchShape ls, cudaStream_t st)
{
    DecArgs base = dec_args(c, (int)m[0].level + 1);
    for (uint32_t first = 0; first < n; first += kMaxSegs) {
        const int cnt = (int)std::min<uint32_t>(kMaxSegs, n - first);
        SegTable t;
        std::memset(&t, 0, sizeof(t));
        fill_starts(t, first, cnt, [&](uint32_t i) { return (u64)m[i].h * m[i].w * m[i].c; });
        for (int s = 0; s < cnt; ++s) {
            t.in0[s] = d_ct[first + s];
            t.dout[s] = out[first + s];
            t.scale[s] = m[first + s].scale;
        }
        CK(launch_decrypt_batch(base, t, ls, c->num_sms, st));
    }
    return ICHEE_OK;
}

ichee_status fused_chunked(ichee_ctx* c, const ichee_cache* k, const uint8_t* const* px, const ichee_image_desc* images,
                           uint32_t n, uint64_t* const* enc, uint64_t* const* filt, LaunchShape ls, cudaStream_t st)
{
    ichee_ctimg_meta m0;
    m0.h = images[0].h;
    m0.w = images[0].w;
    m0.c = images[0].c;
    m0.level = (u32)(c->L - 1);
    m0.scale = c->delta;
    OpsArgs base = ops_base(c, &m0);
    set_k0(c, base, 1.0 / 9.0, c->delta);
    set_rescale(c, base);
    fold_constants(c, base);
    const RadixArgs ra = radix_args(c, k, nullptr, 0, 0, nullptr);
    for (uint32_t first = 0; first < n; first += kMaxSegs) {
        const int cnt = (int)std::min<uint32_t>(kMaxSegs, n - first);
        SegTable t;
        std::memset(&t, 0, sizeof(t));
        fill_starts(t, first, cnt, [&](uint32_t i) {
            return fused_items(c->logn, c->L, ls.threads, images[i].w, images[i].c);
        });
        for (int sg = 0; sg < cnt; ++sg) {
            const uint32_t i = first + sg;
            t.px[sg] = px[i];
            t.out[sg] = enc[i];
            t.out2[sg] = filt[i];
            t.seed[sg] = images[i].seed;
            t.h[sg] = images[i].h;
            t.w[sg] = images[i].w;
            t.c[sg] = images[i].c;
        }
        CK(launch_radix_meanfilter3_batch(ra, base, t, ls, c->num_sms, st));
    }
    return ICHEE_OK;
}

}  // namespace

extern "C" ichee_status ichee_encrypt_meanfilter_batch(ichee_ctx* c, const ichee_cache* k, const uint8_t* const* pixels,
                                                       const ichee_image_desc* images, uint32_t n_images,
                                                       uint64_t* const* d_ct_out, uint64_t* const* d_filtered_out,
                                                       ichee_ctimg_meta* metas_ct, ichee_ctimg_meta* metas_filtered,
                                                       void* stream)
{
    ichee::NvtxRange nvtx_range("ichee_encrypt_meanfilter_batch");
    if (!c || !k || !pixels || !d_ct_out || !d_filtered_out || !metas_ct || !metas_filtered)
        return fail(ICHEE_EINVAL, "null argument");
    if (!c->have_pk) return fail(ICHEE_EINVAL, "no public key (ichee_keygen or ichee_import_key)");
    if (k->ctx != c) return fail(ICHEE_EMISMATCH, "cache belongs to another context");
    if (k->desc.kind != ICHEE_CACHE_RADIX) return fail(ICHEE_EUNSUPPORTED, "the fused pipeline needs a radix cache");
    if (c->L < 2) return fail(ICHEE_ELEVEL, "the mean filter needs a limb to drop");
    ichee_status s = check_desc(images, n_images);
    if (s != ICHEE_OK) return s;
    for (uint32_t i = 0; i < n_images; ++i)
        if (!pixels[i] || !d_ct_out[i] || !d_filtered_out[i]) return fail(ICHEE_EINVAL, "null buffer for image %u", i);
    CK(cudaSetDevice(c->device));
    if ((s = check_pixels(pixels, images, n_images)) != ICHEE_OK) return s;
    if ((s = check_outs(c, d_ct_out, images, n_images, c->L, "ciphertext output")) != ICHEE_OK) return s;
    if ((s = check_outs(c, d_filtered_out, images, n_images, c->L - 1, "filtered output")) != ICHEE_OK) return s;
    if (c->fused_schedule == 1) {
        s = fused_chunked(c, k, pixels, images, n_images, d_ct_out, d_filtered_out, c->shape_fused, (cudaStream_t)stream);
    } else {
        std::vector<ichee_ctimg_meta> m(n_images);
        for (uint32_t i = 0; i < n_images; ++i) {
            m[i].h = images[i].h;
            m[i].w = images[i].w;
            m[i].c = images[i].c;
            m[i].level = (u32)(c->L - 1);
            m[i].scale = c->delta;
        }
        s = encrypt_chunked(c, k, pixels, images, n_images, d_ct_out, (cudaStream_t)stream);
        if (s == ICHEE_OK)
            s = meanfilter_chunked(c, d_ct_out, m.data(), d_filtered_out, n_images, c->shape_meanfilter,
                                   (cudaStream_t)stream);
    }
    if (s != ICHEE_OK) return s;
    for (uint32_t i = 0; i < n_images; ++i) {
        metas_ct[i].h = metas_filtered[i].h = images[i].h;
        metas_ct[i].w = metas_filtered[i].w = images[i].w;
        metas_ct[i].c = metas_filtered[i].c = images[i].c;
        metas_ct[i].level = (u32)(c->L - 1);
        metas_ct[i].scale = c->delta;
        metas_filtered[i].level = (u32)(c->L - 2);
        metas_filtered[i].scale = c->delta * c->delta / (double)c->q[c->L - 1];
    }
    return ICHEE_OK;
}

extern "C" ichee_status ichee_encrypt_batch(ichee_ctx* c, const ichee_cache* k, const uint8_t* const* pixels,
                                            const ichee_image_desc* images, uint32_t n_images,
                                            uint64_t* const* d_ct_out, ichee_ctimg_meta* metas_out, void* stream)
{
    ichee::NvtxRange nvtx_range("ichee_encrypt_batch");
    if (!c || !pixels || !d_ct_out || !metas_out) return fail(ICHEE_EINVAL, "null argument");
    if (!c->have_pk) return fail(ICHEE_EINVAL, "ichee_encrypt_batch: no public key");
    if (k && k->ctx != c) return fail(ICHEE_EMISMATCH, "cache belongs to another context");
    ichee_status s = check_desc(images, n_images);
    if (s != ICHEE_OK) return s;
    for (uint32_t i = 0; i < n_images; ++i)
        if (!pixels[i] || !d_ct_out[i]) return fail(ICHEE_EINVAL, "null buffer for image %u", i);
    CK(cudaSetDevice(c->device));
    if ((s = check_pixels(pixels, images, n_images)) != ICHEE_OK) return s;
    if ((s = check_outs(c, d_ct_out, images, n_images, c->L, "ciphertext output")) != ICHEE_OK) return s;
    s = encrypt_chunked(c, k, pixels, images, n_images, d_ct_out, (cudaStream_t)stream);
    if (s != ICHEE_OK) return s;
    for (uint32_t i = 0; i < n_images; ++i) {
        metas_out[i].h = images[i].h;
        metas_out[i].w = images[i].w;
        metas_out[i].c = images[i].c;
        metas_out[i].level = (u32)(c->L - 1);
        metas_out[i].scale = c->delta;
    }
    return ICHEE_OK;
}

extern "C" ichee_status ichee_eval_batch(ichee_ctx* c, ichee_op op, const uint64_t* const* d_a,
                                         const ichee_ctimg_meta* ma, const uint64_t* const* d_b,
                                         const ichee_ctimg_meta* mb, const double* args, uint32_t n_args,
                                         uint64_t* const* d_out, ichee_ctimg_meta* mout, uint32_t n_images,
                                         void* stream)
{
    ichee::NvtxRange nvtx_range("ichee_eval_batch");
    if (!c || !d_out || !mout) return fail(ICHEE_EINVAL, "null argument");
    CK(cudaSetDevice(c->device));
    ichee_status s = check_metas(c, d_a, ma, n_images, "a");
    if (s != ICHEE_OK) return s;
    for (uint32_t i = 0; i < n_images; ++i) {
        if (!d_out[i]) return fail(ICHEE_EINVAL, "null output for image %u", i);
        if (d_out[i] == d_a[i] && op != ICHEE_OP_BRIGHTNESS && op != ICHEE_OP_PTADD)
            return fail(ICHEE_EINVAL, "only brightness / plaintext add run in place");
        if (!same_scale(ma[i].scale, ma[0].scale)) return fail(ICHEE_ESCALE, "image %u has another scale", i);
    }
    {
        // mean filter and blend drop a limb; brightness / plaintext add keep the level
        const bool drops = op == ICHEE_OP_MEANFILTER3 || op == ICHEE_OP_BLEND;
        if ((s = check_outs(c, d_out, ma, n_images, (int)ma[0].level + (drops ? 0 : 1), "output")) != ICHEE_OK)
            return s;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (op == ICHEE_OP_MEANFILTER3) {
        if (ma[0].level == 0) return fail(ICHEE_ELEVEL, "mean filter needs a limb to drop");
        if (c->n / 2 < c->shape_meanfilter.threads) return fail(ICHEE_EUNSUPPORTED, "ring too small");
        s = meanfilter_chunked(c, d_a, ma, d_out, n_images, c->shape_meanfilter, st);
        if (s != ICHEE_OK) return s;
        for (uint32_t i = 0; i < n_images; ++i) {
            mout[i] = ma[i];
            mout[i].level = ma[i].level - 1;
            mout[i].scale = ma[i].scale * c->delta / (double)c->q[ma[i].level];
        }
        return ICHEE_OK;
    }
    if (op == ICHEE_OP_BRIGHTNESS || op == ICHEE_OP_PTADD) {
        if (!args || n_args != n_images) return fail(ICHEE_EINVAL, "one constant per image expected");
        OpsArgs base = ops_base(c, &ma[0]);
        for (uint32_t first = 0; first < n_images; first += kMaxSegs) {
            const int cnt = (int)std::min<uint32_t>(kMaxSegs, n_images - first);
            SegTable t;
            std::memset(&t, 0, sizeof(t));
            fill_starts(t, first, cnt, [&](uint32_t i) { return (u64)ma[i].h * ma[i].w * ma[i].c; });
            for (int sg = 0; sg < cnt; ++sg) {
                const uint32_t i = first + sg;
                t.in0[sg] = d_a[i];
                t.out[sg] = d_out[i];
                encode_const(c, args[i], ma[i].scale, base.limbs, t.kadd[sg]);
            }
            CK(launch_ptadd_batch(base, t, c->shape_ptadd, c->num_sms, st));
        }
        for (uint32_t i = 0; i < n_images; ++i) mout[i] = ma[i];
        return ICHEE_OK;
    }
    if (op == ICHEE_OP_BLEND) {
        if (!args || n_args != 1) return fail(ICHEE_EINVAL, "blend needs alpha");
        s = check_metas(c, d_b, mb, n_images, "b");
        if (s != ICHEE_OK) return s;
        if (ma[0].level == 0) return fail(ICHEE_ELEVEL, "blend needs a limb to drop");
        for (uint32_t i = 0; i < n_images; ++i) {
            if (mb[i].level != ma[i].level) return fail(ICHEE_ELEVEL, "image %u: levels differ", i);
            if (!same_scale(ma[i].scale, mb[i].scale)) return fail(ICHEE_ESCALE, "image %u: scales differ", i);
            if (mb[i].h != ma[i].h || mb[i].w != ma[i].w || (mb[i].c != ma[i].c && mb[i].c != 1))
                return fail(ICHEE_EMISMATCH, "image %u: shapes differ", i);
        }
        OpsArgs base = ops_base(c, &ma[0]);
        set_k0(c, base, args[0], c->delta);
        set_k1(c, base, 1.0 - args[0], c->delta);
        set_rescale(c, base);
        fold_constants(c, base);
        for (uint32_t first = 0; first < n_images; first += kMaxSegs) {
            const int cnt = (int)std::min<uint32_t>(kMaxSegs, n_images - first);
            SegTable t;
            std::memset(&t, 0, sizeof(t));
            fill_starts(t, first, cnt, [&](uint32_t i) { return (u64)ma[i].h * ma[i].w * ma[i].c; });
            for (int sg = 0; sg < cnt; ++sg) {
                const uint32_t i = first + sg;
                t.in0[sg] = d_a[i];
                t.in1[sg] = d_b[i];
                t.out[sg] = d_out[i];
                t.c[sg] = ma[i].c;
                t.c1[sg] = mb[i].c;
            }
            CK(launch_blend_batch(base, t, c->shape_blend, c->num_sms, st));
        }
        for (uint32_t i = 0; i < n_images; ++i) {
            mout[i] = ma[i];
            mout[i].level = ma[i].level - 1;
            mout[i].scale = ma[i].scale * c->delta / (double)c->q[ma[i].level];
        }
        return ICHEE_OK;
    }
    return fail(ICHEE_EUNSUPPORTED, "operation %d has no batched form", (int)op);
}

extern "C" ichee_status ichee_decrypt_batch(ichee_ctx* c, const uint64_t* const* d_ct, const ichee_ctimg_meta* metas,
                                            double* const* d_out, uint32_t n_images, void* stream)
{
    ichee::NvtxRange nvtx_range("ichee_decrypt_batch");
    if (!c || !d_out) return fail(ICHEE_EINVAL, "null argument");
    if (!c->have_sk) return fail(ICHEE_EINVAL, "no secret key");
    CK(cudaSetDevice(c->device));
    ichee_status s = check_metas(c, d_ct, metas, n_images, "ciphertexts");
    if (s != ICHEE_OK) return s;
    char name[48];
    for (uint32_t i = 0; i < n_images; ++i) {
        if (!is_device_ptr(d_out[i])) return fail(ICHEE_EINVAL, "output of image %u must be device memory", i);
        std::snprintf(name, sizeof(name), "output of image %u", i);
        if ((s = check_span(d_out[i], (u64)metas[i].h * metas[i].w * metas[i].c * 8, name)) != ICHEE_OK) return s;
    }
    return decrypt_chunked(c, d_ct, metas, d_out, n_images, c->shape_decrypt, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------------------
// Autotuner: time every candidate launch shape of the persistent batched kernels on the
// caller's own batch (CUDA events on the caller's stream, best of two runs each) and keep the
// fastest in the context.
// ---------------------------------------------------------------------------------------
extern "C" ichee_status ichee_autotune_batch(ichee_ctx* c, const ichee_cache* k, const uint8_t* const* pixels,
                                             const ichee_image_desc* images, uint32_t n_images,
                                             uint64_t* const* d_ct, uint64_t* const* d_filtered,
                                             ichee_tune_entry* report, uint32_t* n_report, void* stream)
{
    ichee::NvtxRange nvtx_range("ichee_autotune_batch");
    if (!c || !pixels || !d_ct || !d_filtered) return fail(ICHEE_EINVAL, "null argument");
    if (!c->have_pk) return fail(ICHEE_EINVAL, "no public key (ichee_keygen or ichee_import_key)");
    if (k && k->ctx != c) return fail(ICHEE_EMISMATCH, "cache belongs to another context");
    ichee_status s = check_desc(images, n_images);
    if (s != ICHEE_OK) return s;
    if (c->L < 2) return fail(ICHEE_ELEVEL, "tuning the mean filter needs two limbs");
    for (uint32_t i = 0; i < n_images; ++i)
        if (!pixels[i] || !d_ct[i] || !d_filtered[i]) return fail(ICHEE_EINVAL, "null buffer for image %u", i);
    CK(cudaSetDevice(c->device));
    if ((s = check_pixels(pixels, images, n_images)) != ICHEE_OK) return s;
    if ((s = check_outs(c, d_ct, images, n_images, c->L, "ciphertext output")) != ICHEE_OK) return s;
    if ((s = check_outs(c, d_filtered, images, n_images, c->L - 1, "filtered output")) != ICHEE_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    std::vector<ichee_ctimg_meta> metas(n_images);
    for (uint32_t i = 0; i < n_images; ++i) {
        metas[i].h = images[i].h;
        metas[i].w = images[i].w;
        metas[i].c = images[i].c;
        metas[i].level = (u32)(c->L - 1);
        metas[i].scale = c->delta;
    }
    // blocks_per_sm = 0: one block per work item, the launch shape of the single-image kernels
    const LaunchShape cands[] = {{128, 4}, {128, 8}, {128, 16}, {256, 2}, {256, 4}, {256, 8},
                                 {512, 1}, {512, 2}, {512, 4}, {256, 0}, {512, 0}};
    uint32_t nrep = 0;
    const uint32_t cap = n_report ? *n_report : 0;
    auto time_it = [&](auto&& run, float* best) -> ichee_status {
        *best = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            CK(cudaEventRecord(e0, st));
            ichee_status r = run();
            if (r != ICHEE_OK) return r;
            CK(cudaEventRecord(e1, st));
            CK(cudaEventSynchronize(e1));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            *best = std::min(*best, ms);
        }
        return ICHEE_OK;
    };
    auto record = [&](uint32_t kind, LaunchShape ls, float ms) {
        if (report && nrep < cap) {
            report[nrep].kind = kind;
            report[nrep].threads = (uint32_t)ls.threads;
            report[nrep].blocks_per_sm = (uint32_t)ls.blocks_per_sm;
            report[nrep].ms = ms;
        }
        ++nrep;
    };
    // encryption kernel of this cache kind
    const bool radix = k && k->desc.kind == ICHEE_CACHE_RADIX;
    const bool lookup = k && k->desc.kind != ICHEE_CACHE_RADIX;
    if (radix || lookup) {
        LaunchShape& slot = radix ? c->shape_radix : c->shape_lookup;
        LaunchShape best = slot;
        float best_ms = 1e30f;
        for (const LaunchShape& ls : cands) {
            slot = ls;
            float ms;
            s = time_it([&] { return encrypt_chunked(c, k, pixels, images, n_images, d_ct, st); }, &ms);
            if (s != ICHEE_OK) { slot = best; cudaEventDestroy(e0); cudaEventDestroy(e1); return s; }
            record(radix ? ICHEE_TUNE_RADIX : ICHEE_TUNE_LOOKUP, ls, ms);
            if (ms < best_ms) { best_ms = ms; best = ls; }
        }
        slot = best;
    } else {
        s = encrypt_chunked(c, k, pixels, images, n_images, d_ct, st);
        if (s != ICHEE_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return s; }
    }
    // mean filter (its item count depends on the block width, so it is part of the shape)
    {
        LaunchShape best = c->shape_meanfilter;
        float best_ms = 1e30f;
        for (const LaunchShape& ls : cands) {
            if (c->n / 2 < ls.threads) continue;
            float ms;
            s = time_it([&] { return meanfilter_chunked(c, d_ct, metas.data(), d_filtered, n_images, ls, st); }, &ms);
            if (s != ICHEE_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return s; }
            record(ICHEE_TUNE_MEANFILTER, ls, ms);
            if (ms < best_ms) { best_ms = ms; best = ls; }
        }
        c->shape_meanfilter = best;
    }
    // fused radix encryption + mean filter, and the schedule ichee_encrypt_meanfilter_batch uses
    if (radix) {
        const LaunchShape fcands[] = {{256, 4}, {512, 2}, {1024, 1}, {1024, 2}};
        LaunchShape best = c->shape_fused;
        float best_ms = 1e30f;
        for (const LaunchShape& ls : fcands) {
            float ms;
            s = time_it([&] { return fused_chunked(c, k, pixels, images, n_images, d_ct, d_filtered, ls, st); }, &ms);
            if (s != ICHEE_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return s; }
            record(ICHEE_TUNE_FUSED, ls, ms);
            if (ms < best_ms) { best_ms = ms; best = ls; }
        }
        c->shape_fused = best;
        float two_ms;
        s = time_it([&] {
            ichee_status r = encrypt_chunked(c, k, pixels, images, n_images, d_ct, st);
            return r != ICHEE_OK ? r : meanfilter_chunked(c, d_ct, metas.data(), d_filtered, n_images,
                                                          c->shape_meanfilter, st);
        }, &two_ms);
        if (s != ICHEE_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return s; }
        c->fused_schedule = best_ms < two_ms ? 1 : 0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_report) *n_report = nrep;
    return ICHEE_OK;
}

extern "C" ichee_status ichee_tuned_shape(const ichee_ctx* c, uint32_t kind, uint32_t* threads, uint32_t* blocks_per_sm)
{
    if (!c || !threads || !blocks_per_sm) return fail(ICHEE_EINVAL, "null argument");
    LaunchShape ls;
    switch (kind) {
    case ICHEE_TUNE_RADIX: ls = c->shape_radix; break;
    case ICHEE_TUNE_LOOKUP: ls = c->shape_lookup; break;
    case ICHEE_TUNE_MEANFILTER: ls = c->shape_meanfilter; break;
    case ICHEE_TUNE_FUSED: ls = c->shape_fused; break;
    case ICHEE_TUNE_DECRYPT: ls = c->shape_decrypt; break;
    case ICHEE_TUNE_SCHEDULE: *threads = (uint32_t)c->fused_schedule; *blocks_per_sm = 0; return ICHEE_OK;
    case ICHEE_TUNE_MF_STAGED: *threads = (uint32_t)c->mf_staged; *blocks_per_sm = 0; return ICHEE_OK;
    default: return fail(ICHEE_EINVAL, "unknown kernel kind %u", kind);
    }
    *threads = (uint32_t)ls.threads;
    *blocks_per_sm = (uint32_t)ls.blocks_per_sm;
    return ICHEE_OK;
}

// ---------------------------------------------------------------------------------------
// CUDA graphs of batched pipelines
// ---------------------------------------------------------------------------------------
struct ichee_graph {
    int device = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" ichee_status ichee_graph_begin(ichee_ctx* c, void* stream)
{
    if (!c || !stream) return fail(ICHEE_EINVAL, "capture needs a context and a non-default stream");
    CK(cudaSetDevice(c->device));
    CK(cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeThreadLocal));
    return ICHEE_OK;
}

extern "C" ichee_status ichee_graph_end(ichee_ctx* c, void* stream, ichee_graph** out)
{
    if (!c || !stream || !out) return fail(ICHEE_EINVAL, "null argument");
    *out = nullptr;
    CK(cudaSetDevice(c->device));
    ichee_graph* g = new ichee_graph();
    g->device = c->device;
    cudaError_t e = cudaStreamEndCapture((cudaStream_t)stream, &g->graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) {
        ichee_graph_destroy(g);
        return fail(ICHEE_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    }
    *out = g;
    return ICHEE_OK;
}

extern "C" ichee_status ichee_graph_launch(ichee_graph* g, void* stream)
{
    if (!g) return fail(ICHEE_EINVAL, "null graph");
    CK(cudaSetDevice(g->device));
    CK(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return ICHEE_OK;
}

extern "C" void ichee_graph_destroy(ichee_graph* g)
{
    if (!g) return;
    cudaSetDevice(g->device);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

extern "C" ichee_status ichee_set_tuned_shape(ichee_ctx* c, uint32_t kind, uint32_t threads, uint32_t blocks_per_sm)
{
    if (!c) return fail(ICHEE_EINVAL, "null context");
    if (kind == ICHEE_TUNE_SCHEDULE) {
        if (threads > 1) return fail(ICHEE_EINVAL, "schedule must be 0 (two kernels) or 1 (fused)");
        c->fused_schedule = (int)threads;
        return ICHEE_OK;
    }
    if (kind == ICHEE_TUNE_MF_STAGED) {
        if (threads > 1) return fail(ICHEE_EINVAL, "mean-filter form must be 0 (register walk) or 1 (staged)");
        c->mf_staged = (int)threads;
        return ICHEE_OK;
    }
    const bool wide = kind == ICHEE_TUNE_FUSED || kind == ICHEE_TUNE_DECRYPT;   // 1024 threads allowed
    const bool narrow = kind == ICHEE_TUNE_DECRYPT;                            // 32 and 64 too
    if (!(threads == 128 || threads == 256 || threads == 512 || (wide && threads == 1024) ||
          (narrow && (threads == 32 || threads == 64))))
        return fail(ICHEE_EINVAL, "threads %u not supported for kind %u", threads, kind);
    if (blocks_per_sm > 32) return fail(ICHEE_EINVAL, "blocks_per_sm %u above 32", blocks_per_sm);
    if ((kind == ICHEE_TUNE_MEANFILTER) && (uint32_t)(c->n / 2) < threads)
        return fail(ICHEE_EINVAL, "threads %u above N/2 for the mean filter", threads);
    const LaunchShape ls = {(int)threads, (int)blocks_per_sm};
    switch (kind) {
    case ICHEE_TUNE_RADIX: c->shape_radix = ls; break;
    case ICHEE_TUNE_LOOKUP: c->shape_lookup = ls; break;
    case ICHEE_TUNE_MEANFILTER: c->shape_meanfilter = ls; break;
    case ICHEE_TUNE_FUSED: c->shape_fused = ls; break;
    case ICHEE_TUNE_DECRYPT: c->shape_decrypt = ls; break;
    default: return fail(ICHEE_EINVAL, "unknown kernel kind %u", kind);
    }
    return ICHEE_OK;
}
