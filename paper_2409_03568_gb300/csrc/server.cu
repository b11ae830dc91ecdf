// server.cu -- continuous-batching request loop (include/ichee.h, "Serving").
//
// Requests (encrypt, mean filter, brightness, watermark, match) arrive from any host thread.
// A worker thread admits them in arrival order while the device arena -- one allocation of
// the HBM budget made at start -- has room for their buffers, and launches every admission
// round as batched kernels: per ring (context), one batched encryption of all new images, one
// batched launch per operation kind, one batched decryption, then the result copy. Rounds are
// stream-ordered per ring and never wait on the host, so requests that arrive while others
// are on the GPU join the next round and their work runs behind or beside the earlier rounds;
// memory returns to the arena as each round's completion event fires.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "api_internal.h"

using namespace ichee;

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with 256-byte granules; free blocks coalesce.
class Arena {
public:
    void reset(size_t size)
    {
        free_.clear();
        size_ = size;
        if (size) free_[0] = size;
        used_ = peak_ = 0;
    }
    bool alloc(size_t bytes, size_t* off)
    {
        bytes = round(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t at = it->first + bytes;
            free_.erase(it);
            if (rest) free_[at] = rest;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = round(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }
    size_t size() const { return size_; }
    static size_t round(size_t b) { return (b + 255) & ~(size_t)255; }

private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0, peak_ = 0;
};

// A request too large for one piece of the arena, served as row bands ("tiles") that are
// admitted one by one: pixel ranges encrypted with their whole-image ciphertext ids, the mean
// filter of a band from its rows plus one halo row on each side, matching accumulated tile by
// tile into one accumulator and relinearised once (ichee_encrypt_pixels, ichee_meanfilter_rows,
// ichee_sqdiff_accumulate / ichee_sqdiff_finish): the same result as the one-piece request.
struct Job {
    ichee_request r;
    uint64_t ticket = 0;
    double t_submit = 0, t_admit = 0;
    uint32_t n_tiles = 0, tiles_done = 0;
    int32_t status = ICHEE_OK;
    size_t off = 0, bytes = 0;       // arena block of the whole request (match: accumulator, result)
    u64* acc = nullptr;              // matching accumulator
    u64* fin = nullptr;              // matching result ciphertext
    double* res = nullptr;           // matching decoded value
    ichee_ctimg_meta m_img{};        // the encrypted image: whole shape, level, scale
};

struct Req {
    uint64_t ticket = 0;
    ichee_request r;
    Job* job = nullptr;              // set for the tiles of a tiled request
    uint32_t tile = 0;               // tile index, output rows [y0, y1), encrypted rows [r0, r1)
    uint32_t y0 = 0, y1 = 0, r0 = 0, r1 = 0;
    size_t job_off = 0;              // first tile: where the job's block starts inside its block
    double t_submit = 0, t_admit = 0, t_done = 0;
    // device block and its parts
    size_t off = 0, bytes = 0, hoff = 0, hbytes = 0;
    uint8_t* pix_a = nullptr;
    uint8_t* pix_b = nullptr;
    u64* ct_a = nullptr;
    u64* ct_b = nullptr;
    u64* ct_op = nullptr;
    double* res = nullptr;
    uint8_t* h_pix = nullptr;  // pinned staging
    double* h_res = nullptr;
    ichee_ctimg_meta ma, mb, mop;
    uint32_t round_size = 0;
    int32_t status = ICHEE_OK;
};

struct Round {
    cudaEvent_t done = nullptr;
    uint32_t ring = 0;
    std::vector<Req*> reqs;
};

// Rounds a ring may have queued on the GPU: one running and one ready behind it. Requests that
// arrive meanwhile wait in the queue and are admitted together in the ring's next round.
constexpr uint32_t kRoundsPerRing = 2;

}  // namespace

struct ichee_server {
    std::vector<ichee_ctx*> rings;
    std::vector<const ichee_cache*> caches;
    int device = 0;
    uint32_t max_inflight = 0;
    u64* d_base = nullptr;
    uint8_t* h_base = nullptr;
    Arena dev, host;
    std::vector<cudaStream_t> streams;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> pending;
    std::unordered_map<uint64_t, Req*> done;
    std::deque<Round> rounds;
    std::vector<uint32_t> ring_rounds;   // rounds in flight per ring
    uint64_t next_ticket = 1;
    uint32_t inflight = 0;
    size_t tile_bytes = 0;           // requests above this footprint are served in row tiles
    bool stop = false;
    bool hold = false;
    std::atomic<uint32_t> inject_launch_errors{0}, inject_query_errors{0};   // ichee_server_inject_failure
    ichee_server_stats stats{};
    std::thread worker;
};

namespace {

size_t ctb(const ichee_ctx* c, int level) { return ct_words(c, level + 1) * 8; }

// Device bytes a request needs (each part 256-byte aligned) and host staging bytes.
void sizes(const ichee_server* s, const ichee_request& r, size_t* dev, size_t* host)
{
    const ichee_ctx* c = s->rings[r.ring];
    const u64 n_ct = (u64)r.h * r.w * r.c;
    const u64 n_b = r.kind == ICHEE_REQ_WATERMARK ? (u64)r.h * r.w : (r.kind == ICHEE_REQ_MATCH ? n_ct : 0);
    const int L = c->L;
    size_t d = Arena::round(n_ct) + Arena::round(n_b) + Arena::round(n_ct * ctb(c, L - 1)) +
               Arena::round(n_b * ctb(c, L - 1));
    switch (r.kind) {
    case ICHEE_REQ_MEANFILTER:
    case ICHEE_REQ_WATERMARK: d += Arena::round(n_ct * ctb(c, L - 2)); break;
    case ICHEE_REQ_MATCH: d += Arena::round(ctb(c, L - 2)); break;
    default: break;   // brightness runs in place on the encrypted image
    }
    const u64 n_res = r.kind == ICHEE_REQ_MATCH ? 1 : n_ct;
    d += Arena::round(n_res * 8);
    *dev = d;
    *host = Arena::round(n_ct + n_b) + Arena::round(n_res * 8);
}

// Device and host bytes of one tile of request r: output rows [y0, y1), encrypted rows
// [r0, r1) (the mean filter's band plus halo).
void tile_sizes(const ichee_server* s, const ichee_request& r, uint32_t y0, uint32_t y1, uint32_t r0, uint32_t r1,
                size_t* dev, size_t* host)
{
    const ichee_ctx* c = s->rings[r.ring];
    const int L = c->L;
    const u64 row = (u64)r.w * r.c;
    const u64 n_in = (u64)(r1 - r0) * row, n_out = (u64)(y1 - y0) * row;
    const u64 n_b = r.kind == ICHEE_REQ_WATERMARK ? (u64)(r1 - r0) * r.w : (r.kind == ICHEE_REQ_MATCH ? n_in : 0);
    size_t d = Arena::round(n_in) + Arena::round(n_b) + Arena::round(n_in * ctb(c, L - 1)) +
               Arena::round(n_b * ctb(c, L - 1));
    if (r.kind == ICHEE_REQ_MEANFILTER || r.kind == ICHEE_REQ_WATERMARK) d += Arena::round(n_out * ctb(c, L - 2));
    const u64 n_res = r.kind == ICHEE_REQ_MATCH ? 1 : n_out;
    d += Arena::round(n_res * 8);
    *dev = d;
    *host = Arena::round(n_in + n_b) + Arena::round(n_res * 8);
}

// Arena bytes a tiled request holds from its first tile to its last (matching: accumulator,
// result ciphertext and decoded value).
size_t job_bytes(const ichee_server* s, const ichee_request& r)
{
    if (r.kind != ICHEE_REQ_MATCH) return 0;
    const ichee_ctx* c = s->rings[r.ring];
    return Arena::round((size_t)3 * c->L * c->n * 8) + Arena::round(ctb(c, c->L - 2)) + Arena::round(8);
}

// Encrypted rows of the tile with output rows [y0, y1).
void tile_rows(const ichee_request& r, uint32_t y0, uint32_t y1, uint32_t* r0, uint32_t* r1)
{
    const bool halo = r.kind == ICHEE_REQ_MEANFILTER;
    *r0 = halo && y0 > 0 ? y0 - 1 : y0;
    *r1 = halo && y1 < r.h ? y1 + 1 : y1;
}

void carve_tile(ichee_server* s, Req* q)
{
    const ichee_ctx* c = s->rings[q->r.ring];
    const ichee_request& r = q->r;
    const int L = c->L;
    const u64 row = (u64)r.w * r.c;
    const u64 n_in = (u64)(q->r1 - q->r0) * row, n_out = (u64)(q->y1 - q->y0) * row;
    const u64 n_b = r.kind == ICHEE_REQ_WATERMARK ? (u64)(q->r1 - q->r0) * r.w : (r.kind == ICHEE_REQ_MATCH ? n_in : 0);
    uint8_t* p = reinterpret_cast<uint8_t*>(s->d_base) + q->off;
    q->pix_a = p; p += Arena::round(n_in);
    q->pix_b = n_b ? p : nullptr; p += Arena::round(n_b);
    q->ct_a = reinterpret_cast<u64*>(p); p += Arena::round(n_in * ctb(c, L - 1));
    q->ct_b = n_b ? reinterpret_cast<u64*>(p) : nullptr; p += Arena::round(n_b * ctb(c, L - 1));
    q->ct_op = r.kind == ICHEE_REQ_BRIGHTNESS ? q->ct_a : nullptr;
    if (r.kind == ICHEE_REQ_MEANFILTER || r.kind == ICHEE_REQ_WATERMARK) {
        q->ct_op = reinterpret_cast<u64*>(p);
        p += Arena::round(n_out * ctb(c, L - 2));
    }
    q->res = reinterpret_cast<double*>(p);
    q->h_pix = s->h_base + q->hoff;
    q->h_res = reinterpret_cast<double*>(s->h_base + q->hoff + Arena::round(n_in + n_b));
    if (q->tile == 0 && q->job->bytes) {   // the job's block follows the first tile's
        Job* j = q->job;
        j->off = q->off + q->job_off;
        uint8_t* jp = reinterpret_cast<uint8_t*>(s->d_base) + j->off;
        j->acc = reinterpret_cast<u64*>(jp); jp += Arena::round((size_t)3 * c->L * c->n * 8);
        j->fin = reinterpret_cast<u64*>(jp); jp += Arena::round(ctb(c, L - 2));
        j->res = reinterpret_cast<double*>(jp);
    }
}

void carve(ichee_server* s, Req* q)
{
    if (q->job) {
        carve_tile(s, q);
        return;
    }
    const ichee_ctx* c = s->rings[q->r.ring];
    const ichee_request& r = q->r;
    const u64 n_ct = (u64)r.h * r.w * r.c;
    const u64 n_b = r.kind == ICHEE_REQ_WATERMARK ? (u64)r.h * r.w : (r.kind == ICHEE_REQ_MATCH ? n_ct : 0);
    const int L = c->L;
    uint8_t* p = reinterpret_cast<uint8_t*>(s->d_base) + q->off;
    q->pix_a = p; p += Arena::round(n_ct);
    q->pix_b = n_b ? p : nullptr; p += Arena::round(n_b);
    q->ct_a = reinterpret_cast<u64*>(p); p += Arena::round(n_ct * ctb(c, L - 1));
    q->ct_b = n_b ? reinterpret_cast<u64*>(p) : nullptr; p += Arena::round(n_b * ctb(c, L - 1));
    q->ct_op = nullptr;
    switch (r.kind) {
    case ICHEE_REQ_MEANFILTER:
    case ICHEE_REQ_WATERMARK: q->ct_op = reinterpret_cast<u64*>(p); p += Arena::round(n_ct * ctb(c, L - 2)); break;
    case ICHEE_REQ_BRIGHTNESS: q->ct_op = q->ct_a; break;   // in place
    case ICHEE_REQ_MATCH: q->ct_op = reinterpret_cast<u64*>(p); p += Arena::round(ctb(c, L - 2)); break;
    default: break;
    }
    q->res = reinterpret_cast<double*>(p);
    q->h_pix = s->h_base + q->hoff;
    q->h_res = reinterpret_cast<double*>(s->h_base + q->hoff + Arena::round(n_ct + n_b));
}

// One tile of a tiled request, by the single-image entry points on the ring's stream.
ichee_status launch_tile(ichee_server* s, ichee_ctx* c, const ichee_cache* k, Req* q, cudaStream_t st)
{
    const ichee_request& r = q->r;
    Job* j = q->job;
    const u64 row = (u64)r.w * r.c;
    const u64 n_in = (u64)(q->r1 - q->r0) * row, n_out = (u64)(q->y1 - q->y0) * row;
    const u64 n_b = q->pix_b ? (r.kind == ICHEE_REQ_WATERMARK ? (u64)(q->r1 - q->r0) * r.w : n_in) : 0;
    const u64 b_first = r.kind == ICHEE_REQ_WATERMARK ? (u64)q->r0 * r.w : (u64)q->r0 * row;
    std::memcpy(q->h_pix, r.pixels + (u64)q->r0 * row, n_in);
    if (n_b) std::memcpy(q->h_pix + n_in, r.pixels2 + b_first, n_b);
    CK(cudaMemcpyAsync(q->pix_a, q->h_pix, n_in, cudaMemcpyHostToDevice, st));
    if (n_b) CK(cudaMemcpyAsync(q->pix_b, q->h_pix + n_in, n_b, cudaMemcpyHostToDevice, st));
    ichee_status e = ichee_encrypt_pixels(c, k, q->pix_a, n_in, (u64)q->r0 * row, r.seed, q->ct_a, st);
    if (e != ICHEE_OK) return e;
    if (n_b) {
        e = ichee_encrypt_pixels(c, k, q->pix_b, n_b, b_first, r.seed + 1, q->ct_b, st);
        if (e != ICHEE_OK) return e;
    }
    ichee_ctimg_meta band = j->m_img;   // the encrypted rows as an image
    band.h = q->r1 - q->r0;
    const u64* out = q->ct_a;
    ichee_ctimg_meta mo = band;
    switch (r.kind) {
    case ICHEE_REQ_MEANFILTER:
        e = ichee_meanfilter_rows(c, q->ct_a, &j->m_img, q->r0, q->r1 - q->r0, q->y0, q->y1, q->ct_op, &mo, st);
        out = q->ct_op;
        break;
    case ICHEE_REQ_BRIGHTNESS:
        e = ichee_eval(c, ICHEE_OP_BRIGHTNESS, q->ct_a, &band, nullptr, nullptr, &r.arg, 1, q->ct_a, &mo, st);
        break;
    case ICHEE_REQ_WATERMARK: {
        ichee_ctimg_meta mb = band;
        mb.c = 1;
        e = ichee_eval(c, ICHEE_OP_BLEND, q->ct_a, &band, q->ct_b, &mb, &r.arg, 1, q->ct_op, &mo, st);
        out = q->ct_op;
        break;
    }
    case ICHEE_REQ_MATCH:
        e = ichee_sqdiff_accumulate(c, q->ct_a, &band, q->ct_b, &band, j->acc, q->tile > 0 ? 1 : 0, st);
        if (e == ICHEE_OK && q->tile + 1 == j->n_tiles) {
            e = ichee_sqdiff_finish(c, j->acc, &j->m_img, j->fin, &mo, st);
            if (e == ICHEE_OK) e = ichee_decrypt_image(c, j->fin, &mo, j->res, st);
            if (e == ICHEE_OK && r.ct_out) CK(cudaMemcpyAsync(r.ct_out, j->fin, ctb(c, (int)mo.level), cudaMemcpyDeviceToDevice, st));
            if (e == ICHEE_OK) CK(cudaMemcpyAsync(q->h_res, j->res, 8, cudaMemcpyDeviceToHost, st));
        }
        return e;
    default:
        break;
    }
    if (e != ICHEE_OK) return e;
    e = ichee_decrypt_image(c, out, &mo, q->res, st);
    if (e != ICHEE_OK) return e;
    if (r.ct_out)
        CK(cudaMemcpyAsync(r.ct_out + (u64)q->y0 * row * ct_words(c, (int)mo.level + 1), out,
                           n_out * ctb(c, (int)mo.level), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(q->h_res, q->res, n_out * 8, cudaMemcpyDeviceToHost, st));
    return ICHEE_OK;
}

// Launch one admission round for the requests of one ring on that ring's stream: tiles one by
// one, the other requests as batched kernels.
ichee_status launch_round(ichee_server* s, uint32_t ring, const std::vector<Req*>& all, cudaStream_t st)
{
    ichee::NvtxRange nvtx_range("ichee_server round");
    ichee_ctx* c = s->rings[ring];
    const ichee_cache* k = s->caches[ring];
    std::vector<Req*> reqs;
    for (Req* q : all) {
        if (!q->job) {
            reqs.push_back(q);
            continue;
        }
        const ichee_status e = launch_tile(s, c, k, q, st);
        if (e != ICHEE_OK) q->status = e;
    }
    if (reqs.empty()) return ICHEE_OK;
    // inputs to the device
    for (Req* q : reqs) {
        const u64 n_ct = (u64)q->r.h * q->r.w * q->r.c;
        const u64 n_b = q->pix_b ? (q->r.kind == ICHEE_REQ_WATERMARK ? (u64)q->r.h * q->r.w : n_ct) : 0;
        std::memcpy(q->h_pix, q->r.pixels, n_ct);
        if (n_b) std::memcpy(q->h_pix + n_ct, q->r.pixels2, n_b);
        CK(cudaMemcpyAsync(q->pix_a, q->h_pix, n_ct, cudaMemcpyHostToDevice, st));
        if (n_b) CK(cudaMemcpyAsync(q->pix_b, q->h_pix + n_ct, n_b, cudaMemcpyHostToDevice, st));
    }
    // one batched encryption of every image of the round (second images use seed + 1)
    std::vector<const uint8_t*> px;
    std::vector<ichee_image_desc> desc;
    std::vector<uint64_t*> outs;
    std::vector<std::pair<Req*, int>> who;   // (request, 0 = a, 1 = b)
    for (Req* q : reqs) {
        px.push_back(q->pix_a);
        desc.push_back({q->r.h, q->r.w, q->r.c, q->r.seed});
        outs.push_back(q->ct_a);
        who.push_back({q, 0});
        if (q->pix_b) {
            const uint32_t cb = q->r.kind == ICHEE_REQ_WATERMARK ? 1 : q->r.c;
            px.push_back(q->pix_b);
            desc.push_back({q->r.h, q->r.w, cb, q->r.seed + 1});
            outs.push_back(q->ct_b);
            who.push_back({q, 1});
        }
    }
    std::vector<ichee_ctimg_meta> metas(px.size());
    ichee_status st_ = ichee_encrypt_batch(c, k, px.data(), desc.data(), (uint32_t)px.size(), outs.data(), metas.data(), st);
    if (st_ != ICHEE_OK) return st_;
    for (size_t i = 0; i < who.size(); ++i) (who[i].second == 0 ? who[i].first->ma : who[i].first->mb) = metas[i];
    // one batched launch per operation kind (watermark: per distinct alpha)
    auto run_batch = [&](const std::vector<Req*>& rs, ichee_op op, bool with_b, bool per_image_arg,
                         double shared_arg) -> ichee_status {
        if (rs.empty()) return ICHEE_OK;
        std::vector<const uint64_t*> a, b;
        std::vector<uint64_t*> o;
        std::vector<ichee_ctimg_meta> ma, mb, mo(rs.size());
        std::vector<double> args;
        for (Req* q : rs) {
            a.push_back(q->ct_a);
            ma.push_back(q->ma);
            if (with_b) { b.push_back(q->ct_b); mb.push_back(q->mb); }
            o.push_back(q->ct_op);
            if (per_image_arg) args.push_back(q->r.arg);
        }
        if (!per_image_arg) args.push_back(shared_arg);
        ichee_status r = ichee_eval_batch(c, op, a.data(), ma.data(), with_b ? b.data() : nullptr,
                                          with_b ? mb.data() : nullptr, args.data(), (uint32_t)args.size(), o.data(),
                                          mo.data(), (uint32_t)rs.size(), st);
        if (r != ICHEE_OK) return r;
        for (size_t i = 0; i < rs.size(); ++i) rs[i]->mop = mo[i];
        return ICHEE_OK;
    };
    auto of_kind = [&](uint32_t kind) {
        std::vector<Req*> v;
        for (Req* q : reqs)
            if (q->r.kind == kind) v.push_back(q);
        return v;
    };
    st_ = run_batch(of_kind(ICHEE_REQ_MEANFILTER), ICHEE_OP_MEANFILTER3, false, false, 0.0);
    if (st_ != ICHEE_OK) return st_;
    st_ = run_batch(of_kind(ICHEE_REQ_BRIGHTNESS), ICHEE_OP_BRIGHTNESS, false, true, 0.0);
    if (st_ != ICHEE_OK) return st_;
    std::vector<Req*> marks = of_kind(ICHEE_REQ_WATERMARK);
    while (!marks.empty()) {
        const double al = marks.front()->r.arg;
        std::vector<Req*> same, rest;
        for (Req* q : marks) (q->r.arg == al ? same : rest).push_back(q);
        st_ = run_batch(same, ICHEE_OP_BLEND, true, false, al);
        if (st_ != ICHEE_OK) return st_;
        marks.swap(rest);
    }
    for (Req* q : reqs) {
        if (q->r.kind != ICHEE_REQ_MATCH) continue;
        st_ = ichee_eval(c, ICHEE_OP_SQDIFF_SUM, q->ct_a, &q->ma, q->ct_b, &q->mb, nullptr, 0, q->ct_op, &q->mop, st);
        if (st_ != ICHEE_OK) return st_;
    }
    for (Req* q : reqs)
        if (q->r.kind == ICHEE_REQ_ENCRYPT) q->mop = q->ma;
    // batched decryption, one launch per level present
    for (int level = 0; level < c->L; ++level) {
        std::vector<const uint64_t*> cts;
        std::vector<ichee_ctimg_meta> ms;
        std::vector<double*> ds;
        for (Req* q : reqs) {
            if ((int)q->mop.level != level) continue;
            cts.push_back(q->r.kind == ICHEE_REQ_ENCRYPT ? q->ct_a : q->ct_op);
            ms.push_back(q->mop);
            ds.push_back(q->res);
        }
        if (cts.empty()) continue;
        st_ = ichee_decrypt_batch(c, cts.data(), ms.data(), ds.data(), (uint32_t)cts.size(), st);
        if (st_ != ICHEE_OK) return st_;
    }
    for (Req* q : reqs) {
        const u64 n_res = q->r.kind == ICHEE_REQ_MATCH ? 1 : (u64)q->r.h * q->r.w * q->r.c;
        if (q->r.ct_out) {
            const u64* src = q->r.kind == ICHEE_REQ_ENCRYPT ? q->ct_a : q->ct_op;
            CK(cudaMemcpyAsync(q->r.ct_out, src, (u64)q->mop.h * q->mop.w * q->mop.c * ctb(c, (int)q->mop.level),
                               cudaMemcpyDeviceToDevice, st));
        }
        CK(cudaMemcpyAsync(q->h_res, q->res, n_res * 8, cudaMemcpyDeviceToHost, st));
    }
    return ICHEE_OK;
}

// A tile is done: its results go to the request's buffer, its memory back to the arena; the
// last tile completes the request (and frees the request's own block).
void complete_tile(ichee_server* s, Req* q)
{
    Job* j = q->job;
    const ichee_request& r = q->r;
    const bool last_index = q->tile + 1 == j->n_tiles;
    if (q->status == ICHEE_OK) {
        if (r.kind != ICHEE_REQ_MATCH)
            std::memcpy(r.result + (u64)q->y0 * r.w * r.c, q->h_res, (u64)(q->y1 - q->y0) * r.w * r.c * 8);
        else if (last_index)
            std::memcpy(r.result, q->h_res, 8);
    }
    bool finished = false;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (q->status != ICHEE_OK && j->status == ICHEE_OK) j->status = q->status;
        s->dev.release(q->off, q->tile == 0 && j->bytes ? q->job_off : q->bytes);
        s->host.release(q->hoff, q->hbytes);
        s->inflight--;
        if (++j->tiles_done == j->n_tiles) {
            finished = true;
            if (j->bytes) s->dev.release(j->off, j->bytes);
            s->stats.served++;
            s->stats.pixels += (u64)r.h * r.w * r.c;
            q->ticket = j->ticket;
            q->t_submit = j->t_submit;
            q->t_admit = j->t_admit;
            q->t_done = now_s();
            q->status = j->status;
            s->done[q->ticket] = q;   // the request's record; freed with its job when collected
            s->cv_done.notify_all();
        }
        s->cv_work.notify_all();
    }
    if (!finished) delete q;
}

void complete(ichee_server* s, Req* q)
{
    if (q->job) {
        complete_tile(s, q);
        return;
    }
    const u64 n_res = q->r.kind == ICHEE_REQ_MATCH ? 1 : (u64)q->r.h * q->r.w * q->r.c;
    if (q->status == ICHEE_OK) std::memcpy(q->r.result, q->h_res, n_res * 8);
    q->t_done = now_s();
    std::lock_guard<std::mutex> lock(s->mu);
    s->dev.release(q->off, q->bytes);
    s->host.release(q->hoff, q->hbytes);
    s->inflight--;
    s->stats.served++;
    s->stats.pixels += (u64)q->r.h * q->r.w * q->r.c;
    s->done[q->ticket] = q;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
}

void worker_main(ichee_server* s)
{
    cudaSetDevice(s->device);
    for (;;) {
        // completions, in order per ring stream (a round's event covers all its copies)
        for (auto it = s->rounds.begin(); it != s->rounds.end();) {
            cudaError_t e = it->done ? cudaEventQuery(it->done) : cudaErrorInvalidResourceHandle;
            if (e != cudaErrorNotReady && s->inject_query_errors.load() > 0) {   // host-side failure injection
                s->inject_query_errors--;
                e = cudaErrorLaunchFailure;
            }
            if (e == cudaErrorNotReady) {
                ++it;
                continue;
            }
            // Any other answer ends the round: success completes its requests; an error (a
            // sticky launch or execution error, or no event) fails them with ICHEE_ECUDA, so
            // clients are answered, the ring admits again and the worker can stop.
            if (e != cudaSuccess)
                for (Req* q : it->reqs)
                    if (q->status == ICHEE_OK) q->status = ICHEE_ECUDA;
            for (Req* q : it->reqs) complete(s, q);
            s->ring_rounds[it->ring]--;
            if (it->done) cudaEventDestroy(it->done);
            it = s->rounds.erase(it);
        }
        std::vector<Req*> admitted;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            // arrival order; a ring with its rounds full is skipped for this pass, and the first
            // request that does not fit in memory ends the pass
            std::vector<bool> open(s->rings.size());
            for (size_t r = 0; r < open.size(); ++r) open[r] = !s->hold && s->ring_rounds[r] < kRoundsPerRing;
            for (auto it = s->pending.begin(); it != s->pending.end() && s->inflight < s->max_inflight;) {
                Req* q = *it;
                if (!open[q->r.ring]) { ++it; continue; }
                bool ok = s->dev.alloc(q->bytes, &q->off);
                if (ok && !s->host.alloc(q->hbytes, &q->hoff)) {
                    s->dev.release(q->off, q->bytes);
                    ok = false;
                }
                if (!ok) break;   // memory is granted strictly in arrival order (no starvation)
                it = s->pending.erase(it);
                s->inflight++;
                admitted.push_back(q);
            }
            s->stats.peak_arena_bytes = s->dev.peak();
            s->stats.max_inflight = std::max<uint64_t>(s->stats.max_inflight, s->inflight);
            if (admitted.empty()) {
                if (s->stop && s->pending.empty() && s->rounds.empty()) break;
                if (s->rounds.empty())
                    s->cv_work.wait_for(lock, std::chrono::milliseconds(2));
                else
                    lock.unlock(), std::this_thread::sleep_for(std::chrono::microseconds(20));
                continue;
            }
        }
        const double t = now_s();
        for (Req* q : admitted) {
            q->t_admit = t;
            if (q->job && q->tile == 0) q->job->t_admit = t;
            q->round_size = (uint32_t)admitted.size();
            carve(s, q);
        }
        for (uint32_t ring = 0; ring < s->rings.size(); ++ring) {
            std::vector<Req*> mine;
            for (Req* q : admitted)
                if (q->r.ring == ring) mine.push_back(q);
            if (mine.empty()) continue;
            cudaStream_t st = s->streams[ring];
            ichee_status r = ICHEE_ECUDA;
            if (s->inject_launch_errors.load() > 0)   // host-side failure injection: nothing is launched
                s->inject_launch_errors--;
            else
                r = launch_round(s, ring, mine, st);
            if (r != ICHEE_OK)
                for (Req* q : mine) q->status = r;
            Round rd;
            if (cudaEventCreateWithFlags(&rd.done, cudaEventDisableTiming) != cudaSuccess) rd.done = nullptr;
            if (rd.done && cudaEventRecord(rd.done, st) != cudaSuccess) {
                cudaEventDestroy(rd.done);
                rd.done = nullptr;
            }
            rd.ring = ring;
            rd.reqs = mine;
            s->rounds.push_back(rd);
            s->ring_rounds[ring]++;
            s->stats.rounds++;
        }
    }
}

}  // namespace

extern "C" ichee_status ichee_server_create(ichee_ctx* const* rings, const ichee_cache* const* caches, uint32_t n_rings,
                                            size_t hbm_budget_bytes, uint32_t max_inflight, ichee_server** out)
{
    if (!rings || !caches || !out || n_rings == 0 || n_rings > 8) return fail(ICHEE_EINVAL, "bad ring list");
    *out = nullptr;
    for (uint32_t i = 0; i < n_rings; ++i) {
        if (!rings[i] || !rings[i]->have_pk || !rings[i]->have_sk)
            return fail(ICHEE_EINVAL, "ring %u needs its public and secret keys", i);
        if (rings[i]->device != rings[0]->device) return fail(ICHEE_EINVAL, "all rings must share one device");
        if (rings[i]->L < 2) return fail(ICHEE_EINVAL, "ring %u needs two limbs for its operations", i);
        if (caches[i] && caches[i]->ctx != rings[i]) return fail(ICHEE_EMISMATCH, "cache %u belongs to another ring", i);
    }
    if (hbm_budget_bytes < (1u << 20)) return fail(ICHEE_EINVAL, "HBM budget too small");
    ichee_server* s = new ichee_server();
    s->rings.assign(rings, rings + n_rings);
    s->caches.assign(caches, caches + n_rings);
    s->device = rings[0]->device;
    s->max_inflight = max_inflight ? max_inflight : 256;
    auto bail = [&](ichee_status st) {
        ichee_server_destroy(s);
        return st;
    };
    if (cudaSetDevice(s->device) != cudaSuccess) return bail(fail(ICHEE_ECUDA, "cudaSetDevice"));
    if (cudaMalloc(&s->d_base, hbm_budget_bytes) != cudaSuccess)
        return bail(fail(ICHEE_ENOMEM, "cannot reserve the %zu-byte HBM budget", hbm_budget_bytes));
    s->dev.reset(hbm_budget_bytes);
    s->tile_bytes = hbm_budget_bytes / 4;
    const size_t host_bytes = 512ull << 20;
    if (cudaHostAlloc((void**)&s->h_base, host_bytes, cudaHostAllocDefault) != cudaSuccess)
        return bail(fail(ICHEE_ENOMEM, "pinned staging"));
    s->host.reset(host_bytes);
    s->streams.resize(n_rings);
    s->ring_rounds.assign(n_rings, 0);
    for (auto& st : s->streams)
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return bail(fail(ICHEE_ECUDA, "stream"));
    s->stats.arena_bytes = hbm_budget_bytes;
    s->worker = std::thread(worker_main, s);
    *out = s;
    return ICHEE_OK;
}

// Queue a request as row tiles of at most the server's tile bytes (the first tile also holds
// the request's own block). Refused if even a one-row tile does not fit the budget.
static ichee_status submit_tiled(ichee_server* s, const ichee_request* r, uint64_t* ticket)
{
    const size_t jb = job_bytes(s, *r);
    // bytes of a middle tile with `rows` output rows (the mean filter reads a halo row on each side)
    auto cost = [&](uint32_t rows, size_t* dev, size_t* host) {
        tile_sizes(s, *r, 0, rows, 0, rows + (r->kind == ICHEE_REQ_MEANFILTER ? 2 : 0), dev, host);
        *dev += jb;
    };
    auto fits = [&](uint32_t rows) {
        size_t dev, host;
        cost(rows, &dev, &host);
        return dev <= s->tile_bytes && host <= s->host.size() / 16;
    };
    uint32_t rows = 1;
    if (!fits(1)) {   // one row is above the tile size: still served if it fits the whole budget
        size_t dev, host;
        cost(1, &dev, &host);
        if (dev > s->dev.size() || host > s->host.size())
            return fail(ICHEE_EINVAL, "request needs %zu bytes for one image row, more than the %zu-byte budget", dev,
                        s->dev.size());
    } else {
        for (uint32_t step = 1u << 16; step > 0; step >>= 1)   // the largest row count that fits
            if (rows + step <= r->h && fits(rows + step)) rows += step;
    }
    const uint32_t n_tiles = (r->h + rows - 1) / rows;
    const ichee_ctx* c = s->rings[r->ring];
    Job* j = new Job();
    j->r = *r;
    j->n_tiles = n_tiles;
    j->bytes = jb;
    j->m_img.h = r->h;
    j->m_img.w = r->w;
    j->m_img.c = r->c;
    j->m_img.level = (uint32_t)(c->L - 1);
    j->m_img.scale = c->delta;
    std::vector<Req*> tiles;
    for (uint32_t t = 0; t < n_tiles; ++t) {
        Req* q = new Req();
        q->r = *r;
        q->job = j;
        q->tile = t;
        q->y0 = t * rows;
        q->y1 = std::min<uint32_t>(r->h, (t + 1) * rows);
        tile_rows(*r, q->y0, q->y1, &q->r0, &q->r1);
        tile_sizes(s, *r, q->y0, q->y1, q->r0, q->r1, &q->bytes, &q->hbytes);
        if (t == 0 && jb) {
            q->job_off = q->bytes;
            q->bytes += jb;
        }
        tiles.push_back(q);
    }
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) {
        for (Req* q : tiles) delete q;
        delete j;
        return fail(ICHEE_EINVAL, "server is stopping");
    }
    j->ticket = s->next_ticket++;
    j->t_submit = now_s();
    for (Req* q : tiles) {
        q->t_submit = j->t_submit;
        s->pending.push_back(q);
    }
    s->stats.submitted++;
    *ticket = j->ticket;
    s->cv_work.notify_all();
    return ICHEE_OK;
}

extern "C" ichee_status ichee_server_submit(ichee_server* s, const ichee_request* r, uint64_t* ticket)
{
    if (!s || !r || !ticket) return fail(ICHEE_EINVAL, "null argument");
    if (r->ring >= s->rings.size()) return fail(ICHEE_EINVAL, "ring %u out of range", r->ring);
    if (r->kind > ICHEE_REQ_MATCH) return fail(ICHEE_EINVAL, "unknown request kind %u", r->kind);
    if (image_cts(r->h, r->w, r->c) == 0) return fail(ICHEE_EINVAL, "empty or oversized image");
    if (!r->pixels || !r->result) return fail(ICHEE_EINVAL, "request needs pixels and a result buffer");
    if ((r->kind == ICHEE_REQ_WATERMARK || r->kind == ICHEE_REQ_MATCH) && !r->pixels2)
        return fail(ICHEE_EINVAL, "watermark and match need a second image");
    if (r->kind == ICHEE_REQ_MATCH && !s->rings[r->ring]->have_evk)
        return fail(ICHEE_EUNSUPPORTED, "ring %u has no evaluation key for matching", r->ring);
    if (r->kind == ICHEE_REQ_MEANFILTER && s->rings[r->ring]->n / 2 < s->rings[r->ring]->shape_meanfilter.threads)
        return fail(ICHEE_EUNSUPPORTED, "ring too small for the mean filter");
    size_t dev_bytes = 0, host_bytes = 0;
    sizes(s, *r, &dev_bytes, &host_bytes);
    if (dev_bytes > s->tile_bytes || host_bytes > s->host.size() / 16) return submit_tiled(s, r, ticket);
    Req* q = new Req();
    q->r = *r;
    q->bytes = dev_bytes;
    q->hbytes = host_bytes;
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) {
        delete q;
        return fail(ICHEE_EINVAL, "server is stopping");
    }
    q->ticket = s->next_ticket++;
    q->t_submit = now_s();
    s->pending.push_back(q);
    s->stats.submitted++;
    *ticket = q->ticket;
    s->cv_work.notify_all();
    return ICHEE_OK;
}

extern "C" ichee_status ichee_server_wait(ichee_server* s, uint64_t ticket, uint32_t timeout_ms, ichee_request_done* out)
{
    if (!s || !out) return fail(ICHEE_EINVAL, "null argument");
    std::unique_lock<std::mutex> lock(s->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        auto it = s->done.find(ticket);
        if (it != s->done.end()) {
            Req* q = it->second;
            out->ticket = q->ticket;
            out->status = q->status;
            out->t_submit = q->t_submit;
            out->t_admit = q->t_admit;
            out->t_done = q->t_done;
            out->round_size = q->round_size;
            s->done.erase(it);
            delete q->job;
            delete q;
            return out->status == ICHEE_OK ? ICHEE_OK : fail((ichee_status)out->status, "request %llu failed",
                                                             (unsigned long long)ticket);
        }
        if (s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && s->done.find(ticket) == s->done.end())
            return fail(ICHEE_ETIMEOUT, "request %llu not done after %u ms", (unsigned long long)ticket, timeout_ms);
    }
}

extern "C" ichee_status ichee_server_stats_get(ichee_server* s, ichee_server_stats* out)
{
    if (!s || !out) return fail(ICHEE_EINVAL, "null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->stats;
    out->pending = 0;   // requests none of whose pieces has been admitted yet
    for (const Req* q : s->pending)
        if (!q->job || q->tile == 0) out->pending++;
    out->inflight = s->inflight;
    out->arena_used_bytes = s->dev.used();
    return ICHEE_OK;
}

extern "C" ichee_status ichee_server_hold(ichee_server* s, int hold)
{
    if (!s) return fail(ICHEE_EINVAL, "null server");
    std::lock_guard<std::mutex> lock(s->mu);
    s->hold = hold != 0;
    s->cv_work.notify_all();
    return ICHEE_OK;
}

extern "C" ichee_status ichee_server_inject_failure(ichee_server* s, uint32_t launch_errors, uint32_t query_errors)
{
    if (!s) return fail(ICHEE_EINVAL, "null server");
    s->inject_launch_errors = launch_errors;
    s->inject_query_errors = query_errors;
    return ICHEE_OK;
}

extern "C" void ichee_server_destroy(ichee_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->hold = false;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    for (auto& st : s->streams)
        if (st) cudaStreamSynchronize(st), cudaStreamDestroy(st);
    for (auto& kv : s->done) {
        delete kv.second->job;
        delete kv.second;
    }
    for (Req* q : s->pending) delete q;   // (empty: the worker finishes every queued request)
    if (s->d_base) cudaFree(s->d_base);
    if (s->h_base) cudaFreeHost(s->h_base);
    delete s;
}
