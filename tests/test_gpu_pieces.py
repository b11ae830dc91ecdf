"""Images in pieces (GPU): pixel ranges, row bands and partial matching sums give, word for word,
the ciphertexts of the whole-image calls and of the CPU oracle.

These are the entry points that stream an image through limited memory (the server's tiles)
and that split it over several GPUs: ichee_encrypt_pixels (Sec. 3.1: every random draw is keyed
by the ciphertext's index in its image), ichee_meanfilter_rows (Sec. 4.4.1 on a band of rows,
borders of the whole image), ichee_sqdiff_accumulate / ichee_sqdiff_finish (Sec. 4.4.3: the
matching sum is a sum, relinearised and rescaled once).
"""
import numpy as np
import pytest

from oracle import Oracle, Params
from paper_2409_03568_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RING = dict(log_n=10, prime_bits=[60, 40, 40, 40], log2_scale=40, special_bits=61)
KEY_SEED = 4242


@pytest.fixture(scope="module")
def ichee():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03568_gb300 import ichee as mod
    return mod


@pytest.fixture(scope="module")
def ring(ichee):
    ctx = ichee.Context(**RING)
    ctx.keygen(KEY_SEED, with_evk=True)
    o = Oracle(Params(RING["log_n"], RING["prime_bits"], RING["log2_scale"], RING["special_bits"]))
    o.keygen(KEY_SEED, with_evk=True)
    yield ctx, o
    ctx.close()


def as_cts(t, n_ct, limbs, n):
    return t.cpu().numpy().view(np.uint64).reshape(n_ct, 2, limbs, n)


def caches_of(ichee, ctx, img):
    scan = torch.from_numpy(img).cuda()
    return {"fresh": None,
            "radix16": ctx.build_cache(ichee.CACHE_RADIX, 21, radix_base=16, randomize=1),
            "radix10": ctx.build_cache(ichee.CACHE_RADIX, 22, radix_base=10, randomize=1),
            "freq_fresh": ctx.build_cache(ichee.CACHE_FREQ, 23, top_k=6, pool_size=4, scan=scan),
            "freq_radix": ctx.build_cache(ichee.CACHE_FREQ, 24, top_k=6, pool_size=4, scan=scan, miss_policy=1,
                                          radix_base=16),
            "full": ctx.build_cache(ichee.CACHE_FULL, 25, pool_size=8)}


def test_pixel_ranges_equal_whole_image(ichee, ring):
    ctx, o = ring
    h, w, c = 7, 5, 3
    img = inputs.random_field_image(h, w, seed=8, channels=c).reshape(-1)
    n_px, ctw = img.size, ctx.ct_words(ctx.L - 1)
    for name, cache in caches_of(ichee, ctx, img).items():
        whole, _ = ctx.encrypt(torch.from_numpy(img).cuda(), h, w, c, 61, cache=cache)
        pieces = ctx.empty_cts(n_px, ctx.L - 1)
        for lo, hi in ((0, 1), (1, 40), (40, 41), (41, n_px)):
            # host pixels for one piece, device pixels for the others
            px = img[lo:hi].copy() if lo == 1 else torch.from_numpy(img[lo:hi].copy()).cuda()
            ichee.ichee_encrypt_pixels(ctx.handle, cache, px, hi - lo, lo, 61, pieces[lo * ctw:hi * ctw], ctx.stream())
        assert torch.equal(pieces, whole), name
    # and a fresh piece is the oracle's ciphertexts with the same ids
    got = ctx.empty_cts(10, ctx.L - 1)
    ichee.ichee_encrypt_pixels(ctx.handle, None, torch.from_numpy(img[20:30].copy()).cuda(), 10, 20, 61, got, ctx.stream())
    ref = o.encrypt_pixels(img[20:30], 61, ids=np.arange(20, 30, dtype=np.uint64))
    assert np.array_equal(as_cts(got, 10, ctx.L, ctx.n), ref)


def test_meanfilter_row_bands_equal_whole_image(ichee, ring):
    check_meanfilter_bands(ichee, *ring)


def test_meanfilter_row_bands_five_limbs(ichee):
    """Five limbs: whole images and bands run the batched filter kernel as one-image batches."""
    ring5 = dict(RING, prime_bits=[60, 40, 40, 40, 40])
    ctx = ichee.Context(**ring5)
    ctx.keygen(KEY_SEED)
    o = Oracle(Params(ring5["log_n"], ring5["prime_bits"], ring5["log2_scale"], ring5["special_bits"]))
    o.keygen(KEY_SEED)
    try:
        check_meanfilter_bands(ichee, ctx, o)
    finally:
        ctx.close()


def check_meanfilter_bands(ichee, ctx, o):
    h, w, c = 7, 5, 3
    img = inputs.random_field_image(h, w, seed=9, channels=c).reshape(-1)
    row = w * c
    a, ma = ctx.encrypt(torch.from_numpy(img).cuda(), h, w, c, 62)
    whole, mw = ctx.eval(ichee.OP_MEANFILTER3, a, ma, out_level=ma.level - 1)
    ref, sc = o.meanfilter3(o.encrypt_pixels(img, 62), o.delta, h, w, c)
    assert np.array_equal(as_cts(whole, h * row, ctx.L - 1, ctx.n), ref)
    ctw_in, ctw_out = ctx.ct_words(ma.level), ctx.ct_words(ma.level - 1)
    for y0, y1 in ((0, 1), (1, 4), (4, 6), (6, 7), (0, 7)):
        r0, r1 = max(0, y0 - 1), min(h, y1 + 1)
        band = ctx.empty_cts((r1 - r0) * row, ma.level)
        ichee.ichee_encrypt_pixels(ctx.handle, None, torch.from_numpy(img[r0 * row:r1 * row].copy()).cuda(),
                                   (r1 - r0) * row, r0 * row, 62, band, ctx.stream())
        out = ctx.empty_cts((y1 - y0) * row, ma.level - 1)
        m = ichee.ichee_meanfilter_rows(ctx.handle, band, ma, r0, r1 - r0, y0, y1, out, ctx.stream())
        assert (m.h, m.w, m.c, m.level) == (y1 - y0, w, c, ma.level - 1) and m.scale == mw.scale
        assert torch.equal(out, whole[y0 * row * ctw_out:y1 * row * ctw_out]), (y0, y1)
        assert ctw_in > ctw_out
    # a band that lacks a row the output needs is refused before any launch
    band = ctx.empty_cts(2 * row, ma.level)
    out = ctx.empty_cts(2 * row, ma.level - 1)
    with pytest.raises(ichee.IcheeError) as e:
        ichee.ichee_meanfilter_rows(ctx.handle, band, ma, 2, 2, 2, 4, out, ctx.stream())
    assert e.value.status == ichee.EINVAL


def test_matching_in_pieces_equals_whole(ichee, ring):
    ctx, o = ring
    h, w, c = 6, 7, 3
    img = inputs.random_field_image(h, w, seed=10, channels=c).reshape(-1)
    other = inputs.noisy_copy(img, seed=11)
    n_px = img.size
    a, ma = ctx.encrypt(torch.from_numpy(img).cuda(), h, w, c, 63)
    b, mb = ctx.encrypt(torch.from_numpy(other).cuda(), h, w, c, 64)
    whole, mw = ctx.eval(ichee.OP_SQDIFF_SUM, a, ma, b, mb, out_n_ct=1, out_level=ma.level - 1)
    ref, sc = o.match(o.encrypt_pixels(img, 63), o.encrypt_pixels(other, 64), o.delta)
    assert np.array_equal(as_cts(whole, 1, ctx.L - 1, ctx.n), ref)
    ctw = ctx.ct_words(ma.level)
    words = ichee.ichee_sqdiff_acc_words(ctx.handle, ma.level)
    assert words == 3 * ctx.L * ctx.n

    def piece(lo, hi):
        m = ichee.CtImgMeta(hi - lo, 1, 1, ma.level, ma.scale)
        return a[lo * ctw:hi * ctw], m, b[lo * ctw:hi * ctw], m

    # tiles accumulated into one accumulator (any order)
    cuts = [(50, n_px), (0, 1), (1, 50)]
    acc = torch.full((words,), -1, dtype=torch.int64, device="cuda")
    for i, (lo, hi) in enumerate(cuts):
        pa, pm, pb, pbm = piece(lo, hi)
        ichee.ichee_sqdiff_accumulate(ctx.handle, pa, pm, pb, pbm, acc, accumulate=i > 0, stream=ctx.stream())
    out = ctx.empty_cts(1, ma.level - 1)
    m = ichee.ichee_sqdiff_finish(ctx.handle, acc, ma, out, ctx.stream())
    assert (m.h, m.w, m.c, m.level) == (1, 1, 1, mw.level) and m.scale == mw.scale
    assert torch.equal(out, whole)
    # one accumulator per "rank", added as plain 64-bit words (what an all-reduce does), 8 ranks
    bounds = np.linspace(0, n_px, 9).astype(int)
    total = torch.zeros(words, dtype=torch.int64, device="cuda")
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        part = torch.empty(words, dtype=torch.int64, device="cuda")
        pa, pm, pb, pbm = piece(int(lo), int(hi))
        ichee.ichee_sqdiff_accumulate(ctx.handle, pa, pm, pb, pbm, part, stream=ctx.stream())
        total += part
    out2 = ctx.empty_cts(1, ma.level - 1)
    ichee.ichee_sqdiff_finish(ctx.handle, total, ma, out2, ctx.stream())
    assert torch.equal(out2, whole)
    dec = ctx.decrypt(out2, m).cpu().numpy()
    np.testing.assert_allclose(dec, o.decrypt(ref, sc), rtol=1e-9)


def test_fused_rescale_general_constants(ichee):
    """Mean filter and blend where the encoded constants are not below every prime (30-bit
    primes, Delta = 2^36): the general two-product rescale, still bit-exact with the oracle."""
    wl = dict(log_n=10, prime_bits=[50, 30, 30], log2_scale=36, special_bits=0)
    ctx = ichee.Context(**wl)
    ctx.keygen(77)
    o = Oracle(Params(wl["log_n"], wl["prime_bits"], wl["log2_scale"])).keygen(77)
    h, w, c = 4, 5, 1
    img = inputs.random_field_image(h, w, seed=12, channels=c).reshape(-1)
    wm = inputs.binary_pattern(h, w, seed=13).reshape(-1)
    a, ma = ctx.encrypt(torch.from_numpy(img).cuda(), h, w, c, 65)
    b, mb = ctx.encrypt(torch.from_numpy(wm).cuda(), h, w, 1, 66)
    ra, rb = o.encrypt_pixels(img, 65), o.encrypt_pixels(wm, 66)
    assert round(o.delta / 9) > int(o.q[1])   # the general path
    out, _ = ctx.eval(ichee.OP_MEANFILTER3, a, ma, out_level=ma.level - 1)
    ref, _ = o.meanfilter3(ra, o.delta, h, w, c)
    assert np.array_equal(as_cts(out, h * w * c, 2, ctx.n), ref)
    out, _ = ctx.eval(ichee.OP_BLEND, a, ma, b, mb, args=(0.9,), out_level=ma.level - 1)
    ref, _ = o.blend(ra, rb, o.delta, 0.9, c, 1)
    assert np.array_equal(as_cts(out, h * w * c, 2, ctx.n), ref)
    ctx.close()


@pytest.mark.parametrize("shape", [(6, 5, 3), (1, 9, 1), (9, 1, 2), (4, 64, 1), (3, 37, 3)])
def test_meanfilter_forms_agree_with_the_oracle(ichee, ring, shape):
    """Both forms of the mean filter (register walk; input columns staged in shared memory by
    bulk copies), single-image and batched, give the oracle's ciphertexts; also one-row and
    one-column images, and wider rows (64 and 37 columns)."""
    ctx, o = ring
    h, w, c = shape
    img = inputs.random_field_image(h, w, seed=14, channels=c).reshape(-1)
    a, ma = ctx.encrypt(torch.from_numpy(img).cuda(), h, w, c, 67)
    ref, _ = o.meanfilter3(o.encrypt_pixels(img, 67), o.delta, h, w, c)
    img2 = inputs.random_field_image(3, 4, seed=15, channels=1).reshape(-1)
    a2, ma2 = ctx.encrypt(torch.from_numpy(img2).cuda(), 3, 4, 1, 68)
    ref2, _ = o.meanfilter3(o.encrypt_pixels(img2, 68), o.delta, 3, 4, 1)
    try:
        for form in (0, 1):
            ichee.ichee_set_tuned_shape(ctx.handle, ichee.TUNE_MF_STAGED, form)
            assert ichee.ichee_tuned_shape(ctx.handle, ichee.TUNE_MF_STAGED)[0] == form
            out, _ = ctx.eval(ichee.OP_MEANFILTER3, a, ma, out_level=ma.level - 1)
            assert np.array_equal(as_cts(out, h * w * c, ctx.L - 1, ctx.n), ref), form
            outs = [ctx.empty_cts(h * w * c, ma.level - 1), ctx.empty_cts(12, ma.level - 1)]
            ichee.ichee_eval_batch(ctx.handle, ichee.OP_MEANFILTER3, [a, a2], [ma, ma2], outs=outs, stream=ctx.stream())
            assert np.array_equal(as_cts(outs[0], h * w * c, ctx.L - 1, ctx.n), ref), form
            assert np.array_equal(as_cts(outs[1], 12, ctx.L - 1, ctx.n), ref2), form
            ichee.ichee_stream_status(ctx.handle, ctx.stream())
    finally:
        ichee.ichee_set_tuned_shape(ctx.handle, ichee.TUNE_MF_STAGED, 0)
