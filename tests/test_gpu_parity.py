"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by element.

Ciphertexts must be bit-exact; decoded values agree with the oracle's exact decode within 1e-9
relative and, for fresh encryptions, lie within 1e-3 of the pixel. Every input is seeded; the
oracle recomputes its own keys, caches and ciphertexts from the same seeds and never takes a
value from the CUDA path.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import Oracle, Params
from paper_2409_03568_gb300 import inputs, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEY_SEED = 1234
IMG_SEED = 99
CACHE_SEED = 777


@pytest.fixture(scope="module")
def ichee():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03568_gb300 import ichee as mod
    return mod


def oracle_for(wl, with_evk=False, key_seed=KEY_SEED):
    o = Oracle(Params(wl["log_n"], wl["prime_bits"], wl["log2_scale"], wl.get("special_bits", 0)))
    return o.keygen(key_seed, with_evk=with_evk)


def gpu_for(ichee, wl, with_evk=False, key_seed=KEY_SEED):
    ctx = ichee.Context(**W.ctx_kwargs(wl))
    ctx.keygen(key_seed, with_evk=with_evk)
    return ctx


def as_cts(t, n_ct, limbs, n):
    return t.cpu().numpy().view(np.uint64).reshape(n_ct, 2, limbs, n)


# --------------------------------------------------------------------------- set-up
@pytest.mark.parametrize("wl", [W.TOY, W.ENC8192, W.OPS8192, W.RING16384], ids=lambda w: w["name"])
def test_primes_match_oracle(ichee, wl):
    ctx = ichee.Context(**W.ctx_kwargs(wl))
    o = Oracle(Params(wl["log_n"], wl["prime_bits"], wl["log2_scale"], wl.get("special_bits", 0)))
    assert ctx.q == [int(x) for x in o.q]
    assert ctx.P == o.P
    ctx.close()


@pytest.mark.parametrize("wl,evk", [(W.TOY, False), (W.OPS8192, True)], ids=["toy", "ops8192_evk"])
def test_keys_bit_exact(ichee, wl, evk):
    ctx = gpu_for(ichee, wl, with_evk=evk)
    o = oracle_for(wl, with_evk=evk)
    n, L = ctx.n, ctx.L
    s = np.zeros(n, dtype=np.int8)
    ichee.ichee_export_key(ctx.handle, 0, s)
    assert np.array_equal(s, o.s)
    pk = np.zeros((2, L, n), dtype=np.uint64)
    ichee.ichee_export_key(ctx.handle, 1, pk)
    assert np.array_equal(pk, o.pk)
    if evk:
        e = np.zeros((L, 2, L + 1, n), dtype=np.uint64)
        ichee.ichee_export_key(ctx.handle, 2, e)
        assert np.array_equal(e, o.evk)
    ctx.close()


# --------------------------------------------------------------------- fresh (a2, a3, a8)
def test_fresh_toy_bit_exact_and_decodes(ichee):
    wl = W.TOY
    ctx = gpu_for(ichee, wl)
    o = oracle_for(wl)
    pix = W.image_for(wl).reshape(-1)
    ct, meta = ctx.encrypt(torch.from_numpy(pix).cuda(), wl["h"], wl["w"], wl["c"], IMG_SEED)
    assert (meta.h, meta.w, meta.c, meta.level) == (8, 8, 1, 1) and meta.scale == 2.0 ** 25
    got = as_cts(ct, 64, 2, ctx.n)
    ref = o.encrypt_pixels(pix, IMG_SEED)
    assert np.array_equal(got, ref)
    dec = ctx.decrypt(ct, meta).cpu().numpy()
    np.testing.assert_allclose(dec, o.decrypt(ref, o.delta), rtol=1e-9, atol=0)
    assert np.max(np.abs(dec - pix)) < 1e-3
    # host pixels and host output through the same entry points
    ct2, _ = ctx.encrypt(pix.copy(), wl["h"], wl["w"], wl["c"], IMG_SEED)
    assert torch.equal(ct, ct2)
    host_out = np.zeros(64, dtype=np.float64)
    ichee.ichee_decrypt_image(ctx.handle, ct2, meta, host_out, ctx.stream())
    assert np.array_equal(host_out, dec)
    ctx.close()


def test_decrypt_async_into_pinned_memory(ichee):
    """ichee_decrypt_image_async writes page-locked host memory (or device memory) from the
    kernel and returns without waiting; after the stream the values equal the synchronous
    call's. Pageable host memory is refused."""
    wl = W.TOY
    ctx = gpu_for(ichee, wl)
    pix = W.image_for(wl).reshape(-1)
    ct, meta = ctx.encrypt(torch.from_numpy(pix).cuda(), wl["h"], wl["w"], wl["c"], IMG_SEED)
    ref = ctx.decrypt(ct, meta).cpu()
    pinned = torch.full((64,), -1.0, dtype=torch.float64).pin_memory()
    ichee.ichee_decrypt_image_async(ctx.handle, ct, meta, pinned, ctx.stream())
    torch.cuda.synchronize()
    assert torch.equal(pinned, ref)
    dev = torch.empty(64, dtype=torch.float64, device="cuda")
    ichee.ichee_decrypt_image_async(ctx.handle, ct, meta, dev, ctx.stream())
    assert torch.equal(dev.cpu(), ref)
    with pytest.raises(ichee.IcheeError) as e:
        ichee.ichee_decrypt_image_async(ctx.handle, ct, meta, np.zeros(64), ctx.stream())
    assert e.value.status == ichee.EINVAL
    ctx.close()


def test_fresh_enc8192_full_image_sampled(ichee):
    wl = W.ENC8192
    ctx = gpu_for(ichee, wl)
    o = oracle_for(wl)
    pix = W.image_for(wl).reshape(-1)
    n_ct = pix.size
    ct, meta = ctx.encrypt(torch.from_numpy(pix).cuda(), wl["h"], wl["w"], wl["c"], IMG_SEED)
    got = as_cts(ct, n_ct, 3, ctx.n)
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([[0, 1, n_ct - 1], rng.choice(n_ct, 13, replace=False)]))
    ref = o.encrypt_pixels(pix[idx], IMG_SEED, ids=idx.astype(np.uint64))
    for j, k in enumerate(idx):
        assert np.array_equal(got[k], ref[j]), k
    dec = ctx.decrypt(ct, meta).cpu().numpy()
    assert np.max(np.abs(dec - pix)) < 1e-3
    np.testing.assert_allclose(dec[idx], o.decrypt(ref, o.delta), rtol=1e-9, atol=0)
    ctx.close()


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 5, 1), (7, 1, 3), (2, 2, 2)])
def test_fresh_ragged_shapes_toy(ichee, shape):
    wl = W.TOY
    ctx = gpu_for(ichee, wl)
    o = oracle_for(wl)
    h, w, c = shape
    pix = inputs.uniform_image(h, w, seed=5, channels=c).reshape(-1)
    if pix.size >= 2:
        pix[0], pix[-1] = 0, 255
    ct, meta = ctx.encrypt(torch.from_numpy(pix).cuda(), h, w, c, 31)
    assert np.array_equal(as_cts(ct, pix.size, 2, ctx.n), o.encrypt_pixels(pix, 31))
    ctx.close()


# -------------------------------------------------------------------- caches (a4, a5)
@pytest.mark.parametrize("randomize", [1, 0])
def test_radix16_toy_bit_exact(ichee, randomize):
    wl = W.TOY
    ctx = gpu_for(ichee, wl)
    o = oracle_for(wl)
    cache = ctx.build_cache(ichee.CACHE_RADIX, CACHE_SEED, radix_base=16, randomize=randomize)
    oc = o.radix_cache(16, CACHE_SEED)
    radix = np.zeros((2, 2, 2, ctx.n), dtype=np.uint64)
    ichee.ichee_cache_export(cache, 2, radix)
    assert np.array_equal(radix, oc["cts"])
    pix = W.image_for(wl).reshape(-1)
    ct, meta = ctx.encrypt(torch.from_numpy(pix).cuda(), 8, 8, 1, IMG_SEED, cache=cache)
    ref = o.encrypt_radix(pix, oc, IMG_SEED, randomize=bool(randomize))
    assert np.array_equal(as_cts(ct, 64, 2, ctx.n), ref)
    dec = ctx.decrypt(ct, meta).cpu().numpy()
    assert np.max(np.abs(dec - pix)) < 1e-3
    ctx.close()


@pytest.fixture(scope="module")
def enc8192(ichee):
    wl = W.ENC8192
    ctx = gpu_for(ichee, wl)
    o = oracle_for(wl)
    pix = W.image_for(wl).reshape(-1)
    yield wl, ctx, o, pix
    ctx.close()


@pytest.mark.parametrize("base", [10, 16])
def test_radix_enc8192_sampled(ichee, enc8192, base):
    wl, ctx, o, pix = enc8192
    cache = ctx.build_cache(ichee.CACHE_RADIX, CACHE_SEED, radix_base=base, randomize=1)
    oc = o.radix_cache(base, CACHE_SEED)
    n_pow = oc["n_pow"]
    radix = np.zeros((n_pow, 2, 3, ctx.n), dtype=np.uint64)
    ichee.ichee_cache_export(cache, 2, radix)
    assert np.array_equal(radix, oc["cts"])
    ct, meta = ctx.encrypt(torch.from_numpy(pix).cuda(), 64, 64, 1, IMG_SEED, cache=cache)
    got = as_cts(ct, pix.size, 3, ctx.n)
    idx = np.unique(np.concatenate([[0, pix.size - 1], np.random.default_rng(base).choice(pix.size, 30, replace=False)]))
    ref = o.encrypt_radix(pix[idx], oc, IMG_SEED, ids=idx.astype(np.uint64))
    for j, k in enumerate(idx):
        assert np.array_equal(got[k], ref[j]), k
    dec = ctx.decrypt(ct, meta).cpu().numpy()
    assert np.max(np.abs(dec - pix)) < 1e-3


@pytest.mark.parametrize("kind", ["freq", "full", "freq_radix_miss"])
def test_lookup_enc8192_sampled(ichee, enc8192, kind):
    wl, ctx, o, pix = enc8192
    if kind == "freq":
        cache = ctx.build_cache(ichee.CACHE_FREQ, CACHE_SEED, top_k=32, pool_size=64, scan=torch.from_numpy(pix).cuda())
        oc = o.freq_cache(pix, 32, 64, CACHE_SEED)
        miss = 0
    elif kind == "freq_radix_miss":
        cache = ctx.build_cache(ichee.CACHE_FREQ, CACHE_SEED, top_k=32, pool_size=16, miss_policy=1, radix_base=16,
                                scan=pix.copy())
        oc = o.freq_cache(pix, 32, 16, CACHE_SEED, radix_base=16)
        miss = 1
    else:
        cache = ctx.build_cache(ichee.CACHE_FULL, CACHE_SEED, pool_size=64)
        oc = o.full_cache(64, CACHE_SEED)
        miss = 0
    values, pool = ichee.ichee_cache_info(cache)
    assert values == oc["values"] and pool == oc["pool_size"]
    vc = np.zeros((len(values), 2, 3, ctx.n), dtype=np.uint64)
    ichee.ichee_cache_export(cache, 0, vc)
    assert np.array_equal(vc, oc["cts"])
    zc = np.zeros((pool, 2, 3, ctx.n), dtype=np.uint64)
    ichee.ichee_cache_export(cache, 1, zc)
    assert np.array_equal(zc, oc["pool"])
    ct, meta = ctx.encrypt(torch.from_numpy(pix).cuda(), 64, 64, 1, IMG_SEED, cache=cache)
    got = as_cts(ct, pix.size, 3, ctx.n)
    lut = oc["lut"]
    hits = np.nonzero(lut[pix] >= 0)[0]
    misses = np.nonzero(lut[pix] < 0)[0]
    rng = np.random.default_rng(7)
    idx = np.concatenate([rng.choice(hits, min(12, len(hits)), replace=False),
                          rng.choice(misses, min(6, len(misses)), replace=False) if len(misses) else []]).astype(np.int64)
    ref = o.encrypt_lookup(pix[idx], oc, IMG_SEED, miss_policy=miss, ids=idx.astype(np.uint64))
    for j, k in enumerate(idx):
        assert np.array_equal(got[k], ref[j]), (k, int(pix[k]))
    dec = ctx.decrypt(ct, meta).cpu().numpy()
    assert np.max(np.abs(dec - pix)) < 1e-3


# ------------------------------------------------------------- small-ring ops (a6, a7)
SMALL_OPS = dict(name="ops_n1024_l4", log_n=10, prime_bits=[60, 40, 40, 40], log2_scale=40, special_bits=61)


@pytest.fixture(scope="module")
def small_ops(ichee):
    wl = SMALL_OPS
    ctx = gpu_for(ichee, wl, with_evk=True)
    o = oracle_for(wl, with_evk=True)
    h, w, c = 5, 6, 3
    img = inputs.random_field_image(h, w, seed=3, channels=c).reshape(-1)
    img2 = inputs.noisy_copy(img, seed=6)
    wm = inputs.binary_pattern(h, w, seed=5).reshape(-1)
    g = {}
    g["a"], g["ma"] = ctx.encrypt(torch.from_numpy(img).cuda(), h, w, c, 11)
    g["b"], g["mb"] = ctx.encrypt(torch.from_numpy(img2).cuda(), h, w, c, 12)
    g["w"], g["mw"] = ctx.encrypt(torch.from_numpy(wm).cuda(), h, w, 1, 13)
    r = {"a": o.encrypt_pixels(img, 11), "b": o.encrypt_pixels(img2, 12), "w": o.encrypt_pixels(wm, 13)}
    for k in "abw":
        assert np.array_equal(as_cts(g[k], r[k].shape[0], 4, ctx.n), r[k])
    yield ctx, o, (h, w, c), (img, img2, wm), g, r
    ctx.close()


def test_ops_add_sub_ptmul_rescale_small(ichee, small_ops):
    ctx, o, (h, w, c), _, g, r = small_ops
    n, nct = ctx.n, h * w * c
    out, m = ctx.eval(ichee.OP_ADD, g["a"], g["ma"], g["b"], g["mb"])
    assert np.array_equal(as_cts(out, nct, 4, n), o.add(r["a"], r["b"]))
    out, m = ctx.eval(ichee.OP_SUB, g["a"], g["ma"], g["b"], g["mb"])
    assert np.array_equal(as_cts(out, nct, 4, n), o.sub(r["a"], r["b"]))
    out, m = ctx.eval(ichee.OP_PTMUL, g["a"], g["ma"], args=(-0.37,))
    ref, sc = o.ptmul(r["a"], o.delta, -0.37)
    assert np.array_equal(as_cts(out, nct, 4, n), ref)
    assert m.scale == float(sc) and m.level == 3
    out2, m2 = ctx.eval(ichee.OP_RESCALE, out, m, out_level=2)
    ref2 = o.rescale(ref)
    assert np.array_equal(as_cts(out2, nct, 3, n), ref2)
    assert m2.level == 2
    np.testing.assert_allclose(m2.scale, float(sc / int(o.q[3])), rtol=1e-15)
    dec = ctx.decrypt(out2, m2).cpu().numpy()
    np.testing.assert_allclose(dec, o.decrypt(ref2, sc / int(o.q[3])), rtol=1e-9)


def test_ops_brightness_watermark_small(ichee, small_ops):
    ctx, o, (h, w, c), (img, _, _), g, r = small_ops
    n, nct = ctx.n, h * w * c
    beta = inputs.brightness_beta(4)
    out, m = ctx.eval(ichee.OP_BRIGHTNESS, g["a"], g["ma"], args=(beta,))
    ref, sc = o.brightness(r["a"], o.delta, beta)
    assert np.array_equal(as_cts(out, nct, 4, n), ref)
    assert np.max(np.abs(ctx.decrypt(out, m).cpu().numpy() - (img + beta))) < 1e-3
    out, m = ctx.eval(ichee.OP_WATERMARK_PIXEL, g["a"], g["ma"], args=(5.0, 17))
    ref, _ = o.watermark_pixel(r["a"], o.delta, 5.0, 17)
    assert np.array_equal(as_cts(out, nct, 4, n), ref)
    # in place on a copy
    cp = g["a"].clone()
    ctx.eval(ichee.OP_WATERMARK_PIXEL, cp, g["ma"], args=(5.0, 17), out=cp)
    assert torch.equal(cp, out)
    # one constant per ciphertext
    vals = np.linspace(-3, 3, nct)
    out, m = ctx.eval(ichee.OP_PTADD, g["a"], g["ma"], args=tuple(vals))
    ref = o.add_int(r["a"], [o.encode_const(v, o.delta) for v in vals])
    assert np.array_equal(as_cts(out, nct, 4, n), ref)


def test_ops_meanfilter_blend_small(ichee, small_ops):
    ctx, o, (h, w, c), (img, _, wm), g, r = small_ops
    n, nct = ctx.n, h * w * c
    out, m = ctx.eval(ichee.OP_MEANFILTER3, g["a"], g["ma"], out_level=2)
    ref, sc = o.meanfilter3(r["a"], o.delta, h, w, c)
    assert np.array_equal(as_cts(out, nct, 3, n), ref)
    np.testing.assert_allclose(m.scale, float(sc), rtol=1e-15)
    dec = ctx.decrypt(out, m).cpu().numpy()
    np.testing.assert_allclose(dec, o.decrypt(ref, sc), rtol=1e-9)
    out, m = ctx.eval(ichee.OP_BLEND, g["a"], g["ma"], g["w"], g["mw"], args=(0.9,), out_level=2)
    ref, sc = o.blend(r["a"], r["w"], o.delta, 0.9, c, 1)
    assert np.array_equal(as_cts(out, nct, 3, n), ref)


def test_ops_match_small(ichee, small_ops):
    ctx, o, (h, w, c), (img, img2, _), g, r = small_ops
    out, m = ctx.eval(ichee.OP_SQDIFF_SUM, g["a"], g["ma"], g["b"], g["mb"], out_n_ct=1, out_level=2)
    ref, sc = o.match(r["a"], r["b"], o.delta)
    assert np.array_equal(as_cts(out, 1, 3, ctx.n), ref)
    assert (m.h, m.w, m.c, m.level) == (1, 1, 1, 2)
    dec = ctx.decrypt(out, m).cpu().numpy()
    np.testing.assert_allclose(dec, o.decrypt(ref, sc), rtol=1e-9)
    plain = float(((img.astype(np.float64) - img2) ** 2).sum())
    assert abs(dec[0] - plain) < 1e-2


def test_ops_sqdiff_image_small(ichee, small_ops):
    """Per-pixel squared difference, every ciphertext bit for bit, at the top level and one
    level down (the evaluation key's limbs truncated)."""
    ctx, o, (h, w, c), (img, img2, _), g, r = small_ops
    n, nct = ctx.n, h * w * c
    out, m = ctx.eval(ichee.OP_SQDIFF, g["a"], g["ma"], g["b"], g["mb"], out_level=2)
    ref, sc = o.sqdiff_image(r["a"], r["b"], o.delta)
    assert np.array_equal(as_cts(out, nct, 3, n), ref)
    assert (m.h, m.w, m.c, m.level) == (h, w, c, 2)
    np.testing.assert_allclose(m.scale, float(sc), rtol=1e-15)
    dec = ctx.decrypt(out, m).cpu().numpy()
    np.testing.assert_allclose(dec, o.decrypt(ref, sc), rtol=1e-9)
    assert np.max(np.abs(dec - (img.astype(np.float64) - img2) ** 2)) < 1e-3
    # one level down: x 1.0 at scale Delta, then rescale, keeps the scale near Delta
    def down(ct, meta):
        p, mp = ctx.eval(ichee.OP_PTMUL, ct, meta, args=(1.0,))
        return ctx.eval(ichee.OP_RESCALE, p, mp, out_level=2)

    a2, ma2 = down(g["a"], g["ma"])
    b2, mb2 = down(g["b"], g["mb"])
    out2, m2 = ctx.eval(ichee.OP_SQDIFF, a2, ma2, b2, mb2, out_level=1)
    ra2 = o.rescale(o.ptmul(r["a"], o.delta, 1.0)[0])
    rb2 = o.rescale(o.ptmul(r["b"], o.delta, 1.0)[0])
    sc_in = Fraction(o.delta) * o.delta / int(o.q[3])
    ref2, sc2 = o.sqdiff_image(ra2, rb2, sc_in)
    assert np.array_equal(as_cts(out2, nct, 2, n), ref2)
    np.testing.assert_allclose(m2.scale, float(sc2), rtol=1e-12)
    assert np.max(np.abs(ctx.decrypt(out2, m2).cpu().numpy() - (img.astype(np.float64) - img2) ** 2)) < 1e-2


def test_ops_sqdiff_image_more_pixels_than_blocks(ichee, small_ops):
    """700 ciphertexts: more than one persistent block's worth, every output compared."""
    ctx, o = small_ops[0], small_ops[1]
    h, w, c = 10, 35, 2
    a = inputs.random_field_image(h, w, seed=31, channels=c).reshape(-1)
    b = inputs.noisy_copy(a, seed=32)
    ga, ma = ctx.encrypt(torch.from_numpy(a).cuda(), h, w, c, 33)
    gb, mb = ctx.encrypt(torch.from_numpy(b).cuda(), h, w, c, 34)
    out, m = ctx.eval(ichee.OP_SQDIFF, ga, ma, gb, mb, out_level=2)
    ref, sc = o.sqdiff_image(o.encrypt_pixels(a, 33), o.encrypt_pixels(b, 34), o.delta)
    got = as_cts(out, h * w * c, 3, ctx.n)
    bad = [k for k in range(h * w * c) if not np.array_equal(got[k], ref[k])]
    assert not bad, bad[:10]


# ------------------------------------------------------------- the 2^14 ring (serving size)
def test_ring16384_keys_encryption_and_matching(ichee):
    """N = 16384, five primes: the transform and encryption kernels of this ring recompute
    NTT(v) per product and the matching accumulator parks d0 in global scratch."""
    wl = W.RING16384
    ctx = gpu_for(ichee, wl, with_evk=True)
    o = oracle_for(wl, with_evk=True)
    n, L = ctx.n, ctx.L
    pk = np.zeros((2, L, n), dtype=np.uint64)
    ichee.ichee_export_key(ctx.handle, 1, pk)
    assert np.array_equal(pk, o.pk)
    evk = np.zeros((L, 2, L + 1, n), dtype=np.uint64)
    ichee.ichee_export_key(ctx.handle, 2, evk)
    assert np.array_equal(evk, o.evk)
    a = inputs.random_field_image(3, 2, seed=14).reshape(-1).copy()
    b = inputs.noisy_copy(a, seed=15)
    ga, ma = ctx.encrypt(torch.from_numpy(a).cuda(), 3, 2, 1, 61)
    gb, mb = ctx.encrypt(torch.from_numpy(b).cuda(), 3, 2, 1, 62)
    ra, rb = o.encrypt_pixels(a, 61), o.encrypt_pixels(b, 62)
    assert np.array_equal(as_cts(ga, 6, L, n), ra)
    assert np.array_equal(as_cts(gb, 6, L, n), rb)
    assert np.max(np.abs(ctx.decrypt(ga, ma).cpu().numpy() - a)) < 1e-3
    # radix 10 on this ring: the sums of the top two positions would take 84 ciphertexts of
    # 1.3 MB, above the 48 MB bound, so the combine reads the three positions one by one (the
    # N = 8192 and toy-ring tests cover the summed table)
    edge = np.array([0, 255, 100, 9, 200, 99], dtype=np.uint8)
    cache = ctx.build_cache(ichee.CACHE_RADIX, 35, radix_base=10, randomize=1)
    gr, mr = ctx.encrypt(torch.from_numpy(edge).cuda(), 3, 2, 1, 36, cache=cache)
    assert np.array_equal(as_cts(gr, 6, L, n), o.encrypt_radix(edge, o.radix_cache(10, 35), 36, randomize=True))
    assert np.max(np.abs(ctx.decrypt(gr, mr).cpu().numpy() - edge)) < 1e-3
    out, m = ctx.eval(ichee.OP_SQDIFF_SUM, ga, ma, gb, mb, out_n_ct=1, out_level=L - 2)
    ref, sc = o.match(ra, rb, o.delta)
    assert np.array_equal(as_cts(out, 1, L - 1, n), ref)
    assert abs(ctx.decrypt(out, m).cpu().numpy()[0] - float(((a.astype(float) - b) ** 2).sum())) < 1e-2
    mf, mm = ctx.eval(ichee.OP_MEANFILTER3, ga, ma, out_level=L - 2)
    rf, sf = o.meanfilter3(ra, o.delta, 3, 2, 1)
    assert np.array_equal(as_cts(mf, 6, L - 1, n), rf)
    sq, ms = ctx.eval(ichee.OP_SQDIFF, ga, ma, gb, mb, out_level=L - 2)
    rs, ss = o.sqdiff_image(ra, rb, o.delta)
    assert np.array_equal(as_cts(sq, 6, L - 1, n), rs)
    assert np.max(np.abs(ctx.decrypt(sq, ms).cpu().numpy() - (a.astype(float) - b) ** 2)) < 1e-2
    ctx.close()


# ------------------------------------------------------------- saved keys, key-only contexts
def test_saved_keys_resume_and_public_only_context(ichee, tmp_path):
    """Keys saved and loaded into a fresh context give the same ciphertexts; a context holding
    only the public and evaluation keys encrypts and matches but cannot decrypt, and the
    secret-key holder decrypts its results; bad imports are refused."""
    wl = SMALL_OPS
    a = inputs.random_field_image(3, 4, seed=81).reshape(-1).copy()
    b = inputs.noisy_copy(a, seed=82)
    src = gpu_for(ichee, wl, with_evk=True)
    src.save_keys(str(tmp_path / "all.npz"))
    src.save_keys(str(tmp_path / "public.npz"), secret=False)
    ra, ma = src.encrypt(torch.from_numpy(a).cuda(), 3, 4, 1, 5)
    rb, mb = src.encrypt(torch.from_numpy(b).cuda(), 3, 4, 1, 6)
    rm, mm = src.eval(ichee.OP_SQDIFF_SUM, ra, ma, rb, mb, out_n_ct=1, out_level=2)
    resumed = ichee.Context(**W.ctx_kwargs(wl))
    resumed.load_keys(str(tmp_path / "all.npz"))
    ga, _ = resumed.encrypt(torch.from_numpy(a).cuda(), 3, 4, 1, 5)
    assert torch.equal(ga, ra)
    np.testing.assert_array_equal(resumed.decrypt(ga, ma).cpu().numpy(), src.decrypt(ra, ma).cpu().numpy())
    server = ichee.Context(**W.ctx_kwargs(wl))
    server.load_keys(str(tmp_path / "public.npz"))
    sa, sma = server.encrypt(torch.from_numpy(a).cuda(), 3, 4, 1, 5)
    sb, smb = server.encrypt(torch.from_numpy(b).cuda(), 3, 4, 1, 6)
    sm_, smm = server.eval(ichee.OP_SQDIFF_SUM, sa, sma, sb, smb, out_n_ct=1, out_level=2)
    assert torch.equal(sa, ra) and torch.equal(sm_, rm)
    with pytest.raises(ichee.IcheeError) as e:
        server.decrypt(sm_, smm)
    assert e.value.status == ichee.EINVAL
    assert abs(float(src.decrypt(sm_, smm).cpu()[0]) - float(((a.astype(float) - b) ** 2).sum())) < 1e-2
    bad = np.zeros(server.n, dtype=np.int8)
    bad[3] = 2
    with pytest.raises(ichee.IcheeError) as e:
        ichee.ichee_import_key(server.handle, 0, bad)
    assert e.value.status == ichee.EINVAL
    with pytest.raises(ichee.IcheeError) as e:
        ichee.ichee_import_key(server.handle, 1, np.zeros(7, dtype=np.uint64))
    assert e.value.status == ichee.EINVAL
    other = ichee.Context(**W.ctx_kwargs(W.TOY))
    with pytest.raises(ichee.IcheeError):
        other.load_keys(str(tmp_path / "all.npz"))
    for c in (src, resumed, server, other):
        c.close()


# ------------------------------------------------------------- working-memory allocator
def test_torch_allocator_serves_working_memory(ichee):
    """Host-buffer encryption and decryption (staging) and matching (scratch) through PyTorch's
    caching allocator give the same bits as with cudaMalloc; an allocator that fails makes the
    call fail with ENOMEM and leaves the context usable."""
    wl = SMALL_OPS
    h, w, c = 4, 5, 1
    a = inputs.random_field_image(h, w, seed=41).reshape(-1).copy()
    b = inputs.noisy_copy(a, seed=42)
    res = []
    for use_torch in (False, True):
        ctx = gpu_for(ichee, wl, with_evk=True)
        log = ctx.use_torch_allocator() if use_torch else None
        ga, ma = ctx.encrypt(torch.from_numpy(a), h, w, c, 11)      # host pixels: staged
        gb, mb = ctx.encrypt(torch.from_numpy(b), h, w, c, 12)
        m_out, mm = ctx.eval(ichee.OP_SQDIFF_SUM, ga, ma, gb, mb, out_n_ct=1, out_level=2)
        dec = torch.empty(h * w * c, dtype=torch.float64)                # host output: staged
        ichee.ichee_decrypt_image(ctx.handle, ga, ma, dec, ctx.stream())
        torch.cuda.synchronize()
        res.append((ga.cpu(), m_out.cpu(), dec.clone()))
        if use_torch:
            assert len(log) >= 3 and all(n > 0 and p != 0 for n, p in log)
            failing = ichee.ALLOC_FN(lambda n, s_, u: 0)
            keep = ichee.FREE_FN(lambda p, s_, u: None)
            ichee.ichee_set_allocator(ctx.handle, failing, keep)
            with pytest.raises(ichee.IcheeError) as e:
                ctx.eval(ichee.OP_SQDIFF_SUM, ga, ma, gb, mb, out_n_ct=1, out_level=2)
            assert e.value.status == ichee.ENOMEM
            ichee.ichee_set_allocator(ctx.handle, None, None)
            again, _ = ctx.eval(ichee.OP_SQDIFF_SUM, ga, ma, gb, mb, out_n_ct=1, out_level=2)
            assert torch.equal(again.cpu(), res[0][1])
        ctx.close()
    assert all(torch.equal(x, y) for x, y in zip(res[0], res[1]))


# ------------------------------------------------------------- degenerate pixel values
def test_degenerate_pixel_values(ichee):
    """Pixels 0 and 255 and values with a single nonzero radix digit, through every cache kind
    (radix 2 / 7 / 10 / 15 / 16 with and without randomness, full cache with the pool): bit for bit
    against the oracle. Without randomness pixel 0 has no nonzero digit and encrypts to the
    all-zero ciphertext -- the paper's method as stated; its randomness removes that. A
    constant 255 image keeps its value through the mean filter."""
    wl = W.TOY
    ctx = gpu_for(ichee, wl)
    o = oracle_for(wl)
    pix = np.array([0, 255, 1, 16, 240, 128, 2, 100, 0, 255, 10, 15], dtype=np.uint8)
    dp = torch.from_numpy(pix).cuda()
    for base in (2, 7, 10, 15, 16):   # 8, 3, 3, 3 and 2 positions; 7 to 15 and 2 use the pair table
        for rnd in (0, 1):
            cache = ctx.build_cache(ichee.CACHE_RADIX, CACHE_SEED + base, radix_base=base, randomize=rnd)
            ct, meta = ctx.encrypt(dp, 3, 4, 1, IMG_SEED, cache=cache)
            ref = o.encrypt_radix(pix, o.radix_cache(base, CACHE_SEED + base), IMG_SEED, randomize=bool(rnd))
            got = as_cts(ct, 12, 2, ctx.n)
            assert np.array_equal(got, ref), (base, rnd)
            assert np.max(np.abs(ctx.decrypt(ct, meta).cpu().numpy() - pix)) < 1e-3
            if not rnd:
                assert not got[0].any() and not got[8].any()   # pixel 0: the zero ciphertext
    full = ctx.build_cache(ichee.CACHE_FULL, CACHE_SEED, pool_size=8)
    ct, meta = ctx.encrypt(dp, 3, 4, 1, IMG_SEED, cache=full)
    ref = o.encrypt_lookup(pix, o.full_cache(8, CACHE_SEED), IMG_SEED)
    assert np.array_equal(as_cts(ct, 12, 2, ctx.n), ref)
    ctx.close()
    # constant image through the mean filter (four-prime ring: a limb to drop)
    ctx = gpu_for(ichee, SMALL_OPS)
    o = oracle_for(SMALL_OPS)
    const = np.full(5 * 6, 255, dtype=np.uint8)
    ct, meta = ctx.encrypt(torch.from_numpy(const).cuda(), 5, 6, 1, IMG_SEED)
    mf, mm = ctx.eval(ichee.OP_MEANFILTER3, ct, meta, out_level=2)
    ref, sc = o.meanfilter3(o.encrypt_pixels(const, IMG_SEED), o.delta, 5, 6, 1)
    assert np.array_equal(as_cts(mf, 30, 3, ctx.n), ref)
    assert np.max(np.abs(ctx.decrypt(mf, mm).cpu().numpy() - 255.0)) < 0.05
    ctx.close()


# ------------------------------------------------- the paper's ring size and N = 2048
@pytest.mark.parametrize("wl", [
    dict(name="paper_n4096_q109", log_n=12, prime_bits=[45, 32, 32], log2_scale=32, special_bits=50),
    dict(name="n2048", log_n=11, prime_bits=[45, 30, 30], log2_scale=30, special_bits=50),
    dict(name="n1024_8primes", log_n=10, prime_bits=[50, 40, 40, 40, 40, 40, 40, 40], log2_scale=40,
         special_bits=58),
], ids=lambda w: w["name"])
def test_other_rings_bit_exact(ichee, wl):
    """N = 4096 with a 109-bit ciphertext modulus (the paper's parameter set), N = 2048, and
    the largest limb count the library takes (8 primes): keys, fresh and radix encryption, mean
    filter, matching and the per-pixel squared difference, every ciphertext word against the
    oracle."""
    ctx = gpu_for(ichee, wl, with_evk=True)
    o = oracle_for(wl, with_evk=True)
    n, L = ctx.n, ctx.L
    pk = np.zeros((2, L, n), dtype=np.uint64)
    ichee.ichee_export_key(ctx.handle, 1, pk)
    assert np.array_equal(pk, o.pk)
    evk = np.zeros((L, 2, L + 1, n), dtype=np.uint64)
    ichee.ichee_export_key(ctx.handle, 2, evk)
    assert np.array_equal(evk, o.evk)
    h, w = 4, 5
    a = inputs.random_field_image(h, w, seed=91).reshape(-1).copy()
    b = inputs.noisy_copy(a, seed=92)
    ga, ma = ctx.encrypt(torch.from_numpy(a).cuda(), h, w, 1, 31)
    gb, mb = ctx.encrypt(torch.from_numpy(b).cuda(), h, w, 1, 32)
    ra, rb = o.encrypt_pixels(a, 31), o.encrypt_pixels(b, 32)
    assert np.array_equal(as_cts(ga, h * w, L, n), ra)
    assert np.max(np.abs(ctx.decrypt(ga, ma).cpu().numpy() - a)) < 1e-3
    cache = ctx.build_cache(ichee.CACHE_RADIX, 33, radix_base=16, randomize=1)
    gr, _ = ctx.encrypt(torch.from_numpy(a).cuda(), h, w, 1, 34, cache=cache)
    rr = o.encrypt_radix(a, o.radix_cache(16, 33), 34, randomize=True)
    assert np.array_equal(as_cts(gr, h * w, L, n), rr)
    mf, mm = ctx.eval(ichee.OP_MEANFILTER3, ga, ma, out_level=L - 2)
    rf, _ = o.meanfilter3(ra, o.delta, h, w, 1)
    assert np.array_equal(as_cts(mf, h * w, L - 1, n), rf)
    m1, mm1 = ctx.eval(ichee.OP_SQDIFF_SUM, ga, ma, gb, mb, out_n_ct=1, out_level=L - 2)
    r1, s1 = o.match(ra, rb, o.delta)
    assert np.array_equal(as_cts(m1, 1, L - 1, n), r1)
    sq, _ = ctx.eval(ichee.OP_SQDIFF, ga, ma, gb, mb, out_level=L - 2)
    rs, _ = o.sqdiff_image(ra, rb, o.delta)
    assert np.array_equal(as_cts(sq, h * w, L - 1, n), rs)
    np.testing.assert_allclose(ctx.decrypt(m1, mm1).cpu().numpy(), o.decrypt(r1, s1), rtol=1e-9)
    ctx.close()


# ------------------------------------------------------------------------ errors
def test_error_paths(ichee):
    wl = W.TOY
    ctx = gpu_for(ichee, wl)
    pix = torch.zeros(4, dtype=torch.uint8, device="cuda")
    with pytest.raises(ichee.IcheeError) as e:
        ctx.encrypt(pix, 0, 2, 2, 1)
    assert e.value.status == ichee.EINVAL
    host_out = np.zeros(ctx.ct_words(1) * 4, dtype=np.uint64)
    with pytest.raises(ichee.IcheeError) as e:
        ichee.ichee_encrypt_image(ctx.handle, None, pix, 2, 2, 1, 1, host_out, ctx.stream())
    assert e.value.status == ichee.EINVAL
    small = ctx.empty_cts(4, ctx.L - 1)
    for shape in ((1 << 31, 1 << 31, 1), (1 << 20, 1 << 20, 2)):   # products beyond 2^40 ciphertexts
        with pytest.raises(ichee.IcheeError) as e:
            ichee.ichee_encrypt_image(ctx.handle, None, pix, *shape, 1, small, ctx.stream())
        assert e.value.status == ichee.EINVAL and "oversized" in str(e.value)
        with pytest.raises(ichee.IcheeError) as e:
            ichee.ichee_encrypt_batch(ctx.handle, None, [pix], [shape], [1], [small], ctx.stream())
        assert e.value.status == ichee.EINVAL
    ct, m = ctx.encrypt(pix, 2, 2, 1, 1)
    r1, m1 = ctx.eval(ichee.OP_RESCALE, ct, m, out_level=0)
    with pytest.raises(ichee.IcheeError) as e:
        ctx.eval(ichee.OP_RESCALE, r1, m1)
    assert e.value.status == ichee.ELEVEL
    p2, mp = ctx.eval(ichee.OP_PTMUL, ct, m, args=(2.0,))
    with pytest.raises(ichee.IcheeError) as e:
        ctx.eval(ichee.OP_ADD, ct, m, p2, mp)
    assert e.value.status == ichee.ESCALE
    with pytest.raises(ichee.IcheeError) as e:
        ctx.eval(ichee.OP_SQDIFF_SUM, ct, m, ct, m, out_n_ct=1)
    assert e.value.status == ichee.EUNSUPPORTED
    with pytest.raises(ichee.IcheeError) as e:
        ctx.eval(ichee.OP_SQDIFF, ct, m, ct, m)
    assert e.value.status == ichee.EUNSUPPORTED
    other = gpu_for(ichee, wl)
    cache = other.build_cache(ichee.CACHE_RADIX, 1, radix_base=16)
    with pytest.raises(ichee.IcheeError) as e:
        ctx.encrypt(pix, 2, 2, 1, 1, cache=cache)
    assert e.value.status == ichee.EMISMATCH
    with pytest.raises(ichee.IcheeError):
        ichee.Context(log_n=9, prime_bits=[30], log2_scale=20)
    ctx.status()
    other.close()
    ctx.close()


def test_short_device_buffers_are_refused(ichee):
    """A device buffer that ends before the bytes a call needs is refused before any launch (the
    bound is the allocation holding it, from the driver's address-range query); the context
    stays usable."""
    ctx = gpu_for(ichee, W.TOY)
    h = w = 32
    gen = torch.Generator().manual_seed(5)
    pix = torch.randint(0, 256, (h * w,), dtype=torch.uint8, generator=gen).cuda()
    one = ctx.empty_cts(1, ctx.L - 1)                  # room for one ciphertext only
    need = h * w * ctx.ct_words(ctx.L - 1) * 8
    try:
        left = ichee.ichee_buffer_bytes_left(one)
    except ichee.IcheeError:
        pytest.skip("the driver reports no allocation extents here")
    if not 0 < left < need:  # every call below must be refused on the host, never launched
        pytest.skip("the allocator's segment is larger than the image (virtual-memory segments)")
    with pytest.raises(ichee.IcheeError) as e:
        ctx.encrypt(pix, h, w, 1, 1, out=one)
    assert e.value.status == ichee.EINVAL and "allocation" in str(e.value)
    ct, m = ctx.encrypt(pix, h, w, 1, 1)
    with pytest.raises(ichee.IcheeError) as e:
        ctx.eval(ichee.OP_ADD, ct, m, ct, m, out=one)
    assert e.value.status == ichee.EINVAL
    with pytest.raises(ichee.IcheeError) as e:
        ctx.decrypt(one, m)                            # metadata promises 1024 ciphertexts
    assert e.value.status == ichee.EINVAL
    with pytest.raises(ichee.IcheeError) as e:
        ichee.ichee_encrypt_batch(ctx.handle, None, [pix, pix], [(h, w, 1), (h, w, 1)], [1, 2],
                                  [ctx.empty_cts(h * w, ctx.L - 1), one], ctx.stream())
    assert e.value.status == ichee.EINVAL and "image 1" in str(e.value)
    ctx.status()
    np.testing.assert_array_equal(np.rint(ctx.decrypt(ct, m).cpu().numpy()), pix.cpu().numpy())
    ctx.close()


def test_integer_probe_reports_rates(ichee):
    """The throughput probe runs and reports plausible rates (a measurement utility)."""
    imad, bfly = ichee.ichee_probe_int_throughput(0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    per_sm_per_ghz = imad / sms / 1e9
    assert 8 < per_sm_per_ghz < 512
    assert 1e9 < bfly < imad
