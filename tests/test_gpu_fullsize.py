"""GPU parity at full sizes, on sampled outputs the oracle computes one by one.

* The benchmark's launch configuration: the 64x64 image at N = 8192, primes 60/40/60 (plus the
  61-bit special prime of the evaluation key), every image operation the benchmark step runs.
* The four-prime operations workload: a 128x128x3 image at N = 8192, primes 60/40/40/40.
* The 32-image ragged batch (radix-16 encryption + mean filter, 142 GB of ciphertexts) in the
  batched entry points' default launch shapes.

For a sampled output pixel the oracle encrypts exactly the input pixels that output depends
on (same seeds, same ciphertext ids) and applies its own operation; the GPU ciphertext must
match bit for bit. Matching sums over every pixel, so at full size it is checked by its
decrypted value against the plaintext sum of squares, and bit for bit on a 16x16 crop.
"""
import numpy as np
import pytest

from oracle import Oracle, Params
from paper_2409_03568_gb300 import inputs, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEY_SEED = 55
SEED_A, SEED_W, SEED_B = 71, 72, 73


@pytest.fixture(scope="module")
def ichee():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03568_gb300 import ichee as mod
    return mod


def as_cts(t, n_ct, limbs, n):
    return t.cpu().numpy().view(np.uint64).reshape(n_ct, 2, limbs, n)


def _clamp(v, hi):
    return min(max(v, 0), hi - 1)


def check_meanfilter_samples(o, img, h, w, c, seed, got, idx):
    """Oracle mean filter at sampled output indices from the 9 clamped neighbours."""
    flat = img.reshape(-1)
    for k in idx:
        pix, ch = divmod(int(k), c)
        y, x = divmod(pix, w)
        nb = [(_clamp(y + dy, h) * w + _clamp(x + dx, w)) * c + ch for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
        patch = o.encrypt_pixels(flat[nb], seed, ids=np.array(nb, dtype=np.uint64))
        out, _ = o.meanfilter3(patch, o.delta, 3, 3, 1)
        assert np.array_equal(got[k], out[4]), (k, y, x, ch)


def sample_idx(n_ct, count, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, n_ct - 1], rng.choice(n_ct, count, replace=False)]))


@pytest.fixture(scope="module")
def bench_cfg(ichee):
    wl = dict(W.ENC8192)
    ctx = ichee.Context(**W.ctx_kwargs(wl))
    ctx.keygen(KEY_SEED, with_evk=True)
    o = Oracle(Params(wl["log_n"], wl["prime_bits"], wl["log2_scale"], wl["special_bits"])).keygen(KEY_SEED, True)
    h, w, c = wl["h"], wl["w"], wl["c"]
    img = W.image_for(wl).reshape(-1)
    wm = inputs.binary_pattern(h, w, seed=5).reshape(-1)
    noisy = inputs.noisy_copy(img, seed=6)
    g = {}
    g["a"], g["ma"] = ctx.encrypt(torch.from_numpy(img).cuda(), h, w, c, SEED_A)
    g["w"], g["mw"] = ctx.encrypt(torch.from_numpy(wm).cuda(), h, w, 1, SEED_W)
    g["b"], g["mb"] = ctx.encrypt(torch.from_numpy(noisy).cuda(), h, w, c, SEED_B)
    yield ctx, o, (h, w, c), (img, wm, noisy), g
    ctx.close()


def test_bench_cfg_meanfilter_sampled(ichee, bench_cfg):
    ctx, o, (h, w, c), (img, _, _), g = bench_cfg
    out, m = ctx.eval(ichee.OP_MEANFILTER3, g["a"], g["ma"], out_level=1)
    got = as_cts(out, h * w * c, 2, ctx.n)
    check_meanfilter_samples(o, img, h, w, c, SEED_A, got, sample_idx(h * w * c, 10, 1))
    dec = ctx.decrypt(out, m).cpu().numpy().reshape(h, w)
    f = img.reshape(h, w).astype(np.float64)
    ref = sum(f[np.clip(np.arange(h) + dy, 0, h - 1)][:, np.clip(np.arange(w) + dx, 0, w - 1)]
              for dy in (-1, 0, 1) for dx in (-1, 0, 1)) / 9.0
    # the rescale by the 60-bit prime leaves scale ~2^20: rounding noise ~ N / 2^20
    assert np.max(np.abs(dec - ref)) < 0.05


def test_bench_cfg_brightness_blend_sampled(ichee, bench_cfg):
    ctx, o, (h, w, c), (img, wm, _), g = bench_cfg
    beta = inputs.brightness_beta(4)
    n_ct = h * w * c
    out_b, mb = ctx.eval(ichee.OP_BRIGHTNESS, g["a"], g["ma"], args=(beta,))
    out_l, ml = ctx.eval(ichee.OP_BLEND, g["a"], g["ma"], g["w"], g["mw"], args=(0.9,), out_level=1)
    gb = as_cts(out_b, n_ct, 3, ctx.n)
    gl = as_cts(out_l, n_ct, 2, ctx.n)
    idx = sample_idx(n_ct, 12, 2)
    ca = o.encrypt_pixels(img[idx], SEED_A, ids=idx.astype(np.uint64))
    cw = o.encrypt_pixels(wm[idx // c], SEED_W, ids=(idx // c).astype(np.uint64))
    rb, _ = o.brightness(ca, o.delta, beta)
    rl, _ = o.blend(ca, cw, o.delta, 0.9, 1, 1)
    for j, k in enumerate(idx):
        assert np.array_equal(gb[k], rb[j]), k
        assert np.array_equal(gl[k], rl[j]), k
    assert np.max(np.abs(ctx.decrypt(out_b, mb).cpu().numpy() - (img + beta))) < 1e-3
    ref = 0.9 * img.astype(np.float64) + 0.1 * wm.astype(np.float64)
    assert np.max(np.abs(ctx.decrypt(out_l, ml).cpu().numpy() - ref)) < 0.05


def test_bench_cfg_matching(ichee, bench_cfg):
    ctx, o, (h, w, c), (img, _, noisy), g = bench_cfg
    out, m = ctx.eval(ichee.OP_SQDIFF_SUM, g["a"], g["ma"], g["b"], g["mb"], out_n_ct=1, out_level=1)
    plain = float(((img.astype(np.float64) - noisy) ** 2).sum())
    dec = float(ctx.decrypt(out, m).cpu().numpy()[0])
    assert abs(dec - plain) < 1e-6 * plain + 0.05
    # bit for bit on a 16x16 crop (the oracle sums every pixel)
    crop = np.arange(16 * 16)
    rows = (crop // 16) * w + crop % 16
    ca = torch.from_numpy(img.reshape(h, w)[:16, :16].reshape(-1).copy()).cuda()
    cb = torch.from_numpy(noisy.reshape(h, w)[:16, :16].reshape(-1).copy()).cuda()
    ga, ma = ctx.encrypt(ca, 16, 16, 1, SEED_A)
    gb, mb = ctx.encrypt(cb, 16, 16, 1, SEED_B)
    gout, gm = ctx.eval(ichee.OP_SQDIFF_SUM, ga, ma, gb, mb, out_n_ct=1, out_level=1)
    ra = o.encrypt_pixels(img[rows], SEED_A, ids=np.arange(256, dtype=np.uint64))
    rb = o.encrypt_pixels(noisy[rows], SEED_B, ids=np.arange(256, dtype=np.uint64))
    ref, sc = o.match(ra, rb, o.delta)
    assert np.array_equal(as_cts(gout, 1, 2, ctx.n), ref)
    np.testing.assert_allclose(ctx.decrypt(gout, gm).cpu().numpy(), o.decrypt(ref, sc), rtol=1e-9)


def test_bench_cfg_sqdiff_image_sampled(ichee, bench_cfg):
    """Per-pixel squared difference over the whole 64x64 image: sampled ciphertexts bit for
    bit, every pixel's decoded value against the plaintext square."""
    ctx, o, (h, w, c), (img, _, noisy), g = bench_cfg
    n_ct = h * w * c
    out, m = ctx.eval(ichee.OP_SQDIFF, g["a"], g["ma"], g["b"], g["mb"], out_level=1)
    got = as_cts(out, n_ct, 2, ctx.n)
    idx = sample_idx(n_ct, 4, 6)
    ra = o.encrypt_pixels(img[idx], SEED_A, ids=idx.astype(np.uint64))
    rb = o.encrypt_pixels(noisy[idx], SEED_B, ids=idx.astype(np.uint64))
    ref, sc = o.sqdiff_image(ra, rb, o.delta)
    for j, k in enumerate(idx):
        assert np.array_equal(got[k], ref[j]), k
    dec = ctx.decrypt(out, m).cpu().numpy()
    assert np.max(np.abs(dec - (img.astype(np.float64) - noisy) ** 2)) < 0.05


@pytest.fixture(scope="module")
def ops_full(ichee):
    wl = W.OPS8192
    ctx = ichee.Context(**W.ctx_kwargs(wl))
    ctx.keygen(KEY_SEED, with_evk=True)
    o = Oracle(Params(wl["log_n"], wl["prime_bits"], wl["log2_scale"], wl["special_bits"])).keygen(KEY_SEED, True)
    h, w, c = wl["h"], wl["w"], wl["c"]
    img = W.image_for(wl)
    yield ctx, o, wl, img
    ctx.close()


def test_ops_128x128x3_meanfilter_and_brightness(ichee, ops_full):
    ctx, o, wl, img = ops_full
    h, w, c = wl["h"], wl["w"], wl["c"]
    flat = img.reshape(-1)
    n_ct = flat.size
    a, ma = ctx.encrypt(torch.from_numpy(flat).cuda(), h, w, c, SEED_A)
    out, m = ctx.eval(ichee.OP_MEANFILTER3, a, ma, out_level=2)
    got = as_cts(out, n_ct, 3, ctx.n)
    idx = sample_idx(n_ct, 6, 3)
    # include the four corners and an edge pixel of channel 2
    corners = [((y * w + x) * c + 2) for y, x in ((0, 0), (0, w - 1), (h - 1, 0), (h - 1, w - 1), (0, 7))]
    check_meanfilter_samples(o, flat, h, w, c, SEED_A, got, np.unique(np.concatenate([idx, corners])))
    del out, got
    beta = inputs.brightness_beta(wl["beta_seed"])
    ob, mb = ctx.eval(ichee.OP_BRIGHTNESS, a, ma, args=(beta,))
    dec = ctx.decrypt(ob, mb).cpu().numpy()
    assert np.max(np.abs(dec - (flat + beta))) < 1e-3
    sidx = sample_idx(n_ct, 8, 4)
    rb, _ = o.brightness(o.encrypt_pixels(flat[sidx], SEED_A, ids=sidx.astype(np.uint64)), o.delta, beta)
    gb = as_cts(ob, n_ct, 4, ctx.n)
    for j, k in enumerate(sidx):
        assert np.array_equal(gb[k], rb[j]), k


def test_ops_128x128x3_blend_and_matching(ichee, ops_full):
    ctx, o, wl, img = ops_full
    h, w, c = wl["h"], wl["w"], wl["c"]
    flat = img.reshape(-1)
    n_ct = flat.size
    wm = inputs.binary_pattern(h, w, seed=wl["watermark_seed"]).reshape(-1)
    noisy = inputs.noisy_copy(flat, seed=wl["noisy_seed"])
    a, ma = ctx.encrypt(torch.from_numpy(flat).cuda(), h, w, c, SEED_A)
    cw, mw = ctx.encrypt(torch.from_numpy(wm).cuda(), h, w, 1, SEED_W)
    out, m = ctx.eval(ichee.OP_BLEND, a, ma, cw, mw, args=(wl["alpha"],), out_level=2)
    idx = sample_idx(n_ct, 8, 5)
    got = as_cts(out, n_ct, 3, ctx.n)
    ca = o.encrypt_pixels(flat[idx], SEED_A, ids=idx.astype(np.uint64))
    cwr = o.encrypt_pixels(wm[idx // c], SEED_W, ids=(idx // c).astype(np.uint64))
    rl, _ = o.blend(ca, cwr, o.delta, wl["alpha"], 1, 1)
    for j, k in enumerate(idx):
        assert np.array_equal(got[k], rl[j]), k
    ref = wl["alpha"] * flat + (1 - wl["alpha"]) * np.repeat(wm, c).astype(np.float64)
    assert np.max(np.abs(ctx.decrypt(out, m).cpu().numpy() - ref)) < 1e-4
    del out, got
    b, mb = ctx.encrypt(torch.from_numpy(noisy).cuda(), h, w, c, SEED_B)
    om, mm = ctx.eval(ichee.OP_SQDIFF_SUM, a, ma, b, mb, out_n_ct=1, out_level=2)
    plain = float(((flat.astype(np.float64) - noisy) ** 2).sum())
    dec = float(ctx.decrypt(om, mm).cpu().numpy()[0])
    assert abs(dec - plain) < 1e-7 * plain + 0.01


def test_batch32_full_size_sampled(ichee):
    """The 32-image ragged batch at its full size (216,613 pixels, 142 GB of ciphertexts) through
    the batched radix-16 encryption and the batched mean filter in their default launch shapes
    (the autotuner's choice for this batch): sampled ciphertexts and filter outputs of the
    first, the largest and the last image against the oracle, one by one."""
    wl = W.BATCH32
    imgs = inputs.ragged_batch(wl["n_images"], wl["batch_seed"], wl["side_lo"], wl["side_hi"])
    shapes = [(im.shape[0], im.shape[1], 1) for im in imgs]
    n_total = sum(h * w for h, w, _ in shapes)
    need = n_total * (393216 + 262144)
    free, _ = torch.cuda.mem_get_info()
    if free < need + (16 << 30):
        pytest.skip("needs %.0f GB of free device memory" % (need / 1e9))
    ctx = ichee.Context(**W.ctx_kwargs(wl))
    ctx.keygen(77)
    cache = ctx.build_cache(ichee.CACHE_RADIX, 15, radix_base=wl["radix_base"], randomize=1)
    seeds = [500 + i for i in range(len(imgs))]
    d_px = [torch.from_numpy(im.reshape(-1).copy()).cuda() for im in imgs]
    enc = [ctx.empty_cts(h * w, 2) for h, w, _ in shapes]
    filt = [ctx.empty_cts(h * w, 1) for h, w, _ in shapes]
    metas = ichee.ichee_encrypt_batch(ctx.handle, cache, d_px, shapes, seeds, enc, ctx.stream())
    ichee.ichee_eval_batch(ctx.handle, ichee.OP_MEANFILTER3, enc, metas, outs=filt, stream=ctx.stream())
    torch.cuda.synchronize()
    ctx.status()
    o = Oracle(Params(wl["log_n"], wl["prime_bits"], wl["log2_scale"])).keygen(77)
    oc = o.radix_cache(wl["radix_base"], 15)
    n = ctx.n
    largest = int(np.argmax([h * w for h, w, _ in shapes]))
    try:
        for i in (0, largest, len(imgs) - 1):
            h, w, _ = shapes[i]
            flat = imgs[i].reshape(-1)
            idx = sample_idx(h * w, 3, seed=i)
            sel = torch.from_numpy(idx.astype(np.int64)).cuda()
            got_e = enc[i].view(h * w, -1).index_select(0, sel).cpu().numpy().view(np.uint64).reshape(-1, 2, 3, n)
            ref_e = o.encrypt_radix(flat[idx], oc, seeds[i], ids=idx.astype(np.uint64))
            assert np.array_equal(got_e, ref_e), i
            got_f = filt[i].view(h * w, -1).index_select(0, sel).cpu().numpy().view(np.uint64).reshape(-1, 2, 2, n)
            for j, k in enumerate(idx):
                y, x = divmod(int(k), w)
                nb = np.array([_clamp(y + dy, h) * w + _clamp(x + dx, w) for dy in (-1, 0, 1) for dx in (-1, 0, 1)],
                              dtype=np.uint64)
                patch = o.encrypt_radix(flat[nb.astype(np.int64)], oc, seeds[i], ids=nb)
                out, _ = o.meanfilter3(patch, o.delta, 3, 3, 1)
                assert np.array_equal(got_f[j], out[4]), (i, int(k))
    finally:
        del enc, filt, d_px
        ctx.close()
        torch.cuda.empty_cache()
