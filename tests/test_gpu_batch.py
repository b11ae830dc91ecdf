"""Ragged batches, CUDA-graph replay and the autotuner (GPU).

Every image of a batch must get exactly the ciphertexts (bit for bit) and decoded values the
single-image entry points give it -- those are checked against the CPU oracle elsewhere -- and
a sampled image of each batch is also checked directly against the oracle.
"""
import numpy as np
import pytest

from oracle import Oracle, Params
from paper_2409_03568_gb300 import inputs, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEY = 808


@pytest.fixture(scope="module")
def ichee():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03568_gb300 import ichee as mod
    return mod


def ragged_images(n, seed, lo=1, hi=20, channels=(1, 3)):
    rng = np.random.default_rng(seed)
    shapes = []
    imgs = []
    for i in range(n):
        h, w = int(rng.integers(lo, hi + 1)), int(rng.integers(lo, hi + 1))
        c = int(rng.choice(channels))
        shapes.append((h, w, c))
        imgs.append(inputs.random_field_image(h, w, seed=seed * 100 + i, channels=c).reshape(-1).copy())
    return shapes, imgs


def as_cts(t, n_ct, limbs, n):
    return t.cpu().numpy().view(np.uint64).reshape(n_ct, 2, limbs, n)


@pytest.fixture(scope="module")
def ctx8192(ichee):
    ctx = ichee.Context(**W.ctx_kwargs(W.ENC8192))
    ctx.keygen(KEY)
    yield ctx
    ctx.close()


@pytest.mark.parametrize("kind", ["fresh", "radix16", "full_pool", "freq_miss_fresh", "freq_miss_radix"])
def test_batch_encrypt_equals_single(ichee, ctx8192, kind):
    ctx = ctx8192
    shapes, imgs = ragged_images(7, seed={"fresh": 1, "radix16": 2, "full_pool": 3, "freq_miss_fresh": 4,
                                          "freq_miss_radix": 5}[kind], hi=9)
    shapes[0] = (1, 1, 1)
    imgs[0] = np.array([255], dtype=np.uint8)
    cache = None
    if kind == "radix16":
        cache = ctx.build_cache(ichee.CACHE_RADIX, 31, radix_base=16)
    elif kind == "full_pool":
        cache = ctx.build_cache(ichee.CACHE_FULL, 32, pool_size=8)
    elif kind.startswith("freq"):
        allpx = np.concatenate(imgs)
        cache = ctx.build_cache(ichee.CACHE_FREQ, 33, top_k=16, pool_size=4, scan=allpx.copy(),
                                miss_policy=0 if kind == "freq_miss_fresh" else 1, radix_base=16)
    seeds = [1000 + i for i in range(len(shapes))]
    d_px = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [ctx.empty_cts(h * w * c, ctx.L - 1) for (h, w, c) in shapes]
    metas = ichee.ichee_encrypt_batch(ctx.handle, cache, d_px, shapes, seeds, outs, ctx.stream())
    for i, (h, w, c) in enumerate(shapes):
        single, m = ctx.encrypt(d_px[i], h, w, c, seeds[i], cache=cache)
        assert torch.equal(outs[i], single), i
        assert (metas[i].h, metas[i].w, metas[i].c, metas[i].level) == (h, w, c, ctx.L - 1)
    # one image against the oracle directly
    if kind in ("fresh", "radix16"):
        o = Oracle(Params(13, [60, 40, 60], 40)).keygen(KEY)
        i = 3
        h, w, c = shapes[i]
        ref = o.encrypt_pixels(imgs[i], seeds[i]) if kind == "fresh" else \
            o.encrypt_radix(imgs[i], o.radix_cache(16, 31), seeds[i])
        assert np.array_equal(as_cts(outs[i], h * w * c, 3, ctx.n), ref)


def test_batch_ops_and_decrypt_equal_single(ichee, ctx8192):
    ctx = ctx8192
    shapes, imgs = ragged_images(6, seed=9, lo=2, hi=8)
    seeds = [2000 + i for i in range(len(shapes))]
    d_px = [torch.from_numpy(im).cuda() for im in imgs]
    enc = [ctx.empty_cts(h * w * c, 2) for (h, w, c) in shapes]
    metas = ichee.ichee_encrypt_batch(ctx.handle, None, d_px, shapes, seeds, enc, ctx.stream())
    # mean filter
    mf = [ctx.empty_cts(m.n_ct, 1) for m in metas]
    mmf = ichee.ichee_eval_batch(ctx.handle, ichee.OP_MEANFILTER3, enc, metas, outs=mf, stream=ctx.stream())
    for i, m in enumerate(metas):
        single, ms = ctx.eval(ichee.OP_MEANFILTER3, enc[i], m, out_level=1)
        assert torch.equal(mf[i], single), i
        assert mmf[i].scale == ms.scale and mmf[i].level == ms.level
    # brightness, one beta per image
    betas = [inputs.brightness_beta(50 + i) for i in range(len(shapes))]
    br = [ctx.empty_cts(m.n_ct, 2) for m in metas]
    ichee.ichee_eval_batch(ctx.handle, ichee.OP_BRIGHTNESS, enc, metas, args=betas, outs=br, stream=ctx.stream())
    for i, m in enumerate(metas):
        single, _ = ctx.eval(ichee.OP_BRIGHTNESS, enc[i], m, args=(betas[i],))
        assert torch.equal(br[i], single), i
    # the same in place on copies (every second image), the others out of place
    cp = [e.clone() for e in enc]
    outs = [cp[i] if i % 2 == 0 else ctx.empty_cts(m.n_ct, 2) for i, m in enumerate(metas)]
    ichee.ichee_eval_batch(ctx.handle, ichee.OP_BRIGHTNESS, cp, metas, args=betas, outs=outs, stream=ctx.stream())
    for i in range(len(metas)):
        assert torch.equal(outs[i], br[i]), i
    # blend with a one-channel pattern per image
    pats = [inputs.binary_pattern(h, w, seed=70 + i).reshape(-1).copy() for i, (h, w, c) in enumerate(shapes)]
    pshapes = [(h, w, 1) for (h, w, c) in shapes]
    penc = [ctx.empty_cts(h * w, 2) for (h, w, c) in shapes]
    pm = ichee.ichee_encrypt_batch(ctx.handle, None, [torch.from_numpy(p).cuda() for p in pats], pshapes,
                                   [3000 + i for i in range(len(shapes))], penc, ctx.stream())
    bl = [ctx.empty_cts(m.n_ct, 1) for m in metas]
    ichee.ichee_eval_batch(ctx.handle, ichee.OP_BLEND, enc, metas, penc, pm, args=(0.9,), outs=bl, stream=ctx.stream())
    for i, m in enumerate(metas):
        single, _ = ctx.eval(ichee.OP_BLEND, enc[i], m, penc[i], pm[i], args=(0.9,), out_level=1)
        assert torch.equal(bl[i], single), i
    # batched decryption of ciphertexts at level 2 and of the filtered ones at level 1
    dec = [torch.empty(m.n_ct, dtype=torch.float64, device="cuda") for m in metas]
    ichee.ichee_decrypt_batch(ctx.handle, enc, metas, dec, ctx.stream())
    for i, m in enumerate(metas):
        assert torch.equal(dec[i], ctx.decrypt(enc[i], m))
        assert float((dec[i].cpu() - torch.from_numpy(imgs[i]).double()).abs().max()) < 1e-3
    decf = [torch.empty(m.n_ct, dtype=torch.float64, device="cuda") for m in mmf]
    ichee.ichee_decrypt_batch(ctx.handle, mf, mmf, decf, ctx.stream())
    for i, m in enumerate(mmf):
        assert torch.equal(decf[i], ctx.decrypt(mf[i], m))


def test_batch_more_images_than_one_launch(ichee):
    ctx = ichee.Context(**W.ctx_kwargs(W.TOY))
    ctx.keygen(KEY)
    shapes, imgs = ragged_images(70, seed=11, lo=1, hi=4, channels=(1,))
    seeds = list(range(70))
    d_px = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [ctx.empty_cts(h * w * c, 1) for (h, w, c) in shapes]
    cache = ctx.build_cache(ichee.CACHE_RADIX, 5, radix_base=16)
    metas = ichee.ichee_encrypt_batch(ctx.handle, cache, d_px, shapes, seeds, outs, ctx.stream())
    for i in (0, 1, 63, 64, 69):
        h, w, c = shapes[i]
        single, _ = ctx.encrypt(d_px[i], h, w, c, seeds[i], cache=cache)
        assert torch.equal(outs[i], single), i
    mf = [ctx.empty_cts(m.n_ct, 0) for m in metas]
    mm = ichee.ichee_eval_batch(ctx.handle, ichee.OP_MEANFILTER3, outs, metas, outs=mf, stream=ctx.stream())
    for i in (0, 64, 69):
        single, _ = ctx.eval(ichee.OP_MEANFILTER3, outs[i], metas[i], out_level=0)
        assert torch.equal(mf[i], single)
    ctx.close()


def test_graph_replay_and_autotune(ichee, ctx8192):
    ctx = ctx8192
    shapes, imgs = ragged_images(5, seed=12, lo=3, hi=12, channels=(1,))
    seeds = [4000 + i for i in range(len(shapes))]
    cache = ctx.build_cache(ichee.CACHE_RADIX, 41, radix_base=16)
    d_px = [torch.from_numpy(im).cuda() for im in imgs]
    enc = [ctx.empty_cts(h * w * c, 2) for (h, w, c) in shapes]
    filt = [ctx.empty_cts(h * w * c, 1) for (h, w, c) in shapes]
    rep = ichee.ichee_autotune_batch(ctx.handle, cache, d_px, shapes, seeds, enc, filt, ctx.stream())
    kinds = {k for k, *_ in rep}
    assert kinds == {ichee.TUNE_RADIX, ichee.TUNE_FUSED, ichee.TUNE_MEANFILTER}
    assert ichee.ichee_tuned_shape(ctx.handle, ichee.TUNE_SCHEDULE)[0] in (0, 1)
    t, b = ichee.ichee_tuned_shape(ctx.handle, ichee.TUNE_MEANFILTER)
    best = min((e for e in rep if e[0] == ichee.TUNE_MEANFILTER), key=lambda e: e[3])
    assert (t, b) == (best[1], best[2])
    # reference results through single-image calls
    ref_enc, ref_filt = [], []
    for i, (h, w, c) in enumerate(shapes):
        e, m = ctx.encrypt(d_px[i], h, w, c, seeds[i], cache=cache)
        f, _ = ctx.eval(ichee.OP_MEANFILTER3, e, m, out_level=1)
        ref_enc.append(e)
        ref_filt.append(f)
    for i in range(len(shapes)):
        assert torch.equal(enc[i], ref_enc[i]) and torch.equal(filt[i], ref_filt[i])
    # capture encrypt + mean filter into one graph, replay twice on cleared buffers
    stream = torch.cuda.Stream()
    sp = ichee.ctypes.c_void_p(stream.cuda_stream)
    metas_holder = {}
    with torch.cuda.stream(stream):
        for t_ in enc + filt:
            t_.zero_()
        torch.cuda.synchronize()
        ichee.ichee_graph_begin(ctx.handle, sp)
        metas_holder["m"] = ichee.ichee_encrypt_batch(ctx.handle, cache, d_px, shapes, seeds, enc, sp)
        ichee.ichee_eval_batch(ctx.handle, ichee.OP_MEANFILTER3, enc, metas_holder["m"], outs=filt, stream=sp)
        graph = ichee.ichee_graph_end(ctx.handle, sp)
    torch.cuda.synchronize()
    for _ in range(2):
        for t_ in enc + filt:
            t_.zero_()
        torch.cuda.synchronize()
        ichee.ichee_graph_launch(graph, sp)
        stream.synchronize()
        for i in range(len(shapes)):
            assert torch.equal(enc[i], ref_enc[i]) and torch.equal(filt[i], ref_filt[i]), i
    ichee.ichee_graph_destroy(graph)


@pytest.mark.parametrize("base,randomize,threads", [(16, 1, 1024), (10, 1, 256), (16, 0, 128), (2, 1, 512)])
def test_fused_encrypt_meanfilter_equals_two_steps(ichee, ctx8192, base, randomize, threads):
    """Both schedules of ichee_encrypt_meanfilter_batch against single-image encryption + mean
    filter; the fused kernel with strips of 30, 6, 2 and 14 columns (widths up to 67: several
    strips, halo columns at both image borders), 1- and 3-channel images, 1-wide and 1-high
    images, radix bases 2, 10, 16 with and without randomness."""
    ctx = ctx8192
    shapes, imgs = ragged_images(6, seed=20 + base + randomize, lo=1, hi=11)
    shapes[1] = (1, 7, 3)
    imgs[1] = inputs.random_field_image(1, 7, seed=5, channels=3).reshape(-1).copy()
    shapes[2] = (6, 1, 1)
    imgs[2] = inputs.random_field_image(6, 1, seed=6).reshape(-1).copy()
    shapes[3] = (5, 67, 1)
    imgs[3] = inputs.random_field_image(5, 67, seed=7).reshape(-1).copy()
    shapes[4] = (3, 31, 3)
    imgs[4] = inputs.random_field_image(3, 31, seed=8, channels=3).reshape(-1).copy()
    seeds = [5000 + i for i in range(len(shapes))]
    cache = ctx.build_cache(ichee.CACHE_RADIX, 51 + base, radix_base=base, randomize=randomize)
    d_px = [torch.from_numpy(im).cuda() for im in imgs]
    ref = []
    for i, (h, w, c) in enumerate(shapes):
        e, m = ctx.encrypt(d_px[i], h, w, c, seeds[i], cache=cache)
        f, fm = ctx.eval(ichee.OP_MEANFILTER3, e, m, out_level=1)
        ref.append((e, m, f, fm))
    saved = ichee.ichee_tuned_shape(ctx.handle, ichee.TUNE_SCHEDULE)[0]
    ichee.ichee_set_tuned_shape(ctx.handle, ichee.TUNE_FUSED, threads, 2)
    try:
        for schedule in (1, 0):
            ichee.ichee_set_tuned_shape(ctx.handle, ichee.TUNE_SCHEDULE, schedule)
            enc = [ctx.empty_cts(h * w * c, 2) for (h, w, c) in shapes]
            filt = [ctx.empty_cts(h * w * c, 1) for (h, w, c) in shapes]
            mc, mf = ichee.ichee_encrypt_meanfilter_batch(ctx.handle, cache, d_px, shapes, seeds, enc, filt,
                                                          ctx.stream())
            for i, (e, m, f, fm) in enumerate(ref):
                assert torch.equal(enc[i], e), (schedule, i)
                assert torch.equal(filt[i], f), (schedule, i)
                assert mf[i].scale == fm.scale and mf[i].level == fm.level and mc[i].level == m.level
    finally:
        ichee.ichee_set_tuned_shape(ctx.handle, ichee.TUNE_SCHEDULE, saved)


def test_set_tuned_shape_checks(ichee, ctx8192):
    ctx = ctx8192
    for args in ((ichee.TUNE_RADIX, 1024, 2), (ichee.TUNE_FUSED, 2048, 1), (ichee.TUNE_RADIX, 256, 33),
                 (ichee.TUNE_SCHEDULE, 2, 0), (99, 256, 2)):
        with pytest.raises(ichee.IcheeError) as e:
            ichee.ichee_set_tuned_shape(ctx.handle, *args)
        assert e.value.status == ichee.EINVAL
    old = ichee.ichee_tuned_shape(ctx.handle, ichee.TUNE_RADIX)
    ichee.ichee_set_tuned_shape(ctx.handle, ichee.TUNE_RADIX, 256, 3)
    assert ichee.ichee_tuned_shape(ctx.handle, ichee.TUNE_RADIX) == (256, 3)
    ichee.ichee_set_tuned_shape(ctx.handle, ichee.TUNE_RADIX, *old)
    with pytest.raises(ichee.IcheeError):
        ichee.ichee_set_tuned_shape(ctx.handle, ichee.TUNE_RADIX, 64, 0)   # 32 / 64 only for decryption


def test_decrypt_shapes_give_identical_values(ichee, ctx8192):
    """Decryption (single-image and batched) at every block size it accepts gives the same
    doubles, bit for bit; the default is 256 threads."""
    ctx = ctx8192
    assert ichee.ichee_tuned_shape(ctx.handle, ichee.TUNE_DECRYPT) == (256, 0)
    shapes, imgs = ragged_images(3, seed=41, hi=12)
    d_px = [torch.from_numpy(im).cuda() for im in imgs]
    enc = [ctx.empty_cts(h * w * c, 2) for (h, w, c) in shapes]
    metas = ichee.ichee_encrypt_batch(ctx.handle, None, d_px, shapes, [9, 10, 11], enc, ctx.stream())
    ref = None
    try:
        for th in (32, 64, 128, 256, 512, 1024):
            ichee.ichee_set_tuned_shape(ctx.handle, ichee.TUNE_DECRYPT, th, 0 if th != 256 else 2)
            single = [ctx.decrypt(enc[i], metas[i]) for i in range(len(shapes))]
            outs = [torch.empty(m.n_ct, dtype=torch.float64, device="cuda") for m in metas]
            ichee.ichee_decrypt_batch(ctx.handle, enc, metas, outs, ctx.stream())
            torch.cuda.synchronize()
            for i in range(len(shapes)):
                assert torch.equal(single[i], outs[i]), (th, i)
            if ref is None:
                ref = single
                for i in range(len(shapes)):
                    assert np.max(np.abs(single[i].cpu().numpy() - imgs[i])) < 1e-3
            for i in range(len(shapes)):
                assert torch.equal(single[i], ref[i]), (th, i)
    finally:
        ichee.ichee_set_tuned_shape(ctx.handle, ichee.TUNE_DECRYPT, 256, 0)


def test_batch_errors(ichee, ctx8192):
    ctx = ctx8192
    px = torch.zeros(4, dtype=torch.uint8, device="cuda")
    out = ctx.empty_cts(4, 2)
    with pytest.raises(ichee.IcheeError) as e:
        ichee.ichee_encrypt_batch(ctx.handle, None, [px], [(0, 2, 2)], [1], [out], ctx.stream())
    assert e.value.status == ichee.EINVAL
    metas = ichee.ichee_encrypt_batch(ctx.handle, None, [px], [(2, 2, 1)], [1], [out], ctx.stream())
    with pytest.raises(ichee.IcheeError) as e:
        ichee.ichee_eval_batch(ctx.handle, ichee.OP_SQDIFF_SUM, [out], metas, [out], metas, outs=[out],
                               stream=ctx.stream())
    assert e.value.status in (ichee.EINVAL, ichee.EUNSUPPORTED)
    with pytest.raises(ichee.IcheeError) as e:
        ichee.ichee_eval_batch(ctx.handle, ichee.OP_BRIGHTNESS, [out], metas, args=(1.0, 2.0), outs=[ctx.empty_cts(4, 2)],
                               stream=ctx.stream())
    assert e.value.status == ichee.EINVAL


def test_batched_mean_filter_five_limbs(ichee):
    """The N = 16384 ring with five limbs (half of the serving requests): batched radix
    encryption and batched mean filter against the oracle, and the fused encrypt + mean-filter
    kernel (asked for 1024 threads, run at its five-limb bound of 512) against both."""
    wl = W.RING16384
    ctx = ichee.Context(**W.ctx_kwargs(wl))
    ctx.keygen(KEY)
    o = Oracle(Params(wl["log_n"], wl["prime_bits"], wl["log2_scale"])).keygen(KEY)
    n, L = ctx.n, ctx.L
    shapes = [(3, 5, 1), (2, 4, 3), (1, 1, 1)]
    imgs = [inputs.random_field_image(h, w, seed=90 + i, channels=c).reshape(-1).copy()
            for i, (h, w, c) in enumerate(shapes)]
    seeds = [700 + i for i in range(len(shapes))]
    cache = ctx.build_cache(ichee.CACHE_RADIX, 71, radix_base=16)
    ocache = o.radix_cache(16, 71)
    d_px = [torch.from_numpy(im).cuda() for im in imgs]
    enc = [ctx.empty_cts(h * w * c, L - 1) for (h, w, c) in shapes]
    metas = ichee.ichee_encrypt_batch(ctx.handle, cache, d_px, shapes, seeds, enc, ctx.stream())
    filt = [ctx.empty_cts(h * w * c, L - 2) for (h, w, c) in shapes]
    ichee.ichee_eval_batch(ctx.handle, ichee.OP_MEANFILTER3, enc, metas, outs=filt, stream=ctx.stream())
    torch.cuda.synchronize()
    for i, (h, w, c) in enumerate(shapes):
        ref = o.encrypt_radix(imgs[i], ocache, seeds[i])
        assert np.array_equal(as_cts(enc[i], h * w * c, L, n), ref), i
        rf, _ = o.meanfilter3(ref, o.delta, h, w, c)
        assert np.array_equal(as_cts(filt[i], h * w * c, L - 1, n), rf), i
    saved = ichee.ichee_tuned_shape(ctx.handle, ichee.TUNE_SCHEDULE)[0]
    ichee.ichee_set_tuned_shape(ctx.handle, ichee.TUNE_FUSED, 1024, 1)
    ichee.ichee_set_tuned_shape(ctx.handle, ichee.TUNE_SCHEDULE, 1)
    try:
        enc2 = [ctx.empty_cts(h * w * c, L - 1) for (h, w, c) in shapes]
        filt2 = [ctx.empty_cts(h * w * c, L - 2) for (h, w, c) in shapes]
        ichee.ichee_encrypt_meanfilter_batch(ctx.handle, cache, d_px, shapes, seeds, enc2, filt2, ctx.stream())
        torch.cuda.synchronize()
        for i in range(len(shapes)):
            assert torch.equal(enc2[i], enc[i]) and torch.equal(filt2[i], filt[i]), i
    finally:
        ichee.ichee_set_tuned_shape(ctx.handle, ichee.TUNE_SCHEDULE, saved)
    ctx.status()
    ctx.close()
