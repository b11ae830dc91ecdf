"""Continuous-batching server (GPU): every request gives the same result alone and in a mixed
load (bit-exact ciphertexts and decoded values), equal to the single-request entry points;
admission respects the HBM budget; bad requests are refused at submit."""
import numpy as np
import pytest

from paper_2409_03568_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RINGS = [dict(log_n=10, prime_bits=[60, 40, 40], log2_scale=40, special_bits=61),
         dict(log_n=11, prime_bits=[60, 40, 40, 40], log2_scale=40, special_bits=61)]


@pytest.fixture(scope="module")
def ichee():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03568_gb300 import ichee as mod
    return mod


@pytest.fixture(scope="module")
def rings(ichee):
    ctxs, caches = [], []
    for i, r in enumerate(RINGS):
        ctx = ichee.Context(**r)
        ctx.keygen(900 + i, with_evk=True)
        ctxs.append(ctx)
        caches.append(ctx.build_cache(ichee.CACHE_FULL, 60 + i, pool_size=8))
    yield ctxs, caches
    for c in ctxs:
        c.close()


def make_request(ichee, ctxs, kind, ring, h, w, c, seed, keep):
    img = inputs.random_field_image(h, w, seed=seed, channels=c).reshape(-1).copy()
    two = None
    if kind == ichee.REQ_WATERMARK:
        two = inputs.binary_pattern(h, w, seed=seed + 7).reshape(-1).copy()
    elif kind == ichee.REQ_MATCH:
        two = inputs.noisy_copy(img, seed=seed + 9)
    n_res = 1 if kind == ichee.REQ_MATCH else h * w * c
    res = np.zeros(n_res, dtype=np.float64)
    ctx = ctxs[ring]
    L = ctx.L
    out_level = {ichee.REQ_ENCRYPT: L - 1, ichee.REQ_BRIGHTNESS: L - 1}.get(kind, L - 2)
    ct_out = ctx.empty_cts(1 if kind == ichee.REQ_MATCH else h * w * c, out_level)
    r = ichee.Request()
    r.kind, r.ring, r.h, r.w, r.c, r.seed = kind, ring, h, w, c, seed
    r.pixels = img.ctypes.data
    r.pixels2 = two.ctypes.data if two is not None else None
    r.arg = {ichee.REQ_BRIGHTNESS: 17.25, ichee.REQ_WATERMARK: 0.9}.get(kind, 0.0)
    r.result = res.ctypes.data
    r.ct_out = ct_out.data_ptr()
    keep.append((img, two, res, ct_out))
    return r, img, two, res, ct_out


def direct(ichee, ctx, cache, kind, h, w, c, seed, img, two, arg):
    """The same request through the single-request entry points."""
    a, ma = ctx.encrypt(torch.from_numpy(img).cuda(), h, w, c, seed, cache=cache)
    if kind == ichee.REQ_ENCRYPT:
        out, m = a, ma
    elif kind == ichee.REQ_MEANFILTER:
        out, m = ctx.eval(ichee.OP_MEANFILTER3, a, ma, out_level=ma.level - 1)
    elif kind == ichee.REQ_BRIGHTNESS:
        out, m = ctx.eval(ichee.OP_BRIGHTNESS, a, ma, args=(arg,))
    elif kind == ichee.REQ_WATERMARK:
        b, mb = ctx.encrypt(torch.from_numpy(two).cuda(), h, w, 1, seed + 1, cache=cache)
        out, m = ctx.eval(ichee.OP_BLEND, a, ma, b, mb, args=(arg,), out_level=ma.level - 1)
    else:
        b, mb = ctx.encrypt(torch.from_numpy(two).cuda(), h, w, c, seed + 1, cache=cache)
        out, m = ctx.eval(ichee.OP_SQDIFF_SUM, a, ma, b, mb, out_n_ct=1, out_level=ma.level - 1)
    return out, ctx.decrypt(out, m).cpu().numpy()


def test_same_alone_and_in_the_mix(ichee, rings):
    ctxs, caches = rings
    handles = [c.handle for c in ctxs]
    keep = []
    rng = np.random.default_rng(3)
    kinds = [ichee.REQ_ENCRYPT] * 4 + [ichee.REQ_MEANFILTER] * 2 + [ichee.REQ_BRIGHTNESS] * 2 + \
        [ichee.REQ_WATERMARK, ichee.REQ_MATCH]
    specs = []
    for i in range(30):
        kind = int(rng.choice(kinds))
        specs.append((kind, int(rng.integers(0, 2)), int(rng.integers(1, 9)), int(rng.integers(1, 9)),
                      int(rng.choice([1, 3])), 1000 + 17 * i))
    # alone: one server, one request at a time
    alone = []
    srv = ichee.ichee_server_create(handles, caches, 1 << 30)
    for (kind, ring, h, w, c, seed) in specs:
        r, img, two, res, ct = make_request(ichee, ctxs, kind, ring, h, w, c, seed, keep)
        t = ichee.ichee_server_submit(srv, r)
        d = ichee.ichee_server_wait(srv, t)
        assert d.round_size == 1
        alone.append((res.copy(), ct.clone()))
    ichee.ichee_server_destroy(srv)
    # the mix: all at once through a budget that holds only a few requests
    srv = ichee.ichee_server_create(handles, caches, 48 << 20, max_inflight=64)
    built = [make_request(ichee, ctxs, kind, ring, h, w, c, seed, keep) for (kind, ring, h, w, c, seed) in specs]
    ichee.ichee_server_hold(srv, True)        # the whole burst arrives before admission resumes
    subs = [(ichee.ichee_server_submit(srv, r), res, ct, img, two) for (r, img, two, res, ct) in built]
    assert ichee.ichee_server_stats_get(srv)["pending"] == 30
    ichee.ichee_server_hold(srv, False)
    rounds = []
    for (t, res, ct, img, two), (ares, act), spec in zip(subs, alone, specs):
        d = ichee.ichee_server_wait(srv, t)
        rounds.append(d.round_size)
        assert np.array_equal(res, ares), spec
        assert torch.equal(ct, act), spec
    st = ichee.ichee_server_stats_get(srv)
    assert st["served"] == 30 and st["pending"] == 0 and st["inflight"] == 0
    assert st["peak_arena_bytes"] <= 48 << 20
    assert max(rounds) > 1            # requests were batched together
    ichee.ichee_server_destroy(srv)
    # and the single-request entry points agree
    for (kind, ring, h, w, c, seed), (ares, act), (img, two, _, _) in zip(specs[:12], alone, keep[:12]):
        arg = {ichee.REQ_BRIGHTNESS: 17.25, ichee.REQ_WATERMARK: 0.9}.get(kind, 0.0)
        out, dec = direct(ichee, ctxs[ring], caches[ring], kind, h, w, c, seed, img, two, arg)
        assert torch.equal(out, act), (kind, ring)
        assert np.array_equal(dec, ares)
        if kind == ichee.REQ_ENCRYPT:
            assert np.max(np.abs(dec - img)) < 1e-3


def test_server_refuses_bad_requests(ichee, rings):
    ctxs, caches = rings
    srv = ichee.ichee_server_create([c.handle for c in ctxs], caches, 4 << 20)
    keep = []
    r, *_ = make_request(ichee, ctxs, ichee.REQ_MEANFILTER, 0, 64, 64, 3, 5, keep)
    with pytest.raises(ichee.IcheeError) as e:   # larger than the budget
        ichee.ichee_server_submit(srv, r)
    assert e.value.status == ichee.EINVAL
    r2, *_ = make_request(ichee, ctxs, ichee.REQ_ENCRYPT, 0, 2, 2, 1, 6, keep)
    r2.ring = 5
    with pytest.raises(ichee.IcheeError):
        ichee.ichee_server_submit(srv, r2)
    r3, *_ = make_request(ichee, ctxs, ichee.REQ_ENCRYPT, 1, 2, 2, 1, 7, keep)
    t = ichee.ichee_server_submit(srv, r3)
    ichee.ichee_server_wait(srv, t)
    with pytest.raises(ichee.IcheeError) as e:   # collected already
        ichee.ichee_server_wait(srv, t, timeout_ms=10)
    assert e.value.status == ichee.ETIMEOUT
    # a request held back by the host: bounded waits time out, then it completes normally
    r4, _, _, res4, _ = make_request(ichee, ctxs, ichee.REQ_ENCRYPT, 0, 3, 3, 1, 8, keep)
    ichee.ichee_server_hold(srv, True)
    t4 = ichee.ichee_server_submit(srv, r4)
    for _ in range(2):
        with pytest.raises(ichee.IcheeError) as e:
            ichee.ichee_server_wait(srv, t4, timeout_ms=20)
        assert e.value.status == ichee.ETIMEOUT
    assert ichee.ichee_server_stats_get(srv)["pending"] == 1
    ichee.ichee_server_hold(srv, False)
    d = ichee.ichee_server_wait(srv, t4)
    assert d.status == ichee.OK and d.t_done >= d.t_admit >= d.t_submit
    assert np.max(np.abs(res4 - keep[-1][0].astype(np.float64))) < 1e-3
    ichee.ichee_server_destroy(srv)


_ORACLES = {}


def oracle_ring(i):
    """The CPU oracle with the keys and full cache of test ring i (same seeds as the fixture)."""
    if i not in _ORACLES:
        from oracle import Oracle, Params
        r = RINGS[i]
        o = Oracle(Params(r["log_n"], r["prime_bits"], r["log2_scale"], r["special_bits"])).keygen(900 + i,
                                                                                                   with_evk=True)
        _ORACLES[i] = (o, o.full_cache(8, 60 + i))
    return _ORACLES[i]


def oracle_request(ichee, o, cache, kind, h, w, c, seed, img, two, arg):
    """The request as the oracle computes it: full-cache encryption with the pool (Sec. 3.2,
    3.3), then the operation of Sec. 4.4; returns (ciphertexts, exact scale)."""
    a = o.encrypt_lookup(img, cache, seed)
    if kind == ichee.REQ_ENCRYPT:
        return a, o.delta
    if kind == ichee.REQ_MEANFILTER:
        return o.meanfilter3(a, o.delta, h, w, c)
    if kind == ichee.REQ_BRIGHTNESS:
        return o.brightness(a, o.delta, arg)
    if kind == ichee.REQ_WATERMARK:
        return o.blend(a, o.encrypt_lookup(two, cache, seed + 1), o.delta, arg, c, 1)
    return o.match(a, o.encrypt_lookup(two, cache, seed + 1), o.delta)


@pytest.mark.parametrize("budget", [256 << 20, 6 << 20], ids=["whole", "tiled"])
def test_served_results_equal_the_oracle(ichee, rings, budget):
    """Every request kind on both rings, served together in one burst: each served ciphertext
    equals the oracle's word for word and each decoded value its exact decode (rtol 1e-9). With
    the small budget every request is served as row tiles (pixel ranges, mean-filter bands with
    halo rows, matching accumulated tile by tile)."""
    ctxs, caches = rings
    keep, built, specs = [], [], []
    for ring in range(2):
        for kind in range(5):
            h, w, c = 3 + kind, 4 + ring, 1 + 2 * ((kind + ring) % 2)
            seed = 3000 + 31 * (5 * ring + kind)
            specs.append((kind, ring, h, w, c, seed))
            built.append(make_request(ichee, ctxs, kind, ring, h, w, c, seed, keep))
    srv = ichee.ichee_server_create([x.handle for x in ctxs], caches, budget)
    ichee.ichee_server_hold(srv, True)
    tickets = [ichee.ichee_server_submit(srv, r) for (r, *_rest) in built]
    ichee.ichee_server_hold(srv, False)
    for t, (r, img, two, res, ct), (kind, ring, h, w, c, seed) in zip(tickets, built, specs):
        ichee.ichee_server_wait(srv, t)
        o, cache = oracle_ring(ring)
        want, scale = oracle_request(ichee, o, cache, kind, h, w, c, seed, img, two, r.arg)
        got = ct.cpu().numpy().view(np.uint64).reshape(want.shape)
        assert np.array_equal(got, want), (kind, ring)
        np.testing.assert_allclose(res, o.decrypt(want, scale), rtol=1e-9, atol=0)
    st = ichee.ichee_server_stats_get(srv)
    assert st["served"] == len(built) and st["arena_used_bytes"] == 0 and st["peak_arena_bytes"] <= budget
    ichee.ichee_server_destroy(srv)


@pytest.mark.timeout(300)
def test_failed_rounds_complete_and_server_stops(ichee, rings):
    """A round that fails to launch, and a round whose completion reports a device error (both
    injected on the host, no GPU fault), answer their requests with ECUDA; the server keeps
    serving and destroy returns."""
    ctxs, caches = rings
    keep = []
    srv = ichee.ichee_server_create([x.handle for x in ctxs], caches, 64 << 20)
    for launch_errors, query_errors in ((1, 0), (0, 1)):
        ichee.ichee_server_inject_failure(srv, launch_errors, query_errors)
        r, *_ = make_request(ichee, ctxs, ichee.REQ_ENCRYPT, 0, 2, 3, 1, 77, keep)
        t = ichee.ichee_server_submit(srv, r)
        with pytest.raises(ichee.IcheeError) as e:
            ichee.ichee_server_wait(srv, t, timeout_ms=60000)
        assert e.value.status == ichee.ECUDA
    r, img, _, res, _ = make_request(ichee, ctxs, ichee.REQ_ENCRYPT, 1, 2, 3, 1, 78, keep)
    d = ichee.ichee_server_wait(srv, ichee.ichee_server_submit(srv, r))
    assert d.status == ichee.OK and np.max(np.abs(res - img)) < 1e-3
    st = ichee.ichee_server_stats_get(srv)
    assert st["inflight"] == 0 and st["arena_used_bytes"] == 0
    ichee.ichee_server_destroy(srv)
