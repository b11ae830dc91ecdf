"""Pins of the CPU oracle to things other than itself (no GPU needed).

Each test ties one oracle function to a published value, a closed form, an exact algebraic
identity, a library routine or brute force, so that a dropped term, a wrong sign, index or
operand in the oracle fails at least one of them.
"""
import ctypes
import math
import random
from fractions import Fraction

import numpy as np
import pytest

from conftest import read_golden
from oracle import Oracle, Params, llround, mse, psnr
from oracle.ckks import _p, lib, u32p, u64p, i8p
from paper_2409_03568_gb300 import inputs

TOY = Params(10, [30, 30], 25)                      # N=1024, 2 x 30-bit, Delta=2^25
SMALL4 = Params(10, [60, 40, 40, 40], 40, 61)       # config-3 chain at N=1024 (fast)
CFG2 = Params(13, [60, 40, 60], 40)                 # N=8192, 60/40/60, Delta=2^40


@pytest.fixture(scope="module")
def toy():
    return Oracle(TOY).keygen(11)


@pytest.fixture(scope="module")
def small4():
    return Oracle(SMALL4).keygen(21, with_evk=True)


def _fresh_bound(n, bound=19):
    # Dec(Enc(m)) - m = v*e + e0 + e1*s with v, s ternary and |e|,|e0|,|e1| <= bound
    return (2 * n + 1) * bound


def _centered_poly(o, ct):
    return np.array(o.decrypt_poly(ct), dtype=object)


# ----------------------------------------------------------------------------- primes
def test_prime_chain_properties():
    sympy = pytest.importorskip("sympy")
    for params in (TOY, SMALL4, CFG2, Params(14, [60, 40, 40, 40, 40], 40, 61)):
        o = Oracle(params)
        two_n = 2 * params.n
        qs = [int(x) for x in o.q] + ([o.P] if o.P else [])
        bits = params.prime_bits + ([params.special_bits] if o.P else [])
        assert len(set(qs)) == len(qs)
        for q, b in zip(qs, bits):
            assert sympy.isprime(q)
            assert q % two_n == 1
            assert 2 ** (b - 1) < q < 2 ** b
        # "largest downward, skipping used": every candidate above q of the same size
        # congruent to 1 mod 2N is composite or taken earlier in the chain
        for idx, (q, b) in enumerate(zip(qs, bits)):
            c = q + two_n
            while c < 2 ** b:
                assert (not sympy.isprime(c)) or c in qs[:idx]
                c += two_n


def test_miller_rabin_matches_sympy():
    sympy = pytest.importorskip("sympy")
    rng = random.Random(5)
    L = lib()
    L.orc_is_prime.argtypes = [ctypes.c_uint64]
    for _ in range(3000):
        n = rng.getrandbits(rng.choice([8, 20, 40, 61, 64]))
        assert bool(L.orc_is_prime(n)) == sympy.isprime(n)
    # strong pseudoprimes to several small bases
    for n in (3215031751, 3825123056546413051, 318665857834031151167461):
        if n < 2 ** 64:
            assert not L.orc_is_prime(n)


# ---------------------------------------------------------------------------- philox
def test_philox_known_answers():
    for row in read_golden("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        ctr = np.array(v[0:4], dtype=np.uint32)
        key = np.array(v[4:6], dtype=np.uint32)
        out = np.zeros(4, dtype=np.uint32)
        lib().orc_philox4x32_10(_p(ctr, u32p), _p(key, u32p), _p(out, u32p))
        assert [int(x) for x in out] == v[6:10]


# --------------------------------------------------------------------------- samplers
def _exact_folded_cdf(sigma, bound):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    w = [mpmath.mpf(1)] + [2 * mpmath.e ** (-mpmath.mpf(k * k) / (2 * mpmath.mpf(sigma) ** 2))
                           for k in range(1, bound + 1)]
    z = sum(w)
    cdf, acc = [], mpmath.mpf(0)
    for k in range(bound + 1):
        acc += w[k]
        cdf.append(acc / z)
    return cdf, [float(x / z) for x in w]


def test_cdt_table_against_high_precision():
    o = Oracle(TOY)
    cdf, _ = _exact_folded_cdf(3.2, 19)
    T = [int(x) for x in o.T]
    assert T[19] == 2 ** 63
    assert all(T[k] < T[k + 1] for k in range(18))
    for k in range(19):
        exact = int(cdf[k] * 2 ** 63)
        assert abs(T[k] - exact) <= 2, k


def test_gaussian_sampler_distribution():
    o = Oracle(TOY)
    n = 1 << 17
    out = np.zeros(n, dtype=np.int8)
    lib().orc_sample_gauss(ctypes.c_uint64(99), ctypes.c_uint32(1), ctypes.c_uint64(3), ctypes.c_uint32(n),
                           _p(o.T, u64p), ctypes.c_uint32(19), _p(out, i8p))
    x = out.astype(np.int64)
    assert np.abs(x).max() <= 19
    # discrete Gaussian with sigma 3.2: mean 0, variance ~ sigma^2
    assert abs(x.mean()) < 0.05
    assert abs(x.var() - 3.2 ** 2) < 0.15
    # chi-square on |x| against the folded probabilities
    _, probs = _exact_folded_cdf(3.2, 19)
    counts = np.bincount(np.abs(x), minlength=20)
    exp = np.array(probs) * n
    keep = exp > 20
    chi2 = float(((counts[keep] - exp[keep]) ** 2 / exp[keep]).sum())
    assert chi2 < 45, chi2          # dof ~ 13; 45 is far in the tail
    # sign is symmetric
    assert abs(int((x > 0).sum()) - int((x < 0).sum())) < 4 * math.sqrt(n)


def test_ternary_sampler_distribution():
    n = 1 << 17
    out = np.zeros(n, dtype=np.int8)
    lib().orc_sample_ternary(ctypes.c_uint64(7), ctypes.c_uint32(0), ctypes.c_uint64(12), ctypes.c_uint32(n),
                             _p(out, i8p))
    counts = np.array([(out == v).sum() for v in (-1, 0, 1)])
    assert counts.sum() == n
    exp = n / 3
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 14


def test_uniform_sampler_range_and_spread():
    q = (1 << 60) - 93 * (1 << 14) + 1     # any modulus works for this check
    n = 1 << 16
    out = np.zeros(n, dtype=np.uint64)
    lib().orc_sample_uniform(ctypes.c_uint64(5), ctypes.c_uint32(16), ctypes.c_uint64(0), ctypes.c_uint32(n),
                             ctypes.c_uint64(q), _p(out, u64p))
    vals = [int(v) for v in out]
    assert max(vals) < q
    buckets = np.bincount([v * 16 // q for v in vals], minlength=16)
    exp = n / 16
    assert float(((buckets - exp) ** 2 / exp).sum()) < 40


def test_samples_depend_on_every_counter_field():
    base = np.zeros(64, dtype=np.int8)
    lib().orc_sample_ternary(ctypes.c_uint64(1), ctypes.c_uint32(0), ctypes.c_uint64(0), ctypes.c_uint32(64),
                             _p(base, i8p))
    for seed, stream, cid in ((2, 0, 0), (1, 1, 0), (1, 0, 1), (1, 0, 1 << 32), (1 << 32, 0, 0)):
        other = np.zeros(64, dtype=np.int8)
        lib().orc_sample_ternary(ctypes.c_uint64(seed), ctypes.c_uint32(stream), ctypes.c_uint64(cid),
                                 ctypes.c_uint32(64), _p(other, i8p))
        assert not np.array_equal(base, other)


# ---------------------------------------------------------------- negacyclic products
def _bigint_schoolbook(a, b, n, mod):
    c = [0] * n
    for i in range(n):
        for j in range(n):
            if i + j < n:
                c[i + j] += a[i] * b[j]
            else:
                c[i + j - n] -= a[i] * b[j]
    return [x % mod for x in c]


@pytest.mark.parametrize("params", [TOY, SMALL4, CFG2])
@pytest.mark.parametrize("n", [4, 16, 64])
def test_polymul_matches_schoolbook(params, n):
    o = Oracle(params)
    rng = np.random.default_rng(n)
    for q in [int(x) for x in o.q] + ([o.P] if o.P else []):
        a = np.array([int(x) % q for x in rng.integers(0, 2 ** 63, n, dtype=np.uint64)], dtype=np.uint64)
        b = np.array([int(x) % q for x in rng.integers(0, 2 ** 63, n, dtype=np.uint64)], dtype=np.uint64)
        c1 = np.zeros(n, dtype=np.uint64)
        c2 = np.zeros(n, dtype=np.uint64)
        lib().orc_polymul(ctypes.c_uint32(n), ctypes.c_uint64(q), _p(a, u64p), _p(b, u64p), _p(c1, u64p))
        lib().orc_polymul_schoolbook(ctypes.c_uint32(n), ctypes.c_uint64(q), _p(a, u64p), _p(b, u64p),
                                     _p(c2, u64p))
        ref = _bigint_schoolbook([int(x) for x in a], [int(x) for x in b], n, q)
        assert [int(x) for x in c1] == ref
        assert [int(x) for x in c2] == ref


def test_polymul_full_size_ternary_by_shifts():
    """At N=1024 the product with a ternary polynomial is a signed sum of negacyclic shifts."""
    o = Oracle(TOY)
    n = o.n
    q = int(o.q[0])
    rng = np.random.default_rng(3)
    v = rng.integers(-1, 2, n)
    b = rng.integers(0, q, n, dtype=np.uint64)
    acc = np.zeros(n, dtype=object)
    bo = np.array([int(x) for x in b], dtype=object)
    for j in np.nonzero(v)[0]:
        shifted = np.concatenate([-bo[n - j:], bo[:n - j]])      # x^j * b mod X^N + 1
        acc = acc + int(v[j]) * shifted
    ref = [int(x) % q for x in acc]
    vr = np.array([int(x) % q for x in v], dtype=np.uint64)
    c = np.zeros(n, dtype=np.uint64)
    lib().orc_polymul(ctypes.c_uint32(n), ctypes.c_uint64(q), _p(vr, u64p), _p(b, u64p), _p(c, u64p))
    assert [int(x) for x in c] == ref


# ------------------------------------------------------------------- keys and encrypt
def test_public_key_is_rlwe_sample(toy):
    """pk0 + pk1*s = e with |e| <= bound (sign of a*s, Sec. 2.2.2 with the library convention pk0 = -a*s + e)."""
    o = toy
    zero_ct = np.ascontiguousarray(o.pk)        # (pk0, pk1) decrypts like a ciphertext
    e = _centered_poly(o, zero_ct)
    assert max(abs(int(x)) for x in e) <= 19
    assert any(int(x) != 0 for x in e)


def test_encrypt_decrypt_noise_bound_toy(toy):
    o = toy
    pix = inputs.uniform_image(8, 8, seed=1)
    ct = o.encrypt_pixels(pix, seed=123)
    bound = _fresh_bound(o.n)
    for k in (0, 17, 63):
        poly = _centered_poly(o, ct[k])
        m = int(pix.reshape(-1)[k]) * o.delta
        assert abs(poly[0] - m) <= bound
        assert max(abs(int(x)) for x in poly[1:]) <= bound
    dec = o.decrypt(ct, o.delta)
    assert np.max(np.abs(dec - pix.reshape(-1))) < bound / o.delta


def test_encrypt_decrypt_cfg2_within_1e3():
    o = Oracle(CFG2).keygen(2)
    pix = np.array([0, 1, 127, 128, 254, 255], dtype=np.uint8)
    ct = o.encrypt_pixels(pix, seed=9)
    dec = o.decrypt(ct, o.delta)
    assert np.max(np.abs(dec - pix)) < 1e-3
    poly = _centered_poly(o, ct[3])
    assert abs(poly[0] - 128 * o.delta) <= _fresh_bound(o.n)


def test_rns_encryption_equals_bigint_encryption():
    """At N=16 the RNS ciphertext equals the same encryption done over Z_Q with big integers
    and schoolbook products (no NTT, no CRT), reduced into each limb."""
    params = Params(4, [30, 40, 50], 20)
    o = Oracle(params).keygen(77)
    n = o.n
    qs = [int(x) for x in o.q]
    Q = math.prod(qs)
    # rebuild pk over Z_Q from the same samples
    T = o.T
    s = [int(x) for x in o.s]
    e = np.zeros(n, dtype=np.int8)
    lib().orc_sample_gauss(ctypes.c_uint64(77), ctypes.c_uint32(9), ctypes.c_uint64(0), ctypes.c_uint32(n),
                           _p(T, u64p), ctypes.c_uint32(19), _p(e, i8p))
    a_limbs = []
    for l, q in enumerate(qs):
        a = np.zeros(n, dtype=np.uint64)
        lib().orc_sample_uniform(ctypes.c_uint64(77), ctypes.c_uint32(16 + l), ctypes.c_uint64(0),
                                 ctypes.c_uint32(n), ctypes.c_uint64(q), _p(a, u64p))
        a_limbs.append([int(x) for x in a])
    a_big = [o.crt([a_limbs[l][i] for l in range(3)]) % Q for i in range(n)]
    as_big = _bigint_schoolbook(a_big, s, n, Q)
    pk0 = [(-as_big[i] + int(e[i])) % Q for i in range(n)]
    pk1 = a_big
    for l, q in enumerate(qs):
        assert [x % q for x in pk0] == [int(x) for x in o.pk[0, l]]
        assert [x % q for x in pk1] == [int(x) for x in o.pk[1, l]]
    # encryption of one message with ct id 5
    v = np.zeros(n, dtype=np.int8)
    e0 = np.zeros(n, dtype=np.int8)
    e1 = np.zeros(n, dtype=np.int8)
    for arr, stream, fn in ((v, 0, "t"), (e0, 1, "g"), (e1, 2, "g")):
        if fn == "t":
            lib().orc_sample_ternary(ctypes.c_uint64(5), ctypes.c_uint32(stream), ctypes.c_uint64(5),
                                     ctypes.c_uint32(n), _p(arr, i8p))
        else:
            lib().orc_sample_gauss(ctypes.c_uint64(5), ctypes.c_uint32(stream), ctypes.c_uint64(5),
                                   ctypes.c_uint32(n), _p(T, u64p), ctypes.c_uint32(19), _p(arr, i8p))
    vi = [int(x) for x in v]
    c0 = _bigint_schoolbook(vi, pk0, n, Q)
    c1 = _bigint_schoolbook(vi, pk1, n, Q)
    msg = 200 * o.delta
    c0 = [(c0[i] + int(e0[i]) + (msg if i == 0 else 0)) % Q for i in range(n)]
    c1 = [(c1[i] + int(e1[i])) % Q for i in range(n)]
    ct = o.encrypt_msgs(np.array([msg]), np.array([5], dtype=np.uint64), seed=5)[0]
    for l, q in enumerate(qs):
        assert [x % q for x in c0] == [int(x) for x in ct[0, l]]
        assert [x % q for x in c1] == [int(x) for x in ct[1, l]]


def test_decrypt_coef0_matches_full_product(toy):
    o = toy
    ct = o.encrypt_pixels(np.array([77], dtype=np.uint8), seed=4)
    poly = _centered_poly(o, ct[0])
    res = o.decrypt_residues(ct)[0]
    assert o.crt(res) == poly[0]


def test_crt_roundtrip():
    o = Oracle(SMALL4)
    qs = [int(x) for x in o.q]
    Q = math.prod(qs)
    rng = random.Random(8)
    for _ in range(200):
        x = rng.randrange(-(Q // 2) + 1, Q // 2)
        assert o.crt([x % q for q in qs]) == x


# ------------------------------------------------------------------ homomorphic ops
def test_add_sub_mul_int_add_int_are_exact_on_decryptions(toy):
    """Dec is linear mod Q, so these identities hold exactly on the centered integers."""
    o = toy
    a = o.encrypt_pixels(np.array([10, 200], dtype=np.uint8), seed=1)
    b = o.encrypt_pixels(np.array([33, 5], dtype=np.uint8), seed=2)
    da = [o.crt(r) for r in o.decrypt_residues(a)]
    db = [o.crt(r) for r in o.decrypt_residues(b)]
    s = [o.crt(r) for r in o.decrypt_residues(o.add(a, b))]
    d = [o.crt(r) for r in o.decrypt_residues(o.sub(a, b))]
    m = [o.crt(r) for r in o.decrypt_residues(o.mul_int(a, -7))]
    p = [o.crt(r) for r in o.decrypt_residues(o.add_int(a, -123456))]
    for k in range(2):
        assert s[k] == da[k] + db[k]
        assert d[k] == da[k] - db[k]
        assert m[k] == -7 * da[k]
        assert p[k] == da[k] - 123456


def test_rescale_divides_by_last_prime(small4):
    o = small4
    ct = o.encrypt_pixels(np.array([200, 3], dtype=np.uint8), seed=6)
    big = o.mul_int(ct, 1 << 39)
    before = [o.crt(r) for r in o.decrypt_residues(big)]
    after = o.rescale(big)
    qt = int(o.q[3])
    got = [o.crt(r) for r in o.decrypt_residues(after)]
    for x, y in zip(before, got):
        # rounding error of c1*s: at most (1 + ||s||_1) / 2
        assert abs(Fraction(x, qt) - y) <= Fraction(1 + o.n, 2) + 1


def test_relin_matches_three_term_decryption(small4):
    o = small4
    a = o.encrypt_pixels(np.array([100], dtype=np.uint8), seed=31)
    b = o.encrypt_pixels(np.array([37], dtype=np.uint8), seed=32)
    t = o.sqdiff_sum_raw(a, b)               # (d0^2, 2 d0 d1, d1^2)
    # three-term decryption t0 + t1 s + t2 s^2, coefficient 0, via the pinned products
    n = o.n
    vals = []
    for l in range(o.L):
        q = int(o.q[l])
        sr = np.array([int(x) % q for x in o.s], dtype=np.uint64)
        s2 = np.zeros(n, dtype=np.uint64)
        p1 = np.zeros(n, dtype=np.uint64)
        p2 = np.zeros(n, dtype=np.uint64)
        lib().orc_polymul(ctypes.c_uint32(n), ctypes.c_uint64(q), _p(sr, u64p), _p(sr, u64p), _p(s2, u64p))
        t1 = np.ascontiguousarray(t[1, l])
        t2 = np.ascontiguousarray(t[2, l])
        lib().orc_polymul(ctypes.c_uint32(n), ctypes.c_uint64(q), _p(t1, u64p), _p(sr, u64p), _p(p1, u64p))
        lib().orc_polymul(ctypes.c_uint32(n), ctypes.c_uint64(q), _p(t2, u64p), _p(s2, u64p), _p(p2, u64p))
        vals.append((int(t[0, l, 0]) + int(p1[0]) + int(p2[0])) % q)
    three_term = o.crt(vals)
    r = o.relin(t)
    two_term = o.crt(o.decrypt_residues(r[None])[0])
    # key-switching noise: sum_j |[d2]_j| * |e_j| * N / P + rounding, far below 2^40
    assert abs(two_term - three_term) < 2 ** 30
    # and the message is the squared difference at scale Delta^2
    assert abs(Fraction(two_term, o.delta ** 2) - 63 ** 2) < Fraction(1, 1000)


def test_relin_depends_on_evk_sign(small4):
    """Flipping the sign of the evk's s^2 term must break decryption (guards the sign of the s^2 term in the key)."""
    o = small4
    a = o.encrypt_pixels(np.array([9], dtype=np.uint8), seed=41)
    b = o.encrypt_pixels(np.array([2], dtype=np.uint8), seed=42)
    t = o.sqdiff_sum_raw(a, b)
    good = o.relin(t)
    bad_t = t.copy()
    for l in range(o.L):
        q = int(o.q[l])
        bad_t[2, l] = np.array([(q - int(x)) % q for x in t[2, l]], dtype=np.uint64)
    bad = o.relin(bad_t)
    g = float(Fraction(o.crt(o.decrypt_residues(good[None])[0]), o.delta ** 2))
    bb = float(Fraction(o.crt(o.decrypt_residues(bad[None])[0]), o.delta ** 2))
    assert abs(g - 49) < 1e-3
    assert abs(bb - 49) > 1.0


def test_sqdiff_image_matches_plaintext_squares(small4):
    """Per-pixel squared difference: every decrypted output equals (p_a - p_b)^2 (FP64)."""
    o = small4
    pa = np.array([0, 255, 100, 37, 200, 1], dtype=np.uint8)
    pb = np.array([255, 0, 37, 100, 200, 2], dtype=np.uint8)
    ca = o.encrypt_pixels(pa, seed=51)
    cb = o.encrypt_pixels(pb, seed=52)
    out, sc = o.sqdiff_image(ca, cb, o.delta)
    assert out.shape == (6, 2, o.L - 1, o.n)
    assert sc == Fraction(o.delta) ** 2 / int(o.q[o.L - 1])
    ref = (pa.astype(np.float64) - pb) ** 2
    np.testing.assert_allclose(o.decrypt(out, sc), ref, atol=1e-3, rtol=0)


def test_sqdiff_image_one_pixel_equals_match(small4):
    """For a one-pixel image the per-pixel and the summed forms are the same computation."""
    o = small4
    ca = o.encrypt_pixels(np.array([91], dtype=np.uint8), seed=53)
    cb = o.encrypt_pixels(np.array([12], dtype=np.uint8), seed=54)
    per_px, s1 = o.sqdiff_image(ca, cb, o.delta)
    summed, s2 = o.match(ca, cb, o.delta)
    assert s1 == s2 and np.array_equal(per_px, summed)


# ------------------------------------------------------------------- caches (Sec. 3)
def _radix_cache_small(base):
    o = Oracle(Params(6, [40, 40], 20)).keygen(3)
    return o, o.radix_cache(base, seed=17)


def test_radix_worked_example():
    (r, i, added, subtracted, times), = [[int(x) for x in row] for row in read_golden("radix_worked_example.txt")]
    o, cache = _radix_cache_small(r)
    assert r ** i == added and r ** (i - 1) == subtracted and times == r
    n, lim = o.n, o.L
    for p in (0, 5, 77, 255):
        plain = np.zeros((1, 2, lim, n), dtype=np.uint64)
        rand = np.zeros((1, 2, lim, n), dtype=np.uint64)
        args = (ctypes.c_uint32(n), ctypes.c_uint32(lim), _p(o.q, u64p), _p(cache["cts"], u64p),
                ctypes.c_uint32(cache["n_pow"]), ctypes.c_uint32(r), ctypes.c_uint32(p))
        lib().orc_radix_encrypt_sequential(*args, ctypes.c_int(0), ctypes.c_uint32(0), _p(plain, u64p))
        lib().orc_radix_encrypt_sequential(*args, ctypes.c_int(1), ctypes.c_uint32(1 << i), _p(rand, u64p))
        # the randomised ciphertext differs by exactly Enc(32) - 2 Enc(16)
        c32 = cache["cts"][i:i + 1]
        c16 = cache["cts"][i - 1:i]
        expect = o.sub(o.sub(o.add(plain, c32), c16), c16)
        assert np.array_equal(expect, rand)
        assert not np.array_equal(plain, rand)
        assert abs(o.decrypt(rand, o.delta)[0] - p) < 1e-3
        assert abs(o.decrypt(plain, o.delta)[0] - p) < 1e-3


@pytest.mark.parametrize("base", [2, 10, 16])
def test_radix_sequential_equals_signed_digits(base):
    o, cache = _radix_cache_small(base)
    n, lim = o.n, o.L
    rng = random.Random(base)
    for p in [0, 1, base - 1, base, 255, 128] + [rng.randrange(256) for _ in range(6)]:
        for bits in (0, 0xFFFFFFFF, rng.getrandbits(32)):
            a = np.zeros((2, lim, n), dtype=np.uint64)
            b = np.zeros((2, lim, n), dtype=np.uint64)
            args = (ctypes.c_uint32(n), ctypes.c_uint32(lim), _p(o.q, u64p), _p(cache["cts"], u64p),
                    ctypes.c_uint32(cache["n_pow"]), ctypes.c_uint32(base), ctypes.c_uint32(p),
                    ctypes.c_int(1), ctypes.c_uint32(bits))
            lib().orc_radix_encrypt_sequential(*args, _p(a, u64p))
            lib().orc_radix_encrypt_signed(*args, _p(b, u64p))
            assert np.array_equal(a, b)
            assert abs(o.decrypt(a[None], o.delta)[0] - p) < 1e-3


def test_radix_powers_count():
    assert [Oracle.radix_powers(b) for b in (2, 10, 16)] == [8, 3, 2]


def test_top_values_brute_force():
    rng = np.random.default_rng(0)
    pix = rng.integers(0, 40, 1000).astype(np.uint8)
    top = Oracle.top_values(pix, 8)
    counts = {v: int((pix == v).sum()) for v in range(256)}
    brute = sorted([v for v in counts if counts[v] > 0], key=lambda v: (-counts[v], v))[:8]
    assert top == brute
    assert Oracle.top_values(np.array([3, 3, 1], dtype=np.uint8), 5) == [3, 1]


def test_cached_encryptions_decrypt_like_fresh(toy):
    """Sec. 3: every cache kind and the pool leave the decrypted pixel unchanged."""
    o = toy
    pix = inputs.random_field_image(8, 8, seed=1).reshape(-1)
    fresh = o.decrypt(o.encrypt_pixels(pix, seed=5), o.delta)
    r16 = o.radix_cache(16, seed=8)
    r10 = o.radix_cache(10, seed=8)
    freq = o.freq_cache(pix, 8, 16, seed=8, radix_base=16)
    full = o.full_cache(4, seed=8)
    outs = [o.encrypt_radix(pix, r16, seed=5), o.encrypt_radix(pix, r10, seed=5),
            o.encrypt_radix(pix, r16, seed=5, randomize=False),
            o.encrypt_lookup(pix, freq, seed=5), o.encrypt_lookup(pix, freq, seed=5, miss_policy=1),
            o.encrypt_lookup(pix, full, seed=5)]
    # noise: up to (digits + randomness) fresh noises for radix; two for the pool
    for ct in outs:
        dec = o.decrypt(ct, o.delta)
        assert np.max(np.abs(dec - pix)) < 64 * _fresh_bound(o.n) / o.delta
        assert np.max(np.abs(dec - fresh)) < 64 * _fresh_bound(o.n) / o.delta
    # pool randomness: equal pixels with different pool picks give different ciphertexts
    ct = outs[5]
    same = [k for k in range(len(pix)) if pix[k] == pix[0]]
    picks = {k: int(lib().orc_pool_index(ctypes.c_uint64(5), ctypes.c_uint64(k), ctypes.c_uint32(4)))
             for k in same}
    for k in same[1:]:
        if picks[k] != picks[same[0]]:
            assert not np.array_equal(ct[k], ct[same[0]])


def test_pool_identity_exact(toy):
    """Enc(p) (+) Enc(0) decrypts to Dec(Enc(p)) + Dec(Enc(0)) exactly (Sec. 3.3)."""
    o = toy
    cp = o.encrypt_pixels(np.array([99], dtype=np.uint8), seed=3)
    z = o.pool(2, seed=4)
    for m in range(2):
        s = o.add(cp, z[m:m + 1])
        x = o.crt(o.decrypt_residues(s)[0])
        assert x == o.crt(o.decrypt_residues(cp)[0]) + o.crt(o.decrypt_residues(z[m:m + 1])[0])
        assert abs(x - 99 * o.delta) <= 2 * _fresh_bound(o.n)


# ------------------------------------------------------------- image ops (Sec. 4.4)
def _box3_clamp(img):
    h, w = img.shape[:2]
    f = img.astype(np.float64)
    out = np.zeros_like(f)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            ys = np.clip(np.arange(h) + dy, 0, h - 1)
            xs = np.clip(np.arange(w) + dx, 0, w - 1)
            out += f[ys][:, xs]
    return out / 9.0


def test_meanfilter_matches_plaintext_box_filter(small4):
    o = small4
    img = inputs.random_field_image(5, 4, seed=3, channels=3)
    ct = o.encrypt_pixels(img.reshape(-1), seed=10)
    out, sc = o.meanfilter3(ct, o.delta, 5, 4, 3)
    assert out.shape[2] == 3
    dec = o.decrypt(out, sc).reshape(5, 4, 3)
    assert np.max(np.abs(dec - _box3_clamp(img))) < 1e-4


def test_brightness_and_watermark_pixel(toy):
    o = toy
    img = inputs.random_field_image(4, 4, seed=5).reshape(-1)
    ct = o.encrypt_pixels(img, seed=2)
    beta = inputs.brightness_beta(4)
    out, sc = o.brightness(ct, o.delta, beta)
    assert np.max(np.abs(o.decrypt(out, sc) - (img + beta))) < 1e-3
    out2, sc2 = o.watermark_pixel(ct, o.delta, 5.0, 6)
    diff = o.decrypt(out2, sc2) - img
    assert abs(diff[6] - 5.0) < 1e-3
    assert np.max(np.abs(np.delete(diff, 6))) < 1e-3


def test_blend_matches_plaintext(small4):
    o = small4
    img = inputs.random_field_image(3, 3, seed=8, channels=3)
    wm = inputs.binary_pattern(3, 3, seed=5)
    ci = o.encrypt_pixels(img.reshape(-1), seed=1)
    cw = o.encrypt_pixels(wm.reshape(-1), seed=2, ids=np.arange(9, dtype=np.uint64) + 1000)
    out, sc = o.blend(ci, cw, o.delta, 0.9, 3, 1)
    ref = 0.9 * img.astype(np.float64) + 0.1 * wm[:, :, None].astype(np.float64)
    assert np.max(np.abs(o.decrypt(out, sc).reshape(3, 3, 3) - ref)) < 1e-4


def test_match_matches_plaintext_sum_of_squares(small4):
    o = small4
    a = inputs.random_field_image(4, 4, seed=3)
    b = inputs.noisy_copy(a, seed=6)
    ca = o.encrypt_pixels(a.reshape(-1), seed=1)
    cb = o.encrypt_pixels(b.reshape(-1), seed=2)
    out, sc = o.match(ca, cb, o.delta)
    assert out.shape == (1, 2, 3, o.n)
    ref = float(((a.astype(np.float64) - b) ** 2).sum())
    assert abs(o.decrypt(out, sc)[0] - ref) < 1e-2


# ----------------------------------------------------------------- metrics, llround
def test_mse_psnr_against_paper_table():
    for label, m, p in read_golden("paper_quality_table.txt"):
        assert abs(psnr(float(m)) - float(p)) < 0.015, label
    assert mse([0, 2], [1, 0]) == 2.5


def test_llround_halves_away_from_zero():
    assert [llround(x) for x in (0.5, 1.5, -0.5, -2.5, 2.4999999999999996, 1e20)] == [1, 2, -1, -3, 2, 10 ** 20]
