"""Python side of the CPU oracle for pixel-level CKKS with cached encryption (arXiv 2409.03568).

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs may import this module. It never imports the CUDA library and shares no code
with it; the one module both sides use is the seeded input generator, which holds none of the
method's arithmetic.

The ring arithmetic lives in ckks_oracle.c (scalar C, 128-bit products). This module strings
those steps together in the paper's order, keeps the scale of every ciphertext as an exact
rational, and decodes with exact big-integer CRT (Python ints):

  * KeyGen / Enc / Dec ............ Sec. 2.2.2, with the library sign convention
                                    pk = (-a*s + e, a), Dec = ct0 + ct1*s (the printed
                                    formulas do not cancel)
  * encoding of one pixel ......... Sec. 2.2 encoding: the pixel fills every slot, so the
                                    plaintext is the constant polynomial Delta*p
  * add / mult / relin / rescale .. Sec. 2.2.3; relin by hybrid key switching with one
                                    special prime P, rescale with centered rounding
  * radix / scanning / full cache . Sec. 3.2
  * radix randomness, zero pool ... Sec. 3.3: one Philox bit per radix position decides the
                                    add/subtract step; the pool index is a Philox draw
  * mean filter, brightness, matching, watermark ... Sec. 4.4 (clamp-to-edge borders, no clamp
                                    of the encrypted brightness, squared L2 distance for
                                    matching, blend alpha*I + (1-alpha)*W)
  * MSE / PSNR .................... Sec. 4.3.2
"""
import ctypes
import math
from fractions import Fraction

import numpy as np

from . import build as _build

u64p = ctypes.POINTER(ctypes.c_uint64)
i64p = ctypes.POINTER(ctypes.c_int64)
u32p = ctypes.POINTER(ctypes.c_uint32)
i32p = ctypes.POINTER(ctypes.c_int32)
i8p = ctypes.POINTER(ctypes.c_int8)
u8p = ctypes.POINTER(ctypes.c_uint8)

ID_POOL_BASE = 1 << 32      # ct ids of the randomness-pool zeros
ID_RADIX_BASE = 1 << 33     # ct ids of the cached radix powers
# value-cache slot j is encrypted with ct id j

_lib = None


def lib():
    """Load (building first if needed) the oracle's C library."""
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        _lib.orc_radix_bits.restype = ctypes.c_uint32
        _lib.orc_pool_index.restype = ctypes.c_uint32
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def llround(x):
    """C llround of an FP64 value: nearest integer, halves away from zero (exact)."""
    f = Fraction(float(x))
    r = math.floor(abs(f) + Fraction(1, 2))
    return -r if f < 0 else r


class Params:
    """CKKS parameters (Sec. 2.2 parameter table): ring dimension N = 2^log_n, ciphertext
    primes of the given bit sizes (for each size, the largest unused prime q < 2^bits with
    q = 1 mod 2N), scale Delta = 2^log2_scale, special prime bits
    for the evaluation key (0 = none), Gaussian sigma and tail bound."""

    def __init__(self, log_n, prime_bits, log2_scale, special_bits=0, sigma=3.2, bound=19):
        self.log_n = int(log_n)
        self.n = 1 << self.log_n
        self.prime_bits = [int(b) for b in prime_bits]
        self.L = len(self.prime_bits)
        self.log2_scale = int(log2_scale)
        self.special_bits = int(special_bits)
        self.sigma = float(sigma)
        self.bound = int(bound)


class Oracle:
    def __init__(self, params):
        self.params = params
        self.n = params.n
        self.L = params.L
        L = lib()
        q = np.zeros(self.L, dtype=np.uint64)
        P = np.zeros(1, dtype=np.uint64)
        bits = np.array(params.prime_bits, dtype=np.uint32)
        rc = L.orc_gen_primes(ctypes.c_uint32(params.log_n), ctypes.c_uint32(self.L), _p(bits, u32p),
                              ctypes.c_uint32(params.special_bits), _p(q, u64p), _p(P, u64p))
        if rc != 0:
            raise ValueError("no prime chain for these parameters")
        self.q = q
        self.P = int(P[0])
        self.T = np.zeros(params.bound + 1, dtype=np.uint64)
        L.orc_cdt_table(ctypes.c_double(params.sigma), ctypes.c_uint32(params.bound), _p(self.T, u64p))
        self.delta = 1 << params.log2_scale
        self.s = None
        self.pk = None
        self.evk = None

    # ---------------------------------------------------------------- keys
    def keygen(self, seed, with_evk=False):
        """KeyGen (Sec. 2.2.2): s, pk = (-a s + e, a); evk for relinearisation if asked."""
        n, L = self.n, self.L
        self.s = np.zeros(n, dtype=np.int8)
        self.pk = np.zeros((2, L, n), dtype=np.uint64)
        lib().orc_keygen(ctypes.c_uint32(n), ctypes.c_uint32(L), _p(self.q, u64p), ctypes.c_uint64(seed),
                         _p(self.T, u64p), ctypes.c_uint32(self.params.bound), _p(self.s, i8p),
                         _p(self.pk, u64p))
        if with_evk:
            if not self.P:
                raise ValueError("evaluation key needs a special prime")
            self.evk = np.zeros((L, 2, L + 1, n), dtype=np.uint64)
            lib().orc_keygen_evk(ctypes.c_uint32(n), ctypes.c_uint32(L), _p(self.q, u64p),
                                 ctypes.c_uint64(self.P), ctypes.c_uint64(seed), _p(self.T, u64p),
                                 ctypes.c_uint32(self.params.bound), _p(self.s, i8p), _p(self.evk, u64p))
        return self

    # ------------------------------------------------------------- encrypt
    def encrypt_msgs(self, msgs, ids, seed):
        """Fresh public-key encryption of encoded constant messages (Sec. 2.2.2)."""
        msgs = np.ascontiguousarray(msgs, dtype=np.int64)
        ids = _u64(ids)
        out = np.zeros((len(msgs), 2, self.L, self.n), dtype=np.uint64)
        lib().orc_encrypt_batch(ctypes.c_uint32(self.n), ctypes.c_uint32(self.L), _p(self.q, u64p),
                                _p(self.pk, u64p), ctypes.c_uint64(seed), _p(ids, u64p), _p(msgs, i64p),
                                ctypes.c_uint64(len(msgs)), _p(self.T, u64p),
                                ctypes.c_uint32(self.params.bound), _p(out, u64p))
        return out

    def encode_pixels(self, pixels):
        """Encoding (Sec. 2.2): pixel p fills every slot, so its plaintext is the constant Delta*p."""
        return np.asarray(pixels, dtype=np.int64).reshape(-1) * self.delta

    def encrypt_pixels(self, pixels, seed, ids=None):
        """Pixel-level fresh encryption (Sec. 3.1): ciphertext k gets ct id ids[k] (default k)."""
        pix = np.asarray(pixels, dtype=np.uint8).reshape(-1)
        if ids is None:
            ids = np.arange(len(pix), dtype=np.uint64)
        return self.encrypt_msgs(self.encode_pixels(pix), ids, seed)

    # -------------------------------------------------------------- caches
    @staticmethod
    def radix_powers(base):
        """Number of base-r digits a value in [0, 255] needs (Sec. 3.2 radix caching)."""
        n = 1
        while base ** n <= 255:
            n += 1
        return n

    def radix_cache(self, base, seed):
        """Cache Enc(r^k) for every power r^k <= 255 (Sec. 3.2), ct ids ID_RADIX_BASE + k."""
        n_pow = self.radix_powers(base)
        powers = np.array([base ** k for k in range(n_pow)], dtype=np.int64)
        cts = self.encrypt_msgs(powers * self.delta, ID_RADIX_BASE + np.arange(n_pow, dtype=np.uint64), seed)
        return {"kind": "radix", "base": base, "n_pow": n_pow, "cts": cts}

    @staticmethod
    def top_values(scan_pixels, k):
        """Scanning step of Sec. 3.2: the k most frequent values present, ties to the smaller
        value; values absent from the scan are never cached."""
        counts = np.bincount(np.asarray(scan_pixels, dtype=np.uint8).reshape(-1), minlength=256)
        order = sorted(range(256), key=lambda v: (-int(counts[v]), v))
        return [v for v in order if counts[v] > 0][:k]

    def pool(self, size, seed):
        """Randomness pool of `size` encryptions of zero (Sec. 3.3), ct ids ID_POOL_BASE + m."""
        if size == 0:
            return np.zeros((0, 2, self.L, self.n), dtype=np.uint64)
        return self.encrypt_msgs(np.zeros(size, dtype=np.int64),
                                 ID_POOL_BASE + np.arange(size, dtype=np.uint64), seed)

    def value_cache(self, values, pool_size, seed, radix_base=0):
        """Scanning-based (values = top-K) or full (values = 0..255) caching, Sec. 3.2: slot j
        holds Enc(values[j]) with ct id j; plus the zero pool; plus radix powers when misses
        are to be radix-encrypted."""
        values = [int(v) for v in values]
        cts = self.encrypt_msgs(np.array(values, dtype=np.int64) * self.delta,
                                np.arange(len(values), dtype=np.uint64), seed)
        lut = np.full(256, -1, dtype=np.int32)
        for j, v in enumerate(values):
            lut[v] = j
        c = {"kind": "lookup", "values": values, "cts": cts, "lut": lut,
             "pool": self.pool(pool_size, seed), "pool_size": pool_size}
        if radix_base:
            c["radix"] = self.radix_cache(radix_base, seed)
        return c

    def freq_cache(self, scan_pixels, top_k, pool_size, seed, radix_base=0):
        return self.value_cache(self.top_values(scan_pixels, top_k), pool_size, seed, radix_base)

    def full_cache(self, pool_size, seed):
        return self.value_cache(list(range(256)), pool_size, seed)

    def encrypt_radix(self, pixels, cache, seed, randomize=True, ids=None):
        """Radix-cached encryption with the add/subtract randomness (Sec. 3.2, 3.3), sequential
        form."""
        pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.uint8).reshape(-1))
        if ids is None:
            ids = np.arange(len(pix), dtype=np.uint64)
        ids = _u64(ids)
        out = np.zeros((len(pix), 2, self.L, self.n), dtype=np.uint64)
        lib().orc_radix_encrypt_batch(ctypes.c_uint32(self.n), ctypes.c_uint32(self.L), _p(self.q, u64p),
                                      _p(cache["cts"], u64p), ctypes.c_uint32(cache["n_pow"]),
                                      ctypes.c_uint32(cache["base"]), _p(pix, u8p), _p(ids, u64p),
                                      ctypes.c_uint64(len(pix)), ctypes.c_uint64(seed),
                                      ctypes.c_int(1 if randomize else 0), _p(out, u64p))
        return out

    def encrypt_lookup(self, pixels, cache, seed, miss_policy=0, ids=None):
        """Scanning-based / full cached encryption with the zero pool (Sec. 3.2, 3.3). A value
        outside the cache is encrypted fresh (miss_policy 0) or radix-encrypted with
        randomness (miss_policy 1)."""
        pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.uint8).reshape(-1))
        if ids is None:
            ids = np.arange(len(pix), dtype=np.uint64)
        ids = _u64(ids)
        out = np.zeros((len(pix), 2, self.L, self.n), dtype=np.uint64)
        lib().orc_lookup_encrypt_batch(ctypes.c_uint32(self.n), ctypes.c_uint32(self.L), _p(self.q, u64p),
                                       _p(cache["cts"], u64p), _p(cache["lut"], i32p),
                                       _p(cache["pool"], u64p), ctypes.c_uint32(cache["pool_size"]),
                                       _p(pix, u8p), _p(ids, u64p), ctypes.c_uint64(len(pix)),
                                       ctypes.c_uint64(seed), _p(out, u64p))
        miss = np.nonzero(cache["lut"][pix] < 0)[0]
        if len(miss):
            if miss_policy == 0:
                out[miss] = self.encrypt_pixels(pix[miss], seed, ids=ids[miss])
            else:
                out[miss] = self.encrypt_radix(pix[miss], cache["radix"], seed, True, ids=ids[miss])
        return out

    # ----------------------------------------------------------------- ops
    def _limbs(self, ct):
        return ct.shape[-2]

    def add(self, a, b):
        out = np.empty_like(a)
        lim = self._limbs(a)
        for k in range(a.shape[0]):
            lib().orc_ct_add(ctypes.c_uint32(self.n), ctypes.c_uint32(lim), _p(self.q, u64p),
                             _p(np.ascontiguousarray(a[k]), u64p), _p(np.ascontiguousarray(b[k]), u64p),
                             _p(out[k], u64p))
        return out

    def sub(self, a, b):
        out = np.empty_like(a)
        lim = self._limbs(a)
        for k in range(a.shape[0]):
            lib().orc_ct_sub(ctypes.c_uint32(self.n), ctypes.c_uint32(lim), _p(self.q, u64p),
                             _p(np.ascontiguousarray(a[k]), u64p), _p(np.ascontiguousarray(b[k]), u64p),
                             _p(out[k], u64p))
        return out

    def add_int(self, a, k):
        """Plaintext add of the encoded integer k (coefficient 0 of c0)."""
        out = np.empty_like(a)
        lim = self._limbs(a)
        for j in range(a.shape[0]):
            kk = int(k[j]) if np.ndim(k) else int(k)
            lib().orc_ct_add_int(ctypes.c_uint32(self.n), ctypes.c_uint32(lim), _p(self.q, u64p),
                                 _p(np.ascontiguousarray(a[j]), u64p), ctypes.c_int64(kk), _p(out[j], u64p))
        return out

    def mul_int(self, a, k):
        """Plaintext multiply by the encoded integer k (every coefficient)."""
        out = np.empty_like(a)
        lim = self._limbs(a)
        for j in range(a.shape[0]):
            lib().orc_ct_mul_int(ctypes.c_uint32(self.n), ctypes.c_uint32(lim), _p(self.q, u64p),
                                 _p(np.ascontiguousarray(a[j]), u64p), ctypes.c_int64(int(k)), _p(out[j], u64p))
        return out

    def rescale(self, a):
        """Rescale by the last prime q_t (Sec. 2.2.3): c_j <- (c_j - [c_t]_centered) * q_t^-1 mod q_j,
        centered in (-q_t/2, q_t/2]."""
        lim = self._limbs(a)
        out = np.zeros(a.shape[:-2] + (lim - 1, self.n), dtype=np.uint64)
        for j in range(a.shape[0]):
            lib().orc_rescale(ctypes.c_uint32(self.n), ctypes.c_uint32(lim), _p(self.q, u64p),
                              _p(np.ascontiguousarray(a[j]), u64p), _p(out[j], u64p))
        return out

    def encode_const(self, value, scale):
        """A real plaintext constant at a given scale: llround(value * scale) in FP64, halves away
        from zero."""
        return llround(float(value) * float(scale))

    # brightness, Sec. 4.4.2: beta added to coefficient 0, no clamp in the encrypted domain
    def brightness(self, a, scale, beta):
        return self.add_int(a, self.encode_const(beta, scale)), Fraction(scale)

    def watermark_pixel(self, a, scale, x, index):
        """Sec. 4.4.4 as printed: add x to one chosen pixel's ciphertext."""
        out = a.copy()
        out[index:index + 1] = self.add_int(a[index:index + 1], self.encode_const(x, scale))
        return out, Fraction(scale)

    def ptmul(self, a, scale, c):
        k = self.encode_const(c, self.delta)
        return self.mul_int(a, k), Fraction(scale) * self.delta

    def meanfilter3(self, a, scale, h, w, ch):
        """3x3 mean filter (Sec. 4.4.1): clamp-to-edge 9-neighbour sum, x encoded 1/9, rescale."""
        lim = self._limbs(a)
        k9 = self.encode_const(1.0 / 9.0, self.delta)
        out = np.zeros((h * w * ch, 2, lim - 1, self.n), dtype=np.uint64)
        a = np.ascontiguousarray(a)
        lib().orc_meanfilter3(ctypes.c_uint32(self.n), ctypes.c_uint32(lim), _p(self.q, u64p), _p(a, u64p),
                              ctypes.c_uint32(h), ctypes.c_uint32(w), ctypes.c_uint32(ch), ctypes.c_int64(k9),
                              _p(out, u64p))
        return out, Fraction(scale) * self.delta / int(self.q[lim - 1])

    def blend(self, img, wm, scale, alpha, ch, ch_w):
        """Watermark blend alpha*I + (1-alpha)*W, W an encrypted pattern (the workload's form of
        Sec. 4.4.4)."""
        lim = self._limbs(img)
        ka = self.encode_const(alpha, self.delta)
        kb = self.encode_const(1.0 - float(alpha), self.delta)
        out = np.zeros((img.shape[0], 2, lim - 1, self.n), dtype=np.uint64)
        img = np.ascontiguousarray(img)
        wm = np.ascontiguousarray(wm)
        lib().orc_blend(ctypes.c_uint32(self.n), ctypes.c_uint32(lim), _p(self.q, u64p), _p(img, u64p),
                        _p(wm, u64p), ctypes.c_uint64(img.shape[0]), ctypes.c_uint32(ch), ctypes.c_uint32(ch_w),
                        ctypes.c_int64(ka), ctypes.c_int64(kb), _p(out, u64p))
        return out, Fraction(scale) * self.delta / int(self.q[lim - 1])

    def sqdiff_sum_raw(self, a, b):
        """Sum over ciphertexts of (a - b) (x) (a - b), degree 2, [3][limbs][n]."""
        lim = self._limbs(a)
        out = np.zeros((3, lim, self.n), dtype=np.uint64)
        a = np.ascontiguousarray(a)
        b = np.ascontiguousarray(b)
        lib().orc_sqdiff_sum(ctypes.c_uint32(self.n), ctypes.c_uint32(lim), _p(self.q, u64p), _p(a, u64p),
                             _p(b, u64p), ctypes.c_uint64(a.shape[0]), _p(out, u64p))
        return out

    def relin(self, d):
        """Relinearise a degree-2 ciphertext [3][limbs][n] (Sec. 2.2.3) by hybrid key switching:
        one digit per ciphertext prime, one special prime P, mod-down with centered rounding."""
        lim = d.shape[1]
        out = np.zeros((2, lim, self.n), dtype=np.uint64)
        d = np.ascontiguousarray(d)
        lib().orc_relin(ctypes.c_uint32(self.n), ctypes.c_uint32(lim), ctypes.c_uint32(self.L), _p(self.q, u64p),
                        ctypes.c_uint64(self.P), _p(self.evk, u64p), _p(d, u64p), _p(out, u64p))
        return out

    def match(self, a, b, scale):
        """Image matching (Sec. 4.4.3; |x| is not a CKKS polynomial, so the squared L2 distance):
        sum of squared differences, relinearised
        once and rescaled once. Returns ([1][2][limbs-1][n], scale)."""
        lim = self._limbs(a)
        t = self.sqdiff_sum_raw(a, b)
        r = self.relin(t)[None]
        return self.rescale(r), Fraction(scale) * Fraction(scale) / int(self.q[lim - 1])

    def sqdiff_image(self, a, b, scale):
        """Squared difference pixel by pixel (the per-pixel form of Sec. 4.4.3, squared):
        for every ciphertext pair d = a - b, d (x) d, relinearised and rescaled on its own.
        Returns ([count][2][limbs-1][n], scale)."""
        lim = self._limbs(a)
        out = np.zeros((a.shape[0], 2, lim - 1, self.n), dtype=np.uint64)
        for k in range(a.shape[0]):
            t = self.sqdiff_sum_raw(a[k:k + 1], b[k:k + 1])
            out[k] = self.rescale(self.relin(t)[None])[0]
        return out, Fraction(scale) * Fraction(scale) / int(self.q[lim - 1])

    # ------------------------------------------------------------- decrypt
    def decrypt_residues(self, ct):
        """Coefficient 0 of c0 + c1*s per limb (Sec. 2.2.2), [count][limbs]."""
        ct = np.ascontiguousarray(ct)
        lim = self._limbs(ct)
        out = np.zeros((ct.shape[0], lim), dtype=np.uint64)
        for k in range(ct.shape[0]):
            lib().orc_decrypt_coef0(ctypes.c_uint32(self.n), ctypes.c_uint32(lim), _p(self.q, u64p),
                                    _p(self.s, i8p), _p(ct[k], u64p), _p(out[k], u64p))
        return out

    def crt(self, residues):
        """Exact CRT of residues mod q_0..q_{t-1} to the centered integer in (-Q/2, Q/2]."""
        lim = len(residues)
        qs = [int(x) for x in self.q[:lim]]
        Q = math.prod(qs)
        x = 0
        for i in range(lim):
            Qi = Q // qs[i]
            x += (int(residues[i]) * pow(Qi, -1, qs[i]) % qs[i]) * Qi
        x %= Q
        if x > Q // 2:
            x -= Q
        return x

    def decrypt(self, ct, scale):
        """Decrypt and decode: centered CRT of coefficient 0 divided by the exact scale."""
        res = self.decrypt_residues(ct)
        sc = Fraction(scale)
        return np.array([float(Fraction(self.crt(r)) / sc) for r in res], dtype=np.float64)

    def decrypt_poly(self, ct):
        """All coefficients of c0 + c1*s as centered integers (for noise checks)."""
        ct = np.ascontiguousarray(ct)
        lim = self._limbs(ct)
        out = np.zeros((lim, self.n), dtype=np.uint64)
        lib().orc_decrypt_poly(ctypes.c_uint32(self.n), ctypes.c_uint32(lim), _p(self.q, u64p),
                               _p(self.s, i8p), _p(ct, u64p), _p(out, u64p))
        return [self.crt(out[:, i]) for i in range(self.n)]


def mse(a, b):
    """Mean squared error between two images (Sec. 4.3.2)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.mean((a - b) ** 2))


def psnr(mse_value, max_i=255.0):
    """Peak signal-to-noise ratio in dB (Sec. 4.3.2)."""
    return 10.0 * math.log10(max_i * max_i / mse_value)
