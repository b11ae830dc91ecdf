"""Host-side checks, with exact Python integers, of three shortcuts in the kernels' modular
arithmetic, on the prime chains of every workload (primes from the oracle's generator):

* the per-pixel squared difference lifts a digit of t2 (Sec. 2.2.3, relinearisation by hybrid
  key switching; the digit is centered, its magnitude below half its prime q_j) into a
  modulus q >= q_j without a reduction: v if v <= (q_j - 1) / 2, else q - (q_j - v);
* fresh encryption (Sec. 2.2.2) adds the Gaussian noise e (|e| <= 31) to an inverse-transform
  output r in [0, 2q) as r + (q + e), then subtracts 2q and q conditionally;
* the key-switching accumulators stay in [0, 2q): acc + p with acc, p in [0, 2q), one
  conditional subtraction of 2q.

Each must give the canonical residue (or stay in its range) and never leave 64 bits."""
import random

import pytest

from oracle.ckks import Oracle, Params
from paper_2409_03568_gb300 import workloads as W

U64 = 1 << 64
RINGS = [W.ENC8192, W.OPS8192, W.RING16384,
         dict(log_n=10, prime_bits=[60, 40, 40, 40], log2_scale=40, special_bits=61)]


def moduli(ring):
    o = Oracle(Params(ring["log_n"], ring["prime_bits"], ring["log2_scale"], ring["special_bits"]))
    return [int(q) for q in o.q], int(o.P)


def csub(x, m):
    return x - m if x >= m else x


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: r.get("name", "n1024_4primes"))
def test_digit_lift_without_reduction(ring):
    qs, P = moduli(ring)
    rng = random.Random(5)
    pairs = 0
    for qj in qs:
        half = (qj - 1) // 2
        for q in qs + [P]:
            if q == qj or qj > q:
                continue   # these pairs keep the Barrett reduction
            pairs += 1
            for v in [0, 1, half - 1, half, half + 1, qj - 2, qj - 1] + [rng.randrange(qj) for _ in range(200)]:
                lifted = v if v <= half else q - (qj - v)
                centered = v if v <= half else v - qj
                assert 0 <= lifted < q
                assert lifted == centered % q
    assert pairs > 0   # at least the lifts into P take the shortcut


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: r.get("name", "n1024_4primes"))
def test_noise_epilogue(ring):
    qs, _ = moduli(ring)
    rng = random.Random(6)
    for q in qs:
        outs = [0, 1, q - 1, q, q + 1, 2 * q - 1] + [rng.randrange(2 * q) for _ in range(100)]
        for r in outs:
            for e in range(-31, 32):
                v = (r + ((q + e) % U64)) % U64   # the kernel's 64-bit adds
                assert v == r + q + e < U64       # no wrap: [q - 31, 3q + 31)
                v = csub(csub(v, 2 * q), q)
                assert v == (r + e) % q


@pytest.mark.parametrize("ring", RINGS, ids=lambda r: r.get("name", "n1024_4primes"))
def test_lazy_accumulators(ring):
    qs, P = moduli(ring)
    rng = random.Random(7)
    for q in qs + [P]:
        assert 4 * q < U64
        acc = 0
        total = 0
        for _ in range(500):
            p = rng.choice([0, 1, q - 1, q, 2 * q - 1, rng.randrange(2 * q)])
            acc = csub(acc + p, 2 * q)
            total += p
            assert 0 <= acc < 2 * q
            assert acc % q == total % q
