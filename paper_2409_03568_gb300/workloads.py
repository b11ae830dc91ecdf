"""Named parameter sets and seeded input recipes of the workloads this library is measured and
tested on (shapes of the paper's experiments, Sec. 4.2-4.4, at the ring sizes used here).

Parameters only: prime sizes, scale, image shapes, seeds. No cryptographic arithmetic.
"""
from . import inputs

# Toy CKKS (insecure, tests only): N=1024, two ~30-bit primes, Delta=2^25; an 8x8 uniform
# grayscale image, fresh and base-16 radix encryption.
TOY = dict(name="toy_n1024_l2", log_n=10, prime_bits=[30, 30], log2_scale=25, special_bits=0,
           h=8, w=8, c=1, image_seed=1)

# Encryption workload: N=8192, primes 60/40/60, Delta=2^40; one 64x64 grayscale random field
# encrypted fresh, with radix caches of base 10 and 16, a top-32 frequent-value cache with a
# 64-entry zero pool and a full 256-value cache; then decrypted. The special prime (61 bits)
# only serves the evaluation key of matching.
ENC8192 = dict(name="enc_n8192_l3_64x64", log_n=13, prime_bits=[60, 40, 60], log2_scale=40, special_bits=61,
               h=64, w=64, c=1, image_seed=2, top_k=32, pool_size=64)

# Image operations: N=8192, primes 60/40/40/40 + 61-bit special prime, Delta=2^40; a 128x128x3
# random-field image; brightness beta ~ U[-40, 40]; binary 128x128 watermark W at alpha=0.9;
# matching against a noisy copy (sigma 5 px).
OPS8192 = dict(name="ops_n8192_l4_128x128x3", log_n=13, prime_bits=[60, 40, 40, 40], log2_scale=40, special_bits=61,
               h=128, w=128, c=3, image_seed=3, beta_seed=4, watermark_seed=5, noisy_seed=6, alpha=0.9)

# Batched form: a ragged batch of 32 grayscale random-field images with sides uniform in
# 16..128 (seed 7), N=8192, primes 60/40/60; radix-16 encryption with randomness, then the 3x3
# mean filter.
BATCH32 = dict(name="batch32_n8192_l3_ragged", log_n=13, prime_bits=[60, 40, 60], log2_scale=40, special_bits=0,
               n_images=32, side_lo=16, side_hi=128, batch_seed=7, radix_base=16)

# Serving: Poisson arrivals at 200 requests/s, image sides uniform in 8..128, 1 or 3 channels,
# operation encrypt-only / mean filter / brightness / watermark / match at 4:2:2:1:1, ring
# N=8192 (primes 60/40/60) or N=16384 (primes 60/40/40/40/40) with probability 1/2 each,
# 120 GB HBM admission budget, full 256-value caches with 64-entry pools (seed 8).
SERVE = dict(name="serve_poisson200_mixed", rate=200.0, duration_s=60.0, side_lo=8, side_hi=128,
             op_weights=(4, 2, 2, 1, 1), budget_gb=120, seed=8,
             rings=(dict(log_n=13, prime_bits=[60, 40, 60], log2_scale=40, special_bits=61),
                    dict(log_n=14, prime_bits=[60, 40, 40, 40, 40], log2_scale=40, special_bits=61)))

# Serving-size ring: N=16384 with five primes.
RING16384 = dict(name="n16384_l5", log_n=14, prime_bits=[60, 40, 40, 40, 40], log2_scale=40, special_bits=61)


def image_for(wl):
    """The seeded image of a workload (uniform for the toy case, random field otherwise)."""
    if wl is TOY or wl.get("name") == TOY["name"]:
        return inputs.uniform_image(wl["h"], wl["w"], seed=wl["image_seed"], channels=wl["c"])
    return inputs.random_field_image(wl["h"], wl["w"], seed=wl["image_seed"], channels=wl["c"])


def ctx_kwargs(wl):
    return dict(log_n=wl["log_n"], prime_bits=list(wl["prime_bits"]), log2_scale=wl["log2_scale"],
                special_bits=wl.get("special_bits", 0))
