"""The allocation-free matching entry point, for callers that cannot allocate device memory.

ichee_sqdiff_sum_noalloc works in one static device array instead of allocating scratch.
Its result must be the ciphertext ichee_eval(ICHEE_OP_SQDIFF_SUM) produces, bit for bit (the
tolerance every ciphertext comparison in these tests uses), on two calls in a row -- the
second call finds the first call's leftovers in the shared array. This file is named to be
collected last, and it builds its own context so it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2409_03568_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    dict(log_n=10, prime_bits=[60, 40, 40, 40], log2_scale=40, special_bits=61, shape=(5, 6, 3)),
    dict(log_n=13, prime_bits=[60, 40, 40, 40], log2_scale=40, special_bits=61, shape=(4, 4, 3)),
    # N = 2^14: the accumulation runs as two half transforms per limb (its own scratch slices)
    dict(log_n=14, prime_bits=[60, 40, 40, 40, 40], log2_scale=40, special_bits=61, shape=(3, 3, 1)),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "n%d" % (1 << c["log_n"]))
def test_noalloc_matching_equals_allocating_matching(case):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03568_gb300 import ichee
    h, w, c = case["shape"]
    ctx = ichee.Context(case["log_n"], case["prime_bits"], case["log2_scale"], case["special_bits"])
    ctx.keygen(4321, with_evk=True)
    img = inputs.random_field_image(h, w, seed=3, channels=c).reshape(-1)
    other = inputs.noisy_copy(img, seed=6)
    a, ma = ctx.encrypt(torch.from_numpy(img).cuda(), h, w, c, 11)
    b, mb = ctx.encrypt(torch.from_numpy(other).cuda(), h, w, c, 12)
    ref, mref = ctx.eval(ichee.OP_SQDIFF_SUM, a, ma, b, mb, out_n_ct=1, out_level=ma.level - 1)
    ref_dec = ctx.decrypt(ref, mref).cpu().numpy()
    for _ in range(2):
        out = ctx.empty_cts(1, ma.level - 1)
        out.fill_(-1)
        m = ichee.ichee_sqdiff_sum_noalloc(ctx.handle, a, ma, b, mb, out, ctx.stream())
        assert (m.h, m.w, m.c, m.level) == (mref.h, mref.w, mref.c, mref.level)
        assert m.scale == mref.scale
        assert torch.equal(out, ref)
        np.testing.assert_allclose(ctx.decrypt(out, m).cpu().numpy(), ref_dec, rtol=1e-9)
    plain = float(((img.astype(np.float64) - other) ** 2).sum())
    assert abs(ref_dec[0] - plain) < 1e-2
    ctx.close()
