"""The reference arm of bench.py (the oracle on the host cores) runs without a GPU: one bounded
step, one JSON line carrying the keys the main arm's line carries, the same metric and unit."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    for key in ("value", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling", "vs_baseline",
                "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "enc_n8192_l3_64x64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_parity_on_sample_compares_word_for_word():
    """The bench's parity check (its ciphertexts against the oracle's on the CPU-baseline sample)
    accepts identical words and names every result that differs in one word."""
    import sys
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import bench
    ref = {}
    bench.cpu_baseline(sample_steps=1, sample=9, keep=ref)
    idx = ref["idx"].astype(np.int64)
    n_px, n = 4096, 8192
    enc = {}
    for m in ("fresh", "radix16", "radix10", "freq32_pool64", "full256_pool64"):
        t = np.zeros((n_px, 2, 3, n), dtype=np.uint64)
        t[idx] = ref[m]
        enc[m] = torch.from_numpy(t.view(np.int64).reshape(-1))
    ops = {}
    for name, limbs in (("brightness", 3), ("blend", 2)):
        t = np.zeros((n_px, 2, limbs, n), dtype=np.uint64)
        t[idx] = ref[name]
        ops[name] = torch.from_numpy(t.view(np.int64).reshape(-1))
    ok = bench.parity_on_sample(None, enc, ops, ref, n_check=9)
    assert ok["bit_exact"] and ok["pixels"] == 9 and len(ok["results"]) == 7
    flipped = enc["radix10"].view(n_px, -1)
    flipped[int(idx[4]), 12345] ^= 1
    bad = bench.parity_on_sample(None, enc, ops, ref, n_check=9)
    assert not bad["bit_exact"] and bad["mismatched"] == ["radix10"]


def test_serving_roofline_bytes():
    """The serving record's algorithmic bytes: encryption written once, each operation's inputs
    read and output written once (brightness in place), decryption reads half a ciphertext;
    refused requests count nothing."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    wl = {"rings": ({"log_n": 10, "prime_bits": [60, 40, 60]},)}
    n, L = 1024, 3
    ct, ct1 = 2 * L * n * 8, 2 * (L - 1) * n * 8
    reqs = [dict(kind=0, ring=0, h=2, w=3, c=1), dict(kind=1, ring=0, h=2, w=2, c=3),
            dict(kind=2, ring=0, h=1, w=1, c=1), dict(kind=3, ring=0, h=2, w=2, c=3),
            dict(kind=4, ring=0, h=1, w=2, c=1), dict(kind=0, ring=0, h=9, w=9, c=3)]
    got = bench.serve_algorithmic_bytes(wl, reqs, [True] * 5 + [False])
    want = (6 * ct + 6 * ct // 2) + (12 * ct + 12 * (ct + ct1) + 12 * ct1 // 2) + (ct + ct // 2) + \
        ((12 + 4) * ct + 12 * (ct + ct1) + 4 * ct + 12 * ct1 // 2) + (4 * ct + 4 * ct)
    assert got == want
