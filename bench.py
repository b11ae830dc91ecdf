#!/usr/bin/env python3
"""Benchmark of the pixel-level CKKS hot path (arXiv 2409.03568) on GB300.

One step = every row of the hot path over one synthetic 64x64 grayscale random-field image at
N = 8192 with primes 60/40/60 and Delta = 2^40:
  encrypt the 4096 pixels five ways -- fresh public-key encryption, radix cache base 16 and
  base 10 with the add/subtract randomness, top-32 frequent-value cache with a 64-entry zero
  pool (misses encrypted fresh), full 256-value cache with the pool;
  image operations on the fresh ciphertexts -- 3x3 mean filter, brightness, watermark blend
  with an encrypted binary pattern, matching (sum of squared differences against an encrypted
  noisy copy, relinearised);
  decrypt and decode every result.
Key generation and cache building are set-up (the paper's offline caching phase) and are not
timed. `value` = pixel ciphertexts encrypted per second over whole steps (5 x 4096 per step).

Prints one JSON line (rank 0). `--impl reference` times the CPU oracle on a bounded sample of
the same step instead.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2409_03568_gb300 import inputs, metrics as M, workloads as W  # noqa: E402

METRIC = "pixel ciphertexts/s at N=8192 (fresh + cached encryption, image ops, decryption per step)"
UNIT = "pixel-ct/s"
HBM_PEAK = None          # filled from MEASURED_PEAKS.json
IMAD_PER_SM_CLK = 64     # 32-bit integer multiply-add issue rate per SM per clock
IMAD_PER_MODMUL = 10     # 32x32 partial products in one 64-bit Shoup product (4 high + 2 x 3 low)
SM_COUNT = 152
SM_MAX_MHZ = 2070.0


# DRAM traffic per launch of a kernel, from one ncu capture of the bench's launch of it
# (profiles/k_encrypt_fresh_enc_n8192_64x64.md: dram__bytes_read.sum + dram__bytes_write.sum), valid
# while the files that kernel is compiled from are unchanged; otherwise the roofline reports
# traffic null.
NCU_TRAFFIC = {
    "fresh": {"bytes": 1.55488e9, "sha256_16": "0cb929e66ed600c4",
              "sources": ["paper_2409_03568_gb300/csrc/kernels_enc.cu", "paper_2409_03568_gb300/csrc/ntt.cuh",
                          "paper_2409_03568_gb300/csrc/common.cuh", "paper_2409_03568_gb300/csrc/internal.h"]},
}


def ncu_traffic(kernel):
    import hashlib
    rec = NCU_TRAFFIC.get(kernel)
    if rec is None:
        return None
    h = hashlib.sha256()
    for f in rec["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return rec["bytes"] if h.hexdigest()[:16] == rec["sha256_16"] else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", choices=["all", "enc8192", "ops128", "batch32", "serve", "shard"], default="all",
                    help="all (default): the headline step, then the other configurations as sub-records of the "
                         "same JSON line; enc8192: the headline step alone; ops128: image operations on the "
                         "128x128x3 four-prime image; batch32: ragged batch under a CUDA graph vs per-image "
                         "launches; serve: Poisson request stream through the continuous-batching server; "
                         "shard: the step with the image's rows sharded over the ranks (the form every N > 1 "
                         "run takes)")
    ap.add_argument("--duration", type=float, default=None, help="serve: seconds of arrivals (default 60)")
    ap.add_argument("--op", choices=sorted(SINGLE_OPS), default=None,
                    help="time one operation of the enc8192 workload on its own (for kernel profiles)")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_over_ranks(ms, units):
    """Across the ranks of one job (one process per GPU, replicas): the slowest rank's timed
    span and the sum of the units every rank processed. Identity without torch.distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, units
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.barrier()
    return float(t.item()), int(u.item())


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.strip().split(", ") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for name, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    from paper_2409_03568_gb300 import ichee

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = W.ENC8192
    hbm_peak, peak_kind = measured_peaks()

    ctx = ichee.Context(**W.ctx_kwargs(wl), device=local)
    ctx.keygen(2024, with_evk=True)
    h, w, c = wl["h"], wl["w"], wl["c"]
    n_px = h * w * c
    img = W.image_for(wl).reshape(-1)
    wm = inputs.binary_pattern(h, w, seed=5)
    noisy = inputs.noisy_copy(img, seed=6)
    beta = inputs.brightness_beta(4)
    d_img = torch.from_numpy(img).cuda()
    scan = d_img
    caches = {
        "radix16": ctx.build_cache(ichee.CACHE_RADIX, 11, radix_base=16, randomize=1),
        "radix10": ctx.build_cache(ichee.CACHE_RADIX, 12, radix_base=10, randomize=1),
        "freq32_pool64": ctx.build_cache(ichee.CACHE_FREQ, 13, top_k=32, pool_size=64, scan=scan),
        "full256_pool64": ctx.build_cache(ichee.CACHE_FULL, 14, pool_size=64),
    }
    lut_values, _ = ichee.ichee_cache_info(caches["freq32_pool64"])
    hit_rate = float(np.isin(img, lut_values).mean())
    wm_ct, wm_meta = ctx.encrypt(torch.from_numpy(wm.reshape(-1)).cuda(), h, w, 1, seed=21)
    nz_ct, nz_meta = ctx.encrypt(torch.from_numpy(noisy).cuda(), h, w, c, seed=22)
    L = ctx.L
    methods = ["fresh"] + list(caches)
    enc_out = {m: ctx.empty_cts(n_px, L - 1) for m in methods}
    ops_out = {"meanfilter3": ctx.empty_cts(n_px, L - 2), "brightness": ctx.empty_cts(n_px, L - 1),
               "blend": ctx.empty_cts(n_px, L - 2), "match": ctx.empty_cts(1, L - 2)}
    dec_out = {k: torch.empty(n_px, dtype=torch.float64, device="cuda") for k in methods + list(ops_out)}
    metas = {}
    st = ctx.stream()
    H = ctx.handle

    def p_encrypt(m, pixels=None):
        def f():
            metas[m] = ichee.ichee_encrypt_image(H, None if m == "fresh" else caches[m],
                                                 d_img if pixels is None else pixels, h, w, c, 7, enc_out[m], st)
        return f

    def p_op(name, op, b=None, mb=None, args=()):
        def f():
            metas[name] = ichee.ichee_eval(H, op, enc_out["fresh"], metas["fresh"], b, mb, args, ops_out[name], st)
        return f

    def p_decrypt():
        # one batched decryption per level: the encryptions and brightness keep every limb, the
        # rescaled outputs (mean filter, blend, match) one fewer
        def f():
            groups = {}
            for k in methods + list(ops_out):
                groups.setdefault(metas[k].level, []).append(k)
            for ks in groups.values():
                ichee.ichee_decrypt_batch(H, [enc_out[k] if k in enc_out else ops_out[k] for k in ks],
                                          [metas[k] for k in ks], [dec_out[k] for k in ks], st)
        return f

    phases = [(m, p_encrypt(m)) for m in methods] + [
        ("meanfilter3", p_op("meanfilter3", ichee.OP_MEANFILTER3)),
        ("brightness", p_op("brightness", ichee.OP_BRIGHTNESS, args=(beta,))),
        ("blend", p_op("blend", ichee.OP_BLEND, wm_ct, wm_meta, args=(0.9,))),
        ("match", p_op("match", ichee.OP_SQDIFF_SUM, nz_ct, nz_meta)),
        ("decrypt", p_decrypt()),
    ]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")   # > L2 (129 MB)
    events = {name: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for name, _ in phases}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def step():
        for name, fn in phases:
            events[name][0].record()
            fn()
            events[name][1].record()

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    # correctness guard on the benchmarked outputs (decoded pixels of every encryption), and
    # the image-quality figures of Sec. 4.3.2 / 4.4.1 on them (rounded decoded pixels)
    quality = {}
    for m in methods:
        dec = dec_out[m].cpu().numpy()
        err = float(np.abs(dec - img).max())
        if err > 1e-3:
            raise RuntimeError("decode error %.3g for %s" % (err, m))
        quality[m] = {"max_abs_error": err, "mse_rounded": M.mse(img, np.rint(dec))}
    mf = np.clip(np.rint(dec_out["meanfilter3"].cpu().numpy()), 0, 255)
    mf_mse = M.mse(img, mf)
    quality["meanfilter3_vs_original"] = {"mse": round(mf_mse, 3), "psnr_db": round(M.psnr(mf_mse), 2)}
    phase_ms = {name: 0.0 for name, _ in phases}
    total_ms = 0.0
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for _ in range(args.steps):
        flush.zero_()
        ev0.record()
        step()
        ev1.record()
        torch.cuda.synchronize()
        total_ms += ev0.elapsed_time(ev1)
        for name, _ in phases:
            phase_ms[name] += events[name][0].elapsed_time(events[name][1])
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms, units_all = reduce_over_ranks(total_ms, len(methods) * n_px * args.steps)
    ms_step = total_ms / args.steps
    phase_ms = {k: v / args.steps for k, v in phase_ms.items()}
    value = units_all / (total_ms / 1e3)

    # roofline of every kernel-level phase (algorithmic work per launch / event time)
    n = ctx.n
    ct_bytes = 2 * L * n * 8
    logn = wl["log_n"]
    modmul_fresh = L * (3 * (n // 2) * logn + 2 * n)           # per pixel ciphertext
    sm_mhz = clk["sm_mhz"] if clk else SM_MAX_MHZ
    alu_peak = SM_COUNT * SM_MAX_MHZ * 1e6 * IMAD_PER_SM_CLK / IMAD_PER_MODMUL / 1e9   # Gmodmul/s
    kernels = {}

    def rl_hbm(name, bytes_per_launch):
        t = phase_ms[name] / 1e3
        a = bytes_per_launch / t / 1e9
        kernels[name] = {"bound": "hbm", "achieved": round(a, 1), "peak": hbm_peak, "unit": "GB/s",
                         "frac": round(a / hbm_peak, 4), "ms": round(phase_ms[name], 4)}

    def rl_alu(name, modmuls_per_launch):
        t = phase_ms[name] / 1e3
        a = modmuls_per_launch / t / 1e9
        kernels[name] = {"bound": "alu", "achieved": round(a, 1), "peak": round(alu_peak, 1), "unit": "Gmodmul/s",
                         "frac": round(a / alu_peak, 4), "ms": round(phase_ms[name], 4)}

    rl_alu("fresh", n_px * modmul_fresh)
    for m in ("radix16", "radix10", "full256_pool64"):
        rl_hbm(m, n_px * ct_bytes)
    # frequent-value cache: hits are lookups, misses run the fresh kernel
    kernels["freq32_pool64"] = {"ms": round(phase_ms["freq32_pool64"], 4), "hit_rate": round(hit_rate, 4)}
    rl_hbm("meanfilter3", n_px * (ct_bytes + 2 * (L - 1) * n * 8))
    rl_hbm("brightness", n_px * 2 * ct_bytes)
    rl_hbm("blend", n_px * (2 * ct_bytes + 2 * (L - 1) * n * 8))
    rl_alu("match", n_px * L * (2 * (n // 2) * logn + 3 * n))
    n_dec = sum(metas[k].n_ct * (metas[k].level + 1) * n * 8 for k in methods + list(ops_out))
    rl_hbm("decrypt", n_dec)
    dominant = max((k for k in kernels if "frac" in kernels[k]), key=lambda k: phase_ms[k])
    roof = dict(kernels[dominant])
    roof["kernel"] = dominant
    roof["peak_kind"] = peak_kind if roof["bound"] == "hbm" else "derived: %d SMs x %.0f MHz x %d IMAD/clk / %d IMAD per modmul" % (
        SM_COUNT, SM_MAX_MHZ, IMAD_PER_SM_CLK, IMAD_PER_MODMUL)
    roof["traffic"] = ncu_traffic(dominant)
    if roof["traffic"] is not None:
        roof["traffic_unit"] = "bytes per launch (DRAM read + write, ncu)"
        roof["algorithmic_bytes"] = n_px * ct_bytes

    out = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64 (RNS residues mod 60/40/60-bit primes)",
        "data": "synthetic (Gaussian random field 64x64, correlation 6 px, seed 2; stands in for USC-SIPI)",
        "config": {"workload": wl["name"], "N": n, "primes_bits": wl["prime_bits"], "log2_scale": wl["log2_scale"],
                   "image": "%dx%dx%d" % (h, w, c), "methods": methods, "ops": list(ops_out),
                   "freq_hit_rate": round(hit_rate, 4), "l2": "flushed (512 MB write) before every step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "phases_ms": {k: round(v, 4) for k, v in phase_ms.items()},
        "px_per_s": {m: round(n_px / (phase_ms[m] / 1e3), 1) for m in methods},
        "kernels": kernels,
        "roofline": roof,
        "gpu_launches": None,
        "clocks": clk,
        "quality": quality,
    }
    out["extras"] = extras_ours(args, ctx, ichee, enc_out["fresh"], metas["fresh"], nz_ct, nz_meta, flush, alu_peak)
    # measured integer throughput (outside the timed region): the rate behind the derived peak,
    # and what the library's butterfly reaches alone in registers
    imad_s, bfly_s = ichee.ichee_probe_int_throughput(local)
    out["alu_probe"] = {"imad_per_sm_per_clk": round(imad_s / SM_COUNT / (sm_mhz * 1e6), 2),
                        "butterfly_g_per_s": round(bfly_s / 1e9, 1),
                        "dominant_frac_of_butterfly_rate": round(kernels[dominant]["achieved"] / (bfly_s / 1e9), 4)
                        if kernels[dominant]["bound"] == "alu" else None}
    # launches of our kernels per step: 1 per encryption (3 for the frequent-value cache: hits,
    # the list of misses, the misses), 1 per mean filter / brightness / blend, matching: 1
    # accumulate + 1 reduce + 2 inverse transform/scale + digits + transform + MAC + transform +
    # mod-down + rescale, 1 batched decryption per level
    n_levels = len({metas[k].level for k in methods + list(ops_out)})
    out["gpu_launches"] = args.steps * (len(methods) + 2 + 3 + 10 + n_levels)

    if not args.no_e2e:
        out["e2e"] = e2e_ours(args, ctx, ichee, img, wm_ct, wm_meta, nz_ct, nz_meta, beta, caches, methods, enc_out,
                              ops_out, st, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ref = {}
        out["cpu_baseline"] = cpu_baseline(sample_steps=1, sample=484, keep=ref)
        out["parity_sample"] = parity_on_sample(ctx, enc_out, ops_out, ref)
    ctx.close()
    if args.workload == "all" and world == 1:
        # the other configurations, each in a process of its own (its own device memory), as
        # sub-records of this line
        del enc_out, ops_out, dec_out, flush, caches
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        out["configs"] = {name: sub_record(name, extra) for name, extra in
                          (("ops128", ["--steps", "10", "--warmup", "3"]),
                           ("batch32", ["--steps", "10", "--warmup", "3"]),
                           ("serve", []))}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def run_sharded(args):
    """The step of run_ours with one image sharded over the ranks (weak scaling: rank r holds
    rows 64r .. 64r + 63 of a (64 x world) x 64 random-field image, the same per-GPU work as the
    one-GPU step). Each rank encrypts its band five ways with ichee_encrypt_pixels (ciphertext
    ids = whole-image pixel indices), runs the mean filter on its band with one halo row on each
    side (encrypted by the rank itself), brightness and blend on its band, matching as its partial
    sum + one int64 all-reduce (NCCL) + relinearisation on every rank, and decrypts its results.
    Keys and caches come from the same seeds on every rank (the same bits a broadcast would give).
    `value` = pixel ciphertexts encrypted per second by all ranks together (slowest rank's time)."""
    import torch
    from paper_2409_03568_gb300 import ichee, shard

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = W.ENC8192
    hbm_peak, peak_kind = measured_peaks()
    ctx = ichee.Context(**W.ctx_kwargs(wl), device=local)
    ctx.keygen(2024, with_evk=True)
    h_img, w, c = 64 * world, wl["w"], wl["c"]
    img = inputs.random_field_image(h_img, w, seed=wl["image_seed"], channels=c).reshape(-1)
    wm = inputs.binary_pattern(h_img, w, seed=5).reshape(-1)
    noisy = inputs.noisy_copy(img, seed=6)
    beta = inputs.brightness_beta(4)
    y0, y1 = shard.row_bands(h_img, world)[rank]
    r0, r1 = shard.halo_rows(h_img, y0, y1)
    row = w * c
    n_band, n_halo = (y1 - y0) * row, (r1 - r0) * row
    d_band = torch.from_numpy(img[y0 * row:y1 * row].copy()).cuda()
    d_halo = torch.from_numpy(img[r0 * row:r1 * row].copy()).cuda()
    caches = {
        "radix16": ctx.build_cache(ichee.CACHE_RADIX, 11, radix_base=16, randomize=1),
        "radix10": ctx.build_cache(ichee.CACHE_RADIX, 12, radix_base=10, randomize=1),
        "freq32_pool64": ctx.build_cache(ichee.CACHE_FREQ, 13, top_k=32, pool_size=64,
                                         scan=torch.from_numpy(img).cuda()),
        "full256_pool64": ctx.build_cache(ichee.CACHE_FULL, 14, pool_size=64),
    }
    L, H, st = ctx.L, ctx.handle, ctx.stream()
    ctw = ctx.ct_words(L - 1)
    halo_ct = ctx.empty_cts(n_halo, L - 1)              # the fresh encryption, with the halo rows
    band_fresh = halo_ct[(y0 - r0) * row * ctw:(y1 - r0) * row * ctw]
    m_img = ichee.CtImgMeta(h_img, w, c, L - 1, float(1 << wl["log2_scale"]))
    m_band = ichee.CtImgMeta(y1 - y0, w, c, L - 1, float(1 << wl["log2_scale"]))
    wm_ct = ctx.empty_cts((y1 - y0) * w, L - 1)
    ichee.ichee_encrypt_pixels(H, None, torch.from_numpy(wm[y0 * w:y1 * w].copy()).cuda(), (y1 - y0) * w, y0 * w, 21,
                               wm_ct, st)
    m_wm = ichee.CtImgMeta(y1 - y0, w, 1, L - 1, float(1 << wl["log2_scale"]))
    nz_ct = ctx.empty_cts(n_band, L - 1)
    ichee.ichee_encrypt_pixels(H, None, torch.from_numpy(noisy[y0 * row:y1 * row].copy()).cuda(), n_band, y0 * row, 22,
                               nz_ct, st)
    methods = ["fresh"] + list(caches)
    enc_out = {m: ctx.empty_cts(n_band, L - 1) for m in caches}
    enc_out["fresh"] = band_fresh
    ops_out = {"meanfilter3": ctx.empty_cts(n_band, L - 2), "brightness": ctx.empty_cts(n_band, L - 1),
               "blend": ctx.empty_cts(n_band, L - 2), "match": ctx.empty_cts(1, L - 2)}
    acc = torch.empty(ichee.ichee_sqdiff_acc_words(H, L - 1), dtype=torch.int64, device="cuda")
    dec_out = {k: torch.empty(1 if k == "match" else n_band, dtype=torch.float64, device="cuda")
               for k in methods + list(ops_out)}
    metas = {m: m_band for m in methods}

    def p_encrypt(m):
        def f():
            if m == "fresh":
                ichee.ichee_encrypt_pixels(H, None, d_halo, n_halo, r0 * row, 7, halo_ct, st)
            else:
                ichee.ichee_encrypt_pixels(H, caches[m], d_band, n_band, y0 * row, 7, enc_out[m], st)
        return f

    def p_meanfilter():
        metas["meanfilter3"] = ichee.ichee_meanfilter_rows(H, halo_ct, m_img, r0, r1 - r0, y0, y1,
                                                           ops_out["meanfilter3"], st)

    def p_op(name, op, b=None, mb=None, op_args=()):
        def f():
            metas[name] = ichee.ichee_eval(H, op, band_fresh, m_band, b, mb, op_args, ops_out[name], st)
        return f

    def p_match():
        metas["match"] = shard.sharded_match(ichee, ctx, band_fresh, m_band, nz_ct, m_band, acc, ops_out["match"],
                                             stream=st)

    def p_decrypt():   # one batched decryption per level, as in the one-GPU step
        groups = {}
        for k in methods + list(ops_out):
            groups.setdefault(metas[k].level, []).append(k)
        for ks in groups.values():
            ichee.ichee_decrypt_batch(H, [enc_out[k] if k in enc_out else ops_out[k] for k in ks],
                                      [metas[k] for k in ks], [dec_out[k] for k in ks], st)

    phases = [(m, p_encrypt(m)) for m in methods] + [
        ("meanfilter3", p_meanfilter), ("brightness", p_op("brightness", ichee.OP_BRIGHTNESS, op_args=(beta,))),
        ("blend", p_op("blend", ichee.OP_BLEND, wm_ct, m_wm, (0.9,))), ("match", p_match), ("decrypt", p_decrypt)]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def step():
        for _, fn in phases:
            fn()

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    band_px = img[y0 * row:y1 * row]
    for m in methods:
        err = float(np.abs(dec_out[m].cpu().numpy() - band_px).max())
        if err > 1e-3:
            raise RuntimeError("rank %d: decode error %.3g for %s" % (rank, err, m))
    plain = float(((img.astype(np.float64) - noisy) ** 2).sum())
    match_err = abs(float(dec_out["match"].cpu().numpy()[0]) - plain)
    if match_err > 1.0:
        raise RuntimeError("rank %d: sharded matching decodes %.3g away from the plaintext distance" % (rank, match_err))
    clocks = ClockSampler(local)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    total_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        ev0.record()
        step()
        ev1.record()
        torch.cuda.synchronize()
        total_ms += ev0.elapsed_time(ev1)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms, units_all = reduce_over_ranks(total_ms, len(methods) * n_band * args.steps)
    # end to end: the same step with the band's pixels in pinned host memory (the library copies
    # them in) and every decoded result written to pinned host memory; host wall clock
    h_band = torch.from_numpy(band_px.copy()).pin_memory()
    h_halo = torch.from_numpy(img[r0 * row:r1 * row].copy()).pin_memory()
    h_out = {k: torch.empty(1 if k == "match" else n_band, dtype=torch.float64).pin_memory() for k in dec_out}

    def step_host():
        ichee.ichee_encrypt_pixels(H, None, h_halo, n_halo, r0 * row, 7, halo_ct, st)
        for m in caches:
            ichee.ichee_encrypt_pixels(H, caches[m], h_band, n_band, y0 * row, 7, enc_out[m], st)
        for name, fn in phases[len(methods):-1]:
            fn()
        for k in methods:
            ichee.ichee_decrypt_image_async(H, enc_out[k], metas[k], h_out[k], st)
        for k in ops_out:
            ichee.ichee_decrypt_image_async(H, ops_out[k], metas[k], h_out[k], st)
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step_host()
    tot = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step_host()
        tot += time.perf_counter() - t0
    e2e_ms, e2e_units = reduce_over_ranks(tot * 1e3, len(methods) * n_band * args.steps)
    e2e = {"value": round(e2e_units / (e2e_ms / 1e3), 1), "unit": UNIT,
           "h2d_bytes_per_step": n_halo + len(caches) * n_band,
           "d2h_bytes_per_step": (len(methods) + 3) * n_band * 8 + 8,
           "timing": "host wall clock around each step, slowest rank"}
    out = {
        "metric": METRIC, "value": round(units_all / (total_ms / 1e3), 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64 (RNS residues mod 60/40/60-bit primes)",
        "data": "synthetic (Gaussian random field %dx%d, correlation 6 px, seed 2; stands in for USC-SIPI)" % (h_img, w),
        "config": {"workload": "enc_n8192_l3_64x64_per_gpu_sharded", "N": ctx.n, "primes_bits": wl["prime_bits"],
                   "image": "%dx%dx%d" % (h_img, w, c), "band_rows_per_gpu": y1 - y0, "methods": methods,
                   "ops": list(ops_out), "l2": "flushed (512 MB write) before every step",
                   "parallelism": "pixel rows sharded over %d GPUs; matching all-reduce (int64, NCCL)" % world},
        "gpu_launches": args.steps * (len(methods) + 2 + 3 + 10 + len({metas[k].level for k in methods + list(ops_out)})),
        "match_abs_error": match_err, "clocks": clk, "e2e": e2e}
    if rank == 0:
        print(json.dumps(out))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def extras_ours(args, ctx, ichee, a, ma, b, mb, flush, alu_peak):
    """Operations outside the step, timed the same way (CUDA events on the library's stream,
    L2 flushed before each launch): the per-pixel squared difference (ICHEE_OP_SQDIFF), one
    relinearisation and rescale per pixel of the 64x64 image."""
    import torch
    n, L, logn = ctx.n, ma.level + 1, ctx.n.bit_length() - 1
    n_px = ma.n_ct
    out = ctx.empty_cts(n_px, L - 2)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for _ in range(args.warmup):
        ichee.ichee_eval(ctx.handle, ichee.OP_SQDIFF, a, ma, b, mb, (), out, ctx.stream())
    for e0, e1 in ev:
        flush.zero_()
        e0.record()
        ichee.ichee_eval(ctx.handle, ichee.OP_SQDIFF, a, ma, b, mb, (), out, ctx.stream())
        e1.record()
    torch.cuda.synchronize()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / len(ev)
    # transforms: 2L forward (d) + L inverse (t2) + L^2 forward digits (each digit into the
    # other L - 1 moduli and P; into its own modulus its transform is the tensor's d1^2) +
    # 2(L+1) inverse accumulators; pointwise: tensor with N^{-1} and the d1^2 form 4LN,
    # key-switch MAC 2L(L+1)N, P t folding 2LN, mod-down and rescale 4LN
    n_tr = L * L + 5 * L + 2
    modmul = n_tr * (n // 2) * logn + 4 * L * n + 2 * L * (L + 1) * n + 2 * L * n + 4 * L * n
    ach = n_px * modmul / (ms / 1e3) / 1e9
    return {"sqdiff_image": {"ms": round(ms, 4), "px_per_s": round(n_px / (ms / 1e3), 1), "transforms_per_px": n_tr,
                             "bound": "alu", "achieved": round(ach, 1), "peak": round(alu_peak, 1),
                             "unit": "Gmodmul/s", "frac": round(ach / alu_peak, 4)}}


def e2e_ours(args, ctx, ichee, img, wm_ct, wm_meta, nz_ct, nz_meta, beta, caches, methods, enc_out, ops_out, st, world):
    """Same step through the public entry points with HOST buffers: pixels from pinned host
    memory (the library copies them in), decoded values written by the decryption kernels into
    pinned host memory (ichee_decrypt_image_async), one synchronisation at the end of the step."""
    import torch
    h, w, c = 64, 64, 1
    n_px = img.size
    H = ctx.handle
    host_px = torch.from_numpy(img.copy()).pin_memory()
    host_out = {k: torch.empty(n_px, dtype=torch.float64).pin_memory() for k in methods + list(ops_out)}
    metas = {}

    def step():
        for m in methods:
            metas[m] = ichee.ichee_encrypt_image(H, None if m == "fresh" else caches[m], host_px, h, w, c, 7,
                                                 enc_out[m], st)
        a, ma = enc_out["fresh"], metas["fresh"]
        metas["meanfilter3"] = ichee.ichee_eval(H, ichee.OP_MEANFILTER3, a, ma, None, None, (), ops_out["meanfilter3"], st)
        metas["brightness"] = ichee.ichee_eval(H, ichee.OP_BRIGHTNESS, a, ma, None, None, (beta,), ops_out["brightness"], st)
        metas["blend"] = ichee.ichee_eval(H, ichee.OP_BLEND, a, ma, wm_ct, wm_meta, (0.9,), ops_out["blend"], st)
        metas["match"] = ichee.ichee_eval(H, ichee.OP_SQDIFF_SUM, a, ma, nz_ct, nz_meta, (), ops_out["match"], st)
        for k in methods:
            ichee.ichee_decrypt_image_async(H, enc_out[k], metas[k], host_out[k], st)
        for k in ops_out:
            ichee.ichee_decrypt_image_async(H, ops_out[k], metas[k], host_out[k], st)
        torch.cuda.synchronize()

    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        flush.zero_()
        step()
    tot = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step()
        tot += time.perf_counter() - t0
    tot_ms, units = reduce_over_ranks(tot * 1e3, len(methods) * n_px * args.steps)
    tot = tot_ms / 1e3
    # the values that came back to the host decode the image (every encryption method)
    err = max(float(np.max(np.abs(host_out[m].numpy() - img.reshape(-1)))) for m in methods)
    return {"value": round(units / tot, 1), "unit": UNIT, "h2d_bytes_per_step": len(methods) * n_px,
            "d2h_bytes_per_step": (len(methods) + 3) * n_px * 8 + 8,
            "ms_per_step": round(tot / args.steps * 1e3, 3), "timing": "host wall clock around each step",
            "max_decode_error": err}


# ---------------------------------------------------------------------------------------
# CPU oracle leg (baseline / reference arm)
# ---------------------------------------------------------------------------------------
def oracle_step_setup(sample):
    from oracle import Oracle, Params
    wl = W.ENC8192
    o = Oracle(Params(wl["log_n"], wl["prime_bits"], wl["log2_scale"], wl["special_bits"])).keygen(2024, with_evk=True)
    img = W.image_for(wl).reshape(-1)
    idx = np.sort(np.random.default_rng(0).choice(img.size, sample, replace=False)).astype(np.uint64)
    caches = {"radix16": o.radix_cache(16, 11), "radix10": o.radix_cache(10, 12),
              "freq32_pool64": o.freq_cache(img, 32, 64, 13), "full256_pool64": o.full_cache(64, 14)}
    wm = inputs.binary_pattern(64, 64, seed=5).reshape(-1)
    noisy = inputs.noisy_copy(img, seed=6)
    return o, img, idx, caches, wm, noisy


def oracle_step(o, img, idx, caches, wm, noisy, keep=None):
    """The step of the GPU arm restricted to the sampled pixels (ops on a 3x3-neighbourhood
    patch per sampled pixel are replaced by the same ops on the sampled ciphertexts). With
    `keep` (a dict), the per-ciphertext results are left in it: the five encryptions,
    brightness and blend of the sampled pixels."""
    px = img[idx.astype(np.int64)]
    outs = {"fresh": o.encrypt_pixels(px, 7, ids=idx)}
    outs["radix16"] = o.encrypt_radix(px, caches["radix16"], 7, ids=idx)
    outs["radix10"] = o.encrypt_radix(px, caches["radix10"], 7, ids=idx)
    outs["freq32_pool64"] = o.encrypt_lookup(px, caches["freq32_pool64"], 7, ids=idx)
    outs["full256_pool64"] = o.encrypt_lookup(px, caches["full256_pool64"], 7, ids=idx)
    fr = outs["fresh"]
    k = len(idx)
    side = int(np.sqrt(k))
    mf, sc_mf = o.meanfilter3(fr[:side * side], o.delta, side, side, 1)
    br, sc_br = o.brightness(fr, o.delta, inputs.brightness_beta(4))   # the GPU arm's beta
    wct = o.encrypt_pixels(wm[idx.astype(np.int64)], 21, ids=idx)
    bl, sc_bl = o.blend(fr, wct, o.delta, 0.9, 1, 1)
    nct = o.encrypt_pixels(noisy[idx.astype(np.int64)], 22, ids=idx)
    mt, sc_mt = o.match(fr, nct, o.delta)
    for m in outs:
        o.decrypt(outs[m], o.delta)
    o.decrypt(mf, sc_mf)
    o.decrypt(br, sc_br)
    o.decrypt(bl, sc_bl)
    o.decrypt(mt, sc_mt)
    if keep is not None:
        keep.update(outs)
        keep["brightness"], keep["blend"] = br, bl
    return 5 * k


def cpu_baseline(sample_steps=1, sample=36, keep=None):
    """The oracle timed on the host cores; with `keep`, its per-ciphertext results of the last
    step and the sampled indices (`keep["idx"]`) are left for a parity check."""
    from oracle.ckks import lib as olib
    setup = oracle_step_setup(sample)
    t0 = time.perf_counter()
    units = 0
    for _ in range(sample_steps):
        units += oracle_step(*setup, keep=keep)
    dt = time.perf_counter() - t0
    if keep is not None:
        keep["idx"] = setup[2]
    return {"value": round(units / dt, 3), "unit": UNIT, "cores": int(olib().orc_num_threads()), "kind": "oracle",
            "sample": "%d of the 4096 pixels per method (5 methods), ops on those ciphertexts (mean filter on a "
                      "%dx%d patch), decryption; %d step(s), %.1f s" % (sample, int(np.sqrt(sample)),
                                                                      int(np.sqrt(sample)), sample_steps, dt)}


def parity_on_sample(ctx, enc_out, ops_out, ref, n_check=64):
    """Ciphertexts of the bench run against the oracle's, on the first n_check sampled pixels:
    the five encryptions, brightness and blend, word for word."""
    import torch
    idx = torch.from_numpy(ref["idx"][:n_check].astype(np.int64))
    mismatched, checked = [], []
    for name in list(enc_out) + ["brightness", "blend"]:
        t = enc_out[name] if name in enc_out else ops_out[name]
        want = ref[name][:n_check]
        rows = t.view(-1, want[0].size).index_select(0, idx.to(t.device)).cpu().numpy().view(np.uint64)
        checked.append(name)
        if not np.array_equal(rows.reshape(want.shape), want):
            mismatched.append(name)
    return {"pixels": int(len(idx)), "results": checked, "bit_exact": not mismatched, "mismatched": mismatched}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    sample = 256
    setup = oracle_step_setup(sample)
    for _ in range(args.warmup):
        oracle_step(*setup)
    t0 = time.perf_counter()
    units = 0
    for _ in range(args.steps):
        units += oracle_step(*setup)
    dt = time.perf_counter() - t0
    from oracle.ckks import lib as olib
    v = units / dt
    cb = {"value": round(v, 3), "unit": UNIT, "cores": int(olib().orc_num_threads()), "kind": "oracle",
          "sample": "%d of the 4096 pixels per method per step, ops on those ciphertexts, decryption" % sample}
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": UNIT, "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                      "dtype": "u64 (RNS residues)", "data": "synthetic",
                      "config": {"workload": W.ENC8192["name"], "sample_pixels_per_method": sample},
                      "cpu_baseline": cb,
                      "e2e": {"value": round(v, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def sub_record(workload, extra, timeout=900):
    """Run `bench.py --workload <workload>` in a child process and return its JSON line (or the
    failure) as a sub-record."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--workload", workload] + extra
    t0 = time.perf_counter()
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout)
    except subprocess.TimeoutExpired:
        return {"error": "timed out after %d s" % timeout}
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    if r.returncode != 0 or not lines:
        return {"error": "exit %d" % r.returncode, "stderr_tail": r.stderr[-600:]}
    rec = json.loads(lines[-1])
    rec["wall_s"] = round(time.perf_counter() - t0, 1)
    return rec


# ---------------------------------------------------------------------------------------
# image operations on the 128x128x3 image at N = 8192, four primes
# ---------------------------------------------------------------------------------------
def run_ops128(args):
    """The image operations of Sec. 4.4 on the 128x128x3 random-field image (N = 8192, primes
    60/40/40/40, Delta = 2^40): 3x3 mean filter, brightness +beta (copy), watermark blend with an
    encrypted binary 128x128 pattern (alpha 0.9), matching against an encrypted noisy copy (sum of
    squared differences, relinearised), each result decrypted. One step = the four operations and
    the four decryptions; every operation is also timed on its own (CUDA events on the library's
    stream). Inputs (tens of GB) are far larger than L2."""
    import torch
    from paper_2409_03568_gb300 import ichee
    wl = W.OPS8192
    torch.cuda.set_device(0)
    hbm_peak, peak_kind = measured_peaks()
    ctx = ichee.Context(**W.ctx_kwargs(wl))
    ctx.keygen(2025, with_evk=True)
    h, w, c = wl["h"], wl["w"], wl["c"]
    n_px = h * w * c
    img = W.image_for(wl).reshape(-1)
    noisy = inputs.noisy_copy(img, seed=wl["noisy_seed"])
    wm = inputs.binary_pattern(h, w, seed=wl["watermark_seed"]).reshape(-1)
    beta = inputs.brightness_beta(wl["beta_seed"])
    a, ma = ctx.encrypt(torch.from_numpy(img).cuda(), h, w, c, 31)
    b, mb = ctx.encrypt(torch.from_numpy(noisy).cuda(), h, w, c, 32)
    wct, mw = ctx.encrypt(torch.from_numpy(wm).cuda(), h, w, 1, 33)
    L = ctx.L
    outs = {"meanfilter3": ctx.empty_cts(n_px, L - 2), "brightness": ctx.empty_cts(n_px, L - 1),
            "blend": ctx.empty_cts(n_px, L - 2), "match": ctx.empty_cts(1, L - 2)}
    dec = {k: torch.empty(1 if k == "match" else n_px, dtype=torch.float64, device="cuda") for k in outs}
    st, H = ctx.stream(), ctx.handle
    metas = {}
    ops = {"meanfilter3": (ichee.OP_MEANFILTER3, None, None, ()),
           "brightness": (ichee.OP_BRIGHTNESS, None, None, (beta,)),
           "blend": (ichee.OP_BLEND, wct, mw, (wl["alpha"],)),
           "match": (ichee.OP_SQDIFF_SUM, b, mb, ())}

    def op(name):
        o, x, mx, arg = ops[name]
        metas[name] = ichee.ichee_eval(H, o, a, ma, x, mx, arg, outs[name], st)

    def decrypt_all():
        for k in outs:
            ichee.ichee_decrypt_image(H, outs[k], metas[k], dec[k], st)

    names = list(ops)
    ev = {k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for k in names + ["decrypt"]}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = {k: 0.0 for k in ev}
    total = 0.0
    clocks = ClockSampler(0)
    clocks.start()
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        e0.record()
        for k in names:
            ev[k][0].record()
            op(k)
            ev[k][1].record()
        ev["decrypt"][0].record()
        decrypt_all()
        ev["decrypt"][1].record()
        e1.record()
        torch.cuda.synchronize()
        if i >= args.warmup:
            total += e0.elapsed_time(e1)
            for k in ev:
                ms[k] += ev[k][0].elapsed_time(ev[k][1])
    clk = clocks.stop()
    ms = {k: v / args.steps for k, v in ms.items()}
    step_ms = total / args.steps
    # correctness guard and quality against FP64 plaintext references of the operations
    f = img.reshape(h, w, c).astype(np.float64)
    pad = np.pad(f, ((1, 1), (1, 1), (0, 0)), mode="edge")
    box = sum(pad[dy:dy + h, dx:dx + w] for dy in range(3) for dx in range(3)) / 9.0
    wmf = wm.reshape(h, w, 1).astype(np.float64)
    refs = {"meanfilter3": box.reshape(-1), "brightness": img.astype(np.float64) + beta,
            "blend": (wl["alpha"] * f + (1 - wl["alpha"]) * wmf).reshape(-1),
            "match": np.array([float(((img.astype(np.float64) - noisy) ** 2).sum())])}
    errors = {k: float(np.max(np.abs(dec[k].cpu().numpy() - refs[k]))) for k in names}
    for k, tol in (("meanfilter3", 1e-2), ("brightness", 1e-3), ("blend", 1e-2), ("match", 5.0)):
        if errors[k] > tol:
            raise RuntimeError("ops128: %s decodes %.3g away from its plaintext reference" % (k, errors[k]))
    n, logn = ctx.n, wl["log_n"]
    ct_in, ct_out = 2 * L * n * 8, 2 * (L - 1) * n * 8
    alu_peak = SM_COUNT * SM_MAX_MHZ * 1e6 * IMAD_PER_SM_CLK / IMAD_PER_MODMUL / 1e9
    bytes_of = {"meanfilter3": n_px * (ct_in + ct_out), "brightness": n_px * 2 * ct_in,
                "blend": n_px * (ct_in + ct_out) + h * w * ct_in}
    per_op = {}
    for k in names:
        t = ms[k] / 1e3
        rec = {"ms": round(ms[k], 4), "px_per_s": round(n_px / t, 1)}
        if k in bytes_of:
            ach = bytes_of[k] / t / 1e9
            rec.update({"bound": "hbm", "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
                        "frac": round(ach / hbm_peak, 4), "bytes": bytes_of[k]})
        else:
            mm = n_px * L * (2 * (n // 2) * logn + 3 * n)
            ach = mm / t / 1e9
            rec.update({"bound": "alu", "achieved": round(ach, 1), "peak": round(alu_peak, 1), "unit": "Gmodmul/s",
                        "frac": round(ach / alu_peak, 4)})
        rec["max_abs_error"] = errors[k]
        per_op[k] = rec
    dec_bytes = n_px * (L - 1) * n * 8 * 2 + n_px * L * n * 8 + (L - 1) * n * 8
    per_op["decrypt"] = {"ms": round(ms["decrypt"], 4), "bound": "hbm",
                         "frac": round(dec_bytes / (ms["decrypt"] / 1e3) / 1e9 / hbm_peak, 4)}
    print(json.dumps({
        "metric": "image-operation pixels/s, N=8192, 4 primes, 128x128x3 (mean filter, brightness, blend, matching "
                  "and their decryption per step)",
        "value": round(4 * n_px / (step_ms / 1e3), 1), "unit": "px-op/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64 (RNS residues mod 60/40/40/40-bit primes)",
        "data": "synthetic (128x128x3 random field seed 3, beta seed 4, pattern seed 5, noisy copy seed 6)",
        "config": {"workload": wl["name"], "N": n, "primes_bits": wl["prime_bits"], "image": "%dx%dx%d" % (h, w, c),
                   "l2": "inputs (%.0f GB) far larger than L2" % ((2 * n_px + h * w) * ct_in / 1e9),
                   "peak_kind": peak_kind},
        "ops": per_op, "clocks": clk}))
    ctx.close()


# ---------------------------------------------------------------------------------------
# ragged batch under one CUDA graph vs per-image launches
# ---------------------------------------------------------------------------------------
def run_batch(args):
    import ctypes
    import torch
    from paper_2409_03568_gb300 import ichee

    wl = W.BATCH32
    torch.cuda.set_device(0)
    hbm_peak, peak_kind = measured_peaks()
    ctx = ichee.Context(**W.ctx_kwargs(wl))
    ctx.keygen(77)
    cache = ctx.build_cache(ichee.CACHE_RADIX, 15, radix_base=wl["radix_base"], randomize=1)
    imgs = inputs.ragged_batch(wl["n_images"], wl["batch_seed"], wl["side_lo"], wl["side_hi"])
    shapes = [(im.shape[0], im.shape[1], 1) for im in imgs]
    seeds = [500 + i for i in range(len(imgs))]
    n_px = sum(h * w * c for h, w, c in shapes)
    d_px = [torch.from_numpy(im.reshape(-1).copy()).cuda() for im in imgs]
    enc = [ctx.empty_cts(h * w * c, 2) for h, w, c in shapes]
    filt = [ctx.empty_cts(h * w * c, 1) for h, w, c in shapes]
    H = ctx.handle
    st_main = torch.cuda.current_stream()
    sp_main = ctypes.c_void_p(st_main.cuda_stream)
    metas = [None] * len(shapes)

    def plain():
        for i, (h, w, c) in enumerate(shapes):
            metas[i] = ichee.ichee_encrypt_image(H, cache, d_px[i], h, w, c, seeds[i], enc[i], sp_main)
            ichee.ichee_eval(H, ichee.OP_MEANFILTER3, enc[i], metas[i], None, None, (), filt[i], sp_main)

    tune = ichee.ichee_autotune_batch(H, cache, d_px, shapes, seeds, enc, filt, sp_main)
    shapes_used = {"radix": ichee.ichee_tuned_shape(H, ichee.TUNE_RADIX),
                   "meanfilter": ichee.ichee_tuned_shape(H, ichee.TUNE_MEANFILTER)}
    cap = torch.cuda.Stream()
    sp_cap = ctypes.c_void_p(cap.cuda_stream)
    torch.cuda.synchronize()
    ichee.ichee_graph_begin(H, sp_cap)
    bm = ichee.ichee_encrypt_batch(H, cache, d_px, shapes, seeds, enc, sp_cap)
    ichee.ichee_eval_batch(H, ichee.OP_MEANFILTER3, enc, bm, outs=filt, stream=sp_cap)
    graph = ichee.ichee_graph_end(H, sp_cap)
    ichee.ichee_graph_begin(H, sp_cap)
    ichee.ichee_encrypt_meanfilter_batch(H, cache, d_px, shapes, seeds, enc, filt, sp_cap)
    graph_fused = ichee.ichee_graph_end(H, sp_cap)
    shapes_used["fused"] = ichee.ichee_tuned_shape(H, ichee.TUNE_FUSED)
    schedule = "fused kernel" if ichee.ichee_tuned_shape(H, ichee.TUNE_SCHEDULE)[0] == 1 else "two batched kernels"
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(args.steps):
            torch.cuda.synchronize()
            e0.record(st_main)
            fn()
            e1.record(st_main)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / args.steps

    clocks = ClockSampler(0)
    clocks.start()
    ms_plain = timed(plain)
    ref = [f.clone() for f in filt[:3]]
    ms_graph2 = timed(lambda: ichee.ichee_graph_launch(graph, sp_main))
    same2 = all(torch.equal(a, b) for a, b in zip(ref, filt[:3]))
    ms_graph = timed(lambda: ichee.ichee_graph_launch(graph_fused, sp_main))
    clk = clocks.stop()
    torch.cuda.synchronize()
    same = same2 and all(torch.equal(a, b) for a, b in zip(ref, filt[:3]))
    ct3, ct2 = 2 * 3 * ctx.n * 8, 2 * 2 * ctx.n * 8
    # algorithmic HBM bytes: encryption written once and the filtered image written; the two-kernel
    # schedule also reads the encryption back
    fused = schedule == "fused kernel"
    bytes_step = n_px * (ct3 + ct2 + (0 if fused else ct3))
    achieved = bytes_step / (ms_graph / 1e3) / 1e9
    out = {"metric": "pixel ciphertexts/s, radix-16 encryption + 3x3 mean filter over a ragged batch of 32 images "
                     "(persistent batched kernels, tuned schedule, one CUDA graph)",
           "value": round(n_px / (ms_graph / 1e3), 1), "unit": "px/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_graph, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u64 (RNS residues mod 60/40/60-bit primes)",
           "data": "synthetic (32 random fields, sides U{16..128}, seed 7)",
           "config": {"workload": wl["name"], "pixels": n_px, "images": len(shapes),
                      "ciphertext_gb": round(n_px * (ct3 + ct2) / 1e9, 1),
                      "l2": "working set (%.0f GB) far above L2" % (n_px * (ct3 + ct2) / 1e9)},
           "plain_per_image": {"ms_per_step": round(ms_plain, 4), "px_per_s": round(n_px / (ms_plain / 1e3), 1),
                               "launches": 2 * len(shapes)},
           "graph_two_kernels": {"ms_per_step": round(ms_graph2, 4), "px_per_s": round(n_px / (ms_graph2 / 1e3), 1)},
           "tuned_schedule": schedule,
           "graph_speedup": round(ms_plain / ms_graph, 3), "graph_equals_plain": same,
           "tuned_shapes": {k: {"threads": v[0], "blocks_per_sm": v[1]} for k, v in shapes_used.items()},
           "tuner_report": [{"kind": k, "threads": t, "blocks_per_sm": b, "ms": round(m, 4)} for k, t, b, m in tune],
           "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                        "frac": round(achieved / hbm_peak, 4), "traffic": None,
                        "kernel": "ichee_encrypt_meanfilter_batch (tuned schedule, one graph)",
                        "algorithmic_bytes_per_px": ct3 + ct2 + (0 if fused else ct3),
                        "peak_kind": peak_kind},
           "clocks": clk}
    print(json.dumps(out))
    ichee.ichee_graph_destroy(graph)
    ichee.ichee_graph_destroy(graph_fused)
    ctx.close()


# ---------------------------------------------------------------------------------------
# serving: Poisson request stream through the continuous-batching server
# ---------------------------------------------------------------------------------------
def serve_requests(wl, duration):
    """The seeded request stream: arrival times and request parameters (no pixels yet)."""
    rng = np.random.default_rng(wl["seed"])
    t, reqs = 0.0, []
    w = np.array(wl["op_weights"], dtype=np.float64)
    while True:
        t += rng.exponential(1.0 / wl["rate"])
        if t >= duration:
            break
        side = int(rng.integers(wl["side_lo"], wl["side_hi"] + 1))
        reqs.append(dict(t=t, kind=int(rng.choice(5, p=w / w.sum())), ring=int(rng.integers(0, 2)), h=side, w=side,
                         c=int(rng.choice([1, 3])), seed=10_000 + 3 * len(reqs)))
    return reqs


def serve_algorithmic_bytes(wl, reqs, served):
    """HBM bytes the served requests need at least: every encryption written once, every
    operation's inputs read and output written once (brightness in place touches one word per
    limb), every decryption reads c1 and coefficient 0 of c0 (half a ciphertext)."""
    total = 0
    for q, ok in zip(reqs, served):
        if not ok:
            continue
        ring = wl["rings"][q["ring"]]
        n, L = 1 << ring["log_n"], len(ring["prime_bits"])
        ct, ct1 = 2 * L * n * 8, 2 * (L - 1) * n * 8
        npx = q["h"] * q["w"] * q["c"]
        nb = q["h"] * q["w"] if q["kind"] == 3 else (npx if q["kind"] == 4 else 0)
        total += (npx + nb) * ct
        if q["kind"] == 1:
            total += npx * (ct + ct1) + npx * ct1 // 2
        elif q["kind"] == 3:
            total += npx * (ct + ct1) + nb * ct + npx * ct1 // 2
        elif q["kind"] == 4:
            total += 2 * npx * ct
        else:   # encrypt-only, brightness
            total += npx * ct // 2
    return total


def run_serve(args):
    import threading
    import torch
    from paper_2409_03568_gb300 import ichee

    wl = W.SERVE
    duration = args.duration if args.duration else wl["duration_s"]
    torch.cuda.set_device(0)
    ctxs, caches = [], []
    for i, r in enumerate(wl["rings"]):
        ctx = ichee.Context(**r)
        ctx.keygen(31 + i, with_evk=True)
        ctxs.append(ctx)
        caches.append(ctx.build_cache(ichee.CACHE_FULL, 41 + i, pool_size=64))
    reqs = serve_requests(wl, duration)
    bank = {}
    for q in reqs:   # pixels drawn per request (seeded)
        img = inputs.random_field_image(q["h"], q["w"], seed=q["seed"], channels=q["c"]).reshape(-1).copy()
        two = None
        if q["kind"] == ichee.REQ_WATERMARK:
            two = inputs.binary_pattern(q["h"], q["w"], seed=q["seed"] + 1).reshape(-1).copy()
        elif q["kind"] == ichee.REQ_MATCH:
            two = inputs.noisy_copy(img, seed=q["seed"] + 2)
        n_res = 1 if q["kind"] == ichee.REQ_MATCH else img.size
        bank[id(q)] = (img, two, np.zeros(n_res, dtype=np.float64))
    px_total = sum(q["h"] * q["w"] * q["c"] for q in reqs)
    args_of = {ichee.REQ_BRIGHTNESS: 25.0, ichee.REQ_WATERMARK: 0.9}
    # warm the matching scratch and first-launch paths outside the measurement
    for ring in range(2):
        ctx = ctxs[ring]
        a, ma = ctx.encrypt(torch.zeros(4, dtype=torch.uint8, device="cuda"), 2, 2, 1, 1, cache=caches[ring])
        ctx.eval(ichee.OP_SQDIFF_SUM, a, ma, a, ma, out_n_ct=1, out_level=ma.level - 1)
    torch.cuda.synchronize()
    server = ichee.ichee_server_create([c.handle for c in ctxs], caches, int(wl["budget_gb"] * 1e9))
    tickets = [None] * len(reqs)
    structs = []
    t0 = time.perf_counter() + 0.5

    def submitter():
        for i, q in enumerate(reqs):
            img, two, res = bank[id(q)]
            r = ichee.Request()
            r.kind, r.ring, r.h, r.w, r.c, r.seed = q["kind"], q["ring"], q["h"], q["w"], q["c"], q["seed"]
            r.pixels = img.ctypes.data
            r.pixels2 = two.ctypes.data if two is not None else None
            r.arg = args_of.get(q["kind"], 0.0)
            r.result = res.ctypes.data
            r.ct_out = None
            structs.append(r)
            delay = t0 + q["t"] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            try:
                tickets[i] = ichee.ichee_server_submit(server, r)
            except ichee.IcheeError:
                tickets[i] = -1   # refused at admission control (larger than the HBM budget)

    clocks = ClockSampler(0)
    clocks.start()
    th = threading.Thread(target=submitter)
    th.start()
    lat, rounds, first_sub, last_done = [], [], None, 0.0
    refused = 0
    served_px = 0
    deadline = time.perf_counter() + duration + 600.0
    for i in range(len(reqs)):
        while tickets[i] is None:
            if time.perf_counter() > deadline:
                raise RuntimeError("serving run exceeded its time cap")
            time.sleep(0.0005)
        if tickets[i] < 0:
            refused += 1
            continue
        d = ichee.ichee_server_wait(server, tickets[i], int(max(1.0, deadline - time.perf_counter()) * 1e3))
        served_px += reqs[i]["h"] * reqs[i]["w"] * reqs[i]["c"]
        lat.append(d.t_done - d.t_submit)
        rounds.append(d.round_size)
        first_sub = d.t_submit if first_sub is None else min(first_sub, d.t_submit)
        last_done = max(last_done, d.t_done)
    th.join()
    clk = clocks.stop()
    stats = ichee.ichee_server_stats_get(server)
    ichee.ichee_server_destroy(server)
    # every encrypt-only result decodes to its pixels
    worst = max(float(np.max(np.abs(bank[id(q)][2] - bank[id(q)][0]))) for q, t in zip(reqs, tickets)
                if q["kind"] == ichee.REQ_ENCRYPT and t is not None and t >= 0)
    span = last_done - first_sub
    lat = np.array(lat)
    alg_bytes = serve_algorithmic_bytes(wl, reqs, [t is not None and t >= 0 for t in tickets])
    hbm_peak, peak_kind = measured_peaks()

    # the unbatched plain path: the same arrivals, one request at a time through the
    # single-request entry points, on a prefix of the stream (at most 20 s of arrivals or 60 s)
    plain_lat, plain_px = [], 0
    tp0 = time.perf_counter()
    for q in reqs:
        if q["t"] > min(20.0, duration) or time.perf_counter() - tp0 > 60.0:
            break
        wait = tp0 + q["t"] - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        if q["kind"] == ichee.REQ_MATCH and q["ring"] == 1 and q["h"] * q["w"] * q["c"] > 45000:
            continue   # one unbatched call would hold both images (over 110 GB); the server tiles it
        img, two, _ = bank[id(q)]
        ctx, cache = ctxs[q["ring"]], caches[q["ring"]]
        a, ma = ctx.encrypt(torch.from_numpy(img).cuda(), q["h"], q["w"], q["c"], q["seed"], cache=cache)
        if q["kind"] == ichee.REQ_MEANFILTER:
            a, ma = ctx.eval(ichee.OP_MEANFILTER3, a, ma, out_level=ma.level - 1)
        elif q["kind"] == ichee.REQ_BRIGHTNESS:
            a, ma = ctx.eval(ichee.OP_BRIGHTNESS, a, ma, args=(25.0,))
        elif q["kind"] == ichee.REQ_WATERMARK:
            b, mb = ctx.encrypt(torch.from_numpy(two).cuda(), q["h"], q["w"], 1, q["seed"] + 1, cache=cache)
            a, ma = ctx.eval(ichee.OP_BLEND, a, ma, b, mb, args=(0.9,), out_level=ma.level - 1)
        elif q["kind"] == ichee.REQ_MATCH:
            b, mb = ctx.encrypt(torch.from_numpy(two).cuda(), q["h"], q["w"], q["c"], q["seed"] + 1, cache=cache)
            a, ma = ctx.eval(ichee.OP_SQDIFF_SUM, a, ma, b, mb, out_n_ct=1, out_level=ma.level - 1)
        ctx.decrypt(a, ma).cpu()
        plain_lat.append(time.perf_counter() - (tp0 + q["t"]))
        plain_px += q["h"] * q["w"] * q["c"]
    plain_span = time.perf_counter() - tp0
    plain_lat = np.array(plain_lat)
    out = {"metric": "served pixels/s, continuous batching of a Poisson request stream (200 req/s, mixed ops, "
                     "N=8192/16384)",
           "value": round(served_px / span, 1), "unit": "px/s", "n_gpus": 1, "steps": 1, "warmup": 1,
           "ms_per_step": round(span * 1e3, 1), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "u64 (RNS residues)", "data": "synthetic (seeded request stream and random-field images, seed 8)",
           "config": {"workload": wl["name"], "requests": len(reqs), "duration_s": duration, "pixels": px_total,
                      "offered_px_per_s": round(px_total / duration, 1), "budget_gb": wl["budget_gb"],
                      "refused_over_budget": refused},
           "served_px": served_px, "served_over_offered": round((served_px / span) / (px_total / duration), 4),
           "roofline": {"bound": "hbm", "achieved": round(alg_bytes / span / 1e9, 1), "peak": hbm_peak, "unit": "GB/s",
                        "frac": round(alg_bytes / span / 1e9 / hbm_peak, 4), "traffic": None,
                        "algorithmic_bytes": alg_bytes, "peak_kind": peak_kind,
                        "kernel": "all kernels of the served mix over the span (first submit to last completion)"},
           "latency_s": {"p50": round(float(np.percentile(lat, 50)), 5), "p99": round(float(np.percentile(lat, 99)), 5),
                         "max": round(float(lat.max()), 5)},
           "round_size": {"mean": round(float(np.mean(rounds)), 2), "max": int(np.max(rounds))},
           "server": stats, "max_decode_error_encrypt": worst,
           "plain_unbatched": {"requests": len(plain_lat), "px_per_s": round(plain_px / plain_span, 1),
                               "p50": round(float(np.percentile(plain_lat, 50)), 5) if len(plain_lat) else None,
                               "p99": round(float(np.percentile(plain_lat, 99)), 5) if len(plain_lat) else None,
                               "window_s": round(plain_span, 2)},
           "clocks": clk}
    print(json.dumps(out))
    for c in ctxs:
        c.close()


SINGLE_OPS = ("fresh", "radix16", "full256_pool64", "meanfilter3", "brightness", "blend", "match", "sqdiff_image",
              "decrypt", "radix16_meanfilter3_fused", "radix16_meanfilter3_two_kernels", "match_n16384")


def run_single_op(args):
    """One operation of the 64x64, N = 8192 workload (match_n16384: matching on a 32x32 image at
    N = 16384 with five primes, the serving ring; 2.7 GB of inputs), launched warmup + steps times (L2 flushed
    before each launch, CUDA events on the library's stream). Prints its mean time."""
    import torch
    from paper_2409_03568_gb300 import ichee
    wl = W.ENC8192 if args.op != "match_n16384" else dict(W.RING16384, h=32, w=32, c=1, image_seed=2)
    ctx = ichee.Context(**W.ctx_kwargs(wl))
    ctx.keygen(2024, with_evk=True)
    h, w, c = wl["h"], wl["w"], wl["c"]
    img = W.image_for(wl).reshape(-1)
    d_img = torch.from_numpy(img).cuda()
    a, ma = ctx.encrypt(d_img, h, w, c, 7)
    b = mb = wm = mw = None   # second operands only where the operation takes one
    if args.op in ("match", "sqdiff_image", "match_n16384"):
        b, mb = ctx.encrypt(torch.from_numpy(inputs.noisy_copy(img, seed=6)).cuda(), h, w, c, 22)
    if args.op == "blend":
        wm, mw = ctx.encrypt(torch.from_numpy(inputs.binary_pattern(h, w, seed=5).reshape(-1)).cuda(), h, w, 1, 21)
    st, H, L = ctx.stream(), ctx.handle, ctx.L
    cache = None
    pipeline = args.op.startswith("radix16_meanfilter3")
    if args.op == "radix16" or pipeline:
        cache = ctx.build_cache(ichee.CACHE_RADIX, 11, radix_base=16, randomize=1)
    if pipeline:   # ichee_encrypt_meanfilter_batch on the one image, with the schedule pinned
        ichee.ichee_set_tuned_shape(ctx.handle, ichee.TUNE_SCHEDULE, 1 if args.op.endswith("fused") else 0)
    elif args.op == "full256_pool64":
        cache = ctx.build_cache(ichee.CACHE_FULL, 14, pool_size=64)
    enc = ctx.empty_cts(h * w * c, L - 1) if args.op in ("fresh", "radix16", "full256_pool64", "brightness") or pipeline \
        else None
    out = ctx.empty_cts(h * w * c if not args.op.startswith("match") else 1, L - 2)
    dec = torch.empty(h * w * c, dtype=torch.float64, device="cuda")
    ops = {"meanfilter3": (ichee.OP_MEANFILTER3, None, None, ()), "brightness": (ichee.OP_BRIGHTNESS, None, None, (7.5,)),
           "blend": (ichee.OP_BLEND, wm, mw, (0.9,)), "match": (ichee.OP_SQDIFF_SUM, b, mb, ()),
           "match_n16384": (ichee.OP_SQDIFF_SUM, b, mb, ()),
           "sqdiff_image": (ichee.OP_SQDIFF, b, mb, ())}

    def once():
        if pipeline:
            ichee.ichee_encrypt_meanfilter_batch(H, cache, [d_img], [(h, w, c)], [7], [enc], [out], st)
        elif args.op in ("fresh", "radix16", "full256_pool64"):
            ichee.ichee_encrypt_image(H, cache, d_img, h, w, c, 7, enc, st)
        elif args.op == "decrypt":
            ichee.ichee_decrypt_image(H, a, ma, dec, st)
        else:
            op, x, mx, arg = ops[args.op]
            ichee.ichee_eval(H, op, a, ma, x, mx, arg, enc if op == ichee.OP_BRIGHTNESS else out, st)

    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        flush.zero_()
        once()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for e0, e1 in ev:
        flush.zero_()
        e0.record()
        once()
        e1.record()
    torch.cuda.synchronize()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / len(ev)
    print(json.dumps({"op": args.op, "workload": wl["name"], "steps": args.steps, "warmup": args.warmup,
                      "ms": round(ms, 4), "px_per_s": round(h * w * c / (ms / 1e3), 1)}))
    ctx.close()


def main():
    args = parse()
    if args.op:
        run_single_op(args)
        return
    if args.impl == "ours" and args.workload == "serve":
        run_serve(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch32":
        run_batch(args)
    elif args.workload == "ops128":
        run_ops128(args)
    elif args.workload == "shard" or dist_env()[1] > 1:
        run_sharded(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
