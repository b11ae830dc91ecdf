"""Pixel sharding over CPU ranks (gloo, world size 2): the row bands cover the image once, and
the all-reduce of the ranks' partial matching sums (Sec. 4.4.3) equals the whole image's sum
word for word once reduced. The partial sums here are the CPU oracle's (coefficient domain);
the library's accumulators are another linear representation of the same sums, added by the
same collective (the GPU side of the split is tested in test_gpu_pieces.py)."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2409_03568_gb300 import shard  # noqa: E402


def test_row_bands_cover_each_row_once():
    for h in (0, 1, 2, 7, 64, 129):
        for world in (1, 2, 3, 8):
            bands = shard.row_bands(h, world)
            assert len(bands) == world
            rows = [y for y0, y1 in bands for y in range(y0, y1)]
            assert rows == list(range(h))
            sizes = [y1 - y0 for y0, y1 in bands]
            assert max(sizes) - min(sizes) <= 1
    assert shard.halo_rows(10, 0, 4) == (0, 5)
    assert shard.halo_rows(10, 4, 7) == (3, 8)
    assert shard.halo_rows(10, 7, 10) == (6, 10)
    with pytest.raises(ValueError):
        shard.row_bands(4, 0)


def test_worst_case_sum_fits_int64():
    """Eight accumulators of the largest residue of a 60-bit prime stay below 2^63."""
    q = (1 << 60) - 1
    assert shard.MAX_RANKS * (q - 1) < (1 << 63)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import Oracle, Params
        from paper_2409_03568_gb300 import inputs
        o = Oracle(Params(6, [60, 40, 60], 40, 61)).keygen(5, with_evk=True)
        h, w, c = 7, 3, 2
        img = inputs.random_field_image(h, w, seed=3, channels=c).reshape(-1)
        other = inputs.noisy_copy(img, seed=4)
        y0, y1 = shard.row_bands(h, world)[rank]
        lo, hi = y0 * w * c, y1 * w * c
        ids = np.arange(lo, hi, dtype=np.uint64)
        part = o.sqdiff_sum_raw(o.encrypt_pixels(img[lo:hi], 11, ids=ids), o.encrypt_pixels(other[lo:hi], 12, ids=ids))
        acc = torch.from_numpy(part.reshape(-1).view(np.int64).copy())
        shard.allreduce_accumulator(acc)
        total = acc.numpy().view(np.uint64).reshape(part.shape)
        q = o.q.astype(np.uint64)
        reduced = total % q[None, :, None]
        full = o.sqdiff_sum_raw(o.encrypt_pixels(img, 11), o.encrypt_pixels(other, 12))
        # and the match result of the summed tensor decodes to the plaintext distance
        rel = o.rescale(o.relin(reduced)[None])
        dec = o.decrypt(rel, o.delta * o.delta / int(o.q[-1]))[0]
        plain = float(((img.astype(np.float64) - other) ** 2).sum())
        results.put((rank, bool(np.array_equal(reduced, full)), bool(abs(dec - plain) < 1e-2), y1 - y0))
    except Exception as e:   # reported to the parent
        results.put((rank, False, repr(e), 0))
    finally:
        dist.destroy_process_group()


def test_allreduce_of_partial_matching_sums_is_exact():
    world = 2
    ctx = mp.get_context("spawn")
    results = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, results)) for r in range(world)]
    for p in procs:
        p.start()
    got = [results.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    assert [g[0] for g in got] == [0, 1]
    for rank, equal, decodes, rows in got:
        assert equal is True, (rank, decodes)
        assert decodes is True
        assert rows >= 3


def test_allreduce_without_a_process_group_is_the_identity():
    acc = torch.arange(6, dtype=torch.int64)
    assert torch.equal(shard.allreduce_accumulator(acc.clone()), acc)
    with pytest.raises(TypeError):
        shard.allreduce_accumulator(acc.to(torch.int32))
