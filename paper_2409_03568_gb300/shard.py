"""Pixel sharding of one image over the ranks of a torch.distributed process group (one GPU per
rank).

Pixel-level encryption makes every pixel's ciphertext independent of the others (Sec. 3.1), so
rank r of W takes a contiguous band of image rows. It encrypts its band with
ichee_encrypt_pixels: ciphertext ids are the pixels' indices in the whole image, so its
ciphertexts are exactly the ones a single GPU makes for those pixels. Row-local operations
(brightness, blend, decryption) run on the band alone. The 3x3 mean filter (Sec. 4.4.1) needs
the rows just above and below the band: the rank encrypts them itself (the same ciphertexts its
neighbours make, so nothing is exchanged) and filters with ichee_meanfilter_rows.

Matching (Sec. 4.4.3) is the one real exchange: each rank accumulates its band's partial sum
of (a - b) (x) (a - b) (ichee_sqdiff_accumulate), one all-reduce adds the accumulators word by
word, and every rank relinearises and rescales the sum (ichee_sqdiff_finish). The words are
residues below 2^60, so the sum of at most 8 accumulators stays below 2^63 and an int64 SUM
(NCCL on GPUs, gloo on CPUs) is exact; ichee_sqdiff_finish reduces it.

Argument marshalling and collectives only: no CKKS arithmetic happens here.
"""

MAX_RANKS = 8


def row_bands(h, world):
    """Contiguous row bands [(y0, y1), ...], one per rank, covering rows 0..h-1 once; sizes
    differ by at most one row (a band is empty when h < world)."""
    if h < 0 or world < 1:
        raise ValueError("bad image height or world size")
    base, extra = divmod(h, world)
    bands, y = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        bands.append((y, y + n))
        y += n
    return bands


def halo_rows(h, y0, y1):
    """Rows a band's mean filter reads: the band plus one row on each side, clamped to the image."""
    return max(0, y0 - 1), min(h, y1 + 1)


def allreduce_accumulator(acc, group=None):
    """Add the ranks' matching accumulators in place (int64 words; at most 8 ranks)."""
    import torch
    import torch.distributed as dist
    if acc.dtype != torch.int64:
        raise TypeError("accumulators are int64 words")
    if not (dist.is_available() and dist.is_initialized()):
        return acc   # one process: nothing to add
    world = dist.get_world_size(group)
    if world > MAX_RANKS:
        raise ValueError("accumulator sums are exact for at most %d ranks, not %d" % (MAX_RANKS, world))
    dist.all_reduce(acc, op=dist.ReduceOp.SUM, group=group)
    return acc


def sharded_match(ichee, ctx, a_band, m_band, b_band, mb_band, acc, out, group=None, stream=None):
    """Matching of an image split into bands: this rank's partial sum, the all-reduce, and the
    relinearisation + rescale (every rank ends with the same ciphertext in `out`). Returns its
    metadata. `acc` is a device int64 tensor of ichee_sqdiff_acc_words words; a rank whose band is
    empty passes a_band = None and contributes zeros. The collective runs on the current torch
    stream, which must be the stream the library calls use."""
    if a_band is None:
        acc.zero_()
    else:
        ichee.ichee_sqdiff_accumulate(ctx.handle, a_band, m_band, b_band, mb_band, acc, accumulate=False,
                                      stream=stream)
    allreduce_accumulator(acc, group)
    return ichee.ichee_sqdiff_finish(ctx.handle, acc, m_band, out, stream=stream)
