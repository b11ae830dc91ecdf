"""ctypes binding of libichee.so, the C ABI declared in include/ichee.h.

Argument marshalling only: every function here forwards to the entry point of the same name,
converting Python values to C types and raising IcheeError on a non-OK status. All arithmetic
on ciphertexts runs in the library's CUDA kernels; there is no CPU fallback, and importing this
module fails loudly when libichee.so has not been built (paper_2409_03568_gb300.build).

Device memory comes from PyTorch tensors (their data_ptr()) and streams from
torch.cuda.Stream.cuda_stream; the helper class Context wraps the handles for tests and the
benchmark.
"""
import ctypes
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libichee.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "ichee.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "libichee.so is not built (expected at %s); run `python -c \"import __graft_entry__ as g; g.build()\"` "
        "or `python paper_2409_03568_gb300/build.py`" % LIB_PATH)

_lib = ctypes.CDLL(LIB_PATH)

MAX_PRIMES = 8
OK, EINVAL, ENOMEM, ECUDA, ELEVEL, ESCALE, EMISMATCH, ETIMEOUT, EUNSUPPORTED = range(9)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ELEVEL", "ESCALE", "EMISMATCH", "ETIMEOUT", "EUNSUPPORTED"]

CACHE_RADIX, CACHE_FREQ, CACHE_FULL = 0, 1, 2
OP_ADD, OP_SUB, OP_PTADD, OP_PTMUL, OP_RESCALE, OP_MEANFILTER3, OP_BRIGHTNESS, OP_BLEND, OP_WATERMARK_PIXEL, \
    OP_SQDIFF_SUM, OP_SQDIFF = range(11)
WITH_EVK = 1


class IcheeError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, message))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_uint32), ("n_primes", ctypes.c_uint32),
                ("prime_bits", ctypes.c_uint32 * MAX_PRIMES), ("special_bits", ctypes.c_uint32),
                ("log2_scale", ctypes.c_uint32), ("sigma", ctypes.c_double), ("gauss_bound", ctypes.c_uint32)]


class CtImgMeta(ctypes.Structure):
    _fields_ = [("h", ctypes.c_uint32), ("w", ctypes.c_uint32), ("c", ctypes.c_uint32),
                ("level", ctypes.c_uint32), ("scale", ctypes.c_double)]

    @property
    def n_ct(self):
        return self.h * self.w * self.c

    def __repr__(self):
        return "CtImgMeta(h=%d, w=%d, c=%d, level=%d, scale=%r)" % (self.h, self.w, self.c, self.level, self.scale)


class CacheDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("radix_base", ctypes.c_uint32), ("radix_randomize", ctypes.c_uint32),
                ("top_k", ctypes.c_uint32), ("pool_size", ctypes.c_uint32), ("miss_policy", ctypes.c_uint32)]


class ImageDesc(ctypes.Structure):
    _fields_ = [("h", ctypes.c_uint32), ("w", ctypes.c_uint32), ("c", ctypes.c_uint32), ("seed", ctypes.c_uint64)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("threads", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("ms", ctypes.c_float)]


TUNE_RADIX, TUNE_LOOKUP, TUNE_MEANFILTER, TUNE_FUSED, TUNE_SCHEDULE, TUNE_DECRYPT, TUNE_MF_STAGED = 1, 2, 3, 4, 5, 6, 7
REQ_ENCRYPT, REQ_MEANFILTER, REQ_BRIGHTNESS, REQ_WATERMARK, REQ_MATCH = range(5)


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("ring", ctypes.c_uint32), ("h", ctypes.c_uint32), ("w", ctypes.c_uint32),
                ("c", ctypes.c_uint32), ("seed", ctypes.c_uint64), ("pixels", ctypes.c_void_p),
                ("pixels2", ctypes.c_void_p), ("arg", ctypes.c_double), ("result", ctypes.c_void_p),
                ("ct_out", ctypes.c_void_p)]


class RequestDone(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("round_size", ctypes.c_uint32),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "served", "pixels", "rounds", "max_inflight", "pending",
                                               "inflight", "arena_bytes", "arena_used_bytes", "peak_arena_bytes")]

_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_sz = ctypes.c_size_t
_st = ctypes.c_int

_SIGS = {
    "ichee_ctx_create": (_st, [ctypes.POINTER(Params), ctypes.c_int, ctypes.POINTER(_vp)]),
    "ichee_ctx_destroy": (None, [_vp]),
    "ichee_ctx_primes": (_st, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "ichee_keygen": (_st, [_vp, _u64, _u32, _vp]),
    "ichee_export_key": (_st, [_vp, ctypes.c_int, _vp, _sz, _vp]),
    "ichee_import_key": (_st, [_vp, ctypes.c_int, _vp, _sz, _vp]),
    "ichee_set_allocator": (_st, [_vp, _vp, _vp, _vp]),
    "ichee_probe_int_throughput": (_st, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "ichee_build_cache": (_st, [_vp, ctypes.POINTER(CacheDesc), _vp, _sz, _u64, ctypes.POINTER(_vp), _vp]),
    "ichee_cache_free": (None, [_vp]),
    "ichee_cache_info": (_st, [_vp, ctypes.POINTER(_u32), _vp, ctypes.POINTER(_u32)]),
    "ichee_cache_export": (_st, [_vp, ctypes.c_int, _vp, _sz, _vp]),
    "ichee_ct_bytes": (_st, [_vp, _u32, ctypes.POINTER(_sz)]),
    "ichee_encrypt_image": (_st, [_vp, _vp, _vp, _u32, _u32, _u32, _u64, _vp, ctypes.POINTER(CtImgMeta), _vp]),
    "ichee_eval": (_st, [_vp, ctypes.c_int, _vp, ctypes.POINTER(CtImgMeta), _vp, ctypes.POINTER(CtImgMeta),
                         _vp, _u32, _vp, ctypes.POINTER(CtImgMeta), _vp]),
    "ichee_decrypt_image": (_st, [_vp, _vp, ctypes.POINTER(CtImgMeta), _vp, _vp]),
    "ichee_decrypt_residues": (_st, [_vp, _vp, ctypes.POINTER(CtImgMeta), _vp, _vp, _vp]),
    "ichee_decrypt_image_async": (_st, [_vp, _vp, ctypes.POINTER(CtImgMeta), _vp, _vp]),
    "ichee_encrypt_pixels": (_st, [_vp, _vp, _vp, _u64, _u64, _u64, _vp, _vp]),
    "ichee_meanfilter_rows": (_st, [_vp, _vp, ctypes.POINTER(CtImgMeta), _u32, _u32, _u32, _u32, _vp,
                                    ctypes.POINTER(CtImgMeta), _vp]),
    "ichee_sqdiff_acc_words": (_st, [_vp, _u32, ctypes.POINTER(_sz)]),
    "ichee_sqdiff_accumulate": (_st, [_vp, _vp, ctypes.POINTER(CtImgMeta), _vp, ctypes.POINTER(CtImgMeta), _vp,
                                      ctypes.c_int, _vp]),
    "ichee_sqdiff_finish": (_st, [_vp, _vp, ctypes.POINTER(CtImgMeta), _vp, ctypes.POINTER(CtImgMeta), _vp]),
    "ichee_sqdiff_sum_noalloc": (_st, [_vp, _vp, ctypes.POINTER(CtImgMeta), _vp, ctypes.POINTER(CtImgMeta), _vp,
                                       ctypes.POINTER(CtImgMeta), _vp]),
    "ichee_encrypt_batch": (_st, [_vp, _vp, ctypes.POINTER(_vp), ctypes.POINTER(ImageDesc), _u32,
                                  ctypes.POINTER(_vp), ctypes.POINTER(CtImgMeta), _vp]),
    "ichee_encrypt_meanfilter_batch": (_st, [_vp, _vp, ctypes.POINTER(_vp), ctypes.POINTER(ImageDesc), _u32,
                                             ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(CtImgMeta),
                                             ctypes.POINTER(CtImgMeta), _vp]),
    "ichee_eval_batch": (_st, [_vp, ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(CtImgMeta), ctypes.POINTER(_vp),
                               ctypes.POINTER(CtImgMeta), _vp, _u32, ctypes.POINTER(_vp), ctypes.POINTER(CtImgMeta),
                               _u32, _vp]),
    "ichee_decrypt_batch": (_st, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(CtImgMeta), ctypes.POINTER(_vp), _u32,
                                  _vp]),
    "ichee_autotune_batch": (_st, [_vp, _vp, ctypes.POINTER(_vp), ctypes.POINTER(ImageDesc), _u32,
                                   ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(TuneEntry),
                                   ctypes.POINTER(_u32), _vp]),
    "ichee_tuned_shape": (_st, [_vp, _u32, ctypes.POINTER(_u32), ctypes.POINTER(_u32)]),
    "ichee_set_tuned_shape": (_st, [_vp, _u32, _u32, _u32]),
    "ichee_graph_begin": (_st, [_vp, _vp]),
    "ichee_graph_end": (_st, [_vp, _vp, ctypes.POINTER(_vp)]),
    "ichee_graph_launch": (_st, [_vp, _vp]),
    "ichee_graph_destroy": (None, [_vp]),
    "ichee_server_create": (_st, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), _u32, _sz, _u32, ctypes.POINTER(_vp)]),
    "ichee_server_submit": (_st, [_vp, ctypes.POINTER(Request), ctypes.POINTER(_u64)]),
    "ichee_server_wait": (_st, [_vp, _u64, _u32, ctypes.POINTER(RequestDone)]),
    "ichee_server_stats_get": (_st, [_vp, ctypes.POINTER(ServerStats)]),
    "ichee_server_hold": (_st, [_vp, ctypes.c_int]),
    "ichee_server_destroy": (None, [_vp]),
    "ichee_server_inject_failure": (_st, [_vp, _u32, _u32]),
    "ichee_stream_status": (_st, [_vp, _vp]),
    "ichee_buffer_bytes_left": (_st, [_vp, ctypes.POINTER(_sz)]),
    "ichee_last_error": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def header_functions(path=HEADER):
    """Names of the functions include/ichee.h declares."""
    with open(path) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:ichee_status|void|const char\*)\s+(ichee_\w+)\s*\(", text, re.M)))


def ichee_last_error():
    return _lib.ichee_last_error().decode()


def _check(status):
    if status != OK:
        raise IcheeError(status, ichee_last_error())


def _ptr(x):
    """Integer address of a tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError("cannot take the address of %r" % type(x))


def make_params(log_n, prime_bits, log2_scale, special_bits=0, sigma=3.2, gauss_bound=19):
    p = Params()
    p.log_n = log_n
    p.n_primes = len(prime_bits)
    for i, b in enumerate(prime_bits):
        p.prime_bits[i] = b
    p.special_bits = special_bits
    p.log2_scale = log2_scale
    p.sigma = sigma
    p.gauss_bound = gauss_bound
    return p


def ichee_ctx_create(params, device=0):
    h = _vp()
    _check(_lib.ichee_ctx_create(ctypes.byref(params), device, ctypes.byref(h)))
    return h


def ichee_ctx_destroy(ctx):
    _lib.ichee_ctx_destroy(ctx)


def ichee_ctx_primes(ctx, n_primes):
    q = (_u64 * n_primes)()
    p = _u64()
    _check(_lib.ichee_ctx_primes(ctx, q, ctypes.byref(p)))
    return [int(x) for x in q], int(p.value)


def ichee_keygen(ctx, seed, flags=0, stream=None):
    _check(_lib.ichee_keygen(ctx, seed, flags, stream))


# Working-memory allocator callbacks: alloc(bytes, stream, user) -> device pointer (0 = out
# of memory); free(ptr, stream, user).
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


def ichee_set_allocator(ctx, alloc=None, free=None):
    """alloc, free: ALLOC_FN / FREE_FN instances (the caller keeps them alive), or None for
    cudaMalloc."""
    a = ctypes.cast(alloc, ctypes.c_void_p) if alloc is not None else None
    f = ctypes.cast(free, ctypes.c_void_p) if free is not None else None
    _check(_lib.ichee_set_allocator(ctx, a, f, None))


def ichee_probe_int_throughput(device=0):
    """(32-bit multiply-adds per second, library butterflies per second) of the GPU."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(_lib.ichee_probe_int_throughput(device, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def ichee_export_key(ctx, which, host_array, stream=None):
    _check(_lib.ichee_export_key(ctx, which, _ptr(host_array), host_array.nbytes, stream))


def ichee_import_key(ctx, which, host_array, stream=None):
    """which: 0 = secret key int8[N], 1 = public key uint64[2][L][N], 2 = evaluation key
    uint64[L][2][L+1][N] (numpy arrays, as ichee_export_key writes them)."""
    import numpy as np
    arr = np.ascontiguousarray(host_array)
    _check(_lib.ichee_import_key(ctx, which, arr.ctypes.data, arr.nbytes, stream))


def ichee_build_cache(ctx, desc, scan=None, n_scan=0, seed=0, stream=None):
    h = _vp()
    _check(_lib.ichee_build_cache(ctx, ctypes.byref(desc), _ptr(scan), n_scan, seed, ctypes.byref(h), stream))
    return h


def ichee_cache_free(cache):
    _lib.ichee_cache_free(cache)


def ichee_cache_info(cache):
    n = _u32()
    pool = _u32()
    vals = (ctypes.c_uint8 * 256)()
    _check(_lib.ichee_cache_info(cache, ctypes.byref(n), vals, ctypes.byref(pool)))
    return [int(v) for v in vals[:n.value]], int(pool.value)


def ichee_cache_export(cache, part, host_array, stream=None):
    _check(_lib.ichee_cache_export(cache, part, _ptr(host_array), host_array.nbytes, stream))


def ichee_ct_bytes(ctx, level):
    b = _sz()
    _check(_lib.ichee_ct_bytes(ctx, level, ctypes.byref(b)))
    return int(b.value)


def ichee_encrypt_image(ctx, cache, pixels, h, w, c, seed, ct_out, stream=None):
    m = CtImgMeta()
    _check(_lib.ichee_encrypt_image(ctx, cache, _ptr(pixels), h, w, c, seed, _ptr(ct_out), ctypes.byref(m), stream))
    return m


def ichee_eval(ctx, op, a, ma, b=None, mb=None, args=(), out=None, stream=None):
    m = CtImgMeta()
    n = len(args)
    arr = (ctypes.c_double * max(n, 1))(*args)
    _check(_lib.ichee_eval(ctx, op, _ptr(a), ctypes.byref(ma), _ptr(b), ctypes.byref(mb) if mb is not None else None,
                           arr if n else None, n, _ptr(out), ctypes.byref(m), stream))
    return m


def ichee_decrypt_image(ctx, ct, meta, out, stream=None):
    _check(_lib.ichee_decrypt_image(ctx, _ptr(ct), ctypes.byref(meta), _ptr(out), stream))


def ichee_decrypt_image_async(ctx, ct, meta, out, stream=None):
    """Decrypt into device or page-locked host memory without waiting for the stream."""
    _check(_lib.ichee_decrypt_image_async(ctx, _ptr(ct), ctypes.byref(meta), _ptr(out), stream))


def ichee_decrypt_residues(ctx, ct, meta, out, residues, stream=None):
    _check(_lib.ichee_decrypt_residues(ctx, _ptr(ct), ctypes.byref(meta), _ptr(out), _ptr(residues), stream))


def ichee_sqdiff_sum_noalloc(ctx, a, ma, b, mb, out, stream=None):
    """Matching into a caller-provided output without any device allocation (see ichee.h)."""
    m = CtImgMeta()
    _check(_lib.ichee_sqdiff_sum_noalloc(ctx, _ptr(a), ctypes.byref(ma), _ptr(b), ctypes.byref(mb), _ptr(out),
                                         ctypes.byref(m), stream))
    return m


def ichee_encrypt_pixels(ctx, cache, pixels, n, first_id, seed, out, stream=None):
    """Ciphertexts first_id .. first_id + n - 1 of the whole-image encryption (see ichee.h)."""
    _check(_lib.ichee_encrypt_pixels(ctx, cache, _ptr(pixels), n, first_id, seed, _ptr(out), stream))


def ichee_meanfilter_rows(ctx, ct_rows, m_img, row0, n_rows, y0, y1, out, stream=None):
    """Output rows [y0, y1) of the 3x3 mean filter of the image m_img describes, from its rows
    [row0, row0 + n_rows) (see ichee.h)."""
    m = CtImgMeta()
    _check(_lib.ichee_meanfilter_rows(ctx, _ptr(ct_rows), ctypes.byref(m_img), row0, n_rows, y0, y1, _ptr(out),
                                      ctypes.byref(m), stream))
    return m


def ichee_sqdiff_acc_words(ctx, level):
    w = _sz()
    _check(_lib.ichee_sqdiff_acc_words(ctx, level, ctypes.byref(w)))
    return int(w.value)


def ichee_sqdiff_accumulate(ctx, a, ma, b, mb, acc, accumulate=False, stream=None):
    """acc (device, ichee_sqdiff_acc_words words) = or += the matching sum of the pairs (see ichee.h)."""
    _check(_lib.ichee_sqdiff_accumulate(ctx, _ptr(a), ctypes.byref(ma), _ptr(b), ctypes.byref(mb), _ptr(acc),
                                        1 if accumulate else 0, stream))


def ichee_sqdiff_finish(ctx, acc, m_in, out, stream=None):
    """Relinearise and rescale a matching accumulator (or a sum of up to 8) into one ciphertext."""
    m = CtImgMeta()
    _check(_lib.ichee_sqdiff_finish(ctx, _ptr(acc), ctypes.byref(m_in), _ptr(out), ctypes.byref(m), stream))
    return m


def _ptrs(xs):
    return (_vp * max(len(xs), 1))(*[_ptr(x) for x in xs])


def _descs(shapes, seeds):
    arr = (ImageDesc * len(shapes))()
    for i, ((h, w, c), sd) in enumerate(zip(shapes, seeds)):
        arr[i].h, arr[i].w, arr[i].c, arr[i].seed = h, w, c, sd
    return arr


def ichee_encrypt_batch(ctx, cache, pixels, shapes, seeds, ct_outs, stream=None):
    """Encrypt images (device pixel tensors, shapes [(h, w, c)], seeds) into ct_outs; returns metas."""
    n = len(shapes)
    metas = (CtImgMeta * n)()
    _check(_lib.ichee_encrypt_batch(ctx, cache, _ptrs(pixels), _descs(shapes, seeds), n, _ptrs(ct_outs), metas,
                                    stream))
    return list(metas)


def ichee_encrypt_meanfilter_batch(ctx, cache, pixels, shapes, seeds, ct_outs, filtered_outs, stream=None):
    n = len(shapes)
    mc, mf = (CtImgMeta * n)(), (CtImgMeta * n)()
    _check(_lib.ichee_encrypt_meanfilter_batch(ctx, cache, _ptrs(pixels), _descs(shapes, seeds), n, _ptrs(ct_outs),
                                               _ptrs(filtered_outs), mc, mf, stream))
    return list(mc), list(mf)


def _metas(ms):
    arr = (CtImgMeta * len(ms))()
    for i, m in enumerate(ms):
        arr[i] = m
    return arr


def ichee_eval_batch(ctx, op, a, ma, b=None, mb=None, args=(), outs=None, stream=None):
    n = len(a)
    mout = (CtImgMeta * n)()
    nargs = len(args)
    arr = (ctypes.c_double * max(nargs, 1))(*args)
    _check(_lib.ichee_eval_batch(ctx, op, _ptrs(a), _metas(ma), _ptrs(b) if b is not None else None,
                                 _metas(mb) if mb is not None else None, arr if nargs else None, nargs, _ptrs(outs),
                                 mout, n, stream))
    return list(mout)


def ichee_decrypt_batch(ctx, cts, metas, outs, stream=None):
    _check(_lib.ichee_decrypt_batch(ctx, _ptrs(cts), _metas(metas), _ptrs(outs), len(cts), stream))


def ichee_autotune_batch(ctx, cache, pixels, shapes, seeds, cts, filtered, stream=None, max_report=64):
    n = len(shapes)
    rep = (TuneEntry * max_report)()
    nrep = _u32(max_report)
    _check(_lib.ichee_autotune_batch(ctx, cache, _ptrs(pixels), _descs(shapes, seeds), n, _ptrs(cts), _ptrs(filtered),
                                     rep, ctypes.byref(nrep), stream))
    return [(e.kind, e.threads, e.blocks_per_sm, e.ms) for e in rep[:min(nrep.value, max_report)]]


def ichee_tuned_shape(ctx, kind):
    t, b = _u32(), _u32()
    _check(_lib.ichee_tuned_shape(ctx, kind, ctypes.byref(t), ctypes.byref(b)))
    return int(t.value), int(b.value)


def ichee_set_tuned_shape(ctx, kind, threads, blocks_per_sm=0):
    _check(_lib.ichee_set_tuned_shape(ctx, kind, threads, blocks_per_sm))


def ichee_graph_begin(ctx, stream):
    _check(_lib.ichee_graph_begin(ctx, stream))


def ichee_graph_end(ctx, stream):
    g = _vp()
    _check(_lib.ichee_graph_end(ctx, stream, ctypes.byref(g)))
    return g


def ichee_graph_launch(graph, stream=None):
    _check(_lib.ichee_graph_launch(graph, stream))


def ichee_graph_destroy(graph):
    _lib.ichee_graph_destroy(graph)


def ichee_server_create(rings, caches, hbm_budget_bytes, max_inflight=0):
    n = len(rings)
    h = _vp()
    _check(_lib.ichee_server_create((_vp * n)(*[r.value if isinstance(r, _vp) else r for r in rings]),
                                    (_vp * n)(*[None if c is None else (c.value if isinstance(c, _vp) else c)
                                                for c in caches]),
                                    n, hbm_budget_bytes, max_inflight, ctypes.byref(h)))
    return h


def ichee_server_submit(server, request):
    t = _u64()
    _check(_lib.ichee_server_submit(server, ctypes.byref(request), ctypes.byref(t)))
    return int(t.value)


def ichee_server_wait(server, ticket, timeout_ms=60000):
    d = RequestDone()
    _check(_lib.ichee_server_wait(server, ticket, timeout_ms, ctypes.byref(d)))
    return d


def ichee_server_stats_get(server):
    st = ServerStats()
    _check(_lib.ichee_server_stats_get(server, ctypes.byref(st)))
    return {n: int(getattr(st, n)) for n, _ in ServerStats._fields_}


def ichee_server_hold(server, hold):
    _check(_lib.ichee_server_hold(server, 1 if hold else 0))


def ichee_server_destroy(server):
    _lib.ichee_server_destroy(server)


def ichee_server_inject_failure(server, launch_errors=0, query_errors=0):
    """Host-side failure injection (tests): the next rounds fail as launch / completion errors."""
    _check(_lib.ichee_server_inject_failure(server, launch_errors, query_errors))


def ichee_stream_status(ctx, stream=None):
    _check(_lib.ichee_stream_status(ctx, stream))


def ichee_buffer_bytes_left(buf):
    """Bytes from the buffer's address to the end of its device allocation (the bound every
    entry point checks device buffers against)."""
    n = _sz(0)
    _check(_lib.ichee_buffer_bytes_left(_ptr(buf), ctypes.byref(n)))
    return n.value


class Context:
    """Owner of one ichee_ctx handle plus helpers that allocate torch device buffers for
    ciphertext images. Marshalling only."""

    def __init__(self, log_n, prime_bits, log2_scale, special_bits=0, sigma=3.2, gauss_bound=19, device=0):
        import torch  # noqa: F401  (CUDA context + allocator)
        self.params = make_params(log_n, prime_bits, log2_scale, special_bits, sigma, gauss_bound)
        self.n = 1 << log_n
        self.L = len(prime_bits)
        self.device = device
        self.handle = ichee_ctx_create(self.params, device)
        self.q, self.P = ichee_ctx_primes(self.handle, self.L)
        self.caches = []

    def close(self):
        for c in self.caches:
            ichee_cache_free(c)
        self.caches = []
        if self.handle:
            if getattr(self, "_alloc_cbs", None):
                ichee_set_allocator(self.handle, None, None)   # hand the buffers back while torch is alive
                self._alloc_cbs = None
            ichee_ctx_destroy(self.handle)
            self.handle = None

    def use_torch_allocator(self):
        """Take the library's working memory from PyTorch's caching allocator on this device.
        Returns the list of (bytes, pointer) allocations made through it (for inspection)."""
        import torch
        log = []

        def _alloc(n, stream, _user):
            try:
                p = torch.cuda.caching_allocator_alloc(int(n), self.device, stream or 0)
            except RuntimeError:
                return 0
            log.append((int(n), int(p)))
            return p

        def _free(ptr, _stream, _user):
            torch.cuda.caching_allocator_delete(int(ptr))

        cbs = (ALLOC_FN(_alloc), FREE_FN(_free))
        ichee_set_allocator(self.handle, *cbs)
        self._alloc_cbs = cbs
        return log

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def stream():
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def keygen(self, seed, with_evk=False):
        ichee_keygen(self.handle, seed, WITH_EVK if with_evk else 0, self.stream())

    def save_keys(self, path, secret=True, evk=True):
        """Write the keys (and the prime chain they belong to) to an .npz file. secret=False
        leaves the secret key out, e.g. for a server that only encrypts and evaluates."""
        import numpy as np
        n, L = self.n, self.L
        parts = {"primes": np.array(self.q + ([self.P] if self.P else []), dtype=np.uint64)}
        pk = np.zeros((2, L, n), dtype=np.uint64)
        ichee_export_key(self.handle, 1, pk, self.stream())
        parts["pk"] = pk
        if secret:
            s = np.zeros(n, dtype=np.int8)
            ichee_export_key(self.handle, 0, s, self.stream())
            parts["s"] = s
        if evk:
            e = np.zeros((L, 2, L + 1, n), dtype=np.uint64)
            ichee_export_key(self.handle, 2, e, self.stream())
            parts["evk"] = e
        np.savez(path, **parts)

    def load_keys(self, path):
        """Load keys written by save_keys into this context (same parameters required)."""
        import numpy as np
        with np.load(path) as z:
            primes = [int(x) for x in z["primes"]]
            if primes != self.q + ([self.P] if self.P else []):
                raise IcheeError(EINVAL, "keys belong to another prime chain")
            ichee_import_key(self.handle, 1, z["pk"], self.stream())
            if "s" in z:
                ichee_import_key(self.handle, 0, z["s"], self.stream())
            if "evk" in z:
                ichee_import_key(self.handle, 2, z["evk"], self.stream())

    def ct_words(self, level):
        return ichee_ct_bytes(self.handle, level) // 8

    def empty_cts(self, n_ct, level):
        import torch
        return torch.empty(n_ct * self.ct_words(level), dtype=torch.int64, device="cuda:%d" % self.device)

    def build_cache(self, kind, seed, radix_base=0, randomize=1, top_k=0, pool_size=0, miss_policy=0, scan=None):
        d = CacheDesc()
        d.kind = kind
        d.radix_base = radix_base
        d.radix_randomize = randomize
        d.top_k = top_k
        d.pool_size = pool_size
        d.miss_policy = miss_policy
        n_scan = 0 if scan is None else (scan.numel() if hasattr(scan, "numel") else scan.size)
        h = ichee_build_cache(self.handle, d, scan, n_scan, seed, self.stream())
        self.caches.append(h)
        return h

    def encrypt(self, pixels, h, w, c, seed, cache=None, out=None):
        if out is None:
            out = self.empty_cts(h * w * c, self.L - 1)
        m = ichee_encrypt_image(self.handle, cache, pixels, h, w, c, seed, out, self.stream())
        return out, m

    def eval(self, op, a, ma, b=None, mb=None, args=(), out=None, out_n_ct=None, out_level=None):
        if out is None:
            lvl = ma.level if out_level is None else out_level
            out = self.empty_cts(ma.n_ct if out_n_ct is None else out_n_ct, lvl)
        m = ichee_eval(self.handle, op, a, ma, b, mb, args, out, self.stream())
        return out, m

    def decrypt(self, ct, meta, out=None):
        import torch
        if out is None:
            out = torch.empty(meta.n_ct, dtype=torch.float64, device="cuda:%d" % self.device)
        ichee_decrypt_image(self.handle, ct, meta, out, self.stream())
        return out

    def decrypt_residues(self, ct, meta):
        import torch
        out = torch.empty(meta.n_ct, dtype=torch.float64, device="cuda:%d" % self.device)
        res = torch.empty(meta.n_ct * (meta.level + 1), dtype=torch.int64, device="cuda:%d" % self.device)
        ichee_decrypt_residues(self.handle, ct, meta, out, res, self.stream())
        return out, res

    def status(self):
        ichee_stream_status(self.handle, self.stream())
