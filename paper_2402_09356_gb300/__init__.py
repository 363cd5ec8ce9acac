"""GB300 (sm_103a) Tile Low-Rank Matern log-likelihood -- Python binding.

A thin ctypes layer over the C ABI in include/tlr.h (libtlr.so, built in-tree
by paper_2402_09356_gb300/build.py).  Every function here has the name of the
C entry point it calls and only marshals arguments: torch tensors supply
device memory (their data pointers) and the current CUDA stream.  All
computation happens in the library's CUDA kernels; there is no CPU fallback:
if libtlr.so is missing or cannot be loaded, importing the functions raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libtlr.so")

TLR_OK, TLR_ERR_ARG, TLR_ERR_CUDA, TLR_ERR_OOM, TLR_ERR_RANK, TLR_ERR_NOT_SPD, TLR_ERR_TIMEOUT, TLR_ERR_NAN = range(8)
ORDERS = {"identity": 0, "random": 1, "morton": 2, "hilbert": 3, "kdtree": 4, "maxmin": 5}
TLR_ORDER_QUANTIZE = 1
TLR_PREC_FP64 = 0
TLR_PREC_MIXED = 1
TLR_PREC_AUTO = 2
TLR_PREC_TENSOR = 3
TLR_AUTO_PIVOT2 = 3e-5


class TlrError(RuntimeError):
    def __init__(self, code: int, msg: str, info: int = -1):
        super().__init__("TLR error %d: %s" % (code, msg))
        self.code = code
        self.info = info


class tlr_theta(ctypes.Structure):
    _fields_ = [("sigma2", ctypes.c_double), ("beta", ctypes.c_double), ("nu", ctypes.c_double)]


class tlr_opts(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int32), ("maxrank", ctypes.c_int32), ("eps", ctypes.c_double),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class tlr_result(ctypes.Structure):
    _fields_ = [("loglik", ctypes.c_double), ("logdet", ctypes.c_double), ("quad", ctypes.c_double),
                ("info", ctypes.c_int64), ("max_rank", ctypes.c_int32), ("mean_rank", ctypes.c_double),
                ("offdiag_bytes", ctypes.c_int64), ("dense_bytes", ctypes.c_int64),
                ("flops", ctypes.c_double), ("ms_total", ctypes.c_float), ("precision_used", ctypes.c_int32),
                ("min_pivot2", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class tlr_buckets(ctypes.Structure):
    _fields_ = [("qr_edge", ctypes.c_int32 * 4), ("qr_size", ctypes.c_int32 * 4),
                ("svd_edge", ctypes.c_int32 * 4), ("svd_size", ctypes.c_int32 * 4)]

    def as_dict(self) -> dict:
        return {f: list(getattr(self, f)) for f, _ in self._fields_}


class tlr_pool_opts(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("nb", ctypes.c_int32), ("maxrank", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("hbm_budget", ctypes.c_int64)]


_lib = None

_SIGS = {
    "tlr_version": (ctypes.c_char_p, []),
    "tlr_launch_count": (ctypes.c_int64, []),
    "tlr_ctx_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "tlr_ctx_destroy": (None, [ctypes.c_void_p]),
    "tlr_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "tlr_ctx_set_buckets": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "tlr_ctx_get_buckets": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tlr_buckets)]),
    "tlr_order": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64,
                                 ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p]),
    "tlr_order_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tlr_gather": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                  ctypes.c_void_p, ctypes.c_void_p]),
    "tlr_tiles_size": (ctypes.c_int64, [ctypes.c_int64, ctypes.c_int]),
    "tlr_generate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, tlr_theta,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    "tlr_gemm_tc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                   ctypes.c_void_p]),
    "tlr_matern": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, tlr_theta, ctypes.c_void_p,
                                  ctypes.c_void_p]),
    "tlr_mat_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "tlr_mat_destroy": (None, [ctypes.c_void_p]),
    "tlr_mat_create_compact": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "tlr_mat_bytes": (ctypes.c_int64, [ctypes.c_void_p]),
    "tlr_mat_plan_bytes": (ctypes.c_int64, [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "tlr_mat_layout": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p)]),
    "tlr_mat_ranks": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tlr_mat_tile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]),
    "tlr_compress": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]),
    "tlr_potrf": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(ctypes.c_int64),
                                 ctypes.c_void_p]),
    "tlr_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "tlr_lmul": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tlr_loglik": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, tlr_theta,
                                  ctypes.POINTER(tlr_opts), ctypes.c_void_p, ctypes.POINTER(tlr_result),
                                  ctypes.c_void_p]),
    "tlr_loglik_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tlr_loglik_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_int, ctypes.c_uint64, tlr_theta, ctypes.POINTER(tlr_opts),
                                       ctypes.c_void_p, ctypes.POINTER(tlr_result), ctypes.c_void_p]),
    "tlr_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_int)]),
    "tlr_stage_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "tlr_compress_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "tlr_compress_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "tlr_kernel_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "tlr_detail_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "tlr_mle": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                               ctypes.POINTER(tlr_opts), tlr_theta, tlr_theta, tlr_theta, ctypes.c_double,
                               ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(tlr_theta),
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "tlr_pool_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(tlr_pool_opts), ctypes.POINTER(ctypes.c_void_p)]),
    "tlr_pool_destroy": (None, [ctypes.c_void_p]),
    "tlr_pool_last_error": (ctypes.c_char_p, []),
    "tlr_pool_add": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                    ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "tlr_pool_remove": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "tlr_pool_dataset": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_int32)]),
    "tlr_pool_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, tlr_theta, ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int64)]),
    "tlr_pool_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(tlr_result),
                                     ctypes.POINTER(ctypes.c_double)]),
    "tlr_pool_loglik": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "tlr_pool_mle": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int, tlr_theta,
                                    tlr_theta, tlr_theta, ctypes.c_double, ctypes.c_int, ctypes.POINTER(tlr_theta),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    "tlr_pool_tune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, tlr_theta, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]),
    "tlr_pool_configure": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "tlr_pool_get_config": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(tlr_buckets)]),
    "tlr_pool_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_int)]),
    "tlr_pool_footprint": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "tlr_pool_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "tlr_shard_place": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "tlr_sched_simulate": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
}


def load_library(path: str = LIB_PATH):
    """Load libtlr.so and declare the C signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libtlr.so not built (%s); run paper_2402_09356_gb300/build.py" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _theta(theta) -> tlr_theta:
    if isinstance(theta, tlr_theta):
        return theta
    s2, b, nu = theta
    return tlr_theta(float(s2), float(b), float(nu))


def _check_f64(name, t, numel=None):
    import torch
    if t.device.type != "cuda" or t.dtype != torch.float64 or not t.is_contiguous():
        raise TlrError(TLR_ERR_ARG, "%s must be a contiguous float64 CUDA tensor" % name)
    if numel is not None and t.numel() != numel:
        raise TlrError(TLR_ERR_ARG, "%s must have %d elements" % (name, numel))


class Context:
    """Owns a tlr_ctx on one device."""

    def __init__(self, device: int = 0):
        lib = load_library()
        h = ctypes.c_void_p()
        rc = lib.tlr_ctx_create(int(device), ctypes.byref(h))
        if rc != TLR_OK:
            raise TlrError(rc, "tlr_ctx_create failed on device %d" % device)
        self.h = h
        self.device = device

    def check(self, rc: int, info: int = -1):
        if rc != TLR_OK:
            msg = load_library().tlr_last_error(self.h).decode()
            raise TlrError(rc, msg, info)

    def close(self):
        if getattr(self, "h", None):
            load_library().tlr_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TlrMatrix:
    """Owns a tlr_mat (TLR matrix or factor) of a context."""

    def __init__(self, ctx: Context, n: int, nb: int, maxrank: int = 0, rank_map=None):
        """rank_map (NT x NT int32, e.g. tlr_mat_ranks of an earlier factor): compact storage."""
        self.ctx = ctx
        h = ctypes.c_void_p()
        if rank_map is None:
            ctx.check(load_library().tlr_mat_create(ctx.h, int(n), int(nb), int(maxrank), ctypes.byref(h)))
        else:
            import numpy as np
            rm = np.ascontiguousarray(rank_map, dtype=np.int32)
            nt = (int(n) + int(nb) - 1) // int(nb)
            if rm.size != nt * nt:
                raise TlrError(TLR_ERR_ARG, "rank_map must be NT x NT")
            ctx.check(load_library().tlr_mat_create_compact(ctx.h, int(n), int(nb), int(maxrank),
                                                            ctypes.c_void_p(rm.ctypes.data), ctypes.byref(h)))
        self.h = h
        self.n, self.nb = int(n), int(nb)
        self.nt = (self.n + self.nb - 1) // self.nb
        self.maxrank = self.layout()["maxrank"]

    def nbytes(self) -> int:
        return int(load_library().tlr_mat_bytes(self.h))

    def layout(self) -> dict:
        n, nb, nt, mr = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        D, U, V, R = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        load_library().tlr_mat_layout(self.h, ctypes.byref(n), ctypes.byref(nb), ctypes.byref(nt), ctypes.byref(mr),
                                      ctypes.byref(D), ctypes.byref(U), ctypes.byref(V), ctypes.byref(R))
        return {"n": n.value, "nb": nb.value, "nt": nt.value, "maxrank": mr.value,
                "D": D.value, "U": U.value, "V": V.value, "ranks": R.value}

    def close(self):
        if getattr(self, "h", None):
            load_library().tlr_mat_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tlr_ctx_set_buckets(ctx: Context, buckets=None):
    """Rank buckets of the compression (tlr_buckets or a dict with its four
    lists); None restores the default."""
    if buckets is None:
        ctx.check(load_library().tlr_ctx_set_buckets(ctx.h, None))
        return
    b = buckets if isinstance(buckets, tlr_buckets) else tlr_buckets(
        *[(ctypes.c_int32 * 4)(*[int(v) for v in buckets[f]]) for f, _ in tlr_buckets._fields_])
    ctx.check(load_library().tlr_ctx_set_buckets(ctx.h, ctypes.byref(b)))


def tlr_ctx_get_buckets(ctx: Context) -> dict:
    b = tlr_buckets()
    ctx.check(load_library().tlr_ctx_get_buckets(ctx.h, ctypes.byref(b)))
    return b.as_dict()


def tlr_version() -> str:
    return load_library().tlr_version().decode()


def tlr_launch_count() -> int:
    return int(load_library().tlr_launch_count())


def tlr_order(ctx: Context, xy, method, seed: int = 3, flags: int = 0, perm=None, codes=None, xy_out=None,
              stream=None):
    """Order SoA locations xy (float64 CUDA, 2n).  Returns perm (int64 CUDA, n)."""
    import torch
    n = xy.numel() // 2
    _check_f64("xy", xy, 2 * n)
    if isinstance(method, str):
        method = ORDERS[method]
    if perm is None:
        perm = torch.empty(n, dtype=torch.int64, device=xy.device)
    rc = load_library().tlr_order(ctx.h, _ptr(xy), n, int(method), ctypes.c_uint64(seed & (2**64 - 1)),
                                  int(flags), _ptr(perm), _ptr(codes), _ptr(xy_out), _stream(stream))
    ctx.check(rc)
    return perm


def tlr_order_noalloc(xy, method, seed: int = 3, perm=None, codes=None, stream=None):
    """tlr_order for random / Morton / Hilbert without device allocation in the library.

    For callers that cannot allocate while running; uses the library's fixed
    scratch array (n <= 262,144).  perm (int64 CUDA, n) is returned.
    """
    import torch
    n = xy.numel() // 2
    _check_f64("xy", xy, 2 * n)
    if isinstance(method, str):
        method = ORDERS[method]
    if perm is None:
        perm = torch.empty(n, dtype=torch.int64, device=xy.device)
    rc = load_library().tlr_order_noalloc(_ptr(xy), n, int(method), ctypes.c_uint64(seed & (2**64 - 1)),
                                          _ptr(perm), _ptr(codes), _stream(stream))
    if rc != TLR_OK:
        raise TlrError(rc, "tlr_order_noalloc failed")
    return perm


def tlr_gather(ctx: Context, perm, src, dst=None, stream=None):
    import torch
    n = perm.numel()
    if dst is None:
        dst = torch.empty(n, dtype=torch.float64, device=src.device)
    ctx.check(load_library().tlr_gather(ctx.h, _ptr(perm), _ptr(src), n, _ptr(dst), _stream(stream)))
    return dst


def tlr_tiles_size(n: int, nb: int) -> int:
    return int(load_library().tlr_tiles_size(int(n), int(nb)))


def tlr_generate(ctx: Context, xy, nb: int, theta, tiles=None, stream=None):
    """Packed lower-triangular dense covariance tiles (float64 CUDA)."""
    import torch
    n = xy.numel() // 2
    _check_f64("xy", xy, 2 * n)
    if tiles is None:
        tiles = torch.empty(tlr_tiles_size(n, nb), dtype=torch.float64, device=xy.device)
    ctx.check(load_library().tlr_generate(ctx.h, _ptr(xy), n, int(nb), _theta(theta), _ptr(tiles), _stream(stream)))
    return tiles


def tlr_gemm_tc(ctx: Context, A, B, C=None, alpha: float = 1.0, beta: float = 0.0, trans_a: bool = False,
                trans_b: bool = False, slices: int = 5, stream=None):
    """C = alpha op(A) op(B) + beta C on the tensor cores (BF16 slices).  A, B, C
    are float64 CUDA tensors holding column-major matrices as their transposes
    (a torch (cols, rows) row-major tensor is a column-major rows x cols matrix)."""
    import torch
    for name, t in (("A", A), ("B", B)):
        _check_f64(name, t)
        if t.dim() != 2 or not t.is_contiguous():
            raise ValueError("%s must be a contiguous 2-D tensor" % name)
    # column-major view: rows = size(1), cols = size(0), ld = size(1)
    ar, ac = A.shape[1], A.shape[0]
    br, bc = B.shape[1], B.shape[0]
    m, k = (ac, ar) if trans_a else (ar, ac)
    kb, n = (bc, br) if trans_b else (br, bc)
    if k != kb:
        raise ValueError("inner dimensions differ: %d vs %d" % (k, kb))
    if C is None:
        C = torch.zeros((n, m), dtype=torch.float64, device=A.device)
    _check_f64("C", C)
    if tuple(C.shape) != (n, m) or not C.is_contiguous():
        raise ValueError("C must be a contiguous (n, m) tensor")
    ctx.check(load_library().tlr_gemm_tc(ctx.h, int(trans_a), int(trans_b), m, n, k, float(alpha), _ptr(A),
                                         max(ar, 1), _ptr(B), max(br, 1), float(beta), _ptr(C), max(m, 1),
                                         int(slices), _stream(stream)))
    return C


def tlr_matern(ctx: Context, d, theta, out=None, stream=None):
    import torch
    _check_f64("d", d)
    if out is None:
        out = torch.empty_like(d)
    ctx.check(load_library().tlr_matern(ctx.h, _ptr(d), d.numel(), _theta(theta), _ptr(out), _stream(stream)))
    return out


def tlr_mat_plan_bytes(n: int, nb: int, maxrank: int = 0, rank_map=None) -> int:
    """Bytes a uniform (rank_map None) or compact TLR matrix would hold (host only)."""
    import numpy as np
    ptr = ctypes.c_void_p(0)
    if rank_map is not None:
        rm = np.ascontiguousarray(rank_map, dtype=np.int32)
        ptr = ctypes.c_void_p(rm.ctypes.data)
    return int(load_library().tlr_mat_plan_bytes(int(n), int(nb), int(maxrank), ptr))


def tlr_mat_ranks(mat: TlrMatrix):
    import numpy as np
    r = np.zeros((mat.nt, mat.nt), dtype=np.int32)
    mat.ctx.check(load_library().tlr_mat_ranks(mat.ctx.h, mat.h, ctypes.c_void_p(r.ctypes.data)))
    return r


def tlr_mat_tile(mat: TlrMatrix, i: int, j: int, stream=None):
    """Tile (i, j) as torch tensors: D (m_i x m_i) for i == j, else (U, V) of the factor."""
    import torch
    nb = mat.nb
    dev = torch.device("cuda", mat.ctx.device)
    # a column-major nb x cols matrix is a row-major (cols, nb) tensor
    a = torch.zeros((nb if i == j else mat.maxrank, nb), dtype=torch.float64, device=dev)
    b = torch.zeros((mat.maxrank, nb), dtype=torch.float64, device=dev) if i != j else None
    r = ctypes.c_int32()
    rc = load_library().tlr_mat_tile(mat.ctx.h, mat.h, int(i), int(j), _ptr(a), _ptr(b), ctypes.byref(r),
                                     _stream(stream))
    mat.ctx.check(rc)
    mi = min(nb, mat.n - i * nb)
    mj = min(nb, mat.n - j * nb)
    if i == j:
        return a.t()[:mi, :mi]
    return a.t()[:mi, :r.value], b.t()[:mj, :r.value]


def tlr_compress(mat: TlrMatrix, tiles, eps_abs: float, stream=None):
    info = ctypes.c_int64(-1)
    rc = load_library().tlr_compress(mat.ctx.h, _ptr(tiles), mat.n, mat.nb, float(eps_abs), mat.h,
                                     ctypes.byref(info), _stream(stream))
    mat.ctx.check(rc, info.value)
    return mat


def tlr_potrf(mat: TlrMatrix, eps_abs: float, stream=None):
    info = ctypes.c_int64(-1)
    rc = load_library().tlr_potrf(mat.ctx.h, mat.h, float(eps_abs), ctypes.byref(info), _stream(stream))
    mat.ctx.check(rc, info.value)
    return mat


def tlr_solve(mat: TlrMatrix, z, y=None, stream=None):
    """y = L^-1 z; returns (y, logdet, quad)."""
    import torch
    _check_f64("z", z, mat.n)
    if y is None:
        y = torch.empty_like(z)
    ld, q = ctypes.c_double(), ctypes.c_double()
    rc = load_library().tlr_solve(mat.ctx.h, mat.h, _ptr(z), _ptr(y), ctypes.byref(ld), ctypes.byref(q),
                                  _stream(stream))
    mat.ctx.check(rc)
    return y, ld.value, q.value


def tlr_lmul(mat: TlrMatrix, w, z=None, stream=None):
    import torch
    _check_f64("w", w, mat.n)
    if z is None:
        z = torch.empty_like(w)
    mat.ctx.check(load_library().tlr_lmul(mat.ctx.h, mat.h, _ptr(w), _ptr(z), _stream(stream)))
    return z


@dataclass
class Options:
    nb: int = 800
    eps: float = 1e-7
    maxrank: int = 0
    precision: int = TLR_PREC_FP64

    def c(self) -> tlr_opts:
        return tlr_opts(int(self.nb), int(self.maxrank), float(self.eps), int(self.precision), 0)


def tlr_loglik(mat: TlrMatrix, xy, z, theta, opts: Options, stream=None) -> dict:
    """l(theta) (Eq. 1.2) for ordered xy / z; `mat` receives the factor."""
    _check_f64("xy", xy, 2 * mat.n)
    _check_f64("z", z, mat.n)
    res = tlr_result()
    o = opts.c()
    rc = load_library().tlr_loglik(mat.ctx.h, _ptr(xy), _ptr(z), mat.n, _theta(theta), ctypes.byref(o), mat.h,
                                   ctypes.byref(res), _stream(stream))
    mat.ctx.check(rc, res.info)
    return res.as_dict()


def tlr_loglik_batch(mats, xys, zs, thetas, opts, stream=None):
    """l(theta_g) (Eq. 1.2) for several ordered datasets on one context, their
    factorisations advanced together (one launch per step for all).  mats,
    xys, zs, thetas: sequences of equal length (1..32); opts: one Options or
    one per entry (same precision).  Returns (results, statuses): a dict per
    entry and its TLR status (entries that fail do not raise; an error of
    the whole call does)."""
    g = len(mats)
    if not (len(xys) == len(zs) == len(thetas) == g):
        raise TlrError(TLR_ERR_ARG, "mats, xys, zs and thetas must have equal lengths")
    ctx = mats[0].ctx
    ol = list(opts) if isinstance(opts, (list, tuple)) else [opts] * g
    for m, x, z in zip(mats, xys, zs):
        _check_f64("xy", x, 2 * m.n)
        _check_f64("z", z, m.n)
    P = ctypes.c_void_p * g
    xa = P(*[x.data_ptr() for x in xys])
    za = P(*[z.data_ptr() for z in zs])
    la = P(*[m.h.value for m in mats])
    na = (ctypes.c_int64 * g)(*[m.n for m in mats])
    ta = (tlr_theta * g)(*[_theta(t) for t in thetas])
    oa = (tlr_opts * g)(*[o.c() for o in ol])
    res = (tlr_result * g)()
    st = (ctypes.c_int * g)()
    rc = load_library().tlr_loglik_batch(ctx.h, g, xa, za, na, ta, oa, la, res, st, _stream(stream))
    if rc != TLR_OK and all(v == rc for v in st) and rc not in (TLR_ERR_NOT_SPD, TLR_ERR_RANK, TLR_ERR_NAN):
        ctx.check(rc)
    return [r.as_dict() for r in res], [int(v) for v in st]


def tlr_loglik_host(mat: TlrMatrix, xy, z, theta, opts: Options, order="hilbert", seed: int = 3,
                    stream=None) -> dict:
    """l(theta) from host arrays (numpy float64 or pinned CPU tensors) in
    generation order: the call copies them to the device, orders and
    evaluates (Sec. 3, Eq. 1.2)."""
    import numpy as np
    xp, zp = _host_ptr(xy, 2 * mat.n), _host_ptr(z, mat.n)
    res = tlr_result()
    o = opts.c()
    method = ORDERS[order] if isinstance(order, str) else int(order)
    rc = load_library().tlr_loglik_host(mat.ctx.h, xp, zp, mat.n, method, int(seed), _theta(theta),
                                        ctypes.byref(o), mat.h, ctypes.byref(res), _stream(stream))
    mat.ctx.check(rc, res.info)
    return res.as_dict()


def _host_ptr(a, numel):
    """Address of a contiguous float64 host array (numpy or CPU tensor) of numel elements."""
    import numpy as np
    if hasattr(a, "data_ptr"):
        if a.device.type != "cpu" or str(a.dtype) != "torch.float64" or not a.is_contiguous() or a.numel() != numel:
            raise TlrError(TLR_ERR_ARG, "host input must be a contiguous float64 CPU tensor of %d elements" % numel)
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.size != numel:
        raise TlrError(TLR_ERR_ARG, "host input must be a contiguous float64 array of %d elements" % numel)
    return ctypes.c_void_p(a.ctypes.data)


def tlr_profile(ctx: Context, enable: bool = True) -> dict:
    ms, fl, me, pl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    ctx.check(load_library().tlr_profile(ctx.h, 1 if enable else 0, ctypes.byref(ms), ctypes.byref(fl),
                                         ctypes.byref(me), ctypes.byref(pl)))
    return {"gemm_ms": ms.value, "gemm_flops": fl.value, "matern_entries": me.value, "panel_launches": pl.value}


STAGES = ("build", "panel", "potrf", "compress", "trsm")


def tlr_stage_times(ctx: Context) -> dict:
    a = (ctypes.c_double * 5)()
    ctx.check(load_library().tlr_stage_times(ctx.h, a))
    return {k: a[i] for i, k in enumerate(STAGES)}


COMPRESS_STEPS = ("sample", "qr_y", "project", "qr_b", "svd", "host", "uv")


def tlr_compress_times(ctx: Context) -> dict:
    a = (ctypes.c_double * 7)()
    ctx.check(load_library().tlr_compress_times(ctx.h, a))
    return {k: a[i] for i, k in enumerate(COMPRESS_STEPS)}


DETAILS = ("build", "correct", "ahead_wait", "solve_update", "split", "panel", "diag_copy", "compress", "join_wait",
           "trsm", "solve", "gram", "potrf", "inverse", "ahead_build", "ahead_panel")


def tlr_detail_times(ctx: Context) -> dict:
    a = (ctypes.c_double * len(DETAILS))()
    n = load_library().tlr_detail_times(ctx.h, a, len(DETAILS))
    if n < 0:
        ctx.check(n)
    return {k: a[i] for i, k in enumerate(DETAILS[:n])}


def tlr_kernel_stats(ctx: Context) -> dict:
    """The 16-CTA cluster Jacobi of the last profiled factorisation."""
    a = (ctypes.c_double * 4)()
    ctx.check(load_library().tlr_kernel_stats(ctx.h, a))
    return {"jacobi16_ms": a[0], "jacobi16_flops": a[1], "jacobi16_launches": int(a[2]),
            "jacobi16_clusters": int(a[3])}


COMPRESS_STATS = ("tiles", "rounds", "sweeps", "max_sweeps", "sweeps32", "qr_global", "svd_global")


def tlr_compress_stats(ctx: Context) -> dict:
    a = (ctypes.c_int64 * len(COMPRESS_STATS))()
    ctx.check(load_library().tlr_compress_stats(ctx.h, a))
    return {k: int(a[i]) for i, k in enumerate(COMPRESS_STATS)}


def tlr_mle(mat: TlrMatrix, xy, z, opts: Options, theta0, lo, hi, tol: float = 1e-9, max_iter: int = 500,
            stream=None) -> dict:
    th, ll, it = tlr_theta(), ctypes.c_double(), ctypes.c_int()
    o = opts.c()
    rc = load_library().tlr_mle(mat.ctx.h, _ptr(xy), _ptr(z), mat.n, ctypes.byref(o), _theta(theta0), _theta(lo),
                                _theta(hi), float(tol), int(max_iter), mat.h, ctypes.byref(th), ctypes.byref(ll),
                                ctypes.byref(it), _stream(stream))
    mat.ctx.check(rc)
    return {"theta": (th.sigma2, th.beta, th.nu), "loglik": ll.value, "iters": it.value}


# ---- many datasets: batched evaluation and serving ----------------------------

POOL_STATS = ("budget", "used", "peak", "resident_data_bytes", "resident_factor_bytes", "resident_factors",
              "evictions", "completed", "queued", "running", "max_running", "allocations", "groups",
              "grouped_requests")


def _pool_check(rc: int):
    if rc != TLR_OK:
        raise TlrError(rc, load_library().tlr_pool_last_error().decode())


def _host_or_device_ptr(a):
    """Address of a contiguous float64 numpy array or torch tensor (host or CUDA)."""
    import numpy as np
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TlrError(TLR_ERR_ARG, "arrays must be contiguous float64")
        return ctypes.c_void_p(a.ctypes.data)
    import torch
    if a.dtype != torch.float64 or not a.is_contiguous():
        raise TlrError(TLR_ERR_ARG, "tensors must be contiguous float64")
    return ctypes.c_void_p(a.data_ptr())


class Pool:
    """Owns a tlr_pool: resident datasets evaluated by concurrent workers."""

    def __init__(self, device: int = 0, workers: int = 4, nb: int = 800, maxrank: int = 0, hbm_budget: int = 0):
        lib = load_library()
        o = tlr_pool_opts(int(workers), int(nb), int(maxrank), 0, int(hbm_budget))
        h = ctypes.c_void_p()
        _pool_check(lib.tlr_pool_create(int(device), ctypes.byref(o), ctypes.byref(h)))
        self.h = h
        self.device = device
        self._keep = []

    def close(self):
        if getattr(self, "h", None):
            load_library().tlr_pool_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tlr_pool_create(device: int = 0, workers: int = 4, nb: int = 800, maxrank: int = 0, hbm_budget: int = 0) -> Pool:
    return Pool(device, workers, nb, maxrank, hbm_budget)


def tlr_pool_destroy(pool: Pool):
    pool.close()


def tlr_pool_add(pool: Pool, xy, z, order="morton", seed: int = 3, nb: int = 0) -> int:
    """Register a dataset (xy SoA 2n and z n, float64 numpy or torch, host or CUDA); returns its id."""
    n = z.shape[0] if hasattr(z, "shape") else len(z)
    if (xy.numel() if hasattr(xy, "numel") else xy.size) != 2 * n:
        raise TlrError(TLR_ERR_ARG, "xy must hold 2n values")
    if isinstance(order, str):
        order = ORDERS[order]
    i = ctypes.c_int(-1)
    _pool_check(load_library().tlr_pool_add(pool.h, _host_or_device_ptr(xy), _host_or_device_ptr(z), int(n),
                                            int(order), ctypes.c_uint64(seed & (2**64 - 1)), int(nb),
                                            ctypes.byref(i)))
    return i.value


def tlr_pool_remove(pool: Pool, id: int):
    _pool_check(load_library().tlr_pool_remove(pool.h, int(id)))


def tlr_pool_dataset(pool: Pool, id: int) -> dict:
    """The dataset's resident data as CUDA tensors (views of the pool's memory; read while it is idle)."""
    import torch
    n, nb, mr = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int32()
    xy, z, perm = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _pool_check(load_library().tlr_pool_dataset(pool.h, int(id), ctypes.byref(n), ctypes.byref(nb),
                                                ctypes.byref(xy), ctypes.byref(z), ctypes.byref(perm),
                                                ctypes.byref(mr)))
    dev = torch.device("cuda", pool.device)

    def copy(addr, count, typestr):
        # a zero-copy view through the CUDA array interface, then an owned copy
        buf = _CudaArray(addr, count, typestr)
        return torch.as_tensor(buf, device=dev).clone()

    N = n.value
    return {"n": N, "nb": nb.value, "last_max_rank": mr.value,
            "xy": copy(xy.value, 2 * N, "<f8"), "z": copy(z.value, N, "<f8"), "perm": copy(perm.value, N, "<i8")}


class _CudaArray:
    def __init__(self, addr: int, count: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr, "data": (addr, False),
                                         "version": 2, "strides": None}


def tlr_pool_submit(pool: Pool, id: int, theta, eps: float = 1e-7, precision: int = TLR_PREC_FP64) -> int:
    t = ctypes.c_int64()
    _pool_check(load_library().tlr_pool_submit(pool.h, int(id), _theta(theta), float(eps), int(precision),
                                               ctypes.byref(t)))
    return t.value


def tlr_pool_wait(pool: Pool, ticket: int):
    """Block for a request; returns (result dict, times_ms dict).  Raises TlrError if it failed."""
    res = tlr_result()
    tm = (ctypes.c_double * 3)()
    rc = load_library().tlr_pool_wait(pool.h, int(ticket), ctypes.byref(res), tm)
    if rc != TLR_OK:
        raise TlrError(rc, load_library().tlr_pool_last_error().decode(), res.info)
    return res.as_dict(), {"queue_ms": tm[0], "run_ms": tm[1], "latency_ms": tm[2]}


def tlr_pool_loglik(pool: Pool, ids, thetas, eps: float = 1e-7, precision: int = TLR_PREC_FP64):
    """Batched evaluation; returns (list of result dicts, list of status codes)."""
    cnt = len(ids)
    ida = (ctypes.c_int * cnt)(*[int(i) for i in ids])
    tha = (tlr_theta * cnt)(*[_theta(t) for t in thetas])
    out = (tlr_result * cnt)()
    st = (ctypes.c_int * cnt)()
    load_library().tlr_pool_loglik(pool.h, cnt, ida, tha, float(eps), int(precision), out, st)
    return [out[i].as_dict() for i in range(cnt)], [st[i] for i in range(cnt)]


def tlr_pool_mle(pool: Pool, id: int, theta0, lo, hi, eps: float = 1e-7, precision: int = TLR_PREC_FP64,
                 tol: float = 1e-9, max_iter: int = 200):
    th, ll, it = tlr_theta(), ctypes.c_double(), ctypes.c_int()
    _pool_check(load_library().tlr_pool_mle(pool.h, int(id), float(eps), int(precision), _theta(theta0),
                                            _theta(lo), _theta(hi), float(tol), int(max_iter), ctypes.byref(th),
                                            ctypes.byref(ll), ctypes.byref(it)))
    return (th.sigma2, th.beta, th.nu), ll.value, it.value


def tlr_pool_tune(pool: Pool, id: int, theta, cands, eps: float = 1e-7, precision: int = TLR_PREC_FP64):
    """Tile-size autotuning of one dataset; returns (best nb, {nb: ms})."""
    k = len(cands)
    ca = (ctypes.c_int32 * k)(*[int(c) for c in cands])
    ms = (ctypes.c_double * k)()
    best = ctypes.c_int32()
    _pool_check(load_library().tlr_pool_tune(pool.h, int(id), _theta(theta), float(eps), int(precision), ca, k,
                                             ctypes.byref(best), ms))
    return best.value, {int(cands[i]): ms[i] for i in range(k)}


def _buckets(b):
    if b is None or isinstance(b, tlr_buckets):
        return b
    return tlr_buckets(*[(ctypes.c_int32 * 4)(*[int(v) for v in b[f]]) for f, _ in tlr_buckets._fields_])


def tlr_pool_configure(pool: Pool, group: int = 1, buckets=None):
    """Requests a worker evaluates together (tlr_loglik_batch) and the rank
    buckets of every worker's context (None: the default)."""
    b = _buckets(buckets)
    _pool_check(load_library().tlr_pool_configure(pool.h, int(group), None if b is None else ctypes.byref(b)))


def tlr_pool_get_config(pool: Pool) -> dict:
    g, b = ctypes.c_int(), tlr_buckets()
    _pool_check(load_library().tlr_pool_get_config(pool.h, ctypes.byref(g), ctypes.byref(b)))
    return {"group": g.value, "buckets": b.as_dict()}


def tlr_pool_autotune(pool: Pool, ids, thetas, candidates, eps: float = 1e-7, precision: int = TLR_PREC_FP64,
                      rounds: int = 1):
    """Throughput tuning over candidates [(group, buckets or None), ...] on the
    requests (ids[i], thetas[i]); the pool keeps the fastest.  Returns
    (best index, evals/s per candidate)."""
    k, c = len(ids), len(candidates)
    ia = (ctypes.c_int * k)(*[int(i) for i in ids])
    ta = (tlr_theta * k)(*[_theta(t) for t in thetas])
    ga = (ctypes.c_int32 * c)(*[int(g) for g, _ in candidates])
    cur = tlr_pool_get_config(pool)["buckets"]
    ba = (tlr_buckets * c)(*[_buckets(b if b is not None else cur) for _, b in candidates])
    rates = (ctypes.c_double * c)()
    best = ctypes.c_int()
    _pool_check(load_library().tlr_pool_autotune(pool.h, k, ia, ta, float(eps), int(precision), c, ga, ba,
                                                 int(rounds), rates, ctypes.byref(best)))
    return best.value, [rates[i] for i in range(c)]


def tlr_pool_footprint(n: int, nb: int, maxrank: int = 0) -> dict:
    """Bytes the pool's admission charges for a dataset: resident data, factor storage, first workspace estimate."""
    a = (ctypes.c_int64 * 3)()
    _pool_check(load_library().tlr_pool_footprint(int(n), int(nb), int(maxrank), a))
    return {"base": a[0], "factor": a[1], "work": a[2]}


def tlr_pool_stats(pool: Pool) -> dict:
    a = (ctypes.c_int64 * len(POOL_STATS))()
    k = load_library().tlr_pool_stats(pool.h, a, len(POOL_STATS))
    if k < 0:
        _pool_check(k)
    return {POOL_STATS[i]: a[i] for i in range(k)}


def tlr_shard_place(footprints, nranks: int, budgets=None):
    """Rank of every dataset (host only): largest footprint first onto the
    least-loaded rank with room (tlr_shard_place)."""
    import numpy as np
    b = np.ascontiguousarray(footprints, dtype=np.int64)
    out = np.zeros(len(b), dtype=np.int32)
    bud = None if budgets is None else np.ascontiguousarray(budgets, dtype=np.int64)
    vp = lambda a: ctypes.c_void_p(a.ctypes.data)
    _pool_check(load_library().tlr_shard_place(len(b), vp(b), int(nranks), None if bud is None else vp(bud), vp(out)))
    return out


def tlr_sched_simulate(budget: int, workers: int, base, factor, work, req_data, req_arrival, req_cost):
    """Host-only simulation of the pool's admission policy; returns (start, finish, peak, evictions)."""
    import numpy as np
    base = np.ascontiguousarray(base, dtype=np.int64)
    factor = np.ascontiguousarray(factor, dtype=np.int64)
    work = np.ascontiguousarray(work, dtype=np.int64)
    rd = np.ascontiguousarray(req_data, dtype=np.int32)
    ra = np.ascontiguousarray(req_arrival, dtype=np.float64)
    rc_ = np.ascontiguousarray(req_cost, dtype=np.float64)
    start = np.zeros(len(rd))
    finish = np.zeros(len(rd))
    peak, ev = ctypes.c_int64(), ctypes.c_int64()
    vp = lambda a: ctypes.c_void_p(a.ctypes.data)
    rc = load_library().tlr_sched_simulate(int(budget), int(workers), len(base), vp(base), vp(factor), vp(work),
                                           len(rd), vp(rd), vp(ra), vp(rc_), vp(start), vp(finish),
                                           ctypes.byref(peak), ctypes.byref(ev))
    _pool_check(rc)
    return start, finish, peak.value, ev.value
