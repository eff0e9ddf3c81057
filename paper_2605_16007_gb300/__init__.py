"""Python binding of librq (IVF-RaBitQ on one GB300).

Argument marshalling only: every computation runs in the CUDA library
behind the C ABI declared in ``include/rq.h``. The module-level functions
carry the C names (``rq_build``, ``rq_search``, ...); ``Index`` and
``Server`` wrap them for convenience. Arrays may be numpy arrays (host) or
torch tensors (host or CUDA); outputs are allocated by the caller or here.

Importing the module does not need a GPU. Loading the library needs it to be
built (``build()``); a missing library raises instead of falling back to
anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB, build  # noqa: F401

RQ_OK, RQ_ERR_INVALID_ARG, RQ_ERR_OOM, RQ_ERR_CUDA, RQ_ERR_TIMEOUT = 0, 1, 2, 3, 4
RQ_ERR_BUSY, RQ_ERR_IO, RQ_ERR_NOT_IMPLEMENTED, RQ_ERR_DEVICE = 5, 6, 7, 8
RQ_F32, RQ_U8 = 0, 1
RQ_SCAN_AUTO, RQ_SCAN_PLAIN, RQ_SCAN_GROUPED, RQ_SCAN_MMA = 0, 1, 2, 3
RQ_EST_BQ4, RQ_EST_LUT = 0, 1


class RQError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"rq status {status}: {msg}")
        self.status = status


class BuildOpts(C.Structure):
    _fields_ = [("kmeans_iters", C.c_int32), ("keep_float_raw", C.c_int32),
                ("train_size", C.c_int64), ("raw_on_host", C.c_int32)]


class SearchDump(C.Structure):
    _fields_ = [("qrot", C.c_void_p), ("probe_ids", C.c_void_p),
                ("probe_dist", C.c_void_p), ("qparams", C.c_void_p),
                ("planes", C.c_void_p), ("bound", C.c_void_p),
                ("selected", C.c_void_p), ("n_candidates", C.c_void_p)]


class SearchOpts(C.Structure):
    _fields_ = [("scan_mode", C.c_int32), ("no_prune", C.c_int32),
                ("use_graph", C.c_int32), ("test_stall", C.c_int32),
                ("dump", C.POINTER(SearchDump)), ("stage_ms", C.POINTER(C.c_float)),
                ("plain_chunk", C.c_int32), ("estimator", C.c_int32)]


STAGES = ("rotate", "probe", "quantize", "bound", "worklist", "scan", "select", "rerank")


class Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("dim", C.c_int32), ("dim_pad", C.c_int32),
                ("nlist", C.c_int32), ("code_bytes", C.c_int32),
                ("min_list", C.c_int64), ("max_list", C.c_int64),
                ("index_bytes", C.c_int64), ("raw_bytes", C.c_int64),
                ("auto_scan_mode", C.c_int32), ("reserved", C.c_int32)]


class IndexView(C.Structure):
    _fields_ = [("n", C.c_int64), ("dim", C.c_int32), ("dim_pad", C.c_int32),
                ("nlist", C.c_int32), ("code_bytes", C.c_int32),
                ("P", C.c_void_p), ("centroids", C.c_void_p), ("cR", C.c_void_p),
                ("offsets", C.c_void_p), ("codes", C.c_void_p), ("r", C.c_void_p),
                ("alpha", C.c_void_p), ("factors", C.c_void_p), ("ids", C.c_void_p),
                ("assign", C.c_void_p), ("raw", C.c_void_p),
                ("raw_dtype", C.c_int32), ("reserved", C.c_int32)]


class ServerOpts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("max_batch", C.c_int32),
                ("memory_budget", C.c_int64), ("max_queue", C.c_int32),
                ("scan_mode", C.c_int32)]


_lib = None

_SIGS = {
    "rq_build": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_int32, C.c_int32,
                           C.c_uint64, C.POINTER(BuildOpts), C.POINTER(C.c_void_p)]),
    "rq_build_with": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_int32, C.c_int32,
                                C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "rq_kmeans": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_uint64,
                            C.c_int32, C.c_int64, C.c_void_p]),
    "rq_philox_gaussian": (C.c_int, [C.c_uint64, C.c_uint32, C.c_int64, C.c_void_p]),
    "rq_search": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int32,
                            C.c_int32, C.c_void_p, C.c_void_p, C.POINTER(SearchOpts),
                            C.c_void_p]),
    "rq_search_mixed": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                  C.c_void_p, C.POINTER(SearchOpts), C.c_void_p]),
    "rq_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int32,
                              C.c_char_p]),
    "rq_get_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "rq_get_view": (C.c_int, [C.c_void_p, C.POINTER(IndexView)]),
    "rq_export": (C.c_int, [C.c_void_p, C.c_char_p]),
    "rq_import": (C.c_int, [C.c_char_p, C.POINTER(C.c_void_p)]),
    "rq_free": (None, [C.c_void_p]),
    "rq_device_error": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "rq_status_str": (C.c_char_p, [C.c_int]),
    "rq_last_error": (C.c_char_p, []),
    "rq_version": (C.c_int32, []),
    "rq_server_create": (C.c_int, [C.c_void_p, C.POINTER(ServerOpts),
                                   C.POINTER(C.c_void_p)]),
    "rq_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int32,
                            C.c_int32, C.POINTER(C.c_uint64)]),
    "rq_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_int32,
                          C.POINTER(C.c_double)]),
    "rq_server_destroy": (None, [C.c_void_p]),
    "rq_probe_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                  C.c_void_p, C.c_void_p, C.c_void_p]),
    "rq_test_fail_allocations": (None, [C.c_int64]),
}


def lib():
    """The loaded librq (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"librq.so not found at {LIB}: run "
                               "paper_2605_16007_gb300.build() first")
        L = C.CDLL(LIB)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != RQ_OK:
        raise RQError(status, lib().rq_last_error().decode(errors="replace"))


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _shape(a):
    return tuple(a.shape)


def _is_u8(a):
    dt = getattr(a, "dtype", None)
    return str(dt) in ("uint8", "torch.uint8")


# ------------------------------------------------------------------ C names
def rq_build(base, nlist: int, seed: int, kmeans_iters: int = 10,
             train_size: int = 0, keep_float_raw: bool = False,
             raw_on_host: bool = False) -> "Index":
    """raw_on_host: `base` is a page-locked host buffer (a pinned torch CPU
    tensor, for instance) that the index's re-rank reads in place; keep it
    alive and unchanged while the index lives."""
    n, dim = _shape(base)
    opts = BuildOpts(kmeans_iters, int(keep_float_raw), train_size, int(raw_on_host))
    h = C.c_void_p()
    _check(lib().rq_build(_ptr(base), RQ_U8 if _is_u8(base) else RQ_F32, n, dim, nlist,
                          seed, C.byref(opts), C.byref(h)))
    return Index(h)


def rq_build_with(base, centroids, P) -> "Index":
    n, dim = _shape(base)
    nlist = _shape(centroids)[0]
    h = C.c_void_p()
    _check(lib().rq_build_with(_ptr(base), RQ_U8 if _is_u8(base) else RQ_F32, n, dim,
                               nlist, _ptr(centroids), _ptr(P), C.byref(h)))
    return Index(h)


def rq_kmeans(base, nlist: int, seed: int, iters: int = 10, train_size: int = 0,
              out=None):
    n, dim = _shape(base)
    if out is None:
        out = np.empty((nlist, dim), np.float32)
    _check(lib().rq_kmeans(_ptr(base), n, dim, nlist, seed, iters, train_size, _ptr(out)))
    return out


def rq_philox_gaussian(seed: int, stream: int, count: int, out=None):
    if out is None:
        out = np.empty(count, np.float64)
    _check(lib().rq_philox_gaussian(seed, stream, count, _ptr(out)))
    return out


def rq_import(path: str) -> "Index":
    h = C.c_void_p()
    _check(lib().rq_import(path.encode(), C.byref(h)))
    return Index(h)


def rq_status_str(status: int) -> str:
    return lib().rq_status_str(status).decode()


def rq_version() -> int:
    return lib().rq_version()


def rq_test_fail_allocations(after: int):
    """Test hook: the after-th next device allocation of the library fails
    (-1 disarms); see include/rq.h."""
    lib().rq_test_fail_allocations(after)


def _opts(scan_mode, no_prune, use_graph, dump, stage_ms=None, test_stall=False, plain_chunk=0,
          estimator=RQ_EST_BQ4):
    o = SearchOpts(scan_mode, int(no_prune), int(use_graph), int(test_stall), None, None,
                   int(plain_chunk), int(estimator))
    if stage_ms is not None:
        o.stage_ms = stage_ms
    if dump is not None:
        d = SearchDump(*[_ptr(dump.get(f)) if dump.get(f) is not None else None
                         for f, _ in SearchDump._fields_])
        o._dump_keep = d
        o.dump = C.pointer(d)
    return o


class Index:
    """An index on the GPU; frees itself when garbage-collected."""

    def __init__(self, handle: C.c_void_p):
        self.h = handle

    # -- search ----------------------------------------------------------
    def rq_search(self, queries, nprobe: int, k: int, n_rerank: int, out_ids=None,
                  out_dist=None, scan_mode: int = RQ_SCAN_AUTO, no_prune: bool = False,
                  use_graph: bool = False, dump=None, stream=None, stage_times=None,
                  test_stall: bool = False, plain_chunk: int = 0, estimator: int = RQ_EST_BQ4):
        """stage_times: a dict that receives each stage's device time (ms).
        test_stall: the failure-path test hook of rq_search_opts."""
        nq = _shape(queries)[0]
        if out_ids is None:
            out_ids = np.empty((nq, k), np.int64)
            out_dist = np.empty((nq, k), np.float32)
        ms = (C.c_float * len(STAGES))() if stage_times is not None else None
        o = _opts(scan_mode, no_prune, use_graph, dump, ms, test_stall, plain_chunk, estimator)
        _check(lib().rq_search(self.h, _ptr(queries), nq, nprobe, k, n_rerank,
                               _ptr(out_ids), _ptr(out_dist), C.byref(o),
                               _stream_ptr(stream)))
        if stage_times is not None:
            stage_times.update({name: ms[i] for i, name in enumerate(STAGES)})
        return out_ids, out_dist

    search = rq_search

    def rq_search_mixed(self, queries, nprobe, k, n_rerank, k_stride=None, out_ids=None,
                        out_dist=None, scan_mode: int = RQ_SCAN_AUTO,
                        no_prune: bool = False, use_graph: bool = False, dump=None,
                        stream=None, stage_times=None, plain_chunk: int = 0,
                        estimator: int = RQ_EST_BQ4):
        nq = _shape(queries)[0]
        nprobe = np.ascontiguousarray(nprobe, np.int32)
        k = np.ascontiguousarray(k, np.int32)
        n_rerank = np.ascontiguousarray(n_rerank, np.int32)
        if k_stride is None:
            k_stride = int(k.max())
        if out_ids is None:
            out_ids = np.empty((nq, k_stride), np.int64)
            out_dist = np.empty((nq, k_stride), np.float32)
        ms = (C.c_float * len(STAGES))() if stage_times is not None else None
        o = _opts(scan_mode, no_prune, use_graph, dump, ms, False, plain_chunk, estimator)
        _check(lib().rq_search_mixed(self.h, _ptr(queries), nq, _ptr(nprobe), _ptr(k),
                                     _ptr(n_rerank), k_stride, _ptr(out_ids),
                                     _ptr(out_dist), C.byref(o), _stream_ptr(stream)))
        if stage_times is not None:
            stage_times.update({name: ms[i] for i, name in enumerate(STAGES)})
        return out_ids, out_dist

    search_mixed = rq_search_mixed

    def rq_autotune(self, queries, nprobe: int, n_rerank: int, cache_path=None):
        _check(lib().rq_autotune(self.h, _ptr(queries), _shape(queries)[0], nprobe,
                                 n_rerank, cache_path.encode() if cache_path else None))

    autotune = rq_autotune

    def rq_probe_static(self, queries, nprobe: int, out_ids, out_dist, stream=None):
        """Rotation + centroid ranking without any allocation (device arrays
        only); see rq_probe_static in include/rq.h.

        The C entry point sees bare pointers, so the shapes, dtypes and
        device are checked here: queries a contiguous float32 CUDA tensor of
        shape (nq, dim), out_ids int32 and out_dist float32 CUDA tensors of
        shape (nq, nprobe), all on the current device (the library checks
        that the current device holds the index)."""
        import torch

        dev = torch.cuda.current_device()
        nq = _shape(queries)[0] if hasattr(queries, "shape") else -1
        _require_cuda(queries, "queries", "torch.float32", (nq, self.stats()["dim"]), dev)
        _require_cuda(out_ids, "out_ids", "torch.int32", (nq, nprobe), dev)
        _require_cuda(out_dist, "out_dist", "torch.float32", (nq, nprobe), dev)
        _check(lib().rq_probe_static(self.h, _ptr(queries), nq, nprobe,
                                     _ptr(out_ids), _ptr(out_dist), _stream_ptr(stream)))
        return out_ids, out_dist

    probe_static = rq_probe_static

    # -- inspection --------------------------------------------------------
    def stats(self) -> dict:
        s = Stats()
        _check(lib().rq_get_stats(self.h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def view(self) -> dict:
        v = IndexView()
        _check(lib().rq_get_view(self.h, C.byref(v)))
        return {f: getattr(v, f) for f, _ in IndexView._fields_}

    def offsets(self) -> np.ndarray:
        """List offsets (nlist + 1) copied to the host."""
        v = self.view()
        out = np.empty(v["nlist"] + 1, np.int64)
        memcpy_d2h(out, v["offsets"])
        return out

    def to_host(self) -> dict:
        """Host copies (numpy) of the index arrays, read through the view."""
        v = self.view()
        n, dim, dp, nl, cb = v["n"], v["dim"], v["dim_pad"], v["nlist"], v["code_bytes"]

        def grab(ptr, count, dtype):
            out = np.empty(count, dtype)
            memcpy_d2h(out, ptr)
            return out

        raw_dt = np.uint8 if v["raw_dtype"] == RQ_U8 else np.float32
        return dict(
            n=n, dim=dim, dp=dp, nlist=nl,
            P=grab(v["P"], dp * dp, np.float64).reshape(dp, dp),
            centroids=grab(v["centroids"], nl * dim, np.float32).reshape(nl, dim),
            cR=grab(v["cR"], nl * dp, np.float32).reshape(nl, dp),
            offsets=grab(v["offsets"], nl + 1, np.int64),
            codes=grab(v["codes"], n * cb, np.uint8).reshape(n, cb),
            r=grab(v["r"], n, np.float32),
            alpha=grab(v["alpha"], n, np.float32),
            factors=grab(v["factors"], 2 * n, np.float32).reshape(n, 2),
            ids=grab(v["ids"], n, np.uint32).astype(np.int64),
            assign=grab(v["assign"], n, np.int32),
            raw=grab(v["raw"], n * dim, raw_dt).reshape(n, dim),
        )

    def rq_export(self, path: str):
        _check(lib().rq_export(self.h, path.encode()))

    export = rq_export

    def rq_device_error(self) -> int:
        c = C.c_int32()
        _check(lib().rq_device_error(self.h, C.byref(c)))
        return c.value

    device_error = rq_device_error

    def rq_free(self):
        if self.h:
            lib().rq_free(self.h)
            self.h = None

    free = rq_free

    def __del__(self):
        try:
            self.rq_free()
        except Exception:
            pass


def _require_cuda(t, name, dtype, shape, device):
    """Raises ValueError unless t is a contiguous CUDA tensor of the given
    dtype (as its str) and shape on CUDA device `device`."""
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise ValueError(f"{name} must be a CUDA tensor")
    if str(t.dtype) != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, not {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, not {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.device.index != device:
        raise ValueError(f"{name} is on cuda:{t.device.index}, the index on cuda:{device}")


_cudart = None


def _load_cudart():
    global _cudart
    if _cudart is None:
        import torch  # noqa: F401  (loads the CUDA runtime library)
        for name in ("libcudart.so.13", "libcudart.so.12", "libcudart.so"):
            try:
                _cudart = C.CDLL(name)
                break
            except OSError:
                continue
        if _cudart is None:
            raise RuntimeError("CUDA runtime library not found")
        _cudart.cudaMemcpy.restype = C.c_int
        _cudart.cudaMemcpy.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]
    return _cudart


def memcpy_d2h(dst: np.ndarray, src_ptr: int):
    """Copy device memory at src_ptr into the host array dst (CUDA runtime)."""
    if dst.nbytes == 0:
        return
    rc = _load_cudart().cudaMemcpy(C.c_void_p(dst.ctypes.data), C.c_void_p(src_ptr), dst.nbytes, 4)
    if rc != 0:
        raise RuntimeError(f"cudaMemcpy failed with {rc}")


class Server:
    """Continuous-batching server over an index (rq_server_*)."""

    def __init__(self, index: Index, slots=4, max_batch=1024, memory_budget=0,
                 max_queue=65536, scan_mode=RQ_SCAN_AUTO):
        self.index = index
        o = ServerOpts(slots, max_batch, memory_budget, max_queue, scan_mode)
        self.h = C.c_void_p()
        _check(lib().rq_server_create(index.h, C.byref(o), C.byref(self.h)))
        self._shapes = {}

    def rq_submit(self, queries: np.ndarray, nprobe: int, k: int, n_rerank: int) -> int:
        q = np.ascontiguousarray(queries, np.float32)
        t = C.c_uint64()
        _check(lib().rq_submit(self.h, _ptr(q), q.shape[0], nprobe, k, n_rerank, C.byref(t)))
        self._shapes[t.value] = (q.shape[0], k)
        return t.value

    submit = rq_submit

    def rq_wait(self, ticket: int, timeout_ms: int = -1):
        nq, k = self._shapes[ticket]
        ids = np.empty((nq, k), np.int64)
        dist = np.empty((nq, k), np.float32)
        lat = C.c_double()
        _check(lib().rq_wait(self.h, ticket, _ptr(ids), _ptr(dist), timeout_ms, C.byref(lat)))
        del self._shapes[ticket]
        return ids, dist, lat.value

    wait = rq_wait

    def close(self):
        if self.h:
            lib().rq_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
