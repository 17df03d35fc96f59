"""Python binding of the EBIC GB300 C ABI (include/ebic.h), argument marshalling only.

Every ``ebic_*`` function below has the name and meaning of the C entry point it calls; arrays
may be numpy arrays (host memory) or torch tensors (host or CUDA memory of the context's device),
passed by pointer.  All computation happens in the CUDA kernels of ``libebic_gb300.so``: this
module fails loudly (ImportError) when that library is missing, and never computes a result.
``Context`` wraps the same calls for convenience.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libebic_gb300.so")

EBIC_OK = 0
EBIC_EINVAL = -1
EBIC_ENAN = -2
EBIC_ENOMEM = -3
EBIC_ECUDA = -4
EBIC_ETIMEOUT = -5
EBIC_ESTATE = -6

MODE_AUTO, MODE_DIRECT, MODE_BITMAP, MODE_PLAIN, MODE_STAGED = 0, 1, 2, 3, 4
ROW_MAJOR, COL_MAJOR = 0, 1
MAX_LEN = 64

_ERR_NAMES = {-1: "EBIC_EINVAL", -2: "EBIC_ENAN", -3: "EBIC_ENOMEM", -4: "EBIC_ECUDA",
              -5: "EBIC_ETIMEOUT", -6: "EBIC_ESTATE"}


class EbicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("neg_trends", ctypes.c_int32), ("ratio_num", ctypes.c_int32),
                ("ratio_den", ctypes.c_int32), ("min_rows", ctypes.c_int32),
                ("col_cap", ctypes.c_int32), ("overlap_num", ctypes.c_int32),
                ("overlap_den", ctypes.c_int32), ("n_biclusters", ctypes.c_int32),
                ("init_min_len", ctypes.c_int32), ("init_max_len", ctypes.c_int32),
                ("max_len", ctypes.c_int32), ("pop_size", ctypes.c_int32),
                ("elite", ctypes.c_int32), ("tournament", ctypes.c_int32),
                ("max_attempts", ctypes.c_int32), ("tabu_hit_limit", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("mode", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("non_strict", ctypes.c_int32),
                ("last_kept", ctypes.c_int32), ("ipw", ctypes.c_int32),
                ("fuse_pairs", ctypes.c_int32)]

    @classmethod
    def make(cls, **kw):
        p = cls()
        _lib.ebic_default_params(ctypes.byref(p))
        for k, v in kw.items():
            if not hasattr(p, k):
                raise AttributeError(k)
            setattr(p, k, int(v))
        return p

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class RunReport(ctypes.Structure):
    _fields_ = [("gens_done", ctypes.c_int32), ("stopped", ctypes.c_int32),
                ("last_hits", ctypes.c_int32), ("n_top", ctypes.c_int32),
                ("n_evaluated", ctypes.c_int64), ("eval_mode", ctypes.c_int32),
                ("fuse_pairs", ctypes.c_int32), ("n_fused", ctypes.c_int64),
                ("n_table", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_VP = ctypes.c_void_p
_I32, _I64 = ctypes.c_int32, ctypes.c_int64

# name -> (restype, argtypes), mirroring include/ebic.h
SIGNATURES = {
    "ebic_default_params": (None, [_VP]),
    "ebic_version": (ctypes.c_char_p, []),
    "ebic_create": (ctypes.c_int, [_VP, _I32, _VP]),
    "ebic_destroy": (ctypes.c_int, [_VP]),
    "ebic_last_error": (ctypes.c_char_p, [_VP]),
    "ebic_load_matrix": (ctypes.c_int, [_VP, _VP, _I64, _I32, _I32]),
    "ebic_build_bitmap": (ctypes.c_int, [_VP]),
    "ebic_bitmap_bytes": (ctypes.c_int64, [_I64, _I32]),
    "ebic_copy_bitmap": (ctypes.c_int, [_VP, _VP, _I64]),
    "ebic_copy_pair_counts": (ctypes.c_int, [_VP, _VP, _I64]),
    "ebic_eval_population": (ctypes.c_int, [_VP, _VP, _VP, _I32, _VP, _VP, _VP, _VP, _VP]),
    "ebic_run_generations": (ctypes.c_int, [_VP, _VP, _I32, _VP]),
    "ebic_get_toplist": (ctypes.c_int, [_VP, _I32, _VP, _VP, _VP, _VP, _VP, _VP]),
    "ebic_get_population": (ctypes.c_int, [_VP, _I32, _VP, _VP, _VP, _VP]),
    "ebic_extract_biclusters": (ctypes.c_int, [_VP, _I32, _VP, _VP]),
    "ebic_state_bytes": (ctypes.c_int64, [_VP]),
    "ebic_save_state": (ctypes.c_int, [_VP, _VP, _I64]),
    "ebic_load_state": (ctypes.c_int, [_VP, _VP, _VP, _I64]),
    "ebic_profile_enable": (ctypes.c_int, [_VP, _I32]),
    "ebic_profile_read": (ctypes.c_int, [_VP, _I32, _VP]),
    "ebic_autotune": (ctypes.c_int, [_VP, _VP, _VP, _I32, _VP, _I32, _VP]),
    "ebic_job_footprint": (ctypes.c_int64, [_I64, _I32, _VP, _I32]),
    "ebic_server_create": (ctypes.c_int, [_VP, _I32, _I64, _I32]),
    "ebic_server_destroy": (ctypes.c_int, [_VP]),
    "ebic_server_submit": (ctypes.c_int, [_VP, _VP, _I64, _I32, _I32, _VP, _I32, _VP]),
    "ebic_server_wait": (ctypes.c_int, [_VP, _I64, _I32, _VP, _I32, _VP, _VP, _VP, _VP, _VP]),
    "ebic_server_stats": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "ebic_eval_population_noalloc": (ctypes.c_int, [_VP, _I64, _I32, _VP, _VP, _I32, _VP, _VP,
                                                    _VP, _VP, _VP, _I32, _VP, _VP, _I32]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built: run `python -m paper_2105_01196_gb300.build`"
                          " (the CUDA library is required; there is no fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        if hasattr(lib, name):
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
    return lib


_lib = _load()


def lib():
    return _lib


# ----------------------------------------------------------------------------- marshalling

def _is_torch(a):
    return type(a).__module__.startswith("torch")


def ptr(a):
    """Address of an array argument: torch tensor, numpy array, ctypes object or None."""
    if a is None:
        return None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if isinstance(a, int):
        return a
    return ctypes.addressof(a)


def _check(ctx, status):
    if status != EBIC_OK:
        msg = _lib.ebic_last_error(ctx).decode() if ctx else ""
        raise EbicError(status, msg)
    return status


def _as_dtype(a, np_dtype, torch_name):
    if a is None:
        return None
    if _is_torch(a):
        if str(a.dtype) != f"torch.{torch_name}":
            raise TypeError(f"expected torch.{torch_name}, got {a.dtype}")
        return a
    return np.ascontiguousarray(a, dtype=np_dtype)


# ----------------------------------------------------------------------------- the C names

def ebic_version():
    return _lib.ebic_version().decode()


def ebic_default_params():
    return Params.make()


def ebic_create(device=0, stream=None):
    out = ctypes.c_void_p()
    _check(None, _lib.ebic_create(ctypes.byref(out), int(device), stream))
    return out.value


def ebic_destroy(ctx):
    return _lib.ebic_destroy(ctx)


def ebic_last_error(ctx):
    return _lib.ebic_last_error(ctx).decode()


def ebic_load_matrix(ctx, x, layout=ROW_MAJOR):
    x = _as_dtype(x, np.float32, "float32")
    if layout == ROW_MAJOR:
        rows, cols = x.shape
    else:
        cols, rows = x.shape
    _check(ctx, _lib.ebic_load_matrix(ctx, ptr(x), int(rows), int(cols), int(layout)))


def ebic_build_bitmap(ctx):
    _check(ctx, _lib.ebic_build_bitmap(ctx))


def ebic_bitmap_bytes(rows, cols):
    return int(_lib.ebic_bitmap_bytes(int(rows), int(cols)))


def ebic_copy_bitmap(ctx, out):
    _check(ctx, _lib.ebic_copy_bitmap(ctx, ptr(out), int(out.numel() if _is_torch(out) else out.size)))
    return out


def ebic_copy_pair_counts(ctx, out):
    _check(ctx, _lib.ebic_copy_pair_counts(ctx, ptr(out),
                                           int(out.numel() if _is_torch(out) else out.size)))
    return out


def ebic_eval_population(ctx, col_idx, offsets, params, rows_pos=None, rows_neg=None,
                         rows_any=None, fitness=None):
    """Evaluates a CSR population.  With no outputs given, returns four new numpy arrays."""
    col_idx = _as_dtype(col_idx, np.int32, "int32")
    offsets = _as_dtype(offsets, np.int32, "int32")
    n = (offsets.numel() if _is_torch(offsets) else offsets.size) - 1
    if rows_pos is None and rows_neg is None and rows_any is None and fitness is None:
        rows_pos = np.zeros(n, np.int32)
        rows_neg = np.zeros(n, np.int32)
        rows_any = np.zeros(n, np.int32)
        fitness = np.zeros(n, np.uint64)
    _check(ctx, _lib.ebic_eval_population(ctx, ptr(col_idx), ptr(offsets), int(n),
                                          ctypes.byref(params), ptr(rows_pos), ptr(rows_neg),
                                          ptr(rows_any), ptr(fitness)))
    return rows_pos, rows_neg, rows_any, fitness


def ebic_run_generations(ctx, params, n_gen):
    rep = RunReport()
    _check(ctx, _lib.ebic_run_generations(ctx, ctypes.byref(params), int(n_gen),
                                          ctypes.byref(rep)))
    return rep


def ebic_get_toplist(ctx, capacity=256):
    cols = np.zeros((capacity, MAX_LEN), np.int32)
    lens = np.zeros(capacity, np.int32)
    fit = np.zeros(capacity, np.uint64)
    keys = np.zeros(capacity, np.uint64)
    rows = np.zeros((capacity, 3), np.int32)
    n = ctypes.c_int32()
    _check(ctx, _lib.ebic_get_toplist(ctx, capacity, ctypes.byref(n), ptr(cols), ptr(lens),
                                      ptr(fit), ptr(keys), ptr(rows)))
    k = n.value
    return [dict(cols=tuple(int(c) for c in cols[e, :lens[e]]), f=int(fit[e]), h=int(keys[e]),
                 rows_pos=int(rows[e, 0]), rows_neg=int(rows[e, 1]), rows_any=int(rows[e, 2]))
            for e in range(k)]


def ebic_get_population(ctx, pop_size):
    cols = np.zeros((pop_size, MAX_LEN), np.int32)
    lens = np.zeros(pop_size, np.int32)
    dead = np.zeros(pop_size, np.uint8)
    fit = np.zeros(pop_size, np.uint64)
    _check(ctx, _lib.ebic_get_population(ctx, pop_size, ptr(cols), ptr(lens), ptr(dead), ptr(fit)))
    return cols, lens, dead, fit


def ebic_extract_biclusters(ctx, rows, capacity=256):
    w = ((int(rows) + 127) // 128) * 4
    masks = np.zeros((capacity, w), np.uint32)
    n = ctypes.c_int32()
    _check(ctx, _lib.ebic_extract_biclusters(ctx, capacity, ptr(masks), ctypes.byref(n)))
    return masks[:n.value]


def ebic_state_bytes(ctx):
    return int(_lib.ebic_state_bytes(ctx))


def ebic_save_state(ctx):
    size = ebic_state_bytes(ctx)
    if size <= 0:
        raise EbicError(EBIC_ESTATE, ebic_last_error(ctx))
    blob = np.zeros(size, np.uint8)
    _check(ctx, _lib.ebic_save_state(ctx, ptr(blob), size))
    return blob


def ebic_load_state(ctx, params, blob):
    blob = np.ascontiguousarray(blob, np.uint8)
    _check(ctx, _lib.ebic_load_state(ctx, ctypes.byref(params), ptr(blob), int(blob.size)))


KERNEL_EVAL, KERNEL_BITMAP_BUILD, KERNEL_ALL, KERNEL_EVOLVE, KERNEL_FINISH = 0, 1, 2, 3, 4
KERNEL_RANK_CODES = 5


class KernelStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("timed_launches", ctypes.c_int64),
                ("ms", ctypes.c_double), ("alg_bytes", ctypes.c_double),
                ("alg_ops", ctypes.c_double), ("units", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


def ebic_profile_enable(ctx, on=True):
    _check(ctx, _lib.ebic_profile_enable(ctx, int(bool(on))))


def ebic_profile_read(ctx, kernel):
    st = KernelStats()
    _check(ctx, _lib.ebic_profile_read(ctx, int(kernel), ctypes.byref(st)))
    return st.as_dict()


class TuneReport(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("seg_direct", ctypes.c_int32),
                ("seg_bitmap", ctypes.c_int32), ("seg_loop", ctypes.c_int32),
                ("direct_ms", ctypes.c_double), ("bitmap_ms", ctypes.c_double),
                ("build_ms", ctypes.c_double), ("staged_ms", ctypes.c_double),
                ("ipw_bitmap", ctypes.c_int32), ("ipw_loop", ctypes.c_int32),
                ("fuse_loop", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


def ebic_autotune(ctx, col_idx, offsets, params, expected_sweeps=1):
    col_idx = _as_dtype(col_idx, np.int32, "int32")
    offsets = _as_dtype(offsets, np.int32, "int32")
    n = (offsets.numel() if _is_torch(offsets) else offsets.size) - 1
    rep = TuneReport()
    _check(ctx, _lib.ebic_autotune(ctx, ptr(col_idx), ptr(offsets), int(n), ctypes.byref(params),
                                   int(expected_sweeps), ctypes.byref(rep)))
    return rep.as_dict()


class JobResult(ctypes.Structure):
    _fields_ = [("job_id", ctypes.c_int64), ("status", ctypes.c_int32),
                ("gens_done", ctypes.c_int32), ("stopped", ctypes.c_int32),
                ("n_top", ctypes.c_int32), ("n_evaluated", ctypes.c_int64),
                ("eval_mode", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("footprint_bytes", ctypes.c_int64), ("queued_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


def ebic_job_footprint(rows, cols, params, n_gen):
    return int(_lib.ebic_job_footprint(int(rows), int(cols), ctypes.byref(params), int(n_gen)))


def ebic_server_create(device=0, hbm_budget_bytes=16 << 30, max_running=8):
    out = ctypes.c_void_p()
    _check(None, _lib.ebic_server_create(ctypes.byref(out), int(device), int(hbm_budget_bytes),
                                         int(max_running)))
    return out.value


def ebic_server_destroy(srv):
    return _lib.ebic_server_destroy(srv)


def ebic_server_submit(srv, x, params, n_gen, layout=ROW_MAJOR):
    x = _as_dtype(x, np.float32, "float32")
    rows, cols = x.shape if layout == ROW_MAJOR else x.shape[::-1]
    jid = ctypes.c_int64()
    _check(None, _lib.ebic_server_submit(srv, ptr(x), int(rows), int(cols), int(layout),
                                         ctypes.byref(params), int(n_gen), ctypes.byref(jid)))
    return jid.value


def ebic_server_wait(srv, job_id, timeout_ms=-1, capacity=256):
    res = JobResult()
    cols = np.zeros((capacity, MAX_LEN), np.int32)
    lens = np.zeros(capacity, np.int32)
    fit = np.zeros(capacity, np.uint64)
    keys = np.zeros(capacity, np.uint64)
    rows = np.zeros((capacity, 3), np.int32)
    _check(None, _lib.ebic_server_wait(srv, int(job_id), int(timeout_ms), ctypes.byref(res),
                                       capacity, ptr(cols), ptr(lens), ptr(fit), ptr(keys),
                                       ptr(rows)))
    out = res.as_dict()
    out["top"] = [dict(cols=tuple(int(c) for c in cols[e, :lens[e]]), f=int(fit[e]),
                       h=int(keys[e]), rows_pos=int(rows[e, 0]), rows_neg=int(rows[e, 1]),
                       rows_any=int(rows[e, 2])) for e in range(res.n_top)]
    return out


def ebic_server_stats(srv):
    q, r, b = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(None, _lib.ebic_server_stats(srv, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b)))
    return {"queued": q.value, "running": r.value, "reserved": b.value}


class Server:
    """Continuous-batching job server on one GPU (see ebic_server_create)."""

    def __init__(self, device=0, hbm_budget_bytes=16 << 30, max_running=8):
        self.handle = ebic_server_create(device, hbm_budget_bytes, max_running)

    def submit(self, x, params, n_gen, layout=ROW_MAJOR):
        return ebic_server_submit(self.handle, x, params, n_gen, layout)

    def wait(self, job_id, timeout_ms=-1):
        return ebic_server_wait(self.handle, job_id, timeout_ms)

    def stats(self):
        return ebic_server_stats(self.handle)

    def close(self):
        if self.handle:
            ebic_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


NOALLOC_MAX_IND = 65536


def _noalloc_check(name, a, dtypes, device, min_numel=None, ndim=None):
    """Checks one argument of the allocation-free call; never converts (a conversion would
    allocate)."""
    if not _is_torch(a):
        raise EbicError(EBIC_EINVAL, f"{name} must be a CUDA tensor (caller-owned device memory)")
    if a.device.type != "cuda" or (a.device.index or 0) != device:
        raise EbicError(EBIC_EINVAL, f"{name} must be on cuda:{device}, not {a.device}")
    if str(a.dtype) not in dtypes:
        raise EbicError(EBIC_EINVAL, f"{name} must be {' or '.join(dtypes)}, not {a.dtype}")
    if not a.is_contiguous():
        raise EbicError(EBIC_EINVAL, f"{name} must be contiguous")
    if ndim is not None and a.dim() != ndim:
        raise EbicError(EBIC_EINVAL, f"{name} must be {ndim}-D, not {a.dim()}-D")
    if min_numel is not None and a.numel() < min_numel:
        raise EbicError(EBIC_EINVAL, f"{name} holds {a.numel()} entries, fewer than {min_numel}")


def ebic_eval_population_noalloc(x_colmajor, col_idx, offsets, params, rows_pos=None,
                                 rows_neg=None, rows_any=None, fitness=None, device=0,
                                 stream=None):
    """Allocation-free evaluation for callers that cannot let the library allocate GPU memory.

    Every array is caller-owned, contiguous device memory of `device`: x_colmajor float32
    [cols, rows], col_idx and offsets int32 (offsets 1-D with n + 1 entries), rows_* int32 and
    fitness int64/uint64 with at least n entries each (any output may be None).  Nothing is
    converted, since a conversion would allocate: a wrong dtype, device, shape or length raises
    EbicError(EBIC_EINVAL) before the library is called.  Returns the outputs passed in and
    raises EbicError with the library's message on failure."""
    _noalloc_check("x_colmajor", x_colmajor, ("torch.float32",), device, ndim=2)
    _noalloc_check("offsets", offsets, ("torch.int32",), device, min_numel=1, ndim=1)
    n = offsets.numel() - 1
    _noalloc_check("col_idx", col_idx, ("torch.int32",), device, ndim=1)
    if n > 0:
        first, last = int(offsets[0].item()), int(offsets[-1].item())   # views: no allocation
        if first < 0 or last < first or col_idx.numel() < last:
            raise EbicError(EBIC_EINVAL, f"col_idx holds {col_idx.numel()} entries but offsets "
                                         f"run from {first} to {last}")
    for name, o, dts in (("rows_pos", rows_pos, ("torch.int32",)),
                         ("rows_neg", rows_neg, ("torch.int32",)),
                         ("rows_any", rows_any, ("torch.int32",)),
                         ("fitness", fitness, ("torch.int64", "torch.uint64"))):
        if o is not None:
            _noalloc_check(name, o, dts, device, min_numel=n)
    cols, rows = x_colmajor.shape
    buf = ctypes.create_string_buffer(256)
    status = _lib.ebic_eval_population_noalloc(
        ptr(x_colmajor), int(rows), int(cols), ptr(col_idx), ptr(offsets), int(n),
        ctypes.byref(params), ptr(rows_pos), ptr(rows_neg), ptr(rows_any), ptr(fitness),
        int(device), stream, buf, 256)
    if status != EBIC_OK:
        raise EbicError(status, buf.value.decode())
    return rows_pos, rows_neg, rows_any, fitness


class Context:
    """One EBIC job on one GPU: owns the C context (see ebic_create)."""

    def __init__(self, device=0, stream=None):
        self.handle = ebic_create(device, stream)

    def close(self):
        if self.handle:
            ebic_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_matrix(self, x, layout=ROW_MAJOR):
        ebic_load_matrix(self.handle, x, layout)

    def build_bitmap(self):
        ebic_build_bitmap(self.handle)

    def copy_bitmap(self, out):
        return ebic_copy_bitmap(self.handle, out)

    def copy_pair_counts(self, out):
        return ebic_copy_pair_counts(self.handle, out)

    def eval_population(self, col_idx, offsets, params, *outs):
        return ebic_eval_population(self.handle, col_idx, offsets, params, *outs)

    def run_generations(self, params, n_gen):
        return ebic_run_generations(self.handle, params, n_gen)

    def toplist(self, capacity=256):
        return ebic_get_toplist(self.handle, capacity)

    def population(self, pop_size):
        return ebic_get_population(self.handle, pop_size)

    def extract_biclusters(self, rows, capacity=256):
        return ebic_extract_biclusters(self.handle, rows, capacity)

    def save_state(self):
        return ebic_save_state(self.handle)

    def load_state(self, params, blob):
        ebic_load_state(self.handle, params, blob)

    def last_error(self):
        return ebic_last_error(self.handle)

    def autotune(self, col_idx, offsets, params, expected_sweeps=1):
        return ebic_autotune(self.handle, col_idx, offsets, params, expected_sweeps)

    def profile_enable(self, on=True):
        ebic_profile_enable(self.handle, on)

    def profile_read(self, kernel):
        return ebic_profile_read(self.handle, kernel)
