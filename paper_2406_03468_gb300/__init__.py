"""Python binding of liblsq (include/lsq.h): FOSSILS and SPIR least-squares
solvers on GB300 (sm_103a).

The functions here carry the C ABI's names and only marshal arguments:
torch tensors (or raw device pointers) go in as pointers, status codes come
back as exceptions.  Every step of a solve runs in the CUDA library; there is
no CPU fallback, and importing fails loudly when the library cannot be built
or loaded.
"""
import ctypes
import os

from . import _build

__all__ = [
    "LsqError", "LsqOptions", "LsqInfo", "lsq_options_default", "lsq_plan_create",
    "lsq_plan_destroy", "lsq_plan_configure", "lsq_sketch", "lsq_solve_fossils", "lsq_solve_spir",
    "lsq_solve_spir_lsqr", "lsq_solve_host", "lsq_solve_complex", "lsq_solve_csr",
    "lsq_solve_fossils_multi",
    "lsq_sketch_pattern", "lsq_get_sketch", "lsq_get_sketch_raw", "lsq_get_R", "lsq_apply_normal",
    "lsq_apply_normal_multi", "lsq_residual", "lsq_sketched_kw",
    "lsq_trsv", "lsq_apply_normal_noalloc", "lsq_last_error", "Plan", "lsq_server_create",
    "lsq_submit", "lsq_poll", "lsq_server_stats", "lsq_server_destroy", "library_path", "EXPORTED",
    "LsqBatchItem", "lsq_batch_create", "lsq_batch_solve", "lsq_batch_destroy",
    "lsq_server_create_batched",
    "LSQ_PREC_AUTO", "LSQ_PREC_FP64", "LSQ_PREC_FP32_INNER",
]

LSQ_OK = 0
LSQ_PENDING = 1
LSQ_WARN_RANK_DEFICIENT = 2
LSQ_PREC_AUTO, LSQ_PREC_FP64, LSQ_PREC_FP32_INNER = 0, 1, 2
LSQ_MAX_REFINE = 8

_STATUS = {0: "LSQ_OK", 1: "LSQ_PENDING", 2: "LSQ_WARN_RANK_DEFICIENT", -1: "LSQ_ERR_INVALID",
           -2: "LSQ_ERR_OOM", -3: "LSQ_ERR_CUDA", -4: "LSQ_ERR_NOT_CONVERGED",
           -5: "LSQ_ERR_TIMEOUT", -6: "LSQ_ERR_NONFINITE"}


class LsqError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class LsqOptions(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("lda", ctypes.c_int64),
                ("d", ctypes.c_int32), ("zeta", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("eta", ctypes.c_double), ("col_scale", ctypes.c_int32),
                ("max_inner", ctypes.c_int32), ("max_refine", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("fp32_cond_max", ctypes.c_double),
                ("stop_gamma", ctypes.c_double), ("stop_rho", ctypes.c_double),
                ("fixed_inner", ctypes.c_int32), ("timing", ctypes.c_int32),
                ("inner_fp64_fma", ctypes.c_int32), ("nrhs", ctypes.c_int32),
                ("qr_wait_us", ctypes.c_int32), ("kw_stop", ctypes.c_int32),
                ("sparse", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class LsqInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32 * LSQ_MAX_REFINE), ("refine_steps", ctypes.c_int32),
                ("path", ctypes.c_int32), ("passes", ctypes.c_int32), ("status", ctypes.c_int32),
                ("condest", ctypes.c_double), ("normest", ctypes.c_double),
                ("cnorm", ctypes.c_double * LSQ_MAX_REFINE), ("resid0", ctypes.c_double),
                ("thresh1", ctypes.c_double), ("ms_sketch", ctypes.c_float),
                ("ms_qr", ctypes.c_float), ("ms_refine", ctypes.c_float),
                ("ms_total", ctypes.c_float), ("launches", ctypes.c_int32),
                ("n_inner_pass", ctypes.c_int32), ("ms_inner_pass", ctypes.c_float),
                ("n_resid_pass", ctypes.c_int32), ("ms_resid_pass", ctypes.c_float),
                ("ms_sketch_pass", ctypes.c_float), ("inner_kernel", ctypes.c_int32),
                ("bytes_a", ctypes.c_double), ("be_sketch_est", ctypes.c_double)]

    def as_dict(self):
        k = self.refine_steps
        return {"iters": list(self.iters[:k]), "refine_steps": k, "path": self.path,
                "passes": self.passes, "status": self.status, "condest": self.condest,
                "normest": self.normest, "cnorm": list(self.cnorm[:k]), "resid0": self.resid0,
                "thresh1": self.thresh1, "ms_sketch": self.ms_sketch, "ms_qr": self.ms_qr,
                "ms_refine": self.ms_refine, "ms_total": self.ms_total,
                "launches": self.launches, "n_inner_pass": self.n_inner_pass,
                "ms_inner_pass": self.ms_inner_pass, "n_resid_pass": self.n_resid_pass,
                "ms_resid_pass": self.ms_resid_pass, "ms_sketch_pass": self.ms_sketch_pass,
                "inner_kernel": self.inner_kernel, "bytes_a": self.bytes_a,
                "be_sketch_est": self.be_sketch_est}


class LsqBatchItem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("A", ctypes.c_void_p),
                ("b", ctypes.c_void_p), ("x", ctypes.c_void_p), ("seed", ctypes.c_uint64),
                ("method", ctypes.c_int32), ("status", ctypes.c_int32)]


_vp = ctypes.c_void_p
_i32 = ctypes.c_int
_dp = ctypes.POINTER(ctypes.c_double)
# name -> (restype, argtypes); every function of include/lsq.h
EXPORTED = {
    "lsq_options_default": (None, [ctypes.POINTER(LsqOptions)]),
    "lsq_plan_create": (_i32, [ctypes.POINTER(LsqOptions), _vp, ctypes.POINTER(_vp)]),
    "lsq_plan_destroy": (None, [_vp]),
    "lsq_plan_configure": (_i32, [_vp, ctypes.POINTER(LsqOptions)]),
    "lsq_sketch": (_i32, [_vp, _vp, _vp]),
    "lsq_solve_fossils": (_i32, [_vp, _vp, _vp, _vp, ctypes.POINTER(LsqInfo)]),
    "lsq_solve_spir": (_i32, [_vp, _vp, _vp, _vp, ctypes.POINTER(LsqInfo)]),
    "lsq_solve_spir_lsqr": (_i32, [_vp, _vp, _vp, _vp, ctypes.POINTER(LsqInfo)]),
    "lsq_solve_host": (_i32, [_vp, _i32, _vp, _vp, _vp, ctypes.POINTER(LsqInfo)]),
    "lsq_solve_fossils_multi": (_i32, [_vp, _vp, _vp, ctypes.c_int64, _vp,
                                       ctypes.POINTER(LsqInfo)]),
    "lsq_solve_complex": (_i32, [_vp, _i32, _vp, ctypes.c_int64, _vp, _vp, _vp,
                                 ctypes.POINTER(LsqInfo)]),
    "lsq_solve_csr": (_i32, [_vp, _i32, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp,
                             ctypes.POINTER(LsqInfo)]),
    "lsq_sketch_pattern": (_i32, [_vp, _vp, _vp]),
    "lsq_get_sketch": (_i32, [_vp, _vp, _vp]),
    "lsq_get_sketch_raw": (_i32, [_vp, _vp]),
    "lsq_get_R": (_i32, [_vp, _vp, _vp, _vp, _dp, _dp]),
    "lsq_apply_normal": (_i32, [_vp, _vp, _vp, _vp]),
    "lsq_apply_normal_multi": (_i32, [_vp, _vp, _vp, _vp]),
    "lsq_residual": (_i32, [_vp, _vp, _vp, _vp, _vp, _dp]),
    "lsq_sketched_kw": (_i32, [_vp, _vp, _vp, _vp, _dp]),
    "lsq_trsv": (_i32, [_vp, _i32, _vp, _vp]),
    "lsq_apply_normal_noalloc": (_i32, [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                        _vp, _vp, _vp]),
    "lsq_batch_create": (_i32, [_i32, ctypes.c_int64, ctypes.c_int64, _vp, ctypes.POINTER(_vp)]),
    "lsq_batch_solve": (_i32, [_vp, _i32, ctypes.POINTER(LsqBatchItem), ctypes.POINTER(LsqInfo)]),
    "lsq_batch_destroy": (None, [_vp]),
    "lsq_server_create": (_i32, [ctypes.c_size_t, _i32, ctypes.c_int64, ctypes.c_int64,
                                 ctypes.POINTER(_vp)]),
    "lsq_server_create_batched": (_i32, [ctypes.c_size_t, _i32, _i32, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.POINTER(_vp)]),
    "lsq_submit": (_i32, [_vp, ctypes.POINTER(LsqOptions), _i32, _vp, _vp, _i32,
                          ctypes.POINTER(ctypes.c_uint64)]),
    "lsq_poll": (_i32, [_vp, ctypes.c_uint64, _vp, ctypes.POINTER(LsqInfo), _dp]),
    "lsq_server_stats": (_i32, [_vp, ctypes.POINTER(ctypes.c_int64)]),
    "lsq_server_destroy": (None, [_vp]),
    "lsq_last_error": (ctypes.c_char_p, []),
}

_LIB = None


def library_path():
    return _build.LIB


def _lib():
    """Load liblsq.so (building it with nvcc when missing or stale)."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        if not os.path.exists(path):
            raise ImportError("liblsq.so is missing and could not be built")
        lib = ctypes.CDLL(path)
        for name, (res, args) in EXPORTED.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
    return _LIB


def _ptr(x):
    """Device pointer of a torch tensor (or an int pointer, or None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _check(status):
    if status < 0:
        raise LsqError(status, lsq_last_error())
    return status


def lsq_last_error():
    return (_lib().lsq_last_error() or b"").decode()


def lsq_options_default(**kw):
    o = LsqOptions()
    _lib().lsq_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError("unknown option %r" % k)
        setattr(o, k, v)
    return o


def lsq_plan_create(opts, stream=None):
    """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None (default stream)."""
    h = _vp()
    s = getattr(stream, "cuda_stream", stream)
    _check(_lib().lsq_plan_create(ctypes.byref(opts), s, ctypes.byref(h)))
    return h


def lsq_plan_configure(plan, opts):
    return _check(_lib().lsq_plan_configure(plan, ctypes.byref(opts)))


def lsq_plan_destroy(plan):
    _lib().lsq_plan_destroy(plan)


def lsq_sketch(plan, A, b):
    return _check(_lib().lsq_sketch(plan, _ptr(A), _ptr(b)))


def _solve(fn, plan, A, b, x, info):
    inf = info if info is not None else LsqInfo()
    st = _check(fn(plan, _ptr(A), _ptr(b), _ptr(x), ctypes.byref(inf)))
    return st, inf


def lsq_solve_fossils(plan, A, b, x, info=None):
    return _solve(_lib().lsq_solve_fossils, plan, A, b, x, info)


def lsq_solve_spir(plan, A, b, x, info=None):
    return _solve(_lib().lsq_solve_spir, plan, A, b, x, info)


def lsq_solve_spir_lsqr(plan, A, b, x, info=None):
    return _solve(_lib().lsq_solve_spir_lsqr, plan, A, b, x, info)


def lsq_solve_csr(plan, method, row_ptr, col, val, b, x, info=None):
    """Sparse A in CSR form: row_ptr (int64, m + 1), col (int32, nnz), val
    (float64, nnz), b (m), x (n): device tensors; plan created with
    sparse=1.  method: 0 FOSSILS, 1 SPIR, 2 LSQR-SPIR."""
    inf = info if info is not None else LsqInfo()
    nnz = int(val.numel()) if hasattr(val, "numel") else int(len(val))
    st = _check(_lib().lsq_solve_csr(plan, int(method), nnz, _ptr(row_ptr), _ptr(col), _ptr(val),
                                     _ptr(b), _ptr(x), ctypes.byref(inf)))
    return st, inf


def lsq_solve_complex(plan, method, A, b, x, work, lda=0, info=None):
    """Complex least squares through the real embedding.  A (m x n), b (m), x
    (n): complex128 device tensors; work: 4 m n doubles on the device; plan
    created for (2m, 2n).  method: 0 FOSSILS, 1 SPIR, 2 LSQR-SPIR."""
    inf = info if info is not None else LsqInfo()
    st = _check(_lib().lsq_solve_complex(plan, int(method), _ptr(A), int(lda), _ptr(b), _ptr(x),
                                         _ptr(work), ctypes.byref(inf)))
    return st, inf


def lsq_solve_fossils_multi(plan, A, B, ldb, X, info=None):
    inf = info if info is not None else LsqInfo()
    st = _check(_lib().lsq_solve_fossils_multi(plan, _ptr(A), _ptr(B), int(ldb), _ptr(X),
                                               ctypes.byref(inf)))
    return st, inf


def lsq_solve_host(plan, method, A, b, x, info=None):
    """Host-buffer solve: A, b, x are host tensors / numpy arrays (pointer via
    .data_ptr() or .ctypes.data)."""
    def hp(a):
        return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
    inf = info if info is not None else LsqInfo()
    st = _check(_lib().lsq_solve_host(plan, int(method), hp(A), hp(b), hp(x), ctypes.byref(inf)))
    return st, inf


def lsq_sketch_pattern(plan, rows, signbits):
    return _check(_lib().lsq_sketch_pattern(plan, _ptr(rows), _ptr(signbits)))


def lsq_get_sketch(plan, SAb, colnorm):
    return _check(_lib().lsq_get_sketch(plan, _ptr(SAb), _ptr(colnorm)))


def lsq_get_sketch_raw(plan, SAb):
    return _check(_lib().lsq_get_sketch_raw(plan, _ptr(SAb)))


def lsq_get_R(plan, R=None, t=None, x0=None):
    ce = ctypes.c_double()
    ne = ctypes.c_double()
    _check(_lib().lsq_get_R(plan, _ptr(R), _ptr(t), _ptr(x0), ctypes.byref(ce), ctypes.byref(ne)))
    return ce.value, ne.value


def lsq_apply_normal(plan, A, z, h):
    return _check(_lib().lsq_apply_normal(plan, _ptr(A), _ptr(z), _ptr(h)))


def lsq_apply_normal_multi(plan, A, Z, H):
    """H = A^T (A Z) for the plan's nrhs vectors (Z, H: n x k column-major)."""
    return _check(_lib().lsq_apply_normal_multi(plan, _ptr(A), _ptr(Z), _ptr(H)))


def lsq_sketched_kw(plan, A, b, x):
    """The sketched Karlson-Walden estimate of x's backward error (absolute)."""
    est = ctypes.c_double()
    _check(_lib().lsq_sketched_kw(plan, _ptr(A), _ptr(b), _ptr(x), ctypes.byref(est)))
    return est.value


def lsq_residual(plan, A, b, x, g):
    r2 = ctypes.c_double()
    _check(_lib().lsq_residual(plan, _ptr(A), _ptr(b), _ptr(x), _ptr(g), ctypes.byref(r2)))
    return r2.value


def lsq_apply_normal_noalloc(A, m, n, lda, z, h, stream=None):
    """dh = A^T (A dz) without any device allocation (see include/lsq.h)."""
    s = getattr(stream, "cuda_stream", stream)
    return _check(_lib().lsq_apply_normal_noalloc(_ptr(A), int(m), int(n), int(lda), _ptr(z),
                                                  _ptr(h), s))


def lsq_trsv(plan, trans, y, x):
    return _check(_lib().lsq_trsv(plan, int(trans), _ptr(y), _ptr(x)))


def lsq_batch_create(max_items, n_max, elems_max, stream=None):
    """Workspace for batched solves (see include/lsq.h)."""
    h = _vp()
    s = getattr(stream, "cuda_stream", stream)
    _check(_lib().lsq_batch_create(int(max_items), int(n_max), int(elems_max), s,
                                   ctypes.byref(h)))
    return h


def lsq_batch_solve(batch, problems, seeds=None, methods=None):
    """problems: list of (A, b, x) device tensors (A m x n row-major);
    returns (status, [item statuses], [LsqInfo])."""
    count = len(problems)
    arr = (LsqBatchItem * count)()
    infos = (LsqInfo * count)()
    for i, (A, b, x) in enumerate(problems):
        arr[i].m, arr[i].n = int(A.shape[0]), int(A.shape[1])
        arr[i].A, arr[i].b, arr[i].x = _ptr(A), _ptr(b), _ptr(x)
        arr[i].seed = int(seeds[i]) if seeds is not None else 0
        arr[i].method = int(methods[i]) if methods is not None else 0
    st = _lib().lsq_batch_solve(batch, count, arr, infos)
    if st < 0 and not any(arr[i].status < 0 for i in range(count)):
        _check(st)  # an error of the call itself, not of an item
    return st, [arr[i].status for i in range(count)], list(infos)


def lsq_batch_destroy(batch):
    _lib().lsq_batch_destroy(batch)


def lsq_server_create(arena_bytes, max_slots, m_max, n_max):
    h = _vp()
    _check(_lib().lsq_server_create(int(arena_bytes), int(max_slots), int(m_max), int(n_max),
                                    ctypes.byref(h)))
    return h


def lsq_server_create_batched(arena_bytes, workers, max_batch, m_max, n_max):
    h = _vp()
    _check(_lib().lsq_server_create_batched(int(arena_bytes), int(workers), int(max_batch),
                                            int(m_max), int(n_max), ctypes.byref(h)))
    return h


def lsq_submit(server, opts, method, A, b, on_device):
    """A, b: device tensors (on_device=1) or host arrays/tensors (on_device=0)."""
    def p(a):
        if on_device:
            return _ptr(a)
        return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
    t = ctypes.c_uint64()
    _check(_lib().lsq_submit(server, ctypes.byref(opts), int(method), p(A), p(b), int(on_device),
                             ctypes.byref(t)))
    return t.value


def lsq_poll(server, ticket, x=None, info=None):
    """Returns (status, info, latency_s); status LSQ_PENDING (1) while not done.
    x: host float64 array of length n (or None)."""
    inf = info if info is not None else LsqInfo()
    lat = ctypes.c_double()
    xp = None if x is None else (x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data)
    st = _lib().lsq_poll(server, ctypes.c_uint64(ticket), xp, ctypes.byref(inf), ctypes.byref(lat))
    if st != LSQ_PENDING:
        _check(st)
    return st, inf, lat.value


def lsq_server_stats(server):
    out = (ctypes.c_int64 * 7)()
    _check(_lib().lsq_server_stats(server, out))
    keys = ("submitted", "completed", "queued", "running", "arena_bytes", "arena_used",
            "arena_peak")
    return dict(zip(keys, list(out)))


def lsq_server_destroy(server):
    _lib().lsq_server_destroy(server)


class Plan:
    """Owns an lsq_plan (destroyed with the object)."""

    def __init__(self, m, n, stream=None, **opts):
        self.opts = lsq_options_default(m=m, n=n, **opts)
        self.handle = lsq_plan_create(self.opts, stream)

    def close(self):
        if self.handle:
            lsq_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, A, b, x, method="fossils"):
        fn = {"fossils": lsq_solve_fossils, "spir": lsq_solve_spir,
              "spir_lsqr": lsq_solve_spir_lsqr}[method]
        st, info = fn(self.handle, A, b, x)
        return st, info.as_dict()
