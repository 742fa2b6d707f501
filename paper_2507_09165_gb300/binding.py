"""Thin ctypes binding of libpsdproj (include/psdproj.h), same names as the C ABI.

Argument marshalling only: every step of the projection runs in the CUDA
library.  Pointers may be given as integers or as objects with ``data_ptr()``
(torch tensors); streams as integers, ``None`` (legacy default stream) or
objects with ``cuda_stream``.  A non-zero status raises ``PsdError``.  If the
library has not been built, ``lib()`` raises: there is no fallback.

Storage note for torch users: the library reads the column-major upper
triangle X[i + j*ld], i <= j.  For a C-contiguous (row-major) tensor T of
shape (n, n) with ld = T.stride(0), that is T[r][c] with r >= c.  Symmetric
inputs need no care.
"""
import ctypes
import os

from . import _build

PSD_OK = 0
STATUS = {0: "PSD_OK", 1: "PSD_ERR_INVALID_ARG", 2: "PSD_ERR_CUDA", 3: "PSD_ERR_NO_MEMORY",
          4: "PSD_ERR_NONFINITE", 5: "PSD_ERR_BOUND", 6: "PSD_ERR_TIMEOUT", 7: "PSD_ERR_UNSUPPORTED",
          8: "PSD_ERR_CANCELED"}
PRECISION = {"fp32": 0, "fp16": 1, "bf16": 2, "mixed": 3, "fp8_early": 4, "fp8_late": 5}


class PsdError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = int(status)
        super().__init__("%s (%d) %s" % (STATUS.get(self.status, "?"), self.status, what))


class psd_info_t(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("lanczos_steps", ctypes.c_int32),
                ("lambda_bound", ctypes.c_double), ("lanczos_sigma", ctypes.c_double),
                ("lanczos_resid", ctypes.c_double), ("fro_X", ctypes.c_double),
                ("max_diag", ctypes.c_double), ("overshoot_max", ctypes.c_double),
                ("compl_resid", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class psd_block_desc_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("X", ctypes.c_void_p), ("ld", ctypes.c_int64),
                ("out", ctypes.c_void_p), ("ld_out", ctypes.c_int64), ("info", ctypes.c_void_p)]


class psd_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("canceled", ctypes.c_uint64),
                ("steps", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("queued", ctypes.c_int32), ("admitted", ctypes.c_int32), ("max_running", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("arena_rows", ctypes.c_int64), ("peak_rows", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


_lib = None

_VP, _I64, _I32, _SZ, _D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t, ctypes.c_double
_SIGS = {
    "psd_project": ([_I64, _VP, _I64, _VP, _I32, _VP], _I32),
    "psd_project_ex": ([_I64, _VP, _I64, _VP, _I64, _I32, _VP, _VP, _SZ, _VP], _I32),
    "psd_workspace_size": ([_I64, _I32], _SZ),
    "psd_last_info": ([_VP, ctypes.POINTER(psd_info_t)], _I32),
    "psd_release_workspaces": ([], _I32),
    "psd_norm_bound": ([_I64, _VP, _I64, _VP, _VP], _I32),
    "psd_norm_bound_noalloc": ([_I64, _VP, _I64, _VP, _VP], _I32),
    "psd_project_batched": ([_I32, _VP, _I32, _VP], _I32),
    "psd_symm_product": ([_I64, _VP, _VP, _I64, _VP, _I64, _I32, _I32, ctypes.POINTER(_D), _VP, _I64, _VP,
                          _VP], _I32),
    "psd_status_string": ([_I32], ctypes.c_char_p),
    "psd_schedule": ([_I32, ctypes.POINTER(_I32), ctypes.POINTER(_D), ctypes.POINTER(_D)], _I32),
    "psd_gemm_count": ([_I32], _I32),
    "psd_kernel_launches": ([_I64, _I32, _VP], _I32),
    "psd_version": ([], ctypes.c_char_p),
    "psd_server_create": ([_SZ, _I32, _I64, _I32, ctypes.POINTER(_VP)], _I32),
    "psd_server_submit": ([_VP, _I64, _VP, _I64, _VP, _I64, _I32, _VP, ctypes.POINTER(ctypes.c_uint64)], _I32),
    "psd_server_poll": ([_VP, ctypes.c_uint64, ctypes.POINTER(_I32), ctypes.POINTER(psd_info_t),
                         ctypes.POINTER(_D)], _I32),
    "psd_server_wait": ([_VP, ctypes.c_uint64, _I64, ctypes.POINTER(psd_info_t), ctypes.POINTER(_D)], _I32),
    "psd_server_cancel": ([_VP, ctypes.c_uint64], _I32),
    "psd_server_stats": ([_VP, ctypes.POINTER(psd_server_stats_t)], _I32),
    "psd_server_destroy": ([_VP], _I32),
    "psd_project_deflate": ([_I64, _VP, _I64, _VP, _I64, _I32, _I32, _VP, _VP, _VP], _I32),
    "psd_batched_force_schedule": ([_I32], _I32),
    "psd_batched_force_form": ([_I32], _I32),
    "psd_batched_force_bound": ([_I32], _I32),
    "psd_debug_set": ([_I32, ctypes.c_double], _I32),
    "psd_batched_last_tuning": ([ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_float)], _I32),
}


def lib():
    """Open libpsdproj.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libpsdproj.so is not built (%s); run __graft_entry__.build(). "
                               "There is no CPU fallback." % path)
        h = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            if hasattr(h, name):
                f = getattr(h, name)
                f.argtypes = args
                f.restype = res
        _lib = h
    return _lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, ctypes.c_void_p):
        return x.value
    raise TypeError("expected a device pointer, got %r" % type(x))


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    raise TypeError("expected a CUDA stream, got %r" % type(s))


def _prec(p):
    return PRECISION[p] if isinstance(p, str) else int(p)


def _check(st, what=""):
    if st != PSD_OK:
        raise PsdError(st, what)


def psd_project(n, X, ld, out, precision="fp16", stream=None):
    _check(lib().psd_project(n, _ptr(X), ld, _ptr(out), _prec(precision), _stream(stream)), "psd_project")


def psd_project_ex(n, X, ld, out, ld_out, precision="fp16", d_info=None, workspace=None, ws_bytes=0,
                   stream=None):
    _check(lib().psd_project_ex(n, _ptr(X), ld, _ptr(out), ld_out, _prec(precision), _ptr(d_info),
                                _ptr(workspace), ws_bytes, _stream(stream)), "psd_project_ex")


def psd_project_deflate(n, X, ld, out, ld_out, precision="fp16", kmax=8, d_info=None, d_kused=None,
                        stream=None):
    _check(lib().psd_project_deflate(n, _ptr(X), ld, _ptr(out), ld_out, _prec(precision), kmax, _ptr(d_info),
                                     _ptr(d_kused), _stream(stream)), "psd_project_deflate")


def psd_batched_force_schedule(index):
    """Force grouped-product schedule `index` (0..5) for batched plans built next; -1: autotune."""
    return int(lib().psd_batched_force_schedule(int(index)))


def psd_batched_force_form(form):
    """Product form of batched plans built next: 1 chain (one persistent launch), 0 one launch
    per product, -1 default (chain where it applies)."""
    return int(lib().psd_batched_force_form(int(form)))


def psd_batched_force_bound(form):
    """Norm-bound form of batched plans built next: 1 one launch over a work-item list with
    per-block counters, 0 or -1 (default) one grouped launch per phase."""
    return int(lib().psd_batched_force_bound(int(form)))


DEBUG_BOUND_SCALE = 1         # PSD_DEBUG_BOUND_SCALE
DEBUG_BARRIER_LIMIT_NS = 2    # PSD_DEBUG_BARRIER_LIMIT_NS


def psd_debug_set(knob, value):
    """Host-side fault injection into the norm bound (test hook): knob 1 = factor on lam~,
    knob 2 = grid-barrier wait limit in ns."""
    _check(lib().psd_debug_set(int(knob), float(value)), "psd_debug_set")


def psd_batched_last_tuning():
    """(chosen, [ms per candidate]) of the most recently built batched plan."""
    chosen, ncand = _I32(), _I32()
    ms = (ctypes.c_float * 16)()
    _check(lib().psd_batched_last_tuning(ctypes.byref(chosen), ctypes.byref(ncand), ms), "psd_batched_last_tuning")
    return int(chosen.value), [float(ms[i]) for i in range(ncand.value)]


def psd_workspace_size(n, precision="fp16"):
    return int(lib().psd_workspace_size(n, _prec(precision)))


def psd_last_info(stream=None):
    info = psd_info_t()
    _check(lib().psd_last_info(_stream(stream), ctypes.byref(info)), "psd_last_info")
    return info.as_dict()


def psd_release_workspaces():
    _check(lib().psd_release_workspaces(), "psd_release_workspaces")


def psd_norm_bound(n, X, ld, d_info, stream=None):
    _check(lib().psd_norm_bound(n, _ptr(X), ld, _ptr(d_info), _stream(stream)), "psd_norm_bound")


def psd_norm_bound_noalloc(n, X, ld, d_info, stream=None):
    _check(lib().psd_norm_bound_noalloc(n, _ptr(X), ld, _ptr(d_info), _stream(stream)),
           "psd_norm_bound_noalloc")


def psd_project_batched(count, d_descs, precision="bf16", stream=None):
    _check(lib().psd_project_batched(count, _ptr(d_descs), _prec(precision), _stream(stream)),
           "psd_project_batched")


_PRODUCT_BYTES = {"fp16": (1, 2), "bf16": (1, 2), "mixed": (2, 2), "fp32": (2, 4), "fp8_late": (1, 1)}
_FP8_PARAMS = {0: 3, 1: 6, 2: 4}  # epilogue params followed by (in_scale, y_scale, out_scale)


def _check_extent(t, need, what):
    """Refuse a tensor smaller than the bytes the C ABI will touch (raw pointers carry no size)."""
    if hasattr(t, "numel") and hasattr(t, "element_size"):
        have = t.numel() * t.element_size()
        if have < need:
            raise ValueError("%s holds %d bytes, the product needs %d" % (what, have, need))


EPI_GROUPED = 0x100         # PSD_EPI_GROUPED
EPI_F16_PAIR_OUT = 0x200    # PSD_EPI_F16_PAIR_OUT
EPI_CTA_PAIR = 0x400        # PSD_EPI_CTA_PAIR


def psd_symm_product(n, A, B, ld, C, ld_out=0, precision="fp16", epi=0, params=(), aux=None, ld_aux=0,
                     d_absmax=None, stream=None):
    pname = precision if isinstance(precision, str) else {v: k for k, v in PRECISION.items()}.get(precision)
    kind = epi & 0xFF  # the epilogue; the bits above are PSD_EPI_* flags
    if pname in _PRODUCT_BYTES and n > 0:
        parts, esz = _PRODUCT_BYTES[pname]
        need = ((parts - 1) * n * ld + (n - 1) * ld + n) * esz  # pairs: hi, then lo at + n * ld
        _check_extent(A, need, "A")
        _check_extent(B, need, "B")
        if kind == 3:
            _check_extent(C, ((n - 1) * ld_out + n) * 4, "C (FP32 output)")
            _check_extent(aux, ((n - 1) * ld_aux + n) * 4, "aux (FP32 input)")
        else:
            _check_extent(C, need + (n * ld * esz if epi & EPI_F16_PAIR_OUT else 0), "C")
            if kind == 1:
                _check_extent(aux, need, "aux (Y)")
    if pname == "fp8_late" and len(params) < _FP8_PARAMS.get(kind, 0):
        raise ValueError("fp8_late epilogue %d takes %d params" % (kind, _FP8_PARAMS[kind]))
    arr = (ctypes.c_double * max(1, len(params)))(*params) if params else None
    _check(lib().psd_symm_product(n, _ptr(A), _ptr(B), ld, _ptr(C), ld_out, _prec(precision), epi, arr,
                                  _ptr(aux), ld_aux, _ptr(d_absmax), _stream(stream)), "psd_symm_product")


def psd_status_string(status):
    return lib().psd_status_string(status).decode()


def psd_schedule(precision):
    T = ctypes.c_int32()
    coef = (ctypes.c_double * 30)()
    post = (ctypes.c_double * 10)()
    _check(lib().psd_schedule(_prec(precision), ctypes.byref(T), coef, post), "psd_schedule")
    t = T.value
    return [tuple(coef[3 * i:3 * i + 3]) for i in range(t)], list(post[:t])


def psd_gemm_count(precision):
    return int(lib().psd_gemm_count(_prec(precision)))


def psd_kernel_launches(n, precision="fp16", stream=None):
    return int(lib().psd_kernel_launches(n, _prec(precision), _stream(stream)))


def psd_version():
    return lib().psd_version().decode()


def block_descs(blocks, device="cuda"):
    """Device array of psd_block_desc_t for psd_project_batched.

    blocks: list of (n, X, ld, out, ld_out, info) with X, out, info device
    pointers (integers or tensors; info may be None).  Returns a uint8 torch
    tensor on `device` holding the descriptors (keep it alive for the call).
    """
    import torch
    arr = (psd_block_desc_t * len(blocks))()
    for i, (n, X, ld, out, ld_out, info) in enumerate(blocks):
        arr[i] = psd_block_desc_t(n, _ptr(X), ld, _ptr(out), ld_out, _ptr(info))
    raw = bytes(arr)
    return torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device)


def psd_server_create(hbm_budget_bytes, device=0, max_order=8192, max_batch=64):
    """Returns the server handle (an integer)."""
    h = ctypes.c_void_p()
    _check(lib().psd_server_create(hbm_budget_bytes, device, max_order, max_batch, ctypes.byref(h)),
           "psd_server_create")
    return h.value


def _event(e):
    if e is None:
        return None
    if hasattr(e, "cuda_event"):
        return e.cuda_event
    return int(e)


def psd_server_submit(server, n, X, ld, out, ld_out, precision="bf16", ready=None):
    """Queues one projection; `ready` is an event (torch.cuda.Event or handle) to wait for. Returns the ticket."""
    t = ctypes.c_uint64()
    _check(lib().psd_server_submit(server, n, _ptr(X), ld, _ptr(out), ld_out, _prec(precision), _event(ready),
                                   ctypes.byref(t)), "psd_server_submit")
    return t.value


def psd_server_poll(server, ticket):
    """(done, info dict or None, latency_ms or None); a completed ticket is retired."""
    done, info, lat = _I32(), psd_info_t(), _D()
    _check(lib().psd_server_poll(server, ticket, ctypes.byref(done), ctypes.byref(info), ctypes.byref(lat)),
           "psd_server_poll")
    return (True, info.as_dict(), lat.value) if done.value else (False, None, None)


def psd_server_wait(server, ticket, timeout_ms=0):
    """Blocks until the ticket completes; returns (info dict, latency_ms)."""
    info, lat = psd_info_t(), _D()
    _check(lib().psd_server_wait(server, ticket, timeout_ms, ctypes.byref(info), ctypes.byref(lat)),
           "psd_server_wait")
    return info.as_dict(), lat.value


def psd_server_cancel(server, ticket):
    _check(lib().psd_server_cancel(server, ticket), "psd_server_cancel")


def psd_server_stats(server):
    st = psd_server_stats_t()
    _check(lib().psd_server_stats(server, ctypes.byref(st)), "psd_server_stats")
    return st.as_dict()


def psd_server_destroy(server):
    _check(lib().psd_server_destroy(server), "psd_server_destroy")


INFO_BYTES = ctypes.sizeof(psd_info_t)
DESC_BYTES = ctypes.sizeof(psd_block_desc_t)


def info_from_bytes(raw):
    """Decode a psd_info_t copied from the device (bytes of length INFO_BYTES)."""
    return psd_info_t.from_buffer_copy(bytes(raw)).as_dict()
