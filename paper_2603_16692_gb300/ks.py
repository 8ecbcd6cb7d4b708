"""Thin ctypes binding of libks.so (include/ks.h), same names as the C-ABI.

Only argument marshalling happens here: every step of the KeySwitch runs in the
library's CUDA kernels. PyTorch supplies device memory (uint64 / int8 / int32
tensors) and streams. There is no CPU fallback: if libks.so cannot be built or
loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

KS_OK, KS_EINVAL, KS_EPRIME, KS_ENOMEM, KS_ECUDA, KS_ETIMEOUT, KS_EALIGN = 0, -1, -2, -3, -4, -5, -6
KS_AUTO, KS_DSOB, KS_DPOB, KS_DSOC, KS_DPOC = 0, 1, 2, 3, 4
KS_UNFUSED = 0x100
KS_RADIX4 = 0x200
KS_RADIX16 = 0x400
KS_STAGE_SHIFT = 16
KS_ST_INV, KS_ST_UPC, KS_ST_KM, KS_ST_DNC, KS_ST_DNR = 0, 1, 2, 3, 4
KS_R4, KS_R8, KS_R16 = 1, 2, 3
KS_COLALT_INV, KS_COLALT_UPC, KS_COLALT_DNC = 0x4000000, 0x8000000, 0x10000000
KS_COLTILE_ALT = KS_COLALT_INV | KS_COLALT_UPC | KS_COLALT_DNC
KS_SPLIT_DOWN = 0x20000000
KS_BCONV_TC = 0x800
KS_BCONV_TC_DOWN = 0x1000
STAGE_NAMES = ("inv", "upc", "km", "dnc", "dnr")


def KS_STAGE_RADIX(stage: int, code: int) -> int:
    return code << (KS_STAGE_SHIFT + 2 * stage)
KS_BATCH_GRAPH, KS_BATCH_AUTOTUNE, KS_BATCH_PERSISTENT, KS_BATCH_SELECT = 0x1, 0x2, 0x4, 0x8
KS_BATCH_TEST_STALL = 0x100
VARIANTS = {"DSOB": KS_DSOB, "DPOB": KS_DPOB, "DSOC": KS_DSOC, "DPOC": KS_DPOC}


class KSError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = f"{where}: {strerror(code)} ({code})"
        if code in (KS_ECUDA, KS_ENOMEM):
            msg += ": " + load().ks_cuda_error_string().decode()
        super().__init__(msg)


class ks_params(ctypes.Structure):
    _fields_ = [("dnum", ctypes.c_uint32), ("log2n", ctypes.c_uint32), ("L", ctypes.c_uint32),
                ("q", ctypes.POINTER(ctypes.c_uint64)), ("nq", ctypes.c_uint32),
                ("p", ctypes.POINTER(ctypes.c_uint64)), ("np", ctypes.c_uint32)]


class ks_info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint32), ("alpha", ctypes.c_uint32), ("beta", ctypes.c_uint32),
                ("QP", ctypes.c_uint32), ("nq", ctypes.c_uint32), ("np", ctypes.c_uint32),
                ("evk_words", ctypes.c_size_t), ("in_words", ctypes.c_size_t),
                ("out_words", ctypes.c_size_t), ("table_bytes", ctypes.c_size_t),
                ("tuned_variant", ctypes.c_int), ("tuned_chunks", ctypes.c_int),
                ("tuned_batch", ctypes.c_int), ("tuned_ms", ctypes.c_float),
                ("L", ctypes.c_int), ("top_L", ctypes.c_int),
                ("selected_variant", ctypes.c_int), ("selected_chunks", ctypes.c_int),
                ("tc", ctypes.c_int)]


class ks_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("ops", ctypes.c_double), ("macs", ctypes.c_double),
                ("tensor_flops", ctypes.c_double)]


KS_MLP_PARAMS, KS_MLP_MAX_BATCH = 4868, 4096


class ks_selector(ctypes.Structure):
    _fields_ = [("params", ctypes.c_float * KS_MLP_PARAMS), ("x_mean", ctypes.c_double * 6),
                ("x_std", ctypes.c_double * 6), ("t_mean", ctypes.c_double * 4),
                ("t_std", ctypes.c_double * 4), ("variant", ctypes.c_int * 4),
                ("chunks", ctypes.c_int * 4), ("l2_bytes", ctypes.c_longlong)]


class ks_job(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("d_dev", ctypes.c_void_p),
                ("evk_dev", ctypes.c_void_p), ("out_dev", ctypes.c_void_p),
                ("variant", ctypes.c_int), ("chunks", ctypes.c_int)]


_lib = None
_lock = threading.Lock()

# exported symbols declared in include/ks.h
SYMBOLS = ("ks_context_create", "ks_context_destroy", "ks_context_info", "ks_keygen",
           "ks_workspace_size", "ks_switch", "ks_switch_host", "ks_switch_batch",
           "ks_sync_status", "ks_strerror", "ks_cuda_error_string", "ks_profile_begin",
           "ks_profile_end", "ks_noalloc_scratch_bytes", "ks_switch_noalloc", "ks_tune",
           "ks_mlp_forward", "ks_mlp_grad", "ks_mlp_train", "ks_batch_status",
           "ks_context_at_level", "ks_keygen_relin", "ks_keygen_galois",
           "ks_eval_workspace_size", "ks_hmul", "ks_hrot", "ks_calibrate",
           "ks_switch_host_async", "ks_selector_load", "ks_select", "ks_host_workspace_size",
           "ks_switch_host_async_ws")


def lib_path() -> str:
    return _build.SO


def load(build: bool = True):
    """Load libks.so (building it first if needed). Raises if that fails."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build else _build.SO
        if not os.path.exists(path):
            raise RuntimeError(f"libks.so missing at {path}: the CUDA extension is required")
        l = ctypes.CDLL(path)
        vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        l.ks_context_create.argtypes = [ctypes.POINTER(ks_params), ctypes.POINTER(vp)]
        l.ks_context_destroy.argtypes = [vp]
        l.ks_context_destroy.restype = None
        l.ks_context_info.argtypes = [vp, ctypes.POINTER(ks_info)]
        l.ks_keygen.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        l.ks_workspace_size.argtypes = [vp, i, i, ctypes.POINTER(sz)]
        l.ks_switch.argtypes = [vp, vp, vp, vp, i, i, vp, sz, vp]
        l.ks_switch_host.argtypes = [vp, vp, vp, vp, i, i, vp]
        l.ks_switch_host_async.argtypes = [vp, vp, vp, vp, i, i, vp]
        l.ks_host_workspace_size.argtypes = [vp, i, i, ctypes.POINTER(ctypes.c_size_t)]
        l.ks_switch_host_async_ws.argtypes = [vp, vp, vp, vp, i, i, vp, ctypes.c_size_t, vp]
        l.ks_switch_batch.argtypes = [ctypes.POINTER(ks_job), i, i, vp]
        l.ks_tune.argtypes = [vp, vp, vp, vp, i, ctypes.POINTER(i), ctypes.POINTER(i), vp]
        l.ks_mlp_forward.argtypes = [vp, vp, i, vp, vp]
        l.ks_mlp_grad.argtypes = [vp, vp, vp, vp, i, vp, vp, vp]
        l.ks_mlp_train.argtypes = [vp, vp, vp, vp, vp, vp, vp, i, i, ctypes.c_float, i, vp, vp]
        l.ks_sync_status.argtypes = [vp, vp]
        l.ks_batch_status.argtypes = [vp]
        l.ks_context_at_level.argtypes = [vp, i, ctypes.POINTER(vp)]
        l.ks_keygen_relin.argtypes = [vp, vp, vp, vp, vp, vp]
        l.ks_keygen_galois.argtypes = [vp, vp, ctypes.c_uint32, vp, vp, vp, vp]
        l.ks_eval_workspace_size.argtypes = [vp, i, i, i, ctypes.POINTER(sz)]
        l.ks_hmul.argtypes = [vp, vp, vp, vp, vp, i, i, vp, sz, vp]
        l.ks_hrot.argtypes = [vp, vp, ctypes.c_uint32, vp, vp, i, i, vp, sz, vp]
        l.ks_calibrate.argtypes = [i, i, ctypes.POINTER(ctypes.c_double), vp]
        l.ks_selector_load.argtypes = [ctypes.POINTER(ks_selector)]
        l.ks_select.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), vp]
        l.ks_strerror.argtypes = [i]
        l.ks_strerror.restype = ctypes.c_char_p
        l.ks_noalloc_scratch_bytes.argtypes = []
        l.ks_noalloc_scratch_bytes.restype = sz
        l.ks_switch_noalloc.argtypes = [vp, vp, vp, vp, i, i, vp]
        l.ks_profile_begin.argtypes = []
        l.ks_profile_end.argtypes = [ctypes.POINTER(ks_kernel_stat), i, ctypes.POINTER(i)]
        l.ks_cuda_error_string.argtypes = []
        l.ks_cuda_error_string.restype = ctypes.c_char_p
        for name in SYMBOLS:
            if name not in ("ks_context_destroy", "ks_strerror", "ks_cuda_error_string",
                            "ks_noalloc_scratch_bytes"):
                getattr(l, name).restype = i
        _lib = l
        return l


def strerror(code: int) -> str:
    return load().ks_strerror(code).decode()


def _check(rc: int, where: str):
    if rc != KS_OK:
        raise KSError(rc, where)


def _ptr(t) -> int:
    """Device pointer of a tensor; the C-ABI takes dense row-major arrays only."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("libks takes contiguous (row-major) tensors; got strides "
                         f"{tuple(t.stride())} for shape {tuple(t.shape)}")
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def ks_context_create(dnum: int, log2n: int, L: int, q, p) -> int:
    """Returns an opaque context handle (int)."""
    qa = (ctypes.c_uint64 * len(q))(*[int(x) for x in q])
    pa = (ctypes.c_uint64 * len(p))(*[int(x) for x in p])
    prm = ks_params(dnum, log2n, L, qa, len(q), pa, len(p))
    h = ctypes.c_void_p()
    _check(load().ks_context_create(ctypes.byref(prm), ctypes.byref(h)), "ks_context_create")
    return h.value


def ks_context_at_level(ctx: int, level: int) -> int:
    """Handle of a level view of ctx (KeySwitch at `level` with ctx's keys)."""
    h = ctypes.c_void_p()
    _check(load().ks_context_at_level(ctx, level, ctypes.byref(h)), "ks_context_at_level")
    return h.value


def ks_context_destroy(ctx: int):
    load().ks_context_destroy(ctx)


def ks_context_info(ctx: int) -> dict:
    inf = ks_info()
    _check(load().ks_context_info(ctx, ctypes.byref(inf)), "ks_context_info")
    return {k: getattr(inf, k) for k, _ in ks_info._fields_}


def ks_keygen(ctx: int, s_from, s_to, a, e, evk, stream=None):
    _check(load().ks_keygen(ctx, _ptr(s_from), _ptr(s_to), _ptr(a), _ptr(e), _ptr(evk),
                            _stream(stream)), "ks_keygen")


def ks_keygen_relin(ctx: int, s, a, e, evk, stream=None):
    _check(load().ks_keygen_relin(ctx, _ptr(s), _ptr(a), _ptr(e), _ptr(evk), _stream(stream)),
           "ks_keygen_relin")


def ks_keygen_galois(ctx: int, s, galois_elt: int, a, e, evk, stream=None):
    _check(load().ks_keygen_galois(ctx, _ptr(s), galois_elt, _ptr(a), _ptr(e), _ptr(evk),
                                   _stream(stream)), "ks_keygen_galois")


KS_OP_SWITCH, KS_OP_HMUL, KS_OP_HROT = 0, 1, 2


def ks_eval_workspace_size(ctx: int, op: int, variant: int = 0, chunks: int = 0) -> int:
    n = ctypes.c_size_t()
    _check(load().ks_eval_workspace_size(ctx, op, variant, chunks, ctypes.byref(n)),
           "ks_eval_workspace_size")
    return n.value


def _ws(workspace):
    return workspace.numel() * workspace.element_size() if workspace is not None else 0


def ks_hmul(ctx: int, ct1, ct2, rlk, out, variant: int = 0, chunks: int = 0, workspace=None,
            stream=None):
    _check(load().ks_hmul(ctx, _ptr(ct1), _ptr(ct2), _ptr(rlk), _ptr(out), variant, chunks,
                          _ptr(workspace), _ws(workspace), _stream(stream)), "ks_hmul")


def ks_hrot(ctx: int, ct, galois_elt: int, rtk, out, variant: int = 0, chunks: int = 0,
            workspace=None, stream=None):
    _check(load().ks_hrot(ctx, _ptr(ct), galois_elt, _ptr(rtk), _ptr(out), variant, chunks,
                          _ptr(workspace), _ws(workspace), _stream(stream)), "ks_hrot")


def galois_elt(r: int, N: int) -> int:
    """Galois element of a rotation by r slots (5^r mod 2N); r = None: conjugation."""
    return 2 * N - 1 if r is None else pow(5, r % (N // 2), 2 * N)


def ks_workspace_size(ctx: int, variant: int, chunks: int = 0) -> int:
    n = ctypes.c_size_t()
    _check(load().ks_workspace_size(ctx, variant, chunks, ctypes.byref(n)), "ks_workspace_size")
    return n.value


def ks_switch(ctx: int, d, evk, out, variant: int = KS_AUTO, chunks: int = 0, workspace=None,
              stream=None):
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(load().ks_switch(ctx, _ptr(d), _ptr(evk), _ptr(out), variant, chunks,
                            _ptr(workspace), ws_bytes, _stream(stream)), "ks_switch")


def prepare_switch(ctx: int, d, evk, out, variant: int = KS_AUTO, chunks: int = 0,
                   workspace=None, stream=None):
    """A zero-argument callable that runs ks_switch on these buffers. Pointers, sizes and
    the stream are marshalled once, so a loop over the same buffers pays one ctypes call
    per KeySwitch; the buffers must stay alive while the callable is used."""
    f = load().ks_switch
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    vp = ctypes.c_void_p
    args = (vp(ctx), vp(_ptr(d)), vp(_ptr(evk)), vp(_ptr(out)), ctypes.c_int(variant),
            ctypes.c_int(chunks), vp(_ptr(workspace)), ctypes.c_size_t(ws_bytes),
            vp(_stream(stream)))

    def call():
        rc = f(*args)
        if rc != KS_OK:
            raise KSError(rc, "ks_switch")
    return call


def ks_noalloc_scratch_bytes() -> int:
    return load().ks_noalloc_scratch_bytes()


def ks_switch_noalloc(ctx: int, d, evk, out, variant: int = KS_AUTO, chunks: int = 0,
                      stream=None):
    """ks_switch on the library's static scratch (no device allocation).

    For callers that cannot allocate device memory while switching keys (inside
    CUDA-graph capture, under a fixed memory budget). Raises ValueError when the
    workload's scratch exceeds ks_noalloc_scratch_bytes()."""
    need = ks_workspace_size(ctx, variant, chunks)
    if need > ks_noalloc_scratch_bytes():
        raise ValueError(f"ks_switch_noalloc: needs {need} bytes of scratch, the static scratch "
                         f"holds {ks_noalloc_scratch_bytes()}; use an OutputChunked variant or "
                         f"ks_switch with a workspace")
    _check(load().ks_switch_noalloc(ctx, _ptr(d), _ptr(evk), _ptr(out), variant, chunks,
                                    _stream(stream)), "ks_switch_noalloc")


def _host_ptr(x) -> int:
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("libks takes contiguous (row-major) host arrays")
        return x.ctypes.data
    return _ptr(x)


def ks_switch_host(ctx: int, d_host, evk, out_host, variant: int = KS_AUTO, chunks: int = 0,
                   stream=None):
    """d_host / out_host: CPU tensors (pinned for full bandwidth) or numpy arrays."""
    _check(load().ks_switch_host(ctx, _host_ptr(d_host), _ptr(evk), _host_ptr(out_host),
                                 variant, chunks, _stream(stream)), "ks_switch_host")


def ks_switch_host_async(ctx: int, d_host, evk, out_host, variant: int = KS_AUTO,
                         chunks: int = 0, stream=None):
    """ks_switch_host without the synchronization; d_host / out_host must be pinned CPU
    tensors. The result is in out_host once the stream has passed the call."""
    _check(load().ks_switch_host_async(ctx, _host_ptr(d_host), _ptr(evk), _host_ptr(out_host),
                                       variant, chunks, _stream(stream)), "ks_switch_host_async")


def ks_host_workspace_size(ctx: int, variant: int = KS_AUTO, chunks: int = 0) -> int:
    n = ctypes.c_size_t()
    _check(load().ks_host_workspace_size(ctx, variant, chunks, ctypes.byref(n)),
           "ks_host_workspace_size")
    return n.value


def ks_switch_host_async_ws(ctx: int, d_host, evk, out_host, workspace, variant: int = KS_AUTO,
                            chunks: int = 0, stream=None):
    """Host-buffer KeySwitch on a caller scratch (ks_host_workspace_size bytes), the
    transfers on the copy engines; pinned host buffers."""
    nbytes = workspace.numel() * workspace.element_size()
    _check(load().ks_switch_host_async_ws(ctx, _host_ptr(d_host), _ptr(evk), _host_ptr(out_host),
                                          variant, chunks, _ptr(workspace), nbytes,
                                          _stream(stream)), "ks_switch_host_async_ws")


def prepare_switch_host_async_ws(ctx: int, d_host, evk, out_host, workspace,
                                 variant: int = KS_AUTO, chunks: int = 0, stream=None):
    """ks_switch_host_async_ws on fixed buffers as a zero-argument callable."""
    f = load().ks_switch_host_async_ws
    vp = ctypes.c_void_p
    args = (vp(ctx), vp(_host_ptr(d_host)), vp(_ptr(evk)), vp(_host_ptr(out_host)),
            ctypes.c_int(variant), ctypes.c_int(chunks), vp(_ptr(workspace)),
            ctypes.c_size_t(workspace.numel() * workspace.element_size()), vp(_stream(stream)))

    def call():
        rc = f(*args)
        if rc != KS_OK:
            raise KSError(rc, "ks_switch_host_async_ws")
    return call


def prepare_switch_host_async(ctx: int, d_host, evk, out_host, variant: int = KS_AUTO,
                              chunks: int = 0, stream=None):
    """ks_switch_host_async on fixed buffers as a zero-argument callable (arguments
    marshalled once, as prepare_switch does)."""
    f = load().ks_switch_host_async
    vp = ctypes.c_void_p
    args = (vp(ctx), vp(_host_ptr(d_host)), vp(_ptr(evk)), vp(_host_ptr(out_host)),
            ctypes.c_int(variant), ctypes.c_int(chunks), vp(_stream(stream)))

    def call():
        rc = f(*args)
        if rc != KS_OK:
            raise KSError(rc, "ks_switch_host_async")
    return call


def ks_switch_batch(jobs, flags: int = 0, stream=None):
    """jobs: sequence of (ctx, d, evk, out[, variant, chunks]) with device tensors."""
    arr = (ks_job * len(jobs))()
    for k, jb in enumerate(jobs):
        ctx, d, evk, out = jb[:4]
        v, c = (jb[4], jb[5]) if len(jb) > 4 else (0, 0)
        arr[k] = ks_job(ctx, _ptr(d), _ptr(evk), _ptr(out), v, c)
    _check(load().ks_switch_batch(arr, len(jobs), flags, _stream(stream)), "ks_switch_batch")


def ks_profile_begin():
    _check(load().ks_profile_begin(), "ks_profile_begin")


def ks_profile_end() -> list:
    """[{name, launches, ms, bytes, ops, macs, tensor_flops}] aggregated over the profiled
    launches."""
    arr = (ks_kernel_stat * 64)()
    n = ctypes.c_int()
    _check(load().ks_profile_end(arr, 64, ctypes.byref(n)), "ks_profile_end")
    return [{"name": arr[k].name.decode(), "launches": arr[k].launches, "ms": arr[k].ms,
             "bytes": arr[k].bytes, "ops": arr[k].ops, "macs": arr[k].macs,
             "tensor_flops": arr[k].tensor_flops}
            for k in range(min(n.value, 64))]


KS_CAL_BUTTERFLY, KS_CAL_MAC = 1, 2


def ks_calibrate(kind: int, iters: int = 4096, stream=None) -> float:
    """Measured ceiling of the library's modular arithmetic on this device: forward
    butterflies/s (KS_CAL_BUTTERFLY) or 128-bit multiply-accumulate terms/s (KS_CAL_MAC)."""
    r = ctypes.c_double()
    _check(load().ks_calibrate(kind, iters, ctypes.byref(r), _stream(stream)), "ks_calibrate")
    return r.value


def ks_selector_load(params, x_mean, x_std, t_mean, t_std, plans, l2_bytes: int = 0):
    """Installs a trained selector network in the library: params (KS_MLP_PARAMS floats),
    the feature and target standardisation, and plans = four (variant, chunks)."""
    import numpy as np
    sel = ks_selector()
    p = np.ascontiguousarray(params, dtype=np.float32).ravel()
    if p.size != KS_MLP_PARAMS or len(plans) != 4:
        raise ValueError("ks_selector_load: 4868 parameters and four plans")
    ctypes.memmove(sel.params, p.ctypes.data, p.nbytes)
    for k in range(6):
        sel.x_mean[k], sel.x_std[k] = float(x_mean[k]), float(x_std[k])
    for k in range(4):
        sel.t_mean[k], sel.t_std[k] = float(t_mean[k]), float(t_std[k])
        sel.variant[k], sel.chunks[k] = int(plans[k][0]), int(plans[k][1])
    sel.l2_bytes = int(l2_bytes)
    _check(load().ks_selector_load(ctypes.byref(sel)), "ks_selector_load")


def ks_select(ctx: int, stream=None):
    """The installed selector's plan for the context (also recorded as its selected
    plan). Returns (variant, chunks)."""
    v, c = ctypes.c_int(), ctypes.c_int()
    _check(load().ks_select(ctx, ctypes.byref(v), ctypes.byref(c), _stream(stream)),
           "ks_select")
    return v.value, c.value


def ks_tune(ctx: int, d, evk, out, batch: int = 1, stream=None):
    """Times the dataflows on this job and makes the fastest the context's KS_AUTO plan.
    Returns (variant, chunks)."""
    v, c = ctypes.c_int(), ctypes.c_int()
    _check(load().ks_tune(ctx, _ptr(d), _ptr(evk), _ptr(out), batch, ctypes.byref(v),
                          ctypes.byref(c), _stream(stream)), "ks_tune")
    return v.value, c.value


def variant_name(v: int, chunks: int = 0) -> str:
    names = {KS_DSOB: "DSOB", KS_DPOB: "DPOB", KS_DSOC: "DSOC", KS_DPOC: "DPOC"}
    s = names.get(v & 0xff, "AUTO")
    if (v & 0xff) in (KS_DSOC, KS_DPOC):
        s += f"-c{chunks or 2}"
    if v & KS_RADIX4:
        s += "-r4"
    if v & KS_RADIX16:
        s += "-r16"
    if v & KS_UNFUSED:
        s += "-unfused"
    sched = [f"{STAGE_NAMES[st]}{(4, 8, 16)[code - 1]}" for st in range(5)
             if (code := (v >> (KS_STAGE_SHIFT + 2 * st)) & 3)]
    if sched:
        s += "[" + ",".join(sched) + "]"
    alt = [n for n, b in (("inv", KS_COLALT_INV), ("upc", KS_COLALT_UPC), ("dnc", KS_COLALT_DNC))
           if v & b]
    if alt:
        s += "-colalt" if len(alt) == 3 else "-colalt(" + ",".join(alt) + ")"
    if v & KS_SPLIT_DOWN:
        s += "-split"
    if v & KS_BCONV_TC:
        s += "-tc"
    elif v & KS_BCONV_TC_DOWN:
        s += "-tcdown"
    return s




def ks_mlp_forward(params, x, y, stream=None):
    _check(load().ks_mlp_forward(_ptr(params), _ptr(x), x.shape[0], _ptr(y), _stream(stream)),
           "ks_mlp_forward")


def ks_mlp_grad(params, x, t, mask, grad, loss, stream=None):
    _check(load().ks_mlp_grad(_ptr(params), _ptr(x), _ptr(t), _ptr(mask), x.shape[0], _ptr(grad),
                              _ptr(loss), _stream(stream)), "ks_mlp_grad")


def ks_mlp_train(params, adam_m, adam_v, grad, x, t, mask, steps, lr, step0, loss, stream=None):
    _check(load().ks_mlp_train(_ptr(params), _ptr(adam_m), _ptr(adam_v), _ptr(grad), _ptr(x),
                               _ptr(t), _ptr(mask), x.shape[0], steps, lr, step0, _ptr(loss),
                               _stream(stream)), "ks_mlp_train")


def ks_sync_status(ctx: int, stream=None) -> int:
    return load().ks_sync_status(ctx, _stream(stream))


def ks_batch_status(stream=None) -> int:
    """Error code of the last persistent batch (synchronizes the stream): KS_OK, or
    KS_ETIMEOUT when one of its bounded waits gave up."""
    return load().ks_batch_status(_stream(stream))


class Context:
    """Owns a ks_context for one parameter set (workload.Params), or a level view of
    another Context (``Context.at_level``)."""

    def __init__(self, prm, _handle=None):
        self.prm = prm
        self.h = _handle or ks_context_create(prm.dnum, prm.logn, prm.L, prm.q, prm.p)
        self.info = ks_context_info(self.h)
        self.level = self.info["L"]
        self.nq = self.info["nq"]

    def at_level(self, level: int) -> "Context":
        """KeySwitch / HMUL / HROT at `level` with this context's keys."""
        return Context(self.prm, ks_context_at_level(self.h, level))

    def close(self):
        if self.h:
            ks_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def keygen(self, s_from, s_to, a, e, stream=None):
        import torch
        prm = self.prm
        evk = torch.empty((prm.beta, 2, prm.QP, prm.N), dtype=torch.uint64, device=a.device)
        ks_keygen(self.h, s_from, s_to, a, e, evk, stream)
        return evk

    def keygen_relin(self, s, a, e, stream=None):
        import torch
        prm = self.prm
        evk = torch.empty((prm.beta, 2, prm.QP, prm.N), dtype=torch.uint64, device=a.device)
        ks_keygen_relin(self.h, s, a, e, evk, stream)
        return evk

    def keygen_galois(self, s, k, a, e, stream=None):
        import torch
        prm = self.prm
        evk = torch.empty((prm.beta, 2, prm.QP, prm.N), dtype=torch.uint64, device=a.device)
        ks_keygen_galois(self.h, s, k, a, e, evk, stream)
        return evk

    def _out(self, like):
        import torch
        return torch.empty((2, self.nq, self.prm.N), dtype=torch.uint64, device=like.device)

    def switch(self, d, evk, out=None, variant=KS_AUTO, chunks=0, workspace=None, stream=None):
        if out is None:
            out = self._out(d)
        ks_switch(self.h, d, evk, out, variant, chunks, workspace, stream)
        return out

    def hmul(self, ct1, ct2, rlk, out=None, variant=KS_AUTO, chunks=0, workspace=None,
             stream=None):
        if out is None:
            out = self._out(ct1)
        ks_hmul(self.h, ct1, ct2, rlk, out, variant, chunks, workspace, stream)
        return out

    def hrot(self, ct, k, rtk, out=None, variant=KS_AUTO, chunks=0, workspace=None,
             stream=None):
        if out is None:
            out = self._out(ct)
        ks_hrot(self.h, ct, k, rtk, out, variant, chunks, workspace, stream)
        return out
