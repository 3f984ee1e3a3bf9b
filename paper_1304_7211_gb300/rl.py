"""ctypes binding of the C ABI declared in ``include/rl.h``.

Argument marshalling only: every step of the Richardson-Lucy iteration runs in
the CUDA kernels of ``librl_gb300.so``.  The functions keep the C names
(``rl_create``, ``rl_set_psf``, ``rl_iterate``, ``rl_destroy``,
``rl_last_error``).  Buffers may be passed as raw integer addresses, torch
tensors (device or host) or numpy arrays (host); PyTorch is used only for
device memory and the CUDA stream handle.

There is no fallback: if the shared library is missing this module raises,
and the library itself refuses to run on anything but an sm_103 GPU.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librl_gb300.so")

RL_OK, RL_ERR_INVALID_ARG, RL_ERR_UNSUPPORTED, RL_ERR_OOM, RL_ERR_CUDA, \
    RL_ERR_TIMEOUT, RL_ERR_STATE = range(7)
RL_PSF_MOTION, RL_PSF_DISC, RL_PSF_DENSE = range(3)
RL_STORAGE_F32, RL_STORAGE_BF16, RL_STORAGE_F16 = range(3)
RL_BOUNDARY_MIRROR, RL_BOUNDARY_CLAMP = range(2)
RL_PATH_AUTO, RL_PATH_RUNSUM, RL_PATH_SPAN, RL_PATH_STENCIL, RL_PATH_SAT = range(5)

STORAGE = {"f32": RL_STORAGE_F32, "bf16": RL_STORAGE_BF16, "f16": RL_STORAGE_F16}
BOUNDARY = {"mirror": RL_BOUNDARY_MIRROR, "clamp": RL_BOUNDARY_CLAMP}
PATH = {"auto": RL_PATH_AUTO, "runsum": RL_PATH_RUNSUM, "span": RL_PATH_SPAN,
        "stencil": RL_PATH_STENCIL, "sat": RL_PATH_SAT}
PATH_NAME = {v: k for k, v in PATH.items()}
STATUS_NAME = {RL_OK: "RL_OK", RL_ERR_INVALID_ARG: "RL_ERR_INVALID_ARG",
               RL_ERR_UNSUPPORTED: "RL_ERR_UNSUPPORTED", RL_ERR_OOM: "RL_ERR_OOM",
               RL_ERR_CUDA: "RL_ERR_CUDA", RL_ERR_TIMEOUT: "RL_ERR_TIMEOUT",
               RL_ERR_STATE: "RL_ERR_STATE"}


class rl_psf_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("axis", ctypes.c_int), ("length", ctypes.c_int),
                ("radius", ctypes.c_int), ("kw", ctypes.c_int), ("kh", ctypes.c_int),
                ("anchor_x", ctypes.c_int), ("anchor_y", ctypes.c_int),
                ("taps", ctypes.POINTER(ctypes.c_float))]


class rl_thinning(ctypes.Structure):
    _fields_ = [("threshold", ctypes.c_float), ("relative", ctypes.c_int),
                ("reset_period", ctypes.c_int), ("update_period", ctypes.c_int),
                ("schedule", ctypes.c_void_p)]


RL_FLAG_PER_ITERATION = 1
RL_FLAG_ADJOINT_TRANSPOSE = 2
RL_FLAG_PERSISTENT = 4
RL_FLAG_AUTOTUNE = 8
ADJOINT = {"padflip": 0, "transpose": RL_FLAG_ADJOINT_TRANSPOSE}


class rl_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("storage", ctypes.c_int), ("boundary", ctypes.c_int), ("path", ctypes.c_int),
                ("flags", ctypes.c_int)]


class rl_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_longlong), ("pixel_iterations", ctypes.c_longlong),
                ("active_pixel_iterations", ctypes.c_longlong), ("device_ms", ctypes.c_double),
                ("path", ctypes.c_int), ("launches", ctypes.c_int),
                ("flux_f", ctypes.c_double), ("flux_u", ctypes.c_double)]


class rl_job(ctypes.Structure):
    _fields_ = [("f", ctypes.c_void_p), ("u0", ctypes.c_void_p), ("u_out", ctypes.c_void_p),
                ("f_host", ctypes.c_void_p), ("u_host", ctypes.c_void_p), ("W", ctypes.c_int),
                ("H", ctypes.c_int), ("pitch", ctypes.c_longlong), ("iterations", ctypes.c_int),
                ("psf", rl_psf_desc), ("thin", ctypes.POINTER(rl_thinning))]


class RLError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAME.get(status, status)}: {message}")
        self.status = status
        self.message = message


_lib = None

# Every symbol include/rl.h declares.
EXPORTS = ("rl_create", "rl_set_psf", "rl_iterate", "rl_destroy", "rl_last_error", "rl_version",
           "rl_get_mask", "rl_motion_x_noalloc", "rl_batch_create", "rl_batch_submit",
           "rl_batch_query", "rl_batch_wait", "rl_batch_sync", "rl_batch_destroy",
           "rl_batch_last_error", "rl_batch_cancel", "rl_iterate_tiles", "rl_selftest_wait_timeout",
           "rl_test_fail_allocation", "rl_test_persist_ctas", "rl_test_persist_wait_ns")
RL_NOALLOC_MAX_PIXELS = 4194304


def load() -> ctypes.CDLL:
    """Load ``librl_gb300.so`` (build it first with ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    lib.rl_create.restype = ctypes.c_int
    lib.rl_create.argtypes = [ctypes.POINTER(rl_config), ctypes.POINTER(P)]
    lib.rl_set_psf.restype = ctypes.c_int
    lib.rl_set_psf.argtypes = [P, ctypes.POINTER(rl_psf_desc)]
    lib.rl_iterate.restype = ctypes.c_int
    lib.rl_iterate.argtypes = [P, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                               ctypes.c_int, ctypes.POINTER(rl_thinning), ctypes.POINTER(rl_stats)]
    lib.rl_destroy.restype = ctypes.c_int
    lib.rl_destroy.argtypes = [P]
    lib.rl_last_error.restype = ctypes.c_char_p
    lib.rl_last_error.argtypes = [P]
    lib.rl_version.restype = ctypes.c_char_p
    lib.rl_version.argtypes = []
    lib.rl_get_mask.restype = ctypes.c_int
    lib.rl_get_mask.argtypes = [P, P, ctypes.c_longlong]
    lib.rl_batch_create.restype = ctypes.c_int
    lib.rl_batch_create.argtypes = [ctypes.POINTER(rl_config), ctypes.c_int, ctypes.POINTER(P)]
    lib.rl_batch_submit.restype = ctypes.c_int
    lib.rl_batch_submit.argtypes = [P, ctypes.POINTER(rl_job), ctypes.POINTER(ctypes.c_longlong)]
    lib.rl_batch_query.restype = ctypes.c_int
    lib.rl_batch_query.argtypes = [P, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int)]
    lib.rl_batch_wait.restype = ctypes.c_int
    lib.rl_batch_wait.argtypes = [P, ctypes.c_longlong]
    lib.rl_batch_sync.restype = ctypes.c_int
    lib.rl_batch_sync.argtypes = [P]
    lib.rl_batch_destroy.restype = ctypes.c_int
    lib.rl_batch_destroy.argtypes = [P]
    lib.rl_batch_last_error.restype = ctypes.c_char_p
    lib.rl_batch_last_error.argtypes = [P]
    lib.rl_batch_cancel.restype = ctypes.c_int
    lib.rl_batch_cancel.argtypes = [P, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int)]
    lib.rl_test_fail_allocation.restype = None
    lib.rl_test_fail_allocation.argtypes = [ctypes.c_int]
    lib.rl_test_persist_ctas.restype = None
    lib.rl_test_persist_ctas.argtypes = [ctypes.c_int]
    lib.rl_test_persist_wait_ns.restype = None
    lib.rl_test_persist_wait_ns.argtypes = [ctypes.c_ulonglong]
    lib.rl_iterate_tiles.restype = ctypes.c_int
    lib.rl_iterate_tiles.argtypes = [P, ctypes.POINTER(rl_job), ctypes.c_int]
    lib.rl_motion_x_noalloc.restype = ctypes.c_int
    lib.rl_motion_x_noalloc.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                                        ctypes.c_char_p, ctypes.c_int]
    lib.rl_selftest_wait_timeout.restype = ctypes.c_int
    lib.rl_selftest_wait_timeout.argtypes = [ctypes.c_int, ctypes.c_int]
    _lib = lib
    return lib


def rl_last_error(ctx) -> str:
    return load().rl_last_error(ctx).decode()


def _check(rc: int, ctx) -> None:
    if rc != RL_OK:
        raise RLError(rc, rl_last_error(ctx))


def rl_create(device: int = 0, stream=None, storage="f32", boundary="mirror", path="auto",
              flags: int = 0):
    """Create a context; ``stream`` is a ``cudaStream_t`` as int, a
    ``torch.cuda.Stream`` or None (default stream)."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    cfg = rl_config(device, stream or None, STORAGE.get(storage, storage),
                    BOUNDARY.get(boundary, boundary), PATH.get(path, path), flags)
    h = ctypes.c_void_p()
    rc = load().rl_create(ctypes.byref(cfg), ctypes.byref(h))
    _check(rc, None)
    _CTX_ESIZE[h.value] = ESIZE.get(cfg.storage)
    return h


def psf_desc(spec) -> tuple[rl_psf_desc, object]:
    """Descriptor from a PSF spec with attributes kind/axis/length/radius/
    taps/kw/kh (e.g. ``synth.PsfSpec``).  Returns (desc, keepalive)."""
    kind = {"motion": RL_PSF_MOTION, "disc": RL_PSF_DISC, "dense": RL_PSF_DENSE}[spec.kind]
    keep = None
    taps = None
    kw = kh = 0
    if kind == RL_PSF_DENSE:
        keep = (ctypes.c_float * len(spec.taps))(*spec.taps)
        taps = ctypes.cast(keep, ctypes.POINTER(ctypes.c_float))
        kw, kh = spec.kw, spec.kh
    ax = getattr(spec, "anchor_x", -1)
    ay = getattr(spec, "anchor_y", -1)
    d = rl_psf_desc(kind, getattr(spec, "axis", 0), getattr(spec, "length", 0),
                    getattr(spec, "radius", 0), kw, kh, ax, ay, taps)
    return d, keep


def rl_set_psf(ctx, spec_or_desc) -> None:
    if isinstance(spec_or_desc, rl_psf_desc):
        d, keep = spec_or_desc, None
    else:
        d, keep = psf_desc(spec_or_desc)
    _check(load().rl_set_psf(ctx, ctypes.byref(d)), ctx)
    del keep


ESIZE = {RL_STORAGE_F32: 4, RL_STORAGE_BF16: 2, RL_STORAGE_F16: 2}
_CTX_ESIZE = {}  # context handle -> bytes per stored image element


def _ctx_esize(ctx):
    return _CTX_ESIZE.get(getattr(ctx, "value", ctx))


def _bytes_from(x) -> int | None:
    """Bytes from the first element of a torch tensor or numpy array to the
    end of the memory it lies in, or None when that is not known."""
    if hasattr(x, "untyped_storage"):
        return x.untyped_storage().nbytes() - x.storage_offset() * x.element_size()
    if hasattr(x, "ctypes") and hasattr(x, "nbytes"):
        root = x
        while getattr(root, "base", None) is not None and hasattr(root.base, "ctypes"):
            root = root.base
        if root.base is not None:
            return None
        return root.ctypes.data + root.nbytes - x.ctypes.data
    return None


def _check_span(name: str, x, W: int, H: int, pitch: int, esize: int | None) -> None:
    """Refuse an image buffer (torch tensor or numpy array) that ends before
    the last pixel a C call with (W, H, pitch) would touch: (H - 1) pitch + W
    elements of the context's storage type.  Raw addresses are the caller's
    responsibility; sizes the library rejects itself are left to it."""
    if x is None or isinstance(x, int) or esize is None or W < 1 or H < 1 or pitch < W:
        return
    have = _bytes_from(x)
    need = ((H - 1) * pitch + W) * esize
    if have is not None and have < need:
        raise ValueError(f"{name} holds {have} bytes from its start; W={W}, H={H}, pitch={pitch} "
                         f"need {need}")


def _addr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):          # torch tensor
        return x.data_ptr()
    if hasattr(x, "ctypes"):            # numpy array
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def rl_iterate(ctx, f, u0, u_out, W: int, H: int, pitch: int, iterations: int,
               thinning: rl_thinning | None = None, stats: bool = False):
    """Run RL iterations; returns an ``rl_stats`` when ``stats`` is true."""
    st = rl_stats() if stats else None
    es = _ctx_esize(ctx)
    for name, x in (("f", f), ("u0", u0), ("u_out", u_out)):
        _check_span(name, x, W, H, pitch, es)
    rc = load().rl_iterate(ctx, _addr(f), _addr(u0), _addr(u_out), W, H, pitch, iterations,
                           ctypes.byref(thinning) if thinning is not None else None,
                           ctypes.byref(st) if st is not None else None)
    _check(rc, ctx)
    return st


def rl_iterate_tiles(ctx, jobs) -> None:
    """Batched (request, tile) form: ``jobs`` is a sequence of
    ``(f, u0, u_out, W, H, pitch, iterations)`` on the device, all under the
    context's PSF (disc or box kernel)."""
    arr = (rl_job * max(len(jobs), 1))()
    es = _ctx_esize(ctx)
    for i, (f, u0, u_out, W, H, pitch, iterations) in enumerate(jobs):
        for name, x in (("f", f), ("u0", u0), ("u_out", u_out)):
            _check_span(f"job {i}: {name}", x, W, H, pitch, es)
        arr[i] = rl_job(_addr(f), _addr(u0), _addr(u_out), None, None, W, H, pitch, iterations,
                        rl_psf_desc(), None)
    rc = load().rl_iterate_tiles(ctx, arr, len(jobs))
    _check(rc, ctx)


def rl_get_mask(ctx, dst, dst_pitch: int) -> None:
    """Copy the active mask left by the last thinned rl_iterate into dst."""
    _check(load().rl_get_mask(ctx, _addr(dst), dst_pitch), ctx)


def rl_motion_x_noalloc(f, u0, u_out, W: int, H: int, pitch: int, length: int,
                        boundary="mirror", iterations: int = 1, stream=None) -> None:
    """Allocation-free running-sum RL for horizontal motion blur (FP32, device
    pointers, current device); see include/rl.h.  Raises RLError on failure.

    f, u0 (or None) and u_out are FP32 CUDA tensors (or raw device addresses
    as int): this entry point cannot stage host memory, so numpy arrays, CPU
    tensors and other dtypes are refused here, before the library is called."""
    for name, t in (("f", f), ("u0", u0), ("u_out", u_out)):
        if t is None and name == "u0":
            continue
        if isinstance(t, int):
            continue
        if not hasattr(t, "data_ptr") or not getattr(t, "is_cuda", False) or str(t.dtype) != "torch.float32":
            raise TypeError(f"rl_motion_x_noalloc: {name} must be a float32 CUDA tensor or a device address")
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    buf = ctypes.create_string_buffer(256)
    rc = load().rl_motion_x_noalloc(_addr(f), _addr(u0), _addr(u_out), W, H, pitch, length,
                                    BOUNDARY.get(boundary, boundary), iterations, stream or None,
                                    buf, len(buf))
    if rc != RL_OK:
        raise RLError(rc, buf.value.decode())


def rl_destroy(ctx) -> None:
    if ctx:
        _CTX_ESIZE.pop(getattr(ctx, "value", ctx), None)
        load().rl_destroy(ctx)


def thinning(threshold: float, relative: bool = True, reset_period: int = 10,
             update_period: int = 1, schedule=None) -> rl_thinning:
    """Selective-convolution parameters; ``schedule`` (optional, uint8
    iterations x H x W, host or device) replays a recorded used-pixel mask."""
    t = rl_thinning(float(threshold), int(bool(relative)), int(reset_period),
                    int(update_period), _addr(schedule))
    t._keep = schedule
    return t


STORAGE_DTYPE = {"f32": "float32", "bf16": "bfloat16", "f16": "float16"}


def _image_view(x, name: str) -> tuple:
    """(H, W, row pitch in elements, element stride along x, dtype name,
    CUDA device index or None) of a 2-D torch tensor or numpy array.  The
    stride of a dimension of extent 1 is never used, so a single row reads
    as pitch W and a single column as element stride 1."""
    if hasattr(x, "data_ptr") and hasattr(x, "stride") and callable(x.stride):  # torch tensor
        if x.dim() != 2:
            raise ValueError(f"{name} must be a 2-D image, got {x.dim()} dimensions")
        dev = x.device.index if x.is_cuda else None
        H, W, pitch, sx, dt = x.shape[0], x.shape[1], x.stride(0), x.stride(1), str(x.dtype)
        dt = dt.replace("torch.", "")
    elif hasattr(x, "ctypes") and hasattr(x, "strides"):  # numpy array
        if x.ndim != 2:
            raise ValueError(f"{name} must be a 2-D image, got {x.ndim} dimensions")
        es = x.itemsize
        if x.strides[0] % es or x.strides[1] % es:
            raise ValueError(f"{name}: strides must be whole elements")
        H, W, pitch, sx, dt, dev = x.shape[0], x.shape[1], x.strides[0] // es, x.strides[1] // es, \
            str(x.dtype), None
    else:
        raise TypeError(f"{name} must be a torch tensor or a numpy array, got {type(x)}")
    if W == 1:
        sx = 1
    if H == 1 and sx == 1:
        pitch = W
    return H, W, pitch, sx, dt, dev


def check_images(storage: str, f, u0=None, out=None, device: int | None = None) -> tuple:
    """Check that f, u0 and out describe one image layout the C call can take
    with a single (W, H, pitch): 2-D, pixels contiguous along x, the storage
    element type of the context, one row pitch >= W for all three, and CUDA
    tensors on the context's device.  Returns (W, H, pitch).  A mismatch
    would make the library read or write past a buffer, so it raises here."""
    if not isinstance(storage, str):
        storage = {v: k for k, v in STORAGE.items()}[storage]
    want = STORAGE_DTYPE[storage]
    H, W, pitch, sx, dt, dev = _image_view(f, "f")
    if H < 1 or W < 1:
        raise ValueError(f"f is empty ({H}x{W})")
    if sx != 1 or pitch < W:
        raise ValueError("f: pixels along a row must be contiguous and rows must not overlap "
                         f"(strides {pitch}, {sx})")
    for name, x, d in (("f", f, dev), ("u0", u0, None), ("out", out, None)):
        if x is None:
            continue
        if x is not f:
            h, w, p, s, dt, d = _image_view(x, name)
            if (h, w) != (H, W) or s != 1 or p != pitch:
                raise ValueError(f"{name} must be a {H}x{W} image with contiguous rows of pitch {pitch} "
                                 f"(the layout of f); got {h}x{w}, strides ({p}, {s})")
        if dt != want:
            raise TypeError(f"{name} has element type {dt}; this context stores {want}")
        if d is not None and device is not None and d != device:
            raise ValueError(f"{name} is on cuda:{d}; this context runs on cuda:{device}")
    return W, H, pitch


def _empty_like_layout(f, H: int, W: int, pitch: int):
    """An uninitialised image with the dtype, device and row pitch of f."""
    if hasattr(f, "new_empty_strided"):
        return f.new_empty_strided((H, W), (pitch, 1))
    import numpy as np
    return np.empty((H, pitch), dtype=f.dtype)[:, :W]


class Deconvolver:
    """Owns one context and one PSF; runs RL on torch tensors or numpy arrays.

    ``run(f, iterations)`` with a CUDA tensor returns a CUDA tensor (work is
    issued on the current torch stream); with a numpy array or CPU tensor the
    library stages the data itself and the result comes back on the host.
    """

    def __init__(self, spec, device: int = 0, storage="f32", boundary="mirror",
                 path="auto", stream=None, flags: int = 0, adjoint="padflip"):
        self.device = device
        flags |= ADJOINT[adjoint]
        self.storage = storage
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:  # pragma: no cover - torch is optional here
                stream = None
        self.ctx = rl_create(device, stream, storage, boundary, path, flags)
        rl_set_psf(self.ctx, spec)

    def close(self):
        if self.ctx:
            rl_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def mask(self):
        """Active mask (uint8 numpy array) left by the last thinned run."""
        import numpy as np
        m = np.zeros((self._last_hw[0], self._last_hw[1]), np.uint8)
        rl_get_mask(self.ctx, m, m.shape[1])
        return m

    def run(self, f, iterations: int, u0=None, out=None, thin: rl_thinning | None = None,
            stats: bool = False):
        W, H, pitch = check_images(self.storage, f, u0, out, self.device)
        self._last_hw = (H, W)
        if out is None:
            out = _empty_like_layout(f, H, W, pitch)
        st = rl_iterate(self.ctx, f, u0, out, W, H, pitch, iterations, thin, stats)
        return (out, st) if stats else out


class Batch:
    """Many independent deconvolutions over ``slots`` CUDA streams (the C
    ``rl_batch_*`` API).  ``submit`` returns a ticket at once; jobs on
    different slots overlap on the GPU."""

    def __init__(self, slots: int = 8, device: int = 0, storage="f32", boundary="mirror",
                 path="auto", flags: int = 0):
        cfg = rl_config(device, None, STORAGE.get(storage, storage),
                        BOUNDARY.get(boundary, boundary), PATH.get(path, path), flags)
        h = ctypes.c_void_p()
        rc = load().rl_batch_create(ctypes.byref(cfg), slots, ctypes.byref(h))
        if rc != RL_OK:
            raise RLError(rc, "rl_batch_create failed")
        self.h = h
        self.esize = ESIZE.get(cfg.storage)

    def _check(self, rc):
        if rc != RL_OK:
            raise RLError(rc, load().rl_batch_last_error(self.h).decode())

    def submit(self, spec, f, u_out, iterations: int, W: int, H: int, pitch: int | None = None,
               u0=None, f_host=None, u_host=None, thin: rl_thinning | None = None) -> int:
        for name, x in (("f", f), ("u0", u0), ("u_out", u_out)):
            _check_span(name, x, W, H, pitch or W, self.esize)
        for name, x in (("f_host", f_host), ("u_host", u_host)):  # packed rows
            _check_span(name, x, W, H, W, self.esize)
        d, keep = psf_desc(spec)
        job = rl_job(_addr(f), _addr(u0), _addr(u_out), _addr(f_host), _addr(u_host), W, H,
                     pitch or W, iterations, d,
                     ctypes.pointer(thin) if thin is not None else None)
        t = ctypes.c_longlong()
        self._check(load().rl_batch_submit(self.h, ctypes.byref(job), ctypes.byref(t)))
        del keep
        return t.value

    def query(self, ticket: int) -> bool:
        done = ctypes.c_int()
        self._check(load().rl_batch_query(self.h, ticket, ctypes.byref(done)))
        return bool(done.value)

    def wait(self, ticket: int) -> None:
        self._check(load().rl_batch_wait(self.h, ticket))

    def cancel(self, ticket: int) -> bool:
        """Cancel a job; returns True if it was already on the GPU (it runs to
        the end and its result is to be discarded), False if it was dropped
        before it started."""
        running = ctypes.c_int()
        self._check(load().rl_batch_cancel(self.h, ticket, ctypes.byref(running)))
        return bool(running.value)

    def sync(self) -> None:
        self._check(load().rl_batch_sync(self.h))

    def close(self) -> None:
        if self.h:
            load().rl_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
