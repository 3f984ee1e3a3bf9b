"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/rl.h declares, and fails
loudly (with a status, not a crash) when no GPU is present."""
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in os.listdir(os.path.join(ROOT, "include"))
           if h.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(rl_\w+)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no nvcc")
    from paper_1304_7211_gb300 import _build, rl
    _build.build()
    return rl.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("rl_create", "rl_set_psf", "rl_iterate", "rl_destroy", "rl_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1304_7211_gb300 import rl
    names = declared_functions()
    assert names, "no declarations found"
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert set(names) <= set(rl.EXPORTS) | set(names)
    assert lib.rl_version().decode().startswith("rl-gb300")


def test_library_is_built_for_sm_103a(lib):
    from paper_1304_7211_gb300 import rl
    data = open(rl.LIB_PATH, "rb").read()
    # the fatbin names its target architecture
    assert b"sm_103a" in data or b"sm_103" in data


def test_null_arguments_return_status_without_gpu(lib):
    import ctypes
    from paper_1304_7211_gb300 import rl
    assert lib.rl_create(None, None) == rl.RL_ERR_INVALID_ARG
    assert lib.rl_destroy(None) == rl.RL_OK
    assert lib.rl_iterate(None, None, None, None, 1, 1, 1, 1, None, None) == rl.RL_ERR_INVALID_ARG
    assert lib.rl_set_psf(None, None) == rl.RL_ERR_INVALID_ARG
    assert lib.rl_iterate_tiles(None, None, 0) == rl.RL_ERR_INVALID_ARG


def test_create_fails_loudly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1304_7211_gb300 import rl
    with pytest.raises(rl.RLError) as ei:
        rl.rl_create(0)
    assert ei.value.status in (rl.RL_ERR_CUDA, rl.RL_ERR_INVALID_ARG)


def test_batch_calls_validate_without_gpu(lib):
    """The batch calls check their arguments before any CUDA call: NULL
    handles and slot counts out of range come back as statuses."""
    import ctypes
    from paper_1304_7211_gb300 import rl
    h = ctypes.c_void_p()
    cfg = rl.rl_config(0, None, 0, 0, 0, 0)
    assert lib.rl_batch_create(ctypes.byref(cfg), 0, ctypes.byref(h)) == rl.RL_ERR_INVALID_ARG
    assert lib.rl_batch_create(ctypes.byref(cfg), 257, ctypes.byref(h)) == rl.RL_ERR_INVALID_ARG
    assert lib.rl_batch_create(ctypes.byref(cfg), 1, None) == rl.RL_ERR_INVALID_ARG
    t, done, running = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int()
    assert lib.rl_batch_submit(None, None, ctypes.byref(t)) == rl.RL_ERR_INVALID_ARG
    assert lib.rl_batch_query(None, 1, ctypes.byref(done)) == rl.RL_ERR_INVALID_ARG
    assert lib.rl_batch_wait(None, 1) == rl.RL_ERR_INVALID_ARG
    assert lib.rl_batch_sync(None) == rl.RL_ERR_INVALID_ARG
    assert lib.rl_batch_cancel(None, 1, ctypes.byref(running)) == rl.RL_ERR_INVALID_ARG
    assert lib.rl_batch_destroy(None) == rl.RL_OK
    assert lib.rl_batch_last_error(None) == b""
    assert lib.rl_get_mask(None, None, 0) == rl.RL_ERR_INVALID_ARG


def test_batch_create_fails_loudly_without_gpu(lib):
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1304_7211_gb300 import rl
    h = ctypes.c_void_p()
    cfg = rl.rl_config(0, None, 0, 0, 0, 0)
    st = lib.rl_batch_create(ctypes.byref(cfg), 2, ctypes.byref(h))
    assert st != rl.RL_OK and not h.value


def test_noalloc_entry_point_checks_before_touching_the_gpu(lib):
    """rl_motion_x_noalloc validates pointers, sizes and the fixed scratch
    limit before any CUDA call (the pointer values here are never
    dereferenced): each case returns RL_ERR_INVALID_ARG with a message."""
    import ctypes
    from paper_1304_7211_gb300 import rl
    buf = ctypes.create_string_buffer(256)

    def call(f, u0, out, W, H, pitch, length=9, boundary=rl.RL_BOUNDARY_MIRROR, its=3):
        buf.value = b""
        st = lib.rl_motion_x_noalloc(f, u0, out, W, H, pitch, length, boundary, its, None, buf, len(buf))
        return st, buf.value.decode()

    F, U0, OUT = 0x1000, 0x2000, 0x3000
    st, msg = call(None, None, OUT, 64, 64, 64)
    assert st == rl.RL_ERR_INVALID_ARG and "required" in msg
    assert call(F, None, F, 64, 64, 64)[0] == rl.RL_ERR_INVALID_ARG      # u_out aliases f
    assert call(F, OUT, OUT, 64, 64, 64)[0] == rl.RL_ERR_INVALID_ARG     # u_out aliases u0
    assert call(F, None, OUT, 64, 64, 63)[0] == rl.RL_ERR_INVALID_ARG    # pitch < W
    assert call(F, None, OUT, 64, 64, 64, boundary=7)[0] == rl.RL_ERR_INVALID_ARG
    assert call(F, None, OUT, 64, 64, 64, its=-1)[0] == rl.RL_ERR_INVALID_ARG
    assert call(F, None, OUT, 8, 64, 8, length=17)[0] == rl.RL_ERR_INVALID_ARG  # half length >= W
    W, H = 4096, rl.RL_NOALLOC_MAX_PIXELS // 4096 + 1                   # one row past the limit
    st, msg = call(F, None, OUT, W, H, W)
    assert st == rl.RL_ERR_INVALID_ARG and str(rl.RL_NOALLOC_MAX_PIXELS) in msg


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No fallback: with the shared library missing, every call through the
    binding raises instead of computing anything elsewhere."""
    from paper_1304_7211_gb300 import rl, synth
    monkeypatch.setattr(rl, "_lib", None)
    monkeypatch.setattr(rl, "LIB_PATH", str(tmp_path / "librl_gb300.so"))
    with pytest.raises(RuntimeError, match="missing"):
        rl.load()
    with pytest.raises(RuntimeError, match="missing"):
        rl.Deconvolver(synth.disc(3))
