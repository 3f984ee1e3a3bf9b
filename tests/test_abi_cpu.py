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
