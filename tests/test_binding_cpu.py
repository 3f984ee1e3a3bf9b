"""Host-side checks that need no GPU: the ctypes binding agrees with the C
header it marshals for (struct layouts, constants, argument counts), and the
host logic of the bench and the server (ncu ingestion, the source-hash gate
on a DRAM capture, the roofline arithmetic, the FIFO baseline's queue)
computes what it states."""
import ctypes
import json
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rl.h")

STRUCTS = ("rl_psf_desc", "rl_thinning", "rl_config", "rl_stats", "rl_job")
CONSTANTS = ("RL_OK", "RL_ERR_INVALID_ARG", "RL_ERR_UNSUPPORTED", "RL_ERR_OOM", "RL_ERR_CUDA",
             "RL_ERR_TIMEOUT", "RL_ERR_STATE", "RL_PSF_MOTION", "RL_PSF_DISC", "RL_PSF_DENSE",
             "RL_STORAGE_F32", "RL_STORAGE_BF16", "RL_STORAGE_F16", "RL_BOUNDARY_MIRROR",
             "RL_BOUNDARY_CLAMP", "RL_PATH_AUTO", "RL_PATH_RUNSUM", "RL_PATH_SPAN", "RL_PATH_STENCIL",
             "RL_PATH_SAT", "RL_FLAG_PER_ITERATION", "RL_FLAG_ADJOINT_TRANSPOSE", "RL_FLAG_PERSISTENT",
             "RL_FLAG_AUTOTUNE", "RL_NOALLOC_MAX_PIXELS")


@pytest.fixture(scope="module")
def header_layout(tmp_path_factory):
    """sizeof / offsetof of every field of the public structs and the value
    of every public constant, as the C compiler sees include/rl.h."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1304_7211_gb300 import rl
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "rl.h"', "int main(void) {",
             '  printf("{");']
    for s in STRUCTS:
        fields = [f for f, _ in getattr(rl, s)._fields_]
        lines.append(f'  printf("\\"{s}\\": {{\\"size\\": %zu", sizeof({s}));')
        for f in fields:
            lines.append(f'  printf(", \\"{f}\\": %zu", offsetof({s}, {f}));')
        lines.append('  printf("}, ");')
    for c in CONSTANTS:
        lines.append(f'  printf("\\"{c}\\": %lld, ", (long long)({c}));')
    lines += ['  printf("\\"end\\": 0}\\n");', "  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "probe.c", d / "probe"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe)], check=True, capture_output=True)
    return json.loads(subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout)


@pytest.mark.parametrize("name", STRUCTS)
def test_binding_struct_layout_matches_header(header_layout, name):
    from paper_1304_7211_gb300 import rl
    cls = getattr(rl, name)
    want = header_layout[name]
    assert ctypes.sizeof(cls) == want["size"], name
    for f, _ in cls._fields_:
        assert getattr(cls, f).offset == want[f], (name, f)


def test_binding_constants_match_header(header_layout):
    from paper_1304_7211_gb300 import rl
    for c in CONSTANTS:
        assert getattr(rl, c) == header_layout[c], c


def _prototypes():
    """name -> number of parameters, from the function declarations of the header."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    src = re.sub(r"^\s*#.*$", "", src, flags=re.M)
    out = {}
    for m in re.finditer(r"\b(rl_\w+)\s*\(([^()]*)\)\s*;", src):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argument_counts_match_header():
    """Every exported function the binding types has as many argtypes as the
    header declares parameters (a dropped argument would shift the rest)."""
    from paper_1304_7211_gb300 import _build, rl
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no nvcc")
    _build.build()
    lib = rl.load()
    protos = _prototypes()
    assert set(rl.EXPORTS) == set(protos), set(rl.EXPORTS) ^ set(protos)
    for name, n in protos.items():
        fn = getattr(lib, name)
        if fn.argtypes is not None:
            assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)


def test_psf_descriptor_marshalling():
    from paper_1304_7211_gb300 import rl, synth
    d, keep = rl.psf_desc(synth.disc(12))
    assert (d.kind, d.radius, keep) == (rl.RL_PSF_DISC, 12, None)
    d, _ = rl.psf_desc(synth.motion(31, 1))
    assert (d.kind, d.axis, d.length) == (rl.RL_PSF_MOTION, 1, 31)
    spec = synth.gaussian(7, 1.5)
    d, keep = rl.psf_desc(spec)
    assert (d.kind, d.kw, d.kh) == (rl.RL_PSF_DENSE, 7, 7)
    taps = np.ctypeslib.as_array(d.taps, shape=(49,))
    np.testing.assert_array_equal(taps, np.asarray(spec.taps, dtype=np.float32))
    t = rl.thinning(1e-4, True, 10, 10)
    assert (t.relative, t.reset_period, t.update_period, t.schedule) == (1, 10, 10, None)
    assert t.threshold == pytest.approx(1e-4)


# ---- bench host logic ------------------------------------------------------

def test_kernel_key_strips_namespaces_and_parameters():
    import bench
    assert bench.kernel_key("void (anonymous namespace)::k_disc_persist<float, DiscOp<8, 64, 4, 64>, 0>"
                            "(rl::PersistArgs)") == "k_disc_persist<float, DiscOp<8, 64, 4, 64>, 0>"
    assert bench.kernel_key("<unnamed>::k_sum_final(const double *, double *, int)") == "k_sum_final"
    assert bench.kernel_key("void rl::k_transpose<unsigned int>(const unsigned int *, unsigned int *)") \
        == "k_transpose<unsigned int>"


def test_ingest_ncu_scales_units_and_averages_per_launch(tmp_path):
    import bench
    csv = tmp_path / "launches.csv"
    csv.write_text(
        "==PROF== Connected to process\n"
        '"ID","Kernel Name","dram__bytes_read.sum","dram__bytes_write.sum","gpu__time_duration.sum"\n'
        '"","","Mbyte","Kbyte","usecond"\n'
        '"0","void k_a<float>(int)","2","500","10"\n'
        '"1","void k_a<float>(int)","4","1,500","30"\n'
        '"2","k_b(int)","1","0","1"\n')
    out = bench.ingest_ncu(str(csv), str(tmp_path / "t.json"), "w", "cmd")
    a, b = out["kernels"]["k_a<float>"], out["kernels"]["k_b"]
    assert a["launches"] == 2 and b["launches"] == 1
    assert a["dram_bytes_per_launch"] == pytest.approx((2e6 + 5e5 + 4e6 + 1.5e6) / 2)
    assert a["us_per_launch"] == pytest.approx(20.0)
    assert b["dram_bytes_per_launch"] == pytest.approx(1e6)
    assert out["build_sha"] == bench.source_sha()
    assert json.load(open(tmp_path / "t.json")) == out


def test_traffic_capture_counts_only_for_its_own_sources(tmp_path, monkeypatch):
    import bench
    cap = {"build_sha": bench.source_sha(), "kernels": {"k_disc_persist<float, DiscOp<8, 64, 4, 64>, 0>":
                                                         {"dram_bytes_per_launch": 2000.0}}}
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(cap))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(p))
    assert bench.measured_traffic() == cap
    cap["build_sha"] = "0" * 16
    p.write_text(json.dumps(cap))
    assert bench.measured_traffic() is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "absent.json"))
    assert bench.measured_traffic() is None


def test_solve_roofline_arithmetic():
    import bench
    from paper_1304_7211_gb300 import synth
    pk = {"hbm_gbs": 6000.0, "sm_max_mhz": 2000.0}
    px = bench.SIZE * bench.SIZE
    cap = {"kernels": {"k_disc_persist<float, DiscOp<8, 64, 4, 64>, 0>": {"dram_bytes_per_launch": 4e6},
                       "k_motion_x_tb<float, 0, 13, 0>": {"dram_bytes_per_launch": 3e6}}}
    # disc r = 8, one persistent launch of 200 iterations taking 8 ms
    r = bench.solve_roofline(synth.disc(8), 8.0, 1, pk, "measured", 100, cap)
    assert r["bound"] == "alu"
    assert r["algorithmic_per_unit"] == px * (4 * 17 + 4)
    assert r["peak"] == pytest.approx(100 * 128 * 2000e6 / 1e12)
    unit_s = 8e-3 / bench.ITERS
    assert r["achieved"] == pytest.approx(px * 72 / unit_s / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] == pytest.approx(4e6 / bench.ITERS)
    assert r["hbm_equiv_gbs"] == pytest.approx(12 * px / unit_s / 1e9)
    # two launches per iteration: no capture of the halves -> traffic unknown
    assert bench.solve_roofline(synth.disc(8), 8.0, 400, pk, "measured", 100, cap)["traffic"] is None
    # motion with rows resident: 12 B/px-it effective over the whole solve
    m = bench.solve_roofline(synth.motion(31, 0), 2.0, 1, pk, "measured", 100, cap)
    assert m["bound"] == "hbm" and m["peak"] == 6000.0
    assert m["achieved"] == pytest.approx(12 * px * bench.ITERS / 2e-3 / 1e9)
    assert m["traffic"] == pytest.approx(3e6)


# ---- server host logic -----------------------------------------------------

def test_fifo_baseline_is_a_single_server_queue():
    """Request i starts at max(arrival_i, end of request i-1): arrivals
    0, 1, 1.5 s with service 2, 1, 1 s end at 2, 3, 4 s."""
    from paper_1304_7211_gb300 import serve
    f = np.zeros((10, 10), np.float32)
    reqs = [serve.Request(j, t, f, None, 5) for j, t in enumerate((1.5, 0.0, 1.0))]
    svc = [1.0, 2.0, 1.0]  # matched to reqs: request at 1.5 s takes 1 s, at 0 s 2 s, at 1 s 1 s
    rep = serve.fifo_report(reqs, svc)
    lat = np.array([2000.0, 2000.0, 2500.0])
    assert rep.n == 3
    assert rep.wall_s == pytest.approx(4.0)
    assert rep.p50_ms == pytest.approx(np.percentile(lat, 50))
    assert rep.p99_ms == pytest.approx(np.percentile(lat, 99))
    assert rep.mean_ms == pytest.approx(lat.mean())
    assert rep.px_it == 3 * 100 * 5
    assert rep.mpx_it_per_s == pytest.approx(1500 / 4.0 / 1e6)


# ---- Deconvolver.run: one image layout for f, u0 and out -------------------

def test_image_layout_checks():
    """Deconvolver.run hands f, u0 and out to the C call with a single
    (W, H, pitch); layouts that call could not describe are refused before
    it (they would make the library read or write past a buffer)."""
    import torch
    from paper_1304_7211_gb300 import rl
    f = torch.rand(33, 50)
    assert rl.check_images("f32", f) == (50, 33, 50)
    assert rl.check_images(rl.RL_STORAGE_F32, f) == (50, 33, 50)
    # a padded view: the pitch is its row stride, and a new output gets the same
    wide = torch.rand(33, 87)
    view = wide[:, :50]
    assert rl.check_images("f32", view, u0=torch.rand(33, 87)[:, :50]) == (50, 33, 87)
    out = rl._empty_like_layout(view, 33, 50, 87)
    assert out.shape == (33, 50) and out.stride() == (87, 1) and out.dtype == torch.float32
    assert rl.check_images("f32", view, out=out) == (50, 33, 87)
    with pytest.raises(ValueError):  # a packed output for a padded input
        rl.check_images("f32", view, out=torch.empty(33, 50))
    # numpy, contiguous and padded
    a = np.zeros((20, 30), np.float32)
    assert rl.check_images("f32", a) == (30, 20, 30)
    b = np.zeros((20, 64), np.float32)[:, :30]
    assert rl.check_images("f32", b) == (30, 20, 64)
    nb = rl._empty_like_layout(b, 20, 30, 64)
    assert nb.shape == (20, 30) and nb.strides == (256, 4)
    # element type must be the context's storage
    with pytest.raises(TypeError):
        rl.check_images("f32", f.to(torch.bfloat16))
    with pytest.raises(TypeError):
        rl.check_images("bf16", f)
    assert rl.check_images("bf16", f.to(torch.bfloat16)) == (50, 33, 50)
    with pytest.raises(TypeError):
        rl.check_images("f32", a.astype(np.float64))
    with pytest.raises(TypeError):
        rl.check_images("f32", f, u0=f.double())
    # shape, strides, dimensions
    with pytest.raises(ValueError):
        rl.check_images("f32", f.t())                   # columns contiguous
    with pytest.raises(ValueError):
        rl.check_images("f32", torch.rand(1, 50).expand(33, 50))  # rows overlap
    with pytest.raises(ValueError):
        rl.check_images("f32", torch.rand(2, 33, 50))
    with pytest.raises(ValueError):
        rl.check_images("f32", f, u0=torch.rand(33, 49))
    with pytest.raises(ValueError):
        rl.check_images("f32", torch.rand(0, 5))
    with pytest.raises(TypeError):
        rl.check_images("f32", [[1.0]])


def test_image_layout_single_rows_and_columns():
    """Strides of extent-1 dimensions carry no layout: a single row taken out
    of a transposed column, or a single column of a wide image, is accepted
    with the pitch that describes it."""
    import torch
    from paper_1304_7211_gb300 import rl
    row = torch.rand(40, 1).t()                 # shape (1, 40), strides (1, 1)
    assert rl.check_images("f32", row) == (40, 1, 40)
    col = torch.rand(30, 9)[:, 4:5]             # shape (30, 1), strides (9, 1)
    assert rl.check_images("f32", col) == (1, 30, 9)
    assert rl.check_images("f32", np.zeros((30, 9), np.float32)[:, 4:5]) == (1, 30, 9)


def test_buffer_span_checks():
    """The low-level calls take (W, H, pitch) from the caller; a tensor or
    array that ends before the last pixel those describe is refused before
    the C call (it would read or write past the buffer)."""
    import torch
    from paper_1304_7211_gb300 import rl
    f = torch.zeros(10, 16)
    rl._check_span("f", f, 16, 10, 16, 4)                 # exactly the buffer
    rl._check_span("f", f, 12, 10, 16, 4)                 # a pitched sub-image
    rl._check_span("f", f.to(torch.bfloat16), 16, 10, 16, 2)
    with pytest.raises(ValueError):
        rl._check_span("f", f, 16, 11, 16, 4)             # one row too many
    with pytest.raises(ValueError):
        rl._check_span("f", f, 16, 10, 17, 4)             # pitch past the rows
    with pytest.raises(ValueError):                       # bf16 buffer, f32 context
        rl._check_span("f", f.to(torch.bfloat16), 16, 10, 16, 4)
    with pytest.raises(ValueError):                       # a view starting inside the buffer
        rl._check_span("f", f[1:], 16, 10, 16, 4)
    rl._check_span("f", f[1:], 16, 9, 16, 4)
    a = np.zeros((10, 16), np.float32)
    rl._check_span("a", a, 16, 10, 16, 4)
    rl._check_span("a", a[2:, 3:], 13, 8, 16, 4)          # ends exactly at the last element
    with pytest.raises(ValueError):
        rl._check_span("a", a[2:, 3:], 14, 8, 16, 4)
    # left to the library: raw addresses, unknown storage, sizes it rejects
    rl._check_span("p", 12345, 16, 10, 16, 4)
    rl._check_span("f", f, 16, 11, 16, None)
    rl._check_span("f", f, 16, 10, 8, 4)


def test_bench_oracle_checks_fill_the_sub_line_reports():
    """The oracle comparisons of the bench's 256^2 and thinned sub-lines run
    in its CPU-baseline leg: the pending GPU outputs get their relative L-inf
    difference from the oracle written into the reports they came from."""
    import bench
    import oracle
    rng = np.random.default_rng(5)
    f = rng.uniform(10, 200, size=(30, 34))
    taps = np.ones((1, 5)) / 5
    psf = oracle.psf_dense(taps, 2, 0)
    u = oracle.rl(f, psf, 4).u
    rep1 = {"rel_linf_vs_oracle": None}
    pend = [{"kind": "config1", "f": f, "taps": taps, "iters": 4, "u": u * (1 + 1e-3), "report": rep1}]
    g = rng.uniform(10, 200, size=(28, 27))
    rows = [{"k": None}, {"k": None}, {"k": None}]
    plain = oracle.rl(g, oracle.psf_disc(12), 3).u
    thin = oracle.rl(g, oracle.psf_disc(12), 3, threshold=1e-3, update_period=10).u
    rep3 = {"oracle_cpu_s": None, "rows": rows}
    pend.append({"kind": "thinned", "f": g, "iters": 3, "key": "k", "report": rep3,
                 "outputs": [(rows[0], None, plain), (rows[1], 1e-3, thin), (rows[2], None, plain + 1.0)]})
    secs = bench.oracle_checks(pend)
    assert secs >= 0 and rep3["oracle_cpu_s"] is not None
    assert rep1["rel_linf_vs_oracle"] == pytest.approx(1e-3 * np.max(np.abs(u)) / np.max(np.abs(u)), rel=1e-6)
    assert rows[0]["k"] == 0.0 and rows[1]["k"] == 0.0
    assert rows[2]["k"] == pytest.approx(1.0 / np.max(np.abs(plain)))


def test_bench_metrics_match_the_oracle_definitions():
    import bench
    import oracle
    rng = np.random.default_rng(6)
    a, b = rng.normal(size=(9, 11)), rng.normal(size=(9, 11)) + 3
    assert bench.rel_linf(a, b) == pytest.approx(oracle.rel_linf(a, b), rel=1e-12)
    assert bench.psnr_db(a, b) == pytest.approx(oracle.psnr_db(a, b), rel=1e-12)
    assert bench.psnr_db(b, b) == float("inf")
