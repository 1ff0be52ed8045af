"""The C-ABI library builds, loads on a machine without a GPU, and exports every entry
point that include/pf.h declares (no compute call is made here)."""
import ctypes
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "pf.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pf_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2308_00763_gb300 import build
    return build.build()


def test_header_compiles_as_c():
    out = os.path.join(ROOT, "paper_2308_00763_gb300", "_build", "hdr_check.o")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-x", "c", "-c", "-o", out, "-"],
                   input=b'#include "pf.h"\nint pf_check_sizes(void){return (int)sizeof(pf_config);}\n',
                   cwd=os.path.join(ROOT, "include"), check=True)


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    declared = _declared()
    assert "pf_create" in declared and "pf_step_frame" in declared and "pf_estimate" in declared
    missing = [name for name in declared if not hasattr(lib, name)]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    import paper_2308_00763_gb300 as pf
    for name in _declared():
        assert name in pf.EXPORTED and callable(getattr(pf, name)), name
    assert pf.pf_status_string(pf.PF_ERR_TIMEOUT) == "device wait timed out"


def test_struct_layouts_match_c(libpath):
    import paper_2308_00763_gb300 as pf
    src = ('#include <stdio.h>\n#include <stddef.h>\n#include "pf.h"\nint main(void){printf("%zu %zu %zu %zu %zu",'
           ' sizeof(pf_config), offsetof(pf_config, seed), offsetof(pf_config, est_capacity),'
           ' sizeof(pf_state_header), offsetof(pf_state_header, est_y)); return 0;}\n')
    exe = os.path.join(ROOT, "paper_2308_00763_gb300", "_build", "layout_check")
    subprocess.run(["gcc", "-x", "c", "-o", exe, "-", "-I", os.path.join(ROOT, "include")],
                   input=src.encode(), check=True)
    got = list(map(int, subprocess.run([exe], capture_output=True, check=True).stdout.split()))
    want = [ctypes.sizeof(pf.PfConfig), pf.PfConfig.seed.offset, pf.PfConfig.est_capacity.offset,
            ctypes.sizeof(pf.PfStateHeader), pf.PfStateHeader.est_y.offset]
    assert got == want


def test_invalid_configs_rejected_without_gpu(libpath):
    """Argument validation happens on the host before any CUDA call."""
    import paper_2308_00763_gb300 as pf
    bad = [dict(num_particles=0), dict(disk_radius=-1), dict(disk_radius=65), dict(width=0),
           dict(precision=7), dict(sigma=(-1.0, 1.0)), dict(init=(float("nan"), 0.0)),
           dict(resampler=6), dict(resampler=-1),
           # stratified points in FP32 are ordered only while (float)j is exact
           dict(resampler="stratified", num_particles=(1 << 24) + 1),
           # Gumbel-max draws N^2 variates a frame
           dict(resampler="gumbel", num_particles=(1 << 16) + 1),
           dict(resampler="gumbel", num_particles=(1 << 16) + 1, precision="ref64"),
           # Metropolis: the offspring index lives in the draw tag; chain length in [0, 4096]
           dict(resampler="metropolis", num_particles=(1 << 24) + 1),
           dict(resampler="metropolis", resampler_steps=-1),
           dict(resampler="metropolis", resampler_steps=4097),
           dict(resampler="systematic", resampler_steps=8),
           # rejection: at most 65536 tries per offspring
           dict(resampler="rejection", resampler_steps=65537),
           dict(resampler="rejection", num_particles=(1 << 24) + 1)]
    for b in bad:
        kw = dict(width=64, height=64, num_particles=100, disk_radius=3, precision="f32")
        kw.update({k: v for k, v in b.items() if k in kw})
        extra = {k: v for k, v in b.items() if k not in kw}
        cfg = pf.make_config(kw["width"], kw["height"], kw["num_particles"], kw["disk_radius"],
                             kw["precision"], **extra)
        h = ctypes.c_void_p()
        rc = pf.lib().pf_create(ctypes.byref(cfg), None, ctypes.byref(h))
        assert rc == pf.PF_ERR_ARG, b
        assert not h.value
    assert pf.lib().pf_create(None, None, None) == pf.PF_ERR_ARG
    assert pf.lib().pf_destroy(None) == pf.PF_OK


def test_server_stream_bytes_without_gpu(libpath):
    """The arena bytes a serving stream takes: both ping-pong slots of x, y, L at the
    precision's width, plus the frame queue when it is fed from host memory."""
    import paper_2308_00763_gb300 as pf
    for prec, width in (("ref64", 8), ("f32", 4), ("f16", 2), ("bf16", 2)):
        for N in (1000, 123457, 1 << 20):
            c = pf.make_config(640, 480, N, 5, prec)
            dev = pf.pf_server_stream_bytes(c, 0, 4)
            host = pf.pf_server_stream_bytes(c, 1, 4)
            assert dev >= 6 * N * width and dev < 6 * N * width + 64 * 1024 + N // 4
            assert host - dev == ((640 + 15) // 16 * 16) * 480 * 4
            assert pf.pf_server_stream_bytes(c, 0, 1) == dev
    with pytest.raises(pf.PfError):
        pf.pf_server_stream_bytes(pf.make_config(0, 480, 10, 5, "f16"), 0, 4)
    with pytest.raises(pf.PfError):    # the server launches one kernel per tick: no multinomial streams
        pf.pf_server_stream_bytes(pf.make_config(640, 480, 10, 5, "f16", resampler="multinomial"), 0, 4)
    with pytest.raises(pf.PfError):    # nor Gumbel-max or Metropolis streams (ancestor and pull kernels)
        pf.pf_server_stream_bytes(pf.make_config(640, 480, 10, 5, "f16", resampler="gumbel"), 0, 4)
    for scheme in ("metropolis", "rejection"):
        with pytest.raises(pf.PfError):
            pf.pf_server_stream_bytes(pf.make_config(640, 480, 10, 5, "f16", resampler=scheme), 0, 4)


def test_tuning_cache_without_gpu(libpath):
    """The launch-shape cache is host state keyed by the shape bucket (precision,
    floor(log2 N), larger sigma in quarter pixels, radius, floor(log2 W*H), SM count);
    invalid shapes are refused."""
    import paper_2308_00763_gb300 as pf
    pf.pf_tuning_clear()
    a = pf.make_config(512, 512, 1 << 20, 5, "f16", sigma=(1.0, 1.0))
    same_bucket = pf.make_config(512, 600, (1 << 21) - 1, 5, "f16", sigma=(1.1, 0.9))
    others = [pf.make_config(512, 512, 1 << 20, 5, "f32", sigma=(1.0, 1.0)),     # precision
              pf.make_config(512, 512, 1 << 21, 5, "f16", sigma=(1.0, 1.0)),     # N bucket
              pf.make_config(512, 512, 1 << 20, 5, "f16", sigma=(2.0, 1.0)),     # sigma
              pf.make_config(512, 512, 1 << 20, 9, "f16", sigma=(1.0, 1.0)),     # radius
              pf.make_config(1024, 1024, 1 << 20, 5, "f16", sigma=(1.0, 1.0))]   # frame size
    assert pf.pf_tuning_lookup(a) is None
    pf.pf_tuning_store(a, 2048, 1, 1)
    t = pf.pf_tuning_lookup(same_bucket)
    assert t is not None and (t.tile, t.window, t.ctas_per_sm) == (2048, 1, 1)
    for o in others:
        assert pf.pf_tuning_lookup(o) is None
    for bad in ((1000, 0, 0), (8192, 0, 0), (2048, 3, 0), (2048, 0, -1)):
        with pytest.raises(pf.PfError):
            pf.pf_tuning_store(a, *bad)
    pf.pf_tuning_clear()
    assert pf.pf_tuning_lookup(a) is None


def test_thread_block_study_builds_are_separate(monkeypatch):
    """The thread-block study builds (-DPF_STEP_THREADS) live beside the library and are
    selected only through PF_STEP_THREADS; 512 threads is the library itself."""
    from paper_2308_00763_gb300 import binding, build
    assert build.lib_path(None) == build.LIB == build.lib_path(512)
    paths = {build.lib_path(t) for t in build.STUDY_THREADS}
    assert len(paths) == len(build.STUDY_THREADS)
    monkeypatch.setenv("PF_STEP_THREADS", "256")
    assert binding.library_path() == build.lib_path(256) != build.LIB
    monkeypatch.delenv("PF_STEP_THREADS")
    assert binding.library_path() == build.LIB
    with pytest.raises(ValueError):
        build.build(threads=96)


def test_checked_build_is_separate(monkeypatch):
    """The checked build (-DPF_CHECKED) lives beside the library, selected by PF_CHECKED."""
    from paper_2308_00763_gb300 import binding, build
    assert build.lib_path(checked=True) not in (build.LIB,) + tuple(build.lib_path(t) for t in build.STUDY_THREADS)
    monkeypatch.setenv("PF_CHECKED", "1")
    assert binding.library_path() == build.lib_path(checked=True)
    monkeypatch.setenv("PF_CHECKED", "0")
    assert binding.library_path() == build.LIB
    with pytest.raises(ValueError):
        build.build(threads=256, checked=True)


def test_naive_study_build_is_separate(monkeypatch):
    from paper_2308_00763_gb300 import binding, build
    assert build.lib_path(naive=True) not in (build.LIB, build.lib_path(checked=True))
    monkeypatch.setenv("PF_NAIVE", "1")
    assert binding.library_path() == build.lib_path(naive=True)
    with pytest.raises(ValueError):
        build.build(naive=True, checked=True)
