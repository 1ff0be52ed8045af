"""Variant builds run in child processes: the checked build and the naive-resampling study
build.

The checked build (-DPF_CHECKED): every kernel index that is in range by construction
is tested on the device; a miss would raise the tracker's bounds bit, redirect the access
to element 0 and fail the step with PF_ERR_STATE.  compute-sanitizer is not part of this
project's runs, so this build is how the index arithmetic is exercised on the GPU.

A child process loads the checked library (PF_CHECKED=1) and runs a spread of workloads:
every precision at ragged sizes, the six resampling schemes, a batch, radii 0 and 12 with
template pixels off the frame, one dominant particle (a tile's offspring all from one
ancestor), the bench's 2^20-particle configuration, a served trace and the
allocation-free entry point.  Each must finish without a status error, and its tracks
must equal the library's (the checks change no arithmetic).
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, os, sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import paper_2308_00763_gb300 as pf
from paper_2308_00763_gb300 import synth
pf.lib(build_if_missing=True)
out = {"lib": pf.library_path()}
fr_cache = {}
def frames(v):
    return torch.from_numpy(v.frames).cuda()
tracks = {}
v = synth.make_video(160, 120, 6, 4, noise=5.0, seed=5, v=(1.0, -1.0))
fr = frames(v)
for prec in ("ref64", "f32", "f16", "bf16"):
    for N in (1, 4097, 3 * 4096 + 17):
        for rs in ("systematic", "stratified", "multinomial", "gumbel", "metropolis", "rejection"):
            f = pf.Filter(v.W, v.H, N, 4, prec, init=tuple(v.centres[0]), seed=3, resampler=rs,
                          flags=pf.PF_FLAG_DEBUG_ARRAYS)
            f.run(fr)
            tracks["%s/%d/%s" % (prec, N, rs)] = f.estimates(0, v.T).tolist()
            f.close()
# radii 0 and 12, template pixels off the frame (a disk near the corner)
ve = synth.make_video(70, 45, 4, 3, noise=5.0, seed=13, c0=(2.0, 43.0), v=(0.0, 0.0))
fe = frames(ve)
for r in (0, 12):
    for prec in ("ref64", "f16"):
        f = pf.Filter(ve.W, ve.H, 5000, r, prec, init=tuple(ve.centres[0]), seed=2)
        f.run(fe)
        tracks["edge/%d/%s" % (r, prec)] = f.estimates(0, ve.T).tolist()
        f.close()
# one dominant particle: every offspring of its tile from one ancestor
f = pf.Filter(64, 64, 5000, 2, "f32", init=(32.0, 32.0), seed=2, flags=pf.PF_FLAG_DEBUG_ARRAYS)
st = {"t": 1, "max_l": 0.0, "sum_e": 1.0, "anchor_x": 32.0, "anchor_y": 32.0, "next_anchor_x": 32.0,
      "next_anchor_y": 32.0, "est_x": 32.0, "est_y": 32.0}
x = np.full(5000, 10.0); y = np.full(5000, 10.0); L = np.full(5000, -500.0)
x[3777], y[3777], L[3777] = 40.25, 20.5, 0.0
st.update(x=x, y=y, L=L)
f.set_state(st)
f.step(np.full((64, 64), 100, np.uint8))
assert np.all(f.debug(0) == 3777)
f.close()
# a batch of uneven trackers
vids = [synth.make_video(96, 96, 5, 3, noise=5.0, seed=20 + i, v=(1.0, -1.0)) for i in range(3)]
cfgs = [pf.make_config(w.W, w.H, n, w.radius, "f16", init=tuple(w.centres[0]), seed=30 + i, tracker_id=i,
                       resampler=rs)
        for i, (w, n, rs) in enumerate(zip(vids, (1000, 3 * 4096 + 7, 17), ("systematic", "multinomial", "stratified")))]
b = pf.Batch(cfgs)
bf = [frames(w) for w in vids]
for t in range(5):
    b.step([g[t] for g in bf])
tracks["batch"] = [b.estimates(t).tolist() for t in range(5)]
b.close()
# the bench's configuration, a few frames
vb = synth.make_video(512, 512, 4, 5, noise=5.0, seed=1)
f = pf.Filter(512, 512, 1 << 20, 5, "f16", init=tuple(vb.centres[0]), seed=1)
f.run(frames(vb))
tracks["bench"] = f.estimates(0, 4).tolist()
f.close()
# a served trace
s = pf.Server(1 << 28, max_streams=4, queue_depth=2)
sid = s.open(pf.make_config(v.W, v.H, 9000, 4, "f16", init=tuple(v.centres[0]), seed=4, est_capacity=16))
for t in range(v.T):
    assert s.submit(sid, fr[t])
    s.drain()
tracks["served"] = [list(s.result(sid, t)) for t in range(v.T)]
s.close()
# the allocation-free entry point, two frames
N = 3 * 4096 + 11
cfg = pf.make_config(v.W, v.H, N, 4, "f32", init=tuple(v.centres[0]), seed=77)
hdr = pf.PfStateHeader(magic=0x31534650, precision=cfg.precision, num_particles=N, t=0)
bufs = [[torch.zeros(N, dtype=torch.float32, device="cuda") for _ in range(3)] for _ in range(2)]
ptr = [[q.data_ptr() for q in slot] for slot in bufs]
o0 = pf.pf_step_frame_noalloc(cfg, hdr, 0, 0, 0, fr[0].data_ptr(), fr.stride(1), *ptr[0])
o1 = pf.pf_step_frame_noalloc(cfg, o0, *ptr[0], fr[1].data_ptr(), fr.stride(1), *ptr[1])
tracks["noalloc"] = [o0.est_x, o0.est_y, o1.est_x, o1.est_y]
torch.cuda.synchronize()
out["tracks"] = tracks
print(json.dumps(out))
'''


def _run(checked):
    env = dict(os.environ)
    env.pop("PF_STEP_THREADS", None)
    env.pop("PF_NAIVE", None)
    if checked:
        env["PF_CHECKED"] = "1"
    else:
        env.pop("PF_CHECKED", None)
    p = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, (p.stdout[-2000:], p.stderr[-4000:])
    import json
    return json.loads(p.stdout.strip().splitlines()[-1])


def test_checked_build_runs_every_workload_clean():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    checked = _run(True)
    assert "/checked/" in checked["lib"]
    plain = _run(False)
    assert "/checked/" not in plain["lib"]
    assert checked["tracks"] == plain["tracks"]


NAIVE_CHILD = r'''
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import oracle
import paper_2308_00763_gb300 as pf
from paper_2308_00763_gb300 import synth
pf.lib(build_if_missing=True)
v = synth.make_video(160, 120, 5, 4, noise=8.0, seed=9, v=(1.0, -1.0))
fr = torch.from_numpy(v.frames).cuda()
res = {"lib": pf.library_path(), "cases": []}
for prec in ("ref64", "f32", "f16", "bf16"):
    for N in (3, 4097, 3 * 4096 + 17):
        f = pf.Filter(v.W, v.H, N, 4, prec, init=tuple(v.centres[0]), seed=6, sigma=(2.0, 2.0),
                      flags=pf.PF_FLAG_DEBUG_ARRAYS)
        f.run(fr)
        anc = f.debug(0).astype(np.int64)
        C = f.debug(1).astype(np.float64)
        a_o = oracle.resample(C, oracle.resample_u0(6, v.T - 2), "f64" if prec == "ref64" else "f32", divide=True)
        res["cases"].append([prec, N, bool(np.array_equal(anc, a_o)), bool(np.all(np.diff(C) >= 0) and C[-1] == 1.0)])
        f.close()
# the first frame's likelihoods (no resampling yet) must not depend on how pixels enter half
f = pf.Filter(v.W, v.H, 5000, 4, "f16", init=tuple(v.centres[0]), seed=6)
f.step(fr[0])
res["L0"] = f.get_state()["L"].astype(np.float64).tolist()
f.close()
print(json.dumps(res))
'''


def test_naive_resampling_study_build_is_exact_for_its_own_arithmetic():
    """The naive study build (-DPF_NAIVE_RESAMPLE, PF_NAIVE=1) divides by S and N per
    element: its ancestors equal the oracle's systematic resampling with points (j + u0)/N
    on the CDF the step computed, in every precision; and its per-pixel integer-to-half
    conversion leaves the likelihoods unchanged."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import json
    env = dict(os.environ)
    env.pop("PF_STEP_THREADS", None)
    env.pop("PF_CHECKED", None)
    out = {}
    for naive in (True, False):
        if naive:
            env["PF_NAIVE"] = "1"
        else:
            env.pop("PF_NAIVE", None)
        p = subprocess.run([sys.executable, "-c", NAIVE_CHILD, ROOT], env=env, capture_output=True, text=True,
                           timeout=900)
        assert p.returncode == 0, (p.stdout[-2000:], p.stderr[-4000:])
        out[naive] = json.loads(p.stdout.strip().splitlines()[-1])
    assert "/naive/" in out[True]["lib"] and "/naive/" not in out[False]["lib"]
    for prec, N, exact, monotone in out[True]["cases"]:
        assert exact and monotone, (prec, N)
    assert out[True]["L0"] == out[False]["L0"]


TPB_CHILD = r'''
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import oracle
import paper_2308_00763_gb300 as pf
from paper_2308_00763_gb300 import synth
pf.lib(build_if_missing=True)
threads = int(sys.argv[2])
tile = 8 * threads
v = synth.make_video(160, 120, 5, 4, noise=8.0, seed=9, v=(1.0, -1.0))
fr = torch.from_numpy(v.frames).cuda()
res = {"lib": pf.library_path(), "cases": []}
precs = ("f32", "f16", "bf16") if threads == 1024 else ("ref64", "f32", "f16", "bf16")
for prec in precs:
    for N in (3, tile - 1, tile + 1, 3 * tile + 17):
        f = pf.Filter(v.W, v.H, N, 4, prec, init=tuple(v.centres[0]), seed=6, sigma=(2.0, 2.0),
                      flags=pf.PF_FLAG_DEBUG_ARRAYS)
        f.run(fr)
        est = f.estimates(0, v.T)
        anc = f.debug(0).astype(np.int64)
        C = f.debug(1).astype(np.float64)
        a_o = oracle.resample(C, oracle.resample_u0(6, v.T - 2), "f64" if prec == "ref64" else "f32")
        est_o, _, _ = oracle.track(v.frames, N, 4, init=tuple(v.centres[0]), seed=6, sigma=(2.0, 2.0))
        if prec == "ref64":
            err = float(np.abs(est - est_o).max()); ok = err <= 1e-9
        elif prec == "f32":
            err = float(np.abs(est - est_o).max()); ok = err <= 1e-3
        else:
            err = float(np.sqrt(np.mean(np.sum((est - est_o) ** 2, axis=1)))); ok = err <= 0.5
        res["cases"].append([prec, N, bool(np.array_equal(anc, a_o)),
                             bool(np.all(np.diff(C) >= 0) and C[-1] == 1.0), ok, err])
        f.close()
print(json.dumps(res))
'''


@pytest.mark.parametrize("threads", [128, 256, 1024])
def test_thread_block_study_builds_keep_the_method(threads):
    """The thread-block study builds (threads per CTA 128, 256 and 1024; the paper varies
    threads per block from 32 to 1024 in its Sec. V): in each, at ragged sizes around its
    own tile (8 elements a thread), the ancestors equal the oracle's systematic resampling
    of the CDF the step computed bit for bit, the CDF is monotone and ends at 1, and the
    track matches the oracle's at the stated tolerance of its precision."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import json
    from paper_2308_00763_gb300 import build as pbuild
    pbuild.build(threads=threads)
    env = dict(os.environ)
    env.pop("PF_CHECKED", None)
    env.pop("PF_NAIVE", None)
    env["PF_STEP_THREADS"] = str(threads)
    p = subprocess.run([sys.executable, "-c", TPB_CHILD, ROOT, str(threads)], env=env, capture_output=True,
                       text=True, timeout=900)
    assert p.returncode == 0, (p.stdout[-2000:], p.stderr[-4000:])
    out = json.loads(p.stdout.strip().splitlines()[-1])
    assert ("/t%d/" % threads) in out["lib"]
    for prec, N, exact, monotone, ok, err in out["cases"]:
        assert exact and monotone and ok, (threads, prec, N, err)
