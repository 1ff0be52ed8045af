"""Autotuned launch shapes (pf_autotune, PF_FLAG_TUNED).

A shape changes the tile (how the FP scan is partitioned), the likelihood window policy
and the CTAs per SM, never a formula.  The checks: the tuner returns and caches a valid
shape; under every shape the step's ancestors are exactly those of the CDF it computed
and the track stays within tolerance of the default shape's; equal configurations tile
alike alone and in a batch.
"""
import numpy as np
import pytest

import oracle
from paper_2308_00763_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_00763_gb300 as m
    m.lib(build_if_missing=True)
    oracle.build()
    yield m
    m.pf_tuning_clear()


def _vid(T=6, seed=91):
    import torch
    v = synth.make_video(160, 120, T, 4, noise=5.0, seed=seed, v=(1.0, -1.0))
    return v, torch.from_numpy(v.frames).cuda()


def test_autotune_caches_a_valid_shape(pf):
    pf.pf_tuning_clear()
    v, fr = _vid()
    cfg = pf.make_config(v.W, v.H, 50000, v.radius, "f16", init=tuple(v.centres[0]), seed=5)
    t, us = pf.autotune(cfg, fr, copies=2)
    assert us > 0
    assert t["tile"] in (0, 1024, 2048, 3072, 4096) and t["window"] in (0, 1, 2) and t["ctas_per_sm"] in (0, 1)
    c = pf.pf_tuning_lookup(cfg)
    assert c is not None and c.as_dict() == t


SHAPES = [(1024, 1, 0), (2048, 2, 1), (3072, 0, 1), (4096, 1, 0)]


@pytest.mark.parametrize("prec", ["ref64", "f32", "f16"])
@pytest.mark.parametrize("shape", SHAPES)
def test_every_shape_keeps_the_method(pf, prec, shape):
    v, fr = _vid(T=8)
    N = 10 * 1024 + 37
    kw = dict(init=tuple(v.centres[0]), seed=13)
    base = pf.Filter(v.W, v.H, N, v.radius, prec, **kw)
    base.run(fr)
    want = base.estimates(0, v.T)
    base.close()

    cfg = pf.make_config(v.W, v.H, N, v.radius, prec, **kw)
    pf.pf_tuning_store(cfg, *shape)
    f = pf.Filter(v.W, v.H, N, v.radius, prec, flags=pf.PF_FLAG_TUNED | pf.PF_FLAG_DEBUG_ARRAYS, **kw)
    f.run(fr[:v.T - 1])
    f.step(fr[v.T - 1])
    # ancestors: exactly the systematic resampling of the CDF this step computed
    anc = f.debug(0).astype(np.int64)
    C = f.debug(1).astype(np.float64)
    assert np.all(np.diff(C) >= 0) and C[-1] == 1.0
    a_o = oracle.resample(C, oracle.resample_u0(13, v.T - 2), "f64" if prec == "ref64" else "f32")
    assert np.array_equal(anc, a_o)
    got = f.estimates(0, v.T)
    f.close()
    tol = {"ref64": 1e-9, "f32": 1e-3, "f16": 0.05}[prec]
    assert np.abs(got - want).max() <= tol, (prec, shape)
    pf.pf_tuning_clear()


def test_tuned_batch_equals_tuned_singles(pf):
    pf.pf_tuning_clear()
    vids = [_vid(T=5, seed=95), _vid(T=5, seed=96)]
    Ns = [9000, 70000]
    cfgs = [pf.make_config(v.W, v.H, n, v.radius, "f16", init=tuple(v.centres[0]), seed=40 + i, tracker_id=i,
                           flags=pf.PF_FLAG_TUNED) for i, ((v, _), n) in enumerate(zip(vids, Ns))]
    pf.pf_tuning_store(cfgs[1], 2048, 2, 1)          # only the second tracker's bucket is tuned
    b = pf.Batch(cfgs)
    for t in range(5):
        b.step([vids[0][1][t], vids[1][1][t]])
    got = np.stack([b.estimates(t) for t in range(5)], axis=1)
    b.close()
    for i, ((v, fr), n) in enumerate(zip(vids, Ns)):
        f = pf.Filter(v.W, v.H, n, v.radius, "f16", init=tuple(v.centres[0]), seed=40 + i, tracker_id=i,
                      flags=pf.PF_FLAG_TUNED)
        f.run(fr)
        assert np.array_equal(f.estimates(0, 5), got[i])
        f.close()
    pf.pf_tuning_clear()


def test_autotune_batch_caches_every_bucket(pf):
    pf.pf_tuning_clear()
    vids = [_vid(T=4, seed=97), _vid(T=4, seed=98), _vid(T=4, seed=99)]
    Ns = [3000, 40000, 300000]
    cfgs = [pf.make_config(v.W, v.H, n, v.radius, "f32", init=tuple(v.centres[0]), seed=60 + i, tracker_id=i)
            for i, ((v, _), n) in enumerate(zip(vids, Ns))]
    t, us = pf.autotune_batch(cfgs, [fr for _, fr in vids])
    assert us > 0 and t["tile"] in (0, 1024, 2048, 3072, 4096)
    for c in cfgs:
        got = pf.pf_tuning_lookup(c)
        assert got is not None and got.as_dict() == t
    pf.pf_tuning_clear()
