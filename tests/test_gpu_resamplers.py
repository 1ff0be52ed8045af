"""Alternative resampling schemes on the GPU (pf_config.resampler).

Stratified: the fused step with one independent offset per stratum, u_j = (j + v_j) / N
(Sec. III names stratified resampling beside the paper's systematic scheme of Sec. IV).
Multinomial: the step kernel writes the CDF, the pull kernel gives offspring j the first
particle whose CDF value reaches an independent uniform v_j (Sec. IV's categorical draw).
Gumbel-max: the argmax kernel gives offspring j the particle maximising L_k + g_jk (the
log-domain form of the same draw that Sec. IV weighs), the pull kernel gathers them.
Metropolis: offspring j's B-step chain on exp(L) (the reduction-free scheme Sec. III cites).
Rejection: offspring j's first candidate (j, then uniform proposals) passing u <= w/w_max.
The checks: the ancestors are exactly the oracle's resampling of the CDF the step computed,
with the draws from the oracle's own Philox; the REF64 track equals the oracle's FP64 track
of the same scheme within 1e-9 px; stratified offspring counts stay within two strata of
N w_k; the option takes effect; the schemes share a batch, each tracker equal to its own
single run; the bench's launch configuration (2^20 particles) resamples exactly.
Gumbel-max, Metropolis and rejection ancestors equal the oracle's decisions in the
kernel's precision up to near ties (FP32 logs may differ in the last bit between the two
sides).
"""
import numpy as np
import pytest

import oracle
from paper_2308_00763_gb300 import synth

pytestmark = pytest.mark.gpu

TILE = 4096  # particles per tile of the step kernel


@pytest.fixture(scope="module")
def pf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_00763_gb300 as m
    m.lib(build_if_missing=True)
    oracle.build()
    return m


def _frames(v):
    import torch
    return torch.from_numpy(v.frames).cuda()


def _last_step(pf, v, N, prec, seed, *, resampler="stratified", tracker=0, sigma=(1.0, 1.0), T=None):
    """Run T frames with debug arrays; the ancestors and CDF of the last step."""
    T = v.T if T is None else T
    f = pf.Filter(v.W, v.H, N, v.radius, prec, init=tuple(v.centres[0]), seed=seed, tracker_id=tracker,
                  sigma=sigma, flags=pf.PF_FLAG_DEBUG_ARRAYS, resampler=resampler)
    fr = _frames(v)
    f.run(fr[:T])
    anc = f.debug(0).astype(np.int64)
    C = f.debug(1).astype(np.float64)
    f.close()
    return anc, C


@pytest.mark.parametrize("prec", ["ref64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("N", [1, 3, TILE + 1, 3 * TILE + 17])
def test_stratified_ancestors_exact(pf, prec, N):
    v = synth.make_video(128, 128, 4, 5, noise=5.0, seed=41)
    anc, C = _last_step(pf, v, N, prec, 17, tracker=2)
    assert np.all(np.diff(C) >= 0) and C[-1] == 1.0
    offs = oracle.stratified_offsets(17, v.T - 2, N, 2)
    a_o = oracle.resample_stratified(C, offs, "f64" if prec == "ref64" else "f32")
    assert np.array_equal(anc, a_o)


def test_stratified_ref64_track_within_1e9(pf):
    v = synth.make_video(128, 128, 10, 5, noise=5.0, seed=1)
    for N in (1000, 3 * TILE + 17):
        est_o, M_o, _ = oracle.track(v.frames, N, 5, init=tuple(v.centres[0]), seed=1, resampler="stratified")
        f = pf.Filter(v.W, v.H, N, 5, "ref64", init=tuple(v.centres[0]), seed=1, resampler="stratified")
        f.run(_frames(v))
        est, ms = f.estimates(0, v.T, with_stats=True)
        f.close()
        assert np.abs(est - est_o).max() <= 1e-9, N
        assert np.array_equal(ms[:, 0], M_o)


@pytest.mark.parametrize("prec", ["ref64", "f32", "f16"])
def test_stratified_counts_within_two_strata(pf, prec):
    v = synth.make_video(160, 120, 4, 4, noise=15.0, seed=33)
    N = 5 * TILE + 123
    anc, C = _last_step(pf, v, N, prec, 8, sigma=(3.0, 3.0))
    w = np.diff(np.concatenate([[0.0], C]))
    cnt = np.bincount(anc, minlength=N)
    slack = 1e-9 if prec == "ref64" else N * 2.0 ** -21
    assert cnt.sum() == N and np.all(np.diff(anc) >= 0)
    assert np.all(np.abs(cnt - N * w) < 2.0 + slack)


def test_stratified_differs_from_systematic(pf):
    v = synth.make_video(128, 128, 4, 5, noise=15.0, seed=42)
    N = 2 * TILE + 9
    a_s, C_s = _last_step(pf, v, N, "f32", 5, resampler="stratified", sigma=(2.0, 2.0))
    a_y, C_y = _last_step(pf, v, N, "f32", 5, resampler="systematic", sigma=(2.0, 2.0))
    assert not np.array_equal(a_s, a_y)
    # the systematic run is the oracle's systematic resampling of its own CDF
    assert np.array_equal(a_y, oracle.resample(C_y, oracle.resample_u0(5, v.T - 2), "f32"))


def test_mixed_resamplers_batch_equals_singles(pf):
    vids = [synth.make_video(96, 96, 5, 3, noise=5.0, seed=50 + i, v=(1.0, -1.0)) for i in range(3)]
    Ns = [3000, 2 * TILE + 5, 777]
    rs = ["stratified", "systematic", "stratified"]
    for prec in ("ref64", "f16"):
        cfgs = [pf.make_config(v.W, v.H, n, v.radius, prec, init=tuple(v.centres[0]), seed=60 + i,
                               tracker_id=i, resampler=r) for i, (v, n, r) in enumerate(zip(vids, Ns, rs))]
        b = pf.Batch(cfgs)
        fr = [_frames(v) for v in vids]
        for t in range(5):
            b.step([f[t] for f in fr])
        got = np.stack([b.estimates(t) for t in range(5)], axis=1)
        b.close()
        for i, (v, n, r) in enumerate(zip(vids, Ns, rs)):
            s = pf.Filter(v.W, v.H, n, v.radius, prec, init=tuple(v.centres[0]), seed=60 + i, tracker_id=i,
                          resampler=r)
            s.run(fr[i])
            assert np.array_equal(s.estimates(0, 5), got[i]), (prec, i)
            s.close()


@pytest.mark.parametrize("prec", ["ref64", "f16"])
def test_stratified_full_size_ancestors_exact(pf, prec):
    """512x512, r = 5, N = 2^20 (the bench's launch configuration, balanced tiles)."""
    v = synth.make_video(512, 512, 3, 5, noise=5.0, seed=1)
    N = 1 << 20
    anc, C = _last_step(pf, v, N, prec, 1)
    offs = oracle.stratified_offsets(1, v.T - 2, N, 0)
    assert np.array_equal(anc, oracle.resample_stratified(C, offs, "f64" if prec == "ref64" else "f32"))


# ----------------------------------------------------------------------------- multinomial
@pytest.mark.parametrize("prec", ["ref64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("N", [1, 3, TILE + 1, 3 * TILE + 17])
def test_multinomial_ancestors_exact(pf, prec, N):
    v = synth.make_video(128, 128, 4, 5, noise=5.0, seed=43)
    anc, C = _last_step(pf, v, N, prec, 19, tracker=5, resampler="multinomial")
    assert np.all(np.diff(C) >= 0) and C[-1] == 1.0
    draws = oracle.stratified_offsets(19, v.T - 2, N, 5)
    assert np.array_equal(anc, oracle.resample_multinomial(C, draws, "f64" if prec == "ref64" else "f32"))


def test_multinomial_ref64_track_within_1e9(pf):
    v = synth.make_video(128, 128, 10, 5, noise=5.0, seed=1)
    for N in (1000, 3 * TILE + 17):
        est_o, M_o, _ = oracle.track(v.frames, N, 5, init=tuple(v.centres[0]), seed=1, resampler="multinomial")
        f = pf.Filter(v.W, v.H, N, 5, "ref64", init=tuple(v.centres[0]), seed=1, resampler="multinomial")
        f.run(_frames(v))
        est, ms = f.estimates(0, v.T, with_stats=True)
        f.close()
        assert np.abs(est - est_o).max() <= 1e-9, N
        assert np.array_equal(ms[:, 0], M_o)


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_multinomial_tracks_the_truth_and_steps_equal_runs(pf, prec):
    """Free-running multinomial tracks stay within half a pixel of the oracle's FP64
    multinomial track (RMSE); single steps equal a graph-replayed run bit for bit."""
    v = synth.make_video(128, 128, 10, 5, noise=5.0, seed=1)
    est_o, _, _ = oracle.track(v.frames, 1000, 5, init=tuple(v.centres[0]), seed=1, resampler="multinomial")
    fr = _frames(v)
    a = pf.Filter(v.W, v.H, 1000, 5, prec, init=tuple(v.centres[0]), seed=1, resampler="multinomial")
    a.run(fr)
    b = pf.Filter(v.W, v.H, 1000, 5, prec, init=tuple(v.centres[0]), seed=1, resampler="multinomial")
    for t in range(v.T):
        b.step(fr[t])
    ea, eb = a.estimates(0, v.T), b.estimates(0, v.T)
    a.close()
    b.close()
    assert np.array_equal(ea, eb)
    assert np.sqrt(np.mean(np.sum((ea - est_o) ** 2, axis=1))) <= 0.5


def test_all_schemes_in_one_batch_equal_singles(pf):
    vids = [synth.make_video(96, 96, 5, 3, noise=5.0, seed=70 + i, v=(1.0, -1.0)) for i in range(4)]
    Ns = [3000, 2 * TILE + 5, 777, 5000]
    rs = ["multinomial", "systematic", "stratified", "multinomial"]
    for prec in ("ref64", "f32", "f16"):
        cfgs = [pf.make_config(v.W, v.H, n, v.radius, prec, init=tuple(v.centres[0]), seed=80 + i,
                               tracker_id=i, resampler=r) for i, (v, n, r) in enumerate(zip(vids, Ns, rs))]
        b = pf.Batch(cfgs)
        fr = [_frames(v) for v in vids]
        for t in range(5):
            b.step([f[t] for f in fr])
        got = np.stack([b.estimates(t) for t in range(5)], axis=1)
        b.close()
        for i, (v, n, r) in enumerate(zip(vids, Ns, rs)):
            s = pf.Filter(v.W, v.H, n, v.radius, prec, init=tuple(v.centres[0]), seed=80 + i, tracker_id=i,
                          resampler=r)
            s.run(fr[i])
            assert np.array_equal(s.estimates(0, 5), got[i]), (prec, i, r)
            s.close()


@pytest.mark.parametrize("prec", ["ref64", "f16"])
def test_multinomial_full_size_ancestors_exact(pf, prec):
    v = synth.make_video(512, 512, 3, 5, noise=5.0, seed=1)
    N = 1 << 20
    anc, C = _last_step(pf, v, N, prec, 1, resampler="multinomial")
    draws = oracle.stratified_offsets(1, v.T - 2, N, 0)
    assert np.array_equal(anc, oracle.resample_multinomial(C, draws, "f64" if prec == "ref64" else "f32"))


@pytest.mark.parametrize("scheme,N", [("stratified", 1 << 24), ("multinomial", 1 << 22)])
def test_alternative_schemes_at_large_sizes(pf, scheme, N):
    """1024x1024, r = 10: stratified at N = 2^24 (the sweep's largest configuration, and in
    FP32 the largest N whose points stay ordered), multinomial at 2^22 (the oracle's N
    binary searches stay within seconds): every ancestor exact."""
    v = synth.make_video(1024, 1024, 3, 10, noise=15.0, seed=3)
    anc, C = _last_step(pf, v, N, "f16", 3, resampler=scheme)
    draws = oracle.stratified_offsets(3, v.T - 2, N, 0)
    fn = oracle.resample_stratified if scheme == "stratified" else oracle.resample_multinomial
    assert np.array_equal(anc, fn(C, draws, "f32"))


# ----------------------------------------------------------------------------- Gumbel-max
def _gumbel_step(pf, v, N, prec, seed, *, tracker=0, T=None):
    """Run T - 1 frames, read the state's log weights, run frame T - 1 with debug arrays:
    (ancestors of that step, the log weights they were drawn from, the draws' frame)."""
    T = v.T if T is None else T
    f = pf.Filter(v.W, v.H, N, v.radius, prec, init=tuple(v.centres[0]), seed=seed, tracker_id=tracker,
                  flags=pf.PF_FLAG_DEBUG_ARRAYS, resampler="gumbel")
    fr = _frames(v)
    f.run(fr[:T - 1])
    st = f.get_state()
    f.step(fr[T - 1])
    anc = f.debug(0).astype(np.int64)
    f.close()
    return anc, st["L"].astype(np.float64), int(st["t"]) - 1


def _near_tie(L, seed, t, tracker, j, k_want, k_got, prec):
    """Offspring j's values at the two indices are within the decision precision's
    rounding (FP64 variates, the kernel's FP32 or FP64 sum)."""
    g = oracle.gumbel_variates(seed, t, int(j), L.size, tracker)
    v = L + g
    tol = (1e-12 if prec == "ref64" else 1e-5) * max(1.0, abs(v[k_want]))
    return abs(v[k_want] - v[k_got]) <= tol


def _check_gumbel(L, seed, t, tracker, anc, prec):
    """Ancestors equal the oracle's Gumbel-max decisions in the kernel's precision; where
    they differ (FP32 logs of the two sides may differ in the last bit) the two values
    are a near tie, and such offspring are rare."""
    want = oracle.resample_gumbel(L, seed, t, tracker, "f64" if prec == "ref64" else "f32")
    bad = np.nonzero(anc != want)[0]
    assert np.all((anc >= 0) & (anc < L.size))
    assert bad.size <= max(1, L.size // 1000), bad[:10]
    for j in bad:
        assert _near_tie(L, seed, t, tracker, j, want[j], anc[j], prec), (j, want[j], anc[j])


@pytest.mark.parametrize("prec", ["ref64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("N", [1, 3, 1000, TILE + 1])
def test_gumbel_ancestors_exact(pf, prec, N):
    v = synth.make_video(128, 128, 4, 5, noise=5.0, seed=47)
    anc, L, t = _gumbel_step(pf, v, N, prec, 23, tracker=6)
    _check_gumbel(L, 23, t, 6, anc, prec)


def test_gumbel_ragged_tiles_f16(pf):
    """Three tiles and a ragged tail (argmax CTAs of 8 offspring, the last one partial)."""
    v = synth.make_video(160, 120, 4, 4, noise=5.0, seed=48, v=(1.0, -1.0))
    anc, L, t = _gumbel_step(pf, v, 3 * TILE + 17, "f16", 24, tracker=1)
    _check_gumbel(L, 24, t, 1, anc, "f16")


@pytest.mark.parametrize("prec", ["ref64", "f16"])
def test_gumbel_largest_tracker_sampled(pf, prec):
    """N = 2^16, the largest Gumbel-max tracker: 96 sampled offspring are the argmax of
    L + g computed one by one from the oracle's variates (up to a near tie)."""
    v = synth.make_video(512, 512, 3, 5, noise=5.0, seed=1)
    N = 1 << 16
    anc, L, t = _gumbel_step(pf, v, N, prec, 1)
    assert np.all((anc >= 0) & (anc < N))
    rng = np.random.default_rng(3)
    for j in np.concatenate([[0, N - 1], rng.choice(N, 94, replace=False)]):
        best = int(np.argmax(L + oracle.gumbel_variates(1, t, int(j), N, 0)))
        assert anc[j] == best or _near_tie(L, 1, t, 0, j, best, anc[j], prec), (j, best, anc[j])


def test_gumbel_ref64_track_within_1e9(pf):
    v = synth.make_video(128, 128, 10, 5, noise=5.0, seed=1)
    est_o, M_o, _ = oracle.track(v.frames, 1000, 5, init=tuple(v.centres[0]), seed=1, resampler="gumbel")
    f = pf.Filter(v.W, v.H, 1000, 5, "ref64", init=tuple(v.centres[0]), seed=1, resampler="gumbel")
    f.run(_frames(v))
    est, ms = f.estimates(0, v.T, with_stats=True)
    f.close()
    assert np.abs(est - est_o).max() <= 1e-9
    assert np.array_equal(ms[:, 0], M_o)


@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
def test_gumbel_tracks_the_truth_and_steps_equal_runs(pf, prec):
    v = synth.make_video(128, 128, 10, 5, noise=5.0, seed=1)
    est_o, _, _ = oracle.track(v.frames, 1000, 5, init=tuple(v.centres[0]), seed=1, resampler="gumbel")
    fr = _frames(v)
    a = pf.Filter(v.W, v.H, 1000, 5, prec, init=tuple(v.centres[0]), seed=1, resampler="gumbel")
    a.run(fr)
    b = pf.Filter(v.W, v.H, 1000, 5, prec, init=tuple(v.centres[0]), seed=1, resampler="gumbel")
    for t in range(v.T):
        b.step(fr[t])
    ea, eb = a.estimates(0, v.T), b.estimates(0, v.T)
    a.close()
    b.close()
    assert np.array_equal(ea, eb)
    assert np.sqrt(np.mean(np.sum((ea - est_o) ** 2, axis=1))) <= 0.5


def test_four_schemes_in_one_batch_equal_singles(pf):
    vids = [synth.make_video(96, 96, 5, 3, noise=5.0, seed=90 + i, v=(1.0, -1.0)) for i in range(5)]
    Ns = [3000, 2 * TILE + 5, 777, 5000, 1500]
    rs = ["gumbel", "systematic", "stratified", "multinomial", "gumbel"]
    for prec in ("ref64", "f32", "f16"):
        cfgs = [pf.make_config(v.W, v.H, n, v.radius, prec, init=tuple(v.centres[0]), seed=60 + i,
                               tracker_id=i, resampler=r) for i, (v, n, r) in enumerate(zip(vids, Ns, rs))]
        b = pf.Batch(cfgs)
        fr = [_frames(v) for v in vids]
        for t in range(5):
            b.step([f[t] for f in fr])
        got = np.stack([b.estimates(t) for t in range(5)], axis=1)
        c = b.counters()
        b.close()
        assert c["kernel_launches"] == 5 * 4, c      # step, CDF, argmax, pull
        for i, (v, n, r) in enumerate(zip(vids, Ns, rs)):
            s = pf.Filter(v.W, v.H, n, v.radius, prec, init=tuple(v.centres[0]), seed=60 + i, tracker_id=i,
                          resampler=r)
            s.run(fr[i])
            assert np.array_equal(s.estimates(0, 5), got[i]), (prec, i, r)
            s.close()


def test_gumbel_limits_and_debug(pf):
    """N <= 2^16; no CDF to read back; the server refuses Gumbel-max streams."""
    with pytest.raises(pf.PfError):
        pf.Filter(64, 64, (1 << 16) + 1, 3, "f16", resampler="gumbel")
    f = pf.Filter(64, 64, 100, 3, "f32", init=(32.0, 32.0), resampler="gumbel", flags=pf.PF_FLAG_DEBUG_ARRAYS)
    f.step(np.full((64, 64), 100, np.uint8))
    with pytest.raises(pf.PfError):
        f.debug(1)
    f.close()
    s = pf.Server(1 << 26, max_streams=2, queue_depth=2)
    with pytest.raises(pf.PfError):
        s.open(pf.make_config(64, 64, 100, 3, "f16", resampler="gumbel"))
    s.close()


# ----------------------------------------------------------------------------- Metropolis
def _metropolis_step(pf, v, N, prec, seed, *, tracker=0, steps=0):
    """As _gumbel_step, for a Metropolis tracker of chain length `steps` (0 = 64)."""
    f = pf.Filter(v.W, v.H, N, v.radius, prec, init=tuple(v.centres[0]), seed=seed, tracker_id=tracker,
                  flags=pf.PF_FLAG_DEBUG_ARRAYS, resampler="metropolis", resampler_steps=steps)
    fr = _frames(v)
    f.run(fr[:v.T - 1])
    st = f.get_state()
    f.step(fr[v.T - 1])
    anc = f.debug(0).astype(np.int64)
    f.close()
    return anc, st["L"].astype(np.float64), int(st["t"]) - 1


def _check_metropolis(L, B, seed, t, tracker, anc, prec):
    """Ancestors equal the oracle's chains in the kernel's precision; a chain that ends
    elsewhere must pass an acceptance test within rounding of its threshold (FP32 logs of
    the two sides may differ in the last bit), and such chains are rare."""
    want = oracle.resample_metropolis(L, B, seed, t, tracker, "f64" if prec == "ref64" else "f32")
    bad = np.nonzero(anc != want)[0]
    assert np.all((anc >= 0) & (anc < L.size))
    assert bad.size <= max(1, L.size // 1000), bad[:10]
    tol = 1e-12 if prec == "ref64" else 1e-4
    for j in bad:
        _, margins = oracle.metropolis_chain(L, B, seed, t, int(j), tracker)
        assert min(margins) <= tol, (j, want[j], anc[j], min(margins))


@pytest.mark.parametrize("prec", ["ref64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("N", [1, 3, 1000, TILE + 1, 3 * TILE + 17])
def test_metropolis_ancestors_exact(pf, prec, N):
    v = synth.make_video(128, 128, 4, 5, noise=5.0, seed=49)
    anc, L, t = _metropolis_step(pf, v, N, prec, 27, tracker=7)
    _check_metropolis(L, 64, 27, t, 7, anc, prec)


@pytest.mark.parametrize("steps", [1, 2, 7, 300])
def test_metropolis_chain_lengths(pf, steps):
    v = synth.make_video(128, 128, 4, 5, noise=5.0, seed=50)
    anc, L, t = _metropolis_step(pf, v, 5000, "f32", 28, tracker=2, steps=steps)
    _check_metropolis(L, steps, 28, t, 2, anc, "f32")


@pytest.mark.parametrize("prec", ["ref64", "f16"])
def test_metropolis_full_size_ancestors_exact(pf, prec):
    """The bench's configuration, 2^20 particles: every chain checked."""
    v = synth.make_video(512, 512, 3, 5, noise=5.0, seed=1)
    anc, L, t = _metropolis_step(pf, v, 1 << 20, prec, 1)
    _check_metropolis(L, 64, 1, t, 0, anc, prec)


def test_metropolis_ref64_track_within_1e9(pf):
    v = synth.make_video(128, 128, 10, 5, noise=5.0, seed=1)
    for N in (1000, 3 * TILE + 17):
        est_o, M_o, _ = oracle.track(v.frames, N, 5, init=tuple(v.centres[0]), seed=1, resampler="metropolis")
        f = pf.Filter(v.W, v.H, N, 5, "ref64", init=tuple(v.centres[0]), seed=1, resampler="metropolis")
        f.run(_frames(v))
        est, ms = f.estimates(0, v.T, with_stats=True)
        f.close()
        assert np.abs(est - est_o).max() <= 1e-9, N
        assert np.array_equal(ms[:, 0], M_o)


@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
def test_metropolis_tracks_the_truth_and_steps_equal_runs(pf, prec):
    v = synth.make_video(128, 128, 10, 5, noise=5.0, seed=1)
    est_o, _, _ = oracle.track(v.frames, 1000, 5, init=tuple(v.centres[0]), seed=1, resampler="metropolis")
    fr = _frames(v)
    a = pf.Filter(v.W, v.H, 1000, 5, prec, init=tuple(v.centres[0]), seed=1, resampler="metropolis")
    a.run(fr)
    b = pf.Filter(v.W, v.H, 1000, 5, prec, init=tuple(v.centres[0]), seed=1, resampler="metropolis")
    for t in range(v.T):
        b.step(fr[t])
    ea, eb = a.estimates(0, v.T), b.estimates(0, v.T)
    a.close()
    b.close()
    assert np.array_equal(ea, eb)
    assert np.sqrt(np.mean(np.sum((ea - est_o) ** 2, axis=1))) <= 0.5


# ----------------------------------------------------------------------------- rejection
def _check_rejection(L, M, seed, t, tracker, anc, prec, tries=4096):
    """Ancestors equal the oracle's tries in the kernel's precision (bound M from the
    state); an offspring that ends elsewhere must have met a test within rounding of its
    threshold, and such offspring are rare."""
    want = oracle.resample_rejection(L, M, seed, t, tracker, "f64" if prec == "ref64" else "f32", tries)
    bad = np.nonzero(anc != want)[0]
    assert np.all((anc >= 0) & (anc < L.size))
    assert bad.size <= max(1, L.size // 1000), bad[:10]
    tol = 1e-12 if prec == "ref64" else 1e-4
    for j in bad:
        _, margins = oracle.rejection_trace(L, M, seed, t, int(j), tracker, tries)
        assert min(margins) <= tol, (j, want[j], anc[j], min(margins))


def _rejection_step(pf, v, N, prec, seed, *, tracker=0, tries=0):
    f = pf.Filter(v.W, v.H, N, v.radius, prec, init=tuple(v.centres[0]), seed=seed, tracker_id=tracker,
                  flags=pf.PF_FLAG_DEBUG_ARRAYS, resampler="rejection", resampler_steps=tries)
    fr = _frames(v)
    f.run(fr[:v.T - 1])
    st = f.get_state()
    f.step(fr[v.T - 1])
    anc = f.debug(0).astype(np.int64)
    f.close()
    return anc, st["L"].astype(np.float64), float(st["max_l"]), int(st["t"]) - 1


@pytest.mark.parametrize("prec", ["ref64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("N", [1, 3, 1000, TILE + 1, 3 * TILE + 17])
def test_rejection_ancestors_exact(pf, prec, N):
    v = synth.make_video(128, 128, 4, 5, noise=5.0, seed=51)
    anc, L, M, t = _rejection_step(pf, v, N, prec, 29, tracker=8)
    assert M == L.max() or prec != "ref64"
    _check_rejection(L, M, 29, t, 8, anc, prec)


@pytest.mark.parametrize("tries", [1, 2, 5])
def test_rejection_truncated_tries(pf, tries):
    """Few tries: many offspring keep their last candidate, exactly as the oracle does."""
    v = synth.make_video(128, 128, 4, 5, noise=5.0, seed=52)
    anc, L, M, t = _rejection_step(pf, v, 5000, "f32", 30, tracker=3, tries=tries)
    _check_rejection(L, M, 30, t, 3, anc, "f32", tries)


def test_rejection_full_size_ancestors_exact(pf):
    v = synth.make_video(512, 512, 3, 5, noise=5.0, seed=1)
    anc, L, M, t = _rejection_step(pf, v, 1 << 20, "f16", 1)
    _check_rejection(L, M, 1, t, 0, anc, "f16")


def test_rejection_ref64_track_within_1e9(pf):
    v = synth.make_video(128, 128, 10, 5, noise=5.0, seed=1)
    for N in (1000, 3 * TILE + 17):
        est_o, M_o, _ = oracle.track(v.frames, N, 5, init=tuple(v.centres[0]), seed=1, resampler="rejection")
        f = pf.Filter(v.W, v.H, N, 5, "ref64", init=tuple(v.centres[0]), seed=1, resampler="rejection")
        f.run(_frames(v))
        est, ms = f.estimates(0, v.T, with_stats=True)
        f.close()
        assert np.abs(est - est_o).max() <= 1e-9, N
        assert np.array_equal(ms[:, 0], M_o)


@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
def test_rejection_tracks_the_truth_and_steps_equal_runs(pf, prec):
    v = synth.make_video(128, 128, 10, 5, noise=5.0, seed=1)
    est_o, _, _ = oracle.track(v.frames, 1000, 5, init=tuple(v.centres[0]), seed=1, resampler="rejection")
    fr = _frames(v)
    a = pf.Filter(v.W, v.H, 1000, 5, prec, init=tuple(v.centres[0]), seed=1, resampler="rejection")
    a.run(fr)
    b = pf.Filter(v.W, v.H, 1000, 5, prec, init=tuple(v.centres[0]), seed=1, resampler="rejection")
    for t in range(v.T):
        b.step(fr[t])
    ea, eb = a.estimates(0, v.T), b.estimates(0, v.T)
    a.close()
    b.close()
    assert np.array_equal(ea, eb)
    assert np.sqrt(np.mean(np.sum((ea - est_o) ** 2, axis=1))) <= 0.5


def test_six_schemes_in_one_batch_equal_singles(pf):
    vids = [synth.make_video(96, 96, 5, 3, noise=5.0, seed=100 + i, v=(1.0, -1.0)) for i in range(7)]
    Ns = [3000, 2 * TILE + 5, 777, 5000, 1500, 2 * TILE + 300, 2500]
    rs = ["metropolis", "systematic", "stratified", "multinomial", "gumbel", "metropolis", "rejection"]
    steps = [0, 0, 0, 0, 0, 9, 0]
    for prec in ("ref64", "f32", "f16"):
        cfgs = [pf.make_config(v.W, v.H, n, v.radius, prec, init=tuple(v.centres[0]), seed=40 + i,
                               tracker_id=i, resampler=r, resampler_steps=b)
                for i, (v, n, r, b) in enumerate(zip(vids, Ns, rs, steps))]
        bt = pf.Batch(cfgs)
        fr = [_frames(v) for v in vids]
        for t in range(5):
            bt.step([f[t] for f in fr])
        got = np.stack([bt.estimates(t) for t in range(5)], axis=1)
        c = bt.counters()
        bt.close()
        assert c["kernel_launches"] == 5 * 6, c      # step, CDF, argmax, chains, tries, pull
        for i, (v, n, r, b) in enumerate(zip(vids, Ns, rs, steps)):
            s1 = pf.Filter(v.W, v.H, n, v.radius, prec, init=tuple(v.centres[0]), seed=40 + i, tracker_id=i,
                           resampler=r, resampler_steps=b)
            s1.run(fr[i])
            assert np.array_equal(s1.estimates(0, 5), got[i]), (prec, i, r)
            s1.close()
            # every tracker of the mixed batch against the oracle's track with its scheme:
            # REF64 within 1e-9 px; F32 within 1e-3 px for the schemes decided by a search of the
            # CDF; otherwise (FP32 near ties of argmax / acceptance tests, half arithmetic) RMSE 0.5 px
            est_o, _, _ = oracle.track(v.frames, n, v.radius, init=tuple(v.centres[0]), seed=40 + i, tracker=i,
                                       resampler=r, iters=b or None)
            if prec == "ref64":
                assert np.abs(got[i] - est_o).max() <= 1e-9, (prec, i, r)
            elif prec == "f32" and r in ("systematic", "stratified", "multinomial"):
                assert np.abs(got[i] - est_o).max() <= 1e-3, (prec, i, r)
            else:
                assert np.sqrt(np.mean(np.sum((got[i] - est_o) ** 2, axis=1))) <= 0.5, (prec, i, r)


def test_metropolis_limits_and_debug(pf):
    """N <= 2^24 and chain length <= 4096; other schemes take no chain length; no CDF to
    read back; the server refuses Metropolis streams."""
    for kw in (dict(num_particles=(1 << 24) + 1), dict(resampler_steps=4097), dict(resampler_steps=-2)):
        args = dict(num_particles=100, resampler_steps=0)
        args.update(kw)
        with pytest.raises(pf.PfError):
            pf.Filter(64, 64, args["num_particles"], 3, "f16", resampler="metropolis",
                      resampler_steps=args["resampler_steps"])
    with pytest.raises(pf.PfError):
        pf.Filter(64, 64, 100, 3, "f16", resampler="stratified", resampler_steps=5)
    f = pf.Filter(64, 64, 100, 3, "f32", init=(32.0, 32.0), resampler="metropolis", flags=pf.PF_FLAG_DEBUG_ARRAYS)
    f.step(np.full((64, 64), 100, np.uint8))
    with pytest.raises(pf.PfError):
        f.debug(1)
    f.close()
    s = pf.Server(1 << 26, max_streams=2, queue_depth=2)
    for scheme in ("metropolis", "rejection"):
        with pytest.raises(pf.PfError):
            s.open(pf.make_config(64, 64, 100, 3, "f16", resampler=scheme))
    s.close()
    with pytest.raises(pf.PfError):
        pf.Filter(64, 64, 100, 3, "f16", resampler="rejection", resampler_steps=65537)


def test_counters_count_launches_graphs_and_host_bytes(pf):
    """pf_get_counters: one kernel per frame for systematic trackers, three for multinomial
    (step kernel skipped: CDF and pull), one graph replay per resident run, host bytes."""
    v = synth.make_video(96, 80, 7, 3, noise=5.0, seed=44)
    fr = _frames(v)
    for rs, per in (("systematic", 1), ("multinomial", 2), ("gumbel", 2), ("metropolis", 2), ("rejection", 2)):
        f = pf.Filter(v.W, v.H, 3000, 3, "f32", init=tuple(v.centres[0]), seed=2, resampler=rs)
        f.step(v.frames[0])                      # host frame
        f.step(fr[1])
        f.run(fr[2:7])                            # one graph replay of 5 steps
        c = f.counters()
        f.close()
        assert c == {"frames": 7, "step_launches": 7, "kernel_launches": 7 * per, "graph_launches": 1,
                     "host_frame_bytes": v.W * v.H, "status": 0}, (rs, c)
    cfgs = [pf.make_config(v.W, v.H, n, 3, "f16", init=tuple(v.centres[0]), seed=5 + i, tracker_id=i, resampler=rs)
            for i, (n, rs) in enumerate(((2000, "systematic"), (900, "multinomial")))]
    b = pf.Batch(cfgs)
    for t in range(3):
        b.step([fr[t], fr[t]])
    c = b.counters()
    b.close()
    assert c["frames"] == 6 and c["step_launches"] == 3 and c["kernel_launches"] == 9 and c["graph_launches"] == 0
