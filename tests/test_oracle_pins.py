"""Pins of the CPU FP64 oracle to things other than itself (no GPU needed).

Each test checks the oracle against what the paper or mathematics fixes: a library run
as a black box (cuRAND's host Philox generator, numpy, scipy), closed forms of Eq. 3,
invariants of systematic resampling (Sec. IV), brute force on tiny inputs, and recovery
of the known ground-truth trajectory of the synthetic video (Sec. V, verification).
"""
import ctypes
import ctypes.util
import glob
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2308_00763_gb300 import synth
from conftest import GOLDEN


# ----------------------------------------------------------------------------- Philox
def _curand():
    cands = []
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d:
            cands += sorted(glob.glob(os.path.join(d, "lib64", "libcurand.so*")))
            cands += sorted(glob.glob(os.path.join(d, "targets", "*", "lib", "libcurand.so*")))
    found = ctypes.util.find_library("curand")
    if found:
        cands.append(found)
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


def _curand_host_words(lib, seed, n_words, offset=0):
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(n_words, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n_words)) == 0
        return out
    finally:
        lib.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [1, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
@pytest.mark.parametrize("offset_blocks", [0, 65536 * 3 + 17, 1 << 48])
def test_philox_matches_curand_host_generator(seed, offset_blocks):
    """cuRAND's host Philox4x32-10 generator (run on the CPU as a black box) emits, in its
    default ordering, block B of four words = Philox(ctr = (B >> 16 as a 64-bit value in
    words 0-1, B & 0xffff in word 2, 0), key = seed).  That layout was read off the
    library's output; the oracle must reproduce every block bit for bit."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    nblk = 4096
    words = _curand_host_words(lib, seed, 4 * nblk, offset=4 * offset_blocks).reshape(nblk, 4)
    B = np.arange(offset_blocks, offset_blocks + nblk, dtype=np.uint64)
    hi = B >> np.uint64(16)
    ctr = np.stack([(hi & np.uint64(0xFFFFFFFF)).astype(np.uint32),
                    (hi >> np.uint64(32)).astype(np.uint32),
                    (B & np.uint64(0xFFFF)).astype(np.uint32),
                    np.zeros(nblk, np.uint32)], axis=1)
    got = oracle.philox(ctr, seed)
    assert np.array_equal(got, words)


def test_propagation_draw_mapping():
    """One Philox block per particle pair: particle j uses block j // 2 (counter word 0),
    words 2(j % 2) and 2(j % 2) + 1, frame t in word 1, tag 0, tracker id in word 3."""
    seed, t, trk = 77, 5, 3
    n = 1001
    nx, ny = oracle.normals(seed, t, n, tracker=trk, start=10)
    j = np.arange(10, 10 + n)
    ctr = np.stack([(j // 2).astype(np.uint32), np.full(n, t, np.uint32), np.zeros(n, np.uint32),
                    np.full(n, trk, np.uint32)], axis=1)
    w = oracle.philox(ctr, seed)
    h = 2 * (j % 2)
    ua = oracle.uniform(w[np.arange(n), h])
    ub = oracle.uniform(w[np.arange(n), h + 1])
    bx, by = oracle.box_muller(ua, ub)
    assert np.array_equal(nx, bx) and np.array_equal(ny, by)


def test_philox_counter_words_all_matter():
    base = np.array([[5, 6, 7, 8]], np.uint32)
    ref = oracle.philox(base, 42)
    for i in range(4):
        c = base.copy()
        c[0, i] ^= 1
        assert not np.array_equal(oracle.philox(c, 42), ref)
    assert not np.array_equal(oracle.philox(base, 43), ref)
    assert not np.array_equal(oracle.philox(base, 42 | (1 << 40)), ref)


# ----------------------------------------------------------------------------- uniforms / normals
def test_uniform_grid_exact_in_fp32():
    w = np.array([0, 511, 512, 1 << 31, 0xFFFFFFFF, 0xFFFFFE00, 0x12345678], np.uint32)
    u = oracle.uniform(w)
    assert u[0] == 2.0 ** -24 and u[1] == 2.0 ** -24          # low 9 bits dropped
    assert u[2] == 3 * 2.0 ** -24
    assert u[3] == 0.5 + 2.0 ** -24
    assert u[4] == 1.0 - 2.0 ** -24 and u[5] == u[4]
    ctr = np.stack([np.arange(200000, dtype=np.uint32)] + [np.zeros(200000, np.uint32)] * 3, 1)
    uu = oracle.uniform(oracle.philox(ctr, 7).ravel())
    assert np.all(uu.astype(np.float32).astype(np.float64) == uu)   # every value exact in FP32
    assert uu.min() > 0.0 and uu.max() < 1.0
    # uniformity: chi-square over 64 equal bins (scipy as the reference)
    stats = pytest.importorskip("scipy.stats")
    counts, _ = np.histogram(uu, bins=64, range=(0, 1))
    assert stats.chisquare(counts).pvalue > 1e-4


def test_box_muller_normals():
    stats = pytest.importorskip("scipy.stats")
    n = 1 << 20
    nx, ny = oracle.normals(seed=1, t=3, n=n)
    for v in (nx, ny):
        assert abs(v.mean()) < 5.0 / math.sqrt(n)
        assert abs(v.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
        assert stats.kstest(v, "norm").pvalue > 1e-4
    assert abs(np.corrcoef(nx, ny)[0, 1]) < 5.0 / math.sqrt(n)
    # the 23-bit uniforms bound every draw by sqrt(-2 ln 2^-24)
    assert np.abs(nx).max() <= math.sqrt(48 * math.log(2)) + 1e-12
    # closed form of the transform: n_x^2 + n_y^2 = -2 ln u_a, atan2 gives 2 pi u_b
    ua = np.array([0.25, 0.5, 0.75, 2.0 ** -24])
    ub = np.array([0.0, 0.125, 0.5, 0.75])
    bx, by = oracle.box_muller(ua, ub)
    np.testing.assert_allclose(bx * bx + by * by, -2.0 * np.log(ua), rtol=1e-14)
    np.testing.assert_allclose(np.mod(np.arctan2(by, bx), 2 * np.pi), 2 * np.pi * ub, atol=1e-14)


# ----------------------------------------------------------------------------- template / rounding
def test_disk_counts_golden():
    with open(os.path.join(GOLDEN, "disk_counts.json")) as f:
        counts = json.load(f)["counts"]
    for r, n in counts.items():
        assert oracle.disk_count(int(r)) == n


def test_round_pixel_special_values():
    v = np.array([2.5, np.nextafter(2.5, 0), -0.5, np.nextafter(-0.5, -1), 7.0, -7.0,
                  1e6 + 0.5, 0.49999999999999994, 3.75, -3.25])
    want = np.array([3, 2, 0, -1, 7, -7, 1000001, 0, 4, -3])
    assert np.array_equal(oracle.round_pixel(v), want)
    # away from the half-way points it is numpy's rounding
    rng = np.random.default_rng(0)
    x = rng.uniform(-600, 600, 100000)
    x = x[np.abs(x - np.floor(x) - 0.5) > 1e-6]
    assert np.array_equal(oracle.round_pixel(x), np.rint(x).astype(np.int64))


# ----------------------------------------------------------------------------- likelihood, Eq. 3
def _golden_L():
    with open(os.path.join(GOLDEN, "likelihood_closed_forms.json")) as f:
        return json.load(f)


def test_likelihood_uniform_frame_closed_form():
    g = _golden_L()
    for case in g["uniform_frame"]:
        frame = np.full((40, 50), case["c"], np.uint8)
        for r in (1, 3, 5, 10):
            for (px, py) in [(25, 20), (0, 0), (49, 39), (3, 37)]:
                got = oracle.likelihood_at(frame, r, px, py)
                assert abs(got - float(Fraction(case["L"]))) < 1e-12


def test_likelihood_half_plane_closed_form():
    g = _golden_L()["half_plane"]["cases"]
    X0 = 30
    frame = np.full((64, 64), 100, np.uint8)
    frame[:, :X0] = 228
    for case in g:
        assert oracle.disk_count(case["r"]) == case["D"]
        got = oracle.likelihood_at(frame, case["r"], X0, 32)
        assert abs(got - float(Fraction(case["L"]))) < 1e-12
        # the transposed frame needs the transposed position (x = column, y = row)
        got_t = oracle.likelihood_at(frame.T.copy(), case["r"], 20, X0)
        assert abs(got_t - float(Fraction(case["L"]))) < 1e-12
        # r columns left of the edge the template is all foreground
        assert abs(oracle.likelihood_at(frame, case["r"], X0 - 1 - case["r"], 32) - 327.68) < 1e-12


def test_likelihood_corner_clamp_closed_form():
    g = _golden_L()["corner_clamp"]
    frame = np.full((16, 16), 100, np.uint8)
    frame[0, 0] = 228
    assert abs(oracle.likelihood_at(frame, g["r"], 0, 0) - float(Fraction(g["L"]))) < 1e-12
    # the opposite corner clamps the same way
    frame2 = np.full((16, 20), 100, np.uint8)
    frame2[15, 19] = 228
    assert abs(oracle.likelihood_at(frame2, 1, 19, 15) - float(Fraction(g["L"]))) < 1e-12


def test_likelihood_noiseless_disk_video():
    v = synth.make_video(96, 80, 6, 5, v=(1, -2), noise=0.0, seed=3)
    for t in range(v.T):
        cx, cy = (int(c) for c in v.centres[t])
        assert oracle.likelihood_at(v.frames[t], 5, cx, cy) == pytest.approx(327.68, abs=1e-12)
        # shifted by one column: the closed form with m counted by brute force on the frame
        m = 0
        for dy in range(-5, 6):
            for dx in range(-5, 6):
                if dx * dx + dy * dy <= 25 and v.frames[t][cy + dy, cx + 1 + dx] == 100:
                    m += 1
        want = 8192.0 * (81 - 2 * m) / (25.0 * 81)
        assert oracle.likelihood_at(v.frames[t], 5, cx + 1, cy) == pytest.approx(want, abs=1e-12)
    # far from the disk: pure background
    assert oracle.likelihood_at(v.frames[0], 5, 10, 70) == pytest.approx(-327.68, abs=1e-12)


def test_likelihood_integer_form_identity():
    """(256 * sum(I) - 41984 |D|) / (50 |D|) equals the per-pixel Eq. 3 sum exactly: the
    integer disk sum is a second, independent calculation of the same value."""
    rng = np.random.default_rng(5)
    frame = rng.integers(0, 256, size=(37, 53), dtype=np.uint8)
    for r in (1, 3, 5, 12):
        D = oracle.disk_count(r)
        for _ in range(200):
            px, py = int(rng.integers(-3, 56)), int(rng.integers(-3, 40))
            s = oracle.disk_sum(frame, r, px, py)
            assert oracle.likelihood_at(frame, r, px, py) == (256.0 * s - 41984.0 * D) / (50.0 * D)


# ----------------------------------------------------------------------------- Eq. 4 in half precision
def test_half_rounding_helpers_match_library_conversions():
    """The rounding helpers against library conversions from binary32 (one rounding
    there too): numpy's float32 -> float16 and torch's float32 -> bfloat16, both
    round-to-nearest-even, on random values, exact ties and their neighbours."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    v = np.concatenate([rng.normal(0, 30, 20000), rng.uniform(-1, 1, 20000) * 2.0 ** -8,
                        1.0 + np.arange(-64, 64) * 2.0 ** -11, 256.0 + np.arange(-64, 64) * 2.0 ** -3])
    v32 = v.astype(np.float32)
    assert np.array_equal(oracle.round_half(v32.astype(np.float64)), v32.astype(np.float16).astype(np.float64))
    want = torch.from_numpy(v32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(oracle.round_bf16(v32.astype(np.float64)), want)
    # ties to even, exactly representable values unchanged
    assert oracle.round_half(1.0 + 2.0 ** -11) == 1.0 and oracle.round_half(1.0 + 3 * 2.0 ** -11) == 1.0 + 2 ** -9
    assert oracle.round_bf16(1.0 + 2.0 ** -8) == 1.0 and oracle.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2 ** -6
    assert np.array_equal(oracle.round_half(np.arange(-2048.0, 2049.0)), np.arange(-2048.0, 2049.0))


def test_half_likelihood_uniform_frame_by_float16_arithmetic():
    """Uniform frames: every template term is the same binary16 value, formed and summed
    here with numpy's own float16 arithmetic (each operation exact in binary32 at these
    magnitudes, then rounded once) row by row, the row sums then added top to bottom; the
    oracle's emulation must give the same bits."""
    for r in (1, 3, 5, 10):
        D = oracle.disk_count(r)
        kap = np.float16(np.float32(1.0 / math.sqrt(50.0 * D)))
        for c in (0, 37, 100, 150, 164, 228, 255):
            a = np.float16(np.float16(c - 100) * kap)
            b = np.float16(np.float16(c - 228) * kap)
            term = np.float16(np.float64(a) * np.float64(a) - np.float64(np.float16(b * b)))
            # row widths of the disk: 2 floor(sqrt(r^2 - dy^2)) + 1
            widths = [2 * math.isqrt(r * r - dy * dy) + 1 for dy in range(-r, r + 1)]
            assert sum(widths) == D
            acc = np.float16(0.0)
            acc32 = np.float32(0.0)
            for n in widths:
                row = np.float16(0.0)
                row32 = np.float32(0.0)
                for _ in range(n):
                    row = np.float16(row + term)
                    row32 = np.float32(row32 + np.float32(term))
                acc = np.float16(acc + row)
                acc32 = np.float32(acc32 + row32)
            frame = np.full((40, 50), c, np.uint8)
            got = oracle.likelihood_half(np.array([25.0, 0.2]), np.array([20.0, 39.0]), frame, r, "f16")
            assert np.all(got == np.float64(acc)), (r, c)
            # and the FP32-accumulated form
            got32 = oracle.likelihood_half(np.array([25.0]), np.array([20.0]), frame, r, "f16acc32")
            assert got32[0] == np.float64(np.float16(acc32)), (r, c)


@pytest.mark.parametrize("kind", ["f16", "f16acc32", "bf16"])
def test_half_likelihood_within_the_rounding_bound(kind):
    """Against the FP64 Eq. 3 value: the half result differs by at most the rounding bound
    of its operations -- per term the roundings of a, b, b b and a a - b b (and kappa's own
    rounding, a relative 2u on the whole sum), per addition u times the running sum, u the
    unit roundoff of the lane type (2^-11 binary16, 2^-8 bfloat16) or of binary32 for the
    accumulation.  (The bound is loose; the GPU's half likelihoods are compared with this
    emulation bit for bit.)"""
    u = 2.0 ** -8 if kind == "bf16" else 2.0 ** -11
    u_acc = 2.0 ** -11 if kind == "f16" else 2.0 ** -24
    rng = np.random.default_rng(2)
    v = synth.make_video(128, 128, 3, 5, noise=5.0, seed=1)
    frame = v.frames[2]
    x = rng.uniform(30, 100, 3000)
    y = rng.uniform(30, 100, 3000)
    r = 5
    D = oracle.disk_count(r)
    L = oracle.likelihood_all(x, y, frame, r)
    Lh = oracle.likelihood_half(x, y, frame, r, kind)
    px, py = oracle.round_pixel(x), oracle.round_pixel(y)
    kap2 = 1.0 / (50.0 * D)
    s = np.zeros(x.size)
    bound = np.zeros(x.size)
    for dx, dy in oracle.template_offsets(r):
        I = frame[np.clip(py + dy, 0, 127), np.clip(px + dx, 0, 127)].astype(np.float64)
        a2, b2 = (I - 100.0) ** 2 * kap2, (I - 228.0) ** 2 * kap2
        s = s + (a2 - b2)
        bound += 4.0 * u * (a2 + b2) + u_acc * np.abs(s) * 1.01
    bound += 2.1 * u * np.abs(L) + u * np.abs(L)
    assert np.all(np.abs(Lh - L) <= bound)
    assert np.abs(Lh - L).max() > 0.0            # it is a half computation, not the FP64 one


# ----------------------------------------------------------------------------- weights, normalisation, CDF
def test_weights_shift_invariance_and_dominance():
    rng = np.random.default_rng(1)
    L = np.round(rng.uniform(-300, 300, 1000) * 8) / 8
    M, e = oracle.weights(L)
    assert M == L.max() and e.max() == 1.0 and np.all(e >= 0)
    M2, e2 = oracle.weights(L + 1024.0)
    assert M2 == M + 1024.0 and np.array_equal(e, e2)
    M3, e3 = oracle.weights(np.array([-1000.0, 0.0, -1000.0]))
    assert M3 == 0.0 and np.array_equal(e3, [0.0, 1.0, 0.0])


def test_normalise_invariants():
    rng = np.random.default_rng(2)
    e = rng.uniform(0, 1, 5000)
    x = rng.uniform(0, 512, 5000)
    y = rng.uniform(0, 512, 5000)
    S, xh, yh = oracle.normalise(e, x, y)
    assert abs(S - math.fsum(e)) <= 4 * np.finfo(float).eps * S
    assert abs(math.fsum(e / S) - 1.0) < 5000 * np.finfo(float).eps
    assert abs(xh - math.fsum(e * x) / math.fsum(e)) < 1e-12
    assert x.min() <= xh <= x.max() and y.min() <= yh <= y.max()
    S1, xh1, yh1 = oracle.normalise(np.array([0.25]), np.array([3.5]), np.array([-7.25]))
    assert (S1, xh1, yh1) == (0.25, 3.5, -7.25)
    S2, xh2, yh2 = oracle.normalise(e[:100], np.full(100, 123.375), np.full(100, 9.0625))
    assert abs(xh2 - 123.375) < 1e-12 and abs(yh2 - 9.0625) < 1e-12


def test_cdf_matches_cumsum_and_is_monotone():
    rng = np.random.default_rng(3)
    for n in (1, 2, 7, 1000, 100003):
        e = rng.exponential(size=n) * (rng.uniform(size=n) < 0.3)
        e[rng.integers(n)] = 1.0
        S, _, _ = oracle.normalise(e, np.zeros(n), np.zeros(n))
        C = oracle.cdf(e, S)
        assert C[-1] == 1.0
        assert np.all(np.diff(C) >= 0)
        np.testing.assert_allclose(C, np.cumsum(e) / e.sum(), rtol=0, atol=n * np.finfo(float).eps)


# ----------------------------------------------------------------------------- systematic resampling
def _counts(a, n):
    return np.bincount(a, minlength=n)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_resample_uniform_weights_identity(prec):
    for n in (1, 2, 8, 1024, 1 << 16):
        C = (np.arange(n, dtype=np.float64) + 1) / n     # exact for powers of two
        # in FP32, j + u0 must itself be exact (u0 = 2^-24 vanishes next to j >= 1)
        offsets = (2.0 ** -24, 0.5, 1 - 2.0 ** -24) if prec == "f64" else (0.25, 0.5, 0.75)
        for u0 in offsets:
            a = oracle.resample(C, u0, prec)
            assert np.array_equal(a, np.arange(n))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_resample_offspring_counts_floor_ceil(prec):
    rng = np.random.default_rng(4)
    for n in (1, 2, 3, 7, 100, 1000, 4097):
        for trial in range(5):
            e = rng.exponential(size=n) ** 3
            S, _, _ = oracle.normalise(e, np.zeros(n), np.zeros(n))
            C = oracle.cdf(e, S)
            if prec == "f32":
                C = C.astype(np.float32).astype(np.float64)
            u0 = float(oracle.uniform([rng.integers(0, 2 ** 32, dtype=np.uint64)])[0])
            a = oracle.resample(C, u0, prec)
            assert np.all(np.diff(a) >= 0) and a.min() >= 0 and a.max() < n
            cnt = _counts(a, n)
            assert cnt.sum() == n
            w = np.diff(np.concatenate([[0.0], C]))
            if prec == "f64":   # the FP32 strata are themselves rounded; the bound is for exact u_j
                assert np.all(cnt >= np.floor(n * w - 1e-9)) and np.all(cnt <= np.ceil(n * w + 1e-9))


def test_resample_brute_force_expectation():
    """N <= 8: averaged over a fine grid of offsets u0, the offspring count of particle k
    equals N * w_k (systematic resampling is unbiased)."""
    rng = np.random.default_rng(6)
    for n in (1, 2, 3, 5, 8):
        e = rng.uniform(0.01, 1.0, n)
        S, _, _ = oracle.normalise(e, np.zeros(n), np.zeros(n))
        C = oracle.cdf(e, S)
        w = np.diff(np.concatenate([[0.0], C]))
        G = 20000
        tot = np.zeros(n)
        for g in range(G):
            u0 = (g + 0.5) / G
            tot += _counts(oracle.resample(C, u0, "f64"), n)
        np.testing.assert_allclose(tot / G, n * w, atol=n / G * 2)


def test_resample_dominant_and_clamp():
    C = np.array([0.0, 0.0, 1.0, 1.0])
    assert np.array_equal(oracle.resample(C, 0.3, "f64"), [2, 2, 2, 2])
    C2 = np.array([0.2, 0.5, 0.9])     # no entry reaches the last strata: clamp to N-1
    assert np.array_equal(oracle.resample(C2, 0.9, "f64"), [1, 2, 2])
    # ties: a stratum point equal to a CDF entry belongs to that entry (first C_k >= u_j)
    C3 = np.array([0.25, 0.5, 0.75, 1.0])
    for prec in ("f64", "f32"):
        assert np.array_equal(oracle.resample(C3, 1.0, prec), [0, 1, 2, 3])
        assert np.array_equal(oracle.resample(C3, 0.0, prec), [0, 0, 1, 2])


# ----------------------------------------------------------------------------- naive form (division)
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_resample_by_division_pins(prec):
    """Points formed as (j + u0) / N: for N a power of two the division and the product
    with 1/N are the same exact operation, so the decisions equal the saved-constant form;
    for any N the offspring counts keep the floor/ceil property (FP64) and the ancestors
    are ordered."""
    rng = np.random.default_rng(18)
    for n in (1, 2, 8, 1024, 1 << 14):
        e = rng.exponential(size=n) ** 2
        S, _, _ = oracle.normalise(e, np.zeros(n), np.zeros(n))
        C = oracle.cdf(e, S)
        for u0 in (0.125, 0.5, 0.875):
            assert np.array_equal(oracle.resample(C, u0, prec, divide=True), oracle.resample(C, u0, prec))
    for n in (3, 7, 100, 4097):
        e = rng.exponential(size=n) ** 3
        S, _, _ = oracle.normalise(e, np.zeros(n), np.zeros(n))
        C = oracle.cdf(e, S)
        a = oracle.resample(C, 0.37, prec, divide=True)
        assert np.all(np.diff(a) >= 0) and a.min() >= 0 and a.max() < n
        cnt = _counts(a, n)
        assert cnt.sum() == n
        if prec == "f64":
            w = np.diff(np.concatenate([[0.0], C]))
            assert np.all(cnt >= np.floor(n * w - 1e-9)) and np.all(cnt <= np.ceil(n * w + 1e-9))


# ----------------------------------------------------------------------------- stratified resampling
def test_stratified_offsets_are_the_tag1_words():
    """v_j = uniform word (j mod 4) of Philox(j / 4, t, 1, tracker); v_0 is the systematic u0."""
    seed, t, trk, n = 0x5EED, 7, 3, 11
    v = oracle.stratified_offsets(seed, t, n, trk)
    ctrs = np.array([[j // 4, t, 1, trk] for j in range(n)], np.uint32)
    words = oracle.philox(ctrs, seed)
    want = oracle.uniform(np.array([words[j, j % 4] for j in range(n)], np.uint32))
    assert np.array_equal(v, want)
    assert v[0] == oracle.resample_u0(seed, t, trk)
    assert len(set(v.tolist())) == n


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_stratified_with_equal_offsets_is_systematic(prec):
    """With every v_j = u0 the stratified points are the systematic ones."""
    rng = np.random.default_rng(12)
    for n in (1, 2, 5, 100, 4097):
        e = rng.exponential(size=n) ** 2
        S, _, _ = oracle.normalise(e, np.zeros(n), np.zeros(n))
        C = oracle.cdf(e, S)
        for u0 in (0.125, 0.5, 0.875):
            assert np.array_equal(oracle.resample_stratified(C, np.full(n, u0), prec),
                                  oracle.resample(C, u0, prec))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_stratified_uniform_weights_identity(prec):
    """Equal weights (N a power of two, exact CDF): u_j lies in stratum j's own CDF step."""
    rng = np.random.default_rng(13)
    for n in (1, 2, 8, 1024, 1 << 16):
        C = (np.arange(n, dtype=np.float64) + 1) / n
        v = rng.uniform(0.25, 0.75, n)     # (float)j + v_j stays inside (j, j + 1) in FP32 too
        assert np.array_equal(oracle.resample_stratified(C, v, prec), np.arange(n))


def test_stratified_counts_within_two_strata():
    """Each stratum holds one point, so particle k (CDF step of width w_k) receives between
    N w_k - 2 and N w_k + 2 offspring (exclusive); the ancestors are ordered."""
    rng = np.random.default_rng(14)
    for n in (1, 3, 7, 100, 1000, 4097):
        for trial in range(4):
            e = rng.exponential(size=n) ** 3
            S, _, _ = oracle.normalise(e, np.zeros(n), np.zeros(n))
            C = oracle.cdf(e, S)
            v = oracle.uniform(rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32))
            a = oracle.resample_stratified(C, v, "f64")
            assert np.all(np.diff(a) >= 0) and a.min() >= 0 and a.max() < n
            cnt = _counts(a, n)
            w = np.diff(np.concatenate([[0.0], C]))
            assert cnt.sum() == n
            assert np.all(np.abs(cnt - n * w) < 2.0)


def test_stratified_monte_carlo_expectation():
    """N <= 8: over independent offsets the mean offspring count of particle k is N w_k
    (stratified resampling is unbiased); 20000 draws, 6 standard errors."""
    rng = np.random.default_rng(15)
    trials = 20000
    for n in (2, 3, 5, 8):
        e = rng.uniform(0.01, 1.0, n)
        S, _, _ = oracle.normalise(e, np.zeros(n), np.zeros(n))
        C = oracle.cdf(e, S)
        w = np.diff(np.concatenate([[0.0], C]))
        tot = np.zeros(n)
        sq = np.zeros(n)
        for _ in range(trials):
            c = _counts(oracle.resample_stratified(C, rng.uniform(0.0, 1.0, n), "f64"), n)
            tot += c
            sq += c * c
        mean = tot / trials
        se = np.sqrt(np.maximum(sq / trials - mean ** 2, 1e-12) / trials)
        assert np.all(np.abs(mean - n * w) <= 6 * se + 1e-12)


def test_stratified_dominant_and_clamp():
    C = np.array([0.0, 0.0, 1.0, 1.0])
    assert np.array_equal(oracle.resample_stratified(C, [0.1, 0.9, 0.5, 0.3], "f64"), [2, 2, 2, 2])
    C2 = np.array([0.2, 0.5, 0.9])     # a point above every entry: clamp to N-1
    assert np.array_equal(oracle.resample_stratified(C2, [0.1, 0.2, 0.95], "f64"), [0, 1, 2])
    assert np.array_equal(oracle.resample_stratified(C2, [0.9, 0.6, 0.7], "f64"), [1, 2, 2])


# ----------------------------------------------------------------------------- multinomial resampling
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_multinomial_equal_weights_is_floor_of_n_u(prec):
    """Equal weights, N a power of two (C_k = (k + 1)/N exact): the ancestor of draw v is
    the first step reaching it, ceil(N v) - 1, which is floor(N v) here (a draw is an odd
    multiple of 2^-24, so N v is never an integer)."""
    rng = np.random.default_rng(16)
    for n in (1, 2, 8, 1024, 1 << 16):
        C = (np.arange(n, dtype=np.float64) + 1) / n
        v = oracle.uniform(rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32))
        a = oracle.resample_multinomial(C, v, prec)
        want = np.ceil(v * n).astype(np.int64) - 1       # first k with (k + 1)/N >= v
        assert np.array_equal(a, want) and np.array_equal(want, np.floor(v * n).astype(np.int64))


def test_multinomial_counts_mean_and_variance():
    """Counts of particle k are Binomial(N, w_k): mean N w_k and variance N w_k (1 - w_k)
    over 4000 independent sets of draws (6 standard errors; variance within 15 %)."""
    rng = np.random.default_rng(17)
    n, trials = 6, 4000
    e = rng.uniform(0.05, 1.0, n)
    S, _, _ = oracle.normalise(e, np.zeros(n), np.zeros(n))
    C = oracle.cdf(e, S)
    w = np.diff(np.concatenate([[0.0], C]))
    cnts = np.array([_counts(oracle.resample_multinomial(C, rng.uniform(0.0, 1.0, n), "f64"), n)
                     for _ in range(trials)], np.float64)
    mean, var = cnts.mean(axis=0), cnts.var(axis=0)
    want_var = n * w * (1 - w)
    assert np.all(np.abs(mean - n * w) <= 6 * np.sqrt(want_var / trials))
    assert np.all(np.abs(var / want_var - 1.0) < 0.15)


def test_multinomial_dominant_clamp_and_order():
    C = np.array([0.0, 0.0, 1.0, 1.0])
    assert np.array_equal(oracle.resample_multinomial(C, [0.9, 0.1, 0.5, 1e-6], "f64"), [2, 2, 2, 2])
    C2 = np.array([0.2, 0.5, 0.9])     # a draw above every entry: clamp to N-1
    assert np.array_equal(oracle.resample_multinomial(C2, [0.95, 0.2, 0.21], "f64"), [2, 0, 1])
    # ancestors follow the draws, not the offspring index (no ordering)
    C3 = np.array([0.25, 0.5, 0.75, 1.0])
    assert np.array_equal(oracle.resample_multinomial(C3, [0.9, 0.6, 0.3, 0.1], "f32"), [3, 2, 1, 0])


# ----------------------------------------------------------------------------- Gumbel-max resampling
# The variates are bounded: u lies in [2^-24, 1 - 2^-24], so g = -ln(-ln u) lies in
# [-ln(24 ln 2), -ln(-ln(1 - 2^-24))] = [-2.81, 16.64].
G_LO = -math.log(24 * math.log(2.0))
G_HI = -math.log(-math.log1p(-2.0 ** -24))


def _softmax(L):
    z = np.exp(np.asarray(L, np.float64) - np.max(L))
    return z / z.sum()


def test_gumbel_counts_follow_the_categorical_law():
    """Gumbel-max property: argmax_k (L_k + g_k) is distributed as exp(L_k) / sum exp(L).
    Over 4000 frames of 6 offspring each, the counts of particle k have mean N p_k and
    variance N p_k (1 - p_k) (6 standard errors; variance within 15 %), with p the
    softmax of L computed here by numpy."""
    rng = np.random.default_rng(21)
    n, trials = 6, 4000
    L = rng.uniform(-2.0, 2.0, n)
    p = _softmax(L)
    cnts = np.array([_counts(oracle.resample_gumbel(L, 5, t, 2), n) for t in range(trials)], np.float64)
    mean, var = cnts.mean(axis=0), cnts.var(axis=0)
    want_var = n * p * (1 - p)
    assert np.all(np.abs(mean - n * p) <= 6 * np.sqrt(want_var / trials))
    assert np.all(np.abs(var / want_var - 1.0) < 0.15)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_gumbel_two_particles_closed_form(prec):
    """L = (0, ln 3): particle 1 is drawn with probability 3/4 (binomial, 5 standard
    errors over 2 x 10000 draws); swapping the weights swaps the law."""
    n_frames = 10000
    a = np.concatenate([oracle.resample_gumbel([0.0, math.log(3.0)], 9, t, 0, prec) for t in range(n_frames)])
    se = math.sqrt(0.75 * 0.25 / a.size)
    assert abs(np.mean(a == 1) - 0.75) <= 5 * se
    b = np.concatenate([oracle.resample_gumbel([math.log(3.0), 0.0], 9, t, 0, prec) for t in range(n_frames)])
    assert abs(np.mean(b == 0) - 0.75) <= 5 * se


def test_gumbel_equal_weights_are_uniform():
    """Equal log weights: every particle equally likely (chi-square over 64 particles,
    64 x 200 draws, below the 0.9999 quantile with 63 degrees of freedom)."""
    n, frames = 64, 200
    L = np.full(n, -3.5)
    c = sum(_counts(oracle.resample_gumbel(L, 11, t, 1), n) for t in range(frames)).astype(np.float64)
    expect = frames * np.ones(n)
    chi2 = float(np.sum((c - expect) ** 2 / expect))
    assert chi2 < 116.0                     # chi2_{63}(0.9999) = 115.3


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_gumbel_gap_beyond_the_variate_range_is_deterministic(prec):
    """A particle whose L exceeds every other by more than G_HI - G_LO always wins; one
    below the best by more than that is never drawn."""
    gap = G_HI - G_LO
    L = np.array([0.0, 0.0, gap + 0.05, 0.0, -1.0])
    for t in range(20):
        assert np.all(oracle.resample_gumbel(L, 3, t, 0, prec) == 2)
    L2 = np.array([1.0, 1.0 - gap - 0.05, 0.5, 1.0 - gap - 0.05])
    seen = np.concatenate([oracle.resample_gumbel(L2, 3, t, 0, prec) for t in range(300)])
    assert not np.any((seen == 1) | (seen == 3))
    assert set(np.unique(seen)) == {0, 2}


def test_gumbel_fp32_decisions_agree_with_fp64_outside_near_ties():
    """FP32 decisions equal the FP64 ones except where the two best values of an offspring
    lie within FP32 rounding of each other."""
    rng = np.random.default_rng(22)
    L = np.round(rng.normal(0.0, 3.0, 700), 3)
    for t in range(3):
        a64 = oracle.resample_gumbel(L, 7, t, 0, "f64")
        a32 = oracle.resample_gumbel(L, 7, t, 0, "f32")
        for j in np.nonzero(a64 != a32)[0]:
            g = oracle.gumbel_variates(7, t, int(j), L.size)
            v = L + g
            assert abs(v[a64[j]] - v[a32[j]]) <= 1e-5 * max(1.0, abs(v[a64[j]])), (t, j)
        assert np.mean(a64 == a32) >= 0.999


# ----------------------------------------------------------------------------- Metropolis resampling
def _chain_matrix(L):
    """Transition matrix of one Metropolis step on exp(L): propose k' uniformly (itself
    included), move with probability min(1, exp(L_k' - L_k))."""
    L = np.asarray(L, np.float64)
    n = L.size
    P = np.zeros((n, n))
    for k in range(n):
        for kp in range(n):
            if kp != k:
                P[k, kp] = min(1.0, math.exp(L[kp] - L[k])) / n
        P[k, k] = 1.0 - P[k].sum()
    return P


def test_metropolis_zero_steps_is_identity():
    L = np.array([0.0, 5.0, -3.0, 2.0, 1.0])
    assert np.array_equal(oracle.resample_metropolis(L, 0, 1, 0), np.arange(5))


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("B", [1, 2, 5])
def test_metropolis_small_chains_follow_the_transition_matrix(prec, B):
    """N = 3: offspring j's ancestor after B steps is distributed as row j of P^B, P the
    Metropolis transition matrix (built here from its definition); 6000 frames, every
    entry within 5 binomial standard errors."""
    L = np.array([0.0, math.log(3.0), -0.7])
    PB = np.linalg.matrix_power(_chain_matrix(L), B)
    frames = 6000
    a = np.array([oracle.resample_metropolis(L, B, 13, t, 3, prec) for t in range(frames)])
    for j in range(3):
        freq = np.bincount(a[:, j], minlength=3) / frames
        se = np.sqrt(PB[j] * (1 - PB[j]) / frames)
        assert np.all(np.abs(freq - PB[j]) <= 5 * se + 1e-12), (j, freq, PB[j])


def test_metropolis_long_chains_reach_the_categorical_law():
    """The chain's stationary law is exp(L_k) / sum exp(L): after 200 steps the counts
    over 3000 frames of 5 offspring match the softmax (6 standard errors)."""
    L = np.array([0.0, 1.0, -0.5, 0.7, 0.2])
    p = _softmax(L)
    frames, n = 3000, L.size
    c = sum(_counts(oracle.resample_metropolis(L, 200, 17, t, 0), n) for t in range(frames)).astype(np.float64)
    tot = frames * n
    assert np.all(np.abs(c / tot - p) <= 6 * np.sqrt(p * (1 - p) / tot))


def test_metropolis_equal_weights_take_the_last_proposal():
    """Equal log weights: ln u < 0 accepts every proposal, so the ancestor is uniform over
    the particles whatever the start (chi-square, 0.9999 quantile, 63 dof)."""
    n, frames = 64, 200
    c = sum(_counts(oracle.resample_metropolis(np.full(n, 2.5), 3, 19, t, 0), n) for t in range(frames))
    expect = frames * np.ones(n)
    assert float(np.sum((c - expect) ** 2 / expect)) < 116.0


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_metropolis_dominant_particle_absorbs(prec):
    """One particle far above the rest (which share one log weight): a chain that proposes
    it moves there and never leaves, so a_j is the dominant particle exactly when one of
    the B proposals hits it (or j is it), which happens with probability
    1 - (1 - 1/N)^B."""
    n, B, d = 16, 12, 5
    L = np.full(n, -500.0)
    L[d] = 0.0
    frames = 3000
    a = np.concatenate([oracle.resample_metropolis(L, B, 23, t, 0, prec) for t in range(frames)])
    starts = np.tile(np.arange(n), frames)
    others = starts != d
    p = 1.0 - (1.0 - 1.0 / n) ** B
    se = math.sqrt(p * (1 - p) / others.sum())
    assert abs(np.mean(a[others] == d) - p) <= 5 * se
    assert np.all(a[~others] == d)


def test_metropolis_fp32_decisions_agree_with_fp64():
    rng = np.random.default_rng(25)
    L = np.round(rng.normal(0.0, 2.0, 3000), 3)
    a64 = oracle.resample_metropolis(L, 32, 29, 4, 1, "f64")
    a32 = oracle.resample_metropolis(L, 32, 29, 4, 1, "f32")
    for j in np.nonzero(a64 != a32)[0]:
        _, margins = oracle.metropolis_chain(L, 32, 29, 4, int(j), 1)
        assert min(margins) <= 1e-5, j                 # a near tie in some acceptance test
    assert np.mean(a64 == a32) >= 0.999


# ----------------------------------------------------------------------------- rejection resampling
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_rejection_equal_weights_keep_every_particle(prec):
    """Equal log weights: w_k / w_max = 1 and ln u < 0, so the first candidate (j itself)
    is accepted: the identity."""
    L = np.full(333, -7.25)
    assert np.array_equal(oracle.resample_rejection(L, -7.25, 3, 0, 0, prec), np.arange(333))


def test_rejection_per_offspring_law_and_unbiased_counts():
    """Offspring j keeps j with probability r_j = w_j / w_max at the first try, otherwise
    rejection sampling draws from p = softmax(L): P(a_j = k) = r_j [k = j] + (1 - r_j) p_k
    (checked entry by entry over 4000 frames, 5 binomial standard errors), so the expected
    count of particle k is N p_k (6 standard errors)."""
    rng = np.random.default_rng(31)
    n, trials = 6, 4000
    L = rng.uniform(-2.0, 2.0, n)
    p = _softmax(L)
    r = np.exp(L - L.max())
    a = np.array([oracle.resample_rejection(L, L.max(), 7, t, 1) for t in range(trials)])
    for j in range(n):
        want = (1 - r[j]) * p
        want[j] += r[j]
        freq = np.bincount(a[:, j], minlength=n) / trials
        assert np.all(np.abs(freq - want) <= 5 * np.sqrt(want * (1 - want) / trials) + 1e-12), (j, freq, want)
    cnts = np.array([_counts(row, n) for row in a], np.float64)
    se = np.sqrt(cnts.var(axis=0) / trials)
    assert np.all(np.abs(cnts.mean(axis=0) - n * p) <= 6 * se)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_rejection_two_particles_closed_form(prec):
    """w = (1, 3): offspring 1 passes its first try (w_1 = w_max); offspring 0 keeps itself
    with probability 1/3, else draws particle 1 with probability 3/4, so P(a_0 = 1) = 1/2
    (5 standard errors over 10000 frames)."""
    L = [0.0, math.log(3.0)]
    a = np.array([oracle.resample_rejection(L, max(L), 9, t, 0, prec) for t in range(10000)])
    assert np.all(a[:, 1] == 1)
    assert abs(np.mean(a[:, 0] == 1) - 0.5) <= 5 * math.sqrt(0.25 / a.shape[0])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_rejection_dominant_particle_takes_everything(prec):
    """One particle at the maximum, the rest 1000 below: every other candidate is refused,
    so every offspring ends on the dominant particle (the first proposal hitting it)."""
    n, d = 16, 11
    L = np.full(n, -1000.0)
    L[d] = 0.0
    for t in range(50):
        assert np.all(oracle.resample_rejection(L, 0.0, 5, t, 0, prec) == d)


def test_rejection_truncation_keeps_the_last_candidate():
    """With R tries and no acceptance possible the offspring keeps the last candidate
    (bound M above every weight by far: nothing passes)."""
    L = np.zeros(50)
    a = oracle.resample_rejection(L, 1000.0, 2, 3, 0, "f64", tries=5)
    for j in (0, 13, 49):
        cands, _ = oracle.rejection_trace(L, 1000.0, 2, 3, j, 0, tries=5)
        assert len(cands) == 5 and a[j] == cands[-1]


def test_rejection_fp32_decisions_agree_with_fp64():
    rng = np.random.default_rng(33)
    L = np.round(rng.normal(0.0, 1.5, 3000), 3)
    a64 = oracle.resample_rejection(L, L.max(), 37, 2, 1, "f64")
    a32 = oracle.resample_rejection(L, L.max(), 37, 2, 1, "f32")
    for j in np.nonzero(a64 != a32)[0]:
        _, margins = oracle.rejection_trace(L, L.max(), 37, 2, int(j), 1)
        assert min(margins) <= 1e-5, j
    assert np.mean(a64 == a32) >= 0.999


# ----------------------------------------------------------------------------- propagation, Eq. 1-2
def test_propagation_moments_paper_motion():
    """Eq. 1-2: x ~ N(1 + x_anc, 5^2), y ~ N(2 + y_anc, 2^2)."""
    n = 200000
    x, y = oracle.propagate(n, 4, 9, None, None, None, init=(100.0, 50.0), drift=(1.0, 2.0),
                            sigma=(5.0, 2.0))
    assert abs(x.mean() - 101.0) < 5 * 5.0 / math.sqrt(n)
    assert abs(y.mean() - 52.0) < 5 * 2.0 / math.sqrt(n)
    assert abs(x.std() - 5.0) < 0.05 and abs(y.std() - 2.0) < 0.02


def test_propagation_gathers_ancestors():
    n = 1000
    rng = np.random.default_rng(8)
    xa = rng.uniform(0, 100, n)
    ya = rng.uniform(0, 100, n)
    anc = np.sort(rng.integers(0, n, n))
    x, y = oracle.propagate(n, 2, 5, xa, ya, anc, drift=(0.5, -1.5), sigma=(0.0, 0.0))
    assert np.array_equal(x, xa[anc] + 0.5) and np.array_equal(y, ya[anc] - 1.5)
    # the noise is keyed by (particle, frame): other frames draw other numbers
    x1, _ = oracle.propagate(n, 2, 5, xa, ya, anc, sigma=(1.0, 1.0))
    x2, _ = oracle.propagate(n, 3, 5, xa, ya, anc, sigma=(1.0, 1.0))
    assert not np.allclose(x1, x2)


# ----------------------------------------------------------------------------- whole tracker
def test_track_recovers_ground_truth_config1():
    """128x128, 10 frames, r = 5, noise 5, 1000 particles, sigma 1, seed 1: the FP64 track
    stays within a pixel of the true disk centre (Sec. V, verification)."""
    v = synth.make_video(128, 128, 10, 5, noise=5.0, seed=1)
    est, M, S = oracle.track(v.frames, 1000, 5, init=tuple(v.centres[0]), seed=1)
    err = np.sqrt(np.sum((est - v.centres) ** 2, axis=1))
    assert np.sqrt(np.mean(err ** 2)) < 1.0 and err.max() < 1.5
    assert np.all(S >= 1.0) and np.all(M <= 11648 / 25)


def test_track_stratified_recovers_ground_truth_config1():
    v = synth.make_video(128, 128, 10, 5, noise=5.0, seed=1)
    est, _, _ = oracle.track(v.frames, 1000, 5, init=tuple(v.centres[0]), seed=1, resampler="stratified")
    err = np.sqrt(np.sum((est - v.centres) ** 2, axis=1))
    assert np.sqrt(np.mean(err ** 2)) < 1.0 and err.max() < 1.5
    recs = list(oracle.track_steps(v.frames, 1000, 5, init=tuple(v.centres[0]), seed=1, resampler="stratified"))
    assert np.array_equal(np.array([r.est for r in recs]), est)


def test_track_multinomial_recovers_ground_truth_config1():
    v = synth.make_video(128, 128, 10, 5, noise=5.0, seed=1)
    est, _, _ = oracle.track(v.frames, 1000, 5, init=tuple(v.centres[0]), seed=1, resampler="multinomial")
    err = np.sqrt(np.sum((est - v.centres) ** 2, axis=1))
    assert np.sqrt(np.mean(err ** 2)) < 1.0 and err.max() < 1.5
    recs = list(oracle.track_steps(v.frames, 1000, 5, init=tuple(v.centres[0]), seed=1, resampler="multinomial"))
    assert np.array_equal(np.array([r.est for r in recs]), est)


def test_track_gumbel_recovers_ground_truth_config1():
    v = synth.make_video(128, 128, 10, 5, noise=5.0, seed=1)
    est, _, _ = oracle.track(v.frames, 1000, 5, init=tuple(v.centres[0]), seed=1, resampler="gumbel")
    err = np.sqrt(np.sum((est - v.centres) ** 2, axis=1))
    assert np.sqrt(np.mean(err ** 2)) < 1.0 and err.max() < 1.5
    recs = list(oracle.track_steps(v.frames, 1000, 5, init=tuple(v.centres[0]), seed=1, resampler="gumbel"))
    assert np.array_equal(np.array([r.est for r in recs]), est)


def test_track_metropolis_recovers_ground_truth_config1():
    v = synth.make_video(128, 128, 10, 5, noise=5.0, seed=1)
    est, _, _ = oracle.track(v.frames, 1000, 5, init=tuple(v.centres[0]), seed=1, resampler="metropolis")
    err = np.sqrt(np.sum((est - v.centres) ** 2, axis=1))
    assert np.sqrt(np.mean(err ** 2)) < 1.0 and err.max() < 1.5
    recs = list(oracle.track_steps(v.frames, 1000, 5, init=tuple(v.centres[0]), seed=1, resampler="metropolis"))
    assert np.array_equal(np.array([r.est for r in recs]), est)
    # the chain is the oracle's own: its states, replayed step by step, end at a_j
    L = recs[4].L
    a = oracle.resample_metropolis(L, 64, 1, 4, 0)
    for j in (0, 17, 999):
        states, _ = oracle.metropolis_chain(L, 64, 1, 4, j, 0)
        assert states[-1] == a[j]


def test_track_rejection_recovers_ground_truth_config1():
    v = synth.make_video(128, 128, 10, 5, noise=5.0, seed=1)
    est, _, _ = oracle.track(v.frames, 1000, 5, init=tuple(v.centres[0]), seed=1, resampler="rejection")
    err = np.sqrt(np.sum((est - v.centres) ** 2, axis=1))
    assert np.sqrt(np.mean(err ** 2)) < 1.0 and err.max() < 1.5
    recs = list(oracle.track_steps(v.frames, 1000, 5, init=tuple(v.centres[0]), seed=1, resampler="rejection"))
    assert np.array_equal(np.array([r.est for r in recs]), est)


def test_track_noiseless_recovers_integer_centres():
    v = synth.make_video(128, 128, 12, 5, noise=0.0, seed=2)
    est, _, _ = oracle.track(v.frames, 4000, 5, init=tuple(v.centres[0]), seed=11)
    assert np.array_equal(oracle.round_pixel(est[:, 0]), v.centres[:, 0].astype(np.int64))
    assert np.array_equal(oracle.round_pixel(est[:, 1]), v.centres[:, 1].astype(np.int64))


def test_track_phases_equal_whole_and_thread_count_invariant():
    v = synth.make_video(128, 96, 6, 3, noise=8.0, seed=4, v=(2, 1))
    kw = dict(init=tuple(v.centres[0]), seed=21, tracker=3)
    est1, M1, S1 = oracle.track(v.frames, 5000, 3, nthreads=1, **kw)
    est4, M4, S4 = oracle.track(v.frames, 5000, 3, nthreads=4, **kw)
    assert np.array_equal(est1, est4) and np.array_equal(M1, M4) and np.array_equal(S1, S4)
    recs = list(oracle.track_steps(v.frames, 5000, 3, **kw))
    assert np.array_equal(np.array([r.est for r in recs]), est1)
    assert np.array_equal(np.array([r.M for r in recs]), M1)
