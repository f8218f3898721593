"""Pins of the CPU oracle against values fixed by the workload definitions and by mathematics.

Each test is chosen so that a plausible slip in the oracle (a wrong clamp, an
inclusive instead of exclusive scan, a dropped abs, a swapped channel, a
transposed weight, a rounded instead of floored division) fails it.  None of
them re-types the oracle's own loop: they use hand-worked cases, closed forms,
invariants and independent library routines (scipy.ndimage with edge
replication, numpy.bincount, scipy.stats.norm.cdf, exact rational arithmetic).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import datagen
import oracle
from oracle import mlp

ndimage = pytest.importorskip("scipy.ndimage")


def _read_cases(path):
    cases, cur = {}, None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, _, rest = line.partition(" ")
        if key == "case":
            cur = cases.setdefault(rest, {})
        else:
            cur[key] = np.array([[int(v) for v in row.split()] for row in rest.split("/")], np.uint8)
    return cases


def _read_rows(path):
    return np.array([[int(v) for v in l.split()] for l in open(path)
                     if l.strip() and not l.startswith("#")], np.int64)


# ---------------------------------------------------------------- blur + hist (blur job)

def test_blur_hand_cases(golden_dir):
    # ramp3: every output is a neighbourhood sum that is a multiple of 9, e.g. the corner
    # o[0][0] sees rows (0,0,1) x cols (0,0,1): 2*(0+0+9) + (27+27+36) = 108 -> 12.
    # floor2: o[0][0] sees the 255 twice (dx=+1 on rows -1 and 0, both clamped to 0): 510/9 = 56.7 -> 56;
    # o[0][1] sees it four times: 1020/9 = 113.3 -> 113; o[1][0] once: 28.3 -> 28; o[1][1] twice -> 56.
    for name, c in _read_cases(os.path.join(golden_dir, "blur3x3_hand.txt")).items():
        assert np.array_equal(oracle.blur3x3(c["in"]), c["out"]), name


@pytest.mark.parametrize("c", [0, 1, 128, 255])
def test_blur_constant(c):
    img = np.full((7, 11), c, np.uint8)
    assert np.array_equal(oracle.blur3x3(img), img)


@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (2, 3), (17, 31), (256, 256)])
def test_blur_vs_edge_replicated_correlate(shape):
    img = np.random.default_rng(sum(shape)).integers(0, 256, shape, dtype=np.uint8)
    s = ndimage.correlate(img.astype(np.int64), np.ones((3, 3), np.int64), mode="nearest")
    assert np.array_equal(oracle.blur3x3(img), (s // 9).astype(np.uint8))


def test_hist_bincount_and_total():
    img = datagen.blur_job(3)
    h = oracle.hist256(img)
    assert h.sum() == img.size
    assert np.array_equal(h, np.bincount(img.ravel(), minlength=256).astype(np.uint32))
    hb, _ = oracle.job_blur_hist(img)[1], None
    assert hb.sum() == 65536


def test_blur_job_is_blur_then_hist():
    img = datagen.blur_job(5)
    b, h = oracle.job_blur_hist(img)
    s = ndimage.correlate(img.astype(np.int64), np.ones((3, 3), np.int64), mode="nearest") // 9
    assert np.array_equal(b, s.astype(np.uint8))
    assert np.array_equal(h, np.bincount(b.ravel(), minlength=256).astype(np.uint32))


# ---------------------------------------------------------------- saxpy / scan / max (scan job)

def test_saxpy_special_cases():
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, 1000).astype(np.float32)
    y = rng.uniform(-1, 1, 1000).astype(np.float32)
    assert np.array_equal(oracle.saxpy(0.0, x, y), y)
    assert np.array_equal(oracle.saxpy(1.0, x, -x), np.zeros_like(x))
    assert np.array_equal(oracle.saxpy(-1.0, x, x), np.zeros_like(x))


def _nearest_f32(q: Fraction) -> np.float32:
    """fp32 nearest to the exact rational q (ties to even), found by bracketing."""
    f = np.float32(float(q))
    best = f
    for cand in (np.nextafter(f, np.float32(-np.inf)), np.nextafter(f, np.float32(np.inf))):
        dc, db = abs(Fraction(float(cand)) - q), abs(Fraction(float(best)) - q)
        if dc < db or (dc == db and (cand.view(np.uint32) & 1) == 0):
            best = cand
    return best


def test_saxpy_is_single_rounding_fma():
    # z must be the fp32 value nearest to the exact a*x + y (one rounding), which a
    # separately rounded multiply-then-add misses on a fraction of inputs.
    a, xy = datagen.scan_job(0, n=4096)
    x, y = xy[:4096], xy[4096:]
    z = oracle.saxpy(a, x, y)
    two_roundings_differ = 0
    for i in range(0, 4096, 7):
        exact = Fraction(float(np.float32(a))) * Fraction(float(x[i])) + Fraction(float(y[i]))
        assert z[i] == _nearest_f32(exact), i
        two_roundings_differ += int(np.float32(np.float32(a) * x[i]) + y[i] != z[i])
    assert two_roundings_differ > 0  # the check above can tell fma from mul+add


def test_exscan_hand_and_closed_forms():
    S, A = oracle.exscan(np.array([1, 2, 3, 4, 5], np.float32))
    assert S.tolist() == [0, 1, 3, 6, 10]
    assert A.tolist() == [0, 1, 3, 6, 10]
    S, A = oracle.exscan(np.array([3, -10, 4], np.float32))
    assert S.tolist() == [0, 3, -7] and A.tolist() == [0, 3, 13]
    assert oracle.maxabs(S) == 7.0  # |-7|, not max(S) = 3
    n = 1 << 16
    S, A = oracle.exscan(np.ones(n, np.float32))
    assert np.array_equal(S, np.arange(n, dtype=np.float64))
    assert oracle.maxabs(S) == n - 1


def test_exscan_total_and_differences():
    a, xy = datagen.scan_job(1)
    z, S, A, m = oracle.job_saxpy_scan_max(a, xy[:65536], xy[65536:])
    total = math.fsum(float(v) for v in z)  # exactly rounded sum
    assert abs(S[-1] + float(z[-1]) - total) <= 1e-12 * A[-1] + 1e-300
    assert S[0] == 0.0
    d = np.diff(S) - z[:-1].astype(np.float64)
    assert np.max(np.abs(d)) <= 1e-12 * max(A[-1], 1.0)
    assert m == np.max(np.abs(S))
    assert np.array_equal(z, oracle.saxpy(a, xy[:65536], xy[65536:]))


# ---------------------------------------------------------------- gray / gauss / sobel (img job)

def test_gray_channels():
    px = np.array([[[255, 0, 0], [0, 255, 0], [0, 0, 255], [255, 255, 255], [0, 0, 0], [7, 7, 7]]], np.uint8)
    # (77*255)>>8 = 76, (150*255)>>8 = 149, (29*255)>>8 = 28; R=G=B=c -> c since 77+150+29 = 256
    assert oracle.gray(px).tolist() == [[76, 149, 28, 255, 0, 7]]


def test_gauss_impulse(golden_dir):
    g = np.zeros((9, 9), np.uint8)
    g[4, 4] = 255
    want = np.zeros((9, 9), np.int64)
    want[2:7, 2:7] = _read_rows(os.path.join(golden_dir, "gauss5_impulse.txt"))
    assert np.array_equal(oracle.gauss5(g), want.astype(np.uint8))


def test_gauss_constant_and_ramp():
    assert np.array_equal(oracle.gauss5(np.full((6, 9), 77, np.uint8)), np.full((6, 9), 77, np.uint8))
    ramp = np.tile(np.arange(40, dtype=np.uint8), (8, 1))
    q = oracle.gauss5(ramp)
    assert np.array_equal(q[:, 2:-2], ramp[:, 2:-2])  # symmetric kernel preserves a linear ramp


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (5, 1), (3, 4), (23, 19), (64, 130)])
def test_gauss_sobel_vs_edge_replicated_correlate(shape):
    rng = np.random.default_rng(shape[0] * 1000 + shape[1])
    g = rng.integers(0, 256, shape, dtype=np.uint8)
    w = np.array([1, 4, 6, 4, 1], np.int64)
    q_ref = ndimage.correlate(g.astype(np.int64), np.outer(w, w), mode="nearest") >> 8
    q = oracle.gauss5(g)
    assert np.array_equal(q, q_ref.astype(np.uint8))
    kx = np.array([[-1, 0, 1], [-2, 0, 2], [-1, 0, 1]], np.int64)
    gx = ndimage.correlate(q.astype(np.int64), kx, mode="nearest")
    gy = ndimage.correlate(q.astype(np.int64), kx.T, mode="nearest")
    assert np.array_equal(oracle.sobel(q), np.minimum(np.abs(gx) + np.abs(gy), 255).astype(np.uint8))


def test_sobel_hand_and_special(golden_dir):
    q = np.tile(np.array([0, 0, 10, 10], np.uint8), (4, 1))
    want = _read_rows(os.path.join(golden_dir, "sobel_step.txt"))
    assert np.array_equal(oracle.sobel(q), np.tile(want, (4, 1)).astype(np.uint8))
    assert np.array_equal(oracle.sobel(q.T.copy()), np.tile(want, (4, 1)).T.astype(np.uint8))  # gy
    assert not oracle.sobel(np.full((5, 6), 200, np.uint8)).any()  # constant -> 0
    step = np.tile(np.array([0, 0, 100, 100], np.uint8), (3, 1))  # |gx| = 400 -> clamped
    assert oracle.sobel(step)[1].tolist() == [0, 255, 255, 0]
    ramp = np.tile(np.arange(12, dtype=np.uint8), (5, 1))  # interior 8, borders 4
    assert oracle.sobel(ramp)[2].tolist() == [4] + [8] * 10 + [4]


def test_img_job_chain_and_hist():
    rgb = datagen.img_job(0, dims=(37, 29))
    s, h = oracle.job_img_sobel_hist(rgb)
    assert np.array_equal(s, oracle.sobel(oracle.gauss5(oracle.gray(rgb))))
    assert h.sum() == 37 * 29
    assert np.array_equal(h, np.bincount(s.ravel(), minlength=256).astype(np.uint32))


def test_img_all_same_gray_gives_zero_sobel():
    rgb = np.zeros((11, 13, 3), np.uint8)
    rgb[...] = (10, 200, 30)
    s, h = oracle.job_img_sobel_hist(rgb)
    assert not s.any() and h[0] == 11 * 13


# ---------------------------------------------------------------- MLP + LayerNorm (mlp job)

def test_gelu_textbook_values():
    from scipy.stats import norm
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert math.isclose(mlp.gelu(np.array([1.0]))[0], 0.8413447460685429, rel_tol=1e-15)
    assert math.isclose(mlp.gelu(np.array([-1.0]))[0], -0.15865525393145705, rel_tol=1e-14)
    v = np.linspace(-6, 6, 1001)
    assert np.allclose(mlp.gelu(v), v * norm.cdf(v), rtol=1e-13, atol=1e-16)  # GELU(v) = v Phi(v)


def test_layernorm_closed_forms():
    assert not mlp.layernorm(np.full((2, 1024), 3.25)).any()  # constant row -> 0
    alt = np.tile([1.0, -1.0], (1, 512))
    assert np.allclose(mlp.layernorm(alt), alt / math.sqrt(1 + 1e-5), rtol=1e-14)
    k = np.arange(1024, dtype=np.float64)[None]
    var = (1024 ** 2 - 1) / 12.0
    assert np.allclose(mlp.layernorm(k), (k - 511.5) / math.sqrt(var + 1e-5), rtol=1e-12)
    sh = mlp.layernorm(k * 3.0 + 11.0)  # affine invariance up to eps
    assert np.allclose(sh, (k - 511.5) / math.sqrt(var + 1e-5 / 9), rtol=1e-12)


def test_mlp_hand_case(golden_dir):
    vals = dict(l.split() for l in open(os.path.join(golden_dir, "mlp_hand.txt")) if not l.startswith("#"))
    g1, gm1 = float(vals["g1"]), float(vals["gm1"])
    x = np.array([[1, 0, 0], [0, 1, -1]], np.float64)
    w1 = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], np.float64)
    w2 = np.array([[1, 0, 0, 0], [0, 1, 0, 1], [0, 0, 2, -1]], np.float64)
    s0, s1 = math.sqrt(2 / 9 + 1e-5), math.sqrt(2 / 3 + 1e-5)
    want = np.array([[g1 + (2 / 3) / s0, g1 - (1 / 3) / s0, -g1 - (1 / 3) / s0],
                     [0.0, g1 + 1 / s1, 2 * gm1 - 1 / s1]])
    assert np.allclose(mlp.mlp_ln(x, w1, w2), want, rtol=1e-14, atol=1e-15)


def test_mlp_identity_weights_reduce_to_gelu_plus_ln():
    from scipy.stats import norm
    x_b = datagen.mlp_job(0, m=5)
    x = datagen.bf16_to_f32(x_b).astype(np.float64)
    w1 = np.zeros((4096, 1024)); w1[:1024, :1024] = np.eye(1024)
    w2 = np.zeros((1024, 4096)); w2[:, :1024] = np.eye(1024)
    got = mlp.mlp_ln(x, w1, w2)
    mu = x.mean(1, keepdims=True)
    sd = np.sqrt(((x - mu) ** 2).sum(1, keepdims=True) / 1024 + 1e-5)
    assert np.allclose(got, x * norm.cdf(x) + (x - mu) / sd, rtol=1e-12, atol=1e-12)


def test_mlp_job_bf16_widening_is_exact():
    x_b = datagen.mlp_job(2, m=3)
    w1, w2 = datagen.mlp_weights(d=8, f=16)
    out = oracle.job_mlp_ln(x_b[:, :8].copy(), w1, w2)
    x = datagen.bf16_to_f32(x_b[:, :8]).astype(np.float64)
    assert out.shape == (3, 8) and np.isfinite(out).all()
    assert np.allclose(out, mlp.mlp_ln(x, datagen.bf16_to_f32(w1), datagen.bf16_to_f32(w2)), rtol=1e-15)


# ---- hotspot job: compact thermal RC grid, K explicit Euler steps ----

def _hot_physics(R, C):
    # die 16 mm x 16 mm x 0.5 mm, k = 100 W/(m K), c_v = 1.75e6 J/(m^3 K): slab conductances
    dx, dy, t, k = 0.016 / C, 0.016 / R, 0.0005, 100.0
    return dict(gx=k * t * dy / dx, gy=k * t * dx / dy, gz=k * dx * dy / t, cap=1.75e6 * t * dx * dy)


@pytest.mark.parametrize("R,C", [(5, 7), (512, 512), (64, 300)])
def test_hotspot_params_are_the_slab_conductances(R, C):
    p, ph = oracle.hotspot_params(R, C), _hot_physics(R, C)
    for key in ("gx", "gy", "gz", "cap"):
        assert p[key] == pytest.approx(ph[key], rel=1e-14), key
    # the step is a fifth of the positivity limit of the explicit scheme
    assert p["dt"] * (2 * p["gx"] + 2 * p["gy"] + p["gz"]) / p["cap"] == pytest.approx(0.2, rel=1e-14)
    assert p["t_amb"] == 80.0


def test_hotspot_equilibrium_is_fixed():
    T0 = np.full((6, 9), 80.0, np.float32)
    T = oracle.hotspot(T0, np.zeros_like(T0), 7)
    assert np.array_equal(T, np.full((6, 9), 80.0))


@pytest.mark.parametrize("R,C,K", [(6, 9, 5), (3, 1, 11), (1, 1, 4)])
def test_hotspot_uniform_fields_closed_form(R, C, K):
    # a uniform field never has lateral flux (adiabatic edges), so each cell follows the scalar
    # recurrence x' = x + dt/Cap (p - Gz x) with x = T - T_amb:
    #   x_K = (1 - a)^K x_0 + (p / Gz) (1 - (1 - a)^K),  a = dt Gz / Cap
    ph = _hot_physics(R, C)
    p = oracle.hotspot_params(R, C)
    a = p["dt"] * ph["gz"] / ph["cap"]
    for T0v, Pv in ((90.0, 0.0), (80.0, 1e-3), (84.5, 3e-4)):
        T0 = np.full((R, C), T0v, np.float32)
        P = np.full((R, C), Pv, np.float32)
        x0, pw = float(np.float32(T0v)) - 80.0, float(np.float32(Pv))
        xK = (1 - a) ** K * x0 + pw / ph["gz"] * (1 - (1 - a) ** K)
        assert np.allclose(oracle.hotspot(T0, P, K), 80.0 + xK, rtol=0, atol=1e-12)


def _path_laplacian(n):
    A = np.eye(n, k=1) + np.eye(n, k=-1)
    return np.diag(A.sum(axis=1)) - A


@pytest.mark.parametrize("R,C,K", [(5, 7, 4), (1, 6, 3), (8, 1, 2), (4, 4, 6)])
def test_hotspot_matches_graph_laplacian_iteration(R, C, K):
    # the same model as a linear map on the flattened grid: lateral coupling through the
    # Laplacians of the row and column path graphs (no edges leave the die = adiabatic edges),
    # T' = T + dt/Cap (P - (Gx Lx + Gy Ly) T - Gz (T - T_amb)).  Non-square cells make Gx != Gy,
    # so a transposed neighbour or a swapped conductance fails.
    rng = np.random.default_rng(R * 100 + C)
    T0 = rng.uniform(80, 90, (R, C)).astype(np.float32)
    P = rng.uniform(0, 1e-3, (R, C)).astype(np.float32)
    ph = _hot_physics(R, C)
    dt = oracle.hotspot_params(R, C)["dt"]
    Lx = np.kron(np.eye(R), _path_laplacian(C))
    Ly = np.kron(_path_laplacian(R), np.eye(C))
    M = ph["gx"] * Lx + ph["gy"] * Ly
    T = T0.astype(np.float64).ravel()
    for _ in range(K):
        T = T + dt / ph["cap"] * (P.astype(np.float64).ravel() - M @ T - ph["gz"] * (T - 80.0))
    assert np.allclose(oracle.hotspot(T0, P, K).ravel(), T, rtol=0, atol=1e-10)


def test_hotspot_heat_balance_and_max_principle():
    # lateral flux only moves heat between cells: sum(T - T_amb) follows the scalar recurrence of
    # a single cell driven by the total power; and with P = 0 the scheme (coefficients positive,
    # summing to at most one) keeps every value inside the range of T0 and T_amb
    R, C, K = 37, 53, 9
    rng = np.random.default_rng(7)
    T0 = rng.uniform(80, 90, (R, C)).astype(np.float32)
    P = rng.uniform(0, 1e-3, (R, C)).astype(np.float32)
    ph = _hot_physics(R, C)
    a = oracle.hotspot_params(R, C)["dt"] * ph["gz"] / ph["cap"]
    b = oracle.hotspot_params(R, C)["dt"] / ph["cap"]
    s = float((T0.astype(np.float64) - 80.0).sum())
    for _ in range(K):
        s = (1 - a) * s + b * float(P.astype(np.float64).sum())
    T = oracle.hotspot(T0, P, K)
    assert (T - 80.0).sum() == pytest.approx(s, rel=1e-11)
    T = oracle.hotspot(T0, np.zeros_like(P), K)
    assert T.min() >= 80.0 and T.max() <= float(T0.max())
