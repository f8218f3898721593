"""The seeded input generators: published SplitMix64 outputs, ranges, exactness, determinism."""
import numpy as np

import datagen


def test_splitmix64_published_outputs():
    # SplitMix64 (Steele, Lea, Flood 2014) started at state 0: first outputs.
    assert datagen.rand(0, 0) == 0xE220A8397B1DCDAF
    assert datagen.rand(0, 1) == 0x6E789E6AA1B965F4
    assert datagen.rand(0, 2) == 0x06C45D188009454F


def test_uniform_ranges_and_exactness():
    a, xy = datagen.scan_job(7)
    assert -2.0 <= a < 2.0
    assert xy.dtype == np.float32 and xy.size == 2 * 65536
    assert xy.min() >= -1.0 and xy.max() < 1.0
    k = (xy.astype(np.float64) + 1.0) * 2 ** 23  # k * 2^-23 - 1 with k a 24-bit integer
    assert np.array_equal(k, np.round(k)) and k.min() >= 0 and k.max() < 2 ** 24
    assert abs(float(xy.mean())) < 0.01


def test_image_and_mlp_shapes():
    dims = [datagen.img_dims(j) for j in range(2000)]
    assert all(128 <= w <= 2048 and 128 <= h <= 2048 for w, h in dims)
    lw = np.log([w for w, _ in dims])
    assert abs(lw.mean() - (np.log(128) + np.log(2048)) / 2) < 0.05  # log-uniform midpoint
    ms = [datagen.mlp_rows(j) for j in range(3000)]
    assert min(ms) == 1 and max(ms) == 256
    x = datagen.bf16_to_f32(datagen.mlp_job(0, m=64))
    assert abs(x.mean()) < 0.02 and abs(x.std() - 1) < 0.02


def test_determinism_and_independence():
    assert np.array_equal(datagen.blur_job(4), datagen.blur_job(4))
    assert not np.array_equal(datagen.blur_job(4), datagen.blur_job(5))
    t1, k1, _ = datagen.serve_trace(1000.0, 500)
    t2, k2, _ = datagen.serve_trace(1000.0, 500)
    assert np.array_equal(t1, t2) and np.array_equal(k1, k2)
    assert set(np.unique(k1)) <= {1, 3, 4}


def test_hotspot_inputs_ranges_and_determinism():
    a = datagen.hot_job(11, 40, 70)
    b = datagen.hot_job(11, 40, 70)
    c = datagen.hot_job(12, 40, 70)
    assert a.dtype == np.float32 and a.size == 2 * 40 * 70
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    T0, P = a[:2800], a[2800:]
    assert T0.min() >= 80.0 and T0.max() < 90.0 and abs(float(T0.mean()) - 85.0) < 0.3
    assert P.min() >= 0.0 and P.max() < 1e-3 and abs(float(P.mean()) - 5e-4) < 3e-5
