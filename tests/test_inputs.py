"""The seeded input generators shared by the oracle and the CUDA path (they hold none of the
method's arithmetic): determinism, shapes and the distributions the input recipe states."""
import numpy as np
import pytest

import oracle
from paper_2605_02726_gb300 import inputs


@pytest.mark.parametrize("H,W", [(1, 1), (7, 5), (512, 768), (1365, 2048), (16384, 3)])
def test_grid_shapes_are_ceil_halvings_and_match_the_oracle(H, W):
    shapes = inputs.grid_shapes(H, W)
    assert len(shapes) == 7
    for k, (h, w) in enumerate(shapes):
        assert (h, w) == (-(-H // 2 ** k), -(-W // 2 ** k))
    assert inputs.latent_count(H, W) == sum(h * w for h, w in shapes) == oracle.latent_count(H, W)
    assert [tuple(s) for s in oracle.grid_shapes(H, W)] == [tuple(s) for s in shapes]


def test_parameter_layout_is_contiguous_and_1415_long():
    o = 0
    for name, shape in inputs.PARAM_BLOCKS:
        assert inputs.PARAM_OFFSETS[name] == (o, shape)
        o += int(np.prod(shape))
    assert o == inputs.N_PARAMS == 1415


def test_image_is_seeded_in_range_with_a_1_over_f2_spectrum():
    a = inputs.image(256, 384, seed=4)
    assert a.shape == (3, 256, 384) and a.dtype == np.float32
    assert np.array_equal(a, inputs.image(256, 384, seed=4))
    assert not np.array_equal(a, inputs.image(256, 384, seed=5))
    assert a.min() >= 0.0 and a.max() <= 1.0
    for c in range(3):  # min-max scaled per channel
        assert a[c].min() == 0.0 and a[c].max() == 1.0
    # radially averaged power falls as f^-2: slope of log power against log f near -2
    p = np.abs(np.fft.rfft2(a[0] - a[0].mean())) ** 2
    fy = np.fft.fftfreq(256)[:, None]
    fx = np.fft.rfftfreq(384)[None, :]
    f = np.sqrt(fy * fy + fx * fx)
    bins = np.geomspace(0.01, 0.4, 12)
    logf, logp = [], []
    for lo, hi in zip(bins[:-1], bins[1:]):
        m = (f >= lo) & (f < hi)
        logf.append(np.log(np.sqrt(lo * hi)))
        logp.append(np.log(p[m].mean()))
    slope = np.polyfit(logf, logp, 1)[0]
    assert -2.3 < slope < -1.7


def test_texture_noise_is_added_to_the_same_field_and_clipped():
    a = inputs.image(128, 128, seed=1)
    b = inputs.image(128, 128, seed=1, texture_sigma=0.02)
    assert b.min() >= 0.0 and b.max() <= 1.0
    # channel 0 is the same field plus N(0, 0.02^2) (the later channels draw after the noise)
    d = (b[0] - a[0]).astype(np.float64)
    assert 0.015 < d.std() < 0.025 and abs(d.mean()) < 0.005


def test_initial_state_recipe():
    lat, par = inputs.initial_state(512, 768, seed=2)
    assert lat.shape == (inputs.latent_count(512, 768),) and par.shape == (1415,)
    assert lat.dtype == np.float32 and par.dtype == np.float32
    assert abs(lat.std() - 0.01) < 1e-4 and abs(lat.mean()) < 1e-4
    hidden = {"arm.w1", "arm.w2", "ifce0.w", "ifce1.w", "ifce2.w", "syn.w1"}
    for name, shape in inputs.PARAM_BLOCKS:
        v = inputs.block(par, name)
        if name in hidden:
            bound = 1.0 / np.sqrt(shape[1])
            assert np.all(np.abs(v) <= bound) and np.abs(v).max() > 0.5 * bound, name
        elif name == "up.taps":
            assert np.array_equal(v, np.tile(np.array(inputs.BICUBIC_TAPS, np.float32), (6, 1)))
        else:
            assert not np.any(v), name
    lat2, par2 = inputs.initial_state(512, 768, seed=2)
    assert np.array_equal(lat, lat2) and np.array_equal(par, par2)


def test_random_state_exercises_every_block():
    _, par = inputs.random_state(40, 56, seed=3)
    for name, _ in inputs.PARAM_BLOCKS:
        assert np.any(inputs.block(par, name)), name


def test_batch_and_serving_workloads():
    sizes = inputs.batch_workload(32)
    assert len(sizes) == 32 and set(sizes) <= set(inputs.BATCH_SIZES)
    assert sizes == inputs.batch_workload(32)
    reqs = inputs.serve_requests(8.0, 200)
    t = np.array([r[0] for r in reqs])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0.0)
    assert 0.8 / 8.0 < np.diff(t).mean() < 1.25 / 8.0  # Poisson arrivals at 8 per second
    assert {r[1] for r in reqs} <= set(inputs.SERVE_SIZES)
    assert {r[2] for r in reqs} <= set(inputs.SERVE_LAMBDAS)
