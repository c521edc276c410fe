"""The drifting trajectory (host definition in synth, device copy in bench):
frame 0 is the static thermal frame, the walk accumulates with the stated
step, and both generators draw from the same distribution."""
import numpy as np
import pytest

import synth


def _mi(d, box):
    return d - box * np.round(d / box)


@pytest.fixture(scope="module")
def small():
    return synth.wurtzite_system(3000, cfg=3)


def test_frame_zero_is_the_static_thermal_frame(small):
    f0 = next(synth.drift_trajectory(small, 1))
    assert np.array_equal(f0, synth.perturbed_frame(small, 0))


def test_walk_accumulates_with_the_stated_step(small):
    box = np.asarray(small.box)
    frames = list(synth.drift_trajectory(small, 17, step_sigma=0.02, sigma=0.0))
    base = small.base[:, :3].astype(np.float64)
    # sigma = 0: frame f - base is the walk W_f, of variance f step^2 per coordinate
    for f in (1, 4, 16):
        w = _mi(frames[f][:, :3].astype(np.float64) - base, box)
        assert np.std(w) == pytest.approx(0.02 * np.sqrt(f), rel=0.05)
    # successive increments are independent
    d1 = _mi(frames[2][:, :3].astype(np.float64) - frames[1][:, :3], box)
    d2 = _mi(frames[3][:, :3].astype(np.float64) - frames[2][:, :3], box)
    assert abs(np.corrcoef(d1.ravel(), d2.ravel())[0, 1]) < 0.05
    assert np.array_equal(frames[5][:, 3], small.base[:, 3])
    assert np.all(frames[16][:, :3] >= 0) and np.all(frames[16][:, :3] < box.astype(np.float32))


def test_device_generator_draws_from_the_same_distribution(small):
    torch = pytest.importorskip("torch")
    import bench
    box = np.asarray(small.box)
    out = bench.device_drift_frames(small, 9, 0.02, 0.05, torch.device("cpu"), seed=7).numpy()
    assert out.shape == (9, small.n, 4) and out.dtype == np.float32
    base = small.base[:, :3].astype(np.float64)
    host = list(synth.drift_trajectory(small, 9, step_sigma=0.02, sigma=0.05))
    for f in (0, 8):
        dev_std = np.std(_mi(out[f, :, :3].astype(np.float64) - base, box))
        host_std = np.std(_mi(host[f][:, :3].astype(np.float64) - base, box))
        want = np.sqrt(f * 0.02 ** 2 + 0.05 ** 2)
        assert dev_std == pytest.approx(want, rel=0.05) and host_std == pytest.approx(want, rel=0.05)
    assert np.array_equal(out[3, :, 3], small.base[:, 3])
    assert np.all(out[:, :, :3] >= 0) and np.all(out[:, :, :3] < box.astype(np.float32))


def test_served_arrivals_streams():
    arr, wof = synth.served_arrivals(5, 32, 4000, 10000.0, seed=1)
    assert np.all(np.diff(arr) >= 0) and np.mean(np.diff(arr)) == pytest.approx(1e-4, rel=0.05)
    assert wof.min() >= 0 and wof.max() < 32 and len(np.unique(wof)) == 32
    arr2, wof2 = synth.served_arrivals(5, 32, 4000, 10000.0, seed=2)
    assert not np.array_equal(arr, arr2) and not np.array_equal(wof, wof2)
    burst, _ = synth.served_arrivals(5, 32, 100, float("inf"), seed=3)
    assert np.all(burst == 0.0)
    # the walkers (sizes) are the served trace's whatever the stream
    n, _, _ = synth.served_trace(5, n_walkers=32, n_requests=10)
    assert n.shape == (32,)
