"""Host-side pieces of the serving form (no GPU): the open-loop Poisson
request schedule -- arrival statistics, the level mix, per-level sample ids,
per-request seeds and stimulus centres -- and its determinism."""
import numpy as np

from paper_1911_06066_gb300 import serving as S


def test_poisson_arrivals_rate_and_mix():
    n, rate = 20000, 2000.0
    mix = [0.75, 0.2, 0.05]
    t, levels, seeds, ids, stim = S.poisson_schedule(rate, n, mix, rng_seed=3)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and np.all(np.diff(t) > 0)
    # exponential inter-arrival times: mean 1/rate, coefficient of variation 1
    assert abs(gaps.mean() * rate - 1.0) < 0.03
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05
    frac = np.bincount(levels, minlength=3) / n
    assert np.all(np.abs(frac - mix) < 4 * np.sqrt(np.asarray(mix) * (1 - np.asarray(mix)) / n))
    # sample ids count up per level, so no (level, id) pair repeats
    for l in range(3):
        assert np.array_equal(ids[levels == l], np.arange((levels == l).sum()))
    assert np.all(seeds == 0) and stim is None


def test_per_request_seeds_and_stimulus_box():
    t, levels, seeds, ids, stim = S.poisson_schedule(500.0, 4000, [0.5, 0.5], rng_seed=1,
                                                     per_request_seed=True, stim_box=(0.0, 0.2))
    assert seeds.dtype == np.uint64 and len(np.unique(seeds)) == len(seeds)
    assert stim.shape == (4000, 3) and np.all(stim[:, 2] == 0.0)
    assert np.all((stim[:, :2] >= 0.0) & (stim[:, :2] < 0.2))
    assert abs(stim[:, :2].mean() - 0.1) < 0.005


def test_schedule_is_reproducible():
    a = S.poisson_schedule(100.0, 300, [0.3, 0.7], rng_seed=9, per_request_seed=True,
                           stim_box=(0.0, 0.2), dim=3)
    b = S.poisson_schedule(100.0, 300, [0.3, 0.7], rng_seed=9, per_request_seed=True,
                           stim_box=(0.0, 0.2), dim=3)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.all(a[4][:, 2] >= 0.0) and np.any(a[4][:, 2] > 0.0)
