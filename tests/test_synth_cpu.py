"""The seeded input recipe (Sec. 5.1 random walks, Sec. 5.3 noisy members):
what the generators draw matches the recipe stated for every workload."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


def test_random_walks_recipe_and_determinism():
    raw = synth.random_walks(400, 256, seed=3, znorm=False).astype(np.float64)
    steps = np.diff(raw, axis=1)
    assert abs(steps.mean()) < 0.01 and abs(steps.std() - 1.0) < 0.01       # x_t = x_{t-1} + N(0, 1)
    assert abs(raw[:, 0].std() - 1.0) < 0.1                                    # x_0 ~ N(0, 1)
    z = synth.random_walks(400, 256, seed=3)
    assert z.dtype == np.float32 and z.shape == (400, 256)
    assert np.max(np.abs(z.astype(np.float64).mean(axis=1))) < 1e-5          # z-normalised rows
    assert np.max(np.abs(z.astype(np.float64).std(axis=1) - 1.0)) < 1e-5     # population std
    assert np.array_equal(z, synth.random_walks(400, 256, seed=3))
    assert not np.array_equal(z, synth.random_walks(400, 256, seed=4))


def test_noisy_members_add_the_stated_noise():
    data = synth.random_walks(1000, 128, seed=5)
    for sigma in (0.1, 0.5, 1.0):
        q, ids = synth.noisy_members(data, 200, sigma, seed=6)
        assert q.shape == (200, 128) and ids.min() >= 0 and ids.max() < 1000
        noise = q.astype(np.float64) - data[ids].astype(np.float64)
        assert abs(noise.std() - sigma) < 0.02 * sigma                        # not re-normalised
        assert abs(noise.mean()) < 0.02 * sigma


def test_query_mix_proportions():
    data = synth.random_walks(1000, 64, seed=8)
    q = synth.query_mix(data, 11, seed=9)
    assert q.shape == (11, 64)
    fresh = synth.random_walks(5, 64, seed=9)
    assert np.array_equal(q[:5], fresh)                                        # half fresh walks
    # the rest: 2 + 2 + 2 noisy members at sigma 0.1, 0.5, 1.0
    for i, (lo, hi, s) in enumerate(((5, 7, 0.1), (7, 9, 0.5), (9, 11, 1.0))):
        ref, _ = synth.noisy_members(data, hi - lo, s, seed=synth.NOISE_SEED + i)
        assert np.array_equal(q[lo:hi], ref)


def test_torch_back_end_same_recipe():
    z = synth.random_walks_torch(300, 128, seed=10, device="cpu", chunk=128)
    assert z.dtype == torch.float32 and tuple(z.shape) == (300, 128)
    zz = z.double()
    assert float(zz.mean(dim=1).abs().max()) < 1e-5
    assert float((zz.std(dim=1, unbiased=False) - 1.0).abs().max()) < 1e-5
    assert torch.equal(z, synth.random_walks_torch(300, 128, seed=10, device="cpu", chunk=128))
    q = synth.query_mix_torch(z, 9)
    assert tuple(q.shape) == (9, 128)
    noisy, ids = synth.noisy_members_torch(z, 50, 0.5)
    noise = (noisy - z[ids]).double()
    assert abs(float(noise.std()) - 0.5) < 0.02
