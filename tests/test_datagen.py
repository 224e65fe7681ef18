"""The seeded input generators: shapes, determinism and the stated recipes."""
import numpy as np

from paper_2006_06743_gb300 import datagen


def test_mixture_2d_recipe():
    x = datagen.mixture_2d(10_000, seed=0)
    assert x.shape == (10_000, 2) and x.dtype == np.float32
    np.testing.assert_array_equal(x, datagen.mixture_2d(10_000, seed=0))
    assert not np.array_equal(x, datagen.mixture_2d(10_000, seed=1))


def test_gaussian_mixture_siblings_share_distribution():
    a, ta = datagen.gaussian_mixture(5000, 8, 10, 0.03, seed=1, master_seed=42,
                                     return_truth=True)
    b, tb = datagen.gaussian_mixture(5000, 8, 10, 0.03, seed=2, master_seed=42,
                                     return_truth=True)
    assert not np.array_equal(a, b)
    assert (ta < 0).sum() == (tb < 0).sum() == 150
    # same centres: per-component means agree
    for k in range(10):
        if (ta == k).sum() > 50 and (tb == k).sum() > 50:
            assert np.abs(a[ta == k].mean(0) - b[tb == k].mean(0)).max() < 0.5


def test_sphere_embeddings_unit_norm():
    x = datagen.sphere_embeddings(3000, 16, 10, 0.05, seed=3)
    np.testing.assert_allclose(np.linalg.norm(x, axis=1), 1.0, atol=1e-5)


def test_point_clouds_offsets():
    x, off = datagen.point_clouds(5, seed=0, n_min=200, n_max=500)
    assert off[0] == 0 and off[-1] == x.shape[0] and x.shape[1] == 4
    sizes = np.diff(off)
    assert (sizes >= 200).all() and (sizes <= 500).all()
    assert (x[:, 3] == 0).all()


def test_eps_quantile_nearest_rank():
    x = np.arange(10, dtype=np.float32).reshape(-1, 1)
    e = datagen.eps_quantile(x, q=0.5, n_pairs=10_000, seed=0)
    assert 2.0 <= e <= 4.0


def test_bf16_round_ties_even():
    v = np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-8, -2.5, np.inf, 3.0e38], dtype=np.float32)
    r = datagen.bf16_to_f32(datagen.bf16_round(v))
    np.testing.assert_array_equal(r[:4], [1.0, 1.0, 1.0 + 2**-6, -2.5])
    assert np.isinf(r[4])
    assert np.isfinite(r[5]) and r[5] > 2.9e38
