"""The seeded input generators: deterministic, with the recipe's sizes, signs and sample statistics."""
import numpy as np

from paper_2603_29227_gb300 import scenes


def test_plane2d_recipe():
    w = scenes.workload("plane2d")
    assert w.x.shape == (2000, 2) and w.xq.shape == (128 * 128, 2) and w.xq.dtype == np.float32
    assert w.params["cell"] == 1.0 and w.params["n_max"] == 64 and w.params["lambda"] == 500.0
    w2 = scenes.workload("plane2d")
    assert np.array_equal(w.x, w2.x) and np.array_equal(w.var, w2.var)
    # samples lie within a few noise sigmas of the boundary, with variance (0.01 U[0.5, 2])^2
    free = ~w.scene.occupied(w.x)
    assert np.max(np.abs(w.scene.dist_free(w.x[free]))) < 0.06
    assert w.var.min() >= (0.005 ** 2) * 0.999 and w.var.max() <= (0.02 ** 2) * 1.001
    assert np.allclose(np.linalg.norm(w.normals, axis=1), 1.0, atol=1e-6)
    assert set(np.unique(w.sign)) <= {-1, 1}


def test_room3d_small_and_signs():
    w = scenes.workload("room3d", n_samples=5000, n_queries=2000)
    assert w.x.shape == (5000, 3) and w.xq.shape == (2000, 3)
    occ = w.scene.occupied(w.xq.astype(np.float64))
    assert np.array_equal(w.sign == -1, occ)
    assert np.all((w.xq >= 0) & (w.xq <= np.array([20, 20, 5], dtype=np.float32)))


def test_traj3d_shape():
    w = scenes.workload("traj3d", n_samples=3000, n_queries=64 * 8 * 3)
    assert w.xq.shape == (3 * 64 * 8, 3)
