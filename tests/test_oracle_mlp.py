"""Pins of the FP64 network reference: its hand-written gradient against
central finite differences, its patch extraction against an index-coded map,
and the loss against its closed form at zero weights.  CPU only."""
import numpy as np
import pytest

from oracle import mlp


def _params(seed, scale=0.1):
    r = np.random.default_rng(seed)
    return r.normal(0, scale, mlp.P)


def test_gradient_matches_central_differences():
    r = np.random.default_rng(1)
    X = r.normal(0, 1, (12, mlp.D))
    y = (r.random(12) < 0.5).astype(float)
    p = _params(2)
    g = mlp.grad(X, y, p)
    idx = np.concatenate([r.choice(mlp.H * mlp.D, 40, replace=False),
                          mlp.H * mlp.D + np.arange(2 * mlp.H + 1)])
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.P); e[i] = h
        fd = (mlp.loss(X, y, p + e) - mlp.loss(X, y, p - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, i


def test_loss_at_zero_weights_is_log2():
    X = np.random.default_rng(0).normal(0, 1, (5, mlp.D))
    assert mlp.loss(X, np.array([0, 1, 0, 1, 1.0]), np.zeros(mlp.P)) == pytest.approx(np.log(2.0), rel=1e-15)


def test_patches_of_an_index_coded_map():
    M, NB = 12, 50
    mm, bb = np.meshgrid(np.arange(M), np.arange(NB), indexing="ij")
    smap = np.sinh(mm * 50.0 + bb)           # asinh recovers the code (all codes < 700)
    cells = [(6, 25), (0, 0), (11, 49)]
    X = mlp.patches(smap, cells).reshape(3, mlp.T, mlp.B)
    # centre cell
    assert X[0, 4, 16] == pytest.approx(6 * 50 + 25)
    assert X[0, 0, 0] == pytest.approx((6 - 4) * 50 + (25 - 16))
    # corners outside the map are zero, inside are their codes
    assert X[1, 0, 0] == 0.0 and X[1, 4, 16] == pytest.approx(0.0) and X[1, 8, 32] == pytest.approx(4 * 50 + 16)
    assert X[2, 8, 32] == 0.0 and X[2, 4, 16] == pytest.approx(11 * 50 + 49)
