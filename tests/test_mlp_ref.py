"""Pins of the numpy MLP reference: its analytic gradient against central
finite differences of its own loss, and the bfloat16 rounding helper
against the format's definition."""
import numpy as np

from oracle import mlp_ref


def _setup(rng, M=64):
    params = []
    for no, ni in mlp_ref.SIZES:
        params.append(rng.uniform(-1, 1, no * ni) * np.sqrt(6.0 / ni))
        params.append(rng.normal(0, 0.1, no))
    params = np.concatenate(params)
    norm = np.concatenate([rng.normal(0, 1, 32), rng.uniform(0.5, 2, 32), rng.normal(0, 1, 16), rng.uniform(0.5, 2, 16)])
    X = rng.normal(0, 1, (M, 32))
    Y = rng.normal(0, 1, (M, 16))
    return params, norm, X, Y


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    params, norm, X, Y = _setup(rng)
    _, g = mlp_ref.loss_and_grad(params, norm, X, Y)
    idx = np.concatenate([rng.choice(params.size, 60, replace=False),
                          [0, 4096, 4096 + 128 + 5, params.size - 1, params.size - 17]])
    for i in idx:
        h = 1e-6 * max(1.0, abs(params[i]))
        p1, p2 = params.copy(), params.copy()
        p1[i] += h
        p2[i] -= h
        fd = (mlp_ref.loss_only(p1, norm, X, Y) - mlp_ref.loss_only(p2, norm, X, Y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * (abs(g).max() + abs(fd))


def test_head_padding_carries_no_gradient_and_head_is_linear_in_xu():
    rng = np.random.default_rng(1)
    params, norm, X, Y = _setup(rng)
    _, g = mlp_ref.loss_and_grad(params, norm, X, Y)
    W4, b4 = mlp_ref.unpack(g)[3]
    assert np.all(W4[77:] == 0) and np.all(b4[77:] == 0)
    # the prediction is affine in the standardised increment features x_U
    X2 = X.copy()
    X2[:, :10] = 2 * X[:, :10] - norm[:10]      # doubles the standardised x_U
    X0 = X.copy()
    X0[:, :10] = norm[:10]                      # standardised x_U = 0
    p1 = mlp_ref.predict(params, norm, X)
    p2 = mlp_ref.predict(params, norm, X2)
    p0 = mlp_ref.predict(params, norm, X0)
    # the body also sees x_U, so only check the head's algebra on the body output
    out = np.random.default_rng(5).normal(size=(4, 80))
    xu = np.random.default_rng(6).normal(size=(4, 10))
    assert np.allclose(mlp_ref.head(out, 2 * xu) - mlp_ref.head(out, xu),
                       mlp_ref.head(out, xu) - mlp_ref.head(out, 0 * xu))
    assert p1.shape == p2.shape == p0.shape == (X.shape[0], 16)


def test_bf16_rounding():
    # bfloat16 keeps 8 significant bits: 1 + 2^-8 rounds to 1 (tie to even), 1 + 3*2^-8 to 1 + 2^-6... exact cases
    assert mlp_ref.bf16(1.0 + 2 ** -8) == 1.0
    assert mlp_ref.bf16(1.0 + 2 ** -7) == 1.0 + 2 ** -7
    assert mlp_ref.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6
    x = np.random.default_rng(2).normal(0, 10, 1000)
    assert np.all(np.abs(mlp_ref.bf16(x) - x) <= np.abs(x) * 2 ** -8)
