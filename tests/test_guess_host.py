"""Host logic of the learned start's training driver (no GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_drop_outliers_keeps_the_bulk():
    """Rows beyond the limit (in spans of the central 99.8 %) in any feature
    or target are dropped; constant columns (the Minkowski metric entries,
    the padded targets) do not count; the bulk is kept in order.  A column
    that is zero in most rows (a velocity where most zones are at rest)
    marks none of its other rows as outlying."""
    from paper_1702_01106_b300.guess import drop_outliers
    g = torch.Generator().manual_seed(3)
    X = torch.randn(20000, 32, generator=g)
    Y = torch.randn(20000, 16, generator=g)
    X[:, 10:20] = -1.0          # constant features
    Y[:, 5:8] = 0.0             # targets not predicted
    X[7, 3] = 1e4               # outliers in a feature and in a target
    Y[11, 2] = -1e3
    X[:15000, 4] = 0.0          # mostly at rest: its deviation is zero, its span is not
    Xk, Yk = drop_outliers(X, Y, 10.0)
    assert Xk.shape == (19998, 32) and Yk.shape == (19998, 16)
    keep = np.ones(20000, bool)
    keep[[7, 11]] = False
    assert torch.equal(Xk, X[torch.from_numpy(keep)]) and torch.equal(Yk, Y[torch.from_numpy(keep)])
    # a generous limit keeps every row
    Xa, _ = drop_outliers(X, Y, 1e6)
    assert Xa.shape[0] == 20000
