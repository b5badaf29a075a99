"""The training contraction C = A B^T (bfloat16 operands, float32
accumulation on the tensor cores) element by element against float64.

Every product of two bfloat16 numbers is exact in float32 and float64, so
the float64 sum of the same bfloat16 values is the exact result up to
float64 rounding; the kernel differs from it only by its float32
accumulation.  Recursive float32 summation of K terms errs by at most
gamma_K sum_k |a_ik b_jk| with gamma_K ~ K u, u = 2^-24; the bound below
takes 2 K u to leave room for the tensor cores' order of additions and the
split sums.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _operands(dev, M, N, K, pad=0, seed=0):
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(M, K + pad, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K + pad, generator=g).to(torch.bfloat16)
    return A.to(dev)[:, :K], B.to(dev)[:, :K]


def _check(C, A, B):
    a = A.float().cpu().double().numpy()
    b = B.float().cpu().double().numpy()
    exact = a @ b.T
    bound = 2.0 * a.shape[1] * 2.0 ** -24 * (np.abs(a) @ np.abs(b).T) + 1e-30
    err = np.abs(C.cpu().double().numpy() - exact)
    assert np.all(err <= bound), float((err / bound).max())


# (M, N, K): the network's shapes at a batch of 4096 (forward, the weight
# gradients with K = batch, the input gradients), then ragged cases: rows
# short of a 128-row tile, two column tiles with a short second one, K not a
# multiple of the 64-column chunk nor of 8 (a strided view whose row stride
# is a multiple of 8), and a single 16-column tile.
SHAPES = [(4096, 128, 32), (4096, 80, 128), (80, 128, 4096), (128, 32, 4096), (4096, 128, 80),
          (200, 144, 200), (77, 16, 100), (1, 48, 8), (300, 256, 1000)]


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_gemm_matches_float64(dev, M, N, K):
    from paper_1702_01106_b300.grim import gemm_nt_bf16
    A, B = _operands(dev, M, N, K, pad=(-K) % 8)
    _check(gemm_nt_bf16(A, B), A, B)


@pytest.mark.parametrize("splits", [2, 3, 16])
def test_split_k_sums_match_float64(dev, splits):
    """K = 4096 in 64 chunks split 2, 3 (22 + 22 + 20 chunks) and 16 ways."""
    from paper_1702_01106_b300.grim import gemm_nt_bf16
    A, B = _operands(dev, 128, 128, 4096, seed=splits)
    _check(gemm_nt_bf16(A, B, splits=splits), A, B)


def test_strided_output(dev):
    """C written into a column block of a wider matrix (ldc > N) leaves the
    rest of the matrix untouched."""
    from paper_1702_01106_b300.grim import gemm_nt_bf16
    A, B = _operands(dev, 160, 32, 64, seed=5)
    wide = torch.full((160, 100), 7.0, device=dev)
    gemm_nt_bf16(A, B, out=wide[:, 36:68])
    _check(wide[:, 36:68], A, B)
    assert torch.all(wide[:, :36] == 7.0) and torch.all(wide[:, 68:] == 7.0)


@pytest.mark.parametrize("M,N,K,why", [(64, 40, 64, "N not a multiple of 16"), (64, 32, 12, "row stride 12")])
def test_unsupported_shapes_are_refused(dev, M, N, K, why):
    from paper_1702_01106_b300.grim import gemm_nt_bf16
    A, B = _operands(dev, M, N, K)
    with pytest.raises(RuntimeError, match="invalid"):
        gemm_nt_bf16(A.contiguous(), B.contiguous())


def test_training_gradient_is_deterministic_at_batch_4096(dev):
    """The weight gradients sum 16 K-slices in a fixed order: two gradient
    evaluations of the same batch agree bit for bit."""
    from paper_1702_01106_b300.grim import MLP
    rng = np.random.default_rng(8)
    X = torch.from_numpy(rng.normal(0, 1, (4096, 32)).astype(np.float32)).to(dev)
    Y = torch.from_numpy(rng.normal(0, 1, (4096, 16)).astype(np.float32)).to(dev)
    m = MLP(seed=2)
    g1, l1 = m.gradient(X, Y)
    g2, l2 = m.gradient(X, Y)
    m.close()
    assert np.array_equal(g1, g2)
    assert np.isfinite(g1).all() and np.abs(g1).max() > 0
