"""Plain numpy reference of the learned-initial-guess MLP -- TEST INFRASTRUCTURE ONLY.

Forward pass, loss and backward pass of the network the library trains
(30 features -> 128 -> 128 -> 128 -> head of 80, SiLU, inputs padded to 32),
written directly from the layer equations z = W a + b, a = SiLU(z) and the
chain rule, in float64.  The head holds a 7x10 matrix M (row-major, first
70 outputs) and an offset c (next 7); the standardised prediction of the
seven predicted fields (rho, u, u^1..3, q~, dP~) is y = M x_U + c with x_U
the first ten standardised features.  With `bf16=True` the inputs of every matrix product
(standardised features, activations, weights, output-side gradients) are
rounded to bfloat16 at the points where the device kernels round them.

Parameter vector layout (float32 on the device): W1[128][32], b1[128],
W2[128][128], b2[128], W3[128][128], b3[128], W4[80][128], b4[80].
Standardisation vector: x_mean[32], x_std[32], y_mean[16], y_std[16].
Loss: mean over rows and over the seven predicted fields (rho, u, u^1..3,
q~, dP~) of the squared error of the standardised targets.
"""
import numpy as np

SIZES = [(128, 32), (128, 128), (128, 128), (80, 128)]
FIELDS = np.array([0, 1, 2, 3, 4, 8, 9])       # predicted fields, in head order
NP, NXU = 7, 10


def head(out, xu):
    """y [M][7] from head outputs [M][80] and features x_U [M][10]."""
    M = out[:, :NP * NXU].reshape(-1, NP, NXU)
    return np.einsum("mij,mj->mi", M, xu) + out[:, NP * NXU:NP * NXU + NP]


def unpack(params):
    out, o = [], 0
    for no, ni in SIZES:
        W = np.asarray(params[o:o + no * ni], dtype=np.float64).reshape(no, ni)
        o += no * ni
        b = np.asarray(params[o:o + no], dtype=np.float64)
        o += no
        out.append((W, b))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def bf16(x):
    """Round float64/float32 values to the nearest bfloat16 (ties to even)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def standardise(X, Y, norm):
    """Standardised features and targets; a target whose std is 0 (constant
    over the training set) standardises to 0."""
    xm, xs, ym, ys = norm[:32], norm[32:64], norm[64:80], norm[80:96]
    ys = np.asarray(ys, np.float64)
    yd = np.where(ys > 0, ys, 1.0)
    return (np.asarray(X, np.float64) - xm) / xs, np.where(ys > 0, (np.asarray(Y, np.float64) - ym) / yd, 0.0)


def loss_and_grad(params, norm, X, Y, bf16_round=False):
    """(loss, gradient vector) over the rows of X [M][32], Y [M][16]."""
    r = bf16 if bf16_round else (lambda v: v)
    layers = unpack(params)
    xs, ys = standardise(X, Y, norm)
    xu = xs[:, :NXU]
    a = r(xs)
    acts, zs = [a], []
    for l, (W, b) in enumerate(layers):
        z = a @ r(W).T + b
        zs.append(z)
        if l < 3:
            a = r(silu(z))
            acts.append(a)
    out = zs[-1]
    y = head(out, xu)
    M = X.shape[0]
    e = y - ys[:, FIELDS]
    loss = float((e ** 2).sum() / (7.0 * M))
    de = 2.0 * e / (7.0 * M)
    gf = np.zeros_like(out)            # output-side gradient of the current layer
    gf[:, :NP * NXU] = (de[:, :, None] * xu[:, None, :]).reshape(M, -1)
    gf[:, NP * NXU:NP * NXU + NP] = de
    grads = [None] * 4
    for l in range(3, -1, -1):
        W, b = layers[l]
        g = r(gf)                      # rounded where it feeds a matrix product
        grads[l] = (g.T @ acts[l], gf.sum(axis=0))
        if l == 0:
            break
        gf = (g @ r(W)) * silu_grad(zs[l - 1])
    return loss, pack(grads)


def loss_only(params, norm, X, Y):
    return loss_and_grad(params, norm, X, Y)[0]


def predict(params, norm, X, bf16_round=False):
    """Unstandardised predictions [M][16] (float64; zero for the fields not
    predicted); with `bf16_round` the standardised inputs, the weights and
    the hidden activations are rounded to bfloat16 as the device rounds them."""
    r = bf16 if bf16_round else (lambda v: v)
    layers = unpack(params)
    xs = (np.asarray(X, np.float64) - norm[:32]) / norm[32:64]
    a = r(xs)
    for l, (W, b) in enumerate(layers):
        a = a @ r(W).T + b
        if l < 3:
            a = r(silu(a))
    y = head(a, xs[:, :NXU])
    out = np.zeros((X.shape[0], 16))
    out[:, FIELDS] = y * norm[80:96][FIELDS] + norm[64:80][FIELDS]
    return out
