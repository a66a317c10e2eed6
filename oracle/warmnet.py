"""FP64 NumPy oracle of the warm-start network (include/wsnet.h).

TEST INFRASTRUCTURE ONLY. A plain restatement of the network's definition --
3x3 zero-padded convolutions written as sums over the nine kernel offsets,
2x2 average pooling, nearest upsampling, skip additions, ReLU, softplus and
the mean squared error -- with the backward pass derived by hand from the
same definitions. Weights are rounded to BF16 (nearest even) before use, as
the CUDA kernels do; biases stay in full precision. Pinned in
tests/test_warmnet_oracle.py by central finite differences.
"""
import numpy as np

CHANNELS = lambda Q, n_dual=0: [(Q + 1, 64), (64, 64), (64, 128), (128, 128), (128, 256), (256, 128), (128, 64),
                                (64, 64), (64, Q * (1 + n_dual))]


def layout(Q, n_dual=0):
    """[(w_offset, b_offset, ci, co)] of the packed parameter vector, and its length."""
    out, off = [], 0
    for ci, co in CHANNELS(Q, n_dual):
        w0 = off
        off += ci * co * 9
        out.append((w0, off, ci, co))
        off += co
    return out, off


def bf16(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params, Q, round_weights=True, n_dual=0):
    lay, _ = layout(Q, n_dual)
    ws = []
    for w0, b0, ci, co in lay:
        W = params[w0:w0 + ci * co * 9]
        W = (bf16(W) if round_weights else np.asarray(W, np.float64)).reshape(co, ci, 3, 3)
        b = np.asarray(params[b0:b0 + co], np.float64)
        ws.append((W, b))
    return ws


def conv(x, W, b):
    """y[n,o,h,w] = b[o] + sum_{c,kh,kw} x[n,c,h+kh-1,w+kw-1] W[o,c,kh,kw] (zero outside)."""
    N, C, H, Wd = x.shape
    xp = np.zeros((N, C, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    y = np.zeros((N, W.shape[0], H, Wd)) + b[None, :, None, None]
    for kh in range(3):
        for kw in range(3):
            y += np.einsum("nchw,oc->nohw", xp[:, :, kh:kh + H, kw:kw + Wd], W[:, :, kh, kw])
    return y


def conv_back(x, W, dy):
    """Gradients of conv: dx, dW, db."""
    N, C, H, Wd = x.shape
    xp = np.zeros((N, C, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for kh in range(3):
        for kw in range(3):
            dW[:, :, kh, kw] = np.einsum("nohw,nchw->oc", dy, xp[:, :, kh:kh + H, kw:kw + Wd])
            dxp[:, :, kh:kh + H, kw:kw + Wd] += np.einsum("nohw,oc->nchw", dy, W[:, :, kh, kw])
    return dxp[:, :, 1:-1, 1:-1], dW, dy.sum(axis=(0, 2, 3))


def pool(x):
    return 0.25 * (x[:, :, 0::2, 0::2] + x[:, :, 1::2, 0::2] + x[:, :, 0::2, 1::2] + x[:, :, 1::2, 1::2])


def pool_back(dy):
    return 0.25 * np.repeat(np.repeat(dy, 2, axis=2), 2, axis=3)


def up(x):
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def up_back(dy):
    return dy[:, :, 0::2, 0::2] + dy[:, :, 1::2, 0::2] + dy[:, :, 0::2, 1::2] + dy[:, :, 1::2, 1::2]


def softplus(z):
    return np.where(z > 20, z, np.log1p(np.exp(np.minimum(z, 20))))


def forward(params, x, Q, keep=False, round_weights=True, n_dual=0):
    """Network output for x [N, Q+1, H, W]: softplus(z) on the Q image channels,
    z itself on the n_dual * Q dual channels; with keep, also the activations."""
    w = unpack(params, Q, round_weights, n_dual)
    relu = lambda a: np.maximum(a, 0.0)
    a1 = relu(conv(x, *w[0]))
    a2 = relu(conv(a1, *w[1]))
    p1 = pool(a2)
    a3 = relu(conv(p1, *w[2]))
    a4 = relu(conv(a3, *w[3]))
    p2 = pool(a4)
    a5 = relu(conv(p2, *w[4]))
    a6 = relu(conv(a5, *w[5]))
    s1 = up(a6) + a4
    a7 = relu(conv(s1, *w[6]))
    s2 = up(a7) + a2
    a8 = relu(conv(s2, *w[7]))
    z = conv(a8, *w[8])
    out = z.copy()
    out[:, :Q] = softplus(z[:, :Q])
    if keep:
        return out, dict(x=x, a1=a1, a2=a2, p1=p1, a3=a3, a4=a4, p2=p2, a5=a5, a6=a6, s1=s1, a7=a7, s2=s2,
                         a8=a8, z=z, w=w)
    return out


def loss_grad(params, x, target, Q, round_weights=True, n_dual=0):
    """(loss, gradient packed like params): loss = mean((out - target)^2) over
    every output, the gradient taken with respect to the (rounded) weights the
    forward pass used (the image channels through softplus, whose derivative
    is the logistic function; the dual channels directly)."""
    out, A = forward(params, x, Q, keep=True, round_weights=round_weights, n_dual=n_dual)
    M = out.size
    loss = float(np.mean((out - target) ** 2))
    z = A["z"]
    gz = 2.0 * (out - target) / M
    gz[:, :Q] = gz[:, :Q] / (1.0 + np.exp(-z[:, :Q]))
    w = A["w"]
    grads = [None] * 9
    mask = lambda g, a: g * (a > 0)
    g8, dW, db = conv_back(A["a8"], w[8][0], gz)
    grads[8] = (dW, db)
    g8 = mask(g8, A["a8"])
    gs2, dW, db = conv_back(A["s2"], w[7][0], g8)
    grads[7] = (dW, db)
    g2 = gs2.copy()
    g7 = mask(up_back(gs2), A["a7"])
    gs1, dW, db = conv_back(A["s1"], w[6][0], g7)
    grads[6] = (dW, db)
    g4 = gs1.copy()
    g6 = mask(up_back(gs1), A["a6"])
    g5, dW, db = conv_back(A["a5"], w[5][0], g6)
    grads[5] = (dW, db)
    g5 = mask(g5, A["a5"])
    gp2, dW, db = conv_back(A["p2"], w[4][0], g5)
    grads[4] = (dW, db)
    g4 = mask(g4 + pool_back(gp2), A["a4"])
    g3, dW, db = conv_back(A["a3"], w[3][0], g4)
    grads[3] = (dW, db)
    g3 = mask(g3, A["a3"])
    gp1, dW, db = conv_back(A["p1"], w[2][0], g3)
    grads[2] = (dW, db)
    g2 = mask(g2 + pool_back(gp1), A["a2"])
    g1, dW, db = conv_back(A["a1"], w[1][0], g2)
    grads[1] = (dW, db)
    g1 = mask(g1, A["a1"])
    _, dW, db = conv_back(A["x"], w[0][0], g1)
    grads[0] = (dW, db)
    lay, P = layout(Q, n_dual)
    flat = np.zeros(P)
    for (w0, b0, ci, co), (dW, db) in zip(lay, grads):
        flat[w0:w0 + ci * co * 9] = dW.ravel()
        flat[b0:b0 + co] = db
    return loss, flat
