"""FP64 numpy reference of the proposal network (test infrastructure only).

Same architecture and flat parameter order as the CUDA implementation: input averaged over
down x down pixels and standardised per image (population variance); six 3x3 convolutions with
zero padding 1, strides 1, 2, 1, 2, 1, 2, each followed by ReLU; two linear heads (orientation bins,
defocus bins); loss = mean over the batch of the two cross-entropies.  Gradients are written out
from the chain rule (no automatic differentiation).  Pinned by tests/test_cnn_oracle.py against
scipy's correlate2d and log_softmax and by finite differences of its own forward pass.
"""
from __future__ import annotations

import numpy as np

STRIDES = (1, 2, 1, 2, 1, 2)


def layout(S: int, C: int, n_q: int, n_d: int):
    """Offsets of every tensor in the flat parameter vector, and the feature size F."""
    offs = []
    p = 0
    cin = 1
    for _ in STRIDES:
        w = (p, (C, cin, 3, 3))
        p += C * cin * 9
        b = (p, (C,))
        p += C
        offs.append((w, b))
        cin = C
    F = C * (S // 8) ** 2
    wq = (p, (n_q, F)); p += n_q * F
    bq = (p, (n_q,)); p += n_q
    wd = (p, (n_d, F)); p += n_d * F
    bd = (p, (n_d,)); p += n_d
    return offs, (wq, bq, wd, bd), F, p


def unpack(theta, S, C, n_q, n_d):
    offs, heads, F, n = layout(S, C, n_q, n_d)
    assert theta.size == n
    get = lambda o: theta[o[0]:o[0] + int(np.prod(o[1]))].reshape(o[1])
    return [(get(w), get(b)) for w, b in offs], [get(h) for h in heads]


def prepare(images, down: int):
    """[B, n, n] -> [B, 1, S, S]: 2-D average over down x down blocks, then zero mean, unit variance."""
    x = np.asarray(images, dtype=np.float64)
    B, n, _ = x.shape
    S = n // down
    x = x.reshape(B, S, down, S, down).mean(axis=(2, 4))
    m = x.mean(axis=(1, 2), keepdims=True)
    v = x.var(axis=(1, 2), keepdims=True)
    return ((x - m) / np.sqrt(v))[:, None]


def conv_forward(x, W, b, stride):
    """y[b,co,i,j] = b[co] + sum_{ci,ky,kx} W[co,ci,ky,kx] xpad[b,ci,i s + ky, j s + kx]."""
    B, cin, H, _ = x.shape
    Ho = H // stride
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    y = np.zeros((B, W.shape[0], Ho, Ho)) + b[None, :, None, None]
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky:ky + stride * Ho:stride, kx:kx + stride * Ho:stride]   # [B, cin, Ho, Ho]
            y += np.einsum("bchw,oc->bohw", patch, W[:, :, ky, kx])
    return y


def conv_backward(x, W, gy, stride):
    """Gradients of sum(gy * conv_forward(x, W, b, stride)) w.r.t. x, W and b."""
    B, cin, H, _ = x.shape
    Ho = gy.shape[2]
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky:ky + stride * Ho:stride, kx:kx + stride * Ho:stride]
            gW[:, :, ky, kx] = np.einsum("bohw,bchw->oc", gy, patch)
            gxp[:, :, ky:ky + stride * Ho:stride, kx:kx + stride * Ho:stride] += np.einsum("bohw,oc->bchw", gy,
                                                                                          W[:, :, ky, kx])
    return gxp[:, :, 1:-1, 1:-1], gW, gy.sum(axis=(0, 2, 3))


def log_softmax(z):
    m = z.max(axis=1, keepdims=True)
    return z - m - np.log(np.exp(z - m).sum(axis=1, keepdims=True))


def forward(theta, images, down, C, n_q, n_d):
    """Logits of both heads and the cached activations."""
    x0 = prepare(images, down)
    S = x0.shape[2]
    convs, (Wq, bq, Wd, bd) = unpack(theta, S, C, n_q, n_d)
    acts = [x0]
    for (W, b), s in zip(convs, STRIDES):
        acts.append(np.maximum(conv_forward(acts[-1], W, b, s), 0.0))
    feat = acts[-1].reshape(len(images), -1)
    return feat @ Wq.T + bq, feat @ Wd.T + bd, acts


def loss_and_grad(theta, images, yq, yd, down, C, n_q, n_d):
    """Per-sample losses and the gradient of their mean w.r.t. the flat parameters."""
    lq, ld, acts = forward(theta, images, down, C, n_q, n_d)
    B = len(images)
    S = acts[0].shape[2]
    convs, (Wq, bq, Wd, bd) = unpack(theta, S, C, n_q, n_d)
    pq, pd = log_softmax(lq), log_softmax(ld)
    losses = -pq[np.arange(B), yq] - pd[np.arange(B), yd]
    gq = np.exp(pq)
    gq[np.arange(B), yq] -= 1.0
    gd = np.exp(pd)
    gd[np.arange(B), yd] -= 1.0
    gq /= B
    gd /= B
    feat = acts[-1].reshape(B, -1)
    offs, heads, F, n = layout(S, C, n_q, n_d)
    grad = np.zeros(n)

    def put(o, v):
        grad[o[0]:o[0] + v.size] = v.ravel()

    put(heads[0], gq.T @ feat)
    put(heads[1], gq.sum(axis=0))
    put(heads[2], gd.T @ feat)
    put(heads[3], gd.sum(axis=0))
    g = (gq @ Wq + gd @ Wd).reshape(acts[-1].shape)
    for li in range(len(STRIDES) - 1, -1, -1):
        g = g * (acts[li + 1] > 0)
        W = convs[li][0]
        gx, gW, gb = conv_backward(acts[li], W, g, STRIDES[li])
        put(offs[li][0], gW)
        put(offs[li][1], gb)
        g = gx
    return losses, grad
