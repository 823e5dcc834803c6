"""CNN oracle (test infrastructure only): the small classifier that replaces
the paper's YOLOv11n detector (Sec. 2.5; its weights and data sets are not
available), written as plain numpy definitions.

Network (reading): input NHWC [N][64][64][2] (channel 0 DM-time, 1 freq-time
cut-out); three blocks conv3x3 (pad 1, stride 1, + bias) -> ReLU -> 2x2 max
pool with 2 -> 16 -> 32 -> 64 channels; global average pool; fully connected
64 -> 2; softmax cross-entropy with labels {0: not a pulse, 1: pulse}.
Max-pool ties go to the first element in (dy, dx) raster order.

Precision policy of the GPU kernels, mirrored here when bf16=True: every
tensor a kernel reads as a tensor-core operand is rounded to bfloat16 (input,
weights, each block's pooled activation, and the back-propagated activation
gradients), accumulation is float32 (here float64), biases and weight
gradients are float32.  With bf16=False everything is float64 (used for the
finite-difference pins).
"""
import numpy as np

from .cutout import bf16_round

CH = [2, 16, 32, 64]


def _r(x, bf16):
    return bf16_round(x).astype(np.float64) if bf16 else np.asarray(x, dtype=np.float64)


def init_params(seed=0):
    """He-normal weights [Cout][3][3][Cin], zero biases, FC [2][64]."""
    rng = np.random.default_rng(seed)
    p = {}
    for l in range(3):
        cin, cout = CH[l], CH[l + 1]
        p["w%d" % l] = rng.normal(0.0, np.sqrt(2.0 / (9 * cin)), (cout, 3, 3, cin)).astype(np.float32)
        p["b%d" % l] = np.zeros(cout, dtype=np.float32)
    p["fw"] = rng.normal(0.0, np.sqrt(1.0 / 64), (2, 64)).astype(np.float32)
    p["fb"] = np.zeros(2, dtype=np.float32)
    return p


def conv3x3(x, w, b):
    """y[n,h,x,o] = b[o] + sum_{dy,dx,i} x[n, h+dy-1, x+dx-1, i] w[o,dy,dx,i], zero padding."""
    n, H, W, cin = x.shape
    xp = np.zeros((n, H + 2, W + 2, cin))
    xp[:, 1:H + 1, 1:W + 1, :] = x
    y = np.zeros((n, H, W, w.shape[0]))
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("nhwi,oi->nhwo", xp[:, dy:dy + H, dx:dx + W, :], w[:, dy, dx, :])
    return y + b


def conv3x3_grads(x, w, dy_):
    """Gradients of conv3x3 w.r.t. its input and weights."""
    n, H, W, cin = x.shape
    xp = np.zeros((n, H + 2, W + 2, cin))
    xp[:, 1:H + 1, 1:W + 1, :] = x
    dw = np.zeros(w.shape)
    dxp = np.zeros(xp.shape)
    for a in range(3):
        for c in range(3):
            dw[:, a, c, :] = np.einsum("nhwo,nhwi->oi", dy_, xp[:, a:a + H, c:c + W, :])
            dxp[:, a:a + H, c:c + W, :] += np.einsum("nhwo,oi->nhwi", dy_, w[:, a, c, :])
    return dxp[:, 1:H + 1, 1:W + 1, :], dw, dy_.sum(axis=(0, 1, 2))


def maxpool2(x):
    n, H, W, c = x.shape
    v = x.reshape(n, H // 2, 2, W // 2, 2, c).transpose(0, 1, 3, 2, 4, 5).reshape(n, H // 2, W // 2, 4, c)
    idx = np.argmax(v, axis=3)            # first maximum in raster order (0,0),(0,1),(1,0),(1,1)
    return np.take_along_axis(v, idx[:, :, :, None, :], axis=3)[:, :, :, 0, :], idx


def maxpool2_grad(dout, idx, shape):
    n, H, W, c = shape
    g = np.zeros((n, H // 2, W // 2, 4, c))
    np.put_along_axis(g, idx[:, :, :, None, :], dout[:, :, :, None, :], axis=3)
    return g.reshape(n, H // 2, W // 2, 2, 2, c).transpose(0, 1, 3, 2, 4, 5).reshape(shape)


def forward(p, x, bf16=True):
    """x: [N][64][64][2].  Returns logits [N][2] and the cache for backward."""
    cache = {"a0": _r(x, bf16)}
    a = cache["a0"]
    for l in range(3):
        z = conv3x3(a, _r(p["w%d" % l], bf16), np.asarray(p["b%d" % l], dtype=np.float64))
        r = np.maximum(z, 0.0)
        pooled, idx = maxpool2(r)
        cache["in%d" % l], cache["relu%d" % l], cache["idx%d" % l] = a, r, idx
        a = _r(pooled, bf16)
    cache["a3"] = a
    g = a.mean(axis=(1, 2))
    cache["gap"] = g
    logits = g @ np.asarray(p["fw"], dtype=np.float64).T + np.asarray(p["fb"], dtype=np.float64)
    return logits, cache


def softmax_ce(logits, y):
    z = logits - logits.max(axis=1, keepdims=True)
    e = np.exp(z)
    pr = e / e.sum(axis=1, keepdims=True)
    loss = -np.mean(np.log(pr[np.arange(len(y)), y]))
    d = pr.copy()
    d[np.arange(len(y)), y] -= 1.0
    return loss, d / len(y), pr


def backward(p, cache, dlogits, bf16=True):
    """Gradients of the mean loss; dlogits from softmax_ce."""
    grads = {}
    g = cache["gap"]
    grads["fw"] = dlogits.T @ g
    grads["fb"] = dlogits.sum(axis=0)
    dg = dlogits @ np.asarray(p["fw"], dtype=np.float64)
    a3 = cache["a3"]
    da = np.broadcast_to(dg[:, None, None, :] / (a3.shape[1] * a3.shape[2]), a3.shape).copy()
    for l in (2, 1, 0):
        da = _r(da, bf16)
        r = cache["relu%d" % l]
        dr = maxpool2_grad(da, cache["idx%d" % l], r.shape)
        dz = dr * (r > 0)
        dz = _r(dz, bf16)
        dx, dw, db = conv3x3_grads(cache["in%d" % l], _r(p["w%d" % l], bf16), dz)
        grads["w%d" % l], grads["b%d" % l] = dw, db
        da = dx
    grads["x"] = da
    return grads


def loss_and_grads(p, x, y, bf16=True):
    logits, cache = forward(p, x, bf16)
    loss, dl, _ = softmax_ce(logits, y)
    return loss, logits, backward(p, cache, dl, bf16)


def adam_step(p, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam on float32 master weights (Kingma & Ba 2015), bias-corrected."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        g = np.asarray(grads[k], dtype=np.float32)
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = beta1 * m + (1 - beta1) * g
        v[...] = beta2 * v + (1 - beta2) * g * g
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        p[k] = (p[k] - lr * mh / (np.sqrt(vh) + eps)).astype(np.float32)
    return p
