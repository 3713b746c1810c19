"""FP64 oracle of the proposal network and its training step.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). The network of the learned
sampling proposal: x -> relu(x W1 + b1) -> relu(. W2 + b2) -> relu(. W3 + b3)
-> z = . W4 + b4, PDF = softmax(z[:32]), T^ = sigmoid(z[32]). The library
evaluates it with BF16 weights and BF16 layer inputs; this oracle rounds at the
same points (round to nearest even) and does every other operation in FP64.
With round_bf16=False it is the plain FP64 network (used by the finite-
difference pins).

Loss per ray (targets: 32 profile bins and the final transmittance T):
w KL(q || p) + (T^ - T)^2 with q = bins / sum(bins) and w = sum(bins); the mean
over rays. The backward treats BF16 rounding as the identity.
"""
import numpy as np

LAYERS = ((112, 64), (64, 64), (64, 64), (64, 40))
N_PARAMS = 18152
BINS = 32


def bf16(x):
    """Round to the nearest BF16 value (ties to even), via FP32."""
    x32 = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = x32.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params):
    p = np.asarray(params, dtype=np.float64).reshape(-1)
    assert p.size == N_PARAMS
    out, off = [], 0
    for k, n in LAYERS:
        out.append(p[off:off + k * n].reshape(k, n))
        off += k * n
        out.append(p[off:off + n])
        off += n
    return out


def forward(params, feat, round_bf16=True):
    r = bf16 if round_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(params)
    x = r(feat)
    Wb = [r(W) for W in (W1, W2, W3, W4)]
    z1 = x @ Wb[0] + b1
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ Wb[1] + b2
    h2 = r(np.maximum(z2, 0.0))
    z3 = h2 @ Wb[2] + b3
    h3 = r(np.maximum(z3, 0.0))
    z4 = h3 @ Wb[3] + b4
    zl = z4[:, :BINS]
    lse = zl.max(axis=1, keepdims=True)
    lse = lse + np.log(np.exp(zl - lse).sum(axis=1, keepdims=True))
    logp = zl - lse
    pdf = np.exp(logp)
    that = 1.0 / (1.0 + np.exp(-z4[:, BINS]))
    return dict(pdf=pdf, that=that, logp=logp, x=x, h=(h1, h2, h3), Wb=Wb, z4=z4)


def loss_and_grad(params, feat, target, round_bf16=True):
    f = forward(params, feat, round_bf16)
    t = np.asarray(target, dtype=np.float64)
    n = t.shape[0]
    bins, T = t[:, :BINS], t[:, BINS]
    S = bins.sum(axis=1)
    has = S > 0
    q = np.where(has[:, None], bins / np.where(has, S, 1.0)[:, None], 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        kl = np.where(q > 0, q * (np.log(np.where(q > 0, q, 1.0)) - f["logp"]), 0.0).sum(axis=1)
    dt = f["that"] - T
    loss = float((S * kl + dt * dt).sum() / n)
    dz4 = np.zeros_like(f["z4"])
    dz4[:, :BINS] = np.where(has[:, None], S[:, None] * (f["pdf"] - q), 0.0) / n
    dz4[:, BINS] = 2.0 * dt * f["that"] * (1.0 - f["that"]) / n
    h1, h2, h3 = f["h"]
    Wb = f["Wb"]
    acts = (f["x"], h1, h2, h3)
    grads = [None] * 8
    dz = dz4
    for li in (3, 2, 1, 0):
        grads[2 * li] = acts[li].T @ dz
        grads[2 * li + 1] = dz.sum(axis=0)
        if li > 0:
            dz = (dz @ Wb[li].T) * (acts[li] > 0)
    return loss, np.concatenate([g.reshape(-1) for g in grads])


def adam(params, m, v, grad, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, 2015) in FP64."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
