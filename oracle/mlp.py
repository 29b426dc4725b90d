"""FP64 reference of the learned proposal's network (test infrastructure only).

Model (the search's own definition; the paper proposes no network):
  input   9 x 33 patch of an n_sigma map around a cell (templates m-4..m+4,
          bins b-16..b+16, zero outside the map), each value through asinh
  network z1 = W1 x + b1 (64), h = max(z1, 0), logit = w2 . h + b2
  loss    mean over the batch of softplus(logit) - y logit (binary cross
          entropy with logits)
Parameters are one vector: W1 [64][297] row-major, b1 [64], w2 [64], b2.
The backward pass is written out by hand; the tests pin it against central
finite differences of `loss`.
"""
import numpy as np

T, B, D, H = 9, 33, 297, 64
P = H * D + 2 * H + 1


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    W1 = p[:H * D].reshape(H, D)
    b1 = p[H * D:H * D + H]
    w2 = p[H * D + H:H * D + 2 * H]
    b2 = p[-1]
    return W1, b1, w2, b2


def fp16_weights(params):
    """Parameters with W1 and w2 rounded to FP16 (what the GPU multiplies by)."""
    p = np.array(params, dtype=np.float64)
    p[:H * D] = p[:H * D].astype(np.float16).astype(np.float64)
    p[H * D + H:H * D + 2 * H] = p[H * D + H:H * D + 2 * H].astype(np.float16).astype(np.float64)
    return p


def patches(stat_map, cells):
    """Network inputs of the listed (m, b) cells of a [templates, bins] map."""
    M, NB = stat_map.shape
    out = np.zeros((len(cells), T, B))
    for k, (m, b) in enumerate(cells):
        for r in range(T):
            mm = m + r - T // 2
            if mm < 0 or mm >= M:
                continue
            for c in range(B):
                bb = b + c - B // 2
                if 0 <= bb < NB:
                    out[k, r, c] = np.arcsinh(stat_map[mm, bb])
    return out.reshape(len(cells), D)


def forward(X, params):
    W1, b1, w2, b2 = unpack(params)
    z1 = X @ W1.T + b1
    h = np.maximum(z1, 0.0)
    return h @ w2 + b2, z1


def loss(X, y, params):
    z, _ = forward(X, params)
    return float(np.mean(np.logaddexp(0.0, z) - y * z))


def grad(X, y, params):
    """Analytic gradient of `loss` with respect to the parameter vector."""
    W1, b1, w2, b2 = unpack(params)
    z, z1 = forward(X, params)
    n = X.shape[0]
    dz = (1.0 / (1.0 + np.exp(-z)) - y) / n
    h = np.maximum(z1, 0.0)
    g_w2 = h.T @ dz
    g_b2 = dz.sum()
    dh = np.outer(dz, w2) * (z1 > 0)
    g_W1 = dh.T @ X
    g_b1 = dh.sum(axis=0)
    return np.concatenate([g_W1.ravel(), g_b1, g_w2, [g_b2]])
