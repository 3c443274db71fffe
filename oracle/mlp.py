"""CPU oracle of the learned form's network and features (test
infrastructure only: tests, the smoke check and the benchmark's CPU baseline
may import it; the library never does).

The paper has no learned part; what is restated here is this library's own
definition of it, written from the mathematics in float64 numpy:

- BF16 rounding: a float32 value keeps its top 16 bits, rounded to nearest,
  ties to even (the IEEE rule applied at bit 16 of the float32 pattern).
- Network: z = w3 . relu(W2 relu(W1 x + b1) + b2) + b3, weights rounded to
  BF16, biases as given.
- Loss: mean binary cross-entropy with logits, mean(softplus(z) - y z).
- Gradient: backpropagation of that loss, the BF16 rounding taken as the
  identity (the gradient is with respect to the master values).
- Adam (Kingma and Ba 2015): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
  p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
- Features of a block-pair visit from the record of its previous visit (see
  ``features``).
"""
import numpy as np

F, H = 8, 64
OFF_W1 = 0
OFF_B1 = OFF_W1 + H * F
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H
PARAMS = OFF_B3 + 1


def bf16_round(x):
    """float32 values rounded to the nearest BF16 value (ties to even), as float64."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p, round_weights=True):
    p = np.asarray(p, dtype=np.float64)
    rw = (lambda w: bf16_round(w.astype(np.float32))) if round_weights else (lambda w: w)
    W1 = rw(p[OFF_W1:OFF_B1]).reshape(H, F)
    b1 = p[OFF_B1:OFF_W2]
    W2 = rw(p[OFF_W2:OFF_B2]).reshape(H, H)
    b2 = p[OFF_B2:OFF_W3]
    w3 = rw(p[OFF_W3:OFF_B3])
    b3 = p[OFF_B3]
    return W1, b1, W2, b2, w3, b3


def forward(p, X, round_weights=True):
    """Logits z for the rows of X (n x 8)."""
    W1, b1, W2, b2, w3, b3 = unpack(p, round_weights)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ w3 + b3


def loss_grad(p, X, y, round_weights=True):
    """(mean loss, gradient with respect to the parameter vector)."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = X.shape[0]
    W1, b1, W2, b2, w3, b3 = unpack(p, round_weights)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ w3 + b3
    loss = np.mean(np.logaddexp(0.0, z) - y * z)
    dz = (1.0 / (1.0 + np.exp(-z)) - y) / n
    g = np.zeros(PARAMS)
    g[OFF_W3:OFF_B3] = h2.T @ dz
    g[OFF_B3] = dz.sum()
    d2 = np.outer(dz, w3) * (a2 > 0)
    g[OFF_W2:OFF_B2] = (d2.T @ h1).ravel()
    g[OFF_B2:OFF_W3] = d2.sum(axis=0)
    d1 = (d2 @ W2) * (a1 > 0)
    g[OFF_W1:OFF_B1] = (d1.T @ X).ravel()
    g[OFF_B1:OFF_W2] = d1.sum(axis=0)
    return loss, g


def adam_step(p, m, v, g, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step; returns new (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def record(A, sg, b):
    """The visit record of a 2b x 2b pivot block A_P (Sec. 2) with signs sg:
    [max scaled |a_ij| over the I x J block, Frobenius norm of that scaled
    block, (rotations: filled by the caller), mean a_ii over I, mean a_jj over
    J, fraction of (i, j) in I x J with opposite signs]."""
    A = np.asarray(A, dtype=np.float64)
    d = np.diag(A)
    S = np.abs(A[:b, b:]) / np.sqrt(np.outer(d[:b], d[b:]))
    pi, pj = int((sg[:b] > 0).sum()), int((sg[b:] > 0).sum())
    return np.array([S.max(), np.sqrt((S * S).sum()), 0.0, d[:b].mean(), d[b:].mean(),
                     (pi * (b - pj) + (b - pi) * pj) / float(b * b)])


def features(rec, prev_skip, I, J, b, nb, sweep, max_sweeps, tol):
    """The 8 features of a visit of block columns I, J for sweep `sweep` from
    the record `rec` of its last computed visit (rec[2] = inner rotations)."""
    tiny = 1e-30
    return np.array([
        np.log2(max(rec[0], tiny) / tol) / 64.0,
        np.log2(max(rec[1], tiny)) / 64.0,
        rec[2] / float(b * b),
        sweep / float(max_sweeps),
        rec[5],
        np.log2(max(rec[3], tiny) / max(rec[4], tiny)) / 64.0,
        abs(I - J) / float(nb),
        float(prev_skip),
    ])
