"""Seeded synthetic inputs for the hyperbolic SVD (G, J).

This module only draws random matrices; it holds none of the method's
arithmetic, so both the CUDA path and the CPU oracle may take their inputs
from it.  Every generator takes an explicit seed and returns a column-major
float64 ``G`` (m x n) and an int8 signature vector ``J`` (+1 / -1 per column).

Shapes follow the paper's workloads (square factors of an indefinite matrix,
Sec. 5) and the five measured configurations:

=========  ===============================================================
gaussian   G i.i.d. N(0,1), J = diag(+1 x p, -1 x (n-p))
graded     G = B diag(10^(-decades*i/n)), B i.i.d. N(0,1) (graded columns)
haar       G = Q1 diag(sigma) Q2, Q Haar orthogonal, sigma log-uniform
batch      many small square N(0,1) factors of uneven order, random J
paper      the spectrum shape of the paper's test matrices (Sec. 5,
           Table 5.2): lambda uniform on [-a,-a 1e-5) U (a 1e-5, a],
           G = Q |Lambda|^(1/2) K with K J-unitary, so sigma = sqrt|lambda|
           is known by construction
wide       a wide factor (m < n, Sec. 1: its transpose is tall) with the
           same spectrum shape: G = Q |Lambda|^(1/2) [I 0] K, K J-unitary,
           so G J G^T = Q Lambda Q^T is known by construction
=========  ===============================================================
"""
import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _pow10(exponents):
    """10**x rounded to float64 through 40-digit decimal arithmetic, so the
    bytes do not depend on the platform's libm (its pow() may differ in the
    last bit between machines)."""
    import decimal

    ctx = decimal.Context(prec=40)
    ten = decimal.Decimal(10)
    return np.array([float(ctx.power(ten, decimal.Decimal(repr(float(x))))) for x in exponents])


def _haar(rng, n):
    """Haar-distributed orthogonal matrix: QR of a Gaussian matrix with the
    signs of R's diagonal moved into Q."""
    X = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(X)
    Q *= np.sign(np.diag(R))[None, :]
    return Q


def signs_block(n, p):
    """J = diag(+1 x p, -1 x (n - p))."""
    J = -np.ones(n, dtype=np.int8)
    J[:p] = 1
    return J


def signs_random(rng, n, p):
    """J with exactly p entries +1 at random positions."""
    J = -np.ones(n, dtype=np.int8)
    J[rng.permutation(n)[:p]] = 1
    return J


def gaussian(n, m=None, p=None, seed=1):
    """G i.i.d. N(0,1) (m x n), J = diag(+1 x p, -1 x (n-p)); p defaults to n/2."""
    rng = _rng(seed)
    m = n if m is None else m
    p = n // 2 if p is None else p
    G = np.asfortranarray(rng.standard_normal((m, n)))
    return G, signs_block(n, p)


def graded(n, decades=6.0, m=None, p=None, seed=2):
    """G = B diag(10^(-decades*i/n)), i = 0..n-1, B i.i.d. N(0,1)."""
    rng = _rng(seed)
    m = n if m is None else m
    p = n // 2 if p is None else p
    B = rng.standard_normal((m, n))
    scale = _pow10(-decades * np.arange(n) / n)
    G = np.asfortranarray(B * scale[None, :])
    return G, signs_block(n, p)


def haar(n, lo=1e-6, hi=1.0, p=None, seed=3):
    """G = Q1 diag(sigma) Q2, sigma log-uniform on [lo, hi], J with p random +1."""
    rng = _rng(seed)
    p = n // 2 if p is None else p
    Q1 = _haar(rng, n)
    Q2 = _haar(rng, n)
    sigma = _pow10(rng.uniform(np.log10(lo), np.log10(hi), size=n))
    G = np.asfortranarray((Q1 * sigma[None, :]) @ Q2)
    return G, signs_random(rng, n, p)


def batch(count, nmin=16, nmax=256, seed=4):
    """``count`` square N(0,1) factors, n uniform on [nmin, nmax], each with a
    random number p in [0, n] of +1 signs at random positions.  Returns a list
    of (G, J)."""
    rng = _rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        p = int(rng.integers(0, n + 1))
        G = np.asfortranarray(rng.standard_normal((n, n)))
        out.append((G, signs_random(rng, n, p)))
    return out


def paper_a(n):
    """Spectrum half-width a used for order n in the paper's tests (Table 5.2)."""
    if n <= 3168:
        return 20.0
    if n <= 6368:
        return 30.0
    if n <= 9568:
        return 40.0
    return 50.0


def paper(n, p=None, tanh_max=0.5, mixes=2, seed=6):
    """Known-answer factor: G = Q diag(sqrt|lambda|) K with Q Haar orthogonal
    and K a product of random J-unitary plane rotations (trigonometric inside
    a sign group, hyperbolic with |tanh| <= tanh_max across groups), so the
    hyperbolic singular values are sqrt|lambda| by construction and V = K^T.

    Returns (G, J, sigma_true)."""
    rng = _rng(seed)
    p = n // 2 if p is None else p
    a = paper_a(n)
    mag = rng.uniform(a * 1e-5, a, size=n)
    lam = np.concatenate([mag[:p], -mag[p:]])
    J = np.where(lam > 0, 1, -1).astype(np.int8)
    sigma = np.sqrt(np.abs(lam))
    K = np.eye(n)
    for _ in range(mixes):
        perm = rng.permutation(n)
        for k in range(0, n - 1, 2):
            i, j = perm[k], perm[k + 1]
            if J[i] == J[j]:
                phi = rng.uniform(-np.pi, np.pi)
                c, s = np.cos(phi), np.sin(phi)
                R = np.array([[c, s], [-s, c]])
            else:
                th = rng.uniform(-tanh_max, tanh_max)
                ch = 1.0 / np.sqrt(1.0 - th * th)
                R = np.array([[ch, th * ch], [th * ch, ch]])
            K[[i, j], :] = R @ K[[i, j], :]
    Q = _haar(rng, n)
    G = np.asfortranarray((Q * sigma[None, :]) @ K)
    return G, J, sigma


def wide(m, n, p=None, tanh_max=0.5, mixes=2, seed=9):
    """Known-answer wide factor G (m x n, m <= n): K (n x n) a product of
    random J-unitary plane rotations (trigonometric inside a sign group,
    hyperbolic with |tanh| <= tanh_max across groups), so K J K^T = J and
    G = Q diag(sqrt|lambda|) K[:m, :] gives G J G^T = Q diag(lambda) Q^T with
    lambda_j = |lambda_j| J_j for the first m positions of J (random signs,
    p of the n positive).

    Returns (G, J, lambda_true) with lambda_true sorted ascending."""
    rng = _rng(seed)
    p = n // 2 if p is None else p
    J = signs_random(rng, n, p)
    a = paper_a(m)
    mag = rng.uniform(a * 1e-5, a, size=m)
    K = np.eye(n)
    for _ in range(mixes):
        perm = rng.permutation(n)
        for k in range(0, n - 1, 2):
            i, j = perm[k], perm[k + 1]
            if J[i] == J[j]:
                phi = rng.uniform(-np.pi, np.pi)
                c, s = np.cos(phi), np.sin(phi)
                R = np.array([[c, s], [-s, c]])
            else:
                th = rng.uniform(-tanh_max, tanh_max)
                ch = 1.0 / np.sqrt(1.0 - th * th)
                R = np.array([[ch, th * ch], [th * ch, ch]])
            K[[i, j], :] = R @ K[[i, j], :]
    Q = _haar(rng, m)
    G = np.asfortranarray((Q * np.sqrt(mag)[None, :]) @ K[:m, :])
    lam = np.sort(mag * J[:m].astype(np.float64))
    return G, J, lam
