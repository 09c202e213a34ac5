"""Element algebra and matrix products from their definitions (oracle; test only).

Tropical semiring, Eq. 2:  x (+) y = max(x, y),  x (.) y = x + y,
zero element -inf, unit element 0.

Counting tuples, Sec. II (the equation after Eq. 3):
  (x1, n1) (.) (x2, n2) = (x1 + x2, n1 * n2)
  (x1, n1) (+) (x2, n2) = (x1, n1 + n2) if x1 == x2,
                          (x1, n1)      if x1 >  x2,
                          (x2, n2)      if x1 <  x2.
"""
import numpy as np

NEG_INF = -np.inf


def t_add(x, y):
    return np.maximum(x, y)


def t_mul(x, y):
    return x + y


def c_mul(a, b):
    """Counting-tuple product of (x, n) pairs (arrays broadcast)."""
    return a[0] + b[0], a[1] * b[1]


def c_add(a, b):
    """Counting-tuple sum of (x, n) pairs, element-wise, following the three cases."""
    x1, n1 = a
    x2, n2 = b
    x = np.maximum(x1, x2)
    n = np.where(x1 == x2, n1 + n2, np.where(x1 > x2, n1, n2))
    return x, n


def maxplus_matmul(A, B):
    """C[..., m, n] = max_k (A[..., m, k] + B[..., k, n]), batched over leading axes.

    Plain definition by broadcasting; the sum is taken in A's dtype (float64
    for reals, int64 for integers), then max-reduced over k.
    """
    A = np.asarray(A)
    B = np.asarray(B)
    return np.max(A[..., :, :, None] + B[..., None, :, :], axis=-2)


def counting_matmul(Ax, An, Bx, Bn, mod=None):
    """Counting-tuple matrix product, folding (+) over k in increasing order.

    Counts are Python integers (object arrays) unless ``mod`` is given, in which
    case every product and sum is reduced modulo ``mod``.
    """
    Ax, Bx = np.asarray(Ax), np.asarray(Bx)
    An = np.asarray(An, dtype=object)
    Bn = np.asarray(Bn, dtype=object)
    K = Ax.shape[-1]
    x = None
    for k in range(K):
        tx, tn = c_mul((Ax[..., :, k, None], An[..., :, k, None]),
                       (Bx[..., None, k, :], Bn[..., None, k, :]))
        if mod is not None:
            tn = tn % mod
        if x is None:
            x, n = tx, tn
        else:
            x, n = c_add((x, n), (tx, tn))
            if mod is not None:
                n = n % mod
    return x, n
