"""FP64 CPU oracle of the physics-attention module of the Transolver backbone (Method,
subsection "Transolver": slice, token attention, deslice).

TEST INFRASTRUCTURE (see oracle/fem.py): only tests/, __graft_entry__.smoke() and bench.py's
CPU baseline may import it; it shares no code with the CUDA path.

Notation of the subsection: N points with C feature channels X (N x C), S physics-aware
tokens.
  * U = MLP_U(X) (N x C) and the slice logits MLP_M(X) (N x S), each MLP read as one affine
    map (the subsection gives no depth); M = softmax of the logits along the S axis.
  * Tokens Z_JK = sum_I M_IJ U_IK / sum_I M_IJ (S x C).  A token whose weight sum is exactly
    zero (every weight underflowed) is read as the zero token; the formula leaves it undefined.
  * Q, K, V = MLP(Z), again one affine map each; multi-head self-attention over the token
    axis: the C channels split into H heads of C/H channels and, per head,
    Z^t_h = softmax(scale * Q_h K_h^T) V_h.  The subsection prints softmax(Q K^T) with no
    scale (scale = 1 is the printed form); the scale is a parameter.
  * Deslice X^t_IK = sum_J M_IJ Z^t_JK (N x C), with the same weights M.
Weights are (in, out) matrices: an affine map is X @ W + b.

`rnd` (identity by default) is applied at the points where a kernel stores an intermediate
in a narrower type (U and M before the slice sums, Z^t before the deslice, X^t on output);
tests pass a rounding function there to emulate a storage precision.  It is not part of the
method.
"""

import numpy as np


def _ident(a):
    return a


def affine(X, W, b):
    """One affine layer X W + b (X: rows of inputs; W: (in, out); b: (out,))."""
    return np.asarray(X, np.float64) @ np.asarray(W, np.float64) + np.asarray(b, np.float64)


def softmax_rows(A):
    """Softmax of each row (subtracting the row maximum first)."""
    A = np.asarray(A, np.float64)
    e = np.exp(A - A.max(axis=-1, keepdims=True))
    return e / e.sum(axis=-1, keepdims=True)


def slice_weights(X, Wm, bm):
    """M = softmax over the S tokens of the slice logits (N x S)."""
    return softmax_rows(affine(X, Wm, bm))


def tokens(M, U):
    """Z = (M^T U) / (column sums of M), S x C; zero tokens where a column sum is zero."""
    num = M.T @ U
    den = M.sum(axis=0)
    safe = np.where(den > 0.0, den, 1.0)
    return np.where((den > 0.0)[:, None], num / safe[:, None], 0.0)


def token_attention(Z, P, n_heads, scale=1.0):
    """Multi-head self-attention along the token axis: per head h (channels h*d..(h+1)*d-1,
    d = C / n_heads), softmax(scale * Q_h K_h^T) V_h.  Returns (Z^t, (Q, K, V))."""
    Q = affine(Z, P["wq"], P["bq"])
    K = affine(Z, P["wk"], P["bk"])
    V = affine(Z, P["wv"], P["bv"])
    C = Z.shape[1]
    if C % n_heads:
        raise ValueError("channels must split evenly into heads")
    d = C // n_heads
    Zt = np.empty_like(Q)
    for h in range(n_heads):
        cols = slice(h * d, (h + 1) * d)
        A = softmax_rows(scale * (Q[:, cols] @ K[:, cols].T))
        Zt[:, cols] = A @ V[:, cols]
    return Zt, (Q, K, V)


def deslice(M, Zt):
    """X^t = M Z^t (N x C)."""
    return M @ Zt


def physics_attention(X, P, n_heads, scale=1.0, rnd=None):
    """The module's forward pass.  P holds wu (C x C), bu (C), wm (C x S), bm (S), wq, wk, wv
    (C x C) and bq, bk, bv (C).  Returns a dict with U, M, Z, Zt and Xt."""
    r = _ident if rnd is None else rnd
    X = np.asarray(X, np.float64)
    U = r(affine(X, P["wu"], P["bu"]))
    M = r(slice_weights(X, P["wm"], P["bm"]))
    if X.shape[0] == 0:
        S, C = np.asarray(P["wm"]).shape[1], X.shape[1]
        return {"U": U, "M": M, "Z": np.zeros((S, C)), "Zt": np.zeros((S, C)), "Xt": np.zeros((0, C))}
    Z = tokens(M, U)
    Zt, _ = token_attention(Z, P, n_heads, scale)
    Xt = r(deslice(M, r(Zt)))
    return {"U": U, "M": M, "Z": Z, "Zt": Zt, "Xt": Xt}
