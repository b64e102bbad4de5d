"""Pins of the physics-attention oracle (Method, subsection "Transolver") to facts other than
its own formulas: brute-force sums on tiny inputs, closed forms of degenerate slicings and
attentions, the symmetries the weighted averages imply, and library attention/softmax.
A dropped normalisation, a transposed weight or a head split on the wrong axis fails one of
them."""

import numpy as np
import pytest
import scipy.special

from oracle import attention as at
from pfem_inputs import attention as ai


def _params(C, S, seed, gain=1.0):
    return ai.layer_params(C, S, seed, slice_gain=gain)


def test_brute_force_loops_tiny():
    """Every sum of the slice / attend / deslice written as explicit loops on N=5, C=4, S=3,
    two heads."""
    C, S, N, H = 4, 3, 5, 2
    P = _params(C, S, 1, gain=3.0)
    X = ai.random_features(N, C, 2)
    out = at.physics_attention(X, P, H, scale=0.7)
    U = [[P["bu"][k] + sum(X[i, c] * P["wu"][c, k] for c in range(C)) for k in range(C)] for i in range(N)]
    M = []
    for i in range(N):
        lg = [P["bm"][j] + sum(X[i, c] * P["wm"][c, j] for c in range(C)) for j in range(S)]
        e = [np.exp(v) for v in lg]
        M.append([v / sum(e) for v in e])
    Z = [[sum(M[i][j] * U[i][k] for i in range(N)) / sum(M[i][j] for i in range(N)) for k in range(C)]
         for j in range(S)]
    proj = {}
    for nm in ("q", "k", "v"):
        proj[nm] = [[P["b" + nm][k] + sum(Z[j][c] * P["w" + nm][c, k] for c in range(C)) for k in range(C)]
                    for j in range(S)]
    d = C // H
    Zt = [[0.0] * C for _ in range(S)]
    for h in range(H):
        for a in range(S):
            sc = [0.7 * sum(proj["q"][a][h * d + t] * proj["k"][b][h * d + t] for t in range(d)) for b in range(S)]
            w = [np.exp(v) for v in sc]
            w = [v / sum(w) for v in w]
            for t in range(d):
                Zt[a][h * d + t] = sum(w[b] * proj["v"][b][h * d + t] for b in range(S))
    Xt = [[sum(M[i][j] * Zt[j][k] for j in range(S)) for k in range(C)] for i in range(N)]
    np.testing.assert_allclose(out["U"], U, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(out["M"], M, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(out["Z"], Z, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(out["Zt"], Zt, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(out["Xt"], Xt, rtol=1e-12, atol=1e-14)


def test_single_token_closed_form():
    """S = 1: every weight is 1, the token is the mean of U, attention over one token returns
    its value row, so every output row is mean(U) W_v + b_v."""
    C, N = 8, 37
    P = _params(C, 1, 3)
    X = ai.random_features(N, C, 4)
    out = at.physics_attention(X, P, 2)
    ubar = (X @ P["wu"] + P["bu"]).mean(axis=0)
    expect = ubar @ P["wv"] + P["bv"]
    np.testing.assert_allclose(out["Xt"], np.tile(expect, (N, 1)), rtol=1e-12, atol=1e-13)


def test_uniform_slices_closed_form():
    """Zero slice weights: M = 1/S everywhere, every token equals mean(U), all attention rows
    are identical, and every output row is mean(U) W_v + b_v whatever W_q, W_k."""
    C, S, N = 8, 6, 50
    P = _params(C, S, 5)
    P["wm"] = np.zeros_like(P["wm"])
    P["bm"] = np.zeros_like(P["bm"])
    X = ai.random_features(N, C, 6)
    out = at.physics_attention(X, P, 4, scale=3.0)
    np.testing.assert_allclose(out["M"], 1.0 / S, rtol=1e-15)
    ubar = (X @ P["wu"] + P["bu"]).mean(axis=0)
    np.testing.assert_allclose(out["Z"], np.tile(ubar, (S, 1)), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(out["Xt"], np.tile(ubar @ P["wv"] + P["bv"], (N, 1)), rtol=1e-12, atol=1e-13)


def test_hard_slices_are_cluster_means():
    """Slice logits scaled up until the softmax is one-hot: each token is the plain mean of U
    over the points whose largest logit is that token (computed by boolean selection)."""
    C, S, N = 8, 4, 200
    P = _params(C, S, 7)
    X = ai.random_features(N, C, 8)
    logits = X @ P["wm"] + P["bm"]
    top = np.sort(logits, axis=1)
    assert (top[:, -1] - top[:, -2]).min() > 1e-4
    Q = dict(P, wm=P["wm"] * 1e7, bm=P["bm"] * 1e7)
    out = at.physics_attention(X, Q, 2)
    U = X @ P["wu"] + P["bu"]
    lab = logits.argmax(axis=1)
    for j in range(S):
        np.testing.assert_allclose(out["Z"][j], U[lab == j].mean(axis=0), rtol=1e-10, atol=1e-12)
    np.testing.assert_array_equal(out["M"].argmax(axis=1), lab)


def test_point_permutation_and_duplication():
    """The tokens are weighted averages over points: permuting the points permutes the output
    rows and leaves the tokens; listing every point twice leaves the tokens and repeats the
    output rows."""
    C, S, N = 16, 8, 90
    P = _params(C, S, 9, gain=2.0)
    X = ai.random_features(N, C, 10)
    a = at.physics_attention(X, P, 4, scale=0.25)
    perm = np.random.default_rng(11).permutation(N)
    b = at.physics_attention(X[perm], P, 4, scale=0.25)
    np.testing.assert_allclose(b["Z"], a["Z"], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(b["Xt"], a["Xt"][perm], rtol=1e-12, atol=1e-13)
    c = at.physics_attention(np.concatenate([X, X]), P, 4, scale=0.25)
    np.testing.assert_allclose(c["Z"], a["Z"], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(c["Xt"], np.concatenate([a["Xt"], a["Xt"]]), rtol=1e-12, atol=1e-13)


def test_softmax_shift_invariance_and_rows():
    """A constant added to every slice bias changes nothing; M rows are scipy's softmax."""
    C, S, N = 8, 5, 30
    P = _params(C, S, 12)
    X = ai.random_features(N, C, 13)
    a = at.physics_attention(X, P, 2)
    b = at.physics_attention(X, dict(P, bm=P["bm"] + 17.0), 2)
    np.testing.assert_allclose(b["Xt"], a["Xt"], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(a["M"], scipy.special.softmax(X @ P["wm"] + P["bm"], axis=1), rtol=1e-13)


def test_token_attention_matches_library_attention():
    """The multi-head token attention equals torch's scaled_dot_product_attention (FP64,
    heads as a batch axis) on the same Q, K, V."""
    torch = pytest.importorskip("torch")
    C, S, H = 32, 12, 4
    P = _params(C, S, 14)
    Z = ai.random_features(S, C, 15)
    Zt, (Q, K, V) = at.token_attention(Z, P, H, scale=0.3)
    d = C // H

    def heads(A):
        return torch.tensor(A).reshape(S, H, d).permute(1, 0, 2)

    ref = torch.nn.functional.scaled_dot_product_attention(heads(Q), heads(K), heads(V), scale=0.3)
    np.testing.assert_allclose(Zt, ref.permute(1, 0, 2).reshape(S, C).numpy(), rtol=1e-12, atol=1e-13)


def test_zero_query_attention_is_value_mean():
    """W_q = 0, b_q = 0: every attention row is uniform, so every transformed token is the
    mean of the value rows of its head."""
    C, S = 8, 7
    P = _params(C, S, 16)
    P["wq"] = np.zeros_like(P["wq"])
    P["bq"] = np.zeros_like(P["bq"])
    Z = ai.random_features(S, C, 17)
    Zt, (_, _, V) = at.token_attention(Z, P, 2, scale=5.0)
    np.testing.assert_allclose(Zt, np.tile(V.mean(axis=0), (S, 1)), rtol=1e-12, atol=1e-13)


def test_empty_cloud_and_zero_weight_tokens():
    """N = 0 gives an empty output; a token whose weights all underflow is the zero token."""
    C, S = 8, 3
    P = _params(C, S, 18)
    out = at.physics_attention(np.zeros((0, C)), P, 2)
    assert out["Xt"].shape == (0, C)
    M = np.array([[1.0, 0.0, 0.0], [0.5, 0.5, 0.0]])
    U = np.arange(2 * C, dtype=float).reshape(2, C)
    Z = at.tokens(M, U)
    np.testing.assert_array_equal(Z[2], 0.0)
    np.testing.assert_allclose(Z[1], U[1])
    np.testing.assert_allclose(Z[0], (U[0] + 0.5 * U[1]) / 1.5)


def test_bf16_grid_helper():
    """The input helper rounds to the nearest bfloat16 with ties to even."""
    v = np.array([1.0, 1.00390625, 1.005859375, 1.01171875, -3.14159, 0.0])
    np.testing.assert_array_equal(ai.to_bf16_grid(v), [1.0, 1.0, 1.0078125, 1.015625, -3.140625, 0.0])
    np.testing.assert_array_equal(ai.bf16_bits(np.array([1.0, -2.0])), [0x3F80, 0xC000])
