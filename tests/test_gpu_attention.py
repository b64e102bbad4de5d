"""Physics attention on the GPU (pfem_attn_forward, tcgen05 slice and deslice kernels) against
the FP64 oracle of the Method's subsection "Transolver".

Bars, from the kernel's storage precision (bf16, unit roundoff u = 2^-9; FP32 elsewhere):
  * against the oracle's steps with the kernel's bf16 roundings (X W_U and M before the sums,
    b_U added to the tokens, Z^t before the deslice, X^t on output): slice weights
    within one bf16 ulp (the FP32 logits and exponential may move a value across a rounding
    boundary), tokens Z and Z^t within rel L2 1e-3 (FP32 sums of up to 2^20 products,
    rounding flips), X^t within rel L2 2e-3;
  * against the plain FP64 oracle: X^t and Z within rel L2 1e-2 (four bf16 roundings in
    sequence, each at most u = 1.95e-3 relative, first order 4u = 7.8e-3).
Ragged tails (N not a multiple of the 128-point tile), N < 128, every supported token count
class (S <= 64 and S > 64, S not a multiple of 64), several head counts and scales, bitwise
repeatability, a full 2^20-point cloud checked through a closed form, and refused inputs.
"""

import numpy as np
import pytest
import torch

from oracle import attention as at
from pfem_inputs import attention as ai
from tests.gpu_util import pfem, rel_l2

pytestmark = pytest.mark.gpu

C = 128


def _bf16(t):
    return torch.tensor(np.asarray(t, np.float32), device="cuda").to(torch.bfloat16)


def _run(P, params, X, H, scale, tokens=True):
    attn = P.Attention(params, H, scale)
    out = attn.forward(_bf16(X), tokens=tokens)
    attn.sync()
    attn.close()
    if tokens:
        xt, m, z, zt = out
        return xt.float().cpu().numpy(), m.float().cpu().numpy(), z.cpu().numpy(), zt.cpu().numpy()
    return out.float().cpu().numpy()


def _emulated(X, params, H, scale):
    """The oracle's steps with the kernel's storage roundings: bf16 slice weights and X W_U
    (the bias of U joins the tokens after the weighted sums: a token's weights sum to its
    weight sum, so sum_I M_IJ (X_I W_U + b_U) / sum_I M_IJ = Z'_J + b_U), bf16 Z^t before the
    deslice and bf16 X^t."""
    r = ai.to_bf16_grid
    M = r(at.slice_weights(X, params["wm"], params["bm"]))
    U = r(at.affine(X, params["wu"], np.zeros_like(params["bu"])))
    Z = at.tokens(M, U) + params["bu"]
    Zt, _ = at.token_attention(Z, params, H, scale)
    return {"M": M, "Z": Z, "Zt": Zt, "Xt": r(at.deslice(M, r(Zt)))}


def _check(params, X, H, scale, got):
    xt, m, z, zt = got
    S = params["wm"].shape[1]
    ref = at.physics_attention(X, params, H, scale)
    emu = _emulated(X, params, H, scale)
    # slice weights: within one bf16 ulp of the emulated value (2^(e - 7) for a value in
    # [2^e, 2^(e+1))), pad columns exactly zero
    assert np.all(m[:, S:] == 0.0)
    ulp = 2.0 ** (np.floor(np.log2(np.maximum(np.abs(emu["M"]), 1e-30))) - 7)
    np.testing.assert_array_less(np.abs(m[:, :S] - emu["M"]), ulp * 1.0001 + 1e-12)
    assert rel_l2(z, emu["Z"]) <= 1e-3
    assert rel_l2(zt, emu["Zt"]) <= 1e-3
    assert rel_l2(xt, emu["Xt"]) <= 2e-3
    assert rel_l2(xt, ref["Xt"]) <= 1e-2
    assert rel_l2(z, ref["Z"]) <= 1e-2


@pytest.mark.parametrize("S,H,scale,N", [
    (128, 8, 1.0, 1000),     # 8 tiles, ragged tail of 104
    (64, 4, 0.25, 777),
    (32, 8, 1.0, 300),
    (48, 2, 1.0, 129),       # one point in the second tile
    (96, 16, 0.5, 2048),     # exact multiple of the tile
    (16, 8, 1.0, 77),        # fewer points than one tile
    (128, 8, 1.0, 1),
])
def test_attention_matches_oracle(S, H, scale, N):
    P = pfem()
    params = ai.layer_params(C, S, seed=S + N, slice_gain=4.0)
    X = ai.random_features(N, C, seed=N)
    _check(params, X, H, scale, _run(P, params, X, H, scale))


def test_attention_tpms_cloud_matches_oracle():
    """The 131,072 material points of a 64^3 gyroid cell with Fourier features, 128 tokens,
    8 heads: many tiles per CTA (the accumulated token sums, the M stores and the staging
    buffers of consecutive tiles)."""
    P = pfem()
    pts = ai.tpms_points(64)
    X = ai.point_features(pts, C, seed=3)
    params = ai.layer_params(C, 128, seed=5, slice_gain=4.0)
    _check(params, X, 8, 1.0, _run(P, params, X, 8, 1.0))


def test_attention_bitwise_repeatable():
    P = pfem()
    params = ai.layer_params(C, 64, seed=7, slice_gain=3.0)
    X = ai.random_features(50_000, C, seed=8)
    attn = P.Attention(params, 8, 1.0)
    xd = _bf16(X)
    a = [t.clone() for t in attn.forward(xd, tokens=True)]
    b = [t.clone() for t in attn.forward(xd, tokens=True)]
    attn.sync()
    for u, v in zip(a, b):
        assert torch.equal(u, v)
    attn.close()


def test_attention_full_cloud_uniform_slices():
    """2^20 points (the benchmark size) with zero slice weights: every weight is exactly 1/S,
    each token is the mean of U, and every output row is bf16(mean(U) W_v + b_v); checked
    against that closed form evaluated by the oracle's affine map, and all rows bitwise
    equal."""
    P = pfem()
    N, S = 1 << 20, 128
    params = ai.layer_params(C, S, seed=9)
    params["wm"] = np.zeros_like(params["wm"])
    params["bm"] = np.zeros_like(params["bm"])
    X = ai.random_features(N, C, seed=10)
    xt = _run(P, params, X, 8, 1.0, tokens=False)
    assert np.all(xt == xt[0])
    ubar = ai.to_bf16_grid(at.affine(X, params["wu"], np.zeros_like(params["bu"]))).mean(axis=0) + params["bu"]
    expect = at.affine(ubar[None, :], params["wv"], params["bv"])[0]
    assert rel_l2(xt[0], expect) <= 2e-3


def test_attention_refusals_and_empty():
    P = pfem()
    from paper_2601_03086_gb300._lib import PfemError

    params = ai.layer_params(C, 64, seed=11)
    with pytest.raises(PfemError, match="UNSUPPORTED"):
        P.Attention(ai.layer_params(64, 64, seed=1), 4)
    with pytest.raises(PfemError, match="UNSUPPORTED"):
        P.Attention(ai.layer_params(C, 40, seed=1), 4)
    with pytest.raises(PfemError, match="UNSUPPORTED"):
        P.Attention(params, 1)
    bad = dict(params, wq=params["wq"].copy())
    bad["wq"][0, 0] = np.nan
    with pytest.raises(PfemError, match="INVALID_ARG"):
        P.Attention(bad, 4)
    attn = P.Attention(params, 4)
    flat = torch.zeros(3 * C + 1, dtype=torch.bfloat16, device="cuda")
    xt = torch.empty((3, C), dtype=torch.bfloat16, device="cuda")
    from paper_2601_03086_gb300 import _lib
    import ctypes

    st = _lib.lib().pfem_attn_forward(attn.handle, 3, ctypes.c_void_p(flat.data_ptr() + 2),
                                      ctypes.c_void_p(xt.data_ptr()), None, None, None)
    assert _lib.STATUS[st] == "PFEM_ERR_INVALID_ARG"
    empty = attn.forward(torch.zeros((0, C), dtype=torch.bfloat16, device="cuda"))
    assert empty.shape == (0, C)
    attn.sync()
    attn.close()
