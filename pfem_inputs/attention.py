"""Seeded inputs for the physics-attention module: point-feature matrices and random layer
weights (no trained weights exist), every value exactly representable in bfloat16 so that a
kernel that stores bf16 and the FP64 oracle start from identical numbers.  Nothing here
evaluates the module."""

import numpy as np

from .problems import _TPMS


def to_bf16_grid(a):
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    x = np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))
    bits = x.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits(a):
    """The bfloat16 bit patterns (uint16) of values already on the bf16 grid."""
    x = np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))
    return (x.view(np.uint32) >> 16).astype(np.uint16)


def layer_params(C, S, seed, slice_gain=1.0):
    """Weights of one physics-attention module, PyTorch-Linear-style uniform(+-1/sqrt(C))
    initialisation; the slice logits' weights scaled by slice_gain (sharper slices for
    gain > 1).  Keys wu, bu, wm, bm, wq, bq, wk, bk, wv, bv; weights are (in, out)."""
    rng = np.random.default_rng(seed)
    a = 1.0 / np.sqrt(C)

    def u(*shape, g=1.0):
        return to_bf16_grid(g * rng.uniform(-a, a, shape))

    return {"wu": u(C, C), "bu": u(C), "wm": u(C, S, g=slice_gain), "bm": u(S, g=slice_gain),
            "wq": u(C, C), "bq": u(C), "wk": u(C, C), "bk": u(C), "wv": u(C, C), "bv": u(C)}


def point_features(points, C, seed, extra=None):
    """Feature rows for a point cloud: C random Fourier features of the coordinates (and of
    `extra` per-point scalars, e.g. a material value), each row shifted and scaled to zero
    mean and unit variance the way a LayerNorm leaves its output; bf16 grid."""
    rng = np.random.default_rng(seed)
    P = np.asarray(points, np.float64)
    if extra is not None:
        P = np.concatenate([P, np.asarray(extra, np.float64).reshape(P.shape[0], -1)], axis=1)
    w = rng.normal(0.0, 2.0 * np.pi, (P.shape[1], C))
    ph = rng.uniform(0.0, 2.0 * np.pi, C)
    F = np.sin(P @ w + ph)
    F -= F.mean(axis=1, keepdims=True)
    F /= np.sqrt((F * F).mean(axis=1, keepdims=True) + 1e-6)
    return to_bf16_grid(F)


def random_features(N, C, seed):
    """N x C standard-normal features on the bf16 grid (small and ragged test cases)."""
    return to_bf16_grid(np.random.default_rng(seed).standard_normal((N, C)))


def tpms_points(n=64, family="gyroid", c=0.0):
    """Material points of a TPMS cell of n^3 voxels: the centres of the solid voxels
    (level set above c) in the unit cube, the point cloud the homogenisation backbone reads."""
    centres = (np.arange(n) + 0.5) / n
    X, Y, Z = np.meshgrid(centres, centres, centres, indexing="ij")
    solid = _TPMS[family](X, Y, Z) > c
    return np.stack([X[solid], Y[solid], Z[solid]], axis=1)
