"""Structured and voxel-masked simplex meshes (topology and coordinates only)."""

import itertools

import numpy as np

# Kuhn (Freudenthal) split of a hex into 6 tetrahedra sharing the diagonal from local
# vertex 0 = (0,0,0) to vertex 7 = (1,1,1); local vertex id = i + 2 j + 4 k. Every hex
# uses the same diagonal direction, so neighbouring hexes meet on matching triangles.
_KUHN_TETS = []
for _perm in itertools.permutations(range(3)):
    _a = 1 << _perm[0]
    _b = _a | (1 << _perm[1])
    _KUHN_TETS.append((0, _a, _b, 7))
_KUHN_TETS = np.array(_KUHN_TETS, dtype=np.int64)

# Square split along the diagonal (0,0) -> (1,1); local vertex id = i + 2 j.
_SQUARE_TRIS = np.array([(0, 1, 3), (0, 3, 2)], dtype=np.int64)


def grid_tri(nx, ny, lx=1.0, ly=1.0, keep=None):
    """P1 triangles on an nx x ny grid of squares over [0,lx] x [0,ly].

    keep: optional bool array (nx, ny); squares with keep=False are removed and unused
    nodes are dropped (remaining nodes keep lexicographic order).
    Returns coords (N,2) float64, conn (E,3) int32.
    """
    xs = np.linspace(0.0, lx, nx + 1)
    ys = np.linspace(0.0, ly, ny + 1)
    gx, gy = np.meshgrid(xs, ys, indexing="ij")
    coords = np.stack([gx.ravel(order="F"), gy.ravel(order="F")], axis=1)
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    i = i.ravel(order="F")
    j = j.ravel(order="F")
    if keep is not None:
        sel = np.asarray(keep, dtype=bool)[i, j]
        i, j = i[sel], j[sel]
    stride = nx + 1
    corner = np.stack([i + stride * j, i + 1 + stride * j, i + stride * (j + 1), i + 1 + stride * (j + 1)], axis=1)
    conn = corner[:, _SQUARE_TRIS].reshape(-1, 3)
    return _compact(coords, conn)


def grid_tet(nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, keep=None, h=None):
    """P1 tetrahedra from an nx x ny x nz grid of hexes (6 Kuhn tets per hex).

    The box is [0,lx] x [0,ly] x [0,lz]; if h is given, the box is [0,nx h] x ... instead.
    keep: optional bool array (nx, ny, nz) of hexes to keep (voxel masking).
    Node numbering is lexicographic (x fastest); element order is hex-major.
    Returns coords (N,3) float64, conn (E,4) int32.
    """
    if h is not None:
        lx, ly, lz = nx * h, ny * h, nz * h
    xs = np.linspace(0.0, lx, nx + 1)
    ys = np.linspace(0.0, ly, ny + 1)
    zs = np.linspace(0.0, lz, nz + 1)
    gx, gy, gz = np.meshgrid(xs, ys, zs, indexing="ij")
    coords = np.stack([gx.ravel(order="F"), gy.ravel(order="F"), gz.ravel(order="F")], axis=1)
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    i = i.ravel(order="F")
    j = j.ravel(order="F")
    k = k.ravel(order="F")
    if keep is not None:
        sel = np.asarray(keep, dtype=bool)[i, j, k]
        i, j, k = i[sel], j[sel], k[sel]
    sx = nx + 1
    sxy = (nx + 1) * (ny + 1)
    base = i + sx * j + sxy * k
    offs = np.array([(v & 1) + sx * ((v >> 1) & 1) + sxy * ((v >> 2) & 1) for v in range(8)], dtype=np.int64)
    corner = base[:, None] + offs[None, :]
    conn = corner[:, _KUHN_TETS].reshape(-1, 4)
    return _compact(coords, conn)


def _compact(coords, conn):
    used = np.zeros(coords.shape[0], dtype=bool)
    used[conn.ravel()] = True
    if used.all():
        return coords.copy(), conn.astype(np.int32)
    new_id = np.cumsum(used) - 1
    return coords[used].copy(), new_id[conn].astype(np.int32)


def bbox(coords):
    return coords.min(axis=0), coords.max(axis=0)


def boundary_facets(coords, conn, axis=None, value=None, tol=1e-9):
    """Boundary facets (edges of triangles / faces of tets used by exactly one element).

    If axis/value are given, keep only facets whose nodes all satisfy
    |coords[:, axis] - value| <= tol. Returns (F, dim) int32.
    """
    nv = conn.shape[1]
    if axis is not None:
        # keep only elements with at least nv-1 nodes on the plane, then their on-plane faces
        # (all copies of a face share its nodes, so counting among them is exact)
        on_node = np.abs(coords[:, axis] - value) <= tol
        conn = conn[on_node[conn].sum(axis=1) >= nv - 1]
    faces = np.concatenate([np.delete(conn, a, axis=1) for a in range(nv)], axis=0)
    if axis is not None:
        faces = faces[np.all(on_node[faces], axis=1)]
    if faces.shape[0] == 0:
        return np.zeros((0, nv - 1), dtype=np.int32)
    key = np.sort(faces, axis=1)
    _, inv, counts = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    inv = inv.ravel()
    return faces[counts[inv] == 1].astype(np.int32)


def jitter_nodes(coords, conn, amount, h, rng, fixed=None):
    """Move nodes by uniform noise in [-amount*h, amount*h] per coordinate.

    Nodes on the bounding box (or with fixed[n]=True) stay put so faces stay planar.
    Raises if any simplex changes orientation sign or collapses.
    """
    lo, hi = bbox(coords)
    on_box = np.any((np.abs(coords - lo) < 1e-12) | (np.abs(coords - hi) < 1e-12), axis=1)
    if fixed is not None:
        on_box |= fixed
    noise = rng.uniform(-amount * h, amount * h, size=coords.shape)
    noise[on_box] = 0.0
    new = coords + noise
    s0 = _signed_measure(coords, conn)
    s1 = _signed_measure(new, conn)
    if np.any(np.sign(s0) != np.sign(s1)) or np.any(np.abs(s1) < 0.05 * np.abs(s0)):
        raise ValueError("jitter too large: an element inverted or collapsed")
    return new


def _signed_measure(coords, conn):
    # Orientation check only (sign and rough size of the simplex), used by the generator.
    x = coords[conn]
    d = x[:, 1:, :] - x[:, :1, :]
    return np.linalg.det(d)


def permute_mesh(coords, conn, rng, mask=None, values=None):
    """Random node renumbering, element reordering and per-element corner rotation.

    Returns new (coords, conn, node_perm) where new node i is old node node_perm[i];
    mask/values (per-node arrays) are permuted alongside if given and appended.
    """
    n = coords.shape[0]
    perm = rng.permutation(n)
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    conn2 = inv[conn]
    conn2 = conn2[rng.permutation(conn2.shape[0])]
    nv = conn2.shape[1]
    shift = rng.integers(0, nv, size=conn2.shape[0])
    idx = (np.arange(nv)[None, :] + shift[:, None]) % nv
    conn2 = np.take_along_axis(conn2, idx, axis=1)
    out = [coords[perm].copy(), conn2.astype(np.int32), perm]
    if mask is not None:
        out.append(mask[perm].copy())
    if values is not None:
        out.append(values[perm].copy())
    return tuple(out)
