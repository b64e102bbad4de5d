"""Workload builders: the five benchmark problems, scaled variants and warm-start inputs.

Every random draw is seeded; the recipe of each workload is spelled out in its docstring.
Nothing here evaluates the finite-element operator.
"""

import math

import numpy as np

from .meshes import boundary_facets, grid_tet, grid_tri, jitter_nodes, permute_mesh, bbox


def _problem(dim, coords, conn, kind, mat_a, mat_b, mask, values, facets, traction, name, seed, f_extra=None):
    return dict(
        dim=dim,
        coords=np.ascontiguousarray(coords, dtype=np.float64),
        conn=np.ascontiguousarray(conn, dtype=np.int32),
        kind=kind,
        mat_a=np.ascontiguousarray(mat_a, dtype=np.float64),
        mat_b=np.ascontiguousarray(mat_b, dtype=np.float64),
        dirichlet_mask=np.ascontiguousarray(mask, dtype=np.uint8),
        dirichlet_values=np.ascontiguousarray(values, dtype=np.float64),
        facets=np.ascontiguousarray(facets, dtype=np.int32).reshape(-1, dim),
        traction=np.ascontiguousarray(traction, dtype=np.float64).reshape(-1, dim),
        f_ext_extra=f_extra,
        name=name,
        seed=seed,
    )


def _face_mask(coords, axis, value, tol=1e-9):
    return np.abs(coords[:, axis] - value) <= tol


# ---------------------------------------------------------------------------------------
# Benchmark problems
# ---------------------------------------------------------------------------------------


def cfg1_plate(n=32):
    """2-D plane-strain plate: unit square, (n+1)^2 nodes, 2 n^2 P1 triangles.

    E = 1, nu = 0.3 everywhere; left edge (x=0) u = 0; right edge (x=1) traction (1, 0).
    n = 32 gives 33 x 33 nodes and 2048 triangles.
    """
    coords, conn = grid_tri(n, n)
    ne = conn.shape[0]
    mask = np.zeros(coords.shape, dtype=np.uint8)
    mask[_face_mask(coords, 0, 0.0)] = 1
    facets = boundary_facets(coords, conn, axis=0, value=1.0)
    traction = np.tile([1.0, 0.0], (facets.shape[0], 1))
    return _problem(2, coords, conn, "linear", np.full(ne, 1.0), np.full(ne, 0.3), mask,
                    np.zeros(coords.shape), facets, traction, f"plate2d_{n}x{n}", 1)


def cube_problem(n, seed, traction_z=-0.1, jitter=0.0):
    """3-D linear-elastic unit cube: n^3 hexes x 6 Kuhn tets, (n+1)^3 nodes.

    Per element E = exp(0.5 * N(0,1)) (lognormal(0, 0.5)) and nu ~ U[0.25, 0.35], drawn
    iid with numpy's default_rng(seed) in element order (E first, then nu).
    z=0 face: all DOFs fixed at 0. z=1 face: traction (0, 0, traction_z).
    """
    coords, conn = grid_tet(n, n, n)
    rng = np.random.default_rng(seed)
    ne = conn.shape[0]
    E = np.exp(0.5 * rng.standard_normal(ne))
    nu = rng.uniform(0.25, 0.35, ne)
    if jitter > 0:
        coords = jitter_nodes(coords, conn, jitter, 1.0 / n, np.random.default_rng(seed + 1000))
    mask = np.zeros(coords.shape, dtype=np.uint8)
    mask[_face_mask(coords, 2, 0.0)] = 1
    facets = boundary_facets(coords, conn, axis=2, value=1.0)
    traction = np.tile([0.0, 0.0, traction_z], (facets.shape[0], 1))
    return _problem(3, coords, conn, "linear", E, nu, mask, np.zeros(coords.shape), facets, traction,
                    f"cube_{n}^3x6", seed)


def cfg2_cube():
    """40^3 hexes -> 384,000 tets, 68,921 nodes, lognormal E (seed 2)."""
    return cube_problem(40, 2)


def bar_problem(nx, ny, nz, seed, stretch=0.2, length=4.0):
    """3-D compressible Neo-Hookean bar [0,length] x [0,1] x [0,1], nx x ny x nz hexes x 6 tets.

    mu = 1 (1 + U[-0.2,0.2]), lambda = 4 (1 + U[-0.2,0.2]) per element, drawn with
    default_rng(seed) in element order (mu factors first, then lambda factors).
    x=0 face clamped; x=length face gripped: u = (stretch*length, 0, 0) at full load.
    """
    coords, conn = grid_tet(nx, ny, nz, length, 1.0, 1.0)
    rng = np.random.default_rng(seed)
    ne = conn.shape[0]
    mu = 1.0 * (1.0 + rng.uniform(-0.2, 0.2, ne))
    lam = 4.0 * (1.0 + rng.uniform(-0.2, 0.2, ne))
    mask = np.zeros(coords.shape, dtype=np.uint8)
    values = np.zeros(coords.shape)
    left = _face_mask(coords, 0, 0.0)
    right = _face_mask(coords, 0, length)
    mask[left] = 1
    mask[right] = 1
    values[right, 0] = stretch * length
    return _problem(3, coords, conn, "neohookean", mu, lam, mask, values, np.zeros((0, 3), np.int32),
                    np.zeros((0, 3)), f"nhbar_{nx}x{ny}x{nz}", seed)


def cfg3_bar():
    """64 x 16 x 16 hexes -> 98,304 tets, 18,785 nodes; 20% stretch (seed 3)."""
    return bar_problem(64, 16, 16, 3)


def roofline_cube():
    """Scaled cfg2 cube at 160^3 hexes: 24,576,000 tets, 4,173,281 nodes (seed 2)."""
    return cube_problem(160, 2)


def _domain_mesh(domain, target_tets, h, rng):
    """Voxel domain with about target_tets tets at hex edge h.

    cube: s^3 hexes; lshape: s^3 cube minus the quarter prism i,j >= s/2 (kept 3/4);
    plate: s x s x max(2, s//4) slab with 3 to 6 cylindrical holes along z, radii in
    [s/12, s/6], centres uniform in the slab's interior (drawn from rng).
    """
    if domain == "cube":
        s = max(2, round((target_tets / 6.0) ** (1 / 3)))
        return grid_tet(s, s, s, h=h)
    if domain == "lshape":
        s = max(2, round((target_tets / (6.0 * 0.75)) ** (1 / 3)))
        i, j, _ = np.meshgrid(np.arange(s), np.arange(s), np.arange(s), indexing="ij")
        keep = ~((i >= s // 2) & (j >= s // 2))
        return grid_tet(s, s, s, keep=keep, h=h)
    if domain == "plate":
        s = max(8, round((target_tets / (6.0 * 0.25 * 0.85)) ** (1 / 3)))
        nz = max(2, s // 4)
        nh = int(rng.integers(3, 7))
        ci = rng.uniform(0.2 * s, 0.8 * s, size=(nh, 2))
        rad = rng.uniform(s / 12.0, s / 6.0, size=nh)
        i, j, _ = np.meshgrid(np.arange(s), np.arange(s), np.arange(nz), indexing="ij")
        keep = np.ones((s, s, nz), dtype=bool)
        for (cx, cy), r in zip(ci, rad):
            keep &= (i + 0.5 - cx) ** 2 + (j + 0.5 - cy) ** 2 > r * r
        return grid_tet(s, s, nz, keep=keep, h=h)
    raise ValueError(domain)


def cfg4_batch(n_meshes=64, seed=4, lo=5_000, hi=200_000, h=0.25, field_std=0.01):
    """Ragged batch for the differentiable energy loss.

    For each mesh (rng = default_rng(seed), drawn in this order per mesh): domain uniform
    over {cube, lshape, plate}; target tet count log-uniform in [lo, hi]; material kind
    linear or Neo-Hookean with probability 1/2; the voxel geometry (holes for plates).
    Linear: E = 1 (1 + U[-0.2,0.2]), nu = 0.3 + U[-0.02,0.02]; Neo-Hookean: mu = 1 (1 +
    U[-0.2,0.2]), lambda = 4 (1 + U[-0.2,0.2]), per element. x=0 face clamped (as the hard
    boundary multiplier of the paper's network output would do); x=max face traction
    (0.05, 0, 0). The displacement field is N(0, field_std) per DOF, zero on clamped DOFs,
    rounded to float32. Returns a list of (problem, u) pairs.
    """
    rng = np.random.default_rng(seed)
    out = []
    for m in range(n_meshes):
        domain = ["cube", "lshape", "plate"][int(rng.integers(0, 3))]
        target = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        kind = "linear" if rng.uniform() < 0.5 else "neohookean"
        coords, conn = _domain_mesh(domain, target, h, rng)
        ne = conn.shape[0]
        if kind == "linear":
            a = 1.0 * (1.0 + rng.uniform(-0.2, 0.2, ne))
            b = 0.3 + rng.uniform(-0.02, 0.02, ne)
        else:
            a = 1.0 * (1.0 + rng.uniform(-0.2, 0.2, ne))
            b = 4.0 * (1.0 + rng.uniform(-0.2, 0.2, ne))
        lo_b, hi_b = bbox(coords)
        mask = np.zeros(coords.shape, dtype=np.uint8)
        mask[_face_mask(coords, 0, lo_b[0])] = 1
        facets = boundary_facets(coords, conn, axis=0, value=hi_b[0])
        traction = np.tile([0.05, 0.0, 0.0], (facets.shape[0], 1))
        prob = _problem(3, coords, conn, kind, a, b, mask, np.zeros(coords.shape), facets, traction,
                        f"batch{m}_{domain}_{kind}_{ne}", seed)
        u = (field_std * rng.standard_normal(coords.shape)).astype(np.float32)
        u[mask.astype(bool)] = 0.0
        out.append((prob, u))
    return out


def cfg5_requests(n_requests=1000, seed=5, lo=2_000, hi=2_000_000):
    """Serving workload: a list of request records (meshes are built on demand).

    Per request (default_rng(seed), in this order): unit-rate exponential inter-arrival gap
    (scaled by 1/rate at run time), target tets log-uniform in [lo, hi], kind cube-linear
    with probability 0.7 else bar-Neo-Hookean, warm start with probability 0.5, a material
    seed. Cube: n = round((t/6)^(1/3)) hexes per side (>= 7). Bar: 4m x m x m hexes with
    m = round((t/24)^(1/3)) (>= 3); 10% stretch.
    """
    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(n_requests):
        gap = rng.exponential(1.0)
        t = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        linear = rng.uniform() < 0.7
        warm = rng.uniform() < 0.5
        mseed = int(rng.integers(0, 2**31 - 1))
        if linear:
            n = max(7, round((t / 6.0) ** (1 / 3)))
            dims = (n, n, n)
        else:
            m = max(3, round((t / 24.0) ** (1 / 3)))
            dims = (4 * m, m, m)
        reqs.append(dict(id=r, gap=gap, kind="linear" if linear else "neohookean", dims=dims,
                         n_tets=6 * dims[0] * dims[1] * dims[2], warm=warm, seed=mseed))
    return reqs


def request_problem(req):
    """Build the problem of one serving request record."""
    if req["kind"] == "linear":
        return cube_problem(req["dims"][0], req["seed"])
    nx, ny, nz = req["dims"]
    return bar_problem(nx, ny, nz, req["seed"], stretch=0.1)


# ---------------------------------------------------------------------------------------
# Small problems for parity tests
# ---------------------------------------------------------------------------------------


def small_problem(dim, kind, n=4, seed=0, jitter=0.15, permute=True, traction=True, prescribed=0.0,
                  shape=None):
    """Irregular test problem: jittered structured mesh, random node/element order.

    dim 2: n x n squares on [0,1]^2; dim 3: n x n x n hexes (or `shape`) on the box of
    edge 1 per hex direction scaled by the counts. Material per element: linear E in
    [0.5, 2], nu in [0.2, 0.4]; Neo-Hookean mu in [0.5, 2], lambda in [1, 6].
    x=0 face clamped; x=max face gets traction (0.3, -0.2[, 0.1]) if traction; if
    prescribed != 0 the x=max face instead has u_x prescribed to that value.
    """
    rng = np.random.default_rng(seed)
    if dim == 2:
        nx, ny = shape if shape is not None else (n, n)
        coords, conn = grid_tri(nx, ny, 1.0, ny / nx)
        hh = 1.0 / nx
    else:
        nx, ny, nz = shape if shape is not None else (n, n, n)
        coords, conn = grid_tet(nx, ny, nz, 1.0, ny / nx, nz / nx)
        hh = 1.0 / nx
    if jitter > 0:
        coords = jitter_nodes(coords, conn, jitter, hh, rng)
    ne = conn.shape[0]
    if kind == "linear":
        a = rng.uniform(0.5, 2.0, ne)
        b = rng.uniform(0.2, 0.4, ne)
    else:
        a = rng.uniform(0.5, 2.0, ne)
        b = rng.uniform(1.0, 6.0, ne)
    lo, hi = bbox(coords)
    mask = np.zeros(coords.shape, dtype=np.uint8)
    values = np.zeros(coords.shape)
    mask[_face_mask(coords, 0, lo[0])] = 1
    if prescribed != 0.0:
        right = _face_mask(coords, 0, hi[0])
        mask[right] = 1
        values[right, 0] = prescribed
    if traction and prescribed == 0.0:
        facets = boundary_facets(coords, conn, axis=0, value=hi[0])
        t = np.array([0.3, -0.2, 0.1][:dim])
        trac = np.tile(t, (facets.shape[0], 1))
    else:
        facets = np.zeros((0, dim), np.int32)
        trac = np.zeros((0, dim))
    if permute:
        coords, conn, perm, mask, values = permute_mesh(coords, conn, rng, mask, values)
        if facets.shape[0]:
            inv = np.empty_like(perm)
            inv[perm] = np.arange(perm.size)
            facets = inv[facets].astype(np.int32)
    return _problem(dim, coords, conn, kind, a, b, mask, values, facets, trac,
                    f"small{dim}d_{kind}_{ne}", seed)


# ---------------------------------------------------------------------------------------
# Warm starts and random fields
# ---------------------------------------------------------------------------------------


def smooth_shape(coords, seed):
    """Smooth vector field: delta_i(x) = sum_k c_{k,i} prod_j sin(k_j pi x_j / L_j + phi).

    k ranges over {1,2,3}^dim, c ~ N(0,1)/|k|^2 and phi ~ U[0, 2 pi) per (k, i, j), drawn
    with default_rng(seed). L_j is the bounding-box extent in direction j, x_j is measured
    from the box's low corner. Returns (n_nodes, dim) float64.
    """
    dim = coords.shape[1]
    rng = np.random.default_rng(seed)
    lo, hi = bbox(coords)
    ext = np.maximum(hi - lo, 1e-300)
    xr = (coords - lo) / ext
    out = np.zeros(coords.shape)
    import itertools

    for k in itertools.product((1, 2, 3), repeat=dim):
        kk = np.array(k, dtype=np.float64)
        c = rng.standard_normal(dim) / float(kk @ kk)
        phi = rng.uniform(0.0, 2.0 * np.pi, size=(dim, dim))
        for i in range(dim):
            term = np.ones(coords.shape[0])
            for j in range(dim):
                term *= np.sin(kk[j] * np.pi * xr[:, j] + phi[i, j])
            out[:, i] += c[i] * term
    return out


def dirichlet_envelope(problem, frac=0.15):
    """tanh(dist / l): 0 on Dirichlet nodes, rising linearly away from them, -> 1 inside.

    dist is the Euclidean distance to the nearest node with any prescribed DOF and l is
    frac times the bounding-box diagonal. Mimics the hard-boundary multiplier x / L that
    makes a network prediction (and so its error) vanish smoothly at a clamped face.
    """
    from scipy.spatial import cKDTree

    coords = problem["coords"]
    dn = np.asarray(problem["dirichlet_mask"]).any(axis=1)
    if not dn.any():
        return np.ones(coords.shape[0])
    lo, hi = bbox(coords)
    ell = frac * float(np.linalg.norm(hi - lo))
    dist, _ = cKDTree(coords[dn]).query(coords)
    return np.tanh(dist / ell)


def make_warm_start(problem, u_star, seed, rel=0.01):
    """u_star + delta with ||delta||_2 = rel ||u_star||_2 (all DOFs).

    delta = smooth_shape(seed) x dirichlet_envelope: smooth, and zero on Dirichlet DOFs
    (every DOF of a node with a prescribed DOF is left exact as well).
    """
    u_star = np.asarray(u_star, dtype=np.float64)
    shape = smooth_shape(problem["coords"], seed) * dirichlet_envelope(problem)[:, None]
    shape[problem["dirichlet_mask"].astype(bool)] = 0.0
    shape = shape.reshape(u_star.shape)
    nrm = np.linalg.norm(shape)
    if nrm == 0.0:
        return u_star.copy()
    return u_star + shape * (rel * np.linalg.norm(u_star) / nrm)


def random_field(problem, seed, std=0.01, zero_masked=True):
    """N(0, std) per DOF (float64), zero on Dirichlet DOFs if zero_masked."""
    rng = np.random.default_rng(seed)
    u = std * rng.standard_normal(problem["coords"].shape)
    if zero_masked:
        u[problem["dirichlet_mask"].astype(bool)] = 0.0
    return u


# ---------------------------------------------------------------------------------------
# Periodic unit cells for the homogenisation (synthetic TPMS geometry)
# ---------------------------------------------------------------------------------------

_TPMS = {
    # level-set functions phi(x, y, z) of the triply periodic minimal surfaces of the TPMS
    # appendix (unit period)
    "primitive": lambda x, y, z: np.cos(2 * np.pi * x) + np.cos(2 * np.pi * y) + np.cos(2 * np.pi * z),
    "gyroid": lambda x, y, z: (np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + np.sin(2 * np.pi * y) *
                               np.cos(2 * np.pi * z) + np.sin(2 * np.pi * z) * np.cos(2 * np.pi * x)),
    "diamond": lambda x, y, z: (np.cos(2 * np.pi * x) * np.cos(2 * np.pi * y) * np.cos(2 * np.pi * z) -
                                np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) * np.sin(2 * np.pi * z)),
    "fischer_koch_s": lambda x, y, z: (np.cos(4 * np.pi * x) * np.sin(2 * np.pi * y) * np.cos(2 * np.pi * z) +
                                       np.cos(2 * np.pi * x) * np.cos(4 * np.pi * y) * np.sin(2 * np.pi * z) +
                                       np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) * np.cos(4 * np.pi * z)),
}


def periodic_pairs(n):
    """Node pairs (a, b) of opposite faces of the n^3-hex unit cell (lexicographic nodes, x
    fastest): (0, j, k)-(n, j, k), (i, 0, k)-(i, n, k), (i, j, 0)-(i, j, n) for all indices,
    so edge and corner nodes are chained around the cell (ring-type coupling)."""
    s = n + 1
    idx = np.arange(s)
    a, b = [], []
    J, K = np.meshgrid(idx, idx, indexing="ij")
    for axis in range(3):
        if axis == 0:
            lo, hi = 0 + s * J + s * s * K, n + s * J + s * s * K
        elif axis == 1:
            lo, hi = J + 0 * s + s * s * K, J + n * s + s * s * K
        else:
            lo, hi = J + s * K + 0, J + s * K + s * s * n
        a.append(lo.ravel())
        b.append(hi.ravel())
    return np.stack([np.concatenate(a), np.concatenate(b)], axis=1).astype(np.int32)


def tpms_cell(n, family="gyroid", c=0.0, network="solid", E_solid=1.0, nu=0.3, void_ratio=1e-3):
    """Periodic TPMS unit cell [0,1]^3 as an n^3 voxel grid split into 6 Kuhn tets per voxel.

    A voxel is solid where the level set at its centre satisfies phi > c (solid network) or
    -c <= phi <= c (sheet network); solid voxels get E_solid, void voxels void_ratio * E_solid
    (a soft phase keeps the operator definite; the appendix's void has E = 0), nu everywhere.
    Node 0 (the origin) is fixed in all DOFs (removes the rigid translations left by the
    periodic coupling); no traction. Returns the problem dict with the extra keys "pairs"
    (periodic node pairs), "solid" (per-element bool) and "volume_fraction"."""
    h = 1.0 / n
    centres = (np.arange(n) + 0.5) * h
    X, Y, Z = np.meshgrid(centres, centres, centres, indexing="ij")
    phi = _TPMS[family](X, Y, Z)
    solid_vox = phi > c if network == "solid" else np.abs(phi) <= c
    coords, conn = grid_tet(n, n, n)
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    vox = solid_vox[i.ravel(order="F"), j.ravel(order="F"), k.ravel(order="F")]
    solid = np.repeat(vox, 6)
    E = np.where(solid, E_solid, void_ratio * E_solid)
    nuv = np.full(conn.shape[0], nu)
    mask = np.zeros(coords.shape, dtype=np.uint8)
    mask[0, :] = 1
    p = _problem(3, coords, conn, "linear", E, nuv, mask, np.zeros(coords.shape), np.zeros((0, 3), np.int32),
                 np.zeros((0, 3)), f"tpms_{family}_{network}_{n}^3", 0)
    p["pairs"] = periodic_pairs(n)
    p["solid"] = solid
    p["volume_fraction"] = float(vox.mean())
    return p


def laminate_cell(n, layers=(1.0, 5.0), nus=(0.3, 0.2), axis=0):
    """Periodic laminate on the n^3 grid: voxel slabs perpendicular to `axis` alternate
    between the phases (Young's moduli `layers`, Poisson's ratios `nus`) with n / len(layers)
    voxels each; node 0 fixed, periodic pairs as in tpms_cell."""
    coords, conn = grid_tet(n, n, n)
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    coord = (i, j, k)[axis].ravel(order="F")
    m = len(layers)
    phase = np.repeat((coord * m) // n, 6)
    E = np.asarray(layers, dtype=np.float64)[phase]
    nuv = np.asarray(nus, dtype=np.float64)[phase]
    mask = np.zeros(coords.shape, dtype=np.uint8)
    mask[0, :] = 1
    p = _problem(3, coords, conn, "linear", E, nuv, mask, np.zeros(coords.shape), np.zeros((0, 3), np.int32),
                 np.zeros((0, 3)), f"laminate_{n}^3", 0)
    p["pairs"] = periodic_pairs(n)
    p["phase_fraction"] = [float(np.mean(phase == q)) for q in range(m)]
    return p
