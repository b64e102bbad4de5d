"""Quadrilateral (Q4 / Q8) plane-strain meshes: structured grids mapped onto a quadrilateral
domain, and the two hyperelastic benchmark geometries of Sec. "Nonlinear hyperelasticity"
(a 4 x 1 cantilever beam and Cook's membrane) as synthetic stand-ins. Nothing here evaluates
the finite-element operator."""

import numpy as np


def quad_grid(nx, ny, corners, npe=4, jitter=0.0, rng=None):
    """nx x ny quadrilaterals on the domain bilinearly mapped from the unit square onto
    `corners` ((x0,y0), (x1,y1), (x2,y2), (x3,y3), counterclockwise). Q4: corner nodes of a
    (nx+1) x (ny+1) lattice; Q8: the (2nx+1) x (2ny+1) lattice minus the cell centres.
    Element node order: corners counterclockwise, then mid-edge nodes of edges 0-1, 1-2, 2-3,
    3-0. jitter > 0 moves every interior lattice point by up to jitter lattice spacings in the
    unit square before the mapping (boundary points stay, so the domain is unchanged).
    Returns coords (N, 2), conn (E, npe) int32."""
    c = np.asarray(corners, dtype=np.float64)
    sx, sy = (nx, ny) if npe == 4 else (2 * nx, 2 * ny)
    s, t = np.meshgrid(np.linspace(0, 1, sx + 1), np.linspace(0, 1, sy + 1), indexing="ij")
    s, t = s.ravel(order="F"), t.ravel(order="F")
    if jitter > 0:
        inner = (s > 0) & (s < 1) & (t > 0) & (t < 1)
        d = rng.uniform(-jitter, jitter, (s.size, 2))
        s = s + np.where(inner, d[:, 0] / sx, 0.0)
        t = t + np.where(inner, d[:, 1] / sy, 0.0)
    keep = np.ones(s.size, dtype=bool)
    if npe == 8:
        ii, jj = np.meshgrid(np.arange(sx + 1), np.arange(sy + 1), indexing="ij")
        keep = ~((ii.ravel(order="F") % 2 == 1) & (jj.ravel(order="F") % 2 == 1))
    xy = ((1 - s) * (1 - t))[:, None] * c[0] + (s * (1 - t))[:, None] * c[1] + (s * t)[:, None] * c[2] + \
        ((1 - s) * t)[:, None] * c[3]
    new = -np.ones(s.size, dtype=np.int64)
    new[keep] = np.arange(int(keep.sum()))
    lid = lambda i, j: new[i + (sx + 1) * j]  # noqa: E731
    conn = []
    for j in range(ny):
        for i in range(nx):
            if npe == 4:
                conn.append([lid(i, j), lid(i + 1, j), lid(i + 1, j + 1), lid(i, j + 1)])
            else:
                a, b = 2 * i, 2 * j
                conn.append([lid(a, b), lid(a + 2, b), lid(a + 2, b + 2), lid(a, b + 2),
                             lid(a + 1, b), lid(a + 2, b + 1), lid(a + 1, b + 2), lid(a, b + 1)])
    return xy[keep], np.asarray(conn, dtype=np.int32)


def _edge_facets(coords, conn, npe, side):
    """Boundary edges on the element side `side` (0: edge 0-1, 1: 1-2, 2: 2-3, 3: 3-0) of the
    boundary elements, as (a, b[, mid]) node ids."""
    ends = [(0, 1), (1, 2), (2, 3), (3, 0)]
    a, b = ends[side]
    e = conn[:, [a, b] + ([4 + side] if npe == 8 else [])]
    return e


def quad_problem(nx, ny, corners, npe, kind, mat_a, mat_b, clamp_side="left", traction=None, seed=0,
                 jitter=0.0):
    """Plane-strain problem on quad_grid: nodes on the x = min edge (clamp_side 'left') fixed,
    constant traction on the right element edges (the edges 1-2 of the last column)."""
    coords, conn = quad_grid(nx, ny, corners, npe, jitter, np.random.default_rng(seed))
    ne = conn.shape[0]
    mask = np.zeros(coords.shape, dtype=np.uint8)
    xmin = coords[:, 0].min()
    mask[np.abs(coords[:, 0] - xmin) <= 1e-9] = 1
    right_col = np.arange(ne).reshape(ny, nx)[:, -1]
    facets = _edge_facets(coords, conn[right_col], npe, 1)
    t = np.zeros((facets.shape[0], 2)) if traction is None else np.tile(np.asarray(traction, float), (facets.shape[0], 1))
    return dict(dim=2, coords=np.ascontiguousarray(coords), conn=np.ascontiguousarray(conn), kind=kind,
                mat_a=np.full(ne, float(mat_a)) if np.isscalar(mat_a) else np.asarray(mat_a, float),
                mat_b=np.full(ne, float(mat_b)) if np.isscalar(mat_b) else np.asarray(mat_b, float),
                dirichlet_mask=mask, dirichlet_values=np.zeros(coords.shape),
                facets=np.ascontiguousarray(facets, dtype=np.int32), traction=t, f_ext_extra=None,
                name=f"quad{npe}_{nx}x{ny}", seed=seed, npe=npe)


def nh_beam(nx=50, ny=50, npe=4, traction=(0.0, -0.01)):
    """Neo-Hookean 4 x 1 cantilever (the beam of the hyperelasticity results): mu = 1,
    lambda = 4, left end clamped, downward traction on the right end (the default load bends
    the tip by about a fifth of the length; the oracle's Newton needs 5 steps from zero in one
    load step, close to the paper's ~4.9)."""
    return quad_problem(nx, ny, [(0, 0), (4, 0), (4, 1), (0, 1)], npe, "neohookean", 1.0, 4.0, traction=traction)


def cook_membrane(n=30, npe=8, traction=(0.0, 0.02)):
    """Neo-Hookean Cook membrane (the tapered panel of the hyperelasticity results): corners
    (0,0), (48,44), (48,60), (0,44), mu = 1, lambda = 4, left edge clamped, vertical shear
    traction on the right edge."""
    return quad_problem(n, n, [(0, 0), (48, 44), (48, 60), (0, 44)], npe, "neohookean", 1.0, 4.0,
                        traction=traction)
