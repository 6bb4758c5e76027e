"""Seeded synthetic inputs: surface meshes and right-hand sides.

This module holds no arithmetic of the method.  It only generates the flat
triangulations (Section 4.2: a triangulation of the boundary into flat
triangles, one piecewise-constant density per triangle) and the random data
vectors that both the CUDA path and the CPU oracle consume.

Meshes are returned as ``(verts float64[nv,3], tris int32[M,3])``; the
triangles are oriented outward.  Every coordinate is produced with plain
element-wise NumPy operations (no BLAS reductions), so the same call gives
bit-identical meshes on x86 and Arm hosts.

Workloads stand in for the paper's own meshes (the cube discretisations of
Section 6.1 and the beam of Section 6.2 are not published):

* ``icosphere(level)``      -- radius-1 sphere, 20*4**level triangles.
* ``cube_surface(n)``       -- surface of [-1,1]^3, n*n squares per face, each
  cut along the same diagonal: 12*n*n triangles.
* ``ellipsoid(n, a, b, c)`` -- cube-sphere (the cube surface projected to the
  unit sphere) scaled by the semi-axes (a, b, c).
* ``ball_points`` / ``shell_points`` -- evaluation points inside a ball or in
  a spherical shell (the points x_i of the domain at which Section 5, Eq. (vector_eq)
  evaluates the displacement), by rejection from a cube: only comparisons and
  products, no library function whose last bit could differ between hosts.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "icosphere",
    "cube_surface",
    "ellipsoid",
    "uniform_rhs",
    "ellipsoid_batch_specs",
    "sample_rows",
    "ball_points",
    "shell_points",
]


def _normalise(p: np.ndarray) -> np.ndarray:
    n = np.sqrt(p[:, 0] * p[:, 0] + p[:, 1] * p[:, 1] + p[:, 2] * p[:, 2])
    return p / n[:, None]


def icosphere(level: int):
    """Icosahedron, midpoint-subdivided ``level`` times, vertices projected to
    the unit sphere after every subdivision.  M = 20 * 4**level."""
    if level < 0:
        raise ValueError("level must be >= 0")
    t = (1.0 + np.sqrt(5.0)) / 2.0
    v = np.array(
        [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
         (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)], dtype=np.float64)
    v = _normalise(v)
    f = np.array(
        [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)], dtype=np.int64)
    for _ in range(level):
        nv = v.shape[0]
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
        key = np.minimum(e[:, 0], e[:, 1]) * nv + np.maximum(e[:, 0], e[:, 1])
        uk, inv = np.unique(key, return_inverse=True)
        a = uk // nv
        b = uk % nv
        mid = _normalise((v[a] + v[b]) * 0.5)
        mid_id = nv + inv
        nf = f.shape[0]
        ab, bc, ca = mid_id[:nf], mid_id[nf:2 * nf], mid_id[2 * nf:]
        f = np.concatenate([
            np.stack([f[:, 0], ab, ca], 1),
            np.stack([f[:, 1], bc, ab], 1),
            np.stack([f[:, 2], ca, bc], 1),
            np.stack([ab, bc, ca], 1)], axis=0)
        v = np.concatenate([v, mid], axis=0)
    return np.ascontiguousarray(v), np.ascontiguousarray(f.astype(np.int32))


def cube_surface(n: int, half: float = 1.0):
    """Surface of [-half, half]^3 with n x n squares per face; every square is
    cut along its (v00, v11) diagonal.  Shared edge/corner vertices are merged."""
    if n < 1:
        raise ValueError("n must be >= 1")
    g = np.arange(n + 1, dtype=np.float64) * (2.0 / n) - 1.0
    verts, tris = [], []
    base = 0
    # (fixed axis, sign, (u axis, v axis)) chosen so that (u x v) points outward
    faces = [(0, 1.0, (1, 2)), (0, -1.0, (2, 1)), (1, 1.0, (2, 0)),
             (1, -1.0, (0, 2)), (2, 1.0, (0, 1)), (2, -1.0, (1, 0))]
    for ax, sg, (ua, va) in faces:
        U, Vv = np.meshgrid(g, g, indexing="ij")
        p = np.zeros(((n + 1) * (n + 1), 3))
        p[:, ax] = sg
        p[:, ua] = U.ravel()
        p[:, va] = Vv.ravel()
        verts.append(p)
        i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        v00 = (i * (n + 1) + j).ravel() + base
        v10 = ((i + 1) * (n + 1) + j).ravel() + base
        v01 = (i * (n + 1) + j + 1).ravel() + base
        v11 = ((i + 1) * (n + 1) + j + 1).ravel() + base
        t = np.empty((2 * n * n, 3), dtype=np.int64)
        t[0::2] = np.stack([v00, v10, v11], 1)
        t[1::2] = np.stack([v00, v11, v01], 1)
        tris.append(t)
        base += p.shape[0]
    V = np.concatenate(verts) * half
    T = np.concatenate(tris)
    uv, inv = np.unique(V, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    return np.ascontiguousarray(uv), np.ascontiguousarray(inv[T].astype(np.int32))


def ellipsoid(n: int, a: float, b: float, c: float):
    """Cube-sphere with n x n squares per face, mapped to the unit sphere and
    scaled by the semi-axes (a, b, c).  M = 12 n^2."""
    V, T = cube_surface(n)
    V = _normalise(V) * np.array([a, b, c], dtype=np.float64)[None, :]
    return np.ascontiguousarray(V), T


def uniform_rhs(ndof: int, seed: int, nrhs: int = 1) -> np.ndarray:
    """i.i.d. uniform[-1,1] data vectors, dof index 3*i + d in the mesh's
    original triangle order.  Shape (nrhs, ndof); column r uses seed + r."""
    out = np.empty((nrhs, ndof), dtype=np.float64)
    for r in range(nrhs):
        out[r] = np.random.default_rng(seed + r).uniform(-1.0, 1.0, ndof)
    return out


def ellipsoid_batch_specs(count: int = 64, seed: int = 3,
                          tmin: float = 2000.0, tmax: float = 40000.0):
    """Parameters of the batched ellipsoid workload: semi-axes uniform[0.5, 2],
    triangle counts log-uniform in [tmin, tmax] (n = round(sqrt(T/12)) squares
    per cube face edge), Poisson ratio uniform[0.2, 0.45]."""
    rng = np.random.default_rng(seed)
    specs = []
    for m in range(count):
        a, b, c = rng.uniform(0.5, 2.0, 3)
        tri = np.exp(rng.uniform(np.log(tmin), np.log(tmax)))
        n = max(2, int(round(np.sqrt(tri / 12.0))))
        nu = rng.uniform(0.2, 0.45)
        specs.append(dict(n=n, a=float(a), b=float(b), c=float(c), nu=float(nu), E=1.0,
                          seed=1000 + m))
    return specs


def sample_rows(M: int, count: int, seed: int) -> np.ndarray:
    """Sorted sample of ``count`` distinct triangle indices in [0, M)."""
    rng = np.random.default_rng(seed)
    count = min(count, M)
    return np.sort(rng.choice(M, size=count, replace=False)).astype(np.int64)


def shell_points(count: int, r_in: float, r_out: float, seed: int) -> np.ndarray:
    """``count`` points uniform in the shell r_in <= |x| <= r_out (r_in = 0:
    the ball), in the order drawn: uniform in [-r_out, r_out]^3, kept when
    their squared norm lies in [r_in^2, r_out^2].  Shape (count, 3)."""
    rng = np.random.default_rng(seed)
    out = np.empty((0, 3), dtype=np.float64)
    lo2, hi2 = r_in * r_in, r_out * r_out
    while out.shape[0] < count:
        p = rng.uniform(-r_out, r_out, (max(2 * count, 64), 3))
        q = p[:, 0] * p[:, 0] + p[:, 1] * p[:, 1] + p[:, 2] * p[:, 2]
        out = np.concatenate([out, p[(q >= lo2) & (q <= hi2)]])
    return np.ascontiguousarray(out[:count])


def ball_points(count: int, radius: float, seed: int) -> np.ndarray:
    """``count`` points uniform in the ball |x| <= radius.  Shape (count, 3)."""
    return shell_points(count, 0.0, radius, seed)
