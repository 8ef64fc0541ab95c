"""Seeded synthetic triangle soups for the Hausdorff branch-and-bound workloads.

This module produces *inputs only*: vertex and face arrays plus the tolerance of
each workload.  It contains none of the method's arithmetic (no distances, no
bounds), so both the FP64 CPU oracle and the CUDA path can draw from it.

Random numbers come from SplitMix64 in its counter form (value k of a stream is
the SplitMix64 finaliser applied to ``seed + (k + 1) * 0x9E3779B97F4A7C15``),
Gaussians from Box-Muller.  Seeds: ``1000 + workload index`` (workloads are
numbered 1..5), split into independent streams for A and B.

The workloads stand in for the public datasets of the paper's Section 5
(Thingi10K, TetWild outputs, the near-zero pairs of Kang et al.), which are not
available here.  Each mimics the structure of one of those benchmarks:
  1 tiny FP64 sphere pair          (a near-identical pair, small)
  2 near-identical torus pair      (near-zero Hausdorff distance, like Kang's pairs)
  3 thin-triangle stress           (slivers, the case the fourth bound targets)
  4 batched uneven pairs           (many independent pairs of mixed sizes)
  5 large soup                     (millions of triangles, disconnected pieces)
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

TOL_ABS = 0
TOL_REL = 1


class Stream:
    """One SplitMix64 stream in counter form; successive calls continue the counter."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.k = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.k + 1, self.k + 1 + n, dtype=np.uint64)
        self.k += n
        with np.errstate(over="ignore"):
            z = self.seed + idx * _GAMMA
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """Uniform doubles in [lo, hi) from the top 53 bits."""
        x = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * x

    def normal(self, n: int, sigma: float = 1.0) -> np.ndarray:
        """Box-Muller Gaussians; uses two uniforms per pair of outputs."""
        m = (n + 1) // 2
        u1 = 1.0 - self.uniform(m)  # (0, 1]
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
        return sigma * z[:n]

    def loguniform(self, n: int, lo: float, hi: float) -> np.ndarray:
        return np.exp(self.uniform(n, math.log(lo), math.log(hi)))


def stream(seed: int, sub: int) -> Stream:
    """Independent sub-stream ``sub`` of workload seed ``seed``."""
    return Stream((seed << 16) ^ (sub * 0x632BE59BD9B4E019))


@dataclasses.dataclass
class Pair:
    """One (A, B) input: row-major vertex arrays (m x 3), int32 face arrays (n x 3)."""

    name: str
    VA: np.ndarray
    FA: np.ndarray
    VB: np.ndarray
    FB: np.ndarray
    tol: float
    tol_mode: int  # TOL_ABS or TOL_REL (relative to the bbox diagonal of A)

    @property
    def sizes(self):
        return (len(self.VA), len(self.FA), len(self.VB), len(self.FB))


# ----------------------------------------------------------------------------- meshes


def icosphere(level: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit icosphere: icosahedron, ``level`` times 1->4 split, vertices projected to r=1."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    V = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5),
         (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    V = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in V]
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(i: int, j: int) -> int:
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = V[i] + V[j]
                V.append(m / np.linalg.norm(m))
                cache[key] = len(V) - 1
            return cache[key]

        F2 = []
        for a, b, c in F:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            F2 += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = F2
    return np.array(V), np.array(F, dtype=np.int32)


def grid_faces(nu: int, nv: int, wrap_u: bool, wrap_v: bool) -> np.ndarray:
    """Two triangles per cell of an nu x nv vertex grid (vertex (i,j) -> i*nv + j), fixed diagonal."""
    cu = nu if wrap_u else nu - 1
    cv = nv if wrap_v else nv - 1
    i, j = np.meshgrid(np.arange(cu), np.arange(cv), indexing="ij")
    i, j = i.ravel(), j.ravel()
    i1, j1 = (i + 1) % nu, (j + 1) % nv
    v00, v10, v11, v01 = i * nv + j, i1 * nv + j, i1 * nv + j1, i * nv + j1
    F = np.empty((2 * len(i), 3), dtype=np.int32)
    F[0::2] = np.stack([v00, v10, v11], 1)
    F[1::2] = np.stack([v00, v11, v01], 1)
    return F


def torus(R: float, r: float, nu: int, nv: int, jitter: float = 0.0, rng: Stream | None = None):
    """Torus on an nu (major) x nv (minor) periodic grid; optional parameter jitter in cells."""
    i, j = np.meshgrid(np.arange(nu, dtype=np.float64), np.arange(nv, dtype=np.float64), indexing="ij")
    i, j = i.ravel(), j.ravel()
    if jitter:
        i = i + rng.uniform(len(i), -jitter, jitter)
        j = j + rng.uniform(len(j), -jitter, jitter)
    u, v = 2 * np.pi * i / nu, 2 * np.pi * j / nv
    P = np.stack([(R + r * np.cos(v)) * np.cos(u), (R + r * np.cos(v)) * np.sin(u), r * np.sin(v)], 1)
    N = np.stack([np.cos(v) * np.cos(u), np.cos(v) * np.sin(u), np.sin(v)], 1)
    return P, grid_faces(nu, nv, True, True), N


def _spow(x, e):
    return np.sign(x) * np.abs(x) ** e


def superquadric(e1: float, e2: float, scale: float, n_lon: int, n_lat: int, jitter: float = 0.0,
                 rng: Stream | None = None):
    """Superellipsoid (exponent e1 in latitude, e2 in longitude) on a lat-long grid.

    Rows j = 0..n_lat run pole to pole; each pole row holds n_lon coincident
    vertices, so the first and last band contain zero-area triangles on purpose.
    """
    j, i = np.meshgrid(np.arange(n_lat + 1, dtype=np.float64), np.arange(n_lon, dtype=np.float64),
                       indexing="ij")
    j, i = j.ravel(), i.ravel()
    if jitter:
        interior = (j > 0) & (j < n_lat)
        j = j + np.where(interior, rng.uniform(len(j), -jitter, jitter), 0.0)
        i = i + rng.uniform(len(i), -jitter, jitter)
    eta = -np.pi / 2 + np.pi * j / n_lat
    om = -np.pi + 2 * np.pi * i / n_lon
    ce, se = np.cos(eta), np.sin(eta)
    ce = np.where(np.abs(ce) < 1e-15, 0.0, ce)
    P = scale * np.stack([_spow(ce, e1) * _spow(np.cos(om), e2), _spow(ce, e1) * _spow(np.sin(om), e2),
                          _spow(se, e1)], 1)
    # faces: rows are contiguous runs of n_lon vertices, longitude wraps, latitude does not
    F = grid_faces(n_lat + 1, n_lon, False, True)
    return P, F


def _superquadric_point_normal(e1, e2, scale, eta, om):
    """Points of the superquadric at parameters (eta, om) and their unit normals, the
    normalised gradient of its implicit form F = (|x|^(2/e2) + |y|^(2/e2))^(e2/e1) + |z|^(2/e1)
    (closed form: no finite differences, whose cancellation would magnify the last-bit
    differences of libm between machines into visible ones)."""
    ce = np.cos(eta)
    P = scale * np.stack([_spow(ce, e1) * _spow(np.cos(om), e2), _spow(ce, e1) * _spow(np.sin(om), e2),
                          _spow(np.sin(eta), e1)], 1)
    U = P / scale
    ax, ay, az = np.abs(U[:, 0]), np.abs(U[:, 1]), np.abs(U[:, 2])
    S = ax ** (2 / e2) + ay ** (2 / e2)
    f = (2 / e1) * S ** (e2 / e1 - 1)
    N = np.stack([f * ax ** (2 / e2 - 1) * np.sign(U[:, 0]), f * ay ** (2 / e2 - 1) * np.sign(U[:, 1]),
                  (2 / e1) * az ** (2 / e1 - 1) * np.sign(U[:, 2])], 1)
    N /= np.maximum(np.linalg.norm(N, axis=1, keepdims=True), 1e-300)
    return P, N


def sliver_sphere(n_target: int, aspect_lo: float, aspect_hi: float, noise: float, rng: Stream):
    """Thin triangles tiling the unit sphere in latitude bands (a soup: bands share no vertices).

    Each band draws an aspect ratio a ~ logU[aspect_lo, aspect_hi]; its angular
    height is H = sqrt(2 * (4 pi / n_target) / a) and its cells are about a*H long
    in longitude, two triangles per cell.  Vertices get isotropic N(0, noise).
    """
    area = 4 * np.pi / n_target
    theta = 0.0
    Vs, Fs, nv = [], [], 0
    while theta < np.pi - 1e-12:
        a = float(rng.loguniform(1, aspect_lo, aspect_hi)[0])
        H = math.sqrt(2 * area / a)
        t0, t1 = theta, min(theta + H, np.pi)
        tm = 0.5 * (t0 + t1)
        nc = max(3, int(round(2 * np.pi * math.sin(tm) / (a * H))))
        phase = float(rng.uniform(1, 0, 2 * np.pi)[0])
        phi = phase + 2 * np.pi * np.arange(nc) / nc
        ring0 = np.stack([np.sin(t0) * np.cos(phi), np.sin(t0) * np.sin(phi), np.full(nc, np.cos(t0))], 1)
        ring1 = np.stack([np.sin(t1) * np.cos(phi), np.sin(t1) * np.sin(phi), np.full(nc, np.cos(t1))], 1)
        k = np.arange(nc)
        k1 = (k + 1) % nc
        a0, a1, b0, b1 = nv + k, nv + k1, nv + nc + k, nv + nc + k1
        F = np.empty((2 * nc, 3), dtype=np.int64)
        F[0::2] = np.stack([a0, a1, b1], 1)
        F[1::2] = np.stack([a0, b1, b0], 1)
        Vs += [ring0, ring1]
        Fs.append(F)
        nv += 2 * nc
        theta = t1
    V = np.concatenate(Vs)
    V = V + rng.normal(3 * len(V), noise).reshape(-1, 3)
    return V, np.concatenate(Fs).astype(np.int32)


def random_triangles_near_superquadric(n: int, e1, e2, scale, edge, offset, rng: Stream):
    """n disconnected triangles of edge ~``edge``, random orientation, centred on the surface
    and pushed along its normal by +-U(0, offset)."""
    eta = rng.uniform(n, -np.pi / 2 + 0.05, np.pi / 2 - 0.05)
    om = rng.uniform(n, -np.pi, np.pi)
    P, N = _superquadric_point_normal(e1, e2, scale, eta, om)
    C = P + N * rng.uniform(n, -offset, offset)[:, None]
    g1 = rng.normal(3 * n).reshape(n, 3)
    g2 = rng.normal(3 * n).reshape(n, 3)
    x = g1 / np.linalg.norm(g1, axis=1, keepdims=True)
    y = g2 - np.sum(g2 * x, 1, keepdims=True) * x
    y /= np.linalg.norm(y, axis=1, keepdims=True)
    rad = edge / math.sqrt(3.0)
    ang = np.array([0.0, 2 * np.pi / 3, 4 * np.pi / 3])
    V = C[:, None, :] + rad * (np.cos(ang)[None, :, None] * x[:, None, :] + np.sin(ang)[None, :, None] * y[:, None, :])
    return V.reshape(-1, 3), np.arange(3 * n, dtype=np.int32).reshape(n, 3)


def _mean_edge(V, F):
    e = np.linalg.norm(V[F[:, 1]] - V[F[:, 0]], axis=1)
    return float(np.mean(e))


# ----------------------------------------------------------------------------- workloads


def workload(k: int, scale: float = 1.0) -> Pair:
    """Workload ``k`` in 1..5 (see the module docstring).  ``scale`` < 1 shrinks the
    triangle counts (about linearly) with the same construction, for fast parity runs."""
    seed = 1000 + k
    if k == 1:
        VA, FA = icosphere(2)
        rb = stream(seed, 2)
        VB = VA + rb.normal(len(VA), 0.01)[:, None] * VA  # unit sphere: normal = position
        return Pair("icosphere-l2-320f-noise0.01", VA, FA, VB, FA.copy(), 1e-4, TOL_ABS)
    if k == 2:
        s = math.sqrt(scale)
        nu, nv = max(8, int(round(400 * s))), max(6, int(round(250 * s)))
        mu, mv = max(6, int(round(224 * s))), max(4, int(round(112 * s)))
        ra, rb = stream(seed, 1), stream(seed, 2)
        PA, FA, NA = torus(1.0, 0.3, nu, nv)
        VA = PA + NA * ra.normal(len(PA), 1e-3)[:, None]
        VB, FB, _ = torus(1.0, 0.3, mu, mv, jitter=0.3, rng=rb)
        return Pair(f"torus-{nu}x{nv}-vs-{mu}x{mv}", VA.astype(np.float32), FA, VB.astype(np.float32), FB,
                    1e-5, TOL_REL)
    if k == 3:
        ra, rb = stream(seed, 1), stream(seed, 2)
        VA, FA = sliver_sphere(max(200, int(100_000 * scale)), 10.0, 1e4, 1e-4, ra)
        s = math.sqrt(scale)
        VB, FB = superquadric(0.8, 1.2, 0.999, max(8, int(round(1000 * s))), max(4, int(round(500 * s))))
        return Pair(f"slivers-{len(FA)}-vs-superquadric-{len(FB)}", VA.astype(np.float32), FA,
                    VB.astype(np.float32), FB, 1e-6, TOL_REL)
    if k == 5:
        ra, rb = stream(seed, 1), stream(seed, 2)
        s = math.sqrt(scale)
        na = max(8, int(round(975 * s)))
        PA, FA = superquadric(0.8, 1.2, 1.0, na, na)
        nr = max(4, int(100_000 * scale))
        R, FR = random_triangles_near_superquadric(nr, 0.8, 1.2, 1.0, _mean_edge(PA, FA), 0.1, ra)
        VA = np.concatenate([PA, R])
        FA = np.concatenate([FA, FR + len(PA)]).astype(np.int32)
        nb = max(8, int(round(1000 * s)))
        VB, FB = superquadric(0.8, 1.2, 1.0, nb, nb, jitter=0.3, rng=rb)
        return Pair(f"soup-{len(FA)}-vs-superquadric-{len(FB)}", VA.astype(np.float32), FA,
                    VB.astype(np.float32), FB, 1e-6, TOL_REL)
    if k == 4:
        raise ValueError("workload 4 is a batch; use batch_workload()")
    raise ValueError(f"unknown workload {k}")


def _shape_mesh(shape: int, n_faces: int, jitter: float, rng: Stream):
    if shape == 0:  # sphere: lat-long grid, unit radius
        nlat = max(3, int(round(math.sqrt(n_faces / 4))))
        return superquadric(1.0, 1.0, 1.0, 2 * nlat, nlat, jitter, rng)
    if shape == 1:  # torus R=1, r=0.3
        nv = max(4, int(round(math.sqrt(n_faces / 8))))
        P, F, _ = torus(1.0, 0.3, 4 * nv, nv, jitter, rng)
        return P, F
    nlat = max(3, int(round(math.sqrt(n_faces / 4))))
    return superquadric(0.8, 1.2, 1.0, 2 * nlat, nlat, jitter, rng)


def _vertex_normals(V, F):
    N = np.zeros_like(V)
    n = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    for c in range(3):
        np.add.at(N, F[:, c], n)
    return N / np.maximum(np.linalg.norm(N, axis=1, keepdims=True), 1e-300)


def batch_workload(n_pairs: int = 1024, lo: int = 1000, hi: int = 200_000) -> list[Pair]:
    """Workload 4: independent pairs, face counts ~ logU[lo, hi] per side, shape uniform in
    {sphere, torus, superquadric}; B is either A perturbed along its normals by N(0, sigma)
    (sigma ~ logU[1e-5, 1e-2]) or the same shape re-triangulated at B's own count with 0.3-cell
    jitter.  Tolerance 1e-4 relative.  Seed of pair i: 5000 + i."""
    pairs = []
    for i in range(n_pairs):
        r = Stream(5000 + i)
        na, nb = (int(x) for x in r.loguniform(2, lo, hi))
        shape = int(r.u64(1)[0] % np.uint64(3))
        perturbed = bool(r.u64(1)[0] & np.uint64(1))
        sigma = float(r.loguniform(1, 1e-5, 1e-2)[0])
        VA, FA = _shape_mesh(shape, na, 0.0, r)
        if perturbed:
            VB = VA + _vertex_normals(VA, FA) * r.normal(len(VA), sigma)[:, None]
            FB = FA.copy()
        else:
            VB, FB = _shape_mesh(shape, nb, 0.3, r)
        pairs.append(Pair(f"pair{i}-shape{shape}-{'pert' if perturbed else 'retri'}", VA.astype(np.float32), FA,
                          VB.astype(np.float32), FB, 1e-4, TOL_REL))
    return pairs
