"""The seeded synthetic workloads match their stated recipes (sizes, shapes, noise, seeding).

These inputs stand in for the paper's datasets (Section 5), so their construction is part of
what the measurements mean: each check below restates one line of the recipe.
"""
import numpy as np

import meshgen as mg


def _torus_minor(V):
    V = np.asarray(V, float)
    return np.sqrt((np.hypot(V[:, 0], V[:, 1]) - 1.0) ** 2 + V[:, 2] ** 2)


def test_workload1_icosphere_with_normal_noise():
    p = mg.workload(1)
    assert p.sizes == (162, 320, 162, 320) and p.tol == 1e-4 and p.tol_mode == mg.TOL_ABS
    assert np.allclose(np.linalg.norm(p.VA, axis=1), 1.0, atol=1e-15)
    d = p.VB - p.VA
    radial = np.einsum("ij,ij->i", d, p.VA)
    # displaced along the normal only (the normal of the unit sphere is the position)
    assert np.abs(d - radial[:, None] * p.VA).max() < 1e-15
    assert 0.008 < radial.std() < 0.012 and abs(radial.mean()) < 0.003
    assert np.array_equal(p.FA, p.FB)


def test_workload2_torus_pair():
    p = mg.workload(2)
    assert p.sizes == (100_000, 200_000, 25_088, 50_176)
    assert p.VA.dtype == np.float32 and p.tol == 1e-5 and p.tol_mode == mg.TOL_REL
    dA = _torus_minor(p.VA) - 0.3
    assert 0.0009 < dA.std() < 0.0011 and abs(dA.mean()) < 1e-4  # N(0, 1e-3) along the normal
    # B is re-triangulated with jitter in parameter space, so it stays on the torus
    assert np.abs(_torus_minor(p.VB) - 0.3).max() < 1e-6
    # and its vertices are not the regular 224 x 112 grid: the jitter moved them
    phi = np.arctan2(p.VB[:, 1], p.VB[:, 0]).astype(float)
    step = 2 * np.pi / 224
    off = np.abs(((phi / step) + 0.5) % 1.0 - 0.5)
    assert off.max() > 0.2


def test_workload3_slivers_and_superquadric():
    p = mg.workload(3)
    nA, fA, nB, fB = p.sizes
    assert 99_000 <= fA <= 102_000 and fB == 1_000_000 and p.tol == 1e-6
    V = np.asarray(p.VA, float)
    assert np.abs(np.linalg.norm(V, axis=1) - 1.0).max() < 1e-3  # on the unit sphere + N(0, 1e-4)
    T = V[p.FA]
    e = np.stack([np.linalg.norm(T[:, (k + 1) % 3] - T[:, k], axis=1) for k in range(3)], 1)
    area = 0.5 * np.linalg.norm(np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0]), axis=1)
    aspect = e.max(1) ** 2 / (2 * area)  # longest edge over its height
    # each latitude band draws its aspect from logU[10, 1e4]; every triangle has the same area,
    # so taller (low-aspect) bands hold more triangles and the per-triangle median is lower
    q = np.quantile(aspect, [0.001, 0.5, 0.99, 0.999])
    assert q[0] > 8 and q[3] < 3e4 and q[2] > 1e3 and 15 < q[1] < 150
    VB = np.asarray(p.VB, float)
    assert np.allclose(np.abs(VB).max(0), 0.999, atol=1e-6)  # superquadric at scale 0.999


def test_workload5_large_soup():
    p = mg.workload(5)
    nA, fA, nB, fB = p.sizes
    assert fA == 975 * 975 * 2 + 100_000 and fB == 1_000 * 1_000 * 2 and p.tol == 1e-6


def test_workload4_batch_counts_and_seeding():
    ps = mg.batch_workload(16)
    assert len(ps) == 16
    for p in ps:
        _, fA, _, fB = p.sizes
        assert 500 <= fA <= 250_000 and 500 <= fB <= 250_000 and p.tol == 1e-4
    kinds = {p.name.split("-")[-1] for p in ps}
    assert kinds == {"pert", "retri"}
    again = mg.batch_workload(4)
    for a, b in zip(ps[:4], again):
        assert np.array_equal(a.VA, b.VA) and np.array_equal(a.FB, b.FB)


def test_seeded_and_reduced():
    a, b = mg.workload(2, 0.02), mg.workload(2, 0.02)
    assert np.array_equal(a.VA, b.VA) and np.array_equal(a.VB, b.VB)
    assert a.sizes[1] < 10_000  # the reduced instance the parity tests use
