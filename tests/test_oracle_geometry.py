"""Pins for the oracle's quadrature, meshes and RWG functions (CPU only)."""

import os
from math import factorial

import numpy as np
import pytest

from aim_inputs import plate_mesh, icosphere_mesh, icosphere_frequency, mesh_mean_edge
from oracle.quadrature import triangle_rule, gauss_legendre_01
from oracle.rwg import RWG


@pytest.mark.parametrize("n", [2, 3, 4, 5, 9])
def test_triangle_rule_exact_to_degree_2n_minus_2(n):
    # int over the unit right triangle of x^a y^b = a! b! / (a + b + 2)!
    xi1, xi2, w = triangle_rule(n)
    for a in range(0, 2 * n - 1):
        for b in range(0, 2 * n - 1 - a):
            exact = factorial(a) * factorial(b) / factorial(a + b + 2)
            got = 0.5 * np.sum(w * xi1 ** a * xi2 ** b)
            assert abs(got - exact) <= 1e-15 + 1e-13 * exact, (n, a, b)


def test_triangle_rule_not_exact_beyond_degree():
    # the rule's degree is sharp for the x^(2n-1) monomial (catches a wrong Jacobian)
    n = 3
    xi1, xi2, w = triangle_rule(n)
    a = 2 * n
    exact = factorial(a) / factorial(a + 2)
    assert abs(0.5 * np.sum(w * xi1 ** a) - exact) > 1e-8


def test_gauss_legendre_nodes():
    x, w = gauss_legendre_01(4)
    assert np.all((x > 0) & (x < 1))
    assert abs(w.sum() - 1.0) < 1e-15


def test_plate_counts():
    for n in (1, 2, 9, 20):
        v, t = plate_mesh(1.0, n)
        r = RWG(v, t)
        assert len(t) == 2 * n * n
        assert r.N == 2 * n * (n + 1) + n * n - 4 * n
    v, t = plate_mesh(1.0, 9)
    assert RWG(v, t).N == 225  # 1 lambda plate, 9 x 9 squares


def test_plate_normals_up():
    v, t = plate_mesh(2.0, 5)
    c = np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])
    assert np.all(c[:, 2] > 0)


@pytest.mark.parametrize("f", [1, 2, 5])
def test_icosphere_topology(f):
    v, t = icosphere_mesh(1.0, f)
    assert len(v) == 10 * f * f + 2 and len(t) == 20 * f * f
    r = RWG(v, t)
    assert r.N == 30 * f * f  # closed surface: every edge interior
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-15)
    c = np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])
    cen = v[t].mean(axis=1)
    assert np.all((c * cen).sum(1) > 0)  # outward orientation
    # Euler characteristic of a sphere
    assert len(v) - r.N + len(t) == 2


def test_icosphere_frequency_rule():
    f = icosphere_frequency(1.0)
    assert mesh_mean_edge(*icosphere_mesh(1.0, f)) <= 1.0 / 9.0
    assert mesh_mean_edge(*icosphere_mesh(1.0, f - 1)) > 1.0 / 9.0


def test_rwg_normal_continuity_and_charge():
    """Across its edge, f has unit normal component on both halves; int div f = 0."""
    v, t = icosphere_mesh(1.0, 3)
    r = RWG(v, t)
    rng = np.random.default_rng(0)
    for m in rng.choice(r.N, 20, replace=False):
        a, b = v[r.edge[m, 0]], v[r.edge[m, 1]]
        s = rng.uniform()
        pt = a + s * (b - a)
        fp, fm = r.eval_f(m, pt)
        e = (b - a) / np.linalg.norm(b - a)
        for tri, f, sgn in ((r.tri_p[m], fp, 1.0), (r.tri_m[m], fm, -1.0)):
            P = v[t[tri]]
            nrm = np.cross(P[1] - P[0], P[2] - P[0])
            nrm /= np.linalg.norm(nrm)
            # in-plane edge normal pointing from T+ to T-
            u = np.cross(e, nrm)
            free = r.free_p[m] if sgn > 0 else r.free_m[m]
            if np.dot(u, pt - v[free]) < 0:
                u = -u
            comp = np.dot(f, u)
            assert abs(comp - sgn * 1.0) < 1e-12
        q = r.length[m] / r.area_p[m] * r.area_p[m] - r.length[m] / r.area_m[m] * r.area_m[m]
        assert abs(q) < 1e-15


def test_rwg_order_and_halves():
    v, t = plate_mesh(1.0, 3)
    r = RWG(v, t)
    keys = r.edge[:, 0] * 10000 + r.edge[:, 1]
    assert np.all(np.diff(keys) > 0)
    assert np.all(r.tri_p < r.tri_m)
    for m in range(r.N):
        assert r.free_p[m] not in r.edge[m] and r.free_m[m] not in r.edge[m]
        assert t[r.tri_p[m], r.slot_p[m]] == r.free_p[m]
        assert t[r.tri_m[m], r.slot_m[m]] == r.free_m[m]


def _table1():
    rows = []
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_plates.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            rows.append([int(v) for v in line.split()])
    return rows


@pytest.mark.parametrize("L", [1, 2, 4, 8, 16, 32])
def test_plate_unknowns_match_table1(L):
    """Table 1's plates are square meshes of 10 L_P x 10 L_P squares (lambda/10 edges),
    each split by one diagonal: the oracle's RWG count (interior edges) gives the
    printed N for every plate it can build here.  The printed 76 840 of the 16 lambda
    row reads as 76 480 (two digits transposed): 2 n (n - 1) + n^2 with n = 160,
    the count every other row also follows.  The grid's third extent is M + 1 = 4
    nodes for the paper's M = 3 on a plate lying in one node plane."""
    row = {r[0]: r for r in _table1()}[L]
    v, t = plate_mesh(float(L), 10 * L)
    r = RWG(v, t)
    printed = 76480 if L == 16 else row[1]
    assert r.N == printed
    if L <= 4:
        from oracle import aim

        anc = aim.anchors(r.centre, 0.1, 3)
        assert anc[:, 2].max() + 3 - anc[:, 2].min() + 1 == row[4]
