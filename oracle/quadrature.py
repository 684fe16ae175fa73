"""Triangle quadrature (oracle; test infrastructure only).

The paper does not state its quadrature.  The rule used throughout is the
collapsed (Duffy) product of Gauss-Legendre rules: for a triangle with vertices
(r0, r1, r2) in the stored order and Gauss-Legendre nodes/weights (s_i, w_i),
(t_j, w_j) on [0, 1],

    xi1 = s_i,  xi2 = t_j (1 - s_i),  r = r0 + xi1 (r1 - r0) + xi2 (r2 - r0),
    integral_T f dS  ~=  A * sum_ij  2 w_i w_j (1 - s_i) f(r_ij).

With n nodes per direction the rule integrates every polynomial of total
degree <= 2n - 2 exactly.  Points are ordered i-major (s outer, t inner).
"""

import numpy as np


def gauss_legendre_01(n):
    """n-point Gauss-Legendre nodes and weights on [0, 1] (numpy's leggauss)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def triangle_rule(n):
    """Collapsed GL rule with n x n points.

    Returns (xi1, xi2, w): barycentric-style coordinates of the points and the
    weights normalised to sum to 1 (so that integral = area * sum w f).
    """
    s, ws = gauss_legendre_01(n)
    t, wt = gauss_legendre_01(n)
    S, T = np.meshgrid(s, t, indexing="ij")
    WS, WT = np.meshgrid(ws, wt, indexing="ij")
    xi1 = S.ravel()
    xi2 = (T * (1.0 - S)).ravel()
    w = (2.0 * WS * WT * (1.0 - S)).ravel()
    return xi1, xi2, w


def triangle_points(verts, tris, n):
    """Quadrature points of every triangle: [nt, q, 3] points, [q] weights."""
    xi1, xi2, w = triangle_rule(n)
    r0 = verts[tris[:, 0]]
    r1 = verts[tris[:, 1]]
    r2 = verts[tris[:, 2]]
    pts = r0[:, None, :] + xi1[None, :, None] * (r1 - r0)[:, None, :] + xi2[None, :, None] * (r2 - r0)[:, None, :]
    return pts, w


# Rules used by the method (fixed choices; the paper is silent on them).
N_WEIGHT = 5   # moment-matching weights: exact to degree 8 >= 3M+1 = 7 at M=2
N_TEST = 3     # EFIE testing (outer) integral, triangles without a common vertex
N_TEST_SING = 5  # EFIE testing integral, triangles sharing a vertex (or equal)
N_SOURCE = 4   # EFIE source (inner) integral
N_RHS = 4      # plane-wave right-hand side
N_FAR = 3      # far-field radiation integral
