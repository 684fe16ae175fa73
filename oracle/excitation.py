"""Plane-wave right-hand side (oracle; test infrastructure only).

Section 2.1: the scatterers are lit by plane waves.  With exp(+j w t),
E_inc(r) = pol * exp(-j k khat . r), and the Galerkin right-hand side is

    V_m = int f_m(r) . E_inc(r) dS

integrated with the collapsed Gauss-Legendre rule N_RHS on each half.
"""

import numpy as np

from .quadrature import triangle_rule, N_RHS


def planewave_rhs(rwg, k, khat, pol, n_rule=N_RHS):
    """V[nrhs, N] for incidence directions khat[nrhs, 3] and polarisations pol[nrhs, 3]."""
    khat = np.atleast_2d(khat)
    pol = np.atleast_2d(pol)
    xi1, xi2, w = triangle_rule(n_rule)
    verts, tris = rwg.verts, rwg.tris
    V = np.zeros((len(khat), rwg.N), dtype=np.complex128)
    for tri, free, _slot, sgn, area in rwg.halves():
        r0, r1, r2 = verts[tris[tri, 0]], verts[tris[tri, 1]], verts[tris[tri, 2]]
        pts = r0[:, None] + xi1[None, :, None] * (r1 - r0)[:, None] + xi2[None, :, None] * (r2 - r0)[:, None]
        f = (sgn * rwg.length / (2.0 * area))[:, None, None] * (pts - verts[free][:, None, :])
        wa = area[:, None] * w[None, :]
        for b in range(len(khat)):
            ph = np.exp(-1j * k * (pts @ khat[b]))  # [N, q]
            V[b] += ((f @ pol[b]) * ph * wa).sum(-1)
    return V
