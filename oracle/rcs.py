"""Bistatic RCS and the error measure of eq. (1) (oracle; test infrastructure only).

Far field of the solved surface current J = sum_m x_m f_m (exp(+j w t)):

    N(rhat) = sum_m x_m int f_m(r') exp(+j k rhat . r') dS'
    sigma_thth(rhat) = (k^2 eta^2 / 4 pi) |thetahat . N(rhat)|^2

for unit incident amplitude.  Eq. (1) of the paper, the relative RMS error
of sigma_thth integrated over the sphere of directions, is evaluated with
Gauss-Legendre nodes in cos(theta) and uniform nodes in phi (the paper does
not state its quadrature): n_theta = max(64, 4 ceil(k a)), n_phi = 2 n_theta.
"""

import numpy as np

from . import ETA0
from .quadrature import triangle_rule, N_FAR


def direction_grid(n_theta, n_phi):
    """(theta, phi, weight) of the eq. (1) quadrature, flattened theta-major."""
    mu, wmu = np.polynomial.legendre.leggauss(n_theta)
    theta = np.arccos(mu)
    phi = (np.arange(n_phi) + 0.5) * (2.0 * np.pi / n_phi)
    T, P = np.meshgrid(theta, phi, indexing="ij")
    W = np.repeat(wmu, n_phi) * (2.0 * np.pi / n_phi)
    return T.ravel(), P.ravel(), W


def far_field(rwg, k, X, theta, phi, n_rule=N_FAR):
    """N_theta, N_phi [nrhs, ndir] of currents X[nrhs, N]."""
    X = np.atleast_2d(X)
    st, ct, sp, cp = np.sin(theta), np.cos(theta), np.sin(phi), np.cos(phi)
    rhat = np.stack([st * cp, st * sp, ct], axis=1)
    that = np.stack([ct * cp, ct * sp, -st], axis=1)
    phat = np.stack([-sp, cp, np.zeros_like(sp)], axis=1)
    xi1, xi2, w = triangle_rule(n_rule)
    verts, tris = rwg.verts, rwg.tris
    Nv = np.zeros((X.shape[0], len(theta), 3), dtype=np.complex128)
    for tri, free, _slot, sgn, area in rwg.halves():
        r0, r1, r2 = verts[tris[tri, 0]], verts[tris[tri, 1]], verts[tris[tri, 2]]
        pts = r0[:, None] + xi1[None, :, None] * (r1 - r0)[:, None] + xi2[None, :, None] * (r2 - r0)[:, None]
        f = (sgn * rwg.length / (2.0 * area))[:, None, None] * (pts - verts[free][:, None, :])  # [N,q,3]
        wa = area[:, None] * w[None, :]
        for d0 in range(0, len(theta), 256):
            sl = slice(d0, d0 + 256)
            ph = np.exp(1j * k * np.einsum("nqx,dx->dnq", pts, rhat[sl]))  # [d, N, q]
            fw = f * wa[..., None]
            # sum over basis and points: [b, d, 3]
            Nv[:, sl] += np.einsum("bn,dnq,nqx->bdx", X, ph, fw)
    Nt = np.einsum("bdx,dx->bd", Nv, that)
    Np = np.einsum("bdx,dx->bd", Nv, phat)
    return Nt, Np


def sigma_thth(rwg, k, X, theta, phi):
    Nt, _ = far_field(rwg, k, X, theta, phi)
    return (k * k * ETA0 * ETA0 / (4.0 * np.pi)) * np.abs(Nt) ** 2


def err_thth(sig, sig_ref, weights):
    """Eq. (1): sqrt( int |s - s_ref|^2 dOmega / int |s_ref|^2 dOmega )."""
    num = (np.abs(sig - sig_ref) ** 2 * weights).sum(axis=-1)
    den = (np.abs(sig_ref) ** 2 * weights).sum(axis=-1)
    return np.sqrt(num / den)


def default_ntheta(ka):
    return max(64, 4 * int(np.ceil(ka)))
