"""Plane-wave incidence sets and seeded random vectors.

A plane wave is given by its propagation direction ``khat`` (unit vector the
wave travels along) and its polarisation ``pol`` (unit vector, orthogonal to
khat).  Arrays are float64 [nrhs, 3].
"""

import numpy as np


def _sph(theta, phi):
    st, ct = np.sin(theta), np.cos(theta)
    sp, cp = np.sin(phi), np.cos(phi)
    rhat = np.stack([st * cp, st * sp, ct], axis=-1)
    that = np.stack([ct * cp, ct * sp, -st], axis=-1)
    phat = np.stack([-sp, cp, np.zeros_like(sp)], axis=-1)
    return rhat, that, phat


def planewave_minus_z_xpol(nrhs=1):
    """x-polarised wave travelling toward -z (Section 2.1 plate and sphere)."""
    khat = np.tile(np.array([0.0, 0.0, -1.0]), (nrhs, 1))
    pol = np.tile(np.array([1.0, 0.0, 0.0]), (nrhs, 1))
    return khat, pol


def random_incidence(n_dirs, seed=0, theta_max_deg=80.0, both_pols=True, rng=None):
    """Random arrival directions with theta and phi polarisations.

    Draw order: theta ~ U[0, theta_max] degrees (n_dirs values), then
    phi ~ U[0, 360) degrees (n_dirs values), from ``numpy.random.default_rng``.
    The wave arrives from (theta, phi), so it travels along -rhat(theta, phi).
    With ``both_pols`` every direction gives two right-hand sides, polarised
    along theta-hat and phi-hat (in that order, direction-major).
    """
    if rng is None:
        rng = np.random.default_rng(seed)
    th = np.deg2rad(rng.uniform(0.0, theta_max_deg, n_dirs))
    ph = np.deg2rad(rng.uniform(0.0, 360.0, n_dirs))
    rhat, that, phat = _sph(th, ph)
    if not both_pols:
        return -rhat, that
    khat = np.repeat(-rhat, 2, axis=0)
    pol = np.empty_like(khat)
    pol[0::2] = that
    pol[1::2] = phat
    return khat, pol


def sphere_four_directions():
    """Four travel directions (-z, -x, -y, -(1,1,1)/sqrt3), two polarisations each.

    For a travel direction -rhat(theta, phi) the polarisations are theta-hat
    and phi-hat of the arrival direction; for -z these are x-hat and y-hat.
    """
    dirs = np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0], [1, 1, 1]], dtype=np.float64)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    th = np.arccos(np.clip(dirs[:, 2], -1, 1))
    ph = np.arctan2(dirs[:, 1], dirs[:, 0])
    rhat, that, phat = _sph(th, ph)
    khat = np.repeat(-dirs, 2, axis=0)
    pol = np.empty_like(khat)
    pol[0::2] = that
    pol[1::2] = phat
    return khat, pol


def random_complex(shape, seed=0, dtype=np.complex128):
    """Seeded complex vector with independent N(0,1) real and imaginary parts."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im).astype(dtype)
