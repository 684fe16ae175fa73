"""Mie series for a PEC sphere (oracle; test infrastructure only).

Section 2.2 uses the analytic Mie series as the reference RCS of the sphere
(its ref. [7], Balanis).  Written from the standard expansion (Bohren &
Huffman, Ch. 4) in the perfect-conductor limit:

    a_n = [x j_n(x)]' / [x h_n(x)]',   b_n = j_n(x) / h_n(x),   x = k a
    S1(t) = sum_n (2n+1)/(n(n+1)) (a_n pi_n + b_n tau_n)
    S2(t) = sum_n (2n+1)/(n(n+1)) (a_n tau_n + b_n pi_n)

with pi_n, tau_n the angular functions (upward recurrence) and the series cut
at n_max = x + 4 x^(1/3) + 10.  For an x-polarised wave travelling along +z,
sigma_thth(theta, phi) = (lambda^2 / pi) |S2(theta)|^2 cos^2(phi).  The
paper's sphere is lit by a wave travelling along -z: rotating the problem by
pi about the x axis maps (theta, phi) to (pi - theta, -phi) and thetahat to
minus thetahat, so sigma_thth^(-z)(theta, phi) = sigma_thth^(+z)(pi - theta, phi).
|S|^2 is the same under exp(+jwt) and exp(-iwt).
"""

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def coefficients(x):
    nmax = int(np.ceil(x + 4.0 * x ** (1.0 / 3.0) + 10.0))
    n = np.arange(1, nmax + 1)
    jn = spherical_jn(n, x)
    jnp = spherical_jn(n, x, derivative=True)
    yn = spherical_yn(n, x)
    ynp = spherical_yn(n, x, derivative=True)
    hn = jn + 1j * yn
    hnp = jnp + 1j * ynp
    a = (jn + x * jnp) / (hn + x * hnp)
    b = jn / hn
    return n, a, b


def angular(nmax, mu):
    """pi_n(mu), tau_n(mu) for n = 1..nmax: arrays [nmax, len(mu)]."""
    mu = np.atleast_1d(mu)
    pi = np.zeros((nmax + 1, len(mu)))
    tau = np.zeros((nmax + 1, len(mu)))
    pi[1] = 1.0
    tau[1] = mu
    for n in range(2, nmax + 1):
        pi[n] = ((2 * n - 1) * mu * pi[n - 1] - n * pi[n - 2]) / (n - 1)
        tau[n] = n * mu * pi[n] - (n + 1) * pi[n - 1]
    return pi[1:], tau[1:]


def amplitudes(x, theta):
    n, a, b = coefficients(x)
    pi, tau = angular(len(n), np.cos(theta))
    c = ((2 * n + 1) / (n * (n + 1)))[:, None]
    S1 = (c * (a[:, None] * pi + b[:, None] * tau)).sum(0)
    S2 = (c * (a[:, None] * tau + b[:, None] * pi)).sum(0)
    return S1, S2


def sigma_thth_minus_z(radius, theta, phi, wavelength=1.0):
    """Bistatic sigma_thth of a PEC sphere, x-polarised wave travelling -z."""
    k = 2.0 * np.pi / wavelength
    _, S2 = amplitudes(k * radius, np.pi - np.asarray(theta))
    return (wavelength ** 2 / np.pi) * np.abs(S2) ** 2 * np.cos(phi) ** 2


def efficiencies(x):
    """(Q_ext from the optical theorem, Q_sca from the coefficient sum, Q_back)."""
    n, a, b = coefficients(x)
    qsca = (2.0 / x ** 2) * ((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2)).sum()
    qext = (2.0 / x ** 2) * ((2 * n + 1) * (a + b)).real.sum()
    qback = np.abs(((2 * n + 1) * (-1.0) ** n * (a - b)).sum()) ** 2 / x ** 2
    return qext, qsca, qback
