"""Host-only RCS utilities of the library (aim_rcs_grid, aim_err_thth,
aim_mie_sigma_thth) against the oracle's own versions and closed forms.
They run on the CPU: no device is touched."""

import os

import numpy as np
import pytest

from oracle import mie, rcs


@pytest.fixture(scope="module")
def g():
    from paper_1010_1456_gb300 import _lib

    if not os.path.exists(_lib.LIB_PATH):
        from paper_1010_1456_gb300 import build

        build.build()
    import paper_1010_1456_gb300 as pkg

    return pkg


@pytest.mark.parametrize("nt,nphi", [(1, 2), (7, 5), (64, 128), (404, 808)])
def test_direction_grid_matches_oracle(g, nt, nphi):
    th, ph, w = g.rcs_direction_grid(nt, nphi)
    rt, rp, rw = rcs.direction_grid(nt, nphi)
    assert np.abs(np.cos(th) - np.cos(rt)).max() <= 1e-14
    assert np.abs(ph - rp).max() <= 1e-14
    # the same Gauss weights: numpy's leggauss drifts to ~5e-10 relative at the ends for n = 404,
    # while these integrate polynomials to 1e-16 (next test)
    assert np.abs(w / rw - 1).max() <= 1e-9
    assert abs(w.sum() - 4 * np.pi) <= 1e-12


def test_direction_grid_integrates_polynomials(g):
    """Gauss-Legendre in cos(theta) with n nodes is exact to degree 2n - 1."""
    for nt in (6, 404):
        th, ph, w = g.rcs_direction_grid(nt, 2)
        mu = np.cos(th)
        for p in list(range(12)) + [2 * nt - 2, 2 * nt - 1]:
            exact = 2 * np.pi * (2.0 / (p + 1) if p % 2 == 0 else 0.0)
            assert abs((w * mu ** p).sum() - exact) <= 1e-14


def test_err_thth_matches_oracle_and_scale(g):
    rng = np.random.default_rng(3)
    th, ph, w = g.rcs_direction_grid(16)
    s = rng.random((3, len(w)))
    r = rng.random((3, len(w)))
    got = g.err_thth(s, r, w)
    ref = rcs.err_thth(s, r, w)
    assert np.abs(got - ref).max() <= 1e-14
    assert g.err_thth(s[0], s[0], w) == 0.0
    assert abs(g.err_thth(1.01 * s[0], s[0], w) - 0.01) <= 1e-14
    with pytest.raises(g.AIMError):
        g.err_thth(s[0], np.zeros_like(s[0]), w)


@pytest.mark.parametrize("radius", [0.05, 0.25, 1.0, 4.0, 16.0])
def test_mie_matches_oracle(g, radius):
    nt = max(64, 4 * int(np.ceil(2 * np.pi * radius)))
    th, ph, w = g.rcs_direction_grid(nt)
    got = g.mie_sigma_thth(radius, th, ph)
    ref = mie.sigma_thth_minus_z(radius, th, ph)
    # pointwise where the pattern is not in a null, and by eq. (1) overall
    assert rcs.err_thth(got, ref, w) <= 1e-10
    big = ref > 1e-6 * ref.max()
    assert np.abs(got[big] / ref[big] - 1).max() <= 1e-8


def test_mie_small_sphere_backscatter(g):
    """Rayleigh limit: backscatter sigma / (pi a^2) -> 9 (ka)^4 for ka << 1
    (backscatter of a wave travelling -z is theta = 0)."""
    a = 0.05 / (2 * np.pi)  # ka = 0.05
    s = g.mie_sigma_thth(a, np.array([0.0]), np.array([0.0]))[0]
    assert abs(s / (np.pi * a * a) / (9 * 0.05 ** 4) - 1) < 2e-3
