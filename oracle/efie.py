"""EFIE Galerkin entries with singularity extraction (oracle; test infrastructure only).

Section 2.2 of the paper solves the electric-field integral equation for PEC
surfaces by the method of moments.  With time convention exp(+j w t),
Green's function G(R) = exp(-j k R) / (4 pi R) and RWG functions f_m, the
Galerkin entries are

    Z_mn = j k eta [ <f_m, G * f_n> - k^-2 <div f_m, G * div f_n> ].

The paper states no quadrature or singular rule; the fixed choices are:

* outer (testing) integral: collapsed Gauss-Legendre rule N_TEST, or
  N_TEST_SING when the two triangles share a vertex; inner (source)
  integral: rule N_SOURCE (see ``quadrature``);
* if the test and source triangles share at least one vertex (including the
  same triangle), the inner integral is split as
  G = [exp(-jkR) - 1] / (4 pi R) + 1 / (4 pi R): the first part by the
  quadrature rule, evaluated in the cancellation-free form
  -(j k / 4 pi) * sinc(k R / 2) * exp(-j k R / 2), and the second part in
  closed form (the classical analytic potential integrals of a planar
  triangle, Wilton et al. 1984 / Graglia 1993, derived again below);
* near-zone entries are symmetrised: Z_mn := (Z_mn + Z_nm) / 2.
"""

import numpy as np

from . import ETA0
from .quadrature import triangle_rule, N_TEST, N_TEST_SING, N_SOURCE


def potential_integrals(r, tv):
    """Closed-form I0 = int_T 1/R dS' and I1 = int_T (rho' - rho)/R dS'.

    ``r``: observation points [K, 3]; ``tv``: triangle vertices [K, 3, 3]
    (one triangle per point).  R = |r - r'|, rho = projection of r on the
    triangle's plane.  Returns (I0 [K], I1 [K, 3], rho [K, 3]).

    Derivation: with d the height of r over the plane, the in-plane gradient
    of R is (rho' - rho)/R, so by the divergence theorem I1 is the sum over
    the edges of (outward edge normal u) * int_edge R dl, and I0 follows from
    the solid-angle form of int 1/R.  For edge i from a to b with unit
    direction lhat, u = lhat x nhat, t = (a - rho).u (signed distance of rho
    to the edge line), l+/- = (b/a - rho).lhat, R0^2 = t^2 + d^2,
    R+/- = sqrt(R0^2 + l+/-^2):

      I0 = sum_i t ln[(R+ + l+)/(R- + l-)]
               - |d| [atan(t l+ / (R0^2 + |d| R+)) - atan(t l- / (R0^2 + |d| R-))]
      I1 = 1/2 sum_i u [R0^2 ln((R+ + l+)/(R- + l-)) + l+ R+ - l- R-]

    R + l is evaluated as R0^2 / (R - l) when l < 0 (no cancellation).  Terms
    with R0 = 0 (observation point on an edge line) are dropped: their limit
    is 0.
    """
    r = np.asarray(r, dtype=np.float64)
    v0, v1, v2 = tv[:, 0], tv[:, 1], tv[:, 2]
    nrm = np.cross(v1 - v0, v2 - v0)
    nhat = nrm / np.sqrt((nrm * nrm).sum(-1))[:, None]
    d = ((r - v0) * nhat).sum(-1)
    rho = r - d[:, None] * nhat
    ad = np.abs(d)
    I0 = np.zeros(len(r))
    I1 = np.zeros((len(r), 3))
    for a, b in ((v0, v1), (v1, v2), (v2, v0)):
        e = b - a
        elen = np.sqrt((e * e).sum(-1))
        lhat = e / elen[:, None]
        u = np.cross(lhat, nhat)
        lp = ((b - rho) * lhat).sum(-1)
        lm = ((a - rho) * lhat).sum(-1)
        t = ((a - rho) * u).sum(-1)
        R02 = t * t + d * d
        Rp = np.sqrt(R02 + lp * lp)
        Rm = np.sqrt(R02 + lm * lm)
        ok = R02 > 1e-30 * elen * elen
        R02s = np.where(ok, R02, 1.0)
        with np.errstate(divide="ignore", invalid="ignore"):
            num = np.where(lp >= 0.0, Rp + lp, R02s / (Rp - lp))
            den = np.where(lm >= 0.0, Rm + lm, R02s / (Rm - lm))
            f2 = np.where(ok, np.log(num / den), 0.0)
        at = np.arctan(t * lp / (R02s + ad * Rp)) - np.arctan(t * lm / (R02s + ad * Rm))
        I0 += np.where(ok, t * f2 - ad * at, 0.0)
        I1 += 0.5 * u * np.where(ok, R02 * f2, 0.0)[:, None] + 0.5 * u * (lp * Rp - lm * Rm)[:, None]
    return I0, I1, rho


def _smooth_kernel(k, R):
    """[exp(-jkR) - 1] / (4 pi R) as -(jk/4pi) sinc(kR/2) exp(-jkR/2)."""
    x = 0.5 * k * R
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(x == 0.0, 1.0, np.sin(x) / np.where(x == 0.0, 1.0, x))
    return (-1j * k / (4.0 * np.pi)) * s * np.exp(-1j * x)


def triangle_pair_blocks(verts, tris, P, Q, k, singular=None, n_test=N_TEST, n_src=N_SOURCE,
                         n_test_sing=N_TEST_SING, chunk=4096):
    """Triangle-pair blocks T[K, 3, 3] for test triangles P[K] and sources Q[K].

    T[p, a, b] = sum_i W_i [ (r_i - P_a) . V_b(r_i) / (4 A_P A_Q)
                              - S0(r_i) / (k^2 A_P A_Q) ]
    with S0(r) = int_Q G dS', V_b(r) = int_Q (r' - Q_b) G dS', r_i/W_i the
    test points/weights on P and P_a, Q_b the vertices of P and Q (slot a =
    the RWG whose free vertex is vertex a).  Then, for RWG m with slot a on P
    (sign s_m) and n with slot b on Q (sign s_n),
        Z_mn += j k eta s_m s_n l_m l_n T[p, a, b].
    ``singular[p]`` (default: P and Q share a vertex) selects the extraction.
    """
    P = np.asarray(P, dtype=np.int64)
    Q = np.asarray(Q, dtype=np.int64)
    if singular is None:
        tp, tq = tris[P], tris[Q]
        singular = (tp[:, :, None] == tq[:, None, :]).any(axis=(1, 2))
    x1s, x2s, ws = triangle_rule(n_src)
    out = np.empty((len(P), 3, 3), dtype=np.complex128)
    area = _areas(verts, tris)
    for is_sing, nr in ((False, n_test), (True, n_test_sing)):
        x1t, x2t, wt = triangle_rule(nr)
        sel = np.nonzero(singular == is_sing)[0]
        for s0 in range(0, len(sel), chunk):
            ii = sel[s0 : s0 + chunk]
            out[ii] = _pair_chunk(verts, tris, area, P[ii], Q[ii], singular[ii], k, x1t, x2t, wt, x1s, x2s, ws)
    return out


def _areas(verts, tris):
    r0, r1, r2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    c = np.cross(r1 - r0, r2 - r0)
    return 0.5 * np.sqrt((c * c).sum(-1))


def _pair_chunk(verts, tris, area, P, Q, sing, k, x1t, x2t, wt, x1s, x2s, ws):
    K = len(P)
    pv = verts[tris[P]]  # [K,3,3]
    qv = verts[tris[Q]]
    AP = area[P]
    AQ = area[Q]
    rt = pv[:, None, 0] + x1t[None, :, None] * (pv[:, None, 1] - pv[:, None, 0]) + x2t[None, :, None] * (pv[:, None, 2] - pv[:, None, 0])
    rs = qv[:, None, 0] + x1s[None, :, None] * (qv[:, None, 1] - qv[:, None, 0]) + x2s[None, :, None] * (qv[:, None, 2] - qv[:, None, 0])
    D = rt[:, :, None, :] - rs[:, None, :, :]  # [K, nt, ns, 3]
    R = np.sqrt((D * D).sum(-1))
    G = np.exp(-1j * k * R) / (4.0 * np.pi * np.where(R == 0.0, 1.0, R))
    if sing.any():
        Ks = _smooth_kernel(k, R[sing])
        G[sing] = Ks
    Gw = G * (AQ[:, None, None] * ws[None, None, :])  # weighted source kernel
    S0 = Gw.sum(-1)  # [K, nt]
    # V_b = sum_q Gw (rs_q - Q_b)
    rsb = rs[:, None, :, :] - qv[:, :, None, :]  # [K, 3(b), ns, 3]
    V = np.einsum("kiq,kbqx->kibx", Gw, rsb)  # [K, nt, 3(b), 3]
    if sing.any():
        idx = np.nonzero(sing)[0]
        nt = rt.shape[1]
        robs = rt[idx].reshape(-1, 3)
        tvv = np.repeat(qv[idx], nt, axis=0)
        I0, I1, rho = potential_integrals(robs, tvv)
        I0 = I0.reshape(len(idx), nt) / (4.0 * np.pi)
        I1 = I1.reshape(len(idx), nt, 3) / (4.0 * np.pi)
        rho = rho.reshape(len(idx), nt, 3)
        S0[idx] += I0
        # int (r' - Q_b)/R = I1 + (rho - Q_b) I0
        V[idx] += I1[:, :, None, :] + (rho[:, :, None, :] - qv[idx][:, None, :, :]) * I0[:, :, None, None]
    W = AP[:, None] * wt[None, :]  # [K, nt]
    rta = rt[:, :, None, :] - pv[:, None, :, :]  # [K, nt, 3(a), 3]
    dot = np.einsum("kiax,kibx->kiab", rta, V)  # [K, nt, 3, 3]
    T = np.einsum("ki,kiab->kab", W, dot) / (4.0 * AP * AQ)[:, None, None]
    T -= (np.einsum("ki,ki->k", W, S0) / (k * k * AP * AQ))[:, None, None]
    return T


def _scatter_pairs(rwg, T_lookup, rows, cols, k):
    """Z values for RWG pairs (rows[i], cols[i]) from triangle-pair blocks."""
    val = np.zeros(len(rows), dtype=np.complex128)
    for tri_m, _, slot_m, sgn_m, _ in rwg.halves():
        for tri_n, _, slot_n, sgn_n, _ in rwg.halves():
            val += sgn_m * sgn_n * T_lookup(tri_m[rows], tri_n[cols], slot_m[rows], slot_n[cols])
    return (1j * k * ETA0) * rwg.length[rows] * rwg.length[cols] * val


def dense_Z(rwg, k):
    """Full EFIE matrix (unsymmetrised Galerkin fill) for small meshes."""
    nt = len(rwg.tris)
    P, Q = np.meshgrid(np.arange(nt), np.arange(nt), indexing="ij")
    T = triangle_pair_blocks(rwg.verts, rwg.tris, P.ravel(), Q.ravel(), k).reshape(nt, nt, 3, 3)
    N = rwg.N
    rows, cols = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    rows = rows.ravel()
    cols = cols.ravel()
    val = _scatter_pairs(rwg, lambda a, b, sa, sb: T[a, b, sa, sb], rows, cols, k)
    return val.reshape(N, N)


def mom_entries(rwg, rows, cols, k):
    """Galerkin entries Z_mn for an explicit list of RWG pairs (unsymmetrised)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    nt = len(rwg.tris)
    keys = []
    for tri_m, *_ in rwg.halves():
        for tri_n, *_ in rwg.halves():
            keys.append(tri_m[rows] * nt + tri_n[cols])
    ukeys = np.unique(np.concatenate(keys))
    T = triangle_pair_blocks(rwg.verts, rwg.tris, ukeys // nt, ukeys % nt, k)

    def lookup(a, b, sa, sb):
        return T[np.searchsorted(ukeys, a * nt + b), sa, sb]

    return _scatter_pairs(rwg, lookup, rows, cols, k)
