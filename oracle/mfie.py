"""MFIE and CFIE Galerkin entries and their AIM form (oracle; test infrastructure only).

Section 2.2 of the paper solves closed bodies with the combined-field
integral equation, CFIE = alpha EFIE + (1 - alpha) eta MFIE with alpha = 0.6.
With exp(+j w t), G(R) = exp(-j k R) / (4 pi R) and outward unit normals n,
the magnetic-field equation on a PEC surface is

    J / 2 - n x PV int grad G(r - r') x J(r') dS' = n x H_inc,

and its Galerkin form with RWG functions is

    ZM_mn = 1/2 <f_m, f_n> - <f_m, n x int grad G x f_n>,
    VM_m  = <f_m, n x H_inc>,  H_inc = (1/eta) khat x pol exp(-j k khat . r).

Fixed choices where the paper is silent:

* the same collapsed Gauss-Legendre rules as the EFIE entries (test rule
  N_TEST, or N_TEST_SING when the triangles share a vertex; source rule
  N_SOURCE), with no singularity extraction: the kernel is O(1/R^2) only
  where non-coplanar triangles touch, and the two rules' points never meet;
* a pair of coplanar triangles (in particular a triangle with itself)
  contributes nothing to the second term: every vector in it lies in the
  plane, so n x (grad G x f) vanishes identically;
* AIM form of the second term: the curl of the interpolated vector potential,
  so with the grid potentials Phi_c (c = x, y, z) of the EFIE product,

      <f_m, n x curl A> ~= sum_u sum_c W^c_m(u) Phi_c(u),
      W^c_m(u) = int f_m . (n x (grad L_u x e_c)) dS,

  the moment-matched weights of the differentiated interpolation: they
  reproduce int f_m . (n x (grad q x e_c)) dS for every polynomial q of
  per-axis degree <= M (solved on the same moment system as Lambda).
"""

import numpy as np

from . import ETA0
from .aim import aim_pair_values, grid_kernel, n_weight_rule, stencil_offsets
from .quadrature import triangle_rule, N_TEST, N_TEST_SING, N_SOURCE, N_RHS


def tri_normals(verts, tris):
    """Unit normals (r1 - r0) x (r2 - r0) / |.| of the triangles."""
    r0, r1, r2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    c = np.cross(r1 - r0, r2 - r0)
    return c / np.sqrt((c * c).sum(-1))[:, None]


def _areas(verts, tris):
    r0, r1, r2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    c = np.cross(r1 - r0, r2 - r0)
    return 0.5 * np.sqrt((c * c).sum(-1))


def mfie_pair_blocks(verts, tris, P, Q, k, chunk=4096):
    """Blocks B[K, 3, 3] of the second MFIE term for test triangles P[K] and sources Q[K]:

        B[p, a, b] = 1/(4 A_P A_Q) int_P int_Q (r - P_a) . (n_P x (grad G(r - r') x (r' - Q_b))) dS' dS

    so that, for RWG m with slot a on P (sign s_m) and n with slot b on Q (sign s_n),
    <f_m, n x int grad G x f_n> += s_m s_n l_m l_n B[p, a, b].  Coplanar pairs give 0.
    Also returns the Gram blocks C[K, 3, 3] = 1/(4 A_P^2) int_P (r - P_a).(r - P_b) dS
    where P == Q (else 0): <f_m, f_n> += s_m s_n l_m l_n C[p, a, b].
    """
    P = np.asarray(P, dtype=np.int64)
    Q = np.asarray(Q, dtype=np.int64)
    nrm = tri_normals(verts, tris)
    area = _areas(verts, tris)
    tp, tq = tris[P], tris[Q]
    touching = (tp[:, :, None] == tq[:, None, :]).any(axis=(1, 2))
    coplanar = (np.abs(np.cross(nrm[P], nrm[Q])).max(-1) == 0.0) & (
        np.abs(((verts[tq[:, 0]] - verts[tp[:, 0]]) * nrm[P]).sum(-1)) == 0.0)
    coplanar |= P == Q
    x1s, x2s, ws = triangle_rule(N_SOURCE)
    B = np.zeros((len(P), 3, 3), dtype=np.complex128)
    for is_t, nr in ((False, N_TEST), (True, N_TEST_SING)):
        x1t, x2t, wt = triangle_rule(nr)
        sel = np.nonzero((touching == is_t) & ~coplanar)[0]
        for s0 in range(0, len(sel), chunk):
            ii = sel[s0 : s0 + chunk]
            pv = verts[tris[P[ii]]]
            qv = verts[tris[Q[ii]]]
            n = nrm[P[ii]]
            rt = pv[:, None, 0] + x1t[None, :, None] * (pv[:, None, 1] - pv[:, None, 0]) + x2t[None, :, None] * (pv[:, None, 2] - pv[:, None, 0])
            rs = qv[:, None, 0] + x1s[None, :, None] * (qv[:, None, 1] - qv[:, None, 0]) + x2s[None, :, None] * (qv[:, None, 2] - qv[:, None, 0])
            D = rt[:, :, None, :] - rs[:, None, :, :]  # r - r'  [K, nt, ns, 3]
            R = np.sqrt((D * D).sum(-1))
            g = -(1.0 + 1j * k * R) * np.exp(-1j * k * R) / (4.0 * np.pi * R ** 3)  # grad G = g (r - r')
            gw = g * (area[Q[ii]][:, None, None] * ws[None, None, :])
            rta = rt[:, :, None, :] - pv[:, None, :, :]  # r - P_a   [K, nt, 3a, 3]
            rsb = rs[:, :, None, :] - qv[:, None, :, :]  # r' - Q_b  [K, ns, 3b, 3]
            # (r - P_a) . (n x (D x rsb)) = ((r - P_a) . D)(n . rsb) - ((r - P_a) . rsb)(n . D)
            aD = np.einsum("kiax,kijx->kija", rta, D)  # [K, nt, ns, 3a]
            nb = np.einsum("kx,kjbx->kjb", n, rsb)  # [K, ns, 3b]
            ab = np.einsum("kiax,kjbx->kijab", rta, rsb)  # [K, nt, ns, 3a, 3b]
            nD = np.einsum("kx,kijx->kij", n, D)  # [K, nt, ns]
            integrand = aD[..., :, None] * nb[:, None, :, None, :] - ab * nD[..., None, None]
            inner = np.einsum("kij,kijab->kiab", gw, integrand)
            W = area[P[ii]][:, None] * wt[None, :]
            B[ii] = np.einsum("ki,kiab->kab", W, inner) / (4.0 * area[P[ii]] * area[Q[ii]])[:, None, None]
    # Gram blocks on equal triangles: a degree-2 polynomial, exact with any rule of >= 2 points
    C = np.zeros((len(P), 3, 3))
    same = np.nonzero(P == Q)[0]
    if len(same):
        x1, x2, w = triangle_rule(3)
        pv = verts[tris[P[same]]]
        pts = pv[:, None, 0] + x1[None, :, None] * (pv[:, None, 1] - pv[:, None, 0]) + x2[None, :, None] * (pv[:, None, 2] - pv[:, None, 0])
        ra = pts[:, :, None, :] - pv[:, None, :, :]
        A = area[P[same]]
        C[same] = np.einsum("i,kiax,kibx->kab", w, ra, ra) * (A / (4.0 * A * A))[:, None, None]
    return B, C


def _scatter(rwg, lookup, rows, cols):
    val = np.zeros(len(rows), dtype=np.complex128)
    for tri_m, _, slot_m, sgn_m, _ in rwg.halves():
        for tri_n, _, slot_n, sgn_n, _ in rwg.halves():
            val += sgn_m * sgn_n * lookup(tri_m[rows], tri_n[cols], slot_m[rows], slot_n[cols])
    return rwg.length[rows] * rwg.length[cols] * val


def mfie_entries(rwg, rows, cols, k):
    """ZM_mn = 1/2 <f_m, f_n> - <f_m, n x int grad G x f_n> for explicit RWG pairs."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    nt = len(rwg.tris)
    keys = []
    for tri_m, *_ in rwg.halves():
        for tri_n, *_ in rwg.halves():
            keys.append(tri_m[rows] * nt + tri_n[cols])
    ukeys = np.unique(np.concatenate(keys))
    B, C = mfie_pair_blocks(rwg.verts, rwg.tris, ukeys // nt, ukeys % nt, k)
    T = 0.5 * C - B

    def lookup(a, b, sa, sb):
        return T[np.searchsorted(ukeys, a * nt + b), sa, sb]

    return _scatter(rwg, lookup, rows, cols)


def dense_ZM(rwg, k):
    """Full MFIE matrix for small meshes."""
    N = rwg.N
    rows, cols = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    return mfie_entries(rwg, rows.ravel(), cols.ravel(), k).reshape(N, N)


def dense_ZC(rwg, k, alpha, ZE=None):
    """Full CFIE matrix alpha ZE + (1 - alpha) eta ZM (ZE: the EFIE matrix, unsymmetrised)."""
    from .efie import dense_Z

    ZE = dense_Z(rwg, k) if ZE is None else ZE
    return alpha * ZE + (1.0 - alpha) * ETA0 * dense_ZM(rwg, k)


def planewave_rhs_mfie(rwg, k, khat, pol, n_rule=N_RHS):
    """VM[nrhs, N] = <f_m, n x H_inc>, H_inc = (1/eta) khat x pol exp(-j k khat . r)."""
    khat = np.atleast_2d(khat)
    pol = np.atleast_2d(pol)
    xi1, xi2, w = triangle_rule(n_rule)
    verts, tris = rwg.verts, rwg.tris
    nrm = tri_normals(verts, tris)
    V = np.zeros((len(khat), rwg.N), dtype=np.complex128)
    for tri, free, _slot, sgn, area in rwg.halves():
        r0, r1, r2 = verts[tris[tri, 0]], verts[tris[tri, 1]], verts[tris[tri, 2]]
        pts = r0[:, None] + xi1[None, :, None] * (r1 - r0)[:, None] + xi2[None, :, None] * (r2 - r0)[:, None]
        f = (sgn * rwg.length / (2.0 * area))[:, None, None] * (pts - verts[free][:, None, :])
        wa = area[:, None] * w[None, :]
        n = nrm[tri]
        for b in range(len(khat)):
            h = np.cross(khat[b], pol[b]) / ETA0
            nxh = np.cross(n, h)  # [N, 3] constant on the triangle
            ph = np.exp(-1j * k * (pts @ khat[b]))
            V[b] += ((f * nxh[:, None, :]).sum(-1) * ph * wa).sum(-1)
    return V


def planewave_rhs_cfie(rwg, k, khat, pol, alpha):
    from .excitation import planewave_rhs

    return alpha * planewave_rhs(rwg, k, khat, pol) + (1.0 - alpha) * ETA0 * planewave_rhs_mfie(rwg, k, khat, pol)


def _dmono(p, s):
    """d/ds s^p."""
    return p * s ** (p - 1) if p > 0 else np.zeros_like(s)


def mfie_weights(rwg, h, M, anc):
    """Differentiated-interpolation weights W[N, 3, S] (c = x, y, z):

        sum_u W^c_m(u) q(u) = int f_m . (n x (grad q x e_c)) dS

    for every polynomial q of per-axis degree <= M, imposed on the monomials
    in the centred, scaled coordinate s = (xi - M/2)/(M/2) per axis (the
    moment system of ``aim.moment_weights``), with
    f . (n x (grad q x e_c)) = (f . grad q) n_c - f_c (n . grad q).
    """
    off = stencil_offsets(M)
    S = len(off)
    P = M + 1
    half = 0.5 * M
    xi1, xi2, w = triangle_rule(n_weight_rule(M))
    nrm = tri_normals(rwg.verts, rwg.tris)
    mom = np.zeros((S, rwg.N, 3))
    verts, tris = rwg.verts, rwg.tris
    for tri, free, _slot, sgn, area in rwg.halves():
        r0, r1, r2 = verts[tris[tri, 0]], verts[tris[tri, 1]], verts[tris[tri, 2]]
        pts = r0[:, None] + xi1[None, :, None] * (r1 - r0)[:, None] + xi2[None, :, None] * (r2 - r0)[:, None]
        f = (sgn * rwg.length / (2.0 * area))[:, None, None] * (pts - verts[free][:, None, :])  # [N, q, 3]
        n = nrm[tri]  # [N, 3]
        sc = ((pts - h * anc[:, None, :]) / h - half) / half
        ds = 1.0 / (half * h)  # ds/dr per axis
        wa = area[:, None] * w[None, :]
        for qi, q in enumerate(off):
            mx, my, mz = sc[..., 0] ** q[0], sc[..., 1] ** q[1], sc[..., 2] ** q[2]
            grad = np.stack([_dmono(q[0], sc[..., 0]) * my * mz, mx * _dmono(q[1], sc[..., 1]) * mz,
                             mx * my * _dmono(q[2], sc[..., 2])], axis=-1) * ds  # [N, q, 3]
            fg = (f * grad).sum(-1)  # [N, q]
            ng = (n[:, None, :] * grad).sum(-1)
            for c in range(3):
                mom[qi, :, c] += ((fg * n[:, None, c] - f[..., c] * ng) * wa).sum(-1)
    V1 = np.vander((np.arange(P, dtype=np.float64) - half) / half, increasing=True).T
    W = mom.reshape(P, P, P, -1)
    for axis in range(3):
        moved = np.moveaxis(W, axis, 0)
        W = np.moveaxis(np.linalg.solve(V1, moved.reshape(P, -1)).reshape(moved.shape), 0, axis)
    return np.ascontiguousarray(W.reshape(S, rwg.N, 3).transpose(1, 2, 0))


def mfie_pair_values(W, lam, anc, rows, cols, h, k, M):
    """Grid approximation of <f_m, n x curl A_n>: sum_c W^c_m . G Lambda^c_n (c = x, y, z)."""
    off = stencil_offsets(M)
    d = anc[rows] - anc[cols]
    keys, inv = np.unique(d, axis=0, return_inverse=True)
    inv = inv.ravel()
    out = np.zeros(len(rows), dtype=np.complex128)
    for gi, dv in enumerate(keys):
        sel = np.nonzero(inv == gi)[0]
        Gd = grid_kernel(dv[None, None, :] + off[:, None, :] - off[None, :, :], h, k)
        t = np.einsum("pcs,st->pct", W[rows[sel]], Gd)
        out[sel] = np.einsum("pct,pct->p", t, lam[cols[sel]][:, :3, :])
    return out
