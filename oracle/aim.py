"""Adaptive integral method, plain FP64 (oracle; test infrastructure only).

Section 2.2 of the paper accelerates the EFIE matrix-vector product with AIM
(its refs. [1]-[4]): every basis function's current and charge is replaced by
point sources on a regular auxiliary grid whose moments match (the paper
matches moments up to a stated order), the grid sources are convolved with
Green's function by zero-padded 3-D FFTs on the doubled grid (Section 4.1),
the grid potentials are interpolated back onto the testing functions
(Section 4.1, footnote 2), and the near-zone interactions (within gamma
grid spacings, gamma = 3) are corrected with the exact MoM entries minus
their grid approximation.

Readings fixed here where the paper defers to its companion paper:

* stencil: (M+1)^3 grid nodes per basis function, tensor-product moments
  x^p y^q z^r with p, q, r <= M matched about the anchor node;
* anchor: a = floor(c / h - (M - 1) / 2) per axis (c = basis centre, IEEE
  division then subtraction), nodes a .. a+M; grid box [min a, max a + M];
* grid Green's function: G_h(D) = exp(-j k h |D|) / (4 pi h |D|), G_h(0) = 0;
* padded length per axis: smallest 2,3,5-smooth integer >= 2 n - 1;
* near pair: d2 = (dx*dx + dy*dy) + dz*dz <= r*r with d = c_m - c_n in FP64
  and r the near radius (gamma h), self pairs included;
* near value: Z_mn (symmetrised MoM entry) minus its grid approximation.
"""

import numpy as np
import scipy.fft
import scipy.sparse

from . import ETA0
from .quadrature import triangle_rule
from .efie import mom_entries


def n_weight_rule(M):
    """Points per direction of the weight rule: exact to degree 3M+1."""
    return (3 * M + 4) // 2


def smooth_length(m):
    """Smallest integer >= m whose only prime factors are 2, 3 and 5."""
    L = max(int(m), 1)
    while True:
        x = L
        for p in (2, 3, 5):
            while x % p == 0:
                x //= p
        if x == 1:
            return L
        L += 1


def anchors(centres, h, M):
    """Stencil anchor per basis function (integer node index per axis)."""
    t = centres / h
    return np.floor(t - 0.5 * (M - 1)).astype(np.int64)


def grid_box(anc, M):
    """(lo, n): first node index and node count of the grid per axis."""
    lo = anc.min(axis=0)
    hi = anc.max(axis=0) + M
    return lo, hi - lo + 1


def stencil_offsets(M):
    """Local node offsets (i, j, k), index s = (k (M+1) + j) (M+1) + i."""
    r = np.arange(M + 1)
    K, J, I = np.meshgrid(r, r, r, indexing="ij")
    return np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)


def moment_weights(rwg, h, M, anc):
    """Moment-matching weights Lambda[N, 4, S] (components x, y, z, charge).

    For basis m with anchor a and local coordinates xi = (r - h a) / h, the
    weights match every moment of per-axis degree <= M:

        sum_u Lambda^c_m(u) p(u) = int g^c_m(r) p(xi) dS

    for all polynomials p of per-axis degree <= M, with g^c = f_x, f_y, f_z,
    div f.  The equations are imposed on the basis of monomials in the
    centred, scaled coordinate s = (xi - M/2) / (M/2) on each axis (the same
    polynomial space as the monomials in xi, so the same weights, but a
    far better conditioned system: the 1-D matrix has condition number 64
    at M = 5 against 5.8e4 for monomials in xi).  The moments are integrated
    with the collapsed Gauss-Legendre rule ``n_weight_rule(M)``, exact for
    this polynomial degree.  The (M+1)^3 x (M+1)^3 system is the Kronecker
    cube of the 1-D Vandermonde matrix on the scaled nodes and is solved axis
    by axis with numpy.linalg.solve.
    """
    off = stencil_offsets(M)  # nodes u (in local units); exponent triples in the same order
    S = len(off)
    P = M + 1
    half = 0.5 * M
    xi1, xi2, w = triangle_rule(n_weight_rule(M))
    mom = np.zeros((S, rwg.N, 4))
    verts, tris = rwg.verts, rwg.tris
    for tri, free, _slot, sgn, area in rwg.halves():
        r0, r1, r2 = verts[tris[tri, 0]], verts[tris[tri, 1]], verts[tris[tri, 2]]
        pts = r0[:, None] + xi1[None, :, None] * (r1 - r0)[:, None] + xi2[None, :, None] * (r2 - r0)[:, None]
        coef = sgn * rwg.length / (2.0 * area)
        g = np.empty(pts.shape[:2] + (4,))
        g[..., :3] = coef[:, None, None] * (pts - verts[free][:, None, :])
        g[..., 3] = (sgn * rwg.length / area)[:, None]
        sc = ((pts - h * anc[:, None, :]) / h - half) / half  # scaled local coordinates
        wa = area[:, None] * w[None, :]
        for qi, q in enumerate(off):
            mono = sc[..., 0] ** q[0] * sc[..., 1] ** q[1] * sc[..., 2] ** q[2]
            mom[qi] += np.einsum("mq,mqc->mc", wa * mono, g)
    # V[(p,q,r)][(i,j,k)] = s_i^p s_j^q s_k^r is the Kronecker product of the
    # 1-D matrix V1[p][i] = s_i^p with itself, so V Lambda = mom is solved one
    # axis at a time.
    V1 = np.vander((np.arange(P, dtype=np.float64) - half) / half, increasing=True).T
    lam = mom.reshape(P, P, P, -1)  # [exponent z, y, x][basis, component]
    for axis in range(3):
        moved = np.moveaxis(lam, axis, 0)
        lam = np.moveaxis(np.linalg.solve(V1, moved.reshape(P, -1)).reshape(moved.shape), 0, axis)
    lam = lam.reshape(S, rwg.N, 4)
    return np.ascontiguousarray(lam.transpose(1, 2, 0))


def green_grid(n, L, h, k):
    """Circulant embedding of G_h on the padded grid, array [Lz, Ly, Lx].

    Per axis, padded index i maps to offset i (i < n), i - L (i > L - n) and is
    0 in between; G_h(0) = 0.
    """
    axes = []
    for d in range(3):
        i = np.arange(L[d])
        o = np.where(i < n[d], i, np.where(i > L[d] - n[d], i - L[d], 0))
        valid = (i < n[d]) | (i > L[d] - n[d])
        axes.append((o, valid))
    (ox, vx), (oy, vy), (oz, vz) = axes
    OZ, OY, OX = np.meshgrid(oz, oy, ox, indexing="ij")
    VZ, VY, VX = np.meshgrid(vz, vy, vx, indexing="ij")
    r = h * np.sqrt((OX * OX + OY * OY + OZ * OZ).astype(np.float64))
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.exp(-1j * k * r) / (4.0 * np.pi * r)
    g[r == 0.0] = 0.0
    g[~(VX & VY & VZ)] = 0.0
    return g


def grid_kernel(D, h, k):
    """G_h at integer offset vectors D[..., 3] (G_h(0) = 0)."""
    r = h * np.sqrt((D.astype(np.float64) ** 2).sum(-1))
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.exp(-1j * k * r) / (4.0 * np.pi * r)
    return np.where(r == 0.0, 0.0, g)


def convolve_fft(Q, Ghat, n, L):
    """Phi(u) = sum_v G_h(u - v) Q(v) on the n-grid via FFTs on the L-grid.

    Q: [..., nz, ny, nx] complex.  Ghat = fftn(green_grid).  scipy.fft with
    all host cores.
    """
    pad = np.zeros(Q.shape[:-3] + (L[2], L[1], L[0]), dtype=np.complex128)
    pad[..., : n[2], : n[1], : n[0]] = Q
    F = scipy.fft.fftn(pad, axes=(-3, -2, -1), workers=-1)
    F *= Ghat
    out = scipy.fft.ifftn(F, axes=(-3, -2, -1), workers=-1)
    return out[..., : n[2], : n[1], : n[0]]


def convolve_direct(Q, h, k):
    """Brute-force O(Nc^2) grid convolution (used to pin convolve_fft)."""
    nz, ny, nx = Q.shape[-3:]
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    D = pts[:, None, :] - pts[None, :, :]
    Gm = grid_kernel(D, h, k)
    q = Q.reshape(Q.shape[:-3] + (-1,))
    return (q @ Gm.T).reshape(Q.shape)


def convolve_direct_at(Q, nodes, h, k, chunk=1 << 22):
    """Phi(u) = sum_v G_h(u - v) Q(v) at listed nodes u only, by direct summation.

    Q: [..., nz, ny, nx] complex; nodes: [T, 3] integer (x, y, z) grid indices.
    The sum runs over every node v where some leading slice of Q is nonzero
    (the others add nothing), in chunks of about ``chunk`` (u, v) pairs.
    G_h(D) depends on D only through the integer |D|^2, so it is tabulated
    once over 0 .. max |D|^2 with the arithmetic of ``grid_kernel`` (same
    values, bit for bit) and looked up per pair.  Returns [..., T].  This is
    the definition of the grid convolution restricted to a few output nodes:
    it serves products of very large grids checked on sampled rows, where the
    padded FFT of ``convolve_fft`` would hold tens of GB of host memory.
    """
    lead = Q.shape[:-3]
    nz, ny, nx = Q.shape[-3:]
    q = Q.reshape((-1, nz * ny * nx))
    src = np.nonzero(np.any(q != 0, axis=0))[0]
    sx = src % nx
    sy = (src // nx) % ny
    sz = src // (nx * ny)
    spts = np.stack([sx, sy, sz], axis=1)
    qs = q[:, src]  # [B, nsrc]
    nodes = np.asarray(nodes, dtype=np.int64).reshape(-1, 3)
    ext = np.maximum(np.abs(nodes).max(axis=0) if len(nodes) else 0, [nx, ny, nz]) + np.array([nx, ny, nz])
    d2max = int((ext.astype(np.int64) ** 2).sum())
    r = h * np.sqrt(np.arange(d2max + 1, dtype=np.float64))
    with np.errstate(divide="ignore", invalid="ignore"):
        tab = np.exp(-1j * k * r) / (4.0 * np.pi * r)
    tab[0] = 0.0  # G_h(0) = 0
    out = np.zeros((q.shape[0], len(nodes)), dtype=np.complex128)
    step = max(1, chunk // max(len(nodes), 1))
    nd = nodes.astype(np.int32)
    sp = spts.astype(np.int32)
    for s0 in range(0, len(src), step):
        d2 = np.zeros((len(nodes), min(step, len(src) - s0)), dtype=np.int32)
        for ax in range(3):  # |u - v|^2 summed axis by axis: [T, chunk]
            dd = nd[:, ax, None] - sp[None, s0 : s0 + step, ax]
            d2 += dd * dd
        out += qs[:, s0 : s0 + step] @ tab[d2].T
    return out.reshape(lead + (len(nodes),))


def near_pairs(centres, radius):
    """All (m, n) with |c_m - c_n| <= radius, row-major sorted, self included."""
    from scipy.spatial import cKDTree

    tree = cKDTree(centres)
    cand = tree.query_pairs(radius * (1.0 + 1e-9), output_type="ndarray")
    a, b = cand[:, 0], cand[:, 1]
    d = centres[a] - centres[b]
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    keep = d2 <= radius * radius
    a, b = a[keep], b[keep]
    N = len(centres)
    rows = np.concatenate([a, b, np.arange(N)])
    cols = np.concatenate([b, a, np.arange(N)])
    order = np.lexsort((cols, rows))
    return rows[order], cols[order]


def aim_pair_values(lam, anc, rows, cols, h, k, M):
    """Grid approximation of Z_mn for explicit pairs.

    Z^AIM_mn = j k eta [ sum_{c=x,y,z} Lambda^c_m . G Lambda^c_n
                         - k^-2 Lambda^rho_m . G Lambda^rho_n ],
    G[s, t] = G_h(a_m + u_s - a_n - u_t).  Pairs are grouped by anchor offset
    so that each group shares one S x S matrix G.
    """
    off = stencil_offsets(M)
    d = anc[rows] - anc[cols]  # a_m - a_n
    keys, inv = np.unique(d, axis=0, return_inverse=True)
    inv = inv.ravel()
    out = np.zeros(len(rows), dtype=np.complex128)
    fac = np.array([1.0, 1.0, 1.0, -1.0 / (k * k)])
    for gi, dv in enumerate(keys):
        sel = np.nonzero(inv == gi)[0]
        Gd = grid_kernel(dv[None, None, :] + off[:, None, :] - off[None, :, :], h, k)  # [S, S]
        lm = lam[rows[sel]]  # [P, 4, S]
        ln = lam[cols[sel]]
        t = np.einsum("pcs,st->pct", lm, Gd)
        out[sel] = np.einsum("pct,pct,c->p", t, ln, fac)
    return (1j * k * ETA0) * out


class AIMOperator:
    """Plain FP64 AIM approximation of the EFIE matrix (Section 2.2), or of the
    CFIE matrix alpha ZE + (1 - alpha) eta ZM when alpha < 1 (closed bodies;
    the MFIE part is in ``mfie``)."""

    def __init__(self, rwg, k, h, M=2, near_radius=None, near_rows=None, alpha=1.0):
        self.rwg = rwg
        self.k = float(k)
        self.h = float(h)
        self.M = int(M)
        self.alpha = float(alpha)
        self.radius = 3.0 * h if near_radius is None else float(near_radius)
        self.N = rwg.N
        self.anc = anchors(rwg.centre, h, M)
        self.lo, self.n = grid_box(self.anc, M)
        self.L = np.array([smooth_length(2 * v - 1) for v in self.n])
        self.loc = self.anc - self.lo  # anchor in grid index space
        self.lam = moment_weights(rwg, h, M, self.anc)
        if self.alpha != 1.0:
            from .mfie import mfie_weights

            self.W = mfie_weights(rwg, h, M, self.anc)
        self._Ghat = None  # transformed on first use (convolve), see Ghat
        rows, cols = near_pairs(rwg.centre, self.radius)
        if near_rows is not None:  # restrict the correction to some rows
            keep = np.isin(rows, near_rows)
            rows, cols = rows[keep], cols[keep]
        self.near_rows, self.near_cols = rows, cols
        self.near_vals = self._near_values(rows, cols)
        self.Znear = scipy.sparse.csr_matrix((self.near_vals, (rows, cols)), shape=(self.N, self.N))

    @property
    def Ghat(self):
        """fftn of the circulant-embedded G_h on the padded grid (computed once, on first use)."""
        if self._Ghat is None:
            self._Ghat = scipy.fft.fftn(green_grid(self.n, self.L, self.h, self.k), workers=-1)
        return self._Ghat

    def _near_values(self, rows, cols):
        zmn = mom_entries(self.rwg, rows, cols, self.k)
        znm = mom_entries(self.rwg, cols, rows, self.k)
        zsym = 0.5 * (zmn + znm)
        ze = zsym - aim_pair_values(self.lam, self.anc, rows, cols, self.h, self.k, self.M)
        if self.alpha == 1.0:
            return ze
        from .mfie import mfie_entries, mfie_pair_values

        # ZM exact minus its grid form -<f_m, n x curl A_n>  (= -sum_c W^c_m G Lambda^c_n)
        zm = mfie_entries(self.rwg, rows, cols, self.k) + mfie_pair_values(
            self.W, self.lam, self.anc, rows, cols, self.h, self.k, self.M)
        return self.alpha * ze + (1.0 - self.alpha) * ETA0 * zm

    # --- the four steps of one product -----------------------------------
    def project(self, x, comps=(0, 1, 2, 3)):
        """Q_c(u) = sum_m Lambda^c_m(u - a_m) x_m on the n-grid: [B, len(comps), nz, ny, nx]
        for the components c in ``comps`` (0, 1, 2: x, y, z current; 3: charge)."""
        x = np.atleast_2d(x)
        B = x.shape[0]
        nx, ny, nz = self.n
        Q = np.zeros((B, len(comps), nz * ny * nx), dtype=np.complex128)
        off = stencil_offsets(self.M)
        node = self.loc[:, None, :] + off[None, :, :]  # [N, S, 3]
        flat = (node[..., 2] * ny + node[..., 1]) * nx + node[..., 0]
        for b in range(B):
            for ci, c in enumerate(comps):
                np.add.at(Q[b, ci], flat.ravel(), (self.lam[:, c, :] * x[b][:, None]).ravel())
        return Q.reshape(B, len(comps), nz, ny, nx)

    def convolve(self, Q):
        return convolve_fft(Q, self.Ghat, self.n, self.L)

    def interpolate(self, Phi, comps=(0, 1, 2, 3)):
        """y_m = j k eta [sum_{x,y,z} <Lambda^c_m, Phi_c> - k^-2 <Lambda^rho_m, Phi_rho>].

        Phi: [B, len(comps), nz, ny, nx], the potentials of the components in
        ``comps``; the sum runs over those components only (all four give the
        product's grid part)."""
        B = Phi.shape[0]
        nx, ny, nz = self.n
        off = stencil_offsets(self.M)
        node = self.loc[:, None, :] + off[None, :, :]
        flat = (node[..., 2] * ny + node[..., 1]) * nx + node[..., 0]
        P = Phi.reshape(B, len(comps), -1)
        fac = np.array([1.0, 1.0, 1.0, -1.0 / (self.k * self.k)])
        y = np.zeros((B, self.N), dtype=np.complex128)
        for ci, c in enumerate(comps):
            y += fac[c] * np.einsum("ms,bms->bm", self.lam[:, c, :], P[:, ci][:, flat])
        y = (1j * self.k * ETA0) * y
        if self.alpha == 1.0:
            return y
        # MFIE: -<f_m, n x curl A> with the differentiated interpolation weights
        ym = np.zeros((B, self.N), dtype=np.complex128)
        for ci, c in enumerate(comps):
            if c < 3:
                ym -= np.einsum("ms,bms->bm", self.W[:, c, :], P[:, ci][:, flat])
        return self.alpha * y + (1.0 - self.alpha) * ETA0 * ym

    def matvec(self, x):
        """One AIM product: projection, FFT convolution, interpolation, near correction."""
        x = np.atleast_2d(np.asarray(x, dtype=np.complex128))
        y = self.interpolate(self.convolve(self.project(x)))
        y += (self.Znear @ x.T).T
        return y

    def matvec_rows(self, x, rows):
        """Rows ``rows`` of one product, with the grid convolution summed directly
        at the stencil nodes of those rows (``convolve_direct_at``) instead of the
        padded FFT: the same four steps (projection of every basis function,
        convolution, interpolation, near correction) evaluated only where the
        listed rows read them.  The near correction must cover these rows
        (``near_rows`` at construction includes them, or is None)."""
        x = np.atleast_2d(np.asarray(x, dtype=np.complex128))
        rows = np.asarray(rows, dtype=np.int64)
        Q = self.project(x)  # [B, 4, nz, ny, nx]
        off = stencil_offsets(self.M)
        node = self.loc[rows][:, None, :] + off[None, :, :]  # [R, S, 3]
        uniq, inv = np.unique(node.reshape(-1, 3), axis=0, return_inverse=True)
        phi_u = convolve_direct_at(Q, uniq, self.h, self.k)  # [B, 4, U]
        P = phi_u[..., inv.ravel()].reshape(x.shape[0], 4, len(rows), len(off))  # [B, 4, R, S]
        fac = np.array([1.0, 1.0, 1.0, -1.0 / (self.k * self.k)])
        y = np.zeros((x.shape[0], len(rows)), dtype=np.complex128)
        for c in range(4):
            y += fac[c] * np.einsum("rs,brs->br", self.lam[rows, c, :], P[:, c])
        y = (1j * self.k * ETA0) * y
        if self.alpha != 1.0:
            ym = np.zeros_like(y)
            for c in range(3):
                ym -= np.einsum("rs,brs->br", self.W[rows, c, :], P[:, c])
            y = self.alpha * y + (1.0 - self.alpha) * ETA0 * ym
        y += (self.Znear[rows] @ x.T).T
        return y

    def far_matvec(self, x):
        """Grid part only (no near correction)."""
        x = np.atleast_2d(np.asarray(x, dtype=np.complex128))
        return self.interpolate(self.convolve(self.project(x)))

    def diagonal(self):
        """diag(Z~): grid self term plus the near (self) correction = MoM self term."""
        d = self.Znear.diagonal().copy()
        idx = np.arange(self.N)
        ge = aim_pair_values(self.lam, self.anc, idx, idx, self.h, self.k, self.M)
        if self.alpha == 1.0:
            return d + ge
        from .mfie import mfie_pair_values

        gm = -mfie_pair_values(self.W, self.lam, self.anc, idx, idx, self.h, self.k, self.M)
        return d + self.alpha * ge + (1.0 - self.alpha) * ETA0 * gm
