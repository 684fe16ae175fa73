"""RWG basis functions on a triangle mesh (oracle; test infrastructure only).

The paper meshes its scatterers with triangles (Section 2.1) and solves the
EFIE by the method of moments (Section 2.2); the unknowns are the standard
Rao-Wilton-Glisson edge functions, one per interior edge:

    f(r) = +l / (2 A+) (r - p+)   on T+,     div f = +l / A+
    f(r) = -l / (2 A-) (r - p-)   on T-,     div f = -l / A-

Conventions (the paper is silent; these are fixed choices):
* the unknowns are the interior edges sorted by (low vertex, high vertex);
* T+ is the lower-indexed of the two triangles, T- the higher;
* p+/p- is the vertex of T+/T- that is not on the edge;
* the centre c of a basis function is the edge midpoint (v_lo + v_hi) * 0.5.
"""

import numpy as np


class RWG:
    """Plain container for the RWG data of a mesh."""

    def __init__(self, verts, tris):
        verts = np.asarray(verts, dtype=np.float64)
        tris = np.asarray(tris, dtype=np.int64)
        self.verts = verts
        self.tris = tris
        nt = len(tris)
        r0, r1, r2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
        cr = np.cross(r1 - r0, r2 - r0)
        self.tri_area = 0.5 * np.sqrt((cr * cr).sum(axis=1))
        # edge -> triangles, plain dictionary walk
        owners = {}
        for t in range(nt):
            for k in range(3):
                a, b = int(tris[t, k]), int(tris[t, (k + 1) % 3])
                key = (min(a, b), max(a, b))
                owners.setdefault(key, []).append(t)
        for key, ts in owners.items():
            if len(ts) > 2:
                raise ValueError(f"non-manifold edge {key}")
        interior = sorted(key for key, ts in owners.items() if len(ts) == 2)
        N = len(interior)
        self.N = N
        self.edge = np.array(interior, dtype=np.int64).reshape(N, 2)
        self.tri_p = np.empty(N, dtype=np.int64)
        self.tri_m = np.empty(N, dtype=np.int64)
        self.free_p = np.empty(N, dtype=np.int64)
        self.free_m = np.empty(N, dtype=np.int64)
        # local slot of the basis function in each triangle = index (0..2) of
        # its free vertex in the triangle's stored vertex list
        self.slot_p = np.empty(N, dtype=np.int64)
        self.slot_m = np.empty(N, dtype=np.int64)
        for m, key in enumerate(interior):
            tp, tm = sorted(owners[key])
            self.tri_p[m], self.tri_m[m] = tp, tm
            for t, fv, sl in ((tp, self.free_p, self.slot_p), (tm, self.free_m, self.slot_m)):
                for k in range(3):
                    v = int(tris[t, k])
                    if v != key[0] and v != key[1]:
                        fv[m] = v
                        sl[m] = k
        d = verts[self.edge[:, 1]] - verts[self.edge[:, 0]]
        self.length = np.sqrt((d * d).sum(axis=1))
        self.centre = (verts[self.edge[:, 0]] + verts[self.edge[:, 1]]) * 0.5
        self.area_p = self.tri_area[self.tri_p]
        self.area_m = self.tri_area[self.tri_m]

    def halves(self):
        """Iterate over the two halves: (tri, free vertex, slot, sign, area)."""
        yield self.tri_p, self.free_p, self.slot_p, 1.0, self.area_p
        yield self.tri_m, self.free_m, self.slot_m, -1.0, self.area_m

    def eval_f(self, m, r):
        """f_m at points r [..., 3] lying on T+ (first) or T- (second), by half.

        Returns (f on T+ evaluated at r, f on T- evaluated at r); the caller
        picks the half its points lie on.
        """
        l = self.length[m]
        fp = (l / (2.0 * self.area_p[m])) * (r - self.verts[self.free_p[m]])
        fm = -(l / (2.0 * self.area_m[m])) * (r - self.verts[self.free_m[m]])
        return fp, fm
