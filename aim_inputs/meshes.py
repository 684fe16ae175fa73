"""Triangle meshes of the benchmark scatterers (Section 2.1 of the paper).

Lengths are in wavelengths.  Every mesh is returned as ``(verts, tris)`` with
``verts`` float64 [nv, 3] and ``tris`` int32 [nt, 3]; every triangle is
ordered counter-clockwise about its outward (plate: +z) normal.  The vertex
and triangle orders are deterministic, so a mesh built twice is bit-identical.
"""

import numpy as np


def plate_mesh(side, n_squares):
    """Square plate [-side/2, side/2]^2 in the z=0 plane.

    The plate is cut into ``n_squares`` x ``n_squares`` squares; square (i, j)
    (i along x, j along y) is split by its diagonal from (x_i, y_j) to
    (x_{i+1}, y_{j+1}) into the triangles (v_ij, v_i+1j, v_i+1j+1) and
    (v_ij, v_i+1j+1, v_ij+1).  Vertex (i, j) has index j*(n_squares+1)+i.
    Section 2.1: plate centred at the origin on the x-y plane, mean edge about
    lambda/9 (side=1, n_squares=9 gives edges lambda/9 and diagonals
    sqrt(2) lambda/9).
    """
    n = int(n_squares)
    if n < 1:
        raise ValueError("n_squares must be >= 1")
    t = np.arange(n + 1, dtype=np.float64) * (float(side) / n) - 0.5 * float(side)
    X, Y = np.meshgrid(t, t, indexing="xy")  # [j, i]
    verts = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    i = i.ravel()
    j = j.ravel()
    v00 = j * (n + 1) + i
    v10 = v00 + 1
    v01 = v00 + (n + 1)
    v11 = v01 + 1
    tris = np.empty((2 * n * n, 3), dtype=np.int32)
    tris[0::2] = np.stack([v00, v10, v11], axis=1)
    tris[1::2] = np.stack([v00, v11, v01], axis=1)
    return verts, tris


def rect_plate_mesh(side_x, side_y, nx_squares, ny_squares):
    """Rectangular plate [-side_x/2, side_x/2] x [-side_y/2, side_y/2] in the z=0
    plane, cut into nx_squares x ny_squares cells split as in ``plate_mesh``
    (vertex (i, j) has index j*(nx_squares+1)+i).  Long strips of it give
    padded grid lengths far apart on the two axes."""
    nx, ny = int(nx_squares), int(ny_squares)
    if nx < 1 or ny < 1:
        raise ValueError("square counts must be >= 1")
    tx = np.arange(nx + 1, dtype=np.float64) * (float(side_x) / nx) - 0.5 * float(side_x)
    ty = np.arange(ny + 1, dtype=np.float64) * (float(side_y) / ny) - 0.5 * float(side_y)
    X, Y = np.meshgrid(tx, ty, indexing="xy")  # [j, i]
    verts = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    i = i.ravel()
    j = j.ravel()
    v00 = j * (nx + 1) + i
    v10 = v00 + 1
    v01 = v00 + (nx + 1)
    v11 = v01 + 1
    tris = np.empty((2 * nx * ny, 3), dtype=np.int32)
    tris[0::2] = np.stack([v00, v10, v11], axis=1)
    tris[1::2] = np.stack([v00, v11, v01], axis=1)
    return verts, tris


def _icosahedron():
    phi = (1.0 + np.sqrt(5.0)) / 2.0
    v = []
    for a in (-1.0, 1.0):
        for b in (-phi, phi):
            v.append((0.0, a, b))
            v.append((a, b, 0.0))
            v.append((b, 0.0, a))
    v = np.array(v, dtype=np.float64)
    # order vertices deterministically (lexicographic)
    order = np.lexsort((v[:, 2], v[:, 1], v[:, 0]))
    v = v[order]
    faces = []
    d2 = ((v[:, None, :] - v[None, :, :]) ** 2).sum(-1)
    adj = np.abs(d2 - 4.0) < 1e-9  # edge length 2 for this vertex set
    for a in range(12):
        for b in range(a + 1, 12):
            if not adj[a, b]:
                continue
            for c in range(b + 1, 12):
                if adj[a, c] and adj[b, c]:
                    nrm = np.cross(v[b] - v[a], v[c] - v[a])
                    if np.dot(nrm, v[a] + v[b] + v[c]) > 0:
                        faces.append((a, b, c))
                    else:
                        faces.append((a, c, b))
    assert len(faces) == 20
    return v, faces


def icosphere_mesh(radius, freq):
    """Class-I geodesic icosphere of frequency ``freq`` projected to ``radius``.

    Each icosahedron face (A, B, C) is cut into freq^2 triangles on the
    barycentric lattice P(i, j) = A + (i/freq)(B-A) + (j/freq)(C-A); all
    lattice points are then pushed radially onto the sphere.  Lattice points on
    an icosahedron edge are computed from that edge alone (low vertex index to
    high), so every shared vertex has one set of coordinates.  10 f^2 + 2
    vertices, 20 f^2 triangles, 30 f^2 edges (all interior: the surface is
    closed).
    """
    f = int(freq)
    if f < 1:
        raise ValueError("freq must be >= 1")
    iv, faces = _icosahedron()
    coords = [iv[k] for k in range(12)]
    edge_base = {}
    edges = sorted({(min(a, b), max(a, b)) for (A, B, C) in faces for (a, b) in ((A, B), (B, C), (C, A))})
    for (a, b) in edges:
        edge_base[(a, b)] = len(coords)
        for s in range(1, f):
            coords.append(iv[a] + (s / f) * (iv[b] - iv[a]))

    def edge_point(a, b, s):
        # point s/f of the way from ico vertex a to ico vertex b
        if s == 0:
            return a
        if s == f:
            return b
        if a < b:
            return edge_base[(a, b)] + s - 1
        return edge_base[(b, a)] + (f - s) - 1

    tris = []
    for (A, B, C) in faces:
        idx = {}
        for i in range(f + 1):
            for j in range(f + 1 - i):
                k = f - i - j  # weight on A
                if i == 0 and j == 0:
                    idx[(i, j)] = A
                elif i == f:
                    idx[(i, j)] = B
                elif j == f:
                    idx[(i, j)] = C
                elif j == 0:
                    idx[(i, j)] = edge_point(A, B, i)
                elif i == 0:
                    idx[(i, j)] = edge_point(A, C, j)
                elif k == 0:
                    idx[(i, j)] = edge_point(B, C, j)
                else:
                    idx[(i, j)] = len(coords)
                    coords.append(iv[A] + (i / f) * (iv[B] - iv[A]) + (j / f) * (iv[C] - iv[A]))
        for i in range(f):
            for j in range(f - i):
                tris.append((idx[(i, j)], idx[(i + 1, j)], idx[(i, j + 1)]))
                if i + j <= f - 2:
                    tris.append((idx[(i + 1, j)], idx[(i + 1, j + 1)], idx[(i, j + 1)]))
    P = np.array(coords, dtype=np.float64)
    P = P * (float(radius) / np.sqrt((P * P).sum(axis=1)))[:, None]
    return P, np.array(tris, dtype=np.int32)


def mesh_mean_edge(verts, tris):
    """Mean length over the unique edges of a triangle mesh."""
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    e = np.unique(np.sort(e, axis=1), axis=0)
    d = verts[e[:, 0]] - verts[e[:, 1]]
    return float(np.sqrt((d * d).sum(axis=1)).mean())


def icosphere_frequency(radius, target_edge=1.0 / 9.0):
    """Smallest icosphere frequency whose mean edge is <= ``target_edge``.

    Section 2.1 meshes the sphere at a mean edge of about lambda/9.  The mean
    edge times the frequency tends to a constant, so the search starts from
    the estimate made at frequency 16 and walks to the exact answer.
    """
    c = mesh_mean_edge(*icosphere_mesh(1.0, 16)) * 16.0
    f = max(1, int(np.ceil(c * radius / target_edge)) - 1)
    while f > 1 and mesh_mean_edge(*icosphere_mesh(radius, f - 1)) <= target_edge:
        f -= 1
    while mesh_mean_edge(*icosphere_mesh(radius, f)) > target_edge:
        f += 1
    return f
