"""Closed, outward-oriented triangle meshes used as synthetic workloads.

Every generator returns ``(verts, tris)``: ``verts`` float64 (Nv, 3) in metres,
``tris`` int32 (Nt, 3) with counter-clockwise vertex order seen from outside
(right-hand normal points out of the enclosed volume).  All meshes are closed
2-manifolds, so every edge is shared by exactly two triangles.
"""
import numpy as np


def _icosahedron():
    p = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([
        [-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
        [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
        [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1],
    ], dtype=np.float64)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int64)
    return v / np.linalg.norm(v, axis=1, keepdims=True), f


def icosphere(level, radius=1.0, equal_volume=False):
    """Icosahedron refined ``level`` times (each triangle split in 4) and
    projected onto the sphere of the given radius: 20*4**level triangles,
    30*4**level edges.  equal_volume=True scales the vertices out so that the
    polyhedron encloses the same volume as the sphere (the flat faces of an
    inscribed mesh otherwise shrink the scatterer by O(h^2))."""
    v, f = _icosahedron()
    verts = [tuple(x) for x in v]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = np.add(verts[a], verts[b]) * 0.5
                m /= np.linalg.norm(m)
                verts.append(tuple(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        f = np.array(nf, dtype=np.int64)
    V = np.array(verts, dtype=np.float64) * radius
    # orient outward (the base icosahedron list is outward; keep a check)
    g = V[f].mean(axis=1)
    n = np.cross(V[f[:, 1]] - V[f[:, 0]], V[f[:, 2]] - V[f[:, 0]])
    flip = np.einsum("ij,ij->i", n, g) < 0
    f[flip] = f[flip][:, [0, 2, 1]]
    if equal_volume:
        a, b, c = V[f[:, 0]], V[f[:, 1]], V[f[:, 2]]
        vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0
        V = V * (4.0 / 3.0 * np.pi * radius ** 3 / vol) ** (1.0 / 3.0)
    return V, f.astype(np.int32)


def box(size, divisions, center=(0.0, 0.0, 0.0)):
    """Axis-aligned box with side lengths ``size`` = (Lx, Ly, Lz), each face
    split into a structured grid of ``divisions`` = (nx, ny, nz) cells per axis,
    every cell cut into two right triangles."""
    L = np.asarray(size, dtype=np.float64)
    nd = np.asarray(divisions, dtype=np.int64)
    c0 = np.asarray(center, dtype=np.float64) - 0.5 * L
    index = {}
    verts = []

    def vid(i, j, k):
        key = (i, j, k)
        if key not in index:
            index[key] = len(verts)
            verts.append(c0 + L * np.array([i, j, k], dtype=np.float64) / nd)
        return index[key]

    tris = []
    # each face: fixed axis a at side s (0 or n_a); the two in-plane axes (b, c)
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        for s in (0, nd[a]):
            for i in range(nd[b]):
                for j in range(nd[c]):
                    def node(di, dj):
                        idx = [0, 0, 0]
                        idx[a], idx[b], idx[c] = s, i + di, j + dj
                        return vid(*idx)
                    q = [node(0, 0), node(1, 0), node(1, 1), node(0, 1)]
                    # (b, c, a) is right-handed, so CCW in (b, c) points along +a
                    if s == 0:
                        q = q[::-1]
                    tris.append([q[0], q[1], q[2]])
                    tris.append([q[0], q[2], q[3]])
    return np.array(verts, dtype=np.float64), np.array(tris, dtype=np.int32)


def bar_cluster(seed, target_triangles=200_000, unit=1e-6):
    """Seeded cluster of 1-8 parallel rectangular bars.

    Bar length U[50, 500] um, cross-section sides U[1, 10] um, spacing between
    neighbours U[2, 20] um; faces meshed with structured right triangles whose
    cell size is chosen so that the whole cluster has about
    ``target_triangles`` triangles.  Returns (verts, tris, obj_id)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nbar = int(rng.integers(1, 9))
    dims = []
    for _ in range(nbar):
        dims.append((rng.uniform(50, 500) * unit, rng.uniform(1, 10) * unit,
                     rng.uniform(1, 10) * unit))
    gaps = [rng.uniform(2, 20) * unit for _ in range(nbar)]
    area = sum(2 * (a * b + b * c + c * a) for a, b, c in dims)
    cell = np.sqrt(area / (target_triangles / 2.0))
    V, T, O = [], [], []
    y = 0.0
    for i, (lx, ly, lz) in enumerate(dims):
        div = [max(1, int(round(lx / cell))), max(1, int(round(ly / cell))),
               max(1, int(round(lz / cell)))]
        v, t = box((lx, ly, lz), div, center=(0.0, y + 0.5 * ly, 0.0))
        T.append(t + sum(len(x) for x in V))
        V.append(v)
        O.append(np.full(len(t), i, dtype=np.int32))
        y += ly + gaps[i]
    return np.vstack(V), np.vstack(T).astype(np.int32), np.concatenate(O)


def mesh_edges_count(tris):
    """Number of distinct undirected edges of a triangle list."""
    e = np.sort(np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]]), axis=1)
    return len(np.unique(e, axis=0))
