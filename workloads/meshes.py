"""Structured and Kuhn-split meshes as element-to-DOF connectivity.

Every generator returns ``int32 [n_e, n_loc]`` with the DOFs of each element
in local order.  DOFs are interleaved per node, ``dof = d*node + comp``, which
is the layout the paper's d-benchmark assumes (the DOFs of one node are
contiguous, §4 remark on the h-, p- and d-benchmarks).
"""

import numpy as np


def _interleave(node_conn: np.ndarray, d: int) -> np.ndarray:
    """Expand node connectivity [n_e, n_nodes] to DOFs [n_e, n_nodes*d]."""
    node_conn = np.asarray(node_conn, dtype=np.int64)
    if d == 1:
        return node_conn.astype(np.int32)
    comp = np.arange(d, dtype=np.int64)
    dofs = node_conn[:, :, None] * d + comp[None, None, :]
    return dofs.reshape(node_conn.shape[0], -1).astype(np.int32)


def quad_q1_grid(m: int, d: int = 1):
    """m x m bilinear Q1 quads on the unit square, natural node numbering.

    Node (i, j) has id ``i + (m+1)*j``.  Local node order is counter-clockwise:
    (i,j), (i+1,j), (i+1,j+1), (i,j+1).  Elements are numbered x fastest.
    Returns (elem_dofs int32 [m*m, 4*d], n_dofs).
    """
    i, j = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    i = i.ravel()
    j = j.ravel()
    s = m + 1
    nodes = np.stack([i + s * j, i + 1 + s * j, i + 1 + s * (j + 1), i + s * (j + 1)], axis=1)
    return _interleave(nodes, d), d * s * s


def quad_qp_grid(m: int, p: int, d: int = 1):
    """m x m structured Lagrange Q_p quads (equispaced nodes), natural numbering.

    The global node lattice is (m*p+1)^2 with id ``a + (m*p+1)*b``; the local
    nodes of an element are its (p+1)^2 lattice points, x fastest.
    Returns (elem_dofs int32 [m*m, (p+1)^2*d], n_dofs).
    """
    s = m * p + 1
    ei, ej = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    ei = ei.ravel()
    ej = ej.ravel()
    la, lb = np.meshgrid(np.arange(p + 1), np.arange(p + 1), indexing="xy")
    la = la.ravel()
    lb = lb.ravel()
    a = ei[:, None] * p + la[None, :]
    b = ej[:, None] * p + lb[None, :]
    nodes = a + s * b
    return _interleave(nodes, d), d * s * s


def paper_sweep_points():
    """The p- and d-benchmark meshes of §4 on structured squares, as
    (benchmark, m, p, d): Q_p quads on the 4th mesh (48 x 48) for p = 1..8 at
    d = 1 and p = 1..4 at d = 4; Q1 on the 6th mesh (192 x 192) for d = 1..8;
    Q1 on the 4th mesh at d = 20."""
    pts = [("p_d1", 48, p, 1) for p in range(1, 9)]
    pts += [("p_d4", 48, p, 4) for p in range(1, 5)]
    pts += [("d", 192, 1, d) for d in range(1, 9)]
    pts.append(("d20", 48, 1, 20))
    return pts


def hex_q1_grid(n: int, d: int = 1):
    """n^3 trilinear Q1 hexes on the unit cube, natural lexicographic numbering.

    Node (i, j, k) has id ``i + (n+1)*j + (n+1)^2*k``; local node order is
    lexicographic with x fastest: (0,0,0), (1,0,0), (0,1,0), (1,1,0),
    (0,0,1), ...  Elements are numbered x fastest.
    Returns (elem_dofs int32 [n^3, 8*d], n_dofs).
    """
    s = n + 1
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    i = i.ravel().astype(np.int64)
    j = j.ravel().astype(np.int64)
    k = k.ravel().astype(np.int64)
    base = i + s * j + s * s * k
    offs = np.array([dx + s * dy + s * s * dz
                     for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)], dtype=np.int64)
    nodes = base[:, None] + offs[None, :]
    return _interleave(nodes, d), d * s ** 3


_KUHN_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))
_P2_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


def tet_p2_kuhn(n: int, d: int = 3, seed: int = 0, permute: bool = True,
                with_coords: bool = False, jitter: float = 0.2):
    """Quadratic P2 tets from an n^3 hex grid split into 6 Kuhn tets per cube.

    The tets of a cube follow the 6 monotone lattice paths from corner
    (0,0,0) to (1,1,1), one per axis permutation.  The P2 nodes are the
    vertices and edge midpoints; on the Kuhn split they are exactly the
    points of the (2n+1)^3 half-step lattice.  Local order: v0..v3, then the
    midpoints of edges 01, 02, 03, 12, 13, 23.  With ``permute`` the global
    node ids are shuffled by a seeded permutation.  Node coordinates (only
    produced on request) are jittered by up to ``jitter*h`` at interior
    vertices; assembly does not depend on them.

    Returns (elem_dofs int32 [6 n^3, 10*d], n_dofs) and, with
    ``with_coords``, the float64 [(2n+1)^3, 3] coordinates as a third item.
    """
    s = 2 * n + 1
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    corner = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.int64) * 2
    n_cubes = corner.shape[0]
    eye = np.eye(3, dtype=np.int64) * 2
    tets = []
    for perm in _KUHN_PERMS:
        v0 = np.zeros(3, dtype=np.int64)
        v1 = v0 + eye[perm[0]]
        v2 = v1 + eye[perm[1]]
        v3 = np.full(3, 2, dtype=np.int64)
        verts = [v0, v1, v2, v3]
        loc = verts + [(verts[a] + verts[b]) // 2 for a, b in _P2_EDGES]
        tets.append(np.stack(loc, axis=0))  # [10, 3]
    tets = np.stack(tets, axis=0)  # [6, 10, 3]
    pts = corner[:, None, None, :] + tets[None, :, :, :]  # [n_cubes, 6, 10, 3]
    nodes = pts[..., 0] + s * pts[..., 1] + s * s * pts[..., 2]
    nodes = nodes.reshape(n_cubes * 6, 10)
    n_nodes = s ** 3
    if permute:
        rng = np.random.default_rng(seed)
        perm = rng.permutation(n_nodes).astype(np.int64)
        nodes = perm[nodes]
    else:
        perm = None
    out = (_interleave(nodes, d), d * n_nodes)
    if with_coords:
        rng = np.random.default_rng(seed + 0x9E3779B9)
        c, b, a = np.meshgrid(np.arange(s), np.arange(s), np.arange(s), indexing="ij")
        lat = np.stack([a.ravel(), b.ravel(), c.ravel()], axis=1)
        xyz = lat.astype(np.float64) / (2 * n)
        is_vertex = np.all(lat % 2 == 0, axis=1)
        interior = np.all((lat > 0) & (lat < 2 * n), axis=1)
        move = is_vertex & interior
        xyz[move] += rng.uniform(-jitter, jitter, size=(int(move.sum()), 3)) / n
        if perm is not None:
            coords = np.empty_like(xyz)
            coords[perm] = xyz
        else:
            coords = xyz
        out = out + (coords,)
    return out


def batched_mesh_sizes(count: int = 256, lo: int = 8, hi: int = 48, seed: int = 0):
    """Side lengths of a batch of hex meshes, log-uniform in [lo, hi].

    ``n = round(exp(U(ln lo, ln hi)))`` from a seeded generator.  The first
    half of the batch is scalar (d = 1), the second half vector (d = 3).
    Returns a list of (n, d) pairs.
    """
    rng = np.random.default_rng(seed)
    u = rng.uniform(np.log(lo), np.log(hi), size=count)
    ns = np.rint(np.exp(u)).astype(int)
    half = count // 2
    return [(int(ns[t]), 1 if t < half else 3) for t in range(count)]
