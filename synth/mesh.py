"""Layer-conforming mapped-grid meshes of 10-node (quadratic) tetrahedra.

The paper meshes each candidate ground model with second-order tetrahedra
(Section 3, computational-cost paragraph).  Its octree mesher is not
available, so the synthetic stand-in is a structured lateral grid whose
vertical levels follow the layer interfaces column by column:

* lateral cells of size ``Lx/nx`` by ``Ly/ny``;
* in every column the depth range of layer ``l`` is split into ``n_l``
  uniform cells, so every layer interface passes through mesh nodes and each
  element lies in exactly one layer;
* each hexahedral cell is cut into the 6 Kuhn (Freudenthal) tetrahedra that
  share its (0,0,0)-(1,1,1) diagonal, which is conforming across cells;
* the mid-edge nodes sit on the doubled lattice at the midpoints of the
  edges, so every element is straight-sided (affine) and the node count is
  ``(2nx+1)(2ny+1)(2nz+1)`` (``2nx * 2ny * (2nz+1)`` when periodic).

Node ordering is lexicographic on the doubled lattice (x fastest, then y,
then z from the base upward).  Element ordering is cell by cell in the same
lexicographic order, six tetrahedra per cell.

Element node order is the VTK quadratic-tetrahedron order: vertices 0..3,
then the mid-edge nodes of edges (0,1), (1,2), (0,2), (0,3), (1,3), (2,3).
Vertices are ordered so that det[x1-x0, x2-x0, x3-x0] > 0.

Boundary faces are 6-node triangles (3 vertices, then the mid-edge nodes of
edges (0,1), (1,2), (2,0)) tagged ``FACE_TOP`` (free surface z = 0),
``FACE_BASE`` (z = -depth) or ``FACE_SIDE`` (x or y extremes; absent when
periodic).  ``face_elem`` names the element each face belongs to.
"""
import itertools

import numpy as np

VTK_TET10_EDGES = ((0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3))
TRI6_EDGES = ((0, 1), (1, 2), (2, 0))
FACE_TOP, FACE_BASE, FACE_SIDE = 0, 1, 2


def _kuhn_corners():
    """Corner offsets (0/1 per axis) of the 6 Kuhn tetrahedra of a unit cube."""
    tets = []
    for perm in itertools.permutations(range(3)):
        cur = np.zeros(3, dtype=np.int64)
        corners = [cur.copy()]
        for ax in perm:
            cur[ax] = 1
            corners.append(cur.copy())
        tets.append(np.array(corners))
    return tets


def column_levels(depths_top_to_bottom, counts):
    """Depth levels (top to bottom) of one column.

    ``depths_top_to_bottom``: interface depths d_0 = 0 < d_1 < ... < d_L (the
    last is the model bottom).  ``counts``: cells per layer.  Returns
    ``sum(counts) + 1`` depths, uniform inside each layer.
    """
    out = [0.0]
    for l, n in enumerate(counts):
        a, b = depths_top_to_bottom[l], depths_top_to_bottom[l + 1]
        out.extend(list(a + (b - a) * np.arange(1, n + 1) / n))
    return np.array(out)


def layered_box(nx, ny, Lx, Ly, counts, interfaces, depth, periodic=False):
    """Build a layered box mesh.

    Parameters
    ----------
    nx, ny : lateral cell counts.
    Lx, Ly : lateral extent in metres (x in [0, Lx], y in [0, Ly]).
    counts : cells per layer, top layer first (layer index = material id).
    interfaces : list of ``len(counts) - 1`` arrays of shape (nx+1, ny+1)
        (or scalars) with the depth of the bottom of layers 0..L-2 at the
        lateral vertex lattice points.  Must be strictly increasing with
        layer index and strictly shallower than ``depth``.
    depth : model bottom depth (flat base at z = -depth).
    periodic : wrap the lattice in x and y (laterally uniform levels only).

    Returns a dict with float64 ``xyz`` [N,3], int32 ``conn`` [E,10],
    int32 ``elem_mat`` [E], int32 ``faces`` [F,6], int32 ``face_elem`` [F],
    int32 ``face_tag`` [F], float64 ``period`` [2] (0 = not periodic) and the
    lattice sizes.
    """
    counts = [int(c) for c in counts]
    nz = sum(counts)
    nL = len(counts)
    assert len(interfaces) == nL - 1
    hx, hy = Lx / nx, Ly / ny
    # depth of every interface at every lateral vertex
    dep = np.zeros((nL + 1, nx + 1, ny + 1))
    for l, itf in enumerate(interfaces):
        dep[l + 1] = np.broadcast_to(np.asarray(itf, dtype=np.float64), (nx + 1, ny + 1))
    dep[nL] = depth
    assert np.all(np.diff(dep, axis=0) > 0), "interfaces must be strictly increasing in depth"
    # z of vertex level k (k = 0 base ... nz top) per column
    Z = np.zeros((nx + 1, ny + 1, nz + 1))
    for i in range(nx + 1):
        for j in range(ny + 1):
            lev = column_levels(dep[:, i, j], counts)  # top to bottom depths
            Z[i, j, :] = -lev[::-1]
    if periodic:
        # element extents must stay below half a period for minimum-image unwrapping
        assert nx >= 3 and ny >= 3, "periodic meshes need at least 3 cells per direction"
        assert np.allclose(Z, Z[:1, :1, :]), "periodic meshes need laterally uniform levels"

    NX2 = 2 * nx if periodic else 2 * nx + 1
    NY2 = 2 * ny if periodic else 2 * ny + 1
    NZ2 = 2 * nz + 1
    n_nodes = NX2 * NY2 * NZ2

    def nid(I, J, K):
        if periodic:
            I = I % NX2
            J = J % NY2
        return (K * NY2 + J) * NX2 + I

    # unwrapped coordinates of the full doubled lattice
    full = np.zeros((2 * nx + 1, 2 * ny + 1, NZ2, 3))
    Iv, Jv, Kv = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    full[2 * Iv, 2 * Jv, 2 * Kv, 0] = Iv * hx
    full[2 * Iv, 2 * Jv, 2 * Kv, 1] = Jv * hy
    full[2 * Iv, 2 * Jv, 2 * Kv, 2] = Z

    # layer of each cell layer k (k from the base)
    layer_of_k = np.zeros(nz, dtype=np.int32)
    kk = nz
    for l, n in enumerate(counts):  # top layer first
        layer_of_k[kk - n:kk] = l
        kk -= n

    corners = _kuhn_corners()
    # orientation decided on the undistorted lattice
    tet_vertices = []
    for c in corners:
        d = np.linalg.det(np.stack([c[1] - c[0], c[2] - c[0], c[3] - c[0]], axis=1).astype(float))
        if d < 0:
            c = c[[0, 2, 1, 3]]
        tet_vertices.append(c)

    E = nx * ny * nz * 6
    conn = np.zeros((E, 10), dtype=np.int64)
    elem_mat = np.zeros(E, dtype=np.int32)
    lat = np.zeros((E, 10, 3), dtype=np.int64)  # doubled-lattice coords (unwrapped)
    e = 0
    cells = [(i, j, k) for k in range(nz) for j in range(ny) for i in range(nx)]
    base = np.array(cells, dtype=np.int64)  # [C,3]
    C = len(cells)
    for t, cv in enumerate(tet_vertices):
        V = 2 * base[:, None, :] + 2 * cv[None, :, :]  # [C,4,3]
        lat[t::6, :4] = V
        for m, (a, b) in enumerate(VTK_TET10_EDGES):
            lat[t::6, 4 + m] = (V[:, a] + V[:, b]) // 2
    # element order: cell-major, 6 tets per cell
    cell_of_e = np.repeat(np.arange(C), 6)
    elem_mat[:] = layer_of_k[base[cell_of_e, 2]]
    # mid-edge coordinates = average of edge endpoints
    for m, (a, b) in enumerate(VTK_TET10_EDGES):
        A = lat[:, a]
        B = lat[:, b]
        M = lat[:, 4 + m]
        full[M[:, 0], M[:, 1], M[:, 2]] = 0.5 * (full[A[:, 0], A[:, 1], A[:, 2]] + full[B[:, 0], B[:, 1], B[:, 2]])
    conn[:] = nid(lat[..., 0], lat[..., 1], lat[..., 2])

    xyz = np.zeros((n_nodes, 3))
    I2, J2, K2 = np.meshgrid(np.arange(NX2), np.arange(NY2), np.arange(NZ2), indexing="ij")
    xyz[nid(I2, J2, K2).ravel()] = full[I2, J2, K2].reshape(-1, 3)

    # boundary faces: faces of each tet whose 3 vertices lie on one boundary plane
    faces, face_elem, face_tag = [], [], []
    for opp in range(4):
        fv = [v for v in range(4) if v != opp]
        L = lat[:, fv]  # [E,3,3]
        planes = [(FACE_BASE, L[..., 2] == 0), (FACE_TOP, L[..., 2] == 2 * nz)]
        if not periodic:
            planes += [(FACE_SIDE, L[..., 0] == 0), (FACE_SIDE, L[..., 0] == 2 * nx),
                       (FACE_SIDE, L[..., 1] == 0), (FACE_SIDE, L[..., 1] == 2 * ny)]
        for tag, on in planes:
            sel = np.nonzero(on.all(axis=1))[0]
            if sel.size == 0:
                continue
            vv = conn[sel][:, fv]
            mids = np.stack([nid(*((lat[sel, fv[a]] + lat[sel, fv[b]]) // 2).T)
                             for (a, b) in TRI6_EDGES], axis=1)
            faces.append(np.concatenate([vv, mids], axis=1))
            face_elem.append(sel)
            face_tag.append(np.full(sel.size, tag))
    faces = np.concatenate(faces) if faces else np.zeros((0, 6))
    face_elem = np.concatenate(face_elem) if face_elem else np.zeros(0)
    face_tag = np.concatenate(face_tag) if face_tag else np.zeros(0)
    out = dict(
        xyz=xyz,
        conn=conn.astype(np.int32),
        elem_mat=elem_mat,
        faces=np.array(faces, dtype=np.int32).reshape(-1, 6),
        face_elem=np.array(face_elem, dtype=np.int32),
        face_tag=np.array(face_tag, dtype=np.int32),
        period=np.array([Lx, Ly] if periodic else [0.0, 0.0]),
        nx=nx, ny=ny, nz=nz, Lx=Lx, Ly=Ly, depth=depth, counts=list(counts),
    )
    return out
