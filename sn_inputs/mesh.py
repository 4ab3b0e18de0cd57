"""Structured curved-mesh generators with explicit, general connectivity.

The generators only place control points and build topology: a Cartesian grid of
Q_r elements whose geometry nodes are displaced by a smooth field.  Connectivity
(neighbour, neighbour face, orientation) is derived from global node ids, so an
element's local numbering may be any rotation of the reference element.
"""
from dataclasses import dataclass, field
import itertools
import numpy as np


@dataclass
class Mesh:
    dim: int
    r: int                      # geometry order (Q_r)
    ctrl: np.ndarray            # [n_elem][(r+1)^dim][dim] float64 control points
    face_nbr: np.ndarray        # [n_elem][2 dim] int64, -1 = domain boundary
    nbr_face: np.ndarray        # [n_elem][2 dim] int32
    orient: np.ndarray          # [n_elem][2 dim] int32 (see package docstring)
    nodes: np.ndarray = field(repr=False, default=None)       # [n_nodes][dim] global node positions
    elem_nodes: np.ndarray = field(repr=False, default=None)  # [n_elem][(r+1)^dim] global node ids
    shape: tuple = ()           # logical grid size (nx, ny[, nz])
    simplex: bool = False       # triangles with P_r geometry (see triangle_mesh) instead of Q_r

    @property
    def n_elem(self):
        return self.ctrl.shape[0]


def _local_index(idx, r):
    m = 0
    for k in reversed(range(len(idx))):
        m = m * (r + 1) + idx[k]
    return m


def structured_mesh(shape, r, disp=None, domain=None, fast_connectivity=True):
    """Cartesian grid of Q_r elements on [0,1]^dim (or `domain` = [(lo,hi),...]).

    shape : (nx, ny) or (nx, ny, nz) elements.  Element index e = i + nx j (+ nx ny k).
    disp  : callable X[n,dim] -> displacement[n,dim] applied to every geometry node, or None.
    fast_connectivity : use the grid's own neighbour structure (all orientation codes 0)
                        instead of matching faces by global node ids.
    """
    dim = len(shape)
    if domain is None:
        domain = [(0.0, 1.0)] * dim
    counts = [s * r + 1 for s in shape]
    axes = [np.array([lo + (hi - lo) * g / (s * r) for g in range(c)], dtype=np.float64)
            for (lo, hi), s, c in zip(domain, shape, counts)]
    grids = np.meshgrid(*axes, indexing="ij")
    # global node id: g0 + c0 g1 + c0 c1 g2
    X = np.stack([g.transpose(tuple(reversed(range(dim)))).reshape(-1) for g in grids], axis=1)
    if disp is not None:
        X = X + disp(X.copy())
    n_elem = int(np.prod(shape))
    strides = [1]
    for c in counts[:-1]:
        strides.append(strides[-1] * c)
    # element grid indices (i, j[, k]) in element order, local node offsets (a, b[, c]) in local order
    eg = np.stack(np.meshgrid(*[np.arange(s) for s in reversed(shape)], indexing="ij"), -1)
    eg = eg.reshape(-1, dim)[:, ::-1]
    lg = np.stack(np.meshgrid(*[np.arange(r + 1)] * dim, indexing="ij"), -1).reshape(-1, dim)[:, ::-1]
    gidx = eg[:, None, :] * r + lg[None, :, :]
    elem_nodes = (gidx * np.array(strides)[None, None, :]).sum(-1).astype(np.int64)
    if fast_connectivity:
        ctrl = np.ascontiguousarray(X[elem_nodes])
        face_nbr, nbr_face, orient = _structured_connectivity(shape)
        return Mesh(dim=dim, r=r, ctrl=ctrl, face_nbr=face_nbr, nbr_face=nbr_face, orient=orient,
                    nodes=X, elem_nodes=elem_nodes, shape=tuple(shape))
    return _finish(dim, r, X, elem_nodes, tuple(shape))


def _structured_connectivity(shape):
    dim = len(shape)
    n_elem = int(np.prod(shape))
    e = np.arange(n_elem, dtype=np.int64)
    idx = []
    rem = e.copy()
    for s in shape:
        idx.append(rem % s)
        rem = rem // s
    stride = 1
    face_nbr = -np.ones((n_elem, 2 * dim), dtype=np.int64)
    nbr_face = -np.ones((n_elem, 2 * dim), dtype=np.int32)
    for a, s in enumerate(shape):
        lo = idx[a] > 0
        hi = idx[a] < s - 1
        face_nbr[lo, 2 * a] = e[lo] - stride
        nbr_face[lo, 2 * a] = 2 * a + 1
        face_nbr[hi, 2 * a + 1] = e[hi] + stride
        nbr_face[hi, 2 * a + 1] = 2 * a
        stride *= s
    return face_nbr, nbr_face, np.zeros((n_elem, 2 * dim), dtype=np.int32)


def _finish(dim, r, X, elem_nodes, shape):
    ctrl = np.ascontiguousarray(X[elem_nodes])
    face_nbr, nbr_face, orient = connectivity_from_nodes(dim, r, elem_nodes)
    return Mesh(dim=dim, r=r, ctrl=ctrl, face_nbr=face_nbr, nbr_face=nbr_face, orient=orient,
                nodes=X, elem_nodes=elem_nodes, shape=shape)


def _face_node_grid(dim, r, f):
    """Global-local node indices of face f as an array indexed [s1][s0] (2D faces: [s0])."""
    axis, side = f // 2, f % 2
    others = [a for a in range(dim) if a != axis]
    if dim == 2:
        out = np.zeros(r + 1, dtype=np.int64)
        for i in range(r + 1):
            loc = [0, 0]
            loc[axis] = side * r
            loc[others[0]] = i
            out[i] = _local_index(loc, r)
        return out
    out = np.zeros((r + 1, r + 1), dtype=np.int64)
    for j in range(r + 1):
        for i in range(r + 1):
            loc = [0, 0, 0]
            loc[axis] = side * r
            loc[others[0]] = i
            loc[others[1]] = j
            out[j, i] = _local_index(loc, r)
    return out


def orient_apply(code, i, j, n):
    """Map face-node grid indices (i along s0, j along s1) of one side to the other side's.

    n = number of nodes per face axis minus one (equispaced/symmetric node sets).
    """
    u0, u1 = (j, i) if code & 4 else (i, j)
    t0 = n - u0 if code & 1 else u0
    t1 = n - u1 if code & 2 else u1
    return t0, t1


def connectivity_from_nodes(dim, r, elem_nodes):
    n_elem = elem_nodes.shape[0]
    nf = 2 * dim
    face_nbr = -np.ones((n_elem, nf), dtype=np.int64)
    nbr_face = -np.ones((n_elem, nf), dtype=np.int32)
    orient = np.zeros((n_elem, nf), dtype=np.int32)
    grids = [_face_node_grid(dim, r, f) for f in range(nf)]
    table = {}
    for e in range(n_elem):
        for f in range(nf):
            ids = elem_nodes[e][grids[f]]
            key = frozenset(ids.reshape(-1).tolist())
            table.setdefault(key, []).append((e, f))
    codes = [0, 1] if dim == 2 else list(range(8))
    for key, lst in table.items():
        if len(lst) == 1:
            continue
        if len(lst) != 2:
            raise ValueError("non-conforming mesh: a face is shared by more than two elements")
        (e, f), (e2, f2) = lst
        for (a, fa, b, fb) in ((e, f, e2, f2), (e2, f2, e, f)):
            ga = elem_nodes[a][grids[fa]]
            gb = elem_nodes[b][grids[fb]]
            found = None
            for c in codes:
                ok = True
                if dim == 2:
                    for i in range(r + 1):
                        t0, _ = orient_apply(c, i, 0, r)
                        if ga[i] != gb[t0]:
                            ok = False
                            break
                else:
                    for j in range(r + 1):
                        for i in range(r + 1):
                            t0, t1 = orient_apply(c, i, j, r)
                            if ga[j, i] != gb[t1, t0]:
                                ok = False
                                break
                        if not ok:
                            break
                if ok:
                    found = c
                    break
            if found is None:
                raise ValueError("could not match face orientation")
            face_nbr[a, fa] = b
            nbr_face[a, fa] = fb
            orient[a, fa] = found
    return face_nbr, nbr_face, orient


def _rotations(dim):
    """Orientation-preserving symmetries of [0,1]^dim as (perm, flips):
    new_xi[k] = 1 - old_xi[perm[k]] if flips[k] else old_xi[perm[k]]."""
    out = []
    for perm in itertools.permutations(range(dim)):
        psign = np.linalg.det(np.eye(dim)[list(perm)])
        for flips in itertools.product((0, 1), repeat=dim):
            s = psign * np.prod([-1 if fl else 1 for fl in flips])
            if s > 0:
                out.append((perm, flips))
    return out


def reorient_elements(mesh, seed):
    """Renumber every element's local nodes by a random rotation of the reference element.

    The physical mesh is unchanged; local face numbering and neighbour orientation
    codes change, which exercises the general face-matching logic of any consumer.
    """
    rng = np.random.default_rng(seed)
    rots = _rotations(mesh.dim)
    dim, r = mesh.dim, mesh.r
    new_nodes = np.empty_like(mesh.elem_nodes)
    for e in range(mesh.n_elem):
        perm, flips = rots[rng.integers(len(rots))]
        for loc in itertools.product(*[range(r + 1)] * dim):
            loc = tuple(reversed(loc))              # new local index tuple
            old = [0] * dim
            # new_xi[k] = f(old_xi[perm[k]])  =>  old_xi[perm[k]] = f^-1(new_xi[k])
            for k in range(dim):
                old[perm[k]] = r - loc[k] if flips[k] else loc[k]
            new_nodes[e, _local_index(loc, r)] = mesh.elem_nodes[e, _local_index(old, r)]
    return _finish(dim, r, mesh.nodes, new_nodes, mesh.shape)


# ---------------------------------------------------------------- displacement fields

def disp_sine_2d(amp=0.05):
    """x' = x + amp sin(2 pi x) sin(2 pi y), y' = y + the same (zero on the unit-square boundary)."""
    def f(X):
        d = amp * np.sin(2 * np.pi * X[:, 0]) * np.sin(2 * np.pi * X[:, 1])
        return np.stack([d, d], axis=1)
    return f


def disp_random_smooth(h, seed, amp_frac=0.1, n_modes=8, kmax=None):
    """Seeded smooth random displacement of amplitude <= amp_frac*h, zero on the boundary.

    Each component: A * sin(pi x) sin(pi y) * sum_j a_j sin(2 pi k_j . x + phi_j) / sum_j |a_j|
    with A = amp_frac*h, integer wavevectors k_j in [1, kmax]^dim (kmax = max(1, 1/(4h))),
    a_j ~ U[-1,1], phi_j ~ U[0, 2 pi), drawn from numpy PCG64(seed).
    """
    rng = np.random.default_rng(seed)
    if kmax is None:
        kmax = max(1, int(round(1.0 / (4.0 * h))))
    params = []
    for _comp in range(2):
        k = rng.integers(1, kmax + 1, size=(n_modes, 2)).astype(np.float64)
        a = rng.uniform(-1.0, 1.0, size=n_modes)
        ph = rng.uniform(0.0, 2 * np.pi, size=n_modes)
        params.append((k, a, ph))
    A = amp_frac * h

    def f(X):
        env = np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])
        out = np.zeros_like(X)
        for c, (k, a, ph) in enumerate(params):
            s = np.zeros(X.shape[0])
            for j in range(len(a)):
                s += a[j] * np.sin(2 * np.pi * (k[j, 0] * X[:, 0] + k[j, 1] * X[:, 1]) + ph[j])
            out[:, c] = A * env * s / np.abs(a).sum()
        return out
    return f


def disp_random_smooth_3d(h, seed, amp_frac=0.1, n_modes=8, kmax=None):
    """3D version of disp_random_smooth (envelope sin(pi x) sin(pi y) sin(pi z), 3 components)."""
    rng = np.random.default_rng(seed)
    if kmax is None:
        kmax = max(1, int(round(1.0 / (4.0 * h))))
    params = []
    for _comp in range(3):
        k = rng.integers(1, kmax + 1, size=(n_modes, 3)).astype(np.float64)
        a = rng.uniform(-1.0, 1.0, size=n_modes)
        ph = rng.uniform(0.0, 2 * np.pi, size=n_modes)
        params.append((k, a, ph))
    A = amp_frac * h

    def f(X):
        env = np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])
        out = np.zeros_like(X)
        for c, (k, a, ph) in enumerate(params):
            s = np.zeros(X.shape[0])
            for j in range(len(a)):
                s += a[j] * np.sin(2 * np.pi * (X @ k[j]) + ph[j])
            out[:, c] = A * env * s / np.abs(a).sum()
        return out
    return f


def disp_twist(total_angle=np.pi / 3):
    """Rotate (x, y) about (1/2, 1/2) by theta = total_angle * z (a z-dependent twist)."""
    def f(X):
        th = total_angle * X[:, 2]
        x, y = X[:, 0] - 0.5, X[:, 1] - 0.5
        xn = np.cos(th) * x - np.sin(th) * y
        yn = np.sin(th) * x + np.cos(th) * y
        out = np.zeros_like(X)
        out[:, 0] = xn - x
        out[:, 1] = yn - y
        return out
    return f


def disp_bubble_3d(amp):
    """amp sin(pi x) sin(pi y) sin(pi z) (cos(pi y), cos(pi z), cos(pi x)): a smooth displacement that
    vanishes on the unit cube's boundary (interior elements curve, the domain stays the cube)."""
    def f(X):
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        b = amp * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        return np.stack([b * np.cos(np.pi * y), b * np.cos(np.pi * z), b * np.cos(np.pi * x)], axis=1)
    return f


# ---------------------------------------------------------------- curved-boundary domain, straightening

def annulus_mesh(n_rho, n_theta, r, rho=(0.5, 1.0), theta=(0.0, 0.5 * np.pi)):
    """Sector of an annulus, rho in [rho0, rho1], theta in [theta0, theta1], as an n_rho x n_theta
    grid of Q_r elements (element index i + n_rho j, i along rho).  The control points are the
    exact polar images of the equispaced reference nodes, so inner and outer boundaries are
    curved arcs represented to order r."""
    def to_polar(X):
        rr = rho[0] + (rho[1] - rho[0]) * X[:, 0]
        th = theta[0] + (theta[1] - theta[0]) * X[:, 1]
        return np.stack([rr * np.cos(th) - X[:, 0], rr * np.sin(th) - X[:, 1]], axis=1)
    return structured_mesh((n_rho, n_theta), r, to_polar)


def _lagrange_1d(nodes, j, x):
    v = 1.0
    for k, nk in enumerate(nodes):
        if k != j:
            v = v * (x - nk) / (nodes[j] - nk)
    return v


def straighten(mesh, n_ref):
    """The straightened low-order mesh of a curved Q_r mesh: every element divided n_ref times
    along each reference axis, the sub-cell vertices placed at their images under the element's
    map, and those vertices taken as the nodes of a mesh of straight-sided Q_1 elements.  Shared
    vertices of neighbouring elements are merged by position (rounded to 1e-10)."""
    dim, r = mesh.dim, mesh.r
    geo = [a / r for a in range(r + 1)]
    t = [a / n_ref for a in range(n_ref + 1)]
    # map weights of the sub-lattice points: [(n_ref+1)^dim][(r+1)^dim]
    lat = list(itertools.product(*[range(n_ref + 1)] * dim))
    lat = [tuple(reversed(l)) for l in lat]          # x fastest
    W = np.zeros((len(lat), (r + 1) ** dim))
    for a, l in enumerate(lat):
        for m in range((r + 1) ** dim):
            v = 1.0
            for k in range(dim):
                v *= _lagrange_1d(geo, (m // (r + 1) ** k) % (r + 1), t[l[k]])
            W[a, m] = v
    P = np.einsum("am,emd->ead", W, mesh.ctrl)       # [E][(n_ref+1)^dim][dim]
    key = np.round(P.reshape(-1, dim) * 1e10).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    nodes = P.reshape(-1, dim)[first]
    gid = inv.reshape(mesh.n_elem, len(lat))
    lidx = {l: a for a, l in enumerate(lat)}
    elem_nodes = []
    for e in range(mesh.n_elem):
        for cell in itertools.product(*[range(n_ref)] * dim):
            cell = tuple(reversed(cell))
            loc = []
            for corner in itertools.product(*[range(2)] * dim):
                corner = tuple(reversed(corner))
                loc.append(gid[e, lidx[tuple(c + o for c, o in zip(cell, corner))]])
            elem_nodes.append(loc)
    elem_nodes = np.array(elem_nodes, dtype=np.int64)
    return _finish(dim, 1, nodes, elem_nodes, ())


# ---------------------------------------------------------------- triangles (P_r geometry)
#
# Reference triangle {(xi, eta): xi, eta >= 0, xi + eta <= 1}, vertices v0 = (0,0), v1 = (1,0),
# v2 = (0,1); faces (edges) counterclockwise f0: v0 -> v1, f1: v1 -> v2, f2: v2 -> v0, each with
# its own coordinate s in [0, 1] from the first vertex to the second.  Node numbering of an
# order-k node set: v0, v1, v2, the k - 1 interior nodes of f0, of f1, of f2 (each in increasing
# s), then the interior nodes (k = 3: the centroid).  Geometry (P_r) nodes sit at s = a/r on the
# edges.  orient[e][f] = 1 when the neighbour runs the shared edge in the opposite direction
# (always, for counterclockwise elements), 0 otherwise.

TRI_VERTS = ((0.0, 0.0), (1.0, 0.0), (0.0, 1.0))
TRI_EDGES = ((0, 1), (1, 2), (2, 0))


def tri_node_coords(k, edge_pos):
    """Reference coordinates [(k+1)(k+2)/2][2] of the order-k node set whose edge nodes sit at
    the 1D positions edge_pos[1..k-1] (k <= 3)."""
    pts = [TRI_VERTS[0], TRI_VERTS[1], TRI_VERTS[2]]
    for a, b in TRI_EDGES:
        A, B = TRI_VERTS[a], TRI_VERTS[b]
        for j in range(1, k):
            s = edge_pos[j]
            pts.append((A[0] + s * (B[0] - A[0]), A[1] + s * (B[1] - A[1])))
    if k == 3:
        pts.append((1.0 / 3.0, 1.0 / 3.0))
    elif k > 3:
        raise ValueError("orders up to 3")
    return np.array(pts)


def tri_edge_nodes(k, f):
    """Local node indices of face f of an order-k node set, in increasing edge coordinate."""
    a, b = TRI_EDGES[f]
    return [a] + [3 + f * (k - 1) + j for j in range(k - 1)] + [b]


def triangle_mesh(shape, r, disp=None):
    """Each cell (i, j) of an nx x ny grid on [0,1]^2 cut by its diagonal (i, j) - (i+1, j+1) into
    the counterclockwise triangles (i,j), (i+1,j), (i+1,j+1) (element 2 (i + nx j)) and
    (i,j), (i+1,j+1), (i,j+1) (element 2 (i + nx j) + 1), with P_r geometry: the control points
    are the lattice positions of the reference nodes, displaced by disp (as structured_mesh)."""
    nx, ny = shape
    ref = tri_node_coords(r, [a / r for a in range(r + 1)])      # geometry nodes
    cx, cy = nx * r + 1, ny * r + 1                               # global lattice of spacing h / r
    elem_nodes, pos = [], []
    for j in range(ny):
        for i in range(nx):
            for tri in ((0, 1, 2), (0, 2, 3)):
                corner = [(i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)]
                P0, P1, P2 = (np.array(corner[t], dtype=float) for t in tri)
                ids = []
                for (xi, eta) in ref:
                    g = P0 + xi * (P1 - P0) + eta * (P2 - P0)
                    gi, gj = int(round(g[0] * r)), int(round(g[1] * r))
                    ids.append(gi + cx * gj)
                elem_nodes.append(ids)
    elem_nodes = np.array(elem_nodes, dtype=np.int64)
    gx, gy = np.meshgrid(np.arange(cx) / (nx * r), np.arange(cy) / (ny * r), indexing="xy")
    X = np.stack([gx.reshape(-1), gy.reshape(-1)], axis=1)
    if disp is not None:
        X = X + disp(X.copy())
    return _finish_tri(r, X, elem_nodes, tuple(shape))


def _finish_tri(r, X, elem_nodes, shape):
    n_elem = elem_nodes.shape[0]
    face_nbr = -np.ones((n_elem, 3), dtype=np.int64)
    nbr_face = -np.ones((n_elem, 3), dtype=np.int32)
    orient = np.zeros((n_elem, 3), dtype=np.int32)
    table = {}
    for e in range(n_elem):
        for f in range(3):
            ids = elem_nodes[e][tri_edge_nodes(r, f)]
            table.setdefault(frozenset(ids.tolist()), []).append((e, f))
    for lst in table.values():
        if len(lst) == 1:
            continue
        if len(lst) != 2:
            raise ValueError("non-conforming mesh: an edge is shared by more than two elements")
        (e, f), (e2, f2) = lst
        a = elem_nodes[e][tri_edge_nodes(r, f)]
        b = elem_nodes[e2][tri_edge_nodes(r, f2)]
        code = 0 if np.array_equal(a, b) else (1 if np.array_equal(a, b[::-1]) else -1)
        if code < 0:
            raise ValueError("could not match edge orientation")
        face_nbr[e, f], nbr_face[e, f], orient[e, f] = e2, f2, code
        face_nbr[e2, f2], nbr_face[e2, f2], orient[e2, f2] = e, f, code
    ctrl = np.ascontiguousarray(X[elem_nodes])
    return Mesh(dim=2, r=r, ctrl=ctrl, face_nbr=face_nbr, nbr_face=nbr_face, orient=orient,
                nodes=X, elem_nodes=elem_nodes, shape=shape, simplex=True)


def rotate_triangles(mesh, seed):
    """Renumber every triangle's local nodes by a random rotation of the reference triangle
    (v0 v1 v2 -> v1 v2 v0 or v2 v0 v1); the physical mesh is unchanged, local faces and the
    neighbours' face indices change."""
    rng = np.random.default_rng(seed)
    r = mesh.r
    ne = mesh.n_elem
    new_nodes = mesh.elem_nodes.copy()
    nv = (r + 1) * (r + 2) // 2
    for e in range(ne):
        k = int(rng.integers(3))
        if k == 0:
            continue
        perm = list(range(nv))
        # vertex v_i -> v_{(i+k) % 3}; edge f interiors -> edge (f+k) % 3; centroid fixed
        for i in range(3):
            perm[i] = (i + k) % 3
        for f in range(3):
            for j in range(r - 1):
                perm[3 + f * (r - 1) + j] = 3 + ((f + k) % 3) * (r - 1) + j
        new_nodes[e] = mesh.elem_nodes[e][perm]
    return _finish_tri(r, mesh.nodes, new_nodes, mesh.shape)


# ---------------------------------------------------------------- tetrahedra (affine, P_1 geometry)
#
# Reference tetrahedron with vertices v0 = (0,0,0), v1 = (1,0,0), v2 = (0,1,0), v3 = (0,0,1).
# Face f is opposite vertex f, with the vertex triple TET_FACES[f] ordered so that
# (B - A) x (C - A) points out of the element.  A face's own coordinates are the barycentric
# (s, t) of the triple: x = A + s (B - A) + t (C - A).  orient[e][f] = index k of the permutation
# TRI_PERMS[k] that takes this face's triple to the neighbour's: the neighbour's vertex
# TRI_PERMS[k][j] of its triple is our vertex j.

TET_FACES = ((1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1))
TRI_PERMS = ((0, 1, 2), (1, 2, 0), (2, 0, 1), (0, 2, 1), (2, 1, 0), (1, 0, 2))


def tet_mesh(n, disp=None, r=1):
    """The unit cube as n^3 cubes, each cut into the six tetrahedra of the Kuhn triangulation
    (vertex paths from the cube's corner (0,0,0) to (1,1,1) along the axes in every order;
    conforming across cubes), vertices ordered for positive volume.  r = 1: P_1 geometry (the
    control points are the vertices), optionally displaced by disp (an affine disp keeps it
    exact).  r = 2: P_2 geometry, control points the vertices then the edge midpoints in
    TET_EDGES order, every node (vertices and the straight edges' midpoints) moved by disp, so
    that the edges and faces curve; an edge's midpoint node is shared by all its tetrahedra."""
    import itertools as it
    if r not in (1, 2):
        raise ValueError("tetrahedra: geometry order 1 or 2")
    c = n + 1
    gid = lambda i, j, k: i + c * (j + c * k)
    elems = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                for perm in it.permutations(range(3)):
                    p = [0, 0, 0]
                    verts = [gid(i, j, k)]
                    for ax in perm:
                        p[ax] += 1
                        verts.append(gid(i + p[0], j + p[1], k + p[2]))
                    elems.append(verts)
    g = np.arange(c) / n
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    nodes0 = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], axis=1)
    elems = np.array(elems, dtype=np.int64)
    edge_ids = {}
    if r == 2:
        for e in range(elems.shape[0]):
            for a, b in TET_EDGES:
                edge_ids.setdefault(frozenset((int(elems[e, a]), int(elems[e, b]))), None)
        keys = sorted(edge_ids, key=lambda k: tuple(sorted(k)))
        for m, key in enumerate(keys):
            edge_ids[key] = nodes0.shape[0] + m
        mids = np.array([0.5 * (nodes0[min(k)] + nodes0[max(k)]) for k in keys]).reshape(-1, 3)
        nodes0 = np.concatenate([nodes0, mids], axis=0)
    nodes = nodes0 + disp(nodes0.copy()) if disp is not None else nodes0
    # positive volume (of the vertex tetrahedron): swap the last two vertices where it is negative
    P = nodes[elems]
    vol = np.einsum("ei,ei->e", np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), P[:, 3] - P[:, 0])
    neg = vol < 0
    elems[neg, 2], elems[neg, 3] = elems[neg, 3].copy(), elems[neg, 2].copy()
    if r == 2:
        en = [[edge_ids[frozenset((int(v[a]), int(v[b])))] for a, b in TET_EDGES] for v in elems]
        elems = np.concatenate([elems, np.array(en, dtype=np.int64).reshape(-1, 6)], axis=1)
    return _finish_tet(nodes, elems, (n, n, n))


def _finish_tet(nodes, elems, shape):
    ne = elems.shape[0]
    face_nbr = -np.ones((ne, 4), dtype=np.int64)
    nbr_face = -np.ones((ne, 4), dtype=np.int32)
    orient = np.zeros((ne, 4), dtype=np.int32)
    table = {}
    for e in range(ne):
        for f in range(4):
            tri = tuple(int(elems[e, v]) for v in TET_FACES[f])
            table.setdefault(frozenset(tri), []).append((e, f, tri))
    for lst in table.values():
        if len(lst) == 1:
            continue
        if len(lst) != 2:
            raise ValueError("non-conforming mesh: a face is shared by more than two elements")
        for (a, fa, ta), (b, fb, tb) in ((lst[0], lst[1]), (lst[1], lst[0])):
            code = next(k for k, pm in enumerate(TRI_PERMS) if all(tb[pm[j]] == ta[j] for j in range(3)))
            face_nbr[a, fa], nbr_face[a, fa], orient[a, fa] = b, fb, code
    ctrl = np.ascontiguousarray(nodes[elems])
    return Mesh(dim=3, r=1 if elems.shape[1] == 4 else 2, ctrl=ctrl, face_nbr=face_nbr, nbr_face=nbr_face,
                orient=orient, nodes=nodes, elem_nodes=elems, shape=shape, simplex=True)


TET_EDGES = ((0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3))
_EVEN_PERMS = tuple(p for p in itertools.permutations(range(4))
                    if sum(1 for i in range(4) for j in range(i + 1, 4) if p[i] > p[j]) % 2 == 0)


def rotate_tets(mesh, seed):
    """Renumber every tetrahedron's vertices by a random even permutation (orientation kept);
    the physical mesh is unchanged, local faces and orientation codes change (and, for P_2
    geometry, the edge nodes follow their edges)."""
    rng = np.random.default_rng(seed)
    en = mesh.elem_nodes.copy()
    for e in range(mesh.n_elem):
        p = list(_EVEN_PERMS[rng.integers(len(_EVEN_PERMS))])
        old = mesh.elem_nodes[e]
        en[e, :4] = old[p]
        if en.shape[1] == 10:
            edge = {frozenset((int(old[a]), int(old[b]))): int(old[4 + k]) for k, (a, b) in enumerate(TET_EDGES)}
            en[e, 4:] = [edge[frozenset((int(en[e, a]), int(en[e, b])))] for a, b in TET_EDGES]
    return _finish_tet(mesh.nodes, en, mesh.shape)
