"""Tetrahedra for the oracle: tetrahedra with P_r geometry, r = 1 (straight-sided, affine) or r = 2
(curved edges and faces), and a P_p DG basis, p = 1, 2 (paper Sec. 2: simplicial elements,
geometry in P_r and DG in P_s).  ORACLE: test infrastructure only -- imported by tests/, the smoke check and the bench's
CPU legs, never by the product path.

Reference tetrahedron with vertices v0 = (0,0,0), v1 = (1,0,0), v2 = (0,1,0), v3 = (0,0,1),
barycentrics l0 = ((1 - x) - y) - z, l1 = x, l2 = y, l3 = z.  Face f is opposite vertex f, with the
vertex triple FACES[f] ordered so that (B - A) x (C - A) points out of the element; the face's
coordinates (s, t) are the barycentrics of B and C: x = A + s (B - A) + t (C - A).  DG nodes: the
vertices, then (p = 2) the midpoints of the edges EDGES in that order; face nodes: A, B, C, then
(p = 2) the midpoints of AB, BC, CA.  Bases in closed form: p = 1, l_i; p = 2, l_i ((2 l_i) - 1)
at the vertices and (4 l_a) l_b at the edges (the same operation order on the device, so that
face quantities agree bit for bit).  The orientation code k of a shared face: the neighbour's
vertex PERMS[k][j] of its triple is our vertex j, so the neighbour's face barycentrics are ours
permuted.  Readings: on a flat face (r = 1) Omega . n is constant, so every face is whole-inflow
or not, and faces use the collapsed triangle rule with p + 1 points per direction.  r = 2: the
control points are the P_2 nodes (vertices, then the edge midpoints in EDGES order), the face map
x(s, t) = sum_j x_j psi_j(s, t) over the face's six nodes with the P_2 face basis psi, and the
scaled normal x_s x x_t is a quadratic in (s, t) that can change sign on a face: the face is
mapped to the unit square by the collapse s = u, t = v (1 - u) (ds dt = (1 - u) du dv), on which
n(u, v (1 - u)) (1 - u) has degree <= 3 = 2r - 1 in each coordinate, and integrated by the
hexahedron's kink-aligned rule (face_rule_3d, K x K composite pieces split at the roots of
Omega . n, p + r points per piece and axis).  Volume integrals by the collapsed Gauss rule
x = u, y = v (1 - u), z = w (1 - u)(1 - v) with p + 1 + r points per direction (exact for the mass
and stiffness integrands, of degree 2p + 3 and 2p + 1 when r = 2).
"""
import numpy as np

from .basis import gauss_legendre, gll_nodes
from .dg import Discretization, dot_omega, face_rule_3d, pos
from .geometry import det, cofactor

FACES = ((1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1))
EDGES = ((0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3))
PERMS = ((0, 1, 2), (1, 2, 0), (2, 0, 1), (0, 2, 1), (2, 1, 0), (1, 0, 2))
FACE_EDGES = ((0, 1), (1, 2), (2, 0))


def edge_index(a, b):
    return next(k for k, (x, y) in enumerate(EDGES) if {x, y} == {a, b})


def face_nodes(p, f):
    """Volume node indices of the face nodes of face f (A, B, C, then the AB, BC, CA midpoints)."""
    a, b, c = FACES[f]
    out = [a, b, c]
    if p == 2:
        out += [4 + edge_index(a, b), 4 + edge_index(b, c), 4 + edge_index(c, a)]
    return out


def bary(x, y, z):
    return [((1.0 - x) - y) - z, x, y, z]


def basis_values(p, x, y, z):
    """[N] arrays of the DG basis at (x, y, z) (closed form in the barycentrics)."""
    l = bary(x, y, z)
    if p == 1:
        return l
    out = [l[i] * ((2.0 * l[i]) - 1.0) for i in range(4)]
    out += [(4.0 * l[a]) * l[b] for (a, b) in EDGES]
    return out


def basis_grads(p, x, y, z):
    """[N][3] arrays of the reference gradients."""
    l = bary(x, y, z)
    gl = [(-1.0, -1.0, -1.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)]
    one = np.ones_like(np.asarray(x, dtype=np.float64))
    if p == 1:
        return [[gl[i][k] * one for k in range(3)] for i in range(4)]
    out = [[((4.0 * l[i]) - 1.0) * gl[i][k] for k in range(3)] for i in range(4)]
    out += [[4.0 * (l[b] * gl[a][k] + l[a] * gl[b][k]) for k in range(3)] for (a, b) in EDGES]
    return out


def face_basis_values(p, s, t):
    """[Nf] arrays of the face-node basis at face coordinates (s, t)."""
    m = [(1.0 - s) - t, s, t]
    if p == 1:
        return m
    out = [m[i] * ((2.0 * m[i]) - 1.0) for i in range(3)]
    out += [(4.0 * m[a]) * m[b] for (a, b) in FACE_EDGES]
    return out


def face_geom_derivs(s, t):
    """d/ds and d/dt of the six P_2 face basis functions (A, B, C, AB, BC, CA) at (s, t):
    vertex i: ((4 m_i) - 1) dm_i, edge (a, b): 4 ((m_b dm_a) + (m_a dm_b)), m = ((1 - s) - t, s, t)
    with dm/ds = (-1, 1, 0), dm/dt = (-1, 0, 1)."""
    m = [(1.0 - s) - t, s, t]
    out = []
    for dm in ((-1.0, 1.0, 0.0), (-1.0, 0.0, 1.0)):
        d = [((4.0 * m[i]) - 1.0) * dm[i] for i in range(3)]
        d += [4.0 * ((m[b] * dm[a]) + (m[a] * dm[b])) for (a, b) in FACE_EDGES]
        out.append(d)
    return out


def face_normal_tet_p2(ctrl, f, s, t, aligned=False):
    """Scaled outward normal x_s x x_t of face f of P_2 tetrahedra (ctrl [E, 10, 3]) at face
    coordinates (s, t): tangents summed over the face's six nodes in order from 0.0, component
    c = u_a v_b - u_b v_a (a = c + 1, b = c + 2 mod 3), as face_normal_tet for straight faces.
    aligned=False: (s, t) shared by all elements, result [E, *shape, 3]; True: the element axis
    is already first, result [*shape, 3]."""
    ds, dt = face_geom_derivs(s, t)
    cshape = np.broadcast(np.asarray(s), np.asarray(t)).shape
    if aligned:
        oshape, ext = cshape, (slice(None),) + (None,) * (len(cshape) - 1)
    else:
        oshape, ext = (ctrl.shape[0],) + cshape, (slice(None),) + (None,) * len(cshape)
    u = np.zeros(oshape + (3,))
    v = np.zeros(oshape + (3,))
    for j, m in enumerate(face_nodes(2, f)):
        a = np.broadcast_to(ds[j], cshape)
        b = np.broadcast_to(dt[j], cshape)
        for c in range(3):
            u[..., c] = u[..., c] + ctrl[:, m, c][ext] * a
            v[..., c] = v[..., c] + ctrl[:, m, c][ext] * b
    n = np.empty(oshape + (3,))
    for c in range(3):
        a, b = (c + 1) % 3, (c + 2) % 3
        n[..., c] = u[..., a] * v[..., b] - u[..., b] * v[..., a]
    return n


def face_normal_collapsed(ctrl, f, u, v, aligned=False):
    """The P_2 face normal on the collapsed square: n(u, v (1 - u)) (1 - u), so that
    integrals over the face in (u, v) carry the collapse's Jacobian (1 - u) in the normal."""
    om = 1.0 - u
    n = face_normal_tet_p2(ctrl, f, u, v * om, aligned=aligned)
    return n * np.broadcast_to(om, n.shape[:-1])[..., None] if aligned else n * np.broadcast_to(om, n.shape[1:-1])[None, ..., None]


def orient_face(code, s, t):
    """The neighbour's face coordinates of our (s, t): barycentrics permuted by PERMS[code]."""
    m = [(1.0 - s) - t, s, t]
    mp = [None, None, None]
    for j in range(3):
        mp[PERMS[code][j]] = m[j]
    return mp[1], mp[2]


def volume_rule(n):
    """Collapsed Gauss rule on the tetrahedron: points q = i + n (j + n k) at
    (u_i, v_j (1 - u_i), w_k (1 - u_i)(1 - v_j)), weights ((((w_i w_j) w_k)(1 - u_i))(1 - u_i))(1 - v_j)."""
    g, wg = gauss_legendre(n)
    pts, w = [], []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                u, v, ww = g[i], g[j], g[k]
                pts.append((u, v * (1.0 - u), (ww * (1.0 - u)) * (1.0 - v)))
                w.append(((((wg[i] * wg[j]) * wg[k]) * (1.0 - u)) * (1.0 - u)) * (1.0 - v))
    return np.array(pts), np.array(w)


def face_rule_points(n):
    """Collapsed triangle rule: points q = i + n j at (u_i, v_j (1 - u_i)), weights (w_i w_j)(1 - u_i)."""
    g, wg = gauss_legendre(n)
    s, t, w = [], [], []
    for j in range(n):
        for i in range(n):
            s.append(g[i])
            t.append(g[j] * (1.0 - g[i]))
            w.append((wg[i] * wg[j]) * (1.0 - g[i]))
    return np.array(s), np.array(t), np.array(w)


def face_normal_tet(ctrl, f):
    """Outward scaled normal (B - A) x (C - A) of face f: component c = u_a v_b - u_b v_a with
    a = c + 1, b = c + 2 (mod 3).  ctrl [E, 4, 3] -> [E, 3]."""
    A, B, C = (ctrl[:, v, :] for v in FACES[f])
    u, v = B - A, C - A
    return np.stack([u[:, (c + 1) % 3] * v[:, (c + 2) % 3] - u[:, (c + 2) % 3] * v[:, (c + 1) % 3]
                     for c in range(3)], axis=-1)


class TetDiscretization(Discretization):
    """All element- and face-level DG data of one tetrahedron problem (P_1 or P_2 geometry); the
    interface of Discretization on the same DG forms."""

    def __init__(self, prob, face_subdiv=2):
        mesh = prob.mesh
        if mesh.dim != 3 or not getattr(mesh, "simplex", False) or mesh.r not in (1, 2):
            raise ValueError("tetrahedra with P_1 or P_2 geometry only")
        if prob.p not in (1, 2):
            raise ValueError("tetrahedra: DG order 1 or 2")
        self.prob = prob
        self.dim = 3
        self.r = r = mesh.r
        self.p = p = prob.p
        self.N = 4 if p == 1 else 10
        self.Nf = 3 if p == 1 else 6
        self.E = mesh.n_elem
        self.nv = p + 1 + r
        self.nf = p + r
        self.K = face_subdiv if r == 2 else 1
        self.Nv = 4 if r == 1 else 10
        self.gll = gll_nodes(p)
        self.omega = np.asarray(prob.omega, dtype=np.float64)
        self.w = np.asarray(prob.w, dtype=np.float64)
        self.M_dirs = self.omega.shape[0]
        self.n_faces = 4
        self.fnode = [face_nodes(p, f) for f in range(4)]
        self._volume()
        self._faces()

    def vol_points(self):
        return volume_rule(self.nv)

    def _tables(self, pts):
        x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
        B = np.stack(basis_values(self.p, x, y, z), axis=1)                       # [Q, N]
        dB = np.stack([np.stack(g, axis=-1) for g in basis_grads(self.p, x, y, z)], axis=1)   # [Q, N, 3]
        V = np.stack(basis_values(self.r, x, y, z), axis=1)                       # [Q, Nv]
        dV = np.stack([np.stack(g, axis=-1) for g in basis_grads(self.r, x, y, z)], axis=1)
        return B, dB, V, dV

    def _jacobian(self, ctrl, dV):
        J = np.zeros((ctrl.shape[0], dV.shape[0], 3, 3))
        for m in range(self.Nv):
            for i in range(3):
                for j in range(3):
                    J[..., i, j] = J[..., i, j] + ctrl[:, m, i][:, None] * dV[None, :, m, j]
        return J

    def _volume(self):
        pts, wq = self.vol_points()
        ctrl = self.prob.mesh.ctrl
        B, dB, V, dV = self._tables(pts)
        J = self._jacobian(ctrl, dV)
        dJ = det(J)
        if np.any(dJ <= 0.0):
            raise ValueError("invalid mesh: det J <= 0 at a volume quadrature point")
        C = cofactor(J)
        self.detJ = dJ
        self.B, self.dB, self.wq = B, dB, wq
        self.M = np.einsum("q,eq,qm,qn->emn", wq, dJ, B, B)
        grad = np.einsum("eqkj,qmj->eqmk", C, dB)
        self.S = np.einsum("q,eqmk,qn->ekmn", wq, grad, B)
        self.xq = np.einsum("qm,emd->eqd", V, ctrl)
        nodes = [(0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)]
        if self.p == 2:
            nodes += [tuple(0.5 * (np.array(nodes[a]) + np.array(nodes[b]))) for (a, b) in EDGES]
        nodes = np.array(nodes)
        Vn = np.stack(basis_values(self.r, nodes[:, 0], nodes[:, 1], nodes[:, 2]), axis=1)
        self.xnodes = np.einsum("nm,emd->end", Vn, ctrl)

    def mass_exact_order(self, e_idx):
        pts, wq = self.vol_points()
        B, _dB, _V, dV = self._tables(pts)
        dJ = det(self._jacobian(self.prob.mesh.ctrl[e_idx], dV))
        out = np.zeros((len(e_idx), self.N, self.N))
        for m in range(self.N):
            for n in range(self.N):
                acc = np.zeros(len(e_idx))
                for q in range(len(wq)):
                    acc = acc + ((wq[q] * dJ[:, q]) * B[q, m]) * B[q, n]
                out[:, m, n] = acc
        return out

    def _face_rule(self, ctrl, f, om):
        """(s0, s1, w, g), each [F, D, P] with (s0, s1) the face coordinates (s, t).  r = 1: the
        collapsed triangle rule on face f and g = Omega_d . n (the scaled normal is constant on a
        flat face).  r = 2: the kink-aligned rule of face_rule_3d on the collapsed square with
        the normal n(u, v (1 - u)) (1 - u); its points are returned as s = u, t = v (1 - u)."""
        if self.r == 2:
            def normal(c, u, v, aligned=False):
                return face_normal_collapsed(c, f, u, v, aligned=aligned)
            u, v, w, g = face_rule_3d(ctrl, 2, f, om, self.nf, self.K, normal=normal)
            return u, v * (1.0 - u), w, g
        s, t, w = face_rule_points(self.nf)
        nv = face_normal_tet(ctrl, f)                                   # [F, 3]
        F, D, P = ctrl.shape[0], om.shape[0], len(w)
        omk = [om[:, k][None, :, None] for k in range(3)]
        g = dot_omega(omk, nv[:, None, None, :])                        # [F, D, 1]
        g = np.broadcast_to(g, (F, D, P)).copy()
        s0 = np.broadcast_to(s, (F, D, P)).copy()
        s1 = np.broadcast_to(t, (F, D, P)).copy()
        ww = np.broadcast_to(w, (F, D, P)).copy()
        return s0, s1, ww, g

    def _face_basis(self, s0, s1):
        return face_basis_values(self.p, s0, s1)

    def _orient(self, code, s0, s1):
        return orient_face(code, s0, s1)
