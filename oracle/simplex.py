"""Simplicial elements for the oracle: triangles with P_r geometry and a P_p DG basis (paper
Sec. 2: for simplices the geometry basis spans P_r and the DG basis P_s, polynomials of total
degree r and s).  ORACLE: test infrastructure only -- imported by tests/, the smoke check and
the bench's CPU legs, never by the product path.

Reference triangle {(xi, eta): xi, eta >= 0, xi + eta <= 1}, vertices v0 = (0,0), v1 = (1,0),
v2 = (0,1); faces counterclockwise f0: v0 -> v1, f1: v1 -> v2, f2: v2 -> v0, each with its own
coordinate s in [0, 1] from its first to its second vertex.  An order-k node set is numbered
v0, v1, v2, the k - 1 interior nodes of f0, f1, f2 (increasing s), then the interior nodes (k = 3:
the centroid).  Geometry nodes sit at s = a/r on the edges (the meshes' control points); DG nodes
at the Gauss-Lobatto-Legendre positions of order p, so that the DG basis restricted to a face is
the 1D Lagrange basis on those positions (the same face basis as the tensor elements').
Readings (the paper gives no formulas for simplices): nodal Lagrange bases on these node sets;
volume integrals by the collapsed (Duffy) Gauss rule xi = u, eta = v (1 - u), weight
w_i w_j (1 - u_i), n_v = p + r points per direction (exact for the straight-sided mass and
stiffness products); faces as for the tensor elements: n_f = p + r Gauss points per piece, pieces
split at the sign changes of Omega . n(s), whose scaled normal along a face is the rotated tangent
of the face's P_r curve, n(s) = (T_y, -T_x) with T(s) = sum_j x_j l_j'(s) over the face's r + 1
control points in increasing s (outward for counterclockwise elements).
"""
import numpy as np

from .basis import gauss_legendre, gll_nodes, equispaced_nodes, lagrange_deriv
from .dg import Discretization, face_rule
from .geometry import det, cofactor

VERTS = ((0.0, 0.0), (1.0, 0.0), (0.0, 1.0))
EDGES = ((0, 1), (1, 2), (2, 0))


def node_coords(k, edge_pos):
    """[(k+1)(k+2)/2, 2] reference coordinates of the order-k node set with edge nodes at the
    1D positions edge_pos[1..k-1]."""
    pts = list(VERTS)
    for a, b in EDGES:
        A, B = np.array(VERTS[a]), np.array(VERTS[b])
        for j in range(1, k):
            pts.append(tuple(A + edge_pos[j] * (B - A)))
    if k == 3:
        pts.append((1.0 / 3.0, 1.0 / 3.0))
    return np.array(pts, dtype=np.float64)


def edge_nodes(k, f):
    """Local indices of the nodes of face f of an order-k node set, in increasing s."""
    a, b = EDGES[f]
    return [a] + [3 + f * (k - 1) + j for j in range(k - 1)] + [b]


def monomials(k):
    return [(a, d - a) for d in range(k + 1) for a in range(d, -1, -1)]


class LagrangeTri:
    """Nodal Lagrange basis of total degree k on the triangle node set `nodes`: the monomial
    coefficients are the columns of the inverse Vandermonde matrix."""

    def __init__(self, k, nodes):
        self.k = k
        self.mono = monomials(k)
        V = np.array([[x ** a * y ** b for (a, b) in self.mono] for (x, y) in nodes])
        self.C = np.linalg.inv(V)

    def values(self, pts):
        P = np.array([[x ** a * y ** b for (a, b) in self.mono] for (x, y) in pts])
        return P @ self.C                                               # [P, n]

    def grads(self, pts):
        dx = np.array([[a * x ** max(a - 1, 0) * y ** b if a > 0 else 0.0 for (a, b) in self.mono]
                       for (x, y) in pts])
        dy = np.array([[b * x ** a * y ** max(b - 1, 0) if b > 0 else 0.0 for (a, b) in self.mono]
                       for (x, y) in pts])
        return np.stack([dx @ self.C, dy @ self.C], axis=-1)            # [P, n, 2]


def volume_rule(n):
    """Collapsed Gauss rule on the triangle: points q = i + n j at (u_i, v_j (1 - u_i)), weights
    (w_i w_j) (1 - u_i), with (u, w) the n-point Gauss-Legendre rule on [0, 1]."""
    t, wt = gauss_legendre(n)
    pts, w = [], []
    for j in range(n):
        for i in range(n):
            pts.append((t[i], t[j] * (1.0 - t[i])))
            w.append((wt[i] * wt[j]) * (1.0 - t[i]))
    return np.array(pts), np.array(w)


def face_normal_tri(ctrl, r, f, s, aligned=False):
    """Scaled outward normal n(s) = (T_y, -T_x) of face f, T(s) = sum_j x_j l_j'(s) in
    increasing j from 0.0 over the face's control points (equispaced 1D nodes).
    aligned=False: s shared by all elements -> [E, *shape(s), 2]; aligned=True: s carries the
    element axis first -> [*shape(s), 2]."""
    gn = equispaced_nodes(r)
    ids = edge_nodes(r, f)
    s = np.asarray(s, dtype=np.float64)
    if aligned:
        ext = (slice(None),) + (None,) * (s.ndim - 1)
        T = [np.zeros(s.shape), np.zeros(s.shape)]
        for j, m in enumerate(ids):
            dv = lagrange_deriv(gn, j, s)
            for c in range(2):
                T[c] = T[c] + ctrl[:, m, c][ext] * dv
    else:
        E = ctrl.shape[0]
        ext = (slice(None),) + (None,) * s.ndim
        T = [np.zeros((E,) + s.shape), np.zeros((E,) + s.shape)]
        for j, m in enumerate(ids):
            dv = np.broadcast_to(lagrange_deriv(gn, j, s), s.shape)
            for c in range(2):
                T[c] = T[c] + ctrl[:, m, c][ext] * dv
    return np.stack([T[1], -T[0]], axis=-1)


class SimplexDiscretization(Discretization):
    """All element- and face-level DG data of one triangle-mesh problem; the interface of
    Discretization (face blocks, local systems, mass matrices) on the same DG forms."""

    def __init__(self, prob, face_subdiv=2):
        mesh = prob.mesh
        if mesh.dim != 2 or not getattr(mesh, "simplex", False):
            raise ValueError("triangle meshes only")
        self.prob = prob
        self.dim = 2
        self.r = r = mesh.r
        self.p = p = prob.p
        self.N = (p + 1) * (p + 2) // 2
        self.Nf = p + 1
        self.E = mesh.n_elem
        self.nv = p + r
        self.nf = p + r
        self.K = 1
        self.gll = gll_nodes(p)
        self.omega = np.asarray(prob.omega, dtype=np.float64)[:, :2]
        self.w = np.asarray(prob.w, dtype=np.float64)
        self.M_dirs = self.omega.shape[0]
        self.n_faces = 3
        self.fnode = [edge_nodes(p, f) for f in range(3)]
        self.dg = LagrangeTri(p, node_coords(p, self.gll))
        self.geo = LagrangeTri(r, node_coords(r, equispaced_nodes(r)))
        self._volume()
        self._faces()

    def vol_points(self):
        return volume_rule(self.nv)

    def _jacobian(self, ctrl, pts):
        dV = self.geo.grads(pts)                                       # [Q, Nv, 2]
        J = np.zeros((ctrl.shape[0], len(pts), 2, 2))
        for m in range(ctrl.shape[1]):
            for i in range(2):
                for j in range(2):
                    J[..., i, j] = J[..., i, j] + ctrl[:, m, i][:, None] * dV[None, :, m, j]
        return J

    def _volume(self):
        pts, wq = self.vol_points()
        ctrl = self.prob.mesh.ctrl
        B = self.dg.values(pts)
        dB = self.dg.grads(pts)
        J = self._jacobian(ctrl, pts)
        dJ = det(J)
        if np.any(dJ <= 0.0):
            raise ValueError("invalid mesh: det J <= 0 at a volume quadrature point")
        C = cofactor(J)
        self.detJ = dJ
        self.B, self.dB, self.wq = B, dB, wq
        self.M = np.einsum("q,eq,qm,qn->emn", wq, dJ, B, B)
        grad = np.einsum("eqkj,qmj->eqmk", C, dB)
        self.S = np.einsum("q,eqmk,qn->ekmn", wq, grad, B)
        V = self.geo.values(pts)
        self.xq = np.einsum("qm,emd->eqd", V, ctrl)
        self.xnodes = np.einsum("nm,emd->end", self.geo.values(node_coords(self.p, self.gll)), ctrl)

    def mass_exact_order(self, e_idx):
        pts, wq = self.vol_points()
        B = self.dg.values(pts)
        dJ = det(self._jacobian(self.prob.mesh.ctrl[e_idx], pts))
        out = np.zeros((len(e_idx), self.N, self.N))
        for m in range(self.N):
            for n in range(self.N):
                acc = np.zeros(len(e_idx))
                for q in range(len(wq)):
                    acc = acc + ((wq[q] * dJ[:, q]) * B[q, m]) * B[q, n]
                out[:, m, n] = acc
        return out

    def _face_rule(self, ctrl, f, om):
        def normal(c, s, aligned=False):
            return face_normal_tri(c, self.r, f, s, aligned=aligned)
        return face_rule(ctrl, self.r, 2, f, om, self.nf, 1, normal=normal)
