"""Manufactured-solution and attenuation inputs (nodal source and inflow values).

These generators evaluate closed-form fields at the physical positions of the DG nodes
(tensor Gauss-Lobatto-Legendre nodes of order p mapped through the element's Q_r map),
which is how the library takes direction-dependent sources and incident fluxes.
"""
import math
import numpy as np


def _gll(p):
    if p == 1:
        return [0.0, 1.0]
    if p == 2:
        return [0.0, 0.5, 1.0]
    if p == 3:
        a = 1.0 / math.sqrt(5.0)
        return [0.0, 0.5 * (1.0 - a), 0.5 * (1.0 + a), 1.0]
    raise ValueError(p)


def _lag(nodes, j, x):
    v = 1.0
    for k, nk in enumerate(nodes):
        if k != j:
            v = v * (x - nk) / (nodes[j] - nk)
    return v


def _tri_lagrange_values(nodes, pts):
    """[len(pts)][len(nodes)] values of the Lagrange basis of the triangle node set `nodes`
    (total degree k with (k+1)(k+2)/2 nodes) at `pts`, through the monomial Vandermonde."""
    n = len(nodes)
    k = {3: 1, 6: 2, 10: 3}[n]
    mono = [(a, d - a) for d in range(k + 1) for a in range(d, -1, -1)]
    V = np.array([[x ** a * y ** b for (a, b) in mono] for (x, y) in nodes])
    C = np.linalg.inv(V)                                   # columns: node basis coefficients
    P = np.array([[x ** a * y ** b for (a, b) in mono] for (x, y) in pts])
    return P @ C


def dg_node_positions(mesh, p):
    """[n_elem][N][dim] physical positions of the DG nodes."""
    if getattr(mesh, "simplex", False) and mesh.dim == 3 and mesh.r == 2:
        return mesh.ctrl[:, :(4 if p == 1 else 10)].copy()      # the DG nodes are P_2 geometry nodes
    if getattr(mesh, "simplex", False) and mesh.dim == 3:
        from .mesh import TET_EDGES
        lam = [[1.0, 0.0, 0.0, 0.0], [0.0, 1.0, 0.0, 0.0], [0.0, 0.0, 1.0, 0.0], [0.0, 0.0, 0.0, 1.0]]
        if p == 2:
            lam += [[0.5 if k in e else 0.0 for k in range(4)] for e in TET_EDGES]
        return np.einsum("nm,emd->end", np.array(lam), mesh.ctrl)
    if getattr(mesh, "simplex", False):
        from .mesh import tri_node_coords
        dg = tri_node_coords(p, _gll(p))
        geo = tri_node_coords(mesh.r, [a / mesh.r for a in range(mesh.r + 1)])
        W = _tri_lagrange_values(geo, dg)                  # [N][Nv]
        return np.einsum("nm,emd->end", W, mesh.ctrl)
    dim, r = mesh.dim, mesh.r
    g = _gll(p)
    geo = [a / r for a in range(r + 1)]
    n = p + 1
    out = np.zeros((mesh.n_elem, n ** dim, dim))
    for m in range(n ** dim):
        xi = [g[(m // n ** k) % n] for k in range(dim)]
        for c in range((r + 1) ** dim):
            v = 1.0
            for k in range(dim):
                v *= _lag(geo, (c // (r + 1) ** k) % (r + 1), xi[k])
            out[:, m, :] += v * mesh.ctrl[:, c, :]
    return out


def boundary_faces(mesh):
    """Boundary faces (e, f) in increasing (e, f) order: the library's boundary numbering."""
    nfc = mesh.face_nbr.shape[1]
    return [(e, f) for e in range(mesh.n_elem) for f in range(nfc) if mesh.face_nbr[e, f] < 0]


def _face_ids(mesh, p, f):
    if getattr(mesh, "simplex", False) and mesh.dim == 3:
        from .mesh import TET_FACES, TET_EDGES
        a, b, c = TET_FACES[f]
        ids = [a, b, c]
        if p == 2:
            ei = lambda x, y: next(k for k, e in enumerate(TET_EDGES) if set(e) == {x, y})
            ids += [4 + ei(a, b), 4 + ei(b, c), 4 + ei(c, a)]
        return ids
    if getattr(mesh, "simplex", False):
        from .mesh import tri_edge_nodes
        return tri_edge_nodes(p, f)
    return face_node_ids(p, mesh.dim, f)


def _n_face_nodes(mesh, p):
    if getattr(mesh, "simplex", False):
        return (p + 1) * (p + 2) // 2 if mesh.dim == 3 else p + 1
    return (p + 1) ** (mesh.dim - 1)


def face_node_ids(p, dim, f):
    axis, side = f // 2, f % 2
    others = [a for a in range(dim) if a != axis]
    n = p + 1
    out = []
    for fn in range(n ** (dim - 1)):
        t = [0] * dim
        t[axis] = side * p
        t[others[0]] = fn % n
        if dim == 3:
            t[others[1]] = fn // n
        out.append(sum(t[k] * n ** k for k in range(dim)))
    return out


def annulus_mms(prob, sigma_t=1.0, sigma_s=0.5):
    """Manufactured psi_d(x, y) = [ (1 + x^2 + y^2)/2 + cos(3x + 3y/2) ] (mu_d^2 + eta_d)
    (the paper's annulus MMS form, Sec. 4.1).  Sets uniform sigma_t/sigma_s and the nodal
    q_dir and psi_inc that make it the exact solution of the S_N equation; returns
    (prob, f, phi_exact_factor) with phi_exact(x) = f(x) * phi_exact_factor."""
    mesh = prob.mesh
    X = dg_node_positions(mesh, prob.p)
    x, y = X[..., 0], X[..., 1]
    f = 0.5 * (1.0 + x * x + y * y) + np.cos(3 * x + 1.5 * y)
    fx = x - 3.0 * np.sin(3 * x + 1.5 * y)
    fy = y - 1.5 * np.sin(3 * x + 1.5 * y)
    om, w = prob.omega, prob.w
    ang = om[:, 0] ** 2 + om[:, 1]
    phi_fac = float(np.sum(w * ang))
    ne = mesh.n_elem
    prob.sigma_t = sigma_t * np.ones(ne)
    prob.sigma_s = sigma_s * np.ones(ne)
    prob.q = np.zeros_like(f)
    qd = np.empty((len(w),) + f.shape)
    for d in range(len(w)):
        qd[d] = (om[d, 0] * fx + om[d, 1] * fy) * ang[d] + sigma_t * f * ang[d] - sigma_s / (4 * np.pi) * f * phi_fac
    prob.q_dir = qd
    bf = boundary_faces(mesh)
    nf = _n_face_nodes(mesh, prob.p)
    pin = np.zeros((len(w), len(bf), nf))
    for k, (e, fc) in enumerate(bf):
        ids = _face_ids(mesh, prob.p, fc)
        pin[:, k, :] = f[e, ids][None, :] * ang[:, None]
    prob.psi_inc = pin

    def exact_f(P):
        return 0.5 * (1.0 + P[..., 0] ** 2 + P[..., 1] ** 2) + np.cos(3 * P[..., 0] + 1.5 * P[..., 1])
    return prob, exact_f, phi_fac


def attenuation(prob, sigma_t=2.0):
    """Pure absorber (sigma_s = 0, q = 0) on the unit square/cube with inflow
    psi_inc = exp(-sigma_t * dist) where dist is the path length back to the x-inflow plane
    along -Omega:  psi_d(x) = exp(-sigma_t (x - x_in)/mu_d), x_in = 0 (mu > 0) or 1 (mu < 0).
    That field is smooth and solves Omega.grad psi + sigma_t psi = 0 exactly."""
    mesh = prob.mesh
    om = prob.omega
    ne = mesh.n_elem
    prob.sigma_t = sigma_t * np.ones(ne)
    prob.sigma_s = np.zeros(ne)
    X = dg_node_positions(mesh, prob.p)
    prob.q = np.zeros(X.shape[:2])
    prob.q_dir = None
    bf = boundary_faces(mesh)
    nf = _n_face_nodes(mesh, prob.p)
    pin = np.zeros((len(om), len(bf), nf))
    for k, (e, fc) in enumerate(bf):
        ids = _face_ids(mesh, prob.p, fc)
        xb = X[e, ids, 0]
        for d in range(len(om)):
            x_in = 0.0 if om[d, 0] > 0 else 1.0
            pin[d, k, :] = np.exp(-sigma_t * (xb - x_in) / om[d, 0])
    prob.psi_inc = pin

    def exact(P, d):
        x_in = 0.0 if om[d, 0] > 0 else 1.0
        return np.exp(-sigma_t * (P[..., 0] - x_in) / om[d, 0])
    return prob, exact
