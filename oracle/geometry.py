"""Curved-element geometry (paper Sec. 2, 'Discrete representation of the HO mesh').

x_e(xi) = sum_m x_{e,m} v_m(xi)                       (eq. 1, Q_r Lagrange map)
J^e(xi) = sum_m x_{e,m} [grad v_m(xi)]^T               (eq. 14)
|J| J^{-T} = cof(J)   (used to map reference gradients, eqs. 11-13)
Face normal scaled by the face Jacobian: n |J^Gamma| = cof(J) n_hat (Nanson), which only
involves derivatives tangential to the face, i.e. the face's own control points.

Arrays are vectorised over elements (leading axis) and evaluation points; the
arithmetic per (element, point) follows the order stated in each docstring.
"""
import numpy as np
from .basis import equispaced_nodes, lagrange, lagrange_deriv


def local_index_tuples(order, dim):
    """Tensor node tuples (i0, i1[, i2]) in local order m = i0 + (order+1) i1 + ..."""
    n = order + 1
    out = []
    for m in range(n ** dim):
        t, rem = [], m
        for _ in range(dim):
            t.append(rem % n)
            rem //= n
        out.append(tuple(t))
    return out


def shape_factor(nodes, idx, x, deriv):
    """One 1D factor of a tensor basis function: l_idx(x) or l_idx'(x)."""
    return lagrange_deriv(nodes, idx, x) if deriv else lagrange(nodes, idx, x)


def tensor_value(nodes, idx_tuple, coords, deriv_axis=None):
    """prod_k factor_k, multiplied left to right starting from 1.0, factor_k = l'_{i_k}
    on deriv_axis and l_{i_k} elsewhere.  coords: per-axis scalars or arrays."""
    v = 1.0
    for k, (i, x) in enumerate(zip(idx_tuple, coords)):
        v = v * shape_factor(nodes, i, x, k == deriv_axis)
    return v


def jacobian(ctrl, r, coords):
    """J[..., i, j] = sum_m x_{m,i} dv_m/dxi_j, summed in increasing m from 0.0 (eq. 14).

    ctrl   : [E, Nv, dim] control points.
    coords : list of dim arrays broadcastable against each other (reference coordinates).
    Returns J with shape broadcast(E-leading) + [dim, dim]: ctrl's E axis is placed first
    and the coordinate arrays' shape after it.
    """
    E, Nv, dim = ctrl.shape
    gn = equispaced_nodes(r)
    tup = local_index_tuples(r, dim)
    cshape = np.broadcast(*coords).shape
    J = np.zeros((E,) + cshape + (dim, dim))
    ext = (slice(None),) + (None,) * len(cshape)
    for m in range(Nv):
        dv = [np.broadcast_to(tensor_value(gn, tup[m], coords, deriv_axis=j), cshape) for j in range(dim)]
        for i in range(dim):
            xm = ctrl[:, m, i][ext]
            for j in range(dim):
                J[..., i, j] = J[..., i, j] + xm * dv[j]
    return J


def det(J):
    """2D: J00 J11 - J01 J10.  3D: J00 (J11 J22 - J12 J21) - J01 (J10 J22 - J12 J20)
    + J02 (J10 J21 - J11 J20), evaluated ((t0 - t1) + t2)."""
    if J.shape[-1] == 2:
        return J[..., 0, 0] * J[..., 1, 1] - J[..., 0, 1] * J[..., 1, 0]
    t0 = J[..., 0, 0] * (J[..., 1, 1] * J[..., 2, 2] - J[..., 1, 2] * J[..., 2, 1])
    t1 = J[..., 0, 1] * (J[..., 1, 0] * J[..., 2, 2] - J[..., 1, 2] * J[..., 2, 0])
    t2 = J[..., 0, 2] * (J[..., 1, 0] * J[..., 2, 1] - J[..., 1, 1] * J[..., 2, 0])
    return (t0 - t1) + t2


def cofactor(J):
    """cof(J) = |J| J^{-T}: cof[i][j] = (-1)^{i+j} minor_ij."""
    C = np.empty_like(J)
    if J.shape[-1] == 2:
        C[..., 0, 0] = J[..., 1, 1]
        C[..., 0, 1] = -J[..., 1, 0]
        C[..., 1, 0] = -J[..., 0, 1]
        C[..., 1, 1] = J[..., 0, 0]
        return C
    for i in range(3):
        for j in range(3):
            r0, r1 = [a for a in range(3) if a != i]
            c0, c1 = [a for a in range(3) if a != j]
            minor = J[..., r0, c0] * J[..., r1, c1] - J[..., r0, c1] * J[..., r1, c0]
            C[..., i, j] = minor if (i + j) % 2 == 0 else -minor
    return C


def physical_points(ctrl, r, coords):
    """x(xi) = sum_m x_m v_m(xi) in increasing m from 0.0 (eq. 1)."""
    E, Nv, dim = ctrl.shape
    gn = equispaced_nodes(r)
    tup = local_index_tuples(r, dim)
    cshape = np.broadcast(*coords).shape
    X = np.zeros((E,) + cshape + (dim,))
    ext = (slice(None),) + (None,) * len(cshape)
    for m in range(Nv):
        v = np.broadcast_to(tensor_value(gn, tup[m], coords), cshape)
        for i in range(dim):
            X[..., i] = X[..., i] + ctrl[:, m, i][ext] * v
    return X


def face_reference_coords(dim, f, s0, s1=None):
    """Reference coordinates of face f (= 2*axis + side) at face coordinates (s0[, s1]):
    xi_axis = side, the other axes in increasing order take s0, s1."""
    axis, side = f // 2, f % 2
    others = [a for a in range(dim) if a != axis]
    coords = [None] * dim
    coords[axis] = float(side)
    coords[others[0]] = s0
    if dim == 3:
        coords[others[1]] = s1
    return coords


def face_normal(ctrl, r, f, s0, s1=None, aligned=False):
    """Outward normal scaled by the face Jacobian, n |J^Gamma| = cof(J) n_hat, at face
    coordinates (s0[, s1]) of local face f of each element in ctrl ([E, Nv, dim]).
    aligned=False: the coordinates are shared by all elements, result [E, *shape(s), dim];
    aligned=True : the coordinate arrays already carry the element axis first, result
                   [*shape(s), dim].

    Only tangential derivatives enter: T_b = sum_m x_m dv_m/dxi_b (increasing m from 0.0).
    2D, axis 0: (T_1[1], -T_1[0]); axis 1: (-T_0[1], T_0[0]).
    3D, axis a: T_{(a+1)%3} x T_{(a+2)%3}, component i = u_{i+1} v_{i+2} - u_{i+2} v_{i+1}.
    Side 0 (xi_axis = 0) negates the vector.  Returns [E, *shape(s), dim].
    """
    E, Nv, dim = ctrl.shape
    axis, side = f // 2, f % 2
    coords = face_reference_coords(dim, f, s0, s1)
    gn = equispaced_nodes(r)
    tup = local_index_tuples(r, dim)
    cshape = np.broadcast(*[c for c in coords]).shape
    if aligned:
        oshape = cshape
        ext = (slice(None),) + (None,) * (len(cshape) - 1)
    else:
        oshape = (E,) + cshape
        ext = (slice(None),) + (None,) * len(cshape)
    tang_axes = [(axis + 1) % dim] if dim == 2 else [(axis + 1) % 3, (axis + 2) % 3]
    T = {b: np.zeros(oshape + (dim,)) for b in tang_axes}
    for m in range(Nv):
        for b in tang_axes:
            dv = np.broadcast_to(tensor_value(gn, tup[m], coords, deriv_axis=b), cshape)
            for i in range(dim):
                T[b][..., i] = T[b][..., i] + ctrl[:, m, i][ext] * dv
    n = np.empty(oshape + (dim,))
    if dim == 2:
        t = T[tang_axes[0]]
        if axis == 0:
            n[..., 0] = t[..., 1]
            n[..., 1] = -t[..., 0]
        else:
            n[..., 0] = -t[..., 1]
            n[..., 1] = t[..., 0]
    else:
        u, v = T[tang_axes[0]], T[tang_axes[1]]
        for i in range(3):
            a, b = (i + 1) % 3, (i + 2) % 3
            n[..., i] = u[..., a] * v[..., b] - u[..., b] * v[..., a]
    if side == 0:
        n = -n
    return n
