"""Upwind DG blocks of the S_N transport equation on curved elements (paper Sec. 2).

Row index m = test function, column n = trial function (eq. 5: G_mn = -int (Omega.grad u_m) u_n).

  G_e^(d)      = -sum_k Omega_k S^k,  S^k_mn = int (du_m/dx_k) u_n dx          (eqs. 5, 11)
  M_e          = int u_m u_n dx;  M_t = sigma_t M_e,  M_s = sigma_s M_e          (eqs. 6-7, 12-13)
  F_e^(d)      = sum over all faces of e of int max(Omega.n_e, 0) u_m u_n ds     (eqs. 9, 15)
  Fbar_{e,e'}  = int max(-Omega.n_e, 0) u^e_m u^{e'}_n ds  (inflow from e')      (eqs. 10, 16)
  q_e^(d)      = int q_d u_m dx + int_{dD} max(-Omega.n_e, 0) u_m psi_inc ds     (eq. 8)

Readings (the paper is garbled or silent here):
 * eqs. 10/16 print +(|W.n|/2 - W.n/2) for the coupling; upwinding gives a contribution
   of -int (W.n_e) psi_{e'} u_m over inflow points, so the coupling enters the row of e as
   -Fbar_{e,e'} psi_{e'}: (G + F_e + M_t) psi_e - sum_e' Fbar_{e,e'} psi_{e'} = rhs.
 * eq. 8's boundary term uses (W.n + |W.n|)/2 with a minus sign, which vanishes on inflow
   faces; the inflow magnitude max(-W.n, 0) with a plus sign is used.
 * Sources q and psi_inc are given as nodal values and represented by their nodal
   interpolants, so int q u_m = (M q)_m and psi_inc(x_q) = sum_j psi_inc,j phi_j(x_q).
 * Quadrature (paper: Gauss-Legendre; Romberg suggested for kinked face integrands):
   volume: tensor GL with n_v = p + ceil(dim r / 2) points per axis (exact for the mass and
   streaming integrands with element-constant sigma).  Faces: n_f = p + r GL points per axis.
   2D faces are split at the real roots of Omega.n(s) in (0,1) (a polynomial of degree
   r - 1 <= 2), so each piece's integrand is a polynomial and the rule is exact.  3D faces are
   split where the kink curve Omega.n = 0 crosses the face edges (outer coordinate) and at the
   roots of Omega.n along every outer quadrature line (inner coordinate), on top of a K x K
   composite rule (K = face_subdiv), n_f GL points per piece and axis (face_rule_3d).
 * A face shared by e and e' is owned by min(e, e'): its points and normal are computed
   from the owner's control points; the other side uses the negated normal at the same
   points, mapped to its own face coordinates by the orientation code.
"""
import numpy as np
from .basis import gauss_legendre, gll_nodes, lagrange, lagrange_deriv
from .geometry import (local_index_tuples, tensor_value, jacobian, det, cofactor, face_normal,
                       physical_points)


def n_vol_points(p, r, dim):
    return p + (dim * r + 1) // 2


def n_face_points(p, r):
    return p + r


def dot_omega(om, vec):
    """Omega . v = Omega_0 v_0 + Omega_1 v_1 (+ Omega_2 v_2), summed left to right.
    om: list of per-component arrays (broadcastable), vec: [..., dim]."""
    g = om[0] * vec[..., 0]
    for k in range(1, vec.shape[-1]):
        g = g + om[k] * vec[..., k]
    return g


def pos(x):
    """max(x, 0) as (x > 0 ? x : 0.0)."""
    return np.where(x > 0.0, x, 0.0)


def orient_coords(code, s0, s1):
    """Owner face coordinates -> neighbour face coordinates: swap (bit 2), then
    t0 = 1 - u0 (bit 0), t1 = 1 - u1 (bit 1)."""
    if s1 is None:
        return (1.0 - s0 if code & 1 else s0), None
    u0, u1 = (s1, s0) if code & 4 else (s0, s1)
    t0 = 1.0 - u0 if code & 1 else u0
    t1 = 1.0 - u1 if code & 2 else u1
    return t0, t1


def face_node_volume_index(p, dim, f):
    """Volume node index of each face node (face node i [+ (p+1) j], i along s0, j along s1)."""
    axis, side = f // 2, f % 2
    others = [a for a in range(dim) if a != axis]
    n = p + 1
    out = []
    for fn in range((p + 1) ** (dim - 1)):
        i, j = fn % n, fn // n
        t = [0] * dim
        t[axis] = side * p
        t[others[0]] = i
        if dim == 3:
            t[others[1]] = j
        out.append(sum(t[k] * n ** k for k in range(dim)))
    return np.array(out, dtype=np.int64)


def face_basis(gll, dim, t0, t1):
    """Face-node basis values (the trace of the element basis on a face) at face
    coordinates: l_i(t0) in 2D, l_i(t0) * l_j(t1) in 3D; list over face nodes."""
    n = len(gll)
    if dim == 2:
        return [lagrange(gll, i, t0) for i in range(n)]
    out = []
    for fn in range(n * n):
        i, j = fn % n, fn // n
        out.append(lagrange(gll, i, t0) * lagrange(gll, j, t1))
    return out


BISECT_STEPS = 60     # fixed bisection count of the root isolation (interval width 2^-60)


def poly_from_samples(vals):
    """Monomial coefficients c[0..D] (list of arrays) of the degree-D polynomial through the
    points (k/D, vals[..., k]), k = 0..D.  Newton divided differences, updated in place for
    j = 1..D and k = D down to j: a_k = (a_k - a_{k-1}) / (x_k - x_{k-j}); the Newton form is then
    expanded by nested multiplication for k = D-1 down to 0: c <- c (x - x_k) + a_k, i.e.
    new_0 = a_k - x_k c_0, new_i = c_{i-1} - x_k c_i, new_m = c_{m-1} (m = current length)."""
    D = vals.shape[-1] - 1
    x = [float(k) / float(D) for k in range(D + 1)]
    a = [vals[..., k].copy() for k in range(D + 1)]
    for j in range(1, D + 1):
        for k in range(D, j - 1, -1):
            a[k] = (a[k] - a[k - 1]) / (x[k] - x[k - j])
    c = [a[D]]
    for k in range(D - 1, -1, -1):
        m = len(c)
        new = [a[k] - x[k] * c[0]]
        for i in range(1, m):
            new.append(c[i - 1] - x[k] * c[i])
        new.append(c[m - 1])
        c = new
    return c


def poly_eval(c, t):
    """Horner: P(t) = (...(c_D t + c_{D-1}) t + ...) t + c_0."""
    v = c[-1]
    for i in range(len(c) - 2, -1, -1):
        v = v * t + c[i]
    return v


def roots_01(c):
    """Roots in the open interval (0, 1) where the polynomial changes sign, ascending, as a list
    of D arrays with 1.0 in the unused slots (D = degree, elementwise over the arrays in c).

    D = 1: -c0 / c1 (c1 != 0).  D = 2: the closed form of the 2D face split: c2 == 0: -c0/c1;
    else disc = c1 c1 - (4 c2) c0 >= 0, qq = -0.5 (c1 + (c1 >= 0 ? sq : -sq)), roots qq/c2 and
    c0/qq (qq != 0); min first.  D >= 3: the roots of the derivative (d_i = (i+1) c_{i+1}, this
    function) cut [0, 1] into intervals on which P is monotone; an interval [lo, hi] with a strict
    sign change (P(lo) < 0 < P(hi) or P(lo) > 0 > P(hi)) holds one root, found by BISECT_STEPS
    bisections m = 0.5 (lo + hi) (lo <- m when P(m) > 0 equals P(lo) > 0, else hi <- m) and
    returned as 0.5 (lo + hi).  Only sign changes split a face integrand: a double root is no kink.
    """
    D = len(c) - 1
    shape = np.shape(c[0])
    one = np.ones(shape)
    if D == 1:
        with np.errstate(divide="ignore", invalid="ignore"):
            r = np.where(c[1] != 0.0, -c[0] / np.where(c[1] != 0.0, c[1], 1.0), 2.0)
        return [np.where((r > 0.0) & (r < 1.0), r, 1.0)]
    if D == 2:
        c0, c1, c2 = c
        with np.errstate(divide="ignore", invalid="ignore"):
            lin = c2 == 0.0
            c1nz = c1 != 0.0
            r_lin = np.where(lin & c1nz, -c0 / np.where(c1nz, c1, 1.0), 2.0)
            disc = c1 * c1 - (4.0 * c2) * c0
            dok = (~lin) & (disc >= 0.0)
            sq = np.sqrt(np.where(dok, disc, 0.0))
            qq = -0.5 * (c1 + np.where(c1 >= 0.0, sq, -sq))
            qnz = qq != 0.0
            ra = np.where(dok, qq / np.where(lin, 1.0, c2), 2.0)
            rb = np.where(dok & qnz, c0 / np.where(qnz, qq, 1.0), 2.0)
        ra = np.where(lin, r_lin, ra)
        rb = np.where(lin, 2.0, rb)
        ra = np.where((ra > 0.0) & (ra < 1.0), ra, 1.0)
        rb = np.where((rb > 0.0) & (rb < 1.0), rb, 1.0)
        return [np.minimum(ra, rb), np.maximum(ra, rb)]
    dc = [float(i + 1) * c[i + 1] for i in range(D)]
    crit = roots_01(dc)
    brk = [np.zeros(shape)] + crit + [one]
    found = []
    for k in range(D):
        lo, hi = brk[k].copy(), brk[k + 1].copy()
        flo, fhi = poly_eval(c, lo), poly_eval(c, hi)
        change = ((flo < 0.0) & (fhi > 0.0)) | ((flo > 0.0) & (fhi < 0.0))
        plo = flo > 0.0
        for _ in range(BISECT_STEPS):
            m = 0.5 * (lo + hi)
            same = (poly_eval(c, m) > 0.0) == plo
            lo = np.where(same, m, lo)
            hi = np.where(same, hi, m)
        found.append(np.where(change, 0.5 * (lo + hi), 1.0))
    srt = np.sort(np.stack(found, axis=-1), axis=-1)
    return [srt[..., k] for k in range(D)]


def face_rule(ctrl, r, dim, f, omega, nf, K, normal=None):
    """Per-direction face quadrature for local face f of the owner elements in ctrl.

    Returns s0, s1 (None in 2D), w, g with shape [F, D, P]; g = Omega_d . n_owner(s), n the
    unweighted scaled normal of face_normal.
    2D: pieces between breakpoints 0 <= rho1 <= rho2 <= 1, the roots of
        g(s) = c0 + c1 s + c2 s^2 built from g(0), g(1/2), g(1): c0 = g0,
        c2 = 2((g0 - 2 gh) + g1), c1 = (g1 - g0) - c2.  c2 == 0: root -c0/c1 (c1 != 0);
        else disc = c1 c1 - (4 c2) c0 >= 0, qq = -0.5 (c1 + (c1 >= 0 ? sq : -sq)), roots qq/c2
        and c0/qq (qq != 0).  Roots outside (0,1) are replaced by 1.0; rho1 = min, rho2 = max.
        Each piece [lo, hi] carries the n_f GL points s = lo + (hi - lo) t_i, w = (hi - lo) w_i.
    3D: face_rule_3d (kink-aligned splitting in both face coordinates).
    normal: (ctrl, s, aligned) -> scaled normals, for 2D faces of other element shapes
    (default: face_normal of the tensor element's face f).
    """
    t, wt = gauss_legendre(nf)
    if normal is None:
        def normal(c, s, aligned=False):
            return face_normal(c, r, f, s, aligned=aligned)
    F = ctrl.shape[0]
    D = omega.shape[0]
    om = [omega[:, k][None, :, None] for k in range(dim)]       # each [1, D, 1]
    if dim == 2:
        nref = normal(ctrl, np.array([0.0, 0.5, 1.0]))              # [F, 3, 2]
        om2 = [omega[:, k][None, :] for k in range(dim)]
        g0 = dot_omega(om2, nref[:, None, 0, :])
        gh = dot_omega(om2, nref[:, None, 1, :])
        g1 = dot_omega(om2, nref[:, None, 2, :])
        c0 = g0
        c2 = 2.0 * ((g0 - 2.0 * gh) + g1)
        c1 = (g1 - g0) - c2
        with np.errstate(divide="ignore", invalid="ignore"):
            lin = c2 == 0.0
            c1nz = c1 != 0.0
            r_lin = np.where(lin & c1nz, -c0 / np.where(c1nz, c1, 1.0), np.nan)
            disc = c1 * c1 - (4.0 * c2) * c0
            dok = (~lin) & (disc >= 0.0)
            sq = np.sqrt(np.where(dok, disc, 0.0))
            qq = -0.5 * (c1 + np.where(c1 >= 0.0, sq, -sq))
            qnz = qq != 0.0
            ra = np.where(dok, qq / np.where(lin, 1.0, c2), np.nan)
            rb = np.where(dok & qnz, c0 / np.where(qnz, qq, 1.0), np.nan)
            ra = np.where(lin, r_lin, ra)
            rb = np.where(lin, np.nan, rb)
            va = (ra > 0.0) & (ra < 1.0)
            vb = (rb > 0.0) & (rb < 1.0)
        ra = np.where(va, ra, 1.0)
        rb = np.where(vb, rb, 1.0)
        rho1 = np.minimum(ra, rb)
        rho2 = np.maximum(ra, rb)
        brk = [np.zeros_like(rho1), rho1, rho2, np.ones_like(rho1)]
        s0s, ws = [], []
        for piece in range(3):
            lo, hi = brk[piece], brk[piece + 1]
            ln = hi - lo
            for i in range(nf):
                s0s.append(lo + ln * t[i])
                ws.append(ln * wt[i])
        s0 = np.stack(s0s, axis=-1)                     # [F, D, P]
        w = np.stack(ws, axis=-1)
        nvec = normal(ctrl, s0, aligned=True)               # [F, D, P, 2]
        g = dot_omega(om, nvec)
        return s0, None, w, g
    return face_rule_3d(ctrl, r, f, omega, nf, K)


def _sorted_breaks(K, roots, shape):
    """[0, 1/K, ..., 1] merged with the roots (1.0 where unused), ascending: list of arrays."""
    base = [np.full(shape, float(k) / float(K)) for k in range(K + 1)]
    srt = np.sort(np.stack(base + [np.broadcast_to(x, shape) for x in roots], axis=-1), axis=-1)
    return srt


def _pieces_used(brk):
    """Number of leading pieces that can have nonzero length: breakpoints below 1.0 (the
    pieces after them start at 1.0 and are empty)."""
    return max(1, int((brk < 1.0).sum(axis=-1).max()))


def face_rule_3d(ctrl, r, f, omega, nf, K, normal=None):
    """3D face quadrature aligned with the kink of max(+-Omega.n, 0) (paper Sec. 2, last
    paragraph: the face integrands are only piecewise smooth where Omega.n changes sign; the
    paper suggests Romberg integration, this reading splits at the kink instead).

    g(s0, s1) = Omega . n(s0, s1) is a polynomial of degree D = 2r - 1 in each face coordinate
    (n = T0 x T1 with T0, T1 the tangents of the Q_r face map).
      outer (s1): breakpoints k/K (k = 0..K) merged with the roots in (0, 1) of the edge
        polynomials g(0, s1) and g(1, s1) (roots_01 of the interpolant through s1 = k/D): where
        the kink curve g = 0 crosses the face edges s0 = 0 and s0 = 1.  Piece [lo, hi] carries
        s1 = lo + (hi - lo) t_j, w1 = (hi - lo) w_j (n_f GL points).
      inner (s0), at every outer point: breakpoints k/K merged with the roots in (0, 1) of
        g(., s1) (interpolant through s0 = k/D): s0 = lo + (hi - lo) t_i, w = w1 ((hi - lo) w_i).
    Each inner piece integrates a polynomial exactly (n_f = p + r points); along s1 the inner
    integral is smooth on each outer piece (its kinks are where the kink curve leaves the face),
    so doubling K converges fast.  Without roots the rule is the K x K composite rule.
    Point order: outer piece, outer point, inner piece, inner point.  Pieces that start at 1.0
    are empty; they are dropped when no face/direction of the call uses them, and otherwise
    carry points of weight 0 (whose terms are +-0 and change no sum).
    normal: (ctrl, s0, s1, aligned) -> scaled normals with face_normal's conventions, for faces
    of other element shapes whose normal is of degree <= 2r - 1 in each coordinate of the unit
    square (default: face_normal of the hexahedron's face f).
    Returns s0, s1, w, g of shape [F, Dd, P].
    """
    if normal is None:
        def normal(c, a0, a1, aligned=False):
            return face_normal(c, r, f, a0, a1, aligned=aligned)
    t, wt = gauss_legendre(nf)
    F, Dd = ctrl.shape[0], omega.shape[0]
    Dg = 2 * r - 1
    xs = np.array([float(k) / float(Dg) for k in range(Dg + 1)])
    om3 = [omega[:, k][None, :, None, None] for k in range(3)]
    # edge polynomials g(0, s1), g(1, s1)
    nE = normal(ctrl, np.array([0.0, 1.0])[:, None], xs[None, :])                 # [F, 2, Dg+1, 3]
    gE = dot_omega(om3, nE[:, None, :, :, :])                                       # [F, Dd, 2, Dg+1]
    rE = roots_01(poly_from_samples(gE))                                             # Dg x [F, Dd, 2]
    brk_o = _sorted_breaks(K, [x[..., 0] for x in rE] + [x[..., 1] for x in rE], (F, Dd))
    n_o = _pieces_used(brk_o)
    s1o, w1o = [], []
    for v in range(n_o):
        lo, hi = brk_o[..., v], brk_o[..., v + 1]
        ln = hi - lo
        for j in range(nf):
            s1o.append(lo + ln * t[j])
            w1o.append(ln * wt[j])
    s1o = np.stack(s1o, axis=-1)                                                     # [F, Dd, NO]
    w1o = np.stack(w1o, axis=-1)
    NO = s1o.shape[-1]
    # inner polynomial along each outer point's line
    s0g = np.broadcast_to(xs, (F, Dd, NO, Dg + 1))
    s1g = np.broadcast_to(s1o[..., None], (F, Dd, NO, Dg + 1))
    nI = normal(ctrl, s0g, s1g, aligned=True)                                       # [F, Dd, NO, Dg+1, 3]
    gI = dot_omega([omega[:, k][None, :, None, None] for k in range(3)], nI)
    rI = roots_01(poly_from_samples(gI))                                             # Dg x [F, Dd, NO]
    brk_i = _sorted_breaks(K, rI, (F, Dd, NO))
    n_i = _pieces_used(brk_i)
    s0l, s1l, wl = [], [], []
    for u in range(n_i):
        lo, hi = brk_i[..., u], brk_i[..., u + 1]
        ln = hi - lo
        for i in range(nf):
            s0l.append(lo + ln * t[i])
            s1l.append(s1o)
            wl.append(w1o * (ln * wt[i]))
    P = NO * n_i * nf
    s0 = np.stack(s0l, axis=-1).reshape(F, Dd, P)        # [F, Dd, NO, n_i nf] -> (outer, inner) order
    s1 = np.stack(s1l, axis=-1).reshape(F, Dd, P)
    w = np.stack(wl, axis=-1).reshape(F, Dd, P)
    nvec = normal(ctrl, s0, s1, aligned=True)                                        # [F, Dd, P, 3]
    g = dot_omega([omega[:, k][None, :, None] for k in range(3)], nvec)
    return s0, s1, w, g


def coupling_block(a, phi_r, phi_u):
    """B[i][j] = sum_q (a_q * phi_r_i(q)) * phi_u_j(q), summed over q in order from 0.0.
    a: [..., P]; phi_r, phi_u: lists over face nodes of [..., P].  Returns [..., Nf, Nf]."""
    nfn = len(phi_r)
    out = np.zeros(a.shape[:-1] + (nfn, len(phi_u)))
    zero = np.zeros(a.shape[:-1] + (1,))
    for i in range(nfn):
        ar = a * phi_r[i]
        for j in range(len(phi_u)):
            # np.add.accumulate adds strictly left to right: acc_q = acc_{q-1} + term_q, acc = 0.0
            terms = np.concatenate([zero, ar * phi_u[j]], axis=-1)
            out[..., i, j] = np.add.accumulate(terms, axis=-1)[..., -1]
    return out


class Discretization:
    """All element- and face-level DG data of one problem (sn_inputs.configs.Problem)."""

    def __init__(self, prob, face_subdiv=2):
        mesh = prob.mesh
        self.prob = prob
        self.dim = dim = mesh.dim
        self.r = r = mesh.r
        self.p = p = prob.p
        self.N = (p + 1) ** dim
        self.Nf = (p + 1) ** (dim - 1)
        self.E = mesh.n_elem
        self.nv = n_vol_points(p, r, dim)
        self.nf = n_face_points(p, r)
        self.K = face_subdiv if dim == 3 else 1
        self.gll = gll_nodes(p)
        self.omega = np.asarray(prob.omega, dtype=np.float64)[:, :dim]
        self.w = np.asarray(prob.w, dtype=np.float64)
        self.M_dirs = self.omega.shape[0]
        self.n_faces = 2 * dim
        self.fnode = [face_node_volume_index(p, dim, f) for f in range(2 * dim)]
        self._volume()
        self._faces()

    # ---------------------------------------------------------------- volume
    def vol_points(self):
        t, wt = gauss_legendre(self.nv)
        dim = self.dim
        pts, wts = [], []
        for q in range(self.nv ** dim):
            idx = [(q // self.nv ** k) % self.nv for k in range(dim)]
            pts.append([t[i] for i in idx])
            w = 1.0
            for i in idx:
                w = w * wt[i]
            wts.append(w)
        return np.array(pts), np.array(wts)

    def _volume(self):
        """M_e, S^k_e at tensor GL points (eqs. 11-13); accuracy-level arithmetic (einsum)."""
        dim, p = self.dim, self.p
        pts, wq = self.vol_points()
        coords = [pts[:, k] for k in range(dim)]
        tup = local_index_tuples(p, dim)
        B = np.stack([tensor_value(self.gll, tup[m], coords) * np.ones(len(wq)) for m in range(self.N)], 1)
        dB = np.stack([np.stack([tensor_value(self.gll, tup[m], coords, deriv_axis=j) * np.ones(len(wq))
                                 for j in range(dim)], -1) for m in range(self.N)], 1)   # [Q, N, dim]
        J = jacobian(self.prob.mesh.ctrl, self.r, coords)            # [E, Q, dim, dim]
        dJ = det(J)
        if np.any(dJ <= 0.0):
            raise ValueError("invalid mesh: det J <= 0 at a volume quadrature point")
        C = cofactor(J)
        self.detJ = dJ
        self.B, self.dB, self.wq = B, dB, wq
        self.M = np.einsum("q,eq,qm,qn->emn", wq, dJ, B, B)
        grad = np.einsum("eqkj,qmj->eqmk", C, dB)                     # |J| d u_m / d x_k
        self.S = np.einsum("q,eqmk,qn->ekmn", wq, grad, B)
        # physical DG node positions (used for diagnostics and tests)
        nodes = [np.array([self.gll[tp[k]] for tp in tup]) for k in range(dim)]
        self.xnodes = physical_points(self.prob.mesh.ctrl, self.r, nodes)    # [E, N, dim]
        self.xq = physical_points(self.prob.mesh.ctrl, self.r, coords)       # [E, Q, dim]

    def mass_exact_order(self, e_idx):
        """M_e[m][n] = sum_q ((w_q * detJ_q) * u_m(q)) * u_n(q), in increasing q from 0.0
        (the mass matrix in the fixed order used by the SigInvFace weight).  [E', N, N]."""
        dim = self.dim
        pts, wq = self.vol_points()
        coords = [pts[:, k] for k in range(dim)]
        tup = local_index_tuples(self.p, dim)
        B = [np.broadcast_to(tensor_value(self.gll, tup[m], coords), (len(wq),)) for m in range(self.N)]
        ctrl = self.prob.mesh.ctrl[e_idx]
        dJ = det(jacobian(ctrl, self.r, coords))                     # [E', Q]
        out = np.zeros((len(e_idx), self.N, self.N))
        for m in range(self.N):
            for n in range(self.N):
                acc = np.zeros(len(e_idx))
                for q in range(len(wq)):
                    acc = acc + ((wq[q] * dJ[:, q]) * B[m][q]) * B[n][q]
                out[:, m, n] = acc
        return out

    # ---------------------------------------------------------------- faces
    def _face_rule(self, ctrl, f, om):
        """Face quadrature of face f of the elements in ctrl for the directions om (face_rule)."""
        return face_rule(ctrl, self.r, self.dim, f, om, self.nf, self.K)

    def _face_basis(self, s0, s1):
        """Face-node basis values at face coordinates (list of Nf arrays)."""
        return face_basis(self.gll, self.dim, s0, s1)

    def _orient(self, code, s0, s1):
        """The neighbour's face coordinates of our face coordinates (orientation code)."""
        return orient_coords(code, s0, s1)

    def _faces(self):
        mesh = self.prob.mesh
        self.iface = []      # (owner, f, nbr, f_nbr, orient owner->nbr)
        self.bface = []      # (e, f) in increasing (e, f): the boundary-face numbering
        for e in range(self.E):
            for f in range(self.n_faces):
                n = int(mesh.face_nbr[e, f])
                if n < 0:
                    self.bface.append((e, f))
                elif e < n:
                    self.iface.append((e, f, n, int(mesh.nbr_face[e, f]), int(mesh.orient[e, f])))
        self.bface_index = {ef: k for k, ef in enumerate(self.bface)}

    def face_blocks(self, dirs):
        """Face quadrature data and N_f x N_f blocks for the directions in `dirs`.

        Interior face k, direction slot j:
          out_o[k,j]  = sum_q max(g,0) w phi^o_i phi^o_j       (owner's F_e block)
          out_n[k,j]  = sum_q max(-g,0) w phi^n_i phi^n_j      (neighbour's F_e block)
          bar_o[k,j]  = sum_q max(-g,0) w phi^o_i phi^n_j      (Fbar owner <- neighbour)
          bar_n[k,j]  = sum_q max(g,0) w phi^n_i phi^o_j       (Fbar neighbour <- owner)
        Boundary face k: bout[k,j] (F_e block), bin[k,j] (inflow block for psi_inc).
        Inflow amounts are a = max(-/+ g, 0) * w (max first, then the weight).
        """
        dim = self.dim
        ctrl = self.prob.mesh.ctrl
        om = self.omega[list(dirs)]
        res = {}
        iface = np.array(self.iface, dtype=np.int64).reshape(-1, 5)
        D = len(dirs)
        Nf = self.Nf
        out_o = np.zeros((len(iface), D, Nf, Nf))
        out_n = np.zeros_like(out_o)
        bar_o = np.zeros_like(out_o)
        bar_n = np.zeros_like(out_o)
        for f in range(self.n_faces):
            sel = np.nonzero(iface[:, 1] == f)[0] if len(iface) else np.zeros(0, dtype=np.int64)
            if len(sel) == 0:
                continue
            s0, s1, w, g = self._face_rule(ctrl[iface[sel, 0]], f, om)
            ao = pos(-g) * w
            an = pos(g) * w
            phi_o = self._face_basis(s0, s1)
            codes = iface[sel, 4]
            phi_n = [np.zeros_like(s0) for _ in range(Nf)]
            for code in np.unique(codes):
                cs = codes == code
                t0, t1 = self._orient(int(code), s0[cs], None if s1 is None else s1[cs])
                vals = self._face_basis(t0, t1)
                for i in range(Nf):
                    phi_n[i][cs] = vals[i]
            out_o[sel] = coupling_block(an, phi_o, phi_o)
            out_n[sel] = coupling_block(ao, phi_n, phi_n)
            bar_o[sel] = coupling_block(ao, phi_o, phi_n)
            bar_n[sel] = coupling_block(an, phi_n, phi_o)
        bface = np.array(self.bface, dtype=np.int64).reshape(-1, 2)
        bout = np.zeros((len(bface), D, Nf, Nf))
        bin_ = np.zeros_like(bout)
        for f in range(self.n_faces):
            sel = np.nonzero(bface[:, 1] == f)[0] if len(bface) else np.zeros(0, dtype=np.int64)
            if len(sel) == 0:
                continue
            s0, s1, w, g = self._face_rule(ctrl[bface[sel, 0]], f, om)
            phi = self._face_basis(s0, s1)
            bout[sel] = coupling_block(pos(g) * w, phi, phi)
            bin_[sel] = coupling_block(pos(-g) * w, phi, phi)
        res.update(out_o=out_o, out_n=out_n, bar_o=bar_o, bar_n=bar_n, bout=bout, bin=bin_)
        return res

    # ---------------------------------------------------------------- local systems
    def local_system(self, e, d_slot, d, fb):
        """(A, couplings, rhs_bdr) for element e, direction d (fb = face_blocks(...), d_slot its slot).

        A = G + F_e + M_t (eq. 17's left side restricted to e's block row);
        couplings: list of (e', Fbar_{e,e'} as [N, N] full matrix);
        rhs_bdr: boundary inflow part of q_e^(d) (needs psi_inc)."""
        N = self.N
        A = -np.einsum("k,kmn->mn", self.omega[d], self.S[e]) + self.prob.sigma_t[e] * self.M[e]
        coup = []
        rhs_b = np.zeros(N)
        mesh = self.prob.mesh
        for f in range(self.n_faces):
            n = int(mesh.face_nbr[e, f])
            idx = self.fnode[f]
            if n < 0:
                k = self.bface_index[(e, f)]
                A[np.ix_(idx, idx)] += fb["bout"][k, d_slot]
                if self.prob.psi_inc is not None:
                    rhs_b[idx] += fb["bin"][k, d_slot] @ self.prob.psi_inc[d, k]
                continue
            fn = int(mesh.nbr_face[e, f])
            nidx = self.fnode[fn]
            if e < n:
                k = self._iface_index(e, f)
                A[np.ix_(idx, idx)] += fb["out_o"][k, d_slot]
                blk = fb["bar_o"][k, d_slot]
            else:
                k = self._iface_index(n, fn)
                A[np.ix_(idx, idx)] += fb["out_n"][k, d_slot]
                blk = fb["bar_n"][k, d_slot]
            full = np.zeros((N, N))
            full[np.ix_(idx, nidx)] = blk
            coup.append((n, full))
        return A, coup, rhs_b

    def _iface_index(self, owner, f):
        if not hasattr(self, "_iface_map"):
            self._iface_map = {(o, ff): k for k, (o, ff, _n, _fn, _c) in enumerate(self.iface)}
        return self._iface_map[(owner, f)]
