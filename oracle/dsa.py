"""Diffusion synthetic acceleration of source iteration (the paper's named follow-up for
scattering-dominated problems: Sec. 4 opening and the conclusions; its DSA equations are in a
separate reference and not printed, so the operator below is this project's reading).

After a transport sweep and its moment phi_half = sum_d w_d psi_d (eq. 2), the scalar-flux error
e = phi - phi_half of a scattering-dominated problem is approximated by the diffusion problem

    -div(D grad dphi) + sigma_a dphi = sigma_s (phi_half - phi_prev),   D = 1 / (3 sigma_t),

discretised on the transport's own DG space (same curved elements, same nodal basis) with the
symmetric interior-penalty form of Wang and Ragusa's "modified interior penalty" (MIP):

  a(u, v) = sum_K int_K (D grad u . grad v + sigma_a u v)
          + sum_{interior F} int_F (kappa [[u]] [[v]] - {{D grad u . n}} [[v]] - [[u]] {{D grad v . n}})
          + sum_{boundary F} int_F (kappa u v - 1/2 (D grad u . n) v - 1/2 u (D grad v . n)),

[[u]] = u_owner - u_neighbour, n the owner's outward unit normal, {{x}} the two-sided average,
kappa = max(kappa_IP, 1/4), kappa_IP = (c/2)(D-/h- + D+/h+) on interior faces and c D / h on
boundary faces, c = 2 p (p + 1) (penalty_constant), h = |K| / |F| (element measure over face
measure).  The accelerated
iterate is phi_half + dphi.  The correction vanishes when phi_half = phi_prev, so the fixed point
is that of plain source iteration.

Quadrature: the volume rule of the transport discretisation; faces: the composite rule without
kink splitting (the integrands here have no kink).  Arithmetic is plain numpy/scipy; the system
is solved by a sparse direct factorisation.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .basis import gauss_legendre
from .geometry import (local_index_tuples, tensor_value, jacobian, det, cofactor, face_normal,
                       face_reference_coords)
from .dg import orient_coords


def _base_face_points(dim, nf, K):
    """Face points (s0[, s1]) and weights of the rule without splitting: n_f GL points (2D) or
    the K x K composite of n_f x n_f points (3D)."""
    t, wt = gauss_legendre(nf)
    if dim == 2:
        return np.array(t), None, np.array(wt)
    s0, s1, w = [], [], []
    for v in range(K):
        for u in range(K):
            for j in range(nf):
                for i in range(nf):
                    s0.append((u + t[i]) / K)
                    s1.append((v + t[j]) / K)
                    w.append((wt[i] / K) * (wt[j] / K))
    return np.array(s0), np.array(s1), np.array(w)


def _basis_and_grad(disc, ctrl, coords):
    """Values [E', P, N] and physical gradients [E', P, N, dim] of all DG basis functions at the
    reference points `coords` (shared by the elements of ctrl): grad u = cof(J) grad_ref u / det J."""
    dim, p = disc.dim, disc.p
    tup = local_index_tuples(p, dim)
    P = np.broadcast(*coords).shape[0]
    val = np.stack([np.broadcast_to(tensor_value(disc.gll, tup[m], coords), (P,)) for m in range(disc.N)], -1)
    dref = np.stack([np.stack([np.broadcast_to(tensor_value(disc.gll, tup[m], coords, deriv_axis=j), (P,))
                               for j in range(dim)], -1) for m in range(disc.N)], 1)        # [P, N, dim]
    J = jacobian(ctrl, disc.r, coords)                                                    # [E', P, dim, dim]
    C = cofactor(J)
    dJ = det(J)
    grad = np.einsum("epkj,pmj->epmk", C, dref) / dJ[:, :, None, None]
    return np.broadcast_to(val, (ctrl.shape[0],) + val.shape), grad


def penalty_constant(p):
    """c of kappa_IP = c D / h: 2 p (p + 1).  Twice the usual straight-element value: on curved
    elements the trace inequality constant is larger, and with p (p + 1) the symmetric form loses
    positive definiteness on the sine-perturbed test meshes (smallest eigenvalue -0.04 .. -0.10 at
    p = 1..3 with sigma_a near 0; +0.02 .. +0.08 with the doubled constant)."""
    return 2 * p * (p + 1)


class DiffusionOperator:
    """The MIP matrix of one problem (Discretization `disc`) as a scipy CSR matrix [E N x E N]."""

    def __init__(self, disc, c_ip=None):
        self.disc = disc
        prob = disc.prob
        dim, N, E = disc.dim, disc.N, disc.E
        self.D = 1.0 / (3.0 * prob.sigma_t)
        self.sigma_a = prob.sigma_t - prob.sigma_s
        c_ip = penalty_constant(disc.p) if c_ip is None else c_ip
        ctrl = prob.mesh.ctrl
        # volume terms
        grad = np.einsum("eqkj,qmj->eqmk", cofactor(jacobian(ctrl, disc.r, [disc.vol_points()[0][:, k]
                                                                             for k in range(dim)])),
                         disc.dB) / disc.detJ[:, :, None, None]
        K = np.einsum("q,eq,eqik,eqjk->eij", disc.wq, disc.detJ, grad, grad)
        self.K = K
        vol = np.einsum("q,eq->e", disc.wq, disc.detJ)
        blocks = {}
        self.kappa_bdr = {}                       # (e, f) -> kappa of boundary face f of e

        def add(r, c, B):
            blocks[(r, c)] = blocks.get((r, c), 0.0) + B
        for e in range(E):
            add(e, e, self.D[e] * K[e] + self.sigma_a[e] * disc.M[e])
        s0, s1, wf = _base_face_points(dim, disc.nf, disc.K if dim == 3 else 1)
        mesh = prob.mesh
        for f in range(2 * dim):
            own = [e for e in range(E) if mesh.face_nbr[e, f] < 0 or e < mesh.face_nbr[e, f]]
            if not own:
                continue
            own = np.array(own)
            co = face_reference_coords(dim, f, s0, s1)
            co = [np.broadcast_to(np.asarray(x, dtype=float), s0.shape) for x in co]
            vo, go = _basis_and_grad(disc, ctrl[own], co)                 # [F, P, N], [F, P, N, dim]
            nt = face_normal(ctrl[own], disc.r, f, s0, s1)                 # [F, P, dim] scaled normal
            area = np.einsum("p,fp->f", wf, np.linalg.norm(nt, axis=-1))
            dn_o = np.einsum("fpmk,fpk->fpm", go, nt)                     # grad u . n~ (owner side)
            for k, e in enumerate(own.tolist()):
                nb = int(mesh.face_nbr[e, f])
                h_o = vol[e] / area[k]
                a_q = wf * np.linalg.norm(nt[k], axis=-1)                  # w |n~|
                if nb < 0:
                    kap = max(c_ip * self.D[e] / h_o, 0.25)
                    self.kappa_bdr[(e, f)] = kap
                    B = kap * np.einsum("p,pi,pj->ij", a_q, vo[k], vo[k])
                    T = np.einsum("p,pj,pi->ij", wf, dn_o[k], vo[k])        # int (grad u_j . n) v_i
                    add(e, e, B - 0.5 * self.D[e] * (T + T.T))
                    continue
                fn = int(mesh.nbr_face[e, f])
                t0, t1 = orient_coords(int(mesh.orient[e, f]), s0, s1)
                cn = face_reference_coords(dim, fn, t0, t1)
                cn = [np.broadcast_to(np.asarray(x, dtype=float), s0.shape) for x in cn]
                vn, gn = _basis_and_grad(disc, ctrl[nb:nb + 1], cn)
                vn, gn = vn[0], gn[0]
                dn_n = np.einsum("pmk,pk->pm", gn, nt[k])                  # neighbour grad . owner n~
                h_n = vol[nb] / area[k]
                kap = max(0.5 * c_ip * (self.D[e] / h_o + self.D[nb] / h_n), 0.25)
                side = {0: (e, vo[k], dn_o[k], self.D[e], 1.0), 1: (nb, vn, dn_n, self.D[nb], -1.0)}
                for sv in (0, 1):                    # test function side
                    rv, v, dv, Dv, sgv = side[sv]
                    for su in (0, 1):                # trial function side
                        ru, u, du, Du, sgu = side[su]
                        B = sgu * sgv * kap * np.einsum("p,pj,pi->ij", a_q, u, v)
                        B = B - sgv * 0.5 * Du * np.einsum("p,pj,pi->ij", wf, du, v)
                        B = B - sgu * 0.5 * Dv * np.einsum("p,pj,pi->ij", wf, u, dv)
                        add(rv, ru, B)
        rows, cols, vals = [], [], []
        ii, jj = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        for (r, c), B in blocks.items():
            rows.append((r * N + ii).ravel())
            cols.append((c * N + jj).ravel())
            vals.append(np.asarray(B).ravel())
        self.blocks = blocks
        self.A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(E * N, E * N))
        self._lu = None

    def solve(self, rhs):
        """A x = rhs (sparse LU, factored once); rhs [E, N] -> [E, N]."""
        if self._lu is None:
            self._lu = spla.splu(self.A.tocsc())
        return self._lu.solve(np.asarray(rhs, dtype=np.float64).ravel()).reshape(rhs.shape)

    def correction(self, phi_half, phi_prev):
        """dphi of one DSA step: A dphi = sigma_s M (phi_half - phi_prev)."""
        disc = self.disc
        rhs = np.einsum("e,emn,en->em", disc.prob.sigma_s, disc.M, phi_half - phi_prev)
        return self.solve(rhs)


def dsa_source_iterate(sweeper, op, tol=1e-8, max_iter=1000, phi0=None):
    """Source iteration with a DSA step after every sweep: phi_{l+1} = phi_half + dphi; the
    convergence test is the one of plain source iteration on the accelerated iterates."""
    disc = sweeper.disc
    psi = np.zeros((disc.M_dirs, disc.E, disc.N))
    phi = np.zeros((disc.E, disc.N)) if phi0 is None else phi0.copy()
    hist = []
    for it in range(1, max_iter + 1):
        psi = sweeper.sweep(phi, psi)
        half = sweeper.moment(psi)
        new = half + op.correction(half, phi)
        res = np.abs(new - phi).max() / max(np.abs(new).max(), 1e-300)
        hist.append(res)
        phi = new
        if res < tol:
            return dict(phi=phi, psi=psi, iters=it, history=hist, converged=True)
    return dict(phi=phi, psi=psi, iters=max_iter, history=hist, converged=False)
