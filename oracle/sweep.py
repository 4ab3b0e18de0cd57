"""Lagged transport sweep and source iteration (paper Sec. 3, eqs. 17-21).

Source iteration (eq. 18):  (G + F + M_t) psi^(d)_{l+1} = q^(d) + M_s phi_l / (4 pi),
phi_l = sum_d omega_d psi^(d)_l (eq. 2).  The sweep solves it element by element in an
order of the acyclic graph left after cycle breaking; the coupling through removed arcs
uses the previous iterate (eq. 21):
    (G + F_<= + M_t) psi_{l+1} = q + M_s phi_l/(4 pi) - F_> psi_l,
written with this module's sign reading as A_e psi_e = rhs_e + sum_kept Fbar psi_{l+1,e'}
+ sum_removed Fbar psi_{l,e'}.
Any topological order of the kept graph gives the same result; elements are taken by
increasing (level, element id).

Convergence (Sec. 4.1 prints a garbled successive-difference norm and stops near 1e-14):
stop when ||phi_{l+1} - phi_l||_inf / ||phi_{l+1}||_inf < tol.  max_d ||psi_{l+1} - psi_l||_inf
is recorded as well.
"""
import numpy as np
import scipy.linalg as sla

FOUR_PI = 4.0 * np.pi


class Sweeper:
    """Per-(element, direction) local systems of one problem, factored once."""

    def __init__(self, disc, graph, dirs=None, chunk=8):
        self.disc = disc
        self.graph = graph
        self.dirs = list(range(disc.M_dirs)) if dirs is None else list(dirs)
        E = disc.E
        self.lu = {}
        self.coup = {}
        self.rhs_b = {}
        rem = graph["removed"]
        self.removed = set(map(tuple, rem.tolist()))
        for c0 in range(0, len(self.dirs), chunk):
            ds = self.dirs[c0:c0 + chunk]
            fb = disc.face_blocks(ds)
            for slot, d in enumerate(ds):
                for e in range(E):
                    A, coup, rb = disc.local_system(e, slot, d, fb)
                    self.lu[(d, e)] = sla.lu_factor(A)
                    self.coup[(d, e)] = [(n, F, (d, e, n) in self.removed) for (n, F) in coup]
                    self.rhs_b[(d, e)] = rb
        self.order = {d: sorted(range(E), key=lambda e: (int(graph["levels"][d, e]), e)) for d in self.dirs}

    def source_vector(self, phi):
        """s_e = M_e (q_e + sigma_s,e phi_e / (4 pi)): isotropic source plus scattering (eq. 18)."""
        disc, prob = self.disc, self.disc.prob
        x = prob.q + (prob.sigma_s[:, None] / FOUR_PI) * phi
        return np.einsum("emn,en->em", disc.M, x)

    def sweep(self, phi, psi_old, dirs=None):
        """One lagged sweep (eq. 21) over `dirs`; returns psi_new [M, E, N] (other directions 0)."""
        disc, prob = self.disc, self.disc.prob
        s = self.source_vector(phi)
        psi = np.zeros_like(psi_old)
        for d in (self.dirs if dirs is None else dirs):
            for e in self.order[d]:
                b = s[e] + self.rhs_b[(d, e)]
                if prob.q_dir is not None:
                    b = b + disc.M[e] @ prob.q_dir[d, e]
                for (n, F, lagged) in self.coup[(d, e)]:
                    b = b + F @ (psi_old[d, n] if lagged else psi[d, n])
                psi[d, e] = sla.lu_solve(self.lu[(d, e)], b)
        return psi

    def moment(self, psi):
        """phi = sum_d omega_d psi^(d) (eq. 2)."""
        return np.einsum("d,den->en", self.disc.w, psi)

    def source_iterate(self, tol=1e-8, max_iter=1000, phi0=None):
        disc = self.disc
        psi = np.zeros((disc.M_dirs, disc.E, disc.N))
        phi = np.zeros((disc.E, disc.N)) if phi0 is None else phi0.copy()
        hist, hist_psi = [], []
        for it in range(1, max_iter + 1):
            psi_new = self.sweep(phi, psi)
            phi_new = self.moment(psi_new)
            res = np.abs(phi_new - phi).max() / max(np.abs(phi_new).max(), 1e-300)
            hist.append(res)
            hist_psi.append(np.abs(psi_new - psi).max())
            psi, phi = psi_new, phi_new
            if res < tol:
                return dict(phi=phi, psi=psi, iters=it, history=hist, psi_history=hist_psi, converged=True)
        return dict(phi=phi, psi=psi, iters=max_iter, history=hist, psi_history=hist_psi, converged=False)


def global_matrix(disc):
    """The full coupled system of eq. 4 for all directions at once:
    (G + F + M_t) psi^(d) - (1/4pi) M_s sum_d' omega_d' psi^(d') = q^(d)  (dense, tiny meshes)."""
    M_, E, N = disc.M_dirs, disc.E, disc.N
    prob = disc.prob
    n = M_ * E * N
    K = np.zeros((n, n))
    rhs = np.zeros(n)
    fb = disc.face_blocks(list(range(M_)))
    idx = lambda d, e: (d * E + e) * N
    for d in range(M_):
        for e in range(E):
            A, coup, rb = disc.local_system(e, d, d, fb)
            i0 = idx(d, e)
            K[i0:i0 + N, i0:i0 + N] += A
            for (nb, F) in coup:
                j0 = idx(d, nb)
                K[i0:i0 + N, j0:j0 + N] -= F
            for d2 in range(M_):
                j0 = idx(d2, e)
                K[i0:i0 + N, j0:j0 + N] -= (prob.sigma_s[e] / (4.0 * np.pi)) * disc.w[d2] * disc.M[e]
            b = disc.M[e] @ prob.q[e] + rb
            if prob.q_dir is not None:
                b = b + disc.M[e] @ prob.q_dir[d, e]
            rhs[i0:i0 + N] = b
    return K, rhs


def global_solve(disc):
    """Direct solve of eq. 4; returns (psi [M, E, N], phi [E, N])."""
    K, rhs = global_matrix(disc)
    x = np.linalg.solve(K, rhs)
    psi = x.reshape(disc.M_dirs, disc.E, disc.N)
    return psi, np.einsum("d,den->en", disc.w, psi)
