"""Pins of the oracle's geometry and DG blocks against closed forms, conservation identities,
manufactured solutions and the dense coupled solve (Sec. 2-3 of the paper)."""
import numpy as np
import pytest

import sn_inputs as si
from sn_inputs.mms import annulus_mms, attenuation, dg_node_positions
from oracle.basis import gll_nodes, gauss_legendre
from oracle.geometry import jacobian, det, face_normal
from oracle.dg import Discretization, face_rule
from oracle.graph import build_graph
from oracle.sweep import Sweeper, global_solve


def affine_disp(A, b):
    A = np.asarray(A, dtype=float)

    def f(X):
        return X @ (A - np.eye(A.shape[0])).T + b
    return f


def lagrange_poly_1d(nodes):
    """Cardinal polynomials of the nodes via numpy polyfit (independent of the oracle)."""
    out = []
    for j in range(len(nodes)):
        y = np.zeros(len(nodes)); y[j] = 1.0
        out.append(np.poly1d(np.polyfit(nodes, y, len(nodes) - 1)))
    return out


def integ01(poly):
    P = np.polyint(poly)
    return P(1.0) - P(0.0)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_affine_mass_and_streaming_match_closed_form(p):
    A = np.array([[1.2, 0.3], [-0.1, 0.9]])
    n = 3
    prob = si.make_config("2d_sine_q2_p1_s4", n=n, p=p)
    prob.mesh = si.structured_mesh((n, n), 2, affine_disp(A, np.array([0.1, -0.2])))
    D = Discretization(prob)
    L = lagrange_poly_1d(gll_nodes(p))
    M1 = np.array([[integ01(a * b) for b in L] for a in L])
    D1 = np.array([[integ01(np.polyder(a) * b) for b in L] for a in L])
    J = A / n
    dJ = np.linalg.det(J)
    Jit = np.linalg.inv(J).T
    M_ex = dJ * np.kron(M1, M1)
    d0 = np.kron(M1, D1)          # int d/dxi0 u_m u_n  (m = i + (p+1) j)
    d1 = np.kron(D1, M1)
    S_ex = [dJ * (Jit[k, 0] * d0 + Jit[k, 1] * d1) for k in range(2)]
    for e in range(D.E):
        assert np.allclose(D.M[e], M_ex, atol=1e-14)
        for k in range(2):
            assert np.allclose(D.S[e, k], S_ex[k], atol=1e-13)


@pytest.mark.parametrize("name,n", [("2d_sine_q2_p1_s4", 6), ("2d_smooth_q3_p3_s8", 6), ("3d_smooth_q2_p2_s12", 3)])
def test_measure_and_closed_surface(name, n):
    prob = si.make_config(name, n=n)
    D = Discretization(prob)
    # the displacement vanishes on the boundary: the union of the curved elements is [0,1]^dim
    assert abs(np.einsum("q,eq->", D.wq, D.detJ) - 1.0) < 1e-13
    # divergence theorem: the scaled normals of a closed element surface integrate to zero
    t, w = gauss_legendre(D.nf)
    tot = np.zeros((D.E, D.dim))
    for f in range(2 * D.dim):
        if D.dim == 2:
            nv = face_normal(prob.mesh.ctrl, D.r, f, t)
            tot += np.einsum("q,eqk->ek", w, nv)
        else:
            nv = face_normal(prob.mesh.ctrl, D.r, f, t[:, None], t[None, :])
            tot += np.einsum("i,j,ejik->ek", w, w, nv)
    assert np.abs(tot).max() < 1e-14


@pytest.mark.parametrize("name,n,seed", [("2d_sine_q2_p1_s4", 4, 3), ("3d_twist_q2_p2_s8", 2, 5)])
def test_shared_face_normals_are_opposite(name, n, seed):
    prob = si.make_config(name, n=n, reorient_seed=seed)
    mesh = prob.mesh
    from oracle.dg import orient_coords
    rng = np.random.default_rng(0)
    s0 = rng.uniform(size=5)
    s1 = rng.uniform(size=5) if mesh.dim == 3 else None
    for e in range(mesh.n_elem):
        for f in range(2 * mesh.dim):
            nb = mesh.face_nbr[e, f]
            if nb < 0:
                continue
            t0, t1 = orient_coords(int(mesh.orient[e, f]), s0, s1)
            a = face_normal(mesh.ctrl[e:e + 1], mesh.r, f, s0, s1, aligned=False)[0] if mesh.dim == 2 else \
                face_normal(mesh.ctrl[e:e + 1], mesh.r, f, s0, s1)[0]
            b = face_normal(mesh.ctrl[nb:nb + 1], mesh.r, int(mesh.nbr_face[e, f]), t0, t1)[0]
            assert np.allclose(a, -b, atol=1e-13)


@pytest.mark.parametrize("name,n,p", [("2d_sine_q2_p1_s4", 4, 2), ("2d_smooth_q3_p3_s8", 3, 3), ("3d_twist_q2_p2_s8", 2, 2)])
def test_divergence_identity_of_local_blocks(name, n, p):
    """(G + F_e) 1 = sum of the inflow blocks applied to 1: -int W.grad u_m = -oint (W.n) u_m,
    so F_e - (W.n) = max(-W.n, 0) on every face (a dropped term or flipped sign fails)."""
    prob = si.make_config(name, n=n, p=p)
    D = Discretization(prob)
    dirs = list(range(0, D.M_dirs, 3))
    fb = D.face_blocks(dirs)
    ones = np.ones(D.N)
    for slot, d in enumerate(dirs):
        for e in range(D.E):
            A, coup, _ = D.local_system(e, slot, d, fb)
            lhs = (A - prob.sigma_t[e] * D.M[e]) @ ones
            rhs = sum(F @ ones for _, F in coup) if coup else np.zeros(D.N)
            for f in range(2 * D.dim):
                if prob.mesh.face_nbr[e, f] < 0:
                    k = D.bface_index[(e, f)]
                    rhs = rhs.copy()
                    rhs[D.fnode[f]] += fb["bin"][k, slot] @ np.ones(D.Nf)
            assert np.allclose(lhs, rhs, atol=1e-14), (e, d)


def test_one_sweep_is_exact_on_acyclic_mesh_without_scattering():
    prob = si.make_config("2d_sine_q2_p1_s4", n=4, p=2)
    prob.mesh = si.structured_mesh((4, 4), 2, affine_disp([[1.0, 0.2], [0.0, 1.1]], np.zeros(2)))
    prob.sigma_s = np.zeros(prob.mesh.n_elem)
    prob.sigma_t = np.linspace(0.5, 3.0, prob.mesh.n_elem)
    D = Discretization(prob)
    G = build_graph(D, "face")
    assert len(G["removed"]) == 0
    S = Sweeper(D, G)
    psi = S.sweep(np.zeros((D.E, D.N)), np.zeros((D.M_dirs, D.E, D.N)))
    psi_ref, _ = global_solve(D)
    assert np.abs(psi - psi_ref).max() <= 1e-13 * np.abs(psi_ref).max()


@pytest.mark.parametrize("weighting", ["unity", "face", "siginvface"])
def test_converged_lagged_si_equals_dense_coupled_solve(weighting):
    prob = si.make_config("2d_sine_q2_p1_s4", n=4, p=2)
    prob.mesh = si.structured_mesh((4, 4), 2, si.disp_sine_2d(0.08))
    D = Discretization(prob)
    G = build_graph(D, weighting)
    assert len(G["removed"]) > 0          # the curved mesh has cycles: lagging is exercised
    R = Sweeper(D, G).source_iterate(tol=1e-13)
    _, phi_ref = global_solve(D)
    assert np.abs(R["phi"] - phi_ref).max() <= 1e-10 * np.abs(phi_ref).max()


def test_particle_balance():
    """Leakage + absorption = source at convergence (constant test function, Sec. 2)."""
    prob = si.make_config("2d_sine_q2_p1_s4", n=6, p=2)
    prob.sigma_t = np.linspace(0.5, 2.0, prob.mesh.n_elem)
    prob.sigma_s = 0.6 * prob.sigma_t
    D = Discretization(prob)
    G = build_graph(D, "face")
    R = Sweeper(D, G).source_iterate(tol=1e-13)
    fb = D.face_blocks(list(range(D.M_dirs)))
    leak = 0.0
    for k, (e, f) in enumerate(D.bface):
        for d in range(D.M_dirs):
            leak += D.w[d] * np.sum(fb["bout"][k, d] @ R["psi"][d, e, D.fnode[f]])
    absorb = np.einsum("e,emn,en->", prob.sigma_t - prob.sigma_s, D.M, R["phi"])
    source = 4 * np.pi * np.einsum("emn,en->", D.M, prob.q)
    assert abs(leak + absorb - source) <= 1e-10 * source


def _l2(D, vals_q):
    return np.sqrt(np.einsum("q,eq,eq->", D.wq, D.detJ, vals_q ** 2))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_mms_scalar_flux_converges_at_order_p_plus_1(p):
    errs = []
    for n in (4, 8, 16):
        prob = si.make_config("2d_sine_q2_p1_s4", n=n, p=p)
        prob, fex, fac = annulus_mms(prob)
        D = Discretization(prob)
        R = Sweeper(D, build_graph(D, "face")).source_iterate(tol=1e-12)
        phi_q = np.einsum("qm,em->eq", D.B, R["phi"])
        errs.append(_l2(D, phi_q - fac * fex(D.xq)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] >= p + 1 - 0.2, (errs, orders)


@pytest.mark.parametrize("p", [1, 2])
def test_pure_absorber_attenuation_converges(p):
    errs = []
    for n in (4, 8, 16):
        prob = si.make_config("2d_sine_q2_p1_s4", n=n, p=p)
        prob, exact = attenuation(prob, sigma_t=2.0)
        D = Discretization(prob)
        S = Sweeper(D, build_graph(D, "face"))
        R = S.source_iterate(tol=1e-13)
        e2 = 0.0
        for d in range(D.M_dirs):
            psi_q = np.einsum("qm,em->eq", D.B, R["psi"][d])
            e2 += D.w[d] * _l2(D, psi_q - exact(D.xq, d)) ** 2
        errs.append(np.sqrt(e2))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] >= p + 1 - 0.2, (errs, orders)


def test_reoriented_elements_give_the_same_solution():
    base = si.make_config("2d_sine_q2_p1_s4", n=4, p=2)
    rot = si.make_config("2d_sine_q2_p1_s4", n=4, p=2, reorient_seed=7)
    assert np.any(rot.mesh.orient != 0)
    out = []
    for prob in (base, rot):
        D = Discretization(prob)
        R = Sweeper(D, build_graph(D, "face")).source_iterate(tol=1e-13)
        out.append(np.einsum("emn,en->e", D.M, R["phi"]))     # int_e phi, numbering-independent
    assert np.allclose(out[0], out[1], rtol=1e-11, atol=0)


# ---------------------------------------------------------------- 3D (hexahedra)

@pytest.mark.parametrize("p", [1, 2])
def test_affine_hex_mass_and_streaming_match_closed_form(p):
    """Affine hexes: M = |J| (M1 x M1 x M1) and S^k = |J| sum_j (J^-1)_jk D_j with D_j the 1D
    derivative matrix on axis j (tensor products from numpy polynomials, not the oracle)."""
    A = np.array([[1.1, 0.2, -0.1], [0.05, 0.9, 0.3], [-0.2, 0.1, 1.3]])
    n = 2
    prob = si.make_config("3d_twist_q2_p2_s8", n=n, p=p, sn=2)
    prob.mesh = si.structured_mesh((n, n, n), 2, affine_disp(A, np.array([0.1, -0.2, 0.05])))
    D = Discretization(prob)
    L = lagrange_poly_1d(gll_nodes(p))
    M1 = np.array([[integ01(a * b) for b in L] for a in L])
    D1 = np.array([[integ01(np.polyder(a) * b) for b in L] for a in L])
    J = A / n
    dJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    kron3 = lambda z, y, x: np.kron(z, np.kron(y, x))     # node m = i0 + (p+1) i1 + (p+1)^2 i2
    M_ex = dJ * kron3(M1, M1, M1)
    d = [kron3(M1, M1, D1), kron3(M1, D1, M1), kron3(D1, M1, M1)]
    S_ex = [dJ * sum(Jinv[j, k] * d[j] for j in range(3)) for k in range(3)]
    for e in range(D.E):
        assert np.allclose(D.M[e], M_ex, atol=1e-14)
        for k in range(3):
            assert np.allclose(D.S[e, k], S_ex[k], atol=1e-13)


@pytest.mark.parametrize("p,sn,reorient", [(1, 4, None), (2, 2, None), (2, 2, 5), (1, 4, 5)])
@pytest.mark.parametrize("weighting", ["unity", "face", "siginvface"])
def test_converged_lagged_si_equals_dense_coupled_solve_on_hexes(p, sn, reorient, weighting):
    """2x2x2 hexes twisted 60 degrees (cyclic: arcs are lagged), with and without a random
    renumbering of every element's nodes (orientation codes that swap the face axes)."""
    prob = si.make_config("3d_twist_q2_p2_s8", n=2, p=p, sn=sn, reorient_seed=reorient)
    if reorient is not None:
        assert np.any(prob.mesh.orient >= 4)
    D = Discretization(prob)
    G = build_graph(D, weighting)
    assert len(G["removed"]) > 0
    R = Sweeper(D, G).source_iterate(tol=1e-13)
    _, phi_ref = global_solve(D)
    assert np.abs(R["phi"] - phi_ref).max() <= 1e-10 * np.abs(phi_ref).max()


@pytest.mark.parametrize("p", [1, 2])
def test_pure_absorber_attenuation_converges_on_twisted_hexes(p):
    """exp(-sigma_t (x - x_in)/mu) solves the pure-absorber S_N equation on any domain; on the
    twisted (curved-faced, cyclic) hex meshes the L2 error must fall at order p + 1."""
    errs = []
    for n in (2, 4, 8):
        prob = si.make_config("3d_twist_q2_p2_s8", n=n, p=p, sn=2)
        prob, exact = attenuation(prob, sigma_t=2.0)
        D = Discretization(prob)
        R = Sweeper(D, build_graph(D, "face")).source_iterate(tol=1e-13)
        e2 = 0.0
        for d in range(D.M_dirs):
            psi_q = np.einsum("qm,em->eq", D.B, R["psi"][d])
            e2 += D.w[d] * _l2(D, psi_q - exact(D.xq, d)) ** 2
        errs.append(np.sqrt(e2))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] >= p + 1 - 0.2, (errs, orders)


@pytest.mark.parametrize("p", [1, 2])
def test_reoriented_hexes_give_the_same_solution(p):
    """Renumbering every element's local nodes by a rotation of the reference cube (orientation
    codes with the swap bit) must not change the physical solution: a wrong neighbour face-node
    map or orientation transform fails here.  The kink-aligned face rule follows the owner's face
    coordinates, so a renumbered face is integrated on other points: the two solutions agree to
    the rule's accuracy (measured 9e-9 at p = 1, 5e-10 at p = 2), not to rounding."""
    base = si.make_config("3d_twist_q2_p2_s8", n=3, p=p, sn=2)
    rot = si.make_config("3d_twist_q2_p2_s8", n=3, p=p, sn=2, reorient_seed=11)
    assert np.any(rot.mesh.orient >= 4) and np.any(rot.mesh.orient & 3)
    out = []
    for prob in (base, rot):
        prob, _ = attenuation(prob, sigma_t=1.5)
        prob.sigma_s = 0.5 * prob.sigma_t
        prob.q = np.ones_like(prob.q)
        D = Discretization(prob)
        R = Sweeper(D, build_graph(D, "face")).source_iterate(tol=1e-13)
        out.append(np.einsum("emn,en->e", D.M, R["phi"]))     # int_e phi, numbering-independent
    assert np.allclose(out[0], out[1], rtol=1e-7, atol=0)
