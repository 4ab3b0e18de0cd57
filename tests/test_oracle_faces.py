"""Pins of the oracle's 3D face quadrature for the kinked upwind integrands (Sec. 2, last
paragraph: max(+-Omega.n, 0) u_m u_n is only piecewise smooth where Omega.n changes sign).

- root isolation against numpy's companion-matrix roots;
- on faces extruded from a 2D curve the block factorises into the exact 1D integral split at the
  roots (numpy polynomial integration) times the 1D mass matrix: the rule must reproduce it;
- on twisted faces the rule converges quickly as the composite subdivision K doubles, far faster
  than the unsplit composite rule does."""
import numpy as np
import pytest

import sn_inputs as si
from oracle.basis import gauss_legendre, gll_nodes
from oracle.dg import (face_rule_3d, face_basis, coupling_block, pos, dot_omega, poly_from_samples,
                       roots_01)
from oracle.geometry import face_normal


@pytest.mark.parametrize("deg", [1, 2, 3, 5])
def test_roots_01_matches_numpy_roots(deg):
    rng = np.random.default_rng(deg)
    xs = np.array([k / deg for k in range(deg + 1)])
    for _ in range(40):
        rts = rng.uniform(-0.5, 1.5, size=deg)
        vals = rng.uniform(0.5, 2.0) * np.prod(xs[:, None] - rts[None, :], axis=1)
        got = np.array([x for x in (r.item() for r in roots_01(poly_from_samples(vals[None, :]))) if x < 1.0])
        want = np.sort([x for x in rts if 1e-9 < x < 1 - 1e-9])
        # roots closer than ~1e-6 to each other or to 0/1 are not generated above with any weight
        assert len(got) == len(want), (rts, got)
        np.testing.assert_allclose(got, want, atol=1e-9)


def _lagrange_polys(nodes):
    out = []
    for j in range(len(nodes)):
        y = np.zeros(len(nodes))
        y[j] = 1.0
        out.append(np.poly1d(np.polyfit(nodes, y, len(nodes) - 1)))
    return out


def _exact_split_integral(gpoly, L):
    """int_0^1 max(-g(s), 0) l_i(s) l_j(s) ds exactly: numpy roots of g, numpy polyint per piece."""
    rts = sorted(x.real for x in np.roots(gpoly.coeffs) if abs(x.imag) < 1e-12 and 0.0 < x.real < 1.0)
    brk = [0.0] + rts + [1.0]
    B = np.zeros((len(L), len(L)))
    for lo, hi in zip(brk[:-1], brk[1:]):
        mid = 0.5 * (lo + hi)
        if gpoly(mid) >= 0.0:
            continue
        for i in range(len(L)):
            for j in range(len(L)):
                P = np.polyint(-gpoly * L[i] * L[j])
                B[i, j] += P(hi) - P(lo)
    return B


def test_extruded_faces_match_the_exact_split_integral():
    """2D sine-perturbed quads extruded along z: on an x- or y-face, Omega.n depends on the
    in-plane face coordinate only, so the coupling block is kron(M1D(s1), B1D(s0))."""
    n, p, r = 3, 2, 2
    base = si.disp_sine_2d(0.12)

    def disp(X):
        d = np.zeros_like(X)
        d[:, :2] = base(X[:, :2])
        return d
    mesh = si.structured_mesh((n, n, n), r, disp)
    om, w = si.level_symmetric(4, 3)
    gll = gll_nodes(p)
    L = _lagrange_polys(gll)
    M1 = np.array([[np.polyint(a * b)(1.0) - np.polyint(a * b)(0.0) for b in L] for a in L])
    kinked = 0
    for f in (1, 3):       # x- and y-faces: face coordinate s1 runs along z
        ctrl = mesh.ctrl
        s0, s1, wq, g = face_rule_3d(ctrl, r, f, om, p + r, 2)
        phi = face_basis(gll, 3, s0, s1)
        B = coupling_block(pos(-g) * wq, phi, phi)
        xs = np.linspace(0.0, 1.0, 2 * r)                    # g is a polynomial of degree 2r - 1 in s0
        nv = face_normal(ctrl, r, f, xs, np.full_like(xs, 0.37))     # [E, 4, 3]
        for e in range(mesh.n_elem):
            for d in range(len(w)):
                gv = nv[e] @ om[d]
                gpoly = np.poly1d(np.polyfit(xs, gv, 2 * r - 1))
                kinked += int(np.any(np.sign(gv) != np.sign(gv[0])))
                ref = np.kron(M1, _exact_split_integral(gpoly, L))
                scale = max(np.abs(ref).max(), np.abs(gv).max() * 1e-3)
                assert np.abs(B[e, d] - ref).max() <= 1e-12 * scale, (f, e, d)
    assert kinked > 0          # the mesh has faces where the integrand is kinked


def _composite_blocks(ctrl, r, f, om, nf, K, gll):
    t, wt = gauss_legendre(nf)
    pts = [((u + t[i]) / K, (v + t[j]) / K, (wt[i] / K) * (wt[j] / K))
           for v in range(K) for u in range(K) for j in range(nf) for i in range(nf)]
    s0, s1, wl = (np.array(x) for x in zip(*pts))
    nv = face_normal(ctrl, r, f, s0, s1)
    g = dot_omega([om[:, k][None, :, None] for k in range(3)], nv[:, None])
    F, D, P = ctrl.shape[0], om.shape[0], len(s0)
    phi = face_basis(gll, 3, np.broadcast_to(s0, (F, D, P)), np.broadcast_to(s1, (F, D, P)))
    return coupling_block(pos(-g) * wl, phi, phi)


def test_twisted_faces_converge_as_the_subdivision_doubles():
    prob = si.make_config("3d_twist_q2_p2_s8", n=4)
    mesh = prob.mesh
    om = np.asarray(prob.omega)
    gll = gll_nodes(2)
    sel = [e for e in range(mesh.n_elem) if mesh.face_nbr[e, 1] >= 0][:8]
    ctrl = mesh.ctrl[sel]
    Bk = {}
    for K in (2, 4, 8):
        s0, s1, w, g = face_rule_3d(ctrl, 2, 1, om, 4, K)
        phi = face_basis(gll, 3, s0, s1)
        Bk[K] = coupling_block(pos(-g) * w, phi, phi)
    scale = np.abs(Bk[8]).max()
    d24 = np.abs(Bk[2] - Bk[8]).max() / scale
    d48 = np.abs(Bk[4] - Bk[8]).max() / scale
    comp = np.abs(_composite_blocks(ctrl, 2, 1, om, 4, 2, gll) - Bk[8]).max() / scale
    assert d24 < 3e-6 and d48 < 1e-7, (d24, d48)
    assert comp > 30 * d24                   # the unsplit composite rule at K = 2 is far less accurate
