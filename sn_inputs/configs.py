"""The benchmark workloads as seeded synthetic problems.

Each config mirrors one of the five workload descriptions of this project
(2D sine-perturbed Q2 16x16 S4; 2D random-smooth Q3 128x128 S8; 3D twisted Q2 32^3 S8;
a batch of 256 uneven 2D problems; 3D random-smooth Q2 48^3 S12).  `n` overrides
the grid size so that the same recipe yields small test cases.
"""
from dataclasses import dataclass
import numpy as np
from .mesh import structured_mesh, disp_sine_2d, disp_random_smooth, disp_twist, disp_random_smooth_3d
from .quadrature import level_symmetric


@dataclass
class Problem:
    name: str
    mesh: object
    p: int
    omega: np.ndarray        # [M][3]
    w: np.ndarray            # [M]
    sigma_t: np.ndarray      # [n_elem]
    sigma_s: np.ndarray      # [n_elem]
    q: np.ndarray            # [n_elem][N] nodal isotropic source
    q_dir: np.ndarray = None     # [M][n_elem][N] nodal direction-dependent source, or None
    psi_inc: np.ndarray = None   # [M][n_bdr_faces][N_f] nodal incident flux, or None (vacuum)
    sn_order: int = 0

    @property
    def dim(self):
        return self.mesh.dim

    @property
    def n_dofs(self):
        if getattr(self.mesh, "simplex", False) and self.mesh.dim == 3:
            return (self.p + 1) * (self.p + 2) * (self.p + 3) // 6
        if getattr(self.mesh, "simplex", False):
            return (self.p + 1) * (self.p + 2) // 2
        return (self.p + 1) ** self.mesh.dim


CONFIGS = {
    "2d_sine_q2_p1_s4": dict(dim=2, n=16, r=2, p=1, sn=4),
    "2d_smooth_q3_p3_s8": dict(dim=2, n=128, r=3, p=3, sn=8),
    "3d_twist_q2_p2_s8": dict(dim=3, n=32, r=2, p=2, sn=8),
    "3d_smooth_q2_p2_s12": dict(dim=3, n=48, r=2, p=2, sn=12),
}


def make_config(name, n=None, sn=None, p=None, reorient_seed=None, seed=None):
    """Build one workload (optionally at a reduced grid size n).  seed replaces the mesh and
    material seeds of the random workloads by (seed, seed + 1)."""
    c = dict(CONFIGS[name])
    if n is not None:
        c["n"] = n
    if sn is not None:
        c["sn"] = sn
    if p is not None:
        c["p"] = p
    dim, n, r, p_, sn_ = c["dim"], c["n"], c["r"], c["p"], c["sn"]
    h = 1.0 / n
    if name == "2d_sine_q2_p1_s4":
        mesh = structured_mesh((n, n), r, disp_sine_2d(0.05))
        ne = mesh.n_elem
        st = np.ones(ne)
        ss = 0.5 * np.ones(ne)
    elif name == "2d_smooth_q3_p3_s8":
        mesh = structured_mesh((n, n), r, disp_random_smooth(h, seed=11 if seed is None else seed))
        ne = mesh.n_elem
        rng = np.random.default_rng(12 if seed is None else seed + 1)
        st = rng.uniform(0.5, 5.0, size=ne)
        ss = 0.9 * st
    elif name == "3d_twist_q2_p2_s8":
        mesh = structured_mesh((n, n, n), r, disp_twist(np.pi / 3))
        ne = mesh.n_elem
        st = np.ones(ne)
        ss = 0.8 * np.ones(ne)
    elif name == "3d_smooth_q2_p2_s12":
        mesh = structured_mesh((n, n, n), r, disp_random_smooth_3d(h, seed=41 if seed is None else seed))
        ne = mesh.n_elem
        rng = np.random.default_rng(42 if seed is None else seed + 1)
        st = np.exp(rng.normal(0.0, 1.0, size=ne))
        ss = 0.99 * st
    else:
        raise KeyError(name)
    if reorient_seed is not None:
        from .mesh import reorient_elements
        mesh = reorient_elements(mesh, reorient_seed)
    om, w = level_symmetric(sn_, dim)
    N = (p_ + 1) ** dim
    q = np.ones((mesh.n_elem, N))
    return Problem(name=name, mesh=mesh, p=p_, omega=om, w=w, sigma_t=st, sigma_s=ss, q=q, sn_order=sn_)


def batch_problems(count=256, seed=31, nmin=8, nmax=64):
    """Many independent uneven 2D problems: n ~ U{nmin..nmax}, p ~ U{1,2,3}, r ~ U{2,3},
    S_N ~ U{4,6,8}, sigma_t ~ U[0.1,10] per element, scattering ratio c ~ U[0.5,0.95] per problem.
    Problem i draws from numpy PCG64 substream (seed, i)."""
    out = []
    for i in range(count):
        rng = np.random.default_rng([seed, i])
        n = int(rng.integers(nmin, nmax + 1))
        p = int(rng.integers(1, 4))
        r = int(rng.integers(2, 4))
        sn = int(rng.choice([4, 6, 8]))
        c = float(rng.uniform(0.5, 0.95))
        mseed = int(rng.integers(0, 2**31 - 1))
        mesh = structured_mesh((n, n), r, disp_random_smooth(1.0 / n, seed=mseed))
        st = rng.uniform(0.1, 10.0, size=mesh.n_elem)
        om, w = level_symmetric(sn, 2)
        N = (p + 1) ** 2
        out.append(Problem(name=f"batch{i}", mesh=mesh, p=p, omega=om, w=w, sigma_t=st, sigma_s=c * st,
                           q=np.ones((mesh.n_elem, N)), sn_order=sn))
    return out


def annulus_problem(n_rho, n_theta, r, p, sn=4):
    """Quarter annulus rho in [0.5, 1] (curved inner and outer boundaries) as an n_rho x n_theta
    Q_r mesh, DG order p, level-symmetric S_sn, sigma_t = 1, sigma_s = 0.5, q = 1 (the materials
    and sources are replaced by sn_inputs.mms.annulus_mms for manufactured-solution runs)."""
    from .mesh import annulus_mesh
    mesh = annulus_mesh(n_rho, n_theta, r)
    om, w = level_symmetric(sn, 2)
    ne = mesh.n_elem
    N = (p + 1) ** 2
    return Problem(name=f"annulus_{n_rho}x{n_theta}_r{r}_p{p}", mesh=mesh, p=p, omega=om, w=w,
                   sigma_t=np.ones(ne), sigma_s=0.5 * np.ones(ne), q=np.ones((ne, N)), sn_order=sn)


def straightened_problem(prob, n_ref, p=1):
    """The same problem on the straightened mesh (sn_inputs.mesh.straighten: every element divided
    n_ref times per axis, straight-sided Q_1 sub-elements) with DG order p (low order by default)."""
    from .mesh import straighten
    mesh = straighten(prob.mesh, n_ref)
    ne = mesh.n_elem
    N = (p + 1) ** mesh.dim
    return Problem(name=prob.name + f"_straight{n_ref}", mesh=mesh, p=p, omega=prob.omega, w=prob.w,
                   sigma_t=np.ones(ne), sigma_s=0.5 * np.ones(ne), q=np.ones((ne, N)), sn_order=prob.sn_order)


def triangle_problem(n, r, p, sn=4, amp=0.05, rotate_seed=None):
    """n x n cells of [0,1]^2 cut into 2 n^2 counterclockwise triangles with P_r geometry,
    interior nodes displaced by amp sin(2 pi x) sin(2 pi y) on both coordinates (zero on the
    boundary), DG order p (P_p, (p+1)(p+2)/2 unknowns), S_sn, sigma_t = 1, sigma_s = 0.5, q = 1.
    rotate_seed renumbers the triangles' local nodes by random rotations."""
    from .mesh import triangle_mesh, rotate_triangles
    mesh = triangle_mesh((n, n), r, disp_sine_2d(amp))
    if rotate_seed is not None:
        mesh = rotate_triangles(mesh, rotate_seed)
    om, w = level_symmetric(sn, 2)
    ne = mesh.n_elem
    N = (p + 1) * (p + 2) // 2
    return Problem(name=f"tri_{n}_r{r}_p{p}_s{sn}", mesh=mesh, p=p, omega=om, w=w, sigma_t=np.ones(ne),
                   sigma_s=0.5 * np.ones(ne), q=np.ones((ne, N)), sn_order=sn)


def tet_problem(n, p, sn=4, rotate_seed=None, twist=0.0, r=1, bubble=0.0):
    """The unit cube as n^3 cubes of six tetrahedra each (6 n^3 elements), geometry order r (1:
    straight-sided; 2: P_2 geometry with curved edges and faces), DG order p (1 or 2: 4 or 10
    unknowns), S_sn, sigma_t = 1, sigma_s = 0.5, q = 1.  rotate_seed renumbers the tetrahedra's
    vertices by random even permutations; twist rotates the nodes about the cube's vertical axis
    by twist * z radians (a twisted column, whose sweep graphs have cycles for large enough
    twist); bubble moves the nodes by disp_bubble_3d(bubble) (curved interior, the domain stays
    the cube)."""
    from .mesh import tet_mesh, rotate_tets, disp_bubble_3d
    disp = None
    if twist and bubble:
        raise ValueError("twist or bubble, not both")
    if twist:
        disp = disp_twist(twist)
    elif bubble:
        disp = disp_bubble_3d(bubble)
    mesh = tet_mesh(n, disp, r=r)
    if rotate_seed is not None:
        mesh = rotate_tets(mesh, rotate_seed)
    om, w = level_symmetric(sn, 3)
    ne = mesh.n_elem
    N = (p + 1) * (p + 2) * (p + 3) // 6
    return Problem(name=f"tet_{n}_r{r}_p{p}_s{sn}" + (f"_tw{twist:g}" if twist else "") + (f"_b{bubble:g}" if bubble else ""),
                   mesh=mesh, p=p, omega=om, w=w, sigma_t=np.ones(ne),
                   sigma_s=0.5 * np.ones(ne), q=np.ones((ne, N)), sn_order=sn)
