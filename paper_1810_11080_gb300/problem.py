"""Upload a problem description (mesh, quadrature, materials) into a Context."""
import numpy as np

from ._lib import Context


def setup_problem(prob, device=0, stream=None, face_subdiv=2, ctx=None):
    """Create (or reuse) a Context and pass it the arrays of an sn_inputs Problem."""
    ctx = ctx or Context(device, stream)
    m = prob.mesh
    simplex = getattr(m, "simplex", False)
    setm = ctx.sn_set_mesh_simplex if simplex else ctx.sn_set_mesh
    setm(m.dim, m.n_elem, m.r, np.ascontiguousarray(m.ctrl, dtype=np.float64),
         np.ascontiguousarray(m.face_nbr, dtype=np.int64), np.ascontiguousarray(m.nbr_face, dtype=np.int32),
         np.ascontiguousarray(m.orient, dtype=np.int32))
    ctx.sn_set_discretization(prob.p, face_subdiv)
    if simplex:
        ctx._N = (prob.p + 1) * (prob.p + 2) // 2 if m.dim == 2 else (prob.p + 1) * (prob.p + 2) * (prob.p + 3) // 6
    else:
        ctx._N = (prob.p + 1) ** m.dim
    ctx.sn_set_quadrature(np.ascontiguousarray(prob.omega, dtype=np.float64),
                          np.ascontiguousarray(prob.w, dtype=np.float64))
    arr = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
    ctx.sn_set_materials(arr(prob.sigma_t), arr(prob.sigma_s), arr(prob.q), arr(prob.q_dir), arr(prob.psi_inc))
    return ctx
