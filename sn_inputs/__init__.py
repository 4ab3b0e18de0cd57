"""Seeded synthetic inputs for the S_N sweep: curved meshes, angular quadrature sets, materials.

This package generates *problem data* only.  It holds none of the discretisation,
graph or sweep arithmetic of the method; both the CPU oracle and the GPU library
consume what it produces.

Mesh convention (shared by every consumer, and by the C ABI):

* Reference element = [0,1]^dim.  Geometry is a Q_r Lagrange map whose control
  points sit on the *equispaced* reference nodes t_a = a/r (eq. 1 of the paper's
  Sec. 2: x_{e,m} = T_e(xi_m)).  Control point m = a + (r+1) b (+ (r+1)^2 c), x fastest.
* Local faces f = 2*axis + side: side 0 is xi_axis = 0, side 1 is xi_axis = 1.
  A face's own coordinates (s0[, s1]) are the remaining reference axes in
  increasing order.
* face_nbr[e][f]  = neighbour element or -1 (domain boundary).
  nbr_face[e][f]  = the neighbour's local face index.
  orient[e][f]    = map from e's face coordinates to the neighbour's:
                    bit0 swap (s0,s1); bit1 flip first result (1-t); bit2 flip second.
"""
from .mesh import (Mesh, structured_mesh, connectivity_from_nodes, reorient_elements,
                   disp_sine_2d, disp_random_smooth, disp_twist, disp_random_smooth_3d)
from .quadrature import level_symmetric
from .configs import make_config, CONFIGS, batch_problems

__all__ = ["Mesh", "structured_mesh", "connectivity_from_nodes", "reorient_elements",
           "disp_sine_2d", "disp_random_smooth", "disp_twist", "disp_random_smooth_3d",
           "level_symmetric", "make_config", "CONFIGS", "batch_problems"]
