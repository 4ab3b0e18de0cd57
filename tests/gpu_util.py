"""Helpers shared by the GPU parity tests: run the oracle and the CUDA library on the same
seeded problem."""
import numpy as np

from oracle.dg import Discretization
from oracle.graph import build_graph
from oracle.sweep import Sweeper


def oracle_disc(prob):
    if getattr(prob.mesh, "simplex", False) and prob.mesh.dim == 3:
        from oracle.simplex3 import TetDiscretization
        return TetDiscretization(prob)
    if getattr(prob.mesh, "simplex", False):
        from oracle.simplex import SimplexDiscretization
        return SimplexDiscretization(prob)
    return Discretization(prob)


def oracle_graph(prob, weighting="face", exact_max=10):
    disc = oracle_disc(prob)
    return disc, build_graph(disc, weighting, exact_max)


def gpu_ctx(prob, weighting="face", exact_max=10, stream=None):
    import torch
    import paper_1810_11080_gb300 as g
    if stream is None:
        stream = torch.cuda.Stream()
    ctx = g.setup_problem(prob, device=0, stream=stream.cuda_stream)
    ctx._torch_stream = stream
    stats = ctx.sn_build_graph(weighting, exact_max)
    return ctx, stats


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def random_state(prob, seed=0):
    rng = np.random.default_rng(seed)
    N = (prob.p + 1) ** prob.mesh.dim
    M = len(prob.w)
    E = prob.mesh.n_elem
    phi = rng.uniform(0.5, 2.0, size=(E, N))
    psi_old = rng.uniform(0.0, 1.0, size=(M, E, N))
    return phi, psi_old
