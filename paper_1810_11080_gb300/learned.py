"""Training and use of the learned flux predictor.

Training data come from solves of the method itself: this library's source iteration on seeded
synthetic problems.  Per-element features, initial-guess targets and correction samples are
computed by the library's predictor kernels; both MLPs are trained by the library's own
forward/backward/Adam kernels (sn_mlp_train).  This module only sequences those calls and
holds the arrays between them.
"""
import numpy as np

from ._lib import MLP, sn_predictor_cfg, SN_FEATURES, SN_PREC_FP64
from .problem import setup_problem

CORR_ITERS = (3, 4, 6, 8, 11, 15, 20, 27, 36, 48, 64)


def solve_history(ctx, precision=SN_PREC_FP64, tol=1e-11, max_iter=3000):
    """Plain source iteration from phi = 0, returning every iterate [phi_0 = 0, phi_1, ...]."""
    E, N = ctx._n_elem, ctx._N
    ctx.sn_si_begin()
    phis = [np.zeros((E, N))]
    for _ in range(max_iter):
        res, _ = ctx.sn_si_step(precision)
        phi = np.zeros((E, N))
        ctx.sn_si_result(phi, None)
        phis.append(phi)
        if res < tol:
            break
    return phis


def generate(problems, precision=SN_PREC_FP64, stream=None):
    """Features / targets of every training problem: returns dict of stacked float32 arrays."""
    xi, ti, xc, tc = [], [], [], []
    for prob in problems:
        ctx = setup_problem(prob, stream=stream)
        ctx._N = (prob.p + 1) ** prob.mesh.dim
        ctx.sn_build_graph("face", 10)
        phis = solve_history(ctx, precision)
        phi_inf = phis[-1]
        feat, _ref = ctx.sn_predictor_features()
        xi.append(feat)
        ti.append(ctx.sn_predictor_init_targets(phi_inf))
        for it in CORR_ITERS:
            if it + 1 >= len(phis) - 1:
                break
            x, t = ctx.sn_predictor_corr_data(phis[it - 2], phis[it - 1], phis[it], phi_inf)
            xc.append(x)
            tc.append(t[:, None])
        ctx.close()
    return dict(xi=np.concatenate(xi), ti=np.concatenate(ti), xc=np.concatenate(xc), tc=np.concatenate(tc))


def _norm(x):
    mean = x.mean(0).astype(np.float32)
    std = x.std(0).astype(np.float32)
    istd = np.where(std > 1e-12, 1.0 / np.maximum(std, 1e-12), 0.0).astype(np.float32)
    return mean, istd


def train(data, epochs=40, batch_rows=4096, lr=2e-3, seed=0, stream=None):
    """Train the initial-guess and correction MLPs; returns a model dict (params + normalisation)."""
    rng = np.random.default_rng(seed)
    im, iis = _norm(data["xi"])
    cm, cis = _norm(data["xc"])
    xi = (data["xi"] - im) * iis
    xc = (data["xc"] - cm) * cis
    pi = rng.permutation(len(xi))
    pc = rng.permutation(len(xc))
    n_out = data["ti"].shape[1]
    init = MLP(SN_FEATURES, n_out, seed=seed + 1, stream=stream)
    corr = MLP(SN_FEATURES + 2, 1, seed=seed + 2, stream=stream)
    li = init.sn_mlp_train(xi[pi], data["ti"][pi], epochs, batch_rows, lr, seed + 3)
    lc = corr.sn_mlp_train(xc[pc], data["tc"][pc], epochs, batch_rows, lr, seed + 4)
    return dict(init_params=init.get_params(), corr_params=corr.get_params(), n_out=n_out, init_mean=im,
                init_istd=iis, corr_mean=cm, corr_istd=cis, init_loss=li, corr_loss=lc,
                rows_init=len(xi), rows_corr=len(xc))


def save(model, path):
    np.savez(path, **{k: np.asarray(v) for k, v in model.items()})


def load(path):
    z = np.load(path)
    return {k: z[k] for k in z.files}


def build(model, corr_start=3, corr_every=4, stream=None):
    """(init MLP, correction MLP, sn_predictor_cfg) ready for sn_source_iterate_learned."""
    n_out = int(model["n_out"])
    init = MLP(SN_FEATURES, n_out, stream=stream)
    init.set_params(model["init_params"])
    corr = MLP(SN_FEATURES + 2, 1, stream=stream)
    corr.set_params(model["corr_params"])
    cfg = sn_predictor_cfg()
    cfg.init_mean[:] = [float(v) for v in model["init_mean"]]
    cfg.init_istd[:] = [float(v) for v in model["init_istd"]]
    cfg.corr_mean[:] = [float(v) for v in model["corr_mean"]]
    cfg.corr_istd[:] = [float(v) for v in model["corr_istd"]]
    cfg.corr_start = corr_start
    cfg.corr_every = corr_every
    return init, corr, cfg
