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


# Iterates a correction sample needs: phi_{it-2}, phi_{it-1}, phi_it for it in CORR_ITERS.
KEEP = frozenset(k for it in CORR_ITERS for k in (it - 2, it - 1, it))


def solve_history(ctx, precision=SN_PREC_FP64, tol=1e-11, max_iter=3000):
    """Plain source iteration from phi = 0: ({iteration: phi} for the iterates in KEEP and the
    last one, number of iterations)."""
    E, N = ctx._n_elem, ctx._N
    ctx.sn_si_begin()
    hist = {0: np.zeros((E, N))}
    n = 0
    for n in range(1, max_iter + 1):
        res, _ = ctx.sn_si_step(precision)
        if n in KEEP or res < tol:
            phi = np.zeros((E, N))
            ctx.sn_si_result(phi, None)
            hist[n] = phi
        if res < tol:
            break
    if n not in hist:
        hist[n] = np.zeros((E, N))
        ctx.sn_si_result(hist[n], None)
    return hist, n


def batched_histories(problems, start=None, group=128, precision=SN_PREC_FP64, tol=1e-11, max_iter=3000,
                      stream=None):
    """Source-iteration histories of many problems, solved group by group in batched launches.
    start(ctx) -> phi_0 (or None for 0).  Yields (ctx, {iteration: phi}, last iteration) with the
    iterates in KEEP and the last one (the converged flux); the context is closed after the
    caller's loop body."""
    from ._lib import Batch
    for g0 in range(0, len(problems), group):
        grp = problems[g0:g0 + group]
        ctxs = []
        for prob in grp:
            c = setup_problem(prob, stream=stream)
            c.sn_build_graph("face", 10)
            ctxs.append(c)
        phi0 = [None if start is None else start(c) for c in ctxs]
        b = Batch(ctxs, stream)
        b.sn_batch_si_begin(phi0)
        hist = [{0: np.zeros((c._n_elem, c._N)) if p is None else p} for c, p in zip(ctxs, phi0)]
        last = [0] * len(ctxs)
        done = [False] * len(ctxs)
        for n in range(1, max_iter + 1):
            res, _ = b.sn_batch_si_step(precision)
            for k, c in enumerate(ctxs):
                if done[k]:
                    continue
                last[k] = n
                done[k] = res[k] < tol
                if n in KEEP or done[k] or n == max_iter:
                    phi = np.zeros((c._n_elem, c._N))
                    c.sn_si_result(phi, None)
                    hist[k][n] = phi
            if all(done):
                break
        b.close()
        for c, h, n in zip(ctxs, hist, last):
            yield c, h, n
            c.close()


def corr_samples(ctx, hist, n):
    """Correction samples at the iterations in CORR_ITERS that precede the last iterate n - 1."""
    phi_inf = hist[n]
    xs, ts = [], []
    for it in CORR_ITERS:
        if it + 1 >= n:
            break
        x, t = ctx.sn_predictor_corr_data(hist[it - 2], hist[it - 1], hist[it], phi_inf)
        xs.append(x)
        ts.append(t[:, None])
    return xs, ts


def generate(problems, precision=SN_PREC_FP64, stream=None, group=128):
    """Stage-1 data (histories from phi = 0): features, initial-guess targets, correction samples."""
    xi, ti, xc, tc = [], [], [], []
    for ctx, hist, n in batched_histories(problems, None, group, precision, stream=stream):
        feat, _ref = ctx.sn_predictor_features()
        xi.append(feat)
        ti.append(ctx.sn_predictor_init_targets(hist[n]))
        x, t = corr_samples(ctx, hist, n)
        xc += x
        tc += t
    return dict(xi=np.concatenate(xi), ti=np.concatenate(ti), xc=np.concatenate(xc), tc=np.concatenate(tc))


def generate_stage2(problems, model, precision=SN_PREC_FP64, stream=None, group=128):
    """Correction samples from histories started at the initial-guess model's prediction (the
    iterates the correction model meets when the predictor is used)."""
    init, _corr, cfg = build(model, stream=stream)
    xc, tc = [], []
    for ctx, hist, n in batched_histories(problems, lambda c: c.sn_predictor_initial_phi(init, cfg), group,
                                          precision, stream=stream):
        x, t = corr_samples(ctx, hist, n)
        xc += x
        tc += t
    return dict(xc=np.concatenate(xc), tc=np.concatenate(tc))


def _norm(x):
    mean = x.mean(0).astype(np.float32)
    std = x.std(0).astype(np.float32)
    istd = np.where(std > 1e-12, 1.0 / np.maximum(std, 1e-12), 0.0).astype(np.float32)
    return mean, istd


def train_corr(model, data, epochs=40, batch_rows=4096, lr=2e-3, seed=0, stream=None):
    """Retrain the correction MLP on new samples (e.g. generate_stage2); returns the updated model."""
    rng = np.random.default_rng(seed)
    cm, cis = _norm(data["xc"])
    xc = (data["xc"] - cm) * cis
    pc = rng.permutation(len(xc))
    corr = MLP(SN_FEATURES + 2, 1, seed=seed + 2, stream=stream)
    lc = corr.sn_mlp_train(xc[pc], data["tc"][pc], epochs, batch_rows, lr, seed + 4)
    out = dict(model)
    out.update(corr_params=corr.get_params(), corr_mean=cm, corr_istd=cis, corr_loss=lc, rows_corr=len(xc))
    return out


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


def build(model, corr_start=5, corr_every=5, stream=None):
    """(init MLP, correction MLP, sn_predictor_cfg) ready for sn_source_iterate_learned.

    corr_start / corr_every: first iteration and interval of the correction attempts.  5 / 5 was
    picked from a small grid (start 4-7, interval 3-5, with and without the initial guess) on
    held-out problems (seeds 5002, 5004 at 16^3 and 5006 at 20^3): 119 iterations in total
    instead of 209 for plain source iteration; attempts from iteration 3 were rejected."""
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
