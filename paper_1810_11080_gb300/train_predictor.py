"""Train the learned flux predictor for the 3D Q2 p=2 S12 workload family (random smooth
perturbation 0.1 h, log-normal sigma_t, scattering ratio 0.99, q = 1, vacuum) on solves the
method itself generates, and save the model.

    python -m paper_1810_11080_gb300.train_predictor --solves 2000 --n 8 --out <path.npz>

Training problems use seeds 1000, 1002, ... (mesh seed s, material seed s + 1); evaluation
problems elsewhere use seeds >= 5000.  Stage 1 trains the initial-guess model on histories from
phi = 0; stage 2 retrains the correction model on histories started at the predicted flux.
"""
import argparse
import json
import time

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--solves", type=int, default=2000)
    ap.add_argument("--n", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--precision", default="mixed_ds", choices=["fp64", "mixed_ds"],
                    help="sweep form of the training solves (double-single: ~1e-13 from FP64, faster)")
    ap.add_argument("--out", required=True)
    args = ap.parse_args()
    import torch
    import sn_inputs as si
    from . import learned
    from ._lib import SN_PREC_FP64, SN_PREC_MIXED_DS
    prec = SN_PREC_FP64 if args.precision == "fp64" else SN_PREC_MIXED_DS
    stream = torch.cuda.Stream()
    t0 = time.time()
    probs = [si.make_config("3d_smooth_q2_p2_s12", n=args.n, seed=1000 + 2 * k) for k in range(args.solves)]
    # stage 1: histories from phi = 0 -> initial-guess model (and a first correction model)
    data = learned.generate(probs, precision=prec, stream=stream.cuda_stream)
    t1 = time.time()
    model = learned.train(data, epochs=args.epochs, stream=stream.cuda_stream)
    # stage 2: histories started at the predicted flux -> the correction model it will meet
    t2 = time.time()
    data2 = learned.generate_stage2(probs, model, precision=prec, stream=stream.cuda_stream)
    t3 = time.time()
    model = learned.train_corr(model, data2, epochs=args.epochs, stream=stream.cuda_stream)
    t4 = time.time()
    model["train_solves"] = args.solves
    model["train_n"] = args.n
    model["train_precision"] = args.precision
    learned.save(model, args.out)
    print(json.dumps({"solves": args.solves, "n": args.n, "rows_init": int(model["rows_init"]),
                      "rows_corr": int(model["rows_corr"]), "init_loss": float(model["init_loss"]),
                      "corr_loss": float(model["corr_loss"]), "precision": args.precision,
                      "gen1_s": t1 - t0, "train1_s": t2 - t1, "gen2_s": t3 - t2, "train2_s": t4 - t3}))


if __name__ == "__main__":
    main()
