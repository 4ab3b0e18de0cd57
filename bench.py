"""Benchmark: lagged S_N transport sweep inside source iteration on one GB300.

Workload (default): 2D 128x128 curved quad mesh, Q3 geometry with seeded smooth perturbation
(amplitude 0.1 h), DG p = 3 (16 unknowns/element), level-symmetric S8 (40 directions),
sigma_t ~ U[0.5, 5] per element, scattering ratio 0.9, q = 1, vacuum boundaries:
16384 x 40 = 655,360 element-direction updates per sweep.

A step is one source iteration through the C ABI (sn_si_step): the lagged sweep over every
level and direction, then the fused scalar-flux moment + scattering-source update + residual.
value = element-direction updates per second over the timed steps, in the paper's arithmetic
(FP64 form).  The mixed forms (FP32 LU + one refinement) are measured beside it: their
updates/s and their wall time to the same 1e-8 scalar-flux residual.

--impl reference times the CPU FP64 oracle (the plain numpy restatement of the method) on a
bounded sample of the same workload, on all host cores (one direction per process).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sweep elem-direction updates/s and time-to-1e-8 residual vs plain FP64 sweep"
WORKLOAD = "2d_smooth_q3_p3_s8"
WORKLOAD_DESC = ("2D 128x128 quads on [0,1]^2, Q3 geometry, seeded smooth perturbation 0.1h, DG p=3 (16 dofs), "
                 "S8 (40 dirs), sigma_t~U[0.5,5], c=0.9, q=1, vacuum; 655360 updates/sweep")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 pipe peak: 152 SMs x 2 DFMA/clk/SM (measured 1/64 of the FP32 FMA rate on GB300) x 2 flop
# x SM clock.  At the 2070 MHz maximum clock: 1.259 TFLOP/s; measured with the DFMA/FFMA
# microbenchmark bench_fp_peaks.cu: 1.20 TFLOP/s FP64 and 75.0 TFLOP/s FP32.
FP64_PEAK_TFLOPS = 1.20

DTYPES = {"fp64": "f64", "mixed": "f32+f64", "mixed_ds": "f32+f32x2+f64", "fp64_inv": "f64", "ds_inv": "f32x2+f64"}
PRECISION_DESC = {
    "fp64": "FP64 assembly, LU and solve",
    "mixed": "FP32 assembly and LU, one refinement with an FP64 residual",
    "mixed_ds": "FP32 LU, one refinement; row and residual in double-single (FP32 pairs), FP64 right-hand side",
    "fp64_inv": "FP64; local inverses formed once per problem (Gauss-Jordan, partial pivoting), applied each sweep",
    "ds_inv": "local inverses formed once per problem in FP64, stored as FP32 (hi, lo) pairs and applied in "
              "double-single arithmetic each sweep",
}


# Algorithmic work of one (element, direction) update of the method, per workload shape (dim, p):
# local assembly from the direction-independent element matrices, inflow face terms, LU and the two
# triangular solves (flops); the angular flux written, the inflow traces read and the element
# factors and source amortised over the directions (bytes).  These are the per-update figures the
# roofline fractions are computed from, whatever the form's own instruction count.
ALG_WORK = {
    (2, 1): {"flops": 250.0, "bytes": 200.0},        # 16x16 p=1 S4 (latency bound)
    (2, 3): {"flops": 5800.0, "bytes": 350.0},       # 128x128 p=3 S8
    (3, 2): {"flops": 35000.0, "bytes": 770.0},      # 32^3 p=2 S8 / 48^3 p=2 S12
}


def alg_work(dim, p):
    return ALG_WORK.get((dim, p), {"flops": None, "bytes": None})


def inv_alg_bytes(dim, p, simplex=False):
    """DRAM bytes one update of a stored-inverse form must move: its record, read once per sweep
    and far larger than L2 -- the inverse (N^2 entries) and one block per inflow face (2D: the
    folded N x Nf block, 3D: the Nf x Nf block; dim inflow faces on average for quadrilaterals
    and hexahedra, 1.5 for triangles, 2 for tetrahedra) -- plus the angular flux written (N) and
    about N entries of traces and source; 8 bytes per entry."""
    if simplex and dim == 3:
        N, Nf, faces = (p + 1) * (p + 2) * (p + 3) // 6, (p + 1) * (p + 2) // 2, 2.0
    elif simplex:
        N, Nf, faces = (p + 1) * (p + 2) // 2, p + 1, 1.5
    else:
        N, Nf, faces = (p + 1) ** dim, (p + 1) ** (dim - 1), dim
    blk = N * Nf if dim == 2 else Nf * Nf
    return 8.0 * (N * N + faces * blk + 2 * N)


class ClockSampler:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, device_index=0):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or not parts[1].replace(".", "").isdigit():
                continue
            if int(parts[0]) != device_index:
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(rows[0][2]), "samples": len(rows),
                "reasons": sorted(reasons)}


def make_problem(n=None):
    import sn_inputs as si
    return si.make_config(WORKLOAD, n=n)


def max_over_ranks(value):
    """Largest value over all ranks (the job is as slow as its slowest replica)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world_size, units_per_rank, steps, ms_max):
    """Whole-job units per second: every replica processes units_per_rank per step."""
    return world_size * units_per_rank * steps / (ms_max / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def ds_fp32_issued_flops_per_update(dim, p, inflow_faces):
    """FP32 flops the double-single form issues per update (its implementation's work, not the
    method's): row assembly in double-single ((dim+1) products of 7 flops, dim sums of 8 per
    entry), inflow-face blocks, FP32 Gauss-Jordan 2N^3/3, two inverse applications 4N^2,
    double-single residual 12 N^2."""
    N = (p + 1) ** dim
    Nf = (p + 1) ** (dim - 1)
    row = N * N * ((dim + 1) * 7 + dim * 8)
    faces = inflow_faces * Nf * Nf * (dim * 7 + (dim - 1) * 8 + 8)
    return row + faces + 2.0 * N ** 3 / 3 + 4 * N * N + 12 * N * N


FP32_PEAK_TFLOPS = 75.0

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the dominant sweep
# kernel of a form, from one ncu capture of this workload.  Valid only for the kernel sources it
# was taken on (SHA-256 of the files below); any later change to them reports null.
KERNEL_SOURCES = ["paper_1810_11080_gb300/csrc/" + f for f in
                  ("sweep.cu", "sweep_inv.cu", "sweep_kernels.cuh", "sweep_body.cuh", "inverse_body.cuh",
                   "devmath.cuh", "common.h")]
TRAFFIC = {
    # one launch = one sweep: the whole launch captured (351.7 MB read + 153.7 MB written)
    ("fp64", "dataflow"): {"bytes_per_launch": 505401856, "capture": "ncu --metrics dram__bytes_read.sum,"
                           "dram__bytes_write.sum, sweep_flow_kernel<2,3,0>, first timed launch",
                           "sources_sha256": "a99cfce41db0ee1b51e1e0d181ee4ac18d07fdd21f5ef51fb9b414ab79756f24"},
    # three mid-sweep level launches (5,000-5,080 pairs, 18.3-18.5 MB read, writes still in L2 at the
    # end of each launch), scaled to the sweep's average level of 2,570 pairs at 3,653 bytes per pair
    ("ds_inv", "levels"): {"bytes_per_launch": 9389154, "capture": "ncu --metrics dram__bytes_read.sum,"
                           "dram__bytes_write.sum, el_level_kernel<TensorEl<2,3>,4>, levels 128-130 scaled per pair",
                           "sources_sha256": "a99cfce41db0ee1b51e1e0d181ee4ac18d07fdd21f5ef51fb9b414ab79756f24"},
}

def kernel_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_for(kind, schedule):
    """(bytes per launch, capture id) of the form's kernel on the given schedule, or (None, None)."""
    t = TRAFFIC.get((kind, schedule))
    if t is None or t["sources_sha256"] != kernel_sources_sha256():
        return None, None
    return t["bytes_per_launch"], t["capture"]


def run_gpu(args):
    import torch
    import paper_1810_11080_gb300 as g

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    if args.quick and args.quick_simplex:
        leg = run_triangles if args.quick_simplex == "triangles" else run_tets
        return {"metric": METRIC, "quick": True, "leg": args.quick_simplex, "result": leg(g, torch, args)}
    if args.quick and args.quick_workload:
        import sn_inputs as si
        prob = si.make_config(args.quick_workload)
    else:
        prob = make_problem()
    dim, E, N, M = prob.mesh.dim, prob.mesh.n_elem, (prob.p + 1) ** prob.mesh.dim, len(prob.w)
    updates = E * M
    stream = torch.cuda.Stream(device=local)
    ctx = g.setup_problem(prob, device=local, stream=stream.cuda_stream)
    t0 = time.time()
    gstats = ctx.sn_build_graph("face", 10)
    t_graph = time.time() - t0

    def set_schedule(prec):
        """Launch schedule of a form: the library's autotuner (levels or dataflow, CTAs per SM),
        or the one named by --launch."""
        if args.launch == "auto":
            mode, bps = ctx.sn_autotune(prec)
        else:
            mode, bps = (g.SN_LAUNCH_DATAFLOW if args.launch == "dataflow" else g.SN_LAUNCH_LEVELS), 0
            ctx.sn_set_launch(mode, bps)
        return {"mode": "dataflow" if mode == g.SN_LAUNCH_DATAFLOW else "levels", "blocks_per_sm": bps}

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    def timed_steps(prec):
        sched = set_schedule(prec)
        ctx.sn_si_begin(None)
        for _ in range(args.warmup):
            ctx.sn_si_step(prec)
        l0 = ctx.sn_kernel_launches()
        clocks = ClockSampler()
        clocks.start()
        barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        sweep_ms = 0.0
        for _ in range(args.steps):
            _res, ms = ctx.sn_si_step(prec, time_sweep=True)
            sweep_ms += ms
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop(local)
        ms_total = max_over_ranks(ev0.elapsed_time(ev1))
        return dict(value=job_throughput(ws, updates, args.steps, ms_total), ms_per_step=ms_total / args.steps,
                    sweep_ms_per_step=sweep_ms / args.steps, launches=int(ctx.sn_kernel_launches() - l0),
                    clocks=clk, schedule=sched)

    def use_schedule(sched):
        ctx.sn_set_launch(g.SN_LAUNCH_DATAFLOW if sched["mode"] == "dataflow" else g.SN_LAUNCH_LEVELS,
                          sched["blocks_per_sm"])

    forms = {"fp64": g.SN_PREC_FP64, "mixed": g.SN_PREC_MIXED, "mixed_ds": g.SN_PREC_MIXED_DS,
             "fp64_inv": g.SN_PREC_FP64_INV, "ds_inv": g.SN_PREC_DS_INV}
    if args.quick and args.quick_forms:
        forms = {k: forms[k] for k in args.quick_forms.split(",")}
    meas = {k: timed_steps(v) for k, v in forms.items()}
    if args.quick:
        if rank == 0:
            return {"metric": METRIC, "quick": True, "workload": args.quick_workload or WORKLOAD,
                    **{k: {kk: vv for kk, vv in m.items() if kk != "clocks"} for k, m in meas.items()}}
        return None
    head = args.form
    hp = forms[head]

    # ---- end to end through the C ABI with pinned host buffers (copies inside the timed region):
    # every step uploads phi and psi_old, sweeps, downloads psi_new, uploads psi_new and phi_prev
    # for the moment and downloads phi (sn_sweep / sn_moment stage host buffers themselves)
    phi_h = torch.zeros((E, N), dtype=torch.float64, pin_memory=True).numpy()
    phi2_h = torch.zeros((E, N), dtype=torch.float64, pin_memory=True).numpy()
    psa = torch.zeros((M, E, N), dtype=torch.float64, pin_memory=True).numpy()
    psb = torch.zeros((M, E, N), dtype=torch.float64, pin_memory=True).numpy()
    use_schedule(meas[head]["schedule"])
    for _ in range(max(1, args.warmup)):
        ctx.sn_sweep(phi_h, psa, psb, hp)
        ctx.sn_moment(psb, phi_h, phi2_h)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.sn_sweep(phi_h, psa, psb, hp)
        ctx.sn_moment(psb, phi_h, phi2_h)
        phi_h, phi2_h = phi2_h, phi_h
        psa, psb = psb, psa
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()
    h2d = phi_h.nbytes + psa.nbytes + psb.nbytes + phi_h.nbytes
    d2h = psb.nbytes + phi_h.nbytes

    # ---- time to a 1e-8 relative scalar-flux change, full solves from phi = 0
    tts = {}
    phis = {}
    inv_ms = {k: ctx.sn_prepare_inverse(forms[k]) for k in ("fp64_inv", "ds_inv") if k in forms}
    for k, prec in forms.items():
        phis[k] = np.zeros((E, N))
        use_schedule(meas[k]["schedule"])
        if prec in (g.SN_PREC_FP64_INV, g.SN_PREC_DS_INV):
            ctx.sn_release_inverse()         # formed again inside the timed solve
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = ctx.sn_source_iterate(1e-8, 2000, prec, phi_out=phis[k])
        tts[k] = dict(seconds=time.perf_counter() - t0, iters=res["iters"], converged=res["converged"])
    diffs = {k: float(np.linalg.norm(phis[k] - phis["fp64"]) / np.linalg.norm(phis["fp64"])) for k in forms}
    # the same solves with diffusion synthetic acceleration after every sweep
    dsa = {}
    for k in ("fp64", "mixed_ds", "ds_inv"):
        phi_k = np.zeros((E, N))
        use_schedule(meas[k]["schedule"])
        ctx.sn_set_dsa(True, args.dsa_rtol, args.dsa_max_cg)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = ctx.sn_source_iterate(1e-8, 2000, forms[k], phi_out=phi_k)
        dsa[k] = {"seconds": time.perf_counter() - t0, "iters": res["iters"], "converged": res["converged"],
                  "last_cg_iters": ctx.sn_dsa_last_iters(),
                  "phi_rel_l2_vs_plain_fp64": float(np.linalg.norm(phi_k - phis["fp64"]) / np.linalg.norm(phis["fp64"]))}
        ctx.sn_set_dsa(False, args.dsa_rtol, args.dsa_max_cg)

    if rank != 0:
        return None
    pk, pk_kind = peaks()
    inflow_faces = dim            # on average dim of the 2 dim faces of an element are inflow faces
    work = alg_work(dim, prob.p)

    def roofline(kind, m):
        pcode = {"fp64": 0, "mixed": 1, "mixed_ds": 2, "fp64_inv": 3, "ds_inv": 4}[kind]
        flow = m["schedule"]["mode"] == "dataflow"
        kname = (f"sweep_flow_kernel<{dim},{prob.p},{pcode}> (one persistent launch per sweep)" if flow else
                 f"sweep_level_kernel<{dim},{prob.p},{pcode}> (all level launches of one sweep)")
        if kind in ("fp64_inv", "ds_inv"):
            sweep_s = m["sweep_ms_per_step"] / 1e3
            ib = inv_alg_bytes(dim, prob.p)
            ach = ib * updates / sweep_s / 1e9
            traffic, capture = traffic_for(kind, m["schedule"]["mode"])
            return {"bound": "hbm", "kernel": kname, "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / pk["hbm_gbs"], "peak_source": f"MEASURED_PEAKS.json hbm_gbs (of {pk_kind})",
                    "alg_bytes_per_update": ib, "traffic": traffic,
                    "traffic_unit": "bytes per launch" + (" (one launch per sweep)" if flow else
                                                          " (level launch, sweep average)"),
                    "traffic_capture": capture, "sweep_launches_per_step": m["launches"] // max(1, args.steps) - 1,
                    "sweep_ms_per_step": m["sweep_ms_per_step"]}
        if kind == "fp64":
            peak, unit, src = FP64_PEAK_TFLOPS, "TFLOP/s (FP64 pipe)", "FP64 DFMA microbenchmark (of measured)"
        else:
            peak, unit, src = FP32_PEAK_TFLOPS, "TFLOP/s (FP32 pipe)", "FP32 FFMA microbenchmark (of measured)"
        sweep_s = m["sweep_ms_per_step"] / 1e3
        ach = work["flops"] * updates / sweep_s / 1e12
        traffic, capture = traffic_for(kind, m["schedule"]["mode"])
        launches = m["launches"] // max(1, args.steps) - 1          # sweep launches (one moment launch)
        out = {"bound": "alu", "kernel": kname, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
               "peak_source": src, "alg_flops_per_update": work["flops"], "alg_bytes_per_update": work["bytes"],
               "hbm_achieved_gbs": work["bytes"] * updates / sweep_s / 1e9,
               "hbm_frac_of_measured": work["bytes"] * updates / sweep_s / 1e9 / pk["hbm_gbs"],
               "traffic": traffic, "traffic_unit": "bytes per launch" + (" (one launch per sweep)" if flow else
                                                                          " (level launch, sweep average)"),
               "traffic_capture": capture, "sweep_launches_per_step": launches,
               "sweep_ms_per_step": m["sweep_ms_per_step"]}
        if kind == "mixed_ds":
            out["issued_fp32_flops_per_update"] = ds_fp32_issued_flops_per_update(dim, prob.p, inflow_faces)
        return out

    def form_line(k):
        return {"value": meas[k]["value"], "unit": "updates/s", "ms_per_step": meas[k]["ms_per_step"],
                "dtype": DTYPES[k], "schedule": meas[k]["schedule"], "precision": PRECISION_DESC[k],
                "roofline": roofline(k, meas[k]), "gpu_launches": meas[k]["launches"], "clocks": meas[k]["clocks"],
                "time_to_1e-8_s": tts[k]["seconds"], "iters_to_1e-8": tts[k]["iters"],
                "converged": tts[k]["converged"], "phi_rel_l2_vs_fp64": diffs[k]}

    out = {
        "metric": METRIC, "value": meas[head]["value"], "unit": "updates/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": meas[head]["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[head], "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "precision": PRECISION_DESC[head],
                   "weighting": "face", "parallelism": "replicas" if ws > 1 else "single",
                   "launch": args.launch, "schedule": meas[head]["schedule"],
                   "l2": "inputs larger than L2 (psi 2x84 MB + element factors 117 MB; FP32 splits 2x117 MB)"},
        "roofline": roofline(head, meas[head]),
        "e2e": {"value": updates * args.steps / e2e_s, "unit": "updates/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": meas[head]["launches"],
        "clocks": meas[head]["clocks"],
        "mixed_ds": form_line("mixed_ds"),
        "time_to_1e-8": {"fp64_s": tts["fp64"]["seconds"], "mixed_ds_s": tts["mixed_ds"]["seconds"],
                         "mixed_s": tts["mixed"]["seconds"], "fp64_inv_s": tts["fp64_inv"]["seconds"],
                         "ds_inv_s": tts["ds_inv"]["seconds"],
                         "speedup_mixed_ds_vs_fp64": tts["fp64"]["seconds"] / tts["mixed_ds"]["seconds"],
                         "speedup_fp64_inv_vs_fp64": tts["fp64"]["seconds"] / tts["fp64_inv"]["seconds"],
                         "speedup_ds_inv_vs_fp64": tts["fp64"]["seconds"] / tts["ds_inv"]["seconds"],
                         "fp64_iters": tts["fp64"]["iters"], "mixed_ds_iters": tts["mixed_ds"]["iters"],
                         "fp64_inv_iters": tts["fp64_inv"]["iters"], "ds_inv_iters": tts["ds_inv"]["iters"],
                         "phi_rel_l2_mixed_ds_vs_fp64": diffs["mixed_ds"],
                         "phi_rel_l2_fp64_inv_vs_fp64": diffs["fp64_inv"],
                         "phi_rel_l2_ds_inv_vs_fp64": diffs["ds_inv"],
                         "stored_inverse_forms_include": "allocation and formation of the stored inverses"},
        "stored_inverses": {"inverse_ms": inv_ms, "inverse_bytes": int(M) * int(E) * N * N * 8,
                            "fp64_inv": form_line("fp64_inv"), "ds_inv": form_line("ds_inv")},
        "forms": {k: form_line(k) for k in forms},
        "dsa": {"cg_rtol": args.dsa_rtol, "cg_max_iter": args.dsa_max_cg, **dsa,
                "speedup_fp64_dsa_vs_fp64": tts["fp64"]["seconds"] / dsa["fp64"]["seconds"],
                "speedup_mixed_ds_dsa_vs_fp64": tts["fp64"]["seconds"] / dsa["mixed_ds"]["seconds"],
                "speedup_ds_inv_dsa_vs_fp64": tts["fp64"]["seconds"] / dsa["ds_inv"]["seconds"]},
        "graph": {"build_s": t_graph, "removed": gstats["n_removed"], "levels": gstats["max_level"] + 1,
                  "max_scc": gstats["max_scc"], "mixed_faces": gstats["n_mixed_faces"],
                  "graph_ms": {k: gstats[k] for k in ("ms_geometry", "ms_weights", "ms_fas", "ms_levels")}},
        "peaks_file": pk_kind,
    }
    ctx.close()
    if not args.no_small:
        out["small_2d"] = run_small(g, torch, args)
    if not args.no_batch:
        out["batched"] = run_batch(g, torch, args)
    if not args.no_3d:
        out["twisted_3d"] = run_3d(g, torch, args)
    if not args.no_learned:
        out["learned"] = run_learned(g, torch, args)
    if not args.no_dsa_thick:
        out["dsa_thick"] = run_dsa_thick(g, torch, args)
    if not args.no_straightening:
        out["straightening"] = run_straightening(g, torch, args)
    if not args.no_triangles:
        out["triangles"] = run_triangles(g, torch, args)
    if not args.no_tets:
        out["tetrahedra"] = run_tets(g, torch, args)
    if not args.no_cpu_baseline:
        iters = {"2d": tts["fp64"]["iters"],
                 "3d_twist": out.get("twisted_3d", {}).get("fp64", {}).get("iters"),
                 "3d_s12": out.get("learned", {}).get("plain_fp64", {}).get("iters")}
        out["cpu_baseline"] = cpu_baseline(args, iters)
    return out


def run_small(g, torch, args):
    """16x16 sine-perturbed Q2 quads, p = 1 (4 unknowns), S4 (12 directions), sigma_t = 1,
    sigma_s = 0.5, q = 1: 3,072 updates per sweep, latency bound (31 levels of ~100 pairs).
    Reported per level, and as time to a 1e-8 residual next to the oracle's on one host core."""
    import sn_inputs as si
    prob = si.make_config("2d_sine_q2_p1_s4")
    stream = torch.cuda.Stream()
    ctx = g.setup_problem(prob, device=0, stream=stream.cuda_stream)
    gs = ctx.sn_build_graph("face", 10)
    levels = int(gs["max_level"] + 1)
    E, N = prob.mesh.n_elem, 4
    ups = E * len(prob.w)
    res = {"workload": "16x16 Q2 quads, x' = x + 0.05 sin(2 pi x) sin(2 pi y) on both coordinates, p=1, S4 (12 dirs), "
                       "sigma_t=1, sigma_s=0.5, q=1", "updates_per_sweep": ups, "levels": levels}
    for name, prec in (("fp64", g.SN_PREC_FP64), ("mixed_ds", g.SN_PREC_MIXED_DS),
                       ("fp64_inv", g.SN_PREC_FP64_INV), ("ds_inv", g.SN_PREC_DS_INV)):
        mode, bps = ctx.sn_autotune(prec)
        for _ in range(args.warmup):
            ctx.sn_si_step(prec)
        steps = max(20, args.steps)
        tot = 0.0
        for _ in range(steps):
            _, ms = ctx.sn_si_step(prec, time_sweep=True)
            tot += ms
        phi = np.zeros((E, N))
        if prec in (g.SN_PREC_FP64_INV, g.SN_PREC_DS_INV):
            ctx.sn_release_inverse()         # formed again inside the timed solve
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = ctx.sn_source_iterate(1e-8, 1000, prec, phi_out=phi)
        res[name] = {"sweep_us": 1e3 * tot / steps, "us_per_level": 1e3 * tot / steps / levels,
                     "sweep_updates_per_s": ups * steps / (tot / 1e3),
                     "schedule": {"mode": "dataflow" if mode == 1 else "levels", "blocks_per_sm": bps},
                     "time_to_1e-8_s": time.perf_counter() - t0, "iters": r["iters"], "converged": r["converged"]}
    ctx.close()
    if not args.no_cpu_baseline:
        res["oracle_time_to_1e-8"] = oracle_small_solve()
    return res


def oracle_small_solve():
    """The oracle's source iteration to 1e-8 on the 16x16 p=1 S4 workload, one host thread
    (discretisation, graph, local factorisations and every sweep)."""
    from oracle.dg import Discretization
    from oracle.graph import build_graph
    from oracle.sweep import Sweeper
    import sn_inputs as si
    prob = si.make_config("2d_sine_q2_p1_s4")
    t0 = time.perf_counter()
    disc = Discretization(prob)
    G = build_graph(disc, "face")
    R = Sweeper(disc, G).source_iterate(tol=1e-8)
    return {"seconds": time.perf_counter() - t0, "iters": R["iters"], "cores": 1,
            "kind": "oracle", "note": "numpy/scipy FP64, single thread, whole solve from phi = 0"}


def run_3d(g, torch, args):
    """3D cyclic workload: 32^3 hexahedra, Q2 geometry twisted by 60 degrees about z, p = 2 (27 dofs),
    S8 (80 directions), sigma_t = 1, sigma_s = 0.8, q = 1: 2,621,440 updates per sweep."""
    import sn_inputs as si
    prob = si.make_config("3d_twist_q2_p2_s8")
    stream = torch.cuda.Stream()
    ctx = g.setup_problem(prob, device=0, stream=stream.cuda_stream)
    t0 = time.time()
    gs = ctx.sn_build_graph("face", 10)
    res = {"workload": "32^3 Q2 hexes twisted 60 deg about z, p=2, S8 (80 dirs), sigma_t=1, sigma_s=0.8, q=1",
           "updates_per_sweep": int(prob.mesh.n_elem * len(prob.w)), "graph_build_s": time.time() - t0,
           "removed_arcs": int(gs["n_removed"]), "max_scc": int(gs["max_scc"]), "levels": int(gs["max_level"] + 1),
           "mixed_faces": int(gs["n_mixed_faces"]), "n_scc": int(gs["n_scc"]),
           "graph_ms": {k: gs[k] for k in ("ms_geometry", "ms_weights", "ms_fas", "ms_levels")}}
    ups = prob.mesh.n_elem * len(prob.w)
    E, N = prob.mesh.n_elem, 27
    pk, pk_kind = peaks()
    for name, prec in (("mixed_ds", g.SN_PREC_MIXED_DS), ("fp64", g.SN_PREC_FP64), ("fp64_inv", g.SN_PREC_FP64_INV),
                       ("ds_inv", g.SN_PREC_DS_INV)):
        mode, bps = ctx.sn_autotune(prec)
        for _ in range(args.warmup):
            ctx.sn_si_step(prec)
        tot = 0.0
        steps = max(5, args.steps // 4)
        for _ in range(steps):
            _, ms = ctx.sn_si_step(prec, time_sweep=True)
            tot += ms
        phi = np.zeros((E, N))
        inv_ms = None
        stored = prec in (g.SN_PREC_FP64_INV, g.SN_PREC_DS_INV)
        if stored:
            inv_ms = ctx.sn_prepare_inverse(prec)
            ctx.sn_release_inverse()         # formed again inside the timed solve
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        r = ctx.sn_source_iterate(1e-8, 3000, prec, phi_out=phi)
        rate = ups * steps / (tot / 1e3)
        work = alg_work(3, prob.p)
        if stored:
            ib = inv_alg_bytes(3, prob.p)
            roof = {"bound": "hbm", "achieved_gbs": rate * ib / 1e9, "peak_gbs": pk["hbm_gbs"],
                    "frac": rate * ib / 1e9 / pk["hbm_gbs"], "alg_bytes_per_update": ib}
        else:
            peak = FP64_PEAK_TFLOPS if prec == g.SN_PREC_FP64 else FP32_PEAK_TFLOPS
            roof = {"bound": "alu", "achieved_tflops": rate * work["flops"] / 1e12,
                    "peak_tflops": peak, "frac": rate * work["flops"] / 1e12 / peak,
                    "pipe": "FP64" if prec == g.SN_PREC_FP64 else "FP32",
                    "alg_flops_per_update": work["flops"], "alg_bytes_per_update": work["bytes"]}
        res[name] = {"sweep_updates_per_s": rate, "sweep_ms": tot / steps,
                     "schedule": {"mode": "dataflow" if mode == 1 else "levels", "blocks_per_sm": bps},
                     "roofline": roof,
                     "time_to_1e-8_s": time.perf_counter() - t1, "iters": r["iters"], "converged": r["converged"]}
        if inv_ms is not None:
            res[name]["inverse_ms"] = inv_ms
            res[name]["inverse_bytes"] = int(E) * len(prob.w) * N * N * 8
            ctx.sn_release_inverse()
    ctx.close()
    return res


def run_dsa_thick(g, torch, args):
    """Where diffusion synthetic acceleration is the tool: the 2D Q3 p=3 S8 workload family on a
    64 x 64 mesh with sigma_t ~ U[10, 100] per element (optically thick cells) and scattering ratio
    0.995.  Time to a 1e-8 scalar-flux change, double-single sweeps, plain vs DSA."""
    import sn_inputs as si
    prob = si.make_config("2d_smooth_q3_p3_s8", n=64)
    prob.sigma_t = 20.0 * prob.sigma_t
    prob.sigma_s = 0.995 * prob.sigma_t
    stream = torch.cuda.Stream()
    ctx = g.setup_problem(prob, device=0, stream=stream.cuda_stream)
    ctx.sn_build_graph("face", 10)
    ctx.sn_autotune(g.SN_PREC_MIXED_DS)
    E, N = prob.mesh.n_elem, 16
    out = {"workload": "64x64 Q3 quads, smooth perturbation 0.1h, p=3, S8 (40 dirs), sigma_t~U[10,100], c=0.995, q=1",
           "updates_per_sweep": int(E * len(prob.w))}
    ref = None
    for name, acc in (("plain_mixed_ds", False), ("dsa_mixed_ds", True)):
        phi = np.zeros((E, N))
        ctx.sn_set_dsa(acc, args.dsa_rtol, args.dsa_max_cg)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = ctx.sn_source_iterate(1e-8, 20000, g.SN_PREC_MIXED_DS, phi_out=phi)
        dt = time.perf_counter() - t0
        if ref is None:
            ref = phi.copy()
        out[name] = {"seconds": dt, "iters": r["iters"], "converged": r["converged"],
                     "phi_rel_l2_vs_plain": float(np.linalg.norm(phi - ref) / np.linalg.norm(ref))}
        if acc:
            out[name]["last_cg_iters"] = ctx.sn_dsa_last_iters()
    out["speedup_dsa"] = out["plain_mixed_ds"]["seconds"] / out["dsa_mixed_ds"]["seconds"]
    ctx.close()
    return out


def run_straightening(g, torch, args):
    """The paper's straightened low-order comparison (Sec. 4.1) on a quarter annulus (radii 0.5
    and 1, curved boundaries): its manufactured solution solved with cubic elements (p = 3) on a
    cubic (Q3) mesh, coarse and refined, and with linear elements (p = 1) on the straightened
    meshes (each element divided 3 times per direction, straight-sided Q1 cells).  L2 error of the
    scalar flux against the exact one at the volume quadrature points, unknowns, lagged arcs, time
    of the graph build and of the solve to a 1e-12 change (stored inverses, double-single)."""
    import sn_inputs.configs as C
    from sn_inputs.mms import annulus_mms
    out = {"workload": "quarter annulus rho in [0.5, 1], S4 (12 dirs), sigma_t=1, sigma_s=0.5, manufactured "
                       "psi = [(1 + x^2 + y^2)/2 + cos(3x + 3y/2)] (mu^2 + eta)"}
    for label, prob in (("ho_coarse", C.annulus_problem(12, 24, 3, 3)),
                        ("ho_refined", C.annulus_problem(24, 48, 3, 3)),
                        ("straightened_coarse", C.straightened_problem(C.annulus_problem(12, 24, 3, 3), 3, 1)),
                        ("straightened_refined", C.straightened_problem(C.annulus_problem(24, 48, 3, 3), 3, 1))):
        prob, fex, fac = annulus_mms(prob)
        stream = torch.cuda.Stream()
        ctx = g.setup_problem(prob, device=0, stream=stream.cuda_stream)
        t0 = time.perf_counter()
        gs = ctx.sn_build_graph("face", 10)
        t1 = time.perf_counter()
        E, N = prob.mesh.n_elem, (prob.p + 1) ** 2
        phi = np.zeros((E, N))
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        r = ctx.sn_source_iterate(1e-12, 500, g.SN_PREC_DS_INV, phi_out=phi)
        t3 = time.perf_counter()
        err = ctx.sn_l2_error(phi, fac * fex(ctx.sn_volume_points()))
        out[label] = {"elements": int(E), "geometry_order": int(prob.mesh.r), "dg_order": int(prob.p),
                      "unknowns": int(E * N), "l2_error": err, "removed_arcs": int(gs["n_removed"]),
                      "iters": r["iters"], "converged": r["converged"], "graph_s": t1 - t0, "solve_s": t3 - t2}
        ctx.close()
    out["error_ratio_straightened_vs_ho_coarse"] = out["straightened_coarse"]["l2_error"] / out["ho_coarse"]["l2_error"]
    out["error_ratio_straightened_vs_ho_refined"] = (out["straightened_refined"]["l2_error"] /
                                                     out["ho_refined"]["l2_error"])
    return out


def run_triangles(g, torch, args):
    """Simplicial elements (Sec. 2): 128 x 128 cells of [0,1]^2 cut into 32,768 counterclockwise
    triangles, P3 geometry with the sine perturbation 0.05 sin(2 pi x) sin(2 pi y), P3 DG (10
    unknowns), S8 (40 directions), sigma_t = 1, sigma_s = 0.5, q = 1: 1,310,720 updates per sweep,
    swept by the two stored-inverse forms; sweep rate, HBM fraction and time to a 1e-8 change
    (formation of the stored inverses included)."""
    import sn_inputs.configs as C
    n = getattr(args, "simplex_n", None) or 128
    return run_simplex(g, torch, args, C.triangle_problem(n, 3, 3, sn=8),
                       f"{2 * n * n} P3 triangles ({n}x{n} cells), sine perturbation 0.05, P3 DG, S8 (40 dirs), "
                       "sigma_t=1, sigma_s=0.5, q=1")


def run_tets(g, torch, args):
    """Straight-sided tetrahedra (Sec. 2): the unit cube as 32^3 cubes of six Kuhn tetrahedra
    (196,608 elements), twisted about the vertical axis by pi/3 over its height, P2 DG (10
    unknowns), S8 (80 directions), sigma_t = 1, sigma_s = 0.5, q = 1: 15,728,640 updates per
    sweep, swept by the two stored-inverse forms as the triangles are."""
    import sn_inputs.configs as C
    n = getattr(args, "simplex_n", None) or 32
    return run_simplex(g, torch, args, C.tet_problem(n, 2, sn=8, twist=math.pi / 3),
                       f"{6 * n ** 3} straight P2 tetrahedra ({n}^3 Kuhn-cut cubes), twist pi/3, S8 (80 dirs), "
                       "sigma_t=1, sigma_s=0.5, q=1")


def run_simplex(g, torch, args, prob, workload):
    stream = torch.cuda.Stream()
    ctx = g.setup_problem(prob, device=0, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    gs = ctx.sn_build_graph("face", 10)
    E, N, dim = prob.mesh.n_elem, ctx._N, prob.mesh.dim
    ups = E * len(prob.w)
    pk, _ = peaks()
    ib = inv_alg_bytes(dim, prob.p, simplex=True)
    out = {"workload": workload, "updates_per_sweep": int(ups),
           "graph_build_s": time.perf_counter() - t0, "removed_arcs": int(gs["n_removed"]),
           "levels": int(gs["max_level"] + 1), "mixed_faces": int(gs["n_mixed_faces"])}
    launch = getattr(args, "launch", "auto")
    forms = (("fp64_inv", g.SN_PREC_FP64_INV), ("ds_inv", g.SN_PREC_DS_INV))
    if getattr(args, "quick", False) and getattr(args, "quick_forms", None):
        forms = tuple(f for f in forms if f[0] in args.quick_forms.split(","))
    for name, prec in forms:
        if launch == "auto":
            mode, bps = ctx.sn_autotune(prec)
        else:
            mode, bps = (g.SN_LAUNCH_DATAFLOW if launch == "dataflow" else g.SN_LAUNCH_LEVELS), 0
            ctx.sn_set_launch(mode, bps)
            ctx.sn_si_begin(None)
        for _ in range(args.warmup):
            ctx.sn_si_step(prec)
        tot = 0.0
        steps = max(10, args.steps // 2)
        for _ in range(steps):
            _, ms = ctx.sn_si_step(prec, time_sweep=True)
            tot += ms
        rate = ups * steps / (tot / 1e3)
        inv_ms = ctx.sn_prepare_inverse(prec)
        ctx.sn_release_inverse()             # formed again inside the timed solve
        phi = np.zeros((E, N))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        r = ctx.sn_source_iterate(1e-8, 2000, prec, phi_out=phi)
        out[name] = {"sweep_updates_per_s": rate, "sweep_ms": tot / steps,
                     "schedule": {"mode": "dataflow" if mode == 1 else "levels", "blocks_per_sm": bps},
                     "roofline": {"bound": "hbm", "achieved_gbs": rate * ib / 1e9, "peak_gbs": pk["hbm_gbs"],
                                  "frac": rate * ib / 1e9 / pk["hbm_gbs"], "alg_bytes_per_update": ib},
                     "inverse_ms": inv_ms, "time_to_1e-8_s": time.perf_counter() - t1, "iters": r["iters"],
                     "converged": r["converged"]}
        ctx.sn_release_inverse()
    ctx.close()
    return out


def run_learned(g, torch, args):
    """3D learned-predictor workload family: n^3 Q2 hexes with seeded smooth perturbation 0.1h,
    p = 2, S12 (168 directions), sigma_t = exp(N(0,1)), c = 0.99, q = 1, the workload's own seeds
    (41, 42; the predictor was trained on seeds >= 1000).  Time to a 1e-8 relative scalar-flux
    change: plain FP64 source iteration vs the predictor (FP64 and double-single sweeps)."""
    import sn_inputs as si
    from paper_1810_11080_gb300 import learned
    path = os.path.join(ROOT, "paper_1810_11080_gb300", "models", "predictor_3d_q2_p2_s12.npz")
    if not os.path.exists(path):
        return {"unavailable": "trained predictor file not present"}
    stream = torch.cuda.Stream()
    model = learned.load(path)
    init, corr, cfg = learned.build(model, stream=stream.cuda_stream)
    prob = si.make_config("3d_smooth_q2_p2_s12", n=args.learned_n)
    ctx = g.setup_problem(prob, device=0, stream=stream.cuda_stream)
    ctx.sn_build_graph("face", 10)
    E, N = prob.mesh.n_elem, 27
    out = {"workload": f"{args.learned_n}^3 Q2 hexes, smooth perturbation 0.1h (seed 41), p=2, S12 (168 dirs), "
                       f"sigma_t=exp(N(0,1)) (seed 42), c=0.99, q=1",
           "updates_per_sweep": int(E * len(prob.w)), "train_solves": int(model.get("train_solves", 0)),
           "train_n": int(model.get("train_n", 0))}
    ref = np.zeros((E, N))
    runs = {}
    for name, prec, use, acc in (("plain_fp64", g.SN_PREC_FP64, False, False),
                                 ("learned_fp64", g.SN_PREC_FP64, True, False),
                                 ("plain_fp64_inv", g.SN_PREC_FP64_INV, False, False),
                                 ("learned_fp64_inv", g.SN_PREC_FP64_INV, True, False),
                                 ("plain_ds_inv", g.SN_PREC_DS_INV, False, False),
                                 ("learned_ds_inv", g.SN_PREC_DS_INV, True, False),
                                 ("plain_mixed_ds", g.SN_PREC_MIXED_DS, False, False),
                                 ("learned_mixed_ds", g.SN_PREC_MIXED_DS, True, False),
                                 ("dsa_mixed_ds", g.SN_PREC_MIXED_DS, False, True),
                                 ("learned_dsa_mixed_ds", g.SN_PREC_MIXED_DS, True, True)):
        phi = np.zeros((E, N))
        ctx.sn_set_dsa(acc, args.dsa_rtol, args.dsa_max_cg)
        ctx.sn_release_inverse()             # the stored-inverse runs form them inside the timed solve
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if use:
            r = ctx.sn_source_iterate_learned(1e-8, 5000, prec, init, corr, cfg, phi_out=phi)
        else:
            r = ctx.sn_source_iterate(1e-8, 5000, prec, phi_out=phi)
        dt = time.perf_counter() - t0
        if name == "plain_fp64":
            ref = phi.copy()
        runs[name] = {"seconds": dt, "iters": r["iters"], "converged": r["converged"],
                      "phi_rel_l2_vs_plain_fp64": float(np.linalg.norm(phi - ref) / np.linalg.norm(ref))}
        if use:
            runs[name]["corrections_accepted"] = r["accepted"]
            runs[name]["corrections_rejected"] = r["rejected"]
    out.update(runs)
    out["speedup_learned_mixed_ds_vs_plain_fp64"] = runs["plain_fp64"]["seconds"] / runs["learned_mixed_ds"]["seconds"]
    out["speedup_learned_fp64_vs_plain_fp64"] = runs["plain_fp64"]["seconds"] / runs["learned_fp64"]["seconds"]
    for k in ("dsa_mixed_ds", "learned_dsa_mixed_ds", "plain_fp64_inv", "learned_fp64_inv", "plain_ds_inv",
              "learned_ds_inv"):
        out[f"speedup_{k}_vs_plain_fp64"] = runs["plain_fp64"]["seconds"] / runs[k]["seconds"]
    out["dsa_cg"] = {"rtol": args.dsa_rtol, "max_iter": args.dsa_max_cg}
    ctx.sn_release_inverse()
    ctx.close()
    return out


def run_batch(g, torch, args):
    """256 independent 2D problems (n ~ U{8..64}, p ~ U{1,2,3}, r ~ U{2,3}, S4-S8, sigma_t ~ U[0.1,10],
    c ~ U[0.5,0.95]) swept in one launch per step; schedule picked by the autotuner."""
    import sn_inputs as si
    probs = si.batch_problems(count=256, seed=31)
    stream = torch.cuda.Stream()
    ctxs = []
    for p in probs:
        c = g.setup_problem(p, device=0, stream=stream.cuda_stream)
        c.sn_build_graph("face", 10)
        ctxs.append(c)
    b = g.Batch(ctxs, stream.cuda_stream)
    ups = b.sn_batch_updates_per_sweep()
    res = {"workload": "256 uneven 2D problems, n~U{8..64}, p~U{1,2,3}, r~U{2,3}, S4-S8, seed 31",
           "updates_per_sweep": int(ups), "elements": int(sum(p.mesh.n_elem for p in probs))}
    for name, prec in (("mixed_ds", g.SN_PREC_MIXED_DS), ("fp64", g.SN_PREC_FP64), ("fp64_inv", g.SN_PREC_FP64_INV),
                       ("ds_inv", g.SN_PREC_DS_INV)):
        mode, bps = b.sn_batch_tune(prec)
        b.sn_batch_si_begin()
        for _ in range(args.warmup):
            b.sn_batch_si_step(prec)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        steps = max(5, args.steps // 4)
        for _ in range(steps):
            b.sn_batch_si_step(prec)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        if prec in (g.SN_PREC_FP64_INV, g.SN_PREC_DS_INV):
            for c in ctxs:
                c.sn_release_inverse()       # formed again inside the timed solve
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = b.sn_batch_source_iterate(1e-8, 3000, prec)
        res[name] = {"value": ups * steps / (ms / 1e3), "unit": "updates/s", "ms_per_step": ms / steps,
                     "schedule": {"mode": "dataflow" if mode == 1 else "levels", "blocks_per_sm": bps},
                     "time_to_1e-8_s": time.perf_counter() - t0, "max_iters": int(r["iters"].max()),
                     "converged": r["status"] == 0}
    b.close()
    return res


def _oracle_worker(conn, d, workload=None, n=None):
    """One host process of the oracle timing: builds the workload's discretisation and direction
    d's graph once, then on every "go" times the oracle's work for one direction of one sweep
    (local assembly + factorisation of every element's system, and the lagged sweep)."""
    from oracle.dg import Discretization
    from oracle.graph import build_graph_dirs
    from oracle.sweep import Sweeper
    if workload is None:
        prob = make_problem()
    else:
        import sn_inputs as si
        prob = si.make_config(workload, n=n)
    disc = Discretization(prob)
    G = build_graph_dirs(disc, [d], "face")
    E, N, M = disc.E, disc.N, disc.M_dirs
    phi, psi_old = np.ones((E, N)), np.zeros((M, E, N))
    conn.send(("ready", E))
    while True:
        msg = conn.recv()
        if msg != "go":
            break
        t0 = time.perf_counter()
        Sweeper(disc, G, dirs=[d]).sweep(phi, psi_old, dirs=[d])
        conn.send(time.perf_counter() - t0)
    conn.close()


class OracleWorkers:
    """`procs` spawned processes (spawn start method: safe after CUDA initialisation), process i
    owning direction i mod 40 of the workload; round() runs one direction in every process at
    once and returns the wall time until the last one finishes."""

    def __init__(self, procs, workload=None, n=None, n_dirs=40):
        import multiprocessing as mp
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"                                # one thread per process
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for i in range(procs):
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_oracle_worker, args=(b, i % n_dirs, workload, n), daemon=True)
            pr.start()
            self.conns.append(a)
            self.procs.append(pr)
        self.E = [c.recv()[1] for c in self.conns][0]

    def round(self):
        t0 = time.perf_counter()
        for c in self.conns:
            c.send("go")
        for c in self.conns:
            c.recv()
        return time.perf_counter() - t0

    def close(self):
        for c in self.conns:
            c.send("stop")
        for pr in self.procs:
            pr.join(timeout=30)


def oracle_procs():
    """Host processes for the all-core oracle timing: every core, at most 16 (each holds ~0.5 GB)."""
    return max(1, min(os.cpu_count() or 1, 16))


def cpu_baseline(args, iters=None):
    """The oracle as it stands, on a bounded sample of the workload: one direction of one sweep
    per process (local assembly + factorisation + the lagged sweep), on one core and on all cores;
    and the same for the 3D p = 2 family on a 12^3 twisted mesh.  iters = the GPU's source-iteration
    counts to 1e-8 ({"2d": .., "3d_twist": .., "3d_s12": ..}) turn the all-core rates into
    extrapolated oracle times to 1e-8 of the full workloads (stated as extrapolations)."""
    import multiprocessing as mp
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    single = OracleWorkers(1)
    single.round()
    dt1 = single.round()
    single.close()
    P = oracle_procs()
    pool = OracleWorkers(P)
    pool.round()
    dtp = pool.round()
    pool.close()
    E = pool.E
    rate = E * P / dtp
    out = {"value": rate, "unit": "updates/s", "cores": P, "nproc": os.cpu_count(), "kind": "oracle",
           "sample": f"{P} directions of one sweep of the same workload at once, one per process "
                     f"({E * P} updates in {dtp:.1f} s): local assembly, LU and the lagged sweep, numpy/scipy FP64",
           "single_core": {"value": E / dt1, "unit": "updates/s", "cores": 1,
                           "sample": f"one direction ({E} updates) in {dt1:.1f} s"},
           "start_method": mp.get_context("spawn").get_start_method()}
    # 3D p = 2 sample: one direction of a 12^3 twisted Q2 mesh per process
    pool3 = OracleWorkers(P, workload="3d_twist_q2_p2_s8", n=12, n_dirs=80)
    pool3.round()
    dt3 = pool3.round()
    pool3.close()
    rate3 = pool3.E * P / dt3
    out["3d_p2"] = {"value": rate3, "unit": "updates/s", "cores": P,
                    "sample": f"{P} directions of one sweep of a 12^3 twisted Q2 p=2 mesh, one per process "
                              f"({pool3.E * P} updates in {dt3:.1f} s)"}
    if iters:
        ext = {"note": "oracle all-core rate x the workload's updates per sweep x the GPU's iteration count"}
        if iters.get("2d"):
            ext["2d_128x128_p3_s8_s"] = 655360 * iters["2d"] / rate
        if iters.get("3d_twist"):
            ext["3d_32cubed_p2_s8_s"] = 2621440 * iters["3d_twist"] / rate3
        if iters.get("3d_s12"):
            ext["3d_48cubed_p2_s12_s"] = 18579456 * iters["3d_s12"] / rate3
        out["extrapolated_time_to_1e-8"] = ext
    return out


def run_reference(args):
    """The oracle as it stands on the host cores: each step sweeps one direction of the same
    workload in each of P processes at once (local assembly + factorisation + lagged sweep);
    value in updates/s."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    P = oracle_procs()
    pool = OracleWorkers(P)
    for _ in range(args.warmup):
        pool.round()
    times = [pool.round() for _ in range(args.steps)]
    pool.close()
    E = pool.E
    v = E * P * len(times) / sum(times)
    cb = {"value": v, "unit": "updates/s", "cores": P, "nproc": os.cpu_count(), "kind": "oracle",
          "sample": f"each step: {P} of the 40 directions of one sweep of the same workload at once, one per "
                    f"process ({E * P} updates): local assembly, LU and the lagged sweep, numpy/scipy FP64"}
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "precision": "fp64", "weighting": "face",
                       "step": f"{P} directions of one sweep, one per host process"},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-problem batched measurement")
    ap.add_argument("--no-3d", action="store_true", help="skip the 3D twisted-mesh measurement")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-predictor measurement")
    ap.add_argument("--no-small", action="store_true", help="skip the 16x16 p=1 S4 measurement")
    ap.add_argument("--dsa-rtol", type=float, default=1e-4,
                    help="relative residual of the conjugate-gradient DSA solve in the accelerated legs")
    ap.add_argument("--dsa-max-cg", type=int, default=100, help="CG iteration cap of one DSA solve")
    ap.add_argument("--no-dsa-thick", action="store_true", help="skip the optically thick DSA measurement")
    ap.add_argument("--no-triangles", action="store_true", help="skip the triangle-mesh measurement")
    ap.add_argument("--no-tets", action="store_true", help="skip the tetrahedral-mesh measurement")
    ap.add_argument("--no-straightening", action="store_true",
                    help="skip the curved high-order vs straightened low-order comparison")
    ap.add_argument("--learned-n", type=int, default=48, help="mesh size n^3 of the learned-predictor measurement")
    ap.add_argument("--launch", default="auto", choices=["auto", "levels", "dataflow"],
                    help="sweep schedule per form: the autotuner's choice, one launch per level, or one persistent dataflow launch")
    ap.add_argument("--form", default="fp64", choices=["fp64", "mixed", "mixed_ds", "fp64_inv", "ds_inv"],
                    help="form reported as the headline value (all three are measured; default: the paper's FP64)")
    ap.add_argument("--quick", action="store_true",
                    help="timed steps only (no e2e, time-to-tolerance or CPU legs): for profiler launch lists")
    ap.add_argument("--quick-forms", default=None,
                    help="with --quick: comma-separated forms to time (fp64, mixed, mixed_ds, fp64_inv, ds_inv; "
                         "default all)")
    ap.add_argument("--quick-workload", default=None,
                    choices=["2d_sine_q2_p1_s4", "2d_smooth_q3_p3_s8", "3d_twist_q2_p2_s8", "3d_smooth_q2_p2_s12"],
                    help="with --quick: time this configuration instead of the default workload")
    ap.add_argument("--quick-simplex", default=None, choices=["triangles", "tetrahedra"],
                    help="with --quick: run only this simplex-mesh measurement (for profiler captures)")
    ap.add_argument("--simplex-n", type=int, default=None,
                    help="cells per side of the simplex-mesh measurements (default 128 triangles, 32 tetrahedra)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    out = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
