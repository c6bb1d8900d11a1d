#!/usr/bin/env python
"""Benchmark of the two-site DMRG Davidson sigma step on GB300.

One step = one sigma = H_eff psi at the centre bond (stage-1 and stage-2 block
GEMMs over all normal/complementary operator terms, the local terms and the
scatter into sigma), with the renormalised operators resident in HBM.
Default workload: L = 32 orbitals, 16 alpha + 16 beta electrons, D = 2048,
seeded synthetic integrals (seed 3), seeded random block-sparse MPS basis.

    python bench.py [--gpus N --steps K --warmup W] [--precision fp64|mixed]
    python bench.py --impl reference        # the CPU oracle on the host cores

Prints one JSON line (rank 0).  With N > 1 (torchrun), every rank runs an
independent replica of the workload (weak scaling, no collective on the data
path); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sigma TFLOP/s & sweep time, L=32 D=2048, mixed vs FP64 at |dE|<=1e-6 Eh"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=32)
    ap.add_argument("--na", type=int, default=None)
    ap.add_argument("--nb", type=int, default=None)
    ap.add_argument("--D", type=int, default=2048)
    ap.add_argument("--bond", type=int, default=None)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--fp64-steps", type=int, default=1, help="FP64 sigma steps timed beside the mixed ones")
    ap.add_argument("--cpu-sample", default="12,6,6,256", help="L,na,nb,D of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweeps", type=int, default=1,
                    help="also time this many full two-site sweeps at bond dimension D (fresh seeded basis)")
    ap.add_argument("--sweep-tol", type=float, default=1e-6, help="Davidson residual tolerance of the timed sweeps")
    ap.add_argument("--sweep-max-iter", type=int, default=100, help="Davidson iteration limit per sweep step")
    ap.add_argument("--mem-cap-gb", type=float, default=0.0,
                    help="mem_cap_bytes of the sweep handles (chunks the per-term intermediates; 0 = library default)")
    ap.add_argument("--refine-all", action="store_true",
                    help="split-BF16 sweeps: FP64 refinement at every step (not only the reported one)")
    ap.add_argument("--differentiate", default="",
                    help="L,na,nb,D,n_sweeps: converge split-BF16 sweeps (D ramp from D/4), then time the adjoint "
                         "(dmrg_sigma_backward: one- and two-particle densities) and the orbital gradient at the "
                         "final state, checked by central differences of E(exp(kappa)) with h = 1e-5")
    ap.add_argument("--mode-opt", default="",
                    help="L,na,nb,D,n_macro: mode optimisation (Sec. 2.2) -- n_macro macro iterations, each one sweep "
                         "with swap-gate layers and one sweep of micro-steps, after two plain sweeps; energies, "
                         "entropies of the cuts and seconds, next to the same number of plain sweeps")
    ap.add_argument("--batched-davidson", type=int, default=0,
                    help="with --batched: for the first n problems, Davidson at the centre bond in FP64 and in "
                         "split-BF16 with refinement from the same start vector (per-problem |dE| and seconds)")
    ap.add_argument("--batched", type=int, default=0,
                    help="also time the batched form on this many independent problems (L ~ U[10,20], "
                         "electrons = L with alpha/beta split within +-2, D in {256,512,1024}, seeds 100..)")
    ap.add_argument("--sweep-ramp", default="",
                    help="comma list of bond dimensions: one full sweep at each, in order, on one handle from the "
                         "seeded product-state basis (the D ramp of the headline sweep); per-sweep times and energies")
    ap.add_argument("--no-extras", action="store_true",
                    help="time the sigma step only (no sweep, no Davidson comparisons)")
    ap.add_argument("--compare-davidson", default="32,16,16,512",
                    help="L,na,nb,D: Davidson (Diag_H) at the centre bond of a fixed seeded basis in FP64 and in "
                         "split-BF16 with FP64 refinement, same start vector; times, energies and |dE|")
    ap.add_argument("--davidson-tol", type=float, default=1e-6)
    ap.add_argument("--davidson-max-iter", type=int, default=300)
    ap.add_argument("--compare-sweeps", default="",
                    help="L,na,nb,D,n_sweeps: time n full sweeps in FP64 and in split-BF16 from the same seeded "
                         "basis and report both sweep times and |dE| (mixed vs FP64)")
    a = ap.parse_args()
    if a.no_extras:
        a.sweeps, a.compare_davidson = 0, ""
    a.na = a.L // 2 if a.na is None else a.na
    a.nb = a.L // 2 if a.nb is None else a.nb
    a.bond = a.L // 2 - 1 if a.bond is None else a.bond
    return a


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.p = None
        self.lines = []

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, world, device):
    """Largest value of x over the ranks of the job (every rank gets it)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_tflops(flops_per_rank, world, ms):
    """Whole-job rate: every rank runs an independent replica of the same workload,
    so the job does world x flops_per_rank in the slowest rank's time ms."""
    return flops_per_rank * world / (ms * 1e-3) / 1e12


def cpu_baseline(args, flops_of):
    """The oracle (projected sigma through the FCI space) timed on the host cores on a bounded sample."""
    import oracle as O
    from paper_2501_18263_gb300 import inputs as I
    L, na, nb, D = (int(x) for x in args.cpu_sample.split(","))
    bond = L // 2 - 1
    t, v = I.synthetic_integrals(L, args.seed)
    bp = I.bond_problem(L, na, nb, D, bond, seed=args.seed + 1)
    flops = flops_of(t, v, na, nb, D, bp, bond)
    O.build()
    t0 = time.perf_counter()
    O.projected_sigma(t, v, na, nb, bp, bp.psi)
    dt = time.perf_counter() - t0
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"one projected sigma (FCI embedding, fci.c) at the centre bond of L={L}, {na}a+{nb}b, "
                      f"D={D}, same integral generator; rate = that bond's algorithmic sigma flops / oracle seconds",
            "seconds": dt}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:   # the replicas time the sigma step; the sweep and Davidson extras run at N = 1
        args.sweeps, args.compare_davidson = 0, ""

    import torch
    import torch.distributed as dist
    from paper_2501_18263_gb300 import binding as B
    from paper_2501_18263_gb300 import inputs as I

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream(dev)
    prec = B.PREC_FP64 if args.precision == "fp64" else B.PREC_MIXED_BF16

    t_setup = time.perf_counter()
    t, v = I.synthetic_integrals(args.L, args.seed)
    bp = I.bond_problem(args.L, args.na, args.nb, args.D, args.bond, seed=args.seed + 1)
    d = B.Dmrg(t, v, args.na, args.nb, D=args.D, precision=prec, seed=args.seed, stream=stream.cuda_stream)
    d.load_bond_problem(bp)
    d.prepare(args.bond)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    st = d.stats()
    flops = st["flops_stage1"] + st["flops_stage2"]
    n = st["psi_size"]
    psi = torch.tensor(B.pack_psi(bp.psi), dtype=torch.float64, device=dev)
    sig = torch.empty_like(psi)

    for _ in range(args.warmup):
        d.sigma(args.bond, psi.data_ptr(), sig.data_ptr())
    torch.cuda.synchronize()

    clk = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    d.profile_start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    for _ in range(args.steps):
        d.sigma(args.bond, psi.data_ptr(), sig.data_ptr())
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    prof = d.profile_stop()
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    value = job_tflops(flops, world, ms)

    # the FP64 path on the same handle and operators, timed beside the mixed one
    fp64 = None
    if prec == B.PREC_MIXED_BF16 and args.fp64_steps > 0:
        d.sigma_ex(args.bond, psi.data_ptr(), sig.data_ptr(), B.PREC_FP64)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.fp64_steps):
            d.sigma_ex(args.bond, psi.data_ptr(), sig.data_ptr(), B.PREC_FP64)
        f1.record(stream)
        torch.cuda.synchronize()
        fms = f0.elapsed_time(f1) / args.fp64_steps
        ref64 = sig.clone()
        d.sigma(args.bond, psi.data_ptr(), sig.data_ptr())
        torch.cuda.synchronize()
        relerr = float(torch.linalg.norm(sig - ref64) / torch.linalg.norm(ref64))
        fp64 = {"value": round(flops / (fms * 1e-3) / 1e12, 4), "unit": "TFLOP/s", "ms_per_step": round(fms, 3),
                "steps": args.fp64_steps, "mixed_vs_fp64_rel_err": relerr}

    # end to end through the public host-buffer entry point
    psi_h = np.ascontiguousarray(B.pack_psi(bp.psi))
    d.sigma_host(args.bond, psi_h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ke = max(1, args.steps)
    for _ in range(ke):
        d.sigma_host(args.bond, psi_h)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / ke, world, dev)

    pk, pk_kind = peaks()
    if prec == B.PREC_FP64:
        key = "gemm_f64"
        mhz = pk.get("sm_max_mhz", 2070.0)
        peak = 152 * 2 * 2 * mhz * 1e6 / 1e12   # 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x max clock
        bound, unit, peak_kind = "alu", "TFLOP/s", "derived (152 SM x 2 DFMA/clk x 2 flop x sm_max_mhz)"
    else:
        key = "gemm_bf16x"
        peak = pk["bf16_tflops"]
        bound, unit, peak_kind = "tensor", "TFLOP/s", pk_kind
    keys = [key] if key == "gemm_f64" else ["gemm_bf16x", "gemm_bf16x_stage1"]
    kms_tot = sum(prof[k]["ms"] for k in keys)
    kms = kms_tot / args.steps if kms_tot > 0 else None
    achieved = flops / (kms * 1e-3) / 1e12 if kms else None
    launches = sum(c["launches"] for c in prof.values())

    out = {
        "metric": METRIC,
        "value": round(value, 4),
        "unit": "TFLOP/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if prec == B.PREC_FP64 else "bf16x3-split/f32acc",
        "data": "synthetic (seeded integrals and random block-sparse MPS basis)",
        "config": {
            "workload": f"sigma step at the centre bond (k={args.bond}) of L={args.L}, {args.na}a+{args.nb}b, "
                        f"D={args.D}, synthetic integrals seed {args.seed}",
            "L": args.L, "n_alpha": args.na, "n_beta": args.nb, "D": args.D, "bond": args.bond,
            "precision": args.precision, "psi_size": n, "terms": st["n_terms"],
            "flops_per_sigma": flops, "operator_bytes": st["op_bytes"],
            "l2": "inputs larger than L2 (renormalised operators %.1f GB resident)" % (st["op_bytes"] / 1e9),
            "setup_s": round(t_setup, 1),
            "plan": {k: st[k] for k in ("mix_tiles1", "mix_steps1", "mix_tiles2", "mix_steps2", "mix_x_elems",
                                        "mix_plane_bytes", "gemm_problems", "gemm_segments")},
        },
        "clocks": clocks,
        "e2e": {"value": round(job_tflops(flops, world, e2e_s * 1e3), 4), "unit": "TFLOP/s",
                "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8},
        "gpu_launches": launches,
        "roofline": {"bound": bound, "achieved": round(achieved, 4) if achieved else None,
                     "peak": round(peak, 3), "unit": unit,
                     "frac": round(achieved / peak, 4) if achieved else None,
                     # DRAM counters take several ncu passes, which the size rule allows only on a
                     # small case: they were captured at D = 512 (profiles/), where the bytes per
                     # flop differ from D = 2048, so no full-size figure is reported
                     "traffic": None,
                     "traffic_note": "DRAM bytes per launch captured on the D = 512 case only "
                                     "(profiles/mixed_gemm_kernel_L32_D512_full.md); not scaled to D = 2048",
                     "kernel": key, "peak_source": peak_kind,
                     # the split-BF16 path performs six BF16 products per algorithmic multiply-add,
                     # so its own ceiling in algorithmic flops is the BF16 peak / 6
                     "split_ceiling": round(peak / 6, 3) if key != "gemm_f64" else None,
                     "frac_of_split_ceiling": (round(achieved / (peak / 6), 4)
                                               if (achieved and key != "gemm_f64") else None),
                     "kernel_ms_per_step": round(kms, 3) if kms else None},
        "profile_ms_per_step": {k: round(v["ms"] / args.steps, 3) for k, v in prof.items() if v["launches"]},
        "fp64": fp64,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        def flops_of(t_, v_, na_, nb_, D_, bp_, bond_):
            dd = B.Dmrg(t_, v_, na_, nb_, D=D_, stream=stream.cuda_stream)
            dd.load_bond_problem(bp_)
            dd.prepare(bond_)
            s_ = dd.stats()
            dd.close()
            return s_["flops_stage1"] + s_["flops_stage2"]
        try:
            out["cpu_baseline"] = cpu_baseline(args, flops_of)
        except Exception as e:  # pragma: no cover
            out["cpu_baseline"] = {"error": str(e)}
    if args.compare_davidson and prec == B.PREC_MIXED_BF16 and rank == 0:
        try:
            out["davidson_headline"] = headline_davidson(args, B, d, bp, dev)
        except Exception as e:  # pragma: no cover
            out["davidson_headline"] = {"error": f"{type(e).__name__}: {e}"}
    d.close()
    if args.sweeps > 0:
        # full L->R->L sweeps from the seeded kept-product-state basis, every bond at
        # dimension D; the phase split follows the paper's Sec. 4.1 categories
        torch.cuda.synchronize()
        ds = B.Dmrg(t, v, args.na, args.nb, D=args.D, precision=prec, seed=args.seed, stream=stream.cuda_stream)
        t0 = time.perf_counter()
        ds.profile_start()
        energies = ds.sweep(args.sweeps, [args.D] * args.sweeps, tol=args.sweep_tol, check=False)
        torch.cuda.synchronize()
        ts = time.perf_counter() - t0
        sprof = ds.profile_stop()
        slog = ds.sweep_log()
        out["sweep"] = {"workload": f"{args.sweeps} full sweep(s) L->R->L of L={args.L}, {args.na}a+{args.nb}b, "
                                    f"D={args.D} at every bond, from the seeded product-state basis, "
                                    f"Davidson tol {args.sweep_tol:g}",
                        "seconds_per_sweep": round(ts / args.sweeps, 2),
                        "phases_s": {k: round(x, 2) for k, x in ds.sweep_phases().items()},
                        "kernel_s": {k: round(x["ms"] / 1e3, 2) for k, x in sprof.items() if x["launches"]},
                        "energies": [float(x) for x in energies],
                        "steps": len(slog),
                        "davidson_iterations": sum(x["iters"] for x in slog),
                        "steps_by_status": {name: sum(1 for x in slog if x["status"] == k) for k, name in
                                            enumerate(["converged", "split_floor", "max_iter", "exhausted"])},
                        "reported_step": {k: slog[-1][k] for k in ("iters", "status", "rnorm")} if slog else None}
        ds.close()
    # optional extra measurements; a failure is recorded in the line instead of ending the run
    extras = []
    if args.batched > 0:
        extras.append(("batched", lambda: batched_bench(args, B, I)))
    if args.sweep_ramp:
        extras.append(("sweep_ramp", lambda: sweep_ramp(args, B, t, v, prec, stream)))
    if args.compare_davidson:
        extras.append(("davidson_compare", lambda: compare_davidson(args, B, I, stream)))
    if args.compare_sweeps:
        extras.append(("sweep_compare", lambda: compare_sweeps(args, B, I, stream)))
    if args.differentiate:
        extras.append(("differentiation", lambda: differentiate(args, B, I, stream)))
    if args.mode_opt:
        extras.append(("mode_optimisation", lambda: mode_optimisation(args, B, I, stream)))
    for key, fn in extras:
        try:
            out[key] = fn()
        except Exception as e:  # pragma: no cover
            out[key] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def sweep_ramp(args, B, t, v, prec, stream):
    """One full sweep per bond dimension of the ramp, continuing on one handle: wall seconds,
    Sec. 4.1 phase split and energy of each sweep."""
    import torch
    Ds = [int(x) for x in args.sweep_ramp.split(",")]
    d = B.Dmrg(t, v, args.na, args.nb, D=Ds[0], precision=prec, seed=args.seed, stream=stream.cuda_stream,
               mem_cap=int(args.mem_cap_gb * 2 ** 30))
    res = {"workload": f"one full sweep L->R->L per D in {Ds} on one handle, L={args.L}, {args.na}a+{args.nb}b, "
                       f"from the seeded product-state basis, Davidson tol {args.sweep_tol:g}"
                       + (f", mem_cap {args.mem_cap_gb:g} GB" if args.mem_cap_gb else ""), "sweeps": []}
    for D in Ds:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e = d.sweep(1, [D], tol=args.sweep_tol, refine_all=args.refine_all, check=False, max_iter=args.sweep_max_iter)
        torch.cuda.synchronize()
        res["sweeps"].append({"D": D, "seconds": round(time.perf_counter() - t0, 2), "energy": float(e[0]),
                              "phases_s": {k: round(x, 2) for k, x in d.sweep_phases().items()}})
    d.close()
    return res


def compare_davidson(args, B, I, stream):
    """Diag_H of one bond in FP64 and in split-BF16 (with its FP64 residual refinement) on the same
    seeded basis and start vector: wall seconds, iterations, energies and |dE|."""
    import torch
    L, na, nb, D = (int(x) for x in args.compare_davidson.split(","))
    bond = L // 2 - 1
    t, v = I.synthetic_integrals(L, args.seed)
    bp = I.bond_problem(L, na, nb, D, bond, seed=args.seed + 1)
    res = {"workload": f"Davidson at the centre bond (k={bond}) of L={L}, {na}a+{nb}b, D={D}, fixed seeded basis "
                       f"and start vector, residual tol {args.davidson_tol:g}"}
    for name, prec in (("fp64", B.PREC_FP64), ("mixed", B.PREC_MIXED_BF16)):
        d = B.Dmrg(t, v, na, nb, D=D, precision=prec, seed=args.seed, stream=stream.cuda_stream)
        d.load_bond_problem(bp)
        d.prepare(bond)
        x = torch.tensor(B.pack_psi(bp.psi), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        d.profile_start()
        t0 = time.perf_counter()
        e, it = d.davidson(bond, x.data_ptr(), tol=args.davidson_tol, max_iter=args.davidson_max_iter,
                           check=False)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        kp = d.profile_stop()
        res[name] = {"seconds": round(secs, 3), "iterations": it, "energy": e,
                     "converged": bool(d.last_status == B.OK),
                     "kernel_s": {k: round(v_["ms"] / 1e3, 3) for k, v_ in kp.items() if v_["launches"]}}
        d.close()
    res["abs_dE"] = abs(res["fp64"]["energy"] - res["mixed"]["energy"])
    res["speedup_mixed_vs_fp64"] = round(res["fp64"]["seconds"] / res["mixed"]["seconds"], 3)
    return res


def headline_davidson(args, B, d, bp, dev):
    """Diag_H at the benchmark's own bond (split-BF16 sigma with FP64 residual refinement):
    wall seconds, iterations and kernel time split; the energy is the FP64 Rayleigh quotient
    of the returned vector and its FP64 residual norm is at most the tolerance (convergence
    is only declared on an exact residual)."""
    import torch
    x = torch.tensor(B.pack_psi(bp.psi), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    d.profile_start()
    t0 = time.perf_counter()
    e, it = d.davidson(args.bond, x.data_ptr(), tol=args.davidson_tol, max_iter=args.davidson_max_iter, check=False)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    kp = d.profile_stop()
    # independent FP64 check of the returned vector: Rayleigh quotient and residual norm
    s64 = torch.empty_like(x)
    d.sigma_ex(args.bond, x.data_ptr(), s64.data_ptr(), B.PREC_FP64)
    torch.cuda.synchronize()
    rq = float((x * s64).sum() / (x * x).sum())
    rn = float(torch.linalg.norm(s64 - rq * x) / torch.linalg.norm(x))
    return {"workload": f"Davidson at the centre bond (k={args.bond}) of L={args.L}, {args.na}a+{args.nb}b, D={args.D} "
                        f"(the sigma workload above), split-BF16 sigma with FP64 refinement, tol {args.davidson_tol:g}",
            "seconds": round(secs, 3), "iterations": it, "energy": e, "converged": bool(d.last_status == B.OK),
            "kernel_s": {k: round(v_["ms"] / 1e3, 3) for k, v_ in kp.items() if v_["launches"]},
            "fp64_check": {"rayleigh_quotient": rq, "abs_dE": abs(rq - e), "residual_norm": rn}}


def compare_sweeps(args, B, I, stream):
    """Full sweeps of one problem in FP64 and in split-BF16 from the same seeded basis:
    wall seconds per sweep (with the Sec. 4.1 phase split) and the energy difference."""
    import torch
    f = args.compare_sweeps.split(",")
    L, na, nb = int(f[0]), int(f[1]), int(f[2])
    Ds = [int(x) for x in f[3].split("/")]
    ns = int(f[4]) if len(f) > 4 else len(Ds)
    Ds = (Ds + [Ds[-1]] * ns)[:ns]
    D = Ds[-1]
    t, v = I.synthetic_integrals(L, args.seed)
    res = {"workload": f"{ns} full sweep(s) L->R->L of L={L}, {na}a+{nb}b, D per sweep {Ds}, synthetic "
                       f"integrals seed {args.seed}, same seeded product-state basis for both precisions, "
                       f"Davidson tol {args.sweep_tol:g}" + (", split-BF16 refined at every step" if args.refine_all
                                                             else "")}
    for name, prec in (("fp64", B.PREC_FP64), ("mixed", B.PREC_MIXED_BF16)):
        torch.cuda.synchronize()
        d = B.Dmrg(t, v, na, nb, D=D, precision=prec, seed=args.seed, stream=stream.cuda_stream)
        per, e, lg, ph = [], [], [], {}
        for k in range(ns):   # one call per sweep: wall seconds of each
            t0 = time.perf_counter()
            e += list(d.sweep(1, [Ds[k]], tol=args.sweep_tol, refine_all=args.refine_all, check=False,
                              max_iter=args.sweep_max_iter))
            torch.cuda.synchronize()
            per.append(round(time.perf_counter() - t0, 2))
            lg += d.sweep_log()
            for kk, x in d.sweep_phases().items():
                ph[kk] = ph.get(kk, 0.0) + x
        ts = sum(per)
        res[name] = {"seconds_per_sweep": round(ts / ns, 2), "seconds_each": per, "energies": [float(x) for x in e],
                     "phases_s_all_sweeps": {k: round(x, 2) for k, x in ph.items()},
                     "davidson_iterations": sum(x["iters"] for x in lg),
                     "steps_by_status": {nm: sum(1 for x in lg if x["status"] == k) for k, nm in
                                         enumerate(["converged", "split_floor", "max_iter", "exhausted"])}}
        d.close()
    ef, em = res["fp64"]["energies"], res["mixed"]["energies"]
    res["abs_dE_per_sweep"] = [abs(a - b) for a, b in zip(ef, em)]
    res["speedup_mixed_vs_fp64"] = round(res["fp64"]["seconds_per_sweep"] / res["mixed"]["seconds_per_sweep"], 3)
    res["speedup_last_sweep"] = round(res["fp64"]["seconds_each"][-1] / res["mixed"]["seconds_each"][-1], 3)
    return res


def _rotated(t, v, p, q, h):
    """Integrals rotated by U = exp(kappa), kappa = h (e_pq - e_qp) (a plane rotation: U is the
    Givens matrix of angle h in the (p, q) plane), t' = U t U^T, v'_abcd = U_ai U_bj U_ck U_dl v_ijkl."""
    U = np.eye(t.shape[0])
    c, s = np.cos(h), np.sin(h)
    U[p, p] = U[q, q] = c
    U[p, q] = s
    U[q, p] = -s
    return U @ t @ U.T, np.einsum("ai,bj,ck,dl,ijkl->abcd", U, U, U, U, v, optimize=True)


def differentiate(args, B, I, stream):
    """The differentiation form at a converged state: split-BF16 sweeps with a D ramp, then
    dmrg_sigma_backward (one- and two-particle densities by the adjoint), dmrg_orbital_gradient,
    and central differences of E(exp(kappa)) for a few generators kappa_pq (same state)."""
    import torch
    L, na, nb, D, ns = (int(x) for x in args.differentiate.split(","))
    t, v = I.synthetic_integrals(L, 5)
    Ds = [max(16, D // 4), max(16, D // 2)] + [D] * max(1, ns - 2)
    d = B.Dmrg(t, v, na, nb, D=D, precision=B.PREC_MIXED_BF16, seed=5, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    e = d.sweep(len(Ds), Ds, tol=1e-7, check=False)
    torch.cuda.synchronize()
    t_sweep = time.perf_counter() - t0
    bond, n = d.sweep_state()
    psi = torch.empty(n, dtype=torch.float64, device="cuda")
    d.sweep_state(psi.data_ptr())
    d.prepare(bond)
    e0 = d.expectation(bond, psi.data_ptr(), psi.data_ptr())
    g1 = torch.zeros((L, L), dtype=torch.float64, device="cuda")
    g2 = torch.zeros((L, L, L, L), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    d.profile_start()
    t0 = time.perf_counter()
    d.sigma_backward(bond, psi.data_ptr(), psi.data_ptr(), g1.data_ptr(), g2.data_ptr())
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0
    kp = d.profile_stop()
    grad = torch.zeros((L, L), dtype=torch.float64, device="cuda")
    d.orbital_gradient(g1.data_ptr(), g2.data_ptr(), grad.data_ptr())
    torch.cuda.synchronize()
    G1, G2, GR = g1.cpu().numpy(), g2.cpu().numpy(), grad.cpu().numpy()
    checks = []
    h = 1e-5
    pairs = [(1, 0), (L // 2, L // 2 - 1), (L - 1, 0), (L - 1, L // 3)]
    for (p, q) in pairs:
        es = []
        for sgn in (+1, -1):
            tr, vr = _rotated(t, v, p, q, sgn * h)
            d.set_integrals(tr, vr)
            d.prepare(bond)
            es.append(d.expectation(bond, psi.data_ptr(), psi.data_ptr()))
        fd = (es[0] - es[1]) / (2 * h)
        checks.append({"p": p, "q": q, "analytic": float(GR[p, q]), "central_difference": fd,
                       "abs_diff": abs(fd - float(GR[p, q]))})
    d.set_integrals(t, v)
    d.close()
    return {"workload": f"L={L}, {na}a+{nb}b, split-BF16 sweeps with D = {Ds}, synthetic integrals seed 5; adjoint "
                        f"and orbital gradient at the final state (bond {bond}, psi_size {n})",
            "sweep_s": round(t_sweep, 2), "sweep_energies": [float(x) for x in e], "energy": e0,
            "adjoint_s": round(t_adj, 3),
            "adjoint_kernel_s": {k: round(x["ms"] / 1e3, 3) for k, x in kp.items() if x["launches"]},
            "trace_g1": float(np.trace(G1)), "electrons": na + nb,
            "energy_from_densities": float(np.sum(t * G1) + 0.5 * np.sum(v * G2)),
            "abs_dE_densities": abs(float(np.sum(t * G1) + 0.5 * np.sum(v * G2)) - e0),
            "orbital_gradient_norm": float(np.linalg.norm(GR)),
            "fd_checks_h1e-5": checks,
            "max_abs_diff_fd": max(c["abs_diff"] for c in checks)}


def mode_optimisation(args, B, I, stream):
    """Mode optimisation (Sec. 2.2): plain sweeps, then macro iterations of a sweep with swap-gate
    layers and a sweep of micro-steps (rotation of least half-Renyi entropy at every left-to-right
    step); the same total number of plain sweeps beside it."""
    import torch
    L, na, nb, D, nm = (int(x) for x in args.mode_opt.split(","))
    t, v = I.synthetic_integrals(L, 7)
    res = {"workload": f"L={L}, {na}a+{nb}b, D={D}, synthetic integrals seed 7: 2 plain sweeps, then {nm} macro "
                       f"iteration(s) of one swap-layer sweep and one micro-step sweep (split-BF16, tol 1e-7)"}
    dm = B.Dmrg(t, v, na, nb, D=D, seed=7, precision=B.PREC_MIXED_BF16, stream=stream.cuda_stream)
    dp = B.Dmrg(t, v, na, nb, D=D, seed=7, precision=B.PREC_MIXED_BF16, stream=stream.cuda_stream)
    e0 = list(dm.sweep(2, [D, D], tol=1e-7, check=False))
    ep = list(dp.sweep(2, [D, D], tol=1e-7, check=False))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    macro = []
    for k in range(nm):
        es = dm.sweep(1, [D], tol=1e-7, check=False, swap_layers=True)
        em = dm.sweep(1, [D], tol=1e-7, check=False, mode_opt=True)
        lg = dm.mode_log()
        macro.append({"energy_after_swaps": float(es[-1]), "energy_after_micro": float(em[-1]),
                      "sum_S_half_before": float(sum(x["s_before"] for x in lg)),
                      "sum_S_half_after": float(sum(x["s_after"] for x in lg)),
                      "max_abs_theta": float(max(abs(x["theta"]) for x in lg))})
    torch.cuda.synchronize()
    t_mo = time.perf_counter() - t0
    t0 = time.perf_counter()
    ep += list(dp.sweep(2 * nm, [D] * (2 * nm), tol=1e-7, check=False))
    torch.cuda.synchronize()
    t_pl = time.perf_counter() - t0
    res.update({"plain_energies": [float(x) for x in ep], "mode_opt_start": [float(x) for x in e0],
                "macro_iterations": macro, "mode_opt_s": round(t_mo, 2), "plain_s": round(t_pl, 2),
                "final_energy_mode_opt": macro[-1]["energy_after_micro"] if macro else None,
                "final_energy_plain": float(ep[-1])})
    dm.close()
    dp.close()
    return res


def batched_bench(args, B, I):
    """Split-BF16 sigma steps of many independent problems (each at its centre bond):
    one by one through dmrg_sigma, batched in shared grouped launches, and batched
    from a captured CUDA graph; problems/s = sigma steps of all problems per second."""
    import torch
    stream = torch.cuda.Stream()
    ds, bonds, psis, sigs, flops, meta = [], [], [], [], 0, []
    for i in range(args.batched):
        L, na, nb, D, seed = I.batched_problem(i)
        bond = L // 2 - 1
        t, v = I.synthetic_integrals(L, seed)
        bp = I.bond_problem(L, na, nb, D, bond, seed=seed + 1000)
        try:
            d = B.Dmrg(t, v, na, nb, D=D, precision=B.PREC_MIXED_BF16, seed=seed, stream=stream.cuda_stream)
            d.load_bond_problem(bp)
            d.prepare(bond)
        except B.DmrgError as e:
            if e.status != B.ERR_OOM:
                raise
            break
        st = d.stats()
        flops += st["flops_stage1"] + st["flops_stage2"]
        x = B.pack_psi(bp.psi)
        psis.append(torch.tensor(x / np.linalg.norm(x), dtype=torch.float64, device="cuda"))
        sigs.append(torch.empty_like(psis[-1]))
        ds.append(d)
        bonds.append(bond)
        meta.append((L, na, nb, D))
    torch.cuda.synchronize()
    n = len(ds)
    pp = [p.data_ptr() for p in psis]
    sp = [s.data_ptr() for s in sigs]
    batch = B.Batch(ds, bonds)
    sched = batch.tuning()   # tile order and tile width per launch, with every candidate's time

    def timed(fn, k):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / k

    def one_by_one():
        for d, b, p, s in zip(ds, bonds, pp, sp):
            d.sigma(b, p, s)

    k = max(3, args.steps // 3)
    t_seq = timed(one_by_one, k)
    t_eager = timed(lambda: batch.sigma(pp, sp, graph=False), k)
    t_graph = timed(lambda: batch.sigma(pp, sp, graph=True), k)
    # per-problem energy-scale error of the batched split-BF16 sigma against FP64:
    # |<psi|sigma_mixed> - <psi|sigma_fp64>| with psi normalised
    batch.sigma(pp, sp, graph=True)
    torch.cuda.synchronize()
    e_mix = [float((p * s).sum()) for p, s in zip(psis, sigs)]
    de = []
    for d, b, x, s, em in zip(ds, bonds, psis, sigs, e_mix):
        d.sigma_ex(b, x.data_ptr(), s.data_ptr(), B.PREC_FP64)
        de.append(abs(em - float((x * s).sum())))
    batch.close()
    dav = []
    for i in range(min(args.batched_davidson, n)):
        d, b, x0 = ds[i], bonds[i], psis[i]
        rec = {"problem": i, "L": meta[i][0], "D": meta[i][3]}
        for name, prec in (("fp64", B.PREC_FP64), ("mixed", B.PREC_MIXED_BF16)):
            x = x0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if prec == B.PREC_FP64:
                # the FP64 solve on its own handle (same integrals, basis and start vector)
                L_, na_, nb_, D_, seed_ = I.batched_problem(i)
                t_, v_ = I.synthetic_integrals(L_, seed_)
                bp_ = I.bond_problem(L_, na_, nb_, D_, b, seed=seed_ + 1000)
                d64 = B.Dmrg(t_, v_, na_, nb_, D=D_, seed=seed_, stream=stream.cuda_stream)
                d64.load_bond_problem(bp_)
                d64.prepare(b)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                e, it = d64.davidson(b, x.data_ptr(), tol=args.davidson_tol, max_iter=args.davidson_max_iter,
                                     check=False)
                torch.cuda.synchronize()
                d64.close()
            else:
                e, it = d.davidson(b, x.data_ptr(), tol=args.davidson_tol, max_iter=args.davidson_max_iter,
                                   check=False)
                torch.cuda.synchronize()
            rec[name] = {"energy": e, "iterations": it, "seconds": round(time.perf_counter() - t0, 3)}
        rec["abs_dE"] = abs(rec["fp64"]["energy"] - rec["mixed"]["energy"])
        dav.append(rec)
    for d in ds:
        d.close()
    extra = {}
    if dav:
        extra["davidson_per_problem"] = dav
        extra["davidson_max_abs_dE"] = max(r["abs_dE"] for r in dav)
    return {**extra, "workload": f"{n} independent problems, problem i: seed 100+i, L ~ U[10,20], electrons = L with "
                        f"alpha-beta in {{-2..2}}, D in {{256,512,1024}}, centre bond, synthetic integrals",
            "problems": n, "flops_per_step": flops,
            "problems_per_s": {"one_by_one": round(n / t_seq, 1), "batched": round(n / t_eager, 1),
                               "batched_graph": round(n / t_graph, 1)},
            "tflops": {"one_by_one": round(flops / t_seq / 1e12, 3), "batched": round(flops / t_eager / 1e12, 3),
                       "batched_graph": round(flops / t_graph / 1e12, 3)},
            "ms_per_step": {"one_by_one": round(t_seq * 1e3, 3), "batched": round(t_eager * 1e3, 3),
                            "batched_graph": round(t_graph * 1e3, 3)},
            "abs_dE_mixed_vs_fp64": {"max": max(de), "median": float(np.median(de))},
            "schedule": sched,
            "L_D": [[m[0], m[3]] for m in meta]}


def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores, same metric and unit (bounded sample per step)."""
    if rank != 0:
        return
    import oracle as O
    from paper_2501_18263_gb300 import inputs as I
    L, na, nb, D = (int(x) for x in args.cpu_sample.split(","))
    bond = L // 2 - 1
    t, v = I.synthetic_integrals(L, args.seed)
    bp = I.bond_problem(L, na, nb, D, bond, seed=args.seed + 1)
    flops = None
    try:  # algorithmic flops of the sample bond from the method's own count
        import torch
        from paper_2501_18263_gb300 import binding as B
        if torch.cuda.is_available():
            dd = B.Dmrg(t, v, na, nb, D=D, stream=torch.cuda.current_stream().cuda_stream)
            dd.load_bond_problem(bp)
            dd.prepare(bond)
            s_ = dd.stats()
            flops = s_["flops_stage1"] + s_["flops_stage2"]
            dd.close()
    except Exception:
        flops = None
    O.build()
    for _ in range(args.warmup and 1):
        O.projected_sigma(t, v, na, nb, bp, bp.psi)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.projected_sigma(t, v, na, nb, bp, bp.psi)
    dt = (time.perf_counter() - t0) / args.steps
    val = flops / dt / 1e12 if flops else None
    sample = (f"one projected sigma per step (FCI embedding, fci.c) at the centre bond of L={L}, {na}a+{nb}b, D={D}, "
              f"same integral generator")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": sample, "L": L, "n_alpha": na, "n_beta": nb, "D": D, "bond": bond},
        "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "sample": sample, "value": val},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


if __name__ == "__main__":
    main()
