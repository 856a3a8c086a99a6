"""Benchmark of the density-fitted RHF hot path on GB300.

Workload: a seeded 32-water cluster (1600 basis functions, 4384 auxiliary functions, 160 occupied
orbitals, packed whitened B of 46.7 GB resident in HBM), synthetic geometry and even-tempered bases.

A step is one density-fitted Fock build from the resident B: gamma = B.D, J = B^T gamma, the
half-transform Y = B C_occ and K = sum_P Y_P Y_P^T (paper eqs. 1-3). By default the exchange is the
split-precision form (BF16 Ozaki slices on the tensor cores) at the 5 slices the SCF uses for its
final iterations; --precision fp64 times the FP64 form. `value` is seconds per J/K build with inputs
already on the device (CUDA events on the stream the library launches on, max over ranks); `e2e` is
the same through the C ABI with host buffers (D and C_occ copied in, J and K copied out inside the
timed region). `time_to_converge_s` is one full SCF (integrals + whitening + iterations) to
|dE| < 1e-10 Eh and max|FDS - SDF| < 1e-7, from the core-Hamiltonian guess ("split") and from the
learned guess ("split_learned"), both with incremental Fock builds late; "split_learned_full" repeats
the learned run with full 5-slice builds. `compare` holds the per-iteration time of the early split
form (3 slices) and of the FP64 form on the same density.

Inputs (46.7 GB of B) are far larger than L2 (126 MB), so no flush is needed between steps.
Under torchrun with N > 1 each rank runs an independent replica (the path has no exchange step).
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

WORKLOAD = "water32"
METRIC = "SCF time-to-converge & DF J/K s/iter: split-prec+batched+learned vs FP64"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def max_over_ranks(value, device=None):
    """The largest `value` over all ranks of the process group (a replicated job takes as long as its
    slowest replica); `value` itself when no group is initialised or it has one rank."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def batch_members(count, rank, wmax=8):
    """The clusters of one rank's batched-SCF measurement: `count` (waters, seed) pairs, sizes drawn
    uniformly from 1-wmax waters, seeds 1000 + rank * count + k, so replicas solve disjoint molecule sets
    of the same size distribution (weak scaling: the work per GPU does not change with the rank count)."""
    from paper_1707_03771_gb300 import clusters
    rng = clusters.SplitMix64(4242 + rank)
    return [(1 + min(wmax - 1, int(rng.uniform() * wmax)), 1000 + rank * count + k) for k in range(count)]


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of the same kernel and tile on the same workload;
# keyed by (workload, kernel, slices, tile width). Anything not captured reports null. 32 waters, B slices as
# full rows, Y and K 32 columns, K split 4 (one pass per launch).
NCU_TRAFFIC = {("water32", "Y", 5, 32): 114.57e9 + 8.97e9, ("water32", "K", 5, 32): 27.58e9 + 0.04341e9}

def core_density(h):
    """A physical density for the timed builds: the core-Hamiltonian orbitals of the handle's molecule."""
    S_ov, H = h.matrix("S"), h.matrix("H")
    sv, U = np.linalg.eigh(S_ov)
    X = U[:, sv > 1e-7] / np.sqrt(sv[sv > 1e-7])
    _, Cp = np.linalg.eigh(X.T @ H @ X)
    C = np.ascontiguousarray((X @ Cp)[:, :h.nocc])
    return C, 2 * C @ C.T


def _scf_info(res):
    return {"energy": res["energy"], "iterations": res["iterations"], "converged": bool(res["converged"]),
            "t_total_s": res["t_total_s"], "t_build_s": res["t_build_s"], "t_iter_s": res["t_iter_s"],
            "t_jk_s": res["t_jk_s"], "ramp_iteration": res["ramp_iteration"],
            "incremental_builds": res["incremental_builds"], "approx_steps": res["approx_steps"]}


# FP64 multiply-adds per clock per SM of GB300 (its nominal 1.25 TFLOP/s dense FP64 at the 2070 MHz maximum
# SM clock over 152 SMs is 2 multiply-adds, 4 flops, per clock per SM)
FP64_FMA_PER_SM_CLOCK = 2


def fp64_peak(binding, gpu_index, sm_count, sm_mhz):
    """The FP64 pipe's peak for the roofline: unit count x SMs x the SM clock sampled during the timed J/K
    builds (flops = 2 x multiply-adds). Beside it, two loops measured now with the clock sampled meanwhile:
    DFMA and FP64 mma.sync (about 1 s each); they stay below the unit-count figure, which the bandwidth-free
    FP64 kernels here (gamma and coulomb) come within a few per cent of."""
    with ClockSampler(gpu_index) as clk:
        dfma, ms_a = binding.fp64_rate(0, 480000)
        dmma, ms_b = binding.fp64_rate(1, 120000)
    c = clk.summary()
    peak = 2.0 * FP64_FMA_PER_SM_CLOCK * sm_count * (sm_mhz or 2070.0) * 1e6 / 1e12
    out = {"peak_tflops": peak,
           "peak_source": f"{FP64_FMA_PER_SM_CLOCK} FP64 multiply-adds per clock per SM x {sm_count} SMs x "
                          f"{sm_mhz or 2070.0:.0f} MHz (median SM clock of the timed builds)",
           "measured_dfma_tflops": dfma, "measured_dmma_tflops": dmma, "measured_ms": [ms_a, ms_b],
           "measured_clocks": c,
           "how": "df_fp64_rate: 4 CTAs x 256 threads per SM; DFMA 8 independent chains per thread, "
                  "DMMA 4 independent m8n8k4 accumulations per warp; 2 flops per multiply-add"}
    if c.get("sm_mhz"):
        out["measured_fp64_flops_per_sm_per_clock"] = max(dfma, dmma) * 1e12 / (sm_count * c["sm_mhz"] * 1e6)
    return out


def jk_steps(h, lib, dev, stream, D, C, precision, slices, warmup, steps, ws=1):
    """Device-timed J/K builds from resident D and C (CUDA events on the stream the library launches on);
    returns (ms per build, per-build phase timings, the last K as a device tensor)."""
    import torch
    import torch.distributed as tdist
    n, nocc = h.n, C.shape[1]
    dD = torch.from_numpy(D).to(dev)
    dC = torch.from_numpy(np.ascontiguousarray(C)).to(dev)
    dJ = torch.empty((n, n), dtype=torch.float64, device=dev)
    dK = torch.empty((n, n), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    lib.df_set_stream(h.h, ctypes_ptr(stream.cuda_stream))
    try:
        for _ in range(warmup):
            h.jk_device(dD.data_ptr(), dC.data_ptr(), nocc, dJ.data_ptr(), dK.data_ptr(), precision, slices)
        torch.cuda.synchronize()
        if ws > 1:
            tdist.barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        per = []
        ev0.record(stream)
        for _ in range(steps):
            h.jk_device(dD.data_ptr(), dC.data_ptr(), nocc, dJ.data_ptr(), dK.data_ptr(), precision, slices)
            per.append(dict(h.timings()))
        ev1.record(stream)
        torch.cuda.synchronize()
    finally:
        lib.df_set_stream(h.h, None)
    total = max_over_ranks(ev0.elapsed_time(ev1), dev)
    return total / steps, per, dK


def gpu_arm(args):
    import torch
    import torch.distributed as tdist

    from paper_1707_03771_gb300 import binding, build, clusters

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    if ws > 1:
        tdist.barrier()
    lib = binding.load()
    system = clusters.workload(args.workload)
    guess_net = None
    learned = None
    if args.ttc and args.learned > 0:
        guess_net, learned = learned_guess_net(binding, clusters, args.learned)
    split = args.precision == "split"
    prec = binding.DF_PREC_SPLIT if split else binding.DF_PREC_FP64
    S = args.slices
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    t0 = time.perf_counter()
    h = binding.Handle(system)
    h.build_B(whitening=None if split else binding.DF_WHITEN_FP64)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    build_ms = h.timings()
    n, nocc = h.n, h.nocc
    C, D = core_density(h)

    with ClockSampler(local) as clocks:
        ms_per_step, per, dK_main = jk_steps(h, lib, dev, stream, D, C, prec, S, args.warmup, args.steps, ws)
    K_main = dK_main.clone()

    # end to end through the C ABI with host buffers (copies in and out inside the timed region)
    for _ in range(2):
        Jh, Kh = h.jk(D, C, prec, S)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _ in range(args.steps):
        Jh, Kh = h.jk(D, C, prec, S)
    e2e_s = max_over_ranks((time.perf_counter() - t1) / args.steps, dev)

    # comparisons on the same density: the early split form (3 slices) and the FP64 form, and the accuracy
    # of the split exchange against the FP64 exchange on the same B
    compare = {}
    k_accuracy = None
    if split:
        ms3, _, dK3 = jk_steps(h, lib, dev, stream, D, C, binding.DF_PREC_SPLIT, 3, 1, 3)
        compare["split_s3_s_per_iter"] = ms3 / 1000.0
        K3 = dK3.clone()
        if not args.no_fp64_compare:
            ms64, _, dK64 = jk_steps(h, lib, dev, stream, D, C, binding.DF_PREC_FP64, 0, 1, 2)
            compare["fp64_s_per_iter"] = ms64 / 1000.0
            kmax = float(dK64.abs().max())
            k_accuracy = {"density": "core-Hamiltonian orbitals", "max_abs_K": kmax,
                          f"S{S}_max_rel_dK_vs_fp64": float((K_main - dK64).abs().max()) / kmax,
                          "S3_max_rel_dK_vs_fp64": float((K3 - dK64).abs().max()) / kmax}

    # time to a converged SCF from the core-Hamiltonian guess (B already built: its build time is added),
    # and from the learned guess (network trained beforehand on smaller clusters; training not timed)
    ttc, scf_info, hist = {}, {}, {}
    if args.ttc:
        # split precision: S = 3 early, then a 5-slice reference K every 8 iterations with 3-slice
        # density-change builds in between (incremental Fock); "_full" keeps full 5-slice builds
        inc = 1 if split else 0
        runs = [("split" if split else "fp64", prec, None, inc),
                ("split_sad" if split else "fp64_sad", prec, "sad", inc)]
        if split:
            # the SAD start builds its first exchange from the atoms' occupied orbitals (7 per water) in blocks of
            # nocc and 2 per water columns: the autotuner's one-time choice for the second width is made here,
            # outside the timed runs
            nw = len(system.atoms) // 3
            h.jk(D, np.ascontiguousarray(C[:, :7 * nw - nocc]), prec, 3)
        if guess_net is not None:
            t0 = time.perf_counter()
            D0 = guess_net.guess(h)
            t_guess = time.perf_counter() - t0
            learned["t_guess_s"] = t_guess
            runs.append(("split_learned" if split else "fp64_learned", prec, (D0, t_guess), inc))
            if split:
                runs.append(("split_learned_full", prec, (D0, t_guess), 0))
        for label, p, g, inc_ in runs:
            res = h.scf(precision=p, slices=3, incremental=inc_, approx_diag=inc_,
                        guess=g if g is None or isinstance(g, str) else g[0])
            hrows = h.history()
            hist[label] = hrows[:, 1]
            ttc[label] = t_build + res["t_total_s"] + (g[1] if isinstance(g, tuple) else 0.0)
            scf_info[label] = _scf_info(res)
            # the last iterations' energy change and largest DIIS error element
            scf_info[label]["last_dE_err"] = [[float(f"{r[2]:.3g}"), float(f"{r[3]:.3g}")] for r in hrows[-6:]]

    peaks, peak_src = _peaks()
    keys = ["gamma_ms", "coulomb_ms", "ytransform_ms", "kcontract_ms", "split_ms", "split_y_ms", "split_k_ms",
            "split_other_ms"]
    avg = {k: float(np.mean([d[k] for d in per])) for k in keys}
    naux = h.naux
    b_bytes = naux * h.packed_row * 8.0
    packed_gb = h.naux * h.packed_row * 8 / 1e9
    tuned = per[-1]
    h.close()

    # the plain FP64 path end to end: B whitened in FP64, FP64 exchange, full eigensolves, from the
    # core-Hamiltonian guess; then the split SCF on that same B (energy difference due to the exchange's
    # precision alone)
    de = None
    if split and args.ttc and not args.no_fp64_ttc:
        with binding.Handle(system) as h64:
            res64 = h64.scf()
            hist["fp64"] = h64.history()[:, 1]
            ttc["fp64"] = res64["t_total_s"]
            scf_info["fp64"] = dict(_scf_info(res64), whitening="fp64", exchange="fp64")
            res_s = h64.scf(precision=binding.DF_PREC_SPLIT, slices=3, incremental=1, approx_diag=1)
            h_s = h64.history()[:, 1]
        a, b = h_s, hist["fp64"]
        m = min(len(a), len(b))
        de = {"same_B": {"B": "FP64 whitening", "at_convergence": float(res_s["energy"] - res64["energy"]),
                         "split_iterations": res_s["iterations"], "fp64_iterations": res64["iterations"],
                         "per_iteration": [float(f"{x:.3e}") for x in (a[:m] - b[:m])]},
              "split_vs_plain_fp64": {"at_convergence": float(scf_info["split"]["energy"] - res64["energy"]),
                                      "note": "split SCF on the tensor-core-whitened B against the plain FP64 "
                                              "path (FP64 whitening and exchange)"}}
        if "split_learned" in scf_info:
            de["split_learned_vs_plain_fp64"] = {"at_convergence": float(scf_info["split_learned"]["energy"]
                                                                         - res64["energy"])}

    # the 40-water configuration (n=2000, naux=5480, nocc=200): split J/K and time to converge
    c2 = None
    if split and args.ttc and args.c2:
        c2 = c2_measure(args, binding, clusters, lib, dev, stream, guess_net)
    if guess_net is not None:
        guess_net.close()

    clk_summary = clocks.summary()
    fp64pk = fp64_peak(binding, local, torch.cuda.get_device_properties(dev).multi_processor_count,
                       clk_summary.get("sm_mhz"))
    fp64_peak_tf = fp64pk["peak_tflops"]
    alg_k_flops = 2.0 * naux * n * n * nocc + 1.0 * naux * n * n * nocc   # Y = B C and K = sum Y Y^T
    if not split:
        flops = 2.0 * naux * n * n * nocc
        achieved = flops / (avg["ytransform_ms"] * 1e-3) / 1e12
        roofline = {"kernel": "y_transform_kernel (FP64 DFMA)", "bound": "alu", "achieved": achieved,
                    "peak": fp64_peak_tf, "unit": "TFLOP/s", "frac": achieved / fp64_peak_tf,
                    "peak_source": fp64pk["peak_source"], "traffic": None}
    else:
        npad = (n + 63) // 64 * 64
        ldy = (nocc + 31) // 32 * 32
        pairs = S * (S + 1) // 2
        nt = npad // 64
        y_hw = pairs * 2.0 * naux * npad * npad * ldy
        k_hw = pairs * 2.0 * (nt * (nt + 1) // 2) * 64 * 64 * naux * ldy
        y_tf = y_hw / (avg["split_y_ms"] * 1e-3) / 1e12
        k_tf = k_hw / (avg["split_k_ms"] * 1e-3) / 1e12
        dom_y = avg["split_y_ms"] >= avg["split_k_ms"]
        achieved = y_tf if dom_y else k_tf
        pk = peaks.get("bf16_tflops")
        tc = os.environ.get("DFHF_SPLIT_TC", "1") != "0" and S in (3, 5)
        kname = ("ozaki_tc_kernel<Y>" if dom_y else "ozaki_tc_kernel<K>") + " (tcgen05 BF16, TMEM, TMA)" if tc else \
            ("y_split_kernel" if dom_y else "k_split_kernel") + " (BF16 mma.sync)"
        tile = int(tuned.get("tc_y_tile_n" if dom_y else "tc_k_tile_n", 0))
        traffic = NCU_TRAFFIC.get((args.workload, "Y" if dom_y else "K", S, tile)) if tc else None
        roofline = {"kernel": kname + ", Ozaki slices",
                    "bound": "tensor", "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
                    "frac": achieved / pk if pk else None,
                    "peak_source": f"{peak_src} bf16_tflops (cuBLAS burst)",
                    "traffic": traffic,
                    "traffic_unit": "bytes per launch (ncu DRAM read + write)",
                    "algorithmic_bytes": (S * naux * npad * npad * 2 + naux * npad * ldy * 8) if dom_y else
                                         (S * naux * npad * ldy * 2),
                    "y_split_tflops": y_tf, "k_split_tflops": k_tf,
                    "k_split_frac": k_tf / pk if pk else None,
                    "fp64_equivalent_tflops": alg_k_flops / ((avg["split_y_ms"] + avg["split_k_ms"] + avg["split_other_ms"]) * 1e-3) / 1e12}
    kernel_ms = {k: round(v, 3) for k, v in avg.items()}
    # the other rows' rooflines: DF-J reads packed B twice (gamma, coulomb) against HBM and does one FMA per
    # element read against the FP64 pipe; the integral kernels write packed (P|mu nu) once (FP64 ALU bound);
    # whitening counts naux^2 * npair FP64-equivalent flops
    npair = n * (n + 1) // 2
    hbm = peaks.get("hbm_gbs")
    j_s = (avg["gamma_ms"] + avg["coulomb_ms"]) * 1e-3
    j_gbs = 2.0 * b_bytes / j_s / 1e9
    j_tf = 2.0 * 2.0 * naux * h.packed_row / j_s / 1e12
    eri_s = build_ms["eri3c_ms"] * 1e-3
    n_triples = int(len(system.aux)) * (len(system.basis) * (len(system.basis) + 1) // 2)
    wh_s = build_ms["whiten_ms"] * 1e-3
    other_rooflines = {
        "df_j": {"kernels": "gamma_kernel + coulomb_kernel (FP64)", "bound": "alu",
                 "algorithmic_bytes": 2.0 * b_bytes, "achieved_gbs": j_gbs, "hbm_peak": hbm,
                 "hbm_frac": j_gbs / hbm if hbm else None, "peak_source": f"{peak_src} hbm_gbs",
                 "fp64_tflops": j_tf, "fp64_frac": j_tf / fp64_peak_tf},
        "eri3c": {"kernels": "eri3c_kernel (FP64 Rys)", "bound": "alu",
                  "shell_triples": n_triples, "gtriples_per_s": n_triples / eri_s / 1e9,
                  "write_bytes": naux * npair * 8.0, "write_gbs": naux * npair * 8.0 / eri_s / 1e9,
                  "write_frac_of_hbm": naux * npair * 8.0 / eri_s / 1e9 / hbm if hbm else None},
        "whitening": {"kernels": ("ozaki_tc_kernel<W> (tcgen05 BF16, 7 slices)" if split else
                                  "dgemm_kernel (FP64 DFMA, in place by 64-row blocks)"),
                      "fp64_equivalent_flops": float(naux) * naux * npair,
                      "fp64_equivalent_tflops": float(naux) * naux * npair / wh_s / 1e12,
                      "vs_fp64_peak": float(naux) * naux * npair / wh_s / 1e12 / fp64_peak_tf},
    }
    autotune = {"y_tile_n": int(tuned.get("tc_y_tile_n", 0)), "k_tile_n": int(tuned.get("tc_k_tile_n", 0)),
                "k_split": int(tuned.get("tc_k_split", 0)),
                "tuning_ms_this_process": round(float(tuned.get("autotune_ms", 0.0)), 1)} if split else None

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(system, budget_s=args.cpu_budget)

    line = {
        "metric": METRIC, "value": ms_per_step / 1000.0, "unit": "s/iter (DF J+K build)",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": f"bf16 Ozaki x{S} slices, exact f32 chunk sums, f32x2 accumulate, f64 J" if split else "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: seeded water cluster, n={n}, naux={naux}, nocc={nocc}, "
                               f"packed B {packed_gb:.1f} GB",
                   "precision": args.precision + (f" (S={S})" if split else ""),
                   "l2": "inputs larger than L2 (B resident, no flush)",
                   "parallelism": f"replicas x{ws}"},
        "e2e": {"value": e2e_s, "unit": "s/iter (DF J+K build, host buffers)",
                "h2d_bytes_per_step": int(D.nbytes + C.nbytes), "d2h_bytes_per_step": int(Jh.nbytes + Kh.nbytes)},
        "gpu_launches": int(sum(d.get("jk_launches", launches_per_step(prec)) for d in per)),
        "roofline": roofline,
        "other_rooflines": other_rooflines,
        "fp64_peak": fp64pk,
        "kernel_ms": kernel_ms,
        "autotune": autotune,
        "compare": compare,
        "k_accuracy": k_accuracy,
        "build_B": {"wall_s": t_build, "eri3c_ms": build_ms["eri3c_ms"], "cholesky_ms": build_ms["cholesky_ms"],
                    "potrf_ms": build_ms.get("potrf_ms"), "trtri_ms": build_ms.get("trtri_ms"),
                    "whiten_ms": build_ms["whiten_ms"], "init_ms": build_ms["init_ms"],
                    "eri_triples": n_triples},
        "time_to_converge_s": ttc or None, "scf": scf_info or None, "dE_split_vs_fp64": de,
        "c2_water40": c2,
        "batched": None,
        "learned_guess": learned,
        "clocks": clocks.summary(),
        "cpu_baseline": cpu,
    }
    # many small clusters, after the large cluster's tensors have left the device
    if args.batch > 0:
        line["batched"] = batched_measure(binding, clusters, args.batch, torch, rank, dev, args.batch_max_waters)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        tdist.destroy_process_group()


def c2_measure(args, binding, clusters, lib, dev, stream, guess_net):
    """The 40-water cluster (n=2000, naux=5480, nocc=200): B build, split J/K per iteration (5 and 3 slices)
    and one FP64 J/K build on the same density, then split SCFs to convergence from the core-Hamiltonian and
    the learned guess (incremental Fock and approximate diagonalisation late)."""
    import torch
    system = clusters.workload("water40")
    out = {"workload": f"water40: seeded water cluster, n={system.nbf}, naux={system.naux}, nocc={system.nocc}"}
    t0 = time.perf_counter()
    with binding.Handle(system) as h:
        h.build_B()
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        bms = h.timings()
        out["build_B"] = {"wall_s": t_build, "eri3c_ms": bms["eri3c_ms"], "cholesky_ms": bms["cholesky_ms"],
                          "whiten_ms": bms["whiten_ms"]}
        out["packed_B_gb"] = h.naux * h.packed_row * 8 / 1e9
        C, D = core_density(h)
        ms5, per5, _ = jk_steps(h, lib, dev, stream, D, C, binding.DF_PREC_SPLIT, 5, 1, 3)
        ms3, _, _ = jk_steps(h, lib, dev, stream, D, C, binding.DF_PREC_SPLIT, 3, 1, 2)
        ms64, _, _ = jk_steps(h, lib, dev, stream, D, C, binding.DF_PREC_FP64, 0, 0, 1)
        out["jk_s_per_iter"] = {"split_s5": ms5 / 1000, "split_s3": ms3 / 1000, "fp64": ms64 / 1000}
        out["split_s5_kernel_ms"] = {k: round(float(np.mean([d[k] for d in per5])), 3)
                                     for k in ("gamma_ms", "coulomb_ms", "split_y_ms", "split_k_ms", "split_other_ms")}
        res = h.scf(precision=binding.DF_PREC_SPLIT, slices=3, incremental=1, approx_diag=1)
        out["ttc_split_s"] = t_build + res["t_total_s"]
        out["scf_split"] = _scf_info(res)
        nw = len(system.atoms) // 3
        h.jk(D, np.ascontiguousarray(C[:, :7 * nw - h.nocc]), binding.DF_PREC_SPLIT, 3)   # tuner warm-up (SAD)
        res_s = h.scf(precision=binding.DF_PREC_SPLIT, slices=3, incremental=1, approx_diag=1, guess="sad")
        out["ttc_split_sad_s"] = t_build + res_s["t_total_s"]
        out["scf_split_sad"] = _scf_info(res_s)
        out["dE_sad_vs_core"] = res_s["energy"] - res["energy"]
        if guess_net is not None:
            t1 = time.perf_counter()
            D0 = guess_net.guess(h)
            t_guess = time.perf_counter() - t1
            res_l = h.scf(precision=binding.DF_PREC_SPLIT, slices=3, incremental=1, approx_diag=1, guess=D0)
            out["ttc_split_learned_s"] = t_build + res_l["t_total_s"] + t_guess
            out["scf_split_learned"] = _scf_info(res_l)
            out["dE_learned_vs_core"] = res_l["energy"] - res["energy"]
    return out


class GuessNets:
    """The learned guess's two networks: each water's diagonal block and the blocks of water pairs within
    binding.PAIR_CUTOFF."""

    def __init__(self, diag, pair):
        self.diag, self.pair = diag, pair

    def guess(self, h):
        return h.mlp_guess(self.diag, bf16=True, pair_mlp=self.pair)

    def close(self):
        self.diag.close()
        self.pair.close()


def _fit(binding, X, Y, nin, epochs, batch, seed):
    """A 256 x 3 ReLU network fitted to (X, Y), its last layer started at the mean target (zero weights)."""
    nout = Y.shape[1]
    net = binding.Mlp(nin, 256, 3, nout, seed=seed)
    p = net.params()
    p[-nout:] = Y.mean(axis=0)
    p[-nout - nout * 256:-nout] = 0.0
    net.set_params(p)
    hist = net.train(X, Y, epochs=epochs, batch=batch, lr=3e-4, seed=seed + 1)
    return net, hist


def train_guess(binding, clusters, members, epochs=200, precision=None):
    """Train the density-guess networks on the converged densities of the seeded clusters `members`
    ((waters, seed) pairs), generated by this library's SCF. Returns (GuessNets, summary)."""
    import torch
    t0 = time.perf_counter()
    systems = [clusters.water_cluster(w, seed) for w, seed in members]
    X = [binding.water_features(s) for s in systems]
    pair_lists = [binding.water_pairs(s) for s in systems]
    Y = [None] * len(systems)
    YP = [None] * len(systems)

    def keep(k, hh, res):
        if not res["converged"]:
            raise RuntimeError(f"training cluster {members[k]} did not converge")
        D = hh.matrix("D")
        Y[k] = hh.water_blocks(D)
        pairs = pair_lists[k][0]
        YP[k] = hh.pair_blocks(D, pairs).reshape(len(pairs), -1)

    # the converged densities come from the batched SCF, in waves planned against the free device memory
    free, _ = torch.cuda.mem_get_info()
    binding.scf_waves(systems, int(0.5 * free), precision=binding.DF_PREC_FP64 if precision is None else precision,
                      slices=3, on_done=keep, **({} if precision is None else dict(incremental=1, approx_diag=1)))
    t_data = time.perf_counter() - t0
    X, Y = np.concatenate(X), np.concatenate(Y)
    XP = np.concatenate([pl[1] for pl in pair_lists])
    YP = np.concatenate(YP)
    t0 = time.perf_counter()
    net, hist = _fit(binding, X, Y, binding.DF_MLP_NFEAT, epochs, 16, 7)
    # the pair network sees about 3 samples per water: larger batches, and at most about 60000 steps
    ep_pair = int(min(epochs, max(10, 60000 * 64 // max(1, len(XP)))))
    pnet, hist_p = _fit(binding, XP, YP, binding.DF_MLP_NPFEAT, ep_pair, 64, 17)
    t_train = time.perf_counter() - t0
    nbw = int(round(np.sqrt(YP.shape[1])))
    return GuessNets(net, pnet), {
        "train_clusters": len(members), "train_waters": int(sum(w for w, _ in members)),
        "train_samples": int(len(X)), "network": f"57-256x3-{Y.shape[1]} ReLU, FP32 weights, BF16 inference",
        "epochs": epochs, "loss_first": float(hist[0]), "loss_last": float(hist[-1]),
        "pair_cutoff_bohr": binding.PAIR_CUTOFF, "pair_samples": int(len(XP)),
        "pair_network": f"{binding.DF_MLP_NPFEAT}-256x3-{nbw * nbw} ReLU, FP32 weights, BF16 inference",
        "pair_epochs": ep_pair, "pair_loss_first": float(hist_p[0]), "pair_loss_last": float(hist_p[-1]),
        "t_data_s": t_data, "t_train_s": t_train}


def learned_guess_net(binding, clusters, n_train):
    """The density-guess network trained on `n_train` seeded clusters of 4-14 waters (seeds 10000+,
    converged densities of the split-precision SCF). Trained before the benchmark cluster's tensors take
    the device memory; the training is an offline step and not part of the time to converge."""
    rng = clusters.SplitMix64(9090)
    members = [(4 + min(10, int(rng.uniform() * 11)), 10000 + k) for k in range(n_train)]
    return train_guess(binding, clusters, members, precision=binding.DF_PREC_SPLIT)


def guess_study(args):
    """The learned guess on held-out clusters: train on n_train clusters of 4-24 waters (seeds 10000+),
    evaluate on n_eval clusters of 8-32 waters (seeds 20000+) against the core-Hamiltonian and SAD guesses,
    with the diagonal and pair networks and with the diagonal network alone, all with the split-precision
    SCF (incremental Fock late). Prints one JSON line."""
    from paper_1707_03771_gb300 import binding, build, clusters
    build.build()
    binding.load()
    n_train, n_eval = (int(x) for x in args.guess_study.split(","))
    rng = clusters.SplitMix64(7070)
    train = [(4 + min(20, int(rng.uniform() * 21)), 10000 + k) for k in range(n_train)]
    evals = [(8 + min(24, int(rng.uniform() * 25)), 20000 + k) for k in range(n_eval)]
    prec = binding.DF_PREC_SPLIT
    if args.guess_net and os.path.exists(args.guess_net):
        # networks saved by an earlier run of the same study (same training set and epochs)
        with np.load(args.guess_net) as f:
            summary = json.loads(str(f["summary"]))
            if summary["train_clusters"] != n_train or summary["epochs"] != args.guess_epochs:
                raise SystemExit(f"{args.guess_net} holds networks trained on {summary['train_clusters']} "
                                 f"clusters for {summary['epochs']} epochs")
            net = binding.Mlp(binding.DF_MLP_NFEAT, 256, 3, int(f["nout"]), seed=7)
            net.set_params(f["params"])
            pnet = binding.Mlp(binding.DF_MLP_NPFEAT, 256, 3, int(f["nout_pair"]), seed=17)
            pnet.set_params(f["params_pair"])
        nets = GuessNets(net, pnet)
        summary["loaded_from_file"] = True
    else:
        nets, summary = train_guess(binding, clusters, train, epochs=args.guess_epochs, precision=prec)
        if args.guess_net:
            np.savez(args.guess_net, params=nets.diag.params(), nout=nets.diag.nout, params_pair=nets.pair.params(),
                     nout_pair=nets.pair.nout, summary=json.dumps(summary))
    print(json.dumps({"training": summary}), file=sys.stderr, flush=True)
    lo, hi = (int(x) for x in args.guess_eval_range.split(":")) if args.guess_eval_range else (0, n_eval)
    rows = []
    for w, seed in evals[lo:hi]:
        with binding.Handle(clusters.water_cluster(w, seed)) as h:
            h.build_B()
            core = h.scf(precision=prec, slices=3, incremental=1, approx_diag=1)
            sadr = h.scf(precision=prec, slices=3, incremental=1, approx_diag=1, guess="sad")
            t0 = time.perf_counter()
            D0 = nets.guess(h)
            t_guess = time.perf_counter() - t0
            lrn = h.scf(precision=prec, slices=3, incremental=1, approx_diag=1, guess=D0)
            # the same diagonal network without the pair blocks
            lrd = h.scf(precision=prec, slices=3, incremental=1, approx_diag=1, guess=h.mlp_guess(nets.diag, bf16=True))
        rows.append({"waters": w, "seed": seed, "iterations_core": core["iterations"],
                     "iterations_sad": sadr["iterations"], "iterations_learned": lrn["iterations"],
                     "iterations_learned_diag": lrd["iterations"],
                     "t_scf_core_s": core["t_total_s"], "t_scf_sad_s": sadr["t_total_s"],
                     "t_scf_learned_s": lrn["t_total_s"] + t_guess,
                     "dE_learned_vs_core": lrn["energy"] - core["energy"],
                     "dE_learned_diag_vs_core": lrd["energy"] - core["energy"],
                     "dE_sad_vs_core": sadr["energy"] - core["energy"],
                     "converged": bool(core["converged"] and lrn["converged"] and sadr["converged"]
                                       and lrd["converged"])})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)   # progress, one line per held-out cluster
    nets.close()
    it_c = [r["iterations_core"] for r in rows]
    it_s = [r["iterations_sad"] for r in rows]
    it_l = [r["iterations_learned"] for r in rows]
    print(json.dumps({"study": "learned initial guess on held-out clusters", "training": summary,
                      "eval_clusters": n_eval, "eval_range": [lo, hi], "mean_iterations_core": float(np.mean(it_c)),
                      "mean_iterations_sad": float(np.mean(it_s)),
                      "mean_iterations_learned": float(np.mean(it_l)),
                      "mean_iterations_learned_diag_only": float(np.mean([r["iterations_learned_diag"] for r in rows])),
                      "iterations_saved_vs_core": 1.0 - float(np.sum(it_l)) / float(np.sum(it_c)),
                      "iterations_saved_vs_sad": 1.0 - float(np.sum(it_l)) / float(np.sum(it_s)),
                      "time_saved_vs_sad": 1.0 - float(sum(r["t_scf_learned_s"] for r in rows))
                                           / float(sum(r["t_scf_sad_s"] for r in rows)),
                      "max_abs_dE_learned_vs_core": float(max(max(abs(r["dE_learned_vs_core"]),
                                                                   abs(r["dE_learned_diag_vs_core"])) for r in rows)),
                      "max_abs_dE_sad_vs_core": float(max(abs(r["dE_sad_vs_core"]) for r in rows)),
                      "all_converged": all(r["converged"] for r in rows), "clusters": rows}))


def _oracle_scf_child(name):
    """The oracle's whole DF-RHF (integrals, whitening, SCF) on one workload; prints one JSON line."""
    from oracle import dfrhf
    from paper_1707_03771_gb300 import clusters
    s = clusters.workload(name)
    dfrhf.build()
    t0 = time.perf_counter()
    r = dfrhf.scf(s)
    print(json.dumps({"t_s": time.perf_counter() - t0, "energy": r.energy, "iterations": r.iterations}))


def open_shell_study(args):
    """DF-UHF and DF-ROHF on the GPU: for each named workload, the cation (one electron removed: a doublet)
    with B built once, UHF and ROHF to convergence in FP64 and in split precision (3 slices, then 5). Prints
    one JSON line with times, iterations, energies and <S^2>."""
    import copy

    from paper_1707_03771_gb300 import binding, build, clusters
    build.build()
    binding.load()
    rows = []
    for name in args.open_shell.split(","):
        system = copy.deepcopy(clusters.workload(name))
        system.charge = 1
        ne = system.n_electrons
        na, nb = (ne + 1) // 2, ne // 2
        with binding.Handle(system, open_shell=True) as h:
            t0 = time.perf_counter()
            h.build_B()
            t_build = time.perf_counter() - t0
            row = {"workload": name, "n": h.n, "naux": h.naux, "nalpha": na, "nbeta": nb, "t_build_B_s": t_build}
            # FP64 exchange builds up to 800 basis functions (at 1600 one FP64 iteration of UHF takes ~10 s)
            precs = (("fp64", binding.DF_PREC_FP64), ("split", binding.DF_PREC_SPLIT)) if h.n <= 800 else \
                (("split", binding.DF_PREC_SPLIT),)
            for label, prec in precs:
                # UHF from the core Hamiltonian, ROHF, then UHF from the ROHF spin densities
                for kind in ("uhf", "rohf", "uhf_from_rohf"):
                    if kind == "rohf":
                        r = h.scf_rohf(na, nb, precision=prec, slices=3)
                    else:
                        r = h.scf_uhf(na, nb, precision=prec, slices=3, guess="spin" if kind != "uhf" else "core")
                    row[f"{kind}_{label}"] = {"energy": r["energy"], "iterations": r["iterations"],
                                              "converged": bool(r["converged"]), "s2": r["s2"],
                                              "t_total_s": r["t_total_s"], "t_jk_s": r["t_jk_s"]}
            for kind in ("uhf", "rohf", "uhf_from_rohf"):
                if f"{kind}_fp64" in row:
                    row[f"dE_{kind}_split_vs_fp64"] = row[f"{kind}_split"]["energy"] - row[f"{kind}_fp64"]["energy"]
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"study": "DF-UHF and DF-ROHF of water-cluster cations", "workloads": rows}))


def mp2_study(args):
    """DF-MP2 on the GPU: for each named workload, B and the FP64 SCF, then df_mp2 of its canonical orbitals
    (FP64). Prints one JSON line with times and energies."""
    from paper_1707_03771_gb300 import binding, build, clusters
    build.build()
    binding.load()
    rows = []
    for name in args.mp2.split(","):
        system = clusters.workload(name)
        with binding.Handle(system) as h:
            r = h.scf()
            nmo = h.n - r["n_dropped"]
            t0 = time.perf_counter()
            e2 = h.mp2(n_dropped=r["n_dropped"])
            t_mp2 = time.perf_counter() - t0
            nocc, nvir = h.nocc, nmo - h.nocc
            # FP64 work: the second transformation 2 naux nvir nocc n, the pair integrals over j <= i
            flops = 2.0 * h.naux * nvir * nocc * h.n + 2.0 * nvir * nvir * h.naux * nocc * (nocc + 1) / 2
            rows.append({"workload": name, "n": h.n, "naux": h.naux, "nocc": nocc, "nvir": nvir,
                         "e_scf": r["energy"], "e_mp2_corr": e2, "t_scf_s": r["t_total_s"], "t_mp2_s": t_mp2,
                         "mp2_fp64_gflop": flops / 1e9, "mp2_fp64_tflops": flops / t_mp2 / 1e12})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"study": "DF-MP2 correlation energy (FP64) of water clusters", "workloads": rows}))


def oracle_scf_study(args):
    """Whole SCF runs beside the oracle on the same host: for each workload, the GPU FP64 and split-precision
    SCF (B built and timed) and the oracle's DF-RHF on all host cores, and on one core for workloads of at
    most 100 basis functions. The oracle runs in child processes. Prints one JSON line."""
    import torch
    from paper_1707_03771_gb300 import binding, build, clusters
    build.build()
    binding.load()
    rows = []
    for name in args.oracle_scf.split(","):
        s = clusters.workload(name)
        row = {"workload": name, "n": s.nbf, "naux": s.naux, "nocc": s.nocc}
        with binding.Handle(s) as h:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.build_B()
            torch.cuda.synchronize()
            t_build = time.perf_counter() - t0
            for label, p, inc in (("gpu_fp64", binding.DF_PREC_FP64, 0), ("gpu_split", binding.DF_PREC_SPLIT, 1)):
                r = h.scf(precision=p, slices=3, incremental=inc, approx_diag=inc)
                row[label] = {"t_s": t_build + r["t_total_s"], "energy": r["energy"],
                              "iterations": r["iterations"], "converged": bool(r["converged"])}
        threads = [("oracle", os.cpu_count())] + ([("oracle_1_thread", 1)] if s.nbf <= 100 else [])
        for label, nt in threads:
            env = dict(os.environ)
            if nt == 1:
                env.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
            out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-scf-child", name],
                                 env=env, capture_output=True, text=True, check=True)
            row[label] = dict(json.loads(out.stdout.strip().splitlines()[-1]), cores=nt)
        row["dE_gpu_fp64_vs_oracle"] = row["gpu_fp64"]["energy"] - row["oracle"]["energy"]
        row["dE_gpu_split_vs_oracle"] = row["gpu_split"]["energy"] - row["oracle"]["energy"]
        rows.append(row)
    print(json.dumps({"study": "whole SCF: GPU (build B + SCF) beside the oracle on the host cores",
                      "workloads": rows}))


def batched_measure(binding, clusters, count, torch, rank=0, dev=None, wmax=8):
    """Many small clusters (batch_members): time to converge all of them with the split-precision SCF,
    one after another versus together (scf_run_batch in waves); times are the maximum over ranks."""
    members = batch_members(count, rank, wmax)
    sizes = [w for w, _ in members]
    systems = [clusters.water_cluster(w, seed) for w, seed in members]
    prec = binding.DF_PREC_SPLIT
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq = []
    for s in systems:
        with binding.Handle(s) as h:
            seq.append(h.scf(precision=prec, slices=3, incremental=1, approx_diag=1))
    torch.cuda.synchronize()
    t_seq = max_over_ranks(time.perf_counter() - t0, dev)
    free, _ = torch.cuda.mem_get_info()
    t0 = time.perf_counter()
    res = binding.scf_waves(systems, int(0.5 * free), precision=prec, slices=3, incremental=1, approx_diag=1)
    torch.cuda.synchronize()
    t_batch = max_over_ranks(time.perf_counter() - t0, dev)
    de = max(abs(a["energy"] - b["energy"]) for a, b in zip(seq, res))
    return {"molecules": count, "waters": sizes, "basis_functions": int(sum(s.nbf for s in systems)),
            "t_sequential_s": t_seq, "t_batched_s": t_batch, "speedup": t_seq / t_batch,
            "all_converged": bool(all(r["converged"] for r in res)), "max_abs_dE_batch_vs_single": de,
            "precision": "split (3 slices early; late: 5-slice reference + 3-slice incremental builds, "
                         "approximate diagonalisation)"}


def ctypes_ptr(v):
    import ctypes
    return ctypes.c_void_p(v)


def launches_per_step(precision):
    # J: pack D, gamma, coulomb, split-sum, unpack; pad C; then FP64 K: Y transform, K contraction, K reduce,
    # or split K: split C, split Y-GEMM, re-split Y, split K contraction, reduce
    return 9 if precision == 0 else 11


def _oracle_jk_sample(system, rows, rng):
    """Oracle J/K (eqs. 1-3) on `rows` auxiliary rows of a synthetic B with the workload's shape."""
    from oracle import dfrhf
    n, nocc = system.nbf, system.nocc
    B = rng.standard_normal((rows, n, n))
    B = 0.5 * (B + B.transpose(0, 2, 1))
    C = rng.standard_normal((n, nocc))
    D = 2 * C @ C.T
    t0 = time.perf_counter()
    dfrhf.df_J(B, D)
    dfrhf.df_K(B, C)
    return time.perf_counter() - t0


def cpu_baseline(system, budget_s=15.0):
    """The oracle's J/K contraction (numpy, as it stands) on a bounded sample of auxiliary rows,
    scaled linearly to all naux rows (the cost of eqs. 1-3 is linear in naux)."""
    rng = np.random.default_rng(0)
    rows = 2
    t = _oracle_jk_sample(system, rows, rng)
    while t < budget_s / 4 and rows < 64:
        rows *= 2
        t = _oracle_jk_sample(system, rows, rng)
    per_iter = t / rows * system.naux
    try:
        import numpy.__config__  # noqa: F401
        threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    except Exception:
        threads = os.cpu_count()
    return {"value": per_iter, "unit": "s/iter (DF J+K build)", "cores": threads, "kind": "oracle",
            "sample": f"oracle df_J + df_K on {rows} of {system.naux} auxiliary rows "
                      f"(n={system.nbf}, nocc={system.nocc}), {t:.1f} s, scaled by naux/{rows}"}


def reference_arm(args):
    """The oracle (numpy DF J/K, eqs. 1-3) on the host cores. One step times the oracle's J and K on a
    bounded sample of 4 auxiliary rows of the workload; `value` scales the per-row cost to all naux rows
    (the cost of eqs. 1-3 is linear in naux), while `ms_per_step` is the measured time of the sampled
    step, so steps x ms_per_step is the timed region."""
    ws, rank = _dist()
    if rank != 0:
        return
    from paper_1707_03771_gb300 import clusters
    system = clusters.workload(args.workload)
    rng = np.random.default_rng(1)
    rows = 4
    for _ in range(args.warmup):
        _oracle_jk_sample(system, rows, rng)
    t = [_oracle_jk_sample(system, rows, rng) for _ in range(args.steps)]
    v = float(np.mean(t)) / rows * system.naux
    cores = os.cpu_count()
    sample = (f"oracle df_J + df_K on {rows} of {system.naux} auxiliary rows per step "
              f"({float(np.mean(t)):.2f} s measured per step), scaled by naux/{rows}")
    line = {"metric": METRIC, "value": v, "unit": "s/iter (DF J+K build)", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean(t)) * 1000, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "extrapolated": {"measured_rows_per_step": rows, "naux": system.naux,
                             "value_is": "measured time per row x naux"},
            "config": {"workload": f"{args.workload}: seeded water cluster, n={system.nbf}, naux={system.naux}, "
                                   f"nocc={system.nocc}", "precision": "fp64"},
            "cpu_baseline": {"value": v, "unit": "s/iter (DF J+K build)", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "s/iter (DF J+K build)", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="split", choices=["fp64", "split"])
    ap.add_argument("--slices", type=int, default=5, help="slices of the timed split builds (the late-SCF precision)")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-fp64-ttc", action="store_true",
                    help="skip the plain FP64 SCF to convergence (FP64 whitening and exchange; minutes)")
    ap.add_argument("--no-c2", dest="c2", action="store_false", help="skip the 40-water measurement")
    ap.add_argument("--no-ttc", dest="ttc", action="store_false")
    ap.add_argument("--batch", type=int, default=256, help="molecules in the batched-SCF measurement (0: skip)")
    ap.add_argument("--batch-max-waters", type=int, default=16, help="cluster sizes 1..W in the batched measurement")
    ap.add_argument("--guess-study", default=None, metavar="NTRAIN,NEVAL",
                    help="only the learned-guess study on held-out clusters (one JSON line)")
    ap.add_argument("--guess-epochs", type=int, default=200)
    ap.add_argument("--guess-net", default=None, metavar="NPZ",
                    help="guess study: load the trained network from this file if it exists, else save it there")
    ap.add_argument("--guess-eval-range", default=None, metavar="LO:HI",
                    help="guess study: evaluate only held-out clusters LO..HI-1")
    ap.add_argument("--learned", type=int, default=32, help="training clusters for the learned guess (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--oracle-scf", default=None, metavar="WORKLOADS",
                    help="only whole SCF runs, GPU beside the oracle, e.g. water2,water8 (one JSON line)")
    ap.add_argument("--oracle-scf-child", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--mp2", default=None, metavar="WORKLOADS",
                    help="only DF-MP2 after the FP64 SCF of these workloads, e.g. water8,water16 (one JSON line)")
    ap.add_argument("--open-shell", default=None, metavar="WORKLOADS",
                    help="only DF-UHF and DF-ROHF of the cations of these workloads, e.g. water8,water32 (one JSON line)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.oracle_scf_child:
        _oracle_scf_child(args.oracle_scf_child)
    elif args.open_shell:
        open_shell_study(args)
    elif args.mp2:
        mp2_study(args)
    elif args.oracle_scf:
        oracle_scf_study(args)
    elif args.guess_study:
        guess_study(args)
    elif args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
