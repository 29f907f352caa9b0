#!/usr/bin/env python3
"""Benchmark of the GB300 Ito-KMC step (one JSON line on rank 0).

Workload: the single-positive-streamer configuration -- 256^3 cells over a
2 cm cube, 1.5 MV/m applied, dt = 5 ps, ppc = 32, photoionization on -- with
a synthetic developed discharge tree (4 channels, Gaussian radial profile,
peak 1e19 m^-3) sampled to ``--particles`` superparticles and quasi-neutral
ion counts with a positive head charge at each channel tip.  A step is one
full pass of the hot path: interpolate, push, sort, deposit (a1-a4), KMC
(a6), products, photons and merge/split (a7-a9) and the multigrid field
solve (a5).  The particle records (GBs) exceed the 129 MB L2, so no flush is
needed between steps.

--impl reference times the FP64 CPU oracle (its OpenMP build on every core the
process may use; the arithmetic as it stands) on a bounded sample of the same
workload per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# DRAM bytes per particle of the transport stage (push, transport scans,
# scatter, mover kernels): dram__bytes_read.sum + dram__bytes_write.sum of
# those kernels in one ncu capture of the streamer workload at 128^3 (9.97e6
# particles, one transport stage, the same kernels as the timed run), divided
# by its particles, keyed by "FP64 form"; multiplied by the timed run's
# particle count (both grids hold about the same particles per cell, so the
# per-cell arrays weigh alike per particle; the 256^3 field array no longer
# fits in L2, which makes the full-size figure somewhat higher).  Captured:
# FP64 1.401 GB, mixed 0.855 GB.  The cudaMemsetAsync zeroing of the
# per-cell count arrays is not a kernel and is not in the figure.
TRANSPORT_DRAM_PER_PARTICLE = {True: 140.5, False: 85.8}
# FP64 arithmetic of the FP64 push per particle (ncu thread-instruction counts
# of DADD, DMUL and DFMA over a launch, divided by its particles; an FMA
# counts as two operations: 12.4 + 30.6 + 2 x 37.1).  The peak it is set
# against is measured in the run (itokmc_probe_fp64_peak: register-resident
# FMA chains on every SM).
FP64_FLOP_PER_PARTICLE = 117.3

METRIC = "particle-steps/s (push+sort+deposit+KMC), HBM roofline %; FP32 vs FP64 at stated err"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ workload
def workload(args):
    from paper_2307_01797_gb300 import synth
    ph = synth.physics_streamer(args.n)
    if getattr(args, "recombination", False):
        ph = synth.with_recombination(ph)
    if getattr(args, "mobile_ions", False):
        ph = synth.with_mobile_ions(ph)
        ph["mobile_ions"] = True
    st = synth.streamer_tree_state(ph, int(args.particles), seed=7)
    ions = synth.streamer_ions(ph, st, seed=8)
    return ph, st, ions


# ------------------------------------------------------------------ clocks
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(ph, st, ions, max_particles, seed):
    """A bounded sample of the workload for the oracle: the particles of a
    contiguous run of cells (canonical order) holding about max_particles."""
    import oracle
    p = oracle.make_params(ph, seed=seed)
    S = oracle.canonical(p, st)
    N = len(S["w"])
    start = N // 2 - max_particles // 2 if N > max_particles else 0
    sl = slice(max(start, 0), max(start, 0) + max_particles)
    sub = {k: v[sl] for k, v in S.items()}
    n3 = ph["n"] ** 3
    sub["Npos"] = np.asarray(ions[0], np.int64)
    sub["Nneg"] = np.asarray(ions[1], np.int64)
    return sub


def time_oracle_step(ph, sub, E, step, seed):
    """push + sort + deposit + KMC of the oracle on the sample (the metric's
    scope); returns (seconds, particles)."""
    import oracle
    p = oracle.make_params(ph, seed=seed, step=step)
    t0 = time.perf_counter()
    xo, yo, zo, cell = oracle.push(p, sub["x"], sub["y"], sub["z"], E)
    perm = oracle.sort_by_cell(cell, ph["n"] ** 3)
    ne, Xe = oracle.deposit(p, xo[perm], yo[perm], zo[perm], sub["w"][perm], cell[perm])
    oracle.kmc(p, Xe, E)
    return time.perf_counter() - t0, len(sub["w"])


def reference_arm(args, rank, world):
    if rank != 0:
        return
    from paper_2307_01797_gb300 import synth
    ph, st, ions = workload(args)
    E = synth.random_field(ph, seed=3, amp=1e6, base=ph["E0"])
    import oracle
    oracle.use_openmp(True)
    ncores = len(os.sched_getaffinity(0))
    sub = oracle_sample(ph, st, ions, args.ref_particles, seed=1)
    for w in range(args.warmup):
        time_oracle_step(ph, sub, E, w, 1)
    tot_t, tot_n = 0.0, 0
    for k in range(args.steps):
        t, n = time_oracle_step(ph, sub, E, args.warmup + k, 1)
        tot_t += t
        tot_n += n
    v = tot_n / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "particle-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(args, len(st["w"])),
            "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": ncores, "kind": "oracle",
                             "sample": f"{len(sub['w'])} particles of a contiguous cell run of the workload, "
                                       "push+sort+deposit+KMC per step on the full grid, the C oracle's OpenMP "
                                       "build on every core of the process's affinity"},
            "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(args, nparticles, fp64=True):
    return {"workload": f"single positive streamer, {args.n}^3 cells over a 2 cm cube, 1.5 MV/m, dt 5 ps, ppc 32, "
                        f"photoionization on, synthetic 4-channel discharge tree",
            "grid": args.n, "particles": int(nparticles), "ppc": 32,
            "form": "fp64 plain" if fp64 else "mixed (fp32 + fixed point)",
            "chemistry": ("ionization, attachment, photon emission, e-ion and ion-ion recombination (air)"
                          if getattr(args, "recombination", False) else "ionization, attachment, photon emission"),
            "ions": ("Ito particles (mu_ion 2e-4 m^2/Vs, D from the Einstein relation)"
                     if getattr(args, "mobile_ions", False) else "per-cell counts"),
            "l2": "inputs > L2 (particle records of several GB; no flush)"}


# ------------------------------------------------------------------ our arm
def aggregate_ranks(ms, processed, dist, device):
    """Whole-job figures of a replica run: the slowest rank's time (max over
    ranks) and the particle-steps of all ranks (sum); identity on one rank."""
    if not dist:
        return float(ms), float(processed)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([float(processed)], dtype=torch.float64, device=device)
    dist.all_reduce(p)
    return float(t.item()), float(p.item())


def run_form(args, itokmc, form, ph, st, ions, rank, world, dist, dev, with_e2e):
    """Warm up and time args.steps full steps of one form on the workload;
    returns the measurements (rank-local) and the handle's stats."""
    import torch
    from paper_2307_01797_gb300 import synth
    N0 = len(st["w"])
    mobile = bool(ph.get("mobile_ions", False))
    if mobile:
        # the ion counts as ion superparticles (the merge brings every species
        # to ppc per occupied cell within a step)
        ip = synth.ions_from_counts(ph, ions[0], seed=9, per_cell=ph["ppc"])
        N0 += len(ip["w"])
    # photoelectrons landing in empty cells are split up to ppc particles each,
    # so the count grows from step to step
    cap = int(N0 * args.cap_factor) + 20_000_000
    H = itokmc.Handle(itokmc.make_config(ph, cap, seed0=1 + rank, precision=form))
    if mobile:
        sp = np.concatenate([np.zeros(len(st["w"]), np.int32), np.ones(len(ip["w"]), np.int32)])
        H.itokmc_set_particles_species(*(np.concatenate([st[k], ip[k]]) for k in ("x", "y", "z", "w")), sp)
    else:
        H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
        H.itokmc_set_ions(*ions)
    H.itokmc_solve_field()
    tune = None if args.no_tune else H.itokmc_autotune()
    for _ in range(args.warmup):
        H.itokmc_step(1)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = H.itokmc_get_stats()["kernel_launches"]
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stage = {"transport": 0.0, "kmc": 0.0, "particles": 0.0, "field": 0.0}
    processed = 0
    movers = 0
    mg_cycles = []
    counts = []
    last = {}
    e0.record(stream)
    for _ in range(args.steps):
        nk = H.itokmc_num_particles()
        counts.append(nk)
        processed += nk
        H.itokmc_step(1)
        s = H.itokmc_get_stats()
        stage["transport"] += s["ms_transport"]; stage["kmc"] += s["ms_kmc"]
        stage["particles"] += s["ms_particles"]; stage["field"] += s["ms_field"]
        movers += s["n_movers"]
        mg_cycles.append(s["mg_cycles"])
        last = {k: s[k] for k in ("merge_cells", "merge_elements", "merge_elements_sq", "merge_max_list",
                                  "n_new_particles", "photon_emissions", "ionizations", "attachments", "recombinations_ep",
                                  "recombinations_np",
                                  "mg_rel_residual")}
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = H.itokmc_get_stats()["kernel_launches"] - l0
    ms, processed_all = aggregate_ranks(e0.elapsed_time(e1), processed, dist, "cuda")
    # push+sort+deposit+KMC scope (stage times from CUDA events on the
    # library's stream)
    core_ms = stage["transport"] + stage["kmc"]
    # roofline of the transport stage (push + sort + deposit, the metric's
    # particle stream): algorithmic bytes = read + write of every record plus
    # the per-cell mesh terms amortised over ppc
    R = 32 if form == itokmc.FP64 else 20
    mesh = (24 + 8 + 8) if form == itokmc.FP64 else (12 + 8 + 8)
    bpp = 2 * R + mesh / 32
    ach = processed * bpp / (stage["transport"] / 1e3) / 1e9
    # measured DRAM bytes of the same stage (dram__bytes_read.sum +
    # dram__bytes_write.sum of its kernels in one ncu capture of the same
    # kernels on a smaller case), per step at the timed mean particle count
    tpp = TRANSPORT_DRAM_PER_PARTICLE[form == itokmc.FP64]
    traffic = tpp * processed / args.steps if tpp else None
    out = {"value": processed_all / (ms / 1e3), "ms_per_step": ms / args.steps,
           "push_sort_deposit_kmc_rate": processed / (core_ms / 1e3),
           "stage_ms_per_step": {k: v / args.steps for k, v in stage.items()},
           "movers_per_step": movers / args.steps, "mg_cycles": mg_cycles, "particles_per_step": counts,
           "last_step_counters": last, "gpu_launches": int(launches), "clocks": clk,
           "transport_achieved_gbs": ach, "bytes_per_particle": bpp, "traffic": traffic,
           "traffic_per_particle": tpp,
           "mg_smoothing": {"nu1": tune["mg_nu1"], "nu2": tune["mg_nu2"], "autotuned": True,
                            "deposit_window": tune["dep_win"],
                            "deposit_window_ms": {str(w): round(ms, 4) for w, ms in tune["dep_tried"]}} if tune else
           {"nu1": 2, "nu2": 2, "autotuned": False}}
    if with_e2e:
        # e2e through the public API: the state (electron particles and ion
        # counts) uploaded from pinned host memory, one step, the electron
        # density read back, every step; each step starts from the same
        # state, so none drifts from the workload
        pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in st.items()}
        pin_ions = [torch.from_numpy(np.ascontiguousarray(v, dtype=np.int64)).pin_memory() for v in ions]
        ne_host = torch.empty(args.n ** 3, dtype=torch.int64).pin_memory()
        K2 = max(1, min(args.steps, 5))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done = 0
        lib = itokmc.lib()
        for _ in range(K2):
            H.itokmc_set_particles(pin["x"], pin["y"], pin["z"], pin["w"], mem=itokmc.HOST)
            H.itokmc_set_ions(*pin_ions)
            done += N0
            H.itokmc_step(1)
            itokmc._check(lib.itokmc_read_densities(H.h, 0, itokmc.NE_FIX, itokmc._ptr(ne_host),
                                                    ne_host.numel() * 8), H.h)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        out["e2e"] = {"value": done / te, "unit": "particle-steps/s",
                      "h2d_bytes_per_step": N0 * (3 * 8 + 4) + 2 * args.n ** 3 * 8,
                      "d2h_bytes_per_step": args.n ** 3 * 8, "steps": K2}
    E = None
    if rank == 0 and not args.no_cpu_baseline and form == itokmc.FP64:
        E = tuple(np.asarray(b).reshape(args.n, args.n, args.n) for b in H.itokmc_read_densities(itokmc.E))
    H.close()
    return out, E


def our_arm(args, rank, world):
    import torch
    from paper_2307_01797_gb300 import itokmc

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    ph, st, ions = workload(args)
    N0 = len(st["w"])
    forms = {"fp64": [itokmc.FP64], "mixed": [itokmc.MIXED], "both": [itokmc.FP64, itokmc.MIXED]}[args.form]
    res = {}
    E = None
    for f in forms:
        r, e = run_form(args, itokmc, f, ph, st, ions, rank, world, dist, dev, with_e2e=(f == forms[0]
                                                                                        and not args.no_e2e))
        res[f] = r
        E = E if E is not None else e
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        if E is None:
            from paper_2307_01797_gb300 import synth
            E = synth.random_field(ph, seed=3, amp=1e6, base=ph["E0"])
        import oracle
        sub = oracle_sample(ph, st, ions, args.ref_particles, seed=1)
        rates = {}
        for omp in (True, False):
            # all cores this process may use (the OpenMP build), then one thread
            oracle.use_openmp(omp)
            t_tot, n_tot, k = 0.0, 0, 0
            while t_tot < args.cpu_seconds / 2 and k < 20:
                t, n = time_oracle_step(ph, sub, E, k, 1)
                t_tot += t; n_tot += n; k += 1
            rates[omp] = (n_tot / t_tot, k)
        oracle.use_openmp(False)
        ncores = len(os.sched_getaffinity(0))
        cpu = {"value": rates[True][0], "unit": "particle-steps/s", "cores": ncores, "kind": "oracle",
               "sample": f"{len(sub['w'])} particles (a contiguous cell run of the workload) x {rates[True][1]} "
                         "steps of push+sort+deposit+KMC on the full grid, the C oracle's OpenMP build on every "
                         "core of the process's affinity",
               "single_thread": {"value": rates[False][0], "cores": 1, "steps": rates[False][1]}}
    P = res[forms[0]]
    pk, pk_kind = peaks()
    fp64_peak, _ = itokmc.itokmc_probe_fp64_peak(torch.cuda.current_stream().cuda_stream)
    line = {
        "metric": METRIC, "value": P["value"], "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": P["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if forms[0] == itokmc.FP64 else "f32",
        "data": "synthetic (seeded discharge-tree state; no dataset)",
        "config": config_of(args, N0, forms[0] == itokmc.FP64),
        "push_sort_deposit_kmc_rate": P["push_sort_deposit_kmc_rate"],
        "stage_ms_per_step": P["stage_ms_per_step"], "movers_per_step": P["movers_per_step"],
        "mg_cycles": P["mg_cycles"], "mg_smoothing": P["mg_smoothing"], "particles_per_step": P["particles_per_step"],
        "last_step_counters": P["last_step_counters"],
        "roofline_hbm": {"bound": "hbm", "kernel": "transport stage (push+sort+deposit)",
                         "achieved": P["transport_achieved_gbs"], "peak": pk, "peak_kind": pk_kind, "unit": "GB/s",
                         "frac": P["transport_achieved_gbs"] / pk, "traffic": P["traffic"],
                         "bytes_per_particle": P["bytes_per_particle"],
                         "traffic_per_particle": P["traffic_per_particle"]},
        "cpu_baseline": cpu, "e2e": P.get("e2e"), "gpu_launches": P["gpu_launches"], "clocks": P["clocks"],
    }
    if forms[0] == itokmc.FP64:
        # the FP64 transport is bound by GB300's FP64 units, not by HBM: its
        # roofline is the FP64 arithmetic rate (measured above)
        t_tr = P["stage_ms_per_step"]["transport"] / 1e3
        ach = FP64_FLOP_PER_PARTICLE * (sum(P["particles_per_step"]) / len(P["particles_per_step"])) / t_tr / 1e12
        line["roofline"] = {"bound": "alu", "kernel": "transport stage (push+sort+deposit), FP64 arithmetic",
                            "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
                            "traffic": P["traffic"], "flop_per_particle": FP64_FLOP_PER_PARTICLE,
                            "peak_kind": "measured (FP64 FMA loop, itokmc_probe_fp64_peak)"}
    else:
        line["roofline"] = line["roofline_hbm"]
    if len(forms) > 1:
        M = res[itokmc.MIXED]
        line["mixed_form"] = {
            "dtype": "f32 positions/push/leaps, int64 deposit, fixed-point potential with FP32 V-cycles",
            "value": M["value"], "ms_per_step": M["ms_per_step"],
            "push_sort_deposit_kmc_rate": M["push_sort_deposit_kmc_rate"],
            "stage_ms_per_step": M["stage_ms_per_step"], "mg_cycles": M["mg_cycles"], "mg_smoothing": M["mg_smoothing"],
            "particles_per_step": M["particles_per_step"], "gpu_launches": M["gpu_launches"],
            "clocks": M["clocks"],
            "roofline": {"bound": "hbm", "kernel": "transport stage (push+sort+deposit)",
                         "achieved": M["transport_achieved_gbs"], "peak": pk, "unit": "GB/s",
                         "frac": M["transport_achieved_gbs"] / pk, "traffic": M["traffic"],
                         "bytes_per_particle": M["bytes_per_particle"], "traffic_per_particle": M["traffic_per_particle"]},
            "speedup_vs_fp64": M["value"] / P["value"]}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------------------ precision study
def precision_study(args):
    """The FP32/fixed-point form against the FP64 plain form on the same GPU:
    the small-blob physics (1 cm, 1.5 MV/m, dt 1 ps, ppc 8, photons off) on
    an n^3 grid, both forms stepped in lockstep from one state with the same
    seeds (common random numbers), and per step the relative L2 differences
    of the electron density (ne_fix) and of E.  Variant "deterministic": D = 0
    and reactions off, which leaves only the rounding of the push and field."""
    import torch
    from paper_2307_01797_gb300 import itokmc, synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    out = {"study": "precision", "grid": args.n, "steps": args.study_steps, "variants": {}}
    for variant in ("full", "deterministic"):
        ph = synth.physics_small(args.n)
        if variant == "deterministic":
            ph.update(D=0.0, alpha_A=0.0, eta=0.0)
        st = synth.blob_state(ph, seed=1, sigma=5e-4, peak=1e18, zfrac=0.8)
        N0 = len(st["w"])
        hs = {}
        for name, form in (("fp64", itokmc.FP64), ("mixed", itokmc.MIXED)):
            H = itokmc.Handle(itokmc.make_config(ph, 8 * N0 + 1_000_000, seed0=1, precision=form))
            H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
            H.itokmc_solve_field()
            hs[name] = H
        l2_ne, l2_E, counts = [], [], []
        for k in range(args.study_steps):
            for H in hs.values():
                H.itokmc_step(1)
            a = hs["mixed"].itokmc_read_densities(itokmc.NE_FIX).astype(np.float64)
            b = hs["fp64"].itokmc_read_densities(itokmc.NE_FIX).astype(np.float64)
            l2_ne.append(float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)))
            a = hs["mixed"].itokmc_read_densities(itokmc.E).ravel()
            b = hs["fp64"].itokmc_read_densities(itokmc.E).ravel()
            l2_E.append(float(np.linalg.norm(a - b) / np.linalg.norm(b)))
            counts.append([hs["fp64"].itokmc_num_particles(), hs["mixed"].itokmc_num_particles()])
        for H in hs.values():
            H.close()
        out["variants"][variant] = {"particles0": N0, "l2_ne": l2_ne, "l2_E": l2_E, "particles": counts}
    out["variants"]["ensemble"] = precision_ensemble(itokmc, synth, args.members if args.members != 64 else 16,
                                                     args.study_steps)
    print(json.dumps(out), flush=True)


def precision_ensemble(itokmc, synth, R, K):
    """The mixed form's statistical tolerance: R realizations (keys 1..R) of
    the small-blob physics on its 64^3 grid in one handle per form, common
    random numbers, K steps; per step the relative difference of the
    ensemble-mean electron count, its standard error, and the relative L2
    differences of the ensemble-mean density and field."""
    ph = synth.physics_small(64)
    st = synth.blob_state(ph, seed=1, sigma=5e-4, peak=1e18, zfrac=0.8)
    N0 = len(st["w"])
    n3 = ph["n"] ** 3
    rep = {k: np.tile(np.asarray(st[k]), R) for k in ("x", "y", "z", "w")}
    real = np.repeat(np.arange(R, dtype=np.int32), N0)
    hs = {}
    for name, form in (("fp64", itokmc.FP64), ("mixed", itokmc.MIXED)):
        H = itokmc.Handle(itokmc.make_config(ph, 8 * R * N0 + 1_000_000, realizations=R, seed0=1, precision=form))
        H.itokmc_set_particles(rep["x"], rep["y"], rep["z"], rep["w"], real)
        H.itokmc_solve_field()
        hs[name] = H
    rel_total, sem, l2_ne, l2_E = [], [], [], []
    for k in range(K):
        for H in hs.values():
            H.itokmc_step(1)
        ne = {m: H.itokmc_read_densities(itokmc.NE_FIX, realization=-1).reshape(R, n3).astype(np.float64)
              for m, H in hs.items()}
        tot = {m: v.sum(axis=1) for m, v in ne.items()}
        rel_total.append(float(abs(tot["mixed"].mean() - tot["fp64"].mean()) / tot["fp64"].mean()))
        sem.append(float(tot["fp64"].std(ddof=1) / np.sqrt(R) / tot["fp64"].mean()))
        a, b = ne["mixed"].mean(axis=0), ne["fp64"].mean(axis=0)
        l2_ne.append(float(np.linalg.norm(a - b) / np.linalg.norm(b)))
        Ea = hs["mixed"].itokmc_read_densities(itokmc.E, realization=-1).reshape(3, R, n3).mean(axis=1)
        Eb = hs["fp64"].itokmc_read_densities(itokmc.E, realization=-1).reshape(3, R, n3).mean(axis=1)
        l2_E.append(float(np.linalg.norm(Ea - Eb) / np.linalg.norm(Eb)))
    for H in hs.values():
        H.close()
    return {"realizations": R, "grid": 64, "particles0": N0, "rel_diff_mean_electrons": rel_total,
            "rel_std_error_mean_electrons": sem, "l2_mean_ne": l2_ne, "l2_mean_E": l2_E}


# ------------------------------------------------------------------ ensemble study
def ensemble_partition(R, world, rank):
    """Members [first, first + count) of an R-member ensemble that rank
    `rank` of `world` advances: contiguous blocks, the first R mod world ranks
    one member more.  A rank's handle takes seed0 + first as its Philox base,
    so its local realization r draws with key seed0 + first + r, the global
    member's own key."""
    base, extra = divmod(int(R), int(world))
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


def ensemble_members(R, rng_seed=2024):
    """Peaks of the R seed blobs, log-uniform in [1e17, 1e19] m^-3 (member r's
    peak does not depend on how the ensemble is split)."""
    rng = np.random.default_rng(rng_seed)
    return [float(p) for p in 10.0 ** rng.uniform(17.0, 19.0, int(R))]


def ensemble_study(args):
    """Batched ensemble against sequential single runs on the same GPU: R
    independent realizations (member r: Philox key 1 + r) of the 1 cm, 128^3
    physics with photoionization, ppc 16, each seeded on the device from a
    Gaussian blob (sigma 0.5 mm at (L/2, L/2, 0.8 L)) whose peak is
    log-uniform in [1e17, 1e19] m^-3 (uneven particle counts), as
    electron-ion pairs (--electron-seeds: electrons only, whose space charge
    drives an avalanche that leaves the fixed-point range within a few
    steps).  The batched
    handle advances all of a rank's members in every launch; the sequential
    runs advance one single-realization handle per member.  Under torchrun
    the members are split R/N per rank (ensemble_partition): no collective
    on the data path, the slowest rank's time and every rank's particle-steps
    make the whole-job figures."""
    import torch
    from paper_2307_01797_gb300 import itokmc, synth
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    R, K = args.members, args.study_steps
    first, Rl = ensemble_partition(R, world, rank)
    peaks = ensemble_members(R)[first:first + Rl]
    ph = synth.physics_ensemble_member(args.n)
    L = ph["hi"][0] - ph["lo"][0]
    center = (L / 2, L / 2, 0.8 * L)

    coupling = itokmc.SEMI_IMPLICIT if args.coupling == "semi" else itokmc.EXPLICIT

    def handle(form, blobs, R_, seed0, cap):
        cfg = itokmc.make_config(ph, cap, realizations=R_, seed0=seed0, precision=form, coupling=coupling,
                                 graph_step=1 if args.graph else 0)
        arr = itokmc.blob_array(blobs)
        cfg.blobs = itokmc.ctypes.cast(arr, itokmc.ctypes.c_void_p)
        cfg.n_blobs = len(blobs)
        cfg.seed_flags = 0 if args.electron_seeds else itokmc.SEED_NEUTRAL
        return itokmc.Handle(cfg)

    def timed(H):
        for _ in range(args.warmup):
            H.itokmc_step(1)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        done = 0
        t0 = time.perf_counter()
        for _ in range(K):
            done += H.itokmc_num_particles()
            H.itokmc_step(1)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, done

    out = {"study": "ensemble", "grid": args.n, "members": R, "steps": K, "ranks": world, "coupling": args.coupling,
           "seeds": "electrons" if args.electron_seeds else "electron-ion pairs",
           "members_per_rank": [ensemble_partition(R, world, q)[1] for q in range(world)], "forms": {}}
    # the semi-implicit step exists in the FP64 form
    forms = (("fp64", itokmc.FP64),) if args.coupling == "semi" else (("fp64", itokmc.FP64), ("mixed", itokmc.MIXED))
    for name, form in forms:
        blobs = [dict(center=center, sigma=5e-4, peak=peaks[r], realization=r) for r in range(Rl)]
        H = handle(form, blobs, Rl, 1 + first, 4_000_000 * Rl + 4_000_000)
        assert H.itokmc_num_particles() > 0
        counts0 = H.itokmc_num_particles()
        tb, done = timed(H)
        counts_end = H.itokmc_num_particles()
        graph_steps = H.itokmc_get_stats()["graph_steps"]
        H.close()
        tb, done = aggregate_ranks(tb, done, dist, "cuda")
        res = {"particles0": counts0, "particles_end": counts_end, "batched_ms_per_step": 1e3 * tb / K,
               "batched_particle_steps_per_s": done / tb, "graph_steps": graph_steps}
        if name == "fp64" or not args.batched_only:
            ts, dn = 0.0, 0
            for r in range(Rl):
                H = handle(form, [dict(center=center, sigma=5e-4, peak=peaks[r], realization=0)], 1, 1 + first + r,
                           8_000_000 + 1_000_000)
                t, d = timed(H)
                ts += t
                dn += d
                H.close()
            ts, dn = aggregate_ranks(ts, dn, dist, "cuda")
            res.update({"sequential_ms_per_step": 1e3 * ts / K, "sequential_particle_steps_per_s": dn / ts,
                        "batched_speedup": ts / tb})
        out["forms"][name] = res
    fp = out["forms"]["fp64"]
    if "mixed" in out["forms"]:
        out["mixed_batched_vs_fp64_sequential"] = fp["sequential_ms_per_step"] / out["forms"]["mixed"][
            "batched_ms_per_step"]
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------------------ small config (C1)
def semi_study(args):
    """The semi-implicit transport stage (Sec. 4.3, Sec. 4.7 steps 1-5) on the
    benchmark workload, FP64 form, against the explicit transport stage plus
    the field solve it replaces: the time of each and the V-cycles of the
    variable-coefficient solve (stage calls, each ending in a host
    synchronisation)."""
    import torch
    from paper_2307_01797_gb300 import itokmc
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ph, st, ions = workload(args)
    N0 = len(st["w"])
    H = itokmc.Handle(itokmc.make_config(ph, int(N0 * args.cap_factor) + 20_000_000, seed0=1,
                                         precision=itokmc.FP64))
    H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
    H.itokmc_set_ions(*ions)
    H.itokmc_solve_field()
    K = args.study_steps
    out = {"study": "semi", "grid": args.n, "particles": N0, "steps": K}
    for mode in ("explicit", "semi"):
        for _ in range(max(1, args.warmup)):
            if mode == "semi":
                H.itokmc_transport_semi_implicit()
            else:
                H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
                H.itokmc_run_stage(itokmc.STAGE_FIELD)
            H.itokmc_advance_counter()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cyc = []
        for _ in range(K):
            if mode == "semi":
                cyc.append(H.itokmc_transport_semi_implicit()[0])
            else:
                H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
                H.itokmc_run_stage(itokmc.STAGE_FIELD)
                cyc.append(H.itokmc_get_stats()["mg_cycles"])
            H.itokmc_advance_counter()
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0) / K
        out[mode] = {"ms_per_transport_and_field": ms, "mg_cycles": cyc,
                     "particle_steps_per_s": H.itokmc_num_particles() / (ms / 1e3)}
    H.close()
    # whole steps of each coupling (the explicit step overlaps its field
    # solve with KMC and merge; the semi-implicit one solves inside its
    # transport stage), from the same state
    for mode, coupling in (("explicit", itokmc.EXPLICIT), ("semi", itokmc.SEMI_IMPLICIT)):
        H = itokmc.Handle(itokmc.make_config(ph, int(N0 * args.cap_factor) + 20_000_000, seed0=1,
                                             precision=itokmc.FP64, coupling=coupling))
        H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
        H.itokmc_set_ions(*ions)
        H.itokmc_solve_field()
        for _ in range(max(1, args.warmup)):
            H.itokmc_step(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done = 0
        for _ in range(K):
            done += H.itokmc_num_particles()
            H.itokmc_step(1)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        s_ = H.itokmc_get_stats()
        out[mode]["full_step"] = {"ms_per_step": 1e3 * t / K, "particle_steps_per_s": done / t,
                                  "ms_transport_last": s_["ms_transport"], "ms_particles_last": s_["ms_particles"]}
        H.close()
    print(json.dumps(out), flush=True)


def transport_study(args):
    """The transport stage alone (push, sort, deposit: the roofline's subject)
    on the streamer workload, or on a count-pinned uniform z-slab
    (--slab: ``--particles`` particles uniform in z in [0.4 L, 0.6 L), weight
    100, on the streamer physics of the chosen grid), each form: W untimed
    stages, then K stages timed by CUDA events on the library's stream
    (itokmc_get_stats ms_transport).  --dt-scale multiplies dt (the sort stress
    case: at x100 a particle moves about one cell per step)."""
    import torch
    from paper_2307_01797_gb300 import itokmc, synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ph = synth.physics_streamer(args.n) if args.physics == "streamer" else synth.physics_tree(args.n)
    ph["dt"] *= args.dt_scale
    if args.slab:
        st = synth.uniform_slab_state(ph, int(args.particles), seed=1)
        ions = None
    else:
        st = synth.streamer_tree_state(ph, int(args.particles), seed=7)
        ions = synth.streamer_ions(ph, st, seed=8)
    N0 = len(st["w"])
    pk, pk_kind = peaks()
    forms = {"fp64": [itokmc.FP64], "mixed": [itokmc.MIXED], "both": [itokmc.FP64, itokmc.MIXED]}[args.form]
    out = {"study": "transport", "grid": args.n, "physics": args.physics, "slab": bool(args.slab),
           "dt": ph["dt"], "particles": N0, "forms": {}}
    for form in forms:
        H = itokmc.Handle(itokmc.make_config(ph, int(1.3 * N0) + 1_000_000, seed0=1, precision=form))
        H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
        if ions is not None:
            H.itokmc_set_ions(*ions)
        H.itokmc_solve_field()
        for _ in range(args.warmup):
            H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
            H.itokmc_advance_counter()
        ms, npart, movers = [], [], []
        for _ in range(args.steps):
            npart.append(H.itokmc_num_particles())
            H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
            H.itokmc_advance_counter()
            s = H.itokmc_get_stats()
            ms.append(s["ms_transport"])
            movers.append(s["n_movers"])
        H.close()
        fp64 = form == itokmc.FP64
        bpp = 2 * (32 if fp64 else 20) + ((24 + 8 + 8) if fp64 else (12 + 8 + 8)) / ph["ppc"]
        med = statistics.median(ms)
        n_avg = sum(npart) / len(npart)
        gbs = n_avg * bpp / (med / 1e3) / 1e9
        tpp = TRANSPORT_DRAM_PER_PARTICLE[fp64]
        out["forms"]["fp64" if fp64 else "mixed"] = {
            "ms_median": med, "ms": ms, "particles": npart, "movers_per_stage": sum(movers) / len(movers),
            "bytes_per_particle": bpp, "achieved_gbs": gbs, "frac_hbm": gbs / pk, "peak_gbs": pk, "peak_kind": pk_kind,
            "particles_per_s": n_avg / (med / 1e3),
            "traffic_per_particle": tpp, "traffic": tpp * n_avg if tpp else None}
    print(json.dumps(out), flush=True)


def tree_study(args):
    """The discharge-tree configuration: 512^3 cells over a 4 cm cube, 1.8 MV/m,
    dt 5 ps, ppc 64, photoionization on; four Gaussian electron seeds (sigma
    0.3 mm, peak 5e18 m^-3) at (L/2 +- 5 mm, L/2 +- 5 mm, 0.9 L) sampled on
    the device (itokmc_init with blobs); the mixed form (FP32 particles,
    fixed-point potential with FP32 V-cycles); K full steps after W, with the
    particle count per step and the transport stage's HBM roofline."""
    import torch
    from paper_2307_01797_gb300 import itokmc, synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ph = synth.physics_tree(args.n)
    L = ph["hi"][0] - ph["lo"][0]
    blobs = [dict(center=(L / 2 + sx * 5e-3, L / 2 + sy * 5e-3, 0.9 * L), sigma=3e-4, peak=5e18)
             for sx in (-1, 1) for sy in (-1, 1)]
    form = {"fp64": itokmc.FP64, "mixed": itokmc.MIXED}[args.form if args.form != "both" else "mixed"]
    cfg = itokmc.make_config(ph, int(args.particles), seed0=1, precision=form)
    arr = itokmc.blob_array(blobs)
    cfg.blobs = itokmc.ctypes.cast(arr, itokmc.ctypes.c_void_p)
    cfg.n_blobs = len(blobs)
    t0 = time.perf_counter()
    H = itokmc.Handle(cfg)
    torch.cuda.synchronize()
    t_init = time.perf_counter() - t0
    N0 = H.itokmc_num_particles()
    tune = H.itokmc_autotune()
    for _ in range(args.warmup):
        H.itokmc_step(1)
    pk, pk_kind = peaks()
    counts, ms, tr, mg = [], [], [], []
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        counts.append(H.itokmc_num_particles())
        H.itokmc_step(1)
        s = H.itokmc_get_stats()
        tr.append(s["ms_transport"])
        mg.append(s["mg_cycles"])
    e1.record(stream)
    torch.cuda.synchronize()
    tot = e0.elapsed_time(e1)
    H.close()
    fp64 = form == itokmc.FP64
    bpp = 2 * (32 if fp64 else 20) + ((24 + 8 + 8) if fp64 else (12 + 8 + 8)) / ph["ppc"]
    n_avg = sum(counts) / len(counts)
    gbs = n_avg * bpp / (statistics.median(tr) / 1e3) / 1e9
    out = {"study": "tree", "grid": args.n, "form": "fp64" if fp64 else "mixed", "init_s": t_init,
           "particles0": N0, "particles_per_step": counts, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": tot / args.steps, "particle_steps_per_s": sum(counts) / (tot / 1e3),
           "steps_per_s": args.steps / (tot / 1e3), "transport_ms": tr, "mg_cycles": mg,
           "mg_smoothing": [tune["mg_nu1"], tune["mg_nu2"]],
           "roofline": {"bound": "hbm", "kernel": "transport stage (push+sort+deposit)", "achieved": gbs,
                        "peak": pk, "peak_kind": pk_kind, "unit": "GB/s", "frac": gbs / pk,
                        "bytes_per_particle": bpp}}
    print(json.dumps(out), flush=True)


def kmc0d_study(args):
    """0-D KMC ensembles against the reaction rate equation (Sec. 3.2.4,
    Fig. AvalancheAttachment, with the configuration's alpha(E) and eta):
    --members realizations of a single cell, X0 electrons, K steps of 1 ps at
    several field magnitudes, in both forms on the GPU (itokmc_kmc0d into
    device memory, timed with CUDA events) and a sample on the oracle (one
    host core).  Reports realization-steps/s and, per field, the ensemble
    mean and variance at the last step beside the rate equation's
    X0 exp((k_ion - k_att) t)."""
    import torch
    import oracle
    from paper_2307_01797_gb300 import itokmc, synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ph = synth.physics_small(8)
    M, K, X0 = args.members, args.study_steps, 100
    out = {"study": "kmc0d", "realizations": M, "steps": K, "X0": X0, "dt": ph["dt"], "fields": {}}
    stream = torch.cuda.current_stream()
    for E in (2.0e6, 3.54e6, 5.0e6):
        ve = ph["mu"] * E
        ka = ph["alpha_A"] * math.exp(-ph["alpha_B"] / E) * ve
        kb = ph["eta"] * ve
        rec = {"k_ion": ka, "k_att": kb, "rre_mean": X0 * math.exp((ka - kb) * K * ph["dt"])}
        for name, form in (("fp64", itokmc.FP64), ("mixed", itokmc.MIXED)):
            cfg = itokmc.make_config(ph, 1, seed0=1, precision=form, stream=stream.cuda_stream)
            X = torch.empty((M, K + 1), dtype=torch.int64, device="cuda")
            for _ in range(max(1, args.warmup)):
                itokmc._check(itokmc.lib().itokmc_kmc0d(itokmc.ctypes.byref(cfg), E, X0, M, K, X.data_ptr(),
                                                        itokmc.DEVICE))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            itokmc._check(itokmc.lib().itokmc_kmc0d(itokmc.ctypes.byref(cfg), E, X0, M, K, X.data_ptr(),
                                                    itokmc.DEVICE))
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            last = X[:, -1].double()
            rec[name] = {"ms": ms, "realization_steps_per_s": M * K / (ms / 1e3), "mean": float(last.mean()),
                         "var": float(last.var()), "extinct": float((X[:, -1] == 0).double().mean())}
        m_or = max(1, min(M, 2000))
        t0 = time.perf_counter()
        oracle.kmc0d(oracle.make_params(ph, seed=1), E, X0, m_or, K)
        t = time.perf_counter() - t0
        rec["oracle"] = {"realizations": m_or, "s": t, "realization_steps_per_s": m_or * K / t, "cores": 1}
        out["fields"][f"{E:.3g}"] = rec
    print(json.dumps(out), flush=True)


def small_study(args):
    """The plain FP64 configuration in full: 64^3 over a 1 cm cube, 1.5 MV/m,
    a Gaussian blob (sigma 0.5 mm, peak 1e18 m^-3 at 0.8 L) sampled at ppc 8
    (about 2e5 particles), photons off, dt 1 ps, Philox seed 1, 10 steps.
    The GPU steps are timed (FP64 and mixed); the oracle runs the same 10
    steps with its exact field solve (timed on one host core), and the GPU
    FP64 run, fed the oracle's field before each step, is compared with it
    particle by particle."""
    import torch
    import oracle
    from oracle import poisson
    from paper_2307_01797_gb300 import itokmc, synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ph = synth.physics_small(64)
    st = synth.blob_state(ph, seed=1, sigma=5e-4, peak=1e18, zfrac=0.8)
    N0, K = len(st["w"]), args.study_steps
    out = {"study": "small", "grid": 64, "particles0": N0, "steps": K, "forms": {}}
    for name, form in (("fp64", itokmc.FP64), ("mixed", itokmc.MIXED)):
        for graph in (0, 1):
            H = itokmc.Handle(itokmc.make_config(ph, 8 * N0 + 100000, seed0=1, precision=form, graph_step=graph))
            H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
            H.itokmc_solve_field()
            # the swapped device buffers cycle with period six: eight warm-up
            # steps capture every graph a replayed run uses (both variants
            # get the same warm-up)
            for _ in range(max(args.warmup, 8)):
                H.itokmc_step(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            done = 0
            for _ in range(K):
                done += H.itokmc_num_particles()
                H.itokmc_step(1)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            gs = H.itokmc_get_stats()["graph_steps"]
            H.close()
            out["forms"][name + ("_graph" if graph else "")] = {
                "ms_per_step": 1e3 * t / K, "particle_steps_per_s": done / t, "graph_steps": gs}
    # oracle chain and the GPU FP64 run on the oracle's fields
    p0 = oracle.make_params(ph, seed=1)
    S = oracle.canonical(p0, st)
    n3 = ph["n"] ** 3
    S["Npos"] = np.zeros(n3, np.int64)
    S["Nneg"] = np.zeros(n3, np.int64)
    ne, _ = oracle.deposit(p0, S["x"], S["y"], S["z"], S["w"], S["cell"])
    _, E = poisson.solve(oracle.rho_fixed(p0, ne, S["Npos"], S["Nneg"]), ph)
    H = itokmc.Handle(itokmc.make_config(ph, 8 * N0 + 100000, seed0=1, precision=itokmc.FP64))
    H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
    H.itokmc_set_field(*E)
    t_or, n_or, exact = 0.0, 0, 0
    for k in range(K):
        t0 = time.perf_counter()
        n_or += len(S["w"])
        S, info = oracle.step(oracle.make_params(ph, seed=1, step=k), S, E)
        _, E = poisson.solve(info["rho_fixed"], ph)
        t_or += time.perf_counter() - t0
        H.itokmc_step(1)
        G = H.itokmc_read_particles()
        same = (len(G["w"]) == len(S["w"]) and all(np.array_equal(np.asarray(G[c]).view(np.uint64),
                                                                    np.asarray(S[c]).view(np.uint64))
                                                     for c in ("x", "y", "z"))
                and np.array_equal(G["w"], S["w"]) and np.array_equal(G["cell"], S["cell"])
                and np.array_equal(H.itokmc_read_densities(itokmc.NPOS), S["Npos"]))
        exact += int(same)
        H.itokmc_set_field(*E)
    H.close()
    out["oracle"] = {"ms_per_step": 1e3 * t_or / K, "particle_steps_per_s": n_or / t_or, "cores": 1,
                     "scope": "full step (push, sort, deposit, KMC, products, merge, exact field solve)"}
    out["fp64_steps_bit_exact_with_oracle"] = f"{exact}/{K}"
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="both", choices=["fp64", "mixed", "both"],
                    help="both: the FP64 plain form gives the headline, the mixed form is reported beside it")
    ap.add_argument("--n", type=int, default=None,
                    help="cells per edge (default 256; the ensemble study defaults to 128 per member)")
    ap.add_argument("--particles", type=float, default=1e8,
                    help="target superparticle count of the synthetic discharge tree (about 7e7 are placed)")
    ap.add_argument("--ref-particles", type=int, default=2000000)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cap-factor", type=float, default=4.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default smoother counts (2, 2)")
    ap.add_argument("--recombination", action="store_true",
                    help="add the air recombination coefficients to the chemistry (five reactions)")
    ap.add_argument("--graph", action="store_true",
                    help="ensemble study: replay steps from captured CUDA graphs (graph_step = 1)")
    ap.add_argument("--mobile-ions", action="store_true",
                    help="the ions as Ito particles beside the electrons (all-particle model)")
    ap.add_argument("--study", default=None, choices=["precision", "ensemble", "small", "semi", "transport", "tree", "kmc0d"],
                    help="instead of the benchmark: one of the studies (see each function's docstring)")
    ap.add_argument("--slab", action="store_true", help="transport study: count-pinned uniform z-slab")
    ap.add_argument("--physics", default="streamer", choices=["streamer", "tree"],
                    help="transport study: streamer (2 cm, ppc 32) or discharge-tree physics (4 cm, ppc 64)")
    ap.add_argument("--dt-scale", type=float, default=1.0, help="transport study: dt multiplier (sort stress)")
    ap.add_argument("--electron-seeds", action="store_true",
                    help="ensemble study: seed electrons only (default: electron-ion pairs)")
    ap.add_argument("--coupling", default="explicit", choices=["explicit", "semi"],
                    help="ensemble study: explicit or semi-implicit field coupling (FP64 form)")
    ap.add_argument("--study-steps", type=int, default=None,
                    help="steps of a study (default: precision 20, small 10, ensemble 5)")
    ap.add_argument("--members", type=int, default=64)
    ap.add_argument("--batched-only", action="store_true")
    args = ap.parse_args()
    if args.n is None:
        args.n = {"ensemble": 128, "tree": 512}.get(args.study, 256)
    if args.study_steps is None:
        args.study_steps = {"ensemble": 5, "small": 10, "semi": 3, "kmc0d": 500}.get(args.study, 20)
    if args.study == "precision":
        precision_study(args)
        return
    if args.study == "ensemble":
        ensemble_study(args)
        return
    if args.study == "small":
        small_study(args)
        return
    if args.study == "semi":
        semi_study(args)
        return
    if args.study == "transport":
        transport_study(args)
        return
    if args.study == "tree":
        tree_study(args)
        return
    if args.study == "kmc0d":
        kmc0d_study(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.mobile_ions:
        # a study of the all-particle model, not the headline: device-timed
        # steps only (the end-to-end leg and the CPU leg use electrons only)
        args.no_e2e = True
        args.no_cpu_baseline = True
    if args.impl == "reference":
        reference_arm(args, rank, world)
    else:
        our_arm(args, rank, world)


if __name__ == "__main__":
    main()
