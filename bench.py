#!/usr/bin/env python
"""Benchmark of the clover-Wilson Dslash + SAP smoother hot path on GB300.

One step is one mixed-precision solve of D x = b to a relative residual of
1e-10 on the 32^3 x 64 workload: FP64 defect correction (the double-precision
Richardson iteration of Sec. 2, with the FP64 operator of Eq. (1) for the true
residual) around an FP32 flexible GCR inner solve preconditioned by the
multiplicative SAP smoother (Sec. 2 and 3: 4 sweeps x 4 MR steps on 4^4
domains) in FP32 arithmetic on FP16 storage with per-site scales and 12-real
links.  Beside the headline the line reports the plain FP64 GPU path, the
Dslash and smoother kernels alone, the batched workload and the link force.

`value` is the algorithmic throughput of the step in GB/s: the library counts,
for every kernel it launches, the bytes that launch must read or write (each
field once) and the timed region divides their sum by the device time.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Dslash/SAP sweep GB/s & %HBM peak; mixed vs FP64 time-to-1e-10 solve"
WORKLOAD = dict(name="32^3x64", dims=(32, 32, 32, 64), block=(4, 4, 4, 4), eps=0.5, kappa=0.1370,
                csw=1.0, config_index=2, prec=16, compress=12, n_cy=4, n_mr=4, restart=16, tol=1e-10, inner_tol=2e-6)
# bounded CPU sample of the same recipe (same eps, kappa, c_sw, solver) at 1/64 of the volume
CPU_SAMPLE_DIMS = (16, 16, 16, 8)
# derived FP32 FMA peak (SMs x FP32 lanes x 2 x max SM clock), reported beside
# the rate mgc_fma_peak measures in the run, which is the roofline's peak
FP32_FMA_PEAK_DERIVED_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# DRAM bytes (read + write) of one k_sap_m16 colour launch per lattice site,
# from an ncu capture on 24^3 x 48 (155,398,144 + 8,841,728 B over 663,552
# sites); the kernel's traffic is per domain, so it scales with the sites
SAP_DRAM_BYTES_PER_SITE = (155398144.0 + 8841728.0) / 663552
# conventional flop counts per site: hopping 1320, clover 504, kappa axpy 48
FLOP_D = 1872.0


def workload_desc(w):
    return (f"clover-Wilson {w['name']}, eps={w['eps']}, kappa={w['kappa']}, c_sw={w['csw']}, "
            f"FP16 storage + per-site FP32 scale, 12-real links, FP32 smoother arithmetic, "
            f"SAP {w['n_cy']} sweeps x {w['n_mr']} MR on 4^4 domains, FP32 FGCR({w['restart']}) inner solve "
            f"to {w['inner_tol']:g} inside FP64 defect correction, tol {w['tol']:g}")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.proc = None
        self.lines = []
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_uuid(dev):
    import torch

    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


def reduce_over_ranks(dist, t_dev, t_e2e, nbytes, nbytes_e2e, device):
    """Replicas: the job's time is the slowest rank's, its work the sum over
    ranks.  Returns (t_max, t_e2e_max, total bytes, total e2e bytes)."""
    if not dist:
        return t_dev, t_e2e, nbytes, nbytes_e2e
    import torch

    tt = torch.tensor([t_dev, t_e2e], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    bb = torch.tensor([nbytes, nbytes_e2e], dtype=torch.float64, device=device)
    dist.all_reduce(bb, op=dist.ReduceOp.SUM)
    return float(tt[0]), float(tt[1]), float(bb[0]), float(bb[1])


def counters(lib, reset=False):
    n = C.c_longlong(0)
    b = C.c_double(0)
    lib.mgc_counters(C.byref(n), C.byref(b), int(reset))
    return int(n.value), float(b.value)


# ---------------------------------------------------------------------- CPU side
def oracle_solve_sample(dims, seed_offset=0):
    """The FP64 oracle's full solve (FGCR + SAP) on a bounded lattice of the
    workload's recipe.  Returns (seconds, outer iterations, sites, threads)."""
    from oracle import oracle as O
    from paper_2112_00501_gb300 import synth

    w = WORKLOAD
    U = synth.gauge_field(dims, w["eps"], synth.gauge_seed(w["config_index"]) + 100 + seed_offset)
    b = synth.gaussian_spinor(dims, synth.source_seed(w["config_index"]) + 100 + seed_offset)
    t0 = time.perf_counter()
    Cl = O.clover(dims, w["kappa"], w["csw"], U)
    x, st, it, res = O.solve(dims, w["block"], -1, w["kappa"], U, Cl, b, method="fgcr", precond="sap",
                             ncy=w["n_cy"], nmr=w["n_mr"], m=w["restart"], tol=w["tol"])
    dt = time.perf_counter() - t0
    if st != 0:
        raise RuntimeError("oracle sample did not converge")
    return dt, it, synth.volume(dims), O.threads()


def _oracle_sample_fields(dims, seed_offset=0):
    from paper_2112_00501_gb300 import synth

    w = WORKLOAD
    U = synth.gauge_field(dims, w["eps"], synth.gauge_seed(w["config_index"]) + 100 + seed_offset)
    b = synth.gaussian_spinor(dims, synth.source_seed(w["config_index"]) + 100 + seed_offset)
    return U, b


def oracle_legs(dims, threads):
    """The oracle's D apply, one SAP sweep (4 MR steps per domain, from x = 0)
    and full solve on a bounded lattice of the workload's recipe, on `threads`
    threads.  Returns seconds per leg."""
    from oracle import oracle as O

    w = WORKLOAD
    U, b = _oracle_sample_fields(dims)
    n0 = O.threads()
    O.set_threads(threads)
    try:
        Cl = O.clover(dims, w["kappa"], w["csw"], U)
        t0 = time.perf_counter()
        O.dirac(dims, -1, w["kappa"], U, Cl, b)
        t1 = time.perf_counter()
        O.sap(dims, w["block"], -1, w["kappa"], U, Cl, b, ncy=1, nmr=w["n_mr"])
        t2 = time.perf_counter()
        x, st, it, res = O.solve(dims, w["block"], -1, w["kappa"], U, Cl, b, method="fgcr", precond="sap",
                                 ncy=w["n_cy"], nmr=w["n_mr"], m=w["restart"], tol=w["tol"])
        t3 = time.perf_counter()
    finally:
        O.set_threads(n0)
    if st != 0:
        raise RuntimeError("oracle sample did not converge")
    return {"threads": threads, "d_apply_s": t1 - t0, "sap_sweep_s": t2 - t1, "solve_s": t3 - t2,
            "solve_outer_iterations": it}


def errors_vs_oracle(dims, U, b, d_sites, d_gpu, sap_gpu):
    """Relative L2 error against the FP64 oracle on the original fields of one
    D apply (sampled sites) and of one SAP sweep from x = 0 (sampled domains of
    both colours: a red domain's result is MR_k(D_B, b_B), a black domain's
    needs its eight red neighbours first), computed site by site."""
    import numpy as np

    from oracle import oracle as O
    from paper_2112_00501_gb300 import synth

    w = WORKLOAD
    kappa, csw, block, nmr = w["kappa"], w["csw"], w["block"], w["n_mr"]
    ref = O.dirac_at(dims, -1, kappa, csw, U, b, d_sites)
    e_d = float(np.linalg.norm(d_gpu - ref) / np.linalg.norm(ref))
    nb = [d // q for d, q in zip(dims, block)]
    doms = [bc for bc in np.ndindex(*nb[::-1])]
    doms = [tuple(reversed(bc)) for bc in doms]
    red = [bc for bc in doms if sum(bc) % 2 == 0]
    black = [bc for bc in doms if sum(bc) % 2 == 1]
    g = synth.rng(199)
    got, want = [], []
    for k in g.choice(len(red), 3, replace=False):
        sites = O.block_sites(dims, block, red[k])
        got.append(sap_gpu(sites))
        want.append(O.mr_block_at(dims, block, red[k], kappa, csw, U, b[sites], nmr))
    for k in g.choice(len(black), 2, replace=False):
        bc = black[k]
        x = np.zeros_like(b)
        for mu in range(4):
            for d in (-1, 1):
                nbc = list(bc)
                nbc[mu] = (nbc[mu] + d) % nb[mu]
                s = O.block_sites(dims, block, nbc)
                x[s] = O.mr_block_at(dims, block, nbc, kappa, csw, U, b[s], nmr)
        sites = O.block_sites(dims, block, bc)
        r = b[sites] - O.dirac_at(dims, -1, kappa, csw, U, x, sites)
        got.append(sap_gpu(sites))
        want.append(O.mr_block_at(dims, block, bc, kappa, csw, U, r, nmr))
    a, c = np.concatenate(got), np.concatenate(want)
    return e_d, float(np.linalg.norm(a - c) / np.linalg.norm(c))


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from oracle import build as obuild

    obuild.build()
    # bytes per site per outer iteration of the GPU path (its byte model), from a
    # tiny GPU-free constant: measured on the GPU path and recorded here as the
    # unit conversion for the oracle's sites x iterations per second
    bpsi = float(os.environ.get("MGC_BYTES_PER_SITE_ITER", "0")) or None
    times, its = [], []
    for k in range(args.warmup + args.steps):
        dt, it, V, thr = oracle_solve_sample(CPU_SAMPLE_DIMS, seed_offset=k % 2)
        if k >= args.warmup:
            times.append(dt)
            its.append(it)
    T = sum(times)
    site_iters = sum(its) * V
    unit_conv = bpsi if bpsi else BYTES_PER_SITE_ITER_DEFAULT
    value = unit_conv * site_iters / T / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_desc(WORKLOAD), "sample": "x".join(map(str, CPU_SAMPLE_DIMS))},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": thr, "kind": "oracle",
                         "sample": f"FP64 oracle FGCR+SAP solve to 1e-10 of the same recipe on "
                                   f"{'x'.join(map(str, CPU_SAMPLE_DIMS))}; {sum(its)} outer iterations "
                                   f"in {T:.1f} s; GB/s = GPU-path algorithmic bytes per site-iteration "
                                   f"({unit_conv:.0f} B) x site-iterations/s"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# algorithmic bytes per site per inner iteration of the mixed solve (FP16
# storage, 12-real links, 4 x 4 SAP) as measured on the GPU path; converts the
# oracle's site-iterations per second into the same unit when the reference
# arm runs without a GPU measurement at hand (MGC_BYTES_PER_SITE_ITER overrides)
BYTES_PER_SITE_ITER_DEFAULT = 4258.0


# ---------------------------------------------------------------------- GPU side
# batched workload: several lattices and right-hand sides in one launch per step
BATCH_WORKLOAD = dict(lattices=[((24, 24, 24, 48), 12), ((16, 16, 16, 16), 8), ((8, 8, 8, 8), 8)],
                      block=(4, 4, 4, 4), eps=0.4, kappa=0.1355, csw=1.0, config_index=3, prec=32, compress=18,
                      n_cy=4, n_mr=4, restart=16, tol=1e-10, inner_tol=2e-6)
# two-level multigrid on the bench system: the paper's 8x4x4x4 aggregates and 16 null vectors
MG_AGG, MG_NVEC, MG_RHS = (8, 4, 4, 4), 16, 12
# the mid-size single-lattice case: FP32 fields and smoother inside FP64 FGCR
C1_WORKLOAD = dict(dims=(16, 16, 16, 32), block=(4, 4, 4, 4), eps=0.4, kappa=0.1355, csw=1.0, config_index=1,
                   prec=32, compress=18, n_cy=4, n_mr=4, restart=16, tol=1e-10, inner_tol=2e-6)
# link force workload
FORCE_WORKLOAD = dict(dims=(24, 24, 24, 48), block=(4, 4, 4, 4), eps=0.4, kappa=0.1355, csw=1.0, config_index=4,
                      prec=32, compress=18)


def bench_batch(lib, stream, prec=None, compress=None):
    """The batched workload: batched D and smoother against one launch per
    lattice, and the lock-step batched solve of all systems against solving
    them one after another; at the workload's storage unless prec/compress
    are given."""
    import torch

    from paper_2112_00501_gb300 import api, synth

    bw = dict(BATCH_WORKLOAD)
    if prec is not None:
        bw["prec"], bw["compress"] = prec, compress
    ops, bs, nrhs = [], [], []
    for dims, nr in bw["lattices"]:
        U = synth.gauge_field(dims, bw["eps"], synth.gauge_seed(bw["config_index"]))
        lat = api.Lattice(dims, bw["block"], -1)
        g = api.Gauge(lat, torch.from_numpy(U).cuda(), storage_prec=bw["prec"], compress=bw["compress"])
        ops.append(api.CloverOperator(g, bw["kappa"], bw["csw"]))
        bs.append(torch.from_numpy(synth.gaussian_spinor(dims, synth.source_seed(bw["config_index"]),
                                                         nrhs=nr)).cuda())
        nrhs.append(nr)
    B = api.Batch(ops, nrhs)
    storage = ("FP32 storage" if bw["prec"] == 32 else
               f"FP16 storage + per-site scale, {bw['compress']}-real links")
    out = {"workload": " + ".join(f"{nr} RHS on {'x'.join(map(str, d))}" for d, nr in bw["lattices"]) +
           f", eps={bw['eps']}, kappa={bw['kappa']}, c_sw={bw['csw']}, {storage}, FP32 smoother arithmetic "
           f"({bw['n_cy']} sweeps x {bw['n_mr']} MR, 4^4 domains) inside FP64 defect correction, "
           f"tol {bw['tol']:g}"}
    prec = bw["prec"]
    out["shape_d"] = B.tune(prec)
    xs = [op.lattice.pack(b, prec) for op, b in zip(ops, bs)]
    ys = B.empty_packed(prec)

    def timed(fn, n):
        fn()
        torch.cuda.synchronize()
        counters(lib, reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        e1.synchronize()
        nl, nb = counters(lib, reset=True)
        return e0.elapsed_time(e1) / 1e3 / n, nb / n, nl / n

    t, nb, nl = timed(lambda: B.apply_D(xs, prec, out=ys), 20)
    t1, nb1, nl1 = timed(lambda: [op.apply_D(x, prec, nr, y) for op, x, nr, y in zip(ops, xs, nrhs, ys)], 20)
    out["dslash_batched"] = {"us": 1e6 * t, "gbs": nb / t / 1e9, "launches": nl}
    out["dslash_per_lattice"] = {"us": 1e6 * t1, "gbs": nb1 / t1 / 1e9, "launches": nl1}
    zs = B.zeros_packed(prec)
    t, nb, nl = timed(lambda: B.sap_smooth(xs, zs, prec, bw["n_cy"], bw["n_mr"], x_is_zero=False), 5)
    t1, nb1, nl1 = timed(lambda: [op.sap_smooth(x, z, prec, nr, bw["n_cy"], bw["n_mr"])
                                  for op, x, z, nr in zip(ops, xs, zs, nrhs)], 5)
    out["sap_batched_graph"] = {"us": 1e6 * t, "gbs": nb / t / 1e9, "launches": nl}
    out["sap_per_lattice"] = {"us": 1e6 * t1, "gbs": nb1 / t1 / 1e9, "launches": nl1}
    params = api.solve_params(method=2, precond=1, smoother_prec=prec, n_cy=bw["n_cy"], n_mr=bw["n_mr"],
                              restart=bw["restart"], tol=bw["tol"], max_iter=500, inner_tol=bw["inner_tol"])
    xsol = [torch.empty_like(b) for b in bs]

    def batched_solve():
        _, infos = B.solve(bs, params, out=xsol)
        bad = [i for i in infos if i.status != 0 or i.true_res > bw["tol"]]
        if bad:
            raise RuntimeError(f"batched solve failed on {len(bad)} systems")
        return infos

    infos = batched_solve()
    torch.cuda.synchronize()
    counters(lib, reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("batch_solve")  # lets a profiler select these launches
    e0.record(stream)
    infos = batched_solve()
    e1.record(stream)
    e1.synchronize()
    torch.cuda.nvtx.range_pop()
    t_b = e0.elapsed_time(e1) / 1e3
    nl, nb = counters(lib, reset=True)

    def sequential():
        res = []
        for op, b, nr in zip(ops, bs, nrhs):
            for q in range(nr):
                _, inf = op.solve(b[q], params)
                res.append(inf)
        return res

    sequential()
    torch.cuda.synchronize()
    counters(lib, reset=True)
    e0.record(stream)
    seq = sequential()
    e1.record(stream)
    e1.synchronize()
    t_s = e0.elapsed_time(e1) / 1e3
    nl_s, nb_s = counters(lib, reset=True)
    out["solve_batched"] = {"ms": 1e3 * t_b, "systems": len(infos), "launches": nl, "gbs": nb / t_b / 1e9,
                            "max_true_res": max(i.true_res for i in infos),
                            "inner_iters_max": max(i.iters for i in infos)}
    out["solve_sequential"] = {"ms": 1e3 * t_s, "launches": nl_s, "gbs": nb_s / t_s / 1e9,
                               "max_true_res": max(i.true_res for i in seq)}
    out["batched_over_sequential_speedup"] = t_s / t_b
    del B
    return out


def bench_mg(lib, stream, op, b, params, w):
    """The two-level multigrid on the bench system: setup (M_SAP on random
    vectors, 4 adaptive passes), one solve to 1e-10, and MG_RHS solves on the
    same setup against MG_RHS solves of the bench's own method."""
    import torch

    from paper_2112_00501_gb300 import api

    V = op.lattice.volume
    gen = torch.Generator(device="cuda").manual_seed(5000)
    eta = torch.complex(torch.randn((MG_NVEC, V, 4, 3), generator=gen, device="cuda", dtype=torch.float64),
                        torch.randn((MG_NVEC, V, 4, 3), generator=gen, device="cuda", dtype=torch.float64))
    eta = eta * (0.5 ** 0.5)
    mg = api.Multigrid(op, MG_AGG, MG_NVEC)
    mp = api.mg_params(n_cy=2, n_jacobi=4, smoother_prec=w["prec"], coarse_tol=5e-2, coarse_maxit=100, n_adapt=4)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("mg_setup")  # lets a profiler select these launches
    t0 = time.perf_counter()
    mg.setup(eta, mp)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    torch.cuda.nvtx.range_pop()
    del eta
    ps = api.solve_params(tol=w["tol"], max_iter=500)
    x, info = mg.solve(b, ps, mp)
    if info.status != 0 or info.true_res > w["tol"]:
        raise RuntimeError(f"multigrid solve failed: status {info.status}, residual {info.true_res}")
    torch.cuda.synchronize()
    counters(lib, reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("mg_solve")
    e0.record(stream)
    x, info = mg.solve(b, ps, mp)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.nvtx.range_pop()
    t_solve = e0.elapsed_time(e1) / 1e3
    nl, nb = counters(lib, reset=True)
    # MG_RHS equations on one configuration (sources: the bench source rotated by a site shift)
    srcs = [torch.roll(b, shifts=k * 97, dims=0) for k in range(MG_RHS)]
    e0.record(stream)
    for q in srcs:
        _, iq = mg.solve(q, ps, mp)
        if iq.status != 0:
            raise RuntimeError("multigrid solve failed")
    e1.record(stream)
    e1.synchronize()
    t_mg12 = e0.elapsed_time(e1) / 1e3
    e0.record(stream)
    for q in srcs:
        _, iq = op.solve(q, params)
        if iq.status != 0:
            raise RuntimeError("two-level solve failed")
    e1.record(stream)
    e1.synchronize()
    t_tl12 = e0.elapsed_time(e1) / 1e3
    counters(lib, reset=True)
    del mg
    return {"method": f"flexible BiCGStab (FP64) with the two-level preconditioner: {MG_NVEC} null vectors, "
                      f"{'x'.join(map(str, MG_AGG))} aggregates split by chirality, coarse BiCGStab to "
                      f"{mp.coarse_tol:g}, post-smoother {mp.n_cy} SAP-for-A sweeps x {mp.n_jacobi} Jacobi, "
                      f"setup with {mp.n_adapt} adaptive passes",
            "setup_s": t_setup, "solve_ms": 1e3 * t_solve, "outer_iters": info.iters, "true_residual": info.true_res,
            "solve_launches": nl, "solve_gbs": nb / t_solve / 1e9,
            f"{MG_RHS}_equations": {"mg_setup_plus_solves_s": t_setup + t_mg12, "mg_solves_s": t_mg12,
                                   "two_level_solves_s": t_tl12}}


def bench_c1(lib, stream):
    """16^3 x 32 with FP32 fields: D (FP32, FP64), one smoother sweep (FP32,
    4 MR steps per domain, both colours) and the solve to 1e-10 with FP64
    FGCR around the FP32 smoother, beside the default two-level solve.  The
    fields (about 110 MB at FP32) fit in the 129 MB L2, so its GB/s figures
    are L2-assisted, not HBM figures."""
    import torch

    from paper_2112_00501_gb300 import api, synth

    cw = C1_WORKLOAD
    dims = cw["dims"]
    U = synth.gauge_field(dims, cw["eps"], synth.gauge_seed(cw["config_index"]))
    b = torch.from_numpy(synth.gaussian_spinor(dims, synth.source_seed(cw["config_index"]))).cuda()
    lat = api.Lattice(dims, cw["block"], -1)
    op = api.CloverOperator(api.Gauge(lat, torch.from_numpy(U).cuda(), storage_prec=cw["prec"],
                                      compress=cw["compress"]), cw["kappa"], cw["csw"])

    def timed(fn, n):
        fn()
        torch.cuda.synchronize()
        counters(lib, reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            out = fn()
        e1.record(stream)
        e1.synchronize()
        _, nb = counters(lib, reset=True)
        t = e0.elapsed_time(e1) / 1e3 / n
        return t, nb / n, out

    res = {"workload": f"{'x'.join(map(str, dims))}, eps={cw['eps']}, kappa={cw['kappa']}, c_sw={cw['csw']}, "
                       f"FP32 storage (18-real links), SAP {cw['n_cy']} sweeps x {cw['n_mr']} MR on 4^4 domains",
           "note": "fields fit in L2: GB/s are L2-assisted"}
    for prec in (32, 64):
        xin, out = lat.pack(b, prec), lat.empty_packed(prec)
        t, nb, _ = timed(lambda: op.apply_D(xin, prec, 1, out), 20)
        res[f"dslash_fp{prec}"] = {"us": 1e6 * t, "gbs": nb / t / 1e9}
    rl, zl = lat.pack(b, 32), lat.zeros_packed(32)
    t, nb, _ = timed(lambda: op.sap_smooth(rl, zl, 32, 1, 1, cw["n_mr"], x_is_zero=False), 10)
    res["sap_sweep_fp32"] = {"us": 1e6 * t, "gbs": nb / t / 1e9}
    for name, method in (("fgcr_fp64_outer", 0), ("two_level", 2)):
        params = api.solve_params(method=method, precond=1, smoother_prec=32, n_cy=cw["n_cy"], n_mr=cw["n_mr"],
                                  restart=cw["restart"], tol=cw["tol"], max_iter=500, inner_tol=cw["inner_tol"])
        t, nb, (x, info) = timed(lambda: op.solve(b, params), 3)
        if info.status != 0 or not info.true_res <= cw["tol"]:
            raise RuntimeError(f"c1 {name} solve failed: status {info.status}, residual {info.true_res}")
        res[name] = {"ms": 1e3 * t, "iters": info.iters, "true_res": info.true_res, "gbs": nb / t / 1e9}
    return res


def bench_force(lib, stream, prec=None, compress=None):
    """dS/dU for S = phi^+ (D^+ D)^-1 phi on 24^3 x 48 (two solves and the
    force kernels); the solves' smoother at the workload's storage unless
    prec/compress are given."""
    import torch

    from paper_2112_00501_gb300 import api, synth

    fw = dict(FORCE_WORKLOAD)
    if prec is not None:
        fw["prec"], fw["compress"] = prec, compress
    dims = fw["dims"]
    U = synth.gauge_field(dims, fw["eps"], synth.gauge_seed(fw["config_index"]))
    phi = torch.from_numpy(synth.gaussian_spinor(dims, synth.source_seed(fw["config_index"]))).cuda()
    lat = api.Lattice(dims, fw["block"], -1)
    op = api.CloverOperator(api.Gauge(lat, torch.from_numpy(U).cuda(), storage_prec=fw["prec"],
                                      compress=fw["compress"]), fw["kappa"], fw["csw"])
    params = api.solve_params(method=2, precond=1, smoother_prec=fw["prec"], tol=1e-10, max_iter=500)
    op.force(phi, params)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 3
    torch.cuda.nvtx.range_push("force")  # lets a profiler select these launches
    e0.record(stream)
    for _ in range(n):
        g, S, info = op.force(phi, params)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.nvtx.range_pop()
    t = e0.elapsed_time(e1) / 1e3 / n
    V = synth.volume(dims)
    storage = "FP32 storage" if fw["prec"] == 32 else f"FP16 storage, {fw['compress']}-real links"
    return {"workload": f"{'x'.join(map(str, dims))}, eps={fw['eps']}, kappa={fw['kappa']}, c_sw={fw['csw']}, "
                        f"two-level solves (smoother: {storage}, FP32 arithmetic) to 1e-10, FP64 force kernels",
            "ms": 1e3 * t, "links_per_s": 4 * V / t, "solve_iters": info.iters}


def profile_kernel(which):
    """A few launches of one kernel on 24^3 x 48 at the workload's storage format
    (working set above the L2 size, about 2 GB on the device), for ncu; `force`:
    one link-force evaluation on 16^4 (its FP64 fields about 0.5 GB)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2112_00501_gb300 import api, synth

    if which == "force":
        fw = FORCE_WORKLOAD
        fdims = (16, 16, 16, 16)
        Uf = synth.gauge_field(fdims, fw["eps"], synth.gauge_seed(fw["config_index"]))
        phi = torch.from_numpy(synth.gaussian_spinor(fdims, synth.source_seed(fw["config_index"]))).cuda()
        lat = api.Lattice(fdims, fw["block"], -1)
        op = api.CloverOperator(api.Gauge(lat, torch.from_numpy(Uf).cuda(), storage_prec=fw["prec"],
                                          compress=fw["compress"]), fw["kappa"], fw["csw"])
        params = api.solve_params(method=2, precond=1, smoother_prec=fw["prec"], tol=1e-10, max_iter=500)
        op.force(phi, params)
        torch.cuda.synchronize()
        print("profile run done")
        return 0
    if which in ("dslash_batch", "sap_batch"):
        # the batched workload (12 + 8 + 8 right-hand sides on three lattices), its
        # autotuned operator launch or one smoother sweep over the batch
        bw = BATCH_WORKLOAD
        ops, xs, nrhs = [], [], []
        for bdims, nr in bw["lattices"]:
            Ub = synth.gauge_field(bdims, bw["eps"], synth.gauge_seed(bw["config_index"]))
            lat = api.Lattice(bdims, bw["block"], -1)
            g = api.Gauge(lat, torch.from_numpy(Ub).cuda(), storage_prec=bw["prec"], compress=bw["compress"])
            op = api.CloverOperator(g, bw["kappa"], bw["csw"])
            bb = torch.from_numpy(synth.gaussian_spinor(bdims, synth.source_seed(bw["config_index"]), nrhs=nr)).cuda()
            ops.append(op)
            xs.append(lat.pack(bb, bw["prec"]))
            nrhs.append(nr)
        B = api.Batch(ops, nrhs)
        # the shape the autotuner picks for this batch on the GB300 (two RHS per
        # thread, 128 threads, right-hand-side groups of a site block adjacent)
        B.set_shape(bw["prec"], 2, 128, 1, 1)
        ys = B.empty_packed(bw["prec"])
        zs = B.zeros_packed(bw["prec"])
        for _ in range(2):
            if which == "dslash_batch":
                B.apply_D(xs, bw["prec"], out=ys)
            else:
                B.sap_smooth(xs, zs, bw["prec"], 1, bw["n_mr"], x_is_zero=False)
        torch.cuda.synchronize()
        print("profile run done")
        return 0
    w = WORKLOAD
    dims = (24, 24, 24, 48)
    U = synth.gauge_field(dims, w["eps"], synth.gauge_seed(3))
    b = torch.from_numpy(synth.gaussian_spinor(dims, synth.source_seed(3))).cuda()
    lat = api.Lattice(dims, w["block"], -1)
    op = api.CloverOperator(api.Gauge(lat, torch.from_numpy(U).cuda(), storage_prec=w["prec"],
                                      compress=w["compress"]), w["kappa"], w["csw"])
    bp = lat.pack(b, w["prec"])
    xp = lat.zeros_packed(w["prec"])
    prec = {"dslash64": 64, "dslash32": 32, "sap32": 32}.get(which, w["prec"])
    if prec != w["prec"]:
        bp, xp = lat.pack(b, prec), lat.empty_packed(prec)
    if which == "dslash16x18":
        op = api.CloverOperator(api.Gauge(lat, torch.from_numpy(U).cuda(), storage_prec=w["prec"], compress=18),
                                w["kappa"], w["csw"])
    for _ in range(2):
        if which in ("sap", "sap32"):
            op.sap_smooth(bp, xp, prec, 1, 1, w["n_mr"], x_is_zero=False)
        else:
            op.apply_D(bp, prec, 1, xp)
    torch.cuda.synchronize()
    print("profile run done")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-path", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-force", action="store_true")
    ap.add_argument("--no-qws", action="store_true")
    ap.add_argument("--no-mg", action="store_true")
    ap.add_argument("--no-c1", action="store_true")
    ap.add_argument("--profile-kernel", choices=["sap", "sap32", "dslash", "dslash32", "dslash16x18", "dslash64",
                                                 "dslash_batch", "sap_batch", "force"],
                    default=None,
                    help="run only a few launches of one kernel (for ncu captures)")
    args = ap.parse_args()
    if args.profile_kernel:
        return profile_kernel(args.profile_kernel)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    import __graft_entry__

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    from paper_2112_00501_gb300 import _lib, api, synth

    lib = _lib.load()
    w = WORKLOAD
    dims = w["dims"]
    V = synth.volume(dims)
    U = synth.gauge_field(dims, w["eps"], synth.gauge_seed(w["config_index"]))
    b_host = synth.gaussian_spinor(dims, synth.source_seed(w["config_index"]))
    lat = api.Lattice(dims, w["block"], -1)
    Ud = torch.from_numpy(U).cuda()
    gauge = api.Gauge(lat, Ud, storage_prec=w["prec"], compress=w["compress"])
    op = api.CloverOperator(gauge, w["kappa"], w["csw"])
    b = torch.from_numpy(b_host).cuda()
    params = api.solve_params(method=2, precond=1, smoother_prec=w["prec"], n_cy=w["n_cy"], n_mr=w["n_mr"],
                              restart=w["restart"], tol=w["tol"], max_iter=500, inner_tol=w["inner_tol"])
    stream = torch.cuda.current_stream()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------- device-resident timed region
    for _ in range(args.warmup):
        x, info = op.solve(b, params)
        assert info.status == 0, info.status
    barrier()
    counters(lib, reset=True)
    sampler = ClockSampler(gpu_uuid(local))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select exactly these launches
    ev0.record(stream)
    iters = []
    for _ in range(args.steps):
        x, info = op.solve(b, params)
        iters.append(info.iters)
        if info.status != 0 or info.true_res > w["tol"]:
            raise RuntimeError(f"solve failed: status {info.status}, residual {info.true_res}")
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    barrier()
    clocks = sampler.stop()
    t_dev = ev0.elapsed_time(ev1) / 1e3
    launches, nbytes = counters(lib, reset=True)
    true_res = info.true_res

    # ---------------- end to end through the C ABI with host buffers
    t_e2e, nbytes_e2e = float("nan"), 0.0
    if not args.no_e2e:
        b_pin = torch.from_numpy(b_host).pin_memory()
        x_pin = torch.empty_like(b_pin).pin_memory()
        op.solve(b_pin, params, out=x_pin)
        barrier()
        counters(lib, reset=True)
        e_ms = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            xh, info_e = op.solve(b_pin, params, out=x_pin)
            e1.record(stream)
            e1.synchronize()
            e_ms.append(e0.elapsed_time(e1))
        barrier()
        # the median step: host transfers vary from process to process
        t_e2e = statistics.median(e_ms) * args.steps / 1e3
        _, nbytes_e2e = counters(lib, reset=True)

    # ---------------- the dominant kernel: SAP colour launches, timed alone
    rl = lat.pack(b, w["prec"])
    zl = lat.zeros_packed(w["prec"])
    reps = 10
    for _ in range(2):
        zl.zero_()
        op.sap_smooth(rl, zl, w["prec"], 1, w["n_cy"], w["n_mr"], x_is_zero=True)
    torch.cuda.synchronize()
    sap_ms = []
    counters(lib, reset=True)
    for _ in range(reps):
        zl.zero_()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        op.sap_smooth(rl, zl, w["prec"], 1, w["n_cy"], w["n_mr"], x_is_zero=True)
        s1.record(stream)
        s1.synchronize()
        sap_ms.append(s0.elapsed_time(s1))
    sap_launches, sap_bytes = counters(lib, reset=True)
    launches_per_call = sap_launches // reps
    t_launch = statistics.median(sap_ms) / 1e3 / launches_per_call
    bytes_launch = sap_bytes / sap_launches
    # flops of one colour launch: residual (skipped when x = 0) + n_mr MR steps
    # (Dirichlet D_B: 6 of 8 hops stay inside a 4^4 domain; dots 144; two caxpys 192)
    flop_mr = (1320.0 * 6 / 8 + 504 + 48) + 144 + 192
    flop_res = FLOP_D + 24 + 24
    n_x0 = 1  # launches per call with x == 0
    flops_call = 0.5 * V * (launches_per_call * w["n_mr"] * flop_mr + (launches_per_call - n_x0) * flop_res)
    sap_tflops = flops_call / (statistics.median(sap_ms) / 1e3) / 1e12

    # ---------------- measured FMA rates (the roofline's peak for the arithmetic-bound kernels)
    f32_peak, f64_peak = C.c_double(0), C.c_double(0)
    if lib.mgc_fma_peak(32, C.byref(f32_peak), C.c_void_p(stream.cuda_stream)) != 0 or \
            lib.mgc_fma_peak(64, C.byref(f64_peak), C.c_void_p(stream.cuda_stream)) != 0:
        raise RuntimeError("mgc_fma_peak failed: " + lib.mgc_last_error().decode())
    fp32_peak_tflops, fp64_peak_tflops = f32_peak.value / 1e12, f64_peak.value / 1e12
    counters(lib, reset=True)

    # ---------------- results for the error against the FP64 oracle (CPU leg)
    d_sites = synth.rng(77).choice(V, 2048, replace=False)
    d_sites = np.concatenate([d_sites, [0, V - 1]])
    d_gpu = op.D(b, prec=w["prec"]).cpu().numpy()[d_sites]
    sap_full = op.sap(b, prec=w["prec"], n_cy=1, n_mr=w["n_mr"]).cpu().numpy()
    counters(lib, reset=True)

    # ---------------- Dslash alone (workload storage and FP64)
    def time_dslash(prec, dop=op):
        xin = lat.pack(b, prec)
        out = lat.empty_packed(prec)
        for _ in range(3):
            dop.apply_D(xin, prec, 1, out)
        torch.cuda.synchronize()
        counters(lib, reset=True)
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = 20
        d0.record(stream)
        for _ in range(n):
            dop.apply_D(xin, prec, 1, out)
        d1.record(stream)
        d1.synchronize()
        _, by = counters(lib, reset=True)
        t = d0.elapsed_time(d1) / 1e3 / n
        return t, by / n

    t_d16, by_d16 = time_dslash(w["prec"])
    t_d32, by_d32 = time_dslash(32)
    t_d64, by_d64 = time_dslash(64)
    # the FP16 operator with 18-real links: 48 B more per site, no row-2 rebuild
    g18 = api.Gauge(lat, Ud, storage_prec=w["prec"], compress=18)
    op18 = api.CloverOperator(g18, w["kappa"], w["csw"])
    t_d16_18, by_d16_18 = time_dslash(w["prec"], op18)
    del op18, g18

    # ---------------- plain FP64 GPU path for the time-to-solution comparison
    fp64 = None
    if not args.no_fp64_path:
        g64 = api.Gauge(lat, Ud, storage_prec=64)
        op64 = api.CloverOperator(g64, w["kappa"], w["csw"])
        p64 = api.solve_params(method=0, precond=1, smoother_prec=64, n_cy=w["n_cy"], n_mr=w["n_mr"],
                               restart=w["restart"], tol=w["tol"], max_iter=500)
        x64, i64 = op64.solve(b, p64)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        x64, i64 = op64.solve(b, p64)
        f1.record(stream)
        f1.synchronize()
        fp64 = {"ms": f0.elapsed_time(f1), "iters": i64.iters, "true_res": i64.true_res}
        del op64, g64
    counters(lib, reset=True)

    # ---------------- FP64 FGCR (FP64 vectors, inner products and orthogonalisation
    # in every iteration) around the FP16 smoother, beside the default two-level
    # solve whose inner solve works in FP32
    fgcr16 = None
    if not args.no_fp64_path:
        pf = api.solve_params(method=0, precond=1, smoother_prec=w["prec"], n_cy=w["n_cy"], n_mr=w["n_mr"],
                              restart=w["restart"], tol=w["tol"], max_iter=500)
        xf, inf = op.solve(b, pf)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        nf = 3
        for _ in range(nf):
            xf, inf = op.solve(b, pf)
            if inf.status != 0 or inf.true_res > w["tol"]:
                raise RuntimeError(f"FGCR solve failed: status {inf.status}, residual {inf.true_res}")
        g1.record(stream)
        g1.synchronize()
        fgcr16 = {"method": "FGCR(16) with FP64 vectors, inner products and orthogonalisation, FP64 operator, "
                            "preconditioned by the FP16-storage smoother",
                  "ms": g0.elapsed_time(g1) / nf, "iters": inf.iters, "true_res": inf.true_res}
    counters(lib, reset=True)

    # ---------------- the paper's own QWS solve (method 3) on the same system
    qws = None
    if not args.no_qws:
        pq = api.solve_params(method=3, precond=1, smoother_prec=w["prec"], n_cy=w["n_cy"], n_mr=w["n_mr"],
                              tol=w["tol"], max_iter=500, inner_tol=w["inner_tol"])
        xq, iq = op.solve(b, pq)
        torch.cuda.synchronize()
        counters(lib, reset=True)
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        nq = 3
        for _ in range(nq):
            xq, iq = op.solve(b, pq)
            if iq.status != 0 or iq.true_res > w["tol"]:
                raise RuntimeError(f"QWS solve failed: status {iq.status}, residual {iq.true_res}")
        q1.record(stream)
        q1.synchronize()
        nlq, nbq = counters(lib, reset=True)
        t_q = q0.elapsed_time(q1) / 1e3 / nq
        # one colour launch of the smoother for A (Jacobi, same storage)
        zl.zero_()
        op.sap_smooth_A(rl, zl, w["prec"], 1, 1, w["n_mr"], x_is_zero=True)
        torch.cuda.synchronize()
        sa = []
        for _ in range(reps):
            zl.zero_()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            op.sap_smooth_A(rl, zl, w["prec"], 1, w["n_cy"], w["n_mr"], x_is_zero=True)
            a1.record(stream)
            a1.synchronize()
            sa.append(a0.elapsed_time(a1))
        # the default method with even-odd preconditioned MR domain solves in the smoother
        peo = api.solve_params(method=2, precond=1, smoother_prec=w["prec"], n_cy=w["n_cy"], n_mr=w["n_mr"],
                               restart=w["restart"], tol=w["tol"], max_iter=500, inner_tol=w["inner_tol"],
                               sap_solver=2)
        xe, ie = op.solve(b, peo)
        torch.cuda.synchronize()
        q0.record(stream)
        for _ in range(nq):
            xe, ie = op.solve(b, peo)
            if ie.status != 0 or ie.true_res > w["tol"]:
                raise RuntimeError(f"even-odd smoother solve failed: status {ie.status}")
        q1.record(stream)
        q1.synchronize()
        t_eo = q0.elapsed_time(q1) / 1e3 / nq
        se = []
        for _ in range(reps):
            zl.zero_()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            op.sap_smooth_eo(rl, zl, w["prec"], 1, w["n_cy"], w["n_mr"], x_is_zero=True)
            a1.record(stream)
            a1.synchronize()
            se.append(a0.elapsed_time(a1))
        counters(lib, reset=True)
        eo = {"method": "the default two-level solve with even-odd preconditioned MR domain solves",
              "ms": 1e3 * t_eo, "inner_iters": ie.iters, "true_residual": ie.true_res,
              "sap_eo_launch_us": 1e3 * statistics.median(se) / launches_per_call}
        qws = {"method": "QWS (Sec. 2): FP64 Richardson around FP32 BiCGStab on A M_SAP, A = C^-1 D, "
                         f"SAP for A with {w['n_mr']} Jacobi iterations per domain",
               "ms": 1e3 * t_q, "bicgstab_iters": iq.iters, "true_residual": iq.true_res,
               "gbs": nbq / nq / t_q / 1e9, "launches": nlq // nq,
               "sap_A_launch_us": 1e3 * statistics.median(sa) / launches_per_call, "even_odd_smoother": eo}
        counters(lib, reset=True)

    # ---------------- batched workload and link force (reported beside the headline)
    mgres = None if args.no_mg else bench_mg(lib, stream, op, b, params, w)
    batch = None if args.no_batch else bench_batch(lib, stream)
    if batch is not None:
        # the same batch at the benchmark's FP16 storage (FP32 arithmetic)
        batch["fp16_storage"] = bench_batch(lib, stream, prec=16, compress=12)
    force = None if args.no_force else bench_force(lib, stream)
    if force is not None:
        force["fp16_storage"] = bench_force(lib, stream, prec=16, compress=12)
    c1 = None if args.no_c1 else bench_c1(lib, stream)
    counters(lib, reset=True)

    # ---------------- reduce over ranks
    t_max, t_e2e, tot_bytes, nbytes_e2e = reduce_over_ranks(dist, t_dev, t_e2e, nbytes, nbytes_e2e, "cuda")
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    value = tot_bytes / t_max / 1e9
    bytes_per_site_iter = nbytes / (V * sum(iters))
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": workload_desc(w), "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (FP64 links alone 1.2 GB)"},
        "gpu_launches": launches,
        "clocks": clocks,
        "time_to_solution_ms": 1e3 * t_max / args.steps,
        "outer_iterations": iters[-1],
        "true_residual": true_res,
        "fp64_path": fp64,
        "mixed_over_fp64_speedup": (fp64["ms"] / (1e3 * t_max / args.steps)) if fp64 else None,
        "fgcr_fp64_fp16_smoother": fgcr16,
        "dslash": {"fp16_12real_gbs": by_d16 / t_d16 / 1e9, "fp16_us": 1e6 * t_d16,
                   "fp64_tflops": FLOP_D * V / t_d64 / 1e12,
                   "fp64_frac_fp64_peak": FLOP_D * V / t_d64 / 1e12 / fp64_peak_tflops,
                   "fp32_12real_gbs": by_d32 / t_d32 / 1e9, "fp32_us": 1e6 * t_d32,
                   "fp32_frac_hbm": (by_d32 / t_d32 / 1e9 / hbm) if hbm else None,
                   "fp64_gbs": by_d64 / t_d64 / 1e9, "fp64_us": 1e6 * t_d64,
                   "fp16_frac_hbm": (by_d16 / t_d16 / 1e9 / hbm) if hbm else None,
                   "fp16_18real_gbs": by_d16_18 / t_d16_18 / 1e9, "fp16_18real_us": 1e6 * t_d16_18,
                   "fp16_18real_frac_hbm": (by_d16_18 / t_d16_18 / 1e9 / hbm) if hbm else None},
        "sap_sweep": {"launch_us": 1e6 * t_launch, "algorithmic_gbs": bytes_launch / t_launch / 1e9,
                      "frac_hbm": (bytes_launch / t_launch / 1e9 / hbm) if hbm else None,
                      "tflops_fp32": sap_tflops, "frac_fp32_peak": sap_tflops / fp32_peak_tflops,
                      "frac_fp32_peak_derived": sap_tflops / FP32_FMA_PEAK_DERIVED_TFLOPS},
        "fma_peaks": {"fp32_tflops": fp32_peak_tflops, "fp64_tflops": fp64_peak_tflops,
                      "fp32_derived_tflops": FP32_FMA_PEAK_DERIVED_TFLOPS,
                      "source": "mgc_fma_peak in this run: 8 independent FMA chains per thread, "
                                "eight 256-thread blocks per SM, fastest of five launches"},
        "roofline": {
            "kernel": "k_sap_m16 (SAP colour launch, FP16 storage, 12-real links, 4^4 domains, 4 MR steps)",
            "bound": "alu",
            "achieved": sap_tflops,
            "peak": fp32_peak_tflops,
            "unit": "TFLOP/s",
            "frac": sap_tflops / fp32_peak_tflops,
            "traffic": SAP_DRAM_BYTES_PER_SITE * V if SAP_DRAM_BYTES_PER_SITE else None,
            "algorithmic_bytes": bytes_launch,
            "algorithmic_gbs": bytes_launch / t_launch / 1e9,
            "frac_hbm": (bytes_launch / t_launch / 1e9 / hbm) if hbm else None,
            "peak_source": "FP32 FMA rate measured in this run (mgc_fma_peak, of measured); HBM fraction "
                           "against MEASURED_PEAKS.json hbm_gbs (of measured)",
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch on 24^3x48, "
                              "scaled by sites",
        },
        "e2e": {"value": nbytes_e2e / t_e2e / 1e9, "unit": "GB/s", "h2d_bytes_per_step": V * 192,
                "d2h_bytes_per_step": V * 192, "ms_per_step": 1e3 * t_e2e / args.steps,
                "ms_steps": e_ms if not args.no_e2e else None,
                "timing": "median of the per-step times (each step bracketed by its own events) x steps"},
        "bytes_per_site_iteration": bytes_per_site_iter,
        "qws_solve": qws,
        "multigrid": mgres,
        "batched": batch,
        "force": force,
        "c1": c1,
    }
    if not args.no_cpu_baseline:
        # the CPU leg: the FP64 oracle timed on the host cores (one thread and
        # all cores of this process's affinity), and the error of the timed
        # storage format's results against it
        ncores = len(os.sched_getaffinity(0))
        legs = [oracle_legs(CPU_SAMPLE_DIMS, 1), oracle_legs(CPU_SAMPLE_DIMS, ncores)]
        Vs = 1
        for d in CPU_SAMPLE_DIMS:
            Vs *= d
        it = legs[1]["solve_outer_iterations"]
        cpu_val = bytes_per_site_iter * it * Vs / legs[1]["solve_s"] / 1e9
        line["cpu_baseline"] = {
            "value": cpu_val, "unit": "GB/s", "cores": ncores, "kind": "oracle",
            "sample": f"FP64 oracle on {'x'.join(map(str, CPU_SAMPLE_DIMS))} ({Vs} sites) of the same recipe: "
                      f"D apply, one SAP sweep (4 MR steps per domain) and the FGCR+SAP solve to 1e-10 "
                      f"({it} outer iterations), on 1 thread and on {ncores}; value = the {ncores}-thread "
                      f"solve as this run's algorithmic bytes per site-iteration ({bytes_per_site_iter:.0f} B) x "
                      f"site-iterations/s",
            "legs": legs}
        e_d, e_s = errors_vs_oracle(dims, U, b_host, d_sites, d_gpu, lambda sites: sap_full[sites])
        line["error_vs_oracle"] = {
            "dslash": e_d, "sap_sweep": e_s, "tolerance": 2e-3,
            "what": "relative L2 error against the FP64 oracle on the original fields, at the timed storage "
                    "(FP16 + per-site scale, 12-real links): D on 2050 sampled sites of 32^3x64; one SAP sweep "
                    "from x = 0 (4 MR steps) on 3 red and 2 black sampled domains"}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
