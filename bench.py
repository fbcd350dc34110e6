"""Throughput of the fTWA hot path on one or more GB300s.

Workload (one "step" = one pass of the whole path over one batch): the
198-site open honeycomb flake (11 x 18 brick wall, 277 bonds), U/t = 1.6,
half filling with the charge-imbalanced Fock start (doubly occupied central
hexagon, six emptied edge sites), M = 16384 samples, FP32 state, RK4 with
dt = 0.01 to T = 10 (1000 steps), snapshots every 10 steps (101 rows), FP64
moments (occupations, connected Gram, g2).  Per step: ftwa_sample ->
ftwa_evolve -> ftwa_moments.

metric: sample-RK4-steps/s = M * 1000 / (seconds per step), whole job.

Multi-GPU: samples are independent, so ranks take disjoint sample ranges
(Philox counters are keyed by the global sample index) with no collective
on the data path (weak scaling).

--impl reference: the CPU oracle (plain FP64 C, OpenMP) on the host cores,
timed on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fTWA sample-RK4-steps/s at 198 sites, FP32 vs FP64 GPU at stated error; adjoint time"
UNIT = "sample-RK4-steps/s"
FLOP_PER_ELEMENT_STEP = 152          # 4 stages x (2x(3+3) hopping FMAs + U term + i) + RK4 combine
SMEM_BYTES_PER_ELEMENT_STEP = 256    # 4 stages x (7 complex FP32 reads + 1 write) of the stage state


def workload(M=16384, steps=1000, every=10, U=1.6):
    import workloads as W
    lat = W.brick_wall_flake(11, 18)
    nu, nd = W.charge_imbalanced_state(lat)
    return dict(lat=lat, n_up=nu, n_dn=nd, U=U, M=M, steps=steps, every=every)


def config_dict(wl, extra=None):
    c = {"workload": "fTWA 198-site honeycomb flake (brick wall 11x18), charge-imbalanced Fock start",
         "n_sites": 198, "U_over_t": wl["U"], "samples_per_gpu": wl["M"], "rk4_steps": wl["steps"],
         "dt": 0.01, "T": 10.0, "out_every": wl["every"], "state": "fp32 complex",
         "moments": "FP64 sample means, BF16x3 tcgen05 connected Gram (FP32 accumulate), FP64 estimators",
         "l2": "inputs larger than L2 (state 10.3 GB per GPU)"}
    if extra:
        c.update(extra)
    return c


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    import torch
    import torch.distributed as dist
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return rank, local, ws


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    from paper_2212_04352_gb300 import shard
    return shard.max_over_ranks(x, ws)


def traffic_record(kernel_src, record="tile_stepper_fp32_198_traffic.txt"):
    """ncu DRAM bytes per launch recorded for this kernel source (or None)."""
    path = os.path.join(ROOT, "profiles", record)
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    if kv.get("source_sha256_16") != sha:
        return None
    try:
        return float(kv["dram_bytes_per_launch_full_workload"])
    except (KeyError, ValueError):
        return None


def count_kernels(fn, sessions=2):
    """Kernels (not copies or memsets) that fn() launches, counted from the
    CUPTI activity records that torch.profiler collects (the raw records:
    kernels launched outside torch have no CPU-side op) in the last of
    `sessions` profiled calls (the first session of a process may miss device
    records); NCCL's kernels are left out.  None if the profiler is
    unavailable or saw no kernel."""
    import torch
    try:
        from torch.profiler import ProfilerActivity, profile
        for _ in range(sessions):
            with profile(activities=[ProfilerActivity.CUDA]) as prof:
                fn()
                torch.cuda.synchronize()
        n = 0
        for e in prof.profiler.kineto_results.events():
            if not str(e.device_type()).endswith("CUDA"):
                continue
            name = e.name()
            if name.startswith(("Memcpy", "Memset", "memcpy", "memset")) or "nccl" in name.lower():
                continue
            n += 1
        return n if n > 0 else None
    except Exception as exc:   # profiler missing on this build: no count
        print(f"note: kernel count unavailable ({exc})", file=sys.stderr)
        return None


def cpu_baseline(seconds_target=15.0):
    """The oracle on the host cores, bounded sample: S samples x n steps of the
    198-site workload (FP64, all cores)."""
    import oracle
    wl = workload()
    threads = os.cpu_count() or 1
    S, n = max(threads, 16), 20
    t0 = time.perf_counter()
    oracle.run(wl["lat"], wl["U"], wl["n_up"], wl["n_dn"], 2, 0, S, 0.01, n, 10, threads=threads)
    dt = time.perf_counter() - t0
    # scale the sample to ~seconds_target
    n2 = max(n, int(n * seconds_target / max(dt, 1e-3)))
    n2 = min(n2, 1000)
    n2 -= n2 % 10
    t0 = time.perf_counter()
    oracle.run(wl["lat"], wl["U"], wl["n_up"], wl["n_dn"], 2, 0, S, 0.01, n2, 10, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": S * n2 / dt, "unit": UNIT, "cores": threads, "cpu_model": cpu_model(), "kind": "oracle",
            "sample": f"{S} samples x {n2} RK4 steps of the 198-site workload (FP64 C oracle, OpenMP)"}


def cpu_model():
    """The host CPU's model name (lscpu), for the CPU baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args):
    rank, local, ws = int(os.environ.get("RANK", "0")), 0, int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    wl = workload()
    threads = os.cpu_count() or 1
    S = max(threads, 16)
    # size one step to a few seconds of CPU work
    t0 = time.perf_counter()
    oracle.run(wl["lat"], wl["U"], wl["n_up"], wl["n_dn"], 2, 0, S, 0.01, 10, 10, threads=threads)
    per = (time.perf_counter() - t0) / 10
    n = max(10, min(1000, int(8.0 / max(per, 1e-4))))
    n -= n % 10
    for _ in range(args.warmup):
        oracle.run(wl["lat"], wl["U"], wl["n_up"], wl["n_dn"], 2, 0, S, 0.01, 10, 10, threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(wl["lat"], wl["U"], wl["n_up"], wl["n_dn"], 2, 0, S, 0.01, n, 10, threads=threads)
        times.append(time.perf_counter() - t0)
    ms = 1000 * sum(times) / len(times)
    v = S * n / (ms / 1000)
    sample = f"{S} samples x {n} RK4 steps of the 198-site workload per step (FP64 C oracle, OpenMP)"
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": config_dict(wl, {"reference_sample": sample}),
                      "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "cpu_model": cpu_model(),
                                       "kind": "oracle", "sample": sample},
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))



def g2_error_bar(X):
    """Delta-method standard error of the Eq. 10 estimator g2_kl =
    mean(x_k x_l) / (mean x_k mean x_l), x = X + 1/2, from the samples
    X [T, M, K] (FP32 products of centred columns: the scale of an error bar)."""
    import torch
    T, M, K = X.shape
    out = torch.empty((T, K, K), dtype=torch.float64, device=X.device)
    for t in range(T):
        x = X[t].double() + 0.5
        mu = x.mean(0)
        xc = (x - mu).float()
        x2 = xc * xc
        cov = (xc.T @ xc).double() / M
        e22 = (x2.T @ x2).double() / M
        e21 = (x2.T @ xc).double() / M
        B, C = mu[:, None], mu[None, :]
        g = (cov + B * C) / (B * C)
        var = e22 / (B * C) ** 2 - (cov / (B * C)) ** 2 + 2 * (1 - g) * (e21 / B + e21.T / C) / (B * C)
        va = torch.diagonal(cov)
        var = var + (1 - g) ** 2 * (va[:, None] / B ** 2 + 2 * cov / (B * C) + va[None, :] / C ** 2)
        out[t] = torch.sqrt(var.clamp_min(0) / M)
    return out


def observable_errors(X64, o64, c64, g64, o32, c32, g32, M, floor=1e-6):
    """max |FP32 - FP64| over times and entries, in units of each observable's
    statistical error bar: s_k/sqrt(M) (occupations), s_k s_l/sqrt(M)
    (connected correlator), the delta-method error (g2); floor 1e-6 where the
    bar vanishes (deterministic t = 0 diagonals)."""
    import torch
    s = torch.sqrt(torch.diagonal(c64, dim1=1, dim2=2).clamp_min(0))
    bo = (s / M ** 0.5).clamp_min(floor)
    bc = (s[:, :, None] * s[:, None, :] / M ** 0.5).clamp_min(floor)
    bg = g2_error_bar(X64).clamp_min(floor)
    ok = ~torch.isnan(g64) & ~torch.isnan(g32)
    return {"occupation": ((o32 - o64).abs() / bo).max().item(),
            "connected_correlator": ((c32 - c64).abs() / bc).max().item(),
            "g2": ((g32 - g64).abs()[ok] / bg[ok]).max().item()}


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def bench_adjoint(F, args):
    """Config 4: 96-site hexagonal flake (k = 4), U/t = 1.6, M samples, T = 5
    (500 RK4 steps, dt = 0.01), checkpoints every 50 steps, outputs every 10
    steps; loss sum_t,k (<n_k>(t) - target)^2 with a seeded synthetic target;
    gradients w.r.t. U, all 132 bond hoppings and the 192 initial
    occupations (softened Fock state 0.05/0.95 so that every noise scale is
    positive).  Reports the adjoint's wall time and its ratio to the forward
    pass of the same samples."""
    import numpy as np
    import torch
    import workloads as W
    lat = W.hexagonal_flake(4)
    nu, nd = W.neel_state(lat)
    nu, nd = W.softened(nu), W.softened(nd)
    M, steps, ck, every = args.adjoint_samples, 500, 50, 10
    rng = np.random.default_rng(4)
    target = torch.from_numpy(0.5 + 0.05 * rng.standard_normal((steps // every + 1, 2 * lat.n_sites))).cuda()
    out = {"workload": f"96-site flake, U/t=1.6, M={M}, T=5 (500 steps), checkpoints every 50",
           "samples": M}
    for name, prec in (("fp64", F.FTWA_FP64), ("fp32", F.FTWA_FP32)):
        P = F.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=prec, out_every=every)
        rho = P.sample(21, M)
        a, b = _events()
        a.record()
        X = P.evolve(rho, steps)
        b.record()
        occ, _, _ = P.moments(X, g2=False)
        torch.cuda.synchronize()
        fwd_ms = a.elapsed_time(b)
        loss = float(((occ - target) ** 2).sum())
        g = 2.0 * (occ - target)
        a, b = _events()
        a.record()
        gU, gt, gn = P.adjoint(21, M, steps, ck, g)
        b.record()
        torch.cuda.synchronize()
        if P.status() != 0:
            raise RuntimeError("adjoint device status")
        out[name] = {"adjoint_s": a.elapsed_time(b) / 1000.0, "forward_s": fwd_ms / 1000.0,
                     "ratio_to_forward": a.elapsed_time(b) / fwd_ms, "loss": loss, "dL_dU": gU.item(),
                     "dL_dt_norm": float(gt.norm()), "dL_dn0_norm": float(gn.norm())}
        P.close()
        del rho, X
    # finite-difference spot check at this workload's size (FP64, 64 samples,
    # the full 500 steps): dL/dU and two bond gradients by central differences
    # (h = 1e-5, same seed) of the GPU forward, against the adjoint
    Mfd, h = 64, 1e-5
    tb0 = np.array(lat.t_bond, dtype=np.float64)

    def loss_of(U, tb):
        lt = lat.with_t(tb)
        with F.Plan(lt, U, n_up=nu, n_dn=nd, precision=F.FTWA_FP64, out_every=every) as Q:
            o, _, _ = Q.moments(Q.evolve(Q.sample(21, Mfd), steps), g2=False)
            return float(((o - target) ** 2).sum()), o

    _, occ = loss_of(1.6, tb0)
    with F.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=F.FTWA_FP64, out_every=every) as Q:
        gU, gt, _ = Q.adjoint(21, Mfd, steps, ck, 2.0 * (occ - target))
    checks = [("dL_dU", gU.item(), (loss_of(1.6 + h, tb0)[0] - loss_of(1.6 - h, tb0)[0]) / (2 * h))]
    for bnd in (0, lat.n_bonds // 2):
        e = np.zeros(lat.n_bonds)
        e[bnd] = h
        checks.append((f"dL_dt{bnd}", gt[bnd].item(), (loss_of(1.6, tb0 + e)[0] - loss_of(1.6, tb0 - e)[0]) / (2 * h)))
    out["fd_check"] = {"samples": Mfd, "steps": steps, "h": h,
                       "values": {k: {"adjoint": a_, "central_difference": f_} for k, a_, f_ in checks},
                       "max_rel_err": max(abs(a_ - f_) / max(abs(f_), 1e-300) for _, a_, f_ in checks)}
    return out


def bench_general(F, args):
    """General initial state (Sec. 8(f) first extension): the 198-site flake in
    the thermal state of its hopping Hamiltonian (beta = 2, mu = 0.3), FP32,
    M samples: ftwa_sample = Eq. 7 in the eigenbasis + rho = V rho~ V^dagger
    (two complex N^3 products per sample and spin on the CUDA cores)."""
    import torch
    import workloads as W
    M = args.general_samples
    lat = W.brick_wall_flake(11, 18)
    nu, nd = W.neel_state(lat)
    lam, V = W.thermal_basis(lat, beta=2.0, mu=0.3)
    P = F.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=F.FTWA_FP32)
    P.set_initial_basis(lam, V)
    rho = P.new_state(M)
    P.sample(1, M, out=rho)
    torch.cuda.synchronize()
    a, b = _events()
    a.record()
    P.sample(2, M, out=rho)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    if P.status() != 0:
        raise RuntimeError("general sampling device status")
    N = lat.n_sites
    flops = 2 * 8.0 * N ** 3 * 2 * M
    pk = peaks()
    sm_count = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    fp32_peak = sm_count * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    P.close()
    del rho
    torch.cuda.empty_cache()
    return {"workload": f"198-site flake, thermal state of -J (beta=2, mu=0.3), FP32, M={M}",
            "ms": ms, "samples_per_s": M / (ms / 1000), "rotation_tflops": flops / (ms / 1000) / 1e12,
            "rotation_frac_of_fp32_peak": flops / (ms / 1000) / 1e12 / fp32_peak}


def bench_drive(F, args):
    """Tabulated diagonal field (Sec. 8(f) second and third extensions): the
    198-site workload in FP32 with a Gaussian-envelope pulse on every site,
    and with a long-range interaction u_ij over all pairs, against the plain
    on-site integration (M samples, n steps)."""
    import numpy as np
    import torch
    M, steps = args.drive_samples, args.drive_steps
    wl = workload(M=M, steps=steps)
    rng = np.random.default_rng(8)
    amp = rng.uniform(-1.0, 1.0, (2, wl["lat"].n_sites))
    import workloads as W
    out = {"workload": f"198-site flake, FP32, M={M}, {steps} RK4 steps; driven: pulse t0=0.5 sigma=0.3 "
                       f"omega=5 on all sites; longrange: u_ii = U, u_ij = 0.4 / r_ij (all pairs)"}
    for name in ("undriven", "driven", "longrange"):
        P = F.Plan(wl["lat"], wl["U"], n_up=wl["n_up"], n_dn=wl["n_dn"], precision=F.FTWA_FP32)
        if name == "driven":
            P.set_drive(amp, 0.5, 0.3, 5.0, 0.0)
        if name == "longrange":
            P.set_interaction(W.coulomb_interaction(wl["lat"], wl["U"], 0.4))
        rho = P.sample(1, M)
        P.evolve(rho, 5, snap=None)
        torch.cuda.synchronize()
        a, b = _events()
        a.record()
        P.evolve(rho, steps, snap=None, t_start=0.0)
        b.record()
        torch.cuda.synchronize()
        if P.status() != 0:
            raise RuntimeError("drive device status")
        out[name] = M * steps / (a.elapsed_time(b) / 1000.0)
        P.close()
        del rho
    out["unit"] = "sample-RK4-steps/s"
    out["driven_over_undriven"] = out["driven"] / out["undriven"]
    out["longrange_over_onsite"] = out["longrange"] / out["undriven"]
    torch.cuda.empty_cache()
    return out


def bench_ed(F, args):
    """GPU exact diagonalisation (Sec. 8(f) fourth extension): the 16-site
    brick-wall flake (4 x 4) at half filling, N_up = N_dn = 8 (basis
    12870^2 = 1.66e8 determinants), Neel start, U/t = 1.6, propagated to
    T = 1 in 10 Chebyshev intervals with <n> and <n n> at every interval."""
    import numpy as np
    import torch
    from scipy.special import jv
    import workloads as W
    lat = W.brick_wall_flake(4, 4)
    nu, nd = W.neel_state(lat)
    G = F.ED(lat, 1.6, int(nu.sum()), int(nd.sum()))
    dim, a_sp, _ = G.info()
    dt, n_out = 0.1, 10
    G.evolve(nu, nd, dt, 1)              # warm-up
    torch.cuda.synchronize()
    a, b = _events()
    a.record()
    occ, _ = G.evolve(nu, nd, dt, n_out)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    G.close()
    x = a_sp * dt                        # Chebyshev terms per interval, the library's rule
    k = 0
    while not (k > x + 10 and abs(jv(k, x)) < 1e-17):
        k += 1
    terms = k * n_out
    bytes_per_term = 80.0 * dim          # read T_k, T_k-1, acc; write T_k+1, acc (complex128)
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6784.5)
    gbs = bytes_per_term * terms / (ms / 1000.0) / 1e9
    return {"workload": "16-site brick-wall flake, N_up = N_dn = 8, U/t = 1.6, T = 1 (10 intervals of 0.1)",
            "dim": dim, "ms": ms, "chebyshev_terms": terms, "ms_per_term": ms / terms,
            "achieved_gbs": gbs, "hbm_peak_gbs": hbm, "frac_of_hbm_peak": gbs / hbm,
            "occ_sum_check": float(occ[-1].sum().item())}


def bench_batched(F, args):
    """Config 3: honeycomb flakes of 24, 54, 96, 150 and 198 sites x U/t in
    {0.5, 1.0, 1.6, 2.5}, M samples each, FP32 state, timed over
    args.batch_steps RK4 steps: one persistent kernel drawing (problem,
    sample batch) items from a cost-ordered queue (cluster and CTA sizes
    picked by the batch's autotuner), captured in a CUDA graph; beside it the
    earlier form, a graph of the 20 problems' own persistent steppers with
    per-problem autotuned shapes."""
    import torch
    import workloads as W
    lats = [W.hexagonal_flake(2), W.hexagonal_flake(3), W.hexagonal_flake(4), W.hexagonal_flake(5),
            W.brick_wall_flake(11, 18)]
    Us = [0.5, 1.0, 1.6, 2.5]
    M, steps = args.batch_samples, args.batch_steps
    plans, rhos, shapes = [], [], {}
    t0 = time.perf_counter()
    for lat in lats:
        nu, nd = W.neel_state(lat)
        tuner = F.Plan(lat, Us[0], n_up=nu, n_dn=nd, precision=F.FTWA_FP32)
        info = tuner.autotune(M, probe_steps=10)
        shapes[lat.n_sites] = {"variant": info["variant"], "cluster": info["cluster"]}
        tuner.close()
        for U in Us:
            P = F.Plan(lat, U, n_up=nu, n_dn=nd, precision=F.FTWA_FP32, variant=info["variant"],
                       cluster=info["cluster"])
            plans.append(P)
            rhos.append(P.sample(31, M))
    tune_s = time.perf_counter() - t0
    B = F.Batch(plans, rhos, steps)
    B.launch()                      # warm-up
    torch.cuda.synchronize()
    a, b = _events()
    a.record()
    B.launch()
    b.record()
    torch.cuda.synchronize()
    ms_graph = a.elapsed_time(b)
    B.close()
    t0 = time.perf_counter()
    B = F.Batch(plans, rhos, steps, persistent=True, tune=True)
    tune_p = time.perf_counter() - t0
    B.launch()                      # warm-up
    torch.cuda.synchronize()
    a, b = _events()
    a.record()
    B.launch()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    pshape = plans[-1].info()
    for P in plans:
        if P.status() != 0:
            raise RuntimeError("batched device status")
    total = len(plans) * M * steps
    flops = sum(FLOP_PER_ELEMENT_STEP * lt.n_sites * (lt.n_sites + 1) for lt in lats) * len(Us) * M * steps
    pk = max(F.measure_peak("fp32"), F.measure_peak("fp32x2")) / 1e12
    pks = F.measure_peak("smem") / 1e12
    achieved = flops / (ms / 1000.0) / 1e12
    smem_tb = achieved * 1e12 / FLOP_PER_ELEMENT_STEP * SMEM_BYTES_PER_ELEMENT_STEP / 1e12
    out = {"workload": f"flakes 24/54/96/150/198 sites x U in {Us}, M={M} each, FP32, {steps} RK4 steps",
           "problems": len(plans), "value": total / (ms / 1000.0), "unit": UNIT, "ms": ms,
           "launch": "one persistent kernel, cost-ordered work queue, CUDA graph",
           "persistent_shape": {"cluster_of_198_sites": pshape["cluster"], "threads": pshape["threads"]},
           "autotune_s": tune_p, "graph_launches": 1,
           "per_problem_graph": {"value": total / (ms_graph / 1000.0), "ms": ms_graph, "shapes": shapes,
                                 "autotune_s": tune_s},
           "roofline": {"bound": "smem", "achieved": smem_tb, "peak": pks, "unit": "TB/s", "frac": smem_tb / pks,
                        "fp32": {"achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk}}}
    B.close()
    for P in plans:
        P.close()
    return out


def bench_gram(F, args):
    """Config 5 shape: all-pairs connected correlator of M = 65536 samples x
    396 site-spin occupations at 200 output times, BF16x3 tensor-core Gram
    against the FP64 Gram.  Snapshots are synthetic FP32 values with the
    value range of Re rho_ii (uniform in [-1/2, 1/2] plus a per-site mean)."""
    import torch
    M, K, T = args.gram_samples, 396, args.gram_times
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    X = (torch.rand((T, M, K), generator=g, device="cuda", dtype=torch.float32) - 0.5)
    X += 0.1 * torch.rand((1, 1, K), generator=g, device="cuda")
    import workloads as W
    lat = W.brick_wall_flake(11, 18)
    nu, nd = W.neel_state(lat)
    P = F.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=F.FTWA_FP32)
    res = {}
    for name, mode in (("bf16x3", F.FTWA_GRAM_BF16X3), ("fp64", F.FTWA_GRAM_FP64)):
        P.moments(X, gram_mode=mode, g2=True)       # warm-up (workspace)
        torch.cuda.synchronize()
        a, b = _events()
        a.record()
        occ, conn, g2 = P.moments(X, gram_mode=mode, g2=True)
        b.record()
        torch.cuda.synchronize()
        res[name] = (a.elapsed_time(b), conn)
    if P.status() != 0:
        raise RuntimeError("gram device status")
    c16, c64 = res["bf16x3"][1], res["fp64"][1]
    d = torch.sqrt(torch.diagonal(c64, dim1=1, dim2=2).clamp_min(0))
    stat = d[:, :, None] * d[:, None, :] / (M ** 0.5)        # statistical error scale of C_kl
    err = ((c16 - c64).abs() / stat.clamp_min(1e-30)).max().item()
    n_kt = (K + 127) // 128
    # MMA work issued: M = 128 rows per tile, N = 128 columns, or the real
    # columns of the last site block rounded up to 16
    ncol = [min(128, K - 128 * lt) for lt in range(n_kt)]
    n_of = [(c + 15) // 16 * 16 for c in ncol]
    tiles = n_kt * (n_kt + 1) // 2
    mma_flops = 3 * 2.0 * M * 128 * sum(n_of[lt] for kt in range(n_kt) for lt in range(kt, n_kt)) * T
    useful = 2.0 * M * K * (K + 1) / 2 * T
    pk = peaks()
    ms16 = res["bf16x3"][0]
    out = {"workload": f"M={M} samples x K={K} x T={T} times, synthetic FP32 snapshots",
           "bf16x3_ms": ms16, "fp64_ms": res["fp64"][0], "speedup": res["fp64"][0] / ms16,
           "bf16_mma_tflops": mma_flops / (ms16 / 1000) / 1e12,
           "useful_tflops": useful / (ms16 / 1000) / 1e12,
           "frac_of_bf16_peak": mma_flops / (ms16 / 1000) / 1e12 / pk.get("bf16_tflops", 1912.7),
           "max_err_over_stat_err": err}
    P.close()
    del X, res, c16, c64
    torch.cuda.empty_cache()
    return out

def run_gpu(args):
    import numpy as np
    import torch

    rank, local, ws = dist_init()
    torch.cuda.set_device(local)
    import paper_2212_04352_gb300 as F
    F.load()
    wl = workload(M=args.samples)
    lat, M, steps, every = wl["lat"], wl["M"], wl["steps"], wl["every"]
    N = lat.n_sites
    from paper_2212_04352_gb300 import shard
    first, _ = shard.sample_range(rank, ws, M)
    P = F.Plan(lat, wl["U"], n_up=wl["n_up"], n_dn=wl["n_dn"], precision=F.FTWA_FP32, out_every=every)
    stream = torch.cuda.current_stream()
    rho = P.new_state(M)
    X = torch.empty((P.n_out(steps), M, 2 * N), dtype=torch.float32, device="cuda")
    K = 2 * N
    T = P.n_out(steps)
    occ = torch.empty((T, K), dtype=torch.float64, device="cuda")
    conn = torch.empty((T, K, K), dtype=torch.float64, device="cuda")
    g2 = torch.empty((T, K, K), dtype=torch.float64, device="cuda")
    from paper_2212_04352_gb300 import _lib, check, load
    import ctypes
    lib = load()
    sp = ctypes.c_void_p(stream.cuda_stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]

    def one_step(k, timed):
        check(lib.ftwa_sample(P._h, 7, first, M, ctypes.c_void_p(rho.data_ptr()), sp), "sample")
        if timed:
            ev[k][0].record(stream)
        check(lib.ftwa_evolve(P._h, ctypes.c_void_p(rho.data_ptr()), M, steps, ctypes.c_void_p(X.data_ptr()), sp),
              "evolve")
        if timed:
            ev[k][1].record(stream)
        check(lib.ftwa_moments(P._h, ctypes.c_void_p(X.data_ptr()), M, T, ctypes.c_void_p(occ.data_ptr()),
                               ctypes.c_void_p(conn.data_ptr()), ctypes.c_void_p(g2.data_ptr()), F.FTWA_GRAM_BF16X3,
                               sp), "moments")
        if ws > 1:
            # exchange step: the estimators over the union of all ranks' samples
            shard.combine_moments(M, occ, conn, ws)

    # the last two warm-up steps run under the profiler (the first session of a
    # process may miss device records); the last one counts the kernels of a step
    n_prof = 2 if args.warmup >= 2 else max(args.warmup, 1)
    for _ in range(args.warmup - n_prof):
        one_step(0, False)
    launches_per_step = count_kernels(lambda: one_step(0, False), sessions=n_prof)
    torch.cuda.synchronize()
    if P.status() != 0:
        raise RuntimeError("device status after warm-up")
    info = P.info()
    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(args.steps):
        one_step(k, True)
    end.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    total_ms = start.elapsed_time(end)
    total_ms = max_over_ranks(total_ms, ws)
    evolve_ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    if P.status() != 0:
        raise RuntimeError("device status after timed region")
    ms_per_step = total_ms / args.steps
    value = ws * M * steps / (ms_per_step / 1000.0)

    # ---- end to end through the public API with host buffers ---------------------
    e2e = None
    if not args.no_e2e:
        occ_h = torch.empty((T, K), dtype=torch.float64, pin_memory=True)
        conn_h = torch.empty((T, K, K), dtype=torch.float64, pin_memory=True)
        g2_h = torch.empty((T, K, K), dtype=torch.float64, pin_memory=True)
        nu_h = torch.from_numpy(np.asarray(wl["n_up"], dtype=np.float64)).pin_memory()
        nd_h = torch.from_numpy(np.asarray(wl["n_dn"], dtype=np.float64)).pin_memory()
        n_dev = torch.empty((2, N), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            # inputs of the step: the initial occupations (host -> device)
            n_dev[0].copy_(nu_h, non_blocking=True)
            n_dev[1].copy_(nd_h, non_blocking=True)
            torch.cuda.synchronize()
            Pk = F.Plan(lat, wl["U"], n_up=n_dev[0].cpu().numpy(), n_dn=n_dev[1].cpu().numpy(),
                        precision=F.FTWA_FP32, out_every=every)
            Pk.sample(7, M, first_sample=first, out=rho)
            Xk = Pk.evolve(rho, steps, snap=X)
            o, c, g = Pk.moments(X, gram_mode=F.FTWA_GRAM_BF16X3)
            occ_h.copy_(o, non_blocking=True)
            conn_h.copy_(c, non_blocking=True)
            g2_h.copy_(g, non_blocking=True)
            torch.cuda.synchronize()
            Pk.close()
        dt = time.perf_counter() - t0
        dt = max_over_ranks(dt, ws)
        e2e = {"value": ws * M * steps * args.e2e_steps / dt, "unit": UNIT,
               "h2d_bytes_per_step": 2 * N * 8 + lat.n_bonds * 8 * 3,
               "d2h_bytes_per_step": (T * K + 2 * T * K * K) * 8}

    # ---- FP64 GPU path on a subset, and the FP32 path's error against it ---------
    # (the FP64 path is pinned to the oracle trajectory by trajectory; every
    # reported observable: max |FP32 - FP64| in units of its error bar)
    fp64 = None
    if not args.no_fp64:
        Ms = args.fp64_samples
        fp64 = {"unit": UNIT, "samples": Ms, "errors": {}}
        for U in (1.0, wl["U"]):
            P64 = F.Plan(lat, U, n_up=wl["n_up"], n_dn=wl["n_dn"], precision=F.FTWA_FP64, out_every=every)
            P32 = F.Plan(lat, U, n_up=wl["n_up"], n_dn=wl["n_dn"], precision=F.FTWA_FP32, out_every=every)
            r64 = P64.sample(11, Ms)
            r32 = P32.sample(11, Ms)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            X64 = P64.evolve(r64, steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms64 = e0.elapsed_time(e1)
            X32 = P32.evolve(r32, steps)
            o64, c64, g64 = P64.moments(X64)
            o32, c32, g32 = P32.moments(X32, gram_mode=F.FTWA_GRAM_BF16X3)
            err = observable_errors(X64, o64, c64, g64, o32, c32, g32, Ms)
            fp64["errors"][f"U={U}"] = err
            if U == wl["U"]:
                fp64["value"] = Ms * steps / (ms64 / 1000.0)
                fp64["fp32_speedup_vs_fp64"] = (M * steps / (evolve_ms / 1000.0)) / fp64["value"]
            P64.close()
            P32.close()
            del r64, r32, X64, X32
        fp64["gate"] = "max error / error bar < 0.1 for every observable (occupation, connected correlator, g2)"
        fp64["gate_met"] = all(v < 0.1 for e in fp64["errors"].values() for v in e.values())
        fp64["peak_fp64_tflops"] = F.measure_peak("fp64") / 1e12
        flops64 = FLOP_PER_ELEMENT_STEP * N * (N + 1) * fp64["value"]
        fp64["roofline"] = {"bound": "alu", "achieved": flops64 / 1e12, "peak": fp64["peak_fp64_tflops"],
                            "unit": "TFLOP/s", "frac": flops64 / 1e12 / fp64["peak_fp64_tflops"],
                            "peak_source": "measured: ftwa_measure_peak FP64 FMA"}

    # ---- the same step at U/t = 1.0 (the paper's regime U = J) -----------------------
    u_alt = None
    if not args.no_u1:
        Pu = F.Plan(lat, 1.0, n_up=wl["n_up"], n_dn=wl["n_dn"], precision=F.FTWA_FP32, out_every=every)
        Pu.sample(7, M, first_sample=first, out=rho)
        Pu.evolve(rho, 5, snap=None)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Pu.sample(7, M, first_sample=first, out=rho)
        Pu.evolve(rho, steps, snap=X)
        Pu.moments(X, gram_mode=F.FTWA_GRAM_BF16X3)
        e1.record(stream)
        torch.cuda.synchronize()
        if Pu.status() != 0:
            raise RuntimeError("U = 1.0 leg device status")
        u_alt = {"U_over_t": 1.0, "value": ws * M * steps / (e0.elapsed_time(e1) / 1000.0), "unit": UNIT,
                 "ms_per_step": e0.elapsed_time(e1)}
        Pu.close()

    extra = {}
    if not args.no_adjoint:
        extra["adjoint"] = bench_adjoint(F, args)
    if not args.no_batch:
        extra["batched"] = bench_batched(F, args)
    if not args.no_gram:
        extra["gram"] = bench_gram(F, args)
    if not args.no_general:
        extra["general_state"] = bench_general(F, args)
    if not args.no_drive:
        extra["drive"] = bench_drive(F, args)
    if not args.no_ed:
        extra["ed"] = bench_ed(F, args)

    # ---- roofline of the dominant kernel (the RK4 stepper) -----------------------
    # bound: shared memory (the smaller of the stepper's two bounds); the FP32
    # fraction beside it.  Peaks measured on this device by the library's
    # micro-benchmarks (MEASURED_PEAKS.json has neither).
    pk_smem = F.measure_peak("smem") / 1e12                         # TB/s
    pk_fp32 = max(F.measure_peak("fp32"), F.measure_peak("fp32x2")) / 1e12   # TFLOP/s
    flops = FLOP_PER_ELEMENT_STEP * N * (N + 1) * M * steps
    achieved = flops / (evolve_ms / 1000.0) / 1e12
    info_kernel = {1: "band_stepper<float>", 2: "rk4_stepper<float>", 3: "tile_stepper<float>"}.get(info["variant"])
    src = "ftwa_tile.cu" if info["variant"] == 3 else "ftwa_evolve.cu"
    rec = "tile_stepper_fp32_198_traffic.txt" if info["variant"] == 3 else "band_stepper_fp32_198_traffic.txt"
    traffic = traffic_record(os.path.join(ROOT, "paper_2212_04352_gb300", "csrc", src), rec)
    smem_bytes = SMEM_BYTES_PER_ELEMENT_STEP * N * (N + 1) * M * steps
    smem_achieved = smem_bytes / (evolve_ms / 1000.0) / 1e12
    roof = {"bound": "smem", "achieved": smem_achieved, "peak": pk_smem, "unit": "TB/s",
            "frac": smem_achieved / pk_smem, "traffic": traffic, "kernel": info_kernel,
            "bytes_per_element_step": SMEM_BYTES_PER_ELEMENT_STEP,
            "peak_source": "measured: ftwa_measure_peak shared-memory load bandwidth (all SMs, 16-byte loads)",
            "fp32": {"achieved": achieved, "peak": pk_fp32, "unit": "TFLOP/s", "frac": achieved / pk_fp32,
                     "flop_per_element_step": FLOP_PER_ELEMENT_STEP,
                     "peak_source": "measured: ftwa_measure_peak FP32 FMA (max of scalar and packed pairs)"}}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": config_dict(wl, {"parallelism": f"samples split over {ws} GPU(s); estimators all-reduced "
                                                        f"at the end of each step when more than one",
                                       "launch": info}),
            "e2e": e2e, "roofline": roof, "clocks": clk, "gpu_launches": (launches_per_step * args.steps if launches_per_step is not None else None),
            "evolve_ms": evolve_ms, "fp64": fp64, "u_1p0": u_alt, **extra}
    if rank == 0 and ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line))
    P.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_profile_case(args):
    """A small invocation for ncu captures: one sample -> evolve -> moments pass
    on the 198-site workload with few samples and steps."""
    import torch
    import paper_2212_04352_gb300 as F
    wl = workload(M=args.samples, steps=args.prof_steps)
    prec = F.FTWA_FP64 if args.precision == "fp64" else F.FTWA_FP32
    P = F.Plan(wl["lat"], wl["U"], n_up=wl["n_up"], n_dn=wl["n_dn"], precision=prec, out_every=wl["every"],
               variant=args.variant)
    for _ in range(args.prof_repeat):
        rho = P.sample(7, wl["M"])
        X = P.evolve(rho, wl["steps"])
        P.moments(X, gram_mode=args.gram)
    torch.cuda.synchronize()
    st = P.status()
    print(json.dumps({"profile_case": True, "samples": wl["M"], "steps": wl["steps"], "status": st,
                      "launch": P.info()}))
    if st != 0:
        raise SystemExit(1)


def run_profile_gram(args):
    """A small Gram case for ncu: T times (default 15, one batch of the
    tensor-core Gram) of M = 65536 synthetic FP32 snapshots of the 198-site
    workload's 396 site-spin occupations."""
    import torch
    import paper_2212_04352_gb300 as F
    import workloads as W
    M, K, T = 65536, 396, args.gram_prof_times
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    X = torch.rand((T, M, K), generator=g, device="cuda", dtype=torch.float32) - 0.5
    lat = W.brick_wall_flake(11, 18)
    nu, nd = W.neel_state(lat)
    P = F.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=F.FTWA_FP32)
    for _ in range(args.prof_repeat):
        P.moments(X, gram_mode=F.FTWA_GRAM_BF16X3)
    torch.cuda.synchronize()
    st = P.status()
    print(json.dumps({"profile_gram": True, "M": M, "K": K, "T": T, "status": st}))
    if st != 0:
        raise SystemExit(1)


def run_profile_adjoint(args):
    """A small adjoint case for ncu: 96-site flake, U/t = 1.6, softened Neel
    occupations, 608 samples (one per CTA slot), 50 RK4 steps, checkpoints and
    outputs every 10 steps, repeated --prof-repeat times (CUDA-event times)."""
    import torch
    import paper_2212_04352_gb300 as F
    import workloads as W
    lat = W.hexagonal_flake(4)
    nu, nd = W.neel_state(lat)
    nu, nd = W.softened(nu), W.softened(nd)
    M, steps, every, ckpt = 608, 50, 10, 10
    prec = F.FTWA_FP64 if args.precision == "fp64" else F.FTWA_FP32
    times = []
    with F.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=prec, out_every=every) as P:
        g = torch.full((steps // every + 1, 2 * lat.n_sites), 0.3, dtype=torch.float64, device="cuda")
        for _ in range(args.prof_repeat):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            P.adjoint(1, M, steps, ckpt, g)
            e.record()
            torch.cuda.synchronize()
            times.append(s.elapsed_time(e))
        st = P.status()
    print(json.dumps({"profile_adjoint": True, "precision": args.precision, "samples": M, "steps": steps,
                      "ms": times, "status": st}))
    if st != 0:
        raise SystemExit(1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--samples", type=int, default=16384)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--fp64-samples", type=int, default=512)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-gram", action="store_true")
    ap.add_argument("--no-general", action="store_true")
    ap.add_argument("--no-drive", action="store_true")
    ap.add_argument("--no-ed", action="store_true")
    ap.add_argument("--no-u1", action="store_true")
    ap.add_argument("--drive-samples", type=int, default=4096)
    ap.add_argument("--drive-steps", type=int, default=200)
    ap.add_argument("--general-samples", type=int, default=4096)
    ap.add_argument("--adjoint-samples", type=int, default=4096)
    ap.add_argument("--batch-samples", type=int, default=4096)
    ap.add_argument("--batch-steps", type=int, default=1000)
    ap.add_argument("--gram-samples", type=int, default=65536)
    ap.add_argument("--gram-times", type=int, default=200)
    ap.add_argument("--profile", action="store_true", help="small case for ncu captures")
    ap.add_argument("--profile-gram", action="store_true", help="small Gram case for ncu captures")
    ap.add_argument("--profile-adjoint", action="store_true", help="small adjoint case for ncu captures")
    ap.add_argument("--prof-steps", type=int, default=20)
    ap.add_argument("--prof-repeat", type=int, default=2)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--gram", type=int, default=0)
    ap.add_argument("--gram-prof-times", type=int, default=15)
    ap.add_argument("--variant", type=int, default=0, help="stepper variant of the profile case (0 automatic)")
    args = ap.parse_args()
    if args.profile:
        run_profile_case(args)
        return
    if args.profile_gram:
        run_profile_gram(args)
        return
    if args.profile_adjoint:
        run_profile_adjoint(args)
        return
    if args.warmup < 3 and args.impl == "native":
        print("note: fewer than 3 warm-up steps; the timing contract asks for >= 3", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
