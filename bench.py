"""Benchmark: site-updates/s of the kagome DQMC sweep on GB300.

One step = one sweep (up + down pass, 2 N M Metropolis proposals) of one
Markov chain per GPU, on synthetic input (Philox-initialised Ising field).
Default workload: L = 24 (N = 1728), beta = 24, dtau = 0.1 (M = 240), U = -4
(|U| = 4 attractive), mu = -1, delay rank k = 32, stabilisation every 8
slices, mixed precision.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
               [--workload NAME] [--precision fp64|mixed|fp32]
Under torchrun every rank runs its own chain (seed + rank): replicas, weak
scaling, no data-path collective. Rank 0 prints one JSON line.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from dqmc_inputs import WORKLOADS  # noqa: E402

METRIC = "site-updates/s per GB300 at L=24 kagome: FP32+FP64-stab vs plain FP64 at |ΔG|≤1e-6"
UNIT = "site-updates/s"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# GB300: 152 SMs; per SM per clock 128 FP32 FMA and 2 FP64 FMA (the FP64 rate
# is 1/64 of FP32 on this part: 152 * 2 * 2 * 2.07 GHz = 1.26 TFLOP/s, the
# nominal 1.25 TFLOP/s)
N_SM = 152


def alu_peak_tflops(kind, mhz):
    per_sm_flops = {"fp64": 2 * 2, "fp32": 128 * 2}[kind]
    return N_SM * per_sm_flops * mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[4:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ("active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = set()
        for _, _, flags in rows:
            for n, v in zip(names[1:], flags[1:]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def workload(args):
    w = dict(WORKLOADS[args.workload])
    if args.precision:
        w["precision"] = args.precision
    return w


def parse_options(items):
    """--option key=value (repeatable): library options set on the chain
    before its first sweep, e.g. pipeline=0 for a single-stream sweep."""
    out = {}
    for it in items or []:
        key, _, val = it.partition("=")
        if not key or not val:
            raise SystemExit(f"--option expects key=value, got {it!r}")
        out[key] = float(val)
    return out


def config_dict(w, world):
    L = w["L"]
    M = int(round(w["beta"] / w["dtau"]))
    opts = parse_options(args_global.option)
    extra = {"options": opts} if opts else {}
    return {**extra, 
        "workload": f"{args_global.workload}: kagome L={L} (N={3 * L * L}), beta={w['beta']}, dtau={w['dtau']} "
                    f"(M={M}), U={w['U']}, mu={w['mu']}, k={w['k']}, n_stab={w['n_stab']}, "
                    f"precision={w['precision']}, one chain per GPU",
        "L": L, "N": 3 * L * L, "M": M, "beta": w["beta"], "U": w["U"], "mu": w["mu"], "k": w["k"],
        "n_stab": w["n_stab"], "precision": w["precision"], "parallelism": f"replicas x{world}",
        "l2": "working set larger than L2 (UDV stacks and G per chain)",
    }


def cpu_oracle_sample(w, budget_s=20.0):
    """The oracle as it stands on this host: wrap + N proposals per slice visit
    (refresh excluded), the number of visits sized to ~budget_s."""
    from oracle import dqmc as odqmc
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    t1, n1, _ = odqmc.time_slice_visits(w["L"], w["beta"], w["dtau"], w["U"], w["mu"], w["seed"], 1,
                                        n_stab=w["n_stab"], with_refresh=False)
    M = int(round(w["beta"] / w["dtau"]))
    visits = max(1, min(64, M, int(budget_s / max(t1, 1e-3))))
    t, n, _ = odqmc.time_slice_visits(w["L"], w["beta"], w["dtau"], w["U"], w["mu"], w["seed"], visits,
                                      n_stab=w["n_stab"], with_refresh=False)
    return {"value": n / t, "unit": UNIT, "cores": cores, "kind": "oracle", "proposals": n, "seconds": t,
            "refresh_excluded": True,
            "sample": f"{visits} up-pass slice visits at L={w['L']} (wrap + {3 * w['L'] ** 2} one-at-a-time "
                      f"proposals each, numpy FP64 on {cores} host threads), UDV refresh excluded "
                      f"(so the rate overstates a whole oracle sweep), {t:.1f} s"}


def run_reference(args, rank, world):
    w = workload(args)
    if rank != 0:
        return
    per_step = []
    samples = None
    for i in range(args.warmup + args.steps):
        s = cpu_oracle_sample(w, budget_s=max(2.0, 60.0 / max(1, args.warmup + args.steps)))
        if i >= args.warmup:
            per_step.append(s)
        samples = s
    # each step is a bounded sample (a few slice visits, not a whole sweep):
    # value = proposals / s over the samples, ms_per_step = the samples' own time
    props = sum(s["proposals"] for s in per_step)
    secs = sum(s["seconds"] for s in per_step)
    value = props / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * secs / len(per_step),
        "step_definition": "a bounded sample of up-pass slice visits of the workload (wrap + N "
                           "one-at-a-time proposals each), UDV refresh excluded; not a whole sweep",
        "extrapolated": False, "refresh_excluded": True,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (Philox-initialised Ising field)", "config": config_dict(w, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": samples["cores"], "kind": "oracle",
                         "sample": samples["sample"], "refresh_excluded": True},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def prop_microbench(L, prec, nstack, reps=5):
    """Left propagation e^{-dtau K} X (Eq. 5-6) on a stacked operand X of
    nstack N x N blocks side by side (N x nstack N, larger than L2), in place;
    returns the algorithmic HBM rate (one read + one write of X per launch)."""
    import numpy as np
    import torch

    import paper_2608_03894_gb300 as pkg
    N = 3 * L * L
    dt = torch.float32 if prec == "fp32" else torch.float64
    X = torch.randn((N, nstack * N), dtype=dt, device="cuda")
    df = prec == "df"
    for _ in range(2):
        pkg.ops.propagate(L, -0.1, 0, X, Y=X, df=df)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        pkg.ops.propagate(L, -0.1, 0, X, Y=X, df=df)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    nbytes = 2.0 * X.numel() * X.element_size()
    L2 = float(L * L)
    flops = (15.0 * L2 * np.log2(L2) + 36.0 * L2) * nstack * N
    del X
    return {"L": L, "arith": prec, "operand_MB": round(nbytes / 2 / 1e6, 1), "ms_per_launch": round(ms, 4),
            "GB_s": round(nbytes / (ms * 1e-3) / 1e9, 1), "TFLOP_s": round(flops / (ms * 1e-3) / 1e12, 3)}


def gemm_microbench(n, mode, reps=5):
    """The stabilisation GEMM C = A B (n x n x n, FP64 data) in one of its
    arithmetics: FP64 FMA, double-float, digit slices on the bf16 tensor cores."""
    import torch

    import paper_2608_03894_gb300 as pkg
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    B = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    C = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    for _ in range(2):
        pkg.ops.gemm(A, B, C, mode=mode)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        pkg.ops.gemm(A, B, C, mode=mode)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"n": n, "mode": mode, "ms": round(ms, 4), "TFLOP_s_fp64_equivalent": round(2.0 * n ** 3 / (ms * 1e-3) / 1e12, 3)}


def metro_microbench(L, k, df, reps=200):
    """One delayed-update block alone (decisions + Woodbury coefficients) on a
    G-like block of the L x L torus, then the rank-k flush of that block:
    device time per launch (CUDA events around `reps` back-to-back launches,
    buffers allocated once)."""
    import ctypes as C

    import torch

    from dqmc_inputs import random_green_like
    from paper_2608_03894_gb300 import _lib
    lib = _lib.load()
    N = 3 * L * L
    G = torch.as_tensor(random_green_like(N, 1), dtype=torch.float64, device="cuda")
    s = torch.ones(N, dtype=torch.int8, device="cuda")
    g = G[:k, :k].contiguous()
    Gcol, Grow = G[:, :k].contiguous(), G[:k, :].contiguous()
    al = torch.zeros((k, k), dtype=torch.float64, device="cuda")
    be = torch.zeros((k, k), dtype=torch.float64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    P = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    metro = lib.dqmc_op_metropolis_block_df if df else lib.dqmc_op_metropolis_block
    flush = lib.dqmc_op_flush_df if df else lib.dqmc_op_flush_f64
    res = {}
    for name in ("metropolis", "flush"):
        for i in range(reps + 5):
            if i == 5:
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
            if name == "metropolis":
                _lib.check(metro(N, 0, k, P(g), k, P(s), 0.6538, 1, 0, i, 1, None, P(al), P(be), P(cnt), P(st), stream))
            else:
                _lib.check(flush(N, 0, k, P(G), P(Gcol), P(Grow), P(al), P(be), P(cnt), stream))
        e1.record()
        torch.cuda.synchronize()
        res[name + "_us"] = round(1000.0 * e0.elapsed_time(e1) / reps, 2)
    res["accepted"] = int(cnt.item())
    return {"L": L, "k": k, "arith": "df" if df else "f64", **res}


def update_microbench(L, reps=4):
    """One delayed-update block of the mixed-precision sweep through the C ABI,
    repeated: the double-float Metropolis block (k = 32) on a G-like block, then
    the tensor-core flush (digit tiles + tcgen05 update) of that block. Device
    time per repetition (CUDA events). Also the driver of the ncu captures of
    these kernels (profiles/)."""
    import torch

    import paper_2608_03894_gb300 as pkg
    from dqmc_inputs import random_field, random_green_like
    k, N = 32, 3 * L * L
    site0 = min(N - k, (N // 2) // k * k)
    G0 = torch.as_tensor(random_green_like(N, 3), dtype=torch.float64, device="cuda")
    s0 = torch.as_tensor(random_field(1, N, seed=3)[0], dtype=torch.int8, device="cuda")
    g = G0[site0:site0 + k, site0:site0 + k].contiguous()
    Gcol, Grow = G0[:, site0:site0 + k].contiguous(), G0[site0:site0 + k, :].contiguous()
    ts = []
    for _ in range(reps):
        s = s0.clone()
        G = G0.clone()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        al, be, cnt, st = pkg.ops.metropolis_block(N, site0, k, g, s, 0.6538, 11, 0, 1, 1, df=True)
        pkg.ops.flush(N, site0, k, G, Gcol, Grow, al, be, cnt, mode="tc")
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) * 1000.0)
    return {"L": L, "k": k, "accepted": int(cnt.item()), "block_us_incl_op_overheads": [round(t, 1) for t in ts]}


def stab_microbench(L):
    """A short mixed-precision chain at the bench size (beta = L / 10: M = L
    slices, n_stab = 8): one sweep, whose refreshes run the stabilisation
    kernels of the full workload (QR panels, digit-slice GEMMs) at N = 3 L^2.
    Wall time of the sweep. Also the driver of the ncu captures of those
    kernels (profiles/)."""
    import time

    import torch

    import paper_2608_03894_gb300 as pkg
    with pkg.DQMC(L, L / 10.0, 0.1, -4.0, -1.0, seed=1, k=32, n_stab=8, precision="mixed") as d:
        t = time.time()
        d.sweep(1)
        torch.cuda.synchronize()
        return {"L": L, "M": L, "sweep_s": round(time.time() - t, 3), "max_drift": d.stats()["max_drift"]}


def batch_microbench(steps=2, warmup=1):
    """The batched-chain workload: 64 independent chains on one GPU, 32 at
    L = 12 (beta = 12, M = 120) and 32 at L = 16 (beta = 16, M = 160), U
    cycling through -3, -4, -5, -6, mu = -1, dtau = 0.1, mixed precision,
    every chain on its own stream and host thread (dqmc_batch_sweep). The
    autotuner picks first the delay rank of each size (k in 16, 32, 64 at
    U = -4, n_stab 8), then the refresh interval of each U at the larger size
    (n_stab in 4, 6, 8, drift bar 3e-7 over its two sweeps: stronger coupling
    amplifies the wrap error faster). One step = one sweep of every chain;
    site-updates/s over the whole batch, device time between two full
    synchronisations (CUDA events)."""
    import torch

    import paper_2608_03894_gb300 as pkg
    sizes = ((12, 12.0), (16, 16.0))
    Us = (-3.0, -4.0, -5.0, -6.0)

    def table(r):
        return {f"k={k},n_stab={n}": (None if t is None else round(t, 4)) for (k, n), t in r["table"].items()}

    tuned_k, tuned_ns = {}, {}
    for L, beta in sizes:
        r = pkg.autotune(L, beta, 0.1, -4.0, -1.0, seed=1, precision="mixed", ks=(16, 32, 64), n_stabs=(8,),
                         warmup=1, sweeps=1, drift_bar=1e-6)
        tuned_k[L] = {"k": r["k"], "sec_per_sweep": round(r["sec_per_sweep"], 4), "table": table(r)}
    L, beta = sizes[-1]
    for U in Us:
        try:
            r = pkg.autotune(L, beta, 0.1, U, -1.0, seed=1, precision="mixed", ks=(tuned_k[L]["k"],),
                             n_stabs=(4, 6, 8), warmup=1, sweeps=1, drift_bar=3e-7)
        except pkg.DQMCError:
            r = pkg.autotune(L, beta, 0.1, U, -1.0, seed=1, precision="mixed", ks=(tuned_k[L]["k"],),
                             n_stabs=(2,), warmup=1, sweeps=1, drift_bar=1e-6)
        tuned_ns[U] = {"n_stab": r["n_stab"], "sec_per_sweep": round(r["sec_per_sweep"], 4), "table": table(r)}
    params = []
    for L, beta in sizes:
        for i in range(32):
            params.append((L, beta, 0.1, Us[i % 4], -1.0, len(params) + 1))
    units = sum(2 * 3 * L * L * int(round(beta / 0.1)) for L, beta, *_ in params)
    with pkg.Batch(params, precision="mixed") as b:
        for c, p in zip(b.chains, params):
            c.set_option("k", tuned_k[p[0]]["k"])
            c.set_option("n_stab", tuned_ns[p[3]]["n_stab"])
        b.sweep(warmup)
        sampler = ClockSampler(0)
        torch.cuda.synchronize()
        with sampler:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            t0 = time.perf_counter()
            b.sweep(steps)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            e1.record()
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        stats = [c.stats() for c in b.chains]
    drift = {f"L={L},U={U}": max(s["max_drift"] for s, p in zip(stats, params) if p[0] == L and p[3] == U)
             for L, _ in sizes for U in Us}
    return {"workload": "batch64: 32 chains at L=12 (N=432, beta=12, M=120) + 32 at L=16 (N=768, beta=16, "
                        "M=160), U in {-3,-4,-5,-6}, mu=-1, dtau=0.1, mixed precision, autotuned k and "
                        "n_stab, one stream and host thread per chain",
            "value": units * steps / (ms / 1000.0), "unit": UNIT, "steps": steps, "warmup": warmup,
            "ms_per_step": ms / steps, "wall_s_per_step": wall / steps,
            "chain_sweeps_per_s": len(params) * steps / (ms / 1000.0), "site_updates_per_step": units,
            "autotune_k": {str(k): v for k, v in tuned_k.items()},
            "autotune_n_stab": {str(u): v for u, v in tuned_ns.items()},
            "max_drift": max(drift.values()), "max_drift_by_group": drift,
            "acceptance": sum(s["accepted"] for s in stats) / max(1, sum(s["proposed"] for s in stats)),
            "clocks": sampler.summary()}


def run_micro(args):
    import torch
    torch.cuda.set_device(0)
    peaks, src = load_peaks()
    out = []
    if args.micro == "update":
        print(json.dumps({"micro": "update", "results": [update_microbench(args.micro_L)]}), flush=True)
        return
    if args.micro == "batch":
        print(json.dumps({"micro": "batch", "results": [batch_microbench()]}), flush=True)
        return
    if args.micro == "stab":
        print(json.dumps({"micro": "stab", "results": [stab_microbench(args.micro_L)]}), flush=True)
        return
    if args.micro == "metro":
        for df in (False, True):
            out.append(metro_microbench(args.micro_L, 32, df))
            out.append(metro_microbench(args.micro_L, 64, df))
        print(json.dumps({"micro": "metro", "results": out}), flush=True)
        return
    if args.micro == "gemm":
        for mode in args.micro_prec.split(","):
            out.append(gemm_microbench(args.micro_n, mode))
        print(json.dumps({"micro": "gemm", "results": out}), flush=True)
        return
    for prec in args.micro_prec.split(","):
        r = prop_microbench(args.micro_L, prec, args.micro_stack)
        r["frac_of_hbm"] = round(r["GB_s"] / peaks["hbm_gbs"], 3)
        r["hbm_peak_source"] = src
        out.append(r)
    print(json.dumps({"micro": "prop", "results": out}), flush=True)


def soft(fn):
    """Run an optional leg of the bench; an exception becomes {"error": ...} in
    the JSON line instead of losing the line (the timed value stands alone).
    A leg that returns a dict is passed through; anything else is wrapped."""
    try:
        out = fn()
    except Exception as exc:
        return {"error": f"{type(exc).__name__}: {exc}"}
    return out if isinstance(out, dict) else {"value": out}


def replica(w, rank):
    """Replicas: every rank runs its own chain, seed + rank and chain id rank
    (independent Philox streams), no collective on the data path."""
    return {"seed": w["seed"] + rank, "chain": rank}


def max_over_ranks(x, dist, device):
    """The slowest rank's time (the whole-job time of weakly scaled replicas)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args, rank, world, local_rank):
    import ctypes as C

    import numpy as np
    import torch

    import paper_2608_03894_gb300 as pkg
    from paper_2608_03894_gb300 import _lib

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    w = workload(args)
    L, N = w["L"], 3 * w["L"] ** 2
    M = int(round(w["beta"] / w["dtau"]))
    units_per_step = 2 * N * M
    rp = replica(w, rank)
    d = pkg.DQMC(w["L"], w["beta"], w["dtau"], w["U"], w["mu"], seed=rp["seed"], k=w["k"],
                 n_stab=w["n_stab"], precision=w["precision"], chain=rp["chain"])
    for key, val in parse_options(args.option).items():
        d.set_option(key, val)
    stream = torch.cuda.current_stream()
    d.sweep(args.warmup)
    launches0 = d.stats()["launches"]

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- timed region: K sweeps, device time on the library's stream
    sampler = ClockSampler(local_rank)
    barrier()
    torch.cuda.synchronize()
    with sampler:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        d.sweep(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = ev0.elapsed_time(ev1)
    st = d.stats()
    launches = st["launches"] - launches0
    ms = max_over_ranks(ms, dist, "cuda")
    value = units_per_step * args.steps * world / (ms / 1000.0)
    clocks = sampler.summary()

    # ---- end to end through the public API: field in from pinned host memory,
    # one sweep with measurements, field and observables back to the host
    def e2e_leg():
        lib = _lib.load()
        fin = torch.empty((M, N), dtype=torch.int8, pin_memory=True)
        fout = torch.empty((M, N), dtype=torch.int8, pin_memory=True)
        fin.numpy()[:] = d.field
        obs = _lib.Obs()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _lib.check(lib.dqmc_set_field(d.h, C.c_void_p(fin.data_ptr())))
            _lib.check(lib.dqmc_sweep(d.h, 1, 1))
            _lib.check(lib.dqmc_get_field(d.h, C.c_void_p(fout.data_ptr())))
            _lib.check(lib.dqmc_measure(d.h, C.byref(obs)))
            fin.copy_(fout)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        te = max_over_ranks(te, dist, "cuda")
        return {"value": units_per_step * args.steps * world / te, "unit": UNIT,
                "h2d_bytes_per_step": M * N, "d2h_bytes_per_step": M * N + 6 * 8 * (-(-M // w["n_stab"]))}

    e2e = None if args.no_e2e else soft(e2e_leg)

    # ---- one extra sweep with per-kernel-family CUDA events for the roofline
    def roofline_leg():
        d.set_option("timing", 2)
        s0 = d.stats()
        d.sweep(1)
        s1 = d.stats()
        d.set_option("timing", 0)
        fam = {}
        for f in s1["ms_kernel"]:
            dt = s1["ms_kernel"][f] - s0["ms_kernel"][f]
            n = s1["n_kernel"][f] - s0["n_kernel"][f]
            fam[f] = {"ms": dt, "launches": n, "flops": s1["flops_kernel"][f] - s0["flops_kernel"][f],
                      "bytes": s1["bytes_kernel"][f] - s0["bytes_kernel"][f]}
        total_ms = sum(v["ms"] for v in fam.values())
        # the flush's work is counted at m = k flips per block on the host; the
        # true rank is the number of accepted flips: rescale to the accepted count
        acc = s1["accepted"] - s0["accepted"]
        prop_n = s1["proposed"] - s0["proposed"]
        if fam["flush"]["flops"] > 0 and prop_n > 0:
            fam["flush"]["flops"] *= acc / float(prop_n)
        # dominant kernel family on the critical path ("other" is many small kernels;
        # the look-ahead Metropolis overlaps the flush)
        dom = max(("prop", "flush", "gemm", "qr_panel"), key=lambda f: fam[f]["ms"])
        peaks, peak_src = load_peaks()
        mhz_max = peaks.get("sm_max_mhz", 2070.0)
        fd = fam[dom]
        per_launch_s = fd["ms"] / 1000.0 / max(1, fd["launches"])
        mixed = w["precision"] == "mixed"
        if dom == "prop":
            achieved = fd["bytes"] / max(1, fd["launches"]) / per_launch_s / 1e9
            roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "peak_source": f"{peak_src} copy bandwidth"}
        elif dom == "gemm" and mixed:
            # digit slices: 45 bf16 products per FP64-equivalent multiply-add
            achieved = 45.0 * fd["flops"] / max(1, fd["launches"]) / per_launch_s / 1e12
            roof = {"bound": "tensor", "achieved": achieved, "peak": peaks.get("bf16_tflops_sustained", 1700.0),
                    "unit": "TFLOP/s", "peak_source": f"{peak_src} sustained bf16 (cuBLAS); bf16 MMA rate of the "
                                                       "digit-slice GEMM = 45 x its FP64-equivalent rate"}
        elif dom == "flush" and mixed and w["k"] == 32:
            # the tensor-core flush streams G once (read and write): HBM roofline on 2 N^2 8 bytes
            achieved = fd["bytes"] / max(1, fd["launches"]) / per_launch_s / 1e9
            roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "peak_source": f"{peak_src} copy bandwidth; G (N^2 FP64) read and written once per flush"}
        elif dom == "flush" and mixed:
            # double-float MAC = 12 FP32 instructions: peak FP64-equivalent rate = FP32 FMA issue rate / 12 x 2
            achieved = fd["flops"] / max(1, fd["launches"]) / per_launch_s / 1e12
            peak = alu_peak_tflops("fp32", mhz_max) / 12.0
            roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "peak_source": f"FP64-equivalent double-float rate: 152 SMs x 128 FP32 lanes x {mhz_max:.0f} MHz "
                                   "/ 12 instructions per multiply-add x 2"}
        else:
            achieved = fd["flops"] / max(1, fd["launches"]) / per_launch_s / 1e12
            peak = alu_peak_tflops("fp64", mhz_max)
            roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "peak_source": f"fp64 issue rate x 152 SMs x {mhz_max:.0f} MHz"}
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof["kernel"] = dom
        roof["traffic"] = None
        roof["share_of_device_time"] = fd["ms"] / max(total_ms, 1e-9)
        return fam, roof

    fam, roof = {}, None
    r = soft(roofline_leg)
    if "error" in r:
        roof = r
    else:
        fam, roof = r["value"]

    # FFT propagation alone on a stacked operand larger than L2 (HBM roofline of
    # the propagation kernels, FP32 / double-float / FP64 arithmetic)
    fft = None
    if rank == 0:
        hbm = load_peaks()[0]["hbm_gbs"]

        def fft_leg(prec):
            r = prop_microbench(L, prec, max(1, (800 << 20) // (N * N * 4)))
            r["frac_of_hbm"] = round(r["GB_s"] / hbm, 3)
            return r

        fft = [soft(lambda p=prec: fft_leg(p)) for prec in ("fp32", "df", "fp64")]

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = soft(lambda: cpu_oracle_sample(w, budget_s=args.cpu_budget))

    # ---- the metric's comparison: the plain FP64 GPU path (and plain FP32 as
    # context) on the same workload, delay rank and refresh interval, timed the
    # same way; the mixed arm's chain is released first
    d_stats = st
    d.close()
    arms = {}
    if rank == 0 and w["precision"] == "mixed" and args.compare_steps > 0:
        for prec in ("fp64", "fp32"):
            arms[prec] = soft(lambda p=prec: comparator_arm(w, p, rp, args.compare_steps))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "mixed": "f64 (emulated on f32 pairs and bf16 digit slices) + f64",
                      "fp32": "f32 + f64 stab"}[w["precision"]],
            "data": "synthetic (Philox-initialised Ising field, seed 1 + rank)",
            "config": config_dict(w, world),
            "max_drift": d_stats["max_drift"],
            "acceptance": d_stats["accepted"] / max(1, d_stats["proposed"]),
            "sweeps_per_s": args.steps * world / (ms / 1000.0),
            "phase_breakdown_ms": {f: round(v["ms"], 3) for f, v in fam.items()},
            "launches_before_timed": int(launches0),
            "roofline": roof, "fft_roofline": fft, "cpu_baseline": cpu, "e2e": e2e,
            "fp64_arm": arms.get("fp64"), "fp32_arm": arms.get("fp32"),
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        fa = arms.get("fp64")
        if fa and "value" in fa and "error" not in fa:
            line["fp64_value"] = fa["value"]
            line["fp64_max_drift"] = fa["max_drift"]
            line["speedup_vs_fp64"] = value / fa["value"]
            line["mixed_drift_within_bar"] = bool(d_stats["max_drift"] <= 1e-6)
        print(json.dumps(line), flush=True)


def comparator_arm(w, prec, rp, steps):
    """One more chain of the same workload (same seed, k, n_stab) in another
    precision: one untimed warm-up sweep, then `steps` sweeps timed with CUDA
    events on the library's stream. Returns its site-updates/s and drift."""
    import torch

    import paper_2608_03894_gb300 as pkg
    L, N = w["L"], 3 * w["L"] ** 2
    M = int(round(w["beta"] / w["dtau"]))
    kw = {"drift_limit": 10.0} if prec == "fp32" else {}
    with pkg.DQMC(L, w["beta"], w["dtau"], w["U"], w["mu"], seed=rp["seed"], k=w["k"],
                  n_stab=w["n_stab"], precision=prec, chain=rp["chain"], **kw) as c:
        for key, val in parse_options(args_global.option).items():
            c.set_option(key, val)
        stream = torch.cuda.current_stream()
        c.sweep(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.sweep(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        s = c.stats()
    return {"precision": prec, "value": 2 * N * M * steps / (ms / 1000.0), "unit": UNIT,
            "steps": steps, "warmup": 1, "ms_per_step": ms / steps, "max_drift": s["max_drift"],
            "acceptance": s["accepted"] / max(1, s["proposed"]),
            "note": {"fp64": "plain FP64 GPU path, same k and n_stab: the metric's denominator",
                     "fp32": "plain FP32 propagation and flush (context: misses the |dG| <= 1e-6 bar)"}[prec]}


def main():
    global args_global
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default="L24_mixed", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=("fp64", "mixed", "fp32"))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--option", action="append", default=[],
                    help="library option key=value for the chain (repeatable), e.g. pipeline=0")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--compare-steps", type=int, default=2,
                    help="sweeps timed for the plain FP64 (and FP32) comparator arms of a mixed "
                         "run; 0 skips them")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--micro", default=None, choices=("prop", "gemm", "metro", "update", "stab", "batch"),
                    help="only a microbenchmark: the FFT propagation on a stacked operand larger "
                         "than L2 (prop; --micro-prec fp32,df,fp64), the stabilisation GEMM "
                         "(gemm; --micro-prec f64,df,oz,tc, size --micro-n), one delayed-update "
                         "block (metro; update: Metropolis + tensor-core flush, --micro-L), or a "
                         "short chain whose refreshes run the stabilisation kernels (stab, --micro-L), "
                         "or the 64-chain batched workload with autotuned delay ranks and refresh "
                         "intervals (batch)")
    ap.add_argument("--micro-n", type=int, default=1728)
    ap.add_argument("--micro-L", type=int, default=24)
    ap.add_argument("--micro-stack", type=int, default=64)
    ap.add_argument("--micro-prec", default="fp32,df,fp64")
    args = ap.parse_args()
    args_global = args
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.micro:
        if rank == 0:
            run_micro(args)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


args_global = None

if __name__ == "__main__":
    main()
