#!/usr/bin/env python
"""Throughput of the DQMC sweep (honeycomb Hubbard model, L = 24, beta t = 24).

One step = one full sweep (forward + backward pass over all M slices: wraps,
delayed updates, QR recomputations of G, measurements) of one Markov chain.
The metric is proposed single-site HS-field flips per second: 2 N M per sweep.
The headline value is the L = 24 precision workload (delayed-update flush as
split-TF32 tensor-core products, everything else FP64); the plain FP64 sweep
on the same seed is timed after it and reported under "fp64".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 it runs under torch.distributed.run, one rank per GPU, one
independent chain per rank (weak scaling, no collective on the data path; the
only collectives are the timing barrier and the max over ranks).
--impl reference times the FP64 CPU oracle on the host cores (the reference arm).
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
sys.path.insert(0, ROOT)

from synth import WORKLOADS, random_field  # noqa: E402

METRIC = "HS-field updates/s per sweep at L=24, beta*t=24, vs plain FP64; % of TC peak"
UNIT = "updates/s"
WORKLOAD_KEY = "L24_beta24"
FP64_PEAK_TFLOPS = 1.25      # nominal B300 FP64 rate (SIMT and tensor); DFMA microbenchmark on this pool: 1.13


def _tf32_peak():
    """TF32 dense peak = measured BF16 burst rate (MEASURED_PEAKS.json: cuBLAS bf16
    GEMM timed alone, the way the roofline pass below times the slice kernel) x the
    nominal TF32/BF16 ratio 1.1/2.25.  Fallback: the recipe's 1.8 PFLOP/s burst."""
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return pk["bf16_tflops"] * 1.1 / 2.25, "measured", pk.get("sm_max_mhz")
    except Exception:
        return 1800.0 * 1.1 / 2.25, "fallback", None


TF32_PEAK_TFLOPS, TF32_PEAK_SOURCE, PEAK_SM_MHZ = _tf32_peak()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD_KEY, choices=sorted(WORKLOADS) + ["batched", "learned", "precision"],
                    help="batched: 64 chains, L in {6, 9, 12}, 16 twists each, one graph per batched sweep")
    ap.add_argument("--no-autotune", action="store_true", help="batched: skip the autotuner (n_delay 16, all SMs)")
    ap.add_argument("--twists", choices=["grid", "quasirandom"], default="grid",
                    help="batched: the uniform 4x4 twist grid, or the first 16 points of the library's "
                         "quasi-random (Halton 2,3) twist sequence")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tau-sweeps", type=int, default=15,
                    help="extra sweeps per chain (after the timed and e2e ones) for the autocorrelation time")
    ap.add_argument("--precision", type=int, default=3, choices=[0, 1, 2, 3, 6, 7],
                    help="bit 0: split-TF32 tensor-core flush (the L=24 precision workload); bit 1: stabilisation "
                         "products on the BF16 tensor cores with FP64 accuracy (Ozaki); bit 2 (with bit 1): blocked "
                         "solves of G with those products as couplings; 0: plain FP64")
    ap.add_argument("--no-fp64", action="store_true", help="skip timing the plain FP64 sweep")
    ap.add_argument("--update-ctas", type=int, default=0,
                    help="CTAs of the cooperative slice kernel per chain (0: one per SM)")
    ap.add_argument("--chains", type=int, default=3,
                    help="independent chains per GPU, each on its own CUDA stream and host thread "
                         "(3 saturates the L=24 workload: 2 -> 260k, 3 -> 289k, 4 -> 289k updates/s)")
    return ap.parse_args()


def workload_config(key):
    w = WORKLOADS[key]
    M = int(round(w["beta"] / w["dtau"]))
    N = 2 * w["L"] * w["L"]
    return w, N, M


# --------------------------------------------------------------------------- oracle timing
def oracle_sample(key, seed=11):
    """Time the FP64 CPU oracle on a bounded sample of the workload: one wrap, one
    slice update (N proposals) and one stabilisation (n_stab slice products,
    pivoted QR, stable inverse), at the workload's N, U, dtau, n_delay, n_stab.
    Returns (seconds per slice incl. wraps, seconds per stabilisation)."""
    from oracle.dqmc import Model, Chain
    from oracle.linalg import udt_left_multiply, stable_green
    w, N, M = workload_config(key)
    ns = w["n_stab"]
    m = Model(w["L"], U=w["U"], beta=2 * ns * w["dtau"], dtau=w["dtau"],
              hs_channel=w.get("hs_channel", 0))                            # same N and B_l, 2 n_stab slices
    f = random_field(m.M, m.N, seed)
    ch = Chain(m, n_delay=w["n_delay"], n_stab=ns, seed=seed, field=f)
    t0 = time.perf_counter()
    ch.G = m.wrap(ch.G, ch.field[0])
    ch.update_slice(1, 0)
    t1 = time.perf_counter()
    C = m.chain_product(ch.field, 1, ns)
    ch.Rstack[1] = udt_left_multiply(C, ch.Rstack[0])
    ch.G = stable_green(ch.Rstack[1], ch.Lstack[1])
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1, ch.accepted / max(ch.proposed, 1)


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [p["num_threads"] for p in threadpool_info() if p.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def sweep_rate_from_sample(key, t_slice, t_stab):
    w, N, M = workload_config(key)
    t_sweep = 2 * M * t_slice + 2 * (M // w["n_stab"]) * t_stab
    return 2 * N * M / t_sweep, t_sweep


def cpu_baseline(key):
    t_slice, t_stab, acc = oracle_sample(key)
    rate, t_sweep = sweep_rate_from_sample(key, t_slice, t_stab)
    w, N, M = workload_config(key)
    return {"value": rate, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
            "sample": (f"numpy FP64 oracle at N={N}: one wrap + one slice update ({N} proposals, "
                       f"acceptance {acc:.3f}) = {t_slice:.2f} s and one stabilisation (n_stab={w['n_stab']} "
                       f"dense slice products, pivoted QR, stable inverse) = {t_stab:.2f} s, extrapolated to the "
                       f"{2 * M} slices and {2 * (M // w['n_stab'])} stabilisations of one sweep "
                       f"({t_sweep:.0f} s/sweep); CPU: {cpu_model()}")}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if not reports(rank):
        return
    key = args.workload
    w, N, M = workload_config(key)
    for _ in range(args.warmup):
        oracle_sample(key)
    ts, tb = [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        a, b, acc = oracle_sample(key)
        ts.append(a)
        tb.append(b)
    wall = time.perf_counter() - t0
    per_slice = sum(ts) / len(ts) + (sum(tb) / len(tb)) / w["n_stab"]
    value = N / per_slice
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": key, "L": w["L"], "N_sites": N, "beta": w["beta"], "dtau": w["dtau"], "M": M,
                      "U": w["U"], "n_delay": w["n_delay"], "n_stab": w["n_stab"], "precision": 0,
                      "hs_channel": w.get("hs_channel", 0), "parallelism": "host cores (numpy/BLAS threads)"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                            "sample": (f"each step: one wrap + one slice update ({N} proposals) + one "
                                       f"stabilisation of the FP64 numpy oracle; value = N / (t_slice + "
                                       f"t_stab/n_stab), the oracle's amortised sweep rate; CPU: {cpu_model()}")},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                if int(parts[0]) != self.gpu_index:
                    continue
                rows.append(parts)
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        reasons = set()
        for r in rows:
            for name, col in (("hw_slowdown", 5), ("hw_thermal_slowdown", 6), ("sw_thermal_slowdown", 7),
                              ("sw_power_cap", 8)):
                if r[col].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "samples": len(rows), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------- roofline
def algorithmic_flops(family, N, Nc, accepted_per_update, cplx=False):
    """Algorithmic FP64 flops of one launch of each kernel family (all matrices N x N,
    N physical sites).  cplx: complex matrices (charge channel), counted as complex
    arithmetic (a complex multiply-add is 4 real ones); the device's real 2N x 2N
    embedding does twice that work, which shows as a lower fraction."""
    import math
    c = 4.0 if cplx else 1.0
    if family == "gemm":
        return c * 2.0 * N ** 3
    if family == "qr":
        return c * 4.0 * N ** 3 / 3.0                   # Householder QR, square
    if family == "lu":
        return c * 2.0 * N ** 3 / 3.0                   # LU with partial pivoting, square
    if family == "update":
        return c * 2.0 * N * N * accepted_per_update    # Eq. FinalDelay: 2 N^2 per accepted flip
    if family == "propagate":
        # real: N/2 complex row pairs; complex: N complex rows.  Each: 4 complex FFTs of
        # size Nc (5 n log2 n) + 2x2 block per k (32 flops)
        rows = N if cplx else N / 2.0
        return rows * (4 * 5.0 * Nc * math.log2(max(Nc, 2)) + 32.0 * Nc)
    return None


# --------------------------------------------------------------------------- ranks
def rank_chains(rank, chains):
    """Chains of one rank: whole independent chains per rank (weak scaling), so
    the data path has no collective.  Returns (seed, chain indices); the chain
    index selects the random stream, so every (rank, chain) pair is a distinct
    Markov chain."""
    return 1000 + rank, [rank * chains + c for c in range(chains)]


def combine_ranks(dist, ms, proposed, device):
    """Whole-job numbers: the slowest rank's time (max) and all ranks' proposals (sum)."""
    import torch
    if dist is None:
        return ms, float(proposed)
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([float(proposed)], dtype=torch.float64, device=device)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p.item())


def reports(rank):
    """Only rank 0 prints the JSON line (and runs the CPU reference arm)."""
    return rank == 0


def time_chain(pkg, torch, args, key, precision, rank, world, dev, dist, stream):
    """Create C chains (one CUDA stream and one host thread each), run W warm-up
    sweeps, time K sweeps of every chain with CUDA events on the chains' streams
    (per-launch timing enabled).  Returns a result dict (chain 0's observables)."""
    import threading
    w, N, M = workload_config(key)
    C = max(1, args.chains)
    streams = [stream] + [torch.cuda.Stream(device=dev) for _ in range(C - 1)]
    chains = []
    seed, idx = rank_chains(rank, C)
    for c in range(C):
        params = pkg.make_params(L=w["L"], beta=w["beta"], dtau=w["dtau"], U=w["U"], n_delay=w["n_delay"],
                                 n_stab=w["n_stab"], seed=seed, chain=idx[c], measure=1,
                                 device=dev, precision=precision, update_ctas=args.update_ctas,
                                 hs_channel=w.get("hs_channel", 0))
        chains.append(pkg.Chain(params, stream=streams[c].cuda_stream))
    ch = chains[0]

    def run_all(fn):
        if C == 1:
            fn(0)
            return
        ts = [threading.Thread(target=fn, args=(c,)) for c in range(C)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()

    run_all(lambda c: chains[c].sweep(args.warmup))
    for c in range(C):
        chains[c].observables()
    torch.cuda.synchronize(dev)

    def family_times():
        t = None
        for c in range(C):
            x = pkg.afqmc_get_timing(chains[c].h)
            t = x if t is None else {k: (t[k][0] + x[k][0], t[k][1] + x[k][1]) for k in x}
        return t

    # breakdown pass (outside the timed region): one sweep per chain with every
    # launch bracketed by events, to find the dominant kernel family
    for c in range(C):
        pkg.afqmc_set_timing(chains[c].h, True)
    run_all(lambda c: chains[c].sweep(1))
    breakdown = family_times()
    dominant = max((k for k in breakdown if breakdown[k][0] > 0), key=lambda k: breakdown[k][1])
    # timed region: events only around the dominant family's launches
    for c in range(C):
        pkg.afqmc_set_timing(chains[c].h, [dominant])

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    clocks = ClockSampler(dev)
    barrier()
    clocks.start()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(C)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(C)]
    for c in range(C):
        e0[c].record(streams[c])
    stats = [[0, 0, 0, 0.0] for _ in range(C)]

    def steps(c):
        for _ in range(args.steps):
            st = chains[c].sweep(1)
            stats[c][0] += st.proposed
            stats[c][1] += st.accepted
            stats[c][2] += st.launches
            stats[c][3] = max(stats[c][3], st.max_stab_drift)
        e1[c].record(streams[c])

    run_all(steps)
    barrier()
    ck = clocks.stop()
    ms = max(e0[0].elapsed_time(e1[c]) for c in range(C))
    proposed = sum(x[0] for x in stats)
    accepted = sum(x[1] for x in stats)
    launches = sum(x[2] for x in stats)
    drift = max(x[3] for x in stats)
    timing = family_times()
    for c in range(C):
        pkg.afqmc_set_timing(chains[c].h, 0)
    obs = ch.observables()
    for c in range(1, C):
        chains[c].observables()
    ms_max, total_proposed = combine_ranks(dist, ms, proposed, dev)
    return dict(chain=ch, chains=chains, run_all=run_all, ms=ms_max, value=total_proposed / (ms_max / 1e3), proposed=proposed,
                total_proposed=total_proposed, accepted=accepted, launches=launches, drift=drift,
                timing=timing, breakdown=breakdown, dominant=dominant, obs=obs, clocks=ck, barrier=barrier)


# DRAM bytes per launch of a kernel family from one ncu capture, valid only while
# the kernel's source files still hash as they did when the counters were taken
# (an ncu capture of the slice kernel at the L=24 workload's N and n_delay; the
# hash covers update.cuh and common.cuh, which it includes).  Fill in after a
# capture: sha256 of the two files' bytes, concatenated in this order.
TRAFFIC_SOURCES = ("paper_2609_14668_b300/csrc/update.cuh", "paper_2609_14668_b300/csrc/common.cuh")
CAPTURED_TRAFFIC = {
    ("update", 1, 1152): (TRAFFIC_SOURCES, "8c8a82715706c07bc5e7610d3651fa10846a7538020d284b78d6150b29144905", 10.748160e6 + 0.355584e6),
    ("update", 3, 1152): (TRAFFIC_SOURCES, "8c8a82715706c07bc5e7610d3651fa10846a7538020d284b78d6150b29144905", 10.748160e6 + 0.355584e6),
}


def sources_sha256(paths):
    import hashlib
    h = hashlib.sha256()
    for path in paths:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), path), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def captured_traffic(fam, precision, N):
    ent = CAPTURED_TRAFFIC.get((fam, precision, N))
    if ent is None:
        return None
    paths, sha, nbytes = ent
    try:
        if sources_sha256(paths) != sha:
            return None
    except OSError:
        return None
    return nbytes


def isolated_family_time(pkg, torch, chain, fam, dev):
    """(launches, ms) of one kernel family over one sweep of a single chain with
    nothing else running on the GPU: per-launch CUDA events on the chain's stream
    then bracket the kernel alone, so their average is a kernel duration (with
    several chains in flight the events of one stream also count the time other
    chains' kernels hold the SMs)."""
    torch.cuda.synchronize(dev)
    pkg.afqmc_set_timing(chain.h, [fam])
    chain.sweep(1)
    t = pkg.afqmc_get_timing(chain.h)
    pkg.afqmc_set_timing(chain.h, 0)
    chain.observables()
    return t[fam]


def roofline_of(res, N, precision, cplx=False):
    """Roofline of the dominant kernel family: its algorithmic work per launch over
    its average launch duration, from the isolated single-chain pass."""
    breakdown, fam, accepted = res["breakdown"], res["dominant"], res["accepted"]
    Nc = N // 2
    nl, tms = res["isolated"]
    acc_per_update = accepted / max(res["timing"]["update"][0], 1)
    clocks = res.get("iso_clocks") or {}
    if fam == "update" and (precision & 1):
        # flush on the tensor cores: 2 N^2 algorithmic flops per accepted flip (x 4 for
        # complex G), each product done as three TF32 products (split-TF32), so the
        # peak is TF32 / 3
        fl = (4.0 if cplx else 1.0) * 2.0 * N * N * acc_per_update
        peak, bound, unit = TF32_PEAK_TFLOPS / 3.0, "tensor", "TFLOP/s"
        note = (f"split-TF32 peak = TF32 dense / 3; TF32 dense = {TF32_PEAK_SOURCE} BF16 burst rate "
                f"(the kernel is timed alone) x nominal TF32/BF16 ratio 1.1/2.25; peak measured at "
                f"up to {PEAK_SM_MHZ} MHz SM clock")
    else:
        fl = algorithmic_flops(fam, N, Nc, acc_per_update, cplx)
        peak, bound, unit = FP64_PEAK_TFLOPS, "alu", "TFLOP/s"
        note = "nominal B300 FP64 (DFMA microbenchmark on this pool: 1.13 TFLOP/s)"
    if fl is None:
        return None
    ach = fl / (tms / nl / 1e3) / 1e12
    cnl, ctms = res["timing"][fam]
    return {"bound": bound, "kernel": fam, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
            "traffic": None if cplx else captured_traffic(fam, precision, N), "peak_note": note,
            "flops_per_launch": fl, "avg_launch_ms": tms / nl, "launches_timed": nl,
            "timing_note": ("CUDA events around each launch of the family during one extra sweep of one chain "
                            "with no other chain running (after the timed region); the concurrent figure is "
                            "the same events inside the timed region with every chain in flight"),
            "concurrent_avg_launch_ms": ctms / max(cnl, 1),
            "clocks_during_isolated_pass": clocks,
            "share_of_step": breakdown[fam][1] / sum(v[1] for v in breakdown.values()),
            "share_note": "share of device time in one breakdown sweep per chain with every launch timed"}


def run_ours(args):
    import torch
    import paper_2609_14668_b300 as pkg
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group(backend="nccl")
    dev = local if world > 1 else 0
    key = args.workload
    w, N, M = workload_config(key)
    cplx = w.get("hs_channel", 0) == 1
    stream = torch.cuda.Stream(device=dev)
    # headline: the reduced-precision workload (split-TF32 flush); then the plain FP64 sweep
    head = time_chain(pkg, torch, args, key, args.precision, rank, world, dev, dist, stream)
    ref64 = None
    if args.precision != 0 and not args.no_fp64:
        ref64 = time_chain(pkg, torch, args, key, 0, rank, world, dev, dist, stream)
        ref64["isolated"] = isolated_family_time(pkg, torch, ref64["chain"], ref64["dominant"], dev)
        for c in ref64["chains"]:
            c.close()
    ch = head["chain"]
    barrier = head["barrier"]
    # the dominant family's kernel duration, timed alone (for the roofline)
    iso_ck = ClockSampler(dev)
    iso_ck.start()
    head["isolated"] = isolated_family_time(pkg, torch, ch, head["dominant"], dev)
    head["iso_clocks"] = iso_ck.stop()

    series = [[] for _ in head["chains"]]   # per-sweep observables of each chain
    # e2e: the public call a user makes per step (one sweep) plus reading the step's
    # results back to host memory (observable averages and the field); state stays resident.
    e2e = None
    if not args.no_e2e:
        nb = [0] * len(head["chains"])

        def e2e_steps(c):
            chn = head["chains"][c]
            for _ in range(args.steps):
                chn.sweep(1)
                o = chn.observables()
                f = chn.field()
                nb[c] = 10 * 8 + o["Czz"].nbytes + o["nk"].nbytes + f.nbytes
                series[c].append(o)
        barrier()
        t0 = time.perf_counter()
        head["run_all"](e2e_steps)
        barrier()
        wall = time.perf_counter() - t0
        nbytes = sum(nb)
        wall_max, total = combine_ranks(dist, wall, head["proposed"], dev)
        e2e_val = total / wall_max
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": nbytes}

    # autocorrelation: per-sweep energy and m^2 of every chain (e2e sweeps + extra ones)
    if args.tau_sweeps > 0:
        def more(c):
            chn = head["chains"][c]
            for _ in range(args.tau_sweeps):
                chn.sweep(1)
                series[c].append(chn.observables())
        head["run_all"](more)
    autocorr = None
    if min(len(x) for x in series) >= 4:
        from paper_2609_14668_b300.autocorr import tau_int
        taus = {}
        for k in ("energy", "m2"):
            t, wdw, n = tau_int([[o[k] for o in x] for x in series])
            taus[k] = {"tau_int": t, "window": wdw}
        tmax = max(v["tau_int"] for v in taus.values())
        autocorr = {"tau_int_sweeps": taus, "sweeps_per_chain": min(len(x) for x in series),
                    "chains": len(series), "value_per_2tau": head["value"] / (2.0 * tmax),
                    "definition": "tau_int = 1/2 + sum rho(t) over Sokal's window (c = 6), per-sweep averages, "
                                  "chains pooled; corrected rate = value / (2 max tau_int)",
                    "note": (f"chains start from a random field {args.warmup + 1 + args.steps} sweeps "
                             "before the series; at L=24 that is short of equilibrium, so the relaxation "
                             "inflates tau_int")}

    out = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": head["ms"] / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": {0: "f64", 1: "f64 (flush: tf32x3, f32 accumulate)",
                     2: "f64 (stabilisation products: bf16 Ozaki, FP64-accurate)",
                     3: "f64 (flush: tf32x3, f32 accumulate; stabilisation products: bf16 Ozaki, FP64-accurate)",
                     6: "f64 (stabilisation products and blocked solves of G: bf16 Ozaki, FP64-accurate)",
                     7: "f64 (flush: tf32x3, f32 accumulate; stabilisation products and blocked solves of G: "
                        "bf16 Ozaki, FP64-accurate)"}
                    [args.precision],
           "data": "synthetic (random initial Ising field from the seed; no dataset)",
           "config": {"workload": key, "L": w["L"], "N_sites": N, "beta": w["beta"], "dtau": w["dtau"], "M": M,
                      "U": w["U"], "n_delay": w["n_delay"], "n_stab": w["n_stab"], "precision": args.precision,
                      "hs_channel": w.get("hs_channel", 0),
                      "chains_per_gpu": max(1, args.chains), "update_ctas": args.update_ctas or "one per SM",
                      "parallelism": f"replicas{world}",
                      "l2": "no flush: a sweep streams the UDT stacks (1.3 GB) through the 126 MB L2"},
           "roofline": roofline_of(head, N, args.precision, cplx),
           "gpu_launches": int(head["launches"]),
           "acceptance": head["accepted"] / max(head["proposed"], 1), "max_stab_drift": head["drift"],
           "kernel_ms_breakdown_sweep": {k: {"launches": v[0], "ms": v[1]} for k, v in head["breakdown"].items()},
           "observables": {k: head["obs"][k] for k in ("energy", "double_occ", "S_af", "m2", "chi_e", "n_samples")}}
    if ref64 is not None:
        diff = {k: head["obs"][k] - ref64["obs"][k] for k in ("energy", "double_occ", "S_af")}
        diff["note"] = ("same seeds and random numbers, averages over the timed sweeps: the chains part after a "
                        "few sweeps, so this is sweep-to-sweep noise, not the bias of the reduced precision; "
                        "the bias, (TF32 - FP64) +- sigma over independent equilibrated chains, is what "
                        "bench.py --workload precision measures")
        out["fp64"] = {"value": ref64["value"], "ms_per_step": ref64["ms"] / args.steps,
                       "speedup": head["value"] / ref64["value"],
                       "obs_diff_vs_fp64_same_seeds": diff,
                       "kernel_ms_breakdown_sweep": {k: {"launches": v[0], "ms": v[1]}
                                                     for k, v in ref64["breakdown"].items()},
                       "roofline": roofline_of(ref64, N, 0, cplx)}
    if e2e:
        out["e2e"] = e2e
    if autocorr:
        out["autocorr"] = autocorr
    if head["clocks"]:
        out["clocks"] = head["clocks"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(key)
    for c in head["chains"]:
        c.close()
    if reports(rank):
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def run_batched(args):
    """The batched twist-averaging workload: 64 independent chains of three sizes
    and 16 twists each, one CUDA graph launch per batched sweep.  The delay
    rank and the slice kernel's grid are chosen per size by the library's
    autotuner (throughput of the size's chains swept together)."""
    import torch
    import paper_2609_14668_b300 as pkg
    from synth import BATCHED, batched_chains
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")
    twist_list = pkg.afqmc_quasirandom_twists(BATCHED["twists"] ** 2, 1) if args.twists == "quasirandom" else None
    spec = batched_chains(twist_list)

    def params(i, L, beta, th, nd, ct):
        return pkg.make_params(L=L, beta=beta, dtau=BATCHED["dtau"], U=BATCHED["U"], n_delay=nd,
                               n_stab=BATCHED["n_stab"], seed=500 + rank, chain=rank * len(spec) + i,
                               measure=1, device=dev, theta=th, update_ctas=ct)

    tuned = {}
    t_tune = time.perf_counter()
    for L, _ in BATCHED["sizes"]:
        # tune on 8 of the size's chains (8 different twists) swept together
        group = [params(i, *c[:3], 16, 0) for i, c in enumerate(spec) if c[0] == L][::2][:8]
        if args.no_autotune:
            tuned[L] = (16, 16, None)
        else:
            tuned[L] = pkg.afqmc_batch_autotune(group, [8, 16, 32], [4, 8, 16, 32], n_timed=1)
    t_tune = time.perf_counter() - t_tune
    plist = [params(i, L, beta, th, tuned[L][0], tuned[L][1]) for i, (L, beta, th, _) in enumerate(spec)]
    batch = pkg.Batch(plist)
    batch.sweep(args.warmup)
    for c in batch.chains:
        c.observables()
    clocks = ClockSampler(dev)
    torch.cuda.synchronize(dev)
    clocks.start()
    t0 = time.perf_counter()
    st = batch.sweep(args.steps)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    ck = clocks.stop()
    wall, total = combine_ranks(dist, wall, st.proposed, dev)
    value = total / wall
    # the same chains swept one after another with the plain per-chain call
    singles = [pkg.Chain(p) for p in plist]
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    seq = 0
    for c in singles:
        seq += c.sweep(1).proposed
    torch.cuda.synchronize(dev)
    seq_rate = seq / (time.perf_counter() - t1)
    for c in singles:
        c.close()
    # twist-averaged observables per size (the chains' sweep averages)
    avg = {}
    for L, _ in BATCHED["sizes"]:
        obs = [batch.chains[i].observables() for i, c in enumerate(spec) if c[0] == L]
        avg[f"L{L}"] = {k: statistics.fmean([o[k] for o in obs]) for k in ("energy", "double_occ", "S_af")}
    batch.close()
    if dist is not None:
        dist.destroy_process_group()
    if not reports(rank):
        return
    out = {"metric": "HS-field updates/s, batched twist-averaging chains (64 chains, L in {6,9,12}, 16 twists)",
           "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": wall * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (random initial Ising fields; no dataset)",
           "config": {"workload": "batched", "chains": len(spec), "sizes": [list(x) for x in BATCHED["sizes"]],
                      "twist_grid": (f"{BATCHED['twists']}x{BATCHED['twists']}" if args.twists == "grid" else
                                     f"quasi-random: Halton (2, 3) points 1..{BATCHED['twists'] ** 2}"),
                      "dtau": BATCHED["dtau"],
                      "U": BATCHED["U"], "n_stab": BATCHED["n_stab"], "beta": "t*beta = L",
                      "l2": "no flush: 64 chains' stacks (~0.9 GB) exceed the 126 MB L2",
                      "timing": "host wall clock around the batched sweeps, synchronised on both sides "
                                "(the graph runs on the library's own stream)"},
           "autotuned": {f"L{L}": {"n_delay": v[0], "update_ctas": v[1], "rate": v[2]} for L, v in tuned.items()},
           "autotune_s": t_tune, "gpu_launches": int(st.launches), "graph_launches": args.steps,
           "acceptance": st.accepted / max(st.proposed, 1), "max_stab_drift": st.max_stab_drift,
           "sequential_plain_sweeps": {"value": seq_rate, "speedup_of_batch": value / seq_rate},
           "observables_twist_avg": avg}
    if ck:
        out["clocks"] = ck
    print(json.dumps(out))


def run_learned(args):
    """Learned block proposals at L = 6, beta t = 6: train the network on the GPU
    on configurations of the plain sampler, then compare a chain of plain sweeps
    with a chain that adds one block pass per sweep, by wall time per sweep and
    by the integrated autocorrelation time of the per-sweep m^2 and energy."""
    import torch
    import paper_2609_14668_b300 as pkg
    from paper_2609_14668_b300.autocorr import tau_int
    import numpy as np
    from synth import LEARNED as C
    torch.cuda.set_device(0)
    mk = lambda seed: pkg.make_params(L=C["L"], beta=C["beta"], dtau=C["dtau"], U=C["U"], n_delay=C["n_delay"],
                                      n_stab=C["n_stab"], seed=seed, measure=1)
    sweeps = max(args.steps, 50)
    # training data: one configuration per sweep of a plain chain
    t0 = time.perf_counter()
    src = pkg.Chain(mk(31))
    src.sweep(max(args.warmup, 50))
    cfgs = []
    for _ in range(C["n_cfg"]):
        src.sweep(1)
        cfgs.append(src.field())
    src.close()
    cfgs = np.stack(cfgs)
    t_data = time.perf_counter() - t0
    net = pkg.Net(C["b"], C["T"], C["h"], C["ht"], C["hidden"], seed=1)
    loss0 = pkg.afqmc_net_train(net.net, cfgs, C["L"], C["L"], 1, C["batch"], lr=0.0, seed=1)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss = pkg.afqmc_net_train(net.net, cfgs, C["L"], C["L"], C["train_steps"], C["batch"], lr=C["lr"], seed=2)
    t_train = time.perf_counter() - t1
    untrained = pkg.Net(C["b"], C["T"], C["h"], C["ht"], C["hidden"], seed=1)

    def run(chain_seed, netp):
        ch = pkg.Chain(mk(chain_seed))
        ch.sweep(max(args.warmup, 20))
        ch.observables()
        series, acc, prop, flips = [], 0, 0, 0
        torch.cuda.synchronize()
        ts = time.perf_counter()
        for _ in range(sweeps):
            st = ch.sweep(1)
            if netp is not None:
                b = pkg.afqmc_block_sweep(ch.h, netp.net)
                acc, prop, flips = acc + b.accepted, prop + b.proposed, flips + b.flipped
            series.append(ch.observables())
        torch.cuda.synchronize()
        wall = time.perf_counter() - ts
        n_local = sweeps * 2 * ch.N * ch.M
        ch.close()
        taus = {k: tau_int([[o[k] for o in series]])[0] for k in ("m2", "energy")}
        rate = n_local / wall
        return {"updates_per_s": rate, "s_per_sweep": wall / sweeps, "tau_int_sweeps": taus,
                "per_2tau": rate / (2.0 * max(taus.values())),
                "block_acceptance": (acc / prop) if prop else None, "block_flips_per_sweep": flips / sweeps,
                "m2": float(np.mean([o["m2"] for o in series]))}

    plain = run(41, None)
    learned = run(41, net)
    base = run(41, untrained)
    out = {"metric": "autocorrelation-corrected HS-field updates/s with learned block proposals (L=6, beta*t=6)",
           "value": learned["per_2tau"], "unit": "updates/s per 2 tau_int", "n_gpus": 1, "steps": sweeps,
           "warmup": max(args.warmup, 20), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64 chain, f32 network", "data": "synthetic (training fields from the plain sampler)",
           "config": {"workload": "learned", **{k: C[k] for k in C}},
           "training": {"configurations_s": t_data, "train_s": t_train, "loss_initial": loss0, "loss_final": loss},
           "plain": plain, "learned": learned, "untrained_network": base,
           "gain_vs_plain": learned["per_2tau"] / plain["per_2tau"],
           "note": "updates/s counts the local proposals only; tau_int from per-sweep averages of one chain each "
                   "(Sokal window), a rough estimate at this length"}
    print(json.dumps(out))


def precision_comparison(pkg, cfg, seed0, sizes=("energy", "double_occ", "S_af", "m2")):
    """Equilibrium averages of the split-TF32 flush (precision 3) and plain FP64
    (precision 0) from independent chains, all swept together in one batch:
    per observable, each precision's mean of chain means and its standard error
    (chains are independent, so the spread of the chain means carries the
    autocorrelation), the difference and its z-score."""
    import numpy as np
    C = cfg["chains"]
    plist = []
    for prec in (3, 0):
        for c in range(C):
            plist.append(pkg.make_params(L=cfg["L"], beta=cfg["beta"], dtau=cfg["dtau"], U=cfg["U"],
                                         n_delay=cfg["n_delay"], n_stab=cfg["n_stab"], seed=seed0 + prec,
                                         chain=c, measure=1, precision=prec))
    batch = pkg.Batch(plist)
    batch.sweep(cfg["warm"])
    for c in batch.chains:
        c.observables()
    series = np.zeros((2 * C, cfg["meas"], len(sizes)))
    drift = 0.0
    for s in range(cfg["meas"]):
        st = batch.sweep(1)
        drift = max(drift, st.max_stab_drift)
        for i, c in enumerate(batch.chains):
            o = c.observables()
            series[i, s] = [o[k] for k in sizes]
    batch.close()
    out = {}
    for j, k in enumerate(sizes):
        cm = series[:, :, j].mean(axis=1)
        a, b = cm[:C], cm[C:]
        ma, mb = a.mean(), b.mean()
        sa, sb = a.std(ddof=1) / np.sqrt(C), b.std(ddof=1) / np.sqrt(C)
        d, sd = ma - mb, float(np.hypot(sa, sb))
        out[k] = {"tf32": [ma, sa], "fp64": [mb, sb], "diff": d, "sigma": sd, "z": d / sd if sd > 0 else 0.0,
                  "rel_diff": d / abs(mb) if mb else None}
    return out, drift


def run_precision(args):
    """The split-TF32 flush against the FP64 flush.  (1) Drift of the wrapped G
    from its QR recomputation after n_stab slices, n_stab in 1, 2, 4, 8, for
    both precisions at L = 12 and L = 24 (one chain each, after a warm-up
    sweep).  (2) Equilibrium e, D, S_AF, m^2 of independent chains of both
    precisions at L = 12 (and at L = 24 unless --steps 0), as (TF32 - FP64) +- sigma."""
    import torch
    import paper_2609_14668_b300 as pkg
    from synth import PRECISION_STUDY as P
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    drift = {}
    for key in ("L12", "L24"):
        cfg = P[key]
        drift[key] = {}
        for prec in (3, 0):
            row = {}
            for ns in P["DRIFT_NS"]:
                ch = pkg.Chain(pkg.make_params(L=cfg["L"], beta=cfg["beta"], dtau=cfg["dtau"], U=cfg["U"],
                                               n_delay=cfg["n_delay"], n_stab=ns, seed=77, precision=prec))
                ch.sweep(1)
                row[ns] = ch.sweep(1).max_stab_drift
                ch.close()
            drift[key][{3: "tf32", 0: "fp64"}[prec]] = row
    t_drift = time.perf_counter() - t0
    clocks = ClockSampler(0)
    clocks.start()
    t1 = time.perf_counter()
    comp = {"L12": precision_comparison(pkg, P["L12"], 1200)}
    if args.steps > 0:
        comp["L24"] = precision_comparison(pkg, P["L24"], 2400)
    t_comp = time.perf_counter() - t1
    ck = clocks.stop()
    out = {"metric": "split-TF32 flush vs FP64: drift and equilibrium observables (difference +- sigma)",
           "value": max(abs(v["z"]) for c in comp.values() for v in c[0].values()), "unit": "max |z|",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
           "dtype": "f64 vs f64 with tf32x3 flush", "data": "synthetic (random initial fields)",
           "config": {"workload": "precision", "study": {k: v for k, v in P.items()}},
           "drift_max_abs_vs_n_stab": drift, "drift_s": t_drift,
           "comparison": {k: {"observables": v[0], "max_stab_drift": v[1]} for k, v in comp.items()},
           "comparison_s": t_comp}
    if ck:
        out["clocks"] = ck
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "precision":
        run_precision(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
