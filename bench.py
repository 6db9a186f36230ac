"""Throughput of the lattice kick-drift step on GB300.

Workload (one GPU): two scalar fields, V = phi^4/4 + (q/2) phi^2 chi^2 with
q = 100, 256^3 periodic lattice, kIR = 0.1, alpha = 1, self-consistent
expansion (f*/m_p = 0.5), Yoshida-4 composition of velocity Verlet (VV4),
dt = 0.005, vacuum-fluctuation initial conditions from seed 1
((omega*/f*)^2 = 1e-4).  Headline: fields and momenta stored in FP32 with FP64
reductions; the plain FP64 path is timed on the same workload beside it.

A step is one full dt of the integrator (three fused drift+kick passes over
the whole lattice); value = site-updates/s = sites x steps / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (oracle/, FP64, one thread) on a
bounded sample of the same workload.  Under torchrun (N > 1) every rank
advances its own independent lattice (replicas, different seeds): there is
no exchange between ranks on the data path.
"""
import argparse
import hashlib
import json
import os
import signal
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "site-updates/s, 2-field φ⁴ 256³: FP32-store vs FP64 plain, % of HBM roofline"
N_LAT, KIR, ALPHA, SEED = 256, 0.1, 1.0, 1
PARAMS = dict(dt=0.005, integrator=4, q=100.0, phi0=[1.0, 0.0], fluct_amp2=1e-4, expansion=1,
              fstar_over_mp=0.5)
WORKLOAD = ("lphi4+chi q=100, 256^3, kIR=0.1, alpha=1, VV4 dt=0.005, self-consistent expansion, "
            "vacuum fluctuations (omega*/f*)^2=1e-4 seed 1")
# bytes one DK pass must move: 2 fields x (field, momentum) x (read + write)
PASS_BYTES_PER_SITE = {"f32": 2 * 2 * 2 * 4, "f64": 2 * 2 * 2 * 8}
PASSES_PER_STEP = 3
# DRAM bytes (read + write) per DK pass from one ncu capture of the FP32 pass
# at 256^3 (one cooperative launch of the three VV4 passes of a step, divided
# by 3), valid only for the kernel source it was taken on.
NCU_TRAFFIC = {"f32": {"source_hash": "e0b8777e15c09017", "bytes_per_launch": 503365461}}
# FP64 instructions (DFMA, DADD, DMUL) and operations (FMA = 2) per site per pass
# of the FP64 plain kernel, from one ncu capture of the instruction counters of
# the FP64 pass at 256^3
NCU_FP64_OPS = {"source_hash": "e0b8777e15c09017", "instructions_per_site_pass": 34.109,
                "flops_per_site_pass": 49.144}


# Thread instructions per site of the doublet passes without expansion at the
# benchmark size (kd_pass_su2<float,0,32,8,false,256> for the SU(2) x U(1)
# doublet, kd_pass_su2<float,0,32,16,true,256> for the lphi4SU2U1 model; one
# leapfrog pass of 256^3 each) and their DRAM bytes per site (the same kernels
# built for any N, one pass of 128^3), from ncu captures, valid for the kernel
# source they were taken on.
NCU_SU2 = {"source_hash": "85bf812048b7f8dc", "thread_instructions_per_site": 1400.0,
           "dram_bytes_per_site": 268.8}
NCU_FULL = {"source_hash": "85bf812048b7f8dc", "thread_instructions_per_site": 1616.3,
            "dram_bytes_per_site": 318.0}
# The same for the U(1) pass without expansion at the benchmark size
# (dk_pass_u1<float,0,true,256>, one leapfrog pass of 256^3).
NCU_U1 = {"source_hash": "68ec87c02aca2e4a", "thread_instructions_per_site": 255.8,
          "dram_bytes_per_site": 80.4}
# instruction issue of the whole GPU: 152 SMs x 4 schedulers x 32 lanes at the 2070 MHz maximum SM clock
ISSUE_PEAK_LANE_INSTR_PER_S = 152 * 4 * 32 * 2.070e9


def u1_source_hash():
    h = hashlib.sha256()
    for name in ("pass_u1.cu", "ring.cuh", "kd_drift.cuh", "trig2.cuh", "common.cuh", "tail.cuh"):
        with open(os.path.join(ROOT, "paper_2102_01031_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def su2_source_hash():
    h = hashlib.sha256()
    for name in ("pass_su2_kd.cu", "su2_common.cuh", "kd_drift.cuh", "trig2.cuh", "common.cuh", "tail.cuh"):
        with open(os.path.join(ROOT, "paper_2102_01031_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the scalar pass kernel, its headers and the work split (what
    decides the pass's DRAM traffic and FP64 operation count)."""
    h = hashlib.sha256()
    for name in ("pass_scalar.cu", "common.cuh", "tail.cuh", "worklist.h"):
        with open(os.path.join(ROOT, "paper_2102_01031_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_fp64_ops():
    """(FP64 instructions, FP64 operations) per site-pass of the FP64 plain kernel
    from the last ncu capture, or (None, None) if the kernel source changed since."""
    if NCU_FP64_OPS["source_hash"] != kernel_source_hash():
        return None, None
    return NCU_FP64_OPS["instructions_per_site_pass"], NCU_FP64_OPS["flops_per_site_pass"]


def ncu_traffic(prec):
    """DRAM bytes per launch of the DK pass from the last ncu capture, or None
    if the kernel source changed since the capture."""
    e = NCU_TRAFFIC.get(prec)
    if not e or e["source_hash"] != kernel_source_hash():
        return None
    return float(e["bytes_per_launch"])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms in the
    background; summary() keeps the samples taken inside a window of host
    times (the timed region), so a sampler started before the warm-up does
    not count the set-up."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.rows = []

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def stop(self):
        if self.proc is not None:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 10:
                        try:
                            t = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                            t += float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                        except (ValueError, IndexError):
                            continue
                        self.rows.append([t] + parts[1:])
            os.unlink(self.path)
        except OSError:
            pass
        return self

    def summary(self, t0=None, t1=None):
        rows = [r for r in self.rows if (t0 is None or r[0] >= t0) and (t1 is None or r[0] <= t1)]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        pw = [float(r[4]) for r in rows if r[4].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
                "power_w_max": max(pw) if pw else None}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device="cuda"):
    """The largest x over the ranks of the process group (x itself for one rank):
    the whole job takes as long as its slowest replica."""
    if ws <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_rate(ws, units_per_rank, seconds):
    """Whole-job throughput of ws replicas that each processed units_per_rank units,
    over the slowest replica's time."""
    return ws * units_per_rank / seconds


def cpu_oracle_rate(budget_s, steps_hint=None):
    """The oracle, as it stands, on a bounded sample of the workload: the same
    model and lattice spacing on a smaller periodic box; site-updates/s."""
    import oracle as O
    sizes = [16, 24, 32, 48, 64, 96, 128]
    rate_guess = 1.0e6
    if steps_hint is None:
        n_ref = 128
        steps = max(1, int(budget_s * rate_guess / n_ref ** 3))
    else:
        steps = steps_hint
        n_ref = max([s for s in sizes if s ** 3 * steps <= budget_s * rate_guess] or [16])
    kir = KIR * N_LAT / n_ref   # same dx as the 256^3 workload
    p = O.make_params(**PARAMS)
    L = O.Oracle(O.MODEL_LPHI4_CHI, n_ref, kir, ALPHA, SEED, p)
    return L, n_ref, steps


def _oracle_replica(job):
    """One replica of the all-core baseline (a spawned process): the oracle as
    it stands, one VV4 lattice of n_ref^3 sites with the workload's spacing,
    seed `seed`, timed over `steps` steps after one warm-up step."""
    n_ref, steps, seed = job
    import oracle as O
    L = O.Oracle(O.MODEL_LPHI4_CHI, n_ref, KIR * N_LAT / n_ref, ALPHA, seed, O.make_params(**PARAMS))
    L.step(1)
    t0 = time.perf_counter()
    L.step(steps)
    return n_ref ** 3 * steps, time.perf_counter() - t0


def cpu_oracle_all_cores(n_ref=64, steps=12):
    """The oracle on every host core at once: one independent replica (its own
    seed) per core, in spawned processes (started with 'spawn', never forked
    from a process that holds a CUDA context).  Whole-host site-updates/s =
    all replicas' site-updates over the slowest replica's time."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_replica, [(n_ref, steps, SEED + i) for i in range(cores)])
    units = sum(u for u, _ in res)
    slowest = max(t for _, t in res)
    return {"value": units / slowest, "unit": "site-updates/s", "cores": cores, "kind": "oracle",
            "sample": "%d independent replicas (one per host core, spawned processes), each %d VV4 steps of "
                      "the same model on a %d^3 box with the 256^3 lattice spacing, oracle FP64; value = all "
                      "site-updates / the slowest replica's time" % (cores, steps, n_ref)}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O  # noqa: F401
    L, n_ref, _ = cpu_oracle_rate(args.ref_budget, steps_hint=args.steps + args.warmup)
    for _ in range(args.warmup):
        L.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        L.step(1)
    dt = time.perf_counter() - t0
    value = n_ref ** 3 * args.steps / dt
    sample = ("each step: one VV4 step of the same model on a %d^3 periodic box with the 256^3 "
              "lattice spacing (kIR=%.4g), oracle FP64 single thread" % (n_ref, KIR * N_LAT / n_ref))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "site-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded vacuum fluctuations)",
        "config": {"workload": WORKLOAD, "sample_lattice": n_ref},
        "cpu_baseline": {"value": value, "unit": "site-updates/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def time_device(P, torch, lat, steps, warmup, rank, ws, min_window_s=0.0):
    """K steps bracketed by barrier + synchronize, CUDA events on the lattice
    stream.  With min_window_s > 0 the same K-step region is then repeated,
    each repeat timed alike, until that much time has passed since the timed
    region began, so that a clock sampler running in the background sees the
    GPU under this load (the reported time is the first region's)."""
    stream = torch.cuda.current_stream()
    lat.step(warmup)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    lat.pass_timing(reset=True)
    lat.enable_pass_timing(True)
    n0 = lat.launches()
    torch.cuda.synchronize()
    t_start = time.time()
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    lat.enable_pass_timing(False)
    launches = lat.launches() - n0
    ms = e0.elapsed_time(e1)
    pass_ms, npass = lat.pass_timing(reset=True)
    repeats = []
    while time.time() - t_start < min_window_s:
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        repeats.append(e0.elapsed_time(e1))
    t_end = time.time()
    ms = max_over_ranks(ms, ws)
    return ms, launches, pass_ms / max(npass, 1), npass, (t_start, t_end, repeats)


def run_ours(args):
    import torch

    import paper_2102_01031_gb300 as P

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    P.build()
    stream = P.torch_stream()
    sites = N_LAT ** 3
    peak, peak_kind = peaks()

    def make(prec, seed):
        return P.Lattice(P.MODEL_LPHI4_CHI, N_LAT, KIR, ALPHA, seed,
                         P.make_params(precision=prec, stream=stream, **PARAMS))

    results = {}
    for prec, name in ((P.FP32, "f32"), (P.FP64, "f64")):
        lat = make(prec, SEED + rank)
        steps = args.steps if name == "f32" else max(1, min(args.steps, args.fp64_steps))
        sampler = ClockSampler(local if ws > 1 else 0)
        clocks = None
        if name == "f32":
            sampler.start()
            time.sleep(0.3)   # nvidia-smi's first sample
        ms, launches, pass_ms, npass, (t0, t1, repeats) = time_device(
            P, torch, lat, steps, args.warmup, rank, ws, min_window_s=1.0 if name == "f32" else 0.0)
        if name == "f32":
            clocks = sampler.stop().summary(t0 - 0.05, t1 + 0.05)
            clocks["window"] = ("the timed region and %d repeats of it (%.0f ms in all); repeat median "
                                "%.4f ms per step" % (len(repeats), (t1 - t0) * 1e3,
                                                      statistics.median(repeats) / steps if repeats else
                                                      ms / steps))
        e = lat.energies(allow_nonfinite=True)
        results[name] = dict(ms=ms, steps=steps, launches=launches, pass_ms=pass_ms, npass=npass,
                             clocks=clocks, rho=e["rho"], a=e["a"], nonfinite=e["nonfinite"])
        if name == "f32":
            # end to end through the C ABI: every step uploads its state from pinned
            # host memory, runs one step and reads the energies back.  Serial: one
            # context, upload -> step -> energies.  Pipelined: two contexts on two
            # streams take the steps in turn, so one step's upload (copy engine)
            # overlaps the other's passes (SMs); each step still moves its own bytes.
            nbytes = lat.state_bytes()
            host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
            lat.download(host.data_ptr(), nbytes)
            k2 = max(1, min(args.steps, args.e2e_steps))

            def e2e_serial(n):
                for _ in range(n):
                    lat.upload(host.data_ptr(), nbytes)
                    lat.step(1)
                    lat.energies(allow_nonfinite=True)

            s2 = torch.cuda.Stream()
            with torch.cuda.stream(s2):
                lat2 = P.Lattice(P.MODEL_LPHI4_CHI, N_LAT, KIR, ALPHA, SEED + rank,
                                 P.make_params(precision=P.FP32, stream=P.torch_stream(), **PARAMS))
            pair = (lat, lat2)

            def e2e_pipelined(n):
                pair[0].upload(host.data_ptr(), nbytes)
                pair[0].step(1)
                for k in range(n):
                    if k + 1 < n:
                        nxt = pair[(k + 1) % 2]
                        nxt.upload(host.data_ptr(), nbytes)
                        nxt.step(1)
                    pair[k % 2].energies(allow_nonfinite=True)

            def timed(fn):
                fn(2)
                torch.cuda.synchronize()
                if ws > 1:
                    torch.distributed.barrier()
                t0 = time.perf_counter()
                fn(k2)
                torch.cuda.synchronize()
                return max_over_ranks(time.perf_counter() - t0, ws)

            t_serial = timed(e2e_serial)
            t_pipe = timed(e2e_pipelined)
            lat2.close()
            del lat2
            results["e2e"] = dict(value=replica_rate(ws, sites * k2, t_pipe),
                                  serial=replica_rate(ws, sites * k2, t_serial),
                                  h2d=nbytes, d2h=ctypes_sizeof_energies(P), steps=k2)
        lat.close()
        del lat
        torch.cuda.synchronize()

    if rank != 0:
        if ws > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return 0

    f32, f64 = results["f32"], results["f64"]
    value = replica_rate(ws, sites * f32["steps"], f32["ms"] * 1e-3)
    v64 = replica_rate(ws, sites * f64["steps"], f64["ms"] * 1e-3)
    bpl = PASS_BYTES_PER_SITE["f32"] * sites
    achieved = bpl / (f32["pass_ms"] * 1e-3) / 1e9
    bpl64 = PASS_BYTES_PER_SITE["f64"] * sites
    achieved64 = bpl64 / (f64["pass_ms"] * 1e-3) / 1e9
    traffic = ncu_traffic("f32")
    # the FP64 plain pass is bound by the FP64 pipe: roof = the measured FMA
    # instruction rate (an FMA, an add and a multiply each take one issue slot)
    fp64_rate = P.measure_fp64_rate(stream)
    ins64, ops64 = ncu_fp64_ops()
    ins_rate = None if ins64 is None else ins64 * sites / (f64["pass_ms"] * 1e-3)
    others = other_workloads(P, torch, stream, peak) if not args.no_extra else None
    budget = float(args.cpu_budget)
    L, n_ref, csteps = cpu_oracle_rate(budget)
    t0 = time.perf_counter()
    L.step(csteps)
    cdt = time.perf_counter() - t0
    cpu_value = n_ref ** 3 * csteps / cdt
    try:
        cpu_all = cpu_oracle_all_cores() if not args.no_extra else None
    except Exception as e:  # noqa: BLE001
        cpu_all = {"error": str(e)[:300]}
    line = {
        "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": ws,
        "steps": f32["steps"], "warmup": args.warmup, "ms_per_step": f32["ms"] / f32["steps"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic: vacuum-fluctuation initial conditions generated on the GPU from the seed",
        "config": {"workload": WORKLOAD, "storage": "fp32 fields/momenta, fp64 reductions and a, a'",
                   "replicas": ws, "sites": sites, "passes_per_step": PASSES_PER_STEP,
                   "l2": "no flush: each pass streams 537 MB (> 126 MB L2) through ping-pong buffers"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "dk_pass_scalar<float,2,1>", "bytes_per_launch": bpl,
                     "avg_launch_ms": f32["pass_ms"], "launches_timed": f32["npass"],
                     "peak_kind": peak_kind},
        "cpu_baseline": {"value": cpu_value, "unit": "site-updates/s", "cores": 1, "kind": "oracle",
                         "sample": "%d VV4 steps of the same model on a %d^3 box with the same "
                                   "lattice spacing, oracle FP64 single thread" % (csteps, n_ref)},
        "cpu_baseline_all_cores": cpu_all,
        "e2e": {"value": results["e2e"]["value"], "unit": "site-updates/s",
                "h2d_bytes_per_step": results["e2e"]["h2d"],
                "d2h_bytes_per_step": results["e2e"]["d2h"], "steps": results["e2e"]["steps"],
                "mode": "two contexts on two streams take the steps in turn (upload overlaps the other "
                        "context's passes); every step uploads its state and reads its energies",
                "serial_value": results["e2e"]["serial"]},
        "gpu_launches": f32["launches"],
        # one site advanced by one DK pass (an integrator stage): VV4 has three per step
        "stage_site_updates_per_s": value * PASSES_PER_STEP,
        "clocks": f32["clocks"],
        "fp64_plain": {"value": v64, "unit": "site-updates/s", "steps": f64["steps"],
                       "stage_site_updates_per_s": v64 * PASSES_PER_STEP,
                       "ms_per_step": f64["ms"] / f64["steps"], "achieved_gbs": achieved64,
                       "frac_hbm": achieved64 / peak, "avg_launch_ms": f64["pass_ms"],
                       "fp32_speedup": value / v64,
                       "roofline": {"bound": "alu", "kernel": "dk_pass_scalar<double,2,1>",
                                    "achieved": None if ins_rate is None else ins_rate / 1e9,
                                    "peak": fp64_rate / 2 / 1e9, "unit": "G FP64 instructions/s",
                                    "frac": None if ins_rate is None else ins_rate / (fp64_rate / 2),
                                    "fp64_instructions_per_site_pass": ins64,
                                    "fp64_flops_per_site_pass": ops64,
                                    "measured_fp64_tflops": fp64_rate / 1e12,
                                    "peak_kind": "measured: cl_measure_fp64_rate (independent FMA chains), "
                                                 "FMA instructions per second"}},
        "sanity": {"rho_f32": f32["rho"], "rho_f64": f64["rho"], "a_f32": f32["a"],
                   "nonfinite": f32["nonfinite"] + f64["nonfinite"]},
        "other_rows": others,
    }
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


# SU(2) x U(1) doublet workload: equal homogeneous components, vacuum
# fluctuations, links at the identity, electric fields from the Gauss laws
def su2_params(P):
    return dict(dt=0.01, integrator=P.LF, lam=1.0, v=0.5, gQ=0.6, gQB=0.8, fstar_over_omegastar=1.3,
                phi0=[0.5] * 4, dphi0=[0.1] * 4, fluct_amp2=1e-2, expansion=P.EXP_OFF, fstar_over_mp=0.5)


def other_workloads(P, torch, stream, peak):
    """The other hot-path rows, timed briefly with the library's pass-timing hook
    (CUDA events around every launch on the lattice stream): the U(1) and the
    SU(2) x U(1) passes at 256^3, the two-field step at 512^3, the 64-lattice
    ensemble, and the adjoint sweep's cost at 128^3."""
    SU2 = su2_params(P)
    out = {}
    # U(1) Abelian-Higgs, 256^3, FP32, leapfrog dt = 0.01, no expansion
    u1 = dict(dt=0.01, integrator=P.LF, lam=1.0, v=1.0, gQ=0.5, fstar_over_omegastar=1.0,
              phi0=[1.0, 1.0], fluct_amp2=1e-2, expansion=P.EXP_OFF, fstar_over_mp=0.5)
    lat = P.Lattice(P.MODEL_U1_HIGGS, 256, 0.1, 1.0, 1, P.make_params(precision=P.FP32, stream=stream, **u1))
    rel0 = lat.gauss()[0]
    lat.step(20)
    torch.cuda.synchronize()
    sampler = ClockSampler(0).start()
    time.sleep(0.3)
    lat.pass_timing(reset=True)
    lat.enable_pass_timing(True)
    t0 = time.time()
    lat.step(500)
    torch.cuda.synchronize()
    t1 = time.time()
    ms, n = lat.pass_timing(reset=True)
    lat.enable_pass_timing(False)
    clocks = sampler.stop().summary(t0 - 0.05, t1 + 0.05)
    lat.step(2480)   # the rest of the 3000-step run of the workload
    rel = lat.gauss()[0]
    lat.close()
    gbs = 256 ** 3 * 10 * 2 * 4 / (ms / n * 1e-3) / 1e9
    row = {"site_updates_per_s": 256 ** 3 * n / (ms * 1e-3), "pass_us": ms / n * 1e3,
           "achieved_gbs": gbs, "frac_hbm": gbs / peak, "bytes_per_site_pass": 80,
           "gauss_rel_at_start": rel0, "gauss_rel_after_3000_steps": rel,
           "kernel": "dk_pass_u1<float,0,true,256>", "clocks": clocks}
    if NCU_U1["source_hash"] == u1_source_hash():
        ipc = NCU_U1["thread_instructions_per_site"]
        ach = 256 ** 3 * ipc / (ms / n * 1e-3)
        row["issue_roof"] = {"thread_instructions_per_site": ipc, "achieved_lane_instr_per_s": ach,
                             "peak_lane_instr_per_s": ISSUE_PEAK_LANE_INSTR_PER_S,
                             "frac": ach / ISSUE_PEAK_LANE_INSTR_PER_S,
                             "ncu_dram_bytes_per_site": NCU_U1["dram_bytes_per_site"]}
    out["u1_higgs_256_fp32_lf"] = row
    # C2 at its larger size: 512^3, two fields, FP32 storage, VV4, self-consistent expansion
    try:
        lat = P.Lattice(P.MODEL_LPHI4_CHI, 512, KIR, ALPHA, SEED, P.make_params(precision=P.FP32, stream=stream,
                                                                               **PARAMS))
        lat.step(3)
        torch.cuda.synchronize()
        lat.pass_timing(reset=True)
        lat.enable_pass_timing(True)
        lat.step(20)
        torch.cuda.synchronize()
        ms, n = lat.pass_timing(reset=True)
        lat.close()
        gbs = 512 ** 3 * PASS_BYTES_PER_SITE["f32"] / (ms / n * 1e-3) / 1e9
        out["c2_512_fp32_vv4"] = {"site_updates_per_s": 512 ** 3 * (n / PASSES_PER_STEP) / (ms * 1e-3),
                                  "pass_us": ms / n * 1e3, "achieved_gbs": gbs, "frac_hbm": gbs / peak,
                                  "bytes_per_site_pass": PASS_BYTES_PER_SITE["f32"],
                                  "kernel": "dk_pass_scalar<float,2,1>"}
    except Exception as e:  # noqa: BLE001
        out["c2_512_fp32_vv4"] = {"error": str(e)[:300]}
    # SU(2) x U(1) doublet, 256^3, FP32, leapfrog dt = 0.01, no expansion
    lat = P.Lattice(P.MODEL_SU2U1_HIGGS, 256, 0.1, 1.0, 1, P.make_params(precision=P.FP32, stream=stream, **SU2))
    lat.step(10)
    torch.cuda.synchronize()
    lat.pass_timing(reset=True)
    lat.enable_pass_timing(True)
    lat.step(200)
    torch.cuda.synchronize()
    ms, n = lat.pass_timing(reset=True)
    rel = lat.gauss()[0]
    lat.close()
    gbs = 256 ** 3 * 35 * 2 * 4 / (ms / n * 1e-3) / 1e9
    row = {"site_updates_per_s": 256 ** 3 * n / (ms * 1e-3), "pass_us": ms / n * 1e3,
           "achieved_gbs": gbs, "frac_hbm": gbs / peak, "bytes_per_site_pass": 280,
           "gauss_rel_after_210_steps": rel, "kernel": "kd_pass_su2<float,0,32,8,false,256>"}
    if NCU_SU2["source_hash"] == su2_source_hash():
        ipc = NCU_SU2["thread_instructions_per_site"]
        ach = 256 ** 3 * ipc / (ms / n * 1e-3)
        row["issue_roof"] = {"thread_instructions_per_site": ipc, "achieved_lane_instr_per_s": ach,
                             "peak_lane_instr_per_s": ISSUE_PEAK_LANE_INSTR_PER_S,
                             "frac": ach / ISSUE_PEAK_LANE_INSTR_PER_S,
                             "ncu_dram_bytes_per_site": NCU_SU2["dram_bytes_per_site"]}
    out["su2u1_doublet_256_fp32_lf"] = row
    # the lphi4SU2U1 model (doublet, singlet, U(1)-charged scalar, both gauge fields), 256^3, FP32, LF
    try:
        lat = P.Lattice(P.MODEL_LPHI4_SU2U1, 256, 0.1, 1.0, 1,
                        P.make_params(precision=P.FP32, stream=stream, **dict(SU2, v=0.0, qG=1.5, qH=0.8, Qc=0.7)))
        lat.step(10)
        torch.cuda.synchronize()
        lat.pass_timing(reset=True)
        lat.enable_pass_timing(True)
        lat.step(200)
        torch.cuda.synchronize()
        ms, n = lat.pass_timing(reset=True)
        rel = lat.gauss()[0]
        lat.close()
        gbs = 256 ** 3 * 41 * 2 * 4 / (ms / n * 1e-3) / 1e9
        row = {"site_updates_per_s": 256 ** 3 * n / (ms * 1e-3), "pass_us": ms / n * 1e3,
               "achieved_gbs": gbs, "frac_hbm": gbs / peak, "bytes_per_site_pass": 328,
               "gauss_rel_after_210_steps": rel, "kernel": "kd_pass_su2<float,0,32,16,true,256>"}
        if NCU_FULL["source_hash"] == su2_source_hash():
            ipc = NCU_FULL["thread_instructions_per_site"]
            ach = 256 ** 3 * ipc / (ms / n * 1e-3)
            row["issue_roof"] = {"thread_instructions_per_site": ipc, "achieved_lane_instr_per_s": ach,
                                 "peak_lane_instr_per_s": ISSUE_PEAK_LANE_INSTR_PER_S,
                                 "frac": ach / ISSUE_PEAK_LANE_INSTR_PER_S,
                                 "ncu_dram_bytes_per_site": NCU_FULL["dram_bytes_per_site"]}
        out["lphi4su2u1_256_fp32_lf"] = row
    except Exception as e:  # noqa: BLE001
        out["lphi4su2u1_256_fp32_lf"] = {"error": str(e)[:300]}
    # ensemble: 16 each of 32^3, 64^3, 96^3, 128^3, FP32, VV4 with expansion, seeds 1..64
    Ns = [32] * 16 + [64] * 16 + [96] * 16 + [128] * 16
    E = P.Ensemble(P.MODEL_LPHI4_CHI, Ns, [KIR * N_LAT / n for n in Ns], ALPHA, list(range(1, 65)),
                   P.make_params(precision=P.FP32, stream=stream, **PARAMS))
    E.step(5)
    torch.cuda.synchronize()
    E.pass_timing(reset=True)
    E.enable_pass_timing(True)
    E.step(100)
    torch.cuda.synchronize()
    ms, n = E.pass_timing(reset=True)
    E.close()
    sites = sum(x ** 3 for x in Ns)
    gbs = sites * 32 / (ms / n * 1e-3) / 1e9
    out["ensemble_64_fp32_vv4"] = {"site_updates_per_s": sites * 100 / (ms * 1e-3), "pass_us": ms / n * 1e3,
                                   "achieved_gbs": gbs, "frac_hbm": gbs / peak, "sites": sites,
                                   "launches_per_step_call": 1}
    # adjoint: 128^3 FP32, VV4 dt = 0.005, 4000 steps, checkpoints every 500, with
    # self-consistent expansion (the model's runs) and without
    for tag, adj in (("self", dict(PARAMS, expansion=P.EXP_SELF)), ("noexp", dict(PARAMS, expansion=P.EXP_OFF))):
        g = P.Lattice(P.MODEL_LPHI4_CHI, 128, KIR * N_LAT / 128, ALPHA, SEED,
                      P.make_params(precision=P.FP32, stream=stream, **adj))
        g.step(5)
        g.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(4000)
        g.sync()
        torch.cuda.synchronize()
        t_fwd = time.perf_counter() - t0
        sampler = ClockSampler(0).start()
        time.sleep(0.3)
        g.enable_pass_timing(True)
        g.pass_timing(reset=True)
        g.adjoint_pass_timing(reset=True)
        t0 = time.perf_counter()
        w0 = time.time()
        J, dq, _, ab = g.adjoint(4000, 500, scale=True)
        torch.cuda.synchronize()
        t_adj = time.perf_counter() - t0
        w1 = time.time()
        g.enable_pass_timing(False)
        ams, an = g.adjoint_pass_timing(reset=True)
        fms, fn = g.pass_timing(reset=True)
        clocks = sampler.stop().summary(w0 - 0.05, w1 + 0.05)
        g.close()
        sites = 128 ** 3
        agbs = sites * 64 / (ams / an * 1e-3) / 1e9
        out["adjoint_128_fp32_vv4_" + tag] = {
            "forward_s": t_fwd, "forward_plus_reverse_s": t_adj,
            "reverse_over_forward": (t_adj - t_fwd) / t_fwd, "J": J, "dJ_dq": dq, "dJ_da": ab[0], "dJ_db": ab[1],
            "steps": 4000, "ckpt_every": 500,
            "adjoint_pass_us": ams / an * 1e3, "adjoint_passes": an, "adjoint_bytes_per_site_pass": 64,
            "adjoint_pass_gbs": agbs, "adjoint_frac_hbm": agbs / peak,
            "forward_pass_us_inside_adjoint": fms / max(fn, 1) * 1e3,
            "adjoint_pass_over_forward_pass": (ams / an) / (fms / max(fn, 1)) if fn else None,
            "clocks": clocks,
            "note": "reverse = the cl_adjoint call minus a plain forward run of the same steps; pass times from "
                    "CUDA events around each launch (cl_adjoint_pass_timing)"}
    # initial conditions and spectra at 256^3, outside a run's timed loop: wall time
    # of cl_init (allocation, Fourier-space draws, inverse FFTs, IC kernels) and of
    # cl_spectrum of one field (complex conversion, three FFT axis passes, shell
    # sums); a failure here leaves the other rows standing
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat = P.Lattice(P.MODEL_LPHI4_CHI, N_LAT, KIR, ALPHA, SEED,
                        P.make_params(precision=P.FP32, stream=stream, **PARAMS))
        torch.cuda.synchronize()
        t_init = time.perf_counter() - t0
        lat.spectrum(0)
        torch.cuda.synchronize()
        reps = 10
        t0 = time.perf_counter()
        for _ in range(reps):
            lat.spectrum(0)
        torch.cuda.synchronize()
        t_spec = (time.perf_counter() - t0) / reps
        lat.close()
        sites = N_LAT ** 3
        gbs = sites * 52 / t_spec / 1e9
        out["ics_and_spectrum_256_fp32"] = {
            "init_s": t_init, "spectrum_ms": t_spec * 1e3, "model_bytes_per_site": 52,
            "spectrum_gbs": gbs, "frac_hbm": gbs / peak,
            "note": "host wall time; 52 B/site through the half spectrum = the FP32 field read 4 + the half "
                    "spectrum written 8 by the x-axis transform + y and z axis passes 16 each + shell sums 8; "
                    "includes the call's read-back and synchronisation; the transform is bound by its FP64 "
                    "butterflies, not by memory"}
    except Exception as e:  # noqa: BLE001
        out["ics_and_spectrum_256_fp32"] = {"error": str(e)[:300]}
    return out


def profile_case(name):
    """Small cases for ncu captures: one launch of the kernel named in
    profiles/ after a short setup (no timing, no JSON line)."""
    import torch

    import paper_2102_01031_gb300 as P
    torch.cuda.set_device(0)
    P.build()
    stream = P.torch_stream()
    if name == "scalar256":   # one cooperative launch of the three VV4 passes of a step
        lat = P.Lattice(P.MODEL_LPHI4_CHI, N_LAT, KIR, ALPHA, SEED,
                        P.make_params(precision=P.FP32, stream=stream, **PARAMS))
        lat.step(1)
    elif name == "u1_128":    # single-pass launches of the leapfrog U(1) pass
        u1 = dict(dt=0.01, integrator=P.LF, lam=1.0, v=1.0, gQ=0.5, fstar_over_omegastar=1.0,
                  phi0=[1.0, 1.0], fluct_amp2=1e-2, expansion=P.EXP_OFF, fstar_over_mp=0.5)
        lat = P.Lattice(P.MODEL_U1_HIGGS, 128, 0.2, ALPHA, SEED, P.make_params(precision=P.FP32, stream=stream, **u1))
        for _ in range(4):
            lat.step(1)
    elif name == "u1_256":    # single-pass launches of the leapfrog U(1) pass at the benchmark size
        u1 = dict(dt=0.01, integrator=P.LF, lam=1.0, v=1.0, gQ=0.5, fstar_over_omegastar=1.0,
                  phi0=[1.0, 1.0], fluct_amp2=1e-2, expansion=P.EXP_OFF, fstar_over_mp=0.5)
        lat = P.Lattice(P.MODEL_U1_HIGGS, 256, 0.1, ALPHA, SEED, P.make_params(precision=P.FP32, stream=stream, **u1))
        for _ in range(4):
            lat.step(1)
    elif name == "su2_128":   # single-pass launches of the leapfrog SU(2) x U(1) doublet pass
        lat = P.Lattice(P.MODEL_SU2U1_HIGGS, 128, 0.2, ALPHA, SEED,
                        P.make_params(precision=P.FP32, stream=stream, **su2_params(P)))
        for _ in range(4):
            lat.step(1)
    elif name == "su2_256":   # the doublet pass at the benchmark size (the variant built for N = 256)
        lat = P.Lattice(P.MODEL_SU2U1_HIGGS, 256, 0.1, ALPHA, SEED,
                        P.make_params(precision=P.FP32, stream=stream, **su2_params(P)))
        for _ in range(4):
            lat.step(1)
    elif name == "full_256":  # the lphi4SU2U1 pass at the benchmark size
        lat = P.Lattice(P.MODEL_LPHI4_SU2U1, 256, 0.1, ALPHA, SEED,
                        P.make_params(precision=P.FP32, stream=stream, **dict(su2_params(P), v=0.0, qG=1.5,
                                                                               qH=0.8, Qc=0.7)))
        for _ in range(4):
            lat.step(1)
    elif name == "full_128":  # single-pass launches of the leapfrog lphi4SU2U1 pass
        lat = P.Lattice(P.MODEL_LPHI4_SU2U1, 128, 0.2, ALPHA, SEED,
                        P.make_params(precision=P.FP32, stream=stream,
                                      **dict(su2_params(P), v=0.0, qG=1.5, qH=0.8, Qc=0.7)))
        for _ in range(4):
            lat.step(1)
    elif name == "ensemble64":   # the 64-lattice ensemble: one cooperative launch of a VV4 step
        Ns = [32] * 16 + [64] * 16 + [96] * 16 + [128] * 16
        E = P.Ensemble(P.MODEL_LPHI4_CHI, Ns, [KIR * N_LAT / n for n in Ns], ALPHA, list(range(1, 65)),
                       P.make_params(precision=P.FP32, stream=stream, **PARAMS))
        for _ in range(4):
            E.step(1)
    elif name == "scalar256_fp64":   # the FP64 plain pass: one cooperative launch of a VV4 step
        lat = P.Lattice(P.MODEL_LPHI4_CHI, N_LAT, KIR, ALPHA, SEED,
                        P.make_params(precision=P.FP64, stream=stream, **PARAMS))
        lat.step(1)
        print("fp64 rate %.4g FLOP/s" % P.measure_fp64_rate(stream))
    elif name == "spectrum256":   # two cl_spectrum calls of one field at 256^3 (FFT, shell sums)
        lat = P.Lattice(P.MODEL_LPHI4_CHI, N_LAT, KIR, ALPHA, SEED,
                        P.make_params(precision=P.FP32, stream=stream, **PARAMS))
        lat.spectrum(0)
        lat.spectrum(1)
    elif name in ("adj128", "adj128self"):    # adjoint sweep of 4 VV4 steps at 128^3
        exp = P.EXP_OFF if name == "adj128" else P.EXP_SELF
        lat = P.Lattice(P.MODEL_LPHI4_CHI, 128, 0.2, ALPHA, SEED,
                        P.make_params(precision=P.FP32, stream=stream, **dict(PARAMS, expansion=exp)))
        lat.adjoint(4, 2)
    else:
        raise SystemExit("unknown profile case %s" % name)
    torch.cuda.synchronize()
    return 0


def ctypes_sizeof_energies(P):
    import ctypes
    return ctypes.sizeof(P.Energies)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--fp64-steps", type=int, default=1000)
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=150.0,
                    help="reference arm: site-steps budget / 1e6 that sizes its oracle box")
    ap.add_argument("--no-extra", action="store_true", help="skip the U(1), ensemble and adjoint rows")
    ap.add_argument("--profile-case", choices=("scalar256", "scalar256_fp64", "u1_128", "u1_256", "su2_128", "full_128", "su2_256", "full_256",
                             "adj128", "adj128self", "spectrum256", "ensemble64"),
                    help="run one small case for an ncu capture and exit")
    args = ap.parse_args()
    if args.profile_case:
        return profile_case(args.profile_case)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
