"""Benchmark: matching-pursuit atoms/s on GB300 through the C ABI.

One step = one pass of the whole hot path on one batch of synthetic input:
mp_analyze (multi-Gabor DGT analysis, E_0, max trees) + mp_run (persistent
selection / update loop until 40 dB residual SNR or K_max atoms).

Default workload (one GPU): ``multi3_2p18`` -- one real signal, L = 2^18 at
44.1 kHz (chirps, notes, transients, pink noise at 30 dB), three Blackman
dictionaries w = M = 512/1024/2048 with a = w/4, kernel threshold 1e-4, stop
at 40 dB or K = 50000 atoms.  The batched form (``batch256``: 256 signals of
log-uniform length 2^14..2^20, stop at 30 dB or K = 20000) is measured as a
secondary figure in the same run.

Printed: one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2202_12380_gb300 import inputs  # noqa: E402
from paper_2202_12380_gb300.shard import partition, reduce_totals  # noqa: E402

METRIC = "MP atoms/sec to 40 dB residual SNR, batched FP32 vs plain form; % HBM roofline"
UNIT = "atoms/s"
L2_FLUSH_BYTES = 512 << 20


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _workload(name):
    cfg = inputs.WORKLOADS[name]
    dicts = [(inputs.make_window(k, w), a, M) for (k, w, a, M) in cfg["dicts"]]
    xs = inputs.workload_signal(name)
    if not isinstance(xs, list):
        xs = [xs]
    return cfg, dicts, xs


def _config_desc(name, cfg, xs):
    return {
        "workload": name,
        "signals": len(xs),
        "L_total": int(sum(len(x) for x in xs)),
        "dicts": ["%s w=%d a=%d M=%d" % d for d in cfg["dicts"]],
        "kern_thr": cfg["eps"],
        "kmax": cfg["kmax"],
        "target_snr_db": cfg["snr_db"],
        "l2": "flushed between steps (%d MiB write)" % (L2_FLUSH_BYTES >> 20),
    }


# --------------------------------------------------------------- clocks ----

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
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
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [s.strip() for s in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ roofline -----

def update_bytes(mg, plan, state, atoms_per_sig):
    """Algorithmic bytes of the residual updates: for every selected atom and
    every dictionary v, the stored coefficients covered by the atom's class
    tile and by its conjugate partner's, each read and written once as
    complex64 (16 bytes)."""
    W = plan.W
    infos = {}
    for u in range(W):
        for v in range(W):
            i0 = mg.mp_plan_tile_info(plan, u, v, 0, 0)
            for cf in range(i0["rf"]):
                for ct in range(i0["rt"]):
                    infos[(u, v, cf, ct)] = mg.mp_plan_tile_info(plan, u, v, cf, ct)
    total = 0
    for atoms in atoms_per_sig:
        if atoms.size == 0:
            continue
        for u in range(W):
            sel = atoms[atoms["dict"] == u]
            if sel.size == 0:
                continue
            Mu, au = plan.M[u], plan.a[u]
            ks = sel["m"].astype(np.int64)
            js = sel["n"].astype(np.int64)
            edge = (ks == 0) | (2 * ks == Mu)
            for v in range(W):
                Mv, av = plan.M[v], plan.a[v]
                Mr = Mv // 2 + 1
                rf = infos[(u, v, 0, 0)]["rf"]
                rt = infos[(u, v, 0, 0)]["rt"]
                ct = js % rt
                for conj in (False, True):
                    kk = (Mu - ks) if conj else ks
                    cf = kk % rf
                    base_m = kk * (Mv // Mu) if Mv >= Mu else (kk - cf) // rf
                    R = np.array([infos[(u, v, int(a), int(b))]["R"] for a, b in zip(cf, ct)])
                    C = np.array([infos[(u, v, int(a), int(b))]["C"] for a, b in zip(cf, ct)])
                    ilo = np.array([infos[(u, v, int(a), int(b))]["i_lo"] for a, b in zip(cf, ct)])
                    A = (base_m + ilo) % Mv
                    p1 = np.clip(np.minimum(np.minimum(A + R, Mv), Mr) - A, 0, None)
                    p2 = np.where(A + R > Mv, np.clip(np.minimum(A + R - Mv, Mr), 0, None), 0)
                    n = (p1 + p2) * C
                    if conj:
                        n = np.where(edge, 0, n)
                    total += int(n.sum()) * 16
    return total


def code_sha256(path):
    """sha256 of a C/CUDA source with // comments, trailing blanks and empty
    lines removed: it changes with the code, not with its comments."""
    lines = []
    for line in open(path, encoding="utf-8").read().splitlines():
        i = line.find("//")
        if i >= 0:
            line = line[:i]
        line = line.rstrip()
        if line:
            lines.append(line)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


def _profile_traffic(kernel_file, workload):
    """dram bytes per launch of the MP loop from the committed ncu summary,
    or None when the kernel's code changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "mp_loop_%s.md" % workload)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"code_sha256:\s*([0-9a-f]{64})", text)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not (m and t):
        return None
    return float(t.group(1)) if code_sha256(kernel_file) == m.group(1) else None


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _profile_l2(workload):
    """lts__t_bytes per launch of the MP loop from the committed ncu summary,
    or None when the kernel's code changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "mp_loop_%s.md" % workload)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"code_sha256:\s*([0-9a-f]{64})", text)
    t = re.search(r"l2_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not (m and t):
        return None
    kf = os.path.join(ROOT, "paper_2202_12380_gb300", "csrc", "mp_loop_kernel.cuh")
    return float(t.group(1)) if code_sha256(kf) == m.group(1) else None


def analysis_flops(plan, lengths):
    """Flops of the split-BF16 analysis GEMMs: per dictionary three BF16
    products of the [Arows x Kp] DFT matrix with the [Kp x frames] frame
    matrix (Arows = 2 Mrp rounded up to 128 rows, Mrp = M/2 + 1 rounded up to
    32 bins; Kp = w rounded up to 64; frames = L / a per signal)."""
    tot = 0
    for w, a, M in zip(plan.wlen, plan.a, plan.M):
        mrp = 32 * -(-(M // 2 + 1) // 32)
        arows = 128 * -(-(2 * mrp) // 128)
        kp = 64 * -(-w // 64)
        frames = sum(int(L) // a for L in lengths)
        tot += 3 * 2 * arows * kp * frames
    return tot


def tensor_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["bf16_tflops"]), "measured (BF16 burst)"
    return 1900.0, "fallback"


def analysis_roofline(plan, lengths, ms):
    flops = analysis_flops(plan, lengths)
    peak, src = tensor_peak()
    achieved = flops / (ms / 1e3) / 1e12
    return {"bound": "tensor", "flops_per_launch": flops, "ms": ms, "achieved": achieved,
            "unit": "TFLOP/s", "peak": peak, "peak_source": src, "frac": achieved / peak,
            "time": "the whole analysis step (BF16 split of the signal, the tcgen05 GEMM of "
                    "every dictionary, tree build, energy), CUDA events"}


def l2_copy_peak(torch, sizes_mib=(2, 4, 8, 16, 24), iters=200):
    """L2 bandwidth of copies whose source and destination (2 x size MiB)
    stay resident in the 129 MB L2: read + write bytes / CUDA-event time,
    best over the sizes of five runs of `iters` back-to-back copies each.
    Returns (GB/s, size in MiB of the best)."""
    best, arg = 0.0, None
    for mbytes in sizes_mib:
        n = (mbytes << 20) // 4
        a = torch.randn(n, device="cuda")
        b = torch.empty_like(a)
        for _ in range(20):
            b.copy_(a)
        for _ in range(5):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e[0].record()
            for _ in range(iters):
                b.copy_(a)
            e[1].record()
            torch.cuda.synchronize()
            gbs = 2.0 * n * 4 * iters / (e[0].elapsed_time(e[1]) / 1e3) / 1e9
            if gbs > best:
                best, arg = gbs, mbytes
        del a, b
    return best, arg


def host_info():
    """CPU model and logical core count of the host that runs the oracle."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"cpu_model": model, "nproc": os.cpu_count(), "machine": os.uname().machine}


# ------------------------------------------------------------- GPU arm -----

def run_gpu(args):
    import torch

    from paper_2202_12380_gb300 import mpgabor as mg

    ws, rank, local = _dist()
    dev = local if torch.cuda.device_count() > 1 else 0
    torch.cuda.set_device(dev)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    cfg, dicts, xs = _workload(args.workload)
    stream = torch.cuda.Stream()
    aflag = mg.MP_ANALYSIS_BF16X3 if args.analysis == "bf16x3" else mg.MP_ANALYSIS_FP32
    plan = mg.mp_plan_create([d[0] for d in dicts], [d[1] for d in dicts], [d[2] for d in dicts],
                             cfg["eps"], aflag, stream)
    xd = [torch.from_numpy(x).cuda() for x in xs]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    K, snr = cfg["kmax"], cfg["snr_db"]
    state = None
    W = len(dicts)

    def one_step(ev):
        nonlocal state
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            state = mg.mp_analyze(plan, xd, state)
            ev[1].record(stream)
            mg.mp_run_async(state, K, snr)
            ev[2].record(stream)

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.zero_()

    for _ in range(args.warmup):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        flush_l2()
        one_step(ev)
    stream.synchronize()
    n0, _, _ = mg.mp_get_status(state)

    # signal gather, energy partials + sum, (BF16 split), one GEMM and one
    # tree build per dictionary, the MP loop
    launches_per_step = 3 + (1 if args.analysis == "bf16x3" else 0) + 2 * W + 1
    clocks = ClockSampler(dev)
    clocks.start()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        flush_l2()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        one_step(ev)
        evs.append(ev)
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [e[0].elapsed_time(e[2]) for e in evs]
    loop_ms = [e[1].elapsed_time(e[2]) for e in evs]
    ana_ms = [e[0].elapsed_time(e[1]) for e in evs]
    n_atoms, stops, snrs = mg.mp_get_status(state)
    atoms_per_step = int(np.sum(n_atoms))
    t_total = sum(step_ms) / 1e3
    # replicas: the slowest rank's time, the atoms of all ranks
    t_total, total_atoms_all = reduce_totals(t_total, float(atoms_per_step) * args.steps,
                                             device="cuda")
    value = total_atoms_all / t_total

    # roofline of the MP loop kernel
    atoms_list = [mg.mp_get_atoms(state, b) for b in range(len(xs))]
    alg_bytes = update_bytes(mg, plan, state, atoms_list)
    loop_s = float(np.mean(loop_ms)) / 1e3
    achieved = alg_bytes / loop_s / 1e9
    peak, peak_src = _peaks()
    traffic = _profile_traffic(os.path.join(ROOT, "paper_2202_12380_gb300", "csrc", "mp_loop_kernel.cuh"),
                               args.workload)

    # end to end through the C ABI with host buffers (pinned)
    e2e = None
    if args.e2e_steps > 0:
        xh = [torch.from_numpy(x).pin_memory() for x in xs]
        st_h = None
        for _ in range(2):
            st_h = mg.mp_analyze_host(plan, xh, st_h)
            mg.mp_run(st_h, K, snr)
            _ = [mg.mp_get_atoms(st_h, b) for b in range(len(xs))]
        h2d = int(sum(x.numel() * 4 for x in xh))
        d2h = 0
        t0 = time.perf_counter()
        tot = 0
        for _ in range(args.e2e_steps):
            st_h = mg.mp_analyze_host(plan, xh, st_h)
            n, _, _ = mg.mp_run(st_h, K, snr)
            got = [mg.mp_get_atoms(st_h, b) for b in range(len(xs))]
            tot += int(sum(g.size for g in got))
            d2h = int(sum(g.nbytes for g in got))
        t1 = time.perf_counter()
        e2e = {"value": tot / (t1 - t0), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": args.e2e_steps}
        st_h.close()

    batched = None
    if args.batched:
        batched = run_batched(args, mg, torch, ws, rank)

    cpu, ref = None, None
    if rank == 0 and ws == 1 and args.cpu_baseline:
        g_atoms = mg.mp_get_atoms(state, 0)
        g_errs = mg.mp_get_errors(state, 0)
        g_E0 = float(g_errs[-1] * 10 ** (snrs[0] / 10)) if g_errs.size else 1.0
        cpu, ref = cpu_baseline(args.workload, args.cpu_atoms, g_atoms, g_errs, g_E0)
        if args.batched and args.cpu_batched_every > 0:
            cpu["batched"] = cpu_baseline_batched(every=args.cpu_batched_every)

    # the other workloads (one signal each): atoms/s and error against the oracle
    secondary = []
    if rank == 0 and args.secondary:
        ref1 = _oracle_sample("single_gauss_16k", inputs.WORKLOADS["single_gauss_16k"]["kmax"],
                              keep=True)[2] if args.cpu_baseline else None
        secondary.append(run_secondary(mg, torch, "single_gauss_16k", ref=ref1, steps=3))
        secondary.append(run_secondary(mg, torch, "multi5_2p20", flags=mg.MP_ANALYSIS_BF16X3,
                                       label="multi5_2p20, split-BF16 analysis"))
        secondary.append(run_secondary(mg, torch, "stress_2p23", steps=1))
        if args.workload == "multi3_2p18":
            secondary.append(run_secondary(mg, torch, "multi3_2p18", flags=mg.MP_COEF_FP64,
                                           ref=ref, label="multi3_2p18, FP64 planes (parity form)"))

    # L2: the loop's state of this workload is L2-resident; its bandwidth
    # ceiling is a copy that stays in L2
    l2_peak, l2_size = l2_copy_peak(torch)
    l2_traffic = _profile_l2(args.workload)

    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": float(np.mean(step_ms)),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded mixture; the paper's audio is not available)",
        "config": dict(_config_desc(args.workload, cfg, xs), analysis=args.analysis,
                       parallelism="replicas" if ws > 1 else "single"),
        "atoms_per_step": atoms_per_step,
        "stop_reasons": [int(s) for s in stops[:8]],
        "final_snr_db": [float(q) for q in snrs[:8]],
        "analysis_ms": float(np.mean(ana_ms)),
        "mp_loop_ms": float(np.mean(loop_ms)),
        "gpu_launches": launches_per_step * args.steps,
        "roofline": {"kernel": "k_mp_loop", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": peak_src,
                     "alg_bytes_per_launch": alg_bytes,
                     "alg_bytes_per_atom": alg_bytes / max(atoms_per_step, 1),
                     "l2": {"achieved": achieved, "peak": l2_peak, "unit": "GB/s",
                            "frac": achieved / l2_peak, "traffic": l2_traffic,
                            "peak_source": "measured here: L2-resident copy (best of 2 x 2..24 "
                                           "MiB, here 2 x %d MiB), read + write bytes / "
                                           "CUDA-event time" % l2_size}},
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    if batched is not None:
        line["batched"] = batched
    if secondary:
        line["secondary"] = secondary
    if rank == 0:
        print(json.dumps(line))
    state.close()
    plan.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_batched(args, mg, torch, ws=1, rank=0):
    """Secondary figure: the batched form (256 uneven signals, one launch),
    launch shape and launch order picked by the autotuner (the order: the
    signals with the most atoms in the tuner's probe of this batch start
    first), analysis + MP captured in a CUDA graph and replayed.  The loop
    time with the default shape and order (longest signal first) is reported
    beside it.  With several ranks the 256 signals are partitioned over the
    ranks by their work: every rank decomposes the whole batch once (the
    same deterministic atoms on every GPU, so every rank computes the same
    partition without an exchange) and takes its share by atoms per signal;
    the totals are reduced."""
    from paper_2202_12380_gb300 import autotune

    cfg, dicts, xs = _workload("batch256")
    n_all, L_all = len(xs), int(sum(len(x) for x in xs))
    stream = torch.cuda.Stream()
    aflag = mg.MP_ANALYSIS_BF16X3 if args.batched_analysis == "bf16x3" else mg.MP_ANALYSIS_FP32
    plan = mg.mp_plan_create([d[0] for d in dicts], [d[1] for d in dicts], [d[2] for d in dicts],
                             cfg["eps"], aflag, stream)
    xd = [torch.from_numpy(x).cuda() for x in xs]
    split = "single"
    if ws > 1:
        probe = mg.mp_analyze(plan, xd)
        mg.mp_run(probe, cfg["kmax"], cfg["snr_db"])
        n_probe, _, _ = mg.mp_get_status(probe)
        probe.close()
        mine = partition([float(v) for v in n_probe], ws)[rank]
        xs, xd = [xs[i] for i in mine], [xd[i] for i in mine]
        split = "signals partitioned over %d ranks by atoms per signal" % ws
    # probe: the workload itself (its K and stop target), so the tail of the
    # long signals is part of what the tuner compares
    # the loop with the default launch order (longest signal first) and the
    # default shape, for comparison with the tuned one
    state = mg.mp_analyze(plan, xd)
    mg.mp_run(state, cfg["kmax"], cfg["snr_db"])  # sizes the atom buffers
    default_shape = mg.mp_state_get_launch(state)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with torch.cuda.stream(stream):
        mg.mp_analyze(plan, xd, state)
        e[0].record(stream)
        mg.mp_run_async(state, cfg["kmax"], cfg["snr_db"])
        e[1].record(stream)
    stream.synchronize()
    loop_default_ms = e[0].elapsed_time(e[1])
    # autotuner: per-signal work from a probe run sets the launch order, then
    # every feasible shape is timed with it
    shape, tune_ms, work = autotune.tune(plan, xd, k_probe=args.tune_atoms or cfg["kmax"],
                                         target_snr_db=cfg["snr_db"], stream=stream,
                                         repeats=args.tune_repeats, with_work=True)
    autotune.apply(state, shape)
    if work is not None:
        mg.mp_state_set_work_hint(state, work)
    mg.mp_run(state, cfg["kmax"], cfg["snr_db"])
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="thread_local"):
        mg.mp_analyze(plan, xd, state)
        mg.mp_run_async(state, cfg["kmax"], cfg["snr_db"])
    res = []
    for it in range(args.batched_steps + 1):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        with torch.cuda.stream(stream):
            e[0].record(stream)
            graph.replay()
            e[1].record(stream)
        stream.synchronize()
        if it > 0:
            res.append(e[0].elapsed_time(e[1]))
    # analysis / loop split, measured once outside the graph
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    with torch.cuda.stream(stream):
        e[0].record(stream)
        mg.mp_analyze(plan, xd, state)
        e[1].record(stream)
        mg.mp_run_async(state, cfg["kmax"], cfg["snr_db"])
        e[2].record(stream)
    stream.synchronize()
    n, stops, snrs = mg.mp_get_status(state)
    atoms = [mg.mp_get_atoms(state, b) for b in range(len(xs))]
    alg = update_bytes(mg, plan, state, atoms)
    step = float(np.mean(res))
    loop = e[1].elapsed_time(e[2])
    peak, _ = _peaks()
    # the slowest rank's step against the atoms of all ranks (one rank: itself)
    t_max, atoms_all = reduce_totals(step / 1e3, float(n.sum()), device="cuda")
    # measured DRAM bytes of one launch (ncu summary, while the source matches)
    traffic = _profile_traffic(os.path.join(ROOT, "paper_2202_12380_gb300", "csrc", "mp_loop_kernel.cuh"),
                               "batch256")
    out = {"workload": "batch256", "analysis": args.batched_analysis, "signals": n_all,
           "L_total": L_all, "launch_shape": list(shape),
           "launch_order": "most work first (atoms per signal from the tuner's probe of this "
                           "batch)" if work is not None else "longest signal first",
           "autotune_ms": {("%dx%d" % k[:2]) + ("/%d keys" % k[2] if k[2] else ""): round(v, 3)
                           for k, v in tune_ms.items()},
           "mp_loop_ms_default": loop_default_ms,
           "default_launch": "%dx%d, longest signal first" % tuple(default_shape),
           "cuda_graph": True, "atoms_per_step": int(atoms_all), "ms_per_step": t_max * 1e3,
           "analysis_ms": e[0].elapsed_time(e[1]), "mp_loop_ms": loop,
           "value": atoms_all / t_max, "unit": UNIT,
           "parallelism": split,
           "scaling": "strong" if ws > 1 else None,
           "analysis_roofline": analysis_roofline(plan, [len(x) for x in xs],
                                                  e[0].elapsed_time(e[1]))
           if args.batched_analysis == "bf16x3" else None,
           "mp_loop_hbm_frac": alg / (loop / 1e3) / 1e9 / peak,
           "mp_loop_traffic": traffic,
           "mp_loop_dram_frac": (traffic / (loop / 1e3) / 1e9 / peak) if traffic else None,
           "stops": {str(k): int(v) for k, v in zip(*np.unique(stops, return_counts=True))}}
    state.close()
    plan.close()
    return out


def _stored_oracle_prefix(name):
    """The oracle's first atoms of a workload as written by
    tests/golden/make_oracle_prefix.py (None if absent)."""
    path = os.path.join(ROOT, "tests", "golden", "%s_oracle_prefix.npz" % name)
    if not os.path.exists(path):
        return None
    z = np.load(path)

    class Ref:
        pass

    r = Ref()
    for k in ("dict", "m", "n", "c", "E", "s1", "s2"):
        setattr(r, k, z[k])
    r.E0 = float(z["E0"])
    r.n_atoms = int(z["dict"].size)
    r.input_sha256 = str(z["input_sha256"])
    return r


def run_secondary(mg, torch, name, flags=0, steps=2, ref=None, label=None):
    """One more workload timed like the headline (analysis + MP per step,
    CUDA events on the plan's stream, L2 flushed between steps), with its
    error against the oracle where one is at hand: a live oracle run (ref),
    or the stored oracle prefix of the workload."""
    import hashlib
    cfg, dicts, xs = _workload(name)
    stream = torch.cuda.Stream()
    plan = mg.mp_plan_create([d[0] for d in dicts], [d[1] for d in dicts], [d[2] for d in dicts],
                             cfg["eps"], flags, stream)
    xd = [torch.from_numpy(x).cuda() for x in xs]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    K, snr = cfg["kmax"], cfg["snr_db"]
    state = None
    ms = []
    for it in range(steps + 1):
        with torch.cuda.stream(stream):
            flush.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e[0].record(stream)
            state = mg.mp_analyze(plan, xd, state)
            mg.mp_run_async(state, K, snr)
            e[1].record(stream)
        stream.synchronize()
        if it > 0:
            ms.append(e[0].elapsed_time(e[1]))
    if flags & mg.MP_ANALYSIS_BF16X3:
        with torch.cuda.stream(stream):
            ea = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ea[0].record(stream)
            mg.mp_analyze(plan, xd, state)
            ea[1].record(stream)
            mg.mp_run_async(state, K, snr)
        stream.synchronize()
        ana = analysis_roofline(plan, [len(x) for x in xs], ea[0].elapsed_time(ea[1]))
    else:
        ana = None
    n, stops, snrs = mg.mp_get_status(state)
    atoms = int(n.sum())
    step = float(np.mean(ms))
    out = {"workload": name, "label": label or name, "flags": int(flags),
           "launch_shape": list(mg.mp_state_get_launch(state)), "atoms_per_step": atoms,
           "ms_per_step": step, "value": atoms / (step / 1e3), "unit": UNIT,
           "stop_reasons": [int(q) for q in stops[:4]], "final_snr_db": [float(q) for q in snrs[:4]]}
    if ana is not None:
        out["analysis_roofline"] = ana
    g_atoms = mg.mp_get_atoms(state, 0)
    g_errs = mg.mp_get_errors(state, 0)
    g_E0 = float(g_errs[-1] * 10 ** (snrs[0] / 10)) if g_errs.size else 1.0
    if ref is None and name != "stress_2p23":
        stored = _stored_oracle_prefix(name)
        if stored is not None:
            sha = hashlib.sha256(np.ascontiguousarray(xs[0], np.float32).tobytes()).hexdigest()
            if sha == stored.input_sha256:
                ref = stored
                out["oracle"] = "stored prefix of %d atoms (tests/golden)" % stored.n_atoms
            else:
                out["oracle"] = "stored prefix not used: this host generated another input"
    elif ref is not None:
        out["oracle"] = "live oracle run of %d atoms" % ref.n_atoms
    if ref is not None:
        out["oracle_error"] = oracle_error(g_atoms, g_errs, g_E0, ref)
    if name == "stress_2p23":
        # the FP64 energy estimate against the true residual of the synthesis
        y = torch.zeros(len(xs[0]), dtype=torch.float32, device="cuda")
        true_snr = mg.mp_synthesize(state, 0, y)
        out["estimate_vs_true_snr_db"] = [float(snrs[0]), float(true_snr)]
    state.close()
    plan.close()
    return out


# -------------------------------------------------------------- CPU arm -----

def _oracle_sample(workload, atoms, keep=False):
    from oracle import cmp
    cfg, dicts, xs = _workload(workload)
    x = xs[0].astype(np.float64)
    t0 = time.perf_counter()
    res = cmp.mp_coef(dicts, x, cfg["eps"], atoms, cfg["snr_db"])
    dt = time.perf_counter() - t0
    return (res.n_atoms, dt, res) if keep else (res.n_atoms, dt)


def _oracle_batch_one(job):
    """One batched-form signal decomposed by the oracle to its own stop
    (process-pool worker)."""
    from oracle import cmp
    x, eps, kmax, snr = job
    cfg, dicts, _ = _workload_dicts_only("batch256")
    t0 = time.perf_counter()
    res = cmp.mp_coef(dicts, x.astype(np.float64), eps, kmax, snr)
    return res.n_atoms, time.perf_counter() - t0


def _workload_dicts_only(name):
    cfg = inputs.WORKLOADS[name]
    return cfg, [(inputs.make_window(k, w), a, M) for (k, w, a, M) in cfg["dicts"]], None


def cpu_baseline_batched(every=8, workers=None):
    """The oracle on the batched form over all host cores: every `every`-th
    signal of batch256 in length order, each decomposed to its own stop (30
    dB or K = 20000) by a spawn process pool with one worker per core.
    atoms/s = atoms of the sample / wall time of the pool."""
    import multiprocessing as mp
    cfg = inputs.WORKLOADS["batch256"]
    order = np.argsort(inputs.batch_lengths(cfg, cfg["id"]), kind="stable")
    pick = [int(i) for i in order[::every]]
    workers = workers or os.cpu_count() or 1
    workers = max(1, min(workers, len(pick)))
    xs = inputs.batch_subset("batch256", pick)
    jobs = [(x, cfg["eps"], cfg["kmax"], cfg["snr_db"]) for x in xs]
    # longest first, so the pool's tail is short
    jobs.sort(key=lambda j: -len(j[0]))
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(workers) as pool:
        res = pool.map(_oracle_batch_one, jobs, chunksize=1)
    wall = time.perf_counter() - t0
    atoms = int(sum(r[0] for r in res))
    return {"value": atoms / wall, "unit": UNIT, "cores": workers, "kind": "oracle",
            "host": host_info(),
            "sample": "FP64 C oracle, process pool of %d workers (one signal each, 1 thread per "
                      "worker): %d of the 256 batch256 signals (every %d-th by length, L_total "
                      "%d) decomposed to their own stop, %d atoms in %.1f s wall" % (
                          workers, len(pick), every, int(sum(len(j[0]) for j in jobs)), atoms,
                          wall)}


def cpu_baseline(workload, atoms, gpu_atoms=None, gpu_errs=None, gpu_E0=None):
    """The oracle timed on the host; with the GPU decomposition of the same
    signal also its error against the oracle over the common prefix."""
    n, dt, ref = _oracle_sample(workload, atoms, keep=True)
    out = {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_info(),
           "sample": "FP64 C oracle (coefficient-domain MP, 1 thread): analysis + first %d atoms "
                     "of the %s signal, %.1f s" % (n, workload, dt)}
    if gpu_atoms is not None:
        out["oracle_error"] = oracle_error(gpu_atoms, gpu_errs, gpu_E0, ref)
    return out, ref


def oracle_error(atoms, errs, E0, ref):
    """Sequence agreement, coefficient error and SNR-curve deviation of a GPU
    decomposition against the FP64 oracle's, up to the oracle's first near
    tie (relative gap of the two largest |rho| below 1e-6)."""
    gap = (ref.s1 - ref.s2) / np.where(ref.s1 > 0, ref.s1, 1.0)
    ties = np.where(gap < 1e-6)[0]
    tie = int(ties[0]) if ties.size else ref.n_atoms
    k = min(atoms.size, ref.n_atoms)
    same = (atoms["dict"][:k] == ref.dict[:k]) & (atoms["m"][:k] == ref.m[:k]) & \
        (atoms["n"][:k] == ref.n[:k])
    div = int(np.argmin(same)) if not same.all() else k
    upto = min(tie, div)
    c = atoms["re"][:upto].astype(np.float64) + 1j * atoms["im"][:upto].astype(np.float64)
    rel = np.abs(c - ref.c[:upto]) / np.abs(ref.c[:upto]) if upto else np.zeros(1)
    dsnr = np.abs(10 * np.log10(E0 / errs[:k]) - 10 * np.log10(ref.E0 / ref.E[:k]))
    return {"first_near_tie": tie, "first_divergence": div, "compared": upto,
            "coef_rel_max": float(rel.max()),
            "coef_normwise": float(np.linalg.norm(c - ref.c[:upto]) / np.linalg.norm(ref.c[:upto]))
            if upto else 0.0,
            "snr_db_max_to_tie": float(dsnr[:upto].max()) if upto else 0.0,
            "snr_db_max_common": float(dsnr.max()) if k else 0.0,
            "atoms_gpu": int(atoms.size), "atoms_oracle": int(ref.n_atoms)}


def run_reference(args):
    """The oracle as it stands on one host core, on the GPU arm's workload and
    work per step: analysis + matching pursuit to the workload's own stop
    (40 dB or K_max for multi3_2p18), so both arms time the same atoms.
    Warm-up steps are short samples (first 1000 atoms)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    cfg, dicts, xs = _workload(args.workload)
    for _ in range(args.warmup):
        _oracle_sample(args.workload, min(1000, cfg["kmax"]))
    tot_atoms, tot_t = 0, 0.0
    for _ in range(args.steps):
        n, dt = _oracle_sample(args.workload, cfg["kmax"])
        tot_atoms += n
        tot_t += dt
    value = tot_atoms / tot_t
    sample = ("FP64 C oracle (coefficient-domain MP, 1 thread): analysis + decomposition of the "
              "%s signal to its stop (%d atoms per step), %d steps" % (
                  args.workload, tot_atoms // max(args.steps, 1), args.steps))
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_t / max(args.steps, 1),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded mixture; the paper's audio is not available)",
        "config": dict(_config_desc(args.workload, cfg, xs), analysis=args.analysis,
                       parallelism="single"),
        "atoms_per_step": tot_atoms // max(args.steps, 1),
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": 1,
                         "host": host_info(), "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="multi3_2p18",
                    choices=["multi3_2p18", "single_gauss_16k", "multi5_2p20", "stress_2p23"])
    ap.add_argument("--analysis", default="fp32", choices=["fp32", "bf16x3"],
                    help="analysis precision (bf16x3: split-BF16 DFT-GEMM on tcgen05)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--batched-analysis", default="bf16x3", choices=["fp32", "bf16x3"],
                    help="analysis precision of the batched form")
    ap.add_argument("--batched-steps", type=int, default=3)
    ap.add_argument("--tune-atoms", type=int, default=0,
                    help="atoms per launch-shape probe of the batched autotuner "
                         "(0: the workload's K)")
    ap.add_argument("--tune-repeats", type=int, default=2,
                    help="timed runs per launch shape in the autotuner (the best counts)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-atoms", type=int, default=50000)
    ap.add_argument("--cpu-batched-every", type=int, default=8,
                    help="batched CPU baseline: every n-th batch256 signal (0: skip)")
    ap.add_argument("--no-secondary", dest="secondary", action="store_false",
                    help="skip the single_gauss_16k / multi5_2p20 / stress_2p23 / FP64 figures")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
