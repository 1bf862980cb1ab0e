"""Benchmark of the exact GF(p) dot-product hot path on GB300.

Default workload (one step = one persistent kernel launch): batched uneven
dot products, 4096 pairs with lengths floor(2^U), U ~ Uniform(8, 20), primes
uniform over {32749, 65521, 67108859, 2^31-1, 2^32-5}, residues uniform in
[0, p) from the seeded counter-based generator, representation and work-unit
length per (p, n) chosen by the in-library autotuner at setup.  The operands
(about 4.1 GB) are larger than L2, so consecutive steps read HBM cold.

Prints ONE JSON line (rank 0).  Multi-GPU (torchrun): every rank runs its own
batch (weak scaling, no data-path collective); time is the max over ranks.
``--impl reference`` times the CPU oracle instead, on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gfp_inputs as gi  # noqa: E402

METRIC = "GF(p) Gmac/s & % HBM roofline vs plain per-term-% kernel; serve p50/p99 ms"
UNIT = "Gmac/s"
COUNT = 4096
SEED = gi.BASE_SEED + 1
WORKLOAD = ("batched uneven dot products over GF(p): 4096 pairs, lengths floor(2^U), "
            "U~Uniform(8,20), p uniform over {32749, 65521, 67108859, 2147483647, 4294967291}, "
            "uint32 residues uniform in [0,p); one persistent launch per step; autotuned "
            "representation and work-unit length per (p, n)")


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def hbm_peak():
    pk = peaks()
    if pk and pk.get("hbm_gbs"):
        return float(pk["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


_OWN_PEAKS = {}


def own_peaks() -> dict:
    """Ceilings measured in this run by the project's own probe kernels
    (libgfppeaks): a read-only HBM stream (the ceiling of kernels that only
    read, as the dot products do), L2-to-SM reads and the DFMA rate.  Measured
    once per process, after the clock-sampled load phase."""
    if not _OWN_PEAKS:
        from paper_cs_0404008_gb300 import peaks as pk
        for kind, nb, reps in (("read_hbm", 4 << 30, 12), ("read_l2", 64 << 20, 8), ("dfma", 0, 4)):
            r = pk.measure(kind, nb, reps)
            _OWN_PEAKS[kind] = {"peak": r["rate"], "unit": r["unit"],
                                "source": f"libgfppeaks {kind} (best of {reps}), this run"}
    return _OWN_PEAKS


def with_read_peak(roof: dict) -> dict:
    """Adds the fraction of the measured read-only stream ceiling to an HBM roofline."""
    rp = own_peaks()["read_hbm"]
    roof["read_stream"] = {"peak": rp["peak"], "frac": roof["achieved"] / rp["peak"],
                           "unit": "GB/s", "source": rp["source"]}
    return roof


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def rank_seed(rank: int) -> int:
    """Weak scaling: every rank runs its own batch of the same recipe."""
    return SEED + 1000 * rank


def reduce_max(value: float, device: str = "cpu") -> float:
    """Max over the ranks of the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks sampler (nvidia-smi during the timed region)
# ---------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self.t:
                self.t.join(timeout=2)

    def summary(self, t0, t1):
        rows = [l for (t, l) in self.lines if t0 <= t <= t1] or [l for (_, l) in self.lines]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in rows:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    lens, ps = gi.batched_shapes(COUNT, SEED)
    sel = np.arange(0, COUNT, 4)           # bounded sample: every 4th pair
    lens_s, ps_s = lens[sel], ps[sel]
    off, total, x, y = gi.batched_operands(lens_s, ps_s, SEED)
    macs = float(lens_s.sum())
    for _ in range(max(args.warmup, 0)):
        oracle.dot_batch(ps_s, lens_s, off, x, y, threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.dot_batch(ps_s, lens_s, off, x, y, threads=cores)
    dt = time.perf_counter() - t0
    value = macs * args.steps / dt / 1e9
    sample = (f"every 4th pair of the 4096-pair batch ({len(sel)} pairs, {macs:.3e} MACs per step), "
              f"per-term Zpz oracle over {cores} host threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "every 4th pair"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def traffic_record(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    sources are unchanged since it was taken (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kernel)
    except Exception:
        return None
    if not rec:
        return None
    if source_hash(rec.get("sources", [])) != rec.get("sha256"):
        return None
    return rec


def source_hash(files) -> str:
    """SHA-256 of the sources a traffic record was captured from, as the
    release build compiles them: blocks under `#ifdef GFP_DEVICE_CHECKS`,
    `GFP_DCHECK(` lines, whole-line `//` comments and blank lines are left
    out."""
    h = hashlib.sha256()
    for f in files:
        skip = False
        for line in open(os.path.join(ROOT, f), encoding="utf-8"):
            st = line.strip()
            if st.startswith("#ifdef GFP_DEVICE_CHECKS"):
                skip = True
                continue
            if skip:
                skip = not st.startswith("#endif")
                continue
            if not st or st.startswith("//") or "GFP_DCHECK(" in line:
                continue
            h.update(line.encode())
    return h.hexdigest()


def traffic_for(kernel: str, alg_bytes: float):
    """DRAM bytes of one launch of `kernel` on this line's workload: the
    committed ncu ratio of DRAM bytes to algorithmic bytes times the line's
    algorithmic bytes per launch (None when there is no record or the
    kernel's sources changed since it was taken)."""
    rec = traffic_record(kernel)
    return rec["dram_bytes_per_algorithmic_byte"] * alg_bytes if rec else None


class Batch:
    """The batched workload generated on the device (same definition as the
    host generator: pair i uses streams 2+2i and 3+2i)."""

    def __init__(self, g, torch, seed, count=COUNT):
        self.lens, self.ps = gi.batched_shapes(count, seed)
        self.off, self.total = gi.aligned_offsets(self.lens)
        self.x = torch.empty(self.total, dtype=torch.int32, device="cuda")
        self.y = torch.empty(self.total, dtype=torch.int32, device="cuda")
        for i, (n, p, o) in enumerate(zip(self.lens, self.ps, self.off)):
            if n:
                g.gfp_fill_uniform(int(p), seed, 2 + 2 * i, self.x[int(o):int(o) + int(n)])
                g.gfp_fill_uniform(int(p), seed, 3 + 2 * i, self.y[int(o):int(o) + int(n)])
        torch.cuda.synchronize()
        self.macs = float(self.lens.sum())
        self.bytes = 8.0 * self.macs + 4.0 * count

    def pairs(self, repr_=0, mask=None):
        out = []
        for i, (n, p, o) in enumerate(zip(self.lens, self.ps, self.off)):
            if mask is not None and not mask[i]:
                continue
            o, n = int(o), int(n)
            out.append((int(p), self.x[o:o + n], self.y[o:o + n], n, repr_))
        return out


def time_plan(torch, plan, out, steps, stream):
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    with torch.cuda.stream(stream):
        evs[0].record(stream)
        for i in range(steps):
            plan.exec(out, stream)
            evs[i + 1].record(stream)
    torch.cuda.synchronize()
    per = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]
    return sum(per), per


def run_gpu(args):
    import torch
    from paper_cs_0404008_gb300 import gfpdot as g

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev_index = torch.cuda.current_device()
    g.load()
    ctx = g.Context(dev_index)
    stream = torch.cuda.Stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v: float) -> float:
        return reduce_max(v, "cuda")

    # --- autotune (install-time selection, per (p, n) bucket) ---
    t_tune = time.perf_counter()
    if not args.no_tune:
        g.gfp_tune(ctx, list(gi.PRIMES_BATCHED), 8, 20, None)
    t_tune = time.perf_counter() - t_tune

    count = args.pairs
    batch = Batch(g, torch, rank_seed(rank), count)
    out = torch.empty(count, dtype=torch.int32, device="cuda")
    plan = g.BatchPlan(ctx, batch.pairs())
    n_units, _ = plan.info()

    # warm-up, then a load phase under the clock sampler, then the timed steps
    for _ in range(max(args.warmup, 3)):
        plan.exec(out, stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(dev_index)
    sampler.start()
    t_load = time.time()
    while not args.no_clocks and time.time() - t_load < 1.0:
        for _ in range(50):
            plan.exec(out, stream)
        torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    barrier()
    tw0 = time.time()
    total_ms, per = time_plan(torch, plan, out, args.steps, stream)
    barrier()
    tw1 = time.time()
    launches = ctx.launch_count() - launches0
    time.sleep(0.25)
    sampler.stop()
    clocks = sampler.summary(t_load, tw1 + 0.2)
    total_ms = max_over_ranks(total_ms)
    ms_step = total_ms / args.steps
    value = batch.macs * world * args.steps / (total_ms / 1e3) / 1e9
    avg_launch_ms = statistics.mean(per)
    peak, peak_kind = hbm_peak()
    achieved = batch.bytes / (avg_launch_ms / 1e3) / 1e9
    trec = traffic_record("k_dot_batched")

    # --- the same batch through other representations (same GPU, same inputs) ---
    extra = {}
    if not args.quick:
        for name, rp, mask in (("perterm", g.GFP_REPR_PERTERM, None),
                               ("u64_carry", g.GFP_REPR_U64_CARRY, None),
                               ("centered", g.GFP_REPR_CENTERED, None),
                               ("montgomery", g.GFP_REPR_MONTGOMERY, None),
                               ("fp64_p_lt_2^26", g.GFP_REPR_FP64, batch.ps < (1 << 26))):
            pl = g.BatchPlan(ctx, batch.pairs(rp, mask))
            sel = batch.lens if mask is None else batch.lens[mask]
            o2 = torch.empty(max(len(sel), 1), dtype=torch.int32, device="cuda")
            time_plan(torch, pl, o2, 3, stream)
            ms, _ = time_plan(torch, pl, o2, 10, stream)
            macs = float(sel.sum())
            extra[name] = {"gmacs": macs * 10 / (ms / 1e3) / 1e9, "ms_per_launch": ms / 10,
                           "gbs": (8 * macs) * 10 / (ms / 1e3) / 1e9}
            if rp == g.GFP_REPR_FP64:
                # one fma (2 flops) per multiply-add: the FP64 loop's own roofline
                dp = own_peaks()["dfma"]
                tf = 2 * macs * 10 / (ms / 1e3) / 1e12
                extra[name]["dfma"] = {"bound": "alu", "achieved": tf, "peak": dp["peak"],
                                       "unit": "TFLOP/s", "frac": tf / dp["peak"],
                                       "source": dp["source"]}
            pl.close()
        # tuned vs per-term speed-up on identical exact results
        extra["tuned_over_perterm"] = value / world / extra["perterm"]["gmacs"]

    # --- end to end through the host-buffer entry point ---
    e2e = None
    if not args.no_e2e:
        xh = torch.empty(batch.total, dtype=torch.int32, pin_memory=True)
        yh = torch.empty(batch.total, dtype=torch.int32, pin_memory=True)
        xh.copy_(batch.x)
        yh.copy_(batch.y)
        oh = torch.empty(count, dtype=torch.int32, pin_memory=True)
        lens_u = batch.lens.astype(np.uint64)
        offs_u = batch.off.astype(np.uint64)
        ps_u = batch.ps.astype(np.uint32)
        g.gfp_dot_batched_host(ctx, ps_u, lens_u, offs_u, xh, yh, oh, stream)
        e2e_steps = max(3, min(args.steps, 10))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            g.gfp_dot_batched_host(ctx, ps_u, lens_u, offs_u, xh, yh, oh, stream)
        barrier()
        dt = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": batch.macs * world * e2e_steps / dt / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(2 * 4 * batch.total), "d2h_bytes_per_step": int(4 * count)}
        # the host link bounds this path: measure one large pinned copy on the
        # same pinned buffer and report the step's input bytes against it
        dst = torch.empty(batch.total, dtype=torch.int32, device="cuda")
        dst.copy_(xh, non_blocking=True)
        torch.cuda.synchronize()
        c0, c1 = _events(torch, 2)
        c0.record()
        for _ in range(3):
            dst.copy_(xh, non_blocking=True)
        c1.record()
        torch.cuda.synchronize()
        link = 3 * 4.0 * batch.total / (c0.elapsed_time(c1) / 1e3) / 1e9
        step_h2d = 2 * 4.0 * batch.total * e2e_steps / dt / 1e9
        e2e["link"] = {"h2d_gbs_measured": link, "step_input_gbs": step_h2d, "frac": step_h2d / link,
                       "note": "pinned host-to-device copy of one input vector, same buffers"}
        del dst
        # results of the e2e path equal the device path
        torch.cuda.synchronize()
        if not np.array_equal(oh.numpy().view(np.uint32), out.cpu().numpy().view(np.uint32)):
            raise SystemExit("e2e result differs from the device-resident result")
        del xh, yh

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline()

    # the other workloads, measured after the timed region (one GPU, rank 0)
    also = None
    if rank == 0 and world == 1 and not args.quick and not args.no_also:
        also = {}
        plan.close()
        plan._keep = None
        batch.x = batch.y = None
        torch.cuda.empty_cache()
        for name in ("dot", "matvec", "block", "csr", "gfq"):
            ln = measure_secondary(args, name, g, torch, ctx, stream)
            also[name] = {k: ln[k] for k in ("value", "unit", "ms_per_step", "config", "roofline")
                          if k in ln}
            for k in ("single_call_us", "graph_of_256_single_dots", "single_dot_2^27", "same_gpu",
                      "fields", "p_2^31-1", "prepared"):
                if k in ln:
                    also[name][k] = ln[k]
            torch.cuda.empty_cache()
        sv = measure_serve(args, g)
        also["serve"] = {"value": sv["value"], "unit": sv["unit"], "config": sv["config"],
                         **sv["serve"]}
        # the same service at 50 % and 90 % of its measured capacity, same stream length
        sweep = {}
        for ld in (0.5, 0.9):
            a2 = argparse.Namespace(**vars(args))
            a2.load = ld
            s2 = measure_serve(a2, g)["serve"]
            sweep[f"{int(ld * 100)}%"] = {k: s2[k] for k in ("p50_ms", "p99_ms", "achieved_jobs_per_s",
                                                             "all_ok", "verify_mismatches")}
            sweep[f"{int(ld * 100)}%"]["requests"] = a2.requests
        also["serve"]["load_sweep"] = sweep

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD if count == COUNT else WORKLOAD.replace("4096 pairs", f"{count} pairs"),
                       "pairs": count, "macs_per_step": batch.macs,
                       "operand_bytes_per_step": batch.bytes, "work_units": n_units,
                       "l2": "inputs larger than L2 (operands ~4.1 GB per step)",
                       "parallelism": f"weak: {world} independent batch(es)",
                       "tune_seconds": round(t_tune, 2),
                       "plan": "built-in rules" if args.no_tune else "tuned at setup"},
            "gpu_launches": int(launches),
            "roofline": with_read_peak(
                {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                 "frac": achieved / peak, "peak_kind": f"{peak_kind} hbm_gbs (copy test)",
                 "kernel": "k_dot_batched",
                 "traffic": (trec["dram_bytes_per_algorithmic_byte"] * batch.bytes
                             if trec else None),
                 "traffic_source": ("ncu dram bytes of a 512-pair capture, scaled by "
                                    "algorithmic bytes" if trec else None)}),
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "same_gpu": extra,
            "also": also,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def cpu_baseline():
    """The oracle (per-term Zpz, Section 2.1) on the host cores: the whole
    batch once for warm-up plus a timed pass over every 4th pair."""
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    lens, ps = gi.batched_shapes(COUNT, SEED)
    sel = np.arange(0, COUNT, 4)
    lens_s, ps_s = lens[sel], ps[sel]
    off, total, x, y = gi.batched_operands(lens_s, ps_s, SEED)
    oracle.dot_batch(ps_s[:64], lens_s[:64], off[:64], x, y, threads=cores)
    # repeat the sample until about 1 s of wall time (roughly 10-30 s of CPU
    # work on the host cores), at least 3 times
    reps = 0
    t0 = time.perf_counter()
    while reps < 3 or (time.perf_counter() - t0 < 1.0 and reps < 40):
        oracle.dot_batch(ps_s, lens_s, off, x, y, threads=cores)
        reps += 1
    dt = time.perf_counter() - t0
    macs = float(lens_s.sum()) * reps
    line = {"value": macs / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"every 4th pair of the batch ({len(sel)} pairs, {lens_s.sum():.3e} MACs) "
                      f"x {reps} repetitions, {dt:.2f} s wall on {cores} threads"}
    line["context"] = cpu_context(ps_s, lens_s, off, x, y, cores, oracle)
    return line


def cpu_context(ps, lens, off, x, y, cores, oracle):
    """Context beside the oracle figure, on the same sample: the oracle on one
    thread, and the paper's delayed division on the CPU (libgfpsweep: 64-bit
    blocks of Section 3.1, and the block-overflow hybrid of Section 3.4, which
    needs no remainder inside the loop even for p near 2^32) on all cores."""
    from concurrent.futures import ThreadPoolExecutor

    from paper_cs_0404008_gb300 import sweep
    macs = float(lens.sum())
    t0 = time.perf_counter()
    oracle.dot_batch(ps, lens, off, x, y, threads=1)
    single = macs / (time.perf_counter() - t0) / 1e9
    out = {"oracle_1_thread": single, "unit": UNIT}
    ref = oracle.dot_batch(ps, lens, off, x, y, threads=cores)
    for v in ("block64", "hybrid64"):
        def run(j):
            a, n = int(off[j]), int(lens[j])
            return sweep.dot(v, int(ps[j]), x[a:a + n], y[a:a + n])
        with ThreadPoolExecutor(cores) as ex:
            list(ex.map(run, range(min(64, len(ps)))))   # warm-up
            t0 = time.perf_counter()
            got = list(ex.map(run, range(len(ps))))
            dt = time.perf_counter() - t0
        if not np.array_equal(np.array(got, np.uint32), ref):
            raise SystemExit(f"cpu {v} differs from the oracle")
        out[f"delayed_{v}_{cores}_threads"] = macs / dt / 1e9
    return out


# ---------------------------------------------------------------------------
# secondary workloads (one JSON line each): single dot, Wiedemann matvec
# ---------------------------------------------------------------------------

def _events(torch, n):
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def run_secondary(args):
    import torch
    from paper_cs_0404008_gb300 import gfpdot as g

    torch.cuda.set_device(0)
    g.load()
    ctx = g.Context(0)
    stream = torch.cuda.Stream()
    line = measure_secondary(args, args.workload, g, torch, ctx, stream)
    ctx.close()
    print(json.dumps(line), flush=True)


GFQ_FIELDS = [(2, 8), (3, 10), (65521, 1)]


def gfq_kernel(p: int, k: int) -> str:
    """The kernel the library runs for GF(p^k) (values summed for prime fields,
    characteristic 2 and small odd extensions, Zech additions otherwise)."""
    if p == 2 or k == 1:
        return "k_gfq_dot_exp"
    return "k_gfq_dot_add" if p ** k <= 256 else "k_gfq_dot"
GFQ_N = 1 << 27


def measure_gfq(args, g, torch, stream, line, peak, peak_kind):
    """Discrete-logarithm dot products over GF(2^8), GF(3^10) and GF(65521):
    2^27 16-bit codes per vector (256 MiB each, larger than L2), one launch per
    dot product; 4 bytes read per multiply-add."""
    res = {}
    n = GFQ_N
    fields = GFQ_FIELDS
    if args.gfq_fields:
        fields = [tuple(int(t) for t in f.split("^")) for f in args.gfq_fields.split(",")]
    for p, k in fields:
        q = p ** k
        f = g.gfp_gfq_find_primitive(p, k)
        fq = g.Field(p, k, f)
        v = torch.empty(n, dtype=torch.int32, device="cuda")
        X = torch.empty(n, dtype=torch.int16, device="cuda")
        Y = torch.empty(n, dtype=torch.int16, device="cuda")
        out = torch.empty(8, dtype=torch.int16, device="cuda")
        seed = gi.BASE_SEED + 7
        g.gfp_fill_uniform(q, seed, 0, v)
        fq.to_log(v, X)
        g.gfp_fill_uniform(q, seed, 1, v)
        fq.to_log(v, Y)
        del v
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                fq.dot(X, Y, out, n, stream)
            reps = max(10, args.steps // 10)
            e0, e1 = _events(torch, 2)
            e0.record(stream)
            for _ in range(reps):
                fq.dot(X, Y, out, n, stream)
            e1.record(stream)
        torch.cuda.synchronize()
        assert fq.check() == g.GFP_OK
        t = e0.elapsed_time(e1) / reps
        gbs = 4.0 * n / (t / 1e3) / 1e9
        res[f"GF({p}^{k})"] = {"q": q, "ms": t, "gmacs": n / (t / 1e3) / 1e9, "gbs": gbs,
                               "frac": gbs / peak, "kernel": gfq_kernel(p, k)}
        fq.close()
        del X, Y
        torch.cuda.empty_cache()
    best = max(res.values(), key=lambda r: r["gmacs"])
    worst = min(res.values(), key=lambda r: r["gmacs"])
    line.update({
        "value": worst["gmacs"], "ms_per_step": worst["ms"],
        "config": {"workload": "dot products over GF(q) in the discrete-logarithm (Zech) "
                               "representation, 2^27 uint16 codes per vector, uniform elements, "
                               "fields " + ", ".join(res),
                   "value_is": "the slowest field"},
        "roofline": with_read_peak(
            {"bound": "hbm", "achieved": worst["gbs"], "peak": peak, "unit": "GB/s",
             "frac": worst["frac"], "kernel": worst["kernel"],
             "traffic": traffic_for(worst["kernel"], 4.0 * n),
             "peak_kind": f"{peak_kind} hbm_gbs", "best_field_frac": best["frac"]}),
        "fields": res,
        "gpu_launches": 1,
    })
    return line


def measure_secondary(args, workload, g, torch, ctx, stream):
    """One secondary workload on an existing context; returns its JSON line."""
    peak, peak_kind = hbm_peak()
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic"}
    if workload == "gfq":
        return measure_gfq(args, g, torch, stream, line, peak, peak_kind)
    if workload == "dot":
        p, n, nvec = 65521, 1 << 20, 256
        seed = gi.BASE_SEED
        # 256 operand pairs on rotating buffers: 2 GiB, larger than L2
        X = torch.empty((nvec, n), dtype=torch.int32, device="cuda")
        Y = torch.empty((nvec, n), dtype=torch.int32, device="cuda")
        for i in range(nvec):
            g.gfp_fill_uniform(p, seed, 2 * i, X[i])
            g.gfp_fill_uniform(p, seed, 2 * i + 1, Y[i])
        out = torch.empty(nvec, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        # (i) single-call latency, back to back on one buffer (8 MiB, L2-resident)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                g.gfp_dot(ctx, p, X[0], Y[0], out[0:1], stream)
            ev = _events(torch, args.steps + 1)
            ev[0].record(stream)
            for i in range(args.steps):
                g.gfp_dot(ctx, p, X[0], Y[0], out[0:1], stream)
                ev[i + 1].record(stream)
        torch.cuda.synchronize()
        lat = sorted(ev[i].elapsed_time(ev[i + 1]) * 1e3 for i in range(args.steps))
        # (ii) 256 dots captured in one CUDA graph, rotating buffers (L2 cold)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            for i in range(nvec):
                g.gfp_dot(ctx, p, X[i], Y[i], out[i:i + 1], stream)
            torch.cuda.synchronize()
            with torch.cuda.graph(graph, stream=stream):
                for i in range(nvec):
                    g.gfp_dot(ctx, p, X[i], Y[i], out[i:i + 1], stream)
        for _ in range(3):
            graph.replay()
        torch.cuda.synchronize()
        e0, e1 = _events(torch, 2)
        reps = max(5, args.steps // 20)
        e0.record()
        for _ in range(reps):
            graph.replay()
        e1.record()
        torch.cuda.synchronize()
        t_graph = e0.elapsed_time(e1) / reps
        # (ii') one large single dot (2^27 elements per operand, 1 GiB, larger than L2)
        nl = 1 << 27
        XL = torch.empty(nl, dtype=torch.int32, device="cuda")
        YL = torch.empty(nl, dtype=torch.int32, device="cuda")
        g.gfp_fill_uniform(p, seed, 1000, XL)
        g.gfp_fill_uniform(p, seed, 1001, YL)
        with torch.cuda.stream(stream):
            for _ in range(3):
                g.gfp_dot(ctx, p, XL, YL, out[0:1], stream)
            e0, e1 = _events(torch, 2)
            e0.record(stream)
            for _ in range(10):
                g.gfp_dot(ctx, p, XL, YL, out[0:1], stream)
            e1.record(stream)
        torch.cuda.synchronize()
        t_large = e0.elapsed_time(e1) / 10
        del XL, YL
        # (iii) the same 256 dots as one persistent batched launch
        plan = g.BatchPlan(ctx, [(p, X[i], Y[i], n) for i in range(nvec)])
        ms, per = time_plan(torch, plan, out, max(10, args.steps // 10), stream)
        t_batch = ms / len(per)
        # (iv) the plain per-term kernel (one remainder per term) on the same pairs
        ctx.set_repr(g.GFP_REPR_PERTERM)
        plan_pt = g.BatchPlan(ctx, [(p, X[i], Y[i], n) for i in range(nvec)])
        ctx.set_repr(0)
        out_pt = torch.empty(nvec, dtype=torch.int32, device="cuda")
        ms_pt, per_pt = time_plan(torch, plan_pt, out_pt, 5, stream)
        t_pt = ms_pt / len(per_pt)
        plan_pt.close()
        if not torch.equal(out_pt, out):
            raise SystemExit("per-term and tuned batched dots differ")
        macs = float(nvec * n)
        gm = lambda t_ms: macs / (t_ms / 1e3) / 1e9
        line.update({
            "value": gm(t_batch), "ms_per_step": t_batch,
            "config": {"workload": "256 dot products over GF(65521), n=2^20 each, uint32 uniform "
                                   "residues on rotating buffers (2 GiB, larger than L2)",
                       "step": "one persistent batched launch over the 256 pairs"},
            "single_call_us": {"p50": lat[len(lat) // 2], "p10": lat[len(lat) // 10],
                               "p90": lat[(9 * len(lat)) // 10]},
            "same_gpu": {"perterm_ms": t_pt, "perterm_gmacs": gm(t_pt),
                         "speedup_over_perterm": t_pt / t_batch},
            "graph_of_256_single_dots": {"ms": t_graph, "gmacs": gm(t_graph),
                                          "gbs": 8 * macs / (t_graph / 1e3) / 1e9},
            "single_dot_2^27": {"ms": t_large, "gmacs": nl / (t_large / 1e3) / 1e9,
                                "gbs": 8.0 * nl / (t_large / 1e3) / 1e9,
                                "frac": 8.0 * nl / (t_large / 1e3) / 1e9 / peak,
                                "what": "one gfp_dot call over 2^27-element operands (1 GiB), "
                                        "back to back, L2-cold"},
            "roofline": with_read_peak(
                {"bound": "hbm", "achieved": 8 * macs / (t_batch / 1e3) / 1e9, "peak": peak,
                 "unit": "GB/s", "frac": 8 * macs / (t_batch / 1e3) / 1e9 / peak,
                 "kernel": "k_dot_batched",
                 "traffic": traffic_for("k_dot_batched", 8 * macs + 4.0 * nvec),
                 "peak_kind": f"{peak_kind} hbm_gbs"}),
            "gpu_launches": len(per),
        })
        plan.close()
    elif workload == "matvec":
        p, n, iters = 2147483647, args.mv_n, args.mv_iters
        A = torch.empty((n, n), dtype=torch.int32, device="cuda")
        g.gfp_fill_uniform(p, gi.BASE_SEED + 2, 0, A)
        x0 = torch.empty(n, dtype=torch.int32, device="cuda")
        g.gfp_fill_uniform(p, gi.BASE_SEED + 2, 1, x0)
        Y = torch.empty(iters * n, dtype=torch.int32, device="cuda")
        res = {}
        for name, rp in (("auto", 0), ("perterm", g.GFP_REPR_PERTERM)):
            ctx.set_repr(rp)
            with torch.cuda.stream(stream):
                for _ in range(2):
                    g.gfp_matvec_iterate(ctx, p, A, x0, Y, iters, stream)
                torch.cuda.synchronize()
                reps = 3 if name == "auto" else 1
                e0, e1 = _events(torch, 2)
                e0.record(stream)
                for _ in range(reps):
                    g.gfp_matvec_iterate(ctx, p, A, x0, Y, iters, stream)
                e1.record(stream)
            torch.cuda.synchronize()
            res[name] = e0.elapsed_time(e1) / reps
        ctx.set_repr(0)
        macs = float(iters) * n * n
        t = res["auto"]
        achieved = 4 * macs / (t / 1e3) / 1e9
        line.update({
            "value": macs / (t / 1e3) / 1e9, "ms_per_step": t,
            "config": {"workload": f"Wiedemann iteration over GF(2147483647): A {n}x{n} uint32 "
                                   f"uniform, x_(t+1) = A x_t for {iters} iterations in one CUDA graph",
                       "l2": "A is 4 GiB, larger than L2"},
            "roofline": with_read_peak(
                {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                 "frac": achieved / peak, "kernel": "k_matvec",
                 "traffic": traffic_for("k_matvec", 4.0 * n * n + 8.0 * n),
                 "peak_kind": f"{peak_kind} hbm_gbs"}),
            "same_gpu": {"perterm_ms": res["perterm"],
                         "perterm_gmacs": macs / (res["perterm"] / 1e3) / 1e9,
                         "speedup_over_perterm": res["perterm"] / t},
            "gpu_launches": iters,
        })
    elif workload in ("block", "csr"):
        p, m, k, nb = (args.block_p if workload == "block" else 65521), args.block_m, 16384, 64
        seed = gi.BASE_SEED + 3
        B = torch.empty((k, nb), dtype=torch.int32, device="cuda")
        g.gfp_fill_uniform(p, seed, 1, B)
        C = torch.empty((m, nb), dtype=torch.int32, device="cuda")
        macs = float(m) * k * nb

        def timed(fn, reps):
            with torch.cuda.stream(stream):
                for _ in range(2):
                    fn()
                torch.cuda.synchronize()
                e0, e1 = _events(torch, 2)
                e0.record(stream)
                for _ in range(reps):
                    fn()
                e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        if workload == "block":
            A = torch.empty((m, k), dtype=torch.int32, device="cuda")
            g.gfp_fill_uniform(p, seed, 0, A)
            passes = rns_passes(p, k)
            res = {}
            variants = [("f16tc", g.GFP_REPR_F16TC, max(10, args.steps // 4))]
            if not args.quick:
                variants += [("u64_block_cuda_core", g.GFP_REPR_U64_BLOCK, 5),
                             ("perterm_cuda_core", g.GFP_REPR_PERTERM, 2)]
            for name, rp, reps in variants:
                ctx.set_repr(rp)
                res[name] = timed(lambda: g.gfp_matmul_block(ctx, p, A, B, C, stream), reps)
            large = {}
            if not args.quick and p <= 65791:
                # a word-size prime beyond the digit range: residue passes on the tensor
                # cores against the CUDA-core kernel, same shape, inputs below 2^31 - 1
                pl = 2147483647
                Al = torch.empty((m, k), dtype=torch.int32, device="cuda")
                Bl = torch.empty((k, nb), dtype=torch.int32, device="cuda")
                g.gfp_fill_uniform(pl, seed, 4, Al)
                g.gfp_fill_uniform(pl, seed, 5, Bl)
                for name, rp, reps in (("f16tc_residue_passes", g.GFP_REPR_F16TC, max(5, args.steps // 10)),
                                       ("u64_carry_cuda_core", g.GFP_REPR_U64_CARRY, 3)):
                    ctx.set_repr(rp)
                    large[name] = timed(lambda: g.gfp_matmul_block(ctx, pl, Al, Bl, C, stream), reps)
            ctx.set_repr(0)
            # A prepared once (digit images in the layout the tensor cores read),
            # as for a resident matrix used by many products
            prep = g.BlockPrep(ctx, p, A)
            C2 = torch.empty((m, nb), dtype=torch.int32, device="cuda")
            t_prep = timed(lambda: prep.matmul(ctx, B, C2, stream), max(10, args.steps // 4))
            prep_bytes, prep_passes = prep.info()
            prep.close()
            g.gfp_matmul_block(ctx, p, A, B, C, stream)   # C was last written by other products
            torch.cuda.synchronize()
            if not torch.equal(C2, C):
                raise SystemExit("prepared and unprepared block products differ")
            if large:
                prep_l = g.BlockPrep(ctx, pl, Al)
                large["f16tc_prepared"] = timed(lambda: prep_l.matmul(ctx, Bl, C2, stream),
                                                max(5, args.steps // 10))
                prep_l.close()
            assert g.gfp_context_check(ctx) == g.GFP_OK
            t = res["f16tc"]
            # A is read once per residue pass; the residues (4 bytes each) are
            # written and read back once by the recombination
            abytes = passes * (4.0 * m * k + 4.0 * k * nb) + 4.0 * m * nb
            if passes > 1:
                abytes += 2 * passes * 4.0 * m * nb
            achieved = abytes / (t / 1e3) / 1e9
            tflops = passes * 4 * 2 * macs / (t / 1e3) / 1e12   # four digit products per multiply-add
            path = ("tensor-core path (balanced fp16 digits)" if passes == 1 else
                    f"tensor-core path through {passes} residue passes (balanced fp16 digits)")
            line.update({
                "value": macs / (t / 1e3) / 1e9, "ms_per_step": t,
                "config": {"workload": f"block product over GF({p}): A {m}x{k} times B {k}x{nb}, "
                                       f"uint32 uniform residues, {path}",
                           "l2": "A is larger than L2" if m * k * 4 > (129 << 20) else "A fits L2"},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "kernel": "k_block_tc (+k_block_prep_b, k_block_finish)",
                             "traffic": traffic_for("k_block_tc", abytes) if passes == 1 else None,
                             "peak_kind": f"{peak_kind} hbm_gbs",
                             "tensor_tflops_fp16": tflops},
                "same_gpu": {n: {"ms": v, "gmacs": macs / (v / 1e3) / 1e9} for n, v in res.items()},
                "gpu_launches": 3 if passes == 1 else 3 * passes + 1,
            })
            ppasses = rns_passes(p, k, 65536)
            ptf = ppasses * 4 * 2 * macs / (t_prep / 1e3) / 1e12
            pk = peaks() or {}
            tpk, tpk_kind = ((float(pk["bf16_tflops"]), "measured bf16_tflops (burst)")
                             if pk.get("bf16_tflops") else (1900.0, "fallback bf16 dense"))
            pbytes = prep_bytes + ppasses * 4.0 * k * nb + 4.0 * m * nb
            if ppasses > 1:
                pbytes += 2 * ppasses * 4.0 * m * nb
            pach = pbytes / (t_prep / 1e3) / 1e9
            line["prepared"] = {
                "ms": t_prep, "gmacs": macs / (t_prep / 1e3) / 1e9, "passes": prep_passes,
                "what": "A prepared once into 8-bit digit planes (2 bytes per entry per pass), "
                        "then one product per call (B digits, tensor-core kernel widening "
                        "A's digits in shared memory, partial sums to C)",
                "roofline": {"bound": "tensor", "achieved": ptf, "peak": tpk, "unit": "TFLOP/s",
                             "frac": ptf / tpk, "kernel": "k_block_tc (prepared A) + k_block_prep_b + k_block_finish",
                             "peak_kind": tpk_kind,
                             "what": "fp16 digit products (4 per multiply-add, 2 flops each) against "
                                     "the measured bf16 dense rate (fp16 runs at the same rate)",
                             "hbm": with_read_peak({"bound": "hbm", "achieved": pach, "peak": peak,
                                                    "unit": "GB/s", "frac": pach / peak,
                                                    "traffic": (traffic_for("k_block_tc_prepared", pbytes)
                                                                if ppasses == 1 else None),
                                                    "peak_kind": f"{peak_kind} hbm_gbs"})}}
            if large:
                line["p_2^31-1"] = {n: {"ms": v, "gmacs": macs / (v / 1e3) / 1e9} for n, v in large.items()}
                del Al, Bl
        else:
            row_ptr, col, val = gi.csr_pattern(m, k, 0.01, p, seed)
            rp_d = torch.from_numpy(row_ptr.view(np.int32)).cuda()
            col_d = torch.from_numpy(col.view(np.int32)).cuda()
            val_d = torch.from_numpy(val.view(np.int32)).cuda()
            nnz = int(row_ptr[-1])
            # the CSR arrays and B (26 MB) fit L2: each timed product starts from a
            # flushed L2 (256 MiB written on the same stream, outside the events)
            flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
            reps = max(10, args.steps // 4)
            with torch.cuda.stream(stream):
                for _ in range(2):
                    g.gfp_matmul_block_csr(ctx, p, k, rp_d, col_d, val_d, B, C, stream)
                ev = _events(torch, 2 * reps)
                for i in range(reps):
                    flush.fill_(i & 0xFF)
                    ev[2 * i].record(stream)
                    g.gfp_matmul_block_csr(ctx, p, k, rp_d, col_d, val_d, B, C, stream)
                    ev[2 * i + 1].record(stream)
            torch.cuda.synchronize()
            t = sum(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(reps)) / reps
            del flush
            cmacs = float(nnz) * nb
            abytes = 8.0 * nnz + 4.0 * (m + 1) + 4.0 * k * nb + 4.0 * m * nb
            # gathers from L2: one B row (nb stored elements) per nonzero
            csr_kernel, bpe = "k_block_csr_wide", 4
            gbytes = float(nnz) * nb * bpe
            l2p = own_peaks()["read_l2"]
            line.update({
                "value": cmacs / (t / 1e3) / 1e9, "ms_per_step": t,
                "config": {"workload": f"sparse-row block product over GF(65521): CSR A {m}x{k} with "
                                       f"Bernoulli(0.01) rows ({nnz} nonzeros) times B {k}x{nb}",
                           "nnz": nnz,
                           "l2": "flushed before each timed product (inputs 26 MB fit L2)"},
                "roofline": {"bound": "hbm", "achieved": abytes / (t / 1e3) / 1e9, "peak": peak,
                             "unit": "GB/s", "frac": abytes / (t / 1e3) / 1e9 / peak,
                             "kernel": csr_kernel,
                             "traffic": traffic_for(csr_kernel, abytes),
                             "peak_kind": f"{peak_kind} hbm_gbs",
                             "note": "B is re-read from L2 per nonzero; HBM bytes count it once",
                             "l2": {"bound": "l2", "achieved": gbytes / (t / 1e3) / 1e9,
                                    "peak": l2p["peak"], "unit": "GB/s",
                                    "frac": gbytes / (t / 1e3) / 1e9 / l2p["peak"],
                                    "bytes_per_launch": gbytes,
                                    "what": f"B-row gathers: {bpe} bytes per stored B element, "
                                            "nb elements per nonzero",
                                    "source": l2p["source"]}},
                "gpu_launches": 1,
            })
    torch.cuda.synchronize()
    return line


# ---------------------------------------------------------------------------
# serving: Poisson stream of mixed jobs through the continuous-batching server
# ---------------------------------------------------------------------------

def run_serve(args):
    import torch
    from paper_cs_0404008_gb300 import gfpdot as g
    torch.cuda.set_device(0)
    g.load()
    print(json.dumps(measure_serve(args, g)), flush=True)


def measure_serve(args, g):
    import threading as th

    seed = gi.BASE_SEED + 5
    srv = g.Server(device=0, mem_budget=16 << 30, n_streams=8, batch_window_us=50,
                   max_inflight=256, block_sm_percent=args.serve_block_sms)
    # resident matrix pools (registered once): sides log-uniform
    pools = {kind: [(srv.register_matrix(p, side, side, seed=mseed), p, side, mseed)
                    for p, side, mseed in specs]
             for kind, specs in gi.serve_pool_specs(seed).items()}
    if args.serve_prepared:
        # block matrices are resident: build their tensor-core digit images once
        for h, _, _, _ in pools[2]:
            srv.prepare_matrix(h)
    reqs = gi.serve_requests(args.requests, seed)

    def submit(r):
        k, p, n, mi, sd = r
        if k == 0:
            return srv.submit(g.GFP_JOB_DOT, p, n=n, seed=sd)
        h, mp, side, _ = pools[k][mi]
        if k == 1:
            return srv.submit(g.GFP_JOB_MATVEC, mp, matrix=h, seed=sd)
        return srv.submit(g.GFP_JOB_BLOCK, mp, matrix=h, nb=64, seed=sd)

    def macs(r):
        k, p, n, mi, sd = r
        if k == 0:
            return float(n)
        side = pools[k][mi][2]
        return float(side) * side * (64 if k == 2 else 1)

    # warm-up and capacity: a closed burst
    burst = reqs[:min(2000, len(reqs))]
    for r in burst[:50]:
        st, _ = srv.wait(submit(r))
    t0 = time.perf_counter()
    tks = [submit(r) for r in burst]
    for t in tks:
        st, res = srv.wait(t)
        srv.release(t)
    cap = len(burst) / (time.perf_counter() - t0)
    lam = args.load * cap

    # open-loop Poisson arrivals
    gaps = -np.log1p(-gi.unit_doubles(seed, 30, len(reqs))) / lam
    sample = set(range(0, len(reqs), 100))           # 1% checked against direct calls
    results = [None] * len(reqs)
    outs = {}
    tickets = [None] * len(reqs)
    ready = th.Semaphore(0)

    def collector():
        for i in range(len(reqs)):
            ready.acquire()
            st, res = srv.wait(tickets[i], 600_000_000)
            results[i] = (st, res.status, res.value, res.t_submit_ns, res.t_done_ns, res.batch,
                          res.t_admit_ns, res.t_start_ns)
            if i in sample and res.status == g.GFP_OK and reqs[i][0] != 0:
                outs[i] = srv.result_copy(tickets[i], res.out_elems)
            srv.release(tickets[i])

    col = th.Thread(target=collector, daemon=True)
    col.start()
    stats0 = srv.stats()
    t_start = time.perf_counter()
    t_next = t_start
    for i, r in enumerate(reqs):
        t_next += gaps[i]
        while True:
            d = t_next - time.perf_counter()
            if d <= 0:
                break
            if d > 2e-4:
                time.sleep(d - 1e-4)
        tickets[i] = submit(r)
        ready.release()
    col.join()
    wall = time.perf_counter() - t_start
    stats1 = srv.stats()
    lat = np.array([(x[4] - x[3]) / 1e6 for x in results])
    # latency by job kind (and, for block jobs, by whether the tensor-core path applies)
    by_kind = {}
    kinds = np.array([r[0] for r in reqs])
    # where the time goes: queued (submit -> admit), launching (admit -> launch
    # calls returned), on the device until the dispatcher saw it done
    queued = np.array([(x[6] - x[3]) / 1e6 for x in results])
    launching = np.array([(x[7] - x[6]) / 1e6 for x in results])
    running = np.array([(x[4] - x[7]) / 1e6 for x in results])
    for kname, kid in (("dot", 0), ("matvec", 1), ("block", 2)):
        sel = kinds == kid
        if sel.any():
            by_kind[kname] = {"count": int(sel.sum()), "p50_ms": float(np.percentile(lat[sel], 50)),
                              "p99_ms": float(np.percentile(lat[sel], 99)),
                              "max_ms": float(lat[sel].max()),
                              "stages_p50_ms": {"queued": float(np.percentile(queued[sel], 50)),
                                                "launching": float(np.percentile(launching[sel], 50)),
                                                "running": float(np.percentile(running[sel], 50))},
                              "stages_p99_ms": {"queued": float(np.percentile(queued[sel], 99)),
                                                "launching": float(np.percentile(launching[sel], 99)),
                                                "running": float(np.percentile(running[sel], 99))}}
    top = np.argsort(lat)[-max(1, len(lat) // 100):]
    by_kind["slowest_1pct_kinds"] = {kname: int((kinds[top] == kid).sum())
                                     for kname, kid in (("dot", 0), ("matvec", 1), ("block", 2))}
    ok = all(x[0] == g.GFP_OK and x[1] == g.GFP_OK for x in results)
    total_macs = sum(macs(r) for r in reqs)

    # verification: sampled results against the library's direct entry points on
    # the same operands regenerated on the device from their seeds (the server's
    # scheduling, batching and memory handling are what is checked here; the
    # arithmetic itself is checked against the oracle by the tests), and a replay
    # of some jobs alone
    import torch
    vctx = g.Context(0)
    bad = 0
    checked = 0
    for i in sorted(sample):
        k, p, n, mi, sd = reqs[i]
        if k == 0:
            xd = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
            yd = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
            g.gfp_fill_uniform(p, sd, 0, xd, n)
            g.gfp_fill_uniform(p, sd, 1, yd, n)
            od = torch.empty(1, dtype=torch.int32, device="cuda")
            g.gfp_dot(vctx, p, xd[:n], yd[:n], od)
            torch.cuda.synchronize()
            bad += int(results[i][2] != int(od.cpu().numpy().view(np.uint32)[0]))
            checked += 1
        else:
            h, mp, side, mseed = pools[k][mi]
            Ad = torch.empty((side, side), dtype=torch.int32, device="cuda")
            g.gfp_fill_uniform(mp, mseed, 0, Ad)
            if k == 1:
                vd = torch.empty(side, dtype=torch.int32, device="cuda")
                g.gfp_fill_uniform(mp, sd, 0, vd)
                wd = torch.empty(side, dtype=torch.int32, device="cuda")
                g.gfp_matvec(vctx, mp, Ad, vd, wd)
            else:
                vd = torch.empty((side, 64), dtype=torch.int32, device="cuda")
                g.gfp_fill_uniform(mp, sd, 0, vd)
                wd = torch.empty((side, 64), dtype=torch.int32, device="cuda")
                g.gfp_matmul_block(vctx, mp, Ad, vd, wd)
            torch.cuda.synchronize()
            want = wd.cpu().numpy().view(np.uint32).ravel()
            bad += int(not np.array_equal(outs[i], want))
            checked += 1
            del Ad, vd, wd
    vctx.close()
    replay_bad = 0
    for i in sorted(sample)[:20]:
        t = submit(reqs[i])
        st, res = srv.wait(t)
        if reqs[i][0] == 0:
            replay_bad += int(res.value != results[i][2])
        elif i in outs:
            replay_bad += int(not np.array_equal(srv.result_copy(t, res.out_elems), outs[i]))
        srv.release(t)
    srv.close()
    line = {
        "metric": METRIC, "value": total_macs / wall / 1e9, "unit": UNIT, "n_gpus": 1,
        "steps": 1, "warmup": 50, "ms_per_step": wall * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"serving: Poisson stream of {len(reqs)} requests, 70% dot "
                               "(n log-uniform [2^10,2^22]), 25% matvec (16 resident square "
                               "matrices, side log-uniform [2^10,2^14]), 5% block (16 resident "
                               "m=k log-uniform [2^10,2^13], nb=64), p uniform over {65521, "
                               "67108859, 4294967291}, server-generated operands",
                   "load": args.load,
                   "block_sm_percent": args.serve_block_sms or 100,
                   "block_matrices": ("prepared at registration (digit images)" if args.serve_prepared
                                      else "converted on every product"),
                   "checks": "1% of the results recomputed by direct library calls on the same "
                             "operands regenerated on the device; 20 jobs replayed alone"},
        "serve": {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                  "mean_ms": float(lat.mean()), "capacity_jobs_per_s": cap,
                  "lambda_jobs_per_s": lam, "achieved_jobs_per_s": len(reqs) / wall,
                  "all_ok": bool(ok), "verified": checked, "verify_mismatches": bad,
                  "replayed_alone": min(20, len(sample)), "replay_mismatches": replay_bad,
                  "admission_stalls": stats1["admission_stalls"] - stats0["admission_stalls"],
                  "dot_launches": stats1["dot_launches"] - stats0["dot_launches"],
                  "mean_dot_batch": float(np.mean([x[5] for x, r in zip(results, reqs) if r[0] == 0])),
                  "mem_peak_bytes": stats1["mem_peak"],
                  "by_kind": by_kind},
        "gpu_launches": stats1["kernel_launches"] - stats0["kernel_launches"],
    }
    return line


# ---------------------------------------------------------------------------
# Host representation sweep (the paper's CPU comparison, Section 3)
# ---------------------------------------------------------------------------

SWEEP_SEED = gi.BASE_SEED + 6
SWEEP_N = 512   # the vector length of the paper's comparison
SWEEP_PAPER_PRIMES_32 = [2887, 2897, 2903, 32749, 40009, 40499, 46337, 65521]
SWEEP_PAPER_PRIMES_64 = [94906249, 2147483647, 3037000493, 4294967291]


def rns_passes(p: int, k: int, direct_max: int = 65791) -> int:
    """Tensor-core passes of a k-deep block product over GF(p): one for
    p <= direct_max (65791 for uint32 A, 65536 for a prepared A), else the
    number of largest primes <= 65536 whose product exceeds k (p-1)^2 (the
    residue moduli the library picks)."""
    if p <= direct_max:
        return 1
    bound, prod, count, c = k * (p - 1) ** 2, 1, 0, 65536
    while prod <= bound:
        while not is_prime(c):
            c -= 1
        prod *= c
        count += 1
        c -= 1
    return count


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (bases 2..41)."""
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41)
    for q in small:
        if n % q == 0:
            return n == q
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in small:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def sweep_primes(lo: int, hi: int, count: int):
    """The largest prime at or below each of `count` log-spaced points of [lo, hi]."""
    out = set()
    for t in np.linspace(np.log(lo), np.log(hi), count):
        q = int(round(float(np.exp(t))))
        q = min(max(q, lo), hi)
        while q >= 2 and not is_prime(q):
            q -= 1
        if q >= 2:
            out.add(q)
    return sorted(out)


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_cpu_sweep(args):
    """Times each host representation of libgfpsweep on 512-long vectors (one
    thread) for primes spread over its domain, as the paper's Figures 5-8 do
    on older CPUs; prints one JSON line (Mop/s = million multiply-adds/s)."""
    import platform

    from paper_cs_0404008_gb300 import sweep
    rank, _, _ = dist_env()
    if rank != 0:
        return
    p32 = sorted(set(sweep_primes(3, 65521, args.sweep_points)) | set(SWEEP_PAPER_PRIMES_32))
    p64 = sorted(set(sweep_primes(3, 4294967291, args.sweep_points)) | set(SWEEP_PAPER_PRIMES_64))
    results, residues = {}, {}
    t_start = time.perf_counter()
    for v in sweep.VARIANTS:
        rows = []
        for p in (p32 if v in sweep.WORD32 else p64):
            if not sweep.supported(v, p):
                continue
            x = gi.uniform(p, SWEEP_N, SWEEP_SEED, 0)
            y = gi.uniform(p, SWEEP_N, SWEEP_SEED, 1)
            sec, r = sweep.time(v, p, x, y, 200)
            reps = max(200, int(200 * 2e-3 / max(sec, 1e-9)))   # about 2 ms per trial
            best = min(sweep.time(v, p, x, y, reps)[0] for _ in range(3))
            rows.append([p, round(SWEEP_N * reps / best / 1e6, 1)])
            residues.setdefault(p, set()).add(r)
        results[v] = rows
    consistent = all(len(s) == 1 for s in residues.values())
    line = {"metric": "host dot-product representation sweep (paper Section 3, Figures 5-8)",
            "unit": "Mop/s (million multiply-adds per second)", "n": SWEEP_N, "threads": 1,
            "host": platform.machine(), "cpu": cpu_model(), "data": "synthetic",
            "inputs": "uint32 residues uniform in [0,p), counter-based generator",
            "variants_agree": consistent, "seconds": round(time.perf_counter() - t_start, 1),
            "block_lengths": {v: {str(p): sweep.block(v, p) for p, _ in rows}
                              for v, rows in results.items()},
            "results": results}
    print(json.dumps(line), flush=True)
    if args.sweep_table:
        with open(args.sweep_table, "w") as f:
            for title, fam, ps in (("32-bit words", sweep.WORD32, p32), ("64-bit words and doubles", sweep.WORD64, p64)):
                f.write(f"### {title} (Mop/s, n = {SWEEP_N}, one thread, {line['host']} {line['cpu']})\n\n")
                f.write("| p | " + " | ".join(fam) + " |\n|" + "---|" * (len(fam) + 1) + "\n")
                table = {v: dict((q, m) for q, m in results[v]) for v in fam}
                for p in ps:
                    f.write(f"| {p} | " + " | ".join(str(table[v].get(p, "")) for v in fam) + " |\n")
                f.write("\n")
    if not consistent:
        sys.exit(1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gfpdot", choices=["gfpdot", "reference"])
    ap.add_argument("--quick", action="store_true", help="skip the per-representation comparisons")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-also", action="store_true", help="skip the other workloads")
    ap.add_argument("--no-tune", action="store_true", help="built-in representation rules")
    ap.add_argument("--no-clocks", action="store_true", help="skip the clock-sampling load phase")
    ap.add_argument("--pairs", type=int, default=COUNT, help="batch size (smaller for profiling)")
    ap.add_argument("--workload", default="batched",
                    choices=["batched", "dot", "matvec", "block", "csr", "gfq", "serve", "cpu_sweep"])
    ap.add_argument("--sweep-points", type=int, default=24,
                    help="cpu_sweep: log-spaced primes per word size")
    ap.add_argument("--sweep-table", default=None, help="cpu_sweep: also write a markdown table")
    ap.add_argument("--requests", type=int, default=100000, help="serve: Poisson requests")
    ap.add_argument("--load", type=float, default=0.7, help="serve: arrival rate / capacity")
    ap.add_argument("--serve-block-sms", type=int, default=50,
                    help="serve: percent of the SMs a block job's kernel may occupy (0: all)")
    ap.add_argument("--serve-prepared", type=int, default=1,
                    help="serve: prepare the block matrices' digit images at registration (1) or not (0)")
    ap.add_argument("--block-m", type=int, default=16384, help="block workload rows (profiling)")
    ap.add_argument("--gfq-fields", default=None,
                    help="gfq workload: comma-separated fields p^k (default 2^8,3^10,65521^1)")
    ap.add_argument("--block-p", type=int, default=65521,
                    help="block workload prime; above 65791 the product runs through residue passes")
    ap.add_argument("--mv-n", type=int, default=32768, help="matvec side (profiling)")
    ap.add_argument("--mv-iters", type=int, default=64, help="matvec iterations (profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_gpu(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "cpu_sweep":
        run_cpu_sweep(args)
    else:
        run_secondary(args)


if __name__ == "__main__":
    main()
