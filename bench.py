"""Benchmark of the lattice Burgers functional-integral hot path on GB300.

One step = one pass of the whole path over the paper-shaped workload: a 10x2
lattice (20 dimensions, nu = D = a = tau = 1), the box [-5,5]^20 bisected
along coordinates 0..9 into 1024 subvolumes, 2^20 Philox4x32-10 points per
subvolume (2^30 samples), evaluated in FP64: points, action, shifted
weights, products, per-subvolume reduction and the FP64 merge into Z, C(r)
and their errors.  The metric is samples per second.

With N ranks (torchrun, one GPU each) the box is bisected into 1024 N
subvolumes and rank r integrates subvolumes [1024 r, 1024 (r + 1)) (weak
scaling); the per-subvolume records are then gathered to rank 0, which merges
them (the only exchange of the method).

--impl reference times the plain FP64 CPU oracle on a bounded sample of the
same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SAMPLES_PER_SUB = 1 << 20
NSUB_PER_RANK = 1024
NX, NT = 10, 2
D = NX * NT
R = NX // 2 + 1
K = 2 + 3 * R
FP32_SAMPLES_PER_SUB = 1 << 24      # the 2^34-point FP32 form of the same job

# Peaks, from GB300's unit counts (152 SMs; per SM and clock: 128 FP32/INT
# lanes, i.e. 4 warp-instructions, and 2 FP64 FMA lanes, the figures ncu
# reports as peak_sustained for ffma and dfma) at the 2070 MHz maximum clock.
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
ISSUE_PEAK_OPS = 128 * SM_COUNT * SM_MAX_MHZ * 1e6   # thread-instructions/s (FP32/INT lanes)
FP64_PEAK_OPS = 2 * SM_COUNT * SM_MAX_MHZ * 1e6      # FP64 operations/s


# DRAM traffic of the FP64 10x2 integrand launch comes from a committed ncu
# summary that records the hash of the kernel sources it was measured on; the
# bench reports it only while those sources are unchanged (else null).
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "integrand_f64_10x2_traffic.txt")
KERNEL_SOURCES = ["bfi_device.cuh", "bfi_kernels.h", "integrand_kernels.cuh", "shapes_table.cuh", "shapes_small.cu"]


def code_only(text):
    """Source text without comments and with whitespace runs collapsed: what a
    change to the compiled kernel would change."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_sources_sha256(read=None):
    """SHA-256 of the kernel sources' code (comments and layout ignored);
    'read' (name -> text) defaults to the files in the tree."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        if read is None:
            with open(os.path.join(ROOT, "paper_1803_07560_gb300", "csrc", name)) as f:
                text = f.read()
        else:
            text = read(name)
        h.update(code_only(text).encode())
    return h.hexdigest()


def measured_traffic(chunk_samples=None):
    """(DRAM bytes read + written per full-size launch, note): the value of the
    committed ncu summary when its kernel-source hash matches and it was taken
    with the chunk size the timed plan uses, else None."""
    try:
        fields = dict(line.split(":", 1) for line in open(TRAFFIC_FILE) if ":" in line and not line.startswith("#"))
    except OSError:
        return None, "no committed traffic summary"
    sha = fields.get("kernel_sources_sha256", "").strip()
    if sha != kernel_sources_sha256():
        return None, "kernel sources changed since the ncu traffic capture"
    if chunk_samples is not None and fields.get("chunk_samples", "").strip() != str(chunk_samples):
        return None, "chunk size changed since the ncu traffic capture"
    return int(fields["dram_bytes_per_launch"].strip()), "ncu dram__bytes_read.sum + dram__bytes_write.sum, " \
        "one full-size launch (" + os.path.relpath(TRAFFIC_FILE, ROOT) + ")"


def screen_ops(nx, nt):
    """Per sample the full FP32 screen examines: Philox words, FP32 point, FP32 action."""
    d = nx * nt
    return ((d + 3) // 4) * 10 * 4 + 2 * d + 8 * d


def partial_ops(nx, nt):
    """Per sample, stage 1 of the two-stage screen: the first BP of the ceil(d/4) Philox blocks (BP about 0.6
    of them), the FP32 points of the MC sites they complete, the residuals of sites 1 .. MC-2."""
    d = nx * nt
    bp = (3 * ((d + 3) // 4) + 4) // 5
    mc = min((4 * bp) // nt, nx)
    return bp * 10 * 4 + 2 * mc * nt + 8 * (mc - 2) * nt


def eval_ops_fp64(nx, nt):
    """Per evaluated sample (FP64 mode): (FP64 operations, integer operations)."""
    d, r = nx * nt, nx // 2 + 1
    k = 2 + 3 * r
    return 2 * d + 8 * d + d * r + 1 + 2 * k, ((d + 3) // 4) * 10 * 4


def eval_ops_fp32(nx, nt):
    """Per evaluated sample (FP32 mode): products, weight, compensated sums."""
    d, r = nx * nt, nx // 2 + 1
    k = 2 + 3 * r
    return d * r + 2 + 4 * k


def rest_ops(nx, nt):
    """Per survivor of stage 1 with Nt = 2: the rest of the action without the sites stage 1 summed (blocks 0
    and BP-1 .. again, their points, the residuals of sites 0 and MC-1 .. Nx-1); other shapes screen in full."""
    d = nx * nt
    nq = (d + 3) // 4
    bp = (3 * nq + 4) // 5
    mc = min((4 * bp) // nt, nx)
    if nt != 2 or bp < 2:
        return screen_ops(nx, nt)
    blocks = 2 + (nq - bp)
    return blocks * 10 * 4 + 2 * 4 * blocks + 8 * (nx - mc + 2) * nt


def screen_work(work, nx, nt):
    """FP32/INT operations of the screen in one launch, from the counted work
    (a dict with samples, stage1, survivors, full_screen): stage 1 for the
    samples of two-stage chunks, the full screen for the others, and stage 2
    (the rest of the action, or the full screen) for stage 1's survivors."""
    rest = rest_ops(nx, nt) if work.get("rest_screen", 1) else screen_ops(nx, nt)
    return (work["stage1"] * partial_ops(nx, nt) + work["full_screen"] * screen_ops(nx, nt) +
            work["survivors"] * rest)


def one_stage_work(n, n_eval=0):
    """The work dict of a launch that screened every sample in one stage."""
    return {"samples": n, "stage1": 0, "survivors": 0, "full_screen": n, "evaluated": n_eval, "rest_screen": 1}


def roofline(work, kern_ms, precision, nx=10, nt=2):
    """Algorithmic work of one launch (the counted work of bfi_plan_get_work)
    against the binding resource."""
    t = kern_ms * 1e-3
    n, n_eval = work["samples"], work["evaluated"]
    w_screen = screen_work(work, nx, nt)
    if precision == "fp64":
        dp, integer = eval_ops_fp64(nx, nt)
        w_issue = w_screen + n_eval * integer
        w_dp = n_eval * dp
    else:
        w_issue = w_screen + n_eval * eval_ops_fp32(nx, nt)
        w_dp = 0
    t_issue, t_dp = w_issue / ISSUE_PEAK_OPS, w_dp / FP64_PEAK_OPS
    if t_issue >= t_dp:
        bound, achieved, peak = "alu", w_issue / t, ISSUE_PEAK_OPS
    else:
        bound, achieved, peak = "alu-fp64", w_dp / t, FP64_PEAK_OPS
    return {"bound": "alu", "resource": "FP32/INT issue" if bound == "alu" else "FP64 pipe",
            "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gop/s", "frac": achieved / peak,
            "traffic": None, "kernel_ms": kern_ms, "samples": n, "evaluated": n_eval,
            "issue_frac": w_issue / t / ISSUE_PEAK_OPS, "fp64_frac": w_dp / t / FP64_PEAK_OPS,
            "screen_ops_per_sample": screen_ops(nx, nt), "partial_ops_per_sample": partial_ops(nx, nt),
            "survivor_ops": rest_ops(nx, nt) if work.get("rest_screen", 1) else screen_ops(nx, nt),
            "stage1_samples": work["stage1"], "survivors": work["survivors"],
            "full_screened": work["full_screen"],
            "peak_source": "unit counts x 2070 MHz: 128 FP32/INT and 2 FP64 lanes per SM, 152 SMs"}


def rank_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs, every
    100 ms with a timestamp; stop(region) keeps the samples inside the timed
    region's host wall-clock interval.  The raw samples go to $BFI_CLOCKS_DIR
    (default: the system temporary directory) as clocks_<pid>.csv."""

    def __init__(self, gpu_index: int):
        import tempfile
        self.proc = None
        self.path = os.path.join(os.environ.get("BFI_CLOCKS_DIR") or tempfile.gettempdir(),
                                 f"clocks_{os.getpid()}.csv")
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def wait_first(self, timeout_s: float = 5.0):
        """Returns once the sampler has written its first sample (or after
        timeout_s), so that sampling is running when the timed region starts."""
        t_end = time.time() + timeout_s
        while self.proc is not None and time.time() < t_end:
            self.fh.flush()
            try:
                if any(len(line.split(",")) >= 10 for line in open(self.path)):
                    return
            except OSError:
                return
            time.sleep(0.02)

    def stop(self, region=None):
        """Median SM clock, the maximum, and the throttle reasons seen, over the
        samples inside region = (t0, t1) host wall-clock seconds (all samples
        when none falls inside, with in_region false)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        return parse_clock_samples(open(self.path).read().splitlines(), region)


def parse_clock_samples(lines, region=None):
    """The clocks record from nvidia-smi CSV lines (timestamp, index, SM clock,
    max SM clock, power, reasons active, hw_slowdown, hw_thermal_slowdown,
    sw_thermal_slowdown, sw_power_cap)."""
    import datetime
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    rows = []
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 10:
            continue
        try:
            ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            rows.append((ts, float(f[2]), float(f[3]), [n for n, v in zip(names, f[6:10]) if v.lower() == "active"]))
        except ValueError:
            continue
    inside = [r for r in rows if region is not None and region[0] <= r[0] <= region[1]]
    use = inside if inside else rows
    return {"sm_mhz": statistics.median(r[1] for r in use) if use else None,
            "sm_max_mhz": max(r[2] for r in use) if use else None,
            "reasons": sorted({n for r in use for n in r[3]}),
            "samples": len(inside), "samples_total": len(rows), "in_region": bool(inside)}


def cpu_sample_job():
    """Bounded sample for the CPU oracle: every 32nd subvolume of the
    10x2 job (32 subvolumes, their own sub_ids) at the full 2^20 points."""
    import workloads
    job = workloads.paper_10x2(SAMPLES_PER_SUB)
    return job.subset(np.arange(0, 1024, 32))


def time_oracle(steps=1):
    import oracle
    job = cpu_sample_job()
    lat = oracle.lattice(job.nx, job.nt)
    cores = os.cpu_count() or 1
    oracle.build()
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle.integrate(lat, job.lo, job.hi, job.samples, job.seed, job.job_id, sub_id=job.sub_id,
                         nthreads=cores)
        times.append(time.perf_counter() - t0)
    return job.total_samples, times, cores


def run_reference(args):
    rank, _, world = rank_info()
    if rank != 0:
        return
    import oracle
    oracle.build()
    samples, times, cores = time_oracle(args.warmup + args.steps)
    t = times[args.warmup:] if len(times) > args.warmup else times
    sec = sum(t) / len(t)
    value = samples / sec
    sample_desc = ("32 of the 1024 subvolumes (every 32nd) x 2^20 points of the 10x2 job, "
                   "FP64 oracle, OpenMP over subvolumes")
    print(json.dumps({
        "impl": "reference", "metric": "samples/s", "value": value, "unit": "samples/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(world),
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": cores, "kind": "oracle",
                         "sample": sample_desc},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def workload_config(world, per_sub=SAMPLES_PER_SUB):
    d = NX * NT
    return {"workload": f"{NX}x{NT} lattice (d={d}), nu=D=a=tau=1, box [-5,5]^{d} bisected along coords "
                        f"0..{min(10, d) - 1} into 1024 subvolumes per GPU, 2^{int(math.log2(per_sub))} "
                        "Philox4x32-10 points each (seed 2), FP64",
            "model": None, "global_batch": world * NSUB_PER_RANK * per_sub,
            "subvolumes_per_gpu": NSUB_PER_RANK, "samples_per_subvolume": per_sub,
            "parallelism": f"subvolume shards x{world}",
            "l2": "flushed between timed steps (256 MiB write, outside the timed intervals)"}


def make_job(rank, world, samples_per_sub):
    import workloads
    k = 10 + int(round(math.log2(world)))
    lo, hi = workloads.bisected_boxes(D, k)   # 2^k boxes for any d (the bisection cycles when d < k)
    assert lo.shape[0] == NSUB_PER_RANK * world
    sl = slice(rank * NSUB_PER_RANK, (rank + 1) * NSUB_PER_RANK)
    return workloads.Job(NX, NT, lo[sl], hi[sl], np.full(NSUB_PER_RANK, samples_per_sub, dtype=np.uint64),
                         seed=2, sub_id=np.arange(sl.start, sl.stop, dtype=np.uint32))


def timed_steps(plan, lo, hi, sid, job, steps, warmup, flush_buf, dist, stream, region=None):
    """Per-step CUDA events on the launch stream; the L2 flush sits between
    steps.  region (a list) receives the timed region's host wall-clock
    interval."""
    import torch
    for _ in range(warmup):
        plan.execute(lo, hi, job.seed, job.job_id, sub_id=sid, stream=stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    plan.set_timing(True)
    total_ms, kern_ms = 0.0, 0.0
    slots = totals = None
    t0 = time.time()
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush_buf.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        slots, totals = plan.execute(lo, hi, job.seed, job.job_id, sub_id=sid, stream=stream)
        ev1.record(stream)
        ev1.synchronize()
        total_ms += ev0.elapsed_time(ev1)
        kern_ms += plan.timing()[0]
    plan.set_timing(False)
    torch.cuda.synchronize()
    if region is not None:
        region.extend([t0, time.time()])
    if dist is not None:
        dist.barrier()
    return total_ms / steps, kern_ms / steps, slots, totals, plan.work().as_dict()


def run_bfi(args):
    import torch
    rank, local_rank, world = rank_info()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=dev)
        dist = tdist
    import __graft_entry__
    __graft_entry__.build()
    import paper_1803_07560_gb300 as bfi

    stream = torch.cuda.Stream(dev)
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    lat = bfi.lattice(NX, NT)

    # ---- headline: FP64, 2^20 points per subvolume ----
    job = make_job(rank, world, 1 << args.samples_log2)
    lo = torch.tensor(job.lo, device=dev)
    hi = torch.tensor(job.hi, device=dev)
    sid = torch.tensor(job.sub_id.astype(np.int32), device=dev)
    plan = bfi.Plan(lat, job.samples, bfi.FP64, device=local_rank)
    info = plan.info()
    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.wait_first()
    region = []
    ms, kern_ms, slots, totals, work = timed_steps(plan, lo, hi, sid, job, args.steps, args.warmup, flush_buf, dist,
                                                   stream, region)
    clocks = sampler.stop(region) if sampler else None

    # the exchange: gather every rank's subvolume records, merge in FP64
    from paper_1803_07560_gb300 import shard
    if dist is not None:
        merged = shard.merge_across_ranks(NX, slots)
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    else:
        merged = bfi.merge_host(NX, slots.cpu().numpy())

    samples_all = world * job.total_samples
    value = samples_all / (ms * 1e-3)
    roof = roofline(work, kern_ms, "fp64", NX, NT)
    roof["kernel"] = f"hint + integrand FP64 <{NX},{NT}>"
    if (NX, NT) == (10, 2) and args.samples_log2 == 20:
        roof["traffic"], roof["traffic_source"] = measured_traffic(info.chunk_samples)

    # ---- FP32 form of the same job with 2^24 points per subvolume ----
    fp32 = None
    if not args.skip_fp32:
        job32 = make_job(rank, world, 1 << (args.samples_log2 + 4))
        plan32 = bfi.Plan(lat, job32.samples, bfi.FP32, device=local_rank)
        ms32, kern32, slots32, tot32, work32 = timed_steps(plan32, lo, hi, sid, job32, max(1, args.steps // 2),
                                                           max(1, args.warmup // 2), flush_buf, dist, stream)
        bound32 = bfi.error_bound(lat, bfi.FP32, slots32, 5.0)
        roof32 = roofline(work32, kern32, "fp32", NX, NT)
        roof32["kernel"] = f"hint + integrand FP32 <{NX},{NT}>"
        plan32.close()
        # the same 2^34-point job in FP64 mode (its own FP64 points): the FP32
        # result's total difference, arithmetic plus point rounding
        plan64 = bfi.Plan(lat, job32.samples, bfi.FP64, device=local_rank)
        _, tot64 = plan64.execute(lo, hi, job32.seed, job32.job_id, sub_id=sid, stream=stream)
        torch.cuda.synchronize()
        plan64.close()
        t32, t64 = tot32.cpu().numpy(), tot64.cpu().numpy()
        fp32 = {"value": world * job32.total_samples / (ms32 * 1e-3), "unit": "samples/s",
                "ms_per_step": ms32, "samples_per_subvolume": int(job32.samples[0]),
                "dtype": "f32 (compensated sums, f64 shift and merge)", "roofline": roof32,
                "logZ": float(t32[0]), "C": [float(x) for x in t32[4:4 + R]],
                "err_bound": {"Z_rel": float(bound32[0]), "C_rel_to_C0": [float(x) for x in bound32[1:]],
                              "note": "stated arithmetic error of this result (bfi_error_bound)"},
                "vs_fp64_mode": {"Z_rel": float(np.expm1(t32[0] - t64[0])),
                                 "C_rel_to_C0": [float(x) for x in (t32[4:4 + R] - t64[4:4 + R]) / t64[4]],
                                 "note": "FP64 mode draws FP64 points; the FP32 arithmetic bound (1e-6) is "
                                         "checked against the oracle on the same float points in the tests"}}

    # ---- the batching workload: 256 uneven jobs in one CUDA graph (FP32) ----
    batch = None
    if not args.skip_batch and world == 1:
        batch = run_batch(bfi, dev, stream)

    # ---- stated error of C(r) against the budget (time to 1e-3) ----
    tte = None
    if not args.skip_tte and world == 1:
        tte = run_time_to_error(bfi, dev, stream)

    # ---- the rows built on the hot path: line protocol, adaptive, samplers ----
    next_rows = None
    if not args.skip_next and world == 1:
        next_rows = run_next_rows(bfi, dev, stream, rows=args.next_rows.split(","),
                                  transform_log2=args.transform_log2)

    # ---- the serving workload: jobs arriving while others run ----
    serving = None
    if args.serving_seconds > 0 and world == 1:
        serving = run_serving(bfi, args.serving_seconds, rate=args.serving_rate)

    # ---- end to end through the host-buffer C-ABI call ----
    e2e = None
    if not args.skip_e2e:
        e2e = run_e2e(bfi, lat, job, local_rank, args, dist, dev, samples_all)

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        samples, times, cores = time_oracle(1)
        cpu = {"value": samples / times[0], "unit": "samples/s", "cores": cores, "kind": "oracle",
               "sample": "32 of the 1024 subvolumes (every 32nd) x 2^20 points of the same job, FP64 oracle"}
    report(args, rank, world, value, ms, roof, cpu, e2e, clocks, info, merged, fp32, job, batch, serving, tte,
           next_rows)
    if dist is not None:
        dist.destroy_process_group()


def run_e2e(bfi, lat, job, local_rank, args, dist, dev, samples_all):
    import torch
    ctx = bfi.Context(local_rank)
    lo_h = torch.empty(job.lo.shape, dtype=torch.float64, pin_memory=True).numpy()
    hi_h = torch.empty(job.hi.shape, dtype=torch.float64, pin_memory=True).numpy()
    lo_h[:] = job.lo
    hi_h[:] = job.hi
    sid_h = torch.empty(job.nsub, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    sid_h[:] = job.sub_id
    slots_h = torch.empty((job.nsub, bfi.slot_len(NX)), dtype=torch.float64, pin_memory=True).numpy()
    tot_h = torch.empty(bfi.totals_len(NX), dtype=torch.float64, pin_memory=True).numpy()
    e2e_steps = max(1, min(args.steps, 3))
    ctx.integrate(lat, lo_h, hi_h, job.samples, job.seed, 0, sub_id=sid_h, out_slots=slots_h, out_totals=tot_h)
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.integrate(lat, lo_h, hi_h, job.samples, job.seed, 0, sub_id=sid_h, out_slots=slots_h,
                      out_totals=tot_h)
    e2e_sec = (time.perf_counter() - t0) / e2e_steps
    if dist is not None:
        t = torch.tensor([e2e_sec], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_sec = float(t.item())
    ctx.close()
    h2d = lo_h.nbytes + hi_h.nbytes + sid_h.nbytes
    d2h = slots_h.nbytes + tot_h.nbytes
    return {"value": samples_all / e2e_sec, "unit": "samples/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h}


def run_batch(bfi, dev, stream, njobs=256):
    """The batching workload: 256 jobs (Nx from {4,6,8,10,16,32}, Nt from
    {2,4}, nu log-uniform in [0.1,10], 64-1024 subvolumes, 2^20-2^28 points,
    seed 3) captured into one CUDA graph, FP32 evaluation and FP64 merge,
    grid autotuned per shape; timed over graph replays with CUDA events."""
    import torch
    import workloads
    jobs = workloads.batch_jobs(njobs, seed=3)
    descs = []
    for j in jobs:
        descs.append(dict(lattice=bfi.lattice(j.nx, j.nt, j.nu, j.D, j.a, j.tau), samples=j.samples,
                          lo=torch.tensor(j.lo, device=dev), hi=torch.tensor(j.hi, device=dev),
                          seed=j.seed, job_id=j.job_id))
    t0 = time.perf_counter()
    b = bfi.Batch(descs, precision=bfi.FP32, nstreams=8, autotune=True)
    create_s = time.perf_counter() - t0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b.launch(stream)
    torch.cuda.synchronize()
    reps, total = 2, 0.0
    for _ in range(reps):
        ev0.record(stream)
        b.launch(stream)
        ev1.record(stream)
        ev1.synchronize()
        total += ev0.elapsed_time(ev1)
    ms = total / reps
    samples = sum(j.total_samples for j in jobs)
    shapes = sorted({(j.nx, j.nt) for j in jobs})
    tuned = {f"{nx}x{nt}": bfi.autotune_grid(bfi.lattice(nx, nt), bfi.FP32) for nx, nt in shapes}
    # the same jobs one after another, each alone on the device with its own plan and the same grid: the
    # sum of their CUDA-event times, against which the graph's replay shows what overlapping them gains
    alone_ms, alone_by_job = 0.0, []
    for j, dsc in zip(jobs, descs):
        plan = bfi.Plan(dsc["lattice"], j.samples, bfi.FP32)
        plan.set_grid(tuned[f"{j.nx}x{j.nt}"])
        plan.execute(dsc["lo"], dsc["hi"], j.seed, j.job_id, stream=stream)
        ev0.record(stream)
        plan.execute(dsc["lo"], dsc["hi"], j.seed, j.job_id, stream=stream)
        ev1.record(stream)
        ev1.synchronize()
        alone_by_job.append(ev0.elapsed_time(ev1))
        alone_ms += alone_by_job[-1]
        plan.close()
    ok = all(bool(torch.isfinite(t[0]).item()) for t in b.totals)
    # the ops-weighted roofline of one replay: every job's counted work (its own screen, stage-1 and evaluation
    # counts) over the replay time, against the FP32/INT issue peak
    issue, by_shape = 0.0, {}
    for k, j in enumerate(jobs):
        w = b.work(k).as_dict()
        ops = screen_work(w, j.nx, j.nt) + w["evaluated"] * eval_ops_fp32(j.nx, j.nt)
        issue += ops
        key = f"{j.nx}x{j.nt}"
        acc = by_shape.setdefault(key, {"jobs": 0, "samples": 0, "Gops": 0.0, "stage1": 0, "alone_ms": 0.0})
        acc["jobs"] += 1
        acc["samples"] += w["samples"]
        acc["Gops"] += ops / 1e9
        acc["stage1"] += w["stage1"]
        acc["alone_ms"] += alone_by_job[k]
    for acc in by_shape.values():
        # the shape's jobs run alone: their counted work over their own time, against the issue peak
        acc["alone_frac"] = acc["Gops"] * 1e9 / (acc["alone_ms"] * 1e-3) / ISSUE_PEAK_OPS
    b.close()
    achieved = issue / (ms * 1e-3)
    roof = {"bound": "alu", "resource": "FP32/INT issue", "achieved": achieved / 1e9, "peak": ISSUE_PEAK_OPS / 1e9,
            "unit": "Gop/s", "frac": achieved / ISSUE_PEAK_OPS, "ops": issue,
            "note": "each job's counted work (screen, stage 1 and survivors, FP32 evaluations) summed over the "
                    "256 jobs, over the graph replay time (hint, integrand and merges of every job)"}
    return {"workload": f"{njobs} jobs, Nx in {{4,6,8,10,16,32}}, Nt in {{2,4}}, nu log-uniform [0.1,10], "
                        "64-1024 subvolumes, 2^20-2^28 points (seed 3), FP32 eval / FP64 merge, one CUDA graph",
            "value": samples / (ms * 1e-3), "unit": "samples/s", "ms_per_launch": ms, "samples": samples,
            "jobs": njobs, "graph_create_s": create_s, "ctas_per_sm": tuned, "all_finite": ok, "roofline": roof,
            "alone_sum_ms": alone_ms,
            "by_shape": by_shape}


def run_time_to_error(bfi, dev, stream, log2_budgets=range(10, 29, 2), target=1e-3):
    """Stated error of C(r) against the sample budget on the 10x2 job (FP32,
    1024 subvolumes x 2^k points), the time of each run (CUDA events), and the
    1/sqrt(n) extrapolation of the budget and time that reach 'target'."""
    import torch
    import workloads
    lat = bfi.lattice(NX, NT)
    curve = []
    for k in log2_budgets:
        job = workloads.paper_10x2(1 << k)
        lo, hi = torch.tensor(job.lo, device=dev), torch.tensor(job.hi, device=dev)
        plan = bfi.Plan(lat, job.samples, bfi.FP32)
        plan.execute(lo, hi, job.seed, stream=stream)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        _, tot = plan.execute(lo, hi, job.seed, stream=stream)
        ev1.record(stream)
        ev1.synchronize()
        t = tot.cpu().numpy()
        C, Ce = t[4:4 + R], t[4 + R:4 + 2 * R]
        curve.append({"samples": job.total_samples, "ms": ev0.elapsed_time(ev1),
                      "C_err_rel_max": float(np.max(Ce / np.abs(C))), "C_err_over_C0_max": float(np.max(Ce) / C[0]),
                      "Z_err_rel": float(t[1])})
        plan.close()
    last = curve[-1]
    rate = last["samples"] / (last["ms"] * 1e-3)
    out = {"workload": "10x2 job (1024 subvolumes), FP32, budgets 2^20..2^38", "target": target, "curve": curve}
    for key in ("C_err_rel_max", "C_err_over_C0_max"):
        need = last["samples"] * (last[key] / target) ** 2
        out[f"samples_to_target_{key}"] = need
        out[f"seconds_to_target_{key}"] = need / rate
    return out


def _time_plan(plan, lo, hi, seed, stream, reps=2):
    """CUDA-event time of one plan execution (after one untimed run), its totals
    and evaluated-sample count."""
    import torch
    plan.execute(lo, hi, seed, stream=stream)
    best, tot = None, None
    for _ in range(reps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        _, tot = plan.execute(lo, hi, seed, stream=stream)
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
        best = ms if best is None else min(best, ms)
    n_eval, _ = plan.stats()
    return best, tot.cpu().numpy(), n_eval


FP64_FMA_PEAK = 2 * 152 * 2.07e9   # FP64 lanes per SM and clock x SMs x clock
# FP64 add, multiply and FMA per sample of the thread-per-sample range-map kernel at 10x2 (d = 20, R = 6):
# 13 d for the map (point, 1 - y^2, two Newton steps, v, J and the running product), 6 d + 3 for S_eff,
# 5 d + d/2 + 1 for the products Q_r, 3 + 6 R for the weight's sums
TRANSFORM_FP64_OPS_10x2 = 13 * 20 + (6 * 20 + 3) + (5 * 20 + 10 + 1) + (3 + 6 * 6)


def _oracle_rate(fn, samples, cores, what):
    """The oracle as it stands, timed once on the host: samples/s."""
    t0 = time.perf_counter()
    fn()
    wall = time.perf_counter() - t0
    return {"value": samples / wall, "unit": "samples/s", "cores": cores, "kind": "oracle", "sample": what}


NEXT_ROWS = ("nsphere", "adaptive", "transform", "gaussian")
# opt-in (minutes of GPU time): the paper's own Sec. 4 configuration, adaptive subdivision with the range map
PAPER_ROWS = ("paper_adaptive",)


def run_next_rows(bfi, dev, stream, rows=NEXT_ROWS, transform_log2=18):
    """The rows built on top of the hot path: the N-sphere integrand of the
    line protocol, adaptive subdivision with the convergence test, and the
    transform and Gaussian samplers, each timed on the GPU ('rows' picks
    some; 'transform_log2' sets the transform's points per subvolume)."""
    out = {}
    lat, d, nr = bfi.lattice(10, 2), 20, 6
    if "nsphere" in rows:
        out.update(_next_nsphere(bfi))
    if "adaptive" in rows:
        out.update(_next_adaptive(bfi, dev))
    if "transform" in rows:
        out.update(_next_transform(bfi, dev, stream, lat, d, nr, transform_log2))
    if "gaussian" in rows:
        out.update(_next_gaussian(bfi, dev, stream, lat, d, nr))
    if "paper_adaptive" in rows:
        out.update(_next_paper_adaptive(bfi, dev, nr))
    return out


def _next_paper_adaptive(bfi, dev, nr, max_depth=12, max_leaves=4096):
    """Sec. 4's configuration: the 10x2 lattice over all of R^20 through the
    range map ([-1,1]^20), 10^6 samples per subvolume doubled to 2 10^6 for
    the convergence test, with the loosest of the paper's criteria (results
    within a factor 1.085, or within 2 of each other, or both below 2).  The
    test compares the subvolume's Z (not each C(r) integral, as the paper's
    wrapper did); depth and subvolumes per round are bounded."""
    ctx = bfi.Context(dev.index or 0)
    try:
        ctx.set_sampler(bfi.SAMPLE_TRANSFORM)
        conv = bfi.convergence(2.0, 0.085, 2.0, 2.0, max_depth, max_leaves)
        t0 = time.perf_counter()
        tot, st = ctx.adaptive_integrate(bfi.lattice(10, 2), -1.0, 1.0, 1_000_000, 2, conv)
        wall = time.perf_counter() - t0
    finally:
        ctx.close()
    return {"paper_adaptive": {
        "workload": "Sec. 4: 10x2, range map over [-1,1]^20, n = 10^6 -> 2 10^6, criteria 1.085 / 2 / 2 on Z_s, "
                    f"max_depth {max_depth}, at most {max_leaves} subvolumes per round, FP64",
        "s_wall": wall, "samples": st.samples, "samples_per_s_wall": st.samples / wall, "stats": st.as_dict(),
        "logZ": float(tot[0]), "Z_err_rel": float(tot[1]), "C": [float(x) for x in tot[4:4 + nr]],
        "C_err": [float(x) for x in tot[4 + nr:4 + 2 * nr]],
        "paper": "about 500 core-hours of Haswell for the cheapest point of Fig. 1 (Sec. 6)"}}


def _next_nsphere(bfi):
    import math
    import oracle
    out = {}
    # N-sphere integrand (Listing 2's integrand; 2^30 samples over [-1,1]^3)
    bfi.nsphere(3, 1 << 20, 1)
    t0 = time.perf_counter()
    res, err, sd = bfi.nsphere(3, 1 << 30, 1)
    wall = time.perf_counter() - t0
    ops = 4 * 3 + 4   # per sample, FP64: point d, |x|^2 2d, half sums d, sqrt, f^2, two sums (Philox is INT)
    out["nsphere"] = {"workload": "f = sqrt(1-|x|^2) over [-1,1]^3, 2^30 samples (FP64 points), synchronous call",
                      "samples_per_s_wall": (1 << 30) / wall, "ms_wall": wall * 1e3, "result": res, "abs_err": err,
                      "exact": math.pi ** 2 / 4, "split_dim": sd,
                      "roofline": {"bound": "fp64", "fp64_ops_per_sample": ops,
                                   "frac_of_fp64_fma_peak": (1 << 30) * ops / wall / FP64_FMA_PEAK,
                                   "note": "wall time of the synchronous call, allocation and copies included"},
                      "cpu_baseline": _oracle_rate(lambda: oracle.nsphere(3, 1 << 21, 1), 1 << 21, 1,
                                                   "oracle.nsphere, 2^21 samples over [-1,1]^3")}
    return out


def _next_adaptive(bfi, dev):
    import math
    import oracle
    out = {}
    # adaptive subdivision: Listing 1's run, and the 10x2 lattice over its box
    conv = bfi.convergence(2.0, 0.003, 0.0, 0.0, 8, 1 << 16)
    t0 = time.perf_counter()
    res, err, st = bfi.adaptive_nsphere(3, 100_000, 1, conv)
    wall = time.perf_counter() - t0
    from oracle.adaptive import Convergence, adaptive_nsphere as oracle_adaptive_nsphere
    t0 = time.perf_counter()
    oracle_adaptive_nsphere(3, 100_000, 1, Convergence(2.0, 0.003, 0.0, 0.0, 8, 1 << 16))
    owall = time.perf_counter() - t0
    out["adaptive_nsphere"] = {"workload": "Listing 1: half the unit 4-ball over [-1,1]^3, n = 1e5, factor 2, "
                                           "rel_tol 0.003, max_depth 8", "ms_wall": wall * 1e3, "result": res,
                               "abs_err": err, "exact": math.pi ** 2 / 4, "stats": st.as_dict(),
                               "cpu_baseline": {"value": owall * 1e3, "unit": "ms", "cores": 1, "kind": "oracle",
                                                "sample": "the same run through oracle.adaptive"}}
    ctx = bfi.Context(dev.index or 0)
    conv = bfi.convergence(2.0, 0.2, 0.0, 0.0, 10, 1 << 12)
    ctx.adaptive_integrate(bfi.lattice(10, 2), -5.0, 5.0, 1 << 16, 2, bfi.convergence(2.0, 0.2, 0.0, 0.0, 1, 4))
    t0 = time.perf_counter()
    tot, st = ctx.adaptive_integrate(bfi.lattice(10, 2), -5.0, 5.0, 1 << 16, 2, conv)
    wall = time.perf_counter() - t0
    ctx.close()
    from oracle.adaptive import adaptive_integrate as oracle_adaptive_integrate
    t0 = time.perf_counter()
    _, oout = oracle_adaptive_integrate(oracle.lattice(10, 2), -5.0, 5.0, 1 << 12, 2,
                                        Convergence(2.0, 0.2, 0.0, 0.0, 4, 1 << 12))
    owall = time.perf_counter() - t0
    out["adaptive_lattice"] = {"workload": "10x2 over [-5,5]^20, n = 2^16, factor 2, rel_tol 0.2, max_depth 10, "
                                           "at most 4096 subvolumes per round, FP64", "ms_wall": wall * 1e3,
                               "samples_per_s_wall": st.samples / wall, "logZ": float(tot[0]),
                               "Z_err_rel": float(tot[1]), "stats": st.as_dict(),
                               "cpu_baseline": {"value": oout.stats["samples"] / owall, "unit": "samples/s",
                                                "cores": 1, "kind": "oracle",
                                                "sample": "oracle.adaptive on the same box, n = 2^12, depth 4"}}
    return out


def _next_transform(bfi, dev, stream, lat, d, nr, log2n):
    import torch
    import oracle
    import workloads
    from oracle import maps
    out = {}
    # transform sampler: [-1,1]^20 (all of R^20) bisected into 1024 subvolumes, 2^log2n points each
    lo_np, hi_np = workloads.bisected_boxes(d, 10, half=1.0)
    lo, hi = torch.tensor(lo_np, device=dev), torch.tensor(hi_np, device=dev)
    samples = np.full(1024, 1 << log2n, dtype=np.uint64)
    plan = bfi.Plan(lat, samples, bfi.FP64)
    plan.set_sampler(bfi.SAMPLE_TRANSFORM)
    ms, t, n_eval = _time_plan(plan, lo, hi, 2, stream)
    plan.close()
    n = int(samples.sum())
    ops = TRANSFORM_FP64_OPS_10x2
    out["transform"] = {"workload": f"10x2, v = y/(1-y^2) over [-1,1]^20 bisected into 1024 subvolumes x "
                                    f"2^{log2n} points, FP64, mass2 = 0", "ms": ms, "samples_per_s": n / (ms * 1e-3),
                        "roofline": {"bound": "fp64", "fp64_ops_per_sample": ops,
                                     "frac_of_fp64_fma_peak": n * ops / (ms * 1e-3) / FP64_FMA_PEAK,
                                     "note": "FP64 add, multiply and FMA of the definition (13 per coordinate "
                                             "for the map with its Newton reciprocal, 6 per residual, the "
                                             "products and sums); the one log and exp per sample not counted"},
                        "logZ": float(t[0]), "Z_err_rel": float(t[1]),
                        "C_err_over_C0_max": float(np.max(t[4 + nr:4 + 2 * nr]) / t[4]),
                        "cpu_baseline": _oracle_rate(
                            lambda: maps.integrate_mapped(oracle.lattice(10, 2), lo_np[:4], hi_np[:4], 1 << 14, 2,
                                                          kind=maps.TRANSFORM), 4 << 14, 1,
                            "oracle.maps (numpy over the C action), 4 subvolumes x 2^14 points")}
    return out


def _next_gaussian(bfi, dev, stream, lat, d, nr):
    import torch
    import oracle
    from oracle import maps
    out = {}
    # Gaussian sampler on the paper's box: the regulated linear-limit proposal
    box_lo = torch.full((1, d), -5.0, dtype=torch.float64, device=dev)
    box_hi = torch.full((1, d), 5.0, dtype=torch.float64, device=dev)
    gauss = []
    for k in (20, 26):
        plan = bfi.Plan(lat, [1 << k], bfi.FP64)
        plan.set_sampler(bfi.SAMPLE_GAUSSIAN, factor=bfi.gaussian_proposal(lat, 6.0))
        ms, t, n_eval = _time_plan(plan, box_lo, box_hi, 2, stream)
        plan.close()
        # FP64 add, multiply and FMA: per sample drawn |z|^2, the triangular F z and the box test; per sample
        # inside the box S_eff, the products and the sums (the Box-Muller log, sqrt and sincospi, and exp, not counted)
        ops = (1 << k) * (d + d * (d + 1) // 2 + 2 * d) + n_eval * ((6 * d + 3) + (5 * d + d // 2 + 1) + 39)
        gauss.append({"samples": 1 << k, "ms": ms, "samples_per_s": (1 << k) / (ms * 1e-3),
                      "inside_box": n_eval / (1 << k),
                      "frac_of_fp64_fma_peak": ops / (ms * 1e-3) / FP64_FMA_PEAK,
                      "logZ": float(t[0]), "Z_err_rel": float(t[1]),
                      "C_err_over_C0_max": float(np.max(t[4 + nr:4 + 2 * nr]) / t[4])})
    F_o = np.linalg.cholesky(maps.proposal_covariance(oracle.lattice(10, 2), 6.0))
    out["gaussian"] = {"workload": "10x2 over the box [-5,5]^20 as one volume, proposal N(0, (A + I/36)^-1) "
                                   "(linear limit, zero modes at sigma0 = 6), FP64", "runs": gauss,
                       "cpu_baseline": _oracle_rate(
                           lambda: maps.integrate_mapped(oracle.lattice(10, 2), -5 * np.ones(20), 5 * np.ones(20),
                                                         1 << 16, 2, kind=maps.GAUSSIAN, factor=F_o), 1 << 16, 1,
                           "oracle.maps (numpy over the C action), 2^16 points"),
                       "note": "the weights exp(-S)/q are heavy-tailed for the nonlinear action (ln Z grows "
                               "with the budget): the linear-limit proposal does not cover the zero-action "
                               "configurations away from the constant line"}
    return out


def run_serving(bfi, seconds, rate=200.0, seed=5):
    """The serving workload: Poisson arrivals at 'rate' jobs/s for 'seconds',
    sizes from the batching distribution plus 5% 64x8 lattices (numpy PCG64,
    seed 5), FP32, 8 stream slots, 40 GB admission budget, subvolumes split
    once when their relative variance exceeds 1e-2.  Latency = submit to
    result; throughput = samples of all passes / wall time until the last
    result."""
    import workloads
    rng = np.random.default_rng(seed)
    srv = bfi.Server(slots=8, precision=bfi.FP32, memory_budget=40 << 30, split_rel_var=1e-2,
                     max_split_rounds=1)
    reqs, offered = [], 0
    t0 = time.perf_counter()
    t_next = 0.0
    while True:
        t_next += float(rng.exponential(1.0 / rate))
        if t_next > seconds:
            break
        job = workloads.batch_jobs(1, seed=3, extra_64x8=0.05, rng=rng)[0]
        job.job_id = len(reqs)
        delay = t0 + t_next - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        reqs.append((srv.submit(bfi.lattice(job.nx, job.nt, job.nu, job.D, job.a, job.tau), job.lo, job.hi,
                                job.samples, job.seed, job.job_id), job))
        offered += job.total_samples
    t_submit_end = time.perf_counter()
    infos, issue = [], 0.0
    for r, job in reqs:
        r.wait(600_000)
        infos.append(r.info())
        w = r.work().as_dict()
        issue += screen_work(w, job.nx, job.nt) + w["evaluated"] * eval_ops_fp32(job.nx, job.nt)
        r.release()
    t_end = time.perf_counter()
    lat = np.array([i.latency_ms for i in infos])
    samples = sum(int(i.samples) for i in infos)
    st = srv.stats()
    srv.close()
    return {"workload": f"Poisson {rate:g} jobs/s for {seconds:g} s, batching sizes + 5% 64x8 (seed 5), FP32, "
                        "8 slots, 40 GB budget, split at Var(Z_s)/Z_s^2 > 1e-2 (1 round)",
            "rate": rate, "jobs": len(reqs), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "samples_per_s": samples / (t_end - t0), "samples": samples,
            "offered_samples_per_s_first_pass": offered / (t_submit_end - t0),
            "wall_s": t_end - t0, "passes": int(sum(i.passes for i in infos)),
            "leaves": int(sum(i.nsub_final for i in infos)), "completed": int(st.completed),
            "failed": int(st.failed), "peak_device_bytes": int(st.bytes_peak),
            "roofline": {"bound": "alu", "resource": "FP32/INT issue", "achieved": issue / (t_end - t0) / 1e9,
                         "peak": ISSUE_PEAK_OPS / 1e9, "unit": "Gop/s", "frac": issue / (t_end - t0) / ISSUE_PEAK_OPS,
                         "note": "every pass's counted work (screen, stage 1 and survivors, FP32 evaluations) "
                                 "over the wall time from the first submission to the last result"}}


def report(args, rank, world, value, ms, roof, cpu, e2e, clocks, info, merged, fp32, job, batch=None,
           serving=None, tte=None, next_rows=None):
    if rank == 0:
        line = {
            "metric": "samples/s", "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(world, int(job.samples[0])),
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": 4 * args.steps,
            "clocks": clocks,
            "plan": {"grid": info.grid, "block": info.block, "chunks": info.chunks,
                     "chunk_samples": info.chunk_samples},
            "result": {"logZ": float(merged[0]), "Z_err_rel": float(merged[1]),
                       "C": [float(x) for x in merged[4:4 + R]],
                       "C_err": [float(x) for x in merged[4 + R:4 + 2 * R]]},
            "fp32": fp32,
            "batch": batch,
            "serving": serving,
            "time_to_error": tte,
            "next_rows": next_rows,
        }
        line["summary"] = summary(value, roof, e2e, fp32, batch, serving, tte)
        print(json.dumps(line), flush=True)


def _sig(x, digits=4):
    return None if x is None else float(f"{x:.{digits}g}")


def summary(value, roof, e2e, fp32, batch, serving, tte):
    """The figures of every workload in a few hundred characters, last in the
    line: config 2 (FP64), config 3 (FP32 at 2^34 points), config 4 (the
    batch), config 5 (serving) and the time to a 1e-3 stated error."""
    out = {"fp64_samples_per_s": _sig(value), "fp64_frac": _sig(roof["frac"], 3),
           "e2e_samples_per_s": _sig(e2e["value"]) if e2e else None}
    if fp32:
        out.update({"fp32_samples_per_s": _sig(fp32["value"]), "fp32_frac": _sig(fp32["roofline"]["frac"], 3),
                    "fp32_vs_fp64_Z_rel": _sig(fp32["vs_fp64_mode"]["Z_rel"], 3),
                    "fp32_vs_fp64_C_rel_max": _sig(max(abs(x) for x in fp32["vs_fp64_mode"]["C_rel_to_C0"]), 3)})
        if "err_bound" in fp32:
            out.update({"fp32_err_bound_Z": _sig(fp32["err_bound"]["Z_rel"], 3),
                        "fp32_err_bound_C": _sig(max(fp32["err_bound"]["C_rel_to_C0"]), 3)})
    if batch:
        out.update({"batch_samples_per_s": _sig(batch["value"]), "batch_frac": _sig(batch["roofline"]["frac"], 3),
                    "batch_ms": _sig(batch["ms_per_launch"]), "batch_alone_sum_ms": _sig(batch.get("alone_sum_ms"))})
    if serving:
        out.update({"serving_rate": serving.get("rate"), "serving_jobs": serving["jobs"],
                    "serving_p50_ms": _sig(serving["p50_ms"]), "serving_p99_ms": _sig(serving["p99_ms"]),
                    "serving_samples_per_s": _sig(serving["samples_per_s"]), "serving_failed": serving["failed"]})
        if "roofline" in serving:
            out["serving_frac"] = _sig(serving["roofline"]["frac"], 3)
    if tte:
        out.update({"tte_samples_to_1e-3_C0": _sig(tte["samples_to_target_C_err_over_C0_max"], 3),
                    "tte_seconds_to_1e-3_C0": _sig(tte["seconds_to_target_C_err_over_C0_max"], 3)})
    return out


def main():
    global NX, NT, D, R, K
    ap = argparse.ArgumentParser()
    ap.add_argument("--lattice", default="10x2",
                    help="NXxNT of the timed job (the workload is 10x2; others for profiling other kernels)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="bfi", choices=["bfi", "reference"])
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp32", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-tte", action="store_true")
    ap.add_argument("--skip-next", action="store_true",
                    help="skip the N-sphere, adaptive and sampler measurements")
    ap.add_argument("--next-rows", default=",".join(NEXT_ROWS),
                    help="which of those rows to run (comma list of " + ", ".join(NEXT_ROWS + PAPER_ROWS) +
                         "; the last is opt-in)")
    ap.add_argument("--transform-log2", type=int, default=18,
                    help="points per subvolume of the transform-sampler row (2^18; smaller for profiling)")
    ap.add_argument("--serving-rate", type=float, default=200.0,
                    help="arrivals per second of the serving workload (the workload is 200)")
    ap.add_argument("--serving-seconds", type=float, default=10.0,
                    help="arrival window of the serving workload (the full workload is 60 s; 0 skips it)")
    ap.add_argument("--samples-log2", type=int, default=20,
                    help="points per subvolume of the FP64 job (the workload is 2^20; smaller for profiling)")
    args = ap.parse_args()
    NX, NT = (int(x) for x in args.lattice.lower().split("x"))
    D, R = NX * NT, NX // 2 + 1
    K = 2 + 3 * R
    if args.impl == "reference":
        run_reference(args)
    else:
        run_bfi(args)


if __name__ == "__main__":
    main()
