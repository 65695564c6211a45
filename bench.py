"""Benchmark: SPMESL solves/s and latency on one GB300 (and N replicas under torchrun).

Default workload (batch256): 256 independent SPMESL fits, fit i drawn with
seed 1000 + i: p log-uniform in [50, 2000], n uniform in [30, 400], the network
AR(1) / Erdos-Renyi / hub at random, X float32 with rows N(0, Theta^{-1}),
lambda0 = sqrt(2 log p / n), tol 1e-6, maxit 1000.  One step is one replay of
the batch's captured CUDA graph in mixed precision: split-BF16 Gram on the
tensor cores for all 256 fits, standardisation, FP32 coordinate descent (lazy
solver, block solver for the columns it hands over) with FP64 sigma updates,
Theta assembly and symmetrisation in FP64.  Inputs are resident in HBM; L2 is
flushed (256 MB write) between steps and the flush is outside the step's
events.

JSON line fields beyond the base contract:
  plain        the same 256 fits one FP32 spmesl_gram + spmesl_fit per fit,
               serialised on one stream: solves/s and per-solve latency
  latency      p50 / p99 of the batched step (every solve of a step completes
               with it) and of the plain per-fit solves
  served       the serving workload: Poisson arrivals of requests (p
               log-uniform in [100, 5000], n = max(p/4, 50)) into the serving
               context (continuous batching, mixed precision) against the plain
               path fed the same arrivals, at 0.5 and 0.9 of the served
               saturation rate; saturation measured three times (spread given)
  er_p2000_x10 ten ER p=2000 n=200 fits as one mixed batch (the single-shape batch)
  accuracy     max|dTheta|/max|Theta| of the batched mixed results against the
               FP64 oracle on every fit of the step, and the largest
               err_est / kkt_viol / dual_gap the device diagnostics state
  e2e          the same batch through the C ABI with host buffers: the 256 X
               copied in from one pinned buffer and the 256 Theta and sigma copied
               out into one each inside the timed region (Batch keeps a batch's
               outputs in one buffer), two batches on two streams in turn
  roofline     the coordinate-descent launches of a step (the dominant kernels):
               the row-synchronous byte model of the coordinate descent over
               their CUDA-event time against the measured HBM copy bandwidth;
               the per-column model beside it
  cpu_baseline the FP64 oracle (Gram + Algorithm 2) on the step's 256 fits on all
               host cores, and on as many as 20 s allow on one core; Gram and
               fit timed apart
  clocks       SM clocks and throttle reasons sampled during the timed region

--impl reference times the FP64 CPU oracle (the only reference this method
has) on a sample of the same workload and prints its line with
"impl": "reference".  --workload names another measurement: a single fit of
synth.WORKLOADS (for example hub_p10000_n500_mixed), er10 (the ten-fit batch
alone), serve, regression, table4 or residual.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SPMESL solves/s + p99 latency, mixed-prec batched vs plain GPU @ dTheta<=1e-4"
WORKLOAD = "batch256"
N_FITS = 256
BATCH_PREC = "mixed"
TOL, MAXIT = 1e-6, 1000
# kernels of one batched mixed step: split/transpose, tcgen05 Gram, prep_diag,
# prep_matrix, the column order (heat histogram, offsets, scatter), lazy
# solver, block solver over the handed-over columns, Theta.  (A batch with a
# fit of 4096 or more columns adds the block solver over the heavy columns on
# a side stream; no fit of this workload is that large.)
KERNELS_PER_STEP = 10
# fits of the batch the oracle solves (accuracy, CPU baseline, reference arm)
ORACLE_SAMPLE = list(range(N_FITS))
REFERENCE_SAMPLE = list(range(0, N_FITS, 32))


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def max_over_ranks(x: float, device=None) -> float:
    """The largest x over the ranks of the default process group (the slowest
    rank's time), or x itself when no group of more than one rank is up."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, max_ms: float) -> float:
    """Units per second of the whole job: every rank processed units_per_rank
    in at most max_ms (weak scaling, no data-path exchange between ranks)."""
    return world * units_per_rank / (max_ms / 1e3)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _sha_of(paths):
    """sha256 of the sources with comments and whitespace removed, so that a
    profile stays attached to the code it measured across comment edits."""
    import hashlib
    import re
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()




# ----------------------------------------------------------------------------- workloads
def batch_problems(only=None):
    """The 256 fits of the batched workload (synth.batch_specs, seeds 1000 + i);
    with `only`, just those fits (None in the other places)."""
    import numpy as np
    import synth
    keep = set(range(N_FITS)) if only is None else set(only)
    return [synth.make_problem(s["kind"], s["p"], s["n"], s["seed"], dtype=np.float32)
            if i in keep else None for i, s in enumerate(synth.batch_specs(N_FITS))]


def oracle_sample(probs, idx, nthreads: int, budget_s: float | None = None):
    """The FP64 oracle (Gram, then Algorithm 2) on the fits idx, in order,
    stopping once budget_s is spent: wall time of the Gram and of the fit
    summed over the fits done, and their Thetas."""
    import numpy as np
    import oracle
    oracle.build()
    t_gram = t_fit = 0.0
    thetas = {}
    t0 = time.perf_counter()
    for i in idx:
        X = probs[i].X.astype(np.float64)
        a = time.perf_counter()
        S = oracle.gram(X)
        b = time.perf_counter()
        ref = oracle.spmesl(S, probs[i].lambda0, tol=TOL, maxit=MAXIT, nthreads=nthreads)
        c = time.perf_counter()
        t_gram += b - a
        t_fit += c - b
        thetas[i] = ref["Theta"]
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    return dict(fits=len(thetas), t_gram=t_gram, t_fit=t_fit, thetas=thetas)


def cpu_baseline(probs, budget_single_s: float = 20.0):
    """The oracle as it stands on the host cores: the sampled fits on all
    cores (OpenMP over columns), then on one core within a time budget."""
    cores = os.cpu_count() or 1
    allc = oracle_sample(probs, ORACLE_SAMPLE, cores)
    one = oracle_sample(probs, ORACLE_SAMPLE, 1, budget_s=budget_single_s)
    ps = [probs[i].p for i in ORACLE_SAMPLE]
    out = {"value": allc["fits"] / (allc["t_gram"] + allc["t_fit"]), "unit": "solves/s",
           "cores": cores, "kind": "oracle",
           "sample": f"all {allc['fits']} fits of one step (p {min(ps)}-{max(ps)}): FP64 Gram, "
                     f"then Algorithm 2 with OpenMP over columns on all cores",
           "gram_s": allc["t_gram"], "fit_s": allc["t_fit"],
           "single_thread": {"value": one["fits"] / (one["t_gram"] + one["t_fit"]),
                             "unit": "solves/s", "cores": 1, "fits": one["fits"],
                             "gram_s": one["t_gram"], "fit_s": one["t_fit"],
                             "sample": f"the first {one['fits']} fits of the same step, one "
                                       f"thread, within {budget_single_s:.0f} s"}}
    return out, allc["thetas"]


def rel_err(T, R) -> float:
    import numpy as np
    return float(np.max(np.abs(T - R)) / np.max(np.abs(R)))


# ----------------------------------------------------------------------------- byte models
def gschedule_bytes(s: int, fits) -> float:
    """Bytes of the row-synchronous schedule with G in memory (coordinate
    descent written on G = S - S B), summed over fits given as dicts of p and
    the device counters: every column sweep reads its p entries of G, every
    coordinate change reads and writes a column of G, every distinct
    coordinate moved in a sweep index reads one row of S, and B is written."""
    b = 0.0
    for f in fits:
        b += s * f["p"] * (f["inner_sweeps"] + 2.0 * f["moves"] + f["rows_moved"]) + 2.0 * s * f["nnz_B"]
    return b


def column_bytes(s: int, fits) -> float:
    """Per-column model of the lazy solver: each column reads S_.j and writes
    b_j, each full-sweep move reads one row of S."""
    b = 0.0
    for f in fits:
        ldp = (f["p"] + 31) // 32 * 32
        b += s * ldp * (2.0 * f["p"] + f["moves"])
    return b


CD_SOURCES = ["paper_2203_15031_gb300/csrc/cd_device.cuh", "paper_2203_15031_gb300/csrc/batch.cu"]
PROFILE = "profiles/batch_cd_lazy_kernel_batch256.md"


def workload_sha() -> str:
    """sha256 of the batched workload's definition: the shapes and seeds of
    the 256 fits and the generator source."""
    import hashlib
    import synth
    h = hashlib.sha256(json.dumps(synth.batch_specs(N_FITS)).encode())
    with open(os.path.join(ROOT, "synth", "__init__.py")) as f:
        h.update(f.read().encode())
    return h.hexdigest()


def measured_traffic():
    """DRAM bytes per launch of the batched lazy kernel from the committed ncu
    summary, or None when the kernel source or the workload changed since."""
    try:
        text = open(os.path.join(ROOT, PROFILE)).read()
    except OSError:
        return None
    vals = dict(ln.split(":", 1) for ln in text.splitlines() if ":" in ln and ln[:1].isalpha())
    try:
        if vals.get("kernel_source_sha256", "").strip() != _sha_of(CD_SOURCES):
            return None
        if vals.get("workload_sha256", "").strip() != workload_sha():
            return None
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ----------------------------------------------------------------------------- headline
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2203_15031_gb300 as sp

    rank, local_rank, world = _env_rank()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    sp.lib()

    probs = batch_problems()
    inputs = [(torch.from_numpy(pr.X).to(dev), pr.lambda0) for pr in probs]
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    # ---- batched mixed path (headline): one graph replay per step
    bt = sp.Batch(inputs, kind="X", precision=BATCH_PREC, tol=TOL, maxit=MAXIT, use_graph=True)
    best_w = bt.tune()
    for _ in range(args.warmup):
        bt.run(stream)
    statuses, _ = bt.result(stream)
    if any(s not in (sp.SPMESL_OK, sp.SPMESL_NOT_CONVERGED) for s in statuses):
        raise RuntimeError(f"warm-up batch failed: {statuses}")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local_rank)
    with clk:
        for i in range(args.steps):
            flush.zero_()                   # evict the inputs from L2 between steps
            ev[i][0].record(stream)
            bt.run(stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    per = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(per), dev)
    value = whole_job_rate(N_FITS * args.steps, world, total_ms)
    statuses, agg = bt.result(stream)

    # ---- the coordinate-descent launches of a step: CUDA events around them
    # in a replay without the graph (same fits), with the distinct moved
    # coordinates counted on the device
    btc = sp.Batch(inputs, kind="X", precision=BATCH_PREC, tol=TOL, maxit=MAXIT,
                   warps_per_block=best_w, record_phase_times=True, count_rows=True)
    cd_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        btc.run(stream)
        _, stc = btc.result(stream)
        if i >= args.warmup:
            cd_ms.append(stc["ms_cd"])
    fit_counters = []
    for i, pr in enumerate(probs):
        fs = btc.fit_stats(i)
        fit_counters.append(dict(p=pr.p, inner_sweeps=fs["inner_sweeps"], moves=fs["moves"],
                                 rows_moved=fs["rows_moved"], nnz_B=fs["nnz_B"]))
    if not torch.equal(btc.Theta[0], bt.Theta[0]):
        raise RuntimeError("counting changed the result")
    btc.close()

    # ---- diagnostics of every fit (one more run, outside the timed region)
    btd = sp.Batch(inputs, kind="X", precision=BATCH_PREC, tol=TOL, maxit=MAXIT,
                   warps_per_block=best_w, diagnostics=True)
    btd.run(stream)
    _, diag = btd.result(stream)
    btd.close()

    # ---- end to end through the C ABI with host buffers (pinned): every step
    # copies its 256 X in and its 256 Theta and sigma out.  The 256 X of a
    # batch sit in one buffer, and its outputs in one buffer each (Batch lays
    # them out so), so a step is one host-to-device copy, the graph replay and
    # two device-to-host copies; two batches on two streams take the steps in
    # turn, so one step's copies run under the next step's compute
    xshapes = [tuple(pr.X.shape) for pr in probs]
    Xh_buf, Xh = sp.aligned_views(xshapes, torch.float32, None, pin=True)
    for d, pr in enumerate(probs):
        Xh[d].copy_(torch.from_numpy(pr.X))
    slots, xbufs = [], []
    for _ in range(2):
        xb, xv = sp.aligned_views(xshapes, torch.float32, dev)
        xb.copy_(Xh_buf)
        xbufs.append(xb)
        slots.append(sp.Batch([(x, lam) for x, (_, lam) in zip(xv, inputs)], kind="X",
                              precision=BATCH_PREC, tol=TOL, maxit=MAXIT, use_graph=True,
                              warps_per_block=best_w))
    streams = [torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)]
    Th = [torch.empty_like(slots[0].Theta_buf, device="cpu").pin_memory() for _ in range(2)]
    sh = [torch.empty_like(slots[0].sigma_buf, device="cpu").pin_memory() for _ in range(2)]

    def e2e_step(i):
        k = i % 2
        b, s = slots[k], streams[k]
        with torch.cuda.stream(s):
            xbufs[k].copy_(Xh_buf, non_blocking=True)
            b.run(s)
            Th[k].copy_(b.Theta_buf, non_blocking=True)
            sh[k].copy_(b.sigma_buf, non_blocking=True)

    for i in range(args.warmup):
        e2e_step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(args.steps):
        e2e_step(i)
    for s in streams:
        s.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    if world > 1:
        dist.barrier()
    h2d = Xh_buf.numel() * 4
    d2h = (Th[0].numel() + sh[0].numel()) * 8
    e2e = {"value": whole_job_rate(N_FITS * args.steps, world, e2e_s * 1e3), "unit": "solves/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "pipeline": "per step one copy of the 256 X in, the graph replay, one copy of the "
                       "256 Theta and one of the 256 sigma out (fits on 256-byte boundaries); "
                       "two batches on two streams in turn; host waits at the end"}
    # the link that bounds it: one more copy of a step's Theta bytes into
    # pinned host memory (best of 3)
    lk_src = torch.zeros(d2h // 8, dtype=torch.float64, device=dev)
    lk_dst = torch.empty(d2h // 8, dtype=torch.float64).pin_memory()
    lk = []
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lk_dst.copy_(lk_src, non_blocking=True)
        b.record(stream)
        b.synchronize()
        lk.append(a.elapsed_time(b))
    link_gbs = d2h / (min(lk) / 1e3) / 1e9
    e2e["link_d2h_gbs"] = link_gbs
    e2e["link_ceiling_solves_per_s"] = world * N_FITS * link_gbs * 1e9 / d2h
    e2e["frac_of_link_ceiling"] = e2e["value"] / e2e["link_ceiling_solves_per_s"]
    # the last step's results as the host got them equal the device-timed batch's
    last = (args.steps - 1) % 2
    for d in (0, N_FITS // 2, N_FITS - 1):
        o = slots[last].Theta[d].data_ptr() - slots[last].Theta_buf.data_ptr()
        host = Th[last][o // 8:o // 8 + probs[d].p ** 2].view(probs[d].p, probs[d].p)
        if not torch.equal(host, bt.Theta[d].cpu()):
            raise RuntimeError("end-to-end results differ from the device-timed batch")
    del lk_src, lk_dst, Th, sh, Xh, Xh_buf, xbufs
    for b in slots:
        b.close()

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    # ---- plain path over the same fits: one spmesl_gram + spmesl_fit per fit
    # through the C ABI, buffers allocated beforehand, serialised on the
    # stream (the second of two passes timed, one event pair per fit)
    opts = sp.spmesl_default_opts()
    opts.precision = sp.FP32
    bufs = []
    for (X, lam), pr in zip(inputs, probs):
        p, n = pr.p, pr.n
        gnb = sp.spmesl_gram_workspace_bytes(n, p, sp.FP32)
        fnb = sp.spmesl_fit_workspace_bytes(p, sp.FP32)
        bufs.append((X, lam, p, n, torch.empty((p, p), dtype=torch.float32, device=dev),
                     torch.empty((p, p), dtype=torch.float64, device=dev),
                     torch.empty(p, dtype=torch.float64, device=dev),
                     sp._workspace(max(gnb, 1), dev), gnb, sp._workspace(fnb, dev), fnb))
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in bufs]
    for rep in range(2):
        flush.zero_()
        for (X, lam, p, n, S, T, sg, (gk, gws), gnb, (fk, fws), fnb), (e0, e1) in zip(bufs, pev):
            e0.record(stream)
            sp._check(sp.spmesl_gram(X, n, p, p, sp.FP32, 0, S, p, gws, gnb, stream), "gram")
            sp._check(sp.spmesl_fit(S, n, p, lam, TOL, MAXIT, opts, T, sg, None, fws, fnb,
                                    stream), "fit")
            e1.record(stream)
        torch.cuda.synchronize()
    plain_per = [a.elapsed_time(b) for a, b in pev]
    plain_value = len(plain_per) / (sum(plain_per) / 1e3)
    plain_theta = {i: bufs[i][5].cpu().numpy() for i in ORACLE_SAMPLE}
    del bufs

    # ---- the served workload (continuous batching) against the plain path
    served = serve_block(dev, requests=args.serve_requests, pool=args.serve_pool,
                         fracs=args.serve_fracs, sat_reps=3)

    # ---- the single-shape batch: ten ER p=2000 n=200 fits
    er10 = er10_block(dev, args.steps, args.warmup)

    # ---- accuracy and the CPU baseline: the FP64 oracle on the step's fits
    hbm, which = _peaks()
    acc = {"bound": 1e-4, "sample": "all 256 fits of the step"}
    cb = None
    if not args.no_cpu_baseline:
        cb, ref = cpu_baseline(probs)
        acc["max_rel_dtheta_batched_mixed_vs_fp64_oracle"] = max(
            rel_err(bt.Theta[i].cpu().numpy(), ref[i]) for i in ref)
        acc["max_rel_dtheta_plain_fp32_vs_fp64_oracle"] = max(
            rel_err(plain_theta[i], ref[i]) for i in ref)
    acc["device_diagnostics"] = {"err_est_max": diag["err_est"], "kkt_viol_max": diag["kkt_viol"],
                                 "dual_gap_max": diag["dual_gap"],
                                 "of": "all 256 fits (err_est: estimate of max|dTheta|/max|Theta|)"}

    # ---- roofline of the coordinate-descent launches
    cdm = statistics.mean(cd_ms)
    bytes_gs = gschedule_bytes(4, fit_counters)
    bytes_col = column_bytes(4, fit_counters)
    achieved = bytes_gs / (cdm / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": measured_traffic(),
            "kernel": "batch_cd_lazy_kernel<float,1> + batch_cd_block_kernel<float,1> "
                      "(the coordinate-descent launches of a step)",
            "peak_kind": which, "model": "row-synchronous schedule with G in memory: "
            "s*p*(column sweeps) + 2*s*p*moves + s*p*(distinct rows moved per sweep index) "
            "+ 2*s*nnz(B), s = 4, counted on the device per fit",
            "algorithmic_bytes_per_launch": bytes_gs, "mean_launch_ms": cdm,
            "cd_timing": "CUDA events around the coordinate-descent launches on the batch's "
                         "stream, in a replay without the graph (same fits, L2 flushed)",
            "column_sweeps": sum(f["inner_sweeps"] for f in fit_counters),
            "moves": sum(f["moves"] for f in fit_counters),
            "rows_moved": sum(f["rows_moved"] for f in fit_counters),
            "per_column_model": {"bytes_per_launch": bytes_col,
                                 "achieved": bytes_col / (cdm / 1e3) / 1e9,
                                 "frac": bytes_col / (cdm / 1e3) / 1e9 / hbm},
            "warps_per_block": best_w, "block_columns": agg["block_columns"],
            "note": "S of most fits sits in L2: the model's bytes are work-equivalent, "
                    "the traffic key gives the DRAM bytes ncu counted"}
    srt = sorted(per)
    psrt = sorted(plain_per)
    q = lambda v, f: v[min(len(v) - 1, int(math.ceil(f * len(v))) - 1)]
    lat = {"batched_p50_ms": statistics.median(per), "batched_p99_ms": q(srt, 0.99),
           "plain_p50_ms": statistics.median(plain_per), "plain_p99_ms": q(psrt, 0.99),
           "unit": "ms from launch to completion of a solve (device); a batched solve "
                   "completes with its step"}
    ps = [pr.p for pr in probs]
    ns = [pr.n for pr in probs]
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "fits_per_step": N_FITS,
                       "p": f"log-uniform [50, 2000] (drawn {min(ps)}-{max(ps)})",
                       "n": f"uniform [30, 400] (drawn {min(ns)}-{max(ns)})",
                       "networks": "ar1 / er / hub_scaled at random", "seeds": "1000-1255",
                       "lambda0": "sqrt(2 log p / n)", "tol": TOL, "maxit": MAXIT,
                       "precision": BATCH_PREC,
                       "gram": "split-bf16 on tcgen05 (hi*hi + hi*lo + lo*hi, fp32 accumulation)",
                       "cd": "fp32", "sigma_theta": "fp64", "graph": True,
                       "warps_per_block": best_w, "inner_rule": "column",
                       "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"replicas x{world}"},
            "plain": {"value": plain_value, "unit": "solves/s", "precision": "fp32",
                      "path": "one spmesl_gram + spmesl_fit per fit, serialised"},
            "latency": lat, "served": served, "er_p2000_x10": er10, "accuracy": acc,
            "e2e": e2e, "roofline": roof, "cpu_baseline": cb,
            "statuses": {"ok": sum(s == sp.SPMESL_OK for s in statuses), "of": N_FITS},
            "gpu_launches": KERNELS_PER_STEP * args.steps, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    bt.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def serve_pool(dev, pool: int):
    """The serving workload's datasets: p log-uniform in [100, 5000],
    n = max(p/4, 50), networks in turn, request i of the pool seed 2000 + i."""
    import numpy as np
    import torch
    import synth
    rng = np.random.default_rng(7)
    kinds = ["ar1", "er", "hub_scaled"]
    out = []
    for i in range(pool):
        p = int(round(math.exp(rng.uniform(math.log(100), math.log(5000)))))
        n = max(p // 4, 50)
        pr = synth.make_problem(kinds[i % 3], p, n, 2000 + i, dtype=np.float32)
        out.append((torch.from_numpy(pr.X).to(dev), pr.lambda0, p, n))
    return out, rng


def serve_block(dev, requests: int = 200, pool: int = 24, fracs=(0.5, 0.9), sat_reps: int = 3):
    """Served path (spmesl_ctx: continuous batching under a 120 GB budget,
    mixed precision) against the plain path (one FP32 fit per launch,
    first-come first-served on one stream), fed the same Poisson arrivals at
    fractions of the served saturation rate.  Latency = completion - arrival
    per request (host clock).  Saturation: every request submitted at once,
    repeated sat_reps times."""
    import numpy as np
    import torch

    import paper_2203_15031_gb300 as sp

    data, rng = serve_pool(dev, pool)
    R = requests
    order = rng.integers(0, len(data), R)

    def serve_run(rate):
        srv = sp.Server(120 << 30, max_slots=256, precision=BATCH_PREC, tol=TOL, maxit=MAXIT)
        gaps = rng.exponential(1.0 / rate, R) if rate else np.zeros(R)
        arrivals = np.cumsum(gaps)
        t0 = time.perf_counter()
        live, lat, done_t = {}, [], []
        k = 0
        while k < R or live:
            now = time.perf_counter() - t0
            while k < R and arrivals[k] <= now:
                X, lam, _, _ = data[order[k]]
                live[srv.submit(X, lam)] = k
                k += 1
            for t in list(live):
                r = srv.poll(t)
                if r is not None:
                    if r[0] not in (sp.SPMESL_OK, sp.SPMESL_NOT_CONVERGED):
                        raise RuntimeError(f"request failed: {r[0]}")
                    lat.append(r[3]["ms_total"])
                    done_t.append(time.perf_counter() - t0)
                    del live[t]
            if not live and k < R:
                time.sleep(max(0.0, min(0.001, arrivals[k] - (time.perf_counter() - t0))))
        srv.close()
        return R / (max(done_t) - arrivals[0]), lat

    S, ws = {}, {}
    opts = sp.spmesl_default_opts()
    opts.precision = sp.FP32

    def plain_fit(idx):
        X, lam, p, n = data[idx]
        if p not in S:
            S[p] = torch.empty((p, p), dtype=torch.float32, device=dev)
            gnb = sp.spmesl_gram_workspace_bytes(n, p, sp.FP32)
            fnb = sp.spmesl_fit_workspace_bytes(p, sp.FP32)
            ws[p] = (sp._workspace(max(gnb, 1), dev), gnb, sp._workspace(fnb, dev), fnb,
                     torch.empty((p, p), dtype=torch.float64, device=dev),
                     torch.empty(p, dtype=torch.float64, device=dev))
        (gk, gws), gnb, (fk, fws), fnb, Th, sg = ws[p]
        sp._check(sp.spmesl_gram(X, n, p, p, sp.FP32, 0, S[p], p, gws, gnb), "spmesl_gram")
        sp._check(sp.spmesl_fit(S[p], n, p, lam, TOL, MAXIT, opts, Th, sg, None, fws, fnb),
                  "spmesl_fit")
        torch.cuda.current_stream().synchronize()

    def plain_run(rate):
        gaps = rng.exponential(1.0 / rate, R) if rate else np.zeros(R)
        arrivals = np.cumsum(gaps)
        t0 = time.perf_counter()
        lat, done_t = [], []
        for k in range(R):
            now = time.perf_counter() - t0
            if arrivals[k] > now:
                time.sleep(arrivals[k] - now)
            plain_fit(order[k])
            t = time.perf_counter() - t0
            lat.append(1e3 * (t - arrivals[k]))
            done_t.append(t)
        return R / (max(done_t) - arrivals[0]), lat

    def q(v, f):
        v = sorted(v)
        return v[min(len(v) - 1, int(math.ceil(f * len(v))) - 1)]

    for i in range(len(data)):                # warm both paths (kernels, pools)
        plain_fit(i)
    serve_run(0)
    sats = [serve_run(0)[0] for _ in range(sat_reps)]
    sat_serve = statistics.median(sats)
    sat_plain, _ = plain_run(0)
    rows = []
    for frac in fracs:
        rate = frac * sat_serve
        sv, slat = serve_run(rate)
        pv, plat = plain_run(rate)
        rows.append({"arrival_rate": rate, "fraction_of_saturation": frac,
                     "served": {"solves_per_s": sv, "p50_ms": q(slat, 0.5), "p99_ms": q(slat, 0.99)},
                     "plain": {"solves_per_s": pv, "p50_ms": q(plat, 0.5), "p99_ms": q(plat, 0.99)}})
    return {"config": {"requests": R, "datasets": len(data), "p": "log-uniform [100, 5000]",
                       "n": "max(p/4, 50)", "networks": "ar1 / er / hub_scaled",
                       "budget_gb": 120, "max_slots": 256, "precision": BATCH_PREC,
                       "plain_precision": "fp32", "arrivals": "Poisson, seed 7"},
            "saturation": {"served_solves_per_s": sat_serve, "served_runs": sats,
                           "served_spread": [min(sats), max(sats)],
                           "plain_solves_per_s": sat_plain},
            "rates": rows, "unit": "solves/s; latency ms from arrival to completion (host)"}


def er10_block(dev, steps: int, warmup: int):
    """Ten ER p=2000 n=200 fits (seeds 0-9) as one mixed batch, one graph
    replay per step, L2 flushed between steps."""
    import numpy as np
    import torch

    import paper_2203_15031_gb300 as sp
    import synth
    probs = [synth.make_problem("er", 2000, 200, s, dtype=np.float32) for s in range(10)]
    inputs = [(torch.from_numpy(pr.X).to(dev), pr.lambda0) for pr in probs]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    bt = sp.Batch(inputs, kind="X", precision=BATCH_PREC, tol=TOL, maxit=MAXIT, use_graph=True)
    w = bt.tune()
    for _ in range(warmup):
        bt.run(stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        bt.run(stream)
        b.record(stream)
    torch.cuda.synchronize()
    per = [a.elapsed_time(b) for a, b in ev]
    bt.close()
    return {"value": 10 * steps / (sum(per) / 1e3), "unit": "solves/s",
            "ms_per_step": statistics.mean(per), "p": 2000, "n": 200, "network": "erdos_renyi",
            "fits_per_step": 10, "seeds": "0-9", "precision": BATCH_PREC, "warps_per_block": w}


def run_batch256_steps(args):
    """The batched workload's steps alone (for profiling): warm-up and timed
    graph replays of the 256-fit mixed batch, nothing else."""
    import torch
    import paper_2203_15031_gb300 as sp
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    sp.lib()
    probs = batch_problems()
    inputs = [(torch.from_numpy(pr.X).to(dev), pr.lambda0) for pr in probs]
    bt = sp.Batch(inputs, kind="X", precision=BATCH_PREC, tol=TOL, maxit=MAXIT, use_graph=True)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        bt.run(stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        bt.run(stream)
    b.record(stream)
    statuses, st = bt.result(stream)
    ms = a.elapsed_time(b) / args.steps
    print(json.dumps({"workload": "batch256_steps", "ms_per_step": ms,
                      "solves_per_s": N_FITS / (ms / 1e3), "ok": sum(x == 0 for x in statuses),
                      "workload_sha256": workload_sha()}), flush=True)
    bt.close()


def run_er10(args):
    import torch
    import paper_2203_15031_gb300 as sp
    torch.cuda.set_device(0)
    sp.lib()
    out = er10_block(torch.device("cuda", 0), args.steps, args.warmup)
    print(json.dumps({"metric": METRIC, "workload": "er_p2000_n200_x10", **out}), flush=True)


def run_serve(args):
    import torch
    import paper_2203_15031_gb300 as sp
    torch.cuda.set_device(0)
    sp.lib()
    out = serve_block(torch.device("cuda", 0), requests=args.serve_requests, pool=args.serve_pool,
                      fracs=args.serve_fracs, sat_reps=3)
    print(json.dumps({"metric": METRIC, "workload": "serve", **out}), flush=True)


def run_reference(args):
    """The FP64 oracle as it stands, on the host cores: each step solves a
    bounded sample of the batched workload (every 32nd fit: Gram, then
    Algorithm 2 with OpenMP over columns on all cores)."""
    rank, _, world = _env_rank()
    if rank != 0:
        return
    probs = batch_problems(REFERENCE_SAMPLE)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_sample(probs, REFERENCE_SAMPLE[:1], cores)
    times = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_sample(probs, REFERENCE_SAMPLE, cores)
        times.append(time.perf_counter() - t0)
    total = time.perf_counter() - t_all
    value = len(REFERENCE_SAMPLE) * args.steps / total
    ps = [probs[i].p for i in REFERENCE_SAMPLE]
    sample = (f"{len(REFERENCE_SAMPLE)} of the 256 fits per step (every 32nd, p {min(ps)}-"
              f"{max(ps)}): FP64 Gram + Algorithm 2, OpenMP over columns on all cores")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "fits_per_step": len(REFERENCE_SAMPLE),
                       "p": "log-uniform [50, 2000]", "n": "uniform [30, 400]",
                       "networks": "ar1 / er / hub_scaled at random", "seeds": "1000-1255",
                       "lambda0": "sqrt(2 log p / n)", "tol": TOL, "maxit": MAXIT},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_single(args):
    """One whole solve per step (Gram + fit) of a single-fit workload, e.g.
    the hub network p = 10000, n = 500 with the split-BF16 tensor-core Gram.
    Reports the coordinate-descent roofline (dominant kernel) and the Gram's
    tensor roofline."""
    import numpy as np
    import torch

    import paper_2203_15031_gb300 as sp
    import synth

    rank, local_rank, world = _env_rank()
    if world > 1:
        raise SystemExit("--workload other than the default runs on one GPU")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    sp.lib()
    w = synth.WORKLOADS[args.workload]
    prec = {"fp64": sp.FP64, "fp32": sp.FP32, "mixed": sp.MIXED}[w["prec"]]
    dt = np.float64 if prec == sp.FP64 else np.float32
    prob = synth.make_problem(w["kind"], w["p"], w["n"], 0, dtype=dt)
    p, n, tol, maxit = w["p"], w["n"], w["tol"], w["maxit"]
    X = torch.from_numpy(prob.X).to(dev)
    S = torch.empty((p, p), dtype=X.dtype, device=dev)
    Theta = torch.empty((p, p), dtype=torch.float64, device=dev)
    sigma = torch.empty(p, dtype=torch.float64, device=dev)
    gnb = sp.spmesl_gram_workspace_bytes(n, p, prec)
    fnb = sp.spmesl_fit_workspace_bytes(p, prec)
    gkeep, gws = sp._workspace(max(gnb, 1), dev)
    fkeep, fws = sp._workspace(fnb, dev)
    opts = sp.spmesl_default_opts()
    opts.precision = prec
    opts.record_phase_times = 1
    opts.count_rows = 1
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def step():
        g0.record(stream)
        sp._check(sp.spmesl_gram(X, n, p, p, prec, 0, S, p, gws, gnb, stream), "spmesl_gram")
        g1.record(stream)
        sp._check(sp.spmesl_fit(S, n, p, prob.lambda0, tol, maxit, opts, Theta, sigma, None, fws,
                                fnb, stream), "spmesl_fit")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = sp.Stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    gram_ms, cd_ms, moves, sweeps, nnzb, act_s, act_m, rows = [], [], [], [], [], [], [], []
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            sp._check(sp.spmesl_fit_result(fws, p, prec, st, stream), "spmesl_fit_result")
            gram_ms.append(g0.elapsed_time(g1))
            cd_ms.append(st.ms_cd)
            moves.append(st.moves)
            sweeps.append(st.inner_sweeps)
            nnzb.append(st.nnz_B)
            act_s.append(st.active_sweeps)
            act_m.append(st.active_moves)
            rows.append(st.rows_moved)
        torch.cuda.synchronize()
    per = [a.elapsed_time(b) for a, b in ev]
    value = args.steps / (sum(per) / 1e3)
    hbm, which = _peaks()
    s = 8 if prec == sp.FP64 else 4
    counters = [dict(p=p, inner_sweeps=statistics.mean(sweeps), moves=statistics.mean(moves),
                     rows_moved=statistics.mean(rows), nnz_B=statistics.mean(nnzb))]
    bytes_gs = gschedule_bytes(s, counters)
    bytes_col = column_bytes(s, counters)
    cdm = statistics.mean(cd_ms)
    roof = {"bound": "hbm", "achieved": bytes_gs / (cdm / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": bytes_gs / (cdm / 1e3) / 1e9 / hbm, "traffic": None,
            "kernel": "cd_column_lazy_kernel + cd_column_block_kernel (the coordinate-descent "
                      "launches of the fit)", "peak_kind": which,
            "model": "row-synchronous schedule with G in memory (device-counted sweeps, moves, "
                     "distinct rows moved per sweep index)",
            "algorithmic_bytes_per_launch": bytes_gs, "mean_launch_ms": cdm,
            "column_sweeps": counters[0]["inner_sweeps"], "moves": counters[0]["moves"],
            "rows_moved": counters[0]["rows_moved"],
            "active_sweeps_per_launch": statistics.mean(act_s),
            "active_moves_per_launch": statistics.mean(act_m),
            "block_columns": st.block_columns,
            "per_column_model": {"bytes_per_launch": bytes_col,
                                 "achieved": bytes_col / (cdm / 1e3) / 1e9,
                                 "frac": bytes_col / (cdm / 1e3) / 1e9 / hbm}}
    gm = statistics.mean(gram_ms)
    roof_gram = None
    if prec == sp.MIXED:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
        # 128 x bn tiles holding an entry of the upper triangle; three MMAs
        # (hi*hi, hi*lo, lo*hi) over the padded sample dimension per tile
        bn = 256 if p > 1024 else 128
        tm_count, tn_count = (p + 127) // 128, (p + bn - 1) // bn
        tiles = sum(tn_count - (128 * tm) // bn for tm in range(tm_count))
        npad = (n + 63) // 64 * 64
        executed = 3.0 * tiles * 128 * bn * npad * 2
        roof_gram = {"bound": "tensor", "achieved": executed / (gm / 1e3) / 1e12, "peak": bf16,
                     "unit": "TFLOP/s", "frac": executed / (gm / 1e3) / 1e12 / bf16,
                     "kernel": "gram_tc_kernel (+ split_transpose_kernel)",
                     "executed_mma_flops": executed, "algorithmic_flops": float(n) * p * (p + 1),
                     "mean_ms": gm, "peak_kind": "measured bf16 burst"}
    srt = sorted(per)
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(per) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == sp.FP64 else "f32", "data": "synthetic",
            "config": {"workload": args.workload, "p": p, "n": n, "network": w["kind"],
                       "precision": w["prec"], "tol": tol, "maxit": maxit,
                       "path": "single fit (spmesl_gram + spmesl_fit)",
                       "l2": "flushed between steps (256 MB write)"},
            "latency": {"p50_ms": statistics.median(per),
                        "p99_ms": srt[min(len(srt) - 1, int(math.ceil(0.99 * len(srt))) - 1)]},
            "roofline": roof, "roofline_gram": roof_gram,
            # Gram (split + tcgen05, or SIMT); prep_diag, prep_matrix, [column
            # order: more columns than resident warps, or heavy routing],
            # [block solver on the heavy columns: p >= 4096], lazy, block solver
            # on the handed-over columns, row count, Theta
            "gpu_launches": ((2 if prec == sp.MIXED else 1) + 6 + (1 if p >= 4096 else 0)
                             + (1 if p >= 3648 else 0)) * args.steps,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    del gkeep, fkeep


def run_residual(args):
    """The residual form (spmesl_fit_residual: gradients from the data, no
    Gram matrix) against the covariance form (spmesl_gram + spmesl_fit) on
    the same data, one whole fit per step each: Erdos-Renyi p=2000, n=200
    (FP32) and the hub network p=10000, n=500 (residual FP32; covariance
    with the split-BF16 Gram).  Reports fits/s, the coordinate-descent launch
    alone, the sweep and move counts, the workspace of each form and the
    largest difference between the two estimates."""
    import numpy as np
    import torch

    import paper_2203_15031_gb300 as sp
    import synth

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    sp.lib()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    cases = []
    with ClockSampler(0) as clk:
        for name, res_prec, cov_prec in (("er_p2000_n200_fp32", sp.FP32, sp.FP32),
                                         ("hub_p10000_n500_mixed", sp.FP32, sp.MIXED)):
            w = synth.WORKLOADS[name]
            prob = synth.make_problem(w["kind"], w["p"], w["n"], 0, dtype=np.float32)
            p, n, tol, maxit = w["p"], w["n"], w["tol"], w["maxit"]
            steps = args.steps if p <= 2000 else max(3, args.steps // 10)
            X = torch.from_numpy(prob.X).to(dev)
            Th_r = torch.empty((p, p), dtype=torch.float64, device=dev)
            Th_c = torch.empty((p, p), dtype=torch.float64, device=dev)
            sg_r = torch.empty(p, dtype=torch.float64, device=dev)
            sg_c = torch.empty(p, dtype=torch.float64, device=dev)
            S = torch.empty((p, p), dtype=torch.float32, device=dev)
            rnb = sp.spmesl_fit_residual_workspace_bytes(n, p, res_prec)
            gnb = sp.spmesl_gram_workspace_bytes(n, p, cov_prec)
            fnb = sp.spmesl_fit_workspace_bytes(p, cov_prec)
            rkeep, rws = sp._workspace(rnb, dev)
            gkeep, gws = sp._workspace(max(gnb, 1), dev)
            fkeep, fws = sp._workspace(fnb, dev)
            ro, co = sp.spmesl_default_opts(), sp.spmesl_default_opts()
            ro.precision, co.precision = res_prec, cov_prec
            ro.record_phase_times = co.record_phase_times = 1

            def res_step():
                sp._check(sp.spmesl_fit_residual(X, n, p, p, prob.lambda0, tol, maxit, ro, Th_r,
                                                  sg_r, None, rws, rnb, stream),
                          "spmesl_fit_residual")

            def cov_step():
                sp._check(sp.spmesl_gram(X, n, p, p, cov_prec, 0, S, p, gws, gnb, stream),
                          "spmesl_gram")
                sp._check(sp.spmesl_fit(S, n, p, prob.lambda0, tol, maxit, co, Th_c, sg_c, None,
                                        fws, fnb, stream), "spmesl_fit")

            out = {"workload": name, "p": p, "n": n, "network": w["kind"], "steps": steps}
            for tag, step, ws, prec in (("residual", res_step, rws, res_prec),
                                        ("covariance", cov_step, fws, cov_prec)):
                for _ in range(args.warmup):
                    step()
                st = sp.Stats()
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(steps)]
                cd = []
                torch.cuda.synchronize()
                for i in range(steps):
                    flush.zero_()
                    ev[i][0].record(stream)
                    step()
                    ev[i][1].record(stream)
                    rc = sp.spmesl_fit_result(ws, p, prec, st, stream)
                    if rc != sp.SPMESL_OK:
                        raise RuntimeError(f"{tag} fit status {rc}")
                    cd.append(st.ms_cd)
                per = [a.elapsed_time(b) for a, b in ev]
                out[tag] = {"fits_per_s": steps / (sum(per) / 1e3),
                            "ms_per_fit": statistics.mean(per), "cd_ms": statistics.mean(cd),
                            "precision": {sp.FP32: "fp32", sp.MIXED: "mixed"}[prec],
                            "full_sweeps": st.inner_sweeps, "moves": st.moves,
                            "active_sweeps": st.active_sweeps, "outer_max": st.outer_iters,
                            "workspace_bytes": rnb if tag == "residual" else gnb + fnb + 4 * p * p}
            scale = float(Th_c.abs().max())
            out["max_rel_dtheta_residual_vs_covariance"] = float((Th_r - Th_c).abs().max()) / scale
            cases.append(out)
            del rkeep, gkeep, fkeep, S, Th_r, Th_c
            torch.cuda.empty_cache()
        torch.cuda.synchronize()
    head = cases[0]
    line = {"metric": "SPMESL fits/s, residual form (spmesl_fit_residual)",
            "value": head["residual"]["fits_per_s"], "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": head["residual"]["ms_per_fit"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "residual_vs_covariance", "tol": 1e-6, "maxit": 1000,
                       "l2": "flushed between steps (256 MB write)"},
            "cases": cases,
            "roofline": {"bound": "latency",
                         "note": "each formed 128-coordinate gradient slice reads n rows of W "
                                 "(512 B each) through L2 in one warp's dependent chain; the "
                                 "covariance form reads 1 + |support| rows of S per slice"},
            # the head value's timed steps: stats, build, coordinate descent,
            # Theta zeroing and Theta per residual fit
            "gpu_launches": 5 * args.steps, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


# Table 4 of the paper (values as printed, with their standard errors): the
# committed fixture tests/golden/table4_ar_p500_n250.json.
TABLE4_FIXTURE = "tests/golden/table4_ar_p500_n250.json"
TABLE4_KEYS = ["n_edges_hat", "sen", "spe", "fdr", "misr", "mcc", "frobenius"]


def run_table4(args, datasets: int = 50):
    """The estimation study's AR(1) and AR(4) rows of Table 4: 50 seeded
    datasets per network (p = 500, n = 250, X ~ N(0, Theta^-1)), each level
    (SPMESL-2: lambda_univ, SPMESL-4: lambda_ub, SPMESL-P: lambda_pb) one FP64
    batch of the 50 fits, measures on the GPU (spmesl_support_metrics), means
    and standard errors against the printed ones."""
    import numpy as np
    import torch

    import paper_2203_15031_gb300 as sp
    import synth

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    sp.lib()
    p, n = 500, 250
    with open(os.path.join(ROOT, TABLE4_FIXTURE)) as fh:
        table4 = json.load(fh)
    rules = {"SPMESL-2": sp.LAMBDA_UNIV, "SPMESL-4": sp.LAMBDA_UB, "SPMESL-P": sp.LAMBDA_PB}
    rows, solve_ms = [], []
    for kind in ("ar1_paper", "ar4"):
        theta = synth.make_theta(kind, p, np.random.default_rng(0))
        theta_d = torch.from_numpy(theta).to(dev)
        Xs = [torch.from_numpy(synth.sample_x(theta, n, np.random.default_rng(7000 + s),
                                              dtype=np.float64)).to(dev)
              for s in range(datasets)]
        for name, rule in rules.items():
            lam = sp.spmesl_lambda(rule, n, p)
            bt = sp.Batch([(X, lam) for X in Xs], kind="X", precision="fp64", tol=1e-8,
                          maxit=1000)
            bt.run()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            bt.run()
            statuses, _ = bt.result()
            solve_ms.append((time.perf_counter() - t0) * 1e3)
            vals = []
            for T in bt.Theta:
                m = sp.support_metrics(T, theta_d)
                vals.append([m["n_edges_hat"], 100 * m["sen"], 100 * m["spe"], 100 * m["fdr"],
                             100 * m["misr"], 100 * m["mcc"], m["frobenius"]])
            v = np.array(vals)
            mean, se = v.mean(0), v.std(0, ddof=1) / math.sqrt(datasets)
            row = next(r for r in table4["rows"] if r["network"] == kind and r["method"] == name)
            paper, paper_se = row["mean"], row["se"]
            rows.append({"network": kind, "method": name, "lambda0": lam,
                         "statuses_ok": int(sum(s == sp.SPMESL_OK for s in statuses)),
                         "ours": dict(zip(TABLE4_KEYS, [round(float(x), 4) for x in mean])),
                         "ours_se": dict(zip(TABLE4_KEYS, [round(float(x), 4) for x in se])),
                         "paper": dict(zip(TABLE4_KEYS, paper)),
                         "paper_se": dict(zip(TABLE4_KEYS, paper_se))})
            bt.close()
    line = {"metric": "estimation measures vs Table 4 (AR(1), AR(4); p=500, n=250, 50 datasets)",
            "workload": "table4", "precision": "fp64", "tol": 1e-8,
            "batch_ms_50_fits": [round(x, 2) for x in solve_ms], "rows": rows}
    print(json.dumps(line), flush=True)


def run_regression(args):
    """One scaled-lasso regression per step (spmesl_scaled_lasso): Erdos-Renyi
    predictors p=2000, n=200, y = X beta + noise with 10 active coefficients;
    the split-BF16 Gram of [X y], then the response column's coordinate
    descent.  The oracle (FP64 Gram of [X y] + Algorithm 1 for that column,
    one thread) is timed beside it."""
    import numpy as np
    import torch

    import paper_2203_15031_gb300 as sp
    import synth

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    sp.lib()
    w = synth.REGRESSION
    r = synth.make_regression(w["kind"], w["p"], w["n"], 0, k=w["k"], noise=w["noise"],
                              dtype=w["dtype"])
    p, n, tol, maxit = r.p, r.n, w["tol"], w["maxit"]
    prec = {"fp64": sp.FP64, "fp32": sp.FP32, "mixed": sp.MIXED}[w["prec"]]
    X, y = torch.from_numpy(r.X).to(dev), torch.from_numpy(r.y).to(dev)
    beta = torch.empty(p, dtype=torch.float64, device=dev)
    sigma = torch.empty(1, dtype=torch.float64, device=dev)
    nb = sp.spmesl_scaled_lasso_workspace_bytes(n, p, prec)
    keep, ws = sp._workspace(nb, dev)
    opts = sp.spmesl_default_opts()
    opts.precision = prec
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        sp._check(sp.spmesl_scaled_lasso(X, y, n, p, r.lambda0, tol, maxit, opts, beta, sigma,
                                         None, ws, nb, stream), "spmesl_scaled_lasso")

    for _ in range(args.warmup):
        step()
    st = sp.Stats()
    rc = sp.spmesl_scaled_lasso(X, y, n, p, r.lambda0, tol, maxit, opts, beta, sigma, st, ws, nb,
                                stream)
    if rc != sp.SPMESL_OK:
        raise RuntimeError(f"warm-up regression status {rc}")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    per = [a.elapsed_time(b) for a, b in ev]
    value = args.steps / (sum(per) / 1e3)
    srt = sorted(per)
    cb = None
    acc = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        Z = np.concatenate([r.X.astype(np.float64), r.y.astype(np.float64)[:, None]], axis=1)
        times = []
        for _ in range(3):
            t0 = time.perf_counter()
            ref = oracle.columns(oracle.gram(Z), [p], r.lambda0, tol=tol, maxit=maxit, nthreads=1)
            times.append(time.perf_counter() - t0)
        tm = statistics.median(times)
        cb = {"value": 1.0 / tm, "unit": "solves/s", "cores": 1, "kind": "oracle",
              "sample": f"3 whole regressions (FP64 Gram of [X y] + Algorithm 1 for the response "
                        f"column, one thread), median {tm:.3f} s"}
        b_ref = ref["b"][0, :p]
        acc = {"max_rel_dbeta_vs_fp64_oracle":
               float(np.max(np.abs(beta.cpu().numpy() - b_ref)) / np.max(np.abs(b_ref))),
               "rel_dsigma": abs(float(sigma.item()) - float(ref["sigma"][0])) / float(ref["sigma"][0])}
    hbm, which = _peaks()
    line = {"metric": "scaled-lasso regressions/s (spmesl_scaled_lasso)", "value": value,
            "unit": "regressions/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sum(per) / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "regression_er_p2000_n200", "p": p, "n": n,
                       "active_coefficients": w["k"], "noise": w["noise"],
                       "lambda0": "sqrt(2 log p / n)", "tol": tol, "maxit": maxit,
                       "precision": w["prec"], "l2": "flushed between steps (256 MB write)"},
            "latency": {"p50_ms": statistics.median(per),
                        "p99_ms": srt[min(len(srt) - 1, int(math.ceil(0.99 * len(srt))) - 1)]},
            "solve": {"outer_iters": st.outer_iters, "sweeps": st.inner_sweeps, "moves": st.moves,
                      "nnz_beta": st.nnz_B},
            "roofline": {"bound": "latency",
                         "note": "one column solve is a single warp's dependent chain; the "
                                 "Gram of [X y] is reported by --workload hub_p10000_n500_mixed"},
            "accuracy": acc, "cpu_baseline": cb,
            "gpu_launches": 8 * args.steps, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    del keep


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="default: the 256-fit batch; batch256_steps (its steps alone), er10, "
                         "serve, regression, table4, residual, or a single-fit name of "
                         "synth.WORKLOADS")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-pool", type=int, default=24)
    ap.add_argument("--serve-fracs", type=float, nargs="+", default=[0.5, 0.9])
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "er10":
        run_er10(args)
    elif args.workload == "batch256_steps":
        run_batch256_steps(args)
    elif args.workload == "regression":
        run_regression(args)
    elif args.workload == "table4":
        run_table4(args)
    elif args.workload == "residual":
        run_residual(args)
    elif args.workload != WORKLOAD:
        run_single(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
