#!/usr/bin/env python
"""Benchmark of Sparse Frequent Directions on one GB300 (or N, one process each).

Workload (one step = one whole stream sketched, every hot-path stage run):
  n = 1,000,000 rows, d = 50,000, l = 100, nnz/row ~ Poisson(50), columns
  Zipf(1.1) without repeats, planted rank-20 signal (10 * 0.8^t) + 0.1 N(0,1),
  fp32 values / int32 indices, seed = rank. 20 buffers of 50,000 rows each go
  through BoostedSparseShrink (SimultaneousIteration with q = 13, VerifySpectral)
  and DenseShrink. The CSR stream (~400 MB) is larger than L2, so successive
  steps start cold.

Metric: input nnz/s (whole job, all ranks). `value` times the device-resident
stream (`sfd_append_rows` with device pointers + `sfd_sketch`); `e2e` times the
same call sequence from pinned host buffers (host->device copy of the stream
and device->host copy of the sketch inside the timed region).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
stream: its first 50,000 rows, i.e. the first buffer exactly as the stream
closes it (m = d = 50,000, q = 13), through BSSh + DSh.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(name="c2", n=1_000_000, d=50_000, ell=100, k=20, mu=50, zipf=1.1, rank=20,
                scale=10.0, decay=0.8, noise=0.1)
DESC = ("SFD stream n=1,000,000 d=50,000 l=100, nnz/row~Poisson(50), Zipf(1.1) columns, "
        "planted rank-20 (10*0.8^t) + 0.1 N(0,1), fp32 CSR")
METRIC = "SFD input nnz/sec at fixed cov-error"
REF_SAMPLE_ROWS = 50_000   # one whole buffer of the stream (rows = d)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rows", type=int, default=WORKLOAD["n"], help="stream length (default: full)")
    ap.add_argument("--no-check", action="store_true", help="skip the cov-err evaluation")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--experiment", default=None, choices=["paper-table1"],
                    help="instead of the benchmark: the paper's Sec. 5 comparison of SFD and "
                         "FrequentDirections on its synthetic data, over the ranges of Table 1")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer timing")
    ap.add_argument("--no-forms", action="store_true",
                    help="time only the chosen form (not the plain FP32, verify-off and "
                         "learned-q forms)")
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1],
                    help="0: FP32 throughout; 1: tensor-core (TF32) Gram and X R^-1 in the "
                         "orthonormalisations of all but the last power iteration")
    ap.add_argument("--slots", type=int, default=0, help="buffers in flight (0: library default)")
    ap.add_argument("--q-mode", default="fixed", choices=["fixed", "learned"],
                    help="power count per buffer: the fixed schedule, or the learned predictor "
                         "(trained before the timed region on labelled streams of other seeds)")
    ap.add_argument("--train-rows", type=int, default=400_000,
                    help="rows of each labelled training stream (learned q)")
    ap.add_argument("--train-streams", type=int, default=2)
    ap.add_argument("--q-margin", type=float, default=3.0,
                    help="learned q: q = ceil(prediction + margin), clamped to the schedule")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def over_ranks(x, world, op="max"):
    """x reduced over the ranks of the process group ("max" or "sum"); x itself
    when world == 1. Host-side (gloo): timings and unit counts only."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_all_ranks, steps, ms):
    """Units per second of the whole job: every rank's units of `steps` steps
    over the slowest rank's time (ms)."""
    return units_all_ranks * steps / (ms / 1e3)


def make_stream(rows, seed):
    from paper_1602_00412_gb300 import synth
    w = WORKLOAD
    return synth.planted(rows, w["d"], w["mu"], w["zipf"], w["rank"], w["scale"], w["decay"],
                         w["noise"], seed, name="c2")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- checks
def cov_err_check(X, B, k):
    """cov-err = ||A^T A - B^T B||_2 / ||A||_F^2 and the FD bound ||A - A_k||_F^2/(l - k)
    (Sec. 5 measures; evaluated with scipy on the host)."""
    import numpy as np
    import scipy.sparse.linalg as spla
    A = X.to_scipy()
    Bd = B.astype(np.float64)
    d = A.shape[1]

    def mv(x):
        x = np.asarray(x).reshape(-1)
        return A.T @ (A @ x) - Bd.T @ (Bd @ x)
    if not np.all(np.isfinite(Bd)):
        raise RuntimeError("sketch has non-finite entries")
    op = spla.LinearOperator((d, d), matvec=mv, dtype=np.float64)
    # A^T A - B^T B is PSD (Prop. 1), so its 2-norm is its largest eigenvalue;
    # Lanczos from a seeded start vector, restarted from another if it breaks down
    lam = None
    for attempt in range(3):
        v0 = np.random.default_rng(attempt).standard_normal(d)
        try:
            lam = spla.eigsh(op, k=1, which="LA", tol=1e-4, ncv=40, v0=v0,
                             return_eigenvectors=False)[0]
            break
        except spla.ArpackError:
            continue
    if lam is None:
        raise RuntimeError("Lanczos did not converge from three start vectors")
    fro2 = float(A.multiply(A).sum())
    s = spla.svds(A, k=k, tol=1e-4, return_singular_vectors=False)
    tail = fro2 - float((s ** 2).sum())
    ell = B.shape[0]
    return {"cov_err": float(lam / fro2), "cov_norm": float(lam),
            "fd_bound": float(tail / (ell - k)), "k": k}


# ------------------------------------------------------------ cpu baseline
def run_oracle_sample(rows, seed, threads):
    """Time the FP64 oracle on the first `rows` rows of the stream in a fresh
    process (spawned, BLAS limited to `threads`). Returns (seconds, nnz)."""
    code = (
        "import sys,time,json; sys.path.insert(0,%r)\n"
        "import bench\n"
        "from oracle import sfd as O\n"
        "X = bench.make_stream(%d, %d)\n"
        "t=time.perf_counter(); O.sfd_stream(X.indptr,X.indices,X.values,%d,%d,%d)\n"
        "print(json.dumps({'sec': time.perf_counter()-t, 'nnz': X.nnz}))\n"
    ) % (ROOT, rows, seed, WORKLOAD["d"], WORKLOAD["ell"], seed)
    env = dict(os.environ)
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(threads)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    return out["sec"], out["nnz"]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


# DRAM bytes per launch of the SpMM stage (dram__bytes_read.sum +
# dram__bytes_write.sum averaged over the stage's launches of one ncu capture),
# valid while csrc/k_sparse.cu hashes to the key; the ncu summary in profiles/
# gives the command and the per-kernel figures.
SPMM_TRAFFIC = {"6fbc0266d65e63bf": 33.85e6}


def traffic_record():
    """DRAM bytes per SpMM-stage launch for the current sparse-kernel source,
    or None when the kernels changed since the counters were taken."""
    src = os.path.join(ROOT, "paper_1602_00412_gb300", "csrc", "k_sparse.cu")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return SPMM_TRAFFIC.get(h)


def oracle_golden(rows, seed):
    """The FP64 oracle's cov-err on this stream, stored by
    tests/golden/make_c2_oracle.py (only for the full stream of seed 0)."""
    p = os.path.join(ROOT, "tests", "golden", "c2_oracle.json")
    try:
        with open(p) as f:
            g = json.load(f)
    except (OSError, ValueError):
        return None
    return g if (g.get("rows") == rows and g.get("seed") == seed) else None


# ------------------------------------------------------------------ arms
def ref_sample_rows(steps, warmup):
    """Rows of the stream one reference step runs: the stream's first buffer
    (50,000 rows, ~10-25 s of CPU) while the whole run stays within a few
    minutes (about 8 such samples), else a proportionally shorter prefix
    (one flushed buffer of fewer rows)."""
    n = steps + warmup
    if n <= 8:
        return REF_SAMPLE_ROWS
    return max(10_000, (REF_SAMPLE_ROWS * 8 // n) // 1000 * 1000)


def reference_arm(args, rank, world):
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    rows = ref_sample_rows(args.steps, args.warmup)
    times, nnz = [], 0
    for i in range(args.warmup + args.steps):
        sec, nnz = run_oracle_sample(rows, 0, threads)
        if i >= args.warmup:
            times.append(sec)
    tot = sum(times)
    val = nnz * len(times) / tot
    sample = ("first %d rows of the c2 stream (%d nnz) through BSSh + DSh in FP64 (%s)" % (
        rows, nnz, "its first buffer, m = d, q = 13" if rows == REF_SAMPLE_ROWS
        else "one flushed buffer of %d rows" % rows))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "nnz/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": DESC, "sample_rows": rows},
            "cpu_baseline": {"value": val, "unit": "nnz/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def train_q_model(sfd, args, d, ell):
    """Labelled streams of other seeds (q_mode 2), then Adam on the GPU."""
    import numpy as np
    t0 = time.time()
    feats, labels = [], []
    for s in range(args.train_streams):
        Xt = make_stream(args.train_rows, 1000 + s)
        tc = sfd.SFD(d, ell, 1000 + s, q_mode=2, precision=args.precision, slots=args.slots)
        tc.append(Xt.indptr, Xt.indices, Xt.values)
        tc.sketch()
        F, L, _ = tc.q_log()
        tc.close()
        feats.append(F)
        labels.append(L)
    F, L = np.concatenate(feats), np.concatenate(labels)
    theta, loss = sfd.sfd_q_train(F, L, sfd.q_init_params(0), epochs=300, batch=8, lr=3e-3)
    info = {"train_buffers": int(len(L)), "labels": sorted(set(int(x) for x in L)),
            "train_loss": loss, "train_s": round(time.time() - t0, 1),
            "train_streams": "%d x %d rows, seeds 1000+" % (args.train_streams, args.train_rows)}
    return theta, info


class Form:
    """One form of the path timed on the same stream: `value` with the stream
    resident in HBM, `e2e` from pinned host buffers (H2D of the stream and D2H
    of the sketch inside the timed region)."""

    def __init__(self, name, **opts):
        self.name, self.opts = name, opts
        self.ms = self.ms_e2e = None
        self.stats, self.clocks, self.B = None, None, None


def time_form(form, sfd, io, args, world, stream, theta=None, clocks_index=None, e2e=True):
    import torch
    import torch.distributed as dist
    d, ell, rank = io["d"], io["ell"], io["rank"]
    ctx = sfd.SFD(d, ell, rank, cuda_stream=stream.cuda_stream, slots=args.slots,
                  q_margin=args.q_margin, **form.opts)
    if form.opts.get("q_mode") == 1:
        ctx.set_q_model(theta)

    def step_device():
        ctx.reset()
        ctx.append(io["ip_d"], io["ix_d"], io["vv_d"])
        ctx.sketch(io["B_d"])

    def step_host():
        ctx.reset()
        ctx.append(io["ip_h"], io["ix_h"], io["vv_h"])
        ctx.sketch(io["B_h"])

    def timed(fn, steps):
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        return over_ranks(e0.elapsed_time(e1), world, "max")

    for _ in range(args.warmup):
        step_device()
    clk = ClockSampler(clocks_index) if clocks_index is not None else None
    if clk:
        clk.start()
    form.ms = timed(step_device, args.steps)
    form.stats = ctx.stats()          # counters of the last timed step (each step resets)
    if clk:
        form.clocks = clk.stop()
    form.B = io["B_d"].cpu().numpy()
    if e2e:
        for _ in range(max(1, args.warmup // 3)):
            step_host()
        form.ms_e2e = timed(step_host, args.steps)
    ctx.close()
    return form


def spmm_roofline_one_slot(sfd, io, args, stream, peak):
    """The SpMM stage's own duration: the stream once more with one buffer in
    flight (slots = 1), every sparse-product launch timed by CUDA events on
    the stream it runs on; there it shares the GPU only with the merge
    stream's DenseShrink."""
    import torch
    iso = sfd.SFD(io["d"], io["ell"], io["rank"], cuda_stream=stream.cuda_stream, profile=1,
                  precision=args.precision, slots=1)
    iso.append(io["ip_d"], io["ix_d"], io["vv_d"])
    iso.sketch(io["B_d"])
    torch.cuda.synchronize()
    st = iso.stats()
    iso.close()
    if not st["spmm_launches"]:
        return None
    per_bytes = st["spmm_bytes"] / st["spmm_launches"]
    per_s = st["spmm_ms"] / 1e3 / st["spmm_launches"]
    return {"achieved": per_bytes / per_s / 1e9, "launches": st["spmm_launches"],
            "bytes_per_launch": per_bytes, "avg_launch_us": per_s * 1e6}


def ours_arm(args, rank, world, local):
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    from paper_1602_00412_gb300.build import build
    build()
    from paper_1602_00412_gb300 import sfd

    X = make_stream(args.rows, rank)
    w = WORKLOAD
    d, ell = w["d"], w["ell"]
    stream = torch.cuda.current_stream()
    io = {"d": d, "ell": ell, "rank": rank,
          "ip_d": torch.from_numpy(X.indptr).cuda(), "ix_d": torch.from_numpy(X.indices).cuda(),
          "vv_d": torch.from_numpy(X.values).cuda(), "B_d": torch.empty((ell, d), device="cuda"),
          "ip_h": torch.from_numpy(X.indptr).pin_memory().numpy(),
          "ix_h": torch.from_numpy(X.indices).pin_memory().numpy(),
          "vv_h": torch.from_numpy(X.values).pin_memory().numpy(),
          "B_h": torch.empty((ell, d), dtype=torch.float32).pin_memory().numpy()}
    theta, qinfo = (None, None)
    if args.q_mode == "learned" or not args.no_forms:
        theta, qinfo = train_q_model(sfd, args, d, ell)
    learned = args.q_mode == "learned"
    chosen = Form("chosen", precision=args.precision, q_mode=1 if learned else 0, profile=1)
    time_form(chosen, sfd, io, args, world, stream, theta, clocks_index=local, e2e=not args.no_e2e)
    forms = [chosen]
    if not args.no_forms:
        # the plain FP32 path (fixed schedule), and SparseShrink without
        # VerifySpectral as in the paper's experiments (Sec. 5)
        if args.precision != 0 or learned:
            forms.append(time_form(Form("plain", precision=0), sfd, io, args, world, stream,
                                   e2e=not args.no_e2e))
        forms.append(time_form(Form("verify_off", precision=args.precision, verify=0,
                                    q_mode=1 if learned else 0), sfd, io, args, world, stream,
                               theta, e2e=False))
        if not learned:  # the learned power count (network trained above)
            forms.append(time_form(Form("learned", precision=args.precision, q_mode=1), sfd, io,
                                   args, world, stream, theta, e2e=False))
    nnz_all = int(over_ranks(X.nnz, world, "sum"))   # each rank's stream has its own seed
    rate = lambda ms: whole_job_rate(nnz_all, args.steps, ms) if ms else None
    st = chosen.stats
    peak, peak_kind = peaks()
    contended = None
    if st["spmm_launches"]:
        per_s = st["spmm_ms"] / 1e3 / st["spmm_launches"]
        contended = {"achieved": st["spmm_bytes"] / st["spmm_launches"] / per_s / 1e9,
                     "avg_launch_us": per_s * 1e6, "launches_per_step": st["spmm_launches"]}
    iso = spmm_roofline_one_slot(sfd, io, args, stream, peak)
    roof = {"kernel": "SpMM stage: k_spmm_h (fp16 blocks) / k_spmm (fp32) for A'X (CSR) and "
                      "A'^T Y (CSC), incl. split fix-up; duration from the one-slot run",
            "bound": "hbm", "achieved": iso["achieved"] if iso else None, "peak": peak,
            "unit": "GB/s", "frac": (iso["achieved"] / peak) if iso else None,
            "peak_kind": "of %s" % peak_kind, "traffic": traffic_record(),
            "algorithmic_bytes_per_launch": iso["bytes_per_launch"] if iso else None,
            "avg_launch_us": iso["avg_launch_us"] if iso else None,
            "achieved_contended": contended["achieved"] if contended else None,
            "frac_contended": contended["achieved"] / peak if contended else None,
            "avg_launch_us_contended": contended["avg_launch_us"] if contended else None,
            "launches_per_step": st["spmm_launches"]}
    out = {"metric": METRIC, "value": rate(chosen.ms), "unit": "nnz/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": chosen.ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if args.precision == 0 else "tf32+f32", "data": "synthetic",
           "config": {"workload": DESC, "rows": X.n, "d": d, "ell": ell, "nnz_per_rank": X.nnz,
                      "precision": ["fp32", "mixed-tf32"][args.precision],
                      "q_mode": args.q_mode, "q_model": qinfo, "q_margin": args.q_margin,
                      "buffers_per_step": st["buffers"], "attempts_per_step": st["attempts"],
                      "q_per_attempt": st["q_total"] / max(1, st["attempts"]),
                      "l2": "inputs larger than L2 (CSR stream %.0f MB per rank)" % (
                          (X.indptr.nbytes + X.indices.nbytes + X.values.nbytes) / 1e6),
                      "parallelism": "independent streams per GPU (weak)" if world > 1 else "1 GPU"},
           "rows_per_s": X.n * world * args.steps / (chosen.ms / 1e3),
           "e2e": {"value": rate(chosen.ms_e2e), "unit": "nnz/s",
                   "h2d_bytes_per_step": int(X.indptr.nbytes + X.indices.nbytes + X.values.nbytes),
                   "d2h_bytes_per_step": int(io["B_h"].nbytes)},
           "roofline": roof,
           "gpu_launches": int(st["kernel_launches"]) * args.steps,
           "gpu_launches_per_step": int(st["kernel_launches"]),
           "clocks": chosen.clocks}
    out["forms"] = {f.name: {"value": rate(f.ms), "e2e": rate(f.ms_e2e),
                             "ms_per_step": f.ms / args.steps,
                             "attempts_per_step": f.stats["attempts"],
                             "vs_rejects_per_step": f.stats["vs_rejects"],
                             "options": {k: v for k, v in f.opts.items() if k != "profile"}}
                    for f in forms}
    if "plain" in out["forms"]:
        out["plain"] = dict(out["forms"]["plain"])
        out["plain"]["chosen_over_plain"] = out["value"] / out["plain"]["value"]
    if rank == 0 and not args.no_check:
        g = oracle_golden(X.n, rank)
        acc = {}
        for f in forms:
            a = cov_err_check(X, f.B, w["k"])
            a["within_fd_bound"] = a["cov_norm"] <= a["fd_bound"]
            if g:
                a["cov_err_oracle"] = g["cov_err"]
                a["rel_to_oracle"] = a["cov_err"] / g["cov_err"] - 1.0
                a["within_2pct_of_oracle"] = abs(a["rel_to_oracle"]) <= 0.02
            acc[f.name] = a
        out["accuracy"] = dict(acc["chosen"])
        out["accuracy"]["forms"] = {k: v for k, v in acc.items() if k != "chosen"}
        out["accuracy"]["oracle"] = ("tests/golden/c2_oracle.json: FP64 oracle on the same stream"
                                     if g else "no stored oracle value for this stream")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        sec, nnz = run_oracle_sample(REF_SAMPLE_ROWS, 0, threads)
        out["cpu_baseline"] = {"value": nnz / sec, "unit": "nnz/s", "cores": threads,
                               "kind": "oracle",
                               "sample": "first %d rows (%d nnz) of the stream: its first buffer "
                                         "(m = d, q = 13) through BSSh + DSh, FP64 numpy/scipy, "
                                         "BLAS threads = host cores" % (REF_SAMPLE_ROWS, nnz)}
    if rank == 0:
        print(json.dumps(out), flush=True)

# ------------------------------------------------------- paper, Table 1
TABLE1_DEFAULT = {"n": 10000, "d": 1000, "ell": 50, "z": 100}
TABLE1_RANGES = {"n": [10000, 20000, 40000, 60000], "d": [1000, 2000, 4000, 6000],
                 "ell": [5, 10, 20, 50, 100], "z": [5, 10, 50, 100, 200, 500]}


def proj_err_check(A, B, k, tail):
    """proj-err = ||A - A V_k V_k^T||_F^2 / ||A - A_k||_F^2, V_k the top-k right
    singular vectors of B (Sec. 5, Measurements)."""
    import numpy as np
    _, _, Vt = np.linalg.svd(B.astype(np.float64), full_matrices=False)
    AV = A @ Vt[:k].T
    fro2 = float(A.multiply(A).sum())
    return (fro2 - float((np.asarray(AV) ** 2).sum())) / tail


def paper_table1(args):
    """The comparison of Sec. 5 on its synthetic data (+-1 entries, z per row,
    head of 1.5 z columns drawn w.p. 0.9), one parameter of Table 1 varied at a
    time: classical FrequentDirections (mode 1) against SFD with SparseShrink
    called directly (verify 0, as the paper runs it), both on this GPU; k = 10.
    Prints one JSON line per point."""
    import numpy as np
    import scipy.sparse.linalg as spla
    import torch
    from paper_1602_00412_gb300.build import build
    build()
    from paper_1602_00412_gb300 import sfd, synth
    k = 10
    for param, values in TABLE1_RANGES.items():
        for v in values:
            p = dict(TABLE1_DEFAULT, **{param: v})
            n, d, ell, z = p["n"], p["d"], p["ell"], p["z"]
            X = synth.headtail(n, d, z, 0)
            A = X.to_scipy()
            ip = torch.from_numpy(X.indptr).cuda()
            ix = torch.from_numpy(X.indices.astype(np.int32)).cuda()
            vv = torch.from_numpy(X.values.astype(np.float32)).cuda()
            fro2 = float(A.multiply(A).sum())
            kk = min(k, ell - 1)
            sv = spla.svds(A, k=kk, tol=1e-8, return_singular_vectors=False)
            tail = fro2 - float((sv ** 2).sum())
            line = {"experiment": "paper Table 1", "param": param, "n": n, "d": d, "ell": ell,
                    "nnz_per_row": z, "k": kk}
            for name, opts in (("fd", {"mode": 1}), ("sfd", {"verify": 0})):
                ctx = sfd.SFD(d, ell, 0, **opts)
                B = torch.empty((ell, d), device="cuda")
                times = []
                for rep in range(4):      # one warm-up, then the median of three
                    ctx.reset()
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    ctx.append(ip, ix, vv)
                    ctx.sketch(B)
                    torch.cuda.synchronize()
                    if rep:
                        times.append(time.perf_counter() - t0)
                ctx.close()
                Bh = B.cpu().numpy()
                acc = cov_err_check(X, Bh, kk)
                line[name] = {"seconds": statistics.median(times), "cov_err": acc["cov_err"],
                              "proj_err": proj_err_check(A, Bh, kk, tail)}
            line["fd_over_sfd_time"] = line["fd"]["seconds"] / line["sfd"]["seconds"]
            print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    if args.experiment == "paper-table1":
        if rank == 0:
            paper_table1(args)
    elif args.impl == "reference":
        reference_arm(args, rank, world)
    else:
        ours_arm(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
