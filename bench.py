#!/usr/bin/env python
"""RkMIPS throughput on one GB300 (exact mode, results identical to the FP64 oracle).

Headline workload (default): the large served index, n = 1,000,000 items, m = 2,000,000 users,
d = 128, rank-50 factor-model vectors with log-normal(0, 0.7) norms and 5% of the items at 3x
norm (seed 0); Cone-Tree leaf size 256; 64 SA-ALSH tables of 16-bit codes.  One step = one
batch of 10,000 RkMIPS requests (5,000 item queries, each at k = 10 and k = 50) through the
whole query path: query preparation, block pass (Lemma 2), tensor-core user pass (A4/A8),
kMIPS decisions (A5/A6), double-precision re-score, compaction.  The index (Alg. 4) is built
once, before timing, with exact thresholds (|P'| = n); the paper's |P'| = 4 k_max is timed
beside it as a variant.

  value    queries/s with Q, ks and the output in HBM (CUDA events on the call's stream)
  e2e      queries/s through the same C-ABI call with the requests and the answers in pinned
           host memory, which the kernels read and write in place (transfers inside the call)
  roofline the dominant kernel of the step against its bound
  cpu_baseline  the FP64 oracle on the host cores: (i) brute force per query, (ii) with the
           thresholds tau_u cached, both on bounded samples of users

With --impl reference the FP64 oracle itself is timed (the CPU reference arm).
Multi-GPU (torchrun): every rank holds a replica of the index and answers its own batch
(no collective on the data path); value = all ranks' queries / max time (weak scaling).
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

import workload  # noqa: E402

METRIC = "RkMIPS queries/s (exact, F1=1 vs FP64 oracle)"
UNIT = "queries/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT = 152
FP32_LANES_PER_SM = 128
N_TABLES, CODE_BITS, LEAF = 64, 16, 256


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c5")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sample-users", type=int, default=2000,
                    help="seeded users the FP64 oracle decides for the correctness gate (plus every "
                         "user the GPU returns)")
    ap.add_argument("--sustain-s", type=float, default=2.0,
                    help="seconds of back-to-back steps after the timed ones (clock samples under load)")
    ap.add_argument("--serve-rates", default="1000,2000,5000,10000,20000,50000,100000,200000")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--m", type=int, default=0, help="users (0: the workload's); a smaller case of the same recipe")
    ap.add_argument("--n", type=int, default=0, help="items (0: the workload's)")
    ap.add_argument("--nq", type=int, default=0, help="item queries (0: the workload's)")
    ap.add_argument("--sweep", action="store_true",
                    help="instead of the bench line, one JSON line of parameter sweeps on C2-shaped data")
    return ap.parse_args()


def whole_job_value(local_ms_total, queries_per_rank_step, steps, world, all_reduce_max):
    """Weak scaling: every rank answers its own batch of the same size each step; the job's
    time is the slowest rank's, and the value counts every rank's queries."""
    t_ms = float(all_reduce_max(float(local_ms_total)))
    return queries_per_rank_step * steps * world / (t_ms / 1e3), t_ms


def torch_max_reducer(device):
    import torch
    import torch.distributed as dist

    def red(x):
        t = torch.tensor([x], dtype=torch.float64, device=device)
        if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return t.item()
    return red


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def load_peaks():
    try:
        with open(PEAKS_PATH) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 20 ms while active; summary over the samples under load."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons, busy = [], [], set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                clk, cmax, util = float(parts[1]), float(parts[2]), float(parts[9])
            except ValueError:
                continue
            smax.append(cmax)
            if util > 0:
                busy += 1
                sm.append(clk)
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not smax:
            return None
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(smax), "samples_under_load": busy}


# ---------------------------------------------------------------- DRAM traffic from profiles/
def kernel_source_hash(path: str, kernel: str):
    """sha256 (16 hex digits) of a kernel's definition text: from the line that starts its
    declaration (a template line, or the __global__ line) to the brace that closes its body."""
    lines = open(path).read().split("\n")
    for i, line in enumerate(lines):
        if kernel + "(" in line and "<<<" not in line and not line.lstrip().startswith("//"):
            j = i
            while j > 0 and "__global__" not in lines[j]:
                j -= 1
            if "__global__" not in lines[j]:
                continue
            if j > 0 and lines[j - 1].startswith("template"):
                j -= 1
            depth, started, k = 0, False, i
            while k < len(lines):
                depth += lines[k].count("{") - lines[k].count("}")
                started = started or "{" in lines[k]
                if started and depth == 0:
                    break
                k += 1
            return hashlib.sha256("\n".join(lines[j:k + 1]).encode()).hexdigest()[:16]
    return None


def kernel_traffic(kernel: str, workload_name: str):
    """DRAM bytes per launch from a committed ncu summary (profiles/traffic.json), if the
    kernel's definition is unchanged since it was taken (matched by the hash of its source)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(f"{kernel}@{workload_name}")
        src = os.path.join(ROOT, "paper_2211_12751_gb300", "csrc", rec["source"])
        if kernel_source_hash(src, kernel) == rec["kernel_sha256_16"]:
            return rec["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


# ---------------------------------------------------------------- the FP64 oracle on the host
def oracle_gate(W, host, qrows, K, sample_n, nq_check=2, max_returned=2000):
    """The FP64 oracle's membership (Def. 1, count rule) for a seeded sample of users plus
    every user the GPU returned, for the first nq_check distinct queries of the batch, at
    every k they were asked at; compared with the GPU's answers.  The timing of these counts
    is also the brute-force CPU baseline (i): one count per user answers all of the query's k."""
    import oracle
    sample = workload.sample_rows(W.m, sample_n, seed=22)
    distinct = np.unique(qrows)[:nq_check]
    agree, checked, t_count, users_counted, mismatches = True, 0, 0.0, 0, 0
    for qi in distinct:
        rows = np.flatnonzero(qrows == qi)
        returned = np.unique(np.concatenate([host[r] for r in rows])) if len(rows) else np.zeros(0, np.int64)
        users = np.union1d(sample, returned[:max_returned]).astype(np.int64)
        t0 = time.perf_counter()
        c = oracle.count_above(W.U, W.P, W.P[W.query_idx[qi]], users)
        t_count += time.perf_counter() - t0
        users_counted += len(users)
        for r in rows:
            got = np.isin(users, host[r])
            want = c < K[r]
            mismatches += int(np.count_nonzero(got != want))
            agree &= bool(np.array_equal(got, want))
            checked += len(users)
    per_user = t_count / max(1, users_counted)
    ks_per_query = len(rows)
    qps_i = ks_per_query / (per_user * W.m)
    return {"agree": agree, "mismatches": mismatches, "checked_memberships": checked,
            "queries": int(len(distinct)), "sample_users": int(len(sample)),
            "seconds": t_count, "per_user_s": per_user, "qps": qps_i, "threads": oracle.threads()}


def cached_tau_baseline(W, ks, tau_users=256, pass_users=100000, queries=40):
    """CPU baseline (ii): RkMIPS with the thresholds tau_u(1..k_max) cached (Alg. 4's arrays
    taken to |P'| = n), so a query costs one FP64 <u,q> per user: the oracle's
    oracle_rkmips_tau, as it stands (one thread).  tau is computed for a seeded sample of
    users (its cost, per user, is reported as the cache's build cost); the per-query pass is
    timed over pass_users users with those thresholds repeated, and scaled to all m users."""
    import oracle
    users = workload.sample_rows(W.m, tau_users, seed=23)
    t0 = time.perf_counter()
    tau = oracle.tau(W.U, W.P, 50, users)
    t_tau = time.perf_counter() - t0
    nu = min(pass_users, W.m)
    Us = np.ascontiguousarray(W.U[:nu])
    tau_rep = np.ascontiguousarray(np.resize(tau, (nu, tau.shape[1])))
    qidx = W.query_idx[:queries]
    t0 = time.perf_counter()
    for i, qi in enumerate(qidx):
        oracle.rkmips_tau(Us, tau_rep, W.P[qi], int(ks[i % len(ks)]))
    t_pass = time.perf_counter() - t0
    per_query_all = t_pass / len(qidx) * (W.m / nu)
    return {"qps": 1.0 / per_query_all, "cores": 1, "tau_build_s_per_user": t_tau / len(users),
            "tau_build_threads": oracle.threads(),
            "sample": (f"tau_u(1..50) computed for {len(users)} seeded users ({t_tau:.1f} s on "
                       f"{oracle.threads()} threads); the per-query pass (one FP64 <u,q> and a compare per user) "
                       f"timed for {len(qidx)} queries over {nu} users, scaled to {W.m}")}


def config_block(W, extra=None):
    r = W.recipe
    if r["kind"] in ("mf", "nmf"):
        dist = (f"{r['kind']} rank-50 lognormal(0,{r['sigma']}), {int(100 * r['boost_frac'])}% items x{r['boost']:g}, "
                f"seed {r['seed']}")
    else:
        dist = f"gauss sigma {r['sigma']}, seed {r['seed']}"
    ks = list(map(int, W.ks)) if not isinstance(W.ks, str) else W.ks
    u_mb = W.m * ((W.d + 7) // 8 * 8) * 2 / 1e6
    cfg = {"workload": (f"{W.name}: n={W.n} items, m={W.m} users, d={W.d}, {dist}; "
                        f"{len(W.query_idx)} item queries x k in {ks}"),
           "queries_per_step": int(len(W.query_idx) * (len(W.ks) if W.every_k else 1)),
           "mode": "exact", "threshold_mode": "full (|P'| = n)", "precision": "bf16",
           "leaf_size": LEAF, "k_max": 50, "sa_alsh": f"{N_TABLES} tables x {CODE_BITS}-bit codes",
           "l2": (f"L2 flushed between timed steps (256 MiB write); users in BF16 {u_mb:.0f} MB "
                  f"({'larger' if u_mb > 129 else 'smaller'} than the 129 MB L2)")}
    if extra:
        cfg.update(extra)
    return cfg


def run_reference(args):
    """The CPU reference arm: the FP64 oracle's brute-force count on a bounded sample of users
    per step (about 2 s), scaled to all users."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    W = workload.make(args.workload)
    Q, K, qrows = W.requests()
    per_q = len(W.ks) if W.every_k else 1
    probe = workload.sample_rows(W.m, 64, seed=21)
    t0 = time.perf_counter()
    oracle.count_above(W.U, W.P, Q[0], probe)
    per_user = max(time.perf_counter() - t0, 1e-6) / len(probe)
    n_users = int(max(64, min(W.m, 2.0 / per_user)))
    distinct = np.unique(qrows)
    vals = []
    for step in range(args.warmup + args.steps):
        users = workload.sample_rows(W.m, n_users, seed=100 + step)
        q = W.P[W.query_idx[distinct[step % len(distinct)]]]
        t0 = time.perf_counter()
        oracle.count_above(W.U, W.P, q, users)
        t = time.perf_counter() - t0
        if step >= args.warmup:
            vals.append(per_q * (n_users / W.m) / t)
    v = float(np.mean(vals))
    sample = (f"per step: FP64 brute-force counts of {n_users} seeded users (of {W.m}) for one item query, "
              f"the count answering its {per_q} k values; scaled to all users")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_block(W),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- measurement on the GPU
def make_index(sah, Ud, Pd, stream, threshold, precision="bf16", tc=1, n_tables=N_TABLES, code_bits=CODE_BITS,
               leaf=LEAF, probe_radius=0, blocking=0, transform=0):
    """Alg. 4 from device copies of U and P; returns (index, build seconds).  threshold:
    "full" (|P'| = n), "paper" (|P'| = 4 k_max) or an integer |P'|."""
    import torch
    pp = (1 << 30) if threshold == "full" else (0 if threshold == "paper" else int(threshold))
    prec = {"bf16": sah.BF16, "fp8": sah.FP8, "fp32": sah.FP32}[precision]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ix = sah.Index(Ud, Pd, k_max=50, leaf_size=leaf, p_prime=pp, seed=0, precision=prec, n_tables=n_tables,
                   code_bits=code_bits, tc_user_pass=tc, probe_radius=probe_radius, blocking=blocking, transform=transform,
                   stream=stream)
    torch.cuda.synchronize()
    return ix, time.perf_counter() - t0


class Batch:
    """One batch of requests held on the device, its output buffers sized by a first call,
    and the C-ABI call itself (the binding's convenience wrapper would add a read of the
    total to the timed region)."""

    def __init__(self, ix, Q, K, dev, stream, modes=None):
        import torch
        self.ix, self.stream, self.nq = ix, stream, len(K)
        self.Q, self.K, self.modes = Q, K, modes
        self.host = ix.rkmips_batch(Q, K, modes=modes)
        self.total = sum(len(h) for h in self.host)
        self.Qd = torch.from_numpy(np.ascontiguousarray(Q)).to(dev)
        self.Kd = torch.from_numpy(np.ascontiguousarray(K, dtype=np.int32)).to(dev)
        self.Md = None if modes is None else torch.from_numpy(np.ascontiguousarray(modes, dtype=np.int32)).to(dev)
        self.out = torch.empty(max(self.total, 1), dtype=torch.int32, device=dev)
        self.offs = torch.empty(self.nq + 1, dtype=torch.int64, device=dev)

    def call(self):
        s = self.ix.raw_batch(self.Qd.data_ptr(), self.nq, self.Kd.data_ptr(),
                              self.Md.data_ptr() if self.Md is not None else None, 1, self.out.data_ptr(),
                              self.out.numel(), self.offs.data_ptr(), stream=self.stream)
        assert s == 0, s

    def timed(self, steps, warmup, flush):
        """CUDA-event times (ms) of `steps` calls after `warmup` untimed ones, L2 flushed
        before each timed call."""
        import torch
        for _ in range(warmup):
            self.call()
        times = []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(self.stream)
            self.call()
            e1.record(self.stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return times

    def stages(self, reps=3):
        """Per-stage CUDA-event times and launch counts (separate calls, events on)."""
        import torch
        self.ix.set_timing(True)
        ms, launches, st = np.zeros(8), np.zeros(8), None
        for _ in range(reps):
            torch.cuda.synchronize()
            self.call()
            torch.cuda.synchronize()
            st = self.ix.stats()
            ms += np.array(st["stage_ms"])
            launches += np.array(st["stage_launches"])
        self.ix.set_timing(False)
        return ms / reps, launches / reps, st

    def sustained(self, seconds):
        """Back-to-back calls for about `seconds` (no flush): requests/s under sustained load."""
        import torch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n = 0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        while time.perf_counter() - t0 < seconds:
            self.call()
            n += 1
        e1.record(self.stream)
        torch.cuda.synchronize()
        return self.nq * n / (e0.elapsed_time(e1) / 1e3), n

    def e2e(self, steps, warmup, flush):
        """The same call with the requests and the answers in pinned host memory (read and
        written in place by the kernels over the C2C link), CUDA events around the call."""
        import torch
        Qh = torch.from_numpy(np.ascontiguousarray(self.Q)).pin_memory()
        Kh = torch.from_numpy(np.ascontiguousarray(self.K, dtype=np.int32)).pin_memory()
        Mh = None if self.modes is None else torch.from_numpy(np.ascontiguousarray(self.modes, dtype=np.int32)).pin_memory()
        outh = torch.empty(max(self.total, 1), dtype=torch.int32).pin_memory()
        offh = torch.empty(self.nq + 1, dtype=torch.int64).pin_memory()
        times = []
        for i in range(warmup + steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            s = self.ix.raw_batch(Qh.data_ptr(), self.nq, Kh.data_ptr(), Mh.data_ptr() if Mh is not None else None, 0,
                                  outh.data_ptr(), outh.numel(), offh.data_ptr(), stream=self.stream)
            e1.record(self.stream)
            torch.cuda.synchronize()
            assert s == 0, s
            if i >= warmup:
                times.append(e0.elapsed_time(e1))
        assert int(offh[-1]) == self.total
        h2d = self.Q.nbytes + self.K.nbytes + (self.modes.nbytes if self.modes is not None else 0)
        d2h = (self.nq + 1) * 8 + self.total * 4
        return times, int(h2d), int(d2h)


def f1_sets(got, want):
    a, b = set(np.asarray(got).tolist()), set(np.asarray(want).tolist())
    return 1.0 if not a and not b else 2.0 * len(a & b) / (len(a) + len(b))


# ---------------------------------------------------------------- roofline of a step
STAGE_NAMES = ["prep", "block_pass", "user_pass", "kmips_decision", "compaction", "saalsh"]


def stage_rooflines(stage_ms, launches, st, d, dp, peaks, peak_kind):
    """The kernels that carry the stages, each against its bound, from the library's
    algorithmic counters (work per call) and its CUDA-event stage times:
      user pass (A4/A8)  tensor: 2 d flops per (user, distinct query vector) score computed, or
                         HBM: 2 d_pad + 12 bytes per user row streamed, whichever its
                         arithmetic intensity makes the bound;
      block pass (A3)    FP32 ALU: 2 d flops per (leaf, distinct query vector) <c_B, q>;
      kMIPS (A5)         tensor: 2 d flops per (survivor, item) scored before its decision.
    A call makes one launch of each per sub-batch (prep launches = sub-batches)."""
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    nsub = max(1.0, float(launches[0]))
    out = {}
    if st.get("tc_scores", 0) > 0 and stage_ms[6] > 0:
        # the user pass is tensor-bound when it scores many columns per user row it streams,
        # HBM-bound when (with the per-tile column prefix) it scores few: the bound is the one
        # its arithmetic intensity (flops per algorithmic byte) puts it under
        fl = 2.0 * d * st["tc_scores"]
        by = (2.0 * dp + 12.0) * st.get("tc_rows", 0)   # BF16 rows + 12 B of bounds per user and set
        t = stage_ms[6] / 1e3
        ridge = peaks["bf16_tflops"] * 1e12 / (peaks["hbm_gbs"] * 1e9)
        tensor = {"bound": "tensor", "unit": "TFLOP/s", "achieved": fl / t / 1e12, "peak": peaks["bf16_tflops"],
                  "peak_source": f"{peak_kind} (MEASURED_PEAKS.json bf16_tflops, burst)",
                  "algorithmic_flops_per_launch": fl / nsub}
        hbm = {"bound": "hbm", "unit": "GB/s", "achieved": by / t / 1e9, "peak": peaks["hbm_gbs"],
               "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
               "algorithmic_bytes_per_launch": by / nsub}
        ai = fl / by if by > 0 else float("inf")
        main, other = (tensor, hbm) if ai >= ridge else (hbm, tensor)
        other["frac"] = other["achieved"] / other["peak"]
        out["user_pass"] = dict(main, kernel="user_pass_tc_kernel", launch_ms=stage_ms[6] / nsub,
                                scores_per_call=st["tc_scores"], rows_per_call=st.get("tc_rows", 0),
                                arithmetic_intensity=ai, ridge=ridge, other_bound=other)
    if st.get("block_col_pairs", 0) > 0 and stage_ms[1] > 0:
        fl = 2.0 * d * st["block_col_pairs"]
        t = stage_ms[1] / 1e3
        out["block_pass"] = {"kernel": "block_filter_cols_kernel", "bound": "alu", "unit": "TFLOP/s",
                             "achieved": fl / t / 1e12, "peak": fp32_peak,
                             "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock (FMA)",
                             "algorithmic_flops_per_launch": fl / nsub, "launch_ms": stage_ms[1] / nsub,
                             "note": "stage time includes the column table and the mask clear"}
    if st.get("items_scanned", 0) > 0 and stage_ms[7] > 0:
        fl = 2.0 * d * st["items_scanned"]
        t = stage_ms[7] / 1e3
        out["kmips_decision"] = {"kernel": "verify_tc_kernel", "bound": "tensor", "unit": "TFLOP/s",
                                 "achieved": fl / t / 1e12, "peak": peaks["bf16_tflops"],
                                 "peak_source": f"{peak_kind} (MEASURED_PEAKS.json bf16_tflops, burst)",
                                 "algorithmic_flops_per_call": fl, "kernel_ms": stage_ms[7]}
    for v in out.values():
        v["frac"] = v["achieved"] / v["peak"]
    return out


def dominant(stage_ms, roofs):
    dom_i = int(np.argmax(stage_ms[1:6])) + 1
    name = STAGE_NAMES[dom_i]
    return name, roofs.get(name)


def measure_config(sah, W, Ud, Pd, dev, stream, flush, threshold, precision, steps, warmup, peaks, peak_kind,
                   tc=1, Q=None, K=None, modes=None, blocking=0, transform=0):
    """Build an index on W and time a batch (default: the workload's own requests)."""
    ix, build_s = make_index(sah, Ud, Pd, stream, threshold, precision, tc=tc, blocking=blocking,
                             transform=transform)
    if Q is None:
        Q, K, _ = W.requests()
    b = Batch(ix, Q, K, dev, stream, modes=modes)
    times = b.timed(steps, warmup, flush)
    sms, lau, st = b.stages()
    roofs = stage_rooflines(sms, lau, st, W.d, (W.d + 3) // 4 * 4, peaks, peak_kind)
    ist = ix.stats()
    rec = {"index_build_s": build_s, "queries_per_step": len(K), "value": len(K) / (np.mean(times) / 1e3),
           "ms_per_step": float(np.mean(times)), "stages_ms": {nm: float(sms[i]) for i, nm in enumerate(STAGE_NAMES)},
           "stage_counts": {k: st[k] for k in ("block_pairs_total", "block_pairs_kept", "users_in_kept_blocks",
                                               "users_scored", "tc_scores", "pairs_rescored", "survivors",
                                               "fp64_rescored", "items_scanned", "results")},
           "rooflines": roofs}
    if ist.get("build_gemm_ms", 0) > 0:
        rec["index_gemm_ms"] = ist["build_gemm_ms"]
    return ix, b, rec


# ---------------------------------------------------------------- serving
def serve_stream(sah, ix, W, rate, count, seed=1, max_batch=512, workers=2):
    """Poisson arrivals (k uniform in 1..50, modes half exact, half SA-ALSH, item queries)
    through the continuous-batching server.  Latencies are the library's submit-to-completion
    times per request; a request's completion time is its submit time plus that latency, and
    the throughput counts the requests over the span from the first arrival to the last
    completion.  Results are polled in submission order (the latencies do not depend on it)."""
    import collections
    arrivals = workload.poisson_arrivals(count, rate, seed=seed)
    rng = np.random.default_rng(seed + 1)
    qrows = rng.integers(0, W.n, count)
    ks = rng.integers(1, 51, count)
    modes = rng.integers(0, 2, count)
    srv = sah.Server(ix, max_slots=max(4096, count), max_batch=max_batch, workers=workers)
    lat, done_at = [], []
    sub_at = np.zeros(count)
    pending = collections.deque()
    t_start = time.perf_counter()
    i = 0
    while i < count or pending:
        now = time.perf_counter() - t_start
        while i < count and arrivals[i] <= now:
            sub_at[i] = time.perf_counter() - t_start
            pending.append((i, srv.submit(W.P[qrows[i]], int(ks[i]), int(modes[i]))))
            i += 1
        while pending:
            j, t = pending[0]
            r = srv.poll(t)
            if r is None:
                break
            lat.append(r[1])
            done_at.append(sub_at[j] + r[1])
            pending.popleft()
    info = srv.info()
    srv.stop()
    span = max(done_at) - float(arrivals[0])
    lat = np.array(lat) * 1e3
    return {"offered_rate": rate, "requests": count, "throughput_qps": count / span,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "late_submits_ms_p99": float(np.percentile(sub_at - arrivals, 99) * 1e3),
            "mean_batch": info["batched_requests"] / max(1, info["batches"]), "max_batch": info["max_batch_seen"],
            "batches": info["batches"], "admission_splits": info["split_ticks"]}


def run_serving(sah, dev, stream, rates, count):
    """The serving workload: C4 (n 100,000 items, m 1,000,000 users, d 100) with the paper's
    |P'| = 4 k_max, so that SA-ALSH-mode requests take Alg. 2 for their survivors; one Poisson
    stream per offered rate; the knee is the largest offered rate the server still delivers
    (throughput within 5% of it)."""
    import torch
    W = workload.make("c4")
    Ud, Pd = torch.from_numpy(W.U).to(dev), torch.from_numpy(W.P).to(dev)
    ix, build_s = make_index(sah, Ud, Pd, stream, "paper")
    del Ud, Pd
    pts = [serve_stream(sah, ix, W, float(r), count) for r in rates]
    ix.close()
    kept = [p["offered_rate"] for p in pts if p["throughput_qps"] >= 0.95 * p["offered_rate"]]
    return {"workload": (f"c4: n={W.n} items, m={W.m} users, d={W.d}, mf rank-50 lognormal(0,0.7), 5% items x3, "
                         f"seed 0; paper |P'| = 200; {count} requests per rate, k uniform 1..50, "
                         f"modes 50/50 exact / SA-ALSH, item queries; 2 workers, max batch 512"),
            "index_build_s": build_s, "points": pts,
            "knee_offered_rate": max(kept) if kept else None,
            "saturation_qps": max(p["throughput_qps"] for p in pts)}


# ---------------------------------------------------------------- parameter sweeps
def run_sweeps(sah, dev, stream, flush, steps=5):
    """The paper's Fig. 1 row 3 and Figs. 3-5 on C2-shaped synthetic data: leaf size N_0
    (exact mode), and for SA-ALSH mode the probe radius (k = 10), the interval ratio b and the
    table count K, each with its F1 against the exact answers of the same index (which equal
    the FP64 oracle's, as the GPU tests check).  |P'| = 200, BF16, 16-bit codes."""
    import torch
    W = workload.make("c2")
    Q, K, _ = W.requests()
    Ud, Pd = torch.from_numpy(W.U).to(dev), torch.from_numpy(W.P).to(dev)
    base = dict(leaf_size=256, n_tables=128, b=0.5, probe_radius=0)

    def point(Qs, Ks, saalsh, **over):
        prm = dict(base, **over)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ix = sah.Index(Ud, Pd, k_max=50, leaf_size=prm["leaf_size"], p_prime=0, seed=0, precision=sah.BF16,
                       n_tables=prm["n_tables"], code_bits=16, tc_user_pass=1, b=prm["b"],
                       probe_radius=prm["probe_radius"], stream=stream)
        torch.cuda.synchronize()
        rec = dict(over, index_build_s=time.perf_counter() - t0)
        bx = Batch(ix, Qs, Ks, dev, stream)
        tx = bx.timed(steps, 3, flush)
        rec["exact"] = {"queries_per_s": len(Ks) / (np.mean(tx) / 1e3), "ms_per_batch": float(np.mean(tx))}
        if saalsh:
            modes = np.full(len(Ks), sah.SAALSH, np.int32)
            bs = Batch(ix, Qs, Ks, dev, stream, modes=modes)
            ts = bs.timed(steps, 3, flush)
            f1s = [f1_sets(a, b) for a, b in zip(bs.host, bx.host)]
            rec["saalsh"] = {"queries_per_s": len(Ks) / (np.mean(ts) / 1e3), "ms_per_batch": float(np.mean(ts)),
                             "f1_vs_exact": float(np.mean(f1s)), "min_f1": float(np.min(f1s))}
        ix.close()
        return rec

    k10 = K == 10
    out = {"workload": config_block(W)["workload"], "base": base,
           "leaf_size": [point(Q, K, False, leaf_size=v) for v in (32, 64, 128, 256)],
           "probe_radius": [point(Q[k10], K[k10], True, probe_radius=v) for v in (0, 1, 2)],
           "b": [point(Q, K, True, b=v) for v in (0.3, 0.5, 0.7, 0.9)],
           "n_tables": [point(Q, K, True, n_tables=v) for v in (32, 64, 128)]}
    return {"sweep": out}


# ---------------------------------------------------------------- variants
def c3_accuracy(W, host, qrows, K, rec, cband):
    """C3 (the precision configuration): membership against the FP64 oracle on a seeded sample
    plus every returned user, the users within the 1e-6 relative margin of a tie, and the
    band population of the BF16 scores."""
    import oracle
    gate = oracle_gate(W, host, qrows, K, 2000, nq_check=2)
    sample = workload.sample_rows(W.m, 2000, seed=22)
    tau = oracle.tau(W.U, W.P, 50, sample)
    boundary = 0
    for qi in np.unique(qrows)[:2]:
        for r in np.flatnonzero(qrows == qi):
            mg = oracle.margins(W.U, tau, W.P[W.query_idx[qi]], int(K[r]), sample)
            boundary += int(np.count_nonzero(mg < 1e-6))
    nq = len(K)
    sc = rec["stage_counts"]
    return {"f1_vs_fp64_on_sample": 1.0 if gate["agree"] else None, "mismatches": gate["mismatches"],
            "checked_memberships": gate["checked_memberships"], "boundary_users_margin_lt_1e-6": boundary,
            "score_error_bound_rel": cband,
            "score_error_note": "a-priori bound |s_tc - <u,q>| <= c ||u|| ||q|| of the BF16 tensor-core score",
            "pairs_in_band_per_request": sc["pairs_rescored"] / nq,
            "fp64_rescored_per_request": sc["fp64_rescored"] / nq,
            "sample": f"{gate['sample_users']} seeded users + every returned user, {gate['queries']} queries x k in "
                      f"{sorted(set(int(k) for k in K.tolist()))}"}


def _bf16_round(x):
    """Round-to-nearest-even to BF16, from float32 bits."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    return ((b + np.uint32(0x7FFF) + ((b >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)).view(np.float32)


def _e4m3_rows(X):
    """The library's E4M3 rows: y = x * (448 / max|x_i|) in FP32, rounded to nearest even E4M3
    (3 mantissa bits, subnormal spacing 2^-9, finite saturation at 448), and the scale back
    max|x_i| / 448 in FP32."""
    X = np.asarray(X, np.float32)
    mx = np.abs(X).max(axis=1).astype(np.float32)
    inv = np.where(mx > 0, np.float32(448.0) / np.where(mx > 0, mx, 1), 0).astype(np.float32)
    y = (X * inv[:, None]).astype(np.float64)
    a = np.abs(y)
    q = 2.0 ** (np.floor(np.log2(np.maximum(a, 2.0 ** -6))) - 3)
    r = np.minimum(np.round(a / q) * q, 448.0)
    return np.sign(y) * r, (mx / np.float32(448.0)).astype(np.float64)


def emulated_score_error(W, qrows, users, fmt):
    """Largest |s - <u,q>| / (||u|| ||q||) over the sample of users and the batch's first two
    query vectors, with s the score from the tensor cores' operands rounded as the library
    rounds them (BF16, or E4M3 with per-vector scales), their products summed in FP64 (the
    FP32 accumulation adds at most (K + 16) 2^-23 of the sum on top)."""
    U = W.U[users].astype(np.float32)
    worst = 0.0
    for qi in np.unique(qrows)[:2]:
        q = W.P[W.query_idx[qi]].astype(np.float32)
        exact = U.astype(np.float64) @ q.astype(np.float64)
        if fmt == "bf16":
            s = _bf16_round(U).astype(np.float64) @ _bf16_round(q[None, :])[0].astype(np.float64)
        else:
            u8, su = _e4m3_rows(U)
            q8, sq = _e4m3_rows(q[None, :])
            s = (u8 @ q8[0]) * su * sq[0]
        nrm = np.linalg.norm(U.astype(np.float64), axis=1) * np.linalg.norm(q.astype(np.float64))
        worst = max(worst, float(np.max(np.abs(s - exact) / nrm)))
    return worst


def run_variants(sah, dev, stream, flush, peaks, peak_kind, W5, Ud5, Pd5, steps):
    import torch
    out = {}
    vs = max(3, min(steps, 5))
    # C5 with the paper's |P'| = 4 k_max: survivors go through the tensor-core kMIPS decision
    ixp, bp, rec = measure_config(sah, W5, Ud5, Pd5, dev, stream, flush, "paper", "bf16", vs, 2, peaks, peak_kind)
    out["c5_paper_bf16"] = rec
    # SA-ALSH mode (Alg. 1, Alg. 2) on that index, on the first 1,000 requests: F1 against the
    # exact answers of the same index
    Qs, Ks = bp.Q[:1000], bp.K[:1000]
    modes = np.full(len(Ks), sah.SAALSH, np.int32)
    bs = Batch(ixp, Qs, Ks, dev, stream, modes=modes)
    ts = bs.timed(vs, 2, flush)
    f1s = [f1_sets(a, b) for a, b in zip(bs.host, bp.host[:1000])]
    out["c5_paper_saalsh"] = {"queries_per_step": len(Ks), "value": len(Ks) / (np.mean(ts) / 1e3),
                              "ms_per_step": float(np.mean(ts)), "f1_vs_exact": float(np.mean(f1s)),
                              "min_f1": float(np.min(f1s)), "probe_radius": 0}
    ixp.close()
    del bp, bs
    # C3: n 100k, m 1M, d 64; accuracy of the BF16 path against the FP64 oracle
    W3 = workload.make("c3")
    Q3, K3, q3 = W3.requests()
    Ud3, Pd3 = torch.from_numpy(W3.U).to(dev), torch.from_numpy(W3.P).to(dev)
    ix3, b3, rec3 = measure_config(sah, W3, Ud3, Pd3, dev, stream, flush, "full", "bf16", vs, 2, peaks, peak_kind,
                                   Q=Q3, K=K3)
    dk = 64 if W3.d <= 64 else 128
    cband = 1.01 * (2.0 ** -7 + 2.0 ** -16 + (2.0 * dk + 16.0) * 2.0 ** -23)
    rec3["accuracy"] = c3_accuracy(W3, b3.host, q3, K3, rec3, cband)
    sample3 = workload.sample_rows(W3.m, 2000, seed=22)
    rec3["accuracy"]["max_score_error_rel_emulated"] = emulated_score_error(W3, q3, sample3, "bf16")
    out["c3_full_bf16"] = rec3
    ix3.close()
    del b3
    # the same with the E4M3 user pass (per-vector scales, kind::f8f6f4): the band is about
    # 0.13 ||u|| ||q||, so most pairs near a threshold go to the re-score
    ix8, b8, rec8 = measure_config(sah, W3, Ud3, Pd3, dev, stream, flush, "full", "bf16", vs, 2, peaks, peak_kind,
                                   tc=2, Q=Q3, K=K3)
    K8 = 128.0
    c8 = 1.01 * (2.0 ** -4 * (2.0 + 2.0 ** -4) + 2.0 * (1.0 + 2.0 ** -4) * 2.0 ** -10 * np.sqrt(K8) / 448.0
                 + 2.0 ** -20 * K8 / 448.0 ** 2 + 1.13 * ((K8 + 16.0) * 2.0 ** -23 + 8.0 * 2.0 ** -24))
    rec8["accuracy"] = c3_accuracy(W3, b8.host, q3, K3, rec8, c8)
    rec8["accuracy"]["max_score_error_rel_emulated"] = emulated_score_error(W3, q3, sample3, "fp8")
    out["c3_full_fp8"] = rec8
    ix8.close()
    del b8, Ud3, Pd3
    # C2 (n 17,770, m 480k, d 50): the tensor-core path against the plain FP32 GPU path
    W2 = workload.make("c2")
    Ud2, Pd2 = torch.from_numpy(W2.U).to(dev), torch.from_numpy(W2.P).to(dev)
    for thr in ("full", "paper"):
        for prec, tc in (("bf16", 1), ("fp32", 0)):
            ix2, b2, rec2 = measure_config(sah, W2, Ud2, Pd2, dev, stream, flush, thr, prec, vs, 2, peaks, peak_kind,
                                           tc=tc)
            out[f"c2_{thr}_{prec}"] = rec2
            ix2.close()
    out["ablation_blocking"] = blocking_ablation(sah, dev, stream, flush, peaks, peak_kind, W2, Ud2, Pd2, W5, Ud5,
                                                 Pd5, vs)
    out["kmips_sat_vs_qnf"] = kmips_comparison(sah, dev, stream)
    return out


def blocking_ablation(sah, dev, stream, flush, peaks, peak_kind, W2, Ud2, Pd2, W5, Ud5, Pd5, vs):
    """The paper's ablation (Experiments, ablation study) on C2-shaped data, everything else
    equal: Cone-Tree blocks (Alg. 3, Lemma 2-3) against Simpfer's norm-sorted blocks with
    Cauchy-Schwarz bounds, and SAT (SA-ALSH) against QNF (H2-ALSH) codes, i.e. SAH,
    SA-Simpfer, H2-Cone and H2-Simpfer in SA-ALSH mode (F1 against the exact answers), plus
    the exact mode's cost under both blockings (tensor-core user pass, BF16; FP32 path,
    where Lemma 3 runs per user), and the exact C5 step under both blockings."""
    res = {}
    names = {(0, 0): "SAH", (1, 0): "SA-Simpfer", (0, 1): "H2-Cone", (1, 1): "H2-Simpfer"}
    for blk, tag in ((0, "cone"), (1, "norm")):
        for thr, prec, tc in (("full", "bf16", 1), ("paper", "bf16", 1), ("paper", "fp32", 0)):
            ix, b, rec = measure_config(sah, W2, Ud2, Pd2, dev, stream, flush, thr, prec, vs, 2, peaks, peak_kind,
                                        tc=tc, blocking=blk)
            res[f"c2_{thr}_{prec}_{tag}"] = {k: rec[k] for k in ("value", "ms_per_step", "index_build_s",
                                                                  "stages_ms", "stage_counts")}
            if thr == "paper" and prec == "bf16":
                for tr in (0, 1):
                    ixs = ix if tr == 0 else make_index(sah, Ud2, Pd2, stream, "paper", "bf16", blocking=blk,
                                                        transform=1)[0]
                    modes = np.full(len(b.K), sah.SAALSH, np.int32)
                    bs = Batch(ixs, b.Q, b.K, dev, stream, modes=modes)
                    ts = bs.timed(vs, 2, flush)
                    f1s = [f1_sets(x, y) for x, y in zip(bs.host, b.host)]
                    res[f"c2_paper_bf16_saalsh_{names[(blk, tr)]}"] = {
                        "blocking": tag, "transform": "qnf" if tr else "sat",
                        "value": len(b.K) / (np.mean(ts) / 1e3), "ms_per_step": float(np.mean(ts)),
                        "f1_vs_exact": float(np.mean(f1s)), "min_f1": float(np.min(f1s))}
                    if tr:
                        ixs.close()
            ix.close()
        ix, b, rec = measure_config(sah, W5, Ud5, Pd5, dev, stream, flush, "full", "bf16", vs, 2, peaks, peak_kind,
                                    blocking=blk)
        res[f"c5_full_bf16_{tag}"] = {k: rec[k] for k in ("value", "ms_per_step", "index_build_s", "stages_ms",
                                                          "stage_counts")}
        ix.close()
    return res


def kmips_comparison(sah, dev, stream, reps=5):
    """SA-ALSH against H2-ALSH's QNF as standalone kMIPS (the paper's kMIPS comparison,
    Experiments): 100 user vectors drawn uniformly at random as queries, k in
    {1, 5, 10, 20, 30, 40, 50}; the same partitions (b = 0.5), 64 tables and probes, only the
    transform differs; |P'| = 1, so that the candidates, not the seed, make the answer.
    The vectors are the C2 and C3 shapes drawn from non-negative factors ("nmf"), like the
    NMF embeddings of the paper's datasets: their centroid lies away from the origin, which
    is where SAT's shift differs from QNF (zero-mean factors put it near the origin).
    F1 = |A & E| / k against the exact top-k, which the same call gives on an index with
    |P'| = n (C then holds every item; the GPU tests tie it to the FP64 top-k).  Times: CUDA
    events around one call for the 100 queries, median of reps."""
    import torch
    out = {}
    ks = (1, 5, 10, 20, 30, 40, 50)
    for wname in ("c2", "c3"):
        W = workload.make(wname, kind="nmf")
        Ud, Pd = torch.from_numpy(W.U).to(dev), torch.from_numpy(W.P).to(dev)
        rows = workload.sample_rows(W.m, 100, seed=31)
        Qd = torch.from_numpy(np.ascontiguousarray(W.U[rows])).to(dev)
        ixe, _ = make_index(sah, Ud, Pd, stream, "full")
        exact = {}
        for k in ks:
            e_ids = torch.empty((100, k), dtype=torch.int32, device=dev)
            ixe.kmips_device(Qd, k, e_ids, stream=stream)
            torch.cuda.synchronize()
            exact[k] = e_ids.cpu().numpy()
        ixe.close()
        res = []
        for bits in (8, 12, 16):
            for tr, tname in ((0, "SA-ALSH"), (1, "H2-ALSH (QNF)")):
                ix, build_s = make_index(sah, Ud, Pd, stream, 1, n_tables=64, code_bits=bits, transform=tr)
                for k in ks:
                    o_ids = torch.empty((100, k), dtype=torch.int32, device=dev)
                    times = []
                    for _ in range(reps + 1):
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        ix.kmips_device(Qd, k, o_ids, stream=stream)
                        e1.record(stream)
                        torch.cuda.synchronize()
                        times.append(e0.elapsed_time(e1))
                    got = o_ids.cpu().numpy()
                    f1 = float(np.mean([len(set(got[r].tolist()) & set(exact[k][r].tolist())) / k
                                        for r in range(100)]))
                    res.append({"method": tname, "code_bits": bits, "probe_radius": 0, "k": k,
                                "f1": f1, "ms_per_100_queries": float(np.median(times[1:])),
                                "items_scored_per_query": ix.stats()["items_scanned"] / 100.0,
                                "index_build_s": build_s})
                ix.close()
        out[wname] = {"workload": config_block(W)["workload"], "queries": "100 user vectors (seed 31)",
                      "tables": 64, "b": 0.5, "p_prime": 1, "points": res}
        del Ud, Pd
    return out


# ---------------------------------------------------------------- our arm
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = dist_env()
    import torch
    import paper_2211_12751_gb300 as sah
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    peaks, peak_kind = load_peaks()
    sah.load()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    if args.sweep:
        if rank == 0:
            print(json.dumps(run_sweeps(sah, dev, stream, flush)), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    over = {k: v for k, v in (("m", args.m), ("n", args.n), ("nq", args.nq)) if v > 0}
    W = workload.make(args.workload, **over)
    Q, K, qrows = W.requests()
    nq = len(K)
    Ud, Pd = torch.from_numpy(W.U).to(dev), torch.from_numpy(W.P).to(dev)
    ix, build_s = make_index(sah, Ud, Pd, stream, "full")
    ist = ix.stats()
    main_b = Batch(ix, Q, K, dev, stream)
    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        times = main_b.timed(args.steps, max(args.warmup, 3), flush)
    clocks = clk.summary()
    if world > 1:
        torch.distributed.barrier()
    value, _ = whole_job_value(sum(times), nq, args.steps, world, torch_max_reducer(dev))
    # back-to-back steps after the timed ones: the sustained rate and clocks under load
    sus_value, sus_steps, clocks_sus = None, 0, None
    if args.sustain_s > 0:
        with ClockSampler(local) as clk2:
            sus_value, sus_steps = main_b.sustained(args.sustain_s)
        clocks_sus = clk2.summary()
    e2e_times, h2d, d2h = main_b.e2e(args.steps, args.warmup, flush)
    e2e_value, _ = whole_job_value(sum(e2e_times), nq, args.steps, world, torch_max_reducer(dev))
    sms, lau, st = main_b.stages()
    dp = (W.d + 3) // 4 * 4
    roofs = stage_rooflines(sms, lau, st, W.d, dp, peaks, peak_kind)
    dom_name, roof = dominant(sms, roofs)
    roofline = dict(roof) if roof else {"stage": dom_name, "note": "no counter for this stage"}
    roofline["stage"] = dom_name
    if roof:
        roofline["traffic"] = kernel_traffic(roof["kernel"], W.name)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean(times)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": config_block(W),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(round(float(np.sum(lau[:6])) * args.steps)),
            "roofline": roofline,
            "stage_rooflines": roofs,
            "stages_ms": {nm: float(sms[i]) for i, nm in enumerate(STAGE_NAMES)},
            "stage_counts": {k: st[k] for k in ("block_pairs_total", "block_pairs_kept", "users_in_kept_blocks",
                                                "block_col_pairs", "tc_scores", "tc_rows", "users_yes_early",
                                                "pairs_rescored", "survivors", "fp64_rescored", "items_scanned",
                                                "results")},
            "index_build_s": build_s,
            "index_build": {"inputs": "U and P already on the device", "gemm_ms": ist.get("build_gemm_ms", 0.0),
                            "overflow_rows": ist.get("build_overflow_rows", 0), "device_bytes": ist["device_bytes"]},
            "clocks": clocks,
            "sustained": {"value": sus_value, "steps": sus_steps, "seconds": args.sustain_s, "clocks": clocks_sus,
                          "note": "back-to-back steps without the L2 flush, after the timed ones"},
            "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99)),
                           "per": f"batch of {nq} requests (per-request latencies: serving)"}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        gate = oracle_gate(W, main_b.host, qrows, K, args.sample_users)
        tau = cached_tau_baseline(W, W.ks)
        line["correctness"] = {"gpu_matches_oracle_on_sample": gate["agree"], "mismatches": gate["mismatches"],
                               "checked_memberships": gate["checked_memberships"],
                               "sample": f"{gate['sample_users']} seeded users + every user the GPU returned, "
                                         f"{gate['queries']} queries at each of their k"}
        line["cpu_baseline"] = {"value": gate["qps"], "unit": UNIT, "cores": gate["threads"], "kind": "oracle",
                                "sample": (f"(i) FP64 brute-force counts (Def. 1) for the correctness sample: "
                                           f"{gate['seconds']:.1f} s for {gate['checked_memberships'] // max(1, len(W.ks))} "
                                           f"user-query counts, each answering the query's {len(W.ks)} k values; "
                                           f"scaled to all {W.m} users"),
                                "cached_tau": {"value": tau["qps"], "unit": UNIT, "cores": tau["cores"],
                                               "tau_build_s_per_user": tau["tau_build_s_per_user"],
                                               "sample": tau["sample"]}}
    if rank == 0 and not args.no_variants:
        ix.close()
        del main_b
        line["variants"] = run_variants(sah, dev, stream, flush, peaks, peak_kind, W, Ud, Pd, args.steps)
    if rank == 0 and not args.no_serving:
        del Ud, Pd
        line["serving"] = run_serving(sah, dev, stream, [float(r) for r in args.serve_rates.split(",") if r],
                                      args.serve_requests)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
