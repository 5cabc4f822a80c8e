"""Benchmark: GLR GAP iterations/s on the 16 x 512 x 512 video-SCI workload.

One step = one outer GAP iteration of the whole hot path on one snapshot:
key selection, global matching (fused running top-K), grouping + WNNM,
aggregation and the GAP projection, on 16 frames of 512 x 512 (P = 8,
N = 4096 keys per frame, K = 64, exhaustive search over 505 x 505 positions).

The chosen form (BF16 tcgen05 matching + exact FP32 re-rank) is the headline;
the plain form (FP32 matching on the CUDA cores) is timed beside it.  Inputs
are resident in HBM before the timed region; L2 (126 MB) is flushed by
writing a 256 MB buffer between timed steps.  `e2e` repeats the measurement
through the public API with the snapshot and masks copied from pinned host
memory and the reconstruction read back every step.

--impl reference times the FP64 CPU oracle (the only other implementation)
on the host cores, on a bounded sample of the same workload, extrapolated to
one full iteration.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GLR GAP iterations/s (chosen BF16 form; match pair-dists/s and plain FP32 form alongside)"
UNIT = "iter/s"


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline); runs in a child process
# with single-threaded BLAS so `cores` is exact.
# ---------------------------------------------------------------------------
def oracle_sample(n_keys: int = 24) -> dict:
    from paper_2301_03047_gb300 import synth

    return _oracle_sample_sci(synth.SCI_LARGE, n_keys)


def oracle_sample_huge(n_keys: int = 6) -> dict:
    """The oracle on one 2048^2 frame of the 24-frame workload, extrapolated the same way."""
    from paper_2301_03047_gb300 import synth

    return _oracle_sample_sci(synth.SCI_HUGE, n_keys)


def _oracle_sample_sci(cfg, n_keys: int) -> dict:
    from oracle import glr_oracle as O
    from paper_2301_03047_gb300 import synth

    prob = synth.sci_problem(synth.scaled(cfg, T=1))  # one frame of the same scene model and size
    sw = cfg.sigma_schedule()[0]
    x = O.gap_init(prob.y, prob.masks)[:, None]  # [1][1][H][W]
    f0 = x[0]
    t0 = time.perf_counter()
    keys, _ = O.select_keys(f0, cfg.P, cfg.N, cfg.edge_th)
    t_select = time.perf_counter() - t0
    t0 = time.perf_counter()
    Q = O.patch_matrix(f0, cfg.P)
    t_q = time.perf_counter() - t0
    sample = keys[:n_keys]
    t0 = time.perf_counter()
    idx, _ = O.match_topk(f0, cfg.P, sample, cfg.K, Q)
    t_match = (time.perf_counter() - t0) / n_keys
    t0 = time.perf_counter()
    g = O.gather_groups(f0, cfg.P, idx, Q)
    xh, _ = O.lowrank_groups(g, sw, cfg.c_wnnm)
    t_low = (time.perf_counter() - t0) / n_keys
    t0 = time.perf_counter()
    O.aggregate(xh, idx, f0, cfg.P)
    t_agg = (time.perf_counter() - t0) / n_keys
    t0 = time.perf_counter()
    O.gap_project(prob.y, prob.masks, x[:, 0])
    t_gap = time.perf_counter() - t0
    per_frame = t_select + t_q + cfg.N * (t_match + t_low + t_agg)
    t_iter = cfg.T * per_frame + t_gap * cfg.T
    pairs = cfg.T * cfg.N * (cfg.H - cfg.P + 1) * (cfg.W - cfg.P + 1)
    return {
        "t_iter_s": t_iter,
        "iters_per_s": 1.0 / t_iter,
        "pair_dists_per_s": pairs / (cfg.T * cfg.N * t_match),
        "sample": f"1 of {cfg.T} frames: full key selection + {n_keys} of {cfg.N} keys matched over all "
        f"{(cfg.H - cfg.P + 1) ** 2} positions, grouped, WNNM, aggregated; GAP on 1 frame; "
        f"extrapolated linearly to {cfg.T} frames x {cfg.N} keys",
        "parts_s": {"select": t_select, "patch_matrix": t_q, "match_per_key": t_match, "lowrank_per_group": t_low,
                    "aggregate_per_group": t_agg, "gap_per_frame": t_gap},
    }


def psnr_framewise(a, b, peak: float = 1.0) -> float:
    """Mean over frames of the per-frame PSNR (result bookkeeping)."""
    import numpy as np

    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    vals = []
    for i in range(a.shape[0]):
        mse = float(np.mean((a[i] - b[i]) ** 2))
        vals.append(float("inf") if mse == 0 else 10.0 * math.log10(peak * peak / mse))
    return float(np.mean(vals))


def oracle_check(path: str) -> dict:
    """Per-result error of the GPU path against the FP64 oracle on one frame of the timed workload
    (part of the CPU-baseline leg; runs in a child process).  The GPU's outputs of one GLR step on
    the frame are compared step by step with the oracle fed the same inputs: key selection, the
    matches of a sample of keys, the WNNM estimates of those keys' groups, and the aggregation."""
    import numpy as np

    from oracle import glr_oracle as O

    z = np.load(path)
    x = z["x"].astype(np.float64)  # [C][H][W]
    P, K, N = int(z["P"]), int(z["K"]), int(z["N"])
    sw, cw, th = float(z["sw"]), float(z["cw"]), float(z["th"])
    keys_g, idx_g, dist_g, grp_g, v_g = z["keys"], z["idx"], z["dist"], z["groups"], z["v"]
    out = {}
    keys_o, _ = O.select_keys(x, P, N, th)
    out["key_selection_equal_frac"] = round(float(np.mean(keys_o == keys_g)), 6)
    Q = O.patch_matrix(x, P)
    sample = np.linspace(0, N - 1, 32).astype(int)
    exact = sep = 0
    dist_err = 0.0
    for i in sample:
        d_all = O.all_distances(x, P, keys_g[i], Q)
        order = np.lexsort((np.arange(len(d_all)), d_all))
        ds = d_all[order]
        dist_err = max(dist_err, float(np.max(np.abs(dist_g[i] - d_all[idx_g[i]]) / np.maximum(d_all[idx_g[i]], 1e-6))))
        for j in range(K):
            lo = ds[j] - ds[j - 1] if j > 0 else np.inf
            hi = ds[j + 1] - ds[j] if j + 1 < len(ds) else np.inf
            if lo > 1e-4 and hi > 1e-4:
                sep += 1
                exact += int(idx_g[i, j] == order[j])
    out["match_ids_exact_where_separated"] = f"{exact}/{sep}"
    out["match_dist_max_rel_err"] = float(f"{dist_err:.3g}")
    Y = O.gather_groups(x, P, idx_g[sample], Q)
    Xo, _ = O.lowrank_groups(Y, sw, cw, eps=1e-8)
    err = grp_g[sample].astype(np.float64) - Xo
    out["wnnm_max_abs_err_rel"] = float(f"{np.abs(err).max() / max(np.abs(Y).max(), 1e-12):.3g}")
    out["wnnm_rms_err_rel"] = float(f"{np.sqrt(np.mean(err ** 2)) / max(np.sqrt(np.mean(Y ** 2)), 1e-12):.3g}")
    vo = O.aggregate(grp_g.astype(np.float64), idx_g, x, P)
    out["aggregate_max_abs_err"] = float(f"{np.abs(v_g - vo).max():.3g}")
    out["sample"] = f"frame 0 after the timed iterations: all {N} keys selected, {len(sample)} keys matched and shrunk, all groups aggregated"
    return out


def run_oracle_check(path: str) -> dict:
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    code = f"import json,sys; sys.path.insert(0,{ROOT!r}); import bench; print(json.dumps(bench.oracle_check({path!r})))"
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle check failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def _oracle_cmd(n_keys: int, fn: str):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    code = f"import json,sys; sys.path.insert(0,{ROOT!r}); import bench; print(json.dumps(bench.{fn}({n_keys})))"
    return [sys.executable, "-c", code], env


def run_oracle_child(n_keys: int, fn: str = "oracle_sample") -> dict:
    cmd, env = _oracle_cmd(n_keys, fn)
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle child failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def _mem_available_gb() -> float:
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) / 2**20
    except OSError:
        pass
    return 0.0


def run_oracle_all_cores(n_keys: int, fn: str = "oracle_sample", procs: int | None = None,
                         gb_per_proc: float = 0.0) -> dict:
    """The same sample on every host core at once: `procs` single-threaded children run side by
    side (their per-key and per-frame times include the contention for memory bandwidth), and the
    full iteration's work is divided over them (frames and keys are independent units).
    gb_per_proc > 0: at most as many children as fit in half of the available host memory."""
    procs = procs or os.cpu_count() or 1
    if gb_per_proc > 0:
        procs = max(1, min(procs, int(0.5 * _mem_available_gb() / gb_per_proc)))
    cmd, env = _oracle_cmd(n_keys, fn)
    children = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env, cwd=ROOT)
                for _ in range(procs)]
    outs = []
    for c in children:
        out, err = c.communicate()
        if c.returncode != 0:
            raise RuntimeError("oracle child failed: " + err[-2000:])
        outs.append(json.loads(out.strip().splitlines()[-1]))
    t_iter_1 = statistics.mean(o["t_iter_s"] for o in outs)  # one core's share of the iteration, under load
    res = dict(outs[0])
    res["t_iter_s"] = t_iter_1 / procs
    res["iters_per_s"] = procs / t_iter_1
    res["pair_dists_per_s"] = sum(o["pair_dists_per_s"] for o in outs)
    res["procs"] = procs
    res["sample"] = f"{procs} single-threaded processes at once, each: " + outs[0]["sample"] + \
        f"; the iteration divided over the {procs} cores"
    return res


def cpu_baseline_entry(n_keys: int, fn: str, unit: str = "iter/s", gb_per_proc: float = 0.0) -> dict:
    """cpu_baseline: the oracle on all host cores (value) and on one core (single_core), nproc recorded."""
    one = run_oracle_child(n_keys, fn)
    allc = run_oracle_all_cores(max(4, n_keys // 4), fn, gb_per_proc=gb_per_proc)
    return {"value": round(allc["iters_per_s"], 8), "unit": unit, "cores": allc["procs"], "nproc": os.cpu_count(),
            "kind": "oracle", "sample": allc["sample"], "t_iter_s": round(allc["t_iter_s"], 1),
            "pair_dists_per_s": round(allc["pair_dists_per_s"], 1),
            "single_core": {"value": round(one["iters_per_s"], 8), "unit": unit, "cores": 1, "sample": one["sample"],
                            "t_iter_s": round(one["t_iter_s"], 1),
                            "pair_dists_per_s": round(one["pair_dists_per_s"], 1)}}


# ---------------------------------------------------------------------------
# distributed helpers (one process per GPU; replicas, no data-path collective)
# ---------------------------------------------------------------------------
def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(backend: str):
    import torch.distributed as dist

    ws, rank, _ = dist_info()
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist if ws > 1 else None


def reduce_max(value: float, dist, device) -> float:
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks sampler
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"glr_bench_clocks_{os.getpid()}_{gpu_index}.csv")
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [t.strip() for t in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1].split()[0]))
                mx.append(float(p[2].split()[0]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------
def peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0,
            "source": "fallback"}


def num_sms() -> int:
    """Streaming multiprocessors of the current device (152 on a GB300)."""
    import torch

    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def fp32_alu_peak_tflops(sm_mhz: float) -> float:
    """FP32 FMA peak: SMs (read from the device) x 128 FP32 lanes x 2 flop x clock."""
    return num_sms() * 128 * 2 * sm_mhz * 1e6 / 1e12


def kernel_hash(fname) -> str:
    """Hash of the kernel's source file(s) (a name or a tuple of names) and the shared headers."""
    h = hashlib.sha1()
    names = tuple(fname) if isinstance(fname, (tuple, list)) else (fname,)
    for f in names + ("glr_common.cuh", "topk_stream.cuh", "glr_kernels.cuh"):
        p = os.path.join(ROOT, "paper_2301_03047_gb300", "csrc", f)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:12]


KERNEL_FILE = {"k_match_tc": ("k_match_tc.cu", "k_match.cu"), "k_match_fp32": "k_match.cu", "k_jacobi_wnnm": "k_lowrank.cu",
               "k_jacobi_smem": "k_lowrank_wide.cu", "k_jacobi_wnnm_c": "k_lowrank.cu", "k_fft_rows": "k_fft.cu",
               "k_match_tc_w": "k_match_tc.cu", "k_gram_wnnm": "k_lowrank_wide.cu",
               "k_jacobi_wnnm_fused": "k_lowrank.cu",
               "k_fft_cols": "k_fft.cu",
               "k_gather": "k_lowrank.cu", "k_scatter": "k_aggregate.cu", "k_gap_step": "k_gap.cu",
               "k_rerank": "k_match.cu"}


def traffic_for(kernel: str, units_per_launch: float):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel)
    if not d or d.get("source_hash") != kernel_hash(KERNEL_FILE.get(kernel, "")):
        return None
    return d["dram_bytes_per_unit"] * units_per_launch


SCHED_KEYS = ("k_over", "splits", "cap", "epi_batch", "bound_pass")


def sched_kw(t) -> dict:
    """A matching schedule tuple (autotuner or --match-schedule) as reconstructor keyword arguments."""
    return dict(zip(SCHED_KEYS, tuple(int(v) for v in t) + (0,) * (len(SCHED_KEYS) - len(t))))


def merge_scans(prof: dict) -> dict:
    """The tensor-core matcher's minima scan and bound kernel counted with its candidate scan:
    together they are one contraction of every key/position pair."""
    prof = dict(prof)
    if "k_match_tc_chunk" in prof:
        # chunk minima (the contraction), the bound and candidate list, the exact evaluation
        ms, n = prof.pop("k_match_tc_chunk")
        extra = [prof.pop(k) for k in ("k_tau_chunk", "k_chunk_topk", "k_patch_norms") if k in prof]
        prof["k_match_tc"] = (ms + sum(e[0] for e in extra), n)
        return prof
    extra = [prof.pop(k) for k in ("k_match_tc_min", "k_tau_bound") if k in prof]
    if extra and "k_match_tc" in prof:
        ms, n = prof["k_match_tc"]
        prof["k_match_tc"] = (ms + sum(e[0] for e in extra), n)
    return prof


def roofline(prof: dict, cfg, sweeps_per_group: float, clocks: dict, pk: dict, n_img: int | None = None,
             d: int | None = None, census: dict | None = None) -> dict:
    """Roofline entry of the kernel with the largest share of the timed region.  The matcher's two
    scans (minima, candidates) count as one unit: the pair FLOPs once, over their summed time."""
    scans = "k_match_tc_min" in prof
    chunks = "k_match_tc_chunk" in prof
    prof = merge_scans(prof)
    name, (ms, n) = max(prof.items(), key=lambda kv: kv[1][0])
    avg_s = ms / n / 1e3
    T = n_img if n_img is not None else cfg.T
    H, W, P, N, K = cfg.H, cfg.W, cfg.P, cfg.N, cfg.K
    d = d if d is not None else P * P
    npos = (H - P + 1) * (W - P + 1)
    sm = clocks.get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    if name in ("k_match_tc", "k_match_fp32"):
        units = T * N * npos  # key/position pairs per launch
        work = 2.0 * d * units
        if name == "k_match_tc":
            out = {"bound": "tensor", "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
                   "peak_note": f"of {pk['source']} cuBLAS bf16 sustained"
                                + ("; time = minima scan + bound + candidate scan" if scans else "")
                                + ("; time = chunk-minima scan + bound + exact evaluation of the candidate chunks"
                                   if chunks else "")}
        else:
            out = {"bound": "alu", "peak": round(fp32_alu_peak_tflops(sm), 1), "unit": "TFLOP/s",
                   "peak_note": f"derived FP32 FMA peak {num_sms()}x128x2 at {sm:.0f} MHz"}
        achieved = work / avg_s / 1e12
        unit_name = "pairs"
    elif name in ("k_jacobi_wnnm", "k_jacobi_smem", "k_jacobi_wnnm_c", "k_jacobi_wnnm_fused"):
        units = T * N
        # complex columns: a complex multiply-add is 4 real ones on 2 real values, twice the real count per value
        work = units * sweeps_per_group * 6.0 * d * K * K * (2.0 if name == "k_jacobi_wnnm_c" else 1.0)
        note = "work = 6 d K^2 per sweep x measured sweeps"
        if census:
            # the timed iterations' own counts: sweeps, power steps of the rank-1 certificate
            # (4 d K each: Y v and Y^T y) and the certified groups' output (4 d K)
            work = units * (census["sweeps_per_group"] * 6.0 * d * K * K
                            + (census["power_steps_per_group"] + census["rank1_per_group"]) * 4.0 * d * K
                            + census["gram_per_group"] * 2.0 * d * K * K)
            note = ("work = 6 d K^2 per sweep + 4 d K per power step and per rank-1 output + 2 d K^2 per Gram "
                    "bound, counts of the timed iterations")
        achieved = work / avg_s / 1e12
        out = {"bound": "alu", "peak": round(fp32_alu_peak_tflops(sm), 1), "unit": "TFLOP/s",
               "peak_note": f"derived FP32 FMA peak {num_sms()}x128x2 at {sm:.0f} MHz; {note}"}
        unit_name = "groups"
    else:
        units = T * N
        if name == "k_gather":
            work = T * N * K * d * 4 + T * H * W * 4
        elif name == "k_scatter":
            work = T * N * K * d * 4 + 2 * T * H * W * 4
        elif name == "k_gap_step":
            work = H * W * 4 * (1 + 3 * T)
        else:
            work = T * N * K * 8
        achieved = work / avg_s / 1e9
        out = {"bound": "hbm", "peak": pk["hbm_gbs"], "unit": "GB/s", "peak_note": f"of {pk['source']} copy bandwidth"}
        unit_name = "groups"
    out.update({"kernel": name, "achieved": round(achieved, 2), "frac": round(achieved / out["peak"], 4),
                "avg_launch_ms": round(avg_s * 1e3, 3), "launches": n, "units_per_launch": units, "unit_kind": unit_name,
                "traffic": traffic_for(name, units)})
    return out


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def workload(name: str):
    """The timed workload: 16 x 512^2 (the headline); smaller cases for profiling captures."""
    from paper_2301_03047_gb300 import synth

    if name == "sci16":
        return synth.SCI_LARGE
    if name == "sci24x2048":  # the learned-proposal workload: 24 frames of 2048^2, 16384 keys per frame
        return synth.SCI_HUGE
    if name == "sci2x2048":  # profiling case of the large frames
        return synth.scaled(synth.SCI_HUGE, T=2, name="sci_2x2048x2048_P8_N16384_K64")
    if name == "sci4":  # profiling case: same frame size, 4 frames (operands still larger than L2)
        return synth.scaled(synth.SCI_LARGE, T=4, name="sci_4x512x512_P8_N4096_K64")
    if name == "sci8":
        return synth.SCI_SMALL
    if name == "msfa32":
        return synth.MSFA_LARGE
    if name == "msfa2":  # profiling case: two images (768, 512), a few GB on the device
        return synth.MsfaConfig("msfa_2img_768-512_16band_P6_K32", 4, sides=(768, 512), bands=16, P=6, K=32, iters=10)
    if name == "msfa4":  # profiling case: four images of the batch
        return synth.MsfaConfig("msfa_4img_512-1024_16band_P6_K32", 4, sides=(1024, 768, 512, 384), bands=16, P=6,
                                K=32, iters=10)
    if name == "mri1024":
        return synth.MRI_LARGE
    if name == "mri256":  # profiling case of the MRI path
        return synth.mri_scaled(synth.MRI_LARGE, H=256, W=256, N=2048, name="mri_256x256_P6_N2048_K48")
    raise ValueError(name)


def lowrank_census(cfg, y, masks, sched, dev, form, sched_kw_form, n_warm, n_steps) -> dict:
    """The low-rank step's work over the timed iterations (untimed replay of the same iterations
    with the status block read after each): sweeps, rank-1 certificate power steps and certified
    groups, per group."""
    import torch

    from paper_2301_03047_gb300 import glr

    rec = glr.SciReconstructor(cfg.T, cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, mode=form, edge_th=cfg.edge_th,
                               device=dev, **sched_kw_form)
    rec.start(y, masks)
    tot = [0, 0, 0, 0, 0, 0]  # sweeps, groups, rank1, power steps, rank1 by the Gram bound, Gram bounds
    for k in range(n_warm + n_steps):
        rec.step(sched[k % len(sched)], cfg.c_wnnm)
        if k >= n_warm:
            torch.cuda.synchronize()
            _, cnt = glr.poll_status(rec.den.ws_lowrank_status)
            tot = [t + c for t, c in zip(tot, (cnt[2], cnt[3], cnt[7], cnt[8], cnt[9], cnt[10]))]
    del rec
    g = max(tot[1], 1)
    return {"sweeps_per_group": tot[0] / g, "rank1_per_group": tot[2] / g, "power_steps_per_group": tot[3] / g,
            "rank1_gram_per_group": tot[4] / g, "gram_per_group": tot[5] / g}


def run_learned(args, cfg, prob, y, masks, sched, dev, fpc, flush, x_final, chosen, plain) -> dict:
    """The learned proposal: an encoder trained on pairs from the exhaustive matcher's own output on
    two frames of the start image (set-up, untimed), then for each embedding operand format (BF16,
    FP8 E4M3) the GAP iterations with K' candidates per key by embedding score re-ranked exactly
    (timed like the other forms), the PSNR against the chosen form, and the recall of the
    exhaustive top-K on frame 0 of the chosen form's final estimate (trained and untrained)."""
    import torch

    from paper_2301_03047_gb300 import glr

    t0 = time.perf_counter()
    x0 = glr.gap_step(y[None], masks, None).view(cfg.T, 1, cfg.H, cfg.W)
    xt = x0[:2].contiguous()
    kt, nt, _ = glr.select_keys(xt, cfg.P, cfg.N, cfg.edge_th)
    it, _ = glr.match_topk(xt, cfg.P, kt, nt, cfg.K, "bf16")
    enc = glr.Encoder(seed=0, device=dev)
    hist = glr.train_encoder(enc, [(xt, cfg.P, kt, nt, it)], steps=args.learned_steps, batch_pairs=32768)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del x0, xt, kt, nt, it
    torch.cuda.empty_cache()
    kov = args.learned_k_over
    # recall of the exhaustive top-K among the learned proposal's K results, frame 0
    x1 = x_final[0:1].reshape(1, 1, cfg.H, cfg.W).contiguous().to(dev)
    k1, n1, _ = glr.select_keys(x1, cfg.P, cfg.N, cfg.edge_th)
    n = int(n1[0].item())
    ie, _ = glr.match_topk(x1, cfg.P, k1, n1, cfg.K, "bf16")
    ie = ie[0, :n]

    def recall(e, kv, fmt):
        il, _ = glr.match_topk(x1, cfg.P, k1, n1, cfg.K, "learned", k_over=kv, encoder=e.params, emb_format=fmt)
        return round(float((il[0, :n, :, None] == ie[:, None, :]).any(-1).float().mean().item()), 4)

    enc0 = glr.Encoder(seed=0, device=dev)
    out = {"k_over": kov, "steps": args.steps,
           "recall_of": f"exhaustive BF16 top-{cfg.K} of all {n} keys of frame 0 (chosen form's final estimate)",
           "train": {"steps": args.learned_steps, "pairs_per_step": 32768, "frames": 2, "s": round(t_train, 2),
                     "loss_first": round(hist[0], 4), "loss_last": round(hist[-1], 4)}}
    for fmt in ("bf16", "e4m3"):
        rec = glr.SciReconstructor(cfg.T, cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, mode="learned", edge_th=cfg.edge_th,
                                   device=dev, k_over=kov, frames_per_call=fpc, encoder=enc.params,
                                   emb_format=fmt)
        rec.start(y, masks)
        k = 0
        for _ in range(args.warmup):
            rec.step(sched[k % len(sched)], cfg.c_wnnm)
            k += 1
        torch.cuda.synchronize()
        glr.profile_enable(True)
        glr.profile_collect()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record()
            rec.step(sched[k % len(sched)], cfg.c_wnnm)
            ev[i][1].record()
            k += 1
        torch.cuda.synchronize()
        prof = glr.profile_collect()
        glr.profile_enable(False)
        ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        psnr = psnr_framewise(rec.x.cpu().numpy()[0], prob.truth)
        _, mcnt = glr.poll_status(rec.den.ws_match)  # counters of the last call (frames_per_call frames)
        cand = mcnt[4] / ((fpc or cfg.T) * cfg.N)
        del rec
        torch.cuda.empty_cache()
        r = {"value": round(1e3 / ms, 4), "unit": UNIT, "ms_per_step": round(ms, 3), "psnr_db": round(psnr, 3),
             "delta_psnr_db_vs_chosen": round(psnr - chosen["psnr"], 4),
             "speedup_vs_chosen": round(chosen["ms_per_step"] / ms, 3),
             "candidate_chunks_per_key": round(cand, 1),
             "recall_trained": {str(kv): recall(enc, kv, fmt) for kv in sorted({kov // 2, kov})},
             "recall_untrained": recall(enc0, kov, fmt),
             "kernels": {kn: {"ms_per_step": round(v[0] / args.steps, 3), "launches": v[1]}
                         for kn, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}}
        if plain is not None:
            r["speedup_vs_plain"] = round(plain["ms_per_step"] / ms, 3)
            r["delta_psnr_db_vs_plain"] = round(psnr - plain["psnr"], 4)
        out[fmt] = r
    return out, enc


def run_quality(args, cfg, prob, y, masks, sched, dev, fpc, tuned, forms, enc) -> dict:
    """PSNR after the workload's full iteration count (untimed), every form from the same start:
    the exhaustive forms and, when an encoder was trained, the learned proposal in both formats."""
    import torch

    from paper_2301_03047_gb300 import glr

    runs = [(f, dict(mode=f, **tuned[f])) for f in forms]
    if enc is not None:
        runs += [(f"learned_{fmt}", dict(mode="learned", k_over=args.learned_k_over, encoder=enc.params,
                                         emb_format=fmt)) for fmt in ("bf16", "e4m3")]
    psnr = {}
    for name, kw in runs:
        rec = glr.SciReconstructor(cfg.T, cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, edge_th=cfg.edge_th, device=dev,
                                   frames_per_call=fpc, **kw)
        rec.start(y, masks)
        for k in range(cfg.iters):
            rec.step(sched[k % len(sched)], cfg.c_wnnm)
        torch.cuda.synchronize()
        psnr[name] = round(psnr_framewise(rec.x.cpu().numpy()[0], prob.truth), 3)
        del rec
        torch.cuda.empty_cache()
    base = psnr[forms[0]]
    return {"iters": cfg.iters, "psnr_db": psnr, "delta_vs_chosen_db": {k: round(v - base, 3) for k, v in psnr.items()}}


def run_glr(args) -> None:
    import numpy as np
    import torch

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = init_dist("nccl")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2301_03047_gb300 import glr, synth

    cfg = workload(args.workload)
    if isinstance(cfg, synth.MriConfig):
        return run_mri(args, cfg, dev, dist)
    if isinstance(cfg, synth.MsfaConfig):
        return run_msfa(args, cfg, dev, dist)
    prob = synth.sci_problem(cfg)
    y = torch.from_numpy(prob.y).to(dev)
    masks = torch.from_numpy(prob.masks).to(dev)
    sched = cfg.sigma_schedule()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    pk = peaks()
    forms = [args.mode] + (["fp32"] if args.mode != "fp32" and not args.no_plain else [])
    results = {}
    prof = None
    clocks_summary = None
    sweeps = 0.0
    census = None
    svd_noconv = None
    stream_stats = None
    launches = 0
    tuned = {}
    # frames of 2048^2: the denoiser works on 8 frames at a time (workspaces sized for 8); the
    # plain form (about 6 s per iteration there) is timed over 3 iterations after 2 warm-ups
    huge = cfg.H * cfg.W >= 2048 * 2048
    fpc = 8 if huge else 0
    for form in forms:
        headline = form == forms[0]
        n_steps = args.steps if (headline or not huge) else min(args.steps, 3)
        n_warm = args.warmup if (headline or not huge) else 2
        # autotune the matching schedule on the start image (set-up, untimed)
        if args.match_schedule and headline:
            tuned[form] = sched_kw(args.match_schedule.split(","))
        elif args.no_tune or huge:
            tuned[form] = sched_kw(())
        else:
            x0 = glr.gap_step(y[None], masks, None).view(cfg.T, 1, cfg.H, cfg.W).contiguous()
            k0, n0, _ = glr.select_keys(x0, cfg.P, cfg.N, cfg.edge_th)
            tuned[form] = sched_kw(glr.autotune_match(x0, cfg.P, k0, n0, cfg.K, form))
            del x0, k0, n0
        rec = glr.SciReconstructor(cfg.T, cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, mode=form, edge_th=cfg.edge_th,
                                   device=dev, frames_per_call=fpc, **tuned[form])
        rec.start(y, masks)
        k = 0
        for _ in range(n_warm):
            rec.step(sched[k % len(sched)], cfg.c_wnnm)
            k += 1
        torch.cuda.synchronize()
        if headline:
            glr.profile_enable(True)
            glr.profile_collect()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_steps)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = glr.launch_count()
        clk = Clocks(local) if headline else None
        if clk:
            clk.__enter__()
        for i in range(n_steps):
            flush.zero_()
            ev[i][0].record()
            rec.step(sched[k % len(sched)], cfg.c_wnnm)
            ev[i][1].record()
            k += 1
        torch.cuda.synchronize()
        if clk:
            clk.__exit__()
            clocks_summary = clk.summary()
        if dist is not None:
            dist.barrier()
        step_ms = [a.elapsed_time(b) for a, b in ev]
        total_s = reduce_max(sum(step_ms) / 1e3, dist, dev)
        if not headline:
            # quality is compared at equal iteration counts: untimed steps up to the chosen form's count
            while k < results[forms[0]]["iters"]:
                rec.step(sched[k % len(sched)], cfg.c_wnnm)
                k += 1
        if headline:
            launches = glr.launch_count() - l0
            prof = glr.profile_collect()
            glr.profile_enable(False)
            bits, cnt = glr.poll_status(rec.den.ws_lowrank_status)
            sweeps = cnt[2] / max(cnt[3], 1)
            svd_noconv = cnt[1]
            if not fpc:  # frames in one call: every iteration's counts can be read back
                census = lowrank_census(cfg, y, masks, sched, dev, form, tuned[form], n_warm, n_steps)
                sweeps = census["sweeps_per_group"]
            _, mcnt = glr.poll_status(rec.den.ws_match)
            stream_stats = {"appends_per_key": round(mcnt[4] / (cfg.T * cfg.N), 1),
                            "compactions_per_key": round(mcnt[5] / (cfg.T * cfg.N), 2)}
        x = rec.x.cpu().numpy()[0]
        if headline:
            x_final = torch.from_numpy(x)
        results[form] = {"total_s": total_s, "ms_per_step": total_s / n_steps * 1e3, "step_ms": step_ms,
                         "psnr": psnr_framewise(x, prob.truth), "iters": k, "steps": n_steps}
        if headline and not args.no_graph:
            # the same noise levels as the eager timing, replayed from CUDA graphs (one per level)
            rec.capture(sched, cfg.c_wnnm)
            for i in range(args.warmup):
                rec.step_graph(sched[i % len(sched)])
            gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()
            for i in range(args.steps):
                flush.zero_()
                gev[i][0].record()
                rec.step_graph(sched[(args.warmup + i) % len(sched)])
                gev[i][1].record()
            torch.cuda.synchronize()
            g_s = reduce_max(sum(a.elapsed_time(b) for a, b in gev) / 1e3, dist, dev)
            results["graph"] = {"ms_per_step": g_s / args.steps * 1e3, "value": ws * args.steps / g_s}
        del rec
        torch.cuda.empty_cache()

    learned = enc = quality = None
    if args.learned == 1 or (args.learned < 0 and huge):
        learned, enc = run_learned(args, cfg, prob, y, masks, sched, dev, fpc, flush, x_final, results[forms[0]],
                                   results.get("fp32"))
    if args.quality == 1 or (args.quality < 0 and huge):
        quality = run_quality(args, cfg, prob, y, masks, sched, dev, fpc, tuned, forms, enc)
    head = results[forms[0]]
    value = ws * args.steps / head["total_s"]
    npos = (cfg.H - cfg.P + 1) * (cfg.W - cfg.P + 1)
    pairs_per_iter = cfg.T * cfg.N * npos

    # e2e through the public API with host buffers (chosen form)
    e2e = None
    if not args.no_e2e:
        y_h = torch.from_numpy(prob.y).pin_memory()
        m_h = torch.from_numpy(prob.masks).pin_memory()
        x_h = torch.empty((1, cfg.T, cfg.H, cfg.W), dtype=torch.float32).pin_memory()
        rec = glr.SciReconstructor(cfg.T, cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, mode=forms[0], edge_th=cfg.edge_th,
                                   device=dev, frames_per_call=fpc, **tuned[forms[0]])
        y_d = torch.empty_like(y)
        m_d = torch.empty_like(masks)
        y_d.copy_(y_h, non_blocking=True)
        m_d.copy_(m_h, non_blocking=True)
        rec.start(y_d, m_d)
        use_graph = not args.no_graph  # the public API's graph replay (SciReconstructor.capture / step_graph)
        if use_graph:
            rec.capture(sched, cfg.c_wnnm)
        run = (lambda s: rec.step_graph(s)) if use_graph else (lambda s: rec.step(s, cfg.c_wnnm))
        for i in range(args.warmup):
            run(sched[i % len(sched)])
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            # this step's snapshot and masks come from pinned host memory, the estimate goes back
            y_d.copy_(y_h, non_blocking=True)
            m_d.copy_(m_h, non_blocking=True)
            run(sched[(args.warmup + i) % len(sched)])
            x_h.copy_(rec.x, non_blocking=True)
            torch.cuda.current_stream().synchronize()
        e2e_s = reduce_max(time.perf_counter() - t0, dist, dev)
        e2e = {"value": round(ws * args.steps / e2e_s, 4), "unit": UNIT,
               "h2d_bytes_per_step": int(y_h.numel() * 4 + m_h.numel() * 4),
               "d2h_bytes_per_step": int(x_h.numel() * 4), "via": "graph replay" if use_graph else "eager"}
        del rec

    # one GLR step of the chosen form on frame 0 of the final state, saved for the oracle check
    oracle_inputs = None
    if rank == 0 and not args.no_cpu:
        import numpy as np

        x1 = x_final[0:1].reshape(1, 1, cfg.H, cfg.W).contiguous().to(dev)
        sw_c = sched[len(sched) // 2]
        k1, n1, _ = glr.select_keys(x1, cfg.P, cfg.N, cfg.edge_th)
        i1, d1 = glr.match_topk(x1, cfg.P, k1, n1, cfg.K, forms[0], **tuned[forms[0]])
        g1, _ = glr.lowrank_groups(x1, cfg.P, i1, n1, sw_c, cfg.c_wnnm)
        v1 = glr.aggregate(g1, i1, n1, x1, cfg.P)
        torch.cuda.synchronize()
        fd, oracle_inputs = tempfile.mkstemp(suffix=".npz")
        os.close(fd)
        np.savez(oracle_inputs, x=x1.cpu().numpy()[0], keys=k1.cpu().numpy()[0], idx=i1.cpu().numpy()[0],
                 dist=d1.cpu().numpy()[0], groups=g1.cpu().numpy()[0], v=v1.cpu().numpy()[0], P=cfg.P, K=cfg.K,
                 N=cfg.N, sw=sw_c, cw=cfg.c_wnnm, th=cfg.edge_th)
        del x1, k1, n1, i1, d1, g1, v1
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu:
        try:
            if huge:  # a 2048^2 frame: each key's scan is 16x longer, so fewer keys
                cpu = cpu_baseline_entry(max(4, args.oracle_keys // 4), "oracle_sample_huge", gb_per_proc=8.0)
            else:
                cpu = cpu_baseline_entry(args.oracle_keys, "oracle_sample")
        except Exception as e:  # the CPU baseline must not hide the GPU result
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": f"failed: {e}"}
        if oracle_inputs is not None:
            try:
                cpu["oracle_error"] = run_oracle_check(oracle_inputs)
            except Exception as e:
                cpu["oracle_error"] = {"failed": str(e)[-300:]}
            os.unlink(oracle_inputs)
    # a launch covers frames_per_call frames when the frames are processed in groups
    rl = roofline(prof, cfg, sweeps, clocks_summary or {}, pk, n_img=fpc or None, census=census) if prof else None
    kernels = {k: {"ms_per_step": round(v[0] / args.steps, 3), "launches": v[1]} for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])} if prof else {}
    line = {
        "metric": METRIC,
        "value": round(value, 4),
        "unit": UNIT,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(head["ms_per_step"], 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if forms[0] == "fp32" else "bf16",
        "data": "synthetic (seeded moving-shapes scenes, Bernoulli masks; stand-in for the paper's CACTI videos)",
        "config": {"workload": cfg.name, "frames": cfg.T, "H": cfg.H, "W": cfg.W, "P": cfg.P, "N": cfg.N, "K": cfg.K,
                   "positions_per_frame": npos, "match_form": forms[0], "parallelism": f"replicas x{ws}",
                   "l2": "flushed (256 MB write) between timed steps"},
        "pair_dists_per_s": round(ws * pairs_per_iter * args.steps / head["total_s"], 1),
        "psnr_db": round(head["psnr"], 3),
        "gpu_launches": launches,
        "kernels": kernels,
        "svd_sweeps_per_group": round(sweeps, 2),
        "svd_rank1_certified": round(census["rank1_per_group"], 4) if census else None,
        "svd_power_steps_per_group": round(census["power_steps_per_group"], 2) if census else None,
        "svd_rank1_by_gram_bound": round(census["rank1_gram_per_group"], 4) if census else None,
        "svd_groups_at_sweep_cap": svd_noconv,
        "topk_streams": stream_stats,
        "roofline": rl,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks_summary,
    }
    line["autotuned_match"] = tuned
    if learned is not None:
        line["learned"] = learned
    if quality is not None:
        line["quality_full_iters"] = quality
    if "graph" in results:
        line["cuda_graph"] = {"value": round(results["graph"]["value"], 4), "unit": UNIT,
                              "ms_per_step": round(results["graph"]["ms_per_step"], 3)}
    if len(forms) > 1:
        pl = results["fp32"]
        line["plain"] = {"value": round(ws * pl["steps"] / pl["total_s"], 4), "unit": UNIT,
                         "ms_per_step": round(pl["ms_per_step"], 3), "psnr_db": round(pl["psnr"], 3),
                         "steps": pl["steps"],
                         "pair_dists_per_s": round(ws * pairs_per_iter * pl["steps"] / pl["total_s"], 1)}
        line["speedup_vs_plain"] = round(pl["ms_per_step"] / head["ms_per_step"], 3)
        line["delta_psnr_db"] = round(head["psnr"] - pl["psnr"], 4)
    print(json.dumps(line))


MRI_METRIC = "GLR ADMM iterations/s on Fourier-domain (MRI) reconstruction (chosen BF16 form; plain FP32 alongside)"


def oracle_sample_mri(n_keys: int = 8) -> dict:
    import numpy as np

    from oracle import glr_oracle as O
    from oracle import mri_oracle as MO
    from paper_2301_03047_gb300 import synth

    cfg = synth.MRI_LARGE
    prob = synth.mri_problem(cfg)
    sw = cfg.sigma_schedule()[0]
    y = MO.planes_to_complex(prob.y)
    x = MO.complex_to_planes(MO.ifft2c(y))
    t0 = time.perf_counter()
    keys, _ = O.select_keys(x, cfg.P, cfg.N, cfg.edge_th)
    t_select = time.perf_counter() - t0
    t0 = time.perf_counter()
    Q = O.patch_matrix(x, cfg.P)
    t_q = time.perf_counter() - t0
    sample = keys[:n_keys]
    t0 = time.perf_counter()
    idx, _ = O.match_topk(x, cfg.P, sample, cfg.K, Q)
    t_match = (time.perf_counter() - t0) / n_keys
    t0 = time.perf_counter()
    g = O.gather_groups(x, cfg.P, idx, Q)
    xh, _ = MO.lowrank_groups_complex(g, sw, cfg.c_wnnm)
    t_low = (time.perf_counter() - t0) / n_keys
    t0 = time.perf_counter()
    O.aggregate(xh, idx, x, cfg.P)
    t_agg = (time.perf_counter() - t0) / n_keys
    t0 = time.perf_counter()
    MO.admm_dc(y, prob.mask, MO.planes_to_complex(x), cfg.rho)
    t_dc = time.perf_counter() - t0
    t_iter = t_select + t_q + cfg.N * (t_match + t_low + t_agg) + t_dc
    npos = (cfg.H - cfg.P + 1) * (cfg.W - cfg.P + 1)
    return {
        "t_iter_s": t_iter,
        "iters_per_s": 1.0 / t_iter,
        "pair_dists_per_s": npos / t_match,
        "sample": f"full key selection + {n_keys} of {cfg.N} keys matched over all {npos} positions, grouped, "
        f"complex WNNM, aggregated; one data-consistency step; extrapolated linearly to {cfg.N} keys",
    }


def run_mri(args, cfg, dev, dist) -> None:
    import numpy as np
    import torch

    from paper_2301_03047_gb300 import glr, synth

    ws, rank, local = dist_info()
    prob = synth.mri_problem(cfg)
    y = torch.from_numpy(prob.y).to(dev)
    mask = torch.from_numpy(prob.mask).to(dev)
    gt = prob.truth[0].astype(np.float64) + 1j * prob.truth[1]
    sched = cfg.sigma_schedule()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    pk = peaks()
    forms = [args.mode] + (["fp32"] if args.mode != "fp32" and not args.no_plain else [])
    results, tuned = {}, {}
    prof = clocks_summary = stream_stats = None
    sweeps, launches = 0.0, 0

    def psnr(rec):
        x = rec.x.cpu().numpy()[0]
        return 10.0 * math.log10(1.0 / float(np.mean(np.abs(x[0] + 1j * x[1] - gt) ** 2)))

    for form in forms:
        x0 = glr.fft2(y[None], inverse=True)
        k0, n0, _ = glr.select_keys(x0, cfg.P, cfg.N, cfg.edge_th)
        if args.match_schedule and form == forms[0]:
            tuned[form] = sched_kw(args.match_schedule.split(","))
        else:
            tuned[form] = sched_kw(glr.autotune_match(x0, cfg.P, k0, n0, cfg.K, form) if not args.no_tune else ())
        del x0, k0, n0
        rec = glr.MriReconstructor(cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, mode=form, edge_th=cfg.edge_th, rho=cfg.rho,
                                   device=dev, **tuned[form])
        rec.start(y, mask)
        k = 0
        for _ in range(args.warmup):
            rec.step(sched[k % len(sched)], cfg.c_wnnm)
            k += 1
        torch.cuda.synchronize()
        headline = form == forms[0]
        if headline:
            glr.profile_enable(True)
            glr.profile_collect()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = glr.launch_count()
        clk = Clocks(local) if headline else None
        if clk:
            clk.__enter__()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record()
            rec.step(sched[k % len(sched)], cfg.c_wnnm)
            ev[i][1].record()
            k += 1
        torch.cuda.synchronize()
        if clk:
            clk.__exit__()
            clocks_summary = clk.summary()
        if dist is not None:
            dist.barrier()
        total_s = reduce_max(sum(a.elapsed_time(b) for a, b in ev) / 1e3, dist, dev)
        if headline:
            launches = glr.launch_count() - l0
            prof = glr.profile_collect()
            glr.profile_enable(False)
            _, cnt = glr.poll_status(rec.den.ws_lowrank_status)
            sweeps = cnt[2] / max(cnt[3], 1)
            _, mcnt = glr.poll_status(rec.den.ws_match)
            stream_stats = {"appends_per_key": round(mcnt[4] / cfg.N, 1),
                            "compactions_per_key": round(mcnt[5] / cfg.N, 2)}
        results[form] = {"total_s": total_s, "ms_per_step": total_s / args.steps * 1e3, "psnr": psnr(rec),
                         "residual": float(rec.residual[0])}
        if headline and not args.no_graph:
            # the same noise levels as the eager timing, replayed from CUDA graphs (one per level)
            rec.capture(sched, cfg.c_wnnm)
            for i in range(args.warmup):
                rec.step_graph(sched[i % len(sched)])
            gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()
            for i in range(args.steps):
                flush.zero_()
                gev[i][0].record()
                rec.step_graph(sched[(args.warmup + i) % len(sched)])
                gev[i][1].record()
            torch.cuda.synchronize()
            g_s = reduce_max(sum(a.elapsed_time(b) for a, b in gev) / 1e3, dist, dev)
            results["graph"] = {"ms_per_step": g_s / args.steps * 1e3, "value": ws * args.steps / g_s}
        del rec
        torch.cuda.empty_cache()

    head = results[forms[0]]
    e2e = None
    if not args.no_e2e:
        y_h = torch.from_numpy(prob.y).pin_memory()
        m_h = torch.from_numpy(prob.mask).pin_memory()
        x_h = torch.empty((1, 2, cfg.H, cfg.W), dtype=torch.float32).pin_memory()
        rec = glr.MriReconstructor(cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, mode=forms[0], edge_th=cfg.edge_th,
                                   rho=cfg.rho, device=dev, **tuned[forms[0]])
        y_d, m_d = torch.empty_like(y), torch.empty_like(mask)
        y_d.copy_(y_h, non_blocking=True)
        m_d.copy_(m_h, non_blocking=True)
        rec.start(y_d, m_d)
        use_graph = not args.no_graph
        if use_graph:
            rec.capture(sched, cfg.c_wnnm)
        run = (lambda s: rec.step_graph(s)) if use_graph else (lambda s: rec.step(s, cfg.c_wnnm))
        for i in range(args.warmup):
            run(sched[i % len(sched)])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.steps):
            y_d.copy_(y_h, non_blocking=True)
            m_d.copy_(m_h, non_blocking=True)
            run(sched[(args.warmup + i) % len(sched)])
            x_h.copy_(rec.x, non_blocking=True)
            torch.cuda.current_stream().synchronize()
        e2e_s = reduce_max(time.perf_counter() - t0, dist, dev)
        e2e = {"value": round(ws * args.steps / e2e_s, 4), "unit": UNIT,
               "h2d_bytes_per_step": int(y_h.numel() * 4 + m_h.numel() * 4), "d2h_bytes_per_step": int(x_h.numel() * 4),
               "via": "graph replay" if use_graph else "eager"}
        del rec
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu:
        try:
            cpu = cpu_baseline_entry(args.oracle_keys, "oracle_sample_mri")
        except Exception as e:
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": f"failed: {e}"}
    npos = (cfg.H - cfg.P + 1) * (cfg.W - cfg.P + 1)
    rl = roofline(prof, cfg, sweeps, clocks_summary or {}, pk, n_img=1, d=2 * cfg.P * cfg.P) if prof else None
    line = {
        "metric": MRI_METRIC, "value": round(ws * args.steps / head["total_s"], 4), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(head["ms_per_step"], 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if forms[0] == "fp32" else "bf16",
        "data": "synthetic (seeded complex ellipse phantom, Cartesian variable-density k-space rows)",
        "config": {"workload": cfg.name, "H": cfg.H, "W": cfg.W, "P": cfg.P, "d": 2 * cfg.P * cfg.P, "N": cfg.N,
                   "K": cfg.K, "rho": cfg.rho, "positions": npos, "match_form": forms[0],
                   "parallelism": f"replicas x{ws}", "l2": "flushed (256 MB write) between timed steps"},
        "pair_dists_per_s": round(ws * cfg.N * npos * args.steps / head["total_s"], 1),
        "psnr_db": round(head["psnr"], 3), "dc_residual": head["residual"], "gpu_launches": launches,
        "kernels": {k: {"ms_per_step": round(v[0] / args.steps, 3), "launches": v[1]}
                    for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])} if prof else {},
        "svd_sweeps_per_group": round(sweeps, 2), "topk_streams": stream_stats, "roofline": rl,
        "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks_summary,
        "autotuned_match": tuned,
    }
    if "graph" in results:
        line["cuda_graph"] = {"value": round(results["graph"]["value"], 4), "unit": UNIT,
                              "ms_per_step": round(results["graph"]["ms_per_step"], 3)}
    if len(forms) > 1:
        pl = results["fp32"]
        line["plain"] = {"value": round(ws * args.steps / pl["total_s"], 4), "unit": UNIT,
                         "ms_per_step": round(pl["ms_per_step"], 3), "psnr_db": round(pl["psnr"], 3)}
        line["speedup_vs_plain"] = round(pl["total_s"] / head["total_s"], 3)
        line["delta_psnr_db"] = round(head["psnr"] - pl["psnr"], 4)
    print(json.dumps(line))


MSFA_METRIC = "GLR GAP iterations/s on MSFA demosaicing of an uneven batch (chosen BF16 form; plain FP32 alongside)"


def oracle_sample_msfa(n_keys: int = 4) -> dict:
    from oracle import glr_oracle as O
    from oracle import msfa_oracle as FO
    from paper_2301_03047_gb300 import synth

    cfg = synth.MSFA_LARGE
    side = 256  # one of the batch's smallest images; the rest scale by their key and position counts
    im = synth.msfa_problem(synth.MsfaConfig("s", cfg.config_no, sides=(side,), bands=cfg.bands, P=cfg.P, K=cfg.K,
                                             iters=1))[0]
    x = FO.mosaic_init(im.y, im.masks, 4)
    t0 = time.perf_counter()
    keys, _ = O.select_keys(x, cfg.P, im.N, cfg.edge_th)
    Q = O.patch_matrix(x, cfg.P)
    t_fixed = time.perf_counter() - t0
    t0 = time.perf_counter()
    idx, _ = O.match_topk(x, cfg.P, keys[:n_keys], cfg.K, Q)
    g = O.gather_groups(x, cfg.P, idx, Q)
    xh, _ = O.lowrank_groups(g, cfg.sigma_schedule()[0], cfg.c_wnnm)
    O.aggregate(xh, idx, x, cfg.P)
    t_key = (time.perf_counter() - t0) / n_keys
    npos0 = (side - cfg.P + 1) ** 2
    # per-key work scales with the positions searched; fixed work with the pixels
    t_iter = sum(t_fixed * (s / side) ** 2 + cfg.N_of(s) * t_key * ((s - cfg.P + 1) ** 2 / npos0) for s in cfg.sides)
    return {"t_iter_s": t_iter, "iters_per_s": 1.0 / t_iter,
            "sample": f"one {side}x{side} image: key selection + {n_keys} of {im.N} keys matched over all {npos0} "
            f"positions, grouped, WNNM, aggregated; extrapolated by pixels and positions to the {len(cfg.sides)} images"}


def run_msfa(args, cfg, dev, dist) -> None:
    import numpy as np
    import torch

    from paper_2301_03047_gb300 import glr, synth

    ws, rank, local = dist_info()
    imgs = synth.msfa_problem(cfg)
    sides = [im.y.shape[0] for im in imgs]
    Ns = [im.N for im in imgs]
    ys = [torch.from_numpy(im.y).to(dev) for im in imgs]
    masks = {s: torch.from_numpy(synth.mosaic_masks(s, s, cfg.bands)).to(dev) for s in set(sides)}
    sched = cfg.sigma_schedule()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    forms = [args.mode] + (["fp32"] if args.mode != "fp32" and not args.no_plain else [])
    results = {}
    prof = clocks_summary = None
    launches = 0
    sweeps = 0.0
    pairs = sum(n * (s - cfg.P + 1) ** 2 for s, n in zip(sides, Ns))

    def psnr(rec):
        return float(np.mean([10 * math.log10(1.0 / float(np.mean((x.cpu().numpy() - im.truth) ** 2)))
                              for x, im in zip(rec.images(), imgs)]))

    fixed = None  # --match-schedule: one schedule for every size class of the chosen form
    if args.match_schedule:
        t = tuple(sched_kw(args.match_schedule.split(",")).values())
        fixed = {(int(sd), int(n)): t for sd, n in zip(sides, Ns)}
    for form in forms:
        # the chosen BF16 form matches the whole batch in one persistent launch (glr_match_topk_batch)
        rec = glr.MsfaBatchReconstructor(sides, Ns, cfg.bands, cfg.P, cfg.K, mode=form, edge_th=cfg.edge_th,
                                         device=dev, tuned=fixed if form == forms[0] else None,
                                         persistent=form == "bf16" and not args.no_persistent)
        rec.start(ys, masks)
        steps = args.steps
        k = 0
        for _ in range(args.warmup):
            rec.step(sched[k % len(sched)], cfg.c_wnnm)
            k += 1
        torch.cuda.synchronize()
        headline = form == forms[0]
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = glr.launch_count()
        clk = Clocks(local) if headline else None
        if clk:
            clk.__enter__()
        for i in range(steps):
            flush.zero_()
            ev[i][0].record()
            rec.step(sched[k % len(sched)], cfg.c_wnnm)
            ev[i][1].record()
            k += 1
        torch.cuda.synchronize()
        if clk:
            clk.__exit__()
            clocks_summary = clk.summary()
        total_s = reduce_max(sum(a.elapsed_time(b) for a, b in ev) / 1e3, dist, dev)
        if headline:
            launches = glr.launch_count() - l0
        results[form] = {"total_s": total_s, "steps": steps, "ms_per_step": total_s / steps * 1e3, "psnr": psnr(rec)}
        if headline:
            # per-kernel times with the classes run one after the other (concurrent classes would
            # stretch each other's event intervals)
            rec.concurrent = False
            glr.profile_enable(True)
            glr.profile_collect()
            rec.step(sched[k % len(sched)], cfg.c_wnnm)
            torch.cuda.synchronize()
            prof = glr.profile_collect()
            glr.profile_enable(False)
            rec.concurrent = True
            sw_groups = [glr.poll_status(c["den"].ws_lowrank_status)[1] for c in rec.classes]
            sweeps = sum(c[2] for c in sw_groups) / max(1, sum(c[3] for c in sw_groups))
            if not args.no_graph:
                rec.capture(sched, cfg.c_wnnm)
                for i in range(args.warmup):
                    rec.step_graph(sched[i % len(sched)])
                gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
                torch.cuda.synchronize()
                for i in range(steps):
                    flush.zero_()
                    gev[i][0].record()
                    rec.step_graph(sched[(args.warmup + i) % len(sched)])
                    gev[i][1].record()
                torch.cuda.synchronize()
                g_s = reduce_max(sum(a.elapsed_time(b) for a, b in gev) / 1e3, dist, dev)
                results["graph"] = {"ms_per_step": g_s / steps * 1e3, "value": ws * steps / g_s}
        del rec
        torch.cuda.empty_cache()
    head = results[forms[0]]
    e2e = None
    if not args.no_e2e:
        y_h = [torch.from_numpy(im.y).pin_memory() for im in imgs]
        rec = glr.MsfaBatchReconstructor(sides, Ns, cfg.bands, cfg.P, cfg.K, mode=forms[0], edge_th=cfg.edge_th,
                                         device=dev, tuned=fixed,
                                         persistent=forms[0] == "bf16" and not args.no_persistent)
        y_d = [torch.empty_like(y) for y in ys]
        for a, b in zip(y_d, y_h):
            a.copy_(b, non_blocking=True)
        rec.start(y_d, masks)
        out_h = [torch.empty((cfg.bands, s, s), dtype=torch.float32).pin_memory() for s in sides]
        use_graph = not args.no_graph
        if use_graph:
            rec.capture(sched, cfg.c_wnnm)
        run = (lambda s: rec.step_graph(s)) if use_graph else (lambda s: rec.step(s, cfg.c_wnnm))
        for i in range(args.warmup):
            run(sched[i % len(sched)])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(head["steps"]):
            for c in rec.classes:  # the snapshots of each class come from pinned host memory
                for j, idx in enumerate(c["ids"]):
                    c["y"][j].copy_(y_h[idx], non_blocking=True)
            run(sched[(args.warmup + i) % len(sched)])
            for o, x in zip(out_h, rec.images()):
                o.copy_(x, non_blocking=True)
            torch.cuda.current_stream().synchronize()
        e2e_s = reduce_max(time.perf_counter() - t0, dist, dev)
        e2e = {"value": round(ws * head["steps"] / e2e_s, 4), "unit": UNIT,
               "h2d_bytes_per_step": int(sum(y.numel() for y in y_h) * 4),
               "d2h_bytes_per_step": int(sum(o.numel() for o in out_h) * 4),
               "via": "graph replay" if use_graph else "eager"}
        del rec
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu:
        try:
            cpu = cpu_baseline_entry(min(args.oracle_keys, 16), "oracle_sample_msfa")
        except Exception as e:
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": f"failed: {e}"}
    pk = peaks()
    rl = None
    if prof:
        scans = "k_match_tc_min" in prof
        name, (ms, n) = max(merge_scans(prof).items(), key=lambda kv: kv[1][0])
        rl = {"kernel": name, "ms_per_step_serial": round(ms, 3), "launches": n,
              "note": "per-kernel times from one iteration with the size classes serialised"
                      + ("; k_match_tc = minima scan + bound + candidate scan" if scans and name == "k_match_tc" else "")}
        if name == "k_match_tc":
            work = 2.0 * cfg.bands * cfg.P * cfg.P * pairs
            rl.update({"bound": "tensor", "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
                       "peak_note": f"of {pk['source']} cuBLAS bf16 sustained",
                       "achieved": round(work / (ms / 1e3) / 1e12, 2), "units_per_launch": pairs / n,
                       "unit_kind": "pairs", "traffic": traffic_for("k_match_tc_w", pairs / n)})
            rl["frac"] = round(rl["achieved"] / rl["peak"], 4)
    line = {
        "metric": MSFA_METRIC, "value": round(ws * head["steps"] / head["total_s"], 4), "unit": UNIT, "n_gpus": ws,
        "steps": head["steps"], "warmup": args.warmup, "ms_per_step": round(head["ms_per_step"], 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if forms[0] == "fp32" else "bf16",
        "data": "synthetic (seeded spectral cubes: 6 materials x 4-Gaussian spectra, textured abundances; 4x4 mosaic)",
        "config": {"workload": cfg.name, "images": len(sides), "sides": sorted(set(sides)), "bands": cfg.bands,
                   "P": cfg.P, "d": cfg.bands * cfg.P * cfg.P, "K": cfg.K, "keys_total": int(sum(Ns)),
                   "pairs_per_iter": int(pairs), "match_form": forms[0], "parallelism": f"replicas x{ws}",
                   "batching": "size classes on concurrent streams",
                   "l2": "flushed (256 MB write) between timed steps"},
        "pair_dists_per_s": round(ws * pairs * head["steps"] / head["total_s"], 1), "psnr_db": round(head["psnr"], 3),
        "gpu_launches": launches,
        "kernels_serial": {k: {"ms": round(v[0], 3), "launches": v[1]}
                           for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])} if prof else {},
        "svd_sweeps_per_group": round(sweeps, 2),
        "roofline": rl, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks_summary,
    }
    if "graph" in results:
        line["cuda_graph"] = {"value": round(results["graph"]["value"], 4), "unit": UNIT,
                              "ms_per_step": round(results["graph"]["ms_per_step"], 3)}
    if len(forms) > 1:
        pl = results["fp32"]
        line["plain"] = {"value": round(ws * pl["steps"] / pl["total_s"], 4), "unit": UNIT,
                         "ms_per_step": round(pl["ms_per_step"], 3), "psnr_db": round(pl["psnr"], 3),
                         "steps": pl["steps"]}
        line["speedup_vs_plain"] = round(pl["ms_per_step"] / head["ms_per_step"], 3)
        line["delta_psnr_db"] = round(head["psnr"] - pl["psnr"], 4)
    print(json.dumps(line))


def run_ablation(args) -> None:
    """Matching strategies of the paper's comparison of global and block matching:
    GM (global, corner keys; BF16 and FP32 forms) against block matching in a
    +-20 window with uniform (BM-U), corner (BM-C) and half-and-half (BM-C-U) keys.
    Reports, per strategy, GAP iterations/s, the PSNR after the full schedule and the
    recall of the exact global top-K on the start image."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2301_03047_gb300 import glr, synth

    cfg = workload(args.workload)
    prob = synth.sci_problem(cfg)
    dev = torch.device("cuda", 0)
    y = torch.from_numpy(prob.y).to(dev)
    masks = torch.from_numpy(prob.masks).to(dev)
    sched = cfg.sigma_schedule()
    strategies = [("GM-bf16", "bf16", 0), ("GM-fp32", "fp32", 0), ("BM-U", "window", cfg.N),
                  ("BM-C", "window", 0), ("BM-C-U", "window", cfg.N // 2)]
    x0 = glr.gap_step(y[None], masks, None).view(cfg.T, 1, cfg.H, cfg.W).contiguous()
    out = {}
    for name, mode, nu in strategies:
        k0, n0, _ = glr.select_keys(x0, cfg.P, cfg.N, cfg.edge_th, n_uniform=nu)
        exact, _ = glr.match_topk(x0, cfg.P, k0, n0, cfg.K, "fp32")
        got, _ = glr.match_topk(x0, cfg.P, k0, n0, cfg.K, mode, window=20)
        e, g = exact.cpu().numpy(), got.cpu().numpy()
        hits = sum(len(set(e[f, i].tolist()) & set(g[f, i].tolist())) for f in range(cfg.T) for i in range(cfg.N))
        rec = glr.SciReconstructor(cfg.T, cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, mode=mode, edge_th=cfg.edge_th,
                                   device=dev, n_uniform=nu, window=20)
        rec.start(y, masks)
        rec.step(sched[0], cfg.c_wnnm)  # warm-up (library set-up)
        rec.start(y, masks)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for s in sched:
            rec.step(s, cfg.c_wnnm)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / len(sched)
        out[name] = {"iter_per_s": round(1e3 / ms, 3), "ms_per_iter": round(ms, 3),
                     "psnr_db": round(psnr_framewise(rec.x.cpu().numpy()[0], prob.truth), 3),
                     "recall_of_global_topk": round(hits / (cfg.T * cfg.N * cfg.K), 4), "n_uniform": nu}
        del rec
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "matching-strategy comparison (GM vs block matching)", "workload": cfg.name,
                      "iterations": len(sched), "window": 20, "strategies": out}))


def run_reference(args) -> None:
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    from paper_2301_03047_gb300 import synth

    cfg = synth.SCI_LARGE
    vals = []
    o = None
    # each step is one bounded oracle sample on all host cores; one short warm-up sample is
    # discarded; one single-core sample is recorded beside the result
    if args.warmup > 0:
        run_oracle_child(2)
    t0 = time.perf_counter()
    for i in range(args.steps):
        o = run_oracle_all_cores(max(4, args.oracle_keys // 4))
        vals.append(o["t_iter_s"])
    wall = time.perf_counter() - t0
    one = run_oracle_child(args.oracle_keys)
    t_iter = statistics.mean(vals)
    value = 1.0 / t_iter
    npos = (cfg.H - cfg.P + 1) * (cfg.W - cfg.P + 1)
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 8),
        "unit": UNIT,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(t_iter * 1e3, 1),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded moving-shapes scenes, Bernoulli masks)",
        "config": {"workload": cfg.name, "frames": cfg.T, "H": cfg.H, "W": cfg.W, "P": cfg.P, "N": cfg.N, "K": cfg.K,
                   "positions_per_frame": npos, "match_form": "oracle FP64 direct distances"},
        "cpu_baseline": {"value": round(value, 8), "unit": UNIT, "cores": o["procs"], "nproc": os.cpu_count(),
                         "kind": "oracle", "sample": o["sample"],
                         "single_core": {"value": round(one["iters_per_s"], 8), "unit": UNIT, "cores": 1,
                                         "sample": one["sample"]}},
        "e2e": {"value": round(value, 8), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": round(wall, 1),
        "pair_dists_per_s": round(o["pair_dists_per_s"], 1),
    }
    print(json.dumps(line))


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="glr", choices=["glr", "reference"])
    ap.add_argument("--mode", default="bf16", choices=["bf16", "fp32", "edge"],
                    help="matching form: bf16 (chosen), fp32 (plain), edge (the paper's heat map of Eq. 4)")
    ap.add_argument("--oracle-keys", type=int, default=96)
    ap.add_argument("--workload", default="sci16",
                    choices=["sci16", "sci4", "sci8", "sci24x2048", "sci2x2048", "mri1024", "mri256", "msfa32",
                             "msfa4", "msfa2"],
                    help="sci16 = the headline workload; sci24x2048 = 24 frames of 2048^2 with 16384 keys per "
                    "frame (adds the learned proposal); mri1024 = the MRI (ADMM) path on 1024^2 complex; "
                    "msfa32 = MSFA demosaicing of 32 images of uneven sizes; sci4 / sci8 / sci2x2048 / mri256 / "
                    "msfa4 are smaller cases for profiling")
    ap.add_argument("--learned", type=int, default=-1,
                    help="1: also time the learned proposal (trained encoder); default on for 2048^2 frames")
    ap.add_argument("--learned-k-over", type=int, default=256, help="candidates per key of the learned proposal")
    ap.add_argument("--learned-steps", type=int, default=300, help="encoder training steps (32768 pairs each)")
    ap.add_argument("--quality", type=int, default=-1,
                    help="1: also report every form's PSNR after the workload's full iteration count (untimed); "
                    "default on for 2048^2 frames")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-persistent", action="store_true",
                    help="msfa workloads: match each size class in its own launch instead of one persistent launch")
    ap.add_argument("--ablation", action="store_true",
                    help="print the matching-strategy comparison (GM vs block matching) instead of the bench line")
    ap.add_argument("--match-schedule", default="",
                    help="k_over,splits,cap,epi_batch[,bound_pass]: a fixed matching schedule instead of the autotuner's")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "glr":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.ablation:
        run_ablation(args)
    else:
        run_glr(args)


if __name__ == "__main__":
    main()
