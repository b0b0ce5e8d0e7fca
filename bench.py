#!/usr/bin/env python3
"""Benchmark of the line-list -> cross-section hot path on B300.

Headline: Voigt line-grid evals/s (and lines/s) on the 1e9-line workload
(5e7 polyatomic states, 1e9 transitions in 1e8-line chunks, T = 2000 K,
P = 0.1 bar, grid 0-30000 cm^-1 at 0.01 cm^-1, cut-off 25 cm^-1, intensity
threshold 1e-30 cm/molecule).  One step = one full pass of the hot path over
all 1e9 lines (partition function, intensities, compaction, exact nu sort,
binning, Voigt accumulation).  Inputs are synthetic and seeded.

  value : device-resident inputs, CUDA events around K steps, max over ranks
  e2e   : the same through pxc_cross_section_streamed from pinned host arrays
          (host->device copies of every step inside the timed region) plus the
          device->host read of sigma
  extras: the batched 200-condition opacity table against 200 sequential calls,
          and forward+backward against forward on the two-temperature list

`--impl reference` times the FP64 oracle (the reference arm: there is no other
implementation to install) on bounded samples of the same workload on the host cores.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Voigt line-grid evals/s & lines/s at 1e9 lines; batched, fwd+bwd vs plain"
UNIT = "line-grid evals/s"
# Far-wing (W4 region I) evaluation of the profile kernel, per line-grid point:
#   x = fma(m, step, x0), v = fma(x, x, c1), den = fma(v, v, e), num = fma(v, K, K),
#   acc = fma(num, rcp(den), acc)
# five FP32 FMAs (ten FLOPs) and one MUFU reciprocal: the algorithmic work of one evaluation.
EVAL_FP32_FMAS = 5
EVAL_MUFU = 1
L2_BYTES = 126 * 2 ** 20

# DRAM traffic per launch from an ncu capture (dram__bytes_read.sum + dram__bytes_write.sum),
# valid only for the kernel source it was taken on (sha256 prefix of the .cu file); scaled by lines
# to one 1e8-line launch of voigt_1e9 from the capture of its first 2e7 lines.
NCU_TRAFFIC = {
    ("profile", "d72efc4fdc838484"): 13.79e6 * 5,               # k_profile<voigt>, tile 0
    ("intensity", "d925ec9669974a9d"): (950.5e6 + 317.5e6) * 5,  # k_lines_pre + k_lines_exact
}


def _src_hash(rel):
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                self.rows.append(p)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def slowest_rank_ms(ms_local: float, world: int, device=None) -> float:
    """The job time of `world` independent replicas: the largest of the ranks' own times (one
    MAX all-reduce of a scalar over the default process group; no data-path collective)."""
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank: float, steps: int, world: int, ms_max: float) -> float:
    """Whole-job throughput: every rank processed units_per_rank per step for `steps` steps."""
    return world * units_per_rank * steps / (ms_max / 1e3)


# ----------------------------------------------------------------------------- reference arm (oracle)

def _cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _conditions(w):
    """(T, T_vib, P) conditions of a workload: its batched table, else its one condition."""
    if w.conditions:
        return [(float(T), 0.0, float(P)) for T, P in w.conditions]
    return [(w.T, w.T_vib, w.P)]


def _oracle_condition(w):
    """The condition the CPU baseline times: the workload's own, or the table's middle one."""
    c = _conditions(w)
    return c[len(c) // 2]


def oracle_sample(w, states, n_lines):
    """The FP64 oracle (Q, intensities, sort, sigma on the full grid) on the first n_lines
    transitions of the workload at one condition: (evals of non-zero lines, lines, seconds, result)."""
    import numpy as np
    import oracle
    E, g, Ev = states
    T, Tv, P = _oracle_condition(w)
    up, lo, A = w.transitions(0, n_lines)
    gr, ne = w.broadening(0, n_lines)
    t0 = time.perf_counter()
    r = oracle.run(E, g, Ev if Tv > 0 else None, up, lo, A, gr, ne, kind=w.profile, T=T, T_vib=Tv, P=P,
                   mass_da=w.mass_da, hwhm=w.hwhm, nu_min=w.nu_min, dnu=w.dnu, n_grid=w.n_grid, cut=w.cutoff,
                   threshold=w.threshold)
    dt = time.perf_counter() - t0
    nz = r["keep"].astype(bool) & (r["I_s"] != 0)
    evals = int(np.sum((r["ihi"] - r["ilo"] + 1)[nz]))
    return evals, n_lines, dt, r


def calibrate_sample(w, states, target_s):
    """Lines of a bounded oracle sample taking about target_s seconds (whole list if smaller)."""
    n0 = min(200_000, w.n_trans)
    _, _, dt, _ = oracle_sample(w, states, n0)
    return int(min(max(n0 * target_s / max(dt, 1e-3), n0), 5e7, w.n_trans))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import synth
    w = synth.workload(args.workload)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    states = w.states()
    n = calibrate_sample(w, states, args.ref_step_s)
    for _ in range(args.warmup):
        oracle_sample(w, states, n)
    tot_ev, tot_t = 0, 0.0
    for _ in range(args.steps):
        ev, _, dt, _ = oracle_sample(w, states, n)
        tot_ev += ev
        tot_t += dt
    val = tot_ev / tot_t
    sample = (f"first {n} of {w.n_trans} transitions per step, full grid, condition {_oracle_condition(w)} "
              f"(oracle FP64, {threads} threads)")
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": w.name, "lines": w.n_trans, "states": w.n_states,
                                            "grid": w.n_grid, "profile": w.profile},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def sigma_errors(got, ref):
    """Error of a GPU sigma against the oracle's: max |d| over the peak, the worst per-bin relative
    error where the reference is above 1e-6 of its peak, and the normalised L1 error (Eq. of Sec. 4)."""
    import numpy as np
    m = float(np.abs(ref).max())
    if m == 0.0:
        return {"max_abs_rel_peak": float(np.abs(got).max()), "worst_bin_rel": None, "l1": None}
    d = np.abs(got - ref)
    big = np.abs(ref) > 1e-6 * m
    return {"max_abs_rel_peak": float(d.max() / m), "worst_bin_rel": float((d[big] / np.abs(ref[big])).max()),
            "l1": float(d.sum() / np.abs(ref).sum())}


# ----------------------------------------------------------------------------- GPU arm

def main_pxc(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    import paper_2609_17273_b300 as pxc
    import synth

    rank, world, local = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pxc.load()
    pipes = pxc.pxc_pipe_rates()   # measured FP32 / MUFU rates of this GPU (untimed)

    w = synth.workload(args.workload)
    if args.lines:
        w = w.scaled(n_trans=args.lines)
    conds = _conditions(w)
    n_c = len(conds)
    batched = n_c > 1
    if args.backward and (batched or (w.chunk and w.chunk < w.n_trans)):
        raise SystemExit("--backward needs a single-condition workload held in one chunk")
    chunk = w.chunk or w.n_trans
    nchunks = (w.n_trans + chunk - 1) // chunk
    states_h = w.states()
    E, g, Ev = states_h
    two_t = any(c[1] > 0 for c in conds)
    states = pxc.States(torch.from_numpy(E).to(dev), torch.from_numpy(g).to(dev),
                        torch.from_numpy(Ev).to(dev) if two_t else None)
    broad = w.profile in ("lorentz", "voigt", "binned_lorentz", "binned_voigt")

    # host (pinned) and device copies of the transition list
    a_dtype = torch.float32 if w.A_f32 else torch.float64
    t_gen = time.perf_counter()
    pin = not args.no_e2e
    h_up = torch.empty(w.n_trans, dtype=torch.int32, pin_memory=pin)
    h_lo = torch.empty(w.n_trans, dtype=torch.int32, pin_memory=pin)
    h_A = torch.empty(w.n_trans, dtype=a_dtype, pin_memory=pin)
    h_gr = torch.empty(w.n_trans, dtype=torch.float32, pin_memory=pin)
    h_ne = torch.empty(w.n_trans, dtype=torch.float32, pin_memory=pin)
    d_up = torch.empty(w.n_trans, dtype=torch.int32, device=dev)
    d_lo = torch.empty_like(d_up)
    d_A = torch.empty(w.n_trans, dtype=a_dtype, device=dev)
    d_gr = torch.empty(w.n_trans, dtype=torch.float32, device=dev)
    d_ne = torch.empty_like(d_gr)
    for c in range(nchunks):
        t0, n = c * chunk, min(chunk, w.n_trans - c * chunk)
        sl = slice(t0, t0 + n)
        w.transitions(t0, n, out=(h_up[sl].numpy(), h_lo[sl].numpy(), h_A[sl].numpy()))
        gr, ne = w.broadening(t0, n)
        h_gr[sl].numpy()[:] = gr
        h_ne[sl].numpy()[:] = ne
        for d, h in ((d_up, h_up), (d_lo, h_lo), (d_A, h_A), (d_gr, h_gr), (d_ne, h_ne)):
            d[sl].copy_(h[sl], non_blocking=False)
    t_gen = time.perf_counter() - t_gen

    nT = len({(c[0], c[1]) for c in conds})
    ws = pxc.Workspace(max_states=w.n_states, max_lines=chunk, max_grid=w.n_grid, max_conditions=n_c,
                       max_temperatures=nT, device=dev)
    grid = (w.nu_min, w.dnu, w.n_grid)
    sigma = torch.empty(n_c, w.n_grid, dtype=torch.float32, device=dev)
    sexp = torch.empty(n_c, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    cond_arg = conds if batched else conds[0]

    def chunk_args(c):
        t0, n = c * chunk, min(chunk, w.n_trans - c * chunk)
        sl = slice(t0, t0 + n)
        tr = pxc.Transitions(d_up[sl], d_lo[sl], d_A[sl])
        prof = pxc.Profile(w.profile, w.cutoff, w.mass_da, w.hwhm, d_gr[sl] if broad else None,
                           d_ne[sl] if broad else None)
        return tr, prof

    wgt = torch.from_numpy(w.weights()).to(dev) if args.backward else None
    if args.backward:
        # the adjoint reads back the forward's kept, sorted line list (same arrays in between)
        ws.set_reuse_forward(True)

    def step(count=None):
        if args.backward:
            # forward and the adjoint of L = sum_i w_i sigma_i (one condition, no chunks)
            tr, prof = chunk_args(0)
            pxc.pxc_cross_section(ws, states, tr, cond_arg, grid, prof, w.threshold, sigma=sigma, sigma_exp=sexp)
            pxc.pxc_cross_section_backward(ws, states, tr, cond_arg, grid, prof, wgt, w.threshold)
            if count is not None:
                s = ws.stats()
                count["evals"] += s["evals_nonzero"]; count["evals_window"] += s["evals_window"]
                count["kept"] += s["n_kept"]
            return
        ws.set_accumulate(nchunks > 1)
        if nchunks > 1:
            sigma.zero_()
            sexp.fill_(pxc.PXC_EXP_EMPTY)
        for c in range(nchunks):
            tr, prof = chunk_args(c)
            pxc.pxc_cross_section(ws, states, tr, cond_arg, grid, prof, w.threshold, sigma=sigma, sigma_exp=sexp)
            if count is not None:
                s = ws.stats()
                for k in count:
                    count[k] += s[{"evals": "evals_nonzero", "evals_window": "evals_window",
                                   "kept": "n_kept"}[k]]
        ws.set_accumulate(False)

    # tile configuration of the profile kernel: timed on the first chunk (setup, untimed)
    tune = None
    kind_id = pxc.PROFILES[w.profile]
    if args.tile < 0:
        tr0, pr0 = chunk_args(0)
        t_best, t_ms, _, _ = pxc.pxc_autotune(ws, states, tr0, cond_arg, grid, pr0, w.threshold, repeats=2,
                                              sigma=sigma, sigma_exp=sexp)
        tune = {"tile": t_best, "ms_per_chunk_call": t_ms}
    else:
        ws.set_tile(kind_id, batched, args.tile)
    tile = ws.get_tile(kind_id, batched)

    # one counted step: algorithmic eval counts (the stats cover the last condition of a batched
    # call, so a table counts each condition's evaluations from one call per condition)
    count = {"evals": 0, "evals_window": 0, "kept": 0}
    if batched:
        wsc = pxc.Workspace(max_states=w.n_states, max_lines=chunk, max_grid=w.n_grid, device=dev)
        s1 = torch.empty(1, w.n_grid, dtype=torch.float32, device=dev)
        e1 = torch.empty(1, dtype=torch.int32, device=dev)
        tr0, pr0 = chunk_args(0)
        for cnd in conds:
            pxc.pxc_cross_section(wsc, states, tr0, cnd, grid, pr0, w.threshold, sigma=s1, sigma_exp=e1)
            st_ = wsc.stats()
            count["evals"] += st_["evals_nonzero"]; count["evals_window"] += st_["evals_window"]
            count["kept"] += st_["n_kept"]
        del wsc, s1, e1
    else:
        step(count)
    evals, evals_window, kept = count["evals"], count["evals_window"], count["kept"]
    ws.sync()

    for _ in range(args.warmup):
        step()
    ws.sync()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    clocks = Clocks(local)
    ws.set_timing(True)
    launches0 = pxc.kernel_launches()
    barrier()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    launches = pxc.kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1)
    tm = ws.timing()
    ws.set_timing(False)
    ws.sync()
    ms_max = slowest_rank_ms(ms, world, dev)
    value = replica_rate(evals, args.steps, world, ms_max)
    lines_per_s = replica_rate(w.n_trans, args.steps, world, ms_max)

    # ---------------------------------------------------------------- e2e through the public API, host buffers
    e2e = None
    if not args.no_e2e and not args.backward:
        h_sig = torch.empty(n_c, w.n_grid, dtype=torch.float32, pin_memory=True)
        h_exp = torch.empty(n_c, dtype=torch.int32, pin_memory=True)
        asz = 4 if w.A_f32 else 8
        h2d = w.n_trans * (4 + 4 + asz + (8 if broad else 0))
        if not batched:
            bufs = None
            prof0 = pxc.Profile(w.profile, w.cutoff, w.mass_da, w.hwhm, None, None)
            s1, e1 = sigma[0], sexp[0:1]

            def step_e2e(bufs):
                sig, e, bufs = pxc.pxc_cross_section_streamed(ws, states, h_up, h_lo, h_A, h_gr if broad else None,
                                                              h_ne if broad else None, cond_arg, grid, prof0,
                                                              w.threshold, bufs=bufs, sigma=s1, sigma_exp=e1)
                h_sig[0].copy_(sig, non_blocking=True)
                h_exp.copy_(e, non_blocking=True)
                return bufs
        else:
            def step_e2e(bufs):
                for d, h in ((d_up, h_up), (d_lo, h_lo), (d_A, h_A), (d_gr, h_gr), (d_ne, h_ne)):
                    d.copy_(h, non_blocking=True)
                tr, prof = chunk_args(0)
                pxc.pxc_cross_section(ws, states, tr, cond_arg, grid, prof, w.threshold, sigma=sigma,
                                      sigma_exp=sexp)
                h_sig.copy_(sigma, non_blocking=True)
                h_exp.copy_(sexp, non_blocking=True)
                return bufs

        bufs = step_e2e(None)
        ws.sync()
        n_e2e = args.steps
        barrier()
        e0, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n_e2e):
            bufs = step_e2e(bufs)
        e1_.record(stream)
        barrier()
        ms_e = slowest_rank_ms(e0.elapsed_time(e1_), world, dev)
        d2h = n_c * (w.n_grid * 4 + 4)
        e2e = {"value": replica_rate(evals, n_e2e, world, ms_e), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": n_e2e, "ms_per_step": ms_e / n_e2e,
               "lines_per_s": replica_rate(w.n_trans, n_e2e, world, ms_e),
               "h2d_gbs": h2d / (ms_e / n_e2e / 1e3) / 1e9,
               "bound": ("host-to-device copy (PCIe): the copies of step c+1 overlap the kernels of step c"
                         if ms_e / n_e2e > 1.5 * ms_max / args.steps else "kernels")}

    # ---------------------------------------------------------------- rooflines
    peaks, peak_src = _peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_max = float(clk.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2032.0))
    clk_hz = sm_max * 1e6
    per_clk = pipes["per_sm_per_clk"]
    fp32_peak = sms * 128 * 2 * clk_hz / 1e12                 # TFLOP/s: SMs x 128 FMA lanes x 2 x clock
    fp32_meas = sms * per_clk["fma"] * 2 * clk_hz / 1e12      # the same from the measured FMA rate
    mufu_peak = sms * per_clk["rcp"] * clk_hz / 1e9           # G reciprocals/s, measured rate
    prof_ms, prof_n = tm["profile"]
    int_ms, int_n = tm["intensity"]
    sort_ms, sort_n = tm["sort"]
    per_launch_evals = evals / max(prof_n // max(args.steps, 1), 1)
    prof_launch_ms = prof_ms / max(prof_n, 1)
    ach_evals = per_launch_evals / (prof_launch_ms / 1e3)
    ach_tflops = 2 * EVAL_FP32_FMAS * ach_evals / 1e12
    roof_profile = {"bound": "alu", "achieved": ach_tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": ach_tflops / fp32_peak, "traffic": NCU_TRAFFIC.get(
                        ("profile", _src_hash("paper_2609_17273_b300/csrc/kernels_profile.cu"))),
                    "kernel": f"k_profile<{w.profile}>",
                    "peak_source": (f"FP32 pipe: {sms} SMs x 128 FMA lanes x 2 FLOP x {sm_max:.0f} MHz "
                                    f"(measured FMA rate {per_clk['fma']:.1f}/SM/clk: {fp32_meas:.2f} TFLOP/s)"),
                    "algorithmic": f"{EVAL_FP32_FMAS} FP32 FMAs + {EVAL_MUFU} MUFU rcp per line-grid evaluation",
                    "evals_per_s": ach_evals,
                    "mufu": {"achieved_G": ach_evals * EVAL_MUFU / 1e9, "peak_G": mufu_peak,
                             "frac": ach_evals * EVAL_MUFU / 1e9 / mufu_peak,
                             "peak_source": f"measured rcp rate {per_clk['rcp']:.2f}/SM/clk"},
                    "issue": {"frac": ach_evals * (EVAL_FP32_FMAS + EVAL_MUFU) / (sms * 128 * clk_hz),
                              "note": "warp-instruction issue slots of the algorithmic work (one per SMSP per clock)"},
                    "launch_ms": prof_launch_ms, "launches_per_step": prof_n / max(args.steps, 1)}
    # algorithmic bytes of one intensity launch: the line arrays read once (upper, lower, A),
    # (key, index, FP64 I) written per kept line, and the state-code table (12-bit codes, five per
    # 64-bit word) read once
    kept_per_launch = kept / nchunks
    a_bytes = 4 if w.A_f32 else 8
    per_launch_bytes = chunk * (4 + 4 + a_bytes) + kept_per_launch * (8 + 4 + 8) + (w.n_states + 4) // 5 * 8
    int_launch_ms = int_ms / max(int_n, 1)
    ach_hbm = per_launch_bytes / (int_launch_ms / 1e3) / 1e9 if int_n else 0.0
    roof_int = {"bound": "hbm", "achieved": ach_hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach_hbm / peaks["hbm_gbs"], "traffic": NCU_TRAFFIC.get(
                    ("intensity", _src_hash("paper_2609_17273_b300/csrc/kernels_lines.cu"))),
                "kernel": "k_lines_pre + k_lines_exact", "peak_source": f"hbm_gbs of {peak_src} MEASURED_PEAKS.json",
                "bytes_per_line": per_launch_bytes / chunk,
                "sector_bytes_per_line": 4 + 4 + a_bytes + 2 * 32, "launch_ms": int_launch_ms}
    dominant = roof_profile if prof_ms >= int_ms else roof_int

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": w.name, "lines": w.n_trans, "states": w.n_states, "grid": w.n_grid,
                      "chunk": chunk, "conditions": n_c, "profile": w.profile, "T": w.T, "T_vib": w.T_vib,
                      "step": "forward + adjoint" if args.backward else "forward",
                      "P": w.P, "cutoff": w.cutoff, "threshold": w.threshold,
                      "parallelism": f"replicas x{world}",
                      "l2": f"inputs ({w.n_trans * (16 if w.A_f32 else 20) / 1e9:.1f} GB) larger than L2"
                            if w.n_trans * 16 > L2_BYTES else "inputs smaller than L2",
                      "fp64": "nu, Boltzmann factors, Q",
                      "profile_tile": {"tile": tile, "segment_points": pxc.TILE_SEGMENT_POINTS[tile],
                                       "autotune": tune}},
           "lines_per_s": lines_per_s,
           "counts": {"kept_lines": kept, "evals_nonzero": evals, "evals_window": evals_window},
           "pass_ms_per_step": {"intensity": int_ms / args.steps, "sort": sort_ms / args.steps,
                                "profile": prof_ms / args.steps},
           "roofline": dominant, "rooflines": {"profile": roof_profile, "intensity": roof_int},
           "pipe_rates": pipes, "gpu_launches": launches, "clocks": clk, "e2e": e2e, "setup_s": t_gen}

    if rank == 0 and not args.no_extras:
        out["extras"] = run_extras(args, pxc, torch, dev, synth)
    if rank == 0 and not args.no_cpu_baseline:
        threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        n = calibrate_sample(w, states_h, args.ref_step_s)
        ev, nl, dt, r = oracle_sample(w, states_h, n)
        # the GPU on the same sample and condition: its error against the oracle
        wsx = pxc.Workspace(max_states=w.n_states, max_lines=nl, max_grid=w.n_grid, device=dev)
        trx = pxc.Transitions(d_up[:nl], d_lo[:nl], d_A[:nl])
        prx = pxc.Profile(w.profile, w.cutoff, w.mass_da, w.hwhm, d_gr[:nl] if broad else None,
                          d_ne[:nl] if broad else None)
        sx, ex = pxc.pxc_cross_section(wsx, states, trx, _oracle_condition(w), grid, prx, w.threshold)
        wsx.sync()
        got = np.ldexp(sx[0].double().cpu().numpy(), int(ex[0].item()))
        del wsx
        out["cpu_baseline"] = {"value": ev / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": (f"first {nl} of {w.n_trans} transitions, full grid, condition "
                                          f"{_oracle_condition(w)}, {dt:.1f} s"),
                               "cpu": _cpu_model(), "oracle_s": dt,
                               "gpu_error_vs_oracle": sigma_errors(got, r["sigma"])}
        # the same oracle on one thread, on a sample a `threads`-th the size
        import oracle
        oracle.set_threads(1)
        ev1, nl1, dt1, _ = oracle_sample(w, states_h, max(1000, n // max(threads, 1)))
        oracle.set_threads(threads)
        out["cpu_baseline"]["one_thread"] = {"value": ev1 / dt1, "sample": f"first {nl1} transitions, {dt1:.1f} s"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_extras(args, pxc, torch, dev, synth):
    """Batched (T, P) table vs sequential plain calls; forward+backward vs forward; non-LTE
    population models and emission; binned profiles on a coarse grid; the cooling function."""
    import numpy as np
    res = {}
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps=1):
        fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    # batched opacity table
    w = synth.workload("table_1e8")
    if args.extras_lines:
        w = w.scaled(n_trans=args.extras_lines)
    E, g, _ = w.states()
    up, lo, A = w.transitions()
    gr, ne = w.broadening()
    st = pxc.States(torch.from_numpy(E).to(dev), torch.from_numpy(g).to(dev), None)
    tr = pxc.Transitions(torch.from_numpy(up).to(dev), torch.from_numpy(lo).to(dev), torch.from_numpy(A).to(dev))
    prof = pxc.Profile("voigt", w.cutoff, w.mass_da, 0.0, torch.from_numpy(gr).to(dev), torch.from_numpy(ne).to(dev))
    grid = (w.nu_min, w.dnu, w.n_grid)
    conds = [(T, 0.0, P) for T, P in w.conditions]
    nT = len({c[0] for c in conds})
    wsb = pxc.Workspace(max_states=w.n_states, max_lines=w.n_trans, max_grid=w.n_grid, max_conditions=len(conds),
                        max_temperatures=nT, device=dev)
    sig = torch.empty(len(conds), w.n_grid, dtype=torch.float32, device=dev)
    se = torch.empty(len(conds), dtype=torch.int32, device=dev)
    tile_b, tune_b, _, _ = pxc.pxc_autotune(wsb, st, tr, conds, grid, prof, 0.0, repeats=1, sigma=sig, sigma_exp=se)
    ms_b = timed(lambda: pxc.pxc_cross_section(wsb, st, tr, conds, grid, prof, 0.0, sigma=sig, sigma_exp=se))
    sb = wsb.stats()
    # the same table replayed from a captured CUDA graph (the first call captures)
    wsb.set_graphs(True)
    ms_g = timed(lambda: pxc.pxc_cross_section(wsb, st, tr, conds, grid, prof, 0.0, sigma=sig, sigma_exp=se), reps=3)
    gstats = wsb.graph_stats()
    wsb.set_graphs(False)
    del wsb
    wsp = pxc.Workspace(max_states=w.n_states, max_lines=w.n_trans, max_grid=w.n_grid, device=dev)
    s1 = torch.empty(1, w.n_grid, dtype=torch.float32, device=dev)
    e1 = torch.empty(1, dtype=torch.int32, device=dev)
    worst = 0.0

    def seq():
        for c in conds:
            pxc.pxc_cross_section(wsp, st, tr, c, grid, prof, 0.0, sigma=s1, sigma_exp=e1)

    tile_s, _, _, _ = pxc.pxc_autotune(wsp, st, tr, conds[len(conds) // 2], grid, prof, 0.0, repeats=1, sigma=s1,
                                       sigma_exp=e1)
    ms_s = timed(seq)
    for i in (0, len(conds) // 2, len(conds) - 1):
        pxc.pxc_cross_section(wsp, st, tr, conds[i], grid, prof, 0.0, sigma=s1, sigma_exp=e1)
        a = torch.ldexp(sig[i].double(), se[i].double())
        b = torch.ldexp(s1[0].double(), e1[0].double())
        worst = max(worst, float((a - b).abs().max() / b.abs().max().clamp_min(1e-300)))
    res["batched_table"] = {"workload": w.name, "conditions": len(conds), "lines": w.n_trans,
                            "batched_ms": ms_b, "graph_replay_ms": ms_g, "graph": gstats,
                            "sequential_ms": ms_s, "speedup": ms_s / ms_b,
                            "max_abs_diff_rel_peak": worst, "kept_lines": sb["n_kept"],
                            "tile_batched": tile_b, "autotune_batched_ms": tune_b, "tile_sequential": tile_s}
    del wsp, st, tr, prof, sig
    torch.cuda.empty_cache()

    # forward + backward on the two-temperature list
    w = synth.workload("nlte_1e7")
    E, g, Ev = w.states()
    up, lo, A = w.transitions()
    gr, ne = w.broadening()
    st = pxc.States(torch.from_numpy(E).to(dev), torch.from_numpy(g).to(dev), torch.from_numpy(Ev).to(dev))
    tr = pxc.Transitions(torch.from_numpy(up).to(dev), torch.from_numpy(lo).to(dev), torch.from_numpy(A).to(dev))
    prof = pxc.Profile("voigt", w.cutoff, w.mass_da, 0.0, torch.from_numpy(gr).to(dev), torch.from_numpy(ne).to(dev))
    grid = (w.nu_min, w.dnu, w.n_grid)
    cond = (w.T, w.T_vib, w.P)
    wt = torch.from_numpy(w.weights()).to(dev)
    wsf = pxc.Workspace(max_states=w.n_states, max_lines=w.n_trans, max_grid=w.n_grid, device=dev)
    ms_f = timed(lambda: pxc.pxc_cross_section(wsf, st, tr, cond, grid, prof), reps=3)
    wsf.set_reuse_forward(True)  # the adjoint reads back the forward's kept, sorted line list

    def fb():
        pxc.pxc_cross_section(wsf, st, tr, cond, grid, prof)
        pxc.pxc_cross_section_backward(wsf, st, tr, cond, grid, prof, wt)

    ms_fb = timed(fb, reps=3)
    wsf.set_reuse_forward(False)
    ev_f = wsf.stats()["evals_nonzero"]
    ms_bwd = max(ms_fb - ms_f, 1e-6)
    res["fwd_bwd"] = {"workload": w.name, "lines": w.n_trans, "fwd_ms": ms_f, "fwd_bwd_ms": ms_fb,
                      "ratio": ms_fb / ms_f, "evals": ev_f, "fwd_evals_per_s": ev_f / (ms_f / 1e3),
                      "bwd_evals_per_s": ev_f / (ms_bwd / 1e3),
                      "note": "backward = one k_adjoint launch over the forward's kept, sorted lines "
                              "(pxc_set_reuse_forward) and the fixed-order reduction; its evaluations are the "
                              "forward's, each with the W4 value and its z-derivative"}

    # vibronic-density populations on the same list (T_rot = 1200 K), absorption and emission
    nv = torch.from_numpy(w.vib_densities()).to(dev)
    std = pxc.States(st.E, st.g, st.E_vib, nv)
    ms_d = timed(lambda: pxc.pxc_cross_section(wsf, std, tr, (w.T, 0.0, w.P), grid, prof), reps=3)
    wsf.set_emission(True)
    ms_de = timed(lambda: pxc.pxc_cross_section(wsf, std, tr, (w.T, 0.0, w.P), grid, prof), reps=3)
    ms_2e = timed(lambda: pxc.pxc_cross_section(wsf, st, tr, cond, grid, prof), reps=3)
    wsf.set_emission(False)
    res["nlte_models"] = {"workload": w.name, "lines": w.n_trans, "treanor_abs_ms": ms_f,
                          "density_abs_ms": ms_d, "density_em_ms": ms_de, "treanor_em_ms": ms_2e}
    del wsf, st, std, tr, prof
    torch.cuda.empty_cache()

    # binned profiles on the 0.1 cm^-1 grid of doppler_1e5 (1e5 lines, widths far below the bin)
    w = synth.workload("doppler_1e5")
    E, g, _ = w.states()
    up, lo, A = w.transitions()
    gr, ne = w.broadening()
    st = pxc.States(torch.from_numpy(E).to(dev), torch.from_numpy(g).to(dev), None)
    tr = pxc.Transitions(torch.from_numpy(up).to(dev), torch.from_numpy(lo).to(dev), torch.from_numpy(A).to(dev))
    grid = (w.nu_min, w.dnu, w.n_grid)
    wsb = pxc.Workspace(max_states=w.n_states, max_lines=w.n_trans, max_grid=w.n_grid, device=dev)
    binned = {}
    for kind in ("gauss_doppler", "binned_gauss_doppler", "voigt", "binned_voigt"):
        prof = pxc.Profile(kind, w.cutoff, w.mass_da, 0.0, torch.from_numpy(gr).to(dev), torch.from_numpy(ne).to(dev))
        ms_k = timed(lambda: pxc.pxc_cross_section(wsb, st, tr, (w.T, 0.0, 1.0), grid, prof), reps=3)
        ev = wsb.stats()["evals_nonzero"]
        binned[kind] = {"ms": ms_k, "evals": ev, "evals_per_s": ev / (ms_k / 1e3)}
    res["binned_profiles"] = {"workload": w.name, "lines": w.n_trans, "grid_step": w.dnu, **binned}
    del wsb, st, tr
    torch.cuda.empty_cache()

    # cooling function on one 1e8-line chunk of voigt_1e9 (5e7 states), 20 temperatures
    w = synth.workload("voigt_1e9")
    n = min(w.chunk, 100_000_000)
    E, g, _ = w.states()
    st = pxc.States(torch.from_numpy(E).to(dev), torch.from_numpy(g).to(dev), None)
    up = torch.empty(n, dtype=torch.int32); lo = torch.empty(n, dtype=torch.int32)
    A = torch.empty(n, dtype=torch.float32)
    w.transitions(0, n, out=(up.numpy(), lo.numpy(), A.numpy()))
    tr = pxc.Transitions(up.to(dev), lo.to(dev), A.to(dev))
    Ts = [float(t) for t in np.geomspace(100.0, 5000.0, 20)]
    wsc = pxc.Workspace(max_states=w.n_states, max_lines=n, max_grid=1, max_conditions=len(Ts), device=dev)
    ms_c = timed(lambda: pxc.pxc_cooling_function(wsc, st, tr, [(t, 0.0, 1.0) for t in Ts]), reps=3)
    res["cooling_function"] = {"workload": w.name, "lines": n, "states": w.n_states, "temperatures": len(Ts),
                               "ms": ms_c, "lines_per_s": n / (ms_c / 1e3)}
    del wsc, st, tr
    torch.cuda.empty_cache()
    return res


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["pxc", "reference"], default="pxc")
    ap.add_argument("--workload", default="voigt_1e9")
    ap.add_argument("--lines", type=int, default=0, help="override the transition count (smaller runs)")
    ap.add_argument("--extras-lines", type=int, default=0, help="override the batched-table transition count")
    ap.add_argument("--tile", type=int, default=-1, help="profile tile configuration (-1: autotune on chunk 0)")
    ap.add_argument("--backward", action="store_true",
                    help="each step is the forward call and its adjoint (single-condition workloads in one chunk)")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-step-s", type=float, default=10.0, help="seconds of oracle work per reference step")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return main_pxc(args)


if __name__ == "__main__":
    sys.exit(main())
