#!/usr/bin/env python
"""Benchmark of one blocked-linear-method step on GB300 (JSON line on stdout).

Workload (default): 16384 parameters in 64 blocks of 256, K = 20 kept directions per block,
10^6 samples streamed to the library in chunks of 65536, FP32 samples resident in HBM (131 GB,
larger than L2, so no L2 flush is needed between steps), split-BF16 tensor-core contractions
with FP32/FP64 accumulation and FP64 centring and solves.  One step = both sweeps and both
solves (first sweep over all chunks, block solves, second sweep over the same chunks, combined
solve); the handle's sums are reset between steps.

Metric: sample-GFLOP/s = useful FLOP of the step / step time, with the useful FLOP per sample
3 sum_b M_b^2 (first sweep: symmetric S_b plus H_b) + 4 n K + 3 (sum_b K_b)^2 (second sweep:
projections and combined sums).  The plain FP64 GPU path is timed on one chunk of the same
workload (FP64 samples) and scaled to the full sample count.

--impl reference times the FP64 CPU oracle (the reference implementation of the method written
from the paper) on a bounded sample of the same workload on the host cores.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = ("n16384", "n16384u", "batch32", "n2048", "n200")
PRECISIONS = {"bf16x4": "BLM_PREC_BF16X4", "tf32x4": "BLM_PREC_TF32X4", "f64": "BLM_PREC_F64"}


def useful_flop_per_sample(wl):
    offs = wl.block_offsets
    m = [offs[b + 1] - offs[b] for b in range(len(offs) - 1)]
    k = [min(wl.n_keep, mb) for mb in m]
    dc = sum(k)
    pass1 = sum(3 * mb * mb for mb in m)
    pass2 = 4 * wl.n * (dc / len(m)) + 3 * dc * dc
    return pass1 + pass2


def profiled_traffic(name):
    """DRAM bytes per launch recorded from an ncu capture in profiles/<name> (a line
    'traffic_bytes_per_launch: <bytes>'), or None."""
    try:
        for line in open(os.path.join(ROOT, "profiles", name)):
            if line.strip().startswith("traffic_bytes_per_launch:"):
                return float(line.split(":", 1)[1].split()[0])
    except Exception:
        pass
    return None


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """Samples nvidia-smi during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu=0):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
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
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# our implementation
# ------------------------------------------------------------------------------------------------
def job_rate(elapsed_ms, steps, flop_per_rank, world, device="cpu"):
    """Whole-job rate of `world` replicas: the slowest rank's time (all-reduce MAX, then a barrier)
    and every rank's work.  Returns (ms per step, sample-GFLOP/s)."""
    if world > 1:
        import torch
        t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.barrier()
        elapsed_ms = float(t.item())
    ms_step = elapsed_ms / steps
    return ms_step, world * flop_per_rank / (ms_step / 1e3) / 1e9


def run_ours(args, rank, world):
    import torch
    import synth
    from synth import device as sdev
    import paper_1702_01481_gb300 as blm

    torch.cuda.set_device(rank % max(1, torch.cuda.device_count()))
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = synth.workload(args.workload)
    if args.samples:
        wl.n_samples = args.samples
    ns, n, chunk = wl.n_samples, wl.n, wl.chunk
    mixed = args.precision != "f64"
    dt = torch.float32 if mixed else torch.float64
    stream = torch.cuda.current_stream()

    # inputs resident in HBM, generated on the device by the seeded generator
    O = torch.empty((ns, n), dtype=dt, device=dev)
    G = torch.empty((ns, n), dtype=dt, device=dev)
    E = torch.empty((ns,), dtype=dt, device=dev)
    dm = sdev.DeviceModel(wl, dev)
    gen_chunk = 32768
    for s0 in range(0, ns, gen_chunk):
        c = min(gen_chunk, ns - s0)
        sdev.fill(dm, s0, O[s0:s0 + c], G[s0:s0 + c], E[s0:s0 + c], stream.cuda_stream)
    torch.cuda.synchronize()

    prec = getattr(blm, PRECISIONS[args.precision])
    inp = blm.BLM_IN_F32 if mixed else blm.BLM_IN_F64
    step = blm.Step(n, wl.block_offsets, wl.n_keep, precision=prec, input_type=inp,
                    stream=stream.cuda_stream, pass_samples=args.pass_samples)
    dmu = torch.empty(n, dtype=torch.float64, device=dev)

    def one_step():
        step.reset()
        for s0 in range(0, ns, chunk):
            c = min(chunk, ns - s0)
            step.accumulate(O[s0:s0 + c], G[s0:s0 + c], E[s0:s0 + c])
        step.block_solve()
        for s0 in range(0, ns, chunk):
            c = min(chunk, ns - s0)
            step.project(O[s0:s0 + c], G[s0:s0 + c], E[s0:s0 + c])
        return step.combined_solve(dmu)

    for _ in range(args.warmup):
        e_pred = one_step()
    torch.cuda.synchronize()
    if args.graph:
        # per-kernel-class times from one profiled eager step (a captured graph records no
        # events), then the whole step captured once and replayed in the timed region
        blm.blm_profile(step.h, 1)
        one_step()
        prof = blm.blm_profile_read(step.h)
        blm.blm_profile(step.h, 0)
        prof = {k: (v[0] * args.steps, v[1] * args.steps) for k, v in prof.items()}
        blm.blm_graph_capture(step.h, O, G, E, None, ns, chunk, n, dmu)
        blm.blm_graph_launch(step.h)
        e_pred = blm.blm_graph_result(step.h)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    if not args.graph:
        blm.blm_profile(step.h, 1)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(args.steps):
        if args.graph:
            blm.blm_graph_launch(step.h)
            e_pred = blm.blm_graph_result(step.h)
        else:
            e_pred = one_step()
    end.record(stream)
    torch.cuda.synchronize()
    if not args.graph:
        prof = blm.blm_profile_read(step.h)
        blm.blm_profile(step.h, 0)
    clk = clocks.stop()
    elapsed_ms = start.elapsed_time(end)
    flop = useful_flop_per_sample(wl) * ns
    ms_step, value = job_rate(elapsed_ms, args.steps, flop, world, dev)
    res = dict(wl=wl, ms_step=ms_step, value=value, prof=prof, clocks=clk, e_pred=e_pred,
               flop=flop, steps=args.steps)

    # roofline of the dominant kernel (largest summed device time in the step)
    pk = peaks()
    kname, (kms, klaunch) = max(prof.items(), key=lambda kv: kv[1][0])
    res["dominant"] = kname
    roof = None
    offs = wl.block_offsets
    m = [offs[b + 1] - offs[b] for b in range(len(offs) - 1)]
    # tcgen05 MACs per sample of the first sweep: 128 x 256 tiles over [O'_b | X'_b] x O'_b
    tile_macs = sum(((mb + 127) // 128) * 2 * ((mb + 255) // 256) * 256 * 128 for mb in m)
    ms1, l1 = prof.get("contract_tc_pass1", (0.0, 0))
    if l1:
        per_launch_samples = ns * res["steps"] / l1
        # executed products: hi*hi + hi*lo + lo*hi + lo*lo (both splits)
        nprod = 4
        exec_flop = 2 * nprod * tile_macs * per_launch_samples
        t_launch = ms1 / l1 / 1e3
        res["tc_pass1"] = {"ms_per_launch": round(ms1 / l1, 3), "launches": l1,
                           "hbm_gbs_algorithmic": round(2 * per_launch_samples * n * 4 / t_launch / 1e9, 1),
                           "tensor_tflops_executed": round(exec_flop / t_launch / 1e12, 1),
                           "useful_tflops": round(sum(3 * mb * mb for mb in m) * per_launch_samples / t_launch / 1e12, 1)}
    if kname == "contract_tc_pass1" and l1:
        # TF32 runs at the nominal dense ratio 1.1 / 2.25 of the measured BF16 peak
        p = pk.get("bf16_tflops_sustained", 1700.0) * (1.1 / 2.25 if args.precision == "tf32x4" else 1.0)
        ach = res["tc_pass1"]["tensor_tflops_executed"]
        roof = {"bound": "tensor", "achieved": ach, "peak": p, "unit": "TFLOP/s",
                "frac": round(ach / p, 4), "traffic": profiled_traffic("tc_op_kernel_n16384.md"),
                "kernel": "tc_op_kernel (first sweep, prepared %s operands)" % args.precision,
                "per_launch_algorithmic_flop": exec_flop,
                "peak_source": "measured bf16 sustained" if "bf16_tflops_sustained" in pk else "fallback"}
    elif kname == "contract_f64" and klaunch:
        per_launch_bytes = 2 * (ns * res["steps"] / klaunch) * n * O.element_size()
        ach = per_launch_bytes / (kms / klaunch / 1e3) / 1e9
        p = pk.get("hbm_gbs", 6800.0)
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": p, "unit": "GB/s",
                "frac": round(ach / p, 4), "traffic": None, "kernel": kname,
                "per_launch_algorithmic_bytes": per_launch_bytes,
                "peak_source": "measured" if "hbm_gbs" in pk else "fallback"}
    elif kname == "eig_blocks" and klaunch:
        # algorithmic work of the block eigen-solves: 10 d^3 per problem of dimension
        # d = 1 + M_b (the dense generalized eigen-solve's usual count); the solver's own
        # phases execute about 15.7 d^3 (Cholesky d^3/3, two triangular solves 2 d^3,
        # Hessenberg 10/3 d^3, QR ~10 d^3).  Peak: the FP64 FMA rate measured on this GPU
        # (1.7 FMA / cycle / SM) x 2 flop x SMs x max clock
        mb = [offs[b + 1] - offs[b] + 1 for b in range(len(offs) - 1)]
        flop = sum(10.0 * d ** 3 for d in mb)
        ach = flop / (kms / klaunch / 1e3) / 1e12
        peak = 1.7 * 2 * 152 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": round(ach, 4), "peak": round(peak, 3), "unit": "TFLOP/s",
                "frac": round(ach / peak, 4), "traffic": None,
                "kernel": "eig_team_kernel (block solves: FP64 reductions on teams of CTAs, FP32 QR)",
                "per_launch_algorithmic_flop": flop,
                "note": "latency bound (serial QR chase, per-column barriers); peak = measured "
                        "FP64 FMA rate x 2 x 152 SMs x max clock"}
    elif kname in ("operand_prep_pass1", "operand_prep_pass2") and klaunch and mixed:
        # HBM: per sample the pass reads its two FP32 source rows (O, G of n values; p, r of dc
        # in the second sweep) and writes the hi | lo operand rows of the A and B arrays
        # (4 bytes per value for BF16X4, 8 for TF32X4)
        width = n if kname.endswith("1") else sum(wl.n_keep for _ in range(len(offs) - 1))
        opb = 8 if args.precision == "tf32x4" else 4
        per_sample = 2 * width * 4 + 2 * width * opb
        per_launch = per_sample * ns * res["steps"] / klaunch
        ach = per_launch / (kms / klaunch / 1e3) / 1e9
        p = pk.get("hbm_gbs", 6800.0)
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": p, "unit": "GB/s",
                "frac": round(ach / p, 4), "traffic": None,
                "kernel": "prep_direct_kernel (%s)" % kname, "per_launch_algorithmic_bytes": per_launch,
                "peak_source": "measured" if "hbm_gbs" in pk else "fallback"}
    elif klaunch:
        roof = {"bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None, "kernel": kname, "note": "no roofline model for this kernel class"}
    res["roofline"] = roof
    res["gpu_launches"] = int(sum(v[1] for v in prof.values()))

    # the plain FP64 GPU path over the same resident samples (FP32 values widened to FP64 on
    # load), one full step: the denominator of the mixed path's speed-up, and the reference the
    # mixed step states its error against (the FP64 path matches the FP64 oracle to 1e-10)
    if mixed and not args.no_fp64 and rank == 0:
        mixed_blocks = [step.block(b) for b in range(wl.n_blocks)]
        mixed_dmu = dmu.cpu().numpy()
        mixed_Sc, mixed_Hc = step.combined()
        step.close()
        s64 = blm.Step(n, wl.block_offsets, wl.n_keep, precision=blm.BLM_PREC_F64,
                       input_type=blm.BLM_IN_F32, stream=stream.cuda_stream)
        d64 = torch.empty(n, dtype=torch.float64, device=dev)
        blm.blm_profile(s64.h, 1)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for s0 in range(0, ns, chunk):
            c = min(chunk, ns - s0)
            s64.accumulate(O[s0:s0 + c], G[s0:s0 + c], E[s0:s0 + c])
        s64.block_solve()
        for s0 in range(0, ns, chunk):
            c = min(chunk, ns - s0)
            s64.project(O[s0:s0 + c], G[s0:s0 + c], E[s0:s0 + c])
        e64 = s64.combined_solve(d64)
        t1.record(stream)
        torch.cuda.synchronize()
        total = t0.elapsed_time(t1)
        res["fp64_path"] = {"ms_per_step": round(total, 1), "samples": ns,
                            "speedup_mixed_over_fp64": round(total / ms_step, 2),
                            "phases_ms": {k: round(v[0], 1) for k, v in
                                          blm.blm_profile_read(s64.h).items() if v[1]}}
        blocks64 = [s64.block(b) for b in range(wl.n_blocks)]
        Sc64, Hc64 = s64.combined()
        s64.close()
        res["err_vs_fp64"] = error_vs_fp64(wl, mixed_blocks, blocks64, res["e_pred"], e64,
                                           mixed_dmu, d64.cpu().numpy(), mixed_Sc, mixed_Hc,
                                           Sc64, Hc64)
    else:
        step.close()
    if mixed and not args.no_hist and rank == 0:
        # "+hist": the same step with N_O = 3 history directions (seeded unit rows), whose
        # projections and sums (Eq. 9-10) join the first sweep's tensor-core launch
        n_old = 3
        rng = np.random.default_rng(12345)
        D = rng.standard_normal((n_old, n))
        D /= np.linalg.norm(D, axis=1, keepdims=True)
        sh = blm.Step(n, wl.block_offsets, wl.n_keep, n_old=n_old, old_dirs=D, precision=prec,
                      input_type=inp, stream=stream.cuda_stream)

        def hist_step():
            sh.reset()
            for s0 in range(0, ns, chunk):
                c = min(chunk, ns - s0)
                sh.accumulate(O[s0:s0 + c], G[s0:s0 + c], E[s0:s0 + c])
            sh.block_solve()
            for s0 in range(0, ns, chunk):
                c = min(chunk, ns - s0)
                sh.project(O[s0:s0 + c], G[s0:s0 + c], E[s0:s0 + c])
            return sh.combined_solve(dmu)

        hist_step()
        blm.blm_profile(sh.h, 1)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        hist_step()
        t1.record(stream)
        torch.cuda.synchronize()
        ph = blm.blm_profile_read(sh.h)
        res["mixed_hist"] = {"n_old": n_old, "ms_per_step": round(t0.elapsed_time(t1), 1),
                             "history_projection_ms": round(ph["history_terms"][0], 1),
                             "contract_tc_pass1_ms": round(ph["contract_tc_pass1"][0], 1),
                             "eig_blocks_ms": round(ph["eig_blocks"][0], 1)}
        sh.close()
    return res


def _corr_err(A, A_ref, S_ref):
    d = np.sqrt(np.abs(np.diag(S_ref)))
    return float(np.max(np.abs(A - A_ref) / np.outer(d, d)))


def error_vs_fp64(wl, blocks, blocks64, e, e64, dmu, dmu64, Sc, Hc, Sc64, Hc64):
    """Error of the mixed step against the FP64 GPU path on the same samples.  Matrix entries in
    correlation scaling |dA_xy| / sqrt(S_xx S_yy) (H also divided by 1 + |H_00|); the mean
    relative error of the overlap diagonal shows any systematic bias of the accumulation.  The
    combined matrices of the two paths are built on their own B^(b), so their difference also
    carries the difference of the retained directions."""
    em, bias = 0.0, []
    for (S, H, lam, B), (S64, H64, lam64, B64) in zip(blocks, blocks64):
        h0 = 1.0 + abs(H64[0, 0])
        em = max(em, _corr_err(S, S64, S64), _corr_err(H, H64, S64) / h0)
        bias.append(np.mean((np.diag(S)[1:] - np.diag(S64)[1:]) / np.diag(S64)[1:]))
    dd = float(np.linalg.norm(dmu - dmu64) / np.linalg.norm(dmu64))
    ec = max(_corr_err(Sc, Sc64, Sc64), _corr_err(Hc, Hc64, Sc64) / (1.0 + abs(Hc64[0, 0])))
    return {"S_b_H_b": float("%.3g" % em), "S_b_diag_bias": float("%.3g" % np.mean(bias)),
            "e_pred_hartree": float("%.3g" % abs(e - e64)), "dmu_rel": float("%.3g" % dd),
            "S_c_H_c_incl_B_difference": float("%.3g" % ec),
            "targets": {"S_b_H_b": 1e-6, "e_pred_hartree": 1e-8}}


def run_error_scan(args):
    """Error of the mixed step against the FP64 GPU path as the sample count grows: the same
    resident samples (the workload's first N) through both paths, for each N of the scan.  The
    zero-mean error of the hi/lo split falls as 1/sqrt(N); a systematic (accumulation) error
    would not."""
    import torch
    import synth
    from synth import device as sdev
    import paper_1702_01481_gb300 as blm

    dev = torch.device("cuda", torch.cuda.current_device())
    wl = synth.workload(args.workload)
    counts = sorted(int(x) for x in args.error_scan.split(","))
    ns_max, n, chunk = counts[-1], wl.n, wl.chunk
    O = torch.empty((ns_max, n), dtype=torch.float32, device=dev)
    G = torch.empty((ns_max, n), dtype=torch.float32, device=dev)
    E = torch.empty((ns_max,), dtype=torch.float32, device=dev)
    dm = sdev.DeviceModel(wl, dev)
    for s0 in range(0, ns_max, 32768):
        c = min(32768, ns_max - s0)
        sdev.fill(dm, s0, O[s0:s0 + c], G[s0:s0 + c], E[s0:s0 + c])
    torch.cuda.synchronize()

    def step(prec, ns):
        st = blm.Step(n, wl.block_offsets, wl.n_keep, precision=prec, input_type=blm.BLM_IN_F32)
        for s0 in range(0, ns, chunk):
            c = min(chunk, ns - s0)
            st.accumulate(O[s0:s0 + c], G[s0:s0 + c], E[s0:s0 + c])
        st.block_solve()
        blocks = [st.block(b) for b in range(wl.n_blocks)]
        for s0 in range(0, ns, chunk):
            c = min(chunk, ns - s0)
            st.project(O[s0:s0 + c], G[s0:s0 + c], E[s0:s0 + c])
        d = torch.empty(n, dtype=torch.float64, device=dev)
        e = st.combined_solve(d)
        Sc, Hc = st.combined()
        st.close()
        return blocks, e, d.cpu().numpy(), Sc, Hc

    out = []
    for ns in counts:
        bm, em, dmm, Scm, Hcm = step(blm.BLM_PREC_BF16X4, ns)
        b64, e64, d64, Sc64, Hc64 = step(blm.BLM_PREC_F64, ns)
        r = error_vs_fp64(wl, bm, b64, em, e64, dmm, d64, Scm, Hcm, Sc64, Hc64)
        r.pop("targets")
        r["samples"] = ns
        out.append(r)
        print(json.dumps(r), file=sys.stderr)
    return {"workload": args.workload, "scan": out}


def run_batch(args):
    """The batch of 32 independent optimisations: every problem's samples resident in HBM, each
    problem's tiles chosen by the autotuner, one step of all 32 captured as one CUDA graph and
    replayed per timed step."""
    import torch
    import synth
    from synth import device as sdev
    import paper_1702_01481_gb300 as blm

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    wls = synth.batch_workloads(32)
    prec = getattr(blm, PRECISIONS[args.precision])
    data = []
    for wl in wls:
        O = torch.empty((wl.n_samples, wl.n), dtype=torch.float32, device=dev)
        G = torch.empty((wl.n_samples, wl.n), dtype=torch.float32, device=dev)
        E = torch.empty((wl.n_samples,), dtype=torch.float32, device=dev)
        dm = sdev.DeviceModel(wl, dev)
        for s0 in range(0, wl.n_samples, 32768):
            c = min(32768, wl.n_samples - s0)
            sdev.fill(dm, s0, O[s0:s0 + c], G[s0:s0 + c], E[s0:s0 + c], stream.cuda_stream)
        data.append((O, G, E))
    torch.cuda.synchronize()
    pass_samples = 8192
    probs = [blm.make_problem(wl.n, wl.block_offsets, wl.n_keep, precision=prec,
                              input_type=blm.BLM_IN_F32, pass_samples=pass_samples) for wl in wls]
    b = blm.blm_batch_create(probs, stream.cuda_stream)
    hs = [blm.blm_batch_handle(b, i) for i in range(len(wls))]
    choices = [blm.blm_autotune(h, d[0], d[1], d[2], None, min(wl.n_samples, pass_samples), wl.n)
               for h, d, wl in zip(hs, data, wls)]
    # per-kernel-class device times: one profiled eager step of every problem
    prof = {}
    for h, (O, G, E), wl in zip(hs, data, wls):
        blm.blm_profile(h, 1)
        for s0 in range(0, wl.n_samples, wl.chunk):
            blm.blm_accumulate(h, O[s0:s0 + wl.chunk], G[s0:s0 + wl.chunk], E[s0:s0 + wl.chunk], None,
                               min(wl.chunk, wl.n_samples - s0), wl.n)
        blm.blm_block_solve(h)
        for s0 in range(0, wl.n_samples, wl.chunk):
            blm.blm_project(h, O[s0:s0 + wl.chunk], G[s0:s0 + wl.chunk], E[s0:s0 + wl.chunk], None,
                            min(wl.chunk, wl.n_samples - s0), wl.n)
        d = torch.empty(wl.n, dtype=torch.float64, device=dev)
        blm.blm_combined_solve(h, d)
        for k, v in blm.blm_profile_read(h).items():
            a = prof.get(k, (0.0, 0))
            prof[k] = (a[0] + v[0], a[1] + v[1])
        blm.blm_profile(h, 0)
        blm.blm_reset(h)
    dmu = [torch.empty(wl.n, dtype=torch.float64, device=dev) for wl in wls]
    blm.blm_batch_capture(b, [d[0] for d in data], [d[1] for d in data], [d[2] for d in data], None,
                          [wl.n_samples for wl in wls], [wl.n for wl in wls], 65536, dmu)
    for _ in range(args.warmup):
        blm.blm_batch_launch(b)
        e, st, rc = blm.blm_batch_result(b, len(wls))
        if rc != 0:
            raise RuntimeError("batch step failed: statuses %s: %s"
                               % (list(st), blm._lib.blm_batch_last_error(b).decode()))
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(args.steps):
        blm.blm_batch_launch(b)
        e, st, rc = blm.blm_batch_result(b, len(wls))
    end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_step = start.elapsed_time(end) / args.steps
    flop = sum(useful_flop_per_sample(wl) * wl.n_samples for wl in wls)
    kname, (kms, kl) = max(prof.items(), key=lambda kv: kv[1][0])
    pk = peaks()
    roof = None
    if kname == "eig_blocks":
        d = [b1 - b0 + 1 for wl in wls for b0, b1 in zip(wl.block_offsets[:-1], wl.block_offsets[1:])]
        fl = sum(10.0 * x ** 3 for x in d)
        peak = 1.7 * 2 * 152 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        ach = fl / (kms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": round(ach, 4), "peak": round(peak, 3), "unit": "TFLOP/s",
                "frac": round(ach / peak, 4), "traffic": None,
                "kernel": "eig_team_kernel (block solves of all problems in one persistent launch; "
                          "summed over the problems' eager steps)",
                "per_launch_algorithmic_flop": fl}
    else:
        roof = {"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None, "kernel": kname, "note": "no roofline model for this class"}
    blm.blm_batch_destroy(b)
    return dict(ms_step=ms_step, value=flop / (ms_step / 1e3) / 1e9, clocks=clk, roofline=roof,
                prof=prof, e_pred=[float(x) for x in e], choices=choices,
                samples=sum(wl.n_samples for wl in wls),
                gpu_launches=int(sum(v[1] for v in prof.values())), dominant=kname)


def run_e2e(args):
    """Same metric through the C ABI with host (pinned) sample buffers: every step copies its
    samples host -> device inside the timed region and reads back Delta mu and E_pred."""
    import torch
    import synth
    from synth import device as sdev
    import paper_1702_01481_gb300 as blm

    dev = torch.device("cuda", torch.cuda.current_device())
    torch.cuda.empty_cache()           # the resident-sample run's memory goes back to the device
    wl = synth.workload(args.workload)
    ns = min(wl.n_samples, args.e2e_samples)
    n = wl.n
    mixed = args.precision != "f64"
    dt = torch.float32 if mixed else torch.float64
    O = torch.empty((ns, n), dtype=dt, pin_memory=True)
    G = torch.empty((ns, n), dtype=dt, pin_memory=True)
    E = torch.empty((ns,), dtype=dt, pin_memory=True)
    dm = sdev.DeviceModel(wl, dev)
    tmp = 16384
    bo = torch.empty((tmp, n), dtype=dt, device=dev)
    bg = torch.empty((tmp, n), dtype=dt, device=dev)
    be = torch.empty((tmp,), dtype=dt, device=dev)
    for s0 in range(0, ns, tmp):
        c = min(tmp, ns - s0)
        sdev.fill(dm, s0, bo[:c], bg[:c], be[:c])
        O[s0:s0 + c].copy_(bo[:c])
        G[s0:s0 + c].copy_(bg[:c])
        E[s0:s0 + c].copy_(be[:c])
    del bo, bg, be
    torch.cuda.synchronize()
    prec = getattr(blm, PRECISIONS[args.precision])
    inp = blm.BLM_IN_F32 if mixed else blm.BLM_IN_F64
    stream = torch.cuda.current_stream()
    step = blm.Step(n, wl.block_offsets, wl.n_keep, precision=prec, input_type=inp,
                    stream=stream.cuda_stream)
    # the first sweep's device copies serve the second sweep (one host-to-device copy of the
    # samples per step)
    blm.blm_set_host_cache(step.h, ns * (2 * n + 2) * O.element_size() + (64 << 20))
    dmu = torch.empty(n, dtype=torch.float64, pin_memory=True)
    chunk = wl.chunk

    def one_step():
        step.reset()
        for s0 in range(0, ns, chunk):
            c = min(chunk, ns - s0)
            step.accumulate(O[s0:s0 + c], G[s0:s0 + c], E[s0:s0 + c])
        step.block_solve()
        for s0 in range(0, ns, chunk):
            c = min(chunk, ns - s0)
            step.project(O[s0:s0 + c], G[s0:s0 + c], E[s0:s0 + c])
        return step.combined_solve(dmu)

    one_step()
    torch.cuda.synchronize()
    # each step timed on its own (host clock around a synchronised step); the median is reported,
    # since a step of the host-to-device stream can be disturbed by the host
    times = []
    for _ in range(max(1, args.e2e_steps)):
        t = time.perf_counter()
        one_step()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
    sec = sorted(times)[len(times) // 2]
    step.close()
    flop = useful_flop_per_sample(wl) * ns
    h2d = 2 * ns * n * O.element_size() + ns * E.element_size()
    return {"value": round(flop / sec / 1e9, 1), "unit": "sample-GFLOP/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8 * n + 8,
            "samples_per_step": ns, "ms_per_step": round(sec * 1e3, 1),
            "ms_per_step_all": [round(x * 1e3, 1) for x in times]}


def cpu_baseline(args, wl, samples):
    """The FP64 oracle on the host cores on a bounded sample of the same workload."""
    import synth
    from oracle import blm_oracle
    O, G, E = synth.samples(wl, count=samples, dtype=np.float32)
    O, G, E = (a.astype(np.float64) for a in (O, G, E))
    t = time.perf_counter()
    blm_oracle.blm_step(O, G, E, None, wl.block_offsets, wl.n_keep)
    sec = time.perf_counter() - t
    flop = useful_flop_per_sample(wl) * samples
    return {"value": round(flop / sec / 1e9, 3), "unit": "sample-GFLOP/s",
            "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d of %d samples of the same workload (full parameter count), one step, %.1f s"
                      % (samples, wl.n_samples, sec)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="n16384", choices=WORKLOADS)
    ap.add_argument("--precision", default=None, choices=list(PRECISIONS))
    ap.add_argument("--graph", action="store_true",
                    help="time the step as one captured CUDA graph (default for n16384u)")
    ap.add_argument("--samples", type=int, default=0)
    ap.add_argument("--pass-samples", type=int, default=0,
                    help="samples per internal pass (operand scratch size; 0: the library's 65536)")
    ap.add_argument("--cpu-samples", type=int, default=2048)
    ap.add_argument("--e2e-samples", type=int, default=524288,
                    help="samples of the end-to-end step (pinned host memory: 4 (2n + 1) bytes "
                         "per sample, 69 GB at the default on the 16384-parameter workload)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-hist", action="store_true")
    ap.add_argument("--error-scan", default="",
                    help="comma-separated sample counts: print the mixed step's error against "
                         "the FP64 GPU path at each (no timing)")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = {"n16384": "bf16x4", "n16384u": "tf32x4",
                          "batch32": "bf16x4"}.get(args.workload, "f64")
    if args.workload == "n16384u":
        args.graph = True

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    import synth
    if args.workload == "batch32":
        if rank != 0:
            return
        r = run_batch(args)
        line = {"metric": "blocked-LM step: sample-GFLOP/s (useful FLOP of both sweeps / step time)",
                "value": round(r["value"], 1), "unit": "sample-GFLOP/s", "n_gpus": 1,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(r["ms_step"], 2),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "%s/f32-acc/f64-solve" % args.precision,
                "data": "synthetic (seeded generator, on device)",
                "config": {"workload": "batch32: 32 independent optimisations, n 500-8000, N_s "
                                       "5e4-4e5 (%d samples in all), N_B 2-32 (blocks <= 640), "
                                       "K <= 10, split tensor-core sweeps + FP64 solves, "
                                       "autotuned tiles, one captured CUDA graph" % r["samples"],
                           "input": "FP32 samples resident in HBM",
                           "l2": "inputs larger than L2 (no flush needed)",
                           "parallelism": "single GPU"},
                "roofline": r["roofline"], "clocks": r["clocks"], "gpu_launches": r["gpu_launches"],
                "phases_ms_per_step": {k: round(v[0], 2) for k, v in r["prof"].items() if v[1]},
                "dominant_kernel": r["dominant"], "tile_choices": r["choices"],
                "e_pred": r["e_pred"][:4], "e2e": None}
        print(json.dumps(line))
        return
    wl = synth.workload(args.workload)
    if args.samples:
        wl.n_samples = args.samples
    path = {"bf16x4": "split-BF16 tensor-core sweeps + FP64 solves",
            "tf32x4": "split-TF32 tensor-core sweeps + FP64 solves",
            "f64": "FP64 sweeps + FP64 solves"}[args.precision]
    blocks = ("%d blocks" % wl.n_blocks if len(set(np.diff(wl.block_offsets))) == 1 else
              "%d uneven blocks of %d-%d" % (wl.n_blocks, min(np.diff(wl.block_offsets)),
                                            max(np.diff(wl.block_offsets))))
    config = {"workload": "%s: n=%d params, N_B=%s, K=%d, N_s=%d samples in chunks of %d, %s%s"
                          % (args.workload, wl.n, blocks, wl.n_keep, wl.n_samples, wl.chunk, path,
                             ", the whole step one captured CUDA graph" if args.graph else ""),
              "input": ("FP32" if args.precision != "f64" else "FP64") + " samples resident in HBM",
              "l2": "inputs larger than L2 (no flush needed)",
              "parallelism": "replicas" if args.gpus > 1 else "single GPU"}
    metric = "blocked-LM step: sample-GFLOP/s (useful FLOP of both sweeps / step time)"

    if args.impl == "reference":
        if rank != 0:
            return
        steps = []
        samples = max(64, args.cpu_samples // 2)
        for _ in range(args.warmup):
            cpu_baseline(args, wl, 64)
        for _ in range(args.steps):
            steps.append(cpu_baseline(args, wl, samples))
        v = sorted(s["value"] for s in steps)[len(steps) // 2]
        flop = useful_flop_per_sample(wl) * wl.n_samples
        line = {"impl": "reference", "metric": metric, "value": v, "unit": "sample-GFLOP/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(flop / (v * 1e9) * 1e3, 1),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded generator)", "config": config,
                "cpu_baseline": {"value": v, "unit": "sample-GFLOP/s", "cores": os.cpu_count(),
                                 "kind": "oracle", "sample": steps[0]["sample"]},
                "e2e": {"value": v, "unit": "sample-GFLOP/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.error_scan:
        print(json.dumps(run_error_scan(args)))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res = run_ours(args, rank, world)
    if rank != 0:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    line = {"metric": metric, "value": round(res["value"], 1), "unit": "sample-GFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(res["ms_step"], 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"bf16x4": "bf16x4/f32-acc/f64-solve", "tf32x4": "tf32x4/f32-acc/f64-solve",
                      "f64": "f64"}[args.precision],
            "data": "synthetic (seeded generator, on device)", "config": config,
            "e_pred": res["e_pred"], "roofline": res["roofline"], "clocks": res["clocks"],
            "gpu_launches": res["gpu_launches"],
            "phases_ms_per_step": {k: round(v[0] / res["steps"], 2) for k, v in res["prof"].items() if v[1]},
            "dominant_kernel": res["dominant"]}
    if "tc_pass1" in res:
        line["tc_pass1"] = {k: (round(v, 3) if isinstance(v, float) else v) for k, v in res["tc_pass1"].items()}
    if "fp64_path" in res:
        line["fp64_path"] = res["fp64_path"]
    if "err_vs_fp64" in res:
        line["err_vs_fp64"] = res["err_vs_fp64"]
    if "mixed_hist" in res:
        line["mixed_hist"] = res["mixed_hist"]
    if not args.no_e2e and world == 1:
        line["e2e"] = run_e2e(args)
    else:
        line["e2e"] = None
    if not args.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_baseline(args, wl, args.cpu_samples)
    print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
