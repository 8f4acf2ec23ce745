"""Benchmark: ChFSI eigenproblems/s at residual <= 1e-10 on a correlated sequence of dense
complex Hermitian generalized eigenproblems (n = 2000, 20 SCF steps, nev = 200, nex = 40,
degree 20; S fixed, each solve seeded with the previous Ritz block).

One benchmark step = one whole sequence (20 eigenproblems: Cholesky of S once, then per
problem the transform, Lanczos and Algorithm 1 to convergence, back-transform).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed] [--impl ours|reference]

Prints one JSON line.  For N > 1 (torchrun) every rank solves its own sequence (replicas,
no collective on the data path); the value is all ranks' eigenproblems over the slowest
rank's time.  --impl reference times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ChFSI eigenproblems/s at resid<=1e-10"
UNIT = "eigenproblems/s"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, max clock, throttle reasons)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# the sources a kernel's DRAM traffic depends on
KERNEL_SOURCES = {
    "ozaki_kernel": ["ozaki.cu", "ozaki.cuh", "zgemm.cuh", "common.cuh"],
    "tc_filter_step_kernel": ["filter_tc.cu", "filter_tc.cuh", "common.cuh"],
}


def kernel_source_hash(kernel: str):
    """Hash of the kernel's sources with comments and blank space removed (a comment edit
    does not change the kernel)."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1305_5120_gb300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(csrc, f), "r") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        text = re.sub(r"\s+", " ", text)
        h.update(f.encode() + text.encode())
    return h.hexdigest()[:16]


def traffic_for(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, when it was taken
    on the kernel's current sources (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        e = t["kernels"][kernel]
        if e.get("source_hash") != kernel_source_hash(kernel):
            return None
        return e["bytes_per_launch"]
    except Exception:
        return None


# the solve's stages in chfsi_info.ms_stage order
STAGES = ["reduce", "lanczos", "filter", "qr", "rayleigh_ritz", "residual_lock", "back_transform", "total"]


def make_inputs(w, seed):
    from paper_1305_5120_gb300 import synth
    seq = list(synth.sequence(w.n, w.n_low, w.high, w.steps, seed))
    S = seq[0][1].S
    Hs = [p.H for _, p in seq]
    X0 = synth.start_block(w.n, w.nev + w.nex, seed)
    return Hs, S, X0


# ----------------------------------------------------------------------------------------
def oracle_sample(w, seed=0):
    """Bounded CPU sample of the workload with the FP64 oracle as it stands: Cholesky of S,
    then for problem 1 the reduction to standard form, Lanczos and ONE outer iteration of
    Algorithm 1 (degree-m filter of the whole block, QR, Rayleigh-Ritz, residuals).
    Rate = problems / (t_chol + problems * (t_reduce + t_lanczos + t_iteration)): an upper
    bound on the oracle's rate, since every problem needs at least one outer iteration."""
    from oracle import chfsi as O2
    from oracle import direct as O1
    from paper_1305_5120_gb300 import synth
    gen = synth.sequence(w.n, w.n_low, w.high, 2, seed)
    _, p0 = next(gen)
    _, p1 = next(gen)
    k = w.nev + w.nex
    t = time.perf_counter()
    L = O1.cholesky(p0.S)
    t_chol = time.perf_counter() - t
    t = time.perf_counter()
    Hs = O1.reduce_to_standard(p1.H, L)
    t_red = time.perf_counter() - t
    t = time.perf_counter()
    v0 = O2.splitmix_complex_block(seed, w.n, 1, stream=0)[:, 0]
    al, be = O2.lanczos(Hs, v0, 20)
    b, a, a0 = O2.lanczos_bounds(al, be, w.n, k)
    t_lz = time.perf_counter() - t
    Y0 = synth.start_block(w.n, k, seed)
    t = time.perf_counter()
    Y = O2.chebyshev_filter(Hs, Y0, w.degree, a, b, a0)
    Q = O2.orthonormalize(None, Y)
    lam, Yr, Z = O2.rayleigh_ritz(Hs, Q)
    O2.residual_norms(Z, Yr, lam)
    t_it = time.perf_counter() - t
    P = w.steps
    rate = P / (t_chol + P * (t_red + t_lz + t_it))
    return rate, {"t_cholesky_s": t_chol, "t_reduce_s": t_red, "t_lanczos_s": t_lz, "t_iteration_s": t_it}


def run_reference(args):
    rank, world, _ = dist_env()
    from paper_1305_5120_gb300 import synth
    w = synth.SEQ_N2000
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_sample(w)
    rates, parts = [], None
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r, parts = oracle_sample(w)
        rates.append(r)
    wall = time.perf_counter() - t0
    value = float(np.mean(rates))
    cores = os.cpu_count()
    sample = ("oracle O2 (numpy/C, FP64): Cholesky + reduction + Lanczos + one outer iteration on problem 1 "
              f"of the n={w.n} sequence; rate = 20/(t_chol + 20*(t_red+t_lz+t_iter)), an upper bound")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(w, "fp64"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "parts": parts},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def aggregate_replicas(ms_local: float, problems_local: int, device: str):
    """Whole-job throughput of independent replicas: every rank's solved problems over the
    slowest rank's device time (max over ranks); no collective touches the data path."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    p = torch.tensor([float(problems_local)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(p, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    problems = int(round(p.item()))
    return ms, problems, problems / (ms / 1000.0)


def kernel_rooflines(infos, n, fp64_peak):
    """Achieved rate of each kernel family over the timed region (device time from CUDA
    events the library records on its own stream around the launches) against its peak.
    The roofline object describes the hot path -- the Chebyshev filter's tensor-core step
    kernel -- and names the kernel family with the most device time."""
    pk, pk_kind = peaks()
    bf16 = pk["bf16_tflops_sustained"]
    f_low = sum(i.ms_filter_lowp for _, i in infos)
    f_all = sum(i.ms_stage[2] for _, i in infos)
    cs_all = sum(i.filter_col_steps for _, i in infos)
    cs_low = sum(i.filter_col_steps_lowp for _, i in infos)
    f_steps_ms = sum(i.ms_filter_steps for _, i in infos)
    f_steps_cols = sum(i.filter_step_cols for _, i in infos)
    g_ms = sum(i.ms_gemm_tc for _, i in infos)
    g_flop = sum(i.gemm_tc_flop for _, i in infos)
    e_ms = sum(i.ms_eig for _, i in infos)
    e_flop = sum(i.eig_flop for _, i in infos)
    c_ms = sum(i.ms_chol for _, i in infos)
    c_flop = sum(i.chol_flop for _, i in infos)
    per_col = 8.0 * n * n          # one column through one recurrence step (complex n x n times n)
    fp64_note = "measured DFMA peak of this GPU (chfsi_fp64_peak: eight FMA chains per thread, all SMs)"
    k = {}
    if f_all - f_low > 0 and cs_all > cs_low:
        a = per_col * (cs_all - cs_low) / ((f_all - f_low) / 1e3) / 1e12
        k["zgemm_kernel"] = {"role": "FP64 filter step (DFMA)", "bound": "alu", "achieved": a, "peak": fp64_peak,
                             "unit": "TFLOP/s", "frac": a / fp64_peak, "ms": f_all - f_low, "peak_note": fp64_note}
    if f_steps_ms > 0:
        a = 6.0 * per_col * f_steps_cols / (f_steps_ms / 1e3) / 1e12
        k["tc_filter_step_kernel"] = {"role": "Chebyshev filter step, split-BF16 (hot path)", "bound": "tensor",
                                      "achieved": a, "peak": bf16, "unit": "TFLOP/s", "frac": a / bf16,
                                      "ms": f_steps_ms, "column_steps": int(f_steps_cols),
                                      "algorithmic_tflops": a / 6.0, "filter_stage_ms": f_low,
                                      "peak_note": f"{pk_kind} bf16 sustained; 6 executed slice products "
                                                   "(48 n^2 flops per column-step)"}
    if g_ms > 0:
        a = 78.0 * g_flop / (g_ms / 1e3) / 1e12
        k["ozaki_kernel"] = {"role": "FP64-accurate GEMM (12-digit BF16 expansion)", "bound": "tensor",
                             "achieved": a, "peak": bf16, "unit": "TFLOP/s", "frac": a / bf16, "ms": g_ms,
                             "fp64_equivalent_tflops": a / 78.0,
                             "peak_note": f"{pk_kind} bf16 sustained; 78 executed digit products"}
    if e_ms > 0:
        a = e_flop / (e_ms / 1e3) / 1e12
        k["reduced_eigensolver"] = {
            "role": "Rayleigh-Ritz eigenproblem: FP32 one-sided Jacobi (os_jacobi_kernel, one cluster) + FP64 "
                    "refinement on the tensor cores; FP64 Jacobi (jacobi_fast_kernel) as fallback",
            "bound": "latency", "ms": e_ms,
            "calls_refined": int(sum(i.eig_refined for _, i in infos)),
            "refine_iterations": int(sum(i.eig_refine_iters for _, i in infos)),
            "f32_sweeps": int(sum(i.eig_f32_sweeps for _, i in infos)),
            "fallbacks": int(sum(i.eig_fallbacks for _, i in infos)),
            "fp64_jacobi": {"sweeps": int(sum(i.eig_sweeps for _, i in infos)),
                            "rounds": int(sum(i.eig_rounds for _, i in infos)),
                            "achieved_tflops_over_eig_span": a, "peak": fp64_peak,
                            "work_note": "28 k^2 flops per rotating round", "peak_note": fp64_note}}
    if c_ms > 0:
        a = c_flop / (c_ms / 1e3) / 1e12
        k["cholesky_of_S"] = {"role": "Cholesky of S and its inverse: blocked, 128-wide FP64 diagonal blocks "
                                      "(chol_inv_kernel) and FP64-accurate tensor-core panels and updates",
                              "bound": "mixed", "ms": c_ms, "fp64_equivalent_tflops": a,
                              "dfma_peak": fp64_peak, "over_dfma_peak": a / fp64_peak,
                              "work_note": "(8/3) n^3 flops per factorisation and inverse; above the DFMA peak "
                                           "because most of it runs on the tensor cores"}
    roof = None
    hot = "tc_filter_step_kernel" if "tc_filter_step_kernel" in k else ("zgemm_kernel" if "zgemm_kernel" in k else None)
    if hot:
        roof = {x: v for x, v in k[hot].items() if x in ("bound", "achieved", "peak", "unit", "frac")}
        roof["kernel"] = hot
        roof["dominant_by_time"] = max(k, key=lambda name: k[name]["ms"])
        roof["traffic"] = traffic_for(hot) if hot in KERNEL_SOURCES else None
    return k, roof


def kernel_case(args):
    """A few launches of one kernel on the benchmark's shapes (n = 2000, block 240), for
    profiling: --kernel-case filter (3 tensor-core filter steps), ozaki (one FP64-accurate
    GEMM n x 240 x n), zgemm (the same GEMM on the FP64 pipe), eig (the reduced eigenproblem
    of a Rayleigh-Ritz step, k = 240), sequence (the first
    --case-problems problems of the n = 2000 sequence, mixed path: a launch list of the
    whole solve)."""
    import torch
    from paper_1305_5120_gb300 import chfsi, synth
    if args.kernel_case == "sequence":
        w = synth.SEQ_N2000
        Hs, S, X0 = make_inputs(w, w.seed)
        ctx = chfsi.Context(device=0, precision=chfsi.CHFSI_PREC_MIXED)
        evals = torch.empty(w.nev, dtype=torch.float64, device="cuda")
        X = torch.empty((w.nev, w.n), dtype=torch.complex128, device="cuda")
        sts = []
        for l in range(args.case_problems):
            Hd = chfsi.colmajor(Hs[l])
            if l == 0:
                st, *_ = ctx.solve(Hd, chfsi.colmajor(S), w.n, w.nev, w.nex, chfsi.colmajor(X0), w.tol, w.degree,
                                   evals, X)
            else:
                st, *_ = ctx.next_in_sequence(Hd, None, evals, X)
            sts.append(int(st))
        torch.cuda.synchronize()
        ctx.close()
        print(json.dumps({"kernel_case": "sequence", "problems": args.case_problems, "status": sts,
                          "launches": chfsi.kernel_launches()}))
        return 0 if all(st == 0 for st in sts) else 1
    n, k = args.n, args.k
    ctx = chfsi.Context(device=0)
    rng = synth.rng_for(5, n)
    H = synth.hermitian_part(synth.complex_gaussian(rng, (n, n)))
    Hd = chfsi.colmajor(H)
    Y = chfsi.colmajor(synth.complex_gaussian(rng, (n, k)))
    torch.cuda.synchronize()
    if args.kernel_case == "filter":
        ctx.filter(n, k, Hd, Y, 3, 2.0, 80.0, -1.0, chfsi.CHFSI_PREC_MIXED)
    elif args.kernel_case == "eig":
        # the reduced eigenproblem of a Rayleigh-Ritz step: k x k Hermitian with the benchmark's
        # spectrum shape (200 wanted eigenvalues in [-1, 0], the rest in [0.5, 80]), dense
        # eigenvectors; solved twice by the mixed-precision path (FP32 sweeps + FP64 refinement)
        lam = synth.prescribed_spectrum(k, min(k - 1, 200), 80.0, 5)
        q = synth.haar_unitary(k, synth.rng_for(5, 7))
        G = chfsi.colmajor(synth.hermitian_part((q * lam[None, :]) @ q.conj().T))
        ev = torch.empty(k, dtype=torch.float64, device="cuda")
        W = torch.empty((k, k), dtype=torch.complex128, device="cuda")
        ctx.close()
        ctx = chfsi.Context(device=0, precision=chfsi.CHFSI_PREC_MIXED)
        for _ in range(2):
            ctx.reduced_eig(k, G, ev, W)
        torch.cuda.synchronize()
        err = float(np.abs(ev.cpu().numpy() - lam).max())
        ctx.close()
        print(json.dumps({"kernel_case": "eig", "k": k, "max_eigenvalue_error": err,
                          "launches": chfsi.kernel_launches()}))
        return 0 if err < 1e-12 * 80 else 1
    else:
        prec = chfsi.CHFSI_PREC_MIXED if args.kernel_case == "ozaki" else chfsi.CHFSI_PREC_FP64
        C = torch.empty_like(Y)
        ctx.gemm("N", "N", n, k, n, 1.0, Hd, n, Y, n, 0.0, C, n, prec)
    torch.cuda.synchronize()
    ctx.close()
    print(json.dumps({"kernel_case": args.kernel_case, "n": n, "k": k, "launches": chfsi.kernel_launches()}))
    return 0


def run_kpoints(args):
    """Batched k-points: 64 independent problems, n ~ U[1500, 4000], nev ~ U[5 %, 15 %] n,
    nex = 0.2 nev, spectra as the single-problem workload (nev values in [-1, 0], the rest in
    [0.5, 50]), per-problem seeds 0..63, cold starts.  All arrive at once; the serving loop
    runs them over --slots concurrent contexts (streams).  Every result is checked against
    the prescribed spectrum and by its residuals on the device."""
    import torch
    from paper_1305_5120_gb300 import chfsi, serve, synth
    rng = np.random.default_rng(0)
    probs = []
    for i in range(args.kpoints):
        n = int(rng.integers(1500, 4001))
        nev = max(4, int(round(n * rng.uniform(0.05, 0.15))))
        nex = max(2, int(round(0.2 * nev)))
        H, S, lam = synth.prescribed_pencil_device(n, nev, 50.0, seed=i)
        probs.append((n, nev, nex, H, S, lam))
    torch.cuda.synchronize()

    def requests():
        out = []
        for i, (n, nev, nex, H, S, lam) in enumerate(probs):
            out.append(serve.SequenceRequest(seq_id=i, arrival=0.0, n=n, nev=nev, nex=nex, steps=1,
                                             make_step=lambda l, H=H, S=S: (H, S), degree=20))
        return out

    lines = {}
    for slots in sorted({1, args.slots}):
        srv = serve.Server(device=0, slots=slots, keep_vectors=False, check_inertia=args.check_inertia,
                           precision=chfsi.CHFSI_PREC_MIXED if args.precision == "mixed" else chfsi.CHFSI_PREC_FP64)
        srv.run(requests()[: min(4, len(probs))], realtime=False)          # warm-up
        recs = srv.run(requests(), realtime=False)
        summ = serve.latency_summary(recs)
        bad, fails = 0, []
        for r in recs:
            n, nev, nex, H, S, lam = probs[r.seq_id]
            err = float(np.abs(r.evals - lam[:nev].cpu().numpy()).max())
            if r.status != 0 or err > 1e-10 * max(1.0, float(lam[:nev].abs().max())):
                bad += 1
                fails.append({"id": r.seq_id, "status": r.status, "n": n, "nev": nev, "err": err,
                              "iterations": r.info["iterations"], "locked": r.info["locked"]})
        lines[slots] = dict(summ, wrong=bad, failures=fails[:8],
                            iterations=int(sum(r.info["iterations"] for r in recs)),
                            eig_ms=float(sum(r.info["ms_eig"] for r in recs)),
                            completeness={str(v): int(sum(1 for r in recs if r.info["completeness"] == v))
                                          for v in sorted({r.info["completeness"] for r in recs})},
                            pairs_under_floor=int(sum(r.info["n_floor"] for r in recs)))
    best = lines[max(lines)]
    line = {"metric": METRIC, "value": best["eigenproblems_per_s"], "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x6+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": f"{args.kpoints} k-points, n ~ U[1500,4000], nev 5-15% n, nex 0.2 nev, cold start",
                       "precision": args.precision, "slots": args.slots},
            "by_slots": lines}
    print(json.dumps(line), flush=True)
    return 0 if all(v["wrong"] == 0 and v["failed"] == 0 for v in lines.values()) else 1


def run_batch(args):
    """Batched k-points (chfsi_solve_batch): the same 64 problems as --workload kpoints (n ~
    U[1500, 4000], nev ~ U[5 %, 15 %] n, nex = 0.2 nev, spectra as the single-problem
    workload, per-problem seeds 0..63, cold starts), solved as one batch: every problem's
    filter of an iteration is one grouped tensor-core launch per recurrence step.  One warm-up
    batch of the first four problems, then the timed batch (CUDA events on the context's
    stream); every result checked against its prescribed spectrum, its completeness (inertia
    count at the gap) and its status."""
    import torch
    from paper_1305_5120_gb300 import chfsi, synth
    rng = np.random.default_rng(0)
    probs = []
    for i in range(args.kpoints):
        n = int(rng.integers(1500, 4001))
        nev = max(4, int(round(n * rng.uniform(0.05, 0.15))))
        nex = max(2, int(round(0.2 * nev)))
        H, S, lam = synth.prescribed_pencil_device(n, nev, 50.0, seed=i)
        probs.append((n, nev, nex, chfsi.colmajor(H), chfsi.colmajor(S), lam[:nev].cpu().numpy()))
        del H, S
    torch.cuda.synchronize()
    prec = chfsi.CHFSI_PREC_MIXED if args.precision == "mixed" else chfsi.CHFSI_PREC_FP64
    ctx = chfsi.Context(device=0, precision=prec, check_inertia=args.check_inertia)

    def solve(ps):
        return ctx.solve_batch([p[3] for p in ps], [p[4] for p in ps], [p[0] for p in ps], [p[1] for p in ps],
                               [p[2] for p in ps], 1e-10, 20)

    solve(probs[:4])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = chfsi.kernel_launches()
    t0 = time.perf_counter()
    e0.record(ctx.stream)
    st, sts, evals, Xs, infos = solve(probs)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = e0.elapsed_time(e1)
    wrong = []
    for q, (n, nev, nex, Hd, Sd, lam) in enumerate(probs):
        err = float(np.abs(evals[q].cpu().numpy() - lam).max())
        if sts[q] != 0 or err > 1e-10 * max(1.0, float(np.abs(lam).max())) or \
                (args.check_inertia and infos[q].completeness != 2):
            wrong.append({"id": q, "status": int(sts[q]), "n": n, "nev": nev, "err": err,
                          "completeness": int(infos[q].completeness)})
    line = {"metric": METRIC, "value": len(probs) / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x6+f64" if prec == chfsi.CHFSI_PREC_MIXED else "f64", "data": "synthetic",
            "config": {"workload": f"batch of {len(probs)} k-points, n ~ U[1500,4000], nev 5-15% n, nex 0.2 nev, "
                                   "cold start, chfsi_solve_batch", "precision": args.precision,
                       "check_inertia": args.check_inertia},
            "wall_s": wall, "wrong": len(wrong), "failures": wrong[:8], "gpu_launches": chfsi.kernel_launches() - launches0,
            "iterations": int(sum(i.iterations for i in infos)),
            "pairs_under_floor": int(sum(i.n_floor for i in infos)),
            "eig": {"ms": float(sum(i.ms_eig for i in infos)), "refined": int(sum(i.eig_refined for i in infos)),
                    "fallbacks": int(sum(i.eig_fallbacks for i in infos))},
            "filter_steps_ms": float(sum(i.ms_filter_steps for i in infos)),
            "chol_ms": float(sum(i.ms_chol for i in infos))}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0 if not wrong else 1


def run_large(args):
    """The large sequence (n = 13000, nev = 1300, nex = 260, degree chosen per vector in
    [10, 25], mixed precision, 8 steps of the perturbation law H_{l+1} = H_l + 1e-2 0.7^l E_l,
    S fixed), generated on the device.  Per step: device time, outer iterations, the
    completeness check (inertia count at the gap), the largest generalized residual (floored
    as the lock test guarantees) and S-orthonormality; at step 0 the error of every
    eigenvalue against the prescribed spectrum; at later steps the Weyl bound
    |lam_l - lam_{l-1}| <= eps_{l-1} ||S^{-1}||_2 (||S^{-1}||_2 = 5.5 for cond(S) = 10)."""
    import torch
    from paper_1305_5120_gb300 import chfsi, synth
    w = synth.SEQ_N13000
    steps = args.large_steps
    H, S, lam = synth.prescribed_pencil_device(w.n, w.n_low, w.high, w.seed)
    Sd = S.T.contiguous()
    ctx = chfsi.Context(device=0, precision=chfsi.CHFSI_PREC_MIXED, per_vector_degree=1, degree_min=10,
                        degree_max=25, check_inertia=1)
    evals = torch.empty(w.nev, dtype=torch.float64, device="cuda")
    X = torch.empty((w.nev, w.n), dtype=torch.complex128, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows, prev, tot_ms = [], None, 0.0
    for l in range(steps):
        if l > 0:
            H = H + (1e-2 * 0.7 ** (l - 1)) * synth.perturbation_device(w.n, w.seed, l - 1)
        Hd = H.T.contiguous()
        torch.cuda.synchronize()
        e0.record(ctx.stream)
        if l == 0:
            st, _, _, info = ctx.solve(Hd, Sd, w.n, w.nev, w.nex, None, w.tol, 0, evals, X)
        else:
            st, _, _, info = ctx.next_in_sequence(Hd, None, evals, X)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        tot_ms += ms
        Xm = X.T
        HX = H @ Xm
        SX = S @ Xm
        a, b, a0 = info.bounds
        hn = max(abs(a0), abs(b))
        num = torch.linalg.vector_norm(HX - SX * evals[None, :], dim=0)
        res = (num / torch.maximum(torch.linalg.vector_norm(HX, dim=0),
                                   1e-4 * hn * torch.linalg.vector_norm(SX, dim=0))).max().item()
        G = Xm.conj().T @ SX
        orth = (G - torch.eye(w.nev, dtype=G.dtype, device=G.device)).abs().max().item()
        row = {"step": l, "status": int(st), "ms": ms, "iterations": int(info.iterations),
               "completeness": int(info.completeness), "max_resid_floored": res, "s_orth": orth,
               "n_floor": int(info.n_floor), "filter_col_steps": int(info.filter_col_steps),
               "eig_refined": int(info.eig_refined), "eig_fallbacks": int(info.eig_fallbacks),
               "ms_eig": float(info.ms_eig), "ms_chol": float(info.ms_chol),
               "stages_ms": dict(zip(STAGES, [float(x) for x in info.ms_stage]))}
        ev = evals.cpu().numpy()
        if l == 0:
            err = np.abs(ev - lam[:w.nev].cpu().numpy())
            if args.large_errors_file:   # every eigenvalue's error, one per line
                np.savetxt(args.large_errors_file, err)
            row["eig_error_vs_prescribed"] = {"max": float(err.max()), "median": float(np.median(err)),
                                              "p99": float(np.percentile(err, 99)),
                                              "worst_index": int(err.argmax())}
        else:
            row["weyl_max_shift"] = float(np.abs(ev - prev).max())
            row["weyl_bound"] = 1e-2 * 0.7 ** (l - 1) * 5.5
        prev = ev
        rows.append(row)
        del HX, SX, G, Xm
    line = {"metric": METRIC, "value": steps / (tot_ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": 0, "ms_per_step": tot_ms / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16x6+f64", "data": "synthetic",
            "config": {"workload": w.name + ", per-vector degree 10..25, check_inertia", "n": w.n, "nev": w.nev,
                       "nex": w.nex, "precision": "mixed"},
            "per_step": rows}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0 if all(r["status"] == 0 for r in rows) else 1


class _ServeSequence:
    """One served sequence: step 0 is a structured pencil with a prescribed spectrum (built in
    O(n^2 log n) on the device), step l > 0 is H_l = H_{l-1} + 1e-2 0.7^(l-1) E_l with S fixed,
    each built when the server asks for it (the next H of an SCF cycle arriving), so that only
    the active sequences hold matrices."""

    def __init__(self, sid, n, nev, nex, steps, seed):
        self.sid, self.n, self.nev, self.nex, self.steps, self.seed = sid, n, nev, nex, steps, seed
        self.H = None
        self.lam = None

    def make_step(self, l):
        from paper_1305_5120_gb300 import synth
        if l == 0:
            self.H, S, self.lam = synth.structured_pencil_device(self.n, self.nev, 80.0, self.seed)
            return self.H, S
        self.H = self.H + (1e-2 * 0.7 ** (l - 1)) * synth.structured_perturbation_device(self.n, self.seed, l - 1)
        H = self.H
        if l == self.steps - 1:
            self.H = None
        return H, None


def _serve_arm(args, plan, prec, rate, label):
    """Serve the sequences of `plan` (sid, n, nev, nex, steps) with Poisson arrivals at `rate`
    sequences/s (seeded), `args.slots` concurrent contexts; every step checked."""
    from paper_1305_5120_gb300 import serve
    rng = np.random.default_rng(11)
    t, reqs, seqs = 0.0, [], {}
    for (sid, n, nev, nex, steps) in plan:
        t += float(rng.exponential(1.0 / rate))
        q = _ServeSequence(sid, n, nev, nex, steps, 500 + sid)
        seqs[sid] = q
        reqs.append(serve.SequenceRequest(seq_id=sid, arrival=t, n=n, nev=nev, nex=nex, steps=steps,
                                          make_step=q.make_step, degree=20))
    srv = serve.Server(device=0, slots=args.slots, keep_vectors=False, precision=prec,
                       check_inertia=args.check_inertia)
    t0 = time.perf_counter()
    recs = srv.run(reqs, realtime=True)
    wall = time.perf_counter() - t0
    summ = serve.latency_summary(recs)
    wrong, failures = 0, []
    for r in recs:
        q = seqs[r.seq_id]
        bad = r.status != 0 or (args.check_inertia and r.info.get("completeness") != 2)
        if not bad and r.step == 0:
            lam = q.lam[:q.nev].cpu().numpy()
            bad = np.abs(r.evals - lam).max() > 1e-10 * max(1.0, float(np.abs(lam).max()))
        if bad:
            wrong += 1
            failures.append({"seq": r.seq_id, "step": r.step, "status": int(r.status), "n": q.n, "nev": q.nev,
                             "iterations": r.info.get("iterations"), "completeness": r.info.get("completeness")})
    expected = sum(p[4] for p in plan)
    return dict(summ, label=label, expected_solves=expected, wrong=wrong, failures=failures, wall_s=wall,
                pairs_under_floor=int(sum(r.info.get("n_floor", 0) for r in recs)),
                iterations=int(sum(r.info.get("iterations", 0) for r in recs)))


def run_serve(args):
    """Serving with continuous batching (the sequence-serving workload): args.serve_sequences
    sequences of args.serve_steps correlated steps, n log-uniform in [2000, args.serve_nmax],
    nev ~ U[3 %, 20 %] n, nex = 0.2 nev, Poisson arrivals at args.serve_rate sequences/s (one
    seeded schedule), step l + 1 issued when step l completes, the Ritz block and bounds kept
    on the device between a sequence's steps, admission by the HBM budget; mixed precision.
    The plain-FP64 arm is too slow for that scale, so both arms also serve the same stated
    subset (args.serve_cmp_sequences sequences of args.serve_cmp_steps steps, n log-uniform in
    [2000, args.serve_cmp_nmax]): their ratio is the mixed/FP64 comparison.  Eigenproblems/s
    over the served span and p50/p99 per-solve latency (ready -> done, building that step's
    matrices included); every result checked (status, inertia count, step 0 against its
    prescribed spectrum)."""
    from paper_1305_5120_gb300 import chfsi
    rng = np.random.default_rng(7)

    def plan(count, steps, nmax):
        out = []
        for sid in range(count):
            n = int(round(np.exp(rng.uniform(np.log(2000), np.log(nmax)))))
            nev = max(4, int(round(n * rng.uniform(0.03, 0.20))))
            out.append((sid, n, nev, max(2, int(round(0.2 * nev))), steps))
        return out

    full = plan(args.serve_sequences, args.serve_steps, args.serve_nmax)
    sub = plan(args.serve_cmp_sequences, args.serve_cmp_steps, args.serve_cmp_nmax)
    scale = _serve_arm(args, full, chfsi.CHFSI_PREC_MIXED, args.serve_rate, "mixed, full scale")
    cmp_rate = args.serve_cmp_rate
    cmp = {"mixed": _serve_arm(args, sub, chfsi.CHFSI_PREC_MIXED, cmp_rate, "mixed, comparison subset"),
           "fp64": _serve_arm(args, sub, chfsi.CHFSI_PREC_FP64, cmp_rate, "fp64, comparison subset")}
    line = {"metric": METRIC, "value": scale["eigenproblems_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.serve_steps, "warmup": 0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16x6+f64", "data": "synthetic (structured FFT-built pencils)",
            "config": {"workload": f"serving: {args.serve_sequences} sequences x {args.serve_steps} steps, n log-U"
                                   f"[2000,{args.serve_nmax}], nev 3-20% n, nex 0.2 nev, Poisson "
                                   f"{args.serve_rate}/s, {args.slots} slots, check_inertia {args.check_inertia}",
                       "n_range_served": [min(p[1] for p in full), max(p[1] for p in full)],
                       "comparison_subset": f"{args.serve_cmp_sequences} sequences x {args.serve_cmp_steps} steps, "
                                            f"n log-U[2000,{args.serve_cmp_nmax}], Poisson {cmp_rate}/s, both arms"},
            "full_scale": scale, "comparison": cmp,
            "mixed_over_fp64": (cmp["mixed"]["eigenproblems_per_s"] / cmp["fp64"]["eigenproblems_per_s"]
                                if cmp["fp64"]["eigenproblems_per_s"] else None)}
    print(json.dumps(line), flush=True)
    ok = all(a["wrong"] == 0 and a["solves"] == a["expected_solves"] for a in [scale] + list(cmp.values()))
    return 0 if ok else 1


def config_dict(w, precision):
    return {"workload": w.name, "n": w.n, "nev": w.nev, "nex": w.nex, "problems_per_step": w.steps,
            "degree": w.degree, "tol": w.tol, "precision": precision, "seed": w.seed,
            "l2": "inputs larger than L2: 20 distinct H (1.3 GB) resident, each read by its own solve",
            "parallelism": "replicas (one sequence per GPU, no collectives)"}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1305_5120_gb300 import chfsi, synth

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    w = synth.SEQ_N2000
    prec = chfsi.CHFSI_PREC_MIXED if args.precision == "mixed" else chfsi.CHFSI_PREC_FP64
    seed = w.seed + rank
    Hs, S, X0 = make_inputs(w, seed)
    n, nev, nex, k = w.n, w.nev, w.nex, w.nev + w.nex
    dev = [chfsi.colmajor(H) for H in Hs]
    S_d = chfsi.colmajor(S)
    X0_d = chfsi.colmajor(X0)
    evals = torch.empty(nev, dtype=torch.float64, device="cuda")
    X = torch.empty((nev, n), dtype=torch.complex128, device="cuda")
    ctx = chfsi.Context(device=local, precision=prec)
    stream = ctx.stream

    def one_sequence(Hlist, Sd, infos):
        st, *_ , info = ctx.solve(Hlist[0], Sd, n, nev, nex, X0_d, w.tol, w.degree, evals, X)
        infos.append((st, info))
        for l in range(1, len(Hlist)):
            st, *_ , info = ctx.next_in_sequence(Hlist[l], None, evals, X)
            infos.append((st, info))

    for _ in range(args.warmup):
        one_sequence(dev, S_d, [])
    torch.cuda.synchronize()
    fp64_peak = chfsi.fp64_peak(local)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = chfsi.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    infos = []
    e0.record(stream)
    for _ in range(args.steps):
        one_sequence(dev, S_d, infos)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = chfsi.kernel_launches() - launches0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    bad = [st for st, _ in infos if st != 0]
    # accuracy of the last problem, checked in FP64 on the host
    lam = evals.cpu().numpy()
    Xh = chfsi.to_numpy(X)
    HX = Hs[-1] @ Xh
    resid = float((np.linalg.norm(HX - (S @ Xh) * lam[None, :], axis=0) / np.linalg.norm(HX, axis=0)).max())
    ms, problems, value = aggregate_replicas(ms, args.steps * w.steps, "cuda")

    # per-kernel accounting from the library's stream-ordered CUDA events
    kernels, roof = kernel_rooflines(infos, n, fp64_peak)
    cs_all = sum(i.filter_col_steps for _, i in infos)
    cs_low = sum(i.filter_col_steps_lowp for _, i in infos)
    stages = np.sum([list(i.ms_stage) for _, i in infos], axis=0).tolist()

    # end to end through the public API with host buffers: per problem H2D of H_l (pinned),
    # solve, D2H of eigenvalues and eigenvectors; S uploaded once per sequence.  The upload
    # of H_{l+1} runs on a second stream while problem l is solved (double-buffered device
    # copy, as an SCF code would prefetch its next matrix); every copy lies inside the timed
    # region.
    e2e = None
    if not args.no_e2e:
        Hh = [torch.from_numpy(np.ascontiguousarray(H.T)).pin_memory() for H in Hs]
        Sh = torch.from_numpy(np.ascontiguousarray(S.T)).pin_memory()
        Hd = [torch.empty_like(dev[0]), torch.empty_like(dev[0])]
        Sd2 = torch.empty_like(S_d)
        ev_h = torch.empty(nev, dtype=torch.float64).pin_memory()
        X_h = torch.empty((nev, n), dtype=torch.complex128).pin_memory()
        up = torch.cuda.Stream()
        ev_up = [torch.cuda.Event(), torch.cuda.Event()]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0.record(stream)
        up.wait_event(e0)
        for _ in range(args.steps):
            with torch.cuda.stream(up):
                Hd[0].copy_(Hh[0], non_blocking=True)
                ev_up[0].record(up)
            Sd2.copy_(Sh, non_blocking=True)
            for l in range(w.steps):
                b = l & 1
                if l + 1 < w.steps:   # the other buffer's last reader (problem l - 1) has returned
                    with torch.cuda.stream(up):
                        Hd[1 - b].copy_(Hh[l + 1], non_blocking=True)
                        ev_up[1 - b].record(up)
                stream.wait_event(ev_up[b])
                if l == 0:
                    ctx.solve(Hd[b], Sd2, n, nev, nex, X0_d, w.tol, w.degree, evals, X)
                else:
                    ctx.next_in_sequence(Hd[b], None, evals, X)
                ev_h.copy_(evals, non_blocking=True)
                X_h.copy_(X, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = e0.elapsed_time(e1)
        h2d = (Hh[0].numel() * 16) * w.steps + Sh.numel() * 16
        d2h = (nev * 8 + nev * n * 16) * w.steps
        e2e = {"value": problems / (ms_e2e / 1000.0), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "wall_s": time.perf_counter() - t0,
               "last_problem_evals_match_device_run": float(np.abs(ev_h.numpy() - lam).max()),
               "note": "upload of the next H overlapped with the current solve (second stream)"}

    # the plain-FP64 arm on the same sequence (every product on the DFMA pipe): one sequence
    # after one warm-up problem, CUDA events on the same stream
    fp64 = None
    if not args.no_fp64_path and prec == chfsi.CHFSI_PREC_MIXED:
        ctx64 = chfsi.Context(device=local, precision=chfsi.CHFSI_PREC_FP64)
        ctx64.solve(dev[0], S_d, n, nev, nex, X0_d, w.tol, w.degree, evals, X)
        infos64 = []
        torch.cuda.synchronize()
        e0.record(ctx64.stream)
        st, *_, info = ctx64.solve(dev[0], S_d, n, nev, nex, X0_d, w.tol, w.degree, evals, X)
        infos64.append((st, info))
        for l in range(1, w.steps):
            st, *_, info = ctx64.next_in_sequence(dev[l], None, evals, X)
            infos64.append((st, info))
        e1.record(ctx64.stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        k64, _ = kernel_rooflines(infos64, n, fp64_peak)
        v64 = w.steps / (ms64 / 1000.0)
        lam64 = evals.cpu().numpy()
        fp64 = {"value": v64, "unit": UNIT, "ms_per_sequence": ms64, "problems": w.steps,
                "failed_solves": int(sum(1 for st, _ in infos64 if st != 0)),
                "iterations": int(sum(i.iterations for _, i in infos64)),
                "filter_kernel": k64.get("zgemm_kernel"), "mixed_over_fp64": None,
                "last_problem_evals_match_mixed": None}
        ctx64.close()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, parts = oracle_sample(w)
        cpu = {"value": r, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": "Cholesky + reduction + Lanczos + one outer iteration of problem 1 (FP64 oracle, "
                         "numpy BLAS threads = all cores); rate = 20/(t_chol + 20*(t_red+t_lz+t_iter)), "
                         "an upper bound", "parts": parts}
        # how loose the bound is: the same rate at the outer-iteration count per problem this
        # run's solves took (the oracle runs the same algorithm)
        its = sum(i.iterations for _, i in infos) / max(1, len(infos))
        pt = parts
        cpu["estimate_at_measured_iterations"] = {
            "iterations_per_problem": its,
            "value": w.steps / (pt["t_cholesky_s"] + w.steps * (pt["t_reduce_s"] + pt["t_lanczos_s"] +
                                                                 its * pt["t_iteration_s"]))}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if prec == chfsi.CHFSI_PREC_FP64 else "bf16x6+f64",
                "data": "synthetic", "config": config_dict(w, args.precision), "roofline": roof,
                "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
                "stages_ms": dict(zip(STAGES, stages)),
                "iterations": int(sum(i.iterations for _, i in infos)), "failed_solves": len(bad),
                "eig_sweeps": int(sum(i.eig_sweeps for _, i in infos)),
                "last_problem_max_resid": resid,
                "pairs_under_residual_floor": int(sum(i.n_floor for _, i in infos)),
                "filter_col_steps": int(cs_all), "filter_col_steps_lowp": int(cs_low),
                "fp64_peak_tflops": fp64_peak, "fp64_path": fp64}
        if fp64:
            fp64["mixed_over_fp64"] = value / fp64["value"]
            fp64["last_problem_evals_match_mixed"] = float(np.abs(lam64 - lam).max())
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0 if not bad else 1


# ----------------------------------------------------------------------------------------
# Sequence-correlation study (the analogue of the paper's seeding experiment, Section 4 / Fig. 1b:
# solving each problem of a sequence from the previous problem's Ritz vectors instead of a
# random block), plus the angles between consecutive eigenvector subspaces (Section 2.2).
def s_angles(X, Y, S):
    """Angles between matched columns of X and Y in the S-inner product (radians)."""
    SX, SY = S @ X, S @ Y
    num = np.abs(np.sum(X.conj() * SY, axis=0))
    den = np.sqrt(np.real(np.sum(X.conj() * SX, axis=0)) * np.real(np.sum(Y.conj() * SY, axis=0)))
    return np.arccos(np.clip(num / den, 0.0, 1.0))


def s_principal_angles(X, Y, S):
    """Principal angles between span(X) and span(Y) in the S-inner product (radians,
    ascending): orthonormalise L^H X and L^H Y (S = L L^H) and take arccos of the singular
    values of their cross product."""
    L = np.linalg.cholesky(S)
    qx, _ = np.linalg.qr(L.conj().T @ X)
    qy, _ = np.linalg.qr(L.conj().T @ Y)
    sv = np.linalg.svd(qx.conj().T @ qy, compute_uv=False)
    return np.sort(np.arccos(np.clip(sv, 0.0, 1.0)))


def run_seeding(args):
    """The n = 2000 sequence (20 problems) solved twice by the GPU path: (seeded) each problem
    from the previous one's Ritz block and filter bounds (chfsi_next_in_sequence), (random)
    each problem from the same random block (chfsi_solve).  Per problem: outer iterations,
    filter column steps, device time (CUDA events on the solver stream), and the angles
    between this problem's eigenvectors and the previous one's.  A second pair of runs lets S
    vary along the sequence (S_l = S + 1e-2 0.7^l E_S, E_S Hermitian with ||E_S||_2 = 1; the
    seeded run carries the block over as L_l^H L_{l-1}^{-H} Y)."""
    import torch
    from paper_1305_5120_gb300 import chfsi, synth
    torch.cuda.set_device(0)
    w = synth.SEQ_N2000
    prec = chfsi.CHFSI_PREC_MIXED if args.precision == "mixed" else chfsi.CHFSI_PREC_FP64
    Hs, S, X0 = make_inputs(w, w.seed)
    n, nev, nex = w.n, w.nev, w.nex
    ES = synth.hermitian_part(synth.complex_gaussian(synth.rng_for(w.seed, 77), (n, n)))
    ES /= np.abs(np.linalg.eigvalsh(ES)).max()
    S_var = [S + 1e-2 * 0.7 ** l * ES for l in range(len(Hs))]
    Hd = [chfsi.colmajor(H) for H in Hs]
    X0_d = chfsi.colmajor(X0)
    ctx = chfsi.Context(device=0, precision=prec)
    evals = torch.empty(nev, dtype=torch.float64, device="cuda")
    X = torch.empty((nev, n), dtype=torch.complex128, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def run(seeded, Slist):
        Sd = [chfsi.colmajor(Sm) for Sm in Slist]
        rows, Xs = [], []
        for l in range(len(Hd)):
            torch.cuda.synchronize()
            e0.record(ctx.stream)
            if l == 0 or not seeded:
                st, _, _, info = ctx.solve(Hd[l], Sd[l], n, nev, nex, X0_d, w.tol, w.degree, evals, X)
            else:
                st, _, _, info = ctx.next_in_sequence(Hd[l], Sd[l] if Slist is not S_fixed else None, evals, X)
            e1.record(ctx.stream)
            torch.cuda.synchronize()
            Xh = chfsi.to_numpy(X)
            lam = evals.cpu().numpy()
            HX = Hs[l] @ Xh
            res = float((np.linalg.norm(HX - (Slist[l] @ Xh) * lam[None, :], axis=0) / np.linalg.norm(HX, axis=0)).max())
            rows.append({"status": int(st), "iterations": int(info.iterations), "ms": e0.elapsed_time(e1),
                         "ms_reduce": float(info.ms_stage[0]), "filter_col_steps": int(info.filter_col_steps),
                         "max_resid": res})
            Xs.append(Xh)
        return rows, Xs

    S_fixed = [S] * len(Hs)
    run(True, S_fixed)   # warm-up (allocations, first-use costs)
    out = {"workload": "seeding study: sequence n=2000 x20 nev=200 nex=40 m=20", "precision": args.precision}
    for name, Slist in (("S_fixed", S_fixed), ("S_varying", S_var)):
        seeded, Xs = run(True, Slist)
        rnd, _ = run(False, Slist)
        ang = []
        for l in range(1, len(Xs)):
            a = s_angles(Xs[l - 1], Xs[l], Slist[l])
            pa = s_principal_angles(Xs[l - 1], Xs[l], Slist[l])
            ang.append({"median_vector_angle": float(np.median(a)), "max_vector_angle": float(a.max()),
                        "max_principal_angle": float(pa[-1])})
        sp_ms = [r["ms"] / s_["ms"] for r, s_ in zip(rnd[1:], seeded[1:])]
        # without the reduction to standard form (the random solves also factor S again)
        sp_it = [(r["ms"] - r["ms_reduce"]) / (s_["ms"] - s_["ms_reduce"]) for r, s_ in zip(rnd[1:], seeded[1:])]
        sp_cs = [r["filter_col_steps"] / s_["filter_col_steps"] for r, s_ in zip(rnd[1:], seeded[1:])]
        out[name] = {"seeded": seeded, "random": rnd, "angles": ang,
                     "speedup_time_median": float(np.median(sp_ms)), "speedup_time_last5": float(np.median(sp_ms[-5:])),
                     "speedup_iteration_time_median": float(np.median(sp_it)),
                     "speedup_filter_steps_median": float(np.median(sp_cs)),
                     "all_converged": all(r["status"] == 0 and r["max_resid"] <= 1e-10 for r in seeded + rnd)}
    ctx.close()
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--kernel-case", choices=["filter", "ozaki", "zgemm", "sequence", "eig"], default=None)
    ap.add_argument("--case-problems", type=int, default=3, help="problems of the sequence kernel case")
    ap.add_argument("--workload", choices=["sequence", "kpoints", "batch", "large", "serve", "seeding"],
                    default="sequence")
    ap.add_argument("--large-steps", type=int, default=8)
    ap.add_argument("--large-errors-file", default=None,
                    help="write step 0's error of every eigenvalue against the prescribed spectrum here")
    ap.add_argument("--serve-sequences", type=int, default=48)
    ap.add_argument("--serve-steps", type=int, default=15)
    ap.add_argument("--serve-nmax", type=int, default=8000)
    ap.add_argument("--serve-rate", type=float, default=0.12, help="sequence arrivals per second")
    ap.add_argument("--serve-cmp-sequences", type=int, default=4)
    ap.add_argument("--serve-cmp-steps", type=int, default=3)
    ap.add_argument("--serve-cmp-nmax", type=int, default=3000)
    ap.add_argument("--serve-cmp-rate", type=float, default=0.5)
    ap.add_argument("--kpoints", type=int, default=64)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--n", type=int, default=2000)
    ap.add_argument("--k", type=int, default=240)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-path", action="store_true", help="skip the plain-FP64 arm of the default run")
    ap.add_argument("--check-inertia", type=int, default=1, choices=[0, 1],
                    help="k-points: count the eigenvalues below the gap after every solve")
    args = ap.parse_args()
    if args.kernel_case:
        return kernel_case(args)
    if args.workload == "kpoints":
        return run_kpoints(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "large":
        return run_large(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "seeding":
        return run_seeding(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
