"""Benchmark: amplitude updates/s of the fused state-vector path on GB300.

Workload (default, --workload random32): 60 layers of seeded U3 on every
qubit plus CX on a random disjoint pairing (2880 gates) applied to |0...0>
on n=32 qubits, complex64 (32 GiB state), then 100 shots and <Z_i> for all
qubits.  One step = state init, plan + fused apply (cost-model planner),
probability block sums, block CDF scan, sampling and <Z>: every stage of the
hot path.  The state is larger than L2 (129 MB), so no flush is needed
between steps.  --workload qft28 runs QFT n=28 (420 gates) on a seeded basis
state instead.

value      = whole-job amplitude updates/s (gates * 2^n per step per GPU),
             device-timed with CUDA events on the library's stream.
e2e        = the same metric through the C ABI with host buffers: gate list
             from host memory in, samples and <Z> copied back every step.
roofline   = the tile-pass kernel: algorithmic bytes per launch (one read and
             one write of the state, 16 B per amplitude) / mean launch time
             from CUDA events recorded by the library around each pass.
greedy     = the same step with the greedy fixed-k planner (the cost model's
             fallback and judge).
plain      = the same step with one kernel per gate (no fusion).
check      = after the timed steps: QFT, sampled amplitudes against the closed
             form; random circuits, the circuit then its inverse from |0>,
             which must give <Z_i> = 1 for every qubit.
cpu_baseline = the FP64 oracle on the host cores over a bounded prefix of
             the same gate list at the same n (rank 0, N=1 only), all cores
             and one thread, extrapolated to the step by gate count.

--impl reference runs the oracle as the reference arm (host cores).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "amplitude updates/s and % HBM roofline, learned-fused vs plain, F≥1-1e-6"
UNIT = "amp_updates/s"


# DRAM traffic of the tile pass per amplitude per launch, from the ncu capture
# summarised in profiles/ (the bench's random U3+CX family at n=26 complex64,
# the 85 passes of one step on the run-time compiled kernels;
# dram__bytes_read.sum + dram__bytes_write.sum), valid only for the kernel,
# compiler and planner sources it was taken with (SHA-256 over the files
# below); a changed kernel reports traffic null until it is captured again.
TRAFFIC_SOURCES = ["paper_2504_03967_gb300/csrc/sv_apply.cu", "paper_2504_03967_gb300/csrc/sv_plan.cpp",
                   "paper_2504_03967_gb300/csrc/sv_internal.h", "paper_2504_03967_gb300/csrc/sv_dev.h",
                   "paper_2504_03967_gb300/csrc/sv_rpass.cuh", "paper_2504_03967_gb300/csrc/sv_jit.cpp"]
TRAFFIC = {"sha256": "4bd6035baccc91a93d8298223b5a143c53015278da0dbc1a6127ae6bba04ed82",
           "bytes_per_amp": 15.398,
           "profile": "profiles/traffic_random26_c64_bench.md (the 85 tile passes of one step at n=26, scaled to 2^n)"}


def sources_sha(read=None):
    """SHA-256 over TRAFFIC_SOURCES without their whole-line comments and
    blank lines (a comment edit does not void a capture)."""
    import hashlib

    hsh = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        if read is None:
            with open(os.path.join(ROOT, f), "rb") as fh:
                text = fh.read()
        else:
            text = read(f)
        for line in text.splitlines():
            t = line.strip()
            if t and not t.startswith(b"//"):
                hsh.update(line + b"\n")
    return hsh.hexdigest()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload(name):
    if name == "qft28":
        n = 28
        g = W.qft(n)
        x = W.random_basis_index(n, W.SEED[2])
        return n, g, x, "QFT n=28 (420 gates) on a seeded random basis state"
    if name.startswith("qft"):
        n = int(name[3:])
        return n, W.qft(n), W.random_basis_index(n, W.SEED[2]), "QFT n=%d" % n
    if name.startswith("random"):
        n = int(name[6:])
        g = W.random_u3_cx(n, 60, W.SEED[4])
        return n, g, 0, "random U3+CX n=%d, 60 layers (%d gates) from |0>" % (n, len(g))
    if name.startswith("cxblocks"):
        # cxblocks<n>: the random CX-block circuits of App. D.1 Alg. 1 (Ry, Rz on both qubits, then CX), 60 n blocks
        n = int(name[8:])
        return n, W.random_cx_blocks(n, 60 * n, W.SEED[4]), 0, "random CX blocks n=%d (%d blocks) from |0>" % (n, 60 * n)
    if name.startswith("qcrank"):
        # qcrank<a>x<d>: one QCrank image circuit (2^a addresses, d data qubits)
        a, d = (int(v) for v in name[6:].split("x"))
        pix = np.random.default_rng(W.SEED[3]).uniform(0, 1, size=(1 << a, d))
        return a + d, W.qcrank(a, d, pix), 0, "QCrank a=%d d=%d (n=%d) from |0>" % (a, d, a + d)
    raise SystemExit("unknown workload " + name)


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform

    return platform.processor() or platform.machine()


def cpu_baseline(n, gates, x, budget_s=12.0):
    """FP64 oracle on the host cores over a bounded prefix of the gate list at
    the same n: one thread for the first gate, all cores for the next ones
    (about budget_s), each extrapolated to the whole list by gate count."""
    import oracle

    cores = len(os.sched_getaffinity(0))
    psi = oracle.basis_state(n, x)  # complex128: 16 B per amplitude
    oracle.set_threads(1)
    t0 = time.perf_counter()
    oracle.apply_inplace(n, gates[:1], psi)
    t1 = time.perf_counter() - t0
    oracle.set_threads(cores)
    t0 = time.perf_counter()
    oracle.apply_inplace(n, gates[1:2], psi)
    tg = time.perf_counter() - t0
    G = int(max(1, min(len(gates) - 2, budget_s / max(tg, 1e-3))))
    t0 = time.perf_counter()
    oracle.apply_inplace(n, gates[2:2 + G], psi)
    dt = time.perf_counter() - t0
    del psi
    N = float(1 << n)
    return {"value": G * N / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "sample": "gates 3..%d of the %d-gate list at n=%d, FP64 complex128, %d threads, %.1f s; extrapolated "
                      "to the whole list by gate count" % (G + 2, len(gates), n, cores, dt),
            "single_thread": {"value": N / t1, "unit": UNIT, "cores": 1,
                              "sample": "gate 1 of the list at n=%d, one thread, %.1f s; extrapolated" % (n, t1)}}


def train_cost_model(S, dt, n):
    """Record pass timings of circuits OTHER than the benchmarked one (short
    random U3+CX, QFT and CX-block circuits at n - 4, n - 2 and n qubits) on
    the run-time compiled passes the bench runs (each candidate compiled by a
    first, unrecorded apply), for every tile width, fusion width and
    tensor-core choice the planners propose, and train the cost model on them
    (GPU kernels)."""
    import torch

    cands = [(k, m, t) for k in (4, 5) for m in (12, 13, 14) for t in ((-1, 1) if dt == S.C64 else (-1,))]
    circuits = [W.random_u3_cx(n - 4, 6, 2001), W.qft(n - 4), W.random_cx_blocks(n - 4, 60, 2002),
                W.random_u3_cx(n - 2, 4, 2003), W.random_u3_cx(n, 2, 2004)]
    feats, times = [], []
    for g in circuits:
        nq = int(max(int(r["q"][:int(r["nq"])].max()) for r in g)) + 1
        hh = S.sv_alloc(nq, dt)
        try:
            for k, m, t in cands:
                for rec in (0, 1):  # the first apply compiles the passes
                    S.sv_init_basis(hh, 0)
                    S.sv_apply_circuit(hh, g, k_max=k, tile_m=m, tensor=t, record=rec, jit=1)
                ms, f = S.sv_pass_times(hh, features=True)
                feats.append(f)
                times.append(ms)
        finally:
            torch.cuda.synchronize()
            S.sv_free(hh)
    F, T = np.concatenate(feats), np.concatenate(times)
    loss = S.sv_cost_model_train(F, T, epochs=3000, lr=3e-3, seed=7)
    return {"train_samples": int(len(T)), "train_loss": loss, "training_circuits": "random U3+CX, QFT and CX-block "
            "circuits at %d, %d and %d qubits (not the benchmarked circuit), compiled passes" % (n - 4, n - 2, n)}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores (rank 0 only), each
    step a bounded slice of the same gate list at the same n."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    n, g, x, desc = workload(args.workload)
    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    psi = oracle.basis_state(n, x)
    per = max(1, args.ref_gates)
    for s in range(args.warmup):
        oracle.apply_inplace(n, g[:per], psi)
    times = []
    for s in range(args.steps):
        lo = (s * per) % len(g)
        t0 = time.perf_counter()
        oracle.apply_inplace(n, g[lo:lo + per], psi)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    val = per * float(1 << n) / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": desc, "n": n, "gates_per_step": per, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                             "sample": "%d gates of the list per step at n=%d, FP64" % (per, n)},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(x, dist, device):
    """The slowest rank's value (every rank gets it); x itself without a
    process group.  Replicas: each rank runs the whole workload on its GPU, so
    the job's time is the slowest rank's and its value is
    world_size * work / that time (weak scaling)."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, units_per_rank, ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / (ms / 1e3)


def _event_ms(torch, stream, fn, reps):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(reps):
        fn(i)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def report_approx(args):
    """QFT n (default 28) complex64 with P/RZ/CP gates below eps dropped:
    1 - F against the closed form QFT|x> = N^-1/2 sum_y e^{2 pi i x y / N}|y>
    over the full state (on the device, in chunks), the bound
    (sum of dropped |lambda| / 2)^2, and the fused apply time."""
    import torch

    import paper_2504_03967_gb300 as S

    n = int(args.workload[3:]) if args.workload.startswith("qft") else 28
    g = W.qft(n)
    x = W.random_basis_index(n, W.SEED[2])
    N = 1 << n
    stream = torch.cuda.current_stream()
    state = torch.empty(2 << n, dtype=torch.float32, device="cuda")
    h = S.sv_attach(n, S.C64, state.data_ptr(), stream.cuda_stream)
    lam = np.array([abs(np.remainder(r["p"][0] + np.pi, 2 * np.pi) - np.pi) for r in g if r["type"] == W.CP])
    rows = []
    for eps in [0.0, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 3e-2, 1e-1]:
        def run(i):
            S.sv_init_basis(h, x)
            S.sv_apply_circuit(h, g, relabel=1, drop_phase_below=eps)
        for i in range(3):
            run(i)
        ms = _event_ms(torch, stream, run, 5)
        run(0)
        S.sv_materialize(h)  # logical order, to compare index by index
        st = state.view(torch.complex64)
        ov = torch.zeros((), dtype=torch.complex128, device="cuda")
        nrm = torch.zeros((), dtype=torch.float64, device="cuda")
        C = 1 << 24
        for off in range(0, N, C):
            y = torch.arange(off, min(N, off + C), dtype=torch.int64, device="cuda")
            ph = ((x * y) % N).to(torch.float64) * (2.0 * np.pi / N)
            ref = torch.polar(torch.full_like(ph, N ** -0.5), ph)
            got = st[off:off + len(y)].to(torch.complex128)
            ov += (ref.conj() * got).sum()
            nrm += (got.abs() ** 2).sum()
        F = float(abs(ov.item()) ** 2 / nrm.item())
        dropped = lam[lam < eps] if eps > 0 else lam[:0]
        kept = S.sv_plan_circuit(n, S.C64, g[g["type"] != W.SWAP], drop_phase_below=eps)["gates"]
        rows.append({"eps": eps, "gates_dropped": int(len(dropped)), "gates_applied": int(kept),
                     "one_minus_F": max(0.0, 1.0 - F), "bound": float((dropped.sum() / 2) ** 2),
                     "ms_per_apply": ms})
    S.sv_free(h)
    print(json.dumps({"report": "approximate QFT (drop P/RZ/CP below eps)", "n": n, "dtype": "c64",
                      "reference": "closed form, full state", "rows": rows}), flush=True)


def report_batch(args):
    """Circuits/s end to end through sv_batch_run (host gate lists in,
    planning included, outputs back): the QCrank batch (512 circuits,
    a ~ U{8..14}, d ~ U{4..10}, 10^5 shots each) and the ansatz sweep
    (4096 parameter sets, n = 20, 8 layers, <Z_i>); and the QCrank read-out
    of Table 2's a = 14 row (3000 * 2^14 shots sampled and decoded on the
    device)."""
    import torch

    import paper_2504_03967_gb300 as S

    out = {"report": "batches and QCrank read-out"}
    parts = set(args.parts.split(","))
    if "qcrank" in parts:
        report_qcrank_batch(S, out)
    if "ansatz" in parts:
        report_ansatz(S, out)
    if "readout" in parts:
        report_qcrank_readout(S, out, torch)
    print(json.dumps(out), flush=True)


def report_qcrank_batch(S, out):
    batch = W.qcrank_batch(512, W.SEED[3], a_range=(8, 14))
    circuits = [(a + d, W.qcrank(a, d, pix)) for a, d, pix in batch]
    gates = int(sum(len(gl) for _, gl in circuits))
    S.sv_batch_run(circuits, dtype=S.C64, shots=100000, seed=31)
    t0 = time.perf_counter()
    S.sv_batch_run(circuits, dtype=S.C64, shots=100000, seed=31)
    dt = time.perf_counter() - t0
    out["qcrank_batch"] = {"circuits": 512, "gates": gates, "shots_per_circuit": 100000, "seconds": dt,
                           "circuits_per_s": 512 / dt}
    # the same first 32 circuits with and without multiplexor recognition
    for mux, tag in ((0, "qcrank_first32"), (-1, "qcrank_first32_no_mux")):
        t0 = time.perf_counter()
        S.sv_batch_run(circuits[:32], dtype=S.C64, shots=100000, seed=31, mux=mux)
        dt = time.perf_counter() - t0
        out[tag] = {"circuits": 32, "seconds": dt, "circuits_per_s": 32 / dt}


def report_ansatz(S, out):
    params = W.hea_params(4096, 20, 8, W.SEED[5])
    hc = [(20, W.hea(20, 8, params[s])) for s in range(4096)]
    S.sv_batch_run(hc[:256], dtype=S.C64, shots=0)
    t0 = time.perf_counter()
    S.sv_batch_run(hc, dtype=S.C64, shots=0)
    dt = time.perf_counter() - t0
    out["ansatz_sweep"] = {"circuits": 4096, "n": 20, "seconds": dt, "circuits_per_s": 4096 / dt}


def report_qcrank_readout(S, out, torch):
    a, d = 14, 6
    pix = np.random.default_rng(5).uniform(0, 1, size=(1 << a, d))
    h = S.sv_alloc(a + d, S.C64)
    S.sv_init_basis(h, 0)
    S.sv_apply_circuit(h, W.qcrank(a, d, pix))
    shots = 3000 << a
    S.sv_qcrank_reconstruct(h, a, d, shots, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rec, counts = S.sv_qcrank_reconstruct(h, a, d, shots, 2)
    dt = time.perf_counter() - t0
    S.sv_free(h)
    err = rec - pix
    c = np.corrcoef(rec.ravel(), pix.ravel())[0, 1]
    out["qcrank_readout"] = {"a": a, "d": d, "shots": shots, "seconds": dt, "shots_per_s": shots / dt,
                             "rms_pixel_error": float(np.sqrt(np.mean(err ** 2))),
                             "shot_noise_rms": float(1.0 / (np.pi * np.sqrt(3000))), "correlation": float(c)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="random32")
    ap.add_argument("--dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--planner", default="mlp", choices=["greedy", "mlp", "plain"])
    ap.add_argument("--cm-n", type=int, default=0, help="qubits of the largest cost-model training circuit (0: n)")
    ap.add_argument("--k", type=int, default=0)
    ap.add_argument("--tile-m", type=int, default=0)
    ap.add_argument("--tensor", type=int, default=0, help="1: tensor cores for c64 blocks of 3..5 qubits")
    ap.add_argument("--shots", type=int, default=100)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ref-gates", type=int, default=4)
    ap.add_argument("--no-relabel", action="store_true", help="SWAP gates move amplitudes instead of relabelling")
    ap.add_argument("--no-jit", action="store_true", help="register passes on the interpreting kernel only")
    ap.add_argument("--parts", default="qcrank,ansatz,readout", help="parts of --report batch to run")
    ap.add_argument("--report", default=None, choices=["approx", "batch"],
                    help="secondary measurements instead of the bench line: approx = QFT fidelity loss and time "
                         "against the rotation-dropping threshold; batch = circuits/s of the QCrank and "
                         "ansatz batches and the QCrank read-out")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)
    if args.report == "approx":
        return report_approx(args)
    if args.report == "batch":
        return report_batch(args)

    import torch

    import paper_2504_03967_gb300 as S

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    S.lib()

    n, g, x, desc = workload(args.workload)
    dt = S.C64 if args.dtype == "c64" else S.C128
    amp_b = 8 if dt == S.C64 else 16
    planner = {"greedy": S.PLAN_GREEDY, "mlp": S.PLAN_MLP, "plain": S.PLAN_PLAIN}[args.planner]
    stream = torch.cuda.current_stream()
    state = torch.empty((amp_b // 4) << n, dtype=torch.float32, device="cuda")
    shots_out = torch.empty(max(1, args.shots), dtype=torch.int64, device="cuda")
    ez_out = torch.empty(n, dtype=torch.float64, device="cuda")
    h = S.sv_attach(n, dt, state.data_ptr(), stream.cuda_stream)
    updates = float(len(g)) * float(1 << n)

    relabel = 0 if args.no_relabel else 1
    jit = -1 if args.no_jit else 1

    def step(i, pl, record):
        S.sv_init_basis(h, x)
        S.sv_apply_circuit(h, g, planner=pl, k_max=args.k, tile_m=args.tile_m, record=record, tensor=args.tensor,
                           relabel=relabel, jit=jit)
        S.sv_measure_device(h, args.shots, 1000 + i, shots_out.data_ptr(), ez_out.data_ptr())

    def barrier():
        if dist:
            dist.barrier()

    def timed(pl, steps, warmup, record, tag="timed_steps"):
        for i in range(warmup):
            step(i, pl, 0)
        torch.cuda.synchronize()
        if record:
            S.sv_pass_times(h)  # clear
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = S.sv_launch_count()
        f0 = S.sv_jit_stats()["filled"]
        torch.cuda.nvtx.range_push(tag)  # lets a profiler select the timed launches
        e0.record(stream)
        for i in range(steps):
            step(i, pl, record)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        launches = S.sv_launch_count() - l0
        timed.fills = S.sv_jit_stats()["filled"] - f0
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1) / steps, dist, "cuda")
        return ms, launches

    cm = None
    if planner == S.PLAN_MLP:
        t0 = time.perf_counter()
        cm = train_cost_model(S, dt, args.cm_n or n)
        cm["seconds"] = time.perf_counter() - t0
        # the judge's timed calls (each of its four trials twice: the model's
        # per-pass plan, its two best option sets, greedy), untimed here; the
        # ninth call plans with the trial the judge kept
        for i in range(9):
            step(i, planner, 0)
        torch.cuda.synchronize()
        cm["chosen"] = S.sv_last_plan(h)
        # trial 0: the model's per-pass plan; then its best option sets; last: greedy
        cm["trials"] = S.sv_cost_model_last_trials()
    with Clocks(local) as clk:
        ms, launches = timed(planner, args.steps, args.warmup, 1)
    fills = timed.fills  # first passes that built their tiles from the deferred basis state
    pass_ms = S.sv_pass_times(h)
    # the gate list the planner sees: with relabelling, SWAPs are not executed
    g_planned = g[g["type"] != W.SWAP] if relabel else g
    if cm is not None:
        cm["judge"] = S.sv_cost_model_stats()
        po = cm["chosen"]
        plan = S.sv_plan_circuit(n, dt, g_planned, k_max=po["k_max"], tile_m=po["tile_m"], tensor=po["tensor"],
                                 pass_kernel=po["pass_kernel"])
        plan_opts = {"k_max": po["k_max"], "tile_m": po["tile_m"], "tensor": po["tensor"],
                     "pass_kernel": po["pass_kernel"], "source": "cost model + judge"}
    else:
        plan = S.sv_plan_circuit(n, dt, g_planned, k_max=args.k, tile_m=args.tile_m, tensor=args.tensor,
                                 planner=S.PLAN_PLAIN if planner == S.PLAN_PLAIN else S.PLAN_GREEDY)
        plan_opts = {"k_max": args.k or 5, "tile_m": args.tile_m or "default", "tensor": args.tensor,
                     "source": args.planner}
    plan_opts.update({"dense_ops": plan["dense_ops"], "gate_ops": plan["gate_ops"], "diag_ops": plan["diag_ops"],
                      "register_passes": plan["reg_passes"], "remaps": plan["remaps"]})
    value = job_value(world, updates, ms)
    hbm, src = peaks()
    # dominant kernel: the tile pass (one read + one write of 2^n amplitudes)
    roof = None
    if len(pass_ms):
        # one read and one write of the state per pass, except a first pass
        # that builds its tiles from the deferred basis state (write only)
        per_launch_bytes = amp_b * float(1 << n) * (2.0 * len(pass_ms) - fills) / len(pass_ms)
        achieved = per_launch_bytes / (float(np.mean(pass_ms)) / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": "tile pass (sv_jit_pass compiled per pass structure; k_rpass / k_pass "
                "interpreting kernels)",
                "achieved": achieved, "peak": hbm,
                "unit": "GB/s", "frac": achieved / hbm, "peak_source": src,
                "frac_of_8tbs_nominal": achieved / 8000.0,
                "traffic": (TRAFFIC["bytes_per_amp"] * float(1 << n)
                            if TRAFFIC["bytes_per_amp"] and TRAFFIC["sha256"] == sources_sha() and dt == S.C64
                            else None),
                "traffic_source": TRAFFIC["profile"],
                "launches_timed": int(len(pass_ms)), "mean_launch_ms": float(np.mean(pass_ms)),
                "launches_built_from_basis": int(fills),
                "algorithmic_bytes_per_launch": per_launch_bytes,
                "step_frac": float(np.sum(pass_ms)) / args.steps / ms}

    plain = None
    if not args.no_plain and planner != S.PLAN_PLAIN:
        # one kernel per gate: about 25 s per step at n=32, so one timed step there
        pms, _ = timed(S.PLAN_PLAIN, 1 if n >= 30 else max(2, args.steps // 3), 1, 0, "plain_steps")
        plain = {"value": world * updates / (pms / 1e3), "ms_per_step": pms,
                 "fused_over_plain": pms / ms}
    greedy = None
    if planner == S.PLAN_MLP and not args.no_plain:
        gms, _ = timed(S.PLAN_GREEDY, max(3, args.steps // 2), 2, 0, "greedy_steps")
        greedy = {"value": world * updates / (gms / 1e3), "ms_per_step": gms, "k_max": 5,
                  "learned_over_greedy": gms / ms}

    e2e = None
    if not args.no_e2e:
        h2 = S.sv_alloc(n, dt)
        gh = np.ascontiguousarray(g)
        for i in range(2):
            S.sv_init_basis(h2, x)
            S.sv_apply_circuit(h2, gh, planner=planner, k_max=args.k, tile_m=args.tile_m, tensor=args.tensor,
                               relabel=relabel, jit=jit)
            S.sv_measure(h2, args.shots, i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        K = max(3, args.steps // 2)
        for i in range(K):
            S.sv_init_basis(h2, x)
            S.sv_apply_circuit(h2, gh, planner=planner, k_max=args.k, tile_m=args.tile_m, tensor=args.tensor,
                               relabel=relabel, jit=jit)
            S.sv_measure(h2, args.shots, 1000 + i)  # shots and <Z> from one read, to host memory
        e2e_ms = 1e3 * (time.perf_counter() - t0) / K
        S.sv_free(h2)
        e2e = {"value": world * updates / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": int(gh.nbytes + 8), "d2h_bytes_per_step": int(8 * args.shots + 8 * n)}

    # correctness after the timed steps.  QFT of a basis state: sampled
    # amplitudes against the closed form.  Random circuits: the circuit and
    # then its inverse from |x> give back |x>, so every <Z_i> = 1 - 2 x_i.
    fid = None
    if args.workload.startswith("qft"):
        st = state.view(torch.complex64 if dt == S.C64 else torch.complex128)
        S.sv_init_basis(h, x)
        S.sv_apply_circuit(h, g, planner=planner, k_max=args.k, tile_m=args.tile_m, tensor=args.tensor,
                           relabel=relabel, jit=jit)
        torch.cuda.synchronize()
        rng = np.random.default_rng(0)
        ys = rng.integers(0, 1 << n, size=1 << 16)
        qmap = S.sv_qubit_map(h)  # logical qubit q sits at bit qmap[q] of the stored index
        phys = np.zeros_like(ys)
        for q in range(n):
            phys |= ((ys >> q) & 1) << qmap[q]
        got = st[torch.from_numpy(phys).cuda()].cpu().numpy().astype(np.complex128)
        N = 1 << n
        ref = np.exp(2j * np.pi * ((x * ys) % N) / N) / np.sqrt(N)
        fid = {"sampled_amplitudes": int(len(ys)), "max_abs_err": float(np.abs(got - ref).max()),
               "max_rel_err": float(np.abs(got - ref).max() * np.sqrt(N))}
    else:
        S.sv_init_basis(h, x)
        S.sv_apply_circuit(h, g, planner=planner, k_max=args.k, tile_m=args.tile_m, tensor=args.tensor,
                           relabel=relabel, jit=jit)
        S.sv_apply_circuit(h, W.inverse(g), planner=S.PLAN_GREEDY, relabel=relabel, jit=jit)
        ez = S.sv_expect_z(h)
        want = np.array([1.0 - 2.0 * ((x >> q) & 1) for q in range(n)])
        err = float(np.abs(ez - want).max())
        nrm = S.sv_norm(h)
        qmap = S.sv_qubit_map(h)
        xp = sum(((x >> q) & 1) << qmap[q] for q in range(n))
        a = complex(state.view(torch.complex64 if dt == S.C64 else torch.complex128)[xp].item())
        one_minus_F = 1.0 - abs(a) ** 2 / nrm  # F = |<x|psi>|^2 / <psi|psi> against the exact |x>
        fid = {"test": "circuit then its inverse from |x>: <Z_i> = 1 - 2 x_i for all i, F = |<x|psi>|^2",
               "max_abs_err_expz": err, "norm": nrm, "one_minus_F": one_minus_F,
               "ok": bool(err < 1e-4 and one_minus_F <= 1e-6)}
    S.sv_free(h)

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu:
        cpu = cpu_baseline(n, g, x)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": desc, "n": n, "gates": len(g), "shots": args.shots, "planner": args.planner,
                       "passes": plan["passes"], "plan_options": plan_opts,
                       "parallelism": "replicas" if world > 1 else "single",
                       "swap_gates": "qubit relabelling (read-outs honour the map)" if relabel else "data movement",
                       "register_passes": "compiled at run time per pass structure (NVRTC)" if jit > 0
                       else "interpreting kernel", "jit": S.sv_jit_stats(),
                       "l2": "inputs larger than L2 (state %d MiB)" % ((amp_b << n) >> 20)},
            "roofline": roof, "plain": plain, "greedy": greedy, "cost_model": cm, "e2e": e2e, "cpu_baseline": cpu,
            "gpu_launches": int(launches), "clocks": clk.summary(), "check": fid}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
