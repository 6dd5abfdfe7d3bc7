#!/usr/bin/env python
"""TensorNet energy+force benchmark on GB300.

One step = one pass of the whole hot path over the workload: cell-list
neighbor search, TensorNet energy (per system, FP64 reduction) and forces
through the hand-written reverse pass.  The step is captured once in a CUDA
graph and replayed; L2 is flushed (a 256 MB write) before every timed step
and the flush is outside the timed events.

Prints ONE JSON line (rank 0).  Metric: energy+force evaluations/s of the
whole job (replicas across ranks; the workload does not shard).
--impl reference times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TensorNet energy+force evals/s and ns/day vs atoms; % of HBM/tensor roofline"
UNIT = "evals/s"
FS_PER_STEP = 0.5            # MD time step used for the ns/day figure
FP32_LANES_PER_SM = 128      # FP32 FMA lanes per SM (4 partitions x 32)
SM_COUNT = 152
SM_MAX_MHZ = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="water96k",
                    help="molecule32, water3000, batch512, solvated24k or water96k (default: the largest, "
                         "the 96,000-atom periodic water box)")
    ap.add_argument("--precision", default="tf32x3", choices=["fp32", "tf32x3", "bf16"],
                    help="fp32: SIMT FP32 GEMMs; tf32x3: FP32-accurate 3xTF32 tensor-core GEMMs; "
                         "bf16: BF16 tensor-core GEMMs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--recompute-edges", default="auto", choices=["auto", "0", "1"],
                    help="1: recompute the radial-MLP activations in the reverse pass instead of keeping "
                         "them (auto: only when keeping them would take over a quarter of device memory)")
    ap.add_argument("--tuning", default="auto",
                    help="auto: autotune launch shapes on this input (cached); default: the library's "
                         "defaults; or a comma-separated knob list")
    ap.add_argument("--profile-steps", type=int, default=3)
    ap.add_argument("--md", type=int, default=0,
                    help="also time this many velocity-Verlet steps (0.5 fs, 1 A skin, rebuild every 20 steps "
                         "and whenever an atom has moved more than skin/2)")
    ap.add_argument("--sweep", choices=["paper"], default=None,
                    help="paper: single random-walk molecules of the paper's five atom counts, cutoff 4.5 A, "
                         "0/1/2 interaction layers (one JSON line)")
    ap.add_argument("--neighbor-bench", action="store_true",
                    help="neighbor search alone: 32,768-particle random cloud (64 neighbors per particle) split "
                         "into 1..1024 systems (one JSON line)")
    ap.add_argument("--neighbor-stress", action="store_true",
                    help="neighbor search alone on the 1,029,000-atom periodic water box at 5 and 6 A "
                         "(one JSON line)")
    ap.add_argument("--radial-table", type=int, default=0,
                    help="n > 0: tabulate the radial projections and filters at n distances (inference "
                         "mode; cubic Hermite interpolation per pair)")
    ap.add_argument("--per-molecule", action="store_true",
                    help="for batched workloads, also time one eager call per molecule")
    return ap.parse_args()


# ------------------------------------------------------------------ utils ---
def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def job_rate(units_per_rank, local_ms, world):
    """Whole-job throughput: units of all ranks / the slowest rank's time."""
    return world * units_per_rank / (allmax(local_ms, world) / 1e3)


def allmax(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def load_workload(name):
    from paper_2402_17660_gb300 import synth
    return synth.workload(name)


def carve_cluster(sys_, n_target, seed=0):
    """Atoms (whole molecules of 3 for water boxes) nearest the box centre,
    unwrapped into one non-periodic cluster: a bounded oracle sample."""
    from paper_2402_17660_gb300 import synth
    if sys_.n_systems > 1:
        # batched workload: the first whole molecules, up to n_target atoms
        ends = np.searchsorted(sys_.batch, np.arange(1, sys_.n_systems + 1))
        k = max(1, int(np.searchsorted(ends, n_target, side="right")))
        n = int(ends[k - 1])
        return synth.System(sys_.name + f"_first{k}mol", sys_.z[:n], sys_.pos[:n], sys_.batch[:n], None, k)
    pos = sys_.pos.astype(np.float64)
    if sys_.box is not None:
        L = np.diag(sys_.box[0]).astype(np.float64)
        c = L / 2
        d = pos - c
        d -= L * np.round(d / L)
        pos = c + d
    else:
        c = pos.mean(0)
    r = np.linalg.norm(pos - c, axis=1)
    idx = np.sort(np.argsort(r)[:n_target])
    return synth.System(sys_.name + f"_sample{n_target}", sys_.z[idx], pos[idx].astype(np.float32),
                        np.zeros(len(idx), np.int32), None, 1)


def oracle_eval_seconds(sys_, W, reps=1, want=False):
    from oracle.neighbors import neighbor_pairs
    from oracle.tensornet import TensorNet as Oracle
    o = Oracle(W)
    t0 = time.perf_counter()
    for _ in range(reps):
        pr = neighbor_pairs(sys_.pos, sys_.batch, sys_.box, 5.0)
        Es, Ei, Fr, _ = o.energy_forces(sys_.z, sys_.pos, sys_.batch, sys_.box, pairs=pr, n_systems=sys_.n_systems)
    t = (time.perf_counter() - t0) / reps
    return (t, (Es, Ei, Fr)) if want else t


ORACLE_THREADS_NOTE = ("the oracle is NumPy: its matrix products run on the BLAS thread pool (up to `cores` "
                       "threads); its elementwise work runs on one thread")


def oracle_eval_seconds_single_thread(sys_, W):
    """The same evaluation as oracle_eval_seconds in a child process whose
    BLAS and OpenMP pools hold one thread (a fresh process, so the setting
    takes effect before NumPy loads its BLAS).  None if the child fails."""
    import pickle
    import tempfile
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    code = ("import pickle, sys; sys.path.insert(0, sys.argv[2]); import bench; "
            "s, W = pickle.load(open(sys.argv[1], 'rb')); print(bench.oracle_eval_seconds(s, W))")
    with tempfile.TemporaryDirectory() as td:
        f = os.path.join(td, "sample.pkl")
        with open(f, "wb") as fh:
            pickle.dump((sys_, W), fh)
        try:
            out = subprocess.run([sys.executable, "-c", code, f, ROOT], env=env, capture_output=True, text=True,
                                 timeout=900, cwd=ROOT)
            return float(out.stdout.strip().splitlines()[-1]) if out.returncode == 0 else None
        except (subprocess.TimeoutExpired, ValueError, IndexError):
            return None


def cpu_baseline(sys_, W, single_thread=True):
    """The oracle as it stands on the host cores, on a bounded sample: the
    whole workload up to 3,000 atoms; above that a 1,500-atom cluster carved
    from it, whose rate is extrapolated to the workload linearly in the atom
    count (said so in the record, with the sample's own measured rate).  The
    same sample is timed again on one thread."""
    if sys_.n_atoms <= 3000:
        t, ref = oracle_eval_seconds(sys_, W, want=True)
        rec = {"value": 1.0 / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one full FP64 oracle energy+force evaluation of {sys_.name} "
                         f"(brute-force pairs + forward + analytic reverse pass), {t:.1f} s",
               "measured_on_full_workload": True, "threads": ORACLE_THREADS_NOTE}
        sample, scale = sys_, 1.0
    else:
        sample = carve_cluster(sys_, 1500)
        n = sample.n_atoms
        t = oracle_eval_seconds(sample, W)
        scale = n / sys_.n_atoms
        ref = None
        rec = {"value": scale / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one FP64 oracle energy+force evaluation of {sample.name}, a {n}-atom open cluster "
                         f"carved from {sys_.name} ({t:.1f} s)",
               "measured_on_full_workload": False,
               "sample_value": 1.0 / t, "sample_unit": f"evals/s of the {n}-atom sample",
               "extrapolation": f"value = the sample's rate x {n}/{sys_.n_atoms} atoms (linear in atoms; the "
                                "oracle's brute-force pair search is quadratic, so the whole workload would "
                                "take longer than this)", "threads": ORACLE_THREADS_NOTE}
    if single_thread:
        t1 = oracle_eval_seconds_single_thread(sample, W)
        rec["single_thread"] = (None if t1 is None else
                                {"value": scale / t1, "unit": UNIT, "cores": 1, "seconds_per_sample_eval": t1,
                                 "how": "the same sample in a child process with one BLAS/OpenMP thread"})
    return rec, ref


def workload_config(sys_, n_pairs, args, graph=True):
    return {"workload": sys_.name, "n_atoms": sys_.n_atoms, "n_systems": sys_.n_systems,
            "periodic": sys_.box is not None, "directed_pairs": int(n_pairs), "cutoff_A": 5.0,
            "layers": 2, "channels": 128, "rbf": 32, "precision": args.precision,
            "radial_functions": (f"tabulated at {args.radial_table} distances, cubic Hermite"
                                 if args.radial_table else "radial MLP per pair"),
            "radial_mlp_activations": "recomputed in the reverse pass" if recompute_edges(args, sys_.n_atoms)
            else "kept from the forward pass",
            "step": "neighbor search + energy + forces", "cuda_graph": graph,
            "l2": "flushed (256 MB write) before every timed step"}


# ------------------------------------------------------------- reference ---
REFERENCE_SAMPLE_ATOMS = 300


def run_reference(args):
    """The oracle, as it stands, on the host cores.  Each step is one FP64
    energy+force evaluation of a bounded sample of the workload (the whole
    workload up to 300 atoms, else a 300-atom cluster carved from it), so
    the whole --warmup + --steps run ends within minutes.  The line reports
    the sample's own evals/s and ms per step and names the sample in
    config.workload; an extrapolation to the whole workload is given apart,
    labelled as one."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2402_17660_gb300 import synth
    sys_ = load_workload(args.workload)
    W = synth.init_weights(synth.ModelShape(), seed=0)
    sample = sys_ if sys_.n_atoms <= REFERENCE_SAMPLE_ATOMS else carve_cluster(sys_, REFERENCE_SAMPLE_ATOMS)
    n = sample.n_atoms
    same = sample is sys_
    for _ in range(args.warmup):
        oracle_eval_seconds(sample, W)
    ts = [oracle_eval_seconds(sample, W) for _ in range(args.steps)]
    per_step = sum(ts) / len(ts)
    value = 1.0 / per_step
    desc = (f"one FP64 oracle energy+force evaluation of {sys_.name} per step" if same else
            f"one FP64 oracle energy+force evaluation per step of {sample.name}, a {n}-atom open cluster carved "
            f"from {sys_.name} ({sys_.n_atoms} atoms)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": sample.name, "n_atoms": n, "sample_of": sys_.name,
                       "sample_of_n_atoms": sys_.n_atoms, "same_config": same, "periodic": sample.box is not None},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if not same:
        line["extrapolated_to_workload"] = {
            "value": value * n / sys_.n_atoms, "unit": f"evals/s of {sys_.name}",
            "method": f"the sample's rate x {n}/{sys_.n_atoms} atoms (an estimate, not a measurement)"}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ ours ---
def stage_work(tag, nu, N, E, F, K, prec, table=0, rec=False):
    """Algorithmic work of one instance of a timed stage: (FLOP, bytes, engine).
    Bytes count each unique operand read once and each result written once,
    including the bf16 operand copies the BF16 mode writes beside a result
    (2 B per element; the 3xTF32 mode writes none: it splits its operands in
    shared memory).  The radial filter g = phi SiLU(a3) is never stored: the
    last radial layer writes a3 alone and the message kernels read a3 and phi.
    rec (activations recomputed in the reverse pass): the forward instances
    of radial layers 1 and 2 write no pre-activation, the reverse-pass
    instances do; the figure is the mean over the two.  table = n > 0:
    tabulated radial functions, whose [n-1][3F] float4 tables are read once
    per launch (they stay in L2; at most one interval per pair) in place of
    the per-pair f and a3 arrays, and whose radial-MLP stages do not run."""
    f = 4.0
    bf16 = prec == "bf16"
    cp = 2.0 if bf16 else 0.0            # operand-copy bytes per element
    hb = 2.0 if bf16 else 4.0            # bytes per element of a GEMM input operand
    if table:
        tab = min(table - 1, nu) * 3 * F * 16.0   # each pair reads one interval
        hermite = 2.0 * 7 * 3 * F * 2 * nu   # value (and slope) of each edge's interval
        if tag == "emb_edges":
            return 2.0 * 12 * F * 2 * nu + hermite / 2, (f + cp) * 9 * N * F + tab, "hbm"
        if tag == "emb_edges_bwd":  # reads gX_raw, writes 16 B per edge, updates dE/dd
            return 2.0 * 43 * F * 2 * nu + hermite / 2, f * (9 * N * F + 2 * nu) + 16.0 * E + tab, "hbm"
        if tag == "message":
            return 2.0 * 9 * F * 2 * nu + hermite / 2, f * 2 * 9 * N * F + 8.0 * E + tab, "hbm"
        if tag == "message_bwd":    # no dE/da3; dE/dd of each pair updated
            rd = f * 3 * 9 * N * F + 8.0 * E + tab
            wr = (f + cp) * 9 * N * F + 2 * f * nu
            return 4.0 * 9 * F * 2 * nu + 2.0 * 3 * F * nu + hermite, rd + wr, "hbm"
        if tag.startswith("mlp"):
            return None
    pre = 0.5 if rec else 1.0            # share of instances that store the pre-activation
    hw = (f if not bf16 else 0.0) + cp   # bytes stored per activation element (fp32 unless BF16 copies only)
    if tag == "mlp1":
        return 2.0 * nu * K * F, nu * (K * f + pre * F * f + F * hw), "alu"
    if tag == "mlp2":
        return 2.0 * nu * F * 2 * F, nu * (F * hb + pre * 2 * F * f + 2 * F * hw), "tensor" if bf16 else "alu"
    if tag == "mlp3":
        return 2.0 * nu * 2 * F * 3 * F, nu * (2 * F * hb + 3 * F * f), "tensor" if bf16 else "alu"
    if tag == "mlp3_bwd":
        return 2.0 * nu * 3 * F * 2 * F, nu * (3 * F * hb + 2 * F * f + 2 * F * f + (2 * F * 2 if bf16 else 0)), \
            "tensor" if bf16 else "alu"
    if tag == "mlp2_bwd":
        return 2.0 * nu * 2 * F * F, nu * (2 * F * hb + F * f + F * f), "tensor" if bf16 else "alu"
    if tag == "mlp1_bwd":
        return 2.0 * nu * F * K, nu * (F * f + 2 * K * f), "alu"
    if tag == "emb_edges":   # read the pair projections once, write X_raw once
        return 2.0 * 12 * F * 2 * nu, f * (3 * F * nu + 9 * N * F) + cp * 9 * N * F, "hbm"
    if tag == "emb_edges_bwd":
        # read gX_raw and the projections, write their adjoint and 16 B per
        # edge; then the projections' input-gradient GEMM (read dE/df, update
        # dE/de)
        return 2.0 * 40 * F * 2 * nu + 2.0 * nu * 3 * F * K, \
            f * (9 * N * F + 6 * F * nu) + 16.0 * E + nu * (3 * F * f + 2 * K * f), "hbm"
    if tag == "message":     # read Y, a3 and phi once, write M once, read the CSR
        return 2.0 * 9 * F * 2 * nu, f * (2 * 9 * N * F + 3 * F * nu + nu) + 8.0 * E, "hbm"
    if tag == "message_bwd":
        # read Y, gM, gY, a3 and phi; write gY (+ copy), dE/da3 (fp32 unless
        # bf16, + copy) and update dE/dphi; read the CSR
        rd = f * (3 * 9 * N * F + 3 * F * nu + nu) + 8.0 * E
        wr = (f + cp) * 9 * N * F + ((0.0 if bf16 else f) + cp) * 3 * F * nu + 2 * f * nu
        return 4.0 * 9 * F * 2 * nu + 6.0 * 3 * F * nu, rd + wr, "hbm"
    return None


def stage_roofline(tag, per_launch_ms, nu, N, E, F, K, prec, table, rec, peaks):
    """Roofline of one stage instance from its algorithmic work (stage_work)
    and its measured time per instance: the bound is the tensor or ALU roof
    when the arithmetic intensity is above that roof's ridge point against
    HBM, else HBM.  3xTF32 GEMMs count useful FLOP against a third of the TF32
    rate (three MMAs per product).  Peaks: MEASURED_PEAKS.json, else the
    fallbacks named in each record."""
    flops, nbytes, engine = stage_work(tag, nu, N, E, F, K, prec, table, rec)
    hbm = peaks.get("hbm_gbs", 6800.0)
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12  # TFLOP/s, derived
    if prec == "tf32x3" and not table and tag in ("mlp2", "mlp3", "mlp3_bwd", "mlp2_bwd"):
        # 3xTF32: three TF32 MMAs per product (the residuals are formed on
        # chip, so the bytes are those of the fp32 operands)
        engine = "tensor_tf32"
    if engine == "tensor":
        cpeak, cname, cnote = bf16_peak, "tensor", "of measured bf16 burst (MEASURED_PEAKS.json)"
    elif engine == "tensor_tf32":
        # useful FLOP against one third of the TF32 rate (nominal TF32 = bf16 / 2)
        cpeak, cname = bf16_peak / 2 / 3, "tensor"
        cnote = "measured bf16 burst x nominal TF32/BF16 ratio 1/2, divided by the 3 MMAs of 3xTF32"
    else:
        cpeak, cname, cnote = fp32_peak, "alu", "FP32 FFMA peak 152 SM x 128 lanes x 2 x 2070 MHz (derived)"
    ridge = cpeak * 1e12 / (hbm * 1e9)            # FLOP per byte where the two roofs meet
    if engine != "hbm" and flops / nbytes >= ridge:
        ach = flops / (per_launch_ms * 1e-3) / 1e12
        out = {"bound": cname, "achieved": ach, "peak": cpeak, "unit": "TFLOP/s", "frac": ach / cpeak,
               "peak_note": cnote}
    else:
        ach = nbytes / (per_launch_ms * 1e-3) / 1e9
        out = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
               "peak_note": "of measured HBM copy bandwidth (MEASURED_PEAKS.json)"}
    out.update({"kernel": tag, "algorithmic_flop_per_launch": flops, "algorithmic_bytes_per_launch": nbytes,
                "launch_ms": per_launch_ms, "arithmetic_intensity": flops / nbytes})
    return out


KEPT_BYTES_PER_PAIR_SLOT = 4.5 * 1024   # a1, h1, a2, h2, a3 at F = 128: per undirected pair and layer


def recompute_edges(args, n_atoms):
    """auto: keep the radial-MLP activations (no second forward through the
    radial MLP in the reverse pass) unless, at the bench's pair capacity of
    75 directed pairs per atom and two layers, they would take more than a
    quarter of the device's memory (about 200,000 atoms on a GB300)."""
    if args.recompute_edges != "auto":
        return args.recompute_edges == "1"
    try:
        import torch
        total = torch.cuda.get_device_properties(0).total_memory
    except Exception:
        total = 280e9
    kept = KEPT_BYTES_PER_PAIR_SLOT * (75 * n_atoms / 2) * 2
    return kept > 0.25 * total


def run_ours(args):
    import torch
    world, rank, local = dist_setup(args)
    from paper_2402_17660_gb300 import _lib, synth
    from paper_2402_17660_gb300.tnet import TensorNet
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    sys_ = load_workload(args.workload)
    shape = synth.ModelShape()
    W = synth.init_weights(shape, seed=0)
    N = sys_.n_atoms
    cap = int(75 * N) + 1024
    prec = {"fp32": 0, "bf16": 1, "tf32x3": 2}[args.precision]
    rec = recompute_edges(args, N)
    m = TensorNet(W, max_atoms=N, max_systems=sys_.n_systems, max_pairs=cap, precision=prec, device=dev,
                  recompute_edges=rec, radial_table=args.radial_table)
    lib = m.lib
    table_build_ms = None
    if args.radial_table:   # one-off per weight set: time a rebuild of the tables
        t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0e.record()
        m.set_weights(W)
        t1e.record()
        torch.cuda.synchronize()
        table_build_ms = t0e.elapsed_time(t1e)
    z = torch.from_numpy(sys_.z).to(dev)
    pos = torch.from_numpy(sys_.pos).to(dev)
    batch = torch.from_numpy(sys_.batch).to(dev) if sys_.n_systems > 1 else None
    box = torch.from_numpy(sys_.box).to(dev) if sys_.box is not None else None
    S = sys_.n_systems

    # eager first call: allocate outputs, check status, learn the pair count
    m.reset_status()
    nl = m.neighbors(pos, batch, box, S)
    E = torch.empty(S, dtype=torch.float64, device=dev)
    Fo = torch.empty((N, 3), dtype=torch.float32, device=dev)
    m.energy_forces(z, pos, nl, batch, box, S, out=(E, Fo, None))
    torch.cuda.synchronize()
    m.check_status("bench warm-up")
    n_pairs = int(nl.n_pairs.item())
    nu = n_pairs // 2

    # launch shapes from the autotuner (timed on this input, cached as JSON)
    from paper_2402_17660_gb300.tnet import autotune
    if args.tuning == "auto":
        knobs, tune_ms = autotune(m, z, pos, nl, batch, box, S)
    else:
        if args.tuning != "default":
            m.set_tuning([int(v) for v in args.tuning.split(",")])
        knobs, tune_ms = m.get_tuning(), {}

    def step():
        m.neighbors(pos, batch, box, S, out=nl)
        m.energy_forces(z, pos, nl, batch, box, S, out=(E, Fo, None))

    # capture the step in a CUDA graph (and count the kernels it launches)
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    c0 = lib.tnet_launch_count()
    with torch.cuda.graph(g):
        step()
    launches_per_step = int(lib.tnet_launch_count() - c0)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    for _ in range(args.warmup):
        flush.zero_()
        g.replay()
    torch.cuda.synchronize()

    # ---- timed region
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record()
        g.replay()
        ends[k].record()
    torch.cuda.synchronize()
    barrier(world)
    ck = clocks.stop() if rank == 0 else None
    times = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    value = job_rate(args.steps, sum(times), world)
    total_ms = world * args.steps / value * 1e3
    m.reset_status()
    g.replay()
    torch.cuda.synchronize()
    m.check_status("bench timed steps")

    # ---- live per-stage timing (eager steps with the library's event profiler)
    F_ = shape.F
    lib.tnet_profile(m.ctx, 1)
    for _ in range(args.profile_steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ntag = 32
    ms = (ctypes.c_float * ntag)()
    cnt = (ctypes.c_int64 * ntag)()
    lib.tnet_profile_read(m.ctx, ntag, ms, cnt)
    lib.tnet_profile(m.ctx, 0)
    stages = {}
    for t in range(ntag):
        name = lib.tnet_profile_tag(t)
        if name is None:
            break
        if cnt[t]:
            stages[name.decode()] = {"ms_per_step": ms[t] / args.profile_steps, "instances": int(cnt[t])}
    roofline = None
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    tab = args.radial_table > 0
    work_tags = [k for k in sorted(stages, key=lambda k: -stages[k]["ms_per_step"])
                 if stage_work(k, nu, N, n_pairs, F_, shape.K, args.precision, args.radial_table, rec) is not None]
    # every stage with a work model, against its own roof (the same live
    # CUDA-event stage times as the dominant stage's line)
    stage_rooflines = {}
    for tag in work_tags:
        per_launch_ms = stages[tag]["ms_per_step"] * args.profile_steps / stages[tag]["instances"]
        r = stage_roofline(tag, per_launch_ms, nu, N, n_pairs, F_, shape.K, args.precision, args.radial_table,
                           rec, peaks)
        stage_rooflines[tag] = {k: r[k] for k in ("bound", "achieved", "unit", "frac")}
    if work_tags:
        tag = work_tags[0]
        per_launch_ms = stages[tag]["ms_per_step"] * args.profile_steps / stages[tag]["instances"]
        roofline = stage_roofline(tag, per_launch_ms, nu, N, n_pairs, F_, shape.K, args.precision,
                                  args.radial_table, rec, peaks)
        traffic = None
        tpath = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tpath):
            tkey = f"{args.workload}:{args.precision}:{tag}" + (f":table{args.radial_table}" if tab else "")
            if tag in ("message", "message_bwd", "emb_edges_bwd") and len(knobs) > 6:
                tkey += f":kernel{knobs[6]}"   # which form of the row kernels ran (the message_kernel knob)
            tr = json.load(open(tpath)).get(tkey)
            if tr and tr.get("kernel_rev") == kernel_revision(tr.get("rev_files")):
                traffic = tr["bytes_per_launch"]
        roofline = {**roofline, "traffic": traffic}

    # ---- end to end through the public API with host buffers
    pos_h = torch.from_numpy(sys_.pos).pin_memory()
    E_h = torch.empty(S, dtype=torch.float64).pin_memory()
    F_h = torch.empty((N, 3), dtype=torch.float32).pin_memory()
    pos_d = torch.empty_like(pos)

    def e2e_step():
        pos_d.copy_(pos_h, non_blocking=True)
        m.neighbors(pos_d, batch, box, S, out=nl)
        m.energy_forces(z, pos_d, nl, batch, box, S, out=(E, Fo, None))
        E_h.copy_(E, non_blocking=True)
        F_h.copy_(Fo, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    e0.record()
    for _ in range(args.steps):
        e2e_step()
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = allmax(e0.elapsed_time(e1), world)
    e2e = {"value": world * args.steps / (e2e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(pos_h.numel() * 4), "d2h_bytes_per_step": int(E_h.numel() * 8 + F_h.numel() * 4),
           "path": "TensorNet.neighbors + TensorNet.energy_forces (eager) with pinned host positions in "
                   "and energy + forces out"}

    # accuracy of this run's result: against the FP32 path on the same GPU, and
    # (below, with the CPU baseline) against the FP64 oracle
    m.energy_forces(z, pos, nl, batch, box, S, out=(E, Fo, None))
    torch.cuda.synchronize()
    E_run, F_run = E.cpu().numpy().copy(), Fo.cpu().numpy().astype(np.float64)
    accuracy = {}
    if prec != 0 or args.radial_table:
        m32 = TensorNet(W, max_atoms=N, max_systems=S, max_pairs=cap, precision=0, device=dev,
                        recompute_edges=rec)
        nl32 = m32.neighbors(pos, batch, box, S)
        E32, F32, _ = m32.energy_forces(z, pos, nl32, batch, box, S)
        torch.cuda.synchronize()
        F32 = F32.cpu().numpy().astype(np.float64)
        E32n = E32.cpu().numpy()
        accuracy["vs_fp32_gpu"] = {
            # RMS over systems, relative to the RMS energy (single molecules of a
            # batch can have energies near zero)
            "energy_rel_rms": float(np.sqrt(np.mean((E_run - E32n) ** 2) / np.mean(E32n ** 2))),
            "energy_abs_max_per_atom": float(np.max(np.abs(E_run - E32n)) / (N / S)),
            "force_rel_rms": float(np.sqrt(np.mean(np.sum((F_run - F32) ** 2, 1)) / np.mean(np.sum(F32 ** 2, 1))))}
        del m32
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {0: "f32", 1: "bf16 GEMM / f32",
                      2: "f32 (GEMMs as 3xTF32 on the tensor cores: FP32-level accuracy)"}[prec],
            "data": "synthetic",
            "config": workload_config(sys_, n_pairs, args),
            "ns_per_day_at_0.5fs": value / world * 86400 * FS_PER_STEP * 1e-6,
            "e2e": e2e, "gpu_launches": launches_per_step * args.steps, "roofline": roofline,
            "stage_rooflines": stage_rooflines,
            "stages_ms_per_step": {k: round(v["ms_per_step"], 4) for k, v in
                                   sorted(stages.items(), key=lambda kv: -kv[1]["ms_per_step"])},
            "clocks": ck, "parallelism": f"replicas x{world}", "accuracy": accuracy,
            "tuning": {"knobs": knobs, "candidates_ms": tune_ms}}
    if args.radial_table:
        line["radial_table"] = {"points": args.radial_table, "build_ms_per_weight_set": table_build_ms,
                                "note": "tables built once per weight set (tnet_radial_tables), outside the "
                                        "timed step; accuracy.vs_fp32_gpu compares with the exact radial MLP"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], ref = cpu_baseline(sys_, W)
        if ref is not None:
            Es, Ei, Fr = ref
            scale = np.maximum(np.abs(Es), np.bincount(sys_.batch, weights=np.abs(Ei), minlength=len(Es)))
            accuracy["vs_fp64_oracle"] = {
                "energy_rel": float(np.max(np.abs(E_run - Es) / scale)),
                "force_rel_rms": float(np.sqrt(np.mean(np.sum((F_run - Fr) ** 2, 1)) / np.mean(np.sum(Fr ** 2, 1))))}
    if args.per_molecule and S > 1:
        line["per_molecule_launches"] = per_molecule(sys_, W, prec, dev, args)
    if args.md > 0:
        del g, m, nl
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        line["md"] = run_md(sys_, shape, prec, dev, args, knobs)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def per_molecule(sys_, W, prec, dev, args):
    """The same batch evaluated with one eager neighbor + energy/force call
    per molecule (the launch pattern the batched, graph-captured form
    replaces)."""
    import torch
    from paper_2402_17660_gb300.tnet import TensorNet
    starts = np.searchsorted(sys_.batch, np.arange(sys_.n_systems + 1))
    nmax = int(np.max(np.diff(starts)))
    m = TensorNet(W, max_atoms=nmax, max_systems=1, max_pairs=nmax * nmax + 64, precision=prec, device=dev)
    mols = []
    for s in range(sys_.n_systems):
        a, b = starts[s], starts[s + 1]
        mols.append((torch.from_numpy(sys_.z[a:b]).to(dev), torch.from_numpy(sys_.pos[a:b]).to(dev)))

    def one_pass():
        for zz, pp in mols:
            nl = m.neighbors(pp)
            m.energy_forces(zz, pp, nl)

    one_pass()
    torch.cuda.synchronize()
    m.check_status("per-molecule pass")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(1, args.steps // 5)
    t0 = time.perf_counter()
    e0.record()
    for _ in range(reps):
        one_pass()
    e1.record()
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) / reps
    gpu = e0.elapsed_time(e1) / 1e3 / reps
    return {"value": 1.0 / max(wall, gpu), "unit": "batch evals/s", "molecules": sys_.n_systems,
            "ms_per_batch": max(wall, gpu) * 1e3, "kernels_per_batch": None,
            "note": "eager: one tnet_neighbors + tnet_energy_forces call per molecule, no graph"}


def run_md(sys_, shape, prec, dev, args, knobs=None):
    """Velocity Verlet through tnet_md_step (blocks of 20 steps replayed as
    one CUDA graph): ns/day and total-energy drift, with the launch shapes
    the autotuner chose for this workload's energy+force step."""
    import torch
    from paper_2402_17660_gb300 import synth
    from paper_2402_17660_gb300.tnet import TensorNet
    if sys_.n_systems != 1:
        return {"skipped": "MD runs one system"}
    Wmd = synth.md_weights(shape, seed=0)
    N = sys_.n_atoms
    m = TensorNet(Wmd, max_atoms=N, max_systems=1, max_pairs=int(100 * N) + 1024, precision=prec, device=dev,
                  recompute_edges=recompute_edges(args, N), radial_table=args.radial_table)
    if knobs is not None:
        m.set_tuning(knobs)
    z = torch.from_numpy(sys_.z).to(dev)
    pos = torch.from_numpy(sys_.pos).to(dev).clone()
    vel = torch.from_numpy(synth.maxwell_boltzmann(sys_, 300.0, seed=1)).to(dev)
    inv_m = torch.from_numpy(1.0 / sys_.masses()).to(dev)
    box = torch.from_numpy(sys_.box).to(dev) if sys_.box is not None else None
    R, dt = 20, 0.5
    n = max(R, (args.md // R) * R)
    m.reset_status()
    m.md(z, inv_m, pos, vel, box, dt, 1.0, R, 2 * R)           # warm-up, graph capture
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ek, ep = m.md(z, inv_m, pos, vel, box, dt, 1.0, R, n)
    e1.record()
    torch.cuda.synchronize()
    status = int(m.status.item())
    sec = e0.elapsed_time(e1) / 1e3
    et = (ek + ep).cpu().numpy()
    return {"steps": n, "dt_fs": dt, "rebuild_every": R, "skin_A": 1.0, "ns_per_day": n * dt * 1e-6 / sec * 86400,
            "steps_per_s": n / sec, "drift_eV_per_atom_per_ps": float((et[-1] - et[0]) / N / (n * dt * 1e-3)),
            "neighbor_builds": m.md_rebuilds(),
            "rebuild_rule": "every 20 steps and in any step where an atom moved > skin/2 (device-side test)",
            "status": status, "weights": "random init, output layer scaled by 0.05",
            "tuning": m.get_tuning()}


def _definition(text: str, name: str) -> str:
    """Source text of the __global__/__device__ function `name`, from its
    qualifier to its matching closing brace."""
    import re
    m = re.search(r"\b(?:__global__|__device__)[^;{}]*?\b" + re.escape(name) + r"\s*\(", text)
    if m is None:
        raise KeyError(name)
    i = text.index("{", m.end())
    depth = 0
    for j in range(i, len(text)):
        depth += {"{": 1, "}": -1}.get(text[j], 0)
        if depth == 0:
            return text[m.start():j + 1]
    raise ValueError(name)


def kernel_revision(parts=None) -> str:
    """Hash of the CUDA source a kernel is compiled from: whole files
    ("internal.cuh") or single function definitions ("model.cu:k_message_bwd");
    default: every file.  A stored ncu traffic figure is used only while that
    source is unchanged."""
    import hashlib
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_2402_17660_gb300", "csrc")
    for part in sorted(parts if parts else os.listdir(d)):
        fname, _, func = part.partition(":")
        with open(os.path.join(d, fname)) as fh:
            text = fh.read()
        h.update((_definition(text, func) if func else text).encode())
    return h.hexdigest()[:12]


def graph_ms(step, steps, warmup):
    """Capture step() in a CUDA graph, replay it `warmup` times, then time
    `steps` replays with CUDA events; ms per replay."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for _ in range(warmup):
        g.replay()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(steps):
        g.replay()
    ev[1].record()
    torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[1]) / steps


# Table tab:prot of the paper (million E+F steps/day, one RTX 4090, the
# whole model in one CUDA graph): context only, other GPU and real molecules.
PAPER_GRAPH_MSTEPS = {22: (172.80, 84.71, 56.47), 49: (154.29, 63.53, 39.82), 166: (77.14, 26.02, 15.57),
                      2489: (5.65, 1.69, 1.00), 5807: (2.33, 0.70, 0.42)}


def run_sweep(args):
    """Single molecules of the paper's five sizes (synthetic random walks),
    cutoff 4.5 A, 0/1/2 interaction layers: graph-replayed neighbor search +
    energy + forces."""
    import torch
    from paper_2402_17660_gb300 import synth
    from paper_2402_17660_gb300.tnet import TensorNet
    dev = torch.device("cuda:0")
    prec = {"fp32": 0, "bf16": 1, "tf32x3": 2}[args.precision]
    rows = []
    for n in (22, 49, 166, 2489, 5807):
        s = synth.random_walk_molecule(n, seed=n)
        z = torch.from_numpy(s.z).to(dev)
        pos = torch.from_numpy(s.pos).to(dev)
        for L in (0, 1, 2):
            shape = synth.ModelShape(L=L, cutoff_upper=4.5)
            W = synth.init_weights(shape, seed=0)
            m = TensorNet(W, L=L, cutoff_upper=4.5, max_atoms=n, max_pairs=64 * n + 64, precision=prec,
                          device=dev)
            nl = m.neighbors(pos, None, None, 1)
            E = torch.empty(1, dtype=torch.float64, device=dev)
            Fo = torch.empty((n, 3), dtype=torch.float32, device=dev)
            m.energy_forces(z, pos, nl, None, None, 1, out=(E, Fo, None))
            torch.cuda.synchronize()
            m.check_status("sweep")
            npairs = int(nl.n_pairs.item())

            def step():
                m.neighbors(pos, None, None, 1, out=nl)
                m.energy_forces(z, pos, nl, None, None, 1, out=(E, Fo, None))

            ms = graph_ms(step, max(args.steps, 50), max(args.warmup, 20))
            m.check_status("sweep")
            rate = 1e3 / ms
            rows.append({"atoms": n, "layers": L, "pairs": npairs, "ms_per_step": ms, "evals_per_s": rate,
                         "Msteps_per_day": rate * 86400 / 1e6,
                         "paper_rtx4090_graph_Msteps_per_day": PAPER_GRAPH_MSTEPS[n][L]})
            del m
    line = {"metric": "paper-shape sweep: TensorNet E+F steps/day, single molecules in vacuum", "unit": "Msteps/day",
            "dtype": {0: "f32", 1: "bf16 GEMM / f32", 2: "f32 (GEMMs as 3xTF32 on the tensor cores)"}[prec],
            "data": "synthetic: self-avoiding random walks (1.5 A steps, H/C/N/O) of the paper's five atom counts, "
                    "random-init weights",
            "config": {"cutoff_A": 4.5, "channels": 128, "rbf": 32, "pair_capacity": "64 per atom",
                       "step": "neighbor search + energy + forces, one CUDA graph", "l2": "not flushed (as the paper)"},
            "sweep": rows,
            "note": "paper column: Table tab:prot, RTX 4090, graph variant, real molecules and trained models "
                    "(context, not a target)"}
    print(json.dumps(line))
    return 0


def run_neighbor_bench(args):
    """tnet_neighbors alone on a random cloud of 32,768 particles at a density
    giving 64 neighbors per particle within the 5 A cutoff, split into 1 to
    1024 independent systems (each its own cloud of that density): the
    paper's neighbor benchmark, where one shared cell list degrades with the
    batch size; here cells are per system."""
    import torch
    from paper_2402_17660_gb300 import synth
    from paper_2402_17660_gb300.tnet import TensorNet
    dev = torch.device("cuda:0")
    n_total, rc, nbr = 32768, 5.0, 64
    rho = nbr / (4.0 / 3.0 * math.pi * rc ** 3)
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm = json.load(open(peaks_path)).get("hbm_gbs", 6800.0) if os.path.exists(peaks_path) else 6800.0
    rng = np.random.default_rng(7)
    rows = []
    W = synth.init_weights(synth.ModelShape(), seed=0)
    for B in (1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024):
        nb = n_total // B
        side = (nb / rho) ** (1.0 / 3.0)
        pos_np = np.concatenate([rng.uniform(0, side, (nb, 3)) for _ in range(B)]).astype(np.float32)
        batch_np = np.repeat(np.arange(B, dtype=np.int32), nb)
        cap = int(nbr * 1.3 * n_total) + 1024
        m = TensorNet(W, max_atoms=n_total, max_systems=B, max_pairs=cap, device=dev)
        pos = torch.from_numpy(pos_np).to(dev)
        batch = torch.from_numpy(batch_np).to(dev) if B > 1 else None
        box = None   # clouds in vacuum: a 32-particle system is far narrower than 2 cutoffs
        nl = m.neighbors(pos, batch, box, B, cutoff=rc)
        torch.cuda.synchronize()
        m.check_status("neighbor bench")
        npairs = int(nl.n_pairs.item())
        ms = graph_ms(lambda: m.neighbors(pos, batch, box, B, cutoff=rc, out=nl), max(args.steps, 50),
                      max(args.warmup, 10))
        m.check_status("neighbor bench")
        # algorithmic bytes: positions, batch, row offsets, one int per pair,
        # and the cell sort (cell index + sorted index + float4 copy per atom)
        nbytes = n_total * (12 + 4 + 4 + 2 * (4 + 4 + 16)) + 4 * npairs
        rows.append({"systems": B, "atoms_per_system": nb, "pairs": npairs, "pairs_per_atom": npairs / n_total,
                     "ms_per_call": ms, "Gpairs_per_s": npairs / ms / 1e6,
                     "hbm_GBs_algorithmic": nbytes / ms / 1e6, "hbm_frac_of_measured": nbytes / ms / 1e6 / hbm})
        del m
    line = {"metric": "tnet_neighbors time vs batch size (32,768 particles, 64 neighbors each)", "unit": "ms",
            "data": "synthetic uniform random clouds in vacuum, one cube per system at the same density "
                    "(small systems have fewer neighbors per particle: their surface)",
            "config": {"cutoff_A": rc, "particles": n_total, "step": "one tnet_neighbors call in a CUDA graph",
                       "l2": "not flushed"},
            "rows": rows}
    print(json.dumps(line))
    return 0


def run_neighbor_stress(args):
    """tnet_neighbors alone on the 1,029,000-atom periodic water box (a 70^3
    lattice of waters at 1 g/cm^3, 217.28 A cube) at the 5 A cutoff and at
    5 + 1 A skin: the size at which the search's algorithmic bytes exceed
    L2, so its HBM fraction can be read."""
    import torch
    from paper_2402_17660_gb300 import synth
    from paper_2402_17660_gb300.tnet import TensorNet
    dev = torch.device("cuda:0")
    t0 = time.perf_counter()
    s = synth.million_water_box()
    gen_s = time.perf_counter() - t0
    N = s.n_atoms
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm = json.load(open(peaks_path)).get("hbm_gbs", 6800.0) if os.path.exists(peaks_path) else 6800.0
    # a context whose workspace holds no per-pair radial-MLP activations: the
    # search does not depend on the model
    shape = synth.ModelShape(F=64, K=8, L=0)
    m = TensorNet(synth.init_weights(shape, seed=0), F=64, K=8, L=0, max_atoms=N, max_systems=1,
                  max_pairs=100 * N, device=dev, radial_table=256)
    pos = torch.from_numpy(s.pos).to(dev)
    box = torch.from_numpy(s.box).to(dev)
    rows = []
    for rc in (5.0, 6.0):
        nl = m.neighbors(pos, None, box, 1, cutoff=rc)
        torch.cuda.synchronize()
        m.check_status("neighbor stress")
        npairs = int(nl.n_pairs.item())
        ms = graph_ms(lambda: m.neighbors(pos, None, box, 1, cutoff=rc, out=nl), max(args.steps, 20),
                      max(args.warmup, 5))
        m.check_status("neighbor stress")
        # algorithmic bytes: positions, row offsets, one int per pair, and the
        # cell sort (cell index + sorted index + float4 copy per atom)
        nbytes = N * (12 + 4 + 2 * (4 + 4 + 16)) + 4 * npairs
        rows.append({"cutoff_A": rc, "pairs": npairs, "pairs_per_atom": npairs / N, "ms_per_call": ms,
                     "Gpairs_per_s": npairs / ms / 1e6, "algorithmic_bytes": nbytes,
                     "hbm_GBs_algorithmic": nbytes / ms / 1e6, "hbm_frac_of_measured": nbytes / ms / 1e6 / hbm})
    line = {"metric": "tnet_neighbors on the 1,029,000-atom periodic water box", "unit": "ms",
            "data": f"synthetic: 343,000 rigid waters on a jittered 70^3 lattice, 217.28 A cube (generated in "
                    f"{gen_s:.0f} s on the host)",
            "config": {"atoms": N, "step": "one tnet_neighbors call in a CUDA graph", "l2": "not flushed",
                       "hbm_peak_GBs": hbm},
            "rows": rows}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    if args.neighbor_bench:
        return run_neighbor_bench(args)
    if args.neighbor_stress:
        return run_neighbor_stress(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
