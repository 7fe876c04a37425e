#!/usr/bin/env python3
"""Benchmark of the GB300 stabilizer simulator on the 180,000-qubit workload.

Workload (synthetic, seeded; stands in for the paper's Qiskit heavy suite):
  180,000 qubits, 1,000 random Clifford layers (CX probability 0.4, seed 3),
  final Z-measurement of all qubits.
One step = one pass of the whole hot path on that circuit:
  tableau init + all 1,000 gate layers (device-resident gate records)
  + layout switch + the first M of the 180,000 final Z-measurements
  + F-shot Pauli-frame sampling of those ops (frames through all 1,000
    layers and the M measurements).
The full final measurement (180,000 sequential measurements, ~10^15 bytes of
row traffic) does not fit a bounded step; its first M measurements are the
most expensive ones (densest tableau) and are timed as the measurement phase.

value = Clifford gates applied / device time of the timed steps (CUDA events on
the sim's stream, max over ranks); the JSON line also gives per-phase rates
(gate-phase gates/s, measurements/s, shots/s), the roofline of the gate-layer
kernel, an end-to-end run through the host-buffer C-ABI calls and the oracle
timed on the host cores.

--impl reference times the CPU oracle (chp_oracle.c) as it stands on the
host cores for the same metric, on a bounded sample of the same workload.
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

from workloads import circuits as C  # noqa: E402

METRIC = "Clifford gates/s and measurements/s at 180k qubits; shots/s; % of HBM roofline"
N_QUBITS = 180_000
DEPTH = 1_000
FALLBACK_HBM_GBS = 6800.0

# ncu DRAM traffic of one gate-layer launch on the 180k workload, and the hash
# of the kernel source it was taken with (null once the kernel changes).
GATE_KERNEL_TRAFFIC = {"bytes_per_launch": (13282589952 + 8048602624 + 13303059968 + 8067709184) // 2,
                       "source_sha256": "8b093ed7c03f304cee9b71df544e81fdafb98d22663872b1f8b277bf7632a761"}


def _kernel_hash() -> str:
    """sha256 over the sources of the gate-layer kernel (its rules included)."""
    h = hashlib.sha256()
    for name in ("qs_gates.cu", "qs_rules.cuh"):
        with open(os.path.join(ROOT, "paper_2603_14641_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ----------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}

    def mean_power_w(self):
        pw = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            try:
                pw.append(float(parts[2]))
            except (IndexError, ValueError):
                continue
        return float(np.mean(pw)) if pw else None


# ----------------------------------------------------------------------
# distributed helpers (replicas: one independent circuit per GPU)
# ----------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(value: float, ws: int, backend_device=None) -> float:
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=backend_device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, ws: int, backend_device=None) -> float:
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=backend_device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------
# algorithmic bytes of one gate layer (columns of 2n bits = n/4 bytes)
# ----------------------------------------------------------------------
COLS_TOUCHED = {C.H: 4, C.S: 3, C.SDG: 3, C.CX: 6, C.CZ: 6, C.CY: 6, C.SWAP: 8, C.ISWAP: 8,
                C.X: 1, C.Z: 1, C.Y: 2}


def layer_bytes(gates: np.ndarray, n: int) -> float:
    cols = sum(COLS_TOUCHED[int(t)] * int(c) for t, c in zip(*np.unique(gates[:, 0],
                                                                           return_counts=True)))
    return cols * (n / 4.0) + n / 2.0  # + signs: read and write 2n bits


# ----------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------
WORKLOADS = {
    "n180k": lambda a: C.random_circuit(a.n, a.depth, 0.4, seed=3, name="n180k_d1000"),
    "n10k": lambda a: C.workload_10k(),
    "n256": lambda a: C.workload_256(),
}


def workload_label(name: str, n: int, depth: int, n_meas: int) -> str:
    """config.workload of both arms (the same string for the same workload)."""
    return (f"random Clifford circuit {name}: n={n} depth={depth} "
            f"({n_meas} Z-measurements in the full program)")


def step_program(circ, max_final: int):
    """The circuit's ops, with the last measurement window cut to its first
    `max_final` qubits when max_final > 0 (the full final measurement of a
    180k-qubit circuit does not fit a bounded step)."""
    ops = list(circ.ops)
    if max_final > 0 and ops and ops[-1][0] == "measure":
        ops[-1] = ("measure", np.asarray(ops[-1][1][:max_final], np.uint32))
    return ops


def run_ours(args):
    import torch
    from paper_2603_14641_gb300 import qs

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    t_gen = time.time()
    circ = WORKLOADS[args.workload](args)
    gen_s = time.time() - t_gen
    n, L = circ.n, circ.n_layers
    shots = args.shots
    seed = 1234 + rank
    prog = step_program(circ, args.measurements if args.workload == "n180k" else 0)
    M = int(sum(len(op[1]) for op in prog if op[0] == "measure"))

    stream = torch.cuda.Stream(device=dev)
    flags = qs.QS_FLAG_NO_FUSION if args.no_fusion else 0
    sim = qs.Simulator(n, device=str(dev), stream=stream, flags=flags)
    packed_host = qs.qs_pack_layers(n, circ.gates, circ.layer_ptr)
    packed_dev = torch.from_numpy(packed_host.view(np.int32)).to(dev)
    lp = np.asarray(circ.layer_ptr, np.int64)
    qdev = [torch.from_numpy(np.asarray(op[1], np.uint32).view(np.int32)).to(dev)
            if op[0] == "measure" else None for op in prog]
    ow = (shots + 63) // 64
    rec_dev = torch.zeros((max(M, 1), ow), dtype=torch.int64, device=dev)
    fw_bytes = 2 * n * ((ow + 3) // 4 * 4) * 8 + max(M, 1) * ow * 8 + 4096
    fws = torch.empty(fw_bytes, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    def step(ev):
        """ev: list of (kind, start event, end event) filled in program order."""
        qs.qs_sim_reset(sim.sim, None)
        for op, qd in zip(prog, qdev):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if op[0] == "layers":
                qs.qs_sim_apply_layers_dev(sim.sim, packed_dev.data_ptr(), lp, op[1], op[2])
            else:
                qs.qs_sim_measure_dev(sim.sim, qd.data_ptr(), qd.numel(), seed, 0)
            b.record(stream)
            ev.append((op[0], a, b))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        qs.qs_sim_sample(sim.sim, shots, seed + 7, rec_dev.data_ptr(), M * ow, fws.data_ptr(),
                         fw_bytes)
        b.record(stream)
        ev.append(("sample", a, b))

    for _ in range(args.warmup):
        step([])
    qs.qs_sim_sync(sim.sim)
    torch.cuda.synchronize()

    if args.full_final and args.workload == "n180k":
        prog = step_program(circ, 0)
        qdev = [torch.from_numpy(np.asarray(op[1], np.uint32).view(np.int32)).to(dev)
                if op[0] == "measure" else None for op in prog]
        M = int(sum(len(op[1]) for op in prog if op[0] == "measure"))
        rec_dev = torch.zeros((max(M, 1), ow), dtype=torch.int64, device=dev)
        fw_bytes = 2 * n * ((ow + 3) // 4 * 4) * 8 + max(M, 1) * ow * 8 + 4096
        fws = torch.empty(fw_bytes, dtype=torch.uint8, device=dev)
        args.steps = 1
    evs = [[] for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    qs.qs_sim_set_timing(sim.sim, True)  # CUDA events around each kernel class, on the sim's stream
    launches0 = qs.qs_sim_launch_count(sim.sim)
    with ClockSampler(local) as clk:
        barrier(ws)
        torch.cuda.synchronize()
        start.record(stream)
        for k in range(args.steps):
            step(evs[k])
        end.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
    launches = qs.qs_sim_launch_count(sim.sim) - launches0
    ktimes = qs.qs_sim_timing(sim.sim)
    qs.qs_sim_set_timing(sim.sim, False)
    qs.qs_sim_sync(sim.sim)  # device self-checks
    kinds = qs.qs_sim_record_kinds(sim.sim) if M else np.zeros(0, np.uint8)  # last step's record
    total_ms = start.elapsed_time(end)
    ph = {"layers": 0.0, "measure": 0.0, "sample": 0.0}
    for ev in evs:
        for kind, a, b in ev:
            ph[kind] += a.elapsed_time(b)
    gate_ms, meas_ms, samp_ms = ph["layers"], ph["measure"], ph["sample"]
    total_ms_max = reduce_max(total_ms, ws, dev)
    gates_step = circ.n_gates
    gates_all = reduce_sum(gates_step * args.steps, ws, dev)
    value = gates_all / (total_ms_max / 1e3)

    # roofline of the gate-layer kernel (its launches dominate the step)
    hbm, peak_kind = _peaks()
    alg_bytes = float(np.mean([layer_bytes(circ.layer(l), n) for l in range(0, L, max(1, L // 50))]))
    per_launch_s = gate_ms / 1e3 / (args.steps * L)
    achieved = alg_bytes / per_launch_s / 1e9
    fused = n * 16 <= 220 * 1024 and not args.no_fusion
    traffic = None
    if not fused and GATE_KERNEL_TRAFFIC["source_sha256"] == _kernel_hash() and \
            args.workload == "n180k":
        traffic = GATE_KERNEL_TRAFFIC["bytes_per_launch"]

    apply_pass = apply_roofline(ktimes, n, hbm, peak_kind)
    full_job = None
    if args.workload == "n180k" and not args.full_final and not args.no_full_job:
        full_job = run_full_job(args, qs, sim, circ, packed_dev, lp, shots, seed, stream, hbm,
                                peak_kind)
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, qs, sim, circ, prog, shots, seed, stream)
    noisy = None
    if args.noise > 0:
        noisy = noisy_sampling(args, qs, sim, circ, prog, packed_dev, lp, qdev, shots, seed, stream,
                               rec_dev, M, ow, fws, fw_bytes)

    clocks = clk.summary()
    power = clk.mean_power_w()
    # X and Z of one layout: 2 x ceil(n/256)*256 columns x ceil(2 ceil(n/64)/4)*4 words
    tab_gb = 2 * ((n + 255) // 256 * 256) * ((2 * ((n + 63) // 64) + 3) // 4 * 4) * 8 / 1e9
    energy = None
    if power is not None:
        j_step = power * total_ms_max / args.steps / 1e3
        energy = {"mean_power_w": power, "joules_per_step": j_step,
                  "gates_per_joule": gates_step / j_step,
                  "how": "runtime x mean nvidia-smi power.draw sampled every 200 ms over the "
                         "timed region (the paper's energy measure: runtime x average power)"}
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "gates/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u64",
        "data": "synthetic",
        "config": {
            "workload": workload_label(circ.name, n, L, circ.n_measurements),
            "step": f"init + {L} gate layers + {M} measurements"
                    + (f" (the first {M} of the {n} final measurements)"
                       if args.workload == "n180k" else "")
                    + f" + {shots}-shot frame sampling",
            "gates_per_step": gates_step,
            "measurements_per_step": M,
            "shots_per_step": shots,
            "fused_segments": fused,
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
            "l2": (f"inputs larger than L2 (tableau {tab_gb:.3g} GB in each layout)" if tab_gb > 0.129
                   else f"tableau ({tab_gb * 1e3:.3g} MB per layout) smaller than L2 "
                        f"(no flush: L2-resident by design)"),
        },
        "phases": {
            "gate_layers": {"gates_per_s": gates_step * args.steps / (gate_ms / 1e3),
                            "ms_per_step": gate_ms / args.steps},
            "measurement": {"measurements_per_s": M * args.steps / (meas_ms / 1e3) if M else None,
                            "ms_per_step": meas_ms / args.steps,
                            "probabilistic": int((kinds == 1).sum()),
                            "deterministic": int((kinds == 0).sum()),
                            "includes": "column->row layout switch (2 transposes) per window",
                            "kernels_ms_per_step": {k: v[0] / args.steps for k, v in ktimes.items()
                                                    if k not in ("gates", "sample")},
                            "apply_pass": apply_pass},
            "sampling": {"shots_per_s": shots * args.steps / (samp_ms / 1e3),
                         "ms_per_step": samp_ms / args.steps,
                         "frame_gate_updates_per_s": gates_step * shots * args.steps /
                         (samp_ms / 1e3)},
            "sampling_noisy": noisy,
        },
        "full_job": full_job,
        "energy": energy,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "kernel": "fused_segment_kernel<true>" if fused else "gate_layer_kernel<true>",
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "note": ("fused: algorithmic bytes are the unfused per-layer bytes, so frac "
                              "is an effective rate" if fused else "per-layer kernel"),
                     "peak_source": f"{peak_kind} hbm_gbs"},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "e2e": e2e,
        "setup_s": {"generate_circuit": gen_s},
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, circ)
    sim.close()
    del packed_dev, qdev, rec_dev, fws
    torch.cuda.empty_cache()
    if rank == 0 and ws == 1 and args.workload == "n180k" and not args.no_extras:
        # the other configurations, compact, so that every bench run records them
        out["serve"] = serve_measure(args, args.serve_count, sweep=False, cpu=False)
        out["batch"] = batch_measure(args, steps=2, warmup=1, cpu=False)
        out["inverse_tableau_10k"] = inverse_mode_summary()
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def inverse_mode_summary():
    """F1 on the 10,000-qubit workload: the whole program (1,000 layers, 19,500
    measurements) in the inverse-tableau mode (Alg. 1's elimination, one
    measurement at a time) and in the default CHP mode (blocked), timed once
    each with CUDA events after a warm-up run; records must be identical."""
    import torch
    from paper_2603_14641_gb300 import qs
    circ = C.workload_10k()
    res = {}
    recs = {}
    for name, flags in (("inverse", qs.QS_FLAG_INVERSE_TABLEAU), ("chp", 0)):
        stream = torch.cuda.Stream()
        sim = qs.Simulator(circ.n, device="cuda:0", stream=stream, flags=flags)
        dc = sim.upload(circ)
        qd = [torch.from_numpy(np.asarray(op[1], np.uint32).view(np.int32)).cuda()
              if op[0] == "measure" else None for op in circ.ops]
        ev = {k: [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True), 0.0]
              for k in ("layers", "measure")}

        def run(timed):
            qs.qs_sim_reset(sim.sim, None)
            for op, q in zip(circ.ops, qd):
                e = ev["layers" if op[0] == "layers" else "measure"]
                if timed:
                    e[0].record(stream)
                if op[0] == "layers":
                    qs.qs_sim_apply_layers_dev(sim.sim, dc.packed.data_ptr(), dc.layer_ptr, op[1], op[2])
                else:
                    qs.qs_sim_measure_dev(sim.sim, q.data_ptr(), q.numel(), 77, 0)
                if timed:
                    e[1].record(stream)
                    e[1].synchronize()
                    e[2] += e[0].elapsed_time(e[1])

        run(False)
        torch.cuda.synchronize()
        run(True)
        recs[name] = sim.record()
        sim.sync()
        g_ms, m_ms = ev["layers"][2], ev["measure"][2]
        res[name] = {"gates_ms": g_ms, "measure_ms": m_ms, "total_ms": g_ms + m_ms,
                     "gates_per_s": circ.n_gates / (g_ms / 1e3),
                     "measurements_per_s": circ.n_measurements / (m_ms / 1e3)}
        sim.close()
    res["records_identical"] = bool(np.array_equal(recs["inverse"], recs["chp"]))
    res["what"] = ("10,000 qubits, 1,000 layers, 19,500 measurements (19 windows of 500 and a final "
                   "round of 10,000); inverse mode: one layer kernel per layer and four launches per "
                   "measurement (Alg. 1); chp: fused gate segments and blocked measurement")
    return res


def apply_roofline(ktimes, n, hbm, peak_kind):
    """The blocked measurement's apply pass (blk_apply_kernel), from the CUDA
    events the library recorded around each of its launches: algorithmic bytes
    per launch = read + write of every row of the row-major tableau (x and z;
    every row is touched in the first blocks of a final measurement of a
    scrambled state: targets, replaced destabilizers and new pivot rows)."""
    ms, cnt = ktimes.get("blk_apply", (0.0, 0))
    if not cnt:
        return None
    nrows = 64 * ((2 * ((n + 63) // 64) + 3) // 4 * 4)
    rs = (n + 255) // 256 * 4
    alg = 2 * 2 * nrows * rs * 8  # read + write, x and z
    per = ms / cnt
    gbs = alg / (per / 1e3) / 1e9
    return {"kernel": "blk_apply_kernel<uint32_t>", "launches": cnt, "ms_per_launch": per,
            "algorithmic_bytes_per_launch": alg, "achieved_gbs": gbs, "peak_gbs": hbm,
            "frac": gbs / hbm, "peak_source": f"{peak_kind} hbm_gbs",
            "timing": "CUDA events recorded by libqs around each launch on the sim's stream "
                      "(qs_sim_set_timing)"}


def run_full_job(args, qs, sim, circ, packed_dev, lp, shots, seed, stream, hbm, peak_kind):
    """The complete program once, outside the timed steps: init, all layers,
    all n final Z-measurements (blocked), and frame sampling of the whole
    program, with CUDA events on the sim's stream around each phase and the
    library's per-kernel-class events."""
    import torch
    dev = sim.device
    prog = step_program(circ, 0)
    qdev = [torch.from_numpy(np.asarray(op[1], np.uint32).view(np.int32)).to(dev)
            if op[0] == "measure" else None for op in prog]
    M = int(sum(len(op[1]) for op in prog if op[0] == "measure"))
    ow = (shots + 63) // 64
    rec_dev = torch.zeros((max(M, 1), ow), dtype=torch.int64, device=dev)
    fw_bytes = 2 * circ.n * ((ow + 3) // 4 * 4) * 8 + max(M, 1) * ow * 8 + 4096
    fws = torch.empty(fw_bytes, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    qs.qs_sim_set_timing(sim.sim, True)
    ev = {k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for k in ("layers", "measure", "sample")}
    ph = {"layers": 0.0, "measure": 0.0, "sample": 0.0}
    t0 = time.perf_counter()
    qs.qs_sim_reset(sim.sim, None)
    for op, qd in zip(prog, qdev):
        a, b = ev["layers" if op[0] == "layers" else "measure"]
        a.record(stream)
        if op[0] == "layers":
            qs.qs_sim_apply_layers_dev(sim.sim, packed_dev.data_ptr(), lp, op[1], op[2])
        else:
            qs.qs_sim_measure_dev(sim.sim, qd.data_ptr(), qd.numel(), seed, 0)
        b.record(stream)
        b.synchronize()
        ph["layers" if op[0] == "layers" else "measure"] += a.elapsed_time(b)
    a, b = ev["sample"]
    a.record(stream)
    qs.qs_sim_sample(sim.sim, shots, seed + 7, rec_dev.data_ptr(), M * ow, fws.data_ptr(), fw_bytes)
    b.record(stream)
    b.synchronize()
    ph["sample"] = a.elapsed_time(b)
    wall = time.perf_counter() - t0
    kt = qs.qs_sim_timing(sim.sim)
    qs.qs_sim_set_timing(sim.sim, False)
    qs.qs_sim_sync(sim.sim)
    kinds = qs.qs_sim_record_kinds(sim.sim)
    dev_s = sum(ph.values()) / 1e3
    return {"what": f"init + {circ.n_layers} layers + all {M} final Z-measurements + {shots}-shot "
                    f"frame sampling of the whole program, once, outside the timed steps",
            "s": dev_s, "wall_s": wall,
            "gates_s": ph["layers"] / 1e3, "measure_s": ph["measure"] / 1e3,
            "sample_s": ph["sample"] / 1e3,
            "measurements_per_s": M / (ph["measure"] / 1e3),
            "probabilistic": int((kinds == 1).sum()), "deterministic": int((kinds == 0).sum()),
            "kernels_s": {k: v[0] / 1e3 for k, v in kt.items()},
            "kernel_groups": {k: v[1] for k, v in kt.items()},
            "apply_pass": _job_apply(apply_roofline(kt, circ.n, hbm, peak_kind))}


def _job_apply(a):
    """Over the whole final measurement the blocks leave a growing share of the
    rows alone (the +-Z_q pivots of earlier blocks are neither read nor
    written), so the full-tableau byte count overstates what later blocks move:
    the job's figures are kept, under names that say so; the roofline fraction
    of the apply pass is the one of `phases.measurement` (dense blocks)."""
    if not a:
        return a
    return {"kernel": a["kernel"], "launches": a["launches"], "ms_per_launch": a["ms_per_launch"],
            "full_tableau_bytes_per_launch": a["algorithmic_bytes_per_launch"],
            "full_tableau_equivalent_gbs": a["achieved_gbs"],
            "note": "average over all blocks; later blocks skip the rows they leave alone, so "
                    "this is not a roofline fraction", "timing": a["timing"]}


def noisy_sampling(args, qs, sim, circ, prog, packed_dev, lp, qdev, shots, seed, stream, rec_dev, M,
                   ow, fws, fw_bytes):
    """Frame sampling of the step's program with circuit-level Pauli noise
    (DEPOLARIZE1/2(p) after every layer on the qubits of its gates, X_ERROR(p)
    before every measurement window), timed alone with CUDA events around the
    qs_sim_sample call, outside the step's timed region."""
    import torch
    base = C.Circuit(n=circ.n, gates=circ.gates, layer_ptr=circ.layer_ptr, ops=list(prog))
    noisy = C.with_circuit_noise(base, args.noise, args.noise)
    qi = 0
    qs.qs_sim_reset(sim.sim, None)
    n_noise = 0
    for op in noisy.ops:
        if op[0] == "layers":
            qs.qs_sim_apply_layers_dev(sim.sim, packed_dev.data_ptr(), lp, op[1], op[2])
        elif op[0] == "noise":
            qs.qs_sim_noise(sim.sim, op[1], op[2], op[3])
            n_noise += 1
        else:
            while qdev[qi] is None:
                qi += 1
            qs.qs_sim_measure_dev(sim.sim, qdev[qi].data_ptr(), qdev[qi].numel(), seed, 0)
            qi += 1
    torch.cuda.synchronize()
    times = []
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        qs.qs_sim_sample(sim.sim, shots, seed + 7, rec_dev.data_ptr(), M * ow, fws.data_ptr(),
                         fw_bytes)
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    qs.qs_sim_sync(sim.sim)
    ms = float(np.median(times))
    return {"shots_per_s": shots / (ms / 1e3), "ms": ms, "shots": shots, "noise_ops": n_noise,
            "noise": f"DEPOLARIZE1/DEPOLARIZE2({args.noise:g}) after every layer, "
                     f"X_ERROR({args.noise:g}) before every measurement window",
            "timing": "median of 3 qs_sim_sample calls, outside the step"}


def run_e2e(args, qs, sim, circ, prog, shots, seed, stream):
    """Same step through the calls a user makes with host buffers: per-layer
    qs_sim_apply_layer (host gate records -> pinned staging -> device),
    qs_sim_measure with host qubits and host outcomes, qs_sim_sample into a
    host record. Timed with CUDA events on the sim's stream around whole steps
    (host->device and device->host copies inside)."""
    import torch
    n = circ.n
    M = int(sum(len(op[1]) for op in prog if op[0] == "measure"))
    layers = [np.ascontiguousarray(circ.layer(l)) for l in range(circ.n_layers)]
    ow = (shots + 63) // 64
    rec_host = np.zeros((max(M, 1), ow), np.uint64)
    fw_bytes = 2 * n * ((ow + 3) // 4 * 4) * 8 + max(M, 1) * ow * 8 + 4096
    fws = torch.empty(fw_bytes, dtype=torch.uint8, device=sim.device)
    steps = max(1, args.e2e_steps)

    def step():
        qs.qs_sim_reset(sim.sim, None)
        for op in prog:
            if op[0] == "layers":
                for l in range(op[1], op[2]):
                    qs.qs_sim_apply_layer(sim.sim, layers[l])
            else:
                qs.qs_sim_measure(sim.sim, op[1], seed, 0, want_outcomes=True)
        qs.qs_sim_sample(sim.sim, shots, seed + 7, rec_host.ctypes.data, M * ow, fws.data_ptr(),
                         fw_bytes)

    step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        step()
    b.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = a.elapsed_time(b)
    h2d = circ.n_gates * 8 + M * 4
    d2h = M + M * ow * 8
    return {"value": circ.n_gates * steps / (ms / 1e3), "unit": "gates/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "steps": steps, "ms_per_step": ms / steps, "wall_s_per_step": wall / steps,
            "path": "qs_sim_apply_layer (host gates) per layer, qs_sim_measure (host outcomes), "
                    "qs_sim_sample (host record)"}


# ----------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ----------------------------------------------------------------------
def oracle_gate_rate(circ, rows: int, layers: int, seed: int = 0):
    """Oracle gates/s on the full n-qubit tableau, from a bounded sample: the
    oracle's gate rules act on every one of the 2n rows independently
    (Sec. 2.4), so `rows` sampled rows are evolved through `layers` layers and
    the time is scaled by 2n / rows."""
    from oracle import oracle as O
    rng = np.random.default_rng(seed)
    n = circ.n
    ids = np.sort(rng.choice(2 * n, size=rows, replace=False)).astype(np.uint32)
    sub = O.RowSubset(n, ids)
    g = circ.gates[:circ.layer_ptr[layers]]
    t0 = time.perf_counter()
    sub.apply(g)
    dt = time.perf_counter() - t0
    full_s = dt * (2 * n) / rows
    return len(g) / full_s, dt, len(g)


def oracle_prefix_run(n: int = 20_000, layers: int = 2, count: int = 64):
    """The oracle on the whole tableau of the same generator (p_cx 0.4, seed 3)
    at n qubits, measured directly (no scaling): `layers` layers, then the
    first `count` final measurements. The unpacked 180k tableau (130 GB) does
    not fit a bounded sample; this is the prefix the parity tests run."""
    from oracle import oracle as O
    c = C.random_circuit(n, layers, 0.4, seed=3, final_measure_all=False)
    o = O.Oracle(n)
    t0 = time.perf_counter()
    o.apply(c.gates)
    tg = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, kinds = o.measure(np.arange(count, dtype=np.uint32), seed=1)
    tm = time.perf_counter() - t0
    return {"n": n, "layers": layers, "gates": int(c.n_gates), "gates_s": tg,
            "gates_per_s": c.n_gates / tg, "measurements": count, "measure_s": tm,
            "measurements_per_s": count / tm, "probabilistic": int(kinds.sum())}


def cpu_baseline(args, circ):
    rate, dt, g = oracle_gate_rate(circ, rows=args.cpu_rows, layers=args.cpu_layers)
    pre = oracle_prefix_run(args.cpu_prefix_n, 2, 64)
    return {"value": rate, "unit": "gates/s", "cores": 1, "kind": "oracle",
            "sample": f"{args.cpu_rows} of {2 * circ.n} generator rows through the first "
                      f"{args.cpu_layers} layers ({g} gates) of the workload's {circ.n}-qubit "
                      f"circuit: measured {dt:.2f} s of CPU; value = gates x rows / 2n per "
                      f"second (the oracle's per-gate cost is proportional to the rows it "
                      f"updates, Sec. 2.4)",
            "measured_s": dt,
            "extrapolated": {"full_tableau_s_for_sample_gates": dt * (2 * circ.n) / args.cpu_rows,
                             "basis": "sample time x 2n / rows"},
            "measurements_per_s": pre["measurements_per_s"],
            "prefix": pre,
            "measurements_sample": f"whole tableau of the same generator at n={pre['n']}: "
                                   f"{pre['layers']} layers ({pre['gates_s']:.1f} s), then the "
                                   f"first {pre['measurements']} final measurements "
                                   f"({pre['measure_s']:.1f} s), measured directly",
            "host_cores_available": os.cpu_count()}


def batch_measure(args, steps: int, warmup: int, subset_every: int = 8, cpu: bool = True):
    """Batched workload: 512 independent circuits (n log-uniform 50..5,000,
    depth 200, 10% of qubits measured after every 10th layer) through qs_batch
    (the n < 1024 circuits in one persistent launch), against the same
    circuits run one at a time through the single-circuit path on the same GPU
    (a seeded subset of every `subset_every`-th circuit for the one-at-a-time
    leg, whose launches take tens of seconds for all 512)."""
    import torch
    from paper_2603_14641_gb300 import qs
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    circs = C.batch_workload(args.batch_count)
    seeds = [5000 + i for i in range(len(circs))]
    gates = sum(c.n_gates for c in circs)
    meas = sum(c.n_measurements for c in circs)
    stream = torch.cuda.Stream(device=dev)
    b = qs.Batch(circs, seeds, device=str(dev), stream=stream)
    tune_path = os.path.join("/tmp", "qs_batch_tuning.txt")
    t0 = time.time()
    tuning = b.autotune(round_limit=2, cache_path=tune_path)
    tune_s = time.time() - t0

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        e.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(e) / steps

    ms_batch = timed(lambda: b.run(tuning), steps, warmup)
    b.sync()
    # one circuit at a time through the single-circuit path (subset)
    idx = list(range(0, len(circs), subset_every))
    sub = [circs[i] for i in idx]
    bs = qs.Batch(sub, [seeds[i] for i in idx], device=str(dev), stream=stream)
    ms_batch_sub = timed(lambda: bs.run(tuning), steps, warmup)
    bs.sync()
    sims, dcs, qd = [], [], []
    for c in sub:
        s_ = qs.Simulator(c.n, device=str(dev), stream=stream)
        sims.append(s_)
        dcs.append(s_.upload(c))
        qd.append([torch.from_numpy(np.asarray(op[1], np.uint32).view(np.int32)).to(dev)
                   if op[0] == "measure" else None for op in c.ops])

    def one_at_a_time():
        for s_, c, dc, qq, i in zip(sims, sub, dcs, qd, idx):
            qs.qs_sim_reset(s_.sim, None)
            for op, q in zip(c.ops, qq):
                if op[0] == "layers":
                    qs.qs_sim_apply_layers_dev(s_.sim, dc.packed.data_ptr(), dc.layer_ptr, op[1], op[2])
                else:
                    qs.qs_sim_measure_dev(s_.sim, q.data_ptr(), q.numel(), seeds[i], 0)

    ms_single_sub = timed(one_at_a_time, 1, 1)
    identical = all(np.array_equal(s_.record(), b.record(i)) for s_, i in zip(sims, idx))
    g_sub = sum(c.n_gates for c in sub)
    m_sub = sum(c.n_measurements for c in sub)
    out = {"value": gates / (ms_batch / 1e3), "unit": "gates/s", "ms_per_run": ms_batch,
           "measurements_per_s": meas / (ms_batch / 1e3),
           "config": {"workload": f"{len(circs)} random Clifford circuits, n log-uniform "
                                  "50..5000, depth 200, p_cx 0.5, 10% measured every 10 layers",
                      "gates": gates, "measurements": meas,
                      "tuning": tuning.as_dict(), "autotune_s": tune_s},
           "subset": {"circuits": len(sub), "gates": g_sub, "measurements": m_sub,
                      "batch_ms": ms_batch_sub, "one_at_a_time_ms": ms_single_sub,
                      "speedup": ms_single_sub / ms_batch_sub,
                      "records_identical": bool(identical)}}
    if cpu:
        out["cpu_baseline"] = batch_cpu_baseline(circs, seeds)
    for s_ in sims:
        s_.close()
    return out


def run_batch(args):
    r = batch_measure(args, args.steps, args.warmup, cpu=not args.no_cpu_baseline)
    out = {"metric": "batched Clifford circuits: gates/s and measurements/s, one persistent "
                     "launch vs one circuit at a time",
           "value": r["value"], "unit": "gates/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_run"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
           "data": "synthetic", "config": r["config"],
           "measurements_per_s": r["measurements_per_s"], "subset": r["subset"],
           "cpu_baseline": r.get("cpu_baseline")}
    print(json.dumps(out))


def batch_cpu_baseline(circs, seeds, budget_s: float = 15.0):
    """The oracle on a seeded 32-circuit subset of the batch (every 16th
    circuit), smallest first, until about `budget_s` seconds of one core are
    spent: gates/s and measurements/s over the circuits it completed."""
    from oracle import oracle as O
    sub = sorted(range(0, len(circs), max(1, len(circs) // 32)), key=lambda i: circs[i].n)
    g = m = 0
    t0 = time.perf_counter()
    done = []
    for i in sub:
        if time.perf_counter() - t0 > budget_s:
            break
        O.run_circuit(circs[i], seed=seeds[i])
        g += circs[i].n_gates
        m += circs[i].n_measurements
        done.append(circs[i].n)
    dt = time.perf_counter() - t0
    return {"value": g / dt, "unit": "gates/s", "cores": 1, "kind": "oracle",
            "measurements_per_s": m / dt,
            "sample": f"{len(done)} circuits (n {min(done)}..{max(done)}) of a 32-circuit subset "
                      f"(every 16th), smallest first, {dt:.1f} s of CPU"}


def serve_measure(args, count: int, sweep: bool = True, cpu: bool = True):
    """Serving workload: Poisson stream of requests (n log-uniform 100..20,000,
    depth 100..500, shots log-uniform 1e3..1e6, each ending with a Z-measurement
    of every qubit). Measures the saturation rate (all requests at t = 0), then
    (if `sweep`) p50/p99 latency and shots/s at 0.5x, 1x and 2x that rate, and the
    same requests served one at a time (one slot) on the same GPU."""
    import torch
    from paper_2603_14641_gb300 import serve
    torch.cuda.set_device(0)
    specs = C.serving_requests(count, rate_hz=1.0, seed=5)
    circs = [C.random_circuit(r.n, r.depth, 0.5, seed=r.seed) for r in specs]
    unit_t = np.array([r.arrival_s for r in specs])

    def reqs(scale):
        return [serve.Request(i, float(unit_t[i] * scale), circs[i], specs[i].shots, specs[i].seed)
                for i in range(len(specs))]

    budget = args.serve_budget_gb << 30

    def fingerprint(res):
        # records in full, samples as (shape, XOR and wrapping sum of the words); the
        # results (samples in pinned host memory) are released before the next run,
        # as a server hands them off, so the pinned-memory cache is reused
        out = {}
        for r in res:
            s = r.samples
            out[r.rid] = (r.record.tobytes(), None if s is None else
                          (s.shape, int(np.bitwise_xor.reduce(s, axis=None)) if s.size else 0,
                           int(np.add.reduce(s, axis=None, dtype=np.uint64)) if s.size else 0))
        return out

    # warm-up: a few small requests through every slot, then the whole stream once
    serve.serve(reqs(0.0)[:args.serve_slots], slots=args.serve_slots, budget_bytes=budget,
                device="cuda:0")
    serve.serve(reqs(0.0), slots=args.serve_slots, budget_bytes=budget, device="cuda:0")
    sat_res, sat, sat_st = serve.serve(reqs(0.0), slots=args.serve_slots, budget_bytes=budget,
                                       device="cuda:0")
    sat_fp = fingerprint(sat_res)
    del sat_res
    sat_rate = len(specs) / sat["makespan_s"]
    sweep_out = {}
    if sweep:
        for mult in (0.5, 1.0, 2.0):
            rate = mult * sat_rate
            res, summ, st = serve.serve(reqs(1.0 / rate), slots=args.serve_slots,
                                        budget_bytes=budget, device="cuda:0")
            summ.update({"rate_hz": rate, "peak_active": st["peak_active"],
                         "peak_bytes": st["peak_bytes"], "batches": st["batches"],
                         "batched_requests": st["batched_requests"]})
            sweep_out[f"{mult}x"] = summ
            del res
    # one request at a time: one slot and no batching
    one_res, one, _ = serve.serve(reqs(0.0), slots=1, budget_bytes=budget, device="cuda:0",
                                  batching=False)
    same = fingerprint(one_res) == sat_fp
    del one_res
    shots = sum(r.shots for r in specs)
    out = {"value": sat["shots_per_s"], "unit": "shots/s",
           "config": {"requests": len(specs), "slots": args.serve_slots,
                      "budget_bytes": budget, "shots_total": shots,
                      "n_range": [int(min(c.n for c in circs)), int(max(c.n for c in circs))],
                      "workload": "n log-uniform 100..20000, depth 100..500, shots log-uniform "
                                  "1e3..1e6, final Z-measurement of all qubits; samples returned "
                                  "to pinned host memory"},
           "saturation": sat, "saturation_rate_hz": sat_rate,
           "saturation_batches": {"batches": sat_st["batches"],
                                  "batched_requests": sat_st["batched_requests"]},
           "sweep": sweep_out,
           "one_at_a_time": one, "speedup_vs_one_at_a_time": one["makespan_s"] / sat["makespan_s"],
           "results_identical_alone_and_mixed": bool(same)}
    if cpu:
        out["cpu_baseline"] = serve_cpu_baseline(specs, circs)
    return out


def run_serve(args):
    r = serve_measure(args, args.serve_count, sweep=True, cpu=not args.no_cpu_baseline)
    out = {"metric": "served many-shot sampling: p50/p99 latency and shots/s under a Poisson "
                     "request stream (continuous batching vs one request at a time)",
           "n_gpus": 1, "higher_is_better": True, "data": "synthetic", "dtype": "u64", **r}
    print(json.dumps(out))


def serve_cpu_baseline(specs, circs, shots: int = 20000):
    """The oracle serving the smallest request: its reference shot plus
    `shots` frame-sampled shots, timed on one core (shots/s)."""
    from oracle import oracle as O
    i = min(range(len(specs)), key=lambda j: circs[j].n)
    c = circs[i]
    t0 = time.perf_counter()
    _, ref, _ = O.run_circuit(c, seed=specs[i].seed)
    O.frames(c, ref, shots, seed=specs[i].seed + 1)
    dt = time.perf_counter() - t0
    return {"value": shots / dt, "unit": "shots/s", "cores": 1, "kind": "oracle",
            "sample": f"request {i} (n={c.n}, depth {c.n_layers}): reference shot + {shots} "
                      f"frame shots, {dt:.1f} s of CPU"}


def run_l2probe(args):
    """Evidence for the fused-depth question at 180k qubits (L2-resident slabs):
    the in-place read-modify-write rate of a buffer that fits L2 against one
    that does not. A slab of generator words evolved through many layers in L2
    moves each layer's column words through L2 instead of HBM, so fusing can
    save at most 1 - (HBM rate / L2 rate) of the gate phase, before the grid-wide
    barrier every layer would need. Timed with CUDA events over back-to-back
    in-place XORs of int64 buffers (torch elementwise kernels; a probe of the
    memory system, not of this library's kernels)."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    out = {}
    for mb in (16, 32, 64, 96, 8192):
        n = mb * (1 << 20) // 8
        a = torch.randint(-2**62, 2**62, (n,), dtype=torch.int64, device=dev)
        b = torch.randint(-2**62, 2**62, (n,), dtype=torch.int64, device=dev)
        reps = max(3, int(4096 // mb))
        for _ in range(3):
            a.bitwise_xor_(b)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(reps):
            a.bitwise_xor_(b)
        e.record()
        torch.cuda.synchronize()
        ms = s.elapsed_time(e) / reps
        # bytes: read a and b, write a
        out[f"{mb}MB"] = {"ms": ms, "tb_per_s": 3 * n * 8 / (ms / 1e3) / 1e12, "reps": reps}
        del a, b
    hbm = out["8192MB"]["tb_per_s"]
    l2 = max(out[k]["tb_per_s"] for k in ("16MB", "32MB", "64MB"))
    res = {"metric": "in-place read-modify-write rate, L2-resident vs HBM-resident buffers",
           "unit": "TB/s", "rates": out, "l2_over_hbm": l2 / hbm,
           "max_gate_phase_saving_from_l2_slabs": 1 - hbm / l2,
           "note": "upper bound on what fused depth through L2-resident slabs can save in the "
                   "180k gate phase (before per-layer grid barriers)"}
    print(json.dumps(res))


def run_dsmemprobe(args):
    """Evidence for the second form of fused depth at 180k qubits (one 64-row
    word slice of every column spread over the shared memory of a 16-CTA
    cluster, layers separated by cluster barriers): the rate of random 16-byte
    read-modify-writes in another CTA's shared memory, against the CTA's own,
    and the cost of a cluster barrier (probes/dsmem_probe.cu, built by
    build.py; a probe of the memory system, not of this library's kernels)."""
    import subprocess
    from paper_2603_14641_gb300 import build as B
    exe = [p for p in B.build_probes() if p.endswith("dsmem_probe")][0]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        raise SystemExit(f"dsmem_probe failed: {r.stdout}{r.stderr}")
    rows = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    print(json.dumps({"metric": "distributed shared memory: random 16-byte read-modify-write rate "
                                "and cluster barrier cost", "unit": "TB/s", "configs": rows,
                      "note": "a 64-row slice of the 180k tableau needs 16 CTAs (16 n bytes); a "
                              "two-qubit gate moves 32 B of a column held by another CTA 15 times "
                              "in 16, one layer ends at a cluster barrier"}))


def run_reference(args):
    """The oracle as it stands on one host core, for the same metric: each step
    evolves `cpu_rows` sampled generator rows of the 180k workload's circuit
    through its first `cpu_layers` layers. ms_per_step is the measured time of
    that step; value is the full-tableau gate rate it implies (gates x rows /
    2n per second: the oracle's gate cost is proportional to the rows it
    updates, Sec. 2.4), and the time the whole tableau would take is reported
    under "extrapolated"."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    circ = C.random_circuit(args.n, max(args.cpu_layers, 1), 0.4, seed=3)
    for _ in range(args.warmup):
        oracle_gate_rate(circ, rows=16, layers=1)
    t0 = time.perf_counter()
    gates = 0
    sample_s = 0.0
    full_s = 0.0
    for k in range(args.steps):
        rate, dt, g = oracle_gate_rate(circ, rows=args.cpu_rows, layers=args.cpu_layers, seed=k)
        gates += g
        sample_s += dt
        full_s += g / rate
    wall = time.perf_counter() - t0
    value = gates / full_s
    out = {"metric": METRIC, "value": value, "unit": "gates/s", "impl": "reference",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": sample_s * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
           "config": {"workload": workload_label("n180k_d1000", args.n, args.depth, args.n),
                      "step": f"oracle gate rules on {args.cpu_rows} sampled generator rows of "
                              f"{2 * args.n} through the first {args.cpu_layers} layers "
                              f"(measured); value = gates x rows / 2n per second"},
           "extrapolated": {"full_tableau_ms_per_step": full_s * 1e3 / args.steps,
                            "basis": "measured sample time x 2n / rows (not measured)"},
           "cpu_baseline": {"value": value, "unit": "gates/s", "cores": 1, "kind": "oracle",
                            "sample": f"{args.cpu_rows} of {2 * args.n} rows x {args.cpu_layers} "
                                      f"layers per step, {wall:.1f} s wall in total"},
           "e2e": {"value": value, "unit": "gates/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="n180k",
                    choices=sorted(WORKLOADS) + ["batch", "serve", "l2probe", "dsmemprobe",
                                                 "inverse"])
    ap.add_argument("--serve-count", type=int, default=64)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=int, default=96)
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--no-fusion", action="store_true")
    ap.add_argument("--n", type=int, default=N_QUBITS)
    ap.add_argument("--depth", type=int, default=DEPTH)
    ap.add_argument("--measurements", type=int, default=512)
    ap.add_argument("--full-final", action="store_true",
                    help="time one step with all n final measurements (warm-up steps use the short program)")
    ap.add_argument("--shots", type=int, default=1024)
    ap.add_argument("--noise", type=float, default=1e-3,
                    help="circuit-level Pauli noise of the extra noisy-sampling phase (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the compact serving, batch and inverse-tableau summaries")
    ap.add_argument("--no-full-job", action="store_true",
                    help="skip the once-timed complete 180k program (all final measurements)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=256)
    ap.add_argument("--cpu-layers", type=int, default=40)
    ap.add_argument("--cpu-prefix-n", type=int, default=20_000,
                    help="qubits of the whole-tableau oracle prefix in cpu_baseline")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "l2probe":
        run_l2probe(args)
    elif args.workload == "dsmemprobe":
        run_dsmemprobe(args)
    elif args.workload == "inverse":
        print(json.dumps({"metric": "inverse-tableau mode (Alg. 1) vs CHP on the 10,000-qubit "
                                    "workload", **inverse_mode_summary()}))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
