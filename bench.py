"""Throughput benchmark of the fused D3Q14/D3Q18 MRT step on one GB300.

Workload: lid-driven cube 128^3, D3Q18, FP32 populations, lid 0.05 along x
on y+, Re = 1000 (nu = U L / Re), synthetic state from rest.  One bench step
is one pass of the whole hot path: 1000 fused lattice updates of the domain
followed by the FP64 reductions that give the residual of Eq.
cavity_creterion (its 1000-step interval), so the default 20 timed steps are
the 20000 updates of the workload.  The timed steps run back to back (the
151 MB population buffer is larger than the 129 MB L2, and each update
sweeps all of it), bracketed by CUDA events on the stream the kernels run
on.  The update is also timed one by one after an L2 flush, as a secondary
figure.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
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

from paper_1503_03337_gb300 import inputs  # noqa: E402

FLUSH_BYTES = 256 << 20
STORAGE_BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20,
                    help="timed bench steps (each: residual-interval lattice updates + one "
                         "FP64 residual reduction)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--Q", type=int, default=18)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--storage", default="f32")
    ap.add_argument("--rounding", default="nearest", choices=("nearest", "stochastic"),
                    help="16-bit stores of the main workload")
    ap.add_argument("--Re", type=float, default=1000.0)
    ap.add_argument("--residual-interval", type=int, default=1000)
    ap.add_argument("--precision-n", type=int, default=256,
                    help="cube side of the storage-precision comparison (0: skip); its "
                         "buffers are several times larger than L2, so steps run back to back")
    ap.add_argument("--precision-steps", type=int, default=200)
    ap.add_argument("--large-n", type=int, default=1024,
                    help="cube side of the large-domain timing (D3Q18 FP16, Q*N >= 2^31, the "
                         "step's 64-bit-offset kernels; 0: skip)")
    ap.add_argument("--porous-n", type=int, default=256,
                    help="cube side of the solid-node (porous medium) timing (0: skip)")
    ap.add_argument("--reduction-n", type=int, default=256,
                    help="cube side of the FP64-reduction timing (D3Q18 FP32 cavity; 0: skip)")
    ap.add_argument("--flushed-steps", type=int, default=400,
                    help="steps timed one by one after an L2 flush (secondary figure)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--kernel-updates", type=int, default=2000,
                    help="back-to-back updates timed without reductions for the step "
                         "kernel's own launch duration (roofline)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tune-trials", type=int, default=16)
    ap.add_argument("--launch", default="",
                    help="fixed launch shape bx,by,cells_per_thread instead of the autotuner")
    ap.add_argument("--workload", default="cavity128",
                    choices=("cavity128", "batch256", "serving", "half_cavity97"),
                    help="cavity128: the fused-step throughput line (default); batch256: "
                         "256 uneven domains, batched vs one launch per domain; serving: "
                         "request trace, batched server vs one domain at a time; "
                         "half_cavity97: the Sec. 4.3 half cavity 97x97x49 at Re 3200, "
                         "throughput and the MRT / LBGK stability comparison")
    ap.add_argument("--batch-steps", type=int, default=200,
                    help="steps of the 256-domain batch comparison in the default run (0: skip)")
    ap.add_argument("--serving-requests", type=int, default=100,
                    help="requests of the serving comparison in the default run (0: skip)")
    ap.add_argument("--batch-domains", type=int, default=256,
                    help="batch256 workload: number of domains of the seed-0 draw")
    ap.add_argument("--batch-lmax", type=int, default=160,
                    help="batch256 workload: largest side of the draw (24 .. lmax)")
    ap.add_argument("--batch-repeats", type=int, default=3)
    ap.add_argument("--requests", type=int, default=100)
    ap.add_argument("--max-steps", type=int, default=1000)
    ap.add_argument("--saturation-cells", type=int, default=8 << 20,
                    help="serving: admit while the active domains hold fewer cells")
    return ap.parse_args()


METRIC = "D3Q%d MRT fused-step GLUPS (lattice updates/s) and HBM-roofline fraction"


def workload_name(a):
    return "lid-driven cavity %d^3 D3Q%d %s Re=%g lid=0.05" % (a.n, a.Q, a.storage.upper(), a.Re)


# ---- clocks ------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi samples (every 50 ms) of SM clock and throttle reasons:
    one nvidia-smi process runs around the region, and only samples whose
    own timestamps fall between __enter__ and __exit__ are kept."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.samples = []
        self._p = None
        self._t = None
        self.t0 = self.t1 = None

    def _read(self):
        for line in self._p.stdout:
            self.lines.append(line)

    def __enter__(self):
        try:
            self._p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            time.sleep(0.3)  # nvidia-smi is up before the region starts
        except Exception:
            self._p = None
        self.t0 = time.time()
        return self

    def __exit__(self, *exc):
        self.t1 = time.time()
        if self._p is None:
            return
        time.sleep(0.2)
        self._p.terminate()
        try:
            self._p.wait(timeout=5)
        except Exception:
            self._p.kill()
        self._t.join(timeout=5)
        import datetime
        for line in self.lines:
            parts = [p.strip() for p in line.strip().split(",")]
            if len(parts) < 8:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                continue
            if self.t0 <= ts <= self.t1:
                self.samples.append(parts[1:])

    def summary(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if s[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples),
                "sampling": "nvidia-smi -lms 50 during the timed region"}


# ---- ncu-derived traffic --------------------------------------------------------

def kernel_source_hash():
    """Hash of the sources the single-domain step kernel is built from."""
    h = hashlib.sha256()
    for name in ("lbm_model.cuh", "lbm_factored.cuh", "lbm_collide.cuh", "lbm_kernels.cuh",
                 "lbm_launch.cuh", "lbm_step.cu", "lbm_step_impl.cuh", "lbm_step_q14.cu",
                 "lbm_step_q18.cu", "lbm_step_q14h.cu", "lbm_step_q18h.cu", "lbm_step_q14b.cu",
                 "lbm_step_q18b.cu"):
        p = os.path.join(ROOT, "paper_1503_03337_gb300", "csrc", name)
        with open(p, "rb") as fh:
            h.update(os.path.basename(p).encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(Q, storage, n):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "step_kernel_dram_traffic.txt")
    if not os.path.exists(path):
        return None
    src_hash = kernel_source_hash()
    key = "Q%d %s %d^3" % (Q, storage, n)
    cur = None
    for line in open(path):
        line = line.strip()
        if line.startswith("source_hash:"):
            cur = line.split(":", 1)[1].strip()
        elif line.startswith(key + ":") and cur == src_hash:
            try:
                return float(line.split(":", 1)[1].split()[0])
            except ValueError:
                return None
    return None


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            v = json.load(fh).get("hbm_gbs")
        if v:
            return float(v), "measured"
    except Exception:
        pass
    return 6800.0, "fallback"


# ---- multi-GPU aggregation (replicas) ------------------------------------------

def max_over_ranks(x, dist, device):
    """The largest of every rank's x (a time): the whole job is as slow as
    its slowest replica.  dist is torch.distributed or None (one process)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, cells, steps, seconds):
    """GLUPS of the whole job: `world` independent replicas, each updating
    `cells` cells `steps` times, in `seconds` (the max over ranks)."""
    return world * cells * steps / seconds / 1e9


# ---- GPU leg -----------------------------------------------------------------------

def storage_error(Q, storage, rounding, launch, stream):
    """max |u - u_FP64| / U of one storage and launch on the two accuracy
    cases (FP64 storage agrees with the oracle to 1e-12 relative)."""
    from paper_1503_03337_gb300 import lbm

    def run(case, steps, st, rnd, lau):
        h = lbm.lbm_create(case.Q, case.nx, case.ny, case.nz, st, stream)
        try:
            lbm.lbm_set_geometry(h, case.faces, case.u_wall)
            lbm.lbm_set_params(h, nu=case.nu, force=case.force, force_period=case.period,
                               rounding=rnd)
            if lau is not None:
                lbm.lbm_set_launch(h, *lau)
            u0 = None if case.init_u is None else np.ascontiguousarray(case.init_u)
            lbm.lbm_init_equilibrium(h, u0, None, 0)
            lbm.lbm_step(h, steps)
            return lbm.read_u(h, case.nx, case.ny, case.nz)
        finally:
            lbm.lbm_destroy(h)

    out = {}
    cav = inputs.cavity(Q, 32, 400.0, U=0.05)
    lau = launch if storage != "f64" else None
    ref = run(cav, 1000, "f64", 0, None)
    out["cavity32"] = float(np.max(np.abs(run(cav, 1000, storage, rounding, lau) - ref)) / 0.05)
    pul = inputs.pulsatile(Q, 64, 8, 1000, 4.0, 1.555e-4, u_ref=0.03)  # max |u| 0.03
    ref = run(pul, 1000, "f64", 0, None)
    out["pulsatile64"] = float(np.max(np.abs(run(pul, 1000, storage, rounding, lau) - ref))
                               / 0.03)
    out["within_1e-3"] = bool(max(out["cavity32"], out["pulsatile64"]) <= 1e-3)
    return out


def run_gpu(a, rank, world, dist):
    import torch

    from paper_1503_03337_gb300 import lbm

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    lbm.load()
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    flush_sink = torch.empty(1, dtype=torch.float32, device="cuda")

    def open_case(Q, storage, residual_interval):
        case = inputs.cavity(Q, a.n, a.Re, U=0.05, storage=storage)
        h = lbm.lbm_create(Q, case.nx, case.ny, case.nz, storage, sp)
        lbm.lbm_set_geometry(h, case.faces, case.u_wall)
        rounding = lbm.LBM_ROUND_STOCHASTIC if a.rounding == "stochastic" else 0
        lbm.lbm_set_params(h, nu=case.nu, residual_interval=residual_interval,
                           rounding=rounding)
        lbm.lbm_init_equilibrium(h)
        if a.launch:
            block = tuple(int(v) for v in a.launch.split(","))
            lbm.lbm_set_launch(h, *block)
        else:
            block, _ = lbm.lbm_autotune(h, a.tune_trials)  # restores the state it used
        return case, h, block

    def timed_steps(h, K, interval):
        """Per-step event times (ms); reduction steps reported separately."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(K)]
        red = []
        n0 = lbm.lbm_get_step(h)
        for k in range(K):
            flush.fill_(float(k))
            flush_sink.copy_(flush.sum().reshape(1))
            ev[k][0].record(stream)
            lbm.lbm_step(h, 1)
            ev[k][1].record(stream)
            if interval and (n0 + k + 1) % interval == 0:
                red.append(k)
        return ev, red

    # --- main workload: back-to-back bench steps ------------------------------------
    # The population buffer (151 MB for D3Q18 FP32 at 128^3) is larger than
    # the 129 MB L2 and every update sweeps all of it, so consecutive updates
    # find nothing useful in L2 (an ncu capture of steady-state updates reads
    # 149 MB and writes 147-153 MB from/to DRAM per update).  A bench step is
    # `interval` updates plus the FP64 residual reduction that lbm_step queues
    # at the end of the interval.
    interval = max(1, a.residual_interval)
    case, h, block = open_case(a.Q, a.storage, interval)
    cells = case.cells
    bytes_per_update = 2 * a.Q * STORAGE_BYTES[a.storage]
    lbm.lbm_step(h, max(3, a.warmup) * interval)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        t0 = time.perf_counter()
        e0.record(stream)
        lbm.lbm_step(h, a.steps * interval)
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms = e0.elapsed_time(e1)
    updates = a.steps * interval
    stats = lbm.lbm_read_stats(h)
    residual = (lbm.lbm_residual(h, lbm.LBM_RESIDUAL_CAVITY) if stats.prev_step >= 0 else None)
    # the step kernel's own launch duration: back-to-back updates with no
    # reduction in between (the dominant kernel of the step, for the roofline)
    lbm.lbm_set_params(h, nu=case.nu, residual_interval=0,
                       rounding=lbm.LBM_ROUND_STOCHASTIC if a.rounding == "stochastic" else 0)
    ku = max(2, a.kernel_updates + (a.kernel_updates & 1))
    e0.record(stream)
    lbm.lbm_step(h, ku)
    e1.record(stream)
    torch.cuda.synchronize()
    kernel_ms = e0.elapsed_time(e1) / ku
    # the reduction alone (kernel + final pass + synchronisation), same domain
    for _ in range(2):
        lbm.lbm_reductions(h)
    e0.record(stream)
    for _ in range(10):
        lbm.lbm_reductions(h)
    e1.record(stream)
    torch.cuda.synchronize()
    reduce_ms = e0.elapsed_time(e1) / 10
    # the same update timed one by one with the L2 flushed in between (a
    # 256 MiB write, then a read of it, so that the flush leaves only clean
    # lines and the timed update pays no write-back of the flush)
    fl_steps = max(2, a.flushed_steps)
    ev, _ = timed_steps(h, fl_steps, 0)
    torch.cuda.synchronize()
    fl_ms = statistics.mean(s0.elapsed_time(s1) for s0, s1 in ev)
    flushed = {"glups": round(cells / (fl_ms * 1e-3) / 1e9, 3), "updates": fl_steps,
               "ms_per_update": round(fl_ms, 6),
               "note": "per-update CUDA events, 256 MiB L2 flush (write then read) before each "
                       "update, outside the events"}
    lbm.lbm_destroy(h)

    total_ms = max_over_ranks(total_ms, dist, "cuda")
    glups = replica_throughput(world, cells, updates, total_ms * 1e-3)
    peak, peak_kind = measured_hbm_peak()
    achieved = bytes_per_update * cells / (kernel_ms * 1e-3) / 1e9
    traffic = recorded_traffic(a.Q, a.storage, a.n)
    share = {"step_kernel": round(kernel_ms * interval / (total_ms / a.steps), 4),
             "reduction": round(reduce_ms / (total_ms / a.steps), 4)}

    # --- e2e through the C-ABI with host buffers ---------------------------------
    # per step: equilibrium from pinned host (u, p), `interval` updates and the
    # residual reduction, the velocity field back to pinned host memory
    e2e = None
    if a.e2e_steps > 0:
        case_e, he, _ = open_case(a.Q, a.storage, interval)
        N = case_e.cells
        u0 = torch.zeros(3 * N, dtype=torch.float64).pin_memory()
        p0 = torch.zeros(N, dtype=torch.float64).pin_memory()
        uout = torch.empty(3 * N, dtype=torch.float64).pin_memory()
        lbm.lbm_init_equilibrium(he, u0, p0, 0)
        lbm.lbm_step(he, 2)
        lbm.lbm_read_fields(he, lbm.LBM_FIELD_U, uout, lbm.LBM_DTYPE_F64, 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.e2e_steps):
            lbm.lbm_init_equilibrium(he, u0, p0, 0)
            lbm.lbm_step(he, interval)
            lbm.lbm_read_fields(he, lbm.LBM_FIELD_U, uout, lbm.LBM_DTYPE_F64, 0)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        lbm.lbm_destroy(he)
        el = max_over_ranks(el, dist, "cuda")
        e2e = {"value": replica_throughput(world, N, interval * a.e2e_steps, el),
               "unit": "GLUPS",
               "h2d_bytes_per_step": 4 * N * 8, "d2h_bytes_per_step": 3 * N * 8,
               "lattice_updates_per_step": interval,
               "calls": "lbm_init_equilibrium(host u,p) + lbm_step(%d, residual every %d) + "
                        "lbm_read_fields(U -> host)" % (interval, interval)}

    # --- storage precision at a size far above L2: back-to-back steps ------------------
    precision = {}
    if a.precision_n > 0 and a.precision_steps > 0 and rank == 0:
        variants = (("f32", 0), ("f16", 0), ("f16", 1), ("bf16", 1))
        for Q in (14, 18, 26):
            for st, rnd in variants:
                cp = inputs.cavity(Q, a.precision_n, a.Re, U=0.05, storage=st)
                hp = lbm.lbm_create(Q, cp.nx, cp.ny, cp.nz, st, sp)
                lbm.lbm_set_geometry(hp, cp.faces, cp.u_wall)
                lbm.lbm_set_params(hp, nu=cp.nu, residual_interval=0, rounding=rnd)
                lbm.lbm_init_equilibrium(hp)
                bp, _ = lbm.lbm_autotune(hp, 4)
                lbm.lbm_step(hp, 10)
                k = a.precision_steps + (a.precision_steps & 1)
                e0.record(stream)
                lbm.lbm_step(hp, k)
                e1.record(stream)
                torch.cuda.synchronize()
                tp = e0.elapsed_time(e1) / k
                lbm.lbm_destroy(hp)
                bpu = 2 * Q * STORAGE_BYTES[st]
                key = "D3Q%d_%s%s" % (Q, st, "_sr" if rnd else "")
                precision[key] = {
                    "rounding": "stochastic" if rnd else "nearest",
                    "launch": list(bp),
                    "glups": round(cp.cells / (tp * 1e-3) / 1e9, 3),
                    "hbm_gbs": round(bpu * cp.cells / (tp * 1e-3) / 1e9, 1),
                    "frac_of_measured_hbm": round(bpu * cp.cells / (tp * 1e-3) / 1e9 / peak, 4)}
                precision[key]["error"] = storage_error(Q, st, rnd, tuple(bp), sp)
            f32 = precision["D3Q%d_f32" % Q]["glups"]
            for st, rnd in variants[1:]:
                key = "D3Q%d_%s%s" % (Q, st, "_sr" if rnd else "")
                precision[key]["vs_f32"] = round(precision[key]["glups"] / f32, 3)
        precision["note"] = ("lid-driven cavity %d^3, %d back-to-back steps after 10, one event "
                             "pair; population buffers %d-%d MB, all far above the 129 MB L2.  "
                             "error: max|u - u_FP64| / U with the same launch, on the 32^3 "
                             "cavity (Re 400, 1000 steps) and the 64x64x8 oscillating channel "
                             "(T 1000, eta 4, one period from rest); the FP64 "
                             "storage run matches the oracle to 1e-12"
                             % (a.precision_n, a.precision_steps,
                                2 * 14 * a.precision_n ** 3 >> 20,
                                4 * 26 * a.precision_n ** 3 >> 20))

    # --- one large domain: Q*N >= 2^31, the step's 64-bit-offset kernels ------------
    large = {}
    if a.large_n > 0 and rank == 0:
        cl = inputs.cavity(18, a.large_n, a.Re, U=0.05, storage="f16")
        hl = lbm.lbm_create(18, cl.nx, cl.ny, cl.nz, "f16", sp)
        try:
            lbm.lbm_set_geometry(hl, cl.faces, cl.u_wall)
            lbm.lbm_set_params(hl, nu=cl.nu, residual_interval=0)
            lbm.lbm_init_equilibrium(hl)
            bl, _ = lbm.lbm_autotune(hl, 2)
            lbm.lbm_step(hl, 4)
            kl = 20
            e0.record(stream)
            lbm.lbm_step(hl, kl)
            e1.record(stream)
            torch.cuda.synchronize()
            tl = e0.elapsed_time(e1) / kl
        finally:
            lbm.lbm_destroy(hl)
        lbytes = 2 * 18 * 2 * cl.cells
        large = {"workload": "lid-driven cavity %d^3 D3Q18 FP16 (%.1f GB of populations, "
                             "Q*N = %.3g >= 2^31)" % (a.large_n, 18 * 2 * cl.cells / 1e9,
                                                      18.0 * cl.cells),
                 "launch": list(bl), "steps": kl,
                 "glups": round(cl.cells / (tl * 1e-3) / 1e9, 3),
                 "hbm_gbs": round(lbytes / (tl * 1e-3) / 1e9, 1),
                 "frac_of_measured_hbm": round(lbytes / (tl * 1e-3) / 1e9 / peak, 4)}

    # --- solid nodes: a porous medium of random spheres, 256^3 --------------------
    porous = {}
    if a.porous_n > 0 and rank == 0:
        pc = inputs.porous_spheres(18, a.porous_n, storage="f32")
        hp = lbm.lbm_create(18, pc.nx, pc.ny, pc.nz, "f32", sp)
        lbm.lbm_set_geometry(hp, pc.faces, pc.u_wall)
        lbm.lbm_set_params(hp, nu=pc.nu, force=pc.force)
        lbm.lbm_set_solid(hp, pc.solid)
        lbm.lbm_init_equilibrium(hp)
        bp, _ = lbm.lbm_autotune(hp, 4)
        lbm.lbm_step(hp, 10)
        k = 200
        e0.record(stream)
        lbm.lbm_step(hp, k)
        e1.record(stream)
        torch.cuda.synchronize()
        tp = e0.elapsed_time(e1) / k
        lbm.lbm_destroy(hp)
        fluid = int(pc.cells - int(pc.solid.sum()))
        # fluid cells move 2Q values and read their link word; solid cells
        # read their link word only
        pbytes = fluid * (2 * 18 * 4 + 4) + (pc.cells - fluid) * 4
        porous = {"workload": "periodic %d^3 box of random spheres (radius 6, seed 0), "
                              "D3Q18 FP32, body force" % a.porous_n,
                  "fluid_fraction": round(fluid / pc.cells, 4), "launch": list(bp),
                  "glups_fluid": round(fluid / (tp * 1e-3) / 1e9, 3),
                  "hbm_gbs": round(pbytes / (tp * 1e-3) / 1e9, 1),
                  "frac_of_measured_hbm": round(pbytes / (tp * 1e-3) / 1e9 / peak, 4),
                  "bytes_model": "fluid cell 2*18*4 + 4 B (link word), solid cell 4 B"}

    # the step kernels plus, per residual check, the reduction kernel and its
    # final pass
    # --- FP64 reductions (residuals, mass, flux, max) at a size far above L2 -----------
    reductions = {}
    if a.reduction_n > 0 and rank == 0:
        cr = inputs.cavity(18, a.reduction_n, a.Re, U=0.05, storage="f32")
        hr = lbm.lbm_create(18, cr.nx, cr.ny, cr.nz, "f32", sp)
        lbm.lbm_set_geometry(hr, cr.faces, cr.u_wall)
        lbm.lbm_set_params(hr, nu=cr.nu, residual_interval=0)
        lbm.lbm_init_equilibrium(hr)
        lbm.lbm_step(hr, 4)
        for _ in range(3):  # snapshot allocated and filled
            lbm.lbm_reductions(hr)
        kr = 20
        e0.record(stream)
        for _ in range(kr):
            lbm.lbm_reductions(hr)
        e1.record(stream)
        torch.cuda.synchronize()
        tr = e0.elapsed_time(e1) / kr
        lbm.lbm_destroy(hr)
        rbytes = cr.cells * (18 * 4 + 2 * 3 * 8)
        reductions = {"workload": "lid-driven cavity %d^3 D3Q18 F32" % a.reduction_n,
                      "ms_per_call": round(tr, 4),
                      "algorithmic_bytes": rbytes,
                      "hbm_gbs": round(rbytes / (tr * 1e-3) / 1e9, 1),
                      "frac_of_measured_hbm": round(rbytes / (tr * 1e-3) / 1e9 / peak, 4),
                      "note": "lbm_reductions (reduction kernel, final pass, host synchronisation) "
                              "timed with CUDA events over %d calls; bytes: 18 FP32 populations "
                              "read, FP64 u snapshot read and written, per cell" % kr}

    launches = a.steps * (interval + 2)  # updates + reduction kernel and final pass
    res = {
        "metric": METRIC % a.Q,
        "value": round(glups, 4),
        "unit": "GLUPS",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": round(total_ms / a.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": a.storage,
        "data": "synthetic (lid-driven cavity from rest)",
        "config": {"workload": workload_name(a), "grid": [a.n, a.n, a.n], "Q": a.Q,
                   "storage": a.storage, "Re": a.Re, "lid_velocity": 0.05,
                   "step": "%d fused lattice updates + one FP64 residual reduction "
                           "(Eq. cavity_creterion interval)" % interval,
                   "lattice_updates": updates,
                   "l2": "inputs larger than L2: back-to-back steps over a %d MB population "
                         "buffer (L2 129 MB); see flushed_per_step for the same step timed one "
                         "by one after an L2 flush" % (bytes_per_update * cells // 2 // 10**6),
                   "launch": {"block": [block[0], block[1]], "cells_per_thread": block[2]},
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "wall_s_timed_region": round(wall, 4)},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": bytes_per_update * cells,
                     "kernel_ms": round(kernel_ms, 6),
                     "kernel_timing": "CUDA events over %d back-to-back updates without "
                                      "reductions, on the launch stream" % ku},
        "time_share": share,
        "reduction_ms": round(reduce_ms, 4),
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "residual_last": {"step": stats.step, "cavity": residual},
        "precision": precision,
        "reductions": reductions,
        "solid_nodes": porous,
        "large_domain": large,
        "flushed_per_step": flushed,
    }
    return res


# ---- CPU oracle ----------------------------------------------------------------------

def oracle_rate(Q, n, Re, storage, budget_s=15.0, max_steps=50):
    import oracle
    case = inputs.cavity(Q, n, Re, U=0.05, storage=storage)
    g = oracle.make_grid(Q, case.nx, case.ny, case.nz, case.faces, case.u_wall)
    prm = oracle.make_params(oracle.rates(Q, oracle.s_nu_of(case.nu)))
    f = oracle.init_equilibrium(g)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    f = oracle.run(g, prm, f, 0, 1, nthreads=threads)
    t1 = time.perf_counter() - t0
    steps = int(max(1, min(max_steps, budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    oracle.run(g, prm, f, 1, steps, nthreads=threads)
    el = time.perf_counter() - t0
    return {"value": case.cells * steps / el / 1e9, "unit": "GLUPS", "cores": min(threads, n),
            "kind": "oracle",
            "sample": "%d steps of the %d^3 D3Q%d cavity in FP64 (oracle, OpenMP over z)"
                      % (steps, n, Q)}


def oracle_reference_arm(a, budget_s=90.0):
    """The oracle as it stands on the host cores: W + K steps of the cavity
    workload, each step one lattice update of a 128 x 128 x nz_s slab of the
    cube (same boundary kinds and per-cell work), nz_s sized so the whole
    run fits in about budget_s."""
    import oracle
    threads = os.cpu_count() or 1
    full = inputs.cavity(a.Q, a.n, a.Re, U=0.05, storage=a.storage)
    # calibrate on one slab step
    probe = inputs.cavity(a.Q, a.n, a.Re, U=0.05, storage=a.storage, nz=min(a.n, 8))
    g = oracle.make_grid(a.Q, probe.nx, probe.ny, probe.nz, probe.faces, probe.u_wall)
    prm = oracle.make_params(oracle.rates(a.Q, oracle.s_nu_of(full.nu)))
    f = oracle.init_equilibrium(g)
    t0 = time.perf_counter()
    oracle.run(g, prm, f, 0, 1, nthreads=threads)
    per_layer = (time.perf_counter() - t0) / probe.nz
    total_steps = max(1, a.steps) + max(0, a.warmup)
    nz_s = int(max(1, min(a.n, budget_s / (total_steps * max(per_layer, 1e-9)))))
    case = inputs.cavity(a.Q, a.n, a.Re, U=0.05, storage=a.storage, nz=nz_s)
    g = oracle.make_grid(a.Q, case.nx, case.ny, case.nz, case.faces, case.u_wall)
    f = oracle.init_equilibrium(g)
    f = oracle.run(g, prm, f, 0, max(0, a.warmup), nthreads=threads)
    t0 = time.perf_counter()
    oracle.run(g, prm, f, max(0, a.warmup), max(1, a.steps), nthreads=threads)
    el = time.perf_counter() - t0
    return {"value": case.cells * max(1, a.steps) / el / 1e9, "unit": "GLUPS",
            "cores": min(threads, nz_s), "kind": "oracle",
            "sample": "each step one FP64 oracle update of a %dx%dx%d slab of the %d^3 D3Q%d "
                      "cavity (walls on all six faces of the slab, lid on y+)"
                      % (a.n, a.n, nz_s, a.n, a.Q)}


def batch_compare(steps, repeats=3, chunk=10, n_domains=256, lmax=160):
    """The seed-0 draw of 256 independent cavities/ducts (sides 24-160,
    Q14/Q18, FP32/FP16): `steps` steps of every domain batched (grouped
    launches in CUDA graphs, and the persistent cooperative kernel) against
    one launch per domain per step, each timed `repeats` times with CUDA
    events on the launch stream."""
    import torch

    from paper_1503_03337_gb300 import lbm
    lbm.load()
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    cases = [inputs.batch_case(d) for d in inputs.batch_draw(n_domains, seed=0,
                                                            lmax=max(24, lmax))]
    cells = sum(c.cells for c in cases)
    steps = max(2, steps + (steps & 1))
    runs = {"grouped": [], "persistent": [], "one_launch_per_domain": []}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return cells * steps / (e0.elapsed_time(e1) * 1e-3) / 1e9

    with torch.cuda.stream(stream):
        b = lbm.lbm_batch_create(n_domains, 0, sp)
        for c in cases:
            slot = lbm.lbm_batch_add(b, c.Q, c.nx, c.ny, c.nz, c.storage, c.faces, c.u_wall,
                                     nu=c.nu, force=c.force)
            lbm.lbm_batch_init_equilibrium(b, slot)
        hs = []
        for c in cases:
            h = lbm.lbm_create(c.Q, c.nx, c.ny, c.nz, c.storage, sp)
            lbm.lbm_set_geometry(h, c.faces, c.u_wall)
            lbm.lbm_set_params(h, nu=c.nu, force=c.force)
            lbm.lbm_set_launch(h, 64, 2, 1)
            lbm.lbm_init_equilibrium(h)
            hs.append(h)
        for _ in range(repeats):
            for mode, persistent in (("grouped", 0), ("persistent", 1)):
                lbm.lbm_batch_set_launch(b, 64, 2, persistent)
                lbm.lbm_batch_step(b, 3 * chunk, chunk)  # graphs captured, warm
                runs[mode].append(timed(lambda: lbm.lbm_batch_step(b, steps, chunk)))

            def one_by_one():
                for _ in range(steps):
                    for h in hs:
                        lbm.lbm_step(h, 1)
            for h in hs:
                lbm.lbm_step(h, 2)
            runs["one_launch_per_domain"].append(timed(one_by_one))
        lbm.lbm_batch_destroy(b)
        for h in hs:
            lbm.lbm_destroy(h)
    out = {k: {"glups": round(statistics.median(v), 3), "min": round(min(v), 3),
               "max": round(max(v), 3)} for k, v in runs.items()}
    base = out["one_launch_per_domain"]
    return {"workload": "%d domains (seed 0), sides 24-%d, Q14/Q18, FP32/FP16, %d cells"
                        % (n_domains, max(24, lmax), cells),
            "steps": steps, "chunk": chunk, "repeats": repeats, "modes": out,
            "speedup_grouped": round(out["grouped"]["glups"] / base["glups"], 3),
            "speedup_persistent": round(out["persistent"]["glups"] / base["glups"], 3),
            "beats_beyond_spread": out["grouped"]["min"] > base["max"]}


def run_batch256(a):
    r = batch_compare(max(2, a.steps), repeats=a.batch_repeats, n_domains=a.batch_domains,
                      lmax=a.batch_lmax)
    return {"metric": "batched GLUPS, 256 uneven domains",
            "value": r["modes"]["grouped"]["glups"], "unit": "GLUPS", "n_gpus": 1,
            "steps": r["steps"], "higher_is_better": True,
            "data": "synthetic (seed-0 draw of cavities and ducts)",
            "config": {"workload": r["workload"], "chunk": r["chunk"]}, "batch": r}


def request_error(case, steps, u, stream):
    """max |u - u_ref| / U of a delivered field against the same request run
    alone with higher-precision storage (FP16 -> FP32, FP32 -> FP64) for the
    same number of steps."""
    from paper_1503_03337_gb300 import lbm
    ref = "f32" if case.storage in ("f16", "bf16") else "f64"
    h = lbm.lbm_create(case.Q, case.nx, case.ny, case.nz, ref, stream)
    try:
        lbm.lbm_set_geometry(h, case.faces, case.u_wall, case.edge)
        lbm.lbm_set_params(h, nu=case.nu, force=case.force, force_period=case.period)
        lbm.lbm_init_equilibrium(h)
        lbm.lbm_step(h, steps)
        ur = lbm.read_u(h, case.nx, case.ny, case.nz)
    finally:
        lbm.lbm_destroy(h)
    return float(np.max(np.abs(u - ur)) / case.u_ref), ref


def serving_compare(requests, max_steps, repeats=3, saturation_cells=8 << 20,
                    check_cells=96 ** 3, lmin=32, lmax=256):
    """The seed-0 Poisson trace (200/s) served by the continuous-batching
    loop and by one domain at a time, from the same arrival times, `repeats`
    times each.  Then every request of at most `check_cells` cells from the
    first batched run is checked against its requested accuracy: its field
    against the same request run alone in higher precision."""
    import torch

    from paper_1503_03337_gb300 import lbm
    from paper_1503_03337_gb300.serving import (BatchBackend, SequentialBackend, Server,
                                                summarize)
    lbm.load()
    stream = torch.cuda.Stream()
    trace = inputs.request_trace(requests, rate=200.0, seed=0, lmin=lmin, lmax=lmax,
                                 max_steps=max_steps)
    runs = {"batched": [], "one_at_a_time": []}
    first = None
    with torch.cuda.stream(stream):
        # one untimed pass of the whole trace through each backend first:
        # allocator pools, graph capture and module loading then belong to
        # no timed repeat
        for be in (BatchBackend(256, 150 << 30, stream.cuda_stream),
                   SequentialBackend(stream.cuda_stream)):
            Server(be, check_every=100, tol=1e-8, chunk=50,
                   max_active_cells=saturation_cells).run(trace)
            torch.cuda.synchronize()
            be.close()
        for rep in range(repeats):
            for name in ("batched", "one_at_a_time"):
                be = (BatchBackend(256, 150 << 30, stream.cuda_stream) if name == "batched"
                      else SequentialBackend(stream.cuda_stream))
                keep = name == "batched" and rep == 0
                t0 = time.perf_counter()
                res = Server(be, check_every=100, tol=1e-8, chunk=50,
                             max_active_cells=saturation_cells, keep_fields=keep).run(trace)
                torch.cuda.synchronize()
                wall = time.perf_counter() - t0
                be.close()
                runs[name].append(summarize(res, wall))
                if keep:
                    first = res
        checks = []
        for r in trace:
            case = inputs.request_case(r)
            o = first[r.rid]
            if case.cells > check_cells or o.u is None:
                continue
            err, ref = request_error(case, o.steps, o.u, stream.cuda_stream)
            checks.append({"rid": r.rid, "kind": r.kind, "L": r.L, "storage": case.storage,
                           "tol": r.tol, "err": err, "ref": ref})
    med = {}
    for name, rs in runs.items():
        med[name] = {k: statistics.median(x[k] for x in rs) for k in ("p50_s", "p99_s", "glups")}
        med[name].update({"p99_s_range": [min(x["p99_s"] for x in rs), max(x["p99_s"] for x in rs)],
                          "glups_range": [min(x["glups"] for x in rs), max(x["glups"] for x in rs)],
                          "converged": rs[0]["converged"], "requests": rs[0]["requests"]})
    b, s = med["batched"], med["one_at_a_time"]
    met = [c for c in checks if c["err"] <= c["tol"]]
    return {"workload": "%d requests, Poisson 200/s (seed 0), cavity/duct/pulsatile, sides "
                        "%d-%d, Q14/Q18, FP32 or FP16 by requested accuracy, residual 1e-8 "
                        "or %d steps, 150 GB budget, admission while < %d active cells"
                        % (requests, lmin, lmax, max_steps, saturation_cells),
            "repeats": repeats, "batched": b, "one_at_a_time": s,
            "glups_beats_beyond_spread": b["glups_range"][0] > s["glups_range"][1],
            "p99_beats_beyond_spread": b["p99_s_range"][1] < s["p99_s_range"][0],
            "accuracy": {"checked": len(checks), "met": len(met),
                         "max_err_over_tol": max((c["err"] / c["tol"] for c in checks),
                                                 default=None),
                         "rule": "requests of at most %d cells from the first batched run; "
                                 "error = max|u - u_ref| / U against the request run alone "
                                 "with FP32 (FP16 requests) or FP64 (FP32 requests) storage"
                                 % check_cells,
                         "worst": sorted(checks, key=lambda c: -c["err"] / c["tol"])[:3]}}


def run_serving(a):
    r = serving_compare(a.requests, a.max_steps, repeats=3,
                        saturation_cells=a.saturation_cells)
    return {"metric": "serving p50/p99 time-to-converged and aggregate GLUPS",
            "value": round(r["batched"]["glups"], 3), "unit": "GLUPS",
            "higher_is_better": True, "n_gpus": 1,
            "data": "synthetic Poisson trace (seed 0, 200/s)",
            "config": {"workload": r["workload"]}, "serving": r}


def run_half_cavity(a):
    """The cavity of Sec. 4.3 on its grid: the 97 x 97 x 49 half cavity
    (symmetry face at z = 1/2, lid 0.1 with the corner velocities), Re 3200,
    D3Q18 FP32.  Throughput of a.steps back-to-back steps under CUDA events,
    then the stability comparison: 50000 steps each with the MRT rates and
    with every rate 1/tau (LBGK), checked every 1000 steps."""
    import torch

    from paper_1503_03337_gb300 import lbm
    lbm.load()
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    case = inputs.half_cavity(18, 97, 3200.0, U=0.1, storage="f32", ku_lid=True)
    s_lbgk = 1.0 / (3.0 * case.nu + 0.5)
    lbgk = dict(s_c=s_lbgk, s_e=s_lbgk, s_q=s_lbgk, s_pi=s_lbgk, s_t=s_lbgk)

    def open_case(rates, interval):
        h = lbm.lbm_create(case.Q, case.nx, case.ny, case.nz, case.storage, sp)
        lbm.lbm_set_geometry(h, case.faces, case.u_wall, case.edge)
        lbm.lbm_set_params(h, nu=case.nu, residual_interval=interval, **rates)
        lbm.lbm_autotune(h)
        lbm.lbm_init_equilibrium(h)
        return h

    out = {}
    with torch.cuda.stream(stream):
        # the 33 MB population buffer fits in L2: each timed step follows a
        # 256 MiB flush (write, then read), outside its event pair
        steps = max(2, min(a.steps, 400) + (min(a.steps, 400) & 1))
        flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
        sink = torch.empty(1, dtype=torch.float32, device="cuda")
        h = open_case({}, 0)
        lbm.lbm_step(h, max(4, a.warmup))
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for k in range(steps):
            flush.fill_(float(k))
            sink.copy_(flush.sum().reshape(1))
            ev[k][0].record(stream)
            lbm.lbm_step(h, 1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps
        launch = lbm.lbm_get_launch(h)
        lbm.lbm_destroy(h)
        for name, rates in (("mrt", {}), ("lbgk", lbgk)):
            h = open_case(rates, 1000)
            diverged = None
            for k in range(0, 50000, 1000):
                try:
                    lbm.lbm_step(h, 1000)
                    st = lbm.lbm_reductions(h)
                except lbm.LBMError:
                    diverged = k + 1000
                    break
                if st.nonfinite:
                    diverged = k + 1000
                    break
            out[name] = {"steps": 50000, "diverged_by_step": diverged,
                         "max_abs_u": None if diverged else st.max_abs_u}
            lbm.lbm_destroy(h)
    peak, peak_kind = measured_hbm_peak()
    bytes_per_step = 2 * case.Q * 4 * case.cells
    achieved = bytes_per_step / (ms * 1e-3) / 1e9
    return {"metric": "half-cavity GLUPS and MRT/LBGK stability at Re 3200",
            "value": round(case.cells / (ms * 1e-3) / 1e9, 3), "unit": "GLUPS",
            "higher_is_better": True, "n_gpus": 1, "steps": steps, "ms_per_step": ms,
            "dtype": "f32", "data": "synthetic (half cavity from rest)",
            "config": {"workload": "half cavity 97x97x49 D3Q18 F32 Re=3200 lid=0.1, "
                                   "symmetry face z+, lid corner velocities 0.3/1.0",
                       "launch": list(launch),
                       "l2": "population buffer 33 MB fits in L2: each timed step follows "
                             "a 256 MiB L2 flush (write then read), outside its events"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                         "peak_kind": peak_kind},
            "stability": out}


def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if a.impl == "reference":
        if rank != 0:
            return
        cb = oracle_reference_arm(a)
        steps_each = max(1, a.steps)
        out = {"metric": METRIC % a.Q,
               "value": cb["value"], "unit": "GLUPS", "n_gpus": 0, "steps": steps_each,
               "warmup": a.warmup, "ms_per_step": None, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic (lid-driven cavity from rest)",
               "config": {"workload": workload_name(a), "grid": [a.n] * 3, "Q": a.Q},
               "impl": "reference", "cpu_baseline": cb,
               "e2e": {"value": cb["value"], "unit": "GLUPS", "h2d_bytes_per_step": 0,
                       "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return
    if a.workload != "cavity128":
        fn = {"batch256": run_batch256, "serving": run_serving,
              "half_cavity97": run_half_cavity}[a.workload]
        if rank == 0:
            print(json.dumps(fn(a)))
        return
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        td.init_process_group("nccl")
        dist = td
    res = run_gpu(a, rank, world, dist)
    if rank == 0 and world == 1:
        # the batched (256 uneven domains) and serving (request trace) halves
        # of the metric, on the same GPU after the single-domain line
        if a.batch_steps > 0:
            res["batch"] = batch_compare(a.batch_steps)
        if a.serving_requests > 0:
            res["serving"] = serving_compare(a.serving_requests, a.max_steps,
                                             saturation_cells=a.saturation_cells)
            # the same trace with small domains only (sides 32-96), where one
            # domain alone cannot fill the device
            res["serving_small"] = serving_compare(a.serving_requests, a.max_steps,
                                                   saturation_cells=a.saturation_cells,
                                                   lmin=32, lmax=96)
    if rank == 0:
        if not a.no_cpu_baseline and world == 1:
            res["cpu_baseline"] = oracle_rate(a.Q, a.n, a.Re, a.storage)
        elif not a.no_cpu_baseline:
            res["cpu_baseline"] = None
        print(json.dumps(res))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
