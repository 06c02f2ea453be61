#!/usr/bin/env python3
"""Benchmark: Barnes-Hut potential at every cell of an AMR mesh on GB300.

One step = the whole hot path on one synthetic field already resident in HBM:
bh_build (block keys, tree topology, FP64 moments and quadrupoles) +
bh_potential (opening radii for theta, walk).  Default workload: the Maclaurin
spheroid (eccentricity 0.9, 2,039,808 cells, 3 AMR levels at the surface),
per-cell opening test at theta 0.75 with the quadrupole term, binary32 walk
with compensated sum -- the largest theta (in steps of 0.01) that keeps the
max relative error against the direct sum below 1e-3 over every cell (9.1e-4,
`accuracy_all_cells`; 0.72 gives 7.0e-4, 0.74 8.0e-4, 0.76 1.02e-3).

Prints one JSON line (rank 0).  `value` is cells/s of the device-resident
step over all ranks; `e2e` the same through bh_solve_host with pinned host
buffers (copies inside the timed region); `vs_plain` the same step with the
plain monopole walk at the largest theta where it meets the same 1e-3 bound
against the direct sum over every cell (0.24: 9.7e-4; 0.25 gives 1.02e-3);
`accuracy_all_cells` compares both with the exhaustive direct sum over all
cells (the library at a theta below which no node is accepted), the CPU
leg with the oracle's direct sum on a sample;
`roofline` puts the walk against the FP32 ALU peak (128 FP32 lanes/SM x SMs x
measured SM clock), counting algorithmic FP32 operations (8 per interaction
with a cell or a monopole node, 20 per quadrupole node interaction, 7 per
opening test; counted by the library's own counting walk); `cpu_baseline`
times the CPU oracle on a bounded sample of targets.

--impl reference times the CPU oracle alone (the reference arm).
With torchrun, every rank solves its own copy of the field (replicas).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
# the batched arm's 64 fields (meshgen.batch_fields), as its walk profile names them
BATCH_WORKLOAD = "batched64_16-128_seeds5000-5063"
sys.path.insert(0, ROOT)

FP32_LANES_PER_SM = 128
FLOP_PER_INTERACTION = 8        # 3 sub, 1 mul + 2 fma for d^2, 1 mul m*rsqrt, 1 add (+1 MUFU)
FLOP_PER_QUAD_INTERACTION = 20  # the above, with 9 ops for d^T Q d / 2 and 3 more for
                                # rinv (M + q rinv^4) in place of the m*rsqrt product
FLOP_PER_TEST = 7
# periodic boundaries (App. A): the minimum-image wrap adds 3 ops per component
# (the y and z ones shared by the x-neighbour pair: 6 per target); chi from the
# table costs 3 axes x 11 ops (index, fraction, three weights; y and z shared
# by the pair) + 39 for the weighted 27-point sum = 61 per target, plus 1 add
FLOP_PER_TEST_PERIODIC = FLOP_PER_TEST + 6
FLOP_PER_INTERACTION_PERIODIC = FLOP_PER_INTERACTION + 61 + 1
FLOP_PER_CELL_WRAP = 6
FLOP_PER_SELF_IMAGE = 61 + 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="maclaurin",
                    choices=["maclaurin", "cloud_core", "uniform_sphere", "batched", "learned"])
    ap.add_argument("--theta", type=float, default=None,
                    help="default 0.75 (the quadrupole headline), 0.7 with --monopole, "
                         "--vote or --periodic; 0.5 for --workload batched; 0.8 for "
                         "--workload learned")
    ap.add_argument("--monopole", action="store_true",
                    help="plain monopole nodes (default: with the quadrupole term)")
    ap.add_argument("--vote", action="store_true",
                    help="the paper's warp vote instead of the per-cell test")
    ap.add_argument("--periodic", action="store_true",
                    help="periodic boundaries (Ewald field, App. A); monopole nodes")
    ap.add_argument("--ewald-grid", type=int, default=64,
                    help="Ewald table points per half box (periodic)")
    ap.add_argument("--plain-theta", type=float, default=None,
                    help="theta of the plain monopole walk timed for vs_plain "
                         "(default 0.24; 0.4 for --workload learned)")
    ap.add_argument("--train-fields", type=int, default=200,
                    help="--workload learned: seeded training fields")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--mlp-gates", default="0.3,0.4,0.5",
                    help="--workload learned: gates s_min of the network also timed (comma "
                         "list; empty for none)")
    ap.add_argument("--walk-shape", default=None,
                    help="W,P,T[,L]: the walk's launch shape (warps per CTA, target pairs "
                         "per lane, groups per take; 0 = plain grid; L = 1: the groups longest "
                         "walk first, the order bh_autotune makes, run untimed before) "
                         "instead of the shape bh_autotune picks")
    ap.add_argument("--all-cells-limit", type=int, default=4_200_000,
                    help="largest field (cells) whose potentials are compared with the "
                         "exhaustive direct sum over every cell (N^2 work)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle sample")
    return ap.parse_args()


def workload(name):
    from paper_1509_07370_gb300 import meshgen as mg
    if name in ("maclaurin", "learned"):
        return mg.maclaurin()
    if name == "cloud_core":
        return mg.cloud_core()
    return mg.uniform_sphere()


# ----------------------------------------------------------------- clocks --
class ClockSampler:
    """SM clock and clock-event (throttle) reasons during the timed region.

    Polls NVML (the driver's libnvidia-ml, through ctypes) from a thread
    every `period_s` (default 2 ms); if NVML cannot be loaded, falls back to
    `nvidia-smi --query-gpu ... -lms 100`.  Only reads; changes nothing."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clocks-event reason bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index: int, period_s: float = 0.002):
        self.index = index
        self.period = period_s
        self.proc = None
        self.thread = None
        self.samples = []           # (sm_mhz, reason bits)
        self.max_mhz = None
        self.path = None

    def _nvml(self):
        import ctypes
        lib = None
        for name in ("libnvidia-ml.so.1", "libnvidia-ml.so"):
            try:
                lib = ctypes.CDLL(name)
                break
            except OSError:
                lib = None
        if lib is None or lib.nvmlInit_v2() != 0:
            return None
        h = ctypes.c_void_p()
        found = False
        try:  # the CUDA device by its PCI address (NVML numbers every GPU of the host)
            import torch
            pr = torch.cuda.get_device_properties(self.index)
            bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
            found = lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) == 0
        except (ImportError, AttributeError, RuntimeError):
            found = False
        if not found and lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index),
                                                           ctypes.byref(h)) != 0:
            return None
        try:
            reasons = lib.nvmlDeviceGetCurrentClocksEventReasons
        except AttributeError:
            reasons = lib.nvmlDeviceGetCurrentClocksThrottleReasons
        return lib, h, reasons

    def _poll(self, lib, h, reasons):
        import ctypes
        clk = ctypes.c_uint()
        bits = ctypes.c_ulonglong()
        mx = ctypes.c_uint()
        if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:  # NVML_CLOCK_SM = 1
            self.max_mhz = float(mx.value)
        while not self.stop.is_set():
            if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0:
                r = reasons(h, ctypes.byref(bits))
                self.samples.append((float(clk.value), int(bits.value) if r == 0 else 0))
            time.sleep(self.period)

    def __enter__(self):
        import threading
        nv = None
        try:
            nv = self._nvml()
        except (OSError, AttributeError):
            nv = None
        if nv is not None:
            self.stop = threading.Event()
            self.thread = threading.Thread(target=self._poll, args=nv, daemon=True)
            self.thread.start()
            return self
        try:
            fd, self.path = tempfile.mkstemp(prefix=f"bh_clocks_{self.index}_", suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.thread is not None:
            self.stop.set()
            self.thread.join(timeout=5)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.thread is not None:
            if not self.samples:
                return None
            sm = [c for c, _ in self.samples]
            reasons = sorted({n for _, b in self.samples for bit, n in self.REASONS.items()
                              if b & bit})
            return {"sm_mhz": float(np.median(sm)),
                    "sm_max_mhz": self.max_mhz if self.max_mhz else float(max(sm)),
                    "samples": len(sm), "period_ms": 1e3 * self.period, "source": "nvml",
                    "reasons": reasons}
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "samples": len(sm), "period_ms": 100.0, "source": "nvidia-smi",
                "reasons": sorted(reasons)}


# ----------------------------------------------------- captured traffic --
def captured_traffic(workload_name, theta, mode):
    """DRAM bytes per walk launch from the committed ncu summary of this walk,
    if that capture is of this workload and of the walk source as it is now."""
    import hashlib
    import re
    profile, files = {
        "quadrupole": ("walk_queue_quadrupole_theta0.75_maclaurin_2M.md",
                       ("bh_walk.cu", "bh_walk_common.cuh")),
        "monopole": ("walk_queue_monopole_theta0.24_maclaurin_2M.md",
                     ("bh_walk.cu", "bh_walk_common.cuh")),
        "periodic64": ("walk_periodic_theta0.7_maclaurin_2M.md",
                       ("bh_walk_periodic.cu", "bh_ewald.cuh", "bh_walk_common.cuh")),
        "batched_monopole": ("walk_queue_batched64_theta0.5.md",
                             ("bh_walk.cu", "bh_walk_common.cuh")),
    }.get(mode, (None, None))
    if profile is None:
        return None
    try:
        txt = open(os.path.join(ROOT, "profiles", profile)).read()
        csrc = os.path.join(ROOT, "paper_1509_07370_gb300", "csrc")
        src = b"".join(open(os.path.join(csrc, f), "rb").read() for f in files)
    except OSError:
        return None
    sha = re.search(r"source_sha256: ([0-9a-f]{64})", txt)
    wl = re.search(r"workload: (\S+) theta=([0-9.]+) mode=(\w+)", txt)
    tb = re.search(r"dram_bytes_per_launch: (\d+)", txt)
    if not (sha and wl and tb):
        return None
    if sha.group(1) != hashlib.sha256(src).hexdigest():
        return None
    if wl.group(1) != workload_name or float(wl.group(2)) != float(theta):
        return None
    if wl.group(3) != mode:
        return None
    return int(tb.group(1))


# ------------------------------------------------------------ CPU oracle --
def oracle_leg(w, theta, cpu_seconds, phi_gpu=None, quad=False, plain=None, periodic=False,
               ewald_grid=64, worst=None):
    """Times the CPU oracle (tree + FP64 moments in full, walk on a sample of
    targets) and extrapolates to cells/s for the whole field."""
    from oracle import oracle as O
    rho = w.density.astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    tree = O.Tree(w.mesh.level, w.mesh.ijk, rho, w.mesh.box_lo, w.mesh.box_len)
    if quad:
        tree.quadrupoles()
    if periodic:
        O.ewald_table(ewald_grid)
    t_build = time.perf_counter() - t0

    def walk(targets, threads=0):
        if periodic:
            return tree.walk_periodic(theta, targets=targets, threads=threads, ng=ewald_grid)
        return tree.walk(theta, targets=targets, quad=quad, threads=threads)

    rng = np.random.default_rng(1234)
    n = w.ncells
    probe = rng.choice(n, min(n, 2000), replace=False)
    per = walk_time_per_cell(walk, rng, n)
    kind = "periodic (Ewald table), monopole" if periodic else (
        "quadrupole" if quad else "monopole")
    if t_build + per * n <= 1.5 * cpu_seconds:
        # whole steps (tree build + walk of every cell), repeated to ~cpu_seconds
        tg = np.arange(n)
        steps, t_total, t_walk = 0, 0.0, 0.0
        while steps == 0 or t_total < cpu_seconds:
            t0 = time.perf_counter()
            tr = O.Tree(w.mesh.level, w.mesh.ijk, rho, w.mesh.box_lo, w.mesh.box_len)
            t1 = time.perf_counter()        # (the oracle's walk reduces the quadrupoles)
            if periodic:
                ref, ni, nt = tr.walk_periodic(theta, targets=tg, ng=ewald_grid)
            else:
                ref, ni, nt = tr.walk(theta, targets=tg, quad=quad)
            t2 = time.perf_counter()
            t_walk += t2 - t1
            t_total += t2 - t0
            steps += 1
            del tr
        k = n
        value = n * steps / t_total
        sample = (f"{steps} whole steps: tree + FP64 moments{' + quadrupoles' if quad else ''}"
                  f" and the per-cell walk of all {n} cells ({kind}, theta {theta}), "
                  f"{t_total:.2f} s in all ({t_walk:.2f} s in the walk call"
                  f"{', quadrupoles included' if quad else ''}); no extrapolation")
    else:
        # a whole step would take too long: the walk of a random sample, scaled
        k = int(min(n, max(len(probe), cpu_seconds / max(per, 1e-9))))
        tg = np.sort(rng.choice(n, k, replace=False))
        t0 = time.perf_counter()
        ref, ni, nt = walk(tg)
        t_walk = time.perf_counter() - t0
        value = n / (t_build + t_walk * (n / k))
        sample = (f"tree + FP64 moments of all {n} cells ({t_build:.2f} s) and the per-cell walk "
                  f"of {k} random cells (seed 1234, {kind}, theta {theta}, {t_walk:.2f} s), "
                  f"the walk time scaled by {n}/{k}: a whole step would exceed "
                  f"{1.5 * cpu_seconds:.0f} s")
    per1 = walk_time_per_cell(lambda tg: walk(tg, threads=1), rng, n)
    out = {"value": value, "unit": "cells/s", "cores": O.max_threads(), "kind": "oracle",
           "value_1core": n / (t_build + per1 * n),
           "sample": sample + "; value_1core: the per-cell walk time on one thread (timed on "
                              "2,000 and 22,000 random cells) times every cell, plus the "
                              "tree build"}
    if phi_gpu is not None and periodic:
        # the periodic field has zero mean and changes sign: errors relative
        # to its largest magnitude; a smaller direct sample (each direct
        # periodic term interpolates the table)
        dt = direct_targets(w, np.random.default_rng(4321), nrandom=200, ndense=1)
        t0 = time.perf_counter()
        d = tree.direct_periodic(targets=dt, ng=ewald_grid)
        t_direct = time.perf_counter() - t0
        wd = walk(dt)[0]
        out["accuracy"] = {
            "max_err_over_max_abs_vs_oracle_walk":
                float(np.max(np.abs(phi_gpu[tg] - ref)) / np.max(np.abs(ref))),
            "max_err_over_max_abs_vs_direct":
                float(np.max(np.abs(phi_gpu[dt] - d)) / np.max(np.abs(d))),
            "oracle_walk_max_err_over_max_abs_vs_direct":
                float(np.max(np.abs(wd - d)) / np.max(np.abs(d))),
            "cells_compared": int(k), "cells_vs_direct": int(len(dt)),
            "direct_sample": "200 random cells (seed 4321) + every cell of the densest block; "
                             "direct periodic sum with the same Ewald table",
            "direct_cells_per_s": len(dt) / t_direct}
    elif phi_gpu is not None:
        dt = direct_targets(w, np.random.default_rng(4321))
        t0 = time.perf_counter()
        d = tree.direct(targets=dt)
        t_direct = time.perf_counter() - t0
        wd = walk(dt)[0]
        out["accuracy"] = {
            "max_rel_vs_oracle_walk": float(np.max(np.abs(phi_gpu[tg] / ref - 1.0))),
            "max_rel_vs_direct": float(np.max(np.abs(phi_gpu[dt] / d - 1.0))),
            "oracle_walk_max_rel_vs_direct": float(np.max(np.abs(wd / d - 1.0))),
            "cells_compared": int(k), "cells_vs_direct": int(len(dt)),
            "direct_sample": "2,000 random cells (seed 4321) + every cell of the 8 densest "
                             "blocks",
            "direct_cells_per_s": len(dt) / t_direct}
        if plain is not None:
            phi_plain, plain_theta = plain
            out["accuracy"]["plain_max_rel_vs_direct"] = float(
                np.max(np.abs(phi_plain[dt] / d - 1.0)))
            out["accuracy"]["plain_theta"] = plain_theta
        if worst is not None:
            # the all-cells check's worst cells, against the oracle's FP64 direct sum: the
            # walks' errors there and the library's own direct sum (the all-cells reference)
            cells, lib_direct = worst
            dw = tree.direct(targets=cells)
            acc = {"cells": int(len(cells)),
                   "how": "the 128 cells of largest error of each walk over every cell "
                          "(against the library's direct sum), against the oracle's FP64 "
                          "direct sum",
                   "library_direct_max_rel_vs_oracle_direct": float(
                       np.max(np.abs(lib_direct / dw - 1.0))),
                   "max_rel_vs_oracle_direct": float(np.max(np.abs(phi_gpu[cells] / dw - 1.0)))}
            if plain is not None:
                acc["plain_max_rel_vs_oracle_direct"] = float(
                    np.max(np.abs(plain[0][cells] / dw - 1.0)))
            out["accuracy"]["worst_cells_vs_oracle_direct"] = acc
    return out


def walk_time_per_cell(walk, rng, n):
    """Per-cell time of the oracle's walk on the host cores: the difference of
    two timed calls on 2,000 and 22,000 random cells, over the 20,000 cells
    between them (each call also pays fixed costs: thread start-up, and for
    the quadrupole walk one reduction of every node's quadrupole)."""
    a = rng.choice(n, min(n, 2000), replace=False)
    b = rng.choice(n, min(n, 22000), replace=False)
    walk(a[:64])                                         # start the OpenMP threads
    t0 = time.perf_counter()
    walk(a)
    ta = time.perf_counter() - t0
    t0 = time.perf_counter()
    walk(b)
    tb = time.perf_counter() - t0
    if len(b) > len(a) and tb > ta:
        return (tb - ta) / (len(b) - len(a))
    return tb / len(b)


def all_cells_error(bh, mesh, d_rho, maxlev, phis, device, stream, periodic=False,
                    ewald_grid=64, limit=4_200_000):
    """Max error of each potential in `phis` over EVERY cell against the
    exhaustive sum the library computes at theta = 2^-maxlev (maxlev = the
    deepest cell level): the smallest internal node has side 2^-(maxlev-1),
    so l/theta = 2 exceeds every box-unit distance (at most sqrt(3)) and no
    internal node is ever accepted -- every cell meets every other cell
    singly, the direct sum of Eq. 2 in binary32 with compensated summation; the
    interaction counts are checked to be N - 1 everywhere.  Relative per
    cell, or, for the zero-mean periodic field, relative to max |Phi|.
    Skipped (None) above `limit` cells (N^2 interactions)."""
    import torch
    n = 512 * len(mesh.level)
    if n > limit:
        return None
    theta = 2.0 ** -maxlev
    ref = bh.Solver(periodic=periodic, device=device.index, stream=stream)
    if periodic and ewald_grid != 64:
        ref.set_ewald(ewald_grid, 3)
    ref.build(mesh.level, mesh.ijk, d_rho)
    ni, _ = ref.walk_counts(theta)
    if int(ni.min().item()) != n - 1 or int(ni.max().item()) != n - 1:
        ref.close()
        return None
    t0 = time.perf_counter()
    d = ref.potential(theta).double()
    torch.cuda.synchronize()
    t_direct = time.perf_counter() - t0
    ref.close()
    out = {"direct": f"the library at theta 2^-{maxlev}: every pair direct (counts N-1 "
                     "checked), binary32, compensated sum", "cells": n, "direct_s": t_direct}
    worst = []
    for key, phi in phis.items():
        if phi is None:
            continue
        p = torch.as_tensor(phi, device=device)
        err = (p - d).abs() / d.abs().max() if periodic else (p / d - 1.0).abs()
        out[key] = float(err.max().item())
        worst.append(torch.topk(err, min(128, n)).indices)
    # the cells where the walks err most, for the oracle's FP64 direct sum
    if worst:
        cells = torch.unique(torch.cat(worst))
        out["_worst_cells"] = cells.cpu().numpy()
        out["_direct_at_worst"] = d[cells].cpu().numpy()
    return out


def direct_targets(w, rng, nrandom=2000, ndense=8):
    """Cells compared with the direct sum: a random sample plus every cell of
    the densest blocks (where the error of the walk tends to peak)."""
    n = w.ncells
    rnd = rng.choice(n, min(n, nrandom), replace=False)
    mean = w.density.reshape(-1, 512).mean(axis=1)
    dense = np.argsort(-mean, kind="stable")[:ndense]
    cells = (dense[:, None] * 512 + np.arange(512)[None, :]).reshape(-1)
    return np.unique(np.concatenate([rnd, cells]))


def reference_arm(args):
    """The reference arm: the CPU oracle, on the host cores, same workload and
    metric.  A step is what the GPU step computes -- the tree with FP64
    moments (and quadrupoles) and the per-cell walk of every cell -- timed
    whole, so ms_per_step is time spent.  If whole steps would take the run
    past about two and a half minutes, fewer steps are timed (`steps` says
    how many); only if a single step is longer than half of that does a step
    walk a random sample of the cells, and the rate is then the cells walked
    over the time spent."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args.workload)
    from oracle import oracle as O
    rho = w.density.astype(np.float32).astype(np.float64)
    n = w.ncells
    rng = np.random.default_rng(99)
    quad = not args.monopole
    budget = 150.0
    t0 = time.perf_counter()
    tree = O.Tree(w.mesh.level, w.mesh.ijk, rho, w.mesh.box_lo, w.mesh.box_len)
    if quad:
        tree.quadrupoles()
    t_build = time.perf_counter() - t0
    per = walk_time_per_cell(lambda tg: tree.walk(args.theta, targets=tg, quad=quad), rng, n)
    del tree
    est = t_build + per * n                                # one whole step
    warmup = min(args.warmup, 1)
    if est <= budget / 2:
        k = n
        steps = max(1, min(args.steps, int(budget / est) - warmup))
    else:
        steps, warmup = 1, 0
        k = int(max(1000, min(n, (budget / 2 - t_build) / max(per, 1e-9))))
    times = []
    for s in range(warmup + steps):
        tg = np.arange(n) if k == n else np.sort(rng.choice(n, k, replace=False))
        t0 = time.perf_counter()
        tr = O.Tree(w.mesh.level, w.mesh.ijk, rho, w.mesh.box_lo, w.mesh.box_len)
        tr.walk(args.theta, targets=tg, quad=quad)          # reduces the quadrupoles too
        if s >= warmup:
            times.append(time.perf_counter() - t0)
        del tr
    t = float(np.sum(times))
    value = k * steps / t
    what = (f"per step: tree + FP64 moments{' + quadrupoles' if quad else ''} of all {n} cells "
            + ("and the walk of every cell (a whole step)" if k == n else
               f"and the walk of {k} random cells (a whole step would take about {est:.0f} s)")
            + f"; {steps} steps timed after {warmup} untimed")
    line = {"impl": "reference", "metric": "cell potentials/sec", "value": value,
            "unit": "cells/s", "n_gpus": args.gpus, "steps": steps, "warmup": warmup,
            "ms_per_step": 1e3 * t / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "cells": n, "theta": args.theta,
                       "walk": "FP64, per-cell opening test"
                               + (", quadrupole nodes" if quad else ", monopole nodes")},
            "cpu_baseline": {"value": value, "unit": "cells/s", "cores": O.max_threads(),
                             "kind": "oracle", "sample": what},
            "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm --
def timed_steps(solver, mesh, d_rho, theta, out, steps, warmup, flush, stream, clk=None):
    """Warm-up, then `steps` timed steps (bh_build + bh_potential), each
    bracketed by CUDA events on the library's stream, L2 flushed before each.
    Returns per-step (step, build, potential) milliseconds."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            flush.zero_()
            solver.build(mesh.level, mesh.ijk, d_rho)
            solver.potential(theta, 1.0, out=out)
        stream.synchronize()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        torch.cuda.synchronize()
        if clk is not None:
            clk.__enter__()
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            solver.build(mesh.level, mesh.ijk, d_rho)
            ev[k][1].record(stream)
            solver.potential(theta, 1.0, out=out)
            ev[k][2].record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        if clk is not None:
            clk.__exit__()
    return ([e[0].elapsed_time(e[2]) for e in ev], [e[0].elapsed_time(e[1]) for e in ev],
            [e[1].elapsed_time(e[2]) for e in ev])


def batched_arm(args):
    """64 independent fields of 16^3-128^3 cells solved as one batch: one
    CUDA-graph launch per step (moments for the step's densities + walk of
    all fields), against the plain way of solving the fields one after the
    other with bh_build + bh_potential."""
    import torch
    from paper_1509_07370_gb300 import bhgrav as bh
    from paper_1509_07370_gb300 import meshgen as mg
    if int(os.environ.get("RANK", "0")) != 0:
        return
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    ws = mg.batch_fields(64)
    nb, level, ijk, lo, ln, rho = mg.concat_fields(ws)
    n = int(512 * nb.sum())
    theta = args.theta
    stream = torch.cuda.Stream(dev)
    d_rho = torch.as_tensor(rho.astype(np.float32), device=dev)
    out = torch.empty(n, dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    s = bh.Solver(device=dev.index, stream=stream)
    s.build_batch(nb, level, ijk, d_rho, lo, ln)
    wpc, npairs, ticket, longest = s.autotune(theta)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            s.solve_graph(d_rho, theta, 1.0, out)
        stream.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        clk = ClockSampler(dev.index)
        clk.__enter__()
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            s.solve_graph(d_rho, theta, 1.0, out)
            e1.record(stream)
        stream.synchronize()
        clk.__exit__()
    s.sync_status()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    value = n / (ms * 1e-3)
    phi = out.cpu().numpy()
    # the plain way: field after field (each with its own context, built once)
    solvers, offs, off = [], [], 0
    for w in ws:
        ps = bh.Solver(device=dev.index, stream=stream)
        solvers.append(ps)
        offs.append(off)
        off += w.ncells
    pouts = [torch.empty(w.ncells, device=dev) for w in ws]
    dslices = [d_rho[o:o + w.ncells] for o, w in zip(offs, ws)]
    psteps = max(3, args.steps // 4)
    with torch.cuda.stream(stream):
        for k in range(args.warmup + psteps):
            if k == args.warmup:
                flush.zero_()
                stream.synchronize()
                t0 = time.perf_counter()
                e0 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            for ps, w, d, po in zip(solvers, ws, dslices, pouts):
                ps.build(w.mesh.level, w.mesh.ijk, d, w.mesh.box_lo, w.mesh.box_len)
                ps.potential(theta, 1.0, out=po)
        e1 = torch.cuda.Event(enable_timing=True)
        e1.record(stream)
        stream.synchronize()
    p_ms = e0.elapsed_time(e1) / psteps
    p_value = n / (p_ms * 1e-3)
    # the plain way without geometry work: new densities field after field
    with torch.cuda.stream(stream):
        for k in range(args.warmup + psteps):
            if k == args.warmup:
                flush.zero_()
                stream.synchronize()
                u0 = torch.cuda.Event(enable_timing=True)
                u0.record(stream)
            for ps, d, po in zip(solvers, dslices, pouts):
                ps.update_density(d)
                ps.potential(theta, 1.0, out=po)
        u1 = torch.cuda.Event(enable_timing=True)
        u1.record(stream)
        stream.synchronize()
    u_ms = u0.elapsed_time(u1) / psteps
    same = all(np.array_equal(po.cpu().numpy(), phi[o:o + w.ncells])
               for po, o, w in zip(pouts, offs, ws))
    # end to end: density from pinned host memory, potential back to it
    h_rho = torch.from_numpy(rho.astype(np.float32)).pin_memory()
    h_out = torch.empty(n, dtype=torch.float32).pin_memory()
    ts = []
    with torch.cuda.stream(stream):
        for k in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d_rho.copy_(h_rho, non_blocking=True)
            s.solve_graph(d_rho, theta, 1.0, out)
            h_out.copy_(out, non_blocking=True)
            stream.synchronize()
            if k >= args.warmup:
                ts.append(time.perf_counter() - t0)
    e2e = {"value": n / float(np.mean(ts)), "unit": "cells/s",
           "h2d_bytes_per_step": int(h_rho.numel() * 4), "d2h_bytes_per_step": int(n * 4)}
    # the dominant kernel (the walk of all fields) alone, and its work
    with torch.cuda.stream(stream):
        wev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(5)]
        for a, b in wev:
            flush.zero_()
            a.record(stream)
            s.potential(theta, 1.0, out=out)
            b.record(stream)
        stream.synchronize()
    walk_ms = float(np.mean([a.elapsed_time(b) for a, b in wev]))
    ni, nt = s.walk_counts(theta)
    n_int = int(ni.sum(dtype=torch.int64).item())
    n_test = int(nt.sum(dtype=torch.int64).item())
    flops = FLOP_PER_INTERACTION * n_int + FLOP_PER_TEST * n_test
    clocks = clk.summary()
    sm_mhz = clocks["sm_mhz"] if clocks else 1440.0
    peak = FP32_LANES_PER_SM * torch.cuda.get_device_properties(dev).multi_processor_count \
        * sm_mhz * 1e6
    roofline = {"bound": "alu", "kernel": "bh_potential walk of all 64 fields (one launch)",
                "walk_ms": walk_ms, "achieved": flops / (walk_ms * 1e-3) / 1e12,
                "peak": peak / 1e12, "unit": "TFLOP/s", "frac": flops / (walk_ms * 1e-3) / peak,
                "traffic": captured_traffic(BATCH_WORKLOAD, theta, "batched_monopole"),
                "ops": "8 per interaction, 7 per test (monopole)",
                "interactions_per_cell": n_int / n, "tests_per_cell": n_test / n}
    cpu = None
    if not args.no_cpu_baseline:  # the oracle on the largest field of the batch
        big = int(np.argmax([w.ncells for w in ws]))
        cpu = oracle_leg(ws[big], theta, args.cpu_seconds,
                         phi[offs[big]:offs[big] + ws[big].ncells].astype(np.float64))
        cpu["sample"] = f"field {big} of the batch ({ws[big].ncells} cells): " + cpu["sample"]
    line = {"metric": "cell potentials/sec", "value": value, "unit": "cells/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "batched: 64 fields of 16^3-128^3 cells, 1-8 Gaussian blobs "
                                   "(seeds 5000-5063)", "cells": n, "fields": len(ws),
                       "field_cells": sorted({w.ncells for w in ws}), "theta": theta,
                       "walk": "binary32, compensated sum, per-cell opening test, monopole nodes",
                       "step": "one CUDA-graph launch: moments + walk of all fields",
                       "tuned_warps_per_cta": wpc, "tuned_target_pairs_per_lane": npairs,
                       "tuned_groups_per_take": ticket, "tuned_longest_first": longest,
                       "l2": "flushed between steps"},
            "vs_plain": {"how": "the same fields one after the other: bh_build + bh_potential",
                         "value": p_value, "ms_per_step": p_ms, "speedup": value / p_value,
                         "identical_potentials": bool(same),
                         "without_geometry_work": {
                             "how": "field after field: bh_update_density + bh_potential",
                             "value": n / (u_ms * 1e-3), "ms_per_step": u_ms,
                             "speedup": value / (n / (u_ms * 1e-3))}},
            "roofline": roofline, "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu,
            # per graph launch: largest-mass pass, k_blocks, k_upper_tree (the
            # rest of the blocks and the top tree), opening radii, walk
            "gpu_launches": 5 * args.steps}
    print(json.dumps(line), flush=True)
    for ps in solvers:
        ps.close()
    s.close()


def learned_oracle_leg(w, theta, wts, plain_theta, phi, cpu_seconds):
    """The CPU oracle's learned walk (FP64, same bf16-rounded weights) timed on
    a sample of targets, and the max relative errors against the direct sum of
    the learned walk and of the plain monopole walk at both thetas."""
    from oracle import oracle as O
    rho = w.density.astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    tree = O.Tree(w.mesh.level, w.mesh.ijk, rho, w.mesh.box_lo, w.mesh.box_len)
    tree.quadrupoles()
    t_build = time.perf_counter() - t0
    rng = np.random.default_rng(4321)
    n = w.ncells
    probe = rng.choice(n, 200, replace=False)
    tree.walk_learned(theta, wts, targets=probe[:16])
    t0 = time.perf_counter()
    tree.walk_learned(theta, wts, targets=probe)
    per = (time.perf_counter() - t0) / len(probe)
    k = int(min(n, max(len(probe), cpu_seconds / max(per, 1e-9))))
    tg = np.sort(rng.choice(n, k, replace=False))
    t0 = time.perf_counter()
    ref = tree.walk_learned(theta, wts, targets=tg)
    t_walk = time.perf_counter() - t0
    dt = direct_targets(w, np.random.default_rng(4321))
    d = tree.direct(targets=dt)

    def rel(a):
        return float(np.max(np.abs(a[dt] / d - 1.0)))
    acc = {"learned_max_rel_vs_direct": rel(phi["learned"]),
           "plain_max_rel_vs_direct": rel(phi["plain"]),
           "plain_same_theta_max_rel_vs_direct": rel(phi["same"]),
           "learned_max_abs_vs_oracle_learned": float(np.max(np.abs(phi["learned"][tg] - ref))),
           "learned_max_rel_vs_oracle_learned": float(np.max(np.abs(phi["learned"][tg] / ref - 1))),
           "theta": theta, "plain_theta": plain_theta,
           "cells_compared": int(k), "cells_vs_direct": int(len(dt)),
           "direct_sample": "2,000 random cells (seed 4321) + every cell of the 8 densest "
                            "blocks"}
    return {"value": n / (t_build + t_walk * n / k), "unit": "cells/s",
            "cores": O.max_threads(), "kind": "oracle",
            "sample": f"tree+FP64 moments+quadrupoles of all {n} cells; learned walk (FP64 MLP) "
                      f"of {k} random cells (seed 4321, theta {theta}) extrapolated to {n}; "
                      f"build {t_build:.2f}s, walk {t_walk:.2f}s",
            "accuracy": acc}


def learned_arm(args):
    """Learned residual correction on the Maclaurin spheroid (2,039,808 cells):
    the walk at theta 0.8 whose accepted nodes' terms are corrected by the
    MLP, against the plain monopole walk at theta 0.4 and, for the gain, at
    0.8.  The network is first trained on the GPU (untimed, reported) from
    the accepted pairs of seeded spheroid fields."""
    import torch
    from paper_1509_07370_gb300 import bhgrav as bh
    from paper_1509_07370_gb300 import learned as L
    if int(os.environ.get("RANK", "0")) != 0:
        return
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    t0 = time.perf_counter()
    x, z = L.make_dataset(nfields=args.train_fields, theta=args.theta, device=local)
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    wts, hist = L.train(x, z, seed=0)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    npairs = int(z.numel())
    del x, z

    w = workload("learned")
    n = w.ncells
    mesh = w.mesh
    rho32 = np.ascontiguousarray(w.density.reshape(-1), dtype=np.float32)
    d_rho = torch.as_tensor(rho32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    res = {}
    phi = {}
    clk = ClockSampler(local)
    for key, theta, learned, steps in (("learned", args.theta, True, args.steps),
                                       ("plain", args.plain_theta, False, args.steps),
                                       ("same", args.theta, False, max(5, args.steps // 3))):
        s = bh.Solver(learned=learned, device=local, stream=stream)
        if learned:
            s.set_mlp(wts)
        out = torch.empty(n, dtype=torch.float32, device=dev)
        st, bt, wt = timed_steps(s, mesh, d_rho, theta, out, steps, args.warmup, flush, stream,
                                 clk if learned else None)
        ni, nt, nc = s.walk_counts(theta, with_cells=True)
        res[key] = {"theta": theta, "steps": steps, "ms_per_step": float(np.mean(st)),
                    "value": n / (float(np.mean(st)) * 1e-3),
                    "phases_ms": {"build": float(np.mean(bt)), "potential": float(np.mean(wt))},
                    "interactions": int(ni.sum(dtype=torch.int64).item()),
                    "cell_interactions": int(nc.sum(dtype=torch.int64).item()),
                    "tests": int(nt.sum(dtype=torch.int64).item())}
        phi[key] = out.double().cpu().numpy()
        if learned:
            wts_dev = s.get_mlp().astype(np.float64)
            _, nn, maxlev = s.tree_size()
            e2e = None
            if not args.no_e2e:
                h_rho = torch.from_numpy(rho32).pin_memory().numpy()
                h_out = torch.empty(n, dtype=torch.float32).pin_memory().numpy()
                for _ in range(max(1, args.warmup)):
                    s.solve_host(mesh.level, mesh.ijk, h_rho, theta, 1.0, h_out)
                ts = []
                for _ in range(args.steps):
                    flush.zero_()
                    torch.cuda.synchronize()
                    t1 = time.perf_counter()
                    s.solve_host(mesh.level, mesh.ijk, h_rho, theta, 1.0, h_out)
                    ts.append(time.perf_counter() - t1)
                e2e = {"value": n / float(np.mean(ts)), "unit": "cells/s",
                       "h2d_bytes_per_step": int(rho32.nbytes + mesh.level.nbytes
                                                 + mesh.ijk.nbytes),
                       "d2h_bytes_per_step": int(h_out.nbytes)}
        s.close()
    # the gate: the network only for accepted nodes with s = l/d >= s_min
    gates = [float(g) for g in args.mlp_gates.split(",") if g.strip()] if args.mlp_gates else []
    gate_sweep = []
    if gates:
        s = bh.Solver(learned=True, device=local, stream=stream)
        s.set_mlp(wts)
        with torch.cuda.stream(stream):
            s.build(mesh.level, mesh.ijk, d_rho)
        out = torch.empty(n, dtype=torch.float32, device=dev)
        for g in gates:
            s.set_mlp_gate(g)
            ts = []
            with torch.cuda.stream(stream):
                for k in range(args.warmup + max(5, args.steps // 3)):
                    flush.zero_()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    s.potential(args.theta, 1.0, out=out)
                    e1.record(stream)
                    stream.synchronize()
                    if k >= args.warmup:
                        ts.append(e0.elapsed_time(e1))
            phi[f"gate_{g}"] = out.double().cpu().numpy()
            gate_sweep.append({"s_min": g, "potential_ms": float(np.median(ts)),
                               "speedup_vs_plain": res["plain"]["phases_ms"]["potential"]
                               / float(np.median(ts))})
        s.close()
    L_ = res["learned"]
    walk_s = L_["phases_ms"]["potential"] * 1e-3
    n_node = L_["interactions"] - L_["cell_interactions"]
    mlp_flops = 2 * (10 * 64 + 64 * 64 + 64) * n_node      # algorithmic MACs x 2
    gelu_ops = 128 * 9 * n_node                             # 128 GELUs of 9 FP32 ops
    walk_ops = (FLOP_PER_INTERACTION * L_["interactions"] + FLOP_PER_TEST * L_["tests"]
                + gelu_ops)
    clocks = clk.summary()
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = clocks["sm_mhz"] if clocks else 1440.0
    alu_peak = FP32_LANES_PER_SM * props.multi_processor_count * sm_mhz * 1e6
    bf16_peak = measured_peak("bf16_tflops") * 1e12
    all_cells = all_cells_error(
        bh, mesh, d_rho, maxlev,
        {"learned_max_rel_vs_direct": phi["learned"], "plain_max_rel_vs_direct": phi["plain"],
         "plain_same_theta_max_rel_vs_direct": phi["same"],
         **{f"gate_{g}_max_rel_vs_direct": phi[f"gate_{g}"] for g in gates}}, dev, stream,
        limit=args.all_cells_limit)
    if all_cells is not None:
        for e in gate_sweep:
            e["max_rel_vs_direct_all_cells"] = all_cells.pop(f"gate_{e['s_min']}_max_rel_vs_direct",
                                                             None)
    if all_cells is not None:  # (the worst cells go to the oracle in the main arm only)
        all_cells.pop("_worst_cells", None)
        all_cells.pop("_direct_at_worst", None)
    cpu = None
    if not args.no_cpu_baseline:
        cpu = learned_oracle_leg(w, args.theta, wts_dev, args.plain_theta, phi, args.cpu_seconds)
    line = {
        "metric": "cell potentials/sec", "value": L_["value"], "unit": "cells/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": L_["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w.name + " learned", "cells": n, "nodes": nn,
                   "theta": args.theta,
                   "walk": "binary32, compensated sum, per-cell opening test, monopole nodes times "
                           "(1 + s^2 MLP(x)); MLP 10-64-64-1 GELU, bf16 weights and "
                           "activations, FP32 accumulate (mma.sync m16n8k16)",
                   "training": {"fields": args.train_fields, "pairs": npairs,
                                "epochs": len(hist), "loss_first_last": [hist[0], hist[-1]],
                                "data_s": t_data, "train_s": t_train, "theta": args.theta},
                   "moments": "f64", "l2": "flushed between steps (256 MiB write)"},
        "phases_ms": L_["phases_ms"],
        "walk_work": {"interactions_per_cell": L_["interactions"] / n,
                      "node_interactions_per_cell": n_node / n,
                      "tests_per_cell": L_["tests"] / n},
        "roofline": {"bound": "alu", "kernel": "bh_potential (s2 prep + learned walk)",
                     "achieved": walk_ops / walk_s / 1e12, "peak": alu_peak / 1e12,
                     "unit": "TFLOP/s", "frac": walk_ops / walk_s / alu_peak, "traffic": None,
                     "peak_basis": f"{FP32_LANES_PER_SM} FP32 lanes x "
                                   f"{props.multi_processor_count} SMs x {sm_mhz:.0f} MHz",
                     "ops": "8 per interaction, 7 per test, 128 x 9 per MLP evaluation (GELU)",
                     "tensor": {"mlp_flops": mlp_flops,
                                "achieved": mlp_flops / walk_s / 1e12,
                                "peak": bf16_peak / 1e12,
                                "frac": mlp_flops / walk_s / bf16_peak,
                                "peak_basis": "measured bf16 dense (burst)"}},
        "vs_plain": {"theta": args.plain_theta, "walk": "binary32, compensated sum, per-cell, monopole",
                     **{k: v for k, v in res["plain"].items() if k != "theta"},
                     "speedup": L_["value"] / res["plain"]["value"]},
        "vs_same_theta": {"theta": args.theta, "walk": "the plain walk, no network",
                          **{k: v for k, v in res["same"].items() if k != "theta"},
                          "speedup": L_["value"] / res["same"]["value"]},
        "accuracy_all_cells": all_cells,
        "gate_sweep": {"how": "the learned walk with the network only for accepted nodes "
                              "with s = l/d >= s_min (bh_set_mlp_gate), potential alone, "
                              "median of the timed walks; speedup against the plain walk's "
                              "potential at plain_theta", "runs": gate_sweep},
        "clocks": clocks, "e2e": e2e,
        "gpu_launches": 9 * args.steps,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def build_roofline(ncells, nnodes, quad, build_ms):
    """The build against HBM: algorithmic bytes = the density read (4 B per
    cell) + per node the walk record, FP64 moments, {l, delta} and level
    (32 + 32 + 8 + 1 B) + a 32-B quadrupole record per internal node."""
    n_int = nnodes - ncells
    traffic = 4 * ncells + 73 * nnodes + (32 * n_int if quad else 0)
    peak = measured_peak("hbm_gbs")
    gbs = traffic / (build_ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "bh_build (keys, topology, FP64 moments)",
            "algorithmic_bytes": traffic, "achieved": gbs, "peak": peak, "unit": "GB/s",
            "frac": gbs / peak, "note": "limited by FP64 arithmetic, not by HBM"}


def max_over_ranks(value, device=None):
    """The largest value over all ranks (the slowest rank's time); the value
    itself without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, steps, total_ms):
    """Whole-job units per second: every rank solves its own replica, the job
    takes as long as its slowest rank."""
    return world * units_per_rank * steps / (total_ms * 1e-3)


def measured_peak(key):
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))[key])
    except (OSError, KeyError, ValueError, TypeError):
        return {"bf16_tflops": 1900.0, "hbm_gbs": 6800.0}.get(key, float("nan"))


def main():
    args = parse()
    if args.theta is None:
        headline = not (args.monopole or args.vote or args.periodic)
        args.theta = {"batched": 0.5, "learned": 0.8}.get(args.workload,
                                                          0.75 if headline else 0.7)
    if args.plain_theta is None:
        args.plain_theta = 0.4 if args.workload == "learned" else 0.24
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "batched":
        return batched_arm(args)
    if args.workload == "learned":
        return learned_arm(args)
    import torch
    import torch.distributed as dist
    from paper_1509_07370_gb300 import bhgrav as bh

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = workload(args.workload)
    n = w.ncells
    mesh = w.mesh
    periodic = args.periodic
    quad = not args.monopole and not periodic
    if periodic and args.vote:
        raise SystemExit("--periodic runs the per-cell walk (no --vote)")
    crit = bh.BH_CRIT_WARP_VOTE if args.vote else bh.BH_CRIT_PER_CELL
    rho32 = np.ascontiguousarray(w.density.reshape(-1), dtype=np.float32)
    stream = torch.cuda.Stream(dev)
    solver = bh.Solver(criterion=crit, quadrupole=quad, periodic=periodic, device=local,
                       stream=stream)
    if periodic and args.ewald_grid != 64:
        solver.set_ewald(args.ewald_grid, 3)
    d_rho = torch.as_tensor(rho32, device=dev)
    out = torch.empty(n, dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    # the walk's launch shape, tuned on this tree (CTA width, targets per warp,
    # plain or persistent grid); untimed
    with torch.cuda.stream(stream):
        solver.build(mesh.level, mesh.ijk, d_rho)
    if args.walk_shape:
        shape = (tuple(int(v) for v in args.walk_shape.split(",")) + (0,))[:4]
        if shape[3]:
            solver.autotune(args.theta)  # makes the longest-first order
        solver.set_walk_shape(*shape)
    else:
        shape = solver.autotune(args.theta)
    if world > 1:
        dist.barrier()
    clk = ClockSampler(local)
    step_ms, build_ms, walk_ms = timed_steps(solver, mesh, d_rho, args.theta, out, args.steps,
                                             args.warmup, flush, stream, clk)
    if world > 1:
        dist.barrier()
    total_ms = max_over_ranks(float(np.sum(step_ms)), dev)
    value = job_rate(world, n, args.steps, total_ms)
    phi_gpu = out.double().cpu().numpy()

    # algorithmic work of the walk (untimed): per-cell counts from the library
    def work(s, theta, with_quad):
        ni, nt, nc = s.walk_counts(theta, with_cells=True)
        n_int = int(ni.sum(dtype=torch.int64).item())
        n_test = int(nt.sum(dtype=torch.int64).item())
        n_cell = int(nc.sum(dtype=torch.int64).item())
        per_node = FLOP_PER_QUAD_INTERACTION if with_quad else FLOP_PER_INTERACTION
        flops = FLOP_PER_INTERACTION * n_cell + per_node * (n_int - n_cell) + FLOP_PER_TEST * n_test
        if s.options.periodic:
            flops = (FLOP_PER_INTERACTION_PERIODIC * n_int + FLOP_PER_CELL_WRAP * n_cell
                     + FLOP_PER_TEST_PERIODIC * n_test + FLOP_PER_SELF_IMAGE * n)
        return n_int, n_test, n_cell, flops

    n_int, n_test, n_cell, flops = work(solver, args.theta, quad)
    walk_s = float(np.mean(walk_ms)) * 1e-3
    clocks = clk.summary()
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = clocks["sm_mhz"] if clocks else 1440.0
    peak = FP32_LANES_PER_SM * props.multi_processor_count * sm_mhz * 1e6
    mode = (f"periodic{args.ewald_grid}" if periodic
            else "quadrupole" if quad else "monopole")
    traffic = captured_traffic(w.name, args.theta, mode) if not args.vote else None
    _, nn, maxlev = solver.tree_size()
    # keys with the largest mass, sort, tiling, scan, top nodes, top-node
    # child lists, k_blocks, k_upper_tree (the rest of the blocks and the top
    # tree), walk
    launches_per_step = 9

    # the plain walk (monopole, per-cell) at the theta of equal accuracy
    plain = None
    phi_plain = None
    if not args.no_plain and not periodic:
        psolver = bh.Solver(device=local, stream=stream)
        pout = torch.empty(n, dtype=torch.float32, device=dev)
        with torch.cuda.stream(stream):
            psolver.build(mesh.level, mesh.ijk, d_rho)
        pshape = psolver.autotune(args.plain_theta)
        psteps = max(5, args.steps // 3)
        p_step, p_build, p_walk = timed_steps(psolver, mesh, d_rho, args.plain_theta, pout,
                                              psteps, args.warmup, flush, stream)
        p_total = max_over_ranks(float(np.sum(p_step)), dev)
        p_value = job_rate(world, n, psteps, p_total)
        pi, pt, pc, pflops = work(psolver, args.plain_theta, False)
        phi_plain = pout.double().cpu().numpy()
        plain = {"theta": args.plain_theta, "walk": "binary32, compensated sum, per-cell, monopole",
                 "walk_shape": {"warps_per_cta": pshape[0], "target_pairs_per_lane": pshape[1],
                                "groups_per_take": pshape[2], "longest_first": pshape[3]},
                 "value": p_value, "unit": "cells/s", "steps": psteps,
                 "ms_per_step": p_total / psteps,
                 "phases_ms": {"build": float(np.mean(p_build)),
                               "potential": float(np.mean(p_walk))},
                 "interactions_per_cell": pi / n, "tests_per_cell": pt / n,
                 "roofline_frac": pflops / (float(np.mean(p_walk)) * 1e-3) / peak,
                 "roofline_frac_with_kahan": (pflops + 3 * (pi - pc))
                                             / (float(np.mean(p_walk)) * 1e-3) / peak,
                 "traffic": captured_traffic(w.name, args.plain_theta, "monopole"),
                 "speedup": value / p_value}
        psolver.close()

    # end to end through the host-memory entry point (pinned buffers)
    e2e = None
    if not args.no_e2e:
        pinned = (torch.from_numpy(rho32).pin_memory(),
                  torch.empty(n, dtype=torch.float32).pin_memory())
        h_rho, h_out = pinned[0].numpy(), pinned[1].numpy()
        host_solver = bh.Solver(criterion=crit, quadrupole=quad, periodic=periodic,
                                device=local, stream=stream)
        if periodic and args.ewald_grid != 64:
            host_solver.set_ewald(args.ewald_grid, 3)
        for _ in range(max(1, args.warmup)):
            host_solver.solve_host(mesh.level, mesh.ijk, h_rho, args.theta, 1.0, h_out)
        # the device arm's launch shape (bh_autotune makes this context's own
        # group order on the tree the warm-up built; untimed)
        host_solver.autotune(args.theta)
        host_solver.set_walk_shape(*shape)
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            host_solver.solve_host(mesh.level, mesh.ijk, h_rho, args.theta, 1.0, h_out)
            ts.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(float(np.sum(ts)), dev)
        e2e = {"value": job_rate(world, n, args.steps, e2e_s * 1e3), "unit": "cells/s",
               "h2d_bytes_per_step": int(rho32.nbytes + mesh.level.nbytes + mesh.ijk.nbytes),
               "d2h_bytes_per_step": int(h_out.nbytes),
               "walk_shape": list(shape)}
        host_solver.close()

    all_cells = None
    if rank == 0:
        all_cells = all_cells_error(
            bh, mesh, d_rho, maxlev,
            {("max_err_over_max_abs_vs_direct" if periodic else "max_rel_vs_direct"): phi_gpu,
             "plain_max_rel_vs_direct": phi_plain},
            dev, stream, periodic=periodic, ewald_grid=args.ewald_grid,
            limit=args.all_cells_limit)
        if all_cells is not None and phi_plain is not None:
            all_cells["plain_theta"] = args.plain_theta

    worst = None
    if all_cells is not None and "_worst_cells" in all_cells:
        worst = (all_cells.pop("_worst_cells"), all_cells.pop("_direct_at_worst"))
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = oracle_leg(w, args.theta, args.cpu_seconds, phi_gpu, quad=quad,
                         plain=(phi_plain, args.plain_theta) if phi_plain is not None else None,
                         periodic=periodic, ewald_grid=args.ewald_grid,
                         worst=None if periodic else worst)

    if rank == 0:
        line = {
            "metric": "cell potentials/sec", "value": value, "unit": "cells/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "cells": n, "nodes": nn, "theta": args.theta,
                       "walk": "binary32, compensated sum, "
                               + ("warp vote (paper)" if args.vote else "per-cell opening test")
                               + (f", periodic boundaries (Ewald table {args.ewald_grid}, "
                                  "series 3)" if periodic else "")
                               + (", quadrupole nodes" if quad else ", monopole nodes"),
                       "moments": "f64", "density_input": "f32",
                       "l2": "flushed between steps (256 MiB write)",
                       "walk_shape": {"warps_per_cta": shape[0],
                                      "target_pairs_per_lane": shape[1],
                                      "groups_per_take": shape[2],
                                      "longest_first": shape[3],
                                      "how": ("set by --walk-shape" if args.walk_shape else
                                              "bh_autotune on this tree before timing")
                                             + " (0 groups per take: plain grid; longest "
                                               "first: the groups sorted by the work of "
                                               "their walks, made by bh_autotune)"},
                       "parallelism": f"replicas x{world}"},
            "phases_ms": {"build": float(np.mean(build_ms)), "potential": float(np.mean(walk_ms)),
                          "step_median": float(np.median(step_ms)),
                          "potential_median": float(np.median(walk_ms)),
                          "potential_p10_p90": [float(np.percentile(walk_ms, 10)),
                                                float(np.percentile(walk_ms, 90))]},
            "walk_only_value": n / walk_s,
            "build_roofline": build_roofline(n, nn, quad, float(np.mean(build_ms))),
            "walk_work": {"interactions": n_int, "cell_interactions": n_cell, "tests": n_test,
                          "interactions_per_cell": n_int / n, "tests_per_cell": n_test / n},
            "roofline": {"bound": "alu", "kernel": "bh_potential (s2 prep + walk)",
                         "achieved": flops / walk_s / 1e12, "peak": peak / 1e12,
                         "unit": "TFLOP/s", "frac": flops / walk_s / peak, "traffic": traffic,
                         "frac_with_kahan": (flops + 3 * (n_int - n_cell)) / walk_s / peak,
                         "frac_monopole_count": (FLOP_PER_INTERACTION * n_int
                                                 + FLOP_PER_TEST * n_test) / walk_s / peak,
                         "kahan_ops": ("3 per node interaction (the compensation of the "
                                       "compensated sum; a bottom node's 8 cell terms are "
                                       "summed plainly and folded once, not counted)"),
                         "mufu_bound_ms": n_int / (16 * props.multi_processor_count
                                                   * sm_mhz * 1e6) * 1e3,
                         "traffic_unit": "bytes per walk launch (ncu dram read+write)",
                         "traffic_source": ("dram__bytes_read.sum + dram__bytes_write.sum of "
                                            "the ncu capture summarised in profiles/ for this "
                                            "walk source (its sha256 checked) and workload; "
                                            "null when the source or workload differs"),
                         "peak_basis": f"{FP32_LANES_PER_SM} FP32 lanes x "
                                       f"{props.multi_processor_count} SMs x {sm_mhz:.0f} MHz "
                                       "(median SM clock measured during the timed region)"},
            "vs_plain": plain,
            "accuracy_all_cells": all_cells,
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
