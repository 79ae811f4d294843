"""Throughput of the DG compressible Navier--Stokes RK stage on GB300.

A step is one full RK(5,4) time step (5 stages, each one evaluation of
L = M^{-1}(-F + F_rhs) with cell and face integrals, inverse mass and the 2N
update) of the Taylor--Green vortex, 64^3 cells, k = 3, FP64, face-centric
kernels (a face kernel that evaluates every face once, then one kernel for the
cells, the face shares, M^{-1} and the update).
Metric: GDoF/s per RK stage = 5 N_nodes * stages / time / 1e9 (DoF counts the
5 conserved fields per node).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Prints one JSON line (rank 0).  N > 1 under torchrun: independent replicas
(one TGV problem per GPU, weak scaling); the path needs no collective.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GDoF/s per RK stage"
UNIT = "GDoF/s"
FP64_PEAK_TFLOPS = 1.2   # measured FP64 FMA throughput of this machine's GB300 (FMA-chain probe, 152 SMs)
FP32_PEAK_TFLOPS = 73.5  # measured FP32 FMA throughput, same probe


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per cell and launch from one ncu capture of
# a kernel kind on a TGV mesh larger than L2, with the digest of the device-code sources it was built from:
# (kind, precision 0/1, N, QC, QV) -> (bytes per cell, sources digest, profile summary under profiles/).
# The roofline reports traffic = bytes per cell x cells only while the sources still have that digest.
TRAFFIC = {
    ("faces", 0, 4, 5, 4): (15115.6, "cc826ba75499d748a67d4103685ebe4090f2818998df31d1db553338e0ad948a",
                            "profiles/face_centric_fp64_tgv64_k3_launches.md"),
    ("cell_stage", 0, 4, 5, 4): (17651.0, "cc826ba75499d748a67d4103685ebe4090f2818998df31d1db553338e0ad948a",
                                 "profiles/face_centric_fp64_tgv64_k3_launches.md"),
    ("faces", 1, 4, 5, 4): (7333.7, "cc826ba75499d748a67d4103685ebe4090f2818998df31d1db553338e0ad948a",
                            "profiles/dg_face_task_kernel_mixed_tgv48_k3.md"),
    ("cell_stage", 1, 4, 5, 4): (13743.6, "cc826ba75499d748a67d4103685ebe4090f2818998df31d1db553338e0ad948a",
                                 "profiles/dg_cell_task_kernel_mixed_tgv48_k3.md"),
}


def kernel_digest():
    """sha256 over the device-code sources (every csrc file but the host plan dgcns.cu) and the compile flags."""
    import hashlib
    from paper_1806_03095_gb300 import build
    h = hashlib.sha256()
    for name in sorted(os.listdir(build.CSRC)):
        if name.endswith((".cuh", ".h")) or name == "dg_inst.cu":
            h.update(name.encode())
            h.update(open(os.path.join(build.CSRC, name), "rb").read())
    h.update(" ".join(build.ARCH + build.FLAGS).encode())
    return h.hexdigest()


def traffic_per_launch(kind, prec, N, QC, QV, Nc):
    entry = TRAFFIC.get((kind, prec, N, QC, QV))
    if entry is None:
        return None, None
    if kernel_digest() != entry[1]:
        return None, entry[2] + " (kernel sources changed since the capture)"
    return entry[0] * Nc, entry[2]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if (args.impl == "native" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(ws, x):
    if ws == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# -- clocks sampled during the timed region ------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.proc = None
        self.path = None
        try:
            uuid = str(torch.cuda.get_device_properties(device).uuid)
            sel = ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            sel = []
        self.cmd = ["nvidia-smi", *sel, "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(self.cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                try:
                    rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
                except ValueError:
                    pass
        os.unlink(self.path)
        if not rows:
            return None
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# -- native arm --------------------------------------------------------------------------------------
def run_stages(ctx, nsteps, dt, t0, bufs):
    """nsteps RK(5,4) steps through dg_cns_rk_steps (ping-pong of U and U_tmp inside the library, the state
    back in U at the end); returns U."""
    U, Ut, dU = bufs
    return ctx.rk_steps(nsteps, dt, t0, U, Ut, dU)


def time_native(cfg, steps, warmup, device, kernel_times=None):
    """Time `steps` RK(5,4) steps after `warmup` untimed ones (CUDA events on torch's current stream, where the
    library launches).  kernel_times (dict): filled with the library's per-kernel CUDA-event times of the timed
    region, {kind: (total ms, launches)}."""
    from paper_1806_03095_gb300 import configs, inputs
    ctx = configs.make_context(cfg, device=device)
    xyz = ctx.node_coords()
    U = inputs.tgv_state(xyz) if cfg["name"].startswith("tgv") else inputs.channel_state(xyz, 1806)
    del xyz
    bufs = (U.contiguous(), ctx.empty_state(), ctx.empty_residual())
    dt = configs.time_step(cfg)
    run_stages(ctx, warmup, dt, 0.0, bufs)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = ctx.dg_cns_launch_count()
    if kernel_times is not None:
        ctx.timing(True)
    e0.record(st)
    run_stages(ctx, steps, dt, 0.0, bufs)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = ctx.dg_cns_launch_count() - n0
    if kernel_times is not None:
        kernel_times.update(ctx.kernel_times())
        ctx.timing(False)
    return ctx, bufs, dt, ms, launches


KERNELS = {"split": 0, "fused": 1, "faces": 2}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default="tgv64_k3")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--kernel", choices=["fused", "split", "faces"], default="faces")
    ap.add_argument("--no-extras", action="store_true", help="skip the mixed/split comparison and CPU baseline")
    ap.add_argument("--mesh", choices=["box", "rotated", "sine"], default="box",
                    help="box: the workload's own mesh; rotated: every cell in a seeded cube frame (seed 1806); "
                         "sine: the same box with aligned frames, deformed by --deform (both non-affine paths)")
    ap.add_argument("--deform", type=float, default=0.0, help="sine deformation amplitude of --mesh rotated/sine")
    ap.add_argument("--geometry", choices=["stored", "fly"], default="fly",
                    help="geometry of --mesh rotated/sine: stored per point or recomputed in the kernels")
    ap.add_argument("--inverse-mass", action="store_true",
                    help="time dg_cns_inverse_mass alone on the workload (one JSON line; not the step metric)")
    ap.add_argument("--stability", action="store_true",
                    help="critical Cr (and with --with-d D) numbers of the TGV, the paper's time-step study")
    ap.add_argument("--schemes", default="lsrk54,lsrk33")
    ap.add_argument("--degrees", default="3")
    ap.add_argument("--with-d", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_init(args)
    if args.impl == "reference":
        return reference_arm(args, ws, rank)
    if args.inverse_mass:
        return inverse_mass_only(args)
    if args.stability:
        return stability(args)

    from paper_1806_03095_gb300 import configs, roofline
    device = local if torch.cuda.is_available() else None
    if device is None:
        raise RuntimeError("bench.py native arm needs a GPU")
    torch.cuda.set_device(device)
    prec = 1 if args.precision == "mixed" else 0
    cfg = configs.WORKLOADS[args.workload](precision=prec, kernel=KERNELS[args.kernel])
    mesh_note = ""
    if args.mesh != "box":
        cfg = dict(cfg, mapping=3 if args.mesh == "rotated" else 2,
                   map_param=1806.0 if args.mesh == "rotated" else args.deform,
                   deform=args.deform if args.mesh == "rotated" else 0.0,
                   geometry=1 if args.geometry == "fly" else 0)
        mesh_note = ", %s mesh (deform %g), geometry %s" % (args.mesh, args.deform, args.geometry)
    N = cfg["k"] + 1
    Nc = cfg["ncells"][0] * cfg["ncells"][1] * cfg["ncells"][2]
    nodes = Nc * N ** 3

    barrier(ws)
    clocks = ClockSampler(device)
    clocks.start()
    ktimes = {}
    ctx, bufs, dt, ms, launches = time_native(cfg, args.steps, args.warmup, device, ktimes)
    clk = clocks.stop()
    ms = allreduce_max(ws, ms)
    barrier(ws)
    stages = 5 * args.steps
    value = ws * 5 * nodes * stages / (ms * 1e-3) / 1e9
    ms_step = ms / args.steps
    out = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if prec == 0 else "f32 arithmetic / f64 state", "data": "synthetic",
           "config": {"workload": "Taylor-Green vortex %d^3 cells, k=%d, nq_conv=%d, nq_visc=%d, RK(5,4), %s, %s kernel%s"
                      % (cfg["ncells"][0], cfg["k"], cfg["nq_conv"], cfg["nq_visc"], args.precision, args.kernel,
                         mesh_note),
                      "cells": Nc, "nodes": nodes, "dofs": 5 * nodes,
                      "stages_timed": stages, "dt": dt,
                      "l2": "inputs larger than L2 (state %.0f MB per vector)" % (nodes * 40 / 1e6),
                      "parallelism": "replicas" if ws > 1 else "1 GPU"},
           "gpu_launches": int(launches)}
    out["roofline"] = roofline_entry(ktimes, cfg, prec, load_peaks())
    if clk:
        out["clocks"] = clk

    if rank == 0 and ws == 1:
        out["e2e"] = e2e_native(ctx, bufs, dt, min(args.steps, 10))
        if not args.no_extras:
            out["cpu_baseline"] = cpu_baseline(cfg)
            out["extras"] = extras(args, cfg)
    del ctx
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


KERNEL_NAMES = {
    "fused": "dg_op_kernel / dg_op_warp_kernel: cells + 6 faces + M^-1 + stage update (fused)",
    "faces": "dg_face_kernel: every face once, both cells' shares (face-centric)",
    "cell_stage": "dg_op_kernel / dg_op_warp_kernel: cells + face shares + M^-1 + stage update (face-centric)",
    "cell": "dg_op_kernel: cell integrals (split)", "face": "dg_op_kernel: element-centric faces (split)",
    "mass": "dg_op_kernel: M^-1 + stage update (split)", "dev": "dg_dev_kernel: FP32 deviation pre-pass"}


def roofline_entry(ktimes, cfg, prec, peaks):
    """ALU roofline of the dominant kernel (largest share of the timed region), from the library's per-kernel
    CUDA-event times: achieved = algorithmic flops per launch / average launch duration; every kernel kind is
    listed with its share, its flop rate and its algorithmic HBM rate."""
    from paper_1806_03095_gb300 import roofline
    N, QC, QV = cfg["k"] + 1, cfg["nq_conv"], cfg["nq_visc"]
    Nc = cfg["ncells"][0] * cfg["ncells"][1] * cfg["ncells"][2]
    rbytes = 4 if prec else 8
    peak = FP32_PEAK_TFLOPS if prec else FP64_PEAK_TFLOPS
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    total = sum(v[0] for v in ktimes.values()) or 1.0
    kernels = {}
    for kind, (kms, n) in ktimes.items():
        t = kms / n * 1e-3
        e = {"launches": n, "avg_ms": round(kms / n, 4), "share": round(kms / total, 4)}
        fl = roofline.kernel_flops(kind, N, QC, QV, Nc)
        by = roofline.kernel_bytes(kind, N, Nc, rbytes) if kind != "dev" else N ** 3 * Nc * 5 * (8 + rbytes)
        if kind in ("fused", "cell_stage", "mass"):
            by -= N ** 3 * Nc * 5 * rbytes / 5.0  # stage 0 of 5 does not read dU
        if fl:
            e["tflops"] = round(fl / t / 1e12, 4)
            e["frac_alu"] = round(fl / t / 1e12 / peak, 4)
        if by:
            e["hbm_gbs"] = round(by / t / 1e9, 2)
        kernels[kind] = e
    if not ktimes:
        return None
    dom = max(ktimes, key=lambda k: ktimes[k][0])
    kms, n = ktimes[dom]
    t = kms / n * 1e-3
    fl = roofline.kernel_flops(dom, N, QC, QV, Nc) or 0.0
    by = kernels[dom].get("hbm_gbs", 0.0) * 1e9 * t
    ach = fl / t / 1e12
    traffic, traffic_src = traffic_per_launch(dom, prec, N, QC, QV, Nc)
    return {"bound": "alu", "achieved": round(ach, 4), "peak": peak, "unit": "TFLOP/s", "frac": round(ach / peak, 4),
            "traffic": traffic, "traffic_source": traffic_src,
            "peak_source": "measured %s FMA probe (no %s entry in MEASURED_PEAKS.json)"
            % ("FP32" if prec else "FP64", "FP32" if prec else "FP64"),
            "kernel": KERNEL_NAMES.get(dom, dom), "avg_launch_ms": round(kms / n, 4), "flops_per_launch": fl,
            "hbm": {"achieved": round(by / t / 1e9, 2), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(by / t / 1e9 / hbm_peak, 5), "bytes_per_launch": by},
            "kernels": kernels}


def e2e_native(ctx, bufs, dt, nsteps):
    """Same metric through the public API with host buffers: per step an H2D copy of the state from pinned
    memory, the 5 stages, and a D2H copy of the new state."""
    U, Ut, dU = bufs
    host = torch.empty(U.shape, dtype=torch.float64, pin_memory=True)
    host.copy_(U)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for n in range(nsteps):
        U.copy_(host, non_blocking=True)
        res = run_stages(ctx, 1, dt, n * dt, (U, Ut, dU))
        host.copy_(res, non_blocking=True)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    nbytes = U.numel() * 8
    return {"value": round(5 * (U.numel() // 5) * 5 * nsteps / (ms * 1e-3) / 1e9, 4), "unit": UNIT,
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": nsteps}


def extras(args, cfg):
    """Beside the headline: the other precision / kernel organisation on the same workload, and the mixed form's
    error against the FP64 path (which matches the oracle) for one evaluation of L(U) at full size."""
    from paper_1806_03095_gb300 import api, configs, inputs
    res = {}
    device = torch.cuda.current_device()
    steps = max(2, args.steps // 2)
    combos = [("%s_%s" % ("fp64" if p == 0 else "mixed", kn), p, kv) for p in (0, 1)
              for kn, kv in (("faces", 2), ("fused", 1), ("split", 0))]
    for name, prec, kern in [c for c in combos if (c[1], c[2]) != (cfg["precision"], cfg["kernel"])]:
        c = dict(cfg, precision=prec, kernel=kern)
        ctx, bufs, dt, ms, _ = time_native(c, steps, 3, device)
        nodes = bufs[0].numel() // 5
        res[name] = {"value": round(5 * nodes * 5 * steps / (ms * 1e-3) / 1e9, 4), "unit": UNIT,
                     "ms_per_step": round(ms / steps, 3)}
        del ctx, bufs
        torch.cuda.empty_cache()
    g64 = configs.make_context(dict(cfg, precision=0, kernel=2), device=device)
    g32 = configs.make_context(dict(cfg, precision=1, kernel=2), device=device)
    U = inputs.tgv_state(g64.node_coords())
    L64 = g64.apply(U, op=api.OP_L)
    L32 = g32.apply(U, op=api.OP_L).double()
    d = L32 - L64
    res["mixed_error_vs_fp64"] = {"quantity": "L(U) of the initial TGV state, 64^3, k=3",
                                  "rel_l2": float(torch.linalg.norm(d) / torch.linalg.norm(L64)),
                                  "rel_max": float(d.abs().max() / L64.abs().max())}
    del g64, g32, U, L64, L32, d
    torch.cuda.empty_cache()
    res["adjoint"], res["adjoint_element_centric"], res["adjoint_mixed"] = adjoint_extras()
    res.update(other_workloads(steps))
    res["rotated_frames"] = rotated_frames(steps)
    res["mixed_dissipation_history"] = dissipation_history()
    res["memory_bound_kernels"] = memory_bound_kernels()
    res["k_sweep"] = k_sweep()
    return res


def _rate(ms, nodes, steps):
    return round(5 * nodes * 5 * steps / (ms * 1e-3) / 1e9, 4)


def other_workloads(steps):
    """Throughput of the other benchmark workloads: TGV 40^3 k=5 (FP64 and mixed, fused) with the mixed form's
    error of L(U); the turbulent channel 32^3 k=3 on the stretched mesh (walls, body force), mixed and FP64, with the
    Jacobians stored per point and recomputed in the kernels from the node coordinates."""
    from paper_1806_03095_gb300 import api, configs, inputs
    device = torch.cuda.current_device()
    out = {}
    for key, wl, prec, geo in (("tgv40_k5_fp64", "tgv40_k5", 0, 0), ("tgv40_k5_mixed", "tgv40_k5", 1, 0),
                               ("channel32_k3_mixed", "channel32_k3", 1, 0), ("channel32_k3_fp64", "channel32_k3", 0, 0),
                               ("channel32_k3_mixed_geometry_on_the_fly", "channel32_k3", 1, 1),
                               ("channel32_k3_fp64_geometry_on_the_fly", "channel32_k3", 0, 1)):
        cfg = dict(configs.WORKLOADS[wl](precision=prec, kernel=2), geometry=geo)
        ctx, bufs, dt, ms, _ = time_native(cfg, steps, 3, device)
        nodes = bufs[0].numel() // 5
        out[key] = {"value": _rate(ms, nodes, steps), "unit": UNIT, "ms_per_step": round(ms / steps, 3), "dt": dt}
        del ctx, bufs
        torch.cuda.empty_cache()
    g64 = configs.make_context(configs.WORKLOADS["tgv40_k5"](precision=0), device=device)
    g32 = configs.make_context(configs.WORKLOADS["tgv40_k5"](precision=1), device=device)
    U = inputs.tgv_state(g64.node_coords())
    L64 = g64.apply(U, op=api.OP_L)
    d = g32.apply(U, op=api.OP_L).double() - L64
    out["tgv40_k5_mixed_error_vs_fp64"] = {"quantity": "L(U) of the initial TGV state, 40^3, k=5",
                                           "rel_l2": float(torch.linalg.norm(d) / torch.linalg.norm(L64)),
                                           "rel_max": float(d.abs().max() / L64.abs().max())}
    del g64, g32, U, L64, d
    torch.cuda.empty_cache()
    return out


def rotated_frames(steps):
    """Rotated-frame meshes (every cell in one of the 48 cube frames, neighbours read through per-face
    orientation codes) against the same box with aligned frames, affine and deformed: TGV 48^3, k = 3, FP64
    and mixed; all three organisations with geometry on the fly, the face-centric one also with stored
    geometry, and the Cartesian box (affine, no geometry arrays) for reference."""
    from paper_1806_03095_gb300 import api, configs
    device = torch.cuda.current_device()
    out = {"workload": "TGV 48^3, k = 3; rotated: frames seeded 1806, aligned: the same box through the same "
                       "kernels with every frame the identity; deformed: the sine deformation of amplitude 0.05 "
                       "on top; geometry on the fly, and stored geometry for the face-centric kernels; "
                       "cartesian: the affine box without geometry arrays"}
    base = configs.WORKLOADS["tgv48_k3"]()
    meshes = (("rotated", api.MAP_ROTATED, 1806.0, 0.0), ("aligned", api.MAP_SINE, 0.0, 0.0),
              ("rotated_deformed", api.MAP_ROTATED, 1806.0, 0.05), ("aligned_deformed", api.MAP_SINE, 0.05, 0.0))
    runs = [(prec, kn, kv, 1, m) for prec in (0, 1) for kn, kv in (("faces", 2), ("fused", 1), ("split", 0))
            for m in meshes]
    runs += [(prec, "faces", 2, 0, m) for prec in (0, 1) for m in meshes]
    runs += [(prec, "faces", 2, 0, ("cartesian", api.MAP_AFFINE, 0.0, 0.0)) for prec in (0, 1)]
    for prec, kn, kv, geo, (frames, mapping, param, deform) in runs:
        cfg = dict(base, precision=prec, kernel=kv, mapping=mapping, map_param=param, deform=deform,
                   geometry=geo)
        ctx, bufs, dt, ms, _ = time_native(cfg, steps, 3, device)
        key = "%s_%s_%s%s" % ("fp64" if prec == 0 else "mixed", kn, frames,
                              "_stored" if geo == 0 and mapping != api.MAP_AFFINE else "")
        out[key] = {"value": _rate(ms, bufs[0].numel() // 5, steps), "unit": UNIT,
                    "ms_per_step": round(ms / steps, 3)}
        del ctx, bufs
        torch.cuda.empty_cache()
    return out


def memory_bound_kernels(reps=20):
    """The kernels the HBM bar applies to: the inverse mass alone (dg_cns_inverse_mass: read R, write M^-1 R)
    and the split organisation's M^-1 + stage-update kernel (read R, dU, U; write dU, U_out), TGV 64^3, k = 3,
    FP64 and mixed, timed with the library's per-kernel CUDA events; both roofs reported (FP64 is ALU-bound
    even here: ~3 flop/B of even-odd sweeps against a ridge of 0.18 flop/B)."""
    from paper_1806_03095_gb300 import configs, inputs, roofline
    device = torch.cuda.current_device()
    hbm_peak = load_peaks().get("hbm_gbs", 6800.0)
    out = {}
    for prec in (0, 1):
        cfg = configs.WORKLOADS["tgv64_k3"](precision=prec, kernel=0)
        g = configs.make_context(cfg, device=device)
        N = cfg["k"] + 1
        Nc = cfg["ncells"][0] * cfg["ncells"][1] * cfg["ncells"][2]
        rb = 4 if prec else 8
        R = inputs.uniform(g.shape, 5).to(device=device, dtype=g.rdtype)
        Y = torch.empty_like(R)
        for _ in range(3):
            g.inverse_mass(R, Y)
        g.timing(True)
        for _ in range(reps):
            g.inverse_mass(R, Y)
        kt = g.kernel_times()
        g.timing(False)
        ms = kt["mass"][0] / kt["mass"][1]
        by = 2 * Nc * N ** 3 * 5 * rb
        fl = roofline.mass_flops(N) * Nc
        peak = FP32_PEAK_TFLOPS if prec else FP64_PEAK_TFLOPS
        name = "fp64" if prec == 0 else "mixed"
        out["inverse_mass_" + name] = {"avg_ms": round(ms, 4), "hbm_gbs": round(by / ms / 1e6, 1),
                                       "hbm_frac": round(by / ms / 1e6 / hbm_peak, 4),
                                       "tflops": round(fl / ms / 1e9, 3), "alu_frac": round(fl / ms / 1e9 / peak, 4),
                                       "bytes_per_launch": by, "flops_per_launch": fl}
        # split stage: the M^-1 + update kernel inside real RK steps
        kt = {}
        ctx, bufs, dt, ms_all, _ = time_native(cfg, 2, 3, device, kt)
        mk = kt["mass"]
        ms = mk[0] / mk[1]
        fl = roofline.kernel_flops("mass", N, cfg["nq_conv"], cfg["nq_visc"], Nc)
        by = roofline.kernel_bytes("mass", N, Nc, rb) - N ** 3 * Nc * 5 * rb / 5.0
        out["split_mass_stage_" + name] = {"avg_ms": round(ms, 4), "hbm_gbs": round(by / ms / 1e6, 1),
                                           "hbm_frac": round(by / ms / 1e6 / hbm_peak, 4),
                                           "tflops": round(fl / ms / 1e9, 3),
                                           "alu_frac": round(fl / ms / 1e9 / peak, 4), "bytes_per_launch": by}
        del g, R, Y, ctx, bufs
        torch.cuda.empty_cache()
    return out


def stability_run(cfg, scheme, number, which, t_final, chunk=50):
    """Integrate the Taylor-Green vortex with the 2N scheme to t_final at Courant number `number` (which = "Cr")
    or viscous number (which = "D", the other restriction made slack); unstable when the state turns
    non-finite or the kinetic energy exceeds twice its initial value.  Returns (stable, steps, t reached)."""
    from paper_1806_03095_gb300 import api, configs, inputs, schemes
    g = configs.make_context(cfg)
    U = inputs.tgv_state(g.node_coords()).contiguous()
    Ut, dU = g.empty_state(), g.empty_residual()
    nu = 1.0 / cfg["Re"]
    if which == "Cr":
        dt = api.cfl_dt(cfg["k"], cfg["h_min"], cfg["u_max"], cfg["Ma"], Cr=number, D=1e9, nu=nu)
    else:
        dt = api.cfl_dt(cfg["k"], cfg["h_min"], cfg["u_max"], cfg["Ma"], Cr=1e9, D=number, nu=nu)
    nsteps = int(math.ceil(t_final / dt))
    ek0 = float(g.diagnostics(U)[0])
    done = 0
    while done < nsteps:
        n = min(chunk, nsteps - done)
        g.lsrk_steps(schemes.SCHEMES[scheme], n, dt, U, Ut, dU)
        done += n
        d = g.diagnostics(U, check=False)
        if not (d[8] == 0 and math.isfinite(float(d[0])) and float(d[0]) <= 2.0 * ek0):
            del g
            return False, done, done * dt
    del g
    return True, done, done * dt


def stability(args):
    """The paper's time-step study (Sec. 4.2.2, critical Cr and D numbers with e = 1.5, f = 3): Taylor-Green
    vortex at effective resolution 60^3 or 64^3 (k = 2, 3, 5 on 20^3, 16^3, 10^3 cells), Re = 1600 to t = 20
    for Cr, Re = 1 to t = 1 for D; bisection to 0.02 between a stable and an unstable number, for each 2N
    scheme of schemes.SCHEMES named in --schemes.  FP64, face-centric kernels.  One JSON line."""
    from paper_1806_03095_gb300 import configs, schemes
    torch.cuda.set_device(0)
    cells = {2: 20, 3: 16, 5: 10}
    out = {"study": "critical Courant and viscous numbers, TGV, e=1.5, f=3 (Sec. 4.2.2)", "results": []}
    for scheme in args.schemes.split(","):
        for k in [int(v) for v in args.degrees.split(",")]:
            # brackets: a number assumed stable (checked) and one assumed unstable (checked)
            cr_lo = 0.3 if len(schemes.SCHEMES[scheme][0]) >= 5 else 0.14
            for which, lo, hi, Re, tf in (("Cr", cr_lo, 1.6, 1600.0, 20.0), ("D", 0.02, 0.2, 1.0, 1.0)):
                if which == "D" and not args.with_d:
                    continue
                cfg = dict(configs.tgv(cells[k], k, precision=0, kernel=2), Re=Re)
                runs = []
                ok_lo = stability_run(cfg, scheme, lo, which, tf)
                ok_hi = stability_run(cfg, scheme, hi, which, tf)
                runs += [(lo, ok_lo[0]), (hi, ok_hi[0])]
                if not ok_lo[0] or ok_hi[0]:
                    out["results"].append({"scheme": scheme, "k": k, "which": which, "bracket_failed": runs})
                    continue
                step = 0.02 if which == "Cr" else 0.002
                while hi - lo > step * 1.0001:
                    mid = round(0.5 * (lo + hi) / step) * step
                    if mid <= lo or mid >= hi:
                        mid = lo + step
                    st = stability_run(cfg, scheme, mid, which, tf)
                    runs.append((round(mid, 4), st[0]))
                    if st[0]:
                        lo = mid
                    else:
                        hi = mid
                out["results"].append({"scheme": scheme, "k": k, "cells": "%d^3" % cells[k], "which": which,
                                       "stable": round(lo, 4), "unstable": round(hi, 4),
                                       "per_stage_stable": round(lo / len(schemes.SCHEMES[scheme][0]), 4),
                                       "runs": runs})
                print(json.dumps(out["results"][-1]), file=sys.stderr, flush=True)
    print(json.dumps(out), flush=True)
    return 0


def inverse_mass_only(args):
    """dg_cns_inverse_mass alone on args.workload in args.precision: warm-up, then args.steps timed calls
    (the library's per-kernel CUDA events); HBM and ALU rates of the kernel."""
    from paper_1806_03095_gb300 import configs, inputs, roofline
    torch.cuda.set_device(0)
    prec = 1 if args.precision == "mixed" else 0
    cfg = configs.WORKLOADS[args.workload](precision=prec, kernel=0)
    g = configs.make_context(cfg, device=0)
    N = cfg["k"] + 1
    Nc = cfg["ncells"][0] * cfg["ncells"][1] * cfg["ncells"][2]
    R = inputs.uniform(g.shape, 5).to(device=0, dtype=g.rdtype)
    Y = torch.empty_like(R)
    for _ in range(args.warmup):
        g.inverse_mass(R, Y)
    g.timing(True)
    for _ in range(args.steps):
        g.inverse_mass(R, Y)
    kt = g.kernel_times()
    g.timing(False)
    g.status()
    ms = kt["mass"][0] / kt["mass"][1]
    by = 2 * Nc * N ** 3 * 5 * (4 if prec else 8)
    fl = roofline.mass_flops(N) * Nc
    peak = FP32_PEAK_TFLOPS if prec else FP64_PEAK_TFLOPS
    hbm = load_peaks().get("hbm_gbs", 6800.0)
    print(json.dumps({"kernel": "inverse mass alone", "workload": args.workload, "precision": args.precision,
                      "launches": kt["mass"][1], "avg_ms": round(ms, 4), "hbm_gbs": round(by / ms / 1e6, 1),
                      "hbm_frac": round(by / ms / 1e6 / hbm, 4), "tflops": round(fl / ms / 1e9, 3),
                      "alu_frac": round(fl / ms / 1e9 / peak, 4)}), flush=True)
    return 0


def k_sweep(steps=2):
    """Throughput against the polynomial degree (the paper's throughput-versus-k study, Sec. 4.1.2): TGV meshes
    of about 84M DoFs for k = 2..8, 11 and 15 (FP64; k = 3..5 also mixed), fused and face-centric kernels
    (k >= 7: face-centric only; from k = 8 the cell kernel's working set in the global workspace), and FP64
    face-centric with the paper's 3/2 rule on both terms (k = 2..5) and the 2k+1 rule on both terms
    (k = 2..5, 7)."""
    from paper_1806_03095_gb300 import configs
    device = torch.cuda.current_device()
    out = {}

    def run(key, cfg):
        ctx, bufs, dt, ms, _ = time_native(cfg, steps, 3, device)
        nodes = bufs[0].numel() // 5
        n = cfg["ncells"][0]
        out[key] = {"cells": "%d^3" % n, "value": _rate(ms, nodes, steps), "unit": UNIT,
                    "nq": [cfg["nq_conv"], cfg["nq_visc"]]}
        del ctx, bufs
        torch.cuda.empty_cache()

    for k in (2, 3, 4, 5, 6, 7, 8, 11, 15):
        n = max(2, int(round((16.78e6 / (k + 1) ** 3) ** (1.0 / 3.0))))
        for prec in ((0, 1) if k in (3, 4, 5) else (0,)):
            for kern in ((1, 2) if k <= 6 else (2,)):
                key = "k%d_%s_%s" % (k, "fp64" if prec == 0 else "mixed", "fused" if kern == 1 else "faces")
                run(key, configs.tgv(n, k, precision=prec, kernel=kern))
        if k <= 5:
            # the paper's own quadrature: the 3/2 rule on the viscous term too
            cfg = dict(configs.tgv(n, k, precision=0, kernel=2))
            cfg["nq_visc"] = cfg["nq_conv"]
            run("k%d_fp64_faces_3/2_rule_both_terms" % k, cfg)
        if k <= 5 or k == 7:
            cfg = dict(configs.tgv(n, k, precision=0, kernel=2))
            cfg["nq_conv"] = cfg["nq_visc"] = 2 * k + 1
            run("k%d_fp64_faces_2k+1_rule_both_terms" % k, cfg)
    return out


GOLDEN_DISSIPATION = os.path.join(ROOT, "tests", "golden", "tgv8_k5_dissipation.json")


def dissipation_history(t_final=2.0, every=8):
    """-de_k/dt over t in [0, 2] on TGV 8^3, k = 5 (the 8^3 subset of the 40^3 workload), FP64 and mixed, from
    L(U) every `every` steps, against the oracle's curve stored in tests/golden (written by the committed
    oracle-only script beside it, with the same time step and sampling)."""
    from paper_1806_03095_gb300 import api, configs, inputs
    device = torch.cuda.current_device()
    cfg64 = configs.tgv(8, 5, precision=0)
    ref = None
    dt = configs.time_step(cfg64)
    nsteps = int(round(t_final / dt))
    if os.path.exists(GOLDEN_DISSIPATION):
        with open(GOLDEN_DISSIPATION) as f:
            gold = json.load(f)
        dt, every, nsteps = gold["dt"], gold["every"], gold["nsteps"]
        ref = torch.tensor([r[4] for r in gold["samples"]], dtype=torch.float64)
    hist = {}
    for prec in (0, 1):
        g = configs.make_context(dict(cfg64, precision=prec), device=device)
        U = inputs.tgv_state(g.node_coords()).contiguous()
        Ut, dU = g.empty_state(), g.empty_residual()
        vals = []
        for n in range(0, nsteps + 1, every):
            vals.append(float(g.diagnostics(U, g.apply(U, op=api.OP_L))[2]))
            if n + every <= nsteps:
                run_stages(g, every, dt, n * dt, (U, Ut, dU))
        hist[prec] = torch.tensor(vals, dtype=torch.float64)
        del g
    a, b = hist[0], hist[1]

    def rel(x, y):
        return {"rel_l2": float(torch.linalg.norm(x - y) / torch.linalg.norm(y)),
                "rel_max": float((x - y).abs().max() / y.abs().max())}

    out = {"quantity": "-de_k/dt, TGV 8^3, k=5, t in [0, %g], dt %.6g, sampled every %d steps (%d samples)"
                       % (nsteps * dt, dt, every, len(a)),
           "mixed_vs_fp64": rel(b, a), "final_fp64": float(a[-1]), "final_mixed": float(b[-1])}
    if ref is not None and len(ref) == len(a):
        out["fp64_vs_oracle"] = rel(a, ref)
        out["mixed_vs_oracle"] = rel(b, ref)
        out["final_oracle"] = float(ref[-1])
    return out


def adjoint_cost(nsteps=200, every=20, kernel=2, fd_dirs=0, precision=0):
    """Discrete adjoint of TGV 24^3, k = 4: forward nsteps RK(5,4) steps with a checkpoint every `every` steps,
    then the gradient of the final kinetic energy with respect to the initial velocity field (recomputation of
    the segments + stage adjoints).  Reports forward and gradient times and their ratio.  kernel 2: face-centric
    forward and adjoint kernels; kernel 1: element-centric (fused forward, element-centric adjoint kernel).
    fd_dirs > 0 (FP64): central differences of the forward integration (step 1e-6) along that many seeded
    directions (inputs.fd_direction) against the adjoint's directional derivatives.  Returns (report, gradient)."""
    from paper_1806_03095_gb300 import adjoint as adj, configs, inputs
    cfg = configs.WORKLOADS["tgv24_k4"](precision=precision, kernel=kernel)
    g = configs.make_context(cfg)
    xyz = g.node_coords()
    U0 = inputs.tgv_state(xyz)
    rho = U0[:, 0].clone()
    u0 = (U0[:, 1:4] / rho[:, None]).clone().requires_grad_(True)
    cv = cfg["R"] / (cfg["gamma"] - 1.0)
    T0 = (1.0 / cfg["Ma"]) ** 2 / (cfg["gamma"] * cfg["R"])
    dt = configs.time_step(cfg)

    def state(u):
        return torch.cat([rho[:, None], rho[:, None] * u, (rho * (cv * T0 + 0.5 * (u * u).sum(1)))[:, None]], 1)

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    ev[0].record()
    J = adj.kinetic_energy(g, adj.integrate(g, state(u0).contiguous(), nsteps, dt, every))
    ev[1].record()
    J.backward()
    ev[2].record()
    torch.cuda.synchronize()
    fwd = ev[0].elapsed_time(ev[1])
    bwd = ev[1].elapsed_time(ev[2])
    grad = u0.grad.detach().clone()
    out = {"workload": "TGV 24^3, k=4, %s, %d RK(5,4) steps, checkpoint every %d, %s kernels"
           % ("FP64" if precision == 0 else "mixed", nsteps, every, "face-centric" if kernel == 2 else "element-centric"),
           "forward_ms": round(fwd, 1), "gradient_ms": round(bwd, 1), "gradient_over_forward": round(bwd / fwd, 3),
           "grad_norm": float(torch.linalg.norm(grad)), "e_k_final": float(J.detach())}
    if fd_dirs:
        h = 1e-6
        u = u0.detach()

        def J_of(uu):
            return float(g.diagnostics(g.rk_steps(nsteps, dt, 0.0, state(uu).contiguous()))[0])

        checks = []
        for i in range(fd_dirs):
            v = inputs.fd_direction(u, xyz, 1806 + i).to(u.device)
            dJ = float((grad * v).sum())
            fd = (J_of(u + h * v) - J_of(u - h * v)) / (2 * h)
            checks.append({"direction": i, "adjoint": dJ, "central_difference": fd, "rel_err": abs(dJ - fd) / abs(fd)})
        out["fd_check"] = {"step": h, "directions": "inputs.fd_direction seeds 1806.., unit RMS", "results": checks,
                           "max_rel_err": max(c["rel_err"] for c in checks)}
    del g
    torch.cuda.empty_cache()
    return out, grad


def adjoint_extras():
    """The adjoint workload in FP64 (cost, and central differences along 2 directions), element-centric, and in
    the mixed form with its gradient's error against the FP64 gradient."""
    fp64, g64 = adjoint_cost(kernel=2, fd_dirs=2)
    ec, _ = adjoint_cost(kernel=1)
    mixed, g32 = adjoint_cost(kernel=2, precision=1)
    d = g32 - g64
    mixed["gradient_error_vs_fp64"] = {"rel_l2": float(torch.linalg.norm(d) / torch.linalg.norm(g64)),
                                       "rel_max": float(d.abs().max() / g64.abs().max())}
    return fp64, ec, mixed


# -- CPU oracle --------------------------------------------------------------------------------------
def oracle_sample(cfg, target_s=12.0, n=None):
    """Time the FP64 oracle's L(U) on a bounded sample of the workload: an n^3-cell periodic TGV mesh (default
    16^3, 8^3 above k = 3) with the workload's k and quadrature (same per-node work), repeated until ~target_s
    seconds, on torch's current CPU thread count."""
    from oracle import physics as ph
    from oracle.mesh import BoxMesh
    from oracle.operator import DGOperator
    from paper_1806_03095_gb300 import inputs
    if n is None:
        n = 16 if cfg["k"] <= 3 else 8
    mesh = BoxMesh((n, n, n), cfg["lo"], cfg["hi"], cfg["periodic"], cfg["k"])
    phys = ph.Physics.from_numbers(cfg["Re"], cfg["Pr"], cfg["Ma"], cfg["gamma"], cfg["R"])
    op = DGOperator(mesh, phys, cfg["nq_conv"], cfg["nq_visc"])
    U = inputs.tgv_state(op.xyz)
    op.L(U)
    reps, t0 = 0, time.perf_counter()
    while True:
        op.L(U)
        reps += 1
        el = time.perf_counter() - t0
        if el > target_s or reps >= 50:
            break
    dofs = 5 * mesh.Nc * mesh.n ** 3
    return {"value": round(dofs * reps / el / 1e9, 6), "unit": UNIT, "cores": torch.get_num_threads(),
            "kind": "oracle", "sample": "oracle L(U) (naive full-matrix FP64 quadrature, PyTorch CPU) on a %d^3-cell "
            "periodic TGV mesh, k=%d, %d evaluations in %.1f s" % (n, cfg["k"], reps, el), "seconds": round(el, 2)}


def oracle_rk_steps(max_steps=10, budget_s=20.0):
    """The oracle's RK(5,4) steps on the Taylor-Green vortex 8^3, k = 3 (the small parity workload): up to
    max_steps steps, stopping once budget_s seconds have passed; GDoF/s per stage."""
    from oracle import physics as ph, rk as ork
    from oracle.mesh import BoxMesh
    from oracle.operator import DGOperator
    from paper_1806_03095_gb300 import configs, inputs
    cfg = configs.tgv(8, 3)
    mesh = BoxMesh(cfg["ncells"], cfg["lo"], cfg["hi"], cfg["periodic"], cfg["k"])
    op = DGOperator(mesh, ph.Physics.from_numbers(cfg["Re"], cfg["Pr"], cfg["Ma"], cfg["gamma"], cfg["R"]),
                    cfg["nq_conv"], cfg["nq_visc"])
    U = inputs.tgv_state(op.xyz)
    dt = configs.time_step(cfg)
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps:
        U = ork.step(lambda V, t: op.L(V), U, dt, steps * dt)
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    dofs = 5 * mesh.Nc * mesh.n ** 3
    return {"value": round(dofs * ork.STAGES * steps / el / 1e9, 6), "unit": UNIT, "cores": torch.get_num_threads(),
            "sample": "%d RK(5,4) steps of the oracle on TGV 8^3, k=3 in %.1f s" % (steps, el), "steps": steps}


def cpu_baseline(cfg):
    """The naive FP64 oracle on the host cores, a reported baseline (not the target): L(U) on a bounded sample
    with every core (nproc), the same on one core, and RK(5,4) steps on TGV 8^3, k = 3."""
    threads = torch.get_num_threads()
    nproc = os.cpu_count() or 1
    try:
        torch.set_num_threads(nproc)
        out = oracle_sample(cfg)
        torch.set_num_threads(1)
        out["single_core"] = oracle_sample(cfg, target_s=8.0, n=8 if cfg["k"] <= 3 else 4)
        torch.set_num_threads(nproc)
        out["rk_steps_tgv8_k3"] = oracle_rk_steps()
    finally:
        torch.set_num_threads(threads)
    out["nproc"] = nproc
    out["label"] = "naive FP64 oracle: a reported baseline, not the target"
    out["paper_context"] = ("the paper's node: 0.33 GDoF/s per stage at k=3 with the 3/2 rule on 28 Haswell cores "
                            "(FP64, PID table; context, not the target)")
    return out


def reference_arm(args, ws, rank):
    if rank != 0:
        return 0
    from paper_1806_03095_gb300 import configs
    cfg = configs.WORKLOADS[args.workload]()
    per = []
    samples = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample(cfg, target_s=2.0)
        if i >= args.warmup:
            per.append(r["value"])
            samples.append(r["seconds"])
    value = statistics.mean(per)
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(samples), 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "Taylor-Green vortex, k=%d, nq_conv=%d, nq_visc=%d; each step a bounded sample: "
                      "one or more oracle L(U) evaluations on a 16^3-cell periodic mesh" % (
                          cfg["k"], cfg["nq_conv"], cfg["nq_visc"])},
           "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": torch.get_num_threads(),
                            "kind": "oracle", "sample": "oracle L(U) on a 16^3-cell TGV mesh, ~2 s per step"},
           "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
