"""Benchmark of the DiscoMatch dual / primal hot path on one GB300 (or N replicas).

A step = the whole hot path on one synthetic shape pair: pair costs and top-k candidate
mask on the device, host compilation of ILP (P) into BDDs and upload, dual iterations
until the lower bound moves less than 1e-6 (relative) over 20 iterations, rounding to a
feasible matching. Inputs (features) are resident in HBM when the timed region starts.

Prints one JSON line: value = BDD node-updates per second over the whole step (one
node-update = one node processed in one half-pass), e2e = the same through the C ABI
with host buffers (features copied in, matching copied out, inside the timed region),
roofline of the dominant kernel (the half-pass kernels), a CPU baseline (the FP64
oracle on host cores) and sampled clocks.

--impl reference times the FP64 oracle itself (the reference arm of this project).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BDD node-updates/s (whole step: costs, candidates, build, dual to converged bound, rounding)"
UNIT = "node-updates/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


HALFPASS_SOURCES = ("kernels.cu", "device_util.cuh", "kernels.h")


def _traffic(workload: str, split_chunk: int):
    """DRAM bytes per half-pass launch from the committed ncu summary of this workload, or
    None when the half-pass sources changed since the counters were taken (sha256 of
    kernels.cu, device_util.cuh and kernels.h, in that order)."""
    profiles = {"icosphere4-5120T-top16": "halfpass_icosphere4-5120T-top16.md",
                "batch64-uneven": "halfpass_batch64-uneven.md"}
    if workload not in profiles or split_chunk != 32:
        return None
    return _profile_traffic(profiles[workload])


def _profile_traffic(profile: str):
    import hashlib
    path = os.path.join(ROOT, "profiles", profile)
    csrc = os.path.join(ROOT, "paper_2310_08230_gb300", "csrc")
    if not os.path.exists(path):
        return None
    h = hashlib.sha256()
    for name in HALFPASS_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    h = h.hexdigest()[:16]
    fields = {}
    with open(path) as f:
        for ln in f:
            if ":" in ln and ln.split(":")[0] in ("sources_sha256_16", "traffic_bytes_per_launch"):
                k, v = ln.split(":", 1)
                fields[k] = v.strip()
    if fields.get("sources_sha256_16") != h:
        return None
    return int(fields["traffic_bytes_per_launch"])


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self):
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", dev, f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def flush_l2(torch, buf):
    buf.add_(1.0)  # 256 MB write, larger than the 129 MB L2


def workload(name):
    from synth import instances as I

    if name == "config3":
        return I.config3()
    if name == "config2":
        return I.config2()
    if name == "config1":
        return I.config1()
    raise ValueError(name)


def replica_throughput(ms: float, updates_per_rank: float, world: int, device: str) -> tuple[float, float]:
    """Replicas (one independent instance per rank, no data-path collective): the job's step
    time is the slowest rank's, its throughput all ranks' updates over that time."""
    if world > 1:
        import torch
        import torch.distributed as dist

        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, updates_per_rank * world / (ms / 1e3)


def gpu_arm(args):
    import torch

    from paper_2310_08230_gb300 import _lib as L
    from paper_2310_08230_gb300.api import _mesh, default_opts

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    lib = L.lib()
    inst = workload(args.config)
    stream = torch.cuda.Stream()
    sptr = int(stream.cuda_stream)
    FX_h = np.ascontiguousarray(inst.FX)
    FY_h = np.ascontiguousarray(inst.FY)
    FX_pin = torch.from_numpy(FX_h).pin_memory()
    FY_pin = torch.from_numpy(FY_h).pin_memory()
    FX = FX_pin.cuda()
    FY = FY_pin.cuda()
    nvx, nvy, dim = inst.X.nv, inst.Y.nv, inst.FX.shape[1]
    d = torch.empty((nvx, nvy), dtype=torch.float32, device="cuda")
    allowed = torch.empty((nvx, nvy), dtype=torch.uint8, device="cuda")
    mx, tx = _mesh(inst.X.T, nvx)
    my, ty = _mesh(inst.Y.T, nvy)
    # replicas on one node share its host cores: each rank's host compiler gets its share
    opts = default_opts(stream=sptr, lb_every=20, conv_rel_tol=1e-6, split_chunk=args.split_chunk,
                        host_threads=max(1, (os.cpu_count() or 1) // world) if world > 1 else 0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    max_iters = args.max_iters

    def step(e2e: bool, stats: dict):
        t0 = time.perf_counter()
        # end to end: the features go in as pinned host buffers through the C ABI (the
        # library copies them to the device); otherwise they are resident in HBM
        fx, fy = (FX_pin, FY_pin) if e2e else (FX, FY)
        L.check(lib.disco_pair_costs(fx.data_ptr(), fy.data_ptr(), nvx, nvy, dim, d.data_ptr(), sptr), "pair_costs")
        L.check(lib.disco_candidates(d.data_ptr(), nvx, nvy, inst.topk, ctypes.byref(mx), ctypes.byref(my),
                                     allowed.data_ptr(), sptr), "candidates")
        t1 = time.perf_counter()
        h = ctypes.c_void_p()
        L.check(lib.disco_build(ctypes.byref(mx), ctypes.byref(my), d.data_ptr(), allowed.data_ptr(),
                                ctypes.byref(opts), ctypes.byref(h)), "build")
        info = L.disco_info_t()
        lib.disco_info(h, ctypes.byref(info))
        # dual to a converged bound: blocks of lb_every iterations, half-pass time on events
        lb_prev = ctypes.c_double()
        L.check(lib.disco_lower_bound(h, ctypes.byref(lb_prev)), "lb")
        lb = ctypes.c_double()
        iters, dual_ms, blocks = 0, 0.0, []
        t_dual0 = time.perf_counter()
        while iters < max_iters:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L.check(lib.disco_dual(h, 20), "dual")
            e1.record(stream)
            L.check(lib.disco_lower_bound(h, ctypes.byref(lb)), "lb")
            blocks.append(e0.elapsed_time(e1))
            dual_ms += blocks[-1]
            iters += 20
            if abs(lb.value - lb_prev.value) < 1e-6 * abs(lb.value):
                break
            lb_prev.value = lb.value
        t_conv = (time.perf_counter() - t_dual0) * 1e3
        x = np.zeros(info.nvars, np.uint8)
        cost = ctypes.c_double()
        t3 = time.perf_counter()
        rc = lib.disco_primal(h, x.ctypes.data, info.nvars, ctypes.byref(cost))
        t4 = time.perf_counter()
        lib.disco_info(h, ctypes.byref(info))
        stats.update(nnodes=info.nnodes, nslots=info.nslots, nvars_free=info.nvars_free, nvars=info.nvars,
                     iters=info.iterations, conv_iters=iters, lb=lb.value, primal=cost.value, primal_ok=rc == 0,
                     dual_ms=dual_ms, conv_ms=t_conv, build_ms=info.build_ms, bytes_per_iter=info.bytes_per_iter,
                     # the kernel's own launch time: the blocks after the first (the first also holds
                     # the initial backward pass, the launch-geometry trials and the graph capture)
                     kernel_blocks_ms=blocks[1:] if len(blocks) > 1 else blocks, kernel_block_iters=20,
                     ntiles=info.ntiles, max_layers=info.max_layers, upload_ms=info.upload_ms,
                     launch_geometry=info.launch_geometry,
                     costs_candidates_ms=(t1 - t0) * 1e3, build_call_ms=(t_dual0 - t1) * 1e3,
                     primal_ms=(t4 - t3) * 1e3)
        t5 = time.perf_counter()
        lib.disco_free(h)
        stats["free_ms"] = (time.perf_counter() - t5) * 1e3
        return x

    def timed(e2e: bool):
        stats = {}
        flush_l2(torch, flush)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        step(e2e, stats)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1), stats

    for _ in range(args.warmup):
        timed(False)
    times, stats_all = [], []
    launches0 = lib.disco_kernel_launches()
    with Clocks() as clk:
        for _ in range(args.steps):
            t, st = timed(False)
            times.append(t)
            stats_all.append(st)
    launches = lib.disco_kernel_launches() - launches0  # whole timed region (all steps)
    e2e_times = [timed(True)[0] for _ in range(max(1, min(args.steps, 3)))]
    st = stats_all[-1]
    updates = 2.0 * st["nnodes"] * st["iters"]
    ms, value = replica_throughput(float(np.mean(times)), updates, world, "cuda")
    e2e_ms = float(np.mean(e2e_times))
    kb = [b for x in stats_all for b in x["kernel_blocks_ms"]]
    half_pass_ms = sum(kb) / (2 * st["kernel_block_iters"] * len(kb))
    alg_bytes = st["bytes_per_iter"] / 2.0
    peak, kind = _peaks()
    achieved = alg_bytes / (half_pass_ms / 1e3) / 1e9
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": inst.name, "nvars": st["nvars"], "nvars_free": st["nvars_free"],
                   "bdd_slots": st["nslots"], "bdd_nodes": st["nnodes"], "max_layers": st["max_layers"],
                   "warps_per_block_autotuned": st["launch_geometry"],
                   "split_chunk": args.split_chunk, "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "ms_to_converged_bound": st["conv_ms"], "converged_iters": st["conv_iters"],
        "dual_node_updates_per_s": 2.0 * st["nnodes"] * st["conv_iters"] / (st["dual_ms"] / 1e3),
        "build_ms": st["build_ms"], "lower_bound": st["lb"], "primal_cost": st["primal"],
        "breakdown_ms": {k: round(st[k], 3) for k in ("costs_candidates_ms", "build_call_ms", "build_ms", "upload_ms",
                                                      "conv_ms", "primal_ms", "free_ms")},
        "primal_feasible": st["primal_ok"],
        "rel_gap": (st["primal"] - st["lb"]) / st["primal"] if st["primal"] else None,
        "e2e": {"value": updates / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(FX_h.nbytes + FY_h.nbytes), "d2h_bytes_per_step": int(st["nvars"]) + 8},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": _traffic(inst.name, args.split_chunk), "kernel": "MMA half-pass (k_forward_fused / k_backward_fused over every width class; the deferred averaging happens in the same launch)",
                     "alg_bytes_per_launch": alg_bytes, "launch_ms": half_pass_ms, "peak_kind": kind,
                     "launch_timing": "CUDA events on the solver stream around each step's dual blocks after "
                                      "the first (CUDA-graph replays of the half-pass kernels); the first block "
                                      "also holds the initial backward pass, the launch-geometry trials and "
                                      "the graph capture"},
        "clocks": clk.summary(),
    }
    # the comparison sections and the CPU baseline run on single-GPU runs only
    if world == 1 and not args.no_batched:
        line["batched"] = batched_vs_single(torch)
    if world == 1 and not args.no_differentiated:
        line["differentiated"] = differentiated(torch)
    if world == 1 and not args.no_quasi_newton:
        from synth import instances as I

        line["quasi_newton"] = quasi_newton_vs_mma(torch, [inst, I.symmetric_pair(3)], args.split_chunk)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
        if "differentiated" in line:
            line["differentiated"]["plain_torch_reference_gradient"] = cpu_baseline_differentiated()
    print(json.dumps(line), flush=True)


def quasi_newton_vs_mma(torch, insts, split_chunk: int) -> dict:
    """Time to the converged bound with quasi-Newton steps (Alg. 1, memory 5, one step per
    lb_every = 20 MMA iterations) against MMA alone (host build excluded), per workload: the
    bench workload, whose relaxation is tight after a few dozen iterations, and a half-turn
    symmetric icosphere pair whose dual needs hundreds."""
    from paper_2310_08230_gb300.api import Solver, candidates, pair_costs

    res = {}
    for inst in insts:
        FX = torch.from_numpy(inst.FX).cuda()
        FY = torch.from_numpy(inst.FY).cuda()
        d = pair_costs(FX, FY)
        al = candidates(d, inst.topk, inst.X.T, inst.Y.T) if inst.topk else None
        out = {}
        for name, kw in (("mma", {}), ("qn", {"qn_memory": 5})):
            s = Solver(inst.X.T, inst.Y.T, d, al, split_chunk=split_chunk, **kw)
            out["bdd_nodes"] = s.info()["nnodes"]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            n, lb, ok = s.converge(20000)
            t1 = time.perf_counter()
            out[name] = {"ms_to_converged_bound": (t1 - t0) * 1e3, "iterations": n, "lower_bound": lb,
                         "converged": ok}
            s.close()
        res[inst.name] = out
    return res


def differentiated(torch, n_pairs: int = 8, iters: int = 50, every: int = 10) -> dict:
    """Learned costs through the solver: 8 pairs of 1280-triangle icospheres, raw 128-d
    features -> 2-layer MLP (128-256-64, ReLU) -> squared distances -> top-16 candidates
    (held fixed) -> bound after 50 iterations; its gradient w.r.t. the MLP parameters by the
    adjoint kernels (checkpoint every 10 iterations), timed beside plain solves of the same
    pairs. (The gradient's values are checked by the GPU tests against the FP64 replica and
    against FP64 central differences of the oracle.)"""
    from paper_2310_08230_gb300.api import Solver, candidates
    from paper_2310_08230_gb300.autograd import dual_bounds
    from synth import instances as I

    insts = I.config5(n_pairs)
    params = [torch.tensor(p, device="cuda", requires_grad=True) for p in I.mlp_params()]
    FX = [torch.from_numpy(i.FX).cuda() for i in insts]
    FY = [torch.from_numpy(i.FY).cuda() for i in insts]
    meshes = [(i.X.T, i.Y.T) for i in insts]

    def mlp(F, ps):
        W1, b1, W2, b2 = ps
        return torch.relu(F @ W1.T + b1) @ W2.T + b2

    def costs(ps):
        out = []
        for fx, fy in zip(FX, FY):
            a, b = mlp(fx, ps), mlp(fy, ps)
            out.append(((a[:, None, :] - b[None, :, :]) ** 2).sum(-1))
        return out

    with torch.no_grad():
        masks = [candidates(d, 16, i.X.T, i.Y.T) for d, i in zip(costs(params), insts)]

    def bounds_plain(ps):
        with torch.no_grad():
            ds = costs(ps)
            s = Solver.batch([(TX, TY, d, m) for d, (TX, TY), m in zip(ds, meshes, masks)], normalize_costs=0)
            s.dual(iters)
            lbs = s.lower_bounds()
            s.close()
        return lbs

    bounds_plain(params)  # warm-up (build caches, autotuner paths)
    # one untimed forward + backward: the first gradient call takes its replay memory from
    # the device pool (kept for every later handle, as in a training loop)
    dual_bounds(costs(params), meshes, masks, iters, every, normalize_costs=0).sum().backward()
    for p in params:
        p.grad = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbs = dual_bounds(costs(params), meshes, masks, iters, every, normalize_costs=0)
    loss = lbs.sum()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    # the plain single-instance path on the same pairs (no recording, no gradient)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    with torch.no_grad():
        ds = costs(params)
        plain = []
        for d, (TX, TY), m in zip(ds, meshes, masks):
            s = Solver(TX, TY, d, m, normalize_costs=0)
            s.dual(iters)
            plain.append(s.lower_bound())
            s.close()
    torch.cuda.synchronize()
    t4 = time.perf_counter()
    return {
        "pairs": n_pairs, "iters": iters, "checkpoint_every": every, "mlp": "128-256-64 relu",
        "params": int(sum(p.numel() for p in params)),
        "bound_sum": float(loss.detach()), "plain_bound_sum": float(np.sum(plain)),
        "fwd_ms": (t1 - t0) * 1e3, "bwd_ms": (t2 - t1) * 1e3,
        "plain_one_by_one_ms": (t4 - t3) * 1e3,
        "note": "steady state (after one untimed forward+backward); times include the host compiler",
    }


def batched_vs_single(torch, iters: int = 300, n_pairs: int = 64, split_chunk: int = 32,
                      one_by_one: bool = True, pipeline_groups=(2, 3, 4)) -> dict:
    """64 uneven pairs: one batched handle against the same pairs solved one after another.

    Both sides run the whole path per pair (pair costs, candidates, build, `iters` dual
    iterations, bound, rounding) on device-resident features; times are CUDA-event times on
    one stream with host work in between included. The batch's last 20 iterations are also
    timed on their own (CUDA events, graph replays of the half-pass launches): with 1.8 GB of
    BDD tables, far beyond L2, that is the batch's HBM roofline point."""
    from paper_2310_08230_gb300 import _lib as L
    from paper_2310_08230_gb300.api import _mesh, balanced_groups, default_opts
    from synth import instances as I

    lib = L.lib()
    insts = I.config4(n_pairs)
    stream = torch.cuda.Stream()
    sptr = int(stream.cuda_stream)
    feats = [(torch.from_numpy(i.FX).cuda(), torch.from_numpy(i.FY).cuda()) for i in insts]
    ds = [torch.empty((i.X.nv, i.Y.nv), dtype=torch.float32, device="cuda") for i in insts]
    al = [torch.empty((i.X.nv, i.Y.nv), dtype=torch.uint8, device="cuda") for i in insts]
    meshes = [(_mesh(i.X.T, i.X.nv), _mesh(i.Y.T, i.Y.nv)) for i in insts]
    opts = default_opts(stream=sptr, split_chunk=split_chunk)

    def costs(k):
        i = insts[k]
        (FX, FY), d, a = feats[k], ds[k], al[k]
        (mx, _), (my, _) = meshes[k]
        L.check(lib.disco_pair_costs(FX.data_ptr(), FY.data_ptr(), i.X.nv, i.Y.nv, i.FX.shape[1], d.data_ptr(), sptr),
                "pair_costs")
        L.check(lib.disco_candidates(d.data_ptr(), i.X.nv, i.Y.nv, i.topk, ctypes.byref(mx), ctypes.byref(my),
                                     a.data_ptr(), sptr), "candidates")

    phases = {}
    steady = {}

    def mark(name, t0):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        phases[name] = phases.get(name, 0.0) + (t1 - t0) * 1e3
        return t1

    def batched():
        t = time.perf_counter()
        for k in range(n_pairs):
            costs(k)
        t = mark("costs_candidates_ms", t)
        MX = (L.disco_mesh * n_pairs)(*[m[0][0] for m in meshes])
        MY = (L.disco_mesh * n_pairs)(*[m[1][0] for m in meshes])
        dp = (ctypes.c_void_p * n_pairs)(*[d.data_ptr() for d in ds])
        ap = (ctypes.c_void_p * n_pairs)(*[a.data_ptr() for a in al])
        h = ctypes.c_void_p()
        L.check(lib.disco_build_batch(n_pairs, MX, MY, ctypes.cast(dp, ctypes.c_void_p), ctypes.cast(ap, ctypes.c_void_p),
                                      ctypes.byref(opts), ctypes.byref(h)), "build_batch")
        t = mark("build_ms", t)
        info = L.disco_info_t()
        lib.disco_info(h, ctypes.byref(info))
        L.check(lib.disco_dual(h, iters - 20), "dual")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.check(lib.disco_dual(h, 20), "dual")
        e1.record(stream)
        e1.synchronize()
        steady["half_pass_ms"] = e0.elapsed_time(e1) / 40.0
        steady["alg_bytes"] = info.bytes_per_iter / 2.0
        lbs = np.zeros(n_pairs)
        L.check(lib.disco_lower_bounds(h, lbs.ctypes.data_as(L.c_double_p), n_pairs), "lbs")
        t = mark("dual_ms", t)
        x = np.zeros(info.nvars, np.uint8)
        cs = np.zeros(n_pairs)
        st = np.zeros(n_pairs, np.int32)
        lib.disco_primal_batch(h, x.ctypes.data, info.nvars, cs.ctypes.data_as(L.c_double_p),
                               st.ctypes.data_as(L.c_int32_p), n_pairs)
        t = mark("primal_ms", t)
        lib.disco_free(h)
        mark("free_ms", t)
        return info.nnodes, lbs, cs, st

    # pipelined: the pairs in G batched stores of about equal size (X triangles x top-k, largest
    # first onto the lightest group), each on its own stream; the host compiles store g + 1
    # while the GPU runs store g's dual iterations (enqueued graph replays), then all round
    gstreams = [torch.cuda.Stream() for _ in range(max(pipeline_groups or (1,)))]
    # no launch-geometry autotuning: its timed trials would wait behind the previous store's
    # dual on the GPU (every geometry gives the same results)
    gopts = [default_opts(stream=int(st.cuda_stream), split_chunk=split_chunk, autotune=0) for st in gstreams]

    def pipelined(G):
        for k in range(n_pairs):
            costs(k)
        torch.cuda.synchronize()  # the costs (on `stream`) are complete before any build reads them
        members = balanced_groups([insts[k].X.nt * insts[k].topk for k in range(n_pairs)], G)
        hs = []
        for g, m in enumerate(members):
            MX = (L.disco_mesh * len(m))(*[meshes[k][0][0] for k in m])
            MY = (L.disco_mesh * len(m))(*[meshes[k][1][0] for k in m])
            dp = (ctypes.c_void_p * len(m))(*[ds[k].data_ptr() for k in m])
            ap = (ctypes.c_void_p * len(m))(*[al[k].data_ptr() for k in m])
            h = ctypes.c_void_p()
            L.check(lib.disco_build_batch(len(m), MX, MY, ctypes.cast(dp, ctypes.c_void_p),
                                          ctypes.cast(ap, ctypes.c_void_p), ctypes.byref(gopts[g]), ctypes.byref(h)),
                    "build_batch")
            L.check(lib.disco_dual(h, iters), "dual")  # enqueued; the next group compiles meanwhile
            hs.append(h)
        nodes = 0
        lbs, cs, st = np.zeros(n_pairs), np.zeros(n_pairs), np.zeros(n_pairs, np.int32)
        for m, h in zip(members, hs):
            info = L.disco_info_t()
            lib.disco_info(h, ctypes.byref(info))
            nodes += info.nnodes
            lbm, csm, stm = np.zeros(len(m)), np.zeros(len(m)), np.zeros(len(m), np.int32)
            L.check(lib.disco_lower_bounds(h, lbm.ctypes.data_as(L.c_double_p), len(m)), "lbs")
            x = np.zeros(info.nvars, np.uint8)
            lib.disco_primal_batch(h, x.ctypes.data, info.nvars, csm.ctypes.data_as(L.c_double_p),
                                   stm.ctypes.data_as(L.c_int32_p), len(m))
            lib.disco_free(h)
            lbs[m], cs[m], st[m] = lbm, csm, stm
        return nodes, lbs, cs, st

    def single():
        nodes, lbs, cs, st = 0, [], [], []
        for k in range(n_pairs):
            costs(k)
            (mx, _), (my, _) = meshes[k]
            h = ctypes.c_void_p()
            L.check(lib.disco_build(ctypes.byref(mx), ctypes.byref(my), ds[k].data_ptr(), al[k].data_ptr(),
                                    ctypes.byref(opts), ctypes.byref(h)), "build")
            info = L.disco_info_t()
            lib.disco_info(h, ctypes.byref(info))
            nodes += info.nnodes
            L.check(lib.disco_dual(h, iters), "dual")
            lb = ctypes.c_double()
            L.check(lib.disco_lower_bound(h, ctypes.byref(lb)), "lb")
            x = np.zeros(info.nvars, np.uint8)
            c = ctypes.c_double()
            rc = lib.disco_primal(h, x.ctypes.data, info.nvars, ctypes.byref(c))
            lib.disco_free(h)
            lbs.append(lb.value)
            cs.append(c.value)
            st.append(rc)
        return nodes, np.array(lbs), np.array(cs), np.array(st)

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    timed(batched)  # warm-up (pool, modules)
    phases.clear()
    tb, (nodes, lbs_b, cs_b, st_b) = timed(batched)
    breakdown = {k: round(v, 1) for k, v in phases.items()}
    upd = 2.0 * nodes * iters
    peak, kind = _peaks()
    achieved = steady["alg_bytes"] / (steady["half_pass_ms"] / 1e3) / 1e9
    out = {"pairs": n_pairs, "iters": iters, "bdd_nodes": int(nodes), "batched_ms": tb,
           "batched_node_updates_per_s": upd / (tb / 1e3), "feasible_batched": int((st_b == 0).sum()),
           "batched_breakdown_ms": breakdown,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "alg_bytes_per_launch": steady["alg_bytes"], "launch_ms": steady["half_pass_ms"],
                        "peak_kind": kind,
                        "traffic": _traffic("batch64-uneven", split_chunk) if n_pairs == 64 else None,
                        "kernel": "MMA half-pass over all 64 pairs (every width-class launch of one half-pass)",
                        "launch_timing": "CUDA events around the batch's last 20 iterations (graph replays)"}}
    pipe = {}
    for G in pipeline_groups or ():
        tp, (nodes_p, lbs_p, cs_p, st_p) = timed(lambda: pipelined(G))
        pipe[str(G)] = {"ms": tp, "node_updates_per_s": upd / (tp / 1e3), "feasible": int((st_p == 0).sum()),
                        "max_rel_bound_diff_vs_batched": float(np.max(np.abs(lbs_p - lbs_b) /
                                                                      np.maximum(np.abs(lbs_b), 1e-12)))}
    if pipe:
        out["pipelined"] = {"groups": pipe, "note": "G batched stores on their own streams; the host compiles store "
                                                    "g + 1 while the GPU runs store g's dual (costs and candidates "
                                                    "of all pairs first, rounding of all stores last)"}
    if one_by_one:
        ts, (nodes_s, lbs_s, cs_s, st_s) = timed(single)
        out.update({"one_by_one_ms": ts, "one_by_one_node_updates_per_s": upd / (ts / 1e3), "speedup": ts / tb,
                    "feasible_one_by_one": int((st_s == 0).sum()),
                    "max_rel_bound_diff": float(np.max(np.abs(lbs_b - lbs_s) / np.maximum(np.abs(lbs_s), 1e-12)))})
        for G, r in pipe.items():
            r["speedup_vs_one_by_one"] = ts / r["ms"]
    return out


def _oracle_workload(config: str, split_chunk: int):
    """The FP64 oracle's decomposition of the bench workload (built untimed)."""
    from oracle import bdd as B
    from oracle import problem as P
    from oracle import solver as S

    t0 = time.perf_counter()
    inst = workload(config)
    prob, d, allowed = P.make_problem(inst)
    fixed, const = P.presolve(prob)
    dec = B.decompose(prob, fixed, const, split_chunk)
    return inst, dec, S.DualOracle(dec), time.perf_counter() - t0


def cpu_baseline_differentiated(iters_sample: int = 4, iters: int = 50, n_pairs: int = 8) -> dict:
    """The plain-PyTorch unrolled reference gradient (the FP64 autograd replica of the dual
    iterations, on the host cores) for the differentiated workload, on a bounded sample: one
    of its pairs for `iters_sample` of its iterations, scaled to all pairs and iterations.
    The pair costs come from the seeded MLP in FP64; its Jacobian is not timed."""
    import torch

    from oracle import bdd as B
    from oracle import grad as G
    from oracle import problem as P
    from synth import instances as I

    inst = I.config5(1)[0]
    W1, b1, W2, b2 = [torch.tensor(p, dtype=torch.float64) for p in I.mlp_params()]
    fa = torch.relu(torch.tensor(inst.FX, dtype=torch.float64) @ W1.T + b1) @ W2.T + b2
    fb = torch.relu(torch.tensor(inst.FY, dtype=torch.float64) @ W1.T + b1) @ W2.T + b2
    d = ((fa[:, None, :] - fb[None, :, :]) ** 2).sum(-1).numpy().astype(np.float32).astype(np.float64)
    allowed = P.candidate_pairs(d, inst.topk, inst.X.T, inst.Y.T)
    prob = P.build_problem(inst.X.T, inst.Y.T, d, allowed, normalize=False)
    fixed, const = P.presolve(prob)
    dec = B.decompose(prob, fixed, const, 0)
    c = d[prob.vm, prob.vn].mean(axis=1)
    t0 = time.perf_counter()
    G.bound_and_grad(dec, c, fixed, iters_sample)
    dt = time.perf_counter() - t0
    total = dt * (iters / iters_sample) * n_pairs
    return {"value": total * 1e3, "unit": "ms per bound-and-gradient of the 8-pair, 50-iteration workload",
            "cores": torch.get_num_threads(), "kind": "oracle (plain PyTorch FP64 unrolled autograd)",
            "sample": f"pair 0 of 8 ({dec.n_nodes} BDD nodes), {iters_sample} of {iters} iterations in "
                      f"{dt:.1f} s, scaled by {iters / iters_sample:.1f} x {n_pairs}"}


def cpu_baseline(args) -> dict:
    """FP64 oracle iterations on the host cores over the bench workload's full decomposition:
    node-updates/s on a bounded sample (as many whole iterations as fit the time)."""
    inst, dec, o, setup_s = _oracle_workload(args.config, args.split_chunk)
    t0 = time.perf_counter()
    n = 0
    while n == 0 or time.perf_counter() - t0 < args.cpu_seconds:
        o.iterate(1)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": 2.0 * dec.n_nodes * n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{inst.name}, chunk {args.split_chunk}: {n} FP64 deferred-MMA iterations over all "
                      f"{dec.n_nodes} BDD nodes in {dt:.1f} s, single-threaded C core; the oracle's Python "
                      f"build ({setup_s:.0f} s) is not counted"}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    inst, dec, o, setup_s = _oracle_workload(args.config, args.split_chunk)
    iters = 1
    for _ in range(args.warmup):
        o.iterate(iters)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.iterate(iters)
        times.append((time.perf_counter() - t0) * 1e3)
    ms = float(np.mean(times))
    value = 2.0 * dec.n_nodes * iters / (ms / 1e3)
    sample = (f"{inst.name}, chunk {args.split_chunk}: {iters} FP64 deferred-MMA iteration per step over all "
              f"{dec.n_nodes} BDD nodes, single-threaded C core; the oracle's Python build ({setup_s:.0f} s) "
              "is not counted")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": inst.name, "bdd_nodes": int(dec.n_nodes), "split_chunk": args.split_chunk},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--config", default="config3")
    ap.add_argument("--split-chunk", type=int, default=32)
    ap.add_argument("--max-iters", type=int, default=20000)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-differentiated", action="store_true")
    ap.add_argument("--no-quasi-newton", action="store_true")
    ap.add_argument("--only", choices=["batched", "differentiated", "quasi_newton"],
                    help="run one comparison section alone (for profiling) and print its object")
    ap.add_argument("--skip-one-by-one", action="store_true", help="with --only batched: the batched handle only")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    else:
        import __graft_entry__

        __graft_entry__.build()
        if args.only:
            import torch

            if args.only == "batched":
                res = batched_vs_single(torch, one_by_one=not args.skip_one_by_one)
            elif args.only == "differentiated":
                res = differentiated(torch)
            else:
                from synth import instances as I

                res = quasi_newton_vs_mma(torch, [workload(args.config), I.symmetric_pair(3)], args.split_chunk)
            print(json.dumps({"only": args.only, args.only: res}), flush=True)
            return
        gpu_arm(args)


if __name__ == "__main__":
    main()
