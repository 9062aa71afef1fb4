#!/usr/bin/env python
"""Throughput benchmark of the fused D2Q9/D2Q5 MRT porous-media LB step.

Workload (default): side-heated porous cavity of 4096 x 4096 nodes, Ra = 1e6,
Da = 1e-4, porosity 0.4, Pr = 1, FP32 deviations (one "step" = one time step
of the whole lattice).  Prints ONE JSON line (rank 0).

  value     coupled MLUPS (nodes x steps / s / 1e6), device-resident state,
            CUDA events on the library's stream around exactly --steps steps.
  roofline  the step kernel (the only kernel in the timed region) against the
            measured HBM copy bandwidth: algorithmic bytes = every population
            read once and written once (FP32: 28 x 4 = 112 B per node-step).
  e2e       same metric through the public API from host memory: the initial
            state is loaded from a host checkpoint (H2D), the Nusselt numbers
            of every step are written to pinned host memory (D2H, one
            lbm_step_nusselt call), the final state is saved to host (D2H);
            host wall clock.  per_step_calls: the same job with one lbm_step
            and one lbm_nusselt_async call per step.
  cpu_baseline  the FP64 CPU oracle, as it stands, on the host cores, on a
            bounded number of steps of the same lattice.
  variants  FP64 and FP16-storage throughput of the same lattice, and the mean
            Nusselt number of FP32 / FP16 against FP64 at equal step counts.

--impl reference times the oracle instead (the CPU reference of the method).
Under torchrun (WORLD_SIZE > 1) every rank runs an independent replica of the
workload on its own GPU (the cavity path has no data-path collective here);
value = all ranks' node updates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled MLUPS & % HBM roofline, FP32 vs FP64 at stated Nu error; adjoint MLUPS"
# every population read once and written once: FP64 14 x 8 B, FP32 14 x 4 B,
# FP16 variant 9 x 2 B (flow) + 5 x 4 B (thermal), each way
# FP32 variants also read and write the node's temperature frame (1 byte, FP32 frame: 4)
BYTES_PER_NODE = {"f64": 28 * 8, "f32": 28 * 4 + 2, "f16": 2 * (9 * 2 + 5 * 4 + 1), "f32t": 30 * 4}
# arithmetic type of the path, and the storage it streams
DTYPE = {"f64": "f64", "f32": "f32", "f16": "f32", "f32t": "f32"}
STORAGE = {"f64": "f64 populations", "f32": "f32 populations, 8-bit per-node temperature frame",
           "f16": "f16 flow (dithered rounding) and f32 thermal populations, 8-bit temperature frame",
           "f32t": "f32 populations, f32 per-node temperature frame"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=64)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--precision", default="f32", choices=["f32", "f64", "f16", "f32t"])
    ap.add_argument("--no-extras", action="store_true", help="only the timed device leg")
    ap.add_argument("--field", action="store_true",
                    help="the heterogeneous workload (log-normal porosity field) at --size, for profiling")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--long-size", type=int, default=1024,
                    help="lattice of the long_run leg (config 2's 50,000 steps against FP64)")
    ap.add_argument("--leg", default=None, choices=["batched", "adjoint", "heterogeneous", "e2e", "long_run"],
                    help="run only this extra leg and print its result (profiling)")
    return ap.parse_args()


def kernel_sources_digest(names=("lbm_device.cuh", "lbm_kernels.cu")):
    import hashlib

    hsh = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_1308_2071_gb300", "csrc", name), "rb") as f:
            hsh.update(f.read())
    return hsh.hexdigest()[:16]


ADJOINT_SOURCES = ("lbm_device.cuh", "lbm_kernels.cu", "lbm_adjoint.cuh", "lbm_adjoint.cu")


def recorded_adjoint_instructions():
    """Warp instructions per launch of the adjoint's kernels at 512^2 from the
    committed ncu summary, if the kernel sources are the ones that were
    measured; else None."""
    try:
        text = open(os.path.join(ROOT, "profiles", "k_adjoint_f32_512.md")).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.split(":", 1)[0] in ("kernel_sources_sha256", "warp_instructions_forward",
                                                      "warp_instructions_k_adjoint", "warp_instructions_k_adjoint_ring"):
            k, v = line.split(":", 1)
            vals[k] = v.strip()
    if vals.get("kernel_sources_sha256") != kernel_sources_digest(ADJOINT_SOURCES):
        return None
    try:
        return {k: int(v) for k, v in vals.items() if k.startswith("warp_")}
    except ValueError:
        return None


def recorded_traffic(precision, n, field=False):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    if the kernel sources are the ones that were measured; else None."""
    path = os.path.join(ROOT, "profiles", f"k_step_{precision}_{n}{'_field' if field else ''}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    vals = dict(line.split(":", 1) for line in text.splitlines() if line.startswith(("traffic_bytes_per_launch:",
                                                                                     "kernel_sources_sha256:")))
    if vals.get("kernel_sources_sha256", "").strip() != kernel_sources_digest():
        return None
    try:
        return int(vals["traffic_bytes_per_launch"].strip())
    except (KeyError, ValueError):
        return None


def workload(n, field=False):
    if field:
        return dict(workload=f"side-heated porous cavity {n}x{n}, log-normal permeability field (correlation "
                             f"length 32 cells, seed 1308, porosity clipped to [0.3, 0.9])", nx=n, ny=n, Ra=1e5,
                    Da=1e-4, phi=0.6, Pr=1.0, Ma=0.1,
                    boundary="NEE walls, hot left / cold right / adiabatic top-bottom",
                    inputs_vs_L2="state larger than L2 (no flush needed)" if n >= 1024 else "L2-resident")
    return dict(workload=f"side-heated porous cavity {n}x{n}", nx=n, ny=n, Ra=1e6, Da=1e-4, phi=0.4,
                Pr=1.0, Ma=0.1, boundary="NEE walls, hot left / cold right / adiabatic top-bottom",
                inputs_vs_L2="state larger than L2 (no flush needed)" if n >= 1024 else "L2-resident")


def field_bytes(precision):
    """Bytes of the per-cell porosity read per node-step (its storage type)."""
    return 8 if precision == "f64" else 4


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---- clocks -------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        self.index = index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        time.sleep(0.1)  # one more reading after the last timed step
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = [r.split(",") for r in (getattr(self, "out", "") or "").strip().splitlines() if r.count(",") >= 7]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][1]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[2]) for r in rows)}


# ---- distributed plumbing ---------------------------------------------------------

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world):
    """Largest x over the ranks (the slowest replica's time); the tensor lives
    where the process group's backend wants it (NCCL: GPU, gloo: host)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_mlups(nodes_per_rank, steps, ms_max, world):
    """Whole-job throughput of N independent replicas: every rank's node
    updates over the slowest rank's time."""
    return world * nodes_per_rank * steps / (ms_max * 1e-3) / 1e6


# ---- legs ----------------------------------------------------------------------------

TUNE_CACHE = os.path.join(ROOT, "paper_1308_2071_gb300", "_build", "tune_cache.txt")


def device_leg(n, precision, steps, warmup, world=1, gpu_index=0, sample_clocks=True, shapes=None, field=False):
    import torch

    from paper_1308_2071_gb300 import Cavity

    w = workload(n, field)
    phi = None
    if field:
        from paper_1308_2071_gb300.inputs import porosity_field

        phi = torch.from_numpy(porosity_field(n, n, phi_bar=0.6, corr_len=32.0, seed=1308)).cuda()
    cav = Cavity(n, n, Ra=w["Ra"], Da=w["Da"], phi=w["phi"], precision=precision, Pr=w["Pr"], Ma=w["Ma"],
                 phi_field=phi)
    shape = cav.tune(TUNE_CACHE)  # the library's autotuner (cached per lattice); resets to t = 0
    if shapes is not None:
        shapes[precision] = dict(block=[shape[0], shape[1]], nodes_per_thread=shape[2])
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # The clock sampler runs from before the warm-up to the end of the timed
    # region.  A short timed region (a few ms) would see no sample, so untimed
    # steps first keep the GPU under load for about a second (clocks settle,
    # the sampler takes its first readings); the state then restarts from
    # t = 0, and the warm-up and the timed steps follow as requested.
    clk = ClockSampler(gpu_index) if sample_clocks else None
    if clk:
        clk.__enter__()
    try:
        if clk:
            t_end = time.perf_counter() + 1.0
            while time.perf_counter() < t_end:
                cav.step(64)
                torch.cuda.synchronize()
            cav.reset()
        cav.step(warmup)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        e0.record(cav.stream)
        cav.step(steps)
        e1.record(cav.stream)
        torch.cuda.synchronize()
    finally:
        if clk:
            clk.__exit__()
    barrier(world)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    obs = cav.observables()
    cav.close()
    summary = clk.summary() if clk else None
    if summary:
        summary["window"] = "1 s of untimed steps, the warm-up and the timed region"
    return ms, obs, summary


def e2e_leg(n, precision, steps):
    """Public API from host memory: load a host checkpoint, run the steps
    with the Nusselt numbers of every step written into pinned host memory
    (lbm_step_nusselt: the step kernel keeps the wall columns' temperatures,
    a small kernel reduces them; the host waits once at the end), save the
    final state to host.  The same job with one lbm_step and one
    lbm_nusselt_async call per step is reported beside it.  One short
    untimed pass of each first (first use of the buffers)."""
    import torch

    from paper_1308_2071_gb300 import Cavity

    w = workload(n)
    kw = dict(Ra=w["Ra"], Da=w["Da"], phi=w["phi"], precision=precision, Pr=w["Pr"], Ma=w["Ma"])
    src = Cavity(n, n, **kw)
    blob = src.save()  # the job's initial state, in host memory
    src.close()
    pinned = torch.empty(len(blob), dtype=torch.uint8, pin_memory=True)
    pinned.numpy()[:] = memoryview(blob)
    del blob
    import ctypes as C

    from paper_1308_2071_gb300 import _lib

    lib = _lib.load()
    cav = Cavity(n, n, **kw)
    cav.tune(TUNE_CACHE)  # the launch shape the device leg uses (cached); the load below sets the state
    out = torch.empty(len(pinned), dtype=torch.uint8, pin_memory=True)
    nus = torch.empty((steps, 2), dtype=torch.float64, pin_memory=True)
    base = nus.data_ptr()

    def job(nsteps, per_call):
        t0 = time.perf_counter()
        _lib.check(lib.lbm_load(cav.handle, C.c_void_p(pinned.data_ptr()), len(pinned)), cav.handle)  # waits
        t_load = time.perf_counter()
        if per_call:
            for k in range(nsteps):
                cav.step(1)
                cav.nusselt_async(base + 16 * k)
        else:
            cav.step_nusselt(nsteps, out=nus)
        cav.stream.synchronize()  # (the save below would wait here anyway)
        t_steps = time.perf_counter()
        _lib.check(lib.lbm_save(cav.handle, C.c_void_p(out.data_ptr()), len(out)), cav.handle)  # waits
        return t0, t_load, t_steps, time.perf_counter()

    res = {}
    for per_call in (False, True):
        job(8, per_call)  # warm-up: first use of the pinned buffers and of the launch path
        torch.cuda.synchronize()
        nus.zero_()
        t0, t_load, t_steps, t1 = job(steps, per_call)
        last = cav.nusselt()
        assert (float(nus[-1, 0]), float(nus[-1, 1])) == last, "read-back disagrees with lbm_nusselt"
        res[per_call] = (n * n * steps / (t1 - t0) / 1e6, t1 - t0, t_load - t0, t1 - t_steps)
    cav.close()
    mlups, secs, load, save = res[False]
    return dict(value=round(mlups, 2), unit="MLUPS", h2d_bytes_per_step=int(len(pinned) / steps),
                d2h_bytes_per_step=int((len(out) + 16 * steps) / steps), steps=steps,
                seconds=round(secs, 4), load_seconds=round(load, 4), save_seconds=round(save, 4),
                api="lbm_step_nusselt",
                per_step_calls=dict(value=round(res[True][0], 2), seconds=round(res[True][1], 4),
                                    api="lbm_step + lbm_nusselt_async per step"))


def long_run_leg(n=1024, steps=50000):
    """Config 2's stated run length at n^2 (Ra 1e6, Da 1e-4, porosity 0.4): FP32
    and FP16-flow storage against the FP64 path after `steps` steps (the FP64
    GPU path matches the oracle to 1e-10 over 2000 steps at this size): max
    velocity error over max |u|, max temperature error over dT, relative error
    of both wall Nusselt numbers."""
    import torch

    from paper_1308_2071_gb300 import Cavity

    w = workload(n)
    res = {}
    for prec in ("f64", "f32", "f16", "f32t"):
        cav = Cavity(n, n, Ra=w["Ra"], Da=w["Da"], phi=w["phi"], precision=prec, Pr=w["Pr"], Ma=w["Ma"])
        cav.tune(TUNE_CACHE)
        cav.step(steps)
        o = cav.observables(fields=True)
        res[prec] = dict(nu=(o["nu_hot"], o["nu_cold"]), ux=o["ux"].double(), uy=o["uy"].double(),
                         T=o["T"].double())
        cav.close()
    ref = res["f64"]
    umax = max(float(ref["ux"].abs().max()), float(ref["uy"].abs().max()))
    out = dict(workload=f"{n}x{n}, Ra 1e6, Da 1e-4, phi 0.4, {steps} steps", nu_f64=list(ref["nu"]))
    for prec in ("f32", "f16", "f32t"):
        r = res[prec]
        out[prec] = dict(
            err_u_rel_max=max(float((r["ux"] - ref["ux"]).abs().max()), float((r["uy"] - ref["uy"]).abs().max())) / umax,
            err_T_max_over_dT=float((r["T"] - ref["T"]).abs().max()),
            err_nu_rel=max(abs(r["nu"][k] - ref["nu"][k]) / abs(ref["nu"][k]) for k in (0, 1)))
    del res
    torch.cuda.empty_cache()
    return out


def batched_leg(steps, warmup, ncav=256, seed=2071):
    """Batched sweep: ncav cavities of uneven size (64^2..512^2), log-uniform Ra
    and Da, uniform porosity (seeded draws), FP32, one persistent
    graph-captured launch per call, autotuned tile shape."""
    import torch

    from paper_1308_2071_gb300 import Batch
    from paper_1308_2071_gb300.inputs import cavity_sweep

    cavs = cavity_sweep(ncav, seed=seed)
    nodes = sum(c["nx"] * c["ny"] for c in cavs)
    b = Batch(cavs, precision="f32")
    tw, th, bps = b.tune(TUNE_CACHE)
    b.step(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.step(steps)
    e1.record(b.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    rc, st = b.status()
    q = b.query()
    b.close()
    peak, _ = load_peaks()
    gbs = nodes * BYTES_PER_NODE["f32"] / (ms * 1e-3 / steps) / 1e9  # 114 B per node-step
    return dict(cavities=ncav, nodes=nodes, steps=steps, mlups=round(nodes * steps / (ms * 1e-3) / 1e6, 2),
                hbm_gbs=round(gbs, 1), hbm_frac=round(gbs / peak, 4), tile=[tw, th], blocks_per_sm=bps,
                tile_kind=("interior node pairs side by side along x, border nodes in tiles of their own"
                           if th == -2 else "runs of node pairs side by side along x" if th == -1 else
                           "runs of consecutive nodes" if th == 0 else "rectangles"),
                nodes_per_thread=(2 if th < 0 else 1 if (tw if th == 0 else tw * th) in (32, 256) else 2),
                mode="one persistent cooperative launch per call, graph-captured",
                blocks=q["nblocks"], tiles=q["ntiles"], launches=1, diverged=int(st.sum()),
                status=int(rc), sizes="U{64..512} square, seed %d" % seed)


def adjoint_leg(n=512, nsteps=2000, ckpt=100):
    """Gradient of the hot-wall mean Nusselt number after nsteps with respect to
    a per-cell porosity field (phi_bar 0.6 plus a seeded perturbation), FP32,
    checkpoint every ckpt steps; adjoint MLUPS = node-steps of the forward
    sweep / wall time of the whole gradient (forward, recompute, reverse)."""
    import torch

    from paper_1308_2071_gb300 import Cavity
    from paper_1308_2071_gb300.inputs import perturbed_porosity

    phi = torch.from_numpy(perturbed_porosity(n, n, phi_bar=0.6, amplitude=0.05, corr_len=8.0, seed=2000))
    cav = Cavity(n, n, Ra=1e5, Da=1e-2, phi=0.6, precision="f32", phi_field=phi.cuda())
    cav.tune(TUNE_CACHE)  # launch shape of the forward and recomputing steps
    cav.adjoint(50, 10)  # warm-up
    torch.cuda.synchronize()
    times = []
    for _ in range(3):  # the median of three gradients
        t0 = time.perf_counter()
        J, g = cav.adjoint(nsteps, ckpt)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    dt = sorted(times)[1]
    cav.close()
    mlups = n * n * nsteps / dt / 1e6
    peak, _ = load_peaks()
    out = dict(workload=f"{n}x{n}, Ra 1e5, Da 1e-2, {nsteps} steps, checkpoint every {ckpt}, FP32",
               mlups=round(mlups, 2), seconds=round(dt, 4), seconds_each=[round(t, 4) for t in times], J=J,
               grad_l2=float(g.double().norm()))
    # The lattice (15 MB per state) and the adjoint state stay in L2, so HBM
    # is not the bound; the kernels are instruction- and latency-bound.  Bound:
    # the instruction issue rate (4 warp instructions per SM per clock at the
    # maximum SM clock) over the warp instructions one gradient executes: the
    # forward sweep and the recomputation (2 N - ceil(N / K) step launches) and
    # N reverse steps (interior and wall-ring kernels), per launch from ncu.
    ins = recorded_adjoint_instructions()
    if ins:
        nseg = -(-nsteps // ckpt)
        total = ((2 * nsteps - nseg) * ins["warp_instructions_forward"]
                 + nsteps * (ins["warp_instructions_k_adjoint"] + ins["warp_instructions_k_adjoint_ring"]))
        nsm = torch.cuda.get_device_properties(0).multi_processor_count
        try:
            mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
        except Exception:
            mhz = 2070.0
        ipeak = nsm * 4 * mhz * 1e6
        out["roofline"] = dict(bound="issue", achieved=round(total / dt / 1e9, 1), peak=round(ipeak / 1e9, 1),
                               unit="G warp instructions/s", frac=round(total / dt / ipeak, 4),
                               warp_instructions=total, source="ncu smsp__inst_executed.sum per launch, "
                                                               "profiles/k_adjoint_f32_512.md")
    else:
        out["roofline"] = dict(bound="issue", achieved=None, frac=None,
                               note="no ncu instruction counts recorded for these kernel sources")
    # HBM fraction for context: per node-step forward recompute 114 B + reverse 56 (state) + 56
    # (lambda in) + 56 (lambda out) + 4 (phi) + 8 (dJ/dphi read and write, FP64), about 294 B
    out.update(bytes_per_node_step=294, frac_of_hbm=round(mlups * 1e6 * 294 / (peak * 1e9), 4))
    return out


def heterogeneous_leg(n=8192, steps=1000, warmup=3):
    """Config 3: n^2 cavity (Ra 1e5, Da 1e-4, mean porosity 0.6) with a seeded
    porosity field whose permeability is log-normal (correlation length 32
    cells, porosity clipped to [0.3, 0.9]); FP32 and FP16-flow storage against
    the FP64 GPU path after the same steps: per-field errors and MLUPS."""
    import torch

    from paper_1308_2071_gb300 import Cavity
    from paper_1308_2071_gb300.inputs import porosity_field

    t0 = time.perf_counter()
    phi = torch.from_numpy(porosity_field(n, n, phi_bar=0.6, corr_len=32.0, seed=1308)).cuda()
    gen_s = time.perf_counter() - t0
    out = dict(workload=f"{n}x{n}, Ra 1e5, Da 1e-4, log-normal K field (corr. 32, seed 1308), {steps} steps",
               field_seconds=round(gen_s, 1))
    fields = {}
    peak, _ = load_peaks()
    for prec in ("f64", "f32", "f16"):
        cav = Cavity(n, n, Ra=1e5, Da=1e-4, phi=0.6, precision=prec, phi_field=phi)
        cav.tune(TUNE_CACHE)
        cav.set_porous_field(phi)  # tuning reset to t = 0; this keeps the field and restarts
        cav.step(warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(cav.stream)
        cav.step(steps - warmup)
        e1.record(cav.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        obs = cav.observables(fields=True)
        bpn = BYTES_PER_NODE[prec] + (16 if prec == "f64" else 8) // 2  # + the porosity read
        gbs = n * n * bpn / (ms * 1e-3 / (steps - warmup)) / 1e9
        out[prec] = dict(mlups=round(n * n * (steps - warmup) / (ms * 1e-3) / 1e6, 2), hbm_gbs=round(gbs, 1),
                         hbm_frac=round(gbs / peak, 4), nu_hot=obs["nu_hot"])
        fields[prec] = {k: obs[k].double() for k in ("ux", "uy", "T")}
        fields[prec]["nu"] = obs["nu_hot"]
        cav.close()
    ref = fields["f64"]
    umax = float(torch.maximum(ref["ux"].abs().max(), ref["uy"].abs().max()))
    for prec in ("f32", "f16"):
        f = fields[prec]
        out[prec]["err_u_rel_max"] = float(torch.maximum((f["ux"] - ref["ux"]).abs().max(),
                                                         (f["uy"] - ref["uy"]).abs().max())) / umax
        out[prec]["err_T_max_over_dT"] = float((f["T"] - ref["T"]).abs().max())
        out[prec]["err_nu_rel"] = abs(f["nu"] - ref["nu"]) / abs(ref["nu"])
    return out


def cpu_leg(n, seconds, warmup=1, max_steps=None, threads=None):
    """The FP64 oracle as it stands, on every host core (or `threads`), on a
    bounded number of steps of the same lattice; returns (MLUPS, threads,
    steps, seconds)."""
    import oracle

    threads = threads or os.cpu_count() or 1
    lat = oracle.derive(n, n, Ra=1e6, Da=1e-4, phi=0.4)
    o = oracle.Oracle(lat)
    t = time.perf_counter()
    o.step(warmup, threads=threads)
    per = max((time.perf_counter() - t) / max(warmup, 1), 1e-6)
    k = max(1, int(seconds / per))
    if max_steps:
        k = min(k, max_steps)
    t = time.perf_counter()
    o.step(k, threads=threads)
    dt = time.perf_counter() - t
    return n * n * k / dt / 1e6, threads, k, dt


# ---- main -------------------------------------------------------------------------------

def main():
    a = parse()
    world, rank, local = dist_init()
    w = workload(a.size)
    if a.impl == "reference":
        if rank != 0:
            return
        # the requested warm-up steps (bounded: an oracle step of 4096^2 takes about 0.3 s on 16 cores)
        wu = min(a.warmup, 64)
        mlups, threads, k, dt = cpu_leg(a.size, seconds=min(a.cpu_seconds * 4, 120.0), warmup=wu,
                                        max_steps=a.steps)
        line = dict(metric=METRIC, value=round(mlups, 3), unit="MLUPS", impl="reference", n_gpus=a.gpus,
                    steps=k, warmup=wu, ms_per_step=round(dt / k * 1e3, 3),
                    higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                    config=dict(w, parallelism="replicas" if a.gpus > 1 else "single GPU", replicas=a.gpus),
                    cpu_baseline=dict(value=round(mlups, 3), unit="MLUPS", kind="oracle", cores=threads,
                                      sample=f"{k} of the requested {a.steps} steps of the {a.size}^2 lattice "
                                             f"after {wu} warm-up steps, FP64 oracle"),
                    e2e=dict(value=round(mlups, 3), unit="MLUPS", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
        print(json.dumps(line), flush=True)
        return

    import torch

    torch.cuda.set_device(local)
    from paper_1308_2071_gb300 import _lib

    _lib.load()
    if a.leg:
        legs = dict(batched=lambda: batched_leg(min(a.steps, 1000), min(a.warmup, 8)),
                    adjoint=adjoint_leg, heterogeneous=heterogeneous_leg,
                    long_run=lambda: long_run_leg(a.long_size),
                    e2e=lambda: e2e_leg(a.size, a.precision, min(a.steps, 1000)))
        print(json.dumps({"leg": a.leg, a.leg: legs[a.leg]()}), flush=True)
        return
    shapes = {}
    ms, obs, clocks = device_leg(a.size, a.precision, a.steps, a.warmup, world, gpu_index=local, shapes=shapes,
                                 field=a.field)
    ms = max_over_ranks(ms, world)
    nodes = a.size * a.size
    mlups = replica_mlups(nodes, a.steps, ms, world)
    peak, peak_kind = load_peaks()
    per_launch_s = ms * 1e-3 / a.steps
    bpn = BYTES_PER_NODE[a.precision] + (field_bytes(a.precision) if a.field else 0)
    achieved = nodes * bpn / per_launch_s / 1e9
    roof = dict(bound="hbm", achieved=round(achieved, 1), peak=peak, unit="GB/s",
                frac=round(achieved / peak, 4),
                traffic=recorded_traffic(a.precision, a.size, a.field), kernel="k_step",
                algorithmic_bytes_per_launch=nodes * bpn, peak_source=peak_kind)
    line = dict(metric=METRIC, value=round(mlups, 2), unit="MLUPS", n_gpus=world, steps=a.steps,
                warmup=a.warmup, ms_per_step=round(ms / a.steps, 5), higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype=DTYPE[a.precision], storage=STORAGE[a.precision],
                data="synthetic (seeded, no dataset)",
                config=dict(workload(a.size, a.field), parallelism="replicas" if world > 1 else "single GPU",
                            replicas=world),
                roofline=roof, clocks=clocks, gpu_launches=a.steps, launch_shape=shapes.get(a.precision),
                nu_hot_at_end=obs["nu_hot"], status=obs["status"])
    if world > 1 and not a.no_extras and not a.field:
        # every replica runs the end-to-end leg; the job's figure takes the slowest
        e = e2e_leg(a.size, a.precision, min(a.steps, 1000))
        secs = max_over_ranks(e["seconds"], world)
        e.update(value=round(replica_mlups(nodes, e["steps"], secs * 1e3, world), 2), seconds=round(secs, 3),
                 replicas=world)
        line["e2e"] = e
    if world == 1 and not a.no_extras and not a.field:  # the extra legs belong to the default workload
        variants = {}
        # FP64 and FP16 storage on the same lattice, and Nu against FP64 at equal steps
        k = min(a.steps, 1000)
        nsteps_cmp = a.warmup + k
        for prec in ("f64", "f16", "f32t"):
            ms_p, obs_p, _ = device_leg(a.size, prec, k, a.warmup, 1, gpu_index=local,
                                        sample_clocks=False, shapes=shapes)
            ach = nodes * BYTES_PER_NODE[prec] / (ms_p * 1e-3 / k) / 1e9
            variants[prec] = dict(mlups=round(nodes * k / (ms_p * 1e-3) / 1e6, 2),
                                  hbm_gbs=round(ach, 1), hbm_frac=round(ach / peak, 4), steps=k,
                                  nu_hot=obs_p["nu_hot"], nu_cold=obs_p["nu_cold"], at_step=nsteps_cmp,
                                  launch_shape=shapes.get(prec))
        _, obs32, _ = device_leg(a.size, "f32", k, a.warmup, 1, gpu_index=local, sample_clocks=False)
        nu64 = variants["f64"]["nu_hot"]
        variants["f32"] = dict(nu_hot=obs32["nu_hot"], at_step=nsteps_cmp)
        variants["nu_rel_err_f32_vs_f64"] = abs(obs32["nu_hot"] - nu64) / abs(nu64)
        variants["nu_rel_err_f16_vs_f64"] = abs(variants["f16"]["nu_hot"] - nu64) / abs(nu64)
        variants["nu_rel_err_f32t_vs_f64"] = abs(variants["f32t"]["nu_hot"] - nu64) / abs(nu64)
        line["variants"] = variants
        line["e2e"] = e2e_leg(a.size, a.precision, min(a.steps, 1000))
        line["batched"] = batched_leg(min(a.steps, 1000), 8)
        line["adjoint"] = adjoint_leg()
        line["heterogeneous"] = heterogeneous_leg()
        line["long_run_precision"] = lr = long_run_leg()
        # the headline variant's error against FP64 after the stated run length
        if a.precision in lr:
            line["u_rel_err"] = lr[a.precision]["err_u_rel_max"]
            line["T_err"] = lr[a.precision]["err_T_max_over_dT"]
            line["nu_rel_err"] = lr[a.precision]["err_nu_rel"]
            line["err_reference"] = ("FP64 GPU path (matches the FP64 oracle to 1e-10 over 2000 steps) after "
                                     "50,000 steps of the same physics at 1024^2; bounds 1e-4 (u), 1e-5 (T), "
                                     "1e-4 (Nu)")
        mlc, threads, k, dt = cpu_leg(a.size, a.cpu_seconds)
        ml1, _, k1, dt1 = cpu_leg(a.size, 1.0, threads=1)
        line["cpu_baseline"] = dict(value=round(mlc, 3), unit="MLUPS", cores=threads, kind="oracle",
                                    sample=f"{k} steps of the {a.size}^2 lattice, FP64 oracle, {dt:.1f} s",
                                    single_thread=dict(value=round(ml1, 3), steps=k1, seconds=round(dt1, 1)))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        barrier(world)
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
