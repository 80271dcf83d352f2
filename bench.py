"""Throughput of the SBFEM full-waveform-inversion hot path on GB300.

One step = the whole path for one batch: set-up of the model (density map,
E-matrices, condensation, global factorisation), forward solve of every shot,
misfit, time-reversed adjoint and Frechet-kernel gradient, on the size workload
(64x64 square S-elements, p = 4, N_r = 32, 8 Ricker shots, 32 receivers, 2000
Newmark steps, 256x256 density grid).  The metric counts element-radial-node-steps
of one shot taken through forward + adjoint + gradient:
units/step = elements * N_r * time steps * shots.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Multi-GPU runs (torchrun) shard shots: the job has
8 shots per rank, every rank runs its own 8 on its own GPU, and the ranks exchange
only the misfit and gradient sum (one all-reduce per step; weak scaling).
"""

import argparse
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "S-element radial-node-steps/s fwd+adj+grad at 1e-10 rel err; p50/p99 latency"
UNIT = "element-radial-node-steps/s"
FP64_PEAK_TFLOPS = 1.25      # GB300 FP64 (vector and tensor), nominal; our DFMA probe measured 1.20 at 2.0 GHz


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


def algorithmic_bytes_per_unit_launch(nb, B):
    """HBM bytes one element-radial-node-step of one shot needs in one pass (forward or
    adjoint): the four n_b x n_b FP64 operators of the radial point shared by the B shots of
    the pass, read+write of u, u-dot, u-ddot, one spill of the condensed load, and the
    forward velocity written to (forward) or read from (adjoint) the store."""
    return 4 * nb * nb * 8 / B + 6 * nb * 8 + 2 * nb * 8 + nb * 8


def profiled_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if the kernel's
    source has not changed since the counters were taken; else None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{kernel}_size_workload.md")
    try:
        text = open(path).read()
    except OSError:
        return None, "no ncu summary"
    m_b = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    hashes = re.findall(r"source_sha256:\s*(\S+)\s+(\S+)", text)    # every file the kernel is built from
    if not m_b or not hashes:
        return None, "ncu summary without traffic"
    for rel, want in hashes:
        try:
            digest = hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest()
        except OSError:
            return None, "kernel source missing"
        if digest != want:
            return None, "kernel changed since the ncu capture"
    return float(m_b.group(1)), os.path.relpath(path, ROOT)


# ---------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
CPU_SAMPLE_NX = 8
CPU_SAMPLE_K = 200

_CPU_CODE = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from sbfwi_inputs import size_workload
from oracle import fwi
w = size_workload(nx={nx}, K={K}, n_shots={ns})
lo, hi = {lo}, {hi}
w.src_nodes, w.wavelets = w.src_nodes[lo:hi], w.wavelets[lo:hi]
wall0 = time.time()
t0 = time.perf_counter()
om = fwi.build_model(w.mesh, w.n_r, w.c, w.rho_start, w.dt)
tr, store, _ = fwi.forward(om, w.src_nodes, w.wavelets, w.rec_nodes)
E, res = fwi.misfit(tr, np.zeros_like(tr), w.dt)
g = fwi.gradient_to_grid(om, fwi.adjoint_gradient(om, store, res, w.rec_nodes), w.gx, w.gy)
t1 = time.perf_counter()
units = w.mesh.n_elem * w.n_r * w.K * w.n_shots
if {save!r}:
    np.savez({save!r}, traces=tr, grad=g, misfit=E)
print(json.dumps({{"seconds": t1 - t0, "units": units, "wall0": wall0, "wall1": time.time()}}))
"""


def run_oracle_sample(nx=CPU_SAMPLE_NX, K=CPU_SAMPLE_K, save=""):
    """The oracle as it stands, single-threaded, in a fresh process (never forked from CUDA).
    With `save`, the sample's traces, gradient and misfit are written there (npz) for the
    accuracy check of the GPU path on the same inputs."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = _CPU_CODE.format(root=ROOT, nx=nx, K=K, ns=8, lo=0, hi=8, save=save)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    if out.returncode != 0:
        raise RuntimeError("oracle sample failed: " + out.stderr[-2000:])
    r = json.loads(out.stdout.strip().splitlines()[-1])
    sample = (f"oracle set-up + {K} Newmark steps forward, misfit, adjoint and gradient of 8 shots on a "
              f"{nx}x{nx} sub-mesh of the same recipe (p=4, N_r=32), float64 time loop, extended-precision set-up")
    return r["units"] / r["seconds"], r["seconds"], sample


def host_cpu():
    """Core count and CPU model of this host (lscpu's model name, else the platform's)."""
    import platform
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count() or 1, "cpu_model": model or platform.processor() or platform.machine()}


def run_oracle_sample_all_cores(nx=CPU_SAMPLE_NX, K=CPU_SAMPLE_K):
    """The same recipe on every host core: one fresh single-threaded oracle process per core,
    each running one shot (its own set-up) of a version of the sample with one top-edge
    source per core; the rate is all processes' units over the wall time from the first
    set-up to the last end."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    procs_n = max(1, min(4 * nx, os.cpu_count() or 1))      # distinct top-edge nodes of the sub-mesh
    procs = [subprocess.Popen([sys.executable, "-c", _CPU_CODE.format(root=ROOT, nx=nx, K=K, ns=procs_n, lo=k,
                                                                      hi=k + 1, save="")],
                              env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for k in range(procs_n)]
    units, starts, ends = 0, [], []
    for p in procs:
        out, err = p.communicate(timeout=900)
        if p.returncode != 0:
            raise RuntimeError("oracle sample failed: " + err[-2000:])
        r = json.loads(out.strip().splitlines()[-1])
        units += r["units"]
        starts.append(r["wall0"])
        ends.append(r["wall1"])
    wall = max(ends) - min(starts)        # from the first process's set-up to the last one's end
    sample = (f"{procs_n} concurrent single-threaded oracle processes, one shot each (set-up repeated in each), "
              f"of the single-core sample's recipe with {procs_n} top-edge sources")
    return units / wall, wall, procs_n, sample


TRACE_TOL, GRAD_TOL = 1e-10, 1e-8


def accuracy_check(lib, dev, oracle_npz, nx=CPU_SAMPLE_NX, K=CPU_SAMPLE_K):
    """The GPU path on the oracle sample's inputs (the same sub-mesh, shots, steps and
    starting model; one pass of 8 shots with the default kernels, as in the timed step):
    relative L2 error of traces, misfit and gradient against the oracle's."""
    import torch
    from sbfwi_inputs import size_workload
    ref = np.load(oracle_npz)
    w = size_workload(nx=nx, K=K, n_shots=8)
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    md = lib.Model(M, w.c, torch.tensor(w.rho_start, device=dev), w.dt)
    tr, st = lib.forward(md, w.src_nodes, torch.tensor(w.wavelets, device=dev), w.rec_nodes)
    E, res = lib.misfit(tr, torch.zeros_like(tr), w.dt)
    g = lib.adjoint_gradient(md, st, res)
    torch.cuda.synchronize()
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    e_tr = rel(tr.cpu().numpy(), ref["traces"])
    e_g = rel(g.cpu().numpy(), ref["grad"])
    e_E = abs(E - float(ref["misfit"])) / abs(float(ref["misfit"]))
    return {"traces_rel_l2": e_tr, "grad_rel_l2": e_g, "misfit_rel": e_E,
            "tol": {"traces": TRACE_TOL, "grad": GRAD_TOL}, "within_tol": bool(e_tr <= TRACE_TOL and e_g <= GRAD_TOL),
            "steps": K, "sample": f"GPU path vs the oracle on the cpu_baseline sample: {nx}x{nx} sub-mesh of the "
                                  f"same recipe (p=4, N_r=32), 8 shots in one pass, {K} Newmark steps, set-up + "
                                  "forward + misfit + adjoint + gradient"}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, path):
        self.path, self.proc = path, None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self, device_index=0):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9 or parts[0] != str(device_index):
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world):
    import torch
    from paper_2501_06748_gb300 import build
    build.build()
    from paper_2501_06748_gb300 import sbfwi as lib
    from paper_2501_06748_gb300.shots import shard, allreduce_misfit_gradient
    from sbfwi_inputs import size_workload, diff_workload

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    # weak scaling: the job has shots x ranks sources; each rank takes its shard
    diff = args.config == "diff"
    K_steps = args.time_steps or (8000 if diff else 2000)
    if diff:
        w = diff_workload(K=K_steps, n_shots=(args.shots or 16) * world)
    else:
        w = size_workload(K=K_steps, n_shots=(args.shots or 8) * world)
    ckpt = lib.CKPT_AUTO if diff else 0
    mine = shard(w.n_shots, rank, world)
    src_nodes = w.src_nodes[mine.start:mine.stop]
    wav_host = np.ascontiguousarray(w.wavelets[mine.start:mine.stop])
    B, K, R = len(mine), w.K, int(w.rec_nodes.shape[0])
    E, N_r = w.mesh.n_elem, w.n_r
    units_per_step = E * N_r * K * B
    M = lib.Mesh.from_inputs(w.mesh, N_r)
    nb, n = M.n_b, N_r - 1

    rho_start = torch.tensor(w.rho_start, device=dev)
    rho_true = torch.tensor(w.rho_true, device=dev)
    wav = torch.tensor(wav_host, device=dev)
    # observed data: the same path on the flawed model (synthetic input, made once, untimed)
    m_true = lib.Model(M, w.c, rho_true, w.dt)
    observed, _ = lib.forward(m_true, src_nodes, wav, w.rec_nodes, keep=False)
    del m_true
    torch.cuda.synchronize()

    observed_host = observed.cpu().numpy()
    chunk = args.shots_per_pass or min(B, 8)
    chunks = [slice(s, min(B, s + chunk)) for s in range(0, B, chunk)]

    def step(host=False):
        """Set-up + forward + misfit + adjoint gradient of all shots; returns (E, grad)."""
        if host:
            rho_in, wav_in, obs_in = w.rho_start, wav_host, observed_host
            grad = np.zeros((w.gy, w.gx))
        else:
            rho_in, wav_in, obs_in = rho_start, wav, observed
            grad = torch.zeros((w.gy, w.gx), dtype=torch.float64, device=dev)
        model = lib.Model(M, w.c, rho_in, w.dt)
        E_tot = 0.0
        for c in chunks:
            tr, st = lib.forward(model, src_nodes[c], wav_in[c], w.rec_nodes, ckpt_every=ckpt)
            Ec, res = lib.misfit(tr, obs_in[c], w.dt)
            lib.adjoint_gradient(model, st, res, grad_out=grad, accumulate=True)
            E_tot += Ec
            del st
        if dist:
            # the one exchange of the path: sum of misfit and gradient over the ranks' shots
            if host:
                g_dev = torch.from_numpy(grad).to(dev)
                E_tot, g_dev = allreduce_misfit_gradient(E_tot, g_dev)
                grad = g_dev.cpu().numpy()
            else:
                E_tot, grad = allreduce_misfit_gradient(E_tot, grad)
        return E_tot, grad

    # the forward velocity store of one pass must fit in HBM; halve the pass if it does not
    while True:
        try:
            step()
            break
        except lib.SbfwiError as err:
            if err.code != lib.ENOMEM or chunk == 1:
                raise
            chunk = (chunk + 1) // 2
            chunks = [slice(s, min(B, s + chunk)) for s in range(0, B, chunk)]
    for _ in range(args.warmup - 1):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(os.path.join(args.clock_log, f"clocks_rank{rank}.csv"))
    lib.profile_read(reset=True)
    lib.profile_enable(True)
    stream = torch.cuda.current_stream(dev)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    evs[0].record(stream)
    for k in range(args.steps):
        step()
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop(dev.index or 0)
    if dist:
        dist.barrier()
    lib.profile_enable(False)
    prof = lib.profile_read(reset=True)
    per_step = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    if dist:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = units_per_step * world * args.steps / (total_ms / 1e3)

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if args.e2e_steps > 0:
        step(host=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            step(host=True)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        ntr = B * R * K * 8
        gbytes = w.gy * w.gx * 8 * len(chunks)
        # H2D: density, wavelets, misfit inputs (traces, observed), residual, gradient (accumulated)
        h2d = w.rho_start.nbytes + wav_host.nbytes + 2 * ntr + ntr + gbytes
        # D2H: traces, residual, misfit values, gradient
        d2h = ntr + ntr + 8 * len(chunks) + gbytes
        if dist:
            h2d += w.gy * w.gx * 8            # the gradient goes through the device for the all-reduce
            d2h += w.gy * w.gx * 8
            t = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": units_per_step * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    # the same path one shot at a time (B = 1 per pass), for comparison with the batched pass
    one_shot = None
    if args.one_shot and not diff:
        def step_one():
            model = lib.Model(M, w.c, rho_start, w.dt)
            tr, st = lib.forward(model, src_nodes[:1], wav[:1], w.rec_nodes)
            _, res = lib.misfit(tr, observed[:1], w.dt)
            return lib.adjoint_gradient(model, st, res)
        step_one()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step_one()
        e1.record(stream)
        torch.cuda.synchronize()
        ms1 = e0.elapsed_time(e1)
        one_shot = {"value": E * N_r * K / (ms1 / 1e3), "unit": UNIT, "ms_per_shot": ms1,
                    "note": "set-up + forward + misfit + adjoint + gradient of shot 0 alone (one pass, B = 1)"}

    # roofline of the dominant kernel (the element step), from its own CUDA events
    el = prof["element"]
    avg_launch_ms = el["ms"] / max(el["intervals"], 1)
    Bc = chunks[0].stop - chunks[0].start
    use_tc = os.environ.get("SBFWI_ELEMENT", "") != "fp64" and nb <= 16 and Bc <= 8
    kernel = "element_step_tc_kernel" if use_tc else "element_step_kernel"
    units_launch = E * N_r * Bc                      # one pass (forward or adjoint) of one time step
    bpu = algorithmic_bytes_per_unit_launch(nb, Bc)
    bytes_launch = bpu * units_launch
    pk, pk_kind = peaks()
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    achieved_gbs = bytes_launch / (avg_launch_ms / 1e3) / 1e9
    flops_launch = 8.0 * nb * nb * units_launch      # four n_b x n_b mat-vecs per radial point and shot
    traffic, traffic_src = profiled_traffic(kernel)
    roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved_gbs / hbm_peak, "traffic": traffic,
                "kernel": kernel, "algorithmic_bytes_per_launch": bytes_launch,
                "bytes_per_unit": bpu, "units_per_launch": units_launch,
                "avg_launch_ms": avg_launch_ms, "launches_timed": el["intervals"],
                "peak_note": f"HBM copy bandwidth, {pk_kind} (burst)", "traffic_source": traffic_src,
                "fp64_view": {"fp64_equiv_tflops": flops_launch / (avg_launch_ms / 1e3) / 1e12,
                              "fp64_nominal_tflops": FP64_PEAK_TFLOPS,
                              "note": "mat-vec flops at FP64 accuracy; the tensor-core kernel computes them "
                                      "as exact FP16 digit products, so this may exceed the FP64 pipe"}}
    launches = sum(v["launches"] for v in prof.values())

    if rank != 0:
        return None
    cpu = cpu_all = accuracy = None
    if not args.no_cpu_baseline:
        hc = host_cpu()
        save = os.path.join(tempfile.mkdtemp(prefix="sbfwi_acc_"), "oracle_sample.npz")
        rate, secs, sample = run_oracle_sample(save=save)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample, "seconds": secs,
               "host_nproc": hc["nproc"], "cpu_model": hc["cpu_model"]}
        rate_all, wall_all, cores_all, sample_all = run_oracle_sample_all_cores()
        cpu_all = {"value": rate_all, "unit": UNIT, "cores": cores_all, "kind": "oracle", "sample": sample_all,
                   "seconds": wall_all, "host_nproc": hc["nproc"], "cpu_model": hc["cpu_model"]}
        if not diff:
            accuracy = accuracy_check(lib, dev, save)
    lat = np.array(per_step)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{w.name}: {w.mesh.nx}x{w.mesh.ny} square S-elements, p=4 (n_b={nb}), N_r={N_r}, "
                               f"{B} Ricker shots, {R} receivers, {K} Newmark steps, {w.gx}x{w.gy} density grid; "
                               "per step: set-up + forward + misfit + adjoint + gradient"
                               + ("; checkpoints at the memory-optimal interval, forward recomputed in the adjoint"
                                  if diff else ""),
                   "elements": E, "n_b": nb, "N_r": N_r, "shots": B, "shots_per_pass": Bc, "time_steps": K,
                   "global_nodes": M.n_nodes, "units_per_step": units_per_step,
                   "flaw_factor": w.info["flaws"]["factor"],
                   "l2": ("inputs larger than L2 (forward velocity store %.0f GB per pass)" % (K * M.n_nodal * Bc * 8 / 1e9)
                          if not diff else "inputs larger than L2 (checkpoints + recompute window > 100 GB per pass)"),
                   "parallelism": f"shots per GPU, {world} GPU(s)"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "per_step": [float(x) for x in per_step]},
        "phases_ms_per_step": {k: v["ms"] / args.steps for k, v in prof.items()},
        "accuracy": accuracy,
        "roofline": roofline, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "e2e": e2e, "one_shot_path": one_shot, "gpu_launches": int(launches),
        "clocks": clk,
    }
    if dist:
        dist.destroy_process_group()
    return out


def run_serving(args, rank, world):
    """Shot requests with Poisson arrivals through the serving engine: continuous batching
    of requests as the slots of library sessions (admitted between windows of 32 steps
    while other slots run), a third of them gradient requests (forward, misfit, adjoint and
    gradient), the rest trace requests."""
    import torch
    from paper_2501_06748_gb300 import build
    build.build()
    from paper_2501_06748_gb300 import sbfwi as lib, serving
    from sbfwi_inputs import structured_mesh, boundary_nodes, flawed_density_ellipses, ricker
    if rank != 0:
        return None
    torch.cuda.set_device(0)
    specs = [(16, 2, 8), (32, 3, 16), (32, 4, 16), (64, 4, 32)]      # (elements per side, p, N_r)
    meshes, recs, dts = {}, {}, {}
    for nx, p, n_r in specs:
        m = structured_mesh(nx, nx, p)
        meshes[(nx, p, n_r)] = (m, lib.Mesh.from_inputs(m, n_r))
        bnd = np.unique(np.concatenate([boundary_nodes(m, s) for s in ("bottom", "left", "right")]))
        recs[(nx, p, n_r)] = bnd[np.linspace(0, len(bnd) - 1, 16).astype(int)]
        dts[(nx, p, n_r)] = 0.5 / (nx * p)

    def build_model(key):
        nx, p, n_r, seed = key
        rho, _ = flawed_density_ellipses(128, 128, n=2, factor=0.5, seed=seed)
        return lib.Model(meshes[(nx, p, n_r)][1], 1.0, rho, dts[(nx, p, n_r)])

    rng = np.random.default_rng(7)
    n_req = args.requests
    keys = [spec + (int(seed),) for spec in specs for seed in (0, 1)]
    reqs, units = [], 0
    for rid in range(n_req):
        key = keys[int(rng.integers(len(keys)))]
        spec = key[:3]
        m = meshes[spec][0]
        K = int(rng.choice([500, 1000]))
        h = 1.0 / (spec[0] * spec[1])
        top = boundary_nodes(m, "top")
        wav = ricker(1.0 / (10 * h), dts[spec], K)
        obs = np.zeros((recs[spec].size, K)) if rid % 3 == 0 else None
        reqs.append(serving.Request(rid, key, int(rng.choice(top)), wav, recs[spec], arrival=0.0, observed=obs))
        units += m.n_elem * spec[2] * K
    for key in keys:
        build_model(key)                          # warm-up of every mesh's device set-up
    # arrival rate: 70 % of the rate one request at a time could sustain (single-shot service
    # times per model: forward, and forward + misfit + adjoint for gradient requests)
    t_fwd, t_grad = {}, {}
    for key in keys:
        md = build_model(key)
        spec = key[:3]
        top = boundary_nodes(meshes[spec][0], "top")
        wav = ricker(1.0 / (10 / (key[0] * key[1])), dts[spec], 200)[None]
        lib.forward(md, [int(top[len(top) // 2])], wav, recs[spec], keep=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lib.forward(md, [int(top[len(top) // 2])], wav, recs[spec], keep=False)
        torch.cuda.synchronize()
        t_fwd[key] = (time.perf_counter() - t0) / 200.0
        t0 = time.perf_counter()
        tr, st = lib.forward(md, [int(top[len(top) // 2])], wav, recs[spec])
        _, res = lib.misfit(tr, np.zeros_like(tr), md.dt)
        lib.adjoint_gradient(md, st, res)
        torch.cuda.synchronize()
        t_grad[key] = (time.perf_counter() - t0) / 200.0
    mean_service = float(np.mean([(t_grad if r.wants_gradient else t_fwd)[r.model_key] * r.K for r in reqs]))
    rate = 0.7 / mean_service
    t = 0.0
    for r in reqs:
        t += float(rng.exponential(1.0 / rate))
        r.arrival = t
    eng = serving.Engine(build_model, max_batch=8, window=32, cache_capacity=len(keys))
    for key in keys:                             # models set up before the clock starts
        eng.cache.get(key)
    clocks = ClockSampler(os.path.join(args.clock_log, "clocks_serving.csv"))
    clocks.start()
    t0 = time.perf_counter()
    eng.run(reqs)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop(0)
    st = serving.latency_stats(reqs)
    st_g = serving.latency_stats([r for r in reqs if r.wants_gradient])
    joined = sum(1 for r in reqs if r.admitted_at and r.admitted_at[1] > 0)
    return {"metric": "serving: element-radial-node-steps/s of served requests; p50/p99 request latency",
            "value": units / wall, "unit": "element-radial-node-steps/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": wall * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "serving: %d requests (one Ricker shot each, 16 receivers; every third also "
                                   "misfit + adjoint + gradient) on 8 seeded flawed models over meshes %s (elements "
                                   "per side, p, N_r), K in {500, 1000}, Poisson arrivals at 70%% of the "
                                   "one-request-at-a-time capacity; continuous batching: requests are the slots "
                                   "(shot columns, 8 per session) of library sessions, admitted between windows of "
                                   "32 steps while the other slots run" % (n_req, specs),
                       "requests": n_req, "gradient_requests": int(sum(r.wants_gradient for r in reqs)),
                       "arrival_rate_per_s": rate, "windows": eng.windows,
                       "mean_slots_busy": float(np.mean(eng.batches)) if eng.batches else 0.0,
                       "admitted_while_others_in_flight": joined, "max_in_flight": eng.max_in_flight,
                       "units": "one element-radial-node-step of a request's path (forward for trace requests, "
                                "forward + adjoint + gradient for gradient requests)",
                       "l2": "models, session state and forward fields stay on the device"},
            "latency_ms": {"p50": st["p50_s"] * 1e3, "p99": st["p99_s"] * 1e3, "mean": st["mean_s"] * 1e3,
                           "gradient_p50": st_g["p50_s"] * 1e3, "gradient_p99": st_g["p99_s"] * 1e3},
            "clocks": clk}


# the paper's Tables 1-2: seconds per L-BFGS epoch (forward + adjoint + gradient of 2 sources, 200
# steps) on 12 CPU threads, Voronoi meshes; hole specimen, 5 and 7 radial intervals
PAPER_EPOCH_S = {(1000, 5): 0.95, (2000, 5): 2.39, (4000, 5): 5.49, (8000, 5): 11.19,
                 (1000, 7): 1.32, (2000, 7): 3.21, (4000, 7): 6.82, (8000, 7): 13.92}
# the same table's low-frequency-expansion column (the paper's comparison method)
PAPER_LFE_EPOCH_S = {1000: 0.23, 2000: 0.46, 4000: 1.27, 8000: 2.70}


def run_paper(args, rank, world):
    """The paper's plate recipe on its centroidal Voronoi meshes (or squares): one evaluation
    (set-up + forward, misfit, adjoint and gradient of both sources) per element count and interval count,
    with the paper's seconds per epoch beside it (context: its meshes are Voronoi
    polygons and it ran on a laptop CPU)."""
    import torch
    from paper_2501_06748_gb300 import build
    build.build()
    from paper_2501_06748_gb300 import sbfwi as lib
    from sbfwi_inputs import paper_workload
    if rank != 0:
        return None
    torch.cuda.set_device(0)
    rows = []
    units_all, secs_all = 0, 0.0
    meshes = {}
    for (n_elem, intervals) in sorted(PAPER_EPOCH_S):
        w = paper_workload(n_elem=n_elem, intervals=intervals, mesh_kind=args.paper_mesh, mesh=meshes.get(n_elem))
        meshes[n_elem] = w.mesh
        L = w.mesh.lx
        M = lib.Mesh.from_inputs(w.mesh, w.n_r)
        mt = lib.Model(M, w.c, w.rho_true, w.dt, lx=L, ly=L)
        obs, _ = lib.forward(mt, w.src_nodes, w.wavelets, w.rec_nodes, keep=False)
        del mt

        def epoch():
            md = lib.Model(M, w.c, w.rho_start, w.dt, lx=L, ly=L)
            tr, st = lib.forward(md, w.src_nodes, w.wavelets, w.rec_nodes)
            E, res = lib.misfit(tr, obs, w.dt)
            return E, lib.adjoint_gradient(md, st, res)

        for _ in range(max(1, args.warmup)):
            epoch()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            epoch()
        torch.cuda.synchronize()
        sec = (time.perf_counter() - t0) / args.steps
        units = w.mesh.n_elem * w.n_r * w.K * w.n_shots
        units_all += units
        secs_all += sec
        nb = getattr(w.mesh, "n_b", None)
        rows.append({"method": "radial FD", "elements": w.mesh.n_elem, "intervals": intervals, "N_r": w.n_r,
                     "receivers": int(len(w.rec_nodes)),
                     "n_b": [int(nb.min()), int(nb.max())] if nb is not None else 4 * w.mesh.p,
                     "s_per_epoch": sec, "units_per_s": units / sec,
                     "paper_s_per_epoch": PAPER_EPOCH_S[(n_elem, intervals)],
                     "paper_over_ours": PAPER_EPOCH_S[(n_elem, intervals)] / sec})
        if intervals == 5:
            # the comparison method on the same mesh and data (its set-up: the Riccati and
            # Lyapunov solves of every element on the device)
            def epoch_lfe():
                md = lib.Model(M, w.c, w.rho_start, w.dt, lx=L, ly=L, lfe=True)
                tr, st = lib.forward(md, w.src_nodes, w.wavelets, w.rec_nodes)
                E, res = lib.misfit(tr, obs, w.dt)
                return E, lib.adjoint_gradient(md, st, res)

            for _ in range(max(1, args.warmup)):
                epoch_lfe()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                epoch_lfe()
            torch.cuda.synchronize()
            sec_l = (time.perf_counter() - t0) / args.steps
            lib.profile_read(reset=True)
            lib.profile_enable(True)
            lib.Model(M, w.c, w.rho_start, w.dt, lx=L, ly=L, lfe=True)
            torch.cuda.synchronize()
            lib.profile_enable(False)
            setup_ms = lib.profile_read(reset=True)["setup"]["ms"]
            lib.profile_enable(True)
            lib.Model(M, w.c, w.rho_start, w.dt, lx=L, ly=L)
            torch.cuda.synchronize()
            lib.profile_enable(False)
            setup_fd_ms = lib.profile_read(reset=True)["setup"]["ms"]
            rows.append({"method": "low-frequency expansion", "elements": w.mesh.n_elem,
                         "s_per_epoch": sec_l, "setup_ms": setup_ms, "fd_setup_ms": setup_fd_ms,
                         "paper_s_per_epoch": PAPER_LFE_EPOCH_S[n_elem],
                         "paper_over_ours": PAPER_LFE_EPOCH_S[n_elem] / sec_l})
    return {"metric": "paper-shaped plate: seconds per epoch (set-up + fwd + adj + grad, 2 sources, 200 steps); "
                      "radial FD rows and the comparison method's",
            "value": units_all / secs_all, "unit": "element-radial-node-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs_all / len(rows), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "paper: 100 mm plate, c = 6000 m/s, rho = 2700 with one circular flaw, 2 sine-burst "
                                   "sources (2 cycles, 500 kHz) 30 mm apart, receivers every 1 mm on 4 edges, 200 steps "
                                   "of 0.2 us; " + ("centroidal Voronoi polygons (the paper's mesh type), line order 2"
                                                    if args.paper_mesh == "voronoi" else
                                                    "square S-elements of order 2 instead of the paper's Voronoi polygons"),
                       "rows": rows, "l2": "small workloads: latency-bound, inputs fit L2"}}


def run_solid(args, rank, world):
    """3-D hexahedral S-elements (the paper's Section 3 preamble: 3-D needs only minor
    changes): per step, set-up + forward + misfit + adjoint + gradient of all shots on the
    3-D recipe, observed data from the flawed model."""
    import torch
    from paper_2501_06748_gb300 import build
    build.build()
    from paper_2501_06748_gb300 import sbfwi as lib
    from sbfwi_inputs import solid_workload
    if rank != 0:
        return None
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    w = solid_workload(K=args.time_steps or 500, p=args.solid_p)
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    wav = torch.tensor(w.wavelets, device=dev)
    mt = lib.Model(M, w.c, torch.tensor(w.rho_true, device=dev), w.dt)
    obs, _ = lib.forward(mt, w.src_nodes, wav, w.rec_nodes, keep=False)
    del mt
    rho0 = torch.tensor(w.rho_start, device=dev)

    def step():
        md = lib.Model(M, w.c, rho0, w.dt)
        tr, st = lib.forward(md, w.src_nodes, wav, w.rec_nodes)
        E, res = lib.misfit(tr, obs, w.dt)
        return E, lib.adjoint_gradient(md, st, res)

    for _ in range(max(3, args.warmup)):
        E, g = step()
    clocks = ClockSampler(os.path.join(args.clock_log, "clocks_solid.csv"))
    clocks.start()
    lib.profile_read(reset=True)
    lib.profile_enable(True)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        E, g = step()
    t1.record()
    torch.cuda.synchronize()
    lib.profile_enable(False)
    prof = lib.profile_read(reset=True)
    clk = clocks.stop(0)
    ms = t0.elapsed_time(t1) / args.steps
    units = w.mesh.n_elem * w.n_r * w.K * w.n_shots
    phases = {k: v["ms"] / args.steps for k, v in prof.items()}
    return {"metric": "3-D S-elements: element-radial-node-steps/s fwd+adj+grad", "value": units / (ms / 1e3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"solid: unit cube in {w.mesh.nx}^3 hexahedral S-elements, faces of order "
                                   f"{w.mesh.p} (n_b = {M.n_b}), N_r = {w.n_r}, {w.n_shots} Ricker shots on the top face, "
                                   f"{len(w.rec_nodes)} receivers, {w.K} Newmark steps, {w.gx}^3 density grid with one "
                                   "spherical flaw; per step: set-up + forward + misfit + adjoint + gradient",
                       "elements": w.mesh.n_elem, "global_nodes": w.mesh.n_nodes, "n_b": M.n_b, "N_r": w.n_r,
                       "shots": w.n_shots, "time_steps": w.K, "tree_levels": M.tree_levels,
                       "factor_entries": M.factor_entries, "misfit": E,
                       "l2": "inputs larger than L2 (forward velocity store per pass)"},
            "phases_ms_per_step": phases, "clocks": clk}


def run_batching(args, rank, world):
    """The batching recipe: 64 shots over three seeded quadtree meshes (p = 2, 3, 5 with
    N_r = 16, 32, 48; elements with 4 to 8 line elements, so n_b varies inside each mesh
    and every mesh runs as one launch per step padded to its largest n_b), 1500 steps.
    One step = set-up of the starting model + forward, misfit, adjoint and gradient of
    every shot of the three meshes, in passes of 8 shots; the meshes run one after another."""
    import torch
    from paper_2501_06748_gb300 import build
    build.build()
    from paper_2501_06748_gb300 import sbfwi as lib
    from paper_2501_06748_gb300 import shots
    from sbfwi_inputs import batching_workload
    if rank != 0:
        return None
    torch.cuda.set_device(0)
    K = args.time_steps or 1500
    per_pass = args.shots_per_pass or 8
    meshes = []
    for i in range(3):
        w = batching_workload(i, K=K)
        M = lib.Mesh.from_inputs(w.mesh, w.n_r)
        mt = lib.Model(M, w.c, w.rho_true, w.dt)
        obs = np.concatenate([lib.forward(mt, w.src_nodes[lo:lo + per_pass], w.wavelets[lo:lo + per_pass],
                                          w.rec_nodes, keep=False)[0]
                              for lo in range(0, w.n_shots, per_pass)])
        del mt
        meshes.append((w, M, obs))

    # schedule per mesh: element kernel x solve schedule timed on 16 steps of all its passes
    choices = []
    for w, M, _ in meshes:
        if args.autotune:
            from paper_2501_06748_gb300 import autotune
            mt = lib.Model(M, w.c, w.rho_start, w.dt)
            choices.append(autotune.tune(mt, w.src_nodes, w.wavelets, w.rec_nodes, shots_per_pass=per_pass))
            del mt
        else:
            choices.append(None)

    def epoch(times=None):
        for k, (w, M, obs) in enumerate(meshes):
            t0 = time.perf_counter()
            md = lib.Model(M, w.c, w.rho_start, w.dt)
            if choices[k] is not None:
                from paper_2501_06748_gb300 import autotune
                autotune.apply(md, choices[k])
            shots.misfit_and_gradient(md, w.src_nodes, w.wavelets, w.rec_nodes, obs, shots_per_pass=per_pass)
            if times is not None:
                times[k] += time.perf_counter() - t0

    for _ in range(max(3, args.warmup)):
        epoch()
    clocks = ClockSampler(os.path.join(args.clock_log, "clocks_batching.csv"))
    clocks.start()
    times = [0.0] * 3
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        epoch(times)
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / args.steps
    clk = clocks.stop()
    units = [w.mesh.n_elem * w.n_r * w.K * w.n_shots for w, _, _ in meshes]
    rows = []
    for (w, M, _), u, t in zip(meshes, units, times):
        nb = w.mesh.n_b
        rows.append({"mesh": w.name, "elements": w.mesh.n_elem, "p": w.mesh.p, "N_r": w.n_r,
                     "n_b": {str(v): int(c) for v, c in zip(*np.unique(nb, return_counts=True))},
                     "padded_n_b": int(M.n_b), "global_nodes": w.mesh.n_nodes, "shots": w.n_shots,
                     "s_per_step": t / args.steps, "units_per_s": u / (t / args.steps)})
    for row, ch in zip(rows, choices):
        if ch is not None:
            row["schedule"] = {"element": ch["element"], "solve": ch["solve"],
                               "candidates_ms_per_step": {f'{c["element"]}/{c["solve"]}': (
                                   None if c["s_per_step"] is None else round(1e3 * c["s_per_step"], 4))
                                   for c in ch["candidates"]}}
    return {"metric": "batching: element-radial-node-steps/s fwd+adj+grad over 3 uneven quadtree meshes",
            "value": sum(units) / sec, "unit": "element-radial-node-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": 1e3 * sec, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"batching: 64 shots over 3 seeded quadtree meshes (16x16 root cells refined 2 "
                                   f"levels around two elliptical flaws, 2:1 balanced, hanging vertices), p = 2, 3, 5, "
                                   f"N_r = 16, 32, 48, {K} steps, {per_pass} shots per pass",
                       "rows": rows, "l2": "inputs larger than L2 (forward velocity store 12-89 GB per pass)"},
            "clocks": clk}


def run_diffcheck(args, rank, world):
    """The differentiation recipe's problem (128x128 elements, p = 4, N_r = 32, 16 shots, 64
    receivers, 512x512 density grid) end to end at a stated step count: the exact gradient
    (checkpointed forward, recomputed in the adjoint) against central differences of the
    misfit along random directions of the grid, the paper's kernel at the same point against
    the exact gradient, then projected L-BFGS iterations (memory 10) from the homogeneous
    start towards the flawed model on the exact gradient (or the paper's kernel)."""
    import torch
    from paper_2501_06748_gb300 import build
    build.build()
    from paper_2501_06748_gb300 import sbfwi as lib, inversion
    from sbfwi_inputs import diff_workload
    if rank != 0:
        return None
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    K = args.time_steps or 500
    w = diff_workload(K=K)
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    wav = torch.tensor(w.wavelets, device=dev)
    rho_start = torch.tensor(w.rho_start, device=dev)
    m_true = lib.Model(M, w.c, torch.tensor(w.rho_true, device=dev), w.dt)
    observed = torch.cat([lib.forward(m_true, w.src_nodes[lo:lo + 8], wav[lo:lo + 8], w.rec_nodes, keep=False)[0]
                          for lo in range(0, w.n_shots, 8)])
    del m_true
    units = w.mesh.n_elem * w.n_r * K * w.n_shots
    stats = {"evaluations": 0, "seconds": 0.0}

    def timed(fg):
        def run(x):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = fg(x)
            torch.cuda.synchronize()
            stats["evaluations"] += 1
            stats["seconds"] += time.perf_counter() - t0
            return out
        return run

    clocks = ClockSampler(os.path.join(args.clock_log, "clocks_diffcheck.csv"))
    clocks.start()
    # the exact gradient against central differences
    fg_exact = inversion.objective(M, w.c, w.dt, w.src_nodes, wav, w.rec_nodes, observed, ckpt_every=lib.CKPT_AUTO,
                                   exact=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    E0, g = fg_exact(rho_start)
    torch.cuda.synchronize()
    t_exact = time.perf_counter() - t0
    f = inversion.misfit_only(M, w.c, w.dt, w.src_nodes, wav, w.rec_nodes, observed)
    rng = np.random.default_rng(16)
    h = 1e-5
    errs = []
    for _ in range(args.fd_directions):
        d = torch.tensor(rng.standard_normal(w.rho_start.shape), device=dev)
        fd = (f(rho_start + h * d) - f(rho_start - h * d)) / (2 * h)
        errs.append(abs(float(torch.sum(g * d)) - fd) / abs(fd))
    # the paper's kernel at the same point, measured against the exact derivative: its cosine,
    # and whether -g_kernel is a descent direction of the discrete misfit
    fg_kernel = inversion.objective(M, w.c, w.dt, w.src_nodes, wav, w.rec_nodes, observed, ckpt_every=lib.CKPT_AUTO)
    _, g_k = fg_kernel(rho_start)
    gx, gk = g.flatten(), g_k.flatten()
    cos_k = float(torch.dot(gx, gk) / (torch.linalg.norm(gx) * torch.linalg.norm(gk)))
    # L-BFGS (the box keeps the density where the radial scheme is stable) with the chosen gradient
    fg = timed(fg_exact if args.lbfgs_gradient == "exact" else fg_kernel)
    _, hist = inversion.lbfgs(fg, rho_start, lo=0.2, hi=2.0, iters=args.lbfgs_iters, m=10)
    clk = clocks.stop(0)
    value = units * stats["evaluations"] / stats["seconds"]
    return {"metric": "differentiation: exact gradient vs central differences, L-BFGS; "
                      "element-radial-node-steps/s of the L-BFGS evaluations",
            "value": value, "unit": UNIT, "n_gpus": 1, "steps": stats["evaluations"], "warmup": 1,
            "ms_per_step": 1e3 * stats["seconds"] / max(1, stats["evaluations"]), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"diff recipe at {K} of its 8000 steps: 128x128 square S-elements, p=4, N_r=32, "
                                   "16 Ricker shots in passes of 8, 64 receivers, 512x512 density grid, checkpoints "
                                   "at the memory-optimal interval (forward recomputed in the adjoint)",
                       "time_steps": K, "fd_directions": args.fd_directions, "fd_step": h,
                       "lbfgs_iterations": args.lbfgs_iters, "lbfgs_memory": 10, "box": [0.2, 2.0],
                       "l2": "inputs larger than L2 (checkpoints and recompute windows of 16 shots)"},
            "fd_check": {"gradient": "exact (SBFWI_GRAD_EXACT)", "max_rel_err": float(max(errs)) if errs else None,
                         "rel_errs": [float(e) for e in errs], "exact_gradient_seconds": t_exact, "misfit": E0},
            "paper_kernel": {"cosine_with_exact": cos_k, "descent_direction": cos_k > 0},
            "lbfgs": {"gradient": args.lbfgs_gradient, "misfit_history": [float(x) for x in hist],
                      "evaluations": stats["evaluations"],
                      "seconds": stats["seconds"], "reduction": float(hist[-1] / hist[0]) if hist[0] else None},
            "clocks": clk}


def run_reference(args, rank, world):
    """The oracle (the only reference this path has) on the host cores, rank 0 only."""
    if rank != 0:
        return None
    for _ in range(args.warmup):
        run_oracle_sample()
    rates, secs = [], []
    sample = None
    for _ in range(args.steps):
        r, s, sample = run_oracle_sample()
        rates.append(r)
        secs.append(s)
    value = float(np.sum([r * s for r, s in zip(rates, secs)]) / np.sum(secs))
    hc = host_cpu()
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "size recipe (p=4, N_r=32, 8 shots), bounded sample: " + sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "host_nproc": hc["nproc"], "cpu_model": hc["cpu_model"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--requests", type=int, default=64, help="serving config: number of requests")
    ap.add_argument("--config", choices=["size", "diff", "serving", "paper", "batching", "diffcheck", "solid"],
                    default="size",
                    help="size: 64x64 elements, 8 shots, 2000 steps, stored forward field (the default); "
                         "diff: 128x128 elements, 16 shots, 8000 steps, checkpointed adjoint; "
                         "serving: forward-modelling requests with continuous batching; "
                         "paper: the paper's plate recipe at its Table 1 element counts; "
                         "batching: 64 shots over 3 quadtree meshes with uneven elements; "
                         "diffcheck: the diff problem with an FD check of the exact gradient and L-BFGS; "
                         "solid: 3-D hexahedral S-elements")
    ap.add_argument("--solid-p", type=int, default=2, help="solid config: face order (1 or 2)")
    ap.add_argument("--fd-directions", type=int, default=16, help="diffcheck config: random directions")
    ap.add_argument("--lbfgs-iters", type=int, default=20, help="diffcheck config: L-BFGS iterations")
    ap.add_argument("--lbfgs-gradient", choices=["exact", "kernel"], default="exact",
                    help="diffcheck config: L-BFGS on the exact derivative or on the paper's kernel")
    ap.add_argument("--clock-log", default=tempfile.gettempdir(),
                    help="directory for the raw nvidia-smi clock samples of the timed region")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="batching config: keep the default schedule instead of timing the candidates per mesh")
    ap.add_argument("--paper-mesh", choices=["voronoi", "square"], default="voronoi",
                    help="paper config: centroidal Voronoi polygons (the paper's) or squares")
    ap.add_argument("--time-steps", type=int, default=0, help="Newmark steps (0: the config's)")
    ap.add_argument("--shots", type=int, default=0, help="shots per rank (0: the config's)")
    ap.add_argument("--shots-per-pass", type=int, default=0, help="0 = all shots in one pass")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-one-shot", dest="one_shot", action="store_false",
                    help="skip the one-shot-per-pass comparison")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.config == "serving":
        out = run_serving(args, rank, world)
    elif args.config == "paper":
        out = run_paper(args, rank, world)
    elif args.config == "batching":
        out = run_batching(args, rank, world)
    elif args.config == "diffcheck":
        out = run_diffcheck(args, rank, world)
    elif args.config == "solid":
        out = run_solid(args, rank, world)
    else:
        out = run_ours(args, rank, world)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
