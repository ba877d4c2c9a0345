#!/usr/bin/env python
"""Throughput of one PINN loss + gradient step (collocation points per second).

Default workload: the steady lid-driven cavity at Re = 100 with Gaussian Fourier
features (128 frequencies, sigma 1), random weight factorisation and a 6 x 256
tanh MLP -> (u, v, p), 65,536 interior + 4 x 1,024 wall points, BF16 jet GEMMs
with FP32 accumulation.  A step is one pinn_loss_grad call (embedding -> jet
forward -> residual/loss -> adjoint -> ordered FP64 reductions).

Prints one JSON line.  Besides the device-resident throughput it reports the
end-to-end figure through the public API with host buffers, the phase timings and
roofline of the dominant kernel, plain torch double-backward autograd on the same
GPU, and the FP64 oracle on the host cores (a baseline only).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--precision fp32|tf32|bf16]
Under torchrun every rank runs an independent replica (no collectives on the data
path); the value is all points processed over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "collocation pts/sec per loss+grad step"
UNIT = "points/s"
CSRC = os.path.join(ROOT, "paper_2604_15645_gb300", "csrc")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ns_cavity_6x256")
    ap.add_argument("--precision", default=None)
    ap.add_argument("--n-res", type=int, default=None, help="interior points (default: the workload's own)")
    ap.add_argument("--no-torch", action="store_true", help="skip the torch autograd baseline")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--chunk-points", type=int, default=0, help="process the batch in chunks of this many points")
    ap.add_argument("--value-split", dest="value_split", action="store_true", default=None,
                    help="BF16: split the weights into high/low halves on the value rows only")
    ap.add_argument("--terms", action="store_true",
                    help="also time the loss-balancing step: per-term gradients + weight update (Sec. 2.6.4)")
    ap.add_argument("--full-split", dest="value_split", action="store_false",
                    help="BF16: split the weights on every jet row (overrides the workload's setting)")
    ap.add_argument("--no-graph", dest="graph", action="store_false", default=True,
                    help="launch every step eagerly instead of replaying one captured CUDA graph")
    return ap.parse_args()


# ------------------------------------------------------------------------------ helpers

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(vals, ws_n, device=None):
    """Element-wise maximum over ranks of per-rank timings; every rank gets it."""
    import torch
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    if ws_n > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(x) for x in t]


def whole_job_rate(points_per_rank, ws_n, ms):
    """Points of all ranks (each rank runs its own replica) per second of the slowest."""
    return points_per_rank * ws_n / (ms / 1e3)


def blas_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        n = [i["num_threads"] for i in info if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


def src_sha():
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = []
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        smax = 0.0
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
            except ValueError:
                continue
            for i, n in enumerate(names):
                if r[5 + i].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------ workload

def workload_inputs(name, n_res=None):
    from synth import make_workload
    w, params, B, batch = make_workload(name)
    if n_res is not None and n_res != batch.n_res:
        frac = n_res / batch.n_res
        batch = make_workload(name, n_res=n_res, n_ic=int(round(batch.n_ic * frac)),
                              n_bc=int(round(batch.n_bc * frac)))[3]
    return w, params, B, batch


def layer_dims_of(spec):
    first_in = 2 * spec.ff_m if spec.ff_m else spec.d_in
    dims, prev = [], first_in
    for width in spec.widths:
        dims.append((prev, width))
        prev = width
    return dims


def algorithmic_work(w, n_cols, n_pts, precision):
    """Algorithmic FLOPs and HBM bytes of one step, per GEMM phase.

    Units: a jet row of the method, 4 per interior point and 1 per initial or
    boundary point (n_cols = 4 N_res + N_ic + N_bc); the kernels also carry three zero
    rows for every initial/boundary point, which is layout, not algorithmic work.  The
    BF16 value-row low halves count once per point (n_pts).  Per row and hidden GEMM layer (fan_in fi,
    fan_out fo), FLOPs are 2 fi fo for each of forward, adjoint and weight
    gradient (no adjoint into the first GEMM after a frozen Fourier embedding; the
    tiny raw-coordinate first layer is not a GEMM).  Bytes per row and layer,
    e = element size (only the activations A are stored; the adjoint is written in
    them):
      forward   read A_in (fi e) + write A_out (fo e)   [+ BF16 value-row low halves,
                                                         2 (fi + fo) bytes per point]
      adjoint   read Zbar_in (fo e) + A_in (fi e) + write Zbar_out (fi e)
      weights   read Zbar (fo e) + A_in (fi e)
    """
    spec = w.spec
    e = 2 if precision == "bf16" else 4
    lo = 2.0 if precision == "bf16" else 0.0   # (fi + fo) * 2 bytes per point
    cols = float(n_cols)
    fl = {"fwd_gemm": 0.0, "dw_gemm": 0.0, "adj_gemm": 0.0}
    by = {"fwd_gemm": 0.0, "dw_gemm": 0.0, "adj_gemm": 0.0}
    for li, (fi, fo) in enumerate(layer_dims_of(spec)):
        if li == 0 and not spec.ff_m:
            continue
        fl["fwd_gemm"] += 2.0 * fi * fo * cols
        by["fwd_gemm"] += cols * (fi + fo) * e + n_pts * lo * (fi + fo)
        fl["dw_gemm"] += 2.0 * fi * fo * cols
        by["dw_gemm"] += cols * (fo + fi) * e
        if li >= 1:
            fl["adj_gemm"] += 2.0 * fi * fo * cols
            by["adj_gemm"] += cols * (fo + 2 * fi) * e
    return fl, by


# ------------------------------------------------------------------------------ arms

def oracle_sample_rate(w, params, B, batch, target_s=10.0, n_res=8192, net=None):
    """FP64 oracle throughput on a bounded sample of the workload (host cores).  With
    `net`, the same sample also runs through the library, and the line states the
    library's relative error against the oracle there (loss total, gradient L2)."""
    import oracle
    frac = min(1.0, n_res / max(batch.n_res, 1))
    sub = batch.subset(min(n_res, batch.n_res), int(round(batch.n_ic * frac)), int(round(batch.n_bc * frac)))
    m = oracle.Model.from_spec(w.spec)
    lam = (w.problem.lambda_pde, w.problem.lambda_ic, w.problem.lambda_bc)
    pts = sub.n_res + sub.n_ic + sub.n_bc
    t0 = time.perf_counter()
    calls = 0
    while True:
        oracle.loss_and_grad(m, params, B, sub, w.problem.nu, lam)
        calls += 1
        if time.perf_counter() - t0 >= target_s:
            break
    dt = time.perf_counter() - t0
    out = {"value": pts * calls / dt, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
           "sample": f"{sub.n_res} interior + {sub.n_ic} initial + {sub.n_bc} boundary points of {w.name}, "
                     f"{calls} loss+grad call(s), FP64 numpy"}
    if net is not None:
        import torch
        from paper_2604_15645_gb300 import api
        terms, g = oracle.loss_and_grad(m, params, B, sub, w.problem.nu, lam)
        prob = api.make_problem(w.problem.nu, *lam)
        t_gpu, g_gpu = net.loss_grad(torch.tensor(params, device=net.device), api.DeviceBatch.from_host(sub, net.device),
                                     prob)
        t0_gpu = float(t_gpu[0])
        g_gpu = g_gpu.cpu().numpy().astype(np.float64)
        out["library_error_vs_oracle"] = {
            "loss_rel": abs(t0_gpu - terms["total"]) / abs(terms["total"]),
            "grad_rel_l2": float(np.linalg.norm(g_gpu - g) / np.linalg.norm(g)), "points": pts}
    return out


def host_description():
    """Architecture, CPU model and logical core count of the host."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware") and model is None:
                    model = line.split(":", 1)[1].strip()
    except OSError:
        pass
    names = {"0xd4f": "Arm Neoverse V2 (0xd4f)", "0xd40": "Arm Neoverse V1 (0xd40)"}
    return {"arch": platform.machine(), "model": names.get(model, model), "nproc": os.cpu_count()}


def oracle_one_core_rate(workload, n_res=2048, target_s=5.0):
    """The oracle on one host core: a child process with every BLAS pool at one thread,
    on a smaller sample of the same workload."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    code = (
        "import sys, time, json\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import oracle\n"
        "from synth import make_workload\n"
        f"w, p, B, b = make_workload({workload!r})\n"
        f"f = min(1.0, {n_res} / max(b.n_res, 1))\n"
        f"s = b.subset(min({n_res}, b.n_res), int(round(b.n_ic * f)), int(round(b.n_bc * f)))\n"
        "m = oracle.Model.from_spec(w.spec)\n"
        "lam = (w.problem.lambda_pde, w.problem.lambda_ic, w.problem.lambda_bc)\n"
        "t0 = time.perf_counter(); n = 0\n"
        "while True:\n"
        "    oracle.loss_and_grad(m, p, B, s, w.problem.nu, lam); n += 1\n"
        f"    if time.perf_counter() - t0 >= {target_s}: break\n"
        "dt = time.perf_counter() - t0\n"
        "pts = s.n_res + s.n_ic + s.n_bc\n"
        "print(json.dumps({'value': pts * n / dt, 'unit': 'points/s', 'cores': 1, "
        "'sample': f'{s.n_res} interior + {s.n_ic} initial + {s.n_bc} boundary points, {n} call(s)'}))\n")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        return json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:   # reported, not hidden
        return {"error": repr(e)[:300]}


TORCH_MAX_POINTS = 320000   # above this the double-backward graph of the larger networks outgrows HBM


def torch_autograd_rate(w, params, B, batch, steps=5, warmup=2, tf32=False):
    """The paper's recipe (torch.autograd.grad create_graph + loss.backward), FP32,
    TF32 off, same parameters and points, CUDA events.  Batches above TORCH_MAX_POINTS
    run on a leading sample of every point set, scaled alike (points/s is a per-point
    rate at a batch far past the launch-bound regime)."""
    import torch
    from baseline import torch_autograd as ta
    n_all = batch.n_res + batch.n_ic + batch.n_bc
    sample = None
    if n_all > TORCH_MAX_POINTS:
        f = TORCH_MAX_POINTS / n_all
        nr, ni, nb = (int(batch.n_res * f), int(batch.n_ic * f), int(batch.n_bc * f))
        batch = batch.subset(nr, ni, nb)
        sample = f"{nr} interior + {ni} initial + {nb} boundary points (the leading {f:.3f} of each set)"

    torch.backends.cuda.matmul.allow_tf32 = tf32
    torch.backends.cudnn.allow_tf32 = tf32
    model = ta.TorchPINN(w.spec, params, B, "cuda", torch.float32)
    bt = ta.batch_to_torch(batch, "cuda", torch.float32)
    lam = (w.problem.lambda_pde, w.problem.lambda_ic, w.problem.lambda_bc)

    def step():
        model.zero_grad()
        total, _ = ta.loss(model, bt, w.problem.nu, lam)
        total.backward()
        return total
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    pts = batch.n_res + batch.n_ic + batch.n_bc
    out = {"value": pts / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "dtype": "f32 (tf32 off)",
           "how": "torch.autograd.grad(create_graph=True) input derivatives + loss.backward(), eager"}
    if sample:
        out["sample"] = sample
    return out


def run_family(args, ws_n, rank, local):
    """The many-network workload: 64 independent Burgers nets, one graph-captured
    training step (loss, adjoint, fused Adam) per timed step."""
    import torch
    from paper_2604_15645_gb300 import _lib, api
    from synth import make_family
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fam = make_family(64)
    precision = args.precision or "bf16"
    multi = api.PinnMulti([s for s, _, _, _ in fam], precision, device=dev)
    multi.set_inputs([api.DeviceBatch.from_host(b, device=dev) for _, _, b, _ in fam],
                     [api.make_problem(pr.nu) for _, _, _, pr in fam])
    p0 = np.concatenate([p for _, p, _, _ in fam]).astype(np.float32)
    params = torch.tensor(p0, device=dev)
    grad, m, v = (torch.zeros_like(params) for _ in range(3))
    multi.autotune(params, grad, os.path.join(ROOT, "paper_2604_15645_gb300", "autotune_cache.json"))
    n_pts = sum(b.n_res + b.n_ic + b.n_bc for _, _, b, _ in fam)
    step = 0
    for _ in range(args.warmup):
        step += 1
        multi.train_step(params, grad, m, v, step)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws_n > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step += 1
        multi.train_step(params, grad, m, v, step)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    status = multi.status_poll()
    ms_max, = max_over_ranks([ms], ws_n, dev)
    if rank != 0:
        return None
    engines = multi.engines()
    return {
        "metric": METRIC, "value": round(whole_job_rate(n_pts, ws_n, ms_max), 1), "unit": UNIT, "n_gpus": ws_n,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": precision, "data": "synthetic",
        "config": {"workload": "burgers_family_64", "networks": 64, "points_per_step": n_pts,
                   "params": int(params.numel()), "step": "loss + adjoint + fused Adam, one CUDA graph",
                   "engines": {"tc": engines.count("tc"), "cuda_cores": engines.count("cuda_cores")},
                   "parallelism": f"replicas x{ws_n}"},
        "clocks": clk, "device_status": status,
    }


def run_ours(args, ws_n, rank, local):
    import torch
    from paper_2604_15645_gb300 import _lib, api
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w, params, B, batch = workload_inputs(args.workload, args.n_res)
    precision = args.precision or w.precision
    value_split = (w.value_split if args.value_split is None else args.value_split) and precision == "bf16"
    net = api.PinnNet.from_spec(w.spec, precision, device=dev, chunk_points=args.chunk_points,
                                value_split=value_split)
    if B is not None:
        net.set_ff_matrix(B)
    db = api.DeviceBatch.from_host(batch, device=dev)
    p = torch.tensor(params, device=dev)
    grad = torch.empty_like(p)
    prob = api.make_problem(w.problem.nu, w.problem.lambda_pde, w.problem.lambda_ic, w.problem.lambda_bc)
    n_pts = batch.n_res + batch.n_ic + batch.n_bc
    ncols = 4 * batch.n_res + batch.n_ic + batch.n_bc
    ws_bytes = net.workspace_bytes(*db.sizes)

    def barrier():
        if ws_n > 1:
            torch.distributed.barrier()

    # warm-up: eager steps, then (graph mode) the capture and one replay
    for _ in range(args.warmup):
        net.loss_grad(p, db, prob, grad=grad)
    if args.graph:
        net.set_graph(True)
        for _ in range(2):
            net.loss_grad(p, db, prob, grad=grad)
    torch.cuda.synchronize()
    assert net.status_poll() == 0, "device status after warm-up"

    clocks = ClockSampler(local)
    clocks.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        net.loss_grad(p, db, prob, grad=grad)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    status = net.status_poll()

    # the spread of single steps: the same K calls again, an event pair around each
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in ev:
        a.record(stream)
        net.loss_grad(p, db, prob, grad=grad)
        b.record(stream)
    torch.cuda.synchronize()
    per_step = np.array([a.elapsed_time(b) for a, b in ev])

    # per-phase kernel times: the same K steps again, launched eagerly with a CUDA
    # event pair around each launch group on the launching stream (graph replays
    # cannot carry them); the kernels are the ones the timed region replays
    _lib.pinn_set_profiling(net.h, True)
    for _ in range(args.steps):
        net.loss_grad(p, db, prob, grad=grad)
    torch.cuda.synchronize()
    prof = _lib.pinn_profile_read(net.h)
    _lib.pinn_set_profiling(net.h, False)

    # end to end through the public API with host buffers: per step, H2D of the
    # collocation sets from pinned memory, the step, D2H of the loss terms.
    host = {k: torch.tensor(getattr(batch, k)).pin_memory() for k in ("x_res", "x_ic", "g_ic", "x_bc", "g_bc")}
    loss_host = torch.empty(8, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = loss_host.numel() * loss_host.element_size()

    def e2e_step():
        for k, t in host.items():
            getattr(db, k).copy_(t, non_blocking=True)
        terms, _ = net.loss_grad(p, db, prob, grad=grad)
        loss_host.copy_(terms, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    for _ in range(2):
        e2e_step()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / args.steps
    barrier()

    # the loss-balancing step (per-term gradients + weight update), if asked for
    terms_ms = None
    if args.terms:
        grads = torch.empty(3, p.numel(), dtype=torch.float32, device=dev)
        lam = torch.ones(3, dtype=torch.float64, device=dev)
        for _ in range(2):
            net.loss_grad_terms(p, db, prob, grads=grads)
            net.loss_balance(grads, lam)
        torch.cuda.synchronize()
        barrier()
        t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0e.record(stream)
        for _ in range(args.steps):
            net.loss_grad_terms(p, db, prob, grads=grads)
            net.loss_balance(grads, lam)
        t1e.record(stream)
        torch.cuda.synchronize()
        terms_ms = t0e.elapsed_time(t1e) / args.steps

    # max over ranks
    ms_max, e2e_ms_max = max_over_ranks([ms, e2e_s * 1e3], ws_n, dev)
    if rank != 0:
        return None

    peaks, peak_src = load_peaks()
    flops, nbytes = algorithmic_work(w, ncols, n_pts, precision)
    phases = {k: prof[k] for k in ("fwd_gemm", "dw_gemm", "adj_gemm", "out_loss", "embed", "reduce", "rwf")}
    # the dominant kernel among those with an algorithmic work model (the GEMM phases)
    modelled = [k for k in phases if k in flops and phases[k][1] > 0] or list(phases)
    dom = max(modelled, key=lambda k: phases[k][0])
    dom_ms, dom_launches = prof[dom]
    roof, roof_alt = None, None
    if dom in flops and dom_launches > 0:
        per_launch_ms = dom_ms / dom_launches
        f_l = flops[dom] * args.steps / dom_launches
        b_l = nbytes[dom] * args.steps / dom_launches
        tflops = f_l / (per_launch_ms / 1e3) / 1e12
        gbs = b_l / (per_launch_ms / 1e3) / 1e9
        if net.tensor_core_layers(*db.sizes) > 0:
            # a kernel inside a long step: the sustained tensor peak (TF32 at half the BF16 rate)
            tpeak = peaks["bf16_tflops_sustained"] * (0.5 if precision == "tf32" else 1.0)
            tbound = "tensor"
        else:
            # CUDA-core FP32 FMA peak: 152 SMs x 128 FMA/clk x 2 FLOP x max SM clock
            tpeak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            tbound = "alu"
        compute = {"bound": tbound, "achieved": round(tflops, 2), "peak": round(tpeak, 1), "unit": "TFLOP/s",
                   "frac": round(tflops / tpeak, 4), "traffic": _traffic(dom, args.workload),
                   "kernel": dom, "flop_per_launch": f_l, "launch_ms": round(per_launch_ms, 4),
                   "peak_source": peak_src}
        memory = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                  "frac": round(gbs / peaks["hbm_gbs"], 4), "traffic": _traffic(dom, args.workload),
                  "kernel": dom, "bytes_per_launch": b_l, "launch_ms": round(per_launch_ms, 4),
                  "peak_source": peak_src}
        roof, roof_alt = (memory, compute) if memory["frac"] >= compute["frac"] else (compute, memory)

    out = {
        "metric": METRIC, "value": round(whole_job_rate(n_pts, ws_n, ms_max), 1), "unit": UNIT, "n_gpus": ws_n,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": precision, "data": "synthetic",
        "interior_points_per_s": round(whole_job_rate(batch.n_res, ws_n, ms_max), 1),
        "ms_per_step_single": {"p10": round(float(np.percentile(per_step, 10)), 4),
                               "p50": round(float(np.percentile(per_step, 50)), 4),
                               "p90": round(float(np.percentile(per_step, 90)), 4),
                               "how": "one event pair around each of K further steps (this rank)"},
        "config": {"workload": w.name, "pde": "ns_steady_2d" if w.spec.pde == 1 else w.spec.pde,
                   "network": f"{'FF' + str(2 * w.spec.ff_m) + ' -> ' if w.spec.ff_m else ''}"
                              f"{len(w.spec.widths)}x{w.spec.widths[0]} tanh -> {w.spec.d_out}"
                              f"{' RWF' if w.spec.rwf else ''}",
                   "n_res": batch.n_res, "n_ic": batch.n_ic, "n_bc": batch.n_bc, "points_per_step": n_pts,
                   "jet_columns": ncols, "parallelism": f"replicas x{ws_n}",
                   "workspace_gb": round(ws_bytes / 1e9, 2), "chunk_points": args.chunk_points,
                   "launch": "one CUDA graph per step" if args.graph else "eager launches",
                   "phase_timing": "CUDA events per launch group in an eager pass of the same K steps",
                   "bf16_weight_split": ("value rows" if value_split else "all rows") if precision == "bf16" else None,
                   "l2": f"working set {ws_bytes / 1e9:.2f} GB per step > 129 MB L2 (no flush needed)"},
        "e2e": {"value": round(whole_job_rate(n_pts, ws_n, e2e_ms_max), 1), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms_max, 4)},
        "gpu_launches": int(sum(v[1] for v in prof.values() if v[1] > 0)),
        "phases_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in prof.items()},
        "roofline": roof,
        "roofline_other": roof_alt,
        "jet_gemms": jet_gemm_rate(flops, prof, args.steps, peaks, precision),
        "loss_balance_step": None if terms_ms is None else {
            "ms_per_step": round(terms_ms, 4), "value": round(n_pts / (terms_ms / 1e3), 1), "unit": UNIT,
            "what": "one forward + three reverse sweeps (unweighted PDE/IC/BC gradients) + device weight update"},
        "clocks": clk,
        "device_status": status,
    }
    if not args.no_torch and ws_n == 1:
        try:
            tr = torch_autograd_rate(w, params, B, batch)
            tr["speedup"] = round(out["value"] / tr["value"], 2)
            out["torch_autograd"] = tr
        except Exception as e:   # reported, not hidden
            out["torch_autograd"] = {"error": repr(e)[:300]}
        try:
            tr = torch_autograd_rate(w, params, B, batch, tf32=True)
            tr["dtype"] = "f32 storage, tf32 matmuls"
            tr["speedup"] = round(out["value"] / tr["value"], 2)
            out["torch_autograd_tf32"] = tr
        except Exception as e:
            out["torch_autograd_tf32"] = {"error": repr(e)[:300]}
    if not args.no_cpu and ws_n == 1:
        out["cpu_baseline"] = oracle_sample_rate(w, params, B, batch, net=net)
        out["cpu_baseline"]["one_core"] = oracle_one_core_rate(w.name)
        out["cpu_baseline"]["host"] = host_description()
    return out


def jet_gemm_rate(flops, prof, steps, peaks, precision):
    """All jet GEMMs of the step together (forward, adjoint, weight gradient):
    algorithmic FLOPs over their summed device time, against the peak of the
    precision's engine (BF16: measured; TF32: measured BF16 x the nominal 1/2;
    FP32: CUDA-core FMA peak from unit counts and the maximum clock)."""
    ms = sum(prof[k][0] for k in ("fwd_gemm", "adj_gemm", "dw_gemm")) / steps
    if ms <= 0:
        return None
    tf = sum(flops.values()) / (ms / 1e3) / 1e12
    if precision == "fp32":
        p_sus = p_burst = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        src = "fp32 FMA: 152 SMs x 128 lanes x 2 FLOP x max clock"
    else:
        r = 0.5 if precision == "tf32" else 1.0
        p_sus, p_burst = r * peaks["bf16_tflops_sustained"], r * peaks["bf16_tflops"]
        src = "measured bf16" + (" x 1/2 (nominal tf32 ratio)" if r < 1 else "")
    return {"tflops": round(tf, 1), "ms_per_step": round(ms, 4), "frac_of_sustained": round(tf / p_sus, 4),
            "frac_of_burst": round(tf / p_burst, 4), "peak_source": src}


def _traffic(kernel, workload):
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(f"{workload}:{kernel}")
    if not e or e.get("src_sha") != src_sha():
        return None
    return e.get("bytes_per_launch")


def run_reference(args, ws_n, rank):
    """The oracle, as it stands, on the host cores: each step is one FP64 loss+grad
    call on a bounded sample of the workload (rank 0 only)."""
    if rank != 0:
        return None
    import oracle
    w, params, B, batch = workload_inputs(args.workload)
    n_res = 1024
    frac = n_res / max(batch.n_res, 1)
    sub = batch.subset(min(n_res, batch.n_res), int(round(batch.n_ic * frac)), int(round(batch.n_bc * frac)))
    m = oracle.Model.from_spec(w.spec)
    lam = (w.problem.lambda_pde, w.problem.lambda_ic, w.problem.lambda_bc)
    for _ in range(args.warmup):
        oracle.loss_and_grad(m, params, B, sub, w.problem.nu, lam)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.loss_and_grad(m, params, B, sub, w.problem.nu, lam)
    dt = (time.perf_counter() - t0) / args.steps
    pts = sub.n_res + sub.n_ic + sub.n_bc
    v = pts / dt
    sample = f"{sub.n_res} interior + {sub.n_ic} initial + {sub.n_bc} boundary points of {w.name} per step"
    return {"impl": "reference", "metric": METRIC, "value": round(v, 2), "unit": UNIT, "n_gpus": ws_n,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "sample": sample, "parallelism": "host cores"},
            "cpu_baseline": {"value": round(v, 2), "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 2), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    ws_n, rank, local = dist_setup()
    if args.impl == "reference":
        out = run_reference(args, ws_n, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    import torch
    if ws_n > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2604_15645_gb300 import _lib
    _lib.load()
    if args.workload == "burgers_family_64":
        out = run_family(args, ws_n, rank, local)
    else:
        out = run_ours(args, ws_n, rank, local)
    if out is not None:
        print(json.dumps(out), flush=True)
    if ws_n > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
