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
DEFAULT_WORKLOAD = "ns_cavity_6x256"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
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
    ap.add_argument("--no-suite", dest="suite", action="store_false", default=True,
                    help="default workload only: skip the other configurations' sub-records")
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


def src_sha(files=None):
    """Hash of the kernel sources a measurement depends on: the named files of the
    package's csrc (the kernel's own file, the headers it includes and the launch plan),
    or all of them."""
    h = hashlib.sha256()
    for name in sorted(files) if files else sorted(os.listdir(CSRC)):
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


def algorithmic_work(w, n_cols, n_pts, precision, engines=None):
    """Algorithmic FLOPs and HBM bytes of one step, per GEMM phase.

    Units: a jet row of the method, 4 per interior point and 1 per initial or
    boundary point (n_cols = 4 N_res + N_ic + N_bc); the kernels also carry three zero
    rows for every initial/boundary point, which is layout, not algorithmic work.  Per
    row and hidden GEMM layer (fan_in fi, fan_out fo), FLOPs are 2 fi fo for each of
    forward, adjoint and weight gradient (no adjoint into the first GEMM after a frozen
    Fourier embedding; the tiny raw-coordinate first layer is not a GEMM).  Bytes per
    row and layer, e = element size (only the activations A are stored; the adjoint is
    written in them):
      forward   read A_in (fi e) + write A_out (fo e)
      adjoint   read Zbar_in (fo e) + A_in (fi e) + write Zbar_out (fi e)
      weights   read Zbar (fo e) + A_in (fi e)
    A layer whose adjoint and weight gradient run as one fused kernel (engines[li] == 2)
    books both GEMMs' FLOPs under "adjdw_gemm", with the adjoint's bytes (the weight
    gradient reads the same two arrays in the same pass).
    Returns (flops, bytes, scheme_bytes): scheme_bytes are the extra bytes of this
    library's BF16 precision scheme (the low halves of the value rows, 2 (fi + fo)
    bytes per point in the forward), which are not the method's work.
    """
    spec = w.spec
    e = 2 if precision == "bf16" else 4
    lo = 2.0 if precision == "bf16" else 0.0
    cols = float(n_cols)
    keys = ("fwd_gemm", "dw_gemm", "adj_gemm", "adjdw_gemm")
    fl, by, sch = ({k: 0.0 for k in keys} for _ in range(3))
    for li, (fi, fo) in enumerate(layer_dims_of(spec)):
        if li == 0 and not spec.ff_m:
            continue
        fl["fwd_gemm"] += 2.0 * fi * fo * cols
        by["fwd_gemm"] += cols * (fi + fo) * e
        sch["fwd_gemm"] += n_pts * lo * (fi + fo)
        if li >= 1 and engines is not None and engines[li] == 2:
            fl["adjdw_gemm"] += 4.0 * fi * fo * cols
            by["adjdw_gemm"] += cols * (fo + 2 * fi) * e
            continue
        fl["dw_gemm"] += 2.0 * fi * fo * cols
        by["dw_gemm"] += cols * (fo + fi) * e
        if li >= 1:
            fl["adj_gemm"] += 2.0 * fi * fo * cols
            by["adj_gemm"] += cols * (fo + 2 * fi) * e
    return fl, by, sch


def tensor_peaks(peaks, precision):
    """(burst, sustained) peak of the engine the jet GEMMs run on, TFLOP/s, and its source:
    BF16 measured; TF32 measured BF16 x the nominal 1/2; FP32 CUDA-core FMA from unit
    counts and the maximum clock (152 SMs x 128 lanes x 2 FLOP)."""
    if precision == "fp32":
        p = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        return p, p, "alu", "fp32 FMA: 152 SMs x 128 lanes x 2 FLOP x max clock"
    r = 0.5 if precision == "tf32" else 1.0
    return (r * peaks["bf16_tflops"], r * peaks["bf16_tflops_sustained"], "tensor",
            "measured bf16" + (" x 1/2 (nominal tf32 ratio)" if r < 1 else ""))


def rooflines(dom, flops, nbytes, scheme, prof, steps, peaks, peak_src, precision, workload):
    """Roofline of the dominant kernel: jet-GEMM FLOPs per launch over its CUDA-event
    launch time against the burst peak of its engine (the kernel is timed in an eager
    pass of short steps, not inside a seconds-long loop), and the HBM model beside it."""
    dom_ms, dom_launches = prof[dom]
    if dom not in flops or dom_launches <= 0:
        return None, None
    per_launch_ms = dom_ms / dom_launches
    f_l = flops[dom] * steps / dom_launches
    b_l = nbytes[dom] * steps / dom_launches
    s_l = scheme[dom] * steps / dom_launches
    tflops = f_l / (per_launch_ms / 1e3) / 1e12
    gbs = b_l / (per_launch_ms / 1e3) / 1e9
    burst, _, bound, src = tensor_peaks(peaks, precision)
    traffic = _traffic(dom, workload if precision == "bf16" else f"{workload}/{precision}")
    compute = {"bound": bound, "achieved": round(tflops, 2), "peak": round(burst, 1), "unit": "TFLOP/s",
               "frac": round(tflops / burst, 4), "traffic": traffic, "kernel": dom, "flop_per_launch": f_l,
               "launch_ms": round(per_launch_ms, 4),
               "peak_source": f"{src}, burst ({peak_src})"}
    memory = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
              "frac": round(gbs / peaks["hbm_gbs"], 4), "traffic": traffic, "kernel": dom,
              "bytes_per_launch": b_l, "scheme_bytes_per_launch": s_l,
              "scheme_bytes_note": "BF16 value-row low halves of this library's precision scheme; not counted "
                                   "in bytes_per_launch or achieved",
              "launch_ms": round(per_launch_ms, 4), "peak_source": peak_src}
    return compute, memory


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


def library_error(w, params, B, batch, net, n_res):
    """The library's relative error against the FP64 oracle on a bounded sample of the
    workload (the leading n_res interior points and a proportional share of the
    initial and boundary sets): loss total and gradient, in L2 norm and per block."""
    import oracle
    import torch
    from paper_2604_15645_gb300 import api
    frac = min(1.0, n_res / max(batch.n_res, 1))
    sub = batch.subset(min(n_res, batch.n_res), int(round(batch.n_ic * frac)), int(round(batch.n_bc * frac)))
    lam = (w.problem.lambda_pde, w.problem.lambda_ic, w.problem.lambda_bc)
    t0 = time.perf_counter()
    terms, g = oracle.loss_and_grad(oracle.Model.from_spec(w.spec), params, B, sub, w.problem.nu, lam)
    oracle_s = time.perf_counter() - t0
    prob = api.make_problem(w.problem.nu, *lam)
    t_gpu, g_gpu = net.loss_grad(torch.tensor(params, device=net.device), api.DeviceBatch.from_host(sub, net.device),
                                 prob, out=torch.empty_like(net.loss_buf))
    return _error_record(float(t_gpu[0]), g_gpu.cpu().numpy().astype(np.float64), terms["total"], g, w.spec,
                         sub.n_res + sub.n_ic + sub.n_bc, oracle_s)


def _error_record(loss, grad, ref_loss, ref_grad, spec, points, oracle_s=None):
    blocks = _blocks(spec)
    worst = max(((n, float(np.linalg.norm(grad[a:b] - ref_grad[a:b]) /
                          max(np.linalg.norm(ref_grad[a:b]), 1e-3 * np.linalg.norm(ref_grad))))
                 for n, a, b in blocks), key=lambda x: x[1])
    out = {"loss_rel": abs(loss - ref_loss) / abs(ref_loss),
           "grad_rel_l2": float(np.linalg.norm(grad - ref_grad) / np.linalg.norm(ref_grad)),
           "grad_worst_block": {"block": worst[0], "rel": worst[1]}, "points": points}
    if oracle_s is not None:
        out["oracle_s"] = round(oracle_s, 2)
    return out


def _blocks(spec):
    """(name, start, stop) of every V, s, b block of the packed parameter vector."""
    out, off, prev = [], 0, (2 * spec.ff_m if spec.ff_m else spec.d_in)
    for l, fo in enumerate(list(spec.widths) + [spec.d_out], start=1):
        for name, n in (("V", fo * prev), ("s", fo if spec.rwf else 0), ("b", fo)):
            if n:
                out.append((f"{name}{l}", off, off + n))
                off += n
        prev = fo
    return out


def run_family(steps, warmup, ws_n, rank, local, precision="bf16", error_nets=4):
    """The many-network workload: 64 independent Burgers nets, one graph-captured
    training step (loss, adjoint, fused Adam) per timed step.  The error record
    compares the first step's gradient of the `error_nets` networks with the fewest
    points against the oracle on their whole batches."""
    import oracle
    import torch
    from paper_2604_15645_gb300 import api
    from synth import make_family
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fam = make_family(64)
    multi = api.PinnMulti([s for s, _, _, _ in fam], precision, device=dev)
    multi.set_inputs([api.DeviceBatch.from_host(b, device=dev) for _, _, b, _ in fam],
                     [api.make_problem(pr.nu) for _, _, _, pr in fam])
    p0 = np.concatenate([p for _, p, _, _ in fam]).astype(np.float32)
    params = torch.tensor(p0, device=dev)
    grad, m, v = (torch.zeros_like(params) for _ in range(3))
    t_tune = time.perf_counter()
    multi.autotune(params, grad, os.path.join(ROOT, "paper_2604_15645_gb300", "autotune_cache.json"))
    t_tune = time.perf_counter() - t_tune
    n_pts = sum(b.n_res + b.n_ic + b.n_bc for _, _, b, _ in fam)
    # error: one step from the initial parameters; grad holds the gradient before Adam
    params.copy_(torch.tensor(p0, device=dev))
    multi.train_step(params, grad, m, v, 1)
    torch.cuda.synchronize()
    err = None
    if rank == 0 and ws_n == 1 and error_nets:
        g = grad.cpu().numpy().astype(np.float64)
        loss = multi.loss.cpu().numpy()
        order = sorted(range(len(fam)), key=lambda i: fam[i][2].n_res)[:error_nets]
        recs = []
        for i in order:
            spec, p, b, pr = fam[i]
            t, rg = oracle.loss_and_grad(oracle.Model.from_spec(spec), p, None, b, pr.nu)
            r = _error_record(float(loss[i][0]), g[multi.offsets[i]:multi.offsets[i + 1]], t["total"], rg, spec,
                              b.n_res + b.n_ic + b.n_bc)
            r["net"] = i
            r["widths"] = f"{len(spec.widths)}x{spec.widths[0]}"
            recs.append(r)
        err = {"networks": recs, "loss_rel_max": max(r["loss_rel"] for r in recs),
               "grad_rel_l2_max": max(r["grad_rel_l2"] for r in recs)}
    params.copy_(torch.tensor(p0, device=dev))
    m.zero_()
    v.zero_()
    step = 0
    for _ in range(warmup):
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
    for _ in range(steps):
        step += 1
        multi.train_step(params, grad, m, v, step)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    clk = clocks.stop()
    status = multi.status_poll()
    # beside it, the same steps with one grouped tcgen05 launch per layer level
    multi.grouped = True
    for _ in range(warmup):
        step += 1
        multi.train_step(params, grad, m, v, step)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        step += 1
        multi.train_step(params, grad, m, v, step)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_grouped = e0.elapsed_time(e1) / steps
    multi.grouped = False
    ms_max, ms_grouped_max = max_over_ranks([ms, ms_grouped], ws_n, dev)
    if rank != 0:
        return None
    engines = multi.engines()
    return {
        "metric": METRIC, "value": round(whole_job_rate(n_pts, ws_n, ms_max), 1), "unit": UNIT, "n_gpus": ws_n,
        "steps": steps, "warmup": warmup, "ms_per_step": round(ms_max, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": precision, "data": "synthetic",
        "config": {"workload": "burgers_family_64", "networks": 64, "points_per_step": n_pts,
                   "params": int(params.numel()),
                   "step": "loss + adjoint + fused Adam, one CUDA graph, each network's launches on one of "
                           "32 worker streams",
                   "grouped_level_launches_ms_per_step": round(ms_grouped_max, 4),
                   "engines": {"tc": engines.count("tc"), "cuda_cores": engines.count("cuda_cores")},
                   "autotune_s": round(t_tune, 2), "parallelism": f"replicas x{ws_n}"},
        "library_error_vs_oracle": err, "clocks": clk, "device_status": status,
    }


def measure(name, precision, value_split, steps, warmup, ws_n, rank, local, graph=True, chunk_points=0,
            n_res=None, terms=False, e2e=True, spread=True):
    """One workload: the timed region (graph replays of pinn_loss_grad), the phase
    times, the roofline of the dominant kernel and (e2e) the end-to-end rate through
    the public API with host buffers.  Returns (record, context) on every rank."""
    import torch
    from paper_2604_15645_gb300 import _lib, api
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w, params, B, batch = workload_inputs(name, n_res)
    precision = precision or w.precision
    value_split = (w.value_split if value_split is None else value_split) and precision == "bf16"
    net = api.PinnNet.from_spec(w.spec, precision, device=dev, chunk_points=chunk_points, value_split=value_split)
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
    for _ in range(warmup):
        net.loss_grad(p, db, prob, grad=grad)
    if graph:
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
    for _ in range(steps):
        net.loss_grad(p, db, prob, grad=grad)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / steps
    clk = clocks.stop()
    status = net.status_poll()

    per_step = None
    if spread:
        # the spread of single steps: the same K calls again, an event pair around each
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
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
    for _ in range(steps):
        net.loss_grad(p, db, prob, grad=grad)
    torch.cuda.synchronize()
    prof = _lib.pinn_profile_read(net.h)
    _lib.pinn_set_profiling(net.h, False)

    e2e_ms, h2d, d2h = None, 0, 0
    if e2e:
        # end to end through the public API with host buffers: per step, H2D of the
        # collocation sets from pinned memory, the step, D2H of the loss terms.
        host = {k: torch.tensor(getattr(batch, k)).pin_memory() for k in ("x_res", "x_ic", "g_ic", "x_bc", "g_bc")}
        loss_host = torch.empty(8, dtype=torch.float64).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in host.values())
        d2h = loss_host.numel() * loss_host.element_size()

        def e2e_step():
            for k, t in host.items():
                getattr(db, k).copy_(t, non_blocking=True)
            terms_, _ = net.loss_grad(p, db, prob, grad=grad)
            loss_host.copy_(terms_, non_blocking=True)
            torch.cuda.current_stream().synchronize()
        for _ in range(2):
            e2e_step()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            e2e_step()
        e2e_ms = (time.perf_counter() - t0) / steps * 1e3
        barrier()

    terms_ms = None
    if terms:
        grads = torch.empty(3, p.numel(), dtype=torch.float32, device=dev)
        lam = torch.ones(3, dtype=torch.float64, device=dev)
        for _ in range(2):
            net.loss_grad_terms(p, db, prob, grads=grads)
            net.loss_balance(grads, lam)
        torch.cuda.synchronize()
        barrier()
        t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0e.record(stream)
        for _ in range(steps):
            net.loss_grad_terms(p, db, prob, grads=grads)
            net.loss_balance(grads, lam)
        t1e.record(stream)
        torch.cuda.synchronize()
        terms_ms = t0e.elapsed_time(t1e) / steps

    ms_max, e2e_ms_max = max_over_ranks([ms, e2e_ms or 0.0], ws_n, dev)
    ctx = dict(w=w, params=params, B=B, batch=batch, net=net, precision=precision)
    if rank != 0:
        return None, ctx

    peaks, peak_src = load_peaks()
    engines = net.layer_engines(*db.sizes)
    flops, nbytes, scheme = algorithmic_work(w, ncols, n_pts, precision, engines)
    phases = {k: prof[k] for k in ("fwd_gemm", "dw_gemm", "adj_gemm", "adjdw_gemm", "out_loss", "embed", "reduce",
                                   "rwf")}
    # the dominant kernel among those with an algorithmic work model (the GEMM phases)
    modelled = [k for k in phases if k in flops and phases[k][1] > 0] or list(phases)
    dom = max(modelled, key=lambda k: phases[k][0])
    roof, roof_alt = rooflines(dom, flops, nbytes, scheme, prof, steps, peaks, peak_src, precision, name)
    rec = {
        "metric": METRIC, "value": round(whole_job_rate(n_pts, ws_n, ms_max), 1), "unit": UNIT, "n_gpus": ws_n,
        "steps": steps, "warmup": warmup, "ms_per_step": round(ms_max, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": precision, "data": "synthetic",
        "interior_points_per_s": round(whole_job_rate(batch.n_res, ws_n, ms_max), 1),
        "config": {"workload": w.name, "pde": PDE_LABEL.get(w.spec.pde, w.spec.pde),
                   "network": f"{'FF' + str(2 * w.spec.ff_m) + ' -> ' if w.spec.ff_m else ''}"
                              f"{len(w.spec.widths)}x{w.spec.widths[0]} tanh -> {w.spec.d_out}"
                              f"{' RWF' if w.spec.rwf else ''}",
                   "n_res": batch.n_res, "n_ic": batch.n_ic, "n_bc": batch.n_bc, "points_per_step": n_pts,
                   "jet_columns": ncols, "parallelism": f"replicas x{ws_n}",
                   "workspace_gb": round(ws_bytes / 1e9, 2), "chunk_points": chunk_points,
                   "launch": "one CUDA graph per step" if graph else "eager launches",
                   "phase_timing": "CUDA events per launch group in an eager pass of the same K steps",
                   "bf16_weight_split": ("value rows" if value_split else "all rows") if precision == "bf16" else None,
                   "layer_engines": "".join("ctf"[x] for x in engines) + " (c CUDA cores, t tensor cores, "
                                    "f tensor cores with fused adjoint + weight gradient)",
                   "l2": f"working set {ws_bytes / 1e9:.2f} GB per step > 129 MB L2 (no flush needed)"},
        "gpu_launches": int(sum(v[1] for v in prof.values() if v[1] > 0)),
        "phases_ms_per_step": {k: round(v[0] / steps, 4) for k, v in prof.items()},
        "roofline": roof,
        "roofline_other": roof_alt,
        "jet_gemms": jet_gemm_rate(flops, prof, steps, peaks, precision),
        "clocks": clk,
        "device_status": status,
    }
    if per_step is not None:
        rec["ms_per_step_single"] = {"p10": round(float(np.percentile(per_step, 10)), 4),
                                     "p50": round(float(np.percentile(per_step, 50)), 4),
                                     "p90": round(float(np.percentile(per_step, 90)), 4),
                                     "how": "one event pair around each of K further steps (this rank)"}
    if e2e:
        rec["e2e"] = {"value": round(whole_job_rate(n_pts, ws_n, e2e_ms_max), 1), "unit": UNIT,
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms_max, 4),
                      "copies": "H2D: the step's collocation coordinates and targets from pinned host memory; "
                                "D2H: the 8 FP64 loss terms.  The P-entry gradient stays on the device, where "
                                "the optimizer (pinn_adam_step / L-BFGS) consumes it."}
    if terms_ms is not None:
        rec["loss_balance_step"] = {
            "ms_per_step": round(terms_ms, 4), "value": round(n_pts / (terms_ms / 1e3), 1), "unit": UNIT,
            "what": "one forward + three reverse sweeps (unweighted PDE/IC/BC gradients) + device weight update"}
    return rec, ctx


PDE_LABEL = {0: "burgers_1d", 1: "ns_steady_2d", 2: "maxwell_te_2d", 3: "advection_1d", 4: "allen_cahn_1d"}

# The other configurations, measured after the headline workload in the default run
# (rank 0 of a single-GPU run): (label, workload, precision, steps, warm-up,
# oracle-sample interior points, torch baseline steps or 0).
SUITE = [
    ("c4", "ns_cavity_8x512", "bf16", 8, 3, 1024, 2),
    ("c2", "maxwell_te_5x512", "bf16", 10, 3, 2048, 3),
    ("c0", "burgers1d_4x64", "fp32", 20, 5, 4096, 3),
    ("c1_tf32", "ns_cavity_6x256", "tf32", 10, 3, 2048, 0),
]


def run_suite(local):
    """Every other configuration at its full size: each sub-record has its own timed
    region, clocks, phase times, roofline and error against the oracle on a sample."""
    import gc
    import torch
    out = {}
    for label, name, precision, steps, warmup, n_err, torch_steps in SUITE:
        t0 = time.perf_counter()
        try:
            rec, ctx = measure(name, precision, None, steps, warmup, 1, 0, local, e2e=(label == "c4"),
                               spread=False)
            rec["library_error_vs_oracle"] = library_error(ctx["w"], ctx["params"], ctx["B"], ctx["batch"],
                                                           ctx["net"], n_err)
            if torch_steps:
                try:
                    tr = torch_autograd_rate(ctx["w"], ctx["params"], ctx["B"], ctx["batch"], steps=torch_steps,
                                             warmup=1)
                    tr["speedup"] = round(rec["value"] / tr["value"], 2)
                    rec["torch_autograd"] = tr
                except Exception as e:   # reported, not hidden
                    rec["torch_autograd"] = {"error": repr(e)[:300]}
            del ctx
        except Exception as e:           # reported, not hidden
            rec = {"error": repr(e)[:500], "workload": name, "dtype": precision}
        rec["wall_s"] = round(time.perf_counter() - t0, 1)
        out[label] = rec
        gc.collect()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    t0 = time.perf_counter()
    try:
        fam = run_family(10, 3, 1, 0, local)
    except Exception as e:
        fam = {"error": repr(e)[:500], "workload": "burgers_family_64"}
    fam["wall_s"] = round(time.perf_counter() - t0, 1)
    out["c3"] = fam
    return out


def run_ours(args, ws_n, rank, local):
    rec, ctx = measure(args.workload, args.precision, args.value_split, args.steps, args.warmup, ws_n, rank, local,
                       graph=args.graph, chunk_points=args.chunk_points, n_res=args.n_res, terms=args.terms)
    if rank != 0:
        return None
    w, params, B, batch, net = ctx["w"], ctx["params"], ctx["B"], ctx["batch"], ctx["net"]
    if not args.no_torch and ws_n == 1:
        try:
            tr = torch_autograd_rate(w, params, B, batch)
            tr["speedup"] = round(rec["value"] / tr["value"], 2)
            rec["torch_autograd"] = tr
        except Exception as e:   # reported, not hidden
            rec["torch_autograd"] = {"error": repr(e)[:300]}
        try:
            tr = torch_autograd_rate(w, params, B, batch, tf32=True)
            tr["dtype"] = "f32 storage, tf32 matmuls"
            tr["speedup"] = round(rec["value"] / tr["value"], 2)
            rec["torch_autograd_tf32"] = tr
        except Exception as e:
            rec["torch_autograd_tf32"] = {"error": repr(e)[:300]}
    if not args.no_cpu and ws_n == 1:
        rec["cpu_baseline"] = oracle_sample_rate(w, params, B, batch, net=net)
        rec["cpu_baseline"]["one_core"] = oracle_one_core_rate(w.name)
        rec["cpu_baseline"]["host"] = host_description()
    return rec


def jet_gemm_rate(flops, prof, steps, peaks, precision):
    """All jet GEMMs of the step together (forward, adjoint, weight gradient):
    algorithmic FLOPs over their summed device time, against the burst and the
    sustained peak of the precision's engine."""
    ms = sum(prof[k][0] for k in ("fwd_gemm", "adj_gemm", "dw_gemm", "adjdw_gemm")) / steps
    if ms <= 0:
        return None
    tf = sum(flops.values()) / (ms / 1e3) / 1e12
    p_burst, p_sus, _, src = tensor_peaks(peaks, precision)
    return {"tflops": round(tf, 1), "ms_per_step": round(ms, 4), "frac_of_burst": round(tf / p_burst, 4),
            "frac_of_sustained": round(tf / p_sus, 4), "peak_source": src}


def _traffic(kernel, workload):
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(f"{workload}:{kernel}")
    if not e or e.get("src_sha") != src_sha(e.get("src_files")):
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
        out = run_family(args.steps, args.warmup, ws_n, rank, local, args.precision or "bf16")
    else:
        out = run_ours(args, ws_n, rank, local)
    if out is not None and args.suite and ws_n == 1 and args.workload == DEFAULT_WORKLOAD:
        out["other_configs"] = run_suite(local)
    if out is not None:
        print(json.dumps(out), flush=True)
    if ws_n > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
