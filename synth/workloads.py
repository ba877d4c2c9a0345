"""Deterministic synthetic PINN workloads.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; the 64-bit finaliser constants of
Vigna's public-domain reference), turned into uniforms by the top 53 bits and into
normals by the Box-Muller transform.  Everything here is input generation: point
coordinates, boundary/initial target values, Xavier-normal / RWF initial
parameters and the frozen Fourier-feature matrix.  The method's own arithmetic
lives elsewhere.

Workloads (sizes as stated for the paper's benchmark problems, seeds
params=1000+k, interior points=2000+k, initial/boundary points=3000+k,
Fourier matrix=4000+k for workload index k):

  k=0 burgers1d_4x64      viscous Burgers u_t+u u_x-nu u_xx (Sec. 4.3 form with
                          viscosity), 2 -> 4x64 tanh -> 1, plain weights
  k=1 ns_cavity_6x256     steady lid-driven cavity (Sec. 4.4, Re=100), Fourier
                          features m=128 sigma=1 (Eq. 14), RWF (Eq. 15), 6x256 -> 3
  k=2 maxwell_te_5x512    2-D TE Maxwell (Sec. 4.8 equations), Gaussian pulse,
                          PEC walls, 5x512 tanh with RWF -> 3
  k=3 burgers_family_64   64 independent Burgers nets of uneven width/depth
  k=4 ns_cavity_8x512     cavity at scale: m=256 sigma=2, 8x512, 1M points
"""
from __future__ import annotations

import copy
import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

PDE_BURGERS = 0
PDE_NS = 1
PDE_MAXWELL = 2
PDE_ADVECTION = 3
PDE_ALLEN_CAHN = 4
PDE_NAMES = {PDE_BURGERS: "burgers_1d", PDE_NS: "ns_steady_2d", PDE_MAXWELL: "maxwell_te_2d",
             PDE_ADVECTION: "advection_1d", PDE_ALLEN_CAHN: "allen_cahn_1d"}

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class SplitMix64:
    """Counter form of SplitMix64: output i (1-based) is mix(seed + i*gamma)."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.count = 0

    def next_u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.count + 1, self.count + n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = self.seed + idx * _GAMMA
        self.count += n
        return _mix64(z)

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1): top 53 bits times 2^-53."""
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        """n standard normals, Box-Muller (cosine branch), two uniforms each."""
        u = self.uniform(2 * n)
        u1 = 1.0 - u[0::2]          # (0, 1]
        u2 = u[1::2]
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


@dataclass
class NetSpec:
    pde: int
    d_in: int
    d_out: int
    widths: List[int]
    ff_m: int = 0
    ff_sigma: float = 0.0
    rwf: bool = False
    rwf_mu: float = 1.0
    rwf_sigma: float = 0.1
    activation: str = "tanh"    # or "sine": sin(omega0 z) in every hidden layer
    omega0: float = 1.0


@dataclass
class Problem:
    nu: float
    lambda_pde: float = 1.0
    lambda_ic: float = 1.0
    lambda_bc: float = 1.0


@dataclass
class Batch:
    """Collocation sets, SoA float32: coordinates [d_in][n], targets [d_out][n]."""
    x_res: np.ndarray
    x_ic: np.ndarray
    g_ic: np.ndarray
    ic_mask: int
    x_bc: np.ndarray
    g_bc: np.ndarray
    bc_mask: int

    @property
    def n_res(self):
        return self.x_res.shape[1]

    @property
    def n_ic(self):
        return self.x_ic.shape[1]

    @property
    def n_bc(self):
        return self.x_bc.shape[1]

    def subset(self, n_res: int, n_ic: Optional[int] = None, n_bc: Optional[int] = None) -> "Batch":
        n_ic = self.n_ic if n_ic is None else n_ic
        n_bc = self.n_bc if n_bc is None else n_bc
        return Batch(self.x_res[:, :n_res].copy(), self.x_ic[:, :n_ic].copy(), self.g_ic[:, :n_ic].copy(),
                     self.ic_mask, self.x_bc[:, :n_bc].copy(), self.g_bc[:, :n_bc].copy(), self.bc_mask)


@dataclass
class Workload:
    name: str
    index: int
    spec: NetSpec
    problem: Problem
    n_res: int
    n_ic: int
    n_bc: int
    precision: str
    note: str = ""
    members: list = field(default_factory=list)   # for the many-network family
    value_split: bool = False   # BF16: split the weights on the value rows only (library option)


def layer_dims(spec: NetSpec):
    """(fan_in, fan_out) of every weight layer l = 1..L+1."""
    first_in = 2 * spec.ff_m if spec.ff_m else spec.d_in
    dims = []
    prev = first_in
    for w in spec.widths:
        dims.append((prev, w))
        prev = w
    dims.append((prev, spec.d_out))
    return dims


def param_count(spec: NetSpec) -> int:
    """Packed layout per layer: V[out*in] (row-major) | s[out] if RWF | b[out]."""
    n = 0
    for fi, fo in layer_dims(spec):
        n += fo * fi + (fo if spec.rwf else 0) + fo
    return n


def init_params(spec: NetSpec, seed: int, random_bias: float = 0.0) -> np.ndarray:
    """Xavier-normal V (std sqrt(2/(fan_in+fan_out))), s ~ N(mu, sigma) for RWF,
    b = 0 (or N(0, random_bias^2) for parity variants that exercise the bias)."""
    rng = SplitMix64(seed)
    out = []
    for fi, fo in layer_dims(spec):
        std = math.sqrt(2.0 / (fi + fo))
        out.append(rng.normal(fo * fi) * std)
        if spec.rwf:
            out.append(spec.rwf_mu + spec.rwf_sigma * rng.normal(fo))
        if random_bias:
            out.append(random_bias * rng.normal(fo))
        else:
            out.append(np.zeros(fo))
    return np.concatenate(out).astype(np.float32)


def ff_matrix(spec: NetSpec, seed: int) -> Optional[np.ndarray]:
    """Frozen Fourier-feature matrix B [d_in][m], entries N(0, sigma^2)."""
    if not spec.ff_m:
        return None
    rng = SplitMix64(seed)
    return (spec.ff_sigma * rng.normal(spec.d_in * spec.ff_m)).reshape(spec.d_in, spec.ff_m).astype(np.float32)


def _r_sequence(n: int, d: int, offset: np.ndarray) -> np.ndarray:
    """Additive-recurrence low-discrepancy points in [0,1)^d: frac(s + i*alpha),
    alpha_k = phi^-k with phi the positive root of x^(d+1) = x + 1."""
    phi = 2.0
    for _ in range(60):
        phi = phi - (phi ** (d + 1) - phi - 1.0) / ((d + 1) * phi ** d - 1.0)
    alpha = np.array([phi ** -(k + 1) for k in range(d)])
    i = np.arange(1, n + 1, dtype=np.float64)[:, None]
    return np.mod(offset[None, :] + i * alpha[None, :], 1.0).T


def make_batch(pde: int, n_res: int, n_ic: int, n_bc: int, seed_res: int, seed_bd: int,
               low_discrepancy: bool = False, maxwell_sigma: float = 0.05, wave_speed: float = 10.0) -> Batch:
    r = SplitMix64(seed_res)
    q = SplitMix64(seed_bd)
    f32 = np.float32
    if pde == PDE_BURGERS:
        # x in [-1,1], t in [0,1]; IC u(x,0) = -sin(pi x); BC u(+-1,t) = 0.
        x = -1.0 + 2.0 * r.uniform(n_res)
        t = r.uniform(n_res)
        x_res = np.stack([x, t])
        xi = -1.0 + 2.0 * q.uniform(n_ic)
        x_ic = np.stack([xi, np.zeros(n_ic)])
        g_ic = (-np.sin(np.pi * xi))[None, :]
        half = n_bc // 2
        xb = np.concatenate([-np.ones(half), np.ones(n_bc - half)])
        tb = q.uniform(n_bc)
        x_bc = np.stack([xb, tb])
        g_bc = np.zeros((1, n_bc))
        return Batch(x_res.astype(f32), x_ic.astype(f32), g_ic.astype(f32), 1,
                     x_bc.astype(f32), g_bc.astype(f32), 1)
    if pde == PDE_ADVECTION:
        # x in [0, 2 pi], t in [0, 1]; IC u(x,0) = sin x (Sec. 4.1).  The periodic walls
        # are given as Dirichlet targets of the exact solution u = sin(x - c t), with the
        # wave speed c passed as `wave_speed`.
        x = 2.0 * np.pi * r.uniform(n_res)
        t = r.uniform(n_res)
        xi = 2.0 * np.pi * q.uniform(n_ic)
        half = n_bc // 2
        xb = np.concatenate([np.zeros(half), 2.0 * np.pi * np.ones(n_bc - half)])
        tb = q.uniform(n_bc)
        return Batch(np.stack([x, t]).astype(f32), np.stack([xi, np.zeros(n_ic)]).astype(f32),
                     np.sin(xi)[None, :].astype(f32), 1, np.stack([xb, tb]).astype(f32),
                     np.sin(xb - wave_speed * tb)[None, :].astype(f32), 1)
    if pde == PDE_ALLEN_CAHN:
        # x in [-1, 1], t in [0, 1]; IC u(x,0) = x^2 cos(pi x) (Sec. 4.2).  The periodic
        # walls are given as the Dirichlet value the initial state has there, u = -1.
        x = -1.0 + 2.0 * r.uniform(n_res)
        t = r.uniform(n_res)
        xi = -1.0 + 2.0 * q.uniform(n_ic)
        half = n_bc // 2
        xb = np.concatenate([-np.ones(half), np.ones(n_bc - half)])
        tb = q.uniform(n_bc)
        return Batch(np.stack([x, t]).astype(f32), np.stack([xi, np.zeros(n_ic)]).astype(f32),
                     (xi ** 2 * np.cos(np.pi * xi))[None, :].astype(f32), 1, np.stack([xb, tb]).astype(f32),
                     -np.ones((1, n_bc), dtype=f32), 1)
    if pde == PDE_NS:
        # (x,y) in [0,1]^2; walls bottom, top (lid u=1), left, right; u,v constrained.
        x_res = np.stack([r.uniform(n_res), r.uniform(n_res)])
        per = n_bc // 4
        counts = [per, per, per, n_bc - 3 * per]
        xs, ys, us = [], [], []
        for wall, c in enumerate(counts):
            s = q.uniform(c)
            if wall == 0:
                xs.append(s); ys.append(np.zeros(c)); us.append(np.zeros(c))
            elif wall == 1:
                xs.append(s); ys.append(np.ones(c)); us.append(np.ones(c))
            elif wall == 2:
                xs.append(np.zeros(c)); ys.append(s); us.append(np.zeros(c))
            else:
                xs.append(np.ones(c)); ys.append(s); us.append(np.zeros(c))
        x_bc = np.stack([np.concatenate(xs), np.concatenate(ys)])
        g_bc = np.stack([np.concatenate(us), np.zeros(n_bc), np.zeros(n_bc)])
        x_ic = np.zeros((2, n_ic)); g_ic = np.zeros((3, n_ic))
        return Batch(x_res.astype(f32), x_ic.astype(f32), g_ic.astype(f32), 0,
                     x_bc.astype(f32), g_bc.astype(f32), 0b011)
    if pde == PDE_MAXWELL:
        # (x,y,t) in [0,1]^3; IC Ez Gaussian pulse, Hx=Hy=0; PEC walls Ez=0.
        if low_discrepancy:
            x_res = _r_sequence(n_res, 3, r.uniform(3))
        else:
            x_res = np.stack([r.uniform(n_res), r.uniform(n_res), r.uniform(n_res)])
        xi, yi = q.uniform(n_ic), q.uniform(n_ic)
        x_ic = np.stack([xi, yi, np.zeros(n_ic)])
        ez0 = np.exp(-((xi - 0.5) ** 2 + (yi - 0.5) ** 2) / (2.0 * maxwell_sigma ** 2))
        g_ic = np.stack([ez0, np.zeros(n_ic), np.zeros(n_ic)])
        per = n_bc // 4
        counts = [per, per, per, n_bc - 3 * per]
        xs, ys = [], []
        for wall, c in enumerate(counts):
            s = q.uniform(c)
            if wall == 0:
                xs.append(np.zeros(c)); ys.append(s)
            elif wall == 1:
                xs.append(np.ones(c)); ys.append(s)
            elif wall == 2:
                xs.append(s); ys.append(np.zeros(c))
            else:
                xs.append(s); ys.append(np.ones(c))
        x_bc = np.stack([np.concatenate(xs), np.concatenate(ys), q.uniform(n_bc)])
        g_bc = np.zeros((3, n_bc))
        return Batch(x_res.astype(f32), x_ic.astype(f32), g_ic.astype(f32), 0b111,
                     x_bc.astype(f32), g_bc.astype(f32), 0b001)
    raise ValueError(f"unknown pde {pde}")


def family_specs(n_nets: int = 64, seed: int = 5003):
    """The many-network Burgers family: per net a width from {32,64,128,256}, a
    hidden depth in 3..6, nu log-uniform in [1e-3, 1e-1] and an interior count
    log-uniform in [1024, 65536] rounded to a multiple of 32."""
    rng = SplitMix64(seed)
    u = rng.uniform(4 * n_nets).reshape(n_nets, 4)
    members = []
    for j in range(n_nets):
        width = (32, 64, 128, 256)[min(3, int(u[j, 0] * 4))]
        depth = 3 + min(3, int(u[j, 1] * 4))
        nu = 10.0 ** (-3.0 + 2.0 * u[j, 2])
        n_res = int(round(2.0 ** (10.0 + 6.0 * u[j, 3]) / 32.0)) * 32
        n_res = max(1024, min(65536, n_res))
        members.append(dict(spec=NetSpec(PDE_BURGERS, 2, 1, [width] * depth), nu=nu,
                            n_res=n_res, n_ic=256, n_bc=256,
                            seed_params=100000 + j, seed_res=200000 + j, seed_bd=300000 + j))
    return members


WORKLOADS = {
    "burgers1d_4x64": Workload(
        "burgers1d_4x64", 0, NetSpec(PDE_BURGERS, 2, 1, [64] * 4),
        Problem(nu=0.01 / math.pi), 4096, 256, 256, "fp32",
        "viscous Burgers, 4096 interior + 256 initial + 256 boundary points"),
    "ns_cavity_6x256": Workload(
        "ns_cavity_6x256", 1, NetSpec(PDE_NS, 2, 3, [256] * 6, ff_m=128, ff_sigma=1.0, rwf=True),
        Problem(nu=1.0 / 100.0), 65536, 0, 4096, "bf16",
        "steady cavity Re=100, 65,536 interior + 4x1024 wall points", value_split=True),
    "maxwell_te_5x512": Workload(
        "maxwell_te_5x512", 2, NetSpec(PDE_MAXWELL, 3, 3, [512] * 5, rwf=True),
        Problem(nu=0.0), 262144, 16384, 16384, "bf16",
        "TE Maxwell, 262,144 low-discrepancy interior + 16,384 initial + 16,384 PEC points"),
    "burgers_family_64": Workload(
        "burgers_family_64", 3, NetSpec(PDE_BURGERS, 2, 1, [64] * 3),
        Problem(nu=0.01), 0, 256, 256, "bf16",
        "64 independent Burgers nets, uneven width/depth/point count"),
    "advection1d_4x128": Workload(
        "advection1d_4x128", 5, NetSpec(PDE_ADVECTION, 2, 1, [128] * 4, ff_m=64, ff_sigma=1.0),
        Problem(nu=10.0), 16384, 512, 512, "bf16",
        "linear advection c=10 on [0, 2 pi] x [0, 1], Fourier features; 16,384 interior + 512 initial + 512 boundary"),
    "allen_cahn1d_4x128": Workload(
        "allen_cahn1d_4x128", 6, NetSpec(PDE_ALLEN_CAHN, 2, 1, [128] * 4),
        Problem(nu=1e-4), 16384, 512, 512, "bf16",
        "Allen-Cahn eps=1e-4 on [-1, 1] x [0, 1]; 16,384 interior + 512 initial + 512 boundary"),
    "ns_cavity_8x512": Workload(
        "ns_cavity_8x512", 4, NetSpec(PDE_NS, 2, 3, [512] * 8, ff_m=256, ff_sigma=2.0, rwf=True),
        Problem(nu=1.0 / 100.0), 1048576, 0, 16384, "bf16",
        "cavity at scale, 1,048,576 interior + 4x4096 wall points", value_split=True),
}


def make_workload(name: str, n_res: Optional[int] = None, n_ic: Optional[int] = None,
                  n_bc: Optional[int] = None, random_bias: float = 0.0):
    """Returns (workload, params float32 [P], B float32 [d][m] or None, Batch)."""
    w = copy.deepcopy(WORKLOADS[name])
    k = w.index
    if name == "burgers_family_64":
        w = replace(w, members=family_specs())
        return w, None, None, None
    n_res = w.n_res if n_res is None else n_res
    n_ic = w.n_ic if n_ic is None else n_ic
    n_bc = w.n_bc if n_bc is None else n_bc
    params = init_params(w.spec, 1000 + k, random_bias)
    B = ff_matrix(w.spec, 4000 + k)
    batch = make_batch(w.spec.pde, n_res, n_ic, n_bc, 2000 + k, 3000 + k,
                       low_discrepancy=(w.spec.pde == PDE_MAXWELL), wave_speed=w.problem.nu)
    return w, params, B, batch


def make_family(n_nets: int = 64, max_res: Optional[int] = None, random_bias: float = 0.0):
    """The many-network Burgers family as a list of (spec, params, batch, problem);
    `max_res` caps the interior points per network (for small test cases)."""
    out = []
    for m in family_specs(n_nets):
        n_res = m["n_res"] if max_res is None else min(m["n_res"], max_res)
        params = init_params(m["spec"], m["seed_params"], random_bias)
        batch = make_batch(PDE_BURGERS, n_res, m["n_ic"], m["n_bc"], m["seed_res"], m["seed_bd"])
        out.append((m["spec"], params, batch, Problem(nu=m["nu"])))
    return out
