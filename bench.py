"""Benchmark of the FC-Gram hot path on one GB300 (or N independent replicas).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Workloads (seeded synthetic fields, no dataset):
  * fc_deriv_z: batch of 3 fields 512 x 512 x 513 (d = 5, C = 25), first and
    second z-derivatives, float32 (headline) and float64.
Inputs (1.6 GB in float32) are larger than the 129 MB L2, so no flush is
needed between timed iterations.  Kernel time is measured with CUDA events on
the launching stream; the end-to-end figure goes through the public Python
API with pinned host buffers, host->device copy of the input and
device->host copy of both derivatives inside the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("RK-stage grid-points/s and fc_deriv_z HBM GB/s (FP32 batched vs FP64 plain); p50/p99")
DERIV_CONFIG = {"workload": "fc_deriv_z 3x512x512x513 d=5 C=25, d/dz and d2/dz2",
                "l2": "inputs 1.6 GB (f32) > 129 MB L2, no flush needed"}


def _measured_traffic(key):
    """DRAM bytes per launch from profiles/traffic.txt, if the kernel sources are
    unchanged since the capture; else None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        k, nbytes, srcs = line.split()[:3]
        if k != key:
            continue
        for item in srcs.split(","):
            fname, h = item.split(":")
            src = os.path.join(ROOT, "paper_2002_01392_gb300", "csrc", fname)
            if not os.path.exists(src) or not hashlib.sha1(open(src, "rb").read()).hexdigest().startswith(h):
                return None
        return float(nbytes)
    return None


def _deriv_alu_roofline(r, peak_tflops, peak_kind, L=1080, Nz=513, C=25, d=5):
    """fc_deriv_z against the arithmetic pipe: algorithmic flops per line pair
    (two real z-lines as one complex line) = three length-L FFTs at
    5 L log2 L, two spectrum products (6 flops per complex multiply), the
    continuation of both lines (2 C d multiply-adds each) and the output
    scaling, over the CUDA-event time; peak = the fused multiply-add rate of the
    arm's precision measured on this GPU (fc_alu_probe, 2 flops per lane
    operation)."""
    pair = 3 * 5 * L * np.log2(L) + 2 * 6 * L + 2 * 2 * C * d * 2 + 2 * 2 * Nz
    pairs = r["points"] / Nz / 2
    achieved = pair * pairs / r["seconds_per_call_mean"] / 1e12
    return {"bound": "alu", "achieved": float(achieved), "peak": float(peak_tflops), "unit": "TFLOP/s",
            "frac": float(achieved / peak_tflops), "flops_per_line_pair": float(pair), "peak_kind": peak_kind}


def measure_alu_peaks(api, torch, iters=4096, reps=5):
    """Arithmetic-pipe ceilings measured on this GPU with the library's probe
    kernel (fc_alu_probe: independent chains of one instruction kind on every
    SM, full occupancy), best of ``reps`` CUDA-event-timed launches after one
    warm-up each.  Per kind: lane operations per second (a packed two-wide
    instruction counts two) and, for the fused multiply-adds, flop/s
    (2 per lane operation)."""
    sink = torch.empty(256, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    out = {}
    for kind in ("ffma", "fadd", "ffma2", "fadd2", "dfma"):
        it = iters if kind != "dfma" else max(64, iters // 32)
        api.alu_probe(kind, it, sink)
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ops = api.alu_probe(kind, it, sink)
            e1.record(stream)
            e1.synchronize()
            t = e0.elapsed_time(e1) * 1e-3
            best = t if best is None else min(best, t)
        rate = ops / best
        out[kind] = {"lane_ops_per_s": rate, "tflops": (2 * rate if kind in ("ffma", "ffma2", "dfma") else rate) / 1e12,
                     "ms": best * 1e3}
    out["how"] = ("fc_alu_probe: 8 x SMs blocks x 256 threads, 8 independent chains per thread, "
                  "best of %d launches (CUDA events)" % reps)
    return out


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._thr = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._thr = threading.Thread(target=self._run, daemon=True)
        self._thr.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._thr.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if len(s) > 3 + i and s[3 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def _barrier_sync(torch):
    """Barrier over the ranks (when several) and device synchronisation: the
    bracket on both sides of every timed region."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


def _max_over_ranks(torch, x: float) -> float:
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(torch, points_per_rank: float, seconds: float) -> float:
    """Whole-job throughput of independent replicas (one per rank, no data
    exchange): the points of all ranks over the slowest rank's time."""
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    return points_per_rank * world / _max_over_ranks(torch, seconds)


DERIV_SHAPE = (3, 512, 512, 513)


def deriv_workload(dtype_np, B=None, Nx=None, Ny=None, Nz=None):
    B = B or DERIV_SHAPE[0]
    Nx = Nx or DERIV_SHAPE[1]
    Ny = Ny or DERIV_SHAPE[2]
    Nz = Nz or DERIV_SHAPE[3]
    import synth
    fields = [synth.SeparableField(Nx, Ny, Nz, seed_offset=b) for b in range(B)]
    return fields, (B, Nz, Ny, Nx)


def bench_deriv(api, torch, dtype_np, steps, warmup, with_e2e=True):
    """Time fc_deriv_z on the 3 x 512^2 x 513 batch; returns a dict."""
    fields, shape = deriv_workload(dtype_np)
    tdt = torch.float32 if dtype_np == np.float32 else torch.float64
    dev = torch.device("cuda", torch.cuda.current_device())
    f = torch.empty(shape, dtype=tdt, device=dev)
    for b, sf in enumerate(fields):
        f[b] = torch.from_numpy(sf.field(0).astype(dtype_np)).to(dev)
    d1, d2 = torch.empty_like(f), torch.empty_like(f)
    plan = api.Plan(5, 25, shape[1])
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        api.fc_deriv_z(plan, f, d1, d2)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    _barrier_sync(torch)
    t_all0.record(stream)
    for i in range(steps):
        ev[i][0].record(stream)
        api.fc_deriv_z(plan, f, d1, d2)
        ev[i][1].record(stream)
    t_all1.record(stream)
    _barrier_sync(torch)
    times = np.array([a.elapsed_time(b) for a, b in ev]) * 1e-3
    total = t_all0.elapsed_time(t_all1) * 1e-3
    pts = int(np.prod(shape))
    es = np.dtype(dtype_np).itemsize
    alg_bytes = 3 * es * pts
    # latency distribution: 200 more timed calls after 20 warm-ups (the timed
    # K calls above give the headline value)
    for _ in range(20):
        api.fc_deriv_z(plan, f, d1, d2)
    dist = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(200)]
    for a0, a1 in dist:
        a0.record(stream)
        api.fc_deriv_z(plan, f, d1, d2)
        a1.record(stream)
    torch.cuda.synchronize()
    lat = np.array([a.elapsed_time(b) for a, b in dist])
    res = {
        "points": pts, "seconds_total": total, "seconds_per_call_mean": float(times.mean()),
        "p50_ms": float(np.percentile(lat, 50)),
        "p99_ms": float(np.percentile(lat, 99)), "latency_reps": 200, "grid_points_per_s": pts * steps / total,
        "alg_bytes_per_call": alg_bytes, "alg_GBps": alg_bytes * steps / total / 1e9, "launches": steps,
    }
    # 64 sampled lines of the input and both outputs: the CPU-baseline leg
    # compares them with the FP64 oracle (reported beside the number)
    g = np.random.default_rng(1)
    B, Nz, Ny, Nx = shape
    bs, ys, xs = g.integers(0, B, 64), g.integers(0, Ny, 64), g.integers(0, Nx, 64)
    res["_samples"] = tuple(t[bs, :, ys, xs].double().cpu().numpy().T for t in (f, d1, d2))
    def e2e():
        # end to end through the host-array entry point (fc_deriv_z_host): the
        # library moves page-locked host arrays through the GPU in slabs, with
        # the copies in both directions overlapping the kernels; host clock
        hf = f.cpu().pin_memory()
        h1 = torch.empty(shape, dtype=tdt).pin_memory()
        h2 = torch.empty(shape, dtype=tdt).pin_memory()
        n_e2e = max(2, steps)
        api.fc_deriv_z_host(plan, hf, h1, h2)          # staging buffers allocated once
        _barrier_sync(torch)
        t0 = time.perf_counter()
        calls = []
        for _ in range(n_e2e):
            tc = time.perf_counter()
            api.fc_deriv_z_host(plan, hf, h1, h2)      # synchronous: returns with the outputs in host memory
            calls.append(time.perf_counter() - tc)
        _barrier_sync(torch)
        te = time.perf_counter() - t0
        same = bool(torch.equal(h1[:, ::16, ::16], d1[:, ::16, ::16].cpu()) and
                    torch.equal(h2[:, ::16, ::16], d2[:, ::16, ::16].cpu()))
        return {"value": replica_value(torch, pts * n_e2e, te), "unit": "grid-points/s",
                "h2d_bytes_per_step": es * pts, "d2h_bytes_per_step": 2 * es * pts,
                "api": "fc_deriv_z_host (host arrays, page-locked)", "bitwise_equal_device_path": same,
                "calls": n_e2e, "ms_per_call_p50": float(np.median(calls) * 1e3),
                "ms_per_call_max": float(max(calls) * 1e3),
                "link_floor_ms": 2 * es * pts / 193.5e9 * 1e3,
                "link_floor_note": "device-to-host bytes / 193.5 GB/s, the pinned copy rate measured on this "
                                   "pool's GB300 hosts (the larger of the two directions)",
                "clock_sampling": "off during this measurement (nvidia-smi queries stall host copies)"}

    def finish():
        nonlocal f, d1, d2
        out = e2e() if with_e2e else None
        del f, d1, d2
        torch.cuda.empty_cache()
        return out

    if with_e2e == "defer":
        # the caller runs the host-array measurement later (outside the clock
        # sampling, whose nvidia-smi queries were measured to stall host copies)
        res["_e2e"] = finish
        return res
    e = finish()
    if e is not None:
        res["e2e"] = e
    return res


class CufftDerivFP64:
    """The plain comparison path: FC-Gram z-derivatives in float64 through
    cuFFT (torch.fft) and separate elementwise / einsum kernels, one field
    after another.  Continuation by the plan's own M_r (Sec. 3), real DFT of
    length N' along z, multiplication by i kz (Nyquist zeroed) and -kz^2,
    inverse DFT, first Nz points."""

    def __init__(self, api, torch, Nz, Lz=1.0, d=5, C=25):
        self.torch = torch
        plan = api.Plan(d, C, Nz)
        Mr = torch.from_numpy(plan.matrix()).cuda()                 # C x d
        self.Mr, self.Ml = Mr, torch.flip(Mr, dims=(0, 1))           # left matrix: row / column reversal
        self.d, self.C, self.Nz, self.Np = d, C, Nz, Nz + C
        dz = Lz / (Nz - 1)
        k = torch.fft.rfftfreq(self.Np, d=dz / (2 * np.pi), device="cuda", dtype=torch.float64)
        k1 = k.clone()
        if self.Np % 2 == 0:
            k1[-1] = 0.0
        self.ik = (1j * k1).to(torch.complex128).view(-1, 1, 1)
        self.mk2 = (-(k * k)).to(torch.complex128).view(-1, 1, 1)

    def __call__(self, f, d1, d2):
        torch, d, Nz, Np = self.torch, self.d, self.Nz, self.Np
        for b in range(f.shape[0]):
            x = f[b]
            cont = torch.einsum("cd,dyx->cyx", self.Mr, x[Nz - d:]) + torch.einsum("cd,dyx->cyx", self.Ml, x[:d])
            X = torch.fft.rfft(torch.cat([x, cont], dim=0), dim=0)
            d1[b] = torch.fft.irfft(X * self.ik, n=Np, dim=0)[:Nz]
            d2[b] = torch.fft.irfft(X * self.mk2, n=Np, dim=0)[:Nz]


class PlainCufftNS:
    """The plain comparison path of the Navier-Stokes / Boussinesq RK step: one
    instance in float64 through cuFFT (torch.fft) and separate torch kernels,
    the method's steps in the paper's order (Sec. 3 continuation, Sec. 4.2
    transforms and products, Sec. 4.3 filter, Sec. 4.4 stage update, wall
    injection, inhomogeneous + analytic homogeneous pressure, projection).
    State: the continued spectral field [nf][N'][Ny][Kx] complex128.  The FC
    tables are the library's (fc_plan_matrix), the correctly rounded doubles
    of the continuation matrix; nothing here is shared with the CUDA path."""

    def __init__(self, api, torch, Nx, Ny, Nz, nu, kappa=0.0, gamma=0.0, forcing_x=0.0, nfields=3,
                 rk_order=3, Lx=2 * np.pi, Ly=2 * np.pi, Lz=1.0, d=5, C=25,
                 filter_beta=16 * np.log(10.0), filter_2p=100.0, device="cuda"):
        self.t = torch
        self.Nx, self.Ny, self.Nz, self.nf, self.o = Nx, Ny, Nz, nfields, rk_order
        self.d, self.Np, self.Kx, self.Lz = d, Nz + C, Nx // 2 + 1, Lz
        self.nu, self.kappa, self.gamma, self.F = nu, kappa, gamma, forcing_x
        dev, f64, c128 = device, torch.float64, torch.complex128
        Mr = torch.from_numpy(api.Plan(d, C, Nz).matrix()).to(dev, c128)
        self.Mr, self.Ml = Mr, torch.flip(Mr, dims=(0, 1))          # left matrix: row / column reversal
        dz = Lz / (Nz - 1)
        kx = 2 * np.pi * np.arange(self.Kx) / Lx
        ky = 2 * np.pi * np.fft.fftfreq(Ny, d=1.0 / Ny) / Ly
        kz = 2 * np.pi * np.fft.fftfreq(self.Np, d=dz)
        odd = lambda k, N, i: np.where(np.arange(k.size) == i, 0.0, k) if N % 2 == 0 else k
        kxo, kyo, kzo = odd(kx, Nx, Nx // 2), odd(ky, Ny, Ny // 2), odd(kz, self.Np, self.Np // 2)
        T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev, f64)
        self.KX, self.KY, self.KZ = T(kxo)[None, None, :], T(kyo)[None, :, None], T(kzo)[:, None, None]
        self.K2 = T(kz)[:, None, None] ** 2 + T(ky)[None, :, None] ** 2 + T(kx)[None, None, :] ** 2
        nx, ny, nz = np.arange(self.Kx), np.fft.fftfreq(Ny, d=1.0 / Ny), np.fft.fftfreq(self.Np, d=1.0 / self.Np)
        fz = np.exp(-filter_beta * (np.abs(nz) / (self.Np / 2)) ** filter_2p)
        self.filt = T(fz[:, None, None] * (3 * np.abs(ny) <= Ny)[None, :, None] * (3 * nx <= Nx)[None, None, :])
        self.kxo1, self.kyo1 = T(kxo)[None, :], T(kyo)[:, None]
        self.z = T(np.arange(Nz) * dz)[:, None, None]

    # transforms between the three spaces
    def xy_f(self, ph):
        return self.t.fft.fft(self.t.fft.rfft(ph, dim=-1), dim=-2)

    def xy_i(self, m):
        return self.t.fft.irfft(self.t.fft.ifft(m, dim=-2), n=self.Nx, dim=-1)

    def z_f(self, m):
        t, d = self.t, self.d
        cont = t.einsum("cd,...dyx->...cyx", self.Mr, m[..., -d:, :, :]) + \
            t.einsum("cd,...dyx->...cyx", self.Ml, m[..., :d, :, :])
        return t.fft.fft(t.cat([m, cont], dim=-3), dim=-3)

    def z_i(self, s):
        return self.t.fft.ifft(s, dim=-3)[..., :self.Nz, :, :]

    def to_spectral(self, ph):
        return self.z_f(self.xy_f(ph))

    def to_physical(self, s):
        return self.xy_i(self.z_i(s))

    def nonlinear_hat(self, st):
        t = self.t
        val = self.to_physical(st)
        grads = [t.stack([self.xy_i(1j * self.KX * self.z_i(c)), self.xy_i(1j * self.KY * self.z_i(c)),
                          self.to_physical(1j * self.KZ * c)]) for c in st]
        u = val[:3]
        N = t.stack([-(u[0] * g[0] + u[1] * g[1] + u[2] * g[2]) for g in grads])
        N[0] += self.F
        if self.nf == 4:
            N[2] += self.gamma * val[3]
            N[3] += self.gamma * val[2]
        return self.to_spectral(N) * self.filt

    def project(self, vs, dtj):
        t = self.t
        kk = self.KX ** 2 + self.KY ** 2 + self.KZ ** 2
        div = self.KX * vs[0] + self.KY * vs[1] + self.KZ * vs[2]
        s = t.where(kk > 0, div / t.where(kk > 0, kk, t.ones_like(kk)), t.zeros_like(div))
        gI = t.stack([self.KX * s, self.KY * s, self.KZ * s])
        wz = self.z_i(vs[2] - gI[2])
        b, tt = wz[0], wz[-1]
        gam = t.sqrt(self.kxo1 ** 2 + self.kyo1 ** 2)
        flat = gam == 0
        g1 = t.where(flat, t.ones_like(gam), gam)
        E = t.exp(-g1 * self.Lz)
        den = g1 * (1 - E * E)
        A = t.where(flat, t.zeros_like(b), (tt - b * E) / den)
        B = t.where(flat, t.zeros_like(b), -(b - tt * E) / den)
        D = t.where(flat, 0.5 * (b + tt), t.zeros_like(b))
        ep, em = t.exp(gam * (self.z - self.Lz)), t.exp(-gam * self.z)
        Phi = A * ep + B * em
        dPhi = gam * (A * ep - B * em) + D
        gHm = t.stack([1j * self.kxo1 * Phi, 1j * self.kyo1 * Phi, dPhi])
        v = vs - gI - self.z_f(gHm)
        gIw = self.z_i(gI[:2])
        gp = t.stack([t.stack([gIw[0, w] + gHm[0, w], gIw[1, w] + gHm[1, w]]) for w in (0, -1)]) / dtj
        return v, gp

    def step(self, st, gp, dt):
        t = self.t
        difs = [self.nu, self.nu, self.nu, self.kappa][:self.nf]
        vj = st
        for j in range(1, self.o + 1):
            dtj = dt / (self.o + 1 - j)
            Nh = self.nonlinear_hat(vj)
            vstar = t.stack([st[c] + dtj * (Nh[c] - difs[c] * self.K2 * vj[c]) for c in range(self.nf)])
            m = self.z_i(vstar)
            for w in (0, -1):
                m[0, w] = dtj * gp[0 if w == 0 else 1, 0]
                m[1, w] = dtj * gp[0 if w == 0 else 1, 1]
                if self.nf == 4:
                    m[3, w] = 0.0
            vsc = self.z_f(m)
            vnew = vsc.clone()
            vnew[:3], gp = self.project(vsc[:3], dtj)
            vj = vnew
        return vj, gp


def bench_cufft64(api, torch, steps, warmup):
    """Time the plain float64 cuFFT path on the 3 x 512^2 x 513 batch."""
    fields, shape = deriv_workload(np.float64)
    f = torch.empty(shape, dtype=torch.float64, device="cuda")
    for b, sf in enumerate(fields):
        f[b] = torch.from_numpy(sf.field(0)).cuda()
    d1, d2 = torch.empty_like(f), torch.empty_like(f)
    run = CufftDerivFP64(api, torch, shape[1])
    for _ in range(warmup):
        run(f, d1, d2)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        ev[i][0].record(stream)
        run(f, d1, d2)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    times = np.array([a.elapsed_time(b) for a, b in ev]) * 1e-3
    pts = int(np.prod(shape))
    res = {"points": pts, "p50_ms": float(np.percentile(times, 50) * 1e3),
           "p99_ms": float(np.percentile(times, 99) * 1e3), "grid_points_per_s": pts / float(times.mean()),
           "what": "torch.fft (cuFFT) float64 + separate einsum / elementwise kernels, one field at a time"}
    # agreement with the library's float64 kernel on the same input (both are the FC derivative)
    plan = api.Plan(5, 25, shape[1])
    e1, e2 = torch.empty_like(f), torch.empty_like(f)
    api.fc_deriv_z(plan, f, e1, e2)
    res["rel_l2_diff_d1_vs_library_fp64"] = float((e1 - d1).norm() / e1.norm())
    res["rel_l2_diff_d2_vs_library_fp64"] = float((e2 - d2).norm() / e2.norm())
    del f, d1, d2, e1, e2
    torch.cuda.empty_cache()
    return res


def band_limited_fields(Nx, Nz, seed, torch=None, kmax=2):
    """Four fields sum_{|kx|,|ky| <= kmax} A(z) cos(kx x + ky y) + B(z) sin(...)
    on an Nx x Nx grid (x = 2 pi i / Nx), A, B seeded polynomials times
    z(1 - z) / (1 + k^2); on the device (float32) when torch is given, else a
    float64 numpy array."""
    g = np.random.default_rng(seed)
    z = np.linspace(0.0, 1.0, Nz)
    modes = [(kx, ky) for kx in range(0, kmax + 1) for ky in range(-kmax, kmax + 1) if kx > 0 or ky >= 0]
    coef = g.uniform(-1, 1, size=(4, len(modes), 2, 3))
    x = 2 * np.pi * np.arange(Nx) / Nx
    out = []
    for f in range(4):
        acc = None
        for m, (kx, ky) in enumerate(modes):
            ph = kx * x[None, :] + ky * x[:, None]
            for part, fn in ((0, np.cos), (1, np.sin)):
                if kx == 0 and ky == 0 and part == 1:
                    continue
                c = coef[f, m, part]
                prof = 0.1 * z * (1 - z) * (1 + c[0] + c[1] * z + c[2] * z * z) / (1 + kx * kx + ky * ky)
                if torch is None:
                    term = prof[:, None, None] * fn(ph)[None]
                else:
                    term = (torch.from_numpy(prof).to("cuda", torch.float32)[:, None, None]
                            * torch.from_numpy(fn(ph)).to("cuda", torch.float32)[None])
                acc = term if acc is None else acc + term
        out.append(acc)
    return np.stack(out) if torch is None else torch.stack(out)


def rk_accuracy(res):
    """Relative L2 error per field of the band-limited full-size RK3 step of
    bench_rk against the oracle's 64^2 step (the CPU leg)."""
    smp = res.pop("_err_sample", None) if res else None
    if not smp:
        return
    from oracle import ns
    Nz, kw = smp["Nz"], smp["kw"]
    P = ns.Params(64, 64, Nz, nfields=4, **kw)
    fc_ = band_limited_fields(64, Nz, smp["seed"])
    st, _ = ns.rk_step(ns.to_spectral(fc_, P), np.zeros((2, 2, 64, P.Kx), complex), P, smp["dt"])
    ref = np.stack([ns.to_physical(c, P) for c in st])
    res["rel_l2_err_vs_oracle_per_field"] = [float(np.linalg.norm(smp["out"][f] - ref[f]) / np.linalg.norm(ref[f]))
                                             for f in range(4)]
    res["error_sample"] = ("one RK3 step of fields band-limited to |kx|,|ky| <= 2 at full size, every "
                           "Nx/64-th point against the oracle's 64^2 step (exact restriction)")


RK_SHAPE = (1024, 1024, 513)


def bench_rk(api, torch, steps, warmup, with_e2e=True, shape=None, tune=True):
    """Boussinesq Rayleigh-Benard RK3 step (4 fields, FP32 transforms) on
    1024 x 1024 x 513, Ra = 1e7, Pr = 1 (nu = kappa = sqrt(Pr/Ra) = 3.162e-4,
    gamma = 1, Lz = 1).  Returns RK-stage grid-points/s = Nx Ny Nz o / t_step."""
    import synth
    Nx, Ny, Nz = shape or RK_SHAPE
    kw = dict(nu=3.162e-4, kappa=3.162e-4, gamma=1.0)
    p = api.ns_params(Nx=Nx, Ny=Ny, Nz=Nz, nfields=4, prec="f32", rk_order=3, **kw)
    ws_bytes = api.ns_workspace_bytes(p)
    sim = api.Sim(p)
    tiles = sim.tune(1 if tune else 0)     # autotuned lines per CTA (ns_tune), or the defaults
    host = synth.boussinesq_fields(Nx, Ny, Nz, dtype=np.float32)
    f = torch.from_numpy(host).cuda()
    sim.set_fields(f)
    dt = 1e-3
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        sim.step(dt)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for i in range(steps):
        ev[i][0].record(stream)
        sim.step(dt)
        ev[i][1].record(stream)
    a1.record(stream)
    torch.cuda.synchronize()
    times = np.array([x.elapsed_time(y) for x, y in ev]) * 1e-3
    total = a0.elapsed_time(a1) * 1e-3
    pts = Nx * Ny * Nz
    res = {"grid": [Nx, Ny, Nz], "fields": 4, "rk_order": 3, "points": pts,
           "seconds_per_step_mean": float(times.mean()), "p50_ms": float(np.percentile(times, 50) * 1e3),
           "p99_ms": float(np.percentile(times, 99) * 1e3),
           "rk_stage_grid_points_per_s": pts * 3 * steps / total, "workspace_GB": ws_bytes / 1e9,
           "launches_per_step": 3 * 7, "tiles_autotuned": tiles}
    # stage roofline of the fused-pass traffic model: 288 B per grid point per
    # stage for the 4-field Boussinesq step in float32 (72 B per field)
    hbm_peak, _ = _peaks()
    stage_s = float(times.mean()) / 3
    res["roofline_stage"] = {"bound": "hbm", "model_bytes_per_point": 288, "achieved": 288 * pts / stage_s / 1e9,
                             "peak": hbm_peak, "unit": "GB/s", "frac": 288 * pts / stage_s / 1e9 / hbm_peak}
    if tune and any(tiles):
        # what the autotuner buys: the same steps with the built-in default variants
        sim.tune(0)
        sim.step(dt)
        torch.cuda.synchronize()
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        for _ in range(steps):
            sim.step(dt)
        d1.record(stream)
        torch.cuda.synchronize()
        res["default_variants_ms_per_step"] = d0.elapsed_time(d1) / steps
        res["autotune_speedup"] = res["default_variants_ms_per_step"] / (total / steps * 1e3)
        sim.tune(1)                          # back to the tuned variants (cached)
    out = sim.get_fields()
    res["finite"] = bool(torch.isfinite(out).all().item())
    res["w_wall_rel"] = float(out[2, [0, -1]].abs().max().item() / max(out[:3].abs().max().item(), 1e-300))
    # error against the oracle, untimed: one step of fields band-limited to
    # |kx|, |ky| <= 2, whose exact result on every (Nx/64)-th point is the exact
    # result of the 64^2 grid the oracle can run (each stage's product at most
    # doubles the bandwidth, which stays inside the 2/3 rule of a 64^2 grid);
    # the comparison runs in the CPU leg (rk_accuracy)
    if Nx % 64 == 0 and Nx == Ny:
        fb = band_limited_fields(Nx, Nz, seed=77 + Nz, torch=torch)
        sim.set_fields(fb)
        del fb
        sim.step(dt)
        r = Nx // 64
        res["_err_sample"] = {"Nz": Nz, "dt": dt, "seed": 77 + Nz, "kw": kw,
                              "out": sim.get_fields()[:, :, ::r, ::r].double().cpu().numpy()}
    if with_e2e:
        hp = torch.from_numpy(host).pin_memory()
        ho = torch.empty_like(hp).pin_memory()
        n_e2e = 2
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n_e2e):
            f.copy_(hp, non_blocking=True)
            sim.set_fields(f)
            sim.step(dt)
            sim.get_fields(out)
            ho.copy_(out, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        te = e0.elapsed_time(e1) * 1e-3
        res["e2e"] = {"value": pts * 3 * n_e2e / te, "unit": "RK-stage grid-points/s",
                      "h2d_bytes_per_step": int(hp.numel() * 4), "d2h_bytes_per_step": int(ho.numel() * 4)}
        del hp, ho
    sim.close()
    del f, out, host
    torch.cuda.empty_cache()
    return res


def bench_ensemble(api, torch, steps=5, warmup=3, n=64):
    """Batched ensemble: n independent channel instances of uneven sizes
    (64^2 x 65, 96^2 x 97, 128^2 x 129, 192^2 x 129; nu log-uniform in
    [1e-3, 1e-2]), FP32 with the float64 mean-flow line, one RK3 step of all
    members = one CUDA graph launch.  Beside it, the same instances stepped
    one after another: FP32 through rk_step (no graph), FP64 through rk_step,
    and the plain path north of the library, FP64 through cuFFT (torch.fft)
    with separate torch kernels (PlainCufftNS).  For the error of each arm
    against the oracle, one instance per grid size is stepped once from its
    initial fields and returned (``_err_samples``; compared in the CPU leg)."""
    import synth
    specs = synth.ensemble_specs(n)
    pts = sum(s["Nx"] * s["Ny"] * s["Nz"] for s in specs)
    stream = torch.cuda.current_stream()
    dt = 2e-4

    def fields(sp):
        return synth.channel_velocity(sp["Nx"], sp["Ny"], sp["Nz"], nu=sp["nu"], seed_offset=sp["seed_offset"])

    def params(sp, prec):
        return api.ns_params(Nx=sp["Nx"], Ny=sp["Ny"], Nz=sp["Nz"], nu=sp["nu"], forcing_x=10 * sp["nu"], prec=prec)

    def make(prec):
        sims = []
        for sp in specs:
            sim = api.Sim(params(sp, prec))
            sim.set_fields(torch.from_numpy(fields(sp)).to("cuda", sim.dtype))
            sims.append(sim)
        return sims

    def timed(fn, k):
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for i in range(k):
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return np.array([a.elapsed_time(b) for a, b in ev]) * 1e-3

    def arm(t):
        return {"p50_ms": float(np.percentile(t, 50) * 1e3), "p99_ms": float(np.percentile(t, 99) * 1e3),
                "rk_stage_grid_points_per_s": pts * 3 / float(t.mean())}

    # one instance of each grid size, one step from the initial fields, per arm
    err_idx = []
    for g in synth.ENSEMBLE_GRIDS:
        for i, sp in enumerate(specs):
            if (sp["Nx"], sp["Ny"], sp["Nz"]) == tuple(g):
                err_idx.append(i)
                break
    samples = {"inputs": [(specs[i], fields(specs[i])) for i in err_idx], "dt": dt}
    for prec in ("f32", "f64"):
        outs = []
        for i in err_idx:
            sim = api.Sim(params(specs[i], prec))
            sim.set_fields(torch.from_numpy(fields(specs[i])).to("cuda", sim.dtype))
            sim.step(dt)
            outs.append(sim.get_fields().double().cpu().numpy())
            sim.close()
        samples[prec] = outs
    outs = []
    for i in err_idx:
        sp = specs[i]
        pl = PlainCufftNS(api, torch, sp["Nx"], sp["Ny"], sp["Nz"], nu=sp["nu"], forcing_x=10 * sp["nu"])
        st = pl.to_spectral(torch.from_numpy(fields(sp)).cuda())
        st, _ = pl.step(st, torch.zeros((2, 2, sp["Ny"], sp["Nx"] // 2 + 1), dtype=torch.complex128, device="cuda"), dt)
        outs.append(pl.to_physical(st).cpu().numpy())
    samples["cufft_f64"] = outs

    # FP32, one graph launch per step of all members: first with every member
    # on the built-in default variants (what the autotuner buys), then tuned
    sims = make("f32")
    batch = api.Batch(sims)
    for s_ in sims:
        s_.tune(0)
    for _ in range(warmup):
        batch.step(dt)
    tdef = timed(lambda: batch.step(dt), steps)
    batch.close()
    for s_ in sims:
        s_.tune(1)
    batch = api.Batch(sims)
    for _ in range(warmup):
        batch.step(dt)
    t = timed(lambda: batch.step(dt), steps)
    info = batch.info()
    # the variants the autotuner kept, per grid (cached per size: tune(1) only reads them back)
    variants = {}
    for sp, sim in zip(specs, sims):
        variants["%dx%dx%d" % (sp["Nx"], sp["Ny"], sp["Nz"])] = sim.tune(1)
    finite = all(bool(torch.isfinite(s.get_fields()).all().item()) for s in sims)
    batch.close()

    # FP32, the same tuned simulations stepped one after another (no graph)
    def seq32():
        for s_ in sims:
            s_.step(dt)
    seq32()
    t32 = timed(seq32, max(2, steps // 2))
    for s_ in sims:
        s_.close()

    # FP64 library kernels, one after another
    sims64 = make("f64")

    def seq64():
        for s_ in sims64:
            s_.step(dt)
    seq64()
    t64 = timed(seq64, max(2, steps // 2))
    for s_ in sims64:
        s_.close()
    torch.cuda.empty_cache()

    # FP64 cuFFT plain path, one instance after another
    plains, states = [], []
    for sp in specs:
        pl = PlainCufftNS(api, torch, sp["Nx"], sp["Ny"], sp["Nz"], nu=sp["nu"], forcing_x=10 * sp["nu"])
        plains.append(pl)
        states.append([pl.to_spectral(torch.from_numpy(fields(sp)).cuda()),
                       torch.zeros((2, 2, sp["Ny"], sp["Nx"] // 2 + 1), dtype=torch.complex128, device="cuda")])

    def seqcu():
        for pl, stg in zip(plains, states):
            stg[0], stg[1] = pl.step(stg[0], stg[1], dt)
    seqcu()
    tcu = timed(seqcu, 2)
    del plains, states
    torch.cuda.empty_cache()

    res = {"instances": n, "grids": [list(g) for g in synth.ENSEMBLE_GRIDS], "points": pts,
           **arm(t), "graph_nodes": info["graph_nodes"], "variants_autotuned": variants,
           "fp32_graph_default_variants": arm(tdef),
           "autotune_speedup": float(np.percentile(tdef, 50) / np.percentile(t, 50)),
           "graph_launches_per_step": 1, "finite": finite,
           "fp32_sequential": arm(t32), "fp64_library_sequential": arm(t64),
           "fp64_cufft_plain_sequential": dict(arm(tcu), what="PlainCufftNS: torch.fft (cuFFT) float64 + "
                                               "separate torch kernels, one instance after another")}
    res["speedup_vs_fp64_cufft_plain"] = res["rk_stage_grid_points_per_s"] / res["fp64_cufft_plain_sequential"]["rk_stage_grid_points_per_s"]
    res["speedup_vs_fp32_sequential"] = res["rk_stage_grid_points_per_s"] / res["fp32_sequential"]["rk_stage_grid_points_per_s"]
    res["_err_samples"] = samples
    return res


def ensemble_accuracy(res):
    """Relative L2 error, against the FP64 oracle, of one RK3 step of one
    instance per grid size for each ensemble arm (the CPU leg: the oracle runs
    only here).  The FP32 graph arm is bitwise the FP32 one-by-one arm (each
    member alone; tests/test_gpu_batch.py), so one figure covers both."""
    samples = res.pop("_err_samples", None)
    if not samples:
        return
    from oracle import ns
    errs = {"f32": [], "f64": [], "cufft_f64": []}
    for k, (sp, f) in enumerate(samples["inputs"]):
        P = ns.Params(sp["Nx"], sp["Ny"], sp["Nz"], nu=sp["nu"], forcing_x=10 * sp["nu"])
        st, _ = ns.rk_step(ns.to_spectral(f, P), np.zeros((2, 2, sp["Ny"], P.Kx), complex), P, samples["dt"])
        ref = np.stack([ns.to_physical(c, P) for c in st])
        for key in errs:
            errs[key].append(float(np.linalg.norm(samples[key][k] - ref) / np.linalg.norm(ref)))
    res["rel_l2_err_vs_oracle"] = {"fp32_graph_and_sequential": max(errs["f32"]), "fp64_library": max(errs["f64"]),
                                   "fp64_cufft_plain": max(errs["cufft_f64"]),
                                   "instances": ["%dx%dx%d" % (sp["Nx"], sp["Ny"], sp["Nz"]) for sp, _ in samples["inputs"]]}


def bench_serving(api, torch, rate=2000.0, duration=2.0, resident=48, slots=8):
    """Serving: Poisson arrivals (mean ``rate`` per second, ``duration``
    seconds) of fc_poisson_project and rk_step requests, 50/50, on ``resident``
    FP32 simulations drawn uniformly from 64^2 x 65, 128^2 x 129, 256^2 x 257,
    admitted by HBM footprint; requests overlap on ``slots`` CUDA streams."""
    import synth
    from paper_2002_01392_gb300 import serve
    grids = ((64, 64, 65), (128, 128, 129), (256, 256, 257))
    g = np.random.default_rng(2002013924)
    free, total = torch.cuda.mem_get_info()
    srv = serve.Server(int(0.5 * free), slots=slots)
    sims, shapes = [], []
    for i in range(resident):
        Nx, Ny, Nz = grids[int(g.integers(0, 3))]
        p = api.ns_params(Nx=Nx, Ny=Ny, Nz=Nz, nu=5e-3, forcing_x=5e-2, prec="f32")
        v = synth.channel_velocity(Nx, Ny, Nz, nu=5e-3, seed_offset=2000 + i)
        sid = srv.admit(p, torch.from_numpy(v.astype(np.float32)).cuda())
        if sid is not None:
            sims.append(sid)
            shapes.append((Nx, Ny, Nz))
    inputs = {sid: torch.from_numpy(synth.channel_velocity(*shapes[k], nu=5e-3, seed_offset=3000 + k)
                                    .astype(np.float32)).cuda() for k, sid in enumerate(sims)}
    reqs = serve.poisson_requests(rate, duration, sims, g, kinds=("project", "step"), dt=2e-4)
    for r in reqs:
        if r.kind == "project":
            r.inp = inputs[r.sim]
    stats = srv.run(reqs, max_wall_s=300.0)
    stats.update({"arrival_rate_per_s": rate, "duration_s": duration, "slots": slots,
                  "grids": [list(x) for x in grids], "mix": "50/50 fc_poisson_project / rk_step"})
    srv.close()
    # error sample (compared with the oracle in the CPU leg): per grid size, one
    # projection and one RK3 step of a simulation as served, from its fields
    smp = []
    for Nx, Ny, Nz in grids:
        p = api.ns_params(Nx=Nx, Ny=Ny, Nz=Nz, nu=5e-3, forcing_x=5e-2, prec="f32")
        v = synth.channel_velocity(Nx, Ny, Nz, nu=5e-3, seed_offset=2000).astype(np.float32)
        vs = synth.channel_velocity(Nx, Ny, Nz, nu=5e-3, seed_offset=3000).astype(np.float32)
        sim = api.Sim(p)
        sim.set_fields(torch.from_numpy(v).cuda())
        proj = sim.project(torch.from_numpy(vs).cuda(), 2e-4).double().cpu().numpy()
        sim.set_fields(torch.from_numpy(v).cuda())
        sim.step(2e-4)
        smp.append(((Nx, Ny, Nz), v, vs, proj, sim.get_fields().double().cpu().numpy()))
        sim.close()
    stats["_err_samples"] = smp
    torch.cuda.empty_cache()
    return stats


def serving_capacity(api, torch, grids, reps=10):
    """GPU time of one request of each kind alone (CUDA events, after warm-up)
    per grid size, and the request rate one GPU sustains for the served mix
    (50/50 projection / RK3 step, grids uniform) with one request at a time:
    1 / (mean request time).  Concurrent streams overlap small requests, so
    the served rate can exceed it somewhat; far above it is impossible."""
    import synth
    stream = torch.cuda.current_stream()
    per = {}
    for Nx, Ny, Nz in grids:
        sim = api.Sim(api.ns_params(Nx=Nx, Ny=Ny, Nz=Nz, nu=5e-3, forcing_x=5e-2, prec="f32"))
        sim.tune(1)
        v = torch.from_numpy(synth.channel_velocity(Nx, Ny, Nz, nu=5e-3).astype(np.float32)).cuda()
        sim.set_fields(v)
        out = {}
        for kind, fn in (("project", lambda: sim.project(v, 2e-4)), ("step", lambda: sim.step(2e-4))):
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            e1.synchronize()
            out[kind] = e0.elapsed_time(e1) / reps
        per["%dx%dx%d" % (Nx, Ny, Nz)] = out
        sim.close()
    mean_ms = float(np.mean([t for g in per.values() for t in g.values()]))
    return {"request_gpu_ms": per, "mean_request_gpu_ms": mean_ms, "sustainable_req_per_s_one_at_a_time": 1e3 / mean_ms}


def serving_accuracy(res):
    """Relative L2 error against the oracle of one projection and one RK3 step
    per grid size of the served simulations (the CPU leg)."""
    smp = res.pop("_err_samples", None) if res else None
    if not smp:
        return
    from oracle import ns
    errs = {}
    for (Nx, Ny, Nz), v, vs, proj, step in smp:
        P = ns.Params(Nx, Ny, Nz, nu=5e-3, forcing_x=5e-2)
        v64, vs64 = v.astype(np.float64), vs.astype(np.float64)
        ref_p, _ = ns.poisson_project(vs64, P, 2e-4)
        st, _ = ns.rk_step(ns.to_spectral(v64, P), np.zeros((2, 2, Ny, P.Kx), complex), P, 2e-4)
        ref_s = np.stack([ns.to_physical(c, P) for c in st])
        errs["%dx%dx%d" % (Nx, Ny, Nz)] = {
            "project": float(np.linalg.norm(proj - ref_p) / np.linalg.norm(ref_p)),
            "rk_step": float(np.linalg.norm(step - ref_s) / np.linalg.norm(ref_s))}
    res["rel_l2_err_vs_oracle"] = errs


class OracleDerivSample:
    """The FP64 oracle (numpy, one thread) on sampled z-lines of the
    3 x 512^2 x 513 fc_deriv_z batch: one call = both derivatives of
    ``lines`` lines."""

    def __init__(self, lines=4096, seed=3):
        import synth
        from oracle import fc, fc_tables
        self.fc = fc
        self.Mr = fc_tables.fc_matrix(5, 25, table_dir=os.path.join(ROOT, "tests", "golden"))
        sf = synth.SeparableField(512, 512, 513, seed_offset=0)
        self.Z = sf.z_profiles(0)
        self.X = sf.X.reshape(sf.X.shape[0], -1)
        self.g = np.random.default_rng(seed)
        self.lines = lines

    def __call__(self):
        idx = self.g.integers(0, self.X.shape[1], self.lines)
        f = self.Z.T @ self.X[:, idx]
        self.fc.fc_deriv_z(f, 1.0, self.Mr, 1, axis=0)
        self.fc.fc_deriv_z(f, 1.0, self.Mr, 2, axis=0)
        return self.lines * 513


def bench_noise(api, torch, reps=5, warmup=3, Nx=1024, Ny=1024, Nz=513):
    """App. A perturbation (fc_noise) on the 1024^2 x 513 Boussinesq grid,
    float32 output (float64 arithmetic): CUDA-event time per call and the
    float64 multiply-add rate of the synthesis (6 per point per kx index)."""
    import synth
    p = api.noise_params()
    cnt = api.noise_modes(p)
    draws = synth.noise_draws(cnt, 13)
    out = torch.empty((3, Nz, Ny, Nx), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        api.fc_noise(p, draws, out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        api.fc_noise(p, draws, out)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3 / reps
    nn = 2 * 5 + 1                       # kx indices -5..5 of the App. A annulus
    pts = Nx * Ny * Nz
    res = {"grid": [Nx, Ny, Nz], "modes": cnt, "ms_per_call": sec * 1e3, "grid_points_per_s": pts / sec,
           "dfma_per_point_synthesis": 6 * nn, "dfma_tflops_synthesis": 2 * 6 * nn * pts / sec / 1e12,
           "_err_sample": (draws, out[:, :, ::64, ::64].double().cpu().numpy(), Nz)}
    del out
    torch.cuda.empty_cache()
    return res


def noise_accuracy(res):
    """Largest error of every 64th x, y column against the oracle on the grid
    of exactly those points, after the one global scale (the CPU leg)."""
    smp = res.pop("_err_sample", None) if res else None
    if not smp:
        return
    from oracle import noise
    draws, sample, Nz = smp
    ref = noise.noise_field(16, 16, Nz, draws)
    c = float((sample * ref).sum() / (ref * ref).sum())
    res["max_abs_err_vs_oracle_sampled"] = float(np.abs(sample - c * ref).max())


def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _single_thread_numpy():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    try:
        import threadpoolctl
        threadpoolctl.threadpool_limits(1)
    except Exception:
        pass


def _oracle_deriv_worker(args):
    """One host core: the oracle on sampled z-lines for ``budget`` seconds
    (after one warm-up call); returns the grid points differentiated."""
    budget, seed, lines = args
    _single_thread_numpy()
    sys.path.insert(0, ROOT)
    run = OracleDerivSample(lines=lines, seed=seed)
    run()
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget:
        done += run()
    return done, time.perf_counter() - t0


def _oracle_rk_worker(args):
    """One host core: oracle RK3 Boussinesq steps of its own N^2 x Nz instance
    for ``budget`` seconds; returns the RK-stage grid points advanced."""
    budget, seed, N, Nz = args
    _single_thread_numpy()
    sys.path.insert(0, ROOT)
    import synth
    from oracle import ns
    P = ns.Params(N, N, Nz, nfields=4, nu=3.162e-4, kappa=3.162e-4, gamma=1.0)
    st = ns.to_spectral(synth.boussinesq_fields(N, N, Nz, seed_offset=seed), P)
    gp = np.zeros((2, 2, N, N // 2 + 1), complex)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget or steps == 0:
        st, gp = ns.rk_step(st, gp, P, 1e-3)
        steps += 1
    return N * N * Nz * 3 * steps, time.perf_counter() - t0


def _on_all_cores(worker, args_of_rank, cores):
    """Run ``worker`` on ``cores`` spawned processes (one per core, each
    single-threaded); returns (total units, wall seconds of the slowest)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(cores) as pool:
        # bounded: a worker that dies (e.g. out of host memory) must not hang the bench
        res = pool.map_async(worker, [args_of_rank(i) for i in range(cores)]).get(timeout=POOL_TIMEOUT_S)
    return sum(r[0] for r in res), max(r[1] for r in res)


POOL_TIMEOUT_S = 300.0


_REF = {}


def _ref_init():
    _single_thread_numpy()
    sys.path.insert(0, ROOT)
    _REF["run"] = OracleDerivSample(lines=1024, seed=7 + os.getpid())


def _ref_step(_):
    return _REF["run"]()


def cpu_baseline_deriv(budget_s=12.0):
    """The FP64 oracle, as it stands, on every host core: each core
    differentiates its own random z-lines of the 3 x 512^2 x 513 batch for
    ~budget_s seconds (the lines are independent, so the cores share no
    work)."""
    cores = host_cores()
    pts, wall = _on_all_cores(_oracle_deriv_worker, lambda i: (budget_s, 100 + i, 2048), cores)
    return {"value": pts / wall, "unit": "grid-points/s", "cores": cores, "kind": "oracle",
            "sample": f"{pts // 513} z-lines (x 513 points) of the 3x512x512x513 fc_deriv_z batch, "
                      f"FP64 numpy pocketfft, {cores} single-threaded processes, ~{budget_s:.0f} s each"}


def oracle_accuracy(res):
    """Relative L2 error of the sampled fc_deriv_z output lines of an arm
    against the FP64 oracle (the CPU-baseline leg: the oracle runs here only)."""
    samples = res.pop("_samples", None)
    if samples is None:
        return
    from oracle import fc, fc_tables
    Mr = fc_tables.fc_matrix(5, 25, table_dir=os.path.join(ROOT, "tests", "golden"))
    lines, o1, o2 = samples
    for order, o in ((1, o1), (2, o2)):
        ref = fc.fc_deriv_z(lines, 1.0, Mr, order, axis=0)
        res[f"rel_l2_err_d{order}_vs_oracle"] = float(np.linalg.norm(o - ref) / np.linalg.norm(ref))


def cpu_baseline_rk(budget_s=15.0, N=128, Nz=129):
    """The FP64 oracle RK3 Boussinesq step on every host core: each core
    advances its own N^2 x Nz instance (a bounded stand-in for the 1024^2 x 513
    step; the oracle's cost per point grows like log N)."""
    cores = host_cores()
    pts, wall = _on_all_cores(_oracle_rk_worker, lambda i: (budget_s, i, N, Nz), cores)
    return {"value": pts / wall, "unit": "RK-stage grid-points/s", "cores": cores, "kind": "oracle",
            "sample": f"RK3 steps of {cores} independent {N}x{N}x{Nz} Boussinesq oracle instances (4 fields, FP64; "
                      f"numpy pocketfft), one single-threaded process per core, ~{budget_s:.0f} s each"}


def main():
    global DERIV_SHAPE
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--rk-steps", type=int, default=5)
    ap.add_argument("--no-rk", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="profile cases: default tiles, no autotuning launches")
    ap.add_argument("--profile-case", default=None,
                    choices=["deriv32", "deriv64", "rk-small", "rk-mid", "rk-full", "rk-smooth", "noise"],
                    help="small single-kernel case for ncu (deriv: fc_deriv_z on 2x256x256x513; rk-*: one RK3 grid; noise: fc_noise on 256x256x513), no e2e / CPU leg")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank != 0:
            return
        # the oracle as it stands, on every host core: each step = both
        # z-derivatives of 1024 sampled z-lines of the 3 x 512^2 x 513 batch on
        # each core (one single-threaded spawned process per core)
        import multiprocessing as mp
        cores = host_cores()
        with mp.get_context("spawn").Pool(cores, initializer=_ref_init) as pool:
            pool.map_async(_ref_step, range(cores)).get(timeout=POOL_TIMEOUT_S)   # tables / fields built, first call
            for _ in range(args.warmup):
                pool.map_async(_ref_step, range(cores)).get(timeout=POOL_TIMEOUT_S)
            t0 = time.perf_counter()
            pts = sum(sum(pool.map_async(_ref_step, range(cores)).get(timeout=POOL_TIMEOUT_S))
                      for _ in range(args.steps))
            dt = time.perf_counter() - t0
        val = pts / dt
        cb = {"value": val, "unit": "grid-points/s", "cores": cores, "kind": "oracle",
              "sample": f"{args.steps} steps x {cores} cores x 1024 z-lines of the 3x512x512x513 fc_deriv_z "
                        f"batch, FP64 numpy, one single-threaded process per core"}
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": val, "unit": "grid-points/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": dict(DERIV_CONFIG, parallelism="host cores", arm="FP64 CPU oracle on sampled z-lines"),
                          "cpu_baseline": cb,
                          "e2e": {"value": val, "unit": "grid-points/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_01392_gb300 import api
    dev_index = torch.cuda.current_device()
    hbm_peak, peak_kind = _peaks()
    if args.profile_case == "noise":
        r = bench_noise(api, torch, reps=args.steps, warmup=args.warmup, Nx=256, Ny=256, Nz=513)
        r.pop("_err_sample", None)
        print(json.dumps({"profile_case": args.profile_case, **r}))
        return
    if args.profile_case and args.profile_case.startswith("rk"):
        shape = {"rk-small": (256, 256, 513), "rk-mid": (1024, 1024, 33), "rk-full": None,
                 "rk-smooth": (1024, 1024, 487)}[args.profile_case]
        r = bench_rk(api, torch, args.steps, args.warmup, with_e2e=False, shape=shape, tune=not args.no_tune)
        r.pop("_err_sample", None)
        print(json.dumps({"profile_case": args.profile_case, **r}))
        return
    if args.profile_case:
        DERIV_SHAPE = (2, 256, 256, 513)
        r = bench_deriv(api, torch, np.float32 if args.profile_case == "deriv32" else np.float64,
                        args.steps, args.warmup, with_e2e=False)
        r.pop("_samples", None)
        print(json.dumps({"profile_case": args.profile_case, **r}))
        return
    # the companions (RK step, ensemble, serving, float64 and smooth-N' arms) are
    # single-GPU context: with several replicas only the headline is timed
    extras = world == 1 and not args.no_rk
    with ClockSampler(dev_index) as clk:
        r32 = bench_deriv(api, torch, np.float32, args.steps, args.warmup, with_e2e="defer")
    r32["e2e"] = r32.pop("_e2e")()
    with ClockSampler(dev_index) as clk_rk:
        rk = bench_rk(api, torch, args.rk_steps, 3) if extras else None
    if rk:
        rk["clocks"] = clk_rk.summary()
    r64 = rc = rks = ens = srv = srv_low = rs = nz = None
    if world == 1:
        r64 = bench_deriv(api, torch, np.float64, max(3, args.steps // 4), 2, with_e2e=False)
        rc = bench_cufft64(api, torch, max(3, args.steps // 4), 2)
        # companion: the paper's kind of smooth N' (512 = 487 + 25) at the same horizontal size
        DERIV_SHAPE = (3, 512, 512, 487)
        rs = bench_deriv(api, torch, np.float32, args.steps, 2, with_e2e=False)
        DERIV_SHAPE = (3, 512, 512, 513)
    if extras:
        # companion: the paper's kind of smooth N' (512 = 487 + 25): direct length-N' z transforms
        rks = bench_rk(api, torch, args.rk_steps, 2, with_e2e=False, shape=(1024, 1024, 487))
        ens = bench_ensemble(api, torch)
        srv = bench_serving(api, torch)
        srv_low = bench_serving(api, torch, rate=300.0)
        srv["capacity"] = serving_capacity(api, torch, ((64, 64, 65), (128, 128, 129), (256, 256, 257)))
        nz = bench_noise(api, torch)
    alu = measure_alu_peaks(api, torch)
    if r64:
        r64["roofline_alu"] = _deriv_alu_roofline(r64, alu["dfma"]["tflops"], "measured DFMA rate (fc_alu_probe)")
    value = replica_value(torch, r32["points"] * args.steps, r32["seconds_total"])
    ms_per_step = _max_over_ranks(torch, r32["seconds_total"]) / args.steps * 1e3
    out = {
        "metric": METRIC, "value": value, "unit": "grid-points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(DERIV_CONFIG, parallelism="replicas" if world > 1 else "single",
                       arm="FP32 transforms, continuation in float-float (FP64-level)"),
        "p50_ms": r32["p50_ms"], "p99_ms": r32["p99_ms"],
        "fc_deriv_z": {"fp32": {k: v for k, v in r32.items() if k != "e2e"}, "fp64": r64,
                       "fp32_smooth_Np512_3x512x512x487": rs, "cufft_fp64_plain": rc,
                       "fp32_speedup_vs_cufft_fp64_plain": (r32["grid_points_per_s"] / rc["grid_points_per_s"]
                                                            if rc else None)},
        "rk_stage": rk,
        "rk_stage_smooth_Np512_1024x1024x487": rks,
        "ensemble_64_uneven_fp32_graph": ens,
        "serving_poisson_2000_per_s": srv,
        "serving_poisson_300_per_s": srv_low,
        "noise_app_a_1024x1024x513": nz,
        "roofline": {"bound": "hbm", "achieved": r32["alg_bytes_per_call"] / r32["seconds_per_call_mean"] / 1e9,
                     "peak": hbm_peak, "unit": "GB/s",
                     "frac": r32["alg_bytes_per_call"] / r32["seconds_per_call_mean"] / 1e9 / hbm_peak,
                     "traffic": _measured_traffic("fc_deriv_z_f32"), "peak_kind": peak_kind,
                     "kernel": "fc_deriv_z conv L=1080 FP32, paired lines, real-valued kernel spectra, registers j >= 16 known zero, rows j < 13 without bounds checks, whole tiles (phased_kernel<DerivPair<float,30,36,4,16,1,13,1>>)",
                     "algorithmic_bytes_per_point": 12, "traffic_source": "profiles/traffic.txt (ncu, small case scaled x6)"},
        "roofline_alu": _deriv_alu_roofline(r32, alu["ffma"]["tflops"], "measured FFMA rate (fc_alu_probe)"),
        "alu_peaks_measured": alu,
        "e2e": r32.get("e2e"),
        "gpu_launches": r32["launches"],
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu:
        # the CPU leg (oracle baselines and errors): a failure here is reported
        # in the line, never lost with it
        def leg(name, fn):
            try:
                fn()
            except Exception as e:                      # noqa: BLE001
                out.setdefault("cpu_leg_errors", {})[name] = f"{type(e).__name__}: {e}"[:300]

        def set_cpu():
            out["cpu_baseline"] = cpu_baseline_deriv()
        leg("cpu_baseline", set_cpu)
        if out.get("rk_stage"):
            def set_rk_cpu():
                out["rk_stage"]["cpu_baseline"] = cpu_baseline_rk()
            leg("rk_cpu_baseline", set_rk_cpu)
        for arm in (out["fc_deriv_z"]["fp32"], r64, rs):
            if arm:
                leg("oracle_accuracy", lambda arm=arm: oracle_accuracy(arm))
        if ens:
            leg("ensemble_accuracy", lambda: ensemble_accuracy(ens))
        leg("rk_accuracy", lambda: rk_accuracy(out.get("rk_stage")))
        leg("rk_smooth_accuracy", lambda: rk_accuracy(out.get("rk_stage_smooth_Np512_1024x1024x487")))
        leg("serving_accuracy", lambda: serving_accuracy(out.get("serving_poisson_2000_per_s")))
        leg("noise_accuracy", lambda: noise_accuracy(nz))
    if nz:
        nz.pop("_err_sample", None)
    for arm in (out["fc_deriv_z"]["fp32"], r64, rs):
        if arm:
            arm.pop("_samples", None)
    if ens:
        ens.pop("_err_samples", None)
    for arm in (out.get("rk_stage"), out.get("rk_stage_smooth_Np512_1024x1024x487")):
        if arm:
            arm.pop("_err_sample", None)
    for arm in (out.get("serving_poisson_2000_per_s"), out.get("serving_poisson_300_per_s")):
        if arm:
            arm.pop("_err_samples", None)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
