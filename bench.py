"""Benchmark: deconvolved Mpoints/s to relative residual 1e-6 on one GB300
(or N GPUs, one process each, weak scaling: every rank solves its own batch).

Workload (default): 16 seeded 2048^2 float32 fields with a k^-3 spectrum
(k_p = 10, exp(-(k/600)^2) cutoff), filtered with the Germano elliptic filter
at gamma = 0.01, deconvolved by BiCGSTAB to h <= 1e-6 with float64 dots and
scalars. One step = one solve of the batch (a single library call); the inputs
(256 MiB) are larger than L2, so no flush is needed between steps. The JSON
line also reports CG and Van Cittert on the same batch, the roofline of the
dominant pass kernel, the oracle timed on the host cores, and clocks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--method bicgstab]
    python bench.py --impl reference     # the CPU oracle, bounded samples
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = dict(name="scalar2d_2048_f32_x16", shape=(2048, 2048), batch=16, gamma=0.01, tol=1e-6,
                kp=10.0, kcut=600.0)
METRIC = "deconvolved Mpoints/s to 1e-6 rel. residual"
UNIT = "Mpoints/s"
VC_MAXIT = 2000


def _spectrum(k):
    from synth import fields
    return fields.spectrum_2d_kraichnan(k, kp=WORKLOAD["kp"], kcut=WORKLOAD["kcut"])


def _fields(seeds):
    from synth import fields
    n = WORKLOAD["shape"]
    out = np.empty((len(seeds),) + tuple(n), dtype=np.float32)
    for i, s in enumerate(seeds):
        out[i] = fields.random_scalar_field(n, s, _spectrum)
    return out


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _kernel_sha():
    h = hashlib.sha256()
    for f in ("fft.cuh", "passes.cuh", "spectral.cuh"):
        with open(os.path.join(ROOT, "paper_1707_09177_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clocks and throttle reasons."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            with open(self.path) as f:
                for line in f:
                    c = [x.strip() for x in line.split(",")]
                    if len(c) < 9:
                        continue
                    try:
                        sm.append(float(c[1]))
                        mx = max(mx, float(c[2]))
                    except ValueError:
                        continue
                    for n, v in zip(names, c[5:9]):
                        if v.lower() == "active":
                            reasons.add(n)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seeds(rank, batch):
    """Seeds of the fields rank `rank` solves: weak scaling, each rank its own
    `batch` fields, disjoint across ranks."""
    return list(range(rank * batch, rank * batch + batch))


def max_over_ranks(x, device):
    """The maximum of a per-rank float over all ranks (the job is as slow as
    its slowest rank); x itself when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mpoints(world, batch, points, seconds):
    """Mpoints/s of the whole job: every rank's fields over the max time."""
    return world * batch * points / seconds / 1e6


def _pass_bytes(kind, op, P, SP, B, method):
    """Algorithmic bytes one launch must move (each array read or written
    once), float32 fields (4 B) and complex64 spectra (8 B)."""
    v, s = 4 * P * B, 8 * SP * B
    if kind == "spec":                                 # spectral vectors read + written
        return {0: 1, 1: 3, 2: 4, 3: 1, 4: 4, 5: 3, 6: 5, 7: 4, 8: 2, 9: 6}[op] * s
    if kind in ("lfwd", "linv"):
        return 2 * s
    if kind == "sten":
        return 2 * v                                   # r in, z = M r out
    if kind == "filt":
        return 2 * s                                   # spectrum in, filtered spectrum out
    if kind == "xfwd":
        rw = {0: (1, 0), 1: (2, 1), 2: (3, 2), 3: (3, 1), 4: (2, 1)}[op]  # (vectors read, written)
        return (rw[0] + rw[1]) * v + s
    if kind == "xinv":
        rw = {0: (0, 1), 1: (1, 1), 2: (1, 0), 3: (1, 1), 4: (1, 1), 5: (2, 2), 6: (1, 1), 7: (4, 2)}[op]
        return s + (rw[0] + rw[1]) * v
    return 2 * s


def _traffic(kind, op, space):
    """DRAM bytes per launch of a pass kernel from profiles/traffic.json (an ncu
    capture), or None when absent or taken with other kernel sources."""
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(tp):
        return None
    with open(tp) as f:
        td = json.load(f)
    k = "%s:%s:%d" % (space, kind, op)
    if td.get("kernel_sha") == _kernel_sha() and k in td.get("bytes_per_launch", {}):
        return td["bytes_per_launch"][k]
    return None


def _traffic_conv():
    """DRAM bytes of one 32 -> 32 layer launch on the 512^3 x 3 velocity from
    profiles/traffic.json (a 256^3 x 1 ncu capture scaled by the grid points:
    the layer streams its input and output once), or None when absent or taken
    with another source of the tensor-core kernel."""
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(tp):
        return None
    with open(tp) as f:
        td = json.load(f)
    with open(os.path.join(ROOT, "paper_1707_09177_gb300", "csrc", "conv_tc.cu"), "rb") as fh:
        sha = hashlib.sha256(fh.read()).hexdigest()[:16]
    if td.get("conv_sha") == sha:
        return td.get("conv_bytes_per_launch_512cubed_x3")
    return None


def _oracle_solve_seconds(ub64, gamma, method, passes):
    """Wall time of one oracle solve with a fixed number of passes (includes
    the initial residual and the final true-residual check)."""
    import oracle
    t = time.perf_counter()
    oracle.solve(method, ub64, gamma, tol=0.0, maxit=passes)
    return time.perf_counter() - t


def _oracle_estimate(ub64, gamma, method, n_target, sample_passes):
    """Seconds of a full oracle solve of n_target passes, from a bounded
    sample: fixed cost (0 passes) plus n_target times the per-pass cost."""
    t0 = _oracle_solve_seconds(ub64, gamma, method, 0)
    tk = _oracle_solve_seconds(ub64, gamma, method, sample_passes)
    per = max(tk - t0, 1e-9) / sample_passes
    return t0 + n_target * per, per, t0


def _golden_count(method, seed):
    p = os.path.join(ROOT, "tests", "golden", "counts_2048.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    for r in d["runs"]:
        if r["method"] == method and r["precision"] == "f64" and r["seed"] == seed:
            return int(r["iterations"])
    return None


def _timed(fn):
    import torch
    fn()                                            # warm-up (plans, graphs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return r, time.perf_counter() - t0


def _extra_workloads(gad, dev, extras, line):
    """Other workloads of the method, one timed solve each after a warm-up,
    each recorded in line["workloads"] as soon as it is measured (a failure is
    recorded in line["errors"] and the next workload still runs): the 3D
    velocity (256^3 x 3 components, gamma = 0.1, BiCGSTAB per component to
    1e-6), the uneven batch (48 seeded sizes, 2D 256..4096 and 3D 64..384,
    gamma by grid size, BiCGSTAB to 1e-6 in one batched call, against the same
    fields solved one shape group at a time) and the 512^3 learned guess."""
    import torch
    out = line["workloads"]
    if "3d256" in extras:
        _guarded(line, "velocity3d_256_f32", lambda: _velocity_256(gad, out, extras))
        torch.cuda.empty_cache()
    if "uneven48" in extras:
        _guarded(line, "uneven48_f32", lambda: _uneven_48(gad, dev, out))
        torch.cuda.empty_cache()
    if "learned512" in extras:
        _guarded(line, "velocity3d_512_f32_learned",
                 lambda: out.__setitem__("velocity3d_512_f32_learned", _learned_512(gad, dev)))
        torch.cuda.empty_cache()


def _velocity_256(gad, out, extras):
    import torch
    from synth import fields
    n = 256
    v = fields.random_velocity_field((n, n, n), 0, fields.spectrum_3d_kolmogorov).astype(np.float32)
    u_true = torch.from_numpy(v).to(torch.device("cuda", torch.cuda.current_device()))
    ub = gad.filter(u_true, 0.1, ndim=3)
    del u_true
    _tune(gad, (n, n, n), 0.1, 3)
    r, t = _timed(lambda: gad.deconvolve(ub, 0.1, method="bicgstab", tol=1e-6, maxit=2000, ndim=3))
    its = [int(x) for x in r.iterations]
    rs, ts = _timed(lambda: gad.deconvolve(ub, 0.1, method="bicgstab", tol=1e-6, maxit=2000, ndim=3,
                                           space="spectral"))
    rp, tp = _timed(lambda: gad.deconvolve(ub, 0.1, method="pcg", tol=1e-6, maxit=2000, ndim=3))
    rq, tq = _timed(lambda: gad.deconvolve(ub, 0.1, method="pcg", tol=1e-6, maxit=2000, ndim=3,
                                           space="spectral"))
    out["velocity3d_256_f32"] = {"mpoints_s": 3 * n ** 3 / t / 1e6, "ms": t * 1e3, "iterations": its,
                                 "converged": bool(np.all(r.status == gad.AD_OK)), "launches": r.launches,
                                 "spectral": {"mpoints_s": 3 * n ** 3 / ts / 1e6, "ms": ts * 1e3,
                                              "iterations": [int(x) for x in rs.iterations],
                                              "converged": bool(np.all(rs.status == gad.AD_OK))},
                                 "pcg": {"mpoints_s": 3 * n ** 3 / tp / 1e6, "ms": tp * 1e3,
                                         "iterations": [int(x) for x in rp.iterations],
                                         "converged": bool(np.all(rp.status == gad.AD_OK))},
                                 "pcg_spectral": {"mpoints_s": 3 * n ** 3 / tq / 1e6, "ms": tq * 1e3,
                                                  "iterations": [int(x) for x in rq.iterations],
                                                  "converged": bool(np.all(rq.status == gad.AD_OK))}}
    if "closure" in extras:
        out["closure_256"] = _closure_stats(gad, ub, r.u, n)


def _uneven_48(gad, dev, out):
    # default tile widths here: tuned plans of different block sizes split the
    # work-list launches into more launch classes (measured slower), and the
    # graph branches gained nothing from them
    import torch
    from synth import fields
    shapes = fields.uneven_batch(0)
    ub, gammas = [], []
    for i, sh in enumerate(shapes):
        spec = _spectrum if len(sh) == 2 else fields.spectrum_3d_kolmogorov
        g = fields.gamma_for_grid(sh)
        ub.append(gad.filter(fields.random_scalar_field_torch(sh, 1000 + i, spec, device=dev), g, ndim=len(sh)))
        gammas.append(g)
    pts = float(sum(np.prod(sh) for sh in shapes))
    # one graph branch per shape group (the default) ...
    gad.set_batched_launch(False)
    res, t = _timed(lambda: gad.deconvolve_batched(ub, gammas, method="bicgstab", tol=1e-6, maxit=3000,
                                                   history=False))
    its = res[1]
    launches = gad.last_launch_count()
    # ... against one launch per pass stage over all shape groups (a work list)
    gad.set_batched_launch(True)
    try:
        resw, t_wl = _timed(lambda: gad.deconvolve_batched(ub, gammas, method="bicgstab", tol=1e-6, maxit=3000,
                                                           history=False))
        launches_wl = gad.last_launch_count()
    finally:
        gad.set_batched_launch(False)
    same = bool(all(np.array_equal(a.cpu().numpy(), b.cpu().numpy()) for a, b in zip(res[0], resw[0])))
    # the same fields, one shape group per call
    groups = {}
    for i, sh in enumerate(shapes):
        groups.setdefault(sh, []).append(i)

    def seq():
        for sh, idx in groups.items():
            stacked = torch.stack([ub[i] for i in idx])
            gad.deconvolve(stacked, gammas[idx[0]], method="bicgstab", tol=1e-6, maxit=3000, ndim=len(sh),
                           history=False)
    _, t_seq = _timed(seq)
    out["uneven48_f32"] = {"mpoints_s": pts / t / 1e6, "ms": t * 1e3, "points": pts, "fields": len(shapes),
                           "shape_groups": len(groups), "iterations_mean": float(np.mean(its)),
                           "converged": bool(np.all(res[2] == gad.AD_OK)), "launches": launches,
                           "launch": "one CUDA graph, one concurrent branch (with its own loop) per shape group",
                           "work_list": {"launch": "one launch per pass stage over all shape groups",
                                         "mpoints_s": pts / t_wl / 1e6, "ms": t_wl * 1e3,
                                         "launches": launches_wl, "bitwise_equal": same},
                           "one_call_per_group_mpoints_s": pts / t_seq / 1e6}


def _closure_stats(gad, ub, ustar, n):
    """The step after the solve, on the 256^3 x 3 velocity: the sub-filter
    stress tau_ij (6 pairs, one batched application of G), the energy
    spectrum of u*, its vorticity and the histogram of omega_x (1000 bins
    over +-6 sigma); each timed once after a warm-up."""
    import torch
    out = {}
    ub, ustar = ub.reshape(1, 3, n, n, n).contiguous(), ustar.reshape(1, 3, n, n, n).contiguous()
    tau, t = _timed(lambda: gad.closure(ub, ustar, 0.1, ncomp=3, ndim=3))
    out["stress"] = {"ms": t * 1e3, "pairs": 6, "mpoints_s": 6 * n ** 3 / t / 1e6}
    e, t = _timed(lambda: gad.spectrum(ustar, n, ncomp=3, ndim=3))
    out["spectrum"] = {"ms": t * 1e3, "shells": n, "energy": float(e.sum())}
    w, t = _timed(lambda: gad.curl(ustar, ndim=3))
    out["curl"] = {"ms": t * 1e3}
    wx = w[0, 0].contiguous()
    sd = float(torch.std(wx))
    h, t = _timed(lambda: gad.histogram(wx, -6 * sd, 6 * sd, 1000))
    out["histogram"] = {"ms": t * 1e3, "bins": 1000, "gb_s": wx.numel() * 4 / t / 1e9,
                        "outside": int(h[1] + h[2] + h[3])}
    del tau, w, wx
    torch.cuda.empty_cache()
    return out


def _learned_512(gad, dev, n=512, npairs=2000, n_train=64, epochs=8, batch=8, lr=1e-4):
    """Learned initial guess against plain BiCGSTAB on a 512^3 x 3 velocity
    (gamma = 0.01, tolerance 1e-6, the residual normalised by ||u_bar - G u_bar||
    for both starts). The network is trained first, on the GPU, on `npairs`
    pairs (u_true, G u_true) of 64^3 fields drawn with the 512^3 field's
    spectrum in grid units (wavenumbers scaled by 512/64: the network is local,
    so it sees the same neighbourhood statistics) and filtered with the same
    grid-unit filter (gamma = 0.01). Learned wall time = inference + solve."""
    import torch
    from synth import fields
    wl = fields.WORKLOADS["velocity3d_512_f32"]
    gamma, spec = wl["gamma"], wl["spectrum"]
    t_gen = time.perf_counter()
    v = fields.random_velocity_field_torch((n,) * 3, 0, spec, device=dev)
    ub = gad.filter(v, gamma, ndim=3)
    del v
    spec_t = lambda k: spec(np.asarray(k) * (n / n_train))
    ut = torch.empty((npairs,) + (n_train,) * 3, device=dev)
    for i in range(0, npairs, 3):
        m = min(3, npairs - i)
        ut[i:i + m] = fields.random_velocity_field_torch((n_train,) * 3, 10_000 + i, spec_t, device=dev)[:m]
    ubt = gad.filter(ut, gamma, ndim=3)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    w = gad.guess_init(seed=1, stencil=True)
    w_stencil = w.clone()
    gad.guess_train(w.clone(), ubt[:batch], ut[:batch], gamma, epochs=1, batch=batch, lr=lr, seed=0)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = gad.guess_train(w, ubt, ut, gamma, epochs=epochs, batch=batch, lr=lr, seed=3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del ut, ubt
    torch.cuda.empty_cache()

    def solve(u0=None, space="physical"):
        return gad.deconvolve(ub, gamma, method="bicgstab", tol=1e-6, maxit=4000, ndim=3, u0=u0, history=False,
                              space=space)

    def timed(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t

    _tune(gad, (n, n, n), gamma, 3)
    gad.deconvolve(ub, gamma, method="bicgstab", tol=1e-6, maxit=2, ndim=3, history=False)     # plans, graph
    gad.guess_infer(w, ub, gamma)
    plain, t_plain = timed(solve)
    u0, t_inf = timed(lambda: gad.guess_infer(w, ub, gamma))
    learned, t_solve = timed(lambda: solve(u0))
    u0s = gad.guess_infer(w_stencil, ub, gamma)
    stencil, t_stencil = timed(lambda: solve(u0s))
    gad.deconvolve(ub, gamma, method="bicgstab", tol=1e-6, maxit=2, ndim=3, history=False, space="spectral")
    sp_plain, t_sp_plain = timed(lambda: solve(space="spectral"))
    sp_learned, t_sp_solve = timed(lambda: solve(u0, space="spectral"))
    gad.deconvolve(ub, gamma, method="pcg", tol=1e-6, maxit=2, ndim=3, history=False)
    pcg, t_pcg = timed(lambda: gad.deconvolve(ub, gamma, method="pcg", tol=1e-6, maxit=4000, ndim=3,
                                              history=False))
    gad.deconvolve(ub, gamma, method="pcg", tol=1e-6, maxit=2, ndim=3, history=False, space="spectral")
    pcs, t_pcs = timed(lambda: gad.deconvolve(ub, gamma, method="pcg", tol=1e-6, maxit=4000, ndim=3,
                                              history=False, space="spectral"))
    diff = float(torch.linalg.vector_norm(learned.u - plain.u) / torch.linalg.vector_norm(plain.u))
    pts = 3.0 * n ** 3
    t_learned = t_inf + t_solve
    return {
        "shape": [n] * 3, "components": 3, "gamma": gamma, "tol": 1e-6,
        "plain": {"ms": t_plain * 1e3, "mpoints_s": pts / t_plain / 1e6,
                  "iterations": [int(x) for x in plain.iterations],
                  "converged": bool(np.all(plain.status == gad.AD_OK))},
        "learned": {"ms": t_learned * 1e3, "infer_ms": t_inf * 1e3, "solve_ms": t_solve * 1e3,
                    "mpoints_s": pts / t_learned / 1e6, "iterations": [int(x) for x in learned.iterations],
                    "converged": bool(np.all(learned.status == gad.AD_OK))},
        "stencil_start_untrained": {"solve_ms": t_stencil * 1e3,
                                    "iterations": [int(x) for x in stencil.iterations]},
        "spectral_space": {
            "plain": {"ms": t_sp_plain * 1e3, "iterations": [int(x) for x in sp_plain.iterations],
                      "converged": bool(np.all(sp_plain.status == gad.AD_OK))},
            "learned": {"ms": (t_inf + t_sp_solve) * 1e3, "solve_ms": t_sp_solve * 1e3,
                        "iterations": [int(x) for x in sp_learned.iterations],
                        "converged": bool(np.all(sp_learned.status == gad.AD_OK))},
            "wall_time_ratio_plain_over_learned": t_sp_plain / (t_inf + t_sp_solve)},
        "wall_time_ratio_plain_over_learned": t_plain / t_learned,
        "preconditioned_cg": {"ms": t_pcg * 1e3, "mpoints_s": pts / t_pcg / 1e6,
                              "iterations": [int(x) for x in pcg.iterations],
                              "converged": bool(np.all(pcg.status == gad.AD_OK)),
                              "spectral": {"ms": t_pcs * 1e3, "mpoints_s": pts / t_pcs / 1e6,
                                           "iterations": [int(x) for x in pcs.iterations],
                                           "converged": bool(np.all(pcs.status == gad.AD_OK))}},
        "rel_l2_learned_vs_plain_solution": diff,
        "train": {"pairs": npairs, "shape": [n_train] * 3, "epochs": epochs, "batch": batch, "lr": lr,
                  "seconds": t_train, "loss_per_epoch": [float(x) for x in hist],
                  "data_generation_s": t_gen, "init": "explicit-inverse stencil"},
    }


_TUNE = [True]


def _tune(gad, shape, gamma, batch, method="bicgstab"):
    """Tile widths of the plan for (shape, batch) picked by the library's
    autotuner (every admissible width of every pass timed with CUDA events,
    the fastest kept), for both iteration spaces; no-op with --no-tune."""
    if _TUNE[0]:
        for space in ("physical", "spectral"):
            gad.autotune(shape, gamma, batch, method=method, space=space)


def _workload_config(args, ws):
    """The config keys that name the workload (the same in both arms)."""
    return {"workload": WORKLOAD["name"], "grid": "%dx%d" % WORKLOAD["shape"], "batch_per_gpu": args.batch,
            "gamma": WORKLOAD["gamma"], "tol": WORKLOAD["tol"], "method": args.method, "space": args.space,
            "parallelism": "replicas" if ws > 1 else "1 gpu"}


def run_reference(args):
    """The CPU oracle timed on the host cores: each step is one BiCGSTAB pass
    over one 2048^2 field; the metric extrapolates the per-pass time to the
    oracle's own iteration count for that field (tests/golden/counts_2048.json)."""
    ws, rank, _ = _dist()
    if ws > 1 and rank != 0:
        return
    os.environ["OMP_NUM_THREADS"] = "1"
    import oracle
    ub = oracle.filter_field(_fields([0])[0].astype(np.float64), WORKLOAD["gamma"])
    ub = ub.astype(np.float32).astype(np.float64)
    g = WORKLOAD["gamma"]
    for _ in range(args.warmup):
        _oracle_solve_seconds(ub, g, args.method, 1)
    t0 = _oracle_solve_seconds(ub, g, args.method, 0)
    ts = [_oracle_solve_seconds(ub, g, args.method, 1) for _ in range(args.steps)]
    per = max(float(np.mean(ts)) - t0, 1e-9)
    n_iter = _golden_count(args.method, 0) or 160
    P = WORKLOAD["shape"][0] * WORKLOAD["shape"][1]
    t_solve = t0 + n_iter * per
    value = P / t_solve / 1e6
    sample = ("oracle %s (float64 NumPy, 1 thread), one 2048^2 field (seed 0): %d timed one-pass solves after %d "
              "warm-up, minus the fixed cost of a zero-pass solve; Mpoints/s = P / (fixed + %d passes x %.2f s), "
              "%d = the oracle's own pass count to 1e-6 for that field"
              % (args.method, args.steps, args.warmup, n_iter, per, n_iter))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(ts)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _workload_config(args, ws),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu_model": _host_cpu()[0], "host_cores": _host_cpu()[1]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--method", default="bicgstab", choices=["bicgstab", "cg", "vancittert", "sd", "pcg"])
    ap.add_argument("--no-extras", action="store_true", help="skip the comparison methods and CPU baseline")
    ap.add_argument("--host-loop", action="store_true",
                    help="drive the iteration loop from the host instead of a graph while node (same kernels; "
                         "profilers cannot see kernel nodes of graphs with conditional nodes)")
    ap.add_argument("--batch", type=int, default=WORKLOAD["batch"], help="fields per GPU")
    ap.add_argument("--space", default="physical", choices=["physical", "spectral"],
                    help="iteration space of the timed solve: physical (G by FFT passes every iteration, the "
                         "paper's formulation) or spectral (iterate on the half spectra, G pointwise)")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default tile widths instead of the library's autotuner (ad_autotune) on every "
                         "plan the benchmark times")
    ap.add_argument("--extras", default="methods,3d512,3d256,closure,uneven48,learned512",
                    help="comma list of extra measurements on rank 0: methods, 3d512 (pass rooflines of the "
                         "512^3 x 3 velocity), 3d256, closure (needs 3d256), uneven48, learned512")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import paper_1707_09177_gb300 as gad

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    B, gamma, tol = args.batch, WORKLOAD["gamma"], WORKLOAD["tol"]
    n = WORKLOAD["shape"]
    P = n[0] * n[1]
    seeds = rank_seeds(rank, B)
    gad.load()
    if args.host_loop:
        gad.set_graph_mode(False)
    _TUNE[0] = not args.no_tune
    _tune(gad, n, gamma, B, args.method)

    # inputs: true fields from the seeded generator, filtered by the library
    u_true = torch.from_numpy(_fields(seeds)).to(dev)
    ubar = gad.filter(u_true, gamma, ndim=2)
    del u_true
    ubar_host = ubar.cpu().pin_memory()
    out = torch.empty_like(ubar)
    stream = torch.cuda.current_stream()

    def step(method, maxit=3000, tol_=tol, space=args.space):
        return gad.deconvolve(ubar, gamma, method=method, tol=tol_, maxit=maxit, ndim=2, out=out, space=space)

    def barrier():
        if ws > 1:
            dist.barrier()

    for _ in range(max(args.warmup, 3)):
        res = step(args.method)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            res = step(args.method)
            launches += res.launches
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    clocks = clk.summary()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dev)
    value = whole_job_mpoints(ws, B, P, ms * 1e-3)
    iters = [int(x) for x in res.iterations]
    ok = bool(np.all(res.status == gad.AD_OK))

    # end to end through the C ABI's host-buffer call: the library copies u_bar
    # in from pinned host memory, solves, and copies u* back out
    host_out = torch.empty(ubar.shape, dtype=ubar.dtype).pin_memory()

    def e2e_step():
        return gad.deconvolve_host(ubar_host, gamma, method=args.method, tol=tol, maxit=3000, ndim=2, out=host_out,
                                   space=args.space)

    e2e_step()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, dev)
    e2e_same = bool(torch.equal(host_out, out.cpu()))     # same kernels on the same values: bitwise equal
    nbytes = ubar.numel() * ubar.element_size()
    e2e = {"value": whole_job_mpoints(ws, B, P, e2e_s), "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(_workload_config(args, ws),
                           dots="f64 (compensated f32 products)",
                           l2="inputs %d MiB per vector, > L2 at batch 16; no flush" % (B * P * 4 >> 20),
                           loop="host" if args.host_loop else "graph while node",
                           tiles="autotuned (ad_autotune)" if _TUNE[0] else "default"),
            "iterations": {"min": min(iters), "max": max(iters), "mean": float(np.mean(iters))},
            "converged": ok, "e2e": e2e, "e2e_equals_device": e2e_same, "gpu_launches": int(launches), "clocks": clocks}
    extras = set() if args.no_extras else set(x for x in args.extras.split(",") if x)
    try:
        if rank == 0 and not args.no_extras:
            _guarded(line, "roofline", lambda: _rooflines(gad, line, args, n, gamma, B))
            _guarded(line, "cpu_baseline", lambda: _cpu_baseline(line, ubar_host, gamma, args.method, iters[0], P))
        if rank == 0 and "methods" in extras:
            _guarded(line, "methods", lambda: _methods(gad, line, step, stream, B, P))
        if rank == 0 and "3d512" in extras:
            _guarded(line, "roofline_3d512", lambda: _roofline_3d512(gad, line))
        if rank == 0 and "learned512" in extras:
            _guarded(line, "roofline_conv", lambda: _roofline_conv(gad, line))
        if rank == 0 and (extras & {"3d256", "closure", "uneven48", "learned512"}):
            del out, host_out
            torch.cuda.empty_cache()
            line["workloads"] = {}
            _extra_workloads(gad, dev, extras, line)
    finally:
        if rank == 0:
            print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def _guarded(line, name, fn):
    """Runs one optional measurement; an exception is recorded in the line's
    "errors" (and printed to stderr) instead of ending the benchmark."""
    try:
        fn()
    except Exception as e:  # noqa: BLE001 - every failure of an extra is reported, none is fatal
        import traceback
        traceback.print_exc()
        line.setdefault("errors", {})[name] = "%s: %s" % (type(e).__name__, str(e)[:400])


def _pass_table(gad, shape, gamma, B, method, space, P, SP, reps=20):
    passes = gad.time_passes(shape, gamma, B, method=method, reps=reps, space=space)
    for p in passes:
        p["bytes"] = _pass_bytes(p["kind"], p["op"], P, SP, B, method)
        p["gbs"] = p["bytes"] / (p["ms"] * 1e-3) / 1e9
    return passes


def _roofline_entry(passes, peak, src, space):
    """The dominant pass kernel (longest per-launch time) against the HBM peak."""
    best = max(passes, key=lambda p: p["ms"])
    total = sum(p["ms"] for p in passes)
    return {"bound": "hbm", "kernel": "%s(op %d)" % (best["kind"], best["op"]),
            "achieved": best["gbs"], "peak": peak, "unit": "GB/s", "frac": best["gbs"] / peak,
            "peak_source": src + " hbm_gbs (copy, burst)",
            "traffic": _traffic(best["kind"], best["op"], space),
            "share_of_iteration": best["ms"] / total,
            "passes": [{k: p[k] for k in ("index", "kind", "op", "ms", "gbs")} for p in passes]}


def _solve_entry(gad, passes, shape, gamma, B, method, space, peak, src, reps=10):
    """One whole iteration body (every pass launch in order, CUDA events around
    the sequence): its algorithmic bytes over its time, against the HBM peak."""
    body_ms = gad.time_body(shape, gamma, B, method=method, reps=reps, space=space)
    nbytes = float(sum(p["bytes"] for p in passes))
    ach = nbytes / (body_ms * 1e-3) / 1e9
    ent = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
           "peak_source": src + " hbm_gbs (copy, burst)", "bytes_per_body": nbytes, "ms_per_body": body_ms,
           "launches_per_body": len(passes), "sum_of_pass_ms": float(sum(p["ms"] for p in passes))}
    # the same body by DRAM bytes (ncu, profiles/traffic.json) when every pass has a capture
    key = space + ("3d" if len(shape) == 3 else "")
    tr = [_traffic(p["kind"], p["op"], key) for p in passes]
    if tr and all(t is not None for t in tr):
        dram = float(sum(tr)) / (body_ms * 1e-3) / 1e9
        ent["dram"] = {"bytes_per_body": float(sum(tr)), "achieved": dram, "frac": dram / peak,
                       "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch"}
    return ent


def _rooflines(gad, line, args, n, gamma, B):
    """Rooflines of the timed workload's passes, timed live with CUDA events:
    the dominant kernel (`roofline`), the whole iteration body
    (`roofline_solve`), the same for the other iteration space, and the
    preconditioned CG pass set with its stencil kernel."""
    P = n[0] * n[1]
    SP = (n[1] // 2 + 1) * n[0]
    peak, src = _peaks()
    other = "spectral" if args.space == "physical" else "physical"
    for space, key in ((args.space, ""), (other, "_" + other)):
        passes = _pass_table(gad, n, gamma, B, args.method, space, P, SP)
        line["roofline" + key] = _roofline_entry(passes, peak, src, space)
        line["roofline_solve" + key] = _solve_entry(gad, passes, n, gamma, B, args.method, space, peak, src)
    pp = _pass_table(gad, n, gamma, B, "pcg", "physical", P, SP)
    line["passes_pcg"] = [{k: p[k] for k in ("index", "kind", "op", "ms", "gbs")} for p in pp]


def _roofline_3d512(gad, line, method="bicgstab"):
    """The 3D 512^3 x 3 velocity (gamma = 0.01): every pass of one BiCGSTAB
    body and the whole body against the HBM peak, physical space."""
    n = (512, 512, 512)
    B, gamma = 3, 0.01
    P = n[0] * n[1] * n[2]
    SP = (n[2] // 2 + 1) * n[0] * n[1]
    peak, src = _peaks()
    _tune(gad, n, gamma, B, method)
    passes = _pass_table(gad, n, gamma, B, method, "physical", P, SP, reps=5)
    ent = _roofline_entry(passes, peak, src, "physical3d")
    ent["solve"] = _solve_entry(gad, passes, n, gamma, B, method, "physical", peak, src, reps=5)
    ent["workload"] = "velocity3d_512_f32 (3 components), %s body" % method
    line["roofline_3d512"] = ent


def _roofline_conv(gad, line):
    """One 32 -> 32 layer of the learned guess's network on the 512^3 x 3
    velocity (the inference launch shape), timed by the library with CUDA
    events, against the measured bf16 tensor peak (burst: the kernel is timed
    alone): 55,296 flop per grid point (27 taps x 32 x 32 multiply-adds)."""
    n, B = 512, 3
    ms, tc = gad.guess_time_conv((n, n, n), B, reps=5)
    flops = B * n ** 3 * 27 * 32 * 32 * 2.0
    peak, src = _bf16_peak()
    ach = flops / (ms * 1e-3) / 1e12
    line["roofline_conv"] = {"bound": "tensor", "kernel": "k_conv_tc" if tc else "k_conv_mma", "achieved": ach,
                             "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "ms": ms,
                             "peak_source": src + " bf16_tflops (cuBLAS, burst)", "traffic": _traffic_conv(),
                             "workload": "velocity3d_512_f32 learned guess, one 32->32 layer, 3 components"}


def _bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


def _host_cpu():
    """The host's CPU model (from /proc/cpuinfo where present) and logical cores."""
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                key = ln.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware"):
                    model = ln.split(":", 1)[1].strip()
                    if key == "model name":
                        break
                    if key == "cpu part":
                        # Arm part numbers of /proc/cpuinfo
                        model = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1",
                                 "0xd0c": "Arm Neoverse N1", "0xd49": "Arm Neoverse N2"}.get(model.lower(),
                                                                                           "Arm cpu part " + model)
    except OSError:
        pass
    return model, os.cpu_count()


def _cpu_baseline(line, ubar_host, gamma, method, n0, P):
    """The oracle on this host's cores (one thread), bounded sample: a 0-pass
    and a 4-pass solve of field 0, extrapolated to the GPU's pass count."""
    os.environ["OMP_NUM_THREADS"] = "1"
    ub0 = ubar_host[0].numpy().astype(np.float64)
    sample_passes = 4
    t_solve, per, t0 = _oracle_estimate(ub0, gamma, method, n0, sample_passes)
    cpu_val = P / t_solve / 1e6
    model, ncpu = _host_cpu()
    line["cpu_baseline"] = {"value": cpu_val, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "cpu_model": model, "host_cores": ncpu,
                            "sample": ("oracle %s (float64 NumPy, 1 thread), field 0 of the batch: a 0-pass "
                                       "solve (%.2f s fixed cost) and a %d-pass solve (%.2f s per pass), "
                                       "extrapolated to the %d passes the GPU solve of that field needed"
                                       % (method, t0, sample_passes, per, n0))}


def _methods(gad, line, step, stream, B, P):
    """Comparison methods on the same batch, one timed solve each."""
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    methods = {}
    line["methods"] = methods
    for m, mi, sp in (("cg", 3000, "physical"), ("bicgstab", 3000, "physical"), ("pcg", 3000, "physical"),
                      ("vancittert", VC_MAXIT, "physical"), ("cg", 3000, "spectral"), ("pcg", 3000, "spectral"),
                      ("bicgstab", 3000, "spectral"), ("vancittert", VC_MAXIT, "spectral")):
        step(m, maxit=mi, space=sp)
        torch.cuda.synchronize()
        ev0.record(stream)
        r = step(m, maxit=mi, space=sp)
        ev1.record(stream)
        torch.cuda.synchronize()
        t = ev0.elapsed_time(ev1)
        its = [int(x) for x in r.iterations]
        reached = bool(np.all(r.status == gad.AD_OK))
        hfin = [float(r.history[b, its[b]]) for b in range(B)]
        key = m if sp == "physical" else m + "_spectral"
        methods[key] = {"ms": t, "iterations_mean": float(np.mean(its)), "reached_tol": reached,
                        "mpoints_s": B * P / (t * 1e-3) / 1e6 if reached else None,
                        "mpoints_s_per_pass": B * P * float(np.mean(its)) / (t * 1e-3) / 1e6,
                        "h_final_max": max(hfin), "launches": r.launches}
        if m == "vancittert":
            methods[key]["maxit"] = VC_MAXIT


if __name__ == "__main__":
    main()
