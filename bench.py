"""Benchmark: FD-preconditioned FGMRES solve of the space-time heat equation.

Workload (the paper's method at scale, synthetic): unit cube x (0, 1), d = 3,
p = 3, 64 elements per direction (n_s = 65, n_t = 66, N = 18,125,250 dofs),
gamma = nu = 1, right-hand side = load of f = u_t - Lap u for the manufactured
solution u = sin(pi x) sin(pi y) sin(pi z) sin(t). One step = one full solve to
a relative residual of 1e-8 from f resident in HBM: every fd_apply (Algorithm
1), st_matvec (eq. syst_mat), Gram-Schmidt and the true-residual check.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: the method's unit of work is one independent solve, so N GPUs run N
replicas (no data-path collective; "scaling": "weak"). `--impl reference`
times the CPU FP64 oracle (the only reference this paper has) on the host.
"""
import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1909_07309_gb300 import inputs  # noqa: E402

METRIC = "fd_apply dofs/s and GMRES time-to-1e-8 residual, FP64 vs TF32/BF16-precond"
UNIT = "dofs/s"
L2_BYTES = 129 * 2 ** 20

# DRAM bytes per launch from one ncu capture at the workload (profiles/): the
# mean over the 8 mode products of one fd_apply, and over the 4 band passes of
# one st_matvec; None once a kernel changes until it is captured again.
NCU_TRAFFIC = {"band_fx64": 4.586e8, "fd_mode_tc7": 2.363e8}

# Arithmetic of the headline solve, no narrower than FP64 anywhere: Algorithm 1
# with the mode products on the tensor cores by seven exact digit slices per
# entry (kept digit pairs accumulated exactly, one rounding to FP64, FP64
# intermediates) and an IEEE-FP64 Step 3; the banded matvec with each product formed
# exactly in integer limbs and rounded once to FP64; FP64 GMRES.
HEADLINE = dict(precond="STFD_FP64TC7", matvec="STFD_OP_FX64", dtype="f64",
                precond_text="Algorithm 1, FP64: mode products on tcgen05 by seven exact BF16 digit slices per entry "
                             "(28 digit pairs, exact FP32 accumulators, one rounding to FP64; FP64 intermediates), "
                             "Step 3 in IEEE FP64",
                matvec_text="FP64 sum-factorised banded products, each formed exactly in 64-bit integer limbs "
                            "and rounded once to FP64 (FP64 intermediates)")


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every `interval_ms` during
    the timed region. All GPUs are queried (nvidia-smi does not follow
    CUDA_VISIBLE_DEVICES) and the lines of this process's GPU are picked by UUID;
    only samples whose timestamps fall inside the marked region are kept."""

    FIELDS = ("timestamp,index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index, uuid=None, interval_ms=50):
        self.gpu = str(gpu_index)
        self.uuid = (uuid or "").lower()
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self, first_sample_timeout_s=5.0):
        """Start nvidia-smi and wait (bounded) for its first sample."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", str(self.interval_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        deadline = time.time() + first_sample_timeout_s
        while not self.lines and time.time() < deadline and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark_start(self):
        self.t0 = time.time()

    def mark_stop(self):
        self.t1 = time.time()

    @staticmethod
    def _stamp(text, fallback):
        try:
            return datetime.datetime.strptime(text, "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return fallback

    def _mine(self, rows):
        """Rows of this process's GPU: by UUID, else the only GPU, else by index."""
        if self.uuid:
            own = [r for r in rows if r["uuid"].lower().endswith(self.uuid)]
            if own:
                return own
        if len({r["index"] for r in rows}) == 1:
            return rows
        return [r for r in rows if r["index"] == self.gpu]

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        if self.t1 is None:
            self.mark_stop()
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait(timeout=5)
        self.thread.join(timeout=5)
        rows = []
        for arrived, line in list(self.lines):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < len(self.FIELDS.split(",")):
                continue
            try:
                sm, smax = float(parts[3]), float(parts[4])
            except ValueError:
                continue
            rows.append({"t": self._stamp(parts[0], arrived), "index": parts[1], "uuid": parts[2], "sm": sm,
                         "smax": smax, "flags": parts[7:11]})
        rows = self._mine(rows)
        t0 = self.t0 if self.t0 is not None else float("-inf")
        window = "timed region"
        sel = [r for r in rows if t0 <= r["t"] <= self.t1]
        if not sel:   # region shorter than the sampling interval: the nearest samples
            window = "timed region +- 0.5 s"
            sel = [r for r in rows if t0 - 0.5 <= r["t"] <= self.t1 + 0.5]
        reasons = sorted({nm for r in sel for nm, flag in zip(self.REASONS, r["flags"])
                          if flag.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r["sm"] for r in sel) if sel else None,
                "sm_max_mhz": max(r["smax"] for r in sel) if sel else None,
                "reasons": reasons, "samples": len(sel), "interval_ms": self.interval_ms, "window": window}


def device_uuid(index):
    """UUID of CUDA device `index` as 8-4-4-4-12 hex (nvidia-smi prints it after "GPU-"), or None."""
    import torch
    try:
        text = str(torch.cuda.get_device_properties(index).uuid)
    except (AttributeError, RuntimeError):
        return None
    return text[4:] if text.upper().startswith("GPU-") else text


def max_over_ranks(x, world, device):
    """Largest value over all ranks (the job's wall time is the slowest replica's)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(N, steps, world, ms):
    """Whole-job dofs/s: every rank solved `steps` independent problems of N dofs."""
    return N * steps * world / (ms * 1e-3)


def build_workload(cfg):
    """Univariate factors from the library's own spline assembly and the RHS load."""
    from paper_1909_07309_gb300 import stfd
    d, p, n_el, T = cfg["d"], cfg["p"], cfg["n_el"], cfg["T"]
    gamma, nu = cfg["gamma"], cfg["nu"]
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el, T=T)
    Fx = stfd.stfd_spline_load_trig(p, n_el, 1.0, stfd.STFD_BC_DIRICHLET, np.pi, 1.0, 0.0)
    Ft = stfd.stfd_spline_load_trig(p, n_el, T, stfd.STFD_BC_INITIAL, 1.0, d * np.pi ** 2 * nu, gamma)
    f = np.ones(1)
    for F in [Fx] * d + [Ft]:                 # vec order: direction 1 fastest, time slowest
        f = np.outer(F, f).ravel()
    return K, M, Wt, Mt, f


def _spline_l2_misfit(p, n_el, length, bc_drop, coef, fn, nq=None):
    """int_0^length (fn - sum_i coef_i b_i)^2 for the reduced open-uniform basis of
    degree p (bc_drop = (first dropped, last dropped)), by Gauss-Legendre per element."""
    from scipy.interpolate import BSpline
    nq = nq or p + 8
    t = np.r_[[0.0] * (p + 1), length * np.arange(1, n_el) / n_el, [length] * (p + 1)]
    full = np.zeros(n_el + p)
    full[int(bc_drop[0]):n_el + p - int(bc_drop[1])] = coef
    s = BSpline(t, full, p, extrapolate=False)
    g, w = np.polynomial.legendre.leggauss(nq)
    h = length / n_el
    x = (np.arange(n_el)[:, None] + 0.5 * (g[None, :] + 1.0)) * h
    return float(np.sum(w[None, :] * (fn(x) - s(x)) ** 2) * 0.5 * h)


def l2_error_sine(cfg, M, Mt, u_dev):
    """Space-time L2 error of the discrete solution u_h = sum_i u_i B_i against
    u = sin(pi x_1) ... sin(pi x_d) sin(t) (Sec. 5.1), split without cancellation:
    ||u - u_h||^2 = ||u - Pi u||^2 + ||Pi u - u_h||^2 with Pi the L2 projection onto
    the trial space. Pi is the tensor product of the 1D projections (u is separable),
    so the first term is prod a_l - prod (a_l - e_l^2) with a_l = ||u_l||^2 and e_l^2
    the 1D projection misfits (expanded over subsets); the second is d^T (M_t (x) M_s) d
    with d = c_Pi - u_h, formed on the device by the library's Kronecker matvec."""
    import itertools

    import torch

    from paper_1909_07309_gb300 import stfd
    d, p, n_el, T = cfg["d"], cfg["p"], cfg["n_el"], cfg["T"]
    Fx = stfd.stfd_spline_load_trig(p, n_el, 1.0, stfd.STFD_BC_DIRICHLET, np.pi, 1.0, 0.0)
    Ft = stfd.stfd_spline_load_trig(p, n_el, T, stfd.STFD_BC_INITIAL, 1.0, 1.0, 0.0)
    cx = np.linalg.solve(M[0], Fx)
    ct = np.linalg.solve(Mt, Ft)
    ex = _spline_l2_misfit(p, n_el, 1.0, (1, 1), cx, lambda x: np.sin(np.pi * x))
    et = _spline_l2_misfit(p, n_el, T, (1, 0), ct, np.sin)
    a = [0.5] * d + [T / 2.0 - np.sin(2.0 * T) / 4.0]
    e = [ex] * d + [et]
    proj = 0.0
    for k in range(1, d + 2):
        for S in itertools.combinations(range(d + 1), k):
            proj += (-1) ** (k + 1) * np.prod([e[l] if l in S else a[l] for l in range(d + 1)])
    c = np.ones(1)
    for v in [cx] * d + [ct]:
        c = np.outer(v, c).ravel()
    diff = torch.from_numpy(c).to(u_dev.device) - u_dev
    mass = stfd.KronOp(M, M, Mt, Mt, 1.0, 0.0, arith=stfd.STFD_OP_FP64)
    Md = torch.empty_like(diff)
    mass.matvec(diff, Md)
    disc = float(torch.dot(diff, Md))
    mass.close()
    return {"l2_error": float(np.sqrt(proj + disc)), "projection_part_sq": float(proj),
            "discrete_part_sq": disc}


def oracle_setup(cfg):
    """Matrices, right-hand side and FD factors of the oracle for one workload (untimed)."""
    from oracle import fd as ofd, loads as oloads, matrices as omat
    d, p, n_el, T = cfg["d"], cfg["p"], cfg["n_el"], cfg["T"]
    K, M = omat.space_matrices(p, n_el)
    Wt, Mt = omat.time_matrices(p, n_el, T)
    Fx = oloads.load_1d(p, n_el, 1.0, lambda x: np.sin(np.pi * x), 12)
    Ft = oloads.load_1d(p, n_el, T, lambda t: d * np.pi ** 2 * cfg["nu"] * np.sin(t) + cfg["gamma"] * np.cos(t),
                        12, True, False)
    f = oloads.load_separable([Fx] * d, Ft)
    fac = ofd.setup([K] * d, [M] * d, Wt, Mt)
    return dict(K=K, M=M, Wt=Wt, Mt=Mt, f=f, fac=fac)


def oracle_solve(cfg, S):
    """One FD-preconditioned GMRES solve by the CPU oracle on the set-up workload S;
    returns (seconds, iters, N, true relative residual)."""
    from oracle import fd as ofd, gmres as ogmres, kron as okron
    d, gamma, nu = cfg["d"], cfg["gamma"], cfg["nu"]
    K, M, Wt, Mt, f = S["K"], S["M"], S["Wt"], S["Mt"], S["f"]
    t1 = time.perf_counter()
    x, info = ogmres.gmres(lambda v: okron.st_matvec(v, [K] * d, [M] * d, Wt, Mt, gamma, nu),
                           lambda v: ofd.apply(S["fac"], v, gamma, nu)[0], f, tol=1e-8, restart=100)
    res = np.linalg.norm(f - okron.st_matvec(x, [K] * d, [M] * d, Wt, Mt, gamma, nu)) / np.linalg.norm(f)
    return time.perf_counter() - t1, info["iters"], f.size, res


def run_oracle_solve(cfg):
    """Set up and solve once by the CPU oracle; returns (solve seconds, setup seconds, iters, N, residual)."""
    t0 = time.perf_counter()
    S = oracle_setup(cfg)
    setup_s = time.perf_counter() - t0
    secs, iters, N, res = oracle_solve(cfg, S)
    return secs, setup_s, iters, N, res


def cuda_time(fn, reps, stream):
    """Average milliseconds of fn() over reps calls (CUDA events on `stream`)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = None
    for _ in range(reps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def mapped_section(args, stream):
    """Mixed-precision workload on the mapped domain: the FP64 vs TF32 / BF16
    geometry-aware preconditioner inside FP64 flexible GMRES whose system matvec
    is FP64 -- the integer-limb stencil (exact row sums rounded once) first, the
    IEEE-FP64 stencil beside it with the FP64 and BF16 preconditioners -- and the
    same preconditioners with the double-float (~48-bit) stencil matvec (and the
    plain parametric preconditioner for the iteration count)."""
    import torch
    from paper_1909_07309_gb300 import stfd
    cfg = dict(inputs.MAPPED)
    if args.mapped_n_el:
        cfg["n_el"] = args.mapped_n_el
    d, p, n_el = cfg["d"], cfg["p"], cfg["n_el"]
    t0 = time.perf_counter()
    prob = stfd.mapped_problem(d, p, n_el, stfd.STFD_GEOM_QUARTER_ANNULUS, c=inputs.c_bilinear,
                               kappa=inputs.kappa_trig, T=cfg["T"])
    host_setup_s = time.perf_counter() - t0
    n = prob["n"]
    N = int(np.prod(n))
    mass = stfd.StencilOp(n, p, prob["Ms"], prob["Ms"], prob["Mt"], prob["Mt"], 1.0, 0.0, arith=stfd.STFD_OP_FP64)
    f = mass.matvec(torch.from_numpy(inputs.standard_normal(N, cfg["rhs_seed"])).cuda())
    mass.close()
    # preconditioner accuracy is stated on an N(0,1) input: on the right-hand side
    # f = (M_t x M_s) c the rounding noise of a low-precision input is of the size
    # of f's own smooth content, which P^{-1} amplifies most
    r = torch.from_numpy(inputs.standard_normal(N, cfg["rhs_seed"] + 1)).cuda()
    steps = args.mapped_steps
    out = {"workload": cfg["name"], "N": N, "host_setup_s": host_setup_s, "steps": steps}
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el, T=cfg["T"])
    y = torch.empty_like(f)
    mv_desc = {"fx64": "stencil, FP64 (time pass IEEE FP64; spatial row sums exact in integer limbs, "
                       "rounded once)",
               "fp64": "stencil, IEEE FP64", "df32": "stencil, double-float (~48-bit)"}
    for mv_name, arith in (("fx64", stfd.STFD_OP_FX64), ("fp64", stfd.STFD_OP_FP64), ("df32", stfd.STFD_OP_DF32)):
        A = stfd.StencilOp(n, p, prob["Ms"], prob["Ks"], prob["Wt"], prob["Mt"], cfg["gamma"], cfg["nu"], arith=arith)
        mv_ms, _ = cuda_time(lambda: A.matvec(f, y), 3, stream)
        sec = {"matvec": mv_desc[mv_name], "st_matvec_ms": mv_ms, "variants": {}}
        if mv_name == "fx64":
            y_fx = y.clone()
        elif mv_name == "fp64":   # the two FP64 matvecs on the same input
            sec["fx64_matvec_rel_diff"] = float(torch.linalg.norm(y_fx - y) / torch.linalg.norm(y))
            del y_fx
        # one untimed solve first, so that no timed solve allocates the Krylov workspace
        Pw = stfd.geometry_preconditioner(prob, cfg["gamma"], cfg["nu"], precision=stfd.STFD_BF16)
        A.gmres(Pw, f, y, tol=1e-8)
        Pw.close()
        s_ref = None
        plist = [("fp64_ieee", stfd.STFD_FP64, True), ("fp64_accurate_df32", stfd.STFD_DF32, True),
                 ("tf32", stfd.STFD_TF32, True), ("bf16", stfd.STFD_BF16, True)]
        if mv_name == "fp64":   # the slowest matvec: the two ends of the comparison only
            plist = [plist[0], plist[3]]
        if mv_name == "df32":
            plist.append(("plain_fp64_accurate_df32", stfd.STFD_DF32, False))
        for name, prec, geo in plist:
            P = stfd.geometry_preconditioner(prob, cfg["gamma"], cfg["nu"], precision=prec) if geo else \
                stfd.FD(K, M, Wt, Mt, cfg["gamma"], cfg["nu"], precision=prec)
            s = torch.empty_like(f)
            P.apply(r, s)
            fd_ms, _ = cuda_time(lambda: P.apply(r, s), 3, stream)
            if s_ref is None:
                s_ref = s.clone()
            err = float(torch.linalg.norm(s - s_ref) / torch.linalg.norm(s_ref)) if geo else None
            reps = steps if (geo and prec in (stfd.STFD_TF32, stfd.STFD_BF16)) else 1
            if geo and reps > 1:
                A.gmres(P, f, y, tol=1e-8)      # warm-up
            gm_ms, (_, info) = cuda_time(lambda: A.gmres(P, f, y, tol=1e-8), reps, stream)
            sec["variants"][name] = {"precond": ("A^G " if geo else "A^ ") + name.replace("plain_", ""),
                                     "fd_apply_ms": fd_ms, "fd_apply_rel_err_vs_fp64_on_N01_input": err,
                                     "gmres_ms": gm_ms,
                                     "gmres_iters": info["iters"], "rel_res_true": info["rel_res_true"]}
            P.close()
        ieee = sec["variants"]["fp64_ieee"]["gmres_ms"]
        for v in sec["variants"].values():
            v["speedup_vs_fp64_ieee_precond"] = ieee / v["gmres_ms"]
        A.close()
        torch.cuda.empty_cache()
        out[mv_name + "_matvec"] = sec
    return out


def adjoint_section(args, stream):
    """Gradient of the L2 misfit w.r.t. the per-element conductivity and the
    source: forward FGMRES + adjoint FGMRES (transposed FD) + device contraction."""
    import torch
    from paper_1909_07309_gb300 import autograd as ag, stfd
    cfg = inputs.ADJOINT
    d, p, n_el = cfg["d"], cfg["p"], cfg["n_el"]
    kap, kap_obs, c = inputs.adjoint_draws(cfg)
    model = ag.MappedHeatModel(d, p, n_el, stfd.STFD_GEOM_QUARTER_ANNULUS, kappa_ref=kap, T=cfg["T"], tol=1e-10)
    f = model.mass.matvec(torch.from_numpy(c).cuda())
    u_obs = ag.solve(torch.as_tensor(kap_obs), f, model).detach()

    def grad_eval():
        kt = torch.tensor(kap, requires_grad=True)
        ft = f.clone().requires_grad_(True)
        L = ag.l2_misfit(ag.solve(kt, ft, model), u_obs, model)
        L.backward()
        return float(L.detach()), kt.grad, ft.grad

    for _ in range(2):
        grad_eval()
    model.iters.clear()
    steps = max(1, args.mapped_steps)
    t0 = time.perf_counter()
    for _ in range(steps):
        L, gk, gf = grad_eval()
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) / steps
    its = model.iters[:2]
    # central differences (h = 1e-6) on two random directions, tight solves
    model.tol = 1e-13
    L, gk, gf = grad_eval()
    g = np.random.default_rng(20)
    worst = 0.0
    for _ in range(2):
        v = g.standard_normal(kap.size)
        with torch.no_grad():
            lp = float(ag.l2_misfit(ag.solve(torch.as_tensor(kap + 1e-6 * v), f, model), u_obs, model))
            lm = float(ag.l2_misfit(ag.solve(torch.as_tensor(kap - 1e-6 * v), f, model), u_obs, model))
        fd = (lp - lm) / 2e-6
        worst = max(worst, abs(fd - float(gk.numpy() @ v)) / (np.linalg.norm(gk.numpy()) * np.linalg.norm(v)))
    N = model.N
    return {"workload": cfg["name"], "N": N, "loss": L, "gradient_ms": wall * 1e3,
            "includes": "host assembly of K_s(kappa), forward FGMRES, adjoint FGMRES with P^-T, element contraction",
            "forward_iters": its[0] if its else None, "adjoint_iters": its[1] if len(its) > 1 else None,
            "fd_check_max_rel_dev": worst, "fd_check": "central differences h=1e-6, 2 directions, tol 1e-13"}


def batch_section(args, stream):
    """Batched workload: 512 uneven unit-square problems in one persistent,
    graph-captured launch; aggregate dofs/s and p50 / p99 per-problem solve time.
    IEEE FP64 with FD-preconditioned refinement to a relative residual of 1e-8
    (the headline of this section), and the double-float batch beside it."""
    import torch
    from paper_1909_07309_gb300 import stfd
    cfg = inputs.BATCH
    n_el, p, nrhs, g = inputs.batch_draws(cfg)
    f = None
    out = {"workload": cfg["name"], "launch": "1 persistent kernel per batch, CUDA graph replay"}
    for name, prec in (("fp64", stfd.STFD_FP64), ("df32", stfd.STFD_DF32)):
        t0 = time.perf_counter()
        B = stfd.Batch(n_el, p, nrhs, d=cfg["d"], T=cfg["T"], gamma=cfg["gamma"], nu=cfg["nu"], autotune=True,
                       precision=prec, tol=1e-8, max_it=5)
        setup_s = time.perf_counter() - t0
        if f is None:
            f = torch.from_numpy(g.standard_normal(B.total)).cuda()
        u = torch.empty_like(f)
        rel = torch.empty(B.n_items, dtype=torch.float64, device="cuda")
        for _ in range(3):
            B.solve(f, u, rel)
        reps = max(3, args.steps // 4)
        ms, _ = cuda_time(lambda: B.solve(f, u, rel), reps, stream)
        us, (th, ct), tune = B.stats()
        its = B.iterations()
        dofs = int(B.total)
        res = {"problems": B.count, "items": B.n_items, "dofs_per_solve": dofs,
               "ms_per_batch": ms, "dofs_per_s": dofs / (ms * 1e-3), "setup_s": setup_s,
               "p50_problem_us": float(np.percentile(us, 50)), "p99_problem_us": float(np.percentile(us, 99)),
               "max_rel_res_true": float(rel.max()), "iterations_max": int(its.max()),
               "items_above_tol": int((rel > 1e-8).sum().item()),
               "config": {"threads": th, "ctas_per_sm": ct}, "autotune_ms": tune,
               "solve": "FD-preconditioned iterative refinement (Algorithm 1 + true residual) to 1e-8, max 5, "
                        + ("IEEE FP64" if prec == stfd.STFD_FP64 else "double-float")}
        B.close()
        if name == "fp64":
            out.update(res)
        else:
            out["df32"] = res
    return out


def blas_threads():
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count() or 1


REFERENCE_BUDGET_S = 120.0   # timed oracle solves stop after this much wall time (at least one)


def reference_main(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg = inputs.SCALE
    S = oracle_setup(cfg)
    for _ in range(args.warmup):
        oracle_solve(cfg, S)
    times = []
    iters = N = 0
    res = None
    for _ in range(args.steps):
        t, iters, N, res = oracle_solve(cfg, S)
        times.append(t)
        if sum(times) > REFERENCE_BUDGET_S:
            break
    total = sum(times)
    value = N * len(times) / total
    cores = blas_threads()
    sample = ("one full oracle solve per step (numpy FP64, complex Algorithm 1, mode-product matvec, "
              "MGS GMRES); setup excluded as in the GPU arm")
    if len(times) < args.steps:
        sample += "; %d of the %d requested steps timed (stopped after %.0f s)" % (len(times), args.steps,
                                                                                  REFERENCE_BUDGET_S)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": len(times), "steps_requested": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg["name"], "N": N, "solve": "FD-preconditioned GMRES to 1e-8, x0 = 0",
                   "gmres_iters": iters, "rel_res_true": res},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--restart", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mapped", action="store_true", help="skip the mapped-domain mixed-precision workload")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint gradient workload")
    ap.add_argument("--mapped-n-el", type=int, default=0, help="elements per direction of the mapped workload")
    ap.add_argument("--mapped-steps", type=int, default=2)
    ap.add_argument("--no-batch", action="store_true", help="skip the batched workload")
    ap.add_argument("--oracle-once", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_once:   # child of the cpu_baseline leg: one oracle solve, one JSON line
        secs, _, iters, Nc, _ = run_oracle_solve(inputs.SCALE)
        print(json.dumps({"value": Nc / secs, "seconds": secs, "iters": iters}), flush=True)
        return 0
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return reference_main(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    from paper_1909_07309_gb300 import stfd
    stfd.load(build_if_missing=False)

    cfg = inputs.SCALE
    K, M, Wt, Mt, f_np = build_workload(cfg)
    t_setup = time.perf_counter()
    A = stfd.KronOp(K, M, Wt, Mt, cfg["gamma"], cfg["nu"], arith=getattr(stfd, HEADLINE["matvec"]))
    P = stfd.FD(K, M, Wt, Mt, cfg["gamma"], cfg["nu"], precision=getattr(stfd, HEADLINE["precond"]))
    head_prec = getattr(stfd, HEADLINE["precond"])
    setup_ms = (time.perf_counter() - t_setup) * 1e3
    N = P.N
    f = torch.from_numpy(f_np).cuda()
    u = torch.empty_like(f)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def solve():
        return A.gmres(P, f, u, tol=1e-8, restart=args.restart)

    for _ in range(args.warmup):
        _, info = solve()
    torch.cuda.synchronize()

    # ---- timed region: K full solves, inputs resident in HBM (working set > L2)
    sampler = ClockSampler(local_rank, uuid=device_uuid(local_rank))
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    launches0 = stfd.stfd_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler.mark_start()
    e0.record(stream)
    infos = []
    for _ in range(args.steps):
        _, info = solve()
        infos.append(info)
    e1.record(stream)
    torch.cuda.synchronize()
    sampler.mark_stop()
    barrier()
    clocks = sampler.stop()
    launches = stfd.stfd_launch_count() - launches0
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    value = job_throughput(N, args.steps, world, ms)

    # ---- end to end through the public API: every step copies its right-hand side
    # from pinned host memory, solves, and copies the solution back. Uploads and
    # downloads run on two more streams (one per direction, so that they use the
    # link both ways at once): the upload of step k+1 and the download of step
    # k-1 overlap the solve of step k (double-buffered device vectors).
    f_host = [torch.from_numpy(f_np).pin_memory() for _ in range(2)]
    u_host = [torch.empty(N, dtype=torch.float64).pin_memory() for _ in range(2)]
    f_dev = [torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(2)]
    u_dev = [torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(2)]
    up_s, down_s = torch.cuda.Stream(), torch.cuda.Stream()
    comp_s = torch.cuda.current_stream()
    h2d = [torch.cuda.Event() for _ in range(2)]
    solved = [torch.cuda.Event() for _ in range(2)]
    d2h = [torch.cuda.Event() for _ in range(2)]
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(up_s):
        f_dev[0].copy_(f_host[0], non_blocking=True)
    h2d[0].record(up_s)
    for k in range(args.steps):
        b = k % 2
        comp_s.wait_event(h2d[b])
        if k + 1 < args.steps:
            nb = (k + 1) % 2           # read by solve k-1, which has returned
            with torch.cuda.stream(up_s):
                f_dev[nb].copy_(f_host[nb], non_blocking=True)
            h2d[nb].record(up_s)
        if k >= 2:
            comp_s.wait_event(d2h[b])  # u_dev[b] still being downloaded for step k-2
        A.gmres(P, f_dev[b], u_dev[b], tol=1e-8, restart=args.restart, stream=comp_s.cuda_stream)
        solved[b].record(comp_s)
        down_s.wait_event(solved[b])
        with torch.cuda.stream(down_s):
            u_host[b].copy_(u_dev[b], non_blocking=True)
        d2h[b].record(down_s)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    u_ref = u.cpu()
    e2e_dev = float(torch.linalg.norm(u_host[(args.steps - 1) % 2] - u_ref) / torch.linalg.norm(u_ref))
    e2e = {"value": N * args.steps * world / e2e_s, "unit": UNIT,
           "overlap": "uploads and downloads on two more streams, overlapping the solves",
           "rel_diff_vs_device_run": e2e_dev,
           "h2d_bytes_per_step": int(f_np.nbytes), "d2h_bytes_per_step": int(f_np.nbytes)}
    # the solve against the exact solution of the manufactured problem (untimed)
    solution = l2_error_sine(cfg, M, Mt, u)
    solution["u"] = "sin(pi x) sin(pi y) sin(pi z) sin(t)"

    # ---- fd_apply and st_matvec alone (CUDA events on the launching stream)
    r = torch.from_numpy(inputs.standard_normal(N, cfg["rhs_seed"])).cuda()
    s = torch.empty_like(r)
    y = torch.empty_like(r)
    for _ in range(3):
        P.apply(r, s)
        A.matvec(s, y)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        P.apply(r, s)
    e1.record(stream)
    torch.cuda.synchronize()
    fd_ms = e0.elapsed_time(e1) / args.steps
    e0.record(stream)
    for _ in range(args.steps):
        A.matvec(s, y)
    e1.record(stream)
    torch.cuda.synchronize()
    mv_ms = e0.elapsed_time(e1) / args.steps
    resid = float(torch.linalg.norm(y - r) / torch.linalg.norm(r))

    # ---- preconditioner variants inside the same FP64 flexible GMRES
    variants = {}
    A64 = stfd.KronOp(K, M, Wt, Mt, cfg["gamma"], cfg["nu"], arith=stfd.STFD_OP_FP64)
    Adf = stfd.KronOp(K, M, Wt, Mt, cfg["gamma"], cfg["nu"], arith=stfd.STFD_OP_DF32)
    vlist = [("fp64_ieee", stfd.STFD_FP64, A64), ("fp64tc7_fx64mv", stfd.STFD_FP64TC7, A),
             ("fp64tc7_fp64mv", stfd.STFD_FP64TC7, A64)]
    vlist += [("fp64tc48_df32mv", stfd.STFD_FP64TC, Adf), ("df32_df32mv", stfd.STFD_DF32, Adf),
              ("tf32", stfd.STFD_TF32, A64), ("bf16", stfd.STFD_BF16, A64)]
    for name, prec, op in vlist:
        Pv = P if prec == head_prec else stfd.FD(K, M, Wt, Mt, cfg["gamma"], cfg["nu"], precision=prec)
        # the matvec of this variant alone, on the same input (CUDA events)
        for _ in range(3):
            Pv.apply(r, s)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            Pv.apply(r, s)
        e1.record(stream)
        torch.cuda.synchronize()
        v_fd = e0.elapsed_time(e1) / args.steps
        s_v = s.clone()
        for _ in range(args.warmup):
            op.gmres(Pv, f, u, tol=1e-8, restart=args.restart)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            _, vinfo = op.gmres(Pv, f, u, tol=1e-8, restart=args.restart)
        e1.record(stream)
        torch.cuda.synchronize()
        v_gm = e0.elapsed_time(e1) / args.steps
        variants[name] = {"precond": name,
                          "matvec": "fp64_ieee" if op is A64 else "fx64 (exact integer limbs)" if op is A else "df32 (2 x FP32, ~48-bit)",
                          "fd_apply_ms": v_fd, "fd_apply_dofs_per_s": N / (v_fd * 1e-3), "gmres_ms": v_gm,
                          "gmres_iters": vinfo["iters"], "rel_res_true": vinfo["rel_res_true"], "_s": s_v}
        if Pv is not P:
            Pv.close()
    A64.close()
    Adf.close()
    ref_s = variants["fp64_ieee"]["_s"]
    for name in variants:
        sv = variants[name].pop("_s")
        variants[name]["fd_apply_rel_err_vs_fp64"] = float(torch.linalg.norm(sv - ref_s) / torch.linalg.norm(ref_s))
    if stfd.load().stfd_device_status() != 0:
        raise RuntimeError("a tensor-core kernel reported a timed-out wait")

    # ---- roofline of the dominant kernel: per-launch CUDA events inside the library
    stfd.stfd_profile_reset()
    stfd.stfd_profile_enable(True)
    for _ in range(args.steps):
        solve()
    torch.cuda.synchronize()
    stfd.stfd_profile_enable(False)
    recs = stfd.stfd_profile_records()
    stfd.stfd_profile_reset()
    total_ms = sum(rc["ms"] for rc in recs) or 1.0
    top = max(recs, key=lambda rc: rc["ms"])
    probe = stfd.stfd_probe_fp64_peak()
    imad_probe = stfd.stfd_probe_imad_wide_peak()
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    mhz = clocks.get("sm_mhz") or 2070.0
    per_launch_s = top["ms"] * 1e-3 / top["launches"]
    achieved = top["flops"] / top["launches"] / per_launch_s
    traffic = NCU_TRAFFIC.get(top["name"])
    peaks, peak_src = measured_peaks()
    common = {"kernel": top["name"], "traffic": traffic, "share_of_step": top["ms"] / total_ms,
              "achieved_gbs": top["bytes"] / top["launches"] / per_launch_s / 1e9,
              "fp64_equivalent_tflops": achieved / 1e12, "fp64_probe_tflops": probe / 1e12,
              "imad_wide_probe_tops": imad_probe / 1e12}
    if top["name"] == "fd_mode_tc7":
        # the issued BF16 MMA work: 28 digit pairs on M = 128 x N = npad x K = npad per 128-row
        # tile slot (R of the rows valid) -- see tc_oz7.cu; peak: measured BF16 GEMM, sustained
        # (the kernel runs inside a seconds-long loop of solves)
        n_t = inputs.sizes(cfg)[1]
        npad = (n_t + 15) // 16 * 16
        R = 128 if n_t <= 64 else 112
        mma_flops_per_row = 28.0 * 2.0 * npad * npad * 128.0 / R
        rows = N / n_t          # rows of one mode product (the same for every mode at this workload)
        tflops = mma_flops_per_row * rows / per_launch_s / 1e12
        peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0))
        roofline = dict(bound="tensor", achieved=tflops, peak=peak, unit="TFLOP/s", frac=tflops / peak,
                        peak_source="BF16 dense GEMM, sustained (MEASURED_PEAKS.json, %s)" % peak_src,
                        achieved_definition="issued BF16 MMA flops of the 28 digit pairs / CUDA-event time",
                        **common)
    elif top["name"] == "band_fx64":
        # three 32 x 32 -> 64-bit multiply-adds per exact tap product; peak = the probe above
        taps = 0.0
        for l in range(cfg["d"] + 1):
            taps += {0: 2, cfg["d"]: 2}.get(l, 3) * (2 * cfg["p"] + 1)
        ops_per_launch = 3.0 * taps * N / (cfg["d"] + 1)     # mean over the d + 1 passes of one matvec
        tops = ops_per_launch / per_launch_s / 1e12
        roofline = dict(bound="alu", achieved=tops, peak=imad_probe / 1e12, unit="Tops/s (mad.wide.s32)",
                        frac=tops * 1e12 / imad_probe,
                        peak_source="32 x 32 -> 64-bit multiply-add throughput probed in this run",
                        achieved_definition="3 multiply-adds per exact tap product x taps of the pass / time",
                        **common)
    elif top["name"].endswith("_df"):
        # double-float kernels issue 12 FP32 instructions per FP64-equivalent FMA
        # (2 flop): peak = 128 FP32 lanes x SMs x clock x 2 / 12
        peak = 128 * sms * mhz * 1e6 * 2 / 12
        roofline = dict(bound="alu", achieved=achieved / 1e12, peak=peak / 1e12, unit="TFLOP/s", frac=achieved / peak,
                        peak_source="FP32 pipes: 128 lanes/SM x %d SMs x %.0f MHz / 12 FP32 ops per double-float FMA"
                        % (sms, mhz), **common)
    else:
        peak = 2 * 2 * sms * mhz * 1e6
        roofline = dict(bound="alu", achieved=achieved / 1e12, peak=peak / 1e12, unit="TFLOP/s", frac=achieved / peak,
                        peak_source="FP64: 2 DFMA/clk/SM x %d SMs x %.0f MHz (sampled)" % (sms, mhz), **common)
    # per kernel family: time share and the achieved rates of its algorithmic work
    # (FP64-equivalent flops, minimum HBM bytes: each input read once, each output written once)
    kernels = {rc["name"]: {"launches": rc["launches"], "ms": round(rc["ms"], 3),
                            "share": round(rc["ms"] / total_ms, 4),
                            "fp64_eq_tflops": round(rc["flops"] / (rc["ms"] * 1e-3) / 1e12, 3) if rc["ms"] > 0 else None,
                            "algorithmic_gbs": round(rc["bytes"] / (rc["ms"] * 1e-3) / 1e9, 1) if rc["ms"] > 0 else None}
               for rc in recs}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": HEADLINE["dtype"], "data": "synthetic",
        "config": {"workload": cfg["name"], "N": N, "solve": "FD-preconditioned flexible GMRES to 1e-8, x0 = 0",
                   "restart": args.restart, "gmres_iters": infos[-1]["iters"],
                   "rel_res_true": infos[-1]["rel_res_true"],
                   "precond": HEADLINE["precond_text"], "matvec": HEADLINE["matvec_text"],
                   "gmres": "FP64 (CGS2, residuals, norms)",
                   "setup_ms": setup_ms,
                   "l2": "inputs larger than L2 (working set %.2f GB > 129 MB)" % (10 * N * 8 / 1e9),
                   "parallelism": "replicas x%d" % world},
        "solution_vs_exact": solution,
        "fd_apply": {"ms": fd_ms, "dofs_per_s": N / (fd_ms * 1e-3)},
        "st_matvec": {"ms": mv_ms, "dofs_per_s": N / (mv_ms * 1e-3), "residual_A_Pinv_r": resid},
        "gmres_time_to_1e-8_ms": ms / args.steps,
        "precond_variants": variants,
        "roofline": roofline, "kernels": kernels, "gpu_launches": launches,
        "clocks": clocks, "e2e": e2e,
    }
    peaks, src = measured_peaks()
    line["hbm_peak_gbs"] = {"value": peaks.get("hbm_gbs"), "source": src}
    A.close()
    P.close()
    torch.cuda.empty_cache()
    # the other workloads are reported once, at N = 1 (replicas add nothing to them)
    if world == 1 and not args.no_batch:
        line["batched"] = batch_section(args, stream)
    if world == 1 and not args.no_adjoint:
        line["adjoint"] = adjoint_section(args, stream)
    if world == 1 and not args.no_mapped:
        line["mapped_mixed_precision"] = mapped_section(args, stream)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        secs, _, iters, Nc, res = run_oracle_solve(cfg)
        line["cpu_baseline"] = {"value": Nc / secs, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                                "sample": "one full oracle solve of the same workload (setup excluded), "
                                          "%d GMRES iteration(s), %.1f s" % (iters, secs)}
        # the paper's setting is serial: the same solve with one BLAS thread, in a child
        # process (the thread count is fixed when numpy loads)
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
        try:
            out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-once"], env=env,
                                 capture_output=True, text=True, timeout=600)
            one = json.loads(out.stdout.strip().splitlines()[-1])
            line["cpu_baseline"]["single_thread_value"] = one["value"]
            line["cpu_baseline"]["single_thread_sample"] = "the same solve, 1 BLAS thread (%.1f s)" % one["seconds"]
        except (subprocess.SubprocessError, ValueError, IndexError, KeyError):
            line["cpu_baseline"]["single_thread_value"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
