"""Small fixed workloads for Nsight Compute captures of one kernel family.

  python -m paper_1909_07309_gb300.ncu_case {fd,matvec,solve} D P N_EL [REPS] [fp64|df32|fp64tc|tf32|bf16|fp64tc7|fx64]
  python -m paper_1909_07309_gb300.ncu_case {stencil,mapped_solve} D P N_EL [REPS] [fp64|df32|tf32|bf16|fx64]
  python -m paper_1909_07309_gb300.ncu_case batch COUNT [REPS] [df32|fp64]

Builds the unit-cube problem (d = D, degree P, N_EL elements per direction),
runs one warm-up and REPS applications of fd_apply, st_matvec or the
preconditioned GMRES solve, synchronises and exits. `fp64tc7` is the
seven-digit tensor-core preconditioner with the FP64 matvec, `fx64` the same
preconditioner with the integer-limb matvec (the bench headline). `stencil` and
`mapped_solve` use the quarter-annulus problem with variable coefficients
(stencil matvec; GMRES with the geometry-aware preconditioner; `fx64` there is
the integer-limb stencil matvec with the IEEE-FP64 preconditioner). `batch` runs
the batched solver on the first COUNT problems of the batched workload
(256 threads x 2 CTAs per SM, no autotuning): double-float, one step, or
IEEE FP64 refined to 1e-8 (at most 5 steps).
"""
import sys


def main(argv):
    import torch

    from . import inputs, stfd
    if argv[0] == "batch":
        count = int(argv[1])
        reps = int(argv[2]) if len(argv) > 2 else 2
        fp64 = len(argv) > 3 and argv[3] == "fp64"
        cfg = dict(inputs.BATCH)
        n_el, p, nrhs, g = inputs.batch_draws(cfg)
        kw = dict(precision=stfd.STFD_FP64, tol=1e-8, max_it=5) if fp64 else {}
        B = stfd.Batch(n_el[:count], p[:count], nrhs[:count], d=cfg["d"], autotune=False, **kw)
        f = torch.from_numpy(g.standard_normal(B.total)).cuda()
        for _ in range(1 + reps):
            B.solve(f)
        torch.cuda.synchronize()
        print("ncu_case batch count=%d dofs=%d reps=%d %s ok" % (count, B.total, reps, "fp64" if fp64 else "df32"))
        return
    what, d, p, n_el = argv[0], int(argv[1]), int(argv[2]), int(argv[3])
    reps = int(argv[4]) if len(argv) > 4 else 2
    arith = argv[5] if len(argv) > 5 else "fp64"
    prec = {"fp64": stfd.STFD_FP64, "df32": stfd.STFD_DF32, "fp64tc": stfd.STFD_FP64TC,
            "tf32": stfd.STFD_TF32, "bf16": stfd.STFD_BF16, "fp64tc7": stfd.STFD_FP64TC7,
            "fx64": stfd.STFD_FP64TC7}[arith]
    mv = {"fp64": stfd.STFD_OP_FP64, "fp64tc7": stfd.STFD_OP_FP64, "fx64": stfd.STFD_OP_FX64}.get(arith, stfd.STFD_OP_DF32)
    if what in ("stencil", "mapped_solve"):
        prob = stfd.mapped_problem(d, p, n_el, stfd.STFD_GEOM_QUARTER_ANNULUS, c=inputs.c_bilinear,
                                   kappa=inputs.kappa_trig)
        A = stfd.StencilOp(prob["n"], p, prob["Ms"], prob["Ks"], prob["Wt"], prob["Mt"],
                           arith={"fp64": stfd.STFD_OP_FP64, "fx64": stfd.STFD_OP_FX64}.get(arith, stfd.STFD_OP_DF32))
        gp = {stfd.STFD_FP64TC: stfd.STFD_DF32, stfd.STFD_FP64TC7: stfd.STFD_FP64}.get(prec, prec)
        P = stfd.geometry_preconditioner(prob, precision=gp)
        r = torch.from_numpy(inputs.standard_normal(A.N, 1)).cuda()
        out = torch.empty_like(r)
        for _ in range(1 + reps):
            if what == "stencil":
                A.matvec(r, out)
            else:
                A.gmres(P, r, out)
        torch.cuda.synchronize()
        print("ncu_case %s d=%d p=%d n_el=%d N=%d reps=%d ok" % (what, d, p, n_el, A.N, reps))
        return
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el)
    P = stfd.FD(K, M, Wt, Mt, precision=prec)
    A = stfd.KronOp(K, M, Wt, Mt, arith=mv)
    r = torch.from_numpy(inputs.standard_normal(P.N, 1)).cuda()
    out = torch.empty_like(r)
    for _ in range(1 + reps):
        if what == "fd":
            P.apply(r, out)
        elif what == "matvec":
            A.matvec(r, out)
        elif what == "solve":
            A.gmres(P, r, out)
        else:
            raise SystemExit("unknown case %s" % what)
    torch.cuda.synchronize()
    print("ncu_case %s d=%d p=%d n_el=%d N=%d reps=%d ok" % (what, d, p, n_el, P.N, reps))


if __name__ == "__main__":
    main(sys.argv[1:])
