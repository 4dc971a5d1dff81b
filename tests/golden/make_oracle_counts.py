"""Write oracle_counts.json: FGMRES(50) iteration counts and final relative
residuals of the FP64 oracle on the full-size synthetic workloads.

Calls only the oracle and the seeded input generators (no GPU code).  The
stored counts pin the CUDA path at full size (iterations within +-1) and
scale the oracle's timed CPU sample in bench.py.
Run:  PYTHONPATH=. python tests/golden/make_oracle_counts.py [workload | workload/precond ...]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import amg, krylov, precond  # noqa: E402
from oracle.cycles import SmootherParams  # noqa: E402
from paper_1605_01522_gb300 import inputs  # noqa: E402

# workload name -> (generator, solver parameters)
WORKLOADS = {
    "coupled_box_3d_ne64_f3": (lambda: inputs.coupled_box_3d(ne=64, nfields=3, seed=1),
                               dict(max_levels=5, coarse_max=1000),
                               {"bgs_amg": {}, "amg_bgs": {}, "simple": {}, "amg_simple": {},
                                "bgs_amg+gs": dict(smoother="gs")}),
    # labels "<precond>+<option>" select SIMPLE's predictor solver or the smoother
    "constrained_box_ne64_f3_m4": (lambda: inputs.constrained_box(ne=64, nfields=3, seed=5),
                                   dict(max_levels=5, coarse_max=1000),
                                   {"simple": {}, "simple+amg_bgs": dict(simple_pred="amg_bgs")}),
    # the split box with an Oseen velocity block (wind 0.2, 0.1, 0); its velocity
    # field takes Petrov-Galerkin transfers ("+sa": P^T restriction instead)
    "oseen_fsi_box_ne48": (lambda: inputs.fsi_box(ne=48, seed=2, wind=(0.2, 0.1, 0.0)),
                           dict(max_levels=5, coarse_max=1000),
                           {"simple": dict(simple_group=[0, 0, 0, 1], simple_approx="diag"),
                            "simple+sa": dict(simple_group=[0, 0, 0, 1], simple_approx="diag", pg_off=True)}),
    # config 2 at 64^3 (1,394,250 dofs) and config 0 (the 3,267-dof 2D system, 3 levels)
    "fsi_box_ne64": (lambda: inputs.fsi_box(ne=64, seed=2), dict(max_levels=5, coarse_max=1000),
                     {"simple": dict(simple_group=[0, 0, 0, 1], simple_approx="diag")}),
    "thermo_elastic_2d_ne32": (lambda: inputs.thermo_elastic_2d(ne=32, seed=0), dict(max_levels=3, coarse_max=0),
                               {"bgs_amg": {}, "amg_bgs": {}, "simple": {}}),
    "fsi_box_ne48": (lambda: inputs.fsi_box(ne=48, seed=2), dict(max_levels=5, coarse_max=1000),
                     {"bgs_amg": {}, "simple": dict(simple_group=[0, 0, 0, 1], simple_approx="diag"),
                      "amg_simple": dict(simple_group=[0, 0, 0, 1], simple_approx="diag")}),
}


def main():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_counts.json")
    only = sys.argv[1:]
    out = {}
    if os.path.exists(path):
        with open(path) as f:
            out = json.load(f)
    for name, (gen, kw, pcs) in WORKLOADS.items():
        pick = [pc for pc in pcs if not only or name in only or f"{name}/{pc}" in only]
        if not pick:
            continue
        s = gen()
        A = s.scipy_blocks()
        D = precond.assemble(A, s.nfields)
        specs = [amg.FieldSpec.of(f) for f in s.fields]
        for pc in pick:
            extra = pcs[pc]
            t0 = time.time()
            ex = dict(extra)
            sp_ = [amg.FieldSpec.of(f) for f in s.fields]
            if ex.pop("pg_off", False):
                for f in sp_:
                    f.pg = False
            if ex.pop("smoother", None) == "gs":
                ex["smoother"] = SmootherParams("gs", omega=0.79, sweeps=1)
            M = precond.Preconditioner(A, sp_, precond.Params(pc.split("+")[0], **kw, **ex))
            t1 = time.time()
            r = krylov.fgmres(lambda v: D @ v, M, s.rhs, 1e-8, 50, maxiter=400)
            t2 = time.time()
            out[f"{name}/{pc}"] = dict(iters=r.iters, relres=r.relres, converged=bool(r.converged),
                                       setup_s=round(t1 - t0, 2), solve_s=round(t2 - t1, 2), **kw, **extra)
            print(name, pc, out[f"{name}/{pc}"], flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
