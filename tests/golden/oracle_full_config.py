"""Record of the CPU oracle on the full benchmark workload.

Runs the oracle (oracle/air_oracle.c, one thread) on the 2D+time HDG trace
system of 48^3 cubes x 6 tetrahedra, p = 2, rotating velocity, nu = 1e-6
(7,934,976 unknowns): l-AIR setup with theta 0.25, distance 1, FCF-Jacobi,
then GMRES(30) to a relative residual of 1e-8.  It writes the level sizes,
the iteration count and the final residual to
oracle_st2d_n48_p2_nu1e-6.json beside this script, with the host's setup
and solve seconds as context.  The benchmark's CPU-baseline sample scales its
per-iteration cost by this iteration count; the GPU's count on the same
workload is compared with it (within one).

    python tests/golden/oracle_full_config.py [--workers 8]

Takes about ten minutes and 20 GB of host memory.
"""
import argparse
import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--n", type=int, default=48)
    args = ap.parse_args()
    import oracle
    from sthdg import assemble
    from sthdg.problems import manufactured_2d
    s = assemble(manufactured_2d(n=args.n, p=2, nu=1e-6), workers=args.workers)
    oracle.build()
    t0 = time.perf_counter()
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, distance=1, max_coarse=1000, copy_levels=False)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, iters, relres, ok, _ = oracle.gmres(s.row_ptr, s.col, s.val, H, s.rhs, rtol=1e-8, restart=30,
                                           max_iter=1000)
    t_solve = time.perf_counter() - t0
    rec = {"workload": f"st2d_hdg_n{args.n}_p2_rotating_nu1e-06", "unknowns": int(s.n), "nnz": int(s.nnz),
           "theta": 0.25, "distance": 1, "relax": "FCF", "restart": 30, "rtol": 1e-8,
           "levels": [list(x) for x in H.sizes()], "iters": int(iters), "relres": float(relres),
           "converged": bool(ok),
           "host": {"setup_s": t_setup, "solve_s": t_solve, "machine": platform.machine(),
                    "processor": platform.processor() or "unknown", "threads": 1}}
    out = os.path.join(HERE, f"oracle_st2d_n{args.n}_p2_nu1e-6.json")
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
