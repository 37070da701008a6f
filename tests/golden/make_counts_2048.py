"""Writes counts_2048.json: the CPU oracle's iteration counts and final
residuals for the benchmark workload (16 seeded 2048^2 fields, k^-3 spectrum
with k_p = 10 and exp(-(k/600)^2) cutoff, gamma = 0.01, tolerance 1e-6) with
BiCGSTAB and CG in float64 and float32-storage precision. Calls only the
oracle and the input generator. Takes about half an hour on 8 cores.

    python tests/golden/make_counts_2048.py [--workers 8]
"""

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

N, GAMMA, TOL, BATCH = 2048, 0.01, 1e-6, 16


def _one(job):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import numpy as np
    import oracle
    from synth import fields
    seed, method, precision = job
    spec = lambda k: fields.spectrum_2d_kraichnan(k, kp=10.0, kcut=600.0)
    u = fields.random_scalar_field((N, N), seed, spec)
    ub = oracle.filter_field(u, GAMMA).astype(np.float32).astype(np.float64)
    t = time.time()
    r = oracle.solve(method, ub, GAMMA, tol=TOL, maxit=3000, precision=precision)
    return dict(seed=seed, method=method, precision=precision, iterations=r.iterations, status=r.status,
                h_final=float(r.history[-1]), h_prev=float(r.history[-2]) if len(r.history) > 1 else None,
                true_residual=r.true_residual, seconds=time.time() - t)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "counts_2048.json"))
    a = ap.parse_args()
    jobs = [(s, m, p) for m in ("bicgstab", "cg") for p in ("f64", "f32") for s in range(BATCH)]
    with mp.get_context("spawn").Pool(a.workers) as pool:
        res = pool.map(_one, jobs, chunksize=1)
    doc = dict(source="CPU oracle (oracle/solvers.py) on synth fields; script tests/golden/make_counts_2048.py",
               workload=dict(n=N, batch=BATCH, gamma=GAMMA, tol=TOL, spectrum="k^-3, k_p=10, cutoff 600",
                             input="oracle filter of the seeded field, rounded to float32"),
               runs=res)
    with open(a.out, "w") as f:
        json.dump(doc, f, indent=1)


if __name__ == "__main__":
    main()
