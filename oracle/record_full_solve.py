"""Record one complete oracle solve of the CI-like benchmark workload.

TEST INFRASTRUCTURE: calls only the CPU oracle (and the seeded input generator).  The
benchmark's CPU legs cannot afford a complete oracle solve of the n = 2,000,000 workload
(the FP64 method needs over a thousand iterations there), so they time a short sample and
scale this record: its wall time, iteration count, threads, and the per-iteration time of
its first iterations measured the same way as the sample.

    python -m oracle.record_full_solve [--n 2000000] [--out oracle/records/ci2m_seed0.json]
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

K, EXTRA, TOL, SEED = 16, 5, 1e-8, 0


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=2_000_000)
    ap.add_argument("--out", default=os.path.join(ROOT, "oracle", "records", "ci2m_seed0.json"))
    ap.add_argument("--maxiter", type=int, default=6000)
    args = ap.parse_args()
    a = synth.sparse_ci(n=args.n, seed=SEED)
    x0 = synth.diag_guess(a.diag, K + EXTRA, seed=SEED, noise=0.0)
    oracle.lib()
    t0 = time.perf_counter()
    oracle.lobpcg(a, a.diag, K, x0, extra=EXTRA, tol=TOL, maxiter=0, hist_cap=2)
    t1 = time.perf_counter()
    oracle.lobpcg(a, a.diag, K, x0, extra=EXTRA, tol=TOL, maxiter=2, hist_cap=4)
    t2 = time.perf_counter()
    init = t1 - t0
    per_it = max((t2 - t1) - init, 1e-9) / 2.0
    t3 = time.perf_counter()
    r = oracle.lobpcg(a, a.diag, K, x0, extra=EXTRA, tol=TOL, maxiter=args.maxiter)
    seconds = time.perf_counter() - t3
    rec = {"workload": f"CI-like n={args.n}, seed {SEED}, k={K} (+{EXTRA} extra), tol {TOL}",
           "status": int(r.status), "iterations": int(r.info["iterations"]), "seconds": seconds,
           "threads": oracle.threads(), "cpu": cpu_model(), "init_seconds": init,
           "per_iteration_seconds": per_it, "evals": [float(v) for v in r.evals],
           "max_resnorm": float(max(r.resnorms)), "active_per_iteration": [int(v) for v in r.hist_mact],
           "command": "python -m oracle.record_full_solve --n %d" % args.n}
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    with open(args.out, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps({k: v for k, v in rec.items() if k not in ("evals", "active_per_iteration")}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
