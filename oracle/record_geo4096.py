"""Run the CPU oracle once, in full, on the n = 4096 benchmark matrix and
record what it did (test infrastructure: calls only ``oracle`` and the seeded
input generators).

    python oracle/record_geo4096.py mixed|plain [out.json] [clustered1024]

(the optional third argument records the n = 1024 clustered case instead)

The mixed run is Algorithm 9 as the oracle implements it (FP32 cyclic-by-row
Jacobi, two Newton-Schulz steps, Q_d^T A Q_d, FP64 cyclic-by-row Jacobi, Q_d V);
the plain run is the FP64 cyclic-by-row Jacobi from V = I.  Each takes hours on
one core.  The record holds the sweep and rotation counts (deterministic: plain
C without contraction, so the same on any IEEE machine), the wall time and the
machine it ran on, and the accuracy of the result against the constructed
spectrum.  The benchmark's CPU baseline uses the counts; its timings are taken
on the machine it runs on.
"""
from __future__ import annotations

import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2509_00495_gb300 import inputs  # noqa: E402


def main() -> None:
    which = sys.argv[1]
    workload = sys.argv[3] if len(sys.argv) > 3 else "geo4096"
    out = sys.argv[2] if len(sys.argv) > 2 else os.path.join(HERE, f"{workload}_{which}.json")
    if workload == "clustered1024":
        A, lam = inputs.clustered_1024(seed=0)
        desc = "clustered1024 (n=1024, 992 eigenvalues linear in [-1,1] + 32 within 1e-8 of 0.5, seed 0)"
    else:
        A, lam = inputs.geo_4096(seed=0)
        desc = "geo4096 (n=4096, |lam| geometric in [1e-6,1], random signs, Haar eigenvectors, seed 0)"
    n = A.shape[0]
    t0 = time.perf_counter()
    if which == "mixed":
        W, Q, info = oracle.syev_mixed(A)
    elif which == "plain":
        W, Q, info = oracle.syev_plain(A)
    else:
        raise SystemExit("mixed or plain")
    wall = time.perf_counter() - t0
    u = 2.0 ** -53
    be = np.linalg.norm(A - (Q * W) @ Q.T) / np.linalg.norm(A)
    orth = np.linalg.norm(Q.T @ Q - np.eye(n))
    rec = {
        "workload": desc,
        "method": which, "orderings": "cyclic-by-row (FP32 and FP64)", "tol": "n 2^-53 ||A||_F",
        "sweeps32": info.sweeps32, "sweeps64": info.sweeps64, "rotations32": info.rotations32,
        "rotations64": info.rotations64, "capped64": info.capped64, "off_cond": info.off_cond,
        "off_final": info.off_final, "wall_seconds": wall, "cores": 1,
        "machine": f"{platform.machine()} {platform.processor() or ''}".strip(),
        "eig_err_over_normA": float(np.abs(W - np.sort(lam)).max() / np.abs(lam).max()),
        "backward_err_over_nu": float(be / (n * u)), "orth_fro_over_nu": float(orth / (n * u)),
    }
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
