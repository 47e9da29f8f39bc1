"""Write tests/golden/oracle_errors.json: the FP64 oracle's solution errors.

Calls only ``oracle/`` and ``workloads``.  For every listed workload it stores

* ``qr``   the least-squares minimiser by column-pivoted QR (rank cut 1e-13),
           where the dense matrix fits in memory;
* ``lsqr`` the paper's protocol (§4.1 "Optimisation and solvers"): SciPy LSQR
           from a = 0, run for the full 15000-iteration budget;

each with the relative L2 error and e_L1 of u_hat against the closed-form
solution on the workload's test points, the residual ||M a - h|| and the
wall time.  Usage:  python tests/golden/make_oracle_errors.py [name ...]
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as WL  # noqa: E402
from oracle import evaluate as OE  # noqa: E402
from oracle import lstsq as OL  # noqa: E402
from oracle import system as OS  # noqa: E402

OUT = os.path.join(HERE, "oracle_errors.json")

WORKLOADS = {
    "poisson1d_J16_K64_N2000": (WL.config_poisson1d, True),
    "dho_L1-8_K24_N1000": (lambda: WL.dho(levels=(1, 2, 4, 8), features=24, n_interior=1000), True),
    "poisson2d_L1-4_K64_N60": (lambda: WL.poisson2d(levels=(1, 2, 4), features=64, n_side=60,
                                                   n_boundary_side=60), True),
    "dho_L1-64_K96_N20000": (WL.config_dho_ml, True),
    "poisson2d_L1-16_K128_N400": (WL.config_poisson2d_ml, False),
}


def run(name):
    make, dense_ok = WORKLOADS[name]
    P = make()
    X = P.test_points
    u = P.exact(X)
    rec = {"name": name, "n_rows": P.n_rows, "n_columns": P.n_columns}
    t = time.time()
    out = OS.assemble(P, fmt="dense" if dense_ok else "csr")
    rec["assemble_s"] = time.time() - t
    M, h = out["M"], out["h"]
    if dense_ok:
        t = time.time()
        a, rank = OL.lstsq_qr(M, h)
        uh = OE.u_hat(P, a, X)
        rec["qr"] = {"rel_l2": OE.rel_l2(uh, u), "e_l1": OE.e_l1(uh, u), "rank": rank,
                     "residual": float(np.linalg.norm(M @ a - h)), "seconds": time.time() - t}
    t = time.time()
    a, info = OL.lstsq_lsqr(M, h, iter_lim=15000, threads=os.cpu_count() or 1)
    uh = OE.u_hat(P, a, X)
    rec["lsqr"] = {"rel_l2": OE.rel_l2(uh, u), "e_l1": OE.e_l1(uh, u), "iterations": info["itn"],
                   "residual": float(np.linalg.norm(M @ a - h)), "seconds": time.time() - t}
    return rec


def main(names):
    for n in names:
        print("oracle:", n, flush=True)
        rec = run(n)
        print(json.dumps(rec), flush=True)
        data = json.load(open(OUT)) if os.path.exists(OUT) else {}   # re-read: runs may overlap
        data[n] = rec
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS))
