"""Write tests/golden/oracle_errors.json: the FP64 oracle's solution errors.

Calls only ``oracle/`` and ``workloads``.  For every listed workload it stores

* ``qr``   the least-squares minimiser by the oracle's own column-pivoted
           Householder QR (rank cut 1e-13), where the dense matrix fits in
           memory;
* ``lsqr`` the paper's protocol (§4.1 "Optimisation and solvers"): SciPy LSQR
           from a = 0, run for the full 15000-iteration budget;

each with the relative L2 error and e_L1 of u_hat against the closed-form
solution on the workload's test points, the residual ||M a - h|| and the
wall time.  The QR entry also holds ``orders``: the same QR solve repeated on
copies of the system whose rows are shuffled (seeded).  A row order changes
no least-squares minimiser, only the rounding, so the spread of these errors
is the part of the QR error that FP64 rounding alone decides; a solver that
orders its rows otherwise (the GPU sorts them by cell) is held to 1.01x the
largest of them.  Usage:
    python tests/golden/make_oracle_errors.py [--only qr|lsqr] [name ...]
``--only`` recomputes one of the two entries and keeps the other.
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
from oracle import decomposition as OD  # noqa: E402
from oracle import evaluate as OE  # noqa: E402
from oracle import lstsq as OL  # noqa: E402
from oracle import system as OS  # noqa: E402

OUT = os.path.join(HERE, "oracle_errors.json")
N_ORDERS = 3   # shuffled row orders per QR entry
N_ORDERS_OF = {"dho_L1-64_K96_N20000": 2}   # 15 minutes per QR on 8 cores

WORKLOADS = {
    "poisson1d_J16_K64_N2000": (WL.config_poisson1d, True),
    "dho_L1-8_K24_N1000": (lambda: WL.dho(levels=(1, 2, 4, 8), features=24, n_interior=1000), True),
    "poisson2d_L1-4_K64_N60": (lambda: WL.poisson2d(levels=(1, 2, 4), features=64, n_side=60,
                                                   n_boundary_side=60), True),
    "dho_L1-64_K96_N20000": (WL.config_dho_ml, True),
    "poisson2d_L1-16_K128_N400": (WL.config_poisson2d_ml, False),
    # §4.4 baseline: Helmholtz on the L-shaped domain, 16^2 - 8^2 subdomains
    "helmholtz_L_w8_J16_K16": (WL.helmholtz_lshape, True),
    # §4.3 baseline: multi-scale Laplace with the hard-constraint ansatz
    "laplace_n4_J16_K16": (WL.laplace_multiscale, True),
}


def run(name, only=None, old=None):
    make, dense_ok = WORKLOADS[name]
    P = make()
    X = P.test_points
    u = P.exact(X)
    rec = dict(old or {})
    rec.update({"name": name, "n_rows": P.n_rows, "n_columns": OD.n_columns(P)})
    t = time.time()
    out = OS.assemble(P, fmt="dense" if dense_ok else "csr")
    rec["assemble_s"] = time.time() - t
    M, h = out["M"], out["h"]
    threads = os.cpu_count() or 1
    if dense_ok and only in (None, "qr"):
        t = time.time()
        a, rank = OL.lstsq_qr(M, h, threads=threads)
        uh = OE.u_hat(P, a, X)
        rec["qr"] = {"rel_l2": OE.rel_l2(uh, u), "e_l1": OE.e_l1(uh, u), "rank": rank,
                     "residual": float(np.linalg.norm(M @ a - h)), "seconds": time.time() - t}
        orders = []
        for seed in range(N_ORDERS_OF.get(name, N_ORDERS)):
            p = np.random.default_rng(seed).permutation(M.shape[0])
            ap, rp = OL.lstsq_qr(M[p], h[p], threads=threads)
            uhp = OE.u_hat(P, ap, X)
            orders.append({"seed": seed, "rel_l2": OE.rel_l2(uhp, u), "rank": rp,
                           "residual": float(np.linalg.norm(M @ ap - h))})
        rec["qr"]["orders"] = orders
        errs = [rec["qr"]["rel_l2"]] + [o["rel_l2"] for o in orders]
        rec["qr"]["rel_l2_max_over_orders"] = max(errs)
    if only == "qr":
        return rec
    t = time.time()
    a, info = OL.lstsq_lsqr(M, h, iter_lim=15000, threads=threads)
    uh = OE.u_hat(P, a, X)
    rec["lsqr"] = {"rel_l2": OE.rel_l2(uh, u), "e_l1": OE.e_l1(uh, u), "iterations": info["itn"],
                   "residual": float(np.linalg.norm(M @ a - h)), "seconds": time.time() - t}
    return rec


def main(names, only=None):
    for n in names:
        print("oracle:", n, flush=True)
        old = json.load(open(OUT)).get(n) if os.path.exists(OUT) else None
        rec = run(n, only, old)
        print(json.dumps(rec), flush=True)
        data = json.load(open(OUT)) if os.path.exists(OUT) else {}   # re-read: runs may overlap
        data[n] = rec
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    args = sys.argv[1:]
    only = None
    if args[:1] == ["--only"]:
        only, args = args[1], args[2:]
    main(args or list(WORKLOADS), only)
