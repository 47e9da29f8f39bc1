"""Write tests/golden/batch_errors.json: the FP64 oracle's errors on 16
instances of the uneven batched 2-D Poisson workload (seed-0 draw of 512).

Calls only ``oracle/`` and ``workloads``.  The instances span n_sub 2..32
subdomains per dimension, K in {32, 64, 128} and grid sides 64..511.  Per
instance the oracle solves by column-pivoted QR where the dense matrix has at
most 4096 columns and 3e8 entries (the least-squares minimiser; repeated on
one shuffled row order, the rounding spread), else by the paper's protocol
(SciPy LSQR from zero for 15000 iterations, §4.1), and stores the relative L2
error and e_L1 of u_hat against the closed-form solution.
Usage:  python tests/golden/make_batch_errors.py [index ...]
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

OUT = os.path.join(HERE, "batch_errors.json")
# QR-solved instances (<= 4096 columns), then paper-protocol ones
INSTANCES = [402, 17, 293, 67, 247, 173, 253, 114, 291, 400, 334, 61, 245, 286, 28, 130]


def run(index: int):
    spec = WL.batch_specs(512, 0)[index]
    P = WL.batch_instance(spec, index, 0)
    X, u = P.test_points, P.exact(P.test_points)
    rec = {"index": index, "n_sub": spec.n_sub, "features": spec.features,
           "n_side": spec.n_side, "k": spec.k, "n_rows": P.n_rows, "n_columns": P.n_columns}
    threads = os.cpu_count() or 1
    dense = P.n_columns <= 4096 and P.n_rows * P.n_columns <= 3e8
    t = time.time()
    out = OS.assemble(P, fmt="dense" if dense else "csr")
    M, h = out["M"], out["h"]
    if dense:
        a, rank = OL.lstsq_qr(M, h, threads=threads)
        uh = OE.u_hat(P, a, X)
        p = np.random.default_rng(0).permutation(M.shape[0])
        a2, rank2 = OL.lstsq_qr(M[p], h[p], threads=threads)
        e2 = OE.rel_l2(OE.u_hat(P, a2, X), u)
        rec["oracle"] = {"kind": "qr", "rel_l2": OE.rel_l2(uh, u), "e_l1": OE.e_l1(uh, u),
                         "rank": rank, "rel_l2_shuffled": e2, "rank_shuffled": rank2,
                         "rel_l2_max_over_orders": max(OE.rel_l2(uh, u), e2),
                         "seconds": time.time() - t}
    else:
        a, info = OL.lstsq_lsqr(M, h, iter_lim=15000, threads=threads)
        uh = OE.u_hat(P, a, X)
        rec["oracle"] = {"kind": "lsqr15000", "rel_l2": OE.rel_l2(uh, u), "e_l1": OE.e_l1(uh, u),
                         "iterations": info["itn"], "seconds": time.time() - t}
    return rec


def main(indices):
    for i in indices:
        print("oracle: batch instance", i, flush=True)
        rec = run(i)
        print(json.dumps(rec), flush=True)
        data = json.load(open(OUT)) if os.path.exists(OUT) else {}
        data[str(i)] = rec
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or INSTANCES)
