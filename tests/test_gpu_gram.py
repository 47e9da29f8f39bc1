"""GPU parity of the tensor-core Gram blocks G_ij = M_i^T M_j.

Two references from the oracle's FP64 matrix M (never from the GPU):
* G_bf = bf16(M)^T bf16(M) in FP64 (M rounded to BF16 by torch): the
  tensor cores multiply these BF16 values and accumulate in FP32; the GPU
  rounds its own FP32 entries, so an entry next to a rounding boundary can
  land one BF16 ulp away from the oracle's rounding.  Bound used:
  |G - G_bf| <= 2^-9 |M|^T|M|, a quarter of the worst-case rounding bound
  below (an operand layout error would show as O(1));
* G = M^T M in FP64: |G_gpu - G| <= (2 u_bf16 + u_bf16^2) |M|^T|M| + FP32
  accumulation, u_bf16 = 2^-8 (the worst-case rounding bound).
"""
import numpy as np
import pytest

import paper_2409_01949_gb300 as E
import workloads as WL
from oracle import system as OS

pytestmark = pytest.mark.gpu

CASES = {
    "poisson2d_L1-4_K64": lambda: WL.poisson2d(levels=(1, 2, 4), features=64, n_side=40,
                                               n_boundary_side=40),
    "poisson2d_L1-2_K128": lambda: WL.poisson2d(levels=(1, 2), features=128, n_side=24,
                                                n_boundary_side=12),
    "dho_L1-8_K24": lambda: WL.dho(levels=(1, 2, 4, 8), features=24, n_interior=700),
    "poisson2d_delta2.9_K40": lambda: WL.poisson2d(levels=(2, 3), features=40, n_side=30,
                                                   n_boundary_side=10, delta=2.9),
}


def _bf16(A):
    torch = pytest.importorskip("torch")
    return torch.from_numpy(A.astype(np.float32)).bfloat16().double().numpy()


@pytest.mark.parametrize("name", list(CASES))
def test_gram_blocks_match_oracle(name):
    P = CASES[name]()
    K = P.features
    ref = OS.assemble(P, fmt="dense")
    M = ref["M"]
    Mb = _bf16(M)
    A = np.abs(M)
    nsub = P.n_subdomains
    # structural pairs from the oracle: blocks of M^T M with a shared row
    nzb = (np.abs(M).reshape(M.shape[0], nsub, K).max(axis=2) > 0)
    share = (nzb.T.astype(np.int64) @ nzb.astype(np.int64)) > 0
    pairs = [(i, j) for i in range(nsub) for j in range(i, nsub) if share[i, j]]
    with E.Solver.from_problem(P, precision=E.MIXED) as s:
        s.assemble_problem(P)
        s.compute_gram()
        sz = s.sizes()
        got = s.gram_blocks(pairs)
    assert sz.n_gram_pairs >= len(pairs)
    worst_bf, worst_ex = 0.0, 0.0
    for q, (i, j) in enumerate(pairs):
        bi, bj = slice(i * K, (i + 1) * K), slice(j * K, (j + 1) * K)
        Gabs = A[:, bi].T @ A[:, bj]
        Gbf = Mb[:, bi].T @ Mb[:, bj]
        Gex = M[:, bi].T @ M[:, bj]
        sc = np.maximum(Gabs, 1e-300)
        worst_bf = max(worst_bf, float((np.abs(got[q] - Gbf) / sc).max()))
        worst_ex = max(worst_ex, float((np.abs(got[q] - Gex) / sc).max()))
    print(f"{name}: {len(pairs)} pairs, max |G-G_bf16|/|M|^T|M| = {worst_bf:.2e}, "
          f"max |G-G|/|M|^T|M| = {worst_ex:.2e}")
    assert worst_bf <= 2.0 ** -9
    assert worst_ex <= 2 * 2.0 ** -8 + 2.0 ** -16 + 1e-4


def test_gram_unsupported_outside_mixed_precision():
    P = WL.poisson1d(levels=(2,), features=8, n_interior=20)
    with E.Solver.from_problem(P, precision=E.FP32) as s:
        s.assemble_problem(P)
        with pytest.raises(E.ElmfbError) as ei:
            s.compute_gram()
        assert ei.value.code == E.ERR_UNSUPPORTED
