"""Graph network of the learned preconditioner (oracle side; not in the paper).

The GPU library learns a correction to its block-Jacobi preconditioner with a
message-passing network over the subdomain graph (nodes = subdomains, edges =
subdomain pairs whose supports share collocation points).  This module is the
plain FP64 definition of that network, used to check the GPU forward pass and
its hand-written gradients.

Network (per sample b, node s; H hidden channels, K features per subdomain):
    A0[s]  = relu(W_in X[s] + b_in)
    for l = 1, 2, 3:
        agg[s] = mean_{t in N(s)} A_{l-1}[t]          (N(s): neighbours, s excluded)
        A_l[s] = relu(W_self_l A_{l-1}[s] + W_nb_l agg[s] + b_l)
    Y[s]   = W_out A3[s] + b_out
Loss: L = (1/B) sum_b w_b sum_s ||Y_b[s] - T_b[s]||^2.

Weight vector layout (the C ABI's): W_in (H x K), b_in (H), then for l = 1..3
W_self_l (H x H), W_nb_l (H x H), b_l (H), then W_out (K x H), b_out (K), all
row-major.

forward_bf16 is the same network with every layer's operands rounded to
bfloat16 where the GPU's tensor-core inference rounds them (the neighbour
mean formed in FP32 first); bf16_round is pinned by round-half-even cases
worked out by hand, forward_bf16 by the hand-computed case below (every
value there is exact in bfloat16) and by inputs, weights and activations
whose rounding that case exposes.

Pinned in tests/test_oracle_gnn.py by a forward pass computed by hand on a
3-node path with distinct inputs and integer weights (a swap of W_self and
W_nb, a sum in place of the mean or a dropped ReLU each change it), by the
zero-weight and equal-input special cases, and by central finite differences
of the loss.  The paper defines no such network, so nothing it prints pins it.
"""
from __future__ import annotations

import numpy as np

N_LAYERS = 3


def n_weights(K: int, H: int = 64) -> int:
    return H * K + H + N_LAYERS * (2 * H * H + H) + K * H + K


def unpack(w: np.ndarray, K: int, H: int = 64):
    w = np.asarray(w, dtype=np.float64)
    o = 0

    def take(n, shape):
        nonlocal o
        v = w[o:o + n].reshape(shape)
        o += n
        return v
    P = {"W_in": take(H * K, (H, K)), "b_in": take(H, (H,))}
    for l in range(N_LAYERS):
        P[f"W_self{l}"] = take(H * H, (H, H))
        P[f"W_nb{l}"] = take(H * H, (H, H))
        P[f"b{l}"] = take(H, (H,))
    P["W_out"] = take(K * H, (K, H))
    P["b_out"] = take(K, (K,))
    assert o == w.size
    return P


def forward(w, X, nbrs, K: int, H: int = 64):
    """X: (B, n_nodes, K); nbrs: list of neighbour index arrays.  Returns Y (B, n, K)."""
    P = unpack(w, K, H)
    A = np.maximum(X @ P["W_in"].T + P["b_in"], 0.0)
    for l in range(N_LAYERS):
        agg = np.stack([A[:, nb, :].mean(axis=1) if len(nb) else np.zeros_like(A[:, 0, :])
                        for nb in nbrs], axis=1)
        A = np.maximum(A @ P[f"W_self{l}"].T + agg @ P[f"W_nb{l}"].T + P[f"b{l}"], 0.0)
    return A @ P["W_out"].T + P["b_out"]


def bf16_round(x) -> np.ndarray:
    """FP32 values rounded to bfloat16 (8 significant bits: the upper 16 bits
    of the FP32 pattern), to nearest with ties to even, returned as FP32.
    Written from the definition of round-half-even on the bit pattern: add
    half a unit of the last kept bit, less one unless that bit is odd, then
    clear the 16 dropped bits."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _mean_f32(A32, nb):
    """Neighbour mean as the network's inference kernel forms it: FP32 sums in
    the neighbour list's order, then one FP32 division by the degree."""
    acc = np.zeros((A32.shape[0], A32.shape[2]), dtype=np.float32)
    for t in nb:
        acc = acc + A32[:, t, :]
    return acc / np.float32(len(nb)) if len(nb) else acc


def forward_bf16(w, X, nbrs, K: int, H: int = 64):
    """forward() with the operands of every layer rounded to bfloat16, as the
    learned preconditioner applies the network on the tensor cores: the
    weights (given as FP32), the FP32 input, each layer's FP32 activations
    (the FP64 result of the layer stored as FP32, then rounded) and the FP32
    neighbour means.  Products and sums are then exact or FP64."""
    P = unpack(np.asarray(w, dtype=np.float32), K, H)
    q = lambda M: bf16_round(np.asarray(M, dtype=np.float32)).astype(np.float64)
    A32 = np.asarray(X, dtype=np.float32)
    A = np.maximum(q(A32) @ q(P["W_in"]).T + P["b_in"], 0.0)
    for l in range(N_LAYERS):
        A32 = A.astype(np.float32)
        agg = np.stack([_mean_f32(A32, nb) for nb in nbrs], axis=1)
        A = np.maximum(q(A32) @ q(P[f"W_self{l}"]).T + q(agg) @ q(P[f"W_nb{l}"]).T + P[f"b{l}"],
                       0.0)
    A32 = A.astype(np.float32)
    return q(A32) @ q(P["W_out"]).T + P["b_out"]


def loss(w, X, T, wb, nbrs, K: int, H: int = 64) -> float:
    Y = forward(w, X, nbrs, K, H)
    per = ((Y - T) ** 2).sum(axis=(1, 2))
    return float((np.asarray(wb) * per).sum() / X.shape[0])


def fd_gradient(w, X, T, wb, nbrs, K: int, idx, H: int = 64, eps: float = 1e-6):
    """Central differences of the loss w.r.t. the weights at indices idx."""
    w = np.asarray(w, dtype=np.float64).copy()
    g = np.zeros(len(idx))
    for n, i in enumerate(idx):
        old = w[i]
        w[i] = old + eps
        lp = loss(w, X, T, wb, nbrs, K, H)
        w[i] = old - eps
        lm = loss(w, X, T, wb, nbrs, K, H)
        w[i] = old
        g[n] = (lp - lm) / (2 * eps)
    return g
