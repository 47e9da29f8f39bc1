"""Pins of the oracle's graph network (the learned preconditioner's definition).

The network is not in the paper; it is pinned to mathematics: special cases
with closed-form outputs (zero weights give the output bias; identical node
inputs give identical outputs under mean aggregation) and central finite
differences checked against a directional derivative of the loss.
"""
import numpy as np

from oracle import gnn as G


def _setup(seed=0, B=2, n=5, K=6, H=4):
    rng = np.random.default_rng(seed)
    w = 0.5 * rng.standard_normal(G.n_weights(K, H))
    X = rng.standard_normal((B, n, K))
    T = rng.standard_normal((B, n, K))
    nbrs = [np.array([1, 2]), np.array([0]), np.array([0, 3]), np.array([2, 4]), np.array([3])]
    return w, X, T, np.array([1.0, 0.5]), nbrs, K, H


def test_weight_count_and_layout():
    K, H = 7, 4
    n = G.n_weights(K, H)
    assert n == H * K + H + 3 * (2 * H * H + H) + K * H + K
    P = G.unpack(np.arange(n, dtype=float), K, H)
    assert P["W_in"][0, 0] == 0 and P["b_out"][-1] == n - 1


def test_zero_weights_output_bias():
    w, X, T, wb, nbrs, K, H = _setup()
    w0 = np.zeros_like(w)
    P = G.unpack(w0, K, H)
    P["b_out"][:] = np.arange(K)       # view into w0
    Y = G.forward(w0, X, nbrs, K, H)
    assert np.allclose(Y, np.arange(K))


def test_mean_aggregation_of_constant_features():
    """All nodes equal: aggregation returns the same vector, so every node's output is equal."""
    w, X, T, wb, nbrs, K, H = _setup()
    Xc = np.repeat(X[:, :1, :], X.shape[1], axis=1)
    Y = G.forward(w, Xc, nbrs, K, H)
    assert np.allclose(Y, Y[:, :1, :])


def test_fd_gradient_consistent_with_directional_derivative():
    w, X, T, wb, nbrs, K, H = _setup(1)
    idx = np.arange(0, G.n_weights(K, H), 7)
    g = G.fd_gradient(w, X, T, wb, nbrs, K, idx, H)
    d = np.zeros_like(w)
    d[idx] = np.random.default_rng(2).standard_normal(idx.size)
    e = 1e-5
    dd = (G.loss(w + e * d, X, T, wb, nbrs, K, H) - G.loss(w - e * d, X, T, wb, nbrs, K, H)) / (2 * e)
    assert abs(dd - g @ d[idx]) <= 1e-5 * max(1.0, abs(dd))


def test_hand_computed_forward_on_three_node_path():
    """Path graph 0 - 1 - 2, K = 1, H = 2, one sample x = (1, -2, 3), integer
    weights, written out by hand:
      W_in = [1, -1]^T, b_in = (0, 1): A0 = (1,0), (0,3), (3,0) (the input
      ReLU clips node 1's first and node 2's second channel);
      every layer W_self = diag(1, 2), W_nb = [[0,1],[1,0]], b = (0, -1):
      A1 = (4,0), (0,7), (6,0); A2 = (11,0), (0,18), (13,0);
      A3 = (29,0), (0,47), (31,0) (means over neighbours; the -1 channel
      clipped by the ReLU at nodes 0 and 2);
      W_out = [1, -1], b_out = 0.5: Y = 29.5, -46.5, 31.5.
    Swapping W_self and W_nb, a sum instead of a mean, or a dropped ReLU all
    change Y."""
    K, H = 1, 2
    w = np.zeros(G.n_weights(K, H))
    P = G.unpack(w, K, H)          # views into w
    P["W_in"][:] = [[1.0], [-1.0]]
    P["b_in"][:] = [0.0, 1.0]
    for l in range(3):
        P[f"W_self{l}"][:] = [[1.0, 0.0], [0.0, 2.0]]
        P[f"W_nb{l}"][:] = [[0.0, 1.0], [1.0, 0.0]]
        P[f"b{l}"][:] = [0.0, -1.0]
    P["W_out"][:] = [[1.0, -1.0]]
    P["b_out"][:] = [0.5]
    X = np.array([[[1.0], [-2.0], [3.0]]])
    nbrs = [np.array([1]), np.array([0, 2]), np.array([1])]
    Y = G.forward(w, X, nbrs, K, H)
    assert np.array_equal(Y[0, :, 0], [29.5, -46.5, 31.5])


def test_bf16_round_half_even_by_hand():
    """bfloat16 keeps 8 significant bits.  Worked by hand: 255 (8 bits) and
    powers of two are kept; 1 + 2^-9 is below half a unit (2^-8) and goes to
    1; 1 + 2^-8 and 257 are ties that go to the even neighbour (1, 256);
    1 + 3 2^-8 and 259 are ties whose lower neighbour is odd (1.015625, 260)."""
    x = np.array([255.0, 0.5, -3.0, 1 + 2**-9, 1 + 2**-8, 257.0, 1 + 3 * 2**-8, 259.0, -259.0],
                 dtype=np.float32)
    want = [255.0, 0.5, -3.0, 1.0, 1.0, 256.0, 1.015625, 260.0, -260.0]
    assert np.array_equal(G.bf16_round(x), np.array(want, dtype=np.float32))


def _hand_case():
    K, H = 1, 2
    w = np.zeros(G.n_weights(K, H))
    P = G.unpack(w, K, H)
    P["W_in"][:] = [[1.0], [-1.0]]
    P["b_in"][:] = [0.0, 1.0]
    for l in range(3):
        P[f"W_self{l}"][:] = [[1.0, 0.0], [0.0, 2.0]]
        P[f"W_nb{l}"][:] = [[0.0, 1.0], [1.0, 0.0]]
        P[f"b{l}"][:] = [0.0, -1.0]
    P["W_out"][:] = [[1.0, -1.0]]
    P["b_out"][:] = [0.5]
    X = np.array([[[1.0], [-2.0], [3.0]]])
    nbrs = [np.array([1]), np.array([0, 2]), np.array([1])]
    return w, P, X, nbrs, K, H


def test_bf16_forward_on_the_hand_case():
    """Every value of the hand-computed case is exact in bfloat16, so the
    rounded network gives the same Y = (29.5, -46.5, 31.5)."""
    w, P, X, nbrs, K, H = _hand_case()
    Y = G.forward_bf16(w, X, nbrs, K, H)
    assert np.array_equal(Y[0, :, 0], [29.5, -46.5, 31.5])


def test_bf16_forward_rounds_input_weights_and_activations():
    """Perturbations below half a bfloat16 unit vanish where the kernel
    rounds: in the input (x_0 = 1 + 2^-9), in a weight (W_in[0] = 1 + 2^-9)
    and in an activation (b_in[0] = 2^-9 makes A0 of node 0 equal 1 + 2^-9,
    which the first message-passing layer reads rounded to 1).  The rounded
    network still gives the hand-computed Y; the unrounded one does not."""
    w, P, X, nbrs, K, H = _hand_case()
    X = X.copy()
    X[0, 0, 0] = 1 + 2**-9
    P["W_in"][0, 0] = 1 + 2**-9
    P["b_in"][0] = 2**-9
    Y = G.forward_bf16(w, X, nbrs, K, H)
    assert np.array_equal(Y[0, :, 0], [29.5, -46.5, 31.5])
    assert not np.array_equal(G.forward(w, X, nbrs, K, H)[0, :, 0], [29.5, -46.5, 31.5])


def test_bf16_forward_close_to_forward():
    """On a random network the rounded forward stays within the error that
    bfloat16 operands allow (relative unit 2^-8 per operand) of the exact one."""
    w, X, T, wb, nbrs, K, H = _setup(4)
    Y = G.forward(w, X, nbrs, K, H)
    Yb = G.forward_bf16(w, X, nbrs, K, H)
    assert not np.array_equal(Y, Yb)
    assert np.abs(Yb - Y).max() <= 0.05 * np.abs(Y).max()
