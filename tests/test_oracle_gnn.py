"""Pins of the GNN oracle (oracle/gnn.py) against facts that do not come from it.

CPU only; nothing here touches the CUDA library.
"""
import numpy as np
import pytest

import synth
from oracle import gnn as G


def _params(seed, scale=0.3):
    return np.random.default_rng(seed).normal(0.0, scale, G.param_count())


def _graph(seed, N=6):
    inst = synth.kings_subgraph(N, 0.8, seed=seed)
    return inst, G.adjacency(inst.n, inst.edges)


def test_param_count():
    """3 layers (8->64, 64->64, 64->64) of W, U (din x 64) and b (64); head 64 + 1."""
    assert G.param_count() == (2 * 8 * 64 + 64) + 2 * (2 * 64 * 64 + 64) + 65


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_finite_differences(seed):
    """Reverse-mode gradient == central differences of the loss (every parameter
    class: W, U, b of each layer and the head)."""
    inst, A = _graph(seed, N=4)
    rng = np.random.default_rng(100 + seed)
    fixed = rng.integers(-1, 2, inst.n)
    X = G.features(inst.n, inst.edges, inst.w, fixed)
    y = (rng.random(inst.n) < 0.4).astype(float)
    m = (rng.random(inst.n) < 0.8).astype(float)
    m[0] = 1.0
    p = _params(seed)
    g = G.grad(p, A, X, y, m)
    # a sample of coordinates from every block of the layout
    idx = np.unique(np.concatenate([rng.integers(0, G.param_count(), 120), [G.param_count() - 1]]))
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (G.loss(p + e, A, X, y, m) - G.loss(p - e, A, X, y, m)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_message_passing_closed_form():
    """Hand-set weights: layer 1 puts deg/8 (own feature 5), twice the overflow share
    (feature 7) and the neighbours' deg/8 into unit 0; layers 2, 3 pass unit 0
    through and add the neighbours' unit 0; the head reads unit 0. With d the
    degree vector and q the shares: h1 = d/8 + 2q + A d/8, h_{l+1} = h_l + A h_l,
    s = h3 -- a closed form in the adjacency matrix."""
    inst, A = _graph(3, N=5)
    p = np.zeros(G.param_count())
    layers, w, _ = G.unpack(p)   # views into p
    W1, U1, _ = layers[0]
    W1[5, 0] = 1.0
    W1[7, 0] = 2.0
    U1[5, 0] = 1.0
    for l in (1, 2):
        W, U, _ = layers[l]
        W[0, 0] = 1.0
        U[0, 0] = 1.0
    w[0] = 1.0
    q = np.random.default_rng(4).random(inst.n)
    X = G.features(inst.n, inst.edges, score=q)
    deg = A.sum(axis=1)
    h1 = deg / 8.0 + 2 * q + A @ deg / 8.0
    h2 = h1 + A @ h1
    h3 = h2 + A @ h2
    s, _ = G.forward(p, A, X)
    np.testing.assert_allclose(s, h3, rtol=1e-12)


def test_loss_is_binary_cross_entropy():
    """softplus(s) - y s == -[y log sigmoid(s) + (1 - y) log(1 - sigmoid(s))]."""
    inst, A = _graph(1)
    rng = np.random.default_rng(7)
    p = _params(5, 0.1)
    X = G.features(inst.n, inst.edges)
    y = (rng.random(inst.n) < 0.5).astype(float)
    m = np.ones(inst.n)
    s, _ = G.forward(p, A, X)
    assert 0.5 < np.abs(s).max() < 20      # away from saturation, not trivially small
    sig = 1.0 / (1.0 + np.exp(-s))
    bce = -(y * np.log(sig) + (1 - y) * np.log(1 - sig)).mean()
    assert abs(G.loss(p, A, X, y, m) - bce) < 1e-12


def test_first_adam_step_is_sign_step():
    """With zero moments, step 1 moves each parameter by lr * g / (|g| + eps)."""
    rng = np.random.default_rng(0)
    g = rng.normal(size=50)
    p = rng.normal(size=50)
    q, _, _ = G.adam(p, g, np.zeros(50), np.zeros(50), 0.01, 1)
    np.testing.assert_allclose(p - q, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9)


def test_permutation_equivariance():
    """Relabelling the vertices permutes the logits the same way."""
    inst, A = _graph(2)
    n = inst.n
    pi = np.random.default_rng(1).permutation(n)      # new index of old vertex v is pi[v]
    edges2 = [(int(pi[i]), int(pi[j])) for i, j in inst.edges]
    p = _params(9)
    X = G.features(n, inst.edges, inst.w)
    X2 = G.features(n, edges2, [inst.w[v] for v in np.argsort(pi)])
    s, _ = G.forward(p, A, X)
    s2, _ = G.forward(p, G.adjacency(n, edges2), X2)
    np.testing.assert_allclose(s2[pi], s, rtol=1e-12, atol=1e-12)


def test_features_by_hand():
    """Path 0-1-2 with vertex 0 fixed to 1, weights 5, 20, 3 and shares 0, 1, 0.5."""
    X = G.features(3, [(0, 1), (1, 2)], [5, 20, 3], [1, -1, -1], [0.0, 1.0, 0.5])
    np.testing.assert_allclose(X[0], [0, 0, 1, 0.5, 1 / 8, 1 / 8, 0, 0])
    np.testing.assert_allclose(X[1], [1, 0, 0, 2.0, 1 / 8, 2 / 8, 1 / 8, 1])
    np.testing.assert_allclose(X[2], [1, 0, 0, 0.3, 1 / 8, 1 / 8, 0, 0.5])


def test_empty_mask_gives_zero_loss_and_gradient():
    inst, A = _graph(0)
    X = G.features(inst.n, inst.edges)
    p = _params(1)
    z = np.zeros(inst.n)
    assert G.loss(p, A, X, z, z) == 0.0
    assert not np.any(G.grad(p, A, X, z, z))
