"""CPU oracle of the learned branch scorer (TEST INFRASTRUCTURE).

Only the test-suite uses this module. It restates, in float64 numpy and with
dense matrices, the model that the library's GNN kernels compute; it shares no
code with the library. The paper gives no network of its own (its discussion only
proposes learned policies in place of the myopic branching heuristics), so the
definition followed here is the one fixed by the library's public interface:

  features of v: [free, fixed 0, fixed 1, |w_v|/10, free neighbours/8, degree/8,
                  neighbours fixed to 1 / 8, overflow share (an input, 0 if absent)]
  layer l = 1..3: Z_l = H_{l-1} W_l + A H_{l-1} U_l + b_l,  H_l = relu(Z_l),  H_0 = X
  head:           s = H_3 w + c
  loss:           sum_v m_v (softplus(s_v) - y_v s_v) / sum_v m_v
  Adam:           beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected moments

Pins (tests/test_oracle_gnn.py): the gradient against central finite
differences of the loss; a hand-set network whose output is a closed form of
the vertex degrees; the loss against the cross-entropy written with log-sigmoid;
the first Adam step against lr * g / (|g| + eps); permutation equivariance.
"""
from __future__ import annotations

import numpy as np

F, HID, LAYERS = 8, 64, 3


def din(l):
    return F if l == 0 else HID


def param_count():
    return sum(2 * din(l) * HID + HID for l in range(LAYERS)) + HID + 1


def unpack(p):
    """Flat parameter vector -> ([(W, U, b)] * 3, w, c) as float64 views."""
    p = np.asarray(p, dtype=np.float64)
    assert p.shape == (param_count(),)
    off, layers = 0, []
    for l in range(LAYERS):
        d = din(l)
        W = p[off:off + d * HID].reshape(d, HID); off += d * HID
        U = p[off:off + d * HID].reshape(d, HID); off += d * HID
        b = p[off:off + HID]; off += HID
        layers.append((W, U, b))
    w = p[off:off + HID]; off += HID
    c = p[off]
    return layers, w, c


def adjacency(n, edges):
    A = np.zeros((n, n))
    for i, j in edges:
        A[i, j] += 1.0
        A[j, i] += 1.0
    return A


def features(n, edges, w=None, fixed=None, score=None):
    """Feature matrix (n x 8) by its definition, vertex by vertex."""
    fx = [-1] * n if fixed is None else [int(v) for v in fixed]
    wv = [1] * n if w is None else [int(v) for v in w]
    nbr = [[] for _ in range(n)]
    for i, j in edges:
        nbr[i].append(j)
        nbr[j].append(i)
    X = np.zeros((n, F))
    for v in range(n):
        X[v, 0] = fx[v] == -1
        X[v, 1] = fx[v] == 0
        X[v, 2] = fx[v] == 1
        X[v, 3] = abs(wv[v]) / 10.0
        X[v, 4] = sum(1 for u in nbr[v] if fx[u] == -1) / 8.0
        X[v, 5] = len(nbr[v]) / 8.0
        X[v, 6] = sum(1 for u in nbr[v] if fx[u] == 1) / 8.0
        X[v, 7] = 0.0 if score is None else float(score[v])
    return X


def forward(p, A, X):
    """Logits s (n,) and the activations needed by the backward pass."""
    layers, w, c = unpack(p)
    H = np.asarray(X, dtype=np.float64)
    cache = []
    for W, U, b in layers:
        M = A @ H
        Z = H @ W + M @ U + b
        cache.append((H, M, Z))
        H = np.maximum(Z, 0.0)
    s = H @ w + c
    return s, (cache, H)


def softplus(z):
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def loss(p, A, X, y, m):
    s, _ = forward(p, A, X)
    m = np.asarray(m, dtype=np.float64)
    cnt = m.sum()
    return float((m * (softplus(s) - y * s)).sum() / cnt) if cnt > 0 else 0.0


def grad(p, A, X, y, m):
    """Gradient of loss() by reverse-mode chain rule, packed like the parameters."""
    layers, w, c = unpack(p)
    s, (cache, H3) = forward(p, A, X)
    m = np.asarray(m, dtype=np.float64)
    cnt = m.sum()
    inv = 1.0 / cnt if cnt > 0 else 0.0
    dS = m * (1.0 / (1.0 + np.exp(-s)) - y) * inv
    gw = H3.T @ dS
    gc = dS.sum()
    dH = np.outer(dS, w)
    grads = [None] * LAYERS
    for l in reversed(range(LAYERS)):
        W, U, b = layers[l]
        Hin, M, Z = cache[l]
        dZ = dH * (Z > 0)
        grads[l] = (Hin.T @ dZ, M.T @ dZ, dZ.sum(axis=0))
        dH = dZ @ W.T + A.T @ (dZ @ U.T)
    out = []
    for gW, gU, gb in grads:
        out += [gW.ravel(), gU.ravel(), gb]
    out += [gw, np.array([gc])]
    return np.concatenate(out)


def adam(p, g, mo, vo, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (step counts from 1); returns new (p, m, v)."""
    mo = b1 * mo + (1 - b1) * g
    vo = b2 * vo + (1 - b2) * g * g
    mh = mo / (1 - b1 ** step)
    vh = vo / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), mo, vo
