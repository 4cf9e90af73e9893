"""CPU oracle for the cost-model side of the learned schedule.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark baseline); shares no
code with the GPU path.

- ``root_features``: the eight per-root features, from their definitions,
  with plain Python sets.
- ``core_numbers``: k-core numbers of G taken as a general graph (U and V
  vertices together), by the textbook peeling definition: at level k,
  repeatedly delete vertices of remaining degree <= k; a vertex deleted at
  level k has core number k.
- ``mlp_*``: the 8 -> 64 -> 64 -> 1 ReLU network in float64 on float16-rounded
  weights and inputs, with activations rounded to float16 after each ReLU
  (the GPU stores them so), and its exact backward pass. ``mlp_fd_grad`` is a
  central finite-difference gradient used to pin the analytic one.

Parameter vector (4801 floats): W1[64][8], b1[64], W2[64][64], b2[64], W3[64], b3.
"""
from __future__ import annotations

import math

import numpy as np

H = 64
F = 8
N_PARAMS = H * F + H + H * H + H + H + 1

FEATURE_NAMES = ("log1p_degree", "log1p_two_hop", "log1p_P0", "log1p_Q0", "log1p_core", "log1p_sum_nbr_degree",
                 "log1p_max_nbr_degree", "frac_roots_with_larger_degree")


def core_numbers(g) -> np.ndarray:
    """Core number of every vertex; U vertices first (0..nU-1), then V (nU..nU+nV-1)."""
    n = g.nU + g.nV
    adj = [[] for _ in range(n)]
    for u in range(g.nU):
        for k in range(g.u_off[u], g.u_off[u + 1]):
            v = g.nU + int(g.u_adj[k])
            adj[u].append(v)
            adj[v].append(u)
    deg = np.array([len(a) for a in adj], dtype=np.int64)
    alive = np.ones(n, dtype=bool)
    core = np.zeros(n, dtype=np.int64)
    remaining = n
    k = 0
    while remaining:
        while True:
            peel = [v for v in range(n) if alive[v] and deg[v] <= k]
            if not peel:
                break
            for v in peel:
                alive[v] = False
                core[v] = k
                remaining -= 1
            for v in peel:
                for w in adj[v]:
                    deg[w] -= 1
        k += 1
    return core


def root_features(g):
    """(raw int64 [nU][8], float64 [nU][8]) features of every U vertex as a root.

    raw: degree d; |N2(r)| (U vertices other than r sharing a neighbour with
    r); |P0| and |Q0| (those after / before r in the (degree, id) order);
    core number; sum and max of the degrees of N(r); number of U vertices of
    larger degree. float: log1p of the first seven, the last divided by |U|.
    Isolated vertices get all-zero features.
    """
    nU = g.nU
    du = np.diff(g.u_off).astype(np.int64)
    dv = np.diff(g.v_off).astype(np.int64)
    core = core_numbers(g)[:nU]
    raw = np.zeros((nU, F), dtype=np.int64)
    larger = np.array([int((du > d).sum()) for d in range(int(du.max(initial=0)) + 2)], dtype=np.int64)
    for r in range(nU):
        d = int(du[r])
        if d == 0:
            continue
        nbrs = g.u_adj[g.u_off[r]:g.u_off[r + 1]]
        two_hop = set()
        for w in nbrs:
            two_hop.update(int(x) for x in g.v_adj[g.v_off[w]:g.v_off[w + 1]])
        two_hop.discard(r)
        p0 = sum(1 for u in two_hop if (du[u], u) > (d, r))
        q0 = len(two_hop) - p0
        raw[r] = (d, len(two_hop), p0, q0, core[r], int(dv[nbrs].sum()), int(dv[nbrs].max()), larger[d])
    fl = np.zeros((nU, F), dtype=np.float64)
    live = du > 0
    fl[live, :7] = np.log1p(raw[live, :7].astype(np.float64))
    fl[live, 7] = raw[live, 7] / max(nU, 1)
    return raw, fl


# ------------------------------------------------------------------ network

def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * F].reshape(H, F); o += H * F
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, W3, b3


def f16(x):
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def mlp_forward(p, X):
    """Predictions and the activations the backward pass needs (float64 arithmetic).

    Weights and inputs are rounded to float16 first (the GPU's operands);
    the hidden activations are float16-rounded after each ReLU; biases stay
    in float32 precision.
    """
    W1, b1, W2, b2, W3, b3 = unpack(p)
    W1, W2, W3 = f16(W1), f16(W2), f16(W3)
    b1 = b1.astype(np.float32).astype(np.float64)
    b2 = b2.astype(np.float32).astype(np.float64)
    b3 = float(np.float32(b3))
    X16 = f16(X)
    H1 = f16(np.maximum(X16 @ W1.T + b1, 0.0))
    H2 = f16(np.maximum(H1 @ W2.T + b2, 0.0))
    y = H2 @ W3 + b3
    return y, (X16, H1, H2, W1, W2, W3)


def mlp_loss_grad(p, X, t):
    """Mean squared error and its gradient w.r.t. the parameter vector (ReLU masks from the stored activations)."""
    y, (X16, H1, H2, W1, W2, W3) = mlp_forward(p, X)
    B = X.shape[0]
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / B
    gW3 = H2.T @ dy
    gb3 = dy.sum()
    dZ2 = np.outer(dy, W3) * (H2 > 0)
    gW2 = dZ2.T @ H1
    gb2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2) * (H1 > 0)
    gW1 = dZ1.T @ X16
    gb1 = dZ1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return loss, g


def mlp_fd_grad(p, X, t, idx, eps=1e-6):
    """Central finite differences of the float64 loss without float16 rounding, for the listed parameters."""
    def loss64(q):
        W1, b1, W2, b2, W3, b3 = unpack(q)
        h1 = np.maximum(X @ W1.T + b1, 0.0)
        h2 = np.maximum(h1 @ W2.T + b2, 0.0)
        y = h2 @ W3 + b3
        return float(np.mean((y - t) ** 2))
    out = []
    for i in idx:
        q = np.array(p, dtype=np.float64)
        q[i] += eps
        lp = loss64(q)
        q[i] -= 2 * eps
        lm = loss64(q)
        out.append((lp - lm) / (2 * eps))
    return np.array(out)


def mlp_grad64(p, X, t):
    """Exact float64 gradient without float16 rounding (the function mlp_fd_grad differentiates)."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    Z1 = X @ W1.T + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2.T + b2
    H2 = np.maximum(Z2, 0.0)
    y = H2 @ W3 + b3
    B = X.shape[0]
    dy = 2.0 * (y - t) / B
    dZ2 = np.outer(dy, W3) * (Z2 > 0)
    dZ1 = (dZ2 @ W2) * (Z1 > 0)
    return np.concatenate([(dZ1.T @ X).ravel(), dZ1.sum(0), (dZ2.T @ H1).ravel(), dZ2.sum(0), H2.T @ dy, [dy.sum()]])


def init_params(seed: int) -> np.ndarray:
    """Uniform(+-1/sqrt(fan_in)) weights, zero biases (reference initialisation for tests)."""
    rng = np.random.default_rng(seed)
    p = np.zeros(N_PARAMS)
    o = 0
    for rows, cols in ((H, F), (H, H), (1, H)):
        lim = 1.0 / math.sqrt(cols)
        p[o:o + rows * cols] = rng.uniform(-lim, lim, rows * cols)
        o += rows * cols + (rows if rows > 1 else 1)
    return p
