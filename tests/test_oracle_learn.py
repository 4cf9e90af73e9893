"""Pins for the cost-model oracle: core numbers, root features, network gradients."""
import numpy as np
import pytest

from oracle import learn as L
from tests import helpers as H


def test_core_numbers_match_networkx():
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(8)
    for _ in range(12):
        g = H.random_graph(rng, int(rng.integers(3, 40)), int(rng.integers(3, 40)), float(rng.choice([0.05, 0.2, 0.5])))
        G = nx.Graph()
        G.add_nodes_from(range(g.nU + g.nV))
        for u, v in H.edges_of(g):
            G.add_edge(u, g.nU + v)
        ref = nx.core_number(G)
        got = L.core_numbers(g)
        assert [ref[i] for i in range(g.nU + g.nV)] == got.tolist()


def test_core_numbers_closed_forms():
    # K_{a,b}: every vertex has core number min(a, b); a matching: 1; isolated: 0
    assert set(L.core_numbers(H.complete(3, 5)).tolist()) == {3}
    assert set(L.core_numbers(H.matching(4)).tolist()) == {1}
    assert L.core_numbers(H.empty(2, 3)).tolist() == [0] * 5


def test_root_features_hand_example():
    # a={1,2,3}, b={1,2}, c={2,3} (a=0, b=1, c=2; V ids 0,1,2); plus isolated d=3
    g = H.graph(4, 3, [(0, 0), (0, 1), (0, 2), (1, 0), (1, 1), (2, 1), (2, 2)])
    raw, fl = L.root_features(g)
    # root a: d=3; N2={b,c}; (deg,id): b=(2,1), c=(2,2) both before a=(3,0) -> P0=0, Q0=2; core 2;
    # nbr degrees 2,3,2 -> sum 7 max 3; U vertices of larger degree: none
    assert raw[0].tolist() == [3, 2, 0, 2, 2, 7, 3, 0]
    # root b: d=2; N2={a,c}; a after, c after (2,2)>(2,1) -> P0=2, Q0=0; nbrs deg 2,3
    assert raw[1].tolist() == [2, 2, 2, 0, 2, 5, 3, 1]
    assert raw[3].tolist() == [0] * 8 and fl[3].tolist() == [0.0] * 8
    assert np.allclose(fl[0, :7], np.log1p(raw[0, :7]))
    assert fl[1, 7] == 1 / 4


def test_two_hop_counts_by_matrix_product():
    rng = np.random.default_rng(9)
    g = H.random_graph(rng, 30, 50, 0.08)
    raw, _ = L.root_features(g)
    A = np.zeros((g.nU, g.nV), dtype=np.int64)
    for u, v in H.edges_of(g):
        A[u, v] = 1
    M = (A @ A.T) > 0
    np.fill_diagonal(M, False)
    deg = A.sum(1)
    assert (raw[:, 1] == np.where(deg > 0, M.sum(1), 0)).all()
    assert (raw[:, 2] + raw[:, 3] == raw[:, 1]).all()


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(10)
    p = L.init_params(3)
    p[L.H * L.F:L.H * L.F + L.H] = rng.normal(0, 0.1, L.H)  # nonzero biases
    X = rng.normal(1.0, 1.0, (40, L.F))
    t = rng.normal(2.0, 1.0, 40)
    g = L.mlp_grad64(p, X, t)
    idx = rng.choice(L.N_PARAMS, 60, replace=False).tolist() + [L.N_PARAMS - 1]
    fd = L.mlp_fd_grad(p, X, t, idx)
    assert np.allclose(g[idx], fd, rtol=1e-5, atol=1e-8)


def test_mlp_rounded_gradient_close_to_exact():
    # the float16-operand gradient (what the GPU computes) is within float16 rounding of the exact one
    rng = np.random.default_rng(11)
    p = L.init_params(4)
    X = rng.normal(1.0, 1.0, (64, L.F))
    t = rng.normal(2.0, 1.0, 64)
    _, g16 = L.mlp_loss_grad(p, X, t)
    g64 = L.mlp_grad64(p, X, t)
    assert np.abs(g16 - g64).max() <= 2e-2 * np.abs(g64).max()


def test_mlp_closed_form_constant_output():
    p = np.zeros(L.N_PARAMS)
    p[-1] = 1.5  # y = b3 for every input
    X = np.ones((8, L.F))
    t = np.arange(8.0)
    loss, g = L.mlp_loss_grad(p, X, t)
    assert loss == pytest.approx(np.mean((1.5 - t) ** 2))
    assert g[-1] == pytest.approx(2 * np.mean(1.5 - t))
    assert np.all(g[:-1] == 0)
