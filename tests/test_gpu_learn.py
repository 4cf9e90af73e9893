"""Learned schedule on the GPU: features, network forward/backward and training against the CPU
oracle, and the schedule itself (identical results, better ordering than the static one)."""
import heapq

import numpy as np
import pytest

import synth
from oracle import learn as L
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mbe():
    import torch
    assert torch.cuda.is_available(), "GPU test"
    import paper_2401_05039_gb300 as m
    m.load()
    return m


def _tuple(r):
    return (int(r.count), int(r.hash), int(r.nodes), int(r.bytes_alg))


def test_features_match_oracle(mbe):
    graphs = [synth.workload("er200x300"), H.random_graph(np.random.default_rng(21), 90, 140, 0.06),
              synth.planted(400, 500, 0.02, 5, (5, 9), (6, 12), 0.3, 7),
              H.graph(4, 3, [(0, 0), (0, 1), (0, 2), (1, 0), (1, 1), (2, 1), (2, 2)])]
    for g in graphs:
        raw_o, fl_o = L.root_features(g)
        G = mbe.Graph.from_synth(g)
        f, r = G.features(raw=True)
        G.close()
        assert (r.cpu().numpy() == raw_o).all(), g.name
        assert np.allclose(f.cpu().numpy(), fl_o, rtol=1e-6, atol=1e-7)


def _rand_params(seed):
    rng = np.random.default_rng(seed)
    p = L.init_params(seed)
    p[L.H * L.F:L.H * L.F + L.H] = rng.normal(0.1, 0.2, L.H)
    p[L.H * L.F + L.H + L.H * L.H:L.H * L.F + 2 * L.H + L.H * L.H] = rng.normal(0.1, 0.2, L.H)
    p[-1] = 0.3
    return p.astype(np.float32)


def test_forward_and_gradient_match_oracle(mbe):
    import torch
    rng = np.random.default_rng(22)
    p = _rand_params(5)
    X = rng.normal(1.5, 1.0, (300, L.F)).astype(np.float32)
    t = rng.normal(3.0, 1.5, 300).astype(np.float32)
    m = mbe.Model(0)
    m.set_params(p)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    y = m.predict(Xd).cpu().numpy()
    y_o, _ = L.mlp_forward(p.astype(np.float64), X.astype(np.float64))
    assert np.allclose(y, y_o, rtol=2e-3, atol=2e-3)
    loss, g = m.loss_grad(Xd, td)
    loss_o, g_o = L.mlp_loss_grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert loss == pytest.approx(loss_o, rel=2e-3)
    scale = np.abs(g_o).max()
    assert np.abs(g - g_o).max() <= 2e-3 * scale
    # per-block relative check on the two big weight matrices
    for a, b in ((0, L.H * L.F), (L.H * L.F + L.H, L.H * L.F + L.H + L.H * L.H)):
        err = np.linalg.norm(g[a:b] - g_o[a:b]) / max(np.linalg.norm(g_o[a:b]), 1e-12)
        assert err <= 1e-2
    m.close()


def test_training_reduces_loss(mbe):
    g = synth.planted(1500, 1500, 0.02, 12, (8, 14), (10, 20), 0.3, 123)
    feat, target = mbe.training_set([g])
    m = mbe.Model(1)
    loss0, _ = m.loss_grad(feat, target)
    loss1 = m.train(feat, target, epochs=40, batch=256, lr=3e-3, seed=2)
    loss2, _ = m.loss_grad(feat, target)
    assert loss2 < 0.5 * loss0, (loss0, loss1, loss2)
    m.close()


def _makespan(order, cost, workers):
    """Greedy list scheduling of roots in `order` (cost = measured subtree nodes) on `workers` machines."""
    heap = [0.0] * workers
    for r in order:
        t = heapq.heappop(heap)
        heapq.heappush(heap, t + float(cost[r]))
    return max(heap)


def test_learned_schedule_same_results_and_better_order(mbe):
    import torch
    # training graphs: shaped like the 20k Chung-Lu and the planted workloads, other seeds
    train = [synth.chung_lu(6000, 15000, 60000, 2.1, 2.3, 2000, 101), synth.planted(2000, 2000, 0.01, 20, (15, 25),
                                                                                   (20, 40), 0.3, 102)]
    feat, target = mbe.training_set(train)
    model = mbe.Model(7)
    model.train(feat, target, epochs=40, batch=512, lr=3e-3, seed=3)
    # held-out graph of the planted family
    g = synth.planted(3000, 3000, 0.01, 40, (15, 25), (20, 40), 0.3, 103)
    G = mbe.Graph.from_synth(g)
    r0, pr0 = G.per_root()
    r1, pr1 = G.per_root(schedule=1, model=model)
    r2, pr2 = G.per_root(schedule=2, model=model)
    # without stealing, schedule 1 pre-splits the predicted-heaviest roots into parts
    r3, pr3 = G.per_root(schedule=1, model=model, steal=0)
    assert _tuple(r0) == _tuple(r1) == _tuple(r2) == _tuple(r3)
    assert (pr0 == pr1).all() and (pr0 == pr2).all() and (pr0 == pr3).all()
    # the learned order ranks roots by predicted cost; checked against the measured subtree nodes
    f = G.features()
    pred = model.predict(f).cpu().numpy()
    live = np.nonzero(np.diff(g.u_off) > 0)[0]
    nodes = pr0[:, 2].astype(np.float64)
    from scipy.stats import spearmanr
    rho = spearmanr(pred[live], np.log1p(nodes[live])).correlation
    assert rho > 0.6, rho
    deg = np.diff(g.u_off)
    static = live[np.argsort(-deg[live], kind="stable")]
    learned = live[np.argsort(-pred[live], kind="stable")]
    workers = 2432
    assert _makespan(learned, nodes, workers) <= _makespan(static, nodes, workers)
    G.close()
    model.close()


def test_nonfinite_prediction_falls_back_to_static(mbe):
    g = synth.workload("er200x300")
    m = mbe.Model(0)
    p = m.get_params()
    p[-1] = np.nan
    m.set_params(p)
    G = mbe.Graph.from_synth(g)
    assert _tuple(G.enumerate(schedule=1, model=m)) == _tuple(G.enumerate())
    G.close()
    m.close()
