"""GPU: push / heuristic / learned schedules stay bit-exact; MLP kernels vs the fp64 oracle.

MLP tolerance: fp32 sums of at most 64 products per layer keep the relative
error near 64 * 2^-24 ~ 4e-6 per layer; the tests allow rtol 2e-4 / atol 2e-5.
"""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from oracle import mlp as omlp
import paper_2010_09913_gb300 as ss

pytestmark = pytest.mark.gpu
SEMIRINGS = ["tropical", "real", "boolean", "selmax"]


@pytest.fixture(scope="module", autouse=True)
def _build():
    ss.build()


def expected(g, r):
    d = oracle.bfs_queue(g.row_ptr, g.col, int(r))
    return d, oracle.dp(g.row_ptr, g.col, d, int(r))


def variants_of(G, iters):
    st, its = G.run_stats(cap=iters + 2)
    return [its[i].variant for i in range(1, st.iterations + 1)]


@pytest.mark.parametrize("policy", ["push", "heuristic", "learned"])
@pytest.mark.parametrize("loop", [1, 0])
def test_adaptive_policies_bit_exact(policy, loop):
    for g in [gg.kronecker(13, seed=2), gg.lattice(48, 0.05, seed=3), gg.erdos_renyi(5000, 6.0, seed=4)]:
        G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=64)
        G.set_option(ss.OPT_DEVICE_LOOP, loop)
        if policy == "learned":  # random weights give an arbitrary mix of variants
            ss.slimsell_selector_load(G.h, gg.mlp_weights(11, scale=3.0))
        for r in gg.roots(g, 2, seed=5):
            d, p = expected(g, r)
            for sr in SEMIRINGS:
                dist, parent = G.bfs(int(r), sr, policy)
                torch.cuda.synchronize()
                np.testing.assert_array_equal(dist.cpu().numpy(), d, err_msg=f"{g.name} {sr}")
                np.testing.assert_array_equal(parent.cpu().numpy(), p, err_msg=f"{g.name} {sr}")
                st, its = G.run_stats(cap=4096)
                levels = oracle.bfs_semiring(g.row_ptr, g.col, int(r), sr)[4]
                got = np.array([its[i].frontier for i in range(st.iterations + 1)])
                np.testing.assert_array_equal(got[: len(levels)], levels)
        G.close()


def test_push_then_pull_schedules_mix():
    g = gg.kronecker(14, seed=1)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=256)
    r = int(gg.roots(g, 1, seed=2)[0])
    G.bfs(r, "tropical", "heuristic")
    seq = variants_of(G, 64)
    assert seq[0] in (ss.V_PUSH, ss.VARIANT_PUSH_LOCAL) and ss.V_PULL_FILTERED in seq, seq
    G.bfs(r, "tropical", "push")
    seq = variants_of(G, 64)
    assert all(v in (ss.V_PUSH, ss.VARIANT_PUSH_LOCAL) for v in seq), seq
    assert ss.V_PUSH in seq and ss.VARIANT_PUSH_LOCAL in seq, seq
    ss.slimsell_selector_load(G.h, gg.mlp_weights(11, scale=3.0))
    G.bfs(r, "boolean", "learned")
    assert len(set(variants_of(G, 64))) >= 1
    ss.slimsell_selector_load(G.h, None)
    G.close()


def test_features_logged():
    g = gg.kronecker(12, seed=3)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col)
    r = int(gg.roots(g, 1, seed=1)[0])
    for loop in (0, 1):
        G.set_option(ss.OPT_DEVICE_LOOP, loop)
        G.bfs(r, "tropical", "heuristic")
        st, its = G.run_stats(cap=64)
        f = ss.slimsell_get_features(G.h, st.iterations + 1)
        # feature 1 is |f_{k-1}| / n and feature 9 is k / (k + 1)
        for k in range(1, st.iterations + 1):
            assert abs(f[k, 1] - its[k - 1].frontier / g.n) < 1e-6
            assert abs(f[k, 9] - k / (k + 1)) < 1e-6
    G.close()


def test_mlp_forward_matches_oracle():
    w = gg.mlp_weights(21)
    rng = np.random.default_rng(22)
    x = rng.normal(0, 1, (300, 16)).astype(np.float32)
    y = torch.empty((300, 4), dtype=torch.float32, device="cuda")
    ss.slimsell_mlp_forward(torch.from_numpy(w).cuda(), torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    want, _ = omlp.forward(w.astype(np.float64), x.astype(np.float64))
    np.testing.assert_allclose(y.cpu().numpy(), want, rtol=2e-4, atol=2e-5)


def test_mlp_gradient_and_adam_match_oracle():
    w = gg.mlp_weights(31)
    rng = np.random.default_rng(32)
    B = 97
    x = rng.normal(0, 1, (B, 16)).astype(np.float32)
    t = rng.normal(0, 1, (B, 4)).astype(np.float32)
    mask = (rng.random((B, 4)) < 0.6).astype(np.float32)
    dw = torch.from_numpy(w.copy()).cuda()
    m = torch.zeros(5508, device="cuda")
    v = torch.zeros(5508, device="cuda")
    grad = torch.empty(5508, device="cuda")
    loss = torch.empty(1, device="cuda")
    cx, ct, cm = (torch.from_numpy(a).cuda() for a in (x, t, mask))
    ss.slimsell_mlp_train_step(dw, m, v, 1, cx, ct, cm, 0.0, grad, loss)  # gradient only
    torch.cuda.synchronize()
    w64 = w.astype(np.float64)
    g_ref = omlp.grad(w64, x.astype(np.float64), t.astype(np.float64), mask.astype(np.float64))
    scale = np.abs(g_ref).max()
    np.testing.assert_allclose(grad.cpu().numpy(), g_ref, rtol=2e-4, atol=2e-5 * scale)
    assert abs(loss.item() - omlp.loss(w64, x, t, mask)) < 2e-4 * max(1.0, loss.item())
    np.testing.assert_array_equal(dw.cpu().numpy(), w)  # lr = 0: no update
    ss.slimsell_mlp_train_step(dw, m, v, 1, cx, ct, cm, 1e-3, grad, loss)
    torch.cuda.synchronize()
    w_ref, _, _ = omlp.adam_step(w64, np.zeros(5508), np.zeros(5508), g_ref, 1, 1e-3)
    # the first Adam step is lr * g / (|g| + eps): insensitive to fp32 rounding of g when
    # |g| >> eps, but where |g| is near eps the update swings within [-lr, lr]
    got = dw.cpu().numpy().astype(np.float64)
    big = np.abs(g_ref) > 1e-4 * scale
    np.testing.assert_allclose(got[big], w_ref[big], rtol=0, atol=2e-6)
    assert np.all(np.abs(got[~big] - w64[~big]) <= 1e-3 * (1 + 1e-4) + 1e-7)


def test_training_reduces_loss():
    rng = np.random.default_rng(41)
    B = 128
    x = rng.normal(0, 1, (B, 16)).astype(np.float32)
    t = np.stack([x[:, 0] + x[:, 1], x[:, 2] * 0.5, -x[:, 3], np.abs(x[:, 4])], 1).astype(np.float32)
    mask = np.ones((B, 4), dtype=np.float32)
    dw = torch.from_numpy(gg.mlp_weights(42)).cuda()
    m, v = torch.zeros(5508, device="cuda"), torch.zeros(5508, device="cuda")
    loss = torch.empty(1, device="cuda")
    cx, ct, cm = (torch.from_numpy(a).cuda() for a in (x, t, mask))
    losses = []
    for step in range(1, 301):
        ss.slimsell_mlp_train_step(dw, m, v, step, cx, ct, cm, 3e-3, None, loss)
        if step in (1, 300):
            torch.cuda.synchronize()
            losses.append(loss.item())
    assert losses[1] < 0.1 * losses[0], losses


def test_selector_training_pipeline():
    """Collect per-iteration variant timings, train the MLP on the GPU, and check what it
    learned: its argmin matches the measured-fastest variant on most iterations, and the
    learned schedule beats plain SlimWork and keeps up with the frontier-size rule."""
    from paper_2010_09913_gb300 import selector

    graphs = [gg.kronecker(15, seed=3), gg.lattice(96, 0.05, seed=2)]
    Xs, Ts, Ms, handles = [], [], [], []
    for g in graphs:
        G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=256)
        X, T, M = selector.collect(G, gg.roots(g, 2, seed=4), "tropical", repeats=2)
        Xs.append(X); Ts.append(T); Ms.append(M); handles.append((G, g))
    X, T, M = np.concatenate(Xs), np.concatenate(Ts), np.concatenate(Ms)
    assert X.shape[1] == 16 and np.all(M.sum(1) == 4)  # every variant ran every iteration
    w, loss = selector.train(X, T, M, steps=2500, lr=3e-3, seed=1)
    assert np.isfinite(loss) and loss < 0.5 * float(np.var(T))
    y = torch.empty((X.shape[0], 4), device="cuda")
    ss.slimsell_mlp_forward(torch.from_numpy(w).cuda(), torch.from_numpy(X).cuda(), y)
    torch.cuda.synchronize()
    pred = y.cpu().numpy().argmin(1)
    best = T.argmin(1)
    # near-ties (within 10%) count as a match
    close = T[np.arange(len(pred)), pred] <= T[np.arange(len(best)), best] + np.log(1.10)
    assert close.mean() >= 0.6, close.mean()
    # what the trained network gains, timed as the library runs it (device-side
    # loop, median of 15 runs per root) on every training family: less time than
    # the plain SlimWork pass by a stated factor (3 % on the small Kronecker graph,
    # where the frontier-size rule itself gains about 11 %; 0.7 on the 96 x 96
    # lattice, whose small levels go to the cluster push: 0.50-0.61 measured on
    # different boxes, with the plain pass running three pull launches per
    # device-side loop trip), and within 10 % of the rule, its fallback: the
    # network overrides the rule only where it predicts a gain of 0.3 log units
    # (about 35 %), and on levels this small (10-30 us, launch overheads of the
    # same size) one mispredicted level moves the total by about 5 % (1.056 of
    # the rule and 0.94 of plain SlimWork measured on the Kronecker graph)
    gain = [0.97, 0.7]
    for (G, g), factor in zip(handles, gain):
        ss.slimsell_selector_load(G.h, w)
        G.set_option(ss.OPT_SELECTOR_MARGIN, 300)
        t = selector.device_times(G, gg.roots(g, 2, seed=4), "tropical",
                                  ["slimwork", "heuristic", "learned"])
        assert t["learned"] <= factor * t["slimwork"], (g.name, t)
        assert t["learned"] <= 1.10 * t["heuristic"], (g.name, t)
        ss.slimsell_selector_load(G.h, None)
        G.close()


def test_learned_margin_falls_back_to_the_rule():
    """With a margin no prediction can clear, the learned policy runs exactly the
    frontier-size rule's schedule; unloading the weights after a learned run
    leaves a usable handle (the captured loop is rebuilt)."""
    g = gg.kronecker(13, seed=5)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=64)
    r = int(gg.roots(g, 1, seed=3)[0])
    d, p = expected(g, r)
    G.bfs(r, "tropical", "heuristic")
    want = variants_of(G, 64)
    ss.slimsell_selector_load(G.h, gg.mlp_weights(11, scale=3.0))
    G.set_option(ss.OPT_SELECTOR_MARGIN, 100000)
    dist, parent = G.bfs(r, "tropical", "learned")
    torch.cuda.synchronize()
    assert variants_of(G, 64) == want
    np.testing.assert_array_equal(dist.cpu().numpy(), d)
    with pytest.raises(ss.SlimSellError):
        G.set_option(ss.OPT_SELECTOR_MARGIN, -1)
    G.set_option(ss.OPT_SELECTOR_MARGIN, 0)
    ss.slimsell_selector_load(G.h, None)
    dist, parent = G.bfs(r, "tropical", "learned")
    torch.cuda.synchronize()
    np.testing.assert_array_equal(parent.cpu().numpy(), p)
    assert variants_of(G, 64) == want  # no weights: the rule
    G.close()

