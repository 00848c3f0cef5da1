"""Pins of the network oracle (oracle/nn.py) against what mathematics fixes: brute-force
loops of the convolution definition, adjoint identities of the convolution, pooling and
upsampling, central finite differences of the whole network's loss, the closed form of
Adam's first step, and exact reproduction of linear fields by the node <-> cell maps."""
import numpy as np
import pytest

from oracle import nn as N


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_conv3_matches_brute_force_loops():
    n, ci, co = 3, 2, 3
    r = _rng(1)
    x = r.standard_normal((n ** 3, ci))
    W = r.standard_normal((27, co, ci))
    b = r.standard_normal(co)
    y = N.conv3(x, W, n, b)
    ref = np.zeros((n ** 3, co))
    T = N.taps()
    for k in range(n):
        for j in range(n):
            for i in range(n):
                v = i + n * (j + n * k)
                for o in range(co):
                    s = b[o]
                    for t, (dx, dy, dz) in enumerate(T):
                        a, bb, c = i + dx, j + dy, k + dz
                        if 0 <= a < n and 0 <= bb < n and 0 <= c < n:
                            for q in range(ci):
                                s += W[t, o, q] * x[a + n * (bb + n * c), q]
                    ref[v, o] = s
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()


def test_conv3_adjoints():
    n, ci, co = 5, 3, 4
    r = _rng(2)
    x = r.standard_normal((n ** 3, ci))
    y = r.standard_normal((n ** 3, co))
    W = r.standard_normal((27, co, ci))
    lhs = np.sum(N.conv3(x, W, n) * y)
    assert np.isclose(lhs, np.sum(x * N.conv3_dgrad(y, W, n)), rtol=1e-12)
    assert np.isclose(lhs, np.sum(W * N.conv3_wgrad(x, y, n)), rtol=1e-12)


def test_pool_and_up_are_adjoint_up_to_eight():
    m = 3
    r = _rng(3)
    a = r.standard_normal((m ** 3, 2))
    b = r.standard_normal(((2 * m) ** 3, 2))
    assert np.isclose(np.sum(N.up(a, m) * b), 8.0 * np.sum(a * N.pool(b, 2 * m)), rtol=1e-12)
    # pool of an upsampled field returns it
    assert np.allclose(N.pool(N.up(a, m), 2 * m), a, rtol=0, atol=1e-15)


def test_backward_matches_finite_differences():
    n = 4
    P = N.init_params(7)
    r = _rng(4)
    for name in P:  # non-zero biases so that every ReLU sees both signs
        P[name] = (P[name][0], 0.1 * r.standard_normal(P[name][1].shape))
    x = r.standard_normal((n ** 3, N.CIN))
    tgt = r.standard_normal((n ** 3, 16))

    def loss(params):
        y, _ = N.forward(params, x, n)
        return N.loss_and_grad_y(y, tgt)[0]

    y, cache = N.forward(P, x, n)
    _, dy = N.loss_and_grad_y(y, tgt)
    G = N.backward(P, cache, dy, n)
    eps = 1e-6
    for name in P:
        W, b = P[name]
        for idx in [(0, 0, 0), (13, W.shape[1] - 1, W.shape[2] - 1), (26, 1, 2)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += eps
            Wm[idx] -= eps
            fd = (loss({**P, name: (Wp, b)}) - loss({**P, name: (Wm, b)})) / (2 * eps)
            assert np.isclose(G[name][0][idx], fd, rtol=1e-5, atol=1e-9), (name, idx)
        bp, bm = b.copy(), b.copy()
        bp[0] += eps
        bm[0] -= eps
        fd = (loss({**P, name: (W, bp)}) - loss({**P, name: (W, bm)})) / (2 * eps)
        assert np.isclose(G[name][1][0], fd, rtol=1e-5, atol=1e-9), name


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    w, m, v = N.adam_step(np.ones(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2
    assert np.allclose(w, 1.0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_node_cell_maps_reproduce_linear_fields():
    n = 6
    t = np.arange(n + 1) / n
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    lin = (0.3 + 2.0 * x - 1.5 * y + 0.25 * z).ravel()
    nodal = np.stack([lin, 2 * lin, -lin, 3 * lin])
    cells = N.target(nodal.ravel(), 2.0, n)
    c = (np.arange(n) + 0.5) / n
    cz, cy, cx = np.meshgrid(c, c, c, indexing="ij")
    lin_c = (0.3 + 2.0 * cx - 1.5 * cy + 0.25 * cz).ravel()
    assert np.allclose(cells[:, 0], N.VEL_SCALE * lin_c / 2.0)
    # pressure: the node mean is removed first (cell means of a linear field keep that mean)
    assert np.allclose(cells[:, 3], 3 * (lin_c - lin.mean()) / 2.0)
    back = N.to_nodes(cells, 2.0, n, np.zeros(4 * (n + 1) ** 3, dtype=bool)).reshape(4, n + 1, n + 1, n + 1)
    inner = (slice(None), slice(1, n), slice(1, n), slice(1, n))
    want = nodal.copy()
    want[3] -= want[3].mean()
    assert np.allclose(back[inner], want.reshape(4, n + 1, n + 1, n + 1)[inner], atol=1e-13)
    f = np.stack([lin, -lin, 0 * lin])
    feats, fs = N.features(np.full(n ** 3, 100.0), f, n)
    assert fs == np.abs(f).max() and np.allclose(feats[:, 0], 2.0) and np.all(feats[:, 4] == 1.0)
    assert np.allclose(feats[:, 1], lin_c / fs) and np.all(feats[:, 5:] == 0.0)


def test_line_search_minimises_the_residual():
    r = _rng(5)
    K = r.standard_normal((6, 6)) + 6 * np.eye(6)
    b = r.standard_normal(6)
    x = r.standard_normal(6)
    xs = N.line_search(K, b, x)
    a = xs[0] / x[0]
    res = lambda t: np.linalg.norm(b - t * (K @ x))
    assert res(a) <= min(res(a - 1e-6), res(a + 1e-6)) and res(a) <= np.linalg.norm(b)
