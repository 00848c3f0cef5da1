"""Plain FP64 numpy reference of the learned initial guess network (TEST INFRASTRUCTURE ONLY).

The network is a small 3D U-Net of 3x3x3 convolutions on the cell grid (N^3 cells, N a
multiple of 4).  Tensors are [V, C] with V = i + N*(j + N*k) (x fastest, the cell order of
the solver) and C channels; weights of a convolution are [27, C_out, C_in] with tap
t = (dz+1)*9 + (dy+1)*3 + (dx+1), and a tap reads the input at offset (dx, dy, dz); outside
the grid the input is zero.  Layers (channels 16 -> 16 -> 16 | pool | 32 -> 32 | pool | 64 |
up | 32 (+skip) -> 32 | up | 16 (+skip) -> 16 -> 16):

    a1 = relu(conv(x, W1) + b1)             N        16 -> 16
    a2 = relu(conv(a1, W2) + b2)            N        16 -> 16   (skip s0)
    a3 = relu(conv(pool(a2), W3) + b3)      N/2      16 -> 32
    a4 = relu(conv(a3, W4) + b4)            N/2      32 -> 32   (skip s1)
    a5 = relu(conv(pool(a4), W5) + b5)      N/4      32 -> 64
    a6 = relu(conv(up(a5), W6) + b6 + a4)   N/2      64 -> 32
    a7 = relu(conv(a6, W7) + b7)            N/2      32 -> 32
    a8 = relu(conv(up(a7), W8) + b8 + a2)   N        32 -> 16
    a9 = relu(conv(a8, W9) + b9)            N        16 -> 16
    y  = conv(a9, W10) + b10                N        16 -> 16   (channels 0..3 used)

pool = mean over 2x2x2 blocks, up = nearest-neighbour (each coarse cell to its 8 children).
Loss: sum over cells and channels 0..3 of (y - target)^2 / (4 V).
Optimiser: Adam (Kingma & Ba 2015) with bias correction.

Every function here is the definition written out (shifted slices and einsum), pinned in
tests/test_oracle_nn.py by brute-force loops, adjoint identities and finite differences.
"""
from __future__ import annotations

import numpy as np

CIN = 16
LAYERS = [  # (name, C_in, C_out, level: 0 = N, 1 = N/2, 2 = N/4)
    ("L1", 16, 16, 0), ("L2", 16, 16, 0), ("L3", 16, 32, 1), ("L4", 32, 32, 1), ("L5", 32, 64, 2),
    ("L6", 64, 32, 1), ("L7", 32, 32, 1), ("L8", 32, 16, 0), ("L9", 16, 16, 0), ("L10", 16, 16, 0),
]
OUT_USED = 4


def taps():
    """Offsets (dx, dy, dz) of the 27 taps in tap order."""
    return [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _grid(x, n):
    return x.reshape(n, n, n, x.shape[-1])  # [k, j, i, c]


def _shifted(x, n, d):
    """x at (i+dx, j+dy, k+dz), zero outside the grid; [V, C]."""
    g = _grid(x, n)
    dx, dy, dz = d
    out = np.zeros_like(g)
    src_k = slice(max(dz, 0), n + min(dz, 0))
    dst_k = slice(max(-dz, 0), n + min(-dz, 0))
    src_j = slice(max(dy, 0), n + min(dy, 0))
    dst_j = slice(max(-dy, 0), n + min(-dy, 0))
    src_i = slice(max(dx, 0), n + min(dx, 0))
    dst_i = slice(max(-dx, 0), n + min(-dx, 0))
    out[dst_k, dst_j, dst_i] = g[src_k, src_j, src_i]
    return out.reshape(-1, x.shape[-1])


def conv3(x, W, n, b=None):
    """y[v, co] = sum_t sum_ci W[t, co, ci] x[v + off_t, ci] (+ b[co])."""
    y = np.zeros((x.shape[0], W.shape[1]))
    for t, d in enumerate(taps()):
        y += _shifted(x, n, d) @ W[t].T
    if b is not None:
        y = y + b[None, :]
    return y


def conv3_dgrad(dy, W, n):
    """Adjoint of conv3 in x: dx[v, ci] = sum_t sum_co W[t, co, ci] dy[v - off_t, co]."""
    dx = np.zeros((dy.shape[0], W.shape[2]))
    for t, (ox, oy, oz) in enumerate(taps()):
        dx += _shifted(dy, n, (-ox, -oy, -oz)) @ W[t]
    return dx


def conv3_wgrad(x, dy, n):
    """Gradient in W: dW[t, co, ci] = sum_v dy[v, co] x[v + off_t, ci]."""
    return np.stack([dy.T @ _shifted(x, n, d) for d in taps()])


def pool(x, n):
    """Mean over 2x2x2 blocks: [n^3, C] -> [(n/2)^3, C]."""
    g = _grid(x, n)
    m = n // 2
    return g.reshape(m, 2, m, 2, m, 2, -1).mean(axis=(1, 3, 5)).reshape(m ** 3, -1)


def up(x, m):
    """Nearest-neighbour upsampling: [m^3, C] -> [(2m)^3, C]."""
    g = _grid(x, m)
    g = np.repeat(np.repeat(np.repeat(g, 2, 0), 2, 1), 2, 2)
    return g.reshape((2 * m) ** 3, -1)


def init_params(seed: int):
    """He-normal weights (std sqrt(2 / (27 C_in))), zero biases; a dict name -> (W, b)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return {name: (rng.standard_normal((27, co, ci)) * np.sqrt(2.0 / (27 * ci)), np.zeros(co))
            for name, ci, co, _ in LAYERS}


def forward(params, x, n):
    """All activations of the network for input x [n^3, 16]; returns (y, cache)."""
    P = params
    relu = lambda z: np.maximum(z, 0.0)
    c = {"x": x}
    c["z1"] = conv3(x, P["L1"][0], n, P["L1"][1]); c["a1"] = relu(c["z1"])
    c["z2"] = conv3(c["a1"], P["L2"][0], n, P["L2"][1]); c["a2"] = relu(c["z2"])
    c["p1"] = pool(c["a2"], n)
    c["z3"] = conv3(c["p1"], P["L3"][0], n // 2, P["L3"][1]); c["a3"] = relu(c["z3"])
    c["z4"] = conv3(c["a3"], P["L4"][0], n // 2, P["L4"][1]); c["a4"] = relu(c["z4"])
    c["p2"] = pool(c["a4"], n // 2)
    c["z5"] = conv3(c["p2"], P["L5"][0], n // 4, P["L5"][1]); c["a5"] = relu(c["z5"])
    c["u1"] = up(c["a5"], n // 4)
    c["z6"] = conv3(c["u1"], P["L6"][0], n // 2, P["L6"][1]) + c["a4"]; c["a6"] = relu(c["z6"])
    c["z7"] = conv3(c["a6"], P["L7"][0], n // 2, P["L7"][1]); c["a7"] = relu(c["z7"])
    c["u2"] = up(c["a7"], n // 2)
    c["z8"] = conv3(c["u2"], P["L8"][0], n, P["L8"][1]) + c["a2"]; c["a8"] = relu(c["z8"])
    c["z9"] = conv3(c["a8"], P["L9"][0], n, P["L9"][1]); c["a9"] = relu(c["z9"])
    y = conv3(c["a9"], P["L10"][0], n, P["L10"][1])
    return y, c


def loss_and_grad_y(y, target):
    """Loss = sum_{v, c < 4} (y - t)^2 / (4 V) and its gradient in y."""
    V = y.shape[0]
    d = np.zeros_like(y)
    d[:, :OUT_USED] = y[:, :OUT_USED] - target[:, :OUT_USED]
    return float(np.sum(d * d) / (OUT_USED * V)), 2.0 * d / (OUT_USED * V)


def backward(params, cache, dy, n):
    """Gradients {name: (dW, db)} of the loss, given dL/dy."""
    P, c = params, cache
    g = {}

    def layer(name, inp, dz, m):
        g[name] = (conv3_wgrad(inp, dz, m), dz.sum(axis=0))
        return conv3_dgrad(dz, P[name][0], m)

    da9 = layer("L10", c["a9"], dy, n)
    dz9 = da9 * (c["z9"] > 0)
    da8 = layer("L9", c["a8"], dz9, n)
    dz8 = da8 * (c["z8"] > 0)
    du2 = layer("L8", c["u2"], dz8, n)
    da2_skip = dz8
    da7 = pool(du2, n) * 8.0                      # adjoint of up: sum over the 8 children
    dz7 = da7 * (c["z7"] > 0)
    da6 = layer("L7", c["a6"], dz7, n // 2)
    dz6 = da6 * (c["z6"] > 0)
    du1 = layer("L6", c["u1"], dz6, n // 2)
    da4_skip = dz6
    da5 = pool(du1, n // 2) * 8.0
    dz5 = da5 * (c["z5"] > 0)
    dp2 = layer("L5", c["p2"], dz5, n // 4)
    da4 = up(dp2, n // 4) / 8.0 + da4_skip        # adjoint of pool: spread / 8
    dz4 = da4 * (c["z4"] > 0)
    da3 = layer("L4", c["a3"], dz4, n // 2)
    dz3 = da3 * (c["z3"] > 0)
    dp1 = layer("L3", c["p1"], dz3, n // 2)
    da2 = up(dp1, n // 2) / 8.0 + da2_skip
    dz2 = da2 * (c["z2"] > 0)
    da1 = layer("L2", c["a1"], dz2, n)
    dz1 = da1 * (c["z1"] > 0)
    layer("L1", c["x"], dz1, n)
    return g


def adam_step(w, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns new (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------- solver <-> network
def _corner_mean(nodal, n):
    """Mean over the 8 corner nodes of every cell: nodal [C, (n+1)^3] -> [n^3, C]."""
    C = nodal.shape[0]
    g = nodal.reshape(C, n + 1, n + 1, n + 1)
    m = sum(g[:, a:a + n, b:b + n, c:c + n] for a in (0, 1) for b in (0, 1) for c in (0, 1)) / 8.0
    return m.reshape(C, n ** 3).T


def features(cell_mu, f_nodal, n):
    """Network input [n^3, 16]: log10 mu, the cell mean of the nodal forcing / fscale (3), a
    constant 1, zeros; fscale = max |f| over nodes and components (1 if f = 0)."""
    fscale = float(np.abs(f_nodal).max()) or 1.0
    x = np.zeros((n ** 3, CIN))
    x[:, 0] = np.log10(np.asarray(cell_mu, dtype=np.float64).ravel())
    x[:, 1:4] = _corner_mean(np.asarray(f_nodal).reshape(3, -1), n) / fscale
    x[:, 4] = 1.0
    return x, fscale


VEL_SCALE = 100.0  # velocity channels are VEL_SCALE u / fscale, pressure (p - mean p) / fscale


def target(x_nodes, fscale, n):
    """Training target [n^3, 16]: cell means of the nodal solution, channels 0..2 scaled to
    VEL_SCALE u / fscale, channel 3 = (p - mean over nodes of p) / fscale (the pressure is
    defined up to a constant without a traction face)."""
    x = np.asarray(x_nodes).reshape(4, -1).copy()
    x[3] -= x[3].mean()
    t = np.zeros((n ** 3, 16))
    t[:, :4] = _corner_mean(x, n) / fscale
    t[:, :3] *= VEL_SCALE
    return t


def to_nodes(y, fscale, n, constrained):
    """Initial guess on the nodes: mean of the prediction over the (1 to 8) cells around
    each node, unscaled (velocity / VEL_SCALE, times fscale); constrained velocity components
    set to zero.  SoA [4 (n+1)^3]."""
    g = y[:, :4].T.reshape(4, n, n, n)
    acc = np.zeros((4, n + 1, n + 1, n + 1))
    cnt = np.zeros((n + 1, n + 1, n + 1))
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                acc[:, a:a + n, b:b + n, c:c + n] += g
                cnt[a:a + n, b:b + n, c:c + n] += 1.0
    out = acc / cnt[None] * fscale
    out[:3] /= VEL_SCALE
    out = out.reshape(-1)
    out[np.asarray(constrained, dtype=bool)] = 0.0
    return out


def line_search(K, b, x):
    """The residual-minimising multiple of x: alpha x with alpha = (Kx, b) / (Kx, Kx)."""
    y = K @ x
    d = float(y @ y)
    return x * (float(y @ b) / d if d > 0 else 0.0)
