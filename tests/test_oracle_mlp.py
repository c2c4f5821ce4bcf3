"""Pins for the oracle's RPNN (Sec. 4.3, Fig. 6), its loss (Sec. 5.2) and Adam.

Each forward pin is a special case of the weights that reduces the network to a
small composition computed here with numpy matrix products; the backward is
pinned by central finite differences of the forward."""
import numpy as np

from paper_1709_05418_gb300 import workloads as W

SMALL = dict(K_=3, din=5, H_=4, ntail=3)
SMALL_O = dict(K=3, din=5, H=4, ntail=3)


def relu(a):
    return np.maximum(a, 0.0)


def zero_parts(**kw):
    return {n: np.zeros(s) for n, s, _ in W.param_shapes(**kw)}


def test_param_count(orc):
    assert orc.net_param_count() == 1_296_601 == W.param_count()
    # 23 layers: 10 two-layer blocks + 3 standard layers; about 1.4 M parameters
    assert len([n for n, _, _ in W.param_shapes() if not n.startswith("b")]) == 10 * 2 + 9 + 3
    assert 1.2e6 < orc.net_param_count() < 1.45e6


def test_zero_weights_give_relu_of_output_bias(orc):
    p = zero_parts()
    p["bT3"][:] = 0.37
    z = np.random.default_rng(0).normal(size=(3, 10, 226))
    g = orc.mlp_forward(W.join_params(p), z)
    assert np.all(g == 0.37)
    p["bT3"][:] = -0.2
    assert np.all(orc.mlp_forward(W.join_params(p), z) == 0.0)


def test_only_block_k_reads_level_k(orc):
    # block k alone active with W2 = I: o^k = relu(relu(V z^k + b1) + o^{k-1}); later
    # blocks pass o through (F2 = 0 and o >= 0); tail = identity, identity, sum
    rng = np.random.default_rng(1)
    H = 200
    z = rng.normal(size=(4, 10, 226))
    for k in (1, 4, 10):
        p = zero_parts()
        V = rng.normal(size=(H, 226)) * 0.1
        b1 = rng.normal(size=H) * 0.1
        p[f"V{k}"], p[f"b1_{k}"], p[f"W2_{k}"] = V, b1, np.eye(H)
        p["T1"], p["T2"] = np.eye(H), np.eye(H)
        w = rng.normal(size=(1, H))
        p["T3"], p["bT3"] = w, np.array([5.0])
        exp = relu(relu(relu(z[:, k - 1] @ V.T + b1)) @ w.T + 5.0)[:, 0]
        np.testing.assert_allclose(orc.mlp_forward(W.join_params(p), z), exp, rtol=1e-13)


def test_block_recurrence_and_residual(orc):
    # blocks 1 and 2 active: o1 = relu(W2a relu(Va z1 + b1a) + b2a),
    # o2 = relu(W2b relu(Vb z2 + W1b o1 + b1b) + b2b + o1); tail relu layers
    rng = np.random.default_rng(2)
    H = 200
    p = zero_parts()
    for k in (1, 2):
        p[f"V{k}"] = rng.normal(size=(H, 226)) * 0.05
        p[f"b1_{k}"] = rng.normal(size=H) * 0.1
        p[f"W2_{k}"] = rng.normal(size=(H, H)) * 0.07
        p[f"b2_{k}"] = rng.normal(size=H) * 0.1
    p["W1_2"] = rng.normal(size=(H, H)) * 0.07
    for t in (1, 2):
        p[f"T{t}"] = rng.normal(size=(H, H)) * 0.1
        p[f"bT{t}"] = rng.normal(size=H) * 0.1
    p["T3"], p["bT3"] = rng.normal(size=(1, H)), np.array([3.0])
    z = rng.normal(size=(5, 10, 226))
    o1 = relu(relu(z[:, 0] @ p["V1"].T + p["b1_1"]) @ p["W2_1"].T + p["b2_1"])
    f1 = relu(z[:, 1] @ p["V2"].T + o1 @ p["W1_2"].T + p["b1_2"])
    o = relu(f1 @ p["W2_2"].T + p["b2_2"] + o1)
    o = relu(o @ p["T1"].T + p["bT1"])
    o = relu(o @ p["T2"].T + p["bT2"])
    exp = relu(o @ p["T3"].T + p["bT3"])[:, 0]
    np.testing.assert_allclose(orc.mlp_forward(W.join_params(p), z), exp, rtol=1e-12)


def test_positive_homogeneity_without_biases(orc):
    params = W.he_init(seed=3, bias=0.0).astype(np.float64)
    z = np.random.default_rng(4).uniform(0, 2, size=(6, 10, 226))
    g1 = orc.mlp_forward(params, z)
    g2 = orc.mlp_forward(params, 2.5 * z)
    np.testing.assert_allclose(g2, 2.5 * g1, rtol=1e-12, atol=1e-14)


def _fd_check(orc, params, z, dg, idx, h=1e-6, **net):
    ana = orc.mlp_backward(params, z, dg, **net)
    for i in idx:
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        num = (np.dot(dg, orc.mlp_forward(pp, z, **net)) - np.dot(dg, orc.mlp_forward(pm, z, **net))) / (2 * h)
        assert abs(num - ana[i]) <= 1e-6 * max(1.0, abs(num)), (i, num, ana[i])
    return ana


def test_backward_matches_finite_differences_small_net(orc):
    rng = np.random.default_rng(5)
    params = W.he_init(seed=6, bias=0.05, **SMALL).astype(np.float64)
    z = rng.uniform(0.1, 2, size=(7, 3, 5))
    dg = rng.normal(size=7)
    _fd_check(orc, params, z, dg, range(params.size), **SMALL_O)


def test_backward_matches_finite_differences_full_net(orc):
    rng = np.random.default_rng(7)
    params = W.he_init(seed=8, bias=0.01).astype(np.float64) * 0.6
    z = rng.uniform(0.0, 2.0, size=(2, 10, 226))
    dg = np.array([1.0, -0.5])
    assert np.all(orc.mlp_forward(params, z) > 0)
    idx = rng.choice(params.size, size=60, replace=False)
    idx = np.concatenate([idx, [0, params.size - 1, params.size - 2]])
    _fd_check(orc, params, z, dg, idx)


def test_logmse_loss_and_gradient(orc):
    e = np.e
    l, dg = orc.logmse_loss(np.array([e - 1.0, 0.0]), np.array([0.0, e - 1.0]))
    assert abs(l - 1.0) < 1e-15                 # ((1 - 0)^2 + (0 - 1)^2) / 2
    rng = np.random.default_rng(9)
    g = rng.uniform(0, 3, 10)
    t = rng.uniform(0, 3, 10)
    _, dg = orc.logmse_loss(g, t)
    for i in range(10):
        gp, gm = g.copy(), g.copy()
        gp[i] += 1e-6
        gm[i] -= 1e-6
        num = (orc.logmse_loss(gp, t, False) - orc.logmse_loss(gm, t, False)) / 2e-6
        assert abs(num - dg[i]) < 1e-8


def test_adam_hand_values(orc):
    p = np.array([1.0, -2.0, 0.5])
    m = np.zeros(3)
    v = np.zeros(3)
    g1 = np.array([0.5, -1.0, 0.0])
    orc.adam(p, m, v, g1, 1, lr=0.1)
    # step 1: m_hat = g, v_hat = g^2 -> p -= lr * g / (|g| + eps)
    np.testing.assert_allclose(p, [1.0 - 0.1 * 0.5 / (0.5 + 1e-8), -2.0 + 0.1 * 1.0 / (1.0 + 1e-8), 0.5],
                               rtol=0, atol=1e-15)
    g2 = np.array([0.25, 1.0, 2.0])
    orc.adam(p, m, v, g2, 2, lr=0.1)
    m2 = 0.9 * 0.1 * g1 + 0.1 * g2
    v2 = 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2
    mh, vh = m2 / (1 - 0.81), v2 / (1 - 0.999 ** 2)
    p_exp = np.array([1.0 - 0.1 * 0.5 / (0.5 + 1e-8), -2.0 + 0.1 / (1.0 + 1e-8), 0.5]) - 0.1 * mh / (np.sqrt(vh) + 1e-8)
    np.testing.assert_allclose(p, p_exp, rtol=1e-14)


def test_mixed_precision_reference_without_rounding_is_the_oracle(orc):
    """The BF16-arithmetic reference the BF16 training kernels are checked against is, with
    its rounding switched off, the oracle's network and chain rule (so a dropped term or a
    transposed product in it would show here); with rounding on it moves the gradient."""
    from mixed_precision_ref import forward_backward
    rng = np.random.default_rng(8)
    params = W.he_init(seed=4)
    params[W.param_count() - 1] = 0.3              # keep the output ReLU active
    z = rng.uniform(0.0, 1.5, size=(7, 10, 226))
    dout = rng.normal(size=7)
    g, dp = forward_backward(params, z, dout, bf16=False)
    assert np.allclose(g, orc.mlp_forward(params.astype(np.float64), z), rtol=1e-12, atol=1e-12)
    ref = orc.mlp_backward(params.astype(np.float64), z, dout)
    assert np.allclose(dp, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
    _, dp16 = forward_backward(params, z, dout, bf16=True)
    assert 1e-5 < np.linalg.norm(dp16 - ref) / np.linalg.norm(ref) < 0.5


def test_dense_mlp_reduces_to_hand_computation(orc):
    """One hidden unit: g = relu(wo * relu(w . x + b) + bo), by hand."""
    x = np.array([[0.5, -1.0, 2.0], [1.0, 1.0, 1.0]])
    w, b, wo, bo = np.array([0.3, 0.2, -0.1]), 0.05, 1.5, -0.01
    params = np.concatenate([w, [b], [wo], [bo]])
    g, _ = orc.dense_forward(params, [1], x)
    h = np.maximum(x @ w + b, 0.0)
    assert np.allclose(g, np.maximum(wo * h + bo, 0.0), rtol=0, atol=1e-15)
    # no hidden layer: a single ReLU unit on the input
    g0, _ = orc.dense_forward(np.array([0.1, -0.2, 0.3, 0.4]), [], x)
    assert np.allclose(g0, np.maximum(x @ [0.1, -0.2, 0.3] + 0.4, 0.0))


def test_dense_mlp_backward_matches_finite_differences(orc):
    rng = np.random.default_rng(12)
    widths, din = [6, 5, 4], 7
    n = din * 6 + 6 + 6 * 5 + 5 + 5 * 4 + 4 + 4 + 1
    params = rng.normal(scale=0.6, size=n)
    params[-1] = 0.5
    x = rng.uniform(-1.0, 1.0, size=(9, din))
    dout = rng.normal(size=9)
    grad = orc.dense_backward(params, widths, x, dout)
    h = 1e-6
    fd = np.zeros(n)
    for i in range(n):
        e = np.zeros(n); e[i] = h
        fp = orc.dense_forward(params + e, widths, x)[0] @ dout
        fm = orc.dense_forward(params - e, widths, x)[0] @ dout
        fd[i] = (fp - fm) / (2 * h)
    assert np.allclose(grad, fd, rtol=1e-6, atol=1e-7)
