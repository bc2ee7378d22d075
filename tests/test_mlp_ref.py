"""Pins of the FP64 surrogate-network reference against what mathematics fixes:
central differences of its own loss, explicit loops for the forward pass, and
the bfloat16 rounding rule."""
import numpy as np

import mlp_ref as M


def _loop_forward(P, x):
    """One sample through the network with explicit index loops."""
    p = M.unpack(P)
    a = list(x)
    for l in (1, 2, 3):
        W, b = p[f"W{l}"], p[f"b{l}"]
        z = [b[j] + sum(W[j][k] * a[k] for k in range(len(a))) for j in range(W.shape[0])]
        a = [zz / (1.0 + np.exp(-zz)) for zz in z]
    W, b = p["W4"], p["b4"]
    return np.array([b[j] + sum(W[j][k] * a[k] for k in range(len(a))) for j in range(W.shape[0])])


def _random(seed, n):
    rng = np.random.Generator(np.random.PCG64(seed))
    P = M.init_params(seed).astype(np.float64)
    P += rng.normal(0, 0.05, P.size)   # non-zero biases too
    X = rng.normal(0, 1, (n, M.N_IN))
    Y = rng.normal(0, 1, (n, M.N_OUT))
    return P, X, Y


def test_parameter_count_and_layout():
    assert M.NPARAMS == 9412 and M.NNORM == 36
    P = np.arange(M.NPARAMS, dtype=np.float64)
    d = M.unpack(P)
    assert d["W1"][1, 0] == 12 and d["b1"][0] == 768 and d["b4"][-1] == M.NPARAMS - 1
    assert np.array_equal(M.pack(d), P)


def test_forward_matches_loops():
    P, X, _ = _random(3, 3)
    out, _ = M.forward(P, X)
    for i in range(3):
        assert np.allclose(out[i], _loop_forward(P, X[i]), rtol=1e-12, atol=1e-12)


def test_gradient_matches_central_differences():
    P, X, Y = _random(5, 7)
    loss, g = M.loss_grad(P, X, Y)
    rng = np.random.Generator(np.random.PCG64(9))
    # every bias and a sample of every weight matrix
    idx = list(range(768, 832)) + list(range(9408, 9412))
    for lo, hi in ((0, 768), (832, 4928), (4992, 9088), (9152, 9408)):
        idx += list(rng.choice(np.arange(lo, hi), 24, replace=False))
    h = 1e-6
    for i in idx:
        e = np.zeros_like(P)
        e[i] = h
        num = (M.loss_grad(P + e, X, Y)[0] - M.loss_grad(P - e, X, Y)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1e-3, abs(num)), (i, num, g[i])


def test_loss_is_mean_square():
    P, X, Y = _random(6, 5)
    out, _ = M.forward(P, X)
    loss, _ = M.loss_grad(P, X, Y)
    assert np.isclose(loss, np.mean((out - Y) ** 2), rtol=1e-14)


def test_bf16_rounding():
    v = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -8 + 2.0 ** -20, -3.0, 0.0, 65280.0])
    r = M.bf16(v)
    assert list(r) == [1.0, 1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, -3.0, 0.0, 65280.0]
    x = np.random.Generator(np.random.PCG64(1)).normal(0, 10, 10000)
    rel = np.abs(M.bf16(x) - x) / np.abs(x)
    assert rel.max() <= 2.0 ** -8 * (1 + 1e-6)


def test_output_transform_round_trip():
    norm = np.concatenate([np.zeros(12), np.ones(12), [0.1, -0.2, 0.3, 0.0], [2.0, 3.0, 4.0, 5.0],
                           [1e-5, 1e-5, 1e-5, 1e-4]])
    R = np.array([[-0.9, 1e-7, -3e-3, 0.5], [0.0, 0.2, 1e-9, -1e-6]])
    O = M.targets_to_output(R, norm)
    assert np.allclose(M.output_to_change(O, norm), R, rtol=1e-12, atol=1e-20)


def test_split_inputs_keep_sixteen_bits():
    v = np.random.Generator(np.random.PCG64(2)).normal(0, 3, 10000).astype(np.float32)
    rel = np.abs(M.split_bf16(v) - v) / np.abs(v)
    assert rel.max() <= 2.0 ** -16
