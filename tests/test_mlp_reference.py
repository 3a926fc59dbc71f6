"""The FP64 backpropagation of tests/mlp_reference.py (used to check the GPU
gradients of the learned law) against central finite differences of its own
loss, and its bfloat16 rounding against the format's definition."""
import numpy as np

import mlp_reference as R


def _case(seed, n=64):
    rng = np.random.default_rng(seed)
    p = rng.normal(size=R.N_PARAMS) * 0.3
    xn = rng.normal(size=(n, 10))
    tn = rng.normal(size=(n, 10))
    return p, xn, tn


def test_parameter_count():
    assert R.N_PARAMS == 9674


def test_gradient_matches_central_differences():
    p, xn, tn = _case(3)
    _, g = R.loss_and_grad(p, xn, tn)
    rng = np.random.default_rng(4)
    # every block of the exchange order, a few entries each
    offs = np.cumsum([0] + [int(np.prod(s)) for s in R.SHAPES])
    idx = np.concatenate([rng.integers(offs[k], offs[k + 1], size=3) for k in range(len(R.SHAPES))])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        num = (R.loss_and_grad(pp, xn, tn)[0] - R.loss_and_grad(pm, xn, tn)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, num, g[i])


def test_gradient_of_a_linear_output_layer():
    """With every hidden unit active the output-layer gradients reduce to the
    least-squares normal equations: dL/dW4 = 2/(n*10) (Y - T)^T A3."""
    p, xn, tn = _case(5, n=32)
    W1, b1, W2, b2, W3, b3, W4, b4 = R.unpack(p)
    b1[:] = 50.0  # large biases and positive inner weights: all units positive
    b2[:] = 50.0
    b3[:] = 50.0
    W2, W3 = np.abs(W2), np.abs(W3)
    p = R.pack([W1, b1, W2, b2, W3, b3, W4, b4])
    a1 = xn @ W1.T + b1
    a2 = a1 @ W2.T + b2
    a3 = a2 @ W3.T + b3
    assert (a1 > 0).all() and (a2 > 0).all() and (a3 > 0).all()
    y = a3 @ W4.T + b4
    _, g = R.loss_and_grad(p, xn, tn)
    gW4 = R.unpack(g)[6]
    assert np.allclose(gW4, 2.0 / (32 * 10) * (y - tn).T @ a3, rtol=1e-12, atol=1e-12)


def test_bf16_rounding():
    # exactly representable values stay, ties go to even, 8 significant bits
    assert R.bf16(np.array([1.0, -2.5, 0.0]))[1] == -2.5
    assert R.bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0          # tie -> even (1.0)
    assert R.bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6  # tie -> even (odd neighbour below)
    assert R.bf16(np.array([1.0 + 2.0 ** -7]))[0] == 1.0 + 2.0 ** -7
    x = np.random.default_rng(0).normal(size=1000)
    r = R.bf16(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8 + 1e-300)
