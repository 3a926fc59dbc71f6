"""FP64 reference of the learned law's perceptron (10 -> 64 -> 64 -> 64 -> 10,
ReLU) for the tests: loss and its gradient by plain backpropagation, in the
parameter exchange order of include/pdn_surrogate.h.

With ``bf16=True`` the operands the GPU kernels feed to the tensor cores are
rounded to bfloat16 at the same places (weights, the input, each hidden
activation, and each backpropagated gradient before it enters a product); the
sums stay FP64.  Without it the whole computation is FP64.  The analytic
gradient of the FP64 version is pinned against central finite differences in
tests/test_mlp_reference.py."""
import numpy as np

SHAPES = [(64, 10), (64,), (64, 64), (64,), (64, 64), (64,), (10, 64), (10,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)


def unpack(p):
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(p[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(a, dtype=np.float64).ravel() for a in parts])


def bf16(a):
    """Round float64 values to the nearest bfloat16 (ties to even), via float32."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def loss_and_grad(p, xn, tn, bf=False):
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(p)
    q = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    x0 = q(xn)
    Wq = [q(W) for W in (W1, W2, W3, W4)]
    z1 = x0 @ Wq[0].T + b1
    a1 = q(np.maximum(z1, 0.0))
    z2 = a1 @ Wq[1].T + b2
    a2 = q(np.maximum(z2, 0.0))
    z3 = a2 @ Wq[2].T + b3
    a3 = q(np.maximum(z3, 0.0))
    y = a3 @ Wq[3].T + b4
    n = xn.shape[0]
    d = y - tn
    loss = float(np.sum(d * d) / (n * 10))
    dy = 2.0 * d / (n * 10)
    dyq = q(dy)
    gW4, gb4 = dyq.T @ a3, dy.sum(0)
    dz3 = (dyq @ Wq[3]) * (a3 > 0) if bf else (dyq @ Wq[3]) * (z3 > 0)
    dz3q = q(dz3)
    gW3, gb3 = dz3q.T @ a2, dz3.sum(0)
    dz2 = (dz3q @ Wq[2]) * ((a2 > 0) if bf else (z2 > 0))
    dz2q = q(dz2)
    gW2, gb2 = dz2q.T @ a1, dz2.sum(0)
    dz1 = (dz2q @ Wq[1]) * ((a1 > 0) if bf else (z1 > 0))
    dz1q = q(dz1)
    gW1, gb1 = dz1q.T @ x0, dz1.sum(0)
    return loss, pack([gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4])


def forward(p, xn):
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(p)
    a = np.maximum(xn @ W1.T + b1, 0.0)
    a = np.maximum(a @ W2.T + b2, 0.0)
    a = np.maximum(a @ W3.T + b3, 0.0)
    return a @ W4.T + b4


def forward_bf16(p, xn):
    """Forward pass with the operands of the tensor-core products rounded to
    bfloat16 (weights, the input, each hidden activation after the ReLU),
    sums and biases in FP64."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(p)
    a = bf16(xn)
    a = bf16(np.maximum(a @ bf16(W1).T + b1, 0.0))
    a = bf16(np.maximum(a @ bf16(W2).T + b2, 0.0))
    a = bf16(np.maximum(a @ bf16(W3).T + b3, 0.0))
    return a @ bf16(W4).T + b4
