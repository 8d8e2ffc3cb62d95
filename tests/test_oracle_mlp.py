"""Pin of the MLP oracle: its backpropagated FP64 gradient equals central
finite differences of its own FP64 loss (no GPU)."""
import numpy as np

from oracle import mlp


def test_mlp_oracle_gradient_is_the_loss_derivative():
    rng = np.random.default_rng(3)
    nin, width, depth, nout = 2, 8, 3, 5
    n = sum((nin if l == 0 else width) * (nout if l == depth else width) + (nout if l == depth else width)
            for l in range(depth + 1))
    p = rng.normal(scale=0.4, size=n)
    x = rng.uniform(-1, 1, size=(7, nin))
    y = rng.normal(size=(7, nout))
    wt = rng.uniform(0.5, 2.0, size=nout)
    loss, g = mlp.loss_and_grad(p, x, y, wt, nin, width, depth, nout)
    h = 1e-6
    for i in rng.choice(n, size=40, replace=False):
        e = np.zeros(n)
        e[i] = h
        lp, _ = mlp.loss_and_grad(p + e, x, y, wt, nin, width, depth, nout)
        lm, _ = mlp.loss_and_grad(p - e, x, y, wt, nin, width, depth, nout)
        assert abs((lp - lm) / (2 * h) - g[i]) <= 1e-7 * (1 + abs(g[i]))


def test_bf16_rounding_is_nearest_even():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.14159265], dtype=np.float32)
    r = mlp.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7 and r[3] == -2.5
    assert abs(r[4] - 3.140625) == 0.0
