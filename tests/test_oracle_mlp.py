"""Pins for the FP64 reference of the surrogate network: its gradient against
central finite differences of its own loss (a different computation: no
backpropagation), and the BF16 rounding against exactly representable cases."""
import numpy as np

from oracle import mlp


def test_bf16_rounding_ties_and_exact_values():
    exact = np.array([1.0, -2.5, 0.15625, 3.0e38], dtype=np.float32)
    assert np.array_equal(mlp.bf16_round(exact)[:3], exact[:3].astype(np.float64))
    one_plus = np.float32(1.0) + np.float32(2.0 ** -8)       # halfway between 1 and 1+2^-7: ties to even
    assert mlp.bf16_round(np.array([one_plus]))[0] == 1.0
    above = np.float32(1.0) + np.float32(2.0 ** -8) + np.float32(2.0 ** -20)
    assert mlp.bf16_round(np.array([above]))[0] == 1.0 + 2.0 ** -7


def test_backprop_matches_central_differences():
    rng = np.random.default_rng(3)
    flat = rng.standard_normal(mlp.NPARAM) * 0.1
    p = mlp.unpack(flat, round_weights=False)
    X = rng.standard_normal((6, mlp.IN))
    t = rng.standard_normal(6)
    _, g = mlp.loss_and_grad(p, X, t)
    gflat = mlp.pack(g)
    h = 1e-6
    offsets = {}
    o = 0
    for name, shape in mlp.SHAPES:
        offsets[name] = (o, int(np.prod(shape)))
        o += int(np.prod(shape))
    for name in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"):
        o, k = offsets[name]
        for j in rng.choice(k, size=min(k, 5), replace=False):
            fp, fm = flat.copy(), flat.copy()
            fp[o + j] += h
            fm[o + j] -= h
            lp, _ = mlp.loss_and_grad(mlp.unpack(fp, False), X, t)
            lm, _ = mlp.loss_and_grad(mlp.unpack(fm, False), X, t)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gflat[o + j]) <= 1e-6 * (1 + abs(fd)), (name, j, fd, gflat[o + j])
