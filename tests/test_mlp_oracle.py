"""Pins of the FP64 warm-start network oracle against facts that do not come from it:
finite differences, a different library routine, closed forms and invariances."""
import numpy as np
import pytest
import torch
from scipy import special

from oracle import mlp


def setup(n=24, seed=0):
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, 0.4, mlp.NPARAMS)
    x = np.column_stack([rng.uniform(0.125, 1, n), rng.uniform(0.5, 0.9, n),
                         rng.uniform(0.09, 0.14, n), rng.uniform(1, 20, n)])
    t = rng.normal(size=(n, 5)) * [0.01, 0.3, 1.0, 0.2, 0.5] + [0.0, -1.0, 5.0, 0.1, -5.0]
    return p, x, t, mlp.fit_scaling(x, t)


def test_packing_sizes():
    assert mlp.NPARAMS == 64 * 4 + 64 + 64 * 64 + 64 + 5 * 64 + 5 == 4805
    p = np.arange(mlp.NPARAMS, dtype=float)
    d = mlp.unpack(p)
    assert d["W1"][1, 0] == 4 and d["b1"][0] == 256 and d["W2"][0, 1] == 321
    assert d["b3"][-1] == mlp.NPARAMS - 1
    assert np.array_equal(mlp.pack(d), p)


def test_gelu_is_x_times_normal_cdf():
    """Against scipy's ndtr (a separate routine from math.erfc)."""
    z = np.linspace(-9, 9, 2001)
    assert np.allclose(mlp.gelu(z), z * special.ndtr(z), rtol=1e-13, atol=1e-300)
    assert mlp.gelu(0.0) == 0.0
    # gelu(z) - gelu(-z) = z, from Phi(z) + Phi(-z) = 1
    assert np.allclose(mlp.gelu(z) - mlp.gelu(-z), z, atol=1e-14)


def test_gelu_grad_matches_finite_differences():
    z = np.linspace(-6, 6, 241)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(z))) < 1e-8
    assert abs(mlp.gelu_grad(0.0) - 0.5) < 1e-16


def test_bf16_round_matches_torch():
    """Round-to-nearest-even, checked against torch's float32 -> bfloat16 conversion, on
    random values and on exact ties (low 16 bits 0x8000) of both parities."""
    rng = np.random.default_rng(3)
    v = rng.normal(0, 3, 20000).astype(np.float32)
    bits = rng.integers(0, 2 ** 31, 2000, dtype=np.uint64).astype(np.uint32)
    ties = ((bits & np.uint32(0xFFFF0000)) | np.uint32(0x8000)).view(np.float32)
    ties = ties[np.isfinite(ties)]
    for arr in (v, ties, np.array([0.0, -0.0, 1.0, 1.00390625, 1.005859375], np.float32)):
        ref = torch.from_numpy(arr.copy()).to(torch.bfloat16).to(torch.float64).numpy()
        assert np.array_equal(mlp.bf16_round(arr), ref)


def test_gradient_matches_central_differences():
    """Every one of the 4805 derivatives against a central difference of the loss."""
    p, x, t, sc = setup(n=12)
    L, g = mlp.gradient(p, x, t, sc)
    assert abs(L - mlp.loss(p, x, t, sc)) < 1e-15 * max(1.0, L)
    h = 1e-6
    fd = np.empty_like(p)
    for k in range(mlp.NPARAMS):
        e = np.zeros_like(p)
        e[k] = h
        fd[k] = (mlp.loss(p + e, x, t, sc) - mlp.loss(p - e, x, t, sc)) / (2 * h)
    scale = np.max(np.abs(g))
    assert np.max(np.abs(fd - g)) <= 1e-7 * scale
    assert np.count_nonzero(g) == mlp.NPARAMS


def test_bf16_gradient_is_gradient_at_rounded_weights():
    p, x, t, sc = setup()
    L1, g1 = mlp.gradient(p, x, t, sc, weights="bf16")
    L2, g2 = mlp.gradient(mlp.bf16_round(p), x, t, sc)
    assert L1 == L2 and np.array_equal(g1, g2)
    assert not np.array_equal(g1, mlp.gradient(p, x, t, sc)[1])


def test_zero_hidden_weights_give_bias_output():
    """With W3 = 0 the output is b3 for every row; the loss gradient of b3 is then
    2 (b3 - mean of standardised targets) / 5 and every other gradient vanishes."""
    p, x, t, sc = setup()
    d = mlp.unpack(p.copy())
    d["W3"][:] = 0.0
    q = mlp.pack(d)
    y, _ = mlp.forward(q, x, sc)
    assert np.array_equal(y, np.broadcast_to(d["b3"], y.shape))
    _, g = mlp.gradient(q, x, t, sc)
    gd = mlp.unpack(g)
    tn = (t - sc["out_mean"]) / sc["out_scale"]
    assert np.allclose(gd["b3"], 2.0 * (d["b3"] - tn.mean(axis=0)) / 5.0, atol=1e-15)
    for k in ("W1", "b1", "W2", "b2"):
        assert not np.any(gd[k])


def test_hidden_unit_permutation_invariance():
    """Permuting the units of a hidden layer (rows of its W and b, columns of the next W)
    leaves the output unchanged and permutes the gradient the same way."""
    p, x, t, sc = setup()
    d = mlp.unpack(p)
    perm = np.random.default_rng(1).permutation(64)
    e = {k: v.copy() for k, v in d.items()}
    e["W2"], e["b2"] = d["W2"][perm], d["b2"][perm]
    e["W3"] = d["W3"][:, perm]
    q = mlp.pack(e)
    assert np.allclose(mlp.forward(p, x, sc)[0], mlp.forward(q, x, sc)[0], rtol=1e-13,
                       atol=1e-13)
    gp = mlp.unpack(mlp.gradient(p, x, t, sc)[1])
    gq = mlp.unpack(mlp.gradient(q, x, t, sc)[1])
    assert np.allclose(gq["W2"], gp["W2"][perm], atol=1e-14)
    assert np.allclose(gq["W3"], gp["W3"][:, perm], atol=1e-14)


def test_standardisation_invariance():
    """fit_scaling makes the network blind to affine rescaling of inputs and targets:
    the loss is unchanged when x and t are scaled and shifted per column."""
    p, x, t, sc = setup()
    x2 = 3.0 * x - 1.0
    t2 = 0.5 * t + 7.0
    assert abs(mlp.loss(p, x2, t2, mlp.fit_scaling(x2, t2)) - mlp.loss(p, x, t, sc)) < 1e-12
    assert np.allclose(sc["in_mean"], x.mean(axis=0)) and np.allclose(sc["in_scale"], x.std(axis=0))


def test_adam_first_step_is_signed_learning_rate():
    """After one step the bias-corrected moments are g and g^2, so the update is
    lr g / (|g| + eps) (Kingma & Ba 2015, Sec. 2.1)."""
    g = np.array([3.0, -1e-3, 0.0, 2e-9])
    p1, m, v = mlp.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    assert np.allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_constant_gradient_steps_are_lr():
    """With a constant gradient, m_hat = g and v_hat = g^2 at every step."""
    p, m, v = np.zeros(2), np.zeros(2), np.zeros(2)
    g = np.array([0.5, -2.0])
    for k in range(1, 51):
        p, m, v = mlp.adam_step(p, g, m, v, k, lr=1e-3, eps=0.0)
    assert np.allclose(p, -50 * 1e-3 * np.sign(g), rtol=1e-12)


@pytest.mark.parametrize("weights", [None, "bf16"])
def test_training_fits_a_smooth_map(weights):
    """Full-batch Adam fits a smooth 4 -> 5 map of the input box well: loss falls by more
    than 100x in 1500 steps."""
    rng = np.random.default_rng(5)
    n = 64
    x = np.column_stack([rng.uniform(0.125, 1, n), rng.uniform(0.5, 0.9, n),
                         rng.uniform(0.09, 0.14, n), rng.uniform(1, 20, n)])
    t = np.column_stack([x[:, 0] * x[:, 1], np.sin(3 * x[:, 1]), x[:, 2] * 10 + x[:, 0],
                         np.log(x[:, 3]), x[:, 1] ** 2])
    sc = mlp.fit_scaling(x, t)
    p0 = rng.uniform(-1, 1, mlp.NPARAMS) * 0.25
    p, losses = mlp.train(p0, x, t, sc, 1500, lr=3e-3, weights=weights)
    assert losses[-1] < 1e-2 * losses[0]
    assert mlp.loss(p, x, t, sc, weights) < 1e-2 * losses[0]
