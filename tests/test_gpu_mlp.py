"""The warm-start network's CUDA kernels against the FP64 oracle (oracle/mlp.py):
forward, gradient (BF16 weights, FP32 accumulation), Adam training, determinism."""
import numpy as np
import pytest

from oracle import mlp as om
from paper_1211_6932_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def rows(n, seed):
    """Inputs over the parameter box of the workloads (a, T/Tc, sigma, viscosity ratio)
    and smooth targets of the size of the warm-start outputs."""
    rng = np.random.default_rng(seed)
    x = np.column_stack([rng.uniform(0.125, 1, n), rng.uniform(0.5, 0.9, n),
                         rng.uniform(0.088, 0.137, n), rng.uniform(1, 20, n)])
    t = np.column_stack([0.01 * x[:, 0] * x[:, 1], np.sin(3 * x[:, 1]) - 1.0,
                         3.0 / np.sqrt(x[:, 0]), 0.1 * x[:, 2] * x[:, 3], np.log(x[:, 3])])
    return x, t


def net(p, x, t, sc, max_rows=None):
    from paper_1211_6932_gb300 import Mlp
    m = Mlp(p, max_rows=max_rows or max(len(x), 8))
    m.set_scaling(sc["in_mean"], sc["in_scale"], sc["out_mean"], sc["out_scale"])
    m.set_data(x, t)
    return m


def test_fit_scaling_matches_oracle():
    from paper_1211_6932_gb300 import Mlp
    x, t = rows(77, 1)
    sc = om.fit_scaling(x, t)
    with Mlp(wl.mlp_init(0), max_rows=77) as m:
        m.fit_scaling(x, t)
        m.set_data(x, t)
        # the library's statistics equal the oracle's up to FP32 rounding of the scaling
        with net(wl.mlp_init(0), x, t, sc) as m2:
            assert np.allclose(m.predict(x), m2.predict(x), rtol=1e-6, atol=1e-9)
            assert m.gradient()[0] == pytest.approx(m2.gradient()[0], rel=1e-6)


@pytest.mark.parametrize("n", [1, 7, 8, 300])
def test_forward_matches_oracle(n):
    """Predictions (physical units) against the oracle evaluated with the same BF16
    weights: FP32 accumulation of 4 + 64 + 64 terms."""
    x, t = rows(max(n, 2), 2)
    x, t = x[:n], t[:n]
    sc = om.fit_scaling(*rows(64, 3))
    p = wl.mlp_init(4)
    with net(p, x, t, sc) as m:
        y = m.predict(x)
    ref = om.predict(p.astype(np.float64), x, sc, weights="bf16")
    err = np.abs(y - ref) / sc["out_scale"]
    assert err.max() <= 2e-6


def test_bf16_copy_is_round_to_nearest_even():
    from paper_1211_6932_gb300 import Mlp
    p = (np.random.default_rng(5).normal(0, 1, om.NPARAMS)).astype(np.float32)
    with Mlp(wl.mlp_init(0), max_rows=4) as m:
        m.set_params(p)
        assert np.array_equal(m.params("master"), p)
        assert np.array_equal(m.params("bf16").astype(np.float64), om.bf16_round(p))


def test_gradient_exact_fp32_variant():
    """Against the oracle's gradient at the same (BF16-rounded) weights: the only
    difference is FP32 versus FP64 arithmetic, bound 1e-5 relative."""
    x, t = rows(256, 6)
    sc = om.fit_scaling(x, t)
    p = wl.mlp_init(7)
    with net(p, x, t, sc) as m:
        L, g = m.gradient()
    Lr, gr = om.gradient(p.astype(np.float64), x, t, sc, weights="bf16")
    assert abs(L - Lr) <= 1e-5 * Lr
    assert np.max(np.abs(g - gr)) <= 1e-5 * np.max(np.abs(gr))


def test_gradient_bf16_against_fp64_weights():
    """Against the oracle's gradient at the unrounded weights: BF16 weights move the
    gradient by well under 1e-2 (relative, in norm and per component scale)."""
    x, t = rows(256, 8)
    sc = om.fit_scaling(x, t)
    p = wl.mlp_init(9)
    with net(p, x, t, sc) as m:
        L, g = m.gradient()
    Lr, gr = om.gradient(p.astype(np.float64), x, t, sc)
    assert abs(L - Lr) <= 1e-2 * Lr
    assert np.linalg.norm(g - gr) <= 1e-2 * np.linalg.norm(gr)


def test_adam_training_matches_oracle():
    """60 full-batch Adam updates (one 50-update graph replay and 10 single updates)
    against the oracle's Adam in FP64 with the same BF16 weight rounding: the loss
    trajectories agree to 1e-3 and all but a few parameters to 1e-5."""
    x, t = rows(200, 10)
    sc = om.fit_scaling(x, t)
    p = wl.mlp_init(11)
    lr = 1e-3
    with net(p, x, t, sc) as m:
        losses = m.train(60, lr=lr)
        pg = m.params("master")
        assert m.update_count == 60
    pr, lr_ref = om.train(p.astype(np.float64), x, t, sc, 60, lr=lr, weights="bf16")
    assert np.max(np.abs(losses - lr_ref) / lr_ref) <= 1e-3
    d = np.abs(pg - pr)
    assert np.mean(d > 1e-5) <= 0.01 and d.max() <= 60 * 2 * lr


def test_training_is_deterministic_and_graph_equals_eager():
    from paper_1211_6932_gb300 import Mlp  # noqa: F401
    x, t = rows(100, 12)
    sc = om.fit_scaling(x, t)
    p = wl.mlp_init(13)
    with net(p, x, t, sc) as a, net(p, x, t, sc) as b, net(p, x, t, sc) as c:
        la = a.train(100, lr=3e-3)                          # two graph replays
        lb = np.concatenate([b.train(1, lr=3e-3) for _ in range(100)])  # single updates
        lc = c.train(100, lr=3e-3)
        assert np.array_equal(la, lb) and np.array_equal(la, lc)
        for w in ("master", "m", "v", "bf16"):
            assert np.array_equal(a.params(w), b.params(w))


def test_training_fits_and_predict_leaves_data_alone():
    x, t = rows(256, 14)
    sc = om.fit_scaling(x, t)
    with net(wl.mlp_init(15), x, t, sc) as m:
        L0, _ = m.gradient()
        losses = m.train(1500, lr=3e-3)
        assert losses[0] == pytest.approx(L0, rel=1e-6)
        L1, _ = m.gradient()
        assert L1 < 1e-2 * L0
        m.predict(rows(50, 16)[0])  # predictions use their own input buffer
        assert m.gradient()[0] == L1
        y = m.predict(x)
        assert np.sqrt(np.mean(((y - t) / sc["out_scale"]) ** 2)) < 0.1


def test_argument_errors():
    from paper_1211_6932_gb300 import LbmError, Mlp
    x, t = rows(10, 17)
    with Mlp(wl.mlp_init(0), max_rows=8) as m:
        with pytest.raises(LbmError) as ei:
            m.set_data(x, t)
        assert ei.value.code == -1
        with pytest.raises(LbmError) as ei:
            m.train(5)
        assert ei.value.code == -1
        with pytest.raises(LbmError):
            m.set_scaling([0] * 4, [1, 1, 0, 1], [0] * 5, [1] * 5)
