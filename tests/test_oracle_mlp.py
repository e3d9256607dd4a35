"""Pins of the learned-bound oracle (oracle/mlp.py) against facts outside it.

* the gradient against central finite differences of the loss (a dropped term,
  a wrong sign or a transposed weight in the backprop fails it);
* GELU against scipy's normal CDF and density;
* the pinball loss: its minimiser over a constant is the tau-quantile;
* Adam: bias correction makes every step of a constant gradient -lr sign(g);
* features: a hand-computed row, exact scale shifts by powers of two, and the
  weight bins against exact rational arithmetic;
* the y* quantile against simulation of the max of k Exp(1).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import mlp


def random_theta(rng, scale=0.3):
    return rng.normal(0.0, scale, size=mlp.P)


def random_batch(rng, n):
    X = np.column_stack([rng.uniform(2, 12, n), rng.uniform(2, 12, n), rng.uniform(0, 3, n),
                         rng.uniform(-3, 0, n), rng.uniform(-1, 1, n), rng.uniform(0, 2, n),
                         rng.uniform(1, 3, n), np.log(rng.choice([256, 1024, 4096], n))])
    return X


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(11)
    theta = random_theta(rng)
    X = random_batch(rng, 40)
    pred, _ = mlp.forward(theta, X)
    t = pred + rng.choice([-1, 1], 40) * rng.uniform(0.2, 1.0, 40)  # away from the kink
    tau = 0.9
    _, g = mlp.loss_and_grad(theta, X, t, tau)
    idx = np.concatenate([rng.choice(mlp.P, 300, replace=False), [mlp.P - 1], np.arange(512, 576)[:8]])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, X, t, tau)[0] - mlp.loss_and_grad(tm, X, t, tau)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_gelu_against_scipy():
    stats = pytest.importorskip("scipy.stats")
    x = np.linspace(-8, 8, 1001)
    assert np.allclose(mlp.gelu(x), x * stats.norm.cdf(x), rtol=1e-13, atol=1e-15)
    assert np.allclose(mlp.gelu_grad(x), stats.norm.cdf(x) + x * stats.norm.pdf(x), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("tau", [0.05, 0.5, 0.95])
def test_pinball_minimiser_is_the_quantile(tau):
    rng = np.random.default_rng(3)
    t = rng.gumbel(size=1001)
    q = np.quantile(t, tau, method="inverted_cdf")
    at_q = np.mean(mlp.pinball(t - q, tau))
    for c in np.linspace(q - 1, q + 1, 401):
        assert np.mean(mlp.pinball(t - c, tau)) >= at_q - 1e-12


def test_adam_constant_gradient_steps_by_lr_sign():
    rng = np.random.default_rng(4)
    g = rng.normal(size=mlp.P)
    theta = rng.normal(size=mlp.P)
    m = np.zeros(mlp.P)
    v = np.zeros(mlp.P)
    lr = 1e-2
    for step in range(1, 11):
        new, m, v = mlp.adam_step(theta, m, v, g, lr, step)
        assert np.allclose(new - theta, -lr * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8), rtol=1e-9, atol=1e-15)
        theta = new


def test_features_of_a_hand_computed_row():
    # weights 1, 2, 4, 8 (+ entries that do not count): n+ = 4, sum 15, max 8;
    # bins 0, 4, 8, 12; ranks ceil(0.4)=1, ceil(2)=2, ceil(3.6)=4, ceil(3.96)=4
    w = [1.0, 0.0, 2.0, -3.0, 4.0, float("nan"), 8.0, float("inf")]
    f = mlp.features(w, 1024)
    c = math.log(2.0) / 4.0
    want = [math.log(4), math.log(15), math.log(8), 0.5 * c, 4.5 * c, 12.5 * c, 12.5 * c, math.log(1024)]
    assert np.allclose(f, want, rtol=0, atol=1e-15)
    assert np.array_equal(mlp.features([], 64), [0, 0, 0, 0, 0, 0, 0, math.log(64)])
    assert np.array_equal(mlp.features([0.0, -1.0], 64), [0, 0, 0, 0, 0, 0, 0, math.log(64)])


def test_features_shift_exactly_under_power_of_two_scaling():
    rng = np.random.default_rng(5)
    w = rng.exponential(size=777)
    f = mlp.features(w, 256)
    for m in (-20, -1, 3, 40):
        g = mlp.features(w * 2.0 ** m, 256)
        assert g[0] == f[0] and g[7] == f[7]
        assert np.allclose(g[1:7] - f[1:7], m * math.log(2.0), rtol=0, atol=1e-12)


def test_weight_bins_against_exact_arithmetic():
    rng = np.random.default_rng(6)
    v = np.exp(rng.uniform(-80, 80, 3000))
    for x in v:
        b = mlp.weight_bin(x)
        X = Fraction(float(x)) ** 4
        assert Fraction(2) ** b <= X < Fraction(2) ** (b + 1), x  # 2^(b/4) <= x < 2^((b+1)/4)
    # the quarter-octave boundaries are the doubles nearest 2^(j/4)
    for j in (1, 2, 3):
        r = 2.0 ** (j / 4.0)
        assert mlp.weight_bin(r) == j and mlp.weight_bin(np.nextafter(r, 0)) == j - 1
        assert mlp.weight_bin(r * 2.0 ** -7) == j - 28
    assert mlp.weight_bin(5e-324) == -512 and mlp.weight_bin(1e300) == 511 and mlp.weight_bin(1.0) == 0


@pytest.mark.parametrize("k", [1, 16, 1024])
def test_ystar_quantile_against_simulation(k):
    rng = np.random.default_rng(7)
    n = 20000
    mx = rng.exponential(size=(n, k)).max(axis=1)
    for p in (0.05, 0.5, 0.95):
        q = math.exp(mlp.ystar_quantile(p, k))
        frac = np.mean(mx <= q)
        assert abs(frac - p) < 4 * math.sqrt(p * (1 - p) / n) + 1e-3, (p, frac)
