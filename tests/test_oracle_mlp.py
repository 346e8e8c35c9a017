"""Pins of the oracle's learned-guess pieces (CPU): the network's
backpropagation against finite differences, its small-weight (linear)
limit, bfloat16 rounding against torch's conversion, the ten inputs against
closed forms of special relativistic MHD and of the Kerr-Schild metric, and
the targets against the Lorentz factor from u^t."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_1912_10192_gb300 import workloads as W


def _rand_params(seed, scale=0.4):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0.0, scale, M.N_PARAMS)
    norm = np.concatenate([rng.normal(0, 1, 10), rng.uniform(0.5, 2.0, 10), rng.normal(0, 1, 2),
                           rng.uniform(0.5, 2.0, 2)])
    return theta, norm


def test_backprop_matches_central_differences():
    theta, norm = _rand_params(1)
    rng = np.random.default_rng(2)
    F = rng.normal(0.0, 1.5, (16, 10))
    T = rng.normal(0.0, 1.0, (16, 2))
    L, g = M.loss_and_grad(theta, norm, F, T)
    h = 1e-4
    idx = np.concatenate([rng.choice(M.N_PARAMS, 300, replace=False), np.arange(M.N_PARAMS - 130, M.N_PARAMS)])

    def at(i, dx):
        t = theta.copy()
        t[i] += dx
        return M.loss_and_grad(t, norm, F, T)[0]
    for i in idx:
        # fourth-order central difference: truncation O(h^4), rounding O(eps / h)
        fd = (-at(i, 2 * h) + 8 * at(i, h) - 8 * at(i, -h) + at(i, -2 * h)) / (12 * h)
        assert abs(fd - g[i]) <= 1e-8 * max(1e-3, abs(g[i])) + 1e-11, (i, fd, g[i])


def test_loss_is_half_the_mean_square_over_outputs():
    """loss_and_grad's loss equals the mean square error of the standardised outputs (loss())."""
    theta, norm = _rand_params(3)
    rng = np.random.default_rng(4)
    F = rng.normal(0.0, 1.0, (32, 10))
    T = rng.normal(0.0, 1.0, (32, 2))
    assert abs(M.loss_and_grad(theta, norm, F, T)[0] - M.loss(theta, norm, F, T)) < 1e-13


def test_small_weights_give_the_linear_composition():
    eps = 1e-3
    theta, norm = _rand_params(5, scale=1.0)
    parts = M.unpack(theta)
    lin = [p * eps if p.ndim == 2 else np.zeros_like(p) for p in parts]
    th = M.pack(lin)
    norm = np.concatenate([np.zeros(10), np.ones(10), np.zeros(2), np.ones(2)])
    rng = np.random.default_rng(6)
    F = rng.normal(0.0, 1.0, (8, 10))
    y = M.forward(th, norm, F)
    W1, _, W2, _, W3, _, W4, _ = lin
    ylin = np.array([W4 @ (W3 @ (W2 @ (W1 @ f))) for f in F])
    # tanh(z) = z (1 + O(z^2)), z ~ 1e-2 here
    assert np.max(np.abs(y - ylin)) < 1e-4 * np.max(np.abs(ylin))


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.normal(0, 10, 20000).astype(np.float32),
                        np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -1.0 - 2 ** -8, 0.0, -0.0, 65504.0,
                                  1e-30, -3.0e38], dtype=np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    got = M.bf16_round(x)
    assert np.array_equal(got, ref)
    assert M.bf16_round(np.float32(1.0 + 2 ** -8)) == 1.0          # tie -> even
    assert M.bf16_round(np.float32(1.0 + 3 * 2 ** -8)) == 1.0 + 2 ** -6  # tie -> even (up)


def _flat_desc(gam=5.0 / 3.0):
    return O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_MINKOWSKI, gam=gam)


def test_features_at_rest_in_flat_space():
    gam = 5.0 / 3.0
    d = _flat_desc(gam)
    rho, u = 0.3, 0.02
    pr = np.array([[rho, u, 0, 0, 0, 0, 0, 0]], dtype=np.float64)
    x1, x2 = np.array([0.7]), np.array([0.2])
    U = O.p2u_many(d, pr, x1, x2)
    f = O.mlp_features(d, U, np.zeros((1, 3)), x1, x2)[0]
    tiny = math.log(1e-30)
    expect = [math.log(rho), math.log(u / rho), tiny, 0.0, math.log((gam - 1.0) * u / rho), tiny, 1.0, tiny,
              0.0, 0.7]
    assert np.allclose(f, expect, rtol=1e-12, atol=1e-12), (f, expect)


def test_features_of_a_moving_magnetised_state_match_srmhd():
    """Noble et al. (2006) energy and momentum relations in special relativity:
    -Q.n = W - p + B^2 (1 + v^2)/2 - (v.B)^2/2, Q.B = W (v.B),
    Qt^2 = v^2 (B^2 + W)^2 - (v.B)^2 (B^2 + 2W)."""
    gam = 4.0 / 3.0
    d = _flat_desc(gam)
    rng = np.random.default_rng(8)
    for _ in range(20):
        rho = 10 ** rng.uniform(-3, 0)
        u = rho * 10 ** rng.uniform(-3, 1)
        ut = rng.normal(0, 2.0, 3)
        B = rng.normal(0, 1.0, 3) * math.sqrt(rho)
        pr = np.array([[rho, u, *ut, *B]])
        U = O.p2u_many(d, pr, np.array([0.0]), np.array([0.0]))
        f = O.mlp_features(d, U, B[None, :], np.array([0.0]), np.array([0.0]))[0]
        g = math.sqrt(1.0 + ut @ ut)
        v = ut / g
        vsq = v @ v
        p = (gam - 1.0) * u
        Wn = (rho + u + p) * g * g
        D = rho * g
        vB = v @ B
        Bsq = B @ B
        E = Wn - p + 0.5 * Bsq * (1.0 + vsq) - 0.5 * vB * vB
        Qtsq = vsq * (Bsq + Wn) ** 2 - vB * vB * (Bsq + 2.0 * Wn)
        QB = Wn * vB
        kappa = p / rho ** gam
        assert abs(f[0] - math.log(D)) < 1e-12
        assert abs(f[1] - math.log((E - D) / D)) < 1e-9
        assert abs(f[2] - math.log(Qtsq / D ** 2 + 1e-30)) < 1e-9
        assert abs(f[3] - QB * QB / (Qtsq * Bsq)) < 1e-9
        assert abs(f[4] - (math.log(kappa) + (gam - 1.0) * math.log(D))) < 1e-9
        assert abs(f[5] - math.log(Bsq / D)) < 1e-12


def test_metric_invariants_in_kerr_schild():
    a = 0.9375
    d = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=a, gam=13.0 / 9.0)
    prim, x1, x2 = W.random_states(50, seed=9, a=a)
    U = O.p2u_many(d, prim, x1, x2)
    f = O.mlp_features(d, U, prim[:, 5:8], x1, x2)
    r = np.exp(x1)
    sig = r * r + a * a * np.cos(x2) ** 2
    z = 2.0 * r / sig
    assert np.allclose(f[:, 6], 1.0 / np.sqrt(1.0 + z), rtol=1e-13)
    assert np.allclose(f[:, 7], np.log(z * z / (1.0 + z) + 1e-30), rtol=1e-12, atol=1e-12)
    assert np.allclose(f[:, 8], np.log(r * sig * np.abs(np.sin(x2)) * np.sqrt(1.0 + z)), rtol=1e-12, atol=1e-12)
    assert np.array_equal(f[:, 9], x1)


def test_targets_from_the_lorentz_factor_and_enthalpy():
    a = 0.9375
    gam = 13.0 / 9.0
    d = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=a, gam=gam)
    prim, x1, x2 = W.random_states(40, seed=10, a=a)
    y = O.mlp_targets(d, prim, x1, x2)
    for s in range(len(prim)):
        ucon, _, _, _, _ = O.state(d, prim[s], x1[s], x2[s])
        al = O.geom(d, x1[s], x2[s])[3]
        g = al * ucon[0]  # Gamma = alpha u^t
        h = 1.0 + gam * prim[s, 1] / prim[s, 0]
        assert abs(y[s, 0] - math.log(h * g)) < 1e-12 * max(1.0, abs(y[s, 0]))
        assert abs(y[s, 1] - 2.0 * math.log(g)) < 1e-11 * max(1.0, abs(y[s, 1]))

