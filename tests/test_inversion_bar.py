"""The parity bar of the energy inversion (tests/helpers.py inversion_bar),
checked on the oracle alone: two correct inversions of the same conserved
states, started from different points, take different rounding paths; the
bar must cover every such pair, and it must not cover a result that is off
by more than the conditioning allows (a planted error in u_g).

Measured spread of the oracle against itself from the two starts over the
full law (rho 1e-6..1, u/rho 1e-4..1e2, Lorentz factor 1..50, sigma
0..100): relative to the largest primitive of a state, median 1.8e-15,
99th percentile 7.8e-13, maximum 4.7e-11; the GPU parity tests hold the
CUDA inversion to the per-state bar and to median 1e-14 / 99th percentile
1e-11, the oracle's own spread with room for a third rounding path (FMA
contraction)."""
import numpy as np

import oracle as O
from paper_1912_10192_gb300 import workloads as W

from helpers import inversion_bar


def two_starts(n, seed, a, gam, **law):
    d = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=a, gam=gam)
    prim, x1, x2 = W.random_states(n, seed=seed, a=a, **law)
    U = O.p2u_many(d, prim, x1, x2)
    g1 = prim.copy()
    g1[:, 0] *= 1.05
    g1[:, 1] *= 0.95
    g1[:, 2:5] *= 1.02
    g2 = prim.copy()
    g2[:, 0] *= 0.8
    g2[:, 1] *= 1.3
    g2[:, 2:5] *= 0.9
    pa, sa, _ = O.c2p_many(d, U, prim[:, 5:8], x1, x2, g1)
    pb, sb, _ = O.c2p_many(d, U, prim[:, 5:8], x1, x2, g2)
    ok = (sa == 0) & (sb == 0)
    bar = inversion_bar(d, U[ok], prim[ok, 5:8], x1[ok], x2[ok], pa[ok], prim[ok])
    return pa[ok], pb[ok], bar


def test_bar_covers_two_correct_inversions_and_flags_planted_errors():
    for law, a, gam, planted in ((dict(), 0.9375, 13.0 / 9.0, 0.4), (dict(lorentz_range=(1, 5), sigma_range=(0, 5)),
                                                                       0.5, 4.0 / 3.0, 0.9)):
        pa, pb, bar = two_starts(40_000, 21, a, gam, **law)
        assert len(pa) > 0.99 * 40_000
        assert np.all(np.abs(pa[:, :5] - pb[:, :5]) <= bar)
        scale = np.abs(pa[:, :5]).max(axis=1, keepdims=True)
        rel = np.abs(pa[:, :5] - pb[:, :5]) / scale
        assert np.median(rel) < 1e-14 and np.quantile(rel, 0.99) < 1e-11
        wrong = pa.copy()
        wrong[:, 1] *= 1.0 + 1e-8
        flagged = (np.abs(wrong[:, :5] - pa[:, :5]) > bar).any(axis=1).mean()
        assert flagged > planted, flagged
