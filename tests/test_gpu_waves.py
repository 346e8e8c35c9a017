"""The paper's linear-wave validation on the GPU path (Sec. 6: 3-D linear
waves of amplitude ~1e-5 with the wave vector along the grid diagonal,
through a refined block that also steps with half the time step, two
periods, L1 error of the primitives against the initial state, second-order
convergence). Fast, Alfven and slow waves about a magnetised state at rest
(eigenvectors from tests/rmhd_modes.py) and an entropy wave advected by a
uniform flow, on a periodic box of 3x3x3 blocks whose centre block is
refined (LAT levels 1 outside, 0 inside)."""
import math

import numpy as np
import pytest

from paper_1912_10192_gb300 import workloads as W

NG = 3
GAM = 5.0 / 3.0
RHO0, P0, AMP = 1.0, 0.5, 1e-5
BPRIME = np.array([0.8, 0.6, 0.0])  # field in the wave frame: oblique to k
pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_10192_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def _frame():
    kh = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
    ey = np.array([1.0, -1.0, 0.0]) / math.sqrt(2.0)
    return np.stack([kh, ey, np.cross(kh, ey)], axis=1)


def wave_error(kind, n, refined=True, split=False):
    import rmhd_modes as M
    from paper_1912_10192_gb300 import hamr
    R = _frame()
    kvec = 2.0 * math.pi * np.array([1.0, 1.0, 1.0])
    lam = 1.0 / math.sqrt(3.0)  # wavelength along k
    if refined:
        blocks = W.flat_box_tree(base=(3, 3, 3), n=n, refine=((1, 1, 1),), lat_coarse=1, lat_fine=0)
    else:
        blocks = W.flat_box_tree(base=(3, 3, 3), n=n, refine=(), lat_coarse=0, lat_fine=0)
    if kind == "entropy":
        # density wave advected by the uniform flow 0.5 k^ (no field): exact at any amplitude
        speed, r = 0.5, np.array([1.0, 0, 0, 0, 0, 0, 0])
        states = W.linear_wave_states(blocks, RHO0, P0, np.zeros(3), kvec, R, r, AMP, gam=GAM)
        u0 = 0.5 / math.sqrt(1.0 - 0.25) * R[:, 0]
        for p, _ in states:
            p[2:5] = u0[:, None, None, None]
    else:
        speed, r = M.named_modes(RHO0, P0, BPRIME, GAM)[kind]
        r = r / np.abs(r).max()
        states = W.linear_wave_states(blocks, RHO0, P0, R @ BPRIME, kvec, R, r, AMP, gam=GAM)
    g = hamr.Grid([hamr.block_from_dict(b) for b in blocks], metric=hamr.METRIC_MINKOWSKI, gam=GAM, cour=0.8,
                  floors=0)
    for i, (p, bf) in enumerate(states):
        g.set_state(p, bf, block=i)
    init = [g.get_state(block=i)[0] for i in range(len(blocks))]
    T = 2.0 * lam / abs(speed)
    hfine = min(b["dx1"] for b in blocks)
    nper = int(math.ceil(T / (2 * 0.25 * hfine)))
    g.set_fine_dt(T / (2 * nper))
    g.batch_step(2 * nper)
    acc = {"all": [0.0, 0.0], "extrema": [0.0, 0.0], "away": [0.0, 0.0]}
    for i, b in enumerate(blocks):
        p, _ = g.get_state(block=i)
        s = (slice(None), slice(NG, NG + b["n3"]), slice(NG, NG + b["n2"]), slice(NG, NG + b["n1"]))
        dv = b["dx1"] * b["dx2"] * b["dx3"]
        e = np.abs(p[s] - init[i][s]).sum(axis=0) * dv
        # cells near the extrema of the initial profile sin(k.x): |cos(k.x)| < 0.3
        x = b["x1min"] + (np.arange(b["n1"]) + 0.5) * b["dx1"]
        y = b["x2min"] + (np.arange(b["n2"]) + 0.5) * b["dx2"]
        z = b["x3min"] + (np.arange(b["n3"]) + 0.5) * b["dx3"]
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        near = np.abs(np.cos(kvec[0] * X + kvec[1] * Y + kvec[2] * Z)) < 0.3
        for key, msk in (("all", np.ones_like(near)), ("extrema", near), ("away", ~near)):
            acc[key][0] += e[msk].sum()
            acc[key][1] += msk.sum() * dv
    g.close()
    out = {k: v[0] / (v[1] * AMP) for k, v in acc.items()}
    return out if split else out["all"]


@pytest.mark.parametrize("kind", ["fast", "alfven", "slow", "entropy"])
def test_linear_wave_converges_through_refinement_and_time_jump(kind):
    """The refined tree converges at the rate of the uniform grid: measured 1.5-1.85 for both between
    8, 16 and 32 cells per block (PPM's limiter clips the wave's extrema at these resolutions), and
    its error is no larger than the uniform grid's at the same base resolution."""
    e = [wave_error(kind, n) for n in (8, 16)]
    uni = wave_error(kind, 16, refined=False)
    rate = math.log2(e[0] / e[1])
    print("%s wave: L1 error / amplitude %.3e (n=8), %.3e (n=16), rate %.2f; uniform n=16 %.3e"
          % (kind, e[0], e[1], rate, uni))
    assert rate > 1.5, (kind, e, rate)
    assert e[1] <= 1.35 * uni, (kind, e[1], uni)


def test_fast_wave_rate_is_set_near_the_extrema():
    """Between 32 and 64 cells per block the fast wave converges at 1.68 overall; split by the phase
    of the initial profile, the cells near its extrema (|cos k.x| < 0.3, where PPM's monotonicity
    constraints flatten the parabolae) converge at 1.24 and the rest at 1.94 (measured on GB300; the
    Alfven and slow waves show the same split, 1.18 / 1.74 and 1.31 / 1.68, the entropy wave 1.65 /
    1.80). The scheme's second order holds away from extrema; the limiter at the extrema sets the
    global rate at these resolutions."""
    e32 = wave_error("fast", 32, split=True)
    e64 = wave_error("fast", 64, split=True)
    rate = {k: math.log2(e32[k] / e64[k]) for k in e32}
    print("fast wave 32 -> 64 cells per block:", e32, e64, rate)
    assert rate["away"] > 1.85 and rate["extrema"] < rate["away"] - 0.4 and rate["all"] > 1.55, rate
