"""The paper's off-centre explosion through the pole on the GPU path (Sec. 6):
flat space in log-r spherical coordinates, a base of 8 x 4 x 4 blocks with
phi-derefined polar blocks (external SMR), the blocks around the explosion
refined (octants, 6-way next to the axis), four LAT levels, without and with
internal SMR; a sphere of radius 2 at (3, 0, 10) at high pressure. Checks: a
LAT period of the magnetised explosion equals the oracle's; after the
hydrodynamic blast has crossed the polar axis its front is as far from the
centre toward and through the axis as across, and no inversion fails."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1912_10192_gb300 import workloads as W

NG = 3
GAM = 5.0 / 3.0
CENTRE = np.array([3.0, 0.0, 10.0])
pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_10192_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def _grid(blocks, states, smr=0):
    from paper_1912_10192_gb300 import hamr
    g = hamr.Grid([hamr.block_from_dict(b) for b in blocks], metric=hamr.METRIC_SPHERICAL, gam=GAM, cour=0.8,
                  floors=0, smr=smr)
    for i, (p, bf) in enumerate(states):
        g.set_state(p, bf, block=i)
    return g


@pytest.mark.parametrize("smr", [0, 1])
def test_magnetised_explosion_period_matches_oracle(smr):
    blocks = W.polar_smr_tree(2.0, 40.0, (8, 4, 4), 8, range(3, 6))
    states = W.explosion_blocks(blocks, beta_max=10.0)
    g = _grid(blocks, states, smr)
    phys = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_SPHERICAL, gam=GAM, cour=0.8, floors=0, smr=smr)
    a = O.AmrGrid(phys, [O.make_block(b["n1"], b["n2"], b["n3"], b["x1min"], b["x2min"], b["x3min"], b["dx1"],
                                      b["dx2"], b["dx3"], b["bc"], b["lat"]) for b in blocks])
    for i, (p, bf) in enumerate(states):
        a.set(i, p, bf)
    lmax = max(b["lat"] for b in blocks)
    a.period()
    g.batch_step(2 ** lmax)
    num = {k: 0.0 for k in ("rho", "u", "utilde", "Bface")}
    den = dict(num)
    for i, b in enumerate(blocks):
        pg, bg = g.get_state(block=i)
        po, bo = a.get(i)
        s = (slice(NG, NG + b["n3"]), slice(NG, NG + b["n2"]), slice(NG, NG + b["n1"]))
        for k, vs in (("rho", (0,)), ("u", (1,)), ("utilde", (2, 3, 4))):
            for v in vs:
                num[k] += np.abs(pg[v][s] - po[v][s]).sum()
                den[k] += np.abs(po[v][s]).sum()
        n1, n2, n3 = b["n1"], b["n2"], b["n3"]
        fs = [(slice(NG, NG + n3), slice(NG, NG + n2), slice(NG, NG + n1 + 1)),
              (slice(NG, NG + n3), slice(NG, NG + n2 + 1), slice(NG, NG + n1)),
              (slice(NG, NG + n3 + 1), slice(NG, NG + n2), slice(NG, NG + n1))]
        for m in range(3):
            num["Bface"] += np.abs(bg[m][fs[m]] - bo[m][fs[m]]).sum()
            den["Bface"] += np.abs(bo[m][fs[m]]).sum()
    g.close()
    errs = {k: num[k] / den[k] for k in num}
    for k, e in errs.items():
        assert e <= 1e-10, (k, e, errs)


@pytest.mark.parametrize("smr", [0, 2])
def test_blast_front_keeps_its_shape_through_the_pole(smr):
    """with two internal SMR levels too (the paper's set-up: one external and two internal SMR
    layers, four LAT levels)"""
    blocks = W.polar_smr_tree(2.0, 40.0, (8, 4, 4), 16, range(3, 6))
    states = W.explosion_blocks(blocks)
    g = _grid(blocks, states, smr)
    lmax = max(b["lat"] for b in blocks)
    t, fails = 0.0, 0
    while t < 5.0:
        st = g.batch_step(2 ** lmax, stats=True)
        t += st["dt_used"] * 2 ** lmax
        fails += st["c2p_fail"]
    # front radius per direction from the centre: the farthest cell with u/rho above 30x the ambient
    amb = 3e-8 / (GAM - 1.0) / 1e-4
    dirs, dist = [], []
    for i, b in enumerate(blocks):
        p, _ = g.get_state(block=i)
        s = (slice(NG, NG + b["n3"]), slice(NG, NG + b["n2"]), slice(NG, NG + b["n1"]))
        hot = p[1][s] / p[0][s] > 30.0 * amb
        if not hot.any():
            continue
        x1 = b["x1min"] + (np.arange(b["n1"]) + 0.5) * b["dx1"]
        x2 = b["x2min"] + (np.arange(b["n2"]) + 0.5) * b["dx2"]
        x3 = b["x3min"] + (np.arange(b["n3"]) + 0.5) * b["dx3"]
        P3, T2, R1 = np.meshgrid(x3, x2, np.exp(x1), indexing="ij")
        xyz = np.stack([R1 * np.sin(T2) * np.cos(P3), R1 * np.sin(T2) * np.sin(P3), R1 * np.cos(T2)], -1)[hot]
        v = xyz - CENTRE
        dd = np.linalg.norm(v, axis=1)
        dirs.append(v / dd[:, None])
        dist.append(dd)
    g.close()
    dirs, dist = np.concatenate(dirs), np.concatenate(dist)
    def front(axis, cone=0.3):
        sel = dirs @ axis > math.cos(cone)
        return dist[sel].max()
    toward_axis = front(np.array([-1.0, 0.0, 0.0]))       # through the pole
    across = [front(np.array([0.0, 1.0, 0.0])), front(np.array([0.0, -1.0, 0.0]))]  # same height, away
    print("smr %d, blast at t=%.2f: front toward/through the axis %.3f, across %.3f %.3f, inversion failures %d"
          % (smr, t, toward_axis, across[0], across[1], fails))
    assert toward_axis > 3.5  # the front has passed the axis (3 from the centre)
    for r in across:
        assert abs(toward_axis - r) < 0.08 * r, (toward_axis, across)
    assert fails == 0
