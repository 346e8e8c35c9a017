"""Exact solution of the one-dimensional special relativistic Riemann problem
for an ideal gas without transverse velocity (the wave curves of Marti &
Mueller 1994, J. Fluid Mech. 258, 317; Pons, Marti & Mueller 2000), used to
pin the oracle's shock capturing against a closed solution.

Written for the tests from the published method: each outer state a is
joined to the intermediate pressure p* by a rarefaction (p* < p_a; the
Riemann invariant arctanh(v) +- A(c) is constant, A(c) = ln((sqrt(G-1) + c)
/ (sqrt(G-1) - c)) / sqrt(G-1)) or a shock (p* > p_a; Taub adiabat, mass flux
j, shock speed); p* is where the two wave curves give the same velocity.
"""
import math


class State:
    def __init__(self, rho, p, v, gam):
        self.rho, self.p, self.v, self.gam = rho, p, v, gam

    @property
    def h(self):
        return 1.0 + self.gam / (self.gam - 1.0) * self.p / self.rho

    @property
    def c(self):
        return math.sqrt(self.gam * self.p / (self.rho * self.h))

    @property
    def W(self):
        return 1.0 / math.sqrt(1.0 - self.v * self.v)


def _A(c, gam):
    s = math.sqrt(gam - 1.0)
    return math.log((s + c) / (s - c)) / s


def _rarefaction_state(a, pstar, sign):
    """State behind a rarefaction at pressure pstar (sign -1: left wave, +1: right wave)."""
    gam = a.gam
    rho = a.rho * (pstar / a.p) ** (1.0 / gam)
    s = State(rho, pstar, 0.0, gam)
    # left wave: arctanh v + A(c) constant; right wave: arctanh v - A(c) constant
    phi = math.atanh(a.v) - sign * (_A(a.c, gam) - _A(s.c, gam))
    s.v = math.tanh(phi)
    return s


def _shock_state(a, pstar, sign):
    """State behind a shock of pressure pstar (sign -1: left-moving, +1: right-moving); also its speed."""
    gam = a.gam
    dp = a.p - pstar
    k = (gam - 1.0) * dp / (gam * pstar)
    # Taub adiabat as a quadratic in h*: h^2 (1 + k) - h k + h_a dp / rho_a - h_a^2 = 0
    qa, qb, qc = 1.0 + k, -k, a.h * dp / a.rho - a.h * a.h
    hs = (-qb + math.sqrt(qb * qb - 4.0 * qa * qc)) / (2.0 * qa)
    rho = gam * pstar / ((gam - 1.0) * (hs - 1.0))
    j2 = -(pstar - a.p) / (hs / rho - a.h / a.rho)
    j = sign * math.sqrt(j2)
    Wa, va = a.W, a.v
    r2w2 = a.rho * a.rho * Wa * Wa
    vs = (r2w2 * va + sign * abs(j) * math.sqrt(j2 + r2w2 * (1.0 - va * va))) / (r2w2 + j2)
    Ws = 1.0 / math.sqrt(1.0 - vs * vs)
    v = (a.h * Wa * va + Ws * (pstar - a.p) / j) / (a.h * Wa + (pstar - a.p) * (Ws * va / j + 1.0 / (a.rho * Wa)))
    s = State(rho, pstar, v, gam)
    return s, vs


def _behind(a, pstar, sign):
    if pstar < a.p:
        return _rarefaction_state(a, pstar, sign), None
    return _shock_state(a, pstar, sign)


def solve(L, R, tol=1e-14):
    """Intermediate pressure and velocity and the states on either side of the contact."""
    def f(p):
        return _behind(L, p, -1)[0].v - _behind(R, p, +1)[0].v
    lo, hi = 1e-14 * min(L.p, R.p), 1e3 * max(L.p, R.p)
    flo = f(lo)
    for _ in range(400):
        mid = math.sqrt(lo * hi)
        fm = f(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
        if hi / lo - 1.0 < tol:
            break
    pstar = math.sqrt(lo * hi)
    SL, vsl = _behind(L, pstar, -1)
    SR, vsr = _behind(R, pstar, +1)
    return pstar, 0.5 * (SL.v + SR.v), SL, SR, vsl, vsr


def _fan_state(a, xi, sign):
    """State inside a rarefaction fan at x/t = xi: (v - sign... ) the characteristic speed
    (v + sign c)/(1 + sign v c) equals xi, with the invariant of the fan."""
    gam = a.gam
    K = a.p / a.rho ** gam

    def at(p):
        return _rarefaction_state(a, p, sign)

    def g(p):
        s = at(p)
        return (s.v + sign * s.c) / (1.0 + sign * s.v * s.c) - xi
    lo, hi = 1e-16 * a.p, a.p
    glo = g(lo)
    for _ in range(300):
        mid = math.sqrt(lo * hi)
        gm = g(mid)
        if (gm > 0) == (glo > 0):
            lo, glo = mid, gm
        else:
            hi = mid
    s = at(math.sqrt(lo * hi))
    del K
    return s


def sample(L, R, xi):
    """(rho, p, v) at x/t = xi of the solution of the Riemann problem (L | R)."""
    pstar, vstar, SL, SR, vsl, vsr = solve(L, R)
    if xi < vstar:  # left of the contact
        if vsl is not None:  # left shock
            return (L.rho, L.p, L.v) if xi < vsl else (SL.rho, SL.p, SL.v)
        head = (L.v - L.c) / (1.0 - L.v * L.c)
        tail = (SL.v - SL.c) / (1.0 - SL.v * SL.c)
        if xi < head:
            return L.rho, L.p, L.v
        if xi > tail:
            return SL.rho, SL.p, SL.v
        s = _fan_state(L, xi, -1)
        return s.rho, s.p, s.v
    if vsr is not None:  # right shock
        return (SR.rho, SR.p, SR.v) if xi < vsr else (R.rho, R.p, R.v)
    head = (R.v + R.c) / (1.0 + R.v * R.c)
    tail = (SR.v + SR.c) / (1.0 + SR.v * SR.c)
    if xi > head:
        return R.rho, R.p, R.v
    if xi < tail:
        return SR.rho, SR.p, SR.v
    s = _fan_state(R, xi, +1)
    return s.rho, s.p, s.v
