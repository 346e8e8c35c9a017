"""Linear eigenmodes of ideal special-relativistic MHD about a uniform state
at rest, for the rotated linear-wave tests (Sec. 6: fast, slow, Alfven and
entropy waves through a refinement boundary with a time-step jump).

Written for the tests from the equations themselves: the conserved
variables and x-fluxes of ideal SRMHD, U = (rho u^0, T^{0x}, T^{0y},
T^{0z}, T^{00}, B^y, B^z) and F = (rho u^x, T^{xx}, T^{xy}, T^{xz}, T^{x0},
b^y u^x - b^x u^y, b^z u^x - b^x u^z), with T = (w + b^2) u u + (p + b^2/2)
eta - b b; their Jacobians in the primitives P = (rho, p, v^x, v^y, v^z,
B^y, B^z) by complex-step differentiation (exact to rounding); and the
generalised eigenproblem F_P r = lambda U_P r, whose eigenvalues are the
wave speeds along x. Nothing here is shared with the oracle or the library.
"""
import numpy as np
import scipy.linalg as sl

ETA = np.diag([-1.0, 1.0, 1.0, 1.0])


def uf(P, Bx, gam):
    """Conserved variables and x-fluxes of primitives P (real or complex)."""
    rho, p, vx, vy, vz, By, Bz = P
    v = np.array([vx, vy, vz])
    B = np.array([Bx, By, Bz])
    lor = 1.0 / np.sqrt(1.0 - v @ v)
    u = np.concatenate([[lor], lor * v])
    b0 = lor * (v @ B)
    b = np.concatenate([[b0], B / lor + b0 * v])
    bsq = -b[0] ** 2 + b[1:] @ b[1:]
    w = rho + p / (gam - 1.0) + p
    T = (w + bsq) * np.outer(u, u) + (p + 0.5 * bsq) * ETA - np.outer(b, b)
    U = np.array([rho * u[0], T[0, 1], T[0, 2], T[0, 3], T[0, 0], By, Bz])
    F = np.array([rho * u[1], T[1, 1], T[1, 2], T[1, 3], T[1, 0], b[2] * u[1] - b[1] * u[2],
                  b[3] * u[1] - b[1] * u[3]])
    return U, F


def jacobians(P0, Bx, gam, h=1e-30):
    n = len(P0)
    UP = np.zeros((n, n))
    FP = np.zeros((n, n))
    for j in range(n):
        P = np.array(P0, dtype=complex)
        P[j] += 1j * h
        U, F = uf(P, Bx, gam)
        UP[:, j] = U.imag / h
        FP[:, j] = F.imag / h
    return UP, FP


def modes(rho, p, B, gam):
    """Wave speeds along x (ascending) and right eigenvectors (columns, in P) of the state at rest
    with field B = (Bx, By, Bz)."""
    P0 = np.array([rho, p, 0.0, 0.0, 0.0, B[1], B[2]])
    UP, FP = jacobians(P0, B[0], gam)
    lam, R = sl.eig(FP, UP)
    lam = lam.real
    order = np.argsort(lam)
    return lam[order], R[:, order].real


def named_modes(rho, p, B, gam):
    """{'fast', 'alfven', 'slow', 'entropy'}: (speed, eigenvector) of the right-going waves (the
    entropy wave has speed 0). Assumes the seven speeds are distinct (B oblique to x, not
    perpendicular)."""
    lam, R = modes(rho, p, B, gam)
    # ascending: -fast, -alfven, -slow, entropy, +slow, +alfven, +fast
    return {"fast": (lam[6], R[:, 6]), "alfven": (lam[5], R[:, 5]), "slow": (lam[4], R[:, 4]),
            "entropy": (lam[3], R[:, 3])}
