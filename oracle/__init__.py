"""ctypes binding of the plain FP64 CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg import
this package. The product path (paper_1912_10192_gb300) never does.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))
NG = 3
BC_OUTFLOW, BC_PERIODIC, BC_POLAR, BC_OUTFLOW_NOINFLOW = 0, 1, 2, 3
METRIC_KS, METRIC_MINKOWSKI = 0, 1
RECON_PPM, RECON_MC, RECON_MINMOD = 0, 1, 2
METRIC_SPHERICAL = 2  # flat space in log-r spherical coordinates
FLUX_HLL, FLUX_LLF = 0, 1
EMF_AVERAGE, EMF_UPWIND = 0, 1
INV_NEWTON, INV_AITKEN = 0, 1
FLOOR_FLUID, FLOOR_DRIFT = 0, 1


class Desc(C.Structure):
    _fields_ = [("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int),
                ("x1min", C.c_double), ("x2min", C.c_double), ("x3min", C.c_double),
                ("dx1", C.c_double), ("dx2", C.c_double), ("dx3", C.c_double),
                ("metric", C.c_int), ("a", C.c_double), ("gam", C.c_double),
                ("cour", C.c_double), ("recon", C.c_int), ("riemann", C.c_int),
                ("bc", C.c_int * 6), ("floors", C.c_int), ("emf", C.c_int), ("flatten", C.c_int),
                ("inversion", C.c_int), ("floor_frame", C.c_int), ("smr", C.c_int)]


_libs = {}

_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def _setup(lib):
    P = C.POINTER(Desc)
    sig = {
        "ora_geom": [P, C.c_double, C.c_double, _D, _D, _D, _D],
        "ora_conn": [P, C.c_double, C.c_double, _D],
        "ora_state": [P, _D, C.c_double, C.c_double, _D, _D, _D, _D, _D],
        "ora_p2uf": [P, _D, C.c_double, C.c_double, C.c_int, _D],
        "ora_vchar": [P, _D, C.c_double, C.c_double, C.c_int, _D, _D],
        "ora_face_flux": [P, _D, _D, C.c_double, C.c_double, C.c_int, _D],
        "ora_source": [P, _D, C.c_double, C.c_double, _D],
        "ora_recon_line": [C.c_int, C.c_int, _D, _D, _D],
        "ora_flatten_line": [C.c_int, C.c_double, _D, _D, _D],
        "ora_nh_map": [C.c_double] * 7 + [_D],
        "ora_floors_many": [P, C.c_long, _D, _D, _D, _D, _I],
        "ora_recon_line_flat": [C.c_int, _D, _D, _D, _D],
        "ora_c2p_many": [P, C.c_long, _D, _D, _D, _D, _D, _I, _I, C.c_int],
        "ora_p2u_many": [P, C.c_long, _D, _D, _D, _D],
        "ora_mlp_features": [P, C.c_long, _D, _D, _D, _D, _D],
        "ora_mlp_targets": [P, C.c_long, _D, _D, _D, _D],
        "ora_grid_new": [P],
        "ora_grid_free": [C.c_void_p],
        "ora_grid_set": [C.c_void_p, _D, _D],
        "ora_grid_get": [C.c_void_p, _D, _D],
        "ora_grid_bc": [C.c_void_p],
        "ora_grid_dt": [C.c_void_p],
        "ora_grid_step": [C.c_void_p, C.c_double],
        "ora_grid_stats": [C.c_void_p, C.POINTER(C.c_longlong)],
        "ora_grid_divb": [C.c_void_p, _D],
        "ora_grid_fluxes": [C.c_void_p, _D],
        "ora_grid_status": [C.c_void_p, _I],
        "ora_flops_reset": [],
        "ora_flops_get": [C.POINTER(C.c_ulonglong)],
        "ora_flops_phase": [C.POINTER(C.c_ulonglong)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = None
    lib.ora_grid_new.restype = C.c_void_p
    lib.ora_grid_dt.restype = C.c_double
    lib.ora_grid_step.restype = C.c_double
    return lib


def lib(counting=False):
    """Load (building first if needed) the oracle library."""
    key = bool(counting)
    if key not in _libs:
        _build.build()
        name = "libhamr_oracle_count.so" if counting else "libhamr_oracle.so"
        _libs[key] = _setup(C.CDLL(os.path.join(HERE, name)))
    return _libs[key]


def _p(a):
    return a.ctypes.data_as(_D)


def make_desc(n1, n2, n3, x1min, x2min, x3min, dx1, dx2, dx3, metric=METRIC_KS, a=0.0,
              gam=13.0 / 9.0, cour=0.8, recon=RECON_PPM, riemann=FLUX_HLL, bc=(0, 0, 0, 0, 1, 1),
              floors=1, emf=EMF_AVERAGE, flatten=0, inversion=0, floor_frame=0, smr=0):
    d = Desc()
    d.n1, d.n2, d.n3 = n1, n2, n3
    d.x1min, d.x2min, d.x3min = x1min, x2min, x3min
    d.dx1, d.dx2, d.dx3 = dx1, dx2, dx3
    d.metric, d.a, d.gam, d.cour = metric, a, gam, cour
    d.recon, d.riemann = recon, riemann
    for m in range(6):
        d.bc[m] = bc[m]
    d.floors = floors
    d.emf = emf
    d.flatten = flatten
    d.inversion = inversion
    d.floor_frame = floor_frame
    d.smr = smr
    return d


def geom(d, x1, x2):
    gcov = np.zeros(16)
    gcon = np.zeros(16)
    gdet = C.c_double()
    alpha = C.c_double()
    lib().ora_geom(C.byref(d), x1, x2, _p(gcov), _p(gcon), C.byref(gdet), C.byref(alpha))
    return gcov.reshape(4, 4), gcon.reshape(4, 4), gdet.value, alpha.value


def conn(d, x1, x2):
    c = np.zeros(64)
    lib().ora_conn(C.byref(d), x1, x2, _p(c))
    return c.reshape(4, 4, 4)


def state(d, pr, x1, x2):
    pr = np.ascontiguousarray(pr, dtype=np.float64)
    out = [np.zeros(4) for _ in range(4)]
    bsq = C.c_double()
    lib().ora_state(C.byref(d), _p(pr), x1, x2, *[_p(o) for o in out], C.byref(bsq))
    return (*out, bsq.value)


def p2uf(d, pr, x1, x2, direction):
    pr = np.ascontiguousarray(pr, dtype=np.float64)
    out = np.zeros(9)
    lib().ora_p2uf(C.byref(d), _p(pr), x1, x2, direction, _p(out))
    return out


def vchar(d, pr, x1, x2, direction):
    pr = np.ascontiguousarray(pr, dtype=np.float64)
    vp, vm = C.c_double(), C.c_double()
    lib().ora_vchar(C.byref(d), _p(pr), x1, x2, direction, C.byref(vp), C.byref(vm))
    return vp.value, vm.value


def face_flux(d, pl, pr, x1, x2, direction):
    pl = np.ascontiguousarray(pl, dtype=np.float64)
    pr = np.ascontiguousarray(pr, dtype=np.float64)
    out = np.zeros(8)
    lib().ora_face_flux(C.byref(d), _p(pl), _p(pr), x1, x2, direction, _p(out))
    return out


def source(d, pr, x1, x2):
    pr = np.ascontiguousarray(pr, dtype=np.float64)
    out = np.zeros(6)
    lib().ora_source(C.byref(d), _p(pr), x1, x2, _p(out))
    return out


def recon_line(recon, q):
    q = np.ascontiguousarray(q, dtype=np.float64)
    al = np.full_like(q, np.nan)
    ar = np.full_like(q, np.nan)
    lib().ora_recon_line(recon, len(q), _p(q), _p(al), _p(ar))
    return al, ar


def floors_many(d, prim, x1, x2, r):
    """The floors on prim (n, 8) (slots 5..7 centre B) -> (floored prim, hit flags)."""
    out = np.ascontiguousarray(prim, dtype=np.float64).copy()
    x1 = np.ascontiguousarray(x1, dtype=np.float64)
    x2 = np.ascontiguousarray(x2, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    hit = np.zeros(len(x1), dtype=np.int32)
    lib().ora_floors_many(C.byref(d), len(x1), _p(out), _p(x1), _p(x2), _p(r), hit.ctypes.data_as(_I))
    return out, hit


def nh_map(E, S2, T2, B2, D, gam, p):
    """Newman-Hamlin pressure map of the Aitken inversion -> (W, v^2, next p); W = -1 if invalid."""
    out = np.zeros(3)
    lib().ora_nh_map(E, S2, T2, B2, D, gam, p, _p(out))
    return out


def flatten_line(gam, u, w):
    """Shock flattening coefficients of a line (PPM, Colella & Woodward 1984)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    f = np.zeros_like(u)
    lib().ora_flatten_line(len(u), gam, _p(u), _p(w), _p(f))
    return f


def recon_line_flat(q, f):
    """PPM edge values of a line with flattening coefficients f."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    al = np.full_like(q, np.nan)
    ar = np.full_like(q, np.nan)
    lib().ora_recon_line_flat(len(q), _p(q), _p(f), _p(al), _p(ar))
    return al, ar


def c2p_many(d, U, B, x1, x2, guess, entropy_only=False):
    """U: (n, 6), B: (n, 3), x1/x2: (n,), guess: (n, 8) -> (prims, status, iters)."""
    n = U.shape[0]
    U = np.ascontiguousarray(U, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    x1 = np.ascontiguousarray(x1, dtype=np.float64)
    x2 = np.ascontiguousarray(x2, dtype=np.float64)
    pr = np.array(guess, dtype=np.float64, copy=True, order="C")
    st = np.zeros(n, dtype=np.int32)
    it = np.zeros(n, dtype=np.int32)
    lib().ora_c2p_many(C.byref(d), n, _p(U), _p(B), _p(x1), _p(x2), _p(pr),
                       st.ctypes.data_as(_I), it.ctypes.data_as(_I), int(entropy_only))
    return pr, st, it


def p2u_many(d, pr, x1, x2):
    n = pr.shape[0]
    pr = np.ascontiguousarray(pr, dtype=np.float64)
    x1 = np.ascontiguousarray(x1, dtype=np.float64)
    x2 = np.ascontiguousarray(x2, dtype=np.float64)
    U = np.zeros((n, 6))
    lib().ora_p2u_many(C.byref(d), n, _p(pr), _p(x1), _p(x2), _p(U))
    return U


def mlp_features(d, U, B, x1, x2):
    """(n, 6) conserved, (n, 3) centre B, positions -> (n, 10) network inputs (FP64)."""
    n = U.shape[0]
    U = np.ascontiguousarray(U, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    x1 = np.ascontiguousarray(x1, dtype=np.float64)
    x2 = np.ascontiguousarray(x2, dtype=np.float64)
    f = np.zeros((n, 10))
    lib().ora_mlp_features(C.byref(d), n, _p(U), _p(B), _p(x1), _p(x2), _p(f))
    return f


def mlp_targets(d, pr, x1, x2):
    """(n, 8) primitives, positions -> (n, 2) targets ln(W/D), ln Gamma^2 (FP64)."""
    n = pr.shape[0]
    pr = np.ascontiguousarray(pr, dtype=np.float64)
    x1 = np.ascontiguousarray(x1, dtype=np.float64)
    x2 = np.ascontiguousarray(x2, dtype=np.float64)
    y = np.zeros((n, 2))
    lib().ora_mlp_targets(C.byref(d), n, _p(pr), _p(x1), _p(x2), _p(y))
    return y


class Grid:
    """Single-block oracle grid holding padded primitive and face-B arrays."""

    def __init__(self, d, counting=False):
        self.d = d
        self.lib = lib(counting)
        self.h = self.lib.ora_grid_new(C.byref(d))
        self.shape = (d.n3 + 2 * NG, d.n2 + 2 * NG, d.n1 + 2 * NG)

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.ora_grid_free(self.h)
            self.h = None

    def set(self, prim, bface):
        prim = np.ascontiguousarray(prim, dtype=np.float64)
        bface = np.ascontiguousarray(bface, dtype=np.float64)
        assert prim.shape == (8, *self.shape) and bface.shape == (3, *self.shape)
        self.lib.ora_grid_set(self.h, _p(prim), _p(bface))

    def get(self):
        prim = np.zeros((8, *self.shape))
        bface = np.zeros((3, *self.shape))
        self.lib.ora_grid_get(self.h, _p(prim), _p(bface))
        return prim, bface

    def bc(self):
        self.lib.ora_grid_bc(self.h)

    def dt(self):
        return self.lib.ora_grid_dt(self.h)

    def step(self, dt=-1.0):
        return self.lib.ora_grid_step(self.h, dt)

    def stats(self):
        s = (C.c_longlong * 4)()
        self.lib.ora_grid_stats(self.h, s)
        return list(s)

    def status(self):
        d = self.d
        out = np.zeros(d.n1 * d.n2 * d.n3, dtype=np.int32)
        self.lib.ora_grid_status(self.h, out.ctypes.data_as(_I))
        return out.reshape(d.n3, d.n2, d.n1)

    def fluxes(self):
        """Face fluxes of the current state, shape (3, 8, n3p, n2p, n1p) (slot 0 mass,
        5 entropy tracer); the dir-face of cell (i, j, k) lies on its lower side."""
        out = np.zeros((3, 8, *self.shape))
        self.lib.ora_grid_fluxes(self.h, _p(out))
        return out

    def divb(self):
        d = self.d
        out = np.zeros(d.n1 * d.n2 * d.n3)
        self.lib.ora_grid_divb(self.h, _p(out))
        return out.reshape(d.n3, d.n2, d.n1)


def flops_reset():
    lib(True).ora_flops_reset()


def flops_get():
    out = (C.c_ulonglong * 5)()
    lib(True).ora_flops_get(out)
    return list(out)


PHASES = ("recon", "flux", "emf", "ct", "update", "cfl")
CLASSES = ("addmul", "div", "sqrt", "transc", "cmp")


def flops_phase():
    """{phase: [add/sub/mul, div, sqrt, transcendental, compare]} of the counting build."""
    out = (C.c_ulonglong * 30)()
    lib(True).ora_flops_phase(out)
    return {p: list(out[5 * k:5 * k + 5]) for k, p in enumerate(PHASES)}

BC_BLOCK = 4


class Block(C.Structure):
    _fields_ = [("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int),
                ("x1min", C.c_double), ("x2min", C.c_double), ("x3min", C.c_double),
                ("dx1", C.c_double), ("dx2", C.c_double), ("dx3", C.c_double),
                ("bc", C.c_int * 6), ("lat", C.c_int)]


def make_block(n1, n2, n3, x1min, x2min, x3min, dx1, dx2, dx3, bc, lat=0):
    b = Block()
    b.n1, b.n2, b.n3 = n1, n2, n3
    b.x1min, b.x2min, b.x3min = x1min, x2min, x3min
    b.dx1, b.dx2, b.dx3 = dx1, dx2, dx3
    for m in range(6):
        b.bc[m] = bc[m]
    b.lat = lat
    return b


_amr_ready = set()


def _amr_setup(L):
    if id(L) in _amr_ready:
        return
    P = C.c_void_p
    L.ora_amr_new.argtypes = [C.POINTER(Desc), C.c_int, C.POINTER(Block)]
    L.ora_amr_new.restype = C.c_void_p
    L.ora_amr_free.argtypes = [P]
    L.ora_amr_set.argtypes = [P, C.c_int, _D, _D]
    L.ora_amr_get.argtypes = [P, C.c_int, _D, _D]
    L.ora_amr_fill.argtypes = [P]
    L.ora_amr_period.argtypes = [P, C.c_double]
    L.ora_amr_period.restype = C.c_double
    L.ora_amr_stats.argtypes = [P, C.POINTER(C.c_longlong)]
    L.ora_amr_regrid.argtypes = [P, C.c_int, C.POINTER(Block)]
    L.ora_amr_regrid.restype = P
    for n in ("ora_amr_free", "ora_amr_set", "ora_amr_get", "ora_amr_fill", "ora_amr_stats"):
        getattr(L, n).restype = None
    _amr_ready.add(id(L))


class AmrGrid:
    """Multi-block oracle grid (static refinement + local adaptive time steps)."""

    def __init__(self, phys, blocks, counting=False):
        self.lib = lib(counting)
        _amr_setup(self.lib)
        self.blocks = list(blocks)
        self._arr = (Block * len(blocks))(*blocks)
        self.phys = phys
        self.h = self.lib.ora_amr_new(C.byref(phys), len(blocks), self._arr)

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.ora_amr_free(self.h)
            self.h = None

    def shape(self, b):
        B = self.blocks[b]
        return (B.n3 + 2 * NG, B.n2 + 2 * NG, B.n1 + 2 * NG)

    def set(self, b, prim, bface):
        prim = np.ascontiguousarray(prim, dtype=np.float64)
        bface = np.ascontiguousarray(bface, dtype=np.float64)
        assert prim.shape == (8, *self.shape(b)) and bface.shape == (3, *self.shape(b))
        self.lib.ora_amr_set(self.h, b, _p(prim), _p(bface))

    def get(self, b):
        prim = np.zeros((8, *self.shape(b)))
        bface = np.zeros((3, *self.shape(b)))
        self.lib.ora_amr_get(self.h, b, _p(prim), _p(bface))
        return prim, bface

    def fill(self):
        self.lib.ora_amr_fill(self.h)

    def period(self, dt_fine=-1.0):
        return self.lib.ora_amr_period(self.h, dt_fine)

    def regrid(self, blocks):
        """A new AmrGrid on `blocks` holding this grid's state (prolongation / restriction / copy)."""
        new = AmrGrid.__new__(AmrGrid)
        new.lib = self.lib
        new.blocks = list(blocks)
        new._arr = (Block * len(blocks))(*blocks)
        new.phys = self.phys
        new.h = self.lib.ora_amr_regrid(self.h, len(blocks), new._arr)
        return new

    def stats(self):
        s = (C.c_longlong * 4)()
        self.lib.ora_amr_stats(self.h, s)
        return list(s)
