"""Thin ctypes binding of libhamr.so (the C ABI of include/hamr.h).

Argument marshalling only: every step of the update runs in the library's
CUDA kernels. Device memory and streams come from PyTorch (tensor data
pointers and torch.cuda streams). The binding fails loudly if the library is
missing; there is no CPU fallback.
"""
import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhamr.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "hamr.h")

OK, EINVAL, ECUDA, ENOMEM, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5
METRIC_KS, METRIC_MINKOWSKI, METRIC_SPHERICAL = 0, 1, 2
RECON_PPM, RECON_MC, RECON_MINMOD = 0, 1, 2
FLUX_HLL, FLUX_LLF = 0, 1
BC_OUTFLOW, BC_PERIODIC, BC_POLAR, BC_OUTFLOW_NOINFLOW, BC_BLOCK = 0, 1, 2, 3, 4
PREC_FP64, PREC_MIXED, PREC_MIXED_FP64INV = 0, 1, 2
EMF_AVERAGE, EMF_UPWIND = 0, 1
C2P_ENTROPY_ONLY, C2P_MLP, C2P_MLP_RESCUE, C2P_AITKEN, C2P_MIXED = 1, 2, 4, 8, 16
INV_NEWTON, INV_AITKEN = 0, 1
FLOOR_FLUID, FLOOR_DRIFT = 0, 1
MLP_FIRST, MLP_RESCUE = 0, 1
NG = 3


class HamrError(RuntimeError):
    pass


class BlockDesc(C.Structure):
    _fields_ = [("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int),
                ("x1min", C.c_double), ("x2min", C.c_double), ("x3min", C.c_double),
                ("dx1", C.c_double), ("dx2", C.c_double), ("dx3", C.c_double),
                ("bc", C.c_int * 6), ("lat", C.c_int)]


class GridDesc(C.Structure):
    _fields_ = [("metric", C.c_int), ("a", C.c_double), ("gam", C.c_double), ("cour", C.c_double),
                ("recon", C.c_int), ("riemann", C.c_int), ("floors", C.c_int), ("precision", C.c_int),
                ("nblocks", C.c_int), ("blocks", C.POINTER(BlockDesc)), ("emf", C.c_int),
                ("flatten", C.c_int), ("inversion", C.c_int), ("floor_frame", C.c_int), ("smr", C.c_int)]


class StepStats(C.Structure):
    _fields_ = [("c2p_ok", C.c_longlong), ("c2p_entropy", C.c_longlong), ("c2p_fail", C.c_longlong),
                ("floor_hits", C.c_longlong), ("dt_used", C.c_double), ("dt_next", C.c_double),
                ("newton_iters", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KernelTime(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_longlong), ("ms", C.c_double)]


class C2PDesc(C.Structure):
    _fields_ = [("metric", C.c_int), ("a", C.c_double), ("gam", C.c_double), ("flags", C.c_uint32),
                ("mlp", C.c_void_p)]


class TuneReport(C.Structure):
    _fields_ = [("recon_seg", C.c_int), ("bs_recon", C.c_int), ("bs_flux", C.c_int), ("bs_update", C.c_int),
                ("ms_seg", C.c_float * 3), ("ms_recon", C.c_float * 3), ("ms_flux", C.c_float * 3),
                ("ms_update", C.c_float * 2), ("recon_x1_sweep", C.c_int), ("ms_x1", C.c_float * 2),
                ("ms_default", C.c_float), ("ms_tuned", C.c_float), ("ms_spread", C.c_float),
                ("kept_tuned", C.c_int)]

    def as_dict(self):
        return {"recon_seg": self.recon_seg, "bs_recon": self.bs_recon, "bs_flux": self.bs_flux,
                "bs_update": self.bs_update, "ms_seg": list(self.ms_seg), "ms_recon": list(self.ms_recon),
                "ms_flux": list(self.ms_flux), "ms_update": list(self.ms_update),
                "recon_x1_sweep": self.recon_x1_sweep, "ms_x1": list(self.ms_x1),
                "ms_default": self.ms_default, "ms_tuned": self.ms_tuned, "ms_spread": self.ms_spread,
                "kept_tuned": self.kept_tuned}


class MlpTrainArgs(C.Structure):
    _fields_ = [("steps", C.c_int64), ("batch", C.c_int32), ("lr", C.c_float), ("lr_final", C.c_float),
                ("seed", C.c_uint64)]


_lib = None


def header_functions():
    """Names of the functions include/hamr.h declares."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(hamr_\w+)\s*\(", txt, re.M)))


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise HamrError("libhamr.so is not built (run __graft_entry__.build()); no fallback exists")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        D = C.POINTER(C.c_double)
        L.hamr_grid_create.argtypes = [C.POINTER(GridDesc), C.POINTER(C.c_void_p)]
        L.hamr_grid_destroy.argtypes = [P]
        L.hamr_grid_set_state.argtypes = [P, C.c_int, P, P, C.c_int, P]
        L.hamr_grid_get_state.argtypes = [P, C.c_int, P, P, C.c_int, P]
        L.hamr_block_step.argtypes = [P, C.c_int, C.c_double, P, C.POINTER(StepStats)]
        L.hamr_batch_step.argtypes = [P, C.c_int, P, C.POINTER(StepStats)]
        L.hamr_grid_stats.argtypes = [P, C.POINTER(StepStats)]
        L.hamr_con2prim.argtypes = [C.POINTER(C2PDesc), C.c_int64, P, P, P, P, P, P, P, P]
        L.hamr_grid_set_timing.argtypes = [P, C.c_int]
        L.hamr_grid_fill_ghosts.argtypes = [P, P]
        L.hamr_grid_block_max.argtypes = [P, C.c_int, D, P]
        L.hamr_grid_set_launch_shapes.argtypes = [P, C.POINTER(TuneReport)]
        L.hamr_grid_set_fine_dt.argtypes = [P, C.c_double]
        L.hamr_grid_set_ghost_maps.argtypes = [P, C.c_int, C.POINTER(C.c_int)]
        L.hamr_grid_regrid.argtypes = [P, C.c_int, C.POINTER(BlockDesc), P]
        L.hamr_tree_adapt.argtypes = [C.POINTER(BlockDesc), C.c_int, C.POINTER(C.c_int), D, D,
                                      C.POINTER(C.c_int), C.POINTER(BlockDesc), C.c_int, C.POINTER(C.c_int)]
        L.hamr_tree_adapt_polar.argtypes = [C.POINTER(BlockDesc), C.c_int, C.POINTER(C.c_int), D, D,
                                            C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(BlockDesc), C.c_int,
                                            C.POINTER(C.c_int)]
        L.hamr_grid_timing.argtypes = [P, C.POINTER(KernelTime), C.c_int, C.POINTER(C.c_int)]
        L.hamr_measure_fp64_peak.argtypes = [P, C.POINTER(C.c_double)]
        L.hamr_check_conversions.argtypes = [C.c_longlong, C.c_ulonglong, C.POINTER(C.c_longlong)]
        L.hamr_block_step_noalloc.argtypes = [C.POINTER(GridDesc), P, P, C.c_double, P]
        L.hamr_prim2cons.argtypes = [C.POINTER(C2PDesc), C.c_int64, P, P, P, P, P]
        L.hamr_mlp_create.argtypes = [C.POINTER(C.c_void_p), C.c_uint64]
        L.hamr_mlp_destroy.argtypes = [P]
        L.hamr_mlp_get_params.argtypes = [P, P, P]
        L.hamr_mlp_set_params.argtypes = [P, P, P]
        L.hamr_mlp_features.argtypes = [C.POINTER(C2PDesc), C.c_int64, P, P, P, P, P, P, P, P]
        L.hamr_mlp_fit_norm.argtypes = [P, C.c_int64, P, P, P]
        L.hamr_mlp_train.argtypes = [P, C.c_int64, P, P, C.POINTER(MlpTrainArgs), P, P]
        L.hamr_mlp_loss_grad.argtypes = [P, C.c_int64, P, P, P, P, P]
        L.hamr_mlp_forward.argtypes = [P, C.c_int64, P, P, C.c_int, P]
        L.hamr_mlp_error_flag.argtypes = [P, C.POINTER(C.c_int)]
        L.hamr_grid_set_mlp.argtypes = [P, P, C.c_int]
        L.hamr_grid_autotune.argtypes = [P, P, C.POINTER(TuneReport)]
        L.hamr_grid_launch_shapes.argtypes = [P, C.POINTER(TuneReport)]
        L.hamr_last_error.argtypes = []
        L.hamr_last_error.restype = C.c_char_p
        for name in header_functions():
            if name != "hamr_last_error":
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def check(rc):
    if rc != OK:
        raise HamrError("hamr error %d: %s" % (rc, lib().hamr_last_error().decode()))
    return rc


def _ptr(x):
    """Device/host address of a torch tensor or numpy array (contiguous)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    assert x.is_contiguous()
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        return None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


def block(n1, n2, n3, x1min, x2min, x3min, dx1, dx2, dx3, bc, lat=0):
    b = BlockDesc()
    b.n1, b.n2, b.n3 = n1, n2, n3
    b.x1min, b.x2min, b.x3min = x1min, x2min, x3min
    b.dx1, b.dx2, b.dx3 = dx1, dx2, dx3
    for m in range(6):
        b.bc[m] = bc[m]
    b.lat = lat
    return b


def tree_adapt(blocks, target, dlo, base_ext, periodic=(1, 1, 1), axis=None):
    """hamr_tree_adapt (axis None) or hamr_tree_adapt_polar (axis = (lower, upper) x2 faces that are
    polar axes): the nested block tree for per-block target levels -> list of BlockDesc."""
    n = len(blocks)
    arr = (BlockDesc * n)(*blocks)
    tg = (C.c_int * n)(*[int(t) for t in target])
    lo = (C.c_double * 3)(*dlo)
    ext = (C.c_double * 3)(*base_ext)
    per = (C.c_int * 3)(*[int(p) for p in periodic])
    nout = C.c_int()
    if axis is None:
        call = lambda o, cap: lib().hamr_tree_adapt(arr, n, tg, lo, ext, per, o, cap, C.byref(nout))
    else:
        ax = (C.c_int * 2)(*[int(a) for a in axis])
        call = lambda o, cap: lib().hamr_tree_adapt_polar(arr, n, tg, lo, ext, per, ax, o, cap, C.byref(nout))
    rc = call(None, 0)
    cap = nout.value
    if rc != 0 and cap <= 0:
        check(rc)
    out = (BlockDesc * cap)()
    check(call(out, cap))
    return [out[i] for i in range(nout.value)]


def block_from_dict(b):
    """BlockDesc of a workloads block dict."""
    return block(b["n1"], b["n2"], b["n3"], b["x1min"], b["x2min"], b["x3min"], b["dx1"], b["dx2"], b["dx3"],
                 b["bc"], b.get("lat", 0))


class Grid:
    """Owner of a hamr_grid handle."""

    def __init__(self, blocks, metric=METRIC_KS, a=0.9375, gam=13.0 / 9.0, cour=0.8, recon=RECON_PPM,
                 riemann=FLUX_HLL, floors=1, precision=PREC_FP64, emf=EMF_AVERAGE, flatten=0, inversion=INV_NEWTON,
                 floor_frame=FLOOR_FLUID, smr=0):
        self._blocks = (BlockDesc * len(blocks))(*blocks)
        d = GridDesc()
        d.metric, d.a, d.gam, d.cour = metric, a, gam, cour
        d.recon, d.riemann, d.floors, d.precision = recon, riemann, floors, precision
        d.emf = emf
        d.flatten = flatten
        d.inversion = inversion
        d.floor_frame = floor_frame
        d.smr = smr
        d.nblocks = len(blocks)
        d.blocks = self._blocks
        self.desc = d
        h = C.c_void_p()
        check(lib().hamr_grid_create(C.byref(d), C.byref(h)))
        self.h = h
        self.blocks = list(blocks)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().hamr_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def padded_shape(self, b=0):
        B = self.blocks[b]
        return (B.n3 + 2 * NG, B.n2 + 2 * NG, B.n1 + 2 * NG)

    def set_state(self, prim, bface, block=0, stream=None):
        on_dev = 0 if isinstance(prim, np.ndarray) else 1
        check(lib().hamr_grid_set_state(self.h, block, _ptr(prim), _ptr(bface), on_dev, _stream(stream)))

    def get_state(self, block=0, prim=None, bface=None, stream=None):
        shp = self.padded_shape(block)
        if prim is None:
            prim = np.zeros((8,) + shp)
        if bface is None:
            bface = np.zeros((3,) + shp)
        on_dev = 0 if isinstance(prim, np.ndarray) else 1
        check(lib().hamr_grid_get_state(self.h, block, _ptr(prim), _ptr(bface), on_dev, _stream(stream)))
        return prim, bface

    def step(self, dt=-1.0, block=0, stream=None, stats=False):
        st = StepStats() if stats else None
        check(lib().hamr_block_step(self.h, block, float(dt), _stream(stream), C.byref(st) if stats else None))
        return st.as_dict() if stats else None

    def batch_step(self, n_fine_substeps, stream=None, stats=False):
        st = StepStats() if stats else None
        check(lib().hamr_batch_step(self.h, int(n_fine_substeps), _stream(stream), C.byref(st) if stats else None))
        return st.as_dict() if stats else None

    def fill_ghosts(self, stream=None):
        check(lib().hamr_grid_fill_ghosts(self.h, _stream(stream)))

    def set_fine_dt(self, dt_fine):
        """Fixed fine dt of the batched periods (<= 0: the CFL dt)."""
        check(lib().hamr_grid_set_fine_dt(self.h, float(dt_fine)))

    def set_ghost_maps(self, on):
        """Ghost fill from the locations stored at creation (True) or located on every stage (False);
        returns the previous setting."""
        was = C.c_int(0)
        check(lib().hamr_grid_set_ghost_maps(self.h, 1 if on else 0, C.byref(was)))
        return bool(was.value)

    def block_max(self, field=0, stream=None):
        """Maximum of primitive `field` over each block's interior cells (numpy array, one per block)."""
        out = np.zeros(len(self.blocks))
        check(lib().hamr_grid_block_max(self.h, int(field), out.ctypes.data_as(C.POINTER(C.c_double)),
                                        _stream(stream)))
        return out

    def regrid(self, blocks, stream=None):
        """Replaces the block tree by `blocks` (BlockDesc list), the state carried over."""
        arr = (BlockDesc * len(blocks))(*blocks)
        check(lib().hamr_grid_regrid(self.h, len(blocks), arr, _stream(stream)))
        self._blocks = arr
        self.blocks = list(blocks)

    def set_timing(self, enable):
        check(lib().hamr_grid_set_timing(self.h, int(bool(enable))))

    def timing(self):
        """{group: (launches, ms)} of the grid's kernel groups since the last reset."""
        arr = (KernelTime * 16)()
        n = C.c_int()
        check(lib().hamr_grid_timing(self.h, arr, 16, C.byref(n)))
        return {arr[k].name.decode(): (arr[k].launches, arr[k].ms) for k in range(min(n.value, 16))}

    def stats(self):
        st = StepStats()
        check(lib().hamr_grid_stats(self.h, C.byref(st)))
        return st.as_dict()

    def autotune(self, stream=None):
        """Pick the fastest launch shapes for this grid's kernels on its current state (hamr_grid_autotune)."""
        r = TuneReport()
        check(lib().hamr_grid_autotune(self.h, _stream(stream), C.byref(r)))
        return r.as_dict()

    def launch_shapes(self):
        r = TuneReport()
        check(lib().hamr_grid_launch_shapes(self.h, C.byref(r)))
        return r.as_dict()

    def set_launch_shapes(self, **shapes):
        """Sets launch shapes (recon_seg, recon_x1_sweep, bs_recon, bs_flux, bs_update); others kept."""
        r = TuneReport()
        check(lib().hamr_grid_launch_shapes(self.h, C.byref(r)))
        for k, v in shapes.items():
            setattr(r, k, int(v))
        check(lib().hamr_grid_set_launch_shapes(self.h, C.byref(r)))

    def set_mlp(self, mlp, mode=0):
        """Attach `mlp` to the grid's inversions (None detaches): mode MLP_FIRST (0) starts Newton from
        its guess, MLP_RESCUE (1) uses it where the start from the previous primitives fails."""
        check(lib().hamr_grid_set_mlp(self.h, mlp.h if mlp is not None else None, int(mode)))
        self._mlp = mlp


def c2p_desc(metric=METRIC_KS, a=0.9375, gam=13.0 / 9.0, flags=0, mlp=None):
    d = C2PDesc()
    d.metric, d.a, d.gam, d.flags = metric, a, gam, flags
    d.mlp = mlp.h if mlp is not None else None
    return d


def con2prim(U, B, x1, x2, prim, status, iters=None, metric=METRIC_KS, a=0.9375, gam=13.0 / 9.0, flags=0,
             stream=None, mlp=None, mlp_mode=MLP_FIRST):
    """Inverts n states in place on the device (SoA torch tensors: U (6, n), B (3, n), prim (8, n)).
    With `mlp` (an Mlp), Newton starts from the network's guess (mlp_mode MLP_FIRST, flag C2P_MLP) or
    uses it where the start from prim fails (MLP_RESCUE, flag C2P_MLP_RESCUE)."""
    if mlp is not None:
        flags |= C2P_MLP if mlp_mode == MLP_FIRST else C2P_MLP_RESCUE
    d = c2p_desc(metric, a, gam, flags, mlp)
    n = prim.shape[1]
    check(lib().hamr_con2prim(C.byref(d), n, _ptr(U), _ptr(B), _ptr(x1), _ptr(x2), _ptr(prim), _ptr(status),
                              _ptr(iters), _stream(stream)))


def prim2cons(prim, x1, x2, U, metric=METRIC_KS, a=0.9375, gam=13.0 / 9.0, stream=None):
    """U (6, n) = the conserved variables of prim (8, n) at positions x1, x2 (device tensors)."""
    d = c2p_desc(metric, a, gam)
    check(lib().hamr_prim2cons(C.byref(d), prim.shape[1], _ptr(prim), _ptr(x1), _ptr(x2), _ptr(U), _stream(stream)))


class Mlp:
    """The learned inversion guess (hamr_mlp_*): a model on the current device."""

    NPARAM, NNORM = 9154, 24

    def __init__(self, seed=0):
        h = C.c_void_p()
        check(lib().hamr_mlp_create(C.byref(h), C.c_uint64(seed)))
        self.h = h.value

    def close(self):
        if getattr(self, "h", None):
            lib().hamr_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        p = np.zeros(self.NPARAM, dtype=np.float32)
        nrm = np.zeros(self.NNORM, dtype=np.float32)
        check(lib().hamr_mlp_get_params(self.h, p.ctypes.data, nrm.ctypes.data))
        return p, nrm

    def set_params(self, params=None, norm=None):
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        nrm = None if norm is None else np.ascontiguousarray(norm, dtype=np.float32)
        check(lib().hamr_mlp_set_params(self.h, None if p is None else p.ctypes.data,
                                        None if nrm is None else nrm.ctypes.data))

    @staticmethod
    def features(U, B, x1, x2, feat, prim=None, targ=None, metric=METRIC_KS, a=0.9375, gam=13.0 / 9.0,
                 stream=None):
        d = c2p_desc(metric, a, gam)
        check(lib().hamr_mlp_features(C.byref(d), U.shape[1], _ptr(U), _ptr(B), _ptr(x1), _ptr(x2), _ptr(prim),
                                      _ptr(feat), _ptr(targ), _stream(stream)))

    def fit_norm(self, feat, targ, stream=None):
        check(lib().hamr_mlp_fit_norm(self.h, feat.shape[1], _ptr(feat), _ptr(targ), _stream(stream)))

    def train(self, feat, targ, steps, batch=8192, lr=2e-3, lr_final=2e-5, seed=5, stream=None):
        a = MlpTrainArgs()
        a.steps, a.batch, a.lr, a.lr_final, a.seed = steps, batch, lr, lr_final, seed
        loss = np.zeros(steps, dtype=np.float32)
        check(lib().hamr_mlp_train(self.h, feat.shape[1], _ptr(feat), _ptr(targ), C.byref(a), loss.ctypes.data,
                                   _stream(stream)))
        return loss

    def loss_grad(self, feat, targ, stream=None):
        g = np.zeros(self.NPARAM, dtype=np.float32)
        L = np.zeros(1, dtype=np.float32)
        check(lib().hamr_mlp_loss_grad(self.h, feat.shape[1], _ptr(feat), _ptr(targ), g.ctypes.data, L.ctypes.data,
                                       _stream(stream)))
        return float(L[0]), g

    def forward(self, feat, out, tensor_cores=True, stream=None):
        check(lib().hamr_mlp_forward(self.h, feat.shape[1], _ptr(feat), _ptr(out), int(bool(tensor_cores)),
                                     _stream(stream)))

    def error_flag(self):
        f = C.c_int()
        check(lib().hamr_mlp_error_flag(self.h, C.byref(f)))
        return f.value


def measure_fp64_peak(stream=None):
    """Measured FP64 FMA rate of the current device in GFLOP/s."""
    g = C.c_double()
    check(lib().hamr_measure_fp64_peak(_stream(stream), C.byref(g)))
    return g.value


def check_conversions(nrandom=1 << 24, seed=10192):
    """The integer-pipe binary32 <-> binary64 conversions against the hardware's:
    (widening mismatches, first bad binary32 pattern, narrowing mismatches, first bad binary64 pattern)."""
    out = (C.c_longlong * 4)()
    check(lib().hamr_check_conversions(int(nrandom), int(seed), out))
    return tuple(out)


def block_step_noalloc(grid, prim, bface, dt=-1.0, stream=None):
    """One step of `grid`'s single block through hamr_block_step_noalloc, on the
    caller's device tensors `prim` (8, ...) and `bface` (3, ...) in place."""
    check(lib().hamr_block_step_noalloc(C.byref(grid.desc), _ptr(prim), _ptr(bface), float(dt), _stream(stream)))
