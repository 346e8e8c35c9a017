// noalloc.cu -- hamr_block_step_noalloc: one midpoint step of one small block
// with every byte of scratch in a fixed, file-scope device array.
//
// For callers that cannot allocate device memory: code that runs inside a
// memory pool it does not own, a host framework that forbids cudaMalloc
// while it holds the device, or a step that must not allocate once it has
// been set up. The caller passes the block's state (inputs and outputs);
// everything else -- geometry tables, the midpoint state, edge values,
// fluxes, EMFs, the U^n cache, status bytes and counters -- lives in
// `g_noalloc_scratch` below, a static array every GPU that loads the library
// holds until the process exits.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "grmhd.cuh"
#include "hamr_internal.h"

namespace hamr {
namespace {

constexpr long NA_CELLS = HAMR_NOALLOC_MAX_CELLS;  // padded cells of the largest block
constexpr long NA_PLANE = HAMR_NOALLOC_MAX_PLANE;  // padded (i, j) points of its tables
constexpr long NA_FIELDS = 8 + 3 + 8 + 8 + 24 + 3 + 6;  // Ph, Bh, QL, QR, F1..3, E, Un
constexpr long NA_TAB = NGEOM_C + 2 * NGEOM;
// doubles: fields + tables + status bytes (as doubles) + 3 x 32 scalars
constexpr long NA_DOUBLES = NA_FIELDS * NA_CELLS + NA_TAB * NA_PLANE + NA_CELLS / 8 + 96;

static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

// device address of the array, per device; filled once by setup()
constexpr int NA_MAXDEV = 64;
double* g_ptr[NA_MAXDEV] = {nullptr};
std::mutex g_mu;

int setup(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(HAMR_ECUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAXDEV) return set_error(HAMR_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return set_error(HAMR_ECUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                             cudaGetErrorString(e));
        g_ptr[dev] = (double*)p;
    }
    *out = g_ptr[dev];
    return HAMR_OK;
}

#define NA_TRY(call)                                                                                          \
    do {                                                                                                      \
        cudaError_t e_ = (call);                                                                              \
        if (e_ != cudaSuccess) return set_error(HAMR_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

}  // namespace
}  // namespace hamr

using namespace hamr;

extern "C" int hamr_block_step_noalloc(const hamr_grid_desc* d, double* prim, double* bface, double dt,
                                       void* stream) {
    // every check hamr_grid_create makes (metric, spin, gam, cour, options, cell widths, boundary
    // placement), then the limits of this entry point
    int vrc = validate_desc(d);
    if (vrc) return vrc;
    if (d->nblocks != 1) return set_error(HAMR_EINVAL, "need a descriptor with one block");
    if (!prim || !bface) return set_error(HAMR_EINVAL, "prim and bface must not be NULL");
    if (!std::isfinite(dt)) return set_error(HAMR_EINVAL, "dt must be finite");
    const hamr_block_desc& B = d->blocks[0];
    const long n1p = B.n1 + 2 * NG, n2p = B.n2 + 2 * NG, n3p = B.n3 + 2 * NG;
    if (n1p * n2p * n3p > NA_CELLS || n1p * n2p > NA_PLANE)
        return set_error(HAMR_EINVAL,
                         "block %dx%dx%d too large for the no-allocation step: (n1+6)(n2+6)(n3+6) must be <= %ld "
                         "and (n1+6)(n2+6) <= %ld",
                         B.n1, B.n2, B.n3, NA_CELLS, NA_PLANE);
    if (d->precision != HAMR_PREC_FP64) return set_error(HAMR_EINVAL, "the no-allocation step is FP64 only");
    if (d->smr != 0) return set_error(HAMR_EINVAL, "the no-allocation step does not do internal SMR");

    double* base = nullptr;
    int rc = setup(&base);
    if (rc) return rc;
    cudaStream_t cs = (cudaStream_t)stream;

    BlockView v;
    std::memset(&v, 0, sizeof(v));
    v.n1 = B.n1;
    v.n2 = B.n2;
    v.n3 = B.n3;
    v.n1p = (int)n1p;
    v.n2p = (int)n2p;
    v.n3p = (int)n3p;
    v.nc = n1p * n2p * n3p;                    // the caller's field stride
    v.n2d = ((n1p * n2p + 31) / 32) * 32;      // table planes on 256-byte boundaries
    v.dx1 = B.dx1;
    v.dx2 = B.dx2;
    v.dx3 = B.dx3;
    v.idx1 = 1.0 / B.dx1;
    v.idx2 = 1.0 / B.dx2;
    v.idx3 = 1.0 / B.dx3;
    v.x1min = B.x1min;
    for (int f = 0; f < 6; f++) v.bc[f] = B.bc[f];

    // carve the array (field stride = the caller's padded cell count)
    double* p = base;
    BlockState s;
    s.P = prim;
    s.B = bface;
    s.Ph = p;
    p += 8 * v.nc;
    s.Bh = p;
    p += 3 * v.nc;
    s.QL = p;
    p += 8 * v.nc;
    s.QR = p;
    p += 8 * v.nc;
    for (int k = 0; k < 3; k++) {
        s.F[k] = p;
        p += 8 * v.nc;
    }
    s.E = p;
    p += 3 * v.nc;
    s.Un = p;
    p += 6 * v.nc;
    s.geom_c = p;
    p += NGEOM_C * v.n2d;
    s.geom_f1 = p;
    p += NGEOM * v.n2d;
    s.geom_f2 = p;
    p += NGEOM * v.n2d;
    s.status = (uint8_t*)p;
    p += (v.nc + 7) / 8;
    s.dscal = p;
    s.dmax = (unsigned long long*)(p + 32);
    s.dcnt = (unsigned long long*)(p + 64);
    v.gc = s.geom_c;
    v.gf1 = s.geom_f1;
    v.gf2 = s.geom_f2;

    PhysArgs ph;
    std::memset(&ph, 0, sizeof(ph));  // FP64 only: no FP32 stage copy, no FP32 fluxes
    ph.gam = d->gam;
    ph.igam = 1.0 / d->gam;
    ph.gfac = (d->gam - 1.0) * ph.igam;
    ph.cour = d->cour;
    ph.recon = d->recon;
    ph.riemann = d->riemann;
    ph.floors = d->floors;
    ph.mixed = 0;
    ph.fp64_inv = 0;
    ph.mlp_img = nullptr;
    ph.mlp_err = nullptr;
    ph.mlp_mode = HAMR_MLP_FIRST;
    default_launch_shapes(ph);
    ph.emf = d->emf;
    ph.flatten = (d->flatten && d->recon == HAMR_RECON_PPM) ? 1 : 0;
    ph.inversion = d->inversion;
    ph.floor_frame = d->floor_frame;
    ph.smr = 0;
    ph.smr_u = nullptr;

    // the array keeps the previous call's contents: clear what must start at zero
    NA_TRY(cudaMemsetAsync(s.Ph, 0, sizeof(double) * 11 * v.nc, cs));
    NA_TRY(cudaMemsetAsync(s.dscal, 0, sizeof(double) * 96, cs));

    GeomArgs A;
    A.metric = d->metric;
    A.a = d->a;
    A.n1 = B.n1;
    A.n2 = B.n2;
    A.n1p = v.n1p;
    A.n2p = v.n2p;
    A.x1min = B.x1min;
    A.x2min = B.x2min;
    A.dx1 = B.dx1;
    A.dx2 = B.dx2;
    A.pole_lo = (B.bc[2] == HAMR_BC_POLAR);
    A.pole_hi = (B.bc[3] == HAMR_BC_POLAR);
    A.table_stride = v.n2d;
    A.centre = s.geom_c;
    A.face1 = s.geom_f1;
    A.face2 = s.geom_f2;
    NA_TRY(launch_geometry(A, cs));

    // the loaded state: centre B from the faces, boundaries, CFL rate
    NA_TRY(launch_centre_b(v, s.P, s.B, cs));
    NA_TRY(launch_bc(v, s.P, s.B, cs));
    NA_TRY(launch_dt_reduce(v, ph, s.P, s.dmax, cs));
    NA_TRY(launch_dt_select(ph, dt, s.dscal, s.dmax, s.dcnt, s.status, v.nc, cs));
    // predictor
    NA_TRY(launch_bc(v, s.P, s.B, cs));
    NA_TRY(launch_kappa(v, ph, s.P, nullptr, s.E, s.Un, cs));
    for (int dir = 1; dir <= 3; dir++) {
        if (ph.flatten) NA_TRY(launch_flatten(v, ph, dir, s.P, nullptr, s.F[dir - 1], cs));
        NA_TRY(launch_recon(v, ph, dir, s.P, nullptr, s.E, s.F[dir - 1], s.QL, s.QR, cs));
        NA_TRY(launch_flux(v, ph, dir, s.QL, s.QR, s.B, s.F[dir - 1], cs));
    }
    NA_TRY(launch_emf(v, s.F, s.E, ph.mixed, s.P, ph.emf ? s.QL : nullptr, cs));
    NA_TRY(launch_ct(v, s.E, s.B, s.Bh, s.dscal, 0.5, cs));
    NA_TRY(launch_update(v, ph, 0, s.P, s.P, s.F, s.Bh, s.Un, s.Ph, s.status, s.dscal, 0.5, s.dmax, s.dcnt, cs));
    // corrector
    NA_TRY(launch_bc(v, s.Ph, s.Bh, cs));
    NA_TRY(launch_kappa(v, ph, s.Ph, nullptr, s.E, nullptr, cs));
    for (int dir = 1; dir <= 3; dir++) {
        if (ph.flatten) NA_TRY(launch_flatten(v, ph, dir, s.Ph, nullptr, s.F[dir - 1], cs));
        NA_TRY(launch_recon(v, ph, dir, s.Ph, nullptr, s.E, s.F[dir - 1], s.QL, s.QR, cs));
        NA_TRY(launch_flux(v, ph, dir, s.QL, s.QR, s.Bh, s.F[dir - 1], cs));
    }
    NA_TRY(launch_emf(v, s.F, s.E, ph.mixed, s.Ph, ph.emf ? s.QL : nullptr, cs));
    NA_TRY(launch_ct(v, s.E, s.B, s.B, s.dscal, 1.0, cs));
    NA_TRY(launch_update(v, ph, 1, s.P, s.Ph, s.F, s.B, s.Un, s.P, s.status, s.dscal, 1.0, s.dmax, s.dcnt, cs));
    NA_TRY(launch_bc(v, s.P, s.B, cs));
    return HAMR_OK;
}
