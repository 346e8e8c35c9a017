// api.cu -- the C ABI declared in include/hamr.h: grid lifetime, state I/O,
// the per-block midpoint step and the standalone inversion.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "grmhd.cuh"
#include "hamr_internal.h"

using namespace hamr;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(call)                                                                                   \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) return fail(HAMR_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// launches a kernel group of `nk` kernels on stream `cs`, counted under `kind`
// and bracketed by events when the grid's timer is on
#define LAUNCH(g, kind, nk, cs, call)                                    \
    do {                                                                 \
        cudaEvent_t ea_ = nullptr, eb_ = nullptr;                        \
        if ((g)->timer.enabled) {                                        \
            ea_ = (g)->timer.get();                                      \
            eb_ = (g)->timer.get();                                      \
            cudaEventRecord(ea_, cs);                                    \
        }                                                                \
        CUDA_TRY(call);                                                  \
        if ((g)->timer.enabled) {                                        \
            cudaEventRecord(eb_, cs);                                    \
            (g)->timer.pending.push_back({kind, ea_, eb_});              \
        }                                                                \
        (g)->timer.launches[kind] += (nk);                               \
    } while (0)

}  // namespace

namespace {

// launch accounting and optional event timing of kernel groups
struct Timer {
    static constexpr int NK = 8;
    const char* names[NK] = {"dt", "bc", "recon", "flux", "emf", "ct", "update", "load"};
    long long launches[NK] = {0};
    double ms[NK] = {0};
    bool enabled = false;
    struct Pending {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    void drain() {  // device must be idle
        for (auto& p : pending) {
            float t = 0.f;
            cudaEventElapsedTime(&t, p.a, p.b);
            ms[p.kind] += t;
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
    }
    void reset() {
        for (int k = 0; k < NK; k++) {
            launches[k] = 0;
            ms[k] = 0.0;
        }
    }
    ~Timer() {
        for (auto& p : pending) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

enum { K_DT = 0, K_BC, K_RECON, K_FLUX, K_EMF, K_CT, K_UPDATE, K_LOAD };

}  // namespace

int hamr::set_error(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

struct hamr_grid {
    Timer timer;
    AmrImpl* amr = nullptr;
    hamr_grid_desc desc;
    std::vector<hamr_block_desc> blocks;
    std::vector<BlockState> st;
    std::vector<BlockView> view;
    std::vector<void*> arena;
    std::vector<int> loaded;
    PhysArgs ph;
    int device;
    double fine_dt = 0.0;  // hamr_grid_set_fine_dt (<= 0: CFL)
    bool stage32_valid = false;  // ph.stage32: the FP32 copy, its kappa and the U^n kappa are the state's
    bool ghosts_valid = false;   // single block: the ghost cells and faces of P, B are the boundary conditions'
};

// The descriptor checks of hamr_grid_create, also run by hamr_block_step_noalloc.
bool hamr::smr_polar(const hamr_block_desc& B) { return B.bc[2] == HAMR_BC_POLAR || B.bc[3] == HAMR_BC_POLAR; }

// log2 of the coarsest polar block's x2 and x3 cell widths over B's; false unless both are powers of 2
// (within 1e-9) between 2^0 and 2^6
bool hamr::smr_factors(const hamr_grid_desc& d, const hamr_block_desc& B, int* l2, int* l3) {
    double h2 = 0.0, h3 = 0.0;
    for (int b = 0; b < d.nblocks; b++)
        if (smr_polar(d.blocks[b])) {
            h2 = std::max(h2, d.blocks[b].dx2);
            h3 = std::max(h3, d.blocks[b].dx3);
        }
    const double r[2] = {h2 / B.dx2, h3 / B.dx3};
    int l[2] = {0, 0};
    for (int q = 0; q < 2; q++) {
        if (!(r[q] >= 1.0 - 1e-9 && r[q] <= 64.0 * (1.0 + 1e-9))) return false;
        l[q] = (int)std::lround(std::log2(r[q]));
        if (std::fabs(r[q] - std::ldexp(1.0, l[q])) > 1e-9 * r[q]) return false;
    }
    *l2 = l[0];
    *l3 = l[1];
    return true;
}

int hamr::validate_desc(const hamr_grid_desc* d) {
    if (!d) return fail(HAMR_EINVAL, "descriptor is NULL");
    if (d->nblocks < 1 || !d->blocks) return fail(HAMR_EINVAL, "nblocks must be >= 1 with a block array");
    if (d->metric != HAMR_METRIC_KS && d->metric != HAMR_METRIC_MINKOWSKI && d->metric != HAMR_METRIC_SPHERICAL)
        return fail(HAMR_EINVAL, "unknown metric %d", d->metric);
    if (d->metric == HAMR_METRIC_KS && !(std::fabs(d->a) < 1.0)) return fail(HAMR_EINVAL, "spin must satisfy |a| < 1");
    if (!(d->gam > 1.0 && d->gam <= 2.0)) return fail(HAMR_EINVAL, "gam must be in (1, 2]");
    if (!(d->cour > 0.0 && d->cour <= 1.0)) return fail(HAMR_EINVAL, "cour must be in (0, 1]");
    if (d->recon < 0 || d->recon > 2) return fail(HAMR_EINVAL, "unknown recon %d", d->recon);
    if (d->riemann < 0 || d->riemann > 1) return fail(HAMR_EINVAL, "unknown riemann %d", d->riemann);
    if (d->precision != HAMR_PREC_FP64 && d->precision != HAMR_PREC_MIXED && d->precision != HAMR_PREC_MIXED_FP64INV)
        return fail(HAMR_EINVAL, "unknown precision %d", d->precision);
    if (d->emf != HAMR_EMF_AVERAGE && d->emf != HAMR_EMF_UPWIND) return fail(HAMR_EINVAL, "unknown emf %d", d->emf);
    if (d->flatten != 0 && d->flatten != 1) return fail(HAMR_EINVAL, "flatten must be 0 or 1, got %d", d->flatten);
    if (d->inversion != HAMR_INV_NEWTON && d->inversion != HAMR_INV_AITKEN)
        return fail(HAMR_EINVAL, "unknown inversion %d", d->inversion);
    if (d->floor_frame != HAMR_FLOOR_FLUID && d->floor_frame != HAMR_FLOOR_DRIFT)
        return fail(HAMR_EINVAL, "unknown floor_frame %d", d->floor_frame);
    if (d->smr < 0 || d->smr > 4) return fail(HAMR_EINVAL, "smr must be in 0..4, got %d", d->smr);
    if (d->smr > 0) {
        // every polar block groups its rows like the coarsest polar blocks (smr_width): its cell widths
        // a power of 2 finer, n3 a multiple of twice its widest group, its grouped rows within half of n2
        bool polar = false;
        for (int b = 0; b < d->nblocks; b++) polar = polar || smr_polar(d->blocks[b]);
        if (!polar) return fail(HAMR_EINVAL, "internal SMR needs a polar x2 boundary");
        for (int b = 0; b < d->nblocks; b++) {
            const hamr_block_desc& B = d->blocks[b];
            if (!smr_polar(B)) continue;
            int l2 = 0, l3 = 0;
            if (!smr_factors(*d, B, &l2, &l3))
                return fail(HAMR_EINVAL, "block %d: internal SMR needs x2 and x3 cell widths a power of 2 finer than "
                            "the coarsest polar block's", b);
            const int rows = (1 << (d->smr - 1)) << l2, wmax = (1 << d->smr) << l3;
            if (B.n3 % (2 * wmax) != 0)
                return fail(HAMR_EINVAL, "block %d: internal SMR needs n3 a multiple of %d", b, 2 * wmax);
            if (B.n2 < 2 * rows) return fail(HAMR_EINVAL, "block %d: internal SMR needs n2 >= %d", b, 2 * rows);
        }
    }
    for (int b = 0; b < d->nblocks; b++) {
        const hamr_block_desc& B = d->blocks[b];
        if (B.n1 < 4 || B.n2 < 4 || B.n3 < 4) return fail(HAMR_EINVAL, "block %d: each n must be >= 4", b);
        if ((long)(B.n1 + 6) * (B.n2 + 6) * (B.n3 + 6) > (1L << 28))
            return fail(HAMR_EINVAL, "block %d: too many cells", b);
        if (!(B.dx1 > 0 && B.dx2 > 0 && B.dx3 > 0)) return fail(HAMR_EINVAL, "block %d: dx must be > 0", b);
        const bool multi = d->nblocks > 1;
        for (int f = 0; f < 6; f++) {
            const int bc = B.bc[f];
            if (bc < 0 || bc > 4) return fail(HAMR_EINVAL, "block %d: unknown bc %d", b, bc);
            if (bc == HAMR_BC_BLOCK && !multi) return fail(HAMR_EINVAL, "block %d: bc BLOCK needs several blocks", b);
            if (bc == HAMR_BC_POLAR && (f / 2) != 1) return fail(HAMR_EINVAL, "block %d: polar bc only on x2", b);
            if (bc == HAMR_BC_OUTFLOW_NOINFLOW && (f / 2) != 0)
                return fail(HAMR_EINVAL, "block %d: noinflow bc only on x1", b);
            if (bc == HAMR_BC_POLAR && (B.n3 % 2) != 0) return fail(HAMR_EINVAL, "block %d: polar bc needs even n3", b);
            if (bc == HAMR_BC_POLAR && d->metric == HAMR_METRIC_MINKOWSKI)
                return fail(HAMR_EINVAL, "block %d: polar bc needs spherical coordinates (KS or SPHERICAL)", b);
        }
        if (!multi && ((B.bc[0] == HAMR_BC_PERIODIC) != (B.bc[1] == HAMR_BC_PERIODIC) ||
                       (B.bc[2] == HAMR_BC_PERIODIC) != (B.bc[3] == HAMR_BC_PERIODIC) ||
                       (B.bc[4] == HAMR_BC_PERIODIC) != (B.bc[5] == HAMR_BC_PERIODIC)))
            return fail(HAMR_EINVAL, "block %d: periodic bc must be on both sides", b);
        const double pi = 3.14159265358979323846;
        if (B.bc[2] == HAMR_BC_POLAR && std::fabs(B.x2min) > 1e-12)
            return fail(HAMR_EINVAL, "block %d: lower polar bc needs x2min = 0", b);
        if (B.bc[3] == HAMR_BC_POLAR && std::fabs(B.x2min + B.n2 * B.dx2 - pi) > 1e-9)
            return fail(HAMR_EINVAL, "block %d: upper polar bc needs x2max = pi", b);
    }
    return HAMR_OK;
}

namespace {

int validate(const hamr_grid_desc* d) { return validate_desc(d); }

void free_grid(hamr_grid* g) {
    if (g->amr) amr_destroy(g->amr);
    for (void* p : g->arena)
        if (p) cudaFree(p);
    delete g;
}

int alloc_block(hamr_grid* g, int b) {
    const hamr_block_desc& B = g->blocks[b];
    BlockView v;
    std::memset(&v, 0, sizeof(v));
    v.n1 = B.n1;
    v.n2 = B.n2;
    v.n3 = B.n3;
    v.n1p = B.n1 + 2 * NG;
    v.n2p = B.n2 + 2 * NG;
    v.n3p = B.n3 + 2 * NG;
    v.nc = (long)v.n1p * v.n2p * v.n3p;
    v.n2d = (long)v.n1p * v.n2p;
    v.dx1 = B.dx1;
    v.dx2 = B.dx2;
    v.dx3 = B.dx3;
    v.idx1 = 1.0 / B.dx1;
    v.idx2 = 1.0 / B.dx2;
    v.idx3 = 1.0 / B.dx3;
    v.x1min = B.x1min;
    for (int f = 0; f < 6; f++) v.bc[f] = B.bc[f];

    // every field and table is padded to a whole number of 256-byte lines
    const size_t fld = align256(sizeof(double) * (size_t)v.nc);
    const size_t tab = align256(sizeof(double) * (size_t)v.n2d);
    v.nc = (long)(fld / sizeof(double));   // stride between two fields
    v.n2d = (long)(tab / sizeof(double));  // stride between two table components
    const int nfields = 8 + 3 + 8 + 3 + 8 + 8 + 27 + 3 + 6;
    const size_t stbytes = align256((size_t)v.nc);
    // mixed precision: the FP32 copy of the primitives and FP32 metric/connection tables
    const bool mixed = (g->desc.precision != HAMR_PREC_FP64);
    const size_t fld32 = align256(sizeof(float) * (size_t)v.nc * NPRIM);
    const size_t tab32 = align256(sizeof(float) * (size_t)v.n2d);
    const int nc32 = NGEOM + 40;  // centre planes the FP32 path reads: metric and connection
    size_t bytes = fld * nfields + stbytes + tab * (NGEOM_C + 2 * NGEOM) + 256 * 3;
    if (mixed) bytes += fld32 + tab32 * (nc32 + 2 * NGEOM);
    void* base = nullptr;
    cudaError_t e = cudaMalloc(&base, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(HAMR_ENOMEM, "cudaMalloc of %zu bytes for block %d failed: %s", bytes, b, cudaGetErrorString(e));
    }
    g->arena.push_back(base);
    char* p = (char*)base;
    auto take = [&](size_t n) {
        char* r = p;
        p += n;
        return r;
    };
    BlockState s;
    s.P = (double*)take(8 * fld);
    s.B = (double*)take(3 * fld);
    s.Ph = (double*)take(8 * fld);
    s.Bh = (double*)take(3 * fld);
    s.QL = (double*)take(8 * fld);
    s.QR = (double*)take(8 * fld);
    for (int d = 0; d < 3; d++) s.F[d] = (double*)take(9 * fld);  // 8 FP64 fields, 2 FP32 (mixed, one block)
    s.E = (double*)take(3 * fld);
    s.Un = (double*)take(6 * fld);
    s.status = (uint8_t*)take(stbytes);
    s.geom_c = (double*)take(tab * NGEOM_C);
    s.geom_f1 = (double*)take(tab * NGEOM);
    s.geom_f2 = (double*)take(tab * NGEOM);
    s.dscal = (double*)take(256);
    s.dmax = (unsigned long long*)take(256);
    s.dcnt = (unsigned long long*)take(256);
    s.P32 = nullptr;
    float *g32c = nullptr, *g32f1 = nullptr, *g32f2 = nullptr;
    if (mixed) {
        s.P32 = (float*)take(fld32);
        g32c = (float*)take(tab32 * nc32);
        g32f1 = (float*)take(tab32 * NGEOM);
        g32f2 = (float*)take(tab32 * NGEOM);
    }
    v.gc = s.geom_c;
    v.gf1 = s.geom_f1;
    v.gf2 = s.geom_f2;
    v.gc32 = g32c;
    v.gf1_32 = g32f1;
    v.gf2_32 = g32f2;
    v.P32 = s.P32;
    CUDA_TRY(cudaMemset(base, 0, bytes));
    GeomArgs A;
    A.metric = g->desc.metric;
    A.a = g->desc.a;
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
    A.centre = s.geom_c;
    A.face1 = s.geom_f1;
    A.face2 = s.geom_f2;
    A.table_stride = v.n2d;
    CUDA_TRY(launch_geometry(A, 0));
    if (mixed) {
        CUDA_TRY(launch_table_f32(s.geom_c, g32c, nc32, v.n2d, 0));
        CUDA_TRY(launch_table_f32(s.geom_f1, g32f1, NGEOM, v.n2d, 0));
        CUDA_TRY(launch_table_f32(s.geom_f2, g32f2, NGEOM, v.n2d, 0));
    }
    g->st.push_back(s);
    g->view.push_back(v);
    g->loaded.push_back(0);
    return HAMR_OK;
}

cudaStream_t S(void* stream) { return (cudaStream_t)stream; }

// after a state load: centre B from the faces, boundaries (single-block grids;
// a multi-block grid fills its ghosts from the neighbouring blocks), CFL rate
cudaError_t load_kernels(const BlockView& v, const PhysArgs& ph, BlockState& s, bool bc, cudaStream_t cs) {
    cudaError_t e = launch_centre_b(v, s.P, s.B, cs);
    if (e == cudaSuccess && bc) e = launch_bc(v, s.P, s.B, cs);
    if (e == cudaSuccess) e = launch_dt_reduce(v, ph, s.P, s.dmax, cs);
    return e;
}

// copy between the user's padded layout (stride n1p*n2p*n3p) and the grid's (stride v.nc)
int copy_fields(double* dst, long dstride, const double* src, long sstride, long n, int nfields, cudaMemcpyKind kind,
                cudaStream_t s, bool sync) {
    for (int f = 0; f < nfields; f++) {
        if (sync)
            CUDA_TRY(cudaMemcpy(dst + f * dstride, src + f * sstride, sizeof(double) * n, kind));
        else
            CUDA_TRY(cudaMemcpyAsync(dst + f * dstride, src + f * sstride, sizeof(double) * n, kind, s));
    }
    return HAMR_OK;
}

int check_block(const hamr_grid* g, int block) {
    if (!g) return fail(HAMR_EINVAL, "grid is NULL");
    if (block < 0 || block >= (int)g->blocks.size()) return fail(HAMR_EINVAL, "block %d out of range", block);
    return HAMR_OK;
}

}  // namespace

extern "C" {

const char* hamr_last_error(void) { return g_err.c_str(); }

int hamr_grid_create(const hamr_grid_desc* d, hamr_grid** out) {
    if (!out) return fail(HAMR_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate(d);
    if (rc) return rc;
    hamr_grid* g = new hamr_grid;
    g->desc = *d;
    g->blocks.assign(d->blocks, d->blocks + d->nblocks);
    g->desc.blocks = g->blocks.data();
    g->ph.gam = d->gam;
    g->ph.igam = 1.0 / d->gam;
    g->ph.gfac = (d->gam - 1.0) * g->ph.igam;
    g->ph.cour = d->cour;
    g->ph.recon = d->recon;
    g->ph.riemann = d->riemann;
    g->ph.floors = d->floors;
    g->ph.mixed = (d->precision != HAMR_PREC_FP64);
    g->ph.fp64_inv = (d->precision == HAMR_PREC_MIXED_FP64INV);
    g->ph.mlp_img = nullptr;
    g->ph.mlp_err = nullptr;
    g->ph.mlp_mode = HAMR_MLP_FIRST;
    default_launch_shapes(g->ph);
    g->ph.emf = d->emf;
    g->ph.flatten = (d->flatten && d->recon == HAMR_RECON_PPM) ? 1 : 0;
    g->ph.inversion = d->inversion;
    g->ph.floor_frame = d->floor_frame;
    g->ph.smr = d->smr;
    g->ph.smr_u = nullptr;
    cudaGetDevice(&g->device);
    for (int b = 0; b < d->nblocks; b++) {
        rc = alloc_block(g, b);
        if (rc) {
            free_grid(g);
            return rc;
        }
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_grid(g);
        return fail(HAMR_ECUDA, "geometry build failed: %s", cudaGetErrorString(e));
    }
    if (d->smr > 0) g->ph.smr_u = g->st[0].QR;  // free once the fluxes are formed
    g->ph.stage32 = 0;
    g->ph.flux32 = g->ph.mixed;  // FP32 copies of the flux field slots for the FP32 EMFs
    g->ph.p32w = nullptr;
    g->ph.k32 = nullptr;
    g->ph.un = nullptr;
    if (d->nblocks == 1 && g->ph.mixed) {  // the update and the boundary kernels keep the FP32 stage copy
        g->ph.stage32 = 1;
        g->ph.p32w = g->st[0].P32;
        g->ph.k32 = reinterpret_cast<float*>(g->st[0].E);
        g->ph.un = g->st[0].Un;
    }
    if (d->nblocks > 1) {
        rc = amr_create(&g->amr, g->desc, g->view, g->st, g->ph);
        if (rc) {
            free_grid(g);
            return rc;
        }
    }
    *out = g;
    return HAMR_OK;
}

int hamr_grid_destroy(hamr_grid* g) {
    if (!g) return HAMR_OK;
    cudaDeviceSynchronize();
    free_grid(g);
    return HAMR_OK;
}

int hamr_grid_set_state(hamr_grid* g, int block, const double* prim, const double* bface, int on_device,
                        void* stream) {
    int rc = check_block(g, block);
    if (rc) return rc;
    if (!prim || !bface) return fail(HAMR_EINVAL, "prim and bface must not be NULL");
    const BlockView& v = g->view[block];
    BlockState& s = g->st[block];
    const long n = (long)v.n1p * v.n2p * v.n3p;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    rc = copy_fields(s.P, v.nc, prim, n, n, 8, kind, S(stream), !on_device);
    if (rc) return rc;
    rc = copy_fields(s.B, v.nc, bface, n, n, 3, kind, S(stream), !on_device);
    if (rc) return rc;
    cudaStream_t cs = S(stream);
    CUDA_TRY(cudaMemsetAsync(s.dmax, 0, sizeof(unsigned long long), cs));
    LAUNCH(g, K_LOAD, g->amr ? 2 : 6, cs, load_kernels(v, g->ph, s, g->amr == nullptr, cs));
    g->stage32_valid = false;
    g->ghosts_valid = (g->amr == nullptr);  // the load applied the boundary conditions
    if (g->amr) {
        rc = amr_after_load(g->amr, block, cs);
        if (rc) return rc;
    }
    g->loaded[block] = 1;
    return HAMR_OK;
}

int hamr_grid_get_state(const hamr_grid* g, int block, double* prim, double* bface, int on_device, void* stream) {
    int rc = check_block(g, block);
    if (rc) return rc;
    const BlockView& v = g->view[block];
    const BlockState& s = g->st[block];
    const long n = (long)v.n1p * v.n2p * v.n3p;
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(S(stream)));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (prim) {
        rc = copy_fields(prim, n, s.P, v.nc, n, 8, kind, S(stream), !on_device);
        if (rc) return rc;
    }
    if (bface) {
        rc = copy_fields(bface, n, s.B, v.nc, n, 3, kind, S(stream), !on_device);
        if (rc) return rc;
    }
    return HAMR_OK;
}

int hamr_block_step(hamr_grid* g, int block, double dt, void* stream, hamr_step_stats* stats) {
    int rc = check_block(g, block);
    if (rc) return rc;
    if (!g->loaded[block]) return fail(HAMR_ESTATE, "block %d has no state: call hamr_grid_set_state first", block);
    if (!std::isfinite(dt)) return fail(HAMR_EINVAL, "dt must be finite");
    if (g->amr) return fail(HAMR_EINVAL, "a multi-block grid advances with hamr_batch_step");
    const BlockView& v = g->view[block];
    BlockState& s = g->st[block];
    const PhysArgs& ph = g->ph;
    cudaStream_t cs = S(stream);
    LAUNCH(g, K_DT, 1, cs, launch_dt_select(ph, dt, s.dscal, s.dmax, s.dcnt, s.status, v.nc, cs));
    // mixed precision: the boundary kernels copy the ghosts of the FP32 stage copy and its kappa, whose
    // interior the cell update wrote; a separate pass forms them where no update did (after loading)
    float* P32g = ph.stage32 ? s.P32 : nullptr;
    float* K32g = ph.stage32 ? reinterpret_cast<float*>(s.E) : nullptr;
    const bool fused = ph.stage32 && g->stage32_valid;
    // predictor: P^n, B^n -> P^{n+1/2}, B^{n+1/2} (the ghosts of P^n are current after a load or a step,
    // which end with the boundary conditions)
    if (!g->ghosts_valid) LAUNCH(g, K_BC, 4, cs, launch_bc(v, s.P, s.B, cs, P32g, K32g));
    g->ghosts_valid = false;  // until this step has ended (an error on the way leaves them unknown)
    g->stage32_valid = false;
    if (ph.mixed && !fused) LAUNCH(g, K_BC, 1, cs, launch_to_f32(v, s.P, s.P32, cs));
    if (!fused) LAUNCH(g, K_RECON, 1, cs, launch_kappa(v, ph, s.P, s.P32, s.E, s.Un, cs));
    for (int dir = 1; dir <= 3; dir++) {
        if (ph.flatten) LAUNCH(g, K_RECON, 1, cs, launch_flatten(v, ph, dir, s.P, s.P32, s.F[dir - 1], cs));
        LAUNCH(g, K_RECON, 1, cs, launch_recon(v, ph, dir, s.P, s.P32, s.E, s.F[dir - 1], s.QL, s.QR, cs));
        LAUNCH(g, K_FLUX, 1, cs, launch_flux(v, ph, dir, s.QL, s.QR, s.B, s.F[dir - 1], cs));
    }
    LAUNCH(g, K_EMF, ph.emf ? 2 : 1, cs, launch_emf(v, s.F, s.E, ph.mixed ? ((ph.flux32 && !ph.emf) ? 2 : 1) : 0, s.P, ph.emf ? s.QL : nullptr, cs));
    if (ph.smr) LAUNCH(g, K_EMF, 1, cs, launch_smr_emf(v, ph, s.E, cs));
    LAUNCH(g, K_CT, 1, cs, launch_ct(v, s.E, s.B, s.Bh, s.dscal, 0.5, cs));
    LAUNCH(g, K_UPDATE, 1, cs,
           launch_update(v, ph, 0, s.P, s.P, s.F, s.Bh, s.Un, s.Ph, s.status, s.dscal, 0.5, s.dmax, s.dcnt, cs));
    if (ph.smr)
        LAUNCH(g, K_UPDATE, 1, cs, launch_smr_cells(v, ph, 0, s.P, s.Bh, s.Ph, s.status, s.dmax, s.dcnt, cs));
    // corrector: U^n and the fluxes of P^{n+1/2} -> P^{n+1}, B^{n+1} (in place)
    LAUNCH(g, K_BC, 4, cs, launch_bc(v, s.Ph, s.Bh, cs, P32g, K32g));
    if (ph.mixed && !ph.stage32) LAUNCH(g, K_BC, 1, cs, launch_to_f32(v, s.Ph, s.P32, cs));
    if (!ph.stage32) LAUNCH(g, K_RECON, 1, cs, launch_kappa(v, ph, s.Ph, s.P32, s.E, nullptr, cs));
    for (int dir = 1; dir <= 3; dir++) {
        if (ph.flatten) LAUNCH(g, K_RECON, 1, cs, launch_flatten(v, ph, dir, s.Ph, s.P32, s.F[dir - 1], cs));
        LAUNCH(g, K_RECON, 1, cs, launch_recon(v, ph, dir, s.Ph, s.P32, s.E, s.F[dir - 1], s.QL, s.QR, cs));
        LAUNCH(g, K_FLUX, 1, cs, launch_flux(v, ph, dir, s.QL, s.QR, s.Bh, s.F[dir - 1], cs));
    }
    LAUNCH(g, K_EMF, ph.emf ? 2 : 1, cs, launch_emf(v, s.F, s.E, ph.mixed ? ((ph.flux32 && !ph.emf) ? 2 : 1) : 0, s.Ph, ph.emf ? s.QL : nullptr, cs));
    if (ph.smr) LAUNCH(g, K_EMF, 1, cs, launch_smr_emf(v, ph, s.E, cs));
    LAUNCH(g, K_CT, 1, cs, launch_ct(v, s.E, s.B, s.B, s.dscal, 1.0, cs));
    LAUNCH(g, K_UPDATE, 1, cs,
           launch_update(v, ph, 1, s.P, s.Ph, s.F, s.B, s.Un, s.P, s.status, s.dscal, 1.0, s.dmax, s.dcnt, cs));
    if (ph.smr)
        LAUNCH(g, K_UPDATE, 1, cs, launch_smr_cells(v, ph, 1, s.Ph, s.B, s.P, s.status, s.dmax, s.dcnt, cs));
    LAUNCH(g, K_BC, 4, cs, launch_bc(v, s.P, s.B, cs, P32g, K32g));
    g->stage32_valid = ph.stage32 != 0;
    g->ghosts_valid = true;
    if (stats) {
        CUDA_TRY(cudaStreamSynchronize(cs));
        return hamr_grid_stats(g, stats);
    }
    return HAMR_OK;
}

int hamr_batch_step(hamr_grid* g, int n_fine_substeps, void* stream, hamr_step_stats* stats) {
    if (!g) return fail(HAMR_EINVAL, "grid is NULL");
    if (!g->amr) return fail(HAMR_EINVAL, "batched AMR/LAT stepping needs a multi-block grid");
    for (size_t b = 0; b < g->loaded.size(); b++)
        if (!g->loaded[b]) return fail(HAMR_ESTATE, "block %zu has no state", b);
    int lmax = 0;
    int rc = amr_info(g->amr, &lmax, nullptr);
    if (rc) return rc;
    const int period = 1 << lmax;
    if (n_fine_substeps <= 0 || n_fine_substeps % period != 0)
        return fail(HAMR_EINVAL, "n_fine_substeps must be a positive multiple of the period %d", period);
    rc = amr_period(g->amr, S(stream), n_fine_substeps / period, true);
    if (rc) return rc;
    if (stats) {
        CUDA_TRY(cudaStreamSynchronize(S(stream)));
        return hamr_grid_stats(g, stats);
    }
    return HAMR_OK;
}

int hamr_grid_fill_ghosts(hamr_grid* g, void* stream) {
    if (!g) return fail(HAMR_EINVAL, "grid is NULL");
    for (size_t b = 0; b < g->loaded.size(); b++)
        if (!g->loaded[b]) return fail(HAMR_ESTATE, "block %zu has no state", b);
    if (g->amr) return amr_fill(g->amr, S(stream));
    LAUNCH(g, K_BC, 4, S(stream), launch_bc(g->view[0], g->st[0].P, g->st[0].B, S(stream)));
    return HAMR_OK;
}

int hamr_grid_set_timing(hamr_grid* g, int enable) {
    if (!g) return fail(HAMR_EINVAL, "grid is NULL");
    CUDA_TRY(cudaDeviceSynchronize());
    g->timer.drain();
    g->timer.reset();
    g->timer.enabled = (enable != 0);
    return HAMR_OK;
}

int hamr_grid_timing(hamr_grid* g, hamr_kernel_time* out, int max, int* n) {
    if (!g || !n || (max > 0 && !out)) return fail(HAMR_EINVAL, "bad arguments");
    CUDA_TRY(cudaDeviceSynchronize());
    g->timer.drain();
    *n = Timer::NK;
    for (int k = 0; k < Timer::NK && k < max; k++) {
        std::memset(out[k].name, 0, sizeof(out[k].name));
        std::strncpy(out[k].name, g->timer.names[k], sizeof(out[k].name) - 1);
        out[k].launches = g->timer.launches[k];
        out[k].ms = g->timer.ms[k];
    }
    return HAMR_OK;
}

int hamr_measure_fp64_peak(void* stream, double* gflops) {
    if (!gflops) return fail(HAMR_EINVAL, "gflops is NULL");
    CUDA_TRY(measure_fp64_peak(S(stream), gflops));
    return HAMR_OK;
}

int hamr_check_conversions(long long nrandom, unsigned long long seed, long long out4[4]) {
    if (!out4) return fail(HAMR_EINVAL, "out4 is NULL");
    if (nrandom < 0) return fail(HAMR_EINVAL, "nrandom must be >= 0");
    unsigned long long r[4];
    CUDA_TRY(check_conversions((unsigned long long)nrandom, seed, r));
    for (int q = 0; q < 4; q++) out4[q] = (long long)r[q];
    return HAMR_OK;
}

int hamr_grid_set_fine_dt(hamr_grid* g, double dt_fine) {
    if (!g) return fail(HAMR_EINVAL, "grid is NULL");
    if (!g->amr) return fail(HAMR_EINVAL, "a single-block grid takes dt in each hamr_block_step call");
    if (!std::isfinite(dt_fine)) return fail(HAMR_EINVAL, "dt_fine must be finite");
    CUDA_TRY(cudaDeviceSynchronize());
    int rc = amr_set_fine_dt(g->amr, dt_fine);
    if (rc) return rc;
    g->fine_dt = dt_fine > 0.0 ? dt_fine : 0.0;
    return HAMR_OK;
}

int hamr_grid_set_ghost_maps(hamr_grid* g, int on, int* was) {
    if (!g) return fail(HAMR_EINVAL, "grid is NULL");
    if (!g->amr) return fail(HAMR_EINVAL, "a single-block grid has no ghost locations");
    if (on != 0 && on != 1) return fail(HAMR_EINVAL, "on must be 0 or 1");
    CUDA_TRY(cudaDeviceSynchronize());
    return amr_set_ghost_maps(g->amr, on, was);
}

int hamr_grid_block_max(const hamr_grid* g, int field, double* out, void* stream) {
    if (!g) return fail(HAMR_EINVAL, "grid is NULL");
    if (!out) return fail(HAMR_EINVAL, "out is NULL");
    if (field < 0 || field >= NPRIM) return fail(HAMR_EINVAL, "field %d out of range 0..7", field);
    const int nb = (int)g->st.size();
    unsigned long long* d = nullptr;
    CUDA_TRY(cudaMalloc(&d, sizeof(unsigned long long) * nb));
    cudaStream_t cs = S(stream);
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long) * nb, cs);
    for (int b = 0; b < nb && e == cudaSuccess; b++) e = launch_block_max(g->view[b], g->st[b].P, field, d + b, cs);
    std::vector<unsigned long long> h(nb, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, sizeof(unsigned long long) * nb, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    cudaFree(d);
    if (e != cudaSuccess) return fail(HAMR_ECUDA, "block maximum failed: %s", cudaGetErrorString(e));
    for (int b = 0; b < nb; b++) out[b] = ordered_to_double(h[b]);
    return HAMR_OK;
}

int hamr_grid_regrid(hamr_grid* g, int nblocks, const hamr_block_desc* blocks, void* stream) {
    if (!g) return fail(HAMR_EINVAL, "grid is NULL");
    if (!g->amr) return fail(HAMR_EINVAL, "regridding needs a multi-block grid (nblocks >= 2 at creation)");
    if (nblocks < 2 || !blocks) return fail(HAMR_EINVAL, "the new tree needs nblocks >= 2 and a block array");
    for (size_t b = 0; b < g->loaded.size(); b++)
        if (!g->loaded[b]) return fail(HAMR_ESTATE, "block %zu has no state", b);
    hamr_grid_desc d = g->desc;
    d.nblocks = nblocks;
    d.blocks = blocks;
    int rc = validate(&d);
    if (rc) return rc;
    // the same domain: the bounding boxes of the two trees agree
    double lo0[3], hi0[3], lo1[3], hi1[3];
    auto box = [](const hamr_block_desc* B, int n, double* lo, double* hi) {
        for (int e = 0; e < 3; e++) {
            lo[e] = 1e300;
            hi[e] = -1e300;
        }
        for (int b = 0; b < n; b++) {
            const double x0[3] = {B[b].x1min, B[b].x2min, B[b].x3min};
            const double ext[3] = {B[b].n1 * B[b].dx1, B[b].n2 * B[b].dx2, B[b].n3 * B[b].dx3};
            for (int e = 0; e < 3; e++) {
                lo[e] = std::min(lo[e], x0[e]);
                hi[e] = std::max(hi[e], x0[e] + ext[e]);
            }
        }
    };
    box(g->blocks.data(), (int)g->blocks.size(), lo0, hi0);
    box(blocks, nblocks, lo1, hi1);
    for (int e = 0; e < 3; e++) {
        const double tol = 1e-9 * (hi0[e] - lo0[e]);
        if (std::fabs(lo0[e] - lo1[e]) > tol || std::fabs(hi0[e] - hi1[e]) > tol)
            return fail(HAMR_EINVAL, "the new tree covers another domain along x%d", e + 1);
    }
    // a region's cell size changes by at most a factor of 2 (the regrid's operators)
    for (int nbk = 0; nbk < nblocks; nbk++) {
        const hamr_block_desc& B = blocks[nbk];
        const double bl[3] = {B.x1min, B.x2min, B.x3min};
        const double bh[3] = {B.x1min + B.n1 * B.dx1, B.x2min + B.n2 * B.dx2, B.x3min + B.n3 * B.dx3};
        for (const hamr_block_desc& Q : g->blocks) {
            const double ql[3] = {Q.x1min, Q.x2min, Q.x3min};
            const double qh[3] = {Q.x1min + Q.n1 * Q.dx1, Q.x2min + Q.n2 * Q.dx2, Q.x3min + Q.n3 * Q.dx3};
            bool over = true;
            for (int e = 0; e < 3 && over; e++) {
                const double tol = 1e-9 * (hi0[e] - lo0[e]);
                over = (bl[e] < qh[e] - tol) && (ql[e] < bh[e] - tol);
            }
            if (!over) continue;
            const double r = Q.dx1 / B.dx1;
            if (r > 2.0 * (1.0 + 1e-9) || r < 0.5 * (1.0 - 1e-9))
                return fail(HAMR_EINVAL, "new block %d changes the cell size by more than 2x (use hamr_tree_adapt "
                                         "steps of one level)", nbk);
        }
    }
    hamr_grid* ng = new hamr_grid;
    ng->desc = d;
    ng->blocks.assign(blocks, blocks + nblocks);
    ng->desc.blocks = ng->blocks.data();
    ng->ph = g->ph;
    ng->device = g->device;
    for (int b = 0; b < nblocks; b++) {
        rc = alloc_block(ng, b);
        if (rc) {
            free_grid(ng);
            return rc;
        }
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_grid(ng);
        return fail(HAMR_ECUDA, "geometry build failed: %s", cudaGetErrorString(e));
    }
    rc = amr_create(&ng->amr, ng->desc, ng->view, ng->st, ng->ph);
    if (rc) {
        free_grid(ng);
        return rc;
    }
    cudaStream_t cs = S(stream);
    rc = amr_regrid_fill(g->amr, ng->amr, cs);
    if (rc == HAMR_OK) {
        e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) rc = fail(HAMR_ECUDA, "regridding failed: %s", cudaGetErrorString(e));
    }
    if (rc) {
        free_grid(ng);
        return rc;
    }
    if (g->fine_dt > 0.0) {
        rc = amr_set_fine_dt(ng->amr, g->fine_dt);
        if (rc) {
            free_grid(ng);
            return rc;
        }
    }
    ng->fine_dt = g->fine_dt;
    ng->loaded.assign(nblocks, 1);
    // the new tree takes the grid's place; the old one is freed with the temporary
    std::swap(g->amr, ng->amr);
    std::swap(g->blocks, ng->blocks);
    std::swap(g->st, ng->st);
    std::swap(g->view, ng->view);
    std::swap(g->arena, ng->arena);
    std::swap(g->loaded, ng->loaded);
    g->desc.nblocks = nblocks;
    g->desc.blocks = g->blocks.data();
    free_grid(ng);
    return HAMR_OK;
}

int hamr_grid_stats(const hamr_grid* g, hamr_step_stats* stats) {
    if (!g || !stats) return fail(HAMR_EINVAL, "grid and stats must not be NULL");
    CUDA_TRY(cudaDeviceSynchronize());
    std::memset(stats, 0, sizeof(*stats));
    for (size_t b = 0; b < g->st.size(); b++) {
        if (!g->loaded[b]) continue;
        unsigned long long cnt[5], mx;
        double dt;
        CUDA_TRY(cudaMemcpy(cnt, g->st[b].dcnt, sizeof(cnt), cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(&mx, g->st[b].dmax, sizeof(mx), cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(&dt, g->st[b].dscal, sizeof(dt), cudaMemcpyDeviceToHost));
        stats->c2p_ok += (long long)cnt[0];
        stats->c2p_entropy += (long long)cnt[1];
        stats->c2p_fail += (long long)cnt[2];
        stats->floor_hits += (long long)cnt[3];
        stats->newton_iters += (long long)cnt[4];
        double rate;
        std::memcpy(&rate, &mx, sizeof(rate));
        const double dn = g->ph.cour / rate;
        if (b == 0 || dt < stats->dt_used) stats->dt_used = dt;
        if (b == 0 || dn < stats->dt_next) stats->dt_next = dn;
    }
    if (g->amr) {  // multi-block: dt_used = the fine step of the last period; rates are of its start
        int lmax = 0;
        double dtf = 0.0;
        int rc = amr_info(g->amr, &lmax, &dtf);
        if (rc) return rc;
        stats->dt_used = dtf;
        stats->dt_next = 0.0;
    }
    return HAMR_OK;
}

int hamr_con2prim(const hamr_c2p_desc* d, int64_t n, const double* U, const double* B, const double* x1,
                  const double* x2, double* prim, int32_t* status, int32_t* iters, void* stream) {
    if (!d) return fail(HAMR_EINVAL, "descriptor is NULL");
    if (n < 0) return fail(HAMR_EINVAL, "n must be >= 0");
    if (n == 0) return HAMR_OK;
    if (!U || !B || !x1 || !x2 || !prim || !status) return fail(HAMR_EINVAL, "array argument is NULL");
    if (d->metric != HAMR_METRIC_KS && d->metric != HAMR_METRIC_MINKOWSKI && d->metric != HAMR_METRIC_SPHERICAL)
        return fail(HAMR_EINVAL, "unknown metric %d", d->metric);
    if (!(d->gam > 1.0 && d->gam <= 2.0)) return fail(HAMR_EINVAL, "gam must be in (1, 2]");
    if (d->flags & ~(HAMR_C2P_ENTROPY_ONLY | HAMR_C2P_MLP | HAMR_C2P_MLP_RESCUE | HAMR_C2P_AITKEN | HAMR_C2P_MIXED))
        return fail(HAMR_EINVAL, "unknown flags 0x%x", d->flags);
    if ((d->flags & HAMR_C2P_MLP) && (d->flags & HAMR_C2P_MLP_RESCUE))
        return fail(HAMR_EINVAL, "HAMR_C2P_MLP and HAMR_C2P_MLP_RESCUE exclude each other");
    if ((d->flags & (HAMR_C2P_MLP | HAMR_C2P_MLP_RESCUE)) && !d->mlp)
        return fail(HAMR_EINVAL, "a network flag without a network");
    CUDA_TRY(launch_con2prim(*d, n, U, B, x1, x2, prim, status, iters, S(stream)));
    return HAMR_OK;
}

namespace {
// time (ms) of one kernel group on the single-block grid's current state (see amr_time_group)
int time_group_block(hamr_grid* g, const PhysArgs& ph, int which, cudaStream_t cs, float* ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    CUDA_TRY(cudaEventCreate(&a));
    CUDA_TRY(cudaEventCreate(&b));
    float total = 0.0f;
    for (size_t k = 0; k < g->st.size(); k++) {
        BlockState& s = g->st[k];
        const BlockView& v = g->view[k];
        if (ph.mixed) CUDA_TRY(launch_to_f32(v, s.P, s.P32, cs));
        if (which == 0) CUDA_TRY(cudaEventRecord(a, cs));
        CUDA_TRY(launch_kappa(v, ph, s.P, s.P32, s.E, s.Un, cs));
        if (which == 0) {
            float t = 0.0f;
            CUDA_TRY(cudaEventRecord(b, cs));
            CUDA_TRY(cudaEventSynchronize(b));
            CUDA_TRY(cudaEventElapsedTime(&t, a, b));
            total += t;
        }
        for (int dir = 1; dir <= 3; dir++) {
            if (which == 0) CUDA_TRY(cudaEventRecord(a, cs));
            if (ph.flatten) CUDA_TRY(launch_flatten(v, ph, dir, s.P, s.P32, s.F[dir - 1], cs));
            CUDA_TRY(launch_recon(v, ph, dir, s.P, s.P32, s.E, s.F[dir - 1], s.QL, s.QR, cs));
            if (which == 1) CUDA_TRY(cudaEventRecord(a, cs));
            if (which != 0) CUDA_TRY(launch_flux(v, ph, dir, s.QL, s.QR, s.B, s.F[dir - 1], cs));
            if (which <= 1) {
                float t = 0.0f;
                CUDA_TRY(cudaEventRecord(b, cs));
                CUDA_TRY(cudaEventSynchronize(b));
                CUDA_TRY(cudaEventElapsedTime(&t, a, b));
                total += t;
            }
        }
        if (which == 2) {
            float t = 0.0f;
            CUDA_TRY(cudaEventRecord(a, cs));
            CUDA_TRY(launch_update(v, ph, 0, s.P, s.P, s.F, s.B, s.Un, s.Ph, s.status, s.dscal, 0.5, s.dmax, s.dcnt,
                                   cs));
            CUDA_TRY(cudaEventRecord(b, cs));
            CUDA_TRY(cudaEventSynchronize(b));
            CUDA_TRY(cudaEventElapsedTime(&t, a, b));
            total += t;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms = total;
    return HAMR_OK;
}

// best of three timed repetitions after one warm-up
int time_group(hamr_grid* g, const PhysArgs& ph, int which, cudaStream_t cs, float* best) {
    *best = 1e30f;
    g->stage32_valid = false;  // the timed kernels overwrite the FP32 stage copy and the U^n cache
    for (int r = 0; r < 4; r++) {
        float t = 0.0f;
        int rc = g->amr ? amr_time_group(g->amr, ph, which, cs, &t) : time_group_block(g, ph, which, cs, &t);
        if (rc) return rc;
        if (r > 0) *best = std::min(*best, t);
    }
    return HAMR_OK;
}
}  // namespace

int hamr_grid_autotune(hamr_grid* g, void* stream, hamr_tune_report* rep) {
    if (!g || !rep) return fail(HAMR_EINVAL, "grid and report must not be NULL");
    for (size_t b = 0; b < g->loaded.size(); b++)
        if (!g->loaded[b]) return fail(HAMR_ESTATE, "block %zu has no state", b);
    cudaStream_t cs = S(stream);
    CUDA_TRY(cudaDeviceSynchronize());
    std::memset(rep, 0, sizeof(*rep));
    // the timed update uses the dt of the last step; the CFL rate that the next step
    // reads (dmax) is not touched
    PhysArgs ph = g->ph;
    const int segs[3] = {8, 16, 32}, bss[3] = {64, 128, 256}, bsu[2] = {64, 128};
    int rc;
    ph.bs_recon = 128;
    for (int c = 0; c < 3; c++) {
        ph.recon_seg = segs[c];
        if ((rc = time_group(g, ph, 0, cs, &rep->ms_seg[c]))) return rc;
    }
    ph.recon_seg = segs[std::min_element(rep->ms_seg, rep->ms_seg + 3) - rep->ms_seg];
    for (int c = 0; c < 2; c++) {
        ph.recon_x1_sweep = c;
        if ((rc = time_group(g, ph, 0, cs, &rep->ms_x1[c]))) return rc;
    }
    ph.recon_x1_sweep = (rep->ms_x1[0] < rep->ms_x1[1]) ? 0 : 1;
    for (int c = 0; c < 3; c++) {
        ph.bs_recon = bss[c];
        if ((rc = time_group(g, ph, 0, cs, &rep->ms_recon[c]))) return rc;
    }
    ph.bs_recon = bss[std::min_element(rep->ms_recon, rep->ms_recon + 3) - rep->ms_recon];
    for (int c = 0; c < 3; c++) {
        ph.bs_flux = bss[c];
        if ((rc = time_group(g, ph, 1, cs, &rep->ms_flux[c]))) return rc;
    }
    ph.bs_flux = bss[std::min_element(rep->ms_flux, rep->ms_flux + 3) - rep->ms_flux];
    for (int c = 0; c < 2; c++) {
        ph.bs_update = bsu[c];
        if ((rc = time_group(g, ph, 2, cs, &rep->ms_update[c]))) return rc;
    }
    ph.bs_update = ph.mlp_img ? 128 : bsu[std::min_element(rep->ms_update, rep->ms_update + 2) - rep->ms_update];
    // the found shapes against the defaults on the same state (the timed launches write only
    // scratch), alternating, five repetitions each of the three groups together
    PhysArgs ph0 = ph;
    default_launch_shapes(ph0);
    float t_def[5], t_tun[5];
    for (int r = 0; r < 5; r++)
        for (int o = 0; o < 2; o++) {
            const bool def = ((r + o) % 2) == 0;
            float sum = 0.0f;
            for (int which = 0; which < 3; which++) {
                float t = 0.0f;
                if ((rc = time_group(g, def ? ph0 : ph, which, cs, &t))) return rc;
                sum += t;
            }
            (def ? t_def : t_tun)[r] = sum;
        }
    std::sort(t_def, t_def + 5);
    std::sort(t_tun, t_tun + 5);
    rep->ms_default = t_def[2];
    rep->ms_tuned = t_tun[2];
    rep->ms_spread = std::max(t_def[4] - t_def[0], t_tun[4] - t_tun[0]);
    rep->kept_tuned = (t_tun[2] < t_def[2] - rep->ms_spread) ? 1 : 0;
    if (!rep->kept_tuned) ph = ph0;
    rep->recon_seg = ph.recon_seg;
    rep->bs_recon = ph.bs_recon;
    rep->bs_flux = ph.bs_flux;
    rep->bs_update = ph.bs_update;
    rep->recon_x1_sweep = ph.recon_x1_sweep;
    g->ph = ph;
    if (g->amr) return amr_set_phys(g->amr, g->ph);
    return HAMR_OK;
}

int hamr_grid_set_launch_shapes(hamr_grid* g, const hamr_tune_report* rep) {
    if (!g || !rep) return fail(HAMR_EINVAL, "grid and report must not be NULL");
    auto in = [](int x, std::initializer_list<int> ok) {
        for (int v : ok)
            if (x == v) return true;
        return false;
    };
    if (!in(rep->recon_seg, {8, 16, 32}) || !in(rep->recon_x1_sweep, {0, 1}) || !in(rep->bs_recon, {64, 128, 256}) ||
        !in(rep->bs_flux, {64, 128, 256}) || !in(rep->bs_update, {64, 128}))
        return fail(HAMR_EINVAL, "launch shapes out of the supported sets");
    if (g->ph.mlp_img && rep->bs_update != 128) return fail(HAMR_EINVAL, "a grid with a network keeps bs_update 128");
    CUDA_TRY(cudaDeviceSynchronize());
    g->ph.recon_seg = rep->recon_seg;
    g->ph.recon_x1_sweep = rep->recon_x1_sweep;
    g->ph.bs_recon = rep->bs_recon;
    g->ph.bs_flux = rep->bs_flux;
    g->ph.bs_update = rep->bs_update;
    if (g->amr) return amr_set_phys(g->amr, g->ph);
    return HAMR_OK;
}

int hamr_grid_launch_shapes(const hamr_grid* g, hamr_tune_report* rep) {
    if (!g || !rep) return fail(HAMR_EINVAL, "grid and report must not be NULL");
    std::memset(rep, 0, sizeof(*rep));
    rep->recon_seg = g->ph.recon_seg;
    rep->bs_recon = g->ph.bs_recon;
    rep->bs_flux = g->ph.bs_flux;
    rep->bs_update = g->ph.bs_update;
    rep->recon_x1_sweep = g->ph.recon_x1_sweep;
    return HAMR_OK;
}

int hamr_grid_set_mlp(hamr_grid* g, const hamr_mlp* m, int mode) {
    if (!g) return fail(HAMR_EINVAL, "grid is NULL");
    if (mode != HAMR_MLP_FIRST && mode != HAMR_MLP_RESCUE) return fail(HAMR_EINVAL, "unknown mode %d", mode);
    if (m) {
        int dev = -1;
        cudaGetDevice(&dev);
        if (dev != g->device) return fail(HAMR_EINVAL, "grid lives on device %d, device %d is current", g->device, dev);
    }
    CUDA_TRY(cudaDeviceSynchronize());  // no step in flight reads the old arguments
    g->ph.mlp_img = mlp_image(m);
    g->ph.mlp_err = mlp_error_ptr(m);
    g->ph.mlp_mode = mode;
    if (g->amr) return amr_set_phys(g->amr, g->ph);
    return HAMR_OK;
}

}  // extern "C"
