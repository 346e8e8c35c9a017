// hamr_internal.h -- host-side structures shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/hamr.h"

namespace hamr {

struct GeomArgs {
    int metric;
    double a;
    int n1, n2, n1p, n2p;
    double x1min, x2min, dx1, dx2;
    int pole_lo, pole_hi;
    long table_stride;  // doubles between two components of a table (>= n1p * n2p)
    double* centre;  // NGEOM_C planes
    double* face1;   // NGEOM planes
    double* face2;   // NGEOM planes
};

// Everything a stage kernel needs about one block. Plain pointers into the
// block's device arrays; `nc` is the padded cell count (stride of a field).
struct BlockView {
    int n1, n2, n3, n1p, n2p, n3p;
    long nc, n2d;
    double dx1, dx2, dx3, idx1, idx2, idx3;
    double x1min;  // x1 of the block's lower face (the learned inversion guess takes x1)
    int bc[6];
    const double* gc;  // centre tables
    const double* gf1; // x1-face tables
    const double* gf2; // x2-face tables
    // FP32 copies (mixed precision only, else null): centre metric + connection
    // (NGEOM + 40 planes), face metric (NGEOM planes each); same plane stride n2d
    const float* gc32;
    const float* gf1_32;
    const float* gf2_32;
    // FP32 copy of the stage's primitives (mixed precision, written at the start of each stage),
    // else null
    const float* P32;
    // internal SMR in a block tree: log2 of the coarsest polar block's x2 and x3 cell widths over
    // this block's (0 on a single block; smr_width)
    int smr_l2, smr_l3;
};

struct PhysArgs {
    double gam;
    double igam, gfac;  // 1/gam and (gam - 1)/gam, formed once on the host
    double cour;
    int recon;
    int riemann;
    int floors;
    int mixed;  // 1: reconstruction and face fluxes in FP32 (HAMR_PREC_MIXED, HAMR_PREC_MIXED_FP64INV)
    int fp64_inv;  // 1 (with mixed): connection source and every Newton iteration in FP64
    const uint8_t* mlp_img;  // inference image of the learned inversion guess (nullptr: not used)
    int* mlp_err;            // set to 1 by a CTA whose network waits gave up
    int mlp_mode;            // HAMR_MLP_FIRST or HAMR_MLP_RESCUE
    // launch shapes (hamr_grid_autotune): threads per CTA of the reconstruction,
    // flux and cell-update kernels, cells per thread of the x2/x3 sweeps
    int bs_recon, bs_flux, bs_update, recon_seg;
    int recon_x1_sweep;  // 1: x1 edge values by pencil sweeps (like x2/x3), 0: by warp rows
    int emf;      // HAMR_EMF_*
    int flatten;  // 1: PPM shock flattening (only set with HAMR_RECON_PPM)
    int inversion;  // HAMR_INV_*
    int floor_frame;  // HAMR_FLOOR_*
    // mixed precision on a single block: the cell update and the boundary kernels keep the next
    // stage's FP32 copy of the primitives (p32w), its entropy tracer kappa (k32, in the EMF array's
    // first field, free from the face update to the next EMFs) and, in the corrector, the next step's
    // U^n kappa, so that no separate pass forms them (0: the separate passes)
    int stage32;
    float* p32w;
    float* k32;
    double* un;       // the U^n cache (its entropy slot takes the next step's kappa)
    int flux32;       // mixed precision: the face fluxes' field slots (6, 7) also in FP32, after the FP64
                      // fields, for the FP32 EMFs
    int smr;          // internal SMR levels next to polar faces (0: off)
    double* smr_u;    // scratch of the deferred conserved states (6 fields, stride nc) when smr > 0
};

// group width in x3 of row j under internal SMR (1: not grouped): row jp from a polar face of the
// coarsest polar blocks is grouped 2^n wide, n the largest level with jp < 2^(smr - n); a polar block
// with 2^smr_l2 times finer x2 cells and 2^smr_l3 times finer x3 cells groups its row j as their row
// j >> smr_l2, over 2^smr_l3 times as many of its own cells (the same phi range)
__host__ __device__ inline int smr_width(const BlockView& v, const PhysArgs& ph, int j) {
    if (ph.smr <= 0) return 1;
    int jp = 1 << 30;
    if (v.bc[2] == HAMR_BC_POLAR) jp = j;
    if (v.bc[3] == HAMR_BC_POLAR) jp = (v.n2 - 1 - j < jp) ? v.n2 - 1 - j : jp;
    const int jb = jp >> v.smr_l2;
    for (int n = ph.smr; n >= 1; n--)
        if (jb < (1 << (ph.smr - n))) return (1 << n) << v.smr_l3;
    return 1;
}

// grouped rows next to each polar face under internal SMR
__host__ __device__ inline int smr_rows(const BlockView& v, const PhysArgs& ph) {
    return (ph.smr > 0) ? ((1 << (ph.smr - 1)) << v.smr_l2) : 0;
}

// threads of one reconstruction launch (FP64): rows along x1 in warps of 32
// lanes that produce RECON_TILE cells each; pencils along x2 or x3 of
// RECON_SEG cells per thread; 7 variables each. FP32: one thread per cell.
constexpr int RECON_TILE = 28;
constexpr int RECON_SEG = 16;  // default sweep length
constexpr int RECON_X1_SWEEP = 1;  // default form of the x1 edge values
__host__ __device__ inline long recon_threads(const BlockView& v, int dir, int fp32, int seg, int x1_sweep = 0) {
    const long n1 = v.n1 + 2, n2 = v.n2 + 2, n3 = v.n3 + 2;
    if (fp32) return n1 * n2 * n3;  // one thread per cell
    // 8 variables: the 7 primitives other than B^dir and the entropy tracer
    if (dir == 1 && !x1_sweep) return ((n1 + RECON_TILE - 1) / RECON_TILE) * 32 * n2 * n3 * 8;
    if (dir == 1) return n2 * n3 * ((n1 + seg - 1) / seg) * 8;
    if (dir == 2) return n1 * n3 * ((n2 + seg - 1) / seg) * 8;
    return n1 * n2 * ((n3 + seg - 1) / seg) * 8;
}
// monotone map of (non-NaN) doubles to unsigned integers and back: maxima by atomicMax
__host__ __device__ inline unsigned long long ordered_bits(double x) {
    unsigned long long u;
    memcpy(&u, &x, sizeof(u));
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__host__ __device__ inline double ordered_to_double(unsigned long long o) {
    const unsigned long long u = (o >> 63) ? (o & 0x7fffffffffffffffull) : ~o;
    double x;
    memcpy(&x, &u, sizeof(x));
    return x;
}

// the launch-shape defaults (what hamr_grid_autotune starts from)
inline void default_launch_shapes(PhysArgs& ph) {
    ph.bs_recon = 128;
    ph.bs_flux = 128;
    ph.bs_update = 128;
    ph.recon_seg = RECON_SEG;
    ph.recon_x1_sweep = RECON_X1_SWEEP;
}

// device scratch/state of one block
struct BlockState {
    double* P;      // 8 fields: primitives at t^n (stepped in place)
    double* B;      // 3 fields: face B at t^n (stepped in place)
    double* Ph;     // 8 fields: primitives at t^{n+1/2}
    double* Bh;     // 3 fields: face B at t^{n+1/2}
    double* QL;     // 8 fields: left edge values of the current direction (FP32 in mixed precision)
    double* QR;     // 8 fields: right edge values of the current direction
    float* P32;     // mixed precision: FP32 copy of the stage's primitives (8 fields, stride nc), else null
    double* F[3];   // 8 fields each: face fluxes (x sqrt(-g)) of directions 1..3
    double* E;      // 3 fields: edge EMFs E1, E2, E3
    double* Un;     // 6 fields: U(P^n) cached by the predictor for the corrector
    uint8_t* status;
    double* geom_c;
    double* geom_f1;
    double* geom_f2;
    // device scalars: [0] dt of the current step, [1] user dt (<=0: CFL),
    // [2] max over cells of sum_i v_f^i/dx^i (as ordered bits), counters
    double* dscal;
    unsigned long long* dmax;  // [0] inverse-dt max bits
    unsigned long long* dcnt;  // [0..3] ok, entropy, fail, floor
};

// one block of a multi-block grid as the batched kernels see it
struct DevBlock {
    BlockView v;
    double lo[4], hi[4], h[4];  // extents and cell sizes, index 1..3
    int lat;
    double *P, *B, *Ph, *Bh, *QL, *QR, *F1, *F2, *F3, *E, *Un, *Pold, *Bold;
    float* P32;  // mixed precision: FP32 copy of the stage's primitives
    uint8_t* status;
    double* dscal;  // [0] dt of the block's step, [1] = 1.0
    unsigned long long *dmax, *dcnt;
    long gofs_cell, gofs_face;  // first stored ghost-cell / ghost-face location of the block
    int ng_cell, ng_face;       // the block's ghost cells / ghost faces (all three directions)
};

// domain and block lookup for the ghost kernels
struct AmrDomain {
    const DevBlock* tab;
    int nb;
    const int* bucket;  // block index of each bucket of a uniform grid over the domain
    int nbk[4];
    double dlo[4], dhi[4], bkh[4];
    int per[4];
};

cudaError_t launch_geometry(const GeomArgs& A, cudaStream_t s);
// FP32 copy of the first nplanes planes (stride `stride` elements) of a table
cudaError_t launch_table_f32(const double* src, float* dst, int nplanes, long stride, cudaStream_t s);

// api.cu: records the calling thread's last-error message and returns `code`
int set_error(int code, const char* fmt, ...);
// api.cu: the descriptor checks of hamr_grid_create (HAMR_OK or HAMR_EINVAL with a message)
int validate_desc(const hamr_grid_desc* d);
// api.cu: internal SMR in a block tree: whether B touches a polar face, and log2 of the coarsest
// polar block's x2 and x3 cell widths over B's (false unless both are powers of 2)
bool smr_polar(const hamr_block_desc& B);
bool smr_factors(const hamr_grid_desc& d, const hamr_block_desc& B, int* l2, int* l3);

// step.cu
cudaError_t launch_centre_b(const BlockView& v, double* P, const double* B, cudaStream_t s);
// atomicMax of ordered_bits(P[q]) over the interior cells into *out (initialise to 0)
cudaError_t launch_block_max(const BlockView& v, const double* P, int q, unsigned long long* out, cudaStream_t s);
cudaError_t launch_bc(const BlockView& v, double* P, double* B, cudaStream_t s, float* P32 = nullptr,
                      float* K32 = nullptr);
// entropy tracer kappa = p / rho^gam of every padded cell into K (FP32 view of K when mixed)
// Un: the U^n cache (predictor) or nullptr (corrector); the predictor stores kappa in its entropy slot
cudaError_t launch_kappa(const BlockView& v, const PhysArgs& ph, const double* P, const float* P32, double* K,
                         double* Un, cudaStream_t s);
// edge values of direction dir: the 7 primitives other than B^dir into their fields of QL / QR,
// kappa (from K) into the B^dir fields; Fl: the flattening coefficients (when ph.flatten)
cudaError_t launch_recon(const BlockView& v, const PhysArgs& ph, int dir, const double* P, const float* P32,
                         const double* K, const double* Fl, double* QL, double* QR, cudaStream_t s);
cudaError_t launch_to_f32(const BlockView& v, const double* P, float* P32, cudaStream_t s);
// PPM shock-flattening coefficients of direction dir into Fl (field 0 of the dir-flux array,
// which launch_flux overwrites after launch_recon has read it)
cudaError_t launch_flatten(const BlockView& v, const PhysArgs& ph, int dir, const double* P, const float* P32,
                           double* Fl, cudaStream_t s);
cudaError_t launch_flux(const BlockView& v, const PhysArgs& ph, int dir, const double* QL, const double* QR,
                        const double* Bf, double* F, cudaStream_t s);
// upwinded EMFs when Ec (3 fields of scratch, stride nc) is given: the cell EMFs of P go there first
cudaError_t launch_emf(const BlockView& v, double* const F[3], double* E, int mixed, const double* P, double* Ec,
                       cudaStream_t s);
cudaError_t launch_ct(const BlockView& v, const double* E, const double* Bbase, double* Bout, const double* dscal,
                      double dt_factor, cudaStream_t s);
// internal SMR (single-block grids): group means of the radial and far-side theta faces and
// interpolated inner phi faces after CT; one inversion per group after the cell update
cudaError_t launch_smr_emf(const BlockView& v, const PhysArgs& ph, double* E, cudaStream_t s);
cudaError_t launch_smr_cells(const BlockView& v, const PhysArgs& ph, int corrector, const double* Pf, const double* Bn,
                             double* Po, uint8_t* status, unsigned long long* dmax, unsigned long long* dcnt,
                             cudaStream_t s);
// threads of one block's SMR EMF and cell kernels (0 where the block groups no row)
long smr_emf_threads(const BlockView& v, const PhysArgs& ph);
long smr_cell_threads(const BlockView& v, const PhysArgs& ph);
// batched over list[0..nlist): the stage's EMFs; the cells of the predictor (sigma 0) or the corrector
// (1); maxwork: the largest smr_*_threads of the listed blocks
cudaError_t launch_smr_emf_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, const PhysArgs& ph,
                                 cudaStream_t s);
cudaError_t launch_smr_cells_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, const PhysArgs& ph,
                                   int sigma, cudaStream_t s);
cudaError_t launch_update(const BlockView& v, const PhysArgs& ph, int corrector, const double* Pbase,
                          const double* Pflux, double* const F[3], const double* Bnew, double* Un, double* Pout,
                          uint8_t* status, const double* dscal, double dt_factor, unsigned long long* dmax,
                          unsigned long long* dcnt, cudaStream_t s);
cudaError_t launch_dt_reduce(const BlockView& v, const PhysArgs& ph, const double* P, unsigned long long* dmax,
                             cudaStream_t s);
cudaError_t launch_dt_select(const PhysArgs& ph, double user_dt, double* dscal, unsigned long long* dmax,
                             unsigned long long* dcnt, uint8_t* status, long nc, cudaStream_t s);

// probe.cu
cudaError_t measure_fp64_peak(cudaStream_t s, double* gflops);
// probe.cu: the integer-pipe conversions (cvt.cuh) against the hardware ones: out = {widening
// mismatches, first mismatching binary32 pattern or ~0, narrowing mismatches, first binary64 pattern or ~0}
cudaError_t check_conversions(unsigned long long nrand, unsigned long long seed, unsigned long long out[4]);

// step.cu, batched over the blocks list[0..nlist) of a table (sigma: 0 predictor, 1 corrector)
cudaError_t launch_to_f32_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, int sigma,
                                cudaStream_t s);
// kappa of each listed block into field 0 of its EMF array (maxwork: largest padded cell count)
cudaError_t launch_kappa_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, const PhysArgs& ph,
                               int sigma, cudaStream_t s);
cudaError_t launch_recon_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, const PhysArgs& ph,
                               int dir, int sigma, cudaStream_t s);
// maxcells: largest (n1 + 2)(n2 + 2)(n3 + 2) of the listed blocks
cudaError_t launch_flatten_batch(const DevBlock* tab, const int* list, int nlist, long maxcells, const PhysArgs& ph,
                                 int dir, int sigma, cudaStream_t s);
cudaError_t launch_flux_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, const PhysArgs& ph,
                              int dir, int sigma, cudaStream_t s);
cudaError_t launch_emf_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, int mixed, int upwind,
                             long maxcells, int sigma, cudaStream_t s);
// sigma 0: Bh = B + dt/2 curl E; 1: B += dt curl E; 2: B += curl E (E holds time-integrated corrections)
cudaError_t launch_ct_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, int sigma, cudaStream_t s);
cudaError_t launch_update_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, const PhysArgs& ph,
                                int sigma, cudaStream_t s);
cudaError_t launch_dt_reduce_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, const PhysArgs& ph,
                                   cudaStream_t s);
cudaError_t launch_save_old_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, cudaStream_t s);
// re-inversion of refluxed cells: cell[i] (block, padded index), Ucorr[6][n] = U(P) + flux correction
cudaError_t launch_reflux_u0(const DevBlock* tab, int n, const int* cblk, const long* cidx, const int* nrec,
                             const int* recs, const double* rec_dU, int nrec_tot, double* Ucorr, const PhysArgs& ph,
                             cudaStream_t s);
cudaError_t launch_reflux_cells(const DevBlock* tab, int n, const int* cblk, const long* cidx, const double* Ucorr,
                                long stride, const PhysArgs& ph, cudaStream_t s);
// refluxed internal-SMR groups: group g's w[g] cells at list positions first[g].. (relative to cblk,
// cidx and Ucorr); inverted as one cell
cudaError_t launch_reflux_groups(const DevBlock* tab, int ngrp, const int* first, const int* w, const int* cblk,
                                 const long* cidx, const double* Ucorr, long stride, const PhysArgs& ph,
                                 cudaStream_t s);

// amr.cu
struct AmrImpl;

// the learned inversion guess (mlp.cu): FP32 master parameters, Adam
// moments, the standardisation and the bf16 inference image, on one device
}  // namespace hamr
struct hamr_mlp {
    float* params = nullptr;  // MLP_NPARAM
    float* grad = nullptr;
    float* m1 = nullptr;      // Adam moments
    float* m2 = nullptr;
    float* norm = nullptr;    // MLP_NNORM: fmean, fstd, ymean, ystd
    uint8_t* img = nullptr;   // inference image (MLP_IMG_BYTES)
    double* sums = nullptr;   // scratch of the standardisation fit
    float* loss = nullptr;    // per-step loss accumulators of a training call
    long loss_cap = 0;
    int* err = nullptr;       // set by a CTA whose network waits gave up
    long long adam_t = 0;
    int device = 0;
};
namespace hamr {
int amr_create(AmrImpl** out, const hamr_grid_desc& d, const std::vector<BlockView>& views,
               const std::vector<BlockState>& st, const PhysArgs& ph);
void amr_destroy(AmrImpl* M);
int amr_after_load(AmrImpl* M, int block, cudaStream_t s);
int amr_period(AmrImpl* M, cudaStream_t s, int nperiods, bool use_graph);
int amr_info(const AmrImpl* M, int* lmax, double* dtf_host);
int amr_links(const AmrImpl* M, int* counts5);
int amr_fill(AmrImpl* M, cudaStream_t s);
// fills every block of M from the old tree at its current state (regridding)
int amr_regrid_fill(const AmrImpl* old, AmrImpl* M, cudaStream_t s);
// fine dt of every following period (<= 0: the CFL dt); read on the device, no graph rebuild
int amr_set_fine_dt(AmrImpl* M, double dt);
// ghost fill from the stored locations (on != 0, the default where they fit) or by locating on every launch
int amr_set_ghost_maps(AmrImpl* M, int on, int* was);
int amr_set_phys(AmrImpl* M, const PhysArgs& ph);
int amr_time_group(AmrImpl* M, const PhysArgs& ph, int which, cudaStream_t cs, float* ms);
const uint8_t* mlp_image(const hamr_mlp* m);
int* mlp_error_ptr(const hamr_mlp* m);

// c2p.cu
cudaError_t launch_con2prim(const hamr_c2p_desc& d, int64_t n, const double* U, const double* B, const double* x1,
                            const double* x2, double* prim, int32_t* status, int32_t* iters, cudaStream_t s);

}  // namespace hamr
