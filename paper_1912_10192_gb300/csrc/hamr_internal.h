// hamr_internal.h -- host-side structures shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

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
    int bc[6];
    const double* gc;  // centre tables
    const double* gf1; // x1-face tables
    const double* gf2; // x2-face tables
};

struct PhysArgs {
    double gam;
    double cour;
    int recon;
    int riemann;
    int floors;
};

// device scratch/state of one block
struct BlockState {
    double* P;      // 8 fields: primitives at t^n (stepped in place)
    double* B;      // 3 fields: face B at t^n (stepped in place)
    double* Ph;     // 8 fields: primitives at t^{n+1/2}
    double* Bh;     // 3 fields: face B at t^{n+1/2}
    double* QL;     // 8 fields: left edge values of the current direction
    double* QR;     // 8 fields: right edge values of the current direction
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

cudaError_t launch_geometry(const GeomArgs& A, cudaStream_t s);

// api.cu: records the calling thread's last-error message and returns `code`
int set_error(int code, const char* fmt, ...);

// step.cu
cudaError_t launch_centre_b(const BlockView& v, double* P, const double* B, cudaStream_t s);
cudaError_t launch_bc(const BlockView& v, double* P, double* B, cudaStream_t s);
cudaError_t launch_recon(const BlockView& v, const PhysArgs& ph, int dir, const double* P, double* QL, double* QR,
                         cudaStream_t s);
cudaError_t launch_flux(const BlockView& v, const PhysArgs& ph, int dir, const double* QL, const double* QR,
                        const double* Bf, double* F, cudaStream_t s);
cudaError_t launch_emf(const BlockView& v, double* const F[3], double* E, cudaStream_t s);
cudaError_t launch_ct(const BlockView& v, const double* E, const double* Bbase, double* Bout, const double* dscal,
                      double dt_factor, cudaStream_t s);
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

// c2p.cu
cudaError_t launch_con2prim(const hamr_c2p_desc& d, int64_t n, const double* U, const double* B, const double* x1,
                            const double* x2, double* prim, int32_t* status, int32_t* iters, cudaStream_t s);

}  // namespace hamr
