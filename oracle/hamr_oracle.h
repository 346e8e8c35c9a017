/* hamr_oracle.h -- C interface of the plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this library. It shares no code with
 * the CUDA path (paper_1912_10192_gb300/csrc) and neither includes the other.
 *
 * Layout used by every array argument of the grid functions ("padded"):
 *   a cell field is [n3+6][n2+6][n1+6] doubles (3 ghost layers per side),
 *   index ((k+3)*(n2+6) + (j+3))*(n1+6) + (i+3), i (x1 = log r) fastest.
 *   Primitive arrays are 8 such fields: rho, u_g, utilde^1..3, B^1..3 (centre).
 *   Face-B arrays are 3 such fields: Bbar^d stored at the lower d-face of the
 *   cell with the same index (Bbar = sqrt(-g) B^d, the staggered CT field).
 */
#ifndef HAMR_ORACLE_H
#define HAMR_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_BC_OUTFLOW = 0, ORA_BC_PERIODIC = 1, ORA_BC_POLAR = 2, ORA_BC_OUTFLOW_NOINFLOW = 3, ORA_BC_BLOCK = 4 };
/* ORA_METRIC_SPHERICAL: flat space in the same log-r spherical coordinates
 * (the Kerr-Schild form with the mass set to 0 and a = 0) */
enum { ORA_METRIC_KS = 0, ORA_METRIC_MINKOWSKI = 1, ORA_METRIC_SPHERICAL = 2 };
enum { ORA_RECON_PPM = 0, ORA_RECON_MC = 1, ORA_RECON_MINMOD = 2 };
enum { ORA_FLUX_HLL = 0, ORA_FLUX_LLF = 1 };
enum { ORA_EMF_AVERAGE = 0, ORA_EMF_UPWIND = 1 };

enum { ORA_INV_NEWTON = 0, ORA_INV_AITKEN = 1 };
enum { ORA_FLOOR_FLUID = 0, ORA_FLOOR_DRIFT = 1 };

typedef struct {
    int n1, n2, n3;                 /* interior cells per direction */
    double x1min, x2min, x3min;     /* lower corner in internal coordinates */
    double dx1, dx2, dx3;           /* uniform cell sizes */
    int metric;                     /* ORA_METRIC_* */
    double a;                       /* black-hole spin (KS) */
    double gam;                     /* adiabatic index */
    double cour;                    /* Courant factor C0 */
    int recon;                      /* ORA_RECON_* */
    int riemann;                    /* ORA_FLUX_* */
    int bc[6];                      /* x1lo x1hi x2lo x2hi x3lo x3hi: ORA_BC_* */
    int floors;                     /* 1: apply the density/energy floors */
    int emf;                        /* ORA_EMF_*: edge EMFs as the 4-flux average or upwinded */
    int flatten;                    /* 1: PPM shock flattening (Colella & Woodward 1984) */
    int inversion;                  /* ORA_INV_*: energy inversion by 2-D Newton or Aitken-accelerated fixed point */
    int floor_frame;                /* ORA_FLOOR_*: floor material added in the fluid frame or the drift frame */
    int smr;                        /* internal SMR levels n_max next to polar faces (0: off; single grids) */
} ora_desc;

/* ---- point-wise pieces (each documented in hamr_oracle.cpp) ---- */
void ora_geom(const ora_desc* d, double x1, double x2, double* gcov16, double* gcon16,
              double* gdet, double* alpha);
void ora_conn(const ora_desc* d, double x1, double x2, double* conn64);
void ora_state(const ora_desc* d, const double* pr8, double x1, double x2, double* ucon4,
               double* ucov4, double* bcon4, double* bcov4, double* bsq);
void ora_p2uf(const ora_desc* d, const double* pr8, double x1, double x2, int dir, double* out9);
void ora_vchar(const ora_desc* d, const double* pr8, double x1, double x2, int dir, double* vp,
               double* vm);
void ora_face_flux(const ora_desc* d, const double* pl8, const double* pr8, double x1, double x2,
                   int dir, double* f8);
void ora_source(const ora_desc* d, const double* pr8, double x1, double x2, double* q6);
void ora_recon_line(int recon, int n, const double* q, double* al, double* ar);
/* PPM shock flattening: coefficients of a line from u and the velocity
 * primitive along it, and PPM edge values with given coefficients */
/* Newman-Hamlin pressure map of the Aitken inversion: normal-frame E = -Q.n,
 * Qt^2, (Q.B)^2, B^2, D and a trial p -> (W, v^2, next p); W = -1 if invalid */
void ora_nh_map(double E, double S2, double T2, double B2, double D, double gam, double p, double* out3);
/* the floors of Sec. 2.7 on n primitive states (slots 5..7: centre B), r[n] the radius of the
 * floor thresholds; hit[n] = 1 where a floor applied */
void ora_floors_many(const ora_desc* d, long n, double* pr8, const double* x1, const double* x2, const double* r,
                     int* hit);
void ora_flatten_line(int n, double gam, const double* u, const double* w, double* f);
void ora_recon_line_flat(int n, const double* q, const double* f, double* al, double* ar);
/* con2prim on n independent states: U6 (sqrt(-g) weighted), B3 centre B^i,
 * x1/x2 positions, pr8 in: guess, out: result; status/iters per state.
 * entropy_only = 1 skips the energy inversion (tests of the backup path). */
void ora_c2p_many(const ora_desc* d, long n, const double* U6, const double* B3,
                  const double* x1, const double* x2, double* pr8, int* status, int* iters,
                  int entropy_only);
void ora_p2u_many(const ora_desc* d, long n, const double* pr8, const double* x1,
                  const double* x2, double* U6);

/* ---- single-block grid ---- */
typedef struct ora_grid ora_grid;
ora_grid* ora_grid_new(const ora_desc* d);
void ora_grid_free(ora_grid* g);
void ora_grid_set(ora_grid* g, const double* prim, const double* bface);
void ora_grid_get(const ora_grid* g, double* prim, double* bface);
void ora_grid_bc(ora_grid* g);
double ora_grid_dt(ora_grid* g);
double ora_grid_step(ora_grid* g, double dt);
void ora_grid_stats(const ora_grid* g, long long* counts4);
void ora_grid_divb(const ora_grid* g, double* divb_cells);
void ora_grid_status(const ora_grid* g, int* status_cells);
/* face fluxes of the current state (ghosts filled first) as a stage computes
 * them: out[d][m][cell] for face direction d = 0..2 and slot m = 0..7 (0..5
 * the conserved variables, 5 the entropy tracer), padded-block layout; a
 * dir-face at cell index (i, j, k) is the face at i - 1/2 (dir 1) etc.;
 * faces outside the computed range are 0 */
void ora_grid_fluxes(ora_grid* g, double* out);

/* ---- multi-block grid: static refinement + local adaptive time steps ----
 * Blocks tile the domain; a face with bc ORA_BC_BLOCK takes its ghosts from
 * the neighbouring blocks, other faces map ghost positions across the
 * physical boundary (outflow, periodic, polar) before looking up the block
 * that holds them. lat = LAT level: the block steps with 2^lat dt_fine. */
typedef struct {
    int n1, n2, n3;
    double x1min, x2min, x3min, dx1, dx2, dx3;
    int bc[6];
    int lat;
} ora_block;
typedef struct ora_amr ora_amr;
/* phys: metric, a, gam, cour, recon, riemann, floors of `phys` are used */
ora_amr* ora_amr_new(const ora_desc* phys, int nb, const ora_block* blocks);
void ora_amr_free(ora_amr* m);
void ora_amr_set(ora_amr* m, int b, const double* prim, const double* bface);
void ora_amr_get(const ora_amr* m, int b, double* prim, double* bface);
/* fills every block's ghosts from the current state (no stepping) */
void ora_amr_fill(ora_amr* m);
/* advances the grid by one schedule period (2^Lmax fine substeps);
 * dt_fine <= 0: the CFL fine step min_b dt_b / 2^lat_b; returns dt_fine */
double ora_amr_period(ora_amr* m, double dt_fine);
void ora_amr_stats(const ora_amr* m, long long* counts4);
/* a new tree with the old tree's state (cells: copy / volume average /
 * MINMOD prolongation of the primitives; faces: copy / area average /
 * Balsara 2001 divergence-free prolongation); the old tree is unchanged
 * apart from its ghost zones */
ora_amr* ora_amr_regrid(ora_amr* old, int nb, const ora_block* blocks);

/* learned inversion guess: the ten inputs of n conserved states (U6 and Bc3
 * as in ora_c2p_many; f10 is n x 10) and the two targets of n primitive
 * states (pr8 n x 8; y2 is n x 2), defined in hamr_oracle.cpp */
void ora_mlp_features(const ora_desc* d, long n, const double* U6, const double* Bc3, const double* x1,
                      const double* x2, double* f10);
void ora_mlp_targets(const ora_desc* d, long n, const double* pr8, const double* x1, const double* x2,
                     double* y2);

/* flop counters (meaningful only in the counting build) */
void ora_flops_reset(void);
void ora_flops_get(unsigned long long* out5);
/* per phase (recon, flux, emf, ct, update, cfl) x counter class, counting build only */
void ora_flops_phase(unsigned long long* out30);

#ifdef __cplusplus
}
#endif
#endif
