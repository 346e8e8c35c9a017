/* hamr.h -- C ABI of the GB300-native GRMHD block-update library.
 *
 * The library advances ideal GRMHD on logarithmic spherical-polar
 * Kerr-Schild grids with the finite-volume scheme of Liska et al.,
 * "H-AMR: A New GPU-accelerated GRMHD Code for Exascale Computing With 3D
 * Adaptive Mesh Refinement and Local Adaptive Time-stepping"
 * (arXiv 1912.10192):
 *   - PPM reconstruction of primitives (Sec. 2.1),
 *   - HLLE (or LLF) fluxes with the approximate fast speed (Sec. 2.1),
 *   - constrained transport: 4-flux EMF average, staggered face-B update and
 *     face-to-centre average (Sec. 2.5, the CT and EMF equations),
 *   - connection source terms sqrt(-g) T^k_l Gamma^l_{nu k} (Sec. 2.5),
 *   - 2-D Newton-Raphson conserved-to-primitive inversion with an entropy
 *     backup, and floors (Sec. 2.6, 2.7),
 *   - the midpoint predictor/corrector step with the CFL time step (Sec. 2.1),
 * advanced block by block under the AMR / local adaptive time-stepping
 * schedule of Sec. 3.2 and 3.4.
 *
 * Conventions shared by every call
 *   - Units G = M = c = 1; internal coordinates x1 = log r, x2 = theta,
 *     x3 = phi (Sec. 2.2).
 *   - Return value: HAMR_OK (0) or a negative HAMR_E* code; a human-readable
 *     message of the last failure in the calling thread is hamr_last_error().
 *     Per-cell physics failures (an inversion that does not converge, a floor)
 *     are not call errors: they are counted in hamr_step_stats.
 *   - Ownership: the caller owns every pointer it passes and keeps it valid
 *     for the duration of the call (device pointers: until the stream work
 *     it enqueued completes). The grid owns its state, scratch and geometry
 *     tables and frees them in hamr_grid_destroy.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *     default stream). Calls enqueue work and return; results are valid once
 *     the stream has synchronised, unless a call says it synchronises.
 *   - State layout ("padded SoA"): a cell field of a block with n1 x n2 x n3
 *     interior cells is an array of (n3+6)(n2+6)(n1+6) doubles (3 ghost
 *     layers per side), index ((k+3)(n2+6) + (j+3))(n1+6) + (i+3), i fastest.
 *     Primitive state = 8 such fields: rho, u_g, utilde^1, utilde^2,
 *     utilde^3, B^1, B^2, B^3 (cell-centred B is derived: it is recomputed
 *     from the face field). Face field = 3 such fields: Bbar^d = sqrt(-g) B^d
 *     on the lower d-face of the cell with the same index.
 */
#ifndef HAMR_H
#define HAMR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define HAMR_OK 0
#define HAMR_EINVAL (-1)   /* invalid argument or descriptor */
#define HAMR_ECUDA (-2)    /* a CUDA runtime call failed */
#define HAMR_ENOMEM (-3)   /* device allocation failed */
#define HAMR_ETIMEOUT (-4) /* a bounded device wait gave up */
#define HAMR_ESTATE (-5)   /* call made in the wrong state (e.g. no initial state set) */

/* ---- option enums ---- */
#define HAMR_METRIC_KS 0        /* Kerr metric, Kerr-Schild, log-r spherical (Sec. 2.2) */
#define HAMR_METRIC_MINKOWSKI 1 /* flat space, Cartesian (validation problems) */
#define HAMR_METRIC_SPHERICAL 2 /* flat space in the log-r spherical coordinates of HAMR_METRIC_KS (a ignored) */
#define HAMR_RECON_PPM 0        /* piecewise parabolic (Sec. 2.1) */
#define HAMR_RECON_MC 1         /* monotonised-central linear */
#define HAMR_RECON_MINMOD 2     /* minmod linear */
#define HAMR_FLUX_HLL 0         /* HLLE (Sec. 2.1) */
#define HAMR_FLUX_LLF 1         /* local Lax-Friedrichs */
#define HAMR_BC_OUTFLOW 0           /* zero-gradient copy */
#define HAMR_BC_PERIODIC 1          /* periodic */
#define HAMR_BC_POLAR 2             /* transmissive polar axis (Sec. 3.3), x2 only, n3 even */
#define HAMR_BC_OUTFLOW_NOINFLOW 3  /* zero-gradient with utilde^1 clamped to outflow, x1 only */
#define HAMR_BC_BLOCK 4             /* face shared with other blocks of the grid (ghosts from them) */
#define HAMR_EMF_AVERAGE 0 /* the 4-flux average of Sec. 2.5 */
#define HAMR_EMF_UPWIND 1  /* the average plus Gardiner & Stone (2005) upwind corrections (the paper's usual setting) */

/* energy inversion of con2prim (Sec. 2.6); the entropy backup follows either */
#define HAMR_INV_NEWTON 0 /* 2-D Newton-Raphson on (W, v^2) (Noble et al. 2006) */
#define HAMR_INV_AITKEN 1 /* Newman & Hamlin (2014) fixed point in the pressure, Aitken-accelerated */

/* frame in which the floors of Sec. 2.7 add mass and internal energy */
#define HAMR_FLOOR_FLUID 0 /* raise rho and u_g, keep utilde (the fluid frame) */
#define HAMR_FLOOR_DRIFT 1 /* add the material moving with the field lines' drift velocity and re-invert
                              (the paper's choice, after Ressler et al. 2017) */
#define HAMR_PREC_FP64 0  /* every step in FP64 */
#define HAMR_PREC_MIXED 1 /* FP32 reconstruction, fluxes and EMFs; FP64 metric, inversion, accumulation */
/* As HAMR_PREC_MIXED, with the connection source and every Newton iteration of
 * the inversion in FP64 (HAMR_PREC_MIXED iterates in FP32 until the step is
 * below 1e-5 W and finishes in FP64, and takes the source in FP32). */
#define HAMR_PREC_MIXED_FP64INV 2

/* One block: a box of cells uniform in the internal coordinates. In a grid
 * of several blocks (Sec. 3.2), blocks tile the domain with cell sizes that
 * differ by powers of two; a face inside the domain has bc HAMR_BC_BLOCK,
 * faces on the domain boundary keep their physical bc (a periodic face takes
 * its ghosts from the block across the period). `lat` is the block's level of
 * local adaptive time stepping (Sec. 3.4): it advances with 2^lat dt_fine. */
typedef struct {
    int n1, n2, n3;              /* interior cells, each >= 4 */
    double x1min, x2min, x3min;  /* lower corner */
    double dx1, dx2, dx3;        /* cell sizes */
    int bc[6];                   /* x1lo x1hi x2lo x2hi x3lo x3hi: HAMR_BC_* */
    int lat;                     /* LAT level, 0..7 (single-block grids: ignored) */
} hamr_block_desc;

/* A grid: physics options and its blocks. */
typedef struct {
    int metric;          /* HAMR_METRIC_* */
    double a;            /* black-hole spin, |a| < 1 */
    double gam;          /* adiabatic index (p = (gam - 1) u_g), 1 < gam <= 2 */
    double cour;         /* Courant factor C0 of dt = C0 / max_cells sum_i v_f^i / dx^i */
    int recon;           /* HAMR_RECON_* */
    int riemann;         /* HAMR_FLUX_* */
    int floors;          /* 1: apply the Sec. 2.7 floors after every inversion */
    int precision;       /* HAMR_PREC_* */
    int nblocks;         /* >= 1 */
    const hamr_block_desc* blocks; /* nblocks descriptors, copied by hamr_grid_create */
    int emf;             /* HAMR_EMF_*: edge EMFs (Sec. 2.5) */
    int flatten;         /* 1: PPM shock flattener (Sec. 2.1, Colella & Woodward 1984): where a
                            pressure jump above 0.33 of the lower side meets converging flow,
                            the interface values of the cell move toward its value; ignored
                            unless recon is HAMR_RECON_PPM. 0 or 1, else HAMR_EINVAL */
    int inversion;       /* HAMR_INV_*: energy inversion of every cell update */
    int floor_frame;     /* HAMR_FLOOR_*: where floors apply (floors = 1), the frame of the added material */
    int smr;             /* internal SMR levels n_max (Sec. 3.3.2; 0: off, at most 4): the row at
                            distance jp (cells) from a polar x2 face acts as cells 2^n wide in x3, n the
                            largest level with jp < 2^(n_max - n) (faces averaged, inner x3-faces
                            interpolated, one inversion per group, CFL over the group width). Single-
                            block grids with a polar x2 bc, n3 a multiple of 2^(n_max + 1),
                            n2 >= 2^n_max; the no-allocation step refuses it */
} hamr_grid_desc;

/* Counters of the last step (summed over its two stages and all blocks
 * stepped): energy inversions that converged, entropy-backup inversions,
 * cells where both failed (their primitives keep the stage's guess), floor
 * activations; dt of that step and the CFL dt of the resulting state. */
typedef struct {
    long long c2p_ok, c2p_entropy, c2p_fail, floor_hits;
    double dt_used, dt_next;
    long long newton_iters; /* Newton iterations of the energy inversions (every start tried) */
} hamr_step_stats;

typedef struct hamr_grid hamr_grid;

/* Validates the descriptor, allocates the block state, scratch and the
 * geometry tables on the current CUDA device, and builds the tables
 * (metric, inverse metric, sqrt(-g), lapse at cell centres and faces;
 * Christoffel symbols at centres by 4th-order finite differences of the
 * metric, Sec. 2.2). Synchronises the device once. Errors: HAMR_EINVAL for a
 * bad descriptor (sizes, bc/metric mismatch, odd n3 with a polar boundary),
 * HAMR_ENOMEM, HAMR_ECUDA. On error *out is NULL and nothing is leaked. */
int hamr_grid_create(const hamr_grid_desc* d, hamr_grid** out);

/* Frees everything the grid owns. NULL is accepted. Synchronises the device. */
int hamr_grid_destroy(hamr_grid* g);

/* Loads a block's state from `prim` (8 padded fields; slots 5..7 ignored:
 * centre B is recomputed from the faces) and `bface` (3 padded fields).
 * `on_device` = 0: host pointers (copied synchronously); 1: device pointers
 * (copied on `stream`). Ghost values are ignored; boundary conditions refill
 * them. Also computes the CFL dt of the loaded state. */
int hamr_grid_set_state(hamr_grid* g, int block, const double* prim, const double* bface, int on_device,
                        void* stream);

/* Copies a block's state (including ghosts) out, same layout. on_device = 0
 * synchronises the stream and writes host memory. */
int hamr_grid_get_state(const hamr_grid* g, int block, double* prim, double* bface, int on_device,
                        void* stream);

/* One midpoint step of one block (Sec. 2.1): boundary conditions, predictor
 * to t + dt/2 with fluxes, EMFs and sources of P^n, corrector from U^n to
 * t + dt with those of P^{n+1/2}; each stage ends with the CT update, the
 * inversion and the floors. dt > 0: that step; dt <= 0: the CFL step of the
 * current state, read on the device (no host round trip). The CFL dt of the
 * new state is reduced on the device in the same pass. stats: NULL for a
 * fully asynchronous call; otherwise the call synchronises `stream` and fills
 * *stats. */
int hamr_block_step(hamr_grid* g, int block, double dt, void* stream, hamr_step_stats* stats);

/* Advances every block of a multi-block grid by `n_fine_substeps` fine
 * substeps of the local adaptive time-stepping schedule (Sec. 3.4); it must
 * be a multiple of the period 2^Lmax (Lmax = the largest lat). At the start
 * of each period dt_fine = min over blocks of (CFL dt of the block) / 2^lat,
 * reduced on the device. A block of level L is due at substep s when
 * s mod 2^L = 0; levels run coarsest first; every kernel of a stage runs as
 * one batched launch over all due blocks of the level. Ghost zones come from
 * the neighbouring blocks (restriction, MINMOD prolongation, linear time
 * interpolation of a coarser-level neighbour, the current state of a
 * finer-level one, which has not yet advanced; Sec. 3.2, 3.4); same-level blocks
 * share face fluxes and edge EMFs (the finer side's); when a coarse step
 * ends its boundary fluxes and EMFs are replaced by the finer level's time
 * integrals and the cells next to corrected faces are inverted again
 * (refluxing). The period's launches are captured once into a CUDA graph and
 * replayed. stats: NULL or filled after synchronising `stream`.
 * Errors: HAMR_EINVAL (single-block grid, bad count), HAMR_ESTATE (a block
 * without state), HAMR_ECUDA. */
int hamr_batch_step(hamr_grid* g, int n_fine_substeps, void* stream, hamr_step_stats* stats);

/* Fills every block's ghost zones from the current states: the boundary
 * conditions of a single-block grid; for a multi-block grid the sampling of
 * the neighbouring blocks that hamr_batch_step uses (Sec. 3.2), with every
 * block taken at the same time. Asynchronous on `stream`. */
int hamr_grid_fill_ghosts(hamr_grid* g, void* stream);

/* Reads the accumulated counters of the last step; synchronises the device. */
int hamr_grid_stats(const hamr_grid* g, hamr_step_stats* stats);

/* Multi-block grids: the fine time step dt_fine (> 0) of every following
 * hamr_batch_step period (a block of LAT level L steps with 2^L dt_fine), or
 * the CFL step of each period (dt_fine <= 0, the default). Kept across
 * hamr_grid_regrid. For runs that must end at a given time (the convergence
 * tests); the caller keeps dt_fine within the CFL limit. Synchronises the
 * device. HAMR_EINVAL on a single-block grid (it takes dt per step). */
int hamr_grid_set_fine_dt(hamr_grid* g, double dt_fine);

/* Multi-block grids: how the batched step fills ghost cells and faces from
 * the neighbouring blocks (Sec. 3.2: copies, restriction and MINMOD
 * prolongation with linear interpolation in time under LAT). Where a ghost's
 * source lies depends only on the tree, so by default the grid finds it once,
 * when the grid is created or regridded, and every stage only applies it
 * (on = 1); on = 0 finds it again on every stage. Both give the same bits.
 * `was` (may be NULL) receives the previous setting. Synchronises the
 * device; the next hamr_batch_step captures its period again. HAMR_EINVAL on
 * a single-block grid, for on not 0 or 1, or for on = 1 where a ghost's
 * footprint does not fit the stored form (more than 15 source cells along
 * a direction; such grids keep on = 0). */
int hamr_grid_set_ghost_maps(hamr_grid* g, int on, int* was);

/* ---- dynamic refinement (Sec. 3.2: (de)refinement, nesting, prolongation
 * and restriction) ---- */

/* out[b] (host, nblocks doubles) = the maximum of primitive field `field`
 * (0..7) over the interior cells of block b, the input of a refinement
 * criterion (the paper's example: the maximum density of a block).
 * Synchronises `stream`. HAMR_EINVAL for a bad field or a NULL pointer. */
int hamr_grid_block_max(const hamr_grid* g, int field, double* out, void* stream);

/* Replaces the grid's block tree by `blocks` (nblocks >= 2, the same domain
 * and physics; every block's state is filled from the old tree at its current
 * time): cells copied, volume-averaged (restriction) or prolonged with
 * MINMOD-limited slopes; the face field copied, area-averaged or prolonged
 * with the divergence-free reconstruction of Balsara (2001) (next to
 * existing finer blocks, the interior fine faces corrected so that every fine
 * cell stays divergence-free). Primitives are
 * what is prolonged and restricted. The grid must be a multi-block grid
 * (nblocks >= 2 at creation) with every block loaded; the grid keeps its
 * physics options, launch shapes and learned guess. Runs on `stream` and
 * synchronises it before the old blocks are freed. The new tree must cover
 * the old domain and change the cell size of any region by at most a factor
 * of 2 (HAMR_EINVAL otherwise); on any error the old tree is kept. */
int hamr_grid_regrid(hamr_grid* g, int nblocks, const hamr_block_desc* blocks, void* stream);

/* Host-only: the octree that the paper's nesting rule gives for per-block
 * target levels. `cur` (n blocks) is an octree over a base grid of blocks
 * of extent base_ext[3] from corner dlo[3] (a level-L block has extent
 * base_ext / 2^L; every block has the same cell counts); target[b] is the
 * level block b's region should have (e.g. lmax where a criterion holds, 0
 * elsewhere). Each region moves one level toward its target (the regrid
 * prolongs and restricts by factors of 2: call again, with the regridded
 * grid's criterion, until the tree stops changing); then every block whose
 * face or edge neighbour is two or more levels finer is refined until the
 * jump is one level (repeated to a fixed point); regions whose targets fell
 * are derefined where that rule allows. `periodic[3]` marks periodic
 * directions (neighbours across them count). Output: *nout blocks written to
 * out (capacity `cap`; HAMR_EINVAL if exceeded, *nout = the count needed),
 * in base-block order with children in z-order; interior faces get
 * HAMR_BC_BLOCK, domain faces the bc of the input blocks on that side;
 * lat = (finest level - level). Levels above 10 are refused. */
int hamr_tree_adapt(const hamr_block_desc* cur, int n, const int* target, const double dlo[3],
                    const double base_ext[3], const int periodic[3], hamr_block_desc* out, int cap, int* nout);

/* As hamr_tree_adapt, on a spherical grid whose x2 domain faces are polar
 * axes (axis[0]: the lower x2 face, axis[1]: the upper; Sec. 3.3.1): a block
 * touching an axis splits 6-way, the x2 half at the axis into 2 children that
 * keep the parent's x3 cells (halved in x1 and x2), the other half into 4
 * children halved in all three directions, and 6 such children merge back
 * into their parent. Blocks may have different cell counts per base block
 * (e.g. polar rows with fewer x3 cells: external SMR); descendants keep their
 * base block's counts. The nesting rule is applied to cell widths: face and
 * edge neighbours at most a factor 2 apart in every direction (the coarser
 * one is refined until that holds). Output as hamr_tree_adapt; lat = (finest
 * level - level), the level being that of x1 and x2. */
int hamr_tree_adapt_polar(const hamr_block_desc* cur, int n, const int* target, const double dlo[3],
                          const double base_ext[3], const int periodic[3], const int axis[2], hamr_block_desc* out,
                          int cap, int* nout);

/* ---- measurement ---- */
/* Per-kernel device time of the grid's launches. */
typedef struct {
    char name[32];       /* kernel group: "bc", "recon", "flux", "emf", "ct", "update", "dt", ... */
    long long launches;  /* kernels launched in this group since the last reset */
    double ms;           /* summed device time (0 unless timing was enabled) */
} hamr_kernel_time;

/* enable != 0: every kernel group the grid launches is bracketed by CUDA
 * events on the stream it runs on, so hamr_grid_timing can report device
 * time per group (the events add no synchronisation). Launch counts are
 * always kept. Resets the totals. */
int hamr_grid_set_timing(hamr_grid* g, int enable);

/* Synchronises the device and writes up to `max` entries (one per kernel
 * group) to out; *n receives the number of groups. */
int hamr_grid_timing(hamr_grid* g, hamr_kernel_time* out, int max, int* n);

/* Measures the device's FP64 fused multiply-add rate (GFLOP/s, 2 flops per
 * FMA) with a dependency-free FMA loop on every SM; synchronises `stream`.
 * No counterpart in the paper: it is the denominator of the FP64-pipe
 * roofline that bounds the FP64 update on this hardware. */
int hamr_measure_fp64_peak(void* stream, double* gflops);

/* Self-check of the binary32 <-> binary64 conversions the mixed-precision
 * kernels do on the integer pipe instead of the FP64 pipe (IEEE 754 formats;
 * narrowing rounds to nearest, ties to even): widening of every binary32
 * value, and narrowing of every binary32 value's binary64 image, its binary64
 * neighbours, the midpoint to the next binary32 value and that midpoint's
 * neighbours, plus `nrandom` pseudo-random binary64 bit patterns (splitmix64
 * from `seed`), each compared bit for bit with the hardware conversion (a
 * NaN only as a NaN: payloads are the implementation's). No
 * counterpart in the paper. out4 (host): {widening mismatches, the first
 * mismatching binary32 pattern or -1, narrowing mismatches, the first
 * mismatching binary64 pattern or -1}. Synchronises the device; about 0.1 s. */
int hamr_check_conversions(long long nrandom, unsigned long long seed, long long out4[4]);

/* ---- stepping without allocation ---- */
/* Largest block hamr_block_step_noalloc accepts: padded cells
 * (n1+6)(n2+6)(n3+6) and padded (i, j) points (n1+6)(n2+6). */
#define HAMR_NOALLOC_MAX_CELLS 12288
#define HAMR_NOALLOC_MAX_PLANE 1536

/* One midpoint step of one block, like hamr_grid_set_state followed by
 * hamr_block_step, for callers that cannot allocate device memory (a host
 * framework that owns the device's memory pool, or code that must not call
 * cudaMalloc once it runs). No paper counterpart: it is the same step with
 * its scratch (geometry tables, midpoint state, edge values, fluxes, EMFs,
 * U^n cache, counters) in one file-scope device array of about 7 MB, sized
 * for blocks up to HAMR_NOALLOC_MAX_CELLS padded cells, which every GPU
 * that loads the library holds until the process exits. It calls no
 * cudaMalloc or cudaFree.
 *   d: grid descriptor with nblocks == 1 (the block stepped); FP64 only.
 *   prim, bface: device pointers, padded SoA layout; in: the state (centre B
 *     slots recomputed from the faces, ghosts refilled), out: the state
 *     after the step, valid once `stream` has completed.
 *   dt: > 0 that step; <= 0 the CFL step of the input state.
 * Blocks above the limits return HAMR_EINVAL with a message. The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make it before any stream capture. Every call
 * shares the array: calls whose GPU work overlaps (other streams, other
 * threads) race and must be serialised by the caller. */
int hamr_block_step_noalloc(const hamr_grid_desc* d, double* prim, double* bface, double dt, void* stream);

/* ---- standalone inversion (Sec. 2.6) ---- */
#define HAMR_C2P_ENTROPY_ONLY 1u /* skip the energy inversion (tests of the backup) */
#define HAMR_C2P_MLP 2u          /* start Newton from the learned guess of `mlp` (fallback: the prim guess) */
#define HAMR_C2P_MLP_RESCUE 4u   /* start from the prim guess; where that fails, from the learned guess */
#define HAMR_C2P_AITKEN 8u       /* energy inversion by the Aitken-accelerated pressure iteration, not Newton */
#define HAMR_C2P_MIXED 16u       /* Newton in FP32 first, then one FP64 refinement step (the mixed-precision update's) */

typedef struct hamr_mlp hamr_mlp;

typedef struct {
    int metric;           /* HAMR_METRIC_* */
    double a;             /* spin (KS) */
    double gam;           /* adiabatic index */
    uint32_t flags;       /* HAMR_C2P_* */
    const hamr_mlp* mlp;  /* the network of HAMR_C2P_MLP (else ignored; may be NULL) */
} hamr_c2p_desc;

/* Inverts n conserved states on the device. All arrays are device pointers
 * in SoA layout: U[6][n] = sqrt(-g) (rho u^t, T^t_t + rho u^t, T^t_1,
 * T^t_2, T^t_3, kappa rho u^t); B[3][n] centre B^i; x1[n], x2[n] positions;
 * prim[8][n] in: the guess, out: the result (slots 5..7 set to B);
 * status[n]: 0 energy inversion, 1 entropy backup, 2 both failed (prim keeps
 * the guess); iters[n]: Newton iterations of the energy inversion (pressure
 * map evaluations with HAMR_C2P_AITKEN; may be NULL). Asynchronous on
 * `stream`. */
int hamr_con2prim(const hamr_c2p_desc* d, int64_t n, const double* U, const double* B, const double* x1,
                  const double* x2, double* prim, int32_t* status, int32_t* iters, void* stream);

/* Primitive to conserved (Sec. 2.3-2.4) for n states on the device, SoA:
 * prim[8][n] (centre B in slots 5..7), x1[n], x2[n] positions, out U[6][n]
 * = sqrt(-g) (rho u^t, T^t_t + rho u^t, T^t_i, kappa rho u^t) as taken by
 * hamr_con2prim. Generates training pairs for the learned guess.
 * Asynchronous on `stream`. */
int hamr_prim2cons(const hamr_c2p_desc* d, int64_t n, const double* prim, const double* x1, const double* x2,
                   double* U, void* stream);

/* ---- learned starting point of the inversion ----
 * The paper has no counterpart: its inversion starts Newton from the
 * previous primitives (Sec. 2.6). Here a 10 -> 64 -> 64 -> 64 -> 2 tanh
 * network maps ten inputs of a conserved state to a guess of (W, v^2);
 * Newton always refines it and the start from the previous primitives is
 * the fallback, so the network changes iteration counts, never the
 * accepted solution's tolerance. Inputs (float, SoA feat[10][n]):
 *   f0 ln D; f1 ln((-Q.n - D)/D); f2 ln(Qt^2/D^2 + 1e-30);
 *   f3 (Q.B)^2/(Qt^2 B^2) (0 if either is 0); f4 ln(U_kappa/U_rho) + (gam-1) f0;
 *   f5 ln(B^2/D + 1e-30); f6 alpha; f7 ln(beta_i beta^i + 1e-30),
 *   beta^i = alpha^2 g^{ti}; f8 ln(sqrt(-g)/alpha); f9 x1,
 * with D, Q, Qt^2, B^2, Q.B the normal-frame scalars of the inversion.
 * Targets (targ[2][n]): ln(W/D) = ln(h Gamma) and ln Gamma^2.
 * Parameters: one float vector of 9154 values, W1 (64 x 10, row = output
 * unit), b1, W2 (64 x 64), b2, W3, b3, W4 (2 x 64), b4; standardisation:
 * 24 floats fmean[10], fstd[10], ymean[2], ystd[2] (inputs and targets are
 * standardised inside the network). Training runs on the device in FP32
 * (mean squared error of the standardised outputs, Adam); inference uses
 * bfloat16 weights and activations with FP32 accumulation on the tensor
 * cores (tcgen05), biases and tanh in FP32.
 * A model lives on the device that was current at hamr_mlp_create. */

/* Glorot-uniform weights from `seed`, zero biases, identity standardisation. */
int hamr_mlp_create(hamr_mlp** out, uint64_t seed);
int hamr_mlp_destroy(hamr_mlp* m);
/* host arrays params[9154], norm[24]; either may be NULL (not copied) */
int hamr_mlp_get_params(const hamr_mlp* m, float* params, float* norm);
int hamr_mlp_set_params(hamr_mlp* m, const float* params, const float* norm);
/* device arrays: inputs of n conserved states (U, B, x1, x2 as hamr_con2prim)
 * into feat[10][n]; with prim[8][n] (else NULL) also the targets into targ[2][n]. */
int hamr_mlp_features(const hamr_c2p_desc* d, int64_t n, const double* U, const double* B, const double* x1,
                      const double* x2, const double* prim, float* feat, float* targ, void* stream);
/* sets the standardisation to the mean and standard deviation of n samples
 * (device feat[10][n], targ[2][n]); synchronises */
int hamr_mlp_fit_norm(hamr_mlp* m, int64_t n, const float* feat, const float* targ, void* stream);

typedef struct {
    int64_t steps;   /* optimiser steps */
    int32_t batch;   /* samples per step, a multiple of 128 */
    float lr;        /* Adam step size at the start ... */
    float lr_final;  /* ... decayed to this by a cosine schedule */
    uint64_t seed;   /* batch sampling (uniform with replacement) */
} hamr_mlp_train_args;

/* Trains on n samples (device feat[10][n], targ[2][n]); loss (host, may be
 * NULL) receives the mean training loss of every step. Synchronises. */
int hamr_mlp_train(hamr_mlp* m, int64_t n, const float* feat, const float* targ, const hamr_mlp_train_args* a,
                   float* loss, void* stream);
/* Loss over all n samples and its gradient (host grad[9154], loss[1]) by the
 * training kernels, without a step. Synchronises. */
int hamr_mlp_loss_grad(hamr_mlp* m, int64_t n, const float* feat, const float* targ, float* grad, float* loss,
                       void* stream);
/* Outputs out[2][n] (target units) of n samples: tensor_cores = 1 the bf16
 * inference path, 0 the FP32 training path. Asynchronous. */
int hamr_mlp_forward(const hamr_mlp* m, int64_t n, const float* feat, float* out, int tensor_cores, void* stream);
/* 1 if a CTA of an inference gave up waiting on the tensor cores or the
 * copy of the weights since the last call (its cells used the plain start),
 * else 0; clears the flag. Synchronises. */
int hamr_mlp_error_flag(hamr_mlp* m, int* flag);
/* Attaches a network to a grid (NULL detaches); the model must outlive its
 * use by the grid. mode HAMR_MLP_FIRST: every inversion starts Newton from
 * the learned guess, the start from the previous primitives is the
 * fallback. HAMR_MLP_RESCUE: Newton starts from the previous primitives;
 * where that fails the learned guess is tried before the entropy backup
 * (a CTA runs the network only if one of its cells failed). Synchronises. */
#define HAMR_MLP_FIRST 0
#define HAMR_MLP_RESCUE 1
int hamr_grid_set_mlp(hamr_grid* g, const hamr_mlp* m, int mode);

/* ---- launch-shape autotuner (no paper counterpart) ----
 * Times the grid's reconstruction, face-flux and cell-update kernels on its
 * current state for each candidate launch shape and keeps the fastest:
 * cells per thread of the reconstruction sweeps (8, 16, 32; FP64), the form
 * of the x1 edge values (pencil sweeps or warp rows; FP64), then threads per
 * CTA of the reconstruction and flux kernels (64, 128, 256)
 * and of the cell update (64, 128; 128 while a network is attached). Shapes
 * change no result bit. The timed launches write only scratch (edge values,
 * fluxes, the midpoint state); call it after a first step or period so the
 * state and dt are representative. After the search the three groups
 * together are timed with the shapes found and with the default shapes on
 * the same state, five alternating repetitions each; the found shapes are
 * kept only if their median is below the defaults' by more than the larger
 * spread of the repetitions, else the defaults are kept (kept_tuned = 0).
 * Synchronises; a multi-block grid captures its period graph again on the
 * next hamr_batch_step. */
typedef struct {
    int recon_seg, bs_recon, bs_flux, bs_update; /* the shapes set on the grid */
    float ms_seg[3];    /* reconstruction, sweeps of 8, 16, 32 cells (128 threads per CTA) */
    float ms_recon[3];  /* reconstruction, 64, 128, 256 threads per CTA (chosen sweep) */
    float ms_flux[3];   /* face fluxes, 64, 128, 256 threads per CTA */
    float ms_update[2]; /* cell update (predictor), 64, 128 threads per CTA */
    int recon_x1_sweep;  /* chosen x1 form: 1 pencil sweeps (the default), 0 warp rows */
    float ms_x1[2];      /* reconstruction with x1 by warp rows, by sweeps (chosen sweep length) */
    float ms_default;    /* the three groups with the default shapes: median of 5 */
    float ms_tuned;      /* the same with the shapes the search found: median of 5 */
    float ms_spread;     /* the larger (max - min) of the two sets of repetitions */
    int kept_tuned;      /* 1 the found shapes are set, 0 the defaults are */
} hamr_tune_report;

int hamr_grid_autotune(hamr_grid* g, void* stream, hamr_tune_report* report);
/* The grid's current launch shapes (defaults 16, 128, 128, 128) into report
 * (timings zero). */
int hamr_grid_launch_shapes(const hamr_grid* g, hamr_tune_report* report);
/* Sets the launch shapes of report (recon_seg 8/16/32, recon_x1_sweep 0/1,
 * bs_recon and bs_flux 64/128/256, bs_update 64/128; timings ignored), e.g.
 * those a previous hamr_grid_autotune chose. HAMR_EINVAL for other values.
 * Synchronises; results do not change. */
int hamr_grid_set_launch_shapes(hamr_grid* g, const hamr_tune_report* report);

/* Message of the last error in the calling thread ("" if none). */
const char* hamr_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
