/*
 * rsdft.h -- C ABI of the GB300 real-space Kohn-Sham hot path.
 *
 * The operations follow Andrade & Aspuru-Guzik, "Real-space density
 * functional theory on graphical processing units" (arXiv:1306.2953):
 * blocks of orbitals stored point-major with the state index fastest
 * (Sec. IV, Fig. 4b), the Kohn-Sham Hamiltonian applied in operator form
 * (Sec. V, Eq. 3) as a 25-point star finite-difference kinetic term
 * (Sec. V.A), a local potential (Sec. V.B) and Kleinman-Bylander nonlocal
 * projectors (Sec. V.C, Eq. 4), and the overlap / Cholesky
 * orthogonalisation and subspace diagonalisation of Sec. VI (Eqs. 5-8).
 *
 * Conventions
 *  - Every call returns an int status: RS_OK (0) or a negative RS_E* code;
 *    rs_last_error() gives a message for the calling thread.  No C++
 *    exception crosses this boundary.
 *  - Orbital blocks are row-major [npts][ld] arrays: the value of state s at
 *    grid point p is at element p*ld + s; ld >= the number of states used.
 *    Grid points are in the library's order (bricks of 4x4x4 lattice points,
 *    the small-box blocking of Sec. V.A); rs_grid_ijk() gives each
 *    point's integer lattice coordinates.
 *  - dtype is RS_F64 (double) or RS_F32 (float).
 *  - Pointers named *_dev are device pointers on the current CUDA device and
 *    stay owned by the caller; handles own only their internal tables and
 *    workspace.  Device pointers to orbital data must be 16-byte aligned and
 *    ld*sizeof(element) a multiple of 16 bytes whenever the block size is at
 *    least 16 bytes per point.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls marked "asynchronous" only enqueue work on it; calls
 *    marked "blocking" synchronise it before returning.
 */
#ifndef RSDFT_H
#define RSDFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    RS_OK = 0,
    RS_EINVAL = -1,   /* bad argument (null pointer, size, alignment, block size) */
    RS_ENOMEM = -2,   /* host or device allocation failed */
    RS_ECUDA = -3,    /* a CUDA runtime call failed; no GPU; or the kernel image is missing */
    RS_ENOTSPD = -4,  /* overlap matrix not positive definite (Cholesky failed) */
    RS_ENOCONV = -5,  /* an iteration cap was hit */
    RS_ENAN = -6,     /* a non-finite value was detected */
    RS_ETIMEOUT = -7  /* a bounded device-side wait gave up; that call's result is incomplete */
};

enum { RS_F64 = 0, RS_F32 = 1 };
/* Preconditioners: none, the smoothing filter (Sec. III), the learned network,
 * and a few CG iterations on the shifted Poisson operator (RS_PRECOND_CG is
 * set with rs_solver_set_precond_cg, not in rs_solver_cfg). */
enum { RS_PRECOND_NONE = 0, RS_PRECOND_FILTER = 1, RS_PRECOND_LEARNED = 2, RS_PRECOND_CG = 3 };

typedef struct rs_grid rs_grid;
typedef struct rs_proj rs_proj;
typedef struct rs_ham rs_ham;
typedef struct rs_solver rs_solver;

/* Copies the calling thread's last error message into buf (NUL-terminated,
 * truncated to len).  Returns the message length. */
int rs_last_error(char *buf, size_t len);

/* Library version string, e.g. "rsdft 0.1 sm_103a". */
const char *rs_version(void);

/* ------------------------------------------------------------------ grid --
 * Point order (the `order` argument; Sec. V.A orders the grid by small
 * boxes of points for cache locality).  With map coordinates (u, v, w) along
 * axes 0, 1, 2 (w fastest):
 *   0 or 4   bricks of 4x4x4 points in brick raster order, each brick
 *            lexicographic (the default; the FP32 32-state kernel needs it)
 *   1, 2, 8  bricks of order^3 points (1: plain lexicographic)
 *   RS_ORDER_MORTON   the Morton Z-curve (bits of u, v, w interleaved)
 *   RS_ORDER_TILECOL  columns of 16 x 8 points along axes 2 and 1 in raster
 *            order, each column plane by plane along axis 0, each plane row
 *            by row (every tile-plane one contiguous run of points)
 * Every order numbers the same points; kernels other than the FP32
 * 32-state one address neighbours through the point map and run on any. */
enum { RS_ORDER_MORTON = -1, RS_ORDER_TILECOL = -2 };

/* Sec. II (Fig. 1): a uniform grid of spacing h whose shape is the union of
 * spheres of `radius` around the atoms.  Lattice points are r = h*(i,j,k);
 * a point is included iff for some atom A, (x-X)^2+(y-Y)^2+(z-Z)^2 <=
 * radius^2, evaluated in IEEE double in that order with x = h*i (exact
 * integer decisions; no contraction into FMA).  Host-only: no GPU needed.
 *   xyz      host [n_atoms][3] atom positions (Bohr)
 *   order    point order (see above)
 *   out      receives a new handle (free with rs_grid_destroy)
 * Errors: RS_EINVAL for n_atoms < 1, radius <= 0, h <= 0, non-finite input,
 * an unknown order, or a grid that would exceed 2^31-1 points or map entries. */
int rs_grid_create_spheres(const double *xyz, int n_atoms, double radius, double h, int order, rs_grid **out);

/* Full n0 x n1 x n2 box (zero boundary conditions beyond it), point (i,j,k)
 * at ((i-(n0-1)/2) h, (j-(n1-1)/2) h, (k-(n2-1)/2) h), in the given point
 * order.  Host-only. */
int rs_grid_create_box(int n0, int n1, int n2, double h, int order, rs_grid **out);

/* Number of points, lattice coordinate of map element (0,0,0), map
 * dimensions (the bounding box plus a 4-point margin on every side) and the
 * spacing.  Any output pointer may be NULL.  Host-only. */
int rs_grid_info(const rs_grid *g, int64_t *npts, int32_t origin[3], int32_t dims[3], double *h);

/* Integer lattice coordinates of every point, host [npts][3].  Host-only. */
int rs_grid_ijk(const rs_grid *g, int32_t *ijk_out);

/* Cartesian coordinates of every point, host [npts][3] (Bohr).  Host-only. */
int rs_grid_coords(const rs_grid *g, double *xyz_out);

/* The int32 point map over the bounding box, host [dims0][dims1][dims2]:
 * the library index of the point at lattice coordinate origin+(a,b,c), or
 * -1 where that lattice point is not a grid point (the compact neighbour
 * table of Sec. V.A).  Host-only. */
int rs_grid_point_map(const rs_grid *g, int32_t *map_out);

int rs_grid_destroy(rs_grid *g);

/* ------------------------------------------------------------ projectors --
 * Kleinman-Bylander projectors of Sec. V.C, Eq. (4).  For every atom A the
 * four projectors (s, p_x, p_y, p_z) are
 *   g(d) = exp(-d^2/(2 r_c^2)),  gamma_s = N g,  gamma_px = N (x-X) g, ...
 * on the grid points with d^2 <= r_cut^2 (same exact FP64 test as the grid),
 * each normalised on its own point list so that dV*sum(gamma^2) = 1, with
 * one coupling E[A][l] (l = s, p) in Hartree: V_nl = sum E |gamma><gamma|.
 * Host-only. */
typedef struct {
    int n_atoms;
    const double *xyz;   /* host [n_atoms][3] */
    const double *E;     /* host [n_atoms][2]: (E_s, E_p) in Ha */
    double r_c;          /* Gaussian width of the radial function (Bohr) */
    double r_cut;        /* projector sphere radius (Bohr) */
} rs_projector_spec;

int rs_proj_create(const rs_grid *g, const rs_projector_spec *spec, rs_proj **out);

/* Sizes of the sphere lists: n_atoms and the total number of entries. */
int rs_proj_info(const rs_proj *pr, int32_t *n_atoms, int64_t *n_entries);

/* Sphere lists: sph_off host [n_atoms+1], sph_idx host [n_entries] (library
 * point ids, ascending within an atom), gamma host [n_entries][4]
 * (s, px, py, pz).  Any output may be NULL. */
int rs_proj_tables(const rs_proj *pr, int64_t *sph_off, int32_t *sph_idx, double *gamma);

int rs_proj_destroy(rs_proj *pr);

/* ----------------------------------------------------------- Hamiltonian --
 * Builds H = -1/2 Lap + V + V_nl (Eq. 3) on the current CUDA device.
 *   V_host   host [npts] local potential (Ha) in library point order
 *   pr       projectors or NULL (no nonlocal term)
 *   order    stencil half-width m in 1..4 (4 = the paper's 25-point star);
 *            weights are the central second-derivative weights of Sec. V.A
 * Copies every table to the device (blocking).  Errors: RS_EINVAL,
 * RS_ENOMEM, RS_ECUDA (no device). */
int rs_ham_create(const rs_grid *g, const double *V_host, const rs_proj *pr, int order, rs_ham **out);

int rs_ham_destroy(rs_ham *h);

/* hpsi = H psi for a block of nb orbitals (Sec. V; Figs. 9-11), in one pass:
 * the projection integrals of Eq. (4) first, then one fused kernel that
 * applies the 25-point stencil, adds V*psi and gathers the nonlocal term
 * (race-free: every output point sums its covering atoms itself).
 *   psi_dev   device [npts][ld_psi] (first nb columns used), dtype elements
 *   hpsi_dev  device [npts][ld_hpsi]; must not overlap psi_dev
 *   nb        1, 2, 4, 8, 16, 32 or 64 (a power of two, Sec. IV)
 * Asynchronous.  Calls on one handle share its projection-coefficient
 * scratch: issue them on one stream (or order them with events).
 * Errors: RS_EINVAL (nb, ld, alignment, null), RS_ECUDA. */
int rs_ham_apply_block(rs_ham *h, const void *psi_dev, int64_t ld_psi, void *hpsi_dev, int64_t ld_hpsi,
                       int nb, int dtype, void *stream);

/* Status of the bounded shared-memory pipeline waits inside the FP32
 * 32-state H psi kernel (no counterpart in the paper; a failure-detection
 * aid): *flags = 0 when every wait completed, 1 when one gave up after its
 * iteration limit (that call's hpsi is incomplete).  Blocking: it reads a
 * device word after the work queued before it.  Errors: RS_EINVAL, RS_ECUDA. */
int rs_ham_status(rs_ham *h, int *flags);

/* Replaces the local potential of H (an SCF step, Sec. III): V_dev device
 * double [npts] in grid order; every table derived from it (FP32 copy,
 * per-point records of the fused kernels) is rewritten on the device.
 * Asynchronous: later calls on the stream use the new potential. */
int rs_ham_set_potential(rs_ham *h, const double *V_dev, void *stream);

/* Kernel selection of rs_ham_apply_block (a profiling aid for comparisons
 * such as the point-order study): RS_KERNEL_AUTO (0, the default) lets FP32
 * 32-state blocks take the persistent ring kernel where the grid allows it;
 * RS_KERNEL_GENERIC (1) sends every block to the generic fused kernel, which
 * addresses neighbours through the point map in any point order.  Host-only. */
enum { RS_KERNEL_AUTO = 0, RS_KERNEL_GENERIC = 1 };
int rs_ham_select_kernel(rs_ham *h, int which);

/* Clears the status word read by rs_ham_status (blocking). */
int rs_ham_reset_status(rs_ham *h);

/* Failure-detection test hook (no counterpart in the paper): the number of
 * bounded barrier tests (each suspends the waiting thread for at most 20 us)
 * after which a pipeline wait of the FP32 32-state H psi kernel gives up,
 * sets the status word and leaves the kernel.  tests < 0 restores the
 * default (100000, about two seconds); 0 makes every wait give up at once,
 * so a call returns promptly with an incomplete hpsi.  Host-only; takes
 * effect from the next call. */
int rs_ham_set_wait_limit(rs_ham *h, int tests);

/* Algorithmic bytes one rs_ham_apply_block call moves, used for GB/s: psi
 * read once, hpsi written once, V and the point map, one copy of the
 * projector tables and the projection coefficients.  The projection pass's
 * second read of the covered psi rows (L2-resident within a block) and of
 * its own atom-major copy of the tables are not counted. */
int64_t rs_ham_apply_bytes(const rs_ham *h, int nb, int dtype);

/* Per-launch timing of rs_ham_apply_block (a native profiling aid): while
 * enabled, every call records CUDA events on its stream around the
 * projection launch and around the fused stencil launch.
 * rs_ham_timing(h, 1) clears the record and starts; rs_ham_timing(h, 0)
 * stops.  rs_ham_timing_read synchronises on the recorded events (blocking)
 * and returns the summed milliseconds and the number of calls recorded. */
int rs_ham_timing(rs_ham *h, int enable);
int rs_ham_timing_read(rs_ham *h, double *project_ms, double *stencil_ms, int64_t *calls);

/* Bytes of the two launches of one rs_ham_apply_block call, counted as in
 * rs_ham_apply_bytes: project_bytes (sphere tables read, coefficients
 * written) and stencil_bytes (psi read, hpsi written, V, map, point-major
 * projector tables, coefficients read). */
int rs_ham_launch_bytes(const rs_ham *h, int nb, int dtype, int64_t *project_bytes, int64_t *stencil_bytes);

/* ------------------------------------------------------- linear algebra --
 * Overlap S = dV * X^T Y (Sec. VI, Eq. 5; S_jk = <x_j|y_k>), computed by
 * blocks of points and accumulated in FP64.
 *   X_dev [npts][ldx] (nx columns), Y_dev [npts][ldy] (ny columns), dtype
 *   S_dev device double [nx][lds]
 * Asynchronous. */
int rs_overlap_block(const rs_grid *g, const void *X_dev, int64_t ldx, int nx, const void *Y_dev, int64_t ldy,
                     int ny, double *S_dev, int64_t lds, int dtype, void *stream);

/* Tensor-core contractions of FP32 orbitals (5th-generation tensor cores,
 * tcgen05): every FP32 operand is split exactly into three BF16 pieces and
 * the six piece products of weight >= 2^-16 are accumulated in FP32, so the
 * results carry FP32-level accumulation error (not the exactly rounded FP64
 * of rs_overlap_block).  Workspace (device, caller-owned):
 * rs_tc_workspace_bytes(rows_a, rows_b, K) bytes, where the overlap has
 * rows_a = nx, rows_b = ny, K = npts and the rotation rows_a = npts,
 * rows_b = m, K = n.  Blocking (they read a status word). */
int64_t rs_tc_workspace_bytes(int64_t rows_a, int64_t rows_b, int64_t K);

/* S = dV X^T Y (Eq. 5) for FP32 X [npts][ldx] (nx columns) and Y (ny
 * columns); S device double [nx][lds]. */
int rs_overlap_block_tc(const rs_grid *g, const float *X_dev, int64_t ldx, int nx, const float *Y_dev, int64_t ldy,
                        int ny, double *S_dev, int64_t lds, void *work_dev, void *stream);

/* Subspace rotation Y = X C (Eqs. 6 and 8 applied by blocks of points): X
 * FP32 [npts][ldx] (n columns), C device double [n][ldc] (m columns), Y FP32
 * [npts][ldy]; Y may be X (the operands are split before the product). */
int rs_rotate_block(const float *X_dev, int64_t ldx, int n, const double *C_dev, int64_t ldc, int m, float *Y_dev,
                    int64_t ldy, int64_t npts, void *work_dev, void *stream);

/* Device workspace (bytes) that rs_orthonormalize / rs_subspace_diag need
 * for nst states. */
int64_t rs_linalg_workspace_bytes(int nst);

/* Orthonormalisation by Cholesky (Sec. VI, Eqs. 5-6): S = <Psi|Psi>,
 * S = U^T U (FP64, on the device), Psi <- Psi U^-1, i.e. Eq. (6) read as
 * phi_j = sum_k U_kj phibar_k.  Psi is updated in place.
 *   work_dev  device workspace of rs_linalg_workspace_bytes(nst) bytes
 *   Uinv_dev  optional device double [nst][nst] receiving U^-1 (or NULL)
 * Blocking (reads the factorisation status).  Errors: RS_ENOTSPD when S is
 * not positive definite (Psi left unchanged). */
int rs_orthonormalize(const rs_grid *g, void *Psi_dev, int64_t ld, int nst, int dtype, void *work_dev,
                      double *Uinv_dev, void *stream);

/* Allocation-free variant of rs_orthonormalize (no counterpart in the paper:
 * it exists for callers of this library that cannot allocate device memory
 * when they need the operation -- plugins whose host framework owns every
 * device buffer and hands out no workspace, or loops that forbid cudaMalloc
 * after start-up because an allocation can block or fail mid-run).
 * Same operation and arguments as rs_orthonormalize minus the workspace and
 * the U^-1 output; the scratch lives in one fixed __device__ array inside
 * this library, sized for nst <= 256 states (about 2 MB, held by every GPU
 * that loads the library until the process exits).
 *  - nst > 256 is rejected with RS_EINVAL.
 *  - The call allocates nothing (no cudaMalloc / cudaFree, no allocating
 *    library routine).
 *  - The first call on each device looks up the array's device address on
 *    that device (cudaGetSymbolAddress).
 *  - The call is blocking: it reads the factorisation status back to the
 *    host and synchronises `stream` before it returns, so it must not be
 *    issued on a stream that is being captured.
 *  - All calls share the one array: calls that overlap on the GPU (from
 *    different host threads or streams) race and must be serialised by the
 *    caller.  The call writes every scratch word it reads before reading it.
 * Errors: RS_EINVAL, RS_ENOTSPD (Psi left unchanged), RS_ECUDA. */
int rs_orthonormalize_noalloc(const rs_grid *g, void *Psi_dev, int64_t ld, int nst, int dtype, void *stream);

/* Dense symmetric eigensolver of the Rayleigh-Ritz step (Sec. VI, Eqs. 7-8,
 * where the paper diagonalises the small matrix on the CPU with LAPACK):
 * A_dev = V diag(w) V^T, eigenvalues ascending, A_dev device double [n][n]
 * (read only), w_dev [n], V_dev [n][n] (columns are eigenvectors).
 *   refine > 0: FP32 cyclic Jacobi, `refine` FP64 refinement steps
 *               (Ogita-Aishima) and an FP64 Jacobi polish (the default);
 *   refine = 0: FP64 cyclic Jacobi;  refine < 0: FP32 Jacobi only.
 * work_dev: rs_eigh_workspace_bytes(n) bytes.  Blocking.  Errors:
 * RS_ENOCONV when the FP64 Jacobi of refine = 0 hits its sweep cap. */
int64_t rs_eigh_workspace_bytes(int n);
int rs_eigh(const double *A_dev, int n, double *w_dev, double *V_dev, int refine, void *work_dev, void *stream);

/* Subspace diagonalisation (Sec. VI, Eqs. 7-8): HPsi = H Psi, h = <Psi|H|Psi>
 * (symmetrised, FP64), h xi = xi diag(eps) with eps ascending (FP64 on the
 * device), Psi <- Psi xi and HPsi <- HPsi xi.  Psi must be orthonormal.
 *   HPsi_dev  device [npts][ld] receiving H Psi (rotated)
 *   eps_dev   device double [nst]
 *   xi_dev    optional device double [nst][nst] receiving xi (or NULL)
 * Blocking.  Errors: RS_ENOCONV if the dense eigensolver hit its cap. */
int rs_subspace_diag(rs_ham *h, void *Psi_dev, void *HPsi_dev, int64_t ld, int nst, int dtype, int nb,
                     double *eps_dev, double *xi_dev, void *work_dev, void *stream);

/* --------------------------------------------------------------- solver --
 * Block eigensolvers swept block by block with a per-block convergence rule
 * (a block stops only when all its states are converged, Sec. VIII) and
 * orthonormalisation + subspace diagonalisation after every sweep (Sec. VI):
 *   RS_EIG_BLOCK_CG  LOBPCG (Knyazev 2001) on every block;
 *   RS_EIG_RMMDIIS   the paper's RMM-DIIS (Sec. III; Wood and Zunger 1985,
 *                    Kresse and Furthmueller 1996): every state refined on
 *                    its own by a Rayleigh-quotient trial step along K r and
 *                    rmm_steps - 1 DIIS steps that combine the iterates by
 *                    the lowest pair of the pencil (<r_i|r_j>, <x_i|x_j>) and
 *                    step by the same lambda along K of the combined
 *                    residual; H applied rmm_steps times per state and sweep.
 * Precision RS_F64 runs everything in FP64; RS_F32 runs H psi and the inner
 * iterations in FP32 and keeps Cholesky, Rayleigh-Ritz, residual norms,
 * dot products and eigenvalues in FP64. */
enum { RS_EIG_BLOCK_CG = 0, RS_EIG_RMMDIIS = 1 };
typedef struct {
    int nst;              /* states (a multiple of nb) */
    int nb;               /* block size: power of two, 1..64 */
    int dtype;            /* RS_F64 or RS_F32 */
    int precond;          /* RS_PRECOND_NONE, _FILTER or _LEARNED */
    double tol;           /* residual-norm threshold per state */
    double filter_alpha;  /* filter weight alpha (0.5) */
    /* The schedules below look at the largest residual norm r of the lowest
     * n_wanted states after each sweep (0 = all nst; the top block is
     * usually a convergence buffer whose states are not wanted). */
    int n_wanted;
    /* Learned-preconditioner fallback: once stall_sweeps sweeps in a row
     * leave r above stall_ratio times its best value so far, the solver
     * switches to the plain filter for good (0 = never; e.g. 3 and 0.9). */
    int stall_sweeps;
    double stall_ratio;
    /* RS_F32 solvers: the eigenvalues a step reports come from the closing
     * FP64 Rayleigh-Ritz (rs_solver_rayleigh_ritz_f64, timed inside the step)
     * at every sweep with r <= rr64_always, and every rr64_every sweeps once
     * r <= rr64_below (rr64_every = 0: never; e.g. 10, 3e-3, 1e-4). */
    int rr64_every;
    double rr64_below;
    double rr64_always;
    int method;           /* RS_EIG_BLOCK_CG (0) or RS_EIG_RMMDIIS */
    int rmm_steps;        /* RMM-DIIS steps per state and sweep, 1 .. 8 (0: 3) */
} rs_solver_cfg;

/* Creates a solver and allocates its device workspace (blocking).
 * Psi0_dev: device [npts][nst] start vectors (dtype); they are copied,
 * orthonormalised and subspace-diagonalised. */
int rs_solver_create(rs_ham *h, const rs_solver_cfg *cfg, const void *Psi0_dev, void *stream, rs_solver **out);

/* One sweep over all blocks (see above), then the schedules of
 * rs_solver_cfg.  eps_dev / resnorm_dev: device double [nst] (may be NULL);
 * eps_dev receives the sweep's Ritz values, or the FP64 Rayleigh-Ritz
 * eigenvalues when the schedule took that step (rs_solver_stats says which);
 * resnorm_dev the residual norms the sweep measured.  n_converged: host,
 * states with residual norm <= tol (may be NULL).  Blocking (reads the
 * residuals).  Errors: RS_ENAN (a non-finite residual), RS_ETIMEOUT (a
 * bounded wait of an H psi or tensor-core kernel gave up: the sweep's
 * result is incomplete), RS_ECUDA. */
int rs_eigensolver_step(rs_solver *s, double *eps_dev, double *resnorm_dev, int *n_converged, void *stream);

typedef struct {
    int sweeps;                   /* sweeps taken */
    int eps_f64;                  /* 1 when the last step's eigenvalues came from an FP64 Rayleigh-Ritz
                                   * (always 1 for RS_F64 solvers) */
    int precond;                  /* RS_PRECOND_* in use now */
    int fallback_sweep;           /* sweep after which the learned preconditioner gave way to the filter (0: not) */
    double max_residual;          /* largest residual norm of the wanted states in the last sweep */
    double train_target_seconds;  /* last rs_precond_train: residuals and CG targets (wall clock) */
    double train_fit_seconds;     /* last rs_precond_train: tile cutting and Adam steps (wall clock) */
    double lambda_max;            /* estimate of the largest eigenvalue of H taken by
                                   * rs_solver_certify_smoothed (0: not taken yet) */
} rs_solver_stats_t;

/* Host-side statistics of the solver (no device work). */
int rs_solver_stats(rs_solver *s, rs_solver_stats_t *out);

/* ------------------------------------------------ learned preconditioner --
 * Not in the paper (its preconditioner is the filter of Sec. III).  The
 * network maps a residual r to y = L3(relu(L2(relu(L1(r/rms(r)))))) * rms(r)
 * with bias-free 3^3 lattice cross-correlations 1 -> 8 -> 8 -> 1, every
 * layer's output zero off the grid, inputs stored in BF16, weights used in
 * BF16 (rounded from an FP32 master copy) and FP32 accumulation.  Weights:
 * one FP32 array of 2160 values, [8][1][27] | [8][8][27] | [1][8][27], tap
 * t = 9 (a+1) + 3 (b+1) + (c+1) for the lattice offset (a, b, c) along the
 * point-map axes. */

/* Workspace bytes of rs_shifted_poisson_cg. */
int64_t rs_cg_workspace_bytes(int64_t npts, int ncols, int dtype);

/* Training targets: exactly n_iter conjugate-gradient iterations from X = 0
 * on (-1/2 Lap + sigma) X = B, one independent system per column.  h must be
 * a Hamiltonian built with V = sigma everywhere and no projectors; B_dev, X_dev
 * [npts][ld] (ncols columns, a power of two <= 64).  Asynchronous. */
int rs_shifted_poisson_cg(rs_ham *h, const void *B_dev, void *X_dev, int64_t ld, int ncols, int n_iter, int dtype,
                          void *work_dev, void *stream);

/* The network on dense D^3 tiles (training-side kernels): y = network(x)
 * with x rounded to BF16 and zero outside mask; when grad_dev or loss_host is
 * given, loss = sum over valid-and-mask points of (y - target)^2 / count and
 * grad_dev = d loss / d w (FP32 [2160]).
 *   w_dev [2160] FP32 master weights; x_dev, target_dev, y_dev [ntiles][D^3]
 *   FP32; mask_dev [ntiles][D^3] and valid_dev [D^3] bytes (0/1).
 * Blocking. */
int rs_convnet_tiles(const float *w_dev, const float *x_dev, const uint8_t *mask_dev, const float *target_dev,
                     const uint8_t *valid_dev, int ntiles, int D, float *y_dev, float *grad_dev, double *loss_host,
                     void *stream);

/* W = K R on the grid for nb FP32 residual columns (R, W [npts][ld]) with
 * the network weights w_dev (FP32 master copy, rounded to BF16 here).
 * Uses device memory owned by h for activations (held until h is destroyed,
 * grown on demand).  Asynchronous.  The solver applies the same kernels. */
int rs_precond_apply(rs_ham *h, const float *w_dev, const float *R_dev, int64_t ldr, float *W_dev, int64_t ldw, int nb,
                     void *stream);

typedef struct {
    int n_tiles;     /* training tiles cut from the (residual, target) columns */
    int tile;        /* interior edge (16); tiles carry 3 more points of halo */
    int epochs;
    int batch;       /* tiles per Adam step */
    float lr;        /* Adam learning rate (1e-3) */
    uint64_t seed;   /* tile positions (splitmix64) */
} rs_train_cfg;

/* Trains the network on tiles cut around random grid points of the column
 * pairs (R, X) (FP32 [npts][ld], ncols columns: residuals and their CG
 * solutions), inputs and targets scaled by the residual's rms.  w_dev holds
 * the initial FP32 master weights and receives the trained ones; loss_host
 * (may be NULL) receives the mean loss of every epoch.  Blocking. */
int rs_precond_train_pairs(rs_ham *h, const rs_grid *g, const float *R_dev, const float *X_dev, int64_t ld, int ncols,
                           const rs_train_cfg *cfg, float *w_dev, float *loss_host, void *stream);

/* Adam on caller-provided dense tiles (the training kernels alone):
 * x_dev, target_dev FP32 [ntiles][D^3], mask_dev [ntiles][D^3] and valid_dev
 * [D^3] bytes as in rs_convnet_tiles.  `epochs` passes over the tiles in
 * order, one Adam step (beta = 0.9, 0.999; eps = 1e-8; moments zero at the
 * start) per batch of `batch` consecutive tiles, a last partial batch
 * dropped; each step's loss is the mean over the batch's valid grid points.
 * w_dev: initial FP32 weights, receives the trained ones.  Blocking. */
int rs_precond_train_tiles(float *w_dev, const float *x_dev, const uint8_t *mask_dev, const float *target_dev,
                           const uint8_t *valid_dev, int ntiles, int D, int batch, int epochs, float lr,
                           float *loss_host, void *stream);

typedef struct {
    int n_res;          /* residual columns: the Ritz residuals of the lowest n_res states (<= 256) */
    int cg_iters;       /* CG iterations of the targets (200) */
    double sigma;       /* shift of the target operator -1/2 Lap + sigma (1 Ha) */
    rs_train_cfg train; /* tiles and Adam */
} rs_learn_cfg;

/* The learned mode of an RS_F32 solver created with RS_PRECOND_LEARNED, in
 * one call: the Ritz residuals of its lowest n_res states, their targets
 * (cg_iters CG iterations on (-1/2 Lap + sigma) X = R from X = 0, on a
 * Hamiltonian of grid g with V = sigma and no projectors), each target
 * column scaled to unit rms, training on tiles of the pairs
 * (rs_precond_train_pairs), and the trained weights set as the solver's.
 * w_init_dev: FP32 [2160] starting weights (not modified), or NULL to
 * continue from the solver's current weights (for training again on the
 * residuals of a later sweep).  loss_host: train.epochs floats or NULL.
 * Blocking.  Errors: RS_EINVAL (solver not learned / not FP32, sizes, no
 * weights to start from), RS_ENOMEM. */
int rs_precond_train(rs_solver *s, const rs_grid *g, const rs_learn_cfg *cfg, const float *w_init_dev,
                     float *loss_host, void *stream);

/* The solver's learned weights to / from a file: the 4 bytes "RSNN", then
 * little-endian uint32 version (1), uint32 count (2160), the FP32 weights,
 * and the uint32 FNV-1a hash of the weight bytes.  Load needs a solver whose
 * preconditioner is the learned one and rejects files that do not match
 * (RS_EINVAL) or hold non-finite weights (RS_ENAN).  Blocking. */
int rs_precond_save(rs_solver *s, const char *path);
int rs_precond_load(rs_solver *s, const char *path);

/* FP64 Rayleigh-Ritz of the solver's current subspace (Sec. VI, Eq. 7): the
 * FP32 orbitals of an RS_F32 solver are widened to FP64, H is applied in
 * FP64, and h x = eps S x is solved with h and S accumulated in FP64, giving
 * eigenvalues free of the FP32 rounding of H (its potential and stencil
 * weights) -- the closing step of the mixed-precision eigensolve.  The
 * iteration state is not modified.  For RS_F64 solvers it returns the
 * current eigenvalues.  eps_dev: device double [nst].  Blocking; the first
 * call allocates two FP64 copies of the orbitals. */
int rs_solver_rayleigh_ritz_f64(rs_solver *s, double *eps_dev, void *stream);

/* Certificate of the solver's current subspace (no counterpart in the paper;
 * for workloads without a reference solution): the FP64 Rayleigh-Ritz of
 * rs_solver_rayleigh_ritz_f64 (orbitals widened to FP64, H applied in FP64,
 * h x = eps S x solved in FP64), then the Ritz vectors x_k = Psi C_k and
 * their FP64 residual norms r_k = ||H x_k - eps_k x_k|| with <x_k|x_k> = 1.
 * For a symmetric H an eigenvalue lies within r_k of eps_k, and within
 * r_k^2 / gap_k when gap_k separates eps_k from the rest of the spectrum.
 * eps_dev, res_dev: device double [nst].  The iteration state is not
 * modified.  Blocking; the first call allocates two FP64 copies of the
 * orbitals.  The residual norms measure the returned pairs whatever the
 * dense eigensolver's iteration did.  Errors: RS_ENOTSPD. */
int rs_solver_certify(rs_solver *s, double *eps_dev, double *res_dev, void *stream);

/* Smoothed certificate (no counterpart in the paper): rs_solver_certify
 * after n_smooth damped Richardson steps on the FP64 copy of the orbitals,
 *     psi_k <- psi_k - (H psi_k - eps_k psi_k) / (lambda_max - eps_k),
 * eps_k the solver's current eigenvalues, H applied in FP64.  A step leaves
 * an eigenvector of H unchanged and multiplies the component of psi_k along
 * an eigenvector of eigenvalue mu by 1 - (mu - eps_k) / (lambda_max - eps_k):
 * zero at the top of the spectrum, one half midway.  It damps the
 * high-energy rounding noise that FP32 storage leaves in the orbitals, which
 * inflates the residual norms (by the noise times up to lambda_max) far more
 * than it moves the eigenvalues; what the steps do to components inside the
 * subspace (the lower states are amplified by at most
 * 1 + (eps_k - eps_0) / (lambda_max - eps_k)) the Rayleigh-Ritz undoes.  The
 * Ritz pairs returned are exact Rayleigh-Ritz pairs of the smoothed subspace,
 * so their residual norms certify them as in rs_solver_certify.
 * lambda_max > 0 is used as given and must exceed every current eigenvalue
 * (RS_EINVAL otherwise); lambda_max <= 0 takes an estimate of the largest
 * eigenvalue of H: 120 power iterations on H - eps_0 in FP64 from a fixed
 * start vector, the Rayleigh quotient of the last iterate (a lower bound of
 * it; taken once per solver, reported by rs_solver_stats).  n_smooth in
 * 0 .. 16; 0 is rs_solver_certify.  The iteration state is not modified.
 * Blocking.  Errors: RS_EINVAL, RS_ENOTSPD, RS_ENAN (the estimate failed). */
int rs_solver_certify_smoothed(rs_solver *s, int n_smooth, double lambda_max, double *eps_dev, double *res_dev,
                               void *stream);

/* Ritz residuals R = H psi_k - eps_k psi_k of states first..first+ncols-1
 * of the current orbitals (after the last sweep's subspace diagonalisation),
 * into R_dev [npts][ldr] (the solver's dtype): the residuals the method
 * generates, used as training inputs of the learned preconditioner.
 * 1 <= ncols <= 256.  Asynchronous.  Errors: RS_EINVAL (range, ldr). */
int rs_solver_residual(rs_solver *s, int first, int ncols, void *R_dev, int64_t ldr, void *stream);

/* The solver's current orbitals: device [npts][nst] (dtype), owned by the
 * solver; valid until rs_solver_destroy. */
int rs_solver_psi(rs_solver *s, void **psi_dev);

/* Weights of the learned preconditioner (RS_PRECOND_LEARNED, FP32 F32-mode
 * solvers only): w_dev is the 2160-value FP32 array described above (copied).
 * Until weights are set the learned preconditioner refuses to run.
 * Errors: RS_EINVAL when the solver's preconditioner is not the learned one. */
int rs_solver_set_precond_weights(rs_solver *s, const float *w_dev);

/* Replaces the solver's preconditioner (RS_PRECOND_NONE / FILTER / LEARNED;
 * a learned one takes the weights last set or trained, if any) for the sweeps
 * that follow, e.g. the plain filter as the fallback once the learned one
 * stops reducing the residuals.  Blocking (waits for queued sweeps).
 * Errors: RS_EINVAL. */
int rs_solver_set_precond(rs_solver *s, int precond);

/* Replaces the solver's preconditioner, for later sweeps, by n_iter
 * conjugate-gradient iterations from W = 0 on (-1/2 Lap + sigma) W = R, one
 * system per residual column: the operator the learned network is trained
 * to imitate, applied directly.  Not in the paper.  shifted is a Hamiltonian
 * on the solver's grid built with V = sigma everywhere and no projectors;
 * it stays owned by the caller and must outlive the solver or the next
 * preconditioner change.  n_iter in 1 .. 200.  Blocking.  Errors: RS_EINVAL
 * (null argument, n_iter out of range, a grid of another size), RS_ENOMEM. */
int rs_solver_set_precond_cg(rs_solver *s, rs_ham *shifted, int n_iter);

/* Checkpoint and restart (no counterpart in the paper): the iteration state
 * of a solver -- orbitals, H applied to them, block CG's search directions,
 * eigenvalues, residual norms and the sweep count -- to a file, and back
 * into a solver created with the same grid size and configuration, which
 * then continues exactly where the saved one stood.  File: "RSCK", uint32
 * version 1, int64 npts, int32 nst, nb, dtype, method, sweeps, uint32
 * search-direction flag, the raw arrays, and an FNV-1a hash.  Blocking.
 * Errors: RS_EINVAL (cannot open, another shape, damaged file), RS_ECUDA. */
int rs_solver_checkpoint_save(rs_solver *s, const char *path);
int rs_solver_checkpoint_load(rs_solver *s, const char *path);

/* New local potential for the solver's Hamiltonian (an SCF step): the
 * Hamiltonian's potential is replaced (rs_ham_set_potential), the current
 * subspace is rediagonalised with it and the search directions are dropped.
 * V_dev device double [npts].  Blocking. */
int rs_solver_set_potential(rs_solver *s, const double *V_dev, void *stream);

int rs_solver_destroy(rs_solver *s);

/* -------------------------------------------------------------- Hartree --
 * The Hartree potential by FFT (Sec. X; Eq. 2, lap V_H = -4 pi n): the
 * density is copied from the grid to a cube, Fourier transformed, multiplied
 * by the Coulomb-interaction kernel, transformed back and copied to the grid.
 * Free boundary conditions from an enlarged cube and the spherical-cutoff
 * kernel of Rozzi et al. (2006): v(G) = 4 pi (1 - cos(|G| R_c)) / |G|^2,
 * v(0) = 2 pi R_c^2, with R_c = D + h (D: the diagonal of the grid's
 * bounding box) and N_a cube points along axis a, the smallest 2^p 3^q
 * >= extent_a + ceil(R_c / h) + 1 (the radices of the paper's GPU FFT), so
 * that the periodic convolution equals the free-space one on the grid.
 * The transforms are the library's own complex FP64 Stockham kernels. */
typedef struct rs_poisson rs_poisson;

/* Plans the cube for grid g and allocates it on the current device, with
 * the table of v(G) (24 bytes per cube element in all; blocking).  Errors:
 * RS_EINVAL (empty grid, an axis above 768 points), RS_ENOMEM. */
int rs_poisson_create(const rs_grid *g, rs_poisson **out);

/* Cube shape, the cutoff radius R_c (Bohr) and the cube's bytes. */
int rs_poisson_info(const rs_poisson *p, int32_t shape[3], double *r_cut, int64_t *cube_bytes);

/* vh_dev = V_H for the density n_dev (device double [npts] in grid order,
 * electrons per Bohr^3); vh_dev in Hartree.  Calls on one handle share its
 * cube: issue them on one stream.  Asynchronous. */
int rs_poisson_solve(rs_poisson *p, const double *n_dev, double *vh_dev, void *stream);

int rs_poisson_destroy(rs_poisson *p);

/* ------------------------------------------------------------------ SCF --
 * The self-consistent field loop of Sec. III (Fig. 2) around a solver: each
 * step forms the Kohn-Sham potential of the input density n_in (Eq. 3:
 * v_ext + v_H + v_xc, v_H by rs_poisson_solve, v_xc the local density
 * approximation: Slater exchange and the Perdew-Zunger 1981 fit of the
 * Ceperley-Alder correlation, unpolarised), sets it (rs_solver_set_potential),
 * runs `sweeps` eigensolver sweeps, occupies the states with Fermi-Dirac
 * occupations f_k = 2 / (1 + exp((eps_k - mu) / sigma)), sum f_k = n_electrons,
 * forms n_out = sum f_k |phi_k|^2 (Eq. 1b over both spins) and mixes by
 * Broyden's second update with uniform weights (Broyden 1965, Srivastava
 * 1984) in its Anderson form: with F = n_out - n_in and the history dn_i,
 * dF_i of the last `history` steps, n_in <- n_in + alpha F
 * - sum theta_i (dn_i + alpha dF_i), theta minimising |F - sum theta_i dF_i|. */
typedef struct {
    double n_electrons;  /* electrons (at most 2 per state of the solver) */
    double sigma;        /* Fermi smearing width (Ha), > 0 */
    double alpha;        /* mixing parameter, > 0 */
    int history;         /* Broyden history length, 0 .. 16 (0: linear mixing) */
    int sweeps;          /* eigensolver sweeps per SCF step, >= 1 */
} rs_scf_cfg;
typedef struct rs_scf rs_scf;

/* v_ext_host: host double [npts] (the external potential, e.g. the local
 * pseudopotential the solver's Hamiltonian was built with); n0_host: host
 * double [npts] starting density.  The solver's Hamiltonian potential is
 * replaced at every step.  Blocking.  Errors: RS_EINVAL, RS_ENOMEM. */
int rs_scf_create(rs_solver *s, const rs_grid *g, const double *v_ext_host, const double *n0_host,
                  const rs_scf_cfg *cfg, rs_scf **out);

/* One SCF step; residual = ||n_out - n_in|| (grid norm, before mixing) and
 * n_out = sum_k f_k |phi_k|^2 / <phi_k|phi_k>, each orbital's norm summed in
 * FP64 so that the density carries exactly n_electrons; and
 * energy = the Mermin free energy sum f eps - E_H - int n v_xc + E_xc
 * - sigma S of the step's input density (ion-ion repulsion omitted), both
 * may be NULL.  With an RS_F32 solver the eigenvalues eps that set the
 * occupations and the band energy are those of rs_solver_rayleigh_ritz_f64
 * (FP64 H), taken every step.  Blocking.  Errors: RS_ENAN, and the
 * solver's. */
int rs_scf_step(rs_scf *scf, double *residual, double *energy, void *stream);

/* Current input density (device double [npts], may be NULL), the last
 * occupations (host double [nst], may be NULL), mu and the step count. */
int rs_scf_state(rs_scf *scf, double *n_in_dev, double *occupations_host, double *mu, int *iterations);

int rs_scf_destroy(rs_scf *scf);

#ifdef __cplusplus
}
#endif
#endif /* RSDFT_H */
