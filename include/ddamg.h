/*
 * ddamg.h -- C ABI of the GB300 DD-alpha-AMG solver for the lattice
 * Wilson-clover Dirac system D z = b (Frommer, Kahl, Krieg, Leder, Rottmann,
 * "An adaptive aggregation based domain decomposition multilevel method for
 * the lattice Wilson Dirac operator: multilevel results").
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * Lattice: dims = {T, Z, Y, X}; direction mu = 0..3 is t, z, y, x.  A site's
 *   lexicographic index is ((t*Z + z)*Y + y)*X + x.
 * Gauge field (input to ddamg_setup): FP64 complex, [site lex][mu][3][3][re,im],
 *   i.e. 4*9 complex per site.  The time-direction boundary sign (bc_t = -1 for
 *   antiperiodic) is applied by the library; it is not part of the links.
 * Fine fields (level 0): FP64 complex, [n][site lex][spin][colour][re,im]:
 *   12 complex per site, index spin*3 + colour, chiral basis with
 *   Gamma_5 = diag(+1, +1, -1, -1) in spin (Sec. 1 of the paper).
 * Coarse fields (level l >= 1): FP64 complex, [n][coarse site lex][dof][re,im];
 *   level l carries ndof = 2 * n_tv[l-1] dof per site, chirality + first.
 * Pointers may be host or device memory (cudaPointerGetAttributes decides);
 *   the caller owns them.  Host pointers are copied through library-owned
 *   device staging buffers.  Every call returns after its results are
 *   complete (the library stream is synchronised before returning).
 * The library owns every device allocation it makes; ddamg_free releases them.
 * Return values: DDAMG_OK (0) or a negative DDAMG_ERR_* code;
 *   ddamg_last_error() returns a message for the last failure of the thread.
 * Thread safety: one handle must not be used by two threads at once.
 */
#ifndef DDAMG_H
#define DDAMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  DDAMG_OK = 0,
  DDAMG_ERR_ARG = -1,       /* invalid argument or unsupported geometry        */
  DDAMG_ERR_OOM = -2,       /* device allocation failed / admission refused    */
  DDAMG_ERR_NOCONV = -3,    /* outer FGMRES did not reach tol within its limit */
  DDAMG_ERR_CUDA = -4,      /* a CUDA call failed                              */
  DDAMG_ERR_SINGULAR = -5,  /* rank-deficient test vectors / singular block    */
  DDAMG_ERR_ADMISSION = -6  /* serving: device footprint exceeds the budget    */
};

#define DDAMG_MAX_LEVELS 4

/* Parameters of the method (Table 1 of the paper gives the defaults that
 * ddamg_default_params fills in). */
typedef struct ddamg_params {
  int levels;                          /* L >= 2                                         */
  int agg[DDAMG_MAX_LEVELS][4];        /* aggregate of level l (defines P_l), t,z,y,x    */
  int n_tv[DDAMG_MAX_LEVELS];          /* test vectors N_l of level l (P_l has 2N_l cols) */
  int sap_block[DDAMG_MAX_LEVELS][4];  /* SAP block of level l (l < L-1)                 */
  int mr_steps;                        /* MR steps per SAP block solve (Table 1: 3)      */
  int nu;                              /* post-smoothing steps (Table 1: 5)              */
  int mu;                              /* pre-smoothing steps (Table 1: 0)               */
  int n_inv;                           /* iterative setup iterations (Table 1: 6)        */
  int eta_passes;                      /* passes of Alg. 3's smoothing loop (3)          */
  int outer_restart;                   /* n_kv (Table 1: 10), at most 63                 */
  int outer_max_cycles;                /* restart cycles before DDAMG_ERR_NOCONV          */
  int kcycle_len;                      /* K-cycle FGMRES length (Table 1: 5)             */
  int kcycle_cycles;                   /* K-cycle FGMRES cycles (Table 1: 2 restarts)    */
  double kcycle_tol;                   /* K-cycle relative tolerance (Table 1: 0.1)      */
  double coarse_tol;                   /* coarsest relative tolerance (Table 1: 5e-2)    */
  int coarse_restart;                  /* coarsest GMRES restart length (<= 63)          */
  int coarse_cycles;                   /* coarsest GMRES cycles                          */
  int precision;                       /* preconditioner: 0 FP64; 1 FP32; 2 FP32 arithmetic
                                          on FP16 storage (links, clover term, P, coarse
                                          blocks; per-site / per-aggregate scales)        */
  int max_rhs;                         /* right-hand sides per batch                     */
  uint64_t seed;                       /* seed of the random start vectors of Alg. 3 when
                                          ddamg_setup draws them (tv_random = NULL)       */
  int sap_schur;                       /* 1: the FP32 preconditioner's fine-level SAP solves
                                          each block on its even-odd Schur complement (MR on
                                          Dhat_B = D_ee - D_eo D_oo^-1 D_oe, then the odd
                                          back-substitution; needs 4^4 SAP blocks); 0: MR on
                                          D_B (the paper does not say which)              */
  int setup_batch;                     /* test vectors per batched K-cycle of Alg. 4 (0: 4);
                                          the level workspaces hold max(max_rhs, this)
                                          columns; results do not depend on it (passes
                                          that update test vectors two or more levels below
                                          the cycle's start level, L >= 4, run one vector at
                                          a time)                                          */
} ddamg_params;

typedef struct ddamg_stats {
  int iterations;        /* outer FGMRES iterations                          */
  int cycles;            /* outer restart cycles                             */
  int converged;         /* 1 if ||b - D x|| <= tol ||b|| (FP64, true residual) */
  double true_residual;  /* ||b - D x|| / ||b|| at return                    */
} ddamg_stats;

typedef struct ddamg_handle ddamg_handle;

/* Table 1 defaults: L = 3, aggregates 4^4 then 2^4, N = 20, SAP blocks 2^4,
 * 3 MR steps, nu = 5, mu = 0, n_inv = 6, n_kv = 10, K-cycle 5/2/0.1,
 * coarsest tolerance 5e-2 (restart 50, 20 cycles), mixed precision, 1 rhs. */
void ddamg_default_params(ddamg_params* p);

/* Builds the hierarchy: imports the gauge field, builds the clover term
 * (c_sw), runs the initial setup (Alg. 3) and n_inv iterative setup phases
 * (Alg. 4).  Alg. 3 starts from random test vectors:
 *   tv_random = NULL: the library draws them on the device from params.seed
 *     (complex N(0,1) entries, independent real and imaginary parts): entry
 *     (field j, lexicographic site x, dof k) of level l comes from Philox4x32-10
 *     (Salmon et al., SC 2011) on counter (x, k, j, l) with key (seed mod 2^32,
 *     seed div 2^32) and the Box-Muller transform of its two 53-bit uniforms;
 *     level 0 draws fields j = 0..n_tv[0]-1, a level l >= 1 the fields
 *     j = 0..n_tv[l]-n_tv[l-1]-1 that restriction does not provide.  Nothing is
 *     staged through host memory.
 *   otherwise tv_random[0] holds n_tv[0] fine fields (host or device) and
 *     tv_random[l] (l >= 1) holds max(0, n_tv[l] - n_tv[l-1]) level-l fields
 *     (may be NULL when that count is 0).
 * On success *out is a new handle.  Errors: ARG (geometry: extents must be
 * divisible by aggregates and SAP blocks, SAP block counts even or 1, coarsest
 * extents even), OOM, SINGULAR, CUDA. */
int ddamg_setup(const double* gauge, const int dims[4], int bc_t, double m0, double csw,
                const ddamg_params* params, const double* const* tv_random, ddamg_handle** out);

/* Solves D x_i = rhs_i, i < n, with FGMRES(n_kv) in FP64 right-preconditioned
 * by one K-cycle (Alg. 2) per iteration (the preconditioner in FP32 when
 * precision = 1 or 2).  Batches of up to max_rhs right-hand sides share every
 * kernel launch; larger n is split into consecutive batches.  per_rhs may be
 * NULL.  Returns NOCONV (x holds the last iterate) if any rhs missed tol. */
int ddamg_solve(ddamg_handle* h, const double* rhs, double* x, int n, double tol, ddamg_stats* per_rhs);

void ddamg_free(ddamg_handle* h);

/* Hierarchy update after a change of the gauge field (as between the steps of a Monte Carlo
 * chain, where setup cost weighs most: Table 3 of the paper puts it at several times a solve):
 * imports `gauge` (same layout as ddamg_setup, host or device), rebuilds the clover term and
 * every FP32/FP16 copy, rebuilds P_l from the current test vectors and every coarse operator
 * D_{l+1} = P_l^dagger D_l P_l of the new fine operator, then runs n_inv iterative setup phases
 * (Alg. 4) starting from the current test vectors.  m0, c_sw, the geometry and the parameters
 * are kept.  Errors: ARG, SINGULAR, CUDA. */
int ddamg_update_gauge(ddamg_handle* h, const double* gauge, int n_inv);

/* The plain Krylov solver the paper compares the method with (Sec. 3.3, Table 5): CGNR on the
 * fine operator of the handle, in FP64, in its least-squares form (CG on D^+ D x = D^+ b that
 * updates s = b - D x), with D^+ = Gamma_5 D Gamma_5 (gamma_5-symmetry, Sec. 1).  Same layout and
 * batching as ddamg_solve (max_rhs per batch, each column with its own coefficients); a column
 * stops when ||s|| <= tol ||b|| or after max_iter iterations, and its true residual is recomputed
 * at the end (per_rhs: iterations, converged on the true residual, true_residual).  Returns
 * NOCONV if a column missed tol (x holds its last iterate). */
int ddamg_cgnr(ddamg_handle* h, const double* rhs, double* x, int n, double tol, int max_iter, ddamg_stats* per_rhs);

/* Extreme singular values of the fine operator (the quantity the paper's masses are tuned by,
 * Sec. 3): `steps` CG iterations on D^+ D from a random field drawn from `seed` (as the setup
 * draws its vectors, field 0 of level 7), then the smallest and largest eigenvalues of the CG
 * Lanczos matrix (diagonal 1/alpha_j + beta_{j-1}/alpha_{j-1}, off-diagonal sqrt(beta_j)/alpha_j)
 * by Sturm bisection; sigma = sqrt(lambda).  The estimates approach the extreme singular values
 * from inside as steps grows.  sigma_max and steps_taken may be NULL.  Errors: ARG. */
int ddamg_sigma_extremes(ddamg_handle* h, int steps, uint64_t seed, double* sigma_min, double* sigma_max,
                         int* steps_taken);

const char* ddamg_last_error(void);

/* Runs the library's kernels on this CUDA stream from now on (cudaStream_t;
 * NULL = the library's own stream). */
int ddamg_set_stream(ddamg_handle* h, void* stream);

/* Options (ddamg_set_option). */
enum {
  DDAMG_OPT_GRAPHS = 0,  /* 1 (default): each K-cycle runs as one captured CUDA graph whose inner
                            Krylov loops are device-driven conditional WHILE nodes; 0: host-driven */
  DDAMG_OPT_COARSEST_CLUSTER = 1, /* 1 (default, where it fits): the coarsest odd-even GMRES runs as one
                                     persistent thread-block-cluster kernel per right-hand side */
  DDAMG_OPT_SAP_CLUSTER = 2,      /* 1 (default, where it fits): coarse-level SAP sweeps run one
                                     thread-block cluster per SAP block; 2, 4, 8 or 16: try that
                                     cluster size first; 0: one CTA per block */
  DDAMG_OPT_HALF_STORAGE = 3,     /* 1: the FP32 kernels read FP16 copies of the fine links and
                                     clover term (no scale), of P (one FP32 scale per aggregate
                                     and chirality) and of the coarse blocks (one FP32 scale per
                                     site): q = round-to-nearest-even(x / s), s = max |Re|, |Im|
                                     of the group.  Default: 1 iff params.precision = 2.  The
                                     paper keeps FP32 storage; this is a storage format only
                                     (arithmetic stays FP32, the copies follow every rebuild). */
  DDAMG_OPT_COARSE_TC = 4,        /* batch kernels on FP16 storage (coarse stencil, restriction,
                                     prolongation): -1 (default): autotuned per level (see
                                     ddamg_autotune_times); 0: the per-right-hand-side / CUDA-core
                                     kernels; 1..4: the tensor-core kernels with the k dimension
                                     split over that many warp groups (and the batch
                                     prolongation), where they fit */
  DDAMG_OPT_SAP_SCHUR = 5,        /* 0/1: params.sap_schur switched after setup (the per-site
                                     inverse tables are built on first use)            */
  DDAMG_OPT_SAP_PERSIST = 6,      /* coarse-level SAP on FP16 blocks (levels 1..L-2): -1 (default):
                                     autotuned per level between one cluster launch per colour
                                     sweep (0) and one persistent cooperative launch for all
                                     sweeps of a smoother call (1), where all clusters of the
                                     level fit on the device at once (one or, if one does not
                                     fit, two SAP blocks of each colour per cluster); 0/1 force
                                     the choice (1 only where it fits); 2: persistent with two
                                     blocks per cluster.  Same arithmetic in every form. */
  DDAMG_OPT_OUTER_DF = 7          /* 0 (default) / 1: the outer FGMRES forms D z_j and its CGS2
                                     Gram-Schmidt products in double-FP32 arithmetic (Dekker
                                     pairs, about 48 significand bits) on its FP64 vectors; the
                                     restart and final residuals b - D x stay FP64.  GB300's FP64
                                     rate is 1/64 of its FP32 rate, which bounds the FP64
                                     operator and Gram-Schmidt kernels.  The paper's outer solver
                                     is double precision (Sec. 3); this option trades its last
                                     bits (relative error of D about 1e-14) for speed. */
};
int ddamg_set_option(ddamg_handle* h, int option, int value);
/* Effective setting: GRAPHS 0/1; COARSEST_CLUSTER and SAP_CLUSTER the cluster size in use on the
 * coarsest level / on level 1 (FP32 path), 0 when the one-CTA kernels run; HALF_STORAGE 0/1;
 * COARSE_TC the kernel in use on level 1 (0 CUDA cores, k >= 1 tensor cores with k-split k);
 * SAP_PERSIST 1 when level 1's smoother calls run as one persistent launch; OUTER_DF 0/1. */
int ddamg_get_option(ddamg_handle* h, int option, int* value);

/* ---- measurement ----------------------------------------------------------- */

/* Kernel classes timed by ddamg_profile. */
enum {
  DDAMG_PROF_FINE_SAP = 0,      /* one SAP colour sweep on the fine level          */
  DDAMG_PROF_FINE_DSLASH = 1,   /* one fine Wilson-clover application              */
  DDAMG_PROF_COARSE_APPLY = 2,  /* one coarse stencil application                  */
  DDAMG_PROF_COARSE_SAP = 3,    /* one SAP colour sweep on a coarse level          */
  DDAMG_PROF_TRANSFER = 4,      /* one restriction or prolongation                 */
  DDAMG_PROF_PRECOND = 5,       /* one outer preconditioner application (K-cycle)  */
  DDAMG_PROF_OUTER_ORTHO = 6,   /* outer FGMRES Gram-Schmidt + norms of one step    */
  DDAMG_PROF_KINDS = 7
};

/* enable = bitmask (1 << DDAMG_PROF_*): reset the counters and record a CUDA
 * event pair around every launch of the selected classes (on the launching
 * stream); enable = 0 stops recording. */
int ddamg_profile(ddamg_handle* h, int enable);

/* Totals since the last ddamg_profile(h, 1): summed event time in ms, launch
 * count, and the algorithmic bytes those launches move (operator data once per
 * launch, vectors once per right-hand side). */
int ddamg_profile_read(ddamg_handle* h, int kind, double* total_ms, long long* launches, double* algo_bytes);

/* Kernels launched by this library since it was loaded (all handles).  A
 * captured K-cycle graph counts as one launch. */
long long ddamg_launch_count(void);

/* Arnoldi steps taken on a level since setup by its Krylov solver in the given
 * precision (level 0: the outer FGMRES; coarse levels: K-cycle FGMRES or the
 * coarsest GMRES). */
int ddamg_krylov_steps(ddamg_handle* h, int level, int precision, long long* steps);

/* Relative residual norms out[i] = ||rhs_i - D x_i|| / ||rhs_i|| (FP64 fine
 * operator of the handle, FP64 fine fields in the ABI layout), computed without
 * allocating any memory.  The paper has no counterpart: this entry point is for
 * callers that cannot call cudaMalloc, e.g. code running while another
 * allocator owns all free device memory, or code that must not trigger the
 * device synchronisation an allocation implies.  rhs and x must be device
 * pointers (nothing is staged); out may be host or device memory (n doubles).
 * The reduction uses a 1 MiB file-scope __device__ array (n <= 64 right-hand
 * sides; larger n is rejected with DDAMG_ERR_ARG), which every GPU that loads
 * the library holds until the process exits.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  Every call reuses
 * the same array and overwrites every entry it later reads, so nothing needs
 * clearing, but calls that overlap on the GPU (other streams or threads) race
 * on it. */
int ddamg_residual_norm_noalloc(ddamg_handle* h, const double* rhs, const double* x, int n, double* out);

/* Autotuner of the kernels that read FP16 operator data for a whole batch (FP16 storage).
 * kind DDAMG_TUNE_COARSE (levels >= 1): one coarse stencil application by the CUDA-core kernel (0)
 *   and by the tensor-core kernel with k-split 1..4;
 * kind DDAMG_TUNE_RESTRICT (level l -> l+1, l < L-1): the per-right-hand-side kernel (0) and the
 *   tensor-core kernel with k-split 1..4 (P read once per batch);
 * kind DDAMG_TUNE_PROLONG (level l+1 -> l): the per-right-hand-side kernel (0) and the kernel that
 *   reads P once for the batch (1).
 * kind DDAMG_TUNE_SAP (levels 1..L-2): one smoother call (nu SAP applications on the batch) as one
 *   launch per colour sweep (0) and as one persistent launch (1; timed only where it fits and an
 *   eager and a graph-captured trial run without error); ms[2] = the clusters of the persistent
 *   launch's shape the device holds at once (-1: not queried), ms[3] = the clusters it needs,
 *   ms[4] = the SAP blocks of each colour per cluster (1 or 2; 0: no shape fits).
 * ms[0..4] = milliseconds of one application of the handle's batch size per candidate (-1 where
 * the candidate does not fit or was not timed); *chosen = the candidate in use.  The tuner runs at
 * setup and when DDAMG_OPT_HALF_STORAGE, DDAMG_OPT_COARSE_TC or DDAMG_OPT_SAP_PERSIST is set; its
 * choice holds for every batch size.  Errors: ARG. */
enum { DDAMG_TUNE_COARSE = 0, DDAMG_TUNE_RESTRICT = 1, DDAMG_TUNE_PROLONG = 2, DDAMG_TUNE_SAP = 3 };
int ddamg_autotune_times(ddamg_handle* h, int kind, int level, double* ms, int* chosen);

/* ---- building blocks of the method, exposed for parity tests ------------ */

/* Level geometry: dims of level l, its dof per site, its test vectors N_l
 * (0 on the coarsest level). */
int ddamg_level_info(ddamg_handle* h, int level, int dims[4], int* ndof, int* ntv);

/* out = D_l in (n fields of level l).  Level 0 is the Wilson-clover operator of
 * Sec. 1 (the form of the two-level paper the text defers to); level l >= 1 is the
 * Galerkin operator D_l = P_{l-1}^dagger D_{l-1} P_{l-1} of Sec. 1, applied as its
 * 9-point stencil of dense blocks (Sec. 2).  precision 0 = FP64, 1 = FP32 arithmetic
 * on the FP32 path's storage (FP16 while DDAMG_OPT_HALF_STORAGE is on); the same for
 * the precision argument of the calls below.  Here only, precision 2 = double-FP32
 * arithmetic on FP64 vectors (level 0; the operator of DDAMG_OPT_OUTER_DF).  Other
 * values: ARG. */
int ddamg_apply(ddamg_handle* h, int level, int precision, const double* in, double* out, int n);

/* iterations x { z <- z + M_SAP (b - D_l z) } on level l < L-1 (z in/out): the SAP
 * smoother of Sec. 1 (red-black multiplicative Schwarz over lattice blocks, each
 * block solved by mr_steps minimal-residual steps, Table 1), one iteration being
 * the smoothing step of Alg. 1. */
int ddamg_smooth(ddamg_handle* h, int level, int precision, const double* b, double* z, int n, int iterations);

/* coarse = P_l^dagger fine (level l -> l+1): the restriction of Sec. 1, P_l built
 * from the aggregated test vectors (Sec. 2.2). */
int ddamg_restrict(ddamg_handle* h, int level, int precision, const double* fine, double* coarse, int n);

/* fine = P_l coarse (level l+1 -> l): the interpolation of Sec. 1. */
int ddamg_prolong(ddamg_handle* h, int level, int precision, const double* coarse, double* fine, int n);

/* z = K-cycle(l, b): one application of Alg. 2 (Alg. 1 with the coarse solve replaced
 * by FGMRES on D_{l+1} preconditioned by the K-cycle at l+1; coarsest level: the
 * odd-even GMRES of Sec. 3), mu/nu and the inner solver's length, cycles and
 * tolerance from the parameters (Table 1). */
int ddamg_kcycle(ddamg_handle* h, int level, int precision, const double* b, double* z, int n);

/* z = coarsest-level solve of b: odd-even preconditioned GMRES to coarse_tol
 * (Sec. 3; GMRES on the Schur complement, then the odd back-substitution; plain
 * GMRES on a coarsest lattice with an odd extent). */
int ddamg_coarse_solve(ddamg_handle* h, int precision, const double* b, double* z, int n);

/* Test vectors of level l (N_l fields of level l): the vectors Alg. 3 builds and
 * Alg. 4 refines. */
int ddamg_set_testvectors(ddamg_handle* h, int level, const double* tv, int n);
int ddamg_get_testvectors(ddamg_handle* h, int level, double* tv, int n);

/* Rebuilds P_l (CGS2 per aggregate and chirality, Sec. 2.2: the test vectors are
 * aggregated and orthonormalised per chirality) from the current test vectors and
 * D_{l+1} = P_l^dagger D_l P_l (Sec. 1); the step that ends each level of Alg. 3
 * and every pass of Alg. 4. */
int ddamg_rebuild(ddamg_handle* h, int level);

/* P_l as N_l fields of level l (the orthonormalised test vectors, Sec. 2.2). */
int ddamg_get_interpolation(ddamg_handle* h, int level, double* P);

/* D_l (l >= 1) as blocks [coarse site lex][k][row][col] complex, k = 0 self,
 * 1..4 forward mu = t,z,y,x (couples to site + mu), 5..8 backward mu: the
 * nearest-neighbour block structure of the Galerkin operator (Sec. 1, Sec. 2). */
int ddamg_get_coarse_operator(ddamg_handle* h, int level, double* blocks);

/* ---- Setup timing ------------------------------------------------------------
 * Wall-clock seconds the setup of this handle spent per level l and phase:
 * seconds[l * DDAMG_SETUP_KINDS + kind] for n entries (levels beyond the
 * hierarchy read 0).  SMOOTH: smoothing of the random test vectors (Alg. 3);
 * KCYCLE: the K-cycle applied to each test vector (Alg. 4); REBUILD: P
 * orthonormalisation and the Galerkin product of the next level (both
 * algorithms), including ddamg_rebuild.  Errors: ARG. */
enum {
  DDAMG_SETUP_SMOOTH = 0,
  DDAMG_SETUP_KCYCLE = 1,
  DDAMG_SETUP_REBUILD = 2,
  DDAMG_SETUP_KINDS = 3
};
int ddamg_setup_times(ddamg_handle* h, double* seconds, int n);

/* ---- Device footprint ------------------------------------------------------
 * Bytes of the device memory the library allocated for this handle (operators,
 * P, test vectors, Krylov workspaces, FP16 copies, staging buffers). */
int ddamg_device_bytes(ddamg_handle* h, size_t* bytes);
/* Estimate of ddamg_device_bytes for a hierarchy that is not built yet (host
 * arithmetic only, no device call).  Errors: ARG. */
int ddamg_estimate_bytes(const int dims[4], const ddamg_params* params, size_t* bytes);

/* ---- Serving -------------------------------------------------------------------
 * Not in the paper: a request loop over hierarchies that stay resident on the
 * device.  Each registered hierarchy gets a worker thread that runs the outer
 * FGMRES of Sec. 2 one restart cycle at a time on a batch of up to max_rhs
 * right-hand sides (continuous batching): waiting right-hand sides enter free
 * batch slots at every restart boundary, and a right-hand side leaves the batch
 * once its true residual meets its tolerance (or after outer_max_cycles cycles).
 * Every right-hand side is computed with batch-independent reductions, so its
 * result does not depend on what else shares its batch.  Different hierarchies
 * run on their handles' own streams and overlap on the device.  While a handle
 * is registered, no other call may use it; ddamg_server_free returns it. */
typedef struct ddamg_server ddamg_server;
/* hbm_budget: device bytes the registered hierarchies may hold (0: 90% of the
 * device memory). */
int ddamg_server_create(size_t hbm_budget, ddamg_server** out);
/* Registers a built hierarchy; *hid identifies it in submissions.  Errors:
 * ADMISSION if its ddamg_device_bytes exceed the remaining budget, ARG. */
int ddamg_server_add(ddamg_server* s, ddamg_handle* h, int* hid);
/* Queues n right-hand sides (host memory, the ddamg_solve layout, copied before
 * the call returns) at relative tolerance tol; *id names the request.  Returns
 * at once. */
int ddamg_server_submit(ddamg_server* s, int hid, const double* rhs, int n, double tol, long long* id);
/* *done = 1 once the request has finished (its result can be taken by wait). */
int ddamg_server_poll(ddamg_server* s, long long id, int* done);
/* Blocks until request id has finished, copies its n solutions to x (host, the
 * ddamg_solve layout) and per_rhs statistics (may be NULL), and releases it.
 * times (may be NULL) receives 3 doubles in seconds: queueing before its first
 * restart cycle, latency from submission to completion, time in the batch.
 * Returns OK, NOCONV (x holds the last iterates) or the error of its batch. */
int ddamg_server_wait(ddamg_server* s, long long id, double* x, ddamg_stats* per_rhs, double* times);
/* Finishes the right-hand sides in the batches, fails the queued ones, joins
 * the workers and frees the server (not the hierarchies). */
int ddamg_server_free(ddamg_server* s);

#ifdef __cplusplus
}
#endif

#endif /* DDAMG_H */
