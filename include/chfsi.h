/*
 * chfsi.h -- C ABI of a GB300-native Chebyshev filtered subspace iteration (ChFSI) for
 * sequences of dense complex Hermitian generalized eigenproblems  H x = lambda S x
 * (Berljafa & Di Napoli, "A Parallel and Scalable Iterative Solver for Sequences of Dense
 * Eigenproblems Arising in FLAPW", arXiv:1305.5120).
 *
 * Conventions (all entry points):
 *  - Matrices are complex128 with interleaved (re, im) doubles, COLUMN-MAJOR, leading
 *    dimension = number of rows (n for n x n and n x k blocks, k for k x k).
 *  - Every matrix/vector pointer is a DEVICE pointer on the context's device, unless the
 *    comment says "host".  The caller owns all pointers it passes; the library keeps none
 *    of them after a call returns.  The context owns its workspaces and the sequence state.
 *  - Work is ordered on the context's CUDA stream; every call returns after its work has
 *    completed (the host needs residuals to decide locking and termination).
 *  - Errors are returned as chfsi_status.  Outputs are unspecified on error, except that
 *    CHFSI_ERR_NO_CONV still fills the converged prefix and `info`.  After CHFSI_ERR_CUDA
 *    the context must be destroyed; after any other error it stays usable.
 *  - One context = one sequence = one stream.  Contexts are independent; a context must not
 *    be used by two host threads at once.
 */
#ifndef CHFSI_H
#define CHFSI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct chfsi_ctx chfsi_ctx;

typedef enum {
  CHFSI_OK = 0,
  CHFSI_ERR_ARG = 1,       /* invalid argument (sizes, NULL pointers, tolerances) */
  CHFSI_ERR_NOT_HPD = 2,   /* S is not Hermitian positive definite (Cholesky pivot <= 0) */
  CHFSI_ERR_NO_CONV = 3,   /* max_iter outer iterations without nev locked pairs, or the
                              reduced eigensolver did not converge */
  CHFSI_ERR_OOM = 4,       /* device allocation failed */
  CHFSI_ERR_CUDA = 5,      /* a CUDA runtime call failed (context unusable) */
  CHFSI_ERR_TIMEOUT = 6,   /* a bounded device-side wait ran out (kernel returned early) */
  CHFSI_ERR_STATE = 7,     /* call out of order (e.g. next_in_sequence before solve) */
  CHFSI_ERR_NUMERIC = 8,   /* NaN/Inf met in a residual or a filtered block */
  CHFSI_ERR_INCOMPLETE = 9 /* nev pairs passed the residual test but the completeness check
                              failed: a Ritz value outside the returned set lies below the
                              largest returned eigenvalue, or (check_inertia) the count of
                              eigenvalues below the gap differs from nev.  Outputs are filled
                              as for CHFSI_OK but are not the lowest nev eigenpairs. */
} chfsi_status;

enum {
  CHFSI_PREC_FP64 = 0,     /* every filter product in FP64 (DFMA) */
  CHFSI_PREC_MIXED = 1     /* filter products on the tensor cores in split-BF16 (FP32-equivalent)
                              while residuals are large (see mixed_switch), then FP64; Cholesky, transform, QR,
                              Rayleigh-Ritz, residuals and Lanczos always FP64 */
};

typedef struct {
  int degree;              /* filter degree m when per_vector_degree == 0 (default 20) */
  int degree_min;          /* per-vector degree range (default 10 .. 25) */
  int degree_max;
  int per_vector_degree;   /* 0: one degree for the block; 1: degree chosen per vector */
  int max_iter;            /* outer iterations of Algorithm 1 (default 50) */
  int lanczos_steps;       /* Lanczos steps of the spectral bound (default 20, <= 256) */
  int precision;           /* CHFSI_PREC_* (default FP64) */
  double mixed_switch;     /* MIXED: tensor-core filter while the smallest active absolute residual
                              exceeds mixed_switch * max(|a0|, |b|) and still drops at least 10x
                              per pass (default 1e-6) */
  unsigned long long seed; /* SplitMix64 seed of the Lanczos start vectors and of the random
                              start block (default 0) */
  int check_inertia;       /* 0 (default): after convergence, only the Ritz-value test below;
                              1: also count the eigenvalues of H' below the gap sigma between the
                              largest returned eigenvalue and the smallest other Ritz value
                              (Sylvester: H' - sigma I + tau Y Y^H, Y the returned vectors, must
                              be positive definite -- an FP32 Cholesky for n <= 8192, the
                              blocked FP64 one above; valid while the gap exceeds the
                              factorisation's backward error; smaller gaps are reported as
                              inconclusive, not as failures).  Every solve checks
                              that no unreturned Ritz value of the block lies below the largest
                              returned eigenvalue. */
} chfsi_params;

typedef struct {
  int iterations;          /* outer iterations of the last solve */
  int locked;              /* pairs locked */
  long long filter_col_steps;       /* sum over filter launches of (columns x degree) */
  long long filter_col_steps_lowp;  /* of which on the low-precision tensor-core path */
  double max_resid;        /* largest relative residual ||H'y - lam y|| / ||H'y|| returned */
  double kappa_L;          /* upper estimate of cond_2(L), S = L L^H */
  double bounds[3];        /* (a, b, a0) of the last filter: damped interval [a, b], scale point a0 */
  double ms_stage[8];      /* device time per stage: 0 reduce (Cholesky, inverse, H'), 1 Lanczos,
                              2 filter, 3 QR, 4 Rayleigh-Ritz, 5 residual+locking,
                              6 back-transform, 7 whole call */
  double ms_filter_lowp;   /* part of ms_stage[2] spent in tensor-core (low-precision) filter passes */
  double ms_gemm_tc;       /* device time of the FP64-accurate tensor-core GEMMs (all stages) */
  double gemm_tc_flop;     /* their algorithmic work: 8 M N K_eff real flops per complex product */
  double ms_eig;           /* device time of the reduced eigensolver (Rayleigh-Ritz) */
  int eig_sweeps;          /* FP64 Jacobi sweeps that rotated (FP64 mode and fallbacks), summed */
  long long eig_rounds;    /* FP64 Jacobi rounds that rotated (each updates the whole k x k matrix
                              and its eigenvector accumulator), summed over the call */
  double eig_flop;         /* their algorithmic FP64 work: 28 k^2 real flops per rotating round */
  int n_floor;             /* returned pairs whose residual was tested against the absolute floor
                              (|lambda| < 1e-4 ||H'||: Res = ||H'y - lam y|| / (1e-4 ||H'||)) */
  int completeness;        /* 1: Ritz-value test passed; 2: inertia count passed too; -1: inertia
                              count inconclusive (gap below its resolution); 0: not reached */
  double ms_filter_steps;  /* device time of the tensor-core recurrence steps alone (the step
                              kernels of ms_filter_lowp, without operand slicing) */
  long long filter_step_cols; /* column-steps those kernels processed (each: one complex column
                              times the n x n H', 48 n^2 executed / 8 n^2 algorithmic flops) */
  int eig_refined;         /* reduced eigensolves done by FP32 one-sided Jacobi + FP64 refinement */
  int eig_refine_iters;    /* their FP64 refinement iterations */
  int eig_f32_sweeps;      /* their FP32 sweeps */
  int eig_fallbacks;       /* reduced eigensolves that fell back to the FP64 Jacobi */
  double ms_chol;          /* device time of the Cholesky factorisation of S and its inverse */
  double chol_flop;        /* its algorithmic work: (8/3) n^3 real flops (factor and inverse) */
} chfsi_info;

/* Fills *p with the defaults listed above. */
chfsi_status chfsi_default_params(chfsi_params *p);

/* Creates a context on `device` whose work runs on `cuda_stream` (a cudaStream_t, NULL =
 * the legacy default stream).  p may be NULL (defaults).  Allocates nothing on the device
 * until the first solve. */
chfsi_status chfsi_create(chfsi_ctx **out, int device, void *cuda_stream, const chfsi_params *p);

/*
 * First problem of a sequence (Algorithm 1 of the paper, preceded by the reduction to
 * standard form of Section 3):
 *   S = L L^H, H' = L^{-1} H L^{-H}, Lanczos bound, then repeat [Chebyshev filter, QR,
 *   Rayleigh-Ritz, residuals, deflation and locking] until nev pairs are locked.
 * H, S: n x n Hermitian (S positive definite).  X0: n x (nev+nex) start block in the space
 * of x (the library uses Y0 = L^H X0), or NULL for a SplitMix64 random block.  A pair locks
 * when ||H'y - lam y|| / ||H'y|| < tol / kappa_L, which bounds the generalized relative
 * residual ||H x - lam S x|| / ||H x|| by tol.  degree <= 0 takes params.degree.
 * Outputs: evals[nev] ascending (device), X (n x nev, device) S-orthonormal eigenvectors.
 * info may be NULL.
 */
chfsi_status chfsi_solve(chfsi_ctx *c, const void *H, const void *S, int n, int nev, int nex,
                         const void *X0, double tol, int degree, double *evals, void *X,
                         chfsi_info *info);

/*
 * Next problem of the sequence (Section 2: each P^(l) is seeded with the solution of
 * P^(l-1); Algorithm 1 Require: previous eigenvectors and eigenvalues).  Uses the stored
 * Ritz block (nev + nex vectors) as start block and the stored lowest/highest Ritz values
 * as filter bounds; re-runs Lanczos for the upper bound.  S_next == NULL keeps S (and L).
 * Same n, nev, nex, tol and degree as the previous solve.
 */
chfsi_status chfsi_next_in_sequence(chfsi_ctx *c, const void *H_next, const void *S_next,
                                    double *evals, void *X, chfsi_info *info);

/*
 * Many independent problems solved together (the k-point problems of one SCF cycle, Section
 * 2: for every k-point its own H x = lambda S x).  Problem p: H[p], S[p] (n[p] x n[p]),
 * nev[p], nex[p]; random start blocks; every problem to the same tol and degree.  Each
 * problem runs Algorithm 1 as chfsi_solve would (same results); the iterations of all
 * problems advance together, and the filter of one iteration of every problem is one grouped
 * tensor-core launch per recurrence step (a tile scheduler over all problems' tiles, tile
 * width picked by a timing autotuner, the step launches captured into a CUDA graph).
 * Host arrays of device pointers: H, S, evals (evals[p]: nev[p] doubles), X (X[p]: n[p] x
 * nev[p]); host arrays status[count] (per problem) and info[count] (may be NULL).  Returns
 * CHFSI_OK when every problem succeeded, else the first problem's failure status.  The
 * context keeps one internal context per problem slot (device memory for each; released by
 * chfsi_destroy); the problems are not sequences (chfsi_next_in_sequence does not apply).
 */
chfsi_status chfsi_solve_batch(chfsi_ctx *c, int count, const void *const *H, const void *const *S, const int *n,
                               const int *nev, const int *nex, double tol, int degree, double *const *evals,
                               void *const *X, chfsi_status *status, chfsi_info *info);

/* Upper estimate of the device memory (bytes) a context allocates to solve problems of size
 * (n, nev, nex) in the given precision; callers that admit work by memory budget (the
 * serving loop) use it.  Inputs and outputs owned by the caller are not included. */
size_t chfsi_workspace_bytes(int n, int nev, int nex, int precision);

void chfsi_destroy(chfsi_ctx *c);
const char *chfsi_status_string(chfsi_status s);

/* Number of CUDA kernels this library has launched in this process (all contexts).  A
 * diagnostic for benchmarks; the paper has no counterpart. */
unsigned long long chfsi_kernel_launches(void);

/* Measured FP64 (DFMA) throughput of `device` in TFLOP/s (host double): eight independent FMA
 * chains per thread on every SM, best of three timed launches.  The roofline denominator of
 * the FP64 kernels; a diagnostic, the paper has no counterpart. */
chfsi_status chfsi_fp64_peak(int device, double *tflops);

/* ---- Stage entry points (each step of the solve on its own; device pointers) -------- */

/* The dense complex product the stages are built from: C = alpha op(A) op(B) + beta C,
 * op = 'N' (as stored) or 'C' (conjugate transpose); op(A) is M x K, op(B) K x N, all
 * column-major with leading dimensions lda, ldb, ldc.  alpha, beta: host (re, im) pairs.
 * CHFSI_PREC_FP64 runs it on the FP64 pipe; CHFSI_PREC_MIXED as an error-free expansion in
 * BF16 digits on the tensor cores (12 digits per entry relative to its row or column
 * scale -- a 7-bit top digit and eleven of 5 bits --, exact integer accumulation per
 * significance level, levels combined exactly in 64-bit integers: 61 bits of the
 * row/column scale before the single FP64 rounding). */
chfsi_status chfsi_gemm(chfsi_ctx *c, char opA, char opB, int M, int N, int K, const double *alpha,
                        const void *A, int lda, const void *B, int ldb, const double *beta, void *C,
                        int ldc, int precision);

/* a1. S = L L^H (Section 3).  L: n x n lower triangular output (upper part zeroed). */
chfsi_status chfsi_cholesky(chfsi_ctx *c, int n, const void *S, void *L);

/* a2. H' = L^{-1} H L^{-H}, Hermitian part (Section 3 standard form).  L from chfsi_cholesky. */
chfsi_status chfsi_reduce(chfsi_ctx *c, int n, const void *H, const void *L, void *Hs);

/* a3. `steps`-step Lanczos on Hermitian Hs from v0 (n vector, normalised internally; NULL =
 * SplitMix64 stream 0 of params.seed).  alpha[steps], beta[steps]: recurrence coefficients
 * (device).  bounds[4] (device): b_sup = max Ritz value + |beta_last| |z_last| (the residual
 * norm of the top Ritz pair, z its eigenvector of T) + 1e-3 of the Ritz spread (Algorithm 1 line 1),
 * a = first-solve lower end of the damped interval (the Lanczos density-of-states estimate of
 * lambda_{k+1}), a0 = smallest Ritz value, max Ritz value.
 * k = block size used for a. */
chfsi_status chfsi_lanczos(chfsi_ctx *c, int n, const void *Hs, int steps, int k, const void *v0,
                           double *alpha, double *beta, double *bounds);

/* a4 / a4m. Chebyshev filter (Algorithm 1 line 3, Eq. (3term) scaled and shifted):
 * Y <- T_m((H' - cI)/e) Y / T_m((a0 - c)/e), e = (b - a)/2, c = (b + a)/2.
 * Y: n x k, overwritten.  precision: CHFSI_PREC_FP64 or CHFSI_PREC_MIXED (tensor cores). */
chfsi_status chfsi_filter(chfsi_ctx *c, int n, int k, const void *Hs, void *Y, int m, double a,
                          double b, double a0, int precision);

/* a4m, residual-corrected form for a Ritz block: Y (n x k) with Ritz values lam[k] (device)
 * and Z = H' Y (n x k, device), as chfsi_rayleigh_ritz returns them.  Computes the same
 * T_m((H' - cI)/e) Y / T_m((a0 - c)/e) as chfsi_filter, written as Y p_m(lam) + D_m with
 * D_j = fa_j H' D_{j-1} + fb_j D_{j-1} + fg_j D_{j-2} + fa_j (Z - Y diag(lam)) p_{j-1}(lam):
 * the tensor-core products act on D, whose size is proportional to the residual, so their
 * rounding error shrinks with it instead of flooring the subspace accuracy. */
chfsi_status chfsi_filter_ritz(chfsi_ctx *c, int n, int k, const void *Hs, void *Y, const double *lam,
                               const void *Z, int m, double a, double b, double a0);

/* a10 (filter part). Column i filtered with its own degree deg[i] (host array, non-increasing). */
chfsi_status chfsi_filter_degrees(chfsi_ctx *c, int n, int k, const void *Hs, void *Y, const int *deg,
                                  double a, double b, double a0, int precision);

/* a5. Orthonormal basis of Y (n x k, overwritten) orthogonal to the nl orthonormal columns
 * Ylocked (n x nl, may be NULL when nl == 0): two block Gram-Schmidt passes against Ylocked,
 * then CholQR2 (shifted CholQR first when the Gram matrix is too ill-conditioned).  The
 * result equals the Q of a QR factorisation with positive real diagonal R. */
chfsi_status chfsi_orthonormalize(chfsi_ctx *c, int n, int nl, const void *Ylocked, int k, void *Y);

/* a6-a8. Rayleigh-Ritz (Algorithm 1 lines 5-7): G = Y^H H' Y, G W = W Lambda (ascending),
 * Y <- Y W, Z <- H' Y.  Y: n x k orthonormal in, Ritz vectors out; lam[k]; Z: n x k out. */
chfsi_status chfsi_rayleigh_ritz(chfsi_ctx *c, int n, int k, const void *Hs, void *Y, double *lam, void *Z);

/* a7 alone. All eigenpairs of the k x k Hermitian G: lam ascending, W.  Mixed precision with
 * k >= 32: FP32 one-sided Jacobi in one thread-block cluster, refined to FP64 accuracy by
 * FP64-accurate tensor-core products, with the parallel FP64 Jacobi as fallback; FP64
 * precision: the parallel FP64 Jacobi.  Diagnostics: CHFSI_DEBUG_EIG=1 prints every call's
 * sweeps, iterations and any fallback reason to stderr; CHFSI_OS_CLUSTER=8|16 picks the
 * cluster size of the FP32 stage. */
chfsi_status chfsi_reduced_eig(chfsi_ctx *c, int k, const void *G, double *lam, void *W);

/* Allocation-free form of chfsi_reduced_eig, for callers that cannot allocate device memory
 * (a plugin or callback that owns no device allocator, or a loop that must not trigger the
 * device-wide synchronisation of cudaMalloc/cudaFree).  The paper has no counterpart.
 * Same result as chfsi_reduced_eig (G k x k Hermitian, device, not modified; lam[k]
 * ascending and W k x k, device) with no context: work is ordered on `cuda_stream` (NULL =
 * legacy default stream) of the current device and the call returns when it is complete.
 * Scratch lives in one fixed device array of this library, sized for k <= 256
 * (CHFSI_NOALLOC_KMAX); larger k returns CHFSI_ERR_ARG.  The first call on a device looks
 * up that array's device address (a one-time set-up with the device current).  Every call
 * is synchronous: it reads the status word back to host memory and waits for the stream,
 * so it must not be called while the stream is being captured into a CUDA graph.  Every
 * call on a device shares the array and
 * re-initialises it, so calls whose work overlaps on the GPU (other streams, other host
 * threads) race and must be serialised by the caller; the same holds against solves of
 * other contexts running at that time, since both use grid-wide barriers.  Nothing is
 * allocated or freed. */
#define CHFSI_NOALLOC_KMAX 256
chfsi_status chfsi_reduced_eig_noalloc(void *cuda_stream, int k, const void *G, double *lam, void *W);

/* a9. res[j] = ||Z_j - lam_j Y_j|| / ||Z_j|| (Algorithm 1, Res), Z = H' Y. */
chfsi_status chfsi_residuals(chfsi_ctx *c, int n, int k, const void *Z, const void *Y, const double *lam,
                             double *res);

/* a10. Per-vector degree m_i = clamp(ceil(ln(tol/r_i)/ln rho_i), m_min, m_max),
 * rho_i = 1/(|t_i| + sqrt(t_i^2 - 1)), t_i = (lam_i - c)/e.  deg: device int[k]. */
chfsi_status chfsi_degrees(chfsi_ctx *c, int k, const double *lam, const double *res, double a, double b,
                           double tol, int m_min, int m_max, int *deg);

/* a11. X = L^{-H} Y (back-transform to eigenvectors of the pencil).  Y: n x k. */
chfsi_status chfsi_back_transform(chfsi_ctx *c, int n, int k, const void *L, const void *Y, void *X);

#ifdef __cplusplus
}
#endif
#endif /* CHFSI_H */
