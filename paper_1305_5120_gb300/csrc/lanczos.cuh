// Lanczos spectral-bound estimator (Algorithm 1, line 1) and the per-vector degree rule.
#pragma once
#include "common.cuh"

// w = H v for Hermitian H (column-major): w_i = sum_r conj(H[r, i]) v_r, one warp per column
// (each warp streams one contiguous column with 16-byte loads).  For any square H the same
// call gives w = H^H v.
cudaError_t herm_gemv(cudaStream_t s, int n, const cplx* H, long ldh, const cplx* v, cplx* w);
// w = A v for lower-triangular A (column-major): partial sums over 64-column chunks (coalesced
// column reads, chunks above the diagonal skipped) added in a fixed order.  part: n * ceil(n / 64).
cudaError_t lower_gemv(cudaStream_t s, int n, const cplx* A, long lda, const cplx* v, cplx* w, cplx* part);
// v <- v / ||v||   (single CTA)
cudaError_t normalize_vec(cudaStream_t s, int n, cplx* v);
// One Lanczos recurrence step on (v, v_prev, w = Op v):  alpha_j = Re(v^H w);
// w -= alpha_j v + beta_{j-1} v_prev; beta_j = ||w||; v_prev <- v; v <- w / beta_j.
cudaError_t lanczos_step(cudaStream_t s, int n, int j, cplx* v, cplx* v_prev, cplx* w, double* alpha,
                         double* beta);
// From T = tridiag(beta, alpha, beta) of `steps` steps: out[0] = b_sup = mu_max + |beta_last| |z_last|
// + 1e-3 (mu_max - mu_min); out[1] = a, the Lanczos density-of-states estimate of lambda_{k+1}
// (first Ritz value from the second on whose cumulative Gauss weight reaches k / n);
// out[2] = a0 = mu_min; out[3] = mu_max.  Eigenvalues of T by Sturm-count multisection, one
// CTA per eigenvalue; scratch holds 2 steps doubles (the eigenvalues of T and of its trailing
// block).
cudaError_t lanczos_bounds(cudaStream_t s, int steps, int n, int k, const double* alpha, const double* beta,
                           double* out, double* scratch);
// m_i = clamp(ceil(ln(tol / r_i) / ln(rho_i)), m_min, m_max), rho_i = 1 / (|t_i| + sqrt(t_i^2 - 1)),
// t_i = (lam_i - c) / e; m_min for converged vectors, m_max inside the damped interval.
cudaError_t vector_degrees(cudaStream_t s, int k, const double* lam, const double* res, double a, double b,
                           double tol, int m_min, int m_max, int* deg);
