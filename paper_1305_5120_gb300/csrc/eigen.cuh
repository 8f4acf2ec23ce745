// Reduced eigenproblem G w = lam w of Rayleigh-Ritz (Algorithm 1): FP32 one-sided Jacobi in one
// thread-block cluster, then FP64 refinement (the products are issued by the caller).
#pragma once
#include "common.cuh"

constexpr int OA_GROUP_MAX = 32;   // largest group of strongly coupled pairs solved exactly

// B = G + shift I (FP32), then one-sided Jacobi on B's columns until no pair is above the
// threshold (|x^H y| <= tol ||x|| ||y||) or, with the columns in the cluster's shared memory
// (k up to ~450), until a sweep's largest coupling is below 1e-4; at most
// max_sweeps sweeps.  On return B = W, whose columns are multiples of eigenvectors.  nrm:
// max(k, max_sweeps + 1) floats of scratch; counters: max_sweeps + 1 ints (zeroed here);
// *sweeps the sweeps run; *err DEV_ERR_NO_CONV if max_sweeps ran out.  *cluster_used: CTAs in
// the cluster (CHFSI_OS_CLUSTER = 8 or 16 picks it; by default 16 where the device allows it).
cudaError_t os_jacobi_f32(cudaStream_t s, int k, const cplx* G, double shift, float2* B, float* nrm, int* counters,
                          int max_sweeps, float tol, int* err, int* sweeps, int* cluster_used);
// X = the columns of W normalised (FP64).
cudaError_t os_columns(cudaStream_t s, int k, const float2* W, cplx* X);
// From T = X^H [X | G X] (k x 2k, ld k): lam_i = S_ii / (1 - R_ii), R = I - herm(X^H X),
// S = herm(X^H G X) (k x k each), maxbits[0] = bits of max_{i != j} |S_ij|^2, maxbits[1] =
// bits of max |R_ij|^2, maxbits[2] = bits of max |S_ij + lam_j R_ij|^2 / (lam_j - lam_i)^2 over
// the weakly coupled pairs (the squared size of the coming first-order correction), and the
// strongly coupled pairs (|S_ij| > tau |lam_j - lam_i|, i < j): *npairs of them (the first
// `cap` stored in pairs).
cudaError_t oa_analyze(cudaStream_t s, int k, const cplx* T, double tau, double* lam, cplx* R, cplx* S,
                       unsigned long long* maxbits, int* npairs, int cap, int2* pairs);
// Exact FP64 diagonalisation of each group's block of S (group g: members idx[off[g] ..
// off[g+1]), at most OA_GROUP_MAX): eigenvectors into V (c x c at voff[g]).
cudaError_t oa_groups(cudaStream_t s, int k, int ngroups, const cplx* S, const int* off, const int* idx,
                      const int* voff, cplx* V, int* err);
// Y = Z U (rows x k), or with both_sides Y = U^H Z U (k x k, through tmp), U the block-diagonal
// unitary of the groups (identity outside them; gid[j] = group of j or -1, gpos[j] its place).
cudaError_t oa_mix(cudaStream_t s, int rows, int k, const cplx* Z, cplx* Y, bool both_sides, cplx* tmp, const int* gid,
                   const int* gpos, const int* off, const int* idx, const int* voff, const cplx* V);
// First-order correction F (X <- X (I + F)) from S2 = U^H S U and R2 = U^H R U.
cudaError_t oa_update(cudaStream_t s, int k, const cplx* S2, const cplx* R2, const int* gid, cplx* F);
// lam ascending with W's columns in the same order (ties by index) from values d and vectors X.
cudaError_t oa_sort(cudaStream_t s, int k, const double* d, const cplx* X, double* lam, cplx* W);
