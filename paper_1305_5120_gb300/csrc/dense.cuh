// FP64 dense factorisations and small kernels used around the filter.
#pragma once
#include "zgemm.cuh"

// In-place blocked Cholesky A = L L^H of an n x n Hermitian matrix (lower triangle used;
// the strictly upper triangle is zeroed on exit).  A non-positive or non-finite pivot sets
// *err = DEV_ERR_NOT_HPD; later blocks are then skipped by the kernels.
cudaError_t chol_lower(cudaStream_t s, int n, cplx* A, long lda, int* err);
// X = L^{-1} for lower-triangular L (X fully written, upper triangle zero).
cudaError_t trtri_lower(cudaStream_t s, int n, const cplx* L, long ldl, cplx* X, long ldx, int* err);
// A <- (A + A^H) / 2 (diagonal made real).
cudaError_t hermitize(cudaStream_t s, int n, cplx* A, long lda);
// Upper triangle <- conjugate transpose of the lower one (diagonal made real).
cudaError_t herm_from_lower(cudaStream_t s, int n, cplx* A, long lda);
// dst[:, j] = src[:, perm[j]] for j < cnt (n rows); and lam_dst[j] = lam_src[perm[j]].
cudaError_t gather_columns(cudaStream_t s, int n, int cnt, const int* perm, const cplx* src, long lds,
                           cplx* dst, long ldd);
cudaError_t gather_values(cudaStream_t s, int cnt, const int* perm, const double* src, double* dst);
// Column-wise relative residuals res[j] = ||Z_j - lam_j Y_j|| / max(||Z_j||, floor), and abs[j]
// the numerator.
cudaError_t residual_norms(cudaStream_t s, int n, int k, const cplx* Z, long ldz, const cplx* Y, long ldy,
                           const double* lam, double* res, double* resabs, double floor = 0.0);
// lam[j] = Re(Y_j^H Z_j) (Rayleigh quotients when Z = H Y and ||Y_j|| = 1).
cudaError_t rayleigh_quotients(cudaStream_t s, int n, int k, const cplx* Y, long ldy, const cplx* Z, long ldz,
                               double* lam);
// SplitMix64 complex block: element (i, j) = u(2(j n + i)) + i u(2(j n + i) + 1), u in [-0.5, 0.5),
// counter offset stream * 2^40 (the same definition the oracle uses).
cudaError_t splitmix_block(cudaStream_t s, int n, int k, unsigned long long seed, unsigned long long stream,
                           cplx* Y, long ldy);
// Copy an n x k block between leading dimensions.
cudaError_t copy_block(cudaStream_t s, int n, int k, const cplx* src, long lds, cplx* dst, long ldd);
// Hermitian positive definite A (k x k, k <= CHOL_INV_KMAX): lower L (in place, upper zeroed) with
// A = L L^H and X = L^{-1}, in one cooperative launch over all SMs (blocked right-looking,
// 32-wide blocks).  A non-positive pivot sets *err = DEV_ERR_NOT_HPD.  work: chol_inv_work_bytes(k).
// X == NULL factors only (A is still overwritten by L).
constexpr int CHOL_INV_KMAX = 8192;
size_t chol_inv_work_bytes(int k);
cudaError_t chol_inv_small(cudaStream_t s, int k, cplx* A, cplx* X, void* work, int* err);
// The same factorisation in FP32 (complex64 A and X), for well-conditioned Gram matrices whose
// factor only needs FP32 accuracy; work: chol_inv_work_bytes(k).
cudaError_t chol_inv_small_f32(cudaStream_t s, int k, float2* A, float2* X, void* work, int* err);
