// Reduced Hermitian eigenproblem G w = lam w of the Rayleigh-Ritz step (Algorithm 1).
#pragma once
#include "common.cuh"

// All eigenpairs of the k x k Hermitian G (column-major, ld = k, destroyed) by parallel
// cyclic Jacobi in one cooperative launch; writes lam (ascending) and W (k x k, columns =
// eigenvectors in the same order).  `work` must hold jacobi_work_bytes(k).  *err receives
// DEV_ERR_NO_CONV or DEV_ERR_TIMEOUT on failure; *sweeps the count of sweeps that rotated and
// *rounds the count of rounds that rotated (each updates the whole matrix and W).
size_t jacobi_work_bytes(int k);
cudaError_t jacobi_eig(cudaStream_t s, int k, cplx* G, double* lam, cplx* W, void* work, int* err, int* sweeps,
                       int* rounds);
