// FP64 complex GEMM on the DFMA pipe, with the Chebyshev-recurrence epilogue.
#pragma once
#include "common.cuh"

enum GemmOp { OP_N = 0, OP_C = 1 };   // op(X) = X or X^H
enum GemmTri {                        // zero structure of op(A) / op(B) (K-range pruning)
  TRI_NONE = 0,
  TRI_A_LOWER = 1,   // op(A)[i,k] = 0 for k > i
  TRI_A_UPPER = 2,   // op(A)[i,k] = 0 for k < i
  TRI_B_UPPER = 4,   // op(B)[k,j] = 0 for k > j
  TRI_B_LOWER = 8,   // op(B)[k,j] = 0 for k < j
  TRI_C_LOWER = 16   // only C[i,j], i >= j, is wanted: tiles strictly above the diagonal may be
                     // skipped (left unwritten) -- honoured by the digit-expansion GEMM
};
enum GemmEpi { EPI_GEMM = 0, EPI_FILTER = 1 };

struct GemmArgs {
  int M, N, K;
  int opA, opB, tri;
  const cplx* A; long lda;
  const cplx* B; long ldb;
  cplx* C; long ldc;
  cplx alpha, beta;            // EPI_GEMM: C = alpha * op(A) op(B) + beta * C
  int epi;
  // EPI_FILTER: C = fa * (A B) + fb * Ycur + fg * C   (C holds Y_{j-1} on entry, Y_{j+1} on exit)
  const cplx* Ycur; long ldy;
  double fa, fb, fg;
  int splits;                  // split-K factor (>= 1); partial sums go to `work`
  cplx* work;                  // splits * M * N complex when splits > 1
};

// Launch C = epilogue(op(A) op(B)) on `stream`; returns a CUDA error code.
cudaError_t zgemm_launch(const GemmArgs& g, cudaStream_t stream);
// Bytes of workspace zgemm_launch needs for a given split-K factor.
size_t zgemm_work_bytes(int M, int N, int splits);
