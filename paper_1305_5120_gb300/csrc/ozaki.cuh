// FP64-accurate complex GEMM on the BF16 tensor cores (error-free digit splitting).
#pragma once
#include "zgemm.cuh"

struct OzakiGemm;
OzakiGemm* ozaki_new();
void ozaki_free(OzakiGemm* o);
// C = alpha op(A) op(B) + beta C (complex, column-major), same arguments as zgemm_launch
// (EPI_GEMM only; tri flags prune the K range).  `err` is the caller's device error word: a
// bounded wait that runs out records DEV_ERR_TIMEOUT there.  Returns a CUDA error code.
cudaError_t ozaki_gemm(OzakiGemm* o, const GemmArgs& g, cudaStream_t s, int* err);
