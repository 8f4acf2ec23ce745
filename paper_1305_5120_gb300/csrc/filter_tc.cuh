// Chebyshev filter on the tensor cores (tcgen05, split-BF16 operands, FP32 accumulation in
// TMEM, FP64 recurrence state) -- the mixed-precision form of Algorithm 1 line 3.
#pragma once
#include "common.cuh"

struct TcFilter;
TcFilter* tc_filter_new();
void tc_filter_free(TcFilter* f);
// Runs mmax recurrence steps: Y_j = fa[j] H Y_{j-1} + fb[j] Y_{j-1} + fg[j] Y_{j-2} on the
// first cnt[j] columns; Y_j lands in bufs[j & 1] (bufs[0] holds Y_0 on entry).
chfsi_status tc_filter_run(TcFilter* f, cudaStream_t s, int n, const cplx* H, cplx* bufs[2], const int* cnt,
                           int mmax, const double* fa, const double* fb, const double* fg);
