// Shared device helpers for the ChFSI library (complex FP64 arithmetic, reductions,
// bounded grid barrier).  Matrices are complex128, interleaved (re, im), column-major.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "chfsi.h"

typedef double2 cplx;

__host__ __device__ __forceinline__ cplx cmk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ cplx cadd(cplx a, cplx b) { return cmk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cplx csub(cplx a, cplx b) { return cmk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cplx cscale(cplx a, double s) { return cmk(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ cplx cconj(cplx a) { return cmk(a.x, -a.y); }
__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__host__ __device__ __forceinline__ cplx cmulc(cplx a, cplx b) {
  return cmk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// acc += a * b
__device__ __forceinline__ void cfma(cplx& acc, cplx a, cplx b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ cplx warp_sum(cplx v) {
  v.x = warp_sum(v.x);
  v.y = warp_sum(v.y);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum of one double per thread (blockDim.x a multiple of 32, <= 1024).
__device__ __forceinline__ double block_sum(double v, double* sh /* >= 32 doubles */) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = (threadIdx.x < (unsigned)nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  double r = sh[0];
  __syncthreads();
  return r;
}

// Device-side error word: kernels never trap; they record a code and return.
enum { DEV_OK = 0, DEV_ERR_TIMEOUT = 1, DEV_ERR_NOT_HPD = 2, DEV_ERR_NUMERIC = 3, DEV_ERR_NO_CONV = 4 };

// Grid barrier for cooperative launches (all blocks co-resident).  The spin is bounded:
// after `limit` polls it records DEV_ERR_TIMEOUT in *err and returns false, so a caller
// can leave the kernel instead of hanging the device.
struct GridBarrier {
  unsigned int* count;   // zero-initialised
  unsigned int* gen;     // generation counter
};
__device__ __forceinline__ bool grid_barrier(GridBarrier b, unsigned int nblocks, int* err,
                                             long long limit = (1LL << 26)) {
  __syncthreads();
  bool ok = true;
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = b.gen;
    unsigned int g = *vgen;
    __threadfence();
    unsigned int arrived = atomicAdd(b.count, 1u) + 1u;
    if (arrived == nblocks) {
      atomicExch(b.count, 0u);
      __threadfence();
      atomicAdd(b.gen, 1u);
    } else {
      long long polls = 0;
      while (*vgen == g) {
        if (++polls > limit || *(volatile int*)err == DEV_ERR_TIMEOUT) {
          atomicExch(err, DEV_ERR_TIMEOUT);
          ok = false;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  // every thread learns whether the barrier completed
  __shared__ int s_ok;
  if (threadIdx.x == 0) s_ok = ok ? 1 : 0;
  __syncthreads();
  ok = s_ok != 0;
  __syncthreads();
  return ok;
}

#define CHFSI_CUDA_TRY(expr)                                 \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return chfsi_cuda_error(_e, #expr); \
  } while (0)

chfsi_status chfsi_cuda_error(cudaError_t e, const char* what);

// Number of kernels this library has launched (process-wide); chfsi_kernel_launches() reads it.
void count_launch(unsigned long long n = 1);

// Cooperative launch serialised against every other cooperative launch of this library on
// the device (an event chain across streams): kernels whose blocks wait on one another at a
// grid barrier must never share the device with another such kernel, or each could hold
// SMs the other's unscheduled blocks need.
cudaError_t coop_launch(const void* fn, dim3 grid, dim3 block, void** args, cudaStream_t s);
cudaError_t coop_launch_smem(const void* fn, dim3 grid, dim3 block, void** args, size_t smem, cudaStream_t s);
