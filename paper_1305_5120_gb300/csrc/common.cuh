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

// FP64 <-> FP32 by integer operations on the bit patterns (no FP64-pipe conversion).
// to_f32: truncating; values whose exponent falls below FP32's normal range become zero
// (the callers scale by a power of two first, so only negligible values are flushed).
__device__ __forceinline__ float to_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF) - 1023 + 127;
  if (e <= 0) return 0.0f;
  if (e >= 255) return __uint_as_float((unsigned)((b >> 32) & 0x80000000u) | 0x7F7FFFFFu);
  return __uint_as_float((unsigned)((b >> 32) & 0x80000000u) | ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7FFFFF));
}
__device__ __forceinline__ double to_f64(float x) {   // exact for normal numbers and zero
  const unsigned u = __float_as_uint(x);
  const int e = (int)((u >> 23) & 0xFF);
  if (e == 0) return 0.0;
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e - 127 + 1023) << 52) | ((unsigned long long)(u & 0x7FFFFF) << 29);
  return __longlong_as_double((long long)b);
}
// x 2^-E for a normal x by exponent arithmetic (zero if it would leave the normal range)
__device__ __forceinline__ double scale_pow2(double x, int E) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0 || e - E <= 0) return 0.0;
  if (e - E >= 0x7FF) return x;   // not reached for the ratios used here
  return __longlong_as_double((b & ~(0x7FFLL << 52)) | ((long long)(e - E) << 52));
}
__device__ __forceinline__ long long abs_bits(double x) { return __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL; }

// Device-side error word: kernels never trap; they record a code and return.
enum { DEV_OK = 0, DEV_ERR_TIMEOUT = 1, DEV_ERR_NOT_HPD = 2, DEV_ERR_NUMERIC = 3, DEV_ERR_NO_CONV = 4 };

// Grid barrier for cooperative launches (all blocks co-resident).  One 32-bit counter, never
// reset: at every barrier block 0 adds 2^31 - (nblocks - 1) and every other block adds 1, so
// the counter's top bit flips exactly when the last block arrives; each block waits (acquire
// loads) until the top bit differs from the value its own add returned.  A block that runs
// ahead into the next barrier cannot flip the bit again before the slow ones have seen it.
// The spin is bounded: after `limit` polls it records DEV_ERR_TIMEOUT in *err and returns
// false, so a caller can leave the kernel instead of hanging the device.  The counter must be
// zeroed before the launch.
struct GridBarrier {
  unsigned int* count;
};
__device__ __forceinline__ bool grid_barrier(GridBarrier b, unsigned int nblocks, int* err,
                                             long long limit = (1LL << 26)) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    bool ok = true;
    const unsigned int add = blockIdx.x == 0 ? 0x80000000u - (nblocks - 1u) : 1u;
    __threadfence();
    const unsigned int old = atomicAdd(b.count, add);
    long long polls = 0;
    for (;;) {
      unsigned int v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(b.count) : "memory");
      if ((v ^ old) & 0x80000000u) break;
      if (++polls > limit || ((polls & 1023) == 0 && *(volatile int*)err == DEV_ERR_TIMEOUT)) {
        atomicExch(err, DEV_ERR_TIMEOUT);
        ok = false;
        break;
      }
    }
    __threadfence();
    s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  return s_ok != 0;   // every thread learns whether the barrier completed
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
