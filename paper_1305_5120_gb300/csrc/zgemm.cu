// FP64 complex GEMM on the DFMA pipe.
//
// GB300 runs FP64 at about 1.2 TFLOP/s (DFMA; the FP64 mma.sync path measured slower), so
// every FP64 product here is bound by the DFMA issue rate, not by memory: a 64 x 32 complex
// tile per 128-thread CTA with a 4 x 4 register block per thread keeps the pipe busy while
// shared-memory traffic stays far below its limit.  The same kernel serves the plain-FP64
// Chebyshev filter (Section 3, Eq. (3term), with the scaled recurrence fused into the
// epilogue), the Rayleigh-Ritz products, the reduction to standard form, the blocked
// Cholesky updates and the Ritz rotation.
#include "zgemm.cuh"

namespace {

constexpr int BM = 64, BN = 32, BK = 16, TM = 4, TN = 4, NT = 128;
static_assert((BM / TM) * (BN / TN) == NT, "thread layout");

__device__ __forceinline__ cplx load_op(const cplx* X, long ld, int op, long r, long c, long R, long Cn) {
  // element (r, c) of op(X), an R x Cn matrix; zero outside
  if (r >= R || c >= Cn) return cmk(0.0, 0.0);
  if (op == OP_N) return X[r + c * ld];
  cplx v = X[c + r * ld];
  return cmk(v.x, -v.y);
}

__device__ __forceinline__ void k_range(const GemmArgs& g, int m0, int n0, int& kb, int& ke) {
  kb = 0;
  ke = g.K;
  if (g.tri & TRI_A_LOWER) ke = min(ke, m0 + BM);
  if (g.tri & TRI_B_UPPER) ke = min(ke, n0 + BN);
  if (g.tri & TRI_A_UPPER) kb = max(kb, m0);
  if (g.tri & TRI_B_LOWER) kb = max(kb, n0);
  kb = (kb / BK) * BK;
}

__global__ void __launch_bounds__(NT) zgemm_kernel(GemmArgs g) {
  __shared__ cplx As[2][BK][BM];
  __shared__ cplx Bs[2][BK][BN];
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);   // 8 x 16 thread grid

  int kb, ke;
  k_range(g, m0, n0, kb, ke);
  // split-K: this CTA handles [kb, ke) ∩ chunk z
  if (g.splits > 1) {
    int tiles = (ke - kb + BK - 1) / BK;
    int per = (tiles + g.splits - 1) / g.splits;
    int z = blockIdx.z;
    int t0 = min(tiles, z * per), t1 = min(tiles, (z + 1) * per);
    int nkb = kb + t0 * BK, nke = min(ke, kb + t1 * BK);
    kb = nkb;
    ke = max(nkb, nke);
  }

  cplx acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = cmk(0.0, 0.0);

  // register staging for the next tile (global -> regs -> smem)
  constexpr int A_PER = BM * BK / NT;   // 8
  constexpr int B_PER = BN * BK / NT;   // 4
  cplx ra[A_PER], rb[B_PER];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int t = 0; t < A_PER; ++t) {
      int e = tid + t * NT;
      int i, kk;
      if (g.opA == OP_N) { i = e % BM; kk = e / BM; } else { kk = e % BK; i = e / BK; }
      ra[t] = (k0 + kk < ke) ? load_op(g.A, g.lda, g.opA, m0 + i, k0 + kk, g.M, g.K) : cmk(0.0, 0.0);
    }
#pragma unroll
    for (int t = 0; t < B_PER; ++t) {
      int e = tid + t * NT;
      int j, kk;
      if (g.opB == OP_N) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
      rb[t] = (k0 + kk < ke) ? load_op(g.B, g.ldb, g.opB, k0 + kk, n0 + j, g.K, g.N) : cmk(0.0, 0.0);
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int t = 0; t < A_PER; ++t) {
      int e = tid + t * NT;
      int i, kk;
      if (g.opA == OP_N) { i = e % BM; kk = e / BM; } else { kk = e % BK; i = e / BK; }
      As[buf][kk][i] = ra[t];
    }
#pragma unroll
    for (int t = 0; t < B_PER; ++t) {
      int e = tid + t * NT;
      int j, kk;
      if (g.opB == OP_N) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
      Bs[buf][kk][j] = rb[t];
    }
  };

  int buf = 0;
  if (kb < ke) {
    fetch(kb);
    stash(0);
  }
  __syncthreads();
  for (int k0 = kb; k0 < ke; k0 += BK) {
    const bool more = k0 + BK < ke;
    if (more) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      cplx a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty + i * (BM / TM)];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx + j * (BN / TN)];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) cfma(acc[i][j], a[i], b[j]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }

  // epilogue
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const long r = m0 + ty + i * (BM / TM);
    if (r >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const long c = n0 + tx + j * (BN / TN);
      if (c >= g.N) continue;
      cplx v = acc[i][j];
      if (g.splits > 1) {
        g.work[(long)blockIdx.z * g.M * g.N + r + c * (long)g.M] = v;
      } else if (g.epi == EPI_FILTER) {
        cplx y = g.Ycur[r + c * g.ldy];
        cplx o = cmk(g.fa * v.x + g.fb * y.x, g.fa * v.y + g.fb * y.y);
        if (g.fg != 0.0) {
          cplx p = g.C[r + c * g.ldc];
          o.x += g.fg * p.x;
          o.y += g.fg * p.y;
        }
        g.C[r + c * g.ldc] = o;
      } else {
        cplx o = cmul(g.alpha, v);
        if (g.beta.x != 0.0 || g.beta.y != 0.0) o = cadd(o, cmul(g.beta, g.C[r + c * g.ldc]));
        g.C[r + c * g.ldc] = o;
      }
    }
  }
}

// Sums the split-K partials in a fixed order (deterministic) and applies the epilogue.
__global__ void zgemm_splitk_reduce(GemmArgs g) {
  const long total = (long)g.M * g.N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const long r = e % g.M, c = e / g.M;
    cplx v = cmk(0.0, 0.0);
    for (int z = 0; z < g.splits; ++z) v = cadd(v, g.work[(long)z * total + e]);
    if (g.epi == EPI_FILTER) {
      cplx y = g.Ycur[r + c * g.ldy];
      cplx o = cmk(g.fa * v.x + g.fb * y.x, g.fa * v.y + g.fb * y.y);
      if (g.fg != 0.0) {
        cplx p = g.C[r + c * g.ldc];
        o.x += g.fg * p.x;
        o.y += g.fg * p.y;
      }
      g.C[r + c * g.ldc] = o;
    } else {
      cplx o = cmul(g.alpha, v);
      if (g.beta.x != 0.0 || g.beta.y != 0.0) o = cadd(o, cmul(g.beta, g.C[r + c * g.ldc]));
      g.C[r + c * g.ldc] = o;
    }
  }
}

}  // namespace

size_t zgemm_work_bytes(int M, int N, int splits) {
  return splits > 1 ? (size_t)splits * M * N * sizeof(cplx) : 0;
}

cudaError_t zgemm_launch(const GemmArgs& g0, cudaStream_t stream) {
  GemmArgs g = g0;
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (g.splits < 1) g.splits = 1;
  const long total = (long)g.M * g.N;
  const unsigned rblocks = (unsigned)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  if (g.K <= 0) {
    // empty product: only the epilogue remains (the reduce kernel with zero partials)
    g.splits = 0;
    zgemm_splitk_reduce<<<rblocks, 256, 0, stream>>>(g);
    count_launch();
    return cudaGetLastError();
  }
  dim3 grid((g.M + BM - 1) / BM, (g.N + BN - 1) / BN, g.splits);
  zgemm_kernel<<<grid, NT, 0, stream>>>(g);
  count_launch();
  if (g.splits > 1) {
    zgemm_splitk_reduce<<<rblocks, 256, 0, stream>>>(g);
    count_launch();
  }
  return cudaGetLastError();
}
