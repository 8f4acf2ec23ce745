// Blocked Cholesky (reduction of S to L L^H, Section 3), triangular inverse (for the
// two-sided transform H' = L^{-1} H L^{-H} and the back-transform x = L^{-H} y), and the
// small column kernels around Algorithm 1 (residual norms, locking gathers, random start).
#include "dense.cuh"

namespace {
constexpr int NB = 32;   // diagonal block of the blocked factorisations

// Factor the jb x jb diagonal block at A(j0, j0) in shared memory (one CTA, NB*NB threads max).
__global__ void potrf_diag_kernel(cplx* A, long lda, int j0, int jb, int* err) {
  __shared__ cplx T[NB][NB + 1];
  __shared__ int bad;
  if (*(volatile int*)err != DEV_OK) return;
  const int tid = threadIdx.x;
  for (int e = tid; e < jb * jb; e += blockDim.x) {
    int r = e % jb, c = e / jb;
    T[r][c] = A[(j0 + r) + (long)(j0 + c) * lda];
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int c = 0; c < jb; ++c) {
    if (tid == 0) {
      double p = T[c][c].x;
      if (!(p > 0.0) || !isfinite(p)) bad = 1;
      else T[c][c] = cmk(sqrt(p), 0.0);
    }
    __syncthreads();
    if (bad) break;
    const double d = T[c][c].x;
    for (int r = c + 1 + tid; r < jb; r += blockDim.x) T[r][c] = cscale(T[r][c], 1.0 / d);
    __syncthreads();
    // trailing update of the lower part: T[r][q] -= T[r][c] * conj(T[q][c]), r >= q > c
    const int m = jb - c - 1;
    for (int e = tid; e < m * m; e += blockDim.x) {
      int r = c + 1 + e % m, q = c + 1 + e / m;
      if (r >= q) T[r][q] = csub(T[r][q], cmulc(T[r][c], T[q][c]));
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) atomicExch(err, DEV_ERR_NOT_HPD);
    return;
  }
  for (int e = tid; e < jb * jb; e += blockDim.x) {
    int r = e % jb, c = e / jb;
    A[(j0 + r) + (long)(j0 + c) * lda] = (r >= c) ? T[r][c] : cmk(0.0, 0.0);
  }
}

// Rows below the diagonal block: L21 = A21 L11^{-H}, one thread per row (forward substitution
// x_c = (a_c - sum_{q<c} x_q conj(L11[c][q])) / L11[c][c]).
__global__ void potrf_panel_kernel(cplx* A, long lda, int n, int j0, int jb, const int* err) {
  __shared__ cplx Ld[NB][NB + 1];
  if (*(volatile const int*)err != DEV_OK) return;
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    int r = e % jb, c = e / jb;
    Ld[r][c] = A[(j0 + r) + (long)(j0 + c) * lda];
  }
  __syncthreads();
  const long row = (long)j0 + jb + blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (row >= n) return;
  cplx x[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    if (c < jb) {
      cplx a = A[row + (long)(j0 + c) * lda];
      for (int q = 0; q < c; ++q) a = csub(a, cmulc(x[q], Ld[c][q]));
      x[c] = cscale(a, 1.0 / Ld[c][c].x);
    }
  }
#pragma unroll
  for (int c = 0; c < NB; ++c)
    if (c < jb) A[row + (long)(j0 + c) * lda] = x[c];
}

__global__ void zero_upper_kernel(int n, cplx* A, long lda) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)n * n; e += (long)gridDim.x * blockDim.x) {
    long r = e % n, c = e / n;
    if (r < c) A[r + c * lda] = cmk(0.0, 0.0);
  }
}

// Block row i0..i0+jb of X = L^{-1}: on entry X(rows, 0:i0) holds T = L(rows, 0:i0) X(0:i0, 0:i0);
// solves L_ii Z = RHS column by column: RHS = -T for columns < i0 and the identity for the
// diagonal block (one thread per column).
__global__ void trtri_rows_kernel(const cplx* L, long ldl, cplx* X, long ldx, int i0, int jb, const int* err) {
  __shared__ cplx Ld[NB][NB + 1];
  if (*(volatile const int*)err != DEV_OK) return;
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    int r = e % jb, c = e / jb;
    Ld[r][c] = L[(i0 + r) + (long)(i0 + c) * ldl];
  }
  __syncthreads();
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= i0 + jb) return;
  cplx z[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    if (r < jb) {
      cplx rhs;
      if (col < i0) {
        cplx t = X[(i0 + r) + (long)col * ldx];
        rhs = cmk(-t.x, -t.y);
      } else {
        rhs = cmk((col - i0) == r ? 1.0 : 0.0, 0.0);
      }
      for (int q = 0; q < r; ++q) rhs = csub(rhs, cmul(Ld[r][q], z[q]));
      z[r] = cscale(rhs, 1.0 / Ld[r][r].x);
    }
  }
#pragma unroll
  for (int r = 0; r < NB; ++r)
    if (r < jb) X[(i0 + r) + (long)col * ldx] = z[r];
}

__global__ void hermitize_kernel(int n, cplx* A, long lda) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)n * n; e += (long)gridDim.x * blockDim.x) {
    long r = e % n, c = e / n;
    if (r > c) {
      cplx a = A[r + c * lda], b = A[c + r * lda];
      cplx m = cmk(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
      A[r + c * lda] = m;
      A[c + r * lda] = cconj(m);
    } else if (r == c) {
      A[r + c * lda].y = 0.0;
    }
  }
}

__global__ void gather_columns_kernel(int n, int cnt, const int* perm, const cplx* src, long lds, cplx* dst, long ldd) {
  const int j = blockIdx.y;
  if (j >= cnt) return;
  const long sc = perm[j];
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < n; r += (long)gridDim.x * blockDim.x)
    dst[r + j * ldd] = src[r + sc * lds];
}

__global__ void gather_values_kernel(int cnt, const int* perm, const double* src, double* dst) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < cnt) dst[j] = src[perm[j]];
}

__global__ void residual_kernel(int n, const cplx* Z, long ldz, const cplx* Y, long ldy, const double* lam,
                                double* res, double* resabs) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  const double l = lam[j];
  double num = 0.0, den = 0.0;
  for (long r = threadIdx.x; r < n; r += blockDim.x) {
    cplx z = Z[r + j * ldz], y = Y[r + j * ldy];
    cplx d = cmk(z.x - l * y.x, z.y - l * y.y);
    num += cabs2(d);
    den += cabs2(z);
  }
  num = block_sum(num, sh);
  den = block_sum(den, sh);
  if (threadIdx.x == 0) {
    double a = sqrt(num), b = sqrt(den);
    resabs[j] = a;
    res[j] = a / fmax(b, 1e-300);
  }
}

__global__ void rayleigh_quotient_kernel(int n, const cplx* Y, long ldy, const cplx* Z, long ldz, double* lam) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  double acc = 0.0;
  for (long r = threadIdx.x; r < n; r += blockDim.x) {
    cplx y = Y[r + j * ldy], z = Z[r + j * ldz];
    acc += y.x * z.x + y.y * z.y;   // Re(conj(y) z)
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) lam[j] = acc;
}

__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double splitmix_unit(unsigned long long seed, unsigned long long i) {
  return (double)(splitmix64_at(seed, i) >> 11) * 0x1.0p-53 - 0.5;
}

__global__ void splitmix_block_kernel(int n, int k, unsigned long long seed, unsigned long long off, cplx* Y, long ldy) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)n * k; e += (long)gridDim.x * blockDim.x) {
    long r = e % n, c = e / n;
    unsigned long long idx = off + 2ull * (unsigned long long)(c * n + r);
    Y[r + c * ldy] = cmk(splitmix_unit(seed, idx), splitmix_unit(seed, idx + 1));
  }
}

__global__ void copy_block_kernel(int n, int k, const cplx* src, long lds, cplx* dst, long ldd) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)n * k; e += (long)gridDim.x * blockDim.x) {
    long r = e % n, c = e / n;
    dst[r + c * ldd] = src[r + c * lds];
  }
}

unsigned grid_for(long total, int threads = 256, long cap = 152 * 16) {
  long b = (total + threads - 1) / threads;
  if (b < 1) b = 1;
  return (unsigned)(b < cap ? b : cap);
}
}  // namespace

cudaError_t chol_lower(cudaStream_t s, int n, cplx* A, long lda, int* err) {
  for (int j0 = 0; j0 < n; j0 += NB) {
    const int jb = min(NB, n - j0);
    if (j0 > 0) {
      // A(j0:n, j0:j0+jb) -= L(j0:n, 0:j0) L(j0:j0+jb, 0:j0)^H
      GemmArgs g{};
      g.M = n - j0; g.N = jb; g.K = j0;
      g.opA = OP_N; g.opB = OP_C; g.tri = TRI_NONE;
      g.A = A + j0; g.lda = lda;
      g.B = A + j0; g.ldb = lda;
      g.C = A + j0 + (long)j0 * lda; g.ldc = lda;
      g.alpha = cmk(-1.0, 0.0); g.beta = cmk(1.0, 0.0);
      g.epi = EPI_GEMM; g.splits = 1;
      cudaError_t e = zgemm_launch(g, s);
      if (e != cudaSuccess) return e;
    }
    potrf_diag_kernel<<<1, 256, 0, s>>>(A, lda, j0, jb, err); count_launch();
    const int rows = n - j0 - jb;
    if (rows > 0) potrf_panel_kernel<<<(rows + 127) / 128, 128, 0, s>>>(A, lda, n, j0, jb, err); count_launch();
  }
  zero_upper_kernel<<<grid_for((long)n * n), 256, 0, s>>>(n, A, lda); count_launch();
  return cudaGetLastError();
}

cudaError_t trtri_lower(cudaStream_t s, int n, const cplx* L, long ldl, cplx* X, long ldx, int* err) {
  cudaError_t e = cudaMemsetAsync(X, 0, sizeof(cplx) * (size_t)ldx * n, s);
  if (e != cudaSuccess) return e;
  for (int i0 = 0; i0 < n; i0 += NB) {
    const int jb = min(NB, n - i0);
    if (i0 > 0) {
      // T = L(i0:i0+jb, 0:i0) X(0:i0, 0:i0), X lower triangular -> write into X(i0:i0+jb, 0:i0)
      GemmArgs g{};
      g.M = jb; g.N = i0; g.K = i0;
      g.opA = OP_N; g.opB = OP_N; g.tri = TRI_B_LOWER;
      g.A = L + i0; g.lda = ldl;
      g.B = X; g.ldb = ldx;
      g.C = X + i0; g.ldc = ldx;
      g.alpha = cmk(1.0, 0.0); g.beta = cmk(0.0, 0.0);
      g.epi = EPI_GEMM; g.splits = 1;
      e = zgemm_launch(g, s);
      if (e != cudaSuccess) return e;
    }
    const int cols = i0 + jb;
    trtri_rows_kernel<<<(cols + 127) / 128, 128, 0, s>>>(L, ldl, X, ldx, i0, jb, err); count_launch();
  }
  return cudaGetLastError();
}

cudaError_t hermitize(cudaStream_t s, int n, cplx* A, long lda) {
  hermitize_kernel<<<grid_for((long)n * n), 256, 0, s>>>(n, A, lda); count_launch();
  return cudaGetLastError();
}

cudaError_t gather_columns(cudaStream_t s, int n, int cnt, const int* perm, const cplx* src, long lds, cplx* dst,
                           long ldd) {
  if (cnt <= 0) return cudaSuccess;
  dim3 grid((unsigned)min((n + 255) / 256, 64), (unsigned)cnt);
  gather_columns_kernel<<<grid, 256, 0, s>>>(n, cnt, perm, src, lds, dst, ldd); count_launch();
  return cudaGetLastError();
}

cudaError_t gather_values(cudaStream_t s, int cnt, const int* perm, const double* src, double* dst) {
  if (cnt <= 0) return cudaSuccess;
  gather_values_kernel<<<(cnt + 255) / 256, 256, 0, s>>>(cnt, perm, src, dst); count_launch();
  return cudaGetLastError();
}

cudaError_t residual_norms(cudaStream_t s, int n, int k, const cplx* Z, long ldz, const cplx* Y, long ldy,
                           const double* lam, double* res, double* resabs) {
  if (k <= 0) return cudaSuccess;
  residual_kernel<<<k, 256, 0, s>>>(n, Z, ldz, Y, ldy, lam, res, resabs); count_launch();
  return cudaGetLastError();
}

cudaError_t rayleigh_quotients(cudaStream_t s, int n, int k, const cplx* Y, long ldy, const cplx* Z, long ldz,
                               double* lam) {
  if (k <= 0) return cudaSuccess;
  rayleigh_quotient_kernel<<<k, 256, 0, s>>>(n, Y, ldy, Z, ldz, lam); count_launch();
  return cudaGetLastError();
}

cudaError_t splitmix_block(cudaStream_t s, int n, int k, unsigned long long seed, unsigned long long stream,
                           cplx* Y, long ldy) {
  splitmix_block_kernel<<<grid_for((long)n * k), 256, 0, s>>>(n, k, seed, stream << 40, Y, ldy); count_launch();
  return cudaGetLastError();
}

cudaError_t copy_block(cudaStream_t s, int n, int k, const cplx* src, long lds, cplx* dst, long ldd) {
  if (n <= 0 || k <= 0) return cudaSuccess;
  copy_block_kernel<<<grid_for((long)n * k), 256, 0, s>>>(n, k, src, lds, dst, ldd); count_launch();
  return cudaGetLastError();
}
