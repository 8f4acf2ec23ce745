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

// upper triangle <- conjugate of the lower one, diagonal made real
__global__ void herm_from_lower_kernel(int n, cplx* A, long lda) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)n * n; e += (long)gridDim.x * blockDim.x) {
    const long r = e % n, c = e / n;
    if (r < c) A[r + c * lda] = cconj(A[c + r * lda]);
    else if (r == c) A[r + c * lda].y = 0.0;
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
                                double* res, double* resabs, double floor) {
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
    res[j] = a / fmax(fmax(b, floor), 1e-300);
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
    // 32 rows per CTA: the per-row solves are FP64-latency bound, so spread them over SMs
    if (rows > 0) {
      potrf_panel_kernel<<<(rows + 31) / 32, 32, 0, s>>>(A, lda, n, j0, jb, err);
      count_launch();
    }
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
    trtri_rows_kernel<<<(cols + 31) / 32, 32, 0, s>>>(L, ldl, X, ldx, i0, jb, err); count_launch();
  }
  return cudaGetLastError();
}

cudaError_t hermitize(cudaStream_t s, int n, cplx* A, long lda) {
  hermitize_kernel<<<grid_for((long)n * n), 256, 0, s>>>(n, A, lda); count_launch();
  return cudaGetLastError();
}

cudaError_t herm_from_lower(cudaStream_t s, int n, cplx* A, long lda) {
  herm_from_lower_kernel<<<grid_for((long)n * n), 256, 0, s>>>(n, A, lda); count_launch();
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
                           const double* lam, double* res, double* resabs, double floor) {
  if (k <= 0) return cudaSuccess;
  residual_kernel<<<k, 256, 0, s>>>(n, Z, ldz, Y, ldy, lam, res, resabs, floor); count_launch();
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

// ---- small Cholesky + inverse in one cooperative launch ----------------------------------
// The k x k Gram matrices of CholQR (k = nev + nex) are too small for a launch-per-block
// factorisation to keep more than a few SMs busy.  Here every grid barrier separates the
// three phases of a block step -- the 32 x 32 diagonal factor and its inverse (one CTA), the
// panel L21 = A21 L11^{-H} (one warp per row), the trailing update of the lower triangle (all
// threads) -- and then the block rows of X = L^{-1}.  The kernel is written for a real type
// T: double (FP64 factors, the reduction of S and exact QR) and float (the first pass of the
// in-solve QR, whose Gram matrix is column-scaled and well conditioned).
//
// Cost model of this GPU's FP64 pipe: a warp-wide FP64 instruction occupies a
// sub-partition's FP64 unit for about 64 cycles whatever the number of active lanes, and a
// division or square root costs 400-700 cycles.  So the pivot's rsqrt is taken by one thread
// and shared, the diagonal block's trailing update enumerates the lower triangle densely, and
// the dot products are split over eight accumulators.
namespace {
template <typename T> struct Cx;
template <> struct Cx<double> {
  typedef double2 C;
  static __device__ __forceinline__ C mk(double a, double b) { return make_double2(a, b); }
  static __device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
};
template <> struct Cx<float> {
  typedef float2 C;
  static __device__ __forceinline__ C mk(float a, float b) { return make_float2(a, b); }
  static __device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
};
template <typename C> __device__ __forceinline__ C xadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C xsub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C, typename T> __device__ __forceinline__ C xscale(C a, T s) { C r; r.x = a.x * s; r.y = a.y * s; return r; }
template <typename C> __device__ __forceinline__ C xmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __device__ __forceinline__ C xmulc(C a, C b) {   // a conj(b)
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
template <typename C> __device__ __forceinline__ C xzero() { C r; r.x = 0; r.y = 0; return r; }

template <typename T>
struct CholInvArgs {
  typedef typename Cx<T>::C C;
  int k;
  C* A;
  C* X;
  C* Dinv;           // nb blocks of NB x NB: inverses of the diagonal blocks
  C* Tmp;            // NB x k staging of one block row of X
  GridBarrier bar;
  int* err;
  int* fail;
};

constexpr int ACC = 8;

// The w x w (w <= 32) diagonal block at (j0, j0), by one CTA of 256 threads in shared memory:
// L (lower) into A, L^{-1} into X's diagonal block and into Dinv.
template <typename T>
__device__ void diag_factor_cta(typename Cx<T>::C* A, typename Cx<T>::C* X, typename Cx<T>::C* Dinv, int k, int j0,
                                int w, int* fail, int* err, typename Cx<T>::C (*Tm)[NB + 1],
                                typename Cx<T>::C (*Ti)[NB + 1], T* invd, int* bad, T* s_inv) {
  typedef typename Cx<T>::C C;
  const int tid = threadIdx.x;
  for (int e = tid; e < w * w; e += blockDim.x) {
    const int r = e % w, c = e / w;
    Tm[r][c] = A[(j0 + r) + (long)(j0 + c) * k];
  }
  if (tid == 0) *bad = 0;
  __syncthreads();
  for (int c = 0; c < w; ++c) {
    if (tid == 0) {   // the pivot's rsqrt once, shared through shared memory
      const T p = Tm[c][c].x;
      const bool ok = p > (T)0 && isfinite(p);
      const T inv = ok ? Cx<T>::rsq(p) : (T)1;
      *s_inv = inv;
      if (!ok) *bad = 1;
      Tm[c][c] = Cx<T>::mk(p * inv, (T)0);
      invd[c] = inv;
    }
    __syncthreads();
    if (*bad) break;
    const T inv = *s_inv;
    for (int r = c + 1 + tid; r < w; r += blockDim.x) Tm[r][c] = xscale(Tm[r][c], inv);
    __syncthreads();
    // rank-1 update of the lower triangle of the trailing m x m block, enumerated densely
    const int m = w - c - 1;
    for (int e = tid; e < m * (m + 1) / 2; e += blockDim.x) {
      int q = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);   // column within the triangle
      while (q * (q + 1) / 2 > e) --q;
      while ((q + 1) * (q + 2) / 2 <= e) ++q;
      const int rr = e - q * (q + 1) / 2;                              // rr <= q
      // element (row c + 1 + (m - 1 - rr), col c + 1 + (m - 1 - q)): row >= col
      const int row = c + 1 + (m - 1 - rr), col = c + 1 + (m - 1 - q);
      Tm[row][col] = xsub(Tm[row][col], xmulc(Tm[row][c], Tm[col][c]));
    }
    __syncthreads();
  }
  __syncthreads();
  if (*bad) {
    if (tid == 0) {
      *fail = 1;
      atomicExch(err, DEV_ERR_NOT_HPD);
    }
    return;
  }
  // Ti = Tm^{-1} row by row: Ti[r][c] = (delta_rc - sum_{c<=q<r} Tm[r][q] Ti[q][c]) invd[r];
  // 8 threads per column split the sum (shuffle reduction), 32 columns per pass
  const int c = tid >> 3, part = tid & 7;
  for (int r = 0; r < w; ++r) {
    C sacc = xzero<C>();
    if (c < w)
      for (int q = c + part; q < r; q += 8) sacc = xadd(sacc, xmul(Tm[r][q], Ti[q][c]));
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      sacc.x += __shfl_xor_sync(0xffffffffu, sacc.x, o);
      sacc.y += __shfl_xor_sync(0xffffffffu, sacc.y, o);
    }
    if (part == 0 && c < w) {
      const T d = (r == c) ? (T)1 : (T)0;
      Ti[r][c] = (r < c) ? xzero<C>() : Cx<T>::mk((d - sacc.x) * invd[r], -sacc.y * invd[r]);
    }
    __syncthreads();
  }
  for (int e = tid; e < w * w; e += blockDim.x) {
    const int r = e % w, cc = e / w;
    A[(j0 + r) + (long)(j0 + cc) * k] = (r >= cc) ? Tm[r][cc] : xzero<C>();
    if (X) X[(j0 + r) + (long)(j0 + cc) * k] = Ti[r][cc];
    Dinv[r + cc * NB] = Ti[r][cc];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) chol_inv_kernel(CholInvArgs<T> g) {
  typedef typename Cx<T>::C C;
  __shared__ C Tm[NB][NB + 1];
  __shared__ C Ti[NB][NB + 1];
  __shared__ T invd[NB];
  __shared__ T s_inv;
  __shared__ int bad;
  const int k = g.k, nb = (k + NB - 1) / NB;
  const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const long nth = (long)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const long wid = tid >> 5, nwarps = nth >> 5;
  for (int jb = 0; jb < nb; ++jb) {
    const int j0 = jb * NB, w = min(NB, k - j0);
    if (blockIdx.x == 0)
      diag_factor_cta<T>(g.A, g.X, g.Dinv + (long)jb * NB * NB, k, j0, w, g.fail, g.err, Tm, Ti, invd, &bad, &s_inv);
    if (!grid_barrier(g.bar, gridDim.x, g.err)) return;
    if (*(volatile int*)g.fail) return;
    // panel: rows below, L[r, j0+c] = sum_q A[r, j0+q] conj(Ti[c][q])  (one warp per row,
    // lane c; eight interleaved accumulators)
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      const int r = e % w, c = e / w;
      Ti[r][c] = g.Dinv[(long)jb * NB * NB + r + c * NB];
    }
    __syncthreads();
    for (long row = j0 + w + wid; row < k; row += nwarps) {
      const C a = lane < w ? g.A[row + (long)(j0 + lane) * k] : xzero<C>();
      C acc[ACC];
#pragma unroll
      for (int t = 0; t < ACC; ++t) acc[t] = xzero<C>();
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        C aq;
        aq.x = __shfl_sync(0xffffffffu, a.x, q);
        aq.y = __shfl_sync(0xffffffffu, a.y, q);
        if (lane < w && q <= lane) acc[q % ACC] = xadd(acc[q % ACC], xmulc(aq, Ti[lane][q]));
      }
#pragma unroll
      for (int t = 1; t < ACC; ++t) acc[0] = xadd(acc[0], acc[t]);
      if (lane < w) g.A[row + (long)(j0 + lane) * k] = acc[0];
    }
    if (!grid_barrier(g.bar, gridDim.x, g.err)) return;
    // trailing update of the lower triangle
    const int t0 = j0 + w, m = k - t0;
    for (long e = tid; e < (long)m * m; e += nth) {
      const int r = t0 + (int)(e % m), c = t0 + (int)(e / m);
      if (r < c) continue;
      C acc[ACC];
#pragma unroll
      for (int t = 0; t < ACC; ++t) acc[t] = xzero<C>();
#pragma unroll
      for (int q = 0; q < NB; ++q)
        if (q < w) acc[q % ACC] = xadd(acc[q % ACC], xmulc(g.A[r + (long)(j0 + q) * k], g.A[c + (long)(j0 + q) * k]));
#pragma unroll
      for (int t = 1; t < ACC; ++t) acc[0] = xadd(acc[0], acc[t]);
      g.A[r + (long)c * k] = xsub(g.A[r + (long)c * k], acc[0]);
    }
    if (!grid_barrier(g.bar, gridDim.x, g.err)) return;
  }
  // strictly upper triangle of L
  for (long e = tid; e < (long)k * k; e += nth) {
    const long r = e % k, c = e / k;
    if (r < c) g.A[e] = xzero<C>();
  }
  if (!g.X) return;   // factor only
  // block rows of X = L^{-1}: X(i,0:i0) = -Ti (L(i,0:i0) X(0:i0,0:i0))
  for (int ib = 1; ib < nb; ++ib) {
    const int i0 = ib * NB, w = min(NB, k - i0);
    for (long e = tid; e < (long)w * i0; e += nth) {
      const int r = (int)(e % w), c = (int)(e / w);
      C acc[ACC];
#pragma unroll
      for (int t = 0; t < ACC; ++t) acc[t] = xzero<C>();
      int q = c;
      for (; q + ACC <= i0; q += ACC) {
#pragma unroll
        for (int t = 0; t < ACC; ++t)
          acc[t] = xadd(acc[t], xmul(g.A[(i0 + r) + (long)(q + t) * k], g.X[(q + t) + (long)c * k]));
      }
      for (; q < i0; ++q) acc[0] = xadd(acc[0], xmul(g.A[(i0 + r) + (long)q * k], g.X[q + (long)c * k]));
#pragma unroll
      for (int t = 1; t < ACC; ++t) acc[0] = xadd(acc[0], acc[t]);
      g.X[(i0 + r) + (long)c * k] = acc[0];
    }
    if (!grid_barrier(g.bar, gridDim.x, g.err)) return;
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      const int r = e % w, c = e / w;
      Ti[r][c] = g.Dinv[(long)ib * NB * NB + r + c * NB];
    }
    __syncthreads();
    // X(i0 + r, c) = -sum_{q<=r} Ti[r][q] T(q, c): one thread per (r, c), eight accumulators
    for (long e = tid; e < (long)w * i0; e += nth) {
      const int r = (int)(e % w);
      const long c = e / w;
      C acc[ACC];
#pragma unroll
      for (int t = 0; t < ACC; ++t) acc[t] = xzero<C>();
#pragma unroll
      for (int q = 0; q < NB; ++q)
        if (q <= r) acc[q % ACC] = xadd(acc[q % ACC], xmul(Ti[r][q], g.X[(i0 + q) + c * k]));
#pragma unroll
      for (int t = 1; t < ACC; ++t) acc[0] = xadd(acc[0], acc[t]);
      g.Tmp[(long)r + c * NB] = acc[0];
    }
    if (!grid_barrier(g.bar, gridDim.x, g.err)) return;
    for (long e = tid; e < (long)w * i0; e += nth) {
      const int r = (int)(e % w);
      const long c = e / w;
      const C v = g.Tmp[(long)r + c * NB];
      g.X[(i0 + r) + c * k] = Cx<T>::mk(-v.x, -v.y);
    }
    if (!grid_barrier(g.bar, gridDim.x, g.err)) return;
  }
}

int chol_inv_blocks() {
  static int cap = 0;
  if (cap == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cap = sms;   // one CTA per SM (co-resident for the grid barrier)
  }
  return cap;
}

template <typename T>
cudaError_t chol_inv_launch(cudaStream_t s, int k, typename Cx<T>::C* A, typename Cx<T>::C* X, void* work, int* err) {
  typedef typename Cx<T>::C C;
  if (k <= 0) return cudaSuccess;
  if (k > CHOL_INV_KMAX) return cudaErrorInvalidValue;
  const int nb = (k + NB - 1) / NB;
  CholInvArgs<T> g{};
  g.k = k;
  g.A = A;
  g.X = X;
  g.Dinv = (C*)work;
  g.Tmp = g.Dinv + (size_t)nb * NB * NB;
  unsigned* tail = (unsigned*)(g.Tmp + (size_t)NB * k);
  g.bar.count = tail;
  g.fail = (int*)(tail + 2);
  g.err = err;
  cudaError_t e = cudaMemsetAsync(tail, 0, 16, s);
  if (e == cudaSuccess && X) e = cudaMemsetAsync(X, 0, sizeof(C) * (size_t)k * k, s);
  if (e != cudaSuccess) return e;
  void* args[] = {&g};
  e = coop_launch((const void*)chol_inv_kernel<T>, dim3(chol_inv_blocks()), dim3(256), args, s);
  count_launch();
  return e;
}
}  // namespace

size_t chol_inv_work_bytes(int k) {
  const int nb = (k + NB - 1) / NB;
  return sizeof(cplx) * ((size_t)nb * NB * NB + (size_t)NB * k) + 64;
}

cudaError_t chol_inv_small(cudaStream_t s, int k, cplx* A, cplx* X, void* work, int* err) {
  return chol_inv_launch<double>(s, k, A, X, work, err);
}
cudaError_t chol_inv_small_f32(cudaStream_t s, int k, float2* A, float2* X, void* work, int* err) {
  return chol_inv_launch<float>(s, k, A, X, work, err);
}
