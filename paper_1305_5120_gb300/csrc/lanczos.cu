// Lanczos estimate of the spectral upper bound (Algorithm 1, line 1; the estimator of Zhou &
// Li 2011 cited in Section 3): memory-bound Hermitian GEMV plus single-CTA vector updates,
// and Sturm-sequence bisection on the small tridiagonal T.
#include <math.h>
#include "lanczos.cuh"

namespace {

__global__ void herm_gemv_kernel(int n, const cplx* __restrict__ H, long ldh, const cplx* __restrict__ v,
                                 cplx* __restrict__ w) {
  const int lane = threadIdx.x & 31;
  const long col = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
  if (col >= n) return;
  const cplx* hc = H + col * ldh;
  double re = 0.0, im = 0.0;
  for (long r = lane; r < n; r += 32) {
    cplx h = __ldg(hc + r), x = __ldg(v + r);
    // conj(h) * x
    re = fma(h.x, x.x, re);
    re = fma(h.y, x.y, re);
    im = fma(h.x, x.y, im);
    im = fma(-h.y, x.x, im);
  }
  re = warp_sum(re);
  im = warp_sum(im);
  if (lane == 0) w[col] = cmk(re, im);
}

// w = A v for a lower-triangular A (column-major): CTA (rb, cb) takes 128 rows and a chunk of
// GEMV_CHUNK columns (thread = row, coalesced column reads), writing a partial sum that
// gemv_reduce_kernel adds in a fixed order; chunks wholly above the diagonal are skipped.
constexpr int GEMV_ROWS = 128, GEMV_CHUNK = 64;
__global__ void lower_gemv_partial_kernel(int n, const cplx* __restrict__ A, long lda, const cplx* __restrict__ v,
                                          cplx* __restrict__ part) {
  const long row = blockIdx.x * (long)GEMV_ROWS + threadIdx.x;
  const int c0 = blockIdx.y * GEMV_CHUNK;
  const long rmax = blockIdx.x * (long)GEMV_ROWS + GEMV_ROWS - 1;
  double re = 0.0, im = 0.0;
  if (row < n && c0 <= rmax) {
    const int c1 = min(n, c0 + GEMV_CHUNK);
    for (int c = c0; c < c1 && c <= row; ++c) {
      const cplx a = __ldg(A + row + (long)c * lda), x = __ldg(v + c);
      re = fma(a.x, x.x, re);
      re = fma(-a.y, x.y, re);
      im = fma(a.x, x.y, im);
      im = fma(a.y, x.x, im);
    }
  }
  if (row < n) part[(long)blockIdx.y * n + row] = cmk(re, im);
}
__global__ void gemv_reduce_kernel(int n, int chunks, const cplx* part, cplx* w) {
  const long row = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (row >= n) return;
  cplx s = cmk(0.0, 0.0);
  for (int q = 0; q < chunks; ++q) s = cadd(s, part[(long)q * n + row]);
  w[row] = s;
}

__global__ void normalize_kernel(int n, cplx* v) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += cabs2(v[i]);
  s = block_sum(s, sh);
  const double inv = 1.0 / sqrt(s);
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = cscale(v[i], inv);
}

__global__ void lanczos_step_kernel(int n, int j, cplx* v, cplx* vp, cplx* w, double* alpha, double* beta) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    cplx a = v[i], b = w[i];
    s += a.x * b.x + a.y * b.y;     // Re(conj(v) w)
  }
  const double al = block_sum(s, sh);
  const double bp = (j > 0) ? beta[j - 1] : 0.0;
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    cplx x = w[i], a = v[i], p = vp[i];
    x.x -= al * a.x + bp * p.x;
    x.y -= al * a.y + bp * p.y;
    w[i] = x;
    t += cabs2(x);
  }
  const double be = sqrt(block_sum(t, sh));
  const double inv = be > 0.0 ? 1.0 / be : 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    vp[i] = v[i];
    v[i] = cscale(w[i], inv);
  }
  if (threadIdx.x == 0) {
    alpha[j] = al;
    beta[j] = be;
  }
}

// Number of eigenvalues of tridiag(beta, alpha, beta) below x: sign changes of the Sturm
// sequence p_0 = 1, p_i = (alpha_i - x) p_{i-1} - beta_{i-1}^2 p_{i-2} (b2[i] = beta_{i-1}^2,
// b2[0] = 0).  Cost model of this GPU's FP64 pipe (a warp-wide FP64 instruction, compares
// included, holds a sub-partition's FP64 unit for about 64 cycles): three FP64 instructions
// per step; the sign tests, the zero fix-up and the rescaling by 2^-256 when |p| passes 2^256
// are integer operations on the bit patterns.
__device__ int sturm_count(int m, const double* al, const double* b2, double x) {
  int cnt = 0;
  double pm2 = 0.0, pm1 = 1.0;
  for (int i = 0; i < m; ++i) {
    double p = fma(al[i] - x, pm1, -(b2[i] * pm2));
    long long pb = __double_as_longlong(p);
    const long long qb = __double_as_longlong(pm1);
    if ((pb & 0x7FFFFFFFFFFFFFFFLL) == 0) {   // a zero takes the sign opposite to p_{i-1}
      pb = (~qb & (long long)0x8000000000000000ULL) | __double_as_longlong(1e-300);
      p = __longlong_as_double(pb);
    }
    cnt += (int)(((unsigned long long)(pb ^ qb)) >> 63);
    pm2 = pm1;
    pm1 = p;
    if ((int)((pb >> 52) & 0x7FF) > 1023 + 256) {
      pm1 = scale_pow2(pm1, 256);
      pm2 = scale_pow2(pm2, 256);
    }
  }
  return cnt;
}

// index-th smallest eigenvalue (0-based) by warp multisection: each step the 32 lanes count
// at 32 interior points of [lo, hi] and the bracket shrinks 33-fold (the whole warp calls it)
__device__ double tridiag_eig_multisect(int m, const double* al, const double* be, const double* b2, int index) {
  const int lane = threadIdx.x & 31;
  double lo = al[0], hi = al[0];
  for (int i = 0; i < m; ++i) {
    const double r = ((i > 0) ? fabs(be[i - 1]) : 0.0) + ((i + 1 < m) ? fabs(be[i]) : 0.0);
    lo = fmin(lo, al[i] - r);
    hi = fmax(hi, al[i] + r);
  }
  lo -= 1e-300;
  const double cl = to_f64((float)(lane + 1));   // exact small integers without a conversion
  for (int it = 0; it < 14; ++it) {
    const double h = (hi - lo) * (1.0 / 33.0);
    const double x = fma(h, cl, lo);
    const bool below = sturm_count(m, al, b2, x) <= index;   // eigenvalue index is >= x
    const unsigned bal = __ballot_sync(0xffffffffu, below);
    const int j = __popc(bal);                                // points at or below the eigenvalue
    const double nlo = (j == 0) ? lo : fma(h, to_f64((float)j), lo);
    const double nhi = (j == 32) ? hi : fma(h, to_f64((float)(j + 1)), lo);
    if (!(nhi - nlo < hi - lo)) break;
    lo = nlo;
    hi = nhi;
  }
  return 0.5 * (lo + hi);
}

// All Ritz values mu (eigenvalues of T) and the eigenvalues theta of its trailing block
// T(2:m, 2:m): one single-warp CTA per eigenvalue, so that each search has a sub-partition's
// FP64 unit to itself.  eig[0 .. m) = mu, eig[m .. 2m-1) = theta.
__global__ void tridiag_eigs_kernel(int m, const double* alpha, const double* beta, double* eig) {
  __shared__ double al[256], be[256], b2[256];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    al[i] = alpha[i];
    be[i] = beta[i];
  }
  __syncthreads();
  const int idx = blockIdx.x;
  const int off = idx < m ? 0 : 1;   // trailing block: alpha_2.., beta_2..
  const int mm = m - off;
  for (int i = threadIdx.x; i < mm; i += blockDim.x) b2[i] = (i > 0) ? be[off + i - 1] * be[off + i - 1] : 0.0;
  __syncthreads();
  const double v = tridiag_eig_multisect(mm, al + off, be + off, b2, idx < m ? idx : idx - m);
  if (threadIdx.x == 0) eig[idx] = v;
}

// x = m 2^e kept with m in [1, 2): products of many factors without logarithms or overflow
struct MantExp {
  double m;
  int e;
};
__device__ __forceinline__ void me_mul(MantExp& a, double f) {   // f > 0, normal
  const long long b = __double_as_longlong(f);
  a.e += (int)((b >> 52) & 0x7FF) - 1023;
  a.m *= __longlong_as_double((b & 0x000FFFFFFFFFFFFFLL) | (1023LL << 52));
  const long long mb = __double_as_longlong(a.m);   // m in [1, 4): renormalise
  const int me = (int)((mb >> 52) & 0x7FF) - 1023;
  a.e += me;
  a.m = __longlong_as_double((mb & 0x000FFFFFFFFFFFFFLL) | (1023LL << 52));
}

__global__ void lanczos_bounds_kernel(int steps, int n, int k, const double* alpha, const double* beta,
                                      const double* eig, double* out) {
  __shared__ double al[256], be[256], rb[256], w[256];
  const int m = steps;
  const double* mu = eig;
  const double* th = eig + m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    al[i] = alpha[i];
    be[i] = beta[i];
    rb[i] = 1.0 / beta[i];   // reciprocals in parallel: the recurrence below then multiplies
  }
  // Gauss weights w_i = z_1(mu_i)^2 = prod_j (mu_i - theta_j) / prod_{j != i} (mu_i - mu_j)
  // (the squared first component of the i-th eigenvector of T, from the interlacing
  // eigenvalues of the trailing block; positive by interlacing), as mantissa-exponent products
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    MantExp num{1.0, 0}, den{1.0, 0};
    const double mi = mu[i];
    for (int j = 0; j < m - 1; ++j) me_mul(num, fabs(mi - th[j]) + 1e-300);
    for (int j = 0; j < m; ++j)
      if (j != i) me_mul(den, fabs(mi - mu[j]) + 1e-300);
    w[i] = ldexp(num.m / den.m, num.e - den.e);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double mu_max = mu[m - 1], mu_min = mu[0];
    // eigenvector z of T for mu_max by the three-term recurrence
    //   beta_i z_{i+1} = (mu - alpha_i) z_i - beta_{i-1} z_{i-1},  z_0 = 1 (rescaled when it
    // grows); the bound is mu_max + |beta_last| |z_last| / ||z|| (the residual norm of the
    // top Ritz pair) plus 1e-3 of the Ritz spread
    double zm1 = 0.0, z = 1.0, ss = 1.0;
    for (int i = 0; i + 1 < m; ++i) {
      const double zn = ((mu_max - al[i]) * z - (i > 0 ? be[i - 1] * zm1 : 0.0)) * rb[i];
      zm1 = z;
      z = zn;
      ss += z * z;
      if (ss > 1e200) {
        zm1 *= 1e-100;
        z *= 1e-100;
        ss *= 1e-200;
      }
    }
    out[0] = mu_max + fabs(be[m - 1]) * fabs(z) / sqrt(ss) + 1e-3 * (mu_max - mu_min);
    out[3] = mu_max;
    out[2] = mu_min;
    // first-solve a: the first Ritz value (from the second on) whose cumulative Gauss weight
    // reaches k / n -- the Lanczos density-of-states estimate of lambda_{k+1}
    double tot = 0.0;
    for (int i = 0; i < m; ++i) tot += w[i];
    const double target = (double)k / (double)n * tot;
    double cdf = w[0] + w[1];
    int j = 1;
    while (j < m - 2 && cdf < target) {
      ++j;
      cdf += w[j];
    }
    out[1] = mu[j];
  }
}

__global__ void vector_degrees_kernel(int k, const double* lam, const double* res, double a, double b, double tol,
                                      int m_min, int m_max, int* deg) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  const double e = 0.5 * (b - a), c = 0.5 * (b + a);
  const double t = fabs((lam[i] - c) / e), r = res[i];
  int m;
  if (r <= tol) m = m_min;
  else if (t <= 1.0) m = m_max;
  else {
    double rho = 1.0 / (t + sqrt(t * t - 1.0));
    double need = log(tol / r) / log(rho);
    double mc = ceil(need);
    m = mc < m_min ? m_min : (mc > m_max ? m_max : (int)mc);
  }
  deg[i] = m;
}
}  // namespace

cudaError_t herm_gemv(cudaStream_t s, int n, const cplx* H, long ldh, const cplx* v, cplx* w) {
  const long threads = 32L * n;
  herm_gemv_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(n, H, ldh, v, w); count_launch();
  return cudaGetLastError();
}

cudaError_t lower_gemv(cudaStream_t s, int n, const cplx* A, long lda, const cplx* v, cplx* w, cplx* part) {
  const int chunks = (n + GEMV_CHUNK - 1) / GEMV_CHUNK;
  dim3 grid((unsigned)((n + GEMV_ROWS - 1) / GEMV_ROWS), (unsigned)chunks);
  lower_gemv_partial_kernel<<<grid, GEMV_ROWS, 0, s>>>(n, A, lda, v, part); count_launch();
  gemv_reduce_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, chunks, part, w); count_launch();
  return cudaGetLastError();
}

cudaError_t normalize_vec(cudaStream_t s, int n, cplx* v) {
  normalize_kernel<<<1, 1024, 0, s>>>(n, v); count_launch();
  return cudaGetLastError();
}

cudaError_t lanczos_step(cudaStream_t s, int n, int j, cplx* v, cplx* v_prev, cplx* w, double* alpha,
                         double* beta) {
  lanczos_step_kernel<<<1, 1024, 0, s>>>(n, j, v, v_prev, w, alpha, beta); count_launch();
  return cudaGetLastError();
}

cudaError_t lanczos_bounds(cudaStream_t s, int steps, int n, int k, const double* alpha, const double* beta,
                           double* out, double* scratch) {
  if (steps < 2 || steps > 256) return cudaErrorInvalidValue;
  tridiag_eigs_kernel<<<2 * steps - 1, 32, 0, s>>>(steps, alpha, beta, scratch); count_launch();
  lanczos_bounds_kernel<<<1, 256, 0, s>>>(steps, n, k, alpha, beta, scratch, out); count_launch();
  return cudaGetLastError();
}

cudaError_t vector_degrees(cudaStream_t s, int k, const double* lam, const double* res, double a, double b,
                           double tol, int m_min, int m_max, int* deg) {
  if (k <= 0) return cudaSuccess;
  vector_degrees_kernel<<<(k + 127) / 128, 128, 0, s>>>(k, lam, res, a, b, tol, m_min, m_max, deg); count_launch();
  return cudaGetLastError();
}
