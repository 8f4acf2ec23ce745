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
// sequence p_0 = 1, p_i = (alpha_i - x) p_{i-1} - beta_{i-1}^2 p_{i-2} (no division: FP64
// division is a long latency chain here); rescaled by 2^-256 when it grows past 2^256.
__device__ int sturm_count(int m, const double* al, const double* be, double x) {
  int cnt = 0;
  double pm2 = 0.0, pm1 = 1.0;
  for (int i = 0; i < m; ++i) {
    const double b2 = (i > 0) ? be[i - 1] * be[i - 1] : 0.0;
    double p = (al[i] - x) * pm1 - b2 * pm2;
    if (p == 0.0) p = -1e-300 * (pm1 < 0.0 ? -1.0 : 1.0);   // a zero takes the sign opposite to p_{i-1}
    if ((p < 0.0) != (pm1 < 0.0)) ++cnt;
    pm2 = pm1;
    pm1 = p;
    if (fabs(pm1) > 0x1.0p256) {
      pm1 *= 0x1.0p-256;
      pm2 *= 0x1.0p-256;
    }
  }
  return cnt;
}

// index-th smallest eigenvalue (0-based) by warp multisection: each step the 32 lanes count
// at 32 interior points of [lo, hi] and the bracket shrinks 33-fold (the whole warp calls it)
__device__ double tridiag_eig_multisect(int m, const double* al, const double* be, int index) {
  const int lane = threadIdx.x & 31;
  double lo = al[0], hi = al[0];
  for (int i = 0; i < m; ++i) {
    const double r = ((i > 0) ? fabs(be[i - 1]) : 0.0) + ((i + 1 < m) ? fabs(be[i]) : 0.0);
    lo = fmin(lo, al[i] - r);
    hi = fmax(hi, al[i] + r);
  }
  lo -= 1e-300;
  for (int it = 0; it < 14; ++it) {
    const double h = (hi - lo) / 33.0;
    const double x = lo + h * (lane + 1);
    const bool below = sturm_count(m, al, be, x) <= index;   // eigenvalue index is >= x
    const unsigned bal = __ballot_sync(0xffffffffu, below);
    const int j = __popc(bal);                              // points at or below the eigenvalue
    const double nlo = (j == 0) ? lo : lo + h * j;
    const double nhi = (j == 32) ? hi : lo + h * (j + 1);
    if (!(nhi - nlo < hi - lo)) break;
    lo = nlo;
    hi = nhi;
  }
  return 0.5 * (lo + hi);
}

__global__ void lanczos_bounds_kernel(int steps, int n, int k, const double* alpha, const double* beta,
                                      double* out) {
  __shared__ double al[256], be[256], mu[256], th[256], w[256];
  const int m = steps;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    al[i] = alpha[i];
    be[i] = beta[i];
  }
  __syncthreads();
  // all Ritz values (eigenvalues of T) and the eigenvalues of its trailing block T(2:m, 2:m),
  // one warp per eigenvalue
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
  for (int idx = warp; idx < 2 * m - 1; idx += nw) {
    if (idx < m) {
      const double v = tridiag_eig_multisect(m, al, be, idx);
      if (lane == 0) mu[idx] = v;
    } else {
      const double v = tridiag_eig_multisect(m - 1, al + 1, be + 1, idx - m);
      if (lane == 0) th[idx - m] = v;
    }
  }
  __syncthreads();
  // Gauss weights w_i = z_1(mu_i)^2 = prod_j (mu_i - theta_j) / prod_{j != i} (mu_i - mu_j)
  // (the squared first component of the i-th eigenvector of T, from the interlacing
  // eigenvalues of the trailing block; positive by interlacing)
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double lg = 0.0;
    for (int j = 0; j < m - 1; ++j) lg += log(fabs(mu[i] - th[j]) + 1e-300);
    for (int j = 0; j < m; ++j)
      if (j != i) lg -= log(fabs(mu[i] - mu[j]) + 1e-300);
    w[i] = exp(lg);
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
      const double zn = ((mu_max - al[i]) * z - (i > 0 ? be[i - 1] * zm1 : 0.0)) / be[i];
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
                           double* out) {
  if (steps < 2 || steps > 256) return cudaErrorInvalidValue;
  lanczos_bounds_kernel<<<1, 1024, 0, s>>>(steps, n, k, alpha, beta, out); count_launch();
  return cudaGetLastError();
}

cudaError_t vector_degrees(cudaStream_t s, int k, const double* lam, const double* res, double a, double b,
                           double tol, int m_min, int m_max, int* deg) {
  if (k <= 0) return cudaSuccess;
  vector_degrees_kernel<<<(k + 127) / 128, 128, 0, s>>>(k, lam, res, a, b, tol, m_min, m_max, deg); count_launch();
  return cudaGetLastError();
}
