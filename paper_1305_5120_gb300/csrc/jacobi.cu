// Reduced eigenproblem of Rayleigh-Ritz (Algorithm 1: "Solving reduced problem G w = lam w";
// the paper used the parallel MRRR solver of its library).  On the GPU a parallel cyclic
// Jacobi is used instead: in each round the k/2 disjoint index pairs of a round-robin
// schedule rotate at once, and since the combined transform U is block diagonal over the
// pairs, every 2 x 2 block (P, R) of G is updated independently as U_P^H G_PR U_R, so one
// pass over G per round suffices.  Rounds are separated by a bounded grid barrier inside a
// single cooperative launch.  Near-diagonal G (later outer iterations and sequence solves)
// converges in one or two sweeps.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "jacobi.cuh"

namespace {

struct Rot {
  cplx upp, upq, uqp, uqq;   // U restricted to (p, q): column p = (upp, uqp), column q = (upq, uqq)
  int p, q, on;
  int pad;
};

struct JacobiArgs {
  int k, kk;
  cplx* A;
  cplx* V;
  Rot* rot;
  int* rot_count;     // per sweep
  double* fro;
  GridBarrier bar;
  int* err;
  int* sweeps;
  int* rounds;        // rounds executed (every round of a sweep updates the whole matrix)
  int max_sweeps;
};

__device__ __forceinline__ int rr_slot(int x, int r, int kk) { return x == 0 ? 0 : 1 + (x - 1 + r) % (kk - 1); }

__global__ void fro_kernel(int k, const cplx* A, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long e = threadIdx.x; e < (long)k * k; e += blockDim.x) s += cabs2(A[e]);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *out = sqrt(s);
}

__global__ void __launch_bounds__(256) jacobi_kernel(JacobiArgs g) {
  const int k = g.k, kk = g.kk, np = kk / 2;
  const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const long nth = (long)gridDim.x * blockDim.x;
  const double thresh = 2.220446049250313e-16 * (*g.fro);
  for (long e = tid; e < (long)k * k; e += nth) g.V[e] = cmk((e % k) == (e / k) ? 1.0 : 0.0, 0.0);
  int sweep = 0;
  bool converged = false;
  for (; sweep < g.max_sweeps && !converged; ++sweep) {
    for (int r = 0; r < kk - 1; ++r) {
      // phase 1: rotation of each pair from the current 2 x 2 diagonal block
      for (long j = tid; j < np; j += nth) {
        int p = rr_slot((int)j, r, kk), q = rr_slot(kk - 1 - (int)j, r, kk);
        if (p > q) { int t = p; p = q; q = t; }
        Rot R;
        R.p = p; R.q = q; R.on = 0;
        R.upp = cmk(1, 0); R.uqq = cmk(1, 0); R.upq = cmk(0, 0); R.uqp = cmk(0, 0);
        if (q < k) {
          cplx apq = g.A[p + (long)q * k];
          double ar = sqrt(cabs2(apq));
          if (ar > thresh) {
            double app = g.A[p + (long)p * k].x, aqq = g.A[q + (long)q * k].x;
            cplx ph = cmk(apq.x / ar, apq.y / ar);
            double tau = (aqq - app) / (2.0 * ar);
            double t = (tau < 0.0 ? -1.0 : 1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
            R.upp = cmk(c, 0.0);
            R.uqp = cmk(-s * ph.x, s * ph.y);     // -s conj(ph)
            R.upq = cmk(s, 0.0);
            R.uqq = cmk(c * ph.x, -c * ph.y);     // c conj(ph)
            R.on = 1;
            atomicAdd(&g.rot_count[sweep], 1);
          }
        }
        g.rot[j] = R;
      }
      if (!grid_barrier(g.bar, gridDim.x, g.err)) return;
      // phase 2: G_PR <- U_P^H G_PR U_R for all block pairs, and V_R <- V_R U_R
      const long nblk = (long)np * np;
      for (long e = tid; e < nblk + (long)k * np; e += nth) {
        if (e < nblk) {
          const Rot P = g.rot[e % np], R = g.rot[e / np];
          if (!P.on && !R.on) continue;
          const bool pq_ok = P.q < k, rs_ok = R.q < k;
          cplx b00 = g.A[P.p + (long)R.p * k];
          cplx b01 = rs_ok ? g.A[P.p + (long)R.q * k] : cmk(0, 0);
          cplx b10 = pq_ok ? g.A[P.q + (long)R.p * k] : cmk(0, 0);
          cplx b11 = (pq_ok && rs_ok) ? g.A[P.q + (long)R.q * k] : cmk(0, 0);
          // T = B U_R
          cplx t00 = cadd(cmul(b00, R.upp), cmul(b01, R.uqp));
          cplx t01 = cadd(cmul(b00, R.upq), cmul(b01, R.uqq));
          cplx t10 = cadd(cmul(b10, R.upp), cmul(b11, R.uqp));
          cplx t11 = cadd(cmul(b10, R.upq), cmul(b11, R.uqq));
          // N = U_P^H T
          cplx n00 = cadd(cmul(cconj(P.upp), t00), cmul(cconj(P.uqp), t10));
          cplx n01 = cadd(cmul(cconj(P.upp), t01), cmul(cconj(P.uqp), t11));
          cplx n10 = cadd(cmul(cconj(P.upq), t00), cmul(cconj(P.uqq), t10));
          cplx n11 = cadd(cmul(cconj(P.upq), t01), cmul(cconj(P.uqq), t11));
          if (e % np == e / np && P.on) {   // diagonal block: exactly diagonal afterwards
            n00.y = 0.0; n11.y = 0.0; n01 = cmk(0, 0); n10 = cmk(0, 0);
          }
          g.A[P.p + (long)R.p * k] = n00;
          if (rs_ok) g.A[P.p + (long)R.q * k] = n01;
          if (pq_ok) g.A[P.q + (long)R.p * k] = n10;
          if (pq_ok && rs_ok) g.A[P.q + (long)R.q * k] = n11;
        } else {
          const long f = e - nblk;
          const int i = (int)(f % k);
          const Rot R = g.rot[f / k];
          if (!R.on) continue;
          cplx x = g.V[i + (long)R.p * k], y = g.V[i + (long)R.q * k];
          g.V[i + (long)R.p * k] = cadd(cmul(x, R.upp), cmul(y, R.uqp));
          g.V[i + (long)R.q * k] = cadd(cmul(x, R.upq), cmul(y, R.uqq));
        }
      }
      if (!grid_barrier(g.bar, gridDim.x, g.err)) return;
    }
    converged = (*(volatile int*)&g.rot_count[sweep]) == 0;
  }
  if (tid == 0) {
    *g.sweeps = sweep;
    *g.rounds = sweep * (kk - 1);
    if (!converged) atomicExch(g.err, DEV_ERR_NO_CONV);
  }
}

// One barrier per round (k <= 2 * JF_MAXPAIRS = 2048): A is double-buffered, and every CTA derives
// all rotations of the round from the current buffer's diagonal blocks into shared memory
// (identical in every CTA), so the rotation table needs no grid-wide publication.  All CTAs
// also count the round's rotations identically, which gives a consistent convergence test
// without atomics.  Each round reads A_cur and writes every 2 x 2 block of A_next.
//
// Cost model of this GPU's FP64 pipe: one warp-wide FP64 instruction (including conversions
// to or from FP64) occupies a sub-partition's FP64 unit for about 64 cycles, whatever the
// number of active lanes.  So the rotations, which every CTA computes, keep their FP64
// instruction count low (integer tests and format moves, an FP32 start for the tangent); and
// the update computes each 2 x 2 block of the Hermitian A once (pair index a <= b),
// enumerated densely so that every warp is full, writing the mirrored block as its conjugate
// transpose.
constexpr int JF_MAXPAIRS = 1024;
struct RotS {
  double c, s;      // U = [[c, s], [-s conj(ph), c conj(ph)]] (c, s real, c^2 + s^2 = 1)
  double phx, phy;  // conj(ph), |ph| = 1
  int p, q, on, pad;
};
struct JacobiFastArgs {
  int k, kk;
  cplx* A[2];
  cplx* V;
  double* fro;
  GridBarrier bar;
  int* err;
  int* sweeps;
  int* rounds;       // rounds in which a pair rotated (each updates A and V)
  int* final_buf;
  int* offcount;     // per sweep: off-diagonal entries above the threshold after it (zeroed)
  int max_sweeps;
};


// Rotation of pair (p, q) annihilating a_pq of the current 2 x 2 diagonal block: tangent t of
// t^2 + 2 tau t - 1 = 0 (the smaller root), tau = (a_qq - a_pp) / (2 |a_pq|), c = 1 / sqrt(1 +
// t^2), s = t c, ph = a_pq / |a_pq|.  The tangent starts in FP32 (values moved between the
// formats by integer bit operations) and one FP64 Newton step, whose own reciprocal needs only
// FP32 accuracy, makes it FP64-accurate, so that the sweeps keep their quadratic convergence;
// c, s and ph come from FP64 rsqrt, so U is unitary to FP64 rounding.  About twenty FP64
// instructions in all.  A pair rotates when |a_pq| > thresh; max(|Re a_pq|, |Im a_pq|) <=
// thresh / sqrt(2), an integer test on the bit patterns, rules most others out first.  (The
// threshold eps ||A||_F sits a few rounding units of the largest entry above the rounding
// noise of the update, so it must not be tightened.)
__device__ __forceinline__ RotS make_rot(const cplx* A, int k, int p, int q, long long thr_bits, double thresh2) {
  RotS R;
  if (p > q) { int t = p; p = q; q = t; }
  R.p = p; R.q = q; R.on = 0; R.pad = 0;
  R.c = 1.0; R.s = 0.0; R.phx = 1.0; R.phy = 0.0;
  if (q < k) {
    const cplx apq = A[p + (long)q * k];
    const double ar2 = (abs_bits(apq.x) > thr_bits || abs_bits(apq.y) > thr_bits) ? fma(apq.x, apq.x, apq.y * apq.y) : 0.0;
    if (ar2 > thresh2) {
      const double inv_r = rsqrt(ar2);
      const double d = A[q + (long)q * k].x - A[p + (long)p * k].x;
      const double taud = d * scale_pow2(inv_r, 1);            // (a_qq - a_pp) / (2 |a_pq|)
      const float tau = to_f32(taud);
      const float tf = (tau < 0.f ? -1.f : 1.f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
      double t = to_f64(tf);
      const double f = fma(t, fma(2.0, taud, t), -1.0);
      t = fma(-f, to_f64(0.5f / (tf + tau)), t);
      const double c = rsqrt(fma(t, t, 1.0));
      R.c = c;
      R.s = t * c;
      R.phx = apq.x * inv_r;
      R.phy = -(apq.y * inv_r);
      R.on = 1;
    }
  }
  return R;
}

__global__ void __launch_bounds__(256) jacobi_fast_kernel(JacobiFastArgs g) {
  extern __shared__ RotS rot[];   // kk / 2 rotations of the round
  __shared__ int s_on;
  const int k = g.k, kk = g.kk, np = kk / 2;
  const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const long nth = (long)gridDim.x * blockDim.x;
  // rotation threshold thresh = eps ||A||_F: its square, and thresh / sqrt(2) as a bit pattern
  const double thresh = 2.220446049250313e-16 * (*g.fro);
  const double thresh2 = thresh * thresh;
  const long long thr_bits = abs_bits(0.7071067811865476 * thresh);
  for (long e = tid; e < (long)k * k; e += nth) g.V[e] = cmk((e % k) == (e / k) ? 1.0 : 0.0, 0.0);
  const long ntri = (long)np * (np + 1) / 2;   // blocks (a, b), a <= b
  int cur = 0, sweep = 0, rounds = 0;
  bool converged = false;
  for (; sweep < g.max_sweeps && !converged; ++sweep) {
    int on_sweep = 0;
    for (int r = 0; r < kk - 1; ++r) {
      const cplx* Ac = g.A[cur];
      cplx* An = g.A[cur ^ 1];
      if (threadIdx.x == 0) s_on = 0;
      __syncthreads();
      for (int j = threadIdx.x; j < np; j += blockDim.x) {
        const RotS R = make_rot(Ac, k, rr_slot(j, r, kk), rr_slot(kk - 1 - j, r, kk), thr_bits, thresh2);
        rot[j] = R;
        if (R.on) atomicAdd(&s_on, 1);
      }
      __syncthreads();
      const int on_round = s_on;
      on_sweep += on_round;
      // no pair rotates this round: nothing changes, so every CTA (all computed the same
      // rotations from the same data) skips the copy, the buffer swap and the grid barrier
      if (on_round == 0) continue;
      ++rounds;
      for (long e = tid; e < ntri + (long)k * np; e += nth) {
        if (e < ntri) {
          // triangular index -> (a, b), a <= b: b (b + 1) / 2 <= e < (b + 1) (b + 2) / 2
          int bi = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
          while ((long)bi * (bi + 1) / 2 > e) --bi;
          while ((long)(bi + 1) * (bi + 2) / 2 <= e) ++bi;
          const int ai = (int)(e - (long)bi * (bi + 1) / 2);
          const RotS P = rot[ai], R = rot[bi];
          const bool pq_ok = P.q < k, rs_ok = R.q < k;
          cplx b00 = Ac[P.p + (long)R.p * k];
          cplx b01 = rs_ok ? Ac[P.p + (long)R.q * k] : cmk(0, 0);
          cplx b10 = pq_ok ? Ac[P.q + (long)R.p * k] : cmk(0, 0);
          cplx b11 = (pq_ok && rs_ok) ? Ac[P.q + (long)R.q * k] : cmk(0, 0);
          if (P.on || R.on) {
            // B U_R: one complex product per row (w = b_x1 conj(ph_R)) plus real scalings;
            // then U_P^H (B U_R) likewise
            cplx t00, t01, t10, t11;
            if (R.on) {
              const cplx phR = cmk(R.phx, R.phy);
              const cplx w0 = cmul(b01, phR), w1 = cmul(b11, phR);
              t00 = cmk(R.c * b00.x - R.s * w0.x, R.c * b00.y - R.s * w0.y);
              t01 = cmk(R.s * b00.x + R.c * w0.x, R.s * b00.y + R.c * w0.y);
              t10 = cmk(R.c * b10.x - R.s * w1.x, R.c * b10.y - R.s * w1.y);
              t11 = cmk(R.s * b10.x + R.c * w1.x, R.s * b10.y + R.c * w1.y);
            } else {
              t00 = b00; t01 = b01; t10 = b10; t11 = b11;
            }
            if (P.on) {
              // rows p, q -> (c t_p - s ph t_q, s t_p + c ph t_q), ph = conj of the stored phase
              const cplx phP = cmk(P.phx, -P.phy);
              const cplx v0 = cmul(phP, t10), v1 = cmul(phP, t11);
              b00 = cmk(P.c * t00.x - P.s * v0.x, P.c * t00.y - P.s * v0.y);
              b01 = cmk(P.c * t01.x - P.s * v1.x, P.c * t01.y - P.s * v1.y);
              b10 = cmk(P.s * t00.x + P.c * v0.x, P.s * t00.y + P.c * v0.y);
              b11 = cmk(P.s * t01.x + P.c * v1.x, P.s * t01.y + P.c * v1.y);
            } else {
              b00 = t00; b01 = t01; b10 = t10; b11 = t11;
            }
            if (ai == bi) {   // diagonal block: keep the diagonal real
              b00.y = 0.0;
              b11.y = 0.0;
              b10 = cconj(b01);
            }
          }
          An[P.p + (long)R.p * k] = b00;
          if (rs_ok) An[P.p + (long)R.q * k] = b01;
          if (pq_ok) An[P.q + (long)R.p * k] = b10;
          if (pq_ok && rs_ok) An[P.q + (long)R.q * k] = b11;
          if (ai != bi) {   // mirrored block: (B)^H at rows of R, columns of P
            An[R.p + (long)P.p * k] = cconj(b00);
            if (pq_ok) An[R.p + (long)P.q * k] = cconj(b10);
            if (rs_ok) An[R.q + (long)P.p * k] = cconj(b01);
            if (pq_ok && rs_ok) An[R.q + (long)P.q * k] = cconj(b11);
          }
        } else {
          const long f = e - ntri;
          const int i = (int)(f % k);
          const RotS R = rot[f / k];
          if (!R.on) continue;
          const cplx x = g.V[i + (long)R.p * k], y = g.V[i + (long)R.q * k];
          const cplx w = cmul(y, cmk(R.phx, R.phy));
          g.V[i + (long)R.p * k] = cmk(R.c * x.x - R.s * w.x, R.c * x.y - R.s * w.y);
          g.V[i + (long)R.q * k] = cmk(R.s * x.x + R.c * w.x, R.s * x.y + R.c * w.y);
        }
      }
      if (!grid_barrier(g.bar, gridDim.x, g.err)) return;
      cur ^= 1;
    }
    converged = on_sweep == 0;
    if (!converged && sweep + 1 < g.max_sweeps) {
      // Convergence test without a rotation-free sweep: a sweep in which no pair rotates
      // leaves A unchanged, so it rotates nothing exactly when no off-diagonal entry passes
      // the rotation test now.  One scan (integer pre-filter, FP64 only for candidates), one
      // counter, one grid barrier.
      const cplx* Ac = g.A[cur];
      int cnt = 0;
      for (long e = tid; e < (long)k * k; e += nth) {
        const int i = (int)(e % k), j = (int)(e / k);
        if (i >= j) continue;
        const cplx a = Ac[e];
        if ((abs_bits(a.x) > thr_bits || abs_bits(a.y) > thr_bits) && fma(a.x, a.x, a.y * a.y) > thresh2) ++cnt;
      }
      if (cnt) atomicAdd(&g.offcount[sweep], cnt);
      if (!grid_barrier(g.bar, gridDim.x, g.err)) return;
      converged = *(volatile int*)&g.offcount[sweep] == 0;
    }
  }
  if (tid == 0) {
    *g.sweeps = sweep;   // sweeps that rotated
    *g.rounds = rounds;
    *g.final_buf = cur;
    if (!converged) atomicExch(g.err, DEV_ERR_NO_CONV);
  }
}

// rank sort of the diagonal; W = V permuted, lam ascending (ties by index)
__global__ void jacobi_sort_kernel(int k, const cplx* A, const cplx* V, double* lam, cplx* W) {
  for (int i = blockIdx.x; i < k; i += gridDim.x) {
    const double li = A[i + (long)i * k].x;
    __shared__ int rank_sh;
    if (threadIdx.x == 0) rank_sh = 0;
    __syncthreads();
    int cnt = 0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
      double lj = A[j + (long)j * k].x;
      if (lj < li || (lj == li && j < i)) ++cnt;
    }
    atomicAdd(&rank_sh, cnt);
    __syncthreads();
    const int rk = rank_sh;
    if (threadIdx.x == 0) lam[rk] = li;
    for (int r = threadIdx.x; r < k; r += blockDim.x) W[r + (long)rk * k] = V[r + (long)i * k];
    __syncthreads();
  }
}

__global__ void jacobi_sort_pick_kernel(int k, const cplx* A0, const cplx* A1, const int* final_buf, const cplx* V,
                                        double* lam, cplx* W) {
  const cplx* A = (*final_buf) ? A1 : A0;
  for (int i = blockIdx.x; i < k; i += gridDim.x) {
    const double li = A[i + (long)i * k].x;
    __shared__ int rank_sh;
    if (threadIdx.x == 0) rank_sh = 0;
    __syncthreads();
    int cnt = 0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
      const double lj = A[j + (long)j * k].x;
      if (lj < li || (lj == li && j < i)) ++cnt;
    }
    atomicAdd(&rank_sh, cnt);
    __syncthreads();
    const int rk = rank_sh;
    if (threadIdx.x == 0) lam[rk] = li;
    for (int r = threadIdx.x; r < k; r += blockDim.x) W[r + (long)rk * k] = V[r + (long)i * k];
    __syncthreads();
  }
}

int coop_blocks(int needed) {
  static int cap = 0;
  if (cap == 0) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jacobi_kernel, 256, 0);
    cap = sms * (occ < 1 ? 1 : (occ > 2 ? 2 : occ));
  }
  return needed < cap ? (needed < 1 ? 1 : needed) : cap;
}
}  // namespace

size_t jacobi_work_bytes(int k) {
  const int kk = k + (k & 1);
  const int max_sweeps = 64;
  return 2 * sizeof(cplx) * (size_t)k * k + sizeof(Rot) * (size_t)(kk / 2) + sizeof(int) * max_sweeps +
         sizeof(double) * 2 + sizeof(unsigned) * 4 + 256;
}

int fast_coop_blocks() {
  static int cap = 0;
  if (cap == 0) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(jacobi_fast_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(RotS) * JF_MAXPAIRS));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jacobi_fast_kernel, 256, sizeof(RotS) * JF_MAXPAIRS);
    cap = sms * std::min(std::max(occ, 1), 1);
  }
  return cap;
}

cudaError_t jacobi_eig(cudaStream_t s, int k, cplx* G, double* lam, cplx* W, void* work, int* err, int* sweeps,
                       int* rounds) {
  if (k <= 0) return cudaSuccess;
  if (k <= 2 * JF_MAXPAIRS) {
    // one barrier per round; the second A buffer follows V in the workspace
    const int kk = k + (k & 1);
    const int max_sweeps = 64;
    char* w = (char*)work;
    JacobiFastArgs g{};
    g.k = k;
    g.kk = kk;
    g.A[0] = G;
    g.V = (cplx*)w;                 w += sizeof(cplx) * (size_t)k * k;
    g.A[1] = (cplx*)w;              w += sizeof(cplx) * (size_t)k * k;
    w += sizeof(Rot) * (size_t)(kk / 2);
    char* zero_begin = w;
    g.offcount = (int*)w;           w += sizeof(int) * max_sweeps;
    g.fro = (double*)w;             w += sizeof(double) * 2;
    unsigned* bar = (unsigned*)w;   w += sizeof(unsigned) * 4;
    g.final_buf = (int*)(bar + 2);
    g.bar.count = bar;
    g.err = err;
    g.sweeps = sweeps;
    g.rounds = rounds;
    g.max_sweeps = max_sweeps;
    cudaError_t e = cudaMemsetAsync(zero_begin, 0, (size_t)(w - zero_begin), s);
    if (e != cudaSuccess) return e;
    fro_kernel<<<1, 1024, 0, s>>>(k, G, g.fro);
    count_launch();
    void* args[] = {&g};
    e = coop_launch_smem((const void*)jacobi_fast_kernel, dim3(fast_coop_blocks()), dim3(256), args,
                         sizeof(RotS) * (size_t)(kk / 2), s);
    count_launch();
    if (e != cudaSuccess) return e;
    jacobi_sort_pick_kernel<<<k < 1024 ? k : 1024, 128, 0, s>>>(k, g.A[0], g.A[1], g.final_buf, (const cplx*)g.V, lam,
                                                                W);
    count_launch();
    return cudaGetLastError();
  }
  const int kk = k + (k & 1);
  const int max_sweeps = 64;
  char* w = (char*)work;
  JacobiArgs g{};
  g.k = k;
  g.kk = kk;
  g.A = G;
  g.V = (cplx*)w;                 w += sizeof(cplx) * (size_t)k * k;
  g.rot = (Rot*)w;                w += sizeof(Rot) * (size_t)(kk / 2);
  g.rot_count = (int*)w;          w += sizeof(int) * max_sweeps;
  g.fro = (double*)w;             w += sizeof(double) * 2;
  unsigned* bar = (unsigned*)w;
  g.bar.count = bar;
  g.err = err;
  g.sweeps = sweeps;
  g.rounds = rounds;
  g.max_sweeps = max_sweeps;
  cudaError_t e = cudaMemsetAsync(g.rot_count, 0, sizeof(int) * max_sweeps + sizeof(double) * 2 + sizeof(unsigned) * 4, s);
  if (e != cudaSuccess) return e;
  fro_kernel<<<1, 1024, 0, s>>>(k, G, g.fro); count_launch();
  if (kk < 2) {
    // 1 x 1: nothing to rotate
  }
  const long work_items = (long)(kk / 2) * (kk / 2) + (long)k * (kk / 2);
  int blocks = coop_blocks((int)((work_items + 255) / 256));
  void* args[] = {&g};
  e = coop_launch((const void*)jacobi_kernel, dim3(blocks), dim3(256), args, s);
  count_launch();
  if (e != cudaSuccess) return e;
  jacobi_sort_kernel<<<k < 1024 ? k : 1024, 128, 0, s>>>(k, G, (const cplx*)g.V, lam, W); count_launch();
  return cudaGetLastError();
}

// ---- allocation-free variant ----------------------------------------------------------------
// Some callers cannot allocate device memory: code that runs inside a host process whose
// device memory is owned and budgeted by someone else (a plugin or callback that receives
// only input and output buffers), or a serving loop that must not pay the implicit
// device-wide synchronisation of cudaMalloc/cudaFree while other streams are busy.  For
// them, chfsi_reduced_eig_noalloc keeps its scratch -- a working copy of G, the rotation
// accumulator V, the rotation table, sweep counters, the grid barrier and the error word --
// in one fixed file-scope device array sized for k <= CHFSI_NOALLOC_KMAX.  Every GPU that
// loads this library holds the array until the process exits.

namespace {
constexpr int NOALLOC_KMAX = 256;
constexpr int NOALLOC_SWEEPS = 64;
constexpr size_t NOALLOC_BYTES = 2 * sizeof(cplx) * (size_t)NOALLOC_KMAX * NOALLOC_KMAX +
                                 sizeof(Rot) * (size_t)(NOALLOC_KMAX / 2) + 1024;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_noalloc_mu;
constexpr int NOALLOC_MAX_DEVICES = 64;
void* g_noalloc_base[NOALLOC_MAX_DEVICES] = {};   // device address of the array, per device
}  // namespace

extern "C" chfsi_status chfsi_reduced_eig_noalloc(void* cuda_stream, int k, const void* G, double* lam, void* W) {
  if (k < 1 || k > NOALLOC_KMAX || !G || !lam || !W) return CHFSI_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return chfsi_cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return CHFSI_ERR_ARG;
  char* base = nullptr;
  {
    // one-time set-up per device (with that device current): the host-side name of the
    // array is not a device address, so ask the runtime for the address
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return chfsi_cuda_error(e, "cudaGetSymbolAddress");
      g_noalloc_base[dev] = p;
    }
    base = (char*)g_noalloc_base[dev];
  }
  const int kk = k + (k & 1);
  char* w = base;
  JacobiArgs g{};
  g.k = k;
  g.kk = kk;
  g.A = (cplx*)w;                 w += sizeof(cplx) * (size_t)k * k;
  g.V = (cplx*)w;                 w += sizeof(cplx) * (size_t)k * k;
  g.rot = (Rot*)w;                w += sizeof(Rot) * (size_t)(kk / 2);
  char* zero_begin = w;
  g.rot_count = (int*)w;          w += sizeof(int) * NOALLOC_SWEEPS;
  g.fro = (double*)w;             w += sizeof(double) * 2;
  unsigned* bar = (unsigned*)w;   w += sizeof(unsigned) * 4;
  g.err = (int*)w;                w += sizeof(int);
  g.sweeps = (int*)w;             w += sizeof(int);
  g.rounds = (int*)w;             w += sizeof(int);
  g.bar.count = bar;
  g.max_sweeps = NOALLOC_SWEEPS;
  // the array keeps the previous call's contents: copy G in and clear what must start at zero
  e = cudaMemcpyAsync(g.A, G, sizeof(cplx) * (size_t)k * k, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(zero_begin, 0, (size_t)(w - zero_begin), s);
  if (e != cudaSuccess) return chfsi_cuda_error(e, "scratch set-up");
  fro_kernel<<<1, 1024, 0, s>>>(k, g.A, g.fro);
  count_launch();
  const long work_items = (long)(kk / 2) * (kk / 2) + (long)k * (kk / 2);
  int blocks = coop_blocks((int)((work_items + 255) / 256));
  void* args[] = {&g};
  // serialised with the library's other grid-barrier kernels on this device (see coop_launch)
  e = coop_launch((const void*)jacobi_kernel, dim3(blocks), dim3(256), args, s);
  count_launch();
  if (e != cudaSuccess) return chfsi_cuda_error(e, "jacobi launch");
  jacobi_sort_kernel<<<k < 1024 ? k : 1024, 128, 0, s>>>(k, g.A, (const cplx*)g.V, lam, (cplx*)W);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return chfsi_cuda_error(e, "jacobi sort");
  int herr = 0;
  e = cudaMemcpyAsync(&herr, g.err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return chfsi_cuda_error(e, "jacobi status");
  if (herr == DEV_OK) return CHFSI_OK;
  return herr == DEV_ERR_TIMEOUT ? CHFSI_ERR_TIMEOUT : CHFSI_ERR_NO_CONV;
}
