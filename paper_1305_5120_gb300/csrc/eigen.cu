// Reduced eigenproblem of Rayleigh-Ritz (Algorithm 1, "Solving reduced problem G w = lam w"),
// second solver: an FP32 start refined to FP64 accuracy.
//
// On this GPU a grid-wide round of the FP64 two-sided Jacobi costs ~3 us (FP64 issue rate and
// a grid barrier) and a call takes ~500 of them.  Here:
//
//  1. FP32 one-sided cyclic Jacobi inside ONE thread-block cluster (hardware cluster barrier
//     per round, one warp per column pair, FP32 pipe): the columns of B = G + s I,
//     s = 2 min(||G||_F, max column sum) >= 2 ||G||_2 (so B is positive definite with
//     condition <= 3), are made mutually orthogonal by plane rotations from the right, B J = W.  For Hermitian positive definite B the columns of W
//     are multiples of eigenvectors (B j_i = sigma_i j_i), so no rotation accumulator is kept:
//     x_i = w_i / ||w_i|| (in FP64).
//  2. FP64 refinement of the eigenvector matrix X (a quadratically convergent iteration of
//     the kind analysed by Ogita & Aishima, "Iterative refinement for symmetric eigenvalue
//     decomposition", 2018): with R = I - X^H X and S = X^H G X (both from FP64-accurate
//     products on the tensor cores), lam_i = S_ii / (1 - R_ii) and X <- X (I + F),
//     F_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i) (i != j), F_ii = R_ii / 2 -- the first-order
//     solution of (I + F)^H (I - R)(I + F) = I, (I + F)^H S (I + F) = diagonal.  Pairs whose
//     coupling is not small against their eigenvalue gap (|S_ij| > 0.05 |lam_j - lam_i|) form
//     groups (connected components, found on the host); each group's block of S is
//     diagonalised exactly first (FP64 Jacobi, one CTA per group) and the first-order step
//     acts on the rest.
//
// Host orchestration (the products, the convergence test and the fallback to the FP64 Jacobi
// of jacobi.cu) is in chfsi_api.cu.
#include <math.h>
#include <stdlib.h>

#include <algorithm>

#include <cooperative_groups.h>

#include "eigen.cuh"

void count_launch(unsigned long long n);

namespace {

constexpr int OS_THREADS = 512;
constexpr int OS_WARPS = OS_THREADS / 32;
constexpr int OS_CACHE = 16;   // column elements per lane kept in registers (k <= 512)

__device__ __forceinline__ int slot(int x, int r, int kk) { return x == 0 ? 0 : 1 + (x - 1 + r) % (kk - 1); }

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// mbarriers in shared memory, signalled from other CTAs of the cluster
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
constexpr long OS_WAIT_LIMIT = 1L << 22;

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct OsArgs {
  int k, kk, max_sweeps;
  float tol;           // rotate when |x^H y| > tol ||x|| ||y||
  float2* B;           // k x k, column-major (ld k): G + s I on entry, W = B J on exit
  float* nrm;          // k: squared column norms (scan scratch)
  int* rot_count;      // max_sweeps + 1: pairs above the threshold at each scan, zeroed before the launch
  int* sweeps;         // out: rotating sweeps run
  int* err;            // DEV_ERR_NO_CONV when max_sweeps ran out
};

// One-sided Jacobi step on columns x = b_p, y = b_q: with a = ||x||^2, b = ||y||^2,
// g = x^H y, the 2 x 2 unitary U = [[c, s], [-s conj(ph), c conj(ph)]] (ph = g / |g|,
// tan = t: t^2 + 2 tau t - 1 = 0, tau = (b - a) / (2 |g|), the smaller root) diagonalises
// [[a, g], [conj g, b]], so x' = c x - s conj(ph) y and y' = s x + c conj(ph) y are
// orthogonal.
//
// Convergence is decided before every sweep by one scan of all pairs at once (squared column
// norms first, then every x_p^H x_q against the threshold; no rotation, two cluster barriers):
// a sweep that would rotate nothing is never run, and a block already within the threshold
// (a seeded problem's Rayleigh quotient matrix often is) costs one scan.
__device__ __forceinline__ int os_scan(const OsArgs& g, int gw, int nw, int lane) {
  const int k = g.k;
  for (int p = gw; p < k; p += nw) {
    const float2* bp = g.B + (long)p * k;
    float a = 0.f;
    for (int i = lane; i < k; i += 32) {
      const float2 x = __ldcg(bp + i);
      a = fmaf(x.x, x.x, fmaf(x.y, x.y, a));
    }
    a = warp_sumf(a);
    if (lane == 0) __stcg(g.nrm + p, a);
  }
  cluster_sync_all();
  // row pair j: columns j and k-1-j with all their partners above them (k - 1 products together)
  const float tol2 = g.tol * g.tol;
  const bool cached = k <= 32 * OS_CACHE;
  int viol = 0;
  for (int j = gw; j < (k + 1) / 2; j += nw) {
    for (int h = 0; h < 2; ++h) {
      const int p = h == 0 ? j : k - 1 - j;
      if (h == 1 && p == j) break;
      const float2* bp = g.B + (long)p * k;
      float2 xs[OS_CACHE];
      if (cached) {
#pragma unroll
        for (int t = 0; t < OS_CACHE; ++t) {
          const int i = lane + 32 * t;
          xs[t] = i < k ? __ldcg(bp + i) : make_float2(0.f, 0.f);
        }
      }
      const float a = __ldcg(g.nrm + p);
      int q = p + 1;
      if (cached) {
        // four partners at a time: their loads are in flight together
        for (; q + 4 <= k; q += 4) {
          float gr[4] = {0.f, 0.f, 0.f, 0.f}, gi[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int t = 0; t < OS_CACHE; ++t) {
            const int i = lane + 32 * t;
            if (i < k) {
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const float2 y = __ldcg(g.B + (long)(q + u) * k + i);
                gr[u] = fmaf(xs[t].x, y.x, fmaf(xs[t].y, y.y, gr[u]));
                gi[u] = fmaf(xs[t].x, y.y, fmaf(-xs[t].y, y.x, gi[u]));
              }
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float r = warp_sumf(gr[u]), m = warp_sumf(gi[u]);
            if (fmaf(r, r, m * m) > tol2 * a * __ldcg(g.nrm + q + u)) ++viol;
          }
        }
      }
      for (; q < k; ++q) {
        const float2* bq = g.B + (long)q * k;
        float gr = 0.f, gi = 0.f;
        if (cached) {
#pragma unroll
          for (int t = 0; t < OS_CACHE; ++t) {
            const int i = lane + 32 * t;
            const float2 y = i < k ? __ldcg(bq + i) : make_float2(0.f, 0.f);
            gr = fmaf(xs[t].x, y.x, fmaf(xs[t].y, y.y, gr));
            gi = fmaf(xs[t].x, y.y, fmaf(-xs[t].y, y.x, gi));
          }
        } else {
          for (int i = lane; i < k; i += 32) {
            const float2 x = __ldcg(bp + i), y = __ldcg(bq + i);
            gr = fmaf(x.x, y.x, fmaf(x.y, y.y, gr));
            gi = fmaf(x.x, y.y, fmaf(-x.y, y.x, gi));
          }
        }
        gr = warp_sumf(gr);
        gi = warp_sumf(gi);
        if (fmaf(gr, gr, gi * gi) > tol2 * a * __ldcg(g.nrm + q)) ++viol;
      }
    }
  }
  return viol;   // per warp (every lane holds it)
}

__global__ void __launch_bounds__(OS_THREADS, 1) os_jacobi_kernel(OsArgs g) {
  const int k = g.k, kk = g.kk, np = kk / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * OS_WARPS + warp, nw = gridDim.x * OS_WARPS;   // the grid is one cluster
  const bool cached = k <= 32 * OS_CACHE;
  int sweep = 0;
  bool done = false;
  for (;; ++sweep) {
    const int viol = os_scan(g, gw, nw, lane);
    if (lane == 0 && viol) atomicAdd(&g.rot_count[sweep], viol);
    cluster_sync_all();
    done = *(volatile int*)&g.rot_count[sweep] == 0;
    if (done || sweep == g.max_sweeps) break;
    for (int r = 0; r < kk - 1; ++r) {
      for (int j = gw; j < np; j += nw) {
        int p = slot(j, r, kk), q = slot(kk - 1 - j, r, kk);
        if (p > q) { const int t = p; p = q; q = t; }
        if (q >= k) continue;
        float2* bp = g.B + (long)p * k;
        float2* bq = g.B + (long)q * k;
        float2 xs[OS_CACHE], ys[OS_CACHE];
        float a = 0.f, b = 0.f, gr = 0.f, gi = 0.f;
        if (cached) {
#pragma unroll
          for (int t = 0; t < OS_CACHE; ++t) {
            const int i = lane + 32 * t;
            float2 x = make_float2(0.f, 0.f), y = x;
            if (i < k) {
              x = __ldcg(bp + i);   // other SMs of the cluster wrote these: read through L2
              y = __ldcg(bq + i);
            }
            xs[t] = x;
            ys[t] = y;
            a = fmaf(x.x, x.x, fmaf(x.y, x.y, a));
            b = fmaf(y.x, y.x, fmaf(y.y, y.y, b));
            gr = fmaf(x.x, y.x, fmaf(x.y, y.y, gr));    // conj(x) y
            gi = fmaf(x.x, y.y, fmaf(-x.y, y.x, gi));
          }
        } else {
          for (int i = lane; i < k; i += 32) {
            const float2 x = __ldcg(bp + i), y = __ldcg(bq + i);
            a = fmaf(x.x, x.x, fmaf(x.y, x.y, a));
            b = fmaf(y.x, y.x, fmaf(y.y, y.y, b));
            gr = fmaf(x.x, y.x, fmaf(x.y, y.y, gr));
            gi = fmaf(x.x, y.y, fmaf(-x.y, y.x, gi));
          }
        }
        a = warp_sumf(a);
        b = warp_sumf(b);
        gr = warp_sumf(gr);
        gi = warp_sumf(gi);
        const float ag = sqrtf(fmaf(gr, gr, gi * gi));
        if (!(ag > g.tol * sqrtf(a * b))) continue;   // warp-uniform: every lane holds the sums
        const float phr = gr / ag, phi = gi / ag;
        const float tau = (b - a) / (2.f * ag);
        const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
        const float c = rsqrtf(fmaf(t, t, 1.f)), s = t * c;
        if (cached) {
#pragma unroll
          for (int u = 0; u < OS_CACHE; ++u) {
            const int i = lane + 32 * u;
            if (i >= k) continue;
            const float2 x = xs[u], y = ys[u];
            const float wr = fmaf(phr, y.x, phi * y.y), wi = fmaf(phr, y.y, -phi * y.x);   // conj(ph) y
            __stcg(bp + i, make_float2(fmaf(c, x.x, -s * wr), fmaf(c, x.y, -s * wi)));
            __stcg(bq + i, make_float2(fmaf(s, x.x, c * wr), fmaf(s, x.y, c * wi)));
          }
        } else {
          for (int i = lane; i < k; i += 32) {
            const float2 x = __ldcg(bp + i), y = __ldcg(bq + i);
            const float wr = fmaf(phr, y.x, phi * y.y), wi = fmaf(phr, y.y, -phi * y.x);
            __stcg(bp + i, make_float2(fmaf(c, x.x, -s * wr), fmaf(c, x.y, -s * wi)));
            __stcg(bq + i, make_float2(fmaf(s, x.x, c * wr), fmaf(s, x.y, c * wi)));
          }
        }
      }
      cluster_sync_all();
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *g.sweeps = sweep;
    if (!done) atomicExch(g.err, DEV_ERR_NO_CONV);
  }
}

// The same sweeps with the columns resident in the cluster's shared memory (k up to a few
// hundred): worker j (warp j % W of CTA j / W) owns the two positions j and kk-1-j of the
// round-robin schedule and keeps their columns in its CTA's shared memory.  In a round it
// rotates its pair in place, then moves its two columns to the positions they occupy in the
// next round (position x + 1 -> x, position 1 -> kk - 1, position 0 fixed): into a
// neighbour's slot of the other buffer, in the same CTA or through distributed shared memory;
// no global-memory round trip.  A worker depends only on the two workers whose columns it
// receives, so instead of a cluster-wide barrier per round each worker has one mbarrier per
// buffer that completes when both of its incoming columns have been written (the senders
// store through distributed shared memory, then arrive with release semantics); waits are
// bounded.  After a whole sweep every column is back at its own position; the rotation count
// of a sweep is gathered with one cluster barrier.  The iteration ends after a sweep that rotates
// nothing, or after one whose largest relative coupling |x^H y| / (||x|| ||y||) was at most
// OS_QUAD: Jacobi converges quadratically, so what remains is of order OS_QUAD^2, below the
// rotation threshold -- and the FP64 refinement that follows removes any remainder -- so the
// rotation-free confirming sweep is saved.
constexpr float OS_QUAD = 1e-4f;
__global__ void __launch_bounds__(OS_THREADS, 1) os_dsmem_kernel(OsArgs g, int W) {
  extern __shared__ uint64_t dyn[];   // mbarriers [2 buffers][W workers], then the columns
  uint64_t* bars = dyn;
  float2* sm = (float2*)(dyn + 2 * W);   // [2 buffers][W workers][2 slots][k]
  __shared__ int s_rot;
  __shared__ float s_rel;
  __shared__ int s_timeout;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int k = g.k, kk = g.kk, np = kk / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = (int)cl.block_rank();
  const int j = rank * W + warp;
  const bool active = j < np;
  auto slotp = [&](int buf, int w, int h) { return sm + (((long)buf * W + w) * 2 + h) * k; };
  auto remote = [&](int buf, int t, int h) { return cl.map_shared_rank(slotp(buf, t % W, h), t / W); };
  // worker t's barrier for buffer `buf`, as a cluster address: it completes a phase when both
  // of t's slots of that buffer have been written (two arrivals)
  auto bar_of = [&](int buf, int t) { return cluster_addr(smem_addr(bars + buf * W + t % W), t / W); };
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2 * W; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;" ::"r"(smem_addr(bars + b)));
    s_timeout = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (active) {
    for (int h = 0; h < 2; ++h) {
      const int c = h == 0 ? j : kk - 1 - j;
      float2* d = slotp(0, warp, h);
      for (int i = lane; i < k; i += 32) d[i] = c < k ? __ldcg(g.B + (long)c * k + i) : make_float2(0.f, 0.f);
    }
  }
  if (threadIdx.x == 0) {
    s_rot = 0;
    s_rel = 0.f;
  }
  cluster_sync_all();
  int cur = 0, sweep = 0;
  long rg = 0;   // rounds run so far (over all sweeps)
  bool done = false;
  for (; sweep < g.max_sweeps && !done; ++sweep) {
    for (int r = 0; r < kk - 1; ++r, ++rg) {
      if (active) {
        // this round's two columns were written by the neighbours at the end of the last one
        if (rg > 0) {
          if (lane == 0 && !*(volatile int*)&s_timeout) {
            const uint32_t bar = smem_addr(bars + cur * W + warp);
            const uint32_t par = (uint32_t)((rg - 1) >> 1) & 1u;
            long it = 0;
            while (!mbar_try_cluster(bar, par) && ++it < OS_WAIT_LIMIT) {}
            if (it >= OS_WAIT_LIMIT) {   // bounded: record and stop waiting (the refinement rejects the result)
              s_timeout = 1;
              atomicExch(g.err, DEV_ERR_TIMEOUT);
            }
          }
          __syncwarp();
        }
        int p = slot(j, r, kk), q = slot(kk - 1 - j, r, kk);
        float2* xp = slotp(cur, warp, 0);
        float2* xq = slotp(cur, warp, 1);
        if (p > q) {
          const int t = p; p = q; q = t;
          float2* u = xp; xp = xq; xq = u;
        }
        if (q < k) {
          float a = 0.f, b = 0.f, gr = 0.f, gi = 0.f;
          for (int i = lane; i < k; i += 32) {
            const float2 x = xp[i], y = xq[i];
            a = fmaf(x.x, x.x, fmaf(x.y, x.y, a));
            b = fmaf(y.x, y.x, fmaf(y.y, y.y, b));
            gr = fmaf(x.x, y.x, fmaf(x.y, y.y, gr));    // conj(x) y
            gi = fmaf(x.x, y.y, fmaf(-x.y, y.x, gi));
          }
          a = warp_sumf(a);
          b = warp_sumf(b);
          gr = warp_sumf(gr);
          gi = warp_sumf(gi);
          const float ag = sqrtf(fmaf(gr, gr, gi * gi));
          const float nab = sqrtf(a * b);
          if (ag > g.tol * nab) {   // warp-uniform
            const float phr = gr / ag, phi = gi / ag;
            const float tau = (b - a) / (2.f * ag);
            const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
            const float c = rsqrtf(fmaf(t, t, 1.f)), sn = t * c;
            for (int i = lane; i < k; i += 32) {
              const float2 x = xp[i], y = xq[i];
              const float wr = fmaf(phr, y.x, phi * y.y), wi = fmaf(phr, y.y, -phi * y.x);   // conj(ph) y
              xp[i] = make_float2(fmaf(c, x.x, -sn * wr), fmaf(c, x.y, -sn * wi));
              xq[i] = make_float2(fmaf(sn, x.x, c * wr), fmaf(sn, x.y, c * wi));
            }
            if (lane == 0) {
              atomicAdd(&s_rot, 1);
              // non-negative floats order like their bit patterns
              atomicMax((int*)&s_rel, __float_as_int(fminf(ag / nab, 1.f)));
            }
          }
        }
        // move to the next round's positions (each target slot receives exactly one column)
        const float2* f = slotp(cur, warp, 0);
        const float2* sc = slotp(cur, warp, 1);
        float2* df;
        float2* ds;
        int tf, ts;   // receiving workers
        if (np == 1) {
          df = slotp(cur ^ 1, warp, 0);
          ds = slotp(cur ^ 1, warp, 1);
          tf = ts = j;
        } else {
          tf = j == 0 ? 0 : (j == 1 ? 0 : j - 1);
          ts = j < np - 1 ? j + 1 : j;
          df = j == 0 ? slotp(cur ^ 1, warp, 0) : (j == 1 ? remote(cur ^ 1, 0, 1) : remote(cur ^ 1, j - 1, 0));
          ds = j < np - 1 ? remote(cur ^ 1, j + 1, 1) : slotp(cur ^ 1, warp, 0);
        }
        for (int i = lane; i < k; i += 32) {
          df[i] = f[i];
          ds[i] = sc[i];
        }
        // the copies are visible to the receivers before their barriers are signalled: the
        // warp barrier orders every lane's stores before lane 0's cluster-scope release
        __syncwarp();
        if (lane == 0) {
          asm volatile("fence.acq_rel.cluster;" ::: "memory");
          mbar_arrive_cluster(bar_of(cur ^ 1, tf));
          mbar_arrive_cluster(bar_of(cur ^ 1, ts));
        }
      }
      cur ^= 1;
    }
    // every CTA adds its count and its largest coupling; after the barrier all read the totals
    if (threadIdx.x == 0 && s_rot) {
      atomicAdd(&g.rot_count[sweep], s_rot);
      atomicMax((int*)g.nrm + sweep, __float_as_int(s_rel));
    }
    cluster_sync_all();
    done = *(volatile int*)&g.rot_count[sweep] == 0 ||
           __int_as_float(*((volatile int*)g.nrm + sweep)) <= OS_QUAD;
    if (threadIdx.x == 0) {
      s_rot = 0;
      s_rel = 0.f;
    }
    __syncthreads();
  }
  // after whole sweeps every column is at its own position: worker j holds columns j, kk-1-j
  if (active) {
    for (int h = 0; h < 2; ++h) {
      const int c = h == 0 ? j : kk - 1 - j;
      if (c >= k) continue;
      const float2* src = slotp(cur, warp, h);
      for (int i = lane; i < k; i += 32) __stcg(g.B + (long)c * k + i, src[i]);
    }
  }
  if (rank == 0 && threadIdx.x == 0) {
    *g.sweeps = sweep;
    if (!done) atomicExch(g.err, DEV_ERR_NO_CONV);
  }
  cluster_sync_all();   // no CTA leaves while a peer could still address its shared memory
}

// B = G + s I in FP32 (rounded to nearest)
__global__ void os_init_kernel(int k, const cplx* G, double s, float2* B) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)k * k; e += (long)gridDim.x * blockDim.x) {
    cplx v = G[e];
    if (e % k == e / k) v.x += s;
    B[e] = make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
  }
}

// X (FP64) = normalised columns of W, one warp per column; also copied into P[:, :k]
__global__ void os_columns_kernel(int k, const float2* W, cplx* X) {
  const int lane = threadIdx.x & 31;
  for (int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); col < k; col += gridDim.x * (blockDim.x >> 5)) {
    double s = 0.0;
    for (int i = lane; i < k; i += 32) {
      const float2 w = W[(long)col * k + i];
      s += (double)w.x * w.x + (double)w.y * w.y;
    }
    s = warp_sum(s);
    const double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    for (int i = lane; i < k; i += 32) {
      const float2 w = W[(long)col * k + i];
      X[(long)col * k + i] = cmk(w.x * inv, w.y * inv);
    }
  }
}

// From T = X^H [X | G X] (k x 2k): R = I - herm(T[:, :k]) and S = herm(T[:, k:]) in place of
// the two halves; lam_i = S_ii / (1 - R_ii).  One thread per diagonal entry here.
__global__ void oa_diag_kernel(int k, const cplx* T, double* lam) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
    const double rii = 1.0 - T[i + (long)i * k].x;
    const double sii = T[i + (long)(k + i) * k].x;
    lam[i] = sii / (1.0 - rii);
  }
}

// Pair pass: Hermitian parts of R and S (written to R, S, k x k each), the largest |S_ij|^2
// (i != j) and |R_ij|^2 as ordered bit patterns (non-negative doubles order like their bits),
// and the list of strongly coupled pairs i < j (|S_ij| > tau |lam_j - lam_i|), capped.
// Squared magnitudes throughout: no square root per entry on the FP64 pipe.
__global__ void oa_pairs_kernel(int k, const cplx* T, const double* lam, double tau, cplx* R, cplx* S,
                                unsigned long long* maxbits, int* npairs, int cap, int2* pairs) {
  // maxima reduced in the warp, then the block, then one atomic per block
  unsigned long long ms = 0, mr = 0, mf = 0;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)k * k; e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e % k), j = (int)(e / k);
    const cplx x = T[e], xt = T[j + (long)i * k];                  // X^H X entries (i, j) and (j, i)
    const cplx y = T[e + (long)k * k], yt = T[j + (long)(k + i) * k];
    cplx r = cmk(-0.5 * (x.x + xt.x), -0.5 * (x.y - xt.y));      // I - herm(X^H X)
    const cplx sv = cmk(0.5 * (y.x + yt.x), 0.5 * (y.y - yt.y));
    if (i == j) {
      r.x += 1.0;
      r.y = 0.0;
    }
    R[e] = r;
    S[e] = cmk(sv.x, i == j ? 0.0 : sv.y);
    mr = max(mr, (unsigned long long)__double_as_longlong(cabs2(r)));
    if (i != j) {
      const double sa2 = cabs2(sv), dl = tau * (lam[j] - lam[i]);
      ms = max(ms, (unsigned long long)__double_as_longlong(sa2));
      if (i < j && sa2 > dl * dl) {
        const int slot_i = atomicAdd(npairs, 1);
        if (slot_i < cap) pairs[slot_i] = make_int2(i, j);
      } else if (dl != 0.0) {
        // first-order correction of a weakly coupled pair: F_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i)
        const double d = lam[j] - lam[i];
        const cplx f = cmk(sv.x + lam[j] * r.x, sv.y + lam[j] * r.y);
        mf = max(mf, (unsigned long long)__double_as_longlong(cabs2(f) / (d * d)));
      }
    }
  }
  __shared__ unsigned long long sh[3][32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ms = max(ms, __shfl_xor_sync(0xffffffffu, ms, o));
    mr = max(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    mf = max(mf, __shfl_xor_sync(0xffffffffu, mf, o));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][w] = ms;
    sh[1][w] = mr;
    sh[2][w] = mf;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
      ms = max(ms, sh[0][q]);
      mr = max(mr, sh[1][q]);
      mf = max(mf, sh[2][q]);
    }
    if (ms) atomicMax(maxbits, ms);
    if (mr) atomicMax(maxbits + 1, mr);
    if (mf) atomicMax(maxbits + 2, mf);
  }
}

// Exact diagonalisation of each group's block of S (group g: indices idx[off[g] .. off[g+1]))
// by cyclic FP64 Jacobi in shared memory, one CTA per group; the eigenvectors go to V (the
// group's c x c block at voff[g], column-major).  Groups have at most OA_GROUP_MAX members.
__global__ void __launch_bounds__(256) oa_group_kernel(int k, const cplx* S, const int* off, const int* idx,
                                                       const int* voff, cplx* V, int* err) {
  __shared__ cplx A[OA_GROUP_MAX][OA_GROUP_MAX + 1];
  __shared__ cplx U[OA_GROUP_MAX][OA_GROUP_MAX + 1];
  __shared__ double rc[OA_GROUP_MAX / 2], rs[OA_GROUP_MAX / 2], rpx[OA_GROUP_MAX / 2], rpy[OA_GROUP_MAX / 2];
  __shared__ int rp[OA_GROUP_MAX / 2], rq[OA_GROUP_MAX / 2], ron[OA_GROUP_MAX / 2];
  __shared__ double s_fro;
  __shared__ int s_any;
  const int gidx = blockIdx.x;
  const int o = off[gidx], c = off[gidx + 1] - o;
  const int cc = c + (c & 1);
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
    const int a = e % c, b = e / c;
    A[a][b] = S[idx[o + a] + (long)idx[o + b] * k];
    U[a][b] = cmk(a == b ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double f = 0.0;
    for (int a = 0; a < c; ++a)
      for (int b = 0; b < c; ++b) f += cabs2(A[a][b]);
    s_fro = sqrt(f);
  }
  __syncthreads();
  // rounding of the rotations leaves off-diagonal entries of order c u ||A||_F
  const double thresh = (double)c * 2.220446049250313e-16 * s_fro;
  bool converged = false;
  for (int sweep = 0; sweep < 30 && !converged; ++sweep) {
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    for (int r = 0; r < cc - 1; ++r) {
      if (threadIdx.x < cc / 2) {
        const int jp = threadIdx.x;
        int p = slot(jp, r, cc), q = slot(cc - 1 - jp, r, cc);
        if (p > q) { const int t = p; p = q; q = t; }
        int on = 0;
        double cs = 1.0, sn = 0.0, px = 1.0, py = 0.0;
        if (q < c) {
          const cplx apq = A[p][q];
          const double ar = sqrt(cabs2(apq));
          if (ar > thresh) {
            const double tau = (A[q][q].x - A[p][p].x) / (2.0 * ar);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            cs = 1.0 / sqrt(1.0 + t * t);
            sn = t * cs;
            px = apq.x / ar;
            py = -apq.y / ar;   // conj(ph)
            on = 1;
            s_any = 1;
          }
        }
        rp[jp] = p; rq[jp] = q; ron[jp] = on; rc[jp] = cs; rs[jp] = sn; rpx[jp] = px; rpy[jp] = py;
      }
      __syncthreads();
      // columns: A <- A U_r (pairs act on disjoint column pairs), U <- U U_r
      for (int e = threadIdx.x; e < 2 * c * (cc / 2); e += blockDim.x) {
        const int which = e / (c * (cc / 2));
        const int f = e % (c * (cc / 2));
        const int row = f % c, jp = f / c;
        if (!ron[jp] || rq[jp] >= c) continue;
        const int p = rp[jp], q = rq[jp];
        cplx (*M)[OA_GROUP_MAX + 1] = which ? U : A;
        const cplx x = M[row][p], y = M[row][q];
        const cplx w = cmul(y, cmk(rpx[jp], rpy[jp]));
        M[row][p] = cmk(rc[jp] * x.x - rs[jp] * w.x, rc[jp] * x.y - rs[jp] * w.y);
        M[row][q] = cmk(rs[jp] * x.x + rc[jp] * w.x, rs[jp] * x.y + rc[jp] * w.y);
      }
      __syncthreads();
      // rows: A <- U_r^H A
      for (int e = threadIdx.x; e < c * (cc / 2); e += blockDim.x) {
        const int col = e % c, jp = e / c;
        if (!ron[jp] || rq[jp] >= c) continue;
        const int p = rp[jp], q = rq[jp];
        const cplx x = A[p][col], y = A[q][col];
        const cplx w = cmul(y, cmk(rpx[jp], -rpy[jp]));   // ph y
        A[p][col] = cmk(rc[jp] * x.x - rs[jp] * w.x, rc[jp] * x.y - rs[jp] * w.y);
        A[q][col] = cmk(rs[jp] * x.x + rc[jp] * w.x, rs[jp] * x.y + rc[jp] * w.y);
      }
      __syncthreads();
    }
    converged = s_any == 0;
    __syncthreads();
  }
  if (!converged && threadIdx.x == 0) atomicExch(err, DEV_ERR_NO_CONV);
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) V[voff[gidx] + e] = U[e % c][e / c];
}

// Y = Z U for a block-diagonal unitary U over the groups (identity elsewhere): column j of a
// group becomes sum_b Z[:, idx_b] V[b, pos(j)].  cols_only = false also applies U^H from the
// left (rows), giving U^H Z U (through `tmp`).
__global__ void oa_mix_cols_kernel(int rows, int k, const cplx* Z, cplx* Y, const int* gid, const int* gpos,
                                   const int* off, const int* idx, const int* voff, const cplx* V) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)rows * k; e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e % rows), j = (int)(e / rows);
    const int g = gid[j];
    if (g < 0) {
      Y[e] = Z[e];
      continue;
    }
    const int o = off[g], c = off[g + 1] - o, pj = gpos[j];
    cplx acc = cmk(0.0, 0.0);
    for (int b = 0; b < c; ++b) cfma(acc, Z[i + (long)idx[o + b] * rows], V[voff[g] + b + pj * c]);
    Y[e] = acc;
  }
}
__global__ void oa_mix_rows_kernel(int k, const cplx* Z, cplx* Y, const int* gid, const int* gpos, const int* off,
                                   const int* idx, const int* voff, const cplx* V) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)k * k; e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e % k), j = (int)(e / k);
    const int g = gid[i];
    if (g < 0) {
      Y[e] = Z[e];
      continue;
    }
    const int o = off[g], c = off[g + 1] - o, pi = gpos[i];
    cplx acc = cmk(0.0, 0.0);
    for (int a = 0; a < c; ++a) cfma(acc, cconj(V[voff[g] + a + pi * c]), Z[idx[o + a] + (long)j * k]);
    Y[e] = acc;
  }
}

// F from S2 = U^H S U, R2 = U^H R U: lam2_i = S2_ii / (1 - R2_ii); within a group (and on the
// diagonal) F = R2 / 2, elsewhere the first-order solution (S2_ij + lam2_j R2_ij) / (lam2_j -
// lam2_i).
__global__ void oa_update_kernel(int k, const cplx* S2, const cplx* R2, const int* gid, cplx* F) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)k * k; e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e % k), j = (int)(e / k);
    const cplx r = R2[e];
    const double li = S2[i + (long)i * k].x / (1.0 - R2[i + (long)i * k].x);
    const double lj = S2[j + (long)j * k].x / (1.0 - R2[j + (long)j * k].x);
    const double d = lj - li;
    cplx f;
    if (i == j || (gid[i] >= 0 && gid[i] == gid[j]) || d == 0.0) {
      f = cscale(r, 0.5);
    } else {
      const cplx s = S2[e];
      f = cmk((s.x + lj * r.x) / d, (s.y + lj * r.y) / d);
    }
    F[e] = f;
  }
}

// rank sort: lam[rank] = d_i, W[:, rank] = X[:, i] (ties by index)
__global__ void oa_sort_kernel(int k, const double* d, const cplx* X, double* lam, cplx* W) {
  for (int i = blockIdx.x; i < k; i += gridDim.x) {
    const double li = d[i];
    __shared__ int rank_sh;
    if (threadIdx.x == 0) rank_sh = 0;
    __syncthreads();
    int cnt = 0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
      const double lj = d[j];
      if (lj < li || (lj == li && j < i)) ++cnt;
    }
    atomicAdd(&rank_sh, cnt);
    __syncthreads();
    const int rk = rank_sh;
    if (threadIdx.x == 0) lam[rk] = li;
    for (int r = threadIdx.x; r < k; r += blockDim.x) W[r + (long)rk * k] = X[r + (long)i * k];
    __syncthreads();
  }
}

unsigned grid_for(long total) {
  long b = (total + 255) / 256;
  return (unsigned)std::max(1L, std::min(b, 152L * 8));
}

}  // namespace

cudaError_t os_jacobi_f32(cudaStream_t s, int k, const cplx* G, double shift, float2* B, float* nrm, int* counters,
                          int max_sweeps, float tol, int* err, int* sweeps, int* cluster_used) {
  os_init_kernel<<<grid_for((long)k * k), 256, 0, s>>>(k, G, shift, B);
  count_launch(1);
  cudaError_t e = cudaMemsetAsync(counters, 0, sizeof(int) * (max_sweeps + 1), s);
  if (e != cudaSuccess) return e;
  static int nc_ok = 0;   // largest cluster size that launched (16 needs the non-portable opt-in)
  OsArgs a{};
  a.k = k;
  a.kk = k + (k & 1);
  a.max_sweeps = max_sweeps;
  a.tol = tol;
  a.B = B;
  a.nrm = nrm;
  a.rot_count = counters;
  a.sweeps = sweeps;
  a.err = err;
  // columns resident in the cluster's shared memory when two buffers of every worker's two
  // columns fit (k up to ~450 on 16 CTAs)
  static int nc_ds_ok = 0;
  static const int nc_env = [] {
    const char* v = getenv("CHFSI_OS_CLUSTER");   // 8 or 16: the cluster size (default: 16 when allowed)
    return v ? atoi(v) : 0;
  }();
  e = cudaMemsetAsync(nrm, 0, sizeof(float) * (max_sweeps + 1), s);   // per-sweep largest coupling
  if (e != cudaSuccess) return e;
  for (int nc : {16, 8}) {
    if (nc_ds_ok && nc > nc_ds_ok) continue;
    if (nc_env && nc != nc_env) continue;
    const int np = a.kk / 2, W = (np + nc - 1) / nc;
    const size_t smem = sizeof(uint64_t) * 2 * (size_t)W + sizeof(float2) * 4 * (size_t)W * k;
    if (W > OS_WARPS || smem > 200 * 1024) continue;
    if (nc == 16) cudaFuncSetAttribute(os_dsmem_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(os_dsmem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nc);
    cfg.blockDim = dim3(32 * W);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = nc;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, os_dsmem_kernel, &cfg) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      continue;
    }
    e = cudaLaunchKernelEx(&cfg, os_dsmem_kernel, a, W);
    count_launch(1);
    if (e == cudaSuccess) {
      nc_ds_ok = nc;
      if (cluster_used) *cluster_used = nc;
      return cudaSuccess;
    }
    cudaGetLastError();
  }
  for (int nc : {16, 8}) {
    if (nc_ok && nc > nc_ok) continue;
    if (nc == 16) cudaFuncSetAttribute(os_jacobi_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nc);
    cfg.blockDim = dim3(OS_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = nc;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, os_jacobi_kernel, &cfg) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      continue;
    }
    e = cudaLaunchKernelEx(&cfg, os_jacobi_kernel, a);
    count_launch(1);
    if (e == cudaSuccess) {
      nc_ok = nc;
      if (cluster_used) *cluster_used = nc;
      return cudaSuccess;
    }
    cudaGetLastError();
  }
  return cudaErrorLaunchFailure;
}

cudaError_t os_columns(cudaStream_t s, int k, const float2* W, cplx* X) {
  os_columns_kernel<<<std::max(1, std::min((k + 7) / 8, 152 * 4)), 256, 0, s>>>(k, W, X);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t oa_analyze(cudaStream_t s, int k, const cplx* T, double tau, double* lam, cplx* R, cplx* S,
                       unsigned long long* maxbits, int* npairs, int cap, int2* pairs) {
  cudaError_t e = cudaMemsetAsync(maxbits, 0, 3 * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(npairs, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  oa_diag_kernel<<<(k + 255) / 256, 256, 0, s>>>(k, T, lam);
  count_launch(1);
  oa_pairs_kernel<<<grid_for((long)k * k), 256, 0, s>>>(k, T, lam, tau, R, S, maxbits, npairs, cap, pairs);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t oa_groups(cudaStream_t s, int k, int ngroups, const cplx* S, const int* off, const int* idx,
                      const int* voff, cplx* V, int* err) {
  if (ngroups <= 0) return cudaSuccess;
  oa_group_kernel<<<ngroups, 256, 0, s>>>(k, S, off, idx, voff, V, err);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t oa_mix(cudaStream_t s, int rows, int k, const cplx* Z, cplx* Y, bool both_sides, cplx* tmp, const int* gid,
                   const int* gpos, const int* off, const int* idx, const int* voff, const cplx* V) {
  if (!both_sides) {
    oa_mix_cols_kernel<<<grid_for((long)rows * k), 256, 0, s>>>(rows, k, Z, Y, gid, gpos, off, idx, voff, V);
    count_launch(1);
    return cudaGetLastError();
  }
  oa_mix_cols_kernel<<<grid_for((long)k * k), 256, 0, s>>>(k, k, Z, tmp, gid, gpos, off, idx, voff, V);
  count_launch(1);
  oa_mix_rows_kernel<<<grid_for((long)k * k), 256, 0, s>>>(k, tmp, Y, gid, gpos, off, idx, voff, V);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t oa_update(cudaStream_t s, int k, const cplx* S2, const cplx* R2, const int* gid, cplx* F) {
  oa_update_kernel<<<grid_for((long)k * k), 256, 0, s>>>(k, S2, R2, gid, F);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t oa_sort(cudaStream_t s, int k, const double* d, const cplx* X, double* lam, cplx* W) {
  oa_sort_kernel<<<std::min(k, 1024), 128, 0, s>>>(k, d, X, lam, W);
  count_launch(1);
  return cudaGetLastError();
}
