// Chebyshev filter step on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// One step of the scaled three-term recurrence (Eq. (3term) with shift and scale, Section 3)
//     Y_j = fa_j H' Y_{j-1} + fb_j Y_{j-1} + fg_j Y_{j-2}
// is one launch.  The complex product H' Y_{j-1} runs as a real GEMM through the embedding
//     [Re H' | Im H'] (K interleaved)  x  [[Re Y, Im Y], [-Im Y, Re Y]] (columns interleaved),
// so M = n, N = 2k, K = 2n.  Each operand is held as three BF16 slices (x = s0 + s1 + s2 to
// about 2^-24 |x|) and the six slice products with s + t <= 2 accumulate in FP32 TMEM
// accumulators, one per level s + t: an FP32-equivalent product on the BF16 pipe.
//
// The recurrence state lives only in the slices.  The B operand of step j holds the slices of
// Y_{j-1}; the epilogue rebuilds Y_{j-1} and Y_{j-2} from them in FP32, forms Y_j in FP32 and
// writes its slices over those of Y_{j-2} -- the next step's operand.  A column whose last step
// this is writes its FP64 result instead.  So a step executes no FP64 instruction: this GPU's
// FP64 pipe issues a warp instruction per 64 cycles per sub-partition, the FP32 pipe one per
// cycle, and an FP64 epilogue had cost more than the tensor-core main loop.
//
// Per CTA (one 128 x BN output tile): warp 0 issues TMA loads of the A and B slice tiles
// (128-byte swizzle) into a 3-stage shared-memory ring; warp 1 owns the TMEM accumulators and
// issues tcgen05.mma (three per K step); warps 2-5 drain TMEM and run the recurrence.  Every
// mbarrier wait is bounded: on timeout the kernel records DEV_ERR_TIMEOUT, waits (bounded) for
// the copies and products it has issued, frees its TMEM and leaves.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "filter_tc.cuh"

void count_launch(unsigned long long n);

#define TRY_CHFSI(x)                  \
  do {                                \
    chfsi_status _s = (x);            \
    if (_s != CHFSI_OK) return _s;    \
  } while (0)

namespace {

constexpr int BM = 128;          // tcgen05 M (cta_group::1)
constexpr int BK = 64;           // bf16 per 128-byte swizzle row
constexpr int NSLICE = 3;
constexpr int A_TILE = BM * BK * 2;            // bytes per A slice tile (16 KB)
constexpr int NTHREADS = 192;
constexpr long WAIT_LIMIT = 1L << 24;

// Tile of BN real output columns (BN / 2 complex): the autotuner picks the width per shape.
// TMEM holds the three level accumulators at columns [L BN, (L + 1) BN) (allocation: the next
// power of two); the shared-memory ring has as many stages as fit.
template <int BN>
struct Tile {
  static constexpr int B_TILE = BN * BK * 2;
  static constexpr int STAGE_BYTES = NSLICE * (A_TILE + B_TILE);
  static constexpr int STAGES = BN >= 128 ? 2 : 3;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
  static constexpr int TMEM_COLS = BN <= 32 ? 128 : (BN <= 64 ? 256 : 512);
  static_assert(STAGE_BYTES % 1024 == 0, "stage alignment");
  static_assert(SMEM_BYTES <= 232448, "shared memory");
  static_assert(3 * BN <= TMEM_COLS, "TMEM");
};

struct StepArgs {
  int n, mtiles;                 // rows, row tiles
  int ncols;                     // complex columns this step (cnt[j])
  int ncols_next;                // of which continue to step j + 1 (cnt[j + 1]; 0 on the last step)
  int kblocks;                   // K_pad / BK
  long kpad;                     // bf16 elements per B row
  long npad;                     // rows per B slice
  const __nv_bfloat16* Bcur;     // slices of Y_{j-1}: this step's B operand
  __nv_bfloat16* Bnext;          // in: slices of Y_{j-2} (read when fg != 0); out: slices of Y_j
  cplx* Yfinal;                  // FP64 result of the columns whose last step this is (ld n)
  float fa, fb, fg;
  const float2* R;               // corrected recurrence: R = H Yhat - Yhat diag(lam) (n x ncols), else NULL
  const float* fcol;             // per column fa_j p_{j-1}(lam_col); NULL for the plain recurrence
  int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; false (and the error word set) when the limit ran out or another role failed
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  for (long i = 0; i < WAIT_LIMIT; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 255) == 255 && *(volatile int*)err != DEV_OK) return false;
  }
  atomicExch(err, DEV_ERR_TIMEOUT);
  return false;
}
// bounded wait for work already issued (used on the way out after a failure): does not give
// up early when the error word is set, only after the limit
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity) {
  for (long i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}

// Programmatic dependent launch: the step launches overlap their prologue (barriers, TMEM,
// the first stages' A tiles, which no earlier step writes) with the end of the previous step.
// griddepcontrol.wait returns once the preceding grid has completed and its writes are
// visible (at once without a programmatic predecessor); launch_dependents, issued only after
// that wait, lets the next step's CTAs be scheduled, so a grid never runs ahead of a grid two
// launches back.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

// UMMA shared-memory descriptor: K-major operand, 128-byte swizzle, 8-row atoms 1024 B apart
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);           // start address
  d |= (uint64_t)1 << 16;                            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;                  // stride byte offset
  d |= (uint64_t)1 << 46;                            // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                            // SWIZZLE_128B
  return d;
}

// instruction descriptor: kind::f16, A/B bf16, D f32, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc_n,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc_n), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// FP64 -> FP32 rounded to nearest (half an FP32 unit added before truncation; a carry into
// the exponent field is the correct rounding), by integer operations on the bit pattern.
// Values below FP32's normal range become zero; infinities and NaNs keep their class.
__device__ __forceinline__ float f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned long long m = b & 0x7FFFFFFFFFFFFFFFull;
  if ((m >> 52) == 0x7FF) return __uint_as_float(sign | 0x7F800000u | ((m << 12) ? 0x400000u : 0u));
  const unsigned long long r = m + (1ull << 28);
  const int e = (int)(r >> 52) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((unsigned)e << 23) | (unsigned)((r >> 29) & 0x7FFFFF));
}

// three-way BF16 split of an FP32 value: x = s0 + s1 + s2 + O(2^-27 |x|); both subtractions
// are exact
__device__ __forceinline__ void split3f(float x, uint32_t& s0, uint32_t& s1, uint32_t& s2) {
  const __nv_bfloat16 b0 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(b0);
  const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b1);
  const __nv_bfloat16 b2 = __float2bfloat16_rn(r2);
  s0 = __bfloat16_as_ushort(b0);
  s1 = __bfloat16_as_ushort(b1);
  s2 = __bfloat16_as_ushort(b2);
}

// The B operand layout of one complex entry y in slice t: row 2j holds the pair (Re y, -Im y)
// and row 2j + 1 the pair (Im y, Re y), each pair one 32-bit word (first element low).
__device__ __forceinline__ uint32_t pack_lo_hi(uint32_t lo, uint32_t hi) { return lo | (hi << 16); }
__device__ __forceinline__ void store_slices(uint32_t* B32, long slice_words, long w2j, long w2j1, float re,
                                             float im) {
  uint32_t r0, r1, r2, i0, i1, i2;
  split3f(re, r0, r1, r2);
  split3f(im, i0, i1, i2);
  const uint32_t rs[3] = {r0, r1, r2}, is[3] = {i0, i1, i2};
#pragma unroll
  for (int t = 0; t < NSLICE; ++t) {
    B32[t * slice_words + w2j] = pack_lo_hi(rs[t], is[t] ^ 0x8000u);   // (Re, -Im)
    B32[t * slice_words + w2j1] = pack_lo_hi(is[t], rs[t]);            // (Im,  Re)
  }
}
// Y from the three words of row 2j: Re = s0 + (s1 + s2) (the inner sum is exact), Im likewise
__device__ __forceinline__ float2 join_slices(const uint32_t w[3]) {
  const float re = __uint_as_float(w[0] << 16) + (__uint_as_float(w[1] << 16) + __uint_as_float(w[2] << 16));
  const float nim = __uint_as_float(w[0] & 0xFFFF0000u) +
                    (__uint_as_float(w[1] & 0xFFFF0000u) + __uint_as_float(w[2] & 0xFFFF0000u));
  return make_float2(re, -nim);
}

template <int BN>
__device__ __forceinline__ void step_body(const CUtensorMap* tmA, const CUtensorMap* tmB, const StepArgs& g, int mtile,
                                          int ntile) {
  constexpr int STAGES = Tile<BN>::STAGES;
  constexpr int B_TILE = Tile<BN>::B_TILE;
  constexpr int STAGE_BYTES = Tile<BN>::STAGE_BYTES;
  constexpr int TMEM_COLS = Tile<BN>::TMEM_COLS;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* base_ptr = smem_raw + (base - raw);
  const uint32_t bars = base + STAGES * STAGE_BYTES;          // full[S], empty[S], accum
  uint64_t* bar_ptr = (uint64_t*)(base_ptr + STAGES * STAGE_BYTES);
  uint32_t* tmem_slot = (uint32_t*)(bar_ptr + 2 * STAGES + 1);
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (STAGES + s); };
  const uint32_t accum = bars + 8u * (2 * STAGES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = mtile * BM;
  const int n0 = ntile * BN;   // real column offset

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(accum, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *(volatile uint32_t*)tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // producer: A slice s at rows s*mtiles*BM + m0, B slice t at rows t*npad + n0.  The
      // first stages (empty at start) get their A tiles before the wait for the previous step,
      // their B tiles (that step's output) after it.
      const int pre = g.kblocks < STAGES ? g.kblocks : STAGES;
      for (int kb = 0; kb < pre; ++kb) {
        const uint32_t st = base + kb * STAGE_BYTES;
        mbar_expect_tx(full(kb), STAGE_BYTES);
        for (int q = 0; q < NSLICE; ++q)
          tma_load_2d(st + q * A_TILE, tmA, full(kb), kb * BK, q * g.mtiles * BM + m0);
      }
      pdl_wait();
      asm volatile("fence.proxy.async.global;" ::: "memory");
      pdl_trigger();
      for (int kb = 0; kb < pre; ++kb)
        for (int q = 0; q < NSLICE; ++q)
          tma_load_2d(base + kb * STAGE_BYTES + NSLICE * A_TILE + q * B_TILE, tmB, full(kb), kb * BK,
                      (int)(q * g.npad) + n0);
      int issued = pre;
      for (int kb = pre; kb < g.kblocks; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (!mbar_wait(empty(s), ph ^ 1, g.err)) break;
        mbar_expect_tx(full(s), STAGE_BYTES);
        const uint32_t st = base + s * STAGE_BYTES;
        for (int q = 0; q < NSLICE; ++q)
          tma_load_2d(st + q * A_TILE, tmA, full(s), kb * BK, q * g.mtiles * BM + m0);
        for (int q = 0; q < NSLICE; ++q)
          tma_load_2d(st + NSLICE * A_TILE + q * B_TILE, tmB, full(s), kb * BK, (int)(q * g.npad) + n0);
        issued = kb + 1;
      }
      // After a failure the consumer may have abandoned stages whose copies are still in
      // flight into this CTA's shared memory: wait until each issued stage has landed (each
      // stage's latest phase is the one checked) before the CTA may exit.
      if (*(volatile int*)g.err != DEV_OK)
        for (int kb = std::max(0, issued - STAGES); kb < issued; ++kb)
          mbar_drain(full(kb % STAGES), (kb / STAGES) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer.  The three B slice tiles of a stage lie one after another (slice t at rows
      // BN t of one K-major operand) and level L = s + t accumulates in TMEM columns [BN L,
      // BN L + BN), so the products of A slice s with B slices 0 .. 2 - s are one MMA of
      // N = BN (3 - s) into columns [BN s, 3 BN) (split at N = 256): three to four instructions
      // per 16-wide K step for the six slice products.  Each level has its own accumulator, so
      // the per-instruction truncation of the FP32 accumulation acts on every level at that
      // level's scale.
      for (int kb = 0; kb < g.kblocks; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (!mbar_wait(full(s), ph, g.err)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = base + s * STAGE_BYTES;
        // base descriptors once per stage; slices and K steps are start-address offsets
        const uint64_t da0 = umma_desc(st), db0 = umma_desc(st + NSLICE * A_TILE);
        const uint32_t later = kb != 0;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
          for (int sa = 0; sa < NSLICE; ++sa) {
            const uint64_t da = da0 + (uint64_t)((sa * A_TILE + kk * 32) >> 4);
            const uint32_t acc = (kk != 0 || sa != 0) ? 1u : later;
            constexpr int NMAX = 256;
#pragma unroll
            for (int off = 0; off < BN * (NSLICE - sa); off += NMAX) {
              const int nn = BN * (NSLICE - sa) - off < NMAX ? BN * (NSLICE - sa) - off : NMAX;
              // B rows [off, off + nn) of the stage: 128 bytes per K-major row
              const uint64_t db = db0 + (uint64_t)((off * 128 + kk * 32) >> 4);
              umma_bf16(tmem + (uint32_t)(sa * BN + off), da, db, idesc(nn), acc);
            }
          }
        }
        umma_commit(empty(s));   // frees the stage once these MMAs have read it
      }
      umma_commit(accum);        // arrives when every product issued above has completed
    }
  } else {
    // epilogue: warps 2..5 -> TMEM lane quarter (warp % 4).  It reads the previous steps'
    // output and overwrites the buffer the previous step read: after that step has completed.
    pdl_wait();
    const int q = warp & 3;
    const int row = m0 + q * 32 + lane;
    bool ok = mbar_wait(accum, 0, g.err);
    ok = __all_sync(0xffffffffu, ok && *(volatile int*)g.err == DEV_OK);   // warp-uniform
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16);
      const uint32_t* Bc32 = (const uint32_t*)g.Bcur;
      uint32_t* Bn32 = (uint32_t*)g.Bnext;
      const long kw = g.kpad / 2;                 // 32-bit words per B row
      const long slice_words = g.npad * kw;
      const bool use_prev = g.fg != 0.0f;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {   // 16 real columns (8 complex) per pass
        float l0[16], l1[16], l2[16];
        tmem_ld16(taddr + c0, l0);
        tmem_ld16(taddr + BN + c0, l1);
        tmem_ld16(taddr + 2 * BN + c0, l2);
        const int jb = (n0 + c0) / 2;
        if (row < g.n) {
          // every load of the 8 columns first, then the arithmetic and the stores
          uint32_t wc[8][3], wp[8][3];
          float2 rr[8];
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int j = jb + jj;
            const long w2j = 2L * j * kw + row;
#pragma unroll
            for (int t = 0; t < NSLICE; ++t) {
              wc[jj][t] = j < g.ncols ? Bc32[t * slice_words + w2j] : 0u;
              wp[jj][t] = (use_prev && j < g.ncols) ? Bn32[t * slice_words + w2j] : 0u;
            }
            rr[jj] = (g.R && j < g.ncols) ? g.R[(long)j * g.n + row] : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int j = jb + jj;
            if (j >= g.ncols) continue;
            const float hr = l0[2 * jj] + (l1[2 * jj] + l2[2 * jj]);
            const float hi = l0[2 * jj + 1] + (l1[2 * jj + 1] + l2[2 * jj + 1]);
            const float2 y = join_slices(wc[jj]);
            float ore = fmaf(g.fa, hr, g.fb * y.x);
            float oim = fmaf(g.fa, hi, g.fb * y.y);
            if (use_prev) {
              const float2 p = join_slices(wp[jj]);
              ore = fmaf(g.fg, p.x, ore);
              oim = fmaf(g.fg, p.y, oim);
            }
            if (g.fcol) {   // residual forcing of the corrected recurrence: + fa p_{j-1}(lam_j) R_j
              const float f = g.fcol[j];
              ore = fmaf(f, rr[jj].x, ore);
              oim = fmaf(f, rr[jj].y, oim);
            }
            if (j < g.ncols_next) {
              const long w2j = 2L * j * kw + row;
              store_slices(Bn32, slice_words, w2j, w2j + kw, ore, oim);
            } else {
              g.Yfinal[(long)j * g.n + row] = cmk(to_f64(ore), to_f64(oim));
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    // after a failure the products may still be running: the accumulator barrier arrives when
    // they have completed (bounded), and only then is the TMEM returned
    if (*(volatile int*)g.err != DEV_OK && lane == 0) mbar_drain(accum, 0);
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// One problem: the tensor maps travel in the parameter space.
template <int BN>
__global__ void __launch_bounds__(NTHREADS, 1)
    tc_filter_step_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                          StepArgs g) {
  step_body<BN>(&tmA, &tmB, g, blockIdx.x, blockIdx.y);
}

// Many problems in one launch (one recurrence step of every problem of a batch): a device
// table describes each problem (its tensor maps, step arguments and first tile); CTA t takes
// tile t - tile_begin of the problem whose range holds t.
struct alignas(128) GroupDesc {
  CUtensorMap mapA;
  CUtensorMap mapB;
  StepArgs g;
  int tile_begin, mtiles;
};
template <int BN>
__global__ void __launch_bounds__(NTHREADS, 1) tc_filter_group_kernel(const GroupDesc* __restrict__ d, int ngroups) {
  int gi = 0;
  while (gi + 1 < ngroups && d[gi + 1].tile_begin <= (int)blockIdx.x) ++gi;
  const int t = (int)blockIdx.x - d[gi].tile_begin;
  const StepArgs g = d[gi].g;
  if (threadIdx.x == 0) {
    // the descriptors were written to global memory by a copy: order them for the TMA unit
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&d[gi].mapA) : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&d[gi].mapB) : "memory");
  }
  __syncthreads();
  step_body<BN>(&d[gi].mapA, &d[gi].mapB, g, t % d[gi].mtiles, t / d[gi].mtiles);
}

// A recurrence step launch that may start while the previous step finishes (programmatic
// dependent launch; the kernels order their dependent accesses with griddepcontrol.wait).
template <typename... Params, typename... Args>
cudaError_t launch_pdl(void (*kernel)(Params...), dim3 grid, int smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(NTHREADS);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Slices of H' (column-major, Hermitian) as the A operand: A_s[r][2c] = s_s(Re H'[r,c]),
// A_s[r][2c+1] = s_s(Im H'[r,c]), read through the Hermitian symmetry (row r of H' = conj of
// column r, contiguous).  Each entry is rounded to FP32 (integer operations) and split there;
// padding zero.
__global__ void slice_H_kernel(int n, long kpad, long mpad, const cplx* __restrict__ H, __nv_bfloat16* __restrict__ A) {
  const long r = blockIdx.y;
  uint32_t* A32 = (uint32_t*)A;
  const long slice_words = mpad * kpad / 2;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < kpad / 2; c += (long)gridDim.x * blockDim.x) {
    uint32_t re[3] = {0, 0, 0}, im[3] = {0, 0, 0};
    if (r < n && c < n) {
      const cplx h = H[c + r * (long)n];   // H'[c, r] = conj(H'[r, c])
      split3f(f32_rn(h.x), re[0], re[1], re[2]);
      split3f(f32_rn(-h.y), im[0], im[1], im[2]);
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) A32[t * slice_words + r * (kpad / 2) + c] = pack_lo_hi(re[t], im[t]);
  }
}

// Y (n x ncols, column-major) -> B slices (rows 2j, 2j+1 of each slice; K interleaved); padding zero.
__global__ void slice_Y_kernel(int n, int ncols, long kpad, long npad, const cplx* __restrict__ Y,
                               __nv_bfloat16* __restrict__ B) {
  const long j = blockIdx.y;   // complex column, < npad / 2
  uint32_t* B32 = (uint32_t*)B;
  const long kw = kpad / 2, slice_words = npad * kw;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < kw; c += (long)gridDim.x * blockDim.x) {
    if (j < ncols && c < n) {
      const cplx y = Y[c + j * (long)n];
      store_slices(B32, slice_words, 2 * j * kw + c, (2 * j + 1) * kw + c, f32_rn(y.x), f32_rn(y.y));
    } else {
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        B32[t * slice_words + 2 * j * kw + c] = 0u;
        B32[t * slice_words + (2 * j + 1) * kw + c] = 0u;
      }
    }
  }
}

// R = Z - Yhat diag(lam) (FP64, then kept in FP32: it only ever forces D, which is as small as
// R); D_1 = fa_1 R: its slices for the next product, or its FP64 value for a degree-1 column.
__global__ void refine_first_kernel(int n, int ncols, long kpad, long npad, const cplx* __restrict__ Z,
                                    const cplx* __restrict__ Y, const double* __restrict__ lam, float fa1,
                                    const int* __restrict__ deg, float2* __restrict__ R, cplx* __restrict__ Dout,
                                    __nv_bfloat16* __restrict__ B) {
  const long j = blockIdx.y;
  const double l = lam[j];
  const bool more = deg[j] > 1;
  uint32_t* B32 = (uint32_t*)B;
  const long kw = kpad / 2, slice_words = npad * kw;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
    const long e = j * n + c;
    const cplx z = Z[e], y = Y[e];
    const float2 r = make_float2(f32_rn(z.x - l * y.x), f32_rn(z.y - l * y.y));
    R[e] = r;
    const float dre = fa1 * r.x, dim = fa1 * r.y;
    if (more) store_slices(B32, slice_words, 2 * j * kw + c, (2 * j + 1) * kw + c, dre, dim);
    else Dout[e] = cmk(to_f64(dre), to_f64(dim));
  }
}

// Yhat_j <- Yhat_j p_{m_j}(lam_j) + D_{m_j}
__global__ void refine_combine_kernel(int n, cplx* __restrict__ Y, const cplx* __restrict__ D,
                                      const double* __restrict__ pm, const int* __restrict__ deg) {
  const long j = blockIdx.y;
  if (deg[j] < 1) return;
  const double p = pm[j];
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
    const long e = j * n + c;
    const cplx y = Y[e], d = D[e];
    Y[e] = cmk(p * y.x + d.x, p * y.y + d.y);
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

bool make_map(CUtensorMap* m, void* ptr, long rows, long cols, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

long round_up(long x, long m) { return (x + m - 1) / m * m; }
}  // namespace

struct TcFilter {
  int n = 0, k = 0;
  long kpad = 0, mpad = 0, npad = 0;
  __nv_bfloat16* A = nullptr;
  __nv_bfloat16* B[2] = {nullptr, nullptr};
  cplx* Dout = nullptr;              // corrected recurrence: D_{m_j} of every column
  float2* R = nullptr;               // corrected recurrence forcing
  float* tabf = nullptr;             // forcing scales per step and column
  double* pm = nullptr;              // final p_{m_j}(lam_j) per column
  int* deg = nullptr;
  int tab_cap = 0, k_cap = 0;
  int* err = nullptr;
  CUtensorMap mapA, mapB[2][2];      // B maps per tile width (32, 64) and buffer
  cudaEvent_t ev[2] = {nullptr, nullptr};   // around the step launches
  double ms_steps = 0.0;
  long long col_steps = 0;
  // tile-width trials awaiting their timing: (shape key, width index, events)
  struct Trial {
    long long key;
    int v;
    cudaEvent_t a, b;
  };
  std::vector<Trial> trials;
  std::vector<cudaEvent_t> ev_pool;
};

namespace {
// ---- autotuner of the tile width --------------------------------------------------------
// The two widths compute every output element in the same order (the same K loop, one
// element per accumulator column), so they give bit-identical results and the choice can
// follow measured time alone.  Per launch shape (row tiles, columns) each width is timed on
// its first use (CUDA events on the launching stream, read at the next synchronisation) and
// the faster one is kept for the rest of the process.
constexpr int NVAR = 2;
constexpr int VAR_BN[NVAR] = {32, 64};
struct Tune {
  float ms[NVAR] = {-1.f, -1.f};
  int choice = -1;
};
std::mutex g_tune_mu;
std::map<long long, Tune> g_tune;

// width index for the next launch of shape `key`; *trial = true when this launch is a timed trial
int tune_pick(long long key, bool* trial) {
  // tests pin a width (CHFSI_FILTER_WIDTH=32 or 64) to compare the two
  if (const char* w = getenv("CHFSI_FILTER_WIDTH")) {
    *trial = false;
    return atoi(w) == 32 ? 0 : 1;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  Tune& t = g_tune[key];
  if (t.choice >= 0) {
    *trial = false;
    return t.choice;
  }
  for (int v = NVAR - 1; v >= 0; --v)
    if (t.ms[v] < 0.f) {
      *trial = true;
      return v;
    }
  *trial = false;
  return 1;
}
void tune_record(long long key, int v, float ms) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  Tune& t = g_tune[key];
  if (t.choice >= 0 || ms <= 0.f) return;
  if (t.ms[v] < 0.f || ms < t.ms[v]) t.ms[v] = ms;
  bool all = true;
  for (int q = 0; q < NVAR; ++q) all = all && t.ms[q] > 0.f;
  if (all) t.choice = t.ms[0] < t.ms[1] ? 0 : 1;
}

template <int BN>
cudaError_t set_attr_once() {
  static bool done = false;   // benign race: the attribute is idempotent
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(tc_filter_step_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Tile<BN>::SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_filter_group_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Tile<BN>::SMEM_BYTES);
  done = e == cudaSuccess;
  return e;
}

cudaEvent_t pool_ev(TcFilter* f) {
  if (!f->ev_pool.empty()) {
    cudaEvent_t e = f->ev_pool.back();
    f->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
// after a synchronisation: the trials' times go to the tuner
void flush_trials(TcFilter* f) {
  for (auto& t : f->trials) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) tune_record(t.key, t.v, ms);
    f->ev_pool.push_back(t.a);
    f->ev_pool.push_back(t.b);
  }
  f->trials.clear();
}
}  // namespace

TcFilter* tc_filter_new() { return new TcFilter(); }

double tc_filter_take_ms(TcFilter* f, long long* col_steps) {
  const double ms = f->ms_steps;
  if (col_steps) *col_steps = f->col_steps;
  f->ms_steps = 0.0;
  f->col_steps = 0;
  return ms;
}

void tc_filter_free(TcFilter* f) {
  if (!f) return;
  cudaFree(f->A);
  cudaFree(f->B[0]);
  cudaFree(f->B[1]);
  cudaFree(f->Dout);
  cudaFree(f->R);
  cudaFree(f->tabf);
  cudaFree(f->pm);
  cudaFree(f->deg);
  cudaFree(f->err);
  for (int i = 0; i < 2; ++i)
    if (f->ev[i]) cudaEventDestroy(f->ev[i]);
  for (auto& t : f->trials) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto e : f->ev_pool) cudaEventDestroy(e);
  delete f;
}

static chfsi_status tc_ensure(TcFilter* f, int n, int k, cudaStream_t s) {
  if (n == f->n && k <= f->k && f->A) return CHFSI_OK;
  // cudaFree is not guaranteed to wait for queued kernels that use these buffers, and the
  // memory can go to another thread's allocation at once: drain the stream first
  CHFSI_CUDA_TRY(cudaStreamSynchronize(s));
  cudaFree(f->A);
  cudaFree(f->B[0]);
  cudaFree(f->B[1]);
  cudaFree(f->Dout);
  cudaFree(f->R);
  f->A = f->B[0] = f->B[1] = nullptr;
  f->Dout = nullptr;
  f->R = nullptr;
  f->n = n;
  f->k = k;
  f->kpad = round_up(2L * n, BK);
  f->mpad = round_up(n, BM);
  f->npad = round_up(2L * k, 64);   // a multiple of every tile width
  CHFSI_CUDA_TRY(cudaMalloc(&f->A, sizeof(__nv_bfloat16) * 3 * f->mpad * f->kpad));
  for (int i = 0; i < 2; ++i) {
    CHFSI_CUDA_TRY(cudaMalloc(&f->B[i], sizeof(__nv_bfloat16) * 3 * f->npad * f->kpad));
    // stream-ordered: the caller's stream may be a non-blocking one, which the legacy default
    // stream (a plain cudaMemset) does not order against the filter launches that follow
    CHFSI_CUDA_TRY(cudaMemsetAsync(f->B[i], 0, sizeof(__nv_bfloat16) * 3 * f->npad * f->kpad, s));
  }
  CHFSI_CUDA_TRY(cudaMalloc(&f->Dout, sizeof(cplx) * (size_t)n * k));
  CHFSI_CUDA_TRY(cudaMalloc(&f->R, sizeof(float2) * (size_t)n * k));
  if (!f->err) CHFSI_CUDA_TRY(cudaMalloc(&f->err, sizeof(int)));
  if (!make_map(&f->mapA, f->A, 3 * f->mpad, f->kpad, BM)) return CHFSI_ERR_CUDA;
  for (int v = 0; v < NVAR; ++v)
    for (int i = 0; i < 2; ++i)
      if (!make_map(&f->mapB[v][i], f->B[i], 3 * f->npad, f->kpad, VAR_BN[v])) return CHFSI_ERR_CUDA;
  CHFSI_CUDA_TRY(set_attr_once<32>());
  CHFSI_CUDA_TRY(set_attr_once<64>());
  return CHFSI_OK;
}

// Everything of a filter call before the recurrence steps: buffers, the slices of H' and of
// the start block (or, corrected form, R and D_1).
static chfsi_status tc_prologue(TcFilter* f, cudaStream_t s, int n, const cplx* H, cplx* Y, const int* cnt, int mmax,
                                const double* fa, const TcRefine* ref) {
  const int k = cnt[1];
  chfsi_status st = tc_ensure(f, n, k, s);
  if (st != CHFSI_OK) return st;
  CHFSI_CUDA_TRY(cudaMemsetAsync(f->err, 0, sizeof(int), s));
  {
    dim3 grid((unsigned)((f->kpad / 2 + 255) / 256), (unsigned)f->mpad);
    slice_H_kernel<<<grid, 256, 0, s>>>(n, f->kpad, f->mpad, H, f->A);
    count_launch(1);
  }
  const unsigned cgrid = (unsigned)std::min<long>((n + 255) / 256, 16);
  if (ref) {
    // device tables: rows j = 1..mmax of fa[j] p_{j-1}(lam_i) (FP32), and p_{m_i}(lam_i) (FP64)
    if (f->tab_cap < (mmax + 1) * k || f->k_cap < k) CHFSI_CUDA_TRY(cudaStreamSynchronize(s));
    if (f->tab_cap < (mmax + 1) * k) {
      cudaFree(f->tabf);
      f->tabf = nullptr;
      CHFSI_CUDA_TRY(cudaMalloc(&f->tabf, sizeof(float) * (size_t)(mmax + 1) * k));
      f->tab_cap = (mmax + 1) * k;
    }
    if (f->k_cap < k) {
      cudaFree(f->pm);
      cudaFree(f->deg);
      f->pm = nullptr;
      f->deg = nullptr;
      CHFSI_CUDA_TRY(cudaMalloc(&f->pm, sizeof(double) * (size_t)k));
      CHFSI_CUDA_TRY(cudaMalloc(&f->deg, sizeof(int) * (size_t)k));
      f->k_cap = k;
    }
    std::vector<float> htab((size_t)(mmax + 1) * k, 0.0f);
    std::vector<double> hpm(k, 0.0);
    for (int j = 1; j <= mmax; ++j)
      for (int i = 0; i < k; ++i) htab[(size_t)j * k + i] = (float)(fa[j] * ref->ptab[(size_t)(j - 1) * k + i]);
    for (int i = 0; i < k; ++i) hpm[i] = ref->ptab[(size_t)ref->deg[i] * k + i];
    CHFSI_CUDA_TRY(cudaMemcpyAsync(f->tabf, htab.data(), sizeof(float) * htab.size(), cudaMemcpyHostToDevice, s));
    CHFSI_CUDA_TRY(cudaMemcpyAsync(f->pm, hpm.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s));
    CHFSI_CUDA_TRY(cudaMemcpyAsync(f->deg, ref->deg, sizeof(int) * k, cudaMemcpyHostToDevice, s));
    dim3 g1(cgrid, (unsigned)k);
    refine_first_kernel<<<g1, 256, 0, s>>>(n, k, f->kpad, f->npad, ref->Z, Y, ref->lam, (float)fa[1], f->deg, f->R,
                                           f->Dout, f->B[1]);
    count_launch(1);
  } else {
    dim3 gy((unsigned)((f->kpad / 2 + 255) / 256), (unsigned)(f->npad / 2));
    slice_Y_kernel<<<gy, 256, 0, s>>>(n, k, f->kpad, f->npad, Y, f->B[0]);
    count_launch(1);
  }
  return CHFSI_OK;
}

static StepArgs step_args(TcFilter* f, int n, cplx* Y, const int* cnt, int mmax, int j, const double* fa,
                          const double* fb, const double* fg, const TcRefine* ref) {
  const int k = cnt[1];
  StepArgs g{};
  g.n = n;
  g.mtiles = (int)(f->mpad / BM);
  g.ncols = cnt[j];
  g.ncols_next = j < mmax ? cnt[j + 1] : 0;
  g.kblocks = (int)(f->kpad / BK);
  g.kpad = f->kpad;
  g.npad = f->npad;
  g.Bcur = f->B[(j - 1) & 1];
  g.Bnext = f->B[j & 1];
  g.Yfinal = ref ? f->Dout : Y;
  g.fa = (float)fa[j];
  g.fb = (float)fb[j];
  g.fg = (float)((j >= (ref ? 3 : 2)) ? fg[j] : 0.0);   // Y_{-1} = 0; in the corrected form D_0 = 0
  g.R = ref ? f->R : nullptr;
  g.fcol = ref ? f->tabf + (size_t)j * k : nullptr;
  g.err = f->err;
  return g;
}

static chfsi_status tc_epilogue_launch(TcFilter* f, cudaStream_t s, int n, cplx* Y, int k, const TcRefine* ref) {
  if (ref) {
    const unsigned cgrid = (unsigned)std::min<long>((n + 255) / 256, 16);
    dim3 g2(cgrid, (unsigned)k);
    refine_combine_kernel<<<g2, 256, 0, s>>>(n, Y, f->Dout, f->pm, f->deg);
    count_launch(1);
  }
  return CHFSI_OK;
}

chfsi_status tc_filter_run(TcFilter* f, cudaStream_t s, int n, const cplx* H, cplx* Y, const int* cnt, int mmax,
                           const double* fa, const double* fb, const double* fg, const TcRefine* ref) {
  if (mmax < 1 || cnt[1] < 1) return CHFSI_OK;
  const int k = cnt[1];
  chfsi_status st = tc_prologue(f, s, n, H, Y, cnt, mmax, fa, ref);
  if (st != CHFSI_OK) return st;
  if (!f->ev[0]) {
    CHFSI_CUDA_TRY(cudaEventCreate(&f->ev[0]));
    CHFSI_CUDA_TRY(cudaEventCreate(&f->ev[1]));
  }
  CHFSI_CUDA_TRY(cudaEventRecord(f->ev[0], s));
  for (int j = ref ? 2 : 1; j <= mmax; ++j) {
    const StepArgs g = step_args(f, n, Y, cnt, mmax, j, fa, fb, fg, ref);
    f->col_steps += cnt[j];
    const long long key = ((long long)g.mtiles << 32) | (long long)(2 * cnt[j]);
    bool trial = false;
    const int v = tune_pick(key, &trial);
    cudaEvent_t ta = nullptr, tb = nullptr;
    if (trial) {
      ta = pool_ev(f);
      tb = pool_ev(f);
      CHFSI_CUDA_TRY(cudaEventRecord(ta, s));
    }
    const int BNv = VAR_BN[v];
    dim3 grid((unsigned)g.mtiles, (unsigned)((2L * cnt[j] + BNv - 1) / BNv));
    if (v == 0)
      CHFSI_CUDA_TRY(launch_pdl(tc_filter_step_kernel<32>, grid, Tile<32>::SMEM_BYTES, s, f->mapA,
                                f->mapB[0][(j - 1) & 1], g));
    else
      CHFSI_CUDA_TRY(launch_pdl(tc_filter_step_kernel<64>, grid, Tile<64>::SMEM_BYTES, s, f->mapA,
                                f->mapB[1][(j - 1) & 1], g));
    count_launch(1);
    if (trial) {
      CHFSI_CUDA_TRY(cudaEventRecord(tb, s));
      f->trials.push_back({key, v, ta, tb});
    }
  }
  CHFSI_CUDA_TRY(cudaEventRecord(f->ev[1], s));
  TRY_CHFSI(tc_epilogue_launch(f, s, n, Y, k, ref));
  int h = 0;
  CHFSI_CUDA_TRY(cudaMemcpyAsync(&h, f->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CHFSI_CUDA_TRY(cudaStreamSynchronize(s));
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, f->ev[0], f->ev[1]) == cudaSuccess) f->ms_steps += ms;
  flush_trials(f);
  if (h == DEV_ERR_TIMEOUT) return CHFSI_ERR_TIMEOUT;
  if (h != DEV_OK) return CHFSI_ERR_NUMERIC;
  return CHFSI_OK;
}

// ---- batch: one grouped launch per recurrence step for every problem ----------------------
struct TcBatch {
  GroupDesc* d = nullptr;          // device: descriptors of every step, step after step
  size_t cap = 0;
  std::vector<GroupDesc> h;
  cudaGraphExec_t exec = nullptr;  // the captured step launches, updated in place when possible
  cudaEvent_t ev[2] = {nullptr, nullptr};
  std::vector<int> trial_v;
  std::vector<long long> trial_key;
  std::vector<cudaEvent_t> trial_ev;
};

TcBatch* tc_batch_new() { return new TcBatch(); }
void tc_batch_free(TcBatch* b) {
  if (!b) return;
  cudaFree(b->d);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (int i = 0; i < 2; ++i)
    if (b->ev[i]) cudaEventDestroy(b->ev[i]);
  for (auto e : b->trial_ev) cudaEventDestroy(e);
  delete b;
}

chfsi_status tc_filter_run_batch(TcBatch* b, cudaStream_t s, const TcJob* jobs, int njobs, double* ms_steps,
                                 bool use_graph) {
  if (njobs <= 0) return CHFSI_OK;
  int jmax = 0;
  for (int p = 0; p < njobs; ++p) {
    const TcJob& J = jobs[p];
    if (J.mmax < 1 || J.cnt[1] < 1) continue;
    TRY_CHFSI(tc_prologue(J.f, s, J.n, J.H, J.Y, J.cnt, J.mmax, J.fa, J.ref));
    jmax = std::max(jmax, J.mmax);
  }
  // descriptors of all steps: for step j the problems with j in [start, mmax]
  b->h.clear();
  std::vector<int> step_begin, step_count, step_tiles;
  std::vector<long long> step_key;
  for (int j = 1; j <= jmax; ++j) {
    step_begin.push_back((int)b->h.size());
    int tiles = 0, cnt_groups = 0;
    long long key = 1LL << 62;
    for (int p = 0; p < njobs; ++p) {
      const TcJob& J = jobs[p];
      if (J.mmax < 1 || J.cnt[1] < 1 || j > J.mmax || j < (J.ref ? 2 : 1) || J.cnt[j] < 1) continue;
      GroupDesc d;
      memset(&d, 0, sizeof(d));
      d.g = step_args(J.f, J.n, J.Y, J.cnt, J.mmax, j, J.fa, J.fb, J.fg, J.ref);
      d.mapA = J.f->mapA;
      d.tile_begin = tiles;
      d.mtiles = d.g.mtiles;
      tiles += d.g.mtiles * (int)((2L * J.cnt[j] + 63) / 64);   // counted at width 64 for the key
      key += (long long)d.g.mtiles * 7919 + 2 * J.cnt[j];
      J.f->col_steps += J.cnt[j];
      b->h.push_back(d);
      ++cnt_groups;
    }
    step_count.push_back(cnt_groups);
    step_tiles.push_back(tiles);
    step_key.push_back(key + ((long long)cnt_groups << 40));
  }
  // tile width per step (autotuned on the batch's shape), B maps and tile ranges for that width
  std::vector<int> step_v(jmax), step_grid(jmax);
  std::vector<bool> step_trial(jmax);
  for (int j = 1; j <= jmax; ++j) {
    bool trial = false;
    const int v = step_count[j - 1] ? tune_pick(step_key[j - 1], &trial) : 1;
    step_v[j - 1] = v;
    step_trial[j - 1] = trial;
    int tiles = 0;
    for (int q = 0; q < step_count[j - 1]; ++q) {
      GroupDesc& d = b->h[step_begin[j - 1] + q];
      // the job this descriptor came from: its B buffer of step j
      d.tile_begin = tiles;
      tiles += d.mtiles * (int)((2L * d.g.ncols + VAR_BN[v] - 1) / VAR_BN[v]);
    }
    step_grid[j - 1] = tiles;
  }
  {
    // B maps per descriptor (the job's filter, the buffer read at step j, the chosen width)
    int idx = 0;
    for (int j = 1; j <= jmax; ++j)
      for (int p = 0; p < njobs; ++p) {
        const TcJob& J = jobs[p];
        if (J.mmax < 1 || J.cnt[1] < 1 || j > J.mmax || j < (J.ref ? 2 : 1) || J.cnt[j] < 1) continue;
        b->h[idx++].mapB = J.f->mapB[step_v[j - 1]][(j - 1) & 1];
      }
  }
  const size_t bytes = sizeof(GroupDesc) * std::max<size_t>(1, b->h.size());
  if (b->cap < bytes) {
    CHFSI_CUDA_TRY(cudaStreamSynchronize(s));   // no queued launch may still read the old table
    cudaFree(b->d);
    b->d = nullptr;
    CHFSI_CUDA_TRY(cudaMalloc(&b->d, bytes));
    b->cap = bytes;
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
  }
  CHFSI_CUDA_TRY(cudaMemcpyAsync(b->d, b->h.data(), sizeof(GroupDesc) * b->h.size(), cudaMemcpyHostToDevice, s));
  if (!b->ev[0]) {
    CHFSI_CUDA_TRY(cudaEventCreate(&b->ev[0]));
    CHFSI_CUDA_TRY(cudaEventCreate(&b->ev[1]));
  }
  // the step launches: captured into a graph (re-used through an in-place update when the
  // launch shapes allow), unless a step is a timed autotuning trial
  bool any_trial = false;
  for (int j = 0; j < jmax; ++j) any_trial = any_trial || step_trial[j];
  auto launch_steps = [&](bool timed) -> chfsi_status {
    for (int j = 1; j <= jmax; ++j) {
      if (!step_count[j - 1]) continue;
      cudaEvent_t ta = nullptr, tb = nullptr;
      if (timed && step_trial[j - 1]) {
        ta = nullptr;
        CHFSI_CUDA_TRY(cudaEventCreate(&ta));
        CHFSI_CUDA_TRY(cudaEventCreate(&tb));
        CHFSI_CUDA_TRY(cudaEventRecord(ta, s));
      }
      const GroupDesc* dj = b->d + step_begin[j - 1];
      const int ng = step_count[j - 1];
      if (step_v[j - 1] == 0)
        CHFSI_CUDA_TRY(launch_pdl(tc_filter_group_kernel<32>, dim3(step_grid[j - 1]), Tile<32>::SMEM_BYTES, s, dj, ng));
      else
        CHFSI_CUDA_TRY(launch_pdl(tc_filter_group_kernel<64>, dim3(step_grid[j - 1]), Tile<64>::SMEM_BYTES, s, dj, ng));
      count_launch(1);
      if (ta) {
        CHFSI_CUDA_TRY(cudaEventRecord(tb, s));
        b->trial_ev.push_back(ta);
        b->trial_ev.push_back(tb);
        b->trial_v.push_back(step_v[j - 1]);
        b->trial_key.push_back(step_key[j - 1]);
      }
    }
    return CHFSI_OK;
  };
  CHFSI_CUDA_TRY(cudaEventRecord(b->ev[0], s));
  // only a created stream can be captured (not the legacy or per-thread default stream), and
  // not one that is being captured already
  cudaStreamCaptureStatus cap_now = cudaStreamCaptureStatusNone;
  const bool capturable = s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread &&
                          cudaStreamIsCapturing(s, &cap_now) == cudaSuccess && cap_now == cudaStreamCaptureStatusNone;
  cudaGetLastError();
  bool captured = false;
  if (use_graph && capturable && !any_trial &&
      cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    captured = true;
    cudaGraph_t graph = nullptr;
    chfsi_status lst = launch_steps(false);
    cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (cudaStreamIsCapturing(s, &cap_now) == cudaSuccess && cap_now != cudaStreamCaptureStatusNone) {
      cudaGraph_t g2 = nullptr;   // never leave the caller's stream capturing
      cudaStreamEndCapture(s, &g2);
      if (g2) cudaGraphDestroy(g2);
    }
    if (lst != CHFSI_OK) {
      if (graph) cudaGraphDestroy(graph);
      return lst;
    }
    // nothing ran during the capture: if the graph cannot be made, launch the steps directly
    bool ready = ce == cudaSuccess && graph != nullptr;
    if (ready && b->exec) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(b->exec, graph, &info) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
      }
    }
    if (ready && !b->exec && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) {
      cudaGetLastError();
      b->exec = nullptr;
      ready = false;
    }
    if (graph) cudaGraphDestroy(graph);
    if (ready) CHFSI_CUDA_TRY(cudaGraphLaunch(b->exec, s));
    else captured = false;
  }
  if (!captured) {
    cudaGetLastError();
    TRY_CHFSI(launch_steps(true));
  }
  CHFSI_CUDA_TRY(cudaEventRecord(b->ev[1], s));
  for (int p = 0; p < njobs; ++p) {
    const TcJob& J = jobs[p];
    if (J.mmax < 1 || J.cnt[1] < 1) continue;
    TRY_CHFSI(tc_epilogue_launch(J.f, s, J.n, J.Y, J.cnt[1], J.ref));
  }
  // status words of every problem, one synchronisation
  std::vector<int> herr(njobs, 0);
  for (int p = 0; p < njobs; ++p)
    if (jobs[p].mmax >= 1 && jobs[p].cnt[1] >= 1)
      CHFSI_CUDA_TRY(cudaMemcpyAsync(&herr[p], jobs[p].f->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CHFSI_CUDA_TRY(cudaStreamSynchronize(s));
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]) == cudaSuccess) {
    if (ms_steps) *ms_steps += ms;
    // each problem's share of the grouped launches, by its executed work (columns x n^2)
    double tot = 0.0;
    std::vector<double> w(njobs, 0.0);
    for (int p = 0; p < njobs; ++p) {
      const TcJob& J = jobs[p];
      for (int j = J.ref ? 2 : 1; j <= J.mmax && J.cnt[1] >= 1; ++j) w[p] += (double)J.cnt[j] * J.n * J.n;
      tot += w[p];
    }
    for (int p = 0; p < njobs; ++p)
      if (tot > 0.0) jobs[p].f->ms_steps += ms * (w[p] / tot);
  }
  for (size_t q = 0; q < b->trial_v.size(); ++q) {
    float tms = 0.f;
    if (cudaEventElapsedTime(&tms, b->trial_ev[2 * q], b->trial_ev[2 * q + 1]) == cudaSuccess)
      tune_record(b->trial_key[q], b->trial_v[q], tms);
  }
  for (auto e : b->trial_ev) cudaEventDestroy(e);
  b->trial_ev.clear();
  b->trial_v.clear();
  b->trial_key.clear();
  for (int p = 0; p < njobs; ++p) {
    if (herr[p] == DEV_ERR_TIMEOUT) return CHFSI_ERR_TIMEOUT;
    if (herr[p] != DEV_OK) return CHFSI_ERR_NUMERIC;
  }
  return CHFSI_OK;
}
