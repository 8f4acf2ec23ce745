// FP64-accurate complex GEMM on the BF16 tensor cores.
//
// GB300 executes FP64 at ~1/1700 of its dense BF16 rate, so the FP64 products around the
// filter (reduction to standard form, Rayleigh-Ritz, QR, back-transform) run as an
// error-free digit expansion on tcgen05 (after Ozaki, Ogita, Oishi & Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix multiplication
// and its applications", Numer. Algorithms 2012):
//
//  * the complex product is a real GEMM through [Re A | Im A] (K interleaved) times
//    [[Re B, Im B], [-Im B, Re B]] (columns interleaved);
//  * every row of the real A (every column pair of the real B) is scaled by a power of two
//    sigma >= its largest magnitude and expanded into S = 12 signed digits, a top digit of
//    7 bits and eleven of 5 bits: x = sigma 2^-6 sum_s 2^(-5 s) d_s, |d_0| <= 64,
//    |d_s| <= 16 (exact in BF16);
//  * digit products are integers; all products of one significance level L = s + t
//    (L <= S - 1, 78 products) accumulate in their own TMEM accumulator.  With K <= 3584
//    real terms per pass every partial sum is an integer below 2^24 (level 0: 64 * 64 per
//    term; level L: at most 2 * 64 * 16 + (L - 1) * 256), so the FP32 accumulation is exact
//    even though the tensor core truncates;
//  * the epilogue combines the 12 levels exactly in two 64-bit integers and rounds once to
//    FP64 with the scales applied: each entry carries 61 bits relative to its row (column)
//    scale before that rounding -- the
//    expansion's error is relative to the largest entry of the row, not to the entry, and
//    Hermitian matrices with a wide spectrum (large diagonal, small off-diagonal) need the
//    extra digits to stay at FP64 accuracy.  Longer K runs in passes (split-K) whose FP64
//    partial results a fixed-order reduction sums;
//  * the slicing kernels write every 128 x 16 (A) and 32 x 16 (B) digit tile as the exact
//    shared-memory image the MMA reads (K-major, 32-byte swizzle), ordered so that the twelve
//    slices of one K block are adjacent: a pipeline stage is two contiguous bulk copies
//    (48 KB + 12 KB) instead of 24 tensor-map copies of 32-byte rows, whose per-row requests
//    had saturated the SM's request path to L2;
//  * the products of A slice s with B slices 0 .. S-1-s land in the adjacent level columns
//    [32 s, 32 S) of TMEM, so they are one wide MMA (N up to 256, split above): 16
//    instructions per K block instead of 78.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <utility>

#include "ozaki.cuh"

void count_launch(unsigned long long n);

namespace {

constexpr int SLICES = 12;       // digits per operand: a 7-bit top digit and 11 of 5 bits (61 bits)
constexpr int DIGIT_BITS = 5;    // lower digits: |d| <= 16; top digit: |d| <= 64 (exact in BF16)
constexpr int TOP_SHIFT = 61;    // |x| 2^(61 - e) < 2^61: the integer the digits expand
constexpr int LEVELS = SLICES;   // kept levels L = s + t = 0 .. SLICES-1
// real K per pass: level 0 sums 64 * 64 per term, level L >= 1 at most 2 * 64 * 16 + (L - 1) * 256
// = 4608 at L = 11; 4608 * 3584 < 2^24
constexpr int KPASS = 3584;
constexpr int BM = 128, BN = 32, BK = 16;   // BK bf16 = 32-byte rows, one MMA K step
constexpr int STAGES = 3;
constexpr int A_TILE = BM * BK * 2;           // 4 KB
constexpr int B_TILE = BN * BK * 2;           // 1 KB
constexpr int STAGE_BYTES = SLICES * (A_TILE + B_TILE);
constexpr int NBARS = 2 * STAGES + 1;       // full, empty, accum
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 512;
static_assert(8 * NBARS + 4 <= 512, "barrier area");
constexpr int TMEM_COLS = 512;                // LEVELS * BN = 384 used
constexpr int NTHREADS = 192;
constexpr long WAIT_LIMIT = 1L << 24;
static_assert(LEVELS * BN <= TMEM_COLS, "TMEM");
static_assert(STAGE_BYTES % 1024 == 0, "stage alignment");
static_assert(SMEM_BYTES <= 232448, "shared memory");
static_assert((2L * 64 * 16 + (LEVELS - 2) * 256L) * KPASS < (1L << 24), "exact accumulation");
static_assert(64L * 64 * KPASS < (1L << 24), "exact accumulation (level 0)");

struct OzArgs {
  int M, N2;              // rows, real columns (2N)
  int kblocks;            // K blocks (BK real each) in total
  int per;                // K blocks per split (<= KPASS / BK keeps each split exact)
  int tri;                // GemmTri flags in complex units
  const int* rowexp;      // per row of A: exponent e (sigma = 2^e)
  const int* colexp;      // per complex column of B
  // digit tiles: [row tile][K block][slice], each the shared-memory image of one operand tile
  const __nv_bfloat16* A;
  const __nv_bfloat16* B;
  // output: splits > 1 -> partial[z] (M x N complex, FP64); else C = alpha v + beta C
  cplx* C; long ldc;
  cplx alpha, beta;
  cplx* partial;          // [splits][M*N]
  int splits;
  int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
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
// Bounded wait without the early exit on a raised error word: used after a failure, to let
// work already issued (copies into this CTA's shared memory, products) complete.
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity) {
  for (long i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  for (long i = 0; i < WAIT_LIMIT; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 255) == 255 && *(volatile int*)err != DEV_OK) return false;
  }
  atomicExch(err, DEV_ERR_TIMEOUT);
  return false;
}
// one contiguous global -> shared copy (16-byte aligned, size a multiple of 16) on the TMA engine
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// K-major operand, 32-byte swizzle: 8-row atoms of 256 B
__device__ __forceinline__ uint64_t umma_desc32(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(256 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)6 << 61;    // SWIZZLE_32B
  return d;
}
// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B (both K-major), M = BM, N = n
__host__ __device__ constexpr uint32_t idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}
__device__ __forceinline__ void umma_ss(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc_n,
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

// Programmatic dependent launch between the stages of one product (slicing -> products ->
// split-K sum): a kernel's launch and prologue overlap the end of the kernel before it.
// griddepcontrol.wait returns once the preceding grid has completed and its writes are
// visible (at once without a programmatic predecessor); launch_dependents is issued only
// after that wait, so no grid runs ahead of one two launches back.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// 2^x as a double: the exponent field directly in the normal range, ldexp outside it
__device__ __forceinline__ double pow2(int x) {
  if (x >= -1022 && x <= 1023) return __longlong_as_double((long long)(x + 1023) << 52);
  return ldexp(1.0, x);
}

__global__ void __launch_bounds__(NTHREADS, 1)
    ozaki_kernel(OzArgs g) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* base_ptr = smem_raw + (base - raw);
  const uint32_t bars = base + STAGES * STAGE_BYTES;
  uint32_t* tmem_slot = (uint32_t*)(base_ptr + STAGES * STAGE_BYTES + 8 * NBARS);
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (STAGES + s); };
  const uint32_t accum = bars + 8u * (2 * STAGES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;        // real column offset
  const int z = blockIdx.z;

  // K-block range: this split, pruned by the triangular structure of the tile (complex units
  // -> real K = 2 * complex K)
  int kb0 = z * g.per, kb1 = min(g.kblocks, kb0 + g.per);
  {
    int kc_begin = 0, kc_end = 1 << 30;
    const int cm0 = m0, cm1 = m0 + BM, cn0 = n0 / 2, cn1 = (n0 + BN) / 2;
    if (g.tri & TRI_A_LOWER) kc_end = min(kc_end, cm1);
    if (g.tri & TRI_B_UPPER) kc_end = min(kc_end, cn1);
    if (g.tri & TRI_A_UPPER) kc_begin = max(kc_begin, cm0);
    if (g.tri & TRI_B_LOWER) kc_begin = max(kc_begin, cn0);
    kb0 = max(kb0, (2 * kc_begin) / BK);
    if (kc_end < (1 << 30)) kb1 = min(kb1, (2 * kc_end + BK - 1) / BK);
  }
  const int nkb = max(0, kb1 - kb0);
  // output tile strictly above the diagonal of a lower-triangle-only product: nothing to do
  // (uniform over the CTA, before any barrier or TMEM allocation)
  if ((g.tri & TRI_C_LOWER) && m0 + BM - 1 < n0 / 2) return;

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
  pdl_wait();   // the digit tiles, exponents and C come from earlier launches
  pdl_trigger();

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < nkb; ++i) {
        const int s = i % STAGES;
        const uint32_t ph = (i / STAGES) & 1;
        if (!mbar_wait(empty(s), ph ^ 1, g.err)) break;
        mbar_expect_tx(full(s), STAGE_BYTES);
        const uint32_t st = base + s * STAGE_BYTES;
        // the stage's twelve A tiles and twelve B tiles are each one contiguous run
        const long kb = kb0 + i;
        bulk_load(st, g.A + ((long)blockIdx.x * g.kblocks + kb) * (SLICES * BM * BK), SLICES * A_TILE, full(s));
        bulk_load(st + SLICES * A_TILE, g.B + ((long)blockIdx.y * g.kblocks + kb) * (SLICES * BN * BK),
                  SLICES * B_TILE, full(s));
        issued = i + 1;
      }
      // After a failure the MMA issuer may have abandoned stages whose copies are still in
      // flight into this CTA's shared memory: wait until each issued stage has landed (the
      // latest phase of each stage is the one checked) before the CTA may exit.
      if (*(volatile int*)g.err != DEV_OK)
        for (int i = std::max(0, issued - STAGES); i < issued; ++i) mbar_drain(full(i % STAGES), (i / STAGES) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      for (int i = 0; i < nkb; ++i) {
        const int s = i % STAGES;
        const uint32_t ph = (i / STAGES) & 1;
        if (!mbar_wait(full(s), ph, g.err)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = base + s * STAGE_BYTES;
        // The B digit tiles of the stage lie one after another (slice t at rows 32 t of one
        // K-major operand), and level L = s + t of the products with A slice s sits in TMEM
        // columns 32 L.  So all products of A slice s are one wide MMA: B rows [0, 32 (S - s))
        // into columns [32 s, 32 S), split at N = 256.  Sixteen instructions per K block; the
        // first (s = 0) covers every level and starts the accumulation.
        const uint64_t da0 = umma_desc32(st), db0 = umma_desc32(st + SLICES * A_TILE);
        const uint32_t first = i != 0;
#pragma unroll
        for (int sa = 0; sa < SLICES; ++sa) {
          constexpr int NMAX = 256;
          const int ntot = BN * (LEVELS - sa);
          const int n1 = ntot < NMAX ? ntot : NMAX;
          const uint64_t da = da0 + (uint64_t)((sa * A_TILE) >> 4);
          const uint32_t acc = sa == 0 ? first : 1u;
          umma_ss(tmem + (uint32_t)(sa * BN), da, db0, idesc(n1), acc);
          if (ntot > NMAX)
            umma_ss(tmem + (uint32_t)(sa * BN + NMAX), da, db0 + (uint64_t)((NMAX * BK * 2) >> 4), idesc(ntot - NMAX),
                    acc);
        }
        umma_commit(empty(s));
      }
      umma_commit(accum);
    }
  } else {
    const int q = warp & 3;                 // TMEM lanes 32 q .. 32 q + 31 belong to this warp
    const int row = m0 + q * 32 + lane;
    bool ok = true;
    if (nkb > 0) ok = mbar_wait(accum, 0, g.err);
    ok = __all_sync(0xffffffffu, ok && *(volatile int*)g.err == DEV_OK);
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      // The level accumulators hold exact integers (|acc_L| < 2^24).  Their combination
      // sum_L acc_L 2^(-5 L) is formed exactly in two 64-bit integers, levels 0..4 in units of
      // 2^-20 and levels 5..11 in units of 2^-55 (|hi| < 2^45, |lo| < 2^55), and rounded to FP64
      // once: two conversions and one FMA per entry instead of twelve FP64 FMAs.
      constexpr int LSPLIT = 5;
      const int er = (row < g.M && g.rowexp[row] > -100000) ? g.rowexp[row] : 0;
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16);
#pragma unroll
      for (int c0 = 0; c0 < BN; c0 += 16) {
        long long hi[16], lo[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) hi[c] = lo[c] = 0;
        if (nkb > 0) {
#pragma unroll
          for (int L = 0; L < LEVELS; ++L) {
            float a[16];
            tmem_ld16(taddr + (uint32_t)(L * BN + c0), a);
#pragma unroll
            for (int c = 0; c < 16; ++c) {
              const long long d = (long long)__float2int_rz(a[c]);
              if (L < LSPLIT) hi[c] += d * (1LL << (DIGIT_BITS * (LSPLIT - 1 - L)));
              else lo[c] += d * (1LL << (DIGIT_BITS * (LEVELS - 1 - L)));
            }
          }
        }
        if (row < g.M) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int j = (n0 + c0) / 2 + jj;
            if (2 * j >= g.N2) continue;
            const int ec = g.colexp[j] > -100000 ? g.colexp[j] : 0;
            const int sc = er + ec - 2 * (TOP_SHIFT - DIGIT_BITS * (SLICES - 1));
            const double wh = pow2(sc - DIGIT_BITS * (LSPLIT - 1)), wl = pow2(sc - DIGIT_BITS * (LEVELS - 1));
            const cplx p = cmk(fma((double)hi[2 * jj], wh, (double)lo[2 * jj] * wl),
                               fma((double)hi[2 * jj + 1], wh, (double)lo[2 * jj + 1] * wl));
            const long N = g.N2 / 2;
            if (g.splits > 1) {
              g.partial[(long)z * g.M * N + row + (long)j * g.M] = p;
            } else {
              cplx o = cmul(g.alpha, p);
              if (g.beta.x != 0.0 || g.beta.y != 0.0) o = cadd(o, cmul(g.beta, g.C[row + (long)j * g.ldc]));
              g.C[row + (long)j * g.ldc] = o;
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    // after a failure the products may still be running: the accumulator barrier (committed
    // after the last issued MMA) arrives when they have completed (bounded), and only then is
    // the TMEM returned
    if (*(volatile int*)g.err != DEV_OK && lane == 0) mbar_drain(accum, 0);
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// op(X)[r, c] of an R x Cn complex matrix stored column-major
__device__ __forceinline__ cplx op_at(const cplx* X, long ld, int op, long r, long c) {
  if (op == OP_N) return X[r + c * ld];
  const cplx v = X[c + r * ld];
  return cmk(v.x, -v.y);
}

__device__ __forceinline__ int exp_of(double x) {   // smallest e with |x| < 2^e (x != 0)
  int e;
  frexp(x, &e);
  return e;
}

// Exponent of the largest magnitude in every row of op(X) (rows = true) or column of op(X)
// (rows = false), op(X) being R x C: 32 x 32 tiles read along the contiguous dimension,
// reduced with shared and global atomicMax (order-independent).  out[] starts at a large
// negative sentinel (all-zero rows keep it).
struct ExpJob {
  int R, C;
  const cplx* X;
  long ld;
  int op;
  bool rows;
  int* out;
  unsigned gx, gy;   // this job's grid
};
__device__ __forceinline__ void exp_tile(int R, int C, const cplx* X, long ld, int op, bool rows, int* out, int bx,
                                         int by) {
  __shared__ int m[32];
  const int r0 = by * 32, c0 = bx * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (threadIdx.x < 32) m[threadIdx.x] = -100000;
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    int a, b;   // element (r0 + a, c0 + b) of op(X)
    if (op == OP_N) { a = tx; b = i; } else { a = i; b = tx; }
    const long r = r0 + a, c = c0 + b;
    if (r < R && c < C) {
      const cplx v = op_at(X, ld, op, r, c);
      int e = -100000;
      if (v.x != 0.0) e = max(e, exp_of(v.x));
      if (v.y != 0.0) e = max(e, exp_of(v.y));
      if (e > -100000) atomicMax(&m[rows ? a : b], e);
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const long idx = (rows ? r0 : c0) + threadIdx.x;
    if (m[threadIdx.x] > -100000 && idx < (rows ? R : C)) atomicMax(out + idx, m[threadIdx.x]);
  }
}
// Both operands' exponents in one launch: blockIdx.z picks the job (A's rows, B's columns).
__global__ void exp_tile_kernel(ExpJob a, ExpJob b) {
  pdl_trigger();   // launched in order after the sentinel fill: the slicing may be scheduled now
  const ExpJob& j = blockIdx.z == 0 ? a : b;
  if (blockIdx.x >= j.gx || blockIdx.y >= j.gy) return;
  exp_tile(j.R, j.C, j.X, j.ld, j.op, j.rows, j.out, blockIdx.x, blockIdx.y);
}

// Digits of x / 2^e (|x| < 2^e):  x = 2^e 2^-6 sum_s 2^(-5 s) d_s with |d_0| <= 64 and
// |d_s| <= 16 (s >= 1).  Integer arithmetic on the FP64 bit pattern: G = round(|x| 2^(61-e))
// < 2^61, then balanced base-32 digits from the least significant up (r = G mod 32 taken in
// [-15, 16], G = (G - r) / 32); what remains after eleven is the top digit.  The sign of x
// is applied to every digit.
__device__ __forceinline__ void digits(double x, int e, __nv_bfloat16* d) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int bexp = (int)((bits >> 52) & 0x7FF);
  unsigned long long G = 0;
  if (bexp != 0) {   // zero and subnormals (far below any row scale here) give zero digits
    const unsigned long long man = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = (bexp - 1023) - e + (TOP_SHIFT - 52);   // x = man 2^(bexp-1075); G = man 2^sh
    if (sh >= 0) G = man << sh;
    else if (sh > -64) G = (man >> -sh) + ((man >> (-sh - 1)) & 1ull);
  }
  const bool neg = (bits >> 63) != 0;
  int dig[SLICES];
#pragma unroll
  for (int s = SLICES - 1; s > 0; --s) {
    int r = (int)(G & 31ull);
    if (r > 16) r -= 32;
    dig[s] = r;
    G = (G - (long long)r) >> 5;
  }
  dig[0] = (int)G;
#pragma unroll
  for (int s = 0; s < SLICES; ++s) d[s] = __int2bfloat16_rn(neg ? -dig[s] : dig[s]);
}

// Element offset of (row r, real k) of digit slice s in the tiled layout the GEMM copies from:
// tiles of R rows x BK, ordered [row tile][K block][slice], each stored as the shared-memory
// image of a K-major operand with the 32-byte swizzle (row rr at 32 rr bytes, 16-byte half c
// at physical half c ^ ((rr >> 2) & 1)).
template <int R>
__device__ __forceinline__ long tiled_off(long r, long k, int s, long kblocks) {
  const long rt = r / R, rr = r % R, kb = k / BK;
  const int kc = (int)(k % BK);
  const int c = kc >> 3, e = kc & 7;
  return ((rt * kblocks + kb) * SLICES + s) * (long)(R * BK) + rr * BK + ((c ^ (int)((rr >> 2) & 1)) << 3) + e;
}

// A digits: slice s, row r, columns 2c (Re) and 2c+1 (Im) of the real embedding; the tile is
// staged through shared memory so that both the read (op-dependent) and the write coalesce.
__device__ __forceinline__ void slice_a(int M, int K, const cplx* A, long lda, int op, const int* rowexp, long mpad,
                                        long kpad, __nv_bfloat16* out, cplx (*t)[33], int bx, int by) {
  const int r0 = by * 32, c0 = bx * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  for (int i = ty; i < 32; i += 8) {
    // element (r0 + a, c0 + b); read along the contiguous dimension
    int a, b;
    if (op == OP_N) { a = tx; b = i; } else { a = i; b = tx; }
    const long r = r0 + a, c = c0 + b;
    t[a][b] = (r < M && c < K) ? op_at(A, lda, op, r, c) : cmk(0.0, 0.0);
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const long r = r0 + i, c = c0 + tx;
    if (r >= mpad || 2 * c >= kpad) continue;
    const cplx v = t[i][tx];
    const int e = (r < M && rowexp[r] > -100000) ? rowexp[r] : 0;
    __nv_bfloat16 dr[SLICES], di[SLICES];
    digits(v.x, e, dr);
    digits(v.y, e, di);
#pragma unroll
    for (int s = 0; s < SLICES; ++s) {
      __nv_bfloat162 p;
      p.x = dr[s];
      p.y = di[s];
      *(__nv_bfloat162*)(out + tiled_off<BM>(r, 2 * c, s, kpad / BK)) = p;
    }
  }
}

// B digits: op(B) is K x N; real B^T rows 2j = (Re b, -Im b), 2j+1 = (Im b, Re b) over k.
__device__ __forceinline__ void slice_b(int K, int N, const cplx* B, long ldb, int op, const int* colexp, long npad,
                                        long kpad, __nv_bfloat16* out, cplx (*t)[33], int bx, int by) {
  const int j0 = by * 32, k0 = bx * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int i = ty; i < 32; i += 8) {
    int a, b;   // a: k offset, b: j offset
    if (op == OP_N) { a = tx; b = i; } else { a = i; b = tx; }
    const long kk = k0 + a, j = j0 + b;
    t[b][a] = (kk < K && j < N) ? op_at(B, ldb, op, kk, j) : cmk(0.0, 0.0);
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const long j = j0 + i, kk = k0 + tx;
    if (2 * j >= npad || 2 * kk >= kpad) continue;
    const cplx v = t[i][tx];
    const int e = (j < N && colexp[j] > -100000) ? colexp[j] : 0;
    __nv_bfloat16 dr[SLICES], di[SLICES];
    digits(v.x, e, dr);
    digits(v.y, e, di);
#pragma unroll
    for (int s = 0; s < SLICES; ++s) {
      __nv_bfloat162 p0, p1;
      p0.x = dr[s]; p0.y = __hneg(di[s]);
      p1.x = di[s]; p1.y = dr[s];
      *(__nv_bfloat162*)(out + tiled_off<BN>(2 * j, 2 * kk, s, kpad / BK)) = p0;
      *(__nv_bfloat162*)(out + tiled_off<BN>(2 * j + 1, 2 * kk, s, kpad / BK)) = p1;
    }
  }
}

struct SliceArgs {
  int M, N, K;
  const cplx *A, *B;
  long lda, ldb;
  int opA, opB;
  const int *rowexp, *colexp;
  long mpad, npad, kpad;
  __nv_bfloat16 *outA, *outB;
  unsigned gxa, gya, gxb, gyb;
};
// Both operands' digit tiles in one launch: blockIdx.z = 0 slices A, 1 slices B.
__global__ void slice_kernel(SliceArgs g) {
  __shared__ cplx t[32][33];
  pdl_wait();
  pdl_trigger();
  if (blockIdx.z == 0) {
    if (blockIdx.x >= g.gxa || blockIdx.y >= g.gya) return;
    slice_a(g.M, g.K, g.A, g.lda, g.opA, g.rowexp, g.mpad, g.kpad, g.outA, t, blockIdx.x, blockIdx.y);
  } else {
    if (blockIdx.x >= g.gxb || blockIdx.y >= g.gyb) return;
    slice_b(g.K, g.N, g.B, g.ldb, g.opB, g.colexp, g.npad, g.kpad, g.outB, t, blockIdx.x, blockIdx.y);
  }
}

__global__ void oz_reduce_kernel(int M, int N, int splits, const cplx* partial, cplx* C, long ldc, cplx alpha,
                                 cplx beta) {
  pdl_wait();
  pdl_trigger();
  const long total = (long)M * N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const long r = e % M, c = e / M;
    cplx v = cmk(0.0, 0.0);
    for (int z = 0; z < splits; ++z) v = cadd(v, partial[(long)z * total + e]);
    cplx o = cmul(alpha, v);
    if (beta.x != 0.0 || beta.y != 0.0) o = cadd(o, cmul(beta, C[r + c * ldc]));
    C[r + c * ldc] = o;
  }
}

long round_up(long x, long m) { return (x + m - 1) / m * m; }

// a launch that may start while the previous kernel on the stream finishes
template <typename... Params, typename... Args>
cudaError_t launch_pdl(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
}  // namespace

struct OzakiGemm {
  __nv_bfloat16* A = nullptr;
  __nv_bfloat16* B = nullptr;
  size_t a_bytes = 0, b_bytes = 0;
  int* exps = nullptr;
  size_t exps_n = 0;
  cplx* partial = nullptr;
  size_t partial_bytes = 0;
  bool attr = false;
  int sms = 0;
};

OzakiGemm* ozaki_new() { return new OzakiGemm(); }
void ozaki_free(OzakiGemm* o) {
  if (!o) return;
  cudaFree(o->A);
  cudaFree(o->B);
  cudaFree(o->exps);
  cudaFree(o->partial);
  delete o;
}

// Grows a workspace.  The previous product's kernels may still be queued on the stream and
// use the old buffer, and cudaFree is not guaranteed to wait for them (the memory can go to
// another thread's allocation at once): drain the stream first.
static cudaError_t grow(void** p, size_t* have, size_t need, cudaStream_t s) {
  if (*have >= need) return cudaSuccess;
  cudaError_t es = cudaStreamSynchronize(s);
  if (es != cudaSuccess) return es;
  cudaFree(*p);
  *p = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc(p, need);
  if (e == cudaSuccess) *have = need;
  return e;
}

cudaError_t ozaki_gemm(OzakiGemm* o, const GemmArgs& g, cudaStream_t s, int* err) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (g.K <= 0) {
    // empty product: C = beta C through the DFMA path's epilogue
    return zgemm_launch(g, s);
  }
  const long M = g.M, N = g.N, K = g.K;
  const long mpad = round_up(M, BM), kpad = round_up(2 * K, BK), npad = round_up(2 * N, BN);
  cudaError_t e;
  if ((e = grow((void**)&o->A, &o->a_bytes, sizeof(__nv_bfloat16) * SLICES * mpad * kpad, s)) != cudaSuccess) return e;
  if ((e = grow((void**)&o->B, &o->b_bytes, sizeof(__nv_bfloat16) * SLICES * npad * kpad, s)) != cudaSuccess) return e;
  size_t have = o->exps_n * sizeof(int);
  if ((e = grow((void**)&o->exps, &have, sizeof(int) * (M + N), s)) != cudaSuccess) return e;
  o->exps_n = have / sizeof(int);
  if (!o->attr) {
    if ((e = cudaFuncSetAttribute(ozaki_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES)) != cudaSuccess)
      return e;
    o->attr = true;
  }
  int* rowexp = o->exps;
  int* colexp = o->exps + M;
  // exponents: rows of op(A), columns of op(B) (sentinel 0x80808080 = very negative)
  if ((e = cudaMemsetAsync(o->exps, 0x80, sizeof(int) * (M + N), s)) != cudaSuccess) return e;
  {
    ExpJob ja{(int)M, (int)K, g.A, g.lda, g.opA, true, rowexp, (unsigned)((K + 31) / 32), (unsigned)((M + 31) / 32)};
    ExpJob jb{(int)K, (int)N, g.B, g.ldb, g.opB, false, colexp, (unsigned)((N + 31) / 32), (unsigned)((K + 31) / 32)};
    dim3 grid(std::max(ja.gx, jb.gx), std::max(ja.gy, jb.gy), 2);
    exp_tile_kernel<<<grid, 256, 0, s>>>(ja, jb);
    count_launch(1);
  }
  {
    SliceArgs sa{};
    sa.M = (int)M;
    sa.N = (int)N;
    sa.K = (int)K;
    sa.A = g.A;
    sa.B = g.B;
    sa.lda = g.lda;
    sa.ldb = g.ldb;
    sa.opA = g.opA;
    sa.opB = g.opB;
    sa.rowexp = rowexp;
    sa.colexp = colexp;
    sa.mpad = mpad;
    sa.npad = npad;
    sa.kpad = kpad;
    sa.outA = o->A;
    sa.outB = o->B;
    sa.gxa = (unsigned)((kpad / 2 + 31) / 32);
    sa.gya = (unsigned)(mpad / 32);
    sa.gxb = (unsigned)((kpad / 2 + 31) / 32);
    sa.gyb = (unsigned)((npad / 2 + 31) / 32);
    dim3 grid(std::max(sa.gxa, sa.gxb), std::max(sa.gya, sa.gyb), 2);
    if ((e = launch_pdl(slice_kernel, grid, dim3(256), 0, s, sa)) != cudaSuccess) return e;
    count_launch(1);
  }
  const int kblocks = (int)(kpad / BK);
  const int passes = (int)((kpad + KPASS - 1) / KPASS);
  const long tiles = (mpad / BM) * (npad / BN);
  if (o->sms == 0) {
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&o->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  }
  // K splits (each within one exact pass): one CTA per SM, so the launch takes
  // ceil(tiles * splits / SMs) waves of (K blocks per split + ~8 blocks of pipeline fill and
  // epilogue); take the cheapest split count, the smallest among equals
  int splits = passes;
  {
    long best = -1;
    for (int sp = passes; sp <= 16 * passes; ++sp) {
      if (sp > passes && (long)kblocks / sp < 8) break;
      const long waves = (tiles * sp + o->sms - 1) / o->sms;
      const long cost = waves * ((kblocks + sp - 1) / sp + 8);
      if (best < 0 || cost < best) {
        best = cost;
        splits = sp;
      }
    }
  }
  const int per = (kblocks + splits - 1) / splits;   // <= KPASS / BK since splits >= passes
  OzArgs a{};
  a.M = (int)M;
  a.N2 = (int)(2 * N);
  a.kblocks = kblocks;
  a.per = per;
  a.tri = g.tri;
  a.rowexp = rowexp;
  a.colexp = colexp;
  a.A = o->A;
  a.B = o->B;
  a.C = g.C;
  a.ldc = g.ldc;
  a.alpha = g.alpha;
  a.beta = g.beta;
  a.splits = splits;
  a.err = err;
  if (splits > 1) {
    if ((e = grow((void**)&o->partial, &o->partial_bytes, sizeof(cplx) * splits * M * N, s)) != cudaSuccess) return e;
    a.partial = o->partial;
  }
  dim3 grid((unsigned)(mpad / BM), (unsigned)(npad / BN), (unsigned)splits);
  if ((e = launch_pdl(ozaki_kernel, grid, dim3(NTHREADS), SMEM_BYTES, s, a)) != cudaSuccess) return e;
  count_launch(1);
  if (splits > 1) {
    const long total = M * N;
    if ((e = launch_pdl(oz_reduce_kernel, dim3((unsigned)std::min<long>((total + 255) / 256, 4096)), dim3(256), 0, s,
                        (int)M, (int)N, splits, (const cplx*)o->partial, g.C, g.ldc, g.alpha, g.beta)) != cudaSuccess)
      return e;
    count_launch(1);
  }
  return cudaGetLastError();
}
