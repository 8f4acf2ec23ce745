// Chebyshev filter on the tensor cores (tcgen05, split-BF16 operands, FP32 accumulation in
// TMEM, FP64 recurrence state) -- the mixed-precision form of Algorithm 1 line 3.
#pragma once
#include "common.cuh"

struct TcFilter;
TcFilter* tc_filter_new();
void tc_filter_free(TcFilter* f);

// Residual-corrected form (used when the block is a Ritz block of H):  with H Yhat =
// Yhat diag(lam) + R, the filtered block is Yhat p_m(lam) + D_m where D_0 = 0 and
//     D_j = fa[j] H D_{j-1} + fb[j] D_{j-1} + fg[j] D_{j-2} + fa[j] R diag(p_{j-1}(lam)),
// an exact rewriting of the recurrence in which the low-precision products act on D, whose
// size is proportional to the residual, so their rounding no longer sets an accuracy floor.
struct TcRefine {
  const cplx* Z;        // H Yhat, n x k (device)
  const double* lam;    // Ritz values, k (device)
  const double* ptab;   // host, (mmax + 1) x k: ptab[j * k + i] = p_j(lam_i)
  const int* deg;       // host, per-column degree (non-increasing)
};

// Runs mmax recurrence steps: Y_j = fa[j] H Y_{j-1} + fb[j] Y_{j-1} + fg[j] Y_{j-2} on the
// first cnt[j] columns (cnt non-increasing: column i takes deg_i steps, the number of j with
// i < cnt[j]); Y (n x cnt[1], ld n) holds Y_0 on entry and each column's last Y_j on return.
// With ref the corrected form runs instead, with the same result.
// Device time (ms) of the recurrence step launches since the last call, and the column-steps
// they processed (sum over launches of their complex columns); resets both.
double tc_filter_take_ms(TcFilter* f, long long* col_steps = nullptr);

chfsi_status tc_filter_run(TcFilter* f, cudaStream_t s, int n, const cplx* H, cplx* Y, const int* cnt, int mmax,
                           const double* fa, const double* fb, const double* fg, const TcRefine* ref = nullptr);

// One filter call of a batch: the arguments of tc_filter_run for one problem (its own
// TcFilter state; cnt, fa, fb, fg and ref stay valid until tc_filter_run_batch returns).
struct TcJob {
  TcFilter* f;
  int n;
  const cplx* H;
  cplx* Y;
  const int* cnt;
  int mmax;
  const double *fa, *fb, *fg;
  const TcRefine* ref;
};
struct TcBatch;   // device descriptor table and the captured graph of a batch's step launches
TcBatch* tc_batch_new();
void tc_batch_free(TcBatch* b);
// The filter of every job, recurrence step j of all of them as ONE grouped launch (a tile
// scheduler over the problems' tiles; the tile width per step autotuned); the step launches
// are captured into a CUDA graph when use_graph is set.  Same results as tc_filter_run on
// each job.  *ms_steps += device time of the step launches.
chfsi_status tc_filter_run_batch(TcBatch* b, cudaStream_t s, const TcJob* jobs, int njobs, double* ms_steps,
                                 bool use_graph);
