// Internal declarations shared by the CUDA translation units of the library.
//
// Internal layouts (all float32, row-major, zero padding):
//   M_l  : m_l x n,  leading dimension ldm  = round_up(n, 4)
//   Mt_l : n x m_l,  leading dimension ldmt = round_up(m_l, 4)   (M transposed, kept so
//          that every product reads its long K dimension as the row index)
//   V_l  : m_l x r,  leading dimension rp = round_up(r, 4)
//   Wt   : n x r,    leading dimension rp                        (W transposed)
// Padding columns are zero and are never written by the update kernels, so
// they stay zero for the whole solve.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "nmf.h"

namespace nmfk {

constexpr int kMaxRank = 64;

__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------
// Tall-skinny "TN" product with split-K partial outputs:
//   out[s*split_stride + a*ldo + k] = sum_{kk in split s} X[kk*ldx + a] * Y[kk*ldy + k]
// for a < Na, k < ldo.  Covers A = M W^T (X = Mt), C^T = M^T V (X = M) and the
// Gram matrices W W^T (X = Y = Wt) and V^T V (X = Y = V).
// ---------------------------------------------------------------------------
struct GemmTask {
    const float* X;
    const float* Y;
    float* out;
    int64_t ldx, ldy, ldo, split_stride;
    int64_t K;
    int Na;
    int splits;
    int kchunk;      // K rows per split, multiple of the K tile
    int a_tiles;     // ceil(Na / 64)
    int tile_begin;  // first CTA index of this task in the launch
};

constexpr int kMaxGemmTasks = 4;
struct GemmBatch {
    GemmTask t[kMaxGemmTasks];
    int ntasks;
    int total_tiles;
};

// Fill split/tile fields of a task for a launch on `num_sms` SMs.
void gemm_plan_task(GemmTask& t, int num_sms, int max_splits);
// Launch all tasks of `b` (tile_begin/total_tiles filled here); `br` = padded rank tile (16..64).
cudaError_t gemm_tn_launch(GemmBatch& b, int br, cudaStream_t st);

// ---------------------------------------------------------------------------
// Factor updates.  Each works on the rows of a tall factor F (rows x ldf):
// F = V with (A, B) for the V-step, F = Wt with (C^T, D) for the W-step.
// The products arrive as split-K partials: row a of split s at
// P[s*ps + a*ldp + k]; the Gram matrix occupies rows gram_row .. gram_row+r-1.
// ---------------------------------------------------------------------------
struct UpdateArgs {
    float* F;          // rows x ldf factor, updated in place
    int64_t ldf;
    const float* P;    // factor-product partials: row a of split s at P[s*ps + a*ldp + k]
    int64_t ps, ldp;
    int splits;
    const float* PG;   // Gram partials: row l of split s at PG[s*pgs + l*ldpg + k]
    int64_t pgs, ldpg;
    int gsplits;
    int64_t rows;
    int r;
    double* Gd;        // ANLS: r x r scratch receiving the FP64 sum of the Gram partials
    int max_outer;     // ANLS: cap on the variables added per row (< 0: 3r, the default)
    int bpp;           // ANLS: 1 = block principal pivoting first (active set where it cannot finish)
    int rank_cap;      // ANLS: when the other factor has fewer rows than r, their number (G has at most
                       // that rank, and a passive set of that size already fits P_i exactly); else 0
    const int* skip;   // optional: when *skip != 0 the launch does nothing (converged problem)
};

// ANLS: F rows = argmin_{x>=0} 1/2 x^T G x - p^T x, FP64 active set.  status: device int
// (0 ok, 1 iteration cap hit) OR-ed over all rows.
cudaError_t anls_update_launch(const UpdateArgs& a, int num_sms, int* d_status, cudaStream_t st);
// One-time kernel attribute setup (large dynamic shared memory); call before any capture.
cudaError_t init_kernel_attributes();

// ---------------------------------------------------------------------------
// Grid transfers (Eqs. (4.1) and (4.2)) on column-stacked images:
// X is (h*w) x cols with leading dimension ldx.
// ---------------------------------------------------------------------------
cudaError_t restrict_launch(const float* X, int64_t ldx, int h, int w, int64_t cols, float* Y,
                            int64_t ldy, cudaStream_t st);
cudaError_t prolong_launch(const float* Y, int64_t ldy, int h, int w, int64_t cols, float* X,
                           int64_t ldx, cudaStream_t st);

// Copy a rows x cols matrix between leading dimensions, optionally transposing
// (out[c*ldo + r] = in[r*ldi + c]).
cudaError_t copy2d_launch(const float* in, int64_t ldi, int64_t rows, int64_t cols, float* out,
                          int64_t ldo, bool transpose, cudaStream_t st);

// out[a*ldo + k] = sum_s P[s*ps + a*ldp + k] for a < rows, k < cols (fixed order),
// optionally written transposed (out[k*ldo + a]).
cudaError_t sum_splits_launch(const float* P, int64_t ps, int64_t ldp, int splits, int64_t rows,
                              int64_t cols, float* out, int64_t ldo, bool transpose, cudaStream_t st);

// Validation: counts negative or NaN entries of a rows x cols matrix into *d_bad.
cudaError_t check_nonneg_launch(const float* X, int64_t ld, int64_t rows, int64_t cols,
                                unsigned long long* d_bad, cudaStream_t st);

// ---------------------------------------------------------------------------
// ||M - V Wt^T||_F with FP64 accumulation of the squares, deterministic: partial
// sums per CTA into d_partials (size >= error_partials_needed()), the norm into d_out.
// ---------------------------------------------------------------------------
int64_t error_partials_needed(int64_t m, int64_t n);
// Batched stopping rule: sets *flag once |f_prev - f_now| <= tol * f_now; counts sweeps run.
// ||M||_F of a rows x cols matrix (FP64), through up to max_partials per-block sums.
cudaError_t norm_launch(const float* M, int64_t ld, int64_t rows, int64_t cols, double* d_partials, int64_t max_partials,
                        double* d_out, cudaStream_t st);
// Objective after a sweep from the identity terms written by the W-step half-sweep
// (HalfSweepParams::obj_part, nblocks CTAs) and ||M||_F.
cudaError_t identity_objective_launch(const double* part, int nblocks, const double* mnorm, double* f_out,
                                      const int* skip, cudaStream_t st);
cudaError_t converge_check_launch(const double* f_now, double* state, int* flag, double tol, long long* count,
                                  cudaStream_t st);
cudaError_t error_launch(const float* M, int64_t ldm, const float* V, const float* Wt, int64_t rp,
                         int64_t m, int64_t n, int r, double* d_partials, double* d_out,
                         cudaStream_t st, const int* skip = nullptr);

}  // namespace nmfk
