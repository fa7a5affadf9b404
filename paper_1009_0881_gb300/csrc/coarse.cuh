// Coarse-level sweep runs (coarse.cu): every sweep of one run of HALS or MU
// sweeps on a coarse level of the hierarchy in a single persistent launch.
#pragma once

#include <cuda_runtime.h>

#include "nmf_internal.cuh"

namespace nmfk {

struct CoarseParams {
    const float* M;       // level matrix M_l, m x n, leading dimension ldm
    int64_t ldm;
    float* V;             // m x rp (in: current V_l, out: after the run)
    float* Wt;            // n x rp (in: current W^T, out: after the run)
    int m, n, r, rp;
    int sweeps;           // >= 1
    int nchunk;           // ceil(n / 16): 16-column chunks of M_l (rows of W^T)
    int cpc;              // chunks per CTA = ceil(nchunk / grid)
    float* part;          // nchunk slots of (m + r) x rp floats: partial products of each chunk
    int64_t part_stride;  // floats between slots (multiple of 4)
    float* red;           // (m + r) x rp: reduced products of the V-step
    float* Bout;          // r x rp: W W^T of the final W (the Gram input of the next V-step)
    unsigned* bar;        // grid-barrier counter, zero at launch (the launcher clears it)
    int* err_flag;        // set to 1 if a grid barrier gave up waiting
    uint32_t spins;       // polls of a grid barrier before it gives up (kGridBarrierSpins by default)
};

// Default spin budget of a grid barrier (about a second of polling).
constexpr uint32_t kGridBarrierSpins = 1u << 20;

cudaError_t coarse_init();
// Whether a level of m rows, n columns and rank r can run on at most `max_grid`
// CTAs (one per SM); if so the shared memory per CTA, the chunks per CTA, the
// chunk count and the CTAs to launch.  Results do not depend on the CTA count.
bool coarse_fits(int64_t m, int64_t n, int r, int max_grid, size_t* smem, int* cpc, int* nchunk, int* grid);
// Floats of the partial-product slot of one chunk.
int64_t coarse_slot_floats(int64_t m, int r, int rp);
// mode: 0 HALS, 1 MU.  Clears the barrier counter, then launches `grid` CTAs as a
// cooperative grid (all CTAs co-resident).
cudaError_t coarse_run_launch(const CoarseParams& q, int mode, int grid, size_t smem, cudaStream_t st);

}  // namespace nmfk
