// Grouped half-sweeps (grouped.cu): one persistent launch runs the same half-sweep
// (V-step or W-step of the schedule's current sweep) of many independent problems.
//
// Each problem contributes its 64-row tiles of the factor being updated; the CTAs
// of the launch (two per SM) take tiles from a shared work-list through an atomic
// counter, so small and large problems share the device in one launch.  A tile is
// the whole product over K (no split across CTAs), the HALS or MU update of its rows
// and the Gram slab of its new rows; the Gram matrix it updates with is reduced from
// the previous half-sweep's slabs by a small grouped launch beforehand.  Every sum runs
// in an order fixed by the problem alone, so a problem gives the same bits whatever
// else is in the group and whichever CTA takes its tiles.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "fused.cuh"

namespace nmfk {

constexpr int kGroupTile = 64;  // rows of the factor per tile

// One (problem, level, half) of a grouped solve, in device memory (the tensor maps carry
// their own alignment, which an array of descriptors keeps).  The tensor maps are the
// half-sweep's operands (X: K x Na columns, box 64 x 32; Y: K x rp, box br x 32).
struct GroupDesc {
    CUtensorMap tmX;
    CUtensorMap tmY;
    float* F;            // Na x rp factor, updated in place
    const float* G;      // reduced Gram matrix, r x rp
    float* Gout;         // one slab per tile (r x rp, stride gout_stride)
    const int* skip;     // optional: problem converged, nothing to do
    double* obj_part;    // optional: per tile [2t] = <P rows, new F rows>, [2t+1] = <G, slab t>
    int* err_flag;       // set if a bounded wait gave up
    int64_t K;
    int64_t gout_stride;
    int Na, r, rp, br, mode;
};

// One unit of work: tile `tile` of descriptor `desc`.
struct GroupItem {
    int desc;
    int tile;
};

// G of each listed problem: the sum of its `count` slabs (r x rp, stride `stride`) in slab order.
struct GramJob {
    const float* slabs;
    int64_t stride;
    int count;
    int f4;              // float4 groups of one slab (r * rp / 4)
    float* out;
    const int* skip;
};

// Stopping rule of one problem after a watched W-step: the objective from the identity
// terms the W-step's tiles wrote (tiles summed in order) and ||M||_F, then the test
// |f_{t-1} - f_t| <= tol * f_t (state[0] = f_{t-1}, state[1] = f_t); counts the sweeps.
struct ConvJob {
    const double* part;
    int ntiles;
    const double* mnorm;
    double* state;
    int* flag;
    double tol;
    long long* count;
};

cudaError_t grouped_init();
cudaError_t grouped_converge_launch(const ConvJob* jobs, int njobs, cudaStream_t st);
size_t grouped_smem_bytes();
// The reduction of every job's slabs (one launch); `jobs` in device memory.
cudaError_t grouped_gram_launch(const GramJob* jobs, int njobs, int max_f4, cudaStream_t st);
// One persistent launch over `nitems` work items; `counter` (zero before the launch) hands
// them out.  `ctas`: CTAs of the launch (two per SM fit).
cudaError_t grouped_half_sweep_launch(const GroupDesc* descs, const GroupItem* items, int nitems, int* counter,
                                      int ctas, cudaStream_t st);

}  // namespace nmfk
