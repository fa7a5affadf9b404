// Coarsening of the columns of M (Section 6.1: the columns form a sequence, such as the
// frames of a video or the bands of a hyperspectral image, that varies smoothly along
// its index).  The sequence of n columns is a 1-D grid coarsened like one side of the
// pixel grid: coarse point j sits on fine point 2j, ceil(n / 2) points per level.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace nmfk {

// Y = R X R_n^T for an (h*w) x n matrix X (leading dimension ldx): Eq. (4.1) over the
// pixel grid and the same full weighting (1, 2, 1, renormalised at the ends) along the
// n columns.  Y is (ceil(h/2)*ceil(w/2)) x ceil(n/2) with leading dimension ldy; its
// padding columns are not written.
cudaError_t restrict_both_launch(const float* X, int64_t ldx, int h, int w, int64_t n, float* Y, int64_t ldy,
                                 cudaStream_t st);

}  // namespace nmfk
