// Restriction of M over the pixel grid and along its columns at once (Section 6.1 with
// Eq. (4.1) on both grids).  Run once per level when the hierarchy is formed.
#include "columns.cuh"

namespace nmfk {

namespace {

// One thread per coarse entry (pixel, column): the separable 27-point stencil with
// weights (2-|dy|)(2-|dx|)(2-|dk|) over the in-bounds fine neighbours, divided by the
// kept weight.  Consecutive threads take consecutive coarse columns of one pixel row.
__global__ void restrict_both_kernel(const float* __restrict__ X, int64_t ldx, int h, int w, int64_t n,
                                     float* __restrict__ Y, int64_t ldy) {
    const int hc = (h + 1) / 2, wc = (w + 1) / 2;
    const int64_t nc = (n + 1) / 2;
    const int64_t total = (int64_t)hc * wc * nc;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pix = t / nc;
        const int64_t j = t - pix * nc;
        const int i = (int)(pix / wc), jj = (int)(pix - (int64_t)i * wc);
        float acc = 0.f, wsum = 0.f;
        for (int dy = -1; dy <= 1; ++dy) {
            const int y = 2 * i + dy;
            if (y < 0 || y >= h) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                const int x = 2 * jj + dx;
                if (x < 0 || x >= w) continue;
                const float* row = X + ((int64_t)y * w + x) * ldx;
                const float wp = (float)((2 - abs(dy)) * (2 - abs(dx)));
#pragma unroll
                for (int dk = -1; dk <= 1; ++dk) {
                    const int64_t k = 2 * j + dk;
                    if (k < 0 || k >= n) continue;
                    const float wt = wp * (float)(2 - abs(dk));
                    acc = fmaf(wt, row[k], acc);
                    wsum += wt;
                }
            }
        }
        Y[pix * ldy + j] = acc / wsum;
    }
}

}  // namespace

cudaError_t restrict_both_launch(const float* X, int64_t ldx, int h, int w, int64_t n, float* Y, int64_t ldy,
                                 cudaStream_t st) {
    const int64_t total = (int64_t)((h + 1) / 2) * ((w + 1) / 2) * ((n + 1) / 2);
    if (total == 0) return cudaSuccess;
    const int threads = 256;
    int64_t g = (total + threads - 1) / threads;
    if (g > 65535LL * 16) g = 65535LL * 16;
    restrict_both_kernel<<<(unsigned)g, threads, 0, st>>>(X, ldx, h, w, n, Y, ldy);
    return cudaGetLastError();
}

}  // namespace nmfk
