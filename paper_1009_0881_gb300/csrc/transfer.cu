#include <algorithm>
// Grid transfer operators of Section 4.2, layout helpers, input checks and the
// Frobenius error.
//
// Images are the columns of a row-major (pixels x cols) matrix, so one pixel is
// a contiguous row: a thread handles one output pixel for four adjacent columns
// and every load/store of a warp is a coalesced run along the row.
#include "nmf_internal.cuh"

namespace nmfk {

namespace {

// Eq. (4.1): coarse (i, j) = weighted mean of fine (2i+dy, 2j+dx), weights
// (2-|dy|)(2-|dx|), in-bounds neighbours only, divided by the kept weight.
template <int V>
__global__ void restrict_kernel(const float* __restrict__ X, int64_t ldx, int h, int w, int64_t cols,
                                float* __restrict__ Y, int64_t ldy) {
    const int hc = (h + 1) / 2, wc = (w + 1) / 2;
    const int64_t cq = (cols + V - 1) / V;
    const int64_t total = (int64_t)hc * wc * cq;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pix = t / cq;
        const int64_t c = (t - pix * cq) * V;
        const int i = (int)(pix / wc), j = (int)(pix - (int64_t)i * wc);
        float acc[V];
#pragma unroll
        for (int e = 0; e < V; ++e) acc[e] = 0.f;
        float wsum = 0.f;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int y = 2 * i + dy;
            if (y < 0 || y >= h) continue;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int x = 2 * j + dx;
                if (x < 0 || x >= w) continue;
                const float wt = (float)((2 - abs(dy)) * (2 - abs(dx)));
                wsum += wt;
                const float* src = X + ((int64_t)y * w + x) * ldx + c;
                if (V == 4) {
                    const float4 v = *reinterpret_cast<const float4*>(src);
                    acc[0] = fmaf(wt, v.x, acc[0]);
                    acc[1 % V] = fmaf(wt, v.y, acc[1 % V]);
                    acc[2 % V] = fmaf(wt, v.z, acc[2 % V]);
                    acc[3 % V] = fmaf(wt, v.w, acc[3 % V]);
                } else {
                    acc[0] = fmaf(wt, src[0], acc[0]);
                }
            }
        }
        float* dst = Y + pix * ldy + c;
        if (V == 4) {
            *reinterpret_cast<float4*>(dst) =
                make_float4(acc[0] / wsum, acc[1 % V] / wsum, acc[2 % V] / wsum, acc[3 % V] / wsum);
        } else {
            dst[0] = acc[0] / wsum;
        }
    }
}

// Eq. (4.2): fine (i, j) = mean over coarse (i', j'), i' in rd(i/2), j' in rd(j/2)
// (neighbours past an even-size border dropped).
template <int V>
__global__ void prolong_kernel(const float* __restrict__ Y, int64_t ldy, int h, int w, int64_t cols,
                               float* __restrict__ X, int64_t ldx) {
    const int hc = (h + 1) / 2, wc = (w + 1) / 2;
    const int64_t cq = (cols + V - 1) / V;
    const int64_t total = (int64_t)h * w * cq;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pix = t / cq;
        const int64_t c = (t - pix * cq) * V;
        const int i = (int)(pix / w), j = (int)(pix - (int64_t)i * w);
        const int i0 = i >> 1, i1 = (i & 1) ? ((i + 1) >> 1) : i0;
        const int j0 = j >> 1, j1 = (j & 1) ? ((j + 1) >> 1) : j0;
        const int ia[2] = {i0, i1}, ja[2] = {j0, j1};
        const int ni = (i1 != i0 && i1 < hc) ? 2 : 1;
        const int nj = (j1 != j0 && j1 < wc) ? 2 : 1;
        float acc[V];
#pragma unroll
        for (int e = 0; e < V; ++e) acc[e] = 0.f;
        for (int a = 0; a < ni; ++a)
            for (int b = 0; b < nj; ++b) {
                const float* src = Y + ((int64_t)ia[a] * wc + ja[b]) * ldy + c;
                if (V == 4) {
                    const float4 v = *reinterpret_cast<const float4*>(src);
                    acc[0] += v.x;
                    acc[1 % V] += v.y;
                    acc[2 % V] += v.z;
                    acc[3 % V] += v.w;
                } else {
                    acc[0] += src[0];
                }
            }
        const float cnt = (float)(ni * nj);
        float* dst = X + pix * ldx + c;
        if (V == 4) {
            *reinterpret_cast<float4*>(dst) =
                make_float4(acc[0] / cnt, acc[1 % V] / cnt, acc[2 % V] / cnt, acc[3 % V] / cnt);
        } else {
            dst[0] = acc[0] / cnt;
        }
    }
}

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline unsigned grid_for(int64_t work, int threads) {
    int64_t g = ceil_div(work, threads);
    if (g < 1) g = 1;
    if (g > 65535LL * 16) g = 65535LL * 16;
    return (unsigned)g;
}

__global__ void copy2d_kernel(const float* __restrict__ in, int64_t ldi, int64_t rows, int64_t cols,
                              float* __restrict__ out, int64_t ldo) {
    const int64_t total = rows * cols;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / cols, c = t - r * cols;
        out[r * ldo + c] = in[r * ldi + c];
    }
}

// 32 x 32 tiles through shared memory: reads and writes both coalesced.
__global__ void transpose_kernel(const float* __restrict__ in, int64_t ldi, int64_t rows, int64_t cols,
                                 float* __restrict__ out, int64_t ldo) {
    __shared__ float tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int64_t r = r0 + dy, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[dy][threadIdx.x] = in[r * ldi + c];
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int64_t c = c0 + dy, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[c * ldo + r] = tile[threadIdx.x][dy];
    }
}

__device__ __forceinline__ unsigned not_ok(float v) { return (!(v >= 0.f) || isinf(v)) ? 1u : 0u; }

// Counts the entries of X (rows x cols, leading dimension ld) that are negative,
// NaN or infinite.  A dense X is read as float4 over the whole array; a padded one
// row by row, the threads of a block striding over the columns (no index division).
__global__ void check_kernel(const float* __restrict__ X, int64_t ld, int64_t rows, int64_t cols,
                             unsigned long long* bad) {
    unsigned long long cnt = 0;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (ld == cols) {
        const int64_t total = rows * cols;
        const int64_t n4 = (reinterpret_cast<uintptr_t>(X) % 16 == 0) ? total / 4 : 0;
        const float4* X4 = reinterpret_cast<const float4*>(X);
        for (int64_t t = gid; t < n4; t += stride) {
            const float4 v = X4[t];
            cnt += not_ok(v.x) + not_ok(v.y) + not_ok(v.z) + not_ok(v.w);
        }
        for (int64_t t = 4 * n4 + gid; t < total; t += stride) cnt += not_ok(X[t]);
    } else {
        for (int64_t r = blockIdx.x; r < rows; r += gridDim.x)
            for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) cnt += not_ok(X[r * ld + c]);
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(bad, cnt);
}

// ||M - V Wt^T||_F^2: each CTA owns a 64 x 64 tile of M, recomputes the tile
// of V W from V (64 x r) and Wt (64 x r) in shared memory, sums each thread's
// squared residuals four at a time in FP32 and those sums in FP64; one partial
// per CTA.
constexpr int kErrTile = 64;

__global__ void __launch_bounds__(256) error_tile_kernel(const float* __restrict__ M, int64_t ldm,
                                                         const float* __restrict__ V,
                                                         const float* __restrict__ Wt, int64_t rp,
                                                         int64_t m, int64_t n, int r,
                                                         double* __restrict__ partials, const int* skip) {
    if (skip && *(volatile const int*)skip) return;
    __shared__ float Vs[kMaxRank][kErrTile + 4];
    __shared__ float Ws[kMaxRank][kErrTile + 1];
    const int64_t ntj = ceil_div(n, kErrTile);
    const int64_t ti = blockIdx.x / ntj, tj = blockIdx.x - ti * ntj;
    const int64_t i0 = ti * kErrTile, j0 = tj * kErrTile;
    for (int e = threadIdx.x; e < kErrTile * r; e += blockDim.x) {
        const int row = e / r, k = e - row * r;
        Vs[k][row] = (i0 + row < m) ? V[(i0 + row) * rp + k] : 0.f;
        Ws[k][row] = (j0 + row < n) ? Wt[(j0 + row) * rp + k] : 0.f;
    }
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int k = 0; k < r; ++k) {
        const float4 v4 = *reinterpret_cast<const float4*>(&Vs[k][ty * 4]);
        const float va[4] = {v4.x, v4.y, v4.z, v4.w};
        float wb[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) wb[b] = Ws[k][tx + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(va[a], wb[b], acc[a][b]);
    }
    // the four squared residuals of a row in FP32 (at most 4 rounding steps), then the
    // FP64 sum: GB300 runs FP64 at a small fraction of the FP32 rate
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t i = i0 + ty * 4 + a;
        if (i >= m) continue;
        float sa = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t j = j0 + tx + 16 * b;
            if (j >= n) continue;
            const float e = M[i * ldm + j] - acc[a][b];
            sa = fmaf(e, e, sa);
        }
        s += (double)sa;
    }
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void sum_partials_kernel(const double* __restrict__ partials, int64_t count, double* out,
                                    const int* skip = nullptr) {
    if (skip && *(volatile const int*)skip) return;
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t t = threadIdx.x; t < count; t += blockDim.x) s += partials[t];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sqrt(red[0]);
}

__global__ void sum_splits_kernel(const float* __restrict__ P, int64_t ps, int64_t ldp, int splits,
                                  int64_t rows, int64_t cols, float* __restrict__ out, int64_t ldo,
                                  bool transpose) {
    const int64_t total = rows * cols;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = t / cols, k = t - a * cols;
        float s = 0.f;
        for (int q = 0; q < splits; ++q) s += P[q * ps + a * ldp + k];
        if (transpose)
            out[k * ldo + a] = s;
        else
            out[a * ldo + k] = s;
    }
}

}  // namespace

cudaError_t sum_splits_launch(const float* P, int64_t ps, int64_t ldp, int splits, int64_t rows, int64_t cols,
                              float* out, int64_t ldo, bool transpose, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    sum_splits_kernel<<<grid_for(rows * cols, 256), 256, 0, st>>>(P, ps, ldp, splits, rows, cols, out, ldo,
                                                                   transpose);
    return cudaGetLastError();
}

cudaError_t restrict_launch(const float* X, int64_t ldx, int h, int w, int64_t cols, float* Y, int64_t ldy,
                            cudaStream_t st) {
    const int hc = (h + 1) / 2, wc = (w + 1) / 2;
    const bool vec = (ldx % 4 == 0) && (ldy % 4 == 0) && aligned16(X) && aligned16(Y) &&
                     round_up(cols, 4) <= ldx && round_up(cols, 4) <= ldy;
    const int threads = 256;
    if (vec) {
        restrict_kernel<4><<<grid_for((int64_t)hc * wc * ceil_div(cols, 4), threads), threads, 0, st>>>(
            X, ldx, h, w, cols, Y, ldy);
    } else {
        restrict_kernel<1><<<grid_for((int64_t)hc * wc * cols, threads), threads, 0, st>>>(X, ldx, h, w, cols,
                                                                                            Y, ldy);
    }
    return cudaGetLastError();
}

cudaError_t prolong_launch(const float* Y, int64_t ldy, int h, int w, int64_t cols, float* X, int64_t ldx,
                           cudaStream_t st) {
    const bool vec = (ldx % 4 == 0) && (ldy % 4 == 0) && aligned16(X) && aligned16(Y) &&
                     round_up(cols, 4) <= ldx && round_up(cols, 4) <= ldy;
    const int threads = 256;
    if (vec) {
        prolong_kernel<4><<<grid_for((int64_t)h * w * ceil_div(cols, 4), threads), threads, 0, st>>>(
            Y, ldy, h, w, cols, X, ldx);
    } else {
        prolong_kernel<1><<<grid_for((int64_t)h * w * cols, threads), threads, 0, st>>>(Y, ldy, h, w, cols, X,
                                                                                         ldx);
    }
    return cudaGetLastError();
}

cudaError_t copy2d_launch(const float* in, int64_t ldi, int64_t rows, int64_t cols, float* out, int64_t ldo,
                          bool transpose, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if (transpose) {
        dim3 block(32, 8);
        dim3 grid((unsigned)ceil_div(cols, 32), (unsigned)ceil_div(rows, 32));
        transpose_kernel<<<grid, block, 0, st>>>(in, ldi, rows, cols, out, ldo);
    } else {
        copy2d_kernel<<<grid_for(rows * cols, 256), 256, 0, st>>>(in, ldi, rows, cols, out, ldo);
    }
    return cudaGetLastError();
}

cudaError_t check_nonneg_launch(const float* X, int64_t ld, int64_t rows, int64_t cols,
                                unsigned long long* d_bad, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    int64_t g = ceil_div(rows * cols, 256 * 8);
    if (g < 1) g = 1;
    if (g > 4096) g = 4096;
    check_kernel<<<(unsigned)g, 256, 0, st>>>(X, ld, rows, cols, d_bad);
    return cudaGetLastError();
}

int64_t error_partials_needed(int64_t m, int64_t n) {
    return ceil_div(m, kErrTile) * ceil_div(n, kErrTile);
}

cudaError_t error_launch(const float* M, int64_t ldm, const float* V, const float* Wt, int64_t rp, int64_t m,
                         int64_t n, int r, double* d_partials, double* d_out, cudaStream_t st, const int* skip) {
    const int64_t tiles = error_partials_needed(m, n);
    error_tile_kernel<<<(unsigned)tiles, 256, 0, st>>>(M, ldm, V, Wt, rp, m, n, r, d_partials, skip);
    sum_partials_kernel<<<1, 256, 0, st>>>(d_partials, tiles, d_out, skip);
    return cudaGetLastError();
}

namespace {
// Stopping rule of the batched form: after a finest-level sweep with objective
// f_t, stop once |f_{t-1} - f_t| <= tol * f_t (state[0] holds f_{t-1}, 0 before
// the first sweep).  Counts the sweeps that ran.
__global__ void converge_check_kernel(const double* __restrict__ f_now, double* state, int* flag, double tol,
                                      long long* count) {
    if (*flag) return;
    const double cur = *f_now, prev = state[0];
    *count += 1;
    if (prev > 0.0 && fabs(prev - cur) <= tol * cur) *flag = 1;
    state[0] = cur;
}
}  // namespace

namespace {
// Per-block FP64 sums of squares of a row-major matrix (rows x cols, leading dimension ld).
__global__ void sumsq_kernel(const float* __restrict__ M, int64_t ld, int64_t rows, int64_t cols,
                             double* __restrict__ partials) {
    __shared__ double red[256];
    double s = 0.0;
    const int64_t total = rows * cols;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / cols, j = t - i * cols;
        const double v = M[i * ld + j];
        s += v * v;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// f = sqrt(max(0, ||M||^2 - 2 sum_b part[2b] + sum_b part[2b+1])): the objective
// after a sweep from the identity ||M - VW||^2 = ||M||^2 - 2 <V^T M, W> + <V^T V, W W^T>,
// blocks summed in index order.  Does nothing once the problem is flagged converged.
__global__ void identity_objective_kernel(const double* __restrict__ part, int nblocks, const double* __restrict__ mnorm,
                                          double* __restrict__ f_out, const int* skip) {
    if (skip && *skip) return;
    double s1 = 0.0, s2 = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        s1 += part[2 * b];
        s2 += part[2 * b + 1];
    }
    const double m = *mnorm;
    *f_out = sqrt(fmax(0.0, m * m - 2.0 * s1 + s2));
}
}  // namespace

cudaError_t norm_launch(const float* M, int64_t ld, int64_t rows, int64_t cols, double* d_partials, int64_t max_partials,
                        double* d_out, cudaStream_t st) {
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(max_partials, 256));
    sumsq_kernel<<<(unsigned)blocks, 256, 0, st>>>(M, ld, rows, cols, d_partials);
    sum_partials_kernel<<<1, 256, 0, st>>>(d_partials, blocks, d_out);
    return cudaGetLastError();
}

cudaError_t identity_objective_launch(const double* part, int nblocks, const double* mnorm, double* f_out,
                                      const int* skip, cudaStream_t st) {
    identity_objective_kernel<<<1, 1, 0, st>>>(part, nblocks, mnorm, f_out, skip);
    return cudaGetLastError();
}

cudaError_t converge_check_launch(const double* f_now, double* state, int* flag, double tol, long long* count,
                                  cudaStream_t st) {
    converge_check_kernel<<<1, 1, 0, st>>>(f_now, state, flag, tol, count);
    return cudaGetLastError();
}

}  // namespace nmfk
