// nmf_error_noalloc: the Frobenius error ||M - VW||_F without any device
// allocation, for callers that cannot call cudaMalloc (see include/nmf.h).
//
// The per-tile partial sums that nmf_error keeps in its handle's workspace live
// here in one file-scope device array of fixed size.  Every GPU that loads the
// library holds that array until the process exits; every call on a device
// shares it.
#include <cuda_runtime.h>

#include "nmf_internal.cuh"

namespace {

constexpr int kTile = 64;                        // 64 x 64 tile of M per CTA
constexpr int64_t kMaxTiles = 65536;             // scratch capacity: 64 Ki tiles = 512 KiB of doubles

// slots [0, kMaxTiles): one partial sum per tile; slot kMaxTiles: the result
__device__ __align__(256) double g_error_scratch[kMaxTiles + 1];


// Same arithmetic as the handle-based error kernel, reading the caller's dense
// layouts directly: M (m x n), V (m x r), W (r x n), all row-major.
__global__ void __launch_bounds__(256) error_dense_tile_kernel(const float* __restrict__ M,
                                                               const float* __restrict__ V,
                                                               const float* __restrict__ W, int64_t m, int64_t n,
                                                               int r, double* __restrict__ partials) {
    // rows of Vs are read as float4: 16-byte aligned base, row stride a multiple of 4 floats
    __shared__ __align__(16) float Vs[nmfk::kMaxRank][kTile + 4];
    static_assert((kTile + 4) % 4 == 0, "Vs rows must keep float4 alignment");
    __shared__ float Ws[nmfk::kMaxRank][kTile + 1];
    const int64_t ntj = (n + kTile - 1) / kTile;
    const int64_t ti = blockIdx.x / ntj, tj = blockIdx.x - ti * ntj;
    const int64_t i0 = ti * kTile, j0 = tj * kTile;
    for (int e = threadIdx.x; e < kTile * r; e += blockDim.x) {
        const int row = e / r, k = e - row * r;
        Vs[k][row] = (i0 + row < m) ? V[(i0 + row) * r + k] : 0.f;
        const int col = e % kTile, kk = e / kTile;
        Ws[kk][col] = (j0 + col < n) ? W[(int64_t)kk * n + j0 + col] : 0.f;
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
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(va[a], Ws[k][tx + 16 * b], acc[a][b]);
    }
    // as the allocating error kernel: a thread's four squared residuals of a row in
    // FP32, those sums in FP64
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
            const float e = M[i * n + j] - acc[a][b];
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

// Sums the `count` partials in a fixed order and writes the norm.
__global__ void finish_kernel(const double* __restrict__ partials, int64_t count, double* __restrict__ out) {
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

// Device address of the scratch array on the calling thread's current device.
// Looked up on every call (cheap once the module is loaded), so nothing stale
// survives a device reset or a new primary context.
cudaError_t scratch_address(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_error_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<double*>(p);
    return cudaSuccess;
}

// True if p is device (or managed) memory that the current device can address.
bool on_current_device(const void* p) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" int nmf_error_noalloc(const float* M, const float* V, const float* W, int64_t m, int64_t n, int r,
                                 void* stream, double* err_out) {
    if (!M || !V || !W || !err_out) return NMF_EINVAL;
    if (m < 1 || n < 1 || r < 1 || r > nmfk::kMaxRank) return NMF_EINVAL;
    const int64_t tiles = ((m + kTile - 1) / kTile) * ((n + kTile - 1) / kTile);
    if (tiles > kMaxTiles) return NMF_ETOOBIG;
    // the kernels read the caller's arrays in place: host pointers are rejected, not staged
    if (!on_current_device(M) || !on_current_device(V) || !on_current_device(W)) return NMF_EINVAL;
    double* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) {
        cudaGetLastError();
        return NMF_ECUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Every partial slot [0, tiles) is written before it is read and the result
    // slot is overwritten, so nothing from an earlier call needs clearing.
    error_dense_tile_kernel<<<(unsigned)tiles, 256, 0, st>>>(M, V, W, m, n, r, scratch);
    finish_kernel<<<1, 256, 0, st>>>(scratch, tiles, scratch + kMaxTiles);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(err_out, scratch + kMaxTiles, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return NMF_ECUDA;
    }
    return NMF_OK;
}
