#include <algorithm>
// Kernels around the tcgen05 products of the BF16 precision form: BF16 operand
// copies, the final Gram matrix from per-tile slabs, and the row update.
//
// The row update reads the split-K partial tiles of the product (summed in a
// fixed order), runs the HALS or MU step of Algorithm HALS / MU on 64 rows per
// CTA with the same code as the fused FP32 kernel (rowupdate.cuh), stores the
// new rows in FP32, their transposed BF16 copy (the next product's operand)
// and the Gram slab F_tile^T F_tile of the tile for the other half-sweep.
#include <cuda_bf16.h>

#include "fused.cuh"
#include "ptx.cuh"
#include "rowupdate.cuh"
#include "tc_gemm.cuh"

namespace nmfk {

namespace {

using rowupd::f4add;
constexpr int NT = rowupd::NT;

// out[r ldo + c] = bf16(in[r ldi + c]): rows strided over the blocks, four columns per
// thread (float4 in, 8 bytes out) when both leading dimensions keep rows 16- and 8-byte
// aligned, a scalar tail otherwise.
__global__ void to_bf16_kernel(const float* __restrict__ in, int64_t ldi, int64_t rows, int64_t cols,
                               __nv_bfloat16* __restrict__ out, int64_t ldo) {
    const bool vec = ldi % 4 == 0 && ldo % 4 == 0 && reinterpret_cast<uintptr_t>(in) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(out) % 8 == 0;
    const int64_t c4 = vec ? cols / 4 : 0;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const float* src = in + r * ldi;
        __nv_bfloat16* dst = out + r * ldo;
        for (int64_t q = threadIdx.x; q < c4; q += blockDim.x) {
            const float4 v = reinterpret_cast<const float4*>(src)[q];
            __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
            uint2 packed;
            packed.x = *reinterpret_cast<const unsigned*>(&lo);
            packed.y = *reinterpret_cast<const unsigned*>(&hi);
            reinterpret_cast<uint2*>(dst)[q] = packed;
        }
        for (int64_t c = 4 * c4 + threadIdx.x; c < cols; c += blockDim.x) dst[c] = __float2bfloat16_rn(src[c]);
    }
}

// 32 x 32 tiles through shared memory
__global__ void to_bf16_t_kernel(const float* __restrict__ in, int64_t ldi, int64_t rows, int64_t cols,
                                 __nv_bfloat16* __restrict__ out, int64_t ldo) {
    __shared__ float tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int64_t r = r0 + dy, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[dy][threadIdx.x] = in[r * ldi + c];
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int64_t c = c0 + dy, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[c * ldo + r] = __float2bfloat16_rn(tile[threadIdx.x][dy]);
    }
}

// G[e] = sum of the slabs, in two levels so that thousands of slabs do not
// serialise on one thread: block (x, y) sums slab chunk y of outputs
// 256x .. 256x+255 into part[y], and the last block of column x to finish
// (ticket in cnt[x], reset afterwards) adds the chunk sums in chunk order.
__global__ void gram_final_kernel(const float* __restrict__ slabs, int count, int64_t stride, int n,
                                  float* __restrict__ G, float* __restrict__ part, int* cnt, const int* skip) {
    ptx::grid_dependency_wait();  // the slabs and the flag come from the previous kernel
    ptx::launch_dependents();
    if (skip && *(volatile const int*)skip) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int S = gridDim.y, y = blockIdx.y;
    const int per = (count + S - 1) / S;
    const int q0 = y * per, q1 = min(count, q0 + per);
    if (e < n) {
        float s = 0.f;
        for (int q = q0; q < q1; ++q) s += slabs[(int64_t)q * stride + e];
        part[(int64_t)y * n + e] = s;
    }
    __threadfence();
    __syncthreads();
    __shared__ int last;
    if (threadIdx.x == 0) last = atomicAdd(&cnt[blockIdx.x], 1) == S - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (e < n) {
        float s = 0.f;
        for (int k = 0; k < S; ++k) s += *(volatile const float*)&part[(int64_t)k * n + e];
        G[e] = s;
    }
    if (threadIdx.x == 0) cnt[blockIdx.x] = 0;
}

// Row stride of the transposed tile of BA rows (odd: conflict-free columns).
template <int BA>
__host__ __device__ constexpr int tld() { return BA + 1; }
// G zero-padded to 64 x 64 for the HALS walk, row by row in four 16-column blocks
// with block b at offset 20 b (row stride 80): the four 16-byte reads of a
// quarter-warp (two rows, four blocks at the same offset) fall in distinct bank groups.
constexpr int GBK = 20;
constexpr int GRS = 4 * GBK;

// HALS update (Algorithm HALS) of the BA rows of a tile (64, 32 or 16), four lanes per row
// (all 256 threads busy for 64 rows): lane q of a row's quad holds columns 16q .. 16q+15 of
// F_i and of g = P_i - F_i G in registers.  Columns k = 0 .. r-1 are walked in
// order: the owner lane of column k computes F_ik <- max(0, F_ik + g_k / G_kk)
// and broadcasts the change d within the quad, then every lane applies
// g_j -= d G_kj to its sixteen columns (those at or before k are finished and
// no longer read).  G64 is G zero-padded to 64 x 64 (layout above); the loop over k is fully
// unrolled so that every register index is static.  New rows go back to Fn
// (row-major) and FT (transposed, for the BF16 copy).
template <int BA>
__device__ __forceinline__ void hals_rows_quad(int r, int rp, float* Fn, const float* Ared, const float* Dn,
                                               float* FT, const float* G64, const float* Ginv) {
    constexpr int TLD = tld<BA>();
    const int tid = threadIdx.x;
    if (tid >= 4 * BA) return;  // whole warps: 4 BA is a multiple of 32
    const int rr = tid >> 2, qd = tid & 3;
    const int gbase = (tid & 31) & ~3;
    float f[16], g[16];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int c = 16 * qd + 4 * v;
        const float4 fv = *reinterpret_cast<const float4*>(Fn + rr * kMaxRank + c);
        float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c < rp) {
            const float4 av = *reinterpret_cast<const float4*>(Ared + rr * kMaxRank + c);
            const float4 dv = *reinterpret_cast<const float4*>(Dn + rr * kMaxRank + c);
            gv = make_float4(av.x - dv.x, av.y - dv.y, av.z - dv.z, av.w - dv.w);
        }
        f[4 * v] = fv.x;
        f[4 * v + 1] = fv.y;
        f[4 * v + 2] = fv.z;
        f[4 * v + 3] = fv.w;
        g[4 * v] = gv.x;
        g[4 * v + 1] = gv.y;
        g[4 * v + 2] = gv.z;
        g[4 * v + 3] = gv.w;
    }
    // k = 16 q0 + i0: the block loop stays rolled (compact code), the steps inside
    // are unrolled so that the owner's entry i0 is a register
    for (int q0 = 0; q0 < 4 && 16 * q0 < r; ++q0) {
#pragma unroll
        for (int i0 = 0; i0 < 16; ++i0) {
            const int k = 16 * q0 + i0;
            if (k < r) {
                float dl = 0.f;
                if (qd == q0) {
                    const float nv = fmaxf(0.f, fmaf(g[i0], Ginv[k], f[i0]));
                    dl = nv - f[i0];
                    f[i0] = nv;
                }
                const float d = __shfl_sync(0xffffffffu, dl, gbase + q0);
                const float4* gk = reinterpret_cast<const float4*>(G64 + k * GRS + GBK * qd);
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float4 gv = gk[v];
                    g[4 * v] = fmaf(-d, gv.x, g[4 * v]);
                    g[4 * v + 1] = fmaf(-d, gv.y, g[4 * v + 1]);
                    g[4 * v + 2] = fmaf(-d, gv.z, g[4 * v + 2]);
                    g[4 * v + 3] = fmaf(-d, gv.w, g[4 * v + 3]);
                }
            }
        }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v)
        *reinterpret_cast<float4*>(Fn + rr * kMaxRank + 16 * qd + 4 * v) =
            make_float4(f[4 * v], f[4 * v + 1], f[4 * v + 2], f[4 * v + 3]);
#pragma unroll
    for (int j = 0; j < 16; ++j) FT[(16 * qd + j) * TLD + rr] = f[j];
}

// Dn = Fn G for the 16 RPT rows of a tile (Fn, Dn: rows of kMaxRank floats; G: r x rp):
// thread (ty, tx) of a 16 x 16 arrangement computes columns 4tx .. 4tx+3 of rows
// ty, ty+16, ..., reading F four columns l at a time; each output is the sum
// over l = 0 .. r-1 in increasing order (the order of rowupd::rows_times_gram).
template <int RPT>
__device__ __forceinline__ void rows_times_gram64(int r, int rp, const float* Fn, const float* Gs, float* Dn) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int c0 = 4 * tx;
    float acc[RPT][4];
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    if (c0 < rp) {
        for (int l0 = 0; l0 < r; l0 += 4) {
            float4 fv[RPT], gv[4];
#pragma unroll
            for (int i = 0; i < RPT; ++i) fv[i] = *reinterpret_cast<const float4*>(Fn + (ty + 16 * i) * kMaxRank + l0);
#pragma unroll
            for (int e = 0; e < 4; ++e)
                gv[e] = l0 + e < r ? *reinterpret_cast<const float4*>(Gs + (l0 + e) * rp + c0)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                const float f[4] = {fv[i].x, fv[i].y, fv[i].z, fv[i].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (l0 + e < r) {
                        acc[i][0] = fmaf(f[e], gv[e].x, acc[i][0]);
                        acc[i][1] = fmaf(f[e], gv[e].y, acc[i][1]);
                        acc[i][2] = fmaf(f[e], gv[e].z, acc[i][2]);
                        acc[i][3] = fmaf(f[e], gv[e].w, acc[i][3]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i)
        *reinterpret_cast<float4*>(Dn + (ty + 16 * i) * kMaxRank + c0) =
            make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
}

template <int MODE, int BA>
__global__ void __launch_bounds__(NT, 1) rows_update_kernel(const RowsParams q) {
    constexpr int TLD = tld<BA>();
    extern __shared__ __align__(16) float sm[];
    ptx::grid_dependency_wait();  // the products, the Gram matrix and the flag come from earlier kernels
    ptx::launch_dependents();
    if (q.skip && *(volatile const int*)q.skip) return;  // converged problem: nothing to do
    const int r = q.r, rp = q.rp;
    float* Gs = sm;                       // r x rp
    float* Ginv = Gs + r * rp;            // kMaxRank
    float* Fn = Ginv + kMaxRank;          // BA x kMaxRank
    float* Ared = Fn + BA * kMaxRank;     // BA x kMaxRank
    float* Dn = Ared + BA * kMaxRank;     // BA x kMaxRank
    float* FT = Dn + BA * kMaxRank;       // kMaxRank x TLD (HALS: new rows transposed)
    float* G64 = FT + kMaxRank * TLD;     // kMaxRank x GRS (HALS: G zero-padded)
    const int tid = threadIdx.x;
    const int64_t row0 = (int64_t)blockIdx.x * BA;
    const int R = BA;
    const int Q4 = rp / 4;

    // incoming rows (async), Gram matrix, reduced product rows
    for (int e = tid; e < BA * (kMaxRank / 4); e += NT) {
        const int rr = e / (kMaxRank / 4), k4 = e - rr * (kMaxRank / 4);
        const int64_t row = row0 + rr;
        float* dst = Fn + rr * kMaxRank + 4 * k4;
        if (k4 < Q4)
            ptx::cp_async16(dst, q.F + (row < q.rows ? row : 0) * rp + 4 * k4, row < q.rows ? 16u : 0u);
        else
            *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    ptx::cp_async_commit();
    if (MODE != rowupd::kModeStore) {
        for (int e = tid; e < r * Q4; e += NT)
            reinterpret_cast<float4*>(Gs)[e] = reinterpret_cast<const float4*>(q.G)[e];
        for (int e = tid; e < BA * Q4; e += NT) {
            const int rr = e / Q4, k4 = e - rr * Q4;
            const int64_t row = row0 + rr;
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
            if (row < q.rows) {
                const float4* src = reinterpret_cast<const float4*>(q.P + row * rp) + k4;
                const int64_t ps4 = q.ps / 4;
#pragma unroll 4
                for (int sp = 0; sp < q.splits; ++sp) s = f4add(s, src[sp * ps4]);
            }
            *reinterpret_cast<float4*>(Ared + rr * kMaxRank + 4 * k4) = s;
        }
    }
    ptx::cp_async_wait_all();
    __syncthreads();

    if (MODE != rowupd::kModeStore) {
        for (int k = tid; k < kMaxRank; k += NT) Ginv[k] = (k < r && Gs[k * rp + k] > 0.f) ? 1.f / Gs[k * rp + k] : 0.f;
        rows_times_gram64<BA / 16>(r, rp, Fn, Gs, Dn);
        __syncthreads();
        if (MODE == rowupd::kModeHals) {
            for (int e = tid; e < kMaxRank * kMaxRank; e += NT) {
                const int k = e / kMaxRank, j = e - k * kMaxRank;
                G64[k * GRS + (j >> 4) * GBK + (j & 15)] = (k < r && j < r) ? Gs[k * rp + j] : 0.f;
            }
            __syncthreads();
            hals_rows_quad<BA>(r, rp, Fn, Ared, Dn, FT, G64, Ginv);
            __syncthreads();
            // new rows to the factor in global memory
            for (int e = tid; e < BA * Q4; e += NT) {
                const int rr = e / Q4, k4 = e - rr * Q4;
                const int64_t row = row0 + rr;
                if (row < q.rows)
                    *reinterpret_cast<float4*>(q.F + row * rp + 4 * k4) =
                        *reinterpret_cast<const float4*>(Fn + rr * kMaxRank + 4 * k4);
            }
        } else {
            rowupd::update_rows_any<MODE>(q.F, (int)q.rows, r, rp, R, row0, Fn, Ared, Dn, Gs, Ginv);
        }
        __syncthreads();
    } else {
        // rows past the end read as zero already; nothing to update
        __syncthreads();
    }

    // transposed BF16 copy of the new rows: Fb[k][row]
    if (q.Fb) {
        for (int e = tid; e < r * BA; e += NT) {
            const int k = e / BA, rr = e - k * BA;
            const int64_t row = row0 + rr;
            const float v = MODE == rowupd::kModeHals ? FT[k * TLD + rr] : Fn[rr * kMaxRank + k];
            if (row < q.rows) q.Fb[(int64_t)k * q.ldb + row] = __float2bfloat16_rn(v);
        }
    }
    // Gram slab of the tile, 4 x 4 outputs per thread
    {
        const int tx = tid & 15, ty = tid >> 4;
        float ga[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) ga[i][j] = 0.f;
#pragma unroll 4
        for (int rr = 0; rr < R; ++rr) {
            const float4 u = *reinterpret_cast<const float4*>(Fn + rr * kMaxRank + ty * 4);
            const float4 v = *reinterpret_cast<const float4*>(Fn + rr * kMaxRank + tx * 4);
            const float uu[4] = {u.x, u.y, u.z, u.w}, vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) ga[i][j] = fmaf(uu[i], vv[j], ga[i][j]);
        }
        float* gout = q.Gout + (int64_t)blockIdx.x * q.gout_stride;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int l = ty * 4 + i;
            if (l < r && tx * 4 < rp)
                *reinterpret_cast<float4*>(gout + l * rp + tx * 4) = make_float4(ga[i][0], ga[i][1], ga[i][2], ga[i][3]);
        }
    }
}

// Launch with programmatic stream serialization: the kernel may start while the previous one
// finishes; it waits (griddepcontrol.wait) before reading that kernel's results.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

size_t rows_smem_bytes(int r, int rp, int ba) {
    return sizeof(float) * ((size_t)r * rp + kMaxRank + 3 * ba * kMaxRank + kMaxRank * (ba + 1) + kMaxRank * GRS);
}

}  // namespace

cudaError_t make_tmap_bf16_sw128(CUtensorMap* map, const __nv_bfloat16* base, uint64_t width, uint64_t height,
                                 uint64_t ld, uint32_t box_h) {
    return make_tmap_2d(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, base, width, height, ld * 2, 64, box_h,
                        CU_TENSOR_MAP_SWIZZLE_128B);
}

cudaError_t to_bf16_launch(const float* in, int64_t ldi, int64_t rows, int64_t cols, __nv_bfloat16* out, int64_t ldo,
                           bool transpose, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if (transpose) {
        dim3 block(32, 8), grid((unsigned)ceil_div(cols, 32), (unsigned)ceil_div(rows, 32));
        to_bf16_t_kernel<<<grid, block, 0, st>>>(in, ldi, rows, cols, out, ldo);
    } else {
        int64_t g = std::min<int64_t>(rows, 65535LL * 16);
        to_bf16_kernel<<<(unsigned)g, 256, 0, st>>>(in, ldi, rows, cols, out, ldo);
    }
    return cudaGetLastError();
}

cudaError_t gram_final_launch(const float* slabs, int count, int64_t stride, int r, int rp, float* G, float* part,
                              int* cnt, cudaStream_t st, const int* skip) {
    const int n = r * rp;
    const int S = (int)std::min<int64_t>(kGramChunks, std::max<int64_t>(1, ceil_div(count, 16)));
    return launch_pdl(gram_final_kernel, dim3((unsigned)ceil_div(n, 256), (unsigned)S), dim3(256), 0, st, slabs, count,
                      stride, n, G, part, cnt, skip);
}

template <int BA>
cudaError_t rows_update_init_ba() {
    const int maxs = (int)rows_smem_bytes(kMaxRank, kMaxRank, BA);
    cudaError_t e = cudaFuncSetAttribute(rows_update_kernel<rowupd::kModeHals, BA>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(rows_update_kernel<rowupd::kModeMu, BA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 maxs);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(rows_update_kernel<rowupd::kModeStore, BA>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
    return e;
}

cudaError_t rows_update_init() {
    cudaError_t e = rows_update_init_ba<64>();
    if (e == cudaSuccess) e = rows_update_init_ba<32>();
    return e == cudaSuccess ? rows_update_init_ba<16>() : e;
}

template <int BA>
cudaError_t rows_update_launch_ba(const RowsParams& q, int mode, cudaStream_t st) {
    const size_t smem = rows_smem_bytes(q.r, q.rp, BA);
    const unsigned grid = (unsigned)ceil_div(q.rows, BA);
    switch (mode) {
        case rowupd::kModeHals: return launch_pdl(rows_update_kernel<rowupd::kModeHals, BA>, dim3(grid), dim3(NT), smem, st, q);
        case rowupd::kModeMu: return launch_pdl(rows_update_kernel<rowupd::kModeMu, BA>, dim3(grid), dim3(NT), smem, st, q);
        default: return launch_pdl(rows_update_kernel<rowupd::kModeStore, BA>, dim3(grid), dim3(NT), smem, st, q);
    }
}

cudaError_t rows_update_launch(const RowsParams& q, int mode, cudaStream_t st) {
    if (q.rows <= 0) return cudaSuccess;
    if (q.ba == 16) return rows_update_launch_ba<16>(q, mode, st);
    if (q.ba == 32) return rows_update_launch_ba<32>(q, mode, st);
    if (q.ba == 64) return rows_update_launch_ba<64>(q, mode, st);
    return cudaErrorInvalidValue;
}

}  // namespace nmfk
