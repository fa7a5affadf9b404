// FP32 tall-skinny products of a HALS / MU / ANLS sweep (Section 2, Appendix A.1):
// A = M W^T, B = W W^T, C = V^T M, D = V^T V, all in the "TN" form
//   out[a, k] = sum_kk X[kk, a] * Y[kk, k]
// with the long dimension kk (n for A and B, m for C and D) as the row index of
// both operands, so every operand tile is a coalesced slab of whole rows.
//
// CUDA-core FFMA kernel: the FP32 path must match the FP64 oracle to 1e-5, which
// rules out single-pass TF32/BF16 tensor-core products.  One CTA computes a
// 64 x BR output tile over one K split; tiles of several independent products
// (the factor product and its Gram matrix) share one launch, and each split
// writes its own partial slab, which the consumer reduces in a fixed order.
#include "nmf_internal.cuh"

namespace nmfk {

namespace {

constexpr int BA = 64;   // output rows per CTA
constexpr int BK = 32;   // K rows per stage
constexpr int NT = 256;  // threads per CTA

template <int BR>
__global__ void __launch_bounds__(NT) gemm_tn_kernel(const GemmBatch batch) {
    constexpr int TN = BR / 16;  // output columns per thread
    constexpr int TM = 4;        // output rows per thread
    constexpr int YV = BK * BR / 4;  // float4 per Y stage
    __shared__ __align__(16) float Xs[2][BK][BA];
    __shared__ __align__(16) float Ys[2][BK][BR];

    const int bid = blockIdx.x;
    GemmTask T = batch.t[0];
#pragma unroll
    for (int t = 1; t < kMaxGemmTasks; ++t)
        if (t < batch.ntasks && bid >= batch.t[t].tile_begin) T = batch.t[t];
    const int local = bid - T.tile_begin;
    const int a_tile = local % T.a_tiles;
    const int split = local / T.a_tiles;
    const int64_t k0 = (int64_t)split * T.kchunk;
    const int64_t k1 = min(T.K, k0 + (int64_t)T.kchunk);
    const int a0 = a_tile * BA;
    const int tid = threadIdx.x;
    const int tx = tid & 15;  // column group
    const int ty = tid >> 4;  // row group

    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

    float4 xr[2];
    float4 yr[(YV + NT - 1) / NT];

    auto load = [&](int64_t kb) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int idx = tid + q * NT;  // 512 float4: 32 rows x 16
            const int row = idx >> 4;
            const int col = (idx & 15) * 4;
            const int64_t kk = kb + row;
            const int a = a0 + col;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kk < k1 && a < T.ldx) v = *reinterpret_cast<const float4*>(T.X + kk * T.ldx + a);
            xr[q] = v;
        }
#pragma unroll
        for (int q = 0; q < (YV + NT - 1) / NT; ++q) {
            const int idx = tid + q * NT;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (idx < YV) {
                const int row = idx / (BR / 4);
                const int col = (idx % (BR / 4)) * 4;
                const int64_t kk = kb + row;
                if (kk < k1 && col < T.ldy) v = *reinterpret_cast<const float4*>(T.Y + kk * T.ldy + col);
            }
            yr[q] = v;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int idx = tid + q * NT;
            *reinterpret_cast<float4*>(&Xs[buf][idx >> 4][(idx & 15) * 4]) = xr[q];
        }
#pragma unroll
        for (int q = 0; q < (YV + NT - 1) / NT; ++q) {
            const int idx = tid + q * NT;
            if (idx < YV)
                *reinterpret_cast<float4*>(&Ys[buf][idx / (BR / 4)][(idx % (BR / 4)) * 4]) = yr[q];
        }
    };

    if (k0 < k1) {
        load(k0);
        store(0);
    }
    __syncthreads();
    int buf = 0;
    for (int64_t kb = k0; kb < k1; kb += BK) {
        const bool has_next = kb + BK < k1;
        if (has_next) load(kb + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a4 = *reinterpret_cast<const float4*>(&Xs[buf][kk][ty * TM]);
            const float av[4] = {a4.x, a4.y, a4.z, a4.w};
            float bv[TN];
#pragma unroll
            for (int j = 0; j < TN; ++j) bv[j] = Ys[buf][kk][tx * TN + j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (has_next) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }

    float* out = T.out + (int64_t)split * T.split_stride;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int a = a0 + ty * TM + i;
        if (a >= T.Na) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int k = tx * TN + j;
            if (k < T.ldo) out[(int64_t)a * T.ldo + k] = acc[i][j];
        }
    }
}

}  // namespace

void gemm_plan_task(GemmTask& t, int num_sms, int max_splits) {
    t.a_tiles = (int)ceil_div(t.Na, BA);
    // aim for about two CTAs per SM over all tiles, each split at least 4 K stages
    int64_t by_k = ceil_div(t.K, 4 * BK);
    int64_t want = ceil_div(2 * (int64_t)num_sms, t.a_tiles);
    int64_t s = want < by_k ? want : by_k;
    if (s < 1) s = 1;
    if (s > max_splits) s = max_splits;
    t.kchunk = (int)round_up(ceil_div(t.K, s), BK);
    t.splits = (int)ceil_div(t.K, t.kchunk);
    if (t.splits < 1) t.splits = 1;
}

cudaError_t gemm_tn_launch(GemmBatch& b, int br, cudaStream_t st) {
    int tiles = 0;
    for (int i = 0; i < b.ntasks; ++i) {
        b.t[i].tile_begin = tiles;
        tiles += b.t[i].a_tiles * b.t[i].splits;
    }
    b.total_tiles = tiles;
    if (tiles == 0) return cudaSuccess;
    dim3 grid(tiles), block(NT);
    switch (br) {
        case 16: gemm_tn_kernel<16><<<grid, block, 0, st>>>(b); break;
        case 32: gemm_tn_kernel<32><<<grid, block, 0, st>>>(b); break;
        case 48: gemm_tn_kernel<48><<<grid, block, 0, st>>>(b); break;
        case 64: gemm_tn_kernel<64><<<grid, block, 0, st>>>(b); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace nmfk
