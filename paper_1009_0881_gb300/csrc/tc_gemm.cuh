// BF16 precision form: tcgen05 tall-skinny GEMM (tc_gemm.cu) and the row
// kernels around it (bf16path.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "nmf_internal.cuh"

namespace nmfk {

struct TcGemmParams {
    int Ma;                 // rows of A (= rows of the output)
    int kblocks_total;      // ceil(K / 64)
    int kblocks_per_split;  // K blocks per CTA along grid.y
    int splits;
    float* out;             // [splits][Ma][ldo] FP32 partial tiles
    int64_t ldo, split_stride;
    int ncols;              // output columns stored (multiple of 4)
    int* err_flag;
    const int* skip;        // optional: when *skip != 0 the launch does nothing
};

cudaError_t tc_gemm_init();
int tc_block_n(int r);  // MMA N for rank r (multiple of 16)
void tc_gemm_plan(TcGemmParams& p, int64_t K, int num_sms);
cudaError_t tc_gemm_launch(int bn, const CUtensorMap& tmA, const CUtensorMap& tmB, const TcGemmParams& p,
                           cudaStream_t st);
// BF16 tensor map of a row-major (height x width) matrix with leading dimension ld
// (elements, multiple of 8), box box_h rows x 64 columns, 128-byte swizzle.
cudaError_t make_tmap_bf16_sw128(CUtensorMap* map, const __nv_bfloat16* base, uint64_t width, uint64_t height,
                                 uint64_t ld, uint32_t box_h);

// out[r*ldo + c] = bf16(in[r*ldi + c]) (transpose = false) or out[c*ldo + r] (true)
cudaError_t to_bf16_launch(const float* in, int64_t ldi, int64_t rows, int64_t cols, __nv_bfloat16* out,
                           int64_t ldo, bool transpose, cudaStream_t st);
// G[e] = sum over `count` slabs (stride `stride`) of slab[e], e < r * rp, in a fixed order:
// up to kGramChunks chunk sums (scratch `part`, kGramChunks * r * rp floats) added in chunk
// order.  `cnt` holds ceil(r * rp / 256) ints, zero before the first launch (each launch
// leaves them zero).
constexpr int kGramChunks = 32;
cudaError_t gram_final_launch(const float* slabs, int count, int64_t stride, int r, int rp, float* G, float* part,
                              int* cnt, cudaStream_t st, const int* skip = nullptr);

struct RowsParams {
    float* F;              // rows x rp factor (FP32), updated in place
    int64_t rows;
    int r, rp;
    const float* P;        // product partial slabs: row a of split s at P[s*ps + a*rp + k]
    int64_t ps;
    int splits;
    const float* G;        // final Gram matrix, r x rp
    __nv_bfloat16* Fb;     // transposed BF16 copy written after the update: Fb[k*ldb + row]
    int64_t ldb;
    float* Gout;           // Gram slab of every tile (ba rows) of the new rows
    int64_t gout_stride;
    const int* skip;       // optional: when *skip != 0 the launch does nothing
    int ba;                // rows per CTA tile (64, 32 or 16): one Gram slab per tile
};
// mode: 0 HALS, 1 MU, 2 no update (copy + Gram slabs only)
cudaError_t rows_update_launch(const RowsParams& q, int mode, cudaStream_t st);
cudaError_t rows_update_init();

}  // namespace nmfk
