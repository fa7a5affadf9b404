// Fused half-sweep kernels (fused.cu): products + factor update in one launch.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "nmf_internal.cuh"

namespace nmfk {

enum HalfSweepMode { kModeHals = 0, kModeMu = 1, kModeStore = 2 };

struct HalfSweepParams {
    int Na;            // rows of the factor F (= columns a of the product)
    int64_t K;         // product length
    int kchunk;        // K rows per cluster rank (multiple of the stage height)
    int cs;            // cluster size (CTAs per tile of F)
    int r, rp;         // rank and padded leading dimension of F
    float* F;          // Na x rp factor, updated in place (HALS / MU)
    const float* Gin;  // gin_count Gram partial slabs (r x rp each, stride gin_stride)
    int gin_count;
    int64_t gin_stride;
    float* Gout;       // one Gram slab per tile of F (HALS / MU)
    int64_t gout_stride;
    float* Pout;       // STORE mode: reduced product rows, Na x rp
    int* err_flag;     // set to 1 if a bounded wait gave up
    const int* skip;   // optional: when *skip != 0 the launch does nothing (converged problem)
    double* obj_part;  // optional (HALS / MU): per-CTA terms of the objective identity, 2 per CTA:
                       // [2b] = <P rows, new F rows>, [2b+1] = <G, this CTA's slice of the new slab>
};

struct HalfSweepLaunch {
    CUtensorMap tmX;  // X: K rows x (>= Na) columns, box ba x 32
    CUtensorMap tmY;  // Y: K rows x rp columns, box br x 32
    HalfSweepParams p;
    int br;
    int ba;  // rows of F per tile: 16, 32 or 64
    int mode;
    int tiles;
};

cudaError_t tma_init();
// 2-D tiled tensor map (row-major height x width, ld_bytes between rows).
cudaError_t make_tmap_2d(CUtensorMap* map, CUtensorMapDataType type, const void* base, uint64_t width,
                         uint64_t height, uint64_t ld_bytes, uint32_t box_w, uint32_t box_h,
                         CUtensorMapSwizzle swizzle);
cudaError_t make_tmap_f32(CUtensorMap* map, const float* base, uint64_t width, uint64_t height, uint64_t ld,
                          uint32_t box_w, uint32_t box_h);
cudaError_t half_sweep_init();
// Number of clusters of `cs` CTAs the device can hold at once (0: not schedulable).
int half_sweep_active_clusters(int br, int ba, int r, int cs);
int half_sweep_stage_rows();
size_t half_sweep_smem_bytes(int br, int ba, int r, int cs);
cudaError_t half_sweep_launch(const HalfSweepLaunch& hl, cudaStream_t st);
// Gram partial slabs of a tall factor, one per tile of `tile_rows` (<= 64) rows.
cudaError_t gram_tiles_launch(const float* F, int64_t rows, int r, int rp, int tile_rows, float* out,
                              int64_t out_stride, cudaStream_t st, const int* skip = nullptr);

}  // namespace nmfk
