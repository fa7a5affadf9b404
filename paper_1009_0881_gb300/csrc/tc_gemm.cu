// Tall-skinny BF16 products on the 5th-generation tensor cores (tcgen05) for the
// precision form: out[s][a][k] = sum_{kk in split s} A[a][kk] * B[k][kk]
// with A (Ma x K) and B (N x K) bfloat16, both K-major (K contiguous), and FP32
// accumulation in tensor memory.  Covers A = M W^T (A = M, B = W) and
// C^T = M^T V (A = M^T, B = V^T) of a sweep (Appendix A.1 products).
//
// One CTA computes a 128 x BN tile over one K split:
//   warp 0, one thread  : TMA producer, 64-column K blocks (128-byte rows,
//                         128-byte swizzle) of A and B into a ring of stages;
//   warp 1, one thread  : issues tcgen05.mma (M=128, N=BN, K=16 per
//                         instruction, four per stage) into a TMEM accumulator
//                         and frees each stage with tcgen05.commit;
//   all four warps      : epilogue, tcgen05.ld of the accumulator (warp w owns
//                         TMEM lanes 32w..32w+31 = rows of the tile) and FP32
//                         stores of the split's partial tile.
// Every mbarrier wait is bounded; a wait that gives up sets the error flag.
#include <cuda.h>

#include "nmf_internal.cuh"
#include "ptx.cuh"
#include "tc_gemm.cuh"

namespace nmfk {

namespace {

constexpr int TM_ROWS = 128;          // MMA M
constexpr int KB = 64;                // K columns per stage (128 bytes of bf16)
constexpr int NSTAGE = 4;  // two CTAs per SM (about 99 KB of shared memory each)
constexpr int A_STAGE = TM_ROWS * KB * 2;  // 16 KiB

__device__ __forceinline__ uint32_t elect_lane0() { return (threadIdx.x & 31) == 0; }

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// 8-row core groups 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* p) {
    const uint64_t addr = ptx::smem_u32(p);
    uint64_t d = (addr & 0x3FFFFull) >> 4;  // start address
    d |= 1ull << 16;                         // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
    d |= 1ull << 46;                         // descriptor version
    d |= 2ull << 61;                         // 128-byte swizzle
    return d;
}

// Instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128, N = bn.
__host__ __device__ constexpr uint32_t idesc_bf16(int bn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(TM_ROWS >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, bool accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accum)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     ptx::smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int BN>
__global__ void __launch_bounds__(128, 2)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const TcGemmParams p) {
    constexpr int B_STAGE = BN * KB * 2;
    constexpr int STAGE = A_STAGE + B_STAGE;
    constexpr uint32_t TMEM_COLS = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment of every stage (swizzle atoms)
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(base + NSTAGE * STAGE);
    uint64_t* empty = full + NSTAGE;
    uint64_t* done = empty + NSTAGE;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

    // programmatic dependent launch: the launch overlaps the end of the previous kernel,
    // everything below (the factor operand, the skip flag) waits for its results
    ptx::grid_dependency_wait();
    ptx::launch_dependents();
    if (p.skip && *(volatile const int*)p.skip) return;  // converged problem: nothing to do
    const int warp = threadIdx.x >> 5;
    const int m0 = blockIdx.x * TM_ROWS;
    const int split = blockIdx.y;
    const int kb0 = split * p.kblocks_per_split;
    const int kb1 = min(p.kblocks_total, kb0 + p.kblocks_per_split);
    const int nkb = max(0, kb1 - kb0);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         ptx::smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < NSTAGE; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        ptx::mbar_init(done, 1);
        ptx::fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0 && elect_lane0()) {
        // producer
        for (int i = 0; i < nkb; ++i) {
            const int s = i % NSTAGE;
            if (i >= NSTAGE && !ptx::mbar_wait(&empty[s], (uint32_t)(((i / NSTAGE) - 1) & 1))) ok = false;
            unsigned char* st = base + s * STAGE;
            ptx::mbar_arrive_expect_tx(&full[s], STAGE);
            ptx::tma_load_2d(st, &tmA, &full[s], (kb0 + i) * KB, m0);
            ptx::tma_load_2d(st + A_STAGE, &tmB, &full[s], (kb0 + i) * KB, 0);
        }
    } else if (warp == 1 && elect_lane0()) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(BN);
        for (int i = 0; i < nkb; ++i) {
            const int s = i % NSTAGE;
            if (!ptx::mbar_wait(&full[s], (uint32_t)((i / NSTAGE) & 1))) ok = false;
            tc_fence_after();
            unsigned char* st = base + s * STAGE;
            const uint64_t ad = smem_desc_sw128(st);
            const uint64_t bd = smem_desc_sw128(st + A_STAGE);
#pragma unroll
            for (int kk = 0; kk < KB / 16; ++kk)  // 16 bf16 = 32 bytes per MMA: +2 in descriptor units
                tc_mma(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (i | kk) != 0);
            tc_commit(&empty[s]);  // stage free once these MMAs have read it
        }
        tc_commit(done);  // accumulator complete
    }
    __syncwarp();

    // epilogue: wait for the accumulator, TMEM -> registers -> global partial tile
    if (nkb > 0 && !ptx::mbar_wait(done, 0)) ok = false;
    tc_fence_after();
    const int row = m0 + warp * 32 + (threadIdx.x & 31);
    float* out = p.out + (int64_t)split * p.split_stride;
#pragma unroll
    for (int c = 0; c < BN; c += 16) {
        float v[16];
        if (nkb > 0) {
            tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = 0.f;
        }
        if (row < p.Ma) {
#pragma unroll
            for (int i = 0; i < 16; i += 4)
                if (c + i < p.ncols)
                    *reinterpret_cast<float4*>(out + (int64_t)row * p.ldo + c + i) =
                        make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        }
    }
    if (!ok) atomicExch(p.err_flag, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

template <int BN>
size_t smem_bytes_t() {
    return 1024 + (size_t)NSTAGE * (A_STAGE + BN * KB * 2) + (2 * NSTAGE + 1) * sizeof(uint64_t) + 16;
}

template <int BN>
cudaError_t set_attr_t() {
    return cudaFuncSetAttribute(tc_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes_t<BN>());
}

template <int BN>
cudaError_t launch_t(const CUtensorMap& tmA, const CUtensorMap& tmB, const TcGemmParams& p, cudaStream_t st) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)((p.Ma + TM_ROWS - 1) / TM_ROWS), (unsigned)p.splits);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = smem_bytes_t<BN>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tc_gemm_kernel<BN>, tmA, tmB, p);
}

}  // namespace

int tc_block_n(int r) { return (int)round_up(r, 16); }

cudaError_t tc_gemm_init() {
    cudaError_t e = set_attr_t<16>();
    if (e == cudaSuccess) e = set_attr_t<32>();
    if (e == cudaSuccess) e = set_attr_t<48>();
    if (e == cudaSuccess) e = set_attr_t<64>();
    return e;
}

void tc_gemm_plan(TcGemmParams& p, int64_t K, int num_sms) {
    p.kblocks_total = (int)ceil_div(K, KB);
    const int64_t tiles = ceil_div(p.Ma, TM_ROWS);
    int64_t s = ceil_div(2 * (int64_t)num_sms, tiles);  // about two CTAs per SM
    const int64_t min_kb = 8;                           // keep at least 8 K blocks per split
    if (s > ceil_div(p.kblocks_total, min_kb)) s = ceil_div(p.kblocks_total, min_kb);
    if (s < 1) s = 1;
    p.kblocks_per_split = (int)ceil_div(p.kblocks_total, s);
    p.splits = (int)ceil_div(p.kblocks_total, p.kblocks_per_split);
}

cudaError_t tc_gemm_launch(int bn, const CUtensorMap& tmA, const CUtensorMap& tmB, const TcGemmParams& p,
                           cudaStream_t st) {
    switch (bn) {
        case 16: return launch_t<16>(tmA, tmB, p, st);
        case 32: return launch_t<32>(tmA, tmB, p, st);
        case 48: return launch_t<48>(tmA, tmB, p, st);
        case 64: return launch_t<64>(tmA, tmB, p, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace nmfk
