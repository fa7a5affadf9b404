// Grouped half-sweeps: the batched form's persistent launch (see grouped.cuh).
//
// A tile of 64 rows of the factor F (V in a V-step, W^T in a W-step) is computed by one
// CTA: its product rows P = X^T Y over the whole of K stream in through a TMA/mbarrier
// ring (FP32 FFMA, 4 x BR/16 outputs per thread), then the HALS or MU update of the rows
// (Algorithms HALS and MU; the same row routines as the fused half-sweep kernel) with the
// Gram matrix the preceding grouped reduction formed, then the Gram slab of the new rows
// for the next half-sweep.  The CTAs stay resident and take tiles from the work-list
// until it is empty; the ring's stages run on across tiles, so each mbarrier keeps its
// phase from one tile to the next.
#include <algorithm>

#include "grouped.cuh"
#include "ptx.cuh"
#include "rowupdate.cuh"

namespace nmfk {

static_assert(alignof(GroupDesc) >= 64 && sizeof(GroupDesc) % 64 == 0,
              "tensor maps in an array of descriptors must stay 64-byte aligned");

namespace {

using rowupd::f4add;

constexpr int KS = 32;          // K rows per pipeline stage
constexpr int NST = 4;          // pipeline stages
constexpr int NT = 256;         // threads
constexpr int BA = kGroupTile;  // rows of F per tile

static_assert(NST * KS * BA >= BA * kMaxRank && NST * KS * kMaxRank >= BA * kMaxRank,
              "the ring must hold the product rows and F G of a tile");

struct GSmem {
    size_t xs, ys, gs, ginv, ared, fn, dn, red, bar, slot, total;
};

__host__ __device__ inline size_t galign(size_t v, size_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline GSmem gsmem_layout() {
    GSmem s{};
    size_t o = 0;
    s.xs = o;   o = galign(o + sizeof(float) * NST * KS * BA, 128);
    s.ys = o;   o = galign(o + sizeof(float) * NST * KS * kMaxRank, 128);
    // the product rows and F G live in the ring's buffers once the product is done (no copy is
    // in flight then: every stage of the tile has been waited for and read)
    s.ared = s.xs;
    s.dn = s.ys;
    s.gs = o;   o = galign(o + sizeof(float) * kMaxRank * kMaxRank, 128);
    s.ginv = o; o = galign(o + sizeof(float) * kMaxRank, 128);
    s.fn = o;   o = galign(o + sizeof(float) * BA * kMaxRank, 128);
    s.red = o;  o = galign(o + sizeof(double) * (NT / 32), 128);
    s.bar = o;  o = galign(o + sizeof(uint64_t) * NST, 128);
    s.slot = o; o = galign(o + sizeof(int), 128);
    s.total = o;
    return s;
}

// Sum of one double per thread over the CTA in a fixed order; valid in every thread.
__device__ __forceinline__ double gblock_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    __syncthreads();
    return s;
}

struct Bufs {
    float* Xs;
    float* Ys;
    float* Gs;
    float* Ginv;
    float* Ared;
    float* Fn;
    float* Dn;
    double* red;
    uint64_t* bar;
};

// One tile: rows [64 tile, 64 tile + 64) of d->F.  `stage` counts the ring stages this
// CTA has consumed so far (slot = stage % NST, phase parity = (stage / NST) & 1).
template <int BR, int MODE>
__device__ __forceinline__ void group_tile(const GroupDesc* d, int tile, const Bufs& b, uint32_t& stage, bool& ok) {
    constexpr int TM = BA / 16;
    constexpr int TN = BR / 16;
    constexpr uint32_t kStageBytes = sizeof(float) * KS * (BA + BR);
    const int tid = threadIdx.x;
    const int a0 = tile * BA;
    const int r = d->r, rp = d->rp, Na = d->Na;
    const int nst = (int)((d->K + KS - 1) / KS);

    if (tid == 0) {
        for (int s = 0; s < NST && s < nst; ++s) {
            const int slot = (int)((stage + s) % NST);
            ptx::mbar_arrive_expect_tx(&b.bar[slot], kStageBytes);
            ptx::tma_load_2d(b.Xs + slot * KS * BA, &d->tmX, &b.bar[slot], a0, s * KS);
            ptx::tma_load_2d(b.Ys + slot * KS * BR, &d->tmY, &b.bar[slot], 0, s * KS);
        }
    }
    // incoming rows of F (rows past Na and columns past rp read as 0) and the Gram matrix
    {
        const int Q4 = rp / 4;
        for (int e = tid; e < BA * (kMaxRank / 4); e += NT) {
            const int rr = e / (kMaxRank / 4), k4 = e - rr * (kMaxRank / 4);
            const int64_t row = (int64_t)a0 + rr;
            float* dst = b.Fn + rr * kMaxRank + 4 * k4;
            if (k4 < Q4)
                ptx::cp_async16(dst, d->F + (row < Na ? row : 0) * rp + 4 * k4, row < Na ? 16u : 0u);
            else
                *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const int F4 = r * rp / 4;
        for (int t = tid; t < F4; t += NT) ptx::cp_async16(b.Gs + 4 * t, d->G + 4 * t, 16u);
        ptx::cp_async_commit();
    }

    // ---- product rows over the whole of K, summed in two levels so that a long K does not
    // make one long float32 chain: each stage's 32 terms into a fresh partial, the partials
    // in stage order with compensated (Kahan) addition
    const int tx = tid & 15, ty = tid >> 4;
    float acc[TM][TN], cmp[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = cmp[i][j] = 0.f;
    for (int s = 0; s < nst; ++s) {
        const int slot = (int)((stage + s) % NST);
        if (!ptx::mbar_wait(&b.bar[slot], ((stage + s) / NST) & 1u)) ok = false;
        const float* xs = b.Xs + slot * KS * BA;
        const float* ys = b.Ys + slot * KS * BR;
        float part[TM][TN];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) part[i][j] = 0.f;
#pragma unroll 8
        for (int kk = 0; kk < KS; ++kk) {
            const float4 a4 = *reinterpret_cast<const float4*>(xs + kk * BA + ty * TM);
            const float av[4] = {a4.x, a4.y, a4.z, a4.w};
            float bv[TN];
            if (TN == 4) {
                const float4 b4 = *reinterpret_cast<const float4*>(ys + kk * BR + tx * TN);
                bv[0] = b4.x;
                bv[1 % TN] = b4.y;
                bv[2 % TN] = b4.z;
                bv[3 % TN] = b4.w;
            } else {
#pragma unroll
                for (int j = 0; j < TN; ++j) bv[j] = ys[kk * BR + tx * TN + j];
            }
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) part[i][j] = fmaf(av[i], bv[j], part[i][j]);
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const float y = part[i][j] - cmp[i][j];
                const float t = acc[i][j] + y;
                cmp[i][j] = (t - acc[i][j]) - y;
                acc[i][j] = t;
            }
        __syncthreads();  // every thread is done with this slot
        // after a wait that gave up no further copies are queued (the stage it gave up
        // on may still be in flight into this slot)
        if (tid == 0 && ok && s + NST < nst) {
            ptx::mbar_arrive_expect_tx(&b.bar[slot], kStageBytes);
            ptx::tma_load_2d(b.Xs + slot * KS * BA, &d->tmX, &b.bar[slot], a0, (s + NST) * KS);
            ptx::tma_load_2d(b.Ys + slot * KS * BR, &d->tmY, &b.bar[slot], 0, (s + NST) * KS);
        }
    }
    stage += (uint32_t)nst;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        float* dst = b.Ared + (ty * TM + i) * kMaxRank + tx * TN;
#pragma unroll
        for (int j = 0; j < TN; ++j) dst[j] = acc[i][j];
    }
    ptx::cp_async_wait_all();
    __syncthreads();
    for (int k = tid; k < kMaxRank; k += NT)
        b.Ginv[k] = (k < r && b.Gs[k * rp + k] > 0.f) ? 1.f / b.Gs[k * rp + k] : 0.f;
    __syncthreads();

    // ---- update of the tile's rows: d = F_i G, then Algorithm HALS / MU on each row
    rowupd::rows_times_gram_any(BA, r, rp, b.Fn, b.Gs, b.Dn);
    __syncthreads();
    rowupd::update_rows_any<MODE>(d->F, Na, r, rp, BA, (int64_t)a0, b.Fn, b.Ared, b.Dn, b.Gs, b.Ginv);
    __syncthreads();
    if (d->obj_part) {
        // objective identity, first term: <P_i, new F_i> over the tile's rows (FP64)
        double t = 0.0;
        for (int e = tid; e < BA * r; e += NT) {
            const int rr = e / r, k = e - rr * r;
            t += (double)b.Ared[rr * kMaxRank + k] * (double)b.Fn[rr * kMaxRank + k];
        }
        t = gblock_sum(t, b.red);
        if (tid == 0) d->obj_part[2 * tile] = t;
    }
    // ---- Gram slab of the new rows (rows past Na are zero), 4 x 4 entries per thread
    float ga[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ga[i][j] = 0.f;
#pragma unroll 4
    for (int rr = 0; rr < BA; ++rr) {
        const float4 u = *reinterpret_cast<const float4*>(b.Fn + rr * kMaxRank + ty * 4);
        const float4 v = *reinterpret_cast<const float4*>(b.Fn + rr * kMaxRank + tx * 4);
        const float uu[4] = {u.x, u.y, u.z, u.w}, vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) ga[i][j] = fmaf(uu[i], vv[j], ga[i][j]);
    }
    float* gout = d->Gout + (int64_t)tile * d->gout_stride;
    double t2 = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int l = ty * 4 + i;
        if (l < r && tx * 4 < rp) {
            *reinterpret_cast<float4*>(gout + l * rp + tx * 4) = make_float4(ga[i][0], ga[i][1], ga[i][2], ga[i][3]);
            if (d->obj_part) {
                const float4 g4 = *reinterpret_cast<const float4*>(b.Gs + l * rp + tx * 4);
                t2 += (double)ga[i][0] * g4.x + (double)ga[i][1] * g4.y + (double)ga[i][2] * g4.z +
                      (double)ga[i][3] * g4.w;
            }
        }
    }
    if (d->obj_part) {
        // second term: <G, slab>; G is the Gram matrix this half-sweep used
        t2 = gblock_sum(t2, b.red);
        if (tid == 0) d->obj_part[2 * tile + 1] = t2;
    }
    __syncthreads();  // shared buffers are free for the next tile
}

__global__ void __launch_bounds__(NT, 2)
    grouped_half_sweep_kernel(const GroupDesc* __restrict__ descs, const GroupItem* __restrict__ items, int nitems,
                              int* counter) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const GSmem L = gsmem_layout();
    Bufs b;
    b.Xs = reinterpret_cast<float*>(smem_raw + L.xs);
    b.Ys = reinterpret_cast<float*>(smem_raw + L.ys);
    b.Gs = reinterpret_cast<float*>(smem_raw + L.gs);
    b.Ginv = reinterpret_cast<float*>(smem_raw + L.ginv);
    b.Ared = reinterpret_cast<float*>(smem_raw + L.ared);
    b.Fn = reinterpret_cast<float*>(smem_raw + L.fn);
    b.Dn = reinterpret_cast<float*>(smem_raw + L.dn);
    b.red = reinterpret_cast<double*>(smem_raw + L.red);
    b.bar = reinterpret_cast<uint64_t*>(smem_raw + L.bar);
    int* slot = reinterpret_cast<int*>(smem_raw + L.slot);
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) ptx::mbar_init(&b.bar[s], 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    // everything below reads what the previous kernel wrote
    ptx::grid_dependency_wait();
    ptx::launch_dependents();
    uint32_t stage = 0;
    bool ok = true;
    for (;;) {
        if (tid == 0) *slot = atomicAdd(counter, 1);
        __syncthreads();
        const int it = *slot;
        __syncthreads();
        if (it >= nitems) break;
        const GroupItem item = items[it];
        const GroupDesc* d = descs + item.desc;
        if (d->skip && *(volatile const int*)d->skip) continue;  // converged: set before this launch
        switch (d->br * 4 + d->mode) {
            case 16 * 4 + kModeHals: group_tile<16, kModeHals>(d, item.tile, b, stage, ok); break;
            case 32 * 4 + kModeHals: group_tile<32, kModeHals>(d, item.tile, b, stage, ok); break;
            case 48 * 4 + kModeHals: group_tile<48, kModeHals>(d, item.tile, b, stage, ok); break;
            case 64 * 4 + kModeHals: group_tile<64, kModeHals>(d, item.tile, b, stage, ok); break;
            case 16 * 4 + kModeMu: group_tile<16, kModeMu>(d, item.tile, b, stage, ok); break;
            case 32 * 4 + kModeMu: group_tile<32, kModeMu>(d, item.tile, b, stage, ok); break;
            case 48 * 4 + kModeMu: group_tile<48, kModeMu>(d, item.tile, b, stage, ok); break;
            default: group_tile<64, kModeMu>(d, item.tile, b, stage, ok); break;
        }
        // a wait that gave up leaves the ring's phases unknown: report and stop
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(d->err_flag, 1);
            return;
        }
    }
}

// Chunk c of job j: float4 groups [64 c, 64 c + 64) of the slab sum, the slabs split into
// four contiguous ranges summed by four thread groups and combined in range order.
__global__ void __launch_bounds__(256) grouped_gram_kernel(const GramJob* __restrict__ jobs, int chunks) {
    __shared__ float4 part[256];
    const int job = blockIdx.x / chunks, chunk = blockIdx.x - job * chunks;
    ptx::grid_dependency_wait();
    ptx::launch_dependents();
    const GramJob J = jobs[job];
    if (J.skip && *(volatile const int*)J.skip) return;  // same value in every CTA of the job
    const int j = chunk * 64 + (threadIdx.x & 63);
    const int g = threadIdx.x >> 6;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j < J.f4) {
        const float4* src = reinterpret_cast<const float4*>(J.slabs);
        const int64_t st4 = J.stride / 4;
        const int q0 = (int)((int64_t)J.count * g / 4), q1 = (int)((int64_t)J.count * (g + 1) / 4);
#pragma unroll 8
        for (int q = q0; q < q1; ++q) s = f4add(s, src[(int64_t)q * st4 + j]);
    }
    part[threadIdx.x] = s;
    __syncthreads();
    if (g == 0 && j < J.f4) {
        float4 t = part[threadIdx.x];
        t = f4add(t, part[threadIdx.x + 64]);
        t = f4add(t, part[threadIdx.x + 128]);
        t = f4add(t, part[threadIdx.x + 192]);
        reinterpret_cast<float4*>(J.out)[j] = t;
    }
}

__global__ void grouped_converge_kernel(const ConvJob* __restrict__ jobs, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ConvJob J = jobs[i];
    if (*J.flag) return;
    double s1 = 0.0, s2 = 0.0;
    for (int t = 0; t < J.ntiles; ++t) {
        s1 += J.part[2 * t];
        s2 += J.part[2 * t + 1];
    }
    const double m = *J.mnorm;
    const double cur = sqrt(fmax(0.0, m * m - 2.0 * s1 + s2)), prev = J.state[0];
    J.state[1] = cur;
    *J.count += 1;
    if (prev > 0.0 && fabs(prev - cur) <= J.tol * cur) *J.flag = 1;
    J.state[0] = cur;
}

cudaError_t launch_pdl(const void* kern, dim3 grid, dim3 block, size_t smem, cudaStream_t st, void** args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    // may start while the previous kernel finishes; waits (griddepcontrol.wait) before
    // reading its results
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, kern, args);
}

}  // namespace

size_t grouped_smem_bytes() { return gsmem_layout().total; }

cudaError_t grouped_init() {
    return cudaFuncSetAttribute((const void*)grouped_half_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)gsmem_layout().total);
}

cudaError_t grouped_converge_launch(const ConvJob* jobs, int njobs, cudaStream_t st) {
    if (njobs <= 0) return cudaSuccess;
    grouped_converge_kernel<<<(unsigned)((njobs + 127) / 128), 128, 0, st>>>(jobs, njobs);
    return cudaGetLastError();
}

cudaError_t grouped_gram_launch(const GramJob* jobs, int njobs, int max_f4, cudaStream_t st) {
    if (njobs <= 0) return cudaSuccess;
    int chunks = (max_f4 + 63) / 64;
    if (chunks < 1) chunks = 1;
    void* args[] = {(void*)&jobs, (void*)&chunks};
    return launch_pdl((const void*)grouped_gram_kernel, dim3((unsigned)(njobs * chunks)), dim3(256), 0, st, args);
}

cudaError_t grouped_half_sweep_launch(const GroupDesc* descs, const GroupItem* items, int nitems, int* counter,
                                      int ctas, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    const int grid = std::max(1, std::min(ctas, nitems));
    void* args[] = {(void*)&descs, (void*)&items, (void*)&nitems, (void*)&counter};
    return launch_pdl((const void*)grouped_half_sweep_kernel, dim3((unsigned)grid), dim3(NT), gsmem_layout().total,
                      st, args);
}

}  // namespace nmfk
