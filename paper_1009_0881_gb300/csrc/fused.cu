// Fused half-sweep kernel: one launch does the products and the factor update
// of one half of a HALS or MU sweep (Sections 2.2, 2.3; cost in Appendix A.1).
//
//   V-step:  A = M W^T (row i of A over K = n), B = W W^T, then V's rows.
//   W-step:  C^T = M^T V (K = m),             D = V^T V,  then W's columns
//            (= rows of Wt = W^T).
// Both have the form "rows of a tall factor F from a tall product P = X^T Y
// and an r x r Gram matrix G".
//
// Decomposition: a 64-row tile of F is computed by a thread-block cluster of
// `cs` CTAs, CTA c covering the K-rows [c*kchunk, (c+1)*kchunk).  Operand
// slabs X[kk, a0:a0+64] and Y[kk, 0:BR] stream in through a TMA/mbarrier
// pipeline; each CTA accumulates its partial tile in registers (FP32 FFMA,
// 4 x BR/16 outputs per thread).  The partial tiles are summed through
// distributed shared memory in a fixed order (deterministic), each CTA
// reducing and updating 64/cs rows.  The Gram matrix G arrives as per-tile
// partial slabs written by the previous half-sweep (summed in a fixed order,
// split across the cluster and gathered back through distributed shared
// memory); after the update each cluster writes the partial Gram of its new
// rows (F_tile^T F_tile), which the next half-sweep reduces.  No split-K
// partial product ever goes to global memory.
//
// HALS update of one row (Gauss-Seidel over k, Algorithm HALS):
//   F_ik <- max(0, (P_ik - sum_{l != k} F_il G_lk) / G_kk) = max(0, F_ik + g_k / G_kk)
// with g = P_i - F_i G (F_i G computed by all threads first) updated after each
// k (g_j -= delta G_kj).  A warp owns a row, lane t its entries 4t .. 4t+3; the
// owner of a chunk of four columns runs their four steps locally and broadcasts
// the four deltas, so the dependency chain crosses lanes once per four columns.
// MU update: F_ik <- F_ik P_ik / max((F G)_ik, 1e-30).
// STORE mode writes the reduced product rows for the ANLS solver instead.
#include <cooperative_groups.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "fused.cuh"
#include "ptx.cuh"
#include "rowupdate.cuh"

namespace cg = cooperative_groups;

namespace nmfk {

namespace {

using rowupd::cluster_sum_f4;
using rowupd::f4add;

constexpr int KS = 32;    // K rows per pipeline stage
constexpr int NST = 4;    // pipeline stages
constexpr int NT = 256;   // threads
constexpr unsigned kFull = 0xffffffffu;
// float4 slots staging the Gram slabs of this CTA's slice (smaller for cs = 1, where
// the slice is the whole matrix and the layout would not fit the 227 KiB limit)
__host__ __device__ inline int stage_f4(int cs) { return cs >= 2 ? 3072 : 1920; }

struct Smem {
    // byte offsets inside the dynamic shared-memory block
    size_t xs, ys, pt, gsl, part, gst, gs, ginv, ared, fn, dn, fg, bar, total;
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// float4 groups of one r x rp Gram slab, and the share of each cluster rank
__host__ __device__ inline int slab_f4(int r, int rp) { return r * rp / 4; }
__host__ __device__ inline int slice_f4(int r, int rp, int cs) { return (slab_f4(r, rp) + cs - 1) / cs; }

// Sum of one double per thread over the CTA, in a fixed order (warp butterflies,
// then the warps in order); the result is valid in thread 0.  `red` holds NT/32 doubles.
__device__ __forceinline__ double block_sum_d(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) s += red[w];
    __syncthreads();
    return s;
}

__host__ __device__ inline Smem smem_layout(int br, int BA, int r, int rp, int cs) {
    Smem s{};
    size_t o = 0;
    const int R = BA / cs;
    const int S4 = slice_f4(r, rp, cs);
    s.xs = o;   o = align_up(o + sizeof(float) * NST * KS * BA, 128);
    s.ys = o;   o = align_up(o + sizeof(float) * NST * KS * br, 128);
    s.pt = o;   o = align_up(o + sizeof(float) * BA * br, 128);
    s.gsl = o;  o = align_up(o + sizeof(float4) * S4, 128);
    s.part = o; o = align_up(o + sizeof(float4) * NT, 128);
    s.gst = o;  o = align_up(o + sizeof(float4) * stage_f4(cs), 128);
    s.gs = o;   o = align_up(o + sizeof(float) * r * rp, 128);
    s.ginv = o; o = align_up(o + sizeof(float) * kMaxRank, 128);
    s.ared = o; o = align_up(o + sizeof(float) * R * kMaxRank, 128);
    s.fn = o;   o = align_up(o + sizeof(float) * R * kMaxRank, 128);
    s.dn = o;   o = align_up(o + sizeof(float) * R * kMaxRank, 128);
    s.fg = o;   o = align_up(o + sizeof(float4) * (size_t)cs * S4, 128);
    s.bar = o;  o = align_up(o + sizeof(uint64_t) * NST, 128);
    s.total = o;
    return s;
}

template <int BR, int BA, int MODE>
__global__ void __launch_bounds__(NT, 1)
    half_sweep_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
                      const HalfSweepParams p) {
    constexpr int TM = BA / 16;
    constexpr int TN = BR / 16;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = p.cs;
    const int crank = (int)cluster.block_rank();
    const int tile = blockIdx.x / cs;
    const int r = p.r, rp = p.rp;
    const int R = BA / cs;
    const int F4 = slab_f4(r, rp);
    const int S4 = slice_f4(r, rp, cs);
    const Smem L = smem_layout(BR, BA, r, rp, cs);
    float* Xs = reinterpret_cast<float*>(smem_raw + L.xs);
    float* Ys = reinterpret_cast<float*>(smem_raw + L.ys);
    float* Pt = reinterpret_cast<float*>(smem_raw + L.pt);
    float4* Gsl = reinterpret_cast<float4*>(smem_raw + L.gsl);
    float4* Part = reinterpret_cast<float4*>(smem_raw + L.part);
    float4* Gst = reinterpret_cast<float4*>(smem_raw + L.gst);
    float* Gs = reinterpret_cast<float*>(smem_raw + L.gs);
    float* Ginv = reinterpret_cast<float*>(smem_raw + L.ginv);
    float* Ared = reinterpret_cast<float*>(smem_raw + L.ared);
    float* Fn = reinterpret_cast<float*>(smem_raw + L.fn);
    float* Dn = reinterpret_cast<float*>(smem_raw + L.dn);
    float* Fg = reinterpret_cast<float*>(smem_raw + L.fg);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + L.bar);

    const int tid = threadIdx.x;
    const int a0 = tile * BA;
    const int64_t k0 = (int64_t)crank * p.kchunk;
    const int64_t k1 = min(p.K, k0 + (int64_t)p.kchunk);
    const int nst = k1 > k0 ? (int)((k1 - k0 + KS - 1) / KS) : 0;
    constexpr uint32_t kStageBytes = sizeof(float) * KS * (BA + BR);
    bool ok = true;

    if (tid == 0) {
        ptx::prefetch_tmap(&tmX);
        ptx::prefetch_tmap(&tmY);
        for (int s = 0; s < NST; ++s) ptx::mbar_init(&bar[s], 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    // X (M or its transpose) is constant during the sweeps: its first stages load
    // while the previous half-sweep may still be finishing (programmatic launch).
    // A launch that may be skipped issues nothing before it has read its flag.
    const bool early_x = p.skip == nullptr;
    if (early_x && tid == 0) {
        for (int s = 0; s < NST && s < nst; ++s) {
            ptx::mbar_arrive_expect_tx(&bar[s], kStageBytes);
            ptx::tma_load_2d(Xs + s * KS * BA, &tmX, &bar[s], a0, (int)(k0 + s * KS));
        }
    }
    // everything below reads what the previous kernel wrote (Y, F, Gram slabs, flag)
    ptx::grid_dependency_wait();
    ptx::launch_dependents();
    if (p.skip && *(volatile const int*)p.skip) return;  // same value in every CTA of the grid
    ptx::cluster_arrive_relaxed();                       // matched by the wait before the first push
    if (tid == 0) {
        for (int s = 0; s < NST && s < nst; ++s) {
            if (!early_x) {
                ptx::mbar_arrive_expect_tx(&bar[s], kStageBytes);
                ptx::tma_load_2d(Xs + s * KS * BA, &tmX, &bar[s], a0, (int)(k0 + s * KS));
            }
            ptx::tma_load_2d(Ys + s * KS * BR, &tmY, &bar[s], 0, (int)(k0 + s * KS));
        }
    }

    // ---- the incoming rows of F that this CTA updates, copied asynchronously
    // (rows past Na and columns past rp read as 0); waited for after the main loop
    if (MODE != kModeStore) {
        const int Q4 = rp / 4;
        for (int e = tid; e < R * (kMaxRank / 4); e += NT) {
            const int rr = e / (kMaxRank / 4), k4 = e - rr * (kMaxRank / 4);
            const int64_t row = (int64_t)a0 + crank * R + rr;
            float* dst = Fn + rr * kMaxRank + 4 * k4;
            if (k4 < Q4)
                ptx::cp_async16(dst, p.F + (row < p.Na ? row : 0) * rp + 4 * k4, row < p.Na ? 16u : 0u);
            else
                *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    // ---- Gram slice: float4 groups [crank*S4, (crank+1)*S4) of the slab sum.
    // When the slice of every slab fits the staging area it is copied
    // asynchronously now and summed after the main loop; otherwise it is summed
    // here, slabs split over NG thread groups, groups combined in a fixed order.
    const bool staged = S4 * p.gin_count <= stage_f4(cs);
    if (staged) {
        const float4* gin = reinterpret_cast<const float4*>(p.Gin);
        const int64_t gstride4 = p.gin_stride / 4;
        for (int t = tid; t < S4 * p.gin_count; t += NT) {
            const int q = t / S4, j = t - q * S4;
            const int idx = crank * S4 + j;
            ptx::cp_async16(Gst + t, gin + (int64_t)q * gstride4 + (idx < F4 ? idx : 0), idx < F4 ? 16u : 0u);
        }
    }
    ptx::cp_async_commit();
    if (!staged) {
        const float4* gin = reinterpret_cast<const float4*>(p.Gin);
        const int64_t gstride4 = p.gin_stride / 4;
        const int NG = S4 >= NT ? 1 : min(p.gin_count, NT / S4);
        for (int t = tid; t < S4 * NG; t += NT) {
            const int j = t % S4, grp = t / S4;
            const int idx = crank * S4 + j;
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
            if (idx < F4) {
                int q = grp;
#pragma unroll 4
                for (; q < p.gin_count; q += NG) s = f4add(s, gin[(int64_t)q * gstride4 + idx]);
            }
            if (NG == 1)
                Gsl[j] = s;
            else
                Part[t] = s;
        }
        if (NG > 1) {
            __syncthreads();
            for (int j = tid; j < S4; j += NT) {
                float4 s = Part[j];
                for (int grp = 1; grp < NG; ++grp) s = f4add(s, Part[grp * S4 + j]);
                Gsl[j] = s;
            }
        }
    }

    // ---- partial product tile over this CTA's K rows
    const int tx = tid & 15, ty = tid >> 4;
    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
    for (int s = 0; s < nst; ++s) {
        const int slot = s % NST;
        if (!ptx::mbar_wait(&bar[slot], (uint32_t)((s / NST) & 1))) ok = false;
        const float* xs = Xs + slot * KS * BA;
        const float* ys = Ys + slot * KS * BR;
#pragma unroll 8
        for (int kk = 0; kk < KS; ++kk) {
            float av[TM];
            if (TM == 4) {
                const float4 a4 = *reinterpret_cast<const float4*>(xs + kk * BA + ty * TM);
                av[0] = a4.x;
                av[1 % TM] = a4.y;
                av[2 % TM] = a4.z;
                av[3 % TM] = a4.w;
            } else if (TM == 2) {
                const float2 a2 = *reinterpret_cast<const float2*>(xs + kk * BA + ty * TM);
                av[0] = a2.x;
                av[1 % TM] = a2.y;
            } else {
                av[0] = xs[kk * BA + ty];
            }
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
                for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();  // every thread is done with this slot
        // after a wait that gave up, the issuing thread queues no further copies (the
        // stage it gave up on may still be in flight into this slot)
        if (tid == 0 && ok && s + NST < nst) {
            ptx::mbar_arrive_expect_tx(&bar[slot], kStageBytes);
            ptx::tma_load_2d(Xs + slot * KS * BA, &tmX, &bar[slot], a0, (int)(k0 + (s + NST) * KS));
            ptx::tma_load_2d(Ys + slot * KS * BR, &tmY, &bar[slot], 0, (int)(k0 + (s + NST) * KS));
        }
    }
    ptx::cluster_wait();  // every CTA of the cluster has started: its shared memory may be written
    // push the partial tile rows to the rank that reduces them: row a of the tile
    // belongs to rank a / R, which receives the cs partials at Pt[(c R + a % R) BR + col]
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int a = ty * TM + i;
        const int owner = a / R;
        float* dst = cluster.map_shared_rank(Pt, owner) + (crank * R + (a - owner * R)) * BR + tx * TN;
        if (TN == 4) {
            *reinterpret_cast<float4*>(dst) = make_float4(acc[i][0], acc[i][1 % TN], acc[i][2 % TN], acc[i][3 % TN]);
        } else {
#pragma unroll
            for (int j = 0; j < TN; ++j) dst[j] = acc[i][j];
        }
    }
    if (!ok) atomicExch(p.err_flag, 1);
    ptx::cp_async_wait_all();
    __syncthreads();
    if (staged) {
        // slab sum of the staged slice, slabs in index order
        for (int j = tid; j < S4; j += NT) {
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int q = 0; q < p.gin_count; ++q) s = f4add(s, Gst[q * S4 + j]);
            Gsl[j] = s;
        }
        __syncthreads();
    }
    // push this rank's Gram slice into the full Gram matrix of every rank
    {
        const int n4 = max(0, min(S4, F4 - crank * S4));
        for (int t = tid; t < n4 * cs; t += NT) {
            const int c = t / n4, j = t - c * n4;
            reinterpret_cast<float4*>(cluster.map_shared_rank(Gs, c))[crank * S4 + j] = Gsl[j];
        }
    }

    cluster.sync();  // #1: partial tiles and Gram slices delivered to their ranks

    // ---- this CTA's R rows of the tile: sum of the cs partial tiles in rank order
    const int row0 = crank * R;
    const int Q4 = rp / 4;
    for (int e = tid; e < R * Q4; e += NT) {
        const int rr = e / Q4, k4 = e - rr * Q4;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int c = 0; c < cs; ++c) s = f4add(s, *reinterpret_cast<const float4*>(Pt + (c * R + rr) * BR + 4 * k4));
        *reinterpret_cast<float4*>(Ared + rr * kMaxRank + 4 * k4) = s;
    }
    __syncthreads();
    for (int k = tid; k < kMaxRank; k += NT) Ginv[k] = (k < r && Gs[k * rp + k] > 0.f) ? 1.f / Gs[k * rp + k] : 0.f;
    __syncthreads();

    if (MODE == kModeStore) {
        for (int e = tid; e < R * rp; e += NT) {
            const int rr = e / rp, k = e - rr * rp;
            const int64_t row = (int64_t)a0 + row0 + rr;
            if (row < p.Na) p.Pout[row * rp + k] = Ared[rr * kMaxRank + k];
        }
    } else {
        // d = F_i G for the incoming rows
        rowupd::rows_times_gram_any(R, r, rp, Fn, Gs, Dn);
        __syncthreads();
        rowupd::update_rows_any<MODE>(p.F, p.Na, r, rp, R, (int64_t)a0 + row0, Fn, Ared, Dn, Gs, Ginv);
        __syncthreads();
        if (p.obj_part) {
            // objective identity, first term: <P_i, new F_i> over this CTA's rows (FP64)
            double t = 0.0;
            for (int e = tid; e < R * r; e += NT) {
                const int rr = e / r, k = e - rr * r;
                t += (double)Ared[rr * kMaxRank + k] * (double)Fn[rr * kMaxRank + k];
            }
            t = block_sum_d(t, reinterpret_cast<double*>(Part));
            if (tid == 0) p.obj_part[2 * blockIdx.x] = t;
        }
        // partial Gram of this CTA's new rows, 4 x 4 outputs per thread (rows past Na are zero)
        {
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
            // push to the rank that owns this slice of the slab (Fg there holds cs partials)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int l = ty * 4 + i;
                if (l < r && tx * 4 < rp) {
                    const int idx = (l * rp + tx * 4) / 4;
                    const int owner = idx / S4;
                    reinterpret_cast<float4*>(cluster.map_shared_rank(Fg, owner))[crank * S4 + idx - owner * S4] =
                        make_float4(ga[i][0], ga[i][1], ga[i][2], ga[i][3]);
                }
            }
        }

        cluster.sync();  // #3: every rank's slab partials delivered

        // this rank's slice of the tile's Gram slab: sum of the cs partials in rank order.
        // Nothing reads another rank's shared memory after #3, so no closing barrier.
        float4* gout = reinterpret_cast<float4*>(p.Gout + (int64_t)tile * p.gout_stride);
        const int n4 = max(0, min(S4, F4 - crank * S4));
        double t2 = 0.0;
        for (int j = tid; j < n4; j += NT) {
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int c = 0; c < cs; ++c) s = f4add(s, reinterpret_cast<const float4*>(Fg)[c * S4 + j]);
            gout[crank * S4 + j] = s;
            if (p.obj_part) {
                const float4 g4 = reinterpret_cast<const float4*>(Gs)[crank * S4 + j];
                t2 += (double)s.x * g4.x + (double)s.y * g4.y + (double)s.z * g4.z + (double)s.w * g4.w;
            }
        }
        if (p.obj_part) {
            // second term: <G, slab slice>; G here is the Gram matrix this half-sweep used
            t2 = block_sum_d(t2, reinterpret_cast<double*>(Part));
            if (tid == 0) p.obj_part[2 * blockIdx.x + 1] = t2;
        }
    }
}

// Partial Gram slabs of a tall factor: out[t] = F[bt t : bt t + bt]^T F[bt t : bt t + bt], bt <= 64.
__global__ void __launch_bounds__(256) gram_tiles_kernel(const float* __restrict__ F, int64_t rows, int r, int rp,
                                                         int bt, float* __restrict__ out, int64_t out_stride,
                                                         const int* skip) {
    __shared__ float Fs[64][kMaxRank + 1];
    if (skip && *(volatile const int*)skip) return;  // same value in every CTA
    const int64_t r0 = (int64_t)blockIdx.x * bt;
    for (int e = threadIdx.x; e < bt * rp; e += blockDim.x) {
        const int rr = e / rp, k = e - rr * rp;
        Fs[rr][k] = (r0 + rr < rows) ? F[(r0 + rr) * rp + k] : 0.f;
    }
    __syncthreads();
    float* o = out + (int64_t)blockIdx.x * out_stride;
    for (int idx = threadIdx.x; idx < r * rp; idx += blockDim.x) {
        const int l = idx / rp, k = idx - l * rp;
        float s = 0.f;
        for (int rr = 0; rr < bt; ++rr) s = fmaf(Fs[rr][l], Fs[rr][k], s);
        o[(int64_t)l * rp + k] = s;
    }
}

template <int BR, int BA, int MODE>
cudaError_t launch_t(const HalfSweepLaunch& hl, cudaStream_t st) {
    const Smem L = smem_layout(BR, BA, hl.p.r, hl.p.rp, hl.p.cs);
    auto kern = half_sweep_kernel<BR, BA, MODE>;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(hl.tiles * hl.p.cs));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = L.total;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = hl.p.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    // may start once the previous kernel has started its epilogue; the kernel
    // waits (griddepcontrol.wait) before touching that kernel's results
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kern, hl.tmX, hl.tmY, hl.p);
}

template <int BR, int BA>
cudaError_t set_attrs_br() {
    size_t maxs = 0;
    for (int cs = 1; cs <= 16; cs *= 2) maxs = std::max(maxs, smem_layout(BR, BA, kMaxRank, kMaxRank, cs).total);
    if (maxs > 232448) return cudaErrorInvalidConfiguration;  // 227 KiB opt-in limit per block
    const void* ks[3] = {(const void*)half_sweep_kernel<BR, BA, kModeHals>,
                         (const void*)half_sweep_kernel<BR, BA, kModeMu>,
                         (const void*)half_sweep_kernel<BR, BA, kModeStore>};
    for (const void* k : ks) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)maxs);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int BA>
const void* hals_kernel_ptr(int br) {
    switch (br) {
        case 16: return (const void*)half_sweep_kernel<16, BA, kModeHals>;
        case 32: return (const void*)half_sweep_kernel<32, BA, kModeHals>;
        case 48: return (const void*)half_sweep_kernel<48, BA, kModeHals>;
        default: return (const void*)half_sweep_kernel<64, BA, kModeHals>;
    }
}

}  // namespace

size_t half_sweep_smem_bytes(int br, int ba, int r, int cs) {
    return smem_layout(br, ba, r, (int)round_up(r, 4), cs).total;
}

cudaError_t half_sweep_init() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = set_attrs_br<16, 64>();
    if (e == cudaSuccess) e = set_attrs_br<32, 64>();
    if (e == cudaSuccess) e = set_attrs_br<48, 64>();
    if (e == cudaSuccess) e = set_attrs_br<64, 64>();
    if (e == cudaSuccess) e = set_attrs_br<16, 32>();
    if (e == cudaSuccess) e = set_attrs_br<32, 32>();
    if (e == cudaSuccess) e = set_attrs_br<48, 32>();
    if (e == cudaSuccess) e = set_attrs_br<64, 32>();
    if (e == cudaSuccess) e = set_attrs_br<16, 16>();
    if (e == cudaSuccess) e = set_attrs_br<32, 16>();
    if (e == cudaSuccess) e = set_attrs_br<48, 16>();
    if (e == cudaSuccess) e = set_attrs_br<64, 16>();
    return e;
}

int half_sweep_active_clusters(int br, int ba, int r, int cs) {
    // how many clusters of `cs` CTAs the device can hold at once with this kernel's shared memory
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem_layout(br, ba, r, (int)round_up(r, 4), cs).total;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    const void* k = ba == 16 ? hals_kernel_ptr<16>(br) : (ba == 32 ? hals_kernel_ptr<32>(br) : hals_kernel_ptr<64>(br));
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) == cudaSuccess) return n;
    cudaGetLastError();
    return 0;
}

cudaError_t half_sweep_launch(const HalfSweepLaunch& hl, cudaStream_t st) {
#define NMF_HS_CASE(BRV, BAV)                                                      \
    case BRV:                                                                      \
        if (hl.mode == kModeHals) return launch_t<BRV, BAV, kModeHals>(hl, st);    \
        if (hl.mode == kModeMu) return launch_t<BRV, BAV, kModeMu>(hl, st);        \
        return launch_t<BRV, BAV, kModeStore>(hl, st);
    if (hl.ba == 16) {
        switch (hl.br) {
            NMF_HS_CASE(16, 16)
            NMF_HS_CASE(32, 16)
            NMF_HS_CASE(48, 16)
            NMF_HS_CASE(64, 16)
            default: return cudaErrorInvalidValue;
        }
    }
    if (hl.ba == 32) {
        switch (hl.br) {
            NMF_HS_CASE(16, 32)
            NMF_HS_CASE(32, 32)
            NMF_HS_CASE(48, 32)
            NMF_HS_CASE(64, 32)
            default: return cudaErrorInvalidValue;
        }
    }
    if (hl.ba != 64) return cudaErrorInvalidValue;
    switch (hl.br) {
        NMF_HS_CASE(16, 64)
        NMF_HS_CASE(32, 64)
        NMF_HS_CASE(48, 64)
        NMF_HS_CASE(64, 64)
        default: return cudaErrorInvalidValue;
    }
#undef NMF_HS_CASE
}

cudaError_t gram_tiles_launch(const float* F, int64_t rows, int r, int rp, int tile_rows, float* out,
                              int64_t out_stride, cudaStream_t st, const int* skip) {
    if (tile_rows < 1 || tile_rows > 64) return cudaErrorInvalidValue;
    const int64_t tiles = (rows + tile_rows - 1) / tile_rows;
    if (tiles <= 0) return cudaSuccess;
    gram_tiles_kernel<<<(unsigned)tiles, 256, 0, st>>>(F, rows, r, rp, tile_rows, out, out_stride, skip);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// TMA descriptors
// ---------------------------------------------------------------------------
namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
}

cudaError_t tma_init() {
    if (g_encode) return cudaSuccess;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return cudaSuccess;
}

cudaError_t make_tmap_2d(CUtensorMap* map, CUtensorMapDataType type, const void* base, uint64_t width,
                         uint64_t height, uint64_t ld_bytes, uint32_t box_w, uint32_t box_h,
                         CUtensorMapSwizzle swizzle) {
    if (!g_encode) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {width, height};
    cuuint64_t strides[1] = {ld_bytes};
    cuuint32_t box[2] = {box_w, box_h};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, type, 2, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_tmap_f32(CUtensorMap* map, const float* base, uint64_t width, uint64_t height, uint64_t ld,
                          uint32_t box_w, uint32_t box_h) {
    return make_tmap_2d(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, base, width, height, ld * sizeof(float), box_w, box_h,
                        CU_TENSOR_MAP_SWIZZLE_NONE);
}

int half_sweep_stage_rows() { return KS; }

}  // namespace nmfk
