// Row updates shared by the fused half-sweep kernel and the standalone update
// kernel of the BF16 path: the HALS Gauss-Seidel step (Algorithm HALS) and the
// MU step (Algorithm MU) on rows of a tall factor, plus two small helpers.
#pragma once

#include <cuda_runtime.h>

#include "nmf_internal.cuh"

namespace nmfk {
namespace rowupd {

constexpr int NT = 256;  // threads per CTA of the kernels that use these helpers
constexpr unsigned kFull = 0xffffffffu;
enum { kModeHals = 0, kModeMu = 1, kModeStore = 2 };

__device__ __forceinline__ float4 f4add(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// dst(i, sum_c src(c, i)) for i < n4, c < cs, in a fixed order: the ranks are
// split into NG contiguous groups summed by different threads (so all loads
// are in flight at once), then the group sums are added in group order.
// `scratch` holds NT float4.  Ends with every thread past a __syncthreads if NG > 1.
template <typename Src, typename Dst>
__device__ __forceinline__ void cluster_sum_f4(int n4, int cs, Src src, Dst dst, float4* scratch) {
    const int NG = (n4 <= 0 || n4 >= NT) ? 1 : min(cs, NT / n4);
    const int per = (cs + NG - 1) / NG;
    for (int t = threadIdx.x; t < n4 * NG; t += NT) {
        const int i = t % n4, grp = t / n4;
        const int c0 = grp * per, c1 = min(cs, c0 + per);
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
        for (int c = c0; c < c1; ++c) s = f4add(s, src(c, i));
        if (NG == 1)
            dst(i, s);
        else
            scratch[t] = s;
    }
    if (NG > 1) {
        __syncthreads();
        for (int i = threadIdx.x; i < n4; i += NT) {
            float4 s = scratch[i];
            for (int grp = 1; grp < NG; ++grp) s = f4add(s, scratch[grp * n4 + i]);
            dst(i, s);
        }
    }
}

// Dn = Fn G for R rows (Fn, Dn: rows of kMaxRank floats; G: r x rp, row-major),
// each output the sum over l = 0 .. r-1 in increasing order.  Thread (ty, tx) of
// a 16 x 16 arrangement computes columns 4tx .. 4tx+3 of rows ty, ty+16, ...;
// columns past rp are written as zero.
template <int RPT>
__device__ __forceinline__ void rows_times_gram(int R, int r, int rp, const float* Fn, const float* Gs, float* Dn) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int c0 = 4 * tx;
    for (int rb = 0; rb < R; rb += 16 * RPT) {
        float acc[RPT][4];
#pragma unroll
        for (int i = 0; i < RPT; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        if (c0 < rp) {
#pragma unroll 4
            for (int l = 0; l < r; ++l) {
                const float4 gv = *reinterpret_cast<const float4*>(Gs + l * rp + c0);
#pragma unroll
                for (int i = 0; i < RPT; ++i) {
                    const int rr = rb + ty + 16 * i;
                    const float fv = rr < R ? Fn[rr * kMaxRank + l] : 0.f;
                    acc[i][0] = fmaf(fv, gv.x, acc[i][0]);
                    acc[i][1] = fmaf(fv, gv.y, acc[i][1]);
                    acc[i][2] = fmaf(fv, gv.z, acc[i][2]);
                    acc[i][3] = fmaf(fv, gv.w, acc[i][3]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            const int rr = rb + ty + 16 * i;
            if (rr < R)
                *reinterpret_cast<float4*>(Dn + rr * kMaxRank + c0) =
                    make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        }
    }
}

// Dn = Fn G for up to 16 rows at a time with the thread's row of Fn held in
// registers (one shared-memory load of G per column group and l, no dependent
// load of Fn inside the l loop); thread (ty, tx) computes columns 4tx .. 4tx+3 of
// row ty.  Same summation order as rows_times_gram.
__device__ __forceinline__ void rows_times_gram_reg(int R, int r, int rp, const float* Fn, const float* Gs, float* Dn) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int c0 = 4 * tx;
    for (int rb = 0; rb < R; rb += 16) {
        const int rr = rb + ty;
        float f[kMaxRank];
#pragma unroll
        for (int q = 0; q < kMaxRank / 4; ++q) {
            const float4 v = rr < R ? *reinterpret_cast<const float4*>(Fn + rr * kMaxRank + 4 * q)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
            f[4 * q] = v.x;
            f[4 * q + 1] = v.y;
            f[4 * q + 2] = v.z;
            f[4 * q + 3] = v.w;
        }
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        if (c0 < rp) {
#pragma unroll
            for (int l = 0; l < kMaxRank; ++l) {
                if (l < r) {
                    const float4 gv = *reinterpret_cast<const float4*>(Gs + l * rp + c0);
                    a0 = fmaf(f[l], gv.x, a0);
                    a1 = fmaf(f[l], gv.y, a1);
                    a2 = fmaf(f[l], gv.z, a2);
                    a3 = fmaf(f[l], gv.w, a3);
                }
            }
        }
        if (rr < R) *reinterpret_cast<float4*>(Dn + rr * kMaxRank + c0) = make_float4(a0, a1, a2, a3);
    }
}

// The same product for few rows: S consecutive lanes share one group of four
// outputs, lane s summing l = s, s + S, ..., and the S partial sums are combined
// by butterfly shuffles.  Requires R * (rp/4) * S <= NT.
template <int S>
__device__ __forceinline__ void rows_times_gram_split(int R, int r, int rp, const float* Fn, const float* Gs, float* Dn) {
    const int nq = rp / 4;
    const int t = threadIdx.x;
    const int o = t / S, s = t % S;
    const bool act = o < R * nq;  // uniform over each group of S lanes
    const int rr = act ? o / nq : 0, q = act ? o % nq : 0;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    if (act) {
#pragma unroll 4
        for (int l = s; l < r; l += S) {
            const float4 gv = *reinterpret_cast<const float4*>(Gs + l * rp + 4 * q);
            const float fv = Fn[rr * kMaxRank + l];
            a0 = fmaf(fv, gv.x, a0);
            a1 = fmaf(fv, gv.y, a1);
            a2 = fmaf(fv, gv.z, a2);
            a3 = fmaf(fv, gv.w, a3);
        }
    }
#pragma unroll
    for (int off = S / 2; off > 0; off >>= 1) {
        a0 += __shfl_xor_sync(kFull, a0, off);
        a1 += __shfl_xor_sync(kFull, a1, off);
        a2 += __shfl_xor_sync(kFull, a2, off);
        a3 += __shfl_xor_sync(kFull, a3, off);
    }
    if (act && s == 0) *reinterpret_cast<float4*>(Dn + rr * kMaxRank + 4 * q) = make_float4(a0, a1, a2, a3);
}

// Dn = Fn G for R rows, choosing the split for the number of output groups.
__device__ __forceinline__ void rows_times_gram_any(int R, int r, int rp, const float* Fn, const float* Gs, float* Dn) {
    const int groups = R * (rp / 4);
    if (groups * 8 <= NT)
        rows_times_gram_split<8>(R, r, rp, Fn, Gs, Dn);
    else if (groups * 4 <= NT)
        rows_times_gram_split<4>(R, r, rp, Fn, Gs, Dn);
    else if (groups * 2 <= NT)
        rows_times_gram_split<2>(R, r, rp, Fn, Gs, Dn);
    else if (R <= 16)
        rows_times_gram_reg(R, r, rp, Fn, Gs, Dn);
    else if (R <= 32)
        rows_times_gram<2>(R, r, rp, Fn, Gs, Dn);
    else
        rows_times_gram<4>(R, r, rp, Fn, Gs, Dn);
}

// Update of R rows of F (HALS or MU), RPW rows interleaved per warp.
// Lane t owns the four consecutive entries k = 4t .. 4t+3 of each of its rows
// (lanes 16..31 own nothing for r <= 64).  Inputs in shared memory (rows of
// kMaxRank floats): Fn = incoming rows, Ared = product rows P_i, Dn = F_i G.
// HALS walks the columns in the order k = 0, 1, ..., r-1 of Algorithm HALS:
// the owner of a chunk runs its four steps on private copies (each step's
// delta also corrects the owner's later entries of the chunk), broadcasts the
// four deltas, and every lane applies them, in order, to its own entries.
template <int RPW, int MODE>
__device__ __forceinline__ void update_rows(float* __restrict__ F, int Na, int r, int rp, int R, int64_t rowbase,
                                            float* Fn, const float* Ared, const float* Dn, const float* Gs,
                                            const float* Ginv) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c0 = 4 * lane;
    const bool has = c0 < r;
    for (int base = warp * RPW; base < R; base += (NT / 32) * RPW) {
        float f[RPW][4], g[RPW][4];
        bool act[RPW];
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int rr = base + q;
            act[q] = rr < R && rowbase + rr < Na;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = c0 + e;
                const bool ok = act[q] && k < r;
                f[q][e] = ok ? Fn[rr * kMaxRank + k] : 0.f;
                const float pv = ok ? Ared[rr * kMaxRank + k] : 0.f;
                const float dv = ok ? Dn[rr * kMaxRank + k] : 0.f;
                g[q][e] = MODE == kModeHals ? pv - dv : pv;
                if (MODE == kModeMu) g[q][e] = ok ? f[q][e] * pv / fmaxf(dv, 1e-30f) : 0.f;
            }
        }
        if (MODE == kModeHals) {
            const int nchunks = (r + 3) / 4;
            for (int t = 0; t < nchunks; ++t) {
                // this lane's columns of the Gram rows 4t .. 4t+3
                float Gk[4][4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int kk = 4 * t + e;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (kk < r && c0 < rp) v = *reinterpret_cast<const float4*>(Gs + kk * rp + c0);
                    Gk[e][0] = v.x;
                    Gk[e][1] = v.y;
                    Gk[e][2] = v.z;
                    Gk[e][3] = v.w;
                }
                const float4 gi4 = *reinterpret_cast<const float4*>(Ginv + 4 * t);
                const float gi[4] = {gi4.x, gi4.y, gi4.z, gi4.w};
                const bool own = lane == t;
#pragma unroll
                for (int q = 0; q < RPW; ++q) {
                    // the owner's four sequential steps (computed by every lane on its own
                    // copies; only lane t's results are used)
                    float gt[4] = {g[q][0], g[q][1], g[q][2], g[q][3]};
                    float ft[4] = {f[q][0], f[q][1], f[q][2], f[q][3]};
                    float dl[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float nv = fmaxf(0.f, fmaf(gt[e], gi[e], ft[e]));
                        dl[e] = nv - ft[e];
                        ft[e] = nv;
#pragma unroll
                        for (int e2 = e + 1; e2 < 4; ++e2) gt[e2] = fmaf(-dl[e], Gk[e][e2], gt[e2]);
                    }
                    float d[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) d[e] = __shfl_sync(kFull, dl[e], t);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        f[q][j] = own ? ft[j] : f[q][j];
                        float gj = g[q][j];
#pragma unroll
                        for (int e = 0; e < 4; ++e) gj = fmaf(-d[e], Gk[e][j], gj);
                        g[q][j] = gj;
                    }
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < RPW; ++q)
#pragma unroll
                for (int e = 0; e < 4; ++e) f[q][e] = g[q][e];
        }
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int rr = base + q;
            if (rr < R && c0 < kMaxRank)
                *reinterpret_cast<float4*>(Fn + rr * kMaxRank + c0) =
                    act[q] ? make_float4(f[q][0], f[q][1], f[q][2], f[q][3]) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (act[q] && has) {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (c0 + e < r) F[(rowbase + rr) * rp + c0 + e] = f[q][e];
            }
        }
    }
}


// Update of R rows with a half-warp per row (two rows per warp at a time): the
// same column walk as update_rows, lane s of the half owning entries 4s .. 4s+3.
template <int MODE>
__device__ __forceinline__ void update_rows_half(float* __restrict__ F, int Na, int r, int rp, int R, int64_t rowbase,
                                                 float* Fn, const float* Ared, const float* Dn, const float* Gs,
                                                 const float* Ginv) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sl = lane & 15, half = lane >> 4;
    const int c0 = 4 * sl;
    const bool has = c0 < r;
    for (int base = warp * 2; base < R; base += (NT / 32) * 2) {
        const int rr = base + half;
        const bool act = rr < R && rowbase + rr < Na;
        float f[4], g[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = c0 + e;
            const bool ok = act && k < r;
            f[e] = ok ? Fn[rr * kMaxRank + k] : 0.f;
            const float pv = ok ? Ared[rr * kMaxRank + k] : 0.f;
            const float dv = ok ? Dn[rr * kMaxRank + k] : 0.f;
            g[e] = MODE == kModeHals ? pv - dv : (ok ? f[e] * pv / fmaxf(dv, 1e-30f) : 0.f);
        }
        if (MODE == kModeHals) {
            const int nchunks = (r + 3) / 4;
            for (int t = 0; t < nchunks; ++t) {
                float Gk[4][4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int kk = 4 * t + e;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (kk < r && c0 < rp) v = *reinterpret_cast<const float4*>(Gs + kk * rp + c0);
                    Gk[e][0] = v.x;
                    Gk[e][1] = v.y;
                    Gk[e][2] = v.z;
                    Gk[e][3] = v.w;
                }
                const float4 gi4 = *reinterpret_cast<const float4*>(Ginv + 4 * t);
                const float gi[4] = {gi4.x, gi4.y, gi4.z, gi4.w};
                float gt[4] = {g[0], g[1], g[2], g[3]};
                float ft[4] = {f[0], f[1], f[2], f[3]};
                float dl[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float nv = fmaxf(0.f, fmaf(gt[e], gi[e], ft[e]));
                    dl[e] = nv - ft[e];
                    ft[e] = nv;
#pragma unroll
                    for (int e2 = e + 1; e2 < 4; ++e2) gt[e2] = fmaf(-dl[e], Gk[e][e2], gt[e2]);
                }
                float d[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) d[e] = __shfl_sync(kFull, dl[e], t, 16);
                const bool own = sl == t;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    f[j] = own ? ft[j] : f[j];
                    float gj = g[j];
#pragma unroll
                    for (int e = 0; e < 4; ++e) gj = fmaf(-d[e], Gk[e][j], gj);
                    g[j] = gj;
                }
            }
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) f[e] = g[e];
        }
        if (rr < R)
            *reinterpret_cast<float4*>(Fn + rr * kMaxRank + c0) =
                act ? make_float4(f[0], f[1], f[2], f[3]) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (act && has) {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (c0 + e < r) F[(rowbase + rr) * rp + c0 + e] = f[e];
        }
    }
}

// Dispatch of update_rows on the number of rows per warp: rows are interleaved
// so that the eight warps of the CTA share the R rows.
template <int MODE>
__device__ __forceinline__ void update_rows_any(float* __restrict__ F, int Na, int r, int rp, int R, int64_t rowbase,
                                                float* Fn, const float* Ared, const float* Dn, const float* Gs,
                                                const float* Ginv) {
    if (R > 8 && R <= 16) {
        update_rows_half<MODE>(F, Na, r, rp, R, rowbase, Fn, Ared, Dn, Gs, Ginv);
        return;
    }
    const int rpw = R <= 8 ? 1 : (R <= 16 ? 2 : (R <= 32 ? 4 : 8));
    switch (rpw) {
        case 1: update_rows<1, MODE>(F, Na, r, rp, R, rowbase, Fn, Ared, Dn, Gs, Ginv); break;
        case 2: update_rows<2, MODE>(F, Na, r, rp, R, rowbase, Fn, Ared, Dn, Gs, Ginv); break;
        case 4: update_rows<4, MODE>(F, Na, r, rp, R, rowbase, Fn, Ared, Dn, Gs, Ginv); break;
        default: update_rows<8, MODE>(F, Na, r, rp, R, rowbase, Fn, Ared, Dn, Gs, Ginv); break;
    }
}

}  // namespace rowupd
}  // namespace nmfk
