// Coarse-level sweep runs of the FP32 form (HALS, Algorithm 3; MU, Algorithm 2).
//
// On the coarse levels of the hierarchy (Section 4.2) M_l has few rows, and a
// sweep costs little arithmetic (Appendix A.1: 4 m_l n r + 4 (m_l + n) r^2
// flops); launched as two half-sweep kernels it is bound by fixed costs
// (launch, pipeline ramp-up, cluster synchronisation, Gram slabs through
// memory).  Here one cooperative launch runs all sweeps of a run and keeps the
// level on chip: CTA c holds the columns of M_l and the rows of W^T of its
// 16-column chunks (chunks c, c + G, c + 2G, ... of G CTAs), and every CTA holds
// all of V_l.  One sweep is
//   1. per chunk q: P_q = M_l[:, q] W^T[q, :] (m_l x r) and
//      B_q = W^T[q, :]^T W^T[q, :] (r x r), written to a global slot;
//   2. grid barrier; CTA c sums its share of the slot entries over the chunks
//      (chunks in groups of 8 summed in order, then the groups in order, so the
//      result does not depend on G);
//   3. grid barrier; every CTA reads A = M_l W^T and B = W W^T, updates all rows
//      of V_l (the same arithmetic in every CTA, so the copies agree bit for bit)
//      and forms D = V^T V;
//   4. the W-step on the CTA's own rows of W^T: C = M_l^T V for its columns,
//      then the row update with D.
// After the last sweep B = W W^T of the final W is reduced into Bout, the Gram
// input of the next V-step, and V_l and W^T are written back.
//
// Row updates: four threads per row, thread q of the four holding entries
// 16q .. 16q+15; HALS walks k = 0 .. r-1 in order (the Gauss-Seidel order of
// Algorithm 3) on g = P_i - F_i G, each step broadcasting its delta to the
// other three threads; MU applies F .* P ./ max(F G, 1e-30).
#include <cuda_runtime.h>

#include <algorithm>

#include "coarse.cuh"

namespace nmfk {
namespace {

constexpr int CT = 384;                      // threads per CTA
constexpr int CW = 16;                       // columns of M_l per chunk
constexpr int RS = 68;                       // row stride (floats) of rank-wide row buffers
constexpr int QG = 8;                        // chunks per group of the fixed-order reduction
constexpr int kMaxRows = CT / 4;             // rows a row update covers in one pass (W^T rows per CTA)
constexpr size_t kMaxSmem = 232448;          // 227 KiB opt-in limit per block
constexpr int kMaxVRows = 32;                // coarse runs only where V_l has at most this many rows
// Gram matrices in shared memory: 64 rows of four 16-column blocks, block b of a row
// at offset GB * b (GB = 20 floats), so that the four 16-byte reads of one quarter-warp
// (two rows x four blocks, same offset in each block) fall in distinct bank groups.
constexpr int GB = 20;
constexpr int GS = 80;                       // floats per Gram row
__host__ __device__ inline int gidx(int l, int c) { return l * GS + (c >> 4) * GB + (c & 15); }

struct CLayout {
    size_t ms, ws, vs, ps, bs, ds, binv, dinv, scr, flag, total;
    int JS, MS;
};

__host__ __device__ inline size_t take_floats(size_t& o, size_t floats) {
    const size_t at = o;
    o += ((floats + 3) / 4) * 4 * sizeof(float);
    return at;
}

__host__ __device__ inline CLayout clayout(int m, int cpc, int r) {
    CLayout L;
    L.JS = CW * cpc;
    L.MS = L.JS + 4;
    size_t scr = 4 * CT;
    if (scr < (size_t)4 * CW * 64) scr = (size_t)4 * CW * 64;
    size_t o = 0;
    L.ms = take_floats(o, (size_t)m * L.MS);
    L.ws = take_floats(o, (size_t)L.JS * RS);
    L.vs = take_floats(o, (size_t)m * RS);
    L.ps = take_floats(o, (size_t)(m > L.JS ? m : L.JS) * RS);
    L.bs = take_floats(o, 64 * GS);
    L.ds = take_floats(o, 64 * GS);
    L.binv = take_floats(o, 64);
    L.dinv = take_floats(o, 64);
    L.scr = take_floats(o, scr);
    L.flag = take_floats(o, 4);
    L.total = o;
    return L;
}

__device__ __forceinline__ float4 f4add(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_gpu_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier number `nb` (1, 2, ...): every CTA adds one to the counter and
// waits until it reaches nb * gridDim.x.  The wait is bounded; on expiry (or when
// another CTA has already given up) it raises err_flag and returns false in every
// thread of the CTA, which then leaves the kernel.
__device__ bool grid_sync(unsigned* bar, int* err_flag, unsigned nb, int* flag, uint32_t spins) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = nb * gridDim.x;
        red_release_gpu_add(bar, 1u);  // release: the CTA's writes before the __syncthreads above
        int ok = 1;
        for (uint32_t i = 0;; ++i) {
            if ((int)(ld_acquire_gpu(bar) - target) >= 0) break;
            if (i >= spins || *(volatile int*)err_flag) {
                atomicExch(err_flag, 1);
                ok = 0;
                break;
            }
        }
        *flag = ok;
    }
    __syncthreads();
    return *flag != 0;
}

// Step 1: partial products of this CTA's chunks.  Rows 0 .. m-1 of a slot hold
// P_q (skipped when !with_p), rows m .. m+r-1 hold B_q; each entry a sum over the
// 16 columns of the chunk in increasing order.
__device__ void chunk_partials(const CoarseParams& q, const float* Ms, int MS, const float* Ws, bool with_p) {
    const int nq4 = q.rp / 4;
    const int row0 = with_p ? 0 : q.m;
    const int T = (q.m + q.r - row0) * nq4;
    for (int lq = 0; lq < q.cpc; ++lq) {
        const int chunk = blockIdx.x + lq * gridDim.x;
        if (chunk >= q.nchunk) break;
        float* slot = q.part + (int64_t)chunk * q.part_stride;
        const float* wq = Ws + lq * CW * RS;
        for (int o = threadIdx.x; o < T; o += CT) {
            const int row = row0 + o / nq4, k4 = o % nq4;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            if (row < q.m) {
                const float* mrow = Ms + row * MS + lq * CW;
#pragma unroll
                for (int jj = 0; jj < CW; ++jj) {
                    const float a = mrow[jj];
                    const float4 w = *reinterpret_cast<const float4*>(wq + jj * RS + 4 * k4);
                    acc.x = fmaf(a, w.x, acc.x);
                    acc.y = fmaf(a, w.y, acc.y);
                    acc.z = fmaf(a, w.z, acc.z);
                    acc.w = fmaf(a, w.w, acc.w);
                }
            } else {
                const int l = row - q.m;
#pragma unroll
                for (int jj = 0; jj < CW; ++jj) {
                    const float a = wq[jj * RS + l];
                    const float4 w = *reinterpret_cast<const float4*>(wq + jj * RS + 4 * k4);
                    acc.x = fmaf(a, w.x, acc.x);
                    acc.y = fmaf(a, w.y, acc.y);
                    acc.z = fmaf(a, w.z, acc.z);
                    acc.w = fmaf(a, w.w, acc.w);
                }
            }
            *reinterpret_cast<float4*>(slot + (int64_t)row * q.rp + 4 * k4) = acc;
        }
    }
}

// Step 2: entries [e4_begin, e4_begin + e4_count) (float4 units of a slot) summed
// over the chunks; this CTA takes its contiguous share and writes dst[e - e4_begin].
// Chunks are summed in groups of QG in increasing order, then the groups in order.
__device__ void reduce_slots(const CoarseParams& q, int e4_begin, int e4_count, float4* dst, float4* scr4) {
    const int G = gridDim.x;
    const int S = (e4_count + G - 1) / G;
    const int j_begin = blockIdx.x * S;
    const int j_end = min(e4_count, j_begin + S);
    const int NGq = (q.nchunk + QG - 1) / QG;
    const int Sb = max(1, min(S, CT / NGq));
    const int64_t stride4 = q.part_stride / 4;
    const float4* part4 = reinterpret_cast<const float4*>(q.part);
    for (int jb = j_begin; jb < j_end; jb += Sb) {
        const int nb = min(Sb, j_end - jb);
        for (int t = threadIdx.x; t < nb * NGq; t += CT) {
            const int j = t % nb, g = t / nb;
            const int64_t e4 = e4_begin + jb + j;
            const int c0 = g * QG, c1 = min(q.nchunk, c0 + QG);
            // all loads of the group in flight at once, then added in chunk order
            float4 v[QG];
#pragma unroll
            for (int u = 0; u < QG; ++u)
                v[u] = c0 + u < c1 ? __ldcg(part4 + (int64_t)(c0 + u) * stride4 + e4) : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 s = v[0];
#pragma unroll
            for (int u = 1; u < QG; ++u)
                if (c0 + u < c1) s = f4add(s, v[u]);
            scr4[t] = s;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < nb; j += CT) {
            float4 s = scr4[j];
            for (int g = 1; g < NGq; ++g) s = f4add(s, scr4[g * nb + j]);
            dst[jb + j] = s;
        }
        __syncthreads();
    }
}

// Row update of up to kMaxRows rows (row stride RS) by four threads per row.
// F: rows to update (entries >= r are zero and stay zero); P: product rows;
// G: Gram matrix in the padded layout gidx(), zero outside r x r; ginv: 1 / G_kk
// (0 where G_kk = 0, which leaves that entry unchanged).  `valid`: this thread's
// row exists.
// One step k = 16 q0 + i0 of the HALS walk (Algorithm 3): the thread that owns
// block q0 updates entry i0 of its row, the delta is broadcast to the row's four
// threads and each removes its contribution from its entries of g.  gk holds this
// thread's 16 entries of Gram row k (loaded a step ahead).
__device__ __forceinline__ void hals_step(int i0, int qd, int q0, int gbase, const float4* gk, float* f, float* g,
                                          const float* gi) {
    float dl = 0.f;
    if (qd == q0) {
        const float nv = fmaxf(0.f, fmaf(g[i0], gi[i0], f[i0]));
        dl = nv - f[i0];
        f[i0] = nv;
    }
    const float d = __shfl_sync(0xffffffffu, dl, gbase + q0);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        g[4 * v] = fmaf(-d, gk[v].x, g[4 * v]);
        g[4 * v + 1] = fmaf(-d, gk[v].y, g[4 * v + 1]);
        g[4 * v + 2] = fmaf(-d, gk[v].z, g[4 * v + 2]);
        g[4 * v + 3] = fmaf(-d, gk[v].w, g[4 * v + 3]);
    }
}

// Steps k = 16 q0 .. 16 q0 + nb - 1 in order, the Gram row of step k + 1 loaded while
// step k runs.
template <bool FULL>
__device__ __forceinline__ void hals_block(int q0, int nb, int qd, int gbase, const float* G, float* f, float* g,
                                           const float* gi) {
    float4 cur[4], nxt[4];
    const float4* row0 = reinterpret_cast<const float4*>(G + (16 * q0) * GS + qd * GB);
#pragma unroll
    for (int v = 0; v < 4; ++v) nxt[v] = row0[v];
#pragma unroll
    for (int i0 = 0; i0 < 16; ++i0) {
        if (FULL || i0 < nb) {
#pragma unroll
            for (int v = 0; v < 4; ++v) cur[v] = nxt[v];
            if (i0 + 1 < 16 && (FULL || i0 + 1 < nb)) {
                const float4* rn = reinterpret_cast<const float4*>(G + (16 * q0 + i0 + 1) * GS + qd * GB);
#pragma unroll
                for (int v = 0; v < 4; ++v) nxt[v] = rn[v];
            }
            hals_step(i0, qd, q0, gbase, cur, f, g, gi);
        }
    }
}

template <int MODE>
__device__ __noinline__ void quad_rows(int nrows, bool valid, float* F, const float* P, const float* G,
                                       const float* ginv, int r) {
    const int tid = threadIdx.x;
    if ((tid & ~31) / 4 >= nrows) return;  // whole warp past the last row (warp-uniform)
    const int rr = tid >> 2, qd = tid & 3;
    const int gbase = (tid & 31) & ~3;
    const bool act = rr < nrows && valid;
    float f[16], g[16];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const float4 fv = act ? *reinterpret_cast<const float4*>(F + rr * RS + 16 * qd + 4 * v)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
        f[4 * v] = fv.x;
        f[4 * v + 1] = fv.y;
        f[4 * v + 2] = fv.z;
        f[4 * v + 3] = fv.w;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) g[j] = 0.f;
    // F_i G over l = 0 .. r-1 in increasing order
    if (act) {
#pragma unroll 4
        for (int l = 0; l < r; ++l) {
            const float fl = F[rr * RS + l];
            const float4* gl = reinterpret_cast<const float4*>(G + l * GS + qd * GB);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float4 gv = gl[v];
                g[4 * v] = fmaf(fl, gv.x, g[4 * v]);
                g[4 * v + 1] = fmaf(fl, gv.y, g[4 * v + 1]);
                g[4 * v + 2] = fmaf(fl, gv.z, g[4 * v + 2]);
                g[4 * v + 3] = fmaf(fl, gv.w, g[4 * v + 3]);
            }
        }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const float4 p4 = act ? *reinterpret_cast<const float4*>(P + rr * RS + 16 * qd + 4 * v)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
        const float pv[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = 4 * v + e;
            if (MODE == 0)
                g[j] = pv[e] - g[j];
            else
                f[j] = act ? f[j] * pv[e] / fmaxf(g[j], 1e-30f) : 0.f;
        }
    }
    if (MODE == 0) {
        // this thread's pivots (it owns block qd of every row)
        float gi[16];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float4 t = *reinterpret_cast<const float4*>(ginv + 16 * qd + 4 * v);
            gi[4 * v] = t.x;
            gi[4 * v + 1] = t.y;
            gi[4 * v + 2] = t.z;
            gi[4 * v + 3] = t.w;
        }
        // k = 16 q0 + i0 in increasing order: full blocks without a per-step test,
        // then the last partial block
        const int full = r >> 4;
        for (int q0 = 0; q0 < full; ++q0) hals_block<true>(q0, 16, qd, gbase, G, f, g, gi);
        if (r & 15) hals_block<false>(full, r & 15, qd, gbase, G, f, g, gi);
    }
    __syncwarp();  // the four threads of a row are done reading it
    if (act) {
#pragma unroll
        for (int v = 0; v < 4; ++v)
            *reinterpret_cast<float4*>(F + rr * RS + 16 * qd + 4 * v) =
                make_float4(f[4 * v], f[4 * v + 1], f[4 * v + 2], f[4 * v + 3]);
    }
}

template <int MODE>
__global__ void __launch_bounds__(CT, 1) coarse_run_kernel(const CoarseParams q) {
    extern __shared__ __align__(16) unsigned char csm[];
    const int m = q.m, r = q.r, rp = q.rp, nq4 = rp / 4;
    const CLayout L = clayout(m, q.cpc, r);
    const int JS = L.JS, MS = L.MS;
    float* Ms = reinterpret_cast<float*>(csm + L.ms);
    float* Ws = reinterpret_cast<float*>(csm + L.ws);
    float* Vs = reinterpret_cast<float*>(csm + L.vs);
    float* Ps = reinterpret_cast<float*>(csm + L.ps);
    float* Bs = reinterpret_cast<float*>(csm + L.bs);
    float* Ds = reinterpret_cast<float*>(csm + L.ds);
    float* binv = reinterpret_cast<float*>(csm + L.binv);
    float* dinv = reinterpret_cast<float*>(csm + L.dinv);
    float* scr = reinterpret_cast<float*>(csm + L.scr);
    int* flag = reinterpret_cast<int*>(csm + L.flag);
    const int tid = threadIdx.x;
    const int G = gridDim.x;
    unsigned nb = 0;

    // ---- load the level: M_l columns and W^T rows of this CTA's chunks, all of V_l
    for (int e = tid; e < 64 * GS; e += CT) Bs[e] = Ds[e] = 0.f;
    for (int e = tid; e < (m > JS ? m : JS) * RS; e += CT) Ps[e] = 0.f;
    for (int lq = 0; lq < q.cpc; ++lq) {
        const int chunk = blockIdx.x + lq * G;
        for (int e = tid; e < m * CW; e += CT) {
            const int i = e / CW, jj = e % CW;
            const int64_t j = (int64_t)chunk * CW + jj;
            Ms[i * MS + lq * CW + jj] = (chunk < q.nchunk && j < q.n) ? q.M[i * q.ldm + j] : 0.f;
        }
        for (int e = tid; e < CW * 16; e += CT) {
            const int jj = e / 16, k4 = e % 16;
            const int64_t j = (int64_t)chunk * CW + jj;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (chunk < q.nchunk && j < q.n && 4 * k4 < rp) v = *reinterpret_cast<const float4*>(q.Wt + j * rp + 4 * k4);
            const int c = 4 * k4;
            v.x = c < r ? v.x : 0.f;
            v.y = c + 1 < r ? v.y : 0.f;
            v.z = c + 2 < r ? v.z : 0.f;
            v.w = c + 3 < r ? v.w : 0.f;
            *reinterpret_cast<float4*>(Ws + (lq * CW + jj) * RS + 4 * k4) = v;
        }
    }
    for (int e = tid; e < m * 16; e += CT) {
        const int i = e / 16, k4 = e % 16;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (4 * k4 < rp) v = *reinterpret_cast<const float4*>(q.V + (int64_t)i * rp + 4 * k4);
        const int c = 4 * k4;
        v.x = c < r ? v.x : 0.f;
        v.y = c + 1 < r ? v.y : 0.f;
        v.z = c + 2 < r ? v.z : 0.f;
        v.w = c + 3 < r ? v.w : 0.f;
        *reinterpret_cast<float4*>(Vs + i * RS + 4 * k4) = v;
    }
    __syncthreads();

    // this thread's row of W^T in the W-step row update
    const int wr = tid >> 2;
    const int64_t wrow = (int64_t)(blockIdx.x + (wr / CW) * G) * CW + (wr % CW);
    const bool wvalid = wr < JS && wrow < q.n;
    const int nq = (r + 3) / 4;
    const int NPc = max(1, min(4, CT / (JS * 16)));
    const int perc = (m + NPc - 1) / NPc;

    for (int s = 0; s < q.sweeps; ++s) {
        // ---- 1-2: A = M_l W^T and B = W W^T from the chunk partials
        chunk_partials(q, Ms, MS, Ws, true);
        if (!grid_sync(q.bar, q.err_flag, ++nb, flag, q.spins)) return;
        reduce_slots(q, 0, (m + r) * nq4, reinterpret_cast<float4*>(q.red), reinterpret_cast<float4*>(scr));
        if (!grid_sync(q.bar, q.err_flag, ++nb, flag, q.spins)) return;

        // ---- 3: V-step in every CTA
        // A rows into Ps, B into Bs (columns past rp zero); four loads in flight per thread
        const float4* red4 = reinterpret_cast<const float4*>(q.red);
        for (int base = 0; base < (m + r) * 16; base += 4 * CT) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = base + u * CT + tid, row = e / 16, k4 = e % 16;
                v[u] = (row < m + r && k4 < nq4) ? __ldcg(red4 + row * nq4 + k4) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = base + u * CT + tid, row = e / 16, k4 = e % 16;
                if (row < m)
                    *reinterpret_cast<float4*>(Ps + row * RS + 4 * k4) = v[u];
                else if (row < m + r)
                    *reinterpret_cast<float4*>(Bs + gidx(row - m, 4 * k4)) = v[u];
            }
        }
        __syncthreads();
        for (int k = tid; k < 64; k += CT) binv[k] = (k < r && Bs[gidx(k, k)] > 0.f) ? 1.f / Bs[gidx(k, k)] : 0.f;
        __syncthreads();
        quad_rows<MODE>(m, true, Vs, Ps, Bs, binv, r);
        __syncthreads();
        // ---- D = V^T V (4 x 4 outputs per item, rows of V in increasing order) and the
        // W-step's products C = M_l^T V for this CTA's rows (NPc row ranges of V, added in
        // order) in one pass: both only read V_l
        const int nD = nq * nq, nC = NPc * JS * 16;
        for (int t = tid; t < nD + nC; t += CT) {
            if (t < nD) {
                const int l4 = t / nq, k4 = t % nq;
                float a[4][4];
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) a[x][y] = 0.f;
                for (int i = 0; i < m; ++i) {
                    const float4 u = *reinterpret_cast<const float4*>(Vs + i * RS + 4 * l4);
                    const float4 v = *reinterpret_cast<const float4*>(Vs + i * RS + 4 * k4);
                    const float uu[4] = {u.x, u.y, u.z, u.w}, vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) a[x][y] = fmaf(uu[x], vv[y], a[x][y]);
                }
#pragma unroll
                for (int x = 0; x < 4; ++x)
                    *reinterpret_cast<float4*>(Ds + gidx(4 * l4 + x, 4 * k4)) =
                        make_float4(a[x][0], a[x][1], a[x][2], a[x][3]);
            } else {
                const int tc = t - nD;
                const int part = tc / (JS * 16), rem = tc % (JS * 16);
                const int jr = rem / 16, k4 = rem % 16;
                const int i0 = part * perc, i1 = min(m, i0 + perc);
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                if (k4 < nq4) {
                    for (int i = i0; i < i1; ++i) {
                        const float a = Ms[i * MS + jr];
                        const float4 v = *reinterpret_cast<const float4*>(Vs + i * RS + 4 * k4);
                        acc.x = fmaf(a, v.x, acc.x);
                        acc.y = fmaf(a, v.y, acc.y);
                        acc.z = fmaf(a, v.z, acc.z);
                        acc.w = fmaf(a, v.w, acc.w);
                    }
                }
                if (NPc == 1)
                    *reinterpret_cast<float4*>(Ps + jr * RS + 4 * k4) = acc;
                else
                    *reinterpret_cast<float4*>(scr + (size_t)part * JS * 64 + jr * 64 + 4 * k4) = acc;
            }
        }
        __syncthreads();
        for (int k = tid; k < 64; k += CT) dinv[k] = (k < r && Ds[gidx(k, k)] > 0.f) ? 1.f / Ds[gidx(k, k)] : 0.f;
        if (NPc > 1) {
            for (int e = tid; e < JS * 16; e += CT) {
                const int jr = e / 16, k4 = e % 16;
                float4 sum = *reinterpret_cast<const float4*>(scr + jr * 64 + 4 * k4);
                for (int part = 1; part < NPc; ++part)
                    sum = f4add(sum, *reinterpret_cast<const float4*>(scr + (size_t)part * JS * 64 + jr * 64 + 4 * k4));
                *reinterpret_cast<float4*>(Ps + jr * RS + 4 * k4) = sum;
            }
        }
        __syncthreads();
        quad_rows<MODE>(JS, wvalid, Ws, Ps, Ds, dinv, r);
        __syncthreads();
    }

    // ---- B = W W^T of the final W into Bout; V_l and W^T back to global memory
    chunk_partials(q, Ms, MS, Ws, false);
    if (!grid_sync(q.bar, q.err_flag, ++nb, flag, q.spins)) return;
    reduce_slots(q, m * nq4, r * nq4, reinterpret_cast<float4*>(q.Bout), reinterpret_cast<float4*>(scr));
    for (int e = tid; e < JS * nq4; e += CT) {
        const int jr = e / nq4, k4 = e % nq4;
        const int64_t j = (int64_t)(blockIdx.x + (jr / CW) * G) * CW + (jr % CW);
        if (j < q.n)
            *reinterpret_cast<float4*>(q.Wt + j * rp + 4 * k4) = *reinterpret_cast<const float4*>(Ws + jr * RS + 4 * k4);
    }
    for (int e = tid; e < m * nq4; e += CT) {
        const int i = e / nq4, k4 = e % nq4;
        if (i % G == (int)blockIdx.x)
            *reinterpret_cast<float4*>(q.V + (int64_t)i * rp + 4 * k4) = *reinterpret_cast<const float4*>(Vs + i * RS + 4 * k4);
    }
}

}  // namespace

cudaError_t coarse_init() {
    cudaError_t e = cudaFuncSetAttribute(coarse_run_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(coarse_run_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    return e;
}

int64_t coarse_slot_floats(int64_t m, int r, int rp) { return round_up((m + r) * rp, 64); }

bool coarse_fits(int64_t m, int64_t n, int r, int max_grid, size_t* smem, int* cpc, int* nchunk, int* grid) {
    if (m < 1 || m > kMaxVRows || n < 1 || r < 1 || r > kMaxRank || max_grid < 1) return false;
    const int64_t nc = ceil_div(n, CW);
    if (nc > (int64_t)CT * QG) return false;
    // one CTA per chunk up to the SM count: more CTAs would only add barrier arrivals
    const int g = (int)std::min<int64_t>(nc, max_grid);
    const int c = (int)ceil_div(nc, g);
    if (CW * c > kMaxRows) return false;  // the W-step row update covers kMaxRows rows
    const CLayout L = clayout((int)m, c, r);
    if (L.total > kMaxSmem) return false;
    if (smem) *smem = L.total;
    if (cpc) *cpc = c;
    if (nchunk) *nchunk = (int)nc;
    if (grid) *grid = g;
    return true;
}

cudaError_t coarse_run_launch(const CoarseParams& q, int mode, int grid, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(q.bar, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(CT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return mode == 0 ? cudaLaunchKernelEx(&cfg, coarse_run_kernel<0>, q) : cudaLaunchKernelEx(&cfg, coarse_run_kernel<1>, q);
}

}  // namespace nmfk
