// ANLS factor update (Algorithm ANLS, Section 2.1; Appendix A.2).
//
// The V-step updates the rows of V from (A = M W^T, B = W W^T); the W-step
// updates the rows of Wt = W^T from (C^T = M^T V, D = V^T V).  Each row solves
//     min_{x >= 0} 1/2 x^T G x - P_i x
// by the Lawson-Hanson active-set method in FP64, one warp per row, with the
// Cholesky factor of the passive block grown column by column (HALS and MU are
// updated inside the fused half-sweep kernel and the BF16 row kernel).
#include "nmf_internal.cuh"
#include "ptx.cuh"

namespace nmfk {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// ANLS: warp-per-row Lawson-Hanson NNLS in FP64.
// Distributed vectors: entry k lives in lane k & 31, slot k >> 5.
// ---------------------------------------------------------------------------
constexpr int kAnlsWarps = 8;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// Row i of the packed lower-triangular factor starts at tri(i).
__device__ __forceinline__ int tri(int i) { return i * (i + 1) / 2; }

// Cholesky factor L (packed lower triangle) of G restricted to the passive variables
// ord[0..p), kept in the order the variables entered; inv[k] = position of k;
// dinv[i] = 1 / L_ii (the solves then need no division, which costs about ten
// FP64 multiply-adds).  Full factorization of the set `mask` (variables in
// increasing index order).  Returns false if a pivot falls below 1e-12 of its
// original diagonal (the passive columns are numerically dependent).
__device__ bool chol_full(const double* G, int r, uint64_t mask, double* L, double* dinv, int* ord, int* inv, int& p,
                          int lane) {
    p = __popcll(mask);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int k = lane + 32 * s;
        if (k < r && ((mask >> k) & 1ull)) {
            const int pos = __popcll(mask & ((1ull << k) - 1ull));
            ord[pos] = k;
            inv[k] = pos;
        }
    }
    __syncwarp();
    for (int e = lane; e < p * p; e += 32) {
        const int i = e / p, j = e - i * p;
        if (j <= i) L[tri(i) + j] = G[ord[i] * r + ord[j]];
    }
    __syncwarp();
    for (int k = 0; k < p; ++k) {
        const double d0 = L[tri(k) + k];
        if (!(d0 > 1e-12 * G[ord[k] * r + ord[k]])) return false;  // uniform over the warp
        const double d = sqrt(d0), di = 1.0 / d;
        __syncwarp();
        if (lane == 0) {
            L[tri(k) + k] = d;
            dinv[k] = di;
        }
        for (int i = k + 1 + lane; i < p; i += 32) L[tri(i) + k] *= di;
        __syncwarp();
        // trailing update of the lower triangle, entries spread evenly over the lanes
        const int nt = p - k - 1;
        if (nt > 0) {
            int i = lane / nt, j = lane - (lane / nt) * nt;
            const int di2 = 32 / nt, dj = 32 - di2 * nt;
            for (int e = lane; e < nt * nt; e += 32) {
                if (j <= i) {
                    const int ti = tri(k + 1 + i);
                    L[ti + (k + 1 + j)] -= L[ti + k] * L[tri(k + 1 + j) + k];
                }
                i += di2;
                j += dj;
                if (j >= nt) {
                    j -= nt;
                    ++i;
                }
            }
        }
        __syncwarp();
    }
    return true;
}

// Append variable j to the factor: solve L l = G[ord, j] by forward
// substitution, then l_jj = sqrt(G_jj - l.l).  False (factor unchanged) if
// column j is numerically dependent on the passive ones.
__device__ bool chol_append(const double* G, int r, int j, double* L, double* dinv, int* ord, int* inv, int& p,
                            double* y, int lane) {
    for (int i = lane; i < p; i += 32) y[i] = G[ord[i] * r + j];
    __syncwarp();
    for (int k = 0; k < p; ++k) {
        const double lk = y[k] * dinv[k];
        __syncwarp();
        if (lane == 0) y[k] = lk;
        for (int i = k + 1 + lane; i < p; i += 32) y[i] -= L[tri(i) + k] * lk;
        __syncwarp();
    }
    double ss = 0.0;
    for (int i = lane; i < p; i += 32) ss += y[i] * y[i];
    ss = warp_sum(ss);
    const double gjj = G[j * r + j];
    const double d0 = gjj - ss;
    if (!(d0 > 1e-12 * gjj)) return false;
    for (int i = lane; i < p; i += 32) L[tri(p) + i] = y[i];
    if (lane == 0) {
        const double d = sqrt(d0);
        L[tri(p) + p] = d;
        dinv[p] = 1.0 / d;
        ord[p] = j;
        inv[j] = p;
    }
    ++p;
    __syncwarp();
    return true;
}

// z_P = G_PP^{-1} b_P from the factor (forward and back substitution); z = 0 off P.
__device__ void chol_solve(const double* L, const double* dinv, int r, const int* ord, const int* inv, int p,
                           uint64_t mask, const double* bs, double z[2], double* y, int lane) {
    for (int i = lane; i < p; i += 32) y[i] = bs[ord[i]];
    __syncwarp();
    for (int j = 0; j < p; ++j) {
        const double yj = y[j] * dinv[j];
        __syncwarp();
        if (lane == 0) y[j] = yj;
        for (int i = j + 1 + lane; i < p; i += 32) y[i] -= L[tri(i) + j] * yj;
        __syncwarp();
    }
    for (int j = p - 1; j >= 0; --j) {
        const double zj = y[j] * dinv[j];
        __syncwarp();
        if (lane == 0) y[j] = zj;
        for (int i = lane; i < j; i += 32) y[i] -= L[tri(j) + i] * zj;
        __syncwarp();
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int k = lane + 32 * s;
        z[s] = (k < r && ((mask >> k) & 1ull)) ? y[inv[k]] : 0.0;
    }
    __syncwarp();
}

// Block principal pivoting (the alternative NNLS method of the ANLS footnote in
// Section 2.1): all infeasible variables (x_k < 0 in the passive set F, gradient
// g_k = (G x - b)_k < -tol outside it) change sides at once while their number keeps
// falling; after three exchanges without a fall only the one of largest index moves
// (backup rule).  Each iteration factors G_FF anew.  Returns false when a factor is
// numerically singular or the cap is reached (the caller then runs the active-set
// method); on true, x holds the solution (zero outside F).
__device__ bool bpp_row(const double* G, int r, const double b[2], const double* bs, double tol, double* L,
                        double* dinv, int* ord, int* inv, double* y, int lane, int max_iter, uint64_t warm,
                        double x[2]) {
    // the passive set starts from the support of the incoming row (a sweep's NNLS problems
    // change little from one sweep to the next, so this is usually the final set)
    uint64_t F = warm;
    double xv[2] = {0.0, 0.0};
    double g[2] = {-b[0], -b[1]};
    int nmin = r + 1, backup = 3, p = 0;
    for (int it = 0; it <= max_iter; ++it) {
        if (it > 0 || F) {
            xv[0] = xv[1] = 0.0;
            if (F) {
                if (!chol_full(G, r, F, L, dinv, ord, inv, p, lane)) return false;
                chol_solve(L, dinv, r, ord, inv, p, F, bs, xv, y, lane);
            }
            // gradient outside F: g = G x - b (zero in F)
            g[0] = -b[0];
            g[1] = -b[1];
            for (int l = 0; l < r; ++l) {
                const double xl = __shfl_sync(kFull, xv[l >> 5], l & 31);
                if (xl != 0.0) {
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        const int k = lane + 32 * s;
                        if (k < r) g[s] += G[k * r + l] * xl;
                    }
                }
            }
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int k = lane + 32 * s;
                if (k < r && ((F >> k) & 1ull)) g[s] = 0.0;
            }
        }
        uint64_t bad = 0;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int k = lane + 32 * s;
            const bool inF = k < r && ((F >> k) & 1ull);
            const bool infeasible = k < r && (inF ? xv[s] < 0.0 : g[s] < -tol);
            bad |= (uint64_t)__ballot_sync(kFull, infeasible) << (32 * s);
        }
        if (!bad) {
            x[0] = xv[0];
            x[1] = xv[1];
            return true;
        }
        const int nbad = __popcll(bad);
        if (nbad < nmin) {
            nmin = nbad;
            backup = 3;
            F ^= bad;
        } else if (backup > 0) {
            --backup;
            F ^= bad;
        } else {
            F ^= 1ull << (63 - __clzll((long long)bad));
        }
        if (it == max_iter) break;
    }
    return false;
}

// Per-warp shared memory of the ANLS kernel in doubles: L (packed, r (r+1)/2), dinv, y, bs.
__host__ __device__ inline size_t anls_warp_doubles(int r) { return (size_t)r * (r + 1) / 2 + 3 * kMaxRank; }

// G = sum of the Gram partial slabs in FP64 (slabs in index order), once per
// half-sweep, for all the ANLS rows.
__global__ void gram_reduce_f64_kernel(const UpdateArgs u) {
    ptx::grid_dependency_wait();  // the slabs and the flag come from the previous kernel
    ptx::launch_dependents();
    if (u.skip && *(volatile const int*)u.skip) return;
    const int r = u.r;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= r * r) return;
    const int l = idx / r, k = idx - l * r;
    const float* p = u.PG + (int64_t)l * u.ldpg + k;
    double s = 0;
    for (int q = 0; q < u.gsplits; ++q) s += (double)p[(int64_t)q * u.pgs];
    u.Gd[idx] = s;
}

template <bool BPP>
__global__ void __launch_bounds__(32 * kAnlsWarps) anls_rows_kernel(const UpdateArgs u, int* status) {
    extern __shared__ double smem[];
    ptx::grid_dependency_wait();  // G, the products and the flag come from earlier kernels
    ptx::launch_dependents();
    if (u.skip && *(volatile const int*)u.skip) return;  // same value in every CTA
    const int r = u.r;
    double* G = smem;  // r x r
    for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) G[idx] = u.Gd[idx];
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    double* L = G + r * r + (size_t)warp * anls_warp_doubles(r);
    double* dinv = L + (size_t)r * (r + 1) / 2;
    double* y = dinv + kMaxRank;
    double* bs = y + kMaxRank;
    const int nwarps = blockDim.x >> 5;
    int* ord = reinterpret_cast<int*>(G + r * r + (size_t)nwarps * anls_warp_doubles(r)) + warp * 2 * kMaxRank;
    int* inv = ord + kMaxRank;
    const uint64_t all = (r == 64) ? ~0ull : ((1ull << r) - 1ull);

    for (int64_t row = (int64_t)blockIdx.x * nwarps + warp; row < u.rows;
         row += (int64_t)gridDim.x * nwarps) {
        double b[2], x[2] = {0.0, 0.0}, z[2];
        uint64_t warm = 0;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int k = lane + 32 * s;
            b[s] = 0.0;
            if (k < r) {
                const float* pp = u.P + row * u.ldp + k;
                double acc = 0.0;
                for (int q = 0; q < u.splits; ++q) acc += (double)pp[(int64_t)q * u.ps];
                b[s] = acc;
                bs[k] = acc;
            }
            const bool pos = k < r && u.F[row * u.ldf + k] > 0.f;
            warm |= (uint64_t)__ballot_sync(kFull, pos) << (32 * s);
        }
        __syncwarp();
        const double bmax = warp_max(fmax(fabs(b[0]), fabs(b[1])));
        const double tol = 1e-12 * fmax(1.0, bmax);
        bool capped = false;
        if (BPP && bpp_row(G, r, b, bs, tol, L, dinv, ord, inv, y, lane, 5 * r, warm & all, x)) {
            // solved by block pivoting
        } else {
        uint64_t mask = 0, excluded = 0;
        int p = 0;

        // Warm start from the support of the incoming row: drop the variables
        // whose unconstrained solution is not positive until the rest is.
        mask = warm & all;
        for (int it = 0; it <= r && mask; ++it) {
            if (!chol_full(G, r, mask, L, dinv, ord, inv, p, lane)) {
                mask = 0;
                break;
            }
            chol_solve(L, dinv, r, ord, inv, p, mask, bs, z, y, lane);
            uint64_t badm = 0;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int k = lane + 32 * s;
                const bool bad = k < r && ((mask >> k) & 1ull) && !(z[s] > 0.0);
                badm |= (uint64_t)__ballot_sync(kFull, bad) << (32 * s);
            }
            if (!badm) {
                x[0] = z[0];
                x[1] = z[1];
                break;
            }
            mask &= ~badm;
        }
        if (!mask) {
            x[0] = x[1] = 0.0;
            p = 0;
        }

        // dual w = b - G x, recomputed only when x has changed: a candidate whose column
        // depends on the passive set is excluded without changing x
        double w[2] = {0.0, 0.0};
        bool have_w = false;
        for (int outer = 0;; ++outer) {
            // a passive set as large as G's rank bound spans the other factor's rows: the
            // residual of the row is zero and x is optimal (the duals left are rounding)
            if (u.rank_cap > 0 && p >= u.rank_cap) break;
            if (!have_w) {
                w[0] = b[0];
                w[1] = b[1];
                for (int l = 0; l < r; ++l) {
                    const double xl = __shfl_sync(kFull, x[l >> 5], l & 31);
                    if (xl != 0.0) {
#pragma unroll
                        for (int s = 0; s < 2; ++s) {
                            const int k = lane + 32 * s;
                            if (k < r) w[s] -= G[k * r + l] * xl;
                        }
                    }
                }
                have_w = true;
            }
            // entering variable: largest positive dual outside P (lowest index on ties)
            double best = -1.0;
            int bestk = 1 << 30;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int k = lane + 32 * s;
                if (k < r && !(((mask | excluded) >> k) & 1ull) && w[s] > tol && w[s] > best) {
                    best = w[s];
                    bestk = k;
                }
            }
            const double wbest = warp_max(best);
            if (!(wbest > tol)) break;
            const unsigned cand = __ballot_sync(kFull, best == wbest && bestk < (1 << 30));
            int j = 1 << 30;
            for (unsigned c = cand; c; c &= c - 1) {
                const int ln = __ffs(c) - 1;
                j = min(j, __shfl_sync(kFull, bestk, ln));
            }
            j = __shfl_sync(kFull, j, 0);
            if (outer >= (u.max_outer < 0 ? 3 * r : u.max_outer)) {
                capped = true;
                break;
            }
            // the factor of the passive set grows by one column
            if (!chol_append(G, r, j, L, dinv, ord, inv, p, y, lane)) {
                excluded |= 1ull << j;
                continue;
            }
            mask |= 1ull << j;
            have_w = false;
            for (int it = 0; it <= r; ++it) {
                chol_solve(L, dinv, r, ord, inv, p, mask, bs, z, y, lane);
                uint64_t badm = 0;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const int k = lane + 32 * s;
                    const bool bad = k < r && ((mask >> k) & 1ull) && !(z[s] > 0.0);
                    badm |= (uint64_t)__ballot_sync(kFull, bad) << (32 * s);
                }
                if (!badm) {
                    x[0] = z[0];
                    x[1] = z[1];
                    break;
                }
                // step from x towards z until the first passive variable hits zero
                double ratio[2] = {INFINITY, INFINITY};
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const int k = lane + 32 * s;
                    if (k < r && ((badm >> k) & 1ull)) ratio[s] = x[s] / (x[s] - z[s]);
                }
                const double alpha = warp_min(fmin(ratio[0], ratio[1]));
                uint64_t drop = 0;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const int k = lane + 32 * s;
                    bool inP = k < r && ((mask >> k) & 1ull);
                    if (inP) {
                        x[s] = x[s] + alpha * (z[s] - x[s]);
                        if (ratio[s] <= alpha) x[s] = 0.0;
                    }
                    drop |= (uint64_t)__ballot_sync(kFull, inP && !(x[s] > 0.0)) << (32 * s);
                }
                mask &= ~drop;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const int k = lane + 32 * s;
                    if (k >= r || !((mask >> k) & 1ull)) x[s] = 0.0;
                }
                // the passive set shrank: refactor it
                if (!chol_full(G, r, mask, L, dinv, ord, inv, p, lane)) {
                    mask &= ~(1ull << j);
                    excluded |= 1ull << j;
                    if ((j & 31) == lane) x[j >> 5] = 0.0;
                    if (!chol_full(G, r, mask, L, dinv, ord, inv, p, lane)) {
                        mask = 0;
                        p = 0;
                        x[0] = x[1] = 0.0;
                    }
                    break;
                }
            }
        }
        }  // active set
        if (capped && lane == 0) atomicOr(status, 1);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int k = lane + 32 * s;
            if (k < r) u.F[row * u.ldf + k] = (float)x[s];
        }
    }
}

}  // namespace

static size_t anls_smem_bytes(int r, int nwarps) {
    return sizeof(double) * ((size_t)r * r + nwarps * anls_warp_doubles(r)) + sizeof(int) * nwarps * 2 * kMaxRank;
}

cudaError_t init_kernel_attributes() {
    cudaError_t e = cudaFuncSetAttribute(anls_rows_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)anls_smem_bytes(kMaxRank, kAnlsWarps));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(anls_rows_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)anls_smem_bytes(kMaxRank, kAnlsWarps));
    return e;
}

namespace {
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
}  // namespace

cudaError_t anls_update_launch(const UpdateArgs& u, int num_sms, int* d_status, cudaStream_t st) {
    if (u.rows <= 0) return cudaSuccess;
    if (!u.Gd) return cudaErrorInvalidValue;
    cudaError_t e = launch_pdl(gram_reduce_f64_kernel, dim3((unsigned)ceil_div((int64_t)u.r * u.r, 256)), dim3(256), 0,
                               st, u);
    if (e != cudaSuccess) return e;
    // one warp per row, FP64-bound: fewer warps per CTA when the rows would not reach every
    // SM with kAnlsWarps per CTA (the rows of a coarse level's V-step, for example)
    int nw = kAnlsWarps;
    while (nw > 1 && ceil_div(u.rows, nw) < num_sms) nw /= 2;
    const size_t smem = anls_smem_bytes(u.r, nw);
    int64_t grid = ceil_div(u.rows, nw);
    const int64_t cap = 8LL * num_sms * (kAnlsWarps / nw);
    if (grid > cap) grid = cap;
    if (u.bpp) return launch_pdl(anls_rows_kernel<true>, dim3((unsigned)grid), dim3(32 * nw), smem, st, u, d_status);
    return launch_pdl(anls_rows_kernel<false>, dim3((unsigned)grid), dim3(32 * nw), smem, st, u, d_status);
}

}  // namespace nmfk
