// Global stage (Sec. 2.3, eq. hdg_global_mat; Algorithm 1 steps 2-4):
//   * the skeleton operator (I - A_int): per element y_K = x_K - in2out_K x_in(K), the inflow
//     gathered from the neighbours' outflow blocks (a block-sparse matvec, one thread block per
//     element, in2out streamed once from HBM with 16-byte loads, FP64 accumulation);
//   * restarted GMRES with classical Gram-Schmidt applied twice, FP64 vectors and reductions;
//     every kernel of a restart cycle is enqueued at once and turns into a no-op once the
//     device-side convergence flag is set, so the host synchronises once per cycle;
//   * mean-intensity recovery u^m_K = in2sol_K x_in(K) with the boundary data included.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "elrt_internal.h"
#include "ff.h"

namespace {

constexpr int kThreads = 256;
constexpr int kDotBlocks = 304;  // 2 per SM

struct GmState {
    int done;      // 1 once converged (or broken down) inside the current cycle
    int j_done;    // Arnoldi steps completed in the current cycle
    int pad[2];
    double bnorm;  // ||b||
    double beta;   // ||r0|| of the current cycle
    double res;    // estimated residual norm
    double tol;    // rtol * ||b||
};

// y_K = alpha * xself_K + beta * (Aop_K x_in(K)),  Aop_K: rows x nin (row-major),
// x_in(K) gathered from x (neighbours' outflow, NULL: zero) and g (boundary data, NULL: zero).
// FP32 operators: float-float accumulation; FP64 operators: FP64 accumulation.
template <typename A>
__global__ void __launch_bounds__(kThreads) k_elem_gemv(int nx, int nz, int nin, int nface, int rows,
                                                        const A* __restrict__ Aop, const double* __restrict__ x,
                                                        const double* __restrict__ g, const double* __restrict__ xself,
                                                        double alpha, double beta, double* __restrict__ y,
                                                        const GmState* __restrict__ st) {
    if (st && st->done) return;
    constexpr int kMaxIn = 4 * ELRT_MAX_N1 * (ELRT_MAX_ANG / 2);
    __shared__ __align__(16) double xin[kMaxIn];
    __shared__ __align__(16) ff xff[kMaxIn];
    const int64_t e = blockIdx.x;
    const int ix = (int)(e % nx), iz = (int)(e / nx);
    for (int c = threadIdx.x; c < nin; c += kThreads) {
        const int F = c / nface, off = c - F * nface;
        const int jx = ix + (F == 1) - (F == 3), jz = iz + (F == 2) - (F == 0);
        double v = 0.0;
        if (jx >= 0 && jx < nx && jz >= 0 && jz < nz) {
            if (x) {
                const int G = (F + 2) & 3;  // opposite face
                v = x[((int64_t)jz * nx + jx) * nin + G * nface + off];
            }
        } else if (g) {
            int64_t side0;
            int face;
            switch (F) {
                case 0: side0 = 0; face = ix; break;
                case 1: side0 = (int64_t)nx * nface; face = iz; break;
                case 2: side0 = (int64_t)(nx + nz) * nface; face = ix; break;
                default: side0 = (int64_t)(2 * nx + nz) * nface; face = iz; break;
            }
            v = g[side0 + (int64_t)face * nface + off];
        }
        xin[c] = v;
        xff[c] = ff_from_double(v);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const A* Ae = Aop + e * (int64_t)rows * nin;
    for (int r = warp; r < rows; r += 2 * (kThreads / 32)) {
        const int r2 = r + kThreads / 32;
        double s1 = 0.0, s2 = 0.0;
        if constexpr (sizeof(A) == 4) {
            // float-float: exact products of the FP32 entries with x = xh + xl, TwoSum accumulation
            const int nv = nin / 4;
            const float4* A4 = reinterpret_cast<const float4*>(Ae);
            ff a1{0.f, 0.f}, a2{0.f, 0.f};
            for (int q = lane; q < nv; q += 32) {
                const float4 v1 = __ldcs(A4 + (int64_t)r * nv + q);
                ff_fma_f(a1, v1.x, xff[4 * q]);
                ff_fma_f(a1, v1.y, xff[4 * q + 1]);
                ff_fma_f(a1, v1.z, xff[4 * q + 2]);
                ff_fma_f(a1, v1.w, xff[4 * q + 3]);
                if (r2 < rows) {
                    const float4 v2 = __ldcs(A4 + (int64_t)r2 * nv + q);
                    ff_fma_f(a2, v2.x, xff[4 * q]);
                    ff_fma_f(a2, v2.y, xff[4 * q + 1]);
                    ff_fma_f(a2, v2.z, xff[4 * q + 2]);
                    ff_fma_f(a2, v2.w, xff[4 * q + 3]);
                }
            }
            a1 = ff_warp_sum(ff_norm(a1.h, a1.l));
            a2 = ff_warp_sum(ff_norm(a2.h, a2.l));
            s1 = ff_to_double(a1);
            s2 = ff_to_double(a2);
        } else {
            const int nv = nin / 2;
            const double2* A2 = reinterpret_cast<const double2*>(Ae);
            for (int q = lane; q < nv; q += 32) {
                const double2 v1 = __ldcs(A2 + (int64_t)r * nv + q);
                s1 += v1.x * xin[2 * q] + v1.y * xin[2 * q + 1];
                if (r2 < rows) {
                    const double2 v2 = __ldcs(A2 + (int64_t)r2 * nv + q);
                    s2 += v2.x * xin[2 * q] + v2.y * xin[2 * q + 1];
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                s1 += __shfl_down_sync(0xffffffffu, s1, off);
                s2 += __shfl_down_sync(0xffffffffu, s2, off);
            }
        }
        if (lane == 0) {
            const int64_t o1 = e * rows + r;
            y[o1] = (xself ? alpha * xself[o1] : 0.0) + beta * s1;
            if (r2 < rows) {
                const int64_t o2 = e * rows + r2;
                y[o2] = (xself ? alpha * xself[o2] : 0.0) + beta * s2;
            }
        }
    }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

// partial[i * nblk + blk] = sum over this block's slice of V[i] . w   (grid: nblk x nvec)
__global__ void __launch_bounds__(kThreads) k_dots(const double* __restrict__ V, int64_t n, const double* __restrict__ w,
                                                   double* __restrict__ partial, const GmState* __restrict__ st) {
    if (st && st->done) return;
    __shared__ double red[kThreads / 32];
    const int i = blockIdx.y;
    const double* v = V + (int64_t)i * n;
    double s = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads)
        s += v[k] * w[k];
    s = block_sum(s, red);
    if (threadIdx.x == 0) partial[(int64_t)i * gridDim.x + blockIdx.x] = s;
}

// out[i] (op 0: =, op 1: +=) sum_blk partial[i * nblk + blk], fixed order; op 2: out[0] = sqrt(sum)
__global__ void k_dots_finish(const double* __restrict__ partial, int nblk, double* __restrict__ out, int op,
                              const GmState* __restrict__ st) {
    if (st && st->done) return;
    __shared__ double red[kThreads / 32];
    const int i = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[(int64_t)i * nblk + b];
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        if (op == 0) out[i] = s;
        else if (op == 1) out[i] += s;
        else out[i] = sqrt(s);
    }
}

// w -= sum_{i < nvec} h[i] V[i]
__global__ void __launch_bounds__(kThreads) k_axpy_multi(const double* __restrict__ V, int64_t n, int nvec,
                                                         const double* __restrict__ h, double* __restrict__ w,
                                                         const GmState* __restrict__ st) {
    if (st && st->done) return;
    for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads) {
        double s = w[k];
        for (int i = 0; i < nvec; ++i) s -= h[i] * V[(int64_t)i * n + k];
        w[k] = s;
    }
}

// w /= *d (skipped when *d == 0: lucky breakdown)
__global__ void k_scale(double* __restrict__ w, int64_t n, const double* __restrict__ d, const GmState* __restrict__ st) {
    if (st && st->done) return;
    const double dv = *d;
    if (dv == 0.0) return;
    const double inv = 1.0 / dv;
    for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads) w[k] *= inv;
}

// r = b - r
__global__ void k_bminus(const double* __restrict__ b, double* __restrict__ r, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads)
        r[k] = b[k] - r[k];
}

// Column j of H (column-major, ld = m+1) was filled with h (rows 0..j) and h_{j+1,j}: apply the
// previous Givens rotations, build rotation j, update g and test convergence.
__global__ void k_givens(double* __restrict__ H, int ldh, double* __restrict__ cs, double* __restrict__ sn,
                         double* __restrict__ gv, int j, GmState* __restrict__ st) {
    if (st->done) return;
    double* h = H + (int64_t)j * ldh;
    const double hnext = h[j + 1];
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * h[i] + sn[i] * h[i + 1];
        h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
        h[i] = t;
    }
    const double d = hypot(h[j], h[j + 1]);
    const double c = d > 0 ? h[j] / d : 1.0, s = d > 0 ? h[j + 1] / d : 0.0;
    cs[j] = c;
    sn[j] = s;
    h[j] = d;
    h[j + 1] = 0.0;
    gv[j + 1] = -s * gv[j];
    gv[j] = c * gv[j];
    st->j_done = j + 1;
    st->res = fabs(gv[j + 1]);
    if (st->res <= st->tol || hnext == 0.0) st->done = 1;
}

// y = R^{-1} g on the j_done x j_done upper triangle, then x += V y.
__global__ void k_solve_upper(const double* __restrict__ H, int ldh, const double* __restrict__ gv,
                              double* __restrict__ y, const GmState* __restrict__ st) {
    const int nj = st->j_done;
    for (int i = nj - 1; i >= 0; --i) {
        double s = gv[i];
        for (int k = i + 1; k < nj; ++k) s -= H[(int64_t)k * ldh + i] * y[k];
        const double d = H[(int64_t)i * ldh + i];
        y[i] = d != 0.0 ? s / d : 0.0;
    }
}

__global__ void __launch_bounds__(kThreads) k_update_x(const double* __restrict__ V, int64_t n,
                                                       const double* __restrict__ y, double* __restrict__ x,
                                                       const GmState* __restrict__ st) {
    const int nj = st->j_done;
    for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads) {
        double s = x[k];
        for (int i = 0; i < nj; ++i) s += y[i] * V[(int64_t)i * n + k];
        x[k] = s;
    }
}

__global__ void k_cycle_start(GmState* st, double* gv, int m, const double* beta) {
    st->done = 0;
    st->j_done = 0;
    st->beta = *beta;
    st->res = *beta;
    gv[0] = *beta;
    for (int i = 1; i <= m; ++i) gv[i] = 0.0;
}

template <typename A>
elrt_status launch_gemv(elrt_ctx* ctx, int nx, int nz, int rows, const void* Aop, const double* x, const double* g,
                        const double* xself, double alpha, double beta, double* y, const GmState* st) {
    const Tab& t = ctx->tab;
    const int64_t E = (int64_t)nx * nz;
    if (E > 0x7fffffffLL) return ctx_fail(ctx, ELRT_EINVAL, "too many elements");
    ProfScope ps(ctx, "gemv");
    k_elem_gemv<A><<<(unsigned)E, kThreads, 0, ctx->stream>>>(nx, nz, t.nin, t.nface, rows, (const A*)Aop, x, g, xself,
                                                              alpha, beta, y, st);
    return cuda_check(ctx, cudaGetLastError(), "gemv launch");
}

elrt_status gemv(elrt_ctx* ctx, int dtype, int nx, int nz, int rows, const void* Aop, const double* x, const double* g,
                 const double* xself, double alpha, double beta, double* y, const GmState* st) {
    if (dtype == ELRT_F32) return launch_gemv<float>(ctx, nx, nz, rows, Aop, x, g, xself, alpha, beta, y, st);
    return launch_gemv<double>(ctx, nx, nz, rows, Aop, x, g, xself, alpha, beta, y, st);
}

unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(4 * 152, (n + kThreads - 1) / kThreads)); }

}  // namespace

elrt_status global_apply(elrt_ctx* ctx, int nx, int nz, const void* A, int dtype, const double* x, double* y) {
    return gemv(ctx, dtype, nx, nz, ctx->tab.nin, A, x, nullptr, x, 1.0, -1.0, y, nullptr);
}

elrt_status global_recover(elrt_ctx* ctx, int nx, int nz, const void* A, int dtype, const double* x,
                           const double* inflow, double* mean) {
    return gemv(ctx, dtype, nx, nz, ctx->tab.nm, A, x, inflow, nullptr, 0.0, 1.0, mean, nullptr);
}

elrt_status global_solve(elrt_ctx* ctx, int nx, int nz, const void* A, int dtype, const double* inflow, double rtol,
                         int max_iter, int restart, int use_guess, double* x, elrt_solve_stats* stats) {
    const Tab& t = ctx->tab;
    const int64_t n = (int64_t)nx * nz * t.nin;
    const int m = restart;
    const int nblk = kDotBlocks;
    // workspace: V[(m+1) n], b[n], H[(m+1) m], cs[m], sn[m], g[m+1], y[m], hcol[m+1], partial[(m+1) nblk], state
    const size_t doubles = (size_t)(m + 1) * n + n + (size_t)(m + 1) * m + 4 * (size_t)(m + 1) + (size_t)(m + 1) * nblk + 64;
    elrt_status s = ensure_ws(ctx, &ctx->gm, &ctx->gm_bytes, doubles * sizeof(double) + sizeof(GmState) + 256);
    if (s) return s;
    double* V = (double*)ctx->gm;
    double* b = V + (size_t)(m + 1) * n;
    double* H = b + n;
    double* cs = H + (size_t)(m + 1) * m;
    double* sn = cs + (m + 1);
    double* gv = sn + (m + 1);
    double* yv = gv + (m + 1);
    double* partial = yv + (m + 1);
    double* scal = partial + (size_t)(m + 1) * nblk;  // [0] ||b||, [1] beta
    GmState* st = (GmState*)(scal + 64);
    cudaStream_t sm = ctx->stream;
    const unsigned gb = grid_for(n);
    GmState* hst = (GmState*)ctx->h_pinned;

    // b = A g_bnd
    s = gemv(ctx, dtype, nx, nz, t.nin, A, nullptr, inflow, nullptr, 0.0, 1.0, b, nullptr);
    if (s) return s;
    { ProfScope ps(ctx, "krylov"); k_dots<<<dim3(nblk, 1), kThreads, 0, sm>>>(b, n, b, partial, nullptr); }
    { ProfScope ps(ctx, "krylov"); k_dots_finish<<<1, kThreads, 0, sm>>>(partial, nblk, scal, 2, nullptr); }
    if (!use_guess) {
        s = cuda_check(ctx, cudaMemsetAsync(x, 0, n * sizeof(double), sm), "zero x");
        if (s) return s;
    }
    s = cuda_check(ctx, cudaMemcpyAsync(ctx->h_pinned, scal, sizeof(double), cudaMemcpyDeviceToHost, sm), "read ||b||");
    if (!s) s = cuda_check(ctx, cudaStreamSynchronize(sm), "sync ||b||");
    if (s) return s;
    prof_flush(ctx);
    const double bnorm = *(double*)ctx->h_pinned;
    if (!(bnorm > 0.0)) {
        s = cuda_check(ctx, cudaMemsetAsync(x, 0, n * sizeof(double), sm), "zero x");
        if (!s) s = cuda_check(ctx, cudaStreamSynchronize(sm), "sync");
        if (stats) {
            stats->converged = 1;
            stats->rel_residual = 0.0;
        }
        return s;
    }
    GmState init{};
    init.bnorm = bnorm;
    init.tol = rtol * bnorm;
    s = cuda_check(ctx, cudaMemcpyAsync(st, &init, sizeof(GmState), cudaMemcpyHostToDevice, sm), "state init");
    if (s) return s;
    int its = 0, cycles = 0;
    double rel = 1.0;
    bool converged = false;
    for (;;) {
        // r = b - (I - A_int) x, beta = ||r||
        s = gemv(ctx, dtype, nx, nz, t.nin, A, x, nullptr, x, 1.0, -1.0, V, nullptr);
        if (s) return s;
        { ProfScope ps(ctx, "krylov"); k_bminus<<<gb, kThreads, 0, sm>>>(b, V, n); }
        { ProfScope ps(ctx, "krylov"); k_dots<<<dim3(nblk, 1), kThreads, 0, sm>>>(V, n, V, partial, nullptr); }
        { ProfScope ps(ctx, "krylov"); k_dots_finish<<<1, kThreads, 0, sm>>>(partial, nblk, scal + 1, 2, nullptr); }
        s = cuda_check(ctx, cudaMemcpyAsync(ctx->h_pinned, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, sm), "read beta");
        if (!s) s = cuda_check(ctx, cudaStreamSynchronize(sm), "sync beta");
        if (s) return s;
        prof_flush(ctx);
        const double beta = *(double*)ctx->h_pinned;
        rel = beta / bnorm;
        if (!(beta > rtol * bnorm) || !isfinite(beta)) {
            converged = isfinite(beta);
            break;
        }
        if (its >= max_iter) break;
        { ProfScope ps(ctx, "krylov"); k_scale<<<gb, kThreads, 0, sm>>>(V, n, scal + 1, nullptr); }
        { ProfScope ps(ctx, "krylov"); k_cycle_start<<<1, 1, 0, sm>>>(st, gv, m, scal + 1); }
        const int mj = std::min(m, max_iter - its);
        for (int j = 0; j < mj; ++j) {
            double* vj = V + (size_t)j * n;
            double* w = V + (size_t)(j + 1) * n;
            double* hc = H + (size_t)j * (m + 1);
            s = gemv(ctx, dtype, nx, nz, t.nin, A, vj, nullptr, vj, 1.0, -1.0, w, st);
            if (s) return s;
            // classical Gram-Schmidt, twice
            { ProfScope ps(ctx, "krylov"); k_dots<<<dim3(nblk, j + 1), kThreads, 0, sm>>>(V, n, w, partial, st); }
            { ProfScope ps(ctx, "krylov"); k_dots_finish<<<j + 1, kThreads, 0, sm>>>(partial, nblk, hc, 0, st); }
            { ProfScope ps(ctx, "krylov"); k_axpy_multi<<<gb, kThreads, 0, sm>>>(V, n, j + 1, hc, w, st); }
            { ProfScope ps(ctx, "krylov"); k_dots<<<dim3(nblk, j + 1), kThreads, 0, sm>>>(V, n, w, partial, st); }
            { ProfScope ps(ctx, "krylov"); k_dots_finish<<<j + 1, kThreads, 0, sm>>>(partial, nblk, yv, 0, st); }
            { ProfScope ps(ctx, "krylov"); k_dots_finish<<<j + 1, kThreads, 0, sm>>>(partial, nblk, hc, 1, st); }  // h += second pass
            { ProfScope ps(ctx, "krylov"); k_axpy_multi<<<gb, kThreads, 0, sm>>>(V, n, j + 1, yv, w, st); }
            // h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}
            { ProfScope ps(ctx, "krylov"); k_dots<<<dim3(nblk, 1), kThreads, 0, sm>>>(w, n, w, partial, st); }
            { ProfScope ps(ctx, "krylov"); k_dots_finish<<<1, kThreads, 0, sm>>>(partial, nblk, hc + j + 1, 2, st); }
            { ProfScope ps(ctx, "krylov"); k_scale<<<gb, kThreads, 0, sm>>>(w, n, hc + j + 1, st); }
            { ProfScope ps(ctx, "krylov"); k_givens<<<1, 1, 0, sm>>>(H, m + 1, cs, sn, gv, j, st); }
        }
        { ProfScope ps(ctx, "krylov"); k_solve_upper<<<1, 1, 0, sm>>>(H, m + 1, gv, yv, st); }
        { ProfScope ps(ctx, "krylov"); k_update_x<<<gb, kThreads, 0, sm>>>(V, n, yv, x, st); }
        s = cuda_check(ctx, cudaGetLastError(), "gmres launches");
        if (s) return s;
        s = cuda_check(ctx, cudaMemcpyAsync(hst, st, sizeof(GmState), cudaMemcpyDeviceToHost, sm), "read state");
        if (!s) s = cuda_check(ctx, cudaStreamSynchronize(sm), "sync cycle");
        if (s) return s;
        prof_flush(ctx);
        its += hst->j_done;
        ++cycles;
        if (hst->j_done == 0) break;  // no progress possible
    }
    if (stats) {
        stats->iterations = its;
        stats->restarts = cycles;
        stats->converged = converged ? 1 : 0;
        stats->rel_residual = rel;
    }
    if (!converged) return ctx_fail(ctx, ELRT_ENOCONV, "GMRES did not reach the tolerance");
    return ELRT_OK;
}
