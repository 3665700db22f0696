// Global stage (Sec. 2.3, eq. hdg_global_mat; Algorithm 1 steps 2-4):
//   * the skeleton operator (I - A_int): per element y_K = x_K - in2out_K x_in(K), the inflow
//     gathered from the neighbours' outflow blocks (a block-sparse matvec, one thread block per
//     element, in2out streamed once from HBM with 16-byte loads);
//   * restarted GMRES with classical Gram-Schmidt applied twice; every kernel of a restart cycle
//     is enqueued at once and turns into a no-op once the device-side convergence flag is set, so
//     the host synchronises once per cycle;
//   * mean-intensity recovery u^m_K = in2sol_K x_in(K) with the boundary data included.
// Vectors: with FP32 operators the Krylov vectors are float-float pairs (about 44 bits) and every
// product and sum runs on the FP32 pipes (GB300 issues FP64 at ~1/64 of FP32, and even a one-lane
// FP64 instruction occupies its FP64 pipe for a warp); with FP64 operators they are FP64.  The
// Hessenberg matrix, the Givens rotations and the reduction results are FP64 (a few hundred values).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "elrt_internal.h"
#include "ff.h"

namespace {

constexpr int kThreads = 256;
constexpr int kDotBlocks = 304;  // 2 per SM
constexpr int kMaxRestart = 200;

struct GmState {
    int done;      // 1 once converged (or broken down) inside the current cycle
    int j_done;    // Arnoldi steps completed in the current cycle
    int pad[2];
    double bnorm;  // ||b||
    double beta;   // ||r0|| of the current cycle
    double res;    // estimated residual norm
    double tol;    // rtol * ||b||
};

// ------------------------------------------------------------------------------------------------
// vector arithmetic in FP64 or float-float
// ------------------------------------------------------------------------------------------------

template <typename V> struct VA;
template <> struct VA<double> {
    static __device__ __forceinline__ double zero() { return 0.0; }
    static __device__ __forceinline__ double from_d(double x) { return x; }
    static __device__ __forceinline__ double to_d(double x) { return x; }
    static __device__ __forceinline__ void fma(double& acc, double a, double b) { acc = ::fma(a, b, acc); }
    static __device__ __forceinline__ double add(double a, double b) { return a + b; }
    static __device__ __forceinline__ double neg(double a) { return -a; }
    static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
    static __device__ __forceinline__ double norm(double a) { return a; }
    static __device__ __forceinline__ double shfl_sum(double a) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
        return a;
    }
};
template <> struct VA<ff> {
    static __device__ __forceinline__ ff zero() { return ff{0.f, 0.f}; }
    static __device__ __forceinline__ ff from_d(double x) { return ff_from_double(x); }
    static __device__ __forceinline__ double to_d(ff x) { return ff_to_double(x); }
    static __device__ __forceinline__ void fma(ff& acc, ff a, ff b) { ff_fma(acc, a, b); }
    static __device__ __forceinline__ ff add(ff a, ff b) { return ff_add(a, b); }
    static __device__ __forceinline__ ff neg(ff a) { return ff{-a.h, -a.l}; }
    static __device__ __forceinline__ ff mul(ff a, ff b) { return ff_mul(a, b); }
    static __device__ __forceinline__ ff norm(ff a) { return ff_norm(a.h, a.l); }
    static __device__ __forceinline__ ff shfl_sum(ff a) { return ff_warp_sum(ff_norm(a.h, a.l)); }
};

// ------------------------------------------------------------------------------------------------
// block-sparse matvec
// ------------------------------------------------------------------------------------------------

// y_K = alpha * xself_K + beta * (Aop_K x_in(K)) with alpha, beta in {-1, 0, 1}; Aop_K: rows x nin
// (row-major); x_in(K) gathered from x (neighbours' outflow, NULL: zero) and g (boundary data, NULL:
// zero).  FP32 operators: float-float accumulation; FP64 operators: FP64 accumulation.
template <typename A, typename V>
__global__ void __launch_bounds__(kThreads) k_elem_gemv(int nx, int nz, int nin, int nface, int rows,
                                                        const A* __restrict__ Aop, const V* __restrict__ x,
                                                        const double* __restrict__ g, const V* __restrict__ xself,
                                                        int alpha, int beta, V* __restrict__ y,
                                                        const GmState* __restrict__ st) {
    if (st && st->done) return;
    constexpr int kMaxIn = 4 * ELRT_MAX_N1 * (ELRT_MAX_ANG / 2);
    __shared__ __align__(16) double xin[sizeof(A) == 8 ? kMaxIn : 1];
    __shared__ __align__(16) ff xff[sizeof(A) == 4 ? kMaxIn : 1];
    const int64_t e = blockIdx.x;
    const int ix = (int)(e % nx), iz = (int)(e / nx);
    for (int c = threadIdx.x; c < nin; c += kThreads) {
        const int F = c / nface, off = c - F * nface;
        const int jx = ix + (F == 1) - (F == 3), jz = iz + (F == 2) - (F == 0);
        V v = VA<V>::zero();
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
            v = VA<V>::from_d(g[side0 + (int64_t)face * nface + off]);
        }
        if constexpr (sizeof(A) == 8) {
            xin[c] = VA<V>::to_d(v);
        } else if constexpr (std::is_same<V, double>::value) {
            xff[c] = ff_from_double(v);
        } else {
            xff[c] = v;
        }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const A* Ae = Aop + e * (int64_t)rows * nin;
    for (int r = warp; r < rows; r += 2 * (kThreads / 32)) {
        const int r2 = r + kThreads / 32;
        V s1, s2;
        if constexpr (sizeof(A) == 4) {
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
            if constexpr (std::is_same<V, ff>::value) {
                s1 = a1;
                s2 = a2;
            } else {
                s1 = ff_to_double(a1);
                s2 = ff_to_double(a2);
            }
        } else {
            const int nv = nin / 2;
            const double2* A2 = reinterpret_cast<const double2*>(Ae);
            double d1 = 0.0, d2 = 0.0;
            for (int q = lane; q < nv; q += 32) {
                const double2 v1 = __ldcs(A2 + (int64_t)r * nv + q);
                d1 += v1.x * xin[2 * q] + v1.y * xin[2 * q + 1];
                if (r2 < rows) {
                    const double2 v2 = __ldcs(A2 + (int64_t)r2 * nv + q);
                    d2 += v2.x * xin[2 * q] + v2.y * xin[2 * q + 1];
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                d1 += __shfl_down_sync(0xffffffffu, d1, off);
                d2 += __shfl_down_sync(0xffffffffu, d2, off);
            }
            s1 = VA<V>::from_d(d1);
            s2 = VA<V>::from_d(d2);
        }
        if (lane == 0) {
            const int64_t o1 = e * rows + r;
            V t1 = beta > 0 ? s1 : (beta < 0 ? VA<V>::neg(s1) : VA<V>::zero());
            if (alpha) t1 = VA<V>::add(alpha > 0 ? xself[o1] : VA<V>::neg(xself[o1]), t1);
            y[o1] = t1;
            if (r2 < rows) {
                const int64_t o2 = e * rows + r2;
                V t2 = beta > 0 ? s2 : (beta < 0 ? VA<V>::neg(s2) : VA<V>::zero());
                if (alpha) t2 = VA<V>::add(alpha > 0 ? xself[o2] : VA<V>::neg(xself[o2]), t2);
                y[o2] = t2;
            }
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Krylov kernels
// ------------------------------------------------------------------------------------------------

template <typename V>
__device__ __forceinline__ double block_sum_to_double(V v, V* red) {
    v = VA<V>::shfl_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += VA<V>::to_d(red[w]);
    return s;
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
template <typename V>
__global__ void __launch_bounds__(kThreads) k_dots(const V* __restrict__ Vb, int64_t n, const V* __restrict__ w,
                                                   double* __restrict__ partial, const GmState* __restrict__ st) {
    if (st && st->done) return;
    __shared__ V red[kThreads / 32];
    const int i = blockIdx.y;
    const V* v = Vb + (int64_t)i * n;
    V s = VA<V>::zero();
    for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads)
        VA<V>::fma(s, v[k], w[k]);
    const double tot = block_sum_to_double(VA<V>::norm(s), red);
    if (threadIdx.x == 0) partial[(int64_t)i * gridDim.x + blockIdx.x] = tot;
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

// w += sign * sum_{i < nvec} h[i] V[i]
template <typename V>
__global__ void __launch_bounds__(kThreads) k_axpy_multi(const V* __restrict__ Vb, int64_t n, int nvec,
                                                         const double* __restrict__ h, V* __restrict__ w, int sign,
                                                         const GmState* __restrict__ st) {
    if (st && st->done) return;
    __shared__ V hs[kMaxRestart + 1];
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) hs[i] = VA<V>::from_d(sign < 0 ? -h[i] : h[i]);
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads) {
        V s = w[k];
        for (int i = 0; i < nvec; ++i) VA<V>::fma(s, hs[i], Vb[(int64_t)i * n + k]);
        w[k] = VA<V>::norm(s);
    }
}

// w /= *d (skipped when *d == 0: lucky breakdown)
template <typename V>
__global__ void k_scale(V* __restrict__ w, int64_t n, const double* __restrict__ d, const GmState* __restrict__ st) {
    if (st && st->done) return;
    const double dv = *d;
    if (dv == 0.0) return;
    const V inv = VA<V>::from_d(1.0 / dv);
    for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads)
        w[k] = VA<V>::mul(w[k], inv);
}

// r = b - r
template <typename V>
__global__ void k_bminus(const V* __restrict__ b, V* __restrict__ r, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads)
        r[k] = VA<V>::add(b[k], VA<V>::neg(r[k]));
}

__global__ void k_d2ff(const double* __restrict__ a, ff* __restrict__ b, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads)
        b[k] = ff_from_double(a[k]);
}

__global__ void k_ff2d(const ff* __restrict__ a, double* __restrict__ b, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads)
        b[k] = ff_to_double(a[k]);
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

// y = R^{-1} g on the j_done x j_done upper triangle
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

// x += sum_{i < j_done} y_i V_i
template <typename V>
__global__ void __launch_bounds__(kThreads) k_update_x(const V* __restrict__ Vb, int64_t n,
                                                       const double* __restrict__ y, V* __restrict__ x,
                                                       const GmState* __restrict__ st) {
    __shared__ V ys[kMaxRestart + 1];
    const int nj = st->j_done;
    for (int i = threadIdx.x; i < nj; i += blockDim.x) ys[i] = VA<V>::from_d(y[i]);
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads) {
        V s = x[k];
        for (int i = 0; i < nj; ++i) VA<V>::fma(s, ys[i], Vb[(int64_t)i * n + k]);
        x[k] = VA<V>::norm(s);
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

template <typename A, typename V>
elrt_status launch_gemv(elrt_ctx* ctx, int nx, int nz, int rows, const void* Aop, const V* x, const double* g,
                        const V* xself, int alpha, int beta, V* y, const GmState* st) {
    const Tab& t = ctx->tab;
    const int64_t E = (int64_t)nx * nz;
    if (E > 0x7fffffffLL) return ctx_fail(ctx, ELRT_EINVAL, "too many elements");
    ProfScope ps(ctx, "gemv");
    k_elem_gemv<A, V><<<(unsigned)E, kThreads, 0, ctx->stream>>>(nx, nz, t.nin, t.nface, rows, (const A*)Aop, x, g,
                                                                 xself, alpha, beta, y, st);
    return cuda_check(ctx, cudaGetLastError(), "gemv launch");
}

unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(4 * 152, (n + kThreads - 1) / kThreads)); }

// GMRES with Krylov vectors of type V (operators of type A).
template <typename A, typename V>
elrt_status gmres(elrt_ctx* ctx, int nx, int nz, const void* Aop, const double* inflow, double rtol, int max_iter,
                  int restart, int use_guess, double* xout, elrt_solve_stats* stats) {
    const Tab& t = ctx->tab;
    const int64_t n = (int64_t)nx * nz * t.nin;
    const int m = restart;
    const int nblk = kDotBlocks;
    const bool own_x = !std::is_same<V, double>::value;  // float-float iterate kept apart from the FP64 output
    // workspace: V[(m+1) n], b[n], x[n] (float-float only), then the FP64 small arrays and the state
    const size_t vbytes = ((size_t)(m + 2) * n + (own_x ? n : 0)) * sizeof(V);
    const size_t small = ((size_t)(m + 1) * m + 4 * (size_t)(m + 1) + (size_t)(m + 1) * nblk + 64) * sizeof(double);
    elrt_status s = ensure_ws(ctx, &ctx->gm, &ctx->gm_bytes, vbytes + small + sizeof(GmState) + 512);
    if (s) return s;
    V* Vb = (V*)ctx->gm;
    V* b = Vb + (size_t)(m + 1) * n;
    V* x = own_x ? b + n : (V*)xout;
    double* H = (double*)((unsigned char*)ctx->gm + ((vbytes + 255) & ~(size_t)255));
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
    const int rows = t.nin;

    // b = A g_bnd
    s = launch_gemv<A, V>(ctx, nx, nz, rows, Aop, nullptr, inflow, nullptr, 0, 1, b, nullptr);
    if (s) return s;
    { ProfScope ps(ctx, "krylov"); k_dots<V><<<dim3(nblk, 1), kThreads, 0, sm>>>(b, n, b, partial, nullptr); }
    { ProfScope ps(ctx, "krylov"); k_dots_finish<<<1, kThreads, 0, sm>>>(partial, nblk, scal, 2, nullptr); }
    if (!use_guess) {
        s = cuda_check(ctx, cudaMemsetAsync(x, 0, n * sizeof(V), sm), "zero x");
        if (s) return s;
    } else if constexpr (std::is_same<V, ff>::value) {
        ProfScope ps(ctx, "krylov");
        k_d2ff<<<gb, kThreads, 0, sm>>>(xout, x, n);
    }
    s = cuda_check(ctx, cudaMemcpyAsync(ctx->h_pinned, scal, sizeof(double), cudaMemcpyDeviceToHost, sm), "read ||b||");
    if (!s) s = cuda_check(ctx, cudaStreamSynchronize(sm), "sync ||b||");
    if (s) return s;
    prof_flush(ctx);
    const double bnorm = *(double*)ctx->h_pinned;
    if (!(bnorm > 0.0)) {
        s = cuda_check(ctx, cudaMemsetAsync(xout, 0, n * sizeof(double), sm), "zero x");
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
        s = launch_gemv<A, V>(ctx, nx, nz, rows, Aop, x, nullptr, x, 1, -1, Vb, nullptr);
        if (s) return s;
        { ProfScope ps(ctx, "krylov"); k_bminus<V><<<gb, kThreads, 0, sm>>>(b, Vb, n); }
        { ProfScope ps(ctx, "krylov"); k_dots<V><<<dim3(nblk, 1), kThreads, 0, sm>>>(Vb, n, Vb, partial, nullptr); }
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
        { ProfScope ps(ctx, "krylov"); k_scale<V><<<gb, kThreads, 0, sm>>>(Vb, n, scal + 1, nullptr); }
        { ProfScope ps(ctx, "krylov"); k_cycle_start<<<1, 1, 0, sm>>>(st, gv, m, scal + 1); }
        const int mj = std::min(m, max_iter - its);
        for (int j = 0; j < mj; ++j) {
            V* vj = Vb + (size_t)j * n;
            V* w = Vb + (size_t)(j + 1) * n;
            double* hc = H + (size_t)j * (m + 1);
            s = launch_gemv<A, V>(ctx, nx, nz, rows, Aop, vj, nullptr, vj, 1, -1, w, st);
            if (s) return s;
            // classical Gram-Schmidt, twice
            { ProfScope ps(ctx, "krylov"); k_dots<V><<<dim3(nblk, j + 1), kThreads, 0, sm>>>(Vb, n, w, partial, st); }
            { ProfScope ps(ctx, "krylov"); k_dots_finish<<<j + 1, kThreads, 0, sm>>>(partial, nblk, hc, 0, st); }
            { ProfScope ps(ctx, "krylov"); k_axpy_multi<V><<<gb, kThreads, 0, sm>>>(Vb, n, j + 1, hc, w, -1, st); }
            { ProfScope ps(ctx, "krylov"); k_dots<V><<<dim3(nblk, j + 1), kThreads, 0, sm>>>(Vb, n, w, partial, st); }
            { ProfScope ps(ctx, "krylov"); k_dots_finish<<<j + 1, kThreads, 0, sm>>>(partial, nblk, yv, 0, st); }
            { ProfScope ps(ctx, "krylov"); k_dots_finish<<<j + 1, kThreads, 0, sm>>>(partial, nblk, hc, 1, st); }  // h += second pass
            { ProfScope ps(ctx, "krylov"); k_axpy_multi<V><<<gb, kThreads, 0, sm>>>(Vb, n, j + 1, yv, w, -1, st); }
            // h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}
            { ProfScope ps(ctx, "krylov"); k_dots<V><<<dim3(nblk, 1), kThreads, 0, sm>>>(w, n, w, partial, st); }
            { ProfScope ps(ctx, "krylov"); k_dots_finish<<<1, kThreads, 0, sm>>>(partial, nblk, hc + j + 1, 2, st); }
            { ProfScope ps(ctx, "krylov"); k_scale<V><<<gb, kThreads, 0, sm>>>(w, n, hc + j + 1, st); }
            { ProfScope ps(ctx, "krylov"); k_givens<<<1, 1, 0, sm>>>(H, m + 1, cs, sn, gv, j, st); }
        }
        { ProfScope ps(ctx, "krylov"); k_solve_upper<<<1, 1, 0, sm>>>(H, m + 1, gv, yv, st); }
        { ProfScope ps(ctx, "krylov"); k_update_x<V><<<gb, kThreads, 0, sm>>>(Vb, n, yv, x, st); }
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
    if constexpr (std::is_same<V, ff>::value) {
        ProfScope ps(ctx, "krylov");
        k_ff2d<<<gb, kThreads, 0, sm>>>(x, xout, n);
        s = cuda_check(ctx, cudaStreamSynchronize(sm), "output");
        if (s) return s;
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

}  // namespace

elrt_status global_apply(elrt_ctx* ctx, int nx, int nz, const void* A, int dtype, const double* x, double* y) {
    if (dtype == ELRT_F32) return launch_gemv<float, double>(ctx, nx, nz, ctx->tab.nin, A, x, nullptr, x, 1, -1, y, nullptr);
    return launch_gemv<double, double>(ctx, nx, nz, ctx->tab.nin, A, x, nullptr, x, 1, -1, y, nullptr);
}

elrt_status global_recover(elrt_ctx* ctx, int nx, int nz, const void* A, int dtype, const double* x,
                           const double* inflow, double* mean) {
    if (dtype == ELRT_F32)
        return launch_gemv<float, double>(ctx, nx, nz, ctx->tab.nm, A, x, inflow, nullptr, 0, 1, mean, nullptr);
    return launch_gemv<double, double>(ctx, nx, nz, ctx->tab.nm, A, x, inflow, nullptr, 0, 1, mean, nullptr);
}

elrt_status global_solve(elrt_ctx* ctx, int nx, int nz, const void* A, int dtype, const double* inflow, double rtol,
                         int max_iter, int restart, int use_guess, double* x, elrt_solve_stats* stats) {
    if (restart > kMaxRestart) return ctx_fail(ctx, ELRT_EINVAL, "restart above 200");
    if (dtype == ELRT_F32) return gmres<float, ff>(ctx, nx, nz, A, inflow, rtol, max_iter, restart, use_guess, x, stats);
    return gmres<double, double>(ctx, nx, nz, A, inflow, rtol, max_iter, restart, use_guess, x, stats);
}
