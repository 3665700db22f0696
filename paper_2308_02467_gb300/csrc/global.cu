// Global stage (Sec. 2.3, eq. hdg_global_mat; Algorithm 1 steps 2-4):
//   * the skeleton operator (I - A_int): per element y_K = x_K - in2out_K x_in(K), the inflow
//     gathered from the neighbours' outflow blocks (a block-sparse matvec, one thread block per
//     element, in2out streamed once from HBM with 16-byte loads);
//   * restarted GMRES with classical Gram-Schmidt applied twice; every kernel of a restart cycle
//     is enqueued at once and turns into a no-op once the device-side convergence flag is set, so
//     the host synchronises once per cycle;
//   * mean-intensity recovery u^m_K = in2sol_K x_in(K) with the boundary data included.
// Vectors: with FP32 operators the Krylov basis is FP32 while the iterate, the right-hand side and
// the restart residual are float-float pairs (about 44 bits); every product and sum accumulates in
// float-float on the FP32 pipes (GB300 issues FP64 at ~1/64 of FP32, and even a one-lane FP64
// instruction occupies its FP64 pipe for a warp).  With FP64 operators everything is FP64.  The
// Hessenberg matrix, the Givens rotations and the reduction results are FP64 (a few hundred values).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include "elrt_internal.h"
#include "ff.h"
#include "tc_gemm.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kDotBlocks = 608;  // 4 per SM: enough warps in flight for the Krylov passes
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
// vector arithmetic: FP64 vectors accumulate in FP64; float-float and FP32 vectors accumulate in
// float-float (an FP32 x FP32 product is exact as a float-float pair, TwoProduct by FMA)
// ------------------------------------------------------------------------------------------------

template <typename V> struct KV;
template <> struct KV<double> {
    using acc = double;
    static __device__ __forceinline__ acc zero() { return 0.0; }
    static __device__ __forceinline__ acc load(double v) { return v; }
    static __device__ __forceinline__ acc coef(double c) { return c; }
    static __device__ __forceinline__ void fma_vv(acc& s, double a, double b) { s = ::fma(a, b, s); }
    static __device__ __forceinline__ void fma_cv(acc& s, acc c, double v) { s = ::fma(c, v, s); }
    static __device__ __forceinline__ double store(acc s) { return s; }
    static __device__ __forceinline__ double to_d(acc s) { return s; }
    static __device__ __forceinline__ acc add(acc a, acc b) { return a + b; }
    static __device__ __forceinline__ acc neg(acc a) { return -a; }
    static __device__ __forceinline__ acc mul(acc a, acc b) { return a * b; }
    static __device__ __forceinline__ acc shfl_sum(acc a) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
        return a;
    }
};
struct KVff {  // shared by the float-float and FP32 vector types
    using acc = ff;
    static __device__ __forceinline__ acc zero() { return ff{0.f, 0.f}; }
    static __device__ __forceinline__ acc coef(double c) { return ff_from_double(c); }
    static __device__ __forceinline__ double to_d(acc s) { return ff_to_double(s); }
    static __device__ __forceinline__ acc add(acc a, acc b) { return ff_add(a, b); }
    static __device__ __forceinline__ acc neg(acc a) { return ff{-a.h, -a.l}; }
    static __device__ __forceinline__ acc mul(acc a, acc b) { return ff_mul(a, b); }
    static __device__ __forceinline__ acc shfl_sum(acc a) { return ff_warp_sum(ff_norm(a.h, a.l)); }
};
template <> struct KV<ff> : KVff {
    static __device__ __forceinline__ acc load(ff v) { return v; }
    static __device__ __forceinline__ void fma_vv(acc& s, ff a, ff b) { ff_fma(s, a, b); }
    static __device__ __forceinline__ void fma_cv(acc& s, acc c, ff v) { ff_fma(s, c, v); }
    static __device__ __forceinline__ ff store(acc s) { return ff_norm(s.h, s.l); }
};
template <> struct KV<float> : KVff {
    static __device__ __forceinline__ acc load(float v) { return ff{v, 0.f}; }
    static __device__ __forceinline__ void fma_vv(acc& s, float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = fmaf(a, b, -p);
        float h, t;
        two_sum(s.h, p, h, t);
        s.h = h;
        s.l = __fadd_rn(s.l, __fadd_rn(t, e));
    }
    static __device__ __forceinline__ void fma_cv(acc& s, acc c, float v) { ff_fma_f(s, v, c); }
    static __device__ __forceinline__ float store(acc s) { return __fadd_rn(s.h, s.l); }
};

// staging of a gathered inflow value for the FP32-operator matvec
__device__ __forceinline__ ff to_ff(double v) { return ff_from_double(v); }
__device__ __forceinline__ ff to_ff(ff v) { return v; }
__device__ __forceinline__ ff to_ff(float v) { return ff{v, 0.f}; }

// ------------------------------------------------------------------------------------------------
// Arnoldi step for the FP32 basis (restart length below kArnMaxV), after the matvec of step j:
//   matvec       w = v_j - A v_j; with the streaming matvec its blocks then form h1 = V^T w and
//                ||w||^2 over their own output rows (k_arn_dots otherwise); the last block reduces
//                and decides whether a second Gram-Schmidt pass is needed: only if the first pass
//                removed more than kReorthCancel of ||w||^2 (||w||^2 - ||h1||^2 < 0.1 ||w||^2:
//                selective reorthogonalisation with the remaining norm below 0.32 ||w||)
//   k_arn_axdots w -= V h1; then either h2 = V^T w (second pass) or ||w||^2 on the block's slice
//   k_arn_axnorm second pass only: w -= V h2 and ||w||^2; the last block (or block 0 without a
//                second pass) writes the Hessenberg column h1 + h2, ||w|| and applies the Givens
//                rotations (as k_givens)
// The basis is kept unnormalised: slot i holds W_i with v_i = s_i W_i, s_i = 1 / ||w|| of the step
// that made it (s_0 = 1, the restart residual is scaled when it enters slot 0).  Every consumer
// folds s_i into its coefficients (dots, updates, the iterate) or, in the matvec, into the gathered
// input, so no pass over the vector is spent on the normalisation.
// The block that finishes last (a ticket counter behind a __threadfence of every block's partial
// writes) reduces the blocks' partials in a fixed order, so the results are deterministic; no
// block ever waits for another.  Sums accumulate in float-float, block results in FP64.
// ------------------------------------------------------------------------------------------------
constexpr int kArnThreads = 256;
constexpr int kArnMaxV = 32;  // restart length + 1 supported by this path
// Second Gram-Schmidt pass when the first removed more than this fraction of ||w||^2.  The common
// choice 1/2 (remaining norm below ||w|| / sqrt 2) ran the second pass on most Arnoldi steps of the
// benchmark without changing the iteration count or the final residual; each restart recomputes the
// true residual, so the basis only has to span the Krylov space well enough for the cycle.
constexpr double kReorthCancel = 0.9;

struct ArnState {
    unsigned ticket[4];
    int reorth;  // second Gram-Schmidt pass in this step
    double h1[kArnMaxV], h2[kArnMaxV], nrm;
    double sc[kArnMaxV + 1];  // s_i of the basis slots
};

// block barrier: all threads, or (kNamed) the kArnThreads threads of a block whose other warps
// have left (the streaming matvec's producer warp)
template <bool kNamed>
__device__ __forceinline__ void arn_sync() {
    if constexpr (kNamed) asm volatile("bar.sync 2, %0;" ::"r"(kArnThreads) : "memory");
    else __syncthreads();
}

// true in exactly one block: the last to finish its partial writes (all of which are then visible)
template <bool kNamed = false>
__device__ bool arn_last_block(unsigned* ticket) {
    __shared__ bool last;
    __threadfence();
    arn_sync<kNamed>();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    arn_sync<kNamed>();
    if (last) __threadfence();
    return last;
}

// out[i] = s_i sum_b P[i * nb + b] (i < nv; s_i = sc[i] for i < nsc, else 1), one warp per
// vector, fixed order; ticket reset to 0.  The partials are read through L2 (other blocks wrote
// them), all of a lane's loads issued before the first add, so they are in flight together.
__device__ void arn_finish(const double* P, unsigned nb, int nv, double* out, unsigned* ticket, const double* sc,
                           int nsc) {
    constexpr int kU = 20;  // loads per lane in flight: nb <= 640 in one round
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < nv; i += kArnThreads / 32) {
        const double* Pi = P + (int64_t)i * nb;
        double t = 0.0;
        for (unsigned b0 = 0; b0 < nb; b0 += 32u * kU) {
            double v[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const unsigned b = b0 + lane + 32u * u;
                v[u] = b < nb ? __ldcg(Pi + b) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) t += v[u];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
        if (lane == 0) out[i] = i < nsc ? t * __ldcg(sc + i) : t;
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

// P[i * nb + blk] = sum over the block's packs V_i . w (i < nv), eight vectors per sweep; the
// block's packs are map(t) for t < cnt (float4 indices into each vector)
template <bool kNamed, typename Map>
__device__ void arn_block_dots(const float4* __restrict__ V4, int64_t np, const float4* __restrict__ w4, int nv,
                               int64_t cnt, Map map, double* __restrict__ P, unsigned nb) {
    __shared__ ff red[kArnThreads / 32][8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int ib = 0; ib < nv; ib += 8) {
        ff acc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = ff{0.f, 0.f};
        for (int64_t t = threadIdx.x; t < cnt; t += kArnThreads) {
            const int64_t p = map(t);
            const float4 w = w4[p];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (ib + u < nv) {
                    const float4 v = V4[(int64_t)(ib + u) * np + p];
                    KV<float>::fma_vv(acc[u], v.x, w.x);
                    KV<float>::fma_vv(acc[u], v.y, w.y);
                    KV<float>::fma_vv(acc[u], v.z, w.z);
                    KV<float>::fma_vv(acc[u], v.w, w.w);
                }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const ff sum = ff_warp_sum(ff_norm(acc[u].h, acc[u].l));
            if (lane == 0) red[warp][u] = sum;
        }
        arn_sync<kNamed>();
        if (threadIdx.x < 8 && ib + (int)threadIdx.x < nv) {
            ff t{0.f, 0.f};
            for (int wp = 0; wp < kArnThreads / 32; ++wp) t = ff_add(t, red[wp][threadIdx.x]);
            P[(int64_t)(ib + threadIdx.x) * nb + blockIdx.x] = ff_to_double(t);
        }
        arn_sync<kNamed>();
    }
}

// the last block of the first pass: h1 = s_i (W_i . w) (i <= j), ||w||^2 in h1[j + 1], and the
// decision on the second pass
template <bool kNamed>
__device__ void arn_first_pass_finish(const double* P, unsigned nb, int j, ArnState* as) {
    const int nv = j + 1;
    arn_finish(P, nb, nv + 1, as->h1, &as->ticket[0], as->sc, nv);
    __threadfence_block();
    arn_sync<kNamed>();
    if (threadIdx.x < 32) {  // one warp: ||h1||^2 and the decision
        const int lane = threadIdx.x;
        const double h = lane < nv ? __ldcg(as->h1 + lane) : 0.0;
        double s = h * h;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane < nv) as->h2[lane] = 0.0;
        if (lane == 0) {
            const double w2 = __ldcg(as->h1 + nv);
            as->reorth = (w2 - s < (1.0 - kReorthCancel) * w2) ? 1 : 0;
        }
    }
}

// w -= sum_i c[i] s_i W_i on packs [p0, p1)
__device__ void arn_axpy(const float4* __restrict__ V4, int64_t np, float4* __restrict__ w4, int nv,
                         const double* c, const double* sc, int64_t p0, int64_t p1) {
    __shared__ ff cf[kArnMaxV];
    if (threadIdx.x < nv) cf[threadIdx.x] = KV<float>::coef(-c[threadIdx.x] * sc[threadIdx.x]);
    __syncthreads();
    for (int64_t p = p0 + threadIdx.x; p < p1; p += kArnThreads) {
        const float4 w = w4[p];
        ff a0 = KV<float>::load(w.x), a1 = KV<float>::load(w.y), a2 = KV<float>::load(w.z), a3 = KV<float>::load(w.w);
#pragma unroll 4
        for (int i = 0; i < nv; ++i) {
            const float4 v = V4[(int64_t)i * np + p];
            KV<float>::fma_cv(a0, cf[i], v.x);
            KV<float>::fma_cv(a1, cf[i], v.y);
            KV<float>::fma_cv(a2, cf[i], v.z);
            KV<float>::fma_cv(a3, cf[i], v.w);
        }
        w4[p] = make_float4(KV<float>::store(a0), KV<float>::store(a1), KV<float>::store(a2), KV<float>::store(a3));
    }
}

__device__ __forceinline__ void arn_slice(int64_t n, int64_t& np, int64_t& p0, int64_t& p1) {
    np = n / 4;
    p0 = np * blockIdx.x / gridDim.x;
    p1 = np * (blockIdx.x + 1) / gridDim.x;
}

// partial ||w||^2 of the block's slice into P[blockIdx.x]
__device__ void arn_block_norm(const float4* __restrict__ w4, int64_t p0, int64_t p1, double* __restrict__ P) {
    __shared__ ff red[kArnThreads / 32];
    ff acc{0.f, 0.f};
    for (int64_t p = p0 + threadIdx.x; p < p1; p += kArnThreads) {
        const float4 w = w4[p];
        KV<float>::fma_vv(acc, w.x, w.x);
        KV<float>::fma_vv(acc, w.y, w.y);
        KV<float>::fma_vv(acc, w.z, w.z);
        KV<float>::fma_vv(acc, w.w, w.w);
    }
    const ff sum = ff_warp_sum(ff_norm(acc.h, acc.l));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        ff t{0.f, 0.f};
        for (int wp = 0; wp < kArnThreads / 32; ++wp) t = ff_add(t, red[wp]);
        P[blockIdx.x] = ff_to_double(t);
    }
}

// Hessenberg column j from h1 + h2 and ||w||, s_{j+1} = 1 / ||w||, then the Givens rotations.
// Called by one warp: its lanes fetch the column and the rotations (through L2) into shared memory
// together, lane 0 applies the rotations in order, the lanes write the column back.
__device__ void arn_column(ArnState* as, int j, double nrm, double* H, int ldh, double* cs, double* sn, double* gv,
                           GmState* st) {
    __shared__ double hs[kArnMaxV + 1], css[kArnMaxV], sns[kArnMaxV];
    const int lane = threadIdx.x & 31, nv = j + 1;
    double* h = H + (int64_t)j * ldh;
    if (lane < nv) hs[lane] = __ldcg(as->h1 + lane) + __ldcg(as->h2 + lane);
    if (lane < j) {
        css[lane] = __ldcg(cs + lane);
        sns[lane] = __ldcg(sn + lane);
    }
    __syncwarp();
    if (lane == 0) {
        hs[nv] = nrm;
        as->sc[j + 1] = nrm > 0.0 ? 1.0 / nrm : 0.0;
        for (int i = 0; i < j; ++i) {
            const double t = css[i] * hs[i] + sns[i] * hs[i + 1];
            hs[i + 1] = -sns[i] * hs[i] + css[i] * hs[i + 1];
            hs[i] = t;
        }
        const double d = hypot(hs[j], hs[j + 1]);
        const double c = d > 0 ? hs[j] / d : 1.0, s = d > 0 ? hs[j + 1] / d : 0.0;
        cs[j] = c;
        sn[j] = s;
        hs[j] = d;
        hs[j + 1] = 0.0;
        const double g = __ldcg(gv + j);
        gv[j + 1] = -s * g;
        gv[j] = c * g;
        st->j_done = j + 1;
        st->res = fabs(gv[j + 1]);
        if (st->res <= st->tol || nrm == 0.0) st->done = 1;
    }
    __syncwarp();
    if (lane <= nv) h[lane] = hs[lane];
}

// Fused first Gram-Schmidt pass of the streaming matvec (null: plain matvec)
struct ArnFuse {
    ArnState* as;
    double* P;         // per-block partials, (j + 2) x gridDim.x
    const float* Vb;   // basis slots 0 .. j + 1 (slot j + 1 = the matvec's output w)
    int64_t n;         // vector length
    int j;
};

// ------------------------------------------------------------------------------------------------
// block-sparse matvec
// ------------------------------------------------------------------------------------------------

// y_K = alpha * xself_K + beta * (Aop_K x_in(K)) with alpha, beta in {-1, 0, 1}; Aop_K: rows x nin
// (row-major); x_in(K) gathered from x (neighbours' outflow, NULL: zero) and g (boundary data, NULL:
// zero).  FP32 operators: float-float accumulation; FP64 operators: FP64 accumulation.  The sum
// with the self term is formed in the accumulator type and rounded once to V.
template <typename A, typename V>
__global__ void __launch_bounds__(kThreads) k_elem_gemv(int nx, int nz, int nin, int nface, int rows,
                                                        const A* __restrict__ Aop, const V* __restrict__ x,
                                                        const double* __restrict__ g, const V* __restrict__ xself,
                                                        int alpha, int beta, V* __restrict__ y,
                                                        const GmState* __restrict__ st) {
    if (st && st->done) return;
    using K = KV<V>;
    using Acc = typename K::acc;
    constexpr int kMaxIn = 4 * ELRT_MAX_N1 * (ELRT_MAX_ANG / 2);
    __shared__ __align__(16) double xin[sizeof(A) == 8 ? kMaxIn : 1];
    __shared__ __align__(16) ff xff[sizeof(A) == 4 ? kMaxIn : 1];
    const int64_t e = blockIdx.x;
    const int ix = (int)(e % nx), iz = (int)(e / nx);
    for (int c = threadIdx.x; c < nin; c += kThreads) {
        const int F = c / nface, off = c - F * nface;
        const int jx = ix + (F == 1) - (F == 3), jz = iz + (F == 2) - (F == 0);
        int src = 0;  // 0: zero, 1: neighbour outflow, 2: boundary data
        V xv{};
        double gv = 0.0;
        if (jx >= 0 && jx < nx && jz >= 0 && jz < nz) {
            if (x) {
                const int G = (F + 2) & 3;  // opposite face
                xv = x[((int64_t)jz * nx + jx) * nin + G * nface + off];
                src = 1;
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
            gv = g[side0 + (int64_t)face * nface + off];
            src = 2;
        }
        if constexpr (sizeof(A) == 8) {
            xin[c] = src == 1 ? K::to_d(K::load(xv)) : gv;
        } else {
            xff[c] = src == 1 ? to_ff(xv) : (src == 2 ? ff_from_double(gv) : ff{0.f, 0.f});
        }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const A* Ae = Aop + e * (int64_t)rows * nin;
    for (int r = warp; r < rows; r += 2 * (kThreads / 32)) {
        const int r2 = r + kThreads / 32;
        Acc s1, s2;
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
            if constexpr (std::is_same<Acc, double>::value) {
                s1 = ff_to_double(a1);
                s2 = ff_to_double(a2);
            } else {
                s1 = a1;
                s2 = a2;
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
            s1 = K::coef(d1);
            s2 = K::coef(d2);
        }
        if (lane == 0) {
            const int64_t o1 = e * rows + r;
            Acc t1 = beta > 0 ? s1 : (beta < 0 ? K::neg(s1) : K::zero());
            if (alpha) t1 = K::add(alpha > 0 ? K::load(xself[o1]) : K::neg(K::load(xself[o1])), t1);
            y[o1] = K::store(t1);
            if (r2 < rows) {
                const int64_t o2 = e * rows + r2;
                Acc t2 = beta > 0 ? s2 : (beta < 0 ? K::neg(s2) : K::zero());
                if (alpha) t2 = K::add(alpha > 0 ? K::load(xself[o2]) : K::neg(K::load(xself[o2])), t2);
                y[o2] = K::store(t2);
            }
        }
    }
}

// Streaming variant for FP32 operators and their FP16 copy (the same y_K): a persistent grid walks
// the elements; per block one producer warp copies each element's operator in chunks of 8 RPW rows
// (contiguous in memory) into a ring of shared-memory stages with bulk asynchronous copies, and
// eight consumer warps, RPW rows each, form the row sums from shared memory against the gathered
// inflow (double-buffered per element) and combine them with the self term.  The FP16 copy only
// serves the Arnoldi steps (FP32 vectors in and out).
constexpr int kGvWarps = 8;           // consumer warps
constexpr int kGemvFlag = 16;         // d_flags slot: a copy wait of the streaming matvec timed out
constexpr int kF16Flag = 17;          // d_flags slot: the operator holds a value outside the FP16 range
constexpr int kGvStages = 3;
constexpr int kGvStageBytes = 32768;
constexpr int kGvThreads = 32 * (kGvWarps + 1);

__device__ __forceinline__ ff ff_shfl_xor(ff a, int m) {
    return ff{__shfl_xor_sync(0xffffffffu, a.h, m), __shfl_xor_sync(0xffffffffu, a.l, m)};
}

// Reduce RPW per-lane partial sums (rows q = 0..RPW-1) over the warp.  Afterwards lane L with
// L % (32 / RPW) == 0 holds the sum of row L / (32 / RPW).
template <int RPW>
__device__ __forceinline__ ff warp_rows_reduce(ff (&acc)[RPW], int lane) {
    ff v;
    if constexpr (RPW == 4) {
        const bool P = (lane >> 4) & 1;  // keep rows 2P, 2P + 1
        ff t[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const ff mine = P ? acc[2 + i] : acc[i];
            const ff other = P ? acc[i] : acc[2 + i];
            t[i] = ff_add(mine, ff_shfl_xor(other, 16));
        }
        const bool Q = (lane >> 3) & 1;  // keep row 2P + Q
        const ff mine = Q ? t[1] : t[0];
        const ff other = Q ? t[0] : t[1];
        v = ff_add(mine, ff_shfl_xor(other, 8));
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) v = ff_add(v, ff_shfl_xor(v, off));
    } else if constexpr (RPW == 2) {
        const bool P = (lane >> 4) & 1;
        const ff mine = P ? acc[1] : acc[0];
        const ff other = P ? acc[0] : acc[1];
        v = ff_add(mine, ff_shfl_xor(other, 16));
#pragma unroll
        for (int off = 8; off > 0; off >>= 1) v = ff_add(v, ff_shfl_xor(v, off));
    } else {
        v = acc[0];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v = ff_add(v, ff_shfl_xor(v, off));
    }
    return v;
}

// The same exchange for plain FP32 partial sums (any power-of-two RPW up to 32): each step halves
// the set of rows a lane keeps, selected by one lane bit from the top.
template <int RPW>
__device__ __forceinline__ float warp_rows_reduce_f(float (&v)[RPW], int lane) {
#pragma unroll
    for (int n = RPW, m = 16; n > 1; n >>= 1, m >>= 1) {
        const bool P = lane & m;
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            const float mine = P ? v[n / 2 + i] : v[i];
            const float other = P ? v[i] : v[n / 2 + i];
            v[i] = mine + __shfl_xor_sync(0xffffffffu, other, m);
        }
    }
#pragma unroll
    for (int m = 16 / RPW; m > 0; m >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], m);
    return v[0];
}

template <typename V, int RPW, typename AT>
__global__ void __launch_bounds__(kGvThreads, 2)
    k_gemv_stream(int nx, int nz, int nin, int nface, int rows, const AT* __restrict__ Aop,
                  const V* __restrict__ x, const double* __restrict__ g, const V* __restrict__ xself, int alpha,
                  int beta, V* __restrict__ y, const GmState* __restrict__ st, int* __restrict__ err, ArnFuse fz) {
    static_assert(std::is_same<AT, float>::value || std::is_same<V, float>::value, "FP16 operators: Arnoldi steps only");
    static_assert(32 * kGvWarps == kArnThreads, "the fused dots run on the consumer warps");
    if (st && st->done) return;
    using K = KV<V>;
    using Acc = typename K::acc;
    constexpr int CR = kGvWarps * RPW;  // rows per chunk
    constexpr int kStageElems = kGvStageBytes / (int)sizeof(AT);
    extern __shared__ __align__(128) unsigned char gsm[];
    AT* stages = reinterpret_cast<AT*>(gsm);
    ff* xs = reinterpret_cast<ff*>(gsm + kGvStages * kGvStageBytes);  // [2][nin]
    __shared__ uint64_t full[kGvStages], empty[kGvStages];
    __shared__ int abort_flag;
    volatile int* abort = &abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t E = (int64_t)nx * nz;
    const int nch = (rows + CR - 1) / CR;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kGvStages; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], kGvWarps);
        }
        *abort = 0;
        tc::fence_barrier_init();
    }
    __syncthreads();
    if (warp == kGvWarps) {  // producer
        if (lane == 0) {
            const uint64_t pol = tc::l2_evict_first();  // the operator is read once per matvec
            int it = 0;
            for (int64_t e = blockIdx.x; e < E && !*abort; e += gridDim.x) {
                for (int c = 0; c < nch; ++c, ++it) {
                    const int s = it % kGvStages;
                    if (!tc::mbar_wait(&empty[s], ((it / kGvStages) & 1) ^ 1, abort)) {
                        if (err) atomicOr(err, 1);
                        *abort = 1;
                        break;
                    }
                    const int nr = min(CR, rows - c * CR);
                    const uint32_t bytes = (uint32_t)nr * nin * (uint32_t)sizeof(AT);
                    tc::mbar_expect_tx(&full[s], bytes);
                    tc::bulk_load_hint(stages + (size_t)s * kStageElems, Aop + (e * rows + c * CR) * (int64_t)nin,
                                       bytes, &full[s], pol);
                }
            }
            // let the copies in flight land before the block can exit
            for (int q = (it > kGvStages ? it - kGvStages : 0); q < it; ++q) {
                const long long t0 = clock64();
                while (!tc::mbar_try_wait(&full[q % kGvStages], (q / kGvStages) & 1) && clock64() - t0 < tc::kWaitCycles / 4) {
                }
            }
        }
        return;
    }
    // consumers.  The inflow (and the self term) of the next element are loaded into registers
    // before the chunks of the current one are processed, and published to shared memory after.
    const int ctid = threadIdx.x;  // 0 .. 32 kGvWarps - 1
    constexpr int PF = (4 * ELRT_MAX_N1 * (ELRT_MAX_ANG / 2) + 32 * kGvWarps - 1) / (32 * kGvWarps);
    V* xsv = reinterpret_cast<V*>(xs + 2 * nin);  // [2][rows] self term
    ff pin[PF];
    V pself[PF];
    // fused Arnoldi step: the input is the unnormalised slot W_j, v_j = s_j W_j
    float xsc = 1.f;
    if constexpr (std::is_same<V, float>::value)
        if (fz.as) xsc = (float)((volatile const double*)fz.as->sc)[fz.j];
    auto in_val = [&](V v) -> V {
        if constexpr (std::is_same<V, float>::value) return v * xsc;
        else return v;
    };
    auto prefetch = [&](int64_t e) {
        const int ix = (int)(e % nx), iz = (int)(e / nx);
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            const int c = ctid + u * 32 * kGvWarps;
            ff v{0.f, 0.f};
            if (c < nin) {
                const int F = c / nface, off = c - F * nface;
                const int jx = ix + (F == 1) - (F == 3), jz = iz + (F == 2) - (F == 0);
                if (jx >= 0 && jx < nx && jz >= 0 && jz < nz) {
                    if (x) v = to_ff(x[((int64_t)jz * nx + jx) * nin + ((F + 2) & 3) * nface + off]);
                } else if (g) {
                    int64_t side0;
                    int face;
                    switch (F) {
                        case 0: side0 = 0; face = ix; break;
                        case 1: side0 = (int64_t)nx * nface; face = iz; break;
                        case 2: side0 = (int64_t)(nx + nz) * nface; face = ix; break;
                        default: side0 = (int64_t)(2 * nx + nz) * nface; face = iz; break;
                    }
                    v = ff_from_double(g[side0 + (int64_t)face * nface + off]);
                }
            }
            pin[u] = v;
            if (alpha && c < rows) pself[u] = xself[e * rows + c];
        }
    };
    int it = 0, buf = 0;
    if (blockIdx.x < E) prefetch(blockIdx.x);
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x, buf ^= 1) {
        ff* xe = xs + buf * nin;
        V* se = xsv + buf * rows;
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            // (the scale of a fused Arnoldi step is applied here, after the loads have landed: the
            // prefetch itself never waits on them)
            const int c = ctid + u * 32 * kGvWarps;
            if (c < nin) {
                ff v = pin[u];
                if constexpr (std::is_same<V, float>::value) v.h *= xsc;  // fused step: no boundary data, v = (x, 0)
                xe[c] = v;
            }
            if (alpha && c < rows) se[c] = in_val(pself[u]);
        }
        asm volatile("bar.sync 1, %0;" ::"r"(32 * kGvWarps) : "memory");  // consumers only
        if (e + gridDim.x < E) prefetch(e + gridDim.x);
        for (int c = 0; c < nch; ++c, ++it) {
            const int s = it % kGvStages;
            if (!__all_sync(0xffffffffu, tc::mbar_wait(&full[s], (it / kGvStages) & 1, abort))) {
                // keep walking the loops (every later wait returns at once) so that all consumer
                // warps still meet at the per-element barrier
                if (lane == 0 && err) atomicOr(err, 2);
                *abort = 1;
                continue;
            }
            const AT* Ac = stages + (size_t)s * kStageElems + (size_t)warp * RPW * nin;
            const int rbase = c * CR + warp * RPW;
            if constexpr (std::is_same<AT, __half>::value) {
                // Arnoldi step on the FP16 copy: FP32 throughout (the copy's rounding, ~5e-4, is
                // far above FP32's).  Lanes take column pairs (2 q, 2 q + 1), even and odd columns
                // in separate chains; nin is even.
                const int np = nin >> 1;
                const __half2* A2 = reinterpret_cast<const __half2*>(Ac);
                const float4* x4 = reinterpret_cast<const float4*>(xe);  // (h, l) of two columns
                float f1[RPW], f2[RPW];
#pragma unroll
                for (int q = 0; q < RPW; ++q) f1[q] = f2[q] = 0.f;
                for (int pc = lane; pc < np; pc += 32) {
                    const float4 xv = x4[pc];
#pragma unroll
                    for (int q = 0; q < RPW; ++q) {
                        const float2 a = __half22float2(A2[q * np + pc]);
                        f1[q] = fmaf(a.x, xv.x, f1[q]);
                        f2[q] = fmaf(a.y, xv.z, f2[q]);
                    }
                }
                tc::fence_proxy_async();
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&empty[s])) : "memory");
#pragma unroll
                for (int q = 0; q < RPW; ++q) f1[q] += f2[q];
                const float sum = warp_rows_reduce_f<RPW>(f1, lane);
                constexpr int span = 32 / RPW;
                const int r = rbase + lane / span;
                if (lane % span == 0 && r < rows) {
                    float t = beta > 0 ? sum : (beta < 0 ? -sum : 0.f);
                    if (alpha) t = (alpha > 0 ? (float)se[r] : -(float)se[r]) + t;
                    y[e * rows + r] = (V)t;
                }
                continue;
            }
            ff acc[RPW];
            if constexpr (std::is_same<V, float>::value) {
                // Arnoldi step (FP32 basis vector in, FP32 vector out): each lane's partial sum of
                // its ~nin/32 products in FP32, two chains per row; the lanes' partials, the self
                // term and the final rounding in float-float
                float f1[RPW], f2[RPW];
#pragma unroll
                for (int q = 0; q < RPW; ++q) f1[q] = f2[q] = 0.f;
                int col = lane;
                for (; col + 32 < nin; col += 64) {
                    const float xv = xe[col].h, xw = xe[col + 32].h;
#pragma unroll
                    for (int q = 0; q < RPW; ++q) {
                        f1[q] = fmaf(Ac[q * nin + col], xv, f1[q]);
                        f2[q] = fmaf(Ac[q * nin + col + 32], xw, f2[q]);
                    }
                }
                if (col < nin) {
                    const float xv = xe[col].h;
#pragma unroll
                    for (int q = 0; q < RPW; ++q) f1[q] = fmaf(Ac[q * nin + col], xv, f1[q]);
                }
#pragma unroll
                for (int q = 0; q < RPW; ++q) {
                    float h, l;
                    two_sum(f1[q], f2[q], h, l);
                    acc[q] = (rbase + q < rows) ? ff{h, l} : ff{0.f, 0.f};
                }
            } else {
                // restart residual, right-hand side, recovery: float-float products and sums,
                // two independent chains per row (even / odd 32-column blocks)
                ff acc2[RPW];
#pragma unroll
                for (int q = 0; q < RPW; ++q) acc[q] = acc2[q] = ff{0.f, 0.f};
                int col = lane;
                for (; col + 32 < nin; col += 64) {
                    const ff xv = xe[col], xw = xe[col + 32];
#pragma unroll
                    for (int q = 0; q < RPW; ++q)
                        if (rbase + q < rows) {
                            ff_fma_f(acc[q], Ac[q * nin + col], xv);
                            ff_fma_f(acc2[q], Ac[q * nin + col + 32], xw);
                        }
                }
                if (col < nin) {
                    const ff xv = xe[col];
#pragma unroll
                    for (int q = 0; q < RPW; ++q)
                        if (rbase + q < rows) ff_fma_f(acc[q], Ac[q * nin + col], xv);
                }
#pragma unroll
                for (int q = 0; q < RPW; ++q)
                    acc[q] = ff_add(ff_norm(acc[q].h, acc[q].l), ff_norm(acc2[q].h, acc2[q].l));
            }
            // the stage was read through the generic proxy; the next bulk copy into it writes
            // through the async proxy
            tc::fence_proxy_async();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&empty[s])) : "memory");
            const ff sum = warp_rows_reduce<RPW>(acc, lane);
            constexpr int span = 32 / RPW;
            const int r = rbase + lane / span;
            if (lane % span == 0 && r < rows) {
                Acc sv;
                if constexpr (std::is_same<Acc, double>::value) sv = ff_to_double(sum);
                else sv = sum;
                Acc t = beta > 0 ? sv : (beta < 0 ? K::neg(sv) : K::zero());
                if (alpha) t = K::add(alpha > 0 ? K::load(se[r]) : K::neg(K::load(se[r])), t);
                y[e * rows + r] = K::store(t);
            }
        }
    }
    if constexpr (std::is_same<V, float>::value) {
        if (fz.as) {
            // first Gram-Schmidt pass on this block's output rows: W_i . w (i <= j) and w . w
            // (slot j + 1 is w itself); the rows are the block's elements, rows / 4 packs each
            asm volatile("bar.sync 1, %0;" ::"r"(32 * kGvWarps) : "memory");  // the block's rows of w are stored
            const int q4 = rows >> 2;
            const int64_t nel = (E - blockIdx.x + gridDim.x - 1) / gridDim.x;
            const int64_t np = fz.n >> 2;
            const unsigned G = gridDim.x, B = blockIdx.x;
            arn_block_dots<true>(reinterpret_cast<const float4*>(fz.Vb), np,
                                 reinterpret_cast<const float4*>(fz.Vb + (int64_t)(fz.j + 1) * fz.n), fz.j + 2,
                                 nel * q4,
                                 [=](int64_t t) {
                                     const int64_t k = t / q4;
                                     return (int64_t)(B + k * G) * q4 + (t - k * q4);
                                 },
                                 fz.P, G);
            if (arn_last_block<true>(&fz.as->ticket[0])) arn_first_pass_finish<true>(fz.P, G, fz.j, fz.as);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Krylov kernels
// ------------------------------------------------------------------------------------------------

template <typename Acc, typename K>
__device__ __forceinline__ double block_sum_to_double(Acc v, Acc* red) {
    v = K::shfl_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += K::to_d(red[w]);
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

// 16 bytes of consecutive vector entries (the Krylov length is a multiple of 4, every vector starts
// on a 16-byte boundary)
template <typename V>
struct alignas(16) Pack16 {
    static constexpr int P = 16 / sizeof(V);
    V v[P];
};

// partial[i * nblk + blk] = sum over this block's slice of V[i] . w   (grid: nblk x nvec)
template <typename V>
__global__ void __launch_bounds__(kThreads) k_dots(const V* __restrict__ Vb, int64_t n, const V* __restrict__ w,
                                                   double* __restrict__ partial, const GmState* __restrict__ st) {
    if (st && st->done) return;
    using K = KV<V>;
    using Acc = typename K::acc;
    using Pk = Pack16<V>;
    constexpr int P = Pk::P;
    __shared__ Acc red[kThreads / 32];
    const int i = blockIdx.y;
    const Pk* v = reinterpret_cast<const Pk*>(Vb + (int64_t)i * n);
    const Pk* wp = reinterpret_cast<const Pk*>(w);
    const int64_t np = n / P;
    Acc sa[2] = {K::zero(), K::zero()};
    for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < np; k += (int64_t)gridDim.x * kThreads) {
        const Pk a = v[k], b = wp[k];
#pragma unroll
        for (int q = 0; q < P; ++q) K::fma_vv(sa[q & 1], a.v[q], b.v[q]);
    }
    const double tot = block_sum_to_double<Acc, K>(K::add(sa[0], sa[1]), red);
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
    using K = KV<V>;
    using Acc = typename K::acc;
    using Pk = Pack16<V>;
    constexpr int P = Pk::P;
    __shared__ Acc hs[kMaxRestart + 1];
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) hs[i] = K::coef(sign < 0 ? -h[i] : h[i]);
    __syncthreads();
    const Pk* vb = reinterpret_cast<const Pk*>(Vb);
    Pk* wp = reinterpret_cast<Pk*>(w);
    const int64_t np = n / P;
    for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < np; k += (int64_t)gridDim.x * kThreads) {
        Pk wv = wp[k];
        Acc s[P];
#pragma unroll
        for (int q = 0; q < P; ++q) s[q] = K::load(wv.v[q]);
#pragma unroll 4
        for (int i = 0; i < nvec; ++i) {
            const Pk a = vb[(int64_t)i * np + k];
#pragma unroll
            for (int q = 0; q < P; ++q) K::fma_cv(s[q], hs[i], a.v[q]);
        }
#pragma unroll
        for (int q = 0; q < P; ++q) wv.v[q] = K::store(s[q]);
        wp[k] = wv;
    }
}

// out = in / *d (skipped when *d == 0: lucky breakdown); in and out may be the same vector or of
// two types with one accumulator type (the float-float residual scaled into the FP32 basis)
template <typename VI, typename VO>
__global__ void k_scale(const VI* in, VO* out, int64_t n, const double* __restrict__ d,
                        const GmState* __restrict__ st) {
    static_assert(std::is_same<typename KV<VI>::acc, typename KV<VO>::acc>::value, "one accumulator type");
    if (st && st->done) return;
    const double dv = *d;
    if (dv == 0.0) return;
    const auto inv = KV<VI>::coef(1.0 / dv);
    for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads)
        out[k] = KV<VO>::store(KV<VI>::mul(KV<VI>::load(in[k]), inv));
    // (element-wise: the in-place case needs no ordering beyond each thread's own entries)
}

// r = b - r
template <typename V>
__global__ void k_bminus(const V* __restrict__ b, V* __restrict__ r, int64_t n) {
    using K = KV<V>;
    for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads)
        r[k] = K::store(K::add(K::load(b[k]), K::neg(K::load(r[k]))));
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

__global__ void __launch_bounds__(kArnThreads) k_arn_axdots(float* __restrict__ Vb, int64_t n, int j,
                                                            double* __restrict__ P, ArnState* __restrict__ as,
                                                            const GmState* __restrict__ st) {
    if (st->done) return;
    int64_t np, p0, p1;
    arn_slice(n, np, p0, p1);
    const int nv = j + 1;
    const bool reorth = ((volatile const int*)&as->reorth)[0] != 0;
    const float4* V4 = reinterpret_cast<const float4*>(Vb);
    float4* w4 = reinterpret_cast<float4*>(Vb + (int64_t)nv * n);
    arn_axpy(V4, np, w4, nv, as->h1, as->sc, p0, p1);
    __syncthreads();  // the block's slice of w is final (each thread reads only its own packs)
    if (reorth) {
        arn_block_dots<false>(V4, np, w4, nv, p1 - p0, [=](int64_t t) { return p0 + t; }, P, gridDim.x);
        if (arn_last_block(&as->ticket[1])) arn_finish(P, gridDim.x, nv, as->h2, &as->ticket[1], as->sc, nv);
    } else {
        arn_block_norm(w4, p0, p1, P);
        if (arn_last_block(&as->ticket[1])) {
            __shared__ double nrm2;
            arn_finish(P, gridDim.x, 1, &nrm2, &as->ticket[1], nullptr, 0);
            __syncthreads();
            if (threadIdx.x == 0) as->nrm = sqrt(nrm2);
        }
    }
}

__global__ void __launch_bounds__(kArnThreads) k_arn_axnorm(float* __restrict__ Vb, int64_t n, int j,
                                                            double* __restrict__ P, ArnState* __restrict__ as,
                                                            double* __restrict__ H, int ldh, double* __restrict__ cs,
                                                            double* __restrict__ sn, double* __restrict__ gv,
                                                            GmState* __restrict__ st) {
    if (st->done) return;
    if (!((volatile const int*)&as->reorth)[0]) {  // single pass: the column and the rotation only
        if (blockIdx.x == 0 && threadIdx.x < 32) arn_column(as, j, __ldcg(&as->nrm), H, ldh, cs, sn, gv, st);
        return;
    }
    int64_t np, p0, p1;
    arn_slice(n, np, p0, p1);
    const int nv = j + 1;
    const float4* V4 = reinterpret_cast<const float4*>(Vb);
    float4* w4 = reinterpret_cast<float4*>(Vb + (int64_t)nv * n);
    arn_axpy(V4, np, w4, nv, as->h2, as->sc, p0, p1);
    __syncthreads();
    arn_block_norm(w4, p0, p1, P);
    if (!arn_last_block(&as->ticket[2])) return;
    __shared__ double nrm2;
    arn_finish(P, gridDim.x, 1, &nrm2, &as->ticket[2], nullptr, 0);
    __syncthreads();
    if (threadIdx.x < 32) {
        const double nrm = sqrt(nrm2);
        if (threadIdx.x == 0) as->nrm = nrm;
        arn_column(as, j, nrm, H, ldh, cs, sn, gv, st);
    }
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

// x += sum_{i < j_done} y_i s_i W_i (x of type X, basis of type V, one accumulator type; sc NULL:
// s_i = 1)
template <typename V, typename X>
__global__ void __launch_bounds__(kThreads) k_update_x(const V* __restrict__ Vb, int64_t n,
                                                       const double* __restrict__ y, const double* __restrict__ sc,
                                                       X* __restrict__ x, const GmState* __restrict__ st) {
    using Acc = typename KV<X>::acc;
    static_assert(std::is_same<Acc, typename KV<V>::acc>::value, "one accumulator type");
    __shared__ Acc ys[kMaxRestart + 1];
    const int nj = st->j_done;
    for (int i = threadIdx.x; i < nj; i += blockDim.x) ys[i] = KV<X>::coef(sc ? y[i] * sc[i] : y[i]);
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads) {
        Acc s = KV<X>::load(x[k]);
#pragma unroll 4
        for (int i = 0; i < nj; ++i) KV<V>::fma_cv(s, ys[i], Vb[(int64_t)i * n + k]);
        x[k] = KV<X>::store(s);
    }
}

// x += t (the preconditioned correction of a cycle), in the iterate's arithmetic
template <typename X>
__global__ void __launch_bounds__(kThreads) k_add_f(X* __restrict__ x, const float* __restrict__ t, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads) {
        typename KV<X>::acc s = KV<X>::load(x[k]);
        KV<float>::fma_cv(s, KV<X>::coef(1.0), t[k]);
        x[k] = KV<X>::store(s);
    }
}

// Start of a restart cycle.  A restart residual at or below the tolerance (or not finite) ends the
// solve on the device: the cycle's kernels see done and do nothing, and j_done stays 0.
__global__ void k_cycle_start(GmState* st, double* gv, int m, const double* beta, double* sc0) {
    if (sc0) *sc0 = 1.0;
    const double b = *beta;
    st->done = (b > st->tol && isfinite(b)) ? 0 : 1;
    st->j_done = 0;
    st->beta = b;
    st->res = b;
    gv[0] = b;
    for (int i = 1; i <= m; ++i) gv[i] = 0.0;
}

// ------------------------------------------------------------------------------------------------
// Arnoldi-step matvec on the tensor cores (FP16 copy of the operator): w = v - A v, v = s_j W_j.
// The operators of all elements form one flat FP16 matrix [E rows][nin]; a persistent CTA walks its
// 128-row tiles, which cross element boundaries (at most 5 elements per tile for nin >= 32).  Per
// tile:
//   A  the tile's rows, nin columns zero-padded to kTcKc boxes of 64 (TMA, 128-byte swizzle);
//   B  N = 16 columns: for the k-th element the tile touches, its gathered inflow v_in scaled by
//      2^12 and split into FP16 high part (column 2k) and FP16 remainder (column 2k + 1);
//   D  = A B in FP32 (tensor memory, 128 lanes x 16 columns, double-buffered), so that row r of the
//      k-th element reads (D[r][2k] + D[r][2k + 1]) 2^-12 = (A v_in)_r with v to ~2^-22 and the
//      operator to its FP16 rounding.
// Roles: warps 0-3 epilogue (TMEM lane quarter = warp, one thread per tile row: w = v - A v);
// warps 4-11 build B (one column each); warp 12 TMA producer; warp 13 TMEM allocation and MMA
// issue.  After the tiles, warps 0-7 run the fused first Gram-Schmidt pass over the CTA's rows (as
// the streaming kernel).
// Every wait is bounded; on a timeout the CTA records a code in *err and winds down.
// ------------------------------------------------------------------------------------------------
constexpr int kTcKc = 4;                       // K boxes of 64 columns: nin <= 256
constexpr int kTcStages = 3;
constexpr int kTcA = 128 * 64 * 2;             // one A box (16 KB)
constexpr int kTcB = 16 * 64 * 2;              // one B box (2 KB)
constexpr int kTcStage = kTcKc * (kTcA + kTcB);
constexpr int kTcThreads = 448;
constexpr int kTcSmem = kTcStages * kTcStage + 1024;
constexpr float kTcScale = 4096.f;             // 2^12: keeps the FP16 remainder of |v| <= 1 normal

__device__ __forceinline__ void tma_load_2d_hint(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y,
                                                 uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(
            tc::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(tc::smem_u32(bar)), "r"(x), "r"(y), "l"(pol)
        : "memory");
}

__device__ __forceinline__ uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);  // FP32 D, FP16 A and B
}

// byte offset of element (n, c) of a K-major 128-byte-swizzled B tile of 16 rows (boxes of 64 columns)
__device__ __forceinline__ uint32_t b_off(int n, int c) {
    const int kc = c >> 6, byte = (c & 63) * 2;
    return (uint32_t)(kc * kTcB + (n >> 3) * 1024 + (n & 7) * 128 + ((((byte >> 4) ^ (n & 7))) << 4) + (byte & 15));
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_gemv_tc(const __grid_constant__ CUtensorMap tA, int nx, int nz, int nin, int nface,
              const float* __restrict__ x, float* __restrict__ y, const GmState* __restrict__ st,
              int* __restrict__ err, ArnFuse fz) {
    if (st && st->done) return;
    extern __shared__ __align__(1024) unsigned char tsm_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)tsm_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full[kTcStages], bready[kTcStages], empty[kTcStages], acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    volatile int* abort = &abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t E = (int64_t)nx * nz, NR = E * nin;
    const int64_t T = (NR + 127) / 128;
    const int nkc = (nin + 63) >> 6;
    const float xsc = (float)((volatile const double*)fz.as->sc)[fz.j];
    // zero the B tiles once: padding columns and unused rows stay zero
    for (int i = threadIdx.x; i < kTcStages * kTcKc * kTcB / 16; i += kTcThreads) {
        const int s = i / (kTcKc * kTcB / 16), o = i - s * (kTcKc * kTcB / 16);
        reinterpret_cast<uint4*>(base + s * kTcStage + kTcKc * kTcA)[o] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < kTcStages; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&bready[i], 8);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&acc_full[i], 1);
            tc::mbar_init(&acc_empty[i], 4);
        }
        *abort = 0;
        tc::fence_barrier_init();
    }
    tc::fence_proxy_async();  // the zeroed B tiles are read by the tensor cores
    if (warp == 13) {
        tc::tmem_alloc(&tmem_slot, 32);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_slot;
    int issued = 0, committed = 0;
    if (warp == 12) {  // TMA producer
        if (lane == 0) {
            const uint64_t pol = tc::l2_evict_first();  // read once; the Krylov vectors stay in L2
            int g = 0;
            for (int64_t t = blockIdx.x; t < T; t += gridDim.x, ++g) {
                const int s = g % kTcStages;
                if (!tc::mbar_wait(&empty[s], ((g / kTcStages) & 1) ^ 1, abort)) {
                    if (err) atomicOr(err, 4);
                    *abort = 1;
                    break;
                }
                unsigned char* As = base + s * kTcStage;
                tc::mbar_expect_tx(&full[s], (uint32_t)(nkc * kTcA));
                for (int kc = 0; kc < nkc; ++kc) tma_load_2d_hint(&tA, &full[s], As + kc * kTcA, kc * 64, (int)(t * 128), pol);
                ++issued;
            }
        }
    } else if (warp == 13) {  // MMA issue
        if (lane == 0) {
            const uint32_t idesc = idesc_f16(128, 16);
            int g = 0;
            for (int64_t t = blockIdx.x; t < T; t += gridDim.x, ++g) {
                const int s = g % kTcStages, a = g & 1;
                if (!tc::mbar_wait(&acc_empty[a], ((g >> 1) & 1) ^ 1, abort) ||
                    !tc::mbar_wait(&full[s], (g / kTcStages) & 1, abort) ||
                    !tc::mbar_wait(&bready[s], (g / kTcStages) & 1, abort)) {
                    if (err) atomicOr(err, 8);
                    *abort = 1;
                    break;
                }
                tc::tc_fence_after();
                unsigned char* As = base + s * kTcStage;
                unsigned char* Bs = As + kTcKc * kTcA;
                uint32_t acc = 0;
                for (int kc = 0; kc < nkc; ++kc) {
                    const uint64_t ad = tc::sw128_desc(tc::smem_u32(As + kc * kTcA));
                    const uint64_t bd = tc::sw128_desc(tc::smem_u32(Bs + kc * kTcB));
#pragma unroll
                    for (int k = 0; k < 4; ++k) {  // K = 16 per instruction
                        tc::mma_bf16(tmem + (uint32_t)(a * 16), ad + 2 * k, bd + 2 * k, idesc, acc);
                        acc = 1;
                    }
                }
                tc::mma_commit(&empty[s]);
                tc::mma_commit(&acc_full[a]);
                ++committed;
            }
        }
    } else if (warp >= 4) {  // B builders: gathered inflow of the tile's elements, split in FP16
        // A tile touches at most 127 / nin + 2 <= 5 elements (nin >= 32); builder thread c owns
        // column c of each (nin <= 256), whose face and source offset in the neighbour's outflow
        // block are fixed.  The next tile's values are loaded while this one waits.
        constexpr int kMaxE = 5;
        const int c = threadIdx.x - 128;
        const int cF = c < nin ? c / nface : -1;
        const int csrc = ((cF + 2) & 3) * nface + (c - (c / nface) * nface);
        // (loads are unconditional, from x[0] where there is no value, so that nothing waits on
        // them here; the validity mask is applied when the tile is built)
        auto gather = [&](int t, float (&pv)[kMaxE], unsigned& mask) {
            const int ea = t * 128 / nin, eb = min((int)E - 1, (t * 128 + 127) / nin);
            mask = 0u;
#pragma unroll
            for (int k = 0; k < kMaxE; ++k) {
                const int e = ea + k;
                const int iz = e / nx, ix = e - iz * nx;
                const int jx = ix + (cF == 1) - (cF == 3), jz = iz + (cF == 2) - (cF == 0);
                const bool ok = e <= eb && cF >= 0 && jx >= 0 && jx < nx && jz >= 0 && jz < nz;
                mask |= (ok ? 1u : 0u) << k;
                pv[k] = x[ok ? (jz * nx + jx) * nin + csrc : 0];
            }
        };
        // write tile t's B into its stage; false on a timeout
        auto build = [&](int t, int g, const float (&pv)[kMaxE], unsigned mask) -> bool {
            const int s = g % kTcStages;
            if (!__all_sync(0xffffffffu, tc::mbar_wait(&empty[s], ((g / kTcStages) & 1) ^ 1, abort) && !*abort)) {
                if (err && lane == 0) atomicOr(err, 16);
                *abort = 1;
                return false;
            }
            unsigned char* Bs = base + s * kTcStage + kTcKc * kTcA;
            const int nel = min((int)E - 1, (t * 128 + 127) / nin) - t * 128 / nin + 1;
#pragma unroll
            for (int k = 0; k < kMaxE; ++k)
                if (k < nel && cF >= 0) {
                    const float v = ((mask >> k) & 1u) ? pv[k] * xsc * kTcScale : 0.f;
                    const __half hi = __float2half_rn(v);
                    const __half lo = __float2half_rn(v - __half2float(hi));
                    *reinterpret_cast<__half*>(Bs + b_off(2 * k, c)) = hi;
                    *reinterpret_cast<__half*>(Bs + b_off(2 * k + 1, c)) = lo;
                }
            tc::fence_proxy_async();  // generic-proxy writes read next by the tensor cores
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&bready[s])) : "memory");
            return true;
        };
        // two register sets: the loads of a tile are issued two tiles before it is built
        float pa[kMaxE], pb[kMaxE];
        unsigned ma = 0u, mb = 0u;
        const int G = gridDim.x, T32 = (int)T;
        if ((int)blockIdx.x < T32) gather(blockIdx.x, pa, ma);
        if ((int)blockIdx.x + G < T32) gather(blockIdx.x + G, pb, mb);
        int g = 0;
        for (int t = blockIdx.x; t < T32; t += 2 * G, g += 2) {
            if (!build(t, g, pa, ma)) break;
            if (t + 2 * G < T32) gather(t + 2 * G, pa, ma);
            if (t + G >= T32) break;
            if (!build(t + G, g + 1, pb, mb)) break;
            if (t + 3 * G < T32) gather(t + 3 * G, pb, mb);
        }
    } else {  // epilogue: row r of the tile
        const int r = warp * 32 + lane;
        int g = 0;
        for (int64_t t = blockIdx.x; t < T; t += gridDim.x, ++g) {
            const int a = g & 1;
            const int64_t R = t * 128 + r;
            const float xs = R < NR ? x[R] : 0.f;  // the self term, loaded before the wait
            if (!__all_sync(0xffffffffu, tc::mbar_wait(&acc_full[a], (g >> 1) & 1, abort) && !*abort)) {
                if (err && lane == 0) atomicOr(err, 32);
                *abort = 1;
                break;
            }
            tc::tc_fence_after();
            float v[16];
            tc::tmem_ld16(tmem + (uint32_t)(a * 16) + ((uint32_t)(warp * 32) << 16), v);
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&acc_empty[a])) : "memory");
            if (R < NR) {
                const int k = (int)R / nin - (int)(t * 128) / nin;
                float ax = 0.f;
#pragma unroll
                for (int kk = 0; kk < 5; ++kk)
                    if (kk == k) ax = v[2 * kk] + v[2 * kk + 1];
                y[R] = xsc * xs - ax * (1.f / kTcScale);
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 12 && lane == 0) {  // after a timeout: let the copies in flight land before the CTA exits
        for (int q = (issued > kTcStages ? issued - kTcStages : 0); q < issued; ++q) {
            const long long t1 = clock64();
            while (!tc::mbar_try_wait(&full[q % kTcStages], (q / kTcStages) & 1) && clock64() - t1 < tc::kWaitCycles / 4) {
            }
        }
    }
    if (warp == 13) {
        if (lane == 0 && committed > 0) {  // never free TMEM under an MMA in flight
            const int last = committed - 1;
            const long long t0 = clock64();
            while (!tc::mbar_try_wait(&acc_full[last & 1], (last >> 1) & 1) && clock64() - t0 < tc::kWaitCycles) {
            }
        }
        __syncwarp();
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 32);
    }
    if (warp < 8) {
        // first Gram-Schmidt pass on this CTA's rows (its tiles, 32 packs each; the last tile of the
        // matrix may be shorter): W_i . w (i <= j) and w . w
        const int64_t np = fz.n >> 2;
        const unsigned G = gridDim.x, B = blockIdx.x;
        const int64_t ntb = (T - B + G - 1) / G;
        const bool owns_last = (T - 1) % G == B;
        const int64_t cnt = ntb * 32 - (owns_last ? (T * 32 - np) : 0);
        arn_block_dots<true>(reinterpret_cast<const float4*>(fz.Vb), np,
                             reinterpret_cast<const float4*>(fz.Vb + (int64_t)(fz.j + 1) * fz.n), fz.j + 2, cnt,
                             [=](int64_t i) {
                                 const int64_t k = i >> 5;
                                 return (int64_t)(B + k * G) * 32 + (i & 31);
                             },
                             fz.P, G);
        if (arn_last_block<true>(&fz.as->ticket[0])) arn_first_pass_finish<true>(fz.P, G, fz.j, fz.as);
    }
}

// ---- host side of the tensor-core matvec
PFN_cuTensorMapEncodeTiled_v12000 g_enc16 = nullptr;
std::once_flag g_enc16_once;

bool enc16_ready() {
    std::call_once(g_enc16_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_enc16 = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    return g_enc16 != nullptr;
}

// the tensor-core matvec serves this element size (tiles touch at most 5 elements, K fits kTcKc boxes)
bool gemv_tc_ok(const Tab& t) { return t.nin >= 32 && t.nin <= 64 * kTcKc && t.nin % 8 == 0; }

// the FP16 operator copy as a flat [rows][nin] matrix, boxes of 64 columns x 128 rows, 128-byte
// swizzle (columns beyond nin and rows beyond the end read as zero)
bool map_op16(CUtensorMap* m, const __half* A, int64_t rows, int nin) {
    if (((uintptr_t)A & 15) || (nin * 2) % 16 || !enc16_ready()) return false;
    cuuint64_t dims[2] = {(cuuint64_t)nin, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)nin * 2};
    cuuint32_t box[2] = {64, 128};
    cuuint32_t es[2] = {1, 1};
    return g_enc16(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (void*)A, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

elrt_status launch_gemv_tc(elrt_ctx* ctx, const CUtensorMap& map, int nx, int nz, const float* x, float* y,
                           const GmState* st, const ArnFuse& fz) {
    const Tab& t = ctx->tab;
    const int64_t E = (int64_t)nx * nz, T = (E * t.nin + 127) / 128;
    // algorithmic bytes: the FP16 operator once, the gathered inflow and the self term, the result,
    // and the fused pass's basis slots 0 .. j and w once more
    const double bytes = (double)E * t.nin * ((double)t.nin * 2 + 12.0) + (double)(fz.j + 2) * fz.n * sizeof(float);
    ProfScope ps(ctx, "gemv", 1, bytes, 2.0 * (double)E * t.nin * t.nin);
    cudaError_t ce = cudaFuncSetAttribute(k_gemv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (ce != cudaSuccess) return cuda_check(ctx, ce, "smem attribute");
    const unsigned grid = (unsigned)std::min<int64_t>(T, ctx->sms);
    k_gemv_tc<<<grid, kTcThreads, kTcSmem, ctx->stream>>>(map, nx, nz, t.nin, t.nface, x, y, st,
                                                         ctx->d_flags + kGemvFlag, fz);
    return cuda_check(ctx, cudaGetLastError(), "tensor-core matvec launch");
}

template <typename V, int RPW, typename AT>
cudaError_t launch_stream(elrt_ctx* ctx, unsigned grid, size_t smem, int nx, int nz, int rows, const AT* Aop,
                          const V* x, const double* g, const V* xself, int alpha, int beta, V* y, const GmState* st,
                          const ArnFuse& fz) {
    const Tab& t = ctx->tab;
    cudaError_t ce = cudaFuncSetAttribute(k_gemv_stream<V, RPW, AT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) return ce;
    k_gemv_stream<V, RPW, AT><<<grid, kGvThreads, smem, ctx->stream>>>(nx, nz, t.nin, t.nface, rows, Aop, x, g, xself,
                                                                     alpha, beta, y, st, ctx->d_flags + kGemvFlag, fz);
    return cudaGetLastError();
}

// the streaming kernel serves operators of element size es at this address
bool gemv_streams(const Tab& t, const void* Aop, int es) {
    return ((uintptr_t)Aop & 15) == 0 && (t.nin * es) % 16 == 0 && t.nin * es * 8 <= kGvStageBytes;
}

// A: float or double (operators as given), or __half (the FP16 copy, FP32 vectors only).  fz: fused
// first Gram-Schmidt pass (streaming kernel, FP32 vectors; the caller checks gemv_streams).
template <typename A, typename V>
elrt_status launch_gemv(elrt_ctx* ctx, int nx, int nz, int rows, const void* Aop, const V* x, const double* g,
                        const V* xself, int alpha, int beta, V* y, const GmState* st, ArnFuse fz = ArnFuse{}) {
    const Tab& t = ctx->tab;
    const int64_t E = (int64_t)nx * nz;
    if (E > 0x7fffffffLL) return ctx_fail(ctx, ELRT_EINVAL, "too many elements");
    // algorithmic bytes: the operators once, the gathered inflow (x or g), the self term, the result,
    // and for the fused pass the basis slots 0 .. j and w once more
    const double bytes = (double)E * ((double)rows * t.nin * sizeof(A) + (x ? (double)t.nin * sizeof(V) : 0.0) +
                                      (g ? 8.0 * t.nin : 0.0) + (xself && beta ? (double)rows * sizeof(V) : 0.0) +
                                      (double)rows * sizeof(V)) +
                         (fz.as ? (double)(fz.j + 2) * fz.n * sizeof(float) : 0.0);
    ProfScope ps(ctx, "gemv", 1, bytes, 2.0 * (double)E * rows * t.nin);
    if constexpr (sizeof(A) <= 4) {
        // streaming kernel: 16-byte aligned row chunks (nin % 8 == 0 holds for every valid disc)
        constexpr int es = (int)sizeof(A);
        int rpw = t.nin * es * 32 <= kGvStageBytes ? 4 : (t.nin * es * 16 <= kGvStageBytes ? 2 : 1);
        if (sizeof(A) == 2 && t.nin * es * 64 <= kGvStageBytes) rpw = 8;
        if (gemv_streams(t, Aop, es)) {
            const size_t smem = (size_t)kGvStages * kGvStageBytes + 2 * (size_t)t.nin * sizeof(ff) +
                                2 * (size_t)rows * sizeof(V);
            const unsigned grid = (unsigned)std::min<int64_t>(E, 2 * ctx->sms);
            const A* Ap = (const A*)Aop;
            cudaError_t ce;
            if constexpr (sizeof(A) == 2) {
                if (rpw == 8) {
                    ce = launch_stream<V, 8, A>(ctx, grid, smem, nx, nz, rows, Ap, x, g, xself, alpha, beta, y, st, fz);
                    return cuda_check(ctx, ce, "gemv launch");
                }
            }
            if (rpw == 4) ce = launch_stream<V, 4, A>(ctx, grid, smem, nx, nz, rows, Ap, x, g, xself, alpha, beta, y, st, fz);
            else if (rpw == 2) ce = launch_stream<V, 2, A>(ctx, grid, smem, nx, nz, rows, Ap, x, g, xself, alpha, beta, y, st, fz);
            else ce = launch_stream<V, 1, A>(ctx, grid, smem, nx, nz, rows, Ap, x, g, xself, alpha, beta, y, st, fz);
            return cuda_check(ctx, ce, "gemv launch");
        }
        if constexpr (sizeof(A) == 2) return ctx_fail(ctx, ELRT_EINVAL, "FP16 operator copy not 16-byte aligned");
    }
    if (fz.as) return ctx_fail(ctx, ELRT_EINVAL, "fused Arnoldi pass needs the streaming matvec");
    if constexpr (sizeof(A) != 2) {
        k_elem_gemv<A, V><<<(unsigned)E, kThreads, 0, ctx->stream>>>(nx, nz, t.nin, t.nface, rows, (const A*)Aop, x,
                                                                     g, xself, alpha, beta, y, st);
        return cuda_check(ctx, cudaGetLastError(), "gemv launch");
    }
}

// FP16 copy of an FP32 operator (n4 groups of four entries) for the Arnoldi-step matvecs; *err is
// set when an entry is not finite or lies beyond +-6e4 (the FP16 range ends at 65504)
__global__ void __launch_bounds__(kThreads) k_op_to_f16(const float4* __restrict__ src, uint2* __restrict__ dst,
                                                        int64_t n4, int* __restrict__ err) {
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n4; i += (int64_t)gridDim.x * kThreads) {
        const float4 v = __ldcs(src + i);
        bad |= !(fabsf(v.x) <= 6e4f) || !(fabsf(v.y) <= 6e4f) || !(fabsf(v.z) <= 6e4f) || !(fabsf(v.w) <= 6e4f);
        const __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
        uint2 o;
        o.x = *reinterpret_cast<const uint32_t*>(&a);
        o.y = *reinterpret_cast<const uint32_t*>(&b);
        __stcs(dst + i, o);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, 1);
}

unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(4 * 152, (n + kThreads - 1) / kThreads)); }

// GMRES with operators of type A, Krylov basis of type V and iterate / right-hand side / restart
// residual of type X.  FP64 operators: V = X = double.  FP32 operators: V = float, X = float-float:
// the basis only has to span the Krylov space to FP32 accuracy, while every restart recomputes the
// true residual b - (I - A_int) x in float-float, so the restarts refine the solution to the
// float-float level (all inner products and norms accumulate in float-float, reduced in FP64).
template <typename A, typename V, typename X>
elrt_status gmres(elrt_ctx* ctx, int nx, int nz, const void* Aop, const double* inflow, double rtol, int max_iter,
                  int restart, int use_guess, double* xout, elrt_solve_stats* stats, const double* f2o) {
    const Tab& t = ctx->tab;
    const int64_t n = (int64_t)nx * nz * t.nin;
    const int m = std::max(1, std::min(restart, kMaxRestart));
    const int nblk = kDotBlocks;
    constexpr bool own_x = !std::is_same<X, double>::value;  // float-float iterate kept apart from the output
    constexpr bool own_r = !std::is_same<X, V>::value;       // restart residual in X, basis in V
    // workspace: basis V[(m+1) n], then b[n], x[n] (float-float only), r[n] (when V != X) of type X,
    // then the FP64 small arrays and the state
    const size_t vb_bytes = ((size_t)(m + 1) * n * sizeof(V) + 255) & ~(size_t)255;
    const size_t xbytes = (size_t)n * sizeof(X) * (1 + (own_x ? 1 : 0) + (own_r ? 1 : 0));
    // FP64 small arrays: H, cs, sn, gv, yv, the per-block partials, then the Arnoldi-step state
    const size_t small = ((size_t)(m + 1) * m + 4 * (size_t)(m + 1) + (size_t)(m + 1) * nblk + 128) * sizeof(double) +
                         sizeof(ArnState);
    // sweep preconditioner (FP32 basis): M v_j and the cycle's correction [n] FP32 each, the
    // sweeps' versioned outflow [n] (8 bytes each), the item order [4 E] and two flags
    const int64_t E = (int64_t)nx * nz;
    const bool pc = std::is_same<V, float>::value && ctx->precond == ELRT_PRECOND_SWEEP;
    const size_t pc_words = pc ? ((sweep_words_bytes(t, E) + 255) & ~(size_t)255) : 0;
    const size_t pc_bytes =
        pc ? (((size_t)2 * n * sizeof(float) + 256 + pc_words + (size_t)4 * E * sizeof(int) + 64 + 255) & ~(size_t)255) : 0;
    elrt_status s = ensure_ws(ctx, &ctx->gm, &ctx->gm_bytes, vb_bytes + xbytes + 256 + small + sizeof(GmState) + 512 + pc_bytes);
    if (s) return s;
    V* Vb = (V*)ctx->gm;
    X* b = (X*)((unsigned char*)ctx->gm + vb_bytes);
    X* x = own_x ? b + n : (X*)xout;
    X* r = own_r ? (own_x ? b + 2 * n : b + n) : (X*)Vb;
    double* H = (double*)((unsigned char*)ctx->gm + ((vb_bytes + xbytes + 255) & ~(size_t)255));
    double* cs = H + (size_t)(m + 1) * m;
    double* sn = cs + (m + 1);
    double* gv = sn + (m + 1);
    double* yv = gv + (m + 1);
    double* partial = yv + (m + 1);
    ArnState* arn = (ArnState*)(partial + (size_t)(m + 1) * nblk);
    double* scal = (double*)(arn + 1) + 8;  // [0] ||b||, [1] beta
    GmState* st = (GmState*)(scal + 64);
    float* pc_t = pc ? (float*)(((uintptr_t)(st + 1) + 255) & ~(uintptr_t)255) : nullptr;  // M v_j, M u
    float* pc_u = pc ? pc_t + n : nullptr;                                                 // sum y_i s_i W_i
    void* pc_zw = pc ? (void*)(((uintptr_t)(pc_u + n) + 255) & ~(uintptr_t)255) : nullptr;  // sweep_words_bytes
    int* pc_order = pc ? (int*)((unsigned char*)pc_zw + pc_words) : nullptr;
    int* pc_flags = pc ? pc_order + 4 * E : nullptr;
    // three-launch Arnoldi step: FP32 basis, restarts up to kArnMaxV - 1 and the streaming matvec
    const bool arn4 = std::is_same<V, float>::value && m + 1 <= kArnMaxV && gemv_streams(t, Aop, (int)sizeof(A));
    cudaStream_t sm = ctx->stream;
    const unsigned gb = grid_for(n);
    // algorithmic bytes of a pass that touches nvec vectors of type T once each
    auto kv = [](int nvec, int64_t len, size_t tsize) { return (double)nvec * len * tsize; };
    GmState* hst = (GmState*)ctx->h_pinned;
    const int rows = t.nin;

    if (pc) {
        std::vector<int> ord((size_t)4 * E);
        sweep_orders(nx, nz, ord.data());
        s = cuda_check(ctx, cudaMemcpyAsync(pc_order, ord.data(), ord.size() * sizeof(int), cudaMemcpyHostToDevice, sm),
                       "sweep orders");
        if (!s) s = cuda_check(ctx, cudaStreamSynchronize(sm), "sweep orders");  // (pageable source)
        if (s) return s;
    }
    s = cuda_check(ctx, cudaMemsetAsync(ctx->d_flags + kGemvFlag, 0, 2 * sizeof(int), sm), "clear flags");
    if (!s) s = cuda_check(ctx, cudaMemsetAsync(arn, 0, sizeof(ArnState), sm), "clear Arnoldi state");
    if (s) return s;
    // FP16 copy of the operator for the Arnoldi steps (FP32 operators, unless switched off): the
    // basis is built with it, while b and every restart residual use the operator itself, so the
    // restarts refine the iterate to the solution of the FP32 system (GMRES as the inner solver of
    // a mixed-precision iterative refinement)
    bool use16 = false;
    const __half* A16 = nullptr;
    if constexpr (std::is_same<V, float>::value) {
        const int64_t nop = (int64_t)nx * nz * rows * t.nin;
        if (ctx->krylov_op == ELRT_KRYLOV_F16 && nop % 4 == 0 && ((uintptr_t)Aop & 15) == 0) {
            s = ensure_ws(ctx, &ctx->gm16, &ctx->gm16_bytes, (size_t)nop * sizeof(__half));
            if (s) return s;
            A16 = (const __half*)ctx->gm16;
            ProfScope ps(ctx, "gemv", 1, 6.0 * nop);
            k_op_to_f16<<<4 * ctx->sms, kThreads, 0, sm>>>((const float4*)Aop, (uint2*)ctx->gm16, nop / 4,
                                                      ctx->d_flags + kF16Flag);
            use16 = true;
        }
    }
    // b = A g_bnd (+ f^_u: the source term of eq. hdg_global_mat, converted to X first)
    const X* fsrc = nullptr;
    if (f2o) {
        if constexpr (std::is_same<X, double>::value) {
            fsrc = f2o;
        } else {
            ProfScope ps(ctx, "krylov", 1, 16.0 * n);
            k_d2ff<<<gb, kThreads, 0, sm>>>(f2o, r, n);
            fsrc = r;
        }
    }
    s = launch_gemv<A, X>(ctx, nx, nz, rows, Aop, nullptr, inflow, fsrc, fsrc ? 1 : 0, 1, b, nullptr);
    if (s) return s;
    { ProfScope ps(ctx, "krylov", 1, kv(1, n, sizeof(X))); k_dots<X><<<dim3(nblk, 1), kThreads, 0, sm>>>(b, n, b, partial, nullptr); }
    { ProfScope ps(ctx, "krylov"); k_dots_finish<<<1, kThreads, 0, sm>>>(partial, nblk, scal, 2, nullptr); }
    if (!use_guess) {
        s = cuda_check(ctx, cudaMemsetAsync(x, 0, n * sizeof(X), sm), "zero x");
        if (s) return s;
    } else if constexpr (own_x) {
        ProfScope ps(ctx, "krylov", 1, 16.0 * n);
        k_d2ff<<<gb, kThreads, 0, sm>>>(xout, x, n);
    }
    int* h16 = (int*)((unsigned char*)ctx->h_pinned + 2048 + 64);
    s = cuda_check(ctx, cudaMemcpyAsync(ctx->h_pinned, scal, sizeof(double), cudaMemcpyDeviceToHost, sm), "read ||b||");
    if (!s && use16)
        s = cuda_check(ctx, cudaMemcpyAsync(h16, ctx->d_flags + kF16Flag, sizeof(int), cudaMemcpyDeviceToHost, sm),
                       "read range flag");
    if (!s) s = cuda_check(ctx, cudaStreamSynchronize(sm), "sync ||b||");
    if (s) return s;
    prof_flush(ctx);
    if (use16 && *h16) use16 = false;  // an entry beyond the FP16 range: FP32 operator throughout
    // the Arnoldi-step matvec on the FP16 copy runs on the tensor cores where the element size allows
    CUtensorMap map16;
    bool tc16 = false;
    if constexpr (std::is_same<V, float>::value)
        tc16 = use16 && gemv_tc_ok(t) && (int64_t)nx * nz * rows < (1LL << 30) &&  // 32-bit row indices
               map_op16(&map16, A16, (int64_t)nx * nz * rows, t.nin);
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
    double rel = 1.0, beta_prev = 0.0;
    bool converged = false;
    int* hflag = (int*)((unsigned char*)ctx->h_pinned + 2048);  // [0] matvec copy wait, [1] sweep wait
    hflag[0] = hflag[1] = 0;
    // restart residual r = b - (I - A_int) x and beta = ||r||
    auto enqueue_residual = [&]() -> elrt_status {
        elrt_status e = launch_gemv<A, X>(ctx, nx, nz, rows, Aop, x, nullptr, x, 1, -1, r, nullptr);
        if (e) return e;
        { ProfScope ps(ctx, "krylov", 1, kv(3, n, sizeof(X))); k_bminus<X><<<gb, kThreads, 0, sm>>>(b, r, n); }
        { ProfScope ps(ctx, "krylov", 1, kv(1, n, sizeof(X))); k_dots<X><<<dim3(nblk, 1), kThreads, 0, sm>>>(r, n, r, partial, nullptr); }
        { ProfScope ps(ctx, "krylov"); k_dots_finish<<<1, kThreads, 0, sm>>>(partial, nblk, scal + 1, 2, nullptr); }
        return ELRT_OK;
    };
    // v_0 = r / beta, then mj Arnoldi steps with the FP16 (f16) or the given operator, the small
    // least-squares solve and x += V y; ends with the state and the matvec's timeout flag copied to
    // pinned host memory
    // While profiling (plain launches only), the algorithmic work each Arnoldi step enqueues is
    // recorded, so that the steps the device skips once converged (their kernels return at once)
    // can be taken out of the work counts after the cycle.
    std::vector<std::map<std::string, std::pair<double, double>>> wsnap;
    auto enqueue_cycle = [&](bool f16, int mj) -> elrt_status {
        elrt_status e = ELRT_OK;
        wsnap.clear();
        {
            ProfScope ps(ctx, "krylov", 1, kv(1, n, sizeof(X)) + kv(1, n, sizeof(V)));
            k_scale<X, V><<<gb, kThreads, 0, sm>>>(r, Vb, n, scal + 1, nullptr);
        }
        { ProfScope ps(ctx, "krylov"); k_cycle_start<<<1, 1, 0, sm>>>(st, gv, m, scal + 1, arn4 ? arn->sc : nullptr); }
        for (int j = 0; j < mj; ++j) {
            if (ctx->profiling) wsnap.push_back(ctx->work);
            V* vj = Vb + (size_t)j * n;
            V* w = Vb + (size_t)(j + 1) * n;
            double* hc = H + (size_t)j * (m + 1);
            if constexpr (std::is_same<V, float>::value) {
                if (pc) {  // right preconditioning: the matvec takes M W_j (its scale folded in as before)
                    e = sweep_apply(ctx, nx, nz, f16 ? (const void*)A16 : Aop, f16 ? 2 : (int)sizeof(A), vj, pc_t,
                                    pc_order, pc_zw, pc_flags, &st->done, nullptr);
                    if (e) return e;
                    vj = pc_t;
                }
                if (arn4) {  // matvec with the first Gram-Schmidt pass, then two launches
                    const ArnFuse fz{arn, partial, Vb, n, j};
                    if (f16 && tc16) e = launch_gemv_tc(ctx, map16, nx, nz, vj, w, st, fz);
                    else if (f16) e = launch_gemv<__half, V>(ctx, nx, nz, rows, A16, vj, nullptr, vj, 1, -1, w, st, fz);
                    else e = launch_gemv<A, V>(ctx, nx, nz, rows, Aop, vj, nullptr, vj, 1, -1, w, st, fz);
                    if (e) return e;
                    const double vb = 4.0 * n;
                    // (bytes counted as if the second pass ran: the bound on what these launches move)
                    { ProfScope ps(ctx, "krylov", 1, (2 * j + 5) * vb); k_arn_axdots<<<nblk, kArnThreads, 0, sm>>>(Vb, n, j, partial, arn, st); }
                    {
                        ProfScope ps(ctx, "krylov", 1, (j + 3) * vb);
                        k_arn_axnorm<<<nblk, kArnThreads, 0, sm>>>(Vb, n, j, partial, arn, H, m + 1, cs, sn, gv, st);
                    }
                    continue;
                }
                if (f16) e = launch_gemv<__half, V>(ctx, nx, nz, rows, A16, vj, nullptr, vj, 1, -1, w, st);
                else e = launch_gemv<A, V>(ctx, nx, nz, rows, Aop, vj, nullptr, vj, 1, -1, w, st);
            } else {
                e = launch_gemv<A, V>(ctx, nx, nz, rows, Aop, vj, nullptr, vj, 1, -1, w, st);
            }
            if (e) return e;
            // classical Gram-Schmidt, twice
            const size_t sv = sizeof(V);
            { ProfScope ps(ctx, "krylov", 1, kv(j + 2, n, sv)); k_dots<V><<<dim3(nblk, j + 1), kThreads, 0, sm>>>(Vb, n, w, partial, st); }
            { ProfScope ps(ctx, "krylov"); k_dots_finish<<<j + 1, kThreads, 0, sm>>>(partial, nblk, hc, 0, st); }
            { ProfScope ps(ctx, "krylov", 1, kv(j + 3, n, sv)); k_axpy_multi<V><<<gb, kThreads, 0, sm>>>(Vb, n, j + 1, hc, w, -1, st); }
            { ProfScope ps(ctx, "krylov", 1, kv(j + 2, n, sv)); k_dots<V><<<dim3(nblk, j + 1), kThreads, 0, sm>>>(Vb, n, w, partial, st); }
            { ProfScope ps(ctx, "krylov"); k_dots_finish<<<j + 1, kThreads, 0, sm>>>(partial, nblk, yv, 0, st); }
            { ProfScope ps(ctx, "krylov"); k_dots_finish<<<j + 1, kThreads, 0, sm>>>(partial, nblk, hc, 1, st); }  // h += second pass
            { ProfScope ps(ctx, "krylov", 1, kv(j + 3, n, sv)); k_axpy_multi<V><<<gb, kThreads, 0, sm>>>(Vb, n, j + 1, yv, w, -1, st); }
            // h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}
            { ProfScope ps(ctx, "krylov", 1, kv(1, n, sv)); k_dots<V><<<dim3(nblk, 1), kThreads, 0, sm>>>(w, n, w, partial, st); }
            { ProfScope ps(ctx, "krylov"); k_dots_finish<<<1, kThreads, 0, sm>>>(partial, nblk, hc + j + 1, 2, st); }
            { ProfScope ps(ctx, "krylov", 1, kv(2, n, sv)); k_scale<V, V><<<gb, kThreads, 0, sm>>>(w, w, n, hc + j + 1, st); }
            { ProfScope ps(ctx, "krylov"); k_givens<<<1, 1, 0, sm>>>(H, m + 1, cs, sn, gv, j, st); }
        }
        if (ctx->profiling) wsnap.push_back(ctx->work);
        { ProfScope ps(ctx, "krylov"); k_solve_upper<<<1, 1, 0, sm>>>(H, m + 1, gv, yv, st); }
        if constexpr (std::is_same<V, float>::value) {
            if (pc) {  // x += M (sum y_i s_i W_i)
                e = cuda_check(ctx, cudaMemsetAsync(pc_u, 0, (size_t)n * sizeof(float), sm), "zero correction");
                if (e) return e;
                {
                    ProfScope ps(ctx, "krylov", 1, kv(m, n, sizeof(V)) + kv(2, n, sizeof(float)));
                    k_update_x<V, float><<<gb, kThreads, 0, sm>>>(Vb, n, yv, arn4 ? arn->sc : nullptr, pc_u, st);
                }
                e = sweep_apply(ctx, nx, nz, f16 ? (const void*)A16 : Aop, f16 ? 2 : (int)sizeof(A), pc_u, pc_t,
                                pc_order, pc_zw, pc_flags, nullptr, &st->j_done);
                if (e) return e;
                ProfScope ps(ctx, "krylov", 1, kv(1, n, sizeof(float)) + kv(2, n, sizeof(X)));
                k_add_f<X><<<gb, kThreads, 0, sm>>>(x, pc_t, n);
            }
        }
        if (!pc) {
            ProfScope ps(ctx, "krylov", 1, kv(m, n, sizeof(V)) + kv(2, n, sizeof(X)));
            k_update_x<V, X><<<gb, kThreads, 0, sm>>>(Vb, n, yv, arn4 ? arn->sc : nullptr, x, st);
        }
        e = cuda_check(ctx, cudaGetLastError(), "gmres launches");
        if (!e) e = cuda_check(ctx, cudaMemcpyAsync(hst, st, sizeof(GmState), cudaMemcpyDeviceToHost, sm), "read state");
        if (!e)
            e = cuda_check(ctx, cudaMemcpyAsync(hflag, ctx->d_flags + kGemvFlag, sizeof(int), cudaMemcpyDeviceToHost, sm),
                           "read flag");
        if (!e && pc)
            e = cuda_check(ctx, cudaMemcpyAsync(hflag + 1, pc_flags, sizeof(int), cudaMemcpyDeviceToHost, sm),
                           "read sweep flag");
        return e;
    };
    // Graph path (ctx->graphs, no per-launch timing): a whole restart cycle -- restart residual,
    // convergence test on the device, m Arnoldi steps, update -- is captured once per Arnoldi
    // operator and replayed, one host synchronisation per cycle.  The FP16-to-FP32 switch then acts
    // from the cycle after the one that stalled.  A last partial cycle (max_iter) and the final
    // residual check run as plain launches.
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int64_t gnodes[2] = {0, 0};
    bool graphs = ctx->graphs && !ctx->profiling;
    // The capture runs on a stream of its own (the context's may be the legacy default stream,
    // which cannot be captured); the graph is then launched on the context's stream.
    auto capture = [&](int v) -> bool {
        cudaStream_t cs = nullptr;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        cudaGraph_t g = nullptr;
        const int64_t l0 = ctx->launches;
        const cudaStream_t own = ctx->stream;
        bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) == cudaSuccess;
        if (ok) {
            ctx->stream = sm = cs;
            elrt_status e = enqueue_residual();
            if (!e) e = enqueue_cycle(v == 1, m);
            const cudaError_t ce = cudaStreamEndCapture(cs, &g);
            ctx->stream = sm = own;
            ok = !e && ce == cudaSuccess && g && cudaGraphInstantiate(&gexec[v], g, 0) == cudaSuccess;
        }
        gnodes[v] = ctx->launches - l0;
        ctx->launches = l0;  // counted again at every replay
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (!ok) {
            gexec[v] = nullptr;
            cudaGetLastError();  // a failed capture leaves no error behind: plain launches follow
            ctx->last_error.clear();
        }
        return ok;
    };
    auto release = [&]() {
        for (auto& ge : gexec)
            if (ge) cudaGraphExecDestroy(ge);
    };
    for (;;) {
        if (graphs && its + m <= max_iter) {
            const int v = use16 ? 1 : 0;
            if (!gexec[v] && !capture(v)) {
                graphs = false;  // capture not possible here: plain launches from now on
                continue;
            }
            s = cuda_check(ctx, cudaGraphLaunch(gexec[v], sm), "graph launch");
            if (!s) s = cuda_check(ctx, cudaStreamSynchronize(sm), "sync cycle");
            if (s) {
                release();
                return s;
            }
            ctx->launches += gnodes[v];
            if (hflag[0] || hflag[1]) {
                release();
                return ctx_fail(ctx, ELRT_ETIMEOUT, hflag[0] ? "a copy wait of the streaming matvec timed out"
                                                             : "a wait of the sweep preconditioner timed out");
            }
            const double beta = hst->beta;
            rel = beta / bnorm;
            if (!(beta > rtol * bnorm) || !isfinite(beta)) {
                converged = isfinite(beta);
                break;
            }
            if (use16 && cycles > 0 && beta > 0.9 * beta_prev) use16 = false;
            beta_prev = beta;
            its += hst->j_done;
            ++cycles;
            if (hst->j_done == 0) break;  // no progress possible
            continue;
        }
        s = enqueue_residual();
        if (!s) s = cuda_check(ctx, cudaMemcpyAsync(ctx->h_pinned, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, sm), "read beta");
        if (!s) s = cuda_check(ctx, cudaStreamSynchronize(sm), "sync beta");
        if (s) {
            release();
            return s;
        }
        prof_flush(ctx);
        const double beta = *(double*)ctx->h_pinned;
        rel = beta / bnorm;
        if (!(beta > rtol * bnorm) || !isfinite(beta)) {
            converged = isfinite(beta);
            break;
        }
        if (its >= max_iter) break;
        // a cycle on the FP16 copy that took the true residual down by less than 10%: the rounding
        // of the copy limits the refinement, continue with the FP32 operator
        if (use16 && cycles > 0 && beta > 0.9 * beta_prev) use16 = false;
        beta_prev = beta;
        s = enqueue_cycle(use16, std::min(m, max_iter - its));
        if (!s) s = cuda_check(ctx, cudaStreamSynchronize(sm), "sync cycle");
        if (s) {
            release();
            return s;
        }
        prof_flush(ctx);
        if (hflag[0] || hflag[1]) {
            release();
            return ctx_fail(ctx, ELRT_ETIMEOUT, hflag[0] ? "a copy wait of the streaming matvec timed out"
                                                         : "a wait of the sweep preconditioner timed out");
        }
        if (wsnap.size() >= 2) {  // take the skipped steps j_done .. mj - 1 out of the work counts
            const auto& at = wsnap[std::min<size_t>((size_t)std::max(0, hst->j_done), wsnap.size() - 1)];
            const auto& end = wsnap.back();
            for (const auto& kv : end) {
                const auto it = at.find(kv.first);
                const double b0 = it == at.end() ? 0.0 : it->second.first;
                const double f0 = it == at.end() ? 0.0 : it->second.second;
                ctx->work[kv.first].first -= kv.second.first - b0;
                ctx->work[kv.first].second -= kv.second.second - f0;
            }
        }
        wsnap.clear();
        its += hst->j_done;
        ++cycles;
        if (hst->j_done == 0) break;  // no progress possible
    }
    release();
    if constexpr (own_x) {
        ProfScope ps(ctx, "krylov", 1, 16.0 * n);
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

__global__ void k_add_to(double* __restrict__ y, const double* __restrict__ a, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += a[i];
}

// out_K = self_K + Aop_K x_in(K) for operators of `rows` rows per element (nm: the mean intensity
// with the source part f2m; nu: the radiance with f_u).  The matvec prefetches a self term of at
// most 4 (p+1) N/2 rows per element; longer ones (the radiance) are added by a separate pass.
elrt_status global_recover_rows(elrt_ctx* ctx, int nx, int nz, int rows, const void* A, int dtype, const double* x,
                                const double* inflow, const double* self, double* out) {
    constexpr int kSelfRows = 4 * ELRT_MAX_N1 * (ELRT_MAX_ANG / 2);
    const bool fused = self && rows <= kSelfRows;
    elrt_status s = dtype == ELRT_F32
                        ? launch_gemv<float, double>(ctx, nx, nz, rows, A, x, inflow, fused ? self : nullptr, fused ? 1 : 0,
                                                     1, out, nullptr)
                        : launch_gemv<double, double>(ctx, nx, nz, rows, A, x, inflow, fused ? self : nullptr,
                                                      fused ? 1 : 0, 1, out, nullptr);
    if (s || !self || fused) return s;
    const int64_t n = (int64_t)nx * nz * rows;
    ProfScope ps(ctx, "gemv", 1, 24.0 * n);
    k_add_to<<<grid_for(n), kThreads, 0, ctx->stream>>>(out, self, n);
    return cuda_check(ctx, cudaGetLastError(), "add launch");
}

elrt_status global_recover(elrt_ctx* ctx, int nx, int nz, const void* A, int dtype, const double* x,
                           const double* inflow, double* mean, const double* f2m) {
    return global_recover_rows(ctx, nx, nz, ctx->tab.nm, A, dtype, x, inflow, f2m, mean);
}

elrt_status global_solve(elrt_ctx* ctx, int nx, int nz, const void* A, int dtype, const double* inflow, double rtol,
                         int max_iter, int restart, int use_guess, double* x, elrt_solve_stats* stats,
                         const double* f2o) {
    if (restart == 0) restart = ctx->tune.restart;
    if (restart > kMaxRestart) return ctx_fail(ctx, ELRT_EINVAL, "restart above 200");
    if (dtype == ELRT_F32)
        return gmres<float, float, ff>(ctx, nx, nz, A, inflow, rtol, max_iter, restart, use_guess, x, stats, f2o);
    return gmres<double, double, double>(ctx, nx, nz, A, inflow, rtol, max_iter, restart, use_guess, x, stats, f2o);
}
