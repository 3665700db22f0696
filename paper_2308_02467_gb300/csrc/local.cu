// Local stage (Sec. 2.2.3, eqs. hdg_local_mat, hdg_local_i2u, hdg_local_i2o, ang_ave; App. A):
// per element, assemble [A | -B^], factor A = P L U by blocked right-looking LU with partial
// pivoting while the right-hand sides ride along as extra columns (so the forward substitution
// comes for free), back-substitute, optionally refine in FP64 with the structured residual, and
// restrict the solution to in2out / in2sol.
//
// Layout of the per-element workspace matrix M (row-major, leading dimension ld):
//   columns [0, nu)        the local matrix A, overwritten by L (unit lower, below the diagonal)
//                          and U; panels are swapped LAPACK-style inside a panel and
//                          LINPACK-style across panels (earlier L columns keep their order);
//   columns [nu, nu + nin) the right-hand sides -B^, overwritten by the solution X (or by the
//                          refinement residual / correction).
// One thread block of 256 threads works on one element at a time.
#include <math.h>
#include <stdio.h>

#include <string.h>

#include <algorithm>
#include <type_traits>
#include <string>

#include "elrt_internal.h"
#include "ff.h"

namespace {

constexpr int kThreads = 256;

// ------------------------------------------------------------------------------------------------
// assembly
// ------------------------------------------------------------------------------------------------

// Entry (row r = (k, i), column c) of the augmented matrix [A | -B^] of eq. hdg_local_mat divided
// by (h/2) dth, with kh = kappa_hat_i and om = omega.  Node i = (a, b), column node j = (jc, jd).
__device__ __forceinline__ double aug_entry(const Tab& t, int k, int i, int c, const double* kh, double om) {
    const int nm = t.nm, n1 = t.n1, p = t.p;
    const int a = i % n1, b = i / n1;
    double v = 0.0;
    if (c < t.nu) {
        const int l = c / nm, j = c - l * nm;
        if (l == k) {
            const int jc = j % n1, jd = j / n1;
            const double wj = t.w[jc] * t.w[jd];
            // -C^k_ij = -w_j (sbar_k . grad phi_i)(x_j)
            if (jd == b) v -= wj * t.sx[k] * t.D[jc * n1 + a];
            if (jc == a) v -= wj * t.sz[k] * t.D[jd * n1 + b];
            if (j == i) {
                // B^k_ii: outflow faces through node i; M_ii = w_i kappa_hat_i
                double bd = 0.0;
                if (b == 0 && t.sdn[0][k] > 0) bd += t.w[a] * t.sdn[0][k];
                if (a == p && t.sdn[1][k] > 0) bd += t.w[b] * t.sdn[1][k];
                if (b == p && t.sdn[2][k] > 0) bd += t.w[a] * t.sdn[2][k];
                if (a == 0 && t.sdn[3][k] > 0) bd += t.w[b] * t.sdn[3][k];
                v += bd + t.w[a] * t.w[b] * kh[i];
            }
        }
        if (j == i) {
            int d = k - l;
            if (d < 0) d += t.N;
            v -= t.w[a] * t.w[b] * om * kh[i] * t.wc[d];  // -S
        }
    } else if (c < t.nu + t.nin) {
        const int col = c - t.nu;
        const int F = col / t.nface, rem = col - F * t.nface;
        const int m = rem / t.half, kk = rem - m * t.half;
        if (t.inc[F][kk] == k && face_node(F, m, p) == i) v = -t.w[m] * t.sdn[F][k];  // -B^ (positive)
    }
    return v;
}

// FP32 copies of the tables one block (element e, angular cell k) of the FP32 assembly reads
struct AugF {
    float w[ELRT_MAX_N1], D[ELRT_MAX_N1 * ELRT_MAX_N1], wc[ELRT_MAX_ANG], sdn[4], kh[ELRT_MAX_N1 * ELRT_MAX_N1];
    float sx, sz, om;
};

// The same entries as aug_entry for the candidates of row (k, i), evaluated in FP32: on the FP32
// paths the assembled matrix only feeds the factorisation (the float-float residual of the
// refinement and the right-hand side -B^ it uses come from the FP64 tables), so an entry a few
// FP32 ulps from the rounded FP64 value changes nothing but the factorisation's own rounding, and
// the FP64 pipe (1/64 of the FP32 rate on this GPU) is kept out of the assembly.
__device__ __forceinline__ float aug_entry_f(const Tab& t, const AugF& f, int k, int i, int c) {
    const int nm = t.nm, n1 = t.n1, p = t.p;
    const int a = i % n1, b = i / n1;
    float v = 0.f;
    if (c < t.nu) {
        const int l = c / nm, j = c - l * nm;
        if (l == k) {
            const int jc = j % n1, jd = j / n1;
            const float wj = f.w[jc] * f.w[jd];
            if (jd == b) v -= wj * f.sx * f.D[jc * n1 + a];
            if (jc == a) v -= wj * f.sz * f.D[jd * n1 + b];
            if (j == i) {
                float bd = 0.f;
                if (b == 0 && f.sdn[0] > 0.f) bd += f.w[a] * f.sdn[0];
                if (a == p && f.sdn[1] > 0.f) bd += f.w[b] * f.sdn[1];
                if (b == p && f.sdn[2] > 0.f) bd += f.w[a] * f.sdn[2];
                if (a == 0 && f.sdn[3] > 0.f) bd += f.w[b] * f.sdn[3];
                v += bd + f.w[a] * f.w[b] * f.kh[i];
            }
        }
        if (j == i) {
            int d = k - l;
            if (d < 0) d += t.N;
            v -= f.w[a] * f.w[b] * f.om * f.kh[i] * f.wc[d];
        }
    } else if (c < t.nu + t.nin) {
        const int col = c - t.nu;
        const int F = col / t.nface, rem = col - F * t.nface;
        const int m = rem / t.half, kk = rem - m * t.half;
        if (t.inc[F][kk] == k && face_node(F, m, p) == i) v = -f.w[m] * f.sdn[F];
    }
    return v;
}

// Grid: (E, N).  Block (e, k) writes rows (k, 0..nm-1) of element e; columns >= nu + nin are 0.
// Also validates the inputs (flags[0] |= 1 on a negative or non-finite kappa / h, omega outside [0, 1],
// or kappa_hat = kappa h / 2 above 1e30, beyond which the FP32 modes would overflow).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_assemble(Tab t, double h, const double* __restrict__ h_elem,
                                                       const double* __restrict__ kappa,
                                                       const double* __restrict__ omega, T* __restrict__ M,
                                                       int64_t ld, int64_t estride, T* __restrict__ rhs_out,
                                                       int64_t rhs_ld, int* flags) {
    __shared__ double kh[ELRT_MAX_N1 * ELRT_MAX_N1];
    const int64_t e = blockIdx.x;
    const int k = blockIdx.y;
    const double he = h_elem ? h_elem[e] : h;
    const double om = omega[e];
    for (int i = threadIdx.x; i < t.nm; i += blockDim.x) {
        double kv = kappa[e * t.nm + i];
        if (!(kv >= 0.0) || !isfinite(kv) || !(kv * 0.5 * he <= 1e30)) atomicOr(flags, 1);
        kh[i] = kv * 0.5 * he;
    }
    if (threadIdx.x == 0 && (!(he > 0.0) || !isfinite(he) || !(om >= 0.0 && om <= 1.0))) atomicOr(flags, 1);
    __shared__ AugF fa;  // FP32 tables (FP32 candidate path only)
    if constexpr (sizeof(T) == 4) {
        if (!rhs_out) {
            for (int q = threadIdx.x; q < t.n1 * t.n1; q += blockDim.x) fa.D[q] = (float)t.D[q];
            for (int q = threadIdx.x; q < t.n1; q += blockDim.x) fa.w[q] = (float)t.w[q];
            for (int q = threadIdx.x; q < t.N; q += blockDim.x) fa.wc[q] = (float)t.wc[q];
            if (threadIdx.x < 4) fa.sdn[threadIdx.x] = (float)t.sdn[threadIdx.x][k];
            if (threadIdx.x == 0) {
                fa.sx = (float)t.sx[k];
                fa.sz = (float)t.sz[k];
                fa.om = (float)om;
            }
        }
    }
    __syncthreads();
    if constexpr (sizeof(T) == 4) {
        if (!rhs_out)
            for (int q = threadIdx.x; q < t.nm; q += blockDim.x) fa.kh[q] = (float)kh[q];
        __syncthreads();
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* Me = M + e * estride;
    float amax = 0.f;  // largest |entry| this thread wrote (FP32 candidate path)
    for (int i = warp; i < t.nm; i += kThreads / 32) {
        const int r = k * t.nm + i;
        if (rhs_out) {
            // separate outputs: A into M (ld = nu), -B^ into rhs_out
            for (int c = lane; c < t.nu; c += 32) Me[(int64_t)r * ld + c] = (T)aug_entry(t, k, i, c, kh, om);
            for (int c = lane; c < t.nin; c += 32)
                rhs_out[e * (int64_t)t.nu * rhs_ld + (int64_t)r * rhs_ld + c] = (T)aug_entry(t, k, i, t.nu + c, kh, om);
        } else {
            // the row is zero apart from 2 n1 + N - 2 operator entries (x-line and z-line through
            // node i, node i in the other angular cells) and at most two of -B^: zero-fill it with
            // vector stores, then evaluate only those candidates
            T* row = Me + (int64_t)r * ld;
            constexpr int VW = 16 / sizeof(T);
            using V4 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
            const V4 z{};
            for (int c = lane; c < ld / VW; c += 32) reinterpret_cast<V4*>(row)[c] = z;
            __syncwarp();
            const int n1 = t.n1, a = i % n1, b = i / n1;
            const int ncand = 1 + 2 * (n1 - 1) + (t.N - 1) + 4;
            for (int q = lane; q < ncand; q += 32) {
                int c = -1;
                if (q == 0) {
                    c = k * t.nm + i;  // diagonal
                } else if (q < n1) {   // x-line, j = (q', b) with q' != a
                    const int qq = q - 1 + (q - 1 >= a);
                    c = k * t.nm + qq + n1 * b;
                } else if (q < 2 * n1 - 1) {  // z-line, j = (a, q') with q' != b
                    const int q0 = q - n1;
                    const int qq = q0 + (q0 >= b);
                    c = k * t.nm + a + n1 * qq;
                } else if (q < 2 * n1 - 1 + t.N - 1) {  // node i in angular cell l != k
                    const int l0 = q - (2 * n1 - 1);
                    const int l = l0 + (l0 >= k);
                    c = l * t.nm + i;
                } else {  // -B^ on face F if node i lies on it and cell k enters through it
                    const int F = q - (2 * n1 - 1 + t.N - 1);
                    int m = -1, kk = -1;
                    for (int mm = 0; mm < n1; ++mm)
                        if (face_node(F, mm, t.p) == i) m = mm;
                    for (int x = 0; x < t.half; ++x)
                        if (t.inc[F][x] == k) kk = x;
                    if (m >= 0 && kk >= 0) c = t.nu + F * t.nface + m * t.half + kk;
                }
                if (c >= 0) {
                    if constexpr (sizeof(T) == 4) {
                        const float v = aug_entry_f(t, fa, k, i, c);
                        row[c] = v;
                        amax = fmaxf(amax, fabsf(v));
                    } else {
                        row[c] = (T)aug_entry(t, k, i, c, kh, om);
                    }
                }
            }
        }
    }
    if constexpr (sizeof(T) == 4) {
        // the chunk's largest |entry| (float bits of a non-negative value order as unsigned ints);
        // the common case, a block below the current maximum, reads instead of contending
        for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
        if (lane == 0 && !rhs_out) {
            unsigned* slot = reinterpret_cast<unsigned*>(flags + kAsmMaxFlag);
            const unsigned bits = __float_as_uint(amax);
            if (*(volatile unsigned*)slot < bits) atomicMax(slot, bits);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// blocked LU with partial pivoting on the CUDA cores
// ------------------------------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }

// M[r0 + r][c0 + c] -= sum_q Ls[(lrow0 + r) * lds + q] * Us[q * CW + c]
// for r in [0, nrows), c in [0, ncols) (ncols <= CW), q in [0, jb).
// Thread (tr, tc) = (tid / 32, tid % 32) owns rows tr + 8 s (s < 8) and columns tc + 32 q (q < QN).
template <typename T, int NB, int QN>
__device__ __forceinline__ void rank_update(T* __restrict__ M, int64_t ld, int r0, int nrows, int c0, int ncols,
                                            const T* __restrict__ Ls, int lds, int lrow0, const T* __restrict__ Us,
                                            int jb) {
    constexpr int CW = 32 * QN;
    const int tr = threadIdx.x >> 5, tc = threadIdx.x & 31;
    for (int rb = 0; rb < nrows; rb += 64) {
        T acc[8][QN];
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int r = rb + tr + 8 * s;
#pragma unroll
            for (int q = 0; q < QN; ++q) {
                const int c = tc + 32 * q;
                acc[s][q] = (r < nrows && c < ncols) ? M[(int64_t)(r0 + r) * ld + c0 + c] : T(0);
            }
        }
#pragma unroll 4
        for (int kq = 0; kq < NB; ++kq) {
            if (kq < jb) {
                T bv[QN];
#pragma unroll
                for (int q = 0; q < QN; ++q) bv[q] = Us[kq * CW + tc + 32 * q];
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    const int r = rb + tr + 8 * s;
                    const T av = (r < nrows) ? Ls[(lrow0 + r) * lds + kq] : T(0);
#pragma unroll
                    for (int q = 0; q < QN; ++q) acc[s][q] -= av * bv[q];
                }
            }
        }
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int r = rb + tr + 8 * s;
#pragma unroll
            for (int q = 0; q < QN; ++q) {
                const int c = tc + 32 * q;
                if (r < nrows && c < ncols) M[(int64_t)(r0 + r) * ld + c0 + c] = acc[s][q];
            }
        }
    }
}

// block-wide argmax of |value| (ties: smallest index)
template <typename T>
__device__ __forceinline__ void block_argmax(T v, int idx, T* sval, int* sidx, T* out_v, int* out_i) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        T ov = __shfl_down_sync(0xffffffffu, v, off);
        int oi = __shfl_down_sync(0xffffffffu, idx, off);
        if (ov > v || (ov == v && oi < idx && oi >= 0)) {
            v = ov;
            idx = oi;
        }
    }
    if (lane == 0) {
        sval[warp] = v;
        sidx[warp] = idx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        T bv = sval[0];
        int bi = sidx[0];
        for (int w = 1; w < kThreads / 32; ++w) {
            if (sval[w] > bv || (sval[w] == bv && sidx[w] >= 0 && (bi < 0 || sidx[w] < bi))) {
                bv = sval[w];
                bi = sidx[w];
            }
        }
        *out_v = bv;
        *out_i = bi;
    }
    __syncthreads();
}

// Forward step of panel J on the columns [c_begin, c_end): apply the panel's row swaps, solve with
// the unit lower L11 (rows 0..jb-1 of Ps) and update the rows below with L21.
// Ps holds rows J..nu-1 of the panel columns (relative row index), stride NB + 1.
template <typename T, int NB, int QN>
__device__ void panel_forward(T* __restrict__ M, int64_t ld, int nu, int J, int jb, const int* ipiv_s, const T* Ps,
                              T* Us, int c_begin, int c_end) {
    constexpr int CW = 32 * QN;
    constexpr int lds = NB + 1;
    for (int cs = c_begin; cs < c_end; cs += CW) {
        const int ncols = min(CW, c_end - cs);
        for (int tcol = threadIdx.x; tcol < CW; tcol += kThreads) {
            if (tcol < ncols) {
                const int col = cs + tcol;
                T x[NB];
#pragma unroll
                for (int jj = 0; jj < NB; ++jj) {
                    if (jj < jb) {
                        const int pr = ipiv_s[jj];
                        if (pr != jj) {
                            T a = M[(int64_t)(J + jj) * ld + col];
                            T b = M[(int64_t)(J + pr) * ld + col];
                            M[(int64_t)(J + jj) * ld + col] = b;
                            M[(int64_t)(J + pr) * ld + col] = a;
                        }
                    }
                }
#pragma unroll
                for (int jj = 0; jj < NB; ++jj) x[jj] = (jj < jb) ? M[(int64_t)(J + jj) * ld + col] : T(0);
#pragma unroll
                for (int jj = 1; jj < NB; ++jj) {
                    T s = x[jj];
#pragma unroll
                    for (int ii = 0; ii < jj; ++ii) s -= Ps[jj * lds + ii] * x[ii];
                    x[jj] = s;
                }
#pragma unroll
                for (int jj = 0; jj < NB; ++jj) {
                    if (jj < jb) M[(int64_t)(J + jj) * ld + col] = x[jj];
                    Us[jj * CW + tcol] = x[jj];
                }
            } else {
#pragma unroll
                for (int jj = 0; jj < NB; ++jj) Us[jj * CW + tcol] = T(0);
            }
        }
        __syncthreads();
        rank_update<T, NB, QN>(M, ld, J + jb, nu - J - jb, cs, ncols, Ps, lds, jb, Us, jb);
        __syncthreads();
    }
}

// Backward substitution U X = Y on the columns [c_begin, c_end), panel by panel from the last.
template <typename T, int NB, int QN>
__device__ void backward_sweep(T* __restrict__ M, int64_t ld, int nu, T* Ps, T* Us, int c_begin, int c_end) {
    constexpr int CW = 32 * QN;
    constexpr int lds = NB + 1;
    const int last = ((nu - 1) / NB) * NB;
    for (int J = last; J >= 0; J -= NB) {
        const int jb = min(NB, nu - J);
        // U[0:J+jb, J:J+jb] -> Ps
        for (int idx = threadIdx.x; idx < (J + jb) * NB; idx += kThreads) {
            const int r = idx / NB, c = idx - r * NB;
            Ps[r * lds + c] = (c < jb) ? M[(int64_t)r * ld + J + c] : T(0);
        }
        __syncthreads();
        for (int cs = c_begin; cs < c_end; cs += CW) {
            const int ncols = min(CW, c_end - cs);
            for (int tcol = threadIdx.x; tcol < CW; tcol += kThreads) {
                if (tcol < ncols) {
                    const int col = cs + tcol;
                    T x[NB];
#pragma unroll
                    for (int jj = 0; jj < NB; ++jj) x[jj] = (jj < jb) ? M[(int64_t)(J + jj) * ld + col] : T(0);
#pragma unroll
                    for (int jj = NB - 1; jj >= 0; --jj) {
                        if (jj < jb) {
                            T s = x[jj];
#pragma unroll
                            for (int ii = jj + 1; ii < NB; ++ii)
                                if (ii < jb) s -= Ps[(J + jj) * lds + ii] * x[ii];
                            const T d = Ps[(J + jj) * lds + jj];
                            x[jj] = (d != T(0)) ? s / d : T(0);
                        }
                    }
#pragma unroll
                    for (int jj = 0; jj < NB; ++jj) {
                        if (jj < jb) M[(int64_t)(J + jj) * ld + col] = x[jj];
                        Us[jj * CW + tcol] = x[jj];
                    }
                } else {
#pragma unroll
                    for (int jj = 0; jj < NB; ++jj) Us[jj * CW + tcol] = T(0);
                }
            }
            __syncthreads();
            if (J > 0) rank_update<T, NB, QN>(M, ld, 0, J, cs, ncols, Ps, lds, 0, Us, jb);
            __syncthreads();
        }
    }
}

template <typename T, int NB, int QN>
constexpr size_t lu_smem_bytes(int nu) {
    return (size_t)nu * (NB + 1) * sizeof(T) + (size_t)NB * 32 * QN * sizeof(T);
}

// Factor A (columns [0, nu)) and solve for the right-hand sides (columns [nu, nu + nrhs)).
// estatus[e] |= 1 on an exactly zero pivot (the element's result is then meaningless).
template <typename T, int NB, int QN>
__global__ void __launch_bounds__(kThreads, 1) k_lu_factor_solve(Tab t, T* __restrict__ Mall, int64_t ld,
                                                                 int64_t estride, int* __restrict__ ipiv_all,
                                                                 int* __restrict__ estatus, int64_t E) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Ps = reinterpret_cast<T*>(smem_raw);
    T* Us = Ps + (size_t)t.nu * (NB + 1);
    __shared__ T red_v[kThreads / 32];
    __shared__ int red_i[kThreads / 32];
    __shared__ int ipiv_s[NB];
    __shared__ T piv_v;
    __shared__ int piv_i;
    constexpr int lds = NB + 1;
    const int nu = t.nu, ncols = t.nu + t.nrhs;
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        T* M = Mall + e * estride;
        int* ipiv = ipiv_all + e * (int64_t)nu;
        int bad = 0;
        for (int J = 0; J < nu; J += NB) {
            const int jb = min(NB, nu - J);
            const int R = nu - J;
            for (int idx = threadIdx.x; idx < R * NB; idx += kThreads) {
                const int r = idx / NB, c = idx - r * NB;
                Ps[r * lds + c] = (c < jb) ? M[(int64_t)(J + r) * ld + J + c] : T(0);
            }
            __syncthreads();
            // unblocked LU with partial pivoting of the R x jb panel in shared memory
            for (int jj = 0; jj < jb; ++jj) {
                T bv = T(-1);
                int bi = -1;
                for (int r = jj + threadIdx.x; r < R; r += kThreads) {
                    const T v = tabs(Ps[r * lds + jj]);
                    if (v > bv) {
                        bv = v;
                        bi = r;
                    }
                }
                block_argmax<T>(bv, bi, red_v, red_i, &piv_v, &piv_i);
                // a column without a comparable entry (all NaN, after an overflow) has no argmax:
                // keep the diagonal row, so every row index stays inside the panel (the element is
                // flagged through piv_v below)
                const int pr = (piv_i >= jj && piv_i < R) ? piv_i : jj;
                if (threadIdx.x == 0) ipiv_s[jj] = pr;
                if (!(piv_v > T(0))) bad = 1;
                if (pr != jj) {
                    for (int c = threadIdx.x; c < NB; c += kThreads) {
                        T x = Ps[jj * lds + c];
                        Ps[jj * lds + c] = Ps[pr * lds + c];
                        Ps[pr * lds + c] = x;
                    }
                }
                __syncthreads();
                const T d = Ps[jj * lds + jj];
                const T inv = (d != T(0)) ? T(1) / d : T(0);
                for (int r = jj + 1 + threadIdx.x; r < R; r += kThreads) {
                    const T l = Ps[r * lds + jj] * inv;
                    Ps[r * lds + jj] = l;
                    for (int c = jj + 1; c < jb; ++c) Ps[r * lds + c] -= l * Ps[jj * lds + c];
                }
                __syncthreads();
            }
            for (int idx = threadIdx.x; idx < R * jb; idx += kThreads) {
                const int r = idx / jb, c = idx - r * jb;
                M[(int64_t)(J + r) * ld + J + c] = Ps[r * lds + c];
            }
            if (threadIdx.x < jb) ipiv[J + threadIdx.x] = J + ipiv_s[threadIdx.x];
            __syncthreads();
            panel_forward<T, NB, QN>(M, ld, nu, J, jb, ipiv_s, Ps, Us, J + jb, ncols);
        }
        backward_sweep<T, NB, QN>(M, ld, nu, Ps, Us, nu, ncols);
        if (threadIdx.x == 0 && bad) estatus[e] |= 1;
        __syncthreads();
    }
}

// Solve A D = R for the right-hand sides stored in columns [nu, nu + nrhs), with the factors and
// pivots left by k_lu_factor_solve (forward sweep with the interleaved swaps, then backward).
template <typename T, int NB, int QN>
__global__ void __launch_bounds__(kThreads, 1) k_lu_resolve(Tab t, T* __restrict__ Mall, int64_t ld, int64_t estride,
                                                            const int* __restrict__ ipiv_all, int64_t E) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Ps = reinterpret_cast<T*>(smem_raw);
    T* Us = Ps + (size_t)t.nu * (NB + 1);
    __shared__ int ipiv_s[NB];
    constexpr int lds = NB + 1;
    const int nu = t.nu, ncols = t.nu + t.nrhs;
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        T* M = Mall + e * estride;
        const int* ipiv = ipiv_all + e * (int64_t)nu;
        for (int J = 0; J < nu; J += NB) {
            const int jb = min(NB, nu - J);
            const int R = nu - J;
            for (int idx = threadIdx.x; idx < R * NB; idx += kThreads) {
                const int r = idx / NB, c = idx - r * NB;
                Ps[r * lds + c] = (c < jb) ? M[(int64_t)(J + r) * ld + J + c] : T(0);
            }
            if (threadIdx.x < jb) ipiv_s[threadIdx.x] = ipiv[J + threadIdx.x] - J;
            __syncthreads();
            panel_forward<T, NB, QN>(M, ld, nu, J, jb, ipiv_s, Ps, Us, nu, ncols);
        }
        backward_sweep<T, NB, QN>(M, ld, nu, Ps, Us, nu, ncols);
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------------
// FP64 refinement: structured residual R = -B^ - A X computed from the tables (never from the
// dense A), optional accumulation X += D, per-element max |R|.
// ------------------------------------------------------------------------------------------------

// mode 0: X64 = (double) src;  mode 1: X64 += (double) src.  Afterwards R -> src (as T).
// mode 2: X64 += (double) src only (the final correction when no residual is wanted).
// One block per element; columns in chunks of CWR staged in shared memory as float-float pairs,
// every product and sum in float-float (about 44 bits, at FP32 issue rate).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_residual(Tab t, double h, const double* __restrict__ h_elem,
                                                       const double* __restrict__ kappa,
                                                       const double* __restrict__ omega, T* __restrict__ Mall,
                                                       int64_t ld, int64_t estride, double* __restrict__ X64all,
                                                       int mode, int CWR, double* __restrict__ maxres, int64_t E) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nu = t.nu, nin = t.nin, nm = t.nm, n1 = t.n1, N = t.N, p = t.p;
    ff* Xs = reinterpret_cast<ff*>(smem_raw);  // [nu][CWR]
    ff* dcoef = Xs + (size_t)nu * CWR;         // [nu]: B^k_ii + w_i kappa_hat_i
    __shared__ ff wd[ELRT_MAX_N1 * ELRT_MAX_N1];      // w_q D[q][a]
    __shared__ ff sxw[ELRT_MAX_ANG * ELRT_MAX_N1];    // sx_k w_b
    __shared__ ff szw[ELRT_MAX_ANG * ELRT_MAX_N1];    // sz_k w_a
    __shared__ ff wcf[ELRT_MAX_ANG];                  // circulant phase
    __shared__ ff scoef[ELRT_MAX_N1 * ELRT_MAX_N1];   // w_i omega kappa_hat_i
    __shared__ double red[kThreads / 32];
    const int64_t e = blockIdx.x;
    if (e >= E) return;
    const double he = h_elem ? h_elem[e] : h;
    const double om = omega[e];
    for (int q = threadIdx.x; q < n1 * n1; q += kThreads) wd[q] = ff_from_double(t.w[q / n1] * t.D[q]);
    for (int q = threadIdx.x; q < N * n1; q += kThreads) {
        const int k = q / n1, b = q - k * n1;
        sxw[q] = ff_from_double(t.sx[k] * t.w[b]);
        szw[q] = ff_from_double(t.sz[k] * t.w[b]);
    }
    for (int q = threadIdx.x; q < N; q += kThreads) wcf[q] = ff_from_double(t.wc[q]);
    for (int i = threadIdx.x; i < nm; i += kThreads)
        scoef[i] = ff_from_double(t.w[i % n1] * t.w[i / n1] * om * kappa[e * nm + i] * 0.5 * he);
    for (int r = threadIdx.x; r < nu; r += kThreads) {
        const int k = r / nm, i = r - k * nm;
        const int a = i % n1, b = i / n1;
        double bd = 0.0;
        if (b == 0 && t.sdn[0][k] > 0) bd += t.w[a] * t.sdn[0][k];
        if (a == p && t.sdn[1][k] > 0) bd += t.w[b] * t.sdn[1][k];
        if (b == p && t.sdn[2][k] > 0) bd += t.w[a] * t.sdn[2][k];
        if (a == 0 && t.sdn[3][k] > 0) bd += t.w[b] * t.sdn[3][k];
        dcoef[r] = ff_from_double(bd + t.w[a] * t.w[b] * kappa[e * nm + i] * 0.5 * he);
    }
    T* M = Mall + e * estride;
    double* X64 = X64all + e * (int64_t)nu * nin;
    double rmax = 0.0;
    const int rows_per_pass = kThreads / CWR;
    const int tcol = threadIdx.x % CWR, trow = threadIdx.x / CWR;
    for (int cs = 0; cs < nin; cs += CWR) {
        __syncthreads();
        for (int r = trow; r < nu; r += rows_per_pass) {
            const int col = cs + tcol;
            double v = 0.0;
            if (col < nin) {
                const double d = (double)M[(int64_t)r * ld + nu + col];
                v = (mode == 0) ? d : X64[(int64_t)r * nin + col] + d;
                X64[(int64_t)r * nin + col] = v;
            }
            if (mode != 2) Xs[r * CWR + tcol] = ff_from_double(v);
        }
        if (mode == 2) continue;
        __syncthreads();
        for (int r = trow; r < nu; r += rows_per_pass) {
            const int col = cs + tcol;
            if (col >= nin) continue;
            const int k = r / nm, i = r - k * nm;
            const int a = i % n1, b = i / n1;
            const int base = k * nm;
            // (B + M) X
            ff acc = ff_mul(dcoef[r], Xs[r * CWR + tcol]);
            // - C X along the x-line and the z-line through node i
            ff tx{0.f, 0.f}, tz{0.f, 0.f};
            for (int q = 0; q < n1; ++q) {
                ff_fma(tx, wd[q * n1 + a], Xs[(base + q + n1 * b) * CWR + tcol]);
                ff_fma(tz, wd[q * n1 + b], Xs[(base + a + n1 * q) * CWR + tcol]);
            }
            tx = ff_norm(tx.h, tx.l);
            tz = ff_norm(tz.h, tz.l);
            ff cxz = ff_add(ff_mul(sxw[k * n1 + b], tx), ff_mul(szw[k * n1 + a], tz));
            // - S X
            ff sc{0.f, 0.f};
            for (int l = 0; l < N; ++l) {
                int d = k - l;
                if (d < 0) d += N;
                ff_fma(sc, wcf[d], Xs[(l * nm + i) * CWR + tcol]);
            }
            sc = ff_norm(sc.h, sc.l);
            ff s_term = ff_mul(scoef[i], sc);
            acc = ff_add(acc, ff{-cxz.h, -cxz.l});
            acc = ff_add(acc, ff{-s_term.h, -s_term.l});
            // -B^ entry of this (row, column)
            const int F = col / t.nface, rem = col - F * t.nface;
            const int m = rem / t.half, kk = rem - m * t.half;
            const double rhs = (t.inc[F][kk] == k && face_node(F, m, p) == i) ? -t.w[m] * t.sdn[F][k] : 0.0;
            const double res = rhs - ff_to_double(acc);
            rmax = fmax(rmax, fabs(res));
            M[(int64_t)r * ld + nu + col] = (T)res;
        }
    }
    // block max
    for (int off = 16; off > 0; off >>= 1) rmax = fmax(rmax, __shfl_down_sync(0xffffffffu, rmax, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rmax;
    __syncthreads();
    if (threadIdx.x == 0 && mode != 2) {
        double m = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) m = fmax(m, red[w]);
        maxres[e] = m;
    }
}

// ------------------------------------------------------------------------------------------------
// Float-float refinement residual of the FP32 / TF32 local solves.  The running solution X is kept
// as float-float pairs (no FP64 instruction in the element loop); the structured operator is the
// same as above: (B + M) X on the diagonal, the x- and z-line derivative sums of -C X, and the
// circulant angular sum of -S X (eq. hdg_local_mat).
//   mode 0: X = D;  mode 1: X += D;  mode 2: X += D and no residual.
// In modes 0 and 1, R = -B^ - A X is written over D (FP32) and maxres[e] = max |R|.
// N1T / NAT fix n1 = p + 1 and N at compile time (0: read from the table).
// ------------------------------------------------------------------------------------------------
constexpr int kResThreads = 512;

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.h, -a.l}; }
// acc += c x for a float-float coefficient c and a staged entry x (FP32 in the first pass, where
// X = D exactly, float-float afterwards)
__device__ __forceinline__ void fma_cx(ff& acc, ff c, float x) { ff_fma_f(acc, x, c); }
__device__ __forceinline__ void fma_cx(ff& acc, ff c, ff x) { ff_fma(acc, c, x); }
__device__ __forceinline__ ff as_ff(float x) { return ff{x, 0.f}; }
__device__ __forceinline__ ff as_ff(ff x) { return x; }
// two adjacent staged columns in one shared load (8 or 16 bytes, aligned: even column offsets)
__device__ __forceinline__ void ld_pair(const float* p, float& a, float& b) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void ld_pair(const ff* p, ff& a, ff& b) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = ff{v.x, v.y};
    b = ff{v.z, v.w};
}

// XS: type of the staged X chunk: float for mode 0 (half the shared memory, so twice the
// columns per pass), float-float for modes 1 and 2
template <int N1T, int NAT, typename XS>
__global__ void __launch_bounds__(kResThreads, 2) k_residual_ff(Tab t, double h, const double* __restrict__ h_elem,
                                                             const double* __restrict__ kappa,
                                                             const double* __restrict__ omega, float* __restrict__ Mall,
                                                             int64_t ld, int64_t estride, ff* __restrict__ Xall, int mode,
                                                             int CWR, double* __restrict__ maxres, int64_t E) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = N1T > 0 ? N1T : t.n1;
    const int N = NAT > 0 ? NAT : t.N;
    const int nm = n1 * n1, nu = nm * N, nin = t.nin, p = n1 - 1;
    // shared memory (residual_ff_smem): X chunk, then the per-element tables at their exact sizes
    XS* Xs = reinterpret_cast<XS*>(smem_raw);  // [nu][CWR]
    ff* dcoef = reinterpret_cast<ff*>(Xs + (size_t)nu * CWR);  // [nu]: B^k_ii + w_i kappa_hat_i
    ff* wd = dcoef + nu;                       // [n1][n1]: w_q D[q][a]
    ff* sxw = wd + nm;                         // [N][n1]: sx_k w_b
    ff* szw = sxw + N * n1;                    // [N][n1]: sz_k w_a
    ff* wrot = szw + N * n1;                   // [N][N]: circulant phase, row k rotated: wc[(k - l) mod N]
    ff* scoef = wrot + N * N;                  // [nm]: w_i omega kappa_hat_i
    int* abv = reinterpret_cast<int*>(scoef + nm);  // [nm]: a | b << 8 of node i
    __shared__ float red[kResThreads / 32];
    const int64_t e = blockIdx.x;
    if (e >= E) return;
    const double he = h_elem ? h_elem[e] : h;
    const double om = omega[e];
    for (int q = threadIdx.x; q < nm; q += kResThreads) {
        wd[q] = ff_from_double(t.w[q / n1] * t.D[q]);
        abv[q] = (q % n1) | ((q / n1) << 8);
        scoef[q] = ff_from_double(t.w[q % n1] * t.w[q / n1] * om * kappa[e * nm + q] * 0.5 * he);
    }
    for (int q = threadIdx.x; q < N * n1; q += kResThreads) {
        const int k = q / n1, b = q - k * n1;
        sxw[q] = ff_from_double(t.sx[k] * t.w[b]);
        szw[q] = ff_from_double(t.sz[k] * t.w[b]);
    }
    for (int q = threadIdx.x; q < N * N; q += kResThreads) {
        const int k = q / N, l = q - k * N;
        wrot[q] = ff_from_double(t.wc[k >= l ? k - l : k - l + N]);
    }
    for (int r = threadIdx.x; r < nu; r += kResThreads) {
        const int k = r / nm, i = r - k * nm;
        const int a = i % n1, b = i / n1;
        double bd = 0.0;
        if (b == 0 && t.sdn[0][k] > 0) bd += t.w[a] * t.sdn[0][k];
        if (a == p && t.sdn[1][k] > 0) bd += t.w[b] * t.sdn[1][k];
        if (b == p && t.sdn[2][k] > 0) bd += t.w[a] * t.sdn[2][k];
        if (a == 0 && t.sdn[3][k] > 0) bd += t.w[b] * t.sdn[3][k];
        dcoef[r] = ff_from_double(bd + t.w[a] * t.w[b] * kappa[e * nm + i] * 0.5 * he);
    }
    float* M = Mall + e * estride;
    ff* X = Xall + e * (int64_t)nu * nin;
    float rmax = 0.f;
    const int rpp = kResThreads / CWR;
    const int tcol = threadIdx.x % CWR, trow = threadIdx.x / CWR;
    // compute mapping: CWR / 2 column pairs per row (CWR is even)
    const int ppp = kResThreads / (CWR / 2);
    const int tpair = threadIdx.x % (CWR / 2), prow = threadIdx.x / (CWR / 2);
    // column chunks: all of them in this block, or (small batches: gridDim.y > 1) every gridDim.y-th
    for (int cs = blockIdx.y * CWR; cs < nin; cs += gridDim.y * CWR) {
        const int col = cs + tcol;
        const bool colok = col < nin;
        __syncthreads();
        // stage D (and X) of this column chunk: batches of independent loads, then the updates
        constexpr int SB = 8;
        for (int rb = trow; rb < nu; rb += SB * rpp) {
            float d[SB];
            ff xo[SB];
#pragma unroll
            for (int u = 0; u < SB; ++u) {
                const int r = rb + u * rpp;
                d[u] = 0.f;
                xo[u] = ff{0.f, 0.f};
                if (colok && r < nu) {
                    d[u] = M[(int64_t)r * ld + nu + col];
                    if (mode != 0) xo[u] = X[(int64_t)r * nin + col];
                }
            }
#pragma unroll
            for (int u = 0; u < SB; ++u) {
                const int r = rb + u * rpp;
                if (r >= nu) break;
                ff v{0.f, 0.f};
                if (colok) {
                    v = (mode == 0) ? ff{d[u], 0.f} : ff_add(xo[u], ff{d[u], 0.f});
                    X[(int64_t)r * nin + col] = v;
                }
                if (mode != 2) {
                    if constexpr (sizeof(XS) == 4) Xs[r * CWR + tcol] = v.h;  // mode 0: v = (d, 0)
                    else Xs[r * CWR + tcol] = v;
                }
            }
        }
        if (mode == 2) continue;
        __syncthreads();
        // compute: each thread takes two adjacent staged columns (c0, c0 + 1), so every coefficient
        // load and every staged-value load serves two entries
        const int c0 = cs + 2 * tpair;
        bool ok[2];
        int tr[2];  // the one nonzero of each column of B^: row tr, value tv
        ff tv[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int col = c0 + u;
            ok[u] = col < nin;
            tr[u] = -1;
            tv[u] = ff{0.f, 0.f};
            if (ok[u]) {
                const int F = col / t.nface, rem = col - F * t.nface;
                const int m = rem / t.half, kk = rem - m * t.half;
                const int kin = t.inc[F][kk];
                tr[u] = kin * nm + face_node(F, m, p);
                tv[u] = ff_from_double(-t.w[m] * t.sdn[F][kin]);
            }
        }
        int k = prow / nm, i = prow - k * nm;
        for (int r = prow; r < nu; r += ppp) {
            if (ok[0]) {
                const int ab = abv[i];
                const int a = ab & 0xff, b = ab >> 8;
                const XS* xk = Xs + (size_t)k * nm * CWR + 2 * tpair;  // angle block k, this column pair
                XS x0, x1;
                ld_pair(xk + i * CWR, x0, x1);
                ff acc[2] = {ff_mul(dcoef[r], as_ff(x0)), ff_mul(dcoef[r], as_ff(x1))};
                ff tx[2] = {}, tz[2] = {};
                const XS* xrow = xk + n1 * b * CWR;  // x-line through node i
                const XS* xcol = xk + a * CWR;       // z-line through node i
#pragma unroll
                for (int q = 0; q < n1; ++q) {
                    const ff wx = wd[q * n1 + a], wz = wd[q * n1 + b];
                    ld_pair(xrow + q * CWR, x0, x1);
                    fma_cx(tx[0], wx, x0);
                    fma_cx(tx[1], wx, x1);
                    ld_pair(xcol + q * n1 * CWR, x0, x1);
                    fma_cx(tz[0], wz, x0);
                    fma_cx(tz[1], wz, x1);
                }
                const XS* xi = Xs + (size_t)i * CWR + 2 * tpair;  // node i across angles
                const ff* wk = wrot + k * N;                      // phase row k (fixed offsets below)
                ff sc[2] = {};
#pragma unroll
                for (int l = 0; l < N; ++l) {
                    const ff w = wk[l];
                    ld_pair(xi + (size_t)l * nm * CWR, x0, x1);
                    fma_cx(sc[0], w, x0);
                    fma_cx(sc[1], w, x1);
                }
                const ff cx = sxw[k * n1 + b], cz = szw[k * n1 + a], cs_ = scoef[i];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const ff ttx = ff_norm(tx[u].h, tx[u].l), ttz = ff_norm(tz[u].h, tz[u].l);
                    const ff cxz = ff_add(ff_mul(cx, ttx), ff_mul(cz, ttz));
                    const ff tsc = ff_norm(sc[u].h, sc[u].l);
                    ff v = ff_add(acc[u], ff_neg(cxz));
                    v = ff_add(v, ff_neg(ff_mul(cs_, tsc)));
                    const ff res = (r == tr[u]) ? ff_add(tv[u], ff_neg(v)) : ff_neg(v);
                    const float rf = __fadd_rn(res.h, res.l);
                    if (ok[u]) {
                        rmax = fmaxf(rmax, fabsf(rf));
                        M[(int64_t)r * ld + nu + c0 + u] = rf;
                    }
                }
            }
            i += ppp;
            while (i >= nm) {
                i -= nm;
                ++k;
            }
        }
    }
    if (mode == 2) return;
    for (int off = 16; off > 0; off >>= 1) rmax = fmaxf(rmax, __shfl_down_sync(0xffffffffu, rmax, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < kResThreads / 32; ++w) m = fmaxf(m, red[w]);
        if (gridDim.y == 1) maxres[e] = (double)m;
        else  // several blocks per element: the maximum of non-negative doubles by their bit patterns (zeroed first)
            atomicMax(reinterpret_cast<unsigned long long*>(maxres + e), (unsigned long long)__double_as_longlong((double)m));
    }
}

// Restriction from the float-float solution: in2out = R^o X, in2sol = (1/N) sum_k X (eqs.
// hdg_local_i2o and ang_ave), sums in float-float, rounded once to the output type.  With D given
// (the last refinement correction, FP32, in the right-hand-side columns of the matrix), the
// restriction uses X + D without writing it back.
__device__ __forceinline__ void ff_store(float* dst, ff v) { *dst = __fadd_rn(v.h, v.l); }
__device__ __forceinline__ void ff_store(double* dst, ff v) { *dst = (double)v.h + (double)v.l; }

template <typename O>
__global__ void __launch_bounds__(kThreads) k_restrict_ff(Tab t, const ff* __restrict__ X, const float* __restrict__ D,
                                                          int64_t dld, int64_t destride, ff inv_n,
                                                          O* __restrict__ in2out, O* __restrict__ in2sol,
                                                          int* __restrict__ estatus, int64_t E) {
    const int nin = t.nin, nm = t.nm, half = t.half;
    const int64_t e = blockIdx.x;
    if (e >= E) return;
    const ff* Xe = X + e * (int64_t)t.nu * nin;
    const float* De = D ? D + e * destride : nullptr;
    auto xval = [&](int row, int c) {
        const ff x = Xe[(int64_t)row * nin + c];
        return De ? ff_add(x, ff{De[(int64_t)row * dld + c], 0.f}) : x;
    };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nrows = nin + nm;
    int bad = 0;
    for (int r = warp; r < nrows; r += kThreads / 32) {
        if (r < nin) {
            const int F = r / t.nface, rem = r - F * t.nface;
            const int m = rem / half, kk = rem - m * half;
            const int row = t.outc[F][kk] * nm + face_node(F, m, t.p);
            for (int c = lane; c < nin; c += 32) {
                const ff v = xval(row, c);
                if (!isfinite(v.h) || !isfinite(v.l)) bad = 1;
                ff_store(in2out + e * (int64_t)nin * nin + (int64_t)r * nin + c, v);
            }
        } else {
            const int i = r - nin;
            for (int c = lane; c < nin; c += 32) {
                ff s{0.f, 0.f};
                for (int k = 0; k < t.N; ++k) s = ff_add(s, xval(k * nm + i, c));
                s = ff_mul(s, inv_n);
                if (!isfinite(s.h) || !isfinite(s.l)) bad = 1;
                ff_store(in2sol + e * (int64_t)nm * nin + (int64_t)i * nin + c, s);
            }
        }
    }
    if (bad) atomicOr(&estatus[e], 4);
}

// ------------------------------------------------------------------------------------------------
// restriction (eqs. hdg_local_i2o and ang_ave): in2out = R^o X, in2sol = (1/N) sum_k X[(k, i)]
// ------------------------------------------------------------------------------------------------

// Source X: either the FP64 buffer (X64, leading dim nin) or the T solution in M (leading dim ld).
template <typename S, typename O>
__global__ void __launch_bounds__(kThreads) k_restrict(Tab t, const S* __restrict__ X, int64_t xld, int64_t xestride,
                                                       int64_t xcol0, O* __restrict__ in2out, O* __restrict__ in2sol,
                                                       int* __restrict__ estatus, int64_t E) {
    const int nin = t.nin, nm = t.nm, half = t.half;
    const int64_t e = blockIdx.x;
    if (e >= E) return;
    const S* Xe = X + e * xestride + xcol0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nrows = t.nin + nm;  // n_out == nin rows of in2out, then nm rows of in2sol
    int bad = 0;
    for (int r = warp; r < nrows; r += kThreads / 32) {
        if (r < nin) {
            const int F = r / t.nface, rem = r - F * t.nface;
            const int m = rem / half, kk = rem - m * half;
            const int row = t.outc[F][kk] * nm + face_node(F, m, t.p);
            for (int c = lane; c < nin; c += 32) {
                const double v = (double)Xe[(int64_t)row * xld + c];
                if (!isfinite(v)) bad = 1;
                in2out[e * (int64_t)nin * nin + (int64_t)r * nin + c] = (O)v;
            }
        } else {
            const int i = r - nin;
            for (int c = lane; c < nin; c += 32) {
                double s = 0.0;
                for (int k = 0; k < t.N; ++k) s += (double)Xe[(int64_t)(k * nm + i) * xld + c];
                s /= t.N;
                if (!isfinite(s)) bad = 1;
                in2sol[e * (int64_t)nm * nin + (int64_t)i * nin + c] = (O)s;
            }
        }
    }
    if (bad) atomicOr(&estatus[e], 4);
}

// ------------------------------------------------------------------------------------------------
// volume source (eqs. hdg_local_f2u_i2u, hdg_local_f2o_i2o): one more right-hand-side column,
// column nu + nin of the matrix, solved with the others
// ------------------------------------------------------------------------------------------------

// F[(k, i)] = w_i (h/2) f[e][k][i]: the source term of the element's equation scaled like every
// other term (divided by (h/2) dth, f h/2 on the reference element)
template <typename T>
__global__ void k_source_column(Tab t, double h, const double* __restrict__ h_elem, const double* __restrict__ src,
                                T* __restrict__ M, int64_t ld, int64_t estride, int64_t E) {
    const int64_t e = blockIdx.x;
    if (e >= E) return;
    const double half_h = 0.5 * (h_elem ? h_elem[e] : h);
    T* Mc = M + e * estride + t.nu + t.nin;
    const double* fe = src + e * (int64_t)t.nu;
    for (int r = threadIdx.x; r < t.nu; r += blockDim.x) {
        const int i = r % t.nm;
        Mc[(int64_t)r * ld] = (T)(t.w[i % t.n1] * t.w[i / t.n1] * half_h * fe[r]);
    }
}

// Refinement of the source column in FP64 (one column per element, so FP64 costs nothing here):
// mode 0: Xs = D; 1: Xs += D, then R = F - A Xs over D; 2: Xs += D only.  A from its structure,
// as the residual kernels of the -B^ columns do.  maxres[e] = max(maxres[e], |R|).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_residual_src(Tab t, double h, const double* __restrict__ h_elem,
                                                           const double* __restrict__ kappa,
                                                           const double* __restrict__ omega,
                                                           const double* __restrict__ src, T* __restrict__ Mall,
                                                           int64_t ld, int64_t estride, double* __restrict__ Xall,
                                                           int mode, double* __restrict__ maxres, int64_t E) {
    __shared__ double xs[ELRT_MAX_N1 * ELRT_MAX_N1 * ELRT_MAX_ANG];
    __shared__ double red[kThreads / 32];
    const int64_t e = blockIdx.x;
    if (e >= E) return;
    const int nu = t.nu, nm = t.nm, n1 = t.n1, N = t.N, p = t.p;
    const double he = h_elem ? h_elem[e] : h;
    const double om = omega[e];
    T* Mc = Mall + e * estride + t.nu + t.nin;
    double* X = Xall + e * (int64_t)nu;
    for (int r = threadIdx.x; r < nu; r += kThreads) {
        const double d = (double)Mc[(int64_t)r * ld];
        const double x = mode == 0 ? d : X[r] + d;
        X[r] = x;
        xs[r] = x;
    }
    if (mode == 2) return;
    __syncthreads();
    double rmax = 0.0;
    for (int r = threadIdx.x; r < nu; r += kThreads) {
        const int k = r / nm, i = r - k * nm, a = i % n1, b = i / n1;
        const double kh = kappa[e * nm + i] * 0.5 * he, wi = t.w[a] * t.w[b];
        double bd = 0.0;
        if (b == 0 && t.sdn[0][k] > 0) bd += t.w[a] * t.sdn[0][k];
        if (a == p && t.sdn[1][k] > 0) bd += t.w[b] * t.sdn[1][k];
        if (b == p && t.sdn[2][k] > 0) bd += t.w[a] * t.sdn[2][k];
        if (a == 0 && t.sdn[3][k] > 0) bd += t.w[b] * t.sdn[3][k];
        double tx = 0.0, tz = 0.0;
        for (int q = 0; q < n1; ++q) {
            tx += t.w[q] * t.D[q * n1 + a] * xs[k * nm + q + n1 * b];
            tz += t.w[q] * t.D[q * n1 + b] * xs[k * nm + a + n1 * q];
        }
        double sc = 0.0;
        for (int l = 0; l < N; ++l) {
            int d = k - l;
            if (d < 0) d += N;
            sc += t.wc[d] * xs[l * nm + i];
        }
        const double ax = (bd + wi * kh) * xs[r] - t.sx[k] * t.w[b] * tx - t.sz[k] * t.w[a] * tz - wi * om * kh * sc;
        const double res = wi * 0.5 * he * src[e * (int64_t)nu + r] - ax;
        rmax = fmax(rmax, fabs(res));
        Mc[(int64_t)r * ld] = (T)res;
    }
    for (int off = 16; off > 0; off >>= 1) rmax = fmax(rmax, __shfl_down_sync(0xffffffffu, rmax, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rmax;
    __syncthreads();
    if (threadIdx.x == 0 && maxres) {
        double m = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) m = fmax(m, red[w]);
        maxres[e] = fmax(maxres[e], m);
    }
}

// f^_u = R^o f_u (outflow rows in skeleton order), (1/N) sum_k f_u[(k, i)] and f_u itself, from
// the solved source column: X + e xestride + r xld is f_u[r] (the FP64 refined copy, or the column
// of the matrix when there was no refinement)
template <typename S>
__global__ void k_restrict_src(Tab t, const S* __restrict__ X, int64_t xld, int64_t xestride, double* __restrict__ f2o,
                               double* __restrict__ f2m, double* __restrict__ f2u, int* __restrict__ estatus,
                               int64_t E) {
    const int64_t e = blockIdx.x;
    if (e >= E) return;
    const S* Xe = X + e * xestride;
    const int nm = t.nm, half = t.half;
    int bad = 0;
    for (int r = threadIdx.x; r < t.nin; r += blockDim.x) {
        const int F = r / t.nface, rem = r - F * t.nface;
        const int m = rem / half, kk = rem - m * half;
        const double v = (double)Xe[(int64_t)(t.outc[F][kk] * nm + face_node(F, m, t.p)) * xld];
        if (!isfinite(v)) bad = 1;
        f2o[e * (int64_t)t.nin + r] = v;
    }
    for (int i = threadIdx.x; i < nm; i += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < t.N; ++k) s += (double)Xe[(int64_t)(k * nm + i) * xld];
        f2m[e * (int64_t)nm + i] = s / t.N;
    }
    if (f2u)
        for (int r = threadIdx.x; r < t.nu; r += blockDim.x) f2u[e * (int64_t)t.nu + r] = (double)Xe[(int64_t)r * xld];
    if (bad) atomicOr(&estatus[e], 4);
}

// A_i2u itself (rows [0, nu) of the solution of the -B^ columns) into in2rad [E][nu][nin]: from the
// float-float X (plus the pending last correction D when it was not written back) ...
template <typename O>
__global__ void __launch_bounds__(kThreads) k_write_rad_ff(Tab t, const ff* __restrict__ X, const float* __restrict__ D,
                                                           int64_t dld, int64_t destride, O* __restrict__ out, int64_t E) {
    const int64_t e = blockIdx.x;
    if (e >= E) return;
    const int nin = t.nin;
    const ff* Xe = X + e * (int64_t)t.nu * nin;
    const float* De = D ? D + e * destride : nullptr;
    O* oe = out + e * (int64_t)t.nu * nin;
    for (int64_t q = threadIdx.x; q < (int64_t)t.nu * nin; q += kThreads) {
        const int r = (int)(q / nin), c = (int)(q - (int64_t)r * nin);
        ff v = Xe[q];
        if (De) v = ff_add(v, ff{De[(int64_t)r * dld + c], 0.f});
        ff_store(oe + q, v);
    }
}

// ... or from a plain buffer (the FP64 solution in the matrix or its FP64 copy)
template <typename S, typename O>
__global__ void __launch_bounds__(kThreads) k_write_rad(Tab t, const S* __restrict__ X, int64_t xld, int64_t xestride,
                                                        O* __restrict__ out, int64_t E) {
    const int64_t e = blockIdx.x;
    if (e >= E) return;
    const int nin = t.nin;
    const S* Xe = X + e * xestride;
    O* oe = out + e * (int64_t)t.nu * nin;
    for (int64_t q = threadIdx.x; q < (int64_t)t.nu * nin; q += kThreads) {
        const int r = (int)(q / nin), c = (int)(q - (int64_t)r * nin);
        oe[q] = (O)(double)Xe[(int64_t)r * xld + c];
    }
}

__global__ void k_flag_residual(const double* __restrict__ maxres, int* __restrict__ estatus, double tol, int64_t E) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < E && !(maxres[e] <= tol)) estatus[e] |= 2;
}

__global__ void k_reduce_status(const int* __restrict__ estatus, const double* __restrict__ maxres, int64_t E,
                                int* __restrict__ nflag, unsigned long long* __restrict__ maxbits) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < E) {
        if (estatus[e]) atomicAdd(nflag, 1);
        if (maxres) {
            double v = maxres[e];
            if (!(v >= 0.0)) v = 1e300;
            atomicMax(maxbits, (unsigned long long)__double_as_longlong(v));
        }
    }
}

__global__ void k_copy_status(const int* __restrict__ src, int32_t* __restrict__ dst, int64_t E) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < E) dst[e] = src[e];
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------------

elrt_status local_assemble_f64(elrt_ctx* ctx, int64_t E, double h, const double* h_elem, const double* kappa,
                               const double* omega, double* A, double* rhs) {
    const Tab& t = ctx->tab;
    elrt_status s = cuda_check(ctx, cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), ctx->stream), "memset flags");
    if (s) return s;
    for (int64_t e0 = 0; e0 < E; e0 += 65535) {
        const int64_t n = std::min<int64_t>(65535, E - e0);
        dim3 grid((unsigned)n, t.N);
        ProfScope ps(ctx, "assemble", 1, (double)n * (8.0 * t.nu * (t.nu + t.nin) + 8.0 * (t.nm + 2)));
        k_assemble<double><<<grid, kThreads, 0, ctx->stream>>>(
            t, h, h_elem ? h_elem + e0 : nullptr, kappa + e0 * t.nm, omega + e0, A + e0 * (int64_t)t.nu * t.nu, t.nu,
            (int64_t)t.nu * t.nu, rhs + e0 * (int64_t)t.nu * t.nin, t.nin, ctx->d_flags);
    }
    s = cuda_check(ctx, cudaGetLastError(), "k_assemble launch");
    if (s) return s;
    s = cuda_check(ctx, cudaMemcpyAsync(ctx->h_pinned, ctx->d_flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
                   "flags read-back");
    if (s) return s;
    s = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "elrt_assemble");
    if (s) return s;
    prof_flush(ctx);
    if (*(int*)ctx->h_pinned) return ctx_fail(ctx, ELRT_EINVAL, "negative/non-finite kappa or h, or omega outside [0,1]");
    return ELRT_OK;
}

namespace {

// algorithmic bytes / flops of the refinement residual: per entry of X (nu x nin) the correction D is
// read, X read (modes 1, 2) and written (8 bytes), R written (modes 0, 1); one multiply-add per
// nonzero of the structured row of A (diagonal, 2 (p + 1) line terms, N angular terms)
double residual_bytes(const Tab& t, size_t st, int mode, int64_t n) {
    const double per = (double)st + 8.0 + (mode != 0 ? 8.0 : 0.0) + (mode != 2 ? (double)st : 0.0);
    return per * t.nu * t.nin * (double)n;
}
double residual_flops(const Tab& t, int mode, int64_t n) {
    return mode == 2 ? (double)t.nu * t.nin * n : 2.0 * (1 + 2 * t.n1 + t.N) * (double)t.nu * t.nin * n;
}
// restriction, algorithmic bytes: every row of the solution read once (the kernels read the outgoing
// rows a second time, for the angular means; a one-pass variant was slower), in2out and in2sol
// written once
double restrict_bytes(const Tab& t, size_t ss, size_t so, int64_t n) {
    return ((double)t.nu * t.nin * ss + (double)(t.nin + t.nm) * t.nin * so) * (double)n;
}

// t: the context's table with nrhs set to the right-hand-side columns of this build
template <typename T, int NB, int QN>
elrt_status run_lu(elrt_ctx* ctx, const Tab& t, T* M, int64_t ld, int64_t estride, int* ipiv, int* estatus, int64_t n,
                   bool resolve) {
    const size_t smem = lu_smem_bytes<T, NB, QN>(t.nu);
    if (smem > 227 * 1024) return ctx_fail(ctx, ELRT_EINVAL, "local system too large for the shared-memory panel");
    cudaError_t e;
    if (!resolve) {
        e = cudaFuncSetAttribute(k_lu_factor_solve<T, NB, QN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_check(ctx, e, "smem attribute");
        const double nu = t.nu, nin = t.nin;
        ProfScope ps(ctx, "lu_factor_solve", 1, (double)n * (2.0 * sizeof(T) * nu * (nu + nin) + 4.0 * nu),
                     (double)n * (2.0 / 3.0 * nu * nu * nu + 2.0 * nu * nu * nin));
        k_lu_factor_solve<T, NB, QN><<<(unsigned)n, kThreads, smem, ctx->stream>>>(t, M, ld, estride, ipiv, estatus, n);
    } else {
        e = cudaFuncSetAttribute(k_lu_resolve<T, NB, QN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_check(ctx, e, "smem attribute");
        const double nu = t.nu, nin = t.nin;
        ProfScope ps(ctx, "lu_resolve", 1, (double)n * (sizeof(T) * (nu * nu + 2.0 * nu * nin) + 4.0 * nu),
                     (double)n * 2.0 * nu * nu * nin);
        k_lu_resolve<T, NB, QN><<<(unsigned)n, kThreads, smem, ctx->stream>>>(t, M, ld, estride, ipiv, n);
    }
    return cuda_check(ctx, cudaGetLastError(), "lu launch");
}

template <typename T>
elrt_status run_residual(elrt_ctx* ctx, double h, const double* h_elem, const double* kappa, const double* omega,
                         T* M, int64_t ld, int64_t estride, double* X64, int mode, double* maxres, int64_t n) {
    const Tab& t = ctx->tab;
    int cwr = 32;
    while (cwr > 1 && (size_t)t.nu * (cwr + 1) * sizeof(double) > 212 * 1024) cwr >>= 1;
    const size_t smem = (size_t)t.nu * (cwr + 1) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_residual<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(ctx, e, "smem attribute");
    ProfScope ps(ctx, "residual", 1, residual_bytes(t, sizeof(T), mode, n), residual_flops(t, mode, n));
    k_residual<T><<<(unsigned)n, kThreads, smem, ctx->stream>>>(t, h, h_elem, kappa, omega, M, ld, estride, X64, mode,
                                                                 cwr, maxres, n);
    return cuda_check(ctx, cudaGetLastError(), "residual launch");
}

// shared memory of the float-float residual for cwr staged columns of xs-byte entries
size_t residual_ff_smem(const Tab& t, int cwr, size_t xs) {
    return (size_t)t.nu * cwr * xs + ((size_t)t.nu + t.nm + 2 * (size_t)t.N * t.n1 + (size_t)t.N * t.N + t.nm) * sizeof(ff) +
           t.nm * sizeof(int);
}
// columns staged per pass: as many as leave room for two blocks per SM (one stages its next
// chunk from HBM while the other computes)
int residual_ff_cwr(const Tab& t, size_t xs) {
    int cwr = 32;
    while (cwr > 1 && residual_ff_smem(t, cwr, xs) > 110 * 1024) cwr >>= 1;
    return cwr;
}

template <int N1T, int NAT, typename XS>
elrt_status launch_residual_ff(elrt_ctx* ctx, double h, const double* h_elem, const double* kappa, const double* omega,
                               float* M, int64_t ld, int64_t estride, ff* X, int mode, double* maxres, int64_t n) {
    const Tab& t = ctx->tab;
    const int cwr = residual_ff_cwr(t, sizeof(XS));
    if (cwr < 2) return ctx_fail(ctx, ELRT_EINVAL, "float-float residual: element too large for two staged columns");
    const size_t smem = residual_ff_smem(t, cwr, sizeof(XS));
    cudaError_t e =
        cudaFuncSetAttribute(k_residual_ff<N1T, NAT, XS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(ctx, e, "smem attribute");
    // a batch too small to fill the GPU spreads each element's column chunks over several blocks
    const int nchunk = (t.nin + cwr - 1) / cwr;
    const int gy = (int)std::max<int64_t>(1, std::min<int64_t>(nchunk, (2 * (int64_t)ctx->sms) / std::max<int64_t>(n, 1)));
    if (gy > 1 && mode != 2) {
        e = cudaMemsetAsync(maxres, 0, (size_t)n * sizeof(double), ctx->stream);
        if (e != cudaSuccess) return cuda_check(ctx, e, "residual maxima");
    }
    ProfScope ps(ctx, "residual", 1, residual_bytes(t, sizeof(float), mode, n), residual_flops(t, mode, n));
    k_residual_ff<N1T, NAT, XS><<<dim3((unsigned)n, (unsigned)gy), kResThreads, smem, ctx->stream>>>(
        t, h, h_elem, kappa, omega, M, ld, estride, X, mode, cwr, maxres, n);
    return cuda_check(ctx, cudaGetLastError(), "residual launch");
}

template <int N1T, int NAT>
elrt_status launch_residual_mode(elrt_ctx* ctx, double h, const double* h_elem, const double* kappa,
                                 const double* omega, float* M, int64_t ld, int64_t estride, ff* X, int mode,
                                 double* maxres, int64_t n) {
    if (mode == 0)
        return launch_residual_ff<N1T, NAT, float>(ctx, h, h_elem, kappa, omega, M, ld, estride, X, mode, maxres, n);
    return launch_residual_ff<N1T, NAT, ff>(ctx, h, h_elem, kappa, omega, M, ld, estride, X, mode, maxres, n);
}

// unrolled shapes for Q6 elements with 16 or 28 angular cells; any other shape reads the table
elrt_status run_residual_ff(elrt_ctx* ctx, double h, const double* h_elem, const double* kappa, const double* omega,
                            float* M, int64_t ld, int64_t estride, ff* X, int mode, double* maxres, int64_t n) {
    const Tab& t = ctx->tab;
    if (t.n1 == 7 && t.N == 16)
        return launch_residual_mode<7, 16>(ctx, h, h_elem, kappa, omega, M, ld, estride, X, mode, maxres, n);
    if (t.n1 == 7 && t.N == 28)
        return launch_residual_mode<7, 28>(ctx, h, h_elem, kappa, omega, M, ld, estride, X, mode, maxres, n);
    return launch_residual_mode<0, 0>(ctx, h, h_elem, kappa, omega, M, ld, estride, X, mode, maxres, n);
}

template <typename O>
elrt_status run_restrict_ff(elrt_ctx* ctx, const ff* X, const float* D, int64_t dld, int64_t destride, O* in2out,
                            O* in2sol, int* estatus, int64_t n) {
    const ff inv_n = ff_from_double_host(1.0 / ctx->tab.N);
    ProfScope ps(ctx, "restrict", 1, restrict_bytes(ctx->tab, D ? sizeof(ff) + sizeof(float) : sizeof(ff), sizeof(O), n));
    k_restrict_ff<O><<<(unsigned)n, kThreads, 0, ctx->stream>>>(ctx->tab, X, D, dld, destride, inv_n, in2out, in2sol,
                                                                estatus, n);
    return cuda_check(ctx, cudaGetLastError(), "restrict launch");
}

template <typename S, typename O>
elrt_status run_restrict(elrt_ctx* ctx, const S* X, int64_t xld, int64_t xestride, int64_t xcol0, O* in2out, O* in2sol,
                         int* estatus, int64_t n) {
    ProfScope ps(ctx, "restrict", 1, restrict_bytes(ctx->tab, sizeof(S), sizeof(O), n));
    k_restrict<S, O><<<(unsigned)n, kThreads, 0, ctx->stream>>>(ctx->tab, X, xld, xestride, xcol0, in2out, in2sol,
                                                               estatus, n);
    return cuda_check(ctx, cudaGetLastError(), "restrict launch");
}

template <typename T, int NB, int QN>
elrt_status build_chunked(elrt_ctx* ctx, int64_t E, double h, const double* h_elem, const double* kappa,
                          const double* omega, int mode, int steps, int out_dtype, void* in2out, void* in2sol,
                          int32_t* elem_status, elrt_local_stats* stats, const elrt_local_extras* ex) {
    const Tab& t = ctx->tab;
    const bool has_src = ex && ex->source;
    Tab tl = t;  // the LU's right-hand sides: the -B^ columns, then the source column
    tl.nrhs = t.nin + (has_src ? 1 : 0);
    const int64_t ld = ((t.nu + tl.nrhs + 31) / 32) * 32;
    const int64_t estride = (int64_t)t.nu * ld;
    const bool ir = (mode != ELRT_LOCAL_FP64);
    double bmax = 0.0;  // max |B^| entry, the scale of the residuals
    for (int F = 0; F < 4; ++F)
        for (int k = 0; k < t.N; ++k)
            for (int m = 0; m < t.n1; ++m) bmax = std::max(bmax, fabs(t.w[m] * t.sdn[F][k]));
    const bool want_res = ir || stats || elem_status;
    const bool tc = (mode == ELRT_LOCAL_TF32_IR);
    const size_t side_per = tc ? tc_lu_side_floats(t, ld) * sizeof(float) : 0;
    // bytes per element: M, ipiv, status, maxres, the FP64 solution when refining / measuring,
    // and the split operand buffers of the tensor-core LU
    const size_t src_per = (has_src && ir) ? (size_t)t.nu * sizeof(double) : 0;  // refined source column
    const size_t per = estride * sizeof(T) + t.nu * sizeof(int) + sizeof(int) + sizeof(double) +
                       (want_res ? (size_t)t.nu * t.nin * sizeof(double) : 0) + side_per + src_per;
    // workspace of one chunk: an eighth of the device memory, at most 32 GB (4096 elements at p = 6,
    // N = 16 on a 288 GB device: one chunk for a 64 x 64 field, half the launches of 16 GB chunks)
    const size_t budget = std::min<size_t>((size_t)32 << 30, ctx->dev_bytes / 8);
    int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(E, (int64_t)(budget / per)));
    if (ctx->tune.local_chunk > 0) chunk = std::min<int64_t>(chunk, ctx->tune.local_chunk);
    if (chunk < E) {  // balance the chunks
        const int64_t nch = (E + chunk - 1) / chunk;
        chunk = (E + nch - 1) / nch;
    }
    elrt_status s = ensure_ws(ctx, &ctx->ws, &ctx->ws_bytes, per * chunk + 4096);
    if (s) return s;
    unsigned char* base = (unsigned char*)ctx->ws;
    T* M = (T*)base;
    double* X64 = (double*)(base + (size_t)chunk * estride * sizeof(T));
    double* maxres = X64 + (want_res ? (size_t)chunk * t.nu * t.nin : 0);
    int* ipiv = (int*)(maxres + chunk);
    int* estat = ipiv + (size_t)chunk * t.nu;
    float* side = tc ? (float*)(((uintptr_t)(estat + chunk) + 255) & ~(uintptr_t)255) : nullptr;
    unsigned char* after_side = tc ? (unsigned char*)(side + (size_t)chunk * tc_lu_side_floats(t, ld))
                                   : (unsigned char*)(estat + chunk);
    double* Xs = src_per ? (double*)(((uintptr_t)after_side + 255) & ~(uintptr_t)255) : nullptr;
    s = cuda_check(ctx, cudaMemsetAsync(ctx->d_flags, 0, 4 * sizeof(int) + 2 * sizeof(unsigned long long), ctx->stream),
                   "memset flags");
    if (s) return s;
    const size_t osz = out_dtype == ELRT_F32 ? sizeof(float) : sizeof(double);
    for (int64_t e0 = 0; e0 < E; e0 += chunk) {
        const int64_t n = std::min(chunk, E - e0);
        const double* he = h_elem ? h_elem + e0 : nullptr;
        const double* ka = kappa + e0 * t.nm;
        const double* om = omega + e0;
        s = cuda_check(ctx, cudaMemsetAsync(estat, 0, n * sizeof(int), ctx->stream), "memset status");
        if (!s && tc) s = cuda_check(ctx, cudaMemsetAsync(ctx->d_flags + kAsmMaxFlag, 0, sizeof(int), ctx->stream), "memset max");
        if (s) return s;
        for (int64_t a0 = 0; a0 < n; a0 += 65535) {
            const int64_t m = std::min<int64_t>(65535, n - a0);
            dim3 grid((unsigned)m, t.N);
            ProfScope ps(ctx, "assemble", 1, (double)m * (sizeof(T) * (double)t.nu * (t.nu + t.nin) + 8.0 * (t.nm + 2)));
            k_assemble<T><<<grid, kThreads, 0, ctx->stream>>>(t, h, he ? he + a0 : nullptr, ka + a0 * t.nm, om + a0,
                                                              M + a0 * estride, ld, estride, nullptr, 0, ctx->d_flags);
        }
        if (has_src)
            k_source_column<T><<<(unsigned)n, kThreads, 0, ctx->stream>>>(t, h, he, ex->source + e0 * t.nu, M, ld,
                                                                        estride, n);
        s = cuda_check(ctx, cudaGetLastError(), "assemble launch");
        if (s) return s;
        // 3xFP16 trailing updates when every entry of the chunk's matrices lies in [kLuF16Max / 4096,
        // kLuF16Max] (the entries are O(1): transport 0.5 at the boundary nodes, absorption w^2 kappa_hat)
        // and no source column rides along (its scale is the caller's); the refinement re-solves then
        // run their forward sweep in 3xFP16 too, each element's residual scaled by a power of two into
        // [0.5, 1), and their backward sweep in 3xTF32
        bool f16 = false;
        if (tc && ctx->lu_products == ELRT_LU_PRODUCTS_AUTO && !has_src) {
            unsigned bits = 0;
            s = cuda_check(ctx, cudaMemcpyAsync(ctx->h_pinned, ctx->d_flags + kAsmMaxFlag, sizeof(unsigned),
                                                cudaMemcpyDeviceToHost, ctx->stream), "read max");
            if (!s) s = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "read max");
            if (s) return s;
            memcpy(&bits, ctx->h_pinned, sizeof(bits));
            float amax;
            memcpy(&amax, &bits, sizeof(amax));
            f16 = amax >= kLuF16Max / 4096.f && amax <= kLuF16Max;
        }
        if constexpr (sizeof(T) == 4) {
            if (tc) s = tc_lu_factor_solve(ctx, M, ld, estride, n, estat, side, ctx->d_flags + 2, tl.nrhs, f16);
            else s = run_lu<T, NB, QN>(ctx, tl, M, ld, estride, ipiv, estat, n, false);
        } else {
            s = run_lu<T, NB, QN>(ctx, tl, M, ld, estride, ipiv, estat, n, false);
        }
        if (s) return s;
        // the source column of the refined modes: its own FP64 copy and residual
        auto src_residual = [&](int rmode) {
            ProfScope ps(ctx, "residual", 1, (double)n * t.nu * (rmode == 2 ? 20.0 : 36.0));
            k_residual_src<T><<<(unsigned)n, kThreads, 0, ctx->stream>>>(t, h, he, ka, om, ex->source + e0 * t.nu, M, ld,
                                                                       estride, Xs, rmode, nullptr, n);
        };
        void* o_i2o = (unsigned char*)in2out + (size_t)e0 * t.nin * t.nin * osz;
        void* o_i2m = (unsigned char*)in2sol + (size_t)e0 * t.nm * t.nin * osz;
        if (want_res) {
            if constexpr (sizeof(T) == 4)
                s = run_residual_ff(ctx, h, he, ka, om, M, ld, estride, (ff*)X64, 0, maxres, n);
            else
                s = run_residual<T>(ctx, h, he, ka, om, M, ld, estride, X64, 0, maxres, n);
            if (Xs) src_residual(0);
            // the last correction needs no residual unless statistics or status words are wanted;
            // on the FP32 path the restriction then adds it on the fly (no pass over X)
            const bool last_residual = stats || elem_status;
            bool pending_d = false;
            for (int it = 0; it < (ir ? steps : 0) && !s; ++it) {
                if constexpr (sizeof(T) == 4) {
                    if (tc) s = tc_lu_resolve(ctx, M, ld, estride, n, side, ctx->d_flags + 2, tl.nrhs, f16, maxres);
                    else s = run_lu<T, NB, QN>(ctx, tl, M, ld, estride, ipiv, estat, n, true);
                } else {
                    s = run_lu<T, NB, QN>(ctx, tl, M, ld, estride, ipiv, estat, n, true);
                }
                if (s) break;
                const int rmode = (it + 1 == steps && !last_residual) ? 2 : 1;
                if (Xs) src_residual(rmode);
                if constexpr (sizeof(T) == 4) {
                    if (rmode == 2) pending_d = true;
                    else s = run_residual_ff(ctx, h, he, ka, om, M, ld, estride, (ff*)X64, rmode, maxres, n);
                } else {
                    s = run_residual<T>(ctx, h, he, ka, om, M, ld, estride, X64, rmode, maxres, n);
                }
            }
            if (s) return s;
            // flag elements whose residual exceeds 1e-10 max|B^| (when the last residual was computed)
            if (!(ir && steps > 0 && !last_residual)) {
                ProfScope ps(ctx, "status");
                k_flag_residual<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(maxres, estat, 1e-10 * bmax, n);
            }
            if constexpr (sizeof(T) == 4) {
                const float* D = pending_d ? (const float*)M + t.nu : nullptr;
                if (ex && ex->in2rad) {
                    void* rad = (unsigned char*)ex->in2rad + (size_t)e0 * t.nu * t.nin * osz;
                    if (out_dtype == ELRT_F32)
                        k_write_rad_ff<float><<<(unsigned)n, kThreads, 0, ctx->stream>>>(t, (const ff*)X64, D, ld, estride,
                                                                                       (float*)rad, n);
                    else
                        k_write_rad_ff<double><<<(unsigned)n, kThreads, 0, ctx->stream>>>(t, (const ff*)X64, D, ld, estride,
                                                                                        (double*)rad, n);
                }
                if (out_dtype == ELRT_F32)
                    s = run_restrict_ff<float>(ctx, (const ff*)X64, D, ld, estride, (float*)o_i2o, (float*)o_i2m, estat,
                                               n);
                else
                    s = run_restrict_ff<double>(ctx, (const ff*)X64, D, ld, estride, (double*)o_i2o, (double*)o_i2m,
                                                estat, n);
            } else {
                if (ex && ex->in2rad) {
                    void* rad = (unsigned char*)ex->in2rad + (size_t)e0 * t.nu * t.nin * osz;
                    if (out_dtype == ELRT_F32)
                        k_write_rad<double, float><<<(unsigned)n, kThreads, 0, ctx->stream>>>(
                            t, X64, t.nin, (int64_t)t.nu * t.nin, (float*)rad, n);
                    else
                        k_write_rad<double, double><<<(unsigned)n, kThreads, 0, ctx->stream>>>(
                            t, X64, t.nin, (int64_t)t.nu * t.nin, (double*)rad, n);
                }
                if (out_dtype == ELRT_F32)
                    s = run_restrict<double, float>(ctx, X64, t.nin, (int64_t)t.nu * t.nin, 0, (float*)o_i2o,
                                                    (float*)o_i2m, estat, n);
                else
                    s = run_restrict<double, double>(ctx, X64, t.nin, (int64_t)t.nu * t.nin, 0, (double*)o_i2o,
                                                     (double*)o_i2m, estat, n);
            }
        } else {
            if (ex && ex->in2rad) {
                void* rad = (unsigned char*)ex->in2rad + (size_t)e0 * t.nu * t.nin * osz;
                if (out_dtype == ELRT_F32)
                    k_write_rad<T, float><<<(unsigned)n, kThreads, 0, ctx->stream>>>(t, M + t.nu, ld, estride, (float*)rad, n);
                else
                    k_write_rad<T, double><<<(unsigned)n, kThreads, 0, ctx->stream>>>(t, M + t.nu, ld, estride, (double*)rad,
                                                                                     n);
            }
            if (out_dtype == ELRT_F32)
                s = run_restrict<T, float>(ctx, M, ld, estride, t.nu, (float*)o_i2o, (float*)o_i2m, estat, n);
            else
                s = run_restrict<T, double>(ctx, M, ld, estride, t.nu, (double*)o_i2o, (double*)o_i2m, estat, n);
        }
        if (s) return s;
        if (has_src) {
            double* fo = ex->f2o + e0 * t.nin;
            double* fm = ex->f2m + e0 * t.nm;
            double* fu = ex->f2u ? ex->f2u + e0 * t.nu : nullptr;
            if (Xs)
                k_restrict_src<double><<<(unsigned)n, kThreads, 0, ctx->stream>>>(t, Xs, 1, t.nu, fo, fm, fu, estat, n);
            else
                k_restrict_src<T><<<(unsigned)n, kThreads, 0, ctx->stream>>>(t, M + t.nu + t.nin, ld, estride, fo, fm, fu,
                                                                           estat, n);
            s = cuda_check(ctx, cudaGetLastError(), "source restriction launch");
            if (s) return s;
        }
        ProfScope ps(ctx, "status", elem_status ? 2 : 1);
        k_reduce_status<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(
            estat, want_res ? maxres : nullptr, n, ctx->d_flags + 1, (unsigned long long*)(ctx->d_flags + 4));
        if (elem_status)
            k_copy_status<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(estat, elem_status + e0, n);
        s = cuda_check(ctx, cudaGetLastError(), "status launch");
        if (s) return s;
    }
    s = cuda_check(ctx, cudaMemcpyAsync(ctx->h_pinned, ctx->d_flags, 4 * sizeof(int) + 2 * sizeof(unsigned long long),
                                        cudaMemcpyDeviceToHost, ctx->stream),
                   "flags read-back");
    if (s) return s;
    s = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "elrt_build_local");
    if (s) return s;
    prof_flush(ctx);
    const int* hf = (const int*)ctx->h_pinned;
    if (hf[0]) return ctx_fail(ctx, ELRT_EINVAL, "negative/non-finite kappa or h, or omega outside [0,1]");
    if (hf[2]) return ctx_fail(ctx, ELRT_ETIMEOUT, "a tensor-core LU wait timed out (code " + std::to_string(hf[2]) + ")");
    if (stats) {
        stats->refine_steps = ir ? steps : 0;
        stats->n_flagged = hf[1];
        unsigned long long bits = *(const unsigned long long*)(hf + 4);
        double mr;
        memcpy(&mr, &bits, sizeof(mr));
        stats->max_rel_residual = want_res ? mr / bmax : 0.0;
    }
    return ELRT_OK;
}

}  // namespace

elrt_status local_build(elrt_ctx* ctx, int64_t E, double h, const double* h_elem, const double* kappa,
                        const double* omega, int mode, int refine_steps, int out_dtype, void* in2out, void* in2sol,
                        int32_t* elem_status, elrt_local_stats* stats, const elrt_local_extras* extras) {
    if (mode == ELRT_LOCAL_FP64)
        return build_chunked<double, 16, 4>(ctx, E, h, h_elem, kappa, omega, mode, refine_steps, out_dtype, in2out,
                                            in2sol, elem_status, stats, extras);
    if (mode == ELRT_LOCAL_FP32_IR || mode == ELRT_LOCAL_TF32_IR)
        return build_chunked<float, 32, 8>(ctx, E, h, h_elem, kappa, omega, mode, refine_steps, out_dtype, in2out,
                                           in2sol, elem_status, stats, extras);
    return ctx_fail(ctx, ELRT_EINVAL, "local mode not available in this build");
}

// ------------------------------------------------------------------------------------------------
// Allocation-free variant of elrt_build_local (see elrt_build_local_static in include/elrt.h).
// Its scratch is one file-scope device array; nothing here allocates device or host memory.
// ------------------------------------------------------------------------------------------------

#include <mutex>

static __device__ __align__(256) unsigned char g_static_scratch[(size_t)ELRT_STATIC_SCRATCH_MIB << 20];

namespace {

constexpr size_t kStaticBytes = (size_t)ELRT_STATIC_SCRATCH_MIB << 20;
constexpr size_t kStaticHead = 256;  // input-validation flag
constexpr int kStaticMaxDevices = 64;
void* g_static_addr[kStaticMaxDevices];
std::once_flag g_static_once[kStaticMaxDevices];
cudaError_t g_static_err[kStaticMaxDevices];

// Device address of the array on the current device.  In host code the symbol itself is only a
// host-side stand-in, so the address is looked up once per device, with that device current.
elrt_status static_scratch(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return ELRT_ECUDA;
    std::call_once(g_static_once[dev],
                   [dev] { g_static_err[dev] = cudaGetSymbolAddress(&g_static_addr[dev], g_static_scratch); });
    if (g_static_err[dev] != cudaSuccess || !g_static_addr[dev]) return ELRT_ECUDA;
    *out = g_static_addr[dev];
    return ELRT_OK;
}

// flags[1] |= every non-zero per-element status word (zero pivot, non-finite result)
__global__ void k_static_status(const int* __restrict__ estat, int64_t n, int* __restrict__ flags) {
    int any = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        any |= estat[e];
    any = __reduce_or_sync(0xffffffffu, any);
    if ((threadIdx.x & 31) == 0 && any) atomicOr(flags + 1, any);
}

template <typename T, int NB, int QN>
elrt_status static_build(const Tab& t, cudaStream_t sm, unsigned char* scratch, int64_t E, double h,
                         const double* h_elem, const double* kappa, const double* omega, int mode, int steps,
                         int out_dtype, void* in2out, void* in2sol) {
    const int64_t ld = ((t.nu + t.nin + 31) / 32) * 32;
    const int64_t estride = (int64_t)t.nu * ld;
    const bool ir = mode != ELRT_LOCAL_FP64;
    const size_t per = estride * sizeof(T) + (ir ? (size_t)t.nu * t.nin * sizeof(double) : 0) + sizeof(double) +
                       (size_t)t.nu * sizeof(int) + sizeof(int) + 64;
    if (per > kStaticBytes - kStaticHead) return ELRT_EINVAL;  // one element does not fit the array
    const size_t lu_smem = lu_smem_bytes<T, NB, QN>(t.nu);
    int cwr = 32;
    while (cwr > 1 && (size_t)t.nu * (cwr + 1) * sizeof(double) > 212 * 1024) cwr >>= 1;
    const size_t res_smem = (size_t)t.nu * (cwr + 1) * sizeof(double);
    if (lu_smem > 227 * 1024) return ELRT_EINVAL;
    const int64_t chunk = std::min<int64_t>(E, (int64_t)((kStaticBytes - kStaticHead) / per));
    int* flags = (int*)scratch;
    T* M = (T*)(scratch + kStaticHead);
    double* X64 = (double*)((unsigned char*)M + (size_t)chunk * estride * sizeof(T));
    double* maxres = X64 + (ir ? (size_t)chunk * t.nu * t.nin : 0);
    int* ipiv = (int*)(maxres + chunk);
    int* estat = ipiv + (size_t)chunk * t.nu;
    if (cudaFuncSetAttribute(k_lu_factor_solve<T, NB, QN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lu_smem) ||
        cudaFuncSetAttribute(k_lu_resolve<T, NB, QN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lu_smem) ||
        cudaFuncSetAttribute(k_residual<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)res_smem))
        return ELRT_ECUDA;
    if (cudaMemsetAsync(flags, 0, 2 * sizeof(int), sm) != cudaSuccess) return ELRT_ECUDA;
    const size_t osz = out_dtype == ELRT_F32 ? sizeof(float) : sizeof(double);
    for (int64_t e0 = 0; e0 < E; e0 += chunk) {
        const int64_t n = std::min(chunk, E - e0);
        const double* he = h_elem ? h_elem + e0 : nullptr;
        const double* ka = kappa + e0 * t.nm;
        const double* om = omega + e0;
        if (cudaMemsetAsync(estat, 0, n * sizeof(int), sm) != cudaSuccess) return ELRT_ECUDA;
        k_assemble<T><<<dim3((unsigned)n, t.N), kThreads, 0, sm>>>(t, h, he, ka, om, M, ld, estride, nullptr, 0, flags);
        k_lu_factor_solve<T, NB, QN><<<(unsigned)n, kThreads, lu_smem, sm>>>(t, M, ld, estride, ipiv, estat, n);
        void* o_i2o = (unsigned char*)in2out + (size_t)e0 * t.nin * t.nin * osz;
        void* o_i2m = (unsigned char*)in2sol + (size_t)e0 * t.nm * t.nin * osz;
        if (ir) {
            k_residual<T><<<(unsigned)n, kThreads, res_smem, sm>>>(t, h, he, ka, om, M, ld, estride, X64, 0, cwr, maxres, n);
            for (int it = 0; it < steps; ++it) {
                k_lu_resolve<T, NB, QN><<<(unsigned)n, kThreads, lu_smem, sm>>>(t, M, ld, estride, ipiv, n);
                k_residual<T><<<(unsigned)n, kThreads, res_smem, sm>>>(t, h, he, ka, om, M, ld, estride, X64, 1, cwr,
                                                                      maxres, n);
            }
            if (out_dtype == ELRT_F32)
                k_restrict<double, float><<<(unsigned)n, kThreads, 0, sm>>>(t, X64, t.nin, (int64_t)t.nu * t.nin, 0,
                                                                           (float*)o_i2o, (float*)o_i2m, estat, n);
            else
                k_restrict<double, double><<<(unsigned)n, kThreads, 0, sm>>>(t, X64, t.nin, (int64_t)t.nu * t.nin, 0,
                                                                            (double*)o_i2o, (double*)o_i2m, estat, n);
        } else {
            if (out_dtype == ELRT_F32)
                k_restrict<T, float><<<(unsigned)n, kThreads, 0, sm>>>(t, M, ld, estride, t.nu, (float*)o_i2o,
                                                                      (float*)o_i2m, estat, n);
            else
                k_restrict<T, double><<<(unsigned)n, kThreads, 0, sm>>>(t, M, ld, estride, t.nu, (double*)o_i2o,
                                                                       (double*)o_i2m, estat, n);
        }
        k_static_status<<<(unsigned)std::min<int64_t>(152, (n + 255) / 256), 256, 0, sm>>>(estat, n, flags);
        if (cudaGetLastError() != cudaSuccess) return ELRT_ECUDA;
    }
    int bad[2] = {0, 0};
    if (cudaMemcpyAsync(bad, flags, sizeof(bad), cudaMemcpyDeviceToHost, sm) != cudaSuccess) return ELRT_ECUDA;
    if (cudaStreamSynchronize(sm) != cudaSuccess) return ELRT_ECUDA;
    return bad[0] ? ELRT_EINVAL : bad[1] ? ELRT_ESINGULAR : ELRT_OK;
}

}  // namespace

extern "C" elrt_status elrt_build_local_static(const elrt_disc* disc, void* stream, int64_t n_elems, double h,
                                               const double* h_elem, const double* kappa, const double* omega,
                                               int32_t mode, int32_t refine_steps, int32_t out_dtype, void* in2out,
                                               void* in2sol) {
    if (!elrt_disc_valid(disc) || n_elems < 0 || (n_elems > 0 && (!kappa || !omega || !in2out || !in2sol)) ||
        (!h_elem && !(h > 0)) || (mode != ELRT_LOCAL_FP64 && mode != ELRT_LOCAL_FP32_IR) ||
        (out_dtype != ELRT_F32 && out_dtype != ELRT_F64) || refine_steps < 0 || refine_steps > 8)
        return ELRT_EINVAL;
    if (n_elems == 0) return ELRT_OK;
    Tab t;
    if (!elrt_fill_tab(disc, &t)) return ELRT_EINVAL;
    void* scratch = nullptr;
    elrt_status s = static_scratch(&scratch);
    if (s) return s;
    cudaStream_t sm = (cudaStream_t)stream;
    if (mode == ELRT_LOCAL_FP64)
        return static_build<double, 16, 4>(t, sm, (unsigned char*)scratch, n_elems, h, h_elem, kappa, omega, mode,
                                           refine_steps, out_dtype, in2out, in2sol);
    return static_build<float, 32, 8>(t, sm, (unsigned char*)scratch, n_elems, h, h_elem, kappa, omega, mode,
                                      refine_steps, out_dtype, in2out, in2sol);
}
