// Batched LU without pivoting with tcgen05 trailing updates (local stage of mode TF32_IR).
//
// The local matrix A = B - C + M - S has a positive semidefinite symmetric part (upwind SBP
// transport, scattering with a symmetric doubly-stochastic phase matrix and albedo <= 1), so
// Gaussian elimination needs no pivoting; its growth stays below 1.6 over optical thicknesses
// 1e-4 .. 1e3.  A pivot below the tolerance marks the element in its status word.
//
// The augmented matrix [A | -B^] of each element (FP32, row-major, leading dimension ld) is
// factored in panels of 64 columns, taken in pairs a = [J, J+64), b = [J+64, J+128):
//   k_diag             (one small block per element): LU of the 64 x 64 diagonal block, published
//                      as U11, L11^T, U11^T and 1 / diag(U11);
//   k_rowcol           (blocks of 128 rows or columns per element): L21 from L21 U11 = A21 written
//                      back to the matrix; U12 from L11 U12 = A12 written back to the matrix and,
//                      transposed (K-major), to one side buffer whose rows hold both panels of the
//                      pair (FP32 values and their low TF32 parts, or FP16 high parts and FP16
//                      remainders).  On the right-hand-side columns this is the forward substitution;
//   k_tc_update<NK, H> (tensor cores): C -= L21 U12 with three products hi*hi + hi*lo + lo*hi of
//                      TF32 parts or (H, when the entries fit FP16's range: the factorisation and
//                      the re-solves' forward sweeps, their residuals scaled per element) FP16
//                      parts, both FP32-level accuracy; FP16 needs half the MMA instructions (K = 16
//                      per instruction against 8).  Panel a is applied with rank 64 to panel b's
//                      columns and rows only; once panel b is factored, the rest of the matrix
//                      takes both panels in one rank-128 update, which moves the C tiles half as
//                      often as two rank-64 updates.  The FP32 operands come in by TMA (U12^T from
//                      the side buffer, C from the matrix); the L21 strip goes straight from the
//                      matrix into tensor memory as TF32 (or FP16) high and low parts.
// Panels left over after the pairs (nu not a multiple of 128) are factored one at a time with
// rank-64 updates; in the backward sweeps a last partial panel joins the panel before it.  The
// backward substitution and the forward/backward sweeps of the refinement re-solves reuse the
// stored factors (L21 and U12 in the matrix, the diagonal blocks) with the same kernels.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>

#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include "elrt_internal.h"
#include "tc_gemm.cuh"

namespace {

constexpr int NBP = 64;     // panel width
constexpr int UTK = 256;    // row of the U12^T side buffer: two consecutive panels (K 0 .. 127), then
                            // the low TF32 parts of the same values (K 128 .. 255)
constexpr int UTL = 128;    // K offset of the low parts
// FP16 side buffer (updates with 3xFP16 products): a row holds the FP16 high parts of both panels
// (K 0 .. 127), then the FP16 rounding of the remainders (K 128 .. 255), 512 bytes
constexpr int UTK16 = 256;
constexpr int UTL16 = 128;
constexpr int UBN = 64;     // trailing-update tile width (N of the MMAs)
constexpr int UCB = UBN / 32;  // 32-column (128-byte) boxes of a C tile

__device__ __forceinline__ float tf32_hi(float a) { return __uint_as_float(__float_as_uint(a) & 0xFFFFE000u); }
// two FP16 values in one 32-bit word, the first in the low half (the order of consecutive K)
__device__ __forceinline__ uint32_t pack_h2(__half a, __half b) {
    return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

// ------------------------------------------------------------------------------------------------
// panel kernels (CUDA cores)
// ------------------------------------------------------------------------------------------------

constexpr int TS = NBP + 1;
constexpr int TI = NBP + 4;                                        // factor row stride: 16-byte aligned rows

// Factor layout per element and panel (the side buffer Tinv): [panel][4][64][64]:
//   [0] U11 (upper, row-major), [1] L11^T (the strictly lower part of the unit-lower L11, transposed),
//   [2] U11^T, [3] row 0: 1 / diag(U11).
// Beyond jb the block is padded with the identity (U_ii = 1), so every consumer can run all 64 steps.
constexpr int kInvMats = 4;
constexpr int kDiagThreads = NBP;  // one thread per column of the diagonal block
// Right-looking LU without pivoting of the 64 x 64 diagonal block, one element per block: thread c
// holds column c in registers.  Step j needs the pivot column j (as left by step j - 1) and the
// pivot row entry D[j][c], which thread c already holds; the owner of column j + 1 publishes its
// column, as updated by step j, for step j + 1, so each step takes one barrier (two buffers).
// Every thread forms its multiplier D[j][c] / D[j][j] itself (D[r][c] -= D[r][j] (D[j][c] / D[j][j]));
// the columns of L are scaled by 1 / pivot once, in shared memory, after the last step.  (Ownership
// is tested on a bit mask: a test c == j would let the compiler index the register array by c.)
__global__ void __launch_bounds__(kDiagThreads) k_diag(int nu, int64_t ld, int64_t estride, float* __restrict__ Mall,
                                                       int J, int jb, float* __restrict__ Tinv, int npanels,
                                                       int* __restrict__ estat, float piv_tol) {
    __shared__ float D[NBP][TS];
    __shared__ __align__(16) float lc[2][NBP];
    const int64_t e = blockIdx.x;
    float* M = Mall + e * estride;
    const int c = threadIdx.x;
    const unsigned long long me = 1ull << c;
    // a pivot below the tolerance is replaced by +-tolerance (the element is marked)
    auto clamp_piv = [&](float piv) { return fabsf(piv) >= piv_tol ? piv : (piv < 0.f ? -piv_tol : piv_tol); };
    float a[NBP];
#pragma unroll
    for (int r = 0; r < NBP; ++r)
        a[r] = (r < jb && c < jb) ? M[(int64_t)(J + r) * ld + J + c] : (r == c ? 1.f : 0.f);
    if (c == 0) {
#pragma unroll
        for (int r = 0; r < NBP; ++r) lc[0][r] = a[r];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NBP; ++j) {
        const float* col = lc[j & 1];
        if (c > j) {
            const float m = a[j] * (1.f / clamp_piv(col[j]));
#pragma unroll
            for (int r = j + 1; r < NBP; ++r) a[r] = fmaf(-col[r], m, a[r]);
        }
        if (j + 1 < NBP && ((me >> (j + 1)) & 1ull)) {
#pragma unroll
            for (int r = j + 1; r < NBP; ++r) lc[(j + 1) & 1][r] = a[r];
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < NBP; ++r) D[r][c] = a[r];
    __syncthreads();
    {  // column c of L: D[r][c] / pivot for r > c; the (clamped) pivot on the diagonal
        const float raw = D[c][c], piv = clamp_piv(raw);
        if (c < jb && piv != raw) atomicOr(&estat[e], 1);
        const float rp = 1.f / piv;
        D[c][c] = piv;
        for (int r = c + 1; r < NBP; ++r) D[r][c] *= rp;
    }
    __syncthreads();
    for (int idx = c; idx < jb * jb; idx += kDiagThreads) {
        const int r = idx / jb, cc = idx % jb;
        M[(int64_t)(J + r) * ld + J + cc] = D[r][cc];
    }
    float* Uo = Tinv + ((int64_t)e * npanels + J / NBP) * kInvMats * NBP * NBP;
    float* LT = Uo + NBP * NBP;
    float* UT = LT + NBP * NBP;
    float* rd = UT + NBP * NBP;
    for (int idx = c; idx < NBP * NBP; idx += kDiagThreads) {
        const int r = idx / NBP, cc = idx % NBP;
        Uo[idx] = cc >= r ? D[r][cc] : 0.f;   // U11
        LT[idx] = cc > r ? D[cc][r] : 0.f;    // LT[r][c] = L[c][r], strictly lower part
        UT[idx] = cc <= r ? D[cc][r] : 0.f;   // UT[r][c] = U[c][r]
    }
    rd[c] = 1.f / D[c][c];
}

// Triangular solves of one row or column held in registers, with the factor in shared memory
// (row stride TI) and the reciprocal diagonal rd:
//   SolveKind 0 (row of L21):  x U = a     ->  x_i = a_i / U_ii, a_j -= x_i U[i][j] for j > i
//   SolveKind 1 (forward):     L y = a     ->  y_i = a_i,        a_j -= LT[i][j] y_i for j > i
//   SolveKind 2 (backward):    U y = a     ->  y_i = a_i / U_ii, a_j -= UT[i][j] y_i for j < i
// (right-looking: every step updates independent accumulators).  Each finished 4-wide block of the
// result is handed to put(b, float4): ascending b for kinds 0 and 1, descending for kind 2.
template <int SolveKind, typename Put>
__device__ __forceinline__ void tri_solve(float (&a)[NBP], const float* __restrict__ T, const float* __restrict__ rd,
                                          Put put) {
    if constexpr (SolveKind != 2) {
#pragma unroll
        for (int b = 0; b < NBP / 4; ++b) {
            float y[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = 4 * b + q;
                const float x = SolveKind == 0 ? a[i] * rd[i] : a[i];
                y[q] = x;
                const float* Ti = T + i * TI;
                const int j0 = (i + 4) & ~3;  // scalars up to the next 16-byte boundary, then float4
#pragma unroll
                for (int j = i + 1; j < j0; ++j) a[j] = fmaf(-x, Ti[j], a[j]);
#pragma unroll
                for (int j = j0; j < NBP; j += 4) {
                    const float4 u = *reinterpret_cast<const float4*>(Ti + j);
                    a[j] = fmaf(-x, u.x, a[j]);
                    a[j + 1] = fmaf(-x, u.y, a[j + 1]);
                    a[j + 2] = fmaf(-x, u.z, a[j + 2]);
                    a[j + 3] = fmaf(-x, u.w, a[j + 3]);
                }
            }
            put(b, make_float4(y[0], y[1], y[2], y[3]));
        }
    } else {
#pragma unroll
        for (int b = NBP / 4 - 1; b >= 0; --b) {
            float y[4];
#pragma unroll
            for (int q = 3; q >= 0; --q) {
                const int i = 4 * b + q;
                const float x = a[i] * rd[i];
                y[q] = x;
                const float* Ti = T + i * TI;
                const int j1 = i & ~3;  // float4 below the 16-byte boundary, then scalars
#pragma unroll
                for (int j = 0; j < j1; j += 4) {
                    const float4 u = *reinterpret_cast<const float4*>(Ti + j);
                    a[j] = fmaf(-x, u.x, a[j]);
                    a[j + 1] = fmaf(-x, u.y, a[j + 1]);
                    a[j + 2] = fmaf(-x, u.z, a[j + 2]);
                    a[j + 3] = fmaf(-x, u.w, a[j + 3]);
                }
#pragma unroll
                for (int j = j1; j < i; ++j) a[j] = fmaf(-x, Ti[j], a[j]);
            }
            put(b, make_float4(y[0], y[1], y[2], y[3]));
        }
    }
}

// Row/column work of one panel.  The work items are (element, tile): tiles 0 .. nrt-1 of an
// element are row tiles over rows [r_begin, r_end) (the factorisation only): x = a U11^{-1}
// written back to the matrix; the remaining nct tiles are column tiles over columns [c_begin,
// c_end): y = L11^{-1} a (col_mode 0: factorisation and forward sweep) or y = U11^{-1} a
// (col_mode 1: backward sweep), written back to the matrix (rows < jb) and, transposed, to the side
// buffer Ut[e][column][koff .. koff + 63] (zero beyond jb), with its low TF32 parts at K offset
// UTL + koff.  Persistent, four blocks of 128 threads per SM (one staging buffer each, 128
// registers per thread): each block walks its items, copying an item's 64-wide block and the factor
// of the diagonal block with 16-byte cp.async copies, solving and storing it; the blocks of an SM
// overlap one another's copies and stores.  (One block per SM with two staging buffers, copies of
// the next item in flight, measured 23% slower: 8 warps per SM were too few to hide the
// shared-memory latency of the substitutions.)
constexpr int RS = NBP + 4;                        // staging row stride: 16-byte aligned rows
// one thread per row or column of a tile, PTILE of them; one staging buffer per block
template <int PTILE>
struct RcCfg {
    static constexpr int BUF = PTILE * RS + (NBP + 1) * RS;  // floats: staging + factor + 1/diag
    static constexpr int SMEM = BUF * (int)sizeof(float);
    static constexpr int PER_SM = PTILE == 256 ? 2 : 4;      // resident blocks per SM
    static_assert(PTILE * RS >= NBP * PTILE, "the staging area holds a 64 x PTILE column block");
};
// 128-row tiles, four blocks per SM: measured 2 % faster than 256-row tiles with two blocks per SM
// (the same 16 warps, more independent copy / solve / store phases to overlap)
constexpr int kRcTile = 128;

__device__ __forceinline__ void cp_async16(float* smem, const float* gmem, bool valid) {
    // src-size 0 fills the 16 bytes with zeros and reads nothing
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::smem_u32(smem)), "l"(gmem),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// KIND: 0 = row tiles (factorisation), 1 = column tiles of the factorisation / forward sweep,
// 2 = column tiles of the backward sweep; one unrolled solve per instantiation
// Scale of an element's FP16 operands in a refinement re-solve: the power of two that brings its
// largest residual entry into [0.5, 1), so that the residual and its forward substitution sit in
// FP16's normal range (residuals are ~1e-7 of the O(1) right-hand sides); 1 without a residual
// (the factorisation) or for a zero or non-finite one.  Powers of two scale and unscale exactly.
__device__ __forceinline__ float res_scale(const double* __restrict__ res_max, int64_t e) {
    if (!res_max) return 1.f;
    const double v = res_max[e];
    if (!(v > 0.0) || !isfinite(v)) return 1.f;
    int ex;
    frexp(v, &ex);  // v = f 2^ex, f in [0.5, 1)
    return ldexpf(1.f, -max(-120, min(120, ex)));
}

template <int KIND, int PTILE>
__global__ void __launch_bounds__(PTILE, RcCfg<PTILE>::PER_SM) k_rowcol(int nu, int64_t ld, int64_t estride, float* __restrict__ Mall, int J,
                                                   int jb, const float* __restrict__ Tinv, int npanels, int64_t E,
                                                   int r_begin, int r_end, int nrt, int c_begin, int c_end, int nct,
                                                   float* __restrict__ Ut, int koff, int ut16,
                                                   const double* __restrict__ res_max) {
    constexpr int col_mode = KIND == 2 ? 1 : 0;
    extern __shared__ __align__(16) float sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, t = threadIdx.x;
    const int ntl = nrt + nct;
    const int64_t W = E * ntl;
    // issue the copies of item w into buffer b
    auto load = [&](int64_t w, int b) {
        float* S = sm + b * RcCfg<PTILE>::BUF;
        float* T = S + PTILE * RS;
        const int64_t e = w / ntl;
        const int tile = (int)(w - e * ntl);
        const float* M = Mall + e * estride;
        const float* inv = Tinv + ((int64_t)e * npanels + J / NBP) * kInvMats * NBP * NBP;
        if (tile < nrt) {
            const int r0 = r_begin + tile * PTILE, nr = min(PTILE, r_end - r0);
            for (int idx = t; idx < PTILE * (NBP / 4); idx += PTILE) {
                const int rr = idx >> 4, j4 = idx & 15;
                const bool ok = rr < nr && 4 * j4 < jb;
                cp_async16(S + rr * RS + 4 * j4, ok ? M + (int64_t)(r0 + rr) * ld + J + 4 * j4 : M, ok);
            }
            // U11 (row i: U[i][j])
        } else {
            const int c0 = c_begin + (tile - nrt) * PTILE, nc = min(PTILE, c_end - c0);
            for (int idx = t; idx < NBP * (PTILE / 4); idx += PTILE) {
                const int k = idx / (PTILE / 4), c4 = idx % (PTILE / 4);
                const bool ok = k < jb && 4 * c4 < nc;
                cp_async16(S + k * PTILE + 4 * c4, ok ? M + (int64_t)(J + k) * ld + c0 + 4 * c4 : M, ok);
            }
            inv += (col_mode == 0 ? 1 : 2) * NBP * NBP;  // L11^T or U11^T
        }
        for (int idx = t; idx < NBP * (NBP / 4); idx += PTILE) {
            const int r = idx >> 4, c4 = idx & 15;
            cp_async16(T + r * RS + 4 * c4, inv + r * NBP + 4 * c4, true);
        }
        if (t < NBP / 4) {  // 1 / diag(U11)
            const float* rdg = Tinv + ((int64_t)e * npanels + J / NBP) * kInvMats * NBP * NBP + 3 * NBP * NBP;
            cp_async16(T + NBP * RS + 4 * t, rdg + 4 * t, true);
        }
    };
    const int b = 0;
    for (int64_t w = blockIdx.x; w < W; w += gridDim.x) {
        load(w, b);
        cp_async_commit();
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
        float* S = sm + b * RcCfg<PTILE>::BUF;
        const float* T = S + PTILE * RS;
        const int64_t e = w / ntl;
        const int tile = (int)(w - e * ntl);
        float* M = Mall + e * estride;
        if constexpr (KIND == 0) {
            const int r0 = r_begin + tile * PTILE, nr = min(PTILE, r_end - r0);
            if (t < nr) {  // x U11 = a, written over the row it came from
                float a[NBP];
#pragma unroll
                for (int i = 0; i < NBP; ++i) a[i] = S[t * RS + i];
                float* out = S + t * RS;
                tri_solve<0>(a, T, T + NBP * RS, [&](int bb, float4 v) { *reinterpret_cast<float4*>(out + 4 * bb) = v; });
            }
            __syncthreads();
            // two rows per warp pass, 16-byte stores (a half warp per row; jb % 4 == 0 except in a
            // last panel narrower than 4, which takes the scalar path)
            if ((jb & 3) == 0 && (J & 3) == 0 && (ld & 3) == 0) {
                const int hrow = lane >> 4, q = lane & 15;
                for (int rr = 2 * warp + hrow; rr < nr; rr += 2 * (PTILE / 32))
                    if (4 * q < jb)
                        *reinterpret_cast<float4*>(M + (int64_t)(r0 + rr) * ld + J + 4 * q) =
                            *reinterpret_cast<const float4*>(S + rr * RS + 4 * q);
            } else {
                for (int rr = warp; rr < nr; rr += PTILE / 32)
                    for (int j = lane; j < jb; j += 32) M[(int64_t)(r0 + rr) * ld + J + j] = S[rr * RS + j];
            }
        } else if constexpr (KIND != 0) {
            const int c0 = c_begin + (tile - nrt) * PTILE, nc = min(PTILE, c_end - c0);
            float a[NBP];
            if (t < nc) {
#pragma unroll
                for (int k = 0; k < NBP; ++k) a[k] = S[k * PTILE + t];
            }
            __syncthreads();  // S is reused: from [k][column] staging to [column][i] results
            if (t < nc) {
                // L11 y = a (forward) or U11 y = a (backward)
                const int c = c0 + t;
                float* mc = M + (int64_t)J * ld + c;
                float* sr = S + t * RS;
                auto put = [&](int bb, float4 v) {
                    const int i = 4 * bb;
                    if (i < jb) mc[(int64_t)i * ld] = v.x;
                    if (i + 1 < jb) mc[(int64_t)(i + 1) * ld] = v.y;
                    if (i + 2 < jb) mc[(int64_t)(i + 2) * ld] = v.z;
                    if (i + 3 < jb) mc[(int64_t)(i + 3) * ld] = v.w;
                    *reinterpret_cast<float4*>(sr + i) = v;
                };
                tri_solve<KIND>(a, T, T + NBP * RS, put);
            }
            __syncthreads();
            // two columns per warp pass (a half warp per column), 16-byte stores of the value and of
            // its low TF32 part, split once (UTK, UTL and koff are multiples of 4); or, for the
            // 3xFP16 updates, 8-byte stores of the FP16 high parts and of the FP16 remainders
            float* ut = Ut + e * ld * UTK + koff;
            if (ut16) {
                __half* uh = reinterpret_cast<__half*>(Ut) + e * ld * UTK16 + koff;
                const int hcol = lane >> 4, q = lane & 15;
                // the forward sweep of a scaled re-solve (kind 1); 1 in the factorisation
                const float sc = KIND == 1 ? res_scale(res_max, e) : 1.f;
                for (int cc = 2 * warp + hcol; cc < nc; cc += 2 * (PTILE / 32)) {
                    float4 v = *reinterpret_cast<const float4*>(S + cc * RS + 4 * q);
                    v = make_float4(v.x * sc, v.y * sc, v.z * sc, v.w * sc);
                    const __half h0 = __float2half_rn(v.x), h1 = __float2half_rn(v.y), h2 = __float2half_rn(v.z),
                                 h3 = __float2half_rn(v.w);
                    const __half l0 = __float2half_rn(v.x - __half2float(h0)), l1 = __float2half_rn(v.y - __half2float(h1)),
                                 l2 = __float2half_rn(v.z - __half2float(h2)), l3 = __float2half_rn(v.w - __half2float(h3));
                    *reinterpret_cast<uint2*>(uh + (int64_t)(c0 + cc) * UTK16 + 4 * q) = make_uint2(pack_h2(h0, h1), pack_h2(h2, h3));
                    *reinterpret_cast<uint2*>(uh + (int64_t)(c0 + cc) * UTK16 + UTL16 + 4 * q) = make_uint2(pack_h2(l0, l1), pack_h2(l2, l3));
                }
            } else {
                const int hcol = lane >> 4, q = lane & 15;
                for (int cc = 2 * warp + hcol; cc < nc; cc += 2 * (PTILE / 32)) {
                    const float4 v = *reinterpret_cast<const float4*>(S + cc * RS + 4 * q);
                    const float4 lo = make_float4(v.x - tf32_hi(v.x), v.y - tf32_hi(v.y), v.z - tf32_hi(v.z),
                                                  v.w - tf32_hi(v.w));
                    *reinterpret_cast<float4*>(ut + (int64_t)(c0 + cc) * UTK + 4 * q) = v;
                    *reinterpret_cast<float4*>(ut + (int64_t)(c0 + cc) * UTK + UTL + 4 * q) = lo;
                }
            }
        }
        __syncthreads();  // the buffer is refilled by the next item's copies
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// ------------------------------------------------------------------------------------------------
// trailing update on the tensor cores
// ------------------------------------------------------------------------------------------------

__device__ __forceinline__ void tma_load_3d(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
            tc::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(tc::smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// shared -> global tensor copy (bulk group); the box starts at non-negative coordinates
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(tc::smem_u32(src)), "r"(x), "r"(y), "r"(z)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// kind::f16 with FP16 A and B (format code 0), FP32 D, K-major operands
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// 32 consecutive 32-bit TMEM columns of this thread's lane (shape 32x32b: the warp covers the 32
// lanes of its quarter) from registers; visible to later tcgen05 operations after tmem_st_wait
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float (&v)[32]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])), "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])), "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])), "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])), "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])), "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31])) : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// D (TMEM) (+)= A (TMEM, M x K, one row per lane, two FP16 elements of consecutive K per 32-bit
// column, the first in the low half) x B (shared memory, FP16, K-major): K = 16 per instruction
__device__ __forceinline__ void mma_f16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                           uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate));
}

// D (TMEM) (+)= A (TMEM, M x K, one row per lane, one 32-bit element per column) x B (shared memory)
__device__ __forceinline__ void mma_tf32_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate));
}


// Persistent trailing update C -= L U of rank NK = 64 (one panel) or 128 (two consecutive panels,
// the second already factored against the first; H: FP16 operands, as the notes after the role
// list say): one CTA per SM walks the work items (element,
// 128-row strip) of the launch, the strips of one element consecutively (their U12^T tiles are
// shared through L2).  The L21 strip of an item (columns J .. J+NK-1 of its 128 rows, FP32,
// straight from the matrix) lives in tensor memory as TF32 high and low parts, in 64-column halves
// that rotate through three slots of 128 columns (64 high + 64 low) beside the two accumulators:
// while an item's tiles run, the next item's first half (at NK = 64 the next two strips) is
// already in place and its second half is loaded into registers, ready for the slot the current
// item frees; the first tile of an item issues the passes of its first half before it waits for
// the second.  Shared memory holds two rings that never drain between items: the U12^T tiles
// (64 columns x NK, the FP32 values, which serve as their own TF32 high part, and their low parts,
// both split once by the panel solve; 4 stages at NK = 64, 2 at NK = 128) and the C tiles (128
// rows x 64 columns as two 128-byte-wide boxes, 3 stages).  A U stage is released by the MMA
// commit, a C stage by the store warp, so neither ring waits for the other.  Doubling K halves the
// C bytes per flop: at NK = 64 the update is bound by the C traffic (48 TF32 flops per byte
// issued), at NK = 128 the tensor pipe and HBM are about balanced.
//   warp 0       TMA producer of both rings;
//   warp 1       TMEM allocation; one thread issues the 3xTF32 MMAs (hi*hi + lo*hi + hi*lo,
//                M = 128, N = 64, K = 8, A from tensor memory) into one of two TMEM accumulators;
//   warps 2-5,   epilogue: accumulator (tcgen05.ld) and staged C tile -> C - L U, written back
//   10-13        into the staged tile (warps 2-5 the first 32-column box, 10-13 the second);
//   warp 14      stores each finished tile with TMA tensor stores (the store map's extents are
//                r_end rows and c_end columns, so rows and columns outside the update are
//                clipped) and releases the C stage once the store has read it;
//   warps 6-9    strip preparation: each thread loads one row of a strip half (columns at or
//                beyond jb are 0) into registers, waits for a free slot, splits the row and
//                writes it to its TMEM lane (tcgen05.st).
// U12^T comes from the side buffer [E][ld][UTK] (column-major U12 of the panel pair: K offset 0
// for the first panel, 64 for the second, their low parts UTL further); an NK = 64 update reads
// the half at K offset koff.  With H the side buffer is FP16 ([E][ld][UTK16], the FP16 roundings
// and those of the remainders), the strip preparation packs two FP16 values per TMEM column, and
// an MMA covers K = 16 with the same TMEM-column and descriptor strides as a TF32 one of K = 8.  Every wait is bounded; on a timeout the CTA records a code in *err,
// stops issuing work, lets its copies land and frees its TMEM.
template <int NK, bool H = false>
struct UpdCfg {
    static constexpr int KW = H ? 64 : 32;         // K per 128-byte box row (FP16 or FP32)
    static constexpr int KB = NK / KW;             // K boxes of a U12^T tile
    static constexpr int U_BOX = UBN * 128;        // one box: 64 rows x 128 bytes
    static constexpr int U_STAGE = 2 * KB * U_BOX; // FP32 U12^T tile (KB boxes), then its low part
    static constexpr int U_TX = U_STAGE;
    static constexpr int C_BOX = 128 * 32 * 4;     // one 32-column box of the C tile
    static constexpr int C_STAGE = UCB * C_BOX;
    static constexpr int NU = NK == 64 ? 4 : 2;    // U stages
    static constexpr int NC = 3;                   // C stages
    static constexpr int NH = NK / 64;             // 64-column strip halves per item
    static constexpr int BYTES = NU * U_STAGE + NC * C_STAGE;
    static constexpr int TOTAL = BYTES + 1024 + 512;
};
static_assert(UpdCfg<64>::TOTAL <= 227 * 1024 && UpdCfg<128>::TOTAL <= 227 * 1024 &&
                  UpdCfg<64, true>::TOTAL <= 227 * 1024 && UpdCfg<128, true>::TOTAL <= 227 * 1024,
              "trailing-update shared memory");
// tensor memory: accumulators at columns [0, 2 UBN); strip slot s (of kSlots): the high part of a
// 64-column half at 2 UBN + 128 s, its low part 64 columns further
constexpr int kSlots = 3;
__host__ __device__ constexpr uint32_t slot_col(int s, int lo) {
    return (uint32_t)(2 * UBN) + 128u * (uint32_t)s + 64u * (uint32_t)lo;
}
static_assert(slot_col(kSlots - 1, 1) + 64 <= 512, "tensor memory");
static_assert(UCB == 2, "two epilogue warp groups, one per 32-column box of a C tile");
constexpr int kStripThreads = 480;
constexpr int kEpiWarps = 8;
constexpr uint32_t kTmemCols = 512;

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

template <int NK, bool H>
__global__ void __launch_bounds__(kStripThreads, 1)
    k_tc_update(const __grid_constant__ CUtensorMap tM, const __grid_constant__ CUtensorMap tU,
                const __grid_constant__ CUtensorMap tS, float* __restrict__ Mall, int nu, int64_t ld, int64_t estride,
                int64_t E, int J, int jb, int koff, int r0, int r_end, int c0, int c_end, int* __restrict__ err,
                const double* __restrict__ res_max) {
    using Cfg = UpdCfg<NK, H>;
    constexpr int NU = Cfg::NU, NC = Cfg::NC, NH = Cfg::NH, KB = Cfg::KB, KW = Cfg::KW;
    constexpr int ULO = H ? UTL16 : UTL;  // K offset of the low parts in the side buffer
    extern __shared__ __align__(1024) unsigned char ssm_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)ssm_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* ustage0 = base;                                  // [NU]: U12^T tile and low part (2 KB boxes)
    unsigned char* cstage0 = base + NU * Cfg::U_STAGE;              // [NC]: C tile (UCB boxes)
    uint64_t* s_ready = (uint64_t*)(base + Cfg::BYTES);            // [kSlots]
    uint64_t* s_empty = s_ready + kSlots;                           // [kSlots]
    uint64_t* u_full = s_empty + kSlots;                            // [NU]
    uint64_t* u_empty = u_full + NU;                                // [NU]
    uint64_t* c_full = u_empty + NU;                                // [NC]
    uint64_t* c_done = c_full + NC;                                 // [NC]
    uint64_t* c_empty = c_done + NC;                                // [NC]
    uint64_t* acc_full = c_empty + NC;                              // [2]
    uint64_t* acc_empty = acc_full + 2;                             // [2]
    uint32_t* tmem_slot = (uint32_t*)(acc_empty + 2);
    volatile int* abort = (volatile int*)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nstrips = (r_end - r0 + 127) / 128;
    const int64_t W = (int64_t)nstrips * E;
    const int ntile = (c_end - c0 + UBN - 1) / UBN;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kSlots; ++i) {
            tc::mbar_init(&s_ready[i], 4);
            tc::mbar_init(&s_empty[i], 1);
        }
        for (int i = 0; i < NU; ++i) {
            tc::mbar_init(&u_full[i], 1);
            tc::mbar_init(&u_empty[i], 1);
        }
        for (int i = 0; i < NC; ++i) {
            tc::mbar_init(&c_full[i], 1);
            tc::mbar_init(&c_done[i], kEpiWarps);
            tc::mbar_init(&c_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&acc_full[i], 1);
            tc::mbar_init(&acc_empty[i], kEpiWarps);
        }
        *abort = 0;
        tc::fence_barrier_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    int committed = 0, issued_u = 0, issued_c = 0;
    if (warp == 0 && lane == 0) {
        bool ok = true;
        int g = 0;
        for (int64_t w = blockIdx.x; w < W && ok; w += gridDim.x) {
            const int64_t e = w / nstrips;
            const int m0 = r0 + (int)(w - e * nstrips) * 128;
            for (int t = 0; t < ntile; ++t, ++g) {
                const int su = g % NU, sc = g % NC;
                const int n0 = c0 + t * UBN;
                if (!tc::mbar_wait(&u_empty[su], ((g / NU) & 1) ^ 1, abort)) {
                    ok = false;
                    break;
                }
                unsigned char* us = ustage0 + su * Cfg::U_STAGE;
                tc::mbar_expect_tx(&u_full[su], Cfg::U_TX);
                for (int kb = 0; kb < KB; ++kb) {
                    tma_load_3d(&tU, &u_full[su], us + kb * Cfg::U_BOX, koff + kb * KW, n0, (int)e);
                    tma_load_3d(&tU, &u_full[su], us + (KB + kb) * Cfg::U_BOX, ULO + koff + kb * KW, n0, (int)e);
                }
                ++issued_u;
                if (!tc::mbar_wait(&c_empty[sc], ((g / NC) & 1) ^ 1, abort)) {
                    ok = false;
                    break;
                }
                unsigned char* cs = cstage0 + sc * Cfg::C_STAGE;
                tc::mbar_expect_tx(&c_full[sc], Cfg::C_STAGE);
                for (int cb = 0; cb < UCB; ++cb) tma_load_3d(&tM, &c_full[sc], cs + cb * Cfg::C_BOX, n0 + 32 * cb, m0, (int)e);
                ++issued_c;
            }
        }
        if (!ok) {
            if (err) atomicOr(err, 64);
            *abort = 1;
        }
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = H ? idesc_f16(128, UBN) : idesc_tf32(128, UBN);
        bool ok = true;
        int g = 0, i = 0;
        for (int64_t w = blockIdx.x; w < W && ok; w += gridDim.x, ++i) {
            for (int t = 0; t < ntile; ++t, ++g) {
                const int su = g % NU, a = g & 1;
                if (!tc::mbar_wait(&acc_empty[a], ((g >> 1) & 1) ^ 1, abort) ||
                    !tc::mbar_wait(&u_full[su], (g / NU) & 1, abort)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                unsigned char* us = ustage0 + su * Cfg::U_STAGE;
                const uint32_t d = tmem + (uint32_t)(a * UBN);
                uint32_t acc = 0;
#pragma unroll
                for (int j = 0; j < NH; ++j) {  // strip halves: K columns 64 j .. 64 j + 63
                    const int h = i * NH + j, sl = h % kSlots;
                    // the item's first tile waits for each half (each wait the issuing thread makes
                    // costs MMA issue slots; the slot stays filled until this item's commit below)
                    if (t == 0) {
                        if (!tc::mbar_wait(&s_ready[sl], (h / kSlots) & 1, abort)) {
                            ok = false;
                            break;
                        }
                        tc::tc_fence_after();
                    }
                    const uint32_t a_hi = tmem + slot_col(sl, 0), a_lo = tmem + slot_col(sl, 1);
                    if constexpr (H) {  // one 64-wide K box per half; K = 16 per instruction (8 TMEM columns, 32 bytes)
                        const uint64_t bh = tc::sw128_desc(tc::smem_u32(us + j * Cfg::U_BOX));
                        const uint64_t bl = tc::sw128_desc(tc::smem_u32(us + (KB + j) * Cfg::U_BOX));
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint32_t kc = (uint32_t)(k * 8);
                            mma_f16_ta(d, a_hi + kc, bh + 2 * k, idesc, acc);
                            acc = 1;
                            mma_f16_ta(d, a_lo + kc, bh + 2 * k, idesc, 1);
                            mma_f16_ta(d, a_hi + kc, bl + 2 * k, idesc, 1);
                        }
                    } else {
#pragma unroll
                        for (int kq = 0; kq < 2; ++kq) {
                            const int kb = 2 * j + kq;
                            const uint64_t bh = tc::sw128_desc(tc::smem_u32(us + kb * Cfg::U_BOX));
                            const uint64_t bl = tc::sw128_desc(tc::smem_u32(us + (KB + kb) * Cfg::U_BOX));
#pragma unroll
                            for (int k = 0; k < 4; ++k) {  // K = 8 per instruction
                                const uint32_t kc = (uint32_t)(kq * 32 + k * 8);
                                mma_tf32_ta(d, a_hi + kc, bh + 2 * k, idesc, acc);
                                acc = 1;
                                mma_tf32_ta(d, a_lo + kc, bh + 2 * k, idesc, 1);
                                mma_tf32_ta(d, a_hi + kc, bl + 2 * k, idesc, 1);
                            }
                        }
                    }
                }
                if (!ok) break;
                tc::mma_commit(&u_empty[su]);
                tc::mma_commit(&acc_full[a]);
                ++committed;
            }
            if (ok)
                for (int j = 0; j < NH; ++j) tc::mma_commit(&s_empty[(i * NH + j) % kSlots]);
        }
        if (!ok) {
            if (err) atomicOr(err, 128);
            *abort = 1;
        }
    } else if (warp >= 6 && warp < 10) {  // strip preparation: one row per thread, into its TMEM lane
        const int qa = warp & 3;
        const int row = qa * 32 + lane;
        const uint32_t lane_off = (uint32_t)(qa * 32) << 16;
        bool ok = true;
        int i = 0;
        for (int64_t w = blockIdx.x; w < W && ok; w += gridDim.x, ++i) {
            const int64_t e = w / nstrips;
            const int m = r0 + (int)(w - e * nstrips) * 128 + row;
            const float* src = Mall + e * estride + (int64_t)m * ld + J;
            for (int j = 0; j < NH && ok; ++j) {
                const int h = i * NH + j, sl = h % kSlots;
                // the half's row into registers first: its loads are in flight while the slot drains
                float v[64];
#pragma unroll
                for (int k4 = 0; k4 < 16; ++k4) {
                    const int k = 64 * j + 4 * k4;
                    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (m < nu && k < jb) x = *reinterpret_cast<const float4*>(src + k);  // jb is a multiple of 4
                    v[4 * k4] = x.x;
                    v[4 * k4 + 1] = x.y;
                    v[4 * k4 + 2] = x.z;
                    v[4 * k4 + 3] = x.w;
                }
                if (!__all_sync(0xffffffffu, tc::mbar_wait(&s_empty[sl], ((h / kSlots) & 1) ^ 1, abort) && !*abort)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                if constexpr (H) {  // FP16 high parts and FP16 remainders, two per 32-bit column
                    float hi[32], lo[32];
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        const __half h0 = __float2half_rn(v[2 * k]), h1 = __float2half_rn(v[2 * k + 1]);
                        const __half l0 = __float2half_rn(v[2 * k] - __half2float(h0));
                        const __half l1 = __float2half_rn(v[2 * k + 1] - __half2float(h1));
                        hi[k] = __uint_as_float(pack_h2(h0, h1));
                        lo[k] = __uint_as_float(pack_h2(l0, l1));
                    }
                    tmem_st32(tmem + lane_off + slot_col(sl, 0), hi);
                    tmem_st32(tmem + lane_off + slot_col(sl, 1), lo);
                } else {
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        float hi[32], lo[32];
#pragma unroll
                        for (int k = 0; k < 32; ++k) {
                            hi[k] = tf32_hi(v[hh * 32 + k]);
                            lo[k] = v[hh * 32 + k] - hi[k];
                        }
                        tmem_st32(tmem + lane_off + slot_col(sl, 0) + hh * 32, hi);
                        tmem_st32(tmem + lane_off + slot_col(sl, 1) + hh * 32, lo);
                    }
                }
                tmem_st_wait();
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_ready[sl]);
            }
        }
        if (!ok && lane == 0) {
            if (err) atomicOr(err, 1024);
            *abort = 1;
        }
    } else if (warp == 14) {  // tile stores
        if (lane == 0) {
            int g = 0;
            bool ok = true;
            for (int64_t w = blockIdx.x; w < W && ok; w += gridDim.x) {
                const int64_t e = w / nstrips;
                const int m0 = r0 + (int)(w - e * nstrips) * 128;
                for (int t = 0; t < ntile; ++t, ++g) {
                    const int sc = g % NC;
                    if (!tc::mbar_wait(&c_done[sc], (g / NC) & 1, abort)) {
                        ok = false;
                        break;
                    }
                    for (int cb = 0; cb < UCB; ++cb)  // (a box wholly beyond c_end is not stored)
                        if (c0 + t * UBN + 32 * cb < c_end)
                            tma_store_3d(&tS, cstage0 + sc * Cfg::C_STAGE + cb * Cfg::C_BOX, c0 + t * UBN + 32 * cb, m0,
                                         (int)e);
                    bulk_commit();
                    bulk_wait_read0();  // the stage may be refilled once the store has read it
                    mbar_arrive(&c_empty[sc]);
                }
            }
            bulk_wait0();
            if (!ok) {
                if (err) atomicOr(err, 2048);
                *abort = 1;
            }
        }
    } else if (warp >= 2) {  // epilogue: warps 2-5 (box 0) and 10-13 (box 1)
        const int q = warp & 3;
        const int cb = warp >= 10 ? 1 : 0;
        const int row = q * 32 + lane;
        int g = 0;
        bool ok = true;
        for (int64_t w = blockIdx.x; w < W && ok; w += gridDim.x) {
            // the U^T tiles of a scaled re-solve carry the element's residual scale: undo it here
            const float unscale = 1.f / res_scale(res_max, w / nstrips);
            for (int t = 0; t < ntile; ++t, ++g) {
                const int sc = g % NC, a = g & 1;
                ok = __all_sync(0xffffffffu, tc::mbar_wait(&acc_full[a], (g >> 1) & 1, abort) &&
                                                 tc::mbar_wait(&c_full[sc], (g / NC) & 1, abort) && !*abort);
                if (!ok) {
                    if (err && lane == 0) atomicOr(err, 256);
                    break;
                }
                tc::tc_fence_after();
                float d[32];
#pragma unroll
                for (int c = 0; c < 32; c += 16) {
                    float v[16];
                    tc::tmem_ld16(tmem + (uint32_t)(a * UBN + 32 * cb) + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) d[c + j] = v[j] * unscale;
                }
                // C box cb in shared memory: rows m0 .. m0 + 127 of columns n0 + 32 cb .. + 31,
                // 128-byte rows with the 16-byte chunk index XOR-ed by (row % 8); C - L U goes back
                // in place
                unsigned char* crow = cstage0 + sc * Cfg::C_STAGE + cb * Cfg::C_BOX + row * 128;
                float4 cv[8];
#pragma unroll
                for (int ch = 0; ch < 8; ++ch) cv[ch] = *reinterpret_cast<const float4*>(crow + ((ch ^ (row & 7)) << 4));
#pragma unroll
                for (int ch = 0; ch < 8; ++ch)
                    *reinterpret_cast<float4*>(crow + ((ch ^ (row & 7)) << 4)) =
                        make_float4(cv[ch].x - d[4 * ch], cv[ch].y - d[4 * ch + 1], cv[ch].z - d[4 * ch + 2],
                                    cv[ch].w - d[4 * ch + 3]);
                // written through the generic proxy, read next by the TMA store (async proxy)
                tc::tc_fence_before();
                tc::fence_proxy_async();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&acc_empty[a]);
                    mbar_arrive(&c_done[sc]);
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0 && lane == 0) {  // let every copy this CTA issued land before the CTA exits
        for (int q = (issued_u > NU ? issued_u - NU : 0); q < issued_u; ++q) {
            const long long t1 = clock64();
            while (!tc::mbar_try_wait(&u_full[q % NU], (q / NU) & 1) && clock64() - t1 < tc::kWaitCycles / 4) {
            }
        }
        for (int q = (issued_c > NC ? issued_c - NC : 0); q < issued_c; ++q) {
            const long long t1 = clock64();
            while (!tc::mbar_try_wait(&c_full[q % NC], (q / NC) & 1) && clock64() - t1 < tc::kWaitCycles / 4) {
            }
        }
    }
    if (warp == 1) {
        if (lane == 0 && committed > 0) {  // never free TMEM under an MMA in flight
            const int last = committed - 1;
            const long long t0 = clock64();
            while (!tc::mbar_try_wait(&acc_full[last & 1], (last >> 1) & 1) && clock64() - t0 < tc::kWaitCycles) {
            }
            // and let the strip-slot commits issued after it arrive before the CTA's shared memory goes
            const int items = (int)((W - 1 - blockIdx.x) / gridDim.x) + 1;
            for (int h = (items - 1) * NH; committed == items * ntile && h < items * NH; ++h) {
                const long long t1 = clock64();
                while (!tc::mbar_try_wait(&s_empty[h % kSlots], (h / kSlots) & 1) && clock64() - t1 < tc::kWaitCycles / 4) {
                }
            }
        }
        __syncwarp();
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

// ------------------------------------------------------------------------------------------------
// host orchestration
// ------------------------------------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 g_enc = nullptr;
std::once_flag g_enc_once;

bool enc_ready() {
    std::call_once(g_enc_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_enc = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    return g_enc != nullptr;
}

// [E][rows][UTK] FP32 side buffer, box 32 (k) x box_rows x 1 element, 128-byte swizzle
bool map3(CUtensorMap* m, const float* p, int64_t rows, int64_t E, int box_rows) {
    cuuint64_t dims[3] = {(cuuint64_t)UTK, (cuuint64_t)rows, (cuuint64_t)E};
    cuuint64_t strides[2] = {(cuuint64_t)UTK * 4, (cuuint64_t)rows * UTK * 4};
    cuuint32_t box[3] = {32, (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return g_enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)p, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                 CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// [E][rows][UTK16] FP16 side buffer (within the same allocation), box 64 (k) x box_rows x 1 element,
// 128-byte swizzle
bool map3_16(CUtensorMap* m, const float* p, int64_t rows, int64_t E, int box_rows) {
    cuuint64_t dims[3] = {(cuuint64_t)UTK16, (cuuint64_t)rows, (cuuint64_t)E};
    cuuint64_t strides[2] = {(cuuint64_t)UTK16 * 2, (cuuint64_t)rows * UTK16 * 2};
    cuuint32_t box[3] = {64, (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return g_enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, (void*)p, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                 CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the matrix of every element seen as [E][rows][cols] (row pitch ld), box 32 columns x 128 rows x 1
// element, 128-byte swizzle: with rows = nu, cols = ld the C tiles of the loads; with rows = r_end,
// cols = c_end the stores of an update (whatever lies outside is clipped)
bool mapM(CUtensorMap* m, const float* M, int64_t rows, int64_t cols, int64_t ld, int64_t estride, int64_t E) {
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)E};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 4, (cuuint64_t)estride * 4};
    cuuint32_t box[3] = {32, 128, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return g_enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)M, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                 CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct TcMaps {
    CUtensorMap m, u;
    bool f16;  // trailing updates with 3xFP16 products (FP16 side buffer), else 3xTF32
    const double* res_max = nullptr;  // per-element residual maxima of a scaled FP16 re-solve
};

// Trailing update C -= L U over rows [r0, r_end) and columns [c0, c_end) of every element, with
// L = M[rows, J .. J+k) and U^T from the side buffer at K offset koff: rank k = jb <= 64 (one panel,
// kernel NK = 64) or 64 < k <= 128 (a pair of panels, the second possibly partial, NK = 128, koff 0;
// the strip is zero beyond jb).  Algorithmic bytes: C read and written, the FP32 L strip (R x k) and
// U^T tile (C x k); useful flops 2 R C k.
template <int NK>
elrt_status update(elrt_ctx* ctx, const TcMaps& mp, float* M, int64_t ld, int64_t estride, int64_t E, int J, int jb,
                   int koff, int r0, int r_end, int c0, int c_end, int* err) {
    if (r_end <= r0 || c_end <= c0) return ELRT_OK;
    const double R = r_end - r0, C = c_end - c0;
    ProfScope ps(ctx, "lu_tc_update", 1, (double)E * (8.0 * R * C + 4.0 * (R + C) * jb), (double)E * 2.0 * R * C * jb);
    CUtensorMap tS;  // stores: rows [0, r_end), columns [0, c_end)
    if (!mapM(&tS, M, r_end, c_end, ld, estride, E)) return ctx_fail(ctx, ELRT_EINVAL, "tensor map encoding failed");
    const int64_t items = (int64_t)((r_end - r0 + 127) / 128) * E;
    const unsigned grid = (unsigned)std::min<int64_t>(items, ctx->sms);
    if (mp.f16)
        k_tc_update<NK, true><<<grid, kStripThreads, UpdCfg<NK, true>::TOTAL, ctx->stream>>>(
            mp.m, mp.u, tS, M, ctx->tab.nu, ld, estride, E, J, jb, koff, r0, r_end, c0, c_end, err, mp.res_max);
    else
        k_tc_update<NK, false><<<grid, kStripThreads, UpdCfg<NK, false>::TOTAL, ctx->stream>>>(
            mp.m, mp.u, tS, M, ctx->tab.nu, ld, estride, E, J, jb, koff, r0, r_end, c0, c_end, err, nullptr);
    return cuda_check(ctx, cudaGetLastError(), "tc update launch");
}


template <int PT>
cudaError_t rowcol_attrs() {
    cudaError_t e = cudaFuncSetAttribute(k_rowcol<0, PT>, cudaFuncAttributeMaxDynamicSharedMemorySize, RcCfg<PT>::SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rowcol<1, PT>, cudaFuncAttributeMaxDynamicSharedMemorySize, RcCfg<PT>::SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rowcol<2, PT>, cudaFuncAttributeMaxDynamicSharedMemorySize, RcCfg<PT>::SMEM);
    return e;
}

elrt_status prepare(elrt_ctx* ctx, float* M, int64_t ld, int64_t estride, const float* Ut, int64_t E, TcMaps* mp,
                    bool f16) {
    mp->f16 = f16;
    if (!enc_ready()) return ctx_fail(ctx, ELRT_ECUDA, "cuTensorMapEncodeTiled unavailable");
    if (E > 65535) return ctx_fail(ctx, ELRT_EINVAL, "tensor-core LU chunk above 65535 elements");
    const int nu = ctx->tab.nu;
    // every column block starts at a multiple of 64 or at nu, and the vector accesses and TMA copies
    // need each to start on a 16-byte boundary (n_angles % 4 == 0 already makes nu a multiple of 4)
    if (nu % 4 != 0 || ld % 4 != 0) return ctx_fail(ctx, ELRT_EINVAL, "tensor-core LU needs nu and ld multiples of 4");
    if (!mapM(&mp->m, M, nu, ld, ld, estride, E) || !(f16 ? map3_16(&mp->u, Ut, ld, E, UBN) : map3(&mp->u, Ut, ld, E, UBN)))
        return ctx_fail(ctx, ELRT_EINVAL, "tensor map encoding failed");
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = rowcol_attrs<kRcTile>();
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_tc_update<64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, UpdCfg<64>::TOTAL);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_tc_update<128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, UpdCfg<128>::TOTAL);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_tc_update<64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     UpdCfg<64, true>::TOTAL);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_tc_update<128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     UpdCfg<128, true>::TOTAL);
        if (e != cudaSuccess) return cuda_check(ctx, e, "smem attribute");
        attr_done = true;
    }
    return ELRT_OK;
}

int panels_of(int nu) { return (nu + NBP - 1) / NBP; }

template <int PTILE>
void rowcol_launch(elrt_ctx* ctx, float* M, int64_t ld, int64_t estride, int64_t E, int J, int jb, const float* Tinv,
                   int r_begin, int r_end, int c_begin, int c_end, int col_mode, float* Ut, int koff, int ut16,
                   const double* res_max) {
    using C = RcCfg<PTILE>;
    const int nrt = r_end > r_begin ? (r_end - r_begin + PTILE - 1) / PTILE : 0;
    const int nct = c_end > c_begin ? (c_end - c_begin + PTILE - 1) / PTILE : 0;
    const int np = panels_of(ctx->tab.nu), nu = ctx->tab.nu;
    if (nrt > 0) {  // items: (element, row tile)
        const unsigned grid = (unsigned)std::min<int64_t>(E * nrt, (int64_t)C::PER_SM * ctx->sms);
        k_rowcol<0, PTILE><<<grid, PTILE, C::SMEM, ctx->stream>>>(nu, ld, estride, M, J, jb, Tinv, np, E, r_begin, r_end,
                                                                 nrt, c_begin, c_end, 0, Ut, koff, ut16, nullptr);
    }
    if (nct > 0) {  // items: (element, column tile)
        const unsigned grid = (unsigned)std::min<int64_t>(E * nct, (int64_t)C::PER_SM * ctx->sms);
        if (col_mode == 0)
            k_rowcol<1, PTILE><<<grid, PTILE, C::SMEM, ctx->stream>>>(nu, ld, estride, M, J, jb, Tinv, np, E, r_begin,
                                                                     r_end, 0, c_begin, c_end, nct, Ut, koff, ut16, res_max);
        else
            k_rowcol<2, PTILE><<<grid, PTILE, C::SMEM, ctx->stream>>>(nu, ld, estride, M, J, jb, Tinv, np, E, r_begin,
                                                                     r_end, 0, c_begin, c_end, nct, Ut, koff, ut16, nullptr);
    }
}

elrt_status rowcol(elrt_ctx* ctx, const TcMaps& mp, float* M, int64_t ld, int64_t estride, int64_t E, int J, int jb,
                   const float* Tinv, int r_begin, int r_end, int c_begin, int c_end, int col_mode, float* Ut,
                   int koff = 0) {
    if (r_end <= r_begin && c_end <= c_begin) return ELRT_OK;
    // algorithmic work per element: row tiles read R x jb and write it back; column tiles read and
    // write jb x C and write U^T (C x 64); triangular solves with U11, L11 (unit lower) or U11
    const double R = std::max(0, r_end - r_begin), C = std::max(0, c_end - c_begin);
    const double bytes = 8.0 * R * jb + 8.0 * C * jb + 4.0 * C * NBP + 4.0 * NBP * NBP * ((R > 0) + (C > 0));
    const double flops = R * jb * (jb + 1.0) + (col_mode == 0 ? C * jb * (jb - 1.0) : C * jb * (jb + 1.0));
    ProfScope ps(ctx, "lu_tc_rowcol", (R > 0) + (C > 0), (double)E * bytes, (double)E * flops);
    rowcol_launch<kRcTile>(ctx, M, ld, estride, E, J, jb, Tinv, r_begin, r_end, c_begin, c_end, col_mode, Ut, koff,
                           mp.f16 ? 1 : 0, mp.res_max);
    return cuda_check(ctx, cudaGetLastError(), "rowcol launch");
}

// backward substitution on the right-hand-side columns: X_J = U11^{-1} X_J, then the rows above
// lose U[0..J, J..J+jb) X_J.  With the pair schedule, per pair (a, b), last pair first: X_b, the
// rank-64 update of panel a's rows, X_a, and one rank-128 update of the rows above the pair (both
// panels' solutions, side buffer K offsets 0 and 64).  A last panel narrower than a pair joins the
// last pair's second panel (the grouped form below); otherwise the panels beyond the last pair go
// first, one at a time.
elrt_status backward_sweep_tc(elrt_ctx* ctx, const TcMaps& mp, float* M, int64_t ld, int64_t estride, int64_t E,
                              const float* Tinv, float* Ut, int* err, int nin) {
    const int nu = ctx->tab.nu;
    const int npair = ctx->tune.lu_pairs ? nu / (2 * NBP) : 0;
    const int rem = nu - 2 * NBP * npair;  // columns beyond the last pair
    if (npair > 0 && rem > 0 && rem <= NBP) {
        // the last panel t (rem columns, e.g. 16 of nu = 784) joins the panel b before it: X_t, b's
        // rows lose U[b, t] X_t, X_b, and the rows above b take both in one update of rank 64 + rem
        // (the strip is masked beyond jb, and t's side-buffer slots beyond rem hold zeros: its
        // diagonal block is padded with the identity).  The panels below b then pair up shifted by
        // one, [J, J + 128) for J = 128 q - 64, and panel 0 is solved alone, with no rows above it.
        // Against t on its own, one rank-rem update of all nu - rem rows above t becomes a narrow
        // one of b's 64 rows; the shifted pairs' updates cover 64 rows more each.
        const int Jt = 2 * NBP * npair, Jb = Jt - NBP;
        elrt_status s = rowcol(ctx, mp, M, ld, estride, E, Jt, rem, Tinv, 0, 0, nu, nu + nin, 1, Ut, NBP);
        if (!s) s = update<64>(ctx, mp, M, ld, estride, E, Jt, rem, NBP, Jb, Jt, nu, nu + nin, err);
        if (!s) s = rowcol(ctx, mp, M, ld, estride, E, Jb, NBP, Tinv, 0, 0, nu, nu + nin, 1, Ut, 0);
        if (!s) s = update<128>(ctx, mp, M, ld, estride, E, Jb, NBP + rem, 0, 0, Jb, nu, nu + nin, err);
        for (int J = Jb - 2 * NBP; J >= 0 && !s; J -= 2 * NBP) {
            const int Jh = J + NBP;
            s = rowcol(ctx, mp, M, ld, estride, E, Jh, NBP, Tinv, 0, 0, nu, nu + nin, 1, Ut, NBP);
            if (!s) s = update<64>(ctx, mp, M, ld, estride, E, Jh, NBP, NBP, J, Jh, nu, nu + nin, err);
            if (!s) s = rowcol(ctx, mp, M, ld, estride, E, J, NBP, Tinv, 0, 0, nu, nu + nin, 1, Ut, 0);
            if (!s) s = update<128>(ctx, mp, M, ld, estride, E, J, 2 * NBP, 0, 0, J, nu, nu + nin, err);
        }
        if (!s) s = rowcol(ctx, mp, M, ld, estride, E, 0, NBP, Tinv, 0, 0, nu, nu + nin, 1, Ut, 0);
        return s;
    }
    const int last = ((nu - 1) / NBP) * NBP;
    for (int J = last; J >= 2 * NBP * npair; J -= NBP) {
        const int jb = std::min(NBP, nu - J);
        elrt_status s = rowcol(ctx, mp, M, ld, estride, E, J, jb, Tinv, 0, 0, nu, nu + nin, 1, Ut, 0);
        if (!s) s = update<64>(ctx, mp, M, ld, estride, E, J, jb, 0, 0, J, nu, nu + nin, err);
        if (s) return s;
    }
    for (int q = npair - 1; q >= 0; --q) {
        const int J = 2 * NBP * q, Jb = J + NBP;
        elrt_status s = rowcol(ctx, mp, M, ld, estride, E, Jb, NBP, Tinv, 0, 0, nu, nu + nin, 1, Ut, NBP);
        if (!s) s = update<64>(ctx, mp, M, ld, estride, E, Jb, NBP, NBP, J, Jb, nu, nu + nin, err);
        if (!s) s = rowcol(ctx, mp, M, ld, estride, E, J, NBP, Tinv, 0, 0, nu, nu + nin, 1, Ut, 0);
        if (!s) s = update<128>(ctx, mp, M, ld, estride, E, J, 2 * NBP, 0, 0, J, nu, nu + nin, err);
        if (s) return s;
    }
    return ELRT_OK;
}

struct Side {
    float *Ut, *Tinv;
};

Side carve(float* side, int64_t E, int64_t ld) {
    Side sd;
    sd.Ut = side;
    sd.Tinv = sd.Ut + (size_t)E * ld * UTK;
    return sd;
}

// LU of the 64 x 64 diagonal block at column J (published to Tinv)
void diag_block(elrt_ctx* ctx, float* M, int64_t ld, int64_t estride, int64_t E, int J, int jb, float* Tinv, int* estat) {
    const int nu = ctx->tab.nu;
    const double b3 = (double)jb * jb * jb;
    ProfScope ps(ctx, "lu_tc_diag", 1, (double)E * (8.0 * jb * jb + 4.0 * kInvMats * NBP * NBP), (double)E * 2.0 / 3.0 * b3);
    k_diag<<<(unsigned)E, kDiagThreads, 0, ctx->stream>>>(nu, ld, estride, M, J, jb, Tinv, panels_of(nu), estat, 1e-6f);
}

}  // namespace

// Factor every element's matrix without pivoting and solve for its right-hand sides (columns
// [nu, nu + nrhs)).  side: tc_lu_side_floats() floats per element.  estat[e] |= 1 on a tiny pivot.
elrt_status tc_lu_factor_solve(elrt_ctx* ctx, float* M, int64_t ld, int64_t estride, int64_t E, int* estat, float* side,
                               int* err, int nrhs, bool f16) {
    const int nu = ctx->tab.nu, ncols = nu + nrhs;
    const Side sd = carve(side, E, ld);
    TcMaps mp;
    elrt_status s = prepare(ctx, M, ld, estride, sd.Ut, E, &mp, f16);
    if (s) return s;
    int J = 0;
    // pairs of full panels a = [J, J+64), b = [J+64, J+128): panel a is factored and applied to
    // panel b's columns and rows only (two narrow rank-64 updates), panel b is factored, and the
    // rest of the matrix takes both in one rank-128 update (half the C traffic of two rank-64 ones)
    for (; ctx->tune.lu_pairs && J + 2 * NBP <= nu; J += 2 * NBP) {
        const int Jb = J + NBP, Jn = J + 2 * NBP;
        diag_block(ctx, M, ld, estride, E, J, NBP, sd.Tinv, estat);
        s = rowcol(ctx, mp, M, ld, estride, E, J, NBP, sd.Tinv, Jb, nu, Jb, ncols, 0, sd.Ut, 0);
        if (!s) s = update<64>(ctx, mp, M, ld, estride, E, J, NBP, 0, Jb, nu, Jb, Jn, err);
        if (!s) s = update<64>(ctx, mp, M, ld, estride, E, J, NBP, 0, Jb, Jn, Jn, ncols, err);
        if (s) return s;
        diag_block(ctx, M, ld, estride, E, Jb, NBP, sd.Tinv, estat);
        s = rowcol(ctx, mp, M, ld, estride, E, Jb, NBP, sd.Tinv, Jn, nu, Jn, ncols, 0, sd.Ut, NBP);
        if (!s) s = update<128>(ctx, mp, M, ld, estride, E, J, 2 * NBP, 0, Jn, nu, Jn, ncols, err);
        if (s) return s;
    }
    // the remaining panels one at a time
    for (; J < nu; J += NBP) {
        const int jb = std::min(NBP, nu - J);
        diag_block(ctx, M, ld, estride, E, J, jb, sd.Tinv, estat);
        s = rowcol(ctx, mp, M, ld, estride, E, J, jb, sd.Tinv, J + jb, nu, J + jb, ncols, 0, sd.Ut, 0);
        if (!s) s = update<64>(ctx, mp, M, ld, estride, E, J, jb, 0, J + jb, nu, J + jb, ncols, err);
        if (s) return s;
    }
    return backward_sweep_tc(ctx, mp, M, ld, estride, E, sd.Tinv, sd.Ut, err, nrhs);
}

// Re-solve A D = R for the right-hand sides in columns [nu, nu + nrhs) with the stored factors.
// With f16 (and res_max, the per-element maxima of the residuals in those columns), the forward
// sweep forms its products in 3xFP16 with the residual scaled into FP16's range per element; the
// backward sweep keeps 3xTF32, because U^{-1} shrinks the correction of a thick element far below
// its residual, where FP16 parts would be subnormal.
elrt_status tc_lu_resolve(elrt_ctx* ctx, float* M, int64_t ld, int64_t estride, int64_t E, float* side, int* err,
                          int nrhs, bool f16, const double* res_max) {
    const int nu = ctx->tab.nu, nin = nrhs;
    const Side sd = carve(side, E, ld);
    TcMaps mp;
    const bool f16_fwd = f16 && res_max;
    elrt_status s = prepare(ctx, M, ld, estride, sd.Ut, E, &mp, f16_fwd);
    if (s) return s;
    if (f16_fwd) mp.res_max = res_max;
    int J = 0;
    // forward substitution with the unit lower factor, in the factorisation's panel pairs: X_a, the
    // rank-64 update of panel b's rows, X_b, one rank-128 update of the rows below the pair
    for (; ctx->tune.lu_pairs && J + 2 * NBP <= nu; J += 2 * NBP) {
        const int Jb = J + NBP, Jn = J + 2 * NBP;
        s = rowcol(ctx, mp, M, ld, estride, E, J, NBP, sd.Tinv, 0, 0, nu, nu + nin, 0, sd.Ut, 0);
        if (!s) s = update<64>(ctx, mp, M, ld, estride, E, J, NBP, 0, Jb, Jn, nu, nu + nin, err);
        if (!s) s = rowcol(ctx, mp, M, ld, estride, E, Jb, NBP, sd.Tinv, 0, 0, nu, nu + nin, 0, sd.Ut, NBP);
        if (!s) s = update<128>(ctx, mp, M, ld, estride, E, J, 2 * NBP, 0, Jn, nu, nu, nu + nin, err);
        if (s) return s;
    }
    for (; J < nu; J += NBP) {
        const int jb = std::min(NBP, nu - J);
        s = rowcol(ctx, mp, M, ld, estride, E, J, jb, sd.Tinv, 0, 0, nu, nu + nin, 0, sd.Ut, 0);
        if (!s) s = update<64>(ctx, mp, M, ld, estride, E, J, jb, 0, J + jb, nu, nu, nu + nin, err);
        if (s) return s;
    }
    if (f16_fwd) {  // the backward sweep in 3xTF32: the FP32 side-buffer layout, no scale
        s = prepare(ctx, M, ld, estride, sd.Ut, E, &mp, false);
        if (s) return s;
        mp.res_max = nullptr;
    }
    return backward_sweep_tc(ctx, mp, M, ld, estride, E, sd.Tinv, sd.Ut, err, nrhs);
}

size_t tc_lu_side_floats(const Tab& t, int64_t ld) {
    return (size_t)UTK * ld + (size_t)panels_of(t.nu) * kInvMats * NBP * NBP;
}
