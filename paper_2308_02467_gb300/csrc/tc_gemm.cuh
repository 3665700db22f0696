// tcgen05 / TMEM / TMA building blocks and a BF16 GEMM with fused epilogues for sm_103a.
//
//   D[M][N] = A[M][K] . B[N][K]^T      (A, B bf16, K contiguous; FP32 accumulation in TMEM)
//
// One CTA computes one BM x BN tile: warp 0 issues TMA loads of A and B k-blocks (BK = 64 bf16 =
// 128 bytes per row, 128-byte swizzle) into a STAGES-deep ring guarded by mbarriers; warp 1
// allocates BN TMEM columns and, from one elected lane, issues tcgen05.mma (M = 128, N = BN,
// K = 16 per instruction) and tcgen05.commit to free each stage; warps 2-5 wait for the final
// commit, read the accumulator with tcgen05.ld (warp w owns TMEM lanes 32 (w % 4) .. + 31) and
// run the epilogue.  Every wait is bounded (about 2 s of clock64); on timeout the kernel records
// an error code, stops issuing work, waits (bounded) for its own copies in flight, frees its TMEM
// and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tc {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int kGemmThreads = 320;  // TMA producer, MMA issuer, eight epilogue warps
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity`; false on timeout or when *abort is set.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > kWaitCycles) return false;
    }
    return true;
}

// plain (non-tensor) bulk copy global -> shared completing on an mbarrier: both addresses 16-byte
// aligned, size a multiple of 16 bytes
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// L2 policy for data read once (streamed operators): evicted first, so that vectors reused by the
// next kernels stay in L2
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// bulk_load with an L2 cache policy
__device__ __forceinline__ void bulk_load_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of 128 bytes,
// 8-row groups 1024 bytes apart (tile base 1024-byte aligned).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset between 8-row groups
    d |= (uint64_t)1 << 46;                    // descriptor version
    d |= (uint64_t)2 << 61;                    // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: BF16 A and B (K-major), FP32 D, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------------------------------------
// GEMM with fused epilogues
// ------------------------------------------------------------------------------------------------

enum Epi : int {
    EPI_F32 = 0,        // out_f[m][n] = acc                                  (weight gradients)
    EPI_BIAS_ACT = 1,   // z = acc + bias; h = act(z): out_bf (h), z_out (z), out_bf_t (h^T)
    EPI_OUTPUT = 2,     // y = (acc + bias) * col_std + col_mean -> out_f (n < split) / out_f2 (n >= split)
    EPI_LOSS = 3,       // y = acc + bias; d = sign(y - t) * scale -> out_bf, out_bf_t; loss += |y - t|
    EPI_DACT = 4,       // d = acc * act'(z_in): out_bf, out_bf_t
};

struct EpiArgs {
    const float* bias = nullptr;           // [N]
    __nv_bfloat16* out_bf = nullptr;       // [M][ld_out]
    __nv_bfloat16* out_bf_t = nullptr;     // [N][ld_t]
    __nv_bfloat16* z_out = nullptr;        // [M][ld_out]
    const __nv_bfloat16* z_in = nullptr;   // [M][ld_out]
    float* out_f = nullptr;                // [M][ld_out] (EPI_F32, EPI_OUTPUT n < split)
    float* out_f2 = nullptr;               // [M][ld_out2] (EPI_OUTPUT n >= split)
    const float* col_mean = nullptr;
    const float* col_std = nullptr;
    const float* target = nullptr;         // [M][ld_out] standardised targets
    float* loss_acc = nullptr;             // one float
    float loss_scale = 0.f;
    int split = 0;
    int ld_out = 0, ld_out2 = 0, ld_t = 0;
    int act = 0;                           // 0 GELU (exact, erf), 1 ELU
    int ksplit = 1;                        // K slices (EPI_F32 only): slice s writes out_f + s * part_stride
    size_t part_stride = 0;
    int* err = nullptr;
};

__device__ __forceinline__ float act_f(float z, int act) {
    if (act == 0) return 0.5f * z * (1.f + erff(z * 0.70710678118654752f));
    return z > 0.f ? z : expm1f(z);
}
__device__ __forceinline__ float act_df(float z, int act) {
    if (act == 0) return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
    return z > 0.f ? 1.f : expf(z);
}

// OUT_TMA: EPI_OUTPUT written by TMA tensor stores from a 32 x 16 FP32 staging buffer per epilogue
// warp (the rows of one tile are elements whose outputs lie far apart, so row-wise stores from
// the epilogue threads touch 32 rows per instruction)
template <int BN, bool OUT_TMA = false>
struct GemmSmem {
    static constexpr int STAGES = BN == 256 ? 4 : 6;
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int PARAM_BYTES = 2 * 2 * BN * 4;  // per-tile column parameters (scale and shift, or bias), two tiles
    static constexpr int OUT_BOX = 32 * 16 * 4;          // one staged 32-row x 16-column FP32 box
    static constexpr int OUT_BYTES = OUT_TMA ? 8 * OUT_BOX : 0;
    static constexpr int TOTAL = STAGES * STAGE_BYTES + 1024 /*alignment*/ + 256 /*barriers*/ + PARAM_BYTES + OUT_BYTES;
    static constexpr int TMEM_COLS = 2 * BN;  // two accumulators: epilogue of one tile overlaps the next
};
static_assert(GemmSmem<256, true>::TOTAL <= 227 * 1024 && GemmSmem<128, true>::TOTAL <= 227 * 1024, "GEMM shared memory");

// shared -> global tensor copy of a 2-D box (bulk group); coordinates non-negative
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(smem_u32(src)), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit_group() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void st_f32x16(float* dst, const float (&v)[16]) {
    float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int q = 0; q < 4; ++q) d[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

__device__ __forceinline__ void st_bf16x16(__nv_bfloat16* dst, const float (&v)[16]) {
    uint32_t w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        w[q] = *reinterpret_cast<uint32_t*>(&h2);
    }
    uint4* d = reinterpret_cast<uint4*>(dst);
    d[0] = make_uint4(w[0], w[1], w[2], w[3]);
    d[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// the standardised targets of row m, columns n0c .. n0c+15 (zero beyond N)
__device__ __forceinline__ void load_targets16(const EpiArgs& ep, int m, int n0c, int N, float (&tg)[16]) {
    if (n0c + 16 <= N) {
        const float4* src = reinterpret_cast<const float4*>(ep.target + (size_t)m * ep.ld_out + n0c);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 v4 = __ldcs(src + q);
            tg[4 * q] = v4.x;
            tg[4 * q + 1] = v4.y;
            tg[4 * q + 2] = v4.z;
            tg[4 * q + 3] = v4.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) tg[j] = n0c + j < N ? ep.target[(size_t)m * ep.ld_out + n0c + j] : 0.f;
    }
}

// EPI_LOSS of 16 consecutive columns n0c .. n0c+15 of row m: v holds the accumulator values, sb the
// tile's bias for these columns (shared memory), tg their targets (loaded ahead by the caller)
__device__ __forceinline__ void loss16(const EpiArgs& ep, int m, int n0c, int N, float (&v)[16], float& lsum,
                                       const float* sb, const float (&tg)[16]) {
    const bool full = n0c + 16 <= N;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (n0c + j < N) {
            const float y = v[j] + sb[j];
            const float d = y - tg[j];
            lsum += fabsf(d);
            v[j] = d > 0.f ? ep.loss_scale : (d < 0.f ? -ep.loss_scale : 0.f);
        }
    }
    if (full) {
        st_bf16x16(ep.out_bf + (size_t)m * ep.ld_out + n0c, v);
    } else {
        _Pragma("unroll") for (int j = 0; j < 16; ++j) if (n0c + j < N) ep.out_bf[(size_t)m * ep.ld_out + n0c + j] = __float2bfloat16_rn(v[j]);
    }
    if (ep.out_bf_t)
        _Pragma("unroll") for (int j = 0; j < 16; ++j) if (n0c + j < N)
            ep.out_bf_t[(size_t)(n0c + j) * ep.ld_t + m] = __float2bfloat16_rn(v[j]);
}

// Epilogue of 16 consecutive columns n0c .. n0c+15 of row m (v holds the accumulator values) for
// EPI_F32, EPI_BIAS_ACT and EPI_DACT.  sb: the tile's bias for these 16 columns, staged in shared
// memory (EPI_BIAS_ACT); slice: the K slice (EPI_F32)
__device__ __forceinline__ void epilogue16(int mode, const EpiArgs& ep, int m, int n0c, int N, float (&v)[16],
                                           const float* sb, int slice) {
    const bool full = n0c + 16 <= N;
    if (mode == EPI_F32) {
        float* out = ep.out_f + (size_t)slice * ep.part_stride;
        if (full) {
            st_f32x16(out + (size_t)m * ep.ld_out + n0c, v);
        } else {
            _Pragma("unroll") for (int j = 0; j < 16; ++j) if (n0c + j < N)
out[(size_t)m * ep.ld_out + n0c + j] = v[j];
        }
    } else if (mode == EPI_BIAS_ACT) {
        float z[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int n = n0c + j;
            z[j] = v[j] + (n < N ? sb[j] : 0.f);
            v[j] = act_f(z[j], ep.act);
        }
        if (full) {
            st_bf16x16(ep.out_bf + (size_t)m * ep.ld_out + n0c, v);
            if (ep.z_out) st_bf16x16(ep.z_out + (size_t)m * ep.ld_out + n0c, z);
        } else {
            _Pragma("unroll") for (int j = 0; j < 16; ++j) if (n0c + j < N) {
                ep.out_bf[(size_t)m * ep.ld_out + n0c + j] = __float2bfloat16_rn(v[j]);
                if (ep.z_out) ep.z_out[(size_t)m * ep.ld_out + n0c + j] = __float2bfloat16_rn(z[j]);
            }
        }
        if (ep.out_bf_t)
            _Pragma("unroll") for (int j = 0; j < 16; ++j) if (n0c + j < N)
ep.out_bf_t[(size_t)(n0c + j) * ep.ld_t + m] = __float2bfloat16_rn(v[j]);
    } else {  // EPI_DACT
        if (full) {  // the 16 pre-activations in two 16-byte loads
            const uint4* zp = reinterpret_cast<const uint4*>(ep.z_in + (size_t)m * ep.ld_out + n0c);
            const uint4 za = zp[0], zb = zp[1];
            const uint32_t zw[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float2 z2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&zw[q]));
                v[2 * q] *= act_df(z2.x, ep.act);
                v[2 * q + 1] *= act_df(z2.y, ep.act);
            }
        } else {
            _Pragma("unroll") for (int j = 0; j < 16; ++j) if (n0c + j < N) {
                const float z = __bfloat162float(ep.z_in[(size_t)m * ep.ld_out + n0c + j]);
                v[j] = v[j] * act_df(z, ep.act);
            }
        }
        if (full) {
            st_bf16x16(ep.out_bf + (size_t)m * ep.ld_out + n0c, v);
        } else {
            _Pragma("unroll") for (int j = 0; j < 16; ++j) if (n0c + j < N)
ep.out_bf[(size_t)m * ep.ld_out + n0c + j] = __float2bfloat16_rn(v[j]);
        }
        if (ep.out_bf_t)
            _Pragma("unroll") for (int j = 0; j < 16; ++j) if (n0c + j < N)
ep.out_bf_t[(size_t)(n0c + j) * ep.ld_t + m] = __float2bfloat16_rn(v[j]);
    }
}

// y = acc * scale + shift for 16 consecutive columns
__device__ __forceinline__ void scale16(float (&v)[16], const float* sc, const float* sh) {
#pragma unroll
    for (int j = 0; j < 16; j += 4) {
        const float4 s4 = *reinterpret_cast<const float4*>(sc + j);
        const float4 h4 = *reinterpret_cast<const float4*>(sh + j);
        v[j] = fmaf(v[j], s4.x, h4.x);
        v[j + 1] = fmaf(v[j + 1], s4.y, h4.y);
        v[j + 2] = fmaf(v[j + 2], s4.z, h4.z);
        v[j + 3] = fmaf(v[j + 3], s4.w, h4.w);
    }
}

// EPI_OUTPUT of 16 consecutive columns n0c .. n0c+15 of row m: y = acc * scale + shift into out_f
// (columns below split) or out_f2; the split, a multiple of 16, never falls inside the group
__device__ __forceinline__ void output16(const EpiArgs& ep, int m, int n0c, int N, float (&v)[16], const float* sc,
                                         const float* sh) {
    scale16(v, sc, sh);
    float* dst = n0c < ep.split ? ep.out_f + (size_t)m * ep.ld_out + n0c
                                : ep.out_f2 + (size_t)m * ep.ld_out2 + (n0c - ep.split);
    if (n0c + 16 <= N) {
        st_f32x16(dst, v);
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (n0c + j < N) dst[j] = v[j];
    }
}

// Persistent: each CTA walks work items blockIdx.x, blockIdx.x + gridDim.x, ... (the shorter tile
// dimension fastest, so concurrently running CTAs share the long operand's tile in L2).  The TMA producer streams k-blocks of
// consecutive tiles through the ring without a break; the MMA issuer alternates between two TMEM
// accumulators so the epilogue of one tile overlaps the MMAs of the next.
// tmO / tmO2 (OUT_TMA only): out_f and out_f2 as 2-D FP32 tensors [M][split] and [M][N - split],
// box 16 columns x 32 rows, no swizzle
template <int BN, bool OUT_TMA = false>
__global__ void __launch_bounds__(kGemmThreads, 1)
    k_gemm_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
                int mode, EpiArgs ep, const __grid_constant__ CUtensorMap tmO, const __grid_constant__ CUtensorMap tmO2) {
    using S = GemmSmem<BN, OUT_TMA>;
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)gsm_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* As = base;
    unsigned char* Bs = base + S::STAGES * S::A_BYTES;
    uint64_t* full = (uint64_t*)(base + S::STAGES * S::STAGE_BYTES);
    uint64_t* empty = full + S::STAGES;
    uint64_t* acc_full = empty + S::STAGES;  // [2]
    uint64_t* acc_empty = acc_full + 2;      // [2]
    uint32_t* tmem_slot = (uint32_t*)(acc_empty + 2);
    volatile int* abort = (volatile int*)(tmem_slot + 1);
    float* prm = (float*)(base + S::STAGES * S::STAGE_BYTES + 256);  // [2 tiles][scale BN | shift BN]
    float* ostage = (float*)((unsigned char*)prm + S::PARAM_BYTES);    // OUT_TMA: [8 warps][32 x 16]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkb = (K + BK - 1) / BK;
    const int mt = (M + BM - 1) / BM, ntl = (N + BN - 1) / BN;
    const int ks = ep.ksplit > 1 ? ep.ksplit : 1;
    const int ntiles = mt * ntl * ks;  // work items: output tile, then K slice
    // tile origin of work item `item`: the shorter tile dimension runs fastest, so that the CTAs
    // working at the same time share the long operand's slab (read once from DRAM) while the short
    // operand stays in L2
    auto origin = [&](int item, int& m0, int& n0) {
        const int t = item % (mt * ntl);
        if (mt <= ntl) {
            m0 = (t % mt) * BM;
            n0 = (t / mt) * BN;
        } else {
            m0 = (t / ntl) * BM;
            n0 = (t % ntl) * BN;
        }
    };
    // k-blocks [kb0, kb1) of work item `item`
    auto kslice = [&](int item, int& kb0, int& kb1) {
        const int sl = item / (mt * ntl);
        kb0 = (int)((int64_t)nkb * sl / ks);
        kb1 = (int)((int64_t)nkb * (sl + 1) / ks);
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < S::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 1);
            mbar_init(&acc_empty[a], 8);  // one arrival per epilogue warp
        }
        *abort = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, S::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    int committed = 0;  // accumulator commits issued by this CTA (MMA thread)

    if (warp == 0 && lane == 0) {
        // TMA producer
        int kbg = 0, issued = 0;
        for (int tile = blockIdx.x; tile < ntiles && !*abort; tile += gridDim.x) {
            int m0, n0, kb0, kb1;
            origin(tile, m0, n0);
            kslice(tile, kb0, kb1);
            for (int kb = kb0; kb < kb1; ++kb, ++kbg) {
                const int s = kbg % S::STAGES;
                const uint32_t ph = (kbg / S::STAGES) & 1;
                if (!mbar_wait(&empty[s], ph ^ 1, abort)) {
                    if (ep.err) atomicOr(ep.err, 1);
                    *abort = 1;
                    break;
                }
                mbar_expect_tx(&full[s], S::STAGE_BYTES);
                tma_load_2d(&tmA, &full[s], As + s * S::A_BYTES, kb * BK, m0);
                tma_load_2d(&tmB, &full[s], Bs + s * S::B_BYTES, kb * BK, n0);
                ++issued;
            }
        }
        if (*abort) {  // let every copy this thread issued land before the CTA exits
            for (int q = (issued > S::STAGES ? issued - S::STAGES : 0); q < issued; ++q) {
                const long long t0 = clock64();
                while (!mbar_try_wait(&full[q % S::STAGES], (q / S::STAGES) & 1) && clock64() - t0 < kWaitCycles / 4) {
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(BM, BN);
        int kbg = 0, t = 0;
        for (int tile = blockIdx.x; tile < ntiles && !*abort; tile += gridDim.x, ++t) {
            const int a = t & 1;
            if (!mbar_wait(&acc_empty[a], ((t >> 1) & 1) ^ 1, abort)) {
                if (ep.err) atomicOr(ep.err, 8);
                *abort = 1;
                break;
            }
            tc_fence_after();
            const uint32_t dt = tmem_base + (uint32_t)(a * BN);
            bool ok = true;
            int kb0, kb1;
            kslice(tile, kb0, kb1);
            for (int kb = kb0; kb < kb1; ++kb, ++kbg) {
                const int s = kbg % S::STAGES;
                const uint32_t ph = (kbg / S::STAGES) & 1;
                if (!mbar_wait(&full[s], ph, abort)) {
                    if (ep.err) atomicOr(ep.err, 2);
                    *abort = 1;
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint64_t ad = sw128_desc(smem_u32(As + s * S::A_BYTES));
                const uint64_t bd = sw128_desc(smem_u32(Bs + s * S::B_BYTES));
#pragma unroll
                for (int k = 0; k < BK / 16; ++k)
                    mma_bf16(dt, ad + (uint64_t)(k * 2), bd + (uint64_t)(k * 2), idesc, (kb != kb0 || k != 0) ? 1u : 0u);
                mma_commit(&empty[s]);
            }
            mma_commit(&acc_full[a]);
            ++committed;
            if (!ok) break;
        }
    } else if (warp >= 2) {
        // epilogue: warp w owns TMEM lanes 32 (w % 4) .. + 31 (tile rows) and half (w - 2) / 4 of the
        // tile's columns; EPI_LOSS loads its targets D chunks ahead, the first before the MMAs finish.
        // A warp whose wait gave up stays in the loop without touching memory, so that all eight
        // epilogue warps pass the same number of named barriers.
        constexpr int HB = BN / 2, NCH = HB / 16, D = 4;
        const int q = warp & 3, h = (warp - 2) >> 2, et = threadIdx.x - 64;
        float lsum = 0.f;
        bool dead = false;
        int t = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++t) {
            const int a = t & 1;
            int m0, n0;
            origin(tile, m0, n0);
            const int m = m0 + q * 32 + lane;
            float tg[D][16];
            if (mode == EPI_LOSS && m < M && !dead) {
#pragma unroll
                for (int i = 0; i < D; ++i)
                    if (n0 + h * HB + 16 * i < N) load_targets16(ep, m, n0 + h * HB + 16 * i, N, tg[i]);
            }
            // tcgen05.ld is .sync.aligned: the whole warp must take the same branch
            if (!dead && !__all_sync(0xffffffffu, mbar_wait(&acc_full[a], (t >> 1) & 1, abort) && !*abort)) {
                if (ep.err && lane == 0) atomicOr(ep.err, 4);
                dead = true;
            }
            tc_fence_after();
            const uint32_t tb = tmem_base + (uint32_t)(a * BN) + ((uint32_t)(q * 32) << 16);
            // the tile's column parameters, once per tile in shared memory (two buffers: a warp may
            // start the next tile while others finish this one): scale std and shift bias * std + mean
            // (EPI_OUTPUT), or the bias (EPI_BIAS_ACT, EPI_LOSS)
            float* sp = prm + (t & 1) * 2 * BN;
            if (mode == EPI_OUTPUT) {
                for (int c = et; c < BN; c += 256) {
                    const int n = min(n0 + c, N - 1);
                    const float sd = ep.col_std[n];
                    sp[c] = sd;
                    sp[BN + c] = ep.bias[n] * sd + ep.col_mean[n];
                }
                asm volatile("bar.sync 1, 256;" ::: "memory");  // the eight epilogue warps
            } else if (mode == EPI_BIAS_ACT || mode == EPI_LOSS) {
                for (int c = et; c < BN; c += 256) sp[c] = ep.bias[min(n0 + c, N - 1)];
                asm volatile("bar.sync 1, 256;" ::: "memory");
            }
            if (dead) continue;
            if (mode == EPI_LOSS) {
                // unrolled, so that the target ring is indexed statically
#pragma unroll
                for (int i = 0; i < NCH; ++i) {
                    const int c0 = h * HB + 16 * i;
                    if (n0 + c0 >= N) break;  // warp-uniform
                    float v[16];
                    tmem_ld16(tb + (uint32_t)c0, v);
                    if (m < M) {
                        loss16(ep, m, n0 + c0, N, v, lsum, sp + c0, tg[i % D]);
                        if (i + D < NCH && n0 + c0 + 16 * D < N) load_targets16(ep, m, n0 + c0 + 16 * D, N, tg[i % D]);
                    }
                }
            } else if (OUT_TMA && mode == EPI_OUTPUT) {
                // the warp's 32 rows x 16 columns into its staging box, then one tensor store (rows
                // beyond M and columns beyond N are clipped by the copy engine)
                float* box = ostage + (warp - 2) * 512;
#pragma unroll 1
                for (int i = 0; i < NCH; ++i) {
                    const int c0 = h * HB + 16 * i;
                    const int n0c = n0 + c0;
                    if (n0c >= N) break;  // warp-uniform
                    float v[16];
                    tmem_ld16(tb + (uint32_t)c0, v);
                    scale16(v, sp + c0, sp + BN + c0);
                    if (lane == 0) bulk_wait_read_all();  // the previous store has read the box
                    __syncwarp();
                    float4* row = reinterpret_cast<float4*>(box + lane * 16);
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4)
                        row[q4] = make_float4(v[4 * q4], v[4 * q4 + 1], v[4 * q4 + 2], v[4 * q4 + 3]);
                    fence_proxy_async();  // generic writes, read next by the tensor store (async proxy)
                    __syncwarp();
                    if (lane == 0 && m0 + q * 32 < M) {  // (a box wholly below the last row is not stored)
                        if (n0c < ep.split) tma_store_2d(&tmO, box, n0c, m0 + q * 32);
                        else tma_store_2d(&tmO2, box, n0c - ep.split, m0 + q * 32);
                        bulk_commit_group();
                    }
                }
            } else {
#pragma unroll 1
                for (int i = 0; i < NCH; ++i) {
                    const int c0 = h * HB + 16 * i;
                    if (n0 + c0 >= N) break;  // warp-uniform
                    float v[16];
                    tmem_ld16(tb + (uint32_t)c0, v);
                    if (m < M) {
                        if (mode == EPI_OUTPUT)
                            output16(ep, m, n0 + c0, N, v, sp + c0, sp + BN + c0);
                        else
                            epilogue16(mode, ep, m, n0 + c0, N, v, sp + c0, tile / (mt * ntl));
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[a])) : "memory");
        }
        if (mode == EPI_LOSS && ep.loss_acc) {
            for (int off = 16; off > 0; off >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, off);
            if (lane == 0) atomicAdd(ep.loss_acc, lsum);
        }
        if (OUT_TMA && lane == 0) bulk_wait_all();  // every store of this warp complete before exit
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        // the last commit tracks every MMA this CTA issued: never free TMEM under one in flight
        if (lane == 0 && committed > 0) {
            const int last = committed - 1;
            const long long t0 = clock64();
            while (!mbar_try_wait(&acc_full[last & 1], (last >> 1) & 1) && clock64() - t0 < kWaitCycles) {
            }
        }
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, S::TMEM_COLS);
    }
}

}  // namespace tc
