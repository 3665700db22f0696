// Element network (Sec. 2.4, eq. param2sol; Sec. 3.1 training recipe) on the tcgen05 GEMM of
// tc_gemm.cuh, plus the learned local stage with the energy-balance error estimate and the
// classical fallback.
//
// Per batch of B samples (B a multiple of 64), with w the hidden width and L = n_hidden:
//   forward   H_l = act(H_{l-1} W_l^T + b_l)       GEMM M=B, N=w, K=in     (EPI_BIAS_ACT, keeps Z_l, H_l^T)
//             Y   = H_L W_out^T + b_out             GEMM M=B, N=n_out, K=w  (EPI_OUTPUT or EPI_LOSS)
//   backward  dW_out = dY^T H_L                     GEMM M=n_out, N=w, K=B  (A = dY^T, B = H_L^T)
//             dZ_L = (dY W_out) * act'(Z_L)         GEMM M=B, N=w, K=n_out  (B operand = W_out^T copy)
//             ... down to layer 1; bias gradients are row sums of dZ^T.
// Weights: FP32 masters updated by Adam, BF16 copies W (K-major for the forward) and W^T (K-major
// for the backward) refreshed after every update.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "elrt_internal.h"
#include "tc_gemm.cuh"

using bf16 = __nv_bfloat16;

namespace {

constexpr int kT = 256;

// ------------------------------------------------------------------------------------------------
// tensor maps
// ------------------------------------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool load_encode() {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    return g_encode != nullptr;
}

// 2D bf16 row-major matrix [rows][cols] (cols contiguous), box = box_rows x 64 columns, 128B swizzle.
bool make_map(CUtensorMap* m, const bf16* ptr, int64_t rows, int64_t cols, int box_rows) {
    if (((uintptr_t)ptr & 15) || (cols * 2) % 16) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)ptr, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// an FP32 output matrix [rows][cols] (row pitch ld floats) for the output layer's tensor stores: box
// 16 columns x 32 rows, no swizzle
bool make_out_map(CUtensorMap* m, const float* ptr, int64_t rows, int64_t cols, int64_t ld) {
    if (!ptr || ((uintptr_t)ptr & 15) || (ld * 4) % 16 || cols < 1) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {16, 32};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)ptr, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// ------------------------------------------------------------------------------------------------
// small kernels
// ------------------------------------------------------------------------------------------------

__device__ __forceinline__ uint64_t mix64(uint64_t z) {  // splitmix64 finaliser
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// W[o][i] ~ U(-bound, bound) for i < in, 0 in the padding columns
__global__ void k_init_uniform(float* W, int out, int in, int in_pad, float bound, uint64_t seed) {
    const int64_t n = (int64_t)out * in_pad;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(k % in_pad);
        const double u = (double)(mix64(seed ^ (uint64_t)k * 0x2545F4914F6CDD1Dull) >> 11) * (1.0 / 9007199254740992.0);
        W[k] = i < in ? (float)((2.0 * u - 1.0) * bound) : 0.f;
    }
}

// BF16 copies W (rows x cols) and W^T (cols x rows) through 32 x 32 shared tiles.
__global__ void k_bf16_copies(const float* __restrict__ W, int rows, int cols, bf16* __restrict__ Wb,
                              bf16* __restrict__ Wt) {
    __shared__ float tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int j = ty; j < 32; j += 8) {
        const int r = r0 + j, c = c0 + tx;
        float v = 0.f;
        if (r < rows && c < cols) {
            v = W[(int64_t)r * cols + c];
            Wb[(int64_t)r * cols + c] = __float2bfloat16_rn(v);
        }
        tile[j][tx] = v;
    }
    __syncthreads();
    if (!Wt) return;
    for (int j = ty; j < 32; j += 8) {
        const int c = c0 + j, r = r0 + tx;
        if (r < rows && c < cols) Wt[(int64_t)c * rows + r] = __float2bfloat16_rn(tile[tx][j]);
    }
}

// raw features: log(kappa_hat + 1e-12) (lin = 0) or kappa_hat itself (lin = 1) at the nodes, then
// omega; fp32 [n][fpad] (padding zero)
__global__ void k_features_raw(const double* __restrict__ kappa, const double* __restrict__ omega, double h,
                               const double* __restrict__ h_elem, int64_t n, int nm, int fpad, int lin,
                               float* __restrict__ F) {
    const int64_t total = n * fpad;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = k / fpad;
        const int i = (int)(k - e * fpad);
        float v = 0.f;
        if (i < nm) {
            const double he = h_elem ? h_elem[e] : h;
            const double kh = kappa[e * nm + i] * 0.5 * he;
            v = (float)(lin ? kh : log(kh + 1e-12));
        } else if (i == nm) {
            v = (float)omega[e];
        }
        F[k] = v;
    }
}

// per-column mean and standard deviation of two side-by-side matrices A [n][ca] | B [n][cb]
__global__ void k_col_stats(const float* __restrict__ A, int64_t ca, const float* __restrict__ B, int64_t cb, int64_t n,
                            float* __restrict__ mean, float* __restrict__ stdv, float floor_std) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= ca + cb) return;
    double s = 0.0, s2 = 0.0;
    for (int64_t r = 0; r < n; ++r) {
        const double v = c < ca ? (double)A[r * ca + c] : (double)B[r * cb + (c - ca)];
        s += v;
        s2 += v * v;
    }
    const double m = s / (double)n;
    const double var = fmax(s2 / (double)n - m * m, 0.0);
    mean[c] = (float)m;
    stdv[c] = (float)fmax(sqrt(var), (double)floor_std);
}

// standardised features of batch rows: X[b] = (F[idx(b)] - mean) / std (bf16), and X^T
__global__ void k_batch_features(const float* __restrict__ F, int fpad, int nfeat, const float* __restrict__ mean,
                                 const float* __restrict__ stdv, int64_t n, int64_t b0, int B, uint64_t pa, uint64_t pb,
                                 bf16* __restrict__ X, bf16* __restrict__ Xt) {
    const int64_t total = (int64_t)B * fpad;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(k / fpad), i = (int)(k - (int64_t)b * fpad);
        const int64_t src = (int64_t)(((uint64_t)(b0 + b) * pa + pb) % (uint64_t)n);
        float v = 0.f;
        if (i < nfeat) v = (F[src * fpad + i] - mean[i]) / stdv[i];
        const bf16 x = __float2bfloat16_rn(v);
        X[k] = x;
        if (Xt) Xt[(int64_t)i * B + b] = x;
    }
}

// standardised targets of batch rows from the labels in2out | in2sol: blockIdx.y walks the batch rows
// (the source row once per row, no division per element), blockIdx.x the columns, four at a time when
// both label widths are multiples of 4 (V = 4: no group straddles the in2out | in2sol seam)
template <int V>
__global__ void k_batch_targets(const float* __restrict__ i2o, int64_t co, const float* __restrict__ i2m, int64_t cm,
                                const float* __restrict__ mean, const float* __restrict__ stdv, int64_t n, int64_t b0,
                                int B, uint64_t pa, uint64_t pb, float* __restrict__ T) {
    const int64_t C = co + cm;
    for (int b = blockIdx.y; b < B; b += gridDim.y) {
        const int64_t src = (int64_t)(((uint64_t)(b0 + b) * pa + pb) % (uint64_t)n);
        const float* ro = i2o + src * co;
        const float* rm = i2m + src * cm - co;
        float* t = T + (int64_t)b * C;
        for (int64_t c = V * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x); c < C;
             c += V * (int64_t)gridDim.x * blockDim.x) {
            if constexpr (V == 4) {
                const float4 v = __ldcs(reinterpret_cast<const float4*>(c < co ? ro + c : rm + c));
                const float4 mu = *reinterpret_cast<const float4*>(mean + c);
                const float4 sd = *reinterpret_cast<const float4*>(stdv + c);
                *reinterpret_cast<float4*>(t + c) =
                    make_float4((v.x - mu.x) / sd.x, (v.y - mu.y) / sd.y, (v.z - mu.z) / sd.z, (v.w - mu.w) / sd.w);
            } else {
                const float v = c < co ? __ldcs(ro + c) : __ldcs(rm + c);
                t[c] = (v - mean[c]) / stdv[c];
            }
        }
    }
}

__global__ void k_f32_to_bf16(const float* __restrict__ x, int64_t n, bf16* __restrict__ y) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        y[k] = __float2bfloat16_rn(x[k]);
}

// g[r] = sum_b Dt[r][b]  (bias gradients from the transposed output gradients)
__global__ void k_rowsum_bf16(const bf16* __restrict__ Dt, int rows, int B, float* __restrict__ g) {
    const int r = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    float s = 0.f;
    for (int b = lane; b < B; b += 32) s += __bfloat162float(Dt[(int64_t)r * B + b]);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) g[r] = s;
}

// Adam (Kingma & Ba) with bias correction on FP32 masters
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float bc1, float bc2) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        p[k] -= lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
    }
}

// Adam on a weight matrix W (rows x cols) fused with its BF16 copies W and W^T, through 64 x 32 tiles
// (each element read and written once; the transposed copy leaves in 128-byte rows)
__global__ void k_adam_weights(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                               float* __restrict__ v, int rows, int cols, float lr, float b1, float b2, float eps,
                               float bc1, float bc2, bf16* __restrict__ Wb, bf16* __restrict__ Wt) {
    __shared__ float tile[64][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 64;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int j = ty; j < 64; j += 8) {
        const int r = r0 + j, c = c0 + tx;
        float pk = 0.f;
        if (r < rows && c < cols) {
            const int64_t k = (int64_t)r * cols + c;
            const float gk = __ldcs(g + k);
            const float mk = b1 * m[k] + (1.f - b1) * gk;
            const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
            m[k] = mk;
            v[k] = vk;
            pk = p[k] - lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
            p[k] = pk;
            Wb[k] = __float2bfloat16_rn(pk);
        }
        tile[j][tx] = pk;
    }
    __syncthreads();
    const int r = r0 + 2 * tx;
    for (int j = ty; j < 32; j += 8) {
        const int c = c0 + j;
        if (c >= cols || r >= rows) continue;
        bf16* dst = Wt + (int64_t)c * rows + r;
        if ((rows & 1) == 0) {  // r even, rows even: a 4-byte aligned pair
            *reinterpret_cast<__nv_bfloat162*>(dst) = __floats2bfloat162_rn(tile[2 * tx][j], tile[2 * tx + 1][j]);
        } else {
            dst[0] = __float2bfloat16_rn(tile[2 * tx][j]);
            if (r + 1 < rows) dst[1] = __float2bfloat16_rn(tile[2 * tx + 1][j]);
        }
    }
}

// dZ = (sum over K slices of the partial products) * act'(Z), as BF16 dZ [M][N] and dZ^T [N][M]
__global__ void k_dact_reduce(const float* __restrict__ part, int S, size_t stride, int M, int N,
                              const bf16* __restrict__ z, int act, bf16* __restrict__ out, bf16* __restrict__ out_t) {
    __shared__ float tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int j = ty; j < 32; j += 8) {
        const int r = r0 + j, c = c0 + tx;
        float a = 0.f;
        if (r < M && c < N) {
            const size_t k = (size_t)r * N + c;
            for (int sl = 0; sl < S; ++sl) a += __ldcs(part + sl * stride + k);
            a *= tc::act_df(__bfloat162float(z[k]), act);
            out[k] = __float2bfloat16_rn(a);
        }
        tile[j][tx] = a;
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const int c = c0 + j, r = r0 + tx;
        if (r < M && c < N) out_t[(size_t)c * M + r] = __float2bfloat16_rn(tile[tx][j]);
    }
}

unsigned grid_of(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(152 * 8, (n + kT - 1) / kT)); }

}  // namespace

// ------------------------------------------------------------------------------------------------
// the network object
// ------------------------------------------------------------------------------------------------

struct NetLayer {
    int in = 0, in_pad = 0, out = 0;
    float *W = nullptr, *b = nullptr, *gW = nullptr, *gb = nullptr;
    float *mW = nullptr, *vW = nullptr, *mb = nullptr, *vb = nullptr;
    bf16 *Wb = nullptr, *Wt = nullptr;
};

struct elrt_net {
    elrt_net_desc desc{};
    cudaStream_t stream = nullptr;
    int nm = 0, nin = 0, nfeat = 0, fpad = 0, width = 0, nout = 0, split = 0, act = 0;
    std::vector<NetLayer> L;
    float *feat_mean = nullptr, *feat_std = nullptr, *out_mean = nullptr, *out_std = nullptr;
    float *zeros = nullptr, *ones = nullptr;  // identity standardisation of the outputs (raw forward)
    bool normalised = false;
    int64_t step = 0;
    void* pbuf = nullptr;  // parameters, gradients, moments
    void* bbuf = nullptr;  // batch activations
    size_t bbuf_bytes = 0;
    int bbuf_B = 0;
    int* d_err = nullptr;
    float* d_loss = nullptr;
    float* h_loss = nullptr;
    std::string last_error;
    // batch buffers (valid for bbuf_B)
    bf16 *X0 = nullptr, *X0t = nullptr;
    std::vector<bf16*> Z, H, Ht, dZ, dZt;
    bf16 *dY = nullptr, *dYt = nullptr;
    float* T = nullptr;
    int dh_split = 1;       // K slices of the output layer's input-gradient GEMM
    float* part = nullptr;  // its FP32 partial products [dh_split][B][width]
};

namespace {

elrt_status net_fail(elrt_net* net, elrt_status s, const std::string& m) {
    if (net) net->last_error = m;
    return s;
}

elrt_status net_cuda(elrt_net* net, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return ELRT_OK;
    return net_fail(net, e == cudaErrorMemoryAllocation ? ELRT_ENOMEM : ELRT_ECUDA,
                    std::string(what) + ": " + cudaGetErrorString(e));
}

// K slices for a GEMM with few output tiles and a long K (the output layer's input gradient, K = the
// number of outputs): the count s <= 8 that minimises the rounds of work items per slice length on 152
// SMs, keeping at least 8 k-blocks per slice
int k_slices(int M, int N, int K) {
    const int tiles = ((M + tc::BM - 1) / tc::BM) * ((N + 127) / 128);
    const int nkb = (K + tc::BK - 1) / tc::BK;
    int best = 1;
    double bt = 1.0;
    for (int sl = 2; sl <= 8 && nkb >= 8 * sl; ++sl) {
        const double t = (double)((tiles * sl + 151) / 152) / sl;
        if (t < bt - 1e-9) {
            bt = t;
            best = sl;
        }
    }
    return best;
}

// D = A . B^T with the chosen epilogue (A [M][K], B [N][K] bf16, K % 8 == 0)
elrt_status gemm(elrt_net* net, const bf16* A, const bf16* Bm, int M, int N, int K, int mode, tc::EpiArgs ep) {
    ep.err = net->d_err;
    CUtensorMap ta, tb;
    // 256-column tiles for wide outputs, and for long-M GEMMs with many tiles (the output layer's weight
    // gradient), where they cut the operand bytes each SM streams per flop by a quarter
    const bool wide = N >= 2048 || (N % 256 == 0 && ((M + tc::BM - 1) / tc::BM) * (N / 256) >= 4 * 152);
    if (!make_map(&ta, A, M, K, tc::BM) || !make_map(&tb, Bm, N, K, wide ? 256 : 128))
        return net_fail(net, ELRT_EINVAL, "tensor map encoding failed (alignment or stride)");
    const int tiles = ((M + tc::BM - 1) / tc::BM) * (wide ? (N + 255) / 256 : (N + 127) / 128) * std::max(1, ep.ksplit);
    dim3 grid(std::min(tiles, 152));
    // the output layer writes its tiles with tensor stores when both destinations allow the maps
    CUtensorMap to = ta, to2 = ta;
    const bool otma = mode == tc::EPI_OUTPUT && ep.split % 16 == 0 &&
                      make_out_map(&to, ep.out_f, M, std::min(ep.split, N), ep.ld_out) &&
                      (ep.split >= N || make_out_map(&to2, ep.out_f2, M, N - ep.split, ep.ld_out2));
    if (otma && ep.split >= N) to2 = to;
    if (wide && otma) {
        const int smem = tc::GemmSmem<256, true>::TOTAL;
        cudaFuncSetAttribute(tc::k_gemm_bf16<256, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        tc::k_gemm_bf16<256, true><<<grid, tc::kGemmThreads, smem, net->stream>>>(ta, tb, M, N, K, mode, ep, to, to2);
    } else if (otma) {
        const int smem = tc::GemmSmem<128, true>::TOTAL;
        cudaFuncSetAttribute(tc::k_gemm_bf16<128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        tc::k_gemm_bf16<128, true><<<grid, tc::kGemmThreads, smem, net->stream>>>(ta, tb, M, N, K, mode, ep, to, to2);
    } else if (wide) {
        const int smem = tc::GemmSmem<256>::TOTAL;
        cudaFuncSetAttribute(tc::k_gemm_bf16<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        tc::k_gemm_bf16<256><<<grid, tc::kGemmThreads, smem, net->stream>>>(ta, tb, M, N, K, mode, ep, to, to2);
    } else {
        const int smem = tc::GemmSmem<128>::TOTAL;
        cudaFuncSetAttribute(tc::k_gemm_bf16<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        tc::k_gemm_bf16<128><<<grid, tc::kGemmThreads, smem, net->stream>>>(ta, tb, M, N, K, mode, ep, to, to2);
    }
    return net_cuda(net, cudaGetLastError(), "gemm launch");
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

elrt_status ensure_batch(elrt_net* net, int B) {
    if (net->bbuf && net->bbuf_B == B) return ELRT_OK;
    if (net->bbuf) {
        cudaStreamSynchronize(net->stream);
        cudaFree(net->bbuf);
        net->bbuf = nullptr;
    }
    const int nh = (int)net->L.size() - 1, w = net->width;
    size_t bytes = 0;
    auto add = [&](size_t n) { bytes += align256(n); };
    add((size_t)B * net->fpad * 2);
    add((size_t)B * net->fpad * 2);
    for (int l = 0; l < nh; ++l)
        for (int j = 0; j < 5; ++j) add((size_t)B * w * 2);
    add((size_t)B * net->nout * 2);
    add((size_t)B * net->nout * 2);
    add((size_t)B * net->nout * 4);
    const int dsplit = nh > 0 ? k_slices(B, w, net->nout) : 1;
    if (dsplit > 1) add((size_t)dsplit * B * w * 4);
    cudaError_t e = cudaMalloc(&net->bbuf, bytes);
    if (e != cudaSuccess) return net_cuda(net, e, "batch buffers");
    net->bbuf_bytes = bytes;
    net->bbuf_B = B;
    unsigned char* p = (unsigned char*)net->bbuf;
    auto take = [&](size_t n) {
        unsigned char* q = p;
        p += align256(n);
        return q;
    };
    net->X0 = (bf16*)take((size_t)B * net->fpad * 2);
    net->X0t = (bf16*)take((size_t)B * net->fpad * 2);
    net->Z.assign(nh, nullptr);
    net->H.assign(nh, nullptr);
    net->Ht.assign(nh, nullptr);
    net->dZ.assign(nh, nullptr);
    net->dZt.assign(nh, nullptr);
    for (int l = 0; l < nh; ++l) {
        net->Z[l] = (bf16*)take((size_t)B * w * 2);
        net->H[l] = (bf16*)take((size_t)B * w * 2);
        net->Ht[l] = (bf16*)take((size_t)B * w * 2);
        net->dZ[l] = (bf16*)take((size_t)B * w * 2);
        net->dZt[l] = (bf16*)take((size_t)B * w * 2);
    }
    net->dY = (bf16*)take((size_t)B * net->nout * 2);
    net->dYt = (bf16*)take((size_t)B * net->nout * 2);
    net->T = (float*)take((size_t)B * net->nout * 4);
    net->dh_split = dsplit;
    net->part = dsplit > 1 ? (float*)take((size_t)dsplit * B * w * 4) : nullptr;
    return ELRT_OK;
}

elrt_status refresh_bf16(elrt_net* net) {
    for (auto& ly : net->L) {
        dim3 g((ly.in_pad + 31) / 32, (ly.out + 31) / 32);
        k_bf16_copies<<<g, 256, 0, net->stream>>>(ly.W, ly.out, ly.in_pad, ly.Wb, ly.Wt);
    }
    return net_cuda(net, cudaGetLastError(), "bf16 copies");
}

// Forward over a batch already in X0 (B rows).  mode: 0 inference into (out, out2), 1 training loss.
elrt_status forward_batch(elrt_net* net, int B, int mode, float* out, float* out2, int ld_out, int ld_out2,
                          bool keep, bool raw = false) {
    const int nh = (int)net->L.size() - 1;
    const bf16* in = net->X0;
    int kin = net->fpad;
    elrt_status s;
    for (int l = 0; l < nh; ++l) {
        tc::EpiArgs ep;
        ep.bias = net->L[l].b;
        ep.out_bf = net->H[l];
        ep.z_out = keep ? net->Z[l] : nullptr;
        ep.out_bf_t = keep ? net->Ht[l] : nullptr;
        ep.ld_out = net->width;
        ep.ld_t = B;
        ep.act = net->act;
        s = gemm(net, in, net->L[l].Wb, B, net->width, kin, tc::EPI_BIAS_ACT, ep);
        if (s) return s;
        in = net->H[l];
        kin = net->width;
    }
    NetLayer& o = net->L[nh];
    tc::EpiArgs ep;
    ep.bias = o.b;
    if (mode == 0) {
        ep.out_f = out;
        ep.out_f2 = out2;
        ep.ld_out = ld_out;
        ep.ld_out2 = ld_out2;
        ep.split = out2 ? net->split : net->nout;
        ep.col_mean = raw ? net->zeros : net->out_mean;
        ep.col_std = raw ? net->ones : net->out_std;
        return gemm(net, in, o.Wb, B, net->nout, kin, tc::EPI_OUTPUT, ep);
    }
    ep.target = net->T;
    ep.out_bf = net->dY;
    ep.out_bf_t = net->dYt;
    ep.ld_out = net->nout;
    ep.ld_t = B;
    ep.loss_acc = net->d_loss;
    ep.loss_scale = 1.0f / ((float)B * (float)net->nout);
    return gemm(net, in, o.Wb, B, net->nout, kin, tc::EPI_LOSS, ep);
}

elrt_status backward_batch(elrt_net* net, int B) {
    const int nh = (int)net->L.size() - 1;
    elrt_status s;
    // output layer
    {
        NetLayer& o = net->L[nh];
        const bf16* hin_t = nh > 0 ? net->Ht[nh - 1] : net->X0t;
        const int kin = nh > 0 ? net->width : net->fpad;
        tc::EpiArgs ep;
        ep.out_f = o.gW;
        ep.ld_out = kin;
        s = gemm(net, net->dYt, hin_t, net->nout, kin, B, tc::EPI_F32, ep);
        if (s) return s;
        k_rowsum_bf16<<<(net->nout + 7) / 8, 256, 0, net->stream>>>(net->dYt, net->nout, B, o.gb);
        if (nh > 0 && net->dh_split > 1) {
            // few output tiles, K = the number of outputs: K slices into FP32 partials, then one pass
            // that sums them and applies the activation derivative
            tc::EpiArgs ed;
            ed.out_f = net->part;
            ed.ld_out = net->width;
            ed.ksplit = net->dh_split;
            ed.part_stride = (size_t)B * net->width;
            s = gemm(net, net->dY, o.Wt, B, net->width, net->nout, tc::EPI_F32, ed);
            if (s) return s;
            const dim3 g((net->width + 31) / 32, (B + 31) / 32);
            k_dact_reduce<<<g, 256, 0, net->stream>>>(net->part, net->dh_split, ed.part_stride, B, net->width,
                                                      net->Z[nh - 1], net->act, net->dZ[nh - 1], net->dZt[nh - 1]);
        } else if (nh > 0) {
            tc::EpiArgs ed;
            ed.z_in = net->Z[nh - 1];
            ed.out_bf = net->dZ[nh - 1];
            ed.out_bf_t = net->dZt[nh - 1];
            ed.ld_out = net->width;
            ed.ld_t = B;
            ed.act = net->act;
            s = gemm(net, net->dY, o.Wt, B, net->width, net->nout, tc::EPI_DACT, ed);
            if (s) return s;
        }
    }
    for (int l = nh - 1; l >= 0; --l) {
        NetLayer& ly = net->L[l];
        const bf16* hin_t = l > 0 ? net->Ht[l - 1] : net->X0t;
        const int kin = l > 0 ? net->width : net->fpad;
        tc::EpiArgs ep;
        ep.out_f = ly.gW;
        ep.ld_out = kin;
        s = gemm(net, net->dZt[l], hin_t, net->width, kin, B, tc::EPI_F32, ep);
        if (s) return s;
        k_rowsum_bf16<<<(net->width + 7) / 8, 256, 0, net->stream>>>(net->dZt[l], net->width, B, ly.gb);
        if (l > 0) {
            tc::EpiArgs ed;
            ed.z_in = net->Z[l - 1];
            ed.out_bf = net->dZ[l - 1];
            ed.out_bf_t = net->dZt[l - 1];
            ed.ld_out = net->width;
            ed.ld_t = B;
            ed.act = net->act;
            s = gemm(net, net->dZ[l], ly.Wt, B, net->width, net->width, tc::EPI_DACT, ed);
            if (s) return s;
        }
    }
    return net_cuda(net, cudaGetLastError(), "backward");
}

elrt_status adam_update(elrt_net* net, float lr, float b1, float b2, float eps) {
    net->step += 1;
    const float bc1 = 1.f - powf(b1, (float)net->step), bc2 = 1.f - powf(b2, (float)net->step);
    for (auto& ly : net->L) {
        const dim3 g((ly.in_pad + 31) / 32, (ly.out + 63) / 64);
        k_adam_weights<<<g, kT, 0, net->stream>>>(ly.W, ly.gW, ly.mW, ly.vW, ly.out, ly.in_pad, lr, b1, b2, eps, bc1,
                                                  bc2, ly.Wb, ly.Wt);
        k_adam<<<grid_of(ly.out), kT, 0, net->stream>>>(ly.b, ly.gb, ly.mb, ly.vb, ly.out, lr, b1, b2, eps, bc1, bc2);
    }
    return net_cuda(net, cudaGetLastError(), "adam");
}

elrt_status check_err(elrt_net* net) {
    int herr = 0;
    cudaError_t e = cudaMemcpyAsync(&herr, net->d_err, sizeof(int), cudaMemcpyDeviceToHost, net->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
    if (e != cudaSuccess) return net_cuda(net, e, "sync");
    if (herr) {
        cudaMemsetAsync(net->d_err, 0, sizeof(int), net->stream);
        return net_fail(net, ELRT_ETIMEOUT, "a tensor-core GEMM wait timed out (code " + std::to_string(herr) + ")");
    }
    return ELRT_OK;
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// ABI
// ------------------------------------------------------------------------------------------------

// device arrays of a network in checkpoint order (ckpt_layout)
namespace {
std::vector<float*> ckpt_arrays(elrt_net* net) {
    std::vector<float*> a;
    for (auto& ly : net->L) {
        a.push_back(ly.W);
        a.push_back(ly.b);
        a.push_back(ly.mW);
        a.push_back(ly.vW);
        a.push_back(ly.mb);
        a.push_back(ly.vb);
    }
    a.push_back(net->feat_mean);
    a.push_back(net->feat_std);
    a.push_back(net->out_mean);
    a.push_back(net->out_std);
    return a;
}
}  // namespace

extern "C" {

elrt_status elrt_net_create(elrt_net** out, const elrt_net_desc* d, void* stream) {
    if (!out || !d) return ELRT_EINVAL;
    *out = nullptr;
    elrt_disc disc{d->p, d->n_angles, 0, 0.0};
    if (!elrt_disc_valid(&disc) || d->n_hidden < 0 || d->n_hidden > 8 || d->width < 64 || d->width % 64 ||
        (d->activation != 0 && d->activation != 1) || (d->features != 0 && d->features != 1))
        return ELRT_EINVAL;
    if (!load_encode()) return ELRT_ECUDA;
    elrt_net* net = new (std::nothrow) elrt_net();
    if (!net) return ELRT_ENOMEM;
    net->desc = *d;
    net->stream = (cudaStream_t)stream;
    const int n1 = d->p + 1;
    net->nm = n1 * n1;
    net->nin = 2 * n1 * d->n_angles;
    net->nfeat = net->nm + 1;
    net->fpad = ((net->nfeat + 63) / 64) * 64;
    net->width = d->width;
    net->nout = net->nin * net->nin + net->nm * net->nin;
    net->split = net->nin * net->nin;
    net->act = d->activation;
    const int nl = d->n_hidden + 1;
    net->L.resize(nl);
    size_t floats = 0, halfs = 0;
    for (int l = 0; l < nl; ++l) {
        NetLayer& ly = net->L[l];
        ly.in = l == 0 ? net->nfeat : net->width;
        ly.in_pad = l == 0 ? net->fpad : net->width;
        ly.out = l == nl - 1 ? net->nout : net->width;
        const size_t nw = (size_t)ly.out * ly.in_pad;
        floats += 4 * align256(nw * 4) / 4 + 4 * align256((size_t)ly.out * 4) / 4;  // W gW mW vW, b gb mb vb
        halfs += 2 * align256(nw * 2) / 2;
    }
    floats += 2 * align256((size_t)net->fpad * 4) / 4 + 4 * align256((size_t)net->nout * 4) / 4 + 64;
    cudaError_t e = cudaMalloc(&net->pbuf, floats * 4 + halfs * 2 + 4096);
    if (e == cudaSuccess) e = cudaMallocHost(&net->h_loss, 64);
    if (e != cudaSuccess) {
        if (net->pbuf) cudaFree(net->pbuf);
        delete net;
        return e == cudaErrorMemoryAllocation ? ELRT_ENOMEM : ELRT_ECUDA;
    }
    unsigned char* p = (unsigned char*)net->pbuf;
    auto take = [&](size_t bytes) {
        unsigned char* q = p;
        p += align256(bytes);
        return q;
    };
    for (int l = 0; l < nl; ++l) {
        NetLayer& ly = net->L[l];
        const size_t nw = (size_t)ly.out * ly.in_pad;
        ly.W = (float*)take(nw * 4);
        ly.gW = (float*)take(nw * 4);
        ly.mW = (float*)take(nw * 4);
        ly.vW = (float*)take(nw * 4);
        ly.b = (float*)take((size_t)ly.out * 4);
        ly.gb = (float*)take((size_t)ly.out * 4);
        ly.mb = (float*)take((size_t)ly.out * 4);
        ly.vb = (float*)take((size_t)ly.out * 4);
        ly.Wb = (bf16*)take(nw * 2);
        ly.Wt = (bf16*)take(nw * 2);
    }
    net->feat_mean = (float*)take((size_t)net->fpad * 4);
    net->feat_std = (float*)take((size_t)net->fpad * 4);
    net->out_mean = (float*)take((size_t)net->nout * 4);
    net->out_std = (float*)take((size_t)net->nout * 4);
    net->zeros = (float*)take((size_t)net->nout * 4);
    net->ones = (float*)take((size_t)net->nout * 4);
    net->d_err = (int*)take(64);
    net->d_loss = (float*)take(64);
    cudaStream_t sm = net->stream;
    cudaMemsetAsync(net->pbuf, 0, p - (unsigned char*)net->pbuf, sm);
    for (int l = 0; l < nl; ++l) {
        NetLayer& ly = net->L[l];
        const float bound = 1.0f / sqrtf((float)ly.in);
        k_init_uniform<<<grid_of((int64_t)ly.out * ly.in_pad), kT, 0, sm>>>(ly.W, ly.out, ly.in, ly.in_pad, bound,
                                                                             d->seed * 1315423911ull + l);
        k_init_uniform<<<grid_of(ly.out), kT, 0, sm>>>(ly.b, ly.out, 1, 1, bound, d->seed * 2654435761ull + 101 + l);
    }
    refresh_bf16(net);
    // identity standardisation until fitted
    std::vector<float> ones(std::max(net->fpad, net->nout), 1.f);
    cudaMemcpyAsync(net->feat_std, ones.data(), net->fpad * 4, cudaMemcpyHostToDevice, sm);
    cudaMemcpyAsync(net->out_std, ones.data(), (size_t)net->nout * 4, cudaMemcpyHostToDevice, sm);
    cudaMemcpyAsync(net->ones, ones.data(), (size_t)net->nout * 4, cudaMemcpyHostToDevice, sm);
    e = cudaStreamSynchronize(sm);
    if (e != cudaSuccess) {
        cudaFree(net->pbuf);
        cudaFreeHost(net->h_loss);
        delete net;
        return ELRT_ECUDA;
    }
    *out = net;
    return ELRT_OK;
}

elrt_status elrt_net_destroy(elrt_net* net) {
    if (!net) return ELRT_OK;
    cudaStreamSynchronize(net->stream);
    if (net->bbuf) cudaFree(net->bbuf);
    if (net->pbuf) cudaFree(net->pbuf);
    if (net->h_loss) cudaFreeHost(net->h_loss);
    delete net;
    return ELRT_OK;
}

elrt_status elrt_net_set_stream(elrt_net* net, void* stream) {
    if (!net) return ELRT_EINVAL;
    net->stream = (cudaStream_t)stream;
    return ELRT_OK;
}

const char* elrt_net_last_error(const elrt_net* net) { return net ? net->last_error.c_str() : ""; }

elrt_status elrt_net_sizes(const elrt_net* net, int64_t* n_feat, int64_t* n_feat_pad, int64_t* n_out,
                           int32_t* n_layers, int64_t* n_params) {
    if (!net) return ELRT_EINVAL;
    if (n_feat) *n_feat = net->nfeat;
    if (n_feat_pad) *n_feat_pad = net->fpad;
    if (n_out) *n_out = net->nout;
    if (n_layers) *n_layers = (int32_t)net->L.size();
    if (n_params) {
        int64_t np = 0;
        for (auto& ly : net->L) np += (int64_t)ly.out * ly.in + ly.out;
        *n_params = np;
    }
    return ELRT_OK;
}

elrt_status elrt_net_save(elrt_net* net, const char* path) {
    if (!net || !path) return net_fail(net, ELRT_EINVAL, "elrt_net_save: bad arguments");
    const std::vector<size_t> lay = ckpt_layout(net->desc);
    const std::vector<float*> dev = ckpt_arrays(net);
    size_t total = 0;
    for (size_t c : lay) total += c;
    std::vector<float> host(total);
    std::vector<const float*> ptrs;
    size_t off = 0;
    cudaError_t e = cudaSuccess;
    for (size_t a = 0; a < lay.size() && e == cudaSuccess; ++a) {
        e = cudaMemcpyAsync(host.data() + off, dev[a], lay[a] * 4, cudaMemcpyDeviceToHost, net->stream);
        ptrs.push_back(host.data() + off);
        off += lay[a];
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
    if (e != cudaSuccess) return net_cuda(net, e, "elrt_net_save");
    std::string err;
    if (!ckpt_write(path, net->desc, net->normalised ? 1 : 0, net->step, ptrs, &err))
        return net_fail(net, ELRT_EINVAL, err);
    return ELRT_OK;
}

elrt_status elrt_net_load(elrt_net** out, const char* path, void* stream) {
    if (!out || !path) return ELRT_EINVAL;
    *out = nullptr;
    elrt_net_desc d{};
    int32_t standardised = 0;
    int64_t step = 0, nf = 0;
    std::vector<float> payload;
    std::string err;
    if (!ckpt_read(path, &d, &standardised, &step, &nf, &payload, &err)) return ELRT_EINVAL;
    elrt_net* net = nullptr;
    elrt_status s = elrt_net_create(&net, &d, stream);
    if (s) return s;
    const std::vector<size_t> lay = ckpt_layout(d);
    const std::vector<float*> dev = ckpt_arrays(net);
    size_t off = 0;
    cudaError_t e = cudaSuccess;
    for (size_t a = 0; a < lay.size() && e == cudaSuccess; ++a) {
        e = cudaMemcpyAsync(dev[a], payload.data() + off, lay[a] * 4, cudaMemcpyHostToDevice, net->stream);
        off += lay[a];
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);  // payload is pageable host memory
    if (e == cudaSuccess) {
        net->normalised = standardised != 0;
        net->step = step;
        s = refresh_bf16(net);
        if (!s) e = cudaStreamSynchronize(net->stream);
    }
    if (s || e != cudaSuccess) {
        elrt_net_destroy(net);
        return s ? s : (e == cudaErrorMemoryAllocation ? ELRT_ENOMEM : ELRT_ECUDA);
    }
    *out = net;
    return ELRT_OK;
}

elrt_status elrt_net_params(elrt_net* net, int32_t layer, int32_t what, int32_t dir, float* host) {
    if (!net || !host || layer < 0 || layer >= (int)net->L.size() || what < 0 || what > 3 || dir < 0 || dir > 1 ||
        (dir == 1 && what > 1))
        return net_fail(net, ELRT_EINVAL, "elrt_net_params: bad arguments");
    NetLayer& ly = net->L[layer];
    float* src = what == 0 ? ly.W : what == 1 ? ly.b : what == 2 ? ly.gW : ly.gb;
    const size_t n = (what == 0 || what == 2) ? (size_t)ly.out * ly.in_pad : (size_t)ly.out;
    cudaError_t e = dir == 0 ? cudaMemcpyAsync(host, src, n * 4, cudaMemcpyDeviceToHost, net->stream)
                             : cudaMemcpyAsync(src, host, n * 4, cudaMemcpyHostToDevice, net->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
    if (e != cudaSuccess) return net_cuda(net, e, "elrt_net_params");
    if (dir == 1 && what == 0) {
        elrt_status s = refresh_bf16(net);
        if (s) return s;
        return net_cuda(net, cudaStreamSynchronize(net->stream), "refresh");
    }
    return ELRT_OK;
}

elrt_status elrt_net_forward(elrt_net* net, int64_t n, const float* x, float* y) {
    if (!net || n < 0 || (n > 0 && (!x || !y))) return net_fail(net, ELRT_EINVAL, "elrt_net_forward: bad arguments");
    const int B = std::max(1024, net->bbuf_B);
    elrt_status s = ensure_batch(net, B);
    if (s) return s;
    for (int64_t e0 = 0; e0 < n; e0 += B) {
        const int m = (int)std::min<int64_t>(B, n - e0);
        k_f32_to_bf16<<<grid_of((int64_t)m * net->fpad), kT, 0, net->stream>>>(x + e0 * net->fpad,
                                                                                (int64_t)m * net->fpad, net->X0);
        s = forward_batch(net, m, 0, y + e0 * net->nout, nullptr, net->nout, 0, false, true);
        if (s) return s;
    }
    return check_err(net);
}

elrt_status elrt_net_train_step(elrt_net* net, int64_t n, const float* x, const float* t, float lr, float* loss) {
    if (!net || n <= 0 || n % 64 || !x || !t || n > (1 << 20))
        return net_fail(net, ELRT_EINVAL, "elrt_net_train_step: n must be a positive multiple of 64");
    const int B = (int)n;
    elrt_status s = ensure_batch(net, B);
    if (s) return s;
    cudaStream_t sm = net->stream;
    // features (already standardised by the caller) and their transpose; targets
    {
        // bf16 copy and transpose through the generic copy kernel (rows = B, cols = fpad)
        dim3 g((net->fpad + 31) / 32, (B + 31) / 32);
        k_bf16_copies<<<g, 256, 0, sm>>>(x, B, net->fpad, net->X0, net->X0t);
        cudaMemcpyAsync(net->T, t, (size_t)B * net->nout * 4, cudaMemcpyDeviceToDevice, sm);
    }
    cudaMemsetAsync(net->d_loss, 0, sizeof(float), sm);
    s = forward_batch(net, B, 1, nullptr, nullptr, 0, 0, true);
    if (!s) s = backward_batch(net, B);
    if (!s && lr > 0.f) s = adam_update(net, lr, 0.9f, 0.999f, 1e-8f);
    if (s) return s;
    if (loss) {
        cudaMemcpyAsync(net->h_loss, net->d_loss, sizeof(float), cudaMemcpyDeviceToHost, sm);
        s = check_err(net);
        if (s) return s;
        *loss = net->h_loss[0] / ((float)B * (float)net->nout);
    }
    return ELRT_OK;
}

elrt_status elrt_net_fit(elrt_net* net, int64_t n, const double* kappa, const double* omega, const double* h_elem,
                         const float* in2out, const float* in2sol, const elrt_train_opts* o, float* epoch_loss) {
    if (!net || !o || n < 64 || !kappa || !omega || !h_elem || !in2out || !in2sol || o->epochs < 1 || o->batch < 64 ||
        o->batch % 64 || o->batch > n || !(o->lr > 0))
        return net_fail(net, ELRT_EINVAL, "elrt_net_fit: bad arguments (batch: multiple of 64, <= n)");
    cudaStream_t sm = net->stream;
    const int B = o->batch;
    elrt_status s = ensure_batch(net, B);
    if (s) return s;
    // raw features of the whole set and their statistics
    float* F = nullptr;
    cudaError_t e = cudaMallocAsync(&F, (size_t)n * net->fpad * 4, sm);
    if (e != cudaSuccess) return net_cuda(net, e, "feature buffer");
    k_features_raw<<<grid_of(n * net->fpad), kT, 0, sm>>>(kappa, omega, 1.0, h_elem, n, net->nm, net->fpad,
                                                          net->desc.features, F);
    k_col_stats<<<(net->fpad + 127) / 128, 128, 0, sm>>>(F, net->fpad, nullptr, 0, n, net->feat_mean, net->feat_std,
                                                         1e-3f);
    const int64_t co = (int64_t)net->nin * net->nin, cm = (int64_t)net->nm * net->nin;
    k_col_stats<<<(unsigned)((co + cm + 127) / 128), 128, 0, sm>>>(in2out, co, in2sol, cm, n, net->out_mean,
                                                                   net->out_std, 1e-6f);
    net->normalised = true;
    // sample order per epoch: b -> (b * a + c) mod n with gcd(a, n) = 1
    uint64_t rs = o->seed * 0x9E3779B97F4A7C15ull + 7;
    auto rnd = [&]() {
        rs ^= rs << 13;
        rs ^= rs >> 7;
        rs ^= rs << 17;
        return rs;
    };
    auto gcd = [](uint64_t a, uint64_t b) {
        while (b) {
            uint64_t t = a % b;
            a = b;
            b = t;
        }
        return a;
    };
    const int64_t nb = n / B;
    // float4 target rows: both label widths multiples of 4 and 16-byte aligned label buffers
    const bool vec4 = co % 4 == 0 && cm % 4 == 0 && (uintptr_t)in2out % 16 == 0 && (uintptr_t)in2sol % 16 == 0;
    const dim3 tgrid((unsigned)std::min<int64_t>(vec4 ? 4 : 8, (net->nout + kT - 1) / kT), (unsigned)std::min(B, 65535));
    const float b1 = o->beta1 > 0 ? o->beta1 : 0.9f, b2 = o->beta2 > 0 ? o->beta2 : 0.999f;
    const float eps = o->eps > 0 ? o->eps : 1e-8f;
    for (int ep = 0; ep < o->epochs; ++ep) {
        uint64_t pa = 1 + rnd() % (uint64_t)n;
        while (gcd(pa, (uint64_t)n) != 1) pa = 1 + rnd() % (uint64_t)n;
        const uint64_t pb = rnd() % (uint64_t)n;
        const float lr = o->lr * (ep < o->epochs / 3 ? 1.f : ep < 2 * o->epochs / 3 ? 0.1f : 0.01f);
        cudaMemsetAsync(net->d_loss, 0, sizeof(float), sm);
        for (int64_t bi = 0; bi < nb; ++bi) {
            k_batch_features<<<grid_of((int64_t)B * net->fpad), kT, 0, sm>>>(
                F, net->fpad, net->nfeat, net->feat_mean, net->feat_std, n, bi * B, B, pa, pb, net->X0, net->X0t);
            if (vec4)
                k_batch_targets<4><<<tgrid, kT, 0, sm>>>(in2out, co, in2sol, cm, net->out_mean, net->out_std, n,
                                                         bi * B, B, pa, pb, net->T);
            else
                k_batch_targets<1><<<tgrid, kT, 0, sm>>>(in2out, co, in2sol, cm, net->out_mean, net->out_std, n,
                                                         bi * B, B, pa, pb, net->T);
            s = forward_batch(net, B, 1, nullptr, nullptr, 0, 0, true);
            if (!s) s = backward_batch(net, B);
            if (!s) s = adam_update(net, lr, b1, b2, eps);
            if (s) {
                cudaFreeAsync(F, sm);
                return s;
            }
        }
        if (epoch_loss) {
            cudaMemcpyAsync(net->h_loss, net->d_loss, sizeof(float), cudaMemcpyDeviceToHost, sm);
            s = check_err(net);
            if (s) {
                cudaFreeAsync(F, sm);
                return s;
            }
            epoch_loss[ep] = net->h_loss[0] / ((float)nb * B * (float)net->nout);
        }
    }
    cudaFreeAsync(F, sm);
    return check_err(net);
}

elrt_status elrt_net_infer(elrt_net* net, int64_t n, double h, const double* h_elem, const double* kappa,
                           const double* omega, float* in2out, float* in2sol) {
    if (!net || n < 0 || (n > 0 && (!kappa || !omega || !in2out || !in2sol)) || (!h_elem && !(h > 0)))
        return net_fail(net, ELRT_EINVAL, "elrt_net_infer: bad arguments");
    if (!net->normalised) return net_fail(net, ELRT_ENOTRAINED, "network has no standardisation (not fitted)");
    if (n == 0) return ELRT_OK;
    const int B = 4096;
    cudaStream_t sm = net->stream;
    elrt_status s = ensure_batch(net, std::max(B, net->bbuf_B));
    if (s) return s;
    float* F = (float*)net->T;  // raw features of a chunk live in the target buffer
    for (int64_t e0 = 0; e0 < n; e0 += B) {
        const int m = (int)std::min<int64_t>(B, n - e0);
        k_features_raw<<<grid_of((int64_t)m * net->fpad), kT, 0, sm>>>(
            kappa + e0 * net->nm, omega + e0, h, h_elem ? h_elem + e0 : nullptr, m, net->nm, net->fpad,
            net->desc.features, F);
        k_batch_features<<<grid_of((int64_t)m * net->fpad), kT, 0, sm>>>(F, net->fpad, net->nfeat, net->feat_mean,
                                                                         net->feat_std, m, 0, m, 1, 0, net->X0,
                                                                         nullptr);
        s = forward_batch(net, m, 0, in2out + e0 * (int64_t)net->split, in2sol + e0 * (int64_t)net->nm * net->nin,
                          net->split, net->nm * net->nin, false);
        if (s) return s;
    }
    return net_cuda(net, cudaGetLastError(), "infer");
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// learned local stage: estimate + classical fallback
// ------------------------------------------------------------------------------------------------

namespace {

// Per element: max over inflow columns j of the relative energy-balance defect
//   | w_j |s.n|_j - sum_r w_r (s.n)_r A_i2o[r][j] - N sum_i w_i kappa_hat_i (1 - omega) A_i2m[i][j] | / (w_j |s.n|_j)
// One block per element; thread j sums its column (coalesced across threads).
__global__ void __launch_bounds__(256) k_energy_estimate(Tab t, double h, const double* __restrict__ h_elem,
                                                         const double* __restrict__ kappa,
                                                         const double* __restrict__ omega,
                                                         const float* __restrict__ i2o, const float* __restrict__ i2m,
                                                         float* __restrict__ est, int64_t E) {
    __shared__ float wout[4 * ELRT_MAX_N1 * (ELRT_MAX_ANG / 2)];
    __shared__ float absorb[ELRT_MAX_N1 * ELRT_MAX_N1];
    __shared__ float red[8];
    const int64_t e = blockIdx.x;
    if (e >= E) return;
    const int nin = t.nin, nm = t.nm, n1 = t.n1, half = t.half;
    const double he = h_elem ? h_elem[e] : h;
    const double om = omega[e];
    for (int r = threadIdx.x; r < nin; r += blockDim.x) {
        const int F = r / t.nface, rem = r - F * t.nface, m = rem / half, kk = rem - m * half;
        wout[r] = (float)(t.w[m] * t.sdn[F][t.outc[F][kk]]);
    }
    for (int i = threadIdx.x; i < nm; i += blockDim.x)
        absorb[i] = (float)(t.N * t.w[i % n1] * t.w[i / n1] * kappa[e * nm + i] * 0.5 * he * (1.0 - om));
    __syncthreads();
    float worst = 0.f;
    for (int j = threadIdx.x; j < nin; j += blockDim.x) {
        const int F = j / t.nface, rem = j - F * t.nface, m = rem / half, kk = rem - m * half;
        const float lhs = (float)(t.w[m] * fabs(t.sdn[F][t.inc[F][kk]]));
        // four independent chains (the loads of a column are independent; one chain would serialise
        // the column's 273 multiply-adds behind their loads)
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const float* A = i2o + e * (int64_t)nin * nin + j;
        int r = 0;
        for (; r + 4 <= nin; r += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fmaf(wout[r + u], A[(int64_t)(r + u) * nin], acc[u]);
        }
        for (; r < nin; ++r) acc[0] = fmaf(wout[r], A[(int64_t)r * nin], acc[0]);
        const float* Mm = i2m + e * (int64_t)nm * nin + j;
        int i = 0;
        for (; i + 4 <= nm; i += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fmaf(absorb[i + u], Mm[(int64_t)(i + u) * nin], acc[u]);
        }
        for (; i < nm; ++i) acc[0] = fmaf(absorb[i], Mm[(int64_t)i * nin], acc[0]);
        const float rhs = (acc[0] + acc[1]) + (acc[2] + acc[3]);
        const float d = fabsf(lhs - rhs) / lhs;
        worst = fmaxf(worst, d != d ? 1e30f : d);
    }
    for (int off = 16; off > 0; off >>= 1) worst = fmaxf(worst, __shfl_down_sync(0xffffffffu, worst, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = worst;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
        est[e] = m;
    }
}

__global__ void k_select(const float* __restrict__ est, int64_t E, float tol, int64_t* __restrict__ list,
                         unsigned long long* __restrict__ count) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < E && !(est[e] <= tol)) list[atomicAdd(count, 1ull)] = e;
}

__global__ void k_gather_inputs(const int64_t* __restrict__ list, int64_t n, int nm, const double* __restrict__ kappa,
                                const double* __restrict__ omega, double h, const double* __restrict__ h_elem,
                                double* __restrict__ k2, double* __restrict__ o2, double* __restrict__ h2) {
    const int64_t total = n * nm;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = k / nm;
        const int i = (int)(k - q * nm);
        const int64_t e = list[q];
        k2[k] = kappa[e * nm + i];
        if (i == 0) {
            o2[q] = omega[e];
            h2[q] = h_elem ? h_elem[e] : h;
        }
    }
}

__global__ void k_scatter_ops(const int64_t* __restrict__ list, int64_t n, int64_t per, const float* __restrict__ src,
                              float* __restrict__ dst) {
    const int64_t total = n * per;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = k / per;
        dst[list[q] * per + (k - q * per)] = src[k];
    }
}

}  // namespace

extern "C" elrt_status elrt_build_local_learned(elrt_ctx* ctx, elrt_net* net, int64_t n, double h,
                                                const double* h_elem, const double* kappa, const double* omega,
                                                double tol, float* in2out, float* in2sol, float* estimate,
                                                int64_t* n_fallback) {
    if (!ctx || !net) return ELRT_EINVAL;
    if (ctx->disc.p != net->desc.p || ctx->disc.n_angles != net->desc.n_angles)
        return ctx_fail(ctx, ELRT_EINVAL, "context and network discretisations differ");
    if (n < 0 || (n > 0 && (!kappa || !omega || !in2out || !in2sol)) || (!h_elem && !(h > 0)) || !(tol > 0))
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_build_local_learned: bad arguments");
    if (n_fallback) *n_fallback = 0;
    if (n == 0) return ELRT_OK;
    cudaStream_t old = net->stream;
    net->stream = ctx->stream;
    elrt_status s = elrt_net_infer(net, n, h, h_elem, kappa, omega, in2out, in2sol);
    net->stream = old;
    if (s) return ctx_fail(ctx, s, net->last_error);
    const Tab& t = ctx->tab;
    cudaStream_t sm = ctx->stream;
    float* est = estimate;
    const int64_t per_o = (int64_t)t.nin * t.nin, per_m = (int64_t)t.nm * t.nin;
    // scratch: estimate (if not given), the list, the count
    size_t need = (size_t)n * (sizeof(float) + sizeof(int64_t)) + 1024;
    void* scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, need, sm);
    if (e != cudaSuccess) return cuda_check(ctx, e, "estimate scratch");
    unsigned long long* cnt = (unsigned long long*)scratch;
    int64_t* list = (int64_t*)((unsigned char*)scratch + 256);
    if (!est) est = (float*)(list + n);
    cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), sm);
    {
        ProfScope ps(ctx, "estimate");
        for (int64_t e0 = 0; e0 < n; e0 += 65535) {
            const int64_t m = std::min<int64_t>(65535, n - e0);
            k_energy_estimate<<<(unsigned)m, 256, 0, sm>>>(t, h, h_elem ? h_elem + e0 : nullptr, kappa + e0 * t.nm,
                                                           omega + e0, in2out + e0 * per_o, in2sol + e0 * per_m,
                                                           est + e0, m);
        }
    }
    k_select<<<(unsigned)((n + 255) / 256), 256, 0, sm>>>(est, n, (float)tol, list, cnt);
    unsigned long long hc = 0;
    e = cudaMemcpyAsync(&hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, sm);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sm);
    if (e != cudaSuccess) {
        cudaFree(scratch);
        return cuda_check(ctx, e, "estimate count");
    }
    const int64_t nf = (int64_t)hc;
    if (n_fallback) *n_fallback = nf;
    if (nf > 0) {
        // classical TF32-IR solve of the flagged elements, then scatter into place
        void* fb = nullptr;
        const size_t fbytes = (size_t)nf * (t.nm + 2) * sizeof(double) + (size_t)nf * (per_o + per_m) * sizeof(float) + 1024;
        e = cudaMallocAsync(&fb, fbytes, sm);
        if (e != cudaSuccess) {
            cudaFree(scratch);
            return cuda_check(ctx, e, "fallback scratch");
        }
        double* k2 = (double*)fb;
        double* o2 = k2 + (size_t)nf * t.nm;
        double* h2 = o2 + nf;
        float* a2 = (float*)(h2 + nf);
        float* m2 = a2 + (size_t)nf * per_o;
        k_gather_inputs<<<grid_of(nf * t.nm), kT, 0, sm>>>(list, nf, t.nm, kappa, omega, h, h_elem, k2, o2, h2);
        s = local_build(ctx, nf, 1.0, h2, k2, o2, ELRT_LOCAL_TF32_IR, 1, ELRT_F32, a2, m2, nullptr, nullptr);
        if (!s) {
            k_scatter_ops<<<grid_of(nf * per_o), kT, 0, sm>>>(list, nf, per_o, a2, in2out);
            k_scatter_ops<<<grid_of(nf * per_m), kT, 0, sm>>>(list, nf, per_m, m2, in2sol);
        }
        cudaFreeAsync(fb, sm);
        if (s) {
            cudaFreeAsync(scratch, sm);
            return s;
        }
    }
    cudaFreeAsync(scratch, sm);
    return cuda_check(ctx, cudaStreamSynchronize(sm), "elrt_build_local_learned");
}

bool elrt_net_matches(const elrt_net* net, const elrt_disc* disc) {
    return net && disc && net->desc.p == disc->p && net->desc.n_angles == disc->n_angles;
}
