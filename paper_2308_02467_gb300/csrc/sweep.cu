// Sweep preconditioner of the skeleton GMRES: z = M u, upwind block Gauss-Seidel sweeps of the
// skeleton system (I - A_int) z = u (eq. hdg_global_mat; Sec. 2.3 names transport sweeps among
// the solvers of radiative transfer) from z = 0, one sweep from each mesh corner in turn
// (bottom-left, bottom-right, top-right, top-left: each sweep can start while the one before is
// half done).  A sweep visits the elements in wavefront order from its corner and replaces each
// element's outflow by z_K = u_K + A_i2o^K z_in(K), the inflow gathered from the current z: the
// neighbours one wavefront closer to the corner hold this sweep's values, the others the
// previous sweep's (zero in the first).
//
// One persistent cooperative launch (one CTA of 512 threads per SM) runs all four sweeps.  The
// work items (sweep, element, half of its rows) are ordered by the step at which their
// dependencies allow them to start (1 + the latest start among them; a topological order, built on
// the host), so the four sweeps overlap wherever the dependencies allow, and are dealt to the CTAs
// round robin, so every CTA takes its items in that order.  (Dealing them from a counter to
// whichever CTA had a free stage was slower: a CTA then held the next items of the order before
// they were ready while ready ones waited behind them.)  Instead of a grid barrier per wavefront, every outflow
// value is stored with the sweep that wrote it, one 64-bit word (value, sweep + 1; single-copy
// atomic), and an item polls exactly the words it needs (bounded): the faces of its upwind
// neighbours until this sweep wrote them, those of its downwind neighbours until the previous
// sweep did (so that they are final and the neighbour has read this element's old ones), and its
// own rows until the previous sweep did (they are rewritten here).  Flag and data arrive in one
// round trip.  The last sweep also writes the plain FP32 result.  Everything an item waits for
// comes earlier in the global order and every CTA is resident, so the dataflow cannot deadlock,
// and a sweep starts at its corner as soon as the previous sweeps have passed there.  An item's
// operator block (n_in x n_in, contiguous) is copied to shared memory by the bulk-copy engine in
// a two-stage ring (one stage when two do not fit; read from global memory when one does not),
// so the copy of a CTA's next element overlaps its current one.
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

#include "elrt_internal.h"
#include "tc_gemm.cuh"

namespace {

constexpr int kSwThreads = 512;               // 16 warps
constexpr int kSwWarps = kSwThreads / 32;
constexpr int kSwMaxIn = 4 * ELRT_MAX_N1 * (ELRT_MAX_ANG / 2);
constexpr int kSwChunk = 32768;               // bytes per bulk copy
constexpr int kSwSmemMax = 220 * 1024;        // dynamic shared memory the ring may use
constexpr long long kSwSpin = 1000000000LL;   // ~0.5 s of clock64 per wait

// Sixteen per-lane partial sums (v[k]: row k) reduced across the warp in five butterfly rounds of
// independent shuffles (16 in all): afterwards lanes 2r and 2r + 1 hold the sum of row r.
// Eight per-lane partial sums (v[k]: row k) reduced across the warp in five butterfly rounds (9
// shuffles): afterwards the lanes 4r .. 4r + 3 hold the sum of row r.
__device__ __forceinline__ float warp_sum8(float (&v)[8], int lane) {
#pragma unroll
    for (int h = 4, m = 16; h >= 1; h >>= 1, m >>= 1) {
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = up ? v[i] : v[i + h];
            const float keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
    }
    float t = v[0] + __shfl_xor_sync(0xffffffffu, v[0], 2);
    return t + __shfl_xor_sync(0xffffffffu, t, 1);
}

__device__ __forceinline__ float warp_sum16(float (&v)[16], int lane) {
#pragma unroll
    for (int h = 8, m = 16; h >= 1; h >>= 1, m >>= 1) {
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = up ? v[i] : v[i + h];
            const float keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// wavefront index of element (jx, jz) in sweep c (0 from the bottom-left corner, 1 bottom-right,
// 2 top-right, 3 top-left)
__device__ __forceinline__ int wave_of(int c, int jx, int jz, int nx, int nz) {
    const int dx = (c == 0 || c == 3) ? jx : nx - 1 - jx;
    const int dz = (c == 0 || c == 1) ? jz : nz - 1 - jz;
    return dx + dz;
}

// two consecutive operator entries as floats (generic address: shared or global)
__device__ __forceinline__ float2 ld_pair(const __half* A, int i) {
    return __half22float2(*reinterpret_cast<const __half2*>(A + i));
}
__device__ __forceinline__ float2 ld_pair(const float* A, int i) { return *reinterpret_cast<const float2*>(A + i); }

// an outflow value and the number of sweeps that have written it
struct __align__(8) VerVal {
    float v;
    int ver;
};

// one aligned 64-bit access (single-copy atomic): the value in the low half, the version above
__device__ __forceinline__ VerVal ld_verval(const VerVal* p) {
    unsigned long long b;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(b) : "l"(p) : "memory");
    return VerVal{__uint_as_float((unsigned)b), (int)(b >> 32)};
}
__device__ __forceinline__ void st_verval(VerVal* p, float v, int ver) {
    const unsigned long long b = (unsigned long long)__float_as_uint(v) | ((unsigned long long)(unsigned)ver << 32);
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(b) : "memory");
}

struct SweepArgs {
    int nx, nz, nin, nface;
    int64_t E;
    int stages;            // operator blocks staged in shared memory: 2, 1 or 0 (read from global)
    int parts, prows;      // an element's rows in `parts` work items of prows rows (the last may be shorter)
    const int* order;      // [4 E parts]: the work items (c E + e) parts + part in their global order
    const float* u;        // [E][nin]
    float* z;              // [E][nin] result (written by the last sweep)
    VerVal* zw;            // [E][nin] versioned outflow, zero on entry
    int* err;              // bit 0: a wait timed out
    const int* done;       // nothing to do when *done != 0 (GMRES converged; may be NULL)
    const int* nsteps;     // nothing to do when *nsteps == 0 (no Arnoldi step to apply; may be NULL)
    int* abort;            // set on a timeout: every CTA stops
};

// NP: column pairs per lane and row (nin <= 64 NP)
template <typename AT, int NP>
__global__ void __launch_bounds__(kSwThreads, 1) k_sweep(SweepArgs a, const AT* __restrict__ A) {
    if ((a.done && *a.done) || (a.nsteps && *a.nsteps == 0)) return;
    extern __shared__ __align__(128) unsigned char sw_smem[];
    const int nin = a.nin, nf = a.nface, npair = nin / 2;
    const int blk_bytes = a.prows * nin * (int)sizeof(AT);  // a stage: one item's rows
    const int NS = a.stages;
    AT* stage0 = reinterpret_cast<AT*>(sw_smem);
    float* xin = reinterpret_cast<float*>(sw_smem + (size_t)NS * blk_bytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(xin + ((nin + 3) & ~3));  // [2]
    __shared__ int stop, stop_copy;  // a dependency wait / the copy wait gave up
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int total = (int)(4 * a.E * a.parts);
    const int rows_w = (a.prows + kSwWarps - 1) / kSwWarps;  // rows of a warp (at most 44)
    if (threadIdx.x == 0) {
        for (int i = 0; i < NS; ++i) tc::mbar_init(&bar[i], 1);
        tc::fence_barrier_init();
        stop = stop_copy = 0;
    }
    __syncthreads();
    auto rows_of = [&](int part) { return min(a.prows, nin - part * a.prows); };
    auto issue = [&](int64_t it, int st) {  // the operator rows of item it into stage st
        const int code = a.order[it], part = code % a.parts;
        const int e = (int)((code / a.parts) % a.E);
        const int bytes = rows_of(part) * nin * (int)sizeof(AT);
        const unsigned char* src =
            reinterpret_cast<const unsigned char*>(A + (int64_t)e * nin * nin + (int64_t)part * a.prows * nin);
        unsigned char* dst = reinterpret_cast<unsigned char*>(stage0) + (size_t)st * blk_bytes;
        tc::mbar_expect_tx(&bar[st], (uint32_t)bytes);
        for (int off = 0; off < bytes; off += kSwChunk)
            tc::bulk_load(dst + off, src + off, (uint32_t)min(kSwChunk, bytes - off), &bar[st]);
    };
    if (threadIdx.x == 0)
        for (int s = 0; s < NS; ++s) {
            const int it = blockIdx.x + s * (int)gridDim.x;
            if (it < total) issue(it, s);
        }
    int k = 0;
    int issued = (int)std::min<int64_t>((int64_t)NS, (total - blockIdx.x + gridDim.x - 1) / gridDim.x);
    bool alive = true;
    for (int it = blockIdx.x; it < total && alive; it += gridDim.x, ++k) {
        const int code = a.order[it], part = code % a.parts;
        const int c = code / (a.parts * (int)a.E);
        const int e = (int)((code / a.parts) % a.E);
        const int ix = e % a.nx, iz = e / a.nx;
        const int st = NS ? k % NS : 0;
        const int prow0 = part * a.prows, nrows = rows_of(part);  // this item's rows of the element
        // this lane's right-hand-side values (it writes row r0 + b + lane / 4 of each batch of 8),
        // loaded now so that their latency passes while the item waits for its dependencies
        const int r0 = warp * rows_w;
        float uv[6];
#pragma unroll
        for (int bb = 0; bb < 6; ++bb) {
            const int rl = r0 + 8 * bb + (lane >> 2);
            uv[bb] = (8 * bb + (lane >> 2) < rows_w && rl < nrows) ? __ldg(a.u + (int64_t)e * nin + prow0 + rl) : 0.f;
        }
        // the element's operator block has landed (bounded wait)
        if (NS && threadIdx.x == 0) {
            const long long t0 = clock64();
            while (!tc::mbar_try_wait(&bar[st], (k / NS) & 1))
                if (clock64() - t0 > kSwSpin) {
                    atomicOr(a.err, 2);
                    *(volatile int*)a.abort = 1;
                    stop_copy = 1;
                    break;
                }
        }
        // inflow (threads below nin): each neighbour face value once the sweep it must come from has
        // written it; own rows (the next nin threads): once the previous sweep has written them
        const int we = wave_of(c, ix, iz, a.nx, a.nz);
        bool ok = true;
        for (int i = threadIdx.x; i < nin + nrows && ok; i += kSwThreads) {
            const VerVal* w = nullptr;
            int need = c;
            if (i < nin) {
                const int F = i / nf, off = i - F * nf;
                const int jx = ix + (F == 1) - (F == 3), jz = iz + (F == 2) - (F == 0);
                if (jx < 0 || jx >= a.nx || jz < 0 || jz >= a.nz) {
                    xin[i] = 0.f;
                    continue;
                }
                w = a.zw + (int64_t)(jx + a.nx * jz) * nin + ((F + 2) & 3) * nf + off;
                if (wave_of(c, jx, jz, a.nx, a.nz) < we) need = c + 1;
            } else {
                w = a.zw + (int64_t)e * nin + prow0 + (i - nin);
            }
            VerVal x = ld_verval(w);
            if (x.ver < need) {
                const long long t0 = clock64();
                do {
                    if (*(volatile int*)a.abort || clock64() - t0 > kSwSpin) {
                        ok = false;
                        break;
                    }
                    x = ld_verval(w);
                } while (x.ver < need);
            }
            if (i < nin) xin[i] = x.v;
        }
        if (!ok) {
            atomicOr(a.err, 1);
            *(volatile int*)a.abort = 1;
            stop = 1;
        }
        __syncthreads();
        if (stop || stop_copy) {
            alive = false;
            break;
        }
        const AT* Ab = NS ? stage0 + (size_t)st * a.prows * nin : A + (int64_t)e * nin * nin + (int64_t)prow0 * nin;
        // this warp's rows in batches of 16: per-lane partial sums over the lane's column pairs,
        // then one transposed reduction per batch
        float2 xv[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const int pc = lane + 32 * q;
            xv[q] = pc < npair ? *reinterpret_cast<const float2*>(xin + 2 * pc) : make_float2(0.f, 0.f);
        }
#pragma unroll 1
        for (int b = 0; b < rows_w; b += 8) {
            float v[8];
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                v[kk] = 0.f;
                const int rl = r0 + b + kk;  // row within the item
                if (b + kk < rows_w && rl < nrows) {
#pragma unroll
                    for (int q = 0; q < NP; ++q) {
                        const int pc = lane + 32 * q;
                        if (pc < npair) {
                            const float2 av = ld_pair(Ab, rl * nin + 2 * pc);
                            v[kk] = fmaf(av.x, xv[q].x, v[kk]);
                            v[kk] = fmaf(av.y, xv[q].y, v[kk]);
                        }
                    }
                }
            }
            const float sum = warp_sum8(v, lane);
            const int rl = r0 + b + (lane >> 2);
            if ((lane & 3) == 0 && b + (lane >> 2) < rows_w && rl < nrows) {
                const int64_t i = (int64_t)e * nin + prow0 + rl;
                float uu = uv[0];
#pragma unroll
                for (int bb = 1; bb < 6; ++bb)
                    if (b == 8 * bb) uu = uv[bb];
                const float val = uu + sum;
                st_verval(a.zw + i, val, c + 1);
                if (c == 3) a.z[i] = val;
            }
        }
        __syncthreads();  // the stage is free
        if (threadIdx.x == 0) {
            const int nxt = it + NS * (int)gridDim.x;
            if (NS && nxt < total) {
                issue(nxt, st);
                ++issued;
            }
        }
    }
    // let the copies this CTA issued land before it exits (bounded)
    if (NS && threadIdx.x == 0) {
        for (int q = max(0, issued - NS); q < issued; ++q) {
            const long long t0 = clock64();
            while (!tc::mbar_try_wait(&bar[q % NS], (q / NS) & 1) && clock64() - t0 < kSwSpin) {
            }
        }
    }
}

template <typename AT, int NP>
cudaError_t launch_sweep(cudaLaunchConfig_t cfg, const SweepArgs& a, const void* A) {
    const size_t smem = (size_t)a.stages * a.prows * a.nin * sizeof(AT) + (((a.nin + 3) & ~3) + 32) * sizeof(float);
    static size_t attr = 0;
    if (smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep<AT, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    cfg.dynamicSmemBytes = smem;
    return cudaLaunchKernelEx(&cfg, k_sweep<AT, NP>, a, (const AT*)A);
}

}  // namespace

// Work items per element: its rows in two halves once an element has 128 outflow DOFs or more,
// so that the latency of an element's step on the chain is that of half its rows.
int sweep_parts(const Tab& t) { return t.nin >= 128 ? 2 : 1; }

// Global order of the work items (c E + e) parts + part (sweep c from the bottom-left,
// bottom-right, top-right, top-left corner): by the step t at which an element's sweep can start,
// t = 1 + the largest t among the elements' sweeps it waits for (its upwind neighbours in sweep c,
// its downwind neighbours and itself in sweep c - 1), then by sweep, element and part.  Every item
// comes after everything it waits for.
void sweep_orders(int nx, int nz, int parts, int* out) {
    const int E = nx * nz;
    auto wave = [&](int c, int ix, int iz) {
        const int dx = (c == 0 || c == 3) ? ix : nx - 1 - ix;
        const int dz = (c == 0 || c == 1) ? iz : nz - 1 - iz;
        return dx + dz;
    };
    std::vector<int> t((size_t)4 * E, 0), idx(E), key(E);
    for (int c = 0; c < 4; ++c) {
        // this sweep's elements in wavefront order, so that upwind neighbours are done first
        for (int e = 0; e < E; ++e) {
            key[e] = wave(c, e % nx, e / nx);
            idx[e] = e;
        }
        std::stable_sort(idx.begin(), idx.end(), [&](int p, int q) { return key[p] < key[q]; });
        for (int e : idx) {
            const int ix = e % nx, iz = e / nx, we = key[e];
            int start = c > 0 ? t[(size_t)(c - 1) * E + e] : 0;
            for (int F = 0; F < 4; ++F) {
                const int jx = ix + (F == 1) - (F == 3), jz = iz + (F == 2) - (F == 0);
                if (jx < 0 || jx >= nx || jz < 0 || jz >= nz) continue;
                const int nb = jx + nx * jz;
                if (wave(c, jx, jz) < we) start = std::max(start, t[(size_t)c * E + nb]);
                else if (c > 0) start = std::max(start, t[(size_t)(c - 1) * E + nb]);
            }
            t[(size_t)c * E + e] = start + 1;
        }
    }
    std::vector<int> items((size_t)4 * E);
    for (int i = 0; i < 4 * E; ++i) items[i] = i;
    std::stable_sort(items.begin(), items.end(), [&](int p, int q) { return t[p] < t[q]; });
    for (size_t i = 0; i < items.size(); ++i)
        for (int part = 0; part < parts; ++part) out[i * parts + part] = items[i] * parts + part;
}

// z = M u on the stream, with the operator A (FP16 or FP32, [E][nin][nin], 16-byte aligned);
// order: device [4 E parts] from sweep_orders with parts = sweep_parts(tab); zw: device scratch of 8 E n_in bytes; flags: device ints (err,
// abort), cleared here (err stays set after a timed-out wait); z is zeroed first, so a skipped
// application leaves 0.
elrt_status sweep_apply(elrt_ctx* ctx, int nx, int nz, const void* A, int a_bytes, const float* u, float* z,
                        const int* order, void* zw, int* flags, const int* done, const int* nsteps) {
    const Tab& t = ctx->tab;
    const int64_t E = (int64_t)nx * nz;
    if (t.nin % 8 != 0 || t.nin > kSwMaxIn || E > (1LL << 27) || (a_bytes != 2 && a_bytes != 4) ||
        ((uintptr_t)A & 15) != 0)
        return ctx_fail(ctx, ELRT_EINVAL, "sweep preconditioner: unsupported element size or alignment");
    const int nsm = ctx->sms;
    const int parts = sweep_parts(t), prows = (t.nin + parts - 1) / parts;
    const size_t blk = (size_t)prows * t.nin * a_bytes, extra = (size_t)(t.nin + 36) * sizeof(float);
    const int stages = 2 * blk + extra <= (size_t)kSwSmemMax ? 2 : (blk + extra <= (size_t)kSwSmemMax ? 1 : 0);
    SweepArgs a{nx, nz, t.nin, t.nface, E, stages, parts, prows, order, u, z, (VerVal*)zw, flags, done, nsteps, flags + 1};
    const double nop = (double)E * t.nin * t.nin;
    ProfScope ps(ctx, "sweep", 1, 4.0 * (nop * a_bytes + 12.0 * E * t.nin), 4.0 * 2.0 * nop);
    elrt_status s = cuda_check(ctx, cudaMemsetAsync(z, 0, (size_t)E * t.nin * sizeof(float), ctx->stream), "sweep z");
    if (!s) s = cuda_check(ctx, cudaMemsetAsync(zw, 0, (size_t)E * t.nin * sizeof(VerVal), ctx->stream), "sweep words");
    if (!s) s = cuda_check(ctx, cudaMemsetAsync(flags, 0, 2 * sizeof(int), ctx->stream), "sweep flags");
    if (s) return s;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(4 * E * parts, nsm)));  // one CTA per SM
    cfg.blockDim = dim3(kSwThreads);
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeCooperative;
    attr.val.cooperative = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    const int npair = t.nin / 2;
    cudaError_t e;
    if (npair <= 32 * 4)
        e = a_bytes == 2 ? launch_sweep<__half, 4>(cfg, a, A) : launch_sweep<float, 4>(cfg, a, A);
    else if (npair <= 32 * 8)
        e = a_bytes == 2 ? launch_sweep<__half, 8>(cfg, a, A) : launch_sweep<float, 8>(cfg, a, A);
    else
        e = a_bytes == 2 ? launch_sweep<__half, 11>(cfg, a, A) : launch_sweep<float, 11>(cfg, a, A);
    return cuda_check(ctx, e, "sweep launch");
}

extern "C" elrt_status elrt_apply_precond(elrt_ctx* ctx, int32_t nx, int32_t nz, const void* in2out, int32_t dtype,
                                          const float* r, float* z) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_apply_precond: null context");
    if (nx < 1 || nz < 1 || (int64_t)nx * nz > (1LL << 30) || !in2out || !r || !z || r == z || dtype != ELRT_F32)
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_apply_precond: bad arguments (FP32 in2out, distinct r and z)");
    ctx->last_error.clear();
    const int64_t E = (int64_t)nx * nz;
    // scratch: the versioned outflow [E][n_in], the item order [4 E parts] and two flags
    const int parts = sweep_parts(ctx->tab);
    const size_t wbytes = (size_t)E * ctx->tab.nin * sizeof(VerVal);
    const size_t need = wbytes + (size_t)4 * E * parts * sizeof(int) + 64;
    elrt_status s = ensure_ws(ctx, &ctx->vec, &ctx->vec_bytes, need);
    if (s) return s;
    void* zw = ctx->vec;
    int* order = (int*)((unsigned char*)ctx->vec + wbytes);
    int* flags = order + 4 * E * parts;
    std::vector<int> ord((size_t)4 * E * parts);
    sweep_orders(nx, nz, parts, ord.data());
    s = cuda_check(ctx, cudaMemcpyAsync(order, ord.data(), ord.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream),
                   "sweep orders");
    if (!s) s = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "sweep orders");
    if (!s) s = sweep_apply(ctx, nx, nz, in2out, 4, r, z, order, zw, flags, nullptr, nullptr);
    if (s) return s;
    int h = 0;
    s = cuda_check(ctx, cudaMemcpyAsync(&h, flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "sweep flag");
    if (!s) s = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "sweep");
    if (s) return s;
    if (h) return ctx_fail(ctx, ELRT_ETIMEOUT, "a wait of the sweep preconditioner timed out");
    return ELRT_OK;
}
