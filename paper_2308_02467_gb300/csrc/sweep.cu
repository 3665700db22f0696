// Sweep preconditioner of the skeleton GMRES: z = M u, upwind block Gauss-Seidel sweeps of the
// skeleton system (I - A_int) z = u (eq. hdg_global_mat; Sec. 2.3 names transport sweeps among
// the solvers of radiative transfer) from z = 0, one sweep from each mesh corner in turn
// (bottom-left, bottom-right, top-right, top-left: each sweep can start while the one before is
// half done).  A sweep visits the elements in wavefront order from its corner and recomputes the
// outflow of each element's two downwind faces (those pointing away from the corner: right and top
// from the bottom-left corner, left and top from the bottom-right, left and bottom from the
// top-right, right and bottom from the top-left) as z_F = u_F + A_i2o^K[F rows] z_in(K), the
// inflow gathered from the current z: the neighbours one wavefront closer to the corner hold this
// sweep's values, the others the latest earlier sweep's that wrote the face (zero before any).
// These are the values the sweep's later elements read; each face is recomputed by two of the four
// sweeps, so an application reads every operator row twice instead of four times.  In matrix form
// each sweep solves exactly for its rows given the others (block lower triangular in its
// wavefront order): a multiplicative Schwarz iteration over four overlapping blocks.
//
// One persistent cooperative launch (one CTA of 512 threads per SM) runs all four sweeps.  The
// work items (sweep, element) are ordered by the step at which their dependencies allow them to
// start (1 + the latest start among them; a topological order, built on the host), so the four
// sweeps overlap wherever the dependencies allow, and are dealt to the CTAs round robin, so every
// CTA takes its items in that order.  (Dealing them from a counter to whichever CTA had a free
// stage was slower: a CTA then held the next items of the order before they were ready while ready
// ones waited behind them.)  Instead of a grid barrier per wavefront, every sweep writes its values
// to a slot of its own, one 64-bit word per value (value, written flag; single-copy atomic),
// zeroed at the start of an application, so every word is written once and no value can be
// overwritten before it is read; an item polls exactly the words it needs (bounded).  Flag and
// data arrive in one round trip.  The last sweep that writes a face also writes the plain FP32
// result.  Everything an item waits for comes earlier in the global order and every CTA is
// resident, so the dataflow cannot deadlock.  An item's operator rows (two blocks of n_face rows,
// contiguous each) are copied to shared memory by the bulk-copy engine in a two-stage ring (one
// stage when two do not fit; read from global memory when one does not), so the copy of a CTA's
// next item overlaps its current one.  (The earlier form recomputed all of an element's rows in
// every sweep, as two items per element and sweep; with half the items and half the operator
// reads per application it was the slower one, its items' fixed costs — the polls of the inflow,
// the copies, the barriers — dominating.)
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
    const int* order;      // [4 E]: the work items c E + e in their global order
    const float* u;        // [E][nin]
    float* z;              // [E][nin] result (each face written by the last sweep that recomputes it)
    VerVal* zw;            // [4][E][nin / 2]: sweep c's values of each element's downwind faces, zero on entry
    int* err;              // bit 0: a wait timed out
    const int* done;       // nothing to do when *done != 0 (GMRES converged; may be NULL)
    const int* nsteps;     // nothing to do when *nsteps == 0 (no Arnoldi step to apply; may be NULL)
    int* abort;            // set on a timeout: every CTA stops
};

// Faces 0 bottom, 1 right, 2 top, 3 left.  kDown[c]: the downwind faces sweep c recomputes, in the
// order of its slot; kPrev[c][H]: the latest sweep before c that recomputes face H (-1: none, the
// value is still zero); kLast[H]: the last sweep that recomputes face H.
__host__ __device__ constexpr int sw_down(int c, int k) {
    return k == 0 ? (c == 0 || c == 3 ? 1 : 3) : (c == 0 || c == 1 ? 2 : 0);
}
__host__ __device__ constexpr int sw_prev(int c, int H) {
    for (int q = c - 1; q >= 0; --q)
        if (sw_down(q, 0) == H || sw_down(q, 1) == H) return q;
    return -1;
}
__host__ __device__ constexpr int sw_last(int H) { return sw_prev(4, H); }
static_assert(sw_down(0, 0) == 1 && sw_down(0, 1) == 2 && sw_down(1, 0) == 3 && sw_down(1, 1) == 2 &&
                  sw_down(2, 0) == 3 && sw_down(2, 1) == 0 && sw_down(3, 0) == 1 && sw_down(3, 1) == 0,
              "downwind faces: BL right/top, BR left/top, TR left/bottom, TL right/bottom");
static_assert(sw_last(0) == 3 && sw_last(1) == 3 && sw_last(2) == 1 && sw_last(3) == 2, "last writers");

// NP: column pairs per lane and row (nin <= 64 NP)
template <typename AT, int NP>
__global__ void __launch_bounds__(kSwThreads, 1) k_sweep(SweepArgs a, const AT* __restrict__ A) {
    if ((a.done && *a.done) || (a.nsteps && *a.nsteps == 0)) return;
    extern __shared__ __align__(128) unsigned char sw_smem[];
    const int nin = a.nin, nf = a.nface, npair = nin / 2, nrows = 2 * nf;  // an item: two faces' rows
    const int blk_bytes = nrows * nin * (int)sizeof(AT);                      // a stage: one item's rows
    const int NS = a.stages;
    AT* stage0 = reinterpret_cast<AT*>(sw_smem);
    float* xin = reinterpret_cast<float*>(sw_smem + (size_t)NS * blk_bytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(xin + ((nin + 3) & ~3));  // [2]
    __shared__ int stop, stop_copy;  // a dependency wait / the copy wait gave up
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int total = (int)(4 * a.E);
    const int rows_w = (nrows + kSwWarps - 1) / kSwWarps;  // rows of a warp (at most 44)
    if (threadIdx.x == 0) {
        for (int i = 0; i < NS; ++i) tc::mbar_init(&bar[i], 1);
        tc::fence_barrier_init();
        stop = stop_copy = 0;
    }
    __syncthreads();
    // row rl of item (c, e) is row elem_row(c, rl) of the element (face, offset)
    auto elem_row = [&](int c, int rl) { return rl < nf ? sw_down(c, 0) * nf + rl : sw_down(c, 1) * nf + rl - nf; };
    auto issue = [&](int64_t it, int st) {  // the operator rows of item it into stage st
        const int code = a.order[it];
        const int c = code / (int)a.E, e = code - c * (int)a.E;
        const int bytes = nf * nin * (int)sizeof(AT);
        unsigned char* dst = reinterpret_cast<unsigned char*>(stage0) + (size_t)st * blk_bytes;
        tc::mbar_expect_tx(&bar[st], (uint32_t)(2 * bytes));
        for (int h = 0; h < 2; ++h) {
            const unsigned char* src =
                reinterpret_cast<const unsigned char*>(A + (int64_t)e * nin * nin + (int64_t)sw_down(c, h) * nf * nin);
            for (int off = 0; off < bytes; off += kSwChunk)
                tc::bulk_load(dst + h * bytes + off, src + off, (uint32_t)min(kSwChunk, bytes - off), &bar[st]);
        }
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
        const int code = a.order[it];
        const int c = code / (int)a.E, e = code - c * (int)a.E;
        const int ix = e % a.nx, iz = e / a.nx;
        const int st = NS ? k % NS : 0;
        // this lane's right-hand-side values (it writes row r0 + b + lane / 4 of each batch of 8),
        // loaded now so that their latency passes while the item waits for its dependencies
        const int r0 = warp * rows_w;
        float uv[6];
#pragma unroll
        for (int bb = 0; bb < 6; ++bb) {
            const int rl = r0 + 8 * bb + (lane >> 2);
            uv[bb] = (8 * bb + (lane >> 2) < rows_w && rl < nrows) ? __ldg(a.u + (int64_t)e * nin + elem_row(c, rl)) : 0.f;
        }
        // the item's operator rows have landed (bounded wait)
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
        // inflow: each neighbour's face towards this element, from this sweep's slot when the
        // neighbour is upwind (its face towards us is then one of this sweep's downwind faces),
        // else from the slot of the latest earlier sweep that recomputed that face (none: zero)
        const int we = wave_of(c, ix, iz, a.nx, a.nz);
        bool ok = true;
        for (int i = threadIdx.x; i < nin && ok; i += kSwThreads) {
            const int G = i / nf, off = i - G * nf, H = (G + 2) & 3;
            const int jx = ix + (G == 1) - (G == 3), jz = iz + (G == 2) - (G == 0);
            float xv_in = 0.f;
            const int slot = (jx < 0 || jx >= a.nx || jz < 0 || jz >= a.nz) ? -1
                             : (wave_of(c, jx, jz, a.nx, a.nz) < we ? c : sw_prev(c, H));
            if (slot >= 0) {
                const VerVal* w = a.zw + ((int64_t)slot * a.E + (jx + a.nx * jz)) * npair +
                                  (sw_down(slot, 0) == H ? off : nf + off);
                VerVal x = ld_verval(w);
                if (x.ver == 0) {
                    const long long t0 = clock64();
                    do {
                        if (*(volatile int*)a.abort || clock64() - t0 > kSwSpin) {
                            ok = false;
                            break;
                        }
                        x = ld_verval(w);
                    } while (x.ver == 0);
                }
                xv_in = x.v;
            }
            xin[i] = xv_in;
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
        const AT* Ag = A + (int64_t)e * nin * nin;  // no stage: the rows straight from the element's block
        const AT* Ab = NS ? stage0 + (size_t)st * nrows * nin : nullptr;
        // this warp's rows in batches of 8: per-lane partial sums over the lane's column pairs,
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
                    const AT* Ar = NS ? Ab + (size_t)rl * nin : Ag + (size_t)elem_row(c, rl) * nin;
#pragma unroll
                    for (int q = 0; q < NP; ++q) {
                        const int pc = lane + 32 * q;
                        if (pc < npair) {
                            const float2 av = ld_pair(Ar, 2 * pc);
                            v[kk] = fmaf(av.x, xv[q].x, v[kk]);
                            v[kk] = fmaf(av.y, xv[q].y, v[kk]);
                        }
                    }
                }
            }
            const float sum = warp_sum8(v, lane);
            const int rl = r0 + b + (lane >> 2);
            if ((lane & 3) == 0 && b + (lane >> 2) < rows_w && rl < nrows) {
                float uu = uv[0];
#pragma unroll
                for (int bb = 1; bb < 6; ++bb)
                    if (b == 8 * bb) uu = uv[bb];
                const float val = uu + sum;
                st_verval(a.zw + ((int64_t)c * a.E + e) * npair + rl, val, 1);
                const int er = elem_row(c, rl);
                if (sw_last(er / nf) == c) a.z[(int64_t)e * nin + er] = val;
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
    const size_t smem = (size_t)a.stages * a.nface * 2 * a.nin * sizeof(AT) + (((a.nin + 3) & ~3) + 32) * sizeof(float);
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

// Global order of the work items c E + e (sweep c from the bottom-left, bottom-right, top-right,
// top-left corner): by the step t at which an item can start, t = 1 + the largest t among the
// items whose values it reads (its upwind neighbours in sweep c; for each downwind neighbour, the
// latest earlier sweep that recomputed the neighbour's face towards it), then by sweep and element.
// Every item comes after everything it waits for.
void sweep_orders(int nx, int nz, int* out) {
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
            int start = 0;
            for (int G = 0; G < 4; ++G) {
                const int jx = ix + (G == 1) - (G == 3), jz = iz + (G == 2) - (G == 0);
                if (jx < 0 || jx >= nx || jz < 0 || jz >= nz) continue;
                const int nb = jx + nx * jz;
                const int slot = wave(c, jx, jz) < we ? c : sw_prev(c, (G + 2) & 3);
                if (slot >= 0) start = std::max(start, t[(size_t)slot * E + nb]);
            }
            t[(size_t)c * E + e] = start + 1;
        }
    }
    for (int i = 0; i < 4 * E; ++i) out[i] = i;
    std::stable_sort(out, out + 4 * (size_t)E, [&](int p, int q) { return t[p] < t[q]; });
}

// device scratch of one application's outflow words: four slots of E x n_in / 2 64-bit words
size_t sweep_words_bytes(const Tab& t, int64_t E) { return (size_t)4 * E * (t.nin / 2) * sizeof(VerVal); }

// z = M u on the stream, with the operator A (FP16 or FP32, [E][nin][nin], 16-byte aligned);
// order: device [4 E] from sweep_orders; zw: device scratch of sweep_words_bytes; flags: device ints
// (err, abort), cleared here (err stays set after a timed-out wait); z is zeroed first, so a skipped
// application leaves 0.
elrt_status sweep_apply(elrt_ctx* ctx, int nx, int nz, const void* A, int a_bytes, const float* u, float* z,
                        const int* order, void* zw, int* flags, const int* done, const int* nsteps) {
    const Tab& t = ctx->tab;
    const int64_t E = (int64_t)nx * nz;
    if (t.nin % 8 != 0 || t.nin > kSwMaxIn || E > (1LL << 27) || (a_bytes != 2 && a_bytes != 4) ||
        ((uintptr_t)A & 15) != 0)
        return ctx_fail(ctx, ELRT_EINVAL, "sweep preconditioner: unsupported element size or alignment");
    const int nsm = ctx->sms;
    const size_t blk = (size_t)2 * t.nface * t.nin * a_bytes, extra = (size_t)(t.nin + 36) * sizeof(float);
    const int stages = 2 * blk + extra <= (size_t)kSwSmemMax ? 2 : (blk + extra <= (size_t)kSwSmemMax ? 1 : 0);
    SweepArgs a{nx, nz, t.nin, t.nface, E, stages, order, u, z, (VerVal*)zw, flags, done, nsteps, flags + 1};
    // every operator row is read twice (two of the four sweeps recompute each face); per item the
    // inflow (4 B), the right-hand side, the slot word and the result
    const double nop = (double)E * t.nin * t.nin;
    ProfScope ps(ctx, "sweep", 1, 2.0 * nop * a_bytes + 4.0 * E * (t.nin * 4.0 + (t.nin / 2) * 16.0),
                 2.0 * 2.0 * nop);
    elrt_status s = cuda_check(ctx, cudaMemsetAsync(z, 0, (size_t)E * t.nin * sizeof(float), ctx->stream), "sweep z");
    if (!s) s = cuda_check(ctx, cudaMemsetAsync(zw, 0, sweep_words_bytes(t, E), ctx->stream), "sweep words");
    if (!s) s = cuda_check(ctx, cudaMemsetAsync(flags, 0, 2 * sizeof(int), ctx->stream), "sweep flags");
    if (s) return s;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(4 * E, nsm)));  // one CTA per SM
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
    // scratch: the outflow words of the four sweeps, the item order [4 E] and two flags
    const size_t wbytes = sweep_words_bytes(ctx->tab, E);
    const size_t need = wbytes + (size_t)4 * E * sizeof(int) + 64;
    elrt_status s = ensure_ws(ctx, &ctx->vec, &ctx->vec_bytes, need);
    if (s) return s;
    void* zw = ctx->vec;
    int* order = (int*)((unsigned char*)ctx->vec + wbytes);
    int* flags = order + 4 * E;
    std::vector<int> ord((size_t)4 * E);
    sweep_orders(nx, nz, ord.data());
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
