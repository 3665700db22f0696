// Autotuner of the launch parameters that the library chooses per discretisation (Tuning in
// elrt_internal.h): the number of elements per local-build chunk, the panel schedule of the
// tensor-core LU (pairs of panels with rank-128 trailing updates, or single panels with rank-64
// ones), and the GMRES restart length used by calls that pass restart = 0.  Each candidate is
// timed on a field the caller provides (CUDA events around the local build; the synchronising
// solve call for GMRES) and the fastest is kept in the context.  With ELRT_TUNE_CACHE set to a
// file path, results are appended there as text lines
//     elrt-tune v1 <device name> p N angular mode chunk pairs restart
// and a new context of a matching (device, p, N, angular) takes the last matching line.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <vector>

#include "elrt_internal.h"

namespace {

std::string device_key(int dev) {
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string n = prop.name;
    for (char& c : n)
        if (c == ' ') c = '_';
    return n;
}

// elapsed milliseconds of fn() on the context's stream, CUDA events on both sides
template <typename F>
elrt_status time_events(elrt_ctx* ctx, F fn, double* ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return cuda_check(ctx, e, "tune events");
    }
    cudaEventRecord(a, ctx->stream);
    elrt_status s = fn();
    cudaEventRecord(b, ctx->stream);
    if (!s) s = cuda_check(ctx, cudaEventSynchronize(b), "tune sync");
    float t = 0.f;
    if (!s) cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms = t;
    return s;
}

}  // namespace

// the last cache line matching this context's device and discretisation (no-op without a cache)
void tune_load(elrt_ctx* ctx) {
    const char* path = getenv("ELRT_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    const std::string dev = device_key(ctx->device);
    char line[512];
    while (fgets(line, sizeof line, f)) {
        char tag[32], name[256];
        int ver = 0, p = 0, N = 0, ang = 0, mode = 0, pairs = 1, restart = 12;
        long long chunk = 0;
        if (sscanf(line, "%31s v%d %255s %d %d %d %d %lld %d %d", tag, &ver, name, &p, &N, &ang, &mode, &chunk, &pairs,
                   &restart) != 10)
            continue;
        if (strcmp(tag, "elrt-tune") != 0 || ver != 1 || dev != name || p != ctx->disc.p || N != ctx->disc.n_angles ||
            ang != ctx->disc.angular)
            continue;
        if (chunk < 0 || (pairs != 0 && pairs != 1) || restart < 1 || restart > 200) continue;
        ctx->tune.local_chunk = chunk;
        ctx->tune.lu_pairs = pairs;
        ctx->tune.restart = restart;
        ctx->tune.tuned = 1;
    }
    fclose(f);
}

extern "C" elrt_status elrt_autotune(elrt_ctx* ctx, const elrt_field* fld, int32_t mode, int32_t refine_steps,
                                     double rtol, elrt_tune_report* rep) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_autotune: null context");
    if (!fld || fld->nx < 1 || fld->nz < 1 || !(fld->h > 0) || !fld->kappa || !fld->omega || !fld->inflow ||
        mode < ELRT_LOCAL_FP64 || mode > ELRT_LOCAL_TF32_IR || refine_steps < 0 || refine_steps > 8 || !(rtol > 0))
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_autotune: bad arguments");
    ctx->last_error.clear();
    const Tab& t = ctx->tab;
    const int64_t E = (int64_t)fld->nx * fld->nz;
    const size_t per_o = (size_t)t.nin * t.nin, per_m = (size_t)t.nm * t.nin;
    void* buf = nullptr;
    const size_t bytes = (size_t)E * (per_o + per_m) * sizeof(float) + (size_t)E * t.nin * sizeof(double) + 512;
    cudaError_t ce = cudaMalloc(&buf, bytes);
    if (ce != cudaSuccess) return cuda_check(ctx, ce, "elrt_autotune buffers");
    float* i2o = (float*)buf;
    float* i2m = i2o + (size_t)E * per_o;
    double* sk = (double*)(((uintptr_t)(i2m + (size_t)E * per_m) + 255) & ~(uintptr_t)255);
    const Tuning before = ctx->tune;
    elrt_tune_report r{};
    elrt_status s = ELRT_OK;

    // local stage: chunk sizes (powers of two from 512 up to the field) x panel schedules
    std::vector<int64_t> chunks{0};
    for (int64_t c = 512; c < E; c *= 2) chunks.push_back(c);
    std::vector<int> pairs{1};
    if (mode == ELRT_LOCAL_TF32_IR) pairs.push_back(0);
    double best = 1e300;
    Tuning pick = ctx->tune;
    for (int64_t c : chunks) {
        for (int pr : pairs) {
            ctx->tune.local_chunk = c;
            ctx->tune.lu_pairs = pr;
            auto run = [&] {
                return local_build(ctx, E, fld->h, nullptr, fld->kappa, fld->omega, mode, refine_steps, ELRT_F32, i2o,
                                   i2m, nullptr, nullptr);
            };
            double ms = 0.0, ms2 = 0.0;
            s = time_events(ctx, run, &ms);  // (first run: warm-up and workspace growth)
            if (!s) s = time_events(ctx, run, &ms);
            if (!s) s = time_events(ctx, run, &ms2);
            if (s) break;
            ms = 0.5 * (ms + ms2);
            if (c == 0 && pr == 1) r.local_ms_default = ms;
            ++r.n_candidates;
            if (ms < best) {
                best = ms;
                pick.local_chunk = c;
                pick.lu_pairs = pr;
            }
        }
        if (s) break;
    }
    if (!s) {
        ctx->tune.local_chunk = pick.local_chunk;
        ctx->tune.lu_pairs = pick.lu_pairs;
        r.local_ms_best = best;
        // operators of the chosen configuration, then the restart length
        s = local_build(ctx, E, fld->h, nullptr, fld->kappa, fld->omega, mode, refine_steps, ELRT_F32, i2o, i2m,
                        nullptr, nullptr);
    }
    if (!s) {
        best = 1e300;
        for (int m : {8, 12, 16, 20, 30}) {
            elrt_solve_stats gs{};
            const auto t0 = std::chrono::steady_clock::now();
            elrt_status g = global_solve(ctx, fld->nx, fld->nz, i2o, ELRT_F32, fld->inflow, rtol, 40000, m, 0, sk, &gs);
            const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (g != ELRT_OK && g != ELRT_ENOCONV) {
                s = g;
                break;
            }
            ++r.n_candidates;
            if (m == 12) r.solve_ms_default = ms;
            if (gs.converged && ms < best) {
                best = ms;
                pick.restart = m;
            }
        }
        if (!s) {
            ctx->tune.restart = pick.restart;
            r.solve_ms_best = best < 1e300 ? best : 0.0;
        }
    }
    cudaFree(buf);
    if (s) {
        ctx->tune = before;
        return s;
    }
    ctx->tune.tuned = 1;
    r.local_chunk = ctx->tune.local_chunk;
    r.lu_pairs = ctx->tune.lu_pairs;
    r.restart = ctx->tune.restart;
    if (rep) *rep = r;
    const char* path = getenv("ELRT_TUNE_CACHE");
    if (path && *path) {
        FILE* f = fopen(path, "a");
        if (f) {
            fprintf(f, "elrt-tune v1 %s %d %d %d %d %lld %d %d\n", device_key(ctx->device).c_str(), ctx->disc.p,
                    ctx->disc.n_angles, ctx->disc.angular, mode, (long long)ctx->tune.local_chunk, ctx->tune.lu_pairs,
                    ctx->tune.restart);
            fclose(f);
        }
    }
    return ELRT_OK;
}

extern "C" elrt_status elrt_get_tuning(const elrt_ctx* ctx, int64_t* local_chunk, int32_t* lu_pairs, int32_t* restart,
                                       int32_t* tuned) {
    if (!ctx) return ELRT_EINVAL;
    if (local_chunk) *local_chunk = ctx->tune.local_chunk;
    if (lu_pairs) *lu_pairs = ctx->tune.lu_pairs;
    if (restart) *restart = ctx->tune.restart;
    if (tuned) *tuned = ctx->tune.tuned;
    return ELRT_OK;
}

extern "C" elrt_status elrt_set_tuning(elrt_ctx* ctx, int64_t local_chunk, int32_t lu_pairs, int32_t restart) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_set_tuning: null context");
    if (local_chunk < 0 || (lu_pairs != 0 && lu_pairs != 1) || restart < 1 || restart > 200)
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_set_tuning: chunk >= 0, pairs 0/1, restart 1..200");
    ctx->tune.local_chunk = local_chunk;
    ctx->tune.lu_pairs = lu_pairs;
    ctx->tune.restart = restart;
    return ELRT_OK;
}
