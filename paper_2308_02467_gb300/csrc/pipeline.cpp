// Whole-pipeline entry points (Algorithm 1): one field, and many uneven fields in waves.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <vector>

#include "elrt_internal.h"

namespace {

double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

bool opts_ok(const elrt_solve_opts* o) {
    return o && o->mode >= ELRT_LOCAL_FP64 && o->mode <= ELRT_LOCAL_TF32_IR && o->refine_steps >= 0 &&
           o->refine_steps <= 8 && o->rtol > 0 && o->max_iter >= 1 && o->restart >= 0 && o->restart <= 200 &&
           (!o->net || o->learned_tol > 0);
}

bool field_ok(const elrt_field* f) {
    return f && f->nx >= 1 && f->nz >= 1 && f->h > 0 && f->kappa && f->omega && f->inflow;
}

// local stage of E elements into FP32 operators (classical or learned)
elrt_status local_stage(elrt_ctx* ctx, const elrt_solve_opts* o, int64_t E, double h, const double* h_elem,
                        const double* kappa, const double* omega, float* i2o, float* i2m, elrt_field_stats* st) {
    if (o->net && elrt_net_matches(o->net, &ctx->disc)) {
        int64_t nf = 0;
        elrt_status s =
            elrt_build_local_learned(ctx, o->net, E, h, h_elem, kappa, omega, o->learned_tol, i2o, i2m, nullptr, &nf);
        if (st) st->n_fallback += nf;
        return s;
    }
    elrt_local_stats ls{};
    elrt_status s = local_build(ctx, E, h, h_elem, kappa, omega, o->mode, o->refine_steps, ELRT_F32, i2o, i2m, nullptr,
                                st ? &ls : nullptr);
    if (st) st->local = ls;
    return s;
}

}  // namespace

extern "C" elrt_status elrt_solve_field(elrt_ctx* ctx, const elrt_field* f, const elrt_solve_opts* o, double* mean,
                                        double* skeleton, elrt_field_stats* stats) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_solve_field: null context");
    if (!field_ok(f) || !opts_ok(o) || !mean) return ctx_fail(ctx, ELRT_EINVAL, "elrt_solve_field: bad arguments");
    ctx->last_error.clear();
    if (stats) memset(stats, 0, sizeof(*stats));
    const Tab& t = ctx->tab;
    const int64_t E = (int64_t)f->nx * f->nz;
    const size_t per_o = (size_t)t.nin * t.nin, per_m = (size_t)t.nm * t.nin;
    elrt_status s = ensure_ws(ctx, &ctx->ops, &ctx->ops_bytes, (size_t)E * (per_o + per_m) * sizeof(float) + 256);
    if (s) return s;
    float* i2o = (float*)ctx->ops;
    float* i2m = i2o + (size_t)E * per_o;
    double* sk = skeleton;
    if (!sk) {
        s = ensure_ws(ctx, &ctx->vec, &ctx->vec_bytes, (size_t)E * t.nin * sizeof(double));
        if (s) return s;
        sk = (double*)ctx->vec;
    }
    auto t0 = std::chrono::steady_clock::now();
    s = local_stage(ctx, o, E, f->h, nullptr, f->kappa, f->omega, i2o, i2m, stats);
    if (s) return s;
    s = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "local stage");
    if (s) return s;
    if (stats) stats->local_ms = ms_since(t0);
    t0 = std::chrono::steady_clock::now();
    elrt_solve_stats gs{};
    elrt_status sg = global_solve(ctx, f->nx, f->nz, i2o, ELRT_F32, f->inflow, o->rtol, o->max_iter, o->restart, 0, sk, &gs);
    if (sg != ELRT_OK && sg != ELRT_ENOCONV) return sg;
    s = global_recover(ctx, f->nx, f->nz, i2m, ELRT_F32, sk, f->inflow, mean);
    if (!s) s = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "recover");
    if (stats) {
        stats->global = gs;
        stats->global_ms = ms_since(t0);
    }
    return s ? s : sg;
}

extern "C" elrt_status elrt_solve_batch(elrt_ctx* const* ctxs, int32_t n_ctx, const elrt_field* fields,
                                        const int32_t* field_ctx, int32_t n_fields, const elrt_solve_opts* o,
                                        size_t wave_bytes, int32_t workers, double* const* means,
                                        elrt_field_stats* stats) {
    if (!ctxs || n_ctx < 1 || !fields || !field_ctx || n_fields < 0 || !opts_ok(o) || !means)
        return ctx_fail(nullptr, ELRT_EINVAL, "elrt_solve_batch: bad arguments");
    for (int k = 0; k < n_ctx; ++k)
        if (!ctxs[k]) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_solve_batch: null context");
    for (int f = 0; f < n_fields; ++f)
        if (!field_ok(&fields[f]) || field_ctx[f] < 0 || field_ctx[f] >= n_ctx || !means[f])
            return ctx_fail(nullptr, ELRT_EINVAL, "elrt_solve_batch: bad field " + std::to_string(f));
    if (stats) memset(stats, 0, sizeof(elrt_field_stats) * (size_t)n_fields);
    if (n_fields == 0) return ELRT_OK;
    if (wave_bytes == 0) wave_bytes = (size_t)64 << 30;
    if (workers <= 0) workers = 8;
    workers = std::min(workers, n_fields);
    int dev = 0;
    cudaGetDevice(&dev);

    // worker contexts (one per worker and discretisation) on their own streams
    std::vector<cudaStream_t> streams(workers, nullptr);
    std::vector<std::vector<elrt_ctx*>> wctx(workers, std::vector<elrt_ctx*>(n_ctx, nullptr));
    elrt_status first = ELRT_OK;
    for (int w = 0; w < workers && !first; ++w) {
        if (cudaStreamCreateWithFlags(&streams[w], cudaStreamNonBlocking) != cudaSuccess)
            first = ctx_fail(nullptr, ELRT_ECUDA, "worker stream");
        for (int k = 0; k < n_ctx && !first; ++k) {
            first = elrt_create(&wctx[w][k], &ctxs[k]->disc, streams[w]);
            if (!first) {
                wctx[w][k]->krylov_op = ctxs[k]->krylov_op;
                wctx[w][k]->precond = ctxs[k]->precond;
                wctx[w][k]->lu_products = ctxs[k]->lu_products;
                wctx[w][k]->graphs = ctxs[k]->graphs;
                wctx[w][k]->tune = ctxs[k]->tune;
            }
        }
    }
    auto per_field_ops = [&](int f) {
        const Tab& t = ctxs[field_ctx[f]]->tab;
        return (size_t)fields[f].nx * fields[f].nz * ((size_t)t.nin * t.nin + (size_t)t.nm * t.nin) * sizeof(float);
    };
    int f0 = 0;
    while (!first && f0 < n_fields) {
        // the wave: consecutive fields whose operators fit in wave_bytes (at least one)
        int f1 = f0;
        size_t bytes = 0;
        while (f1 < n_fields && (f1 == f0 || bytes + per_field_ops(f1) <= wave_bytes)) bytes += per_field_ops(f1++);
        // one batched local stage per discretisation
        std::vector<float*> i2o(n_fields, nullptr), i2m(n_fields, nullptr);
        std::vector<void*> bufs;
        for (int k = 0; k < n_ctx && !first; ++k) {
            elrt_ctx* c = ctxs[k];
            const Tab& t = c->tab;
            int64_t E = 0;
            for (int f = f0; f < f1; ++f)
                if (field_ctx[f] == k) E += (int64_t)fields[f].nx * fields[f].nz;
            if (E == 0) continue;
            const size_t per_o = (size_t)t.nin * t.nin, per_m = (size_t)t.nm * t.nin;
            void* buf = nullptr;
            const size_t need = (size_t)E * ((per_o + per_m) * sizeof(float) + (t.nm + 2) * sizeof(double)) + 1024;
            if (cudaMalloc(&buf, need) != cudaSuccess) {
                first = ctx_fail(c, ELRT_ENOMEM, "batch wave buffers");
                break;
            }
            bufs.push_back(buf);
            float* go = (float*)buf;
            float* gm = go + (size_t)E * per_o;
            double* gk = (double*)(gm + (size_t)E * per_m);
            double* gw = gk + (size_t)E * t.nm;
            double* gh = gw + E;
            std::vector<double> hh((size_t)E);
            int64_t e0 = 0;
            for (int f = f0; f < f1; ++f) {
                if (field_ctx[f] != k) continue;
                const int64_t Ef = (int64_t)fields[f].nx * fields[f].nz;
                cudaMemcpyAsync(gk + e0 * t.nm, fields[f].kappa, (size_t)Ef * t.nm * sizeof(double),
                                cudaMemcpyDeviceToDevice, c->stream);
                cudaMemcpyAsync(gw + e0, fields[f].omega, (size_t)Ef * sizeof(double), cudaMemcpyDeviceToDevice,
                                c->stream);
                std::fill(hh.begin() + e0, hh.begin() + e0 + Ef, fields[f].h);
                i2o[f] = go + (size_t)e0 * per_o;
                i2m[f] = gm + (size_t)e0 * per_m;
                e0 += Ef;
            }
            cudaMemcpyAsync(gh, hh.data(), (size_t)E * sizeof(double), cudaMemcpyHostToDevice, c->stream);
            auto t0 = std::chrono::steady_clock::now();
            elrt_field_stats gst{};
            elrt_status s = local_stage(c, o, E, 1.0, gh, gk, gw, go, gm, &gst);
            if (!s) s = cuda_check(c, cudaStreamSynchronize(c->stream), "batched local stage");
            const double lms = ms_since(t0);
            if (stats)
                for (int f = f0; f < f1; ++f)
                    if (field_ctx[f] == k) {
                        stats[f].local = gst.local;
                        stats[f].local_ms = lms;  // shared by the fields of the batched build
                    }
            if (s) first = s;
        }
        // skeleton solves on the workers
        std::atomic<int> next(f0);
        std::vector<elrt_status> wstat(workers, ELRT_OK);
        std::vector<std::thread> pool;
        for (int w = 0; w < workers && !first; ++w) {
            pool.emplace_back([&, w] {
                cudaSetDevice(dev);
                void* skb = nullptr;
                size_t skn = 0;
                for (int f = next++; f < f1; f = next++) {
                    elrt_ctx* c = wctx[w][field_ctx[f]];
                    const int64_t n = (int64_t)fields[f].nx * fields[f].nz * c->tab.nin;
                    if ((size_t)n * sizeof(double) > skn) {
                        if (skb) cudaFree(skb);
                        skb = nullptr;
                        skn = 0;
                        if (cudaMalloc(&skb, (size_t)n * sizeof(double)) != cudaSuccess) {
                            wstat[w] = ELRT_ENOMEM;
                            break;
                        }
                        skn = (size_t)n * sizeof(double);
                    }
                    auto t0 = std::chrono::steady_clock::now();
                    elrt_solve_stats gs{};
                    elrt_status s = global_solve(c, fields[f].nx, fields[f].nz, i2o[f], ELRT_F32, fields[f].inflow,
                                                 o->rtol, o->max_iter, o->restart, 0, (double*)skb, &gs);
                    elrt_status r = global_recover(c, fields[f].nx, fields[f].nz, i2m[f], ELRT_F32, (double*)skb,
                                                   fields[f].inflow, means[f]);
                    if (!r) r = cuda_check(c, cudaStreamSynchronize(c->stream), "recover");
                    if (stats) {
                        stats[f].global = gs;
                        stats[f].global_ms = ms_since(t0);
                    }
                    if (s == ELRT_OK) s = r;
                    if (s != ELRT_OK && wstat[w] == ELRT_OK) wstat[w] = s;
                }
                if (skb) cudaFree(skb);
            });
        }
        for (auto& th : pool) th.join();
        for (int w = 0; w < workers; ++w)
            if (!first && wstat[w]) first = wstat[w];
        for (int k = 0; k < n_ctx; ++k) cudaStreamSynchronize(ctxs[k]->stream);
        for (void* b : bufs) cudaFree(b);
        f0 = f1;
    }
    for (int w = 0; w < workers; ++w) {
        for (int k = 0; k < n_ctx; ++k)
            if (wctx[w][k]) elrt_destroy(wctx[w][k]);
        if (streams[w]) cudaStreamDestroy(streams[w]);
    }
    return first;
}
