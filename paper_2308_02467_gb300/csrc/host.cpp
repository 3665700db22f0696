// Host side of the library: discretisation tables, context management, argument checks and the
// extern "C" entry points declared in include/elrt.h.
//
// The 1D ingredients are computed here from their textbook definitions:
//   * LGL nodes: Newton's method on P_{p-1}(x) - x P_p(x) (= (1-x^2) P_p'(x) / p), whose
//     derivative is -(p+1) P_p(x) by Legendre's equation, from Chebyshev-Lobatto guesses;
//     weights 2 / (p (p+1) P_p(x_j)^2).
//   * Lagrange derivative matrix by the barycentric formula (Berrut & Trefethen 2004).
//   * Gauss-Legendre rule (for the phase integrals) by Newton on P_n.
//   * Phase matrix: the cell-pair double integral of the HG kernel written as one integral of
//     the kernel against the triangle (box * box) weight, Gauss-Legendre on each half.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "elrt_internal.h"

namespace {

const double kPi = 3.14159265358979323846;

void legendre(int n, double x, double* pn, double* pnm1) {
    double p0 = 1.0, p1 = x;
    if (n == 0) { *pn = 1.0; *pnm1 = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *pnm1 = p0;
}

void lgl_rule(int p, double* xi, double* w) {
    xi[0] = -1.0;
    xi[p] = 1.0;
    for (int j = 1; j < p; ++j) {
        double x = -cos(kPi * j / p);
        for (int it = 0; it < 100; ++it) {
            double pn, pm;
            legendre(p, x, &pn, &pm);
            double dx = (pm - x * pn) / ((p + 1.0) * pn);
            x += dx;
            if (fabs(dx) < 1e-16) break;
        }
        xi[j] = x;
    }
    for (int j = 0; j <= p; ++j) {
        double pn, pm;
        legendre(p, xi[j], &pn, &pm);
        w[j] = 2.0 / (p * (p + 1.0) * pn * pn);
    }
}

void gauss_rule(int n, std::vector<double>& x, std::vector<double>& w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = cos(kPi * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double pn, pm;
            legendre(n, z, &pn, &pm);
            double dp = n * (z * pn - pm) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double pn, pm;
        legendre(n, z, &pn, &pm);
        double dp = n * (z * pn - pm) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

void barycentric_derivative(int n1, const double* x, double* D) {
    std::vector<double> lam(n1, 1.0);
    for (int j = 0; j < n1; ++j)
        for (int k = 0; k < n1; ++k)
            if (k != j) lam[j] /= (x[j] - x[k]);
    for (int i = 0; i < n1; ++i) {
        double diag = 0.0;
        for (int j = 0; j < n1; ++j) {
            if (j == i) continue;
            double v = (lam[j] / lam[i]) / (x[i] - x[j]);
            D[i * n1 + j] = v;
            diag -= v;
        }
        D[i * n1 + i] = diag;
    }
}

double hg(double t, double g) { return (1.0 - g * g) / pow(1.0 + g * g - 2.0 * g * cos(t), 1.5); }

// wc[m] = W[m][0]; the matrix is circulant because the cells are uniform.
void phase_first_column(int N, double g, int angular, double* wc) {
    const double dth = 2.0 * kPi / N;
    std::vector<double> gx, gw;
    gauss_rule(64, gx, gw);
    double c = 0.0;  // int_0^{2pi} of the unnormalised kernel
    for (int k = 0; k < N; ++k)
        for (size_t q = 0; q < gx.size(); ++q) c += 0.5 * dth * gw[q] * hg(k * dth + 0.5 * dth * (gx[q] + 1.0), g);
    for (int m = 0; m < N; ++m) {
        double v = 0.0;
        if (angular == ELRT_ANG_FV0) {
            // (1/dth) int_{-dth}^{dth} (dth - |u|) p(m dth + u) du
            for (size_t q = 0; q < gx.size(); ++q) {
                double u = 0.5 * dth * (gx[q] + 1.0);  // in [0, dth]
                v += 0.5 * dth * gw[q] * (dth - u) * (hg(m * dth + u, g) + hg(m * dth - u, g));
            }
            v /= (dth * c);
        } else {
            v = dth * hg(m * dth, g) / c;
        }
        wc[m] = v;
    }
    double s = 0.0;
    for (int m = 0; m < N; ++m) s += wc[m];
    for (int m = 0; m < N; ++m) wc[m] /= s;
}

bool disc_ok(const elrt_disc* d) {
    return d && d->p >= 1 && d->p + 1 <= ELRT_MAX_N1 && d->n_angles >= 4 && d->n_angles <= ELRT_MAX_ANG &&
           d->n_angles % 4 == 0 && (d->angular == ELRT_ANG_FV0 || d->angular == ELRT_ANG_DO) && d->hg_g >= 0.0 &&
           d->hg_g < 1.0;
}

void directions(int N, int angular, double* sx, double* sz) {
    const double dth = 2.0 * kPi / N;
    for (int k = 0; k < N; ++k) {
        if (angular == ELRT_ANG_FV0) {
            sx[k] = (sin((k + 1) * dth) - sin(k * dth)) / dth;
            sz[k] = (cos(k * dth) - cos((k + 1) * dth)) / dth;
        } else {
            sx[k] = cos((k + 0.5) * dth);
            sz[k] = sin((k + 0.5) * dth);
        }
    }
}

bool build_tab(const elrt_disc* d, Tab* t) {
    memset(t, 0, sizeof(Tab));
    const int p = d->p, N = d->n_angles;
    t->p = p;
    t->n1 = p + 1;
    t->nm = (p + 1) * (p + 1);
    t->N = N;
    t->half = N / 2;
    t->nu = t->nm * N;
    t->nface = (p + 1) * (N / 2);
    t->nin = 4 * t->nface;
    t->nrhs = t->nin;
    double xi[ELRT_MAX_N1];
    lgl_rule(p, xi, t->w);
    barycentric_derivative(p + 1, xi, t->D);
    directions(N, d->angular, t->sx, t->sz);
    phase_first_column(N, d->hg_g, d->angular, t->wc);
    const double nx[4] = {0.0, 1.0, 0.0, -1.0}, nz[4] = {-1.0, 0.0, 1.0, 0.0};
    for (int F = 0; F < 4; ++F) {
        int no = 0, ni = 0;
        for (int k = 0; k < N; ++k) {
            double s = t->sx[k] * nx[F] + t->sz[k] * nz[F];
            t->sdn[F][k] = s;
            if (s > 0) {
                if (no >= N / 2) return false;
                t->outc[F][no++] = (signed char)k;
            } else if (s < 0) {
                if (ni >= N / 2) return false;
                t->inc[F][ni++] = (signed char)k;
            } else {
                return false;
            }
        }
        if (no != N / 2 || ni != N / 2) return false;
    }
    return true;
}

thread_local std::string g_err;

}  // namespace

bool elrt_disc_valid(const elrt_disc* d) { return disc_ok(d); }
bool elrt_fill_tab(const elrt_disc* d, Tab* t) { return disc_ok(d) && build_tab(d, t); }

elrt_status ctx_fail(elrt_ctx* ctx, elrt_status s, const std::string& msg) {
    if (ctx) ctx->last_error = msg;
    g_err = msg;
    return s;
}

elrt_status cuda_check(elrt_ctx* ctx, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return ELRT_OK;
    return ctx_fail(ctx, e == cudaErrorMemoryAllocation ? ELRT_ENOMEM : ELRT_ECUDA,
                    std::string(what) + ": " + cudaGetErrorString(e));
}

elrt_status ensure_ws(elrt_ctx* ctx, void** buf, size_t* have, size_t need) {
    if (*have >= need) return ELRT_OK;
    if (*buf) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_check(ctx, e, "sync before workspace growth");
        cudaFree(*buf);
        *buf = nullptr;
        *have = 0;
    }
    cudaError_t e = cudaMalloc(buf, need);
    if (e != cudaSuccess) {
        *buf = nullptr;
        return cuda_check(ctx, e, "workspace allocation");
    }
    *have = need;
    return ELRT_OK;
}

static cudaEvent_t pool_get(elrt_ctx* ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

ProfScope::ProfScope(elrt_ctx* c, const char* name, int nlaunch, double bytes, double flops) : ctx(c), idx(-1) {
    ctx->launches += nlaunch;
    if (!ctx->profiling) return;
    auto& w = ctx->work[name];
    w.first += bytes;
    w.second += flops;
    cudaEvent_t a = pool_get(ctx), b = pool_get(ctx);
    if (!a || !b) return;
    cudaEventRecord(a, ctx->stream);
    ctx->pending.push_back({name, a, b});
    idx = (int)ctx->pending.size() - 1;
}

ProfScope::~ProfScope() {
    if (idx >= 0) cudaEventRecord(ctx->pending[idx].b, ctx->stream);
}

void prof_flush(elrt_ctx* ctx) {
    for (auto& p : ctx->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            auto& v = ctx->prof[p.name];
            v.first += ms;
            v.second += 1;
        }
        ctx->event_pool.push_back(p.a);
        ctx->event_pool.push_back(p.b);
    }
    ctx->pending.clear();
}

extern "C" {

elrt_status elrt_profile_enable(elrt_ctx* ctx, int32_t on) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_profile_enable: null context");
    ctx->profiling = on != 0;
    return ELRT_OK;
}

elrt_status elrt_profile_reset(elrt_ctx* ctx) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_profile_reset: null context");
    cudaStreamSynchronize(ctx->stream);
    prof_flush(ctx);
    ctx->prof.clear();
    ctx->work.clear();
    ctx->launches = 0;
    return ELRT_OK;
}

elrt_status elrt_profile_get(elrt_ctx* ctx, const char* kernel, double* total_ms, int64_t* launches) {
    if (!ctx || !kernel || !total_ms || !launches) return ctx_fail(ctx, ELRT_EINVAL, "elrt_profile_get: bad arguments");
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "elrt_profile_get");
    prof_flush(ctx);
    auto it = ctx->prof.find(kernel);
    *total_ms = it == ctx->prof.end() ? 0.0 : it->second.first;
    *launches = it == ctx->prof.end() ? 0 : it->second.second;
    return ELRT_OK;
}

elrt_status elrt_profile_work(elrt_ctx* ctx, const char* kernel, double* bytes, double* flops) {
    if (!ctx || !kernel || !bytes || !flops) return ctx_fail(ctx, ELRT_EINVAL, "elrt_profile_work: bad arguments");
    auto it = ctx->work.find(kernel);
    *bytes = it == ctx->work.end() ? 0.0 : it->second.first;
    *flops = it == ctx->work.end() ? 0.0 : it->second.second;
    return ELRT_OK;
}

int64_t elrt_launch_count(const elrt_ctx* ctx) { return ctx ? ctx->launches : -1; }

int64_t elrt_n_nodes(const elrt_disc* d) { return disc_ok(d) ? (int64_t)(d->p + 1) * (d->p + 1) : -1; }
int64_t elrt_n_local(const elrt_disc* d) { return disc_ok(d) ? (int64_t)(d->p + 1) * (d->p + 1) * d->n_angles : -1; }
int64_t elrt_n_skel(const elrt_disc* d) { return disc_ok(d) ? (int64_t)2 * (d->p + 1) * d->n_angles : -1; }
int64_t elrt_n_inflow(const elrt_disc* d, int32_t nx, int32_t nz) {
    if (!disc_ok(d) || nx < 1 || nz < 1) return -1;
    return (int64_t)2 * (nx + nz) * (d->p + 1) * (d->n_angles / 2);
}

elrt_status elrt_lgl(int32_t p, double* xi, double* w) {
    if (p < 1 || p + 1 > ELRT_MAX_N1 || !xi || !w) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_lgl: bad arguments");
    lgl_rule(p, xi, w);
    return ELRT_OK;
}

elrt_status elrt_phase_matrix(const elrt_disc* d, double* W) {
    if (!disc_ok(d) || !W) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_phase_matrix: bad arguments");
    double wc[ELRT_MAX_ANG];
    phase_first_column(d->n_angles, d->hg_g, d->angular, wc);
    const int N = d->n_angles;
    for (int k = 0; k < N; ++k)
        for (int l = 0; l < N; ++l) W[k * N + l] = wc[((k - l) % N + N) % N];
    return ELRT_OK;
}

elrt_status elrt_node_coords(const elrt_disc* d, int32_t nx, int32_t nz, double h, double* x, double* z) {
    if (!disc_ok(d) || nx < 1 || nz < 1 || !(h > 0) || !x || !z)
        return ctx_fail(nullptr, ELRT_EINVAL, "elrt_node_coords: bad arguments");
    double xi[ELRT_MAX_N1], w[ELRT_MAX_N1];
    lgl_rule(d->p, xi, w);
    const int n1 = d->p + 1, nm = n1 * n1;
    for (int64_t e = 0; e < (int64_t)nx * nz; ++e) {
        int ix = (int)(e % nx), iz = (int)(e / nx);
        for (int i = 0; i < nm; ++i) {
            int a = i % n1, b = i / n1;
            x[e * nm + i] = ix * h + 0.5 * h * (xi[a] + 1.0);
            z[e * nm + i] = iz * h + 0.5 * h * (xi[b] + 1.0);
        }
    }
    return ELRT_OK;
}

elrt_status elrt_create(elrt_ctx** out, const elrt_disc* disc, void* stream) {
    if (!out) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_create: null output");
    *out = nullptr;
    if (!disc_ok(disc))
        return ctx_fail(nullptr, ELRT_EINVAL,
                        "elrt_create: need 1 <= p <= 10, 4 <= N <= 32 with N % 4 == 0, angular 0/1, 0 <= g < 1");
    elrt_ctx* c = new (std::nothrow) elrt_ctx();
    if (!c) return ctx_fail(nullptr, ELRT_ENOMEM, "elrt_create: host allocation");
    c->disc = *disc;
    if (!build_tab(disc, &c->tab)) {
        delete c;
        return ctx_fail(nullptr, ELRT_EINVAL, "elrt_create: an angular cell is tangent to a face");
    }
    c->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) {
        cudaDeviceProp prop;
        e = cudaGetDeviceProperties(&prop, c->device);
        if (e == cudaSuccess) c->dev_bytes = prop.totalGlobalMem;
    }
    if (e == cudaSuccess) e = cudaMalloc(&c->d_flags, 256 * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_pinned, 4096);
    if (e != cudaSuccess) {
        elrt_status s = cuda_check(nullptr, e, "elrt_create");
        if (c->d_flags) cudaFree(c->d_flags);
        delete c;
        return s;
    }
    tune_load(c);
    *out = c;
    return ELRT_OK;
}

elrt_status elrt_destroy(elrt_ctx* ctx) {
    if (!ctx) return ELRT_OK;
    cudaStreamSynchronize(ctx->stream);
    prof_flush(ctx);
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->gm) cudaFree(ctx->gm);
    if (ctx->gm16) cudaFree(ctx->gm16);
    if (ctx->ops) cudaFree(ctx->ops);
    if (ctx->vec) cudaFree(ctx->vec);
    if (ctx->d_flags) cudaFree(ctx->d_flags);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    delete ctx;
    return ELRT_OK;
}

elrt_status elrt_set_stream(elrt_ctx* ctx, void* stream) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_set_stream: null context");
    ctx->stream = (cudaStream_t)stream;
    return ELRT_OK;
}

elrt_status elrt_set_krylov_op(elrt_ctx* ctx, int32_t op) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_set_krylov_op: null context");
    if (op != ELRT_KRYLOV_F32 && op != ELRT_KRYLOV_F16) return ctx_fail(ctx, ELRT_EINVAL, "elrt_set_krylov_op: op");
    ctx->krylov_op = op;
    return ELRT_OK;
}

elrt_status elrt_set_graphs(elrt_ctx* ctx, int32_t on) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_set_graphs: null context");
    ctx->graphs = on ? 1 : 0;
    return ELRT_OK;
}

elrt_status elrt_set_precond(elrt_ctx* ctx, int32_t kind) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_set_precond: null context");
    if (kind != ELRT_PRECOND_NONE && kind != ELRT_PRECOND_SWEEP)
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_set_precond: ELRT_PRECOND_NONE or ELRT_PRECOND_SWEEP");
    ctx->precond = kind;
    return ELRT_OK;
}

elrt_status elrt_set_lu_products(elrt_ctx* ctx, int32_t mode) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_set_lu_products: null context");
    if (mode != ELRT_LU_PRODUCTS_AUTO && mode != ELRT_LU_PRODUCTS_TF32)
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_set_lu_products: ELRT_LU_PRODUCTS_AUTO or ELRT_LU_PRODUCTS_TF32");
    ctx->lu_products = mode;
    return ELRT_OK;
}

const char* elrt_status_str(elrt_status s) {
    switch (s) {
        case ELRT_OK: return "ok";
        case ELRT_EINVAL: return "invalid argument";
        case ELRT_ENOMEM: return "out of device memory";
        case ELRT_ESINGULAR: return "singular local matrix";
        case ELRT_ENOCONV: return "iteration did not converge";
        case ELRT_ETIMEOUT: return "device wait timed out";
        case ELRT_ECUDA: return "CUDA error";
        case ELRT_ENOTRAINED: return "network not trained";
    }
    return "unknown status";
}

const char* elrt_last_error(const elrt_ctx* ctx) { return ctx ? ctx->last_error.c_str() : g_err.c_str(); }

elrt_status elrt_assemble(elrt_ctx* ctx, int64_t n_elems, double h, const double* h_elem, const double* kappa,
                          const double* omega, double* A, double* rhs) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_assemble: null context");
    if (n_elems < 0 || (n_elems > 0 && (!kappa || !omega || !A || !rhs)) || (!h_elem && !(h > 0)))
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_assemble: bad arguments");
    ctx->last_error.clear();
    if (n_elems == 0) return ELRT_OK;
    return local_assemble_f64(ctx, n_elems, h, h_elem, kappa, omega, A, rhs);
}

elrt_status elrt_build_local(elrt_ctx* ctx, int64_t n_elems, double h, const double* h_elem, const double* kappa,
                             const double* omega, int32_t mode, int32_t refine_steps, int32_t out_dtype,
                             void* in2out, void* in2sol, int32_t* elem_status, elrt_local_stats* stats) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_build_local: null context");
    if (n_elems < 0 || (n_elems > 0 && (!kappa || !omega || !in2out || !in2sol)) || (!h_elem && !(h > 0)))
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_build_local: bad arguments");
    if (mode < ELRT_LOCAL_FP64 || mode > ELRT_LOCAL_TF32_IR)
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_build_local: unknown mode");
    if (out_dtype != ELRT_F32 && out_dtype != ELRT_F64)
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_build_local: unknown output dtype");
    if (refine_steps < 0 || refine_steps > 8)
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_build_local: refine_steps must be in 0..8");
    ctx->last_error.clear();
    if (stats) memset(stats, 0, sizeof(*stats));
    if (n_elems == 0) return ELRT_OK;
    return local_build(ctx, n_elems, h, h_elem, kappa, omega, mode, refine_steps, out_dtype, in2out, in2sol,
                       elem_status, stats);
}

elrt_status elrt_build_local_ex(elrt_ctx* ctx, int64_t n_elems, double h, const double* h_elem, const double* kappa,
                                const double* omega, int32_t mode, int32_t refine_steps, int32_t out_dtype,
                                void* in2out, void* in2sol, const elrt_local_extras* extras, int32_t* elem_status,
                                elrt_local_stats* stats) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_build_local_ex: null context");
    if (extras && extras->source && n_elems > 0 && (!extras->f2o || !extras->f2m))
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_build_local_ex: a source needs f2o and f2m");
    if (n_elems < 0 || (n_elems > 0 && (!kappa || !omega || !in2out || !in2sol)) || (!h_elem && !(h > 0)))
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_build_local_ex: bad arguments");
    if (mode < ELRT_LOCAL_FP64 || mode > ELRT_LOCAL_TF32_IR)
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_build_local_ex: unknown mode");
    if (out_dtype != ELRT_F32 && out_dtype != ELRT_F64)
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_build_local_ex: unknown output dtype");
    if (refine_steps < 0 || refine_steps > 8)
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_build_local_ex: refine_steps must be in 0..8");
    ctx->last_error.clear();
    if (stats) memset(stats, 0, sizeof(*stats));
    if (n_elems == 0) return ELRT_OK;
    return local_build(ctx, n_elems, h, h_elem, kappa, omega, mode, refine_steps, out_dtype, in2out, in2sol,
                       elem_status, stats, extras);
}

elrt_status elrt_global_apply(elrt_ctx* ctx, int32_t nx, int32_t nz, const void* in2out, int32_t dtype,
                              const double* x, double* y) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_global_apply: null context");
    if (nx < 1 || nz < 1 || !in2out || !x || !y || (dtype != ELRT_F32 && dtype != ELRT_F64))
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_global_apply: bad arguments");
    ctx->last_error.clear();
    return global_apply(ctx, nx, nz, in2out, dtype, x, y);
}

elrt_status elrt_solve_global(elrt_ctx* ctx, int32_t nx, int32_t nz, const void* in2out, int32_t dtype,
                              const double* inflow, double rtol, int32_t max_iter, int32_t restart, int32_t use_guess,
                              double* skeleton, elrt_solve_stats* stats) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_solve_global: null context");
    if (nx < 1 || nz < 1 || !in2out || !inflow || !skeleton || (dtype != ELRT_F32 && dtype != ELRT_F64) ||
        !(rtol > 0) || max_iter < 1 || restart < 0 || restart > 200)
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_solve_global: bad arguments (restart must be 0..200)");
    ctx->last_error.clear();
    if (stats) memset(stats, 0, sizeof(*stats));
    return global_solve(ctx, nx, nz, in2out, dtype, inflow, rtol, max_iter, restart, use_guess, skeleton, stats);
}

elrt_status elrt_recover_mean(elrt_ctx* ctx, int32_t nx, int32_t nz, const void* in2sol, int32_t dtype,
                              const double* skeleton, const double* inflow, double* mean) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_recover_mean: null context");
    if (nx < 1 || nz < 1 || !in2sol || !skeleton || !inflow || !mean || (dtype != ELRT_F32 && dtype != ELRT_F64))
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_recover_mean: bad arguments");
    ctx->last_error.clear();
    return global_recover(ctx, nx, nz, in2sol, dtype, skeleton, inflow, mean);
}

elrt_status elrt_solve_global_source(elrt_ctx* ctx, int32_t nx, int32_t nz, const void* in2out, int32_t dtype,
                                     const double* inflow, const double* f2o, double rtol, int32_t max_iter,
                                     int32_t restart, int32_t use_guess, double* skeleton, elrt_solve_stats* stats) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_solve_global_source: null context");
    if (nx < 1 || nz < 1 || !in2out || !inflow || !skeleton || (dtype != ELRT_F32 && dtype != ELRT_F64) ||
        !(rtol > 0) || max_iter < 1 || restart < 0 || restart > 200)
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_solve_global_source: bad arguments (restart must be 0..200)");
    ctx->last_error.clear();
    if (stats) memset(stats, 0, sizeof(*stats));
    return global_solve(ctx, nx, nz, in2out, dtype, inflow, rtol, max_iter, restart, use_guess, skeleton, stats, f2o);
}

elrt_status elrt_recover_mean_source(elrt_ctx* ctx, int32_t nx, int32_t nz, const void* in2sol, int32_t dtype,
                                     const double* f2m, const double* skeleton, const double* inflow, double* mean) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_recover_mean_source: null context");
    if (nx < 1 || nz < 1 || !in2sol || !skeleton || !inflow || !mean || (dtype != ELRT_F32 && dtype != ELRT_F64))
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_recover_mean_source: bad arguments");
    ctx->last_error.clear();
    return global_recover(ctx, nx, nz, in2sol, dtype, skeleton, inflow, mean, f2m);
}

elrt_status elrt_recover_radiance(elrt_ctx* ctx, int32_t nx, int32_t nz, const void* in2rad, int32_t dtype,
                                  const double* f2u, const double* skeleton, const double* inflow, double* u) {
    if (!ctx) return ctx_fail(nullptr, ELRT_EINVAL, "elrt_recover_radiance: null context");
    if (nx < 1 || nz < 1 || !in2rad || !skeleton || !inflow || !u || (dtype != ELRT_F32 && dtype != ELRT_F64))
        return ctx_fail(ctx, ELRT_EINVAL, "elrt_recover_radiance: bad arguments");
    ctx->last_error.clear();
    return global_recover_rows(ctx, nx, nz, ctx->tab.nu, in2rad, dtype, skeleton, inflow, f2u, u);
}

}  // extern "C"
