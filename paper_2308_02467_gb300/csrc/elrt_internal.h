// Internal declarations shared by the host code and the kernels of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/elrt.h"

#define ELRT_MAX_N1 11   // p <= 10
#define ELRT_MAX_ANG 32  // N <= 32

// Everything a kernel needs to know about the element discretisation; passed by value
// (fits in the 4 KB classic kernel-parameter space).
struct Tab {
    int p, n1, nm, N, half, nu, nin, nface;
    int nrhs;                                   // right-hand-side columns the local LU solves: nin (+1 with a source)
    double w[ELRT_MAX_N1];                      // LGL weights
    double D[ELRT_MAX_N1 * ELRT_MAX_N1];        // D[m*n1+a] = l_a'(xi_m)
    double sx[ELRT_MAX_ANG], sz[ELRT_MAX_ANG];  // direction of cell k
    double wc[ELRT_MAX_ANG];                    // circulant phase: W[k][l] = wc[(k-l) mod N]
    double sdn[4][ELRT_MAX_ANG];                // sbar_k . n_F
    signed char outc[4][ELRT_MAX_ANG / 2];      // outflow cells of face F, increasing k
    signed char inc[4][ELRT_MAX_ANG / 2];       // inflow cells of face F, increasing k
};

// volume node at face position m of face F (bottom, right, top, left)
__host__ __device__ inline int face_node(int F, int m, int p) {
    int n1 = p + 1;
    switch (F) {
        case 0: return m;
        case 1: return p + n1 * m;
        case 2: return m + n1 * p;
        default: return n1 * m;
    }
}

// Launch parameters the autotuner (tune.cpp) measures and sets; the defaults are the hand-chosen ones.
struct Tuning {
    int64_t local_chunk = 0;  // elements per local-build chunk (0: as many as the workspace budget holds)
    int lu_pairs = 1;         // tensor-core LU: panels in pairs with rank-128 updates (1) or one at a time (0)
    int restart = 12;         // GMRES restart length of calls that pass restart = 0
    int tuned = 0;            // 1 once measured or loaded from the cache
};

struct elrt_ctx {
    elrt_disc disc;
    Tuning tune;
    Tab tab;
    cudaStream_t stream;
    int device;
    int sms = 152;  // streaming multiprocessors of the device (persistent grids are sized on it)
    size_t dev_bytes = (size_t)128 << 30;  // device memory (the local build's workspace is sized on it)
    std::string last_error;
    // workspace (grown on demand)
    void* ws = nullptr;
    size_t ws_bytes = 0;
    void* gm = nullptr;     // GMRES workspace
    size_t gm_bytes = 0;
    void* gm16 = nullptr;   // FP16 copy of the skeleton operator (Arnoldi steps)
    size_t gm16_bytes = 0;
    int krylov_op = ELRT_KRYLOV_F32;
    int graphs = 1;         // replay GMRES restart cycles from captured CUDA graphs
    int precond = ELRT_PRECOND_SWEEP;
    int lu_products = ELRT_LU_PRODUCTS_AUTO;  // products of the tensor-core LU's trailing updates  // skeleton GMRES preconditioner (FP32 operators)
    void* ops = nullptr;    // in2out / in2sol of elrt_solve_field
    size_t ops_bytes = 0;
    void* vec = nullptr;    // skeleton of elrt_solve_field when the caller passes none
    size_t vec_bytes = 0;
    int* d_flags = nullptr; // small device scratch for flags/counters
    double* h_pinned = nullptr;  // pinned host scratch for small read-backs
    // measurement
    int64_t launches = 0;
    bool profiling = false;
    struct Pending { const char* name; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    std::map<std::string, std::pair<double, int64_t>> prof;
    std::map<std::string, std::pair<double, double>> work;  // algorithmic bytes, flops of timed launches
};

// Brackets kernel launches with events when profiling is on; counts launches always.  bytes and
// flops are the algorithmic work of the bracketed launches (every operand read once, every result
// written once; useful arithmetic only), summed per name while profiling is on.
struct ProfScope {
    elrt_ctx* ctx;
    int idx;
    ProfScope(elrt_ctx* c, const char* name, int nlaunch = 1, double bytes = 0.0, double flops = 0.0);
    ~ProfScope();
};
void prof_flush(elrt_ctx* ctx);  // call after a stream synchronisation

// ---- autotuning (tune.cpp): apply the cached parameters of this device and discretisation
void tune_load(elrt_ctx* ctx);

// ---- host helpers implemented in host.cpp
bool elrt_disc_valid(const elrt_disc* d);
bool elrt_fill_tab(const elrt_disc* d, Tab* t);
elrt_status ctx_fail(elrt_ctx* ctx, elrt_status s, const std::string& msg);
elrt_status cuda_check(elrt_ctx* ctx, cudaError_t e, const char* what);
elrt_status ensure_ws(elrt_ctx* ctx, void** buf, size_t* have, size_t need);

// ---- launchers implemented in local.cu
elrt_status local_assemble_f64(elrt_ctx* ctx, int64_t E, double h, const double* h_elem, const double* kappa,
                               const double* omega, double* A, double* rhs);
elrt_status local_build(elrt_ctx* ctx, int64_t E, double h, const double* h_elem, const double* kappa,
                        const double* omega, int mode, int refine_steps, int out_dtype, void* in2out,
                        void* in2sol, int32_t* elem_status, elrt_local_stats* stats,
                        const elrt_local_extras* extras = nullptr);

// ---- tensor-core LU (lu_tc.cu).  f16: the trailing updates form their products as 3xFP16 (FP16
// high parts and remainders, half the MMA instructions of 3xTF32), allowed for a factorisation when
// every entry of the assembled matrices lies in [kLuF16Max / 4096, kLuF16Max]; the refinement
// re-solves pass false (their right-hand sides are residuals far below FP16's normal range).
constexpr float kLuF16Max = 1024.f;
constexpr int kAsmMaxFlag = 24;  // d_flags slot: largest |entry| of the assembled FP32 matrices (float bits)
elrt_status tc_lu_factor_solve(elrt_ctx* ctx, float* M, int64_t ld, int64_t estride, int64_t E, int* estat, float* side,
                               int* err, int nrhs, bool f16);
elrt_status tc_lu_resolve(elrt_ctx* ctx, float* M, int64_t ld, int64_t estride, int64_t E, float* side, int* err,
                          int nrhs, bool f16, const double* res_max);
size_t tc_lu_side_floats(const Tab& t, int64_t ld);

// ---- launchers implemented in global.cu
elrt_status global_apply(elrt_ctx* ctx, int nx, int nz, const void* A, int dtype, const double* x, double* y);
elrt_status global_solve(elrt_ctx* ctx, int nx, int nz, const void* A, int dtype, const double* inflow,
                         double rtol, int max_iter, int restart, int use_guess, double* x,
                         elrt_solve_stats* stats, const double* f2o = nullptr);
elrt_status global_recover(elrt_ctx* ctx, int nx, int nz, const void* A, int dtype, const double* x,
                           const double* inflow, double* mean, const double* f2m = nullptr);
elrt_status global_recover_rows(elrt_ctx* ctx, int nx, int nz, int rows, const void* A, int dtype, const double* x,
                                const double* inflow, const double* self, double* out);

// ---- sweep preconditioner of the skeleton GMRES (sweep.cu)
void sweep_orders(int nx, int nz, int* out);                 // [4 E] work items in their global order
size_t sweep_words_bytes(const Tab& t, int64_t E);          // scratch of one application's outflow words
elrt_status sweep_apply(elrt_ctx* ctx, int nx, int nz, const void* A, int a_bytes, const float* u, float* z,
                        const int* order, void* zw, int* flags, const int* done, const int* nsteps);

// ---- learned local stage (mlp.cu)
extern "C" elrt_status elrt_build_local_learned(elrt_ctx* ctx, elrt_net* net, int64_t n, double h, const double* h_elem,
                                                const double* kappa, const double* omega, double tol, float* in2out,
                                                float* in2sol, float* estimate, int64_t* n_fallback);
bool elrt_net_matches(const elrt_net* net, const elrt_disc* disc);

// ---- network checkpoint file (ckpt.cpp): layout of the FP32 arrays, CRC-32, encode/decode
uint32_t ckpt_crc32(const void* data, size_t n, uint32_t crc);
std::vector<size_t> ckpt_layout(const elrt_net_desc& d);
bool ckpt_write(const char* path, const elrt_net_desc& d, int32_t standardised, int64_t step,
                const std::vector<const float*>& arrays, std::string* err);
bool ckpt_read(const char* path, elrt_net_desc* d, int32_t* standardised, int64_t* step, int64_t* n_floats,
               std::vector<float>* payload, std::string* err);
