// Internal: the context object behind the C ABI handle and the helpers the
// library's host translation units share (not part of the C ABI).
//
// rq_context.cu: context lifecycle, configuration, column tiles, workspace,
//                forward-pass plan, profiling, info.
// rq_setup.cu:   target set-up (sector blocks of U, dense targets), circuit
//                geometry, translation representatives.
// rq_eval.cu:    the sweep schedule of one evaluation, host evaluations and
//                their CUDA graphs, the full Hessian, evaluation entry points.
#pragma once

#include "rq_internal.h"

#include <cstdint>
#include <string>
#include <vector>

using rq::GateGeom;

struct rq_ctx {
    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    // problem
    bool ready = false;
    rq_target tgt{};
    int n = 0, L = 0, g = 0, P = 0, structure = 0;
    std::vector<int32_t> pairs, param_of;
    std::vector<GateGeom> geo;
    long long n_store = 0;
    // sectors of the target
    int S = 0;
    std::vector<long long> off_basis, off_u;
    std::vector<int32_t> basis_h, sec_of_h, pos_h;
    int32_t *d_sec_of = nullptr, *d_pos = nullptr, *d_basis = nullptr;
    long long *d_off_basis = nullptr, *d_off_u = nullptr;
    double2 *d_U = nullptr;
    long long u_entries = 0;
    // columns and tiles
    long long c0 = 0, c1 = 0;
    int B = 0, log2B = 0, n_tiles = 0, kc = 1;
    int user_B = 0, user_kc = 0;
    std::vector<int> tile_parity;
    int32_t *d_cols = nullptr;
    std::vector<int32_t> cols_h;  // host copy of the column table (tiles x B; -1: padding)
    // workspace
    double2 *d_psi = nullptr, *d_dpsi = nullptr, *d_lam = nullptr, *d_dlam = nullptr;
    double *d_part = nullptr, *d_partd = nullptr;
    int ncta = 0;
    int grid_items = 0;  // rq_set_grid: minimum items per thread of a full sweep (0: fill the GPU)
    double *d_env = nullptr, *d_envd = nullptr;
    int envd_cap = 0;
    double *d_fpart = nullptr, *d_facc = nullptr;
    double2 *d_gates = nullptr, *d_in_gates = nullptr;
    double2 *d_dirs = nullptr, *d_dirs_raw = nullptr;
    int dirs_cap = 0;
    int32_t *d_param_of = nullptr;
    double *d_out = nullptr;
    long long out_cap = 0;
    long long problem_bytes = 0, work_bytes = 0, small_bytes = 0;
    long long launches = 0;
    long long cols_cap = 0;
    int space = 0;  // 0 Riemannian outputs, 1 Euclidean (rq_set_gradient_space)
    int arith = 0;  // 0 FP64 sweeps, 1 double-float sweeps (rq_set_arithmetic)
    // translation-representative basis sums (rq_set_translation)
    int ckpt_r = 1;    // effective: store psi at every ckpt_r-th gate, recompute the rest
    int ckpt_req = 0;  // requested interval (0: automatic, from the memory budget)
    long long alloc_slots = 0;
    int tshift = 0;
    std::vector<int32_t> reps;     // orbit representatives, ascending
    std::vector<double> rep_w;     // orbit sizes
    double *d_wts = nullptr;       // per tile column, parallel to d_cols
    double2 *d_gates_df = nullptr, *d_dirs_df = nullptr;  // df64 copies (float4 per entry)
    // per-kernel profiling (events bracket every launch while enabled)
    struct ProfRec {
        int family;
        cudaEvent_t a, b;
        double flops, bytes;
    };
    bool prof_on = false;
    std::vector<ProfRec> prof;
    size_t prof_used = 0;
    // CUDA graphs of host-memory evaluations, keyed by (k, env_mode); an entry
    // is valid while the context's configuration version is unchanged
    struct GraphEntry {
        cudaGraphExec_t exec = nullptr;
        int k = -1, env = -1;
        long long version = -1, launches = 0, last_use = 0;
    };
    std::vector<GraphEntry> graphs;
    bool use_graphs = true;
    long long version = 0, graph_clock = 0;
    int checks = 0;  // validate the gates of every call (unitarity, parity pattern)
    bool first_layer = true;  // FP64 sweeps of the leading disjoint gates visit only nonzero items
    bool last_layer = true;   // backward sweeps of the trailing disjoint gates skip items with zero adjoint
    // window fusion of the forward pass (rq_set_fusion): execution order of
    // the gates (a reordering of commuting disjoint gates) and its passes
    int fuse_q = 0;  // largest window in stored bits; 0: off (every gate its own pass, original order)
    struct PassPlan {
        int pos, m;        // first position in `order`, number of gates
        long long wmask;   // stored bits of the window
    };
    std::vector<int> order;
    std::vector<PassPlan> plan;
};

namespace rqc {

enum Family : int { kFamFwd = 0, kFamBwdDir, kFamBwdBase, kFamTarget, kFamInit, kFamReduce, kFamGeometry, kFamCheb, kFamCount };
extern const char *const kFamilyName[kFamCount];

// Event bracket of one launch while profiling is on.
struct ProfScope {
    rq_ctx *ctx;
    rq_ctx::ProfRec *rec = nullptr;
    ProfScope(rq_ctx *c, int family, double flops, double bytes) : ctx(c) {
        if (!ctx->prof_on) return;
        if (ctx->prof_used == ctx->prof.size()) {
            rq_ctx::ProfRec r{};
            if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
            ctx->prof.push_back(r);
        }
        rec = &ctx->prof[ctx->prof_used++];
        rec->family = family;
        rec->flops = flops;
        rec->bytes = bytes;
        cudaEventRecord(rec->a, ctx->stream);
    }
    ~ProfScope() {
        if (rec) cudaEventRecord(rec->b, ctx->stream);
    }
};

// Records the message on the context (or, without one, as this thread's
// rq_create error) and returns code.
rq_status fail(rq_ctx *ctx, rq_status code, const char *fmt, ...);

#define RQ_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return fail(ctx, RQ_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define RQ_LAUNCHED()                                                                     \
    do {                                                                                  \
        ++ctx->launches;                                                                  \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess) return fail(ctx, RQ_ECUDA, "kernel launch: %s", cudaGetErrorString(e_)); \
    } while (0)

#define RQ_TRY(expr)                 \
    do {                             \
        rq_status s_ = (expr);       \
        if (s_ != RQ_OK) return s_;  \
    } while (0)

template <typename T>
rq_status dev_alloc(rq_ctx *ctx, T **p, long long count, long long &counter) {
    *p = nullptr;
    if (count <= 0) return RQ_OK;
    const size_t bytes = (size_t)count * sizeof(T);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(ctx, RQ_ENOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    counter += (long long)bytes;
    return RQ_OK;
}

template <typename T>
void dev_free(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

void free_workspace(rq_ctx *ctx);
void free_small(rq_ctx *ctx);
bool workspace_ok(const rq_ctx *ctx);
void drop_graphs(rq_ctx *ctx);
void free_problem(rq_ctx *ctx);
int ilog2(long long v);
void plan_passes(rq_ctx *ctx);
// Whether evaluations run the fused forward schedule (and walk the plan's
// execution order backwards): a fusion window, every state kept, whole
// 32-column chunks per tile, and a plan with at least one multi-gate pass.
bool fused_schedule(const rq_ctx *ctx);
// Last-layer marks of the gates for the backward order the evaluations use.
void mark_tail(rq_ctx *ctx);
long long state_slots(const rq_ctx *ctx);
long long bytes_per_column(const rq_ctx *ctx, int kc);
rq_status rebuild_tiles(rq_ctx *ctx);
rq_status ensure_small(rq_ctx *ctx, int k);
rq::TargetDev target_dev(const rq_ctx *ctx);
rq_status build_target_dense(rq_ctx *ctx, const double *dense);
rq_status build_target(rq_ctx *ctx);
rq_status eval_dev(rq_ctx *ctx, const double *gates, const double *dirs, int k, int env_mode,
                   double *f_out, double *rgrad, double *hvps);

}  // namespace rqc
