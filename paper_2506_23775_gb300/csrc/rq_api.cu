// C ABI entry points: context, target set-up, column tiles, workspace and the
// tile-by-tile sweep schedule of one evaluation.
//
// One evaluation sums over basis columns (Eq. f_target_sum_unit_vec) tile by
// tile.  For a tile of B columns:
//   1. psi_0 = |j_b> for every column b;
//   2. forward pass, caching every psi_l (Fig. forward_pass) and, for each
//      HVP direction swept together, the tangent psi'_l;
//   3. lambda_g = U|j_b> and the cost summands (target blocks, Eq.
//      f_target_sum_unit_vec);
//   4. backward pass, gate by gate in reverse: direction steps first (they
//      read lambda_l), then the base step (environment E_l, lambda update),
//      per-CTA environment partials (Fig. backward_pass_gate_gradient);
//   5. per-gate partials summed in CTA order into the evaluation's
//      accumulators.
// After the last tile one kernel turns the accumulators into f, the
// Riemannian gradient and the HVPs.  Work for one context is queued on its
// stream in a fixed order, so results are reproducible bit for bit.
#include "rq_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

using rq::GateGeom;

namespace rq {
// rq_sweep_df64.cu: shared-memory limits of the double-float kernels
cudaError_t init_sweep_attributes_df64();
}  // namespace rq

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
    // workspace
    double2 *d_psi = nullptr, *d_dpsi = nullptr, *d_lam = nullptr, *d_dlam = nullptr;
    double *d_part = nullptr, *d_partd = nullptr;
    int ncta = 0;
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

namespace {

thread_local std::string g_create_error;  // text of the last rq_create failure of this thread

enum Family : int { kFamFwd = 0, kFamBwdDir, kFamBwdBase, kFamTarget, kFamInit, kFamReduce, kFamGeometry, kFamCheb, kFamCount };
const char *const kFamilyName[kFamCount] = {"fwd_gate", "bwd_gate_dir", "bwd_gate_base", "target_scatter_cost",
                                            "init_unit", "reduce", "geometry", "target_chebyshev"};

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

rq_status fail(rq_ctx *ctx, rq_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf; else g_create_error = buf;
    return code;
}

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

void free_workspace(rq_ctx *ctx) {
    dev_free(ctx->d_psi);
    dev_free(ctx->d_dpsi);
    dev_free(ctx->d_lam);
    dev_free(ctx->d_dlam);
    dev_free(ctx->d_part);
    dev_free(ctx->d_partd);
    dev_free(ctx->d_fpart);
    ctx->work_bytes = 0;
}

void free_small(rq_ctx *ctx) {
    dev_free(ctx->d_env);
    dev_free(ctx->d_envd);
    dev_free(ctx->d_facc);
    dev_free(ctx->d_gates);
    dev_free(ctx->d_in_gates);
    dev_free(ctx->d_dirs);
    dev_free(ctx->d_dirs_raw);
    dev_free(ctx->d_gates_df);
    dev_free(ctx->d_dirs_df);
    dev_free(ctx->d_param_of);
    dev_free(ctx->d_out);
    dev_free(ctx->d_cols);
    dev_free(ctx->d_wts);
    ctx->cols_cap = 0;
    ctx->envd_cap = ctx->dirs_cap = 0;
    ctx->out_cap = 0;
    ctx->small_bytes = 0;
}

// The tile workspace exists (a failed reallocation leaves it released).
bool workspace_ok(const rq_ctx *ctx) {
    return ctx->d_psi && ctx->d_dpsi && ctx->d_lam && ctx->d_dlam && ctx->d_part && ctx->d_partd && ctx->d_fpart;
}

void drop_graphs(rq_ctx *ctx) {
    for (auto &e : ctx->graphs)
        if (e.exec) cudaGraphExecDestroy(e.exec);
    ctx->graphs.clear();
}

void free_problem(rq_ctx *ctx) {
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    drop_graphs(ctx);
    ++ctx->version;
    free_workspace(ctx);
    free_small(ctx);
    dev_free(ctx->d_sec_of);
    dev_free(ctx->d_pos);
    dev_free(ctx->d_basis);
    dev_free(ctx->d_off_basis);
    dev_free(ctx->d_off_u);
    dev_free(ctx->d_U);
    ctx->problem_bytes = 0;
    ctx->ready = false;
}

int ilog2(long long v) {
    int r = 0;
    while ((1LL << r) < v) ++r;
    return r;
}

// Execution order and passes of the forward sweep.  Without fusion every
// gate is its own pass in circuit order.  With fusion (window of at most
// fuse_q stored bits) the leading run of disjoint gates (first-layer
// support) stays first and unfused; then, greedily, a pass starts with the
// next remaining gate and takes every later remaining gate that fits in the
// window and commutes with every remaining gate it moves past -- gates on
// disjoint qubits commute (the gates of a brickwall layer, Sec. "Brick wall
// circuit layout") -- up to kMaxPassGates gates.  Parity gates on the implied
// qubit are never fused; they block their stored bit.  The product of the
// gates in the new order is the same circuit, so f, the gradient and the HVP
// are unchanged (up to rounding order); the backward pass walks the same
// order in reverse.
long long gate_bits(const GateGeom &gg) {
    return gg.mode == rq::kParity2 ? (1LL << gg.pa) : ((1LL << gg.pa) | (1LL << gg.pb));
}

void plan_passes(rq_ctx *ctx) {
    const int g = ctx->g;
    ctx->order.clear();
    ctx->plan.clear();
    int prefix = 0;
    if (ctx->first_layer) {
        long long used = 0;
        for (; prefix < g; ++prefix) {
            const long long b = gate_bits(ctx->geo[prefix]);
            if (used & b) break;
            used |= b;
        }
    }
    if (ctx->fuse_q <= 2) prefix = g;
    for (int l = 0; l < prefix; ++l) {
        ctx->plan.push_back({(int)ctx->order.size(), 1, gate_bits(ctx->geo[l])});
        ctx->order.push_back(l);
    }
    std::vector<int> rest;
    for (int l = prefix; l < g; ++l) rest.push_back(l);
    while (!rest.empty()) {
        const int g0 = rest[0];
        std::vector<int> take = {g0};
        long long W = gate_bits(ctx->geo[g0]);
        if (ctx->geo[g0].mode != rq::kParity2) {
            long long blocked = 0;
            for (size_t i = 1; i < rest.size(); ++i) {
                const GateGeom &gg = ctx->geo[rest[i]];
                const long long b = gate_bits(gg);
                if (gg.mode == rq::kParity2 || (b & blocked) ||
                    __builtin_popcountll(W | b) > ctx->fuse_q || (int)take.size() >= rq::kMaxPassGates) {
                    blocked |= b;
                    continue;
                }
                take.push_back(rest[i]);
                W |= b;
            }
        }
        ctx->plan.push_back({(int)ctx->order.size(), (int)take.size(), W});
        std::vector<int> left;
        size_t t = 0;
        for (int l : rest) {
            if (t < take.size() && take[t] == l) {
                ctx->order.push_back(l);
                ++t;
            } else {
                left.push_back(l);
            }
        }
        rest.swap(left);
    }
}

// Column lists of the current range: one list (general gates) or the even-
// then the odd-parity columns (parity gates: every tile shares one parity).
void column_groups(const rq_ctx *ctx, std::vector<std::vector<int32_t>> &groups, std::vector<int> &parity,
                   std::vector<std::vector<double>> *weights = nullptr) {
    groups.clear();
    parity.clear();
    if (weights) weights->clear();
    if (ctx->tshift > 0) {  // weighted orbit representatives (the range is the whole basis)
        const int ng = ctx->structure == 1 ? 2 : 1;
        groups.resize(ng);
        if (weights) weights->resize(ng);
        for (int gi = 0; gi < ng; ++gi) parity.push_back(gi);
        for (size_t i = 0; i < ctx->reps.size(); ++i) {
            const int gi = ctx->structure == 1 ? (__builtin_popcountll(ctx->reps[i]) & 1) : 0;
            groups[gi].push_back(ctx->reps[i]);
            if (weights) (*weights)[gi].push_back(ctx->rep_w[i]);
        }
        return;
    }
    if (ctx->structure == 1) {
        std::vector<int32_t> ev, od;
        for (long long j = ctx->c0; j < ctx->c1; ++j) (__builtin_popcountll(j) & 1 ? od : ev).push_back((int32_t)j);
        groups.push_back(std::move(ev));
        parity.push_back(0);
        groups.push_back(std::move(od));
        parity.push_back(1);
    } else {
        std::vector<int32_t> all;
        for (long long j = ctx->c0; j < ctx->c1; ++j) all.push_back((int32_t)j);
        groups.push_back(std::move(all));
        parity.push_back(0);
    }
}

// State slots of one checkpoint set: every gate (interval 1), or one
// checkpoint per segment of `interval` gates plus a segment buffer.
long long state_slots(const rq_ctx *ctx) {
    const int r = ctx->ckpt_r;
    if (r <= 1) return ctx->g + 1;
    const long long nseg = (ctx->g + r - 1) / r;
    return nseg + r + 1;
}

long long bytes_per_column(const rq_ctx *ctx, int kc) {
    const long long sets = (long long)(1 + kc) * state_slots(ctx) + 1 + kc;
    return sets * ctx->n_store * (long long)sizeof(double2);
}

// Choose B (columns per tile) and kc (directions per sweep), build the tile
// column table and (re)allocate the sweep workspace.  A new column range with
// the same B and kc only re-uploads the column table.
// Everything a captured evaluation depends on besides the contents of the
// column table: buffer addresses, tile geometry, the segment structure.
std::vector<long long> tile_layout(const rq_ctx *ctx) {
    std::vector<long long> v = {(long long)(uintptr_t)ctx->d_psi, (long long)(uintptr_t)ctx->d_dpsi,
                                (long long)(uintptr_t)ctx->d_lam, (long long)(uintptr_t)ctx->d_dlam,
                                (long long)(uintptr_t)ctx->d_part, (long long)(uintptr_t)ctx->d_partd,
                                (long long)(uintptr_t)ctx->d_fpart, (long long)(uintptr_t)ctx->d_cols,
                                (long long)(uintptr_t)ctx->d_wts, ctx->B, ctx->kc, ctx->ncta, ctx->ckpt_r,
                                ctx->tshift > 0, ctx->n_tiles};
    v.insert(v.end(), ctx->tile_parity.begin(), ctx->tile_parity.end());
    return v;
}

rq_status rebuild_tiles_impl(rq_ctx *ctx);

// New column tables that keep the layout (e.g. the next batch of columns of
// the same size) keep the captured evaluations: the column indices and
// weights are read from device memory at run time.
rq_status rebuild_tiles(rq_ctx *ctx) {
    const std::vector<long long> before = tile_layout(ctx);
    const rq_status st = rebuild_tiles_impl(ctx);
    if (st != RQ_OK || tile_layout(ctx) != before) ++ctx->version;
    return st;
}

rq_status rebuild_tiles_impl(rq_ctx *ctx) {
    RQ_CUDA(cudaStreamSynchronize(ctx->stream));
    std::vector<std::vector<int32_t>> groups;
    std::vector<std::vector<double>> gw;
    std::vector<int> gpar;
    column_groups(ctx, groups, gpar, &gw);
    long long largest = 1;
    for (auto &gr : groups) largest = std::max<long long>(largest, (long long)gr.size());
    const int bcap = ctx->user_B > 0 ? ctx->user_B : (int)std::min<long long>(512, 1LL << ilog2(largest));
    size_t free_b = 0, total_b = 0;
    RQ_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const double avail = (double)free_b + (double)ctx->work_bytes;  // the current workspace can be reused
    const double budget = std::min(0.6 * avail, 96.0 * (1LL << 30));
    int B = 0, kc = 1;
    const int kc_opts[2] = {rq::kMaxDirs, 1};
    const int n_opts = ctx->user_kc > 0 ? 1 : 2;
    // automatic checkpointing: keep every state unless that forces tiles
    // below min(bcap, 256) columns; then a checkpoint every ~sqrt(g) gates
    // (about 2 sqrt(g) states per tile instead of g + 1)
    int r_opts[2] = {1, std::max(2, (int)std::ceil(std::sqrt((double)ctx->g)))};
    const int n_r = ctx->ckpt_req > 0 ? 1 : 2;
    if (ctx->ckpt_req > 0) r_opts[0] = std::max(1, std::min(ctx->ckpt_req, ctx->g));
    for (int ri = 0; ri < n_r && B == 0; ++ri) {
        ctx->ckpt_r = r_opts[ri];
        for (int o = 0; o < n_opts; ++o) {
            const int k = ctx->user_kc > 0 ? ctx->user_kc : kc_opts[o];
            int b = bcap;
            while (b > 1 && (double)b * bytes_per_column(ctx, k) > budget) b >>= 1;
            if ((double)b * bytes_per_column(ctx, k) > budget) continue;
            if (o + 1 < n_opts && b < std::min(bcap, 256)) continue;
            if (ri + 1 < n_r && b < std::min(bcap, 256)) continue;
            B = b;
            kc = k;
            break;
        }
    }
    if (B == 0)
        return fail(ctx, RQ_ENOMEM, "one column needs %lld bytes of workspace, %.0f available",
                    bytes_per_column(ctx, 1), budget);
    const long long items = std::max<long long>(1, ctx->n_store / 4 * B);
    // Sweeps with a full block of items for every CTA: two CTAs per SM.
    // Smaller sweeps: one CTA per SM at most (the general backward kernels fit
    // one CTA per SM, so more would run in two waves), and at least one
    // warp-sized chunk of items per CTA (the kernels hand chunks to CTAs round
    // robin, so a small sweep still reaches every SM).
    const long long full = (long long)ctx->sms * rq::kCtasPerSm * rq::kThreads;
    const int ncta = (int)(items >= full ? (long long)ctx->sms * rq::kCtasPerSm
                                         : std::min<long long>(ctx->sms, (items + 31) / 32));
    std::vector<int32_t> cols;
    std::vector<double> wts;
    std::vector<int> tpar;
    const bool weighted = ctx->tshift > 0;
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        const auto &gr = groups[gi];
        for (size_t s = 0; s < gr.size(); s += B) {
            for (int b = 0; b < B; ++b) {
                cols.push_back(s + b < gr.size() ? gr[s + b] : -1);
                if (weighted) wts.push_back(s + b < gr.size() ? gw[gi][s + b] : 0.0);
            }
            tpar.push_back(gpar[gi]);
        }
    }
    const bool same = ctx->d_psi && B == ctx->B && kc == ctx->kc && ncta == ctx->ncta &&
                      ctx->alloc_slots == state_slots(ctx);
    if (!same) {
        free_workspace(ctx);
        ctx->B = B;
        ctx->log2B = ilog2(B);
        ctx->kc = kc;
        ctx->ncta = ncta;
        ctx->alloc_slots = state_slots(ctx);
        const long long tile = ctx->n_store * B;
        RQ_TRY(dev_alloc(ctx, &ctx->d_psi, tile * state_slots(ctx), ctx->work_bytes));
        RQ_TRY(dev_alloc(ctx, &ctx->d_dpsi, tile * state_slots(ctx) * kc, ctx->work_bytes));
        RQ_TRY(dev_alloc(ctx, &ctx->d_lam, tile, ctx->work_bytes));
        RQ_TRY(dev_alloc(ctx, &ctx->d_dlam, tile * kc, ctx->work_bytes));
        RQ_TRY(dev_alloc(ctx, &ctx->d_part, (long long)ctx->g * ncta * rq::kEnvDoubles, ctx->work_bytes));
        RQ_TRY(dev_alloc(ctx, &ctx->d_partd, (long long)kc * ctx->g * ncta * rq::kEnvDoubles, ctx->work_bytes));
        RQ_TRY(dev_alloc(ctx, &ctx->d_fpart, B, ctx->work_bytes));
    }
    if ((long long)cols.size() > ctx->cols_cap) {
        dev_free(ctx->d_cols);
        dev_free(ctx->d_wts);
        ctx->cols_cap = 0;
        RQ_TRY(dev_alloc(ctx, &ctx->d_cols, (long long)cols.size(), ctx->small_bytes));
        RQ_TRY(dev_alloc(ctx, &ctx->d_wts, (long long)cols.size(), ctx->small_bytes));
        ctx->cols_cap = (long long)cols.size();
    }
    ctx->tile_parity = tpar;
    ctx->n_tiles = (int)tpar.size();
    if (!cols.empty()) {
        RQ_CUDA(cudaMemcpyAsync(ctx->d_cols, cols.data(), cols.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                ctx->stream));
        if (weighted)
            RQ_CUDA(cudaMemcpyAsync(ctx->d_wts, wts.data(), wts.size() * sizeof(double), cudaMemcpyHostToDevice,
                                    ctx->stream));
        RQ_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return RQ_OK;
}

rq_status ensure_small(rq_ctx *ctx, int k) {
    if (k > ctx->dirs_cap) {
        ++ctx->version;
        RQ_CUDA(cudaStreamSynchronize(ctx->stream));
        dev_free(ctx->d_dirs);
        dev_free(ctx->d_dirs_raw);
        dev_free(ctx->d_dirs_df);
        dev_free(ctx->d_envd);
        dev_free(ctx->d_out);
        ctx->out_cap = 0;
        const int cap = std::max(k, 4);
        RQ_TRY(dev_alloc(ctx, &ctx->d_dirs, (long long)cap * ctx->P * 16, ctx->small_bytes));
        RQ_TRY(dev_alloc(ctx, &ctx->d_dirs_df, (long long)cap * ctx->P * 16, ctx->small_bytes));
        RQ_TRY(dev_alloc(ctx, &ctx->d_dirs_raw, (long long)cap * ctx->P * 16, ctx->small_bytes));
        RQ_TRY(dev_alloc(ctx, &ctx->d_envd, (long long)cap * ctx->g * rq::kEnvDoubles, ctx->small_bytes));
        ctx->dirs_cap = ctx->envd_cap = cap;
    }
    // f at [0], then 16-byte aligned complex outputs from [2]
    const long long need = 2 + (long long)(1 + ctx->dirs_cap) * ctx->P * 32;
    if (need > ctx->out_cap) {
        ++ctx->version;
        dev_free(ctx->d_out);
        RQ_TRY(dev_alloc(ctx, &ctx->d_out, need, ctx->small_bytes));
        ctx->out_cap = need;
    }
    return RQ_OK;
}

rq::TargetDev target_dev(const rq_ctx *ctx) {
    rq::TargetDev t;
    t.sec_of = ctx->d_sec_of;
    t.pos = ctx->d_pos;
    t.basis = ctx->d_basis;
    t.off_basis = ctx->d_off_basis;
    t.off_u = ctx->d_off_u;
    t.U = ctx->d_U;
    return t;
}

// Dense target (model 2): the caller's 2^n x 2^n matrix, row-major.  With
// general gates it is one block over all basis states.  With parity gates the
// circuit keeps every column in the parity sector of its basis state, so only
// the two parity-diagonal blocks of U enter f and its derivatives (the
// off-diagonal blocks pair with amplitudes that are zero); they are stored as
// two sectors.  Blocks are stored column by column, like the chain targets.
rq_status build_target_dense(rq_ctx *ctx, const double *dense) {
    const int n = ctx->n;
    const long long dim = 1LL << n;
    const bool by_parity = ctx->structure == 1;
    ctx->S = by_parity ? 2 : 1;
    std::vector<long long> count(ctx->S, 0);
    ctx->sec_of_h.assign(dim, 0);
    ctx->pos_h.assign(dim, 0);
    for (long long x = 0; x < dim; ++x) {
        const int s = by_parity ? (__builtin_popcountll(x) & 1) : 0;
        ctx->sec_of_h[x] = s;
        ctx->pos_h[x] = (int32_t)count[s]++;
    }
    ctx->off_basis.assign(ctx->S + 1, 0);
    ctx->off_u.assign(ctx->S + 1, 0);
    for (int s = 0; s < ctx->S; ++s) {
        ctx->off_basis[s + 1] = ctx->off_basis[s] + count[s];
        ctx->off_u[s + 1] = ctx->off_u[s] + count[s] * count[s];
    }
    ctx->basis_h.assign(dim, 0);
    for (long long x = 0; x < dim; ++x) ctx->basis_h[ctx->off_basis[ctx->sec_of_h[x]] + ctx->pos_h[x]] = (int32_t)x;
    ctx->u_entries = ctx->off_u[ctx->S];
    std::vector<double2> blocks((size_t)ctx->u_entries);
    for (long long j = 0; j < dim; ++j) {
        const int s = ctx->sec_of_h[j];
        const long long m = count[s];
        double2 *col = blocks.data() + ctx->off_u[s] + (long long)ctx->pos_h[j] * m;
        for (long long r = 0; r < m; ++r) {
            const long long x = ctx->basis_h[ctx->off_basis[s] + r];
            col[r] = make_double2(dense[2 * (x * dim + j)], dense[2 * (x * dim + j) + 1]);
        }
    }
    RQ_TRY(dev_alloc(ctx, &ctx->d_sec_of, dim, ctx->problem_bytes));
    RQ_TRY(dev_alloc(ctx, &ctx->d_pos, dim, ctx->problem_bytes));
    RQ_TRY(dev_alloc(ctx, &ctx->d_basis, dim, ctx->problem_bytes));
    RQ_TRY(dev_alloc(ctx, &ctx->d_off_basis, ctx->S + 1, ctx->problem_bytes));
    RQ_TRY(dev_alloc(ctx, &ctx->d_off_u, ctx->S + 1, ctx->problem_bytes));
    RQ_TRY(dev_alloc(ctx, &ctx->d_U, ctx->u_entries, ctx->problem_bytes));
    RQ_CUDA(cudaMemcpyAsync(ctx->d_sec_of, ctx->sec_of_h.data(), dim * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    RQ_CUDA(cudaMemcpyAsync(ctx->d_pos, ctx->pos_h.data(), dim * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    RQ_CUDA(cudaMemcpyAsync(ctx->d_basis, ctx->basis_h.data(), dim * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    RQ_CUDA(cudaMemcpyAsync(ctx->d_off_basis, ctx->off_basis.data(), (ctx->S + 1) * sizeof(long long), cudaMemcpyHostToDevice, ctx->stream));
    RQ_CUDA(cudaMemcpyAsync(ctx->d_off_u, ctx->off_u.data(), (ctx->S + 1) * sizeof(long long), cudaMemcpyHostToDevice, ctx->stream));
    RQ_CUDA(cudaMemcpyAsync(ctx->d_U, blocks.data(), ctx->u_entries * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
    RQ_CUDA(cudaStreamSynchronize(ctx->stream));
    return RQ_OK;
}

// Build the per-sector target blocks on the device (Chebyshev expansion).
rq_status build_target(rq_ctx *ctx) {
    const int n = ctx->n, L = ctx->L, model = ctx->tgt.model;
    const long long dim = 1LL << n, lowmask = (1LL << L) - 1;
    // conserved labels: (N_up, N_down) for the spinful chain, N for the spinless one
    ctx->S = model == 0 ? (L + 1) * (L + 1) : L + 1;
    std::vector<long long> count(ctx->S, 0);
    ctx->sec_of_h.assign(dim, 0);
    ctx->pos_h.assign(dim, 0);
    for (long long x = 0; x < dim; ++x) {
        const int s = model == 0 ? __builtin_popcountll(x >> L) * (L + 1) + __builtin_popcountll(x & lowmask)
                                  : __builtin_popcountll(x);
        ctx->sec_of_h[x] = s;
        ctx->pos_h[x] = (int32_t)count[s]++;
    }
    ctx->off_basis.assign(ctx->S + 1, 0);
    ctx->off_u.assign(ctx->S + 1, 0);
    for (int s = 0; s < ctx->S; ++s) {
        ctx->off_basis[s + 1] = ctx->off_basis[s] + count[s];
        ctx->off_u[s + 1] = ctx->off_u[s] + count[s] * count[s];
    }
    ctx->basis_h.assign(dim, 0);
    for (long long x = 0; x < dim; ++x) ctx->basis_h[ctx->off_basis[ctx->sec_of_h[x]] + ctx->pos_h[x]] = (int32_t)x;
    ctx->u_entries = ctx->off_u[ctx->S];
    std::vector<long long> sizes(count.begin(), count.end());

    // hopping bonds as bit masks (qubit q <-> bit n-1-q): both spin chains
    // (spinful) or the one chain (spinless), plus the wrap bond if periodic
    std::vector<long long> bonds;
    const int n_chains = model == 0 ? 2 : 1;
    for (int ch = 0; ch < n_chains; ++ch) {
        const int off = ch * L;
        for (int j = 0; j + 1 < L; ++j)
            bonds.push_back((1LL << (n - 1 - off - j)) | (1LL << (n - 2 - off - j)));
        if (ctx->tgt.periodic && L > 2) bonds.push_back((1LL << (n - 1 - off - (L - 1))) | (1LL << (n - 1 - off)));
    }
    // diagonal: U n_up n_down on every site (spinful), U n_j n_{j+1} on every bond (spinless)
    auto diag_of = [&](long long x) {
        if (model == 0) return ctx->tgt.U * (double)__builtin_popcountll((x >> L) & (x & lowmask));
        int both = 0;
        for (long long mk : bonds) both += (x & mk) == mk;
        return ctx->tgt.U * both;
    };
    // Gershgorin interval of H
    const double J = ctx->tgt.J, U = ctx->tgt.U, t = ctx->tgt.t;
    double emin = 1e300, emax = -1e300;
    for (long long x = 0; x < dim; ++x) {
        const double diag = diag_of(x);
        int flips = 0;
        for (long long mk : bonds) {
            const long long bits = x & mk;
            flips += (bits != 0 && bits != mk);
        }
        emin = std::min(emin, diag - std::fabs(J) * flips);
        emax = std::max(emax, diag + std::fabs(J) * flips);
    }
    const double alpha = 0.5 * (emax - emin), beta = 0.5 * (emax + emin);
    const double xarg = alpha * std::fabs(t);
    std::vector<double> jv;
    int K = 0;
    if (alpha > 0.0 && xarg > 0.0) {
        const int kmax = (int)(1.5 * xarg) + 60;
        rq::bessel_j_table(xarg, kmax, jv);
        for (int k = 0; k <= kmax; ++k)
            if (std::fabs(jv[k]) > 1e-19) K = k;
    } else {
        jv.assign(1, 1.0);
    }
    const double ph = -beta * t;  // exp(-i beta t)
    auto coef = [&](int k) {
        // (2 - delta_k0) (-i)^k J_k(alpha t) exp(-i beta t); J_k(-x) = (-1)^k J_k(x)
        double a = (k == 0 ? 1.0 : 2.0) * jv[k] * ((t < 0 && (k & 1)) ? -1.0 : 1.0);
        double re = 0, im = 0;  // a * (-i)^k
        switch (k & 3) {
            case 0: re = a; break;
            case 1: im = -a; break;
            case 2: re = -a; break;
            default: im = a; break;
        }
        return make_double2(re * std::cos(ph) - im * std::sin(ph), re * std::sin(ph) + im * std::cos(ph));
    };

    RQ_TRY(dev_alloc(ctx, &ctx->d_sec_of, dim, ctx->problem_bytes));
    RQ_TRY(dev_alloc(ctx, &ctx->d_pos, dim, ctx->problem_bytes));
    RQ_TRY(dev_alloc(ctx, &ctx->d_basis, dim, ctx->problem_bytes));
    RQ_TRY(dev_alloc(ctx, &ctx->d_off_basis, ctx->S + 1, ctx->problem_bytes));
    RQ_TRY(dev_alloc(ctx, &ctx->d_off_u, ctx->S + 1, ctx->problem_bytes));
    RQ_TRY(dev_alloc(ctx, &ctx->d_U, ctx->u_entries, ctx->problem_bytes));
    RQ_CUDA(cudaMemcpyAsync(ctx->d_sec_of, ctx->sec_of_h.data(), dim * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    RQ_CUDA(cudaMemcpyAsync(ctx->d_pos, ctx->pos_h.data(), dim * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    RQ_CUDA(cudaMemcpyAsync(ctx->d_basis, ctx->basis_h.data(), dim * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    RQ_CUDA(cudaMemcpyAsync(ctx->d_off_basis, ctx->off_basis.data(), (ctx->S + 1) * sizeof(long long), cudaMemcpyHostToDevice, ctx->stream));
    RQ_CUDA(cudaMemcpyAsync(ctx->d_off_u, ctx->off_u.data(), (ctx->S + 1) * sizeof(long long), cudaMemcpyHostToDevice, ctx->stream));

    long long scratch = 0;
    double *tA = nullptr, *tB = nullptr;
    long long *d_sizes = nullptr, *d_bonds = nullptr;
    rq_status st = dev_alloc(ctx, &tA, ctx->u_entries, scratch);
    if (st == RQ_OK) st = dev_alloc(ctx, &tB, ctx->u_entries, scratch);
    if (st == RQ_OK) st = dev_alloc(ctx, &d_sizes, ctx->S, scratch);
    if (st == RQ_OK) st = dev_alloc(ctx, &d_bonds, (long long)std::max<size_t>(1, bonds.size()), scratch);
    if (st == RQ_OK) {
        cudaMemcpyAsync(d_sizes, sizes.data(), ctx->S * sizeof(long long), cudaMemcpyHostToDevice, ctx->stream);
        if (!bonds.empty())
            cudaMemcpyAsync(d_bonds, bonds.data(), bonds.size() * sizeof(long long), cudaMemcpyHostToDevice, ctx->stream);
        const rq::TargetDev td = target_dev(ctx);
        {
            ProfScope ps(ctx, kFamCheb, 0.0, 0.0);
            rq::launch_cheb_init(ctx->d_off_u, d_sizes, ctx->S, ctx->u_entries, tA, ctx->d_U, coef(0), ctx->stream);
        }
        ++ctx->launches;
        const double dscale = alpha > 0 ? 1.0 / alpha : 0.0, hop = alpha > 0 ? -J / alpha : 0.0;
        double *prev = tA, *cur = tB;
        for (int k = 1; k <= K; ++k) {
            if (k == 1) {
                rq::launch_cheb_step(td, ctx->S, ctx->u_entries, prev, cur, ctx->d_U, coef(1), 1.0, 1,
                                     dscale, beta, hop, d_bonds, (int)bonds.size(), L, U, model, ctx->stream);
            } else {
                rq::launch_cheb_step(td, ctx->S, ctx->u_entries, cur, prev, ctx->d_U, coef(k), 2.0, 0,
                                     dscale, beta, hop, d_bonds, (int)bonds.size(), L, U, model, ctx->stream);
                std::swap(prev, cur);
            }
            ++ctx->launches;
        }
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) st = fail(ctx, RQ_ECUDA, "target build: %s", cudaGetErrorString(e));
    }
    dev_free(tA);
    dev_free(tB);
    dev_free(d_sizes);
    dev_free(d_bonds);
    return st;
}

// One evaluation over the column range; every pointer is device memory.
// env_mode: 0 no gradient environments (cost, or HVPs whose Riemannian
// correction is not needed), 1 accumulate them, 2 reuse the accumulators of the
// previous evaluation at the same gates (the HVPs of one tCG solve).
rq_status eval_dev(rq_ctx *ctx, const double *gates, const double *dirs, int k, int env_mode,
                   double *f_out, double *rgrad, double *hvps) {
    if (!ctx->ready) return fail(ctx, RQ_ESTATE, "no target set up (call rq_setup_target first)");
    if (k < 0) return fail(ctx, RQ_EINVAL, "k = %d < 0", k);
    if (!gates) return fail(ctx, RQ_EINVAL, "gates is NULL");
    if (k > 0 && !dirs) return fail(ctx, RQ_EINVAL, "dirs is NULL with k = %d", k);
    // complex128 arrays are read and written as 16-byte double2
    const auto misaligned = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) != 0; };
    if (misaligned(gates) || (k > 0 && misaligned(dirs)) || (rgrad && misaligned(rgrad)) || (hvps && misaligned(hvps)))
        return fail(ctx, RQ_EINVAL, "gates, dirs, rgrad and hvps must be 16-byte aligned device pointers");
    RQ_TRY(ensure_small(ctx, k));
    if (!workspace_ok(ctx))
        return fail(ctx, RQ_ESTATE, "the sweep workspace is not allocated (a previous tile, column-range or "
                    "checkpointing change failed): set the tile again");
    cudaStream_t s = ctx->stream;
    const int g = ctx->g, P = ctx->P;
    {
        ProfScope ps(ctx, kFamGeometry, 0.0, 2.0 * P * 16 * sizeof(double2));
        rq::launch_mask_gates(reinterpret_cast<const double2 *>(gates), ctx->d_gates, P, ctx->structure, s);
    }
    RQ_LAUNCHED();
    if (k > 0) {
        ProfScope ps(ctx, kFamGeometry, 0.0, 2.0 * k * P * 16 * sizeof(double2));
        rq::launch_project_dirs(ctx->d_gates, reinterpret_cast<const double2 *>(dirs), ctx->d_dirs, P, k,
                                ctx->structure, ctx->space, s);
        RQ_LAUNCHED();
    }
    if (k > 0 && env_mode == 0) env_mode = 1;  // the HVP correction needs the gradient environments
    const bool want_env = env_mode == 1;
    const bool df = ctx->arith == 1;
    if (env_mode != 2) RQ_CUDA(cudaMemsetAsync(ctx->d_env, 0, sizeof(double) * g * rq::kEnvDoubles, s));
    if (k > 0) RQ_CUDA(cudaMemsetAsync(ctx->d_envd, 0, sizeof(double) * (size_t)k * g * rq::kEnvDoubles, s));
    RQ_CUDA(cudaMemsetAsync(ctx->d_facc, 0, sizeof(double), s));

    if (df) {  // df64 copies of the (masked) gates and (projected) directions
        {
            ProfScope ps(ctx, kFamGeometry, 0.0, 0.0);
            rq::launch_to_df64(ctx->d_gates, ctx->d_gates_df, (long long)P * 16, s);
        }
        RQ_LAUNCHED();
        if (k > 0) {
            {
                ProfScope ps(ctx, kFamGeometry, 0.0, 0.0);
                rq::launch_to_df64(ctx->d_dirs, ctx->d_dirs_df, (long long)k * P * 16, s);
            }
            RQ_LAUNCHED();
        }
    }
    const bool first_layer = ctx->first_layer;
    const double2 *gsrc = df ? ctx->d_gates_df : ctx->d_gates;
    const double2 *dsrc = df ? ctx->d_dirs_df : ctx->d_dirs;
    const int B = ctx->B;
    const long long tile = ctx->n_store * B;
    // State slots: interval 1 keeps psi_l in slot l (the paper's forward-pass
    // cache).  Interval r > 1 keeps psi at the start of every segment of r
    // gates (slots 0 .. nseg-1) plus a segment buffer (slots nseg .. nseg+r);
    // the backward pass recomputes each segment from its checkpoint with the
    // same kernels, so the results are bitwise those of interval 1.
    const int r = ctx->ckpt_r;
    const int nseg = (g + r - 1) / r;
    const long long set = tile * state_slots(ctx);  // one checkpoint set
    const bool backward = want_env || k > 0;
    // fused forward passes: every checkpoint slot exists (interval 1) and a
    // tile has whole 32-column chunks
    const bool fused = ctx->fuse_q > 2 && r == 1 && B >= 32 && (int)ctx->plan.size() < g;
    const int n_chunks = k == 0 ? 1 : (k + ctx->kc - 1) / ctx->kc;
    for (int ch = 0; ch < n_chunks; ++ch) {
        const int d0 = ch * ctx->kc;
        const int kd = k == 0 ? 0 : std::min(ctx->kc, k - d0);
        const bool first = ch == 0;
        for (int ti = 0; ti < ctx->n_tiles; ++ti) {
            const int32_t *cols = ctx->d_cols + (long long)ti * B;
            const double *wts = ctx->tshift > 0 ? ctx->d_wts + (long long)ti * B : nullptr;
            const int par = ctx->tile_parity[ti];
            // gate l from slot si to slot so (with the tangents of this chunk)
            auto fwd = [&](int l, long long si, long long so) -> rq_status {
                const GateGeom &geo = ctx->geo[l];
                rq::FwdArgs a;
                a.psi_in = ctx->d_psi + si * tile;
                a.psi_out = ctx->d_psi + so * tile;
                a.dpsi_in = ctx->d_dpsi + si * tile;
                a.dpsi_out = ctx->d_dpsi + so * tile;
                a.dir_stride = set;
                a.kdirs = kd;
                a.gate = gsrc + (long long)geo.param * 16;
                a.dirs = dsrc + ((long long)d0 * P + geo.param) * 16;
                a.xdir_stride = (long long)P * 16;
                a.geo = geo;
                a.log2B = ctx->log2B;
                a.tile_parity = par;
                a.n_items = (geo.mode == rq::kParity2 ? ctx->n_store / 2 : ctx->n_store / 4) * B;
                if (geo.restricted && first_layer) {
                    // only the items where psi_{l-1} can be nonzero; the rest
                    // of psi_l (and its tangents) is zero
                    a.cols = cols;
                    a.n_items = (long long)B << __builtin_popcountll(geo.free_bits);
                    RQ_CUDA(cudaMemsetAsync(a.psi_out, 0, sizeof(double2) * tile, s));
                    for (int d = 0; d < kd; ++d)
                        RQ_CUDA(cudaMemsetAsync(a.dpsi_out + d * set, 0, sizeof(double2) * tile, s));
                }
                {
                    const double amps = geo.mode == rq::kParity2 ? 2.0 : 4.0;
                    const double cm = geo.mode == rq::kGeneral ? 16.0 : (geo.mode == rq::kParity4 ? 8.0 : 4.0);
                    ProfScope ps(ctx, kFamFwd, (double)a.n_items * 8.0 * cm * (1 + 2 * kd),
                                 (double)a.n_items * amps * sizeof(double2) * 2 * (1 + kd));
                    if (df) rq::launch_fwd_df64(a, ctx->ncta, s);
                    else rq::launch_fwd(a, ctx->ncta, s);
                }
                RQ_LAUNCHED();
                return RQ_OK;
            };
            auto copy_slot = [&](long long from, long long to) -> rq_status {
                RQ_CUDA(cudaMemcpyAsync(ctx->d_psi + to * tile, ctx->d_psi + from * tile, sizeof(double2) * tile,
                                        cudaMemcpyDeviceToDevice, s));
                for (int d = 0; d < kd; ++d)
                    RQ_CUDA(cudaMemcpyAsync(ctx->d_dpsi + d * set + to * tile, ctx->d_dpsi + d * set + from * tile,
                                            sizeof(double2) * tile, cudaMemcpyDeviceToDevice, s));
                return RQ_OK;
            };
            const long long slot0 = r == 1 ? 0 : nseg;
            RQ_CUDA(cudaMemsetAsync(ctx->d_psi + slot0 * tile, 0, sizeof(double2) * tile, s));
            {
                ProfScope ps(ctx, kFamInit, 0.0, (double)B * sizeof(double2));
                if (df) rq::launch_init_unit_df64(ctx->d_psi + slot0 * tile, cols, B, ctx->log2B, ctx->n_store, s);
                else rq::launch_init_unit(ctx->d_psi + slot0 * tile, cols, B, ctx->log2B, ctx->n_store, ctx->structure, s);
            }
            RQ_LAUNCHED();
            for (int d = 0; d < kd; ++d)
                RQ_CUDA(cudaMemsetAsync(ctx->d_dpsi + d * set + slot0 * tile, 0, sizeof(double2) * tile, s));
            // forward pass
            long long final_slot = g;
            if (fused) {
                // in execution order; slot p holds the state before position p
                for (const auto &pp : ctx->plan) {
                    if (pp.m == 1) {
                        RQ_TRY(fwd(ctx->order[pp.pos], pp.pos, pp.pos + 1));
                        continue;
                    }
                    rq::FwdFusedArgs fa{};
                    fa.psi_in = ctx->d_psi + (long long)pp.pos * tile;
                    fa.dpsi_in = ctx->d_dpsi + (long long)pp.pos * tile;
                    fa.psi_base = ctx->d_psi;
                    fa.dpsi_base = ctx->d_dpsi;
                    fa.tile = tile;
                    fa.dir_stride = set;
                    fa.kdirs = kd;
                    fa.mode = ctx->structure == 1 ? rq::kParity4 : rq::kGeneral;
                    fa.gates = gsrc;
                    fa.dirs = dsrc + (long long)d0 * P * 16;
                    fa.xdir_stride = (long long)P * 16;
                    fa.log2B = ctx->log2B;
                    fa.log2chunks = ctx->log2B - 5;
                    const int q = __builtin_popcountll(pp.wmask);
                    fa.n_blocks = (ctx->n_store >> q) << fa.log2chunks;
                    fa.outer_mask = (ctx->n_store - 1) & ~pp.wmask;
                    fa.pass.m = pp.m;
                    fa.pass.q = q;
                    fa.pass.wmask = pp.wmask;
                    double flops = 0.0;
                    for (int j = 0; j < pp.m; ++j) {
                        const GateGeom &geo = ctx->geo[ctx->order[pp.pos + j]];
                        int la = 0, lb = 0;
                        for (int b = 0, i = 0; b < 63; ++b) {
                            if (!((pp.wmask >> b) & 1)) continue;
                            if (b == geo.pa) la = i;
                            if (b == geo.pb) lb = i;
                            ++i;
                        }
                        fa.pass.la[j] = la;
                        fa.pass.lb[j] = lb;
                        fa.pass.param[j] = geo.param;
                        // every state is a checkpoint when the backward pass
                        // needs it; otherwise only the pass's output
                        fa.pass.out_slot[j] = (backward || j == pp.m - 1) ? pp.pos + j + 1 : -1;
                        const double cm = geo.mode == rq::kGeneral ? 16.0 : 8.0;
                        flops += (double)(ctx->n_store / 4) * B * 8.0 * cm * (1 + 2 * kd);
                    }
                    {
                        const double writes = backward ? pp.m : 1;
                        ProfScope ps(ctx, kFamFwd, flops,
                                     (double)tile * sizeof(double2) * (1 + kd) * (1.0 + writes));
                        const long long blocks = fa.n_blocks;
                        const int grid = (int)std::min<long long>(blocks, (long long)ctx->sms * 2);
                        const cudaError_t le = df ? rq::launch_fwd_fused_df64(fa, grid, s)
                                                  : rq::launch_fwd_fused(fa, grid, s);
                        if (le != cudaSuccess) return fail(ctx, RQ_ECUDA, "fused forward pass: %s", cudaGetErrorString(le));
                    }
                    RQ_LAUNCHED();
                }
            } else if (r == 1) {
                for (int l = 0; l < g; ++l) RQ_TRY(fwd(l, l, l + 1));
            } else {
                int prev_len = 0;
                for (int sg = 0; sg < nseg; ++sg) {
                    const int base = sg * r, len = std::min(r, g - base);
                    if (sg > 0) RQ_TRY(copy_slot(nseg + prev_len, nseg));
                    RQ_TRY(copy_slot(nseg, sg));  // checkpoint of the segment start
                    for (int i = 0; i < len; ++i) RQ_TRY(fwd(base + i, nseg + i, nseg + i + 1));
                    prev_len = len;
                }
                final_slot = nseg + prev_len;
            }
            // adjoint start lambda_g = U|j> and the cost summands
            RQ_CUDA(cudaMemsetAsync(ctx->d_lam, 0, sizeof(double2) * tile, s));
            {
                ProfScope ps(ctx, kFamTarget, 0.0, 0.0);
                if (df)
                    rq::launch_scatter_target_df64(target_dev(ctx), cols, wts, B, ctx->log2B, ctx->structure, ctx->n,
                                                   ctx->d_lam, ctx->d_psi + final_slot * tile, ctx->d_fpart, s);
                else
                    rq::launch_scatter_target(target_dev(ctx), cols, wts, B, ctx->log2B, ctx->structure, ctx->n,
                                              ctx->d_lam, ctx->d_psi + final_slot * tile, ctx->d_fpart, s);
            }
            RQ_LAUNCHED();
            if (first) {
                {
                    ProfScope ps(ctx, kFamReduce, 0.0, (double)B * sizeof(double));
                    rq::launch_reduce_f(ctx->d_fpart, B, ctx->d_facc, s);
                }
                RQ_LAUNCHED();
            }
            if (!backward) continue;
            for (int d = 0; d < kd; ++d) RQ_CUDA(cudaMemsetAsync(ctx->d_dlam + d * tile, 0, sizeof(double2) * tile, s));
            const bool acc_env = want_env && first;
            // backward step of gate l, at position pos of the execution order,
            // with the state before it (and its tangents) in slot sl
            auto bwd = [&](int l, long long sl, int pos) -> rq_status {
                const GateGeom &geo = ctx->geo[l];
                rq::BwdArgs a;
                a.lam = ctx->d_lam;
                a.psi = ctx->d_psi + sl * tile;
                a.gate = gsrc + (long long)geo.param * 16;
                a.geo = geo;
                a.log2B = ctx->log2B;
                a.tile_parity = par;
                a.update = pos > 0 ? 1 : 0;
                a.n_items = (geo.mode == rq::kParity2 ? ctx->n_store / 2 : ctx->n_store / 4) * B;
                if (geo.restricted && first_layer) {
                    // E_l needs only the items where psi_{l-1} can be nonzero,
                    // and lambda_{l-1} is read only there by the earlier gates
                    a.cols = cols;
                    a.n_items = (long long)B << __builtin_popcountll(geo.free_bits);
                }
                for (int d = 0; d < kd; ++d) {
                    rq::BwdArgs b = a;
                    b.dlam = ctx->d_dlam + d * tile;
                    b.dpsi = ctx->d_dpsi + d * set + sl * tile;
                    b.dir = dsrc + ((long long)(d0 + d) * P + geo.param) * 16;
                    b.accumulate = 1;
                    b.part = ctx->d_partd + ((long long)d * g + l) * ctx->ncta * rq::kEnvDoubles;
                    {
                        const double amps = geo.mode == rq::kParity2 ? 2.0 : 4.0;
                        const double cm = geo.mode == rq::kGeneral ? 16.0 : (geo.mode == rq::kParity4 ? 8.0 : 4.0);
                        ProfScope ps(ctx, kFamBwdDir, (double)b.n_items * 8.0 * cm * (2 + 2 * b.update),
                                     (double)b.n_items * amps * sizeof(double2) * (4 + b.update));
                        if (df) rq::launch_bwd_dir_df64(b, ctx->ncta, s);
                        else rq::launch_bwd_dir(b, ctx->ncta, s);
                    }
                    RQ_LAUNCHED();
                }
                if (pos > 0 || acc_env) {
                    a.dlam = nullptr;
                    a.dpsi = nullptr;
                    a.dir = nullptr;
                    a.accumulate = acc_env ? 1 : 0;
                    a.part = ctx->d_part + (long long)l * ctx->ncta * rq::kEnvDoubles;
                    {
                        const double amps = geo.mode == rq::kParity2 ? 2.0 : 4.0;
                        const double cm = geo.mode == rq::kGeneral ? 16.0 : (geo.mode == rq::kParity4 ? 8.0 : 4.0);
                        ProfScope ps(ctx, kFamBwdBase, (double)a.n_items * 8.0 * cm * (a.accumulate + a.update),
                                     (double)a.n_items * amps * sizeof(double2) * (1 + a.accumulate + a.update));
                        if (df) rq::launch_bwd_base_df64(a, ctx->ncta, s);
                        else rq::launch_bwd_base(a, ctx->ncta, s);
                    }
                    RQ_LAUNCHED();
                }
                return RQ_OK;
            };
            if (fused) {
                for (int pos = g - 1; pos >= 0; --pos) RQ_TRY(bwd(ctx->order[pos], pos, pos));
            } else if (r == 1) {
                for (int l = g - 1; l >= 0; --l) RQ_TRY(bwd(l, l, l));
            } else {
                for (int sg = nseg - 1; sg >= 0; --sg) {
                    const int base = sg * r, len = std::min(r, g - base);
                    if (sg < nseg - 1) {  // recompute the segment from its checkpoint
                        RQ_TRY(copy_slot(sg, nseg));
                        for (int i = 0; i < len; ++i) RQ_TRY(fwd(base + i, nseg + i, nseg + i + 1));
                    }
                    for (int l = base + len - 1; l >= base; --l) RQ_TRY(bwd(l, nseg + (l - base), l));
                }
            }
            if (acc_env) {
                {
                    ProfScope ps(ctx, kFamReduce, 0.0, (double)g * ctx->ncta * rq::kEnvDoubles * sizeof(double));
                    rq::launch_reduce_env(ctx->d_part, ctx->ncta, g, ctx->d_env, s);
                }
                RQ_LAUNCHED();
            }
            for (int d = 0; d < kd; ++d) {
                {
                    ProfScope ps(ctx, kFamReduce, 0.0, (double)g * ctx->ncta * rq::kEnvDoubles * sizeof(double));
                    rq::launch_reduce_env(ctx->d_partd + (long long)d * g * ctx->ncta * rq::kEnvDoubles, ctx->ncta, g,
                                          ctx->d_envd + (long long)(d0 + d) * g * rq::kEnvDoubles, s);
                }
                RQ_LAUNCHED();
            }
        }
    }
    {
        ProfScope ps(ctx, kFamGeometry, 0.0, 0.0);
        rq::launch_geometry(ctx->d_gates, ctx->d_dirs, ctx->d_env, ctx->d_envd, ctx->d_param_of, g, P, k,
                            ctx->structure, ctx->space, ctx->d_facc, f_out,
                            want_env ? reinterpret_cast<double2 *>(rgrad) : nullptr,
                            reinterpret_cast<double2 *>(hvps), s);
    }
    RQ_LAUNCHED();
    return RQ_OK;
}

}  // namespace

namespace rq {

// Gate validation (rq_set_checks): every parameter gate finite and unitary,
// ||G^H G - I||_F <= 1e-10, and for parity gates no entry above 1e-10 outside
// the parity pattern (the library masks to the pattern; a large entry there
// means the caller's gates are not the parity gates it declared).
rq_status check_gates(rq_ctx *ctx, const double *gates) {
    if (!ctx->checks) return RQ_OK;
    for (int p = 0; p < ctx->P; ++p) {
        const double *G = gates + (long long)p * 32;
        for (int i = 0; i < 32; ++i)
            if (!std::isfinite(G[i])) return fail(ctx, RQ_EINVAL, "gate %d has a non-finite entry", p);
        double dev2 = 0.0, off = 0.0;
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                double re = a == b ? -1.0 : 0.0, im = 0.0;  // (G^H G)[a][b] - I[a][b]
                for (int r = 0; r < 4; ++r) {
                    const double xr = G[2 * (r * 4 + a)], xi = G[2 * (r * 4 + a) + 1];
                    const double yr = G[2 * (r * 4 + b)], yi = G[2 * (r * 4 + b) + 1];
                    re += xr * yr + xi * yi;
                    im += xr * yi - xi * yr;
                }
                dev2 += re * re + im * im;
                if (ctx->structure == 1 && ((__builtin_popcount(a) ^ __builtin_popcount(b)) & 1))
                    off = std::max(off, std::hypot(G[2 * (a * 4 + b)], G[2 * (a * 4 + b) + 1]));
            }
        if (std::sqrt(dev2) > 1e-10)
            return fail(ctx, RQ_EINVAL, "gate %d is not unitary: ||G^H G - I||_F = %.3e", p, std::sqrt(dev2));
        if (off > 1e-10)
            return fail(ctx, RQ_EINVAL, "parity gate %d has an entry of size %.3e outside the parity pattern", p, off);
    }
    return RQ_OK;
}

rq_status check_gates_device(rq_ctx *ctx, const double *d_gates) {
    if (!ctx->checks) return RQ_OK;
    if (!d_gates) return RQ_OK;  // the entry point reports the NULL
    std::vector<double> h((size_t)ctx->P * 32);
    RQ_CUDA(cudaMemcpyAsync(h.data(), d_gates, h.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    RQ_CUDA(cudaStreamSynchronize(ctx->stream));
    return check_gates(ctx, h.data());
}

// Host-memory evaluation shared by the host entry points and the trust
// region: inputs are copied in, outputs copied out, then the stream is
// synchronised.
rq_status eval_host(rq_ctx *ctx, const double *gates, const double *dirs, int k, int want_env, double *f,
                    double *rgrad, double *hvps) {
    if (!ctx) return RQ_EINVAL;
    if (!ctx->ready) return fail(ctx, RQ_ESTATE, "no target set up (call rq_setup_target first)");
    if (!gates) return fail(ctx, RQ_EINVAL, "gates is NULL");
    if (k < 0) return fail(ctx, RQ_EINVAL, "k = %d < 0", k);
    if (k > 0 && !dirs) return fail(ctx, RQ_EINVAL, "dirs is NULL with k = %d", k);
    RQ_TRY(check_gates(ctx, gates));
    RQ_TRY(ensure_small(ctx, k));
    cudaStream_t s = ctx->stream;
    const long long gsz = (long long)ctx->P * 32;
    RQ_CUDA(cudaMemcpyAsync(ctx->d_in_gates, gates, sizeof(double) * gsz, cudaMemcpyHostToDevice, s));
    if (k > 0) RQ_CUDA(cudaMemcpyAsync(ctx->d_dirs_raw, dirs, sizeof(double) * gsz * k, cudaMemcpyHostToDevice, s));
    double *o_f = ctx->d_out, *o_g = ctx->d_out + 2, *o_h = ctx->d_out + 2 + gsz;
    const double *i_g = reinterpret_cast<const double *>(ctx->d_in_gates);
    const double *i_d = reinterpret_cast<const double *>(ctx->d_dirs_raw);
    if (ctx->use_graphs && !ctx->prof_on) {
        // the whole evaluation is captured once per (k, env_mode) and replayed
        // as one graph launch while the configuration is unchanged
        rq_ctx::GraphEntry *hit = nullptr;
        for (auto &e : ctx->graphs) {
            if (e.exec && e.version != ctx->version) {
                cudaGraphExecDestroy(e.exec);
                e = rq_ctx::GraphEntry{};
            }
            if (e.exec && e.k == k && e.env == want_env) hit = &e;
        }
        if (!hit) {
            rq_ctx::GraphEntry *slot = nullptr;
            for (auto &e : ctx->graphs)
                if (!e.exec) slot = &e;
            if (!slot && ctx->graphs.size() < 4) {
                ctx->graphs.emplace_back();
                slot = &ctx->graphs.back();
            }
            if (!slot) {  // evict the least recently used entry
                slot = &ctx->graphs[0];
                for (auto &e : ctx->graphs)
                    if (e.last_use < slot->last_use) slot = &e;
                cudaGraphExecDestroy(slot->exec);
                *slot = rq_ctx::GraphEntry{};
            }
            const long long before = ctx->launches;
            if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                // a stream that cannot be captured (the legacy default stream,
                // or one already capturing): launch directly from now on
                cudaGetLastError();
                ctx->use_graphs = false;
                RQ_TRY(eval_dev(ctx, i_g, i_d, k, want_env, o_f, o_g, o_h));
                goto copy_out;
            }
            const rq_status st = eval_dev(ctx, i_g, i_d, k, want_env, o_f, o_g, o_h);
            cudaGraph_t graph = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(s, &graph);
            if (st != RQ_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (ce != cudaSuccess) return fail(ctx, RQ_ECUDA, "evaluation capture: %s", cudaGetErrorString(ce));
            const cudaError_t ie = cudaGraphInstantiate(&slot->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) {
                slot->exec = nullptr;
                return fail(ctx, RQ_ECUDA, "graph instantiation: %s", cudaGetErrorString(ie));
            }
            slot->k = k;
            slot->env = want_env;
            slot->version = ctx->version;
            slot->launches = ctx->launches - before;
            ctx->launches = before;  // captured, not yet launched
            hit = slot;
        }
        hit->last_use = ++ctx->graph_clock;
        RQ_CUDA(cudaGraphLaunch(hit->exec, s));
        ctx->launches += hit->launches;
    } else {
        RQ_TRY(eval_dev(ctx, i_g, i_d, k, want_env, o_f, o_g, o_h));
    }
copy_out:
    if (f) RQ_CUDA(cudaMemcpyAsync(f, o_f, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (rgrad && want_env == 1) RQ_CUDA(cudaMemcpyAsync(rgrad, o_g, sizeof(double) * gsz, cudaMemcpyDeviceToHost, s));
    if (hvps && k > 0) RQ_CUDA(cudaMemcpyAsync(hvps, o_h, sizeof(double) * gsz * k, cudaMemcpyDeviceToHost, s));
    RQ_CUDA(cudaStreamSynchronize(s));
    return RQ_OK;
}

rq_status set_error(rq_ctx *ctx, rq_status code, const char *msg) { return fail(ctx, code, "%s", msg); }

int gradient_space(const rq_ctx *ctx) { return ctx->space; }

rq_status eval_device(rq_ctx *ctx, const double *gates, const double *dirs, int k, int env_mode, double *f,
                      double *rgrad, double *hvps) {
    return eval_dev(ctx, gates, dirs, k, env_mode, f, rgrad, hvps);
}

rq_status prepare_capacity(rq_ctx *ctx, int k) { return ensure_small(ctx, k); }

cudaStream_t ctx_stream(const rq_ctx *ctx) { return ctx->stream; }

long long workspace_bytes_for(const rq_ctx *ctx, int columns_per_tile, int kc) {
    return (long long)columns_per_tile * bytes_per_column(ctx, kc);
}

CtxView ctx_view(const rq_ctx *ctx) {
    CtxView v{};
    v.ready = ctx->ready;
    v.device = ctx->device;
    v.n = ctx->n;
    v.g = ctx->g;
    v.P = ctx->P;
    v.structure = ctx->structure;
    v.sms = ctx->sms;
    v.n_store = ctx->n_store;
    v.c0 = ctx->c0;
    v.c1 = ctx->c1;
    v.geo = ctx->geo.data();
    v.stream = ctx->stream;
    v.target = target_dev(ctx);
    return v;
}

}  // namespace rq

// ------------------------------------------------------------------ C ABI --

extern "C" {

rq_status rq_create(rq_ctx **out, int device, void *cuda_stream) {
    if (!out) return fail(nullptr, RQ_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev)
        return fail(nullptr, RQ_ECUDA, "device %d unavailable (%d devices): %s", device, ndev,
                    cudaGetErrorString(e));
    if ((e = cudaSetDevice(device)) != cudaSuccess)
        return fail(nullptr, RQ_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    if ((e = rq::init_sweep_attributes()) != cudaSuccess || (e = rq::init_sweep_attributes_df64()) != cudaSuccess)
        return fail(nullptr, RQ_ECUDA, "kernel attributes: %s", cudaGetErrorString(e));
    rq_ctx *ctx = new rq_ctx();
    ctx->device = device;
    cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device);
    if (cuda_stream) {
        ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    } else {
        if ((e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking)) != cudaSuccess) {
            delete ctx;
            return fail(nullptr, RQ_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        }
        ctx->own_stream = true;
    }
    *out = ctx;
    return RQ_OK;
}

rq_status rq_destroy(rq_ctx *ctx) {
    if (!ctx) return RQ_OK;
    cudaSetDevice(ctx->device);
    free_problem(ctx);
    for (auto &r : ctx->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return RQ_OK;
}

rq_status rq_setup_target(rq_ctx *ctx, const rq_target *tgt, const rq_circuit *c) {
    if (!ctx) return RQ_EINVAL;
    if (!tgt || !c) return fail(ctx, RQ_EINVAL, "target or circuit is NULL");
    if (tgt->model < 0 || tgt->model > 2)
        return fail(ctx, RQ_EINVAL, "model %d not supported (0 spinful, 1 spinless Fermi-Hubbard, 2 dense)",
                    tgt->model);
    if (tgt->model == 2) {
        if (!tgt->dense_U) return fail(ctx, RQ_EINVAL, "model 2 needs dense_U");
        if (c->n_qubits < 2 || c->n_qubits > rq::kMaxDenseQubits)
            return fail(ctx, RQ_EINVAL, "model 2: n_qubits %d must be in [2, %d]", c->n_qubits, rq::kMaxDenseQubits);
        const long long entries = 2LL << (2 * c->n_qubits);
        for (long long i = 0; i < entries; ++i)
            if (!std::isfinite(tgt->dense_U[i])) return fail(ctx, RQ_EINVAL, "dense_U has a non-finite entry");
    } else {
        const int per_site = tgt->model == 0 ? 2 : 1;
        if (tgt->n_sites < 1 || per_site * tgt->n_sites != c->n_qubits || c->n_qubits < 2 ||
            c->n_qubits > rq::kMaxQubits)
            return fail(ctx, RQ_EINVAL, "n_qubits %d must equal %d * n_sites (%d), be >= 2 and <= %d", c->n_qubits,
                        per_site, tgt->n_sites, rq::kMaxQubits);
        if (!std::isfinite(tgt->J) || !std::isfinite(tgt->U) || !std::isfinite(tgt->t))
            return fail(ctx, RQ_EINVAL, "J, U, t must be finite");
    }
    if (c->n_gates < 1 || !c->pairs) return fail(ctx, RQ_EINVAL, "circuit needs n_gates >= 1 and pairs");
    if (c->structure != 0 && c->structure != 1) return fail(ctx, RQ_EINVAL, "structure must be 0 or 1");
    const int P = c->param_of ? c->n_params : c->n_gates;
    if (P < 1) return fail(ctx, RQ_EINVAL, "n_params must be >= 1");
    for (int l = 0; l < c->n_gates; ++l) {
        const int a = c->pairs[2 * l], b = c->pairs[2 * l + 1];
        if (a < 0 || b < 0 || a >= c->n_qubits || b >= c->n_qubits || a == b)
            return fail(ctx, RQ_EINVAL, "gate %d: invalid qubit pair (%d, %d)", l, a, b);
        if (c->param_of && (c->param_of[l] < 0 || c->param_of[l] >= P))
            return fail(ctx, RQ_EINVAL, "gate %d: param_of %d outside [0, %d)", l, c->param_of[l], P);
    }
    RQ_CUDA(cudaSetDevice(ctx->device));
    free_problem(ctx);
    ctx->tgt = *tgt;
    ctx->tgt.dense_U = nullptr;  // copied into the device blocks below; the caller keeps ownership
    ctx->n = c->n_qubits;
    ctx->L = tgt->model == 2 ? 0 : tgt->n_sites;
    ctx->g = c->n_gates;
    ctx->P = P;
    ctx->structure = c->structure;
    ctx->pairs.assign(c->pairs, c->pairs + 2 * ctx->g);
    ctx->param_of.resize(ctx->g);
    for (int l = 0; l < ctx->g; ++l) ctx->param_of[l] = c->param_of ? c->param_of[l] : l;
    ctx->n_store = ctx->structure == 1 ? (1LL << (ctx->n - 1)) : (1LL << ctx->n);
    // every field of every gate is reset: a previous problem's first-layer
    // masks must not survive into this one
    ctx->geo.assign(ctx->g, GateGeom{});
    for (int l = 0; l < ctx->g; ++l) {
        const int a = ctx->pairs[2 * l], b = ctx->pairs[2 * l + 1], n = ctx->n;
        GateGeom &gg = ctx->geo[l];
        gg.param = ctx->param_of[l];
        gg.qfirst = 0;
        if (ctx->structure == 0 || (a != 0 && b != 0)) {
            gg.mode = ctx->structure == 0 ? rq::kGeneral : rq::kParity4;
            gg.pa = n - 1 - a;
            gg.pb = n - 1 - b;
        } else {
            const int q = a == 0 ? b : a;
            gg.mode = rq::kParity2;
            gg.pa = n - 1 - q;
            gg.pb = -1;
            gg.qfirst = a != 0 ? 1 : 0;
        }
    }
    // The leading run of pairwise disjoint gates acts on a basis state: before
    // gate l of the run only the qubits of the earlier gates of the run can
    // differ from the column's basis state (bit masks in stored coordinates;
    // the implied qubit of the parity layout has no stored bit).  Gates on two
    // stored qubits then sweep only those items; a parity gate on the implied
    // qubit sweeps all of its (two-amplitude) items.
    {
        const long long all = ctx->n_store - 1;
        long long used = 0;
        for (int l = 0; l < ctx->g; ++l) {
            GateGeom &gg = ctx->geo[l];
            const long long bits = gg.mode == rq::kParity2 ? (1LL << gg.pa) : (1LL << gg.pa) | (1LL << gg.pb);
            if (used & bits) break;
            if (gg.mode != rq::kParity2) {
                gg.free_bits = used;
                gg.fixed_bits = all & ~(used | bits);
                gg.restricted = gg.fixed_bits != 0;
            }
            used |= bits;
        }
    }
    rq_status st = tgt->model == 2 ? build_target_dense(ctx, tgt->dense_U) : build_target(ctx);
    if (st != RQ_OK) {
        free_problem(ctx);
        return st;
    }
    st = dev_alloc(ctx, &ctx->d_env, (long long)ctx->g * rq::kEnvDoubles, ctx->small_bytes);
    if (st == RQ_OK) st = dev_alloc(ctx, &ctx->d_facc, 1, ctx->small_bytes);
    if (st == RQ_OK) st = dev_alloc(ctx, &ctx->d_gates, (long long)P * 16, ctx->small_bytes);
    if (st == RQ_OK) st = dev_alloc(ctx, &ctx->d_in_gates, (long long)P * 16, ctx->small_bytes);
    if (st == RQ_OK) st = dev_alloc(ctx, &ctx->d_gates_df, (long long)P * 16, ctx->small_bytes);
    if (st == RQ_OK) st = dev_alloc(ctx, &ctx->d_param_of, ctx->g, ctx->small_bytes);
    if (st == RQ_OK &&
        (cudaMemcpyAsync(ctx->d_param_of, ctx->param_of.data(), ctx->g * sizeof(int32_t), cudaMemcpyHostToDevice,
                         ctx->stream) != cudaSuccess ||
         cudaStreamSynchronize(ctx->stream) != cudaSuccess))
        st = fail(ctx, RQ_ECUDA, "copy of param_of failed");
    plan_passes(ctx);
    ctx->c0 = 0;
    ctx->c1 = 1LL << ctx->n;
    ctx->tshift = 0;
    ctx->ckpt_r = 1;
    ctx->ckpt_req = 0;
    ctx->reps.clear();
    ctx->rep_w.clear();
    ctx->ready = true;
    if (st == RQ_OK) st = ensure_small(ctx, 1);
    if (st == RQ_OK) st = rebuild_tiles(ctx);
    if (st != RQ_OK) free_problem(ctx);
    return st;
}

rq_status rq_set_columns(rq_ctx *ctx, int64_t col_begin, int64_t col_end) {
    if (!ctx) return RQ_EINVAL;
    if (!ctx->ready) return fail(ctx, RQ_ESTATE, "no target set up");
    if (col_begin < 0 || col_end < col_begin || col_end > (1LL << ctx->n))
        return fail(ctx, RQ_EINVAL, "column range [%lld, %lld) outside [0, %lld)", (long long)col_begin,
                    (long long)col_end, 1LL << ctx->n);
    if (ctx->tshift > 0 && (col_begin != 0 || col_end != (1LL << ctx->n)))
        return fail(ctx, RQ_EINVAL, "translation-representative sums cover the whole basis; disable them first");
    ctx->c0 = col_begin;
    ctx->c1 = col_end;
    return rebuild_tiles(ctx);
}

rq_status rq_set_tile(rq_ctx *ctx, int columns_per_tile, int max_dirs) {
    if (!ctx) return RQ_EINVAL;
    if (!ctx->ready) return fail(ctx, RQ_ESTATE, "no target set up");
    if (columns_per_tile < 0 || (columns_per_tile & (columns_per_tile - 1)) != 0 || columns_per_tile > 65536)
        return fail(ctx, RQ_EINVAL, "columns_per_tile %d is not 0 or a power of two <= 65536", columns_per_tile);
    if (max_dirs < 0 || max_dirs > rq::kMaxDirs) return fail(ctx, RQ_EINVAL, "max_dirs %d outside [0, %d]", max_dirs, rq::kMaxDirs);
    ctx->user_B = columns_per_tile;
    ctx->user_kc = max_dirs;
    return rebuild_tiles(ctx);
}

rq_status rq_hessian(rq_ctx *ctx, const double *gates, double *f, double *egrad, double *hess) {
    if (!ctx) return RQ_EINVAL;
    if (!ctx->ready) return fail(ctx, RQ_ESTATE, "no target set up");
    if (!gates || !hess) return fail(ctx, RQ_EINVAL, "gates or hess is NULL");
    if (ctx->ckpt_r != 1)
        return fail(ctx, RQ_EINVAL, "the full Hessian keeps every state, but the workspace keeps one every %d "
                    "gates: set the checkpoint interval to 1 (a smaller tile if memory is short)", ctx->ckpt_r);
    RQ_TRY(rq::check_gates(ctx, gates));
    RQ_TRY(ensure_small(ctx, 1));
    if (!workspace_ok(ctx))
        return fail(ctx, RQ_ESTATE, "the sweep workspace is not allocated (a previous tile change failed)");
    cudaStream_t s = ctx->stream;
    const int g = ctx->g, P = ctx->P, B = ctx->B;
    const int log2M = ctx->structure == 1 ? 3 : 4, M = 1 << log2M;
    const long long tile = ctx->n_store * B;
    // CTAs of the hole kernels (one thread per item and member, grid M high):
    // one block of items per CTA at most, so small problems launch few CTAs
    const int nh = (int)std::min<long long>((long long)ctx->sms * rq::kCtasPerSm,
                                            std::max<long long>(1, (ctx->n_store / 4 * B + rq::kThreads - 1) / rq::kThreads));
    // temporaries: adjoint checkpoints, two member arrays, partials, block accumulators
    long long tmp_bytes = 0;
    double2 *lamck = nullptr, *arr0 = nullptr, *arr1 = nullptr;
    double *hpart = nullptr, *hacc = nullptr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(s);
        dev_free(lamck);
        dev_free(arr0);
        dev_free(arr1);
        dev_free(hpart);
        dev_free(hacc);
    };
    rq_status st = dev_alloc(ctx, &lamck, tile * g, tmp_bytes);
    if (st == RQ_OK) st = dev_alloc(ctx, &arr0, tile * M, tmp_bytes);
    if (st == RQ_OK) st = dev_alloc(ctx, &arr1, tile * M, tmp_bytes);
    if (st == RQ_OK) st = dev_alloc(ctx, &hpart, (long long)g * M * nh * rq::kEnvDoubles, tmp_bytes);
    if (st == RQ_OK) st = dev_alloc(ctx, &hacc, (long long)g * g * M * rq::kEnvDoubles, tmp_bytes);
    if (st != RQ_OK) {
        cleanup();
        return st;
    }
#define RQH_CUDA(call)                                                                            \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            cleanup();                                                                            \
            return fail(ctx, RQ_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));                 \
        }                                                                                         \
    } while (0)
#define RQH_LAUNCHED() RQH_CUDA((++ctx->launches, cudaGetLastError()))
    RQH_CUDA(cudaMemcpyAsync(ctx->d_in_gates, gates, sizeof(double2) * 16 * P, cudaMemcpyHostToDevice, s));
    rq::launch_mask_gates(ctx->d_in_gates, ctx->d_gates, P, ctx->structure, s);
    RQH_LAUNCHED();
    RQH_CUDA(cudaMemsetAsync(hacc, 0, sizeof(double) * g * g * M * rq::kEnvDoubles, s));
    RQH_CUDA(cudaMemsetAsync(ctx->d_env, 0, sizeof(double) * g * rq::kEnvDoubles, s));
    RQH_CUDA(cudaMemsetAsync(ctx->d_facc, 0, sizeof(double), s));
    for (int ti = 0; ti < ctx->n_tiles; ++ti) {
        const int32_t *cols = ctx->d_cols + (long long)ti * B;
        const double *wts = ctx->tshift > 0 ? ctx->d_wts + (long long)ti * B : nullptr;
        const int par = ctx->tile_parity[ti];
        RQH_CUDA(cudaMemsetAsync(ctx->d_psi, 0, sizeof(double2) * tile, s));
        rq::launch_init_unit(ctx->d_psi, cols, B, ctx->log2B, ctx->n_store, ctx->structure, s);
        RQH_LAUNCHED();
        for (int l = 0; l < g; ++l) {  // forward pass with checkpoints
            const GateGeom &geo = ctx->geo[l];
            rq::FwdArgs a{};
            a.psi_in = ctx->d_psi + l * tile;
            a.psi_out = ctx->d_psi + (l + 1) * tile;
            a.kdirs = 0;
            a.gate = ctx->d_gates + (long long)geo.param * 16;
            a.geo = geo;
            a.log2B = ctx->log2B;
            a.tile_parity = par;
            a.n_items = (geo.mode == rq::kParity2 ? ctx->n_store / 2 : ctx->n_store / 4) * B;
            rq::launch_fwd(a, ctx->ncta, s);
            RQH_LAUNCHED();
        }
        RQH_CUDA(cudaMemsetAsync(ctx->d_lam, 0, sizeof(double2) * tile, s));
        rq::launch_scatter_target(target_dev(ctx), cols, wts, B, ctx->log2B, ctx->structure, ctx->n, ctx->d_lam,
                                  ctx->d_psi + g * tile, ctx->d_fpart, s);
        RQH_LAUNCHED();
        rq::launch_reduce_f(ctx->d_fpart, B, ctx->d_facc, s);
        RQH_LAUNCHED();
        for (int l = g - 1; l >= 0; --l) {  // backward pass, keeping every lambda_l
            const GateGeom &geo = ctx->geo[l];
            RQH_CUDA(cudaMemcpyAsync(lamck + l * tile, ctx->d_lam, sizeof(double2) * tile, cudaMemcpyDeviceToDevice, s));
            rq::BwdArgs a{};
            a.lam = ctx->d_lam;
            a.psi = ctx->d_psi + l * tile;
            a.gate = ctx->d_gates + (long long)geo.param * 16;
            a.geo = geo;
            a.log2B = ctx->log2B;
            a.tile_parity = par;
            a.update = l > 0 ? 1 : 0;
            a.accumulate = 1;
            a.n_items = (geo.mode == rq::kParity2 ? ctx->n_store / 2 : ctx->n_store / 4) * B;
            a.part = ctx->d_part + (long long)l * ctx->ncta * rq::kEnvDoubles;
            rq::launch_bwd_base(a, ctx->ncta, s);
            RQH_LAUNCHED();
        }
        rq::launch_reduce_env(ctx->d_part, ctx->ncta, g, ctx->d_env, s);
        RQH_LAUNCHED();
        // second forward passes: hole of gate l, propagated and contracted at every l' > l
        for (int l = 0; l + 1 < g; ++l) {
            const GateGeom &geo = ctx->geo[l];
            const long long items_l = (geo.mode == rq::kParity2 ? ctx->n_store / 2 : ctx->n_store / 4) * B;
            rq::launch_hole_apply(ctx->d_psi + l * tile, arr0, geo, ctx->log2B, log2M, ctx->structure, par, items_l,
                                  nh, s);
            RQH_LAUNCHED();
            double2 *cur = arr0, *nxt = arr1;
            for (int lp = l + 1; lp < g; ++lp) {
                const GateGeom &gp = ctx->geo[lp];
                const long long items = (gp.mode == rq::kParity2 ? ctx->n_store / 2 : ctx->n_store / 4) * B;
                rq::launch_array_env(lamck + lp * tile, cur, gp, ctx->log2B, log2M, par, items, nh,
                                     hpart + (long long)lp * M * nh * rq::kEnvDoubles, s);
                RQH_LAUNCHED();
                if (lp + 1 < g) {
                    rq::FwdArgs a{};
                    a.psi_in = cur;
                    a.psi_out = nxt;
                    a.kdirs = 0;
                    a.gate = ctx->d_gates + (long long)gp.param * 16;
                    a.geo = gp;
                    a.log2B = ctx->log2B + log2M;
                    a.tile_parity = par;
                    a.n_items = items * M;
                    rq::launch_fwd(a, ctx->ncta, s);
                    RQH_LAUNCHED();
                    std::swap(cur, nxt);
                }
            }
            rq::launch_reduce_rows(hpart + (long long)(l + 1) * M * nh * rq::kEnvDoubles, nh,
                                   (long long)(g - 1 - l) * M, hacc + ((long long)l * g + l + 1) * M * rq::kEnvDoubles, s);
            RQH_LAUNCHED();
        }
    }
    // f and the Euclidean gradient (masked), then the blocks to the host
    const int saved_space = ctx->space;
    ctx->space = 1;
    rq::launch_geometry(ctx->d_gates, ctx->d_dirs, ctx->d_env, ctx->d_envd, ctx->d_param_of, g, P, 0, ctx->structure,
                        1, ctx->d_facc, ctx->d_out, reinterpret_cast<double2 *>(ctx->d_out + 2), nullptr, s);
    ctx->space = saved_space;
    RQH_LAUNCHED();
    std::vector<double> hb((size_t)g * g * M * rq::kEnvDoubles);
    double fh = 0.0;
    std::vector<double> eg((size_t)P * 32);
    RQH_CUDA(cudaMemcpyAsync(hb.data(), hacc, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, s));
    RQH_CUDA(cudaMemcpyAsync(&fh, ctx->d_out, sizeof(double), cudaMemcpyDeviceToHost, s));
    RQH_CUDA(cudaMemcpyAsync(eg.data(), ctx->d_out + 2, sizeof(double) * eg.size(), cudaMemcpyDeviceToHost, s));
    RQH_CUDA(cudaStreamSynchronize(s));
#undef RQH_LAUNCHED
#undef RQH_CUDA
    cleanup();
    if (f) *f = fh;
    if (egrad) std::memcpy(egrad, eg.data(), sizeof(double) * eg.size());
    // tied, symmetric assembly: H[p(l) ab][p(l') cd] += block and its transpose
    static const int members[2][16][2] = {
        {{0, 0}, {0, 1}, {0, 2}, {0, 3}, {1, 0}, {1, 1}, {1, 2}, {1, 3},
         {2, 0}, {2, 1}, {2, 2}, {2, 3}, {3, 0}, {3, 1}, {3, 2}, {3, 3}},
        {{0, 0}, {0, 3}, {3, 0}, {3, 3}, {1, 1}, {1, 2}, {2, 1}, {2, 2},
         {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}}};
    const long long D = (long long)P * 16;
    std::memset(hess, 0, sizeof(double) * 2 * D * D);
    for (int l = 0; l < g; ++l)
        for (int lp = l + 1; lp < g; ++lp)
            for (int m = 0; m < M; ++m) {
                const double *blk = hb.data() + (((long long)l * g + lp) * M + m) * rq::kEnvDoubles;
                const long long row = (long long)ctx->param_of[l] * 16 + members[ctx->structure][m][0] * 4 +
                                      members[ctx->structure][m][1];
                for (int cd = 0; cd < 16; ++cd) {
                    const long long col = (long long)ctx->param_of[lp] * 16 + cd;
                    hess[2 * (row * D + col)] += blk[2 * cd];
                    hess[2 * (row * D + col) + 1] += blk[2 * cd + 1];
                    hess[2 * (col * D + row)] += blk[2 * cd];
                    hess[2 * (col * D + row) + 1] += blk[2 * cd + 1];
                }
            }
    return RQ_OK;
}

rq_status rq_set_translation(rq_ctx *ctx, int shift_sites) {
    if (!ctx) return RQ_EINVAL;
    if (!ctx->ready) return fail(ctx, RQ_ESTATE, "no target set up");
    const int L = ctx->L, n = ctx->n;
    if (shift_sites == 0) {
        ctx->tshift = 0;
        ctx->reps.clear();
        ctx->rep_w.clear();
        return rebuild_tiles(ctx);
    }
    if (shift_sites < 0 || shift_sites >= L || L % shift_sites != 0)
        return fail(ctx, RQ_EINVAL, "shift %d must divide the %d sites and be smaller", shift_sites, L);
    if (ctx->tgt.model == 2 || !ctx->tgt.periodic)
        return fail(ctx, RQ_EINVAL, "translation symmetry needs a periodic chain model");
    // qubit map of the shift: site j -> j + s (mod L) on every chain
    std::vector<int> qmap(n);
    for (int q = 0; q < n; ++q) qmap[q] = (q < L) ? (q + shift_sites) % L : L + (q - L + shift_sites) % L;
    // the circuit must be invariant: in every maximal run of pairwise disjoint
    // (hence commuting) gates, the set of (pair, parameter) maps onto itself
    size_t l0 = 0;
    while (l0 < (size_t)ctx->g) {
        size_t l1 = l0;
        unsigned long long used = 0;
        while (l1 < (size_t)ctx->g) {
            const unsigned long long m = (1ULL << ctx->pairs[2 * l1]) | (1ULL << ctx->pairs[2 * l1 + 1]);
            if (used & m) break;
            used |= m;
            ++l1;
        }
        for (size_t l = l0; l < l1; ++l) {
            const int a = qmap[ctx->pairs[2 * l]], b = qmap[ctx->pairs[2 * l + 1]];
            bool found = false;
            for (size_t m2 = l0; m2 < l1 && !found; ++m2)
                found = ctx->pairs[2 * m2] == a && ctx->pairs[2 * m2 + 1] == b && ctx->param_of[m2] == ctx->param_of[l];
            if (!found)
                return fail(ctx, RQ_EINVAL, "gate %zu on (%d, %d) has no shifted copy in its layer: the circuit is "
                            "not invariant under a shift by %d sites", l, ctx->pairs[2 * l], ctx->pairs[2 * l + 1],
                            shift_sites);
        }
        l0 = l1;
    }
    if (ctx->c0 != 0 || ctx->c1 != (1LL << n))
        return fail(ctx, RQ_EINVAL, "translation-representative sums need the whole basis as the column range");
    // orbits of the basis under the shift: smallest member represents, weight = orbit size
    const long long dim = 1LL << n;
    std::vector<char> seen(dim, 0);
    ctx->reps.clear();
    ctx->rep_w.clear();
    for (long long x = 0; x < dim; ++x) {
        if (seen[x]) continue;
        long long y = x, size = 0;
        do {
            seen[y] = 1;
            ++size;
            long long z = 0;
            for (int q = 0; q < n; ++q)
                if ((y >> (n - 1 - q)) & 1) z |= 1LL << (n - 1 - qmap[q]);
            y = z;
        } while (y != x);
        ctx->reps.push_back((int32_t)x);
        ctx->rep_w.push_back((double)size);
    }
    ctx->tshift = shift_sites;
    return rebuild_tiles(ctx);
}

rq_status rq_set_checkpointing(rq_ctx *ctx, int interval) {
    if (!ctx) return RQ_EINVAL;
    if (!ctx->ready) return fail(ctx, RQ_ESTATE, "no target set up");
    if (interval < 0) return fail(ctx, RQ_EINVAL, "checkpoint interval %d < 0", interval);
    ctx->ckpt_req = interval;
    return rebuild_tiles(ctx);
}

rq_status rq_set_first_layer(rq_ctx *ctx, int enable) {
    if (!ctx) return RQ_EINVAL;
    ctx->first_layer = enable != 0;
    if (ctx->ready) plan_passes(ctx);
    ++ctx->version;
    return RQ_OK;
}

rq_status rq_set_fusion(rq_ctx *ctx, int max_window_qubits) {
    if (!ctx) return RQ_EINVAL;
    if (max_window_qubits != 0 && (max_window_qubits < 3 || max_window_qubits > rq::kMaxWindow))
        return fail(ctx, RQ_EINVAL, "fusion window %d is neither 0 (off) nor in [3, %d]", max_window_qubits,
                    rq::kMaxWindow);
    ctx->fuse_q = max_window_qubits;
    if (ctx->ready) plan_passes(ctx);
    ++ctx->version;
    return RQ_OK;
}

rq_status rq_fusion_info(const rq_ctx *ctx, int *n_passes, int *fused_gates, int *max_pass_gates) {
    if (!ctx) return RQ_EINVAL;
    int np = 0, fg = 0, mx = 0;
    for (const auto &pp : ctx->plan) {
        ++np;
        if (pp.m > 1) fg += pp.m;
        mx = std::max(mx, pp.m);
    }
    if (n_passes) *n_passes = np;
    if (fused_gates) *fused_gates = fg;
    if (max_pass_gates) *max_pass_gates = mx;
    return RQ_OK;
}

rq_status rq_set_checks(rq_ctx *ctx, int enable) {
    if (!ctx) return RQ_EINVAL;
    ctx->checks = enable != 0;
    return RQ_OK;
}

rq_status rq_set_graphs(rq_ctx *ctx, int enable) {
    if (!ctx) return RQ_EINVAL;
    RQ_CUDA(cudaStreamSynchronize(ctx->stream));
    drop_graphs(ctx);
    ctx->use_graphs = enable != 0;
    return RQ_OK;
}

rq_status rq_set_arithmetic(rq_ctx *ctx, int arith) {
    if (!ctx) return RQ_EINVAL;
    if (arith != RQ_ARITH_FP64 && arith != RQ_ARITH_DF64)
        return fail(ctx, RQ_EINVAL, "arithmetic %d is neither RQ_ARITH_FP64 nor RQ_ARITH_DF64", arith);
    ctx->arith = arith;
    ++ctx->version;
    return RQ_OK;
}

rq_status rq_set_gradient_space(rq_ctx *ctx, int space) {
    if (!ctx) return RQ_EINVAL;
    if (space != RQ_SPACE_RIEMANNIAN && space != RQ_SPACE_EUCLIDEAN)
        return fail(ctx, RQ_EINVAL, "space %d is neither RQ_SPACE_RIEMANNIAN nor RQ_SPACE_EUCLIDEAN", space);
    ctx->space = space;
    ++ctx->version;
    return RQ_OK;
}

rq_status rq_cost(rq_ctx *ctx, const double *gates, double *f) {
    if (!ctx) return RQ_EINVAL;
    return rq::eval_host(ctx, gates, nullptr, 0, 0, f, nullptr, nullptr);
}

rq_status rq_grad(rq_ctx *ctx, const double *gates, double *f, double *rgrad) {
    if (!ctx) return RQ_EINVAL;
    return rq::eval_host(ctx, gates, nullptr, 0, 1, f, rgrad, nullptr);
}

rq_status rq_hvp(rq_ctx *ctx, const double *gates, const double *dirs, int k, double *f, double *rgrad,
                 double *hvps) {
    if (!ctx) return RQ_EINVAL;
    return rq::eval_host(ctx, gates, dirs, k, 1, f, rgrad, hvps);
}

rq_status rq_cost_dev(rq_ctx *ctx, const double *gates, double *f) {
    if (!ctx) return RQ_EINVAL;
    RQ_TRY(rq::check_gates_device(ctx, gates));
    return eval_dev(ctx, gates, nullptr, 0, 0, f, nullptr, nullptr);
}

rq_status rq_grad_dev(rq_ctx *ctx, const double *gates, double *f, double *rgrad) {
    if (!ctx) return RQ_EINVAL;
    RQ_TRY(rq::check_gates_device(ctx, gates));
    return eval_dev(ctx, gates, nullptr, 0, 1, f, rgrad, nullptr);
}

rq_status rq_hvp_dev(rq_ctx *ctx, const double *gates, const double *dirs, int k, double *f, double *rgrad,
                     double *hvps) {
    if (!ctx) return RQ_EINVAL;
    RQ_TRY(rq::check_gates_device(ctx, gates));
    return eval_dev(ctx, gates, dirs, k, 1, f, rgrad, hvps);
}

rq_status rq_target_column(rq_ctx *ctx, int64_t j, double *out) {
    if (!ctx) return RQ_EINVAL;
    if (!ctx->ready) return fail(ctx, RQ_ESTATE, "no target set up");
    if (!out || j < 0 || j >= (1LL << ctx->n)) return fail(ctx, RQ_EINVAL, "invalid column %lld", (long long)j);
    const int s = ctx->sec_of_h[j];
    const long long m = ctx->off_basis[s + 1] - ctx->off_basis[s];
    std::vector<double2> col(m);
    RQ_CUDA(cudaStreamSynchronize(ctx->stream));
    RQ_CUDA(cudaMemcpyAsync(col.data(), ctx->d_U + ctx->off_u[s] + (long long)ctx->pos_h[j] * m, m * sizeof(double2),
                            cudaMemcpyDeviceToHost, ctx->stream));
    RQ_CUDA(cudaStreamSynchronize(ctx->stream));
    std::memset(out, 0, sizeof(double) * 2 * (1LL << ctx->n));
    for (long long r = 0; r < m; ++r) {
        const long long x = ctx->basis_h[ctx->off_basis[s] + r];
        out[2 * x] = col[r].x;
        out[2 * x + 1] = col[r].y;
    }
    return RQ_OK;
}

rq_status rq_get_info(const rq_ctx *ctx, rq_info_t *info) {
    if (!ctx || !info) return RQ_EINVAL;
    std::memset(info, 0, sizeof(*info));
    info->kernel_launches = ctx->launches;
    if (!ctx->ready) return RQ_OK;
    info->n_qubits = ctx->n;
    info->n_gates = ctx->g;
    info->n_params = ctx->P;
    info->structure = ctx->structure;
    info->amplitudes_per_column = ctx->n_store;
    info->columns = ctx->c1 - ctx->c0;
    info->columns_per_tile = ctx->B;
    info->n_tiles = ctx->n_tiles;
    info->max_dirs = ctx->kc;
    info->workspace_bytes = ctx->problem_bytes + ctx->work_bytes + ctx->small_bytes;
    info->target_entries = ctx->u_entries;
    return RQ_OK;
}

rq_status rq_profile_start(rq_ctx *ctx) {
    if (!ctx) return RQ_EINVAL;
    ctx->prof_on = true;
    ctx->prof_used = 0;
    ++ctx->version;
    return RQ_OK;
}

rq_status rq_profile_stop(rq_ctx *ctx, rq_kernel_stat *stats, int capacity, int *n_stats) {
    if (!ctx) return RQ_EINVAL;
    ctx->prof_on = false;
    RQ_CUDA(cudaStreamSynchronize(ctx->stream));
    rq_kernel_stat acc[kFamCount];
    for (int i = 0; i < kFamCount; ++i) acc[i] = rq_kernel_stat{kFamilyName[i], 0, 0.0, 0.0, 0.0};
    for (size_t i = 0; i < ctx->prof_used; ++i) {
        const auto &r = ctx->prof[i];
        float ms = 0.0f;
        RQ_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        acc[r.family].launches += 1;
        acc[r.family].total_ms += ms;
        acc[r.family].flops += r.flops;
        acc[r.family].bytes += r.bytes;
    }
    ctx->prof_used = 0;
    int n = 0;
    for (int i = 0; i < kFamCount; ++i) {
        if (acc[i].launches == 0) continue;
        if (stats && n < capacity) stats[n] = acc[i];
        ++n;
    }
    if (n_stats) *n_stats = n;
    return RQ_OK;
}

const char *rq_last_error(const rq_ctx *ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->err.c_str();
}

}  // extern "C"
