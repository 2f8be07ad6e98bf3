// Context lifecycle and configuration: creation, column ranges and tiles,
// the tile workspace, the forward-pass plan (window fusion), profiling and
// the context's info.
#include "rq_context.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

using rq::GateGeom;
using namespace rqc;

namespace rq {
// rq_sweep.cu / rq_sweep_df64.cu: shared-memory limits of the sweep kernels
cudaError_t init_sweep_attributes_df64();
}  // namespace rq

namespace {
thread_local std::string g_create_error;  // text of the last rq_create failure of this thread
}  // namespace

namespace rqc {

const char *const kFamilyName[kFamCount] = {"fwd_gate", "bwd_gate_dir", "bwd_gate_base", "target_scatter_cost",
                                            "init_unit", "reduce", "geometry", "target_chebyshev"};

rq_status fail(rq_ctx *ctx, rq_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf; else g_create_error = buf;
    return code;
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
// support) stays first and unfused; then a pass starts with the next
// remaining gate and adds, one at a time, the later remaining gate that fits
// in the window, commutes with every remaining gate it moves past -- gates on
// disjoint qubits commute (the gates of a brickwall layer, Sec. "Brick wall
// circuit layout") -- and brings the fewest new qubits into the window, up to
// kMaxPassGates gates; the pass keeps the circuit order of its gates.  Parity gates on the implied
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
        std::vector<char> taken(rest.size(), 0);
        taken[0] = 1;
        int m = 1;
        long long W = gate_bits(ctx->geo[g0]);
        // best first: among the remaining gates that commute with every
        // earlier gate not taken, add the one bringing the fewest new bits
        // into the window (earliest on ties), while the window has room
        while (ctx->geo[g0].mode != rq::kParity2 && m < rq::kMaxPassGates) {
            long long blocked = 0;
            int best = -1, best_new = 64;
            for (size_t i = 1; i < rest.size(); ++i) {
                if (taken[i]) continue;
                const GateGeom &gg = ctx->geo[rest[i]];
                const long long b = gate_bits(gg);
                if (gg.mode != rq::kParity2 && !(b & blocked) && __builtin_popcountll(W | b) <= ctx->fuse_q) {
                    const int nb = __builtin_popcountll(b & ~W);
                    if (nb < best_new) {
                        best_new = nb;
                        best = (int)i;
                    }
                }
                blocked |= b;
            }
            if (best < 0) break;
            taken[best] = 1;
            W |= gate_bits(ctx->geo[rest[best]]);
            ++m;
        }
        ctx->plan.push_back({(int)ctx->order.size(), m, W});
        std::vector<int> left;
        for (size_t i = 0; i < rest.size(); ++i) {
            if (taken[i]) ctx->order.push_back(rest[i]);
            else left.push_back(rest[i]);
        }
        rest.swap(left);
    }
    mark_tail(ctx);
}

bool fused_schedule(const rq_ctx *ctx) {
    return ctx->fuse_q > 2 && ctx->ckpt_r == 1 && ctx->B >= 32 && (int)ctx->plan.size() < ctx->g;
}

// Last-layer support: the trailing run of pairwise disjoint gates of the
// order the backward pass walks (the plan's execution order under the fused
// schedule, else the circuit order), which it visits first.  For the gate at
// position pos of the run, the adjoint state it reads differs from U|j> only
// on the qubits of the run's later gates, and U|j> lives in j's particle-
// number sector (spinful chain: up and down counts; spinless chain: one
// count; a dense target has no sectors).  General gates only: parity tiles
// store 2^(n-1) amplitudes without the implied qubit's bit.  Called when the
// plan or the tile configuration (and so the schedule) changes.
void mark_tail(rq_ctx *ctx) {
    for (GateGeom &gg : ctx->geo) {
        gg.tail = 0;
        gg.f_up = gg.f_dn = 0;
        gg.up_out = gg.dn_out = gg.up_mask = gg.dn_mask = 0;
    }
    if (!ctx->last_layer || ctx->structure != 0 || ctx->tgt.model == 2 || (int)ctx->order.size() != ctx->g) return;
    const int n = ctx->n;
    long long upm, dnm;
    if (ctx->tgt.model == 0) {  // qubit q = (site q, up) for q < L, (site q - L, down) after; stored bit n - 1 - q
        upm = ((1LL << ctx->L) - 1) << (n - ctx->L);
        dnm = (1LL << (n - ctx->L)) - 1;
    } else {                    // spinless chain: one particle number over all qubits
        upm = (1LL << n) - 1;
        dnm = 0;
    }
    const bool fused = fused_schedule(ctx);
    long long F = 0;
    for (int pos = ctx->g - 1; pos >= 0; --pos) {
        GateGeom &gg = ctx->geo[fused ? ctx->order[pos] : pos];
        const long long b = gate_bits(gg);
        if (F & b) break;
        F |= b;
        gg.tail = 1;
        gg.up_mask = upm;
        gg.dn_mask = dnm;
        gg.up_out = upm & ~F;
        gg.dn_out = dnm & ~F;
        gg.f_up = __builtin_popcountll(F & upm);
        gg.f_dn = __builtin_popcountll(F & dnm);
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
    // With rq_set_grid(m), at most the CTAs that give every thread m items: a
    // sweep that shares the GPU with other problems' sweeps (a batch, a
    // server) pays its per-CTA set-up and environment reduction fewer times.
    const long long full = (long long)ctx->sms * rq::kCtasPerSm * rq::kThreads;
    int ncta = (int)(items >= full ? (long long)ctx->sms * rq::kCtasPerSm
                                   : std::min<long long>(ctx->sms, (items + 31) / 32));
    if (ctx->grid_items > 0) {
        const long long per_cta = (long long)rq::kThreads * ctx->grid_items;
        ncta = (int)std::max<long long>(1, std::min<long long>(ncta, (items + per_cta - 1) / per_cta));
    }
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
    ctx->cols_h = cols;
    mark_tail(ctx);  // the schedule (fused or not) may have changed with the tile
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

}  // namespace rqc

namespace rq {

rq_status set_error(rq_ctx *ctx, rq_status code, const char *msg) { return fail(ctx, code, "%s", msg); }

int gradient_space(const rq_ctx *ctx) { return ctx->space; }

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

rq_status rq_set_grid(rq_ctx *ctx, int min_items_per_thread) {
    if (!ctx) return RQ_EINVAL;
    if (min_items_per_thread < 0 || min_items_per_thread > (1 << 20))
        return fail(ctx, RQ_EINVAL, "min_items_per_thread %d outside [0, 2^20]", min_items_per_thread);
    ctx->grid_items = min_items_per_thread;
    return ctx->ready ? rebuild_tiles(ctx) : RQ_OK;
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

rq_status rq_set_last_layer(rq_ctx *ctx, int enable) {
    if (!ctx) return RQ_EINVAL;
    ctx->last_layer = enable != 0;
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
    info->ctas_per_sweep = ctx->ncta;
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
