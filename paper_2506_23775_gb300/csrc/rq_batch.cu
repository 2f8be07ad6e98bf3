// Batches of independent circuit-optimisation problems evaluated together.
//
// Every problem of a batch (its own size n, depth, t, U, gates) has its own
// device context and stream.  One evaluation of the whole batch is captured
// once into a CUDA graph: the main stream forks to every problem's stream,
// each problem runs its tile-by-tile sweep there, and the main stream joins
// them.  Replaying the graph is one launch from the host; the GPU runs the
// problems' kernels concurrently, so the many small sweeps of small-n
// problems fill the machine together instead of one after another.  Each
// problem runs exactly the kernels, in exactly the order, of its own context,
// so batched results are bitwise equal to evaluating that problem alone.
//
// The columns-per-tile of every problem is autotuned: candidate tile caps
// that fit the device memory are timed on a captured cost-only evaluation of
// the whole batch and the fastest is kept.  Then the fusion window of the
// forward passes (gates per pass, rq_set_fusion: off, 4, 5 or 6 stored
// qubits) is tuned the same way at that tile, unless the caller fixed it.
// Before that, the sweep grid of the problems (rq_set_grid: 0, 8, 16, 32 or
// 64 items per thread) is tuned on a captured gradient evaluation of the
// batch: the problems' sweeps share the GPU, so each needs fewer CTAs than
// it would alone, and fewer CTAs pay the per-CTA set-up and environment
// reduction fewer times.
#include "rq_internal.h"

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

struct rq_batch {
    int device = 0;
    cudaStream_t main = nullptr;
    std::string err;
    std::vector<rq_ctx *> ctxs;
    std::vector<int> P, n;
    std::vector<long long> goff;   // complex offset of each problem's gates
    long long gtotal = 0;          // sum of n_params * 16
    int tile_cap = 0;              // 0: autotune
    bool tile_fixed = false;       // the caller set the tile (rq_batch_set_tile)
    bool tuned = false;
    double2 *d_gates = nullptr, *d_dirs = nullptr, *d_rgrad = nullptr, *d_hvps = nullptr;
    double *d_f = nullptr;
    int cap_k = -1;
    cudaGraphExec_t exec = nullptr;
    int graph_k = -1, graph_env = -1;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> joins;
    std::vector<double> tune_ms;   // per candidate cap 64, 128, 256, 512 (-1: skipped)
    int fuse_req = -1;             // fusion window for every problem; -1: autotune
    int fuse_q = 0;                // the window in use
    std::vector<double> fuse_ms;   // per candidate window 0, 4, 5, 6 (-1: not timed)
    int grid_req = -1;             // sweep grid (rq_set_grid) of every problem; -1: autotune
    int grid_items = 0;            // the grid in use
    std::vector<double> grid_ms;   // per candidate 0, 8, 16, 32, 64 items per thread (-1: not timed)
};

namespace {

rq_status bfail(rq_batch *b, rq_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    return code;
}

#define RB_CUDA(call)                                                                                  \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return bfail(b, RQ_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

rq_status ctx_fail(rq_batch *b, rq_ctx *c, rq_status st) {
    return bfail(b, st, "%s", rq_last_error(c));
}

int pow2ceil(long long v) {
    int r = 1;
    while (r < v) r <<= 1;
    return r;
}

void drop_graph(rq_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->graph_k = -1;
    b->graph_env = -1;
}

rq_status ensure_buffers(rq_batch *b, int k) {
    if (k <= b->cap_k) return RQ_OK;
    RB_CUDA(cudaStreamSynchronize(b->main));
    cudaFree(b->d_gates);
    cudaFree(b->d_dirs);
    cudaFree(b->d_rgrad);
    cudaFree(b->d_hvps);
    cudaFree(b->d_f);
    b->d_gates = b->d_dirs = b->d_rgrad = b->d_hvps = nullptr;
    b->d_f = nullptr;
    const size_t g = sizeof(double2) * (size_t)b->gtotal, kk = std::max(k, 1);
    if (cudaMalloc(&b->d_gates, g) != cudaSuccess || cudaMalloc(&b->d_rgrad, g) != cudaSuccess ||
        cudaMalloc(&b->d_dirs, g * kk) != cudaSuccess || cudaMalloc(&b->d_hvps, g * kk) != cudaSuccess ||
        cudaMalloc(&b->d_f, sizeof(double) * b->ctxs.size()) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, RQ_ENOMEM, "batch input/output buffers do not fit");
    }
    b->cap_k = k;
    drop_graph(b);
    return RQ_OK;
}

// Queue one evaluation of every problem: concurrently on the problems'
// streams (forked from and joined into the main stream), or one after another.
rq_status enqueue(rq_batch *b, int k, int env_mode, bool plain) {
    const size_t np = b->ctxs.size();
    if (!plain) RB_CUDA(cudaEventRecord(b->fork, b->main));
    cudaStream_t prev = b->main;
    for (size_t p = 0; p < np; ++p) {
        rq_ctx *c = b->ctxs[p];
        cudaStream_t s = rq::ctx_stream(c);
        if (plain) {
            // strictly sequential: wait for the previous problem
            RB_CUDA(cudaEventRecord(b->joins[p], prev));
            RB_CUDA(cudaStreamWaitEvent(s, b->joins[p], 0));
        } else {
            RB_CUDA(cudaStreamWaitEvent(s, b->fork, 0));
        }
        const double *g = reinterpret_cast<const double *>(b->d_gates + b->goff[p]);
        const double *d = reinterpret_cast<const double *>(b->d_dirs + (long long)k * b->goff[p]);
        double *rg = reinterpret_cast<double *>(b->d_rgrad + b->goff[p]);
        double *hv = reinterpret_cast<double *>(b->d_hvps + (long long)k * b->goff[p]);
        const rq_status st = rq::eval_device(c, g, k > 0 ? d : nullptr, k, env_mode, b->d_f + p,
                                             env_mode == 1 ? rg : nullptr, k > 0 ? hv : nullptr);
        if (st != RQ_OK) return ctx_fail(b, c, st);
        if (plain) {
            prev = s;
        } else {
            RB_CUDA(cudaEventRecord(b->joins[p], s));
            RB_CUDA(cudaStreamWaitEvent(b->main, b->joins[p], 0));
        }
    }
    if (plain && np) {
        RB_CUDA(cudaEventRecord(b->joins[np - 1], prev));
        RB_CUDA(cudaStreamWaitEvent(b->main, b->joins[np - 1], 0));
    }
    return RQ_OK;
}

rq_status capture(rq_batch *b, int k, int env_mode) {
    drop_graph(b);
    for (rq_ctx *c : b->ctxs) {
        const rq_status st = rq::prepare_capacity(c, std::max(k, 1));
        if (st != RQ_OK) return ctx_fail(b, c, st);
    }
    RB_CUDA(cudaStreamSynchronize(b->main));
    RB_CUDA(cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal));
    rq_status st = enqueue(b, k, env_mode, false);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->main, &graph);
    if (st != RQ_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return bfail(b, RQ_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    const cudaError_t e2 = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e2 != cudaSuccess) {
        b->exec = nullptr;
        return bfail(b, RQ_ECUDA, "graph instantiation: %s", cudaGetErrorString(e2));
    }
    b->graph_k = k;
    b->graph_env = env_mode;
    return RQ_OK;
}

rq_status apply_cap(rq_batch *b, int cap) {
    for (size_t p = 0; p < b->ctxs.size(); ++p) {
        const int t = std::min(cap, pow2ceil(1LL << b->n[p]));
        const rq_status st = rq_set_tile(b->ctxs[p], t, 1);
        if (st != RQ_OK) return ctx_fail(b, b->ctxs[p], st);
    }
    drop_graph(b);
    return RQ_OK;
}

rq_status apply_grid(rq_batch *b, int m) {
    for (rq_ctx *c : b->ctxs) {
        const rq_status st = rq_set_grid(c, m);
        if (st != RQ_OK) return ctx_fail(b, c, st);
    }
    b->grid_items = m;
    drop_graph(b);
    return RQ_OK;
}

// Capture the evaluation of the given kind and time one replay after a
// warm-up replay.
rq_status time_graph(rq_batch *b, int env_mode, cudaEvent_t e0, cudaEvent_t e1, double &ms_out) {
    rq_status st = capture(b, 0, env_mode);
    if (st != RQ_OK) return st;
    cudaGraphLaunch(b->exec, b->main);  // warm-up
    cudaEventRecord(e0, b->main);
    cudaGraphLaunch(b->exec, b->main);
    cudaEventRecord(e1, b->main);
    if (cudaEventSynchronize(e1) != cudaSuccess)
        return bfail(b, RQ_ECUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ms_out = ms;
    return RQ_OK;
}

rq_status apply_fusion(rq_batch *b, int q) {
    for (rq_ctx *c : b->ctxs) {
        const rq_status st = rq_set_fusion(c, q);
        if (st != RQ_OK) return ctx_fail(b, c, st);
    }
    b->fuse_q = q;
    drop_graph(b);
    return RQ_OK;
}

// Time each feasible tile cap on a captured cost-only evaluation; keep the best.
rq_status autotune(rq_batch *b) {
    const int caps[4] = {64, 128, 256, 512};
    b->tune_ms.assign(4, -1.0);
    RB_CUDA(cudaStreamSynchronize(b->main));
    size_t free_b = 0, total_b = 0;
    // release the current workspaces before measuring what fits
    RB_CUDA(cudaMemGetInfo(&free_b, &total_b));
    long long held = 0;
    for (rq_ctx *c : b->ctxs) {
        rq_info_t inf;
        rq_get_info(c, &inf);
        held += rq::workspace_bytes_for(c, inf.columns_per_tile, inf.max_dirs);
    }
    const double budget = 0.5 * ((double)free_b + (double)held);
    int best = -1;
    double best_ms = 1e300;
    cudaEvent_t e0, e1;
    RB_CUDA(cudaEventCreate(&e0));
    RB_CUDA(cudaEventCreate(&e1));
    for (int i = 0; i < 4 && !b->tile_fixed; ++i) {
        double need = 0;
        for (size_t p = 0; p < b->ctxs.size(); ++p)
            need += (double)rq::workspace_bytes_for(b->ctxs[p], std::min(caps[i], pow2ceil(1LL << b->n[p])), 1);
        if (need > budget) continue;
        rq_status st = apply_cap(b, caps[i]);
        if (st == RQ_OK) st = capture(b, 0, 0);  // cost-only proxy of the sweep
        if (st != RQ_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return st;
        }
        cudaGraphLaunch(b->exec, b->main);  // warm-up
        cudaEventRecord(e0, b->main);
        cudaGraphLaunch(b->exec, b->main);
        cudaEventRecord(e1, b->main);
        RB_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        b->tune_ms[i] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best = caps[i];
        }
    }
    if (b->tile_fixed) best = b->tile_cap;
    if (best < 0) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return bfail(b, RQ_ENOMEM, "no tile size fits the batch in device memory");
    }
    b->tile_cap = best;
    rq_status st = apply_cap(b, best);
    // sweep grid: timed on a gradient evaluation (the backward kernels carry
    // the per-CTA environment reductions that fewer CTAs save)
    const int grids[5] = {0, 8, 16, 32, 64};
    b->grid_ms.assign(5, -1.0);
    if (st == RQ_OK && b->grid_req < 0) {
        int best_m = 0;
        double best_m_ms = 1e300;
        for (int i = 0; i < 5 && st == RQ_OK; ++i) {
            double ms = 0;
            st = apply_grid(b, grids[i]);
            if (st == RQ_OK) st = time_graph(b, 1, e0, e1, ms);
            if (st != RQ_OK) break;
            b->grid_ms[i] = ms;
            if (ms < best_m_ms) {
                best_m_ms = ms;
                best_m = grids[i];
            }
        }
        if (st == RQ_OK) st = apply_grid(b, best_m);
    } else if (st == RQ_OK) {
        st = apply_grid(b, b->grid_req);
    }
    // gates per pass: the fusion window, timed on the cost-only proxy
    const int wins[4] = {0, 4, 5, 6};
    b->fuse_ms.assign(4, -1.0);
    if (st == RQ_OK && b->fuse_req < 0) {
        int best_q = 0;
        double best_q_ms = 1e300;
        for (int i = 0; i < 4 && st == RQ_OK; ++i) {
            double ms = 0;
            st = apply_fusion(b, wins[i]);
            if (st == RQ_OK) st = time_graph(b, 0, e0, e1, ms);
            if (st != RQ_OK) break;
            b->fuse_ms[i] = ms;
            if (ms < best_q_ms) {
                best_q_ms = ms;
                best_q = wins[i];
            }
        }
        if (st == RQ_OK) st = apply_fusion(b, best_q);
    } else if (st == RQ_OK) {
        st = apply_fusion(b, b->fuse_req);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != RQ_OK) return st;
    b->tuned = true;
    return RQ_OK;
}

}  // namespace

extern "C" {

rq_status rq_batch_create(rq_batch **out, int device) {
    if (!out) return RQ_EINVAL;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return RQ_ECUDA;
    rq_batch *b = new rq_batch();
    b->device = device;
    if (cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        delete b;
        return RQ_ECUDA;
    }
    *out = b;
    return RQ_OK;
}

rq_status rq_batch_destroy(rq_batch *b) {
    if (!b) return RQ_OK;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->main);
    drop_graph(b);
    for (rq_ctx *c : b->ctxs) rq_destroy(c);
    for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
    cudaEventDestroy(b->fork);
    cudaFree(b->d_gates);
    cudaFree(b->d_dirs);
    cudaFree(b->d_rgrad);
    cudaFree(b->d_hvps);
    cudaFree(b->d_f);
    cudaStreamDestroy(b->main);
    delete b;
    return RQ_OK;
}

rq_status rq_batch_add(rq_batch *b, const rq_target *t, const rq_circuit *c, int *index) {
    if (!b) return RQ_EINVAL;
    if (!t || !c) return bfail(b, RQ_EINVAL, "target or circuit is NULL");
    RB_CUDA(cudaSetDevice(b->device));
    rq_ctx *ctx = nullptr;
    rq_status st = rq_create(&ctx, b->device, nullptr);
    if (st != RQ_OK) return bfail(b, st, "%s", rq_last_error(nullptr));
    st = rq_setup_target(ctx, t, c);
    if (st != RQ_OK) {
        bfail(b, st, "problem %zu: %s", b->ctxs.size(), rq_last_error(ctx));
        rq_destroy(ctx);
        return st;
    }
    rq_info_t inf;
    rq_get_info(ctx, &inf);
    // a small tile until the batch tile is chosen (keeps the workspace modest)
    st = rq_set_tile(ctx, std::min(b->tile_cap > 0 ? b->tile_cap : 64, pow2ceil(1LL << inf.n_qubits)), 1);
    if (st != RQ_OK) {
        bfail(b, st, "problem %zu: %s", b->ctxs.size(), rq_last_error(ctx));
        rq_destroy(ctx);
        return st;
    }
    st = rq_set_fusion(ctx, b->fuse_q);  // the batch's current window
    if (st == RQ_OK) st = rq_set_grid(ctx, b->grid_items);
    if (st != RQ_OK) {
        bfail(b, st, "problem %zu: %s", b->ctxs.size(), rq_last_error(ctx));
        rq_destroy(ctx);
        return st;
    }
    cudaEvent_t ev;
    RB_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    if (index) *index = (int)b->ctxs.size();
    b->ctxs.push_back(ctx);
    b->joins.push_back(ev);
    b->P.push_back(inf.n_params);
    b->n.push_back(inf.n_qubits);
    b->goff.push_back(b->gtotal);
    b->gtotal += (long long)inf.n_params * 16;
    b->cap_k = -1;
    drop_graph(b);
    return RQ_OK;
}

rq_status rq_batch_set_tile(rq_batch *b, int columns_per_tile) {
    if (!b) return RQ_EINVAL;
    if (columns_per_tile < 0 || (columns_per_tile & (columns_per_tile - 1)) != 0)
        return bfail(b, RQ_EINVAL, "columns_per_tile %d is not 0 or a power of two", columns_per_tile);
    b->tile_cap = columns_per_tile;
    b->tile_fixed = columns_per_tile > 0;
    // else the grid or the fusion window is tuned at the next evaluation
    b->tuned = columns_per_tile > 0 && b->fuse_req >= 0 && b->grid_req >= 0;
    if (columns_per_tile > 0) return apply_cap(b, columns_per_tile);
    return RQ_OK;
}

rq_status rq_batch_hvp(rq_batch *b, const double *gates, const double *dirs, int k, int plain, double *f,
                       double *rgrad, double *hvps) {
    if (!b) return RQ_EINVAL;
    if (b->ctxs.empty()) return bfail(b, RQ_ESTATE, "empty batch");
    if (!gates || !f || k < 0 || (k > 0 && !dirs)) return bfail(b, RQ_EINVAL, "invalid arguments");
    RB_CUDA(cudaSetDevice(b->device));
    rq_status st = ensure_buffers(b, k);
    if (st != RQ_OK) return st;
    const size_t g = sizeof(double2) * (size_t)b->gtotal;
    RB_CUDA(cudaMemcpyAsync(b->d_gates, gates, g, cudaMemcpyHostToDevice, b->main));
    if (k > 0) RB_CUDA(cudaMemcpyAsync(b->d_dirs, dirs, g * k, cudaMemcpyHostToDevice, b->main));
    if (!b->tuned) {  // the autotuner's evaluations see these gates
        st = autotune(b);
        if (st != RQ_OK) return st;
    }
    if (plain) {
        for (rq_ctx *c : b->ctxs) {
            st = rq::prepare_capacity(c, std::max(k, 1));
            if (st != RQ_OK) return ctx_fail(b, c, st);
        }
        st = enqueue(b, k, 1, true);
        if (st != RQ_OK) return st;
    } else {
        if (b->graph_k != k || b->graph_env != 1) {
            RB_CUDA(cudaStreamSynchronize(b->main));
            st = capture(b, k, 1);
            if (st != RQ_OK) return st;
        }
        RB_CUDA(cudaGraphLaunch(b->exec, b->main));
    }
    RB_CUDA(cudaMemcpyAsync(f, b->d_f, sizeof(double) * b->ctxs.size(), cudaMemcpyDeviceToHost, b->main));
    if (rgrad) RB_CUDA(cudaMemcpyAsync(rgrad, b->d_rgrad, g, cudaMemcpyDeviceToHost, b->main));
    if (hvps && k > 0) RB_CUDA(cudaMemcpyAsync(hvps, b->d_hvps, g * k, cudaMemcpyDeviceToHost, b->main));
    RB_CUDA(cudaStreamSynchronize(b->main));
    return RQ_OK;
}

rq_status rq_batch_info(const rq_batch *b, int *n_problems, int *columns_per_tile, double *tune_ms) {
    if (!b) return RQ_EINVAL;
    if (n_problems) *n_problems = (int)b->ctxs.size();
    if (columns_per_tile) *columns_per_tile = b->tile_cap;
    if (tune_ms)
        for (int i = 0; i < 4; ++i) tune_ms[i] = i < (int)b->tune_ms.size() ? b->tune_ms[i] : -1.0;
    return RQ_OK;
}

rq_status rq_batch_set_grid(rq_batch *b, int min_items_per_thread) {
    if (!b) return RQ_EINVAL;
    if (min_items_per_thread < -1 || min_items_per_thread > (1 << 20))
        return bfail(b, RQ_EINVAL, "min_items_per_thread %d is neither -1 (autotune) nor in [0, 2^20]",
                     min_items_per_thread);
    RB_CUDA(cudaSetDevice(b->device));
    RB_CUDA(cudaStreamSynchronize(b->main));
    b->grid_req = min_items_per_thread;
    if (min_items_per_thread >= 0) {
        b->grid_ms.assign(5, -1.0);
        return apply_grid(b, min_items_per_thread);
    }
    b->tuned = false;  // tune again at the next evaluation
    return RQ_OK;
}

rq_status rq_batch_grid_info(const rq_batch *b, int *min_items_per_thread, double *tune_ms) {
    if (!b) return RQ_EINVAL;
    if (min_items_per_thread) *min_items_per_thread = b->grid_items;
    if (tune_ms)
        for (int i = 0; i < 5; ++i) tune_ms[i] = i < (int)b->grid_ms.size() ? b->grid_ms[i] : -1.0;
    return RQ_OK;
}

rq_status rq_batch_set_fusion(rq_batch *b, int max_window_qubits) {
    if (!b) return RQ_EINVAL;
    if (max_window_qubits != -1 && max_window_qubits != 0 && (max_window_qubits < 3 || max_window_qubits > rq::kMaxWindow))
        return bfail(b, RQ_EINVAL, "fusion window %d is neither -1 (autotune), 0 (off) nor in [3, %d]",
                     max_window_qubits, rq::kMaxWindow);
    b->fuse_req = max_window_qubits;
    if (max_window_qubits >= 0) {
        b->fuse_ms.assign(4, -1.0);
        return apply_fusion(b, max_window_qubits);
    }
    b->tuned = false;  // tune again at the next evaluation
    return RQ_OK;
}

rq_status rq_batch_fusion_info(const rq_batch *b, int *window, double *tune_ms) {
    if (!b) return RQ_EINVAL;
    if (window) *window = b->fuse_q;
    if (tune_ms)
        for (int i = 0; i < 4; ++i) tune_ms[i] = i < (int)b->fuse_ms.size() ? b->fuse_ms[i] : -1.0;
    return RQ_OK;
}

const char *rq_batch_last_error(const rq_batch *b) { return b ? b->err.c_str() : ""; }

}  // extern "C"
