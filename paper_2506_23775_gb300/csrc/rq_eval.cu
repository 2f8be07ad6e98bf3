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
//
// This file: that schedule (eval_dev), host-memory evaluations with their
// CUDA graphs, gate validation, the full Hessian's schedule and the
// evaluation entry points.
#include "rq_context.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

using rq::GateGeom;
using namespace rqc;

namespace rqc {

namespace {
// Number of c-bit patterns of m bits with lo <= c <= hi.
double count_window(int m, int lo, int hi) {
    double s = 0.0, binom = 1.0;  // C(m, c), c ascending
    for (int c = 0; c <= m; ++c) {
        if (c >= lo && c <= hi) s += binom;
        binom = binom * (m - c) / (c + 1);
    }
    return s;
}
}  // namespace

// Items of a last-layer gate with work in tile ti (the profile's algorithmic
// counts; the kernels visit every item and skip the others): per column j,
// 2^(bits the run has touched, less the gate's own) times the patterns of
// the untouched up and down bits that can be completed to j's sector.
double tail_items(const rq_ctx *ctx, const GateGeom &geo, int ti) {
    const int mu = __builtin_popcountll(geo.up_out), md = __builtin_popcountll(geo.dn_out);
    const int other = ctx->n - 2 - mu - md;
    double total = 0.0;
    for (int b = 0; b < ctx->B; ++b) {
        const long long j = ctx->cols_h[(size_t)ti * ctx->B + b];
        if (j < 0) continue;
        const int nu = __builtin_popcountll(j & geo.up_mask), nd = __builtin_popcountll(j & geo.dn_mask);
        total += std::ldexp(count_window(mu, nu - geo.f_up, nu) * count_window(md, nd - geo.f_dn, nd), other);
    }
    return total;
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
    const bool fused = fused_schedule(ctx);  // the order the last-layer marks were made for
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
                    // double-buffered block copies while two CTAs still fit on an SM
                    fa.nbuf = rq::fused_smem_bytes(q, kd, pp.m, 2) <= rq::kMaxFusedSmem / 2 ? 2 : 1;
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
                        const cudaError_t le = df ? rq::launch_fwd_fused_df64(fa, ctx->sms, s)
                                                  : rq::launch_fwd_fused(fa, ctx->sms, s);
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
                // last-layer support: the kernels skip the items whose adjoint
                // amplitudes are zero (they read the column table for j); a
                // gate of both runs enumerates its restricted items only when
                // first-layer support is on
                if (geo.tail) {
                    a.cols = cols;
                    if (!first_layer) a.geo.restricted = 0;
                }
                // items with work, for the profile's algorithmic counts
                const double live = ctx->prof_on && geo.tail && !(geo.restricted && first_layer)
                                        ? tail_items(ctx, geo, ti) : (double)a.n_items;
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
                        ProfScope ps(ctx, kFamBwdDir, live * 8.0 * cm * (2 + 2 * b.update),
                                     live * amps * sizeof(double2) * (4 + b.update));
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
                        ProfScope ps(ctx, kFamBwdBase, live * 8.0 * cm * (a.accumulate + a.update),
                                     live * amps * sizeof(double2) * (1 + a.accumulate + a.update));
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

}  // namespace rqc

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

rq_status eval_device(rq_ctx *ctx, const double *gates, const double *dirs, int k, int env_mode, double *f,
                      double *rgrad, double *hvps) {
    return eval_dev(ctx, gates, dirs, k, env_mode, f, rgrad, hvps);
}

}  // namespace rq

extern "C" {

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

}  // extern "C"
