// Target and circuit set-up: the device-resident sector blocks of U
// (Chebyshev expansion, or a caller's dense matrix), the per-gate geometry
// and first-layer masks, translation-representative columns, target columns.
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

}  // namespace rqc

extern "C" {

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

}  // extern "C"
