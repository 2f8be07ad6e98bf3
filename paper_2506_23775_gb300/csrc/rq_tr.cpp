// One Riemannian trust-region iteration on the host (paper Sec. "Riemannian
// optimization": Absil et al. Algorithm 10 with the truncated conjugate-
// gradient inner solver of Algorithm 11), over the product manifold of the
// parameter gates with the metric sum Re Tr[X^dagger Y] and the polar
// retraction R_V(xi) = qpolar(V + xi) (Eq. retraction_qr).  Every cost,
// gradient and Hessian-vector product runs on the device; the host only
// holds vectors of 32 doubles per parameter gate.
#include "rq_internal.h"

#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

namespace {

using Vec = std::vector<double>;

double dot(const Vec &a, const Vec &b) {
    double s = 0.0;
    for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];  // Re(conj(a) b) summed
    return s;
}

void axpy(Vec &y, double a, const Vec &x) {
    for (size_t i = 0; i < y.size(); ++i) y[i] += a * x[i];
}

// Inverse of a 4x4 complex matrix (interleaved) by Gauss-Jordan elimination
// with partial pivoting.  Returns false if singular.
bool inv4(const double *A, double *Ainv) {
    double m[4][8][2];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 8; ++j) {
            m[i][j][0] = j < 4 ? A[2 * (i * 4 + j)] : (j - 4 == i ? 1.0 : 0.0);
            m[i][j][1] = j < 4 ? A[2 * (i * 4 + j) + 1] : 0.0;
        }
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        double best = -1.0;
        for (int r = c; r < 4; ++r) {
            const double v = std::hypot(m[r][c][0], m[r][c][1]);
            if (v > best) { best = v; piv = r; }
        }
        if (!(best > 0.0)) return false;
        if (piv != c)
            for (int j = 0; j < 8; ++j) std::swap(m[piv][j], m[c][j]);
        // scale row c by 1 / pivot
        const double pr = m[c][c][0], pi = m[c][c][1], d = pr * pr + pi * pi;
        const double ir = pr / d, ii = -pi / d;
        for (int j = 0; j < 8; ++j) {
            const double xr = m[c][j][0], xi = m[c][j][1];
            m[c][j][0] = xr * ir - xi * ii;
            m[c][j][1] = xr * ii + xi * ir;
        }
        for (int r = 0; r < 4; ++r) {
            if (r == c) continue;
            const double fr = m[r][c][0], fi = m[r][c][1];
            if (fr == 0.0 && fi == 0.0) continue;
            for (int j = 0; j < 8; ++j) {
                const double xr = m[c][j][0], xi = m[c][j][1];
                m[r][j][0] -= fr * xr - fi * xi;
                m[r][j][1] -= fr * xi + fi * xr;
            }
        }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            Ainv[2 * (i * 4 + j)] = m[i][j + 4][0];
            Ainv[2 * (i * 4 + j) + 1] = m[i][j + 4][1];
        }
    return true;
}

using C4 = std::complex<double>;

void load4(const double *p, C4 (&m)[16]) {
    for (int i = 0; i < 16; ++i) m[i] = C4(p[2 * i], p[2 * i + 1]);
}

void store4(const C4 (&m)[16], double *p) {
    for (int i = 0; i < 16; ++i) {
        p[2 * i] = m[i].real();
        p[2 * i + 1] = m[i].imag();
    }
}

// A^dagger B
void mul_dag(const C4 (&A)[16], const C4 (&B)[16], C4 (&C)[16]) {
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            C4 s = 0;
            for (int k = 0; k < 4; ++k) s += std::conj(A[k * 4 + i]) * B[k * 4 + j];
            C[i * 4 + j] = s;
        }
}

void mul(const C4 (&A)[16], const C4 (&B)[16], C4 (&C)[16]) {
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            C4 s = 0;
            for (int k = 0; k < 4; ++k) s += A[i * 4 + k] * B[k * 4 + j];
            C[i * 4 + j] = s;
        }
}

// (A - A^dagger)/2 (sign -1) or (A + A^dagger)/2 (sign +1)
void herm(const C4 (&A)[16], double sign, C4 (&C)[16]) {
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) C[i * 4 + j] = 0.5 * (A[i * 4 + j] + sign * std::conj(A[j * 4 + i]));
}

bool in_pattern(int e) {
    const int r = e >> 2, c = e & 3;
    return (r == 0 || r == 3) == (c == 0 || c == 3);
}

// P_G(Z) = G skew(G^dagger Z) for every parameter gate
void project_all(const double *G, const Vec &Z, Vec &out, int P) {
    for (int p = 0; p < P; ++p) {
        C4 g[16], z[16], t[16], s[16], r[16];
        load4(G + p * 32, g);
        load4(Z.data() + p * 32, z);
        mul_dag(g, z, t);
        herm(t, -1.0, s);
        mul(g, s, r);
        store4(r, out.data() + p * 32);
    }
}

}  // namespace

namespace rq {

// Unitary polar factor by the Newton iteration Q <- (Q + Q^{-dagger}) / 2
// (quadratically convergent for a nonsingular start, Higham 1986).
int polar_unitary_4x4(const double *A, double *Q) {
    double cur[32], inv[32], nxt[32];
    std::memcpy(cur, A, sizeof(cur));
    for (int it = 0; it < 100; ++it) {
        if (!inv4(cur, inv)) return -1;
        double diff = 0.0, norm = 0.0;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                // (Q^{-1})^dagger [i][j] = conj(inv[j][i])
                const double hr = inv[2 * (j * 4 + i)], hi = -inv[2 * (j * 4 + i) + 1];
                const int k = 2 * (i * 4 + j);
                nxt[k] = 0.5 * (cur[k] + hr);
                nxt[k + 1] = 0.5 * (cur[k + 1] + hi);
                diff += (nxt[k] - cur[k]) * (nxt[k] - cur[k]) + (nxt[k + 1] - cur[k + 1]) * (nxt[k + 1] - cur[k + 1]);
                norm += nxt[k] * nxt[k] + nxt[k + 1] * nxt[k + 1];
            }
        std::memcpy(cur, nxt, sizeof(cur));
        if (diff <= 1e-30 * norm) break;
    }
    std::memcpy(Q, cur, sizeof(cur));
    return 0;
}

}  // namespace rq

extern "C" rq_status rq_tr_step(rq_ctx *ctx, double *gates, rq_tr_state *st) {
    if (!ctx) return RQ_EINVAL;
    if (!gates || !st) return rq::set_error(ctx, RQ_EINVAL, "gates or state is NULL");
    rq_info_t info;
    rq_get_info(ctx, &info);
    if (info.n_params <= 0) return rq::set_error(ctx, RQ_ESTATE, "no target set up");
    if (!(st->radius > 0.0) || !(st->max_radius >= st->radius))
        return rq::set_error(ctx, RQ_EINVAL, "need 0 < radius <= max_radius");
    const int P = info.n_params;
    // the trust region works with Riemannian quantities whatever the context's output option
    struct SpaceGuard {
        rq_ctx *c;
        int saved;
        ~SpaceGuard() {
            if (saved != RQ_SPACE_RIEMANNIAN) rq_set_gradient_space(c, saved);
        }
    } guard{ctx, rq::gradient_space(ctx)};
    if (guard.saved != RQ_SPACE_RIEMANNIAN) rq_set_gradient_space(ctx, RQ_SPACE_RIEMANNIAN);
    const size_t dimv = (size_t)P * 32;
    const int dim = P * (info.structure == 1 ? 8 : 16);
    const int max_inner = st->max_inner > 0 ? st->max_inner : dim;
    const double radius = st->radius;

    Vec grad(dimv), eta(dimv, 0.0), Heta(dimv, 0.0), r(dimv), delta(dimv), Hd(dimv);
    double f = 0.0;
    rq_status s = RQ_OK;
    // full-Hessian mode: gbar, the tied holomorphic Hessian H and the
    // correction matrices sym(G^dagger gbar), once per step
    const bool full = st->full_hessian != 0;
    const long long D = (long long)P * 16;
    std::vector<double> Hh;
    Vec gbar;
    std::vector<C4> symm;
    if (full) {
        Hh.resize((size_t)(2 * D * D));
        gbar.resize(dimv);
        s = rq_hessian(ctx, gates, &f, gbar.data(), Hh.data());
        if (s != RQ_OK) return s;
        project_all(gates, gbar, grad, P);
        symm.resize((size_t)P * 16);
        for (int p = 0; p < P; ++p) {
            C4 g4[16], b4[16], m4[16], s4[16];
            load4(gates + p * 32, g4);
            load4(gbar.data() + p * 32, b4);
            mul_dag(g4, b4, m4);
            herm(m4, +1.0, s4);
            for (int i = 0; i < 16; ++i) symm[(size_t)p * 16 + i] = s4[i];
        }
    } else {
        s = rq::eval_host(ctx, gates, nullptr, 0, 1, &f, grad.data(), nullptr);
        if (s != RQ_OK) return s;
    }
    // Riemannian Hessian of the tangent vector X from H:
    // P_G( mask(-conj(H vec X)) - X sym(G^dagger gbar) )
    auto hess_full = [&](const Vec &X, Vec &out) {
        Vec dg(dimv, 0.0);
        for (long long i = 0; i < D; ++i) {
            C4 acc = 0;
            const double *row = Hh.data() + 2 * i * D;
            for (long long j = 0; j < D; ++j) acc += C4(row[2 * j], row[2 * j + 1]) * C4(X[2 * j], X[2 * j + 1]);
            const bool keep = info.structure != 1 || in_pattern((int)(i & 15));
            dg[2 * i] = keep ? -acc.real() : 0.0;
            dg[2 * i + 1] = keep ? acc.imag() : 0.0;
        }
        for (int p = 0; p < P; ++p) {
            C4 x4[16], s4[16], xs[16];
            load4(X.data() + p * 32, x4);
            for (int i = 0; i < 16; ++i) s4[i] = symm[(size_t)p * 16 + i];
            mul(x4, s4, xs);
            for (int i = 0; i < 16; ++i) {
                dg[p * 32 + 2 * i] -= xs[i].real();
                dg[p * 32 + 2 * i + 1] -= xs[i].imag();
            }
        }
        project_all(gates, dg, out, P);
    };
    r = grad;
    for (size_t i = 0; i < dimv; ++i) delta[i] = -r[i];
    double rr = dot(r, r);
    const double r0 = std::sqrt(rr);
    int code = 3, j = 0;
    // truncated CG (Steihaug); Hess applied by the device HVP
    for (j = 0; j < max_inner; ++j) {
        if (rr == 0.0) { code = 0; break; }
        if (full) {
            hess_full(delta, Hd);
        } else {
            double fh = 0.0;
            // the gradient environments at these gates are still in the accumulators
            s = rq::eval_host(ctx, gates, delta.data(), 1, 2, &fh, nullptr, Hd.data());
            if (s != RQ_OK) return s;
        }
        const double dHd = dot(delta, Hd);
        auto to_boundary = [&]() {
            const double a = dot(delta, delta), b = 2.0 * dot(eta, delta), c = dot(eta, eta) - radius * radius;
            return (-b + std::sqrt(b * b - 4.0 * a * c)) / (2.0 * a);
        };
        if (dHd <= 0.0) {
            const double tau = to_boundary();
            axpy(eta, tau, delta);
            axpy(Heta, tau, Hd);
            code = 1;
            ++j;
            break;
        }
        const double alpha = rr / dHd;
        Vec eta_new = eta;
        axpy(eta_new, alpha, delta);
        if (std::sqrt(dot(eta_new, eta_new)) >= radius) {
            const double tau = to_boundary();
            axpy(eta, tau, delta);
            axpy(Heta, tau, Hd);
            code = 2;
            ++j;
            break;
        }
        eta.swap(eta_new);
        axpy(Heta, alpha, Hd);
        axpy(r, alpha, Hd);
        const double rr_new = dot(r, r);
        if (std::sqrt(rr_new) <= r0 * std::fmin(std::pow(r0, st->theta), st->kappa)) {
            code = 0;
            ++j;
            break;
        }
        const double beta = rr_new / rr;
        rr = rr_new;
        for (size_t i = 0; i < dimv; ++i) delta[i] = -r[i] + beta * delta[i];
    }
    // candidate: polar retraction of every parameter gate
    Vec cand(dimv);
    for (int p = 0; p < P; ++p) {
        double A[32];
        for (int i = 0; i < 32; ++i) A[i] = gates[p * 32 + i] + eta[p * 32 + i];
        if (rq::polar_unitary_4x4(A, &cand[p * 32]) != 0)
            return rq::set_error(ctx, RQ_EINVAL, "retraction: singular gate + step");
    }
    double f_new = 0.0;
    s = rq::eval_host(ctx, cand.data(), nullptr, 0, 0, &f_new, nullptr, nullptr);
    if (s != RQ_OK) return s;
    const double model_decrease = -(dot(grad, eta) + 0.5 * dot(Heta, eta));
    const double rho = model_decrease != 0.0 ? (f - f_new) / model_decrease : 0.0;
    double new_radius = radius;
    if (rho < 0.25) new_radius = 0.25 * radius;
    else if (rho > 0.75 && (code == 1 || code == 2)) new_radius = std::fmin(2.0 * radius, st->max_radius);
    const bool accepted = rho > st->rho_accept;
    if (accepted) std::memcpy(gates, cand.data(), sizeof(double) * dimv);
    st->f = f;
    st->f_new = f_new;
    st->rho = rho;
    st->grad_norm = r0;
    st->step_norm = std::sqrt(dot(eta, eta));
    st->accepted = accepted ? 1 : 0;
    st->n_inner = j;
    st->tcg_exit = code;
    st->radius = new_radius;
    return RQ_OK;
}
