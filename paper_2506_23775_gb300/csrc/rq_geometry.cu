// Reductions and Riemannian post-processing on the device.
//
// * Per-CTA environment partials are summed in CTA order into per-gate
//   accumulators (fixed order: results do not depend on timing).
// * Euclidean gradient (Eq. def_grad): the cost is f = -Re F with F
//   holomorphic in every gate entry, so d_x f + i d_y f = -conj(dF/dG); the
//   copies of a tied gate are summed (Sec. "Brick wall circuit layout");
//   parity-conserving gates keep only their pattern (Eq. paritygatematrix).
// * Riemannian gradient grad f = G skew(G^dagger gbar) (Eq. proj_tangent,
//   Eq. grad_proj).
// * With the Euclidean output option the masked gbar and Dgbar[X] (X a raw
//   complex direction, only masked) are returned instead (autograd use).
// * Riemannian Hessian along a tangent X (Eq. vector_field_derivative,
//   Eq. hessian_def): differentiating xi(V) = V skew(V^dagger gbar(V)) and
//   projecting gives, with X = G Omega and Omega skew-Hermitian,
//       Hess f(G)[X] = P_G( Dgbar[X] - X sym(G^dagger gbar) ),
//   because P_G(X skew(M)) + P_G(G skew(X^dagger gbar)) = -G skew(Omega sym(M))
//   for M = G^dagger gbar.
#include "rq_internal.h"

namespace rq {
namespace {

struct M4 {
    double2 a[16];
};

__device__ __forceinline__ double2 cmul(double2 x, double2 y) {
    return make_double2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x);
}

__device__ __forceinline__ double2 cadd(double2 x, double2 y) { return make_double2(x.x + y.x, x.y + y.y); }

__device__ M4 load4(const double2 *p) {
    M4 m;
    for (int i = 0; i < 16; ++i) m.a[i] = p[i];
    return m;
}

__device__ M4 matmul(const M4 &A, const M4 &B) {
    M4 C;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double2 s = make_double2(0.0, 0.0);
            for (int k = 0; k < 4; ++k) s = cadd(s, cmul(A.a[i * 4 + k], B.a[k * 4 + j]));
            C.a[i * 4 + j] = s;
        }
    return C;
}

// A^dagger B
__device__ M4 matmul_dag(const M4 &A, const M4 &B) {
    M4 C;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double2 s = make_double2(0.0, 0.0);
            for (int k = 0; k < 4; ++k) {
                const double2 a = make_double2(A.a[k * 4 + i].x, -A.a[k * 4 + i].y);
                s = cadd(s, cmul(a, B.a[k * 4 + j]));
            }
            C.a[i * 4 + j] = s;
        }
    return C;
}

// (A - A^dagger) / 2 (sign = -1) or (A + A^dagger) / 2 (sign = +1)
__device__ M4 herm_part(const M4 &A, double sign) {
    M4 C;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            const double2 a = A.a[i * 4 + j], b = A.a[j * 4 + i];
            C.a[i * 4 + j] = make_double2(0.5 * (a.x + sign * b.x), 0.5 * (a.y - sign * b.y));
        }
    return C;
}

__device__ __forceinline__ bool in_pattern(int i) {
    const int r = i >> 2, c = i & 3;
    return ((r == 0 || r == 3) == (c == 0 || c == 3));
}

__device__ void apply_mask(M4 &A, int structure) {
    if (structure != 1) return;
    for (int i = 0; i < 16; ++i)
        if (!in_pattern(i)) A.a[i] = make_double2(0.0, 0.0);
}

// P_G(Z) = G skew(G^dagger Z)
__device__ M4 project(const M4 &G, const M4 &Z) { return matmul(G, herm_part(matmul_dag(G, Z), -1.0)); }

__global__ void k_reduce_env(const double *part, int ncta, double *env) {
    const int l = blockIdx.x, t = threadIdx.x;
    const double *p = part + (long long)l * ncta * kEnvDoubles + t;
    double s = 0.0;
    for (int c = 0; c < ncta; ++c) s += p[(long long)c * kEnvDoubles];
    env[(long long)l * kEnvDoubles + t] += s;
}

__global__ void k_reduce_f(const double *fpart, int B, double *facc) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < B; ++b) s += fpart[b];
    facc[0] += s;
}

__global__ void k_project_dirs(const double2 *gates, const double2 *raw, double2 *out, int P, int k,
                               int structure, int euclidean) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= P * k) return;
    const int p = id % P;
    M4 G = load4(gates + (long long)p * 16);
    M4 X = euclidean ? load4(raw + (long long)id * 16) : project(G, load4(raw + (long long)id * 16));
    apply_mask(X, structure);
    for (int i = 0; i < 16; ++i) out[(long long)id * 16 + i] = X.a[i];
}

__global__ void k_mask_gates(const double2 *in, double2 *out, int P, int structure) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= P * 16) return;
    out[id] = (structure == 1 && !in_pattern(id & 15)) ? make_double2(0.0, 0.0) : in[id];
}

// Thread per (direction slot d in [0, k], parameter p); slot 0 = gradient.
__global__ void k_geometry(const double2 *gates, const double2 *dirs, const double *env,
                           const double *env_dot, const int32_t *param_of, int g, int P, int k,
                           int structure, int euclidean, const double *facc, double *f_out, double2 *rgrad,
                           double2 *hvps) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id == 0 && f_out != nullptr) f_out[0] = facc[0];
    if (id >= P * (k + 1)) return;
    const int d = id / P, p = id % P;
    const M4 G = load4(gates + (long long)p * 16);
    // Euclidean gradient of the parameter gate: -conj of the tied sum
    M4 gb;
    for (int i = 0; i < 16; ++i) gb.a[i] = make_double2(0.0, 0.0);
    for (int l = 0; l < g; ++l) {
        if (param_of[l] != p) continue;
        for (int i = 0; i < 16; ++i) {
            gb.a[i].x -= env[(long long)l * kEnvDoubles + 2 * i];
            gb.a[i].y += env[(long long)l * kEnvDoubles + 2 * i + 1];
        }
    }
    apply_mask(gb, structure);
    if (d == 0) {
        if (rgrad == nullptr) return;
        const M4 R = euclidean ? gb : project(G, gb);
        for (int i = 0; i < 16; ++i) rgrad[(long long)p * 16 + i] = R.a[i];
        return;
    }
    const int dd = d - 1;
    M4 dg;
    for (int i = 0; i < 16; ++i) dg.a[i] = make_double2(0.0, 0.0);
    const double *ed = env_dot + (long long)dd * g * kEnvDoubles;
    for (int l = 0; l < g; ++l) {
        if (param_of[l] != p) continue;
        for (int i = 0; i < 16; ++i) {
            dg.a[i].x -= ed[(long long)l * kEnvDoubles + 2 * i];
            dg.a[i].y += ed[(long long)l * kEnvDoubles + 2 * i + 1];
        }
    }
    apply_mask(dg, structure);
    if (euclidean) {  // Euclidean Hessian applied to the direction: Dgbar[X]
        if (hvps == nullptr) return;
        for (int i = 0; i < 16; ++i) hvps[((long long)dd * P + p) * 16 + i] = dg.a[i];
        return;
    }
    const M4 X = load4(dirs + ((long long)dd * P + p) * 16);
    const M4 XS = matmul(X, herm_part(matmul_dag(G, gb), +1.0));
    for (int i = 0; i < 16; ++i) dg.a[i] = make_double2(dg.a[i].x - XS.a[i].x, dg.a[i].y - XS.a[i].y);
    const M4 H = project(G, dg);
    if (hvps == nullptr) return;
    for (int i = 0; i < 16; ++i) hvps[((long long)dd * P + p) * 16 + i] = H.a[i];
}

}  // namespace

void launch_reduce_env(const double *part, int ncta, int n_gates, double *env, cudaStream_t s) {
    k_reduce_env<<<n_gates, kEnvDoubles, 0, s>>>(part, ncta, env);
}

void launch_reduce_f(const double *fpart, int B, double *facc, cudaStream_t s) {
    k_reduce_f<<<1, 32, 0, s>>>(fpart, B, facc);
}

void launch_project_dirs(const double2 *gates, const double2 *raw, double2 *out, int n_params,
                         int k, int structure, int euclidean, cudaStream_t s) {
    const int n = n_params * k;
    if (n == 0) return;
    k_project_dirs<<<(n + 63) / 64, 64, 0, s>>>(gates, raw, out, n_params, k, structure, euclidean);
}

void launch_mask_gates(const double2 *in, double2 *out, int n_params, int structure, cudaStream_t s) {
    const int n = n_params * 16;
    k_mask_gates<<<(n + 255) / 256, 256, 0, s>>>(in, out, n_params, structure);
}

void launch_geometry(const double2 *gates, const double2 *dirs, const double *env,
                     const double *env_dot, const int32_t *param_of, int n_gates, int n_params,
                     int k, int structure, int euclidean, const double *facc, double *f_out, double2 *rgrad,
                     double2 *hvps, cudaStream_t s) {
    const int n = n_params * (k + 1);
    k_geometry<<<(n + 63) / 64, 64, 0, s>>>(gates, dirs, env, env_dot, param_of, n_gates, n_params,
                                            k, structure, euclidean, facc, f_out, rgrad, hvps);
}

}  // namespace rq
