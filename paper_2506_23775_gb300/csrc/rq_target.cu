// Device-resident target U = exp(-iHt) and its use in the sweep.
//
// The paper applies U "matrix-free" to each basis column (Sec. "Objective
// function and matrix-free evaluation") without saying how.  The spinful
// Fermi-Hubbard H of Eq. sfFH conserves the numbers of up and down particles
// (the spinless H of Eq. slFH_qubit the particle number), so U is block
// diagonal over these sectors and column U|j> lives in the sector of j.  Each block is computed once on the device by the Chebyshev expansion
//     exp(-i H t) = exp(-i b t) sum_k (2 - delta_k0) (-i)^k J_k(a t) T_k(Ht),
// Ht = (H - b) / a with spectrum in [-1, 1] (Gershgorin bound), applied to the
// identity of every sector with the sparse H (the Jacobi-Anger expansion; the
// three-term recurrence T_{k+1} = 2 Ht T_k - T_{k-1} keeps everything real
// until the complex coefficients are added).  Blocks are stored column-major
// so a column U|j> is contiguous.
//
// In the sweep, one kernel scatters U|j_b> into the adjoint start tile
// lambda_N and, in the same pass, forms the cost summand
// -Re <U j_b | psi_N> of Eq. f_target_sum_unit_vec.
#include "rq_internal.h"

#include <cmath>

namespace rq {
namespace {

__device__ __forceinline__ int find_sector(const long long *off, int S, long long e) {
    int lo = 0, hi = S;  // off[lo] <= e < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= e) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_cheb_init(const long long *off_u, const long long *sizes, int S, long long total,
                            double *prev, double2 *acc, double2 c0) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int s = find_sector(off_u, S, e);
        const long long m = sizes[s];
        const long long local = e - off_u[s];
        const double v = (local / m == local % m) ? 1.0 : 0.0;
        prev[e] = v;
        acc[e] = make_double2(c0.x * v, c0.y * v);
    }
}

// out = scale * Ht(cur) - prev (prev ignored when first); prev_out = out;
// acc += coef * out.  Element e = (sector s, column c, row r), column-major.
__global__ void k_cheb_step(const TargetDev t, int S, long long total, const double *cur,
                            double *prev_out, double2 *acc, double2 coef, double scale, int first,
                            double dscale, double dshift, double hop, const long long *bonds,
                            int nb, int L, double U, int model) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long lowmask = (1LL << L) - 1;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int s = find_sector(t.off_u, S, e);
        const long long m = t.off_basis[s + 1] - t.off_basis[s];
        const long long local = e - t.off_u[s];
        const long long c = local / m, r = local - c * m;
        const long long col = t.off_u[s] + c * m;
        const long long x = t.basis[t.off_basis[s] + r];
        double diag = model == 0 ? U * (double)__popcll((x >> L) & (x & lowmask)) : 0.0;
        double hsum = 0.0;
        for (int i = 0; i < nb; ++i) {
            const long long mk = bonds[i];
            const long long bits = x & mk;
            if (bits != 0 && bits != mk) hsum += hop * cur[col + t.pos[x ^ mk]];
            else if (model == 1 && bits == mk) diag += U;  // n_j n_{j+1} on the bond
        }
        const double h = (diag - dshift) * dscale * cur[col + r] + hsum;
        const double out = scale * h - (first ? 0.0 : prev_out[e]);
        prev_out[e] = out;
        double2 a = acc[e];
        a.x = fma(coef.x, out, a.x);
        a.y = fma(coef.y, out, a.y);
        acc[e] = a;
    }
}

// One CTA per column b: lambda[x, b] = w_b U[x, j_b] over the sector of j_b and
// fpart[b] = -w_b Re sum_x conj(U[x, j_b]) psi_N[x, b]; w_b = 1 unless the
// columns are weighted orbit representatives (wts != NULL).  Everything the
// backward pass computes is linear in lambda, so the weight carries through.
__global__ void k_scatter_target(const TargetDev t, const int32_t *cols, const double *wts, int log2B,
                                 long long mask, double2 *lam, const double2 *psi, double *fpart) {
    const int b = blockIdx.x;
    const int j = cols[b];
    const double wb = wts ? wts[b] : 1.0;
    double acc = 0.0;
    if (j >= 0) {
        const int s = t.sec_of[j];
        const long long m = t.off_basis[s + 1] - t.off_basis[s];
        const double2 *ucol = t.U + t.off_u[s] + (long long)t.pos[j] * m;
        const int32_t *bas = t.basis + t.off_basis[s];
        for (long long r = threadIdx.x; r < m; r += blockDim.x) {
            const long long o = (((long long)bas[r] & mask) << log2B) | b;
            const double2 u = make_double2(wb * ucol[r].x, wb * ucol[r].y);
            const double2 p = psi[o];
            lam[o] = u;
            acc = fma(u.x, p.x, acc);
            acc = fma(u.y, p.y, acc);  // Re(conj(u) p)
        }
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
        fpart[b] = -sum;
    }
}

}  // namespace

void launch_cheb_init(const long long *off_u, const long long *sizes, int n_sectors, long long total,
                      double *prev, double2 *acc, double2 c0, cudaStream_t s) {
    const long long blocks = (total + 255) / 256;
    k_cheb_init<<<(int)(blocks < 65536 ? blocks : 65536), 256, 0, s>>>(off_u, sizes, n_sectors, total,
                                                                      prev, acc, c0);
}

void launch_cheb_step(const TargetDev &t, int n_sectors, long long total, const double *cur,
                      double *prev_out, double2 *acc, double2 coef, double scale, int first,
                      double diag_scale, double diag_shift, double hop_scale,
                      const long long *bond_masks, int n_bonds, int L, double U, int model, cudaStream_t s) {
    const long long blocks = (total + 255) / 256;
    k_cheb_step<<<(int)(blocks < 65536 ? blocks : 65536), 256, 0, s>>>(
        t, n_sectors, total, cur, prev_out, acc, coef, scale, first, diag_scale, diag_shift,
        hop_scale, bond_masks, n_bonds, L, U, model);
}

void launch_scatter_target(const TargetDev &t, const int32_t *cols, const double *wts, int B, int log2B,
                           int parity_layout, int n, double2 *lam, const double2 *psi_final,
                           double *fpart, cudaStream_t s) {
    const long long mask = parity_layout ? ((1LL << (n - 1)) - 1) : ((1LL << n) - 1);
    k_scatter_target<<<B, 128, 0, s>>>(t, cols, wts, log2B, mask, lam, psi_final, fpart);
}

// Bessel functions J_0..J_kmax(x), x >= 0, by Miller's backward recurrence
// J_{k-1} = (2k / x) J_k - J_{k+1} started far above kmax and normalised with
// J_0 + 2 sum_{k>=1} J_{2k} = 1.  Returns the start index used.
double bessel_j_table(double x, int kmax, std::vector<double> &out) {
    out.assign(kmax + 1, 0.0);
    if (x == 0.0) {
        out[0] = 1.0;
        return 0.0;
    }
    int start = kmax + 40 + (int)(2.0 * x);
    if (start % 2) ++start;
    std::vector<double> j(start + 2, 0.0);
    j[start + 1] = 0.0;
    j[start] = 1e-300;
    for (int k = start; k >= 1; --k) {
        j[k - 1] = (2.0 * k / x) * j[k] - j[k + 1];
        if (std::fabs(j[k - 1]) > 1e250) {
            for (int i = k - 1; i <= start; ++i) j[i] *= 1e-250;
        }
    }
    double norm = j[0];
    for (int k = 2; k <= start; k += 2) norm += 2.0 * j[k];
    for (int k = 0; k <= kmax; ++k) out[k] = j[k] / norm;
    return (double)start;
}

}  // namespace rq
