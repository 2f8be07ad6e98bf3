// Full-Hessian kernels: gate-hole application and array hole contraction.
//
// Paper Sec. "Efficient gradient and Hessian computation" (Fig.
// hole_application, Fig. hessian_pass_second_gradient) and Sec. "Gate hole
// application": for each gate l the hole of G_l is applied to psi_{l-1},
// giving a state-vector array with one member per entry (a, b) of G_l -- the
// derivative of G_l psi_{l-1} with respect to that entry, e_ab psi_{l-1}.  The
// array is propagated through the later gates like an ordinary state, and at
// every later gate l' the hole of G_l' is contracted between the adjoint state
// and each member, giving the block d^2 F / dG_l[a,b] dG_l'[c,d].
//
// Layout: the paper interleaves the members as the fastest index; here the
// member index sits just above the column index of the tile (array column =
// member * B + column), so an array is an ordinary tile of M * B columns and
// the forward kernels propagate it unchanged.  Parity-conserving gates
// (Eq. paritygatematrix) need only the 8 pattern entries, halving the array
// (Sec. "Parity-conserving gate structure").
#include "rq_internal.h"

namespace rq {
namespace {

// member -> (a, b): general gates all 16 entries, parity gates the pattern
__constant__ int c_members[2][16][2] = {
    {{0, 0}, {0, 1}, {0, 2}, {0, 3}, {1, 0}, {1, 1}, {1, 2}, {1, 3},
     {2, 0}, {2, 1}, {2, 2}, {2, 3}, {3, 0}, {3, 1}, {3, 2}, {3, 3}},
    {{0, 0}, {0, 3}, {3, 0}, {3, 3}, {1, 1}, {1, 2}, {2, 1}, {2, 2},
     {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}}};

__device__ __forceinline__ long long insert_zero(long long r, int p) {
    const long long lo = r & ((1LL << p) - 1);
    return ((r >> p) << (p + 1)) | lo;
}

__device__ __forceinline__ void cmacc(double2 &acc, const double2 a, const double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}

// Stored indices and local 4x4 indices of the amplitudes of item r for a gate.
// Returns the number of amplitudes (4, or 2 for a parity gate on qubit 0).
__device__ __forceinline__ int item_amps(const GateGeom &geo, long long r, int parity, long long (&x)[4],
                                         int (&loc)[4]) {
    if (geo.mode == kParity2) {
        const long long y0 = insert_zero(r, geo.pa);
        x[0] = y0;
        x[1] = y0 | (1LL << geo.pa);
        const int e = (__popcll(y0) & 1) ^ parity;
        if (e == 0) {
            loc[0] = 0;
            loc[1] = 3;
        } else if (geo.qfirst) {
            loc[0] = 1;
            loc[1] = 2;
        } else {
            loc[0] = 2;
            loc[1] = 1;
        }
        return 2;
    }
    const int plo = geo.pa < geo.pb ? geo.pa : geo.pb;
    const int phi = geo.pa < geo.pb ? geo.pb : geo.pa;
    const long long x0 = insert_zero(insert_zero(r, plo), phi);
    const long long sa = 1LL << geo.pa, sb = 1LL << geo.pb;
    x[0] = x0;
    x[1] = x0 | sb;
    x[2] = x0 | sa;
    x[3] = x0 | sa | sb;
    loc[0] = 0;
    loc[1] = 1;
    loc[2] = 2;
    loc[3] = 3;
    return 4;
}

// out_m[x with local a] = psi[x with local b] for member m = (a, b); every
// other amplitude of the item is 0.  One thread per (item, member).
__global__ void k_hole_apply(const double2 *psi, double2 *arr, const GateGeom geo, int log2B, int log2M,
                             int parity_members, int tile_parity, long long n_items) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int M = 1 << log2M;
    const long long Bm = (1LL << log2B) - 1;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n_items * M; t += stride) {
        const int m = (int)(t & (M - 1));
        const long long it = t >> log2M;
        const long long b = it & Bm, r = it >> log2B;
        long long x[4];
        int loc[4];
        const int na = item_amps(geo, r, tile_parity, x, loc);
        const int ea = c_members[parity_members][m][0], eb = c_members[parity_members][m][1];
        double2 src = make_double2(0.0, 0.0);
        for (int i = 0; i < na; ++i)
            if (loc[i] == eb) src = psi[(x[i] << log2B) | b];
        const long long col = ((long long)m << log2B) | b;
        for (int i = 0; i < na; ++i)
            arr[(x[i] << (log2B + log2M)) | col] = loc[i] == ea ? src : make_double2(0.0, 0.0);
    }
}

// Hole of gate l' between lambda (B columns) and array member m = blockIdx.y:
// part[m][cta][32] = sum conj(lambda[c]) arr_m[d] over the CTA's items.
__global__ void __launch_bounds__(kThreads, 1) k_array_env(const double2 *lam, const double2 *arr,
                                                           const GateGeom geo, int log2B, int log2M,
                                                           int tile_parity, long long n_items, double *part) {
    const int m = blockIdx.y;
    double2 E[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) E[i] = make_double2(0.0, 0.0);
    const long long Bm = (1LL << log2B) - 1;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long col_m = (long long)m << log2B;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < n_items; it += stride) {
        const long long b = it & Bm, r = it >> log2B;
        long long x[4];
        int loc[4];
        const int na = item_amps(geo, r, tile_parity, x, loc);
        if (na == 4) {
            double2 l[4], p[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                l[i] = lam[(x[i] << log2B) | b];
                p[i] = arr[(x[i] << (log2B + log2M)) | col_m | b];
            }
            if (geo.mode == kGeneral) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int c = 0; c < 4; ++c) cmacc(E[i * 4 + c], l[i], p[c]);
            } else {
                cmacc(E[0], l[0], p[0]); cmacc(E[3], l[0], p[3]); cmacc(E[12], l[3], p[0]); cmacc(E[15], l[3], p[3]);
                cmacc(E[5], l[1], p[1]); cmacc(E[6], l[1], p[2]); cmacc(E[9], l[2], p[1]); cmacc(E[10], l[2], p[2]);
            }
        } else {
            const double2 l0 = lam[(x[0] << log2B) | b], l1 = lam[(x[1] << log2B) | b];
            const double2 p0 = arr[(x[0] << (log2B + log2M)) | col_m | b];
            const double2 p1 = arr[(x[1] << (log2B + log2M)) | col_m | b];
            double2 c00 = make_double2(0, 0), c01 = c00, c10 = c00, c11 = c00;
            cmacc(c00, l0, p0); cmacc(c01, l0, p1); cmacc(c10, l1, p0); cmacc(c11, l1, p1);
            const int i0 = loc[0];
            if (i0 == 0) {
                E[0].x += c00.x; E[0].y += c00.y; E[3].x += c01.x; E[3].y += c01.y;
                E[12].x += c10.x; E[12].y += c10.y; E[15].x += c11.x; E[15].y += c11.y;
            } else if (i0 == 1) {
                E[5].x += c00.x; E[5].y += c00.y; E[6].x += c01.x; E[6].y += c01.y;
                E[9].x += c10.x; E[9].y += c10.y; E[10].x += c11.x; E[10].y += c11.y;
            } else {
                E[10].x += c00.x; E[10].y += c00.y; E[9].x += c01.x; E[9].y += c01.y;
                E[6].x += c10.x; E[6].y += c10.y; E[5].x += c11.x; E[5].y += c11.y;
            }
        }
    }
    __shared__ double red[kThreads / 32][kEnvDoubles];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        double vx = E[i].x, vy = E[i].y;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vx += __shfl_xor_sync(0xffffffffu, vx, o);
            vy += __shfl_xor_sync(0xffffffffu, vy, o);
        }
        if (lane == 0) {
            red[warp][2 * i] = vx;
            red[warp][2 * i + 1] = vy;
        }
    }
    __syncthreads();
    if (threadIdx.x < kEnvDoubles) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) s += red[w][threadIdx.x];
        part[((long long)m * gridDim.x + blockIdx.x) * kEnvDoubles + threadIdx.x] = s;
    }
}

// hacc[row][32] += sum over CTAs of part[row][cta][32] (rows = gates x members)
__global__ void k_reduce_rows(const double *part, int ncta, double *hacc) {
    const long long row = blockIdx.x;
    const int t = threadIdx.x;
    double s = 0.0;
    for (int c = 0; c < ncta; ++c) s += part[(row * ncta + c) * kEnvDoubles + t];
    hacc[row * kEnvDoubles + t] += s;
}

}  // namespace

void launch_hole_apply(const double2 *psi, double2 *arr, const GateGeom &geo, int log2B, int log2M,
                       int parity_members, int tile_parity, long long n_items, int grid, cudaStream_t s) {
    k_hole_apply<<<grid, kThreads, 0, s>>>(psi, arr, geo, log2B, log2M, parity_members, tile_parity, n_items);
}

void launch_array_env(const double2 *lam, const double2 *arr, const GateGeom &geo, int log2B, int log2M,
                      int tile_parity, long long n_items, int ncta, double *part, cudaStream_t s) {
    dim3 grid(ncta, 1u << log2M);
    k_array_env<<<grid, kThreads, 0, s>>>(lam, arr, geo, log2B, log2M, tile_parity, n_items, part);
}

void launch_reduce_rows(const double *part, int ncta, long long rows, double *hacc, cudaStream_t s) {
    if (rows <= 0) return;
    k_reduce_rows<<<(unsigned)rows, kEnvDoubles, 0, s>>>(part, ncta, hacc);
}

}  // namespace rq
