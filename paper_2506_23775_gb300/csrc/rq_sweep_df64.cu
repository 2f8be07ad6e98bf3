// Double-float ("df64") variant of the sweep kernels.
//
// GB300 executes FP64 at 2 DFMA per clock per SM but FP32 at 128 FMA per
// clock per SM.  These kernels keep every amplitude and gate entry as an
// unevaluated sum of two floats, x = hi + lo with |lo| <= ulp(hi) / 2 (about
// 48 significant bits), and run the gate applications and gate-hole
// contractions of the sweep (same operations, same order of columns and
// gates as the FP64 kernels in rq_sweep.cu) on the FP32 pipe:
//
//   * a product of two df64 numbers is hi*hi split exactly by an FMA
//     (Dekker's two-product with a fused multiply-add) plus the two cross
//     terms hi*lo + lo*hi; lo*lo (below 2^-48 relative) is dropped;
//   * products are summed with Knuth's error-free two-sum on the high parts,
//     the rounding errors and low parts collected in a float, and the result
//     renormalised by one more two-sum (the compensated dot product of Ogita,
//     Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput.
//     26 (2005), in its twice-the-working-precision form).
//
// The storage of a complex amplitude is a float4 (re.hi, re.lo, im.hi,
// im.lo): 16 bytes, like complex128, so tiles and checkpoints keep their
// layout.  Environments are accumulated per thread in df64, converted to FP64
// and reduced with the same fixed-order FP64 reductions as the FP64 path; the
// target overlap, the reductions and the Riemannian post-processing stay FP64.
// Every float operation below is an explicitly rounded intrinsic, so the
// compiler can neither contract nor reassociate the error-free transforms.
#include "rq_items.cuh"

#include <algorithm>

namespace rq {
namespace {

struct Acc {
    float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// a = x * y (first term of a sum)
__device__ __forceinline__ void acc_set(Acc &a, float xh, float xl, float yh, float yl) {
    a.h = __fmul_rn(xh, yh);
    float e = __fmaf_rn(xh, yh, -a.h);
    e = __fmaf_rn(xh, yl, e);
    a.l = __fmaf_rn(xl, yh, e);
}

// a += x * y
__device__ __forceinline__ void acc_mac(Acc &a, float xh, float xl, float yh, float yl) {
    const float p = __fmul_rn(xh, yh);
    float e = __fmaf_rn(xh, yh, -p);
    e = __fmaf_rn(xh, yl, e);
    e = __fmaf_rn(xl, yh, e);
    float s, t;
    two_sum(a.h, p, s, t);
    a.h = s;
    a.l = __fadd_rn(a.l, __fadd_rn(t, e));
}

struct CAcc {
    Acc re, im;
};

__device__ __forceinline__ CAcc czero() { return CAcc{{0.f, 0.f}, {0.f, 0.f}}; }

// c = g * x (complex, first term)
__device__ __forceinline__ void cset(CAcc &c, const float4 g, const float4 x) {
    acc_set(c.re, g.x, g.y, x.x, x.y);
    acc_mac(c.re, -g.z, -g.w, x.z, x.w);
    acc_set(c.im, g.x, g.y, x.z, x.w);
    acc_mac(c.im, g.z, g.w, x.x, x.y);
}

// c += g * x
__device__ __forceinline__ void cmac(CAcc &c, const float4 g, const float4 x) {
    acc_mac(c.re, g.x, g.y, x.x, x.y);
    acc_mac(c.re, -g.z, -g.w, x.z, x.w);
    acc_mac(c.im, g.x, g.y, x.z, x.w);
    acc_mac(c.im, g.z, g.w, x.x, x.y);
}

// c += conj(a) * b
__device__ __forceinline__ void cmacc(CAcc &c, const float4 a, const float4 b) {
    acc_mac(c.re, a.x, a.y, b.x, b.y);
    acc_mac(c.re, a.z, a.w, b.z, b.w);
    acc_mac(c.im, a.x, a.y, b.z, b.w);
    acc_mac(c.im, -a.z, -a.w, b.x, b.y);
}

// c = conj(a) * b (first term)
__device__ __forceinline__ void csetc(CAcc &c, const float4 a, const float4 b) {
    acc_set(c.re, a.x, a.y, b.x, b.y);
    acc_mac(c.re, a.z, a.w, b.z, b.w);
    acc_set(c.im, a.x, a.y, b.z, b.w);
    acc_mac(c.im, -a.z, -a.w, b.x, b.y);
}

__device__ __forceinline__ float4 fin(const CAcc &c) {
    float4 r;
    two_sum(c.re.h, c.re.l, r.x, r.y);
    two_sum(c.im.h, c.im.l, r.z, r.w);
    return r;
}

__device__ __forceinline__ double2 to_double(const CAcc &c) {
    return make_double2((double)c.re.h + (double)c.re.l, (double)c.im.h + (double)c.im.l);
}

// df64 sum a + b, renormalised (two-sum of the high parts, low parts and the
// rounding error added, one more two-sum)
__device__ __forceinline__ float2 df_add(float ah, float al, float bh, float bl) {
    float s, e;
    two_sum(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    float h, l;
    two_sum(s, e, h, l);
    return make_float2(h, l);
}

// General gates in the forward sweep use the three-product form (as the FP64
// kernels do), in its one-sum variant: for m = a + ib and x = u + iv,
// m x = (k - (a + b) v) + i (k + (b - a) u) with k = a (u + v).  In df64 a
// product term costs as much as before but the sum u + v is formed once per
// amplitude and serves all four rows, and a, -(a + b), b - a once per gate
// entry.
struct MatDf3 {
    float2 a[16], ns[16], d[16];  // a, -(a + b), b - a
};

__device__ __forceinline__ void tabulate_df3(MatDf3 &m, const float4 *g, int e) {
    const float4 x = g[e];
    const float2 s = df_add(x.x, x.y, x.z, x.w);
    m.a[e] = make_float2(x.x, x.y);
    m.ns[e] = make_float2(-s.x, -s.y);
    m.d[e] = df_add(x.z, x.w, -x.x, -x.y);
}

// x = u + iv with S = u + v
struct AmpDf3 {
    float uh, ul, vh, vl;
    float2 S;
};

__device__ __forceinline__ AmpDf3 amp_df3(const float4 x) {
    AmpDf3 r;
    r.uh = x.x;
    r.ul = x.y;
    r.vh = x.z;
    r.vl = x.w;
    r.S = df_add(x.x, x.y, x.z, x.w);
    return r;
}

// Local indices that a parity gate couples within its even block {0, 3} and
// odd block {1, 2}: out[i] = sum over c in block(i).
__device__ __forceinline__ int blk(int i, int u) {
    // u = 0, 1: the two members of i's block
    return (i == 0 || i == 3) ? (u == 0 ? 0 : 3) : (u == 0 ? 1 : 2);
}

// y = G x for a general gate in the three-product form (rows finished).
__device__ __forceinline__ void df_matvec3(const MatDf3 &m, const AmpDf3 (&x)[4], float4 (&y)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        Acc k;
        acc_set(k, m.a[i * 4].x, m.a[i * 4].y, x[0].S.x, x[0].S.y);
#pragma unroll
        for (int c = 1; c < 4; ++c) acc_mac(k, m.a[i * 4 + c].x, m.a[i * 4 + c].y, x[c].S.x, x[c].S.y);
        CAcc q{k, k};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            acc_mac(q.re, m.ns[i * 4 + c].x, m.ns[i * 4 + c].y, x[c].vh, x[c].vl);
            acc_mac(q.im, m.d[i * 4 + c].x, m.d[i * 4 + c].y, x[c].uh, x[c].ul);
        }
        y[i] = fin(q);
    }
}

// y = G t + X x (a tangent step), three-product form.
__device__ __forceinline__ void df_matvec3_pair(const MatDf3 &m, const AmpDf3 (&t)[4], const MatDf3 &n,
                                                const AmpDf3 (&x)[4], float4 (&y)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        Acc k;
        acc_set(k, m.a[i * 4].x, m.a[i * 4].y, t[0].S.x, t[0].S.y);
#pragma unroll
        for (int c = 1; c < 4; ++c) acc_mac(k, m.a[i * 4 + c].x, m.a[i * 4 + c].y, t[c].S.x, t[c].S.y);
#pragma unroll
        for (int c = 0; c < 4; ++c) acc_mac(k, n.a[i * 4 + c].x, n.a[i * 4 + c].y, x[c].S.x, x[c].S.y);
        CAcc q{k, k};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            acc_mac(q.re, m.ns[i * 4 + c].x, m.ns[i * 4 + c].y, t[c].vh, t[c].vl);
            acc_mac(q.re, n.ns[i * 4 + c].x, n.ns[i * 4 + c].y, x[c].vh, x[c].vl);
            acc_mac(q.im, m.d[i * 4 + c].x, m.d[i * 4 + c].y, t[c].uh, t[c].ul);
            acc_mac(q.im, n.d[i * 4 + c].x, n.d[i * 4 + c].y, x[c].uh, x[c].ul);
        }
        y[i] = fin(q);
    }
}

// y = G p for a parity gate on two stored qubits (two terms per row).
__device__ __forceinline__ void df_blocks(const float4 *g, const float4 (&p)[4], float4 (&y)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        CAcc q;
        cset(q, g[i * 4 + blk(i, 0)], p[blk(i, 0)]);
        cmac(q, g[i * 4 + blk(i, 1)], p[blk(i, 1)]);
        y[i] = fin(q);
    }
}

// y = G t + X p for a parity gate on two stored qubits.
__device__ __forceinline__ void df_blocks_pair(const float4 *g, const float4 (&t)[4], const float4 *xm,
                                               const float4 (&p)[4], float4 (&y)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        CAcc q;
        cset(q, g[i * 4 + blk(i, 0)], t[blk(i, 0)]);
        cmac(q, g[i * 4 + blk(i, 1)], t[blk(i, 1)]);
        cmac(q, xm[i * 4 + blk(i, 0)], p[blk(i, 0)]);
        cmac(q, xm[i * 4 + blk(i, 1)], p[blk(i, 1)]);
        y[i] = fin(q);
    }
}

__device__ __forceinline__ void offsets2(long long r, long long b, int p, int qfirst, int parity, int log2B,
                                         long long (&off)[2], int &i0, int &i1) {
    const long long y0 = insert_zero(r, p);
    off[0] = (y0 << log2B) | b;
    off[1] = ((y0 | (1LL << p)) << log2B) | b;
    const int e = (__popcll(y0) & 1) ^ parity;
    if (e == 0) {
        i0 = 0;
        i1 = 3;
    } else if (qfirst) {
        i0 = 1;
        i1 = 2;
    } else {
        i0 = 2;
        i1 = 1;
    }
}

__device__ __forceinline__ void block_reduce_store(const CAcc (&acc)[16], double *out) {
    __shared__ double red[kThreads / 32][kEnvDoubles];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const double2 v = to_double(acc[i]);
        double vx = v.x, vy = v.y;
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
        out[threadIdx.x] = s;
    }
}

// ---------------------------------------------------------------- forward --

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) k_fwd_df(const FwdArgs a) {
    __shared__ float4 sg[16];
    __shared__ float4 sx[kMaxDirs][16];
    __shared__ MatDf3 sg3;
    __shared__ MatDf3 sx3[kMaxDirs];
    const float4 *gate = reinterpret_cast<const float4 *>(a.gate);
    const float4 *dirs = reinterpret_cast<const float4 *>(a.dirs);
    if (MODE == kGeneral) {
        if (threadIdx.x < 16) tabulate_df3(sg3, gate, threadIdx.x);
        if (threadIdx.x < 16 * a.kdirs)
            tabulate_df3(sx3[threadIdx.x >> 4], dirs + (threadIdx.x >> 4) * a.xdir_stride, threadIdx.x & 15);
    } else {
        if (threadIdx.x < 16) sg[threadIdx.x] = gate[threadIdx.x];
        if (threadIdx.x < 16 * a.kdirs)
            sx[threadIdx.x >> 4][threadIdx.x & 15] = dirs[(threadIdx.x >> 4) * a.xdir_stride + (threadIdx.x & 15)];
    }
    __syncthreads();
    const float4 *psi_in = reinterpret_cast<const float4 *>(a.psi_in);
    float4 *psi_out = reinterpret_cast<float4 *>(a.psi_out);
    const float4 *dpsi_in = reinterpret_cast<const float4 *>(a.dpsi_in);
    float4 *dpsi_out = reinterpret_cast<float4 *>(a.dpsi_out);
    const long long Bm = (1LL << a.log2B) - 1;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long it = first_item(); it < a.n_items; it += stride) {
        const long long b = it & Bm, r = it >> a.log2B;
        if constexpr (MODE == kGeneral) {
            long long off[4];
            if (!item_offsets4(a.geo, a.cols, r, b, a.log2B, off)) continue;
            AmpDf3 x[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) x[c] = amp_df3(__ldg(&psi_in[off[c]]));
            float4 y[4];
            df_matvec3(sg3, x, y);
#pragma unroll
            for (int i = 0; i < 4; ++i) psi_out[off[i]] = y[i];
            for (int d = 0; d < a.kdirs; ++d) {
                const float4 *din = dpsi_in + d * a.dir_stride;
                float4 *dout = dpsi_out + d * a.dir_stride;
                AmpDf3 t[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) t[c] = amp_df3(__ldg(&din[off[c]]));
                df_matvec3_pair(sg3, t, sx3[d], x, y);  // G psi' + X psi
#pragma unroll
                for (int i = 0; i < 4; ++i) dout[off[i]] = y[i];
            }
        } else if constexpr (MODE == kParity4) {
            long long off[4];
            if (!item_offsets4(a.geo, a.cols, r, b, a.log2B, off)) continue;
            float4 p[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) p[c] = __ldg(&psi_in[off[c]]);
            float4 y[4];
            df_blocks(sg, p, y);
#pragma unroll
            for (int i = 0; i < 4; ++i) psi_out[off[i]] = y[i];
            for (int d = 0; d < a.kdirs; ++d) {
                const float4 *din = dpsi_in + d * a.dir_stride;
                float4 *dout = dpsi_out + d * a.dir_stride;
                float4 t[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) t[c] = __ldg(&din[off[c]]);
                df_blocks_pair(sg, t, sx[d], p, y);
#pragma unroll
                for (int i = 0; i < 4; ++i) dout[off[i]] = y[i];
            }
        } else {  // kParity2
            long long off[2];
            int i0, i1;
            offsets2(r, b, a.geo.pa, a.geo.qfirst, a.tile_parity, a.log2B, off, i0, i1);
            const float4 p0 = __ldg(&psi_in[off[0]]), p1 = __ldg(&psi_in[off[1]]);
            CAcc q0, q1;
            cset(q0, sg[i0 * 4 + i0], p0);
            cmac(q0, sg[i0 * 4 + i1], p1);
            cset(q1, sg[i1 * 4 + i0], p0);
            cmac(q1, sg[i1 * 4 + i1], p1);
            psi_out[off[0]] = fin(q0);
            psi_out[off[1]] = fin(q1);
            for (int d = 0; d < a.kdirs; ++d) {
                const float4 *din = dpsi_in + d * a.dir_stride;
                float4 *dout = dpsi_out + d * a.dir_stride;
                const float4 t0 = __ldg(&din[off[0]]), t1 = __ldg(&din[off[1]]);
                cset(q0, sg[i0 * 4 + i0], t0);
                cmac(q0, sg[i0 * 4 + i1], t1);
                cmac(q0, sx[d][i0 * 4 + i0], p0);
                cmac(q0, sx[d][i0 * 4 + i1], p1);
                cset(q1, sg[i1 * 4 + i0], t0);
                cmac(q1, sg[i1 * 4 + i1], t1);
                cmac(q1, sx[d][i1 * 4 + i0], p0);
                cmac(q1, sx[d][i1 * 4 + i1], p1);
                dout[off[0]] = fin(q0);
                dout[off[1]] = fin(q1);
            }
        }
    }
}

// ---------------------------------------------------------- backward base --

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) k_bwd_base_df(const BwdArgs a) {
    __shared__ float4 sg[16];
    const float4 *gate = reinterpret_cast<const float4 *>(a.gate);
    if (threadIdx.x < 16) sg[threadIdx.x] = gate[threadIdx.x];
    __syncthreads();
    float4 *lam = reinterpret_cast<float4 *>(a.lam);
    const float4 *psi = reinterpret_cast<const float4 *>(a.psi);
    const int accumulate = a.accumulate;
    CAcc E[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) E[i] = czero();
    const long long Bm = (1LL << a.log2B) - 1;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long it = first_item(); it < a.n_items; it += stride) {
        const long long b = it & Bm, r = it >> a.log2B;
        if (MODE == kGeneral || MODE == kParity4) {
            long long off[4];
            if (!item_offsets4(a.geo, a.cols, r, b, a.log2B, off)) continue;
            float4 l[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) l[c] = lam[off[c]];
            if (accumulate) {
                float4 p[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) p[c] = __ldg(&psi[off[c]]);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (MODE == kGeneral) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) cmacc(E[i * 4 + c], l[i], p[c]);
                    } else {
#pragma unroll
                        for (int u = 0; u < 2; ++u) cmacc(E[i * 4 + blk(i, u)], l[i], p[blk(i, u)]);
                    }
                }
            }
            if (a.update) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    CAcc q;
                    if (MODE == kGeneral) {
                        csetc(q, sg[0 * 4 + i], l[0]);
#pragma unroll
                        for (int c = 1; c < 4; ++c) cmacc(q, sg[c * 4 + i], l[c]);
                    } else {
                        csetc(q, sg[blk(i, 0) * 4 + i], l[blk(i, 0)]);
                        cmacc(q, sg[blk(i, 1) * 4 + i], l[blk(i, 1)]);
                    }
                    lam[off[i]] = fin(q);
                }
            }
        } else {  // kParity2
            long long off[2];
            int i0, i1;
            offsets2(r, b, a.geo.pa, a.geo.qfirst, a.tile_parity, a.log2B, off, i0, i1);
            const float4 l0 = lam[off[0]], l1 = lam[off[1]];
            if (accumulate) {
                const float4 p0 = __ldg(&psi[off[0]]), p1 = __ldg(&psi[off[1]]);
                // E[i0][i0], E[i0][i1], E[i1][i0], E[i1][i1], static indices per block
                if (i0 == 0) {
                    cmacc(E[0], l0, p0); cmacc(E[3], l0, p1); cmacc(E[12], l1, p0); cmacc(E[15], l1, p1);
                } else if (i0 == 1) {
                    cmacc(E[5], l0, p0); cmacc(E[6], l0, p1); cmacc(E[9], l1, p0); cmacc(E[10], l1, p1);
                } else {
                    cmacc(E[10], l0, p0); cmacc(E[9], l0, p1); cmacc(E[6], l1, p0); cmacc(E[5], l1, p1);
                }
            }
            if (a.update) {
                CAcc q0, q1;
                csetc(q0, sg[i0 * 4 + i0], l0);
                cmacc(q0, sg[i1 * 4 + i0], l1);
                csetc(q1, sg[i0 * 4 + i1], l0);
                cmacc(q1, sg[i1 * 4 + i1], l1);
                lam[off[0]] = fin(q0);
                lam[off[1]] = fin(q1);
            }
        }
    }
    if (accumulate) block_reduce_store(E, a.part + (long long)blockIdx.x * kEnvDoubles);
}

// ----------------------------------------------------- backward direction --

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) k_bwd_dir_df(const BwdArgs a) {
    __shared__ float4 sg[16];
    __shared__ float4 sx[16];
    const float4 *gate = reinterpret_cast<const float4 *>(a.gate);
    const float4 *dir = reinterpret_cast<const float4 *>(a.dir);
    if (threadIdx.x < 16) {
        sg[threadIdx.x] = gate[threadIdx.x];
        sx[threadIdx.x] = dir[threadIdx.x];
    }
    __syncthreads();
    const float4 *lam = reinterpret_cast<const float4 *>(a.lam);
    float4 *dlam = reinterpret_cast<float4 *>(a.dlam);
    const float4 *psi = reinterpret_cast<const float4 *>(a.psi);
    const float4 *dpsi = reinterpret_cast<const float4 *>(a.dpsi);
    CAcc E[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) E[i] = czero();
    const long long Bm = (1LL << a.log2B) - 1;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long it = first_item(); it < a.n_items; it += stride) {
        const long long b = it & Bm, r = it >> a.log2B;
        if (MODE == kGeneral || MODE == kParity4) {
            long long off[4];
            if (!item_offsets4(a.geo, a.cols, r, b, a.log2B, off)) continue;
            float4 l[4], dl[4], p[4], dp[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                l[c] = __ldg(&lam[off[c]]);
                dl[c] = dlam[off[c]];
                p[c] = __ldg(&psi[off[c]]);
                dp[c] = __ldg(&dpsi[off[c]]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (MODE == kGeneral) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        cmacc(E[i * 4 + c], dl[i], p[c]);
                        cmacc(E[i * 4 + c], l[i], dp[c]);
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        cmacc(E[i * 4 + blk(i, u)], dl[i], p[blk(i, u)]);
                        cmacc(E[i * 4 + blk(i, u)], l[i], dp[blk(i, u)]);
                    }
                }
            }
            if (a.update) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    CAcc q;
                    if (MODE == kGeneral) {
                        csetc(q, sg[0 * 4 + i], dl[0]);
#pragma unroll
                        for (int c = 1; c < 4; ++c) cmacc(q, sg[c * 4 + i], dl[c]);
#pragma unroll
                        for (int c = 0; c < 4; ++c) cmacc(q, sx[c * 4 + i], l[c]);
                    } else {
                        csetc(q, sg[blk(i, 0) * 4 + i], dl[blk(i, 0)]);
                        cmacc(q, sg[blk(i, 1) * 4 + i], dl[blk(i, 1)]);
                        cmacc(q, sx[blk(i, 0) * 4 + i], l[blk(i, 0)]);
                        cmacc(q, sx[blk(i, 1) * 4 + i], l[blk(i, 1)]);
                    }
                    dlam[off[i]] = fin(q);
                }
            }
        } else {  // kParity2
            long long off[2];
            int i0, i1;
            offsets2(r, b, a.geo.pa, a.geo.qfirst, a.tile_parity, a.log2B, off, i0, i1);
            const float4 l0 = __ldg(&lam[off[0]]), l1 = __ldg(&lam[off[1]]);
            const float4 d0 = dlam[off[0]], d1 = dlam[off[1]];
            const float4 p0 = __ldg(&psi[off[0]]), p1 = __ldg(&psi[off[1]]);
            const float4 t0 = __ldg(&dpsi[off[0]]), t1 = __ldg(&dpsi[off[1]]);
            if (i0 == 0) {
                cmacc(E[0], d0, p0); cmacc(E[0], l0, t0); cmacc(E[3], d0, p1); cmacc(E[3], l0, t1);
                cmacc(E[12], d1, p0); cmacc(E[12], l1, t0); cmacc(E[15], d1, p1); cmacc(E[15], l1, t1);
            } else if (i0 == 1) {
                cmacc(E[5], d0, p0); cmacc(E[5], l0, t0); cmacc(E[6], d0, p1); cmacc(E[6], l0, t1);
                cmacc(E[9], d1, p0); cmacc(E[9], l1, t0); cmacc(E[10], d1, p1); cmacc(E[10], l1, t1);
            } else {
                cmacc(E[10], d0, p0); cmacc(E[10], l0, t0); cmacc(E[9], d0, p1); cmacc(E[9], l0, t1);
                cmacc(E[6], d1, p0); cmacc(E[6], l1, t0); cmacc(E[5], d1, p1); cmacc(E[5], l1, t1);
            }
            if (a.update) {
                CAcc q0, q1;
                csetc(q0, sg[i0 * 4 + i0], d0);
                cmacc(q0, sg[i1 * 4 + i0], d1);
                cmacc(q0, sx[i0 * 4 + i0], l0);
                cmacc(q0, sx[i1 * 4 + i0], l1);
                csetc(q1, sg[i0 * 4 + i1], d0);
                cmacc(q1, sg[i1 * 4 + i1], d1);
                cmacc(q1, sx[i0 * 4 + i1], l0);
                cmacc(q1, sx[i1 * 4 + i1], l1);
                dlam[off[0]] = fin(q0);
                dlam[off[1]] = fin(q1);
            }
        }
    }
    block_reduce_store(E, a.part + (long long)blockIdx.x * kEnvDoubles);
}

// ------------------------------------------- two threads per item (4-amp) --
//
// The environment accumulators dominate the registers of the df64 backward
// kernels (16 complex df64 sums = 64 floats).  For gates whose items have four
// amplitudes, two adjacent lanes share an item: lane h accumulates the
// environment rows {2h, 2h+1} and writes the updated amplitudes {2h, 2h+1}.
// Half the accumulators per thread lets two CTAs share an SM (twice the
// resident warps to hide memory latency); the pair's loads coalesce into the
// same transactions.

// Block sum of the 8 entries each lane holds: even lanes carry rows {0, 1}
// (entries 0..7), odd lanes rows {2, 3} (entries 8..15).
__device__ __forceinline__ void block_reduce_store_half(const CAcc (&acc)[8], double *out) {
    __shared__ double red[kThreads / 32][kEnvDoubles];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const double2 v = to_double(acc[i]);
        double vx = v.x, vy = v.y;
#pragma unroll
        for (int o = 16; o > 1; o >>= 1) {  // sums over lanes of the same parity
            vx += __shfl_xor_sync(0xffffffffu, vx, o);
            vy += __shfl_xor_sync(0xffffffffu, vy, o);
        }
        if (lane < 2) {
            red[warp][2 * (lane * 8 + i)] = vx;
            red[warp][2 * (lane * 8 + i) + 1] = vy;
        }
    }
    __syncthreads();
    if (threadIdx.x < kEnvDoubles) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) s += red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// Lane h of a pair owns rows i = 2h + u, u = 0, 1.  Every register index is
// static; the lane's rows are picked with selects (no divergence, no local
// memory).  For a parity gate row i couples the columns of its block:
// {0, 3} if i is 0 or 3, else {1, 2}; "even" below is that test.
// 16-byte asynchronous copy global -> shared (the copying thread sees the data
// after cp.async.wait_group; its partner lane after a __syncwarp)
__device__ __forceinline__ void cp_async16_f4(float4 *smem, const float4 *gmem) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_df() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_df() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// k_bwd_dir_df2 keeps two stages of its items' 16 amplitudes per lane pair in
// dynamic shared memory: slot (stage, c) of pair q at [(stage * 16 + c) *
// (kThreads / 2) + q].  Lane 0 of a pair copies lambda and lambda', lane 1
// psi and psi', while the previous item is computed.
constexpr size_t kDirDfSmem = sizeof(float4) * 2 * 16 * (kThreads / 2);
constexpr size_t kBaseDfSmem = sizeof(float4) * 2 * 8 * (kThreads / 2);

template <int MODE>
__global__ void __launch_bounds__(kThreads, 2) k_bwd_dir_df2(const BwdArgs a) {
    __shared__ float4 sg[16];
    __shared__ float4 sx[16];
    extern __shared__ float4 stage_df[];
    const float4 *gate = reinterpret_cast<const float4 *>(a.gate);
    const float4 *dir = reinterpret_cast<const float4 *>(a.dir);
    if (threadIdx.x < 16) {
        sg[threadIdx.x] = gate[threadIdx.x];
        sx[threadIdx.x] = dir[threadIdx.x];
    }
    __syncthreads();
    const float4 *lam = reinterpret_cast<const float4 *>(a.lam);
    float4 *dlam = reinterpret_cast<float4 *>(a.dlam);
    const float4 *psi = reinterpret_cast<const float4 *>(a.psi);
    const float4 *dpsi = reinterpret_cast<const float4 *>(a.dpsi);
    CAcc E[8];  // general: E[u*4 + c]; parity: E[u*4 + k], k = 0, 1 the block columns
#pragma unroll
    for (int i = 0; i < 8; ++i) E[i] = czero();
    const int h = threadIdx.x & 1;
    // the mask names only the pair, whose lanes always run the same iterations
    const unsigned pair_mask = 0x3u << (threadIdx.x & 30);
    float4 *mine = stage_df + (threadIdx.x >> 1);
    const float4 *src0 = h ? psi : lam;
    const float4 *src1 = h ? dpsi : reinterpret_cast<const float4 *>(dlam);
    auto issue = [&](const long long (&o)[4], int st) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            cp_async16_f4(mine + (st * 16 + 8 * h + c) * (kThreads / 2), src0 + o[c]);
            cp_async16_f4(mine + (st * 16 + 8 * h + 4 + c) * (kThreads / 2), src1 + o[c]);
        }
    };
    const long long Bm = (1LL << a.log2B) - 1;
    const long long stride = ((long long)gridDim.x * blockDim.x) >> 1;
    long long it = first_pair_item();
    long long off[4], nxt[4];
    bool ok = false;
    if (it < a.n_items) {
        ok = item_offsets4(a.geo, a.cols, it >> a.log2B, it & Bm, a.log2B, off) &&
             (MODE != kGeneral || tail_live(a.geo, a.cols, it & Bm, off[0] >> a.log2B));
        if (ok) issue(off, 0);
    }
    cp_async_commit_df();
    int st = 0;
    for (; it < a.n_items; it += stride) {
        __syncwarp(pair_mask);  // both lanes have read the stage about to be refilled
        bool ok_next = false;
        if (it + stride < a.n_items) {
            ok_next = item_offsets4(a.geo, a.cols, (it + stride) >> a.log2B, (it + stride) & Bm, a.log2B, nxt) &&
                      (MODE != kGeneral || tail_live(a.geo, a.cols, (it + stride) & Bm, nxt[0] >> a.log2B));
            if (ok_next) issue(nxt, st ^ 1);
        }
        cp_async_commit_df();
        cp_async_wait_df<1>();
        __syncwarp(pair_mask);  // the partner's copies of this item are visible
        if (ok) {
            float4 l[4], dl[4], p[4], dp[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                l[c] = mine[(st * 16 + c) * (kThreads / 2)];
                dl[c] = mine[(st * 16 + 4 + c) * (kThreads / 2)];
                p[c] = mine[(st * 16 + 8 + c) * (kThreads / 2)];
                dp[c] = mine[(st * 16 + 12 + c) * (kThreads / 2)];
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float4 li = h ? l[2 + u] : l[u];
                const float4 dli = h ? dl[2 + u] : dl[u];
                if (MODE == kGeneral) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        cmacc(E[u * 4 + c], dli, p[c]);
                        cmacc(E[u * 4 + c], li, dp[c]);
                    }
                } else {
                    const bool even = (h == 0) == (u == 0);
                    const float4 pa = even ? p[0] : p[1], pb = even ? p[3] : p[2];
                    const float4 qa = even ? dp[0] : dp[1], qb = even ? dp[3] : dp[2];
                    cmacc(E[u * 4 + 0], dli, pa);
                    cmacc(E[u * 4 + 0], li, qa);
                    cmacc(E[u * 4 + 1], dli, pb);
                    cmacc(E[u * 4 + 1], li, qb);
                }
            }
            if (a.update) {
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int i = 2 * h + u;
                    CAcc q;
                    if (MODE == kGeneral) {
                        csetc(q, sg[0 * 4 + i], dl[0]);
#pragma unroll
                        for (int c = 1; c < 4; ++c) cmacc(q, sg[c * 4 + i], dl[c]);
#pragma unroll
                        for (int c = 0; c < 4; ++c) cmacc(q, sx[c * 4 + i], l[c]);
                    } else {
                        const bool even = (h == 0) == (u == 0);
                        const int c0 = even ? 0 : 1, c1 = even ? 3 : 2;
                        csetc(q, sg[c0 * 4 + i], even ? dl[0] : dl[1]);
                        cmacc(q, sg[c1 * 4 + i], even ? dl[3] : dl[2]);
                        cmacc(q, sx[c0 * 4 + i], even ? l[0] : l[1]);
                        cmacc(q, sx[c1 * 4 + i], even ? l[3] : l[2]);
                    }
                    const long long oi = h ? off[2 + u] : off[u];
                    dlam[oi] = fin(q);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) off[c] = nxt[c];
        ok = ok_next;
        st ^= 1;
    }
    cp_async_wait_df<0>();
    if (MODE != kGeneral) {
        // spread the block columns to their 4x4 positions: row 2h+u, columns c0, c1
#pragma unroll
        for (int u = 1; u >= 0; --u) {
            const bool even = (h == 0) == (u == 0);
            const CAcc k0 = E[u * 4 + 0], k1 = E[u * 4 + 1];
            E[u * 4 + 0] = even ? k0 : czero();
            E[u * 4 + 1] = even ? czero() : k0;
            E[u * 4 + 2] = even ? czero() : k1;
            E[u * 4 + 3] = even ? k1 : czero();
        }
    }
    block_reduce_store_half(E, a.part + (long long)blockIdx.x * kEnvDoubles);
}

// Base step with two lanes per item (same row split as k_bwd_dir_df2).
template <int MODE>
__global__ void __launch_bounds__(kThreads, 2) k_bwd_base_df2(const BwdArgs a) {
    __shared__ float4 sg[16];
    extern __shared__ float4 stage_df[];  // [2][8][kThreads / 2]: lambda (lane 0), psi (lane 1)
    const float4 *gate = reinterpret_cast<const float4 *>(a.gate);
    if (threadIdx.x < 16) sg[threadIdx.x] = gate[threadIdx.x];
    __syncthreads();
    float4 *lam = reinterpret_cast<float4 *>(a.lam);
    const float4 *psi = reinterpret_cast<const float4 *>(a.psi);
    const int accumulate = a.accumulate;
    CAcc E[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) E[i] = czero();
    const int h = threadIdx.x & 1;
    const unsigned pair_mask = 0x3u << (threadIdx.x & 30);
    float4 *mine = stage_df + (threadIdx.x >> 1);
    const float4 *src = h ? psi : reinterpret_cast<const float4 *>(lam);
    const bool copies = h == 0 || accumulate;
    auto issue = [&](const long long (&o)[4], int st) {
        if (!copies) return;
#pragma unroll
        for (int c = 0; c < 4; ++c) cp_async16_f4(mine + (st * 8 + 4 * h + c) * (kThreads / 2), src + o[c]);
    };
    const long long Bm = (1LL << a.log2B) - 1;
    const long long stride = ((long long)gridDim.x * blockDim.x) >> 1;
    long long it = first_pair_item();
    long long off[4], nxt[4];
    bool ok = false;
    if (it < a.n_items) {
        ok = item_offsets4(a.geo, a.cols, it >> a.log2B, it & Bm, a.log2B, off) &&
             (MODE != kGeneral || tail_live(a.geo, a.cols, it & Bm, off[0] >> a.log2B));
        if (ok) issue(off, 0);
    }
    cp_async_commit_df();
    int st = 0;
    for (; it < a.n_items; it += stride) {
        __syncwarp(pair_mask);  // both lanes have read the stage about to be refilled
        bool ok_next = false;
        if (it + stride < a.n_items) {
            ok_next = item_offsets4(a.geo, a.cols, (it + stride) >> a.log2B, (it + stride) & Bm, a.log2B, nxt) &&
                      (MODE != kGeneral || tail_live(a.geo, a.cols, (it + stride) & Bm, nxt[0] >> a.log2B));
            if (ok_next) issue(nxt, st ^ 1);
        }
        cp_async_commit_df();
        cp_async_wait_df<1>();
        __syncwarp(pair_mask);  // the partner's copies of this item are visible
        if (ok) {
            float4 l[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) l[c] = mine[(st * 8 + c) * (kThreads / 2)];
            if (accumulate) {
                float4 p[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) p[c] = mine[(st * 8 + 4 + c) * (kThreads / 2)];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const float4 li = h ? l[2 + u] : l[u];
                    if (MODE == kGeneral) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) cmacc(E[u * 4 + c], li, p[c]);
                    } else {
                        const bool even = (h == 0) == (u == 0);
                        cmacc(E[u * 4 + 0], li, even ? p[0] : p[1]);
                        cmacc(E[u * 4 + 1], li, even ? p[3] : p[2]);
                    }
                }
            }
            if (a.update) {
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int i = 2 * h + u;
                    CAcc q;
                    if (MODE == kGeneral) {
                        csetc(q, sg[0 * 4 + i], l[0]);
#pragma unroll
                        for (int c = 1; c < 4; ++c) cmacc(q, sg[c * 4 + i], l[c]);
                    } else {
                        const bool even = (h == 0) == (u == 0);
                        const int c0 = even ? 0 : 1, c1 = even ? 3 : 2;
                        csetc(q, sg[c0 * 4 + i], even ? l[0] : l[1]);
                        cmacc(q, sg[c1 * 4 + i], even ? l[3] : l[2]);
                    }
                    const long long oi = h ? off[2 + u] : off[u];
                    lam[oi] = fin(q);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) off[c] = nxt[c];
        ok = ok_next;
        st ^= 1;
    }
    cp_async_wait_df<0>();
    if (!accumulate) return;
    if (MODE != kGeneral) {
#pragma unroll
        for (int u = 1; u >= 0; --u) {
            const bool even = (h == 0) == (u == 0);
            const CAcc k0 = E[u * 4 + 0], k1 = E[u * 4 + 1];
            E[u * 4 + 0] = even ? k0 : czero();
            E[u * 4 + 1] = even ? czero() : k0;
            E[u * 4 + 2] = even ? czero() : k1;
            E[u * 4 + 3] = even ? k1 : czero();
        }
    }
    block_reduce_store_half(E, a.part + (long long)blockIdx.x * kEnvDoubles);
}

// ------------------------------------------------------ fused forward pass --
//
// The double-float form of the fused forward pass of rq_sweep.cu: blocks of
// [2^q amplitudes x 32 columns] in shared memory, the pass's gates applied
// there with the same item arithmetic as k_fwd_df, outputs written where a
// checkpoint slot is wanted.  Per gate a 384-byte table: MatDf3 (general) or
// the 16 raw entries (parity gates on two stored qubits).
constexpr int kTabBytes = 384;
static_assert(sizeof(MatDf3) <= kTabBytes && 16 * sizeof(float4) <= kTabBytes, "gate table size");

template <int MODE, int KD>
__global__ void __launch_bounds__(kThreads, 2) k_fwd_fused_df(const FwdFusedArgs a) {
    extern __shared__ __align__(16) unsigned char fused_raw[];
    const FusedPass &p = a.pass;
    const int rows = 1 << p.q, m = p.m;
    const int elems = rows * 32, items = (rows >> 2) * 32;
    float4 *const Sb = reinterpret_cast<float4 *>(fused_raw);                            // [nbuf][1 + KD][rows][32]
    unsigned char *tab = reinterpret_cast<unsigned char *>(Sb + a.nbuf * (1 + KD) * elems);  // [(1 + KD) m][kTabBytes]
    long long *rowoff = reinterpret_cast<long long *>(tab + (size_t)(1 + KD) * m * kTabBytes);
    const float4 *gates = reinterpret_cast<const float4 *>(a.gates);
    const float4 *dirs = reinterpret_cast<const float4 *>(a.dirs);
    auto gtab = [&](int t) { return tab + (size_t)t * kTabBytes; };
    for (int e = threadIdx.x; e < m * 16; e += blockDim.x) {
        const int j = e >> 4, c = e & 15;
        const float4 *g = gates + (long long)p.param[j] * 16;
        if (MODE == kGeneral) tabulate_df3(*reinterpret_cast<MatDf3 *>(gtab(j)), g, c);
        else reinterpret_cast<float4 *>(gtab(j))[c] = g[c];
#pragma unroll
        for (int d = 0; d < KD; ++d) {
            const float4 *x = dirs + d * a.xdir_stride + (long long)p.param[j] * 16;
            if (MODE == kGeneral) tabulate_df3(*reinterpret_cast<MatDf3 *>(gtab((1 + d) * m + j)), x, c);
            else reinterpret_cast<float4 *>(gtab((1 + d) * m + j))[c] = x[c];
        }
    }
    for (int r = threadIdx.x; r < rows; r += blockDim.x) rowoff[r] = deposit_bits(r, p.wmask);
    __syncthreads();
    const float4 *psi_in = reinterpret_cast<const float4 *>(a.psi_in);
    const float4 *dpsi_in = reinterpret_cast<const float4 *>(a.dpsi_in);
    float4 *psi_base = reinterpret_cast<float4 *>(a.psi_base);
    float4 *dpsi_base = reinterpret_cast<float4 *>(a.dpsi_base);
    const long long cmask = (1LL << a.log2chunks) - 1;
    auto load = [&](long long blk, float4 *dst) {
        const long long x0 = deposit_bits(blk >> a.log2chunks, a.outer_mask);
        const long long col0 = (blk & cmask) << 5;
        for (int e = threadIdx.x; e < elems; e += blockDim.x) {
            const long long off = ((x0 | rowoff[e >> 5]) << a.log2B) | (col0 + (e & 31));
            cp_async16_f4(dst + e, psi_in + off);
#pragma unroll
            for (int d = 0; d < KD; ++d) cp_async16_f4(dst + (1 + d) * elems + e, dpsi_in + d * a.dir_stride + off);
        }
    };
    long long blk = blockIdx.x;
    if (blk < a.n_blocks) load(blk, Sb);
    cp_async_commit_df();
    int cur = 0;
    for (; blk < a.n_blocks; blk += gridDim.x) {
        const long long nxt = blk + gridDim.x;
        if (a.nbuf == 2) {
            if (nxt < a.n_blocks) load(nxt, Sb + (cur ^ 1) * (1 + KD) * elems);
            cp_async_commit_df();
            cp_async_wait_df<1>();  // this block's copies have landed
        } else {
            cp_async_wait_df<0>();
        }
        __syncthreads();
        float4 *S = Sb + cur * (1 + KD) * elems;
        const long long x0 = deposit_bits(blk >> a.log2chunks, a.outer_mask);
        const long long col0 = (blk & cmask) << 5;
        for (int j = 0; j < m; ++j) {
            const int la = p.la[j], lb = p.lb[j];
            const int lo = la < lb ? la : lb, hi = la < lb ? lb : la;
            const int slot = p.out_slot[j];
            for (int it = threadIdx.x; it < items; it += blockDim.x) {
                const int col = it & 31;
                const int r0 = (int)insert_zero(insert_zero(it >> 5, lo), hi);
                const int rw[4] = {r0, r0 | (1 << lb), r0 | (1 << la), r0 | (1 << la) | (1 << lb)};
                float4 v[4], y[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) v[c] = S[rw[c] * 32 + col];
                AmpDf3 x[4];
                if constexpr (MODE == kGeneral) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) x[c] = amp_df3(v[c]);
                    df_matvec3(*reinterpret_cast<const MatDf3 *>(gtab(j)), x, y);
                } else {
                    df_blocks(reinterpret_cast<const float4 *>(gtab(j)), v, y);
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) S[rw[c] * 32 + col] = y[c];
                if (slot >= 0) {
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        psi_base[slot * a.tile + (((x0 | rowoff[rw[c]]) << a.log2B) | (col0 + col))] = y[c];
                }
#pragma unroll
                for (int d = 0; d < KD; ++d) {
                    float4 *T = S + (1 + d) * elems;
                    if constexpr (MODE == kGeneral) {
                        AmpDf3 t[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) t[c] = amp_df3(T[rw[c] * 32 + col]);
                        df_matvec3_pair(*reinterpret_cast<const MatDf3 *>(gtab(j)), t,
                                        *reinterpret_cast<const MatDf3 *>(gtab((1 + d) * m + j)), x, y);
                    } else {
                        float4 t[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) t[c] = T[rw[c] * 32 + col];
                        df_blocks_pair(reinterpret_cast<const float4 *>(gtab(j)), t,
                                       reinterpret_cast<const float4 *>(gtab((1 + d) * m + j)), v, y);
                    }
#pragma unroll
                    for (int c = 0; c < 4; ++c) T[rw[c] * 32 + col] = y[c];
                    if (slot >= 0) {
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            dpsi_base[d * a.dir_stride + slot * a.tile +
                                      (((x0 | rowoff[rw[c]]) << a.log2B) | (col0 + col))] = y[c];
                    }
                }
            }
            __syncthreads();  // the next gate (or the next block's copies) may overwrite S
        }
        if (a.nbuf == 2) {
            cur ^= 1;
        } else {
            if (nxt < a.n_blocks) load(nxt, Sb);
            cp_async_commit_df();
        }
    }
    cp_async_wait_df<0>();
}

template <class K>
cudaError_t launch_resident_df(K kernel, const FwdFusedArgs &a, int sms, size_t smem, cudaStream_t s) {
    int per_sm = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem);
    if (e != cudaSuccess) return e;
    const long long grid = std::min<long long>(a.n_blocks, (long long)sms * std::max(per_sm, 1));
    kernel<<<(unsigned)grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_fused_df_mode(const FwdFusedArgs &a, int sms, size_t smem, cudaStream_t s) {
    switch (a.kdirs) {
        case 0: return launch_resident_df(k_fwd_fused_df<MODE, 0>, a, sms, smem, s);
        case 1: return launch_resident_df(k_fwd_fused_df<MODE, 1>, a, sms, smem, s);
        case 2: return launch_resident_df(k_fwd_fused_df<MODE, 2>, a, sms, smem, s);
        case 3: return launch_resident_df(k_fwd_fused_df<MODE, 3>, a, sms, smem, s);
        default: return launch_resident_df(k_fwd_fused_df<MODE, 4>, a, sms, smem, s);
    }
}

template <int MODE>
cudaError_t fused_df_attributes(int bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_fwd_fused_df<MODE, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fwd_fused_df<MODE, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fwd_fused_df<MODE, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fwd_fused_df<MODE, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fwd_fused_df<MODE, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

// psi_0 = |j_b> (the tile is zeroed before): df64 one = (1, 0, 0, 0).
__global__ void k_init_unit_df(float4 *psi0, const int32_t *cols, int B, int log2B, long long mask) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int j = cols[b];
    if (j < 0) return;
    psi0[(((long long)j & mask) << log2B) | b] = make_float4(1.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ float4 split(double2 v) {
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    return make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
}

// complex128 -> df64 for gates and directions
__global__ void k_to_df64(const double2 *in, float4 *out, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = split(in[i]);
}

// lambda_g = U|j_b> in df64 and the cost summands in FP64 (see rq_target.cu).
__global__ void k_scatter_target_df(const TargetDev t, const int32_t *cols, const double *wts, int log2B,
                                    long long mask, float4 *lam, const float4 *psi, double *fpart) {
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
            const float4 p = psi[o];
            lam[o] = split(u);
            acc = fma(u.x, (double)p.x + (double)p.y, acc);
            acc = fma(u.y, (double)p.z + (double)p.w, acc);
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

void launch_fwd_df64(const FwdArgs &a, int grid, cudaStream_t s) {
    switch (a.geo.mode) {
        case kGeneral: k_fwd_df<kGeneral><<<grid, kThreads, 0, s>>>(a); break;
        case kParity4: k_fwd_df<kParity4><<<grid, kThreads, 0, s>>>(a); break;
        default: k_fwd_df<kParity2><<<grid, kThreads, 0, s>>>(a); break;
    }
}

void launch_bwd_base_df64(const BwdArgs &a, int grid, cudaStream_t s) {
    switch (a.geo.mode) {
        case kGeneral: k_bwd_base_df2<kGeneral><<<grid, kThreads, kBaseDfSmem, s>>>(a); break;
        case kParity4: k_bwd_base_df2<kParity4><<<grid, kThreads, kBaseDfSmem, s>>>(a); break;
        default: k_bwd_base_df<kParity2><<<grid, kThreads, 0, s>>>(a); break;
    }
}

void launch_bwd_dir_df64(const BwdArgs &a, int grid, cudaStream_t s) {
    switch (a.geo.mode) {
        case kGeneral: k_bwd_dir_df2<kGeneral><<<grid, kThreads, kDirDfSmem, s>>>(a); break;
        case kParity4: k_bwd_dir_df2<kParity4><<<grid, kThreads, kDirDfSmem, s>>>(a); break;
        default: k_bwd_dir_df<kParity2><<<grid, kThreads, 0, s>>>(a); break;
    }
}

cudaError_t init_sweep_attributes_df64() {
    cudaError_t e = cudaFuncSetAttribute(k_bwd_dir_df2<kGeneral>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kDirDfSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_bwd_dir_df2<kParity4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kDirDfSmem);
    const int fmax = (int)kMaxFusedSmem;
    if (e == cudaSuccess) e = fused_df_attributes<kGeneral>(fmax);
    if (e == cudaSuccess) e = fused_df_attributes<kParity4>(fmax);
    return e;
}

cudaError_t launch_fwd_fused_df64(const FwdFusedArgs &a, int sms, cudaStream_t s) {
    const size_t smem = fused_smem_bytes(a.pass.q, a.kdirs, a.pass.m, a.nbuf);
    return a.mode == kGeneral ? launch_fused_df_mode<kGeneral>(a, sms, smem, s)
                              : launch_fused_df_mode<kParity4>(a, sms, smem, s);
}

void launch_init_unit_df64(double2 *psi0, const int32_t *cols, int B, int log2B, long long n_store,
                           cudaStream_t s) {
    k_init_unit_df<<<(B + 127) / 128, 128, 0, s>>>(reinterpret_cast<float4 *>(psi0), cols, B, log2B, n_store - 1);
}

void launch_to_df64(const double2 *in, double2 *out, long long n, cudaStream_t s) {
    if (n <= 0) return;
    k_to_df64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, reinterpret_cast<float4 *>(out), n);
}

void launch_scatter_target_df64(const TargetDev &t, const int32_t *cols, const double *wts, int B, int log2B,
                                int parity_layout, int n, double2 *lam, const double2 *psi_final, double *fpart,
                                cudaStream_t s) {
    const long long mask = parity_layout ? ((1LL << (n - 1)) - 1) : ((1LL << n) - 1);
    k_scatter_target_df<<<B, 128, 0, s>>>(t, cols, wts, log2B, mask, reinterpret_cast<float4 *>(lam),
                                          reinterpret_cast<const float4 *>(psi_final), fpart);
}

}  // namespace rq
