// Gate sweeps over a tile of basis columns: forward (with tangents) and
// backward (adjoint states with gate-hole environments).
//
// Layout: a tile is [amplitudes x B columns] complex128 with the column index
// fastest, so the four amplitudes a gate mixes are four coalesced rows of B
// columns whatever the qubit pair (the paper's "locally sequential streams"
// of Sec. "Gate application" become full-width coalesced warps here).
//
// * Forward (Fig. forward_pass; Eq. gate_application_neighboring and its
//   general five-leg form): psi_{l+1} = G_l psi_l, and for each HVP direction
//   the forward-mode tangent psi'_{l+1} = G_l psi'_l + X_l psi_l (Appendix
//   "Evaluating Hessian-vector products").
// * Backward (Fig. backward_pass_gate_gradient, Fig. hole_contraction): the
//   paper propagates phi = (U|j>)^* with transposed gates and contracts the
//   gate hole y (x) x; here the adjoint state is kept as the ket
//   lambda = conj(phi), propagated with G^dagger, and the hole is
//   E[a][c] += conj(lambda[a]) psi[c].  The direction step adds
//   E'[a][c] += conj(lambda'[a]) psi[c] + conj(lambda[a]) psi'[c] and
//   lambda' <- G^dagger lambda' + X^dagger lambda (reverse pass over the
//   directed-gradient graph, Fig. directed_gradient_graph).
// * Parity-conserving gates (Eq. paritygatematrix) keep each column in its
//   parity sector, so a tile of equal-parity columns stores 2^(n-1)
//   amplitudes: qubit 0 is implied by the parity of the stored bits.  A gate
//   away from qubit 0 acts as its two 2x2 blocks on four stored amplitudes; a
//   gate on qubit 0 acts as one 2x2 block on two stored amplitudes, the block
//   chosen by the parity of the other stored bits.
//
// * First-layer support: a sweep starts from a basis state |j>, so before
//   gate l of the leading run of pairwise disjoint gates psi is |j> on every
//   qubit outside the run's earlier gates.  For those general gates an item
//   index enumerates only the free bits and takes the fixed ones from j; the
//   forward output outside that set is zero (cleared before the launch) and
//   the backward pass needs lambda_{l-1} only on it (the earlier gates of the
//   run read a subset).
//
// Environments are accumulated per thread in FP64 registers, reduced with a
// fixed warp-shuffle tree and a fixed-order block sum into one partial per
// CTA; a later kernel sums the partials in CTA order (deterministic).
//
// General gates use three real multiply-adds per complex product instead of
// four (Gauss's three-multiplication form), in the variant that needs one sum
// per amplitude: for m = a + ib and x = u + iv,
//   m x = (k - (a + b) v) + i (k + (b - a) u),  k = a (u + v),
// with a, -(a + b) and b - a tabulated once per gate (in shared memory) and
// S = u + v formed once per amplitude and reused by every output and
// environment entry that amplitude meets.  The environment entry conj(l) x,
// l = p + iq, is the same form with m = conj(l): three sums
// A1 = sum p S_x, A2 = sum (p - q) v, A3 = sum (p + q) u, with Re = A1 - A2
// and Im = A1 - A3 formed once per thread before the block reduction (the
// sums p - q, p + q of an adjoint amplitude serve its four entries).
// GB300's FP64 pipe is the bound of these kernels; against four products per
// complex product this cuts the FP64 instructions of a general-gate item by
// 16-19 %.  Parity gates touch two entries per row: their gate applications
// (forward steps, adjoint updates) use the same form, where the one sum per
// amplitude costs less than the product it saves, and their environment
// entries keep four products (two sums per adjoint amplitude would cost as
// much as they save).
#include "rq_items.cuh"

#include <algorithm>

namespace rq {
namespace {


// acc += a * b
__device__ __forceinline__ void cmac(double2 &acc, const double2 a, const double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

// acc += conj(a) * b
__device__ __forceinline__ void cmacc(double2 &acc, const double2 a, const double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}

__device__ __forceinline__ double2 zero2() { return make_double2(0.0, 0.0); }

// A 4x4 complex matrix tabulated for the three-product form: a, ns = -(a + b)
// and d = b - a of each entry m = a + ib, row-major (16-byte aligned, so two
// neighbouring entries of a row load as one 128-bit shared load).
struct __align__(16) Mat3 {
    double a[16], ns[16], d[16];
};

// Tabulate G (adjoint = 0) or G^dagger (adjoint = 1) from 16 complex entries;
// called by threads 0..15, entry e each.
__device__ __forceinline__ void tabulate3(Mat3 &m, const double2 *g, int e, int adjoint) {
    const int r = e >> 2, c = e & 3;
    double re, im;
    if (adjoint) {  // (G^dagger)[r][c] = conj(G[c][r])
        re = g[c * 4 + r].x;
        im = -g[c * 4 + r].y;
    } else {
        re = g[e].x;
        im = g[e].y;
    }
    m.a[e] = re;
    m.ns[e] = -(re + im);
    m.d[e] = im - re;
}

// An amplitude x = u + iv with its sums S = u + v and D = v - u (D only where
// the amplitude is the conjugated factor of an environment entry; unused
// sums are dropped by the compiler).
struct Amp3 {
    double u, v, S, D;
};

__device__ __forceinline__ Amp3 amp3(const double2 x) {
    Amp3 r;
    r.u = x.x;
    r.v = x.y;
    r.S = x.x + x.y;
    r.D = x.y - x.x;
    return r;
}

// y_i = sum_c M[i][c] x_c for the four outputs (three products per term).
__device__ __forceinline__ void matvec3(const Mat3 &m, const Amp3 (&x)[4], double2 (&y)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        double k = m.a[i * 4] * x[0].S;
#pragma unroll
        for (int c = 1; c < 4; ++c) k = fma(m.a[i * 4 + c], x[c].S, k);
        double re = k, im = k;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            re = fma(m.ns[i * 4 + c], x[c].v, re);
            im = fma(m.d[i * 4 + c], x[c].u, im);
        }
        y[i] = make_double2(re, im);
    }
}

// y_i = sum_c M[i][c] x_c + N[i][c] w_c (a tangent step).
__device__ __forceinline__ void matvec3_pair(const Mat3 &m, const Amp3 (&x)[4], const Mat3 &n,
                                             const Amp3 (&w)[4], double2 (&y)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        double k = m.a[i * 4] * x[0].S;
#pragma unroll
        for (int c = 1; c < 4; ++c) k = fma(m.a[i * 4 + c], x[c].S, k);
#pragma unroll
        for (int c = 0; c < 4; ++c) k = fma(n.a[i * 4 + c], w[c].S, k);
        double re = k, im = k;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            re = fma(m.ns[i * 4 + c], x[c].v, re);
            im = fma(m.d[i * 4 + c], x[c].u, im);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            re = fma(n.ns[i * 4 + c], w[c].v, re);
            im = fma(n.d[i * 4 + c], w[c].u, im);
        }
        y[i] = make_double2(re, im);
    }
}

// Columns of row i of a parity gate (Eq. paritygatematrix): {0, 3} for rows 0
// and 3, {1, 2} for rows 1 and 2.
__device__ __forceinline__ int pcol(int i, int u) {
    return (i == 0 || i == 3) ? (u == 0 ? 0 : 3) : (u == 0 ? 1 : 2);
}

// matvec3 for a parity gate: two terms per row.
__device__ __forceinline__ void matvec3_blocks(const Mat3 &m, const Amp3 (&x)[4], double2 (&y)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int c0 = pcol(i, 0), c1 = pcol(i, 1);
        const double k = fma(m.a[i * 4 + c1], x[c1].S, m.a[i * 4 + c0] * x[c0].S);
        const double re = fma(m.ns[i * 4 + c1], x[c1].v, fma(m.ns[i * 4 + c0], x[c0].v, k));
        const double im = fma(m.d[i * 4 + c1], x[c1].u, fma(m.d[i * 4 + c0], x[c0].u, k));
        y[i] = make_double2(re, im);
    }
}

// matvec3_pair for parity gates: y = M x + N w, two terms per row each.
__device__ __forceinline__ void matvec3_pair_blocks(const Mat3 &m, const Amp3 (&x)[4], const Mat3 &n,
                                                    const Amp3 (&w)[4], double2 (&y)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int c0 = pcol(i, 0), c1 = pcol(i, 1);
        double k = m.a[i * 4 + c0] * x[c0].S;
        k = fma(m.a[i * 4 + c1], x[c1].S, k);
        k = fma(n.a[i * 4 + c0], w[c0].S, k);
        k = fma(n.a[i * 4 + c1], w[c1].S, k);
        double re = fma(m.ns[i * 4 + c0], x[c0].v, k);
        re = fma(m.ns[i * 4 + c1], x[c1].v, re);
        re = fma(n.ns[i * 4 + c0], w[c0].v, re);
        re = fma(n.ns[i * 4 + c1], w[c1].v, re);
        double im = fma(m.d[i * 4 + c0], x[c0].u, k);
        im = fma(m.d[i * 4 + c1], x[c1].u, im);
        im = fma(n.d[i * 4 + c0], w[c0].u, im);
        im = fma(n.d[i * 4 + c1], w[c1].u, im);
        y[i] = make_double2(re, im);
    }
}

// Environment sums of conj(l_i) x_c over all 16 (i, c): A1 += p_i S_c,
// A2 += (p_i - q_i) v_c (p - q = -D of l), A3 += (p_i + q_i) u_c (p + q = S of l).
__device__ __forceinline__ void env3(double (&A1)[16], double (&A2)[16], double (&A3)[16], const Amp3 (&l)[4],
                                     const Amp3 (&x)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            A1[i * 4 + c] = fma(l[i].u, x[c].S, A1[i * 4 + c]);
            A2[i * 4 + c] = fma(-l[i].D, x[c].v, A2[i * 4 + c]);
            A3[i * 4 + c] = fma(l[i].S, x[c].u, A3[i * 4 + c]);
        }
}

// E[i] = (A1 - A2, A1 - A3)
__device__ __forceinline__ void env3_finish(const double (&A1)[16], const double (&A2)[16], const double (&A3)[16],
                                            double2 (&E)[16]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) E[i] = make_double2(A1[i] - A2[i], A1[i] - A3[i]);
}

// ------------------------------------------------ pipelined item loads --
//
// The general-gate backward kernels hold ~200 registers, so an SM runs only
// eight of their warps; while a warp waits for its item's amplitudes from
// HBM, the FP64 pipe depends on the others.  Their grid-stride loops (and
// that of the parity-gate base step) therefore copy the next item's
// amplitudes into this thread's own slots of shared memory (cp.async, two
// stages) while the current item is computed.
// Slot (stage, c) of thread t is at [(stage * NA + c) * kThreads + t], so a
// warp's copies and reads of one slot are contiguous.

__device__ __forceinline__ void cp_async16(double2 *smem, const double2 *gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kDirSlots = 16;   // k_bwd_dir: lambda, lambda', psi, psi' (4 amplitudes each)
constexpr int kBaseSlots = 8;   // k_bwd_base: lambda, psi
constexpr size_t kDirSmem = sizeof(double2) * 2 * kDirSlots * kThreads;
constexpr size_t kBaseSmem = sizeof(double2) * 2 * kBaseSlots * kThreads;

// Grid-stride loop over items with the loads of item i + stride in flight
// while item i is computed.  offsets(it, off) -> false for an item with
// nothing to do; issue(off, stage) starts its copies; body(off, stage)
// computes it from the slots.
template <class Offsets, class Issue, class Body>
__device__ __forceinline__ void pipelined_items(long long n_items, Offsets offsets, Issue issue, Body body) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long it = first_item();
    long long off[4], nxt[4];
    bool ok = false;
    if (it < n_items) {
        ok = offsets(it, off);
        if (ok) issue(off, 0);
    }
    cp_async_commit();
    int st = 0;
    for (; it < n_items; it += stride) {
        bool ok_next = false;
        if (it + stride < n_items) {
            ok_next = offsets(it + stride, nxt);
            if (ok_next) issue(nxt, st ^ 1);
        }
        cp_async_commit();
        cp_async_wait<1>();  // this item's copies have landed
        if (ok) body(off, st);
#pragma unroll
        for (int c = 0; c < 4; ++c) off[c] = nxt[c];
        ok = ok_next;
        st ^= 1;
    }
    cp_async_wait<0>();
}

// kParity2 item: the two stored amplitudes differ in the stored qubit at
// bit p; e = bit of the implied qubit for the first one.  Returns the local
// 4x4 indices (i0, i1) of the two amplitudes.
__device__ __forceinline__ void offsets2(long long r, long long b, int p, int qfirst, int parity,
                                         int log2B, long long (&off)[2], int &i0, int &i1) {
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

// ---------------------------------------------------------------- forward --

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) k_fwd(const FwdArgs a) {
    __shared__ double2 sg[16];
    __shared__ double2 sx[kMaxDirs][16];
    __shared__ Mat3 sg3;
    __shared__ Mat3 sx3[kMaxDirs];
    if (MODE == kGeneral || MODE == kParity4) {
        if (threadIdx.x < 16) tabulate3(sg3, a.gate, threadIdx.x, 0);
        if (threadIdx.x < 16 * a.kdirs)
            tabulate3(sx3[threadIdx.x >> 4], a.dirs + (threadIdx.x >> 4) * a.xdir_stride, threadIdx.x & 15, 0);
    } else {
        if (threadIdx.x < 16) sg[threadIdx.x] = a.gate[threadIdx.x];
        if (threadIdx.x < 16 * a.kdirs)
            sx[threadIdx.x >> 4][threadIdx.x & 15] = a.dirs[(threadIdx.x >> 4) * a.xdir_stride + (threadIdx.x & 15)];
    }
    __syncthreads();
    const long long Bm = (1LL << a.log2B) - 1;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long it = first_item(); it < a.n_items; it += stride) {
        const long long b = it & Bm, r = it >> a.log2B;
        if constexpr (MODE == kGeneral) {
            long long off[4];
            if (!item_offsets4(a.geo, a.cols, r, b, a.log2B, off)) continue;
            Amp3 x[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) x[c] = amp3(__ldg(&a.psi_in[off[c]]));
            double2 q[4];
            matvec3(sg3, x, q);
#pragma unroll
            for (int c = 0; c < 4; ++c) a.psi_out[off[c]] = q[c];
            for (int d = 0; d < a.kdirs; ++d) {
                const double2 *din = a.dpsi_in + d * a.dir_stride;
                double2 *dout = a.dpsi_out + d * a.dir_stride;
                Amp3 t[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) t[c] = amp3(__ldg(&din[off[c]]));
                matvec3_pair(sg3, t, sx3[d], x, q);  // G psi' + X psi
#pragma unroll
                for (int c = 0; c < 4; ++c) dout[off[c]] = q[c];
            }
        } else if constexpr (MODE == kParity4) {
            // the three-product form on each row's two entries (block {0, 3}
            // or {1, 2}); the tangent shares the state's sums
            long long off[4];
            if (!item_offsets4(a.geo, a.cols, r, b, a.log2B, off)) continue;
            Amp3 x[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) x[c] = amp3(__ldg(&a.psi_in[off[c]]));
            double2 q[4];
            matvec3_blocks(sg3, x, q);
#pragma unroll
            for (int c = 0; c < 4; ++c) a.psi_out[off[c]] = q[c];
            for (int d = 0; d < a.kdirs; ++d) {
                const double2 *din = a.dpsi_in + d * a.dir_stride;
                double2 *dout = a.dpsi_out + d * a.dir_stride;
                Amp3 t[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) t[c] = amp3(__ldg(&din[off[c]]));
                matvec3_pair_blocks(sg3, t, sx3[d], x, q);  // G psi' + X psi
#pragma unroll
                for (int c = 0; c < 4; ++c) dout[off[c]] = q[c];
            }
        } else {  // kParity2
            long long off[2];
            int i0, i1;
            offsets2(r, b, a.geo.pa, a.geo.qfirst, a.tile_parity, a.log2B, off, i0, i1);
            const double2 p0 = __ldg(&a.psi_in[off[0]]), p1 = __ldg(&a.psi_in[off[1]]);
            double2 q0 = zero2(), q1 = zero2();
            cmac(q0, sg[i0 * 4 + i0], p0); cmac(q0, sg[i0 * 4 + i1], p1);
            cmac(q1, sg[i1 * 4 + i0], p0); cmac(q1, sg[i1 * 4 + i1], p1);
            a.psi_out[off[0]] = q0;
            a.psi_out[off[1]] = q1;
            for (int d = 0; d < a.kdirs; ++d) {
                const double2 *din = a.dpsi_in + d * a.dir_stride;
                double2 *dout = a.dpsi_out + d * a.dir_stride;
                const double2 t0 = __ldg(&din[off[0]]), t1 = __ldg(&din[off[1]]);
                q0 = zero2();
                q1 = zero2();
                cmac(q0, sg[i0 * 4 + i0], t0); cmac(q0, sg[i0 * 4 + i1], t1);
                cmac(q1, sg[i1 * 4 + i0], t0); cmac(q1, sg[i1 * 4 + i1], t1);
                cmac(q0, sx[d][i0 * 4 + i0], p0); cmac(q0, sx[d][i0 * 4 + i1], p1);
                cmac(q1, sx[d][i1 * 4 + i0], p0); cmac(q1, sx[d][i1 * 4 + i1], p1);
                dout[off[0]] = q0;
                dout[off[1]] = q1;
            }
        }
    }
}

// ------------------------------------------------------- block reduction --

// Sum acc over the CTA in a fixed order and store 32 doubles at out.
__device__ __forceinline__ void block_reduce_store(const double2 (&acc)[16], double *out) {
    __shared__ double red[kThreads / 32][kEnvDoubles];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        double vx = acc[i].x, vy = acc[i].y;
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

// ---------------------------------------------------------- backward base --

// E[a][c] += conj(lambda[a]) psi[c]; lambda <- G^dagger lambda.
template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) k_bwd_base(const BwdArgs a) {
    const int accumulate = a.accumulate;
    __shared__ double2 sg[16];
    __shared__ Mat3 sgT3;  // G^dagger, gates on two stored qubits
    if (threadIdx.x < 16) {
        if (MODE != kParity2) tabulate3(sgT3, a.gate, threadIdx.x, 1);
        else sg[threadIdx.x] = a.gate[threadIdx.x];
    }
    __syncthreads();
    double2 E[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) E[i] = zero2();
    double A1[16], A2[16], A3[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) A1[i] = A2[i] = A3[i] = 0.0;
    const long long Bm = (1LL << a.log2B) - 1;
    if constexpr (MODE == kGeneral || MODE == kParity4) {
        // gates on two stored qubits: pipelined item loads
        extern __shared__ double2 pf[];
        double2 *mine = pf + threadIdx.x;
        auto slot = [&](int st, int c) { return mine + (st * kBaseSlots + c) * kThreads; };
        pipelined_items(
            a.n_items,
            [&](long long it, long long (&off)[4]) {
                return item_offsets4(a.geo, a.cols, it >> a.log2B, it & Bm, a.log2B, off) &&
                       (MODE != kGeneral || tail_live(a.geo, a.cols, it & Bm, off[0] >> a.log2B));
            },
            [&](const long long (&off)[4], int st) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    cp_async16(slot(st, c), a.lam + off[c]);
                    if (accumulate) cp_async16(slot(st, 4 + c), a.psi + off[c]);
                }
            },
            [&](const long long (&off)[4], int st) {
                if constexpr (MODE == kGeneral) {
                    Amp3 l[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) l[c] = amp3(*slot(st, c));
                    if (accumulate) {
                        Amp3 p[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) p[c] = amp3(*slot(st, 4 + c));
                        env3(A1, A2, A3, l, p);
                    }
                    if (a.update) {
                        double2 q[4];
                        matvec3(sgT3, l, q);
#pragma unroll
                        for (int c = 0; c < 4; ++c) a.lam[off[c]] = q[c];
                    }
                } else {
                    double2 l[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) l[c] = *slot(st, c);
                    if (accumulate) {
                        double2 p[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) p[c] = *slot(st, 4 + c);
                        cmacc(E[0], l[0], p[0]); cmacc(E[3], l[0], p[3]);
                        cmacc(E[12], l[3], p[0]); cmacc(E[15], l[3], p[3]);
                        cmacc(E[5], l[1], p[1]); cmacc(E[6], l[1], p[2]);
                        cmacc(E[9], l[2], p[1]); cmacc(E[10], l[2], p[2]);
                    }
                    if (a.update) {
                        Amp3 lx[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) lx[c] = amp3(l[c]);
                        double2 q[4];
                        matvec3_blocks(sgT3, lx, q);
#pragma unroll
                        for (int c = 0; c < 4; ++c) a.lam[off[c]] = q[c];
                    }
                }
            });
    } else {  // kParity2: two-amplitude items, plain loads
        const long long stride = (long long)gridDim.x * blockDim.x;
        for (long long it = first_item(); it < a.n_items; it += stride) {
            const long long b = it & Bm, r = it >> a.log2B;
            long long off[2];
            int i0, i1;
            offsets2(r, b, a.geo.pa, a.geo.qfirst, a.tile_parity, a.log2B, off, i0, i1);
            const double2 l0 = a.lam[off[0]], l1 = a.lam[off[1]];
            if (accumulate) {
                const double2 p0 = __ldg(&a.psi[off[0]]), p1 = __ldg(&a.psi[off[1]]);
                // E[i0][i0], E[i0][i1], E[i1][i0], E[i1][i1]; written with
                // static indices per block so the accumulators stay in registers
                double2 c00 = zero2(), c01 = zero2(), c10 = zero2(), c11 = zero2();
                cmacc(c00, l0, p0); cmacc(c01, l0, p1); cmacc(c10, l1, p0); cmacc(c11, l1, p1);
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
            if (a.update) {
                double2 q0 = zero2(), q1 = zero2();
                cmacc(q0, sg[i0 * 4 + i0], l0); cmacc(q0, sg[i1 * 4 + i0], l1);
                cmacc(q1, sg[i0 * 4 + i1], l0); cmacc(q1, sg[i1 * 4 + i1], l1);
                a.lam[off[0]] = q0;
                a.lam[off[1]] = q1;
            }
        }
    }
    if constexpr (MODE == kGeneral) env3_finish(A1, A2, A3, E);
    if (accumulate) block_reduce_store(E, a.part + (long long)blockIdx.x * kEnvDoubles);
}

// ----------------------------------------------------- backward direction --

// E'[a][c] += conj(lambda'[a]) psi[c] + conj(lambda[a]) psi'[c];
// lambda' <- G^dagger lambda' + X^dagger lambda.  Runs before the base step
// of the same gate (it reads lambda_l before that step overwrites it).
// Parity gates: two CTAs per SM (at most 128 registers; their items carry
// half the FP64 work of a general item, so more warps are needed to cover
// the loads).  General gates: one CTA (the three-product sums need ~200).
template <int MODE>
__global__ void __launch_bounds__(kThreads, MODE == kGeneral ? 1 : 2) k_bwd_dir(const BwdArgs a) {
    __shared__ double2 sg[16];
    __shared__ double2 sx[16];
    __shared__ Mat3 sgT3, sxT3;  // G^dagger, X^dagger, gates on two stored qubits
    if (threadIdx.x < 16) {
        if (MODE != kParity2) {
            tabulate3(sgT3, a.gate, threadIdx.x, 1);
            tabulate3(sxT3, a.dir, threadIdx.x, 1);
        } else {
            sg[threadIdx.x] = a.gate[threadIdx.x];
            sx[threadIdx.x] = a.dir[threadIdx.x];
        }
    }
    __syncthreads();
    double2 E[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) E[i] = zero2();
    double A1[16], A2[16], A3[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) A1[i] = A2[i] = A3[i] = 0.0;
    const long long Bm = (1LL << a.log2B) - 1;
    if constexpr (MODE == kGeneral) {
        extern __shared__ double2 pf[];
        double2 *mine = pf + threadIdx.x;
        auto slot = [&](int st, int c) { return mine + (st * kDirSlots + c) * kThreads; };
        pipelined_items(
            a.n_items,
            [&](long long it, long long (&off)[4]) {
                return item_offsets4(a.geo, a.cols, it >> a.log2B, it & Bm, a.log2B, off) &&
                       (MODE != kGeneral || tail_live(a.geo, a.cols, it & Bm, off[0] >> a.log2B));
            },
            [&](const long long (&off)[4], int st) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    cp_async16(slot(st, c), a.lam + off[c]);
                    cp_async16(slot(st, 4 + c), a.dlam + off[c]);
                    cp_async16(slot(st, 8 + c), a.psi + off[c]);
                    cp_async16(slot(st, 12 + c), a.dpsi + off[c]);
                }
            },
            [&](const long long (&off)[4], int st) {
                Amp3 l[4], dl[4], p[4], dp[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    l[c] = amp3(*slot(st, c));
                    dl[c] = amp3(*slot(st, 4 + c));
                    p[c] = amp3(*slot(st, 8 + c));
                    dp[c] = amp3(*slot(st, 12 + c));
                }
                env3(A1, A2, A3, dl, p);
                env3(A1, A2, A3, l, dp);
                if (a.update) {
                    double2 q[4];
                    matvec3_pair(sgT3, dl, sxT3, l, q);  // G^dagger lambda' + X^dagger lambda
#pragma unroll
                    for (int c = 0; c < 4; ++c) a.dlam[off[c]] = q[c];
                }
            });
    } else {  // parity gates: plain loads (two CTAs per SM cover their latency)
        const long long stride = (long long)gridDim.x * blockDim.x;
        for (long long it = first_item(); it < a.n_items; it += stride) {
            const long long b = it & Bm, r = it >> a.log2B;
            if constexpr (MODE == kParity4) {
                long long off[4];
                if (!item_offsets4(a.geo, a.cols, r, b, a.log2B, off)) continue;
                double2 l[4], dl[4], p[4], dp[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    l[c] = __ldg(&a.lam[off[c]]);
                    dl[c] = a.dlam[off[c]];
                    p[c] = __ldg(&a.psi[off[c]]);
                    dp[c] = __ldg(&a.dpsi[off[c]]);
                }
                const int idx[8][2] = {{0, 0}, {0, 3}, {3, 0}, {3, 3}, {1, 1}, {1, 2}, {2, 1}, {2, 2}};
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    cmacc(E[idx[u][0] * 4 + idx[u][1]], dl[idx[u][0]], p[idx[u][1]]);
                    cmacc(E[idx[u][0] * 4 + idx[u][1]], l[idx[u][0]], dp[idx[u][1]]);
                }
                if (a.update) {
                    Amp3 dlx[4], lx[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        dlx[c] = amp3(dl[c]);
                        lx[c] = amp3(l[c]);
                    }
                    double2 q[4];
                    matvec3_pair_blocks(sgT3, dlx, sxT3, lx, q);  // G^dagger lambda' + X^dagger lambda
#pragma unroll
                    for (int c = 0; c < 4; ++c) a.dlam[off[c]] = q[c];
                }
            } else {  // kParity2
                long long off[2];
                int i0, i1;
                offsets2(r, b, a.geo.pa, a.geo.qfirst, a.tile_parity, a.log2B, off, i0, i1);
                const double2 l0 = __ldg(&a.lam[off[0]]), l1 = __ldg(&a.lam[off[1]]);
                const double2 d0 = a.dlam[off[0]], d1 = a.dlam[off[1]];
                const double2 p0 = __ldg(&a.psi[off[0]]), p1 = __ldg(&a.psi[off[1]]);
                const double2 t0 = __ldg(&a.dpsi[off[0]]), t1 = __ldg(&a.dpsi[off[1]]);
                double2 c00 = zero2(), c01 = zero2(), c10 = zero2(), c11 = zero2();
                cmacc(c00, d0, p0); cmacc(c00, l0, t0);
                cmacc(c01, d0, p1); cmacc(c01, l0, t1);
                cmacc(c10, d1, p0); cmacc(c10, l1, t0);
                cmacc(c11, d1, p1); cmacc(c11, l1, t1);
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
                if (a.update) {
                    double2 q0 = zero2(), q1 = zero2();
                    cmacc(q0, sg[i0 * 4 + i0], d0); cmacc(q0, sg[i1 * 4 + i0], d1);
                    cmacc(q0, sx[i0 * 4 + i0], l0); cmacc(q0, sx[i1 * 4 + i0], l1);
                    cmacc(q1, sg[i0 * 4 + i1], d0); cmacc(q1, sg[i1 * 4 + i1], d1);
                    cmacc(q1, sx[i0 * 4 + i1], l0); cmacc(q1, sx[i1 * 4 + i1], l1);
                    a.dlam[off[0]] = q0;
                    a.dlam[off[1]] = q1;
                }
            }
        }
    }
    if constexpr (MODE == kGeneral) env3_finish(A1, A2, A3, E);
    block_reduce_store(E, a.part + (long long)blockIdx.x * kEnvDoubles);
}

// ------------------------------------------------------ fused forward pass --
//
// Window fusion (Sec. "Brick wall circuit layout": the gates of a layer are
// disjoint and commute, so consecutive gates inside a small set of qubits can
// be applied together): a CTA copies a block of [2^q amplitudes x 32 columns]
// -- the amplitudes that differ only in the window's q stored bits, for 32
// consecutive columns -- into shared memory, applies the pass's m gates (and
// their tangent steps) there, and writes a gate's output to HBM only where a
// checkpoint slot is wanted (every gate when the backward pass needs the
// states, the last one otherwise).  Same arithmetic per item as k_fwd.
// Shared memory: nbuf sets of (1 + KD) state blocks, the gates' tables, a
// row -> stored offset table.  With two sets the next block's amplitudes are
// copied in (cp.async) while the current block's gates run.

size_t fused_bytes(int q, int kd, int m, int nbuf) {
    return (size_t)nbuf * (1 + kd) * ((size_t)32 << q) * sizeof(double2) + (size_t)(1 + kd) * m * sizeof(Mat3) +
           ((size_t)1 << q) * sizeof(long long);
}

template <int MODE, int KD>
__global__ void __launch_bounds__(kThreads, 1) k_fwd_fused(const FwdFusedArgs a) {
    extern __shared__ __align__(16) unsigned char fused_raw[];
    const FusedPass &p = a.pass;
    const int rows = 1 << p.q, m = p.m;
    const int elems = rows * 32, items = (rows >> 2) * 32;
    double2 *const Sb = reinterpret_cast<double2 *>(fused_raw);           // [nbuf][1 + KD][rows][32]
    Mat3 *mg = reinterpret_cast<Mat3 *>(Sb + a.nbuf * (1 + KD) * elems);  // [m]
    Mat3 *mx = mg + m;                                                     // [KD][m]
    long long *rowoff = reinterpret_cast<long long *>(mx + KD * m);       // [rows]
    for (int e = threadIdx.x; e < m * 16; e += blockDim.x) {
        const int j = e >> 4;
        tabulate3(mg[j], a.gates + (long long)p.param[j] * 16, e & 15, 0);
#pragma unroll
        for (int d = 0; d < KD; ++d)
            tabulate3(mx[d * m + j], a.dirs + d * a.xdir_stride + (long long)p.param[j] * 16, e & 15, 0);
    }
    for (int r = threadIdx.x; r < rows; r += blockDim.x) rowoff[r] = deposit_bits(r, p.wmask);
    __syncthreads();
    const long long cmask = (1LL << a.log2chunks) - 1;
    auto load = [&](long long blk, double2 *dst) {
        const long long x0 = deposit_bits(blk >> a.log2chunks, a.outer_mask);
        const long long col0 = (blk & cmask) << 5;
        for (int e = threadIdx.x; e < elems; e += blockDim.x) {
            const long long off = ((x0 | rowoff[e >> 5]) << a.log2B) | (col0 + (e & 31));
            cp_async16(dst + e, a.psi_in + off);
#pragma unroll
            for (int d = 0; d < KD; ++d) cp_async16(dst + (1 + d) * elems + e, a.dpsi_in + d * a.dir_stride + off);
        }
    };
    long long blk = blockIdx.x;
    if (blk < a.n_blocks) load(blk, Sb);
    cp_async_commit();
    int cur = 0;
    for (; blk < a.n_blocks; blk += gridDim.x) {
        const long long nxt = blk + gridDim.x;
        if (a.nbuf == 2) {
            if (nxt < a.n_blocks) load(nxt, Sb + (cur ^ 1) * (1 + KD) * elems);
            cp_async_commit();
            cp_async_wait<1>();  // this block's copies have landed
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        double2 *S = Sb + cur * (1 + KD) * elems;
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
                Amp3 x[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) x[c] = amp3(S[rw[c] * 32 + col]);
                double2 y[4];
                if constexpr (MODE == kGeneral) matvec3(mg[j], x, y);
                else matvec3_blocks(mg[j], x, y);
#pragma unroll
                for (int c = 0; c < 4; ++c) S[rw[c] * 32 + col] = y[c];
                if (slot >= 0) {
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        a.psi_base[slot * a.tile + (((x0 | rowoff[rw[c]]) << a.log2B) | (col0 + col))] = y[c];
                }
#pragma unroll
                for (int d = 0; d < KD; ++d) {
                    double2 *T = S + (1 + d) * elems;
                    Amp3 t[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) t[c] = amp3(T[rw[c] * 32 + col]);
                    if constexpr (MODE == kGeneral) matvec3_pair(mg[j], t, mx[d * m + j], x, y);  // G psi' + X psi
                    else matvec3_pair_blocks(mg[j], t, mx[d * m + j], x, y);
#pragma unroll
                    for (int c = 0; c < 4; ++c) T[rw[c] * 32 + col] = y[c];
                    if (slot >= 0) {
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            a.dpsi_base[d * a.dir_stride + slot * a.tile +
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
            cp_async_commit();
        }
    }
    cp_async_wait<0>();
}

// Grid: as many CTAs as fit on every SM at this shared-memory size (blocks
// are dealt grid-stride), never more than there are blocks.
template <class K>
cudaError_t launch_resident(K kernel, const FwdFusedArgs &a, int sms, size_t smem, cudaStream_t s) {
    int per_sm = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem);
    if (e != cudaSuccess) return e;
    const long long grid = std::min<long long>(a.n_blocks, (long long)sms * std::max(per_sm, 1));
    kernel<<<(unsigned)grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_fused_mode(const FwdFusedArgs &a, int sms, size_t smem, cudaStream_t s) {
    switch (a.kdirs) {
        case 0: return launch_resident(k_fwd_fused<MODE, 0>, a, sms, smem, s);
        case 1: return launch_resident(k_fwd_fused<MODE, 1>, a, sms, smem, s);
        case 2: return launch_resident(k_fwd_fused<MODE, 2>, a, sms, smem, s);
        case 3: return launch_resident(k_fwd_fused<MODE, 3>, a, sms, smem, s);
        default: return launch_resident(k_fwd_fused<MODE, 4>, a, sms, smem, s);
    }
}

template <int MODE>
cudaError_t fused_attributes(int bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_fwd_fused<MODE, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fwd_fused<MODE, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fwd_fused<MODE, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fwd_fused<MODE, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fwd_fused<MODE, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

// psi_0 = |j_b> for every column b of the tile (the tile is zeroed before).
__global__ void k_init_unit(double2 *psi0, const int32_t *cols, int B, int log2B, long long mask) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int j = cols[b];
    if (j < 0) return;
    const long long y = (long long)j & mask;
    psi0[(y << log2B) | b] = make_double2(1.0, 0.0);
}

}  // namespace

void launch_fwd(const FwdArgs &a, int grid, cudaStream_t s) {
    switch (a.geo.mode) {
        case kGeneral: k_fwd<kGeneral><<<grid, kThreads, 0, s>>>(a); break;
        case kParity4: k_fwd<kParity4><<<grid, kThreads, 0, s>>>(a); break;
        default: k_fwd<kParity2><<<grid, kThreads, 0, s>>>(a); break;
    }
}

void launch_bwd_base(const BwdArgs &a, int grid, cudaStream_t s) {
    switch (a.geo.mode) {
        case kGeneral: k_bwd_base<kGeneral><<<grid, kThreads, kBaseSmem, s>>>(a); break;
        case kParity4: k_bwd_base<kParity4><<<grid, kThreads, kBaseSmem, s>>>(a); break;
        default: k_bwd_base<kParity2><<<grid, kThreads, 0, s>>>(a); break;
    }
}

void launch_bwd_dir(const BwdArgs &a, int grid, cudaStream_t s) {
    switch (a.geo.mode) {
        case kGeneral: k_bwd_dir<kGeneral><<<grid, kThreads, kDirSmem, s>>>(a); break;
        case kParity4: k_bwd_dir<kParity4><<<grid, kThreads, 0, s>>>(a); break;
        default: k_bwd_dir<kParity2><<<grid, kThreads, 0, s>>>(a); break;
    }
}

size_t fused_smem_bytes(int q, int kdirs, int m, int nbuf) {
    // double-float blocks and tables take the same bytes (float4 amplitudes, float2 triples)
    return fused_bytes(q, kdirs, m, nbuf);
}

cudaError_t launch_fwd_fused(const FwdFusedArgs &a, int sms, cudaStream_t s) {
    const size_t smem = fused_bytes(a.pass.q, a.kdirs, a.pass.m, a.nbuf);
    return a.mode == kGeneral ? launch_fused_mode<kGeneral>(a, sms, smem, s)
                              : launch_fused_mode<kParity4>(a, sms, smem, s);
}

cudaError_t init_sweep_attributes() {
    // the pipelined kernels keep two stages of item slots in dynamic shared
    // memory (128 KB per CTA for k_bwd_dir, 64 KB for k_bwd_base); the fused
    // forward passes up to their largest block and tables
    cudaError_t e = cudaFuncSetAttribute(k_bwd_dir<kGeneral>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kDirSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_bwd_base<kGeneral>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBaseSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_bwd_base<kParity4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBaseSmem);
    const int fmax = (int)kMaxFusedSmem;
    if (e == cudaSuccess) e = fused_attributes<kGeneral>(fmax);
    if (e == cudaSuccess) e = fused_attributes<kParity4>(fmax);
    return e;
}

void launch_init_unit(double2 *psi0, const int32_t *cols, int B, int log2B, long long n_store,
                      int parity_layout, cudaStream_t s) {
    const long long mask = n_store - 1;  // drops the implied top qubit in the parity layout
    (void)parity_layout;
    k_init_unit<<<(B + 127) / 128, 128, 0, s>>>(psi0, cols, B, log2B, mask);
}

}  // namespace rq
