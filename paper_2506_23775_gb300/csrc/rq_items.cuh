// Item addressing shared by the FP64 and double-float sweep kernels.
//
// An item is the set of amplitudes of one column that a gate mixes: four for
// a gate on two stored qubits, two for a parity gate on the implied qubit.
// Amplitude x of column b sits at offset (x << log2B) | b of a tile.
#pragma once

#include "rq_internal.h"

namespace rq {

// First item of this thread in a grid-stride sweep over items (stride
// gridDim.x * blockDim.x): the lanes of a warp take 32 consecutive items
// (coalesced rows), and consecutive warp-sized chunks go to different CTAs
// before they go to the next warp of a CTA, so a sweep with few items still
// reaches every SM.  Chunk w * gridDim.x + blockIdx.x of warp w: a bijection
// onto [0, gridDim.x * blockDim.x).
__device__ __forceinline__ long long first_item() {
    return ((long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32 + (threadIdx.x & 31);
}

// The same for two lanes per item (16 items per warp chunk; stride
// gridDim.x * blockDim.x / 2).
__device__ __forceinline__ long long first_pair_item() {
    return ((long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 16 + ((threadIdx.x & 31) >> 1);
}

// r with a zero bit inserted at position p
__device__ __forceinline__ long long insert_zero(long long r, int p) {
    const long long lo = r & ((1LL << p) - 1);
    return ((r >> p) << (p + 1)) | lo;
}

// Offsets of the four amplitudes of an item whose amplitude with both gate
// bits clear is x0, for a gate on stored bits pa (first listed) and pb.
__device__ __forceinline__ void offsets4_at(long long x0, long long b, int pa, int pb, int log2B,
                                            long long (&off)[4]) {
    const long long sa = 1LL << pa, sb = 1LL << pb;
    off[0] = (x0 << log2B) | b;
    off[1] = ((x0 | sb) << log2B) | b;
    off[2] = ((x0 | sa) << log2B) | b;
    off[3] = ((x0 | sa | sb) << log2B) | b;
}

// ... of item (r, b): r enumerates the other stored bits.
__device__ __forceinline__ void offsets4(long long r, long long b, int pa, int pb, int log2B,
                                         long long (&off)[4]) {
    const int plo = pa < pb ? pa : pb;
    const int phi = pa < pb ? pb : pa;
    offsets4_at(insert_zero(insert_zero(r, plo), phi), b, pa, pb, log2B, off);
}

// The low bits of t placed, in order, at the set bits of mask.
__device__ __forceinline__ long long deposit_bits(long long t, long long mask) {
    long long out = 0;
    for (long long m = mask; m != 0; m &= m - 1, t >>= 1)
        if (t & 1) out |= m & -m;
    return out;
}

// Offsets of item (t, b) of a two-stored-qubit gate.  Unrestricted: t = r.
// A gate of the leading run of disjoint gates (geo.restricted, and the tile's
// columns given): t enumerates only the free bits and the fixed bits are those
// of column b's basis state, the only items where psi_{l-1} can be nonzero.
// Returns false for a padding column (nothing to do).
__device__ __forceinline__ bool item_offsets4(const GateGeom &geo, const int32_t *cols, long long t, long long b,
                                              int log2B, long long (&off)[4]) {
    if (cols != nullptr && geo.restricted) {
        const int j = cols[b];
        if (j < 0) return false;
        offsets4_at(deposit_bits(t, geo.free_bits) | ((long long)j & geo.fixed_bits), b, geo.pa, geo.pb, log2B, off);
        return true;
    }
    offsets4(t, b, geo.pa, geo.pb, log2B, off);
    return true;
}

// False for an item of a gate of the trailing run of disjoint gates whose
// adjoint amplitudes are all zero in column b (see GateGeom::tail): x0 is the
// item's amplitude index with the gate's bits clear.  Also false for a
// padding column.  Only the backward kernels of general gates call this (the
// marks are set for general gates only; a parity kernel leaves the check out
// at compile time).
__device__ __forceinline__ bool tail_live(const GateGeom &geo, const int32_t *cols, long long b, long long x0) {
    if (!geo.tail || cols == nullptr) return true;
    const long long j = cols[b];
    if (j < 0) return false;
    const int nu = __popcll(j & geo.up_mask), nd = __popcll(j & geo.dn_mask);
    const int cu = __popcll(x0 & geo.up_out), cd = __popcll(x0 & geo.dn_out);
    return cu <= nu && nu <= cu + geo.f_up && cd <= nd && nd <= cd + geo.f_dn;
}

}  // namespace rq
