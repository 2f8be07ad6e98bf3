// Internal declarations of the rq library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/rq.h"

namespace rq {

constexpr int kThreads = 256;      // threads per CTA of every sweep kernel
constexpr int kCtasPerSm = 2;      // sweep CTAs launched per SM (grid size)
constexpr int kMaxDirs = 4;        // HVP directions swept together
constexpr int kMaxQubits = 20;
constexpr int kMaxDenseQubits = 14;  // dense targets: 2^28 complex entries at most
constexpr int kEnvDoubles = 32;    // one 4x4 complex environment

// Which kernel family handles a gate.
enum GateMode : int {
    kGeneral = 0,     // general 4x4 gate, full 2^n layout
    kParity4 = 1,     // parity gate on two stored qubits (two 2x2 blocks)
    kParity2 = 2,     // parity gate touching the implied qubit (one 2x2 block per item)
};

struct GateGeom {
    int mode;      // GateMode
    int pa, pb;    // stored bit positions of the listed qubits (kParity2: pa = other qubit, pb = -1)
    int qfirst;    // kParity2: 1 if the stored qubit is listed first
    int param;     // parameter gate index
    // First-layer support (general gates of the leading run of disjoint
    // gates): psi_{l-1} of column j is zero unless the stored bits in
    // fixed_bits equal those of j, so a sweep of gate l visits only the items
    // whose free_bits (the qubits of the earlier gates of the run) take every
    // value.  restricted = 0: every item.
    int restricted = 0;
    long long free_bits = 0, fixed_bits = 0;
    // Last-layer support (general gates of the trailing run of disjoint gates,
    // backward pass): lambda_l of column j starts as U|j>, which lives in j's
    // particle-number sector, and only the later gates of the run have
    // changed it, on their own qubits.  An item of gate l can be nonzero only
    // if the bits outside those qubits and the gate's own (the stored bits in
    // up_out / dn_out) can be completed to a state of j's sector: their up
    // count c_u and down count c_d must satisfy c_u <= N_up(j) <= c_u + f_up
    // and c_d <= N_dn(j) <= c_d + f_dn, where f_up / f_dn count the up / down
    // qubits the run has touched.  N_up(j), N_dn(j) are the counts of j's
    // bits in up_mask / dn_mask (a spinless chain: all qubits up).  tail = 0:
    // every item.
    int tail = 0;
    int f_up = 0, f_dn = 0;
    long long up_out = 0, dn_out = 0, up_mask = 0, dn_mask = 0;
};

// Arguments of one forward gate step over a tile.
struct FwdArgs {
    const double2 *psi_in;
    double2 *psi_out;
    const double2 *dpsi_in;     // direction 0; direction d at + d * dir_stride
    double2 *dpsi_out;
    long long dir_stride;       // elements between directions' checkpoint sets
    int kdirs;
    const double2 *gate;        // 16 entries
    const double2 *dirs;        // direction 0 of this parameter; direction d at + d * xdir_stride
    long long xdir_stride;
    GateGeom geo;
    int log2B;
    int tile_parity;
    long long n_items;
    const int32_t *cols = nullptr;  // column basis states (-1: padding) when geo.restricted
};

// Arguments of one backward gate step over a tile.
struct BwdArgs {
    double2 *lam;               // lambda_l, updated in place to lambda_{l-1} (base step)
    double2 *dlam;              // direction step: lambda-dot_l, updated in place
    const double2 *psi;         // psi_{l-1}
    const double2 *dpsi;        // psi-dot_{l-1} (direction step)
    const double2 *gate;
    const double2 *dir;         // X of this parameter for the direction (direction step)
    GateGeom geo;
    int log2B;
    int tile_parity;
    int update;                 // 0: skip the state update (first gate)
    int accumulate;             // base step: 0 skips the environment (and part)
    long long n_items;
    double *part;               // [gridDim.x][32] per-CTA partial environments
    const int32_t *cols = nullptr;  // column basis states (-1: padding) when geo.restricted
};

// One fused forward pass (window fusion): m consecutive gates of the
// execution order that all act within a window of q stored bits are applied
// to blocks of [2^q amplitudes x 32 columns] held in shared memory, so the
// state is read from HBM once per pass instead of once per gate.
constexpr int kMaxWindow = 6;      // window bits (2^6 rows x 32 columns per block)
constexpr int kMaxPassGates = 16;  // gates per fused pass
struct FusedPass {
    int m = 0, q = 0;
    long long wmask = 0;              // stored bits of the window
    int la[kMaxPassGates];            // window-local bit of the gate's first listed qubit (geo.pa)
    int lb[kMaxPassGates];            // ... of its second listed qubit (geo.pb)
    int param[kMaxPassGates];         // parameter gate index
    int out_slot[kMaxPassGates];      // checkpoint slot written after the gate (-1: none)
};

struct FwdFusedArgs {
    const double2 *psi_in;      // state before the pass (tile)
    const double2 *dpsi_in;     // tangent of direction 0 before the pass; direction d at + d * dir_stride
    double2 *psi_base;          // checkpoint slot 0 (slot s at + s * tile)
    double2 *dpsi_base;         // tangent slot 0 of direction 0
    long long tile;             // elements per slot
    long long dir_stride;       // elements between directions' checkpoint sets
    int kdirs;
    int mode;                   // kGeneral or kParity4 (every gate of the pass)
    const double2 *gates;       // parameter gates [P][16]
    const double2 *dirs;        // direction d of parameter p at dirs + d * xdir_stride + p * 16
    long long xdir_stride;
    int log2B;
    int log2chunks;             // log2(B / 32)
    long long n_blocks;         // (n_store >> q) << log2chunks
    long long outer_mask;       // stored bits outside the window
    int nbuf;                   // 2: copy the next block in while the current one is computed; 1: not
    FusedPass pass;
};

// Sector tables of the stored target.
struct TargetDev {
    const int32_t *sec_of;      // [2^n] sector id of a basis index
    const int32_t *pos;         // [2^n] position inside its sector
    const int32_t *basis;       // concatenated ascending basis lists
    const long long *off_basis; // [S+1]
    const long long *off_u;     // [S+1] offsets of the column-major U blocks
    const double2 *U;
};

// Launchers (rq_sweep.cu).
// Once per device before the first sweep launch (shared-memory limits).
cudaError_t init_sweep_attributes();
void launch_fwd(const FwdArgs &a, int grid, cudaStream_t s);
void launch_bwd_base(const BwdArgs &a, int grid, cudaStream_t s);
void launch_bwd_dir(const BwdArgs &a, int grid, cudaStream_t s);
void launch_init_unit(double2 *psi0, const int32_t *cols, int B, int log2B, long long n_store,
                      int parity_layout, cudaStream_t s);
// Fused forward pass: shared-memory bytes of a launch with nbuf block sets
// (the same for FP64 and double-float), and the most any launch may use.
constexpr size_t kMaxFusedSmem = 227 * 1024;
size_t fused_smem_bytes(int q, int kdirs, int m, int nbuf);
cudaError_t launch_fwd_fused(const FwdFusedArgs &a, int sms, cudaStream_t s);

// Launchers (rq_sweep_df64.cu): the same steps in double-float arithmetic;
// tiles, gates and directions hold float4 (hi, lo, hi, lo) in the same bytes.
void launch_fwd_df64(const FwdArgs &a, int grid, cudaStream_t s);
void launch_bwd_base_df64(const BwdArgs &a, int grid, cudaStream_t s);
void launch_bwd_dir_df64(const BwdArgs &a, int grid, cudaStream_t s);
void launch_init_unit_df64(double2 *psi0, const int32_t *cols, int B, int log2B, long long n_store, cudaStream_t s);
void launch_to_df64(const double2 *in, double2 *out, long long n, cudaStream_t s);
cudaError_t launch_fwd_fused_df64(const FwdFusedArgs &a, int sms, cudaStream_t s);
void launch_scatter_target_df64(const TargetDev &t, const int32_t *cols, const double *wts, int B, int log2B,
                                int parity_layout, int n, double2 *lam, const double2 *psi_final, double *fpart,
                                cudaStream_t s);

// Launchers (rq_target.cu).
void launch_scatter_target(const TargetDev &t, const int32_t *cols, const double *wts, int B, int log2B,
                           int parity_layout, int n, double2 *lam, const double2 *psi_final,
                           double *fpart, cudaStream_t s);
void launch_cheb_step(const TargetDev &t, int n_sectors, long long total, const double *cur,
                      double *prev_out, double2 *acc, double2 coef, double scale, int first,
                      double diag_scale, double diag_shift, double hop_scale,
                      const long long *bond_masks, int n_bonds, int L, double U, int model, cudaStream_t s);
void launch_cheb_init(const long long *off_u, const long long *sizes, int n_sectors, long long total,
                      double *prev, double2 *acc, double2 c0, cudaStream_t s);

// Launchers (rq_hessian.cu).
void launch_hole_apply(const double2 *psi, double2 *arr, const GateGeom &geo, int log2B, int log2M,
                       int parity_members, int tile_parity, long long n_items, int grid, cudaStream_t s);
void launch_array_env(const double2 *lam, const double2 *arr, const GateGeom &geo, int log2B, int log2M,
                      int tile_parity, long long n_items, int ncta, double *part, cudaStream_t s);
void launch_reduce_rows(const double *part, int ncta, long long rows, double *hacc, cudaStream_t s);

// Launchers (rq_geometry.cu).
void launch_reduce_env(const double *part, int ncta, int n_gates, double *env, cudaStream_t s);
void launch_reduce_f(const double *fpart, int B, double *facc, cudaStream_t s);
void launch_project_dirs(const double2 *gates, const double2 *raw, double2 *out, int n_params,
                         int k, int structure, int euclidean, cudaStream_t s);
void launch_mask_gates(const double2 *in, double2 *out, int n_params, int structure, cudaStream_t s);
void launch_geometry(const double2 *gates, const double2 *dirs, const double *env,
                     const double *env_dot, const int32_t *param_of, int n_gates, int n_params,
                     int k, int structure, int euclidean, const double *facc, double *f_out, double2 *rgrad,
                     double2 *hvps, cudaStream_t s);

// Host-memory evaluation (rq_eval.cu): copies inputs in and outputs out and
// synchronises.  want_env: 0 no gradient environments, 1 accumulate them,
// 2 reuse those of the previous evaluation at the same gates (HVPs need them
// for the Riemannian correction).
rq_status eval_host(rq_ctx *ctx, const double *gates, const double *dirs, int k, int want_env, double *f,
                    double *rgrad, double *hvps);
rq_status set_error(rq_ctx *ctx, rq_status code, const char *msg);
rq_status check_gates(rq_ctx *ctx, const double *gates);
rq_status check_gates_device(rq_ctx *ctx, const double *d_gates);
int gradient_space(const rq_ctx *ctx);
// Device-pointer evaluation on the context stream (capturable once the
// context's small buffers hold k directions: prepare_capacity first).
rq_status eval_device(rq_ctx *ctx, const double *gates, const double *dirs, int k, int env_mode, double *f,
                      double *rgrad, double *hvps);
rq_status prepare_capacity(rq_ctx *ctx, int k);
cudaStream_t ctx_stream(const rq_ctx *ctx);
long long workspace_bytes_for(const rq_ctx *ctx, int columns_per_tile, int kc);

// Read-only view of a set-up context for entry points outside the context files.
struct CtxView {
    bool ready;
    int device, n, g, P, structure, sms;
    long long n_store, c0, c1;
    const GateGeom *geo;
    cudaStream_t stream;
    TargetDev target;
};
CtxView ctx_view(const rq_ctx *ctx);

// Host helpers.
int polar_unitary_4x4(const double *A, double *Q);    // rq_tr.cpp; 32 doubles in/out, 0 on success
double bessel_j_table(double x, int kmax, std::vector<double> &out);  // rq_target.cu; J_0..J_kmax(x)

}  // namespace rq
