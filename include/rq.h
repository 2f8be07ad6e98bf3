/*
 * rq.h -- C ABI of the GB300 matrix-free Riemannian circuit optimiser.
 *
 * Problem (paper Sec. "Problem statement and setup"): a sequence of two-qubit
 * gates G_1..G_g (each a 4x4 unitary on a listed qubit pair, G_1 applied
 * first) approximates a target U = exp(-iHt).  The cost is
 *     f(G) = -Re Tr[U^dagger C(G)]                        (Eq. f_target)
 * evaluated as a sum over computational basis columns j,
 *     f(G) = -Re sum_j <j| U^dagger C(G) |j>             (Eq. f_target_sum_unit_vec)
 * with no 2^n x 2^n matrix ever formed.  The library also returns the
 * Riemannian gradient (Eq. def_grad, Eq. grad_proj) and Riemannian
 * Hessian-vector products (Eq. vector_field_derivative, Eq. hessian_def,
 * Appendix "Evaluating Hessian-vector products"), and runs one
 * trust-region / truncated-CG iteration (Sec. "Riemannian optimization").
 *
 * Conventions shared by every call:
 *  - qubit 0 is the most significant bit of an amplitude index;
 *  - a gate on listed pair (a, b) is a 4x4 complex128 matrix, row-major,
 *    interleaved (re, im) doubles, local index 2*bit_a + bit_b
 *    (Eq. gate_application_neighboring and its general form);
 *  - "gates" arrays hold one matrix per parameter gate: [n_params][4][4]
 *    complex128 = 32 doubles per gate; the circuit maps sequential gate l to
 *    parameter param_of[l] (tied copies, Sec. "Brick wall circuit layout");
 *  - structure 1 = parity-conserving gates (Eq. paritygatematrix): entries
 *    outside the pattern are ignored on input and zero on output;
 *  - all results are sums over the current column range (rq_set_columns;
 *    default: all 2^n basis columns).  Partial sums over disjoint ranges add
 *    up to the full result (every output is linear in the per-column terms).
 *
 * Ownership: every pointer argument is owned by the caller; the library
 * copies what it reads before returning (host variants) or in stream order
 * (_dev variants) and keeps no caller pointer.  The library owns its device
 * workspace (allocated at rq_setup_target, freed at rq_destroy).
 *
 * Errors: every call returns RQ_OK (0) or a negative rq_status; the text of
 * the last error of a context is rq_last_error(ctx).  After an error the
 * outputs are unspecified and the context stays usable, except after
 * RQ_ECUDA from a sticky device error.  Calls on one context must not run
 * concurrently from several host threads.
 */
#ifndef RQ_H
#define RQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rq_ctx rq_ctx;
typedef int rq_status;

#define RQ_OK 0
#define RQ_EINVAL (-1)   /* invalid argument (sizes, pairs, indices, NULL) */
#define RQ_ENOMEM (-2)   /* device workspace does not fit */
#define RQ_ECUDA (-3)    /* a CUDA runtime call failed */
#define RQ_ETIMEOUT (-4) /* reserved for a bounded device wait; no kernel of this library spins */
#define RQ_ESTATE (-5)   /* call out of order (no target set up yet) */

/* Circuit topology (paper Sec. "Quantum circuits"): gate l acts on qubits
 * pairs[2l], pairs[2l+1] (distinct, in [0, n_qubits)) with parameter gate
 * param_of[l] in [0, n_params) (NULL: param_of[l] = l, n_params = n_gates).
 * structure: 0 general U(4) gates, 1 parity-conserving gates. */
typedef struct {
    int n_qubits;
    int n_gates;
    int n_params;
    int structure;
    const int32_t *pairs;
    const int32_t *param_of;
} rq_circuit;

/* Target U = exp(-i H t).  model 0: spinful Fermi-Hubbard chain (Eq. sfFH)
 * on n_sites sites, qubit j = (site j, up), qubit n_sites + j = (site j,
 * down), hopping -J on nearest-neighbour bonds of each spin chain (plus the
 * wrap bond without Z string when periodic, Eq. slFH_qubit), on-site U;
 * n_qubits = 2 * n_sites.  model 1: spinless chain in its hard-core boson
 * form (Eq. slFH_qubit): hopping -J and nearest-neighbour interaction
 * U n_j n_{j+1} on every bond (wrap bond if periodic); n_qubits = n_sites.
 * model 2: any dense target matrix (the cost of Eq. f_target_sum_unit_vec
 * with U given entry by entry, for tests and for targets that are not a
 * chain Hamiltonian's evolution): dense_U points to 2^n x 2^n complex128
 * values, row-major, interleaved (re, im), 2 <= n_qubits <= 14; n_sites,
 * periodic, J, U and t are ignored.  The matrix is copied during
 * rq_setup_target and not referenced afterwards.  With parity gates only its
 * two parity-diagonal blocks are used (the circuit keeps each column in its
 * parity sector, so the other entries do not enter f).  Models 0 and 1 leave
 * dense_U unread (NULL is fine). */
typedef struct {
    int model;
    int n_sites;
    int periodic;
    double J;
    double U;
    double t;
    const double *dense_U;
} rq_target;

/* One trust-region iteration (Absil et al. Algorithm 10 with truncated CG,
 * Algorithm 11; paper Sec. "Riemannian optimization").  In: radius,
 * max_radius, rho_accept, kappa, theta, max_inner (0: tangent dimension).
 * Out: f (cost at the input gates), f_new (cost at the candidate), rho,
 * grad_norm, step_norm, accepted, n_inner, tcg_exit (0 residual small,
 * 1 negative curvature, 2 hit the radius, 3 iteration cap); radius is
 * updated in place. */
typedef struct {
    double radius;
    double max_radius;
    double rho_accept;
    double kappa;
    double theta;
    int max_inner;
    double f;
    double f_new;
    double rho;
    double grad_norm;
    double step_norm;
    int accepted;
    int n_inner;
    int tcg_exit;
    int full_hessian;   /* in: 1 = compute the full Hessian once (rq_hessian) and run
                           tCG on it on the host; 0 = one device HVP per tCG step */
} rq_tr_state;

/* Sizes and counters of a set-up context (diagnostics and benchmarking). */
typedef struct {
    int n_qubits;
    int n_gates;
    int n_params;
    int structure;
    int64_t amplitudes_per_column;  /* 2^n, or 2^(n-1) for parity gates */
    int64_t columns;                /* columns in the current range */
    int columns_per_tile;           /* B: basis columns swept together */
    int n_tiles;
    int max_dirs;                   /* HVP directions swept together */
    int64_t workspace_bytes;        /* device memory held by the context */
    int64_t target_entries;         /* complex entries of the stored U blocks */
    int64_t kernel_launches;        /* kernels launched since rq_create */
    int ctas_per_sweep;             /* grid of the sweep kernels (rq_set_grid) */
} rq_info_t;

/* Create a context on CUDA device `device`.  cuda_stream: a cudaStream_t to
 * run on, or NULL to create a private stream.  *out receives the context. */
rq_status rq_create(rq_ctx **out, int device, void *cuda_stream);

/* Free the context and all its device memory.  NULL is accepted. */
rq_status rq_destroy(rq_ctx *ctx);

/* Build the device-resident target and workspace for a circuit.  The matrix
 * -free action of U (paper Sec. "Objective function and matrix-free
 * evaluation") is realised by per-sector blocks: H conserves the spin-resolved
 * particle numbers, so U is block diagonal over (N_up, N_down) sectors; each
 * block is built on the device by a Chebyshev expansion of exp(-iHt) with the
 * sparse H.  Resets the column range to all 2^n columns, the translation
 * and the checkpointing request; the tile request, arithmetic, output space,
 * graphs, checks and first-layer settings of the context persist.  A context
 * may be set up again for another problem at any time (the previous problem's
 * device memory is released first).  Errors: RQ_EINVAL for an invalid
 * circuit/target, RQ_ENOMEM if the target or the workspace does not fit; the
 * context then holds no problem (RQ_ESTATE until the next set-up). */
rq_status rq_setup_target(rq_ctx *ctx, const rq_target *target, const rq_circuit *circuit);

/* Restrict the basis sum to columns j in [col_begin, col_end) (shards of
 * Sec. "Parallelization").  RQ_EINVAL unless 0 <= begin <= end <= 2^n. */
rq_status rq_set_columns(rq_ctx *ctx, int64_t col_begin, int64_t col_end);

/* Tuning: columns per tile (a power of two, 0 = automatic) and the number of
 * HVP directions swept together (1..4, 0 = automatic).  Reallocates the
 * workspace; RQ_ENOMEM if it does not fit.  Directions beyond max_dirs are
 * swept in further chunks, each repeating the forward and adjoint sweeps;
 * the automatic choice keeps tiles of at least 256 columns, which at n = 16
 * means one direction per sweep, so callers that evaluate k > 1 directions
 * per call should pass max_dirs = k (e.g. 128 columns x 4 directions at
 * n = 16: 25 % less work per 4-direction evaluation than 4 chunks). */
rq_status rq_set_tile(rq_ctx *ctx, int columns_per_tile, int max_dirs);

/* Full Hessian (paper Sec. "Efficient gradient and Hessian computation",
 * Fig. hole_application, Fig. hessian_pass_second_gradient): forward and
 * backward pass keeping every state, then for each gate l the hole of G_l
 * applied to psi_{l-1} (a state-vector array with one member per gate entry,
 * 8 for parity gates) propagated through the later gates and contracted at
 * every later gate l'.  Returns, over the column range, f, the Euclidean
 * gradient gbar = d_x f + i d_y f (Eq. def_grad; egrad [n_params][4][4],
 * masked for parity gates; may be NULL) and the holomorphic second
 * derivatives of F = Tr[U^dagger C(G)] (f = -Re F) with tied copies summed:
 * hess[(p*16 + a*4 + b) * D + (q*16 + c*4 + d)] = d^2 F / dG_p[a,b] dG_q[c,d],
 * complex128, D = 16 n_params (symmetric; zero outside the parity pattern).
 * The real Hessian of f in (Re, Im) coordinates is [[-Re H, Im H], [Im H,
 * Re H]], and the Euclidean HVP along X is -conj(H vec(X)).  Runs in FP64
 * whatever rq_set_arithmetic says; allocates (g + 2 * members) tiles of
 * temporaries for the call (RQ_ENOMEM if they do not fit: lower the tile
 * size).  Cost per tile ~ 16 g^2 / 2 gate passes (8 g^2 / 2 for parity). */
rq_status rq_hessian(rq_ctx *ctx, const double *gates, double *f, double *egrad, double *hess);

/* Translation-representative basis sums (paper Sec. "Exploiting
 * translational invariance", applied here to the basis sum).  If the chain is
 * periodic and the circuit is invariant under shifting every site by
 * shift_sites (checked: in each run of pairwise disjoint gates the set of
 * (qubit pair, parameter) maps onto itself, e.g. one tied gate per brickwall
 * layer with shift_sites = 2), U and C(G) both commute with the shift T, so the
 * summand of Eq. f_target_sum_unit_vec -- and the tied gradient and HVP
 * summands -- are equal on every orbit {j, Tj, T^2 j, ...}.  The sums then run
 * over one representative per orbit weighted by the orbit size (about L /
 * shift_sites times fewer columns).  Requires the whole basis as the column
 * range; shift_sites = 0 switches back to plain sums.  RQ_EINVAL if the chain
 * is open, the shift does not divide the sites, or the circuit is not
 * invariant. */
rq_status rq_set_translation(rq_ctx *ctx, int shift_sites);

/* First-layer support, on by default.  The sweeps start from basis states
 * (paper Eq. f_target_sum_unit_vec), so before gate l of the leading run of
 * pairwise disjoint gates (the first brickwall layer) psi of column j
 * differs from |j> only on the qubits of the earlier gates of the run: the
 * sweeps of those gates (FP64 and double-float) visit only the 4^(l-1) items
 * per column where psi can be nonzero (forward and backward; the adjoint
 * state is read later only on that set), about 8 % of the work of a 78-gate
 * n = 16 circuit.  The results equal the full sweeps up to the order of the
 * sums (~1e-16 relative).  A parity gate on the implied qubit 0 sweeps all of
 * its items.  enable = 0 sweeps every item. */
rq_status rq_set_first_layer(rq_ctx *ctx, int enable);

/* Last-layer support, on by default.  The backward sweep of column j starts
 * from U|j> (paper Eq. f_target_sum_unit_vec), which lies in j's particle-
 * number sector (the chain Hamiltonians conserve the up and down counts, or
 * the one count of the spinless chain), and the gates of the trailing run of
 * pairwise disjoint gates (the last brickwall layer) change it only on their
 * own qubits.  So at gate l of the run an item (the four amplitudes the gate
 * mixes) can be nonzero only if the bits outside the qubits of gates l..g of
 * the run can be completed to a state of j's sector; the backward kernels
 * (FP64 and double-float) skip the other items, whose adjoint amplitudes and
 * environment terms are zero (a warp skips when all its 32 columns do).
 * General gates with a chain target only (parity tiles and dense targets
 * sweep every item).  The results equal the full sweeps up to the order of
 * the sums.  enable = 0 sweeps every item. */
rq_status rq_set_last_layer(rq_ctx *ctx, int enable);

/* Gate validation, off by default.  With enable = 1 every rq_cost, rq_grad,
 * rq_hvp, rq_tr_step (each evaluation inside it) and rq_hessian call, and
 * the _dev variants (which then copy the gates to the host and synchronise
 * the stream), first checks each parameter gate: finite entries,
 * ||G^H G - I||_F <= 1e-10 (the gates are points of U(4), Sec. "Riemannian
 * optimization"), and for parity gates (Eq. paritygatematrix) no entry above
 * 1e-10 outside the parity pattern.  A failed check returns RQ_EINVAL with the
 * gate index and the deviation in rq_last_error, before any launch
 * (rq_cost_static included).  The batch calls do not check. */
rq_status rq_set_checks(rq_ctx *ctx, int enable);

/* CUDA graphs for the host-memory calls (rq_cost, rq_grad, rq_hvp and the
 * evaluations inside rq_tr_step; a launch mechanism, no counterpart in the
 * paper): with enable = 1 (default) the kernel sequence of an evaluation is
 * captured once per (k, kind) and replayed as one graph launch until the
 * context's configuration changes what the kernels are given (tile layout,
 * arithmetic, output space, translation, checkpointing, first-layer support,
 * profiling; a new column range of the same layout keeps the graphs), which
 * removes the host's per-kernel launch cost.  Results are bitwise those of
 * direct launches.  enable = 0 launches kernels directly.  A stream that
 * cannot be captured (the legacy default stream) falls back to direct
 * launches. */
rq_status rq_set_graphs(rq_ctx *ctx, int enable);

/* Grid of the sweep kernels (throughput vs latency).  0 (default): every
 * sweep launches enough CTAs to fill the GPU (two per SM when the tile has a
 * full block of items for each, otherwise at most one per SM and one
 * warp-sized chunk of items per CTA), the fastest schedule for a context that
 * has the GPU to itself.  m > 0: at most as many CTAs as give every thread m
 * items of a full sweep, so that each CTA's fixed costs (gate tables, the
 * environment reduction, the pipeline's first load) are paid over more items;
 * meant for contexts whose sweeps run concurrently with other contexts'
 * (rq_batch, a server), which fill the rest of the GPU.  The results change
 * only in the rounding of the environment sums (a different reduction tree),
 * and stay reproducible for a given m.  Reallocates the partial-sum buffers;
 * RQ_EINVAL unless 0 <= m <= 2^20.  rq_get_info reports the grid
 * (ctas_per_sweep). */
rq_status rq_set_grid(rq_ctx *ctx, int min_items_per_thread);

/* Checkpointing of the forward pass (memory vs recomputation).  interval 1
 * (default): every intermediate state of a tile is kept (the paper's
 * forward-pass cache, Fig. forward_pass).  interval r > 1: only the state at
 * the start of every segment of r gates is kept, plus one segment buffer; the
 * backward pass recomputes each segment from its checkpoint (about g / r + r
 * instead of g + 1 states per tile, for one extra forward sweep).  Results are
 * bitwise those of interval 1.  interval 0 (default): automatic -- every
 * state unless that would force tiles below min(256, columns), then a
 * checkpoint every ceil(sqrt(g)) gates.  The workspace is reallocated (the
 * tile size may grow); rq_hessian needs an effective interval of 1. */
rq_status rq_set_checkpointing(rq_ctx *ctx, int interval);

/* Window fusion of the forward pass (Sec. "Brick wall circuit layout": the
 * gates of a layer act on disjoint qubits and commute).  max_window_qubits 0
 * (default): every gate is one pass over the tile, in circuit order.  3..6:
 * after the leading run of disjoint gates, each pass starts at the next gate
 * and takes, one at a time, the later gate that fits in a window of that many
 * stored qubits, moves only past gates on disjoint qubits (with which it
 * commutes) and adds the fewest new qubits to the window: a CTA
 * holds [2^q amplitudes x 32 columns] of the state (and of each tangent) in
 * shared memory, applies the pass's gates (at most 16) there, and writes to
 * HBM only the checkpoints the backward pass needs (every state of a
 * gradient or HVP evaluation; only the pass's output for a cost).  The
 * backward pass runs the same order in reverse.  Parity gates on the implied
 * qubit 0 are not fused.  Fusion applies when the checkpoint interval is 1
 * and tiles have at least 32 columns; otherwise the unfused schedule runs.
 * Results equal the unfused ones up to the order of floating-point sums.
 * Returns RQ_EINVAL for a window outside {0} U [3, 6].  The setting is kept
 * across rq_setup_target.
 *
 * rq_fusion_info: number of passes of the current plan, gates inside
 * multi-gate passes, and the largest pass (any output may be NULL). */
rq_status rq_set_fusion(rq_ctx *ctx, int max_window_qubits);
rq_status rq_fusion_info(const rq_ctx *ctx, int *n_passes, int *fused_gates, int *max_pass_gates);

/* Arithmetic of the sweep kernels (forward, adjoint, environments).
 * RQ_ARITH_FP64 (default): IEEE binary64 on the FP64 pipe.  RQ_ARITH_DF64:
 * every amplitude and gate entry is kept as an unevaluated sum of two floats
 * (about 48 significant bits) and the gate applications and gate-hole
 * contractions run on the FP32 pipe with error-free transformations (two-sum,
 * FMA two-product; a compensated dot product in twice the float precision),
 * which GB300 executes far faster than FP64.  The target, the reductions and
 * the Riemannian post-processing stay FP64; results agree with the FP64 ones
 * to about 1e-13 relative (the tests hold both to 1e-12 against the FP64
 * oracle).  The paper's kernels are FP64 on CPUs; this option has no
 * counterpart there.  RQ_EINVAL for any other value. */
#define RQ_ARITH_FP64 0
#define RQ_ARITH_DF64 1
rq_status rq_set_arithmetic(rq_ctx *ctx, int arith);

/* Output space of rq_grad / rq_hvp (and their _dev variants).
 * RQ_SPACE_RIEMANNIAN (default): grad f = P_G(gbar) (Eq. grad_proj) and
 * Hess f(G)[X] (Eq. hessian_def) with X projected onto the tangent space.
 * RQ_SPACE_EUCLIDEAN: the cost extended to all complex 4x4 matrices (as an
 * autograd framework sees it): gbar = d_x f + i d_y f (Eq. def_grad, tied
 * copies summed) and the Euclidean Hessian applied to the raw direction,
 * Dgbar[X] = d/de gbar(G + e X) at e = 0; for parity circuits both are masked
 * to the pattern of Eq. paritygatematrix.  rq_tr_step always works in the
 * Riemannian space.  RQ_EINVAL for any other value. */
#define RQ_SPACE_RIEMANNIAN 0
#define RQ_SPACE_EUCLIDEAN 1
rq_status rq_set_gradient_space(rq_ctx *ctx, int space);

/* f(G) over the column range (Eq. f_target_sum_unit_vec).  gates: host
 * [n_params][4][4] complex128; f: host double. */
rq_status rq_cost(rq_ctx *ctx, const double *gates, double *f);

/* f and the Riemannian gradient grad f = P_G(d_x f + i d_y f) (Eq. def_grad,
 * Eq. grad_proj; forward and backward pass of Sec. "Efficient gradient and
 * Hessian computation"), tied copies summed.  rgrad: host [n_params][4][4]
 * complex128 (may be NULL). */
rq_status rq_grad(rq_ctx *ctx, const double *gates, double *f, double *rgrad);

/* f, the Riemannian gradient and k Riemannian Hessian-vector products
 * Hess f(G)[X_i] (Eq. hessian_def; forward mode then reverse, Appendix
 * "Evaluating Hessian-vector products").  dirs: host [k][n_params][4][4]
 * complex128 raw directions; each is first projected onto the tangent space
 * (P_G, Eq. proj_tangent, then the parity pattern).  hvps: host
 * [k][n_params][4][4].  k >= 0; rgrad/hvps may be NULL. */
rq_status rq_hvp(rq_ctx *ctx, const double *gates, const double *dirs, int k,
                 double *f, double *rgrad, double *hvps);

/* Device-pointer variants of the three calls above: every pointer is device
 * memory of the same shape, work is queued on the context stream and the
 * call returns without synchronising. */
rq_status rq_cost_dev(rq_ctx *ctx, const double *gates, double *f);
rq_status rq_grad_dev(rq_ctx *ctx, const double *gates, double *f, double *rgrad);
rq_status rq_hvp_dev(rq_ctx *ctx, const double *gates, const double *dirs, int k,
                     double *f, double *rgrad, double *hvps);

/* One trust-region iteration on the host gates (in/out: replaced by the
 * candidate when accepted).  Every cost, gradient and HVP inside runs on the
 * device over the current column range. */
rq_status rq_tr_step(rq_ctx *ctx, double *gates, rq_tr_state *state);

/* Column U|j> of the stored target as 2^n complex128 (host `out`, zero
 * outside the sector of j).  RQ_EINVAL unless 0 <= j < 2^n. */
rq_status rq_target_column(rq_ctx *ctx, int64_t j, double *out);

/* Sizes and counters of the context. */
rq_status rq_get_info(const rq_ctx *ctx, rq_info_t *info);

/* Cost without allocation.  The paper has no counterpart: this entry point
 * exists for callers that cannot let a library call cudaMalloc while they
 * run -- a process whose device memory is all reserved by its own pool
 * allocator, or a latency-critical loop that must not issue cudaMalloc /
 * cudaFree because those calls synchronise the whole device.
 *
 * rq_cost_static computes the same f(G) as rq_cost over the context's column
 * range (host `gates` [n_params][4][4] complex128 in, host `f` out; the call
 * synchronises the context stream) but allocates nothing: all its scratch
 * lives in one file-scope device array of RQ_STATIC_SCRATCH_BYTES that every
 * GPU loading the library holds until the process exits.  A problem whose
 * single column does not fit (two state tiles of 2^n, or 2^(n-1) for parity
 * gates, complex128 amplitudes plus gate and column tables) is rejected with
 * RQ_EINVAL and a message naming the limit; larger column ranges are swept in
 * tiles of at most 256 columns.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current) and
 * caches it; make that first call before any stream capture.  Every call,
 * from any context on the device, shares the array and finds the previous
 * call's contents there (each call clears what must start at zero); calls
 * whose GPU work overlaps race on it and give wrong results.  The cached
 * address does not survive a cudaDeviceReset: do not keep using the library
 * on a device after resetting it.  The sweep is always FP64 over every column
 * of the range (rq_set_arithmetic and rq_set_translation do not apply; the
 * full sum equals the translation-weighted one), and gates are validated as
 * in rq_cost when rq_set_checks is on. */
#define RQ_STATIC_SCRATCH_BYTES (16u << 20)
rq_status rq_cost_static(rq_ctx *ctx, const double *gates, double *f);

/* Batches of independent problems (uneven n, depth, t, U; paper Sec.
 * "Parallelization": the basis sums of different problems are independent).
 * Every problem has its own context (target blocks, workspace, stream).  One
 * evaluation of the whole batch is one CUDA-graph launch whose branches run
 * the problems concurrently; results are bitwise those of each problem
 * evaluated alone with the same sweep grid (rq_batch_set_grid).  The columns-per-tile of the batch is autotuned at the
 * first evaluation (rq_batch_set_tile(b, 0)) or fixed (power of two).
 *
 * rq_batch_hvp: host arrays.  gates: every problem's [n_params][4][4]
 * complex128 concatenated in the order of rq_batch_add; dirs: for each
 * problem [k][n_params][4][4], concatenated the same way; f: [n_problems];
 * rgrad: same layout as gates; hvps: same layout as dirs (Riemannian
 * quantities as in rq_hvp; NULL outputs are skipped).  plain = 1 evaluates
 * the problems one after another without the graph (for comparison).
 * Synchronises.  rq_batch_info: problem count, chosen tile, and the
 * autotuner's timings (ms per cost-only batch evaluation for tile caps 64,
 * 128, 256, 512; -1 where the cap did not fit). */
typedef struct rq_batch rq_batch;
rq_status rq_batch_create(rq_batch **out, int device);
rq_status rq_batch_destroy(rq_batch *b);
rq_status rq_batch_add(rq_batch *b, const rq_target *target, const rq_circuit *circuit, int *index);
rq_status rq_batch_set_tile(rq_batch *b, int columns_per_tile);
rq_status rq_batch_hvp(rq_batch *b, const double *gates, const double *dirs, int k, int plain, double *f,
                       double *rgrad, double *hvps);
rq_status rq_batch_info(const rq_batch *b, int *n_problems, int *columns_per_tile, double *tune_ms);
/* Gates per forward pass of every problem of the batch (rq_set_fusion).
 * max_window_qubits -1 (default): autotuned at the first evaluation after the
 * tile size, by timing the captured cost-only batch evaluation with fusion
 * off and with windows of 4, 5 and 6 stored qubits and keeping the fastest;
 * 0: off; 3..6: that window for every problem.  rq_batch_fusion_info: the
 * window in use and the autotuner's timings (ms for windows 0, 4, 5, 6; -1
 * where not timed). */
rq_status rq_batch_set_fusion(rq_batch *b, int max_window_qubits);
/* Sweep grid of every problem of the batch (rq_set_grid).  min_items_per_thread
 * -1 (default): autotuned at the first evaluation after the tile size, by
 * timing the captured gradient evaluation of the batch with 0, 8, 16, 32 and
 * 64 items per thread and keeping the fastest (the problems' concurrent
 * sweeps share the GPU, so each needs fewer CTAs than alone); 0: every
 * problem's sweeps fill the GPU as if alone; m > 0: that grid for every
 * problem.  The grid applies to the graph and to plain = 1 alike (batched and
 * plain results stay bitwise equal); a one-at-a-time comparison at its own
 * best grid sets 0 first.  rq_batch_grid_info: the grid in use and the
 * autotuner's timings (ms for 0, 8, 16, 32, 64; -1 where not timed). */
rq_status rq_batch_set_grid(rq_batch *b, int min_items_per_thread);
rq_status rq_batch_grid_info(const rq_batch *b, int *min_items_per_thread, double *tune_ms);
rq_status rq_batch_fusion_info(const rq_batch *b, int *window, double *tune_ms);
const char *rq_batch_last_error(const rq_batch *b);

/* Per-kernel timing of one context (benchmarking and roofline accounting).
 * Between rq_profile_start and rq_profile_stop every kernel the context
 * launches is bracketed by CUDA events on the context stream.  One record per
 * kernel family: launches, summed device time (ms) and the algorithmic FP64
 * flops (8 per complex multiply-add) and DRAM bytes (each input read once,
 * each output written once) of those launches.  `name` points to a static
 * string.  rq_profile_stop synchronises the stream, writes at most
 * `capacity` records and sets *n_stats to the number of families seen. */
typedef struct {
    const char *name;
    int64_t launches;
    double total_ms;
    double flops;
    double bytes;
} rq_kernel_stat;

rq_status rq_profile_start(rq_ctx *ctx);
rq_status rq_profile_stop(rq_ctx *ctx, rq_kernel_stat *stats, int capacity, int *n_stats);

/* Text of the last error on this context ("" if none); valid until the next
 * call on the context.  NULL ctx: the last rq_create failure. */
const char *rq_last_error(const rq_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* RQ_H */
