// rq_cost_static: the cost f(G) of a set-up context, computed without any
// device allocation.
//
// Some callers cannot let a library call cudaMalloc while they run: a process
// whose device memory is entirely reserved by its own pool allocator, or a
// latency-critical serving loop that must not issue cudaMalloc/cudaFree
// because those calls synchronise the whole device and stall every other
// stream.  rq_cost (through the context workspace) may grow that workspace;
// this entry point never allocates.  Its scratch -- the two state tiles of a
// ping-pong forward sweep, the masked gates, the column table and the
// per-column cost summands -- lives in one file-scope device array of fixed
// size, RQ_STATIC_SCRATCH_BYTES, that every GPU loading the library holds
// until the process exits.
//
// The array is shared by all calls (and all contexts) on a device and keeps
// the contents of the last call; each call clears what must start at zero.
// Calls whose GPU work overlaps (several host threads, or several streams)
// race on the array and give wrong results: serialise them.
//
// The sweep here is always the FP64 one over the context's whole column range
// (rq_set_arithmetic and rq_set_translation do not apply: the sum over every
// column of the range equals the weighted sum over orbit representatives).
// The array's device address is looked up once per device and kept for the
// life of the process, so the library must not outlive a cudaDeviceReset of a
// device it has used.
#include "rq_internal.h"

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[RQ_STATIC_SCRATCH_BYTES];

// Device address of g_static_scratch per device ordinal.  In host code the
// array's name is only a host-side stand-in, never a device address.
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// Cost summands -Re <U j_b | psi_g[:, b]> of one tile, one CTA per column.
// Same arithmetic and order as the sweep's target kernel, without the adjoint
// start tile (a cost needs no backward pass).
__global__ void k_overlap_static(const rq::TargetDev t, const int32_t *cols, int log2B, long long mask,
                                 const double2 *psi, double *fpart) {
    const int b = blockIdx.x;
    const int j = cols[b];
    double acc = 0.0;
    if (j >= 0) {
        const int s = t.sec_of[j];
        const long long m = t.off_basis[s + 1] - t.off_basis[s];
        const double2 *ucol = t.U + t.off_u[s] + (long long)t.pos[j] * m;
        const int32_t *bas = t.basis + t.off_basis[s];
        for (long long r = threadIdx.x; r < m; r += blockDim.x) {
            const long long o = (((long long)bas[r] & mask) << log2B) | b;
            const double2 u = ucol[r];
            const double2 p = psi[o];
            acc = fma(u.x, p.x, acc);
            acc = fma(u.y, p.y, acc);
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

long long round256(long long x) { return (x + 255) & ~255LL; }

int ilog2i(long long v) {
    int r = 0;
    while ((1LL << r) < v) ++r;
    return r;
}

rq_status err(rq_ctx *ctx, rq_status code, const std::string &msg) { return rq::set_error(ctx, code, msg.c_str()); }

}  // namespace

extern "C" rq_status rq_cost_static(rq_ctx *ctx, const double *gates, double *f) {
    if (!ctx) return RQ_EINVAL;
    const rq::CtxView v = rq::ctx_view(ctx);
    if (!v.ready) return err(ctx, RQ_ESTATE, "no target set up (call rq_setup_target first)");
    if (!gates || !f) return err(ctx, RQ_EINVAL, "gates or f is NULL");
    // the same host-side validation as rq_cost when rq_set_checks is on
    {
        const rq_status cs = rq::check_gates(ctx, gates);
        if (cs != RQ_OK) return cs;
    }
    if (v.device < 0 || v.device >= kMaxDevices) return err(ctx, RQ_EINVAL, "device ordinal too large");

    int prev_dev = 0;
    if (cudaGetDevice(&prev_dev) != cudaSuccess) return err(ctx, RQ_ECUDA, "cudaGetDevice failed");
    if (prev_dev != v.device && cudaSetDevice(v.device) != cudaSuccess)
        return err(ctx, RQ_ECUDA, "cudaSetDevice failed");
    struct Restore {
        int dev, cur;
        ~Restore() {
            if (dev != cur) cudaSetDevice(dev);
        }
    } restore{prev_dev, v.device};

    // once per device, with that device current: the array's device address
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_addr[v.device]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess)
                return err(ctx, RQ_ECUDA, std::string("cudaGetSymbolAddress of the static scratch: ") +
                                              cudaGetErrorString(e));
            g_scratch_addr[v.device] = static_cast<unsigned char *>(p);
        }
        base = g_scratch_addr[v.device];
    }

    // column lists of the range (even- then odd-parity columns for parity gates)
    std::vector<std::vector<int32_t>> groups;
    std::vector<int> gpar;
    if (v.structure == 1) {
        groups.resize(2);
        gpar = {0, 1};
        for (long long j = v.c0; j < v.c1; ++j) groups[__builtin_popcountll(j) & 1].push_back((int32_t)j);
    } else {
        groups.resize(1);
        gpar = {0};
        for (long long j = v.c0; j < v.c1; ++j) groups[0].push_back((int32_t)j);
    }
    long long largest = 1;
    for (auto &gr : groups) largest = std::max<long long>(largest, (long long)gr.size());

    // scratch layout for B columns per tile; the largest B <= 256 that fits
    const long long gbytes = round256((long long)v.P * 16 * (long long)sizeof(double2));
    auto layout_bytes = [&](long long B, long long ntiles) {
        return 2 * gbytes + 256 + round256(B * (long long)sizeof(double)) + round256(ntiles * B * 4) +
               2 * round256(v.n_store * B * (long long)sizeof(double2));
    };
    auto n_tiles_for = [&](long long B) {
        long long t = 0;
        for (auto &gr : groups) t += ((long long)gr.size() + B - 1) / B;
        return t;
    };
    long long B = std::min<long long>(256, 1LL << ilog2i(largest));
    while (B > 1 && layout_bytes(B, n_tiles_for(B)) > (long long)RQ_STATIC_SCRATCH_BYTES) B >>= 1;
    if (layout_bytes(B, n_tiles_for(B)) > (long long)RQ_STATIC_SCRATCH_BYTES)
        return err(ctx, RQ_EINVAL,
                   "problem too large for rq_cost_static: one column needs " +
                       std::to_string(layout_bytes(1, n_tiles_for(1))) + " bytes of static scratch, the maximum is " +
                       std::to_string((long long)RQ_STATIC_SCRATCH_BYTES) + " (RQ_STATIC_SCRATCH_BYTES)");
    const int log2B = ilog2i(B);
    std::vector<int32_t> cols;
    std::vector<int> tpar;
    for (size_t gi = 0; gi < groups.size(); ++gi)
        for (size_t s0 = 0; s0 < groups[gi].size(); s0 += (size_t)B) {
            for (long long b = 0; b < B; ++b)
                cols.push_back(s0 + b < groups[gi].size() ? groups[gi][s0 + b] : -1);
            tpar.push_back(gpar[gi]);
        }

    double2 *g_in = reinterpret_cast<double2 *>(base);
    double2 *g_mask = reinterpret_cast<double2 *>(base + gbytes);
    double *facc = reinterpret_cast<double *>(base + 2 * gbytes);
    double *fpart = reinterpret_cast<double *>(base + 2 * gbytes + 256);
    int32_t *d_cols = reinterpret_cast<int32_t *>(base + 2 * gbytes + 256 + round256(B * (long long)sizeof(double)));
    unsigned char *tiles = base + 2 * gbytes + 256 + round256(B * (long long)sizeof(double)) +
                           round256((long long)tpar.size() * B * 4);
    const long long tile_elems = v.n_store * B;
    double2 *psi[2] = {reinterpret_cast<double2 *>(tiles),
                       reinterpret_cast<double2 *>(tiles + round256(tile_elems * (long long)sizeof(double2)))};

    cudaStream_t s = v.stream;
#define RQS_CUDA(call)                                                                         \
    do {                                                                                       \
        const cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) return err(ctx, RQ_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
    RQS_CUDA(cudaMemcpyAsync(g_in, gates, sizeof(double2) * 16 * v.P, cudaMemcpyHostToDevice, s));
    if (!cols.empty())
        RQS_CUDA(cudaMemcpyAsync(d_cols, cols.data(), cols.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    RQS_CUDA(cudaMemsetAsync(facc, 0, sizeof(double), s));  // the array keeps the last call's sum
    rq::launch_mask_gates(g_in, g_mask, v.P, v.structure, s);
    RQS_CUDA(cudaGetLastError());
    const long long mask = v.structure == 1 ? ((1LL << (v.n - 1)) - 1) : ((1LL << v.n) - 1);
    for (size_t ti = 0; ti < tpar.size(); ++ti) {
        const int32_t *tcols = d_cols + (long long)ti * B;
        RQS_CUDA(cudaMemsetAsync(psi[0], 0, sizeof(double2) * tile_elems, s));
        rq::launch_init_unit(psi[0], tcols, (int)B, log2B, v.n_store, v.structure, s);
        RQS_CUDA(cudaGetLastError());
        int cur = 0;
        for (int l = 0; l < v.g; ++l) {
            const rq::GateGeom &geo = v.geo[l];
            rq::FwdArgs a{};
            a.psi_in = psi[cur];
            a.psi_out = psi[1 - cur];
            a.kdirs = 0;
            a.gate = g_mask + (long long)geo.param * 16;
            a.geo = geo;
            a.log2B = log2B;
            a.tile_parity = tpar[ti];
            a.n_items = (geo.mode == rq::kParity2 ? v.n_store / 2 : v.n_store / 4) * B;
            const long long blocks = (a.n_items + rq::kThreads - 1) / rq::kThreads;
            rq::launch_fwd(a, (int)std::min<long long>((long long)v.sms * rq::kCtasPerSm, std::max<long long>(1, blocks)), s);
            RQS_CUDA(cudaGetLastError());
            cur = 1 - cur;
        }
        k_overlap_static<<<(unsigned)B, 128, 0, s>>>(v.target, tcols, log2B, mask, psi[cur], fpart);
        RQS_CUDA(cudaGetLastError());
        rq::launch_reduce_f(fpart, (int)B, facc, s);
        RQS_CUDA(cudaGetLastError());
    }
    RQS_CUDA(cudaMemcpyAsync(f, facc, sizeof(double), cudaMemcpyDeviceToHost, s));
    RQS_CUDA(cudaStreamSynchronize(s));
#undef RQS_CUDA
    return RQ_OK;
}
