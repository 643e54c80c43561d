// eik_solve_noalloc: one solve that allocates no device memory.
//
// Some callers cannot call cudaMalloc while they solve: code that runs under a
// caching allocator or a memory pool it does not own (an allocation there
// takes memory behind the pool's back, or fails once the pool has reserved
// the device), and embedders that must not grow the process's device
// footprint at solve time.  For them this entry point keeps every piece of
// working memory of a solve (h/F in brick layout, the two psi copies of each
// brick, the Upsilon masks, stamps, work lists, control block and the
// fixed-node tables) in one file-scope device array of fixed size, and its
// host-side set-up uses fixed-size arrays on the stack.  The caller passes the
// speeds and the output buffer, both in device memory.
//
// The array is part of the library image: every GPU that loads libeik holds
// it until the process exits.  Host code cannot use the array's name as a
// device address, so its address is looked up with cudaGetSymbolAddress once
// per device, on the first call made with that device current; make that
// first call before any stream capture.  All calls share the array and it
// keeps the last call's contents, so calls that overlap on the GPU (two host
// threads, or asynchronous work on two streams) race; each call clears what
// must start from zero (stamps, work-list state, control block) itself.
#include "eik.h"
#include "eik_host.h"
#include "eik_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

namespace eikg {
template <typename T>
cudaError_t launch_layout_speed(const T*, T*, int, int, int, int, int, int64_t, double, int*, int, cudaStream_t);
template <typename T>
cudaError_t launch_init_sources(int, const int32_t*, const int32_t*, const double*, int, const int32_t*, int,
                                const int32_t*, int, const int32_t*, T*, unsigned long long*, unsigned long long*,
                                int32_t*, int32_t*, T*, T*, int32_t*, int32_t*, cudaStream_t);
template <typename T>
cudaError_t launch_restore_r(int, const int32_t*, const int32_t*, const T*, T*, cudaStream_t);
template <typename T>
cudaError_t launch_gather_r(int, const int32_t*, const int32_t*, const T*, double*, cudaStream_t);
template <typename T>
cudaError_t launch_result(const T*, const unsigned long long*, T*, int, int, int, int, int, int, cudaStream_t);
template <typename T>
cudaError_t loop_occupancy(int*);
template <typename T>
cudaError_t launch_restart_loop(const LoopParams<T>&, int, cudaStream_t);
}  // namespace eikg

namespace {

constexpr size_t kScratchBytes = EIK_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;
constexpr int kMaxFix = 8 * EIK_NOALLOC_MAX_SOURCES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
thread_local std::string g_err;

eik_status fail(eik_status s, const std::string& m) {
    g_err = m;
    return s;
}

#define NA_CK(call)                                                                                     \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return fail(EIK_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_base(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
    size_t rr, slot, ups, stamp, queued, lists, done, ctrl, err, fix_b, fix_p, fix_v, src_b, enq, saved_r, cand_r,
        end;
};

Layout layout_for(int64_t nb) {
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += up256(bytes);
        return at;
    };
    L.rr = take(static_cast<size_t>(nb) * eikg::kBrick * sizeof(float));
    L.slot = take(static_cast<size_t>(nb) * 2 * eikg::kSlot * sizeof(float));
    L.ups = take(static_cast<size_t>(nb) * 12 * sizeof(unsigned long long));
    L.stamp = take(static_cast<size_t>(nb) * sizeof(unsigned long long));
    L.queued = take(eikg::kRing * static_cast<size_t>(nb) * sizeof(int32_t));
    L.lists = take(eikg::kRing * static_cast<size_t>(nb) * sizeof(int32_t));
    L.done = take(static_cast<size_t>(nb) * sizeof(int32_t));
    L.ctrl = take(sizeof(eikg::Ctrl));
    L.err = take(sizeof(int));
    L.fix_b = take(kMaxFix * sizeof(int32_t));
    L.fix_p = take(kMaxFix * sizeof(int32_t));
    L.fix_v = take(kMaxFix * sizeof(double));
    L.src_b = take(kMaxFix * sizeof(int32_t));
    L.enq = take(7 * kMaxFix * sizeof(int32_t));
    L.saved_r = take(kMaxFix * sizeof(float));
    L.cand_r = take(kMaxFix * sizeof(double));
    L.end = o;
    return L;
}

}  // namespace

extern "C" {

const char* eik_noalloc_last_error(void) { return g_err.c_str(); }

eik_status eik_solve_noalloc(const int32_t dims[3], double h, const float* F, int32_t nsrc, const double* xyz,
                             const eik_params* params, float* psi_out, eik_stats* stats, void* stream) {
    if (!dims || !F || !psi_out || !xyz) return fail(EIK_EINVAL, "eik_solve_noalloc: NULL argument");
    if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1) return fail(EIK_EINVAL, "eik_solve_noalloc: dims must be >= 1");
    if (!(std::isfinite(h) && h > 0.0)) return fail(EIK_EINVAL, "eik_solve_noalloc: h must be finite and > 0");
    if (nsrc < 1 || nsrc > EIK_NOALLOC_MAX_SOURCES)
        return fail(EIK_EINVAL, "eik_solve_noalloc: 1 <= nsrc <= EIK_NOALLOC_MAX_SOURCES");
    eik_params P;
    eik_params_default(&P);
    if (params) P = *params;
    if (!(P.stride > 0.0)) return fail(EIK_EINVAL, "eik_solve_noalloc: stride must be > 0 (+inf allowed)");
    {
        eik_status code;
        if (const char* m = eikh::param_error(P, &code)) return fail(code, std::string("eik_solve_noalloc: ") + m);
    }
    if (P.block_dim != 0 && P.block_dim != 8) return fail(EIK_ENOTSUP, "eik_solve_noalloc: block_dim must be 8");
    if (P.schedule != EIK_SCHED_FIXED) return fail(EIK_ENOTSUP, "eik_solve_noalloc: fixed-stride schedule only");
    if (P.log_restarts)
        return fail(EIK_ENOTSUP, "eik_solve_noalloc: no restart log (its records would need memory)");
    if (P.window == 0.0) P.window = 2.0;
    if (P.width == 0.0) P.width = INFINITY;
    if (P.max_restarts == 0) P.max_restarts = int64_t(1) << 24;
    const int nx = dims[0], ny = dims[1], nz = dims[2];
    const int BX = (nx + 7) / 8, BY = (ny + 7) / 8, BZ = (nz + 7) / 8;
    const int64_t nb = int64_t(BX) * BY * BZ;
    if (nb > EIK_NOALLOC_MAX_BRICKS)
        return fail(EIK_EINVAL, "eik_solve_noalloc: grid needs " + std::to_string(nb) +
                                    " bricks of 8^3 nodes; the fixed scratch holds at most " +
                                    std::to_string(EIK_NOALLOC_MAX_BRICKS));
    const Layout Lo = layout_for(nb);
    if (Lo.end > kScratchBytes) return fail(EIK_EINVAL, "eik_solve_noalloc: grid too large for the fixed scratch");
    for (int s = 0; s < nsrc; ++s)
        for (int a = 0; a < 3; ++a) {
            const double v = xyz[3 * s + a], ext = (dims[a] - 1) * h;
            if (!std::isfinite(v) || v < -1e-9 * h || v > ext + 1e-9 * h)
                return fail(EIK_EINVAL, "eik_solve_noalloc: source outside the grid");
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* base = nullptr;
    NA_CK(scratch_base(&base));
    char* B = static_cast<char*>(base);
    float* rr = reinterpret_cast<float*>(B + Lo.rr);
    float* slot = reinterpret_cast<float*>(B + Lo.slot);
    auto* ups = reinterpret_cast<unsigned long long*>(B + Lo.ups);
    auto* stampv = reinterpret_cast<unsigned long long*>(B + Lo.stamp);
    int32_t* queued = reinterpret_cast<int32_t*>(B + Lo.queued);
    int32_t* lists = reinterpret_cast<int32_t*>(B + Lo.lists);
    int32_t* done = reinterpret_cast<int32_t*>(B + Lo.done);
    auto* ctrl = reinterpret_cast<eikg::Ctrl*>(B + Lo.ctrl);
    int* err = reinterpret_cast<int*>(B + Lo.err);
    int32_t* d_fb = reinterpret_cast<int32_t*>(B + Lo.fix_b);
    int32_t* d_fp = reinterpret_cast<int32_t*>(B + Lo.fix_p);
    double* d_fv = reinterpret_cast<double*>(B + Lo.fix_v);
    int32_t* d_sb = reinterpret_cast<int32_t*>(B + Lo.src_b);
    int32_t* d_enq = reinterpret_cast<int32_t*>(B + Lo.enq);
    float* d_saved = reinterpret_cast<float*>(B + Lo.saved_r);
    double* d_cr = reinterpret_cast<double*>(B + Lo.cand_r);

    // speeds -> h/F in brick layout, with validation
    int bad = 0;
    NA_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    NA_CK(eikg::launch_layout_speed<float>(F, rr, nx, ny, nz, BX, BY, nb, h, err, 1, st));
    NA_CK(cudaMemcpyAsync(&bad, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    // fixed nodes (Alg. 1): the nodes of each source's cell with their h/F, psi0 = distance / F
    const eikh::Bricks geo{BX, BY, BZ, 0};
    eikh::Cand cand[kMaxFix];
    const int nc = eikh::source_candidates_into(xyz, nsrc, nx, ny, nz, h, geo, cand);
    int32_t cb[kMaxFix], cp[kMaxFix];
    for (int t = 0; t < nc; ++t) {
        cb[t] = cand[t].b;
        cp[t] = cand[t].p;
    }
    double cr[kMaxFix];
    NA_CK(cudaMemcpyAsync(d_fb, cb, nc * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(d_fp, cp, nc * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    NA_CK(eikg::launch_gather_r<float>(nc, d_fb, d_fp, rr, d_cr, st));
    NA_CK(cudaMemcpyAsync(cr, d_cr, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if (bad) return fail(EIK_EINVAL, "eik_solve_noalloc: F must be finite and >= 0 everywhere");
    eikh::FixNode fix[kMaxFix];
    const int nfix = eikh::fixed_nodes_into(cand, nc, cr, h, fix);
    // bricks with fixed nodes, and the work list of restart 1
    int32_t sb[kMaxFix], enq[7 * kMaxFix];
    int nsb = 0, nenq = 0;
    eikh::first_active_into(fix, nfix, geo, sb, &nsb, enq, &nenq);
    int32_t fb[kMaxFix], fp[kMaxFix];
    double fv[kMaxFix];
    for (int t = 0; t < nfix; ++t) {
        fb[t] = fix[t].b;
        fp[t] = fix[t].p;
        fv[t] = fix[t].v;
    }
    eikg::Ctrl H;
    std::memset(&H, 0, sizeof(H));
    H.k = nenq ? 1 : 0;
    H.bound_prev = -1.0;
    H.stride = P.stride;
    H.bound = std::fmin(0.0 + P.stride, P.width);
    H.count[1] = nenq;
    H.mode = 8;
    H.action = -1;
    H.pend_action = -1;
    H.r_rmin_bits = 0x7f800000u;
    H.done = nenq ? 0 : 1;
    // state that must start fresh: stamps and work-list marks (all ones), control block
    NA_CK(cudaMemsetAsync(stampv, 0xFF, static_cast<size_t>(nb) * sizeof(unsigned long long), st));
    NA_CK(cudaMemsetAsync(queued, 0xFF, eikg::kRing * static_cast<size_t>(nb) * sizeof(int32_t), st));
    NA_CK(cudaMemsetAsync(lists, 0xFF, eikg::kRing * static_cast<size_t>(nb) * sizeof(int32_t), st));   // empty entries: -1
    NA_CK(cudaMemsetAsync(done, 0, static_cast<size_t>(nb) * sizeof(int32_t), st));
    NA_CK(cudaMemcpyAsync(ctrl, &H, sizeof(H), cudaMemcpyHostToDevice, st));
    if (nfix > 0) {
        NA_CK(cudaMemcpyAsync(d_fb, fb, nfix * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        NA_CK(cudaMemcpyAsync(d_fp, fp, nfix * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        NA_CK(cudaMemcpyAsync(d_fv, fv, nfix * sizeof(double), cudaMemcpyHostToDevice, st));
        NA_CK(cudaMemcpyAsync(d_sb, sb, nsb * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        NA_CK(cudaMemcpyAsync(d_enq, enq, nenq * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        NA_CK(eikg::launch_init_sources<float>(nfix, d_fb, d_fp, d_fv, nsb, d_sb, nenq, d_enq, 0, nullptr, slot, ups,
                                               stampv, queued + nb, nullptr, rr, d_saved, lists + nb, nullptr, st));
    }
    if (nenq > 0) {
        int per_sm = 0, sms = 0, dev = 0;
        NA_CK(cudaGetDevice(&dev));
        NA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        NA_CK(eikg::loop_occupancy<float>(&per_sm));
        eikg::LoopParams<float> L{};
        L.nx = nx;
        L.ny = ny;
        L.nz = nz;
        L.BX = BX;
        L.BY = BY;
        L.BZ = BZ;
        L.nbricks = nb;
        L.slot = slot;
        L.ups = ups;
        L.stamp = stampv;
        L.queued = queued;
        L.rr = rr;
        L.done = done;
        for (int r = 0; r < eikg::kRing; ++r) L.list[r] = lists + r * nb;
        L.early = 1;
        L.groups = 0;                 // 8^3 blocks only: no group work lists
        L.mode_fixed = 8;
        L.ctrl = ctrl;
        L.log = nullptr;
        L.log_cap = 0;
        L.window = P.window;
        L.window_f = static_cast<float>(P.window);
        L.width = P.width;
        L.fallback_tau = P.fallback_tau;
        L.max_restarts = P.max_restarts;
        L.wait_limit = P.wait_polls > 0 ? P.wait_polls : eikg::kWaitPolls;
        L.sched = EIK_SCHED_FIXED;
        L.mlp = nullptr;
        L.h = h;
        L.nmax = std::max(nx, std::max(ny, nz));
        L.seed = 0;
        if (P.loop_events[0]) NA_CK(cudaEventRecord(static_cast<cudaEvent_t>(P.loop_events[0]), st));
        NA_CK(eikg::launch_restart_loop<float>(L, per_sm * sms, st));
        if (P.loop_events[1]) NA_CK(cudaEventRecord(static_cast<cudaEvent_t>(P.loop_events[1]), st));
    }
    if (nfix > 0) NA_CK(eikg::launch_restore_r<float>(nfix, d_fb, d_fp, d_saved, rr, st));
    NA_CK(eikg::launch_result<float>(slot, stampv, psi_out, nx, ny, 0, nz, BX, BY, st));
    NA_CK(cudaMemcpyAsync(&H, ctrl, sizeof(H), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    eik_status out = EIK_OK;
    if (H.status) out = fail(EIK_ETIMEOUT, "eik_solve_noalloc: solve stopped early (restart cap or wait limit)");
    else if (!H.done) out = fail(EIK_ECUDA, "eik_solve_noalloc: solve did not finish");
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->restarts = H.k;
        stats->marches = static_cast<int64_t>(H.marches);
        stats->accepted = static_cast<int64_t>(H.accepted);
        stats->solves = static_cast<int64_t>(H.solves);
        stats->updates = static_cast<int64_t>(H.updates);
        stats->fallbacks = static_cast<int64_t>(H.fallbacks);
        stats->rounds = static_cast<int64_t>(H.rounds);
        stats->device_ms = (H.t_end > H.t_begin) ? static_cast<double>(H.t_end - H.t_begin) * 1e-6 : 0.0;
        stats->final_bound = H.bound;
        stats->status = out;
        stats->block_dim = 8;
    }
    return out;
}

}  // extern "C"
