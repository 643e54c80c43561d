// eik_solve_noalloc: one solve that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code running under a caching allocator
// or a memory pool they do not own, code inside a CUDA stream capture, and
// embedders that must not grow the process's device footprint at solve time.
// For them this entry point keeps every piece of working memory of a solve
// (h/F in brick layout, the two psi copies of each brick, the Upsilon masks,
// stamps, work lists, control block and the fixed-node tables) in one
// file-scope device array of fixed size.  The caller passes the speeds and the
// output buffer, both in device memory.
//
// The array is part of the library image: every GPU that loads libeik holds
// it until the process exits.  Its device address is looked up once per
// device, on the first call made with that device current; make that first
// call before any stream capture.  All calls share the array and it keeps the
// last call's contents, so calls that overlap on the GPU (two host threads,
// or asynchronous work on two streams) race; each call clears what must start
// from zero (stamps, work-list state, control block) itself.
#include "eik.h"
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

int cell_nodes(double s, double h, int n, int out[2]) {
    const double t = s / h;
    const double tn = std::floor(t + 0.5);
    if (std::fabs(t - tn) <= 1e-9) {
        out[0] = std::min(std::max(static_cast<int>(tn), 0), n - 1);
        return 1;
    }
    const int i0 = std::min(std::max(static_cast<int>(std::floor(t)), 0), std::max(n - 2, 0));
    out[0] = i0;
    out[1] = std::min(i0 + 1, n - 1);
    return (out[1] == out[0]) ? 1 : 2;
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
    if (!(P.stride > 0.0)) return fail(EIK_EINVAL, "eik_solve_noalloc: stride must be > 0");
    if (P.block_dim != 0 && P.block_dim != 8) return fail(EIK_ENOTSUP, "eik_solve_noalloc: block_dim must be 8");
    if (P.schedule != EIK_SCHED_FIXED) return fail(EIK_ENOTSUP, "eik_solve_noalloc: fixed-stride schedule only");
    if (P.window == 0.0) P.window = 2.0;
    if (!(P.window > 0.0) || !std::isfinite(P.window)) return fail(EIK_EINVAL, "eik_solve_noalloc: bad window");
    if (P.width == 0.0) P.width = INFINITY;
    if (!(P.width > 0.0)) return fail(EIK_EINVAL, "eik_solve_noalloc: width must be >= 0 (0 = +inf)");
    if (P.max_restarts <= 0) P.max_restarts = int64_t(1) << 24;
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
    // fixed nodes: the nodes of each source's cell, psi0 = distance / F
    double cd[kMaxFix];
    int32_t cb[kMaxFix], cp[kMaxFix];
    int nc = 0;
    for (int q = 0; q < nsrc; ++q) {
        const double* xs = xyz + 3 * q;
        int cx[2], cy[2], cz[2];
        const int mx = cell_nodes(xs[0], h, nx, cx), my = cell_nodes(xs[1], h, ny, cy), mz = cell_nodes(xs[2], h, nz, cz);
        for (int a = 0; a < mz; ++a)
            for (int b2 = 0; b2 < my; ++b2)
                for (int d = 0; d < mx; ++d) {
                    const int i = cx[d], j = cy[b2], k = cz[a];
                    const double dx = i * h - xs[0], dy = j * h - xs[1], dz = k * h - xs[2];
                    cd[nc] = std::sqrt(dx * dx + dy * dy + dz * dz);
                    cb[nc] = ((k >> 3) * BY + (j >> 3)) * BX + (i >> 3);
                    cp[nc] = ((k & 7) * 8 + (j & 7)) * 8 + (i & 7);
                    ++nc;
                }
    }
    double cr[kMaxFix];
    NA_CK(cudaMemcpyAsync(d_fb, cb, nc * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(d_fp, cp, nc * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    NA_CK(eikg::launch_gather_r<float>(nc, d_fb, d_fp, rr, d_cr, st));
    NA_CK(cudaMemcpyAsync(cr, d_cr, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if (bad) return fail(EIK_EINVAL, "eik_solve_noalloc: F must be finite and >= 0 everywhere");
    // keep the smallest psi0 per node
    int32_t fb[kMaxFix], fp[kMaxFix];
    double fv[kMaxFix];
    int nfix = 0;
    for (int t = 0; t < nc; ++t) {
        double v;
        if (cd[t] == 0.0) v = 0.0;
        else if (std::isfinite(cr[t]) && cr[t] > 0.0) v = cd[t] * cr[t] / h;
        else continue;
        int at = -1;
        for (int u = 0; u < nfix; ++u)
            if (fb[u] == cb[t] && fp[u] == cp[t]) at = u;
        if (at < 0) {
            fb[nfix] = cb[t];
            fp[nfix] = cp[t];
            fv[nfix] = v;
            ++nfix;
        } else if (v < fv[at]) {
            fv[at] = v;
        }
    }
    // bricks with fixed nodes, and the work list of restart 1
    int32_t sb[kMaxFix], enq[7 * kMaxFix];
    int nsb = 0, nenq = 0;
    auto add_unique = [](int32_t* a, int& n, int32_t v) {
        for (int i = 0; i < n; ++i)
            if (a[i] == v) return;
        a[n++] = v;
    };
    for (int t = 0; t < nfix; ++t) {
        const int32_t b = fb[t];
        add_unique(sb, nsb, b);
        add_unique(enq, nenq, b);
        const int x = fp[t] & 7, y = (fp[t] >> 3) & 7, z = fp[t] >> 6;
        const int bx = b % BX, by = (b / BX) % BY, bz = b / (BX * BY);
        if (x == 0 && bx > 0) add_unique(enq, nenq, b - 1);
        if (x == 7 && bx < BX - 1) add_unique(enq, nenq, b + 1);
        if (y == 0 && by > 0) add_unique(enq, nenq, b - BX);
        if (y == 7 && by < BY - 1) add_unique(enq, nenq, b + BX);
        if (z == 0 && bz > 0) add_unique(enq, nenq, b - BX * BY);
        if (z == 7 && bz < BZ - 1) add_unique(enq, nenq, b + BX * BY);
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
        L.wait_limit = eikg::kWaitPolls;
        L.sched = EIK_SCHED_FIXED;
        L.mlp = nullptr;
        L.h = h;
        L.nmax = std::max(nx, std::max(ny, nz));
        L.seed = 0;
        NA_CK(eikg::launch_restart_loop<float>(L, per_sm * sms, st));
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
