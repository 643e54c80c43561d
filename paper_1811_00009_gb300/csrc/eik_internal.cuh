// Internal definitions of libeik (not part of the C ABI).
//
// Data layout in HBM (one grid; a batch of grids concatenates the bricks
// of its grids, see SolveDesc):
//   bricks of 8x8x8 nodes, brick b = (bz*BY + by)*BX + bx, node p = (z*8 + y)*8 + x
//   inside a brick; a ragged last brick per axis is padded with barrier nodes.
//   rr[b][512]          h/F (+inf: barrier or padding, -1: fixed source node)
//   slot[b][2][640]     two copies of the brick's psi: 512 interior values,
//                       then its x = 0 and x = 7 faces (64 each, index z*8+y)
//                       stored contiguously for the neighbours' ghost reads
//   ups[b][2][6]        per copy, the 64-bit mask of face nodes lowered in the
//                       march that wrote it (Upsilon of Alg. 2/4), per face
//   stamp[b]            64 bits: restart that wrote the latest copy (high 32),
//                       restart that wrote the other copy (bits 31..1, all ones
//                       if never), index of the latest copy (bit 0); all ones
//                       for a brick no march has touched
//   queued[s][b]        restart whose work list (ring slot s = restart mod kRing)
//                       holds the brick; qgroup[s][g] the same for the group g
//                       of 2x2x2 bricks (16^3 blocks)
//   done[b]             last restart whose march of the brick has finished
// A march at restart k reads the brick's latest copy and its neighbours' copies
// as of the end of restart k-1, and writes the other copy, so no warp ever
// reads memory written during the same restart: the exchange step of Alg. 5
// needs no second grid-wide barrier.  With a fixed stride a warp waiting at
// the barrier of restart k may march a brick of restart k+1 early, once the
// brick and its six neighbours have finished their restart-k marches (done[]):
// it then reads exactly what it would read after the barrier.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace eikg {

constexpr int kEdge = 8;           // brick edge (nodes)
constexpr int kBrick = 512;        // nodes per brick
constexpr int kSlot = 640;         // values per brick copy
constexpr int kXF0 = 512;          // offset of the x = 0 face inside a copy
constexpr int kXF7 = 576;          // offset of the x = 7 face
constexpr int kWarps = 8;          // warps per CTA of the restart loop (one brick per warp)
constexpr long long kWaitPolls = 1ll << 22;   // polls (naps of 32 ns to 4 us) before a wait gives up: seconds
constexpr int kRing = 4;           // work lists in flight: restart k's, k+1's, k+2's (early k+1 marches), k-1's (being cleared)

constexpr unsigned long long kUntouched = ~0ull;   // stamp of a brick no march has written
constexpr unsigned kNever = 0x7fffffffu;           // "other copy never written"

__host__ __device__ inline int stamp_latest(unsigned long long w) { return static_cast<int>(w >> 32); }
__host__ __device__ inline int stamp_other(unsigned long long w) { return static_cast<int>((w >> 1) & kNever); }
__host__ __device__ inline int stamp_copy(unsigned long long w) { return static_cast<int>(w & 1ull); }
__host__ __device__ inline unsigned long long make_stamp(int latest, int other, int copy) {
    return (static_cast<unsigned long long>(static_cast<unsigned>(latest)) << 32) |
           (static_cast<unsigned long long>(static_cast<unsigned>(other) & kNever) << 1) |
           static_cast<unsigned long long>(copy & 1);
}

// status bits of a device run
constexpr int kStWaitTimeout = 1;  // a grid-barrier wait ran out of iterations
constexpr int kStRestartCap = 2;   // max_restarts reached with work left
constexpr int kStRoundCap = 4;     // a march exceeded its round cap

// Control block of one restart loop, in device memory.  Written by the CTA
// that arrives last at each grid barrier, read by all after the release.
struct Ctrl {
    unsigned int bar_count;
    unsigned int bar_gen;
    int32_t pad_bar[30];       // the barrier words in a cache line of their own (polled by waiting warps)
    int32_t k;                 // current restart (1-based)
    int32_t done;
    int32_t status;
    int32_t pad_k[29];
    int32_t count[kRing];      // brick work-list lengths, by ring slot (restart mod kRing)
    int32_t pad_count[28];     // (lengths grow by atomics during a restart; heads are claimed apart)
    int32_t head[kRing];       // next brick work-list entry to hand out
    int32_t pad_head[28];
    int32_t used[kRing];       // length a ring slot's list had when its restart ended (cleared to -1 next restart)
    int32_t gcount[kRing];     // group (16^3 block) work-list lengths, by ring slot
    int32_t ghead[kRing];      // next group work-list entry to hand out
    int32_t mode;              // block edge of restart k: 8 (one warp per brick) or 16 (one CTA per group)
    int32_t action;            // schedule action of restart k (-1: the initial stride and block edge)
    int32_t pend_action;       // action already chosen for restart k+1 (-1: keep restart k's stride and block edge)
    double bound;              // bound_band of restart k
    double bound_prev;         // bound_band of restart k-1 (-1 at k = 1)
    double stride;             // stride that produced `bound`
    unsigned long long t_begin;
    unsigned long long t_restart;
    unsigned long long t_end;
    // accumulators of the current restart
    unsigned long long r_accepted, r_band, r_solves, r_updates, r_fallbacks, r_rounds;
    unsigned int r_rmin_bits, r_rmax_bits;
    // totals
    unsigned long long marches, accepted, solves, updates, fallbacks, rounds;
};

struct RestartRec {            // mirrors eik_restart_rec
    int32_t k;
    int32_t active;
    int64_t band;
    int64_t accepted;
    int64_t solves;
    double bound;
    double stride;
    double rmin;
    double rmax;
    double ms;
    int32_t block_dim;
    int32_t next_action;
    float features[10];
};

// A brick's face as a neighbouring GPU exports it (a grid sharded in z): the 64
// values of the face layer of the brick's latest copy, the Upsilon mask of
// that copy on that face, and the restart that wrote it (-1: untouched).
template <typename T>
struct FaceRec {
    T v[64];
    unsigned long long ups;
    int32_t written;
    int32_t pad;
};

// One grid of a batched launch: its place in the launch's brick and group
// index spaces, its block edge and its stride (bound of restart k = k*stride).
struct SolveDesc {
    int32_t BX, BY, BZ;
    int32_t boff;              // global index of the grid's first brick
    int32_t GX, GY, GZ;
    int32_t goff;              // global index of the grid's first 2x2x2 group
    int32_t mode;              // block edge: 8 (one warp per brick) or 16 (one CTA per group)
    int32_t pad;
    double stride;
};

template <typename T>
struct LoopParams {
    int32_t nx, ny, nz;
    int32_t BX, BY, BZ;
    int64_t nbricks;
    int64_t ngroups;
    T* slot;
    unsigned long long* ups;
    unsigned long long* stamp;
    int32_t* queued;           // kRing x nbricks: queued[s * nbricks + b] = restart of ring slot s holding b
    int32_t* done;             // per brick: last restart whose march of it finished
    const T* rr;
    int32_t* list[kRing];      // brick work lists by ring slot; unused entries are -1
    int32_t GX, GY, GZ;        // groups of 2x2x2 bricks per axis
    int32_t groups;            // non-zero: keep the group work lists (16^3 restarts possible)
    int32_t* qgroup;           // kRing x ngroups, as queued
    int32_t* glist[kRing];     // group work lists by ring slot
    int32_t early;             // non-zero: waiting warps may march the next restart's bricks early
    int32_t own_bz0, own_bz1;  // brick planes (z) this launch owns: bricks outside are ghosts of a grid
                               // sharded across GPUs (their faces are imported; never put on a work list)
    int32_t pause;             // non-zero: stop after every restart (the sharded solve exchanges faces)
    double width;              // width_band of Alg. 6 (+inf: the full solve)
    Ctrl* ctrl;
    RestartRec* log;
    int64_t log_cap;
    double window;             // omega: acceptance window = omega * min(h/F) over the brick
    float window_f;            // omega in single precision (FP32 marches compute the window in float)
    double fallback_tau;       // FP32: double-precision root when D < tau * k * r^2
    int64_t max_restarts;
    long long wait_limit;      // polls before a wait (barrier, list entry, neighbour march) gives up
    int32_t sched;             // 0 fixed, 1 learned, 2 seeded random (exploration data)
    int32_t mode_fixed;        // block edge of every restart under the fixed schedule (8 or 16)
    const float* mlp;          // schedule network weights (learned schedule)
    double h;
    int32_t nmax;              // longest grid axis (feature scale)
    uint32_t seed;             // random schedule seed
    float margin;              // learned schedule: switch action only if predicted cheaper by this much (log)
    // batched launch only (eik_batch.cu)
    const SolveDesc* solves;   // per grid
    const int32_t* bsolve;     // per brick: its grid
    const int32_t* gsolve;     // per group: its grid
    int32_t* last_k;           // per grid: last restart in which one of its blocks marched
    unsigned long long* tend;  // per restart: %globaltimer at its end
    int64_t tend_cap;
    T* gbound;                 // kRing x nsolves: bound of restart j of grid s at [j % kRing][s], rounded
                               // down to T (-1 for j = 0); restart k's end writes j = k + 2
    int32_t nsolves;
};

}  // namespace eikg
