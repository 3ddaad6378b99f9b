// Host-side helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <functional>
#include <vector>

#include "tabsimplex.h"

namespace tsx {

// Records the thread's last error message (read by lp_last_error).
void set_error(const char* fmt, ...);

// The device allocator installed with lp_set_allocator (both null: default);
// null on threads that asked for the default with use_default_allocator.
void current_allocator(lp_alloc_fn* alloc_fn, lp_free_fn* free_fn, void** ctx);

// Handles created on the calling thread ignore lp_set_allocator's hook and use
// cudaMallocAsync / cudaFreeAsync (the request server's worker threads).
void use_default_allocator(bool on);

// Stream-ordered device allocation of the default allocator: a memory pool
// per device, owned by the library, that keeps freed memory for reuse (the
// device's default pool hands freed memory back at every synchronisation, and
// mapping it again made each new handle of a busy server cost ~0.5 ms).
cudaError_t pool_alloc(void** ptr, size_t bytes, cudaStream_t stream);

// Events and non-blocking streams of the current device, recycled through
// per-device free lists instead of created and destroyed per handle: with
// eight server threads calling the runtime, cudaEventCreate took ~30 us and
// cudaEventDestroy ~58 us a call (0.2 us on one thread).  A stream must be
// idle when it is put back; a recycled event is recorded before it is used.
cudaEvent_t event_get(bool timing);
void event_put(cudaEvent_t e, bool timing);
cudaStream_t stream_get();
void stream_put(cudaStream_t s);

// Device alias of a page-locked host array of `count` doubles (cudaHostAlloc,
// cudaHostRegister, torch's pinned tensors) that the current device may read
// directly; null for pageable memory or memory not mapped for it.
const double* host_alias(const double* p, size_t count);

struct DevState;
// Uploads A (mn), b (m) and c (n) from their device aliases (host_alias) with
// one kernel on stream s, reading over the host link; with st != null it also
// checks them (entries finite, b >= 0) and sets st->bad on a violation.
cudaError_t launch_ingest(const double* sA, double* dA, size_t mn, const double* sb, double* db, size_t m,
                          const double* sc, double* dc, size_t n, DevState* st, cudaStream_t s);

// Shared-memory bytes the batched solver has for one LP on the current device,
// and whether an m x n LP fits in them.
size_t batch_smem_limit();
bool batch_fits(int m, int n, size_t limit);

// lp_create_device without the input check: the check (finite data, b >= 0)
// runs during the first solve instead -- in the team kernel's build for
// lp_solve_many, or as lp_create's own check before any other solve.  For
// callers that create many handles at once (the server's waves).
lp_t create_device_unchecked(int m, int n, const double* dA, const double* db, const double* dc,
                             cudaStream_t stream);

// lp_solve_many for callers that overlap its parts: the team launch leaves
// `reserve_blocks` of the co-resident blocks free for other work, and
// `after_kernel` (may be empty) runs on the calling thread as soon as the
// launch has completed, before the per-LP bookkeeping and FP64 recovery.
lp_status solve_many_hooked(lp_t* handles, int count, const lp_options* opt, lp_status* status,
                            int reserve_blocks, const std::function<void()>& after_kernel);

// Continuous team launch for the request server (k_team_serve): LPs are
// added while the launch runs, each solved by the next free team, and each
// reports its end on its own.
struct TeamLane;
// Opens a lane with the given options (precision, tolerances, blocks = narrow
// team size); the launch leaves `reserve_blocks` co-resident blocks free.
// NULL on error.
TeamLane* lane_open(const lp_options* opt, int reserve_blocks);
// Adds an LP (a handle from lp_create or create_device_unchecked, not solved
// concurrently elsewhere) and starts a launch if none runs.  Returns a token
// >= 0; -2 if the LP does not fit a team's shared memory (solve it another
// way); -1 on error.
long long lane_submit(TeamLane* lane, lp_t h);
// Appends the handles whose team has finished (or, after a launch ended, whose
// team gave up) to `done`; starts a new launch when jobs wait and none runs.
// Returns the number of LPs still in the lane; waits on the device only to
// read the claim counters after a launch has ended.
int lane_poll(TeamLane* lane, std::vector<lp_t>& done);
// Statistics and, for FP32, the FP64 recovery of a finished LP on stream s
// (as lp_solve_many); *status receives its outcome.
lp_status lane_finish(TeamLane* lane, lp_t h, cudaStream_t s, lp_status* status);
long long lane_launches(TeamLane* lane);
// Stops the launch (teams leave once idle) and frees the lane.
void lane_close(TeamLane* lane);

}  // namespace tsx

#define TSX_CUDA_TRY(call, ret)                                                           \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            tsx::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                           __LINE__);                                                     \
            return ret;                                                                   \
        }                                                                                 \
    } while (0)
