// Host-side helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <functional>

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

// Shared-memory bytes the batched solver has for one LP on the current device,
// and whether an m x n LP fits in them.
size_t batch_smem_limit();
bool batch_fits(int m, int n, size_t limit);

// lp_solve_many for callers that overlap its parts: the team launch leaves
// `reserve_blocks` of the co-resident blocks free for other work, and
// `after_kernel` (may be empty) runs on the calling thread as soon as the
// launch has completed, before the per-LP bookkeeping and FP64 recovery.
lp_status solve_many_hooked(lp_t* handles, int count, const lp_options* opt, lp_status* status,
                            int reserve_blocks, const std::function<void()>& after_kernel);

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
