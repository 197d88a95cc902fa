// Internal helpers shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "twgrid.h"

namespace tw {

// last CUDA error seen by any entry point (read by tw_last_cuda_error)
void set_cuda_error(cudaError_t e);
// host-side count of kernel launches (read by tw_launch_count)
void count_launches(unsigned long long n);
// while paused (per host thread, nestable), launches are not counted: stream
// capture records kernels that run later, when their graph is launched
void pause_launch_count(bool on);

#define TW_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) {                        \
            ::tw::set_cuda_error(e_);                   \
            return TW_ECUDA;                            \
        }                                               \
    } while (0)

#define TW_CHECK_LAUNCH() TW_CUDA(cudaGetLastError())
// every kernel launch goes through this macro so that launches are counted
#define TW_LAUNCH(kernel, grid, block, smem, stream, ...)                 \
    do {                                                                  \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);       \
        ::tw::count_launches(1);                                          \
    } while (0)

// Bump allocator over a caller-provided workspace.  Every carve is 256-byte
// aligned; `need` accumulates the bytes a layout requires so that the same
// code computes both the size query and the carving.
struct Carver {
    char *base;
    size_t cap;
    size_t need;
    explicit Carver(void *b = nullptr, size_t c = 0) : base((char *)b), cap(c), need(0) {}
    template <class T>
    T *take(size_t count) {
        size_t off = (need + 255) & ~(size_t)255;
        need = off + count * sizeof(T);
        if (!base || need > cap) return nullptr;
        return (T *)(base + off);
    }
    bool ok() const { return base && need <= cap; }
};

inline bool ws_aligned(const void *p) { return ((uintptr_t)p & 255u) == 0; }

inline unsigned ceil_div(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

}  // namespace tw
