// Shared helpers of the gbqr CUDA library: handle, workspace arena, status
// handling, device-wide scans and reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <new>

#include "gbqr.h"

struct gb_handle {
    cudaStream_t stream;
    void* ws;
    size_t ws_bytes;
    size_t required_ws;
    int device;
    int64_t launches;  // kernels launched by the current call
    cudaEvent_t ev0, ev1;  // recursion-kernel timing (created on first use)
};

#define GB_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return GB_ERR_DEVICE;    \
    } while (0)

#define GB_TRY(call)                   \
    do {                               \
        int s_ = (call);               \
        if (s_ != GB_OK) return s_;    \
    } while (0)

// Launch bookkeeping: every kernel launch goes through GB_LAUNCH so the
// report can state how many kernels a call issued.
#define GB_LAUNCH(h, kernel, grid, block, smem, ...)                                  \
    do {                                                                              \
        kernel<<<(grid), (block), (smem), (h)->stream>>>(__VA_ARGS__);                \
        (h)->launches++;                                                              \
        cudaError_t e_ = cudaGetLastError();                                          \
        if (e_ != cudaSuccess) return GB_ERR_DEVICE;                                  \
    } while (0)

// Bump allocator over the caller's workspace.  With base == nullptr it only
// measures (used to answer the *_workspace_size queries with the same code
// that lays the workspace out).
struct Arena {
    char* base;
    size_t cap;
    size_t off;
    explicit Arena(void* b = nullptr, size_t c = 0) : base((char*)b), cap(c), off(0) {}
    template <typename T>
    T* take(size_t count) {
        size_t bytes = count * sizeof(T);
        off = (off + 255) & ~(size_t)255;
        T* p = base ? (T*)(base + off) : nullptr;
        off += bytes;
        return p;
    }
    bool fits() const { return base == nullptr || off <= cap; }
    size_t used() const { return (off + 255) & ~(size_t)255; }
};

static inline int ceil_div_i64(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Exclusive prefix sum of n int64 values (in may alias out).  Temporary
// storage: scan_temp_count(n) int64 elements.  Deterministic.
size_t scan_temp_count(int64_t n);
int exclusive_scan_i64(gb_handle* h, const int64_t* in, int64_t* out, int64_t n, int64_t* temp);

// Copy one int64 / double from device to host (synchronises the stream).
int read_i64(gb_handle* h, const int64_t* d, int64_t* out, int count = 1);
int read_f64(gb_handle* h, const double* d, double* out, int count = 1);
int read_i32(gb_handle* h, const int32_t* d, int32_t* out, int count = 1);

// Device error word shared by the kernels of one call: the first non-zero
// status written wins.
__device__ __forceinline__ void set_error(int* flag, int status) {
    atomicCAS(flag, 0, status);
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
