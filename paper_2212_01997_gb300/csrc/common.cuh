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
    cudaStream_t aux;      // second stream for a size class run beside the others
    cudaEvent_t ev_fork, ev_join;  // (created on first use, no timing)
    int plan_valid;        // gb_plan_autotune's cache: key (n_sub, sub_nnz, m, precision)
    int64_t plan_key[4];
    gb_plan plan;
};

// the CUDA error behind the last GB_ERR_DEVICE (gb_last_device_error)
void gb_note_device_error(cudaError_t e);

#define GB_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) {                        \
            gb_note_device_error(e_);                   \
            return GB_ERR_DEVICE;                       \
        }                                               \
    } while (0)

#define GB_TRY(call)                   \
    do {                               \
        int s_ = (call);               \
        if (s_ != GB_OK) return s_;    \
    } while (0)

// Launch bookkeeping: every kernel launch goes through GB_LAUNCH so the
// report can state how many kernels a call issued.
#define GB_LAUNCH(h, kernel, grid, block, smem, ...)                                  \
    GB_LAUNCH_ON(h, (h)->stream, kernel, grid, block, smem, __VA_ARGS__)
#define GB_LAUNCH_ON(h, st, kernel, grid, block, smem, ...)                           \
    do {                                                                              \
        kernel<<<(grid), (block), (smem), (st)>>>(__VA_ARGS__);                       \
        (h)->launches++;                                                              \
        cudaError_t e_ = cudaGetLastError();                                          \
        if (e_ != cudaSuccess) {                                                      \
            gb_note_device_error(e_);                                                 \
            return GB_ERR_DEVICE;                                                     \
        }                                                                             \
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

// double -> float, round to nearest even, by integer operations (finite
// values; magnitudes below the smallest normal float flush to zero).  Keeps
// per-element work off GB300's narrow FP64 pipe.
__device__ __forceinline__ float d2f_rn(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
    const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // top 23 of 52 mantissa bits
    const uint32_t rem = lo & 0x1fffffffu;                    // the 29 dropped bits
    uint32_t f = ((uint32_t)e << 23) + m;                     // a carry moves into the exponent
    if (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) f += 1u;
    return __uint_as_float(sign | f);
}

__device__ __forceinline__ float warp_sum_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

