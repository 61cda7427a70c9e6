// Warp-wide sort of small integer sets in registers, for the graph builder
// and the partitioner: a row or a subgraph whose (repeated) members fit in
// 32 x EPL values is sorted by one warp and its distinct values read back in
// ascending order (deterministic, independent of scheduling).
#pragma once

#include <stdint.h>

// Sorts the warp's 32 x EPL values ascending in place by a bitonic network.
// Lane-major: lane l holds elements l EPL .. l EPL + EPL - 1 of the sequence.
// Compare-exchanges between elements less than EPL apart stay in a lane's
// registers; farther ones pair lanes by shuffles.  EPL is a power of two; the
// loops unroll fully, so the array stays in registers.
template <int EPL>
__device__ __forceinline__ void warp_bitonic_sort(int32_t (&v)[EPL]) {
    constexpr int N = 32 * EPL;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= EPL) {
                const int lx = stride / EPL;
#pragma unroll
                for (int k = 0; k < EPL; ++k) {
                    const int e = lane * EPL + k;
                    const int32_t o = __shfl_xor_sync(0xffffffffu, v[k], lx);
                    const bool up = (e & size) == 0, low = (e & stride) == 0;
                    v[k] = (low == up) ? min(v[k], o) : max(v[k], o);
                }
            } else {
#pragma unroll
                for (int k = 0; k < EPL; ++k) {
                    if (k & stride) continue;
                    const int k2 = k | stride;
                    const bool up = ((lane * EPL + k) & size) == 0;
                    const int32_t x = v[k], y = v[k2];
                    v[k] = up ? min(x, y) : max(x, y);
                    v[k2] = up ? max(x, y) : min(x, y);
                }
            }
        }
    }
}

// After warp_bitonic_sort: bit k set where v[k] starts a run of equal values
// (the padding INT32_MAX never counts).  EPL <= 32.
template <int EPL>
__device__ __forceinline__ uint32_t warp_run_starts(const int32_t (&v)[EPL]) {
    const int lane = threadIdx.x & 31;
    const int32_t prev_last = __shfl_up_sync(0xffffffffu, v[EPL - 1], 1);
    uint32_t keep = 0;
#pragma unroll
    for (int k = 0; k < EPL; ++k) {
        const int32_t p = k > 0 ? v[k - 1] : (lane > 0 ? prev_last : INT32_MIN);
        if (v[k] != INT32_MAX && v[k] != p) keep |= 1u << k;
    }
    return keep;
}

// Exclusive prefix sum of x over the warp's lanes; *total gets the sum.
__device__ __forceinline__ int warp_exclusive_scan(int x, int* total) {
    const int lane = threadIdx.x & 31;
    int incl = x;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    *total = __shfl_sync(0xffffffffu, incl, 31);
    return incl - x;
}
