// Block-wide sorted compaction of a shared-memory bitmap.  Used by the graph
// builder and the partitioner: neighbour sets are marked in a bitmap of n bits
// (order-independent atomicOr), then read back in ascending vertex order, so
// the output never depends on thread scheduling.
#pragma once

#include <stdint.h>

// Returns the number of set bits among words[0..W) to every thread.  When
// `out` is non-null, writes the indices of the set bits in ascending order to
// out[0..count).  `scan` is shared scratch of blockDim.x int64 values (one
// per warp is used).  Thread t owns a contiguous run of words; the per-thread
// counts are scanned within each warp by shuffles and across warps through
// `scan`: two barriers per call.  blockDim.x must be a multiple of 32.
__device__ inline int64_t bitmap_compact(const uint32_t* words, int W, int32_t* out, int64_t* scan) {
    const int t = threadIdx.x;
    const int nt = blockDim.x;
    const int lane = t & 31, wid = t >> 5, nw = nt >> 5;
    const int chunk = (W + nt - 1) / nt;
    const int w0 = min(W, t * chunk);
    const int w1 = min(W, w0 + chunk);
    int local = 0;
    for (int w = w0; w < w1; ++w) local += __popc(words[w]);
    int incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) scan[wid] = incl;
    __syncthreads();
    int64_t base = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
        const int64_t v = scan[w];
        base += w < wid ? v : 0;
        total += v;
    }
    if (out) {
        int64_t pos = base + incl - local;
        for (int w = w0; w < w1; ++w) {
            uint32_t bits = words[w];
            while (bits) {
                int b = __ffs(bits) - 1;
                bits &= bits - 1;
                out[pos++] = w * 32 + b;
            }
        }
    }
    __syncthreads();
    return total;
}

__device__ inline void bitmap_clear(uint32_t* words, int W) {
    for (int w = threadIdx.x; w < W; w += blockDim.x) words[w] = 0u;
    __syncthreads();
}

__device__ inline void bitmap_set(uint32_t* words, int v) {
    atomicOr(&words[v >> 5], 1u << (v & 31));
}

__device__ inline void bitmap_unset(uint32_t* words, int v) {
    atomicAnd(&words[v >> 5], ~(1u << (v & 31)));
}
