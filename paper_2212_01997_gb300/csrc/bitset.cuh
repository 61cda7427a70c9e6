// Block-wide sorted compaction of a shared-memory bitmap.  Used by the graph
// builder and the partitioner: neighbour sets are marked in a bitmap of n bits
// (order-independent atomicOr), then read back in ascending vertex order, so
// the output never depends on thread scheduling.
#pragma once

#include <stdint.h>

// Returns the number of set bits among words[0..W) to every thread.  When
// `out` is non-null, writes base + the indices of the set bits in ascending
// order to out[0..count) (base: the vertex of bit 0 of a windowed bitmap).  `scan` is shared scratch of blockDim.x int64 values (one
// per warp is used).  Thread t owns a contiguous run of words; the per-thread
// counts are scanned within each warp by shuffles and across warps through
// `scan`: two barriers per call.  blockDim.x must be a multiple of 32.
__device__ inline int64_t bitmap_compact(const uint32_t* words, int W, int32_t* out, int64_t* scan,
                                        int32_t base = 0) {
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
    int64_t before = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
        const int64_t v = scan[w];
        before += w < wid ? v : 0;
        total += v;
    }
    if (out) {
        int64_t pos = before + incl - local;
        for (int w = w0; w < w1; ++w) {
            uint32_t bits = words[w];
            while (bits) {
                int b = __ffs(bits) - 1;
                bits &= bits - 1;
                out[pos++] = base + w * 32 + b;
            }
        }
    }
    __syncthreads();
    return total;
}

// The 32-aligned window [base, base + 32 W) holding every thread's values in
// [lo, hi] (hi < 0: the thread has none; W = 0 when no thread has any).
// `red` is shared scratch of 2 x (blockDim.x / 32) ints; the caller's next
// barrier (e.g. bitmap_clear's) must come before `red` is written again.
__device__ inline void bitmap_window(int32_t lo, int32_t hi, int32_t* red, int32_t& base, int& W) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
        red[warp] = lo;
        red[nw + warp] = hi;
    }
    __syncthreads();
    for (int w = 0; w < nw; ++w) {
        lo = min(lo, red[w]);
        hi = max(hi, red[nw + w]);
    }
    base = hi < 0 ? 0 : (lo & ~31);
    W = hi < 0 ? 0 : ((hi - base) >> 5) + 1;
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
