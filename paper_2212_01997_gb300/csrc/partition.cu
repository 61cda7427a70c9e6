// gb_partition: disjoint cores and distance-1 halos.
//
// Fig. 1 / Sec. "Choosing the graph partitioning": a subgraph is its core plus
// the halo of directly connected vertices; cores may hold several vertices
// (here: one core per group id, e.g. one molecule, or consecutive blocks).
// S_i = sorted(core_i U N(core_i)).  Membership is marked in shared-memory
// bitmaps and read back in ascending order, so the output is bit-exact.
#include "bitset.cuh"
#include "common.cuh"

namespace {

constexpr int SUB_THREADS = 256;

__device__ __forceinline__ int32_t group_of(int32_t v, const int32_t* group, int32_t block) {
    return group ? group[v] : v / block;
}

__global__ void k_group_count(int32_t n, const int32_t* group, int32_t block, int32_t n_groups,
                              int64_t* gcnt, int* err) {
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t g = group_of(v, group, block);
    if (g < 0 || g >= n_groups) {
        set_error(err, GB_ERR_ARG);
        return;
    }
    atomicAdd((unsigned long long*)&gcnt[g], 1ull);
}

__global__ void k_nonempty(int32_t n_groups, const int64_t* gcnt, int64_t* flag) {
    int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n_groups) flag[g] = gcnt[g] > 0 ? 1 : 0;
}

// cidx[g] = exclusive scan of the non-empty flags; core_size[cidx[g]] = gcnt[g]
__global__ void k_core_sizes(int32_t n_groups, const int64_t* gcnt, const int64_t* cidx,
                             int64_t* core_size) {
    int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n_groups && gcnt[g] > 0) core_size[cidx[g]] = gcnt[g];
}

__global__ void k_core_fill(int32_t n, const int32_t* group, int32_t block, const int64_t* cidx,
                            const int64_t* core_ptr, int64_t* cursor, int32_t* core_idx) {
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int64_t c = cidx[group_of(v, group, block)];
    int64_t p = atomicAdd((unsigned long long*)&cursor[c], 1ull);
    core_idx[core_ptr[c] + p] = v;
}

// One block per core: sort the core, then mark core + neighbours.
//   mode 0: sort core members in place and count |S_i| -> sub_size[i]
//   mode 1: write S_i and the local positions of the core members
__global__ void k_subgraphs(int32_t n, int32_t n_sub, const int64_t* gptr, const int32_t* gidx,
                            const int64_t* core_ptr, int32_t* core_idx, int64_t* sub_size,
                            const int64_t* sub_ptr, int32_t* sub_idx, int32_t* core_pos, int mode,
                            int* stats) {
    extern __shared__ uint32_t words[];
    __shared__ int64_t scan[SUB_THREADS];
    __shared__ int32_t red[2 * (SUB_THREADS / 32)];
    for (int32_t i = blockIdx.x; i < n_sub; i += gridDim.x) {
        const int64_t c0 = core_ptr[i], c1 = core_ptr[i + 1];
        // the window of the core and its neighbours (bitmaps cost the window, not n)
        int32_t lo = INT32_MAX, hi = -1;
        for (int64_t e = c0 + threadIdx.x; e < c1; e += blockDim.x) {
            const int32_t v = core_idx[e];
            lo = min(lo, v);
            hi = max(hi, v);
        }
        for (int64_t e = c0; e < c1; ++e) {
            const int32_t v = core_idx[e];
            for (int64_t f = gptr[v] + threadIdx.x; f < gptr[v + 1]; f += blockDim.x) {
                const int32_t u = gidx[f];
                lo = min(lo, u);
                hi = max(hi, u);
            }
        }
        int32_t base;
        int W;
        bitmap_window(lo, hi, red, base, W);
        if (mode == 0) {
            // sorted core (the atomic fill leaves an arbitrary order)
            bitmap_clear(words, W);
            for (int64_t e = c0 + threadIdx.x; e < c1; e += blockDim.x) bitmap_set(words, core_idx[e] - base);
            __syncthreads();
            bitmap_compact(words, W, core_idx + c0, scan, base);
        }
        bitmap_clear(words, W);
        for (int64_t e = c0; e < c1; ++e) {
            int32_t v = core_idx[e];
            if (threadIdx.x == 0) bitmap_set(words, v - base);
            for (int64_t f = gptr[v] + threadIdx.x; f < gptr[v + 1]; f += blockDim.x)
                bitmap_set(words, gidx[f] - base);
        }
        __syncthreads();
        if (mode == 0) {
            int64_t s = bitmap_compact(words, W, nullptr, scan);
            if (threadIdx.x == 0) {
                sub_size[i] = s;
                atomicMax(&stats[0], (int)s);
                atomicMax(&stats[1], (int)(c1 - c0));
            }
        } else {
            int32_t* out = sub_idx + sub_ptr[i];
            int64_t s = bitmap_compact(words, W, out, scan, base);
            __syncthreads();
            for (int64_t e = c0 + threadIdx.x; e < c1; e += blockDim.x) {
                int32_t v = core_idx[e];
                int64_t lo = 0, hi = s;
                while (lo < hi) {
                    int64_t mid = (lo + hi) >> 1;
                    if (out[mid] < v) lo = mid + 1; else hi = mid;
                }
                core_pos[e] = (int32_t)lo;
            }
        }
        __syncthreads();
    }
}

__global__ void k_out_nnz(int32_t n_sub, const int64_t* sub_size, const int64_t* core_ptr,
                          unsigned long long* total) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_sub) atomicAdd(total, (unsigned long long)(sub_size[i] * (core_ptr[i + 1] - core_ptr[i])));
}

struct PartLayout {
    int64_t* gcnt;      // n_groups + 1
    int64_t* cidx;      // n_groups + 1
    int64_t* cursor;    // n
    int64_t* sub_size;  // n + 1
    int64_t* scan_tmp;
    int* err;           // [0] error, [1] max_sub, [2] max_core
    unsigned long long* out_nnz;
};

PartLayout layout_part(Arena& a, int32_t n, int32_t n_groups) {
    PartLayout L;
    int64_t big = (int64_t)(n > n_groups ? n : n_groups) + 1;
    L.gcnt = a.take<int64_t>(n_groups + 1);
    L.cidx = a.take<int64_t>(n_groups + 1);
    L.cursor = a.take<int64_t>(n);
    L.sub_size = a.take<int64_t>(n + 1);
    L.scan_tmp = a.take<int64_t>(scan_temp_count(big) + 64);
    L.err = a.take<int>(8);
    L.out_nnz = a.take<unsigned long long>(1);
    return L;
}

}  // namespace

extern "C" size_t gb_partition_workspace_size(int32_t n, int64_t nnz_g, int32_t n_groups) {
    (void)nnz_g;
    Arena a;
    layout_part(a, n, n_groups > 0 ? n_groups : n);
    return a.used();
}

namespace {

// The subgraph rows S_i of a partition whose cores, sizes and offsets are
// set (the last pass of gb_partition).  The layout is the one partition_impl
// used for these arguments: the workspace arena is laid out the same way.
int partition_fill(gb_handle* h, const gb_graph* G, int32_t n_groups, gb_part* P) {
    const int32_t n = G->n;
    Arena a(h->ws, h->ws_bytes);
    PartLayout L = layout_part(a, n, n_groups);
    const size_t smem = sizeof(uint32_t) * ((n + 31) / 32);
    const int64_t n_sub = P->n_sub;
    const int grid = (int)(n_sub < 152 * 16 ? n_sub : 152 * 16);
    if (n_sub > 0)
        GB_LAUNCH(h, k_subgraphs, grid, SUB_THREADS, smem, n, (int32_t)n_sub, G->ptr, G->idx,
                  (const int64_t*)P->core_ptr, P->core_idx, (int64_t*)nullptr,
                  (const int64_t*)P->sub_ptr, P->sub_idx, P->core_pos, 1, L.err + 1);
    GB_CUDA(cudaStreamSynchronize(h->stream));
    return GB_OK;
}

// gb_partition; with fill = false it stops before writing the subgraph rows
// (sizes, offsets, cores and statistics are set), for the capped partition's
// levels that are decided from sizes alone.
int partition_impl(gb_handle* h, const gb_graph* G, const int32_t* group, int32_t n_groups,
                   int32_t target_core_size, gb_part* P, bool fill) {
    if (!h || !G || !P) return GB_ERR_ARG;
    const int32_t n = G->n;
    if (n <= 0 || !G->ptr || (G->nnz > 0 && !G->idx)) return GB_ERR_ARG;
    if (P->n != n || !P->core_ptr || !P->core_idx || !P->core_pos || !P->sub_ptr) return GB_ERR_ARG;
    if (P->sub_capacity < 0 || (P->sub_capacity > 0 && !P->sub_idx)) return GB_ERR_ARG;
    int32_t block = 1;
    if (group) {
        if (n_groups <= 0) return GB_ERR_ARG;
    } else {
        if (target_core_size <= 0) return GB_ERR_ARG;
        block = target_core_size;
        n_groups = (n + block - 1) / block;
    }
    h->launches = 0;
    Arena a(h->ws, h->ws_bytes);
    PartLayout L = layout_part(a, n, n_groups);
    if (!a.fits() || !h->ws) {
        Arena m;
        layout_part(m, n, n_groups);
        h->required_ws = m.used();
        return GB_ERR_WORKSPACE;
    }
    cudaStream_t s = h->stream;
    GB_CUDA(cudaMemsetAsync(L.gcnt, 0, sizeof(int64_t) * (n_groups + 1), s));
    GB_CUDA(cudaMemsetAsync(L.cursor, 0, sizeof(int64_t) * n, s));
    GB_CUDA(cudaMemsetAsync(L.err, 0, sizeof(int) * 8, s));
    GB_CUDA(cudaMemsetAsync(L.out_nnz, 0, sizeof(unsigned long long), s));
    const int tb = 256;
    GB_LAUNCH(h, k_group_count, (n + tb - 1) / tb, tb, 0, n, group, block, n_groups, L.gcnt, L.err);
    // (out-of-range group ids are skipped by the count and reported with the
    // core count below: one round trip)
    GB_LAUNCH(h, k_nonempty, (n_groups + tb - 1) / tb, tb, 0, n_groups, (const int64_t*)L.gcnt, L.cidx);
    GB_CUDA(cudaMemsetAsync(L.cidx + n_groups, 0, sizeof(int64_t), s));
    GB_TRY(exclusive_scan_i64(h, L.cidx, L.cidx, n_groups + 1, L.scan_tmp));
    int64_t n_sub = 0;
    int herr = 0;
    GB_CUDA(cudaMemcpyAsync(&n_sub, L.cidx + n_groups, sizeof(n_sub), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaMemcpyAsync(&herr, L.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    if (herr) return herr;
    P->n_sub = (int32_t)n_sub;
    GB_LAUNCH(h, k_core_sizes, (n_groups + tb - 1) / tb, tb, 0, n_groups, (const int64_t*)L.gcnt,
              (const int64_t*)L.cidx, P->core_ptr);
    GB_CUDA(cudaMemsetAsync(P->core_ptr + n_sub, 0, sizeof(int64_t), s));
    GB_TRY(exclusive_scan_i64(h, P->core_ptr, P->core_ptr, n_sub + 1, L.scan_tmp));
    GB_LAUNCH(h, k_core_fill, (n + tb - 1) / tb, tb, 0, n, group, block, (const int64_t*)L.cidx,
              (const int64_t*)P->core_ptr, L.cursor, P->core_idx);

    const size_t smem = sizeof(uint32_t) * ((n + 31) / 32);
    if (smem > 200 * 1024) return GB_ERR_UNSUPPORTED;
    GB_CUDA(cudaFuncSetAttribute(k_subgraphs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (int)(n_sub < 152 * 16 ? n_sub : 152 * 16);
    GB_LAUNCH(h, k_subgraphs, grid, SUB_THREADS, smem, n, (int32_t)n_sub, G->ptr, G->idx,
              (const int64_t*)P->core_ptr, P->core_idx, L.sub_size, (const int64_t*)nullptr,
              (int32_t*)nullptr, (int32_t*)nullptr, 0, L.err + 1);
    GB_LAUNCH(h, k_out_nnz, ((int)n_sub + tb - 1) / tb, tb, 0, (int32_t)n_sub,
              (const int64_t*)L.sub_size, (const int64_t*)P->core_ptr, L.out_nnz);
    GB_CUDA(cudaMemsetAsync(L.sub_size + n_sub, 0, sizeof(int64_t), s));
    GB_TRY(exclusive_scan_i64(h, L.sub_size, P->sub_ptr, n_sub + 1, L.scan_tmp));
    int64_t sub_nnz = 0;
    int32_t stats[3] = {0, 0, 0};
    unsigned long long out_nnz = 0;
    // one round trip for the three read-backs
    GB_CUDA(cudaMemcpyAsync(&sub_nnz, P->sub_ptr + n_sub, sizeof(sub_nnz), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaMemcpyAsync(stats, L.err, sizeof(stats), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaMemcpyAsync(&out_nnz, L.out_nnz, sizeof(out_nnz), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    P->sub_nnz = sub_nnz;
    P->max_sub = stats[1];
    P->max_core = stats[2];
    P->out_nnz = (int64_t)out_nnz;
    if (sub_nnz > P->sub_capacity) return GB_ERR_CAPACITY;
    if (!fill) return GB_OK;
    return partition_fill(h, G, n_groups, P);
}

}  // namespace

extern "C" int gb_partition(gb_handle* h, const gb_graph* G, const int32_t* group, int32_t n_groups,
                            int32_t target_core_size, gb_part* P) {
    return partition_impl(h, G, group, n_groups, target_core_size, P, true);
}

// ---------------------------------------------------------------------------
// gb_partition_capped: gb_partition, then cores whose subgraph exceeds max_sub
// are replaced by their subgroups (see include/gbqr.h).
// ---------------------------------------------------------------------------
namespace {

// flag the key of every core whose subgraph is larger than max_sub
__global__ void k_mark_split(int32_t n_sub, const int64_t* sub_ptr, const int64_t* core_ptr,
                             const int32_t* core_idx, const int32_t* key, int32_t max_sub, int32_t* split,
                             int* any) {
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_sub) return;
    if (sub_ptr[k + 1] - sub_ptr[k] > max_sub) {
        split[key[core_idx[core_ptr[k]]]] = 1;
        atomicExch(any, 1);
    }
}

// new key of vertex v: base + (subgroup[v], or v itself) where its key was split
__global__ void k_regroup(int32_t n, const int32_t* key, const int32_t* subgroup, int32_t n_subgroups,
                          int32_t base, const int32_t* split, int32_t* newkey, int* err) {
    const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t part = v;
    if (subgroup) {
        part = subgroup[v];
        if (part < 0 || part >= n_subgroups) {
            set_error(err, GB_ERR_ARG);
            part = 0;
        }
    }
    newkey[v] = split[key[v]] ? base + part : key[v];
}

struct CapLayout {
    int32_t* split;  // n_groups + n_subgroups
    int32_t* key1;   // n
    int32_t* key2;   // n
    int* flags;      // 8
};

int64_t cap_keys(int32_t n, int32_t n_groups, int32_t n_subgroups) {
    return (int64_t)n_groups + n_subgroups + n;
}

CapLayout layout_cap(Arena& a, int32_t n, int32_t n_groups, int32_t n_subgroups) {
    CapLayout L;
    L.split = a.take<int32_t>((size_t)n_groups + n_subgroups);
    L.key1 = a.take<int32_t>(n);
    L.key2 = a.take<int32_t>(n);
    L.flags = a.take<int>(8);
    return L;
}

// one refinement level: flag oversize cores of the partition keyed by `key`,
// rekey their vertices; returns GB_OK with *more = 0 when nothing was split
int cap_level(gb_handle* h, const gb_part* P, const int32_t* key, int32_t n_keys, const int32_t* subgroup,
              int32_t n_subgroups, int32_t max_sub, const CapLayout& L, int32_t* newkey, int64_t* launches,
              int* more) {
    cudaStream_t s = h->stream;
    const int32_t n = P->n;
    const int tb = 256;
    GB_CUDA(cudaMemsetAsync(L.split, 0, sizeof(int32_t) * n_keys, s));
    GB_CUDA(cudaMemsetAsync(L.flags, 0, sizeof(int) * 8, s));
    if (P->n_sub > 0) {
        GB_LAUNCH(h, k_mark_split, (P->n_sub + tb - 1) / tb, tb, 0, P->n_sub, (const int64_t*)P->sub_ptr,
                  (const int64_t*)P->core_ptr, (const int32_t*)P->core_idx, key, max_sub, L.split, L.flags);
        ++*launches;
    }
    int any = 0;
    GB_TRY(read_i32(h, L.flags, &any, 1));
    *more = any;
    if (!any) return GB_OK;
    GB_LAUNCH(h, k_regroup, (n + tb - 1) / tb, tb, 0, n, key, subgroup, n_subgroups, n_keys,
              (const int32_t*)L.split, newkey, L.flags + 1);
    ++*launches;
    int err = 0;
    GB_TRY(read_i32(h, L.flags + 1, &err, 1));
    return err;
}

}  // namespace

extern "C" size_t gb_partition_capped_workspace_size(int32_t n, int64_t nnz_g, int32_t n_groups,
                                                      int32_t n_subgroups) {
    if (n <= 0 || n_groups <= 0 || n_subgroups <= 0 || cap_keys(n, n_groups, n_subgroups) > INT32_MAX) return 0;
    Arena a;
    a.off = gb_partition_workspace_size(n, nnz_g, (int32_t)cap_keys(n, n_groups, n_subgroups));
    layout_cap(a, n, n_groups, n_subgroups);
    return a.used();
}

extern "C" int gb_partition_capped(gb_handle* h, const gb_graph* G, const int32_t* group, int32_t n_groups,
                                   const int32_t* subgroup, int32_t n_subgroups, int32_t max_sub, gb_part* P) {
    if (!h || !G || !P || !group || !subgroup || n_groups <= 0 || n_subgroups <= 0 || max_sub <= 0)
        return GB_ERR_ARG;
    const int32_t n = G->n;
    if (n <= 0 || cap_keys(n, n_groups, n_subgroups) > INT32_MAX) return GB_ERR_ARG;
    // the inner partitions use the front of the workspace, this call's own
    // arrays follow them
    Arena a(h->ws, h->ws_bytes);
    a.off = gb_partition_workspace_size(n, G->nnz, (int32_t)cap_keys(n, n_groups, n_subgroups));
    CapLayout L = layout_cap(a, n, n_groups, n_subgroups);
    if (!h->ws || !a.fits()) {
        h->required_ws = gb_partition_capped_workspace_size(n, G->nnz, n_groups, n_subgroups);
        return GB_ERR_WORKSPACE;
    }
    int64_t launches = 0;
    // level 0: one core per group (sizes only: the rows are written once a
    // level is final)
    int st = partition_impl(h, G, group, n_groups, 0, P, false);
    launches += h->launches;
    if (st != GB_OK && st != GB_ERR_CAPACITY) return st;
    // level 1: oversize group cores -> one core per subgroup
    int more = 0;
    GB_TRY(cap_level(h, P, group, n_groups, subgroup, n_subgroups, max_sub, L, L.key1, &launches, &more));
    if (!more) {
        if (st == GB_OK) {
            h->launches = 0;
            st = partition_fill(h, G, n_groups, P);
            launches += h->launches;
        }
        h->launches = launches;
        return st;
    }
    const int32_t n_keys1 = n_groups + n_subgroups;
    st = partition_impl(h, G, L.key1, n_keys1, 0, P, false);
    launches += h->launches;
    if (st != GB_OK && st != GB_ERR_CAPACITY) return st;
    // level 2: oversize subgroup cores -> one core per vertex
    GB_TRY(cap_level(h, P, L.key1, n_keys1, nullptr, 0, max_sub, L, L.key2, &launches, &more));
    if (!more) {
        if (st == GB_OK) {
            h->launches = 0;
            st = partition_fill(h, G, n_keys1, P);
            launches += h->launches;
        }
        h->launches = launches;
        return st;
    }
    st = gb_partition(h, G, L.key2, n_keys1 + n, 0, P);
    h->launches += launches;
    return st;
}

// ---------------------------------------------------------------------------
// gb_partition_noalloc: gb_partition for callers that cannot allocate device
// memory (see include/gbqr.h).  Its scratch is a fixed file-scope device array
// in place of the handle's workspace; the partition itself is partition_impl,
// run through a handle on the stack whose workspace is that array.
// ---------------------------------------------------------------------------
#include <cuda.h>  // CUcontext (the driver entry point is looked up at run time)

#include <atomic>
#include <mutex>

namespace {

constexpr int32_t NOALLOC_MAX_N = GB_NOALLOC_MAX_VERTICES;
constexpr int NOALLOC_MAX_DEVICES = 64;

// Bytes gb_partition's scratch layout needs at the largest accepted size.
constexpr size_t noalloc_scratch_bytes() {
    // gcnt, cidx (n_groups + 1), cursor (n), sub_size (n + 1), scan temp, err, out_nnz,
    // each rounded to 256 bytes (the arena's alignment)
    return 4 * ((size_t)(NOALLOC_MAX_N + 1) * 8 + 256) + (size_t)(NOALLOC_MAX_N / 1024 + 64 + 256) * 8 * 2 +
           8 * 4 + 256 + 8 + 256;
}

static __device__ __align__(256) unsigned char g_partition_scratch[noalloc_scratch_bytes()];

// The array's device address, per device, with the context it was looked up
// in: a context created again (after cudaDeviceReset) gets a fresh lookup.
struct ScratchAddr {
    CUcontext ctx;
    void* ptr;
};
ScratchAddr g_scratch_addr[NOALLOC_MAX_DEVICES];
std::mutex g_scratch_mutex;

typedef CUresult (*CtxGetCurrent)(CUcontext*);

int current_context(CUcontext* ctx) {
    static std::atomic<CtxGetCurrent> fn{nullptr};
    CtxGetCurrent f = fn.load();
    if (!f) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) gb_note_device_error(e);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) return GB_ERR_DEVICE;
        f = (CtxGetCurrent)p;
        fn.store(f);
    }
    return f(ctx) == CUDA_SUCCESS ? GB_OK : GB_ERR_DEVICE;
}

// Device address of the scratch array on the current device (host code cannot
// use the symbol itself as a device pointer), looked up once per device and
// context.
int noalloc_scratch(void** out) {
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return GB_ERR_UNSUPPORTED;
    CUcontext ctx = nullptr;
    GB_TRY(current_context(&ctx));
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    ScratchAddr& e = g_scratch_addr[dev];
    if (!ctx || !e.ptr || e.ctx != ctx) {
        // (the lookup also brings up the device's primary context when no
        // runtime call has yet)
        void* p = nullptr;
        const cudaError_t ce = cudaGetSymbolAddress(&p, g_partition_scratch);
        if (ce != cudaSuccess) gb_note_device_error(ce);
        if (ce != cudaSuccess || !p) return GB_ERR_DEVICE;
        if (!ctx) GB_TRY(current_context(&ctx));
        e.ctx = ctx;
        e.ptr = p;
    }
    *out = e.ptr;
    return GB_OK;
}

}  // namespace

extern "C" size_t gb_partition_noalloc_scratch_bytes(void) { return sizeof(g_partition_scratch); }

extern "C" int gb_partition_noalloc(void* stream, const gb_graph* G, const int32_t* group, int32_t n_groups,
                                    int32_t target_core_size, gb_part* P) {
    if (!G || !P) return GB_ERR_ARG;
    const int32_t n = G->n;
    if (n <= 0) return GB_ERR_ARG;
    const int32_t groups = group ? n_groups : (target_core_size > 0 ? (n + target_core_size - 1) / target_core_size : 0);
    if (n > NOALLOC_MAX_N || groups > NOALLOC_MAX_N) return GB_ERR_WORKSPACE;
    void* scratch = nullptr;
    GB_TRY(noalloc_scratch(&scratch));
    gb_handle hs;  // on the stack: stream, scratch and launch count only
    hs.stream = (cudaStream_t)stream;
    hs.ws = scratch;
    hs.ws_bytes = sizeof(g_partition_scratch);
    hs.required_ws = 0;
    hs.launches = 0;
    hs.ev0 = hs.ev1 = nullptr;
    hs.aux = nullptr;
    hs.ev_fork = hs.ev_join = nullptr;
    hs.plan_valid = 0;
    GB_CUDA(cudaGetDevice(&hs.device));
    // partition_impl clears every counter it reuses (the array keeps the
    // previous call's contents)
    return partition_impl(&hs, G, group, n_groups, target_core_size, P, true);
}
