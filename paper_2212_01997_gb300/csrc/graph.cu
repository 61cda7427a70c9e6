// gb_graph_build: the thresholded data-dependency graph.
//
// Sec. "Estimating the connectivity graph": the graph is estimated from the
// non-zero structure of the numerically thresholded density matrix of a
// previous step together with the thresholded Hamiltonian, and more
// connectivity is added with paths of length two (or, without a previous
// density, from a power of the thresholded Hamiltonian).
//
//   E = {(i,j): i != j, |H_ij| > tau} U {(i,j): i != j, |D_prev,ij| > tau}
//   E <- E U E^T;  paths2: E <- E U E^2 (minus self loops)
//
// Kernels: count both directions of every surviving entry, prefix-sum,
// scatter, then one block per row marks its neighbours in a shared bitmap and
// reads them back in ascending order (deterministic, duplicate-free) over the
// front of the row's own edge list; a copy moves the rows to their offsets.
#include <string.h>

#include "bitset.cuh"
#include "common.cuh"

namespace {

constexpr int ROW_THREADS = 256;

// |v| > tau on the bit patterns: for non-negative doubles the IEEE order is the
// integer order of the bits (tau >= 0 is checked on entry).  NaN bits lie above
// those of infinity and never pass.  Keeps the graph build off the narrow FP64
// pipe.
__device__ __forceinline__ bool above_tau(double v, unsigned long long tau_bits, bool& nan) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
    nan = a > 0x7ff0000000000000ull;
    return !nan && a > tau_bits;
}

// A warp per row of a compressed matrix (CSR rows or CSC columns; the pair
// (major, minor) is emitted both ways, so orientation does not matter).
__global__ void k_edge_count(int32_t n, const int64_t* ptr, const int32_t* idx, const double* val,
                             unsigned long long tau_bits, int64_t* cnt, int* err) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    int own = 0;
    for (int64_t e = ptr[i] + lane; e < ptr[i + 1]; e += 32) {
        const int32_t j = idx[e];
        if (j < 0 || j >= n) {
            set_error(err, GB_ERR_ARG);
            continue;
        }
        bool nan;
        const bool keep = above_tau(val[e], tau_bits, nan) && j != i;
        if (nan) set_error(err, GB_ERR_NAN);
        if (keep) {
            ++own;
            atomicAdd((unsigned long long*)&cnt[j], 1ull);
        }
    }
    for (int o = 16; o > 0; o >>= 1) own += __shfl_xor_sync(0xffffffffu, own, o);
    if (lane == 0 && own) atomicAdd((unsigned long long*)&cnt[i], (unsigned long long)own);
}

__global__ void k_edge_fill(int32_t n, const int64_t* ptr, const int32_t* idx, const double* val,
                            unsigned long long tau_bits, const int64_t* off, int64_t* cursor, int32_t* edges) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    for (int64_t e0 = ptr[i]; e0 < ptr[i + 1]; e0 += 32) {
        const int64_t e = e0 + lane;
        bool keep = false;
        int32_t j = -1;
        if (e < ptr[i + 1]) {
            j = idx[e];
            bool nan;
            keep = j >= 0 && j < n && j != i && above_tau(val[e], tau_bits, nan);
        }
        const uint32_t m = __ballot_sync(0xffffffffu, keep);
        unsigned long long base = 0;
        if (lane == 0 && m) base = atomicAdd((unsigned long long*)&cursor[i], (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep) {
            const int64_t a = (int64_t)base + __popc(m & ((1u << lane) - 1u));
            const int64_t b = (int64_t)atomicAdd((unsigned long long*)&cursor[j], 1ull);
            edges[off[i] + a] = j;
            edges[off[j] + b] = (int32_t)i;
        }
    }
}

// Row i: mark the (duplicated) edge list, then count or write it sorted.  The
// bitmap covers only the row's window [min, max] of neighbour indices (32-bit
// aligned), so the clear and the compaction cost the window, not n.
__global__ void k_row_unique(int32_t n, const int64_t* off, const int32_t* edges,
                             int64_t* count, const int64_t* out_ptr, int32_t* out_idx) {
    extern __shared__ uint32_t words[];
    __shared__ int64_t scan[ROW_THREADS];
    __shared__ int32_t red[2 * (ROW_THREADS / 32)];
    for (int32_t i = blockIdx.x; i < n; i += gridDim.x) {
        int32_t jmin = INT32_MAX, jmax = -1;
        for (int64_t e = off[i] + threadIdx.x; e < off[i + 1]; e += blockDim.x) {
            const int32_t j = edges[e];
            jmin = min(jmin, j);
            jmax = max(jmax, j);
        }
        int32_t base;
        int W;
        bitmap_window(jmin, jmax, red, base, W);
        bitmap_clear(words, W);  // (its barrier also retires the window's scratch reads)
        for (int64_t e = off[i] + threadIdx.x; e < off[i + 1]; e += blockDim.x)
            bitmap_set(words, edges[e] - base);
        __syncthreads();
        int64_t c = bitmap_compact(words, W, out_idx ? out_idx + out_ptr[i] : nullptr, scan, base);
        if (threadIdx.x == 0 && count) count[i] = c;
    }
}

// Rows of a compressed list moved to their final offsets: row i's
// dst_ptr[i + 1] - dst_ptr[i] entries from src + src_off[i].  A warp per row.
__global__ void k_copy_rows(int32_t n, const int64_t* src_off, const int32_t* src, const int64_t* dst_ptr,
                            int32_t* dst) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < n; i += nw) {
        const int64_t len = dst_ptr[i + 1] - dst_ptr[i];
        const int32_t* a = src + src_off[i];
        int32_t* b = dst + dst_ptr[i];
        for (int64_t e = lane; e < len; e += 32) b[e] = a[e];
    }
}

// Row i of E U E^2: mark N(i) and N(k) for k in N(i), drop i.
__global__ void k_row_paths2(int32_t n, const int64_t* gptr, const int32_t* gidx, int64_t* count,
                             const int64_t* out_ptr, int32_t* out_idx) {
    extern __shared__ uint32_t words[];
    __shared__ int64_t scan[ROW_THREADS];
    const int W = (n + 31) >> 5;
    for (int32_t i = blockIdx.x; i < n; i += gridDim.x) {
        bitmap_clear(words, W);
        const int64_t a = gptr[i], b = gptr[i + 1];
        for (int64_t e = a; e < b; ++e) {
            int32_t k = gidx[e];
            if (threadIdx.x == 0) bitmap_set(words, k);
            for (int64_t f = gptr[k] + threadIdx.x; f < gptr[k + 1]; f += blockDim.x)
                bitmap_set(words, gidx[f]);
        }
        __syncthreads();
        if (threadIdx.x == 0) bitmap_unset(words, i);
        __syncthreads();
        int64_t c = bitmap_compact(words, W, out_idx ? out_idx + out_ptr[i] : nullptr, scan);
        if (threadIdx.x == 0 && count) count[i] = c;
        __syncthreads();
    }
}

struct GraphLayout {
    int64_t* cnt;      // n+1: edge counts -> offsets
    int64_t* cursor;   // n
    int32_t* edges;    // 2 * (nnz_h + nnz_d)
    int64_t* ucnt;     // n+1: unique counts -> base ptr
    int32_t* base;     // 2 * (nnz_h + nnz_d): base graph (paths2 only)
    int64_t* p2cnt;    // n+1 (paths2 only)
    int64_t* scan_tmp;
    int* err;
};

GraphLayout layout_graph(Arena& a, int32_t n, int64_t nnz_h, int64_t nnz_d, int paths2) {
    GraphLayout L;
    int64_t cap = 2 * (nnz_h + nnz_d) + 1;
    L.cnt = a.take<int64_t>(n + 1);
    L.cursor = a.take<int64_t>(n);
    L.edges = a.take<int32_t>(cap);
    L.ucnt = a.take<int64_t>(n + 1);
    L.base = paths2 ? a.take<int32_t>(cap) : nullptr;
    L.p2cnt = paths2 ? a.take<int64_t>(n + 1) : nullptr;
    L.scan_tmp = a.take<int64_t>(scan_temp_count(n + 1) + 64);
    L.err = a.take<int>(4);
    return L;
}

int row_grid(int32_t n) { return n < 152 * 16 ? n : 152 * 16; }

}  // namespace

extern "C" size_t gb_graph_build_workspace_size(int32_t n, int64_t nnz_h, int64_t nnz_dprev, int paths2) {
    Arena a;
    layout_graph(a, n, nnz_h, nnz_dprev, paths2);
    return a.used();
}

extern "C" int gb_graph_build(gb_handle* h, const gb_csr* H, const gb_csc* D_prev, double tau,
                              int paths2, gb_graph* G) {
    if (!h || !H || !G) return GB_ERR_ARG;
    const int32_t n = H->n;
    if (n <= 0 || H->nnz < 0 || !H->ptr || (H->nnz > 0 && (!H->idx || !H->val))) return GB_ERR_ARG;
    if (!(tau >= 0.0) || tau != tau) return GB_ERR_ARG;
    if (G->n != n || !G->ptr || (G->capacity > 0 && !G->idx) || G->capacity < 0) return GB_ERR_ARG;
    int64_t nnz_d = 0;
    if (D_prev) {
        if (D_prev->n != n || !D_prev->ptr || D_prev->nnz < 0 ||
            (D_prev->nnz > 0 && (!D_prev->idx || !D_prev->val)))
            return GB_ERR_ARG;
        nnz_d = D_prev->nnz;
    }
    h->launches = 0;
    Arena a(h->ws, h->ws_bytes);
    GraphLayout L = layout_graph(a, n, H->nnz, nnz_d, paths2);
    if (!a.fits() || !h->ws) {
        Arena m;
        layout_graph(m, n, H->nnz, nnz_d, paths2);
        h->required_ws = m.used();
        return GB_ERR_WORKSPACE;
    }
    cudaStream_t s = h->stream;
    GB_CUDA(cudaMemsetAsync(L.cnt, 0, sizeof(int64_t) * (n + 1), s));
    GB_CUDA(cudaMemsetAsync(L.cursor, 0, sizeof(int64_t) * n, s));
    GB_CUDA(cudaMemsetAsync(L.err, 0, sizeof(int) * 4, s));
    const int tb = 256, gb = (int)(((int64_t)n * 32 + tb - 1) / tb);  // a warp per row
    unsigned long long tb_bits = 0;
    memcpy(&tb_bits, &tau, sizeof(tb_bits));
    tb_bits &= 0x7fffffffffffffffull;  // tau >= 0 (or -0): its bits order like its value
    GB_LAUNCH(h, k_edge_count, gb, tb, 0, n, H->ptr, H->idx, H->val, tb_bits, L.cnt, L.err);
    if (D_prev)
        GB_LAUNCH(h, k_edge_count, gb, tb, 0, n, (const int64_t*)D_prev->ptr,
                  (const int32_t*)D_prev->idx, (const double*)D_prev->val, tb_bits, L.cnt, L.err);
    GB_TRY(exclusive_scan_i64(h, L.cnt, L.cnt, n + 1, L.scan_tmp));
    GB_LAUNCH(h, k_edge_fill, gb, tb, 0, n, H->ptr, H->idx, H->val, tb_bits, (const int64_t*)L.cnt,
              L.cursor, L.edges);
    if (D_prev)
        GB_LAUNCH(h, k_edge_fill, gb, tb, 0, n, (const int64_t*)D_prev->ptr,
                  (const int32_t*)D_prev->idx, (const double*)D_prev->val, tb_bits,
                  (const int64_t*)L.cnt, L.cursor, L.edges);
    // (the input-error flag is read back with the first count below: the
    // kernels in between skip the entries that set it)
    const size_t smem = sizeof(uint32_t) * ((n + 31) / 32);
    if (smem > 200 * 1024) return GB_ERR_UNSUPPORTED;
    GB_CUDA(cudaFuncSetAttribute(k_row_unique, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    GB_CUDA(cudaFuncSetAttribute(k_row_paths2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int rg = row_grid(n);
    // unique neighbour counts of the symmetrised graph; each row's sorted
    // unique list is written in place over the front of its edge list
    GB_CUDA(cudaMemsetAsync(L.ucnt + n, 0, sizeof(int64_t), s));
    GB_LAUNCH(h, k_row_unique, rg, ROW_THREADS, smem, n, (const int64_t*)L.cnt,
              (const int32_t*)L.edges, L.ucnt, (const int64_t*)L.cnt, L.edges);
    GB_TRY(exclusive_scan_i64(h, L.ucnt, L.ucnt, n + 1, L.scan_tmp));

    int herr = 0;
    if (!paths2) {
        int64_t total = 0;
        GB_CUDA(cudaMemcpyAsync(&total, L.ucnt + n, sizeof(total), cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaMemcpyAsync(&herr, L.err, sizeof(int), cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaStreamSynchronize(s));
        if (herr) return herr;
        G->nnz = total;
        if (total > G->capacity) return GB_ERR_CAPACITY;
        GB_CUDA(cudaMemcpyAsync(G->ptr, L.ucnt, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, s));
        GB_LAUNCH(h, k_copy_rows, row_grid(n), ROW_THREADS, 0, n, (const int64_t*)L.cnt,
                  (const int32_t*)L.edges, (const int64_t*)L.ucnt, G->idx);
        GB_CUDA(cudaStreamSynchronize(s));
        return GB_OK;
    }
    GB_TRY(read_i32(h, L.err, &herr));
    if (herr) return herr;
    // base graph materialised, then E U E^2
    GB_LAUNCH(h, k_copy_rows, row_grid(n), ROW_THREADS, 0, n, (const int64_t*)L.cnt,
              (const int32_t*)L.edges, (const int64_t*)L.ucnt, L.base);
    GB_CUDA(cudaMemsetAsync(L.p2cnt + n, 0, sizeof(int64_t), s));
    GB_LAUNCH(h, k_row_paths2, rg, ROW_THREADS, smem, n, (const int64_t*)L.ucnt,
              (const int32_t*)L.base, L.p2cnt, (const int64_t*)nullptr, (int32_t*)nullptr);
    GB_TRY(exclusive_scan_i64(h, L.p2cnt, L.p2cnt, n + 1, L.scan_tmp));
    int64_t total = 0;
    GB_TRY(read_i64(h, L.p2cnt + n, &total));
    G->nnz = total;
    if (total > G->capacity) return GB_ERR_CAPACITY;
    GB_CUDA(cudaMemcpyAsync(G->ptr, L.p2cnt, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, s));
    GB_LAUNCH(h, k_row_paths2, rg, ROW_THREADS, smem, n, (const int64_t*)L.ucnt,
              (const int32_t*)L.base, (int64_t*)nullptr, (const int64_t*)L.p2cnt, G->idx);
    GB_CUDA(cudaStreamSynchronize(s));
    return GB_OK;
}
