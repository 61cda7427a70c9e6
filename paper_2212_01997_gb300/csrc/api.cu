// Handle, workspace, status strings and the small device-wide primitives
// (prefix sums, scalar read-back) shared by the graph, partition and density
// entry points.
#include "common.cuh"

#define GB_VERSION_MAJOR 0
#define GB_VERSION_MINOR 1

extern "C" int gb_create(gb_handle** h, void* stream) {
    if (!h) return GB_ERR_ARG;
    gb_handle* p = new (std::nothrow) gb_handle;
    if (!p) return GB_ERR_ARG;
    p->stream = (cudaStream_t)stream;
    p->ws = nullptr;
    p->ws_bytes = 0;
    p->required_ws = 0;
    p->launches = 0;
    p->ev0 = p->ev1 = nullptr;
    p->aux = nullptr;
    p->ev_fork = p->ev_join = nullptr;
    p->plan_valid = 0;
    const cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        gb_note_device_error(e);
        delete p;
        return GB_ERR_DEVICE;
    }
    *h = p;
    return GB_OK;
}

extern "C" int gb_destroy(gb_handle* h) {
    if (!h) return GB_ERR_ARG;
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->aux) cudaStreamDestroy(h->aux);
    delete h;
    return GB_OK;
}

extern "C" int gb_set_workspace(gb_handle* h, void* dptr, size_t bytes) {
    if (!h) return GB_ERR_ARG;
    if (bytes && !dptr) return GB_ERR_ARG;
    if (((uintptr_t)dptr & 255u) != 0) return GB_ERR_ARG;
    h->ws = dptr;
    h->ws_bytes = bytes;
    return GB_OK;
}

extern "C" size_t gb_required_workspace(const gb_handle* h) { return h ? h->required_ws : 0; }

extern "C" int64_t gb_launch_count(const gb_handle* h) { return h ? h->launches : 0; }

static int g_last_device_error = 0;

void gb_note_device_error(cudaError_t e) { g_last_device_error = (int)e; }

extern "C" int gb_last_device_error(const char** name) {
    if (name) *name = cudaGetErrorName((cudaError_t)g_last_device_error);
    return g_last_device_error;
}

extern "C" const char* gb_status_string(int status) {
    switch (status) {
        case GB_OK: return "GB_OK";
        case GB_ERR_ARG: return "GB_ERR_ARG";
        case GB_ERR_CAPACITY: return "GB_ERR_CAPACITY";
        case GB_ERR_WORKSPACE: return "GB_ERR_WORKSPACE";
        case GB_ERR_MU_BRACKET: return "GB_ERR_MU_BRACKET";
        case GB_ERR_NO_CONVERGE: return "GB_ERR_NO_CONVERGE";
        case GB_ERR_NAN: return "GB_ERR_NAN";
        case GB_ERR_DEVICE: return "GB_ERR_DEVICE";
        case GB_ERR_UNSUPPORTED: return "GB_ERR_UNSUPPORTED";
        case GB_ERR_TIMEOUT: return "GB_ERR_TIMEOUT";
        default: return "GB_ERR_UNKNOWN";
    }
}

extern "C" int gb_version(int32_t* major, int32_t* minor, int32_t* arch) {
    if (major) *major = GB_VERSION_MAJOR;
    if (minor) *minor = GB_VERSION_MINOR;
    if (arch) *arch = 103;
    return GB_OK;
}

// ---------------------------------------------------------------------------
// Exclusive prefix sum over int64: 1024 elements per block (256 threads x 4),
// block totals scanned recursively, then added back.  Fixed order, so the
// result is deterministic.
// ---------------------------------------------------------------------------
static constexpr int SCAN_ITEMS = 4;
static constexpr int SCAN_THREADS = 256;
static constexpr int SCAN_TILE = SCAN_ITEMS * SCAN_THREADS;

__global__ void k_scan_tile(const int64_t* in, int64_t* out, int64_t n, int64_t* tile_sums) {
    __shared__ int64_t s[SCAN_THREADS];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    const int t = threadIdx.x;
    int64_t v[SCAN_ITEMS];
    int64_t local = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + t * SCAN_ITEMS + i;
        v[i] = idx < n ? in[idx] : 0;
        local += v[i];
    }
    s[t] = local;
    __syncthreads();
    for (int o = 1; o < SCAN_THREADS; o <<= 1) {
        int64_t x = t >= o ? s[t - o] : 0;
        __syncthreads();
        s[t] += x;
        __syncthreads();
    }
    if (t == SCAN_THREADS - 1 && tile_sums) tile_sums[blockIdx.x] = s[t];
    int64_t run = s[t] - local;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + t * SCAN_ITEMS + i;
        if (idx < n) {
            out[idx] = run;
            run += v[i];
        }
    }
}

__global__ void k_scan_add(int64_t* out, int64_t n, const int64_t* tile_offsets) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    const int64_t add = tile_offsets[blockIdx.x];
    for (int i = threadIdx.x; i < SCAN_TILE; i += blockDim.x) {
        int64_t idx = base + i;
        if (idx < n) out[idx] += add;
    }
}

size_t scan_temp_count(int64_t n) {
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles <= 1) return 0;
    return (size_t)tiles + scan_temp_count(tiles) + 32;
}

int exclusive_scan_i64(gb_handle* h, const int64_t* in, int64_t* out, int64_t n, int64_t* temp) {
    if (n <= 0) return GB_OK;
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 1) {
        GB_LAUNCH(h, k_scan_tile, 1, SCAN_THREADS, 0, in, out, n, (int64_t*)nullptr);
        return GB_OK;
    }
    int64_t* sums = temp;
    GB_LAUNCH(h, k_scan_tile, (unsigned)tiles, SCAN_THREADS, 0, in, out, n, sums);
    GB_TRY(exclusive_scan_i64(h, sums, sums, tiles, temp + tiles));
    GB_LAUNCH(h, k_scan_add, (unsigned)tiles, SCAN_THREADS, 0, out, n, (const int64_t*)sums);
    return GB_OK;
}

int read_i64(gb_handle* h, const int64_t* d, int64_t* out, int count) {
    GB_CUDA(cudaMemcpyAsync(out, d, sizeof(int64_t) * count, cudaMemcpyDeviceToHost, h->stream));
    GB_CUDA(cudaStreamSynchronize(h->stream));
    return GB_OK;
}

int read_f64(gb_handle* h, const double* d, double* out, int count) {
    GB_CUDA(cudaMemcpyAsync(out, d, sizeof(double) * count, cudaMemcpyDeviceToHost, h->stream));
    GB_CUDA(cudaStreamSynchronize(h->stream));
    return GB_OK;
}

int read_i32(gb_handle* h, const int32_t* d, int32_t* out, int count) {
    GB_CUDA(cudaMemcpyAsync(out, d, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, h->stream));
    GB_CUDA(cudaStreamSynchronize(h->stream));
    return GB_OK;
}
