// gb_mulliken_charges: net Mulliken charges of the atoms and their first-order
// response from the collected density matrix and its responses (Sec. "Response
// in observables": the charges are the subsystem observables of D and D1;
// Sec. "Implementation with SCC-DFTB theory": charges are Mulliken vectors).
// Orthogonal basis, spin restricted:
//   q_I  = Z_I - 2 sum_{o in I} D_oo,      q1_I = -2 sum_{o in I} D1_oo.
// D_oo is found in column o of the collected matrix (rows ascending) by
// binary search; each atom's sum runs in FP64 over its orbitals in the order
// the caller lists them, so the result does not depend on scheduling.
#include "density.cuh"

namespace {

constexpr int CHARGE_THREADS = 128;

// the m response value arrays, passed by value
struct RhsVals {
    const double* v[GB_MAX_RHS];
};

__device__ __forceinline__ double collected_diag(const int64_t* ptr, const int32_t* idx, const double* val,
                                                 int32_t o, int* err) {
    int64_t lo = ptr[o], hi = ptr[o + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (idx[mid] < o) lo = mid + 1; else hi = mid;
    }
    if (lo >= ptr[o + 1] || idx[lo] != o) {  // every core column holds its own row
        set_error(err, GB_ERR_ARG);
        return 0.0;
    }
    return val[lo];
}

__global__ void __launch_bounds__(CHARGE_THREADS) k_mulliken(int32_t n_atoms, const int64_t* atom_ptr,
                                                             const int32_t* atom_orb, const double* z_val,
                                                             const int64_t* ptr, const int32_t* idx,
                                                             const double* dval, RhsVals d1val,
                                                             int32_t m, double* q, double* q1, int32_t n,
                                                             int* err) {
    for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I < n_atoms; I += gridDim.x * blockDim.x) {
        double pop = 0.0;
        double pop1[GB_MAX_RHS];
        for (int r = 0; r < m; ++r) pop1[r] = 0.0;
        for (int64_t e = atom_ptr[I]; e < atom_ptr[I + 1]; ++e) {
            const int32_t o = atom_orb[e];
            if (o < 0 || o >= n) {
                set_error(err, GB_ERR_ARG);
                continue;
            }
            pop += collected_diag(ptr, idx, dval, o, err);
            for (int r = 0; r < m; ++r) pop1[r] += collected_diag(ptr, idx, d1val.v[r], o, err);
        }
        q[I] = z_val[I] - 2.0 * pop;
        for (int r = 0; r < m; ++r) q1[(int64_t)r * n_atoms + I] = -2.0 * pop1[r];
    }
}

}  // namespace

extern "C" int gb_mulliken_charges(gb_handle* h, const gb_csc* D, const gb_csc* D1, int32_t m,
                                   int32_t n_atoms, const int64_t* atom_ptr, const int32_t* atom_orb,
                                   const double* z_val, double* q, double* q1) {
    if (!h || !D || !D->ptr || !D->idx || !D->val || n_atoms <= 0 || !atom_ptr || !atom_orb || !z_val || !q)
        return GB_ERR_ARG;
    if (m < 0 || m > GB_MAX_RHS || (m > 0 && (!D1 || !q1))) return GB_ERR_ARG;
    RhsVals p1 = {};
    for (int r = 0; r < m; ++r) {
        if (!D1[r].val || D1[r].n != D->n) return GB_ERR_ARG;
        p1.v[r] = D1[r].val;
    }
    Arena ar(h->ws, h->ws_bytes);
    int* err = ar.take<int>(8);
    if (!ar.fits() || !h->ws) {
        h->required_ws = ar.used();
        return GB_ERR_WORKSPACE;
    }
    h->launches = 0;
    cudaStream_t st = h->stream;
    GB_CUDA(cudaMemsetAsync(err, 0, sizeof(int) * 8, st));
    const int grid = (n_atoms + CHARGE_THREADS - 1) / CHARGE_THREADS;
    GB_LAUNCH(h, k_mulliken, grid < 1024 ? grid : 1024, CHARGE_THREADS, 0, n_atoms, atom_ptr, atom_orb, z_val,
              (const int64_t*)D->ptr, (const int32_t*)D->idx, (const double*)D->val, p1, m,
              q, q1, D->n, err);
    int herr = 0;
    GB_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    return herr;
}

extern "C" size_t gb_mulliken_workspace_size(void) {
    Arena a;
    a.take<int>(8);
    return a.used();
}
