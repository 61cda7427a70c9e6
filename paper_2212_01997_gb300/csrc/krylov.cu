// The preconditioned low-rank Krylov approximation of the kernel for the
// electronic equations of motion, on the graph method's responses:
// gb_preconditioner (the subgraph preconditioner K0, Eq. PreCond) and
// gb_krylov_update (steps 1-5 of the Krylov expansion, Eqs. LowRankEEOM and
// Newton_SCF).  The charge model is stated in include/gbqr.h.  The density
// solves and responses are gb_density_and_response calls; the vector algebra
// over atoms runs in the small kernels below, every reduction in a fixed order.
#include <math.h>
#include <string.h>

#include <new>

#include "density.cuh"

namespace {

constexpr int KT_THREADS = 256;
constexpr int DOT_THREADS = 1024;
constexpr int MAX_DOTS = 16;

// ---- core atoms of every subgraph ------------------------------------------
// mode 0: count[i] = distinct atoms of core i, sq[i] = count^2, maxna = max;
// mode 1: atoms[atom_ptr[i] + rank] = the atoms, ascending.  A core orbital's
// atom is a first occurrence when no earlier core orbital has it.
__global__ void __launch_bounds__(KT_THREADS) k_core_atoms(int32_t n_sub, const int64_t* core_ptr,
                                                          const int32_t* core_idx, const int32_t* orb_atom,
                                                          int64_t* count, int64_t* sq, int* maxna,
                                                          const int64_t* atom_ptr, int32_t* atoms, int mode) {
    __shared__ int32_t at[GB_EIG_MAX_N];
    __shared__ int cnt;
    for (int32_t i = blockIdx.x; i < n_sub; i += gridDim.x) {
        const int64_t c0 = core_ptr[i];
        const int nc = (int)(core_ptr[i + 1] - c0);
        if (threadIdx.x == 0) cnt = 0;
        for (int e = threadIdx.x; e < nc && e < GB_EIG_MAX_N; e += KT_THREADS) at[e] = orb_atom[core_idx[c0 + e]];
        __syncthreads();
        const int ncs = nc < GB_EIG_MAX_N ? nc : GB_EIG_MAX_N;
        for (int e = threadIdx.x; e < ncs; e += KT_THREADS) {
            bool first = true;
            for (int q = 0; q < e && first; ++q) first = at[q] != at[e];
            if (!first) continue;
            if (mode == 0) {
                atomicAdd(&cnt, 1);
            } else {
                int rank = 0;
                for (int q = 0; q < ncs; ++q) {
                    if (at[q] >= at[e]) continue;
                    bool fq = true;
                    for (int t = 0; t < q && fq; ++t) fq = at[t] != at[q];
                    rank += fq;
                }
                atoms[atom_ptr[i] + rank] = at[e];
            }
        }
        __syncthreads();
        if (mode == 0 && threadIdx.x == 0) {
            const int na = nc > GB_EIG_MAX_N ? GB_PRECOND_MAX_ATOMS + 1 : cnt;  // (a larger core is refused)
            count[i] = na;
            sq[i] = (int64_t)na * na;
            atomicMax(maxna, na);
        }
        __syncthreads();
    }
}

// ---- vector kernels over atoms / orbitals ----------------------------------
// y = C (a - b) (b may be null): row per thread
__global__ void k_csr_apply(int32_t n, const int64_t* ptr, const int32_t* idx, const double* val, const double* a,
                            const double* b, double* y) {
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t p = ptr[r]; p < ptr[r + 1]; ++p) s = fma(val[p], b ? a[idx[p]] - b[idx[p]] : a[idx[p]], s);
        y[r] = s;
    }
}

// H[n]: the values of H0 with (C (n - Z))_atom(r) added to each diagonal entry
__global__ void k_shift_diagonal(int32_t n, const int64_t* ptr, const int32_t* idx, const double* v0,
                                 const int32_t* orb_atom, const double* vatom, double* v, int* err) {
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        bool diag = false;
        for (int64_t p = ptr[r]; p < ptr[r + 1]; ++p) {
            double x = v0[p];
            if (idx[p] == r) {
                x += vatom[orb_atom[r]];
                diag = true;
            }
            v[p] = x;
        }
        if (!diag) set_error(err, GB_ERR_ARG);
    }
}

// H1 = diag_o(vatom[atom(o)]) as CSR
__global__ void k_diag_csr(int32_t n, const int32_t* orb_atom, const double* vatom, int64_t* ptr, int32_t* idx,
                           double* val) {
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r <= n; r += gridDim.x * blockDim.x) {
        ptr[r] = r;
        if (r < n) {
            idx[r] = r;
            val[r] = vatom[orb_atom[r]];
        }
    }
}

// pop_I = 2 sum_{o in I} D_oo (atoms' orbitals in the caller's order)
__global__ void k_populations(int32_t n_atoms, const int64_t* atom_ptr, const int32_t* atom_orb,
                              const int64_t* cptr, const int32_t* cidx, const double* cval, double* pop, int* err) {
    for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I < n_atoms; I += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t e = atom_ptr[I]; e < atom_ptr[I + 1]; ++e) {
            const int32_t o = atom_orb[e];
            int64_t lo = cptr[o], hi = cptr[o + 1];
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (cidx[mid] < o) lo = mid + 1; else hi = mid;
            }
            if (lo < cptr[o + 1] && cidx[lo] == o) s += cval[lo];
            else set_error(err, GB_ERR_ARG);
        }
        pop[I] = 2.0 * s;
    }
}

// y = K0 (x - w): block diagonal (w may be null), or the scalar s when bval == null
__global__ void k_apply_k0(int32_t n_blocks, const int64_t* atom_ptr, const int32_t* atoms, const int64_t* val_ptr,
                           const double* bval, double s, int32_t n_atoms, const double* x, const double* w,
                           double* y) {
    if (!bval) {
        for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I < n_atoms; I += gridDim.x * blockDim.x)
            y[I] = s * (w ? x[I] - w[I] : x[I]);
        return;
    }
    for (int32_t k = blockIdx.x; k < n_blocks; k += gridDim.x) {
        const int64_t a0 = atom_ptr[k];
        const int na = (int)(atom_ptr[k + 1] - a0);
        const double* K = bval + val_ptr[k];
        for (int r = threadIdx.x; r < na; r += blockDim.x) {
            double t = 0.0;
            for (int c = 0; c < na; ++c) {
                const int32_t ac = atoms[a0 + c];
                t = fma(K[(int64_t)r * na + c], w ? x[ac] - w[ac] : x[ac], t);
            }
            y[atoms[a0 + r]] = t;
        }
    }
}

// y = a x + sum_j c_j V_j (up to 8 vectors V_j = V + j * ld)
struct Coefs {
    double c[GB_MAX_RHS];
};
__global__ void k_lincomb(int32_t n, double a, const double* x, const double* V, int64_t ld, int nv, Coefs cf,
                          double* y) {
    for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I < n; I += gridDim.x * blockDim.x) {
        double t = a * x[I];
        for (int j = 0; j < nv; ++j) t = fma(cf.c[j], V[(int64_t)j * ld + I], t);
        y[I] = t;
    }
}

// out[k] = x_k . y_k, one block per product, fixed-order tree
struct DotPairs {
    const double* x[MAX_DOTS];
    const double* y[MAX_DOTS];
};
__global__ void __launch_bounds__(DOT_THREADS) k_dots(int32_t n, DotPairs dp, double* out) {
    __shared__ double red[DOT_THREADS];
    const int k = blockIdx.x;
    const int32_t per = (n + DOT_THREADS - 1) / DOT_THREADS;
    const int32_t i0 = min(n, (int32_t)threadIdx.x * per), i1 = min(n, i0 + per);
    double s = 0.0;
    for (int32_t i = i0; i < i1; ++i) s = fma(dp.x[k][i], dp.y[k][i], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = DOT_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = red[0];
}

int grid_for(int64_t n) { return (int)((n + KT_THREADS - 1) / KT_THREADS < 1024 ? (n + KT_THREADS - 1) / KT_THREADS : 1024); }

// products x_k . y_k to the host (one round trip)
int dots(gb_handle* h, int32_t n, int cnt, const double* const* xs, const double* const* ys, double* dev,
         double* host) {
    DotPairs dp;
    memset(&dp, 0, sizeof(dp));
    for (int k = 0; k < cnt; ++k) {
        dp.x[k] = xs[k];
        dp.y[k] = ys[k];
    }
    GB_LAUNCH(h, k_dots, cnt, DOT_THREADS, 0, n, dp, dev);
    GB_CUDA(cudaMemcpyAsync(host, dev, sizeof(double) * cnt, cudaMemcpyDeviceToHost, h->stream));
    GB_CUDA(cudaStreamSynchronize(h->stream));
    return GB_OK;
}

bool csr_ok(const gb_csr* A, int32_t n) {
    return A && A->n == n && A->ptr && A->nnz >= 0 && (A->nnz == 0 || (A->idx && A->val));
}

struct PcExtra {
    int64_t* dptr;
    int32_t* didx;
    double* dval;
    int64_t* count;
    int64_t* sq;
    int64_t* scan_tmp;
    int* flags;  // [0] max atoms per core
};

PcExtra layout_pc(Arena& ar, const gb_part* P) {
    PcExtra E;
    E.dptr = ar.take<int64_t>(P->n + 1);
    E.didx = ar.take<int32_t>(P->out_nnz);
    E.dval = ar.take<double>(P->out_nnz);
    E.count = ar.take<int64_t>(P->n_sub + 1);
    E.sq = ar.take<int64_t>(P->n_sub + 1);
    E.scan_tmp = ar.take<int64_t>(scan_temp_count(P->n_sub + 1) + 64);
    E.flags = ar.take<int>(8);
    return E;
}

struct KrExtra {
    double* hval;   // H[n] values (nnz H0)
    int64_t* h1ptr;
    int32_t* h1idx;
    double* h1val;
    int64_t* dptr;
    int32_t* didx;
    double* dval;
    double* d1val;
    double* vatom;
    double* pop;
    double* k0f;
    double* w;
    double* dots;
    int* err;
};

KrExtra layout_kr(Arena& ar, int64_t nnz_h0, const gb_part* P, int32_t n_atoms) {
    KrExtra E;
    const int32_t n = P->n;
    E.hval = ar.take<double>(nnz_h0);
    E.h1ptr = ar.take<int64_t>(n + 1);
    E.h1idx = ar.take<int32_t>(n);
    E.h1val = ar.take<double>(n);
    E.dptr = ar.take<int64_t>(n + 1);
    E.didx = ar.take<int32_t>(P->out_nnz);
    E.dval = ar.take<double>(P->out_nnz);
    E.d1val = ar.take<double>(P->out_nnz);
    E.vatom = ar.take<double>(n_atoms);
    E.pop = ar.take<double>(n_atoms);
    E.k0f = ar.take<double>(n_atoms);
    E.w = ar.take<double>(n_atoms);
    E.dots = ar.take<double>(MAX_DOTS);
    E.err = ar.take<int>(8);
    return E;
}

size_t density_bytes(const gb_part* P, int32_t m, int32_t precision) {
    gb_opts o;
    memset(&o, 0, sizeof(o));
    o.precision = precision;
    size_t b = 0;
    gb_density_workspace_size(P, m, &o, &b);
    return (b + 255) & ~(size_t)255;
}

}  // namespace

extern "C" size_t gb_preconditioner_workspace_size(const gb_part* P) {
    if (!P || P->n_sub <= 0) return 0;
    Arena a;
    layout_pc(a, P);
    return density_bytes(P, 0, GB_PREC_EIGEN) + a.used();
}

extern "C" int gb_preconditioner(gb_handle* h, const gb_csr* H, const gb_part* P, double kT, double n_electrons,
                                 const gb_csr* C, const int32_t* orb_atom, int32_t n_atoms, double alpha,
                                 double* mu_inout, gb_blocks* K0) {
    if (!h || !P || !K0 || !mu_inout || !orb_atom || n_atoms <= 0 || !(alpha >= 0.0)) return GB_ERR_ARG;
    if (!csr_ok(H, P->n) || !csr_ok(C, n_atoms)) return GB_ERR_ARG;
    if (!K0->atom_ptr || !K0->atoms || !K0->val_ptr || (K0->val_capacity > 0 && !K0->val)) return GB_ERR_ARG;
    if (P->max_sub > GB_EIG_MAX_N) return GB_ERR_UNSUPPORTED;
    const size_t dbytes = density_bytes(P, 0, GB_PREC_EIGEN);
    if (!h->ws || h->ws_bytes < dbytes) {
        h->required_ws = gb_preconditioner_workspace_size(P);
        return GB_ERR_WORKSPACE;
    }
    Arena ar((char*)h->ws + dbytes, h->ws_bytes - dbytes);
    PcExtra E = layout_pc(ar, P);
    if (!ar.fits()) {
        h->required_ws = gb_preconditioner_workspace_size(P);
        return GB_ERR_WORKSPACE;
    }
    int64_t launches = 0;
    // the eigenbasis of every subgraph and mu at fixed electron count
    gb_opts o;
    memset(&o, 0, sizeof(o));
    o.precision = GB_PREC_EIGEN;
    gb_csc D = {P->n, 0, P->out_nnz, E.dptr, E.didx, E.dval};
    gb_report rep;
    GB_TRY(gb_density_and_response(h, H, nullptr, 0, kT, n_electrons, P, &o, mu_inout, &D, nullptr, nullptr,
                                   &rep));
    launches += h->launches;
    h->launches = 0;
    cudaStream_t st = h->stream;
    const int32_t n_sub = P->n_sub;
    const int sub_grid = n_sub < 152 * 8 ? n_sub : 152 * 8;
    // core atoms: counts, offsets, then the lists
    GB_CUDA(cudaMemsetAsync(E.flags, 0, sizeof(int) * 8, st));
    GB_LAUNCH(h, k_core_atoms, sub_grid, KT_THREADS, 0, n_sub, P->core_ptr, P->core_idx, orb_atom, E.count, E.sq,
              E.flags, (const int64_t*)nullptr, (int32_t*)nullptr, 0);
    GB_CUDA(cudaMemsetAsync(E.count + n_sub, 0, sizeof(int64_t), st));
    GB_CUDA(cudaMemsetAsync(E.sq + n_sub, 0, sizeof(int64_t), st));
    GB_TRY(exclusive_scan_i64(h, E.count, K0->atom_ptr, (int64_t)n_sub + 1, E.scan_tmp));
    GB_TRY(exclusive_scan_i64(h, E.sq, K0->val_ptr, (int64_t)n_sub + 1, E.scan_tmp));
    int64_t tot[2] = {0, 0};
    int maxna = 0;
    GB_CUDA(cudaMemcpyAsync(&tot[0], K0->atom_ptr + n_sub, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(&tot[1], K0->val_ptr + n_sub, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(&maxna, E.flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    K0->n_blocks = n_sub;
    K0->n_atoms_total = tot[0];
    K0->val_nnz = tot[1];
    if (maxna > GB_PRECOND_MAX_ATOMS) return GB_ERR_UNSUPPORTED;
    if (tot[0] != n_atoms) return GB_ERR_ARG;  // every atom in exactly one core
    if (tot[1] > K0->val_capacity) return GB_ERR_CAPACITY;
    GB_LAUNCH(h, k_core_atoms, sub_grid, KT_THREADS, 0, n_sub, P->core_ptr, P->core_idx, orb_atom, E.count, E.sq,
              E.flags, (const int64_t*)K0->atom_ptr, K0->atoms, 1);
    // the blocks, in the eigenbasis left in the workspace by the solve
    EigArgs ea;
    size_t used = 0;
    GB_TRY(eigen_state(h, P, 0, kT, *mu_inout, &ea, &used));
    PrecondArgs pa;
    pa.Cptr = C->ptr;
    pa.Cidx = C->idx;
    pa.Cval = C->val;
    pa.orb_atom = orb_atom;
    pa.alpha = alpha;
    pa.atom_ptr = K0->atom_ptr;
    pa.atoms = K0->atoms;
    pa.val_ptr = K0->val_ptr;
    pa.val = K0->val;
    pa.jc = nullptr;
    GB_CUDA(cudaMemsetAsync(ea.a.err, 0, sizeof(int), st));
    GB_TRY(launch_eig_jacobian(h, ea, pa));
    int herr = 0;
    GB_CUDA(cudaMemcpyAsync(&herr, ea.a.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    h->launches += launches;
    return herr;
}

extern "C" size_t gb_krylov_workspace_size(const gb_csr* H0, const gb_part* P, int32_t n_atoms, const gb_opts* opts) {
    if (!H0 || !P || P->n_sub <= 0 || n_atoms <= 0) return 0;
    const int32_t prec = opts ? opts->precision : GB_PREC_FP64;
    Arena a;
    layout_kr(a, H0->nnz, P, n_atoms);
    return density_bytes(P, 1, prec) + a.used();
}

extern "C" int gb_krylov_update(gb_handle* h, const gb_csr* H0, const gb_part* P, double kT, double n_electrons,
                                const gb_csr* C, const int32_t* orb_atom, const int64_t* atom_ptr,
                                const int32_t* atom_orb, int32_t n_atoms, const double* z, const double* n,
                                const gb_blocks* K0, double k0_scalar, int32_t m, double breakdown,
                                const gb_opts* opts, double* mu_inout, double* f, double* v, double* fv, double* dn,
                                double* M, int32_t* rank) {
    if (!h || !P || !orb_atom || !atom_ptr || !atom_orb || n_atoms <= 0 || !z || !n || !mu_inout) return GB_ERR_ARG;
    if (!csr_ok(H0, P->n) || !csr_ok(C, n_atoms)) return GB_ERR_ARG;
    if (m < 1 || m > GB_MAX_RHS || !(breakdown > 0.0) || !f || !v || !fv || !dn || !M || !rank) return GB_ERR_ARG;
    if (K0 && (K0->n_blocks != P->n_sub || !K0->atom_ptr || !K0->atoms || !K0->val_ptr || !K0->val))
        return GB_ERR_ARG;
    gb_opts o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    const size_t dbytes = density_bytes(P, 1, o.precision);
    if (!h->ws || h->ws_bytes < dbytes) {
        h->required_ws = gb_krylov_workspace_size(H0, P, n_atoms, &o);
        return GB_ERR_WORKSPACE;
    }
    Arena ar((char*)h->ws + dbytes, h->ws_bytes - dbytes);
    KrExtra E = layout_kr(ar, H0->nnz, P, n_atoms);
    if (!ar.fits()) {
        h->required_ws = gb_krylov_workspace_size(H0, P, n_atoms, &o);
        return GB_ERR_WORKSPACE;
    }
    cudaStream_t st = h->stream;
    const int32_t nn = P->n;
    int64_t launches = 0;
    h->launches = 0;
    const int ga = grid_for(n_atoms), go = grid_for(nn + 1);
    const int64_t* kap = K0 ? K0->atom_ptr : nullptr;
    const int32_t* kat = K0 ? K0->atoms : nullptr;
    const int64_t* kvp = K0 ? K0->val_ptr : nullptr;
    const double* kvl = K0 ? K0->val : nullptr;
    const int kb = K0 ? (K0->n_blocks < 152 * 8 ? K0->n_blocks : 152 * 8) : ga;
    GB_CUDA(cudaMemsetAsync(E.err, 0, sizeof(int) * 8, st));
    // H[n] = H0 + diag(C (n - Z)) and the ground state rho0[n] (step 1's residual)
    GB_LAUNCH(h, k_csr_apply, ga, KT_THREADS, 0, n_atoms, C->ptr, C->idx, C->val, n, z, E.vatom);
    GB_LAUNCH(h, k_shift_diagonal, go, KT_THREADS, 0, nn, H0->ptr, H0->idx, H0->val, orb_atom,
              (const double*)E.vatom, E.hval, E.err);
    GB_LAUNCH(h, k_diag_csr, go, KT_THREADS, 0, nn, orb_atom, (const double*)E.vatom, E.h1ptr, E.h1idx, E.h1val);
    int herr = 0;
    GB_CUDA(cudaMemcpyAsync(&herr, E.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    if (herr) return herr;
    launches += h->launches;
    gb_csr Hn = {nn, H0->nnz, H0->ptr, H0->idx, E.hval};
    gb_csc D = {nn, 0, P->out_nnz, E.dptr, E.didx, E.dval};
    gb_csc D1 = {nn, 0, P->out_nnz, nullptr, nullptr, E.d1val};
    gb_report rep;
    GB_TRY(gb_density_and_response(h, &Hn, nullptr, 0, kT, n_electrons, P, &o, mu_inout, &D, nullptr, nullptr,
                                   &rep));
    launches += h->launches;
    h->launches = 0;
    const double mu = *mu_inout;
    GB_LAUNCH(h, k_populations, ga, KT_THREADS, 0, n_atoms, atom_ptr, atom_orb, (const int64_t*)E.dptr,
              (const int32_t*)E.didx, (const double*)E.dval, E.pop, E.err);
    // f = rho0 - n; K0 f; v_1 = K0 f / |K0 f|
    Coefs one;
    memset(&one, 0, sizeof(one));
    one.c[0] = -1.0;
    GB_LAUNCH(h, k_lincomb, ga, KT_THREADS, 0, n_atoms, 1.0, (const double*)E.pop, n, 0, 1, one, f);
    GB_LAUNCH(h, k_apply_k0, kb, KT_THREADS, 0, K0 ? K0->n_blocks : 0, kap, kat, kvp, kvl, k0_scalar, n_atoms,
              (const double*)f, (const double*)nullptr, E.k0f);
    double hv[MAX_DOTS];
    {
        const double* xs[1] = {E.k0f};
        GB_TRY(dots(h, n_atoms, 1, xs, xs, E.dots, hv));
    }
    if (!(hv[0] > 0.0)) return GB_ERR_NAN;  // a zero residual leaves no direction
    Coefs none;
    memset(&none, 0, sizeof(none));
    GB_LAUNCH(h, k_lincomb, ga, KT_THREADS, 0, n_atoms, 1.0 / sqrt(hv[0]), (const double*)E.k0f, n, 0, 0, none, v);
    int k = 0;
    for (; k < m; ++k) {
        double* vk = v + (int64_t)k * n_atoms;
        double* fk = fv + (int64_t)k * n_atoms;
        // step 2: H1 = diag(C v_k) and the graph response at the ground-state mu
        GB_LAUNCH(h, k_csr_apply, ga, KT_THREADS, 0, n_atoms, C->ptr, C->idx, C->val, (const double*)vk,
                  (const double*)nullptr, E.vatom);
        GB_LAUNCH(h, k_diag_csr, go, KT_THREADS, 0, nn, orb_atom, (const double*)E.vatom, E.h1ptr, E.h1idx,
                  E.h1val);
        launches += h->launches;
        gb_csr H1 = {nn, nn, E.h1ptr, E.h1idx, E.h1val};
        gb_opts o1 = o;
        o1.max_newton = 1;
        double mu_k = mu, mu1 = 0.0;
        const int s = gb_density_and_response(h, &Hn, &H1, 1, kT, n_electrons, P, &o1, &mu_k, &D, &D1, &mu1, &rep);
        if (s != GB_OK && s != GB_ERR_NO_CONVERGE) return s;  // (one pass at the solved mu)
        launches += h->launches;
        h->launches = 0;
        // step 3: f_v = K0 (d rho0 - v_k)
        GB_LAUNCH(h, k_populations, ga, KT_THREADS, 0, n_atoms, atom_ptr, atom_orb, (const int64_t*)E.dptr,
                  (const int32_t*)E.didx, (const double*)E.d1val, E.pop, E.err);
        GB_LAUNCH(h, k_apply_k0, kb, KT_THREADS, 0, K0 ? K0->n_blocks : 0, kap, kat, kvp, kvl, k0_scalar, n_atoms,
                  (const double*)E.pop, (const double*)vk, fk);
        if (k + 1 == m) {
            ++k;
            break;
        }
        // step 4: v_{k+1} = f_v orthonormalised against v_0..v_k (twice)
        GB_LAUNCH(h, k_lincomb, ga, KT_THREADS, 0, n_atoms, 1.0, (const double*)fk, (const double*)v, 0, 0, none,
                  E.w);
        for (int pass = 0; pass < 2; ++pass) {
            const double* xs[MAX_DOTS];
            const double* ys[MAX_DOTS];
            for (int j = 0; j <= k; ++j) {
                xs[j] = E.w;
                ys[j] = v + (int64_t)j * n_atoms;
            }
            GB_TRY(dots(h, n_atoms, k + 1, xs, ys, E.dots, hv));
            Coefs cf;
            memset(&cf, 0, sizeof(cf));
            for (int j = 0; j <= k; ++j) cf.c[j] = -hv[j];
            GB_LAUNCH(h, k_lincomb, ga, KT_THREADS, 0, n_atoms, 1.0, (const double*)E.w, (const double*)v, n_atoms,
                      k + 1, cf, E.w);
        }
        {
            const double* xs[2] = {E.w, fk};
            GB_TRY(dots(h, n_atoms, 2, xs, xs, E.dots, hv));
        }
        if (!(sqrt(hv[0]) > breakdown * sqrt(hv[1]))) {  // an invariant subspace: stop
            ++k;
            break;
        }
        GB_LAUNCH(h, k_lincomb, ga, KT_THREADS, 0, n_atoms, 1.0 / sqrt(hv[0]), (const double*)E.w, n, 0, 0, none,
                  v + (int64_t)(k + 1) * n_atoms);
    }
    const int r = k;
    *rank = r;
    // O = F F^T, M = O^-1 (Gauss-Jordan, partial pivoting), c = F (K0 f), dn = -V (M c)
    double O[GB_MAX_RHS][GB_MAX_RHS], Mi[GB_MAX_RHS][2 * GB_MAX_RHS], cvec[GB_MAX_RHS];
    {
        // the r (r + 1) / 2 products f_v_i . f_v_j in batches, then F (K0 f)
        int pi[GB_MAX_RHS * (GB_MAX_RHS + 1) / 2], pj[GB_MAX_RHS * (GB_MAX_RHS + 1) / 2];
        int np = 0;
        for (int i = 0; i < r; ++i)
            for (int j = i; j < r; ++j) {
                pi[np] = i;
                pj[np] = j;
                ++np;
            }
        for (int b0 = 0; b0 < np; b0 += MAX_DOTS) {
            const int cnt = np - b0 < MAX_DOTS ? np - b0 : MAX_DOTS;
            const double* xs[MAX_DOTS];
            const double* ys[MAX_DOTS];
            for (int t = 0; t < cnt; ++t) {
                xs[t] = fv + (int64_t)pi[b0 + t] * n_atoms;
                ys[t] = fv + (int64_t)pj[b0 + t] * n_atoms;
            }
            double tmp[MAX_DOTS];
            GB_TRY(dots(h, n_atoms, cnt, xs, ys, E.dots, tmp));
            for (int t = 0; t < cnt; ++t) O[pi[b0 + t]][pj[b0 + t]] = O[pj[b0 + t]][pi[b0 + t]] = tmp[t];
        }
        const double* xs[MAX_DOTS];
        const double* ys[MAX_DOTS];
        for (int i = 0; i < r; ++i) {
            xs[i] = fv + (int64_t)i * n_atoms;
            ys[i] = E.k0f;
        }
        GB_TRY(dots(h, n_atoms, r, xs, ys, E.dots, cvec));
    }
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < 2 * r; ++j) Mi[i][j] = j < r ? O[i][j] : (j - r == i ? 1.0 : 0.0);
    for (int col = 0; col < r; ++col) {
        int piv = col;
        for (int i = col + 1; i < r; ++i)
            if (fabs(Mi[i][col]) > fabs(Mi[piv][col])) piv = i;
        if (Mi[piv][col] == 0.0) return GB_ERR_NAN;
        for (int j = 0; j < 2 * r; ++j) {
            const double t = Mi[col][j];
            Mi[col][j] = Mi[piv][j];
            Mi[piv][j] = t;
        }
        const double inv = 1.0 / Mi[col][col];
        for (int j = 0; j < 2 * r; ++j) Mi[col][j] *= inv;
        for (int i = 0; i < r; ++i) {
            if (i == col) continue;
            const double fct = Mi[i][col];
            for (int j = 0; j < 2 * r; ++j) Mi[i][j] -= fct * Mi[col][j];
        }
    }
    Coefs cf;
    memset(&cf, 0, sizeof(cf));
    for (int i = 0; i < r; ++i) {
        double y = 0.0;
        for (int j = 0; j < r; ++j) {
            M[i * m + j] = Mi[i][r + j];
            y += Mi[i][r + j] * cvec[j];
        }
        cf.c[i] = -y;
    }
    GB_LAUNCH(h, k_lincomb, ga, KT_THREADS, 0, n_atoms, 0.0, (const double*)v, (const double*)v, n_atoms, r, cf, dn);
    GB_CUDA(cudaMemcpyAsync(&herr, E.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    h->launches += launches;
    return herr;
}
