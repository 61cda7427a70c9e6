// Arguments shared by the per-pass recursion kernels (FP64 and split
// precision).  One pass evaluates, for every subgraph at one chemical
// potential mu, the Fermi recursion and its first-order response, writes the
// core columns of d, d1_lambda and d1_mu, and the per-subgraph core traces.
#pragma once

#include "common.cuh"

constexpr int GB_MAX_RHS = 8;
constexpr int GB_SPLIT_MAX_N = 128;  // largest subgraph of the one-tile tensor-core kernels
constexpr int GB_BIG_MAX_N = 2048;   // largest subgraph of the tiled tensor-core kernel
// per-CTA scratch of the tiled kernel: staged images (hi/lo parts) and FP32
// matrices of the subgraph in flight, sized by the largest subgraph
constexpr int GB_BIG_IMAGES_FIXED = 16;  // + 2 per right-hand side
constexpr int GB_BIG_F32 = 4;
constexpr int GB_BIG_MAX_CTAS = 160;
constexpr int GB_EIG_MAX_N = 1024;    // largest subgraph of the eigenbasis path
constexpr int GB_EIG_MAX_CTAS = 608;  // its CTAs (4 per SM), each with 3 n_max^2 doubles of scratch
// sizes the response scratch of the persistent tensor-core kernels: 64 KB per
// RHS for each of up to this many 128-column CTAs (a small-configuration CTA
// takes 32 KB, so twice as many of those fit)
constexpr int GB_SPLIT_MAX_CTAS = 256;

// Per-subgraph trace slots (tr[i * tr_stride + k])
// TR_MAXW and TR_MAXWC are reduced with max: the largest diagonal element of
// d1_mu over all rows, and over the core rows, of all subgraphs.  A collected
// element (j in S_i, k in core_i) of the PSD d1_mu is bounded by
// sqrt(d1_mu_jj d1_mu_kk) <= sqrt(MAXW MAXWC).  The other slots are summed.
enum TraceSlot {
    TR_D = 0, TR_DD = 1, TR_D1MU = 2, TR_FLOPS = 3, TR_MAXW = 4, TR_MAXWC = 5, TR_FLOPS_S = 6, TR_D1LAM = 7
};
constexpr int TR_FIXED = 7;  // slots before the per-RHS d1_lambda traces
__host__ __device__ __forceinline__ bool trace_slot_is_max(int k) { return k == TR_MAXW || k == TR_MAXWC; }

// Matrix products one pass performs on a subgraph with s steps, J Newton-
// Schulz corrections and m right-hand sides: Taylor start 3 + 6m, every step
// 3 + 2J + 4m, and Z_s^2 at the end.
__host__ __device__ __forceinline__ double pass_gemm_flops(int n, int s, int J, int m) {
    double g = 4.0 + 6.0 * m + (double)s * (3.0 + 2.0 * J + 4.0 * m);
    return g * 2.0 * (double)n * (double)n * (double)n;
}

// The same work counted per recursion step as a fixed budget: (2 + 2J)
// products for d and 3 per right-hand side for the response, plus the core
// traces 2 n^2 n_c (Taylor start, the d1_mu square and the split terms not
// counted).
__host__ __device__ __forceinline__ double pass_flops_per_step_count(int n, int nc, int s, int J, int m) {
    const double n3 = 2.0 * (double)n * (double)n * (double)n;
    return (double)s * (2.0 + 2.0 * J) * n3 + (double)m * s * 3.0 * n3 + 2.0 * (double)n * n * nc;
}

struct PassArgs {
    int32_t n_sub;
    int32_t m;
    const int64_t* sub_ptr;
    const int32_t* sub_idx;
    const int64_t* core_ptr;
    const int32_t* core_idx;
    const int32_t* core_pos;
    // H and H1_r (CSR)
    const int64_t* Hptr;
    const int32_t* Hidx;
    const double* Hval;
    const int64_t* H1ptr[GB_MAX_RHS];
    const int32_t* H1idx[GB_MAX_RHS];
    const double* H1val[GB_MAX_RHS];
    double beta;
    double mu;
    int32_t min_steps;
    int32_t ns_iters;
    int32_t split_kind;  // 0: FP16 parts, 1: BF16 parts (split-precision kernel only)
    const int32_t* work;    // split launches: the subgraphs of this launch's size class,
    const int32_t* work_n;  // ascending, and their count (device; see k_class_lists)
    double* eps_lo;  // per-subgraph Gershgorin interval (written by the split path's gather)
    double* eps_hi;
    // outputs, at the positions of the collected CSC matrices
    const int64_t* col_ptr;
    double* Dval;
    double* D1val[GB_MAX_RHS];
    double* d1mu_val;
    double* tr;
    int32_t tr_stride;
    int32_t* steps_out;
    // FP64 path: dense blocks (offset moff[i] inside each of the pool's buffers)
    double* pool;
    const int64_t* moff;
    int64_t pool_stride;
    // split path: response state Z1 of each CTA's subgraph in flight, per RHS, as
    // a staged image (FP16 hi/lo parts in the shared-memory operand layout)
    float* z1pool;
    // split path: gathered dense blocks beta h^(i) and beta h1_r^(i) (FP32:
    // value rounded to float, times beta in FP32), npad = round16(|S_i|) rows and
    // columns, stored in column groups of four: element (r, c) at
    // ((c / 4) * npad + r) * 4 + c % 4, so a warp reading one group of 32 rows
    // reads 512 contiguous bytes.  Block b of subgraph i is at
    // hblk + b * hblk_stride + boff[i] (b = 0: h, b = 1 + r: h1_r).
    const float* hblk;
    const int64_t* boff;
    int64_t hblk_stride;
    // split path: FP64 diagonal of h^(i), at hdiag[sub_ptr[i] + r]
    const double* hdiag;
    // split path: largest row sum of |h1_r^(i)|, at h1max[i * m + r]
    double* h1max;
    // split path, diagonal perturbations (h1_offdiag[0] == 0: every entry of
    // every H1_r lies on the diagonal, set by k_h1_offdiag before the
    // gather): the one-tile subgraphs' beta h1_r^(i) is kept as its diagonal
    // alone, at h1d[r * h1d_stride + sub_ptr[i] + row] (the same FP32 values
    // the dense block would hold), and no dense h1 block is written for them
    float* h1d;
    int64_t h1d_stride;
    const int* h1_offdiag;
    // tiled split path (|S_i| > 128): per-CTA scratch (big_stride bytes each,
    // laid out for subgraphs of up to big_npmax = round16(max |S_i|) orbitals)
    // and the dynamic work counter of the launch (zeroed before it)
    uint8_t* big_scratch;
    int64_t big_stride;
    int32_t big_npmax;
    int32_t* big_counter;
    int32_t grid_sms;  // SMs a persistent launch may fill (0: all of them)
    int32_t* counter;  // the launch's dynamic work counter (zeroed before it)
    int* err;
};

// bytes of one CTA's scratch of the tiled kernel for subgraphs of up to
// npmax (a multiple of 16) orbitals and m right-hand sides: staged images
// (hi and lo parts of 128 nrb x npmax 16-bit values each), FP32 matrices
// (128 nrb x npmax), the per-core trace terms
__host__ __device__ __forceinline__ int64_t big_cta_bytes(int npmax, int m) {
    const int64_t nrb = (npmax + 127) / 128;
    const int64_t img = 2 * 128 * nrb * npmax * 2;
    const int64_t f32 = 128 * nrb * npmax * 4;
    const int64_t tv = (int64_t)(3 + GB_MAX_RHS) * npmax * 4;
    return (GB_BIG_IMAGES_FIXED + 2 * m) * img + GB_BIG_F32 * f32 + ((tv + 255) & ~(int64_t)255);
}

// Step count s so that x0 = beta (h - mu) / 2^(s+1) has spectral radius <= 1:
// 2^s >= beta max|eps - mu| / 2, bounded below by min_steps.
__device__ __forceinline__ int recursion_steps(double beta, double mu, double lo, double hi, int min_steps) {
    double ymax = 0.5 * beta * fmax(fabs(hi - mu), fabs(lo - mu));
    int s = min_steps;
    while (s < 60 && ldexp(1.0, s) < ymax) ++s;
    return s;
}

int launch_split_pass(gb_handle* h, const PassArgs& a);
// the same launch on another stream (a.grid_sms SMs)
int launch_split_pass_on(gb_handle* h, const PassArgs& a, cudaStream_t stream);
// the same recursion over a list of subgraphs (a.work): the 128-column
// configuration, and the small one for round16(|S_i|) <= 64 (two CTAs per SM)
int launch_split_pass_listed(gb_handle* h, const PassArgs& a);
int launch_split_pass_small(gb_handle* h, const PassArgs& a);
int launch_split_gather(gb_handle* h, const PassArgs& a, float* hblk, double* hdiag);
// The eigenbasis path: per-CTA scratch (3 n_max^2 doubles), the eigenvalues
// and core weights (at sub_ptr[i]) and eigenvectors (eigenvector-major, n_i^2
// at moff[i]) of every subgraph, and a work counter.
struct EigArgs {
    PassArgs a;
    double* scratch;
    int64_t scratch_stride;
    double* eps;
    double* w;
    double* vt;
    int32_t* counter;
    // list mode (list != nullptr): the subgraphs list[list_base + j],
    // j < list_n, with the eigenvectors of item j at vt + j * vt_stride;
    // otherwise every subgraph i with its eigenvectors at vt + a.moff[i]
    const int32_t* list;
    int32_t list_base;
    int32_t list_n;
    int64_t vt_stride;
};
// which = 0: diagonalise every subgraph (of the list); 1: trace terms at a.mu
// from the eigenvalues; 2: core columns of d, d1_mu, d1_lambda at a.mu and
// their core traces
int launch_eigen(gb_handle* h, const EigArgs& ea, int which);

// The subgraph preconditioner's inputs and outputs (see gb_preconditioner):
// the coupling C (atoms x atoms, CSR), the orbitals' atoms, the core atoms of
// every subgraph (atoms[atom_ptr[i] ..], ascending) and the row-major blocks
// k0 (and, when jc is set, j_c) at val_ptr[i].
constexpr int GB_PRECOND_MAX_ATOMS = 40;
// per-CTA scratch of the preconditioner's small blocks: chi, rho_mu, [A | I]
constexpr int GB_PRECOND_SCRATCH = 3 * GB_PRECOND_MAX_ATOMS * GB_PRECOND_MAX_ATOMS + GB_PRECOND_MAX_ATOMS;
struct PrecondArgs {
    const int64_t* Cptr;
    const int32_t* Cidx;
    const double* Cval;
    const int32_t* orb_atom;
    double alpha;
    const int64_t* atom_ptr;
    const int32_t* atoms;
    const int64_t* val_ptr;
    double* val;
    double* jc;
};
int launch_eig_jacobian(gb_handle* h, const EigArgs& ea, const PrecondArgs& pa);
// the eigenbasis state of the last GB_PREC_EIGEN call (partition P, m RHS) in
// the handle's workspace, and the bytes its layout takes
int eigen_state(gb_handle* h, const gb_part* P, int32_t m, double kT, double mu, EigArgs* out,
                size_t* density_bytes);

// the tiled configuration for round16(|S_i|) > 128 over its list (a.work),
// one subgraph per CTA at a time, dynamically scheduled; grid CTAs
int launch_split_pass_big(gb_handle* h, const PassArgs& a, int grid, cudaStream_t stream);
