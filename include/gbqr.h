/*
 * gbqr.h -- C ABI of the graph-based density-matrix and response library.
 *
 * The library evaluates, on one GPU, the data-parallel hot path of graph-based
 * canonical quantum perturbation theory at finite electronic temperature
 * (Negre, Wall & Niklasson, arXiv:2212.01997):
 *
 *   gb_graph_build           thresholded data-dependency graph      (Sec. "Estimating the connectivity graph")
 *   gb_partition             disjoint cores + distance-1 halos       (Fig. 1; Sec. "Choosing the graph partitioning")
 *   gb_density_and_response  D, D1, mu, mu1 on the partitioned graph (Eqs. Fermi, DD0-DD, NewtonRaphson,
 *                                                                      D1, ddlambda, dddmu, dmu_1, dCollect)
 *   gb_mulliken_charges      atomic charges q, q1 from D, D1       (Sec. "Response in observables")
 *   gb_preconditioner        subgraph preconditioner K0            (Sec. "Preconditioner for a partitioned graph")
 *   gb_krylov_update         low-rank Krylov kernel update         (Sec. "Preconditioned Krylov Subspace
 *                                                                      Approximation ...", steps 1-5)
 *
 * Conventions for every entry point:
 *   - Plain C types only.  Pointers marked [device] are CUDA device pointers,
 *     [host] are host pointers.  All memory is owned by the caller; the library
 *     allocates no device memory.  Scratch comes from the caller's workspace
 *     (gb_set_workspace).
 *   - Work is enqueued on the handle's stream.  Calls that must return sizes or
 *     scalars to the host (partition sizes, mu, traces) synchronise that stream.
 *   - Every function returns a gb_status (0 = GB_OK).  None throws, aborts or
 *     traps; device-side waits are bounded and report GB_ERR_TIMEOUT.
 *   - Energies (H, H1, kT, mu) are in eV.  Matrices are square n x n.
 *   - Orthogonal basis (the paper's orthogonalised representation).
 */
#ifndef GBQR_H
#define GBQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gb_status {
    GB_OK = 0,
    GB_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, kT <= 0, ...)      */
    GB_ERR_CAPACITY = 2,     /* an output array is too small; the needed size is reported   */
    GB_ERR_WORKSPACE = 3,    /* workspace too small; see gb_required_workspace              */
    GB_ERR_MU_BRACKET = 4,   /* N_occ cannot be reached for any mu (Ne out of range)        */
    GB_ERR_NO_CONVERGE = 5,  /* mu iteration hit max_newton without meeting the tolerance   */
    GB_ERR_NAN = 6,          /* a non-finite value appeared in the input or the result      */
    GB_ERR_DEVICE = 7,       /* a CUDA runtime call failed                                  */
    GB_ERR_UNSUPPORTED = 8,  /* valid request this build does not handle (e.g. size limit)  */
    GB_ERR_TIMEOUT = 9       /* a bounded device-side wait gave up                          */
} gb_status;

typedef enum gb_precision {
    GB_PREC_FP64 = 0,    /* every product in FP64 (the plain reference GPU path)              */
    GB_PREC_FP16X3 = 1,  /* tensor-core split products hi*hi + hi*lo + lo*hi, FP16 parts,
                            FP32 accumulation in tensor memory; traces, mu, mu1 in FP64        */
    GB_PREC_BF16X3 = 2,  /* as GB_PREC_FP16X3 with BF16 parts                                  */
    GB_PREC_EIGEN = 3    /* FP64 in the eigenbasis: each h^(i) diagonalised (Eq. SmallKS),
                            mu from eigenvalue sums, d, d1 from Eqs. DD and ddlambda;
                            subgraphs up to 1,024 orbitals                                     */
} gb_precision;

/* Square sparse matrix, compressed sparse rows.  [device] arrays.
 * ptr: n+1 row offsets; idx: column indices, ascending inside each row;
 * val: values.  Duplicates are not allowed. */
typedef struct gb_csr {
    int32_t n;
    int64_t nnz;
    const int64_t* ptr;
    const int32_t* idx;
    const double* val;
} gb_csr;

/* Ragged compressed-sparse-column matrix produced by the column collect
 * (Eq. dCollect): column j holds the rows S_i of the subgraph i whose core
 * contains j, in ascending order.  [device] arrays sized by the caller:
 * ptr n+1, idx and val `capacity` entries.  ptr/idx may be NULL for D1 when
 * they are taken from D (they are identical). */
typedef struct gb_csc {
    int32_t n;
    int64_t nnz;       /* out: entries written                                  */
    int64_t capacity;  /* in: entries idx/val can hold                          */
    int64_t* ptr;
    int32_t* idx;
    double* val;
} gb_csc;

/* Undirected graph as a symmetric adjacency (CSR, no self loops, ascending
 * neighbours).  [device] arrays: ptr n+1, idx `capacity` entries. */
typedef struct gb_graph {
    int32_t n;
    int64_t nnz;       /* out: number of directed edges (twice the undirected count) */
    int64_t capacity;  /* in: entries idx can hold                                    */
    int64_t* ptr;
    int32_t* idx;
} gb_graph;

/* Core/halo partition.  [device] arrays sized by the caller:
 *   core_ptr n+1, core_idx n, core_pos n, sub_ptr n+1, sub_idx sub_capacity.
 * Subgraph i has core  core_idx[core_ptr[i] .. core_ptr[i+1])  (ascending),
 * vertex set S_i = sub_idx[sub_ptr[i] .. sub_ptr[i+1]) (ascending, core + halo),
 * and core_pos[k] is the position of core_idx[k] inside S_i. */
typedef struct gb_part {
    int32_t n;
    int32_t n_sub;         /* out: number of subgraphs                                  */
    int32_t max_sub;       /* out: largest |S_i|                                        */
    int32_t max_core;      /* out: largest |core_i|                                     */
    int64_t sub_nnz;       /* out: sum_i |S_i|                                          */
    int64_t out_nnz;       /* out: sum_i |S_i| |core_i| = nnz of a collected matrix     */
    int64_t sub_capacity;  /* in: entries sub_idx can hold                              */
    int64_t* core_ptr;
    int32_t* core_idx;
    int32_t* core_pos;
    int64_t* sub_ptr;
    int32_t* sub_idx;
} gb_part;

typedef struct gb_opts {
    int32_t precision;   /* gb_precision                                                  */
    int32_t max_newton;  /* mu passes (each a full recursion); <= 0 selects 40             */
    double tol_occ;      /* also accept mu when |Tr D - N_occ| <= tol_occ * N_occ
                            (<= 0: this test is off)                                       */
    int32_t min_steps;   /* lower bound on recursion steps; <= 0 selects 6                 */
    int32_t ns_iters;    /* Newton-Schulz corrections per step; <= 0 selects 3 (FP64) / 2 */
    double tol_d;        /* accept mu when the remaining Newton step |dmu| = |Tr D - N_occ|
                            / (dTr D / dmu) would change no collected element of D by more
                            than tol_d, using |dD_jk| <= |dmu| sqrt(w_jj w_kk) for the
                            positive semidefinite w = beta d (I - d), with w_jj bounded by
                            its largest diagonal over all rows and w_kk (k a core vertex)
                            over the core rows.  <= 0 selects 1e-11 (FP64) / 1e-6 (split).
                            When a Newton step no longer halves the residual (trace
                            round-off floor) mu is accepted once that bound is within
                            100 tol_d (split precision) or 10 tol_d (FP64).                 */
    int32_t split_small_npad; /* split precision: subgraphs with round16(|S_i|) <= this (0, 16,
                            32, 48 or 64) run in the small configuration, two CTAs per SM,
                            the rest in the 128-column one.  0: all in the 128-column one.
                            gb_plan_autotune picks it.  Results do not depend on it beyond
                            summation order in the core-column refinement.                 */
    double refine_d1;    /* split precision, m > 0, opt-in (<= 0: off): once mu is accepted,
                            every subgraph of at most 1,024 orbitals whose collected D1_r
                            (any r) holds an entry with |D1| above refine_d1 is recomputed
                            in FP64 in its eigenbasis (Eqs. SmallKS, DD, ddlambda, dddmu) at
                            the same mu, and mu_1 is formed from the updated traces.  The
                            split products' D1 error grows with |D1| where states lie within
                            a few kT of mu (measured up to ~4e-5 relative on distorted water
                            at kT 0.1, against ~1e-6 on the equilibrium boxes); 0.3 held
                            every other entry below 6e-6 there.  Each redone subgraph costs
                            an FP64 diagonalisation (~20 ms alone on one SM at 130
                            orbitals), so it suits calls where many subgraphs qualify.
                            Ignored by the FP64 and eigenbasis precisions.                  */
} gb_opts;

typedef struct gb_report {
    int32_t passes;          /* recursion passes taken by the mu iteration                */
    int32_t max_steps;       /* largest per-subgraph step count of the final pass         */
    int32_t n_sub;           /* subgraphs                                                 */
    int32_t max_sub;         /* largest subgraph                                          */
    double mu;               /* final chemical potential                                  */
    double trace_d;          /* sum_i Tr_c d^(i) at mu                                    */
    double dndmu;            /* beta sum_i Tr_c d^(i)(I - d^(i))                          */
    double occ_residual;     /* trace_d - N_occ                                           */
    double trace_d1mu;       /* sum_i Tr_c d1_mu^(i)                                      */
    double eps_min, eps_max; /* Gershgorin bounds over all subgraphs                      */
    double gemm_flops;       /* algorithmic flops of one pass: 2 |S_i|^3 per matrix product,
                                summed over the products the recursion performs            */
    double gemm_flops_per_step_count; /* the same pass counted as 2 |S_i|^3 x s ((2 + 2J)
                                + 3 m) + 2 |S_i|^2 |core_i| (s steps, J Newton-Schulz
                                corrections, m right-hand sides)                           */
    double pass_kernel_ms;   /* device time of the recursion kernel, summed over passes
                                (CUDA events on the handle's stream)                       */
    double mu_d_bound;       /* bound on the change of D the remaining mu step would make
                                (first order; see gb_opts.tol_d)                          */
    int64_t kernel_launches; /* kernels launched by this call                             */
    int32_t refined;         /* subgraphs recomputed in FP64 (gb_opts.refine_d1)          */
    int32_t refine_skipped;  /* subgraphs above the threshold but above 1,024 orbitals,
                                left in split precision                                    */
    double refine_ms;        /* device time of that redo (CUDA events)                    */
} gb_report;

/* ---- handle ------------------------------------------------------------ */
typedef struct gb_handle gb_handle;

/* Create a handle bound to `stream` (a cudaStream_t; NULL = legacy default
 * stream) on the current CUDA device.  *h receives the handle.
 * Errors: GB_ERR_ARG (h NULL), GB_ERR_DEVICE. */
int gb_create(gb_handle** h, void* stream);
int gb_destroy(gb_handle* h);

/* Give the handle `bytes` of caller-owned [device] scratch at `dptr` (256-byte
 * aligned).  The caller keeps ownership and must keep it alive while calls
 * using the handle are in flight. */
int gb_set_workspace(gb_handle* h, void* dptr, size_t bytes);

/* Bytes of workspace the last call that returned GB_ERR_WORKSPACE needed. */
size_t gb_required_workspace(const gb_handle* h);

/* Kernels launched by the most recent call made with this handle. */
int64_t gb_launch_count(const gb_handle* h);

/* Human-readable name of a status code (static string). */
const char* gb_status_string(int status);

/* The CUDA runtime error (cudaError_t value) behind the most recent
 * GB_ERR_DEVICE returned by any call in this process, 0 if none; *name (if
 * non-NULL) receives its name.  Diagnostic only: not thread-safe. */
int gb_last_device_error(const char** name);

/* Library version and the compute capability it was built for (e.g. 103). */
int gb_version(int32_t* major, int32_t* minor, int32_t* arch);

/* ---- gb_graph_build ---------------------------------------------------- *
 * Estimate the data-dependency graph G (Sec. "Estimating the connectivity
 * graph"; the numerically thresholded matrices of Sec. "Numerically
 * thresholded sparse matrix algebra"):
 *   E = {(i,j): i != j, |H_ij| > tau} U {(i,j): i != j, |D_prev,ij| > tau},
 * symmetrised; with paths2 != 0 the paths of length two are added, E <- E U E^2
 * (the paper's favourite estimate with D_prev, or the ad hoc H^2 without).
 *   H       [device] CSR, n x n.
 *   D_prev  [device] collected density of a previous step (gb_csc) or NULL.
 *   tau     strict threshold >= 0.
 *   G       out; G->ptr, G->idx caller-allocated.  If G->capacity is too small
 *           the call returns GB_ERR_CAPACITY with G->nnz = required entries.
 * Output is bit-exact and independent of thread scheduling.
 * Workspace: gb_graph_build_workspace_size(). */
size_t gb_graph_build_workspace_size(int32_t n, int64_t nnz_h, int64_t nnz_dprev, int paths2);
int gb_graph_build(gb_handle* h, const gb_csr* H, const gb_csc* D_prev, double tau,
                   int paths2, gb_graph* G);

/* ---- gb_partition ------------------------------------------------------ *
 * Split G into disjoint cores and distance-1 halos (Fig. 1: the halo is the
 * set of directly connected vertices; Sec. "Choosing the graph partitioning":
 * multi-vertex cores).
 *   group   [device] group id per vertex in [0, n_groups) or NULL.  With
 *           groups, each non-empty group is one core, in ascending group id.
 *           Without, consecutive blocks of target_core_size vertices.
 *   P       out (see gb_part).  GB_ERR_CAPACITY with P->sub_nnz set when
 *           P->sub_capacity is too small.
 * Output is bit-exact.  Synchronises the stream (sizes are returned in P).
 * Workspace: gb_partition_workspace_size() (n_groups <= 0: blocks). */
size_t gb_partition_workspace_size(int32_t n, int64_t nnz_g, int32_t n_groups);
int gb_partition(gb_handle* h, const gb_graph* G, const int32_t* group, int32_t n_groups,
                 int32_t target_core_size, gb_part* P);

/* ---- gb_partition_capped ----------------------------------------------- *
 * gb_partition with group ids, then a size cap on the subgraphs.  The paper
 * leaves the choice of partition free (Sec. "Choosing the graph
 * partitioning"); this rule keeps every subgraph within the tensor-core
 * kernel's 128-row tile when the graph grows (e.g. built from D_prev):
 *   1. cores = one per nonempty group id, as gb_partition (key g);
 *   2. every core whose subgraph S_i holds more than max_sub vertices is
 *      replaced by one core per distinct subgroup id among its vertices
 *      (for example the atoms of a molecule; key n_groups + subgroup);
 *   3. every replacement core still over max_sub is replaced by one core per
 *      vertex (key n_groups + n_subgroups + v);
 *   cores are ordered by ascending key, and halos and S_i follow as in
 *   gb_partition.  A single-vertex core over max_sub is kept (P->max_sub
 *   reports it).
 *   subgroup  [device] int32[n], 0 <= subgroup[v] < n_subgroups; the vertices
 *             of one subgroup should share one group id.
 *   max_sub   cap on |S_i| (> 0).
 * Other arguments, outputs and the capacity protocol are those of
 * gb_partition (GB_ERR_CAPACITY reports the final sub_nnz).  Errors:
 * GB_ERR_ARG (bad sizes, ids out of range, n_groups + n_subgroups + n over
 * INT32_MAX).  Workspace: gb_partition_capped_workspace_size() (0 for
 * invalid sizes).  Synchronises the stream. */
size_t gb_partition_capped_workspace_size(int32_t n, int64_t nnz_g, int32_t n_groups, int32_t n_subgroups);
int gb_partition_capped(gb_handle* h, const gb_graph* G, const int32_t* group, int32_t n_groups,
                        const int32_t* subgroup, int32_t n_subgroups, int32_t max_sub, gb_part* P);

/* ---- gb_partition_noalloc ---------------------------------------------- *
 * The same partition as gb_partition, for callers that cannot allocate device
 * memory: code running inside a host framework that owns every device
 * allocation (a pre-sized memory pool, a plugin with no allocator handle), or
 * code that must not allocate while it runs.  The paper has no counterpart;
 * this is a library convenience.
 *   stream  cudaStream_t (NULL = legacy default stream) on the current device.
 *   Other arguments and the output are those of gb_partition; inputs and
 *   outputs are still the caller's [device] buffers.
 * Scratch: a fixed array compiled into the library
 * (gb_partition_noalloc_scratch_bytes() bytes, about 2.1 MB, held by every
 * GPU that loads the library until the process exits).  It serves at most
 * GB_NOALLOC_MAX_VERTICES vertices and as many groups; larger requests return
 * GB_ERR_WORKSPACE before any work.  The entry point calls no cudaMalloc,
 * cudaFree or other allocating routine.
 * The first call on a device looks up the array's device address on the
 * current device (cudaGetSymbolAddress), and so does the first call after the
 * device's context was created again (cudaDeviceReset); make such a call
 * before any stream capture.  All calls share the one array and it keeps the last call's
 * contents (the call clears what it needs): calls that overlap on the GPU --
 * on different streams, or from different host threads -- race and must be
 * serialised by the caller.  Synchronises the stream. */
#define GB_NOALLOC_MAX_VERTICES 65536
size_t gb_partition_noalloc_scratch_bytes(void);
int gb_partition_noalloc(void* stream, const gb_graph* G, const int32_t* group, int32_t n_groups,
                         int32_t target_core_size, gb_part* P);

/* ---- gb_density_and_response ------------------------------------------- *
 * For every subgraph i: gather h^(i) = H[S_i,S_i] and h1_r^(i) = H1_r[S_i,S_i]
 * (Eq. sub_f), evaluate the Fermi-Dirac density matrix
 *   d^(i) = [exp(beta (h^(i) - mu I)) + I]^-1                       (Eq. Fermi)
 * with one mu shared by all subgraphs, set by Tr[D_G(mu)] = N_occ = Ne/2 with
 * core traces and Newton-Raphson steps (Eq. NewtonRaphson) safeguarded by
 * bisection; the canonical response (Eqs. D1, ddlambda, dddmu, dmu_1)
 *   d1_lambda^(i) = d/dlambda Theta_beta(mu I - h^(i) - lambda h1^(i)),
 *   d1_mu^(i) = beta d^(i) (I - d^(i)),
 *   mu1_r = -sum_i Tr_c d1_lambda^(i) / sum_i Tr_c d1_mu^(i),
 *   D1_r = {d1_lambda^(i)|_c}_collect + mu1_r {d1_mu^(i)|_c}_collect;
 * and collect the core columns into D and D1_r (Eq. dCollect).
 *   H        [host] struct of [device] CSR arrays.
 *   H1       [host] array of m structs of [device] CSR arrays (m >= 0).
 *   kT       electronic temperature in eV, > 0.
 *   n_electrons  Ne; spin-restricted, N_occ = Ne / 2, 0 < N_occ < n.
 *   P        partition from gb_partition (its [device] arrays).
 *   opts     [host] options or NULL for defaults.
 *   mu_inout [host] initial guess on entry (NaN: start from the spectral
 *            bracket), converged mu on return.
 *   D        out, [device] arrays with capacity >= P->out_nnz.
 *   D1       out, [host] array of m gb_csc with [device] val arrays.
 *   mu1      out, [host] array of m doubles (may be NULL when m == 0).
 *   rep      out, [host] report or NULL.
 * The recursion computes d = (I - Z_s)/2 with Z_s = tanh(beta (h - mu)/2) by
 * s doublings Z <- 2 Z (I + Z^2)^-1 from a Taylor start, and d1_lambda by the
 * exact derivative of the same recursion.  Split-precision modes take
 * subgraphs of up to 128 orbitals in one CTA's tensor memory and larger ones
 * (up to 2,048 orbitals, else GB_ERR_UNSUPPORTED) in a tiled kernel whose
 * per-CTA state lives in the workspace; FP64 has no size limit.
 * Errors: GB_ERR_ARG, GB_ERR_CAPACITY, GB_ERR_WORKSPACE, GB_ERR_MU_BRACKET,
 * GB_ERR_NO_CONVERGE (outputs hold the last pass), GB_ERR_NAN, GB_ERR_DEVICE,
 * GB_ERR_UNSUPPORTED, GB_ERR_TIMEOUT.  Synchronises the stream.
 * Workspace: gb_density_workspace_size(). */
int gb_density_workspace_size(const gb_part* P, int32_t m, const gb_opts* opts,
                              size_t* bytes);
int gb_density_and_response(gb_handle* h, const gb_csr* H, const gb_csr* H1, int32_t m,
                            double kT, double n_electrons, const gb_part* P,
                            const gb_opts* opts, double* mu_inout, gb_csc* D, gb_csc* D1,
                            double* mu1, gb_report* rep);

/* ---- gb_mulliken_charges ------------------------------------------------ *
 * Net Mulliken charges of the atoms and their first-order responses from the
 * collected matrices of gb_density_and_response: the charges are the
 * subsystem observables the paper forms from D and D1 (Sec. "Response in
 * observables"; Sec. "Implementation with SCC-DFTB theory", Mulliken charge
 * vectors).  Orthogonal basis, spin restricted (Tr D = N_occ = Ne / 2):
 *   q_I    = Z_I - 2 sum_{o in I} D_oo,
 *   q1_r,I = -2 sum_{o in I} D1_r,oo.
 *   D        [host] struct of the collected D ([device] ptr, idx, val).
 *   D1       [host] array of m collected responses (their val arrays are read;
 *            the structure is D's), m in [0, 8].
 *   n_atoms  atoms; atom_ptr [device] n_atoms + 1 offsets into atom_orb
 *            [device], the orbitals of each atom (each in [0, n)).  Each
 *            atom's sum runs in FP64 over its orbitals in this order, so the
 *            result is deterministic.
 *   z_val    [device] valence charge Z_I per atom.
 *   q        out, [device] n_atoms charges; q1 out, [device] m x n_atoms
 *            (q1[r * n_atoms + I]); may be NULL when m == 0.
 * Errors: GB_ERR_ARG (bad sizes, an orbital out of range, a column without
 * its diagonal), GB_ERR_WORKSPACE (see gb_mulliken_workspace_size).
 * Synchronises the stream. */
size_t gb_mulliken_workspace_size(void);
int gb_mulliken_charges(gb_handle* h, const gb_csc* D, const gb_csc* D1, int32_t m, int32_t n_atoms,
                        const int64_t* atom_ptr, const int32_t* atom_orb, const double* z_val,
                        double* q, double* q1);

/* ---- the charge model of the kernel and its preconditioner -------------- *
 * The extended-Lagrangian electronic equations of motion act on a vector n of
 * atomic electron populations (Sec. "Approximating the kernel"): n changes H
 * through a charge -> potential map C (atoms x atoms),
 *   H[n] = H0 + diag_o((C (n - Z))_atom(o)),
 * the ground state of H[n] at fixed electron count (the graph method) gives
 * populations rho0[n]_I = 2 sum_{o in I} D_oo, and the residual is
 * f(n) = rho0[n] - n with Jacobian J.  Cores must hold whole atoms.
 *
 * gb_blocks: one dense block per subgraph over its core atoms.  [device]
 * arrays sized by the caller: atom_ptr n_sub + 1, atoms n_atoms, val_ptr
 * n_sub + 1, val val_capacity; block k covers atoms[atom_ptr[k] ..
 * atom_ptr[k+1]) (ascending) and is row-major at val[val_ptr[k] ..]. */
typedef struct gb_blocks {
    int32_t n_blocks;       /* out: blocks (= subgraphs)                              */
    int64_t n_atoms_total;  /* out: atoms over all blocks (= n_atoms)                 */
    int64_t val_nnz;        /* out: sum of squared block sizes                        */
    int64_t val_capacity;   /* in: entries val can hold                               */
    int64_t* atom_ptr;
    int32_t* atoms;
    int64_t* val_ptr;
    double* val;
} gb_blocks;

/* ---- gb_preconditioner ---------------------------------------------------- *
 * The subgraph preconditioner K0 = {k0^(k)} (Sec. "Preconditioner for a
 * partitioned graph", Eq. PreCond).  Every subgraph is diagonalised in FP64
 * (as GB_PREC_EIGEN) and mu solved at fixed electron count; then, in the
 * eigenbasis, the responses of the core atoms' populations to a unit charge
 * on each core atom j (H1 = diag_o(C[atom(o), j]) restricted to the
 * subgraph, Eq. ddlambda) and to mu (Eq. dddmu) give
 *   j_c = chi + rho_mu mu1^T - I,
 * with mu1_j chosen per column so that every column of j_c sums to -1 (the
 * core keeps its charge), and k0 = (j_c - alpha I)^-1.
 *   H        [host] struct of [device] CSR, the Hamiltonian the kernel is for.
 *   P, kT, n_electrons  as gb_density_and_response.
 *   C        [host] struct of [device] CSR, atoms x atoms, columns ascending.
 *   orb_atom [device] atom of every orbital (n).
 *   alpha    regularisation >= 0.
 *   mu_inout [host] initial guess (NaN: none), the solved mu on return.
 *   K0       out (see gb_blocks); GB_ERR_CAPACITY with val_nnz set when
 *            val_capacity is too small.
 * Errors: GB_ERR_ARG (sizes, a core not made of whole atoms),
 * GB_ERR_UNSUPPORTED (a subgraph above 1,024 orbitals or a core above 40
 * atoms), GB_ERR_NAN (a singular block), and those of gb_density_and_response.
 * Workspace: gb_preconditioner_workspace_size().  Synchronises the stream. */
size_t gb_preconditioner_workspace_size(const gb_part* P);
int gb_preconditioner(gb_handle* h, const gb_csr* H, const gb_part* P, double kT, double n_electrons,
                      const gb_csr* C, const int32_t* orb_atom, int32_t n_atoms, double alpha,
                      double* mu_inout, gb_blocks* K0);

/* ---- gb_krylov_update ----------------------------------------------------- *
 * One preconditioned low-rank Krylov approximation of the kernel acting on
 * the residual (Sec. "Preconditioned Krylov Subspace Approximation for the
 * electronic equations of motion", steps 1-5; Eqs. LowRankEEOM, Newton_SCF):
 *   f = rho0[n] - n,  v_1 = K0 f / |K0 f|,
 *   f_v_i = K0 (d rho0[n + lambda v_i] / d lambda - v_i)   (graph response to
 *           H1 = diag(C v_i) at fixed electron count, mu_1 included),
 *   v_{i+1} = f_v_i orthonormalised against v_1..v_i (the projection taken
 *           twice); the expansion stops early when the remainder is below
 *           breakdown |f_v_i| (an invariant subspace),
 *   O_ij = f_v_i . f_v_j,  M = O^-1,
 *   dn = -sum_ij v_i M_ij f_v_j . (K0 f)   (the Newton update n - K f).
 *   H0, P, kT, n_electrons, C, orb_atom  as gb_preconditioner.
 *   atom_ptr, atom_orb  [device] the orbitals of each atom (CSR), for rho0.
 *   z, n     [device] reference populations Z and the current n (n_atoms).
 *   K0       [host] struct of [device] blocks from gb_preconditioner, or NULL
 *            for K0 = k0_scalar I.
 *   m        Krylov vectors at most (1..8); breakdown > 0 (e.g. 1e-6).
 *   opts     [host] precision etc. of the density solves (NULL: FP64).
 *   mu_inout [host] initial guess, the ground-state mu of H[n] on return.
 *   f, dn    out, [device] n_atoms each; v, fv out, [device] m x n_atoms
 *            (row i = vector i; rows beyond *rank untouched).
 *   M        out, [host] m x m (the rank x rank inverse, row-major, stride m).
 *   rank     out, [host] vectors used.
 * Errors: those of gb_density_and_response; GB_ERR_ARG (sizes, H0 without a
 * diagonal entry in some row).  Workspace: gb_krylov_workspace_size().
 * Synchronises the stream. */
size_t gb_krylov_workspace_size(const gb_csr* H0, const gb_part* P, int32_t n_atoms, const gb_opts* opts);
int gb_krylov_update(gb_handle* h, const gb_csr* H0, const gb_part* P, double kT, double n_electrons,
                     const gb_csr* C, const int32_t* orb_atom, const int64_t* atom_ptr, const int32_t* atom_orb,
                     int32_t n_atoms, const double* z, const double* n, const gb_blocks* K0, double k0_scalar,
                     int32_t m, double breakdown, const gb_opts* opts, double* mu_inout, double* f, double* v,
                     double* fv, double* dn, double* M, int32_t* rank);

/* ---- gb_plan_autotune ----------------------------------------------------- *
 * Size bins -> kernel configuration for the split-precision recursion.  The
 * subgraphs are binned by npad = round16(|S_i|) (16, 32, ..., 128); those in
 * bins <= split_small_npad run in the small configuration (8 warps, 256 TMEM
 * columns, two CTAs per SM, so one CTA's staging overlaps the other's MMAs),
 * the rest in the 128-column one (12 warps, one CTA per SM).  Candidates are
 * 0 and every bin edge 16..64 that moves at least one subgraph; each is timed
 * as the device time of one recursion pass (CUDA events) at the fixed mu, the
 * second of two passes, with the caller's inputs and output buffers (which
 * hold that pass on return).  The choice is the fastest candidate, the
 * smallest threshold among those within 2% of it: a function of the timing
 * table alone.  The handle caches the last plan by (n_sub, total size, m,
 * precision); a repeated call with the same key returns it without timing.
 *   H, H1, m, kT, n_electrons, P, D, D1: as gb_density_and_response.
 *   opts     [host] options of the calls the plan is for (split precision);
 *            split_small_npad and max_newton are overridden while timing.
 *   mu       fixed chemical potential of the timed passes (eV).
 *   plan     out, [host].
 * Errors: those of gb_density_and_response; GB_ERR_ARG for an FP64 opts. */
#define GB_PLAN_MAX_CAND 5
typedef struct gb_plan {
    int32_t split_small_npad;              /* the choice: pass as gb_opts.split_small_npad  */
    int32_t n_candidates;
    int32_t candidate[GB_PLAN_MAX_CAND];   /* thresholds timed, ascending                  */
    double pass_ms[GB_PLAN_MAX_CAND];      /* recursion device time of one pass            */
    int64_t bin_count[8];                  /* subgraphs with npad = 16 (k + 1)              */
    int32_t cached;                        /* 1: returned from the handle's cache          */
} gb_plan;
int gb_plan_autotune(gb_handle* h, const gb_csr* H, const gb_csr* H1, int32_t m, double kT,
                     double n_electrons, const gb_part* P, const gb_opts* opts, double mu,
                     gb_csc* D, gb_csc* D1, gb_plan* plan);

#ifdef __cplusplus
}
#endif

#endif /* GBQR_H */
