// gb_density_and_response: gather, spectral bounds, the Fermi recursion and
// its response per subgraph, the shared chemical potential, the global mu_1
// and the column collect.
//
// Per subgraph i (h = H[S_i, S_i], Eq. sub_f):
//   d = [exp(beta (h - mu)) + 1]^-1 = (I - Z_s) / 2,  Z_s = tanh(beta (h - mu) / 2)
// from x0 = beta (h - mu) / 2^(s+1) by a Taylor start Z_0 = x0 (1 - x0^2/3 +
// 2 x0^4/15) and s doublings Z <- 2 Z (I + Z^2)^-1 (tanh(2y) = 2 tanh y /
// (1 + tanh^2 y)); the inverse uses the degree-2 Chebyshev start
// X = (98 I - 80 Y + 32 Y^2)/99 (Y = Z^2, spectrum of I + Y in [1, 2]) and
// Newton-Schulz corrections X <- X + X R, R = I - (I + Y) X.
// The grand-canonical response (Eq. ddlambda) is the exact derivative of the
// same recursion along h1: Z1 <- 2 X Z1 X - (1/2) W Z1 W with W = 2 X Z, and
// d1_lambda = -Z1_s / 2;  d1_mu = beta d (I - d) = beta (I - Z_s^2) / 4
// (Eq. dddmu).  mu follows Eq. NewtonRaphson on the core traces, mu_1 Eq. dmu_1.
#include <math.h>
#include <string.h>

#include "density.cuh"

namespace {

constexpr int FP64_THREADS = 256;
constexpr int TS = 32;         // FP64 GEMM tile
constexpr int NBUF = 7;        // work buffers of the FP64 kernel

// ---------------------------------------------------------------------------
// collected-matrix structure: column j holds the rows S_i of its subgraph
// ---------------------------------------------------------------------------
__global__ void k_csc_lengths(int32_t n_sub, const int64_t* sub_ptr, const int64_t* core_ptr,
                              const int32_t* core_idx, int64_t* len) {
    for (int32_t i = blockIdx.x; i < n_sub; i += gridDim.x) {
        int64_t ni = sub_ptr[i + 1] - sub_ptr[i];
        for (int64_t e = core_ptr[i] + threadIdx.x; e < core_ptr[i + 1]; e += blockDim.x)
            len[core_idx[e]] = ni;
    }
}

__global__ void k_csc_rows(int32_t n_sub, const int64_t* sub_ptr, const int32_t* sub_idx,
                           const int64_t* core_ptr, const int32_t* core_idx, const int64_t* col_ptr,
                           int32_t* row_idx) {
    for (int32_t i = blockIdx.x; i < n_sub; i += gridDim.x) {
        const int64_t s0 = sub_ptr[i];
        const int ni = (int)(sub_ptr[i + 1] - s0);
        for (int64_t e = core_ptr[i]; e < core_ptr[i + 1]; ++e) {
            int32_t* dst = row_idx + col_ptr[core_idx[e]];
            for (int r = threadIdx.x; r < ni; r += blockDim.x) dst[r] = sub_idx[s0 + r];
        }
    }
}

__device__ __forceinline__ int lower_bound_i32(const int32_t* a, int n, int32_t v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// input checks and Gershgorin bounds of every principal submatrix
// ---------------------------------------------------------------------------
// (on the exponent bits: no FP64 instruction per element)
// h1_offdiag[0] |= 1 if row i of a perturbation holds an entry off the diagonal
__global__ void k_h1_offdiag(int32_t n, const int64_t* ptr, const int32_t* idx, int* flag) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t p = ptr[i]; p < ptr[i + 1]; ++p) {
        if (idx[p] != i) {
            atomicOr(flag, 1);
            return;
        }
    }
}

__global__ void k_check_finite(int64_t nnz, const double* v, int* err) {
    const unsigned long long* u = (const unsigned long long*)v;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        if ((u[e] & 0x7ff0000000000000ull) == 0x7ff0000000000000ull) set_error(err, GB_ERR_NAN);
}

// Gershgorin interval of every h^(i) = H[S_i, S_i]: the lanes of a warp walk
// one row's non-zeros, the subgraph's vertex list in shared memory when it
// fits.  The radius is summed in FP32 (values converted by integer
// operations) and widened by 2^-16, which covers the conversions and the
// rounding of up to 2^15 terms: the interval stays an enclosure.  Diagonal
// and interval ends stay FP64, but the FP64 work is done once per 32 rows
// (lane k finishes row k of its warp's batch): GB300's FP64 pipe is narrow.
constexpr int GERSH_THREADS = 128;
constexpr int GERSH_SMEM_N = 2048;
__global__ void __launch_bounds__(GERSH_THREADS) k_gershgorin(int32_t n_sub, const int64_t* sub_ptr,
                                                              const int32_t* sub_idx, const int64_t* Hptr,
                                                              const int32_t* Hidx, const double* Hval,
                                                              double* eps_lo, double* eps_hi) {
    __shared__ int32_t Ss[GERSH_SMEM_N];
    __shared__ double wlo[GERSH_THREADS / 32], whi[GERSH_THREADS / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = GERSH_THREADS / 32;
    for (int32_t i = blockIdx.x; i < n_sub; i += gridDim.x) {
        const int n = (int)(sub_ptr[i + 1] - sub_ptr[i]);
        const int32_t* S = sub_idx + sub_ptr[i];
        if (n <= GERSH_SMEM_N) {
            for (int r = threadIdx.x; r < n; r += GERSH_THREADS) Ss[r] = S[r];
            S = Ss;
        }
        __syncthreads();
        double lo = INFINITY, hi = -INFINITY;
        for (int rb = warp * 32; rb < n; rb += nw * 32) {
            float my_rad = 0.f;
            uint32_t my_dhi = 0u, my_dlo = 0u;  // bits of row (rb + lane)'s diagonal
            const int kn = min(32, n - rb);
            for (int k = 0; k < kn; ++k) {
                const int r = rb + k;
                const int32_t g = S[r];
                float rad = 0.f;
                bool has = false;
                uint32_t dhi = 0u, dlo = 0u;
                for (int64_t p = Hptr[g] + lane; p < Hptr[g + 1]; p += 32) {
                    const int32_t c = Hidx[p];
                    const int lc = lower_bound_i32(S, n, c);
                    if (lc < n && S[lc] == c) {
                        if (lc == r) {
                            const unsigned long long b = (unsigned long long)__double_as_longlong(Hval[p]);
                            dhi = (uint32_t)(b >> 32);
                            dlo = (uint32_t)b;
                            has = true;
                        } else {
                            rad += fabsf(d2f_rn(Hval[p]));
                        }
                    }
                }
                for (int o = 16; o > 0; o >>= 1) rad += __shfl_xor_sync(0xffffffffu, rad, o);
                const uint32_t bal = __ballot_sync(0xffffffffu, has);
                const int src = bal ? __ffs(bal) - 1 : 0;
                dhi = __shfl_sync(0xffffffffu, dhi, src);
                dlo = __shfl_sync(0xffffffffu, dlo, src);
                if (lane == k) {
                    my_rad = rad;
                    my_dhi = bal ? dhi : 0u;
                    my_dlo = bal ? dlo : 0u;
                }
            }
            if (lane < kn) {
                const double diag = __longlong_as_double((long long)(((unsigned long long)my_dhi << 32) | my_dlo));
                const double rd = (double)my_rad * (1.0 + 0x1p-16);
                lo = fmin(lo, diag - rd);
                hi = fmax(hi, diag + rd);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            wlo[warp] = lo;
            whi[warp] = hi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < nw; ++w) {
                lo = fmin(lo, wlo[w]);
                hi = fmax(hi, whi[w]);
            }
            eps_lo[i] = lo;
            eps_hi[i] = hi;
        }
        __syncthreads();
    }
}

// Reduction in a fixed order (deterministic): sums of the per-subgraph trace
// slots, min of eps_lo and max of eps_hi.  Block b takes the fixed range
// [b chunk, (b + 1) chunk) of subgraphs; within it thread t owns a fixed
// contiguous sub-range and accumulates every quantity in one sweep, the
// threads' partials combine by a fixed tree into partial[b][q], and
// k_reduce_final adds the blocks' partials in block order.  (The FP64 work is
// spread over the SMs: one block measured ~70 us a call.)
constexpr int REDUCE_THREADS = 256;  // (stride + 2) x 256 doubles <= 30 KB of shared memory
constexpr int REDUCE_BLOCKS = 160;
constexpr int REDUCE_MAXQ = TR_FIXED + GB_MAX_RHS + 2;
__global__ void __launch_bounds__(REDUCE_THREADS) k_reduce(int32_t n_sub, int32_t stride, const double* tr,
                                                           const double* eps_lo, const double* eps_hi,
                                                           double* partial) {
    extern __shared__ double sh[];  // [stride + 2][REDUCE_THREADS]
    const int nq = stride + 2;
    const int t = threadIdx.x;
    const int32_t chunk = (n_sub + (int32_t)gridDim.x - 1) / (int32_t)gridDim.x;
    const int32_t b0 = min(n_sub, (int32_t)blockIdx.x * chunk), b1 = min(n_sub, b0 + chunk);
    const int32_t per = (b1 - b0 + REDUCE_THREADS - 1) / REDUCE_THREADS;
    const int32_t i0 = min(b1, b0 + t * per), i1 = min(b1, i0 + per);
    double v[REDUCE_MAXQ];
#pragma unroll
    for (int k = 0; k < REDUCE_MAXQ; ++k) v[k] = 0.0;
    v[TR_MAXW] = -INFINITY;
    v[TR_MAXWC] = -INFINITY;
    double lo = INFINITY, hi = -INFINITY;
    for (int32_t i = i0; i < i1; ++i) {
        const double* row = tr + (int64_t)i * stride;
#pragma unroll
        for (int k = 0; k < REDUCE_MAXQ - 2; ++k) {
            if (k < stride) v[k] = trace_slot_is_max(k) ? fmax(v[k], row[k]) : v[k] + row[k];
        }
        lo = fmin(lo, eps_lo[i]);
        hi = fmax(hi, eps_hi[i]);
    }
#pragma unroll
    for (int k = 0; k < REDUCE_MAXQ - 2; ++k)
        if (k < stride) sh[k * REDUCE_THREADS + t] = v[k];
    sh[stride * REDUCE_THREADS + t] = lo;
    sh[(stride + 1) * REDUCE_THREADS + t] = hi;
    __syncthreads();
    for (int o = REDUCE_THREADS / 2; o > 0; o >>= 1) {
        if (t < o) {
            for (int k = 0; k < nq; ++k) {
                const double a = sh[k * REDUCE_THREADS + t], b = sh[k * REDUCE_THREADS + t + o];
                const int op = k < stride ? (trace_slot_is_max(k) ? 2 : 0) : (k == stride ? 1 : 2);  // sum, min, max
                sh[k * REDUCE_THREADS + t] = op == 0 ? a + b : (op == 1 ? fmin(a, b) : fmax(a, b));
            }
        }
        __syncthreads();
    }
    if (t < nq) partial[(int64_t)blockIdx.x * nq + t] = sh[t * REDUCE_THREADS];
}

__global__ void k_reduce_final(int32_t nblocks, int32_t stride, const double* partial, double* sums,
                               double* bounds) {
    const int nq = stride + 2;
    const int k = threadIdx.x;
    if (k >= nq) return;
    const int op = k < stride ? (trace_slot_is_max(k) ? 2 : 0) : (k == stride ? 1 : 2);  // sum, min, max
    double v = partial[k];
    for (int32_t b = 1; b < nblocks; ++b) {
        const double x = partial[(int64_t)b * nq + k];
        v = op == 0 ? v + x : (op == 1 ? fmin(v, x) : fmax(v, x));
    }
    if (k < stride) sums[k] = v;
    else bounds[k - stride] = v;
}

// The subgraphs of the three size classes of the split launches, each list
// in ascending order, class k at work[k n_sub, k n_sub + work_n[k]):
// k = 0: small < round16(|S_i|) <= 128 (the 128-column configuration),
// k = 1: round16(|S_i|) <= small (the small configuration),
// k = 2: round16(|S_i|) > 128 (the tiled configuration).
// One block; thread t takes a fixed contiguous range, offsets by a block scan.
constexpr int CLASS_THREADS = 1024;
__device__ __forceinline__ int size_class(int64_t n, int32_t small) {
    const int64_t np = (n + 15) & ~(int64_t)15;
    return np > GB_SPLIT_MAX_N ? 2 : (np <= small ? 1 : 0);
}
__global__ void __launch_bounds__(CLASS_THREADS) k_class_lists(int32_t n_sub, const int64_t* sub_ptr,
                                                               int32_t small, int32_t* work, int32_t* work_n) {
    __shared__ int32_t wsum[3][CLASS_THREADS / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int32_t per = (n_sub + CLASS_THREADS - 1) / CLASS_THREADS;
    const int32_t i0 = min(n_sub, t * per), i1 = min(n_sub, i0 + per);
    int32_t cnt[3] = {0, 0, 0};
    for (int32_t i = i0; i < i1; ++i) ++cnt[size_class(sub_ptr[i + 1] - sub_ptr[i], small)];
    int32_t incl[3];
    for (int k = 0; k < 3; ++k) {
        int32_t v = cnt[k];
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        incl[k] = v;
        if (lane == 31) wsum[k][warp] = v;
    }
    __syncthreads();
    int32_t pos[3], tot[3];
    for (int k = 0; k < 3; ++k) {
        int32_t b = 0, tt = 0;
        for (int w = 0; w < CLASS_THREADS / 32; ++w) {
            const int32_t v = wsum[k][w];
            b += w < warp ? v : 0;
            tt += v;
        }
        pos[k] = b + incl[k] - cnt[k];
        tot[k] = tt;
    }
    for (int32_t i = i0; i < i1; ++i) {
        const int k = size_class(sub_ptr[i + 1] - sub_ptr[i], small);
        work[(int64_t)k * n_sub + pos[k]++] = i;
    }
    if (t == 0)
        for (int k = 0; k < 3; ++k) work_n[k] = tot[k];
}

// Subgraphs whose collected response holds an entry |d1_lambda_r + mu1_r
// d1_mu| above thr (at most max_n orbitals: into list; larger: counted apart).
struct Mu1s {
    double v[GB_MAX_RHS];
};
__global__ void __launch_bounds__(256) k_flag_refine(PassArgs a, Mu1s mu1, double thr, int max_n, int32_t* list,
                                                     int32_t* count) {
    for (int32_t i = blockIdx.x; i < a.n_sub; i += gridDim.x) {
        const int n = (int)(a.sub_ptr[i + 1] - a.sub_ptr[i]);
        const int64_t c0 = a.core_ptr[i], nq = (a.core_ptr[i + 1] - c0) * n;
        bool big = false;
        for (int64_t q = threadIdx.x; q < nq && !big; q += blockDim.x) {
            const int64_t o = a.col_ptr[a.core_idx[c0 + q / n]] + q % n;
            const double w = a.d1mu_val[o];
            for (int r = 0; r < a.m; ++r) big |= fabs(a.D1val[r][o] + mu1.v[r] * w) > thr;
        }
        if (__syncthreads_or(big) && threadIdx.x == 0) {
            if (n <= max_n) list[atomicAdd(&count[0], 1)] = i;
            else atomicAdd(&count[1], 1);
        }
    }
}

__global__ void k_d1_fixup(int64_t nnz, double mu1, const double* d1mu, double* d1) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        d1[e] += mu1 * d1mu[e];
}

// ---------------------------------------------------------------------------
// FP64 path: one block per subgraph, dense n x n blocks in global memory
// ---------------------------------------------------------------------------
struct GemmSmem {
    double a[TS][TS + 1];
    double b[TS][TS + 1];
};

// C = alpha A B + beta C0 + gamma I  (row-major n x n; C must not alias A, B;
// C0 may alias C).
__device__ void dgemm(int n, double alpha, const double* A, const double* B, double beta,
                      const double* C0, double gamma, double* C, GemmSmem& sm) {
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int nt = (n + TS - 1) / TS;
    for (int tile = 0; tile < nt * nt; ++tile) {
        const int r0 = (tile / nt) * TS, c0 = (tile % nt) * TS;
        double acc00 = 0.0, acc01 = 0.0, acc10 = 0.0, acc11 = 0.0;
        for (int k0 = 0; k0 < n; k0 += TS) {
            for (int e = tid; e < TS * TS; e += FP64_THREADS) {
                const int rr = e / TS, kk = e % TS;
                sm.a[rr][kk] = (r0 + rr < n && k0 + kk < n) ? A[(int64_t)(r0 + rr) * n + k0 + kk] : 0.0;
                sm.b[rr][kk] = (k0 + rr < n && c0 + kk < n) ? B[(int64_t)(k0 + rr) * n + c0 + kk] : 0.0;
            }
            __syncthreads();
#pragma unroll 8
            for (int kk = 0; kk < TS; ++kk) {
                const double a0 = sm.a[ty][kk], a1 = sm.a[ty + 16][kk];
                const double b0 = sm.b[kk][tx], b1 = sm.b[kk][tx + 16];
                acc00 = fma(a0, b0, acc00);
                acc01 = fma(a0, b1, acc01);
                acc10 = fma(a1, b0, acc10);
                acc11 = fma(a1, b1, acc11);
            }
            __syncthreads();
        }
        const double acc[2][2] = {{acc00, acc01}, {acc10, acc11}};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int r = r0 + ty + 16 * a, c = c0 + tx + 16 * b;
                if (r < n && c < n) {
                    const int64_t o = (int64_t)r * n + c;
                    double v = alpha * acc[a][b];
                    if (beta != 0.0) v += beta * C0[o];
                    if (r == c) v += gamma;
                    C[o] = v;
                }
            }
    }
    __syncthreads();
}

// out = scale * (M[S, S] - shift I), M given in CSR
__device__ void gather_scaled(int n, const int32_t* S, const int64_t* ptr, const int32_t* idx,
                              const double* val, double scale, double shift, double* out) {
    for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) out[e] = 0.0;
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const int32_t g = S[r];
        for (int64_t p = ptr[g]; p < ptr[g + 1]; ++p) {
            const int32_t c = idx[p];
            const int lc = lower_bound_i32(S, n, c);
            if (lc < n && S[lc] == c) out[(int64_t)r * n + lc] = scale * val[p];
        }
        out[(int64_t)r * n + r] -= scale * shift;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(FP64_THREADS) k_fermi_fp64(PassArgs a) {
    __shared__ GemmSmem sm;
    __shared__ double red[FP64_THREADS];
    for (int32_t i = blockIdx.x; i < a.n_sub; i += gridDim.x) {
        const int64_t s0 = a.sub_ptr[i];
        const int n = (int)(a.sub_ptr[i + 1] - s0);
        const int32_t* S = a.sub_idx + s0;
        const int64_t base = a.moff[i];
        double* B[NBUF];
#pragma unroll
        for (int k = 0; k < NBUF; ++k) B[k] = a.pool + (int64_t)k * a.pool_stride + base;
        double* Z1[GB_MAX_RHS];
        for (int r = 0; r < a.m; ++r) Z1[r] = a.pool + (int64_t)(NBUF + r) * a.pool_stride + base;

        int s = recursion_steps(a.beta, a.mu, a.eps_lo[i], a.eps_hi[i], a.min_steps);
        double alpha = ldexp(a.beta, -(s + 1));
        double *x0 = B[0], *Q = B[1], *P = B[2], *Z = B[3];
        // Taylor start: Z0 = x0 (I - Q/3 + 2 Q^2/15), Q = x0^2
        gather_scaled(n, S, a.Hptr, a.Hidx, a.Hval, alpha, a.mu, x0);
        dgemm(n, 1.0, x0, x0, 0.0, nullptr, 0.0, Q, sm);
        {
            // rho(x0)^2 <= max_r sum_c |Q_rc|: drop k steps while 2^k x0 stays
            // within spectral radius 1 (x0 scales by 2^k, Q by 4^k, exactly)
            double rs = 0.0;
            for (int r = threadIdx.x; r < n; r += blockDim.x) {
                double t = 0.0;
                for (int c = 0; c < n; ++c) t += fabs(Q[(int64_t)r * n + c]);
                rs = fmax(rs, t);
            }
            red[threadIdx.x] = rs;
            __syncthreads();
            for (int o = blockDim.x / 2; o > 0; o >>= 1) {
                if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
                __syncthreads();
            }
            const double qmax = red[0];
            __syncthreads();
            int k = 0;
            while (k < s - a.min_steps && qmax * ldexp(1.0, 2 * (k + 1)) <= 1.0) ++k;
            if (k > 0) {
                s -= k;
                alpha = ldexp(a.beta, -(s + 1));
                const double f1 = ldexp(1.0, k), f2 = ldexp(1.0, 2 * k);
                for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
                    x0[e] *= f1;
                    Q[e] *= f2;
                }
                __syncthreads();
            }
        }
        dgemm(n, 2.0 / 15.0, Q, Q, -1.0 / 3.0, Q, 1.0, P, sm);
        dgemm(n, 1.0, x0, P, 0.0, nullptr, 0.0, Z, sm);
        for (int r = 0; r < a.m; ++r) {
            // dZ0 = X1 P + x0 P1,  P1 = -Q1/3 + (2/15)(Q Q1 + Q1 Q),  Q1 = x0 X1 + X1 x0
            double *X1 = B[4], *Q1 = B[5], *P1 = B[6];
            gather_scaled(n, S, a.H1ptr[r], a.H1idx[r], a.H1val[r], alpha, 0.0, X1);
            dgemm(n, 1.0, x0, X1, 0.0, nullptr, 0.0, Q1, sm);
            dgemm(n, 1.0, X1, x0, 1.0, Q1, 0.0, Q1, sm);
            dgemm(n, 2.0 / 15.0, Q, Q1, -1.0 / 3.0, Q1, 0.0, P1, sm);
            dgemm(n, 2.0 / 15.0, Q1, Q, 1.0, P1, 0.0, P1, sm);
            dgemm(n, 1.0, X1, P, 0.0, nullptr, 0.0, Z1[r], sm);
            dgemm(n, 1.0, x0, P1, 1.0, Z1[r], 0.0, Z1[r], sm);
        }
        double *Y = B[0], *Y2 = B[1], *X = B[2], *R = B[4], *Xn = B[5], *W = B[6];
        for (int step = 0; step < s; ++step) {
            dgemm(n, 1.0, Z, Z, 0.0, nullptr, 0.0, Y, sm);
            // X0 = (98 I - 80 Y + 32 Y^2) / 99
            dgemm(n, 32.0 / 99.0, Y, Y, -80.0 / 99.0, Y, 98.0 / 99.0, X, sm);
            for (int j = 0; j < a.ns_iters; ++j) {
                dgemm(n, -1.0, Y, X, -1.0, X, 1.0, R, sm);      // R = I - X - Y X
                dgemm(n, 1.0, X, R, 1.0, X, 0.0, Xn, sm);       // X + X R
                double* t = X; X = Xn; Xn = t;
            }
            dgemm(n, 2.0, X, Z, 0.0, nullptr, 0.0, W, sm);      // W = 2 X Z
            for (int r = 0; r < a.m; ++r) {
                double *A1 = R, *T = Y2;
                dgemm(n, 1.0, X, Z1[r], 0.0, nullptr, 0.0, A1, sm);
                dgemm(n, 2.0, A1, X, 0.0, nullptr, 0.0, T, sm);      // 2 X Z1 X
                dgemm(n, 1.0, W, Z1[r], 0.0, nullptr, 0.0, A1, sm);  // W Z1
                dgemm(n, -0.5, A1, W, 1.0, T, 0.0, Z1[r], sm);       // - W Z1 W / 2
            }
            double* t = Z; Z = W; W = t;
        }
        dgemm(n, 1.0, Z, Z, 0.0, nullptr, 0.0, Y, sm);  // Z_s^2 for d (I - d)

        // core columns -> collected CSC positions, and core traces
        const int64_t c0 = a.core_ptr[i], c1 = a.core_ptr[i + 1];
        for (int64_t e = c0; e < c1; ++e) {
            const int kc = a.core_pos[e];
            const int64_t o = a.col_ptr[a.core_idx[e]];
            for (int r = threadIdx.x; r < n; r += blockDim.x) {
                const double id = (r == kc) ? 1.0 : 0.0;
                const double dv = 0.5 * (id - Z[(int64_t)r * n + kc]);
                const double mv = 0.25 * a.beta * (id - Y[(int64_t)r * n + kc]);
                if (!isfinite(dv) || !isfinite(mv)) set_error(a.err, GB_ERR_NAN);
                a.Dval[o + r] = dv;
                a.d1mu_val[o + r] = mv;
                for (int q = 0; q < a.m; ++q) a.D1val[q][o + r] = -0.5 * Z1[q][(int64_t)r * n + kc];
            }
        }
        for (int slot = 0; slot < TR_FIXED + a.m; ++slot) {
            double v = 0.0;
            for (int64_t e = c0 + threadIdx.x; e < c1; e += blockDim.x) {
                const int64_t kk = (int64_t)a.core_pos[e] * (n + 1);
                if (slot == TR_D) v += 0.5 * (1.0 - Z[kk]);
                else if (slot == TR_DD) v += 0.25 * (1.0 - Y[kk]);
                else if (slot == TR_D1MU) v += 0.25 * a.beta * (1.0 - Y[kk]);
                else if (slot >= TR_D1LAM) v += -0.5 * Z1[slot - TR_D1LAM][kk];
            }
            if (slot == TR_FLOPS && threadIdx.x == 0) v = pass_gemm_flops(n, s, a.ns_iters, a.m);
            if (slot == TR_FLOPS_S && threadIdx.x == 0)
                v = pass_flops_per_step_count(n, (int)(c1 - c0), s, a.ns_iters, a.m);
            if (slot == TR_MAXW)
                for (int r = threadIdx.x; r < n; r += blockDim.x)
                    v = fmax(v, 0.25 * a.beta * (1.0 - Y[(int64_t)r * (n + 1)]));
            if (slot == TR_MAXWC)
                for (int64_t e = c0 + threadIdx.x; e < c1; e += blockDim.x)
                    v = fmax(v, 0.25 * a.beta * (1.0 - Y[(int64_t)a.core_pos[e] * (n + 1)]));
            red[threadIdx.x] = v;
            __syncthreads();
            for (int o = blockDim.x / 2; o > 0; o >>= 1) {
                if (threadIdx.x < o)
                    red[threadIdx.x] = trace_slot_is_max(slot) ? fmax(red[threadIdx.x], red[threadIdx.x + o])
                                                       : red[threadIdx.x] + red[threadIdx.x + o];
                __syncthreads();
            }
            if (threadIdx.x == 0) a.tr[(int64_t)i * a.tr_stride + slot] = red[0];
            __syncthreads();
        }
        if (threadIdx.x == 0) a.steps_out[i] = s;
        __syncthreads();
    }
}

// sq[i] = n_i^2 (or npad_i^2 with npad = round16(n_i)), scanned afterwards
__global__ void k_block_sizes(int32_t n_sub, const int64_t* sub_ptr, int64_t* sq, int pad16) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_sub) {
        int64_t ni = sub_ptr[i + 1] - sub_ptr[i];
        if (pad16) ni = (ni + 15) & ~(int64_t)15;
        sq[i] = ni * ni;
    }
}

struct DensityLayout {
    int64_t* moff;      // n_sub + 1
    double* eps_lo;     // n_sub
    double* eps_hi;     // n_sub
    int32_t* steps;     // n_sub
    double* tr;         // n_sub * (TR_FIXED + m)
    double* sums;       // TR_FIXED + m
    double* partial;    // REDUCE_BLOCKS x (TR_FIXED + m + 2): k_reduce's per-block results
    double* bounds;     // 2
    double* d1mu_val;   // out_nnz
    int64_t* scan_tmp;
    int* err;
    double* pool;       // FP64: (NBUF + m) * pool_stride
    float* z1pool;      // split: min(n_sub, GB_SPLIT_MAX_CTAS) x m x 64 KB: staged Z1 images, per CTA
    float* hblk;        // split: (1 + m) * pool_stride dense gathered blocks (FP32)
    double* hdiag;      // split: sub_nnz FP64 diagonals of h^(i)
    double* h1max;      // split: n_sub * m largest |h1| row sums
    float* h1d;         // split, m > 0: m * sub_nnz diagonals of beta h1 (diagonal H1)
    int* h1flag;        // split: set when some H1_r has an off-diagonal entry
    int32_t* work;      // split: subgraph lists of the three size classes (3 x n_sub)
    int32_t* work_n;    // split: their lengths (3) and the tiled launch's work counter
    uint8_t* big;       // split, |S_i| > 128: per-CTA scratch of the tiled kernel
    int64_t big_stride; // bytes per CTA
    int32_t big_ctas;   // CTAs the scratch serves
    int32_t big_npmax;  // round16(max |S_i|)
    double* eig_scratch;  // eigen: per-CTA scratch (3 max_sub^2 doubles each)
    int64_t eig_stride;
    double* eig_eps;      // eigen: eigenvalues and core weights (sub_nnz each)
    double* eig_w;
    int32_t* eig_counter;
    // split, m > 0: the FP64 redo of subgraphs with a large response
    // (gb_opts.refine_d1): their list and counts, and ref_slots eigenvector
    // slots of ref_me^2 doubles (ref_me = min(max |S_i|, GB_EIG_MAX_N)); the
    // eig_* fields above serve it too
    int32_t* ref_list;
    int32_t* ref_n;
    double* ref_vt;
    int32_t ref_slots;
    int32_t ref_me;
    int64_t pool_stride;
};

// CTAs of the tiled kernel: one per SM at most, within a scratch budget
constexpr int64_t BIG_SCRATCH_BUDGET = (int64_t)24 << 30;
// eigenvector slots and scratch of the FP64 redo (gb_opts.refine_d1)
constexpr int64_t REFINE_BUDGET = (int64_t)1 << 30;

DensityLayout layout_density(Arena& ar, const gb_part* P, int32_t m, int precision) {
    DensityLayout L;
    const int64_t n_sub = P->n_sub;
    L.moff = ar.take<int64_t>(n_sub + 1);
    L.eps_lo = ar.take<double>(n_sub);
    L.eps_hi = ar.take<double>(n_sub);
    L.steps = ar.take<int32_t>(n_sub);
    L.tr = ar.take<double>(n_sub * (TR_FIXED + m));
    L.sums = ar.take<double>(TR_FIXED + m + 8);
    L.partial = ar.take<double>((int64_t)REDUCE_BLOCKS * (TR_FIXED + m + 2));
    L.bounds = ar.take<double>(8);
    L.d1mu_val = ar.take<double>(P->out_nnz);
    L.scan_tmp = ar.take<int64_t>(scan_temp_count(n_sub + 1) + 64);
    L.err = ar.take<int>(8);
    L.eig_scratch = nullptr;
    L.eig_stride = 0;
    L.eig_eps = L.eig_w = nullptr;
    L.eig_counter = nullptr;
    L.ref_list = L.ref_n = nullptr;
    L.ref_vt = nullptr;
    L.ref_slots = L.ref_me = 0;
    if (precision == GB_PREC_EIGEN) {
        // eigenvectors of every subgraph (sum_i n_i^2 <= max_sub * sum_i n_i),
        // eigenvalues, core weights, and the per-CTA scratch of the kernels
        L.pool_stride = ((int64_t)P->max_sub * P->sub_nnz + 32 + 63) & ~(int64_t)63;
        L.pool = ar.take<double>(L.pool_stride);
        L.eig_eps = ar.take<double>(P->sub_nnz);
        L.eig_w = ar.take<double>(P->sub_nnz);
        L.eig_stride = 3 * (int64_t)P->max_sub * P->max_sub + GB_PRECOND_SCRATCH;
        const int64_t ctas = n_sub < GB_EIG_MAX_CTAS ? n_sub : GB_EIG_MAX_CTAS;
        L.eig_scratch = ar.take<double>(ctas * L.eig_stride);
        L.eig_counter = ar.take<int32_t>(8);
        L.z1pool = nullptr;
        L.work = nullptr;
        L.work_n = nullptr;
        L.hblk = nullptr;
        L.hdiag = nullptr;
        L.h1max = nullptr;
        L.h1d = nullptr;
        L.h1flag = nullptr;
        L.big = nullptr;
    } else if (precision == GB_PREC_FP64) {
        // sum_i n_i^2 <= max_sub * sum_i n_i
        L.pool_stride = ((int64_t)P->max_sub * P->sub_nnz + 32 + 63) & ~(int64_t)63;
        L.pool = ar.take<double>((NBUF + m) * L.pool_stride);
        L.z1pool = nullptr;
        L.work = nullptr;
        L.work_n = nullptr;
        L.hblk = nullptr;
        L.hdiag = nullptr;
        L.h1max = nullptr;
        L.h1d = nullptr;
        L.h1flag = nullptr;
    } else {
        // sum_i round16(n_i)^2 <= (max_sub + 15) * (sum_i n_i + 15 n_sub)
        // (a multiple of 64 elements: every block stays 16-byte aligned for the
        // vector loads of the staging code)
        L.pool_stride = (((int64_t)P->max_sub + 15) * (P->sub_nnz + 15 * n_sub) + 32 + 63) & ~(int64_t)63;
        L.pool = nullptr;
        const int64_t ctas = n_sub < GB_SPLIT_MAX_CTAS ? n_sub : GB_SPLIT_MAX_CTAS;
        L.z1pool = ar.take<float>(ctas * (int64_t)(m > 0 ? m : 1) * GB_SPLIT_MAX_N * GB_SPLIT_MAX_N);
        L.hblk = ar.take<float>((1 + m) * L.pool_stride);
        L.hdiag = ar.take<double>(P->sub_nnz);
        L.h1max = ar.take<double>(n_sub * (int64_t)(m > 0 ? m : 1));
        L.h1d = ar.take<float>((int64_t)(m > 0 ? m : 1) * P->sub_nnz);
        L.h1flag = ar.take<int>(4);
        L.work = ar.take<int32_t>(3 * n_sub);
        L.work_n = ar.take<int32_t>(8);
        L.big = nullptr;
        L.big_stride = 0;
        L.big_ctas = 0;
        L.big_npmax = 0;
        if (P->max_sub > GB_SPLIT_MAX_N) {
            L.big_npmax = (P->max_sub + 15) & ~15;
            L.big_stride = (big_cta_bytes(L.big_npmax, m) + 255) & ~(int64_t)255;
            int64_t ctas = n_sub < GB_BIG_MAX_CTAS ? n_sub : GB_BIG_MAX_CTAS;
            const int64_t fit = BIG_SCRATCH_BUDGET / L.big_stride;
            if (ctas > fit) ctas = fit > 0 ? fit : 1;
            L.big_ctas = (int32_t)ctas;
            L.big = ar.take<uint8_t>((size_t)(ctas * L.big_stride));
        }
        if (m > 0) {
            const int64_t me = P->max_sub < GB_EIG_MAX_N ? P->max_sub : GB_EIG_MAX_N;
            int64_t slots = REFINE_BUDGET / (4 * me * me * (int64_t)sizeof(double));
            if (slots > GB_EIG_MAX_CTAS) slots = GB_EIG_MAX_CTAS;
            if (slots > n_sub) slots = n_sub;
            if (slots < 1) slots = 1;
            L.ref_me = (int32_t)me;
            L.ref_slots = (int32_t)slots;
            L.ref_list = ar.take<int32_t>(n_sub);
            L.ref_n = ar.take<int32_t>(8);
            L.eig_eps = ar.take<double>(P->sub_nnz);
            L.eig_w = ar.take<double>(P->sub_nnz);
            L.eig_stride = 3 * me * me;
            L.eig_scratch = ar.take<double>(slots * L.eig_stride);
            L.ref_vt = ar.take<double>(slots * me * me);
            L.eig_counter = ar.take<int32_t>(8);
        }
    }
    return L;
}

}  // namespace

// the two launches of the deterministic trace / bound reduction
static int reduce_traces(gb_handle* h, int32_t n_sub, int32_t stride, const DensityLayout& L) {
    const int nb = n_sub < REDUCE_BLOCKS ? n_sub : REDUCE_BLOCKS;
    GB_LAUNCH(h, k_reduce, nb, REDUCE_THREADS, sizeof(double) * (stride + 2) * REDUCE_THREADS, n_sub, stride,
              (const double*)L.tr, (const double*)L.eps_lo, (const double*)L.eps_hi, L.partial);
    GB_LAUNCH(h, k_reduce_final, 1, 32, 0, nb, stride, (const double*)L.partial, L.sums, L.bounds);
    return GB_OK;
}

// The eigenbasis state the last GB_PREC_EIGEN call with this partition and m
// left in the handle's workspace (eigenvectors, eigenvalues, core weights, the
// per-CTA scratch), as the kernels' arguments at chemical potential mu.
int eigen_state(gb_handle* h, const gb_part* P, int32_t m, double kT, double mu, EigArgs* out,
                size_t* density_bytes) {
    Arena ar(h->ws, h->ws_bytes);
    DensityLayout L = layout_density(ar, P, m, GB_PREC_EIGEN);
    if (!ar.fits() || !h->ws) return GB_ERR_WORKSPACE;
    *density_bytes = ar.used();
    memset(out, 0, sizeof(*out));
    PassArgs& a = out->a;
    a.n_sub = P->n_sub;
    a.m = m;
    a.sub_ptr = P->sub_ptr;
    a.sub_idx = P->sub_idx;
    a.core_ptr = P->core_ptr;
    a.core_idx = P->core_idx;
    a.core_pos = P->core_pos;
    a.beta = 1.0 / kT;
    a.mu = mu;
    a.moff = L.moff;
    a.tr = L.tr;
    a.err = L.err;
    out->scratch = L.eig_scratch;
    out->scratch_stride = L.eig_stride;
    out->eps = L.eig_eps;
    out->w = L.eig_w;
    out->vt = L.pool;
    out->counter = L.eig_counter;
    return GB_OK;
}

extern "C" int gb_density_workspace_size(const gb_part* P, int32_t m, const gb_opts* opts,
                                         size_t* bytes) {
    if (!P || !bytes || m < 0 || m > GB_MAX_RHS || P->n_sub <= 0) return GB_ERR_ARG;
    int precision = opts ? opts->precision : GB_PREC_FP64;
    Arena a;
    layout_density(a, P, m, precision);
    *bytes = a.used();
    return GB_OK;
}

static bool csr_ok(const gb_csr* A, int32_t n) {
    return A && A->n == n && A->ptr && A->nnz >= 0 && (A->nnz == 0 || (A->idx && A->val));
}

extern "C" int gb_density_and_response(gb_handle* h, const gb_csr* H, const gb_csr* H1, int32_t m,
                                       double kT, double n_electrons, const gb_part* P,
                                       const gb_opts* opts, double* mu_inout, gb_csc* D, gb_csc* D1,
                                       double* mu1, gb_report* rep) {
    if (!h || !P || !mu_inout || !D) return GB_ERR_ARG;
    const int32_t n = P->n;
    if (!csr_ok(H, n) || m < 0 || m > GB_MAX_RHS || (m > 0 && (!H1 || !D1 || !mu1))) return GB_ERR_ARG;
    for (int r = 0; r < m; ++r)
        if (!csr_ok(&H1[r], n)) return GB_ERR_ARG;
    if (!(kT > 0.0) || !isfinite(kT) || !isfinite(n_electrons)) return GB_ERR_ARG;
    if (P->n_sub <= 0 || !P->core_ptr || !P->core_idx || !P->core_pos || !P->sub_ptr || !P->sub_idx)
        return GB_ERR_ARG;
    const double n_occ = 0.5 * n_electrons;
    if (!(n_occ > 0.0) || !(n_occ < (double)n)) return GB_ERR_MU_BRACKET;
    if (D->n != n || !D->val || D->capacity < P->out_nnz) {
        D->nnz = P->out_nnz;
        return D->val ? GB_ERR_CAPACITY : GB_ERR_ARG;
    }
    for (int r = 0; r < m; ++r) {
        if (D1[r].n != n || !D1[r].val || D1[r].capacity < P->out_nnz) {
            D1[r].nnz = P->out_nnz;
            return D1[r].val ? GB_ERR_CAPACITY : GB_ERR_ARG;
        }
    }
    gb_opts o = {GB_PREC_FP64, 40, 0.0, 6, 0, 0.0, 0, 0.0};
    if (opts) o = *opts;
    if (o.precision < GB_PREC_FP64 || o.precision > GB_PREC_EIGEN) return GB_ERR_ARG;
    if (o.split_small_npad < 0 || o.split_small_npad > 64 || o.split_small_npad % 16 != 0) return GB_ERR_ARG;
    const bool eigen = o.precision == GB_PREC_EIGEN;
    const bool split = o.precision == GB_PREC_FP16X3 || o.precision == GB_PREC_BF16X3;
    if (eigen && P->max_sub > GB_EIG_MAX_N) return GB_ERR_UNSUPPORTED;
    if (o.max_newton <= 0) o.max_newton = 40;
    if (o.min_steps <= 0) o.min_steps = 6;
    if (o.ns_iters <= 0) o.ns_iters = split ? 2 : 3;
    const double tol_d = o.tol_d > 0.0 ? o.tol_d : (split ? 1e-6 : 1e-11);
    if (split && P->max_sub > GB_BIG_MAX_N) return GB_ERR_UNSUPPORTED;
    const bool big = split && P->max_sub > GB_SPLIT_MAX_N;
    if (!D->ptr) return GB_ERR_ARG;  // the value positions follow the column pointers

    h->launches = 0;
    Arena ar(h->ws, h->ws_bytes);
    DensityLayout L = layout_density(ar, P, m, o.precision);
    if (!ar.fits() || !h->ws) {
        Arena mm;
        layout_density(mm, P, m, o.precision);
        h->required_ws = mm.used();
        return GB_ERR_WORKSPACE;
    }
    cudaStream_t st = h->stream;
    const int32_t n_sub = P->n_sub;
    const int tb = 256;
    const int sub_grid = n_sub < 152 * 32 ? n_sub : 152 * 32;
    GB_CUDA(cudaMemsetAsync(L.err, 0, sizeof(int) * 8, st));

    // input checks
    GB_LAUNCH(h, k_check_finite, 1024, tb, 0, H->nnz, H->val, L.err);
    for (int r = 0; r < m; ++r) GB_LAUNCH(h, k_check_finite, 1024, tb, 0, H1[r].nnz, H1[r].val, L.err);

    // collected structure: column pointers, then row indices (shared by D and D1)
    GB_LAUNCH(h, k_csc_lengths, sub_grid, 128, 0, n_sub, P->sub_ptr, P->core_ptr, P->core_idx, D->ptr);
    GB_CUDA(cudaMemsetAsync(D->ptr + n, 0, sizeof(int64_t), st));
    GB_TRY(exclusive_scan_i64(h, D->ptr, D->ptr, (int64_t)n + 1, L.scan_tmp));
    if (D->idx)
        GB_LAUNCH(h, k_csc_rows, sub_grid, 128, 0, n_sub, P->sub_ptr, P->sub_idx, P->core_ptr,
                  P->core_idx, (const int64_t*)D->ptr, D->idx);
    for (int r = 0; r < m; ++r) {
        if (D1[r].ptr)
            GB_CUDA(cudaMemcpyAsync(D1[r].ptr, D->ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, st));
        if (D1[r].idx && D->idx)
            GB_CUDA(cudaMemcpyAsync(D1[r].idx, D->idx, sizeof(int32_t) * P->out_nnz, cudaMemcpyDeviceToDevice, st));
        else if (D1[r].idx)
            GB_LAUNCH(h, k_csc_rows, sub_grid, 128, 0, n_sub, P->sub_ptr, P->sub_idx, P->core_ptr,
                      P->core_idx, (const int64_t*)D->ptr, D1[r].idx);
    }
    // dense block offsets (FP64 path)
    GB_LAUNCH(h, k_block_sizes, (n_sub + tb - 1) / tb, tb, 0, n_sub, P->sub_ptr, L.moff, split ? 1 : 0);
    GB_CUDA(cudaMemsetAsync(L.moff + n_sub, 0, sizeof(int64_t), st));
    GB_TRY(exclusive_scan_i64(h, L.moff, L.moff, (int64_t)n_sub + 1, L.scan_tmp));
    const int stride = TR_FIXED + m;
    PassArgs a;
    memset(&a, 0, sizeof(a));
    a.n_sub = n_sub;
    a.m = m;
    a.sub_ptr = P->sub_ptr;
    a.sub_idx = P->sub_idx;
    a.core_ptr = P->core_ptr;
    a.core_idx = P->core_idx;
    a.core_pos = P->core_pos;
    a.Hptr = H->ptr;
    a.Hidx = H->idx;
    a.Hval = H->val;
    for (int r = 0; r < m; ++r) {
        a.H1ptr[r] = H1[r].ptr;
        a.H1idx[r] = H1[r].idx;
        a.H1val[r] = H1[r].val;
        a.D1val[r] = D1[r].val;
    }
    a.beta = 1.0 / kT;
    a.min_steps = o.min_steps;
    a.ns_iters = o.ns_iters;
    a.split_kind = o.precision == GB_PREC_BF16X3 ? 1 : 0;
    a.eps_lo = L.eps_lo;
    a.eps_hi = L.eps_hi;
    a.col_ptr = D->ptr;
    a.Dval = D->val;
    a.d1mu_val = L.d1mu_val;
    a.tr = L.tr;
    a.tr_stride = stride;
    a.steps_out = L.steps;
    a.pool = L.pool;
    a.moff = L.moff;
    a.pool_stride = L.pool_stride;
    a.z1pool = L.z1pool;
    a.hblk = L.hblk;
    a.boff = L.moff;
    a.hblk_stride = L.pool_stride;
    a.hdiag = L.hdiag;
    a.h1max = L.h1max;
    a.h1d = L.h1d;
    a.h1d_stride = P->sub_nnz;
    a.h1_offdiag = L.h1flag;
    a.big_scratch = L.big;
    a.big_stride = L.big_stride;
    a.big_npmax = L.big_npmax;
    a.big_counter = split ? L.work_n + 3 : nullptr;
    a.counter = split ? L.work_n + 4 : nullptr;
    a.err = L.err;
    // spectral bounds.  Split path: the gather of the dense principal
    // submatrices of H and H1 (once per call: they do not depend on mu) also
    // yields the Gershgorin intervals.
    const bool lists = split && (o.split_small_npad > 0 || big);
    int big_grid = 0;
    if (big) {
        int sms = 0;
        GB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
        big_grid = L.big_ctas < sms ? L.big_ctas : sms;
    }
    if (split) {
        if (lists)
            GB_LAUNCH(h, k_class_lists, 1, CLASS_THREADS, 0, n_sub, P->sub_ptr, o.split_small_npad, L.work,
                      L.work_n);
        // diagonal perturbations (the water workloads' H1 = diag(v)) skip the
        // dense h1 blocks of the one-tile subgraphs
        GB_CUDA(cudaMemsetAsync(L.h1flag, 0, sizeof(int), st));
        for (int r = 0; r < m; ++r)
            GB_LAUNCH(h, k_h1_offdiag, (n + tb - 1) / tb, tb, 0, n, H1[r].ptr, H1[r].idx, L.h1flag);
        GB_TRY(launch_split_gather(h, a, L.hblk, L.hdiag));
    } else {
        GB_LAUNCH(h, k_gershgorin, sub_grid, GERSH_THREADS, 0, n_sub, P->sub_ptr, P->sub_idx, H->ptr, H->idx,
                  H->val, L.eps_lo, L.eps_hi);
    }
    GB_TRY(reduce_traces(h, n_sub, stride, L));
    double bounds[2];
    int herr = 0;
    int32_t nclass[3] = {0, 0, 0};
    GB_CUDA(cudaMemcpyAsync(bounds, L.bounds, sizeof(bounds), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(&herr, L.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (lists) GB_CUDA(cudaMemcpyAsync(nclass, L.work_n, sizeof(nclass), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));  // one round trip for all
    if (herr) return herr;
    // The tiled class runs beside the one-tile classes on a second stream when
    // it holds few subgraphs (one per SM taken from the others' grid), after
    // them when it holds many (then it fills the GPU by itself).
    // When it runs beside them, a second launch of the 128-column kernel
    // follows it on its stream: big_grid more CTAs that draw on the same work
    // counter, so the SMs the tiled class held join the one-tile class once
    // it is done (their response scratch follows the first launch's).
    bool concurrent = false;
    int64_t tail_cta0 = -1;
    if (big) {
        int sms = 0;
        GB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
        big_grid = nclass[2] < big_grid ? nclass[2] : big_grid;
        concurrent = big_grid > 0 && 4 * big_grid <= sms && nclass[0] + nclass[1] > 0;
        if (concurrent) {
            a.grid_sms = sms - big_grid;
            const int64_t z1_ctas = n_sub < GB_SPLIT_MAX_CTAS ? n_sub : GB_SPLIT_MAX_CTAS;
            if (o.split_small_npad <= 0 && sms <= z1_ctas) tail_cta0 = a.grid_sms;
            if (!h->aux) GB_CUDA(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
            if (!h->ev_fork) GB_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
            if (!h->ev_join) GB_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
        }
    }

    // mu: Newton-Raphson on the core traces (Eq. NewtonRaphson), safeguarded
    // by a bisection bracket; each evaluation is one full pass.
    double lo = bounds[0] - 40.0 * kT, hi = bounds[1] + 40.0 * kT;
    double mu = *mu_inout;
    if (!(mu > lo && mu < hi)) mu = 0.5 * (lo + hi);
    double sums[TR_FIXED + GB_MAX_RHS];
    double kernel_ms = 0.0;
    if (!h->ev0) {
        GB_CUDA(cudaEventCreate(&h->ev0));
        GB_CUDA(cudaEventCreate(&h->ev1));
    }
    cudaEvent_t ev0 = h->ev0, ev1 = h->ev1;
    EigArgs ea;
    memset(&ea, 0, sizeof(ea));
    if (eigen) {
        // diagonalise every subgraph once; mu then needs only eigenvalue sums
        ea.scratch = L.eig_scratch;
        ea.scratch_stride = L.eig_stride;
        ea.eps = L.eig_eps;
        ea.w = L.eig_w;
        ea.vt = L.pool;
        ea.counter = L.eig_counter;
        ea.a = a;
        GB_CUDA(cudaEventRecord(ev0, st));
        GB_TRY(launch_eigen(h, ea, 0));
        GB_CUDA(cudaEventRecord(ev1, st));
        GB_CUDA(cudaMemcpyAsync(&herr, L.err, sizeof(int), cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaStreamSynchronize(st));
        if (herr) return herr;
        float ms = 0.f;
        GB_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
        kernel_ms += ms;
    }
    int passes = 0;
    bool converged = false;
    double prev_resid = INFINITY, last_bound = INFINITY;
    for (passes = 1; passes <= o.max_newton; ++passes) {
        a.mu = mu;
        GB_CUDA(cudaEventRecord(ev0, st));
        if (eigen) {
            ea.a = a;
            GB_TRY(launch_eigen(h, ea, 1));
        } else if (split) {
            // the 128-column configuration (for its size class when another
            // class takes subgraphs), the small one, the tiled one
            a.work = L.work;
            a.work_n = L.work_n;
            PassArgs bb = a;
            bb.work = L.work + 2 * (int64_t)n_sub;
            bb.work_n = L.work_n + 2;
            // the three launches' work counters (tiled, 128-column, small)
            GB_CUDA(cudaMemsetAsync(L.work_n + 3, 0, 3 * sizeof(int32_t), st));
            if (concurrent) {
                GB_CUDA(cudaEventRecord(h->ev_fork, st));
                GB_CUDA(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
                GB_TRY(launch_split_pass_big(h, bb, big_grid, h->aux));
                if (tail_cta0 >= 0) {
                    PassArgs t = a;
                    t.grid_sms = big_grid;
                    t.z1pool = a.z1pool + tail_cta0 * (m > 0 ? m : 1) * GB_SPLIT_MAX_N * GB_SPLIT_MAX_N;
                    GB_TRY(launch_split_pass_on(h, t, h->aux));
                }
                GB_CUDA(cudaEventRecord(h->ev_join, h->aux));
            }
            // the 128-column class: its list when the small class is in use,
            // else every subgraph up to 128 orbitals (the kernel skips the rest)
            if (o.split_small_npad > 0) GB_TRY(launch_split_pass_listed(h, a));
            else GB_TRY(launch_split_pass(h, a));
            if (o.split_small_npad > 0) {
                PassArgs b = a;
                b.work = L.work + n_sub;
                b.work_n = L.work_n + 1;
                b.counter = L.work_n + 5;
                GB_TRY(launch_split_pass_small(h, b));
            }
            if (concurrent) GB_CUDA(cudaStreamWaitEvent(st, h->ev_join, 0));
            else if (big && big_grid > 0) GB_TRY(launch_split_pass_big(h, bb, big_grid, st));
        } else {
            GB_LAUNCH(h, k_fermi_fp64, sub_grid, FP64_THREADS, 0, a);
        }
        GB_CUDA(cudaEventRecord(ev1, st));
        GB_TRY(reduce_traces(h, n_sub, stride, L));
        GB_CUDA(cudaMemcpyAsync(sums, L.sums, sizeof(double) * stride, cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaMemcpyAsync(&herr, L.err, sizeof(int), cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaStreamSynchronize(st));  // one round trip per pass
        {
            float ms = 0.f;
            GB_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
            kernel_ms += ms;
        }
        if (herr) return herr;
        if (!isfinite(sums[TR_D]) || !isfinite(sums[TR_DD])) return GB_ERR_NAN;
        const double resid = sums[TR_D] - n_occ;
        const double dn = a.beta * sums[TR_DD];
        // Converged when the occupation residual is within tol_occ * N_occ, or
        // when the remaining Newton correction |resid / dn| would move every
        // collected element of D by less than tol_d (first order, |dD_jk| <=
        // |dmu| sqrt(d1_mu_jj d1_mu_kk) with k a core vertex: d1_mu is PSD).
        const double dmu_newton = dn > 0.0 ? fabs(resid) / dn : INFINITY;
        const double d_bound = dmu_newton * sqrt(fmax(sums[TR_MAXW], 0.0) * fmax(sums[TR_MAXWC], 0.0));
        // Noise floor: once a Newton step no longer halves the residual, the
        // trace round-off dominates and further passes only move mu within it;
        // that floor is accepted when its D-change bound is small.
        const bool stalled = passes >= 2 && fabs(resid) >= 0.5 * prev_resid;
        if ((o.tol_occ > 0.0 && fabs(resid) <= o.tol_occ * n_occ) || d_bound <= tol_d ||
            (stalled && d_bound <= (split ? 100.0 : 10.0) * tol_d)) {
            converged = true;
            last_bound = d_bound;
            break;
        }
        last_bound = d_bound;
        prev_resid = fabs(resid);
        if (passes == o.max_newton) break;
        if (resid < 0.0) lo = mu; else hi = mu;
        double next = dn > 0.0 ? mu - resid / dn : NAN;
        // a Newton step stays inside the bracket and within 20 kT, else bisect
        if (!(next > lo && next < hi) || fabs(next - mu) > 20.0 * kT) next = 0.5 * (lo + hi);
        mu = next;
    }
    if (eigen) {
        // core columns of d, d1_mu and d1_lambda at the final mu, and the
        // d1_lambda traces for mu_1
        a.mu = mu;
        ea.a = a;
        GB_CUDA(cudaEventRecord(ev0, st));
        GB_TRY(launch_eigen(h, ea, 2));
        GB_CUDA(cudaEventRecord(ev1, st));
        GB_TRY(reduce_traces(h, n_sub, stride, L));
        GB_CUDA(cudaMemcpyAsync(sums, L.sums, sizeof(double) * stride, cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaMemcpyAsync(&herr, L.err, sizeof(int), cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaStreamSynchronize(st));
        float ms = 0.f;
        GB_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
        kernel_ms += ms;
        if (herr) return herr;
    }
    *mu_inout = mu;
    // FP64 redo of the subgraphs whose response is large (gb_opts.refine_d1):
    // flag them by |d1_lambda + mu_1 d1_mu| with mu_1 from the split traces,
    // diagonalise them and overwrite their core columns of d, d1_mu, d1_lambda
    // and their traces at the same mu, in waves of the eigenvector slots
    int32_t refined = 0, refine_skipped = 0;
    double refine_ms = 0.0;
    const double refine_thr = o.refine_d1;
    if (split && m > 0 && refine_thr > 0.0 && L.ref_list) {
        Mu1s mv;
        memset(&mv, 0, sizeof(mv));
        for (int r = 0; r < m; ++r) mv.v[r] = sums[TR_D1MU] > 0.0 ? -sums[TR_D1LAM + r] / sums[TR_D1MU] : 0.0;
        a.mu = mu;
        GB_CUDA(cudaEventRecord(ev0, st));
        GB_CUDA(cudaMemsetAsync(L.ref_n, 0, 8 * sizeof(int32_t), st));
        GB_LAUNCH(h, k_flag_refine, sub_grid, tb, 0, a, mv, refine_thr, GB_EIG_MAX_N, L.ref_list, L.ref_n);
        int32_t cnt[2] = {0, 0};
        GB_CUDA(cudaMemcpyAsync(cnt, L.ref_n, sizeof(cnt), cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaStreamSynchronize(st));
        refined = cnt[0];
        refine_skipped = cnt[1];
        if (refined > 0) {
            EigArgs ra;
            memset(&ra, 0, sizeof(ra));
            ra.a = a;
            ra.scratch = L.eig_scratch;
            ra.scratch_stride = L.eig_stride;
            ra.eps = L.eig_eps;
            ra.w = L.eig_w;
            ra.vt = L.ref_vt;
            ra.vt_stride = (int64_t)L.ref_me * L.ref_me;
            ra.counter = L.eig_counter;
            ra.list = L.ref_list;
            for (int32_t base = 0; base < refined; base += L.ref_slots) {
                ra.list_base = base;
                ra.list_n = refined - base < L.ref_slots ? refined - base : L.ref_slots;
                GB_TRY(launch_eigen(h, ra, 0));
                GB_TRY(launch_eigen(h, ra, 2));
            }
            GB_TRY(reduce_traces(h, n_sub, stride, L));
            GB_CUDA(cudaMemcpyAsync(sums, L.sums, sizeof(double) * stride, cudaMemcpyDeviceToHost, st));
            GB_CUDA(cudaMemcpyAsync(&herr, L.err, sizeof(int), cudaMemcpyDeviceToHost, st));
        }
        GB_CUDA(cudaEventRecord(ev1, st));
        GB_CUDA(cudaStreamSynchronize(st));
        float ms = 0.f;
        GB_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
        refine_ms = ms;
        if (herr) return herr;
    }
    // mu_1 (Eq. dmu_1) and D1 = d1_lambda + mu_1 d1_mu
    for (int r = 0; r < m; ++r) {
        const double den = sums[TR_D1MU];
        mu1[r] = den > 0.0 ? -sums[TR_D1LAM + r] / den : 0.0;
        GB_LAUNCH(h, k_d1_fixup, 1024, tb, 0, P->out_nnz, mu1[r], (const double*)L.d1mu_val, D1[r].val);
        D1[r].nnz = P->out_nnz;
    }
    D->nnz = P->out_nnz;
    int32_t max_steps = 0;
    {
        // largest step count of the final pass (small read-back)
        int32_t* hs = new (std::nothrow) int32_t[n_sub];
        if (hs) {
            GB_CUDA(cudaMemcpyAsync(hs, L.steps, sizeof(int32_t) * n_sub, cudaMemcpyDeviceToHost, st));
            GB_CUDA(cudaStreamSynchronize(st));
            for (int32_t i = 0; i < n_sub; ++i) max_steps = hs[i] > max_steps ? hs[i] : max_steps;
            delete[] hs;
        } else {
            GB_CUDA(cudaStreamSynchronize(st));
        }
    }
    if (rep) {
        rep->passes = passes > o.max_newton ? o.max_newton : passes;
        rep->max_steps = max_steps;
        rep->n_sub = n_sub;
        rep->max_sub = P->max_sub;
        rep->mu = mu;
        rep->trace_d = sums[TR_D];
        rep->dndmu = a.beta * sums[TR_DD];
        rep->occ_residual = sums[TR_D] - n_occ;
        rep->trace_d1mu = sums[TR_D1MU];
        rep->eps_min = bounds[0];
        rep->eps_max = bounds[1];
        rep->gemm_flops = sums[TR_FLOPS];
        rep->gemm_flops_per_step_count = sums[TR_FLOPS_S];
        rep->pass_kernel_ms = kernel_ms;
        rep->mu_d_bound = last_bound;
        rep->kernel_launches = h->launches;
        rep->refined = refined;
        rep->refine_skipped = refine_skipped;
        rep->refine_ms = refine_ms;
    }
    return converged ? GB_OK : GB_ERR_NO_CONVERGE;
}

// Size bins -> configuration: time one recursion pass per candidate threshold
// (the second of two, at fixed mu) and keep the fastest; see gbqr.h.
extern "C" int gb_plan_autotune(gb_handle* h, const gb_csr* H, const gb_csr* H1, int32_t m, double kT,
                                double n_electrons, const gb_part* P, const gb_opts* opts, double mu,
                                gb_csc* D, gb_csc* D1, gb_plan* plan) {
    if (!h || !P || !opts || !plan || m < 0 || m > GB_MAX_RHS || !(mu == mu)) return GB_ERR_ARG;
    if (opts->precision == GB_PREC_FP64 || P->n_sub <= 0 || !P->sub_ptr) return GB_ERR_ARG;
    const int64_t key[4] = {P->n_sub, P->sub_nnz, m, opts->precision};
    if (h->plan_valid && key[0] == h->plan_key[0] && key[1] == h->plan_key[1] && key[2] == h->plan_key[2] &&
        key[3] == h->plan_key[3]) {
        *plan = h->plan;
        plan->cached = 1;
        return GB_OK;
    }
    gb_plan pl;
    memset(&pl, 0, sizeof(pl));
    {
        const int64_t n_sub = P->n_sub;
        int64_t* sp = new (std::nothrow) int64_t[n_sub + 1];
        if (!sp) return GB_ERR_ARG;
        cudaError_t e = cudaMemcpyAsync(sp, P->sub_ptr, sizeof(int64_t) * (n_sub + 1), cudaMemcpyDeviceToHost,
                                        h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) {
            gb_note_device_error(e);
            delete[] sp;
            return GB_ERR_DEVICE;
        }
        for (int64_t i = 0; i < n_sub; ++i) {
            const int64_t np = (sp[i + 1] - sp[i] + 15) / 16;  // bins of 16
            if (np >= 1 && np <= 8) ++pl.bin_count[np - 1];
        }
        delete[] sp;
    }
    // candidates: 0 and each bin edge up to 64 that moves more subgraphs
    pl.candidate[pl.n_candidates++] = 0;
    int64_t moved = 0, prev = 0;
    for (int t = 1; t <= 4; ++t) {
        moved += pl.bin_count[t - 1];
        if (moved > prev) pl.candidate[pl.n_candidates++] = 16 * t;
        prev = moved;
    }
    double mu1[GB_MAX_RHS + 1];
    for (int k = 0; k < pl.n_candidates; ++k) {
        gb_opts o = *opts;
        o.split_small_npad = pl.candidate[k];
        o.max_newton = 1;
        for (int rep = 0; rep < 2; ++rep) {
            double mu_c = mu;
            gb_report r;
            memset(&r, 0, sizeof(r));
            const int st = gb_density_and_response(h, H, H1, m, kT, n_electrons, P, &o, &mu_c, D, D1, mu1, &r);
            if (st != GB_OK && st != GB_ERR_NO_CONVERGE) return st;
            pl.pass_ms[k] = r.pass_kernel_ms;
        }
    }
    double best = pl.pass_ms[0];
    for (int k = 1; k < pl.n_candidates; ++k) best = pl.pass_ms[k] < best ? pl.pass_ms[k] : best;
    for (int k = 0; k < pl.n_candidates; ++k) {
        if (pl.pass_ms[k] <= 1.02 * best) {
            pl.split_small_npad = pl.candidate[k];
            break;
        }
    }
    pl.cached = 0;
    h->plan = pl;
    for (int k = 0; k < 4; ++k) h->plan_key[k] = key[k];
    h->plan_valid = 1;
    *plan = pl;
    return GB_OK;
}
