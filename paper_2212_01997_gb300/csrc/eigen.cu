// The eigenbasis (molecular-orbital) route of the graph method in FP64: every
// subgraph's principal submatrix h^(i) is diagonalised (Eq. SmallKS), the
// shared chemical potential follows from eigenvalue sums weighted by the
// eigenvectors' core parts (Eq. NewtonRaphson and the terms after it), and the
// core columns of d^(i) (Eqs. DD0, DD), of d1_mu^(i) = beta d (I - d) (Eq.
// dddmu) and of the response d1_lambda^(i) (Eq. ddlambda) are formed in the
// eigenbasis:
//   d        = V diag(f) V^T,                 f_k = 1 / (exp(beta (e_k - mu)) + 1)
//   d1_mu    = V diag(beta f (1 - f)) V^T
//   d1_lambda= V (F o (V^T h1 V)) V^T,         F_kl = (f_k - f_l) / (e_k - e_l)
// (F_kk = -beta f_k (1 - f_k)).  Once the subgraphs are diagonalised, every mu
// iteration costs only the eigenvalue sums.
//
// Diagonalisation, one CTA per subgraph (textbook methods written out here):
// Householder reduction of h to tridiagonal form T = Q^T h Q; every
// eigenvalue of T by bisection on Sturm counts, one eigenvalue per thread;
// its eigenvector z_k from a twisted factorisation T - lambda_k I = N_r
// Delta_r N_r^T at the twist r of smallest |gamma_r| (one step of inverse
// iteration from e_r); eigenvectors of nearly equal eigenvalues orthogonalised
// against each other (Gram-Schmidt, twice); then V = Q Z.  All of it runs in
// parallel over the eigenvalues: GB300's FP64 pipe makes a serial scalar
// sweep (the implicit QL iteration) far too slow per subgraph.
// Eigenvectors are stored eigenvector-major (Vt[k][r] = component r of
// eigenvector k), so that the updates of the core columns read consecutive
// addresses across a warp.
#include <math.h>

#include "density.cuh"

namespace {

constexpr int EIG_THREADS = 256;
constexpr int TS = 32;          // FP64 GEMM tile

// C = A B tile buffers (the GEMM runs last, over the tridiagonal's arrays)
struct Tile {
    double a[TS][TS + 1];
    double b[TS][TS + 1];
};

struct EigCtl {
    union {
        struct {
            double d[GB_EIG_MAX_N];    // diagonal of T
            double e[GB_EIG_MAX_N];    // its sub-diagonal (e[k] = T[k+1][k])
            double v[GB_EIG_MAX_N];    // a Householder vector; then e^2
            double tau[GB_EIG_MAX_N];  // the Householder factors
            double w[GB_EIG_MAX_N];    // tridiagonalisation work vector; then the eigenvalues
        } s;
        Tile t;
    };
    double red[EIG_THREADS / 32];
    int item;
    int fail;
};

// sum over the block, the same value in every thread (fixed order); red is
// free again on return
__device__ __forceinline__ double block_sum(double x, double* red) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < EIG_THREADS / 32; ++w) t += red[w];
    __syncthreads();
    return t;
}

__device__ __forceinline__ int lower_bound_eig(const int32_t* a, int n, int32_t v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// dense M[S, S] (row-major n x n) from a CSR matrix
__device__ void gather_dense(int n, const int32_t* S, const int64_t* ptr, const int32_t* idx, const double* val,
                             double* M) {
    for (int64_t q = threadIdx.x; q < (int64_t)n * n; q += blockDim.x) M[q] = 0.0;
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const int32_t g = S[r];
        for (int64_t p = ptr[g]; p < ptr[g + 1]; ++p) {
            const int c = lower_bound_eig(S, n, idx[p]);
            if (c < n && S[c] == idx[p]) M[(int64_t)r * n + c] = val[p];
        }
    }
    __syncthreads();
}

// W = M[S, S] V for a CSR matrix M (row-major n x n V and W): one warp per
// row, the row's entries located in the subgraph's vertex list
__device__ void sparse_times(int n, const int32_t* S, const int64_t* ptr, const int32_t* idx, const double* val,
                             const double* V, double* W) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < n; r += EIG_THREADS / 32) {
        const int32_t g = S[r];
        const int64_t p0 = ptr[g], p1 = ptr[g + 1];
        for (int l0 = 0; l0 < n; l0 += 32) {
            const int l = l0 + lane;
            double s = 0.0;
            for (int64_t p = p0; p < p1; ++p) {
                const int c = lower_bound_eig(S, n, idx[p]);
                if (c < n && S[c] == idx[p] && l < n) s = fma(val[p], V[(int64_t)c * n + l], s);
            }
            if (l < n) W[(int64_t)r * n + l] = s;
        }
    }
    __syncthreads();
}

// C = A B (row-major n x n, no aliasing), 32 x 32 tiles through shared memory
__device__ void gemm_nn(int n, const double* A, const double* B, double* C, Tile& t) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int nt = (n + TS - 1) / TS;
    for (int tile = 0; tile < nt * nt; ++tile) {
        const int r0 = (tile / nt) * TS, c0 = (tile % nt) * TS;
        double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
        for (int k0 = 0; k0 < n; k0 += TS) {
            for (int q = threadIdx.x; q < TS * TS; q += EIG_THREADS) {
                const int i = q / TS, j = q % TS;
                t.a[i][j] = (r0 + i < n && k0 + j < n) ? A[(int64_t)(r0 + i) * n + k0 + j] : 0.0;
                t.b[i][j] = (k0 + i < n && c0 + j < n) ? B[(int64_t)(k0 + i) * n + c0 + j] : 0.0;
            }
            __syncthreads();
#pragma unroll 8
            for (int k = 0; k < TS; ++k) {
                const double a0 = t.a[ty][k], a1 = t.a[ty + 16][k], b0 = t.b[k][tx], b1 = t.b[k][tx + 16];
                acc[0][0] = fma(a0, b0, acc[0][0]);
                acc[0][1] = fma(a0, b1, acc[0][1]);
                acc[1][0] = fma(a1, b0, acc[1][0]);
                acc[1][1] = fma(a1, b1, acc[1][1]);
            }
            __syncthreads();
        }
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                const int r = r0 + ty + 16 * i, c = c0 + tx + 16 * j;
                if (r < n && c < n) C[(int64_t)r * n + c] = acc[i][j];
            }
    }
    __syncthreads();
}

// Householder reduction of the symmetric A (row-major, overwritten) to
// tridiagonal form: d, e in c; the vector of step k in column k of A below
// the diagonal, its factor in c.rc[k].
__device__ void tridiagonalize(int n, double* A, EigCtl& c) {
    for (int k = 0; k + 2 < n; ++k) {
        // x = A[k+1.., k] (x1 read before the reduction's barriers, ahead of
        // the writes below)
        const double x1 = A[(int64_t)(k + 1) * n + k];
        double ss = 0.0;
        for (int i = k + 1 + threadIdx.x; i < n; i += EIG_THREADS) {
            const double x = A[(int64_t)i * n + k];
            ss = fma(x, x, ss);
        }
        const double sigma = block_sum(ss, c.red);
        if (sigma == 0.0) {
            if (threadIdx.x == 0) {
                c.s.d[k] = A[(int64_t)k * n + k];
                c.s.e[k] = 0.0;
                c.s.tau[k] = 0.0;
            }
            for (int i = k + 1 + threadIdx.x; i < n; i += EIG_THREADS) c.s.v[i] = 0.0;
            __syncthreads();
            continue;
        }
        const double alpha = x1 >= 0.0 ? -sqrt(sigma) : sqrt(sigma);
        const double vtv = 2.0 * (sigma - x1 * alpha);
        const double tau = 2.0 / vtv;
        for (int i = k + 1 + threadIdx.x; i < n; i += EIG_THREADS) {
            const double vi = i == k + 1 ? x1 - alpha : A[(int64_t)i * n + k];
            c.s.v[i] = vi;
            A[(int64_t)i * n + k] = vi;  // kept for Q
        }
        if (threadIdx.x == 0) {
            c.s.d[k] = A[(int64_t)k * n + k];
            c.s.e[k] = alpha;
            c.s.tau[k] = tau;
        }
        __syncthreads();
        // p = tau A_sub v (column sums: coalesced across j), then K = tau v.p / 2
        double vp = 0.0;
        for (int j = k + 1 + threadIdx.x; j < n; j += EIG_THREADS) {
            double p = 0.0;
            for (int i = k + 1; i < n; ++i) p = fma(A[(int64_t)i * n + j], c.s.v[i], p);
            p *= tau;
            c.s.w[j] = p;
            vp = fma(c.s.v[j], p, vp);
        }
        const double K = 0.5 * tau * block_sum(vp, c.red);
        for (int j = k + 1 + threadIdx.x; j < n; j += EIG_THREADS) c.s.w[j] -= K * c.s.v[j];  // w
        __syncthreads();
        // A_sub -= v w^T + w v^T
        const int m = n - k - 1;
        for (int64_t q = threadIdx.x; q < (int64_t)m * m; q += EIG_THREADS) {
            const int i = k + 1 + (int)(q / m), j = k + 1 + (int)(q % m);
            A[(int64_t)i * n + j] -= c.s.v[i] * c.s.w[j] + c.s.w[i] * c.s.v[j];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (n >= 2) {
            c.s.d[n - 2] = A[(int64_t)(n - 2) * n + n - 2];
            c.s.e[n - 2] = A[(int64_t)(n - 1) * n + n - 2];
        }
        c.s.d[n - 1] = A[(int64_t)(n - 1) * n + n - 1];
        c.s.e[n - 1] = 0.0;
    }
    __syncthreads();
}

// Vt = Q^T = H_{n-3} ... H_0 by backward accumulation (only the trailing
// block changes at each step).  One warp per row of Vt.
__device__ void accumulate_q(int n, const double* A, double* Vt, EigCtl& c) {
    for (int64_t q = threadIdx.x; q < (int64_t)n * n; q += EIG_THREADS) Vt[q] = (q / n == q % n) ? 1.0 : 0.0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = n - 3; k >= 0; --k) {
        const double tau = c.s.tau[k];
        if (tau == 0.0) continue;  // (uniform: rc is in shared memory)
        for (int i = k + 1 + threadIdx.x; i < n; i += EIG_THREADS) c.s.v[i] = A[(int64_t)i * n + k];
        __syncthreads();
        for (int r = k + 1 + warp; r < n; r += EIG_THREADS / 32) {
            double u = 0.0;
            for (int i = k + 1 + lane; i < n; i += 32) u = fma(Vt[(int64_t)r * n + i], c.s.v[i], u);
            for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
            u *= tau;
            for (int i = k + 1 + lane; i < n; i += 32) Vt[(int64_t)r * n + i] -= u * c.s.v[i];
        }
        __syncthreads();
    }
}

// Sturm count: eigenvalues of the tridiagonal (d, e2 = e^2) below x, from the
// sign changes of p_i = (d_i - x) p_{i-1} - e2_{i-1} p_{i-2} (no divisions).
// A ratio q_i = p_i / p_{i-1} of magnitude below pivmin is taken as -pivmin,
// and the pair (p_{i-1}, p_i) is rescaled by powers of two to stay in range.
__device__ __forceinline__ int sturm_count(int n, const double* d, const double* e2, double x, double pivmin) {
    double a = 1.0, b = d[0] - x;
    if (fabs(b) < pivmin) b = -pivmin;
    int cnt = b < 0.0;
    for (int i = 1; i < n; ++i) {
        double c = fma(d[i] - x, b, -e2[i - 1] * a);
        if (fabs(c) < pivmin * fabs(b)) c = -pivmin * b;
        cnt += (c < 0.0) != (b < 0.0);
        a = b;
        b = c;
        const double m = fmax(fabs(a), fabs(b));
        if (m > 0x1p+400) {
            a *= 0x1p-400;
            b *= 0x1p-400;
        } else if (m < 0x1p-400) {
            a *= 0x1p+400;
            b *= 0x1p+400;
        }
    }
    return cnt;
}

// Eigenvector of T for the eigenvalue lam from the twisted factorisation
// T - lam I = L+ D+ L+^T (top down) = U- D- U-^T (bottom up), twisted at r:
// gamma_r = D+_r + D-_r - (d_r - lam); z_r = 1, z_i = -L+_i z_{i+1} above r,
// z_{i+1} = -U-_i z_i below it, at the twist of smallest |gamma_r|.  Lp and Um
// hold the thread's multipliers at stride ld; z (n values, contiguous)
// receives the unit vector.  Returns false when the vector is not finite.
__device__ bool twisted_vector(int n, const double* d, const double* e, double lam, double pivmin, double* Lp,
                               double* Um, int64_t ld, double* z) {
    if (n == 1) {
        z[0] = 1.0;
        return true;
    }
    double Dp = d[0] - lam;
    for (int i = 0; i + 1 < n; ++i) {
        if (fabs(Dp) < pivmin) Dp = Dp < 0.0 ? -pivmin : pivmin;
        const double l = e[i] / Dp;
        Lp[i * ld] = l;
        Dp = (d[i + 1] - lam) - e[i] * l;
    }
    double best = INFINITY;
    int r = n - 1;
    double Dm = d[n - 1] - lam;
    for (int t = n - 1; t >= 0; --t) {
        if (t < n - 1) {
            if (fabs(Dm) < pivmin) Dm = Dm < 0.0 ? -pivmin : pivmin;
            const double u = e[t] / Dm;
            Um[t * ld] = u;
            Dm = (d[t] - lam) - e[t] * u;
        }
        const double g = fabs(t > 0 ? Dm - e[t - 1] * Lp[(t - 1) * ld] : Dm);
        if (g < best) {
            best = g;
            r = t;
        }
    }
    z[r] = 1.0;
    double ss = 1.0;
    for (int i = r - 1; i >= 0; --i) {
        z[i] = -Lp[i * ld] * z[i + 1];
        ss = fma(z[i], z[i], ss);
    }
    for (int i = r; i + 1 < n; ++i) {
        z[i + 1] = -Um[i * ld] * z[i];
        ss = fma(z[i + 1], z[i + 1], ss);
    }
    if (!(ss < INFINITY)) return false;
    const double inv = 1.0 / sqrt(ss);
    for (int i = 0; i < n; ++i) z[i] *= inv;
    return true;
}

// y <- (T - sigma I)^-1 y by Gaussian elimination with partial pivoting (one
// thread): u0, u1, u2 receive the rows of U; a zero pivot becomes `tiny`.
__device__ void tridiagonal_solve(int n, const double* d, const double* e, double sigma, double tiny, double* y,
                                  double* u0, double* u1, double* u2) {
    double a = d[0] - sigma, b = n > 1 ? e[0] : 0.0, c = 0.0;  // pivot row at columns i, i+1, i+2
    for (int i = 0; i + 1 < n; ++i) {
        double a2 = e[i], b2 = d[i + 1] - sigma, c2 = i + 2 < n ? e[i + 1] : 0.0;
        double yi = y[i], yn = y[i + 1];
        if (fabs(a2) > fabs(a)) {
            double t = a; a = a2; a2 = t;
            t = b; b = b2; b2 = t;
            t = c; c = c2; c2 = t;
            t = yi; yi = yn; yn = t;
        }
        if (a == 0.0) a = tiny;
        const double m = a2 / a;
        u0[i] = a;
        u1[i] = b;
        u2[i] = c;
        y[i] = yi;
        a = b2 - m * b;
        b = c2 - m * c;
        c = 0.0;
        y[i + 1] = yn - m * yi;
    }
    if (a == 0.0) a = tiny;
    u0[n - 1] = a;
    y[n - 1] /= u0[n - 1];
    if (n >= 2) y[n - 2] = (y[n - 2] - u1[n - 2] * y[n - 1]) / u0[n - 2];
    for (int i = n - 3; i >= 0; --i) y[i] = (y[i] - u1[i] * y[i + 1] - u2[i] * y[i + 2]) / u0[i];
}

// zk <- zk minus its components along the unit rows k0..k-1 of Z (twice),
// normalised; returns |zk| before normalisation (block-uniform)
__device__ double orthonormalise(int n, double* Z, int k0, int k, double* red) {
    double* zk = Z + (int64_t)k * n;
    for (int pass = 0; pass < 2; ++pass) {
        for (int j = k0; j < k; ++j) {
            const double* zj = Z + (int64_t)j * n;
            double p = 0.0;
            for (int i = threadIdx.x; i < n; i += EIG_THREADS) p = fma(zk[i], zj[i], p);
            p = block_sum(p, red);
            for (int i = threadIdx.x; i < n; i += EIG_THREADS) zk[i] = fma(-p, zj[i], zk[i]);
            __syncthreads();
        }
    }
    double q = 0.0;
    for (int i = threadIdx.x; i < n; i += EIG_THREADS) q = fma(zk[i], zk[i], q);
    q = sqrt(block_sum(q, red));
    if (q > 0.0 && q < INFINITY) {
        const double inv = 1.0 / q;
        for (int i = threadIdx.x; i < n; i += EIG_THREADS) zk[i] *= inv;
    }
    __syncthreads();
    return q;
}

// Eigenpairs of the tridiagonal T (c.s.d, c.s.e): eigenvalues ascending into
// c.s.w, eigenvectors as the rows of Z (n x n, row-major).  Lp and Um are
// scratch of n x min(n, EIG_THREADS) doubles each.  Eigenvalues within ctol of
// their neighbour form clusters whose vectors are orthogonalised in order.
__device__ void tridiagonal_eigen(int n, EigCtl& c, double* Z, double* Lp, double* Um) {
    // split T where the coupling is negligible, |e_i| <= eps (|d_i| + |d_i+1|):
    // the blocks then decouple exactly in the recurrences below (a coupling
    // left at rounding level would be divided by a floored pivot)
    if (threadIdx.x == 0)
        for (int i = 0; i + 1 < n; ++i)
            if (fabs(c.s.e[i]) <= 0x1p-52 * (fabs(c.s.d[i]) + fabs(c.s.d[i + 1]))) c.s.e[i] = 0.0;
    __syncthreads();
    double* e2 = c.s.v;
    for (int i = threadIdx.x; i < n; i += EIG_THREADS) e2[i] = i + 1 < n ? c.s.e[i] * c.s.e[i] : 0.0;
    // Gershgorin interval of T and the pivot floor
    double lo = INFINITY, hi = -INFINITY, m2 = 0.0;
    for (int i = 0; i < n; ++i) {  // (uniform over the block: shared reads)
        const double r = (i > 0 ? fabs(c.s.e[i - 1]) : 0.0) + (i + 1 < n ? fabs(c.s.e[i]) : 0.0);
        lo = fmin(lo, c.s.d[i] - r);
        hi = fmax(hi, c.s.d[i] + r);
        if (i + 1 < n) m2 = fmax(m2, c.s.e[i] * c.s.e[i]);
    }
    __syncthreads();
    const double tnorm = fmax(fabs(lo), fabs(hi));
    const double pivmin = 0x1p-200 * fmax(1.0, m2);
    const double abstol = 0x1p-52 * tnorm;
    lo -= 2.0 * abstol * n + pivmin;
    hi += 2.0 * abstol * n + pivmin;
    // eigenvalue k: count(lo) <= k < count(hi)
    for (int k = threadIdx.x; k < n; k += EIG_THREADS) {
        double a = lo, b = hi;
        for (int it = 0; it < 100; ++it) {
            const double mid = 0.5 * (a + b);
            if (!(b - a > fmax(abstol, 0x1p-52 * fmax(fabs(a), fabs(b)))) || mid <= a || mid >= b) break;
            if (sturm_count(n, c.s.d, e2, mid, pivmin) <= k) a = mid;
            else b = mid;
        }
        c.s.w[k] = 0.5 * (a + b);
    }
    __syncthreads();
    // vectors: thread slot t handles k = t, t + EIG_THREADS, ... (the twisted
    // vector of its own eigenvalue)
    const int nact = n < EIG_THREADS ? n : EIG_THREADS;
    for (int k = threadIdx.x; k < n; k += EIG_THREADS)
        if (!twisted_vector(n, c.s.d, c.s.e, c.s.w[k], pivmin, Lp + threadIdx.x, Um + threadIdx.x, nact,
                            Z + (int64_t)k * n))
            c.fail = 1;
    __syncthreads();
    // runs of equal eigenvalues (gaps <= dtol): the twisted vectors of the
    // members after the first need not be independent, so each is replaced by
    // three steps of inverse iteration at its eigenvalue from a pseudo-random
    // start, orthogonalised against the earlier members after every step
    const double ctol = 0x1p-12 * tnorm, dtol = 0x1p-44 * tnorm;
    for (int k = 1; k < n; ++k) {
        if (!(c.s.w[k] - c.s.w[k - 1] <= dtol)) continue;  // (uniform: shared reads)
        int k0 = k - 1;
        while (k0 > 0 && c.s.w[k0] - c.s.w[k0 - 1] <= dtol) --k0;
        double* zk = Z + (int64_t)k * n;
        for (int i = threadIdx.x; i < n; i += EIG_THREADS) {
            const uint32_t h = (uint32_t)(i + 1) * 2654435761u ^ (uint32_t)(k + 1) * 40503u;
            zk[i] = (double)(h >> 8) * 0x1p-23 - 1.0;
        }
        __syncthreads();
        for (int it = 0; it < 3; ++it) {
            if (threadIdx.x == 0)
                tridiagonal_solve(n, c.s.d, c.s.e, c.s.w[k], 0x1p-52 * fmax(tnorm, pivmin), zk, Lp, Lp + n, Um);
            __syncthreads();
            const double q = orthonormalise(n, Z, k0, k, c.red);
            if (!(q > 0.0 && q < INFINITY)) {
                if (threadIdx.x == 0) c.fail = 1;
                break;
            }
        }
    }
    // neighbours within ctol: Gram-Schmidt of each against the earlier ones
    // (the vectors' own error is ~eps |T| / gap)
    for (int k = 1; k < n; ++k) {
        if (!(c.s.w[k] - c.s.w[k - 1] <= ctol)) continue;  // (uniform)
        int k0 = k - 1;
        while (k0 > 0 && c.s.w[k0] - c.s.w[k0 - 1] <= ctol) --k0;
        if (!(orthonormalise(n, Z, k0, k, c.red) > 0.5) && threadIdx.x == 0) c.fail = 1;
        __syncthreads();
    }
}

// Fermi occupation and 1 - f without cancellation, x = beta (e - mu)
__device__ __forceinline__ double occ(double x) {
    return x >= 0.0 ? exp(-x) / (1.0 + exp(-x)) : 1.0 / (1.0 + exp(x));
}
// f (1 - f) = 1 / (4 cosh^2 (x / 2)) without overflow
__device__ __forceinline__ double occ_weight(double x) {
    const double t = exp(-fabs(x));
    return t / ((1.0 + t) * (1.0 + t));
}

// Divided difference of the Fermi function, times beta: (f(x_k) - f(x_l)) /
// (e_k - e_l), given fk = f(x_k) and fl = f(x_l).  Direct quotient when the
// arguments are apart; otherwise the central Taylor form f'(m) + f'''(m) dx^2 / 24 with f' = -g/4, f''' =
// -(g/8) (3 t^2 - 1), g = sech^2(m/2), t = tanh(m/2) (error O(dx^4)).
__device__ __forceinline__ double fermi_dd(double xk, double xl, double fk, double fl, double beta) {
    const double dx = xk - xl;
    if (fabs(dx) > 1e-4) return beta * (fk - fl) / dx;
    const double m = 0.5 * (xk + xl);
    const double g = 4.0 * occ_weight(m);
    const double t = tanh(0.5 * m);
    return -0.25 * beta * g * (1.0 + (3.0 * t * t - 1.0) * dx * dx / 48.0);
}

// The subgraph i of work item j and the offset of its eigenvectors (list
// mode or every subgraph); false past the end.
__device__ __forceinline__ bool eig_item(const EigArgs& ea, int32_t j, int32_t& i, int64_t& voff) {
    if (ea.list) {
        if (j >= ea.list_n) return false;
        i = ea.list[ea.list_base + j];
        voff = (int64_t)j * ea.vt_stride;
    } else {
        if (j >= ea.a.n_sub) return false;
        i = j;
        voff = ea.a.moff[i];
    }
    return true;
}

}  // namespace

namespace {

__global__ void __launch_bounds__(EIG_THREADS) k_eigen(EigArgs ea) {
    const PassArgs& a = ea.a;
    __shared__ EigCtl c;
    if (threadIdx.x == 0) c.fail = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) c.item = atomicAdd(ea.counter, 1);
        __syncthreads();
        int32_t i;
        int64_t voff;
        if (!eig_item(ea, c.item, i, voff)) break;
        const int64_t s0 = a.sub_ptr[i];
        const int n = (int)(a.sub_ptr[i + 1] - s0);
        double* A = ea.scratch + (int64_t)blockIdx.x * ea.scratch_stride;
        double* Vt = ea.vt + voff;
        double* Um = A + (int64_t)n * n;      // twisted multipliers; then Q^T
        double* Z = Um + (int64_t)n * n;      // eigenvectors of T (rows)
        gather_dense(n, a.sub_idx + s0, a.Hptr, a.Hidx, a.Hval, A);
        tridiagonalize(n, A, c);
        tridiagonal_eigen(n, c, Z, Vt, Um);  // (Vt's storage holds L+ meanwhile)
        if (c.fail) {
            if (threadIdx.x == 0) set_error(a.err, GB_ERR_NO_CONVERGE);
            c.fail = 0;
        }
        for (int k = threadIdx.x; k < n; k += EIG_THREADS) ea.eps[s0 + k] = c.s.w[k];
        accumulate_q(n, A, Um, c);           // Q^T
        __syncthreads();
        gemm_nn(n, Z, Um, Vt, c.t);           // Vt = Z Q^T: row k = (Q z_k)^T
        // the core weights sum_{j in core} V_jk^2
        const int64_t c0 = a.core_ptr[i], c1 = a.core_ptr[i + 1];
        for (int k = threadIdx.x; k < n; k += EIG_THREADS) {
            double wk = 0.0;
            for (int64_t e = c0; e < c1; ++e) {
                const double x = Vt[(int64_t)k * n + a.core_pos[e]];
                wk = fma(x, x, wk);
            }
            ea.w[s0 + k] = wk;
        }
        if (threadIdx.x == 0 && !ea.list) a.steps_out[i] = 0;
    }
}

// Per-subgraph trace terms at a.mu from the eigenvalues alone (plus the
// largest diagonal of d1_mu over all rows and over core rows, n^2 work):
// TR_D = sum_k f_k w_k, TR_DD = sum_k f_k (1 - f_k) w_k, TR_D1MU = beta TR_DD.
__global__ void __launch_bounds__(EIG_THREADS) k_eig_traces(EigArgs ea) {
    const PassArgs& a = ea.a;
    __shared__ double red[EIG_THREADS / 32];
    __shared__ double gk[GB_EIG_MAX_N];
    for (int32_t i = blockIdx.x; i < a.n_sub; i += gridDim.x) {
        const int64_t s0 = a.sub_ptr[i];
        const int n = (int)(a.sub_ptr[i + 1] - s0);
        const double* Vt = ea.vt + a.moff[i];
        double td = 0.0, tdd = 0.0;
        for (int k = threadIdx.x; k < n; k += EIG_THREADS) {
            const double x = a.beta * (ea.eps[s0 + k] - a.mu);
            const double g = occ_weight(x);
            gk[k] = g;
            td = fma(occ(x), ea.w[s0 + k], td);
            tdd = fma(g, ea.w[s0 + k], tdd);
        }
        td = block_sum(td, red);
        tdd = block_sum(tdd, red);
        // diag d1_mu_jj = beta sum_k g_k V_jk^2
        double mx = 0.0;
        for (int j = threadIdx.x; j < n; j += EIG_THREADS) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) {
                const double v = Vt[(int64_t)k * n + j];
                s = fma(gk[k] * v, v, s);
            }
            mx = fmax(mx, s);
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
        __syncthreads();
        double mxw = 0.0;
        for (int w = 0; w < EIG_THREADS / 32; ++w) mxw = fmax(mxw, red[w]);
        __syncthreads();
        // over core rows
        double mc = 0.0;
        for (int64_t e = a.core_ptr[i] + threadIdx.x; e < a.core_ptr[i + 1]; e += EIG_THREADS) {
            const int j = a.core_pos[e];
            double s = 0.0;
            for (int k = 0; k < n; ++k) {
                const double v = Vt[(int64_t)k * n + j];
                s = fma(gk[k] * v, v, s);
            }
            mc = fmax(mc, s);
        }
        for (int o = 16; o > 0; o >>= 1) mc = fmax(mc, __shfl_xor_sync(0xffffffffu, mc, o));
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double mcw = 0.0;
            for (int w = 0; w < EIG_THREADS / 32; ++w) mcw = fmax(mcw, red[w]);
            double* tr = a.tr + (int64_t)i * a.tr_stride;
            tr[TR_D] = td;
            tr[TR_DD] = tdd;
            tr[TR_D1MU] = a.beta * tdd;
            tr[TR_FLOPS] = 0.0;
            tr[TR_FLOPS_S] = 0.0;
            tr[TR_MAXW] = a.beta * mxw;
            tr[TR_MAXWC] = a.beta * mcw;
            for (int r = 0; r < a.m; ++r) tr[TR_D1LAM + r] = 0.0;
        }
        __syncthreads();
    }
}

// Core columns of d, d1_mu and every d1_lambda_r at a.mu into the collected
// outputs, and the d1_lambda core traces.
__global__ void __launch_bounds__(EIG_THREADS) k_eig_response(EigArgs ea) {
    const PassArgs& a = ea.a;
    __shared__ Tile tile;
    __shared__ double red[EIG_THREADS / 32];
    __shared__ double fk[GB_EIG_MAX_N], gk[GB_EIG_MAX_N], yv[GB_EIG_MAX_N];
    __shared__ int item;
    if (threadIdx.x == 0) item = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item = atomicAdd(ea.counter, 1);
        __syncthreads();
        int32_t i;
        int64_t voff;
        if (!eig_item(ea, item, i, voff)) break;
        const int64_t s0 = a.sub_ptr[i];
        const int n = (int)(a.sub_ptr[i + 1] - s0);
        const int32_t* S = a.sub_idx + s0;
        const double* Vt = ea.vt + voff;
        double* M = ea.scratch + (int64_t)blockIdx.x * ea.scratch_stride;  // V^T h1 V, then F o (V^T h1 V)
        double* T = M + (int64_t)n * n;                                    // h1 V
        double* V = T + (int64_t)n * n;                                    // V = Vt^T
        double td = 0.0, tdd = 0.0;
        for (int k = threadIdx.x; k < n; k += EIG_THREADS) {
            const double x = a.beta * (ea.eps[s0 + k] - a.mu);
            fk[k] = occ(x);
            gk[k] = a.beta * occ_weight(x);
            td = fma(fk[k], ea.w[s0 + k], td);
            tdd = fma(occ_weight(x), ea.w[s0 + k], tdd);
        }
        // the core traces at a.mu (as k_eig_traces writes them)
        td = block_sum(td, red);
        tdd = block_sum(tdd, red);
        if (threadIdx.x == 0) {
            double* tr = a.tr + (int64_t)i * a.tr_stride;
            tr[TR_D] = td;
            tr[TR_DD] = tdd;
            tr[TR_D1MU] = a.beta * tdd;
        }
        const int64_t c0 = a.core_ptr[i], c1 = a.core_ptr[i + 1];
        // d and d1_mu core columns: d[r][c] = sum_k Vt[k][r] f_k Vt[k][c]
        for (int64_t e = c0; e < c1; ++e) {
            const int cp = a.core_pos[e];
            const int64_t o = a.col_ptr[a.core_idx[e]];
            for (int r = threadIdx.x; r < n; r += EIG_THREADS) {
                double sd = 0.0, sm = 0.0;
                for (int k = 0; k < n; ++k) {
                    const double p = Vt[(int64_t)k * n + r] * Vt[(int64_t)k * n + cp];
                    sd = fma(fk[k], p, sd);
                    sm = fma(gk[k], p, sm);
                }
                a.Dval[o + r] = sd;
                a.d1mu_val[o + r] = sm;
            }
        }
        if (a.m > 0) {
            for (int64_t q = threadIdx.x; q < (int64_t)n * n; q += EIG_THREADS)
                V[q] = Vt[(q % n) * n + q / n];
            __syncthreads();
        }
        for (int rr = 0; rr < a.m; ++rr) {
            sparse_times(n, S, a.H1ptr[rr], a.H1idx[rr], a.H1val[rr], V, T);  // T = h1 V
            gemm_nn(n, Vt, T, M, tile);                                     // M = V^T h1 V
            for (int64_t q = threadIdx.x; q < (int64_t)n * n; q += EIG_THREADS) {
                const int k = (int)(q / n), l = (int)(q % n);
                M[q] *= fermi_dd(a.beta * (ea.eps[s0 + k] - a.mu), a.beta * (ea.eps[s0 + l] - a.mu), fk[k], fk[l],
                                 a.beta);
            }
            __syncthreads();
            double tl = 0.0;
            for (int64_t e = c0; e < c1; ++e) {
                const int cp = a.core_pos[e];
                const int64_t o = a.col_ptr[a.core_idx[e]];
                // y = (F o h1') u, u_l = V[cp][l] = Vt[l][cp]
                for (int k = threadIdx.x; k < n; k += EIG_THREADS) {
                    double s = 0.0;
                    for (int l = 0; l < n; ++l) s = fma(M[(int64_t)k * n + l], Vt[(int64_t)l * n + cp], s);
                    yv[k] = s;
                }
                __syncthreads();
                for (int r = threadIdx.x; r < n; r += EIG_THREADS) {
                    double s = 0.0;
                    for (int k = 0; k < n; ++k) s = fma(Vt[(int64_t)k * n + r], yv[k], s);
                    a.D1val[rr][o + r] = s;
                    if (r == cp) tl += s;
                }
                __syncthreads();
            }
            tl = block_sum(tl, red);
            if (threadIdx.x == 0) a.tr[(int64_t)i * a.tr_stride + TR_D1LAM + rr] = tl;
            __syncthreads();
        }
    }
}

}  // namespace

int launch_eigen(gb_handle* h, const EigArgs& ea, int which) {
    int sms = 0;
    GB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    int grid = 4 * sms;
    const int32_t items = ea.list ? ea.list_n : ea.a.n_sub;
    if (ea.list && which == 1) return GB_ERR_ARG;
    if (items <= 0) return GB_OK;
    if (grid > items) grid = items;
    if (which == 0) {
        if (grid > GB_EIG_MAX_CTAS) grid = GB_EIG_MAX_CTAS;
        GB_CUDA(cudaMemsetAsync(ea.counter, 0, sizeof(int32_t), h->stream));
        GB_LAUNCH(h, k_eigen, grid, EIG_THREADS, 0, ea);
    } else if (which == 1) {
        GB_LAUNCH(h, k_eig_traces, grid, EIG_THREADS, 0, ea);
    } else {
        if (grid > GB_EIG_MAX_CTAS) grid = GB_EIG_MAX_CTAS;
        GB_CUDA(cudaMemsetAsync(ea.counter, 0, sizeof(int32_t), h->stream));
        GB_LAUNCH(h, k_eig_response, grid, EIG_THREADS, 0, ea);
    }
    return GB_OK;
}

// ---------------------------------------------------------------------------
// The subgraph preconditioner (Sec. "Preconditioner for a partitioned graph"):
// per subgraph, in its eigenbasis at mu, the responses of the core atoms'
// populations p_i = 2 sum_{o in i} d_oo to a unit charge on each core atom j
// (the diagonal perturbation u_o = C[atom(o), j], response d1_lambda of Eq.
// ddlambda) and to mu (d1_mu, Eq. dddmu); mu1_j such that the column sums of
// j_c = chi + rho_mu mu1^T - I are -1 (the core keeps its charge); then
// k0 = (j_c - alpha I)^-1 by Gauss-Jordan elimination with partial pivoting.
// ---------------------------------------------------------------------------
namespace {

__global__ void __launch_bounds__(EIG_THREADS) k_eig_jacobian(EigArgs ea, PrecondArgs pa) {
    const PassArgs& a = ea.a;
    __shared__ Tile tile;
    __shared__ double red[EIG_THREADS / 32];
    __shared__ double gk[GB_EIG_MAX_N], fk[GB_EIG_MAX_N], uv[GB_EIG_MAX_N];
    __shared__ int32_t catom[GB_PRECOND_MAX_ATOMS];
    __shared__ int item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item = atomicAdd(ea.counter, 1);
        __syncthreads();
        const int32_t i = item;
        if (i >= a.n_sub) break;
        const int64_t s0 = a.sub_ptr[i];
        const int n = (int)(a.sub_ptr[i + 1] - s0);
        const int32_t* S = a.sub_idx + s0;
        const double* Vt = ea.vt + a.moff[i];
        double* M = ea.scratch + (int64_t)blockIdx.x * ea.scratch_stride;
        double* T = M + (int64_t)n * n;
        double* V = T + (int64_t)n * n;
        // the small blocks at the end of the CTA's scratch (GB_PRECOND_SCRATCH doubles)
        double* chi = ea.scratch + (int64_t)(blockIdx.x + 1) * ea.scratch_stride - GB_PRECOND_SCRATCH;
        double* rmu = chi + GB_PRECOND_MAX_ATOMS * GB_PRECOND_MAX_ATOMS;
        double* aug = rmu + GB_PRECOND_MAX_ATOMS;
        const int64_t a0 = pa.atom_ptr[i];
        const int na = (int)(pa.atom_ptr[i + 1] - a0);
        const int64_t c0 = a.core_ptr[i], c1 = a.core_ptr[i + 1];
        for (int b = threadIdx.x; b < na; b += EIG_THREADS) catom[b] = pa.atoms[a0 + b];
        for (int k = threadIdx.x; k < n; k += EIG_THREADS) {
            gk[k] = a.beta * occ_weight(a.beta * (ea.eps[s0 + k] - a.mu));
            fk[k] = occ(a.beta * (ea.eps[s0 + k] - a.mu));
        }
        for (int64_t q = threadIdx.x; q < (int64_t)n * n; q += EIG_THREADS) V[q] = Vt[(q % n) * n + q / n];
        for (int q = threadIdx.x; q < na * na; q += EIG_THREADS) chi[q] = 0.0;
        __syncthreads();
        // rho_mu: one thread per core atom, its core orbitals in order
        for (int b = threadIdx.x; b < na; b += EIG_THREADS) {
            double s = 0.0;
            for (int64_t e = c0; e < c1; ++e) {
                if (pa.orb_atom[a.core_idx[e]] != catom[b]) continue;
                const int p = a.core_pos[e];
                for (int k = 0; k < n; ++k) {
                    const double v = Vt[(int64_t)k * n + p];
                    s = fma(gk[k] * v, v, s);
                }
            }
            rmu[b] = 2.0 * s;
        }
        for (int b = 0; b < na; ++b) {
            // u_o = C[atom(S_o), atom j]: binary search in the coupling row
            const int32_t j = catom[b];
            for (int o = threadIdx.x; o < n; o += EIG_THREADS) {
                const int32_t ao = pa.orb_atom[S[o]];
                int64_t lo = pa.Cptr[ao], hi = pa.Cptr[ao + 1];
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (pa.Cidx[mid] < j) lo = mid + 1; else hi = mid;
                }
                uv[o] = (lo < pa.Cptr[ao + 1] && pa.Cidx[lo] == j) ? pa.Cval[lo] : 0.0;
            }
            __syncthreads();
            // T = V^T diag(u) (rows of Vt scaled by u), M = T V = V^T diag(u) V
            for (int64_t q = threadIdx.x; q < (int64_t)n * n; q += EIG_THREADS) T[q] = Vt[q] * uv[q % n];
            __syncthreads();
            gemm_nn(n, T, V, M, tile);
            for (int64_t q = threadIdx.x; q < (int64_t)n * n; q += EIG_THREADS) {
                const int k = (int)(q / n), l = (int)(q % n);
                M[q] *= fermi_dd(a.beta * (ea.eps[s0 + k] - a.mu), a.beta * (ea.eps[s0 + l] - a.mu), fk[k], fk[l],
                                 a.beta);
            }
            __syncthreads();
            // d1_lambda_pp = u_p^T (F o h1') u_p for every core orbital p, u_p[k] = Vt[k][p]
            for (int64_t e = c0; e < c1; ++e) {
                const int p = a.core_pos[e];
                double s = 0.0;
                for (int k = threadIdx.x; k < n; k += EIG_THREADS) {
                    double y = 0.0;
                    for (int l = 0; l < n; ++l) y = fma(M[(int64_t)k * n + l], Vt[(int64_t)l * n + p], y);
                    s = fma(Vt[(int64_t)k * n + p], y, s);
                }
                s = block_sum(s, red);
                if (threadIdx.x == 0) {
                    const int32_t ao = pa.orb_atom[a.core_idx[e]];
                    int r = 0;
                    while (r < na && catom[r] != ao) ++r;
                    if (r < na) chi[r * na + b] += 2.0 * s;
                }
            }
            __syncthreads();
        }
        // j_c, then k0 = (j_c - alpha I)^-1 (thread 0; at most GB_PRECOND_MAX_ATOMS)
        if (threadIdx.x == 0) {
            double rs = 0.0;
            for (int r = 0; r < na; ++r) rs += rmu[r];
            const int w2 = 2 * na;
            for (int b = 0; b < na; ++b) {
                double cs = 0.0;
                for (int r = 0; r < na; ++r) cs += chi[r * na + b];
                const double mu1 = rs > 0.0 ? -cs / rs : 0.0;
                for (int r = 0; r < na; ++r) {
                    const double jc = chi[r * na + b] + rmu[r] * mu1 - (r == b ? 1.0 : 0.0);
                    if (pa.jc) pa.jc[pa.val_ptr[i] + (int64_t)r * na + b] = jc;
                    aug[r * w2 + b] = jc - (r == b ? pa.alpha : 0.0);
                    aug[r * w2 + na + b] = r == b ? 1.0 : 0.0;
                }
            }
            bool singular = false;
            for (int col = 0; col < na && !singular; ++col) {
                int piv = col;
                for (int r = col + 1; r < na; ++r)
                    if (fabs(aug[r * w2 + col]) > fabs(aug[piv * w2 + col])) piv = r;
                if (aug[piv * w2 + col] == 0.0) {
                    singular = true;
                    break;
                }
                if (piv != col)
                    for (int q = 0; q < w2; ++q) {
                        const double t = aug[col * w2 + q];
                        aug[col * w2 + q] = aug[piv * w2 + q];
                        aug[piv * w2 + q] = t;
                    }
                const double inv = 1.0 / aug[col * w2 + col];
                for (int q = 0; q < w2; ++q) aug[col * w2 + q] *= inv;
                for (int r = 0; r < na; ++r) {
                    if (r == col) continue;
                    const double fct = aug[r * w2 + col];
                    if (fct != 0.0)
                        for (int q = 0; q < w2; ++q) aug[r * w2 + q] -= fct * aug[col * w2 + q];
                }
            }
            if (singular) set_error(a.err, GB_ERR_NAN);
            for (int r = 0; r < na; ++r)
                for (int b = 0; b < na; ++b) pa.val[pa.val_ptr[i] + (int64_t)r * na + b] = aug[r * w2 + na + b];
        }
    }
}

}  // namespace

int launch_eig_jacobian(gb_handle* h, const EigArgs& ea, const PrecondArgs& pa) {
    int sms = 0;
    GB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    int grid = 2 * sms;
    if (grid > ea.a.n_sub) grid = ea.a.n_sub;
    if (grid > GB_EIG_MAX_CTAS) grid = GB_EIG_MAX_CTAS;
    GB_CUDA(cudaMemsetAsync(ea.counter, 0, sizeof(int32_t), h->stream));
    GB_LAUNCH(h, k_eig_jacobian, grid, EIG_THREADS, 0, ea, pa);
    return GB_OK;
}
