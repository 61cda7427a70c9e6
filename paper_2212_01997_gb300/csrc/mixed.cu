// Split-precision Fermi / response recursion on the 5th-generation tensor
// cores (tcgen05), one subgraph (|S_i| <= 128) per CTA.
//
// Every matrix product A B is split into FP16 (default) or BF16 parts,
// x = hi + lo, hi = rn(x), lo = rn(x - hi), and summed as
//   A_hi B_hi + A_hi B_lo + A_lo B_hi
// with FP32 accumulation in tensor memory.  An M = 128 tcgen05.mma costs the
// same for any N <= 256, so A_hi B_hi and A_hi B_lo share one instruction of
// N = 2 npad ([B_hi | B_lo] staged side by side): 2 K instructions per
// product instead of 3 K.  The product P lands in two TMEM halves (left:
// A_hi B_hi, right: the cross terms A_hi B_lo + A_lo B_hi) that the staging
// pass adds.
// Quantities close to the identity never pass through the 16-bit parts: the
// Newton-Schulz residual R = (I - X) - Y X is formed in FP32 from the FP32 X
// and the product (I - X exact on the diagonal, where X is in [1/2, 1]).
//
// Scaling (powers of two, so exact): staged operands hold 2^12 x their value,
// which keeps the FP16 lo parts of elements down to ~3e-5 out of the subnormal
// range; every product therefore lands in TMEM as 2^24 x its value, and all
// FP32 state kept in TMEM uses the same 2^24 units.  Each subgraph's
// perturbation is normalised by sigma = 2^-k so that (beta/2) sigma |h1| <= 1
// (the response is linear in h1; d1_lambda is unscaled by 1/sigma at the end),
// which bounds every response matrix by O(1).
//
// Resources per CTA (128-column configuration; the small one halves the
// columns): TMEM 4 NPMAX columns holding Z and X (FP32, npad columns each) and
// P (2 npad); shared memory = three staged operands (128 rows, hi and lo parts,
// NPMAX x 512 bytes each) laid out K-major in 8x8 core matrices without
// swizzle: element (r, k) of the hi part at byte
// (k/8)*2048 + (r/8)*128 + (r%8)*16 + (k%8)*2, the lo part npad*256 bytes on.
//
// The per-step schedule (Z FP32 in TMEM, staged in S0 on entry):
//   P = Z Z;  stage Y -> S1;  X region = Y Y (hi parts: it only seeds
//   Newton-Schulz);  X0 = (98 I - 80 Y + 32 Y^2)/99 -> X and S2;
//   first correction: P = Y X; R = (I - X) - P, hi parts -> lo half of S2;
//     P = X_hi R_hi; X += P -> X, S2;
//   last correction: P = Y X; stage R -> S1 (S0 in the last step, which still
//     needs Y); P = X R; X += P -> X, S2;
//   P = W/2 = X Z; Z = 2 P (next step) -> Z region and S0;
//   per RHS: S1 <- Z1 (bulk copy of its staged image); P = X Z1 -> X region
//            (x2); P = W Z1 -> S1 (x -1/2); P = (-W Z1 / 2) W; stage 2 X Z1 ->
//            S1; P += (2 X Z1) X -> staged image of Z1 in global memory
//            (last step: only its core columns, as d1_lambda).
// The last step also forms d1_mu = beta ((I - Y) X)^2 / 4 and redoes Z_s on
// the core columns on the CUDA cores (see refine_core).
#include "density.cuh"
#include "tc.cuh"

namespace {

// The file is compiled twice: the default configuration (GB_SPLIT_NPMAX 128:
// 12 warps = 4 TMEM lane quadrants x 3 column groups, one CTA per SM, all of
// TMEM and ~207 KB of shared memory) and a small one for subgraphs with
// npad <= 64 (GB_SPLIT_NPMAX 64: 8 warps, 256 TMEM columns, ~106 KB), which
// runs two CTAs per SM so that one CTA's staging overlaps the other's MMAs.
#ifndef GB_SPLIT_NPMAX
#define GB_SPLIT_NPMAX 128
#endif
// GB_SPLIT_LIST: the launch walks a list of subgraphs (one size class) rather
// than all of them.  The 128-column configuration is built both ways: with
// the list, the same kernel measured 5% slower on the water boxes (code
// layout; the per-subgraph work is identical), so it is used only when the
// small class is in use.
#ifndef GB_SPLIT_LIST
#define GB_SPLIT_LIST 0
#endif
#if GB_SPLIT_NPMAX == 128 && !GB_SPLIT_LIST
#define GB_SPLIT_THREADS 384
#define GB_SPLIT_MINB 1
#define GB_SPLIT_KERNEL k_fermi_split
#define GB_SPLIT_LAUNCH launch_split_pass
#elif GB_SPLIT_NPMAX == 128
#define GB_SPLIT_THREADS 384
#define GB_SPLIT_MINB 1
#define GB_SPLIT_KERNEL k_fermi_split_listed
#define GB_SPLIT_LAUNCH launch_split_pass_listed
#elif GB_SPLIT_NPMAX == 64 && GB_SPLIT_LIST
#define GB_SPLIT_THREADS 256
#define GB_SPLIT_MINB 2
#define GB_SPLIT_KERNEL k_fermi_split_small
#define GB_SPLIT_LAUNCH launch_split_pass_small
#else
#error "GB_SPLIT_NPMAX must be 128, or 64 with GB_SPLIT_LIST"
#endif
constexpr int THREADS = GB_SPLIT_THREADS;
constexpr int GROUPS = THREADS / 128;
constexpr int NMAX = GB_SPLIT_MAX_N;  // rows (TMEM lanes, M of every MMA)
constexpr int NPMAX = GB_SPLIT_NPMAX; // largest npad (columns) of this configuration
constexpr int REFINE_ROUNDS = 1;  // refinement rounds of the final step (the tensor-core
                                  // inverse as preconditioner leaves ~1e-14 after one)
constexpr uint32_t HALF_BYTES = NMAX * NPMAX * 2;  // one 16-bit part (128 rows x npad columns)
constexpr uint32_t STAGE_BYTES = 2 * HALF_BYTES;   // hi + lo
constexpr int NSTAGE = 3;
constexpr uint32_t LBO = 128 * (NMAX / 8);         // next 8-column group (K direction)
constexpr uint32_t SBO = 128;                      // next 8-row group (M/N direction)
constexpr uint32_t TMEM_COLS = 4 * NPMAX;  // Z, X, P (2 npad)
constexpr float STAGE_SCALE = 4096.f;               // staged operand = 2^12 x value
constexpr float TMEM_SCALE = 16777216.f;            // TMEM word = 2^24 x value
constexpr float TMEM_INV = 1.f / 16777216.f;

// per-core-vertex trace terms (FP32 values, summed in FP64 at the end)
enum CoreTerm { T_DHI = 0, T_DLO = 1, T_DD = 2, T_L0 = 3, T_COUNT = 3 + GB_MAX_RHS };

struct __align__(16) Ctl {
    unsigned long long mbar;
    unsigned long long mbar_bulk;  // completion of the bulk copy into a staged operand
    uint32_t tmem_base;
    int abort;
    int s;                      // the current subgraph's step count
    int kfew;                   // steps dropped by the bound on Q
    int32_t cur, nxt;           // claimed work items: in flight, next
    int32_t sigk[GB_MAX_RHS];   // perturbation normalisation sigma_r = 2^-sigk[r]
    int32_t cpos[NMAX];         // core vertices' positions in S_i
    int64_t ocol[NMAX];         // their columns' offsets in the collected CSC outputs
    float dg[NMAX];             // diagonal of x0 = alpha (h - mu) (FP64, rounded once)
    float red[THREADS];
    float wred[THREADS / 32];
    float tv[T_COUNT][NMAX];    // d (hi, lo), G^2/4 and d1_lambda_r on the core diagonal
};

constexpr size_t SMEM_BYTES = NSTAGE * STAGE_BYTES + sizeof(Ctl) + 1024;

// A operand, K-major: row m of the staged buffer is row m of A (8-column
// groups LBO apart, 8-row groups SBO apart).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) { return desc_bits(saddr, LBO, SBO); }

// B operand, MN-major on the same staged layout: staged row k holds B[k][:],
// so the 8-row groups (128 B apart) run along K and the 8-column groups
// (2048 B apart) along N.  The product is then A B, not A B^T: symmetric
// matrices carry their rounding asymmetry, and A B^T would feed it back.
__device__ __forceinline__ uint64_t make_desc_b(uint32_t saddr) { return desc_bits(saddr, SBO, LBO); }

__device__ __forceinline__ uint32_t elem_off(int r, int k) {
    return (uint32_t)(k >> 3) * LBO + (uint32_t)(r >> 3) * SBO + (uint32_t)(r & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

// combine sources, each times a coefficient k: nothing, one FP32 TMEM region
// (column c), the packed product (left c + right c2), a staged operand (hi +
// lo).  Distinct types, so every combine is compiled for its own sources.
struct SrcN {
    static constexpr int loads = 0;
    static constexpr bool staged = false;
    float k;
};
struct SrcT {
    static constexpr int loads = 1;
    static constexpr bool staged = false;
    uint32_t c;
    float k;
};
struct SrcP {
    static constexpr int loads = 2;
    static constexpr bool staged = false;
    uint32_t c, c2;
    float k;
};
struct SrcS {
    static constexpr int loads = 0;
    static constexpr bool staged = true;
    int stage;
    float k;
};

struct Kernel {
    const PassArgs& a;
    Ctl& c;
    uint8_t* st0;        // staged operand k at st0 + k STAGE_BYTES (no array:
    uint32_t st_addr0;   // a runtime slot index would move it to local memory)
    uint32_t tbase;
    uint32_t mbar;
    uint32_t phase;
    uint32_t mbar_bulk;
    uint32_t phase_bulk;
    int fmt;
    int n, npad;
    int row;       // this thread's row = TMEM lane
    int grp;       // column group: chunks [ch0, ch1) of 16 columns
    int ch0, ch1;
    uint32_t lane_off;
    uint32_t lo_off;          // bytes from a staged operand's hi part to its lo part (npad x 256)
    uint32_t zc, xc, pl, pr;  // TMEM columns: Z, X (FP32 state), product left / right halves
    bool diag_h1;             // the perturbations are diagonal: X1 staged from a.h1d

    __device__ Kernel(const PassArgs& a_, Ctl& c_, uint8_t* smem) : a(a_), c(c_) {
        st0 = smem;
        st_addr0 = smem_u32(smem);
        mbar = smem_u32(&c.mbar);
        phase = 0;
        mbar_bulk = smem_u32(&c.mbar_bulk);
        phase_bulk = 0;
        fmt = a.split_kind;
        row = threadIdx.x & 127;
        grp = threadIdx.x >> 7;
        lane_off = (uint32_t)((row & ~31) << 16);
        diag_h1 = a.m > 0 && a.h1_offdiag && *a.h1_offdiag == 0;
    }

    // Per-subgraph layout.  Staged operand: hi part in 8-column groups 2048 B
    // apart, lo part right after it (lo_off = npad/8 groups), so [B_hi | B_lo]
    // read MN-major is one operand of N = 2 npad.  TMEM (4 npad <= 512
    // columns): Z at 0, X at npad, the product P at 2 npad (left) and 3 npad
    // (right half: the A_hi B_lo term of a packed product).
    __device__ void set_size(int n_) {
        n = n_;
        npad = (n + 15) & ~15;
        const int nch = npad / 16, per = (nch + GROUPS - 1) / GROUPS;
        ch0 = min(nch, grp * per);
        ch1 = min(nch, ch0 + per);
        lo_off = (uint32_t)npad * 256u;
        zc = 0;
        xc = (uint32_t)npad;
        pl = 2u * (uint32_t)npad;
        pr = 3u * (uint32_t)npad;
    }

    __device__ uint32_t col(uint32_t cidx) const { return tbase + cidx; }
    __device__ uint8_t* st(int k) const { return st0 + (uint32_t)k * STAGE_BYTES; }
    __device__ uint32_t sa_of(int k) const { return st_addr0 + (uint32_t)k * STAGE_BYTES; }

    // combine sources: a TMEM region, the packed product (left + right), a
    // staged operand (hi + lo), each times a coefficient
    __device__ static SrcT T(uint32_t c_, float k) { return {c_, k}; }
    __device__ SrcP Pk(float k) const { return {pl, pr, k}; }
    __device__ static SrcS S(int stage, float k) { return {stage, k}; }
    __device__ static SrcN none() { return {0.f}; }

    // Staged operand sg <- a staged image in global memory (npad x 512 bytes:
    // hi part, then lo part), by one bulk copy.  All threads; no MMA may still
    // read sg.  Earlier generic accesses to sg (and the generic writes of the
    // image, fenced by their writers) are ordered before the copy by the proxy
    // fence and the barrier; wait_bulk() makes the operand usable.
    __device__ void bulk_load(int sg, const uint8_t* g) {
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) bulk_g2s(sa_of(sg), g, (uint32_t)npad * 512u, mbar_bulk);
    }
    __device__ bool wait_bulk() {
        bool ok = mbar_wait(mbar_bulk, phase_bulk);
        phase_bulk ^= 1u;
        if (!ok) {
            c.abort = 1;
            set_error(a.err, GB_ERR_TIMEOUT);
        }
        __syncthreads();
        return c.abort == 0;
    }

    // all threads: make generic smem writes and TMEM stores visible to the MMA
    __device__ void sync_for_mma() {
        fence_proxy_async();
        fence_before();
        __syncthreads();
    }

    __device__ uint64_t da(int sa, uint32_t part, int ks) const {
        return make_desc(sa_of(sa) + part + (uint32_t)ks * 2u * LBO);   // A: 16 columns of K
    }
    __device__ uint64_t db(int sb, uint32_t part, int ks) const {
        return make_desc_b(sa_of(sb) + part + (uint32_t)ks * 2u * SBO); // B: 16 rows of K
    }

    // P = A B (acc = false) or P += A B, split in FP16 parts.  Even K steps:
    //   [left | right] += A_hi [B_hi | B_lo]   (one N = 2 npad instruction)
    //   right          += A_lo B_hi
    // odd K steps, the large term into the other half:
    //   right += A_hi B_hi;  left += A_hi B_lo;  left += A_lo B_hi
    // so each half accumulates the large A_hi B_hi terms of half of the K
    // steps: the tensor cores' FP32 accumulation rounds toward zero, and two
    // accumulators at half the magnitude halve that bias (and its spread).
    // The product is left + right, added by the staging pass.
    __device__ void issue_prod(int sa, int sb, bool acc) {
        const int K = npad / 16;
        const uint32_t id1 = make_idesc(fmt, 0, npad), id2 = make_idesc(fmt, 0, 2 * npad);
        const uint32_t dl = col(pl), dr = col(pr);
        for (int ks = 0; ks < K; ++ks) {
            if ((ks & 1) == 0) {
                mma_f16(dl, da(sa, 0, ks), db(sb, 0, ks), id2, (acc || ks > 0) ? 1u : 0u);
                mma_f16(dr, da(sa, lo_off, ks), db(sb, 0, ks), id1, 1u);
            } else {
                mma_f16(dr, da(sa, 0, ks), db(sb, 0, ks), id1, 1u);
                mma_f16(dl, da(sa, 0, ks), db(sb, lo_off, ks), id1, 1u);
                mma_f16(dl, da(sa, lo_off, ks), db(sb, 0, ks), id1, 1u);
            }
        }
    }

    // left = A_hi B_hi only (a product that only seeds an iteration)
    // (B's hi part read from byte offset bpart of slot sb: lo_off for a hi part
    // parked in a slot's lo half)
    // into TMEM columns dc (the left half of P unless given)
    __device__ void issue_hh(int sa, int sb, uint32_t bpart, uint32_t dc) {
        const int K = npad / 16;
        const uint32_t id1 = make_idesc(fmt, 0, npad);
        for (int ks = 0; ks < K; ++ks) mma_f16(col(dc), da(sa, 0, ks), db(sb, bpart, ks), id1, ks > 0 ? 1u : 0u);
    }

    // wait for every MMA issued so far by thread 0
    __device__ bool wait_mma() {
        if (threadIdx.x == 0) mma_commit(mbar);
        bool ok = mbar_wait(mbar, phase);
        phase ^= 1u;
        fence_after();
        if (!ok) {
            c.abort = 1;
            set_error(a.err, GB_ERR_TIMEOUT);
        }
        __syncthreads();
        return c.abort == 0;
    }

    // one product P = A B (P += A B with acc; hi parts only with hh) of
    // staged operands sa, sb
    __device__ bool gemm(int sa, int sb, bool acc = false, bool hh = false, uint32_t bpart = 0,
                         int dc = -1) {
        sync_for_mma();
        if (threadIdx.x == 0) {
            fence_after();
            if (hh) issue_hh(sa, sb, bpart, dc >= 0 ? (uint32_t)dc : pl);
            else issue_prod(sa, sb, acc);
        }
        return wait_mma();
    }

    // two products P = A1 B1 + A2 B2
    __device__ bool gemm2(int sa1, int sb1, int sa2, int sb2) {
        sync_for_mma();
        if (threadIdx.x == 0) {
            fence_after();
            issue_prod(sa1, sb1, false);
            issue_prod(sa2, sb2, true);
        }
        return wait_mma();
    }

    // 8 columns [c0, c0 + 8) of row `row` of staged operand sg as FP32 (hi +
    // lo, exact), in staged units
    __device__ void load_staged8(int sg, int c0, float (&v)[8]) const {
        const uint8_t* p = st(sg) + elem_off(row, c0);
        const uint4 h4 = *(const uint4*)p, l4 = *(const uint4*)(p + lo_off);
        const uint32_t w[8] = {h4.x, h4.y, h4.z, h4.w, l4.x, l4.y, l4.z, l4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float2 h, l;
            if (fmt == 0) {
                h = __half22float2(*(const __half2*)&w[j]);
                l = __half22float2(*(const __half2*)&w[4 + j]);
            } else {
                h = __bfloat1622float2(*(const __nv_bfloat162*)&w[j]);
                l = __bfloat1622float2(*(const __nv_bfloat162*)&w[4 + j]);
            }
            v[2 * j] = h.x + l.x;
            v[2 * j + 1] = h.y + l.y;
        }
    }

    // issue the TMEM loads of one source for the 8 columns at c0 (no wait)
    template <class Q>
    __device__ void src_issue(const Q& q, int c0, uint32_t (&r1)[8], uint32_t (&r2)[8]) const {
        if constexpr (Q::loads >= 1) tmem_ld8_issue(col(q.c) + lane_off + c0, r1);
        if constexpr (Q::loads == 2) tmem_ld8_issue(col(q.c2) + lane_off + c0, r2);
    }

    // add k x (one source at c0) to v, after the wait
    template <class Q>
    __device__ void src_add(const Q& q, float k, int c0, uint32_t (&r1)[8], uint32_t (&r2)[8],
                            float (&v)[8]) const {
        if constexpr (Q::staged) {
            float w[8];
            load_staged8(q.stage, c0, w);
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = fmaf(w[j], k, v[j]);
        } else if constexpr (Q::loads == 2) {
            pin8(r1);
            pin8(r2);
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = fmaf(__uint_as_float(r1[j]) + __uint_as_float(r2[j]), k, v[j]);
        } else if constexpr (Q::loads == 1) {
            pin8(r1);
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = fmaf(__uint_as_float(r1[j]), k, v[j]);
        }
    }

    // TMEM load registers of one 8-column unit (two sources, up to two loads each)
    struct Regs {
        uint32_t a1[8], a2[8], b1[8], b2[8];
    };

    template <class QA, class QB>
    __device__ __forceinline__ void unit_issue(const QA& A, const QB& B, int u, Regs& r) const {
        src_issue(A, 8 * u, r.a1, r.a2);
        src_issue(B, 8 * u, r.b1, r.b2);
    }

    template <class QA, class QB>
    __device__ __forceinline__ void unit_body(const QA& A, const QB& B, float ka, float kb, float kd, float ks,
                                              bool diag, int out, int sg, uint8_t* gst, int shl, int u,
                                              Regs& r) const {
        const int c0 = 8 * u;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = 0.f;
        src_add(A, ka, c0, r.a1, r.a2, v);
        if (diag && (unsigned)(row - c0) < 8u) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (c0 + j == row) v[j] += kd;
        }
        src_add(B, kb, c0, r.b1, r.b2, v);
        if (out >= 0) tmem_st8(col((uint32_t)out) + lane_off + c0, v);
        if (shl >= 0) {
            uint32_t hi[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) hi[j] = hi_pair(v[2 * j] * ks, v[2 * j + 1] * ks, fmt);
            *(uint4*)(st(shl) + lo_off + elem_off(row, c0)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        }
        if (sg >= 0 || gst) {
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) split_pair(v[2 * j] * ks, v[2 * j + 1] * ks, fmt, hi[j], lo[j]);
            const uint32_t off = elem_off(row, c0);
            if (sg >= 0) {
                uint8_t* p = st(sg) + off;
                *(uint4*)p = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                *(uint4*)(p + lo_off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            }
            if (gst) {
                uint8_t* p = gst + off;
                *(uint4*)p = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                *(uint4*)(p + lo_off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            }
        }
    }

    // Row-wise combination u = (A + cd I) + B (A, B: sources with their
    // coefficients; cd on the diagonal of the n x n block), written to the
    // FP32 TMEM region at column `out` (TMEM units; < 0: none), staged operand
    // `sg` and/or a staged image `gst` in global memory (the layout of a staged
    // operand, npad x 512 bytes; see bulk_load).  With shl >= 0, the hi parts
    // alone go to the lo half of staged operand shl (an operand only a product
    // of hi parts reads; see issue_hh).
    // Every TMEM region and staged operand is exactly zero outside the n x n
    // block, so only the identity needs masking.  The power-of-two unit changes
    // are folded into the coefficients.
    // Work split: 8-column units, unit u to column group u mod 3 (balanced to
    // one unit).  One unit's loads per wait: the other warps of the SM
    // sub-partition cover the load latency (keeping the next unit's loads in
    // flight measured slower, from the extra live registers).
    template <class QA, class QB>
    __device__ __forceinline__ void combine(const QA& A, const QB& B, float cd, int out, int sg, uint8_t* gst,
                                            int shl = -1) {
        const bool stage_only = out < 0;
        const float unit = stage_only ? STAGE_SCALE * TMEM_INV : 1.f;  // TMEM units -> target units
        const float ka = A.k * (QA::staged ? unit * TMEM_SCALE / STAGE_SCALE : unit);
        const float kb = B.k * (QB::staged ? unit * TMEM_SCALE / STAGE_SCALE : unit);
        const float kd = cd * TMEM_SCALE * unit;
        const float ks = stage_only ? 1.f : STAGE_SCALE * TMEM_INV;  // target units -> staged units
        const bool diag = cd != 0.f && row < n;
        constexpr bool tm = QA::loads + QB::loads > 0;
        const int nu = npad / 8;
        Regs r0;
        for (int u = grp; u < nu; u += GROUPS) {
            if constexpr (tm) {
                unit_issue(A, B, u, r0);
                tmem_wait_ld();
            }
            unit_body(A, B, ka, kb, kd, ks, diag, out, sg, gst, shl, u, r0);
        }
        if (out >= 0) tmem_wait_st();
        if (gst) fence_proxy_async_global();  // read back by a bulk copy
    }

    // largest k <= kmax with 4^k max_r sum_c |P_rc| <= 1 for the product P
    // (block-uniform).  Row sums and their maximum in FP32; the factor
    // 1 + 2^-16 covers the sums' rounding, so the bound stays an upper bound.
    __device__ int fewer_steps(int kmax) {
        float rs = 0.f;
        for (int ch = ch0; ch < ch1; ++ch) {
            float v[16], w[16];
            tmem_ld16x2(col(pl) + lane_off + ch * 16, col(pr) + lane_off + ch * 16, v, w);
#pragma unroll
            for (int j = 0; j < 16; ++j) rs += fabsf(v[j] + w[j]);
        }
        c.red[threadIdx.x] = rs;
        __syncthreads();
        if (grp == 0) {
            float tot = c.red[row];
            for (int g = 1; g < GROUPS; ++g) tot += c.red[row + 128 * g];
            for (int o = 16; o > 0; o >>= 1) tot = fmaxf(tot, __shfl_down_sync(0xffffffffu, tot, o));
            if ((threadIdx.x & 31) == 0) c.wred[threadIdx.x >> 5] = tot;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float q = c.wred[0];
            for (int w = 1; w < 4; ++w) q = fmaxf(q, c.wred[w]);
            const double qmax = (double)q * (double)TMEM_INV * (1.0 + 0x1p-16);
            int k = 0;
            while (k < kmax && qmax * ldexp(1.0, 2 * (k + 1)) <= 1.0) ++k;
            c.kfew = k;
        }
        __syncthreads();
        return c.kfew;
    }

    // Matrix times NC vectors on the CUDA cores: P_g[cc][row] = sum over this
    // column group's k of M_row,k v[k][cc], M = scale x TMEM slot sl (scale a
    // power of two, applied to the sums: exact).  v is in shared memory as
    // [k][NC + 4] floats (broadcast float4 reads); FP32 products are summed
    // per 8-column unit (round to nearest; units dealt to the column groups as
    // in combine), the unit sums without rounding error (float pairs).  P
    // holds the column groups' partials as float pairs, [GROUPS][NC][NMAX]
    // (column-major, so the row-indexed stores are conflict-free); the caller
    // adds them after a barrier.
    template <int NC>
    __device__ void rowvec(uint32_t sl, float scale, const float* v, FF* P) {
        constexpr int VL = NC + 4;
        float hi[NC], lo[NC];  // unit sums accumulated as unevaluated float pairs
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) hi[cc] = lo[cc] = 0.f;
        const int nu = npad / 8;
        for (int u = grp; u < nu; u += GROUPS) {
            const int c0 = u * 8;
            uint32_t m[8];
            tmem_ld8_issue(col(sl) + lane_off + c0, m);
            tmem_wait_ld();
            pin8(m);
            float acc[NC];
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) acc[cc] = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float mj = __uint_as_float(m[j]);
                const float4* vr = (const float4*)(v + (c0 + j) * VL);
#pragma unroll
                for (int q = 0; q < NC / 4; ++q) {
                    const float4 x = vr[q];
                    acc[4 * q] = fmaf(mj, x.x, acc[4 * q]);
                    acc[4 * q + 1] = fmaf(mj, x.y, acc[4 * q + 1]);
                    acc[4 * q + 2] = fmaf(mj, x.z, acc[4 * q + 2]);
                    acc[4 * q + 3] = fmaf(mj, x.w, acc[4 * q + 3]);
                }
            }
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) {
                const FF t = two_sum(hi[cc], acc[cc]);
                hi[cc] = t.hi;
                lo[cc] += t.lo;
            }
        }
        FF* Pg = P + grp * (NC * NMAX);
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) {
            const FF t = two_sum(hi[cc], lo[cc]);
            Pg[cc * NMAX + row] = FF{t.hi * scale, t.lo * scale};
        }
    }

    // row `row` of NC float vectors, [row][NC + 4] (16-byte stores, conflict-free)
    template <int NC>
    __device__ void put_row(float* V, const float* x) {
        constexpr int VL = NC + 4;
#pragma unroll
        for (int q = 0; q < NC / 4; ++q)
            *(float4*)(V + row * VL + 4 * q) = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
    }

    // The last doubling on the core columns, on CUDA cores: w = Z_s e_c =
    // 2 (I + Z^2)^-1 Z e_c by iterative refinement with the tensor-core
    // inverse X as preconditioner,  w <- w + X (2 z - w - Z (Z w)),  every
    // product rounded to nearest and every sum carried as a float pair.  The
    // start w0 = 2 X Z e_c is the tensor-core product P = X Z of the step
    // (P must hold it on entry).  The
    // saturated occupations (and Tr_c d) then carry no accumulation bias.
    // Writes d = (I - Z_s)/2 on the core columns and its core diagonal terms.
    // Scratch: staged operands S0 and S1 (free at this point).  All threads.
    template <int NC>
    __device__ void refine_core(uint32_t zs, uint32_t xs, float zsc, int ncore) {
        constexpr int VL = NC + 4;
        float* Vz = (float*)st(0);
        float* Vw = Vz + NMAX * VL;
        float* Vt = Vw + NMAX * VL;
        FF* Wd = (FF*)(Vt + NMAX * VL);  // [NC][NMAX]
        FF* P = Wd + NC * NMAX;          // [GROUPS][NC][NMAX]
        // sum of the column groups' partials, in group order
        auto psum = [&](int cc) {
            FF t = P[cc * NMAX + row];
#pragma unroll
            for (int g = 1; g < GROUPS; ++g) t = ff_add(t, P[(g * NC + cc) * NMAX + row]);
            return t;
        };
        const bool live = grp == 0 && row < n;
        for (int b0 = 0; b0 < ncore; b0 += NC) {
            const int nc = min(NC, ncore - b0);
            float x[NC];
            if (grp == 0) {
                float zv[NC], pl_[NC], pr_[NC];
                tmem_ld_cols<NC>(col(zs) + lane_off, c.cpos + b0, nc, zv);
                // w0 = 2 X z: the tensor-core product P = X Z on these columns
                // (its error is contracted by ~|I - X (I + Z^2)| in the round below)
                tmem_ld_cols<NC>(col(pl) + lane_off, c.cpos + b0, nc, pl_);
                tmem_ld_cols<NC>(col(pr) + lane_off, c.cpos + b0, nc, pr_);
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) x[cc] = (row < n && cc < nc) ? zv[cc] * zsc : 0.f;
                put_row<NC>(Vz, x);
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const FF w0 = (live && cc < nc) ? FF{2.f * (pl_[cc] + pr_[cc]) * zsc, 0.f} : FF{0.f, 0.f};
                    Wd[cc * NMAX + row] = w0;
                    x[cc] = w0.hi;
                }
                put_row<NC>(Vw, x);
            }
            __syncthreads();
            for (int it = 0; it < REFINE_ROUNDS; ++it) {
                rowvec<NC>(zs, zsc, Vw, P);                                     // Z w
                __syncthreads();
                if (grp == 0) {
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc)
                        x[cc] = live ? psum(cc).hi : 0.f;
                    put_row<NC>(Vt, x);
                }
                __syncthreads();
                rowvec<NC>(zs, zsc, Vt, P);                                     // Z (Z w)
                __syncthreads();
                if (grp == 0) {
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) {
                        const FF zz = psum(cc);
                        const FF res = ff_add(ff_add(FF{2.f * Vz[row * VL + cc], 0.f}, ff_neg(Wd[cc * NMAX + row])),
                                              ff_neg(zz));
                        x[cc] = (live && cc < nc) ? res.hi : 0.f;
                    }
                    put_row<NC>(Vt, x);
                }
                __syncthreads();
                rowvec<NC>(xs, TMEM_INV, Vt, P);                                // X r
                __syncthreads();
                if (grp == 0) {
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) {
                        FF w = Wd[cc * NMAX + row];
                        if (live && cc < nc) w = ff_add(w, psum(cc));
                        Wd[cc * NMAX + row] = w;
                        x[cc] = w.hi;
                    }
                    put_row<NC>(Vw, x);
                }
                __syncthreads();
            }
            if (live) {
                for (int cc = 0; cc < nc; ++cc) {
                    const int kc = c.cpos[b0 + cc];
                    // d = (delta - w) / 2 as a float pair (halving is exact)
                    FF d = ff_add(FF{row == kc ? 1.f : 0.f, 0.f}, ff_neg(Wd[cc * NMAX + row]));
                    d = FF{0.5f * d.hi, 0.5f * d.lo};
                    if (!isfinite(d.hi)) set_error(a.err, GB_ERR_NAN);
                    a.Dval[c.ocol[b0 + cc] + row] = f2d(d.hi) + f2d(d.lo);
                    if (row == kc) {
                        c.tv[T_DHI][b0 + cc] = d.hi;
                        c.tv[T_DLO][b0 + cc] = d.lo;
                    }
                }
            }
            __syncthreads();
        }
    }

    // core columns of the product P (left + right, TMEM words) times k into
    // out[ocol + row]; on the core diagonal the word times tk goes to trace
    // term `term`.  Warps of column group 0.
    __device__ void core_columns(int ncore, float k, double* out, int term, float tk) {
        if (grp != 0) return;
        for (int b0 = 0; b0 < ncore; b0 += 16) {
            const int nc = min(16, ncore - b0);
            float g[16], h[16];
            tmem_ld_cols<16>(col(pl) + lane_off, c.cpos + b0, nc, g);
            tmem_ld_cols<16>(col(pr) + lane_off, c.cpos + b0, nc, h);
            if (row < n) {
#pragma unroll
                for (int cc = 0; cc < 16; ++cc) {
                    if (cc < nc) {
                        const float v = g[cc] + h[cc];
                        out[c.ocol[b0 + cc] + row] = f2d(v * k);
                        if (row == c.cpos[b0 + cc]) c.tv[term][b0 + cc] = v * tk;
                    }
                }
            }
        }
    }

    // largest diagonal word of the product P over rows < n into c.wred[0..3]
    // (warps of column group 0; a barrier must follow before reading it)
    __device__ void diag_max() {
        if (grp != 0) return;
        const uint32_t cb = (uint32_t)(row & ~31);
        if ((int)cb >= npad) {  // a warp of padding rows: its 32-column window may lie past the
            if ((threadIdx.x & 31) == 0) c.wred[threadIdx.x >> 5] = 0.f;  // TMEM allocation
            return;
        }
        float u[16], w[16], u2[16], w2[16];
        tmem_ld16x2(col(pl) + lane_off + cb, col(pl) + lane_off + cb + 16, u, w);
        tmem_ld16x2(col(pr) + lane_off + cb, col(pr) + lane_off + cb + 16, u2, w2);
        float d = 0.f;
        const int j = row & 31;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            d = (j == q) ? u[q] + u2[q] : d;
            d = (j == q + 16) ? w[q] + w2[q] : d;
        }
        d = row < n ? d : 0.f;
        for (int o = 16; o > 0; o >>= 1) d = fmaxf(d, __shfl_down_sync(0xffffffffu, d, o));
        if ((threadIdx.x & 31) == 0) c.wred[threadIdx.x >> 5] = d;
    }

    // pull the next subgraph's gathered blocks toward L2 while this one runs
    __device__ void prefetch_blocks(int32_t i) {
        if (i >= a.n_sub) return;
        const int64_t ni = a.sub_ptr[i + 1] - a.sub_ptr[i];
        const int64_t np = (ni + 15) & ~(int64_t)15;
        const int64_t bytes = np * np * (int64_t)sizeof(float);
        for (int b = 0; b <= (diag_h1 ? 0 : a.m); ++b) {
            const char* base = (const char*)(a.hblk + (int64_t)b * a.hblk_stride + a.boff[i]);
            for (int64_t o = (int64_t)threadIdx.x * 128; o < bytes; o += (int64_t)THREADS * 128)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(base + o));
        }
    }

    // staged operand from a gathered block beta M (FP32, column groups of four):
    // scale x blk, scale = 2^-(s+1) [x sigma] (exact power of two), and, with
    // use_diag, the diagonal dscale x c.dg (the x0 diagonal computed in FP64)
    // Staged operand sg times 2^e in place (its hi and lo parts scale exactly
    // unless a lo part is subnormal, ~2^-36 of the value): the same units as
    // combine.  Every thread; the next gemm's barrier orders it.
    __device__ void scale_staged(int sg, int e) {
        const int nu = npad / 8;
        for (int u = grp; u < nu; u += GROUPS) {
            uint4* p = (uint4*)(st(sg) + elem_off(row, 8 * u));
            uint4* q = (uint4*)((uint8_t*)p + lo_off);
            uint4 h = *p, l = *q;
            uint32_t* hv = (uint32_t*)&h;
            uint32_t* lv = (uint32_t*)&l;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (fmt == 0) {
                    const __half2 f = __float2half2_rn(ldexpf(1.f, e));
                    __half2 a = *(__half2*)&hv[j], b = *(__half2*)&lv[j];
                    a = __hmul2(a, f);
                    b = __hmul2(b, f);
                    hv[j] = *(uint32_t*)&a;
                    lv[j] = *(uint32_t*)&b;
                } else {
                    const __nv_bfloat162 f = __float2bfloat162_rn(ldexpf(1.f, e));
                    __nv_bfloat162 a = *(__nv_bfloat162*)&hv[j], b = *(__nv_bfloat162*)&lv[j];
                    a = __hmul2(a, f);
                    b = __hmul2(b, f);
                    hv[j] = *(uint32_t*)&a;
                    lv[j] = *(uint32_t*)&b;
                }
            }
            *p = h;
            *q = l;
        }
    }

    // 8-column units as in combine (unit u to column group u mod 3); all of a
    // thread's global loads are issued before the first conversion.
    __device__ void stage_dense(const float* blk, float scale, bool use_diag, float dscale, int sg) {
        constexpr int MAXU = (NPMAX / 8 + GROUPS - 1) / GROUPS;
        const float k = scale * STAGE_SCALE;
        const bool has_diag = use_diag && row < n;
        const float dv = has_diag ? c.dg[row] * dscale * STAGE_SCALE : 0.f;
        const int nu = npad / 8;
        float4 x[MAXU][2];
#pragma unroll
        for (int i = 0; i < MAXU; ++i) {
            const int u = grp + GROUPS * i;
            if (u < nu && row < npad) {
                x[i][0] = *(const float4*)(blk + ((size_t)(2 * u) * npad + row) * 4);
                x[i][1] = *(const float4*)(blk + ((size_t)(2 * u + 1) * npad + row) * 4);
            } else {
                x[i][0] = x[i][1] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int i = 0; i < MAXU; ++i) {
            const int u = grp + GROUPS * i;
            if (u >= nu) break;
            const int c0 = 8 * u;
            float v[8] = {x[i][0].x * k, x[i][0].y * k, x[i][0].z * k, x[i][0].w * k,
                          x[i][1].x * k, x[i][1].y * k, x[i][1].z * k, x[i][1].w * k};
            if (has_diag && (unsigned)(row - c0) < 8u) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (c0 + j == row) v[j] = dv;
            }
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) split_pair(v[2 * j], v[2 * j + 1], fmt, hi[j], lo[j]);
            uint8_t* p = st(sg) + elem_off(row, c0);
            *(uint4*)p = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *(uint4*)(p + lo_off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
    }

    // staged operand sg <- scale x diag(d) (d[r]: the FP32 diagonal of beta h1
    // at row r), zero elsewhere: what stage_dense writes for a diagonal block
    __device__ void stage_diag(const float* d, float scale, int sg) {
        const float dv = row < n ? d[row] * (scale * STAGE_SCALE) : 0.f;
        const int nu = npad / 8;
        for (int u = grp; u < nu; u += GROUPS) {
            const int c0 = 8 * u;
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = c0 + j == row ? dv : 0.f;
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) split_pair(v[2 * j], v[2 * j + 1], fmt, hi[j], lo[j]);
            uint8_t* p = st(sg) + elem_off(row, c0);
            *(uint4*)p = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *(uint4*)(p + lo_off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
    }
};

__global__ void __launch_bounds__(THREADS, GB_SPLIT_MINB) GB_SPLIT_KERNEL(PassArgs a) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    Ctl& c = *(Ctl*)(smem + NSTAGE * STAGE_BYTES);
    Kernel K(a, c, smem);

    // zero the staged operands once (rows >= n stay zero afterwards)
    for (uint32_t e = threadIdx.x; e < NSTAGE * STAGE_BYTES / 16; e += THREADS)
        ((uint4*)smem)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x == 0) {
        c.abort = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(K.mbar) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(K.mbar_bulk) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&c.tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    K.tbase = c.tmem_base;

    // this launch's subgraphs: a size class's list, or all of them (those
    // above NMAX belong to the tiled kernel and are skipped).  Dynamic
    // scheduling: thread 0 claims work items from the launch's counter, one
    // ahead of the item in flight so that its blocks can be prefetched.
#if GB_SPLIT_LIST
    const int32_t nwork = *a.work_n;
#define GB_ITEM(j) a.work[j]
#else
    const int32_t nwork = a.n_sub;
#define GB_ITEM(j) (j)
#endif
    if (threadIdx.x == 0) {
        c.cur = atomicAdd(a.counter, 1);
        c.nxt = atomicAdd(a.counter, 1);
    }
    for (bool first = true;; first = false) {
        if (!first) {
            __syncthreads();
            if (threadIdx.x == 0) {
                c.cur = c.nxt;
                c.nxt = atomicAdd(a.counter, 1);
            }
        }
        __syncthreads();
        const int32_t j = c.cur, jn = c.nxt;
        if (j >= nwork || c.abort) break;
        const int32_t i = GB_ITEM(j);
        const int64_t s0 = a.sub_ptr[i];
        const int n = (int)(a.sub_ptr[i + 1] - s0);
        if (n > NMAX) continue;
        const int64_t c0 = a.core_ptr[i], c1 = a.core_ptr[i + 1];
        K.set_size(n);
        const int ncore = (int)(c1 - c0);
        for (int e = threadIdx.x; e < ncore; e += THREADS) {
            c.cpos[e] = a.core_pos[c0 + e];
            c.ocol[e] = a.col_ptr[a.core_idx[c0 + e]];
        }
        if (jn < nwork) K.prefetch_blocks(GB_ITEM(jn));
        // the subgraph's scalars, once (FP64 is narrow on this part): step
        // count s, and sigma_r = 2^-k with (beta / 2) sigma max row sum |h1_r| <= 1
        if (threadIdx.x == 0) c.s = recursion_steps(a.beta, a.mu, a.eps_lo[i], a.eps_hi[i], a.min_steps);
        if (threadIdx.x < a.m) {
            const double h1max = a.h1max[(int64_t)i * a.m + threadIdx.x];
            int k = 0;
            double sig = 1.0;
            while (0.5 * a.beta * sig * h1max > 1.0 && k < 100) {
                sig *= 0.5;
                ++k;
            }
            c.sigk[threadIdx.x] = k;
        }
        __syncthreads();
        int s = c.s;
        if (K.grp == 0)
            c.dg[K.row] = K.row < n ? (float)(ldexp(a.beta, -(s + 1)) * (a.hdiag[s0 + K.row] - a.mu)) : 0.f;
        __syncthreads();
        // the response state Z1 of the subgraph in flight: this CTA's scratch
        // (rewritten every step, so it stays in L2)
        uint8_t* z1base = (uint8_t*)a.z1pool + (size_t)blockIdx.x * (a.m > 0 ? a.m : 1) * STAGE_BYTES;

        // ---- Taylor start: Q = x0^2, T = I - Q/3 + 2 Q^2/15 (X region: Q, Z region: T) ----
        const float* hb = a.hblk + a.boff[i];
        K.stage_dense(hb, ldexpf(1.f, -(s + 1)), true, 1.f, 0);          // S0 = x0
        if (!K.gemm(0, 0)) break;                                         // P = Q
        // rho(x0)^2 = rho(Q) <= max_r sum_c |Q_rc| (Gershgorin on the square is
        // tighter than on h): drop k steps while 2^k x0 keeps spectral radius <= 1
        const int k = K.fewer_steps(s - a.min_steps);
        float qscale = 1.f;
        if (k > 0) {
            s -= k;
            qscale = ldexpf(1.f, 2 * k);
            K.scale_staged(0, k);                                          // S0 = 2^k x0
        }
        K.combine(K.Pk(qscale), K.none(), 0.f, K.xc, 1, nullptr);          // X region = Q, S1 = Q
        if (!K.gemm(1, 1)) break;                                         // P = Q^2
        K.combine(K.T(K.xc, -1.f / 3.f), K.Pk(2.f / 15.f), 1.f, K.zc, -1, nullptr);  // Z region = T
        bool ok = true;
        for (int r = 0; r < a.m && ok; ++r) {
            // the perturbation, normalised by sigma_r
            const float* h1b = a.hblk + (int64_t)(1 + r) * a.hblk_stride + a.boff[i];
            const float x1scale = ldexpf(1.f, -(s + 1) - c.sigk[r]);
            // dZ0 = X1 T + x0 T1,  T1 = -Q1/3 + (2/15)(Q Q1 + Q1 Q),  Q1 = x0 X1 + X1 x0
            const float* h1d = a.h1d + (int64_t)r * a.h1d_stride + s0;
            if (K.diag_h1) K.stage_diag(h1d, x1scale, 1);                  // S1 = X1
            else K.stage_dense(h1b, x1scale, false, 0.f, 1);
            if (!(ok = K.gemm2(0, 1, 1, 0))) break;                        // P = Q1
            K.combine(K.Pk(1.f), K.none(), 0.f, -1, 1, nullptr);           // S1 = Q1
            K.combine(K.T(K.xc, 1.f), K.none(), 0.f, -1, 2, nullptr);      // S2 = Q
            if (!(ok = K.gemm2(2, 1, 1, 2))) break;                        // P = Q Q1 + Q1 Q
            K.combine(K.S(1, -1.f / 3.f), K.Pk(2.f / 15.f), 0.f, -1, 1, nullptr);  // S1 = T1
            if (!(ok = K.gemm(0, 1))) break;                               // P = x0 T1
            K.combine(K.T(K.zc, 1.f), K.none(), 0.f, -1, 2, nullptr);      // S2 = T
            if (K.diag_h1) K.stage_diag(h1d, x1scale, 1);                  // S1 = X1
            else K.stage_dense(h1b, x1scale, false, 0.f, 1);
            if (!(ok = K.gemm(1, 2, true))) break;                         // P += X1 T
            K.combine(K.Pk(1.f), K.none(), 0.f, -1, -1, z1base + (size_t)r * STAGE_BYTES);
        }
        if (!ok) break;
        K.combine(K.T(K.zc, 1.f), K.none(), 0.f, -1, 2, nullptr);          // S2 = T
        if (!K.gemm(0, 2)) break;                                         // P = Z0 = x0 T
        K.combine(K.Pk(1.f), K.none(), 0.f, K.zc, 0, nullptr);             // Z region = Z0, S0 = Z0

        // ---- doublings: Z <- 2 X Z, X = (I + Z^2)^-1 ----
        for (int step = 0; step < s && ok; ++step) {
            const bool last = step == s - 1;
            // S0 = Z on entry (staged with the Z region by the previous step)
            if (!(ok = K.gemm(0, 0))) break;                                       // P = Y = Z^2
            K.combine(K.Pk(1.f), K.none(), 0.f, -1, 1, nullptr);                   // S1 = Y
            // Y^2 (hi parts: it only seeds Newton-Schulz) into the X region, so P keeps Y
            if (!(ok = K.gemm(1, 1, false, true, 0, (int)K.xc))) break;
            K.combine(K.Pk(-80.f / 99.f), K.T(K.xc, 32.f / 99.f), 98.f / 99.f, K.xc, 2, nullptr);  // X0
            for (int j = 0; j < a.ns_iters && ok; ++j) {
                // Before the last correction X R only needs a few digits: |R| is
                // about 1e-2 after the Chebyshev start, so the hi parts alone leave
                // an error ~2^-11 |R| in X, which the next correction squares.
                const bool rough = j + 1 < a.ns_iters;
                if (!(ok = K.gemm(1, 2))) break;                                   // P = Y X
                if (rough) {
                    // R_hi alone, parked in the lo half of S2 (X_hi R_hi reads
                    // neither X_lo nor R_lo): S0 keeps Z
                    K.combine(K.T(K.xc, -1.f), K.Pk(-1.f), 1.f, -1, -1, nullptr, 2);  // R = (I - X) - Y X
                    if (!(ok = K.gemm(2, 2, false, true, K.lo_off))) break;          // P = X_hi R_hi
                } else {
                    // the last correction: R where Y was (Y is done) except in
                    // the last step, which still needs Y
                    const int sr = last ? 0 : 1;
                    K.combine(K.T(K.xc, -1.f), K.Pk(-1.f), 1.f, -1, sr, nullptr);  // S_sr = R
                    if (!(ok = K.gemm(2, sr))) break;                              // P = X R
                    if (sr == 1 && a.m > 0) K.bulk_load(1, z1base);                // S1 <- Z1 (R done)
                }
                if (rough) K.combine(K.T(K.xc, 1.f), K.T(K.pl, 1.f), 0.f, K.xc, 2, nullptr);     // X += X R, S2 = X
                else K.combine(K.T(K.xc, 1.f), K.Pk(1.f), 0.f, K.xc, 2, nullptr);
            }
            if (!ok) break;
            if (last) {
                // d (I - d) = (I - Z_s^2) / 4 = ((I - Y) X)^2 / 4: no cancellation
                // near saturation (Y = Z_{s-1}^2, X = (I + Y)^-1)
                K.combine(K.S(1, -1.f), K.none(), 1.f, -1, 1, nullptr);            // S1 = I - Y
                if (!(ok = K.gemm(1, 2))) break;                                   // P = G = (I - Y) X
                K.combine(K.Pk(1.f), K.none(), 0.f, -1, 1, nullptr);               // S1 = G
                if (!(ok = K.gemm(1, 1))) break;                                   // P = G^2
                K.core_columns(ncore, (float)(0.25 * a.beta) * TMEM_INV, a.d1mu_val, T_DD,
                               0.25f * TMEM_INV);                                  // d1_mu = beta G^2 / 4
                K.diag_max();
            }
            if (last || a.ns_iters < 1) K.combine(K.T(K.zc, 1.f), K.none(), 0.f, -1, 0, nullptr);  // S0 = Z
            if (!(ok = K.gemm(2, 0))) break;                                       // P = W / 2 = X Z
            if (last) {
                // ---- the last doubling redone on the core columns (CUDA cores) ----
                // (the small configuration's two slots hold the scratch of 8 columns)
                if (ncore <= 8 || NPMAX < 128) K.refine_core<8>(K.zc, K.xc, TMEM_INV, ncore);
                else K.refine_core<NPMAX < 128 ? 8 : 16>(K.zc, K.xc, TMEM_INV, ncore);
                if (a.m > 0) K.combine(K.Pk(2.f), K.none(), 0.f, -1, 0, nullptr);  // S0 = W
            } else {
                K.combine(K.Pk(2.f), K.none(), 0.f, K.zc, 0, nullptr);             // Z region = W (next Z), S0 = W
            }
            for (int r = 0; r < a.m && ok; ++r) {
                // Z1 <- 2 X Z1 X - (W Z1 / 2) W
                uint8_t* z1 = z1base + (size_t)r * STAGE_BYTES;
                if (r > 0 || last || a.ns_iters < 1) K.bulk_load(1, z1);          // S1 <- Z1
                if (!(ok = K.wait_bulk())) break;                                  // S1 = Z1
                if (!(ok = K.gemm(2, 1))) break;                                   // P = X Z1
                K.combine(K.Pk(2.f), K.none(), 0.f, K.xc, -1, nullptr);            // X region = 2 X Z1
                if (!(ok = K.gemm(0, 1))) break;                                   // P = W Z1
                K.combine(K.Pk(-0.5f), K.none(), 0.f, -1, 1, nullptr);             // S1 = -W Z1 / 2
                if (!(ok = K.gemm(1, 0))) break;                                   // P = -(W Z1 / 2) W
                K.combine(K.T(K.xc, 1.f), K.none(), 0.f, -1, 1, nullptr);          // S1 = 2 X Z1
                if (!(ok = K.gemm(1, 2, true))) break;                             // P += (2 X Z1) X
                if (!last) {
                    K.combine(K.Pk(1.f), K.none(), 0.f, -1, -1, z1);               // Z1 -> global
                } else {
                    const float sc = -ldexpf(0.5f, c.sigk[r]) * TMEM_INV;          // d1_lambda = -Z1_s / (2 sigma)
                    K.core_columns(ncore, sc, a.D1val[r], T_L0 + r, sc);
                }
            }
        }
        if (!ok) break;

        // per-subgraph core traces: the core terms summed in FP64 in a fixed
        // order (deterministic), one slot per thread
        __syncthreads();
        if (threadIdx.x < TR_FIXED + a.m) {
            const int sl = threadIdx.x;
            double v = 0.0;
            if (sl == TR_D) {
                for (int e = 0; e < ncore; ++e) v += (double)c.tv[T_DHI][e] + (double)c.tv[T_DLO][e];
            } else if (sl == TR_DD || sl == TR_D1MU) {
                for (int e = 0; e < ncore; ++e) v += (double)c.tv[T_DD][e];
                if (sl == TR_D1MU) v *= a.beta;
            } else if (sl == TR_FLOPS) {
                v = pass_gemm_flops(n, s, a.ns_iters, a.m);
            } else if (sl == TR_FLOPS_S) {
                v = pass_flops_per_step_count(n, ncore, s, a.ns_iters, a.m);
            } else if (sl == TR_MAXWC) {
                float g = 0.f;
                for (int e = 0; e < ncore; ++e) g = fmaxf(g, c.tv[T_DD][e]);
                v = a.beta * (double)g;
            } else if (sl == TR_MAXW) {
                float g = c.wred[0];
                for (int w = 1; w < 4; ++w) g = fmaxf(g, c.wred[w]);
                v = 0.25 * a.beta * (double)g * (double)TMEM_INV;
            } else {
                for (int e = 0; e < ncore; ++e) v += (double)c.tv[T_L0 + sl - TR_D1LAM][e];
            }
            a.tr[(int64_t)i * a.tr_stride + sl] = v;
        }
        if (threadIdx.x == 0) a.steps_out[i] = s;
        fence_before();
        __syncthreads();
        fence_after();
    }
#undef GB_ITEM
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(K.tbase), "r"(TMEM_COLS)
                     : "memory");
}

#if GB_SPLIT_NPMAX == 128 && !GB_SPLIT_LIST
// Dense principal submatrices beta h^(i) = beta H[S_i, S_i] and beta h1_r^(i)
// (FP32 in column groups of four, zero padding to npad), the FP64 diagonal of
// h^(i), one block per subgraph, one warp per row.  Also the Gershgorin
// interval of h^(i) (eps_lo/eps_hi, FP32 sums widened to an enclosure; this
// path needs no separate bounds kernel) and the largest row sum of |h1_r^(i)| (h1max[i * m + r], an upper bound: FP32 sums
// widened by 2^-16), which fixes the perturbation's normalisation in the
// recursion.  Per element only integer and FP32 work: the value is converted
// by d2f_rn and scaled by beta in FP32 (within 1.5 float ulps of beta x).
__global__ void __launch_bounds__(256) k_gather_dense(PassArgs a, float* hblk, double* hdiag) {
    __shared__ int32_t S[GB_BIG_MAX_N];
    __shared__ float wmax[8], wlo[8], whi[8], wab[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float bf = d2f_rn(a.beta);
    const bool diag_h1 = a.m > 0 && a.h1_offdiag && *a.h1_offdiag == 0;
    for (int32_t i = blockIdx.x; i < a.n_sub; i += gridDim.x) {
        const int64_t s0 = a.sub_ptr[i];
        const int n = (int)(a.sub_ptr[i + 1] - s0);
        const int npad = (n + 15) & ~15;
        // diagonal perturbations of a one-tile subgraph: only their diagonal
        const bool d1 = diag_h1 && n <= NMAX;
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
            S[r] = a.sub_idx[s0 + r];
            hdiag[s0 + r] = 0.0;
            if (d1)
                for (int b = 0; b < a.m; ++b) a.h1d[(int64_t)b * a.h1d_stride + s0 + r] = 0.f;
        }
        // blocks start on 64-element boundaries: zero them 16 bytes at a time
        for (int b = 0; b <= (d1 ? 0 : a.m); ++b) {
            float4* blk4 = (float4*)(hblk + (int64_t)b * a.hblk_stride + a.boff[i]);
            for (int e = threadIdx.x; e < npad * npad / 4; e += blockDim.x) blk4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        for (int b = 0; b <= a.m; ++b) {
            const int64_t* ptr = b == 0 ? a.Hptr : a.H1ptr[b - 1];
            const int32_t* idx = b == 0 ? a.Hidx : a.H1idx[b - 1];
            const double* val = b == 0 ? a.Hval : a.H1val[b - 1];
            float* blk = hblk + (int64_t)b * a.hblk_stride + a.boff[i];
            float rmax = 0.f;
            float glo = INFINITY, ghi = -INFINITY, gab = 0.f;  // Gershgorin interval (b = 0)
            for (int r = warp; r < n; r += blockDim.x / 32) {
                const int32_t g = S[r];
                float rs = 0.f, rad = 0.f, dgf = 0.f;
                for (int64_t p = ptr[g] + lane; p < ptr[g + 1]; p += 32) {
                    const int32_t col = idx[p];
                    int lo = 0, hi = n;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (S[mid] < col) lo = mid + 1; else hi = mid;
                    }
                    if (lo < n && S[lo] == col) {
                        const double x = val[p];
                        const float xf = d2f_rn(x), v = bf * xf;
                        if (b > 0 && d1) a.h1d[(int64_t)(b - 1) * a.h1d_stride + s0 + r] = v;  // lo == r
                        else blk[((size_t)(lo >> 2) * npad + r) * 4 + (lo & 3)] = v;
                        if (b == 0) {
                            if (lo == r) {
                                hdiag[s0 + r] = x;
                                dgf = xf;
                            } else {
                                rad += fabsf(xf);
                            }
                        }
                        rs += fabsf(v);
                    }
                }
                rmax = fmaxf(rmax, warp_sum_f(rs));  // lane 0 holds the row sum
                if (b == 0) {
                    // Gershgorin row (every lane gets the sums)
                    for (int o = 16; o > 0; o >>= 1) {
                        rad += __shfl_xor_sync(0xffffffffu, rad, o);
                        dgf += __shfl_xor_sync(0xffffffffu, dgf, o);  // one lane holds it
                    }
                    glo = fminf(glo, dgf - rad);
                    ghi = fmaxf(ghi, dgf + rad);
                    gab = fmaxf(gab, fabsf(dgf) + rad);
                }
            }
            if (b == 0) {
                if (lane == 0) {
                    wlo[warp] = glo;
                    whi[warp] = ghi;
                    wab[warp] = gab;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    for (int w = 1; w < (int)(blockDim.x / 32); ++w) {
                        glo = fminf(glo, wlo[w]);
                        ghi = fmaxf(ghi, whi[w]);
                        gab = fmaxf(gab, wab[w]);
                    }
                    // FP32 terms within 2^-24 each, < n of them per radius:
                    // widening by (n + 2) 2^-23 of max(|h_rr| + radius) keeps an
                    // enclosure (2^-16 up to 128 orbitals)
                    const double wd = (double)gab * fmax(0x1p-16, (double)(n + 2) * 0x1p-23);
                    a.eps_lo[i] = (double)glo - wd;
                    a.eps_hi[i] = (double)ghi + wd;
                }
                __syncthreads();
            }
            if (b > 0) {
                if (lane == 0) wmax[warp] = rmax;
                __syncthreads();
                if (threadIdx.x == 0) {
                    float v = wmax[0];
                    for (int w = 1; w < (int)(blockDim.x / 32); ++w) v = fmaxf(v, wmax[w]);
                    // sum of |beta h1| in FP32 (<= n terms, each within 2^-23)
                    a.h1max[(int64_t)i * a.m + (b - 1)] =
                        (double)v * (1.0 + fmax(0x1p-16, (double)(n + 2) * 0x1p-22)) / a.beta;
                }
                __syncthreads();
            }
        }
        __syncthreads();
    }
}

#endif  // GB_SPLIT_NPMAX == 128

}  // namespace

#if GB_SPLIT_NPMAX == 128 && !GB_SPLIT_LIST
int launch_split_gather(gb_handle* h, const PassArgs& a, float* hblk, double* hdiag) {
    const int grid = a.n_sub < 152 * 8 ? a.n_sub : 152 * 8;
    GB_LAUNCH(h, k_gather_dense, grid, 256, 0, a, hblk, hdiag);
    return GB_OK;
}

#endif

static int split_launch(gb_handle* h, const PassArgs& a, cudaStream_t stream) {
    static bool configured = false;
    if (!configured) {
        GB_CUDA(cudaFuncSetAttribute(GB_SPLIT_KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
        configured = true;
    }
    int sms = 0;
    GB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    if (a.grid_sms > 0 && a.grid_sms < sms) sms = a.grid_sms;
    // persistent: GB_SPLIT_MINB CTAs per SM, within the response scratch
    // (min(n_sub, GB_SPLIT_MAX_CTAS) x 64 KB per RHS; a CTA takes STAGE_BYTES)
    const int64_t cap = (int64_t)(a.n_sub < GB_SPLIT_MAX_CTAS ? a.n_sub : GB_SPLIT_MAX_CTAS) * 65536 / STAGE_BYTES;
    int64_t grid = (int64_t)GB_SPLIT_MINB * sms;
    if (grid > a.n_sub) grid = a.n_sub;
    if (grid > cap) grid = cap;
    GB_LAUNCH_ON(h, stream, GB_SPLIT_KERNEL, (int)grid, THREADS, SMEM_BYTES, a);
    return GB_OK;
}

int GB_SPLIT_LAUNCH(gb_handle* h, const PassArgs& a) { return split_launch(h, a, h->stream); }

#if GB_SPLIT_NPMAX == 128 && !GB_SPLIT_LIST
int launch_split_pass_on(gb_handle* h, const PassArgs& a, cudaStream_t stream) {
    return split_launch(h, a, stream);
}
#endif
