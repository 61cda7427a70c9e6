// Split-precision Fermi / response recursion on the tensor cores for
// subgraphs of more than 128 orbitals (npad = round16(|S_i|) up to
// GB_BIG_MAX_N).  Same recursion, splits, schedule and scaling as the
// one-tile kernel (mixed.cu): Taylor start, doublings Z <- 2 X Z with
// X = (I + Z^2)^-1 from a Chebyshev start and Newton-Schulz corrections, the
// exact derivative of the recursion for each right-hand side, d1_mu =
// beta ((I - Y) X)^2 / 4, and the last doubling redone on the core columns
// on the CUDA cores.  What changes is where the state lives: a subgraph no
// longer fits in one CTA's tensor memory, so its matrices stay in this CTA's
// scratch in global memory (L2) and every product is computed tile by tile.
//
// Layouts (per subgraph; nrb = ceil(npad / 128) row blocks of 128 rows):
//  * staged image of a matrix (2^12 x value, FP16 or BF16 hi and lo parts):
//    part p at p * nrb * 128 * npad * 2 bytes; element (r, c) at
//    (r / 128) * (128 * npad * 2) + (c / 8) * 2048 + (r % 128) * 16 + (c % 8) * 2.
//    Within a row block this is the one-tile kernel's shared-memory operand
//    layout (8 x 8 core matrices, no swizzle): an A chunk (128 rows x 64
//    columns) is one contiguous 16 KB copy per part, and each 8-column group
//    of a B chunk (64 rows x 8 columns) one contiguous 1 KB copy.
//  * FP32 matrix (2^24 x value, the tensor-memory unit of the one-tile
//    kernel): element (r, c) at (r / 128) * 128 * npad + c * 128 + r % 128,
//    so the 32 lanes of a warp (32 consecutive rows) touch 128 contiguous
//    bytes.
// Every image and FP32 matrix is written in full, zero outside the n x n
// block, so products over the padding vanish and only the identity needs a
// mask (as in the one-tile kernel).
//
// Product tile: 128 rows x up to NT = 128 columns; per 16-wide K step
//   [left | right] += A_hi [B_hi | B_lo]   (one instruction, N = 2 NT)
//   right          += A_lo B_hi
// (the one-tile kernel's packing: the left accumulator holds only the large
// A_hi B_hi terms), with left split in two accumulators by K chunk (see
// mma_chunk: the tensor cores' FP32 accumulation rounds toward zero, and the
// many K steps of a large subgraph would otherwise bias the products
// toward zero).  Thread 0 runs a three-stage ring of 64-wide K chunks
// (bulk copies completing on mbarriers, MMAs releasing the stage through
// tcgen05.commit) and issues the MMAs; then all 8 warps (4 TMEM lane
// quadrants x 2 column halves) run the tile's epilogue, which adds the
// product to FP32 sources and the identity and writes FP32 and/or staged
// outputs.  The operands of a product and its outputs are distinct buffers.
#include "density.cuh"
#include "tc.cuh"

namespace {

constexpr int BT = 256;                             // threads per CTA
constexpr int KC = 64;                              // K chunk of one stage
constexpr int NT = 128;                             // output columns per tile
constexpr int NSTG = 3;                             // pipeline stages
constexpr uint32_t A_PART = 128u * KC * 2u;         // one part of an A chunk (16 KB)
constexpr uint32_t B_PART = (uint32_t)KC * NT * 2u; // one part of a B chunk (16 KB)
constexpr uint32_t STG_BYTES = 2u * A_PART + 2u * B_PART;
constexpr uint32_t TMEM_COLS = 4 * NT;              // [left_a | right | left_b] of one tile (3 NT used)
constexpr float STAGE_SCALE = 4096.f;               // staged value = 2^12 x value
constexpr float TMEM_SCALE = 16777216.f;            // FP32 state = 2^24 x value
constexpr float TMEM_INV = 1.f / 16777216.f;

// staged images of the scratch (then 2 per right-hand side: Z1 ping-pong)
enum Img { I_X0 = 0, I_Q, I_T, I_Y, I_XA, I_XB, I_ZA, I_ZB, I_R, I_IY, I_G, I_X1, I_Q1, I_T1, I_A, I_U, I_Z1 };
static_assert(I_Z1 == GB_BIG_IMAGES_FIXED, "image count");
enum F32Mat { F_Z = 0, F_X, F_Y, F_W };
static_assert(F_W + 1 == GB_BIG_F32, "FP32 matrix count");
// per-core-vertex trace terms, kept in the scratch
enum CoreTerm { T_DHI = 0, T_DLO = 1, T_DD = 2, T_L0 = 3, T_COUNT = 3 + GB_MAX_RHS };

struct __align__(16) Ctl {
    unsigned long long full[NSTG];   // chunk landed (transaction bytes)
    unsigned long long empty[NSTG];  // chunk's MMAs done (tcgen05.commit)
    unsigned long long accf;         // tile's MMAs done
    uint32_t tmem_base;
    int abort;
    int s;
    int kfew;
    int item;
    int dmax;                        // largest diagonal of G^2 (float bits, >= 0)
    int32_t sigk[GB_MAX_RHS];
    float part[2][128];              // row sums of the two column halves of a tile
    float rs[GB_BIG_MAX_N];          // row sums of |Q| (steps dropped by the bound on Q)
    int16_t cmap[GB_BIG_MAX_N];      // column -> core index in this subgraph, or -1
};

constexpr size_t SMEM_BYTES = NSTG * STG_BYTES + sizeof(Ctl) + 1024;

// A chunk (K-major): 8-column groups 2048 B apart, 8-row groups 128 B apart
__device__ __forceinline__ uint64_t desc_a(uint32_t saddr) { return desc_bits(saddr, 2048, 128); }
// B chunk (MN-major): 8-row groups (K) 128 B apart, 8-column groups (N) 1 KB apart
__device__ __forceinline__ uint64_t desc_b(uint32_t saddr) { return desc_bits(saddr, 128, 1024); }

// one product term A B of staged images (indices into the scratch)
struct Term {
    int a, b;
};

// Epilogue of a product: v = kp P + k1 F1 + ks1 S1 + cd I (TMEM units; S1
// read as hi + lo), written to an FP32 matrix and/or a staged image, or (core
// mode) the core columns of v times ck to a collected output with the
// diagonal times ctk as trace term cterm.  Optional: row sums of |v| (rows
// mode), the largest diagonal element (dmax mode).
struct Epi {
    float kp = 1.f;
    int f1 = -1;
    float k1 = 0.f;
    int s1 = -1;
    float ks1 = 0.f;
    float cd = 0.f;
    int fo = -1;
    int so = -1;
    bool rows = false;
    bool dmax = false;
    double* cout = nullptr;
    float ck = 0.f;
    int cterm = -1;
    float ctk = 0.f;
};

struct Big {
    const PassArgs& a;
    Ctl& c;
    uint8_t* stg;
    uint32_t stg_addr;
    uint32_t tbase;
    uint32_t gc;      // K chunks issued so far (thread 0's ring position)
    uint32_t accph;   // phase of accf
    int fmt;
    int row, grp;
    uint32_t lane_off;
    // this subgraph
    int n, npad, nrb;
    int64_t rbi;      // bytes of one image row block (128 npad 2)
    int64_t parti;    // bytes of one image part (nrb rbi)
    int64_t rbf;      // floats of one FP32 row block (128 npad)
    int64_t core0;
    int ncore;
    // this CTA's scratch
    uint8_t* base;
    int64_t img_bytes, f32_bytes;
    int nimg;

    __device__ Big(const PassArgs& a_, Ctl& c_, uint8_t* smem) : a(a_), c(c_) {
        stg = smem;
        stg_addr = smem_u32(smem);
        gc = 0;
        accph = 0;
        fmt = a.split_kind;
        row = threadIdx.x & 127;
        grp = threadIdx.x >> 7;
        lane_off = (uint32_t)((row & ~31) << 16);
        const int64_t nrbm = (a.big_npmax + 127) / 128;
        img_bytes = 2 * 128 * nrbm * a.big_npmax * 2;
        f32_bytes = 128 * nrbm * a.big_npmax * 4;
        nimg = GB_BIG_IMAGES_FIXED + 2 * a.m;
        base = a.big_scratch + (int64_t)blockIdx.x * a.big_stride;
    }

    __device__ void set_size(int n_) {
        n = n_;
        npad = (n + 15) & ~15;
        nrb = (npad + 127) / 128;
        rbi = (int64_t)128 * npad * 2;
        parti = nrb * rbi;
        rbf = (int64_t)128 * npad;
    }

    __device__ uint8_t* img(int k) const { return base + (int64_t)k * img_bytes; }
    __device__ float* f32(int k) const { return (float*)(base + (int64_t)nimg * img_bytes + (int64_t)k * f32_bytes); }
    __device__ float* tv(int term) const {
        return (float*)(base + (int64_t)nimg * img_bytes + (int64_t)GB_BIG_F32 * f32_bytes) +
               (int64_t)term * a.big_npmax;
    }
    __device__ int64_t ioff(int r, int c0) const {  // image byte offset of (r, c0), c0 % 8 == 0
        return (r >> 7) * rbi + (int64_t)(c0 >> 3) * 2048 + (r & 127) * 16;
    }
    __device__ int64_t foff(int r, int col) const { return (r >> 7) * rbf + (int64_t)col * 128 + (r & 127); }

    __device__ void fail(int status) {
        c.abort = 1;
        set_error(a.err, status);
    }

    // ---- thread 0: the K-chunk ring --------------------------------------
    // chunk q of a tile: term q / nkc, K columns [k0, k0 + kw)
    // (swap: the B parts land lo first, then hi, for an odd chunk; see mma_chunk)
    __device__ bool load_chunk(uint32_t g, const Term& t, int mt, int n0, int N, int k0, int kw, bool hh,
                               bool swap) {
        const uint32_t s = g % NSTG;
        if (g >= NSTG && !mbar_wait(smem_u32(&c.empty[s]), ((g / NSTG) - 1) & 1u)) return false;
        const uint32_t sa = stg_addr + s * STG_BYTES;
        const uint32_t sb = sa + 2 * A_PART;
        const int parts = hh ? 1 : 2;
        const uint32_t abytes = (uint32_t)kw * 256u, bbytes = (uint32_t)kw * 16u;
        const int ng = N / 8;
        const uint32_t total = parts * abytes + (uint32_t)parts * ng * bbytes;
        const uint32_t fb = smem_u32(&c.full[s]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(total) : "memory");
        const uint8_t* A = img(t.a) + mt * rbi + (int64_t)(k0 >> 3) * 2048;
        const uint8_t* B = img(t.b) + (k0 >> 7) * rbi + (int64_t)(n0 >> 3) * 2048 + (k0 & 127) * 16;
        for (int p = 0; p < parts; ++p) {
            bulk_copy(sa + p * A_PART, A + p * parti, abytes, fb);
            for (int gi = 0; gi < ng; ++gi)
                bulk_copy(sb + (uint32_t)(((swap ? 1 - p : p) * ng) + gi) * 1024u, B + p * parti + (int64_t)gi * 2048,
                          bbytes, fb);
        }
        return true;
    }

    __device__ static void bulk_copy(uint32_t sdst, const void* gsrc, uint32_t bytes, uint32_t mbar) {
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sdst),
            "l"(gsrc), "r"(bytes), "r"(mbar)
            : "memory");
    }

    // The large A_hi B_hi terms go to two accumulators, even chunks to left_a
    // (columns [0, N)) and odd chunks to left_b ([2N, 3N)), which the epilogue
    // adds in FP32 (round to nearest): each accumulator then takes half of the
    // K steps' round-toward-zero additions at about half the magnitude, which
    // halves their bias.  Even chunk: [left_a | right] += A_hi [B_hi | B_lo]
    // (B staged hi first); odd chunk: [right | left_b] += A_hi [B_lo | B_hi]
    // (B staged lo first); then right += A_lo B_hi.  q is the chunk's index in
    // the tile (the big kernel's tiles hold at least 3 chunks, so left_b is
    // always written).
    __device__ void mma_chunk(uint32_t g, int N, int kw, bool hh, int q) {
        const uint32_t s = g % NSTG;
        const uint32_t sa = stg_addr + s * STG_BYTES;
        const uint32_t sb = sa + 2 * A_PART;
        const uint32_t id1 = make_idesc(fmt, 0, N), id2 = make_idesc(fmt, 0, 2 * N);
        const bool odd = (q & 1) != 0;
        const uint32_t la = tbase, rt = tbase + (uint32_t)N, lb = tbase + 2u * (uint32_t)N;
        const uint32_t hi_grp = (uint32_t)(N / 8) * 1024u;  // the hi part of a swapped B chunk
        for (int ks = 0; ks < kw / 16; ++ks) {
            const uint64_t a_hi = desc_a(sa + (uint32_t)ks * 4096u);
            const uint64_t a_lo = desc_a(sa + A_PART + (uint32_t)ks * 4096u);
            const uint64_t b0 = desc_b(sb + (uint32_t)ks * 256u);
            const bool init = q <= 1 && ks == 0;  // the first K step of left_a / left_b
            if (hh) {
                mma_f16(odd ? lb : la, a_hi, b0, id1, init ? 0u : 1u);
            } else if (!odd) {
                mma_f16(la, a_hi, b0, id2, init ? 0u : 1u);
                mma_f16(rt, a_lo, b0, id1, 1u);
            } else {
                const uint64_t b_hi = desc_b(sb + hi_grp + (uint32_t)ks * 256u);
                if (init) {  // right accumulates, left_b starts: two instructions
                    mma_f16(rt, a_hi, b0, id1, 1u);
                    mma_f16(lb, a_hi, b_hi, id1, 0u);
                } else {
                    mma_f16(rt, a_hi, b0, id2, 1u);
                }
                mma_f16(rt, a_lo, b_hi, id1, 1u);
            }
        }
    }

    // thread 0: all chunks of one tile, then a commit to accf
    __device__ void issue_tile(const Term* t, int nt, int mt, int n0, int N, bool hh) {
        const int nkc = (npad + KC - 1) / KC;
        const int total = nt * nkc;
        const uint32_t g0 = gc;
        bool ok = true;
        int issued = 0, waited = 0;  // chunk loads issued / seen complete
        auto chunk = [&](int q, int& k0, int& kw) {
            k0 = (q % nkc) * KC;
            kw = min(KC, npad - k0);
        };
        for (int q = 0; q < total && q < NSTG - 1 && ok; ++q) {
            int k0, kw;
            chunk(q, k0, kw);
            ok = load_chunk(g0 + q, t[q / nkc], mt, n0, N, k0, kw, hh, (q & 1) && !hh);
            issued += ok;
        }
        for (int q = 0; q < total && ok; ++q) {
            const uint32_t g = g0 + q;
            int k0, kw;
            chunk(q, k0, kw);
            if (!mbar_wait(smem_u32(&c.full[g % NSTG]), (g / NSTG) & 1u)) {
                ok = false;
                break;
            }
            ++waited;
            mma_chunk(g, N, kw, hh, q);
            mma_commit(smem_u32(&c.empty[g % NSTG]));
            if (q + NSTG - 1 < total) {
                int k1, kw1;
                chunk(q + NSTG - 1, k1, kw1);
                ok = load_chunk(g + NSTG - 1, t[(q + NSTG - 1) / nkc], mt, n0, N, k1, kw1, hh,
                                ((q + NSTG - 1) & 1) && !hh);
                issued += ok;
            }
        }
        if (!ok) {
            fail(GB_ERR_TIMEOUT);
            // let the copies still in flight land (bounded) before the CTA
            // may exit: their shared memory must not be reused under them
            for (int q = waited; q < issued; ++q)
                mbar_wait(smem_u32(&c.full[(g0 + q) % NSTG]), ((g0 + q) / NSTG) & 1u);
        }
        gc = g0 + total;
        mma_commit(smem_u32(&c.accf));
    }

    // ---- one product P = sum_t A_t B_t, tile by tile, with its epilogue ----
    __device__ bool gemm(const Term* t, int nt, bool hh, const Epi& e) {
        const int nnt = (npad + NT - 1) / NT;
        for (int mt = 0; mt < nrb; ++mt) {
            for (int jt = 0; jt < nnt; ++jt) {
                const int n0 = jt * NT, N = min(NT, npad - n0);
                fence_proxy_async();
                fence_before();
                __syncthreads();
                if (threadIdx.x == 0) {
                    fence_after();
                    issue_tile(t, nt, mt, n0, N, hh);
                }
                __syncthreads();
                const bool ok = mbar_wait(smem_u32(&c.accf), accph);
                accph ^= 1u;
                fence_after();
                if (!ok) fail(GB_ERR_TIMEOUT);
                __syncthreads();
                if (c.abort) return false;
                epilogue(e, mt, n0, N, !hh);
            }
        }
        fence_before();
        __syncthreads();
        return c.abort == 0;
    }

    __device__ void split_store(uint8_t* dst, const float (&v)[8], float ks) const {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) split_pair(v[2 * j] * ks, v[2 * j + 1] * ks, fmt, hi[j], lo[j]);
        *(uint4*)dst = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *(uint4*)(dst + parti) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }

    __device__ void load_staged(const uint8_t* src, float (&w)[8]) const {
        const uint4 h4 = *(const uint4*)src, l4 = *(const uint4*)(src + parti);
        const uint32_t hw[4] = {h4.x, h4.y, h4.z, h4.w}, lw[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float2 h, l;
            if (fmt == 0) {
                h = __half22float2(*(const __half2*)&hw[j]);
                l = __half22float2(*(const __half2*)&lw[j]);
            } else {
                h = __bfloat1622float2(*(const __nv_bfloat162*)&hw[j]);
                l = __bfloat1622float2(*(const __nv_bfloat162*)&lw[j]);
            }
            w[2 * j] = h.x + l.x;
            w[2 * j + 1] = h.y + l.y;
        }
    }

    __device__ void epilogue(const Epi& e, int mt, int n0, int N, bool right) {
        const int r = mt * 128 + row;
        const float kd = e.cd * TMEM_SCALE;
        const bool diag = kd != 0.f && r < n;
        float rsum = 0.f, dmx = 0.f;
        const float* F1 = e.f1 >= 0 ? f32(e.f1) : nullptr;
        const uint8_t* S1 = e.s1 >= 0 ? img(e.s1) : nullptr;
        float* FO = e.fo >= 0 ? f32(e.fo) : nullptr;
        uint8_t* SO = e.so >= 0 ? img(e.so) : nullptr;
        for (int u = grp; u < N / 8; u += 2) {
            uint32_t r1[8], r2[8], r3[8];
            tmem_ld8_issue(tbase + lane_off + 8 * u, r1);                        // left_a
            tmem_ld8_issue(tbase + lane_off + 2 * N + 8 * u, r3);                // left_b
            if (right) tmem_ld8_issue(tbase + lane_off + N + 8 * u, r2);
            tmem_wait_ld();
            pin8(r1);
            pin8(r3);
            if (right) pin8(r2);
            const int c0 = n0 + 8 * u;
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float big = __uint_as_float(r1[j]) + __uint_as_float(r3[j]);
                const float p = big + (right ? __uint_as_float(r2[j]) : 0.f);
                v[j] = e.kp * p;
            }
            if (F1) {
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = fmaf(F1[foff(r, c0 + j)], e.k1, v[j]);
            }
            if (S1) {
                float w[8];
                load_staged(S1 + ioff(r, c0), w);
                const float k = e.ks1 * (TMEM_SCALE / STAGE_SCALE);
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = fmaf(w[j], k, v[j]);
            }
            if (diag && (unsigned)(r - c0) < 8u) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (c0 + j == r) v[j] += kd;
            }
            if (FO) {
#pragma unroll
                for (int j = 0; j < 8; ++j) FO[foff(r, c0 + j)] = v[j];
            }
            if (SO) split_store(SO + ioff(r, c0), v, STAGE_SCALE * TMEM_INV);
            if (e.rows) {
#pragma unroll
                for (int j = 0; j < 8; ++j) rsum += fabsf(v[j]);
            }
            if (e.dmax && r < n && (unsigned)(r - c0) < 8u) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (c0 + j == r) dmx = fmaxf(dmx, v[j]);
            }
            if (e.cout && r < n) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int ce = c.cmap[c0 + j];
                    if (ce >= 0) {
                        const int64_t oc = a.col_ptr[a.core_idx[core0 + ce]];
                        e.cout[oc + r] = f2d(v[j] * e.ck);
                        if (r == c0 + j) tv(e.cterm)[ce] = v[j] * e.ctk;
                    }
                }
            }
        }
        if (SO) fence_proxy_async_global();  // read back by bulk copies
        if (e.dmax && dmx > 0.f) atomicMax(&c.dmax, __float_as_int(dmx));
        if (e.rows) {
            c.part[grp][row] = rsum;
            __syncthreads();
            if (grp == 0 && r < npad) c.rs[r] += c.part[0][row] + c.part[1][row];
        }
        // the accumulator is read: the next tile may overwrite it
        tmem_wait_ld();
    }

    // ---- elementwise passes over the padded block ------------------------
    // FP32 matrix fo and/or image so = k F[f] + cd I (TMEM units); f < 0: only cd I
    __device__ void ew_stage(int f, float k, float cd, int fo, int so) {
        const float* F = f >= 0 ? f32(f) : nullptr;
        float* FO = fo >= 0 ? f32(fo) : nullptr;
        uint8_t* SO = so >= 0 ? img(so) : nullptr;
        const float kd = cd * TMEM_SCALE;
        for (int mt = 0; mt < nrb; ++mt) {
            const int r = mt * 128 + row;
            for (int u = grp; u < npad / 8; u += 2) {
                const int c0 = 8 * u;
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = F ? F[foff(r, c0 + j)] * k : 0.f;
                if (kd != 0.f && r < n && (unsigned)(r - c0) < 8u) {
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (c0 + j == r) v[j] += kd;
                }
                if (FO) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) FO[foff(r, c0 + j)] = v[j];
                }
                if (SO) split_store(SO + ioff(r, c0), v, STAGE_SCALE * TMEM_INV);
            }
        }
        if (SO) fence_proxy_async_global();
        __syncthreads();
    }

    // image k times 2^e in place (hi and lo parts scale exactly)
    __device__ void scale_image(int k, int e) {
        uint8_t* I = img(k);
        for (int mt = 0; mt < nrb; ++mt) {
            const int r = mt * 128 + row;
            for (int u = grp; u < npad / 8; u += 2) {
                for (int p = 0; p < 2; ++p) {
                    uint4* q = (uint4*)(I + ioff(r, 8 * u) + p * parti);
                    uint4 h = *q;
                    uint32_t* hv = (uint32_t*)&h;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (fmt == 0) {
                            __half2 x = *(__half2*)&hv[j];
                            x = __hmul2(x, __float2half2_rn(ldexpf(1.f, e)));
                            hv[j] = *(uint32_t*)&x;
                        } else {
                            __nv_bfloat162 x = *(__nv_bfloat162*)&hv[j];
                            x = __hmul2(x, __float2bfloat162_rn(ldexpf(1.f, e)));
                            hv[j] = *(uint32_t*)&x;
                        }
                    }
                    *q = h;
                }
            }
        }
        fence_proxy_async_global();
        __syncthreads();
    }

    // image so from a gathered block beta M (FP32, column groups of four,
    // npad x npad): scale x blk, and with use_diag the diagonal x0 computed in
    // FP64 (beta 2^-(s+1) (h_rr - mu), rounded once)
    __device__ void stage_dense(const float* blk, float scale, bool use_diag, int s, int so) {
        const float k = scale * STAGE_SCALE;
        uint8_t* SO = img(so);
        for (int mt = 0; mt < nrb; ++mt) {
            const int r = mt * 128 + row;
            float dv = 0.f;
            if (use_diag && r < n) dv = (float)(ldexp(a.beta, -(s + 1)) * (a.hdiag[sub0 + r] - a.mu)) * STAGE_SCALE;
            for (int u = grp; u < npad / 8; u += 2) {
                const int c0 = 8 * u;
                float v[8];
                if (r < npad) {
                    const float4 x0 = *(const float4*)(blk + ((size_t)(2 * u) * npad + r) * 4);
                    const float4 x1 = *(const float4*)(blk + ((size_t)(2 * u + 1) * npad + r) * 4);
                    v[0] = x0.x * k; v[1] = x0.y * k; v[2] = x0.z * k; v[3] = x0.w * k;
                    v[4] = x1.x * k; v[5] = x1.y * k; v[6] = x1.z * k; v[7] = x1.w * k;
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j) v[j] = 0.f;
                }
                if (use_diag && r < n && (unsigned)(r - c0) < 8u) {
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (c0 + j == r) v[j] = dv;
                }
                split_store(SO + ioff(r, c0), v, 1.f);
            }
        }
        fence_proxy_async_global();
        __syncthreads();
    }
    int64_t sub0;

    // largest k <= kmax with 4^k max_r sum_c |Q_rc| <= 1 (row sums in c.rs, FP32,
    // widened by (1 + n 2^-23) to remain an upper bound)
    __device__ int fewer_steps(int kmax) {
        float q = 0.f;
        for (int r = threadIdx.x; r < npad; r += BT) q = fmaxf(q, c.rs[r]);
        for (int o = 16; o > 0; o >>= 1) q = fmaxf(q, __shfl_xor_sync(0xffffffffu, q, o));
        if ((threadIdx.x & 31) == 0) c.part[0][threadIdx.x >> 5] = q;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = 0.f;
            for (int w = 0; w < BT / 32; ++w) m = fmaxf(m, c.part[0][w]);
            const double qmax = (double)m * (double)TMEM_INV * (1.0 + (double)(n + 2) * 0x1p-23);
            int k = 0;
            while (k < kmax && qmax * ldexp(1.0, 2 * (k + 1)) <= 1.0) ++k;
            c.kfew = k;
        }
        __syncthreads();
        return c.kfew;
    }

    // ---- the last doubling on the core columns (CUDA cores) ---------------
    // w = Z_s e_c = 2 (I + Z^2)^-1 Z e_c by one round of iterative refinement
    // with the tensor-core inverse X as preconditioner, w <- w + X (2 z - w -
    // Z (Z w)), from w0 = W e_c (the tensor-core doubling); every product
    // rounded to nearest in 8-term partial sums, sums as float pairs.  Each
    // thread owns rows tid, tid + 256, ... (RPT of them); the vectors that all
    // rows read sit in shared memory (the stage area, free at this point).
    template <int NC, int RPT>
    __device__ void rowvec(const float* F, const float* V, FF (&out)[RPT][NC]) const {
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int r = threadIdx.x + q * BT;
            float hi[NC], lo[NC];
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) hi[cc] = lo[cc] = 0.f;
            if (r < n) {
                for (int k0 = 0; k0 < npad; k0 += 8) {
                    float acc[NC];
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) acc[cc] = 0.f;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float m = F[foff(r, k0 + j)];
                        const float4* vr = (const float4*)(V + (k0 + j) * NC);
#pragma unroll
                        for (int w = 0; w < NC / 4; ++w) {
                            const float4 x = vr[w];
                            acc[4 * w] = fmaf(m, x.x, acc[4 * w]);
                            acc[4 * w + 1] = fmaf(m, x.y, acc[4 * w + 1]);
                            acc[4 * w + 2] = fmaf(m, x.z, acc[4 * w + 2]);
                            acc[4 * w + 3] = fmaf(m, x.w, acc[4 * w + 3]);
                        }
                    }
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) {
                        const FF t = two_sum(hi[cc], acc[cc]);
                        hi[cc] = t.hi;
                        lo[cc] += t.lo;
                    }
                }
            }
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) {
                const FF t = two_sum(hi[cc], lo[cc]);
                out[q][cc] = FF{t.hi * TMEM_INV, t.lo * TMEM_INV};
            }
        }
    }

    template <int NC, int RPT>
    __device__ void refine_core() {
        float* Vw = (float*)stg;                  // [npad][NC]
        float* Vt = Vw + (size_t)npad * NC;       // [npad][NC]
        const float* FZ = f32(F_Z);
        const float* FX = f32(F_X);
        const float* FW = f32(F_W);
        for (int b0 = 0; b0 < ncore; b0 += NC) {
            const int nc = min(NC, ncore - b0);
            int kc[NC];
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) kc[cc] = a.core_pos[core0 + b0 + (cc < nc ? cc : 0)];
            float z[RPT][NC];
            FF w[RPT][NC];
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int r = threadIdx.x + q * BT;
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const bool live = r < n && cc < nc;
                    z[q][cc] = live ? FZ[foff(r, kc[cc])] * TMEM_INV : 0.f;
                    w[q][cc] = FF{live ? FW[foff(r, kc[cc])] * TMEM_INV : 0.f, 0.f};
                    if (r < npad) Vw[r * NC + cc] = w[q][cc].hi;
                }
            }
            __syncthreads();
            FF t[RPT][NC];
            rowvec<NC, RPT>(FZ, Vw, t);                            // Z w
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int r = threadIdx.x + q * BT;
                if (r < npad)
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) Vt[r * NC + cc] = t[q][cc].hi;
            }
            __syncthreads();
            rowvec<NC, RPT>(FZ, Vt, t);                            // Z (Z w)
            __syncthreads();
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int r = threadIdx.x + q * BT;
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const FF res = ff_add(ff_add(FF{2.f * z[q][cc], 0.f}, ff_neg(w[q][cc])), ff_neg(t[q][cc]));
                    if (r < npad) Vt[r * NC + cc] = (r < n && cc < nc) ? res.hi : 0.f;
                }
            }
            __syncthreads();
            rowvec<NC, RPT>(FX, Vt, t);                            // X r
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int r = threadIdx.x + q * BT;
                if (r >= n) continue;
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    if (cc >= nc) continue;
                    const FF wn = ff_add(w[q][cc], t[q][cc]);
                    FF d = ff_add(FF{r == kc[cc] ? 1.f : 0.f, 0.f}, ff_neg(wn));
                    d = FF{0.5f * d.hi, 0.5f * d.lo};
                    if (!isfinite(d.hi)) set_error(a.err, GB_ERR_NAN);
                    const int e = b0 + cc;
                    a.Dval[a.col_ptr[a.core_idx[core0 + e]] + r] = f2d(d.hi) + f2d(d.lo);
                    if (r == kc[cc]) {
                        tv(T_DHI)[e] = d.hi;
                        tv(T_DLO)[e] = d.lo;
                    }
                }
            }
            __syncthreads();
        }
    }
};

__global__ void __launch_bounds__(BT, 1) k_fermi_split_big(PassArgs a) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    Ctl& c = *(Ctl*)(smem + NSTG * STG_BYTES);
    Big K(a, c, smem);

    if (threadIdx.x == 0) {
        c.abort = 0;
        for (int s = 0; s < NSTG; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&c.full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&c.empty[s])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&c.accf)) : "memory");
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
    const int32_t nwork = *a.work_n;
    const int m = a.m;

    for (;;) {
        if (threadIdx.x == 0) c.item = atomicAdd(a.big_counter, 1);
        __syncthreads();
        const int32_t j = c.item;
        if (j >= nwork || c.abort) break;
        const int32_t i = a.work[j];
        K.sub0 = a.sub_ptr[i];
        K.set_size((int)(a.sub_ptr[i + 1] - K.sub0));
        K.core0 = a.core_ptr[i];
        K.ncore = (int)(a.core_ptr[i + 1] - K.core0);
        const int npad = K.npad;
        for (int e = threadIdx.x; e < npad; e += BT) {
            c.cmap[e] = -1;
            c.rs[e] = 0.f;
        }
        if (threadIdx.x == 0) {
            c.s = recursion_steps(a.beta, a.mu, a.eps_lo[i], a.eps_hi[i], a.min_steps);
            c.dmax = 0;
        }
        if (threadIdx.x < m) {
            const double h1max = a.h1max[(int64_t)i * m + threadIdx.x];
            int k = 0;
            double sig = 1.0;
            while (0.5 * a.beta * sig * h1max > 1.0 && k < 100) {
                sig *= 0.5;
                ++k;
            }
            c.sigk[threadIdx.x] = k;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < K.ncore; e += BT) c.cmap[a.core_pos[K.core0 + e]] = (int16_t)e;
        __syncthreads();
        int s = c.s;
        const float* hb = a.hblk + a.boff[i];

        // ---- Taylor start: Q = x0^2, T = I - Q/3 + 2 Q^2/15, Z0 = x0 T ----
        K.stage_dense(hb, ldexpf(1.f, -(s + 1)), true, s, I_X0);
        {
            const Term t[1] = {{I_X0, I_X0}};
            Epi e;
            e.fo = F_X;
            e.rows = true;
            if (!K.gemm(t, 1, false, e)) break;                            // F_X = Q
        }
        const int kf = K.fewer_steps(s - a.min_steps);
        if (kf > 0) {
            s -= kf;
            K.scale_image(I_X0, kf);                                         // x0 <- 2^k x0
        }
        K.ew_stage(F_X, ldexpf(1.f, 2 * kf), 0.f, F_X, I_Q);                 // Q (x 4^k)
        {
            const Term t[1] = {{I_Q, I_Q}};
            Epi e;
            e.kp = 2.f / 15.f;
            e.f1 = F_X;
            e.k1 = -1.f / 3.f;
            e.cd = 1.f;
            e.fo = F_Z;
            e.so = I_T;
            if (!K.gemm(t, 1, false, e)) break;                            // F_Z = T, I_T
        }
        bool ok = true;
        for (int r = 0; r < m && ok; ++r) {
            const float* h1b = a.hblk + (int64_t)(1 + r) * a.hblk_stride + a.boff[i];
            K.stage_dense(h1b, ldexpf(1.f, -(s + 1) - c.sigk[r]), false, s, I_X1);
            {
                const Term t[2] = {{I_X0, I_X1}, {I_X1, I_X0}};
                Epi e;
                e.so = I_Q1;
                if (!(ok = K.gemm(t, 2, false, e))) break;                 // Q1 = x0 X1 + X1 x0
            }
            {
                const Term t[2] = {{I_Q, I_Q1}, {I_Q1, I_Q}};
                Epi e;
                e.kp = 2.f / 15.f;
                e.s1 = I_Q1;
                e.ks1 = -1.f / 3.f;
                e.so = I_T1;
                if (!(ok = K.gemm(t, 2, false, e))) break;                 // T1
            }
            {
                const Term t[2] = {{I_X0, I_T1}, {I_X1, I_T}};
                Epi e;
                e.so = I_Z1 + 2 * r;
                if (!(ok = K.gemm(t, 2, false, e))) break;                 // Z1_0 = x0 T1 + X1 T
            }
        }
        if (!ok) break;
        {
            const Term t[1] = {{I_X0, I_T}};
            Epi e;
            e.fo = F_Z;
            e.so = I_ZA;
            if (!K.gemm(t, 1, false, e)) break;                            // Z0
        }

        // ---- doublings: Z <- 2 X Z, X = (I + Z^2)^-1 ----
        int zi = 0, xi = 0, z1i = 0;
        for (int step = 0; step < s && ok; ++step) {
            const bool last = step == s - 1;
            const int IZ = I_ZA + zi, IW = I_ZA + (zi ^ 1);
            {
                const Term t[1] = {{IZ, IZ}};
                Epi e;
                e.fo = F_Y;
                e.so = I_Y;
                if (!(ok = K.gemm(t, 1, false, e))) break;                 // Y = Z^2
            }
            {
                const Term t[1] = {{I_Y, I_Y}};
                Epi e;
                e.kp = 32.f / 99.f;
                e.f1 = F_Y;
                e.k1 = -80.f / 99.f;
                e.cd = 98.f / 99.f;
                e.fo = F_X;
                e.so = I_XA + xi;
                if (!(ok = K.gemm(t, 1, true, e))) break;                  // X0 (Y^2 from hi parts)
            }
            for (int jn = 0; jn < a.ns_iters && ok; ++jn) {
                const bool rough = jn + 1 < a.ns_iters;
                {
                    const Term t[1] = {{I_Y, I_XA + xi}};
                    Epi e;
                    e.kp = -1.f;
                    e.f1 = F_X;
                    e.k1 = -1.f;
                    e.cd = 1.f;
                    e.so = I_R;
                    if (!(ok = K.gemm(t, 1, false, e))) break;             // R = (I - X) - Y X
                }
                {
                    const Term t[1] = {{I_XA + xi, I_R}};
                    Epi e;
                    e.f1 = F_X;
                    e.k1 = 1.f;
                    e.fo = F_X;
                    e.so = I_XA + (xi ^ 1);
                    if (!(ok = K.gemm(t, 1, rough, e))) break;             // X += X R
                }
                xi ^= 1;
            }
            if (!ok) break;
            const int IX = I_XA + xi;
            if (last) {
                K.ew_stage(F_Y, -1.f, 1.f, -1, I_IY);                        // I - Y
                {
                    const Term t[1] = {{I_IY, IX}};
                    Epi e;
                    e.so = I_G;
                    if (!(ok = K.gemm(t, 1, false, e))) break;             // G = (I - Y) X
                }
                {
                    const Term t[1] = {{I_G, I_G}};
                    Epi e;
                    e.cout = a.d1mu_val;
                    e.ck = (float)(0.25 * a.beta) * TMEM_INV;
                    e.cterm = T_DD;
                    e.ctk = 0.25f * TMEM_INV;
                    e.dmax = true;
                    if (!(ok = K.gemm(t, 1, false, e))) break;             // d1_mu = beta G^2 / 4
                }
            }
            {
                const Term t[1] = {{IX, IZ}};
                Epi e;
                e.kp = 2.f;
                e.fo = last ? F_W : F_Z;
                e.so = (last && m == 0) ? -1 : IW;
                if (!(ok = K.gemm(t, 1, false, e))) break;                 // W = 2 X Z
            }
            if (last) {
                if (npad <= 512) K.refine_core<8, 2>();
                else if (npad <= 1024) K.refine_core<8, 4>();
                else K.refine_core<4, 8>();
            }
            for (int r = 0; r < m && ok; ++r) {
                // Z1 <- 2 X Z1 X - (W Z1 / 2) W
                const int Z1c = I_Z1 + 2 * r + z1i;
                {
                    const Term t[1] = {{IX, Z1c}};
                    Epi e;
                    e.kp = 2.f;
                    e.so = I_A;
                    if (!(ok = K.gemm(t, 1, false, e))) break;             // A = 2 X Z1
                }
                {
                    const Term t[1] = {{IW, Z1c}};
                    Epi e;
                    e.kp = -0.5f;
                    e.so = I_U;
                    if (!(ok = K.gemm(t, 1, false, e))) break;             // U = -W Z1 / 2
                }
                {
                    const Term t[2] = {{I_U, IW}, {I_A, IX}};
                    Epi e;
                    if (!last) {
                        e.so = I_Z1 + 2 * r + (z1i ^ 1);
                    } else {
                        const float sc = -ldexpf(0.5f, c.sigk[r]) * TMEM_INV;  // d1_lambda = -Z1_s / (2 sigma)
                        e.cout = a.D1val[r];
                        e.ck = sc;
                        e.cterm = T_L0 + r;
                        e.ctk = sc;
                    }
                    if (!(ok = K.gemm(t, 2, false, e))) break;             // Z1 <- U W + A X
                }
            }
            zi ^= 1;
            z1i ^= 1;
        }
        if (!ok) break;

        // per-subgraph core traces, summed in FP64 in a fixed order
        __syncthreads();
        if (threadIdx.x < TR_FIXED + m) {
            const int sl = threadIdx.x;
            const int ncore = K.ncore;
            double v = 0.0;
            if (sl == TR_D) {
                for (int e = 0; e < ncore; ++e) v += (double)K.tv(T_DHI)[e] + (double)K.tv(T_DLO)[e];
            } else if (sl == TR_DD || sl == TR_D1MU) {
                for (int e = 0; e < ncore; ++e) v += (double)K.tv(T_DD)[e];
                if (sl == TR_D1MU) v *= a.beta;
            } else if (sl == TR_FLOPS) {
                v = pass_gemm_flops(K.n, s, a.ns_iters, m);
            } else if (sl == TR_FLOPS_S) {
                v = pass_flops_per_step_count(K.n, ncore, s, a.ns_iters, m);
            } else if (sl == TR_MAXWC) {
                float g = 0.f;
                for (int e = 0; e < ncore; ++e) g = fmaxf(g, K.tv(T_DD)[e]);
                v = a.beta * (double)g;
            } else if (sl == TR_MAXW) {
                v = 0.25 * a.beta * (double)__int_as_float(c.dmax) * (double)TMEM_INV;
            } else {
                for (int e = 0; e < ncore; ++e) v += (double)K.tv(T_L0 + sl - TR_D1LAM)[e];
            }
            a.tr[(int64_t)i * a.tr_stride + sl] = v;
        }
        if (threadIdx.x == 0) a.steps_out[i] = s;
        __syncthreads();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(K.tbase), "r"(TMEM_COLS)
                     : "memory");
}

}  // namespace

int launch_split_pass_big(gb_handle* h, const PassArgs& a, int grid, cudaStream_t stream) {
    static bool configured = false;
    if (!configured) {
        GB_CUDA(cudaFuncSetAttribute(k_fermi_split_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SMEM_BYTES));
        configured = true;
    }
    if (grid <= 0) return GB_OK;
    GB_LAUNCH_ON(h, stream, k_fermi_split_big, grid, BT, SMEM_BYTES, a);
    return GB_OK;
}
