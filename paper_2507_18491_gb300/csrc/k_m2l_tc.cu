// M2L (and, in translation mode, M2M / L2L) of the mixed form on the
// 5th-generation tensor cores (tcgen05).  Two kernels: k_m2l_tc2 (v2 below,
// persistent, three-piece bf16 operands, p <= 12) and k_m2l_tc (this part,
// streamed operands, TF32 hi/lo, p <= 15).
//
// k_m2l_tc: a work item applies one scaled table A (P x P complex, row (nu,mu), column
// (n',m')) to up to 64 phase-shifted source expansions, exactly as the FP32
// SIMT kernel does, but the product runs as a real GEMM in which every
// complex entry a becomes the 2 x 2 block [[Re a, -Im a], [Im a, Re a]]:
//   rows 2r, 2r+1 of the real A  <->  Re, Im of output coefficient r,
//   K index 2k, 2k+1            <->  Re, Im of input coefficient k,
// so a column of the real B is the complex column itself, and M = 2P rows
// fill ceil(2P/128) tiles of 128 (3 tiles at p = 12, 88% used).
//
// FP32 accuracy from TF32 tensor cores (10-bit mantissa) comes from the
// three-term split x = x_hi + x_lo with x_hi = tf32(x), x_lo = tf32(x - x_hi):
//   A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi   (the dropped A_lo B_lo ~ 2^-22).
// The tensor core adds into its FP32 accumulator with truncation, aligned to
// the largest addend, so the two small terms would lose most of their bits
// in the accumulator of the large one: A_hi B_hi and the two small terms
// accumulate in separate tensor-memory accumulators, summed in the epilogue.
//
// Pipeline: all 256 threads stage K-chunks of 8 real K (4 complex inputs)
// into a 3-deep shared-memory ring -- the table chunk split into hi/lo
// planes of A, the phase-shifted expansions into hi/lo planes of B -- while
// one thread issues the MMAs of the previous chunk; tcgen05.commit on a
// per-slot mbarrier frees a slot.  Global loads of chunk c+1 are issued
// before chunk c is stored.  Epilogue: each warp reads a 32-lane quadrant of
// the accumulator with tcgen05.ld, pairs the Re/Im rows with one shuffle,
// applies the output factors of the M2L and adds into the local expansion
// with float2 atomics.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "kernels.cuh"
#include "m2l_cols.cuh"
#include "tc.cuh"

namespace lmf {

namespace {

constexpr int NT = 256;        // threads per CTA
constexpr int BN = 64;         // complex columns per work item (MMA N)
constexpr int STAGES = 3;      // shared-memory ring depth
constexpr int UMAX = 5;        // staging units per thread and chunk (P <= 256)
constexpr int WAIT_POLLS = 1 << 22;
constexpr int MT_MAX = 4;      // M tiles of 128 rows: 2P <= 512, p <= 15

// byte offset of element (row, kk) of a K-major, no-swizzle operand tile with
// 8 real K per row: core matrices of 8 rows x 16 B, the two K halves 128 B
// apart (leading byte offset), 8-row groups 256 B apart (stride byte offset)
__device__ __forceinline__ uint32_t canon_off(int row, int kh) { return (row >> 3) * 256 + kh * 128 + (row & 7) * 16; }

struct TcCol {
    int64_t in_base, out_base;   // (box * 3 + helical v) * P of the source / target
    int pp, kap;                 // pair within the work item, signed kappa
    float cre, cim;              // coefficient x i^(1+kappa) [x -1 for odd negative kappa]
};

struct SmemPlan {
    uint32_t a_plane, b_plane, stage, e_off, col_off, nn_off, bar_off, total;
};

__host__ __device__ inline SmemPlan smem_plan(int p, int MT)
{
    const int P = (p + 1) * (p + 1), MW = 2 * p + 5;
    SmemPlan s;
    s.a_plane = MT * 128 * 8 * 4;
    s.b_plane = BN * 8 * 4;
    s.stage = 2 * s.a_plane + 2 * s.b_plane;
    s.e_off = STAGES * s.stage;
    s.col_off = s.e_off + BN * MW * 8;
    s.nn_off = s.col_off + BN * (uint32_t)sizeof(TcCol);
    s.bar_off = (s.nn_off + P * 2 + 15) & ~15u;
    s.total = s.bar_off + STAGES * 8 + 16;
    return s;
}

__device__ __forceinline__ float4 split_hi(float4 v)
{
    return make_float4(tc::tf32_round(v.x), tc::tf32_round(v.y), tc::tf32_round(v.z), tc::tf32_round(v.w));
}

__device__ __forceinline__ void st_shared4(uint32_t addr, float4 v)
{
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w));
}

}  // namespace

__global__ void __launch_bounds__(NT) k_m2l_tc(int p, int MT, uint32_t tmem_cols, const M2LWork *work,
                                               const GeomDev *geoms, const CompDev *comps,
                                               const M2LPair *pairs, const cf *tab, const cf *me,
                                               cf *le, int *status)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    const int P = (p + 1) * (p + 1);
    const int MW = 2 * p + 5;
    const int nchunk = (P + 3) / 4;
    const int NA = 4 * P;                 // A units: (real row R < 2P, K half)
    const int NU = NA + 2 * BN;           // + B units: (column, K half)
    const SmemPlan sp = smem_plan(p, MT);
    cf *E = (cf *)(smraw + sp.e_off);
    TcCol *cols = (TcCol *)(smraw + sp.col_off);
    short *NN = (short *)(smraw + sp.nn_off);
    uint64_t *bar = (uint64_t *)(smraw + sp.bar_off);
    uint32_t *tslot = (uint32_t *)(bar + STAGES);
    const uint32_t sbase = tc::smem_u32(smraw);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const M2LWork w = work[blockIdx.x];
    const GeomDev &g = geoms[w.geom];
    const CompDev c = comps[g.comp];
    const int t = w.t;
    const int ncpp = (t == 1) ? 1 : 2;
    const int ncol = w.npair * ncpp;
    // odd powers of the in/out factors change sign for a downward component
    // and again for a mirrored source / target box
    const bool flip_in = (c.s < 0) != (c.has_src_refl != 0);
    const bool flip_out = (c.s < 0) != (c.has_tgt_refl != 0);

    if (warp == 0) tc::tmem_alloc(tslot, tmem_cols);
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) tc::mbar_init(&bar[s], 1);
    }
    for (int pp = tid; pp < w.npair; pp += NT) {
        M2LPair pr = pairs[w.pair0 + pp];
        cd b = {pr.cphi, pr.sphi}, e = mkd(1.0);
        cf *row = E + pp * MW + (p + 2);
        row[0] = cf{1.f, 0.f};
        for (int m = 1; m <= p + 2; ++m) {
            e = e * b;
            row[m] = cf{(float)e.x, (float)e.y};
            row[-m] = cf{(float)e.x, (float)(-e.y)};
        }
    }
    for (int col = tid; col < BN; col += NT) {
        TcCol q{};
        if (col < ncol) {
            const int pp = col / ncpp, j = col % ncpp;
            const ColSpec cs = c_cols[t][j];
            const M2LPair pr = pairs[w.pair0 + pp];
            q.in_base = (pr.src * 3 + cs.vin) * (int64_t)P;
            q.out_base = (pr.tgt * 3 + cs.vout) * (int64_t)P;
            q.pp = pp;
            q.kap = cs.kap;
            double cf0 = cs.coef;
            if (cs.kap < 0 && (cs.kap & 1)) cf0 = -cf0;
            cd k1 = ipow<double>(1 + cs.kap);
            q.cre = (float)(cf0 * k1.x);
            q.cim = (float)(cf0 * k1.y);
        }
        cols[col] = q;
    }
    for (int k = tid; k < P; k += NT) {
        int n = (int)sqrtf((float)k + 0.5f);
        while ((n + 1) * (n + 1) <= k) ++n;
        while (n * n > k) --n;
        NN[k] = (short)n;
    }
    tc::fence_smem_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *tslot;
    const cf *A = tab + ((int64_t)g.tab_index * NTAB + t) * P * P;

    // ---- staging: global loads of one chunk into registers ...
    auto load_chunk = [&](int cc, float4 (&v)[UMAX]) {
#pragma unroll
        for (int i = 0; i < UMAX; ++i) {
            const int u = tid + i * NT;
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
            if (u < NA) {
                const int R = u % (2 * P), kh = u / (2 * P);
                const int r = R >> 1, k0 = 4 * cc + 2 * kh;
                const cf *src = A + (int64_t)r * P + k0;
                if (k0 < P) {
                    cf a0 = src[0];
                    x.x = a0.x;
                    x.y = a0.y;
                }
                if (k0 + 1 < P) {
                    cf a1 = src[1];
                    x.z = a1.x;
                    x.w = a1.y;
                }
            } else if (u < NU) {
                const int v2 = u - NA, col = v2 % BN, kh = v2 / BN;
                if (col < ncol) {
                    const TcCol &q = cols[col];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int k = 4 * cc + 2 * kh + h;
                        if (k < P) {
                            const int n = NN[k], m = k - n * n - n;
                            const int ms = q.kap < 0 ? -m : m;
                            cf xm = me[q.in_base + n * n + n + ms];
                            if (h == 0) {
                                x.x = xm.x;
                                x.y = xm.y;
                            } else {
                                x.z = xm.x;
                                x.w = xm.y;
                            }
                        }
                    }
                }
            }
            v[i] = x;
        }
    };
    // ... and from registers into ring slot s, split into TF32 hi / lo planes
    auto store_chunk = [&](int cc, const float4 (&v)[UMAX], int s) {
        const uint32_t st0 = sbase + s * sp.stage;
        const uint32_t ahi = st0, alo = st0 + sp.a_plane;
        const uint32_t bhi = st0 + 2 * sp.a_plane, blo = bhi + sp.b_plane;
#pragma unroll
        for (int i = 0; i < UMAX; ++i) {
            const int u = tid + i * NT;
            if (u < NA) {
                const int R = u % (2 * P), kh = u / (2 * P);
                const float4 a = v[i];
                // row 2r: (Re a, -Im a) per input; row 2r+1: (Im a, Re a)
                const float4 x = (R & 1) ? make_float4(a.y, a.x, a.w, a.z)
                                         : make_float4(a.x, -a.y, a.z, -a.w);
                const float4 hi = split_hi(x);
                const float4 lo = split_hi(make_float4(x.x - hi.x, x.y - hi.y, x.z - hi.z, x.w - hi.w));
                const uint32_t off = canon_off(R, kh);
                st_shared4(ahi + off, hi);
                st_shared4(alo + off, lo);
            } else if (u < NU) {
                const int v2 = u - NA, col = v2 % BN, kh = v2 / BN;
                float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                if (col < ncol) {
                    const TcCol &q = cols[col];
                    const cf *er = E + q.pp * MW + (p + 2);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int k = 4 * cc + 2 * kh + h;
                        if (k < P) {
                            const int n = NN[k], m = k - n * n - n;
                            const int ms = q.kap < 0 ? -m : m;
                            const int e1 = n + ms;
                            cf sc = ipow<float>(e1);
                            if (flip_in && (e1 & 1)) sc = -sc;
                            const cf xm = h == 0 ? cf{v[i].x, v[i].y} : cf{v[i].z, v[i].w};
                            const cf y = sc * (er[ms] * xm);
                            if (h == 0) {
                                x.x = y.x;
                                x.y = y.y;
                            } else {
                                x.z = y.x;
                                x.w = y.y;
                            }
                        }
                    }
                }
                const float4 hi = split_hi(x);
                const float4 lo = split_hi(make_float4(x.x - hi.x, x.y - hi.y, x.z - hi.z, x.w - hi.w));
                const uint32_t off = canon_off(col, kh);
                st_shared4(bhi + off, hi);
                st_shared4(blo + off, lo);
            }
        }
    };

    constexpr uint32_t idesc = tc::idesc_tf32(128, BN, false);
    bool failed = false;
    int issued = -1;   // last chunk whose MMAs were committed
    float4 cur[UMAX];
    load_chunk(0, cur);
    for (int cc = 0; cc < nchunk; ++cc) {
        const int s = cc % STAGES;
        float4 nxt[UMAX];
        if (cc + 1 < nchunk) load_chunk(cc + 1, nxt);
        bool ok = true;
        if (cc >= STAGES) ok = tc::mbar_wait(&bar[s], (uint32_t)((cc / STAGES - 1) & 1), WAIT_POLLS);
        store_chunk(cc, cur, s);
        tc::fence_smem_async();
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (tid == 0) {
            tc::fence_after();
            const uint32_t st0 = sbase + s * sp.stage;
            const uint32_t ahi = st0, alo = st0 + sp.a_plane;
            const uint32_t bhi = st0 + 2 * sp.a_plane, blo = bhi + sp.b_plane;
            const uint64_t dbh = tc::sdesc(bhi, 128, 256), dbl = tc::sdesc(blo, 128, 256);
            for (int mt = 0; mt < MT; ++mt) {
                const uint32_t d = tbase + mt * BN, d2 = d + MT * BN;
                const uint64_t dah = tc::sdesc(ahi + mt * 4096, 128, 256);
                const uint64_t dal = tc::sdesc(alo + mt * 4096, 128, 256);
                tc::mma_tf32(d, dah, dbh, idesc, cc > 0 ? 1u : 0u);
                tc::mma_tf32(d2, dah, dbl, idesc, cc > 0 ? 1u : 0u);
                tc::mma_tf32(d2, dal, dbh, idesc, 1u);
            }
            tc::commit(&bar[s]);
        }
        issued = cc;
#pragma unroll
        for (int i = 0; i < UMAX; ++i) cur[i] = nxt[i];
    }
    // wait for the last committed chunk (commits cover every earlier MMA)
    bool done = true;
    if (issued >= 0)
        done = tc::mbar_wait(&bar[issued % STAGES], (uint32_t)((issued / STAGES) & 1), WAIT_POLLS);
    if (__syncthreads_or(!done) || failed) {
        if (tid == 0) atomicOr(status, 4);
        // give MMAs still in flight a second bounded wait before the
        // accumulator columns are released
        if (issued >= 0)
            tc::mbar_wait(&bar[issued % STAGES], (uint32_t)((issued / STAGES) & 1), WAIT_POLLS);
    } else {
        tc::fence_after();
        // ---- epilogue: warp -> lane quadrant (warp % 4), column half (warp / 4)
        const int q = warp & 3, h = warp >> 2;
        const bool even = (lane & 1) == 0;
        for (int mt = 0; mt < MT; ++mt) {
            const int R = mt * 128 + q * 32 + lane;
            if (mt * 128 + q * 32 >= 2 * P) break;   // warp-uniform
            const int r = R >> 1;
            const int nu = r < P ? NN[r] : 0, mh = r - nu * nu - nu;
            for (int c0 = h * 32; c0 < h * 32 + 32 && c0 < ncol; c0 += 8) {
                uint32_t v[8], v2[8];
                tc::tmem_ld8(tbase + ((uint32_t)(q * 32) << 16) + mt * BN + c0, v);
                tc::tmem_ld8(tbase + ((uint32_t)(q * 32) << 16) + (MT + mt) * BN + c0, v2);
                tc::tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = __float_as_uint(__uint_as_float(v[j]) + __uint_as_float(v2[j]));
                float send[4], recv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    send[j] = __uint_as_float(even ? v[4 + j] : v[j]);
                    recv[j] = __shfl_xor_sync(0xffffffffu, send[j], 1);
                }
                if (r >= P) continue;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int col = c0 + (even ? j : 4 + j);
                    if (col >= ncol) continue;
                    const cf y = even ? cf{__uint_as_float(v[j]), recv[j]}
                                      : cf{recv[j], __uint_as_float(v[4 + j])};
                    const TcCol &cq = cols[col];
                    const int mu = cq.kap < 0 ? -mh : mh;
                    const int e2 = nu + mu;
                    cf sc = ipow<float>(-e2);
                    if (flip_out && (e2 & 1)) sc = -sc;
                    const cf ph = E[cq.pp * MW + (p + 2) + cq.kap - mu];
                    const cf yy = (sc * cf{cq.cre, cq.cim}) * (ph * y);
                    atomicAdd((float2 *)(le + cq.out_base + nu * nu + nu + mu), make_float2(yy.x, yy.y));
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, tmem_cols);
}

// ====================================================================== v2
// Persistent, warp-specialised form with the operand roles exchanged:
//   D (128 x NR) = X (128 x K) T'^T,
// whose 128 rows are real columns -- rows 2c, 2c+1 hold (Re x, -Im x) and
// (Im x, Re x) of complex column c, giving Re (T' x) and Im (T' x) -- and
// whose NR >= P columns are the table rows (nu, mu).  The table enters as
// the B operand unchanged in shape (K = interleaved Re/Im input index); it
// is stored once per build as three bf16 planes (x ~ x1 + x2 + x3, each the
// bf16 rounding of what the previous pieces leave) in exactly the
// shared-memory image of each K-step, with the factors of the M2L that depend
// only on the degrees folded in:
//   T'[nu mu][n' m'] = (-i)^nu f_t^nu  T[nu mu][n' m']  i^n' f_s^n'
// (f = -1 where a downward component or a mirrored box flips odd powers,
// else 1; these are exact in any precision).  What is left per column is one
// complex factor per input order m' (phase e^{i m' phi} and i^m') and one per
// output order mu.  Roles (576 threads, one CTA per SM -- the tensor memory
// holds one CTA's accumulators, so latency is hidden by more warps per role):
//   warps 0-7   X producers, two groups of four warps (one per tensor-memory
//               lane quadrant), group g writing K-step g of every chunk: the
//               work item's 64 columns, coefficients prefetched V2_D chunks
//               ahead, phase-shifted, split once into three bf16 pieces (the
//               two rows of a column share the pieces) and written into a
//               V2_SX-slot tensor-memory ring (A operand);
//   warps 8-15  epilogue, two warps per lane quadrant taking alternate row
//               slabs: accumulators -> a per-CTA column-major scratch in global
//               memory through a per-warp shared tile (L2-resident; tensor
//               memory is free for the next item at once), then the output
//               factors and float2 atomics into the local expansions, then the
//               column data of the item two ahead;
//   warp 16     one bulk copy per table chunk into an S_T-slot shared ring;
//   warp 17     MMA issue, per K-step of 16 real K: X1 T1 into one accumulator,
//               X1 T2 + X2 T1 + X1 T3 + X2 T2 + X3 T1 into a second (the tensor
//               core truncates small addends against a large accumulator).
// A chunk is V2_KS MMA K-steps, so that waits, fences and commits are paid
// once per V2_KS steps; ring positions advance as counters (no division in the
// loops).  In translation mode (M2M, L2L) the chunks run from the highest
// input degree down.  Every wait is bounded; a wait that gives up sets bit 4
// of the status word and its role stops.
namespace {

constexpr int V2_KS = 2;           // MMA K-steps (16 real K each) per ring chunk
constexpr int V2_KC = 8 * V2_KS;   // complex inputs per ring chunk
constexpr int V2_NPC = 3;          // bf16 pieces per value
constexpr int V2_XW = 8 * V2_NPC * V2_KS;   // tensor-memory columns of an X chunk
constexpr int V2_SX = 3;           // X ring slots
constexpr int V2_ST_MAX = 16;      // table ring slots (shared memory)
constexpr int V2_PG = 2;           // producer groups (one K-step of every chunk each)
constexpr int V2_D = 3;            // chunks prefetched into registers
constexpr int V2_NR_MAX = 176;     // table rows padded to 16: 2 NR + V2_SX V2_XW <= 512, p <= 12
constexpr int V2_PT = 128 * V2_PG; // producer threads
constexpr int V2_ET = 256;         // epilogue threads
constexpr int V2_EW = V2_ET / 32;  // epilogue warps
constexpr int V2_RJ = (V2_NR_MAX + 31) / 32;   // rows per lane of a column in the scatter
constexpr int V2_DS = 34;          // row stride (words) of an epilogue warp's 16-row drain tile
constexpr int V2_WTMA = (V2_PT + V2_ET) / 32, V2_WMMA = V2_WTMA + 1;
constexpr int V2_THREADS = (V2_WMMA + 1) * 32;
constexpr uint32_t V2_SMEM_MAX = 227 * 1024;

struct V2Col {
    int64_t in_base, out_base;   // (box * 3 + helical v) * P of the source / target
    int pp, kap;                 // pair within the work item, signed kappa
};

struct V2Plan {
    uint32_t NR, nchunk, SB, CB, ST, MO, g_bytes, cols_bytes, meta_bytes, meta, tabs, mm_n, dtile, bars, total;
};

__host__ __device__ inline V2Plan v2_plan(int p)
{
    const int P = (p + 1) * (p + 1);
    V2Plan s;
    s.NR = (uint32_t)((P + 15) & ~15);
    s.nchunk = (uint32_t)(((P + 7) / 8 + V2_KS - 1) / V2_KS);   // chunks of V2_KS K-steps
    s.SB = s.NR * 32 * V2_NPC;                      // image of a K-step: V2_NPC planes of NR rows x 16 bf16
    s.CB = V2_KS * s.SB;
    s.MO = 2 * p + 1;                               // orders -p..p
    s.g_bytes = BN * s.MO * 8;                      // one factor table: [64][2p+1] complex
    s.cols_bytes = BN * (uint32_t)sizeof(V2Col);
    s.meta_bytes = 2 * s.g_bytes + s.cols_bytes;    // G, O, column records
    s.mm_n = V2_KC * s.nchunk;                      // order table, whole chunks (>= P)
    const uint32_t dtile_bytes = V2_EW * 16 * V2_DS * 4;   // per epilogue warp: 16 rows x 32 lanes
    const uint32_t fixed =
        2 * s.meta_bytes + 2 * s.mm_n + 32 + dtile_bytes + 16 + (2 * V2_ST_MAX + 2 * V2_SX + 12) * 8 + 16;
    uint32_t st = (V2_SMEM_MAX - fixed) / s.CB;
    s.ST = st > V2_ST_MAX ? V2_ST_MAX : st;
    s.meta = s.ST * s.CB;
    s.tabs = (s.meta + 2 * s.meta_bytes + 15) & ~15u;
    s.dtile = (s.tabs + 2 * s.mm_n + 15) & ~15u;
    s.bars = (s.dtile + dtile_bytes + 15) & ~15u;
    s.total = s.bars + (2 * V2_ST_MAX + 2 * V2_SX + 12) * 8 + 16;
    return s;
}

__device__ __forceinline__ cf lds_cf(uint32_t a)
{
    cf v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}

// three-piece bf16 split of a pair, x ~ b1 + b2 + b3 per component (b1 =
// bf16(x), b2 = bf16(x - b1), b3 = bf16(x - b1 - b2): 24 significant bits,
// FP32's exponent range); word j holds piece j, lo in the low half
__device__ __forceinline__ void v2_split_bf16(float lo, float hi, uint32_t (&w)[V2_NPC])
{
    float2 r{lo, hi};
#pragma unroll
    for (int j = 0; j < V2_NPC; ++j) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(r.x, r.y);
        w[j] = *(const uint32_t *)&h;
        if (j + 1 < V2_NPC) {
            const float2 f = __bfloat1622float2(h);
            r = float2{r.x - f.x, r.y - f.y};
        }
    }
}

// i^k v, exact
__device__ __forceinline__ cf mul_ipow(int k, cf v)
{
    switch (k & 3) {
    case 0: return v;
    case 1: return cf{-v.y, v.x};
    case 2: return cf{-v.x, -v.y};
    default: return cf{v.y, -v.x};
    }
}

// per-item column data, all exact transforms of the pair phases
// E[pp][d] = e^{i d phi} (FP64-computed, stored FP32):
//   input factors  G[pp][m'] = i^m' f_s^m' E[m'],
//   output factors O[col][mh] = coef i^(1+kappa) (-i)^mu f_t^mu E[kappa - mu],
//   mu = +-mh (sign of kappa), coef in {1/2, 1, -1/2};
// and the column records.  One warp per pair or column row, one lane per
// order (2p+1 <= 32), so that the fill has no division and no divergence.
__device__ __forceinline__ void v2_fill_meta(int p, int P, const M2LWork &w, const M2LPair *pairs,
                                             const cf *ephase, bool flip_in, bool flip_out, cf *G, cf *O,
                                             V2Col *cols, int tid, int nthr)
{
    const int MO = 2 * p + 1, MW = 2 * p + 5;
    const int t = w.t, ncpp = (t == 1) ? 1 : 2, ncol = w.npair * ncpp;
    const int lane = tid & 31, wi = tid >> 5, nw = nthr >> 5;
    const int m = lane - p;                      // order of this lane
    // rows per warp: at most RB (npair, ncol <= 64 over nw >= 8 warps); every
    // global load of the fill is issued before the first use
    constexpr int RB = 8;
    M2LPair pr{};
    if (tid < ncol) pr = pairs[w.pair0 + (ncpp == 1 ? tid : tid >> 1)];
    cf vg[RB], vo[RB];
    if (lane < MO) {
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const int pp = min(wi + i * nw, w.npair - 1);
            vg[i] = ephase[(w.pair0 + pp) * MW + (p + 2) + m];
        }
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const int col = min(wi + i * nw, ncol - 1);
            const int pp = ncpp == 1 ? col : col >> 1;
            const ColSpec &cs = c_cols[t][ncpp == 1 ? 0 : col & 1];
            const int mu = cs.kap < 0 ? -m : m;
            vo[i] = ephase[(w.pair0 + pp) * MW + (p + 2) + cs.kap - mu];
        }
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const int pp = wi + i * nw;
            if (pp >= w.npair) break;
            cf x = mul_ipow(m, vg[i]);
            if (flip_in && (m & 1)) x = -x;
            G[pp * MO + lane] = x;
        }
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const int col = wi + i * nw;
            if (col >= ncol) break;
            const ColSpec &cs = c_cols[t][ncpp == 1 ? 0 : col & 1];
            const int mu = cs.kap < 0 ? -m : m;
            float cf0 = (float)cs.coef;
            if (cs.kap < 0 && (cs.kap & 1)) cf0 = -cf0;
            if (flip_out && (mu & 1)) cf0 = -cf0;
            O[col * MO + lane] = cf0 * mul_ipow(1 + cs.kap - mu, vo[i]);
        }
    }
    static_assert(BN <= V2_ET, "one column record per epilogue thread");
    if (tid < BN) {
        V2Col q{};
        if (tid < ncol) {
            const ColSpec &cs = c_cols[t][ncpp == 1 ? 0 : tid & 1];
            q.in_base = (pr.src * 3 + cs.vin) * (int64_t)P;
            q.out_base = (pr.tgt * 3 + cs.vout) * (int64_t)P;
            q.pp = ncpp == 1 ? tid : tid >> 1;
            q.kap = cs.kap;
        }
        cols[tid] = q;
    }
}

__device__ __forceinline__ void v2_fill_trans(int p, int P, const M2LWork &w, const int64_t *tsrc,
                                              const int64_t *tdst, cf *G, cf *O, V2Col *cols, int tid, int nthr)
{
    const int MO = 2 * p + 1, ncol = 3 * w.npair;
    for (int e = tid; e < BN * MO; e += nthr) {
        G[e] = cf{1.f, 0.f};
        O[e] = cf{1.f, 0.f};
    }
    for (int col = tid; col < BN; col += nthr) {
        V2Col q{};
        if (col < ncol) {
            const int pp = col / 3, v = col - 3 * pp;
            q.in_base = (tsrc[w.pair0 + pp] * 3 + v) * (int64_t)P;
            q.out_base = (tdst[w.pair0 + pp] * 3 + v) * (int64_t)P;
            q.pp = pp;
            q.kap = 0;
        }
        cols[col] = q;
    }
}

// complex columns of a work item
__device__ __forceinline__ int v2_ncol(const M2LWork &w, int mode)
{
    return mode == 0 ? w.npair * ((w.t == 1) ? 1 : 2) : 3 * w.npair;
}

}  // namespace

__global__ void __launch_bounds__(V2_THREADS, 1)
    k_m2l_tc2(int p, int mode, int64_t nwork, const M2LWork *work, const GeomDev *geoms, const M2LPair *pairs, const cf *ephase, const int64_t *tsrc, const int64_t *tdst,
              const uint32_t *timg, const cf *me, cf *le, float *yscr,
              int *status, const TcProb *probs)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    const int P = (p + 1) * (p + 1);
    const V2Plan sp = v2_plan(p);
    const int NR = (int)sp.NR, nchunk = (int)sp.nchunk, ST = (int)sp.ST, MO = (int)sp.MO;
    // translations take the inputs from the highest degrees down: the accumulator
    // truncates relative to its running sum, so the dominant low-degree terms come
    // last and the low-degree outputs see few truncations at full size
    const bool krev = mode == 1;
    short *MM = (short *)(smraw + sp.tabs);   // order m of index k = n^2 + n + m (0 beyond P)
    uint64_t *bars = (uint64_t *)(smraw + sp.bars);
    uint64_t *tfull = bars, *tempty = bars + V2_ST_MAX, *xfull = bars + 2 * V2_ST_MAX,
             *xempty = xfull + V2_SX;
    uint64_t *accfull = xempty + V2_SX, *accempty = accfull + 1, *metafull = accfull + 2,
             *fin = accfull + 6, *ydone = accfull + 7, *yfree = accfull + 8;
    uint32_t *tslot = (uint32_t *)(accfull + 9);
    auto meta_G = [&](int slot) { return (cf *)(smraw + sp.meta + slot * sp.meta_bytes); };
    auto meta_O = [&](int slot) { return (cf *)(smraw + sp.meta + slot * sp.meta_bytes + sp.g_bytes); };
    auto meta_cols = [&](int slot) {
        return (V2Col *)(smraw + sp.meta + slot * sp.meta_bytes + 2 * sp.g_bytes);
    };

    // the arrays of an item's problem: the launch's own, or a batch entry
    auto prob = [&](const M2LWork &w) {
        if (probs) return probs[w.prob];
        return TcProb{geoms, pairs, ephase, timg, me, le};
    };

    float *Y = yscr + (size_t)blockIdx.x * NR * 128;   // [complex column][r], complex
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t XB = 2 * (uint32_t)NR;              // tensor-memory column of the X ring

    if (warp == 0) tc::tmem_alloc(tslot, 512);
    if (tid == 0) {
        for (int s = 0; s < ST; ++s) {
            tc::mbar_init(&tfull[s], 1);
            tc::mbar_init(&tempty[s], 1);
        }
        for (int s = 0; s < V2_SX; ++s) {
            tc::mbar_init(&xfull[s], V2_PT);   // both producer groups (one K-step each)
            tc::mbar_init(&xempty[s], 1);
        }
        tc::mbar_init(accfull, 1);
        tc::mbar_init(accempty, V2_ET);
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&metafull[i], V2_ET);
        }
        tc::mbar_init(fin, 1);
        tc::mbar_init(ydone, V2_ET);
        tc::mbar_init(yfree, V2_ET);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    for (int k = tid; k < (int)sp.mm_n; k += V2_THREADS) {
        int n = (int)sqrtf((float)k + 0.5f);
        while ((n + 1) * (n + 1) <= k) ++n;
        while (n * n > k) --n;
        MM[k] = k < P ? (short)(k - n * n - n) : (short)0;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *tslot;
    bool failed = false;

    if (warp == V2_WTMA) {
        // ------------------------------------------------ table chunks
        if (lane == 0) {
            uint32_t g = 0, ph = 0;   // chunks issued; parity of the current pass over the ring
            int s = 0;
            for (int64_t it = blockIdx.x; it < nwork && !failed; it += gridDim.x) {
                const M2LWork w = work[it];
                const TcProb pd = prob(w);
                const int64_t ti = mode == 0 ? pd.geoms[w.geom].tab_index * NTAB + w.t : (int64_t)w.geom;
                const unsigned char *src = (const unsigned char *)pd.img + (size_t)ti * nchunk * sp.CB;
                for (int c = 0; c < nchunk; ++c) {
                    if (g >= (uint32_t)ST && !tc::mbar_wait(&tempty[s], ph ^ 1, WAIT_POLLS)) {
                        failed = true;
                        break;
                    }
                    tc::mbar_expect_tx(&tfull[s], sp.CB);
                    tc::bulk_g2s(smraw + s * sp.CB, src + (size_t)(krev ? nchunk - 1 - c : c) * sp.CB, sp.CB,
                                 &tfull[s]);
                    ++g;
                    if (++s == ST) {
                        s = 0;
                        ph ^= 1;
                    }
                }
            }
            // copies still in flight land before the CTA leaves
            for (uint32_t q = g > (uint32_t)ST ? g - ST : 0; q < g; ++q)
                tc::mbar_wait(&tfull[q % ST], (q / ST) & 1, WAIT_POLLS);
        }
    } else if (warp == V2_WMMA) {
        // ------------------------------------------------ MMA issue
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16(128, NR);
            // descriptor of ring slot 0; the address field counts 16-byte units,
            // so slot, K-step and lo-plane offsets add to it directly
            const uint64_t dring0 = tc::sdesc(tc::smem_u32(smraw), 128, 256);
            const uint64_t d_cb = sp.CB >> 4, d_sb = sp.SB >> 4, d_pl = (uint32_t)(NR * 32) >> 4;
            uint64_t dslot = dring0;                       // descriptor of table slot st
            uint32_t aslot = tbase + XB;                   // tensor-memory address of X slot sx
            uint32_t li = 0, tph = 0, xph = 0;
            int st = 0, sx = 0;
            for (int64_t it = blockIdx.x; it < nwork && !failed; it += gridDim.x, ++li) {
                if (li >= 1 && !tc::mbar_wait(accempty, (li - 1) & 1, WAIT_POLLS)) {
                    failed = true;
                    break;
                }
                tc::fence_after();
                for (int c = 0; c < nchunk; ++c) {
                    if (!tc::mbar_wait(&tfull[st], tph, WAIT_POLLS) || !tc::mbar_wait(&xfull[sx], xph, WAIT_POLLS)) {
                        failed = true;
                        break;
                    }
                    tc::fence_after();
#pragma unroll
                    for (int u = 0; u < V2_KS; ++u) {
                        // pieces 1, 2, 3 of X (tensor memory) and of the table (shared memory)
                        const uint32_t a1 = aslot + 8 * V2_NPC * u, a2 = a1 + 8, a3 = a1 + 16;
                        const uint64_t b1 = dslot + u * d_sb, b2 = b1 + d_pl, b3 = b2 + d_pl;
                        const uint32_t acc = (c > 0 || u > 0) ? 1u : 0u;
                        tc::mma_f16_ta(tbase, a1, b1, idesc, acc);        // 1 x 1: large accumulator
                        tc::mma_f16_ta(tbase + NR, a1, b2, idesc, acc);   // the rest: small accumulator
                        tc::mma_f16_ta(tbase + NR, a2, b1, idesc, 1u);
                        tc::mma_f16_ta(tbase + NR, a1, b3, idesc, 1u);
                        tc::mma_f16_ta(tbase + NR, a2, b2, idesc, 1u);
                        tc::mma_f16_ta(tbase + NR, a3, b1, idesc, 1u);
                    }
                    tc::commit(&tempty[st]);
                    tc::commit(&xempty[sx]);
                    dslot += d_cb;
                    aslot += V2_XW;
                    if (++st == ST) {
                        st = 0;
                        tph ^= 1;
                        dslot = dring0;
                    }
                    if (++sx == V2_SX) {
                        sx = 0;
                        xph ^= 1;
                        aslot = tbase + XB;
                    }
                }
                if (failed) break;
                tc::commit(accfull);
            }
            tc::commit(fin);   // every MMA issued above has completed once fin flips
            tc::mbar_wait(fin, 0, WAIT_POLLS);
        }
    } else if (warp < V2_PT / 32) {
        // ------------------------------------------------ X producers
        // group pg writes K-step pg of every chunk; the two lanes of a column
        // (row b = 0: Re, -Im; row b = 1: Im, Re) each load, phase-shift and
        // split four of the K-step's eight inputs, swap the pieces with the
        // partner lane and store the K-step's 24 columns of their own row
        const int pg = warp / 4;
        const int j = tid - pg * 128, cc = j >> 1, b = j & 1;
        const uint32_t lane_base = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
        uint32_t li = 0, g = 0;                        // items, chunks of this CTA so far
        int xs = 0;                                    // ring slot of chunk g
        uint32_t xph = 0;
        for (int64_t it = blockIdx.x; it < nwork && !failed; it += gridDim.x, ++li) {
            const int slot = li & 1;
            cf *G = meta_G(slot);
            V2Col *cols = meta_cols(slot);
            const M2LWork w = work[it];
            // column data of the item, filled by the epilogue warps
            const bool ok = tc::mbar_wait(&metafull[slot], (li >> 1) & 1, WAIT_POLLS);
            if (__any_sync(0xffffffffu, !ok)) {
                failed = true;
                break;
            }
            const int ncol = v2_ncol(w, mode);
            const bool valid = cc < ncol;
            V2Col q{};
            if (valid) q = cols[cc];
            const bool neg = q.kap < 0;
            const uint32_t gr = tc::smem_u32(G + q.pp * MO + p);   // input factors of the column
            const cf *pme = prob(w).me;
            const cf *src = pme + q.in_base;
            constexpr int KQ = 4;                  // inputs per lane and chunk
            const int kk0 = 8 * pg + KQ * b;       // first of them within the chunk
            float2 pre[V2_D][KQ];
            const uint32_t mm0 = tc::smem_u32(MM);
            // orders m' of this lane's inputs (one 8-byte load of the order table)
            auto orders = [&](int ch, int(&mo)[KQ]) {
                uint32_t w0, w1;
                asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(w0), "=r"(w1) : "r"(mm0 + 2 * (V2_KC * ch + kk0)));
                mo[0] = (int)(short)(w0 & 0xffff);
                mo[1] = (int)(short)(w0 >> 16);
                mo[2] = (int)(short)(w1 & 0xffff);
                mo[3] = (int)(short)(w1 >> 16);
            };
            // input (n', m') reads the expansion at (n', +-m'): index k or k - 2m'.
            // Loads are unconditional (from a clamped address) so that they stay in
            // flight until their use V2_D chunks later; the mask is applied there.
            auto fetch = [&](int c, float2(&v)[KQ]) {
                const int ch = krev ? nchunk - 1 - c : c;
                int mo[KQ];
                orders(ch, mo);
#pragma unroll
                for (int h = 0; h < KQ; ++h) {
                    const int k = min(V2_KC * ch + kk0 + h, P - 1);
                    const cf *a = valid ? src + (neg ? k - 2 * mo[h] : k) : pme;
                    v[h] = *(const float2 *)a;
                }
            };
#pragma unroll
            for (int u = 0; u < V2_D; ++u)
                if (u < nchunk) fetch(u, pre[u]);
            for (int c0 = 0; c0 < nchunk && !failed; c0 += V2_D) {
#pragma unroll
                for (int u = 0; u < V2_D; ++u) {
                    const int c = c0 + u;
                    if (c >= nchunk) break;
                    const int ch = krev ? nchunk - 1 - c : c;   // data chunk
                    bool okw = g < (uint32_t)V2_SX || tc::mbar_wait(&xempty[xs], xph ^ 1, WAIT_POLLS);
                    if (__any_sync(0xffffffffu, !okw)) {
                        failed = true;
                        break;
                    }
                    tc::fence_after();
                    int mo[KQ];
                    orders(ch, mo);
                    // the lane's four inputs, phase-shifted and split once: word j of
                    // input h holds piece j of (Re, Im)
                    uint32_t own[KQ][V2_NPC], oth[KQ][V2_NPC];
#pragma unroll
                    for (int h = 0; h < KQ; ++h) {
                        cf y{0.f, 0.f};
                        if (valid && V2_KC * ch + kk0 + h < P)
                            y = lds_cf(gr + 8 * (neg ? -mo[h] : mo[h])) * cf{pre[u][h].x, pre[u][h].y};
                        v2_split_bf16(y.x, y.y, own[h]);
                    }
#pragma unroll
                    for (int h = 0; h < KQ; ++h)
#pragma unroll
                        for (int pc = 0; pc < V2_NPC; ++pc) oth[h][pc] = __shfl_xor_sync(0xffffffffu, own[h][pc], 1);
                    // the K-step's eight inputs in this lane's row: (Re, -Im) = negated
                    // high half, (Im, Re) = swapped halves (the split of -x is -split x);
                    // tensor-memory columns piece-major, even K in the low half
                    uint32_t rw[8 * V2_NPC];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int pc = 0; pc < V2_NPC; ++pc) {
                            const uint32_t wv = (i < KQ) == (b == 0) ? own[i & (KQ - 1)][pc] : oth[i & (KQ - 1)][pc];
                            rw[i + 8 * pc] = b ? __byte_perm(wv, 0, 0x1032) : (wv ^ 0x80000000u);
                        }
                    const uint32_t ta = lane_base + XB + V2_XW * xs + 8 * V2_NPC * pg;
                    static_assert(V2_KS == 2 && V2_NPC == 3, "two K-steps of 24 columns per chunk");
                    if (pg == 0) {
                        tc::tmem_st16(ta, rw);
                        tc::tmem_st8(ta + 16, rw + 16);
                    } else {
                        tc::tmem_st8(ta, rw);
                        tc::tmem_st16(ta + 8, rw + 8);
                    }
                    tc::tmem_st_wait();
                    tc::fence_before();
                    tc::mbar_arrive(&xfull[xs]);
                    ++g;
                    if (++xs == V2_SX) {
                        xs = 0;
                        xph ^= 1;
                    }
                    if (c + V2_D < nchunk) fetch(c + V2_D, pre[u]);
                }
            }
        }
    } else if (warp < V2_WTMA) {
        // ------------------------------------------------ epilogue
        const int ea = tid - V2_PT;                   // 0 .. V2_ET-1
        const int q4 = warp & 3, half = ea / 128;     // lane quadrant, slab parity
        const uint32_t lane_base = tbase + ((uint32_t)(32 * q4) << 16);
        const int ew = ea >> 5;                       // epilogue warp 0 .. V2_EW-1
        int rm[V2_RJ];                                // order m of rows lane + 32 i
#pragma unroll
        for (int i = 0; i < V2_RJ; ++i) rm[i] = MM[min(lane + 32 * i, P - 1)];
        // column data of item w into meta slot `slot`, then release it to the producers
        auto fill = [&](const M2LWork &w, int slot) {
            const TcProb pd = prob(w);
            if (mode == 0)
                v2_fill_meta(p, P, w, pd.pairs, pd.ephase, (w.flags & 1) != 0, (w.flags & 2) != 0, meta_G(slot),
                             meta_O(slot), meta_cols(slot), ea, V2_ET);
            else
                v2_fill_trans(p, P, w, tsrc, tdst, meta_G(slot), meta_O(slot), meta_cols(slot), ea, V2_ET);
            tc::mbar_arrive(&metafull[slot]);
        };
        for (int i = 0; i < 2; ++i)
            if (blockIdx.x + (int64_t)i * gridDim.x < nwork) fill(work[blockIdx.x + (int64_t)i * gridDim.x], i);
        uint32_t li = 0;
        for (int64_t it = blockIdx.x; it < nwork && !failed; it += gridDim.x, ++li) {
            // descriptor of the item two ahead, read now and used after the scatter
            const int64_t itn = it + 2 * (int64_t)gridDim.x;
            const M2LWork wn = work[min(itn, nwork - 1)];
            const M2LWork wc = work[it];
            const int slot = li & 1;
            bool ok = tc::mbar_wait(accfull, li & 1, WAIT_POLLS);
            if (__any_sync(0xffffffffu, !ok)) {
                failed = true;
                break;
            }
            tc::fence_after();
            // scratch layout [column cc][row r] complex.  A 16-row slab of the warp's
            // 32 real columns goes through the warp's shared-memory tile so that each
            // 16-byte store instruction writes four whole 128-byte column segments
            // (lane L: column 4h + L/8 of the warp's 16, rows 2 (L % 8), + 1)
            float *T = (float *)(smraw + sp.dtile) + (ea >> 5) * 16 * V2_DS;
            float4 *Yq = (float4 *)((float2 *)Y + (size_t)(16 * q4) * NR);
            const int lr = 2 * (lane & 7), lc = lane >> 3;
            for (int c0 = 16 * half; c0 < NR; c0 += 32) {   // NR is a multiple of 16
                uint32_t va[16], vb[16];
                tc::tmem_ld16(lane_base + c0, va);
                tc::tmem_ld16(lane_base + NR + c0, vb);
                tc::tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 16; ++i) T[i * V2_DS + lane] = __uint_as_float(va[i]) + __uint_as_float(vb[i]);
                __syncwarp();
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int cl = 4 * h + lc;
                    const float2 x0 = *(const float2 *)(T + lr * V2_DS + 2 * cl);
                    const float2 x1 = *(const float2 *)(T + (lr + 1) * V2_DS + 2 * cl);
                    Yq[((size_t)cl * NR + c0 + lr) >> 1] = make_float4(x0.x, x0.y, x1.x, x1.y);
                }
                __syncwarp();
            }
            tc::fence_before();
            tc::mbar_arrive(accempty);
            tc::mbar_arrive(ydone);
            ok = tc::mbar_wait(ydone, li & 1, WAIT_POLLS) &&
                 tc::mbar_wait(&metafull[slot], (li >> 1) & 1, WAIT_POLLS);
            if (!ok) {
                failed = true;
                break;
            }
            const int ncol = v2_ncol(wc, mode);
            cf *const ple = prob(wc).le;
            const cf *O = meta_O(slot);
            const V2Col *cols = meta_cols(slot);
            // one column per epilogue warp at a time, two in flight: lane j of a
            // column takes rows r = lane + 32 i; the column record is warp-uniform
            // and the scratch reads are coalesced
            for (int c = ew; c < ncol; c += 2 * V2_EW) {
                const int c2 = c + V2_EW;
                const bool two = c2 < ncol;
                float2 y[2][V2_RJ];
#pragma unroll
                for (int i = 0; i < V2_RJ; ++i) {
                    const int r = min(lane + 32 * i, P - 1);   // masked at use
                    y[0][i] = ((const float2 *)Y)[(size_t)c * NR + r];
                    y[1][i] = ((const float2 *)Y)[(size_t)(two ? c2 : c) * NR + r];
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (h == 1 && !two) break;
                    const int cc = h ? c2 : c;
                    const V2Col &cq = cols[cc];
                    const int64_t ob = cq.out_base;
                    const bool kneg = cq.kap < 0;
                    const cf *Oc = O + cc * MO + p;
#pragma unroll
                    for (int i = 0; i < V2_RJ; ++i) {
                        const int r = lane + 32 * i;
                        if (r < P) {
                            const cf yy = Oc[rm[i]] * cf{y[h][i].x, y[h][i].y};
                            // output (nu, mu) with mu = +-mh: index r or r - 2 mh
                            atomicAdd((float2 *)(ple + ob + (kneg ? r - 2 * rm[i] : r)), make_float2(yy.x, yy.y));
                        }
                    }
                }
            }
            // all epilogue threads are done with the scratch and with this meta slot:
            // refill the slot with the item two ahead
            tc::mbar_arrive(yfree);
            if (!tc::mbar_wait(yfree, li & 1, WAIT_POLLS)) {
                failed = true;
                break;
            }
            if (itn < nwork) fill(wn, slot);
        }
    }
    if (failed) atomicOr(status, 4);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

// three-piece bf16 split of a double (host and device)
__host__ __device__ inline void v2_split3(double v, __nv_bfloat16 (&o)[V2_NPC])
{
    o[0] = __float2bfloat16_rn((float)v);
    const double r1 = v - (double)__bfloat162float(o[0]);
    o[1] = __float2bfloat16_rn((float)r1);
    o[2] = __float2bfloat16_rn((float)(r1 - (double)__bfloat162float(o[1])));
}

// element (r, kk) of one plane of one K-step (16 real K) of a tiled image, in
// 16-bit units: NR rows x 16 values, K-major core matrices of 8 rows x 8
// values, the two K halves 128 B apart, 8-row groups 256 B apart
__host__ __device__ inline size_t v2_img_off(int r, int kk)
{
    return (size_t)(((r >> 3) * 256 + (kk >> 3) * 128 + (r & 7) * 16 + (kk & 7) * 2) >> 1);
}

// table image of the persistent kernel: per (geometry, table) nchunk * V2_KS
// K-steps (zero beyond P), each V2_NPC bf16 planes of NR rows x 16 real K,
// from the FP64 table with the level scaling s_t^nu s_s^n' and the degree
// factors (-i)^nu f_t^nu, i^n' f_s^n' applied before the split
__global__ void k_tile_tables(int p, int64_t g0, int64_t ng, const GeomDev *geoms, const CompDev *comps,
                              const cd *tab64, __nv_bfloat16 *img)
{
    const int P = (p + 1) * (p + 1);
    const V2Plan sp = v2_plan(p);
    const int NR = (int)sp.NR, nsub = (int)sp.nchunk * V2_KS;
    const int64_t gi = g0 + blockIdx.y;
    const int t = blockIdx.z;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nsub * NR * 8 || gi >= g0 + ng) return;
    const int c = e / (NR * 8), rem = e % (NR * 8), r = rem >> 3, i = rem & 7;   // input 8c + i
    const int k = 8 * c + i;
    const GeomDev &g = geoms[gi];
    cd v{0.0, 0.0};
    if (r < P && k < P) {
        int nu = (int)sqrt((double)r + 0.5), n1 = (int)sqrt((double)k + 0.5);
        while ((nu + 1) * (nu + 1) <= r) ++nu;
        while (nu * nu > r) --nu;
        while ((n1 + 1) * (n1 + 1) <= k) ++n1;
        while (n1 * n1 > k) --n1;
        const CompDev cp = comps[g.comp];
        const bool flip_in = (cp.s < 0) != (cp.has_src_refl != 0);
        const bool flip_out = (cp.s < 0) != (cp.has_tgt_refl != 0);
        const double f = pow(g.scale_t, (double)nu) * pow(g.scale_s, (double)n1) *
                         ((flip_in && (n1 & 1)) ? -1.0 : 1.0) * ((flip_out && (nu & 1)) ? -1.0 : 1.0);
        const cd a = tab64[((gi - g0) * NTAB + t) * (int64_t)P * P + (int64_t)r * P + k];
        v = ipow<double>(n1 - nu) * (f * a);   // i^n' (-i)^nu = i^(n' - nu)
    }
    __nv_bfloat16 re[V2_NPC], im[V2_NPC];
    v2_split3(v.x, re);
    v2_split3(v.y, im);
    __nv_bfloat16 *sub = img + ((size_t)(g.tab_index * NTAB + t) * nsub + c) * (size_t)(NR * 16 * V2_NPC);
    for (int pc = 0; pc < V2_NPC; ++pc) {
        sub[(size_t)pc * NR * 16 + v2_img_off(r, 2 * i)] = re[pc];
        sub[(size_t)pc * NR * 16 + v2_img_off(r, 2 * i + 1)] = im[pc];
    }
}

namespace {
int tc_mtiles(int p) { return (2 * (p + 1) * (p + 1) + 127) / 128; }
uint32_t tc_tmem_cols(int MT)
{
    uint32_t need = 2u * MT * BN, c = 32;
    while (c < need) c <<= 1;
    return c;
}
}  // namespace

bool m2l_tc_supported(int p) { return p >= 1 && tc_mtiles(p) <= MT_MAX; }
int m2l_tc_cols() { return BN; }

cudaError_t launch_m2l_tc(int p, int64_t nwork, const M2LWork *work, const GeomDev *geoms,
                          const CompDev *comps, const M2LPair *pairs, const cf *tab, const cf *me,
                          cf *le, int *status, cudaStream_t st)
{
    if (nwork <= 0) return cudaSuccess;
    if (!m2l_tc_supported(p)) return cudaErrorInvalidValue;
    const int MT = tc_mtiles(p);
    const uint32_t cols = tc_tmem_cols(MT);
    size_t smem = smem_plan(p, MT).total;
    // never let more CTAs share an SM than its 512 tensor-memory columns hold:
    // pad the shared-memory request until the occupancy bound enforces it
    const size_t sm_smem = 228 * 1024, per_cta_reserved = 1024;
    const int max_ctas = (int)(512 / cols);
    const size_t min_smem = sm_smem / (size_t)(max_ctas + 1) + 1;
    if (smem + per_cta_reserved < min_smem) smem = min_smem - per_cta_reserved;
    k_m2l_tc<<<(unsigned)nwork, NT, smem, st>>>(p, MT, cols, work, geoms, comps, pairs, tab, me, le,
                                                status);
    return cudaGetLastError();
}

bool m2l_tc2_supported(int p)
{
    return p >= 1 && v2_plan(p).NR <= (uint32_t)V2_NR_MAX && 2 * v2_plan(p).NR + V2_SX * V2_XW <= 512 &&
           v2_plan(p).ST >= 4;
}

size_t m2l_tc2_image_bytes(int p, int64_t ngeom)
{
    const V2Plan sp = v2_plan(p);
    return (size_t)ngeom * NTAB * sp.nchunk * sp.CB;
}

size_t m2l_tc2_scratch_floats(int p, int nsm) { return (size_t)nsm * 128 * v2_plan(p).NR; }

void launch_tile_tables(int p, int64_t g0, int64_t ng, const GeomDev *geoms, const CompDev *comps,
                        const cd *tab64, void *img, cudaStream_t st)
{
    if (ng <= 0) return;
    const V2Plan sp = v2_plan(p);
    dim3 grid((sp.nchunk * V2_KS * sp.NR * 8 + 255) / 256, (unsigned)ng, NTAB);
    k_tile_tables<<<grid, 256, 0, st>>>(p, g0, ng, geoms, comps, tab64, (__nv_bfloat16 *)img);
}

static cudaError_t launch_tc2(int p, int mode, int64_t nwork, const M2LWork *work, const GeomDev *geoms,
                              const M2LPair *pairs, const cf *ephase, const int64_t *tsrc,
                              const int64_t *tdst, const void *img, const cf *in, cf *out, float *yscr, int nsm,
                              int *status, cudaStream_t st)
{
    if (nwork <= 0) return cudaSuccess;
    if (!m2l_tc2_supported(p) || nsm < 1) return cudaErrorInvalidValue;
    const int64_t grid = std::min<int64_t>(nwork, (int64_t)nsm);
    // each CTA takes all 512 tensor-memory columns: ask for more than half of
    // an SM's shared memory so that no two CTAs are resident on one SM
    const size_t smem = std::max<size_t>(v2_plan(p).total, 116 * 1024);
    k_m2l_tc2<<<(unsigned)grid, V2_THREADS, smem, st>>>(p, mode, nwork, work, geoms, pairs, ephase, tsrc,
                                                        tdst, (const uint32_t *)img, in, out, yscr, status, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_m2l_tc2_batch(int p, int64_t nwork, const M2LWork *work, const TcProb *probs, float *yscr,
                                 int nsm, int *status, cudaStream_t st)
{
    if (nwork <= 0) return cudaSuccess;
    if (!m2l_tc2_supported(p) || nsm < 1) return cudaErrorInvalidValue;
    const int64_t grid = std::min<int64_t>(nwork, (int64_t)nsm);
    const size_t smem = std::max<size_t>(v2_plan(p).total, 116 * 1024);
    k_m2l_tc2<<<(unsigned)grid, V2_THREADS, smem, st>>>(p, 0, nwork, work, nullptr, nullptr, nullptr, nullptr,
                                                        nullptr, nullptr, nullptr, nullptr, yscr, status, probs);
    return cudaGetLastError();
}

cudaError_t launch_m2l_tc2(int p, int64_t nwork, const M2LWork *work, const GeomDev *geoms,
                           const M2LPair *pairs, const cf *ephase, const void *img,
                           const cf *me, cf *le, float *yscr, int nsm, int *status, cudaStream_t st)
{
    return launch_tc2(p, 0, nwork, work, geoms, pairs, ephase, nullptr, nullptr, img, me, le, yscr, nsm,
                      status, st);
}

cudaError_t launch_trans_tc2(int p, int64_t nwork, const M2LWork *work, const int64_t *tsrc,
                             const int64_t *tdst, const void *img, const cf *in, cf *out, float *yscr, int nsm,
                             int *status, cudaStream_t st)
{
    return launch_tc2(p, 1, nwork, work, nullptr, nullptr, nullptr, tsrc, tdst, img, in, out, yscr, nsm,
                      status, st);
}

size_t tc2_matrix_bytes(int p)
{
    const V2Plan sp = v2_plan(p);
    return (size_t)sp.nchunk * sp.CB;
}

void tile_matrix_tc2(int p, const cd *M, void *img_)
{
    const int P = (p + 1) * (p + 1);
    const V2Plan sp = v2_plan(p);
    const int NR = (int)sp.NR, nsub = (int)sp.nchunk * V2_KS;
    __nv_bfloat16 *img = (__nv_bfloat16 *)img_;
    for (int c = 0; c < nsub; ++c)
        for (int r = 0; r < NR; ++r)
            for (int i = 0; i < 8; ++i) {
                const int k = 8 * c + i;
                cd v{0.0, 0.0};
                if (r < P && k < P) v = M[(size_t)r * P + k];
                __nv_bfloat16 re[V2_NPC], im[V2_NPC];
                v2_split3(v.x, re);
                v2_split3(v.y, im);
                __nv_bfloat16 *sub = img + (size_t)c * NR * 16 * V2_NPC;
                for (int pc = 0; pc < V2_NPC; ++pc) {
                    sub[(size_t)pc * NR * 16 + v2_img_off(r, 2 * i)] = re[pc];
                    sub[(size_t)pc * NR * 16 + v2_img_off(r, 2 * i + 1)] = im[pc];
                }
            }
}

cudaError_t configure_m2l_tc()
{
    cudaError_t e = cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_m2l_tc2, cudaFuncAttributeMaxDynamicSharedMemorySize, V2_SMEM_MAX);
}

}  // namespace lmf
