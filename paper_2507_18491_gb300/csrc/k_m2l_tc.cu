// M2L of the mixed form on the 5th-generation tensor cores (tcgen05).
//
// A work item applies one scaled table A (P x P complex, row (nu,mu), column
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

cudaError_t configure_m2l_tc()
{
    return cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
}

}  // namespace lmf
