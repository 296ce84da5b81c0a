// Translation kernels M2M, L2L and M2L for T = double (FP64 form) or
// T = float (mixed form).  All three are batched complex GEMMs Y = A X with
// A a P x P matrix shared by every column of a work item: the columns of X
// are gathered expansions (with per-column phases for M2L), the products are
// scattered back.  Expansions are stored scaled per level
// (M~_n = M_n / s^n, L~_nu = L_nu s^nu, s = |k| S_level) so that every
// matrix entry and coefficient stays in the float range.
#include "kernels.cuh"
#include "m2l_cols.cuh"

namespace lmf {

// acc += a * x with four fused multiply-adds
template <typename T>
__device__ __forceinline__ void cmac(cx<T> &acc, cx<T> a, cx<T> x)
{
    acc.x = fma(a.x, x.x, acc.x);
    acc.x = fma(-a.y, x.y, acc.x);
    acc.y = fma(a.x, x.y, acc.y);
    acc.y = fma(a.y, x.x, acc.y);
}

template <typename T> struct TileCfg;
template <> struct TileCfg<float> { static constexpr int TM = 4, TN = 4, BK = 16; };
template <> struct TileCfg<double> { static constexpr int TM = 4, TN = 2, BK = 16; };

// Y(P x BN) = A(P x P, row-major, global) X(P x BN, shared, rows BNP apart); 256 threads as a
// 16 x 16 grid, each owning TM rows x TN columns.  A streams through two
// shared-memory tiles of BK x BM (k-major, rows padded to BMP so that the
// transposing stores spread over banks and every thread's TM rows stay 16-byte
// aligned); the next tile is fetched into registers while the current one is
// multiplied.  The TM rows and TN columns of a thread are read with 16-byte
// loads.  One CTA computes the BM rows of row tile r_tile; store(r, c, y) for
// r < P, c < ncol.
template <typename T>
struct GemmTile {
    static constexpr int TM = TileCfg<T>::TM, TN = TileCfg<T>::TN, BK = TileCfg<T>::BK;
    static constexpr int BM = 16 * TM, BN = 16 * TN, BMP = BM + 2;
    static constexpr int BNP = BN + 2;          // row stride of X in shared memory
    static constexpr int LPT = BM * BK / 256;   // tile elements loaded per thread
};

template <typename T, int N>
__device__ __forceinline__ void lds_vec(const cx<T> *src, cx<T> (&dst)[N])
{
    static_assert((N * sizeof(cx<T>)) % 16 == 0, "whole 16-byte words");
    const float4 *s4 = (const float4 *)src;
#pragma unroll
    for (int i = 0; i < (int)(N * sizeof(cx<T>) / 16); ++i) {
        const float4 v = s4[i];
        memcpy((char *)dst + 16 * i, &v, 16);
    }
}

// TRA: multiply by A^T (A read column-wise: consecutive threads take
// consecutive rows of A^T, i.e. consecutive entries of a row of A)
template <typename T, typename Store, bool TRA = false>
__device__ __forceinline__ void tiled_gemm(int P, int r_tile, const cx<T> *__restrict__ A, const cx<T> *X,
                                           cx<T> *As, int ncol, Store store)
{
    using G = GemmTile<T>;
    constexpr int TM = G::TM, TN = G::TN, BK = G::BK, BM = G::BM, BMP = G::BMP;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int nk = (P + BK - 1) / BK;
    auto rk = [](int e, int &r, int &kk) {
        if (TRA) { r = e % BM; kk = e / BM; }
        else { r = e / BK; kk = e % BK; }
    };
    auto fetch = [&](int r0, int k0, cx<T> (&v)[G::LPT]) {
#pragma unroll
        for (int u = 0; u < G::LPT; ++u) {
            int r, kk;
            rk(threadIdx.x + 256 * u, r, kk);
            const int gr = r0 + r, gk = k0 + kk;
            v[u] = (gr < P && gk < P) ? (TRA ? A[(int64_t)gk * P + gr] : A[(int64_t)gr * P + gk])
                                      : cx<T>{T(0), T(0)};
        }
    };
    auto put = [&](int buf, const cx<T> (&v)[G::LPT]) {
#pragma unroll
        for (int u = 0; u < G::LPT; ++u) {
            int r, kk;
            rk(threadIdx.x + 256 * u, r, kk);
            As[buf * BK * BMP + kk * BMP + r] = v[u];
        }
    };
    {
        const int r0 = r_tile * BM;
        cx<T> acc[TM][TN];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = cx<T>{T(0), T(0)};
        cx<T> nxt[G::LPT];
        fetch(r0, 0, nxt);
        put(0, nxt);
        __syncthreads();
        for (int kt = 0; kt < nk; ++kt) {
            const int k0 = kt * BK, buf = kt & 1;
            if (kt + 1 < nk) fetch(r0, k0 + BK, nxt);
            const cx<T> *At = As + buf * BK * BMP;
            const int kmax = min(BK, P - k0);
            for (int kk = 0; kk < kmax; ++kk) {
                cx<T> a[TM], x[TN];
                lds_vec<T, TM>(At + kk * BMP + ty * TM, a);
                lds_vec<T, TN>(X + (k0 + kk) * G::BNP + tx * TN, x);
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) cmac(acc[i][j], a[i], x[j]);
            }
            if (kt + 1 < nk) put(buf ^ 1, nxt);
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            int r = r0 + ty * TM + i;
            if (r >= P) continue;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                int c = tx * TN + j;
                if (c < ncol) store(r, c, acc[i][j]);
            }
        }
    }
}

template <typename T>
__device__ __forceinline__ void atomic_add_cx(cx<T> *o, cx<T> v)
{
    if constexpr (sizeof(T) == 4) {
        atomicAdd((float2 *)o, make_float2(v.x, v.y));
    } else {
        atomicAdd(&o->x, v.x);
        atomicAdd(&o->y, v.y);
    }
}

// ------------------------------------------------------------- M2M / L2L
// Work item = up to BN/3 (child, parent) pairs of one translation group;
// column (pair, v) for the helical components v = 0, 1, 2.
template <typename T>
__global__ void __launch_bounds__(256) k_group_gemm(int p, const GemmWork *work, const cx<T> *mats,
                                                    const int64_t *src, const int64_t *dst,
                                                    const cx<T> *in, cx<T> *out, int atomic)
{
    using G = GemmTile<T>;
    constexpr int BN = G::BN, BNP = G::BNP;
    extern __shared__ unsigned char smraw[];
    const int P = (p + 1) * (p + 1);
    cx<T> *X = (cx<T> *)smraw;
    cx<T> *As = X + (size_t)P * BNP;
    GemmWork w = work[blockIdx.x];
    const int ncol = 3 * w.npair;
    // gather the columns: consecutive threads read consecutive coefficients of
    // one expansion; loads are issued in batches of GB before their stores
    constexpr int GB = 8;
    const int ne = P * BN;
    for (int e0 = threadIdx.x; e0 < ne; e0 += GB * blockDim.x) {
        cx<T> v[GB];
#pragma unroll
        for (int u = 0; u < GB; ++u) {
            const int e = e0 + u * blockDim.x, col = e / P, k = e - col * P;
            v[u] = cx<T>{T(0), T(0)};
            if (e < ne && col < ncol) v[u] = in[(src[w.pair0 + col / 3] * 3 + col % 3) * P + k];
        }
#pragma unroll
        for (int u = 0; u < GB; ++u) {
            const int e = e0 + u * blockDim.x, col = e / P, k = e - col * P;
            if (e < ne) X[k * BNP + col] = v[u];
        }
    }
    __syncthreads();
    const cx<T> *A = mats + (int64_t)w.group * P * P;
    tiled_gemm<T>(P, blockIdx.y, A, X, As, ncol, [&](int r, int c, cx<T> y) {
        cx<T> *o = out + (dst[w.pair0 + c / 3] * 3 + c % 3) * P + r;
        if (atomic) atomic_add_cx(o, y);
        else *o += y;
    });
}

// --------------------------------------------------------------------- M2L

// The M2L of eq. M2L_scale_with_Tnmu with T = (-i)^nu i^(n'+1+d) s^(nu+mu+n'+m')
// e^{i d phi} I-hat, d = m' - mu + kappa, factorised as
//   in(n',m')  = (i s)^(n'+m') e^{i m' phi}  [x (-1)^(n'+m') for a mirrored source]
//   out(nu,mu) = (-i s)^(nu+mu) e^{-i mu phi} [x (-1)^(nu+mu) for a mirrored target]
//   const      = i^(1+kappa) e^{i kappa phi} x coefficient.
// kappa < 0 uses I-hat_{-kappa}[nu,mu,n',m'] = (-1)^kappa I-hat_kappa[nu,-mu,n',-m']:
// the input column is flipped in m before the product, the output after.
// The stored table already carries the level scaling s_t^nu s_s^n'.
template <typename T>
__global__ void __launch_bounds__(256) k_m2l(int p, const M2LWork *work, const GeomDev *geoms,
                                             const CompDev *comps, const M2LPair *pairs,
                                             const cx<T> *tab, const cx<T> *me, cx<T> *le)
{
    constexpr int BN = 16 * TileCfg<T>::TN;
    extern __shared__ unsigned char smraw[];
    const int P = (p + 1) * (p + 1);
    const int MW = 2 * p + 5;           // e^{i m phi}, m = -(p+2) .. p+2
    cx<T> *X = (cx<T> *)smraw;
    cx<T> *As = X + (size_t)P * GemmTile<T>::BNP;
    cx<T> *E = As + 2 * GemmTile<T>::BK * GemmTile<T>::BMP;   // [BN][MW]
    short *NN = (short *)(E + BN * MW);                     // degree of index k
    M2LWork w = work[blockIdx.x];
    const GeomDev &g = geoms[w.geom];
    const CompDev c = comps[g.comp];
    const int t = w.t;
    const int ncpp = (t == 1) ? 1 : 2;
    const int ncol = w.npair * ncpp;
    const bool sneg = c.s < 0;
    // per-pair phase table by powers of (cos phi, sin phi), and the index -> n map
    for (int pp = threadIdx.x; pp < w.npair; pp += blockDim.x) {
        M2LPair pr = pairs[w.pair0 + pp];
        cd b = {pr.cphi, pr.sphi}, e = mkd(1.0);
        cx<T> *row = E + pp * MW + (p + 2);
        row[0] = cx<T>{T(1), T(0)};
        for (int m = 1; m <= p + 2; ++m) {
            e = e * b;
            row[m] = cx<T>{(T)e.x, (T)e.y};
            row[-m] = cx<T>{(T)e.x, (T)(-e.y)};
        }
    }
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        int n = (int)sqrtf((float)k + 0.5f);
        while ((n + 1) * (n + 1) <= k) ++n;
        while (n * n > k) --n;
        NN[k] = (short)n;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < P * BN; e += blockDim.x) {
        int k = e / BN, col = e % BN;
        cx<T> v{T(0), T(0)};
        if (col < ncol) {
            int pp = col / ncpp, j = col % ncpp;
            ColSpec cs = c_cols[t][j];
            int n = NN[k], m = k - n * n - n;
            int ms = cs.kap < 0 ? -m : m;
            cx<T> x = me[(pairs[w.pair0 + pp].src * 3 + cs.vin) * P + n * n + n + ms];
            int e1 = n + ms;
            cx<T> sc = ipow<T>(e1);
            if ((sneg && (e1 & 1)) != (c.has_src_refl && (e1 & 1))) sc = -sc;
            v = sc * (E[pp * MW + (p + 2) + ms] * x);
        }
        X[k * GemmTile<T>::BNP + col] = v;
    }
    __syncthreads();
    const cx<T> *A = tab + ((int64_t)g.tab_index * NTAB + t) * P * P;
    tiled_gemm<T>(P, blockIdx.y, A, X, As, ncol, [&](int r, int col, cx<T> y) {
        int pp = col / ncpp, j = col % ncpp;
        ColSpec cs = c_cols[t][j];
        int nu = NN[r], mh = r - nu * nu - nu;
        int mu = cs.kap < 0 ? -mh : mh;
        int e2 = nu + mu;
        cx<T> sc = ipow<T>(-e2);
        if ((sneg && (e2 & 1)) != (c.has_tgt_refl && (e2 & 1))) sc = -sc;
        T cf = (T)cs.coef;
        if (cs.kap < 0 && (cs.kap & 1)) cf = -cf;
        cx<T> k1 = ipow<T>(1 + cs.kap);
        cx<T> ph = E[pp * MW + (p + 2) + cs.kap - mu];
        cx<T> yy = (cf * sc) * (k1 * (ph * y));
        atomic_add_cx(le + (pairs[w.pair0 + pp].tgt * 3 + cs.vout) * P + nu * nu + nu + mu, yy);
    });
}

// Transpose of k_m2l: the forward map of a column is
//   le[tgt][vout][out(r)] += F_out(r) sum_k A[r][k] F_in(k) me[src][vin][in(k)]
// (F_in, F_out, in(k), out(r) the factors and the kappa < 0 order flips above),
// so its transpose gathers F_out(r) le_bar[tgt][vout][out(r)] into the rows r,
// multiplies by A^T and scatters F_in(k) (A^T x)_k into me_bar[src][vin][in(k)].
template <typename T>
__global__ void __launch_bounds__(256) k_m2l_tr(int p, const M2LWork *work, const GeomDev *geoms,
                                                const CompDev *comps, const M2LPair *pairs,
                                                const cx<T> *tab, const cx<T> *le_bar, cx<T> *me_bar)
{
    constexpr int BN = 16 * TileCfg<T>::TN;
    extern __shared__ unsigned char smraw[];
    const int P = (p + 1) * (p + 1);
    const int MW = 2 * p + 5;
    cx<T> *X = (cx<T> *)smraw;
    cx<T> *As = X + (size_t)P * GemmTile<T>::BNP;
    cx<T> *E = As + 2 * GemmTile<T>::BK * GemmTile<T>::BMP;
    short *NN = (short *)(E + BN * MW);
    M2LWork w = work[blockIdx.x];
    const GeomDev &g = geoms[w.geom];
    const CompDev c = comps[g.comp];
    const int t = w.t;
    const int ncpp = (t == 1) ? 1 : 2;
    const int ncol = w.npair * ncpp;
    const bool sneg = c.s < 0;
    for (int pp = threadIdx.x; pp < w.npair; pp += blockDim.x) {
        M2LPair pr = pairs[w.pair0 + pp];
        cd b = {pr.cphi, pr.sphi}, e = mkd(1.0);
        cx<T> *row = E + pp * MW + (p + 2);
        row[0] = cx<T>{T(1), T(0)};
        for (int m = 1; m <= p + 2; ++m) {
            e = e * b;
            row[m] = cx<T>{(T)e.x, (T)e.y};
            row[-m] = cx<T>{(T)e.x, (T)(-e.y)};
        }
    }
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        int n = (int)sqrtf((float)k + 0.5f);
        while ((n + 1) * (n + 1) <= k) ++n;
        while (n * n > k) --n;
        NN[k] = (short)n;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < P * BN; e += blockDim.x) {
        int r = e / BN, col = e % BN;
        cx<T> v{T(0), T(0)};
        if (col < ncol) {
            int pp = col / ncpp, j = col % ncpp;
            ColSpec cs = c_cols[t][j];
            int nu = NN[r], mh = r - nu * nu - nu;
            int mu = cs.kap < 0 ? -mh : mh;
            int e2 = nu + mu;
            cx<T> sc = ipow<T>(-e2);
            if ((sneg && (e2 & 1)) != (c.has_tgt_refl && (e2 & 1))) sc = -sc;
            T cf = (T)cs.coef;
            if (cs.kap < 0 && (cs.kap & 1)) cf = -cf;
            cx<T> k1 = ipow<T>(1 + cs.kap);
            cx<T> ph = E[pp * MW + (p + 2) + cs.kap - mu];
            cx<T> x = le_bar[(pairs[w.pair0 + pp].tgt * 3 + cs.vout) * P + nu * nu + nu + mu];
            v = (cf * sc) * (k1 * (ph * x));
        }
        X[r * GemmTile<T>::BNP + col] = v;
    }
    __syncthreads();
    const cx<T> *A = tab + ((int64_t)g.tab_index * NTAB + t) * P * P;
    auto store = [&](int k, int col, cx<T> y) {
        int pp = col / ncpp, j = col % ncpp;
        ColSpec cs = c_cols[t][j];
        int n = NN[k], m = k - n * n - n;
        int ms = cs.kap < 0 ? -m : m;
        int e1 = n + ms;
        cx<T> sc = ipow<T>(e1);
        if ((sneg && (e1 & 1)) != (c.has_src_refl && (e1 & 1))) sc = -sc;
        cx<T> yy = sc * (E[pp * MW + (p + 2) + ms] * y);
        atomic_add_cx(me_bar + (pairs[w.pair0 + pp].src * 3 + cs.vin) * P + n * n + n + ms, yy);
    };
    tiled_gemm<T, decltype(store), true>(P, blockIdx.y, A, X, As, ncol, store);
}

// tab_T[g][t][nu mu][n' m'] = I-hat * s_t^nu * s_s^n'  (level scaling, cast to T)
template <typename T>
__global__ void k_scale_tables(int p, int64_t g0, int64_t ng, const GeomDev *geoms,
                               const cd *tab64, cx<T> *tab)
{
    const int P = (p + 1) * (p + 1);
    int64_t gi = g0 + blockIdx.y;
    int t = blockIdx.z;
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P * P || gi >= g0 + ng) return;
    const GeomDev &g = geoms[gi];
    int row = e / P, col = e % P;
    int nu = (int)sqrt((double)row + 0.5), n1 = (int)sqrt((double)col + 0.5);
    while ((nu + 1) * (nu + 1) <= row) ++nu;
    while (nu * nu > row) --nu;
    while ((n1 + 1) * (n1 + 1) <= col) ++n1;
    while (n1 * n1 > col) --n1;
    double f = pow(g.scale_t, (double)nu) * pow(g.scale_s, (double)n1);
    cd v = tab64[((gi - g0) * NTAB + t) * (int64_t)P * P + e];
    tab[(g.tab_index * NTAB + t) * (int64_t)P * P + e] = cx<T>{(T)(f * v.x), (T)(f * v.y)};
}

// ---------------------------------------------------------------- launchers
// shared memory of k_group_gemm: the gathered columns and two tiles of the matrix
template <typename T>
static size_t group_gemm_smem(int p)
{
    using G = GemmTile<T>;
    const size_t P = (size_t)(p + 1) * (p + 1);
    return (P * G::BNP + (size_t)2 * G::BK * G::BMP) * sizeof(cx<T>);
}

// shared memory of k_m2l: as k_group_gemm, plus the pair phases and the degree table
template <typename T>
static size_t gemm_smem(int p)
{
    const int P = (p + 1) * (p + 1);
    using G = GemmTile<T>;
    return ((size_t)P * G::BNP + (size_t)2 * G::BK * G::BMP + (size_t)G::BN * (2 * p + 5)) * sizeof(cx<T>) +
           (size_t)P * sizeof(short) + 16;
}

template <typename T>
int gemm_cols()
{
    return 16 * TileCfg<T>::TN;
}
template int gemm_cols<float>();
template int gemm_cols<double>();

template <typename T>
void launch_group_gemm_t(int p, int64_t nwork, const GemmWork *work, const cx<T> *mats,
                         const int64_t *src, const int64_t *dst, const cx<T> *in, cx<T> *out,
                         bool atomic, cudaStream_t st)
{
    if (nwork <= 0) return;
    const unsigned nrt = (unsigned)(((p + 1) * (p + 1) + GemmTile<T>::BM - 1) / GemmTile<T>::BM);
    k_group_gemm<T><<<dim3((unsigned)nwork, nrt), 256, group_gemm_smem<T>(p), st>>>(p, work, mats, src, dst, in,
                                                                    out, atomic);
}

template <typename T>
void launch_m2l_t(int p, int64_t nwork, const M2LWork *work, const GeomDev *geoms,
                  const CompDev *comps, const M2LPair *pairs, const cx<T> *tab, const cx<T> *me,
                  cx<T> *le, cudaStream_t st)
{
    if (nwork <= 0) return;
    const unsigned nrt = (unsigned)(((p + 1) * (p + 1) + GemmTile<T>::BM - 1) / GemmTile<T>::BM);
    k_m2l<T><<<dim3((unsigned)nwork, nrt), 256, gemm_smem<T>(p), st>>>(p, work, geoms, comps, pairs, tab, me,
                                                             le);
}

template <typename T>
void launch_m2l_tr(int p, int64_t nwork, const M2LWork *work, const GeomDev *geoms,
                   const CompDev *comps, const M2LPair *pairs, const cx<T> *tab, const cx<T> *le_bar,
                   cx<T> *me_bar, cudaStream_t st)
{
    if (nwork <= 0) return;
    const unsigned nrt = (unsigned)(((p + 1) * (p + 1) + GemmTile<T>::BM - 1) / GemmTile<T>::BM);
    k_m2l_tr<T><<<dim3((unsigned)nwork, nrt), 256, gemm_smem<T>(p), st>>>(p, work, geoms, comps, pairs, tab,
                                                                           le_bar, me_bar);
}

template <typename T>
void launch_scale_tables(int p, int64_t g0, int64_t ng, const GeomDev *geoms, const cd *tab64,
                         cx<T> *tab, cudaStream_t st)
{
    if (ng <= 0) return;
    const int P = (p + 1) * (p + 1);
    dim3 grid((P * P + 255) / 256, (unsigned)ng, NTAB);
    k_scale_tables<T><<<grid, 256, 0, st>>>(p, g0, ng, geoms, tab64, tab);
}

template void launch_group_gemm_t<float>(int, int64_t, const GemmWork *, const cf *,
                                         const int64_t *, const int64_t *, const cf *, cf *, bool,
                                         cudaStream_t);
template void launch_group_gemm_t<double>(int, int64_t, const GemmWork *, const cd *,
                                          const int64_t *, const int64_t *, const cd *, cd *,
                                          bool, cudaStream_t);
template void launch_m2l_t<float>(int, int64_t, const M2LWork *, const GeomDev *, const CompDev *,
                                  const M2LPair *, const cf *, const cf *, cf *, cudaStream_t);
template void launch_m2l_t<double>(int, int64_t, const M2LWork *, const GeomDev *,
                                   const CompDev *, const M2LPair *, const cd *, const cd *, cd *,
                                   cudaStream_t);
template void launch_m2l_tr<float>(int, int64_t, const M2LWork *, const GeomDev *, const CompDev *,
                                   const M2LPair *, const cf *, const cf *, cf *, cudaStream_t);
template void launch_m2l_tr<double>(int, int64_t, const M2LWork *, const GeomDev *, const CompDev *,
                                    const M2LPair *, const cd *, const cd *, cd *, cudaStream_t);
template void launch_scale_tables<float>(int, int64_t, int64_t, const GeomDev *, const cd *, cf *,
                                         cudaStream_t);
template void launch_scale_tables<double>(int, int64_t, int64_t, const GeomDev *, const cd *,
                                          cd *, cudaStream_t);

cudaError_t configure_trans_kernels()
{
    const int big = 220 * 1024;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_group_gemm<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_group_gemm<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_m2l<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_m2l<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_m2l_tr<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_m2l_tr<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    // these CTAs hold ~100 KB of shared memory: take the whole carveout so that two fit on an SM
    const int mx = (int)cudaSharedmemCarveoutMaxShared;
    if ((e = cudaFuncSetAttribute(k_group_gemm<float>, cudaFuncAttributePreferredSharedMemoryCarveout, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_group_gemm<double>, cudaFuncAttributePreferredSharedMemoryCarveout, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_m2l<float>, cudaFuncAttributePreferredSharedMemoryCarveout, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_m2l<double>, cudaFuncAttributePreferredSharedMemoryCarveout, mx))) return e;
    return configure_m2l_tc();
}

}  // namespace lmf
