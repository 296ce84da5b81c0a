// Matvec kernels (FP64 form): permutation to helical components, P2M, M2M,
// M2L, L2L, L2P and the near-field S2T, plus the S2T precomputation.
#include "kernels.cuh"
#include "quad.cuh"
#include "specfun.cuh"

namespace lmf {


// ------------------------------------------------------------ permutation
// Caller buffers are complex128 or complex64 [N][3]; the helical work arrays
// are complex128 in sorted order.
template <typename TI>
__device__ __forceinline__ cd load_c(const TI *p) { return cd{(double)p->x, (double)p->y}; }

// q_h[i] = (J_x + i J_y, J_x - i J_y, J_z) of point perm[i] (optionally of conj J)
template <typename TI>
__global__ void k_gather_in(int64_t N, const int64_t *perm, const TI *J, cd *qh, int cj)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int64_t o = perm[i];
    cd x = load_c(J + 3 * o), y = load_c(J + 3 * o + 1), z = load_c(J + 3 * o + 2);
    if (cj) { x = conj(x); y = conj(y); z = conj(z); }
    qh[3 * i] = x + mul_i(y);
    qh[3 * i + 1] = x - mul_i(y);
    qh[3 * i + 2] = z;
}

// Phi[perm[i]] = ((A+B)/2, (A-B)/(2i), C) of the helical result (optionally conj);
// the complex64 output is rounded once from the complex128 sum
template <typename TO>
__global__ void k_scatter_out(int64_t N, const int64_t *perm, const cd *ph, TO *Phi, int cj)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int64_t o = perm[i];
    cd A = ph[3 * i], B = ph[3 * i + 1], C = ph[3 * i + 2];
    cd x = 0.5 * (A + B), y = mul_mi(0.5 * (A - B));
    if (cj) { x = conj(x); y = conj(y); C = conj(C); }
    using E = decltype(Phi->x);
    Phi[3 * o] = TO{(E)x.x, (E)x.y};
    Phi[3 * o + 1] = TO{(E)y.x, (E)y.y};
    Phi[3 * o + 2] = TO{(E)C.x, (E)C.y};
}

void launch_gather_in(int64_t N, const int64_t *perm, const void *J, int dtype, cd *qh, bool conj_in,
                      cudaStream_t st)
{
    if (N <= 0) return;
    const unsigned g = (unsigned)((N + 255) / 256);
    if (dtype == LMFMM_C64)
        k_gather_in<cf><<<g, 256, 0, st>>>(N, perm, (const cf *)J, qh, conj_in);
    else
        k_gather_in<cd><<<g, 256, 0, st>>>(N, perm, (const cd *)J, qh, conj_in);
}
void launch_scatter_out(int64_t N, const int64_t *perm, const cd *phih, void *Phi, int dtype, bool conj_out,
                        cudaStream_t st)
{
    if (N <= 0) return;
    const unsigned g = (unsigned)((N + 255) / 256);
    if (dtype == LMFMM_C64)
        k_scatter_out<cf><<<g, 256, 0, st>>>(N, perm, phih, (cf *)Phi, conj_out);
    else
        k_scatter_out<cd><<<g, 256, 0, st>>>(N, perm, phih, (cd *)Phi, conj_out);
}

// Transposes of the two helical maps, for the transposed operator
// A^T = G^T H^T S^T of A = S H G (G: gather_in, S: scatter_out, H: the helical
// operator).  G = [[1, i, 0], [1, -i, 0], [0, 0, 1]] and
// S = [[1/2, 1/2, 0], [-i/2, i/2, 0], [0, 0, 1]] act on (x, y, z) and (A, B, C).
// ph_bar[i] = S^T y[perm[i]] (optionally of conj y)
template <typename TI>
__global__ void k_gather_tr(int64_t N, const int64_t *perm, const TI *y, cd *phb, int cj)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int64_t o = perm[i];
    cd x = load_c(y + 3 * o), yy = load_c(y + 3 * o + 1), z = load_c(y + 3 * o + 2);
    if (cj) { x = conj(x); yy = conj(yy); z = conj(z); }
    phb[3 * i] = 0.5 * (x - mul_i(yy));
    phb[3 * i + 1] = 0.5 * (x + mul_i(yy));
    phb[3 * i + 2] = z;
}

// out[perm[i]] = G^T qh_bar[i] (optionally conjugated)
template <typename TO>
__global__ void k_scatter_tr(int64_t N, const int64_t *perm, const cd *qhb, TO *out, int cj)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int64_t o = perm[i];
    const cd a = qhb[3 * i], b = qhb[3 * i + 1];
    cd x = a + b, y = mul_i(a - b), z = qhb[3 * i + 2];
    if (cj) { x = conj(x); y = conj(y); z = conj(z); }
    using E = decltype(out->x);
    out[3 * o] = TO{(E)x.x, (E)x.y};
    out[3 * o + 1] = TO{(E)y.x, (E)y.y};
    out[3 * o + 2] = TO{(E)z.x, (E)z.y};
}

void launch_gather_tr(int64_t N, const int64_t *perm, const void *y, int dtype, cd *phb, bool conj_in,
                      cudaStream_t st)
{
    if (N <= 0) return;
    const unsigned g = (unsigned)((N + 255) / 256);
    if (dtype == LMFMM_C64)
        k_gather_tr<cf><<<g, 256, 0, st>>>(N, perm, (const cf *)y, phb, conj_in);
    else
        k_gather_tr<cd><<<g, 256, 0, st>>>(N, perm, (const cd *)y, phb, conj_in);
}
void launch_scatter_tr(int64_t N, const int64_t *perm, const cd *qhb, void *out, int dtype, bool conj_out,
                       cudaStream_t st)
{
    if (N <= 0) return;
    const unsigned g = (unsigned)((N + 255) / 256);
    if (dtype == LMFMM_C64)
        k_scatter_tr<cf><<<g, 256, 0, st>>>(N, perm, qhb, (cf *)out, conj_out);
    else
        k_scatter_tr<cd><<<g, 256, 0, st>>>(N, perm, qhb, (cd *)out, conj_out);
}

// --------------------------------------------------------------- P2M, L2P
// ------------------------------------------------- basis of a chunk of points
// b_nm(r) = scale * j_n(k |r|) Y_n^m(r^) / s^n with Y_n^m = P^_n^|m| e^{i m phi}
// (times (-1)^m for m < 0), s = |k| S_leaf; P2M uses scale = 4 pi and conj(Y)
// (eq. mecoeff).  FP64 form in double; mixed form in float when |k r| < 1.5.
// The whole CTA builds the basis of up to CH points at once: one thread per
// point for the radial factors j_n (and the angle seeds), then one thread per
// (point, pair of orders m, p - m) for the normalised Legendre recurrence in n,
// whose coefficients come from a per-CTA table.
constexpr int SER_K = 14;   // terms of the power series of j_n

template <typename T>
struct LegTab {
    T *a, *b;   // [n(n+1)/2 + m]: P_n^m = a (x P_{n-1}^m - b P_{n-2}^m), n >= m + 2
    T *d;       // [m]: P_{m+1}^m = d x P_m^m
    T *c;       // [m]: P_m^m = -c s P_{m-1}^m, c = sqrt((2m+1)/(2m)), c[0] = 1/sqrt(4 pi)
    T *sk;      // [n][k-1]: 1 / (k (2n+2k+1)), ratio of consecutive series terms of j_n
    T *idf;     // [n]: 1 / (2n+1)!!
};

template <typename T>
__host__ __device__ constexpr size_t legtab_elems(int p)
{
    return (size_t)(p + 1) * (p + 2) + 3 * (size_t)(p + 1) + (size_t)(p + 1) * SER_K;
}

template <typename T>
__device__ inline LegTab<T> legtab_fill(int p, T *mem)
{
    const int NT = (p + 1) * (p + 2) / 2;
    LegTab<T> L{mem, mem + NT, mem + 2 * NT, mem + 2 * NT + p + 1, mem + 2 * NT + 2 * (p + 1),
                mem + 2 * NT + 2 * (p + 1) + (p + 1) * SER_K};
    for (int e = threadIdx.x; e < NT; e += blockDim.x) {
        int n = (int)sqrtf(2.0f * e + 0.25f);
        while ((n + 1) * (n + 2) / 2 <= e) ++n;
        while (n * (n + 1) / 2 > e) --n;
        const int m = e - n * (n + 1) / 2;
        T av = T(0), bv = T(0);
        if (n >= m + 2) {
            av = sqrt(T(4 * n * n - 1) / T(n * n - m * m));
            bv = sqrt(T((n - 1) * (n - 1) - m * m) / T(4 * (n - 1) * (n - 1) - 1));
        }
        L.a[e] = av;
        L.b[e] = bv;
    }
    for (int m = threadIdx.x; m <= p; m += blockDim.x) {
        L.d[m] = sqrt(T(2 * m + 3));
        L.c[m] = m == 0 ? T(0.28209479177387814347) : sqrt(T(2 * m + 1) / T(2 * m));
        T df = T(1);
        for (int i = 1; i <= m; ++i) df *= T(2 * i + 1);
        L.idf[m] = T(1) / df;
    }
    for (int e = threadIdx.x; e < (p + 1) * SER_K; e += blockDim.x) {
        const int n = e / SER_K, k = e - n * SER_K + 1;
        L.sk[e] = T(1) / (T(k) * T(2 * n + 2 * k + 1));
    }
    return L;
}

// angle seeds of point j, geo[j] = (cos theta, sin theta, Re e^{i phi},
// Im e^{i phi}) (conjugated for P2M), and its radial factors jr[j][n]
// (scale / s^n included) when they come from the FP64 recurrence; otherwise
// (mixed form, |k r| < 1.5) kz[j] = (k r, k r / s) for the power series,
// evaluated one degree per thread by series_degree
template <typename T>
__device__ inline void point_seed(int p, cd k, double dx, double dy, double dz, bool conjugate,
                                  double scale, double inv_s, cx<T> *jr, T *geo, cx<T> *kz)
{
    if constexpr (sizeof(T) == 4) {
        // mixed form: angles and k r in FP32 (the FP64 pipe is 1/64 of the FP32 one)
        const float fx = (float)dx, fy = (float)dy, fz = (float)dz;
        const float rxy = sqrtf(fx * fx + fy * fy), r = sqrtf(fx * fx + fy * fy + fz * fz);
        const cf kf{(float)k.x, (float)k.y};
        const cf kr = r * kf;
        if (abs2(kr) < 2.25f) {
            geo[0] = r > 0.f ? fz / r : 1.f;
            geo[1] = r > 0.f ? rxy / r : 0.f;
            geo[2] = rxy > 0.f ? fx / rxy : 1.f;
            geo[3] = rxy > 0.f ? (conjugate ? -fy : fy) / rxy : 0.f;
            kz[0] = cx<T>{kr.x, kr.y};
            kz[1] = (r * (float)inv_s) * cx<T>{kf.x, kf.y};
            return;
        }
    }
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    const double rxy = sqrt(dx * dx + dy * dy);
    geo[0] = (T)(r > 0 ? dz / r : 1.0);
    geo[1] = (T)(r > 0 ? rxy / r : 0.0);
    geo[2] = (T)(rxy > 0 ? dx / rxy : 1.0);
    geo[3] = (T)(rxy > 0 ? (conjugate ? -dy : dy) / rxy : 0.0);
    const cd kr = k * r;
    {
        kz[0] = cx<T>{T(-1), T(0)};   // marker: jr already set
        cd jd[LMF_PMAX + 1];
        sph_bessel_seq(kr, p, jd);
        double sp = scale;
        for (int n = 0; n <= p; ++n) {
            jr[n] = cx<T>{(T)(sp * jd[n].x), (T)(sp * jd[n].y)};
            sp *= inv_s;
        }
    }
}

// scale * j_n(z) / w^n, z = k r, for |z| < 1.5 by the power series
//   j_n(z) = z^n / (2n+1)!! sum_k (-z^2/2)^k / (k! (2n+3)(2n+5)...(2n+2k+1)),
// carried out in T with zeta = z / w so that no power of z over- or underflows
template <typename T>
__device__ inline cx<T> series_degree(int n, cx<T> z, cx<T> zeta, T scale, const LegTab<T> &L)
{
    const cx<T> q = T(-0.5) * (z * z);
    cx<T> zn{T(1), T(0)};
    for (int i = 0; i < n; ++i) zn = zn * zeta;
    cx<T> term{T(1), T(0)}, sum{T(1), T(0)};
    for (int k = 1; k <= SER_K; ++k) {
        term = term * q * L.sk[n * SER_K + k - 1];
        sum += term;
        if (abs2(term) < T(1e-18) * abs2(sum)) break;
    }
    return scale * ((zn * sum) * L.idf[n]);
}

// column m of point j: b_{n, +-m} for n = m..p into bj[n^2 + n +- m], from
// P_m^m (pmm) and e^{i m phi} (em) already advanced to order m
template <typename T>
__device__ inline void basis_column(int p, int m, T x, T pmm, cx<T> em, const cx<T> *jr,
                                    const LegTab<T> &L, cx<T> *bj)
{
    const cx<T> emc = conj(em);
    const T sg = (m & 1) ? T(-1) : T(1);
    auto put = [&](int n, T pl) {
        const cx<T> jv = pl * jr[n];
        bj[n * n + n + m] = jv * em;
        if (m > 0) bj[n * n + n - m] = sg * (jv * emc);
    };
    put(m, pmm);
    if (m == p) return;
    T p0 = pmm, p1 = L.d[m] * x * pmm;
    put(m + 1, p1);
    for (int n = m + 2; n <= p; ++n) {
        const int e = n * (n + 1) / 2 + m;
        const T p2 = L.a[e] * (x * p1 - L.b[e] * p0);
        put(n, p2);
        p0 = p1;
        p1 = p2;
    }
}

// basis of points t0 .. t0+np-1 (np <= CH) into bas[j * P + index]; the caller
// synchronises before reading bas
template <typename T>
__device__ inline void chunk_basis(int p, cd k, const double *xyz, const double *ctr, int64_t t0, int np,
                                   bool conjugate, double scale, double inv_s, const LegTab<T> &L,
                                   cx<T> *jr, T *geo, cx<T> *kz, cx<T> *bas)
{
    const int P = (p + 1) * (p + 1);
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        const int64_t t = t0 + j;
        point_seed<T>(p, k, xyz[3 * t] - ctr[0], xyz[3 * t + 1] - ctr[1], xyz[3 * t + 2] - ctr[2],
                      conjugate, scale, inv_s, jr + j * (p + 1), geo + 4 * j, kz + 2 * j);
    }
    __syncthreads();
    if (sizeof(T) == 4) {
        for (int task = threadIdx.x; task < np * (p + 1); task += blockDim.x) {
            const int j = task / (p + 1), n = task - j * (p + 1);
            const cx<T> z = kz[2 * j];
            if (z.x == T(-1) && z.y == T(0)) continue;   // recurrence path: jr is set
            jr[task] = series_degree<T>(n, z, kz[2 * j + 1], (T)scale, L);
        }
        __syncthreads();
    }
    // orders m and p - m share a task: p + 2 terms of the recurrence per task
    const int nt = p / 2 + 1;
    for (int task = threadIdx.x; task < np * nt; task += blockDim.x) {
        const int j = task / nt, m1 = task - j * nt, m2 = p - m1;
        const T x = geo[4 * j], sv = geo[4 * j + 1];
        const cx<T> e1{geo[4 * j + 2], geo[4 * j + 3]};
        T pmm = L.c[0];
        cx<T> em{T(1), T(0)};
        for (int m = 1; m <= m1; ++m) {
            pmm = -pmm * sv * L.c[m];
            em = em * e1;
        }
        basis_column<T>(p, m1, x, pmm, em, jr + j * (p + 1), L, bas + (size_t)j * P);
        if (m2 != m1) {
            for (int m = m1 + 1; m <= m2; ++m) {
                pmm = -pmm * sv * L.c[m];
                em = em * e1;
            }
            basis_column<T>(p, m2, x, pmm, em, jr + j * (p + 1), L, bas + (size_t)j * P);
        }
    }
}

// shared-memory plan of the P2M / L2P kernels: CH points per chunk
template <typename T>
struct LeafSmem {
    int CH;
    size_t leg, geo, kz, jr, bas, extra, total;   // byte offsets, extra: hq (P2M) or L (L2P)
};

template <typename T>
__host__ __device__ inline LeafSmem<T> leaf_smem(int p, bool l2p, size_t cap)
{
    const size_t P = (size_t)(p + 1) * (p + 1);
    LeafSmem<T> s{};
    for (s.CH = 32; s.CH >= 4; s.CH /= 2) {
        s.leg = 0;
        s.geo = (legtab_elems<T>(p) * sizeof(T) + 15) & ~(size_t)15;
        s.kz = s.geo + ((4 * s.CH * sizeof(T) + 15) & ~(size_t)15);
        s.jr = s.kz + 2 * s.CH * sizeof(cx<T>);
        s.bas = s.jr + s.CH * (p + 1) * sizeof(cx<T>);
        s.extra = s.bas + s.CH * P * sizeof(cx<T>);
        s.total = s.extra + (l2p ? 3 * P : 3 * (size_t)s.CH) * sizeof(cx<T>);
        if (s.total <= cap) break;
    }
    return s;
}

constexpr size_t LEAF_SMEM_CAP = 200 * 1024;   // dynamic shared memory granted to these kernels

// One CTA per leaf: chunks of CH points are turned into their basis by the
// whole CTA, then each thread accumulates its multipole coefficients over the
// chunk's points.  The basis is P2M's (conj_basis, scale = 4 pi: eq. mecoeff)
// or L2P's (plain Y, scale 1), the latter for the transpose of L2P, whose
// coefficients sum the point values against the same functions L2P evaluates.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_p2m(int p, int CH, const int64_t *leaves, const BoxDev *boxes,
                                             const double *xyz, const cd *qh, MediumDev M, LayerScale ls,
                                             cx<T> *me, int conj_basis, double scale)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int P = (p + 1) * (p + 1);
    const LeafSmem<T> sp = leaf_smem<T>(p, false, LEAF_SMEM_CAP);
    const LegTab<T> L = legtab_fill<T>(p, (T *)(smraw + sp.leg));
    T *geo = (T *)(smraw + sp.geo);
    cx<T> *kz = (cx<T> *)(smraw + sp.kz);
    cx<T> *jr = (cx<T> *)(smraw + sp.jr);
    cx<T> *bas = (cx<T> *)(smraw + sp.bas);
    cx<T> *hq = (cx<T> *)(smraw + sp.extra);   // [CH][3]
    const int64_t bi = leaves[blockIdx.x];
    const BoxDev b = boxes[bi];
    const cd k = M.k[b.layer];
    const double inv_s = 1.0 / ls.s[b.layer];
    const int NO = 3 * P;
    constexpr int PERMAX = (3 * (LMF_PMAX + 1) * (LMF_PMAX + 1) + 255) / 256;
    cx<T> acc[PERMAX];
#pragma unroll
    for (int i = 0; i < PERMAX; ++i) acc[i] = cx<T>{T(0), T(0)};
    for (int64_t c0 = b.p0; c0 < b.p1; c0 += CH) {
        const int np = (int)min((int64_t)CH, b.p1 - c0);
        for (int e = threadIdx.x; e < 3 * np; e += blockDim.x)
            hq[e] = cx<T>{(T)qh[3 * c0 + e].x, (T)qh[3 * c0 + e].y};
        chunk_basis<T>(p, k, xyz, b.c, c0, np, conj_basis != 0, scale, inv_s, L, jr, geo, kz, bas);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < PERMAX; ++i) {
            const int o = threadIdx.x + i * blockDim.x;
            if (o < NO) {
                const int v = o / P, nm = o - v * P;
                cx<T> a = acc[i];
                for (int j = 0; j < np; ++j) a += hq[3 * j + v] * bas[j * P + nm];
                acc[i] = a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < PERMAX; ++i) {
        const int o = threadIdx.x + i * blockDim.x;
        if (o < NO) me[bi * NO + o] = acc[i];
    }
}

// One CTA per leaf: chunks of CH target points are turned into their basis by
// the whole CTA, then one warp per point contracts it with the three local
// expansions held in shared memory.  The basis is L2P's (plain Y, scale 1:
// eq. maxwell_LE_layered) or P2M's (conj_basis, scale 4 pi), the latter for the
// transpose of P2M.  accumulate: add into ph instead of overwriting it.
template <typename T>
__global__ void __launch_bounds__(256) k_l2p(int p, int CH, const int64_t *leaves, const BoxDev *boxes,
                                             const double *xyz, const cx<T> *le, MediumDev M, LayerScale ls,
                                             cd *ph, int conj_basis, double scale, int accumulate)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int P = (p + 1) * (p + 1);
    const LeafSmem<T> sp = leaf_smem<T>(p, true, LEAF_SMEM_CAP);
    const LegTab<T> L = legtab_fill<T>(p, (T *)(smraw + sp.leg));
    T *geo = (T *)(smraw + sp.geo);
    cx<T> *kz = (cx<T> *)(smraw + sp.kz);
    cx<T> *jr = (cx<T> *)(smraw + sp.jr);
    cx<T> *bas = (cx<T> *)(smraw + sp.bas);
    cx<T> *Lc = (cx<T> *)(smraw + sp.extra);   // [3][P]
    const int64_t bi = leaves[blockIdx.x];
    const BoxDev b = boxes[bi];
    for (int e = threadIdx.x; e < 3 * P; e += blockDim.x) Lc[e] = le[bi * 3 * P + e];
    const cd k = M.k[b.layer];
    const double inv_s = 1.0 / ls.s[b.layer];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    for (int64_t c0 = b.p0; c0 < b.p1; c0 += CH) {
        const int np = (int)min((int64_t)CH, b.p1 - c0);
        chunk_basis<T>(p, k, xyz, b.c, c0, np, conj_basis != 0, scale, inv_s, L, jr, geo, kz, bas);
        __syncthreads();
        for (int j = warp; j < np; j += nwarp) {
            cx<T> A{T(0), T(0)}, B{T(0), T(0)}, C{T(0), T(0)};
            for (int i = lane; i < P; i += 32) {
                const cx<T> bv = bas[j * P + i];
                A += Lc[i] * bv;
                B += Lc[P + i] * bv;
                C += Lc[2 * P + i] * bv;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                A.x += __shfl_xor_sync(0xffffffffu, A.x, o);
                A.y += __shfl_xor_sync(0xffffffffu, A.y, o);
                B.x += __shfl_xor_sync(0xffffffffu, B.x, o);
                B.y += __shfl_xor_sync(0xffffffffu, B.y, o);
                C.x += __shfl_xor_sync(0xffffffffu, C.x, o);
                C.y += __shfl_xor_sync(0xffffffffu, C.y, o);
            }
            if (lane == 0) {
                const int64_t t = c0 + j;
                cd o[3] = {cd{(double)A.x, (double)A.y}, cd{(double)B.x, (double)B.y}, cd{(double)C.x, (double)C.y}};
                if (accumulate)
                    for (int v = 0; v < 3; ++v) o[v] += ph[3 * t + v];
                ph[3 * t] = o[0];
                ph[3 * t + 1] = o[1];
                ph[3 * t + 2] = o[2];
            }
        }
        __syncthreads();
    }
}

template <typename T>
void launch_p2m(int p, int64_t nleaf, const int64_t *leaves, const BoxDev *boxes,
                const double *xyz, const cd *qh, const MediumDev &M, const LayerScale &ls,
                cx<T> *me, cudaStream_t st, bool l2p_basis)
{
    if (nleaf <= 0) return;
    const LeafSmem<T> sp = leaf_smem<T>(p, false, LEAF_SMEM_CAP);
    k_p2m<T><<<(unsigned)nleaf, 256, sp.total, st>>>(p, sp.CH, leaves, boxes, xyz, qh, M, ls, me, l2p_basis ? 0 : 1,
                                                     l2p_basis ? 1.0 : 4.0 * LMF_PI);
}

template <typename T>
void launch_l2p(int p, int64_t nleaf, const int64_t *leaves, const BoxDev *boxes,
                const double *xyz, const cx<T> *le, const MediumDev &M, const LayerScale &ls,
                cd *phih, cudaStream_t st, bool p2m_basis, bool accumulate)
{
    if (nleaf <= 0) return;
    const LeafSmem<T> sp = leaf_smem<T>(p, true, LEAF_SMEM_CAP);
    k_l2p<T><<<(unsigned)nleaf, 256, sp.total, st>>>(p, sp.CH, leaves, boxes, xyz, le, M, ls, phih, p2m_basis ? 1 : 0,
                                                     p2m_basis ? 4.0 * LMF_PI : 1.0, accumulate ? 1 : 0);
}

template void launch_p2m<float>(int, int64_t, const int64_t *, const BoxDev *, const double *,
                                const cd *, const MediumDev &, const LayerScale &, cf *,
                                cudaStream_t, bool);
template void launch_p2m<double>(int, int64_t, const int64_t *, const BoxDev *, const double *,
                                 const cd *, const MediumDev &, const LayerScale &, cd *,
                                 cudaStream_t, bool);
template void launch_l2p<float>(int, int64_t, const int64_t *, const BoxDev *, const double *,
                                const cf *, const MediumDev &, const LayerScale &, cd *,
                                cudaStream_t, bool, bool);
template void launch_l2p<double>(int, int64_t, const int64_t *, const BoxDev *, const double *,
                                 const cd *, const MediumDev &, const LayerScale &, cd *,
                                 cudaStream_t, bool, bool);

// --------------------------------------------------------------------- S2T
// For every point pair (j in the source leaf, i in the target leaf) of a near
// box pair, the five Sommerfeld integrals
//   I_t = int k J_kappa_t(k rho) Z(k, zbar_j, zbar'_i) sigma_t(k) dk,
//   t: (s1,0) (s5,0) (s2,1) (s4,1) (s3,2),
// on Gamma_1 and a real tail set by the smallest vertical transmission
// distance and the largest horizontal distance of the box pair.
// J_0, J_1, J_2 (kind 0) or H^(1)/2, H^(2)/2 (kinds 1, 2) of k rho
static __device__ inline void bessel_012(int kind, cd z, cd &J0, cd &J1, cd &J2)
{
    if (kind != 0) {
        cd H[3];
        hankel1_seq(kind == 2 ? conj(z) : z, 2, H);
        if (kind == 2) { H[0] = conj(H[0]); H[1] = conj(H[1]); H[2] = conj(H[2]); }
        J0 = 0.5 * H[0];
        J1 = 0.5 * H[1];
        J2 = 0.5 * H[2];
        return;
    }
    if (z.y == 0.0 && z.x > 8.0) {
        double x = z.x;
        double j0v = j0(x), j1v = j1(x);
        J0 = mkd(j0v);
        J1 = mkd(j1v);
        J2 = mkd(2.0 * j1v / x - j0v);
        return;
    }
    cd J[3];
    bessel_j_seq<3>(z, 2, J);
    J0 = J[0];
    J1 = J[1];
    J2 = J[2];
}

__global__ void k_s2t_pre(const NearPair *near, const BoxDev *boxes, const double *xyz,
                          MediumDev M, const CompDev *comps, double a, int node_cap, cd *coef,
                          int *flag)
{
    const int CH = 64;
    __shared__ cd s_w[CH], s_kr[CH], s_kz[CH], s_kzp[CH], s_sg[CH][5];
    __shared__ int s_kind[CH];
    __shared__ QuadPlanDev pl;
    NearPair np = near[blockIdx.x];
    const CompDev c = comps[np.comp];
    BoxDev B = boxes[np.src], C = boxes[np.tgt];
    int64_t nB = B.p1 - B.p0, nC = C.p1 - C.p0;
    int64_t npp = nB * nC;
    if (threadIdx.x == 0) {
        pl = make_plan(a, np.rhomax, np.dzmin, 3, false);
        if (plan_nodes(pl) > node_cap) {
            // bounded work: flag the pair (the build reports LMFMM_ERR_QUAD) and clamp
            atomicOr(flag, 2);
            pl.nmid = 16;
            pl.nray = 0;
        }
    }
    __syncthreads();
    int Q = plan_nodes(pl);
    cd *cf = coef + np.coef0 * 5;
    for (int64_t e = threadIdx.x; e < npp * 5; e += blockDim.x) cf[e] = mkd(0.0);
    cd k = M.k[c.l], kpz = M.k[c.lp];
    __syncthreads();
    for (int q0 = 0; q0 < Q; q0 += CH) {
        int nq = min(CH, Q - q0);
        if (threadIdx.x < nq) {
            int q = q0 + threadIdx.x;
            cd kr, w;
            s_kind[threadIdx.x] = plan_node(pl, q, kr, w);
            s_kr[threadIdx.x] = kr;
            s_w[threadIdx.x] = w;
            s_kz[threadIdx.x] = kz_of(k, kr);
            s_kzp[threadIdx.x] = kz_of(kpz, kr);
            cd sg[5];
            sigmas_dev(M, kr, c.l, c.lp, c.tu, c.su, sg);
            s_sg[threadIdx.x][0] = sg[0];
            s_sg[threadIdx.x][1] = sg[4];
            s_sg[threadIdx.x][2] = sg[1];
            s_sg[threadIdx.x][3] = sg[3];
            s_sg[threadIdx.x][4] = sg[2];
        }
        __syncthreads();
        for (int64_t e = threadIdx.x; e < npp; e += blockDim.x) {
            int64_t ii = e / nB, jj = e % nB;
            int64_t ti = C.p0 + ii, sj = B.p0 + jj;
            double dx = xyz[3 * sj] - xyz[3 * ti], dy = xyz[3 * sj + 1] - xyz[3 * ti + 1];
            double rho = sqrt(dx * dx + dy * dy);
            double zs = comp_src_z(c, xyz[3 * sj + 2]), zt = comp_tgt_z(c, xyz[3 * ti + 2]);
            cd acc[5];
            for (int u = 0; u < 5; ++u) acc[u] = cf[e * 5 + u];
            for (int q = 0; q < nq; ++q) {
                cd J0, J1, J2;
                bessel_012(s_kind[q], s_kr[q] * rho, J0, J1, J2);
                cd Z = cexpd(mul_i(c.s * (s_kz[q] * zs - s_kzp[q] * zt)));
                cd wZ = s_w[q] * Z;
                acc[0] += (wZ * J0) * s_sg[q][0];
                acc[1] += (wZ * J0) * s_sg[q][1];
                acc[2] += (wZ * J1) * s_sg[q][2];
                acc[3] += (wZ * J1) * s_sg[q][3];
                acc[4] += (wZ * J2) * s_sg[q][4];
            }
            for (int u = 0; u < 5; ++u) cf[e * 5 + u] = acc[u];
        }
        __syncthreads();
    }
}

void launch_s2t_pre(int64_t nnear, const NearPair *near, const BoxDev *boxes, const double *xyz,
                    const MediumDev &M, const CompDev *comps, double a, int node_cap, cd *coef,
                    int *dflag, cudaStream_t st)
{
    if (nnear <= 0) return;
    k_s2t_pre<<<(unsigned)nnear, 128, 0, st>>>(near, boxes, xyz, M, comps, a, node_cap, coef, dflag);
}

// Phi_h(i) += G^{*star}(r_j, r_i) q_j for the near pairs, in helical form with
// L_kappa = i^(kappa+1)/(4 pi) e^{i kappa phi} I_t and L_{-kappa} = the same
// with e^{-i kappa phi}; (rho, phi) is the polar form of r_j - r_i.
__global__ void k_s2t_apply(const NearPair *near, const BoxDev *boxes, const double *xyz,
                            const cd *coef, const cd *qh, cd *ph)
{
    NearPair np = near[blockIdx.x];
    BoxDev B = boxes[np.src], C = boxes[np.tgt];
    int64_t nB = B.p1 - B.p0, nC = C.p1 - C.p0;
    const cd *cf = coef + np.coef0 * 5;
    const double f = 1.0 / (4.0 * LMF_PI);
    for (int64_t ii = threadIdx.x; ii < nC; ii += blockDim.x) {
        int64_t ti = C.p0 + ii;
        cd A = mkd(0.0), Bv = mkd(0.0), Cv = mkd(0.0);
        for (int64_t jj = 0; jj < nB; ++jj) {
            int64_t sj = B.p0 + jj;
            double dx = xyz[3 * sj] - xyz[3 * ti], dy = xyz[3 * sj + 1] - xyz[3 * ti + 1];
            double rho = sqrt(dx * dx + dy * dy);
            cd e1 = rho > 0 ? cd{dx / rho, dy / rho} : cd{1.0, 0.0};
            cd e2 = e1 * e1;
            const cd *I = cf + (ii * nB + jj) * 5;
            cd L0s1 = mkd(0.0, f) * I[0];             // i/(4pi)
            cd L0s5 = mkd(0.0, f) * I[1];
            cd L1s2 = -f * (e1 * I[2]), Lm1s2 = -f * (conj(e1) * I[2]);
            cd L1s4 = -f * (e1 * I[3]), Lm1s4 = -f * (conj(e1) * I[3]);
            cd L2s3 = mkd(0.0, -f) * (e2 * I[4]), Lm2s3 = mkd(0.0, -f) * (conj(e2) * I[4]);
            cd a = qh[3 * sj], b = qh[3 * sj + 1], cc = qh[3 * sj + 2];
            A += 0.5 * (L0s1 * a) - 0.5 * (L2s3 * b) + L1s2 * cc;
            Bv += 0.5 * (L0s1 * b) - 0.5 * (Lm2s3 * a) + Lm1s2 * cc;
            Cv += L0s5 * cc + 0.5 * (Lm1s4 * a) + 0.5 * (L1s4 * b);
        }
        atomicAdd(&ph[3 * ti].x, A.x);
        atomicAdd(&ph[3 * ti].y, A.y);
        atomicAdd(&ph[3 * ti + 1].x, Bv.x);
        atomicAdd(&ph[3 * ti + 1].y, Bv.y);
        atomicAdd(&ph[3 * ti + 2].x, Cv.x);
        atomicAdd(&ph[3 * ti + 2].y, Cv.y);
    }
}

// The matvec's near field with the angular factors and constants of the
// helical form folded in once at setup: for target i and source j of a near
// pair, with e = e^{i phi} (phi the horizontal angle of r_j - r_i) and
// c = 1/(4 pi),
//   A += k0 a + k6 b + k2 c_,   B += k0 b + k7 a + k3 c_,   C += k1 c_ + k5 a + k4 b,
//   k0 = i c I0 / 2,  k1 = i c I1,  k2 = -c e I2,  k3 = -c conj(e) I2,
//   k4 = -c e I3 / 2,  k5 = -c conj(e) I3 / 2,  k6 = i c e^2 I4 / 2,  k7 = i c conj(e)^2 I4 / 2,
// (a, b, c_) the helical charges; I0..I4 the five Sommerfeld integrals of
// k_s2t_pre (same terms as k_s2t_apply).  Layout per near pair: [j][k0..k7][i],
// consecutive targets contiguous, 8 coefficients per point pair.
__global__ void k_s2t_combine(const NearPair *near, const BoxDev *boxes, const double *xyz,
                              const cd *coef5, cd *coef8)
{
    NearPair np = near[blockIdx.x];
    BoxDev B = boxes[np.src], C = boxes[np.tgt];
    const int64_t nB = B.p1 - B.p0, nC = C.p1 - C.p0;
    const cd *I5 = coef5 + np.coef0 * 5;
    cd *K = coef8 + np.coef0 * 8;
    const double f = 1.0 / (4.0 * LMF_PI);
    for (int64_t e = threadIdx.x; e < nB * nC; e += blockDim.x) {
        const int64_t ii = e / nB, jj = e % nB;
        const int64_t ti = C.p0 + ii, sj = B.p0 + jj;
        const double dx = xyz[3 * sj] - xyz[3 * ti], dy = xyz[3 * sj + 1] - xyz[3 * ti + 1];
        const double rho = sqrt(dx * dx + dy * dy);
        const cd e1 = rho > 0 ? cd{dx / rho, dy / rho} : cd{1.0, 0.0}, e2 = e1 * e1;
        const cd *I = I5 + e * 5;
        cd k[8];
        k[0] = mkd(0.0, 0.5 * f) * I[0];
        k[1] = mkd(0.0, f) * I[1];
        k[2] = -f * (e1 * I[2]);
        k[3] = -f * (conj(e1) * I[2]);
        k[4] = (-0.5 * f) * (e1 * I[3]);
        k[5] = (-0.5 * f) * (conj(e1) * I[3]);
        k[6] = mkd(0.0, 0.5 * f) * (e2 * I[4]);
        k[7] = mkd(0.0, 0.5 * f) * (conj(e2) * I[4]);
        for (int u = 0; u < 8; ++u) K[(jj * 8 + u) * nC + ii] = k[u];
    }
}

// Phi_h(i) += near-field terms of k_s2t_combine's coefficients.  One thread per
// target row (a target of one near pair against a block of up to S2T_SRC of
// the pair's sources), rows of a pair on consecutive threads: the coefficients
// are read coalesced over targets and the charges are broadcast; small box
// pairs share CTAs, crowded ones spread over many.
__global__ void __launch_bounds__(256) k_s2t_apply8(int64_t nrow, const S2TRow *rows, const NearPair *near,
                                                    const BoxDev *boxes, const cd *coef8, const cd *qh, cd *ph)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nrow) return;
    const S2TRow w = rows[e];
    const NearPair np = near[w.pair];
    const BoxDev B = boxes[np.src], C = boxes[np.tgt];
    const int64_t nC = C.p1 - C.p0, j1 = min((int64_t)w.s0 + S2T_SRC, B.p1 - B.p0);
    const int64_t ii = w.ii;
    const cd *K = coef8 + np.coef0 * 8 + ii;
    cd A = mkd(0.0), Bv = mkd(0.0), Cv = mkd(0.0);
#pragma unroll 4
    for (int64_t jj = w.s0; jj < j1; ++jj) {
        const cd *k = K + jj * 8 * nC;
        const int64_t sj = B.p0 + jj;
        const cd a = qh[3 * sj], b = qh[3 * sj + 1], c = qh[3 * sj + 2];
        const cd k0 = k[0], k1 = k[nC], k2 = k[2 * nC], k3 = k[3 * nC], k4 = k[4 * nC], k5 = k[5 * nC],
                 k6 = k[6 * nC], k7 = k[7 * nC];
        A += k0 * a + k6 * b + k2 * c;
        Bv += k0 * b + k7 * a + k3 * c;
        Cv += k1 * c + k5 * a + k4 * b;
    }
    const int64_t ti = C.p0 + ii;
    atomicAdd(&ph[3 * ti].x, A.x);
    atomicAdd(&ph[3 * ti].y, A.y);
    atomicAdd(&ph[3 * ti + 1].x, Bv.x);
    atomicAdd(&ph[3 * ti + 1].y, Bv.y);
    atomicAdd(&ph[3 * ti + 2].x, Cv.x);
    atomicAdd(&ph[3 * ti + 2].y, Cv.y);
}

// Transpose of k_s2t_apply8: qh_bar(j) += K(i, j)^T ph_bar(i) over the targets i
// of each near pair, K the 3 x 3 helical block of the pair (i, j) with rows
// (A, B, C) = [[k0, k6, k2], [k7, k0, k3], [k5, k4, k1]] in (a, b, c).  One
// warp per (near pair, source j): lanes take the targets (coalesced reads of
// the coefficient rows), a shuffle reduction sums them.
__global__ void __launch_bounds__(256) k_s2t_apply8_tr(int64_t nrow, const S2TRowT *rows, const NearPair *near,
                                                       const BoxDev *boxes, const cd *coef8, const cd *phb,
                                                       cd *qhb)
{
    const int64_t wi = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wi >= nrow) return;
    const S2TRowT w = rows[wi];
    const NearPair np = near[w.pair];
    const BoxDev B = boxes[np.src], C = boxes[np.tgt];
    const int64_t nC = C.p1 - C.p0;
    const cd *K = coef8 + np.coef0 * 8 + (int64_t)w.jj * 8 * nC;
    cd a = mkd(0.0), b = mkd(0.0), c = mkd(0.0);
    for (int64_t ii = lane; ii < nC; ii += 32) {
        const cd *pi = phb + 3 * (C.p0 + ii);
        const cd A = pi[0], Bv = pi[1], Cv = pi[2];
        const cd k0 = K[ii], k1 = K[nC + ii], k2 = K[2 * nC + ii], k3 = K[3 * nC + ii], k4 = K[4 * nC + ii],
                 k5 = K[5 * nC + ii], k6 = K[6 * nC + ii], k7 = K[7 * nC + ii];
        a += k0 * A + k7 * Bv + k5 * Cv;
        b += k6 * A + k0 * Bv + k4 * Cv;
        c += k2 * A + k3 * Bv + k1 * Cv;
    }
    double v[6] = {a.x, a.y, b.x, b.y, c.x, c.y};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int u = 0; u < 6; ++u) v[u] += __shfl_xor_sync(0xffffffffu, v[u], o);
    if (lane == 0) {
        double *q = (double *)(qhb + 3 * (B.p0 + w.jj));
#pragma unroll
        for (int u = 0; u < 6; ++u) atomicAdd(q + u, v[u]);
    }
}

void launch_s2t_apply8_tr(int64_t nrow, const S2TRowT *rows, const NearPair *near, const BoxDev *boxes,
                          const cd *coef8, const cd *phb, cd *qhb, cudaStream_t st)
{
    if (nrow <= 0) return;
    k_s2t_apply8_tr<<<(unsigned)((nrow * 32 + 255) / 256), 256, 0, st>>>(nrow, rows, near, boxes, coef8, phb, qhb);
}

// Free-space near field (Section 2, eq. GEandGH): ph(i) += T G_E^f(r_i - r_j)
// T^{-1} qh(j) over the sources j != i of the near leaf pairs of the target's
// layer, G_E^f = g (a I + b R^ R^T), g = e^{ikR} / (4 pi R),
// a = 1 + (ik/R - 1/R^2)/k^2, b = (3/R^2 - 3ik/R - k^2)/k^2, T the helical map
// (A, B, C) = (x + iy, x - iy, z).  One warp per (near pair, row point): lanes
// take the column points, a shuffle reduction sums them.  transposed: rows are
// the pair's sources and the maps are T^T in, T^{-T} out (G_E^f is symmetric
// and even in R), which is the transpose of the forward sum.
__global__ void __launch_bounds__(256) k_p2p_free(int64_t nrow, const S2TRowT *rows, const int64_t *pairs,
                                                  const BoxDev *boxes, const double *xyz, MediumDev M,
                                                  const cd *in, cd *out, int transposed)
{
    const int64_t wi = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wi >= nrow) return;
    const S2TRowT w = rows[wi];
    const BoxDev Bs = boxes[pairs[2 * w.pair]], Bt = boxes[pairs[2 * w.pair + 1]];
    // forward: row = target (in Bt), columns = sources (Bs); transposed: the reverse
    const BoxDev Br = transposed ? Bs : Bt, Bc = transposed ? Bt : Bs;
    const int64_t ir = Br.p0 + w.jj;
    const cd k = M.k[Br.layer];
    const cd ik2 = inv(k * k);
    const double xr = xyz[3 * ir], yr = xyz[3 * ir + 1], zr = xyz[3 * ir + 2];
    cd vx = mkd(0.0), vy = mkd(0.0), vz = mkd(0.0);
    for (int64_t jc = Bc.p0 + lane; jc < Bc.p1; jc += 32) {
        if (jc == ir) continue;
        const double Rx = xr - xyz[3 * jc], Ry = yr - xyz[3 * jc + 1], Rz = zr - xyz[3 * jc + 2];
        const double R2 = Rx * Rx + Ry * Ry + Rz * Rz, R = sqrt(R2), iR = 1.0 / R;
        const cd g = (0.25 / LMF_PI * iR) * cexpd(mul_i(R * k));
        const cd ikR = mul_i(k * iR);
        const cd a = mkd(1.0) + ik2 * (ikR - mkd(iR * iR));
        const cd b = ik2 * (mkd(3.0 * iR * iR) - 3.0 * ikR - k * k);
        const cd *q = in + 3 * jc;
        cd jx, jy, jz;   // Cartesian input
        if (!transposed) {
            jx = 0.5 * (q[0] + q[1]);
            jy = mul_mi(0.5 * (q[0] - q[1]));
        } else {
            jx = q[0] + q[1];
            jy = mul_i(q[0] - q[1]);
        }
        jz = q[2];
        const cd rj = (iR * iR) * (Rx * jx + Ry * jy + Rz * jz);
        vx += g * (a * jx + b * (Rx * rj));
        vy += g * (a * jy + b * (Ry * rj));
        vz += g * (a * jz + b * (Rz * rj));
    }
    double v[6] = {vx.x, vx.y, vy.x, vy.y, vz.x, vz.y};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int u = 0; u < 6; ++u) v[u] += __shfl_xor_sync(0xffffffffu, v[u], o);
    if (lane == 0) {
        const cd X{v[0], v[1]}, Y{v[2], v[3]};
        cd o0, o1;
        if (!transposed) {
            o0 = X + mul_i(Y);
            o1 = X - mul_i(Y);
        } else {
            o0 = 0.5 * (X - mul_i(Y));
            o1 = 0.5 * (X + mul_i(Y));
        }
        double *op = (double *)(out + 3 * ir);
        atomicAdd(op, o0.x);
        atomicAdd(op + 1, o0.y);
        atomicAdd(op + 2, o1.x);
        atomicAdd(op + 3, o1.y);
        atomicAdd(op + 4, v[4]);
        atomicAdd(op + 5, v[5]);
    }
}

void launch_p2p_free(int64_t nrow, const S2TRowT *rows, const int64_t *pairs, const BoxDev *boxes,
                     const double *xyz, const MediumDev &M, const cd *in, cd *out, bool transposed, cudaStream_t st)
{
    if (nrow <= 0) return;
    k_p2p_free<<<(unsigned)((nrow * 32 + 255) / 256), 256, 0, st>>>(nrow, rows, pairs, boxes, xyz, M, in, out,
                                                                     transposed ? 1 : 0);
}

void launch_s2t_combine(int64_t nnear, const NearPair *near, const BoxDev *boxes, const double *xyz,
                        const cd *coef5, cd *coef8, cudaStream_t st)
{
    if (nnear <= 0) return;
    k_s2t_combine<<<(unsigned)nnear, 128, 0, st>>>(near, boxes, xyz, coef5, coef8);
}

void launch_s2t_apply8(int64_t nrow, const S2TRow *rows, const NearPair *near, const BoxDev *boxes,
                       const cd *coef8, const cd *qh, cd *phih, cudaStream_t st)
{
    if (nrow <= 0) return;
    k_s2t_apply8<<<(unsigned)((nrow + 255) / 256), 256, 0, st>>>(nrow, rows, near, boxes, coef8, qh, phih);
}

void launch_s2t_apply(int64_t nnear, const NearPair *near, const BoxDev *boxes,
                      const double *xyz, const cd *coef, const cd *qh, cd *phih,
                      cudaStream_t st)
{
    if (nnear <= 0) return;
    k_s2t_apply<<<(unsigned)nnear, 64, 0, st>>>(near, boxes, xyz, coef, qh, phih);
}

}  // namespace lmf

namespace lmf {
cudaError_t configure_fmm_kernels()
{
    const int big = (int)LEAF_SMEM_CAP;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_p2m<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_p2m<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_l2p<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_l2p<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    const int mx = (int)cudaSharedmemCarveoutMaxShared;
    if ((e = cudaFuncSetAttribute(k_p2m<float>, cudaFuncAttributePreferredSharedMemoryCarveout, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_p2m<double>, cudaFuncAttributePreferredSharedMemoryCarveout, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_l2p<float>, cudaFuncAttributePreferredSharedMemoryCarveout, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_l2p<double>, cudaFuncAttributePreferredSharedMemoryCarveout, mx))) return e;
    return configure_trans_kernels();
}
}  // namespace lmf
