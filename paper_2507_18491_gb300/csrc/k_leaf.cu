// P2M and L2P of the mixed form (FP32 expansions), one code path per truncation p.
//
// Basis (Section 3.3, eqs. mecoeff and maxwell_LE_layered): for a point at r
// relative to its leaf centre,
//   b_nm(r) = scale j_n(k |r|) Y_n^m(r^) / s^n,   Y_n^m = P^_n^|m| e^{i m phi}
// (times (-1)^m for m < 0), s = |k| S_leaf; P2M takes conj(Y) and scale 4 pi,
// L2P takes Y and scale 1 (the transposes swap the two).
//
// Both kernels keep every SM busy whatever the leaf sizes (the leaves of a
// clustered point set hold from one to several hundred points) and put no
// barrier between the phases of a point:
//   k_l2p_pt  one thread per point over the whole sorted point set; the thread
//             walks the orders m and, for each, the Legendre recurrence in n,
//             contracting the basis with its leaf's three local expansions as
//             it goes (read through L1: the threads of a warp mostly share a leaf);
//   k_p2m_ms  one warp per unit of at most 128 points of one leaf (units largest
//             first); each lane keeps the coefficients of its own pair of orders
//             in registers over a stream of points (see the kernel).
// The recurrence coefficients live in constant memory and every loop over
// (n, m) is unrolled for the compile-time p, so they are immediate operands.
#include <cmath>

#include "kernels.cuh"
#include "specfun.cuh"

namespace lmf {

namespace {

constexpr int LF_PMAX = 15;      // fast path for p <= LF_PMAX
constexpr int LF_SER = 14;       // terms of the power series of j_n
constexpr int LF_NT = (LF_PMAX + 1) * (LF_PMAX + 2) / 2;

// P^_n^m recurrences (orthonormal, Condon-Shortley):
//   P_m^m = -c_m s P_{m-1}^m-1 (P_0^0 = 1/sqrt(4 pi)), P_{m+1}^m = d_m x P_m^m,
//   P_n^m = a_nm (x P_{n-1}^m - b_nm P_{n-2}^m), n >= m + 2  (index n(n+1)/2 + m);
// series of j_n: ratio of consecutive terms -z^2/2 / (k (2n + 2k + 1)), leading 1/(2n+1)!!
__constant__ float c_la[LF_NT], c_lb[LF_NT], c_ld[LF_PMAX + 1], c_lc[LF_PMAX + 1];
__constant__ float c_sk[(LF_PMAX + 1) * LF_SER], c_idf[LF_PMAX + 1];
// the same recurrence per (step t = n - m, order m), for lanes that each run
// their own order: [t][m] = (a, b) with P_{m+t}^m = a (x P_{m+t-1}^m - b P_{m+t-2}^m)
// (t = 1: a = d_m, b = 0), read through L1
__device__ float2 g_lab[(LF_PMAX + 1) * (LF_PMAX + 1)];

}  // namespace

cudaError_t configure_leaf_kernels()
{
    float la[LF_NT], lb[LF_NT], ld[LF_PMAX + 1], lc[LF_PMAX + 1], sk[(LF_PMAX + 1) * LF_SER], idf[LF_PMAX + 1];
    for (int n = 0; n <= LF_PMAX; ++n)
        for (int m = 0; m <= n; ++m) {
            const int e = n * (n + 1) / 2 + m;
            la[e] = lb[e] = 0.f;
            if (n >= m + 2) {
                la[e] = (float)std::sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
                lb[e] = (float)std::sqrt(((n - 1.0) * (n - 1.0) - (double)m * m) / (4.0 * (n - 1.0) * (n - 1.0) - 1.0));
            }
        }
    double df = 1.0;
    for (int m = 0; m <= LF_PMAX; ++m) {
        ld[m] = (float)std::sqrt(2.0 * m + 3.0);
        lc[m] = m == 0 ? 0.28209479177387814347f : (float)std::sqrt((2.0 * m + 1.0) / (2.0 * m));
        if (m > 0) df *= 2.0 * m + 1.0;
        idf[m] = (float)(1.0 / df);
        for (int k = 1; k <= LF_SER; ++k) sk[m * LF_SER + k - 1] = (float)(1.0 / (k * (2.0 * m + 2.0 * k + 1.0)));
    }
    float2 lab[(LF_PMAX + 1) * (LF_PMAX + 1)];
    for (int t = 0; t <= LF_PMAX; ++t)
        for (int m = 0; m <= LF_PMAX; ++m) {
            const int n = m + t;
            float2 v{0.f, 0.f};
            if (t == 1 && n <= LF_PMAX) v = float2{ld[m], 0.f};
            else if (t >= 2 && n <= LF_PMAX) v = float2{la[n * (n + 1) / 2 + m], lb[n * (n + 1) / 2 + m]};
            lab[t * (LF_PMAX + 1) + m] = v;
        }
    cudaError_t e;
    if ((e = cudaMemcpyToSymbol(g_lab, lab, sizeof(lab))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_la, la, sizeof(la))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_lb, lb, sizeof(lb))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_ld, ld, sizeof(ld))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_lc, lc, sizeof(lc))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_sk, sk, sizeof(sk))) != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_idf, idf, sizeof(idf));
}

bool leaf_fast_supported(int p) { return p >= 1 && p <= LF_PMAX; }

namespace {

// Seeds of one point: x = cos theta, sv = sin theta, e1 = e^{i phi} (conjugated
// for P2M's basis) and the radial factors jr[n] = scale j_n(k r) / s^n.  The
// power series runs in FP32 when |k r| < 1.5 (scaled by zeta = k r / s so that
// no power of k r under- or overflows); otherwise the FP64 Miller recurrence.
template <int PP>
__device__ __forceinline__ void leaf_seed(cd k, double dx, double dy, double dz, bool conjugate, double scale,
                                          double inv_s, float &x, float &sv, cf &e1, cf (&jr)[PP + 1])
{
    const float fx = (float)dx, fy = (float)dy, fz = (float)dz;
    const float rxy = sqrtf(fx * fx + fy * fy), r = sqrtf(fx * fx + fy * fy + fz * fz);
    const cf kf{(float)k.x, (float)k.y};
    const cf kr = r * kf;
    if (abs2(kr) < 2.25f) {
        x = r > 0.f ? fz / r : 1.f;
        sv = r > 0.f ? rxy / r : 0.f;
        e1 = rxy > 0.f ? cf{fx / rxy, (conjugate ? -fy : fy) / rxy} : cf{1.f, 0.f};
        const cf q = -0.5f * (kr * kr);
        const cf zeta = (r * (float)inv_s) * kf;
        cf zn{(float)scale, 0.f};
#pragma unroll
        for (int n = 0; n <= PP; ++n) {
            cf term{1.f, 0.f}, sum{1.f, 0.f};
            for (int kk = 1; kk <= LF_SER; ++kk) {
                term = term * q * c_sk[n * LF_SER + kk - 1];
                sum += term;
                if (abs2(term) < 1e-18f * abs2(sum)) break;
            }
            jr[n] = (zn * sum) * c_idf[n];
            zn = zn * zeta;
        }
        return;
    }
    const double rd = sqrt(dx * dx + dy * dy + dz * dz), rxyd = sqrt(dx * dx + dy * dy);
    x = (float)(rd > 0 ? dz / rd : 1.0);
    sv = (float)(rd > 0 ? rxyd / rd : 0.0);
    e1 = rxyd > 0 ? cf{(float)(dx / rxyd), (float)((conjugate ? -dy : dy) / rxyd)} : cf{1.f, 0.f};
    cd jd[PP + 1];
    sph_bessel_seq(k * rd, PP, jd);
    double sp = scale;
#pragma unroll
    for (int n = 0; n <= PP; ++n) {
        jr[n] = cf{(float)(sp * jd[n].x), (float)(sp * jd[n].y)};
        sp *= inv_s;
    }
}

// L2P (or the transpose of P2M): Phi_h(point) = sum_nm L[v][nm] b_nm(point)
// for the helical components v = 0, 1, 2.  One thread per sorted point.
template <int PP>
__global__ void __launch_bounds__(128) k_l2p_pt(int64_t N, const int *pt_box, const BoxDev *boxes,
                                                const double *xyz, const cf *le, MediumDev M, LayerScale ls,
                                                cd *ph, int conj_basis, double scale, int accumulate)
{
    constexpr int P = (PP + 1) * (PP + 1);
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= N) return;
    const int bi = pt_box[t];
    const BoxDev b = boxes[bi];
    float x, sv;
    cf e1, jr[PP + 1];
    leaf_seed<PP>(M.k[b.layer], xyz[3 * t] - b.c[0], xyz[3 * t + 1] - b.c[1], xyz[3 * t + 2] - b.c[2],
                  conj_basis != 0, scale, 1.0 / ls.s[b.layer], x, sv, e1, jr);
    const cf *L0 = le + (int64_t)bi * 3 * P, *L1 = L0 + P, *L2 = L1 + P;
    cf A{0.f, 0.f}, B{0.f, 0.f}, C{0.f, 0.f};
    float pmm = c_lc[0];
    cf em{1.f, 0.f};
#pragma unroll
    for (int m = 0; m <= PP; ++m) {
        if (m > 0) {
            pmm = -pmm * sv * c_lc[m];
            em = em * e1;
        }
        const cf emc = (m & 1) ? cf{-em.x, em.y} : cf{em.x, -em.y};   // (-1)^m conj(e^{i m phi})
        float p0 = 0.f, p1 = 0.f;
#pragma unroll
        for (int n = m; n <= PP; ++n) {
            float pl;
            if (n == m) pl = pmm;
            else if (n == m + 1) pl = c_ld[m] * x * pmm;
            else pl = c_la[n * (n + 1) / 2 + m] * (x * p1 - c_lb[n * (n + 1) / 2 + m] * p0);
            p0 = p1;
            p1 = pl;
            const cf jv = pl * jr[n];
            const cf bp = jv * em;
            const int ip = n * n + n + m;
            A += L0[ip] * bp;
            B += L1[ip] * bp;
            C += L2[ip] * bp;
            if (m > 0) {
                const cf bm = jv * emc;
                const int im = n * n + n - m;
                A += L0[im] * bm;
                B += L1[im] * bm;
                C += L2[im] * bm;
            }
        }
    }
    cd o0{(double)A.x, (double)A.y}, o1{(double)B.x, (double)B.y}, o2{(double)C.x, (double)C.y};
    if (accumulate) {
        o0 += ph[3 * t];
        o1 += ph[3 * t + 1];
        o2 += ph[3 * t + 2];
    }
    ph[3 * t] = o0;
    ph[3 * t + 1] = o1;
    ph[3 * t + 2] = o2;
}

}  // namespace

namespace {

// P2M (or the transpose of L2P): M[v][nm] = sum_j q_j[v] b_nm(r_j) over the
// points of one unit (at most 128 points of one leaf), one warp per unit.
// Lane = 16 s + 8 h + j: stream s takes the points s, s + 2, ...; h is the sign
// of the order and {j, p - j} the lane's pair of orders, whose p + 2
// coefficients (two runs of the Legendre recurrence in n) times the three
// helical components stay in registers until the unit ends: no reduction over
// points until then.  The warp first forms the seeds of 32 points at a time
// (lane = point) in shared memory: cos theta, P^_m^m, e^{-i m phi} (or
// e^{i m phi}), the radial factors and the charges.
template <int PP>
struct P2mSeeds {
    static constexpr int W = 33;    // rows padded: lanes of one point reading different rows hit different banks
    float x[W], pm[PP + 1][W];
    cf jr[PP + 1][W], em[PP + 1][W], q[3][W];
};

template <int PP>
__global__ void __launch_bounds__(32, 12) k_p2m_ms(const LeafUnit *units, const BoxDev *boxes, const double *xyz,
                                                   const cd *qh, MediumDev M, LayerScale ls, cf *me, int conj_basis,
                                                   double scale)
{
    constexpr int P = (PP + 1) * (PP + 1), NS = PP + 2;
    __shared__ P2mSeeds<PP> sd;
    const LeafUnit u = units[blockIdx.x];
    const BoxDev b = boxes[u.box];
    const cd k = M.k[b.layer];
    const double inv_s = 1.0 / ls.s[b.layer];
    const int lane = threadIdx.x, st = lane >> 4, hs = (lane >> 3) & 1, j = lane & 7;
    const bool live = j <= PP / 2;
    const int m1 = live ? j : 0, m2 = live ? PP - j : PP;   // idle lanes keep in-range orders
    const bool run1 = live && !(hs == 1 && m1 == 0);       // +-m1 (no -0)
    const bool run2 = live && m2 != m1;
    const int seg1 = PP - m1 + 1;                           // steps of the first run
    cf acc[NS][3];
#pragma unroll
    for (int t = 0; t < NS; ++t)
#pragma unroll
        for (int v = 0; v < 3; ++v) acc[t][v] = cf{0.f, 0.f};
    for (int64_t c0 = u.i0; c0 < u.i1; c0 += 32) {
        const int np = (int)min((int64_t)32, u.i1 - c0);
        __syncwarp();
        if (lane < np) {
            const int64_t i = c0 + lane;
            float x, sv;
            cf e1, jr[PP + 1];
            leaf_seed<PP>(k, xyz[3 * i] - b.c[0], xyz[3 * i + 1] - b.c[1], xyz[3 * i + 2] - b.c[2], conj_basis != 0,
                          scale, inv_s, x, sv, e1, jr);
            sd.x[lane] = x;
            float pmm = c_lc[0];
            cf em{1.f, 0.f};
#pragma unroll
            for (int m = 0; m <= PP; ++m) {
                if (m > 0) {
                    pmm = -pmm * sv * c_lc[m];
                    em = em * e1;
                }
                sd.pm[m][lane] = pmm;
                sd.em[m][lane] = em;
                sd.jr[m][lane] = jr[m];
            }
#pragma unroll
            for (int v = 0; v < 3; ++v) sd.q[v][lane] = cf{(float)qh[3 * i + v].x, (float)qh[3 * i + v].y};
        }
        __syncwarp();
        for (int pj = st; pj < np; pj += 2) {
            const float x = sd.x[pj];
            const cf q0 = sd.q[0][pj], q1 = sd.q[1][pj], q2 = sd.q[2][pj];
            // azimuthal factor of a run: e^{i m phi}, or (-1)^m conj of it for -m
            auto fac = [&](int m) {
                const cf e = sd.em[m][pj];
                return hs == 0 ? e : ((m & 1) ? cf{-e.x, e.y} : cf{e.x, -e.y});
            };
            cf f = fac(m1);
            float p0 = 0.f, p1 = 0.f;
#pragma unroll
            for (int t = 0; t < NS; ++t) {
                const bool first = t < seg1;
                const int m = first ? m1 : m2;
                const int tn = first ? t : t - seg1;   // step within the run, n = m + tn
                if (t == seg1) {
                    f = fac(m2);
                    p0 = p1 = 0.f;
                }
                float pl;
                if (tn == 0) {
                    pl = sd.pm[m][pj];
                } else {
                    const float2 ab = __ldg(&g_lab[tn * (LF_PMAX + 1) + m]);
                    pl = ab.x * (x * p1 - ab.y * p0);
                }
                p0 = p1;
                p1 = pl;
                if (first ? run1 : run2) {
                    const cf bv = (pl * sd.jr[m + tn][pj]) * f;
                    acc[t][0] += q0 * bv;
                    acc[t][1] += q1 * bv;
                    acc[t][2] += q2 * bv;
                }
            }
        }
    }
    // the two streams hold the same coefficients: add them, then stream 0 writes
#pragma unroll
    for (int t = 0; t < NS; ++t)
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            acc[t][v].x += __shfl_xor_sync(0xffffffffu, acc[t][v].x, 16);
            acc[t][v].y += __shfl_xor_sync(0xffffffffu, acc[t][v].y, 16);
        }
    if (st != 0) return;
    cf *out = me + (int64_t)u.box * 3 * P;
#pragma unroll
    for (int t = 0; t < NS; ++t) {
        const bool first = t < seg1;
        const int m = first ? m1 : m2;
        const int n = m + (first ? t : t - seg1);
        if (!(first ? run1 : run2)) continue;
        const int idx = n * n + n + (hs ? -m : m);
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            if (u.whole) {
                out[v * P + idx] = acc[t][v];
            } else {
                atomicAdd(&out[v * P + idx].x, acc[t][v].x);
                atomicAdd(&out[v * P + idx].y, acc[t][v].y);
            }
        }
    }
}

template <int PP>
void launch_p2m_pp(int64_t nunit, const LeafUnit *units, const BoxDev *boxes, const double *xyz, const cd *qh,
                   const MediumDev &M, const LayerScale &ls, cf *me, bool conj_basis, double scale, cudaStream_t st)
{
    if (nunit <= 0) return;
    k_p2m_ms<PP><<<(unsigned)nunit, 32, 0, st>>>(units, boxes, xyz, qh, M, ls, me, conj_basis ? 1 : 0, scale);
}

template <int PP>
void launch_l2p_pp(int64_t N, const int *pt_box, const BoxDev *boxes, const double *xyz, const cf *le,
                   const MediumDev &M, const LayerScale &ls, cd *ph, bool conj_basis, double scale, bool accumulate,
                   cudaStream_t st)
{
    if (N <= 0) return;
    k_l2p_pt<PP><<<(unsigned)((N + 127) / 128), 128, 0, st>>>(N, pt_box, boxes, xyz, le, M, ls, ph, conj_basis ? 1 : 0,
                                                              scale, accumulate ? 1 : 0);
}

}  // namespace

#define LF_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15)

void launch_l2p_fast(int p, int64_t N, const int *pt_box, const BoxDev *boxes, const double *xyz, const cf *le,
                     const MediumDev &M, const LayerScale &ls, cd *ph, bool conj_basis, double scale, bool accumulate,
                     cudaStream_t st)
{
    switch (p) {
#define LF_CASE(v)                                                                                           \
    case v:                                                                                                  \
        launch_l2p_pp<v>(N, pt_box, boxes, xyz, le, M, ls, ph, conj_basis, scale, accumulate, st);           \
        break;
        LF_CASES(LF_CASE)
#undef LF_CASE
    default: break;
    }
}

void launch_p2m_fast(int p, int64_t nunit, const LeafUnit *units, const BoxDev *boxes, const double *xyz,
                     const cd *qh, const MediumDev &M, const LayerScale &ls, cf *me, bool conj_basis, double scale,
                     cudaStream_t st)
{
    switch (p) {
#define LF_CASE(v)                                                                                           \
    case v:                                                                                                  \
        launch_p2m_pp<v>(nunit, units, boxes, xyz, qh, M, ls, me, conj_basis, scale, st);                    \
        break;
        LF_CASES(LF_CASE)
#undef LF_CASE
    default: break;
    }
}

cudaError_t configure_leaf_fast() { return configure_leaf_kernels(); }

}  // namespace lmf
