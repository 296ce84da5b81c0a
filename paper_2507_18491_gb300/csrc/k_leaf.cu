// L2P of the mixed form (FP32 expansions), one code path per truncation p.
//
// Basis (Section 3.3, eqs. mecoeff and maxwell_LE_layered): for a point at r
// relative to its leaf centre,
//   b_nm(r) = scale j_n(k |r|) Y_n^m(r^) / s^n,   Y_n^m = P^_n^|m| e^{i m phi}
// (times (-1)^m for m < 0), s = |k| S_leaf; P2M takes conj(Y) and scale 4 pi,
// L2P takes Y and scale 1 (the transposes swap the two).
//
// k_l2p_pt is organised so that no barrier separates the phases of a point and
// leaves of any size fill the machine (the leaves of a clustered point set hold
// from one to several hundred points): one thread per point over the whole
// sorted point set; the thread walks the orders m and, for each, the Legendre
// recurrence in n, contracting the basis with its leaf's three local
// expansions as it goes (the expansions are read through L1: the threads of a
// warp mostly share a leaf).
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
    cudaError_t e;
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

cudaError_t configure_leaf_fast() { return configure_leaf_kernels(); }

}  // namespace lmf
