// Position gradient of the FMM operator (FP64 form): for a scalar objective
// whose gradient with respect to the field is g = dL/dconj(E) (the usual
// conjugate-Wirtinger seed), the gradient with respect to a point's
// coordinates is Re sum conj(g) dE/dr.  With nu = S^T conj(g) (the helical
// seed of the transposed pass) it splits into
//   target part: nu_v(i) . grad of the local expansion at r_i (L2P's functions),
//   source part: q_v(j)  . grad of P2M's functions at r_j contracted with the
//                multipole expansions of the transposed pass (ME_bar),
//   near part:   nu(i)^T (dK(r_i, r_j)/dr) q(j) over the near point pairs,
// with q the helical charges of the forward pass (checkpointed).
//
// Gradients of the regular solid harmonics R_n^m = j_n(k r) Y_n^m(r^)
// (orthonormal, Condon-Shortley), with D+- = d/dx +- i d/dy:
//   d/dz R_n^m = k (a-_{nm} R_{n-1}^m - a+_{nm} R_{n+1}^m),
//   D+ R_n^m   = k (b+_{nm} R_{n+1}^{m+1} + b-_{nm} R_{n-1}^{m+1}),
//   D- R_n^m   = -k (c+_{nm} R_{n+1}^{m-1} + c-_{nm} R_{n-1}^{m-1}),
//   a+ = sqrt(((n+1)^2 - m^2) / ((2n+1)(2n+3))),  a- = sqrt((n^2 - m^2) / ((2n-1)(2n+1))),
//   b+ = sqrt((n+m+1)(n+m+2) / ((2n+1)(2n+3))),    b- = sqrt((n-m)(n-m-1) / ((2n-1)(2n+1))),
//   c+ = sqrt((n-m+1)(n-m+2) / ((2n+1)(2n+3))),    c- = sqrt((n+m)(n+m-1) / ((2n-1)(2n+1))),
// from the plane-wave form of R_n^m and the expansions of cos(theta) Y and
// sin(theta) e^{+-i phi} Y in harmonics of degree n +- 1.
//
// Near field: with F_kappa = e^{i kappa phi} int w Z sigma J_kappa(k_rho rho)
// (phi, rho of r_j - r_i), D+ F_kappa = -e^{i(kappa+1)phi} int w Z sigma k_rho J_{kappa+1}
// and D- F_kappa = e^{i(kappa-1)phi} int w Z sigma k_rho J_{kappa-1}, so
//   d/dx F = e^{i(kappa-1)phi} Q_{kappa-1} - e^{i(kappa+1)phi} Q_{kappa+1},
//   d/dy F = i (e^{i(kappa-1)phi} Q_{kappa-1} + e^{i(kappa+1)phi} Q_{kappa+1}),
// Q_m = int w Z sigma (k_rho / 2) J_m, and the heights enter through
// Z = e^{i s (k_z z_s - k'_z z_t)}: d/dz_s -> i s k_z, d/dz_t -> -i s k'_z.
#include "kernels.cuh"
#include "quad.cuh"
#include "specfun.cuh"

namespace lmf {

namespace {

__device__ inline double dsq(double x) { return sqrt(fmax(x, 0.0)); }

// R_n^m for 0 <= n <= N, -n <= m <= n at r (complex k), into R[n^2 + n + m]
__device__ inline void solid_harmonics(int N, cd k, double x, double y, double z, cd *R)
{
    const double r = sqrt(x * x + y * y + z * z), rxy = sqrt(x * x + y * y);
    const double ct = r > 0 ? z / r : 1.0, st = r > 0 ? rxy / r : 0.0;
    const cd e1 = rxy > 0 ? cd{x / rxy, y / rxy} : cd{1.0, 0.0};
    cd jn[LMF_PMAX + 2];
    sph_bessel_seq(k * r, N, jn);
    double P[(LMF_PMAX + 2) * (LMF_PMAX + 3) / 2];
    legendre_norm<double>(N, ct, st, P);
    cd em = mkd(1.0);
    for (int m = 0; m <= N; ++m) {
        const double sg = (m & 1) ? -1.0 : 1.0;
        for (int n = m; n <= N; ++n) {
            const cd v = (P[n * (n + 1) / 2 + m] * jn[n]) * em;
            R[n * n + n + m] = v;
            if (m > 0) R[n * n + n - m] = sg * ((P[n * (n + 1) / 2 + m] * jn[n]) * conj(em));   // Y_n^-m = (-1)^m conj Y_n^m
        }
        em = em * e1;
    }
}

// (d/dz, D+, D-) of R_n^m from the table R (degree up to n + 1)
__device__ inline void grad_solid(const cd *R, cd k, int n, int m, cd &dz, cd &dp, cd &dm)
{
    auto at = [&](int nn, int mm) { return (nn < 0 || mm > nn || mm < -nn) ? mkd(0.0) : R[nn * nn + nn + mm]; };
    const double ap = dsq(((n + 1.0) * (n + 1.0) - (double)m * m) / ((2.0 * n + 1) * (2.0 * n + 3)));
    const double am = n > 0 ? dsq(((double)n * n - (double)m * m) / ((2.0 * n - 1) * (2.0 * n + 1))) : 0.0;
    const double bp = dsq((n + m + 1.0) * (n + m + 2.0) / ((2.0 * n + 1) * (2.0 * n + 3)));
    const double bm = n > 0 ? dsq((n - m + 0.0) * (n - m - 1.0) / ((2.0 * n - 1) * (2.0 * n + 1))) : 0.0;
    const double cp = dsq((n - m + 1.0) * (n - m + 2.0) / ((2.0 * n + 1) * (2.0 * n + 3)));
    const double cm = n > 0 ? dsq((n + m + 0.0) * (n + m - 1.0) / ((2.0 * n - 1) * (2.0 * n + 1))) : 0.0;
    dz = k * (am * at(n - 1, m) - ap * at(n + 1, m));
    dp = k * (bp * at(n + 1, m + 1) + bm * at(n - 1, m + 1));
    dm = -1.0 * (k * (cp * at(n + 1, m - 1) + cm * at(n - 1, m - 1)));
}

}  // namespace

// One thread per point (sorted order) of the leaves: target part with the
// checkpointed local expansions le, source part with the transposed pass's
// multipole expansions meb; grad (caller order, [N][3] real) accumulated.
__global__ void k_grad_leaf(int p, int64_t nleaf, const int64_t *leaves, const BoxDev *boxes, const double *xyz,
                            const int64_t *perm, const cd *le, const cd *meb, const cd *qh, const cd *nu,
                            MediumDev M, LayerScale ls, double *grad)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // the leaf of point t: binary search over the leaves' point ranges
    int64_t lo = 0, hi = nleaf - 1;
    if (hi < 0) return;
    const int64_t Nend = boxes[leaves[hi]].p1;
    if (t >= Nend) return;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (boxes[leaves[mid]].p0 <= t) lo = mid;
        else hi = mid - 1;
    }
    const int64_t bi = leaves[lo];
    const BoxDev b = boxes[bi];
    if (t < b.p0 || t >= b.p1) return;
    const int P = (p + 1) * (p + 1);
    const cd k = M.k[b.layer];
    const double inv_s = 1.0 / ls.s[b.layer];
    cd R[(LMF_PMAX + 2) * (LMF_PMAX + 2)];
    solid_harmonics(p + 1, k, xyz[3 * t] - b.c[0], xyz[3 * t + 1] - b.c[1], xyz[3 * t + 2] - b.c[2], R);
    const cd n0 = nu[3 * t], n1 = nu[3 * t + 1], n2 = nu[3 * t + 2];
    const cd q0 = qh[3 * t], q1 = qh[3 * t + 1], q2 = qh[3 * t + 2];
    const cd *L = le + bi * 3 * P, *Mb = meb + bi * 3 * P;
    cd gz = mkd(0.0), gp = mkd(0.0), gm = mkd(0.0);
    double sn = 1.0;   // s^-n
    for (int n = 0; n <= p; ++n) {
        for (int m = -n; m <= n; ++m) {
            const int e = n * n + n + m;
            // target: L2P functions R_n^m s^-n; source: P2M functions 4 pi (-1)^m R_n^-m s^-n
            const cd ct = sn * (n0 * L[e] + n1 * L[P + e] + n2 * L[2 * P + e]);
            const cd cs = (4.0 * LMF_PI * sn * ((m & 1) ? -1.0 : 1.0)) * (q0 * Mb[e] + q1 * Mb[P + e] + q2 * Mb[2 * P + e]);
            cd dz, dp, dm;
            grad_solid(R, k, n, m, dz, dp, dm);
            gz += ct * dz;
            gp += ct * dp;
            gm += ct * dm;
            grad_solid(R, k, n, -m, dz, dp, dm);
            gz += cs * dz;
            gp += cs * dp;
            gm += cs * dm;
        }
        sn *= inv_s;
    }
    // d/dx = (D+ + D-) / 2, d/dy = (D+ - D-) / (2i)
    const cd gx = 0.5 * (gp + gm), gy = mul_mi(0.5 * (gp - gm));
    const int64_t o = perm[t];
    atomicAdd(grad + 3 * o, gx.x);
    atomicAdd(grad + 3 * o + 1, gy.x);
    atomicAdd(grad + 3 * o + 2, gz.x);
}

// Derivative integrals of every near point pair, 20 per pair ([e][t][4], e the
// pair's index within its near pair as in k_s2t_pre, t the table (s1,0) (s5,0)
// (s2,1) (s4,1) (s3,2) of |kappa| = K): Q_{K-1}, Q_{K+1}, the d/dz_s and
// d/dz_t integrals of I_K (see the top of this file).
__global__ void k_s2t_pre_grad(const NearPair *near, const BoxDev *boxes, const double *xyz, MediumDev M,
                               const CompDev *comps, double a, int node_cap, cd *coef)
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
        // one more Bessel order than the matvec's near field (J_3)
        pl = make_plan(a, np.rhomax, np.dzmin, 4, false);
        if (plan_nodes(pl) > node_cap) {
            pl.nmid = 16;
            pl.nray = 0;
        }
    }
    __syncthreads();
    const int Q = plan_nodes(pl);
    cd *cf = coef + np.coef0 * 20;
    for (int64_t e = threadIdx.x; e < npp * 20; e += blockDim.x) cf[e] = mkd(0.0);
    const cd k = M.k[c.l], kpz = M.k[c.lp];
    const int kap[5] = {0, 0, 1, 1, 2};
    __syncthreads();
    for (int q0 = 0; q0 < Q; q0 += CH) {
        const int nq = min(CH, Q - q0);
        if (threadIdx.x < nq) {
            const int q = q0 + threadIdx.x;
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
            const int64_t ii = e / nB, jj = e % nB;
            const int64_t ti = C.p0 + ii, sj = B.p0 + jj;
            const double dx = xyz[3 * sj] - xyz[3 * ti], dy = xyz[3 * sj + 1] - xyz[3 * ti + 1];
            const double rho = sqrt(dx * dx + dy * dy);
            const double zs = comp_src_z(c, xyz[3 * sj + 2]), zt = comp_tgt_z(c, xyz[3 * ti + 2]);
            cd acc[20];
            for (int u = 0; u < 20; ++u) acc[u] = cf[e * 20 + u];
            for (int q = 0; q < nq; ++q) {
                cd J[4];
                const cd z = s_kr[q] * rho;
                if (s_kind[q] != 0) {
                    hankel1_seq(s_kind[q] == 2 ? conj(z) : z, 3, J);
                    for (int u = 0; u < 4; ++u) J[u] = 0.5 * (s_kind[q] == 2 ? conj(J[u]) : J[u]);
                } else {
                    bessel_j_seq<4>(z, 3, J);
                }
                const cd Z = cexpd(mul_i(c.s * (s_kz[q] * zs - s_kzp[q] * zt)));
                const cd wZ = s_w[q] * Z;
                const cd hk = 0.5 * s_kr[q];
                const cd dzs = mul_i(c.s * s_kz[q]), dzt = mul_mi(c.s * s_kzp[q]);
                for (int t = 0; t < 5; ++t) {
                    const int K = kap[t];
                    const cd base = wZ * s_sg[q][t];
                    const cd jm = K == 0 ? -1.0 * J[1] : J[K - 1];
                    acc[4 * t] += (base * hk) * jm;
                    acc[4 * t + 1] += (base * hk) * J[K + 1];
                    acc[4 * t + 2] += (base * dzs) * J[K];
                    acc[4 * t + 3] += (base * dzt) * J[K];
                }
            }
            for (int u = 0; u < 20; ++u) cf[e * 20 + u] = acc[u];
        }
        __syncthreads();
    }
}

namespace {

// (d/dx, d/dy, d/dz_s, d/dz_t) of L_kappa = i^(kappa+1)/(4 pi) e^{i kappa phi} I_kappa
// of one table (stored |kappa| = K quantities d[0..3]) at signed kappa
__device__ inline void dL(int kappa, const cd *d, cd e1, cd &lx, cd &ly, cd &ls, cd &lt)
{
    const int K = kappa < 0 ? -kappa : kappa;
    cd qa = d[0], qb = d[1], zs = d[2], zt = d[3];   // Q_{K-1}, Q_{K+1}, dz_s I_K, dz_t I_K
    cd qlo, qhi;                                     // Q_{kappa-1}, Q_{kappa+1}
    if (kappa >= 0) {
        qlo = qa;
        qhi = qb;
    } else {
        // J_{-n} = (-1)^n J_n: Q_{-K-1} = (-1)^{K+1} Q_{K+1}, Q_{-K+1} = (-1)^{K-1} Q_{K-1}
        qlo = ((K + 1) & 1) ? -1.0 * qb : qb;
        qhi = ((K - 1) & 1) ? -1.0 * qa : qa;
        if (K & 1) {
            zs = -1.0 * zs;
            zt = -1.0 * zt;
        }
    }
    auto ephase = [&](int m) {
        cd e = mkd(1.0);
        const cd b = m < 0 ? conj(e1) : e1;
        for (int i = 0; i < (m < 0 ? -m : m); ++i) e = e * b;
        return e;
    };
    const cd lo = ephase(kappa - 1) * qlo, hi = ephase(kappa + 1) * qhi;
    const cd pre = (1.0 / (4.0 * LMF_PI)) * ipow<double>(kappa + 1);
    lx = pre * (lo - hi);
    ly = pre * mul_i(lo + hi);
    const cd ek = ephase(kappa);
    ls = pre * (ek * zs);
    lt = pre * (ek * zt);
}

}  // namespace

// One thread per near point pair (i target, j source): gradient of
// nu(i)^T K(i, j) q(j) with respect to both points (caller order).
__global__ void k_grad_near(int64_t nnear, const NearPair *near, const BoxDev *boxes, const double *xyz,
                            const int64_t *perm, const CompDev *comps, const cd *coefg, const cd *qh,
                            const cd *nu, double *grad)
{
    const NearPair np = near[blockIdx.x];
    const CompDev c = comps[np.comp];
    const BoxDev B = boxes[np.src], C = boxes[np.tgt];
    const int64_t nB = B.p1 - B.p0, nC = C.p1 - C.p0;
    const cd *G = coefg + np.coef0 * 20;
    const double ss = c.has_src_refl ? -1.0 : 1.0, st = c.has_tgt_refl ? -1.0 : 1.0;
    for (int64_t e = threadIdx.x; e < nB * nC; e += blockDim.x) {
        const int64_t ii = e / nB, jj = e % nB;
        const int64_t ti = C.p0 + ii, sj = B.p0 + jj;
        const double dx = xyz[3 * sj] - xyz[3 * ti], dy = xyz[3 * sj + 1] - xyz[3 * ti + 1];
        const double rho = sqrt(dx * dx + dy * dy);
        const cd e1 = rho > 0 ? cd{dx / rho, dy / rho} : cd{1.0, 0.0};
        const cd *d = G + e * 20;
        // dL for the (table, kappa) pairs of the helical operator
        cd x0[4], x1[4], x2p[4], x2m[4], x3p[4], x3m[4], x4p[4], x4m[4];
        dL(0, d, e1, x0[0], x0[1], x0[2], x0[3]);           // (s1, 0)
        dL(0, d + 4, e1, x1[0], x1[1], x1[2], x1[3]);       // (s5, 0)
        dL(1, d + 8, e1, x2p[0], x2p[1], x2p[2], x2p[3]);   // (s2, +1)
        dL(-1, d + 8, e1, x2m[0], x2m[1], x2m[2], x2m[3]);  // (s2, -1)
        dL(1, d + 12, e1, x3p[0], x3p[1], x3p[2], x3p[3]);  // (s4, +1)
        dL(-1, d + 12, e1, x3m[0], x3m[1], x3m[2], x3m[3]); // (s4, -1)
        dL(2, d + 16, e1, x4p[0], x4p[1], x4p[2], x4p[3]);  // (s3, +2)
        dL(-2, d + 16, e1, x4m[0], x4m[1], x4m[2], x4m[3]); // (s3, -2)
        const cd a = qh[3 * sj], b = qh[3 * sj + 1], cc = qh[3 * sj + 2];
        const cd nA = nu[3 * ti], nB_ = nu[3 * ti + 1], nC_ = nu[3 * ti + 2];
        double gd[4];
        for (int u = 0; u < 4; ++u) {
            // A = 1/2 L0[s1] a - 1/2 L2[s3] b + L1[s2] c,  B = 1/2 L0[s1] b - 1/2 L-2[s3] a + L-1[s2] c,
            // C = L0[s5] c + 1/2 L-1[s4] a + 1/2 L1[s4] b
            const cd A = 0.5 * (x0[u] * a) - 0.5 * (x4p[u] * b) + x2p[u] * cc;
            const cd Bv = 0.5 * (x0[u] * b) - 0.5 * (x4m[u] * a) + x2m[u] * cc;
            const cd Cv = x1[u] * cc + 0.5 * (x3m[u] * a) + 0.5 * (x3p[u] * b);
            gd[u] = (nA * A + nB_ * Bv + nC_ * Cv).x;
        }
        // d/dx_j = d/d(dx), d/dx_i = -d/d(dx); heights through the image maps
        const int64_t oj = perm[sj], oi = perm[ti];
        atomicAdd(grad + 3 * oj, gd[0]);
        atomicAdd(grad + 3 * oj + 1, gd[1]);
        atomicAdd(grad + 3 * oj + 2, ss * gd[2]);
        atomicAdd(grad + 3 * oi, -gd[0]);
        atomicAdd(grad + 3 * oi + 1, -gd[1]);
        atomicAdd(grad + 3 * oi + 2, st * gd[3]);
    }
}

void launch_grad_leaf(int p, int64_t N, int64_t nleaf, const int64_t *leaves, const BoxDev *boxes, const double *xyz,
                      const int64_t *perm, const cd *le, const cd *meb, const cd *qh, const cd *nu, const MediumDev &M,
                      const LayerScale &ls, double *grad, cudaStream_t st)
{
    if (N <= 0 || nleaf <= 0) return;
    k_grad_leaf<<<(unsigned)((N + 127) / 128), 128, 0, st>>>(p, nleaf, leaves, boxes, xyz, perm, le, meb, qh, nu, M,
                                                               ls, grad);
}

void launch_s2t_pre_grad(int64_t nnear, const NearPair *near, const BoxDev *boxes, const double *xyz,
                         const MediumDev &M, const CompDev *comps, double a, int node_cap, cd *coef, cudaStream_t st)
{
    if (nnear <= 0) return;
    k_s2t_pre_grad<<<(unsigned)nnear, 128, 0, st>>>(near, boxes, xyz, M, comps, a, node_cap, coef);
}

void launch_grad_near(int64_t nnear, const NearPair *near, const BoxDev *boxes, const double *xyz, const int64_t *perm,
                      const CompDev *comps, const cd *coefg, const cd *qh, const cd *nu, double *grad, cudaStream_t st)
{
    if (nnear <= 0) return;
    k_grad_near<<<(unsigned)nnear, 128, 0, st>>>(nnear, near, boxes, xyz, perm, comps, coefg, qh, nu, grad);
}

}  // namespace lmf
