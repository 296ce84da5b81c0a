// Matvec kernels (FP64 form): permutation to helical components, P2M, M2M,
// M2L, L2L, L2P and the near-field S2T, plus the S2T precomputation.
#include "kernels.cuh"
#include "quad.cuh"
#include "specfun.cuh"

namespace lmf {

static __device__ inline void decode_nm(int idx, int &n, int &m)
{
    n = (int)sqrt((double)idx + 0.5);
    while ((n + 1) * (n + 1) <= idx) ++n;
    while (n * n > idx) --n;
    m = idx - n * n - n;
}

// ------------------------------------------------------------ permutation
// q_h[i] = (J_x + i J_y, J_x - i J_y, J_z) of point perm[i] (optionally of conj J)
__global__ void k_gather_in(int64_t N, const int64_t *perm, const cd *J, cd *qh, int cj)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int64_t o = perm[i];
    cd x = J[3 * o], y = J[3 * o + 1], z = J[3 * o + 2];
    if (cj) { x = conj(x); y = conj(y); z = conj(z); }
    qh[3 * i] = x + mul_i(y);
    qh[3 * i + 1] = x - mul_i(y);
    qh[3 * i + 2] = z;
}

// Phi[perm[i]] = ((A+B)/2, (A-B)/(2i), C) of the helical result (optionally conj)
__global__ void k_scatter_out(int64_t N, const int64_t *perm, const cd *ph, cd *Phi, int cj)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int64_t o = perm[i];
    cd A = ph[3 * i], B = ph[3 * i + 1], C = ph[3 * i + 2];
    cd x = 0.5 * (A + B), y = mul_mi(0.5 * (A - B));
    if (cj) { x = conj(x); y = conj(y); C = conj(C); }
    Phi[3 * o] = x;
    Phi[3 * o + 1] = y;
    Phi[3 * o + 2] = C;
}

void launch_gather_in(int64_t N, const int64_t *perm, const cd *J, cd *qh, bool conj_in,
                      cudaStream_t st)
{
    if (N > 0) k_gather_in<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, perm, J, qh, conj_in);
}
void launch_scatter_out(int64_t N, const int64_t *perm, const cd *phih, cd *Phi, bool conj_out,
                        cudaStream_t st)
{
    if (N > 0)
        k_scatter_out<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, perm, phih, Phi, conj_out);
}

// --------------------------------------------------------------- P2M, L2P
// basis b_nm(r) = j_n(k |r|) Y_n^m(r^) with Y_n^m = P^_n^|m| e^{i m phi}
// (times (-1)^m for m < 0); P2M uses 4 pi conj(Y) (eq. mecoeff).
static __device__ inline void point_basis(int p, cd k, double dx, double dy, double dz,
                                          bool conjugate, double scale, cd *out /*[P]*/)
{
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    double rxy = sqrt(dx * dx + dy * dy);
    double ct = r > 0 ? dz / r : 1.0, st = r > 0 ? rxy / r : 0.0;
    cd e1 = rxy > 0 ? cd{dx / rxy, dy / rxy} : cd{1.0, 0.0};
    if (conjugate) e1 = conj(e1);
    cd jn[LMF_PMAX + 1];
    sph_bessel_seq(k * r, p, jn);
    double Pl[(LMF_PMAX + 1) * (LMF_PMAX + 2) / 2];
    legendre_norm<double>(p, ct, st, Pl);
    cd em = mkd(1.0);   // e^{i m phi} (conjugated if requested)
    for (int m = 0; m <= p; ++m) {
        cd emc = conj(em);  // e^{-i m phi} ~ the m < 0 phase
        for (int n = m; n <= p; ++n) {
            double v = scale * Pl[(n * (n + 1)) / 2 + m];
            cd jv = v * jn[n];
            out[n * n + n + m] = jv * em;
            if (m > 0) out[n * n + n - m] = ((m & 1) ? -1.0 : 1.0) * (jv * emc);
        }
        em = em * e1;
    }
}

__global__ void k_p2m(int p, const int64_t *leaves, const BoxDev *boxes, const double *xyz,
                      const cd *qh, MediumDev M, cd *me)
{
    extern __shared__ unsigned char smraw[];
    const int P = (p + 1) * (p + 1);
    const int CH = 32;
    cd *bas = (cd *)smraw;          // [CH][P]
    cd *hq = bas + CH * P;          // [CH][3]
    int64_t bi = leaves[blockIdx.x];
    BoxDev b = boxes[bi];
    cd k = M.k[b.layer];
    const int NO = 3 * P;
    const int PER = (NO + blockDim.x - 1) / blockDim.x;   // <= 8 for P <= 441 w/ 192 thr
    cd acc[8];
    for (int i = 0; i < 8; ++i) acc[i] = mkd(0.0);
    for (int64_t c0 = b.p0; c0 < b.p1; c0 += CH) {
        int np = (int)min((int64_t)CH, b.p1 - c0);
        if (threadIdx.x < CH) {
            int j = threadIdx.x;
            if (j < np) {
                int64_t t = c0 + j;
                point_basis(p, k, xyz[3 * t] - b.c[0], xyz[3 * t + 1] - b.c[1],
                            xyz[3 * t + 2] - b.c[2], true, 4.0 * LMF_PI, bas + j * P);
                hq[3 * j] = qh[3 * t];
                hq[3 * j + 1] = qh[3 * t + 1];
                hq[3 * j + 2] = qh[3 * t + 2];
            }
        }
        __syncthreads();
        for (int i = 0; i < PER; ++i) {
            int o = threadIdx.x + i * blockDim.x;
            if (o >= NO) break;
            int v = o / P, nm = o % P;
            cd a = acc[i];
            for (int j = 0; j < np; ++j) a += hq[3 * j + v] * bas[j * P + nm];
            acc[i] = a;
        }
        __syncthreads();
    }
    for (int i = 0; i < PER; ++i) {
        int o = threadIdx.x + i * blockDim.x;
        if (o < NO) me[bi * NO + o] = acc[i];
    }
}

__global__ void k_l2p(int p, const int64_t *leaves, const BoxDev *boxes, const double *xyz,
                      const cd *le, MediumDev M, cd *ph)
{
    extern __shared__ unsigned char smraw[];
    const int P = (p + 1) * (p + 1);
    cd *L = (cd *)smraw;   // [3][P]
    int64_t bi = leaves[blockIdx.x];
    BoxDev b = boxes[bi];
    for (int e = threadIdx.x; e < 3 * P; e += blockDim.x) L[e] = le[bi * 3 * P + e];
    __syncthreads();
    cd k = M.k[b.layer];
    for (int64_t t = b.p0 + threadIdx.x; t < b.p1; t += blockDim.x) {
        double dx = xyz[3 * t] - b.c[0], dy = xyz[3 * t + 1] - b.c[1], dz = xyz[3 * t + 2] - b.c[2];
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        double rxy = sqrt(dx * dx + dy * dy);
        double ct = r > 0 ? dz / r : 1.0, st = r > 0 ? rxy / r : 0.0;
        cd e1 = rxy > 0 ? cd{dx / rxy, dy / rxy} : cd{1.0, 0.0};
        cd jn[LMF_PMAX + 1];
        sph_bessel_seq(k * r, p, jn);
        double Pl[(LMF_PMAX + 1) * (LMF_PMAX + 2) / 2];
        legendre_norm<double>(p, ct, st, Pl);
        cd A = mkd(0.0), B = mkd(0.0), C = mkd(0.0);
        cd em = mkd(1.0);
        for (int m = 0; m <= p; ++m) {
            cd emc = conj(em);
            double sg = (m & 1) ? -1.0 : 1.0;
            for (int n = m; n <= p; ++n) {
                cd jv = Pl[(n * (n + 1)) / 2 + m] * jn[n];
                cd bp = jv * em;
                int ip = n * n + n + m;
                A += L[ip] * bp;
                B += L[P + ip] * bp;
                C += L[2 * P + ip] * bp;
                if (m > 0) {
                    cd bm = sg * (jv * emc);
                    int im = n * n + n - m;
                    A += L[im] * bm;
                    B += L[P + im] * bm;
                    C += L[2 * P + im] * bm;
                }
            }
            em = em * e1;
        }
        ph[3 * t] = A;
        ph[3 * t + 1] = B;
        ph[3 * t + 2] = C;
    }
}

void launch_p2m(int p, int64_t nleaf, const int64_t *leaves, const BoxDev *boxes,
                const double *xyz, const cd *qh, const MediumDev &M, cd *me, cudaStream_t st)
{
    if (nleaf <= 0) return;
    const int P = (p + 1) * (p + 1);
    size_t sm = (size_t)(32 * P + 32 * 3) * sizeof(cd);
    int thr = 3 * P <= 8 * 128 ? 128 : 256;
    k_p2m<<<(unsigned)nleaf, thr, sm, st>>>(p, leaves, boxes, xyz, qh, M, me);
}

void launch_l2p(int p, int64_t nleaf, const int64_t *leaves, const BoxDev *boxes,
                const double *xyz, const cd *le, const MediumDev &M, cd *phih, cudaStream_t st)
{
    if (nleaf <= 0) return;
    const int P = (p + 1) * (p + 1);
    k_l2p<<<(unsigned)nleaf, 64, 3 * P * sizeof(cd), st>>>(p, leaves, boxes, xyz, le, M, phih);
}

// ---------------------------------------------------------------- GEMM core
// Y(P x ncol) = A(P x P) X(P x NC smem); store(r, c, y) for c < ncol.
// 256 threads: column c = tid % NC, row group tid / NC.
template <int NC, int RCH, typename Store>
__device__ inline void gemm_core(int P, const cd *__restrict__ A, const cd *X, int ncol,
                                 Store store)
{
    const int c = threadIdx.x % NC, rg = threadIdx.x / NC, nrg = blockDim.x / NC;
    for (int r0 = rg; r0 < P; r0 += nrg * RCH) {
        cd acc[RCH];
        for (int i = 0; i < RCH; ++i) acc[i] = mkd(0.0);
        for (int k = 0; k < P; ++k) {
            cd x = X[k * NC + c];
#pragma unroll
            for (int i = 0; i < RCH; ++i) {
                int r = r0 + i * nrg;
                if (r < P) {
                    double2 av = __ldg((const double2 *)(A + (int64_t)r * P + k));
                    acc[i] += cd{av.x, av.y} * x;
                }
            }
        }
        if (c < ncol)
            for (int i = 0; i < RCH; ++i) {
                int r = r0 + i * nrg;
                if (r < P) store(r, c, acc[i]);
            }
    }
}

// M2M (atomic, child -> parent) and L2L (child += parent), columns = (pair, v)
__global__ void k_group_gemm(int p, const GemmWork *work, const cd *mats, const int64_t *src,
                             const int64_t *dst, const cd *in, cd *out, int atomic)
{
    extern __shared__ unsigned char smraw[];
    const int P = (p + 1) * (p + 1);
    const int NC = 30;   // 10 pairs x 3 helical components (padded to 32 columns)
    cd *X = (cd *)smraw; // [P][32]
    GemmWork w = work[blockIdx.x];
    int ncol = 3 * w.npair;
    for (int e = threadIdx.x; e < P * 32; e += blockDim.x) {
        int k = e / 32, col = e % 32;
        cd v = mkd(0.0);
        if (col < ncol) {
            int pp = col / 3, vv = col % 3;
            v = in[(src[w.pair0 + pp] * 3 + vv) * P + k];
        }
        X[e] = v;
    }
    __syncthreads();
    const cd *A = mats + (int64_t)w.group * P * P;
    auto store = [&](int r, int col, cd y) {
        int pp = col / 3, vv = col % 3;
        cd *o = out + (dst[w.pair0 + pp] * 3 + vv) * P + r;
        if (atomic) {
            atomicAdd(&o->x, y.x);
            atomicAdd(&o->y, y.y);
        } else {
            *o += y;
        }
    };
    gemm_core<32, 6>(P, A, X, ncol, store);
    (void)NC;
}

void launch_group_gemm(int p, int64_t nwork, const GemmWork *work, const cd *mats,
                       const int64_t *src, const int64_t *dst, const cd *in, cd *out,
                       bool atomic, cudaStream_t st)
{
    if (nwork <= 0) return;
    const int P = (p + 1) * (p + 1);
    size_t sm = (size_t)P * 32 * sizeof(cd);
    k_group_gemm<<<(unsigned)nwork, 256, sm, st>>>(p, work, mats, src, dst, in, out, atomic);
}

// --------------------------------------------------------------------- M2L
// Column roles per table t: (input helical v, signed kappa, coefficient,
// output helical v) for
//   A' = 1/2 T0[s1] a - 1/2 T2[s3] b + T1[s2] c
//   B' = 1/2 T0[s1] b - 1/2 T-2[s3] a + T-1[s2] c
//   C' = T0[s5] c + 1/2 T-1[s4] a + 1/2 T1[s4] b
struct ColSpec { int vin, kap; double coef; int vout; };
__constant__ ColSpec c_cols[5][2] = {
    {{0, 0, 0.5, 0}, {1, 0, 0.5, 1}},     // (s1, 0)
    {{2, 0, 1.0, 2}, {2, 0, 1.0, 2}},     // (s5, 0)  (one column)
    {{2, 1, 1.0, 0}, {2, -1, 1.0, 1}},    // (s2, 1)
    {{1, 1, 0.5, 2}, {0, -1, 0.5, 2}},    // (s4, 1)
    {{1, 2, -0.5, 0}, {0, -2, -0.5, 1}},  // (s3, 2)
};

// The M2L of eq. M2L_scale_with_Tnmu with T = (-i)^nu i^(n'+1+d) s^(nu+mu+n'+m')
// e^{i d phi} I-hat, d = m' - mu + kappa, factorised as
//   in(n',m')  = (i s)^(n'+m') e^{i m' phi}  [x (-1)^(n'+m') for a mirrored source]
//   out(nu,mu) = (-i s)^(nu+mu) e^{-i mu phi} [x (-1)^(nu+mu) for a mirrored target]
//   const      = i^(1+kappa) e^{i kappa phi} x coefficient.
// kappa < 0 uses I-hat_{-kappa}[nu,mu,n',m'] = (-1)^kappa I-hat_kappa[nu,-mu,n',-m']:
// the input column is flipped in m before the product, the output after.
__global__ void k_m2l(int p, const M2LWork *work, const GeomDev *geoms, const CompDev *comps,
                      const M2LPair *pairs, const cd *tab, const cd *me, cd *le)
{
    extern __shared__ unsigned char smraw[];
    const int P = (p + 1) * (p + 1);
    cd *X = (cd *)smraw;   // [P][32]
    M2LWork w = work[blockIdx.x];
    const GeomDev &g = geoms[w.geom];
    const CompDev c = comps[g.comp];
    const int t = w.t;
    const int ncpp = (t == 1) ? 1 : 2;
    const int ncol = w.npair * ncpp;
    const double s = c.s;
    for (int e = threadIdx.x; e < P * 32; e += blockDim.x) {
        int k = e / 32, col = e % 32;
        cd v = mkd(0.0);
        if (col < ncol) {
            int pp = col / ncpp, j = col % ncpp;
            ColSpec cs = c_cols[t][j];
            M2LPair pr = pairs[w.pair0 + pp];
            int n, m;
            decode_nm(k, n, m);
            int ms = cs.kap < 0 ? -m : m;
            cd x = me[(pr.src * 3 + cs.vin) * P + n * n + n + ms];
            // in(n, ms)
            int e1 = n + ms;
            cd sc = ipow<double>(e1);
            if (s < 0 && (e1 & 1)) sc = -sc;
            if (c.has_src_refl && (e1 & 1)) sc = -sc;
            double phi = atan2(pr.sphi, pr.cphi), sn, cs_;
            sincos(ms * phi, &sn, &cs_);
            v = sc * (cd{cs_, sn} * x);
        }
        X[e] = v;
    }
    __syncthreads();
    const cd *A = tab + ((int64_t)g.tab_index * NTAB + t) * P * P;
    auto store = [&](int r, int col, cd y) {
        int pp = col / ncpp, j = col % ncpp;
        ColSpec cs = c_cols[t][j];
        M2LPair pr = pairs[w.pair0 + pp];
        int nu, mh;
        decode_nm(r, nu, mh);
        int mu = cs.kap < 0 ? -mh : mh;
        int e2 = nu + mu;
        cd sc = ipow<double>(-e2);   // (-i)^(nu+mu)
        if (s < 0 && (e2 & 1)) sc = -sc;
        if (c.has_tgt_refl && (e2 & 1)) sc = -sc;
        double phi = atan2(pr.sphi, pr.cphi), sn, cs_;
        sincos((cs.kap - mu) * phi, &sn, &cs_);
        cd k1 = ipow<double>(1 + cs.kap);
        double cf = cs.coef;
        if (cs.kap < 0 && (cs.kap & 1)) cf = -cf;
        cd yy = cf * (sc * (k1 * (cd{cs_, sn} * y)));
        cd *o = le + (pr.tgt * 3 + cs.vout) * P + nu * nu + nu + mu;
        atomicAdd(&o->x, yy.x);
        atomicAdd(&o->y, yy.y);
    };
    gemm_core<32, 6>(P, A, X, ncol, store);
}

void launch_m2l(int p, int64_t nwork, const M2LWork *work, const GeomDev *geoms,
                const CompDev *comps, const M2LPair *pairs, const cd *tab, const cd *me, cd *le,
                cudaStream_t st)
{
    if (nwork <= 0) return;
    const int P = (p + 1) * (p + 1);
    size_t sm = (size_t)P * 32 * sizeof(cd);
    k_m2l<<<(unsigned)nwork, 256, sm, st>>>(p, work, geoms, comps, pairs, tab, me, le);
}

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
                          MediumDev M, const CompDev *comps, double a, double kp, cd *coef,
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
        if (plan_nodes(pl) > (1 << 20)) {
            atomicOr(flag, 2);
            pl.nmid = 16;
            pl.nray = 0;
        }
    }
    __syncthreads();
    int Q = plan_nodes(pl);
    (void)kp;
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
                    const MediumDev &M, const CompDev *comps, double a, double kp, cd *coef,
                    int *dflag, cudaStream_t st)
{
    if (nnear <= 0) return;
    k_s2t_pre<<<(unsigned)nnear, 128, 0, st>>>(near, boxes, xyz, M, comps, a, kp, coef, dflag);
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
    const int big = 200 * 1024;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_p2m, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_group_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_m2l, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    return cudaSuccess;
}
}  // namespace lmf
