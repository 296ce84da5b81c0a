// Setup kernels: density functions, M2L tabulation by the Chebyshev route of
// Section 3.4, and the M2M / L2L translation matrices.
#include "kernels.cuh"
#include "quad.cuh"
#include "specfun.cuh"

namespace lmf {

// ------------------------------------------------------------- densities
__global__ void k_densities(MediumDev M, int l, int lp, int64_t n, const cd *kr, cd *out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    cd ph[4], ps[4];
    densities_dev(M, kr[i], l, lp, 0, ph);
    densities_dev(M, kr[i], l, lp, 1, ps);
    for (int c = 0; c < 4; ++c) {
        out[i * 8 + c] = ph[c];
        out[i * 8 + 4 + c] = ps[c];
    }
}

void launch_densities(const MediumDev &M, int l, int lp, int64_t n, const cd *kr, cd *out,
                      cudaStream_t st)
{
    if (n <= 0) return;
    k_densities<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(M, l, lp, n, kr, out);
}

// ---------------------------------------------------------- quadrature nodes
// per-node factors for the Chebyshev integrals:
//   base_t = w Z sigma_t   (5 tables), tau_src[4], tau_tgt[4], T_l(x_prim), J_d(k rho)
__global__ void k_tab_nodes(const GeomDev *G, int g0, MediumDev M, const CompDev *comps,
                            int LM, int DJ, cd *Fb, cd *Fs, cd *Ft, cd *FT, cd *FJ, int *flag)
{
    const GeomDev &g = G[g0 + blockIdx.y];
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    int Q = g.plan.n1 + g.plan.nmid + 2 * g.plan.nray;
    if (q >= Q) return;
    int64_t o = g.node0 + q;
    const CompDev c = comps[g.comp];
    cd kr, w;
    int kind = plan_node(g.plan, q, kr, w);
    cd k = M.k[c.l], kp = M.k[c.lp];
    cd kz = kz_of(k, kr), kzp = kz_of(kp, kr);
    cd sg[5];
    sigmas_dev(M, kr, c.l, c.lp, c.tu, c.su, sg);
    cd Z = cexpd(mul_i(c.s * (kz * g.zs - kzp * g.zt)));
    cd wZ = w * Z;
    const int64_t S = g.stride;
    Fb[0 * S + o] = wZ * sg[0];
    Fb[1 * S + o] = wZ * sg[4];
    Fb[2 * S + o] = wZ * sg[1];
    Fb[3 * S + o] = wZ * sg[3];
    Fb[4 * S + o] = wZ * sg[2];
    Fs[0 * S + o] = mkd(1.0);
    Fs[1 * S + o] = k / kz;
    Fs[2 * S + o] = kr / k;
    Fs[3 * S + o] = kr / kz;
    Ft[0 * S + o] = mkd(1.0);
    Ft[1 * S + o] = kp / kzp;
    Ft[2 * S + o] = kr / kp;
    Ft[3 * S + o] = kr / kzp;
    cd kprim = g.src_primary ? k : kp;
    cd x = mkd(1.0) - 2.0 * (kr * kr) / (kprim * kprim);
    cd t0 = mkd(1.0), t1 = x;
    FT[0 * S + o] = t0;
    if (LM > 1) FT[1 * S + o] = t1;
    for (int l = 2; l < LM; ++l) {
        cd t2 = 2.0 * (x * t1) - t0;
        FT[l * S + o] = t2;
        t0 = t1;
        t1 = t2;
    }
    cd J[64];
    if (kind == 0) {
        if (bessel_j_seq<64>(kr * g.rho, DJ - 1, J)) atomicOr(flag, 1);
        for (int dd = 0; dd < DJ; ++dd) FJ[dd * S + o] = J[dd];
    } else {
        // H^(2)_n(z) = conj(H^(1)_n(conj z)) for integer n
        cd z = kr * g.rho;
        if (kind == 2) z = conj(z);
        hankel1_seq(z, DJ - 1, J);
        for (int dd = 0; dd < DJ; ++dd) FJ[dd * S + o] = 0.5 * (kind == 2 ? conj(J[dd]) : J[dd]);
    }
}

// I-breve[t][ts][tt][l][d] = sum_q base_t tau_s tau_t T_l J_d  for one
// geometry, table t and source tau-type ts (blockIdx = (geometry, t*4+ts)).
__global__ void k_tab_contract(const GeomDev *G, int g0, int LM, int DJ, const cd *Fb,
                               const cd *Fs, const cd *Ft, const cd *FT, const cd *FJ,
                               cd *Ibr, int64_t ibr_stride)
{
    extern __shared__ unsigned char smraw[];
    const int CH = 32;
    cd *W = (cd *)smraw;                 // [CH][4][LM]
    cd *Jc = W + CH * 4 * LM;            // [CH][DJ]
    const GeomDev &g = G[g0 + blockIdx.x];
    int t = blockIdx.y / 4, ts = blockIdx.y % 4;
    int Q = g.plan.n1 + g.plan.nmid + 2 * g.plan.nray;
    const int64_t S = g.stride;
    int64_t o0 = g.node0;
    const int NOUT = 4 * LM * DJ;
    const int PER = 12;   // NOUT <= 12 * 256 for p <= 16
    cd acc[PER];
    for (int i = 0; i < PER; ++i) acc[i] = mkd(0.0);
    for (int q0 = 0; q0 < Q; q0 += CH) {
        int nq = min(CH, Q - q0);
        for (int e = threadIdx.x; e < nq * 4 * LM; e += blockDim.x) {
            int q = e / (4 * LM), r = e % (4 * LM), tt = r / LM, l = r % LM;
            int64_t o = o0 + q0 + q;
            W[e] = Fb[t * S + o] * Fs[ts * S + o] * Ft[tt * S + o] * FT[l * S + o];
        }
        for (int e = threadIdx.x; e < nq * DJ; e += blockDim.x) {
            int q = e / DJ, dd = e % DJ;
            Jc[e] = FJ[dd * S + o0 + q0 + q];
        }
        __syncthreads();
        for (int i = 0; i < PER; ++i) {
            int out = threadIdx.x + i * blockDim.x;
            if (out >= NOUT) break;
            int r = out / DJ, dd = out % DJ;
            cd a = acc[i];
            for (int q = 0; q < nq; ++q) a += W[q * 4 * LM + r] * Jc[q * DJ + dd];
            acc[i] = a;
        }
        __syncthreads();
    }
    cd *dst = Ibr + (int64_t)blockIdx.x * ibr_stride + (int64_t)(t * 4 + ts) * NOUT;
    for (int i = 0; i < PER; ++i) {
        int out = threadIdx.x + i * blockDim.x;
        if (out < NOUT) dst[out] = acc[i];
    }
}

__device__ inline int tau_type(int n, int am)
{
    bool no = n & 1, mo = am & 1;
    if (!no && !mo) return 0;   // 1
    if (no && !mo) return 1;    // sec
    if (no && mo) return 2;     // sin
    return 3;                   // tan
}

// I-hat[t][row=(nu,mu)][col=(n',m')] = sgn(m') sgn(mu) sum_l G[(n',|m'|),(nu,|mu|)][l]
//   * I-breve[t][tau(n',m')][tau(nu,mu)][l][|d|] * (-1)^d [d<0],  d = m' - mu + kappa_t
__global__ void k_tab_assemble(const GeomDev *G, int g0, int p, int LM, int DJ, const cd *Gten,
                               const int *comp_gidx, const cd *Ibr, int64_t ibr_stride,
                               cd *tab)
{
    const int P = (p + 1) * (p + 1), T = (p + 1) * (p + 2) / 2;
    const GeomDev &g = G[g0 + blockIdx.z];
    int t = blockIdx.y;
    const int kap[5] = {0, 0, 1, 1, 2};
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P * P) return;
    int row = e / P, col = e % P;
    int nu = (int)sqrt((double)row + 0.5), mu;
    int n1 = (int)sqrt((double)col + 0.5), m1;
    while ((nu + 1) * (nu + 1) <= row) ++nu;
    while (nu * nu > row) --nu;
    mu = row - nu * nu - nu;
    while ((n1 + 1) * (n1 + 1) <= col) ++n1;
    while (n1 * n1 > col) --n1;
    m1 = col - n1 * n1 - n1;
    int am1 = m1 < 0 ? -m1 : m1, amu = mu < 0 ? -mu : mu;
    int dd = m1 - mu + kap[t];
    int ad = dd < 0 ? -dd : dd;
    double sgn = 1.0;
    if (m1 < 0 && (am1 & 1)) sgn = -sgn;
    if (mu < 0 && (amu & 1)) sgn = -sgn;
    if (dd < 0 && (ad & 1)) sgn = -sgn;
    int ts = tau_type(n1, am1), tt = tau_type(nu, amu);
    const cd *Gp = Gten + ((int64_t)comp_gidx[g.comp] * T * T + (int64_t)(((n1 * (n1 + 1)) / 2 + am1) * T
                           + (nu * (nu + 1)) / 2 + amu)) * LM;
    const cd *Ib = Ibr + (int64_t)blockIdx.z * ibr_stride + (int64_t)(t * 4 + ts) * (4 * LM * DJ)
                   + (int64_t)tt * LM * DJ;
    cd s = mkd(0.0);
    for (int l = 0; l < LM; ++l) s += Gp[l] * Ib[l * DJ + ad];
    tab[((int64_t)g.tab_index * NTAB + t) * P * P + e] = sgn * s;
}

// One batch of geometries [g0, g0+nb): node factors, I-breve, I-hat.  The
// scratch holds (5+4+4+LM+DJ) * stride node factors followed by nb I-breve
// blocks; stride is the batch's total node count.
void launch_tab_batch(const GeomDev *dG, int g0, int nb, int qmax, const MediumDev &M,
                      const CompDev *dcomps, int p, const cd *dGten, const int *dcgidx,
                      cd *scratch, int64_t stride, cd *tab, int *dflag, cudaStream_t st)
{
    const int LM = p + 2, DJ = 2 * p + 3, P = (p + 1) * (p + 1);
    const int NOUT = 4 * LM * DJ;
    const int64_t ibr_stride = (int64_t)NTAB * 4 * NOUT;
    const int64_t S = stride;
    cd *Fb = scratch, *Fs = Fb + 5 * S, *Ft = Fs + 4 * S, *FT = Ft + 4 * S, *FJ = FT + LM * S;
    cd *Ibr = FJ + DJ * S;
    dim3 gn((qmax + 127) / 128, nb);
    k_tab_nodes<<<gn, 128, 0, st>>>(dG, g0, M, dcomps, LM, DJ, Fb, Fs, Ft, FT, FJ, dflag);
    size_t sm = (size_t)(32 * 4 * LM + 32 * DJ) * sizeof(cd);
    dim3 gc(nb, NTAB * 4);
    k_tab_contract<<<gc, 256, sm, st>>>(dG, g0, LM, DJ, Fb, Fs, Ft, FT, FJ, Ibr, ibr_stride);
    dim3 ga((P * P + 255) / 256, NTAB, nb);
    k_tab_assemble<<<ga, 256, 0, st>>>(dG, g0, p, LM, DJ, dGten, dcgidx, Ibr, ibr_stride, tab);
}

}  // namespace lmf

namespace lmf {
cudaError_t configure_tab_kernels()
{
    return cudaFuncSetAttribute(k_tab_contract, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                160 * 1024);
}
}  // namespace lmf
