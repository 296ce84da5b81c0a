/*
 * CPU oracle for the interface-induced reaction field of the electric dyadic
 * Green's function of Maxwell's equations in a horizontally layered medium.
 *
 * TEST INFRASTRUCTURE.  This file is the slow, plain FP64 reference that the
 * GPU library is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load it; the library never does.  It shares no
 * code, header or table with the CUDA path.
 *
 * Conventions (Section 3.1): omega = 1 and mu_l = 1 in every layer, so that
 * eps_l = k_l^2.  Layers are 0..L from top to bottom, interface d_l separates
 * layers l and l+1, d_0 > d_1 > ... > d_{L-1}.  k_{lz} = sqrt(k_l^2 - krho^2)
 * with Im k_{lz} >= 0.
 *
 * What is computed, and how (each step is the plain definition):
 *  - the scalar layered Green's functions phi, psi of the interface problems
 *    (eqs. helmholtzb1, helmholtzb2) by a dense 2L x 2L linear solve of the
 *    interface conditions, with the point source as right-hand side;
 *  - the spectral dyad of eq. eq-GEGH-b-latest (J1..J5 terms) minus its
 *    free-space part, integrated over the angle alpha in closed form with the
 *    Jacobi-Anger identity (1/2pi) int e^{i x cos(a-f)} e^{i n a} da
 *    = i^n J_n(x) e^{i n f};
 *  - the remaining k_rho integral (1/2pi) int_0^inf k_rho (...) dk_rho by
 *    adaptive Gauss-Kronrod (7/15) on a path that leaves the real axis below
 *    every pole and branch point, then follows the real axis to a cut-off set
 *    by the vertical decay distance;
 *  - the direct sum Phi_i = sum_j G^r(r_j, r_i) q_j of eq. allcomponents
 *    (first Green's-function slot summed, as in the paper), reaction part
 *    only, self term included;
 *  - the density functions phi^{*star}, psi^{*star} of eq. threedensity as the
 *    coefficients of the four vertical-exponential components, obtained by
 *    driving the same interface system with a source that emits only upward
 *    (star = up) or only downward (star = down) waves;
 *  - single entries of the M2L Sommerfeld integrals of eq.
 *    onedimensionintegral with the normalised Legendre functions evaluated by
 *    their textbook recurrence.
 * Bessel functions: J_n of a real argument from the C library (jn); of a
 * complex argument from Bessel's integral J_n(z) = (1/2pi) int_0^{2pi}
 * e^{i(z sin t - n t)} dt by the trapezoid rule, which is spectrally
 * accurate for this periodic integrand.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;
#define OR_MAXL 12
#define OR_PI 3.14159265358979323846

typedef struct {
    int L;                 /* number of interfaces */
    double d[OR_MAXL];     /* interface heights */
    cplx k[OR_MAXL + 1];   /* layer wavenumbers */
} or_medium;

static void make_medium(or_medium *m, int L, const double *d, const double *kri)
{
    m->L = L;
    for (int i = 0; i < L; ++i) m->d[i] = d[i];
    for (int i = 0; i <= L; ++i) m->k[i] = kri[2 * i] + I * kri[2 * i + 1];
}

static cplx kz_of(cplx k, cplx kr)
{
    cplx s = csqrt(k * k - kr * kr);
    if (cimag(s) < 0.0) s = -s;
    return s;
}

int or_layer_of(int L, const double *d, double z)
{
    for (int i = 0; i < L; ++i)
        if (fabs(z - d[i]) < 1e-12) return -1;
    int l = 0;
    while (l < L && z < d[l]) ++l;
    return l;
}

/* ---------------------------------------------------------------- Bessel */

/* J_0..J_nmax at complex z by the trapezoid rule on Bessel's integral. */
static void besselj_complex(int nmax, cplx z, cplx *out)
{
    int N = (int)ceil(cabs(z) + nmax + 48.0);
    if (N < 64) N = 64;
    for (int n = 0; n <= nmax; ++n) out[n] = 0;
    for (int j = 0; j < N; ++j) {
        double t = 2.0 * OR_PI * j / N;
        cplx e = cexp(I * z * sin(t));
        cplx rot = cexp(-I * t), ph = 1.0;
        for (int n = 0; n <= nmax; ++n) {
            out[n] += e * ph;
            ph *= rot;
        }
    }
    for (int n = 0; n <= nmax; ++n) out[n] /= N;
}

/* J_n(z) = (z/2)^n sum_k (-z^2/4)^k / (k! (n+k)!), summed in long double;
 * used for |z| < 6, where the largest term is below e^6. */
static void besselj_series(int nmax, cplx z, cplx *out)
{
    long double complex h = 0.5L * z, q = -h * h, hn = 1.0L;
    long double nfact = 1.0L;
    for (int n = 0; n <= nmax; ++n) {
        if (n > 0) { hn *= h; nfact *= n; }
        long double complex term = 1.0L / nfact, sum = term;
        for (int k = 1; k < 200; ++k) {
            term *= q / ((long double)k * (long double)(n + k));
            sum += term;
            if (cabsl(term) < 1e-22L * cabsl(sum)) break;
        }
        out[n] = (cplx)(hn * sum);
    }
}

static void besselj_any(int nmax, cplx z, cplx *out)
{
    if (cimag(z) == 0.0 && creal(z) >= 0.0) {
        double x = creal(z);
        for (int n = 0; n <= nmax; ++n) out[n] = jn(n, x);
    } else if (cabs(z) < 6.0) {
        besselj_series(nmax, z, out);
    } else {
        besselj_complex(nmax, z, out);
    }
}

void or_besselj(int nmax, double zr, double zi, double *out)
{
    cplx tmp[256];
    besselj_any(nmax, zr + I * zi, tmp);
    for (int n = 0; n <= nmax; ++n) {
        out[2 * n] = creal(tmp[n]);
        out[2 * n + 1] = cimag(tmp[n]);
    }
}

/* ------------------------------------------------------- 1-D layer solve */

/* Dense complex Gaussian elimination with partial pivoting, nrhs columns. */
static int gauss_solve(int n, cplx *A, int nrhs, cplx *B)
{
    for (int c = 0; c < n; ++c) {
        int piv = c;
        double best = cabs(A[c * n + c]);
        for (int r = c + 1; r < n; ++r)
            if (cabs(A[r * n + c]) > best) { best = cabs(A[r * n + c]); piv = r; }
        if (best == 0.0) return -1;
        if (piv != c) {
            for (int j = 0; j < n; ++j) { cplx t = A[c * n + j]; A[c * n + j] = A[piv * n + j]; A[piv * n + j] = t; }
            for (int j = 0; j < nrhs; ++j) { cplx t = B[c * nrhs + j]; B[c * nrhs + j] = B[piv * nrhs + j]; B[piv * nrhs + j] = t; }
        }
        for (int r = c + 1; r < n; ++r) {
            cplx f = A[r * n + c] / A[c * n + c];
            if (f == 0) continue;
            for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
            for (int j = 0; j < nrhs; ++j) B[r * nrhs + j] -= f * B[c * nrhs + j];
        }
    }
    for (int c = n - 1; c >= 0; --c) {
        for (int j = 0; j < nrhs; ++j) {
            cplx s = B[c * nrhs + j];
            for (int k = c + 1; k < n; ++k) s -= A[c * n + k] * B[k * nrhs + j];
            B[c * nrhs + j] = s / A[c * n + c];
        }
    }
    return 0;
}

/*
 * Interface problem u'' + k_{jz}^2 u = -i delta(z - zp) in layer lp, with u and
 * (1/eta) u' continuous across every interface, eta = 1 for phi (mu = 1,
 * eq. helmholtzb1) and eta = eps = k^2 for psi (eq. helmholtzb2); the source
 * strength -i/omega (-i/(mu omega) for psi) is -i for omega = mu = 1.  In layer
 * j the field is  A_j e^{i k_jz (z - d_j)} + B_j e^{-i k_jz (z - d_{j-1})}
 * plus, in layer lp only, the free-space field F = -e^{i k_z |z - zp|}/(2 k_z).
 * mode: 0 = point source, 1 = only the upward-emitted part of F, 2 = only
 * the downward-emitted part.  Returns, for target layer l, (A_l, B_l) for the
 * source (rhs 0) and for its derivative in zp (rhs 1).
 */
static int solve_1d(const or_medium *m, cplx kr, int psi, int lp, double zp,
                    int mode, int l, cplx AB[2][2])
{
    int L = m->L, n = 2 * L;
    cplx kz[OR_MAXL + 1], eta[OR_MAXL + 1], ej[OR_MAXL + 1];
    cplx A[4 * OR_MAXL * OR_MAXL], B[4 * OR_MAXL];
    AB[0][0] = AB[0][1] = AB[1][0] = AB[1][1] = 0;
    if (L <= 0 || L > OR_MAXL) return L == 0 ? 0 : -1;
    for (int j = 0; j <= L; ++j) {
        kz[j] = kz_of(m->k[j], kr);
        eta[j] = psi ? m->k[j] * m->k[j] : 1.0;
        ej[j] = (j >= 1 && j <= L - 1) ? cexp(I * kz[j] * (m->d[j - 1] - m->d[j])) : 0.0;
    }
    memset(A, 0, sizeof(cplx) * n * n);
    memset(B, 0, sizeof(cplx) * n * 2);
#define IA(j) (2 * (j))
#define IB(j) (2 * (j) - 1)
    for (int i = 0; i < L; ++i) {
        int r0 = 2 * i, r1 = 2 * i + 1;
        int up = i, dn = i + 1;
        /* layer i (above interface i) evaluated at d_i */
        A[r0 * n + IA(up)] += 1.0;
        A[r1 * n + IA(up)] += I * kz[up] / eta[up];
        if (up >= 1) {
            A[r0 * n + IB(up)] += ej[up];
            A[r1 * n + IB(up)] += -I * kz[up] * ej[up] / eta[up];
        }
        /* layer i+1 (below) evaluated at d_i */
        if (dn <= L - 1) {
            A[r0 * n + IA(dn)] -= ej[dn];
            A[r1 * n + IA(dn)] -= I * kz[dn] * ej[dn] / eta[dn];
        }
        A[r0 * n + IB(dn)] -= 1.0;
        A[r1 * n + IB(dn)] -= -I * kz[dn] / eta[dn];
        /* free-space field of the source layer */
        cplx k1 = kz[lp];
        if (lp == up && mode != 1) {          /* bottom interface of source layer */
            cplx F = -cexp(I * k1 * (zp - m->d[i])) / (2.0 * k1);
            cplx Fz = -I * k1 * F, Fp = I * k1 * F, Fzp = k1 * k1 * F;
            B[r0 * 2 + 0] -= F;       B[r1 * 2 + 0] -= Fz / eta[lp];
            B[r0 * 2 + 1] -= Fp;      B[r1 * 2 + 1] -= Fzp / eta[lp];
        }
        if (lp == dn && mode != 2) {          /* top interface of source layer */
            cplx F = -cexp(I * k1 * (m->d[i] - zp)) / (2.0 * k1);
            cplx Fz = I * k1 * F, Fp = -I * k1 * F, Fzp = k1 * k1 * F;
            B[r0 * 2 + 0] += F;       B[r1 * 2 + 0] += Fz / eta[lp];
            B[r0 * 2 + 1] += Fp;      B[r1 * 2 + 1] += Fzp / eta[lp];
        }
    }
    if (gauss_solve(n, A, 2, B)) return -1;
    for (int r = 0; r < 2; ++r) {
        AB[r][0] = (l <= L - 1) ? B[IA(l) * 2 + r] : 0.0;
        AB[r][1] = (l >= 1) ? B[IB(l) * 2 + r] : 0.0;
    }
#undef IA
#undef IB
    return 0;
}

/* Reaction part at (z in layer l, zp in layer lp): out = {u, du/dz, du/dzp,
 * d2u/dz dzp}. */
static int reaction_1d(const or_medium *m, cplx kr, int psi, int l, double z,
                       int lp, double zp, cplx out[4])
{
    cplx AB[2][2];
    if (solve_1d(m, kr, psi, lp, zp, 0, l, AB)) return -1;
    cplx kzl = kz_of(m->k[l], kr);
    cplx eA = (l <= m->L - 1) ? cexp(I * kzl * (z - m->d[l])) : 0.0;
    cplx eB = (l >= 1) ? cexp(-I * kzl * (z - m->d[l - 1])) : 0.0;
    out[0] = AB[0][0] * eA + AB[0][1] * eB;
    out[1] = I * kzl * (AB[0][0] * eA - AB[0][1] * eB);
    out[2] = AB[1][0] * eA + AB[1][1] * eB;
    out[3] = I * kzl * (AB[1][0] * eA - AB[1][1] * eB);
    return 0;
}

void or_reaction_1d(int L, const double *d, const double *kri, double krr,
                    double kri_, int psi, int l, double z, int lp, double zp,
                    double *out)
{
    or_medium m;
    make_medium(&m, L, d, kri);
    cplx o[4];
    reaction_1d(&m, krr + I * kri_, psi, l, z, lp, zp, o);
    for (int i = 0; i < 4; ++i) { out[2 * i] = creal(o[i]); out[2 * i + 1] = cimag(o[i]); }
}

/* ------------------------------------------------- Z-exponential phases */

/* Exponent E with Z^{*star}_{l lp}(z, zp) = e^{i E} (eq. zexponential).
 * tgt_up: * = up; src_up: star = up.  tau_j(z) = 2 d_j - z. */
static cplx z_phase(const or_medium *m, int l, int lp, int tgt_up, int src_up,
                    cplx kz, cplx kzp, double z, double zp)
{
    const double *d = m->d;
#define TAU(j, x) (2.0 * d[(j)] - (x))
    if (tgt_up && src_up)
        return (l < lp) ? kz * z - kzp * zp : kzp * TAU(lp - 1, zp) - kz * TAU(l, z);
    if (tgt_up && !src_up)
        return (l <= lp) ? kz * z - kzp * TAU(lp, zp) : kzp * zp - kz * TAU(l, z);
    if (!tgt_up && src_up)
        return (l < lp) ? kz * TAU(l - 1, z) - kzp * zp : kzp * TAU(lp - 1, zp) - kz * z;
    return (l <= lp) ? kz * TAU(l - 1, z) - kzp * TAU(lp, zp) : kzp * zp - kz * z;
#undef TAU
}

/*
 * Density functions phi^{*star}_{l lp}(krho), psi^{*star}_{l lp}(krho) of
 * eq. threedensity, defined by
 *   u^r_l(z, zp) = -1/(2 k_{lp z}) sum_{*,star} u^{*star} Z^{*star}(z, zp)
 * (omega = mu = 1).  The star = up (down) part is the response to the
 * upward (downward) emitted wave alone; the * = up (down) part is the A (B)
 * coefficient of the target layer.  Order: (up,up), (up,dn), (dn,up), (dn,dn).
 */
static int densities(const or_medium *m, cplx kr, int l, int lp, cplx phi[4], cplx psi[4])
{
    int L = m->L;
    cplx kz = kz_of(m->k[l], kr), kzp = kz_of(m->k[lp], kr);
    for (int c = 0; c < 4; ++c) phi[c] = psi[c] = 0;
    for (int src_up = 1; src_up >= 0; --src_up) {
        if (src_up && lp == 0) continue;      /* nothing above the top layer */
        if (!src_up && lp == L) continue;     /* nothing below the bottom layer */
        double zp = src_up ? m->d[lp - 1] : m->d[lp];
        for (int w = 0; w < 2; ++w) {
            cplx AB[2][2];
            if (solve_1d(m, kr, w, lp, zp, src_up ? 1 : 2, l, AB)) return -1;
            for (int tgt_up = 1; tgt_up >= 0; --tgt_up) {
                if (tgt_up && l == L) continue;
                if (!tgt_up && l == 0) continue;
                double z = tgt_up ? m->d[l] : m->d[l - 1];
                cplx coef = tgt_up ? AB[0][0] : AB[0][1];
                cplx val = 0;
                if (coef != 0) {
                    cplx E = z_phase(m, l, lp, tgt_up, src_up, kz, kzp, z, zp);
                    val = -2.0 * kzp * cexp(clog(coef) - I * E);
                }
                int c = (tgt_up ? 0 : 2) + (src_up ? 0 : 1);
                if (w == 0) phi[c] = val; else psi[c] = val;
            }
        }
    }
    return 0;
}

void or_densities(int L, const double *d, const double *kri, double krr, double kri_,
                  int l, int lp, double *out)
{
    or_medium m;
    make_medium(&m, L, d, kri);
    cplx ph[4], ps[4];
    densities(&m, krr + I * kri_, l, lp, ph, ps);
    for (int c = 0; c < 4; ++c) {
        out[2 * c] = creal(ph[c]); out[2 * c + 1] = cimag(ph[c]);
        out[8 + 2 * c] = creal(ps[c]); out[8 + 2 * c + 1] = cimag(ps[c]);
    }
}

/* sigma_1..sigma_5 of Section 3.1 (eq. after Theta), gamma = 1/k_l^2 for
 * mu = 1.  The psi term of sigma_1 and sigma_3 carries the sign
 * eps = s_tgt * s_src with s_tgt = +1 (* = up), s_src = +1 (star = down):
 * sigma_1 = phi/k'_z - eps gamma k_z psi, sigma_3 = phi/k'_z + eps gamma k_z psi.
 * literal_sigma3 != 0 uses the printed sigma_3 instead (+ for star = down,
 * - for star = up, independent of *). */
static void sigmas(const or_medium *m, cplx kr, int l, int lp, int tgt_up, int src_up,
                   int literal_sigma3, cplx sg[5])
{
    cplx ph[4], ps[4];
    densities(m, kr, l, lp, ph, ps);
    int c = (tgt_up ? 0 : 2) + (src_up ? 0 : 1);
    cplx kz = kz_of(m->k[l], kr), kzp = kz_of(m->k[lp], kr);
    cplx gam = 1.0 / (m->k[l] * m->k[l]);
    double st = tgt_up ? 1.0 : -1.0, ss = src_up ? -1.0 : 1.0, eps = st * ss;
    sg[0] = ph[c] / kzp - eps * gam * kz * ps[c];
    sg[1] = -st * gam * kr * kz * ps[c] / kzp;
    sg[2] = literal_sigma3 ? ph[c] / kzp + ss * gam * kz * ps[c]
                           : ph[c] / kzp + eps * gam * kz * ps[c];
    sg[3] = ss * gam * kr * ps[c];
    sg[4] = gam * kr * kr * ps[c] / kzp;
}

void or_sigmas(int L, const double *d, const double *kri, double krr, double kri_,
               int l, int lp, int tgt_up, int src_up, int literal, double *out)
{
    or_medium m;
    make_medium(&m, L, d, kri);
    cplx sg[5];
    sigmas(&m, krr + I * kri_, l, lp, tgt_up, src_up, literal, sg);
    for (int i = 0; i < 5; ++i) { out[2 * i] = creal(sg[i]); out[2 * i + 1] = cimag(sg[i]); }
}

/* s^{*star}_{l lp} of eq. eq_signs */
static double s_sign(int l, int lp, int src_up)
{
    if (src_up) return (l < lp) ? 1.0 : -1.0;
    return (l <= lp) ? 1.0 : -1.0;
}

/* ----------------------------------------------------- adaptive quadrature */

typedef void (*or_fn)(cplx kr, void *ctx, cplx *out);

static const double GK_X[8] = {
    0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
    0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
    0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
    0.207784955007898467600689403773245, 0.0};
static const double GK_WK[8] = {
    0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
    0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
    0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
    0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double GK_WG[4] = {
    0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
    0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

#define OR_MAXV 40000

typedef struct {
    or_fn f;
    void *ctx;
    int nv;
    long nfev;
    cplx *buf;      /* nv */
    cplx *kr15;     /* 15*nv */
    /* per-component error control (NULL: one tolerance for all components,
     * relative to the largest): the error estimate and L1 magnitude of every
     * component from the last gk15 call, and each component's L1 scale */
    double *cerr, *cmag, *cscale;
} quad_ws;

/* Gauss-Kronrod 7/15 on the straight segment [z0, z1]; returns the error
 * estimate |K15 - G7| (max over components) and, in *l1, the L1 magnitude
 * |h| sum_j w_j |f_j| (max over components), which bounds the round-off. */
static double gk15(quad_ws *w, cplx z0, cplx z1, cplx *K, double *l1)
{
    int nv = w->nv;
    cplx c = 0.5 * (z0 + z1), h = 0.5 * (z1 - z0);
    cplx *G = w->kr15;
    double *A = (double *)malloc(sizeof(double) * nv);
    for (int v = 0; v < nv; ++v) { K[v] = 0; G[v] = 0; A[v] = 0; }
    double err = 0.0, s1 = 0.0;
    for (int j = 0; j < 15; ++j) {
        int idx = j < 7 ? j : (j == 7 ? 7 : 14 - j);
        double x = j < 7 ? -GK_X[j] : (j == 7 ? 0.0 : GK_X[14 - j]);
        w->f(c + h * x, w->ctx, w->buf);
        w->nfev++;
        double wk = GK_WK[idx];
        int gi = (idx % 2 == 1) ? (idx / 2) : -1;   /* Gauss nodes: 1,3,5,7 */
        for (int v = 0; v < nv; ++v) {
            K[v] += wk * w->buf[v];
            A[v] += wk * cabs(w->buf[v]);
            if (gi >= 0) G[v] += GK_WG[gi] * w->buf[v];
        }
    }
    for (int v = 0; v < nv; ++v) {
        K[v] *= h; G[v] *= h;
        double e = cabs(K[v] - G[v]);
        if (e > err) err = e;
        double a = A[v] * cabs(h);
        if (a > s1) s1 = a;
        if (w->cerr) { w->cerr[v] = e; w->cmag[v] = a; }
    }
    free(A);
    if (l1) *l1 = s1;
    return err;
}

static void adapt(quad_ws *w, cplx z0, cplx z1, double tol, int depth, cplx *acc,
                  const cplx *K0, double err0, double mag0)
{
    cplx *K = (cplx *)malloc(sizeof(cplx) * w->nv);
    double mag, err;
    if (K0) {
        for (int v = 0; v < w->nv; ++v) K[v] = K0[v];
        err = err0; mag = mag0;
    } else {
        err = gk15(w, z0, z1, K, &mag);
    }
    if (err <= tol || depth >= 24 || err <= 50.0 * 2.2e-16 * mag) {
        for (int v = 0; v < w->nv; ++v) acc[v] += K[v];
        free(K);
        return;
    }
    free(K);
    cplx zm = 0.5 * (z0 + z1);
    adapt(w, z0, zm, 0.5 * tol, depth + 1, acc, NULL, 0, 0);
    adapt(w, zm, z1, 0.5 * tol, depth + 1, acc, NULL, 0, 0);
}

/* per-component form of adapt: every component must meet its own share of
 * the tolerance, frac times its L1 scale over the whole path (or the
 * round-off floor of its own magnitude on the segment) */
static void adapt_pc(quad_ws *w, cplx z0, cplx z1, double frac, int depth, cplx *acc)
{
    cplx *K = (cplx *)malloc(sizeof(cplx) * w->nv);
    gk15(w, z0, z1, K, NULL);
    int ok = depth >= 24;
    if (!ok) {
        ok = 1;
        for (int v = 0; v < w->nv && ok; ++v)
            if (w->cerr[v] > frac * w->cscale[v] && w->cerr[v] > 50.0 * 2.2e-16 * w->cmag[v]) ok = 0;
    }
    if (ok) {
        for (int v = 0; v < w->nv; ++v) acc[v] += K[v];
        free(K);
        return;
    }
    free(K);
    cplx zm = 0.5 * (z0 + z1);
    adapt_pc(w, z0, zm, 0.5 * frac, depth + 1, acc);
    adapt_pc(w, zm, z1, 0.5 * frac, depth + 1, acc);
}

/*
 * int_0^inf f(kr) dkr along 0 -> -ih -> a-ih -> a (below every pole and
 * branch point, which lie in the closed first quadrant), then [a, X] on the
 * real axis.  X is set from the vertical decay distance D: the integrand
 * decays like e^{-kr D} times a polynomial.  Panels on the real axis are at
 * most half an oscillation of J_n(kr rho) wide.
 */
typedef struct { double a, h, D, rho, rtol; int npoly; double atol; } path_spec;

static void integrate_path(quad_ws *w, const path_spec *ps, cplx *res)
{
    int nv = w->nv;
    cplx *acc = res;
    for (int v = 0; v < nv; ++v) acc[v] = 0;
    double a = ps->a, h = ps->h;
    double D = ps->D > 1e-9 ? ps->D : 1e-9;
    /* tail of k^n e^{-kD} beyond X is below 1e-16 of its integral once XD
     * exceeds about 40 + 2.5 n */
    double X = a + (44.0 + 2.5 * ps->npoly + 3.0 * log(1.0 + a / D)) / D;
    double wosc = ps->rho > 1e-12 ? 2.5 / ps->rho : 1e30;
    double wdec = 4.0 / D;
    double wp = wosc < wdec ? wosc : wdec;
    int nB = 2 + (int)ceil(a / (wosc < a ? wosc : a));
    int nT = (int)ceil((X - a) / wp);
    if (nT < 4) nT = 4;
    /* panel list */
    int np = 2 + nB + nT;
    cplx *pz0 = (cplx *)malloc(sizeof(cplx) * np), *pz1 = (cplx *)malloc(sizeof(cplx) * np);
    int q = 0;
    pz0[q] = 0; pz1[q] = -I * h; ++q;
    for (int j = 0; j < nB; ++j) { pz0[q] = a * j / nB - I * h; pz1[q] = a * (j + 1) / nB - I * h; ++q; }
    pz0[q] = a - I * h; pz1[q] = a; ++q;
    for (int j = 0; j < nT; ++j) { pz0[q] = a + (X - a) * j / nT; pz1[q] = a + (X - a) * (j + 1) / nT; ++q; }
    /* first pass: one GK15 per panel sets the scale */
    cplx *K = (cplx *)malloc(sizeof(cplx) * nv * np);
    cplx *G = (cplx *)malloc(sizeof(cplx) * nv);
    double *err = (double *)malloc(sizeof(double) * np * 2);
    w->kr15 = G;
    double scale = 0.0;
    for (int j = 0; j < np; ++j) {
        err[2 * j] = gk15(w, pz0[j], pz1[j], K + (size_t)j * nv, &err[2 * j + 1]);
        scale += err[2 * j + 1];
    }
    if (w->cscale) {
        /* per component: the scale is the component's own L1 integral */
        for (int v = 0; v < nv; ++v) w->cscale[v] = 0.0;
        for (int j = 0; j < np; ++j) {
            gk15(w, pz0[j], pz1[j], K, NULL);
            for (int v = 0; v < nv; ++v) w->cscale[v] += w->cmag[v];
        }
        for (int j = 0; j < np; ++j) adapt_pc(w, pz0[j], pz1[j], ps->rtol / sqrt((double)np), 0, acc);
        free(pz0); free(pz1); free(K); free(G); free(err);
        w->kr15 = NULL;
        return;
    }
    if (scale == 0.0) scale = 1e-300;
    double tol = ps->rtol * scale;
    if (tol < ps->atol) tol = ps->atol;
    for (int j = 0; j < np; ++j)
        adapt(w, pz0[j], pz1[j], tol / sqrt((double)np), 0, acc, K + (size_t)j * nv,
              err[2 * j], err[2 * j + 1]);
    free(pz0); free(pz1); free(K); free(G); free(err);
    w->kr15 = NULL;
}

static double medium_a(const or_medium *m)
{
    double km = 0;
    for (int j = 0; j <= m->L; ++j) if (cabs(m->k[j]) > km) km = cabs(m->k[j]);
    return 1.5 * km + 1.0;
}

/* decay distance of the reaction field between z (layer l) and zp (layer lp) */
static double decay_distance(const or_medium *m, int l, double z, int lp, double zp)
{
    if (l != lp) return fabs(z - zp);
    double D = 1e300;
    if (l <= m->L - 1) { double t = (z - m->d[l]) + (zp - m->d[l]); if (t < D) D = t; }
    if (l >= 1) { double t = (m->d[l - 1] - z) + (m->d[l - 1] - zp); if (t < D) D = t; }
    return D;
}

/* --------------------------------------------- reaction dyad, direct form */

typedef struct {
    const or_medium *m;
    int l, lp;
    double z, zp, rho, cphi, sphi;
    int freespace;     /* 1: integrate the free-space spectrum instead */
    cplx kfree;
} gr_ctx;

/* integrand (1/2pi) kr * <spectral dyad>_alpha, 9 entries row-major */
static void gr_integrand(cplx kr, void *vctx, cplx *out)
{
    gr_ctx *c = (gr_ctx *)vctx;
    cplx k, phi, psi, psiz, psit, psitz;
    if (c->freespace) {
        k = c->kfree;
        cplx kz = kz_of(k, kr);
        double dz = c->z - c->zp, sg = dz >= 0 ? 1.0 : -1.0;
        cplx E = cexp(I * kz * fabs(dz));
        phi = psi = -E / (2.0 * kz);
        psiz = -I * sg * E / 2.0;
        psit = -I * sg * E / 2.0;          /* -d/dzp psi */
        psitz = kz * E / 2.0;              /* -d2/dz dzp psi */
    } else {
        k = c->m->k[c->l];
        cplx a[4], b[4];
        reaction_1d(c->m, kr, 0, c->l, c->z, c->lp, c->zp, a);
        reaction_1d(c->m, kr, 1, c->l, c->z, c->lp, c->zp, b);
        phi = a[0];
        psi = b[0];
        psiz = b[1];
        psit = -b[2];
        psitz = -b[3];
    }
    cplx J[3];
    besselj_any(2, kr * c->rho, J);
    double c2 = c->cphi * c->cphi - c->sphi * c->sphi, s2 = 2.0 * c->sphi * c->cphi;
    cplx pre = -I / (k * k) * kr / (2.0 * OR_PI);
    cplx C1 = k * k * phi, C2 = kr * kr * psi, N5 = k * k * phi + psitz;
    cplx ax = -kr * J[1] * c->cphi, ay = -kr * J[1] * c->sphi;
    out[0] = pre * (C1 * J[0] - 0.5 * N5 * (J[0] - J[2] * c2));
    out[1] = pre * (0.5 * N5 * J[2] * s2);
    out[2] = pre * (psiz * ax);
    out[3] = out[1];
    out[4] = pre * (C1 * J[0] - 0.5 * N5 * (J[0] + J[2] * c2));
    out[5] = pre * (psiz * ay);
    out[6] = pre * (psit * ax);
    out[7] = pre * (psit * ay);
    out[8] = pre * (C2 * J[0]);
}

static int greact(const or_medium *m, const double *r, const double *rp, double rtol,
                  cplx G[9], long *nfev)
{
    int l = or_layer_of(m->L, m->d, r[2]), lp = or_layer_of(m->L, m->d, rp[2]);
    if (l < 0 || lp < 0) return -1;
    gr_ctx c;
    c.m = m; c.l = l; c.lp = lp; c.z = r[2]; c.zp = rp[2];
    c.freespace = 0;
    double dx = r[0] - rp[0], dy = r[1] - rp[1];
    c.rho = sqrt(dx * dx + dy * dy);
    c.cphi = c.rho > 0 ? dx / c.rho : 1.0;
    c.sphi = c.rho > 0 ? dy / c.rho : 0.0;
    if (m->L == 0) { for (int i = 0; i < 9; ++i) G[i] = 0; return 0; }
    cplx buf[9];
    quad_ws w = {gr_integrand, &c, 9, 0, buf, NULL};
    path_spec ps = {medium_a(m), 0.4, decay_distance(m, l, r[2], lp, rp[2]), c.rho, rtol, 3, 0.0};
    /* absolute floor: rtol times the size of a dyad at the decay distance D,
     * (1 + 1/(k D)^2) / (4 pi D) with the smallest layer wavenumber */
    double kmin = 1e300;
    for (int j = 0; j <= m->L; ++j) if (cabs(m->k[j]) < kmin) kmin = cabs(m->k[j]);
    ps.atol = rtol * (1.0 + 1.0 / (kmin * kmin * ps.D * ps.D)) / (4.0 * OR_PI * ps.D);
    integrate_path(&w, &ps, G);
    if (nfev) *nfev += w.nfev;
    return 0;
}

int or_greact(int L, const double *d, const double *kri, const double *r,
              const double *rp, double rtol, double *out)
{
    or_medium m;
    make_medium(&m, L, d, kri);
    cplx G[9];
    if (greact(&m, r, rp, rtol, G, NULL)) return -1;
    for (int i = 0; i < 9; ++i) { out[2 * i] = creal(G[i]); out[2 * i + 1] = cimag(G[i]); }
    return 0;
}

/* closed form (I + grad grad / k^2) e^{ikR}/(4 pi R), eq. GEandGH */
void or_gfree(double kr_, double ki_, const double *r, const double *rp, double *out)
{
    cplx k = kr_ + I * ki_;
    double R[3] = {r[0] - rp[0], r[1] - rp[1], r[2] - rp[2]};
    double Rn = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
    cplx g = cexp(I * k * Rn) / (4.0 * OR_PI * Rn);
    cplx a = 1.0 + (I * k / Rn - 1.0 / (Rn * Rn)) / (k * k);
    cplx b = (3.0 / (Rn * Rn) - 3.0 * I * k / Rn - k * k) / (k * k);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx v = g * ((i == j ? a : 0.0) + b * R[i] * R[j] / (Rn * Rn));
            out[2 * (3 * i + j)] = creal(v);
            out[2 * (3 * i + j) + 1] = cimag(v);
        }
}

/* the same free-space dyad through the spectral assembly and quadrature */
int or_gfree_spectral(double kr_, double ki_, const double *r, const double *rp,
                      double rtol, double *out)
{
    or_medium m;
    m.L = 0;
    m.k[0] = kr_ + I * ki_;
    gr_ctx c;
    c.m = &m; c.l = 0; c.lp = 0; c.z = r[2]; c.zp = rp[2];
    c.freespace = 1; c.kfree = m.k[0];
    double dx = r[0] - rp[0], dy = r[1] - rp[1];
    c.rho = sqrt(dx * dx + dy * dy);
    c.cphi = c.rho > 0 ? dx / c.rho : 1.0;
    c.sphi = c.rho > 0 ? dy / c.rho : 0.0;
    cplx buf[9], G[9];
    quad_ws w = {gr_integrand, &c, 9, 0, buf, NULL};
    path_spec ps = {medium_a(&m), 0.4, fabs(r[2] - rp[2]), c.rho, rtol, 3, 0.0};
    integrate_path(&w, &ps, G);
    for (int i = 0; i < 9; ++i) { out[2 * i] = creal(G[i]); out[2 * i + 1] = cimag(G[i]); }
    return 0;
}

/* -------------------------------------- reaction dyad, density (sigma) form */

/* G^{*star} of eq. reactcompphysicaldomain, summed over the four components,
 * with L_kappa[sigma] of eq. generalintegral reduced by Jacobi-Anger:
 * L_kappa = i^{kappa+1}/(4 pi) e^{i kappa phi} int kr J_kappa(kr rho) Z sigma dkr,
 * (rho, phi) the polar form of the horizontal part of r - rp. */
typedef struct {
    const or_medium *m;
    int l, lp, tgt_up, src_up, literal;
    double rho, zbar, zpbar, s;
} gs_ctx;

static void gs_integrand(cplx kr, void *vctx, cplx *out)
{
    gs_ctx *c = (gs_ctx *)vctx;
    cplx sg[5], J[3];
    sigmas(c->m, kr, c->l, c->lp, c->tgt_up, c->src_up, c->literal, sg);
    cplx kz = kz_of(c->m->k[c->l], kr), kzp = kz_of(c->m->k[c->lp], kr);
    cplx Z = cexp(c->s * (I * kz * c->zbar - I * kzp * c->zpbar));
    besselj_any(2, kr * c->rho, J);
    /* (sigma, |kappa|) pairs: (s1,0) (s5,0) (s2,1) (s4,1) (s3,2) */
    out[0] = kr * J[0] * Z * sg[0];
    out[1] = kr * J[0] * Z * sg[4];
    out[2] = kr * J[1] * Z * sg[1];
    out[3] = kr * J[1] * Z * sg[3];
    out[4] = kr * J[2] * Z * sg[2];
}

/* image (tau-hat) of the first slot and effective location (tau-breve) of
 * the second slot, eqs. equivalent_imag_for_source/target */
static double tau_hat_z(const or_medium *m, int l, int lp, int tgt_up, int src_up, double z)
{
    const double *d = m->d;
    if (tgt_up && src_up) return (l < lp) ? z : 2 * d[l] - z;
    if (tgt_up && !src_up) return (l <= lp) ? z : 2 * d[l] - z;
    if (!tgt_up && src_up) return (l < lp) ? 2 * d[l - 1] - z : z;
    return (l <= lp) ? 2 * d[l - 1] - z : z;
}
static double tau_breve_z(const or_medium *m, int l, int lp, int src_up, double zp)
{
    const double *d = m->d;
    if (!src_up) return (l <= lp) ? 2 * d[lp] - zp : zp;
    return (l < lp) ? zp : 2 * d[lp - 1] - zp;
}

int or_greact_sigma(int L, const double *d, const double *kri, const double *r,
                    const double *rp, double rtol, int literal, int comp_mask, double *out)
{
    or_medium m;
    make_medium(&m, L, d, kri);
    int l = or_layer_of(L, d, r[2]), lp = or_layer_of(L, d, rp[2]);
    if (l < 0 || lp < 0) return -1;
    double dx = r[0] - rp[0], dy = r[1] - rp[1];
    double rho = sqrt(dx * dx + dy * dy);
    double cph = rho > 0 ? dx / rho : 1.0, sph = rho > 0 ? dy / rho : 0.0;
    cplx G[9];
    for (int i = 0; i < 9; ++i) G[i] = 0;
    for (int tu = 1; tu >= 0; --tu)
        for (int su = 1; su >= 0; --su) {
            if (tu && l == L) continue;
            if (!tu && l == 0) continue;
            if (su && lp == 0) continue;
            if (!su && lp == L) continue;
            if (!((comp_mask >> ((tu ? 0 : 2) + (su ? 0 : 1))) & 1)) continue;
            gs_ctx c = {&m, l, lp, tu, su, literal, rho, 0, 0, s_sign(l, lp, su)};
            c.zbar = tau_hat_z(&m, l, lp, tu, su, r[2]);
            c.zpbar = tau_breve_z(&m, l, lp, su, rp[2]);
            cplx buf[5], Iv[5];
            quad_ws w = {gs_integrand, &c, 5, 0, buf, NULL};
            path_spec ps = {medium_a(&m), 0.4, c.s * (c.zbar - c.zpbar), rho, rtol, 3, 0.0};
            ps.atol = rtol * (1.0 + 1.0 / (ps.D * ps.D)) / (4.0 * OR_PI * ps.D);
            integrate_path(&w, &ps, Iv);
            cplx e1 = cph + I * sph, e2 = e1 * e1;
            cplx pre0 = I / (4 * OR_PI), pre1 = -1.0 / (4 * OR_PI), pre2 = -I / (4 * OR_PI);
            cplx L0s1 = pre0 * Iv[0], L0s5 = pre0 * Iv[1];
            cplx Lp1s2 = pre1 * e1 * Iv[2], Lm1s2 = pre1 * conj(e1) * Iv[2];
            cplx Lp1s4 = pre1 * e1 * Iv[3], Lm1s4 = pre1 * conj(e1) * Iv[3];
            cplx Lp2s3 = pre2 * e2 * Iv[4], Lm2s3 = pre2 * conj(e2) * Iv[4];
            /* M1..M6 of Section 3.1 */
            cplx M1[9] = {0.5, 0, 0, 0, 0.5, 0, 0, 0, 0};
            cplx M2[9] = {-0.25, 0.25 * I, 0, 0.25 * I, 0.25, 0, 0, 0, 0};
            cplx M3[9] = {-0.25, -0.25 * I, 0, -0.25 * I, 0.25, 0, 0, 0, 0};
            cplx M4[9] = {0, 0, 0.5, 0, 0, -0.5 * I, 0, 0, 0};
            cplx M5[9] = {0, 0, 0.5, 0, 0, 0.5 * I, 0, 0, 0};
            cplx M6[9] = {0, 0, 0, 0, 0, 0, 0, 0, 1};
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    int a = 3 * i + j, t = 3 * j + i;
                    G[a] += L0s1 * M1[a] + Lp2s3 * M2[a] + Lm2s3 * M3[a] + Lp1s2 * M4[a]
                          + Lm1s2 * M5[a] + Lp1s4 * M4[t] + Lm1s4 * M5[t] + L0s5 * M6[a];
                }
        }
    for (int i = 0; i < 9; ++i) { out[2 * i] = creal(G[i]); out[2 * i + 1] = cimag(G[i]); }
    return 0;
}

/* ------------------------------------------------------------ direct sum */

/*
 * Phi_i = sum_j G^r(r_j, r_i) q_j  (eq. allcomponents, reaction part only,
 * summed over the first slot, self term j = i included), for the targets
 * tidx[0..nt) and the sources sidx[0..ns) (sidx == NULL: all N points).
 * q and phi are interleaved complex [.][3].  Returns total integrand calls.
 */
long or_direct(int L, const double *d, const double *kri, int64_t N, const double *xyz,
               const double *q, int64_t nt, const int64_t *tidx, int64_t ns,
               const int64_t *sidx, double rtol, int nthreads, double *phi)
{
    or_medium m;
    make_medium(&m, L, d, kri);
    long total = 0;
    int64_t nsrc = sidx ? ns : N;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
#endif
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = tidx[t];
        cplx acc[3] = {0, 0, 0};
        long nf = 0;
        for (int64_t s = 0; s < nsrc; ++s) {
            int64_t j = sidx ? sidx[s] : s;
            cplx G[9];
            if (greact(&m, xyz + 3 * j, xyz + 3 * i, rtol, G, &nf)) continue;
            cplx qj[3];
            for (int c = 0; c < 3; ++c) qj[c] = q[6 * j + 2 * c] + I * q[6 * j + 2 * c + 1];
            for (int a = 0; a < 3; ++a)
                acc[a] += G[3 * a] * qj[0] + G[3 * a + 1] * qj[1] + G[3 * a + 2] * qj[2];
        }
        for (int a = 0; a < 3; ++a) {
            phi[6 * t + 2 * a] = creal(acc[a]);
            phi[6 * t + 2 * a + 1] = cimag(acc[a]);
        }
        total += nf;
    }
    return total;
}

/*
 * Free-space part of the same sum (eq. layeredmediafields): for each target
 * i, Phi^f_i = sum_j G_E^f(r_i, r_j) q_j over the sources j != i in the layer
 * of r_i, with the closed-form dyad of or_gfree at that layer's wavenumber.
 * Same argument conventions as or_direct.
 */
void or_direct_free(int L, const double *d, const double *kri, int64_t N, const double *xyz,
                    const double *q, int64_t nt, const int64_t *tidx, int64_t ns,
                    const int64_t *sidx, int nthreads, double *phi)
{
    or_medium m;
    make_medium(&m, L, d, kri);
    int64_t nsrc = sidx ? ns : N;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = tidx[t];
        int li = or_layer_of(m.L, m.d, xyz[3 * i + 2]);
        cplx acc[3] = {0, 0, 0};
        for (int64_t s = 0; s < nsrc; ++s) {
            int64_t j = sidx ? sidx[s] : s;
            if (j == i || or_layer_of(m.L, m.d, xyz[3 * j + 2]) != li) continue;
            double G[18];
            or_gfree(creal(m.k[li]), cimag(m.k[li]), xyz + 3 * i, xyz + 3 * j, G);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    cplx g = G[2 * (3 * a + b)] + I * G[2 * (3 * a + b) + 1];
                    acc[a] += g * (q[6 * j + 2 * b] + I * q[6 * j + 2 * b + 1]);
                }
        }
        for (int a = 0; a < 3; ++a) {
            phi[6 * t + 2 * a] = creal(acc[a]);
            phi[6 * t + 2 * a + 1] = cimag(acc[a]);
        }
    }
}

/* --------------------------------------------------- Legendre functions */

/* Normalised associated Legendre functions with Condon-Shortley phase,
 * P^_n^m(cos b) for 0 <= m <= n <= nmax, given cos b and sin b separately
 * (the analytic extension of Section 3.3 takes sin b = k_rho/k, cos b =
 * k_z/k).  out[(n*(n+1))/2 + m].  Textbook three-term recurrence in n. */
static void legendre(int nmax, cplx cb, cplx sb, cplx *out)
{
    for (int m = 0; m <= nmax; ++m) {
        /* P^_m^m = (-1)^m sqrt((2m+1)/(4pi) * (2m-1)!!^2/(2m)!) sin^m */
        double f = 1.0 / (4.0 * OR_PI);
        for (int i = 1; i <= m; ++i) f *= (2.0 * i - 1.0) * (2.0 * i - 1.0) / ((2.0 * i - 1.0) * (2.0 * i));
        f *= (2.0 * m + 1.0);
        cplx pmm = ((m & 1) ? -1.0 : 1.0) * sqrt(f);
        for (int i = 0; i < m; ++i) pmm *= sb;
        out[(m * (m + 1)) / 2 + m] = pmm;
        if (m + 1 > nmax) continue;
        cplx p1 = sqrt(2.0 * m + 3.0) * cb * pmm;
        out[((m + 1) * (m + 2)) / 2 + m] = p1;
        cplx p0 = pmm;
        for (int n = m + 2; n <= nmax; ++n) {
            double a = sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
            double b = sqrt((((double)n - 1) * (n - 1) - (double)m * m) / (4.0 * ((double)n - 1) * (n - 1) - 1.0));
            cplx p2 = a * (cb * p1 - b * p0);
            out[(n * (n + 1)) / 2 + m] = p2;
            p0 = p1; p1 = p2;
        }
    }
}

void or_legendre(int nmax, double cr, double ci, double sr, double si, double *out)
{
    int cnt = ((nmax + 1) * (nmax + 2)) / 2;
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * cnt);
    legendre(nmax, cr + I * ci, sr + I * si, tmp);
    for (int i = 0; i < cnt; ++i) { out[2 * i] = creal(tmp[i]); out[2 * i + 1] = cimag(tmp[i]); }
    free(tmp);
}

/* --------------------------------------------- M2L Sommerfeld integrals */

/*
 * I-hat^{nu mu}_{n m kappa}(rho, zs, zt; sigma) of eq. onedimensionintegral,
 * index convention of the M2L: (np, mp) belongs to the expansion about the
 * source centre (wavenumber k = k_l, P^(k_z/k)), (nu, mu) to the target centre
 * (k' = k_lp, P^(k'_z/k')); the Bessel order is dd = mp - mu + kappa, with
 * J_{-n} = (-1)^n J_n.  All (np,mp,nu,mu) up to p at once:
 * out[((np*np+np+mp) * P + (nu*nu+nu+mu))], P = (p+1)^2.
 * which_sigma in 1..5.
 */
typedef struct {
    const or_medium *m;
    int l, lp, tgt_up, src_up, literal, p, sig, kappa;
    double rho, zs, zt, s;
} m2l_ctx;

static void m2l_integrand(cplx kr, void *vctx, cplx *out)
{
    m2l_ctx *c = (m2l_ctx *)vctx;
    int p = c->p, P = (p + 1) * (p + 1);
    cplx sg[5];
    sigmas(c->m, kr, c->l, c->lp, c->tgt_up, c->src_up, c->literal, sg);
    cplx k = c->m->k[c->l], kp = c->m->k[c->lp];
    cplx kz = kz_of(k, kr), kzp = kz_of(kp, kr);
    cplx Z = cexp(c->s * (I * kz * c->zs - I * kzp * c->zt));
    cplx base = kr * Z * sg[c->sig - 1];
    int nj = 2 * p + 2;
    cplx J[64];
    besselj_any(nj, kr * c->rho, J);
    int cnt = ((p + 1) * (p + 2)) / 2;
    cplx Ps[2048], Pt[2048];
    legendre(p, kz / k, kr / k, Ps);
    legendre(p, kzp / kp, kr / kp, Pt);
    for (int np = 0; np <= p; ++np)
        for (int mp = -np; mp <= np; ++mp) {
            int am = mp < 0 ? -mp : mp;
            cplx ps = Ps[(np * (np + 1)) / 2 + am] * ((mp < 0 && (am & 1)) ? -1.0 : 1.0);
            for (int nu = 0; nu <= p; ++nu)
                for (int mu = -nu; mu <= nu; ++mu) {
                    int an = mu < 0 ? -mu : mu;
                    cplx pt = Pt[(nu * (nu + 1)) / 2 + an] * ((mu < 0 && (an & 1)) ? -1.0 : 1.0);
                    int dd = mp - mu + c->kappa;
                    int ad = dd < 0 ? -dd : dd;
                    cplx jd = J[ad] * ((dd < 0 && (ad & 1)) ? -1.0 : 1.0);
                    out[(np * np + np + mp) * P + (nu * nu + nu + mu)] = base * jd * ps * pt;
                }
        }
    (void)cnt;
}

int or_m2l_table(int L, const double *d, const double *kri, int l, int lp, int tgt_up,
                 int src_up, int literal, int sig, int kappa, int p, double rho,
                 double zs, double zt, double rtol, double *out)
{
    or_medium m;
    make_medium(&m, L, d, kri);
    int P = (p + 1) * (p + 1);
    if (P * P > OR_MAXV || p > 40) return -2;
    m2l_ctx c = {&m, l, lp, tgt_up, src_up, literal, p, sig, kappa, rho, zs, zt,
                 s_sign(l, lp, src_up)};
    double D = c.s * (zs - zt);
    if (D <= 0) return -1;
    cplx *buf = (cplx *)malloc(sizeof(cplx) * P * P);
    cplx *res = (cplx *)malloc(sizeof(cplx) * P * P);
    /* every entry is its own Sommerfeld integral: each meets rtol relative to
     * its own magnitude (entries of low and high degree differ by many orders) */
    double *ce = (double *)malloc(sizeof(double) * 3 * P * P);
    quad_ws w = {m2l_integrand, &c, P * P, 0, buf, NULL, ce, ce + P * P, ce + 2 * P * P};
    path_spec ps = {medium_a(&m), 0.4, D, rho, rtol, 2 * p + 3, 0.0};
    integrate_path(&w, &ps, res);
    free(ce);
    for (int i = 0; i < P * P; ++i) { out[2 * i] = creal(res[i]); out[2 * i + 1] = cimag(res[i]); }
    free(buf); free(res);
    return 0;
}
