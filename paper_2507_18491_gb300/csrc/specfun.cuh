// Device special functions: cylindrical Bessel J_n and spherical Bessel j_n
// of complex argument, normalised associated Legendre functions.
#pragma once
#include "cx.cuh"

#define LMF_PI 3.14159265358979323846

// Hankel's large-argument expansion (DLMF 10.17.3) for J_0 and J_1:
// J_nu(z) = sqrt(2/(pi z)) (P cos w - Q sin w),  w = z - nu pi/2 - pi/4,
// P = sum_k (-1)^k a_2k(nu) z^-2k, Q = sum_k (-1)^k a_2k+1(nu) z^-(2k+1),
// a_k(nu) = prod_{j=1..k} (4 nu^2 - (2j-1)^2) / (k! 8^k).
// Used for |z| >= 35, where 20 terms reach double precision.
__device__ inline void bessel_j01_asym(cd z, cd &J0, cd &J1)
{
    cd iz = inv(z);
    cd out[2];
    for (int nu = 0; nu <= 1; ++nu) {
        double mu = 4.0 * nu * nu;
        cd P = mkd(1.0), Q = mkd(0.0);
        cd term = mkd(1.0);   // a_k z^-k with alternating sign folded in below
        double ak = 1.0;
        cd zk = mkd(1.0);
        for (int k = 1; k <= 24; ++k) {
            ak *= (mu - (2.0 * k - 1.0) * (2.0 * k - 1.0)) / (k * 8.0);
            zk = zk * iz;
            term = ak * zk;
            if (k & 1) {
                // odd k = 2j+1 -> Q, sign (-1)^j
                int j = (k - 1) / 2;
                if (j & 1) Q -= term; else Q += term;
            } else {
                int j = k / 2;
                if (j & 1) P -= term; else P += term;
            }
            if (abs2(term) < 1e-36) break;
        }
        cd w = z - mkd(nu * 0.5 * LMF_PI + 0.25 * LMF_PI);
        // cos w, sin w for complex w
        double s, c;
        sincos(w.x, &s, &c);
        double ch = cosh(w.y), sh = sinh(w.y);
        cd cw = {c * ch, -s * sh}, sw = {s * ch, c * sh};
        cd pre = csqrtd(mkd(2.0 / LMF_PI) * iz);
        out[nu] = pre * (P * cw - Q * sw);
    }
    J0 = out[0];
    J1 = out[1];
}

// H^(1)_0..H^(1)_D at complex z with |z| >= 20 and 0 <= arg z <= pi/2:
// Hankel's expansion (DLMF 10.17.5)
//   H^(1)_nu(z) = sqrt(2/(pi z)) e^{i w} sum_k i^k a_k(nu) z^-k,  w = z - nu pi/2 - pi/4,
// for nu = 0, 1 (its terms keep decreasing up to k ~ 2|z|, so 40 terms reach
// double precision), then upward recurrence, which is stable for the
// dominant Hankel solution.
__device__ inline void hankel1_seq(cd z, int D, cd *H)
{
    cd iz = inv(z);
    for (int nu = 0; nu <= 1 && nu <= D; ++nu) {
        double mu = 4.0 * nu * nu;
        cd sum = mkd(1.0), zk = mkd(1.0);
        double ak = 1.0, prev = 1e300;
        for (int k = 1; k <= 48; ++k) {
            ak *= (mu - (2.0 * k - 1.0) * (2.0 * k - 1.0)) / (k * 8.0);
            zk = zk * iz;
            cd term = ipow<double>(k) * (ak * zk);
            double m = abs2(term);
            if (m > prev) break;
            prev = m;
            sum += term;
            if (m < 1e-36 * abs2(sum)) break;
        }
        cd w = z - mkd(nu * 0.5 * LMF_PI + 0.25 * LMF_PI);
        cd pre = csqrtd(mkd(2.0 / LMF_PI) * iz);
        H[nu] = pre * cexpd(mul_i(w)) * sum;
    }
    cd iz2 = 2.0 * iz;
    for (int n = 1; n < D; ++n) H[n + 1] = (double)n * iz2 * H[n] - H[n - 1];
}

// J_0..J_D at complex z (Im z may have either sign).  Miller's backward
// recurrence J_{n-1} = (2n/z) J_n - J_{n+1}, normalised with the
// Jacobi-Anger sum e^{iz} = J_0 + 2 sum i^n J_n (Im z <= 0) or
// e^{-iz} = J_0 + 2 sum (-i)^n J_n (Im z > 0), whichever target has modulus
// >= 1 so that the sum does not cancel.  For |z| >= max(35, D + 12) the
// Hankel expansion of J_0, J_1 and upward recurrence (stable for n < |z|).
// Returns 0, or 1 if the recurrence start was capped.
template <int DMAX>
__device__ inline int bessel_j_seq(cd z, int D, cd *J)
{
    double az = cabsd(z);
    if (az < 1e-300) {
        J[0] = mkd(1.0);
        for (int n = 1; n <= D; ++n) J[n] = mkd(0.0);
        return 0;
    }
    double zthr = fmax(35.0, D + 12.0);
    if (az >= zthr) {
        bessel_j01_asym(z, J[0], J[1]);
        cd iz2 = mkd(2.0) * inv(z);
        for (int n = 1; n < D; ++n) J[n + 1] = (double)n * iz2 * J[n] - J[n - 1];
        return 0;
    }
    int N = D + (int)az + 26;
    int capped = 0;
    if (N > 400) { N = 400; capped = 1; }
    cd iz2 = mkd(2.0) * inv(z);
    bool lower = (z.y <= 0.0);  // use e^{iz}
    cd fnp1 = mkd(0.0), fn = mkd(1e-30);
    cd S = mkd(0.0);
    for (int n = 0; n <= D; ++n) J[n] = mkd(0.0);
    // S accumulates 2 * (+-i)^n f_n for n >= 1 and f_0 at the end
    for (int n = N; n >= 1; --n) {
        // store f_n
        if (n <= D) J[n] = fn;
        cd ph = lower ? ipow<double>(n) : ipow<double>(-n);
        S += 2.0 * (ph * fn);
        cd fnm1 = (double)n * iz2 * fn - fnp1;
        fnp1 = fn;
        fn = fnm1;
        double m = fmax(fabs(fn.x), fabs(fn.y));
        if (m > 1e250) {
            const double sc = 1e-250;
            fn = sc * fn;
            fnp1 = sc * fnp1;
            S = sc * S;
            for (int k = n; k <= D; ++k) J[k] = sc * J[k];
        }
    }
    J[0] = fn;
    S += fn;
    cd target = lower ? cexpd(mul_i(z)) : cexpd(mul_mi(z));
    cd scale = target / S;
    for (int n = 0; n <= D; ++n) J[n] = J[n] * scale;
    return capped;
}

// Spherical Bessel j_0..j_n at complex z by Miller's backward recurrence
// j_{k-1} = ((2k+1)/z) j_k - j_{k+1}, normalised against whichever of
// j_0 = sin z / z and j_1 = sin z / z^2 - cos z / z is larger.
__device__ inline void sph_bessel_seq(cd z, int n, cd *j)
{
    double az = cabsd(z);
    if (az < 1e-14) {
        j[0] = mkd(1.0);
        for (int k = 1; k <= n; ++k) j[k] = mkd(0.0);
        return;
    }
    int N = n + 18 + (int)(1.5 * az);
    cd iz = inv(z);
    cd fnp1 = mkd(0.0), fn = mkd(1e-30);
    for (int k = 0; k <= n; ++k) j[k] = mkd(0.0);
    cd f1 = mkd(0.0);
    for (int k = N; k >= 1; --k) {
        if (k <= n) j[k] = fn;
        if (k == 1) f1 = fn;
        cd fkm1 = (double)(2 * k + 1) * iz * fn - fnp1;
        fnp1 = fn;
        fn = fkm1;
        double m = fmax(fabs(fn.x), fabs(fn.y));
        if (m > 1e250) {
            const double sc = 1e-250;
            fn = sc * fn;
            fnp1 = sc * fnp1;
            f1 = sc * f1;
            for (int q = k; q <= n; ++q) j[q] = sc * j[q];
        }
    }
    j[0] = fn;
    // sin z, cos z
    double s, c;
    sincos(z.x, &s, &c);
    double ch = cosh(z.y), sh = sinh(z.y);
    cd sz = {s * ch, c * sh}, cz = {c * ch, -s * sh};
    cd j0 = sz * iz;
    cd j1 = sz * iz * iz - cz * iz;
    cd scale = (abs2(j0) >= abs2(j1)) ? j0 / fn : j1 / f1;
    for (int k = 0; k <= n; ++k) j[k] = j[k] * scale;
}

// Normalised associated Legendre functions with Condon-Shortley phase,
// P^_n^m(x) = sqrt((2n+1)/(4 pi) (n-m)!/(n+m)!) P_n^m(x), x = cos(theta),
// s = sin(theta) >= 0; writes P[n*(n+1)/2 + m] for 0 <= m <= n <= p.
template <typename T>
__device__ inline void legendre_norm(int p, T x, T s, T *P)
{
    T pmm = T(0.28209479177387814347);  // 1/sqrt(4 pi)
    for (int m = 0; m <= p; ++m) {
        if (m > 0) pmm = -pmm * s * sqrt(T(2 * m + 1) / T(2 * m));
        P[(m * (m + 1)) / 2 + m] = pmm;
        if (m == p) break;
        T p1 = sqrt(T(2 * m + 3)) * x * pmm;
        P[((m + 1) * (m + 2)) / 2 + m] = p1;
        T p0 = pmm;
        for (int n = m + 2; n <= p; ++n) {
            T a = sqrt(T(4 * n * n - 1) / T(n * n - m * m));
            T b = sqrt(T((n - 1) * (n - 1) - m * m) / T(4 * (n - 1) * (n - 1) - 1));
            T p2 = a * (x * p1 - b * p0);
            P[(n * (n + 1)) / 2 + m] = p2;
            p0 = p1;
            p1 = p2;
        }
    }
}
