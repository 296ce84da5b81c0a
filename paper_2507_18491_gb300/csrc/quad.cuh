// k_rho quadrature rule shared by the M2L tabulation and the near field.
#pragma once
#include "kernels.cuh"

namespace lmf {

// Plan of one Sommerfeld integral int_0^inf k f(k) J_d(k rho) dk (Section 3.5):
// Gamma_1 from 0 to a below the real axis; the real axis up to x1; and, when
// rho > dz (oscillation dominates decay), the split 2 J = H^(1) + H^(2) onto
// the rays Gamma_2+- from x1 with direction (dz +- i rho)/r, along which the
// integrand decays like e^{-t r} without oscillating.  x1 >= 20/rho keeps the
// Hankel functions in their large-argument regime; deg is the polynomial
// degree of f (it sets how far the decay must be followed).
// allow_split = false keeps the real axis (needed when one plan serves many
// horizontal distances, some of them near zero).
__host__ __device__ inline QuadPlanDev make_plan(double a, double rho, double dz, int deg,
                                                 bool allow_split = true)
{
    QuadPlanDev pl{};
    pl.a = a;
    pl.kp = 0.5 * a;
    int np1 = 4 + (int)ceil(a * rho / 3.0);
    pl.n1 = 16 * np1;
    double U = 40.0 + 2.5 * deg + 3.0 * log(1.0 + a / dz);
    double w = 2.0 / dz;
    if (rho > 0) w = fmin(w, 2.0 / rho);
    if (allow_split && rho > dz) {
        pl.x1 = fmax(a, 20.0 / rho);
        pl.nmid = pl.x1 > a ? 8 * (int)ceil((pl.x1 - a) / w) : 0;
        double r = sqrt(rho * rho + dz * dz);
        pl.cr = dz / r;
        pl.sr = rho / r;
        pl.tend = (U + deg) / r;
        pl.nray = 8 * (int)ceil(pl.tend * r / 2.0);
    } else {
        pl.x1 = a + U / dz;
        pl.nmid = 8 * (int)ceil((pl.x1 - a) / w);
        if (pl.nmid < 16) pl.nmid = 16;
        pl.nray = 0;
        pl.cr = 1.0;
        pl.sr = 0.0;
        pl.tend = 0.0;
    }
    return pl;
}

__host__ __device__ inline int plan_nodes(const QuadPlanDev &pl) { return pl.n1 + pl.nmid + 2 * pl.nray; }

// k_rho node q of a plan (see QuadPlanDev).  Returns the node, its weight
// including the k_rho dk_rho factor of the integrand, and the Bessel kind:
// 0 = J_d, 1 = H^(1)_d / 2 (ray Gamma_2+), 2 = H^(2)_d / 2 (ray Gamma_2-).
// Gamma_1: k(t) = sqrt(2 kp a u t - a^2 u^2 t^2), u = kp/a - i sqrt(1 - (kp/a)^2),
// so that k dk/dt = kp a u - a^2 u^2 t.
__device__ inline int plan_node(const QuadPlanDev &pl, int q, cd &kr, cd &w)
{
    if (q < pl.n1) {
        int panel = q / 16, j = q % 16;
        int np1 = pl.n1 / 16;
        double t0 = (double)panel / np1, t1 = (double)(panel + 1) / np1;
        double t = 0.5 * (t0 + t1) + 0.5 * (t1 - t0) * c_gl16x[j];
        double wt = 0.5 * (t1 - t0) * c_gl16w[j];
        double cth = pl.kp / pl.a;
        cd u = {cth, -sqrt(fmax(0.0, 1.0 - cth * cth))};
        cd au = pl.a * u;
        cd k2 = (2.0 * pl.kp * t) * au - (t * t) * (au * au);
        kr = csqrtd(k2);
        w = wt * (pl.kp * au - t * (au * au));
        return 0;
    }
    q -= pl.n1;
    if (q < pl.nmid) {
        int panel = q / 8, j = q % 8;
        double h = (pl.x1 - pl.a) / (pl.nmid / 8);
        double x = pl.a + panel * h + 0.5 * h * (1.0 + c_gl8x[j]);
        kr = mkd(x);
        w = mkd(0.5 * h * c_gl8w[j] * x);
        return 0;
    }
    q -= pl.nmid;
    int kind = 1;
    if (q >= pl.nray) { q -= pl.nray; kind = 2; }
    int panel = q / 8, j = q % 8;
    double h = pl.tend / (pl.nray / 8);
    double t = panel * h + 0.5 * h * (1.0 + c_gl8x[j]);
    cd dir = {pl.cr, kind == 1 ? pl.sr : -pl.sr};
    kr = mkd(pl.x1) + t * dir;
    w = (0.5 * h * c_gl8w[j]) * (kr * dir);
    return kind;
}

}  // namespace lmf
