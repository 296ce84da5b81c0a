// Layered medium on the device: density functions of the reaction
// components (eq. threedensity) by generalized reflection/transmission
// recurrences, the sigma densities of Section 3.1, image maps and signs.
#pragma once
#include "cx.cuh"

#define LMF_MAXL 8   // at most 8 interfaces (9 layers)

struct MediumDev {
    int L;                    // number of interfaces
    double d[LMF_MAXL];       // interface heights, decreasing
    cd k[LMF_MAXL + 1];       // layer wavenumbers (omega = mu = 1, eps = k^2)
};

// One reaction component (l, lp, *, star): l = layer of the first Green's
// function slot (the summed points), lp = layer of the second slot (the
// evaluation points); tu = (* == up) at the first slot, su = (star == up).
struct CompDev {
    int l, lp, tu, su;
    double s;                 // s^{* star}_{l lp}, eq. eq_signs
    double refl_src;          // image map of the first slot: z -> 2*refl_src - z if has_src_refl
    double refl_tgt;          // effective map of the second slot
    int has_src_refl, has_tgt_refl;
};

__host__ __device__ inline double comp_sign(int l, int lp, int su)
{
    return su ? (l < lp ? 1.0 : -1.0) : (l <= lp ? 1.0 : -1.0);
}

// Densities phi^{*star}_{l lp}(kr) (w = 0) and psi^{*star}_{l lp}(kr) (w = 1),
// order (up,up), (up,dn), (dn,up), (dn,dn), normalised as in eq.
// threedensity so that the reaction part of the scalar Green's function is
// -1/(2 k_{lp z}) sum u^{*star} Z^{*star} (omega = mu = 1).
//
// Waves in layer j: Y_j = k_jz / eta_j with eta = 1 (phi: u' continuous) or
// eps_j = k_j^2 (psi: u'/eps continuous); Fresnel R(i,j) = (Y_i - Y_j)/(Y_i + Y_j)
// for a wave in layer i meeting layer j, transmission 1 + R(i,j).  Rdn[j]
// (Rup[j]) is the generalized reflection seen by a down- (up-) going wave in
// layer j from everything below (above).  In the source layer the two bounce
// series sum to 1/(1 - Rdn Rup e^2).  Across layers the amplitude picks up
// T/(1 - R Rgen e^2) per interface; the exponential of the straight vertical
// path is carried by Z^{*star}, the rest by a single exponential P of the
// phase left over, which stays bounded as kr -> infinity.
__device__ inline void densities_dev(const MediumDev &M, cd kr, int l, int lp, int w, cd out[4])
{
    const int L = M.L;
    cd kz[LMF_MAXL + 1], Y[LMF_MAXL + 1], e[LMF_MAXL + 1];
    cd Rdn[LMF_MAXL + 1], Rup[LMF_MAXL + 1];
    for (int j = 0; j <= L; ++j) {
        kz[j] = kz_of(M.k[j], kr);
        Y[j] = w ? kz[j] / (M.k[j] * M.k[j]) : kz[j];
        e[j] = (j >= 1 && j <= L - 1) ? cexpd(mul_i(kz[j] * (M.d[j - 1] - M.d[j]))) : mkd(0.0);
    }
    auto R = [&](int i, int j) { return (Y[i] - Y[j]) / (Y[i] + Y[j]); };
    Rdn[L] = mkd(0.0);
    for (int j = L - 1; j >= 0; --j) {
        cd r = R(j, j + 1);
        cd g = Rdn[j + 1] * e[j + 1] * e[j + 1];
        Rdn[j] = (r + g) / (mkd(1.0) + r * g);
    }
    Rup[0] = mkd(0.0);
    for (int j = 1; j <= L; ++j) {
        cd r = R(j, j - 1);
        cd g = Rup[j - 1] * e[j - 1] * e[j - 1];
        Rup[j] = (r + g) / (mkd(1.0) + r * g);
    }
    cd Rd = Rdn[lp], Ru = Rup[lp], ep = e[lp];
    cd Mi = inv(mkd(1.0) - Rd * Ru * ep * ep);
    if (l == lp) {
        out[0] = Rd * Ru * Mi;
        out[1] = Rd * Mi;
        out[2] = Ru * Mi;
        out[3] = Rd * Ru * Mi;
        return;
    }
    cd Tb = mkd(1.0), ph = mkd(0.0);
    if (l < lp) {
        // up through interfaces lp-1 .. l
        for (int j = lp - 1; j >= l; --j) {
            cd T = mkd(1.0) + R(j + 1, j);
            cd den = mkd(1.0) - R(j, j + 1) * Rup[j] * e[j] * e[j];
            Tb = Tb * T / den;
            if (j > l) ph += kz[j] * (M.d[j - 1] - M.d[j]);
        }
        ph += kz[lp] * M.d[lp - 1] - kz[l] * M.d[l];
        cd base = Tb * Mi * cexpd(mul_i(ph));
        out[0] = base;
        out[1] = Rd * base;
        out[2] = Rup[l] * base;
        out[3] = Rup[l] * Rd * base;
    } else {
        // down through interfaces lp .. l-1
        for (int j = lp + 1; j <= l; ++j) {
            cd T = mkd(1.0) + R(j - 1, j);
            cd den = mkd(1.0) - R(j, j - 1) * Rdn[j] * e[j] * e[j];
            Tb = Tb * T / den;
            if (j < l) ph += kz[j] * (M.d[j - 1] - M.d[j]);
        }
        ph += kz[l] * M.d[l - 1] - kz[lp] * M.d[lp];
        cd base = Tb * Mi * cexpd(mul_i(ph));
        out[3] = base;
        out[2] = Ru * base;
        out[1] = Rdn[l] * base;
        out[0] = Rdn[l] * Ru * base;
    }
}

// sigma_1..sigma_5 of Section 3.1 for component (l, lp, tu, su), gamma =
// 1/k_l^2 (mu = 1).  The psi-term of sigma_1 and sigma_3 carries
// eps = s_t * s_s (s_t = +1 for * = up, s_s = +1 for star = down): the
// printed sigma_3 ties the sign to star alone, which does not reproduce the
// Theta matrices when * = down; this reading does (checked against the
// direct assembly of eq. eq-GEGH-b-latest).
__device__ inline void sigmas_dev(const MediumDev &M, cd kr, int l, int lp, int tu, int su,
                                  cd sg[5])
{
    cd ph[4], ps[4];
    densities_dev(M, kr, l, lp, 0, ph);
    densities_dev(M, kr, l, lp, 1, ps);
    int c = (tu ? 0 : 2) + (su ? 0 : 1);
    cd kzl = kz_of(M.k[l], kr), kzp = kz_of(M.k[lp], kr);
    cd gam = inv(M.k[l] * M.k[l]);
    double st = tu ? 1.0 : -1.0, ss = su ? -1.0 : 1.0, eps = st * ss;
    cd ikzp = inv(kzp);
    cd gps = gam * ps[c];
    sg[0] = ph[c] * ikzp - eps * (kzl * gps);
    sg[1] = -st * (kr * kzl * gps * ikzp);
    sg[2] = ph[c] * ikzp + eps * (kzl * gps);
    sg[3] = ss * (kr * gps);
    sg[4] = kr * kr * gps * ikzp;
}

// image (first slot, layer l) and effective (second slot, layer lp) heights,
// eqs. equivalent_imag_for_source / equivalent_imag_for_target
__host__ __device__ inline double comp_src_z(const CompDev &c, double z)
{
    return c.has_src_refl ? 2.0 * c.refl_src - z : z;
}
__host__ __device__ inline double comp_tgt_z(const CompDev &c, double z)
{
    return c.has_tgt_refl ? 2.0 * c.refl_tgt - z : z;
}
