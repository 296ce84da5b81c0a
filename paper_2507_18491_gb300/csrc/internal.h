// Internal declarations shared by the host setup code and the CUDA kernels.
#pragma once
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lmfmm.h"
#include "cx.cuh"
#include "medium.cuh"

namespace lmf {

using zc = std::complex<double>;

inline int nidx(int n, int m) { return n * n + n + m; }        // (n, m) -> 0..P-1
inline int tidx(int n, int m) { return (n * (n + 1)) / 2 + m; }  // (n, |m|) triangle

// Helical components (a, b, c) = (q_x + i q_y, q_x - i q_y, q_z).
constexpr int NTAB = 5;   // (s1,0) (s5,0) (s2,1) (s4,1) (s3,2)

struct Box {
    uint64_t key;       // Morton key at its level
    int level, layer;
    int64_t p0, p1;     // point range in sorted order
    int64_t parent;     // -1 at the root
    int64_t child0;     // first child (children are contiguous), -1 at leaves
    int nchild;
    int ix, iy, iz;     // integer coordinates at its level
    double c[3];        // centre (natural coordinates)
    double r;           // max distance of its points from c
};

struct Geom {           // one distinct M2L table
    int comp, level;
    double rho, zs, zt; // mapped centre heights
    int64_t pair0, pair1;
};

struct M2LPair {        // device-side record
    int64_t src, tgt;   // box indices
    double cphi, sphi;  // direction of (c_s - c_t) in the horizontal plane
};

struct NearPair {       // device-side record
    int comp;
    int pad;
    int64_t src, tgt;   // leaf boxes
    int64_t coef0;      // offset of its point-pair coefficients (5 per pair)
    double dzmin, rhomax;
};

struct TransGroup {     // one M2M/L2L translation matrix and the box pairs using it
    int layer, level, octant;
    double t[3];        // child centre - parent centre
    int64_t pair0, pair1;
};

// k_rho quadrature plan of one tabulated geometry (or near pair)
struct QuadPlan {
    int n1;             // nodes on Gamma_1
    int ntail;          // nodes on the real tail
    double a, kp;       // Gamma_1 end point and shape parameter
    double xend;        // tail end
};

}  // namespace lmf

struct lmfmm_ctx {
    int device = 0;
    lmfmm_params prm{};
    std::string err;
    bool layers_set = false, points_set = false, built = false;

    // medium
    MediumDev med{};
    // points
    int64_t N = 0;
    std::vector<double> xyz;          // original order
    std::vector<int> layer;           // per original point
    std::vector<int64_t> perm;        // sorted -> original
    std::vector<double> sxyz;         // sorted, [N][3]
    // tree
    int depth = 0;
    double root_c[3]{}, root_h = 0;
    std::vector<lmf::Box> boxes;
    std::vector<std::vector<int64_t>> lvl0, lvl1;   // [layer][level] box ranges
    // components: the reaction components (l, l', *, star) first, then (free-space
    // part requested) one free-space pseudo-component per layer with points
    std::vector<CompDev> comps;
    int n_react_comps = 0;
    // far field: reaction geometries first, then the free-space ones
    std::vector<lmf::Geom> geoms;
    size_t n_react_geoms = 0;
    std::vector<lmf::M2LPair> m2l;                  // grouped by geometry
    std::vector<cd> free_tables;                    // [free geometry][5][P][P], unscaled
    std::vector<std::pair<int64_t, int64_t>> free_near;   // (source leaf, target leaf), same layer
    int64_t n_free_pp = 0;
    std::vector<lmf::NearPair> near;
    int64_t n_near_pp = 0;
    std::vector<lmf::TransGroup> tgroups;
    std::vector<int64_t> tpair_child, tpair_parent; // per TransGroup pair
    // Chebyshev tables
    std::vector<double> Bcoef;        // B^k_{n,|m|}, [tidx][KMAX+1]
    int KMAX = 0;
    std::vector<int> comp_gidx;       // component -> G tensor index
    std::vector<cd> Gten;             // per distinct (l, lp): [T][T][LMAX] (T = #triangle)
    int LMAXC = 0;

    // device memory
    void *d_xyz = nullptr, *d_perm = nullptr, *d_box = nullptr;
    void *d_q = nullptr, *d_phi = nullptr;            // helical, sorted
    void *d_me = nullptr, *d_le = nullptr;            // [nbox][3][P]
    void *d_tup = nullptr, *d_tdn = nullptr;          // translation matrices [ngroup][P][P]
    void *d_tpair = nullptr;                          // (child, parent) pairs
    void *d_tab = nullptr;                            // M2L tables [ngeom][5][P][P]
    void *d_m2l = nullptr, *d_geom = nullptr;
    void *d_near = nullptr, *d_s2t = nullptr;
    void *d_comps = nullptr, *d_B = nullptr, *d_G = nullptr;
    void *d_work = nullptr;                           // m2l work items
    int64_t n_work = 0;
    void *d_flag = nullptr;                           // device error flag
    void *d_tmp = nullptr;                            // J/Phi staging for host matvec
    std::vector<void *> allocs;

    lmfmm_stats stats{};
    void *dev = nullptr;      // device state (api.cu)
};

namespace lmf {
// End point a of the contour Gamma_1 (Section 3.5): beyond every layer wavenumber.
inline double medium_a(const MediumDev &M)
{
    double km = 0;
    for (int j = 0; j <= M.L; ++j) km = std::max(km, std::hypot(M.k[j].x, M.k[j].y));
    return 1.5 * km + 0.75;
}

// host_setup.cpp
lmfmm_status build_host_structures(lmfmm_ctx *ctx);
// Free-space part: same-layer dual traversal into far and near pairs, free
// geometries appended to ctx->geoms / ctx->m2l, their tables into free_tables.
lmfmm_status build_free_structures(lmfmm_ctx *ctx);
// The five tables (kernel convention of the reaction M2L, phases factored out)
// of the free-space M2L between two boxes with c_s - c_t = (rho, 0, dz): the
// singular-to-regular translation composed with (I + grad grad / k^2), times
// ik / (4 pi) (eqs. freespace3dmulexpscaled, maxwell_M2L_freespace); out5
// [5][P][P]; blocks9 (optional) [3 out][3 in][P][P] the full helical operator.
void free_m2l_tables(int p, zc k, double rho, double dz, cd *out5, cd *blocks9);
// Every (component, source leaf, target leaf) pair of the context as a near
// pair (the all-pairs direct evaluation), written to out[0 .. cap); returns the
// number of pairs, or -1 if there are more than cap (nothing past cap is
// written).  *npp receives the point-pair count, the pairs' coefficient
// offsets (coef0) run over it.
int64_t all_leaf_pairs(const lmfmm_ctx *ctx, NearPair *out, int64_t cap, int64_t *npp);
void chebyshev_tables(lmfmm_ctx *ctx);
void bcoef_table(int p, int KMAX, std::vector<double> &B);
void gtensor(int p, const std::vector<double> &Bcoef, int KM, zc k, zc kp, cd *dst);
lmfmm_status classify_and_sort(lmfmm_ctx *ctx);
void gaunt_table(int p, std::vector<int64_t> &off, std::vector<int> &lval, std::vector<double> &gval);
void translation_matrix(int p, zc k, const double t[3], const std::vector<int64_t> &off,
                        const std::vector<int> &lval, const std::vector<double> &gval, cd *up,
                        cd *dn);
}  // namespace lmf
