// Device-side records and kernel launchers.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "gauss.cuh"
#include "internal.h"

#define LMF_PMAX 20

namespace lmf {

// k_rho nodes of one Sommerfeld integral (Section 3.5):
//   [0, n1)                Gamma_1 from 0 to a (Gauss-Legendre 16 per panel)
//   [n1, n1+nmid)          real segment [a, x1] with J_d (Gauss-Legendre 8)
//   then, when nray > 0, the rays Gamma_2+ and Gamma_2- from x1,
//   k = x1 + t (dz +- i rho)/r, t in [0, tend], with H^(1)_d/2 and H^(2)_d/2.
struct QuadPlanDev {
    int n1, nmid, nray, pad;
    double a, kp, x1;   // Gamma_1 end, its shape parameter, end of the real segment
    double cr, sr, tend;// ray direction (dz/r, rho/r) and length
};

struct GeomDev {
    int comp, src_primary;
    double rho, zs, zt;
    double scale_s, scale_t;  // |k| S_level of the source and target layers
    QuadPlanDev plan;
    int64_t node0;      // first node within its tabulation batch
    int64_t stride;     // node count of its batch (factor-array stride)
    int64_t tab_index;  // table slot
    int batch, pad;
};

struct LayerScale {      // |k_l| S_leaf per layer (expansion scaling at the leaves)
    double s[LMF_MAXL + 1];
};

struct TransGroupDev {
    int layer, level;
    double t[3];
};

struct BoxDev {
    int64_t p0, p1;
    double c[3];
    int layer, pad;
};

struct LeafUnit {       // P2M work of one warp: points [i0, i1) (at most 128) of leaf box
    int64_t i0, i1;
    int box, whole;     // whole: the unit covers the leaf (plain stores, else atomics)
};


struct GemmWork {       // M2M / L2L: pairs [pair0, pair0 + npair) of one translation group
    int group, npair;
    int64_t pair0;
};

struct M2LWork {        // one M2L table applied to a chunk of pairs of one geometry
    int geom, t, npair;
    int flags;          // bit 0: odd input degrees change sign, bit 1: odd output degrees
    int64_t pair0;
    int prob, pad;      // problem of a batched launch (TcProb index), else 0
};

// per-problem arrays of a batched persistent M2L launch (k_m2l_tc2): one
// problem's geometries, pairs, pair phases, table image and scales, and its
// multipole / local expansions
struct TcProb {
    const GeomDev *geoms;
    const M2LPair *pairs;
    const cf *ephase;
    const void *img;
    const cf *me;
    cf *le;
};

// k_tab.cu
void launch_densities(const MediumDev &M, int l, int lp, int64_t n, const cd *kr, cd *out,
                      cudaStream_t st);
void launch_tab_batch(const GeomDev *dG, int g0, int nb, int qmax, const MediumDev &M,
                      const CompDev *dcomps, int p, const cd *dGten, const int *dcgidx,
                      cd *scratch, int64_t stride, cd *tab, int *dflag, cudaStream_t st);

// k_fmm.cu
cudaError_t configure_fmm_kernels();
cudaError_t configure_tab_kernels();
// J / Phi: caller's [N][3] complex128 (LMFMM_C128) or complex64 (LMFMM_C64)
void launch_gather_in(int64_t N, const int64_t *perm, const void *J, int dtype, cd *qh, bool conj_in,
                      cudaStream_t st);
void launch_scatter_out(int64_t N, const int64_t *perm, const cd *phih, void *Phi, int dtype, bool conj_out,
                        cudaStream_t st);
// P2M of the helical charges qh into me at the leaves; with l2p_basis the
// coefficients are taken against L2P's functions instead (transpose of L2P)
template <typename T>
void launch_p2m(int p, int64_t nleaf, const int64_t *leaves, const BoxDev *boxes,
                const double *xyz, const cd *qh, const MediumDev &M, const LayerScale &ls,
                cx<T> *me, cudaStream_t st, bool l2p_basis = false);
// L2P of le at the leaf points into phih; with p2m_basis the expansions are
// evaluated with P2M's functions (transpose of P2M); accumulate adds into phih
template <typename T>
void launch_l2p(int p, int64_t nleaf, const int64_t *leaves, const BoxDev *boxes,
                const double *xyz, const cx<T> *le, const MediumDev &M, const LayerScale &ls,
                cd *phih, cudaStream_t st, bool p2m_basis = false, bool accumulate = false);

// k_leaf.cu: P2M and L2P of the mixed form for p <= 15 (FP32 expansions), one thread per
// sorted point (pt_box: its leaf box): ph (cd [N][3]) = the expansions le (cf
// [box][3][P]) evaluated at the points (added with accumulate).  conj_basis /
// scale select P2M's functions (conj Y, 4 pi: the transpose of P2M) or L2P's (Y, 1).
bool leaf_fast_supported(int p);
cudaError_t configure_leaf_fast();
void launch_l2p_fast(int p, int64_t N, const int *pt_box, const BoxDev *boxes, const double *xyz, const cf *le,
                     const MediumDev &M, const LayerScale &ls, cd *ph, bool conj_basis, double scale, bool accumulate,
                     cudaStream_t st);
// P2M of the mixed form for p <= 15: one warp per unit, me (cf [box][3][P], zeroed
// beforehand) += the coefficients of the helical charges qh (cd, sorted)
void launch_p2m_fast(int p, int64_t nunit, const LeafUnit *units, const BoxDev *boxes, const double *xyz,
                     const cd *qh, const MediumDev &M, const LayerScale &ls, cf *me, bool conj_basis, double scale,
                     cudaStream_t st);

// k_trans.cu
cudaError_t configure_trans_kernels();
template <typename T> int gemm_cols();
template <typename T>
void launch_group_gemm_t(int p, int64_t nwork, const GemmWork *work, const cx<T> *mats,
                         const int64_t *src, const int64_t *dst, const cx<T> *in, cx<T> *out,
                         bool atomic, cudaStream_t st);
template <typename T>
void launch_m2l_t(int p, int64_t nwork, const M2LWork *work, const GeomDev *geoms,
                  const CompDev *comps, const M2LPair *pairs, const cx<T> *tab, const cx<T> *me,
                  cx<T> *le, cudaStream_t st);
// transpose of the SIMT M2L: me_bar[src] += (M2L)^T le_bar[tgt], same work items
template <typename T>
void launch_m2l_tr(int p, int64_t nwork, const M2LWork *work, const GeomDev *geoms,
                   const CompDev *comps, const M2LPair *pairs, const cx<T> *tab, const cx<T> *le_bar,
                   cx<T> *me_bar, cudaStream_t st);
// k_m2l_tc.cu: mixed-form M2L on tcgen05 tensor cores (3xTF32), p <= 15;
// status gets bit 4 if a tensor-core wait gave up
bool m2l_tc_supported(int p);
int m2l_tc_cols();
// M2L work items of a context whose host structures are built, cut to at most bn
// helical columns, in the order the matvec launches them (api.cu)
int64_t plan_work_items(const lmfmm_ctx *ctx, int bn, std::vector<M2LWork> &mw);
cudaError_t configure_m2l_tc();
cudaError_t launch_m2l_tc(int p, int64_t nwork, const M2LWork *work, const GeomDev *geoms,
                          const CompDev *comps, const M2LPair *pairs, const cf *tab, const cf *me,
                          cf *le, int *status, cudaStream_t st);
// persistent warp-specialised variant (p <= 12) on a pre-tiled image of the
// tables in three bf16 pieces (launch_tile_tables from the FP64 tables);
// ephase holds e^{i d phi} of every pair, d = -(p+2)..p+2 ([npair][2p+5],
// FP32 from FP64); yscr holds m2l_tc2_scratch_floats(p, nsm) floats, nsm =
// CTAs of the launch (the SM count)
bool m2l_tc2_supported(int p);
size_t m2l_tc2_image_bytes(int p, int64_t ngeom);
size_t m2l_tc2_scratch_floats(int p, int nsm);
void launch_tile_tables(int p, int64_t g0, int64_t ng, const GeomDev *geoms, const CompDev *comps,
                        const cd *tab64, void *img, cudaStream_t st);
cudaError_t launch_m2l_tc2(int p, int64_t nwork, const M2LWork *work, const GeomDev *geoms,
                           const M2LPair *pairs, const cf *ephase, const void *img,
                           const cf *me, cf *le, float *yscr, int nsm, int *status, cudaStream_t st);
// the M2L of several problems (same p) in one persistent launch: work items
// carry their problem index into probs (device array)
cudaError_t launch_m2l_tc2_batch(int p, int64_t nwork, const M2LWork *work, const TcProb *probs, float *yscr,
                                 int nsm, int *status, cudaStream_t st);
// M2M or L2L on the same kernel: items M2LWork{geom = translation group, t = 0,
// npair, pair0} over pairs (tsrc[q], tdst[q]), 3 helical columns each; img holds
// one tiled matrix per group (tile_matrix_tc2, tc2_matrix_bytes(p) each)
cudaError_t launch_trans_tc2(int p, int64_t nwork, const M2LWork *work, const int64_t *tsrc,
                             const int64_t *tdst, const void *img, const cf *in, cf *out, float *yscr, int nsm,
                             int *status, cudaStream_t st);
size_t tc2_matrix_bytes(int p);
void tile_matrix_tc2(int p, const cd *M, void *img);   // host: P x P row-major (row = output index)
template <typename T>
void launch_scale_tables(int p, int64_t g0, int64_t ng, const GeomDev *geoms, const cd *tab64,
                         cx<T> *tab, cudaStream_t st);
// five Sommerfeld integrals per point pair of every near pair; a pair whose
// k_rho rule needs more than node_cap nodes sets bit 2 of *dflag (clamped rule)
void launch_s2t_pre(int64_t nnear, const NearPair *near, const BoxDev *boxes, const double *xyz,
                    const MediumDev &M, const CompDev *comps, double a, int node_cap, cd *coef,
                    int *dflag, cudaStream_t st);
// matvec near field: 8 combined coefficients per point pair ([j][8][i] per near pair)
void launch_s2t_combine(int64_t nnear, const NearPair *near, const BoxDev *boxes, const double *xyz,
                        const cd *coef5, cd *coef8, cudaStream_t st);
// one target row of the matvec near field: target ii of near pair `pair`
// against the pair's sources [s0, s0 + S2T_SRC); rows are ordered by pair,
// then source block, then ii
constexpr int S2T_SRC = 64;
struct S2TRow {
    int64_t pair;
    int ii, s0;
};
void launch_s2t_apply8(int64_t nrow, const S2TRow *rows, const NearPair *near, const BoxDev *boxes,
                       const cd *coef8, const cd *qh, cd *phih, cudaStream_t st);
// transposed near field: one row per (near pair, source jj), all targets
struct S2TRowT {
    int64_t pair;
    int jj, pad;
};
void launch_s2t_apply8_tr(int64_t nrow, const S2TRowT *rows, const NearPair *near, const BoxDev *boxes,
                          const cd *coef8, const cd *phb, cd *qhb, cudaStream_t st);
// free-space near field over leaf pairs ([2 * pair] = source leaf, [+1] =
// target leaf); rows {pair, point index within the row box}: targets (forward,
// out = ph) or sources (transposed, out = qh_bar)
void launch_p2p_free(int64_t nrow, const S2TRowT *rows, const int64_t *pairs, const BoxDev *boxes,
                     const double *xyz, const MediumDev &M, const cd *in, cd *out, bool transposed, cudaStream_t st);
// transposes of the helical maps: ph_bar = S^T y (caller order -> sorted),
// out = G^T qh_bar (sorted -> caller order), optional conjugation of y / out
void launch_gather_tr(int64_t N, const int64_t *perm, const void *y, int dtype, cd *phb, bool conj_in,
                      cudaStream_t st);
void launch_scatter_tr(int64_t N, const int64_t *perm, const cd *qhb, void *out, int dtype, bool conj_out,
                       cudaStream_t st);
void launch_s2t_apply(int64_t nnear, const NearPair *near, const BoxDev *boxes,
                      const double *xyz, const cd *coef, const cd *qh, cd *phih,
                      cudaStream_t st);

// k_grad.cu: position gradient of the FP64 form (see the file's header).
// grad (caller order, [N][3] real) is accumulated: zero it first.
void launch_grad_leaf(int p, int64_t N, int64_t nleaf, const int64_t *leaves, const BoxDev *boxes, const double *xyz,
                      const int64_t *perm, const cd *le, const cd *meb, const cd *qh, const cd *nu, const MediumDev &M,
                      const LayerScale &ls, double *grad, cudaStream_t st);
// 20 derivative integrals per near point pair (coef: [pair coef0 + e][20])
void launch_s2t_pre_grad(int64_t nnear, const NearPair *near, const BoxDev *boxes, const double *xyz,
                         const MediumDev &M, const CompDev *comps, double a, int node_cap, cd *coef, cudaStream_t st);
void launch_grad_near(int64_t nnear, const NearPair *near, const BoxDev *boxes, const double *xyz, const int64_t *perm,
                      const CompDev *comps, const cd *coefg, const cd *qh, const cd *nu, double *grad, cudaStream_t st);

}  // namespace lmf
