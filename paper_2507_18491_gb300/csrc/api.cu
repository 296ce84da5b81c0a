// The C ABI (include/lmfmm.h): context, validation, device setup (tree
// upload, M2L tabulation, translation matrices, near-field precomputation)
// and the matvec pipeline P2M -> M2M -> M2L -> L2L -> L2P (+ S2T).
#include <algorithm>
#include <chrono>
#include <map>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>

#include "kernels.cuh"
#include "quad.cuh"

using namespace lmf;

namespace {

thread_local std::string g_err;

struct DevState {
    std::vector<void *> allocs;
    double *xyz = nullptr;           // sorted [N][3]
    int64_t *perm = nullptr;
    BoxDev *boxes = nullptr;
    int64_t *leaves = nullptr;
    int64_t nleaves = 0;
    int *pt_box = nullptr;           // leaf box of every sorted point (mixed form)
    LeafUnit *units = nullptr;       // P2M units: at most 128 points of one leaf, largest first
    int64_t nunits = 0;
    bool leaf_fast = false;          // mixed form, p <= 15: P2M and L2P of k_leaf.cu
    cd *qh = nullptr, *ph = nullptr; // helical, sorted [N][3]
    void *me = nullptr, *le = nullptr; // [nbox][3][P], complex T (scaled)
    CompDev *comps = nullptr;
    GeomDev *geoms = nullptr;
    void *tab = nullptr;             // [ngeom][5][P][P], complex T (scaled)
    LayerScale lscale{};
    M2LPair *m2l = nullptr;
    M2LWork *m2lwork = nullptr;
    int64_t n_m2lwork = 0;
    void *tup = nullptr, *tdn = nullptr;   // [ngroup][P][P], complex T (scaled)
    void *tupT = nullptr, *tdnT = nullptr; // their transposes (SIMT forms: the transposed operator)
    float *yscr = nullptr;           // persistent kernel: per-CTA accumulator scratch
    int64_t *tchild = nullptr, *tparent = nullptr;
    GemmWork *gwork = nullptr;
    std::vector<int64_t> gwork_off;  // per child level: [off[l], off[l+1])
    void *tupi = nullptr, *tdni = nullptr;    // persistent kernel: tiled translation matrices (bf16 x 3)
    M2LWork *twork = nullptr;        // persistent kernel: translation items, per child level
    bool trans_tc = false;           // M2M / L2L on the persistent kernel (tensor_cores = 3)
    std::vector<int64_t> twork_off;
    NearPair *near = nullptr;
    cd *s2t = nullptr;               // near field: 8 combined coefficients per point pair
    S2TRow *s2twork = nullptr;       // near-field target rows
    int64_t n_s2twork = 0;
    S2TRowT *s2tworkT = nullptr;     // transposed near field: (near pair, source) rows
    int64_t n_s2tworkT = 0;
    int64_t *fpairs = nullptr;       // free-space near leaf pairs [n][2] (source, target)
    S2TRowT *frows = nullptr, *frowsT = nullptr;   // ... by target / by source point
    int64_t n_frows = 0, n_frowsT = 0;
    // position gradient (allocated by the first lmfmm_gradient call): checkpoints
    // of the forward pass's local expansions and helical charges, a field buffer,
    // and 20 derivative integrals per near point pair
    cd *le_ck = nullptr, *qh_ck = nullptr, *gfield = nullptr, *s2tg = nullptr;
    int *flag = nullptr;
    int *mvstatus = nullptr;         // matvec status word (bit 4: tensor-core wait gave up)
    int m2l_kernel = 0;              // 0 FP64 SIMT, 1 FP32 SIMT, 2 tcgen05 streamed, 3 tcgen05 persistent
    cf *ephase = nullptr;            // persistent kernel: e^{i d phi} per pair, d = -(p+2)..p+2
    int nsm = 0;
    cd *stage = nullptr;             // [2][N][3] for host-buffer matvec
    cudaEvent_t ev[9]{};
    bool ev_ok = false;
    bool mv_recorded = false;        // stage events hold a matvec
    double bytes = 0;
};

DevState *DS(lmfmm_ctx *c) { return (DevState *)c->dev; }

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
            return e_ == cudaErrorMemoryAllocation ? LMFMM_ERR_OOM : LMFMM_ERR_CUDA;       \
        }                                                                                  \
    } while (0)

void free_dev(lmfmm_ctx *ctx)
{
    DevState *d = DS(ctx);
    if (!d) return;
    cudaSetDevice(ctx->device);
    for (void *p : d->allocs) cudaFree(p);
    d->allocs.clear();
    if (d->ev_ok)
        for (auto &e : d->ev) cudaEventDestroy(e);
    delete d;
    ctx->dev = nullptr;
}

template <typename T>
lmfmm_status dalloc(lmfmm_ctx *ctx, T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T));
    if (e != cudaSuccess) {
        ctx->err = "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes: " +
                   cudaGetErrorString(e);
        return LMFMM_ERR_OOM;
    }
    DS(ctx)->allocs.push_back(q);
    DS(ctx)->bytes += (double)(count * sizeof(T));
    *p = (T *)q;
    return LMFMM_OK;
}

void dfree(lmfmm_ctx *ctx, void *p)
{
    auto &v = DS(ctx)->allocs;
    auto it = std::find(v.begin(), v.end(), p);
    if (it != v.end()) {
        cudaFree(p);
        v.erase(it);
    }
}

template <typename T>
lmfmm_status dupload(lmfmm_ctx *ctx, T **p, const std::vector<T> &h)
{
    lmfmm_status s = dalloc(ctx, p, h.size());
    if (s) return s;
    if (!h.empty()) CK(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return LMFMM_OK;
}

#define TRY(x)                        \
    do {                              \
        lmfmm_status s_ = (x);        \
        if (s_ != LMFMM_OK) return s_; \
    } while (0)

// k_rho quadrature plan of an M2L geometry: the Chebyshev integrands carry
// a polynomial of degree up to 2p+5 in k_rho.
QuadPlanDev geom_plan(double a, int p, double rho, double dz) { return make_plan(a, rho, dz, 2 * p + 5); }

lmfmm_status check_flag(lmfmm_ctx *ctx)
{
    int f = 0;
    CK(cudaMemcpy(&f, DS(ctx)->flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (f) {
        ctx->err = "device quadrature hit its cap (flag " + std::to_string(f) + ")";
        return LMFMM_ERR_QUAD;
    }
    return LMFMM_OK;
}

// Status word of the matvec kernels, cleared by every matvec before its first
// kernel: a tensor-core wait that gave up leaves bit 4.  Reads it after the
// stream's work is done.
lmfmm_status check_mvstatus(lmfmm_ctx *ctx, cudaStream_t st)
{
    int f = 0;
    CK(cudaStreamSynchronize(st));
    CK(cudaMemcpy(&f, DS(ctx)->mvstatus, sizeof(int), cudaMemcpyDeviceToHost));
    if (f) {
        ctx->err = "matvec: a bounded tensor-core wait gave up (status " + std::to_string(f) +
                   "); the result is incomplete";
        return LMFMM_ERR_TIMEOUT;
    }
    return LMFMM_OK;
}

// M2L work items of a built context: per geometry and table, runs of pairs
// giving at most `bn` helical columns (one column per pair for the (s5, 0)
// table, two for the others); prob tags them for a batched launch.  Returns the
// column count.
int64_t m2l_work_items(const lmfmm_ctx *ctx, int bn, int prob, std::vector<M2LWork> &mw)
{
    int64_t ncols = 0;
    for (size_t gi = 0; gi < ctx->geoms.size(); ++gi) {
        const Geom &g = ctx->geoms[gi];
        const CompDev &cg = ctx->comps[g.comp];
        // image maps of the component: the sign of odd degrees flips when the
        // source (target) side is mirrored an odd number of times
        const int flags = (((cg.s < 0) != (cg.has_src_refl != 0)) ? 1 : 0) |
                          (((cg.s < 0) != (cg.has_tgt_refl != 0)) ? 2 : 0);
        for (int t = 0; t < NTAB; ++t) {
            const int per = (t == 1) ? bn : bn / 2;
            for (int64_t q = g.pair0; q < g.pair1; q += per) {
                M2LWork w{};
                w.geom = (int)gi;
                w.t = t;
                w.flags = flags;
                w.pair0 = q;
                w.npair = (int)std::min<int64_t>(per, g.pair1 - q);
                w.prob = prob;
                ncols += w.npair * (t == 1 ? 1 : 2);
                mw.push_back(w);
            }
        }
    }
    return ncols;
}

// Tabulate a list of geometries into `tab` (device), batching node factors
// and Chebyshev integrals through a scratch buffer.
lmfmm_status tabulate(lmfmm_ctx *ctx, std::vector<GeomDev> &hg, const CompDev *dcomps,
                      const cd *dG, const int *dcg, cd *tab, cudaStream_t st, float *ms = nullptr)
{
    const int p = ctx->prm.p;
    const int LM = p + 2, DJ = 2 * p + 3;
    const int64_t per_node = 5 + 4 + 4 + LM + DJ;
    const int64_t ibr = (int64_t)NTAB * 4 * 4 * LM * DJ;
    const size_t scratch_bytes = (size_t)1 << 30;
    // batches
    std::vector<int> bstart;
    std::vector<int64_t> bstride;
    int ng = (int)hg.size();
    int g = 0;
    while (g < ng) {
        int64_t nodes = 0;
        int gb = g;
        while (gb < ng) {
            int64_t q = plan_nodes(hg[gb].plan);
            int64_t need = (nodes + q) * per_node + (int64_t)(gb - g + 1) * ibr;
            if ((size_t)need * sizeof(cd) > scratch_bytes && gb > g) break;
            hg[gb].node0 = nodes;
            nodes += q;
            ++gb;
            if (gb - g >= 2048) break;
        }
        for (int i = g; i < gb; ++i) hg[i].stride = nodes;
        bstart.push_back(g);
        bstride.push_back(nodes);
        g = gb;
    }
    bstart.push_back(ng);
    size_t need_max = 0;
    for (size_t b = 0; b + 1 < bstart.size(); ++b)
        need_max = std::max(need_max, (size_t)(bstride[b] * per_node +
                                               (int64_t)(bstart[b + 1] - bstart[b]) * ibr));
    GeomDev *dgeo = nullptr;
    cd *scr = nullptr;
    void *qg = nullptr, *qs = nullptr;
    CK(cudaMalloc(&qg, std::max<size_t>(1, hg.size()) * sizeof(GeomDev)));
    dgeo = (GeomDev *)qg;
    cudaError_t e = cudaMalloc(&qs, std::max<size_t>(1, need_max) * sizeof(cd));
    if (e != cudaSuccess) {
        cudaFree(qg);
        ctx->err = "tabulation scratch allocation failed";
        return LMFMM_ERR_OOM;
    }
    scr = (cd *)qs;
    lmfmm_status rc = LMFMM_OK;
    if (!hg.empty() &&
        cudaMemcpy(dgeo, hg.data(), hg.size() * sizeof(GeomDev), cudaMemcpyHostToDevice))
        rc = LMFMM_ERR_CUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool timed = ms && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    if (timed) cudaEventRecord(e0, st);
    for (size_t b = 0; rc == LMFMM_OK && b + 1 < bstart.size(); ++b) {
        int g0 = bstart[b], nb = bstart[b + 1] - g0;
        int qmax = 0;
        for (int i = g0; i < g0 + nb; ++i) qmax = std::max(qmax, plan_nodes(hg[i].plan));
        launch_tab_batch(dgeo, g0, nb, qmax, ctx->med, dcomps, p, dG, dcg, scr, bstride[b], tab,
                         DS(ctx)->flag, st);
        if (cudaGetLastError() != cudaSuccess) rc = LMFMM_ERR_CUDA;
    }
    if (timed) cudaEventRecord(e1, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = LMFMM_ERR_CUDA;
    if (timed) {
        if (cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) *ms = 0.f;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    cudaFree(qg);
    cudaFree(qs);
    if (rc) {
        ctx->err = "tabulation kernels failed";
        return rc;
    }
    return check_flag(ctx);
}

}  // namespace

namespace lmf {
// the M2L work items the matvec builds, for the host-side plan check (plan.cpp)
int64_t plan_work_items(const lmfmm_ctx *ctx, int bn, std::vector<M2LWork> &mw)
{
    return m2l_work_items(ctx, bn, 0, mw);
}

// read-only view of the device state for lmfmm_direct_noalloc (noalloc.cu)
bool noalloc_state(lmfmm_ctx *ctx, const int64_t **perm, const BoxDev **boxes, const double **xyz,
                   const CompDev **comps, cd **qh, cd **ph, int **flag)
{
    DevState *d = DS(ctx);
    if (!d || !d->perm || !d->boxes || !d->xyz || !d->comps || !d->qh || !d->ph || !d->flag)
        return false;
    *perm = d->perm;
    *boxes = d->boxes;
    *xyz = d->xyz;
    *comps = d->comps;
    *qh = d->qh;
    *ph = d->ph;
    *flag = d->flag;
    return true;
}
}  // namespace lmf

// --------------------------------------------------------------------- ABI
extern "C" {

lmfmm_status lmfmm_default_params(lmfmm_params *prm)
{
    if (!prm) return LMFMM_ERR_ARG;
    prm->p = 8;
    prm->depth = -1;
    prm->leaf_cap = 64;
    prm->theta = 0.55;
    prm->eta = 0.1;
    prm->quad_tol = 1e-15;
    prm->precision = LMFMM_FP64;
    prm->tensor_cores = 1;
    prm->quad_node_cap = 1 << 20;
    prm->components = LMFMM_REACTION;
    return LMFMM_OK;
}

lmfmm_status lmfmm_create(lmfmm_ctx **out, const lmfmm_params *prm, int device)
{
    if (!out || !prm) {
        g_err = "lmfmm_create: NULL argument";
        return LMFMM_ERR_ARG;
    }
    *out = nullptr;
    if (prm->p < 1 || prm->p > 16 || !(prm->theta > 0 && prm->theta < 1) || !(prm->eta >= 0) ||
        prm->depth > 20 || (prm->depth < 0 && prm->leaf_cap < 1)) {
        g_err = "lmfmm_create: parameter out of range (1 <= p <= 16, 0 < theta < 1, eta >= 0, "
                "depth <= 20)";
        return LMFMM_ERR_ARG;
    }
    if (prm->precision != LMFMM_FP64 && prm->precision != LMFMM_MIXED) {
        g_err = "lmfmm_create: precision must be LMFMM_FP64 or LMFMM_MIXED";
        return LMFMM_ERR_ARG;
    }
    if (prm->tensor_cores < 0 || prm->tensor_cores > 3) {
        g_err = "lmfmm_create: tensor_cores must be 0, 1, 2 or 3";
        return LMFMM_ERR_ARG;
    }
    if (prm->components < LMFMM_REACTION || prm->components > LMFMM_TOTAL) {
        g_err = "lmfmm_create: components must be LMFMM_REACTION, LMFMM_FREE or LMFMM_TOTAL";
        return LMFMM_ERR_ARG;
    }
    if (prm->quad_node_cap < 64) {
        g_err = "lmfmm_create: quad_node_cap must be at least 64";
        return LMFMM_ERR_ARG;
    }
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        g_err = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
        return LMFMM_ERR_CUDA;
    }
    if ((e = configure_fmm_kernels()) != cudaSuccess || (e = configure_tab_kernels()) != cudaSuccess ||
        (e = configure_leaf_fast()) != cudaSuccess) {
        g_err = std::string("kernel configuration: ") + cudaGetErrorString(e);
        return LMFMM_ERR_CUDA;
    }
    lmfmm_ctx *ctx = new lmfmm_ctx();
    ctx->device = device;
    ctx->prm = *prm;
    *out = ctx;
    return LMFMM_OK;
}

lmfmm_status lmfmm_set_layers(lmfmm_ctx *ctx, int L, const double *d, const lmfmm_c128 *k)
{
    if (!ctx) return LMFMM_ERR_ARG;
    if (L < 0 || L > LMF_MAXL || (L > 0 && !d) || !k) {
        ctx->err = "set_layers: need 0 <= L <= " + std::to_string(LMF_MAXL) + " and non-NULL arrays";
        return LMFMM_ERR_ARG;
    }
    for (int i = 0; i < L; ++i) {
        if (!std::isfinite(d[i]) || (i > 0 && !(d[i] < d[i - 1]))) {
            ctx->err = "set_layers: interfaces must be finite and strictly decreasing";
            return LMFMM_ERR_ARG;
        }
    }
    for (int i = 0; i <= L; ++i) {
        if (!std::isfinite(k[i].re) || !std::isfinite(k[i].im) || k[i].im < 0 ||
            (k[i].re == 0 && k[i].im == 0)) {
            ctx->err = "set_layers: wavenumber " + std::to_string(i) + " must be finite, nonzero, Im >= 0";
            return LMFMM_ERR_ARG;
        }
    }
    ctx->med = MediumDev{};
    ctx->med.L = L;
    for (int i = 0; i < L; ++i) ctx->med.d[i] = d[i];
    for (int i = 0; i <= L; ++i) ctx->med.k[i] = cd{k[i].re, k[i].im};
    ctx->layers_set = true;
    ctx->built = false;
    return LMFMM_OK;
}

lmfmm_status lmfmm_set_points(lmfmm_ctx *ctx, int64_t N, const double *xyz)
{
    if (!ctx) return LMFMM_ERR_ARG;
    if (!ctx->layers_set) {
        ctx->err = "set_points: call lmfmm_set_layers first";
        return LMFMM_ERR_STATE;
    }
    if (N < 1 || !xyz) {
        ctx->err = "set_points: need N >= 1 and a non-NULL array";
        return LMFMM_ERR_ARG;
    }
    ctx->N = N;
    ctx->xyz.assign(xyz, xyz + 3 * N);
    ctx->built = false;
    lmfmm_status s = classify_and_sort(ctx);
    ctx->points_set = (s == LMFMM_OK);
    return s;
}

lmfmm_status lmfmm_set_points_device(lmfmm_ctx *ctx, int64_t N, const double *xyz, void *stream)
{
    if (!ctx) return LMFMM_ERR_ARG;
    if (N < 1 || !xyz) {
        ctx->err = "set_points_device: need N >= 1 and a non-NULL array";
        return LMFMM_ERR_ARG;
    }
    CK(cudaSetDevice(ctx->device));
    std::vector<double> h((size_t)N * 3);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(h.data(), xyz, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return lmfmm_set_points(ctx, N, h.data());
}

lmfmm_status lmfmm_build(lmfmm_ctx *ctx, void *stream)
{
    if (!ctx) return LMFMM_ERR_ARG;
    if (!ctx->points_set) {
        ctx->err = "build: call lmfmm_set_points first";
        return LMFMM_ERR_STATE;
    }
    auto t0 = std::chrono::steady_clock::now();
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    free_dev(ctx);
    ctx->dev = new DevState();
    DevState *d = DS(ctx);
    ctx->built = false;
    TRY(build_host_structures(ctx));
    chebyshev_tables(ctx);
    const int p = ctx->prm.p, P = (p + 1) * (p + 1);
    const int64_t N = ctx->N, nbox = (int64_t)ctx->boxes.size();
    // memory estimate (tables dominate)
    const bool img_path = ctx->prm.precision == LMFMM_MIXED &&
                          (ctx->prm.tensor_cores == 1 || ctx->prm.tensor_cores == 3) && m2l_tc2_supported(p);
    double need = (double)ctx->geoms.size() * NTAB * P * P * 16.0 +
                  (img_path ? (double)m2l_tc2_image_bytes(p, (int64_t)ctx->geoms.size()) +
                                  (double)ctx->m2l.size() * (2 * p + 5) * 8.0
                            : 0.0) +
                  (double)nbox * 6 * P * 16.0 + (double)ctx->tgroups.size() * 2 * P * P * 16.0 +
                  (double)ctx->n_near_pp * 13 * 16.0 + (double)N * 200.0;
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    if (need > 0.85 * (double)fr) {
        ctx->err = "build: needs about " + std::to_string(need / 1e9) + " GB of device memory, " +
                   std::to_string(fr / 1e9) + " GB free (reduce p or raise theta/depth)";
        return LMFMM_ERR_OOM;
    }
    CK(cudaMalloc((void **)&d->flag, sizeof(int)));
    d->allocs.push_back(d->flag);
    CK(cudaMemset(d->flag, 0, sizeof(int)));
    CK(cudaMalloc((void **)&d->mvstatus, sizeof(int)));
    d->allocs.push_back(d->mvstatus);
    CK(cudaMemset(d->mvstatus, 0, sizeof(int)));
    for (auto &e : d->ev) CK(cudaEventCreate(&e));
    d->ev_ok = true;
    // points and boxes
    TRY(dupload(ctx, &d->xyz, ctx->sxyz));
    TRY(dupload(ctx, &d->perm, ctx->perm));
    std::vector<BoxDev> hb(nbox);
    std::vector<int64_t> leaves;
    for (int64_t i = 0; i < nbox; ++i) {
        const Box &b = ctx->boxes[i];
        hb[i] = BoxDev{b.p0, b.p1, {b.c[0], b.c[1], b.c[2]}, b.layer, 0};
        if (b.level == ctx->depth) leaves.push_back(i);
    }
    TRY(dupload(ctx, &d->boxes, hb));
    TRY(dupload(ctx, &d->leaves, leaves));
    d->nleaves = (int64_t)leaves.size();
    if (ctx->prm.precision == LMFMM_MIXED && leaf_fast_supported(p)) {
        std::vector<int> ptb(N > 0 ? N : 1, 0);
        std::vector<LeafUnit> units;
        for (int64_t li : leaves) {
            const Box &b = ctx->boxes[li];
            for (int64_t q = b.p0; q < b.p1; ++q) ptb[q] = (int)li;
            for (int64_t c0 = b.p0; c0 < b.p1; c0 += 128)
                units.push_back(LeafUnit{c0, std::min<int64_t>(c0 + 128, b.p1), (int)li, b.p1 - b.p0 <= 128 ? 1 : 0});
        }
        // largest units first, so that the last wave is made of small ones
        std::stable_sort(units.begin(), units.end(),
                         [](const LeafUnit &a, const LeafUnit &b) { return a.i1 - a.i0 > b.i1 - b.i0; });
        TRY(dupload(ctx, &d->pt_box, ptb));
        TRY(dupload(ctx, &d->units, units));
        d->nunits = (int64_t)units.size();
        d->leaf_fast = true;
    }
    TRY(dalloc(ctx, &d->qh, 3 * N));
    TRY(dalloc(ctx, &d->ph, 3 * N));
    const bool f32 = ctx->prm.precision == LMFMM_MIXED;
    d->m2l_kernel = !f32 ? 0
                    : ctx->prm.tensor_cores == 0 ? 1
                    : ((ctx->prm.tensor_cores == 1 || ctx->prm.tensor_cores == 3) && m2l_tc2_supported(p)) ? 3
                    : m2l_tc_supported(p) ? 2 : 1;
    const size_t esz = f32 ? sizeof(cf) : sizeof(cd);
    {
        unsigned char *q1 = nullptr, *q2 = nullptr;
        TRY(dalloc(ctx, &q1, (size_t)nbox * 3 * P * esz));
        TRY(dalloc(ctx, &q2, (size_t)nbox * 3 * P * esz));
        d->me = q1;
        d->le = q2;
    }
    const double Sroot = 2.0 * ctx->root_h;
    auto lev_size = [&](int lev) { return Sroot / (double)(1u << lev); };
    auto kabs = [&](int layer) { return std::hypot(ctx->med.k[layer].x, ctx->med.k[layer].y); };
    for (int j = 0; j <= ctx->med.L; ++j) d->lscale.s[j] = kabs(j) * lev_size(ctx->depth);
    TRY(dupload(ctx, &d->comps, ctx->comps));
    cd *dG = nullptr;
    int *dcg = nullptr;
    TRY(dupload(ctx, &dG, ctx->Gten));
    TRY(dupload(ctx, &dcg, ctx->comp_gidx));
    // M2L geometries, tables and work items
    const double a = medium_a(ctx->med);
    std::vector<GeomDev> hg(ctx->geoms.size());
    int64_t qtot = 0;
    float ms_tab = 0.f;
    for (size_t i = 0; i < ctx->geoms.size(); ++i) {
        const Geom &g = ctx->geoms[i];
        const CompDev &c = ctx->comps[g.comp];
        GeomDev gd{};
        gd.comp = g.comp;
        if (i >= ctx->n_react_geoms) {
            // free-space table: built on the host (addition theorem), not tabulated
            gd.rho = g.rho;
            gd.zs = g.zs;
            gd.zt = g.zt;
            gd.scale_s = gd.scale_t = kabs(c.l) * lev_size(g.level);
            gd.tab_index = (int64_t)i;
            hg[i] = gd;
            continue;
        }
        gd.src_primary = std::hypot(ctx->med.k[c.l].x, ctx->med.k[c.l].y) <=
                         std::hypot(ctx->med.k[c.lp].x, ctx->med.k[c.lp].y);
        gd.rho = g.rho;
        gd.zs = g.zs;
        gd.zt = g.zt;
        gd.plan = geom_plan(a, p, g.rho, c.s * (g.zs - g.zt));
        gd.scale_s = kabs(c.l) * lev_size(g.level);
        gd.scale_t = kabs(c.lp) * lev_size(g.level);
        if (plan_nodes(gd.plan) > ctx->prm.quad_node_cap) {
            ctx->err = "build: an M2L geometry needs " + std::to_string(plan_nodes(gd.plan)) +
                       " quadrature nodes, more than quad_node_cap = " + std::to_string(ctx->prm.quad_node_cap);
            return LMFMM_ERR_QUAD;
        }
        qtot += plan_nodes(gd.plan);
        gd.tab_index = (int64_t)i;
        hg[i] = gd;
    }
    {
        // FP64 Chebyshev tabulation, then level scaling (and cast for the mixed form)
        cd *tab64 = nullptr;
        TRY(dalloc(ctx, &tab64, ctx->geoms.size() * (size_t)NTAB * P * P));
        if (ctx->n_react_geoms > 0) {
            std::vector<GeomDev> hr(hg.begin(), hg.begin() + ctx->n_react_geoms);
            TRY(tabulate(ctx, hr, d->comps, dG, dcg, tab64, st, &ms_tab));
        }
        if (!ctx->free_tables.empty())
            CK(cudaMemcpy(tab64 + ctx->n_react_geoms * (size_t)NTAB * P * P, ctx->free_tables.data(),
                          ctx->free_tables.size() * sizeof(cd), cudaMemcpyHostToDevice));
        TRY(dupload(ctx, &d->geoms, hg));
        if (d->m2l_kernel == 3) {
            unsigned char *img = nullptr;
            TRY(dalloc(ctx, &img, m2l_tc2_image_bytes(p, (int64_t)hg.size())));
            launch_tile_tables(p, 0, (int64_t)hg.size(), d->geoms, d->comps, tab64, img, st);
            CK(cudaGetLastError());
            CK(cudaStreamSynchronize(st));
            dfree(ctx, tab64);
            d->tab = img;
            CK(cudaDeviceGetAttribute(&d->nsm, cudaDevAttrMultiProcessorCount, ctx->device));
            TRY(dalloc(ctx, &d->yscr, m2l_tc2_scratch_floats(p, d->nsm)));
            // phases of every pair: powers in FP64, rounded once to FP32
            const int MW = 2 * p + 5;
            std::vector<cf> ph(ctx->m2l.size() * (size_t)MW);
            for (size_t i = 0; i < ctx->m2l.size(); ++i) {
                const cd b{ctx->m2l[i].cphi, ctx->m2l[i].sphi};
                cd e{1.0, 0.0};
                cf *row = ph.data() + i * MW + (p + 2);
                row[0] = cf{1.f, 0.f};
                for (int m = 1; m <= p + 2; ++m) {
                    e = e * b;
                    row[m] = cf{(float)e.x, (float)e.y};
                    row[-m] = cf{(float)e.x, (float)-e.y};
                }
            }
            TRY(dupload(ctx, &d->ephase, ph));
        } else if (f32) {
            cf *t32 = nullptr;
            TRY(dalloc(ctx, &t32, ctx->geoms.size() * (size_t)NTAB * P * P));
            launch_scale_tables<float>(p, 0, (int64_t)hg.size(), d->geoms, tab64, t32, st);
            CK(cudaGetLastError());
            CK(cudaStreamSynchronize(st));
            dfree(ctx, tab64);
            d->tab = t32;
        } else {
            launch_scale_tables<double>(p, 0, (int64_t)hg.size(), d->geoms, tab64, tab64, st);
            CK(cudaGetLastError());
            d->tab = tab64;
        }
    }
    TRY(dupload(ctx, &d->m2l, ctx->m2l));
    std::vector<M2LWork> mw;
    const int64_t ncols = m2l_work_items(ctx, d->m2l_kernel >= 2 ? m2l_tc_cols()
                                                : f32 ? gemm_cols<float>() : gemm_cols<double>(), 0, mw);
    TRY(dupload(ctx, &d->m2lwork, mw));
    d->n_m2lwork = (int64_t)mw.size();
    // translation matrices (exact addition theorem, host)
    {
        std::vector<int64_t> goff;
        std::vector<int> gl;
        std::vector<double> gv;
        gaunt_table(p, goff, gl, gv);
        size_t ngr = ctx->tgroups.size();
        std::vector<cd> hup(ngr * (size_t)P * P), hdn(ngr * (size_t)P * P);
        std::vector<int> deg(P);
        for (int n = 0; n <= p; ++n)
            for (int m = -n; m <= n; ++m) deg[n * n + n + m] = n;
        for (size_t i = 0; i < ngr; ++i) {
            const TransGroup &g = ctx->tgroups[i];
            cd *U = &hup[i * P * P], *V = &hdn[i * P * P];
            translation_matrix(p, zc(ctx->med.k[g.layer].x, ctx->med.k[g.layer].y), g.t, goff, gl,
                               gv, U, V);
            // scaled expansions: M~ = M / s^n, L~ = L s^nu, s = |k| S_level
            double sc = kabs(g.layer) * lev_size(g.level), sp = kabs(g.layer) * lev_size(g.level - 1);
            for (int r = 0; r < P; ++r)
                for (int c = 0; c < P; ++c) {
                    double fu = std::pow(sc, deg[c]) / std::pow(sp, deg[r]);
                    double fd = std::pow(sc, deg[r]) / std::pow(sp, deg[c]);
                    U[r * P + c] = fu * U[r * P + c];
                    V[r * P + c] = fd * V[r * P + c];
                }
        }
        // the SIMT forms also keep the transposes (the transposed operator runs on them)
        const bool want_tr = d->m2l_kernel <= 1;
        std::vector<cd> hupT, hdnT;
        if (want_tr) {
            hupT.resize(hup.size());
            hdnT.resize(hdn.size());
            for (size_t i = 0; i < ngr; ++i)
                for (int r = 0; r < P; ++r)
                    for (int c = 0; c < P; ++c) {
                        hupT[i * P * P + (size_t)c * P + r] = hup[i * P * P + (size_t)r * P + c];
                        hdnT[i * P * P + (size_t)c * P + r] = hdn[i * P * P + (size_t)r * P + c];
                    }
        }
        if (f32) {
            auto to32 = [](const std::vector<cd> &a) {
                std::vector<cf> o(a.size());
                for (size_t i = 0; i < a.size(); ++i) o[i] = cf{(float)a[i].x, (float)a[i].y};
                return o;
            };
            cf *a1 = nullptr, *a2 = nullptr;
            TRY(dupload(ctx, &a1, to32(hup)));
            TRY(dupload(ctx, &a2, to32(hdn)));
            d->tup = a1;
            d->tdn = a2;
            if (want_tr) {
                TRY(dupload(ctx, &a1, to32(hupT)));
                TRY(dupload(ctx, &a2, to32(hdnT)));
                d->tupT = a1;
                d->tdnT = a2;
            }
        } else {
            cd *a1 = nullptr, *a2 = nullptr;
            TRY(dupload(ctx, &a1, hup));
            TRY(dupload(ctx, &a2, hdn));
            d->tup = a1;
            d->tdn = a2;
            if (want_tr) {
                TRY(dupload(ctx, &a1, hupT));
                TRY(dupload(ctx, &a2, hdnT));
                d->tupT = a1;
                d->tdnT = a2;
            }
        }
        TRY(dupload(ctx, &d->tchild, ctx->tpair_child));
        TRY(dupload(ctx, &d->tparent, ctx->tpair_parent));
        d->trans_tc = d->m2l_kernel == 3 && ctx->prm.tensor_cores == 3;
        if (d->trans_tc) {
            // M2M / L2L on the persistent tensor-core kernel: tiled bf16 three-piece
            // images of the scaled FP64 matrices, items of 21 pairs (63 helical columns)
            const size_t mw = tc2_matrix_bytes(p) / 4;
            std::vector<uint32_t> iu(ngr * mw), id(ngr * mw);
            for (size_t i = 0; i < ngr; ++i) {
                tile_matrix_tc2(p, &hup[i * P * P], &iu[i * mw]);
                tile_matrix_tc2(p, &hdn[i * P * P], &id[i * mw]);
            }
            uint32_t *a1 = nullptr, *a2 = nullptr;
            TRY(dupload(ctx, &a1, iu));
            TRY(dupload(ctx, &a2, id));
            d->tupi = a1;
            d->tdni = a2;
            std::vector<M2LWork> tw;
            d->twork_off.assign(ctx->depth + 2, 0);
            const int per = m2l_tc_cols() / 3;
            for (int lev = 1; lev <= ctx->depth; ++lev) {
                d->twork_off[lev] = (int64_t)tw.size();
                for (size_t gi = 0; gi < ngr; ++gi) {
                    const TransGroup &g = ctx->tgroups[gi];
                    if (g.level != lev) continue;
                    for (int64_t q = g.pair0; q < g.pair1; q += per) {
                        M2LWork w{};
                        w.geom = (int)gi;
                        w.npair = (int)std::min<int64_t>(per, g.pair1 - q);
                        w.pair0 = q;
                        tw.push_back(w);
                    }
                }
            }
            d->twork_off[ctx->depth + 1] = (int64_t)tw.size();
            TRY(dupload(ctx, &d->twork, tw));
        }
        // work items per child level
        std::vector<GemmWork> gw;
        d->gwork_off.assign(ctx->depth + 2, 0);
        for (int lev = 1; lev <= ctx->depth; ++lev) {
            d->gwork_off[lev] = (int64_t)gw.size();
            for (size_t gi = 0; gi < ctx->tgroups.size(); ++gi) {
                const TransGroup &g = ctx->tgroups[gi];
                if (g.level != lev) continue;
                int per = (f32 ? gemm_cols<float>() : gemm_cols<double>()) / 3;
                for (int64_t q = g.pair0; q < g.pair1; q += per)
                    gw.push_back(GemmWork{(int)gi, (int)std::min<int64_t>(per, g.pair1 - q), q});
            }
        }
        d->gwork_off[ctx->depth + 1] = (int64_t)gw.size();
        TRY(dupload(ctx, &d->gwork, gw));
    }
    // near field
    TRY(dupload(ctx, &d->near, ctx->near));
    {
        // five Sommerfeld integrals per point pair, then the 8 combined coefficients
        cd *s2t5 = nullptr;
        TRY(dalloc(ctx, &s2t5, (size_t)ctx->n_near_pp * 5));
        launch_s2t_pre((int64_t)ctx->near.size(), d->near, d->boxes, d->xyz, ctx->med, d->comps, a,
                       ctx->prm.quad_node_cap, s2t5, d->flag, st);
        CK(cudaGetLastError());
        TRY(dalloc(ctx, &d->s2t, (size_t)ctx->n_near_pp * 8));
        launch_s2t_combine((int64_t)ctx->near.size(), d->near, d->boxes, d->xyz, s2t5, d->s2t, st);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(st));
        dfree(ctx, s2t5);
        std::vector<S2TRow> sw;
        for (size_t i = 0; i < ctx->near.size(); ++i) {
            const NearPair &q = ctx->near[i];
            const Box &bs = ctx->boxes[q.src], &bt = ctx->boxes[q.tgt];
            for (int64_t s0 = 0; s0 < bs.p1 - bs.p0; s0 += S2T_SRC)
                for (int64_t ii = 0; ii < bt.p1 - bt.p0; ++ii) sw.push_back(S2TRow{(int64_t)i, (int)ii, (int)s0});
        }
        TRY(dupload(ctx, &d->s2twork, sw));
        d->n_s2twork = (int64_t)sw.size();
        std::vector<S2TRowT> swT;
        for (size_t i = 0; i < ctx->near.size(); ++i) {
            const Box &bs = ctx->boxes[ctx->near[i].src];
            for (int64_t jj = 0; jj < bs.p1 - bs.p0; ++jj) swT.push_back(S2TRowT{(int64_t)i, (int)jj, 0});
        }
        TRY(dupload(ctx, &d->s2tworkT, swT));
        d->n_s2tworkT = (int64_t)swT.size();
        // free-space near field
        std::vector<int64_t> fp;
        std::vector<S2TRowT> fr, frT;
        for (size_t i = 0; i < ctx->free_near.size(); ++i) {
            const auto &pr = ctx->free_near[i];
            fp.push_back(pr.first);
            fp.push_back(pr.second);
            const Box &bs = ctx->boxes[pr.first], &bt = ctx->boxes[pr.second];
            for (int64_t ii = 0; ii < bt.p1 - bt.p0; ++ii) fr.push_back(S2TRowT{(int64_t)i, (int)ii, 0});
            for (int64_t jj = 0; jj < bs.p1 - bs.p0; ++jj) frT.push_back(S2TRowT{(int64_t)i, (int)jj, 0});
        }
        TRY(dupload(ctx, &d->fpairs, fp));
        TRY(dupload(ctx, &d->frows, fr));
        TRY(dupload(ctx, &d->frowsT, frT));
        d->n_frows = (int64_t)fr.size();
        d->n_frowsT = (int64_t)frT.size();
    }
    TRY(check_flag(ctx));
    ctx->built = true;
    auto t1 = std::chrono::steady_clock::now();
    lmfmm_stats &S = ctx->stats;
    S = lmfmm_stats{};
    S.n_points = N;
    S.n_layers = ctx->med.L + 1;
    S.n_components = ctx->n_react_comps;
    S.depth = ctx->depth;
    S.n_boxes = nbox;
    S.n_m2l_pairs = (int64_t)ctx->m2l.size();
    S.n_geometries = (int64_t)ctx->geoms.size();
    S.n_near_pairs = (int64_t)ctx->near.size();
    S.n_near_point_pairs = ctx->n_near_pp;
    S.n_quad_nodes = qtot;
    S.bytes_tables = d->m2l_kernel == 3 ? (double)m2l_tc2_image_bytes(p, (int64_t)ctx->geoms.size())
                     : (double)ctx->geoms.size() * NTAB * P * P * (f32 ? 8.0 : 16.0);
    S.ms_setup = std::chrono::duration<double, std::milli>(t1 - t0).count();
    S.m2l_columns = ncols;
    S.m2l_kernel = d->m2l_kernel;
    for (size_t i = 0; i < ctx->n_react_geoms; ++i)
        if (ctx->comps[ctx->geoms[i].comp].l == ctx->comps[ctx->geoms[i].comp].lp) ++S.n_geometries_same_layer;
    S.n_free_geometries = (int64_t)(ctx->geoms.size() - ctx->n_react_geoms);
    S.n_free_near_point_pairs = ctx->n_free_pp;
    S.ms_tabulate = ms_tab;
    S.adjoint_transposed = d->m2l_kernel <= 1;
    S.tab_flops = 8.0 * (double)qtot * NTAB * 16 * (p + 2) * (2 * p + 3) +
                  8.0 * (double)ctx->geoms.size() * NTAB * (double)P * P * (p + 2);
    return LMFMM_OK;
}

extern "C++" {
// P2M / L2P at the leaves: the mixed form's kernels of k_leaf.cu where they
// apply (P2M one warp per unit of a leaf, L2P one thread per point), else one
// CTA per leaf.  l2p_basis / p2m_basis: the transposes.
template <typename T>
static void leaf_p2m(lmfmm_ctx *ctx, const cd *in, cx<T> *out, bool l2p_basis, cudaStream_t st)
{
    DevState *d = DS(ctx);
    const int p = ctx->prm.p;
    if constexpr (std::is_same<T, float>::value) {
        if (d->leaf_fast) {
            launch_p2m_fast(p, d->nunits, d->units, d->boxes, d->xyz, in, ctx->med, d->lscale, out, !l2p_basis,
                            l2p_basis ? 1.0 : 4.0 * 3.14159265358979323846, st);
            return;
        }
    }
    launch_p2m<T>(p, d->nleaves, d->leaves, d->boxes, d->xyz, in, ctx->med, d->lscale, out, st, l2p_basis);
}

template <typename T>
static void leaf_l2p(lmfmm_ctx *ctx, const cx<T> *in, cd *out, bool p2m_basis, cudaStream_t st)
{
    DevState *d = DS(ctx);
    const int p = ctx->prm.p;
    if constexpr (std::is_same<T, float>::value) {
        if (d->leaf_fast) {
            launch_l2p_fast(p, ctx->N, d->pt_box, d->boxes, d->xyz, in, ctx->med, d->lscale, out, p2m_basis,
                            p2m_basis ? 4.0 * 3.14159265358979323846 : 1.0, false, st);
            return;
        }
    }
    launch_l2p<T>(p, d->nleaves, d->leaves, d->boxes, d->xyz, in, ctx->med, d->lscale, out, st, p2m_basis, false);
}

// stages of one matvec, for the batched launch: the upward pass (gather, P2M,
// M2M), the M2L (own_m2l = false: only the clearing of the local expansions,
// the M2L itself runs in the batch's merged launch), the downward pass
enum { MV_UP = 1, MV_M2L = 2, MV_DOWN = 4, MV_ALL = 7 };

template <typename T>
static lmfmm_status matvec_t(lmfmm_ctx *ctx, const void *J, int dtype, void *Phi,
                             cudaStream_t st, bool cj, int parts = MV_ALL, bool own_m2l = true)
{
    DevState *d = DS(ctx);
    const int p = ctx->prm.p, P = (p + 1) * (p + 1);
    const int64_t N = ctx->N, nbox = (int64_t)ctx->boxes.size();
    cx<T> *me = (cx<T> *)d->me, *le = (cx<T> *)d->le;
    const cx<T> *tup = (const cx<T> *)d->tup, *tdn = (const cx<T> *)d->tdn;
    int nl = 0;   // kernels launched (launchers skip empty work)
    if (parts & MV_UP) {
    CK(cudaEventRecord(d->ev[0], st));
    CK(cudaMemsetAsync(d->mvstatus, 0, sizeof(int), st));
    launch_gather_in(N, d->perm, J, dtype, d->qh, cj, st);
    nl += N > 0;
    nl += d->nleaves > 0;   // P2M
    CK(cudaMemsetAsync(me, 0, (size_t)nbox * 3 * P * sizeof(cx<T>), st));
    leaf_p2m<T>(ctx, d->qh, me, false, st);
    CK(cudaEventRecord(d->ev[1], st));
    for (int lev = ctx->depth; lev >= 1; --lev) {
        if constexpr (std::is_same<T, float>::value) {
            if (d->trans_tc) {
                int64_t w0 = d->twork_off[lev], w1 = d->twork_off[lev + 1];
                CK(launch_trans_tc2(p, w1 - w0, d->twork + w0, d->tchild, d->tparent, d->tupi, me, me,
                                    d->yscr, d->nsm, d->mvstatus, st));
                nl += w1 > w0;
                continue;
            }
        }
        int64_t w0 = d->gwork_off[lev], w1 = d->gwork_off[lev + 1];
        launch_group_gemm_t<T>(p, w1 - w0, d->gwork + w0, tup, d->tchild, d->tparent, me, me, true,
                               st);
        nl += w1 > w0;
    }
    CK(cudaEventRecord(d->ev[2], st));
    }
    if (parts & MV_M2L) {
    nl += d->n_m2lwork > 0;   // M2L
    CK(cudaMemsetAsync(le, 0, (size_t)nbox * 3 * P * sizeof(cx<T>), st));
    if (!own_m2l) {
        // the batch's merged launch applies this problem's M2L
    } else if constexpr (std::is_same<T, float>::value) {
        if (d->m2l_kernel == 3) {
            CK(launch_m2l_tc2(p, d->n_m2lwork, d->m2lwork, d->geoms, d->m2l, d->ephase, d->tab,
                              me, le, d->yscr, d->nsm, d->mvstatus, st));
        }
        else if (d->m2l_kernel == 2)
            CK(launch_m2l_tc(p, d->n_m2lwork, d->m2lwork, d->geoms, d->comps, d->m2l,
                             (const cf *)d->tab, me, le, d->mvstatus, st));
        else
            launch_m2l_t<T>(p, d->n_m2lwork, d->m2lwork, d->geoms, d->comps, d->m2l,
                            (const cx<T> *)d->tab, me, le, st);
    } else {
        launch_m2l_t<T>(p, d->n_m2lwork, d->m2lwork, d->geoms, d->comps, d->m2l,
                        (const cx<T> *)d->tab, me, le, st);
    }
    CK(cudaEventRecord(d->ev[3], st));
    }
    if (parts & MV_DOWN) {
    for (int lev = 1; lev <= ctx->depth; ++lev) {
        if constexpr (std::is_same<T, float>::value) {
            if (d->trans_tc) {
                int64_t w0 = d->twork_off[lev], w1 = d->twork_off[lev + 1];
                CK(launch_trans_tc2(p, w1 - w0, d->twork + w0, d->tparent, d->tchild, d->tdni, le, le,
                                    d->yscr, d->nsm, d->mvstatus, st));
                nl += w1 > w0;
                continue;
            }
        }
        int64_t w0 = d->gwork_off[lev], w1 = d->gwork_off[lev + 1];
        // a child has one parent: reductions (fire and forget) rather than read-modify-write
        launch_group_gemm_t<T>(p, w1 - w0, d->gwork + w0, tdn, d->tparent, d->tchild, le, le, true,
                               st);
        nl += w1 > w0;
    }
    CK(cudaEventRecord(d->ev[4], st));
    leaf_l2p<T>(ctx, le, d->ph, false, st);
    CK(cudaEventRecord(d->ev[5], st));
    launch_s2t_apply8(d->n_s2twork, d->s2twork, d->near, d->boxes, d->s2t, d->qh, d->ph, st);
    launch_p2p_free(d->n_frows, d->frows, d->fpairs, d->boxes, d->xyz, ctx->med, d->qh, d->ph, false, st);
    nl += d->n_frows > 0;
    CK(cudaEventRecord(d->ev[6], st));
    launch_scatter_out(N, d->perm, d->ph, Phi, dtype, cj, st);
    nl += (d->nleaves > 0) + (d->n_s2twork > 0) + (N > 0);   // L2P, near field, scatter
    CK(cudaEventRecord(d->ev[7], st));
    d->mv_recorded = true;
    }
    CK(cudaGetLastError());
    if (parts == MV_ALL) ctx->stats.launches = nl;
    return LMFMM_OK;
}

// The transposed operator A^T = G^T (P2M^T M2M^T M2L^T L2L^T L2P^T + S2T^T) S^T,
// every factor the exact transpose of the forward one (SIMT forms): L2P^T sums
// the point values against L2P's functions (P2M's kernel), L2L^T and M2M^T run
// the transposed matrices up and down the tree, M2L^T applies the transposed
// tables, P2M^T evaluates with P2M's functions (L2P's kernel).  With cj the
// input and output are conjugated: conj(A^T conj y) = A^H y.
template <typename T>
static lmfmm_status matvec_tr_t(lmfmm_ctx *ctx, const void *y, int dtype, void *out, cudaStream_t st, bool cj)
{
    DevState *d = DS(ctx);
    const int p = ctx->prm.p, P = (p + 1) * (p + 1);
    const int64_t N = ctx->N, nbox = (int64_t)ctx->boxes.size();
    cx<T> *me = (cx<T> *)d->me, *le = (cx<T> *)d->le;
    const cx<T> *tupT = (const cx<T> *)d->tupT, *tdnT = (const cx<T> *)d->tdnT;
    int nl = 0;
    CK(cudaEventRecord(d->ev[0], st));
    CK(cudaMemsetAsync(d->mvstatus, 0, sizeof(int), st));
    launch_gather_tr(N, d->perm, y, dtype, d->ph, cj, st);   // ph <- S^T y
    CK(cudaMemsetAsync(le, 0, (size_t)nbox * 3 * P * sizeof(cx<T>), st));
    leaf_p2m<T>(ctx, d->ph, le, true, st);
    nl += (N > 0) + (d->nleaves > 0);
    CK(cudaEventRecord(d->ev[1], st));
    for (int lev = ctx->depth; lev >= 1; --lev) {   // L2L^T: children into parents
        int64_t w0 = d->gwork_off[lev], w1 = d->gwork_off[lev + 1];
        launch_group_gemm_t<T>(p, w1 - w0, d->gwork + w0, tdnT, d->tchild, d->tparent, le, le, true, st);
        nl += w1 > w0;
    }
    CK(cudaEventRecord(d->ev[2], st));
    CK(cudaMemsetAsync(me, 0, (size_t)nbox * 3 * P * sizeof(cx<T>), st));
    launch_m2l_tr<T>(p, d->n_m2lwork, d->m2lwork, d->geoms, d->comps, d->m2l, (const cx<T> *)d->tab, le, me, st);
    nl += d->n_m2lwork > 0;
    CK(cudaEventRecord(d->ev[3], st));
    for (int lev = 1; lev <= ctx->depth; ++lev) {   // M2M^T: parents into children
        int64_t w0 = d->gwork_off[lev], w1 = d->gwork_off[lev + 1];
        launch_group_gemm_t<T>(p, w1 - w0, d->gwork + w0, tupT, d->tparent, d->tchild, me, me, true, st);
        nl += w1 > w0;
    }
    CK(cudaEventRecord(d->ev[4], st));
    leaf_l2p<T>(ctx, me, d->qh, true, st);
    CK(cudaEventRecord(d->ev[5], st));
    launch_s2t_apply8_tr(d->n_s2tworkT, d->s2tworkT, d->near, d->boxes, d->s2t, d->ph, d->qh, st);
    launch_p2p_free(d->n_frowsT, d->frowsT, d->fpairs, d->boxes, d->xyz, ctx->med, d->ph, d->qh, true, st);
    nl += d->n_frowsT > 0;
    CK(cudaEventRecord(d->ev[6], st));
    launch_scatter_tr(N, d->perm, d->qh, out, dtype, cj, st);
    nl += (d->nleaves > 0) + (d->n_s2tworkT > 0) + (N > 0);
    CK(cudaEventRecord(d->ev[7], st));
    CK(cudaGetLastError());
    d->mv_recorded = true;
    ctx->stats.launches = nl;
    return LMFMM_OK;
}

static lmfmm_status matvec_tr_impl(lmfmm_ctx *ctx, const void *y, int dtype, void *out, cudaStream_t st, bool cj)
{
    if (DS(ctx)->m2l_kernel > 1) {
        ctx->err = "the transposed operator runs in the FP64 form and the mixed form with tensor_cores = 0 "
                   "(the tensor-core forms hold their tables only as the tiled image)";
        return LMFMM_ERR_UNSUPPORTED;
    }
    if (ctx->prm.precision == LMFMM_MIXED) return matvec_tr_t<float>(ctx, y, dtype, out, st, cj);
    return matvec_tr_t<double>(ctx, y, dtype, out, st, cj);
}

static lmfmm_status matvec_impl(lmfmm_ctx *ctx, const void *J, int dtype, void *Phi,
                                cudaStream_t st, bool cj)
{
    if (ctx->prm.precision == LMFMM_MIXED) return matvec_t<float>(ctx, J, dtype, Phi, st, cj);
    return matvec_t<double>(ctx, J, dtype, Phi, st, cj);
}
}  // extern "C++"

static lmfmm_status matvec_args(lmfmm_ctx *ctx, const char *who, const void *J, int dtype, const void *Phi)
{
    if (!ctx->built) {
        ctx->err = std::string(who) + ": call lmfmm_build first";
        return LMFMM_ERR_STATE;
    }
    if (!J || !Phi) {
        ctx->err = std::string(who) + ": NULL buffer";
        return LMFMM_ERR_ARG;
    }
    if (dtype != LMFMM_C128 && dtype != LMFMM_C64) {
        ctx->err = std::string(who) + ": dtype must be LMFMM_C128 or LMFMM_C64";
        return LMFMM_ERR_ARG;
    }
    return LMFMM_OK;
}

lmfmm_status lmfmm_matvec(lmfmm_ctx *ctx, const void *J, int dtype, void *Phi, void *stream)
{
    if (!ctx) return LMFMM_ERR_ARG;
    TRY(matvec_args(ctx, "matvec", J, dtype, Phi));
    CK(cudaSetDevice(ctx->device));
    return matvec_impl(ctx, J, dtype, Phi, (cudaStream_t)stream, false);
}

lmfmm_status lmfmm_matvec_adjoint(lmfmm_ctx *ctx, const void *y, int dtype, void *Phi, void *stream)
{
    if (!ctx) return LMFMM_ERR_ARG;
    TRY(matvec_args(ctx, "matvec_adjoint", y, dtype, Phi));
    CK(cudaSetDevice(ctx->device));
    if (DS(ctx)->m2l_kernel <= 1) return matvec_tr_impl(ctx, y, dtype, Phi, (cudaStream_t)stream, true);
    return matvec_impl(ctx, y, dtype, Phi, (cudaStream_t)stream, true);
}

lmfmm_status lmfmm_matvec_transpose(lmfmm_ctx *ctx, const void *y, int dtype, void *out, void *stream)
{
    if (!ctx) return LMFMM_ERR_ARG;
    TRY(matvec_args(ctx, "matvec_transpose", y, dtype, out));
    CK(cudaSetDevice(ctx->device));
    return matvec_tr_impl(ctx, y, dtype, out, (cudaStream_t)stream, false);
}

lmfmm_status lmfmm_matvec_host(lmfmm_ctx *ctx, const void *J, int dtype, void *Phi, void *stream)
{
    if (!ctx) return LMFMM_ERR_ARG;
    TRY(matvec_args(ctx, "matvec_host", J, dtype, Phi));
    CK(cudaSetDevice(ctx->device));
    DevState *d = DS(ctx);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)ctx->N * 3 * (dtype == LMFMM_C64 ? sizeof(cf) : sizeof(cd));
    // staging [2][N][3] complex128, used at the caller's element size
    if (!d->stage) TRY(dalloc(ctx, &d->stage, (size_t)ctx->N * 6));
    unsigned char *sin = (unsigned char *)d->stage, *sout = (unsigned char *)(d->stage + 3 * ctx->N);
    CK(cudaMemcpyAsync(sin, J, bytes, cudaMemcpyHostToDevice, st));
    TRY(matvec_impl(ctx, sin, dtype, sout, st, false));
    CK(cudaMemcpyAsync(Phi, sout, bytes, cudaMemcpyDeviceToHost, st));
    return check_mvstatus(ctx, st);
}

lmfmm_status lmfmm_gradient(lmfmm_ctx *ctx, const void *J, const void *g, int dtype, void *gJ, double *gxyz,
                            void *stream)
{
    if (!ctx) return LMFMM_ERR_ARG;
    TRY(matvec_args(ctx, "gradient", J, dtype, g));
    if (!gJ && !gxyz) {
        ctx->err = "gradient: nothing to compute (gJ and gxyz are NULL)";
        return LMFMM_ERR_ARG;
    }
    if (ctx->prm.precision != LMFMM_FP64 || ctx->prm.components != LMFMM_REACTION) {
        ctx->err = "gradient: the position gradient runs in the FP64 form of the reaction part";
        return LMFMM_ERR_UNSUPPORTED;
    }
    CK(cudaSetDevice(ctx->device));
    DevState *d = DS(ctx);
    cudaStream_t st = (cudaStream_t)stream;
    const int p = ctx->prm.p, P = (p + 1) * (p + 1);
    const int64_t N = ctx->N, nbox = (int64_t)ctx->boxes.size();
    if (!d->le_ck) {
        TRY(dalloc(ctx, &d->le_ck, (size_t)nbox * 3 * P));
        TRY(dalloc(ctx, &d->qh_ck, (size_t)N * 3));
        TRY(dalloc(ctx, &d->gfield, (size_t)N * 3));
        TRY(dalloc(ctx, &d->s2tg, (size_t)std::max<int64_t>(1, ctx->n_near_pp) * 20));
        launch_s2t_pre_grad((int64_t)ctx->near.size(), d->near, d->boxes, d->xyz, ctx->med, d->comps,
                            medium_a(ctx->med), ctx->prm.quad_node_cap, d->s2tg, st);
        CK(cudaGetLastError());
    }
    // forward pass (its result is not needed), then checkpoint what the
    // transposed pass overwrites: the local expansions and the helical charges
    TRY(matvec_t<double>(ctx, J, dtype, d->gfield, st, false));
    CK(cudaMemcpyAsync(d->le_ck, d->le, (size_t)nbox * 3 * P * sizeof(cd), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(d->qh_ck, d->qh, (size_t)N * 3 * sizeof(cd), cudaMemcpyDeviceToDevice, st));
    // transposed pass of conj(g): gJ = A^H g; leaves ph = S^T conj(g), me = its multipole expansions
    TRY(matvec_tr_t<double>(ctx, g, dtype, gJ ? gJ : (void *)d->gfield, st, true));
    if (gxyz) {
        CK(cudaMemsetAsync(gxyz, 0, (size_t)N * 3 * sizeof(double), st));
        launch_grad_leaf(p, N, d->nleaves, d->leaves, d->boxes, d->xyz, d->perm, d->le_ck, (const cd *)d->me,
                         d->qh_ck, d->ph, ctx->med, d->lscale, gxyz, st);
        launch_grad_near((int64_t)ctx->near.size(), d->near, d->boxes, d->xyz, d->perm, d->comps, d->s2tg,
                         d->qh_ck, d->ph, gxyz, st);
        CK(cudaGetLastError());
    }
    return LMFMM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches
struct lmfmm_batch {
    std::vector<lmfmm_ctx *> ctxs;
    int device = 0, p = 0, mixed = 0;
    bool merged = false;          // every problem on the persistent tensor-core M2L: one merged launch
    TcProb *dprobs = nullptr;
    M2LWork *dwork = nullptr;
    int64_t nwork = 0;
    int *status = nullptr;
    int variant = 0;
    double ms_variant[4] = {0, 0, 0, 0};
    cudaStream_t cap = nullptr;   // capture stream of the graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void *> gJ;
    std::vector<void *> gPhi;
    int gdtype = -1;
    std::string err;
};

namespace {

void batch_drop_graph(lmfmm_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// merged work list of a batch: variant bit 0 interleaves the problems' items
// round robin (else one problem after the other), bit 1 cuts items to 32
// helical columns (else 64)
lmfmm_status batch_work(lmfmm_batch *b, int variant, M2LWork **dst, int64_t *n)
{
    std::vector<std::vector<M2LWork>> per(b->ctxs.size());
    for (size_t i = 0; i < b->ctxs.size(); ++i)
        m2l_work_items(b->ctxs[i], (variant & 2) ? m2l_tc_cols() / 2 : m2l_tc_cols(), (int)i, per[i]);
    std::vector<M2LWork> all;
    if (variant & 1) {
        for (size_t k = 0;; ++k) {
            bool any = false;
            for (auto &v : per)
                if (k < v.size()) {
                    all.push_back(v[k]);
                    any = true;
                }
            if (!any) break;
        }
    } else {
        for (auto &v : per) all.insert(all.end(), v.begin(), v.end());
    }
    void *q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(1, all.size()) * sizeof(M2LWork)) != cudaSuccess) return LMFMM_ERR_OOM;
    if (!all.empty() && cudaMemcpy(q, all.data(), all.size() * sizeof(M2LWork), cudaMemcpyHostToDevice)) {
        cudaFree(q);
        return LMFMM_ERR_CUDA;
    }
    *dst = (M2LWork *)q;
    *n = (int64_t)all.size();
    return LMFMM_OK;
}

template <typename T>
lmfmm_status batch_record(lmfmm_batch *b, const void *const *J, void *const *Phi, int dtype, cudaStream_t st)
{
    const size_t n = b->ctxs.size();
    for (size_t i = 0; i < n; ++i) {
        lmfmm_status r = matvec_t<T>(b->ctxs[i], J[i], dtype, Phi[i], st, false, MV_UP | MV_M2L, !b->merged);
        if (r) return r;
    }
    if (b->merged) {
        if (cudaMemsetAsync(b->status, 0, sizeof(int), st) != cudaSuccess) return LMFMM_ERR_CUDA;
        DevState *d0 = DS(b->ctxs[0]);
        if (launch_m2l_tc2_batch(b->p, b->nwork, b->dwork, b->dprobs, d0->yscr, d0->nsm, b->status, st) !=
            cudaSuccess)
            return LMFMM_ERR_CUDA;
    }
    for (size_t i = 0; i < n; ++i) {
        lmfmm_status r = matvec_t<T>(b->ctxs[i], J[i], dtype, Phi[i], st, false, MV_DOWN);
        if (r) return r;
    }
    return LMFMM_OK;
}

}  // namespace

extern "C" {

lmfmm_status lmfmm_batch_create(lmfmm_batch **out, lmfmm_ctx *const *ctxs, int n)
{
    if (!out || !ctxs || n < 1) {
        g_err = "batch_create: need n >= 1 contexts";
        return LMFMM_ERR_ARG;
    }
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i] || !ctxs[i]->built || ctxs[i]->device != ctxs[0]->device || ctxs[i]->prm.p != ctxs[0]->prm.p ||
            ctxs[i]->prm.precision != ctxs[0]->prm.precision) {
            g_err = "batch_create: every context must be built, on one device, with one p and one precision";
            return LMFMM_ERR_ARG;
        }
    if (cudaSetDevice(ctxs[0]->device) != cudaSuccess) return LMFMM_ERR_CUDA;
    lmfmm_batch *b = new lmfmm_batch();
    b->ctxs.assign(ctxs, ctxs + n);
    b->device = ctxs[0]->device;
    b->p = ctxs[0]->prm.p;
    b->mixed = ctxs[0]->prm.precision == LMFMM_MIXED;
    b->merged = true;
    for (int i = 0; i < n; ++i) b->merged = b->merged && DS(ctxs[i])->m2l_kernel == 3;
    lmfmm_status rc = LMFMM_OK;
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc((void **)&b->status, sizeof(int)) != cudaSuccess || cudaMemset(b->status, 0, sizeof(int)))
        rc = LMFMM_ERR_CUDA;
    if (!rc && b->merged) {
        std::vector<TcProb> hp(n);
        for (int i = 0; i < n; ++i) {
            DevState *d = DS(ctxs[i]);
            hp[i] = TcProb{d->geoms, d->m2l, d->ephase, d->tab, (const cf *)d->me, (cf *)d->le};
        }
        if (cudaMalloc((void **)&b->dprobs, n * sizeof(TcProb)) != cudaSuccess ||
            cudaMemcpy(b->dprobs, hp.data(), n * sizeof(TcProb), cudaMemcpyHostToDevice) != cudaSuccess)
            rc = LMFMM_ERR_CUDA;
        if (!rc) rc = batch_work(b, 0, &b->dwork, &b->nwork);
    }
    if (rc) {
        g_err = "batch_create: device setup failed";
        lmfmm_batch_destroy(b);
        return rc;
    }
    *out = b;
    return LMFMM_OK;
}

lmfmm_status lmfmm_batch_matvec(lmfmm_batch *b, const void *const *J, void *const *Phi, int dtype, void *stream)
{
    if (!b) return LMFMM_ERR_ARG;
    const size_t n = b->ctxs.size();
    if (!J || !Phi || (dtype != LMFMM_C128 && dtype != LMFMM_C64)) {
        b->err = "batch_matvec: NULL pointer arrays or bad dtype";
        return LMFMM_ERR_ARG;
    }
    for (size_t i = 0; i < n; ++i)
        if (!J[i] || !Phi[i]) {
            b->err = "batch_matvec: NULL buffer";
            return LMFMM_ERR_ARG;
        }
    if (cudaSetDevice(b->device) != cudaSuccess) return LMFMM_ERR_CUDA;
    const bool same = b->exec && b->gdtype == dtype && std::equal(b->gJ.begin(), b->gJ.end(), J) &&
                      std::equal(b->gPhi.begin(), b->gPhi.end(), Phi);
    if (!same) {
        // record every launch of the batch once, on the capture stream
        batch_drop_graph(b);
        if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            b->err = "batch_matvec: stream capture failed to start";
            return LMFMM_ERR_CUDA;
        }
        lmfmm_status rc = b->mixed ? batch_record<float>(b, J, Phi, dtype, b->cap)
                                   : batch_record<double>(b, J, Phi, dtype, b->cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (rc || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            b->err = "batch_matvec: capture of the batch failed";
            return rc ? rc : LMFMM_ERR_CUDA;
        }
        b->graph = g;
        if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
            batch_drop_graph(b);
            b->err = "batch_matvec: graph instantiation failed";
            return LMFMM_ERR_CUDA;
        }
        b->gJ.assign(J, J + n);
        b->gPhi.assign(Phi, Phi + n);
        b->gdtype = dtype;
    }
    if (cudaGraphLaunch(b->exec, (cudaStream_t)stream) != cudaSuccess) {
        b->err = "batch_matvec: graph launch failed";
        return LMFMM_ERR_CUDA;
    }
    return LMFMM_OK;
}

lmfmm_status lmfmm_batch_tune(lmfmm_batch *b, void *stream)
{
    if (!b) return LMFMM_ERR_ARG;
    if (!b->merged) {
        b->err = "batch_tune: the merged M2L needs every problem on the persistent tensor-core kernel";
        return LMFMM_ERR_UNSUPPORTED;
    }
    if (cudaSetDevice(b->device) != cudaSuccess) return LMFMM_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    DevState *d0 = DS(b->ctxs[0]);
    const int P = (b->p + 1) * (b->p + 1);
    // defined inputs for the timing runs
    for (lmfmm_ctx *c : b->ctxs)
        if (cudaMemsetAsync(DS(c)->me, 0, c->boxes.size() * 3 * (size_t)P * sizeof(cf), st) != cudaSuccess)
            return LMFMM_ERR_CUDA;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LMFMM_ERR_CUDA;
    int best = 0;
    for (int v = 0; v < 4; ++v) {
        M2LWork *w = nullptr;
        int64_t nw = 0;
        lmfmm_status rc = batch_work(b, v, &w, &nw);
        if (rc) return rc;
        float tmin = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, st);
            launch_m2l_tc2_batch(b->p, nw, w, b->dprobs, d0->yscr, d0->nsm, b->status, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tmin = std::min(tmin, ms);   // first run warms the caches
        }
        cudaFree(w);
        b->ms_variant[v] = tmin;
        if (tmin < b->ms_variant[best]) best = v;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) return LMFMM_ERR_CUDA;
    M2LWork *w = nullptr;
    int64_t nw = 0;
    TRY(batch_work(b, best, &w, &nw));
    cudaFree(b->dwork);
    b->dwork = w;
    b->nwork = nw;
    b->variant = best;
    batch_drop_graph(b);   // the next matvec captures the chosen list
    int f = 0;
    cudaMemcpy(&f, b->status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaMemset(b->status, 0, sizeof(int));
    if (f) {
        b->err = "batch_tune: a bounded tensor-core wait gave up during the timing runs";
        return LMFMM_ERR_TIMEOUT;
    }
    return LMFMM_OK;
}

lmfmm_status lmfmm_batch_check(lmfmm_batch *b, void *stream)
{
    if (!b) return LMFMM_ERR_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess || cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return LMFMM_ERR_CUDA;
    int f = 0;
    if (cudaMemcpy(&f, b->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LMFMM_ERR_CUDA;
    for (lmfmm_ctx *c : b->ctxs) {
        int g = 0;
        if (cudaMemcpy(&g, DS(c)->mvstatus, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return LMFMM_ERR_CUDA;
        f |= g;
    }
    if (f) {
        b->err = "batch: a bounded tensor-core wait gave up; the results are incomplete";
        return LMFMM_ERR_TIMEOUT;
    }
    return LMFMM_OK;
}

lmfmm_status lmfmm_batch_info(const lmfmm_batch *b, int *merged, int64_t *nwork, int *variant, double *ms_variant)
{
    if (!b) return LMFMM_ERR_ARG;
    if (merged) *merged = b->merged;
    if (nwork) *nwork = b->nwork;
    if (variant) *variant = b->variant;
    if (ms_variant)
        for (int i = 0; i < 4; ++i) ms_variant[i] = b->ms_variant[i];
    return LMFMM_OK;
}

const char *lmfmm_batch_last_error(const lmfmm_batch *b) { return b ? b->err.c_str() : g_err.c_str(); }

void lmfmm_batch_destroy(lmfmm_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    batch_drop_graph(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->dprobs);
    cudaFree(b->dwork);
    cudaFree(b->status);
    delete b;
}

lmfmm_status lmfmm_check(lmfmm_ctx *ctx, void *stream)
{
    if (!ctx) return LMFMM_ERR_ARG;
    if (!ctx->built || !DS(ctx) || !DS(ctx)->mvstatus) {
        ctx->err = "check: call lmfmm_build first";
        return LMFMM_ERR_STATE;
    }
    CK(cudaSetDevice(ctx->device));
    return check_mvstatus(ctx, (cudaStream_t)stream);
}

lmfmm_status lmfmm_test_set_status(lmfmm_ctx *ctx, int bits)
{
    if (!ctx) return LMFMM_ERR_ARG;
    if (!ctx->built || !DS(ctx) || !DS(ctx)->mvstatus) {
        ctx->err = "test_set_status: call lmfmm_build first";
        return LMFMM_ERR_STATE;
    }
    CK(cudaSetDevice(ctx->device));
    int f = 0;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(&f, DS(ctx)->mvstatus, sizeof(int), cudaMemcpyDeviceToHost));
    f |= bits;
    CK(cudaMemcpy(DS(ctx)->mvstatus, &f, sizeof(int), cudaMemcpyHostToDevice));
    return LMFMM_OK;
}

lmfmm_status lmfmm_direct(lmfmm_ctx *ctx, const lmfmm_c128 *J, lmfmm_c128 *Phi, void *stream)
{
    if (!ctx) return LMFMM_ERR_ARG;
    if (!ctx->built) {
        ctx->err = "direct: call lmfmm_build first";
        return LMFMM_ERR_STATE;
    }
    if (!J || !Phi) {
        ctx->err = "direct: NULL buffer";
        return LMFMM_ERR_ARG;
    }
    CK(cudaSetDevice(ctx->device));
    DevState *d = DS(ctx);
    cudaStream_t st = (cudaStream_t)stream;
    // every (component, source leaf, target leaf) pair is treated as near
    int64_t npp = 0, cnt = 0;
    for (int ci = 0; ci < ctx->n_react_comps; ++ci)
        cnt += (ctx->lvl1[ctx->comps[ci].l][ctx->depth] - ctx->lvl0[ctx->comps[ci].l][ctx->depth]) *
               (ctx->lvl1[ctx->comps[ci].lp][ctx->depth] - ctx->lvl0[ctx->comps[ci].lp][ctx->depth]);
    std::vector<NearPair> all((size_t)cnt);
    all_leaf_pairs(ctx, all.data(), cnt, &npp);
    NearPair *dn = nullptr;
    cd *coef = nullptr;
    void *q1 = nullptr, *q2 = nullptr;
    CK(cudaMalloc(&q1, std::max<size_t>(1, all.size()) * sizeof(NearPair)));
    dn = (NearPair *)q1;
    if (cudaMalloc(&q2, std::max<int64_t>(1, npp) * 5 * sizeof(cd)) != cudaSuccess) {
        cudaFree(q1);
        ctx->err = "direct: coefficient allocation failed";
        return LMFMM_ERR_OOM;
    }
    coef = (cd *)q2;
    lmfmm_status rc = LMFMM_OK;
    if (!all.empty() &&
        cudaMemcpy(dn, all.data(), all.size() * sizeof(NearPair), cudaMemcpyHostToDevice))
        rc = LMFMM_ERR_CUDA;
    if (!rc) {
        double a = medium_a(ctx->med);
        cudaMemsetAsync(d->flag, 0, sizeof(int), st);
        launch_gather_in(ctx->N, d->perm, J, LMFMM_C128, d->qh, false, st);
        cudaMemsetAsync(d->ph, 0, (size_t)ctx->N * 3 * sizeof(cd), st);
        launch_s2t_pre((int64_t)all.size(), dn, d->boxes, d->xyz, ctx->med, d->comps, a,
                       ctx->prm.quad_node_cap, coef, d->flag, st);
        launch_s2t_apply((int64_t)all.size(), dn, d->boxes, d->xyz, coef, d->qh, d->ph, st);
        launch_scatter_out(ctx->N, d->perm, d->ph, Phi, LMFMM_C128, false, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = LMFMM_ERR_CUDA;
    }
    cudaFree(q1);
    cudaFree(q2);
    if (rc) {
        ctx->err = "direct: CUDA failure";
        return rc;
    }
    return check_flag(ctx);
}

lmfmm_status lmfmm_densities(lmfmm_ctx *ctx, int l, int lp, int64_t n, const lmfmm_c128 *krho,
                             lmfmm_c128 *out, void *stream)
{
    if (!ctx) return LMFMM_ERR_ARG;
    if (!ctx->layers_set) {
        ctx->err = "densities: call lmfmm_set_layers first";
        return LMFMM_ERR_STATE;
    }
    if (l < 0 || lp < 0 || l > ctx->med.L || lp > ctx->med.L || n < 0 || (n > 0 && (!krho || !out))) {
        ctx->err = "densities: layer index out of range or NULL buffer";
        return LMFMM_ERR_ARG;
    }
    if (ctx->med.L == 0) {
        ctx->err = "densities: no interfaces";
        return LMFMM_ERR_ARG;
    }
    CK(cudaSetDevice(ctx->device));
    launch_densities(ctx->med, l, lp, n, (const cd *)krho, (cd *)out, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return LMFMM_OK;
}

lmfmm_status lmfmm_m2l_table(lmfmm_ctx *ctx, int l, int lp, int tgt_up, int src_up, double rho,
                             double zs, double zt, lmfmm_c128 *out, void *stream)
{
    if (!ctx) return LMFMM_ERR_ARG;
    if (!ctx->layers_set) {
        ctx->err = "m2l_table: call lmfmm_set_layers first";
        return LMFMM_ERR_STATE;
    }
    const int L = ctx->med.L;
    if (L < 1 || l < 0 || lp < 0 || l > L || lp > L || !out || !(rho >= 0) ||
        (tgt_up && l > L - 1) || (!tgt_up && l < 1) || (src_up && lp < 1) || (!src_up && lp > L - 1)) {
        ctx->err = "m2l_table: no such reaction component or bad argument";
        return LMFMM_ERR_ARG;
    }
    CompDev c{};
    c.l = l;
    c.lp = lp;
    c.tu = tgt_up ? 1 : 0;
    c.su = src_up ? 1 : 0;
    c.s = comp_sign(l, lp, c.su);
    if (!(c.s * (zs - zt) > 0)) {
        ctx->err = "m2l_table: centres are not separated in the direction of the component";
        return LMFMM_ERR_ARG;
    }
    CK(cudaSetDevice(ctx->device));
    const int p = ctx->prm.p, T = (p + 1) * (p + 2) / 2;
    std::vector<double> B;
    int KM = (p + 1) / 2;
    bcoef_table(p, KM, B);
    std::vector<cd> G((size_t)T * T * (p + 2));
    gtensor(p, B, KM, zc(ctx->med.k[l].x, ctx->med.k[l].y), zc(ctx->med.k[lp].x, ctx->med.k[lp].y),
            G.data());
    if (!ctx->dev) ctx->dev = new DevState();
    DevState *d = DS(ctx);
    if (!d->flag) {
        CK(cudaMalloc((void **)&d->flag, sizeof(int)));
        d->allocs.push_back(d->flag);
        CK(cudaMemset(d->flag, 0, sizeof(int)));
    }
    std::vector<GeomDev> hg(1);
    hg[0].comp = 0;
    hg[0].src_primary = std::hypot(ctx->med.k[l].x, ctx->med.k[l].y) <=
                        std::hypot(ctx->med.k[lp].x, ctx->med.k[lp].y);
    hg[0].rho = rho;
    hg[0].zs = zs;
    hg[0].zt = zt;
    hg[0].plan = geom_plan(medium_a(ctx->med), p, rho, c.s * (zs - zt));
    hg[0].tab_index = 0;
    void *qc = nullptr, *qG = nullptr, *qi = nullptr;
    CK(cudaMalloc(&qc, sizeof(CompDev)));
    CK(cudaMalloc(&qG, G.size() * sizeof(cd)));
    CK(cudaMalloc(&qi, sizeof(int)));
    int zero = 0;
    CK(cudaMemcpy(qc, &c, sizeof(CompDev), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(qG, G.data(), G.size() * sizeof(cd), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(qi, &zero, sizeof(int), cudaMemcpyHostToDevice));
    lmfmm_status rc = tabulate(ctx, hg, (const CompDev *)qc, (const cd *)qG, (const int *)qi,
                               (cd *)out, (cudaStream_t)stream);
    cudaFree(qc);
    cudaFree(qG);
    cudaFree(qi);
    return rc;
}

lmfmm_status lmfmm_translation_matrix(int p, lmfmm_c128 k, const double *t, lmfmm_c128 *m2m,
                                      lmfmm_c128 *l2l)
{
    if (p < 1 || p > 16 || !t || !m2m || !l2l || !std::isfinite(t[0]) || !std::isfinite(t[1]) ||
        !std::isfinite(t[2])) {
        g_err = "translation_matrix: bad argument";
        return LMFMM_ERR_ARG;
    }
    std::vector<int64_t> goff;
    std::vector<int> gl;
    std::vector<double> gv;
    gaunt_table(p, goff, gl, gv);
    translation_matrix(p, zc(k.re, k.im), t, goff, gl, gv, (cd *)m2m, (cd *)l2l);
    return LMFMM_OK;
}

lmfmm_status lmfmm_free_m2l_table(int p, lmfmm_c128 k, double rho, double dz, lmfmm_c128 *tables,
                                   lmfmm_c128 *blocks)
{
    if (p < 1 || p > 16 || !tables || !(rho >= 0) || !std::isfinite(rho) || !std::isfinite(dz) ||
        !(rho > 0 || dz != 0)) {
        g_err = "free_m2l_table: bad argument";
        return LMFMM_ERR_ARG;
    }
    free_m2l_tables(p, zc(k.re, k.im), rho, dz, (cd *)tables, (cd *)blocks);
    return LMFMM_OK;
}

lmfmm_status lmfmm_get_stats(const lmfmm_ctx *ctx, lmfmm_stats *out)
{
    if (!ctx || !out) return LMFMM_ERR_ARG;
    lmfmm_ctx *c = (lmfmm_ctx *)ctx;
    *out = c->stats;
    DevState *d = DS(c);
    if (c->built && d && d->ev_ok && d->mv_recorded && cudaEventQuery(d->ev[7]) == cudaSuccess) {
        float ms;
        for (int i = 0; i < 6; ++i)
            if (cudaEventElapsedTime(&ms, d->ev[i], d->ev[i + 1]) == cudaSuccess) out->ms_stage[i] = ms;
        if (cudaEventElapsedTime(&ms, d->ev[6], d->ev[7]) == cudaSuccess) out->ms_stage[6] = ms;
        if (cudaEventElapsedTime(&ms, d->ev[0], d->ev[7]) == cudaSuccess) out->ms_stage[7] = ms;
    }
    return LMFMM_OK;
}

const char *lmfmm_last_error(const lmfmm_ctx *ctx)
{
    if (!ctx) return g_err.c_str();
    return ctx->err.c_str();
}

void lmfmm_destroy(lmfmm_ctx *ctx)
{
    if (!ctx) return;
    free_dev(ctx);
    delete ctx;
}

}  // extern "C"
