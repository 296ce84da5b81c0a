// lmfmm_direct_noalloc: the all-pairs direct evaluation of lmfmm_direct for
// callers that cannot allocate device memory while they run -- for example
// a program whose device memory is entirely reserved by another allocator
// (a framework's caching pool), or one that must not stall or fail on an
// allocation in the middle of a computation.  Its scratch (the list of leaf
// pairs and the per-pair Sommerfeld coefficients) lives in one file-scope
// device array of fixed size instead of memory obtained from cudaMalloc.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "kernels.cuh"

using namespace lmf;

// Scratch shared by every call on a device: 32 MiB, aligned for any record.
#define LMF_NOALLOC_BYTES (32u << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[LMF_NOALLOC_BYTES];

namespace {

// Host-side stand-in for the pair list, so that building it allocates
// nothing either; its capacity bounds the number of (component, leaf pair)
// records a call may use.  h_pairs, the address cache below and the device
// scratch are process-wide: g_lock serialises whole calls (pair list, copy,
// kernels, wait), on every device and context.
constexpr int64_t kMaxPairs = 1 << 16;
NearPair h_pairs[kMaxPairs];
std::mutex g_lock;

// Device address of g_noalloc_scratch, looked up once per device with that
// device current (the symbol name in host code is only a stand-in).
constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices];

lmfmm_status scratch_address(lmfmm_ctx *ctx, void **out)
{
    if (ctx->device < 0 || ctx->device >= kMaxDevices) {
        ctx->err = "direct_noalloc: device index out of range";
        return LMFMM_ERR_ARG;
    }
    if (!g_scratch_ptr[ctx->device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            ctx->err = std::string("direct_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return LMFMM_ERR_CUDA;
        }
        g_scratch_ptr[ctx->device] = p;
    }
    *out = g_scratch_ptr[ctx->device];
    return LMFMM_OK;
}

}  // namespace

// device-state accessors provided by api.cu
namespace lmf {
bool noalloc_state(lmfmm_ctx *ctx, const int64_t **perm, const BoxDev **boxes, const double **xyz,
                   const CompDev **comps, cd **qh, cd **ph, int **flag);
}

extern "C" lmfmm_status lmfmm_direct_noalloc(lmfmm_ctx *ctx, const lmfmm_c128 *J,
                                             lmfmm_c128 *Phi, void *stream)
{
    if (!ctx) return LMFMM_ERR_ARG;
    if (!ctx->built) {
        ctx->err = "direct_noalloc: call lmfmm_build first";
        return LMFMM_ERR_STATE;
    }
    if (!J || !Phi) {
        ctx->err = "direct_noalloc: NULL buffer";
        return LMFMM_ERR_ARG;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) {
        ctx->err = std::string("direct_noalloc: cudaSetDevice: ") + cudaGetErrorString(e);
        return LMFMM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> hold(g_lock);
    void *scratch = nullptr;
    lmfmm_status s = scratch_address(ctx, &scratch);
    if (s) return s;
    const int64_t *perm;
    const BoxDev *boxes;
    const double *xyz;
    const CompDev *comps;
    cd *qh, *ph;
    int *flag;
    if (!noalloc_state(ctx, &perm, &boxes, &xyz, &comps, &qh, &ph, &flag)) {
        ctx->err = "direct_noalloc: context has no device state";
        return LMFMM_ERR_STATE;
    }
    // every (component, source leaf, target leaf) pair, as in lmfmm_direct
    int64_t npp = 0;
    const int64_t np = all_leaf_pairs(ctx, h_pairs, kMaxPairs, &npp);
    if (np < 0) {
        ctx->err = "direct_noalloc: more than " + std::to_string(kMaxPairs) +
                   " leaf pairs (use lmfmm_direct)";
        return LMFMM_ERR_ARG;
    }
    // layout in the scratch: pair records, then 5 complex coefficients per point pair
    size_t off_pairs = 0;
    size_t off_coef = ((size_t)np * sizeof(NearPair) + 255) & ~(size_t)255;
    size_t need = off_coef + (size_t)npp * 5 * sizeof(cd);
    if (need > LMF_NOALLOC_BYTES) {
        ctx->err = "direct_noalloc: needs " + std::to_string(need) + " bytes of scratch, limit " +
                   std::to_string((size_t)LMF_NOALLOC_BYTES) + " (use lmfmm_direct)";
        return LMFMM_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    NearPair *dpairs = (NearPair *)((unsigned char *)scratch + off_pairs);
    cd *coef = (cd *)((unsigned char *)scratch + off_coef);
    if (np > 0 && (e = cudaMemcpyAsync(dpairs, h_pairs, (size_t)np * sizeof(NearPair),
                                       cudaMemcpyHostToDevice, st)) != cudaSuccess) {
        ctx->err = std::string("direct_noalloc: copy of the pair list: ") + cudaGetErrorString(e);
        return LMFMM_ERR_CUDA;
    }
    const double a = medium_a(ctx->med);
    // the coefficient range is zero-filled by the precomputation kernel itself,
    // the helical result buffer and the quadrature flag here
    cudaMemsetAsync(flag, 0, sizeof(int), st);
    launch_gather_in(ctx->N, perm, J, LMFMM_C128, qh, false, st);
    cudaMemsetAsync(ph, 0, (size_t)ctx->N * 3 * sizeof(cd), st);
    launch_s2t_pre(np, dpairs, boxes, xyz, ctx->med, comps, a, ctx->prm.quad_node_cap, coef, flag, st);
    launch_s2t_apply(np, dpairs, boxes, xyz, coef, qh, ph, st);
    launch_scatter_out(ctx->N, perm, ph, Phi, LMFMM_C128, false, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) {
        ctx->err = std::string("direct_noalloc: ") + cudaGetErrorString(e);
        return LMFMM_ERR_CUDA;
    }
    int f = 0;
    if ((e = cudaMemcpy(&f, flag, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) {
        ctx->err = std::string("direct_noalloc: ") + cudaGetErrorString(e);
        return LMFMM_ERR_CUDA;
    }
    if (f) {
        ctx->err = "direct_noalloc: device quadrature hit its cap";
        return LMFMM_ERR_QUAD;
    }
    return LMFMM_OK;
}
