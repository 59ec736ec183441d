// stereo_api.cu -- host side of the C ABI declared in include/stereo.h: argument
// checks, context lifetime (staging buffers, tensor maps, scratch), error reporting.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "internal.cuh"

namespace sgb {

static thread_local char g_err[512] = "no error";

int set_error(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_error(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return STEREO_OK;
    cudaGetLastError();   // clear the sticky-free error state of the runtime
    return set_error(e == cudaErrorMemoryAllocation ? STEREO_ENOMEM : STEREO_ECUDA,
                     "%s: %s", what, cudaGetErrorString(e));
}

static int round_up(int x, int a) { return (x + a - 1) / a * a; }

int compute_geometry(const stereo_params &p, int dc, int wc, Geometry &g)
{
    g.W = p.width;
    g.H = p.height;
    g.pitch = p.pitch;
    g.D = p.max_disp;
    g.rw = p.win / 2;
    g.rb = p.bil / 2;
    g.m = g.rw + g.rb;
    g.n = p.win * p.win;
    g.dc = dc;
    g.wc = wc;
    g.tx = tile_x(wc);
    g.ty = tile_y(wc);
    g.esize = p.cost_dtype == STEREO_F32 ? 4 : 2;
    // the screened form's FP32 refinement computes 16 disparities from any start d <= D - 1,
    // so its target strip holds 16 disparities beyond the last screening chunk
    g.Dp = wc == kScWC ? round_up(g.D, dc) + 16 : round_up(g.D, dc);
    g.ntx = (g.W + g.tx - 1) / g.tx;
    g.nty = (g.H + g.ty - 1) / g.ty;
    g.pad_left = round_up(g.m + g.Dp - 1, 16);
    g.pad_top = g.m;
    g.ref_e = round_up(g.m, 16) - g.m;
    g.ref_box_w = round_up(g.ref_e + g.tx + 2 * g.m, 16);
    g.tgt_e = g.pad_left - (g.m + g.Dp - 1);
    g.tgt_box_w = round_up(g.tgt_e + g.tx + 2 * g.m + g.Dp - 1, 16);
    g.box_h = g.ty + 2 * g.m;
    const int x_last = (g.ntx - 1) * g.tx;
    int end_ref = x_last + g.pad_left - round_up(g.m, 16) + g.ref_box_w;
    int end_tgt = x_last + g.tgt_box_w;
    g.pad_w = round_up((end_ref > end_tgt ? end_ref : end_tgt), 16);
    g.pad_h = g.nty * g.ty + 2 * g.m;
    g.pad_pitch = round_up(g.pad_w, 128);
    g.smem_bytes = fused_smem_bytes(g);
    return STEREO_OK;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// A row of the padded image seen as 16-byte chunks: dims {16, pad_w/16, pad_h}, so one
// box of {16, box_w/16, box_h} lands in shared memory as box_h rows of box_w bytes.
static int make_tensor_map(CUtensorMap *map, void *base, const Geometry &g, int box_w)
{
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                          cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return set_error(STEREO_ECUDA, "cuTensorMapEncodeTiled entry point not found");
        encode = (EncodeTiledFn)fn;
    }
    cuuint64_t dims[3] = {16, (cuuint64_t)(g.pad_w / 16), (cuuint64_t)g.pad_h};
    cuuint64_t strides[2] = {16, (cuuint64_t)g.pad_pitch};
    cuuint32_t box[3] = {16, (cuuint32_t)(box_w / 16), (cuuint32_t)g.box_h};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(STEREO_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return STEREO_OK;
}

static void free_ctx(stereo_ctx *c)
{
    if (!c) return;
    cudaFree(c->ref_pad);
    cudaFree(c->tgt_pad);
    cudaFree(c->ref_stats);
    cudaFree(c->tgt_stats);
    cudaFree(c->row_tab);
    cudaFree(c->mom_part);
    cudaFree(c->dt_coef);
    cudaFree(c->res_dev);
    cudaFree(c->status_dev);
    cudaFree(c->lr_ref);
    cudaFree(c->lr_tgt);
    cudaFree(c->lr_wta);
    cudaFree(c->lr_disp);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    delete c;
}

}  // namespace sgb

using namespace sgb;

extern "C" {

const char *stereo_last_error(void) { return g_err; }

const char *stereo_version(void) { return "paper_1904_06017_gb300 0.1 (sm_103a)"; }

int stereo_params_default(stereo_params *p)
{
    if (!p) return set_error(STEREO_EINVAL, "stereo_params_default: null pointer");
    memset(p, 0, sizeof(*p));
    p->win = 9;
    p->bil = 11;
    p->sigma0 = 1.5f;
    p->sigma1 = 5.5f;
    p->cost_dtype = STEREO_F32;
    p->lambda0 = 10.0;
    p->delta_psi = M_PI / 1.8e6;
    p->max_iters = 100;
    return STEREO_OK;
}

int stereo_create(const stereo_params *p, stereo_ctx **out)
{
    int rc = create_context(p, 0, 0, out);
    if (rc) return rc;
    stereo_ctx *c = *out;
    const size_t img = (size_t)c->p.height * c->p.pitch, map = (size_t)c->p.height * c->p.width;
    if ((rc = cuda_error(cudaMalloc(&c->lr_ref, img), "cudaMalloc lr_ref")) ||
        (rc = cuda_error(cudaMalloc(&c->lr_tgt, img), "cudaMalloc lr_tgt")) ||
        (rc = cuda_error(cudaMalloc(&c->lr_wta, map * sizeof(int32_t)), "cudaMalloc lr_wta")) ||
        (rc = cuda_error(cudaMalloc(&c->lr_disp, map * sizeof(float)), "cudaMalloc lr_disp"))) {
        free_ctx(c);
        *out = nullptr;
        return rc;
    }
    return STEREO_OK;
}

}  // extern "C"

namespace sgb {

int max_smem_optin()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

// Static shared memory of the fused kernel (pair arguments, work item) on top of the dynamic part.
constexpr int kFusedStaticSmem = 2048;

int create_context(const stereo_params *p, int force_dc, int force_wc, stereo_ctx **out)
{
    if (!p || !out) return set_error(STEREO_EINVAL, "stereo_create: null pointer");
    *out = nullptr;
    if (p->width < 1 || p->height < 1 || p->width > kMaxDim || p->height > kMaxDim)
        return set_error(STEREO_EINVAL, "stereo_create: image size %dx%d outside 1..%d",
                         p->width, p->height, kMaxDim);
    if (p->pitch < p->width || p->pitch % 16 != 0)
        return set_error(STEREO_EINVAL, "stereo_create: pitch %d must be >= width and a multiple of 16",
                         p->pitch);
    if (p->max_disp < 1 || p->max_disp > kMaxD)
        return set_error(STEREO_EINVAL, "stereo_create: max_disp %d outside 1..%d", p->max_disp, kMaxD);
    if (p->win < 3 || p->win > 2 * kMaxRW + 1 || p->win % 2 == 0)
        return set_error(STEREO_EINVAL, "stereo_create: win %d must be odd in 3..%d", p->win,
                         2 * kMaxRW + 1);
    if (p->bil < 1 || p->bil > 2 * kMaxRB + 1 || p->bil % 2 == 0)
        return set_error(STEREO_EINVAL, "stereo_create: bil %d must be odd in 1..%d", p->bil,
                         2 * kMaxRB + 1);
    if (!(p->sigma0 > 0.f) || !(p->sigma1 > 0.f) || !isfinite(p->sigma0) || !isfinite(p->sigma1))
        return set_error(STEREO_EINVAL, "stereo_create: sigma0, sigma1 must be positive and finite");
    if (p->cost_dtype != STEREO_F32 && p->cost_dtype != STEREO_F16 && p->cost_dtype != STEREO_BF16)
        return set_error(STEREO_EINVAL, "stereo_create: unknown cost_dtype %d", p->cost_dtype);
    if (p->fused_form < STEREO_FUSED_AUTO || p->fused_form > STEREO_FUSED_TENSOR)
        return set_error(STEREO_EINVAL, "stereo_create: fused_form %d outside 0..2", p->fused_form);
    if (!(p->lambda0 > 0.0) || !(p->delta_psi > 0.0) || p->max_iters < 1 || p->max_iters > 100000)
        return set_error(STEREO_EINVAL, "stereo_create: lambda0, delta_psi must be > 0 and max_iters in 1..100000");

    stereo_ctx *c = new (std::nothrow) stereo_ctx();
    if (!c) return set_error(STEREO_ENOMEM, "stereo_create: host allocation failed");
    c->p = *p;
    int rc;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || c->nsm < 1) {
        free_ctx(c);
        return cuda_error(cudaErrorNoDevice, "stereo_create: no CUDA device");
    }
    // The fused form (stereo_params.fused_form): FP16 / BF16 storage takes the tensor-core form
    // (16 disparities per chunk) where it applies, FP32 storage the screened form (32 per
    // chunk); otherwise the SIMT form with 12 disparities per chunk when its shared memory
    // allows it, else 4
    const int smem_max = max_smem_optin() - kFusedStaticSmem;
    const bool want_tensor = p->fused_form != STEREO_FUSED_SIMT;
    // the kScWC tiles take every storage type up to bil = 13 (the 64 x 36 tensor-core form, whose
    // weights are formed in 16-bit arithmetic, stays a batch tile choice)
    const bool sc = !force_wc && !force_dc && want_tensor && p->bil / 2 <= kScMaxRB;
    const bool tc = !force_wc && !force_dc && want_tensor && !sc && tc_supported(p->cost_dtype, p->bil, p->sigma1);
    if (p->fused_form == STEREO_FUSED_TENSOR && !force_wc && !tc && !sc) {
        free_ctx(c);
        return set_error(STEREO_ENOTSUP, "stereo_create: no tensor-core form for cost_dtype %d, bil %d, sigma1 %g",
                         p->cost_dtype, p->bil, (double)p->sigma1);
    }
    const int wc = force_wc ? force_wc : tc ? kTcWC : sc ? kScWC : kDefaultWC;
    compute_geometry(*p, force_dc ? force_dc : tc ? 16 : sc ? 32 : 12, wc, c->g);
    if ((tc || sc) && (int)c->g.smem_bytes > smem_max) compute_geometry(*p, 12, kDefaultWC, c->g);
    if (!force_dc && c->g.wc != kTcWC && (int)c->g.smem_bytes > smem_max) compute_geometry(*p, 4, c->g.wc, c->g);
    if ((int)c->g.smem_bytes > smem_max) {
        free_ctx(c);
        return set_error(STEREO_ENOTSUP, "stereo_create: fused kernel needs %zu B of shared memory (max %d)",
                         c->g.smem_bytes, smem_max);
    }
    const Geometry &g = c->g;
    size_t img = (size_t)g.pad_pitch * g.pad_h;
    size_t st = (size_t)g.pad_w * g.pad_h * sizeof(int2);
    if ((rc = cuda_error(cudaMalloc(&c->ref_pad, img), "cudaMalloc ref_pad")) ||
        (rc = cuda_error(cudaMalloc(&c->tgt_pad, img), "cudaMalloc tgt_pad")) ||
        (rc = cuda_error(cudaMalloc(&c->ref_stats, st), "cudaMalloc ref_stats")) ||
        (rc = cuda_error(cudaMalloc(&c->tgt_stats, st), "cudaMalloc tgt_stats")) ||
        (rc = cuda_error(cudaMalloc(&c->row_tab, sizeof(int4) * g.H), "cudaMalloc row table")) ||
        (rc = cuda_error(cudaMalloc(&c->mom_part, sizeof(double) * 10 * kDtMaxBlocks), "cudaMalloc moments")) ||
        (rc = cuda_error(cudaMalloc(&c->res_dev, sizeof(stereo_dt_result)), "cudaMalloc result")) ||
        (rc = cuda_error(cudaMalloc(&c->dt_coef, 4 * sizeof(float)), "cudaMalloc coefficients")) ||
        (rc = cuda_error(cudaMalloc(&c->status_dev, sizeof(int)), "cudaMalloc status")) ||
        (rc = cuda_error(cudaMemset(c->ref_pad, 0, img), "cudaMemset")) ||
        (rc = cuda_error(cudaMemset(c->tgt_pad, 0, img), "cudaMemset")) ||
        (rc = cuda_error(cudaMemset(c->status_dev, 0, sizeof(int)), "cudaMemset"))) {
        free_ctx(c);
        return rc;
    }
    if ((rc = make_tensor_map(&c->tmap_ref, c->ref_pad, g, g.ref_box_w)) ||
        (rc = make_tensor_map(&c->tmap_tgt, c->tgt_pad, g, g.tgt_box_w))) {
        free_ctx(c);
        return rc;
    }
    // eq. (omega0) / eq. (omega1) folded into one base-2 exponent:
    // w = 2^(K[dx][dy] - (I_q*s - I_p*s)^2) with K = -log2(e) |dq|^2 / sigma0^2, s = sqrt(log2(e)) / sigma1
    const double log2e = 1.4426950408889634;
    const int kb = 2 * g.rb + 1;
    for (int i = 0; i < kb; ++i)
        for (int j = 0; j < kb; ++j) {
            double dx = i - g.rb, dy = j - g.rb;
            c->kspatial[i * kb + j] = (float)(-log2e * (dx * dx + dy * dy) / ((double)p->sigma0 * p->sigma0));
        }
    c->iscale = (float)(sqrt(log2e) / (double)p->sigma1);
    if ((rc = fused_configure(c))) {
        free_ctx(c);
        return rc;
    }
    *out = c;
    return STEREO_OK;
}

}  // namespace sgb

extern "C" {

int stereo_destroy(stereo_ctx *ctx)
{
    if (!ctx) return STEREO_OK;
    cudaDeviceSynchronize();
    free_ctx(ctx);
    return STEREO_OK;
}

int stereo_row_shift_affine(int32_t height, double c0, double c1, double delta_p, float *shift_host_out)
{
    if (height < 1 || !shift_host_out)
        return set_error(STEREO_EINVAL, "stereo_row_shift_affine: bad height or null output");
    for (int v = 0; v < height; ++v) shift_host_out[v] = (float)(c0 + c1 * v - delta_p);
    return STEREO_OK;
}

int stereo_warp_target(stereo_ctx *ctx, const uint8_t *tgt, const float *shift, uint8_t *out,
                       stereo_stream_t stream)
{
    if (!ctx || !tgt || !shift || !out) return set_error(STEREO_EINVAL, "stereo_warp_target: null pointer");
    if (tgt == out) return set_error(STEREO_EINVAL, "stereo_warp_target: input and output alias");
    if (((uintptr_t)tgt | (uintptr_t)out) % 16)
        return set_error(STEREO_EINVAL, "stereo_warp_target: images must be 16-byte aligned");
    return launch_warp(ctx, tgt, shift, out, (cudaStream_t)stream);
}

int stereo_cost_aggregate_wta(stereo_ctx *ctx, const uint8_t *ref, const uint8_t *tgtw,
                              const float *shift, float *disp, int32_t *wta, uint8_t *valid,
                              stereo_stream_t stream)
{
    return stereo_cost_aggregate_wta_ex(ctx, ref, tgtw, shift, disp, wta, valid, nullptr, stream);
}

int stereo_cost_aggregate_wta_ex(stereo_ctx *ctx, const uint8_t *ref, const uint8_t *tgtw,
                                 const float *shift, float *disp, int32_t *wta, uint8_t *valid,
                                 float *best2, stereo_stream_t stream)
{
    if (!ctx || !ref || !tgtw || !shift || !disp)
        return set_error(STEREO_EINVAL, "stereo_cost_aggregate_wta: null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = launch_prep(ctx, ref, tgtw, s);
    if (!rc) rc = launch_row_tables(ctx, shift, tgtw, s);
    if (rc) return rc;
    int slot = -1;
    if (ctx->prof_on && ctx->prof_n < kProfSlots) {
        slot = ctx->prof_n++;
        cudaEventRecord(ctx->prof_ev[2 * slot], s);
    }
    rc = launch_fused(ctx, shift, disp, wta, valid, s, best2);
    if (slot >= 0) cudaEventRecord(ctx->prof_ev[2 * slot + 1], s);
    return rc;
}

int stereo_disparity_transform(stereo_ctx *ctx, const float *disp, const uint8_t *mask,
                               double psi_init, float delta_t, float *out, stereo_dt_result *res,
                               stereo_stream_t stream)
{
    if (!ctx || !disp || !out) return set_error(STEREO_EINVAL, "stereo_disparity_transform: null pointer");
    if (!isfinite(psi_init) || !isfinite(delta_t))
        return set_error(STEREO_EINVAL, "stereo_disparity_transform: psi_init and delta_t must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    bool host_res = false;
    if (res) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, res) != cudaSuccess) {
            cudaGetLastError();
            host_res = true;
        } else {
            host_res = !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
        }
    }
    stereo_dt_result *rd = (res && !host_res) ? res : ctx->res_dev;
    int rc = launch_dt(ctx, disp, mask, psi_init, delta_t, out, rd, s);
    if (rc) return rc;
    if (host_res) {
        rc = cuda_error(cudaMemcpyAsync(res, rd, sizeof(stereo_dt_result), cudaMemcpyDeviceToHost, s),
                        "stereo_disparity_transform: copy result");
        if (rc) return rc;
        rc = cuda_error(cudaStreamSynchronize(s), "stereo_disparity_transform: synchronize");
    }
    return rc;
}

int stereo_cost_volume(stereo_ctx *ctx, const uint8_t *ref, const uint8_t *tgtw, float *cost,
                       stereo_stream_t stream)
{
    if (!ctx || !ref || !tgtw || !cost) return set_error(STEREO_EINVAL, "stereo_cost_volume: null pointer");
    int rc = launch_prep(ctx, ref, tgtw, (cudaStream_t)stream);
    if (rc) return rc;
    return launch_cost_volume(ctx, cost, (cudaStream_t)stream);
}

int stereo_aggregate_volume(stereo_ctx *ctx, const uint8_t *ref, const float *cost, float *agg,
                            stereo_stream_t stream)
{
    if (!ctx || !ref || !cost || !agg) return set_error(STEREO_EINVAL, "stereo_aggregate_volume: null pointer");
    if ((const void *)cost == (const void *)agg)
        return set_error(STEREO_EINVAL, "stereo_aggregate_volume: cost and agg alias");
    return launch_aggregate_volume(ctx, ref, cost, agg, (cudaStream_t)stream);
}

int stereo_wta_volume(stereo_ctx *ctx, const float *agg, const float *shift, float *disp,
                      int32_t *wta, float *best2, stereo_stream_t stream)
{
    if (!ctx || !agg || !shift || !disp) return set_error(STEREO_EINVAL, "stereo_wta_volume: null pointer");
    return launch_wta_volume(ctx, agg, shift, disp, wta, best2, (cudaStream_t)stream);
}

int stereo_check_device_status(stereo_ctx *ctx, stereo_stream_t stream)
{
    if (!ctx) return set_error(STEREO_EINVAL, "stereo_check_device_status: null pointer");
    int h = 0;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = cuda_error(cudaMemcpyAsync(&h, ctx->status_dev, sizeof(int), cudaMemcpyDeviceToHost, s),
                        "stereo_check_device_status: copy");
    if (!rc) rc = cuda_error(cudaMemsetAsync(ctx->status_dev, 0, sizeof(int), s), "stereo_check_device_status: clear");
    if (!rc) rc = cuda_error(cudaStreamSynchronize(s), "stereo_check_device_status: synchronize");
    if (rc) return rc;
    if (h) return set_error(STEREO_ETIMEOUT, "a kernel gave up a bounded wait (status word 0x%x)", h);
    return STEREO_OK;
}

int stereo_debug_stall_staging(stereo_ctx *ctx, int32_t on)
{
    if (!ctx) return set_error(STEREO_EINVAL, "stereo_debug_stall_staging: null pointer");
    ctx->stall_test = on ? 1 : 0;
    return STEREO_OK;
}

int stereo_profile_enable(stereo_ctx *ctx, int32_t on)
{
    if (!ctx) return set_error(STEREO_EINVAL, "stereo_profile_enable: null pointer");
    if (on && ctx->prof_ev.empty()) {
        ctx->prof_ev.resize(2 * kProfSlots);
        for (auto &e : ctx->prof_ev) {
            int rc = cuda_error(cudaEventCreate(&e), "cudaEventCreate");
            if (rc) return rc;
        }
    }
    ctx->prof_on = on ? 1 : 0;
    ctx->prof_n = 0;
    return STEREO_OK;
}

int stereo_profile_read(stereo_ctx *ctx, int32_t *launches, double *total_ms)
{
    if (!ctx || !launches || !total_ms) return set_error(STEREO_EINVAL, "stereo_profile_read: null pointer");
    double tot = 0.0;
    for (int i = 0; i < ctx->prof_n; ++i) {
        int rc = cuda_error(cudaEventSynchronize(ctx->prof_ev[2 * i + 1]), "cudaEventSynchronize");
        if (rc) return rc;
        float ms = 0.f;
        rc = cuda_error(cudaEventElapsedTime(&ms, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]),
                        "cudaEventElapsedTime");
        if (rc) return rc;
        tot += ms;
    }
    *launches = ctx->prof_n;
    *total_ms = tot;
    ctx->prof_n = 0;
    return STEREO_OK;
}

int stereo_fp32_peak_probe(int32_t blocks_per_sm, double *gflops_scalar, double *gflops_packed)
{
    if (!gflops_scalar || !gflops_packed || blocks_per_sm < 1 || blocks_per_sm > 8)
        return set_error(STEREO_EINVAL, "stereo_fp32_peak_probe: bad argument");
    return run_fp32_probe(blocks_per_sm, gflops_scalar, gflops_packed);
}

}  // extern "C"
