// dt_noalloc.cu -- the disparity transformation without any device allocation.
//
// Some callers cannot allocate device memory at all: code that runs inside a memory
// pool or arena owned by someone else (a host framework that has reserved the whole
// device heap up front), real-time loops where a cudaMalloc could block on a device-wide
// synchronisation and miss a frame deadline, and plug-ins whose host forbids allocation
// after start-up.  stereo_create allocates (staging images, statistics, scratch), so such
// callers get this one entry point instead: the same three kernels as
// stereo_disparity_transform, with their scratch (the per-block partial moments and the
// three coefficients of the final map) in a fixed array that lives in the library's
// device image.  The caller still provides every input and output buffer.
#include <mutex>

#include "internal.cuh"

namespace sgb {

// Scratch of the no-allocation path: kDtMaxBlocks partial moment sets (10 doubles each),
// then 4 floats of coefficients (2 doubles), then room for one stereo_dt_result (6
// doubles) used when the caller passes none.  80 KiB + 64 B, resident on every device
// that loads the library until the process exits.
constexpr size_t kNoAllocMoments = (size_t)kDtMaxBlocks * 10;
static __device__ __align__(256) double g_dt_scratch[kNoAllocMoments + 8];
static_assert(sizeof(stereo_dt_result) <= 6 * sizeof(double), "result slot too small");

// Device address of g_dt_scratch, cached per device together with the unique id of the
// context it was looked up in.  A context that is destroyed and re-created (cudaDeviceReset,
// a reset of the primary context) reloads the library's module at a new address and gets a
// new id (ids are never reused within a process), so a changed id forces a new lookup
// instead of handing the kernels a stale address.  The two driver calls that read the id
// are fetched through the runtime, so the library keeps no link-time dependency on libcuda.
constexpr int kMaxDevices = 64;
struct ScratchSlot {
    unsigned long long ctx_id;   // 0: not looked up yet
    void *ptr;
};
static std::mutex g_scratch_mu;
static ScratchSlot g_scratch[kMaxDevices];

typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);

// The current context's unique id, or 0 when it cannot be read (then every call looks the
// address up again, which is always correct).
static unsigned long long current_context_id()
{
    static std::once_flag once;
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

static int scratch_for_current_device(void **out)
{
    int dev = 0;
    int rc = cuda_error(cudaGetDevice(&dev), "stereo_disparity_transform_noalloc: cudaGetDevice");
    if (rc) return rc;
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(STEREO_ENOTSUP, "stereo_disparity_transform_noalloc: device %d beyond %d", dev, kMaxDevices);
    // the id is read only once a lookup has run: cudaGetSymbolAddress makes the device's
    // primary context current on the first call, so before it there may be no context to read
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchSlot &slot = g_scratch[dev];
    unsigned long long id = slot.ctx_id ? current_context_id() : 0;
    if (!slot.ctx_id || id == 0 || id != slot.ctx_id) {
        void *p = nullptr;
        rc = cuda_error(cudaGetSymbolAddress(&p, g_dt_scratch),
                        "stereo_disparity_transform_noalloc: cudaGetSymbolAddress");
        if (rc) return rc;
        slot.ptr = p;
        slot.ctx_id = current_context_id();   // 0 when unreadable: look up again next call
    }
    *out = slot.ptr;
    return STEREO_OK;
}

}  // namespace sgb

using namespace sgb;

extern "C" int stereo_disparity_transform_noalloc(int32_t width, int32_t height, const float *disp,
                                                  const uint8_t *mask, double psi_init, float delta_t,
                                                  double lambda0, double delta_psi, int32_t max_iters,
                                                  float *out, stereo_dt_result *res_dev,
                                                  stereo_stream_t stream)
{
    if (!disp || !out) return set_error(STEREO_EINVAL, "stereo_disparity_transform_noalloc: null pointer");
    if (width < 1 || height < 1 || width > kMaxDim || height > kMaxDim)
        return set_error(STEREO_EINVAL,
                         "stereo_disparity_transform_noalloc: map size %dx%d outside 1..%d (the fixed "
                         "scratch holds %d partial-moment blocks, enough for any map up to that size)",
                         width, height, kMaxDim, kDtMaxBlocks);
    if (!isfinite(psi_init) || !isfinite(delta_t) || !(lambda0 > 0.0) || !(delta_psi > 0.0) ||
        max_iters < 1 || max_iters > 100000)
        return set_error(STEREO_EINVAL, "stereo_disparity_transform_noalloc: bad search parameters");
    void *base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc) return rc;
    double *part = static_cast<double *>(base);
    float *coef = reinterpret_cast<float *>(part + kNoAllocMoments);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = (size_t)width * height;
    const int nb = dt_moment_blocks(N);
    // every partial block that the solve reads is written first by k_dt_moments, and the
    // coefficients are written by k_dt_solve before k_dt_apply reads them: nothing in the
    // scratch has to start at zero
    k_dt_moments<<<nb, kDtThreads, 0, s>>>(disp, mask, width, height, part);
    if ((rc = cuda_error(cudaGetLastError(), "stereo_disparity_transform_noalloc: moments launch"))) return rc;
    // without res_dev the full result goes to its own slot at the end of the scratch
    stereo_dt_result *r = res_dev ? res_dev : reinterpret_cast<stereo_dt_result *>(part + kNoAllocMoments + 2);
    k_dt_solve<<<1, kDtThreads, 0, s>>>(part, nb, width, height, psi_init, lambda0, delta_psi, max_iters,
                                        delta_t, r, coef);
    if ((rc = cuda_error(cudaGetLastError(), "stereo_disparity_transform_noalloc: solve launch"))) return rc;
    dim3 block(128), grid((width + 4 * 128 - 1) / (4 * 128), height);   // 4 pixels per thread where aligned
    k_dt_apply<<<grid, block, 0, s>>>(disp, width, height, coef, out);
    return cuda_error(cudaGetLastError(), "stereo_disparity_transform_noalloc: apply launch");
}
