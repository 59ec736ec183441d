// batch.cu -- batches of stereo pairs of uneven sizes and search ranges: per-pair staging
// contexts, one persistent fused launch over a heaviest-first (pair, tile) work list, the
// whole batch captured once into a CUDA graph, and the tile autotuner with its JSON cache.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "k_fused_common.cuh"

struct stereo_batch {
    stereo_batch_params bp;
    std::vector<stereo_pair_desc> pairs;
    std::vector<stereo_ctx *> ctx;
    int wc = 0, dc = 0, source = 0;
    sgb::FusedKernel kernel = nullptr;
    size_t smem = 0;
    int nsm = 0;
    sgb::PairDesc *d_pairs = nullptr;
    int2 *d_items = nullptr;
    int *d_counter = nullptr;
    int nitems = 0;
    cudaStream_t cap = nullptr;
    // side streams of the capture: the per-pair launches before and after the fused
    // kernel form independent chains of the graph, so the small kernels of different
    // pairs (single-block roll searches among them) run side by side
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace sgb {

constexpr int kBatchBranches = 16;   // side streams of the captured graph

static void release_build(stereo_batch *b)
{
    for (stereo_ctx *c : b->ctx) stereo_destroy(c);
    b->ctx.clear();
    cudaFree(b->d_pairs);
    cudaFree(b->d_items);
    cudaFree(b->d_counter);
    b->d_pairs = nullptr;
    b->d_items = nullptr;
    b->d_counter = nullptr;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

static stereo_params pair_params(const stereo_batch_params &bp, const stereo_pair_desc &d)
{
    stereo_params p;
    stereo_params_default(&p);
    p.width = d.width;
    p.height = d.height;
    p.pitch = d.pitch;
    p.max_disp = d.max_disp;
    p.win = bp.win;
    p.bil = bp.bil;
    p.sigma0 = bp.sigma0;
    p.sigma1 = bp.sigma1;
    p.cost_dtype = bp.cost_dtype;
    p.lambda0 = bp.lambda0;
    p.delta_psi = bp.delta_psi;
    p.max_iters = bp.max_iters;
    return p;
}

// Contexts, descriptors and the work list for one tile configuration.
static int build(stereo_batch *b, int wc, int dc)
{
    release_build(b);
    int rc;
    const int n = (int)b->pairs.size();
    for (int i = 0; i < n; ++i) {
        stereo_params p = pair_params(b->bp, b->pairs[i]);
        stereo_ctx *c = nullptr;
        if ((rc = create_context(&p, dc, wc, &c))) {
            release_build(b);
            return rc;
        }
        b->ctx.push_back(c);
    }
    b->wc = wc;
    b->dc = dc;
    b->kernel = pick_fused(b->bp.cost_dtype, b->bp.bil / 2, dc, wc);
    if (!b->kernel) {
        release_build(b);
        return set_error(STEREO_ENOTSUP, "batch: no fused kernel for bil=%d dc=%d wc=%d type=%d", b->bp.bil, dc,
                         wc, b->bp.cost_dtype);
    }
    b->smem = 0;
    for (stereo_ctx *c : b->ctx) b->smem = std::max(b->smem, c->g.smem_bytes);
    if ((rc = cuda_error(cudaFuncSetAttribute((const void *)b->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)b->smem),
                         "batch: cudaFuncSetAttribute"))) {
        release_build(b);
        return rc;
    }
    std::vector<PairDesc> hp(n);
    struct Item {
        int key, pair, tile;
    };
    std::vector<Item> items;
    for (int i = 0; i < n; ++i) {
        const stereo_pair_desc &d = b->pairs[i];
        fill_pair_desc(b->ctx[i], d.disp_dev, d.wta_dev, d.valid_dev, hp[i]);
        const Geometry &g = b->ctx[i]->g;
        for (int ty = 0; ty < g.nty; ++ty)
            for (int tx = 0; tx < g.ntx; ++tx) items.push_back({g.Dp, i, tx | (ty << 16)});
    }
    // heaviest tiles first (the work of a tile grows with its pair's search range)
    std::stable_sort(items.begin(), items.end(), [](const Item &x, const Item &y) { return x.key > y.key; });
    std::vector<int2> hi(items.size());
    for (size_t k = 0; k < items.size(); ++k) hi[k] = make_int2(items[k].pair, items[k].tile);
    b->nitems = (int)hi.size();
    if ((rc = cuda_error(cudaMalloc(&b->d_pairs, sizeof(PairDesc) * n), "batch: cudaMalloc pairs")) ||
        (rc = cuda_error(cudaMalloc(&b->d_items, sizeof(int2) * hi.size()), "batch: cudaMalloc items")) ||
        (rc = cuda_error(cudaMalloc(&b->d_counter, sizeof(int)), "batch: cudaMalloc counter")) ||
        (rc = cuda_error(cudaMemcpy(b->d_pairs, hp.data(), sizeof(PairDesc) * n, cudaMemcpyHostToDevice),
                         "batch: copy pairs")) ||
        (rc = cuda_error(cudaMemcpy(b->d_items, hi.data(), sizeof(int2) * hi.size(), cudaMemcpyHostToDevice),
                         "batch: copy items"))) {
        release_build(b);
        return rc;
    }
    return STEREO_OK;
}

static int enqueue_fused(stereo_batch *b, cudaStream_t s)
{
    int rc = cuda_error(cudaMemsetAsync(b->d_counter, 0, sizeof(int), s), "batch: reset counter");
    if (rc) return rc;
    PairDesc unused;
    memset(&unused, 0, sizeof(unused));
    const int grid = std::min(b->nsm, b->nitems);
    b->kernel<<<grid, fused_threads(b->wc), b->smem, s>>>(unused, b->d_pairs, b->d_items, b->nitems, b->d_counter);
    return cuda_error(cudaGetLastError(), "batch: fused launch");
}

// the warp, staging and row tables of pair i (every pair has its own context and buffers)
static int enqueue_pre_pair(stereo_batch *b, size_t i, cudaStream_t s)
{
    const stereo_pair_desc &d = b->pairs[i];
    int rc = launch_warp(b->ctx[i], d.tgt_dev, d.shift_dev, d.tgt_warped_dev, s);
    if (!rc) rc = launch_prep(b->ctx[i], d.ref_dev, d.tgt_warped_dev, s);
    if (!rc) rc = launch_row_tables(b->ctx[i], d.shift_dev, d.tgt_warped_dev, s);
    return rc;
}

// the disparity transformation of pair i
static int enqueue_post_pair(stereo_batch *b, size_t i, cudaStream_t s)
{
    const stereo_pair_desc &d = b->pairs[i];
    return launch_dt(b->ctx[i], d.disp_dev, d.valid_dev, d.psi_init, d.delta_t, d.disp_out_dev, d.res_dev, s);
}

static int enqueue_pre(stereo_batch *b, cudaStream_t s)
{
    int rc = STEREO_OK;
    for (size_t i = 0; i < b->pairs.size() && !rc; ++i) rc = enqueue_pre_pair(b, i, s);
    return rc;
}

// fn(b, i, stream) for every pair, the pairs dealt round-robin to the side streams, which
// are forked from s before and joined into s after
static int enqueue_branches(stereo_batch *b, cudaStream_t s, int (*fn)(stereo_batch *, size_t, cudaStream_t))
{
    const size_t nb = std::min(b->side.size(), b->pairs.size());
    int rc = cuda_error(cudaEventRecord(b->fork, s), "batch: fork");
    for (size_t k = 0; k < nb && !rc; ++k)
        rc = cuda_error(cudaStreamWaitEvent(b->side[k], b->fork, 0), "batch: fork wait");
    for (size_t i = 0; i < b->pairs.size() && !rc; ++i) rc = fn(b, i, b->side[i % nb]);
    for (size_t k = 0; k < nb && !rc; ++k) {
        rc = cuda_error(cudaEventRecord(b->join[k], b->side[k]), "batch: join");
        if (!rc) rc = cuda_error(cudaStreamWaitEvent(s, b->join[k], 0), "batch: join wait");
    }
    return rc;
}

static int capture(stereo_batch *b)
{
    int rc = cuda_error(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "batch: begin capture");
    if (rc) return rc;
    rc = enqueue_branches(b, b->cap, enqueue_pre_pair);
    if (!rc) rc = enqueue_fused(b, b->cap);
    if (!rc) rc = enqueue_branches(b, b->cap, enqueue_post_pair);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if ((rc = cuda_error(e, "batch: end capture"))) return rc;
    b->graph = g;
    return cuda_error(cudaGraphInstantiate(&b->exec, g, 0), "batch: instantiate graph");
}

// ------------------------------------------------------------------ autotuner
static unsigned long long fnv1a(const std::string &s)
{
    unsigned long long h = 1469598103934665603ull;
    for (unsigned char ch : s) {
        h ^= ch;
        h *= 1099511628211ull;
    }
    return h;
}

static std::string tune_key(const stereo_batch *b)
{
    std::string k;
    char buf[96];
    snprintf(buf, sizeof(buf), "c6 w%d k%d t%d sm%d |", b->bp.win, b->bp.bil, b->bp.cost_dtype, b->nsm);
    k += buf;
    for (const stereo_pair_desc &d : b->pairs) {
        snprintf(buf, sizeof(buf), " %dx%dx%d", d.width, d.height, d.max_disp);
        k += buf;
    }
    snprintf(buf, sizeof(buf), "fnv%016llx", fnv1a(k));
    return buf;
}

// The cache is a JSON object, one entry per line: "key": {"wc": W, "dc": D, "ms": T}
static bool cache_lookup(const char *path, const std::string &key, int *wc, int *dc)
{
    FILE *f = path ? fopen(path, "r") : nullptr;
    if (!f) return false;
    char line[512];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        char k[128];
        int w = 0, d = 0;
        if (sscanf(line, " \"%127[^\"]\": {\"wc\": %d, \"dc\": %d", k, &w, &d) == 3 && key == k) {
            *wc = w;
            *dc = d;
            found = true;
        }
    }
    fclose(f);
    return found;
}

static void cache_store(const char *path, const std::string &key, int wc, int dc, double ms)
{
    if (!path) return;
    std::vector<std::string> keep;
    if (FILE *f = fopen(path, "r")) {
        char line[512];
        while (fgets(line, sizeof(line), f)) {
            char k[128];
            if (sscanf(line, " \"%127[^\"]\":", k) == 1 && key != k) {
                std::string l(line);
                while (!l.empty() && (l.back() == '\n' || l.back() == ',' || l.back() == ' ')) l.pop_back();
                keep.push_back(l);
            }
        }
        fclose(f);
    }
    char buf[256];
    snprintf(buf, sizeof(buf), "  \"%s\": {\"wc\": %d, \"dc\": %d, \"ms\": %.4f}", key.c_str(), wc, dc, ms);
    keep.push_back(buf);
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n");
    for (size_t i = 0; i < keep.size(); ++i) fprintf(f, "%s%s\n", keep[i].c_str(), i + 1 < keep.size() ? "," : "");
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), path);
}

// Reads and clears the device status word of every pair of the batch (synchronising the
// capture stream first); true when none was set.
static bool statuses_clear(stereo_batch *b)
{
    if (cudaStreamSynchronize(b->cap) != cudaSuccess) return false;
    bool clear = true;
    for (stereo_ctx *c : b->ctx)
        if (stereo_check_device_status(c, nullptr) != STEREO_OK) clear = false;
    return clear;
}

// Time the persistent fused launch of every candidate (tile shape, chunk size) on this
// batch; keep the fastest.
static int autotune(stereo_batch *b, int *wc_out, int *dc_out, int *source)
{
    const char *path = getenv("STEREO_AUTOTUNE_CACHE");
    const std::string key = tune_key(b);
    if (cache_lookup(path, key, wc_out, dc_out) && pick_fused(b->bp.cost_dtype, b->bp.bil / 2, *dc_out, *wc_out) &&
        (*wc_out != kTcWC || tc_supported(b->bp.cost_dtype, b->bp.bil, b->bp.sigma1))) {
        *source = 1;
        return STEREO_OK;
    }
    const int cand[][2] = {{kScWC, 32}, {kTcWC, 16}, {kWsWC, 12}, {2, 12}, {1, 12}, {4, 12}, {2, 4}};
    double best_ms = 1e30;
    int best_wc = 0, best_dc = 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (const auto &c : cand) {
        if (!pick_fused(b->bp.cost_dtype, b->bp.bil / 2, c[1], c[0])) continue;
        if (c[0] == kTcWC && !tc_supported(b->bp.cost_dtype, b->bp.bil, b->bp.sigma1)) continue;
        if (build(b, c[0], c[1]) != STEREO_OK) continue;   // e.g. shared memory does not fit
        int rc = enqueue_pre(b, b->cap);
        if (!rc) rc = enqueue_fused(b, b->cap);   // warm-up
        float best = 1e30f;
        for (int rep = 0; rep < 3 && !rc; ++rep) {
            cudaEventRecord(e0, b->cap);
            rc = enqueue_fused(b, b->cap);
            cudaEventRecord(e1, b->cap);
            if (!rc) rc = cuda_error(cudaEventSynchronize(e1), "autotune: synchronize");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best = std::min(best, ms);
        }
        if (rc) continue;
        // a candidate whose bounded staging wait gave up returns early and would look fastest:
        // read and clear every pair's status word, and drop the candidate if any was set (so
        // it is neither chosen nor cached, and its status does not reach the first real run)
        if (!statuses_clear(b)) continue;
        if (best < best_ms) {
            best_ms = best;
            best_wc = c[0];
            best_dc = c[1];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    release_build(b);
    if (!best_wc) return set_error(STEREO_ENOTSUP, "batch autotune: no tile configuration runs");
    *wc_out = best_wc;
    *dc_out = best_dc;
    *source = 2;
    cache_store(path, key, best_wc, best_dc, best_ms);
    return STEREO_OK;
}

}  // namespace sgb

using namespace sgb;

extern "C" {

int stereo_batch_params_default(stereo_batch_params *p)
{
    if (!p) return set_error(STEREO_EINVAL, "stereo_batch_params_default: null pointer");
    stereo_params q;
    stereo_params_default(&q);
    memset(p, 0, sizeof(*p));
    p->win = q.win;
    p->bil = q.bil;
    p->sigma0 = q.sigma0;
    p->sigma1 = q.sigma1;
    p->cost_dtype = q.cost_dtype;
    p->lambda0 = q.lambda0;
    p->delta_psi = q.delta_psi;
    p->max_iters = q.max_iters;
    return STEREO_OK;
}

int stereo_batch_create(const stereo_batch_params *p, int32_t n, const stereo_pair_desc *pairs, stereo_batch **out)
{
    if (!p || !pairs || !out) return set_error(STEREO_EINVAL, "stereo_batch_create: null pointer");
    *out = nullptr;
    if (n < 1 || n > 4096) return set_error(STEREO_EINVAL, "stereo_batch_create: n = %d outside 1..4096", n);
    if ((p->tile_wc && p->tile_wc != 1 && p->tile_wc != 2 && p->tile_wc != 4 && p->tile_wc != kWsWC &&
         p->tile_wc != kTcWC && p->tile_wc != kScWC) ||
        (p->tile_dc && p->tile_dc != 4 && p->tile_dc != 12 && p->tile_dc != 16 && p->tile_dc != 32))
        return set_error(STEREO_EINVAL,
                         "stereo_batch_create: tile_wc must be 0, 1, 2, 4, 8, 16 or 32 and tile_dc 0, 4, 12, 16 or 32");
    if (p->tile_wc == kScWC && p->bil / 2 > kScMaxRB)
        return set_error(STEREO_ENOTSUP, "stereo_batch_create: tile_wc 32 needs bil <= 13");
    if (p->tile_wc == kTcWC && !tc_supported(p->cost_dtype, p->bil, p->sigma1))
        return set_error(STEREO_ENOTSUP, "stereo_batch_create: tile_wc 16 needs FP16 / BF16 storage, bil <= 13 and sigma1 <= 150");
    for (int i = 0; i < n; ++i) {
        const stereo_pair_desc &d = pairs[i];
        if (!d.ref_dev || !d.tgt_dev || !d.shift_dev || !d.tgt_warped_dev || !d.disp_dev || !d.valid_dev ||
            !d.disp_out_dev || !d.res_dev)
            return set_error(STEREO_EINVAL, "stereo_batch_create: pair %d has a null buffer", i);
        if (d.width > 0xffff * 32 || d.height > 0xffff)
            return set_error(STEREO_EINVAL, "stereo_batch_create: pair %d too large", i);
    }
    stereo_batch *b = new (std::nothrow) stereo_batch();
    if (!b) return set_error(STEREO_ENOMEM, "stereo_batch_create: host allocation failed");
    b->bp = *p;
    b->pairs.assign(pairs, pairs + n);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
    int rc = cuda_error(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "batch: create stream");
    if (!rc) rc = cuda_error(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "batch: create event");
    for (int k = 0; k < kBatchBranches && !rc; ++k) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        rc = cuda_error(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "batch: create stream");
        if (!rc) b->side.push_back(st);
        if (!rc) rc = cuda_error(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "batch: create event");
        if (!rc) b->join.push_back(ev);
    }
    int wc = p->tile_wc, dc = p->tile_dc;
    if (!rc && (!wc || !dc)) rc = autotune(b, &wc, &dc, &b->source);
    if (!rc) rc = build(b, wc, dc);
    if (!rc) rc = capture(b);
    if (rc) {
        stereo_batch_destroy(b);
        return rc;
    }
    *out = b;
    return STEREO_OK;
}

int stereo_batch_run(stereo_batch *b, stereo_stream_t stream)
{
    if (!b || !b->exec) return set_error(STEREO_EINVAL, "stereo_batch_run: no batch");
    return cuda_error(cudaGraphLaunch(b->exec, (cudaStream_t)stream), "stereo_batch_run: graph launch");
}

int stereo_batch_config(const stereo_batch *b, int32_t *wc, int32_t *dc, int32_t *n_items, int32_t *source)
{
    if (!b || !wc || !dc || !n_items || !source) return set_error(STEREO_EINVAL, "stereo_batch_config: null pointer");
    *wc = b->wc;
    *dc = b->dc;
    *n_items = b->nitems;
    *source = b->source;
    return STEREO_OK;
}

int stereo_batch_check_device_status(stereo_batch *b)
{
    if (!b) return set_error(STEREO_EINVAL, "stereo_batch_check_device_status: null pointer");
    for (stereo_ctx *c : b->ctx) {
        int rc = stereo_check_device_status(c, nullptr);
        if (rc) return rc;
    }
    return STEREO_OK;
}

int stereo_batch_destroy(stereo_batch *b)
{
    if (!b) return STEREO_OK;
    cudaDeviceSynchronize();
    release_build(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (cudaStream_t st : b->side) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->join) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
    return STEREO_OK;
}

}  // extern "C"
