// extern "C" entry points of libpsi: argument checks, context, status word.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "geometry.cuh"

struct psi_ctx {
    int device;
    psi::DevStatus *status;
    char err[512];
    // armed kernel-timing events per psi_kernel_id: [id][0] begin, [id][1] end
    cudaEvent_t time_ev[3][2];
    // launch shape of the compositing kernels per (K class, feature dtype,
    // low-pass[, saved state]) (0 = default; set by the autotuner)
    uint8_t shape_fwd[4][3][2];
    uint8_t shape_bwd[4][3][2][2];
};

namespace {

// One NVTX range per entry point that enqueues GPU work, named after it, so
// that a profiler's timeline groups each call's kernels (no-op without one).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

int fail(psi_ctx *ctx, int code, const char *fmt, ...)
{
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_fail(psi_ctx *ctx, const char *where, cudaError_t e)
{
    return fail(ctx, PSI_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int check_opts(psi_ctx *ctx, const psi_render_opts *o)
{
    if (!o) return fail(ctx, PSI_ERR_INVALID_ARG, "opts is NULL");
    if (o->mode < PSI_ISECT_SPHERE || o->mode > PSI_ISECT_EXACT) return fail(ctx, PSI_ERR_INVALID_ARG, "bad mode %d", o->mode);
    if (o->tile_w != 16 || (o->tile_h != 16 && o->tile_h != 8))
        return fail(ctx, PSI_ERR_UNSUPPORTED, "tile %dx%d unsupported (16x16 or 16x8)", o->tile_w, o->tile_h);
    if (o->top_k < 0 || o->top_k > PSI_MAX_TOPK) return fail(ctx, PSI_ERR_INVALID_ARG, "top_k %d out of [0,32]", o->top_k);
    if (o->tile_h == 8 && (o->top_k < 1 || o->top_k > 8 || o->lowpass))
        return fail(ctx, PSI_ERR_UNSUPPORTED, "16x8 tiles need 1 <= top_k <= 8 and no low-pass filter");
    if (!(o->chi2 > 0.0f) || !(o->chi2 < 1e4f)) return fail(ctx, PSI_ERR_INVALID_ARG, "chi2 must be in (0, 1e4)");
    if (!(o->z_near > 0.0f)) return fail(ctx, PSI_ERR_INVALID_ARG, "z_near must be > 0");
    if (!(o->t_eps >= 0.0f) || !(o->t_eps < 1.0f)) return fail(ctx, PSI_ERR_INVALID_ARG, "t_eps must be in [0,1)");
    if (o->lowpass != 0 && o->lowpass != 1) return fail(ctx, PSI_ERR_INVALID_ARG, "lowpass must be 0 or 1");
    return PSI_OK;
}

int check_cams(psi_ctx *ctx, const psi_camera *cams, int n_views, const psi_render_opts *o)
{
    if (!cams) return fail(ctx, PSI_ERR_INVALID_ARG, "cams is NULL");
    if (n_views < 1 || n_views > PSI_MAX_VIEWS)
        return fail(ctx, PSI_ERR_INVALID_ARG, "n_views %d out of [1,%d]", n_views, PSI_MAX_VIEWS);
    int64_t tiles = 0;
    for (int v = 0; v < n_views; ++v) {
        const psi_camera &c = cams[v];
        if (c.width < 1 || c.height < 1 || c.width > 32768 || c.height > 32768)
            return fail(ctx, PSI_ERR_INVALID_ARG, "view %d: size %dx%d out of [1,32768]", v, c.width, c.height);
        if (!(c.fx > 0.0f) || !(c.fy > 0.0f)) return fail(ctx, PSI_ERR_INVALID_ARG, "view %d: focal must be > 0", v);
        tiles += static_cast<int64_t>((c.width + o->tile_w - 1) / o->tile_w) * ((c.height + o->tile_h - 1) / o->tile_h);
    }
    if (tiles >= (int64_t(1) << 31)) return fail(ctx, PSI_ERR_INVALID_ARG, "too many tiles");
    return PSI_OK;
}

int check_surfels(psi_ctx *ctx, const psi_surfels *s)
{
    if (!s) return fail(ctx, PSI_ERR_INVALID_ARG, "surfels is NULL");
    if (s->n < 0 || s->n >= (int64_t(1) << 31)) return fail(ctx, PSI_ERR_INVALID_ARG, "surfel count out of range");
    if (s->n > 0 && (!s->mu || !s->tu || !s->tv || !s->scale || !s->opacity || !s->rgb))
        return fail(ctx, PSI_ERR_INVALID_ARG, "a surfel array is NULL");
    return PSI_OK;
}

int check_feat(psi_ctx *ctx, const psi_features *f, psi::FeatView &fv)
{
    fv = psi::FeatView{nullptr, nullptr, PSI_F32, 0};
    if (!f || !f->data) return PSI_OK;
    if (f->dtype != PSI_F32 && f->dtype != PSI_BF16 && f->dtype != PSI_FP8_E4M3)
        return fail(ctx, PSI_ERR_INVALID_ARG, "bad feature dtype %d", f->dtype);
    if (f->dim < 16 || f->dim > 256 || f->dim % 16 != 0)
        return fail(ctx, PSI_ERR_INVALID_ARG, "feature dim %d must be a multiple of 16 in [16,256]", f->dim);
    if (!aligned(f->data, 16)) return fail(ctx, PSI_ERR_INVALID_ARG, "feature rows must be 16-byte aligned");
    fv = psi::FeatView{f->data, f->scale, f->dtype, f->dim};
    return PSI_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

} // namespace

extern "C" {

int psi_ctx_create(psi_ctx **out, int device)
{
    if (!out) return PSI_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return PSI_ERR_INVALID_ARG;
    psi_ctx *c = new (std::nothrow) psi_ctx(); // value-initialised: no timing events armed
    if (!c) return PSI_ERR_CUDA;
    c->device = device;
    c->status = nullptr;
    c->err[0] = 0;
    DeviceGuard g(device);
    cudaError_t e = cudaMalloc(&c->status, sizeof(psi::DevStatus));
    psi::DevStatus init{};
    init.wait_limit_ns = psi::kWaitLimitNs;
    if (e == cudaSuccess) e = cudaMemcpy(c->status, &init, sizeof(init), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (c->status) cudaFree(c->status);
        delete c;
        return PSI_ERR_CUDA;
    }
    *out = c;
    return PSI_OK;
}

void psi_ctx_destroy(psi_ctx *ctx)
{
    if (!ctx) return;
    {
        DeviceGuard g(ctx->device);
        if (ctx->status) cudaFree(ctx->status);
    }
    delete ctx;
}

const char *psi_last_error(const psi_ctx *ctx) { return ctx ? ctx->err : "NULL context"; }

int psi_ctx_set_wait_limit_ns(psi_ctx *ctx, uint64_t ns)
{
    if (!ctx) return PSI_ERR_INVALID_ARG;
    if (ns > PSI_WAIT_LIMIT_MAX_NS)
        return fail(ctx, PSI_ERR_INVALID_ARG, "wait limit %llu ns above %llu", static_cast<unsigned long long>(ns),
                    static_cast<unsigned long long>(PSI_WAIT_LIMIT_MAX_NS));
    DeviceGuard g(ctx->device);
    const unsigned long long v = ns ? ns : psi::kWaitLimitNs;
    cudaError_t e = cudaMemcpy(reinterpret_cast<char *>(ctx->status) + offsetof(psi::DevStatus, wait_limit_ns), &v,
                               sizeof(v), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_ctx_set_wait_limit_ns", e);
}

int psi_ctx_time_kernel(psi_ctx *ctx, int kernel, void *ev_begin, void *ev_end)
{
    if (!ctx) return PSI_ERR_INVALID_ARG;
    if (kernel != PSI_KERNEL_BWD_FEAT && kernel != PSI_KERNEL_BWD_WALK)
        return fail(ctx, PSI_ERR_INVALID_ARG, "unknown kernel id %d", kernel);
    if ((ev_begin == nullptr) != (ev_end == nullptr))
        return fail(ctx, PSI_ERR_INVALID_ARG, "give both events or neither");
    ctx->time_ev[kernel][0] = static_cast<cudaEvent_t>(ev_begin);
    ctx->time_ev[kernel][1] = static_cast<cudaEvent_t>(ev_end);
    return PSI_OK;
}

int psi_status_fetch(psi_ctx *ctx, psi_stream stream, int32_t *status_out, int64_t *detail)
{
    if (!ctx || !status_out) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard g(ctx->device);
    psi::DevStatus h{};
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "psi_status_fetch", e);
    e = cudaMemcpy(&h, ctx->status, psi::kDevStatusReportBytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, "psi_status_fetch", e);
    e = cudaMemset(ctx->status, 0, psi::kDevStatusReportBytes);
    if (e != cudaSuccess) return cuda_fail(ctx, "psi_status_fetch", e);
    int code = PSI_OK;
    // report the most severe: timeout, then a failed bounds check (debug
    // builds), then capacity, then invalid argument
    if (h.flags & (1 << PSI_ERR_TIMEOUT))
        code = PSI_ERR_TIMEOUT;
    else if (h.flags & (1 << PSI_ERR_BOUNDS))
        code = PSI_ERR_BOUNDS;
    else if (h.flags & (1 << PSI_ERR_CAPACITY))
        code = PSI_ERR_CAPACITY;
    else if (h.flags & (1 << PSI_ERR_INVALID_ARG))
        code = PSI_ERR_INVALID_ARG;
    *status_out = code;
    if (detail)
        *detail = (code == PSI_ERR_TIMEOUT || code == PSI_ERR_BOUNDS) ? static_cast<int64_t>(h.wait_site)
                                                                      : static_cast<int64_t>(h.required_pairs);
    return PSI_OK;
}

int psi_debug_checks(void)
{
#ifdef PSI_DEBUG
    return 1;
#else
    return 0;
#endif
}

void psi_default_opts(psi_render_opts *o)
{
    if (!o) return;
    o->mode = PSI_ISECT_EXACT;
    o->top_k = 0;
    o->chi2 = 9.0f;
    o->z_near = 0.2f;
    o->opacity_radius = 0;
    o->tile_w = 16;
    o->tile_h = 16;
    o->t_eps = 1e-4f;
    o->lowpass = 0;
}

int psi_view_layout(const psi_camera *cams, int n_views, const psi_render_opts *o, int64_t *tile_base, int64_t *pix_base)
{
    if (!cams || !o || n_views < 0 || !tile_base || !pix_base) return PSI_ERR_INVALID_ARG;
    if (o->tile_w < 1 || o->tile_h < 1) return PSI_ERR_INVALID_ARG;
    tile_base[0] = 0;
    pix_base[0] = 0;
    for (int v = 0; v < n_views; ++v) {
        tile_base[v + 1] = tile_base[v] + static_cast<int64_t>((cams[v].width + o->tile_w - 1) / o->tile_w) *
                                              ((cams[v].height + o->tile_h - 1) / o->tile_h);
        pix_base[v + 1] = pix_base[v] + static_cast<int64_t>(cams[v].width) * cams[v].height;
    }
    return PSI_OK;
}

int psi_intersect_workspace_size(int64_t n_records, size_t *bytes)
{
    if (!bytes || n_records < 0) return PSI_ERR_INVALID_ARG;
    *bytes = psi::intersect_workspace_bytes(n_records);
    return PSI_OK;
}

int psi_sort_workspace_size(int64_t capacity, size_t *bytes)
{
    if (!bytes || capacity < 0) return PSI_ERR_INVALID_ARG;
    *bytes = psi::sort_workspace_bytes(capacity);
    return PSI_OK;
}

int psi_render_bwd_workspace_size(int64_t n_records, int64_t n_pix, int top_k, size_t *bytes)
{
    if (!bytes || n_records < 0 || n_pix < 0 || top_k < 0 || top_k > PSI_MAX_TOPK) return PSI_ERR_INVALID_ARG;
    *bytes = psi::render_bwd_workspace_bytes(n_records, n_pix, top_k);
    return PSI_OK;
}

int psi_project_surfels(psi_ctx *ctx, const psi_surfels *s, const psi_camera *cams, int n_views,
                        const psi_render_opts *o, void *records, void *bin_records, uint32_t *tiles_touched,
                        psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    int rc;
    if ((rc = check_opts(ctx, o)) || (rc = check_cams(ctx, cams, n_views, o)) || (rc = check_surfels(ctx, s))) return rc;
    if (s->n > 0 && (!records || !bin_records || !tiles_touched))
        return fail(ctx, PSI_ERR_INVALID_ARG, "output array is NULL");
    if (!aligned(records, 16) || !aligned(bin_records, 16)) return fail(ctx, PSI_ERR_INVALID_ARG, "records and bin records must be 16-byte aligned");
    if (s->n * n_views >= (int64_t(1) << 32)) return fail(ctx, PSI_ERR_INVALID_ARG, "n_views * N must be < 2^32");
    DeviceGuard g(ctx->device);
    psi::FrameParams fp;
    psi::fill_frame_params(fp, cams, n_views, o, s->n);
    cudaError_t e = psi::launch_project(fp, *s, static_cast<float4 *>(records), static_cast<float4 *>(bin_records),
                                        tiles_touched, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_project_surfels", e);
}

int psi_intersect_tiles(psi_ctx *ctx, const psi_camera *cams, int n_views, const psi_render_opts *o,
                        int64_t n_surfels, const void *bin_records, const uint32_t *tiles_touched, uint64_t *keys,
                        uint32_t *vals, int64_t capacity, int64_t *d_num_pairs, void *workspace,
                        size_t workspace_bytes, psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    int rc;
    if ((rc = check_opts(ctx, o)) || (rc = check_cams(ctx, cams, n_views, o))) return rc;
    if (n_surfels < 0 || n_surfels * n_views >= (int64_t(1) << 32))
        return fail(ctx, PSI_ERR_INVALID_ARG, "n_views * N must be in [0, 2^32)");
    if (capacity < 0 || capacity >= (int64_t(1) << 32)) return fail(ctx, PSI_ERR_INVALID_ARG, "capacity must be in [0, 2^32)");
    if (!d_num_pairs || (capacity > 0 && (!keys || !vals))) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL output");
    if (n_surfels > 0 && (!bin_records || !tiles_touched)) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL input");
    const int64_t R = n_surfels * n_views;
    const size_t need = psi::intersect_workspace_bytes(R);
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256))
        return fail(ctx, PSI_ERR_INVALID_ARG, "workspace must be >= %zu bytes, 256-byte aligned", need);
    DeviceGuard g(ctx->device);
    psi::FrameParams fp;
    psi::fill_frame_params(fp, cams, n_views, o, n_surfels);
    cudaError_t e = psi::launch_intersect(fp, static_cast<const float4 *>(bin_records), tiles_touched, keys, vals,
                                          capacity, d_num_pairs, workspace, ctx->status,
                                          reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_intersect_tiles", e);
}

int psi_sort_keys(psi_ctx *ctx, uint64_t *keys, uint32_t *vals, const int64_t *d_num_pairs, int64_t capacity,
                  int begin_bit, int end_bit, uint32_t *tile_ranges, int64_t n_tiles_total, void *workspace,
                  size_t workspace_bytes, psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    if (begin_bit < 0 || end_bit > 64 || begin_bit >= end_bit)
        return fail(ctx, PSI_ERR_INVALID_ARG, "need 0 <= begin_bit < end_bit <= 64");
    if (capacity < 0 || capacity >= (int64_t(1) << 32)) return fail(ctx, PSI_ERR_INVALID_ARG, "capacity must be in [0, 2^32)");
    if (!d_num_pairs || (capacity > 0 && (!keys || !vals))) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL argument");
    if (n_tiles_total < 0 || (n_tiles_total > 0 && !tile_ranges)) return fail(ctx, PSI_ERR_INVALID_ARG, "bad tile ranges");
    const size_t need = psi::sort_workspace_bytes(capacity);
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256))
        return fail(ctx, PSI_ERR_INVALID_ARG, "workspace must be >= %zu bytes, 256-byte aligned", need);
    DeviceGuard g(ctx->device);
    cudaError_t e = psi::launch_sort(keys, vals, d_num_pairs, capacity, begin_bit, end_bit, tile_ranges, n_tiles_total,
                                     workspace, ctx->status, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_sort_keys", e);
}

int psi_sort_keys_noalloc(psi_ctx *ctx, uint64_t *keys, uint32_t *vals, const int64_t *d_num_pairs,
                          int64_t capacity, int begin_bit, int end_bit, uint32_t *tile_ranges, int64_t n_tiles_total,
                          psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    if (begin_bit < 0 || end_bit > 64 || begin_bit >= end_bit)
        return fail(ctx, PSI_ERR_INVALID_ARG, "need 0 <= begin_bit < end_bit <= 64");
    if (capacity < 0 || capacity > PSI_SORT_NOALLOC_MAX_PAIRS)
        return fail(ctx, PSI_ERR_INVALID_ARG, "psi_sort_keys_noalloc: capacity %lld outside [0, %lld]",
                    static_cast<long long>(capacity), static_cast<long long>(PSI_SORT_NOALLOC_MAX_PAIRS));
    if (!d_num_pairs || (capacity > 0 && (!keys || !vals))) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL argument");
    if (n_tiles_total < 0 || (n_tiles_total > 0 && !tile_ranges)) return fail(ctx, PSI_ERR_INVALID_ARG, "bad tile ranges");
    DeviceGuard g(ctx->device);
    const char *why = nullptr;
    cudaError_t e = psi::launch_sort_noalloc(keys, vals, d_num_pairs, capacity, begin_bit, end_bit, tile_ranges,
                                             n_tiles_total, ctx->status, reinterpret_cast<cudaStream_t>(stream), &why);
    if (why) return fail(ctx, e == cudaErrorInvalidValue ? PSI_ERR_INVALID_ARG : PSI_ERR_CUDA, "psi_sort_keys_noalloc: %s", why);
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_sort_keys_noalloc", e);
}

} // extern "C"

namespace {

int k_class(int K) { return K == 0 ? 0 : K <= 8 ? 1 : K <= 16 ? 2 : 3; }
int dt_class(int dtype) { return dtype == PSI_BF16 ? 1 : dtype == PSI_FP8_E4M3 ? 2 : 0; }

uint8_t &fwd_shape(psi_ctx *ctx, const psi::FrameParams &fp, const psi::FeatView &fv)
{
    return ctx->shape_fwd[k_class(fp.top_k)][fv.data ? dt_class(fv.dtype) : 0][fp.lowpass ? 1 : 0];
}

uint8_t &bwd_shape(psi_ctx *ctx, const psi::FrameParams &fp, const psi::FeatView &fv, bool saved)
{
    return ctx->shape_bwd[k_class(fp.top_k)][fv.data ? dt_class(fv.dtype) : 0][fp.lowpass ? 1 : 0][saved ? 1 : 0];
}

// Runs launch(shape) for every shape that exists for (D, K): once untimed,
// then `reps` times between two events on the stream; ms[shape] = mean ms
// (-1: shape does not exist), *best = the fastest.
template <class Launch>
int time_shapes(psi_ctx *ctx, int D, int K, bool pair_walk, int reps, cudaStream_t st, Launch launch, float *ms,
                int *best, const char *who)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return fail(ctx, PSI_ERR_INVALID_ARG, "%s: cannot time shapes inside a stream capture", who);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best_ms = 0.0f;
    int b = -1;
    for (int sh = 0; sh < psi::kShapes && e == cudaSuccess; ++sh) {
        ms[sh] = -1.0f;
        if (!psi::render_shape_valid(D, K, sh, pair_walk)) continue;
        e = launch(sh);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch(sh);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess) {
            ms[sh] = t / static_cast<float>(reps);
            if (b < 0 || ms[sh] < best_ms) {
                best_ms = ms[sh];
                b = sh;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(ctx, who, e);
    *best = b;
    return PSI_OK;
}

int prepare_fwd(psi_ctx *ctx, const psi_features *f, const void *records, const uint32_t *vals,
                const uint32_t *tile_ranges, const psi_camera *cams, int n_views, int64_t n_surfels,
                const psi_render_opts *o, const psi_fwd_out *out, psi::FrameParams &fp, psi::FeatView &fv)
{
    int rc;
    if ((rc = check_opts(ctx, o)) || (rc = check_cams(ctx, cams, n_views, o))) return rc;
    if ((rc = check_feat(ctx, f, fv))) return rc;
    if (!out || !out->rgb || !out->T) return fail(ctx, PSI_ERR_INVALID_ARG, "out.rgb and out.T are required");
    if (out->F && out->F_dtype != PSI_F32 && out->F_dtype != PSI_BF16)
        return fail(ctx, PSI_ERR_INVALID_ARG, "F_dtype must be PSI_F32 or PSI_BF16");
    if (out->F && !aligned(out->F, 16)) return fail(ctx, PSI_ERR_INVALID_ARG, "out.F must be 16-byte aligned");
    if (out->argmax && (o->top_k <= 0 || !fv.data))
        return fail(ctx, PSI_ERR_INVALID_ARG, "out.argmax needs top_k > 0 and features");
    if (!records || !vals || !tile_ranges) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL input");
    if (!aligned(records, 16)) return fail(ctx, PSI_ERR_INVALID_ARG, "records must be 16-byte aligned");
    if (n_surfels < 0) return fail(ctx, PSI_ERR_INVALID_ARG, "n_surfels < 0");
    psi::fill_frame_params(fp, cams, n_views, o, n_surfels);
    return PSI_OK;
}

int prepare_bwd(psi_ctx *ctx, const psi_surfels *s, const psi_features *f, const void *records,
                const uint32_t *vals, const uint32_t *tile_ranges, const psi_camera *cams, int n_views,
                const psi_render_opts *o, const float *g_rgb, const float *g_F, const psi_fwd_out *saved,
                const psi_grads *grads, void *workspace, size_t workspace_bytes, psi::FrameParams &fp,
                psi::FeatView &fv)
{
    int rc;
    if ((rc = check_opts(ctx, o)) || (rc = check_cams(ctx, cams, n_views, o)) || (rc = check_surfels(ctx, s))) return rc;
    if ((rc = check_feat(ctx, f, fv))) return rc;
    if (!records || !vals || !tile_ranges || !g_rgb || !grads) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL input");
    if (!aligned(records, 16)) return fail(ctx, PSI_ERR_INVALID_ARG, "records must be 16-byte aligned");
    if (g_F && !fv.data) return fail(ctx, PSI_ERR_INVALID_ARG, "g_F given without features");
    if (!aligned(g_F, 16) || !aligned(grads->feat, 16))
        return fail(ctx, PSI_ERR_INVALID_ARG, "g_F and grads->feat must be 16-byte aligned");
    if (saved && (!saved->T || !saved->n_last || (o->top_k > 0 && (!saved->topk_ids || !saved->topk_w))))
        return fail(ctx, PSI_ERR_INVALID_ARG, "saved forward state needs T, n_last and (top_k > 0) topk_ids, topk_w");
    int64_t n_pix_total = 0;
    {
        int64_t tb[PSI_MAX_VIEWS + 1], pb[PSI_MAX_VIEWS + 1];
        if ((rc = psi_view_layout(cams, n_views, o, tb, pb))) return fail(ctx, rc, "camera layout");
        n_pix_total = pb[n_views];
    }
    const size_t need = psi::render_bwd_workspace_bytes(s->n * n_views, n_pix_total, o->top_k);
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256))
        return fail(ctx, PSI_ERR_INVALID_ARG, "workspace must be >= %zu bytes, 256-byte aligned", need);
    psi::fill_frame_params(fp, cams, n_views, o, s->n);
    return PSI_OK;
}

} // namespace

extern "C" {

int psi_render_fwd(psi_ctx *ctx, const psi_features *f, const void *records, const uint32_t *vals,
                   const uint32_t *tile_ranges, const psi_camera *cams, int n_views, int64_t n_surfels,
                   const psi_render_opts *o, const psi_fwd_out *out, psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    psi::FrameParams fp;
    psi::FeatView fv;
    int rc = prepare_fwd(ctx, f, records, vals, tile_ranges, cams, n_views, n_surfels, o, out, fp, fv);
    if (rc) return rc;
    DeviceGuard g(ctx->device);
    cudaError_t e = psi::launch_render_fwd(fp, fv, static_cast<const float4 *>(records), vals, tile_ranges, *out,
                                           ctx->status, reinterpret_cast<cudaStream_t>(stream), fwd_shape(ctx, fp, fv));
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_render_fwd", e);
}

int psi_render_bwd(psi_ctx *ctx, const psi_surfels *s, const psi_features *f, const void *records,
                   const uint32_t *vals, const uint32_t *tile_ranges, const psi_camera *cams, int n_views,
                   const psi_render_opts *o, const float *g_rgb, const float *g_F, const float *g_T,
                   const psi_fwd_out *saved, const psi_grads *grads, void *workspace, size_t workspace_bytes,
                   psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    psi::FrameParams fp;
    psi::FeatView fv;
    int rc = prepare_bwd(ctx, s, f, records, vals, tile_ranges, cams, n_views, o, g_rgb, g_F, saved, grads, workspace,
                         workspace_bytes, fp, fv);
    if (rc) return rc;
    DeviceGuard g(ctx->device);
    cudaError_t e = psi::launch_render_bwd(fp, *s, fv, static_cast<const float4 *>(records), vals, tile_ranges, g_rgb,
                                           g_F, g_T, saved, *grads, workspace, ctx->status,
                                           reinterpret_cast<cudaStream_t>(stream), ctx->time_ev,
                                           bwd_shape(ctx, fp, fv, saved != nullptr));
    for (int k = PSI_KERNEL_BWD_FEAT; k <= PSI_KERNEL_BWD_WALK; ++k) ctx->time_ev[k][0] = ctx->time_ev[k][1] = nullptr;
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_render_bwd", e);
}

int psi_tune_render_fwd(psi_ctx *ctx, const psi_features *f, const void *records, const uint32_t *vals,
                        const uint32_t *tile_ranges, const psi_camera *cams, int n_views, int64_t n_surfels,
                        const psi_render_opts *o, const psi_fwd_out *out, int reps, float *ms, int *best,
                        psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    if (reps < 1 || !ms || !best) return fail(ctx, PSI_ERR_INVALID_ARG, "need reps >= 1, ms and best");
    psi::FrameParams fp;
    psi::FeatView fv;
    int rc = prepare_fwd(ctx, f, records, vals, tile_ranges, cams, n_views, n_surfels, o, out, fp, fv);
    if (rc) return rc;
    DeviceGuard g(ctx->device);
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    auto launch = [&](int shape) {
        return psi::launch_render_fwd(fp, fv, static_cast<const float4 *>(records), vals, tile_ranges, *out,
                                      ctx->status, st, shape);
    };
    rc = time_shapes(ctx, fv.data ? fv.dim : 16, fp.top_k, false, reps, st, launch, ms, best, "psi_tune_render_fwd");
    if (rc) return rc;
    fwd_shape(ctx, fp, fv) = static_cast<uint8_t>(*best);
    return PSI_OK;
}

int psi_tune_render_bwd(psi_ctx *ctx, const psi_surfels *s, const psi_features *f, const void *records,
                        const uint32_t *vals, const uint32_t *tile_ranges, const psi_camera *cams, int n_views,
                        const psi_render_opts *o, const float *g_rgb, const float *g_F, const float *g_T,
                        const psi_fwd_out *saved, const psi_grads *grads, void *workspace, size_t workspace_bytes,
                        int reps, float *ms, int *best, psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    if (reps < 1 || !ms || !best) return fail(ctx, PSI_ERR_INVALID_ARG, "need reps >= 1, ms and best");
    psi::FrameParams fp;
    psi::FeatView fv;
    int rc = prepare_bwd(ctx, s, f, records, vals, tile_ranges, cams, n_views, o, g_rgb, g_F, saved, grads, workspace,
                         workspace_bytes, fp, fv);
    if (rc) return rc;
    DeviceGuard g(ctx->device);
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    auto launch = [&](int shape) {
        return psi::launch_render_bwd(fp, *s, fv, static_cast<const float4 *>(records), vals, tile_ranges, g_rgb, g_F,
                                      g_T, saved, *grads, workspace, ctx->status, st, nullptr, shape);
    };
    rc = time_shapes(ctx, fv.data ? fv.dim : 16, fp.top_k, saved != nullptr && fp.top_k > 0, reps, st, launch, ms, best,
                     "psi_tune_render_bwd");
    if (rc) return rc;
    bwd_shape(ctx, fp, fv, saved != nullptr) = static_cast<uint8_t>(*best);
    // the gradient buffers served as scratch: leave them zeroed
    const size_t n = static_cast<size_t>(s->n);
    const struct {
        float *p;
        size_t count;
    } bufs[] = {{grads->mu, 3 * n},      {grads->tu, 3 * n},  {grads->tv, 3 * n},
                {grads->scale, 2 * n},   {grads->opacity, n}, {grads->rgb, 3 * n},
                {fv.data ? grads->feat : nullptr, fv.data ? n * static_cast<size_t>(fv.dim) : 0}};
    for (const auto &b : bufs) {
        if (!b.p || !b.count) continue;
        cudaError_t e = cudaMemsetAsync(b.p, 0, b.count * sizeof(float), st);
        if (e != cudaSuccess) return cuda_fail(ctx, "psi_tune_render_bwd", e);
    }
    return PSI_OK;
}

int psi_ctx_set_render_shape(psi_ctx *ctx, int which, const psi_render_opts *o, int feat_dtype, int saved, int shape)
{
    if (!ctx || !o) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL argument");
    if (which != 0 && which != 1) return fail(ctx, PSI_ERR_INVALID_ARG, "which must be 0 (forward) or 1 (adjoint)");
    if (shape < 0 || shape >= psi::kShapes) return fail(ctx, PSI_ERR_INVALID_ARG, "shape %d out of range", shape);
    int rc = check_opts(ctx, o);
    if (rc) return rc;
    const int kc = k_class(o->top_k), dc = feat_dtype < 0 ? 0 : dt_class(feat_dtype), lp = o->lowpass ? 1 : 0;
    if (which == 0)
        ctx->shape_fwd[kc][dc][lp] = static_cast<uint8_t>(shape);
    else
        ctx->shape_bwd[kc][dc][lp][saved ? 1 : 0] = static_cast<uint8_t>(shape);
    return PSI_OK;
}

int psi_ctx_get_render_shape(psi_ctx *ctx, int which, const psi_render_opts *o, int feat_dtype, int saved, int *shape)
{
    if (!ctx || !o || !shape) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL argument");
    if (which != 0 && which != 1) return fail(ctx, PSI_ERR_INVALID_ARG, "which must be 0 (forward) or 1 (adjoint)");
    int rc = check_opts(ctx, o);
    if (rc) return rc;
    const int kc = k_class(o->top_k), dc = feat_dtype < 0 ? 0 : dt_class(feat_dtype), lp = o->lowpass ? 1 : 0;
    *shape = which == 0 ? ctx->shape_fwd[kc][dc][lp] : ctx->shape_bwd[kc][dc][lp][saved ? 1 : 0];
    return PSI_OK;
}

int psi_decode_queries(psi_ctx *ctx, const void *F, int64_t n_pix, int D, const void *Q, int n_q, const float *T,
                       int32_t *ids, void *logits, psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    if (n_pix < 0 || n_pix >= (int64_t(1) << 31)) return fail(ctx, PSI_ERR_INVALID_ARG, "n_pix out of range");
    if (D != 64 && D != 128) return fail(ctx, PSI_ERR_UNSUPPORTED, "D must be 64 or 128");
    if (n_q < 1 || n_q > 128) return fail(ctx, PSI_ERR_INVALID_ARG, "n_q must be in [1,128]");
    if (n_pix > 0 && (!F || !Q || !T || !ids)) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL argument");
    if (!aligned(F, 16) || !aligned(Q, 16)) return fail(ctx, PSI_ERR_INVALID_ARG, "F and Q must be 16-byte aligned");
    if (logits && ((!aligned(logits, 4) && (n_q % 2) == 0) || !aligned(logits, 2)))
        return fail(ctx, PSI_ERR_INVALID_ARG, "logits must be 2-byte aligned (4-byte for an even n_q)");
    if (n_pix == 0) return PSI_OK;
    DeviceGuard g(ctx->device);
    const char *why = nullptr;
    cudaError_t e = psi::launch_decode(F, n_pix, D, Q, n_q, T, ids, logits, ctx->status,
                                       reinterpret_cast<cudaStream_t>(stream), &why);
    if (why) return fail(ctx, PSI_ERR_CUDA, "psi_decode_queries: %s", why);
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_decode_queries", e);
}

int psi_attention_workspace_size(int64_t n, int C, int d, int n_q, size_t *bytes)
{
    if (!bytes || n < 0 || C < 1 || d < 1 || n_q < 1) return PSI_ERR_INVALID_ARG;
    *bytes = psi::attention_workspace_bytes(n, C, d, n_q);
    return PSI_OK;
}

int psi_frustum_attention(psi_ctx *ctx, const psi_surfels *s, const psi_features *f, const psi_camera *cam,
                          float z_near, const float *Q, int n_q, const float *W_Q, const float *W_K, const float *W_V,
                          int d, float *out, void *workspace, size_t workspace_bytes, psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    int rc;
    if ((rc = check_surfels(ctx, s))) return rc;
    psi::FeatView fv;
    if ((rc = check_feat(ctx, f, fv))) return rc;
    if (!fv.data) return fail(ctx, PSI_ERR_INVALID_ARG, "features are required");
    if (fv.dtype != PSI_BF16 || fv.scale || (fv.dim != 64 && fv.dim != 128))
        return fail(ctx, PSI_ERR_UNSUPPORTED, "psi_frustum_attention: BF16 features without scale, dim 64 or 128 "
                                              "(convert with psi_quantize_features)");
    if (!cam || cam->width < 1 || cam->height < 1) return fail(ctx, PSI_ERR_INVALID_ARG, "bad camera");
    if (s->n >= (int64_t(1) << 31)) return fail(ctx, PSI_ERR_INVALID_ARG, "too many surfels");
    if (n_q < 1 || n_q > 128 || d < 1 || d > 256) return fail(ctx, PSI_ERR_INVALID_ARG, "need 1 <= n_q <= 128, 1 <= d <= 256");
    if (!Q || !W_Q || !W_K || !W_V || !out) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL argument");
    const size_t need = psi::attention_workspace_bytes(s->n, fv.dim, d, n_q);
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256))
        return fail(ctx, PSI_ERR_INVALID_ARG, "workspace must be >= %zu bytes, 256-byte aligned", need);
    if (s->n == 0) return fail(ctx, PSI_ERR_INVALID_ARG, "no surfels to attend to");
    DeviceGuard g(ctx->device);
    const char *why = nullptr;
    cudaError_t e = psi::launch_attention(*s, fv.data, fv.dim, *cam, z_near, Q, n_q, W_Q, W_K, W_V, d, out, workspace,
                                          ctx->status, reinterpret_cast<cudaStream_t>(stream), &why);
    if (why) return fail(ctx, PSI_ERR_CUDA, "psi_frustum_attention: %s", why);
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_frustum_attention", e);
}

int psi_frustum_attention_bwd(psi_ctx *ctx, const psi_surfels *s, const psi_features *f, const float *Q, int n_q,
                              const float *W_Q, const float *W_K, const float *W_V, int d, const float *g_out,
                              float *g_Q, float *g_WQ, float *g_WK, float *g_WV, const psi_grads *grads,
                              void *workspace, size_t workspace_bytes, psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    int rc;
    if ((rc = check_surfels(ctx, s))) return rc;
    psi::FeatView fv;
    if ((rc = check_feat(ctx, f, fv))) return rc;
    if (!fv.data || s->n == 0) return fail(ctx, PSI_ERR_INVALID_ARG, "features and surfels are required");
    if (fv.dtype != PSI_BF16 || fv.scale || (fv.dim != 64 && fv.dim != 128))
        return fail(ctx, PSI_ERR_UNSUPPORTED, "psi_frustum_attention_bwd: BF16 features without scale, dim 64 or 128");
    if (s->n >= (int64_t(1) << 31)) return fail(ctx, PSI_ERR_INVALID_ARG, "too many surfels");
    if (n_q < 1 || n_q > 128 || d < 1 || d > 256) return fail(ctx, PSI_ERR_INVALID_ARG, "need 1 <= n_q <= 128, 1 <= d <= 256");
    if (!Q || !W_Q || !W_K || !W_V || !g_out) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL argument");
    if (grads && grads->feat && !aligned(grads->feat, 16))
        return fail(ctx, PSI_ERR_INVALID_ARG, "grads->feat must be 16-byte aligned");
    const size_t need = psi::attention_workspace_bytes(s->n, fv.dim, d, n_q);
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256))
        return fail(ctx, PSI_ERR_INVALID_ARG, "workspace must be >= %zu bytes, 256-byte aligned", need);
    DeviceGuard g(ctx->device);
    const char *why = nullptr;
    cudaError_t e = psi::launch_attention_bwd(*s, fv.data, fv.dim, Q, n_q, W_Q, W_K, W_V, d, g_out, g_Q, g_WQ, g_WK,
                                              g_WV, grads ? grads->feat : nullptr, grads ? grads->mu : nullptr,
                                              workspace, ctx->status, reinterpret_cast<cudaStream_t>(stream), &why);
    if (why) return fail(ctx, PSI_ERR_CUDA, "psi_frustum_attention_bwd: %s", why);
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_frustum_attention_bwd", e);
}

int psi_surfel_geometry(psi_ctx *ctx, const psi_surfels *s, const psi_camera *cam, float *table, int ld,
                        psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    int rc = check_surfels(ctx, s);
    if (rc) return rc;
    if (!cam) return fail(ctx, PSI_ERR_INVALID_ARG, "cam is NULL");
    if (ld < 16 || ld > 256 || ld % 16 != 0) return fail(ctx, PSI_ERR_INVALID_ARG, "ld must be a multiple of 16 in [16,256]");
    if (s->n > 0 && (!table || !aligned(table, 16))) return fail(ctx, PSI_ERR_INVALID_ARG, "table must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    cudaError_t e = psi::launch_geometry(*s, *cam, table, ld, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_surfel_geometry", e);
}

int psi_surfel_geometry_bwd(psi_ctx *ctx, const psi_surfels *s, const psi_camera *cam, const float *g_table, int ld,
                            const psi_grads *grads, psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    int rc = check_surfels(ctx, s);
    if (rc) return rc;
    if (!cam || !grads) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL argument");
    if (ld < 16 || ld > 256 || ld % 16 != 0) return fail(ctx, PSI_ERR_INVALID_ARG, "ld must be a multiple of 16 in [16,256]");
    if (s->n > 0 && (!g_table || !aligned(g_table, 16)))
        return fail(ctx, PSI_ERR_INVALID_ARG, "g_table must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    cudaError_t e = psi::launch_geometry_bwd(*s, *cam, g_table, ld, *grads, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_surfel_geometry_bwd", e);
}

int psi_quantize_features(psi_ctx *ctx, const float *f, int64_t n, int dim, int dtype, void *q, float *scale,
                          psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    if (n < 0 || dim < 16 || dim > 256 || dim % 16) return fail(ctx, PSI_ERR_INVALID_ARG, "need n >= 0, dim in [16, 256] a multiple of 16");
    if (dtype != PSI_BF16 && dtype != PSI_FP8_E4M3) return fail(ctx, PSI_ERR_INVALID_ARG, "dtype must be PSI_BF16 or PSI_FP8_E4M3");
    if (n > 0 && (!f || !q)) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL argument");
    if (dtype == PSI_FP8_E4M3 && !scale) return fail(ctx, PSI_ERR_INVALID_ARG, "FP8 needs a scale buffer");
    if (!aligned(f, 16) || !aligned(q, 16) || !aligned(scale, 16))
        return fail(ctx, PSI_ERR_INVALID_ARG, "f, q and scale must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    cudaError_t e = psi::launch_quantize(f, n, dim, dtype, q, scale, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_quantize_features", e);
}

int psi_grads_zero(psi_ctx *ctx, const psi_grads *grads, int64_t n, int dim, psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    if (!grads || n < 0 || dim < 0) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL grads or negative size");
    DeviceGuard g(ctx->device);
    auto st = reinterpret_cast<cudaStream_t>(stream);
    const size_t N = static_cast<size_t>(n);
    float *const ptrs[] = {grads->mu, grads->tu, grads->tv, grads->scale, grads->opacity, grads->rgb, grads->feat};
    const int64_t counts[] = {3 * n, 3 * n, 3 * n, 2 * n, n, 3 * n, static_cast<int64_t>(N) * dim};
    cudaError_t e = psi::launch_zero_parts(ptrs, counts, 7, st);
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_grads_zero", e);
}

int psi_quat_frames(psi_ctx *ctx, const float *q, int64_t n, float *tu, float *tv, psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!q || !tu || !tv))) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL argument or n < 0");
    if (!aligned(q, 16)) return fail(ctx, PSI_ERR_INVALID_ARG, "q must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    cudaError_t e = psi::launch_frames(q, n, tu, tv, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_quat_frames", e);
}

int psi_quat_frames_bwd(psi_ctx *ctx, const float *q, int64_t n, const float *g_tu, const float *g_tv, float *g_q,
                        psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!q || !g_q))) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL argument or n < 0");
    if (!aligned(q, 16) || !aligned(g_q, 16)) return fail(ctx, PSI_ERR_INVALID_ARG, "q and g_q must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    cudaError_t e = psi::launch_frames_bwd(q, n, g_tu, g_tv, g_q, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_quat_frames_bwd", e);
}

int psi_surfel_regularisers(psi_ctx *ctx, const psi_surfels *s, const int32_t *node_of, const float *node_mu,
                            const float *node_n, int64_t n_nodes, float lambda_n, float w_geo, float w_iso,
                            double *losses, const psi_grads *grads, psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    int rc;
    if ((rc = check_surfels(ctx, s))) return rc;
    if (!losses || !grads) return fail(ctx, PSI_ERR_INVALID_ARG, "losses and grads are required");
    if (n_nodes < 0 || (n_nodes > 0 && (!node_mu || !node_n)))
        return fail(ctx, PSI_ERR_INVALID_ARG, "node arrays are required for n_nodes > 0");
    if (!aligned(losses, 8)) return fail(ctx, PSI_ERR_INVALID_ARG, "losses must be 8-byte aligned");
    DeviceGuard g(ctx->device);
    cudaError_t e = psi::launch_regularisers(*s, node_of, node_mu, node_n, n_nodes, lambda_n, w_geo, w_iso, losses,
                                             *grads, ctx->status, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_surfel_regularisers", e);
}

int psi_surfel_logits(psi_ctx *ctx, const psi_features *f, int64_t n, const void *Q, int n_q, void *table,
                      int table_dtype, int ld, psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(ctx, PSI_ERR_INVALID_ARG, "n out of range");
    if (!f || !f->data) return fail(ctx, PSI_ERR_INVALID_ARG, "features are required");
    if (f->dtype != PSI_BF16 || f->scale) return fail(ctx, PSI_ERR_UNSUPPORTED, "logits need BF16 features without scale");
    if (f->dim != 64 && f->dim != 128) return fail(ctx, PSI_ERR_UNSUPPORTED, "D must be 64 or 128");
    if (n_q < 1 || n_q > 128) return fail(ctx, PSI_ERR_INVALID_ARG, "n_q must be in [1,128]");
    if (ld < n_q || ld > 128 || ld % 16 != 0) return fail(ctx, PSI_ERR_INVALID_ARG, "ld must be a multiple of 16 in [n_q, 128]");
    if (table_dtype != PSI_F32 && table_dtype != PSI_BF16)
        return fail(ctx, PSI_ERR_INVALID_ARG, "table_dtype must be PSI_F32 or PSI_BF16");
    if (n > 0 && (!Q || !table)) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL argument");
    if (!aligned(f->data, 16) || !aligned(Q, 16) || !aligned(table, 16))
        return fail(ctx, PSI_ERR_INVALID_ARG, "features, Q and table must be 16-byte aligned");
    if (n == 0) return PSI_OK;
    DeviceGuard g(ctx->device);
    const char *why = nullptr;
    cudaError_t e = psi::launch_logits(f->data, n, f->dim, Q, n_q, table, ld, table_dtype == PSI_BF16, ctx->status,
                                       reinterpret_cast<cudaStream_t>(stream), &why);
    if (why) return fail(ctx, PSI_ERR_CUDA, "psi_surfel_logits: %s", why);
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_surfel_logits", e);
}

int psi_surfel_labels(psi_ctx *ctx, const psi_features *f, const float *centres, int64_t n, const void *Q, int n_q,
                      const float *q_mu, const float *q_cov, void *labels, int labels_dtype, int ld, psi_stream stream)
{
    NvtxRange nvtx_range(__func__);
    if (!ctx) return PSI_ERR_INVALID_ARG;
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(ctx, PSI_ERR_INVALID_ARG, "n out of range");
    if (!f || !f->data) return fail(ctx, PSI_ERR_INVALID_ARG, "features are required");
    if (f->dtype != PSI_BF16 || f->scale) return fail(ctx, PSI_ERR_UNSUPPORTED, "labels need BF16 features without scale");
    if (f->dim != 64 && f->dim != 128) return fail(ctx, PSI_ERR_UNSUPPORTED, "D must be 64 or 128");
    if (n_q < 1 || n_q > 128) return fail(ctx, PSI_ERR_INVALID_ARG, "n_q must be in [1,128]");
    if (ld < n_q || ld > 128 || ld % 16 != 0) return fail(ctx, PSI_ERR_INVALID_ARG, "ld must be a multiple of 16 in [n_q, 128]");
    if (labels_dtype != PSI_F32 && labels_dtype != PSI_BF16)
        return fail(ctx, PSI_ERR_INVALID_ARG, "labels_dtype must be PSI_F32 or PSI_BF16");
    if (n > 0 && (!centres || !Q || !q_mu || !q_cov || !labels)) return fail(ctx, PSI_ERR_INVALID_ARG, "NULL argument");
    if (!aligned(f->data, 16) || !aligned(Q, 16) || !aligned(labels, 16))
        return fail(ctx, PSI_ERR_INVALID_ARG, "features, Q and labels must be 16-byte aligned");
    if (n == 0) return PSI_OK;
    DeviceGuard g(ctx->device);
    const char *why = nullptr;
    cudaError_t e = psi::launch_labels(f->data, n, f->dim, centres, Q, n_q, q_mu, q_cov, labels, ld,
                                       labels_dtype == PSI_BF16, ctx->status, reinterpret_cast<cudaStream_t>(stream), &why);
    if (why) return fail(ctx, PSI_ERR_CUDA, "psi_surfel_labels: %s", why);
    return e == cudaSuccess ? PSI_OK : cuda_fail(ctx, "psi_surfel_labels", e);
}

} // extern "C"
