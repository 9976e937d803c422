/*
 * psi.h -- C ABI of libpsi, a GB300 (sm_103a) implementation of the rendering
 * hot path of "Psi-Map: Panoptic Surface Integrated Mapping Enables Real2Sim
 * Transfer" (arXiv 2604.10982): tile-based differentiable rasterisation of 2D
 * Gaussian surfels carrying RGB and a D-dimensional feature, with Precise Tile
 * Intersection and Top-K Hard Selection (Sec. 5), and the query decode of the
 * rendered feature map (Sec. 4.1, Eq. 4).
 *
 * General rules for every entry point:
 *  - All array pointers are DEVICE pointers owned by the caller, unless a
 *    comment says "host". The library never frees caller memory.
 *  - Work is enqueued asynchronously on the caller's stream `stream`
 *    (a cudaStream_t; NULL = legacy default stream). No entry point
 *    synchronises the host except psi_status_fetch and the launch-shape
 *    tuners psi_tune_render_fwd / psi_tune_render_bwd, so a whole frame of
 *    the other calls can be captured in a CUDA graph.
 *  - Return value: PSI_OK or an error code; psi_last_error(ctx) then holds a
 *    readable message. Host-side argument checks return PSI_ERR_INVALID_ARG
 *    (or PSI_ERR_UNSUPPORTED) before anything is enqueued.
 *  - Errors found on the device (pair-buffer overflow, a bounded wait that gave
 *    up) are OR-ed into the context's device status word; read and clear it
 *    with psi_status_fetch() after the stream has run.
 *  - Camera convention: OpenCV axes (x right, y down, z forward),
 *    x_cam = R x_world + t, pixel (px,py) samples the point (px+1/2, py+1/2).
 *  - Views are concatenated: view v owns tiles [tile_base(v), tile_base(v) +
 *    tiles_x*tiles_y) and pixels [pix_base(v), pix_base(v) + W*H), both
 *    prefix sums over the views in order (see psi_view_layout).
 *  - A "record" is one (view, surfel) pair with index r = v*N + i.
 */
#ifndef PSI_H
#define PSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct psi_ctx psi_ctx;
typedef struct CUstream_st *psi_stream; /* same type as cudaStream_t */

enum psi_status {
    PSI_OK = 0,
    PSI_ERR_INVALID_ARG = 1,
    PSI_ERR_CUDA = 2,
    PSI_ERR_CAPACITY = 3,  /* device: more (tile, surfel) pairs than the key buffer holds */
    PSI_ERR_TIMEOUT = 4,   /* device: a bounded wait gave up (the results are invalid) */
    PSI_ERR_UNSUPPORTED = 5,
    PSI_ERR_BOUNDS = 6     /* device, debug build only: an index taken from data failed a bounds
                              check; the access was clamped to a valid one (results invalid) */
};

/* Tile-intersection modes (Sec. 5, "Precise Tile Intersection"):
 *  SPHERE: square of radius chi*sqrt(lambda_max(Sigma')) -- the isotropic
 *          bounding sphere the paper replaces (its "Baseline" row);
 *  AABB:   the paper's box with half-widths sqrt(chi^2 Sigma'_11),
 *          sqrt(chi^2 Sigma'_22) of the projected covariance;
 *  EXACT:  per tile row, only the tiles whose pixel-centre columns meet the
 *          projected ellipse itself. */
enum psi_isect_mode { PSI_ISECT_SPHERE = 0, PSI_ISECT_AABB = 1, PSI_ISECT_EXACT = 2 };

/* Storage types of the per-surfel feature table (FP32 accumulation always). */
enum psi_dtype { PSI_F32 = 0, PSI_BF16 = 1, PSI_FP8_E4M3 = 2 };

#define PSI_MAX_VIEWS 64
#define PSI_RECORD_BYTES 80     /* render record per (view, surfel) */
#define PSI_BIN_RECORD_BYTES 32 /* binning record per (view, surfel) */
#define PSI_BIN_RECORD_BYTES_LOWPASS 48 /* the same with psi_render_opts.lowpass set */
#define PSI_MAX_TOPK 32

/* Surfels (Sec. 3.1): a 2D Gaussian in the plane through mu spanned by the
 * tangent axes t_u, t_v with scales (s_u, s_v): P(u,v) = mu + s_u u t_u +
 * s_v v t_v; opacity o; colour c. All float32, row-major, N rows. */
typedef struct {
    const float *mu;      /* [N,3] */
    const float *tu;      /* [N,3] */
    const float *tv;      /* [N,3] */
    const float *scale;   /* [N,2] (s_u, s_v) */
    const float *opacity; /* [N] */
    const float *rgb;     /* [N,3] */
    int64_t n;
} psi_surfels;

/* Pinhole camera (host struct). */
typedef struct {
    float R[9];  /* row-major world->camera rotation */
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
} psi_camera;

/* Per-surfel features f_i (Sec. 4.1): [N, dim] row-major in `dtype`.
 * Value of channel c is q[i,c] * scale[c] (scale may be NULL for F32/BF16,
 * meaning 1). dim must be a multiple of 16 in [16, 256]; rows must start on
 * 16-byte boundaries. */
typedef struct {
    const void *data;
    const float *scale; /* [dim] or NULL */
    int32_t dtype;      /* enum psi_dtype */
    int32_t dim;
} psi_features;

/* Options (host struct). Defaults: see psi_default_opts. */
typedef struct {
    int32_t mode;           /* enum psi_isect_mode */
    int32_t top_k;          /* K of Top-K Hard Selection (Sec. 5); 0 = dense features */
    float chi2;             /* squared support radius in (u,v) units (paper: "e.g. 3 sigma" -> 9) */
    float z_near;           /* near plane; the whole support disc must lie beyond it */
    int32_t opacity_radius; /* 1: shrink the radius to where o*exp(-d^2/2) reaches 1/255 */
    int32_t tile_w, tile_h; /* tile size in pixels: 16x16, or 16x8 (top_k in 1..8, no low-pass
                               filter): smaller tiles give shorter lists per CTA for more
                               (tile, surfel) pairs; which is faster depends on the frame */
    float t_eps;            /* stop a pixel after the surfel that takes T below this */
    int32_t lowpass;        /* 1: the 2DGS object-space low-pass filter (Sec. 3.1 surfels
                               follow 2DGS): the Gaussian argument is min(u^2+v^2, 2|x-c|^2),
                               c the pixel position of the projected centre, so a surfel
                               seen edge on still covers about one pixel; the support is
                               that argument <= r^2. Bin records are then
                               PSI_BIN_RECORD_BYTES_LOWPASS bytes. 0: off (default) */
} psi_render_opts;

/* Forward outputs (device pointers; NULL = not written unless stated). Pixel p of
 * view v is at index pix_base(v) + py*W + px.
 *  rgb:      [3][P_total] planar per channel (channel c at c*P_total + p); required
 *  T:        [P_total] final transmittance; required
 *  n_last:   [P_total] int32, 1 + list position of the last surfel composited (0: none)
 *  F:        [P_total, D] feature map in F_dtype (PSI_F32 or PSI_BF16)
 *  topk_ids: [P_total, K] int32 surfel ids of the selected set in list order, -1 padded
 *  topk_w:   [P_total, K] float32 weights omega_j = alpha_j T_j of those surfels, 0 padded
 *  argmax:   [P_total] int32 channel of F's largest value (lowest channel on ties; FP32
 *            before any BF16 rounding), -1 where 1 - T < 1e-4; top_k > 0 only. With F
 *            NULL the feature mixture is formed in registers and never written: for a
 *            label table from psi_surfel_labels this is the instance identity of Eq. 8 */
typedef struct {
    float *rgb;
    float *T;
    int32_t *n_last;
    void *F;
    int32_t F_dtype;
    int32_t *topk_ids;
    float *topk_w;
    int32_t *argmax;
} psi_fwd_out;

/* Gradients (device, float32, ACCUMULATED into: the caller zeroes them). Any
 * member may be NULL to skip it (feat is skipped automatically without g_F). */
typedef struct {
    float *mu;      /* [N,3] */
    float *tu;      /* [N,3] */
    float *tv;      /* [N,3] */
    float *scale;   /* [N,2] */
    float *opacity; /* [N] */
    float *rgb;     /* [N,3] */
    float *feat;    /* [N,D] gradient w.r.t. the dequantised feature values */
} psi_grads;

/* ---- context ---------------------------------------------------------- */

/* Create a context on CUDA device `device` (allocates a 16-byte device status
 * word). *out receives the handle (NULL on failure): PSI_ERR_INVALID_ARG if
 * `device` is not a CUDA device of this machine, PSI_ERR_CUDA if an
 * allocation fails. */
int psi_ctx_create(psi_ctx **out, int device);
void psi_ctx_destroy(psi_ctx *ctx);
/* Message of the last failing call on ctx (never NULL; "" if none). */
const char *psi_last_error(const psi_ctx *ctx);
/* Synchronises `stream`, copies the device status word to *status_out
 * (0 = clean, else a PSI_ERR_* code; TIMEOUT before BOUNDS before CAPACITY
 * before INVALID_ARG) and *detail (may be NULL): for PSI_ERR_CAPACITY the pair
 * count the overflowing frame needed, for PSI_ERR_BOUNDS 100 + the check site
 * (1 tile of the launch order, 2 tile range, 3 record index of a list entry,
 * 4 surfel id of a selected slot, 5 a saved last position past its tile's
 * list), for PSI_ERR_TIMEOUT the code of the first wait
 * that gave up (1 render, 2/3 adjoint passes, 4-6 decode, 7 drain,
 * 8 sort); then
 * clears the word. */
int psi_status_fetch(psi_ctx *ctx, psi_stream stream, int32_t *status_out, int64_t *detail);

/* Failure detection (no counterpart in the paper): every wait of the
 * kernels' copy and MMA pipelines gives up after the context's wait limit
 * (default 1 s), raises PSI_ERR_TIMEOUT with its wait site in the status word
 * and lets the kernel return; the copies and MMA groups it had started are
 * still awaited (with the fixed 1 s limit) before its shared memory and TMEM
 * are released. psi_ctx_set_wait_limit_ns sets the limit for kernels launched
 * after it returns (0 restores 1 s; at most PSI_WAIT_LIMIT_MAX_NS, else
 * PSI_ERR_INVALID_ARG). A limit shorter than a kernel's normal waits makes
 * its outputs invalid: it exists to exercise the give-up path. Synchronous
 * copy to the device: not inside a stream capture. */
#define PSI_WAIT_LIMIT_MAX_NS 10000000000ull
int psi_ctx_set_wait_limit_ns(psi_ctx *ctx, uint64_t ns);

/* 1 if this library was built with PSI_DEBUG: every index the pipeline
 * kernels take from data (the tile launch order, tile ranges, the record
 * index of a list entry, the surfel ids of selected slots, the caller's saved
 * Top-K ids) is checked against its buffer before use; a failure raises
 * PSI_ERR_BOUNDS with the check site and the access is clamped to a valid
 * index instead of faulting. 0 for the release build, which has no checks. */
int psi_debug_checks(void);

/* Kernels psi_ctx_time_kernel can bracket: those that share an entry point
 * with other kernels (psi_render_bwd launches the feature kernel, the list
 * walk and the chain kernel). */
enum psi_kernel_id { PSI_KERNEL_BWD_FEAT = 1, PSI_KERNEL_BWD_WALK = 2 };
/* Kernel timing, a tracing aid with no counterpart in the paper: arm a
 * one-shot pair of CUDA events (cudaEvent_t created with timing enabled,
 * passed as void*) that the next launch of `kernel` through this context
 * records on the call's stream, ev_begin right before the launch and ev_end
 * right after it; the pair is then disarmed (NULL, NULL disarms it early). The
 * caller reads cudaEventElapsedTime once the stream has run. Meant for eager
 * launches: inside a stream capture a plain event record adds no graph node.
 * PSI_ERR_INVALID_ARG for an unknown kernel or only one event. */
int psi_ctx_time_kernel(psi_ctx *ctx, int kernel, void *ev_begin, void *ev_end);
/* Fill *o with the defaults: EXACT, K=0, chi2=9, z_near=0.2, no opacity
 * radius, 16x16 tiles, t_eps=1e-4. */
void psi_default_opts(psi_render_opts *o);
/* Host helper: tile_base[n_views+1] and pix_base[n_views+1] (host arrays). */
int psi_view_layout(const psi_camera *cams, int n_views, const psi_render_opts *o, int64_t *tile_base,
                    int64_t *pix_base);

/* ---- workspace sizes (bytes of caller-allocated scratch, 256-B aligned) -- */
int psi_intersect_workspace_size(int64_t n_records, size_t *bytes);
int psi_sort_workspace_size(int64_t capacity, size_t *bytes);
/* Adjoint scratch: per-record moments (n_records = n_views * N) and, for
 * top_k > 0, one float per (pixel, selected slot) (n_pix = P_total). */
int psi_render_bwd_workspace_size(int64_t n_records, int64_t n_pix, int top_k, size_t *bytes);

/* ---- a1: projection and ray-splat setup --------------------------------
 * Per (view, surfel): camera transform, the pixel-homogeneous 3x3 map M of the
 * surfel plane (the ray-splat intersection of Sec. 3.1 in homogeneous form),
 * culling (opacity < 1/255, or any part of the support disc nearer than
 * z_near), the support radius, the ellipse bounds of the projected covariance
 * (Sec. 5, Precise Tile Intersection) and the tile count of `o->mode`.
 *  records:       [n_views*N] x PSI_RECORD_BYTES, 16-byte aligned (written for visible records)
 *  bin_records:   [n_views*N] x PSI_BIN_RECORD_BYTES (PSI_BIN_RECORD_BYTES_LOWPASS with
 *                 o->lowpass), 16-byte aligned
 *  tiles_touched: [n_views*N] uint32, 0 for culled records
 * cams is a HOST array of n_views (<= PSI_MAX_VIEWS) cameras. */
int psi_project_surfels(psi_ctx *ctx, const psi_surfels *s, const psi_camera *cams, int n_views,
                        const psi_render_opts *o, void *records, void *bin_records, uint32_t *tiles_touched,
                        psi_stream stream);

/* ---- a2: tile intersection and key emission (Sec. 5) -------------------
 * Exclusive scan of tiles_touched, then one (key, value) pair per (tile,
 * record): key = global_tile << 32 | float bits of the camera depth, value =
 * record index; records in index order, tiles row-major within a record.
 *  keys, vals:  [capacity]; d_num_pairs: device int64 receiving the pair count
 *  workspace:   psi_intersect_workspace_size(n_views*N) bytes
 * If the count exceeds capacity, pairs beyond it are dropped, *d_num_pairs is
 * clamped to capacity and PSI_ERR_CAPACITY is raised on the device. */
int psi_intersect_tiles(psi_ctx *ctx, const psi_camera *cams, int n_views, const psi_render_opts *o,
                        int64_t n_surfels, const void *bin_records, const uint32_t *tiles_touched, uint64_t *keys,
                        uint32_t *vals, int64_t capacity, int64_t *d_num_pairs, void *workspace,
                        size_t workspace_bytes, psi_stream stream);

/* ---- a3: key sort and tile ranges ----------------------------------------
 * Stable LSD radix sort of the first *d_num_pairs (key, value) pairs on key
 * bits [begin_bit, end_bit) (in place: results end in keys/vals), then
 * tile_ranges[2*t] = start, [2*t+1] = end of global tile t (0,0 if empty),
 * and tile_ranges[2*n_tiles_total + i], i < n_tiles_total, the launch order of
 * the compositing kernels (tiles by descending list length; the order among
 * tiles of similar length is arbitrary and never changes a result). The
 * tile_ranges buffer therefore holds 3*n_tiles_total uint32.
 * Pass begin_bit=0, end_bit=32+ceil(log2(n_tiles_total)) for the full order.
 * If *d_num_pairs exceeds capacity, only the first capacity pairs are sorted
 * and ranged, and PSI_ERR_CAPACITY (detail: *d_num_pairs) is raised on the
 * device; nothing is read or written past capacity.
 *  workspace: psi_sort_workspace_size(capacity) bytes. */
int psi_sort_keys(psi_ctx *ctx, uint64_t *keys, uint32_t *vals, const int64_t *d_num_pairs, int64_t capacity,
                  int begin_bit, int end_bit, uint32_t *tile_ranges, int64_t n_tiles_total, void *workspace,
                  size_t workspace_bytes, psi_stream stream);

/* ---- a3 without caller scratch (no counterpart in the paper) ------------
 * Same result as psi_sort_keys, for callers that cannot allocate device memory
 * for a workspace: real-time loops that must not stall on an allocator, or
 * plug-ins running under a host framework that owns every device allocation
 * and hands them only their inputs and outputs. The scratch is a fixed array
 * inside the library (PSI_SORT_NOALLOC_SCRATCH_BYTES per device, reserved when
 * the library's module loads on that device and held until the process
 * exits); this call allocates and frees nothing.
 *  - capacity must be <= PSI_SORT_NOALLOC_MAX_PAIRS, else PSI_ERR_INVALID_ARG.
 *  - Devices 0 .. PSI_SORT_NOALLOC_MAX_DEVICES-1 only (PSI_ERR_INVALID_ARG
 *    beyond).
 *  - The first call on a device (with that device current) looks up the
 *    array's device address and keeps it for the life of the process; make
 *    that first call before any stream capture. After cudaDeviceReset the
 *    kept address is stale: do not call this entry point again in that
 *    process.
 *  - All calls on a device share the one array and it keeps the previous
 *    call's contents (the sort needs nothing zeroed in it): calls that overlap
 *    on the GPU (different streams, or concurrent host threads) race and give
 *    wrong results. Serialise them on one stream. */
#define PSI_SORT_NOALLOC_MAX_PAIRS (1 << 20)
#define PSI_SORT_NOALLOC_SCRATCH_BYTES (13 << 20)
#define PSI_SORT_NOALLOC_MAX_DEVICES 64
int psi_sort_keys_noalloc(psi_ctx *ctx, uint64_t *keys, uint32_t *vals, const int64_t *d_num_pairs,
                          int64_t capacity, int begin_bit, int end_bit, uint32_t *tile_ranges, int64_t n_tiles_total,
                          psi_stream stream);

/* ---- a4: per-tile compositing with Top-K Hard Selection -----------------
 * Per pixel, front to back over its tile's list: alpha = min(0.99, o exp(-(u^2
 * +v^2)/2)) (Sec. 3.1), skipped if u^2+v^2 > r^2 or alpha < 1/255; RGB blended
 * densely with Eq. (1); the K largest weights omega_j = alpha_j T_j are kept
 * and F = sum_{j in Top-K} f_j omega_j (Sec. 5), summed in list order;
 * stop after the surfel that takes T below t_eps. K=0: dense features.
 * f may be NULL (RGB only). records/vals/tile_ranges come from a1-a3 with the
 * same cams and opts. */
int psi_render_fwd(psi_ctx *ctx, const psi_features *f, const void *records, const uint32_t *vals,
                   const uint32_t *tile_ranges, const psi_camera *cams, int n_views, int64_t n_surfels,
                   const psi_render_opts *o, const psi_fwd_out *out, psi_stream stream);

/* ---- a5: adjoint of a4 ----------------------------------------------------
 * Takes each pixel's final transmittance, last composited list position and
 * Top-K set from the forward (or recomputes the front-to-back pass, which gives
 * the same values), then walks back to front with suffix sums: dL/dalpha_j =
 * T_j s_j - (sum_{k>j} omega_k s_k + T_final g_T)/(1 - alpha_j), s_j = <gC,
 * c_j> + [j in K]<gF, f_j>, and chains through alpha = o G, (u,v) of the
 * homogeneous ray-splat map, to mu, t_u, t_v, s, o; also dL/dc, dL/df. g_F
 * and g_T may be NULL.
 *  g_rgb: [3][P_total] planar; g_F: [P_total, D] float32, 16-byte aligned
 *  (as grads->feat); g_T: [P_total]
 *  saved: NULL (recompute), or psi_render_fwd's outputs for the same records,
 *  vals, tile_ranges, cams and opts: T and n_last, and topk_ids and topk_w
 *  when top_k > 0 (other members ignored; missing ones are
 *  PSI_ERR_INVALID_ARG). With them the feature part of the adjoint (<gF, f_j>
 *  and dL/df) runs per pixel from the saved selection, outside the list walk.
 *  Outputs that do not belong to this frame give wrong gradients; nothing
 *  checks that.
 *  workspace: psi_render_bwd_workspace_size(n_views*N, P_total, top_k) bytes. */
int psi_render_bwd(psi_ctx *ctx, const psi_surfels *s, const psi_features *f, const void *records,
                   const uint32_t *vals, const uint32_t *tile_ranges, const psi_camera *cams, int n_views,
                   const psi_render_opts *o, const float *g_rgb, const float *g_F, const float *g_T,
                   const psi_fwd_out *saved, const psi_grads *grads, void *workspace, size_t workspace_bytes,
                   psi_stream stream);

/* Zero every non-NULL member of *grads ([n, 3], [n, 2], [n], [n, dim] floats
 * as laid out in psi_grads; 4-byte aligned) on `stream` with one kernel,
 * before an accumulating psi_render_bwd. No counterpart in the paper. */
int psi_grads_zero(psi_ctx *ctx, const psi_grads *grads, int64_t n, int dim, psi_stream stream);

/* ---- launch-shape autotuner for a4 and a5 (no counterpart in the paper) ---
 * The compositing kernels are compiled in PSI_RENDER_SHAPES launch shapes:
 * bit 0 of a shape builds the kernel for the other number of resident CTAs
 * per SM (top_k <= 8: forward and recomputing adjoint 3 -> 4, adjoint from
 * saved state 4 -> 3, its paired walk 4 -> 3; larger K and dense features:
 * 2 -> 1), i.e. registers per
 * thread against occupancy; bit 1 composites dense features
 * (top_k = 0, dim a multiple of 32) 16 channels per pass instead of 32;
 * bit 2 is the persistent launch: a few CTAs per SM, each taking tiles
 * (of all views) longest list first from a work counter kept in the context
 * (the last CTA resets it, so compositing calls through one context must not
 * overlap on the GPU); bit 3 (adjoint from saved state with top_k > 0 only)
 * walks the lists with two pixels per thread instead of one. With 16x8 tiles
 * (psi_render_opts.tile_h = 8) the kernels have one occupancy and bit 0
 * changes nothing.
 * Every shape computes the same result: the forward bit for bit, the adjoint
 * up to the order of its float32 atomic additions. Which one is fastest
 * depends on K, the feature dtype, the scene and the resolution, so it is
 * measured on the caller's own frame.
 * psi_tune_render_fwd / psi_tune_render_bwd take the arguments of
 * psi_render_fwd / psi_render_bwd (same requirements and errors) and run each
 * shape that exists for them once untimed, then `reps` times between two CUDA
 * events on `stream`; they write the mean ms per shape to ms[PSI_RENDER_SHAPES]
 * (-1 for a shape that does not exist), the fastest to *best, and store it in
 * the context for this (call, K class {0, <=8, <=16, <=32}, feature dtype,
 * lowpass, and for the adjoint whether `saved` is given). Later
 * psi_render_fwd / psi_render_bwd calls on the context launch that shape
 * (shape 0 until tuned). They wait for the stream (PSI_ERR_INVALID_ARG inside
 * a stream capture): tune before capturing a graph. The outputs hold a valid
 * result afterwards; the adjoint's gradient buffers are used as scratch and
 * are left zeroed.
 * psi_ctx_set_render_shape / psi_ctx_get_render_shape write or read the
 * stored shape directly: which = 0 forward, 1 adjoint; feat_dtype a
 * psi_dtype, or -1 without features; saved 0/1 (adjoint only). */
#define PSI_RENDER_SHAPES 16
int psi_tune_render_fwd(psi_ctx *ctx, const psi_features *f, const void *records, const uint32_t *vals,
                        const uint32_t *tile_ranges, const psi_camera *cams, int n_views, int64_t n_surfels,
                        const psi_render_opts *o, const psi_fwd_out *out, int reps, float *ms, int *best,
                        psi_stream stream);
int psi_tune_render_bwd(psi_ctx *ctx, const psi_surfels *s, const psi_features *f, const void *records,
                        const uint32_t *vals, const uint32_t *tile_ranges, const psi_camera *cams, int n_views,
                        const psi_render_opts *o, const float *g_rgb, const float *g_F, const float *g_T,
                        const psi_fwd_out *saved, const psi_grads *grads, void *workspace, size_t workspace_bytes,
                        int reps, float *ms, int *best, psi_stream stream);
int psi_ctx_set_render_shape(psi_ctx *ctx, int which, const psi_render_opts *o, int feat_dtype, int saved, int shape);
int psi_ctx_get_render_shape(psi_ctx *ctx, int which, const psi_render_opts *o, int feat_dtype, int saved, int *shape);

/* ---- a6: query decode (Sec. 4.1, Eq. 4 without the monotone sigmoid) -----
 * logits[p,q] = sum_c F[p,c] Q[q,c] on the tensor cores (BF16 in, FP32
 * accumulate), ids[p] = argmax_q (lowest q on ties), or -1 where 1 - T[p] <
 * 1e-4 (nothing rendered).
 *  F: [n_pix, D] BF16, 16-byte aligned rows; Q: [n_q, D] BF16; D in {64,128};
 *  1 <= n_q <= 128; T: [n_pix] float; ids: [n_pix] int32; logits: [n_pix, n_q]
 *  BF16 or NULL, 2-byte aligned (4-byte when n_q is even). */
int psi_decode_queries(psi_ctx *ctx, const void *F, int64_t n_pix, int D, const void *Q, int n_q, const float *T,
                       int32_t *ids, void *logits, psi_stream stream);

/* ---- frustum-constrained cross-attention (Sec. 4.1), forward -------------
 * Over the surfels j whose 99 % confidence disc meets the view frustum of
 * `cam` (the disc's bounding sphere, radius sqrt(chi2_2(0.99)) max(s_u, s_v),
 * against the near plane z_near and the image rectangle's four side planes):
 *   K_j = f_j + psi(mu_j), V_j = f_j,
 *   Q'_i = softmax_j((Q_i W_Q)(K_j W_K)^T / sqrt(d)) (V_j W_V).
 * psi: channel c encodes axis c mod 3 with sin (t = c/3 even) or cos (t odd)
 * at frequency 10000^(-6k/C), k = t/2 (the paper leaves psi open).
 * Computed as e_ij = qh_i . K_j with qh = (Q W_Q) W_K^T / sqrt(d) and Q' =
 * (sum_j P_ij V_j) W_V (associativity), so per surfel only the two
 * contractions with qh and with P run, on the tensor cores: BF16 operands
 * (qh, f, psi(mu), P rounded to BF16), FP32 accumulation, online softmax in
 * FP32; the feature table is read once. Inactive surfels are masked (weight
 * 0); no host synchronisation. An empty active set gives Q' = 0.
 *  f: BF16 feature table without scale, dim C in {64, 128} (other tables:
 *  PSI_ERR_UNSUPPORTED; psi_quantize_features makes one); n < 2^31 surfels;
 *  Q: [n_q, C] float32, 1 <= n_q <= 128; W_Q, W_K, W_V: [C, d] float32,
 *  1 <= d <= 256; out: [n_q, d] float32; all row-major, device.
 *  workspace: psi_attention_workspace_size(n, C, d, n_q) bytes (it keeps the
 *  view, the per-query softmax statistics and the attended values for the
 *  adjoint). */
int psi_attention_workspace_size(int64_t n, int C, int d, int n_q, size_t *bytes);
int psi_frustum_attention(psi_ctx *ctx, const psi_surfels *s, const psi_features *f, const psi_camera *cam,
                          float z_near, const float *Q, int n_q, const float *W_Q, const float *W_K, const float *W_V,
                          int d, float *out, void *workspace, size_t workspace_bytes, psi_stream stream);
/* Its adjoint for L = <g_out, Q'> ([n_q, d]), reusing the workspace exactly as
 * the preceding psi_frustum_attention left it (same surfels, features,
 * queries and weights; the view is taken from the workspace): writes g_Q
 * [n_q, C], g_WQ / g_WK / g_WV [C, d] (each may be NULL) and ADDS dL/df
 * (grads->feat, [n, C] float32, 16-byte aligned) and dL/dmu through psi
 * (grads->mu) for the active surfels. The softmax weights are recomputed per
 * tile of surfels from the forward's per-query maximum and sum; the same BF16
 * operand rounding as the forward. */
int psi_frustum_attention_bwd(psi_ctx *ctx, const psi_surfels *s, const psi_features *f, const float *Q, int n_q,
                              const float *W_Q, const float *W_K, const float *W_V, int d, const float *g_out,
                              float *g_Q, float *g_WQ, float *g_WK, float *g_WV, const psi_grads *grads,
                              void *workspace, size_t workspace_bytes, psi_stream stream);

/* ---- depth and normal maps (the 2D-surfel geometry of Sec. 3.1) -----------
 * psi_surfel_geometry writes, per surfel and for one camera (host struct), a
 * row (z, n_x, n_y, n_z, 0, ...) of ld floats: z = (R mu + t)_z, the camera
 * depth of the centre, and n = R (t_u x t_v) / |t_u x t_v|, the unit normal in
 * camera coordinates turned to face the camera (negated where n . x_cam > 0).
 * Rendered as a dense float32 feature table (dim = ld, top_k = 0, same camera)
 * it gives the expected depth sum_j omega_j z_j and normal sum_j omega_j n_j
 * maps. psi_surfel_geometry_bwd ADDS dL/dmu, dL/dt_u, dL/dt_v (grads->mu, tu,
 * tv; others ignored, any may be NULL) given g_table = dL/dtable, e.g. the
 * feature gradient (grads->feat) of psi_render_bwd for that render.
 *  table, g_table: [N, ld] float32, 16-byte aligned; ld a multiple of 16 in
 *  [16, 256]; t_u x t_v must not vanish. */
int psi_surfel_geometry(psi_ctx *ctx, const psi_surfels *s, const psi_camera *cam, float *table, int ld,
                        psi_stream stream);
int psi_surfel_geometry_bwd(psi_ctx *ctx, const psi_surfels *s, const psi_camera *cam, const float *g_table, int ld,
                            const psi_grads *grads, psi_stream stream);

/* ---- quaternion-parameterised tangent frames (2DGS form) ------------------
 * The paper's surfels follow 2DGS (Sec. 3.1), whose tangent frame is a
 * rotation R(q / |q|) of a quaternion q = (w, x, y, z): t_u, t_v are R's first
 * two columns. psi_quat_frames writes them ([n, 3] float32 each) for use as
 * psi_surfels.tu / tv; psi_quat_frames_bwd ADDS dL/dq ([n, 4]) given dL/dt_u,
 * dL/dt_v (either may be NULL), e.g. psi_grads.tu / tv from psi_render_bwd.
 * q, g_q: [n, 4] float32, 16-byte aligned; q must not be zero. */
int psi_quat_frames(psi_ctx *ctx, const float *q, int64_t n, float *tu, float *tv, psi_stream stream);
int psi_quat_frames_bwd(psi_ctx *ctx, const float *q, int64_t n, const float *g_tu, const float *g_tv, float *g_q,
                        psi_stream stream);

/* ---- geometric and anisotropy regularisers (Sec. 4.2) ---------------------
 * For surfel i with an assigned planar prior k = node_of[i] (k < 0: none;
 * k >= n_nodes raises PSI_ERR_INVALID_ARG in the status word):
 *   L_geo = sum_i |(mu_i - m_k).nhat_k| + lambda_n (1 - |n_i.nhat_k|),
 *           n_i = (t_u x t_v) / |t_u x t_v|   (point-to-plane distance and
 *           normal alignment against the prior)
 *   L_iso = sum_i (s_i1 - s_i2)^2            (anisotropy)
 * losses[0] = L_geo, losses[1] = L_iso (device float64, overwritten); the
 * gradients of w_geo L_geo + w_iso L_iso are ADDED to grads->mu, tu, tv,
 * scale (any may be NULL; other members ignored). node_of may be NULL (no
 * priors). node_mu, node_n: [n_nodes, 3] float32, node_n unit length. The
 * planar priors themselves (the paper's SOGMM nodes) come from the caller. */
int psi_surfel_regularisers(psi_ctx *ctx, const psi_surfels *s, const int32_t *node_of, const float *node_mu,
                            const float *node_n, int64_t n_nodes, float lambda_n, float w_geo, float w_iso,
                            double *losses, const psi_grads *grads, psi_stream stream);

/* ---- storage form of the feature table (precision of the features) -------
 * The paper keeps FP32 features; their stored precision is a reading: BF16 is
 * round-to-nearest-even of each value; FP8-E4M3 uses a per-channel scale
 * scale[c] = max(amax_c, 1e-30) / 448 (amax_c = max over surfels of |f[., c]|,
 * 448 = largest finite E4M3) and q = RNE(f / scale[c]) saturated to +-448, so
 * that f ~= q * scale[c] (psi_features.scale). Accumulation is FP32 always.
 *  f: [n, dim] float32; q: [n, dim] in dtype (PSI_BF16 or PSI_FP8_E4M3);
 *  scale: [dim] float32, written for FP8 (ignored for BF16, may be NULL);
 *  dim a multiple of 16 in [16, 256]; f, q, scale 16-byte aligned. */
int psi_quantize_features(psi_ctx *ctx, const float *f, int64_t n, int dim, int dtype, void *q, float *scale,
                          psi_stream stream);

/* ---- per-surfel query logits: the decode fused into compositing ----------
 * table[g, q] = f_q^T f_g for every surfel (tensor cores, BF16 in, FP32
 * accumulate), zero past n_q. Since sum_j omega_j <f_j, q> = <F, q>, the
 * table rendered as a feature table by psi_render_fwd (Top-K selected) gives
 * every pixel's decode logits, and psi_fwd_out.argmax the decoded id (a6),
 * without the feature map F ever being written (F NULL). Computed once per
 * map (features and queries fixed), then rendered per frame.
 *  f: BF16 without scale, dim 64 or 128; Q: [n_q, D] BF16, 1 <= n_q <= 128;
 *  table: [n, ld] in table_dtype (PSI_F32 or PSI_BF16), 16-byte aligned, ld
 *  a multiple of 16 in [n_q, 128]. */
int psi_surfel_logits(psi_ctx *ctx, const psi_features *f, int64_t n, const void *Q, int n_q, void *table,
                      int table_dtype, int ld, psi_stream stream);

/* ---- per-surfel instance labels (Sec. 4.1, Eqs. 4-7) ---------------------
 * For each surfel g and instance query q:
 *   l[g, q] = softmax over q of sigmoid(f_q^T f_g) * D(q, g),
 *   D(q, g) = exp(-(p_g - mu_q)^T Sigma_q^-1 (p_g - mu_q) / 2),
 * the feature similarity (Eq. 4) times the ratio of the query Gaussian's
 * densities at the surfel centre p_g and at its own centre mu_q (Eq. 5),
 * normalised over the queries (Eqs. 6-7). f_q^T f_g runs on the tensor cores
 * (BF16 in, FP32 accumulate), the rest in FP32. The table has ld columns,
 * zero past n_q, so psi_render_fwd can render it as a feature table: F is
 * then the alpha-blended label mixture I of Eq. 8 (Top-K selected), and
 * psi_fwd_out.argmax its per-pixel instance identity.
 *  f: the surfel feature table, BF16 without scale, dim 64 or 128
 *  centres: [n, 3] float32 surfel centres (psi_surfels.mu); n < 2^31
 *  Q: [n_q, D] BF16 query features, 1 <= n_q <= 128, 16-byte aligned
 *  q_mu: [n_q, 3] float32 query centres; q_cov: [n_q, 6] float32 covariance
 *  entries (xx, xy, xz, yy, yz, zz), positive definite
 *  labels: [n, ld] in labels_dtype (PSI_F32 or PSI_BF16), 16-byte aligned;
 *  ld a multiple of 16 in [n_q, 128].
 * PSI_ERR_UNSUPPORTED for other feature types or dims. No counterpart call in
 * the paper's tables; the equations are its Sec. 4.1. */
int psi_surfel_labels(psi_ctx *ctx, const psi_features *f, const float *centres, int64_t n, const void *Q, int n_q,
                      const float *q_mu, const float *q_cov, void *labels, int labels_dtype, int ld,
                      psi_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* PSI_H */
