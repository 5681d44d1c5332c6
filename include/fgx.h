/*
 * fgx.h - C ABI of a GB300 (sm_103a) library for the generalised geodesic
 * distance transform computed by raster-scan passes.
 *
 * Method (FastGeodis, Implementation section; generalised GDT of the
 * Summary): starting from D0 = v * M (soft seed mask M), every directional
 * pass updates each element x of a line (a row in 2D, a plane in 3D) from the
 * already-updated previous line:
 *     D[x] = min(D[x], min_y D[y] + sqrt((1-lambda)*|x-y|^2_spacing
 *                                        + lambda*|I(x)-I(y)|^2))
 * over the 3 (2D) or 9 (3D) neighbours y of x in the previous line.  2D passes
 * run top-bottom, bottom-top, left-right, right-left; 3D passes run
 * front-back, back-front, top-bottom, bottom-top, left-right, right-left; the
 * whole schedule repeats `iterations` times.  Results are bit-exact to a
 * sequential float32 evaluation with IEEE square root and no fused
 * multiply-add (arithmetic order:
 *     s2 = ((dD*sD)^2 + (dH*sH)^2) + (dW*sW)^2, t = (1-lambda)*s2,
 *     di2 = sum over channels (in order) of (I(x)-I(y))^2,
 *     c = sqrt(t + lambda*di2), cand = D[y] + c).
 *
 * Conventions for every entry point:
 *  - Tensors are caller-owned, device-resident, float32, contiguous:
 *    image [B][C][H][W] or [B][C][D][H][W]; mask and dist [B][1][...].
 *  - The library never allocates device memory.  Entry points that need
 *    scratch take a caller-owned `workspace` whose size comes from the
 *    matching *_workspace_size query; its first 256 bytes hold a device
 *    status word (see fgx_workspace_status).
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *    default stream).  The returned status covers argument checks and launch
 *    errors only; a device-side timeout is reported by fgx_workspace_status
 *    after the caller synchronises.
 *  - dist may alias mask (computed in place); dist must not alias image.
 *  - Inputs must be finite, mask values >= +0 (no -0.0), v > 0 finite,
 *    0 <= lambda <= 1, iterations >= 0 (0 returns v * M), and squared
 *    intensity differences must not overflow float32; results for other
 *    inputs are undefined.
 *  - Host pointers, null pointers and bad sizes are rejected before any
 *    launch, with the codes below.
 */
#ifndef FGX_H
#define FGX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fgx_status {
    FGX_OK = 0,
    FGX_ERR_ARG = -1,             /* null pointer, bad scalar, bad option      */
    FGX_ERR_NOT_DEVICE_PTR = -2,  /* a tensor pointer is not device memory     */
    FGX_ERR_SHAPE = -3,           /* negative or unsupported extent            */
    FGX_ERR_WORKSPACE = -4,       /* workspace/saved buffer missing or small   */
    FGX_ERR_CUDA = -5,            /* a CUDA runtime call or launch failed      */
    FGX_ERR_TIMEOUT = -6,         /* (device status) an inter-block wait gave up */
    FGX_ERR_DEVICE = -7,          /* no usable sm_103 device                   */
    FGX_ERR_UNSUPPORTED = -8      /* valid request this build does not serve   */
} fgx_status;

/* Optional tuning knobs; pass NULL for defaults.  `size` must equal
 * sizeof(fgx_options) (forward compatibility). */
typedef struct fgx_options {
    uint32_t size;
    int32_t tile_lines;   /* lines per exchange block (ring width); 0 = auto.  3D with
                           * tile_width = tile_height = 0: 4 or 8 sets the ring width
                           * of every pass of the plane-tile kernel (8 where its tiles
                           * fit the grid); other values select the tiled engine */
    int32_t tile_width;   /* elements per tile along the inner in-line axis; 0 = auto */
    int32_t tile_height;  /* 3D: elements per tile along the outer in-line axis; 0 = auto */
    int32_t max_blocks;   /* cap on resident thread blocks; 0 = all that fit */
    int32_t timeout_ms;   /* inter-block wait limit; 0 = 2000 ms */
    int32_t segments;     /* 2D single-call forward: line segments per pass run at once
                           * speculatively (exact results; a segment whose start line
                           * changes runs again); 0 = as many as one block per SM
                           * allows, 1 = off, n = at most n (up to 8) */
    int32_t fast_math;    /* forward without parent codes: 1 = edge costs
                           * sqrt.approx(fma(lambda, di2, t_k)) (the intensity sum
                           * fused too) instead of the IEEE-rounded sequence; results
                           * within 1e-5 relative of the exact transform instead of
                           * bit-exact.  Only where the general cost formula applies
                           * (lambda != 0, and not lambda = 1 with one channel, whose
                           * |d| cost is exact and cheap); 0 = exact */
    int32_t no_cost_tables; /* 3D general cost (exact): 0 = the plane-tile kernel reads
                             * the edge costs from tables written once per call
                             * (nine floats per voxel and axis, held in the workspace,
                             * whose size query then includes them; a workspace too
                             * small for them computes the costs in every pass instead,
                             * with identical results); 1 = never (smaller workspace) */
    int32_t split_sms;    /* batches holding both 2D instances (line-chain launch) and
                           * 3D instances (plane-tile launch): the two launches run at
                           * the same time, the 2D one on a stream of the library's own
                           * forked from and joined back into the caller's stream,
                           * each with one thread block per SM of its share; n = the
                           * SMs of the 2D launch (the 3D launch gets the rest;
                           * clamped so that the largest instance of each launch has
                           * all its tiles resident, else one launch after the other),
                           * 0 = shares estimated from the work of each part, -1 = one
                           * launch after the other, each on every SM.  Results are
                           * the same bit for bit whatever the shares */
} fgx_options;

/* Human-readable name of a status code (static string). */
const char* fgx_status_string(int status);

/* Library version as major*10000 + minor*100 + patch. */
int fgx_version(void);

/* ------------------------------------------------------------ forward ---- */

/* Scratch bytes needed by fgx_geodesic2d / fgx_geodesic3d for this shape
 * (2D: D = 1, ndim = 2).  Writes *bytes; returns a status. */
int fgx_geodesic_workspace_size(int ndim, int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                                const fgx_options* opt, size_t* bytes);

/* 2D transform of B images (unit spacing).  image [B][C][H][W], mask and
 * dist [B][1][H][W].  Four passes per iteration (Implementation section). */
int fgx_geodesic2d(const float* image, const float* mask, float* dist, int64_t B, int64_t C,
                   int64_t H, int64_t W, float v, float lambda, int iterations,
                   void* workspace, size_t workspace_bytes, const fgx_options* opt,
                   void* stream);

/* 3D transform of B volumes.  image [B][C][D][H][W], mask and dist
 * [B][1][D][H][W]; spacing = (sD, sH, sW) > 0, read from host memory.  Six
 * passes per iteration (Implementation section). */
int fgx_geodesic3d(const float* image, const float* mask, float* dist, int64_t B, int64_t C,
                   int64_t D, int64_t H, int64_t W, const float spacing[3], float v,
                   float lambda, int iterations, void* workspace, size_t workspace_bytes,
                   const fgx_options* opt, void* stream);

/* Allocation-free forward, for callers that cannot allocate device memory
 * when they need a transform (code inside an allocator callback, real-time
 * loops on a fixed memory budget, plugins whose host framework owns every
 * allocation).  The paper has no counterpart: it
 * concerns only this library's memory handling.  Same arguments and results
 * as fgx_geodesic2d (ndim = 2, D = 1, spacing may be NULL) or fgx_geodesic3d
 * (ndim = 3), but the sweep's scratch (status word, barrier counter, tile
 * progress tags) is a 64 KiB static device array inside the library instead
 * of a caller workspace; every GPU that loads the library holds it until the
 * process exits.  Shapes whose scratch would exceed 64 KiB (about 8,000
 * instance-tiles per pass) are rejected with FGX_ERR_WORKSPACE before any
 * launch.  Each call made outside stream capture looks up the array's
 * device address (cudaGetSymbolAddress, with that device current); a call on
 * a capturing stream uses the address found by the last such call on that
 * device, so make the first call on each device before any stream capture.
 * All calls on one device
 * share that device's copy of the array, which keeps the last call's
 * contents; each call clears the part it uses, so calls that overlap on the
 * same GPU (for example on two streams) race and must be serialised by the
 * caller.  The call returns before the kernels finish; a device-side wait
 * timeout is recorded in the array's status word, which fgx_noalloc_status
 * reads.  No device memory is allocated or freed. */
int fgx_geodesic_noalloc(int ndim, const float* image, const float* mask, float* dist, int64_t B,
                         int64_t C, int64_t D, int64_t H, int64_t W, const float spacing[3],
                         float v, float lambda, int iterations, const fgx_options* opt,
                         void* stream);

/* Status of the last fgx_geodesic_noalloc call queued on `stream` on the
 * current device: copies the static array's status word to the host on
 * `stream` (no allocation), synchronises the stream, and returns FGX_OK or
 * the recorded device error (FGX_ERR_TIMEOUT).  The word is shared by every
 * call on the device, so with calls overlapping on other streams it may hold
 * theirs.  Returns FGX_ERR_CUDA if the copy fails.  The paper has no
 * counterpart. */
int fgx_noalloc_status(void* stream);

/* Device status word held in a workspace: copies it to the host on `stream`,
 * synchronises the stream, and returns FGX_OK or the recorded device error
 * (FGX_ERR_TIMEOUT).  Returns FGX_ERR_CUDA if the copy fails. */
int fgx_workspace_status(const void* workspace, void* stream);

/* Failure detection check: launches one block that waits, with the bounded
 * wait every inter-block hand-over of the library uses, on a tag in the
 * workspace that nothing writes.  After timeout_ms (1..10000) the wait gives
 * up and records FGX_ERR_TIMEOUT in the workspace status word, which
 * fgx_workspace_status then returns; the context stays usable.  The
 * workspace needs 264 bytes; the call clears them first. */
int fgx_probe_wait_timeout(void* workspace, size_t workspace_bytes, int timeout_ms,
                           void* stream);

/* ---------------------------------------------------------- autotune ---- */

/* Times each of the n candidate option sets on the caller's buffers (the
 * forward of fgx_geodesic2d, ndim = 2, D = 1, spacing NULL, or of
 * fgx_geodesic3d) and writes the index of the fastest to *best_index and its
 * mean time in milliseconds to *best_ms (host memory).  Each candidate runs
 * once untimed and then `reps` times between CUDA events on `stream`; the
 * call synchronises the stream (it is a setup step, not for a captured graph).
 * The workspace must hold every candidate's (the largest
 * fgx_geodesic_workspace_size over them).  A candidate the call does not
 * support (status FGX_ERR_UNSUPPORTED) is skipped; another error ends the
 * call with that status.  dist holds the last candidate's result. */
int fgx_autotune(int ndim, const float* image, const float* mask, float* dist, int64_t B,
                 int64_t C, int64_t D, int64_t H, int64_t W, const float spacing[3], float v,
                 float lambda, int iterations, void* workspace, size_t workspace_bytes,
                 const fgx_options* candidates, int n, int reps, int* best_index, float* best_ms,
                 void* stream);

/* ------------------------------------------------ derived transforms ---- */

/* Euclidean-only transform (lambda = 0): the cost of a step is its
 * spacing-weighted length sqrt(s2), no image is read (Summary section: the
 * generalised transform reduces to the Euclidean one when the image term has
 * no weight).  Same mask, dist, workspace and error behaviour as
 * fgx_geodesic2d / fgx_geodesic3d with C = 1 (the workspace size query takes
 * C = 1); results equal those calls with lambda = 0 and any image, bit for
 * bit. */
int fgx_euclidean2d(const float* mask, float* dist, int64_t B, int64_t H, int64_t W, float v,
                    int iterations, void* workspace, size_t workspace_bytes,
                    const fgx_options* opt, void* stream);
int fgx_euclidean3d(const float* mask, float* dist, int64_t B, int64_t D, int64_t H, int64_t W,
                    const float spacing[3], float v, int iterations, void* workspace,
                    size_t workspace_bytes, const fgx_options* opt, void* stream);

/* Scratch bytes of fgx_signed_geodesic2d / 3d: the workspace of a forward of
 * 2B instances plus 2B masks and 2B distance maps of D * H * W floats. */
int fgx_signed_workspace_size(int ndim, int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                              const fgx_options* opt, size_t* bytes);

/* Signed generalised geodesic distance (the paper names it among the
 * applications, without a definition; reading used here): with M the mask in
 * [0, 1], dist = GDT(M) - GDT(1 - M), each term the forward transform of the
 * same image (1 - M and the difference rounded to float32).  Negative inside
 * the region where M = 0, positive where M = 1; swapping M and 1 - M negates
 * the result exactly.  Arguments as fgx_geodesic2d / 3d; dist may alias mask
 * but not image.  Both transforms of every instance run as one launch of 2B
 * transforms of the same B images; a device wait timeout is reported by
 * fgx_workspace_status. */
int fgx_signed_geodesic2d(const float* image, const float* mask, float* dist, int64_t B,
                          int64_t C, int64_t H, int64_t W, float v, float lambda, int iterations,
                          void* workspace, size_t workspace_bytes, const fgx_options* opt,
                          void* stream);
int fgx_signed_geodesic3d(const float* image, const float* mask, float* dist, int64_t B,
                          int64_t C, int64_t D, int64_t H, int64_t W, const float spacing[3],
                          float v, float lambda, int iterations, void* workspace,
                          size_t workspace_bytes, const fgx_options* opt, void* stream);

/* Geodesic symmetric filtering of a segmentation (the paper names GSF among
 * the applications of the transform, without a definition; reading used
 * here, after the geodesic morphology of GeoS).  F in [0, 1] marks the
 * object (F = 1) against the background (F = 0); S(X) = GDT(1 - X) - GDT(X)
 * is the signed distance of the object of an indicator X (negative inside),
 * i.e. fgx_signed_geodesic of the mask 1 - X.  Then
 *   erosion   F_e = [S(F) < -theta_e],   dilation  F_d = [S(F) < theta_d],
 *   out       = [(S(F_e) + S(F_d)) + (theta_d - theta_e) < 0]
 * (1.0 / 0.0 floats; each sum and difference rounded to float32, the
 * thresholds' difference computed in float32 on the host).  Objects thinner
 * than the erosion vanish, holes narrower than the dilation close, and the
 * boundary of a large object stays where it was.  theta_d, theta_e >= 0,
 * finite.  The six transforms run as two launches over the same B images:
 * 2B transforms (1 - F and F), then 4B (1 - F_e, F_e, 1 - F_d, F_d).  Other
 * arguments and errors as fgx_geodesic2d / 3d; out [B][1][...] may alias
 * mask but not image. */
int fgx_gsf_workspace_size(int ndim, int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                           const fgx_options* opt, size_t* bytes);
int fgx_gsf2d(const float* image, const float* mask, float* out, int64_t B, int64_t C, int64_t H,
              int64_t W, float v, float lambda, int iterations, float theta_d, float theta_e,
              void* workspace, size_t workspace_bytes, const fgx_options* opt, void* stream);
int fgx_gsf3d(const float* image, const float* mask, float* out, int64_t B, int64_t C, int64_t D,
              int64_t H, int64_t W, const float spacing[3], float v, float lambda,
              int iterations, float theta_d, float theta_e, void* workspace,
              size_t workspace_bytes, const fgx_options* opt, void* stream);

/* ------------------------------------------------------------ batched ---- */

/* One instance of a batched call (B = 1 per instance).  Pointers are device
 * memory; shapes may differ between instances. */
typedef struct fgx_instance {
    int32_t ndim;        /* 2 or 3                                   */
    int32_t channels;    /* C >= 1                                    */
    int64_t D, H, W;     /* 2D: D = 1                                 */
    const float* image;  /* [C][D][H][W]                              */
    const float* mask;   /* [D][H][W]                                 */
    float* dist;         /* [D][H][W]                                 */
    float spacing[3];    /* (sD, sH, sW); 2D uses (1, 1, 1)           */
    float v, lambda;
    int32_t iterations;
} fgx_instance;

/* Plan of a batched launch, filled by fgx_batched_prepare.  Plain data: the
 * caller keeps it and may replay fgx_batched_run with it as often as it likes
 * (for example inside a captured CUDA graph) while the workspace and the
 * instances' buffers stay valid. */
typedef struct fgx_batched_plan {
    uint32_t size;          /* sizeof(fgx_batched_plan)                      */
    int32_t n;              /* instances on the tiled engine (3D, and 2D with 0 iterations) */
    int32_t grid;           /* thread blocks of that persistent launch       */
    int32_t smem_bytes;     /* dynamic shared memory per block               */
    int32_t rounds;         /* pass-application rounds                       */
    int32_t region, kmax;   /* tile buffer geometry                          */
    int32_t timeout_ms;
    uint64_t clear_bytes;   /* workspace prefix cleared before every run     */
    uint64_t desc_off, waves_off, items_off;  /* table offsets in workspace  */
    void* workspace;
    uint64_t workspace_bytes;
    /* 2D instances with at least one iteration: the line-chain launch      */
    int32_t n2d, grid2d, rounds2d;
    int32_t channels2d;     /* common channel count of the 2D instances (0: mixed) */
    int32_t max_wp2d, max_hp2d;  /* largest padded extents (table init grid) */
    uint64_t desc2d_off, waves2d_off, items2d_off;
    /* 3D instances the plane-tile kernel takes: the plane-tile launch        */
    int32_t n3d, grid3d, rounds3d, smem3d;
    uint64_t desc3d_off, waves3d_off, items3d_off;
    int32_t tables3d;       /* 1: some 3D instance reads cost tables (staging ring of single planes) */
    int32_t concurrent;     /* 1: the line-chain and plane-tile launches run at the same
                             * time on disjoint SM shares (grid2d + grid3d <= SMs) */
} fgx_batched_plan;

/* Workspace bytes for a batched launch of these instances. */
int fgx_batched_workspace_size(const fgx_instance* items, int n, const fgx_options* opt,
                               size_t* bytes);

/* Checks the instances, builds the work list of (instance, pass, line tile)
 * items - instances advance one pass application per round; each round packs
 * whole instances into waves of co-resident thread blocks - and uploads it
 * with the instance descriptors into `workspace` (a copy from host memory on
 * `stream`; `items` may be freed on return).  Writes `plan`. */
int fgx_batched_prepare(const fgx_instance* items, int n, void* workspace,
                        size_t workspace_bytes, const fgx_options* opt,
                        fgx_batched_plan* plan, void* stream);

/* Runs a prepared plan: clears the plan's progress tags and launches the
 * persistent kernels that compute every instance (line chain, plane tiles,
 * tiled engine: those the plan holds).  With plan->concurrent the line-chain
 * launch runs on a stream of the library's own, created with two events per
 * host thread and device on first use (fgx_batched_prepare creates them for
 * its thread) and kept until the thread exits; it waits for the caller's
 * stream and the caller's stream waits for it, so the call stays ordered on
 * `stream` as a whole.  Allocates nothing and copies nothing from the host,
 * so it can be captured in a CUDA graph (the fork and join become graph
 * edges). */
int fgx_batched_run(const fgx_batched_plan* plan, void* stream);

/* fgx_batched_prepare followed by fgx_batched_run.  Results equal n separate
 * fgx_geodesic2d / fgx_geodesic3d calls bit for bit. */
int fgx_geodesic_batched(const fgx_instance* items, int n, void* workspace,
                         size_t workspace_bytes, const fgx_options* opt, void* stream);

/* Batch autotuner (no counterpart in the paper, which runs one instance at a
 * time): prepares and runs the batch once per candidate option set, times
 * `reps` further runs of each between CUDA events on `stream`, and writes the
 * index of the fastest to *best_index and its mean time in ms to *best_ms.
 * The 2D instances take the candidates' line-tile geometry; the 3D instances
 * keep the plane tiles unless a candidate sets tile_height.  `workspace`
 * must hold the largest fgx_batched_workspace_size of the candidates it is
 * to try: a candidate whose plan does not fit it, or that the kernels cannot
 * run (FGX_ERR_UNSUPPORTED), is skipped.  The instances' outputs hold the
 * last candidate's results (all candidates give the same results).  Returns
 * FGX_ERR_UNSUPPORTED when no candidate ran. */
int fgx_batched_autotune(const fgx_instance* items, int n, void* workspace,
                         size_t workspace_bytes, const fgx_options* candidates, int ncand,
                         int reps, int* best_index, float* best_ms, void* stream);

/* ----------------------------------------------------- differentiable ---- */

/* Bytes of the `saved` buffer written by the training forward and read by
 * the backward: one parent code byte per element per pass application,
 * layout [iterations * passes][B][D*H*W] (code 0 = kept its value, k + 1 =
 * offset k of the pass stencil, offsets numbered row-major over the in-line
 * axes taken in (D, H, W) order). */
int fgx_train_saved_size(int ndim, int64_t B, int64_t D, int64_t H, int64_t W, int iterations,
                         size_t* bytes);

/* Forward that also records the parent codes into `saved`.  Same arguments
 * as fgx_geodesic2d / fgx_geodesic3d plus the saved buffer. */
int fgx_geodesic2d_fwd_train(const float* image, const float* mask, float* dist, int64_t B,
                             int64_t C, int64_t H, int64_t W, float v, float lambda,
                             int iterations, void* saved, size_t saved_bytes, void* workspace,
                             size_t workspace_bytes, const fgx_options* opt, void* stream);
int fgx_geodesic3d_fwd_train(const float* image, const float* mask, float* dist, int64_t B,
                             int64_t C, int64_t D, int64_t H, int64_t W,
                             const float spacing[3], float v, float lambda, int iterations,
                             void* saved, size_t saved_bytes, void* workspace,
                             size_t workspace_bytes, const fgx_options* opt, void* stream);

/* Scratch bytes for the backward of `iterations` iterations: status, the
 * adjoint buffers, and (2D) the codes in the line layout of each pass
 * application and the adjoint of every pass application for the image
 * gradient.  The 3D reverse sweep adds each application's image-gradient
 * terms right after sweeping it, so its scratch does not grow with the
 * iterations (two adjoint buffers and the adjoint of one application). */
int fgx_backward_workspace_size(int ndim, int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                                int iterations, const fgx_options* opt, size_t* bytes);

/* Reverse sweep through the recorded codes: pass applications in reverse,
 * lines in reverse sweep order; each element with a parent pushes its
 * adjoint into the parent and adds lambda*(I(x)-I(p))/c times it to the
 * image gradient (0 where c = 0); dL/dM = v * G at the end.  grad_image
 * [B][C][...] and grad_mask [B][1][...] may each be NULL.  Results are
 * bit-exact to the sequential float32 order: a parent gathers its children in
 * offset order, and an element's image gradient receives its parent-side
 * terms before its own child-side term in each pass. */
int fgx_geodesic2d_bwd(const float* grad_dist, const float* image, const void* saved,
                       size_t saved_bytes, float* grad_image, float* grad_mask, int64_t B,
                       int64_t C, int64_t H, int64_t W, float v, float lambda, int iterations,
                       void* workspace, size_t workspace_bytes, const fgx_options* opt,
                       void* stream);
int fgx_geodesic3d_bwd(const float* grad_dist, const float* image, const void* saved,
                       size_t saved_bytes, float* grad_image, float* grad_mask, int64_t B,
                       int64_t C, int64_t D, int64_t H, int64_t W, const float spacing[3],
                       float v, float lambda, int iterations, void* workspace,
                       size_t workspace_bytes, const fgx_options* opt, void* stream);

/* ---------------------------------------------- checkpointed 3D training ----
 *
 * Training with less memory kept between the forward and the backward
 * (Summary and Statement of need: the transform as a differentiable layer on
 * 3D volumes).  Instead of one parent code byte per voxel and pass
 * application, the forward keeps the distance map at the start of every
 * `interval`-th iteration (iterations interval, 2*interval, ...; the
 * starting map v*M is rebuilt from the mask).  The backward replays each
 * segment of `interval` iterations once from its checkpoint, recording that
 * segment's codes in the workspace, and sweeps the segment's pass
 * applications in reverse; gradients equal fgx_geodesic3d_bwd's bit for
 * bit.  The kept buffer shrinks from 6 bytes per voxel and iteration to
 * 4 / interval bytes per voxel and iteration (0 with interval >= iterations);
 * the backward does one more forward's arithmetic and holds one segment's
 * codes (6 * interval bytes per voxel) in its workspace.  Only the 3D
 * plane-tile kernels take this path (at most 3 channels where the image is
 * read, no tile-shape options): otherwise FGX_ERR_UNSUPPORTED. */

/* Bytes of the buffer kept between fgx_geodesic3d_fwd_checkpoint and
 * fgx_geodesic3d_bwd_checkpoint: (ceil(iterations / interval) - 1) float
 * maps of B*D*H*W, layout [checkpoint][B][D][H][W].  interval >= 1. */
int fgx_checkpoint_saved_size(int64_t B, int64_t D, int64_t H, int64_t W, int iterations,
                              int interval, size_t* bytes);

/* Scratch bytes of both checkpointed calls (status word at offset 0, read by
 * fgx_workspace_status after either call). */
int fgx_checkpoint_workspace_size(int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                                  int iterations, int interval, const fgx_options* opt,
                                  size_t* bytes);

/* Forward of fgx_geodesic3d (same arguments and result) that also writes the
 * checkpoints into `saved` (device memory, fgx_checkpoint_saved_size
 * bytes; nullable when that is 0). */
int fgx_geodesic3d_fwd_checkpoint(const float* image, const float* mask, float* dist, int64_t B,
                                  int64_t C, int64_t D, int64_t H, int64_t W,
                                  const float spacing[3], float v, float lambda, int iterations,
                                  int interval, void* saved, size_t saved_bytes, void* workspace,
                                  size_t workspace_bytes, const fgx_options* opt, void* stream);

/* Backward of fgx_geodesic3d_bwd through the checkpoints of
 * fgx_geodesic3d_fwd_checkpoint (same image, mask, v, lambda, spacing,
 * iterations and interval).  grad_image and grad_mask as in
 * fgx_geodesic3d_bwd (at least one non-NULL). */
int fgx_geodesic3d_bwd_checkpoint(const float* grad_dist, const float* image, const float* mask,
                                  const void* saved, size_t saved_bytes, float* grad_image,
                                  float* grad_mask, int64_t B, int64_t C, int64_t D, int64_t H,
                                  int64_t W, const float spacing[3], float v, float lambda,
                                  int iterations, int interval, void* workspace,
                                  size_t workspace_bytes, const fgx_options* opt, void* stream);

/* Scratch bytes of fgx_geodesic_bwd_params: the reverse sweep's workspace
 * (fgx_backward_workspace_size) plus three arrays of B*D*H*W floats and 8 KB
 * of float64 partial sums. */
int fgx_params_workspace_size(int ndim, int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                              int iterations, const fgx_options* opt, size_t* bytes);

/* Gradients with respect to the scalar parameters lambda and v (extension
 * of the differentiable transform), through the codes of
 * fgx_geodesic*_fwd_train.  Since D = D(y) + c for an element whose value
 * came from parent y and c^2 = (1 - lambda) s2 + lambda di2 (s2 the
 * spacing-weighted squared offset, di2 the squared intensity difference),
 * dL/dlambda = sum over pass applications and such elements of
 * A(x) (di2 - s2) / (2c) (0 where c = 0), A the element's adjoint; and since
 * D0 = v M, dL/dv = sum of M(x) G0(x), G0 the adjoint of D0.  lambda_terms
 * and v_terms ([B][D][H][W] float32, nullable) receive the per-element terms
 * (over the applications in reverse order, in float32 with the fixed
 * operation order of the method); grad_lambda and grad_v (device memory, one
 * double each, nullable) receive their sums over the call in float64, by a
 * fixed-shape tree (the same bits on every run).  grad_image and grad_mask
 * (nullable) are the outputs of fgx_geodesic*_bwd.  mask is the forward's
 * mask.  2D: ndim = 2, D = 1, spacing NULL.  Only the warp-chain (2D) and
 * plane-tile (3D) reverse sweeps carry the terms: 3D tile-shape options give
 * FGX_ERR_UNSUPPORTED. */
int fgx_geodesic_bwd_params(int ndim, const float* grad_dist, const float* image,
                            const float* mask, const void* saved, size_t saved_bytes,
                            float* grad_image, float* grad_mask, float* lambda_terms,
                            float* v_terms, double* grad_lambda, double* grad_v, int64_t B,
                            int64_t C, int64_t D, int64_t H, int64_t W, const float spacing[3],
                            float v, float lambda, int iterations, void* workspace,
                            size_t workspace_bytes, const fgx_options* opt, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FGX_H */
