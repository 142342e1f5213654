/*
 * rgx.h -- C ABI of librgx: differentiable volume ray marching through
 * truncated elliptical Gaussians on one NVIDIA B300 (sm_103a).
 *
 * Method: RayGaussX (arXiv 2509.07782).  The density and radiance fields are
 * sums of Gaussians (Eq. 1); a ray is integrated front to back in segments of
 * N_S samples (Eq. 3, Algorithm 1) with empty-space skipping through a BVH
 * ClosestHit query (Algorithm 1, Eq. 4), a distance- and transmittance-
 * adaptive segment size (Eq. 5), early termination at T <= T_eps, Gaussians
 * stored in Z-order (Sec. 3.3) and rays grouped in 2D tiles (Sec. 3.3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Array arguments are DEVICE pointers owned by the caller: contiguous,
 *    float32 unless stated, on the scene's device, and at least as long as
 *    stated (a plain pointer cannot be checked here: a host pointer or a
 *    short buffer is an out-of-bounds access on the device).  Camera arrays
 *    are HOST pointers, copied with a stream-ordered cudaMemcpyAsync: a
 *    pinned array is read when the stream reaches the copy, so it must stay
 *    alive and unchanged until then (a pageable one is staged during the call).
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  Every call only enqueues work on it and returns; no
 *    call synchronises except rgx_sync_status.
 *  - Every call returns an rgx_status.  No C++ exception crosses the ABI.
 *    rgx_last_error() gives a static description of the last failure.
 *  - Problems found on the device (segment limit reached, traversal stack
 *    overflow, bad parameters such as s <= 0 or NaN) are OR-ed into a device
 *    status word held by the scene; rgx_sync_status() synchronises the stream
 *    and returns (and clears) it.  Kernels never trap and never spin without
 *    a bound.
 *  - A scene owns its workspace (BVH, Z-order permutation, packed
 *    parameters, gradient accumulators, the adjoint's chunk scratch of
 *    196 KB per resident warp).  It grows on demand inside
 *    rgx_build_bvh / rgx_render_*; once a scene has seen the largest sizes it
 *    will be used with, later calls allocate nothing and can be captured in a
 *    CUDA graph.
 *  - Calls on one scene must not overlap in time (one stream per scene).
 */
#ifndef RGX_H
#define RGX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t rgx_status;
#define RGX_OK                  0
#define RGX_ERR_INVALID_ARG     1   /* bad pointer, size or option (host check) */
#define RGX_ERR_CUDA            2   /* a CUDA runtime call failed */
#define RGX_ERR_WORKSPACE       3   /* device allocation failed */
#define RGX_ERR_HIT_OVERFLOW    4   /* reserved: hit lists are chunked, never dropped */
#define RGX_ERR_STACK_OVERFLOW  8   /* device: BVH deeper than the traversal stack */
#define RGX_ERR_ITER_LIMIT      16  /* device: a ray reached max_segments (or the 2^20 default ceiling) */
#define RGX_ERR_BAD_PARAMS      32  /* device: NaN/Inf parameter, scale <= 0, |q| = 0 */
#define RGX_ERR_REPLAY          64  /* device: backward replay did not reproduce T_final */
#define RGX_ERR_NOT_BUILT       128 /* render called before rgx_build_bvh */

/* option flags (rgx_opts.flags) */
#define RGX_SKIP      1    /* empty-space skipping: Algorithm 1 ClosestHit, Eq. 4 */
#define RGX_ADAPTIVE  2    /* Eq. 5 segment size instead of uniform dt */
#define RGX_MORTON    4    /* store packed parameters in Z-order (Sec. 3.3) */
#define RGX_ZTILES    8    /* 2D ray tiles in Z-order instead of scanline warps (Sec. 3.3) */
#define RGX_MORTON63  16   /* 63-bit (21 bits/axis) instead of 30-bit Morton codes */
#define RGX_LOWER_FIRST 32 /* scheduling only (with RGX_SKIP): a ray's first chord window, tried over the whole
                              ray, has its end lowered while its chords overflow hit_cap instead of giving up;
                              rgx_autotune tries both, and hit_cap = 0 applies its choice */

typedef struct rgx_scene rgx_scene;   /* opaque */

/* Pinhole camera, OpenCV convention (+z forward, +y down).  Pixel (u, v)
 * looks along c2w[:, :3] ((u+0.5-cx)/fx, (v+0.5-cy)/fy, 1), normalised; the
 * ray starts at the camera centre c2w[:, 3].  t_far <= 0 means "exit of the
 * scene bounding box" (the union of all ellipsoid AABBs). */
typedef struct {
    float c2w[12];               /* row-major 3x4 camera-to-world */
    float fx, fy, cx, cy;        /* intrinsics in pixels */
    int32_t width, height;
    float t_near, t_far;         /* integration bounds t_n, t_f of Algorithm 1 */
} rgx_camera;

/* Marching options: the inputs of Algorithm 1 and Eq. 5. */
typedef struct {
    int32_t flags;               /* RGX_SKIP | RGX_ADAPTIVE | RGX_MORTON | RGX_ZTILES | RGX_MORTON63 | RGX_LOWER_FIRST */
    float dt;                    /* uniform step (Eq. 3) */
    float dt_min, dt_max, beta;  /* Eq. 5 parameters */
    int32_t n_s;                 /* samples per segment N_S: 4, 8, 16 or 32; 0 = the scene's last
                                    rgx_autotune pick, else 16.  N_S is part of the method in adaptive
                                    mode (Eq. 5 scales with it), so 0 may change results after tuning */
    float t_eps;                 /* transmittance threshold T_eps (Algorithm 1) */
    float sigma_eps;             /* truncation density: support is sigma(x) >= sigma_eps */
    float bg[3];                 /* background colour, added as T_final * bg */
    int32_t tile_w, tile_h;      /* ray tile, tile_w * tile_h == 32 (ZTILES only); both 0 = the scene's
                                    last rgx_autotune pick, else 32 x 1 */
    int32_t hit_cap;             /* chord-list capacity per ray (multiple of 32, 32..1024; never drops hits);
                                    0 = the scene's last rgx_autotune pick, else 512 */
    int32_t max_segments;        /* loop bound per ray, >= 0; 0 = derived from the ray length: (t_f - t_n) / dt
                                    (uniform) or / (N_S dt_min) (Eq. 5), plus 8, but at most 2^20
                                    (1,048,576) segments.  A ray stopped by either bound sets
                                    RGX_ERR_ITER_LIMIT and keeps what it has composited so far */
} rgx_opts;
/* Tile shape, hit_cap and (in uniform mode) N_S change scheduling only: results agree to float32
 * rounding for any choice.  Zeros are resolved on the host at each call, so a forward and its
 * adjoint resolve them alike as long as no rgx_autotune runs on the scene in between. */

/* Create / destroy a scene handle bound to CUDA device `device`. */
rgx_status rgx_scene_create(rgx_scene** out, int32_t device);
rgx_status rgx_scene_destroy(rgx_scene* scene);

/*
 * Build the acceleration structure and packed parameters for n Gaussians.
 * Sec. 3.2 (the BVH is rebuilt at every optimisation step) and Sec.
 * 3.3 (Z-order re-indexing); ellipsoid AABB from Supp. Sec. 2.2.
 *
 *   means      [n,3]            Gaussian means mu
 *   scales     [n,3]            linear scales s > 0 (Sigma = R S S^T R^T)
 *   quats      [n,4]            rotations as (w,x,y,z); normalised here
 *   densities  [n]              sigma~ (peak density); sigma~ <= sigma_eps
 *                               gives an empty support
 *   sh         [n,(deg+1)^2,3]  SH coefficients, channel fastest
 *   sh_degree  0..3
 *
 * Steps (all on `stream`): scene bounds of the means, 30/63-bit Morton codes,
 * LSD radix sort of (code, index), Karras radix tree, bottom-up AABB refit,
 * 4-wide half-precision traversal records, and packing of the parameters into
 * float4 records (in Z-order with RGX_MORTON, else in caller order).  The arrays are read during this call
 * only; the scene keeps its own packed copy.  n may be 0.
 */
rgx_status rgx_build_bvh(rgx_scene* scene, int64_t n, int32_t sh_degree,
                         const float* means, const float* scales, const float* quats,
                         const float* densities, const float* sh,
                         const rgx_opts* opts, void* stream);

/*
 * rgx_build_bvh for Gaussians whose colour also has spherical-Gaussian lobes:
 * the SH + SG appearance of Eq. 1 ("parameterized with SH/SG", Sec. 3.1), as in
 * the supplementary's comparison (Supp. Sec. 6.1: nine SH and seven SG per
 * primitive, i.e. sh_degree 2 and n_sg 7).  The colour becomes
 *     c_l(d) = max(0, 1/2 + sum_k Y_k(d) K_lk + sum_j a_lj exp(lambda_lj (mu_lj . d - 1)))
 *   sg   [n, n_sg, 7]  per lobe (u_x, u_y, u_z, lambda, a_r, a_g, a_b): a raw axis u
 *                      (normalised here: mu = u / |u|, |u| > 0), a sharpness
 *                      lambda >= 0 and an RGB amplitude; bad values are flagged
 *                      RGX_ERR_BAD_PARAMS and the lobe is dropped
 *   n_sg 0..7
 * The lobes are packed in the scene (32 B per lobe per Gaussian); their gradients
 * come from rgx_render_backward_ex.
 */
rgx_status rgx_build_bvh_sg(rgx_scene* scene, int64_t n, int32_t sh_degree,
                            const float* means, const float* scales, const float* quats,
                            const float* densities, const float* sh, int32_t n_sg, const float* sg,
                            const rgx_opts* opts, void* stream);

/*
 * Forward render of ncam cameras in one persistent launch (Algorithm 1 for
 * every pixel; Eq. 1 densities and SH colours; Eq. 3 compositing).
 *
 *   cams       HOST [ncam]  cameras (copied on `stream`)
 *   rgba       [R,4]        output, R = sum_c width_c*height_c, camera-major,
 *                           row-major pixels: (C + T bg, 1 - T)
 *   fwd_state  [R] x rgx_fwd_state_bytes()  per-ray record kept for the adjoint
 *                           (may be NULL for inference); opaque: (C, T), the
 *                           collection path the ray took, and where the scene's
 *                           tape holds its first chord list.  The tape (scene
 *                           workspace, hit_cap / 6 entries of 48 B per ray) keeps the
 *                           lists of the LAST forward call only; an adjoint given
 *                           the state of an older call collects them again.  With a
 *                           state the forward also records, for up to 32 segments per
 *                           ray whose chords overflow hit_cap, the segment's per-sample
 *                           sums ((N_S + 1) x 16 B, within 16 GB) and its chords in the
 *                           order met, each as its packed index and the colour it
 *                           evaluated (16 B, up to 2,048 per ray, within 48 GB); the
 *                           adjoint reads them instead of traversing and colouring
 *                           again.  Workspace that cannot be allocated is simply not
 *                           used (same results, more work)
 */
rgx_status rgx_render_forward(rgx_scene* scene, const rgx_camera* cams, int32_t ncam,
                              const rgx_opts* opts, float* rgba, void* fwd_state, void* stream);

/*
 * Same as rgx_render_forward, and also records each ray's evaluated segments
 * (t_S, dt) -- the schedule -- into sched [R, sched_cap, 2] with the count per
 * ray in sched_n [R] (int32; counts beyond sched_cap are still counted).
 * Used to check discrete decisions against a reference.
 */
rgx_status rgx_render_forward_sched(rgx_scene* scene, const rgx_camera* cams, int32_t ncam,
                                    const rgx_opts* opts, float* rgba, void* fwd_state,
                                    float* sched, int32_t sched_cap, int32_t* sched_n, void* stream);

/*
 * Adjoint of rgx_render_forward: replays each ray's march front to back
 * (recomputing, not storing, per-sample densities) and ACCUMULATES (+=)
 * dL/d{means, scales, quats, densities, sh} in the caller's order for the
 * upstream gradient d_rgba [R,4].  Gradients are for the raw inputs of
 * rgx_build_bvh (linear scales, unnormalised quaternions).  The truncation
 * boundary, the schedule and termination are held fixed (piecewise
 * constant).  Rays whose d_rgba row is zero contribute nothing and are
 * skipped.  Must follow rgx_render_forward with the same cameras and options
 * on a scene not rebuilt in between, and be given the fwd_state that forward
 * wrote.  With the state of the scene's last forward call the first chord
 * lists come from the tape; with an older state they are collected again
 * (same result, more work).  Segments whose chords overflow hit_cap are kept
 * in the scene's per-warp scratch between the two adjoint passes; if that
 * scratch cannot be allocated they are traversed twice instead.
 */
rgx_status rgx_render_backward(rgx_scene* scene, const rgx_camera* cams, int32_t ncam,
                               const rgx_opts* opts, const void* fwd_state, const float* d_rgba,
                               float* d_means, float* d_scales, float* d_quats,
                               float* d_densities, float* d_sh, void* stream);

/*
 * rgx_render_backward with its optional outputs (any of them may be NULL):
 *   d_sg   [n, n_sg, 7]  += gradients of the spherical-Gaussian lobes of a scene
 *                        built by rgx_build_bvh_sg (required when it has lobes):
 *                        (raw axis u, sharpness, RGB amplitude), caller order
 *   stat   [n] float32   the densification statistic of Sec. 3.5, Eq. 11, for
 *   count  [n] int32     every camera of the batch (Supp. Sec. 3 relates it to
 *                        the projected mean gradient); both or neither.  With
 *                        L_c = sum over camera c's pixels of <d_rgba, rgba> and
 *                        g_c = dL_c/dmu_l, every Gaussian l with g_c != 0 gets
 *                          stat[l]  += |mu_l - o_c| / f_c * |g_c|
 *                          count[l] += 1
 *                        with o_c the camera centre and f_c its focal length fx
 *                        in pixels (> 0): each camera's own gradient, not the
 *                        gradient of the summed loss.  Densify where stat / count
 *                        > tau (tau = 1.5e-4 in Sec. 4.2).  Per (ray, segment,
 *                        Gaussian) hit the adjoint adds the hit's first moment to
 *                        a per-(Gaussian, camera) slice of scene workspace (16 B x
 *                        n x ncam), finalised by one kernel.
 * The five parameter gradients are those of rgx_render_backward.
 */
rgx_status rgx_render_backward_ex(rgx_scene* scene, const rgx_camera* cams, int32_t ncam, const rgx_opts* opts,
                                  const void* fwd_state, const float* d_rgba, float* d_means, float* d_scales,
                                  float* d_quats, float* d_densities, float* d_sh, float* d_sg, float* stat,
                                  int32_t* count, void* stream);

/* rgx_autotune modes (may be OR-ed) */
#define RGX_TUNE_NS          1   /* also tune N_S over {4, 8, 16, 32} */
#define RGX_TUNE_EXHAUSTIVE  2   /* time the full grid instead of one knob at a time */

/*
 * Autotuner for the open knobs of Algorithm 1 -- samples per segment N_S, the
 * capacity of the hit-primitive buffer H_b (hit_cap) -- and of the 2D ray
 * tiles of Sec. 3.3 (tile_w x tile_h, when RGX_ZTILES is set), timed on the
 * caller's scene and cameras.  Candidates: 4 tile shapes (8x4, 4x8, 16x2,
 * 32x1), hit_cap in {32,64,96,128,192,256,384,512,640,768}, and with RGX_TUNE_NS N_S in
 * {4,8,16,32} (else base->n_s).  By default the knobs are tuned one at a time
 * (tile shape at the base hit_cap, then hit_cap, the other tile shapes again if
 * hit_cap moved, then N_S, then RGX_LOWER_FIRST toggled: at most 4+6+3+3+1
 * candidates); RGX_TUNE_EXHAUSTIVE times every combination.  Each candidate runs
 * once to warm up and twice timed with CUDA events on `stream`, forward only or
 * forward + adjoint (with_backward != 0).  Knobs left at 0 in *base start from
 * the defaults.  The fastest options are written to *best (other fields copied
 * from *base), its time in ms to *best_ms (may be NULL), and kept on the scene:
 * later calls that leave hit_cap, the tile shape or n_s at 0 use them.
 * Synchronises the stream.  rgba, fwd_state, d_rgba and the five gradient
 * arrays are caller-owned scratch buffers laid out as for rgx_render_forward /
 * rgx_render_backward; their contents are undefined afterwards.  N_S changes
 * results in adaptive mode (Eq. 5 scales with N_S); without RGX_TUNE_NS results
 * stay fixed.
 */
rgx_status rgx_autotune(rgx_scene* scene, const rgx_camera* cams, int32_t ncam, const rgx_opts* base,
                        int32_t mode, int32_t with_backward, float* rgba, void* fwd_state,
                        const float* d_rgba, float* d_means, float* d_scales, float* d_quats,
                        float* d_densities, float* d_sh, rgx_opts* best, float* best_ms, void* stream);

/*
 * Isotropic loss, Sec. 3.4 Eqs. 6-8: L_s = 1/n sum_l max(r_max,l - r0, 0) with
 * r_max = 2/(pi sqrt 3) (s1^2+s2^2+s3^2)^(3/2) / (s1 s2 s3), the rotation-free
 * bound of a Gaussian's AABB/ellipsoid volume ratio (Supp. Sec. 2.3).
 * Enqueues on `stream`: *loss += weight * L_s (one device float) and
 * d_scales[n,3] += weight * dL_s/ds (linear scales, s > 0).  The paper uses
 * r0 = 10 and weight lambda_s = 2.5e-4 (Sec. 4.2).
 */
rgx_status rgx_isotropic_loss(int64_t n, const float* scales, float r0, float weight, float* loss,
                              float* d_scales, void* stream);

/*
 * Densification statistic, Sec. 3.5 Eq. 11, for one view: for every Gaussian
 * whose mean gradient d_means[l] (from rgx_render_backward of this single
 * view) is non-zero, stat[l] += |means[l] - o| / f * |d_means[l]| and
 * count[l] += 1 (int32), with o the camera centre and f its focal length fx
 * in pixels (HOST cam).  Densify where stat / count > tau (tau = 1.5e-4 in
 * Sec. 4.2).  Enqueues on `stream`.
 */
rgx_status rgx_densify_accumulate(int64_t n, const float* means, const float* d_means,
                                  const rgx_camera* cam, float* stat, int32_t* count, void* stream);

/*
 * Cap the forward's tape (the finished first chord lists the adjoint reads back
 * instead of traversing again; 48 B per entry, by default hit_cap / 6 entries per
 * ray, e.g. 29 GB for 7.1 M rays at hit_cap 512) at max_entries entries; 0
 * disables the tape and the records of overflowing segments, a negative value
 * restores the default sizing.  Results do not depend on it: rays whose lists
 * find no room are collected again by the adjoint.  Takes effect at the next
 * rgx_render_forward with a state.
 */
rgx_status rgx_set_tape_limit(rgx_scene* scene, int64_t max_entries);

/*
 * Image loss of one training step, Sec. 3.4: per camera c of a batch,
 *     L_c = (1 - lambda) L1 + lambda DSSIM,   DSSIM = 1 - SSIM
 * on the composited RGB of rgba (opacity is not part of the loss), with SSIM over
 * an 11 x 11 Gaussian window (standard deviation 1.5, C1 = 0.01^2, C2 = 0.03^2, zero
 * padding at the image border) and both terms averaged over the view's pixels and
 * channels.  (The paper leaves these constants to the methods it builds on; lambda
 * = 0.2 is the usual choice.)
 *   cams    HOST [ncam]  only width and height are read
 *   rgba    [R,4]        rendered pixels, camera-major, row-major
 *   target  [R,3]        target RGB
 *   loss    [ncam]       device floats, loss[c] += L_c
 *   d_rgba  [R,4]        written (=): dL/d rgba with L = sum_c L_c (opacity column 0),
 *                        ready for rgx_render_backward
 * Scratch (96 B per pixel) is scene workspace; the first call on a scene uploads the
 * window taps (make it before any stream capture).
 */
rgx_status rgx_image_loss(rgx_scene* scene, const rgx_camera* cams, int32_t ncam, const float* rgba,
                          const float* target, float lambda, float* loss, float* d_rgba, void* stream);

/*
 * One Adam step (Kingma & Ba 2015) on a parameter tensor of n floats:
 *   g = grad (or grad * exp(param) with exp_param != 0: the optimiser's variable is
 *       the log of the value the renderer takes, e.g. log-scales and log-densities,
 *       and grad is the gradient with respect to that value)
 *   m = beta1 m + (1 - beta1) g;  v = beta2 v + (1 - beta2) g^2
 *   param -= lr (m / (1 - beta1^step)) / (sqrt(v / (1 - beta2^step)) + eps)
 * and, if activated != NULL, activated = exp(param) (or param): the values the next
 * rgx_build_bvh takes.  step >= 1.  param, m, v are updated in place.
 */
rgx_status rgx_adam_step(int64_t n, float* param, const float* grad, float* m, float* v, float lr, float beta1,
                         float beta2, float eps, int32_t step, int32_t exp_param, float* activated,
                         void* stream);

/*
 * Adaptive density control driven by the criterion of Sec. 3.5, Eq. 11 (the
 * statistic of rgx_render_backward_ex): a Gaussian l with count[l] > 0 and
 * stat[l] / count[l] > tau (Sec. 4.2: tau = 1.5e-4) is cloned when its largest
 * scale is at most size_threshold, else split.  (The paper keeps the clone/split
 * rule of the methods it builds on; the reading taken is that rule.)
 *   action [n] int32  written: 0 keep, 1 clone, 2 split
 *   offset [n] int32  written: first output slot of Gaussian l (exclusive scan of
 *                     1 / 2 / 2 outputs)
 *   n_out  HOST       number of Gaussians after the step; the call synchronises the
 *                     stream to return it (allocate the outputs of rgx_densify_apply)
 */
rgx_status rgx_densify_plan(rgx_scene* scene, int64_t n, const float* stat, const int32_t* count,
                            const float* scales, float tau, float size_threshold, int32_t* action, int32_t* offset,
                            int64_t* n_out, void* stream);

/*
 * Apply a densification plan: every Gaussian l writes its outputs at offset[l]:
 * kept -- itself; cloned -- itself and an identical copy; split -- two children
 * with means mu + R(q) (s * z_k), z_k = normals[l, k, :] (standard normal draws
 * supplied by the caller, [n, 2, 3]), scales s / 1.6, rotation, density, SH and
 * lobes unchanged.  sh_floats / sg_floats: floats per Gaussian of sh and sg (0 for
 * none).  out_src [n_out] (may be NULL) receives each output's source index.
 */
rgx_status rgx_densify_apply(int64_t n, const int32_t* action, const int32_t* offset, const float* normals,
                             const float* means, const float* scales, const float* quats, const float* densities,
                             const float* sh, int32_t sh_floats, const float* sg, int32_t sg_floats,
                             float* out_means, float* out_scales, float* out_quats, float* out_densities,
                             float* out_sh, float* out_sg, int32_t* out_src, void* stream);

/* Synchronise `stream`, return the device status word (RGX_ERR_* bits, 0 if
 * clean) and clear it. */
rgx_status rgx_sync_status(rgx_scene* scene, void* stream);

/* Bytes of per-ray state written by rgx_render_forward (32: C[3], T, the collection path, tape offset,
 * count and tag, and the first window's end -- or, for a ray without a whole-ray first window, its
 * ClosestHit(t_n) and whether it started in a dense stretch). */
size_t rgx_fwd_state_bytes(void);

/* Static description of the last error on this scene (or globally if NULL). */
const char* rgx_last_error(const rgx_scene* scene);

/*
 * Introspection for tests (device output pointers, enqueued on `stream`):
 *   codes  [n]   sorted Morton codes (uint64)
 *   perm   [n]   sorted position -> caller index (int32)
 *   nodes  [max(n-1,1), 16] internal nodes: left lo/hi, right lo/hi boxes and
 *                (first, split, last) leaf ranges as int32 bit patterns at
 *                floats 3, 7, 11
 *   root   [6]   scene box (lo xyz, hi xyz)
 * Any pointer may be NULL.
 */
rgx_status rgx_get_bvh(rgx_scene* scene, uint64_t* codes, int32_t* perm, float* nodes,
                       float* root, void* stream);

/*
 * Work counters of the last forward or backward call (HOST output, 8 x
 * uint64; synchronises the stream): [0] rays, [1] evaluated segments,
 * [2] (ray, segment, Gaussian) hits, [3] (sample, Gaussian) evaluations,
 * [4] BVH node visits, [5] ClosestHit queries, [6] skipped segments,
 * [7] chord windows collected.
 */
rgx_status rgx_get_counters(rgx_scene* scene, uint64_t* out8, void* stream);

/*
 * Allocation-free Morton sort: the Z-order codes and permutation that
 * rgx_build_bvh computes (scene bounds of the means, 30-bit or, with
 * wide != 0, 63-bit codes, stable radix sort of (code, index)), written to
 * codes [n] (uint64, ascending) and perm [n] (int32, sorted position -> input
 * index).  The paper has no counterpart to this entry point; it exists for
 * callers that cannot call cudaMalloc: code that runs while a CUDA graph is
 * being captured, plugins living inside another engine whose allocator owns
 * all device memory, and real-time loops that must not allocate.  It
 * allocates nothing: its scratch is a fixed static device array of about
 * 6.3 MB that every GPU loading the library keeps until the process exits.
 *   - n must be at most 262144; larger n returns RGX_ERR_INVALID_ARG.
 *   - The first call on a device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 *   - Every call shares the one array: calls that overlap on the GPU (other
 *     streams, other threads) race and must be serialised by the caller.
 *   - means, codes and perm are device pointers on the current device;
 *     the work is enqueued on `stream`.
 *   - Means are not checked (unlike rgx_build_bvh, which flags them in the
 *     scene's status word): a NaN coordinate is left out of the bounds and
 *     quantised to cell 0, an infinite one makes the extent infinite so every
 *     code becomes 0; the call still returns RGX_OK.
 */
rgx_status rgx_morton_sort_noalloc(int64_t n, const float* means, int32_t wide, uint64_t* codes,
                                   int32_t* perm, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RGX_H */
