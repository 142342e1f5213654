// tune.cu -- autotuner for the march launch parameters (rgx_autotune).
//
// Algorithm 1 leaves three implementation knobs open: the number of samples
// per segment N_S, the capacity of the hit-primitive buffer H_b, and (Sec.
// 3.3, ray coherence) the shape of the 2D ray tiles.  The best
// values depend on the scene's depth complexity and on the cameras, so they
// are measured: every candidate configuration is run on the caller's actual
// scene and cameras and timed with CUDA events on the caller's stream.
#include <stdio.h>
#include "common.cuh"

extern "C" rgx_status rgx_render_forward(rgx_scene*, const rgx_camera*, int32_t, const rgx_opts*, float*, void*, void*);
extern "C" rgx_status rgx_render_backward(rgx_scene*, const rgx_camera*, int32_t, const rgx_opts*, const void*,
                                          const float*, float*, float*, float*, float*, float*, void*);
extern "C" rgx_status rgx_sync_status(rgx_scene*, void*);

static rgx_status run_once(rgx_scene* s, const rgx_camera* cams, int32_t ncam, const rgx_opts* o, int bwd,
                           float* rgba, void* state, const float* d_rgba, float* const g[5], void* st) {
    rgx_status r = rgx_render_forward(s, cams, ncam, o, rgba, state, st);
    if (r || !bwd) return r;
    return rgx_render_backward(s, cams, ncam, o, state, d_rgba, g[0], g[1], g[2], g[3], g[4], st);
}

extern "C" rgx_status rgx_autotune(rgx_scene* s, const rgx_camera* cams, int32_t ncam, const rgx_opts* base,
                                   int32_t tune_ns, int32_t with_backward, float* rgba, void* fwd_state,
                                   const float* d_rgba, float* d_means, float* d_scales, float* d_quats,
                                   float* d_dens, float* d_sh, rgx_opts* best, float* best_ms, void* stream) {
    if (!s || !base || !best || !rgba || !fwd_state) return set_err(s, RGX_ERR_INVALID_ARG, "rgx_autotune: null argument");
    if (with_backward && (!d_rgba || !d_means || !d_scales || !d_quats || !d_dens || !d_sh))
        return set_err(s, RGX_ERR_INVALID_ARG, "rgx_autotune: backward tuning needs d_rgba and gradient buffers");
    cudaStream_t st = (cudaStream_t)stream;
    float* const g[5] = {d_means, d_scales, d_quats, d_dens, d_sh};
    const int tiles[4][2] = {{8, 4}, {4, 8}, {16, 2}, {32, 1}};
    const int ntiles = (base->flags & RGX_ZTILES) ? 4 : 1;
    const int caps[7] = {128, 192, 256, 384, 512, 640, 768};
    const int nss[3] = {8, 16, 32};
    const int nns = tune_ns ? 3 : 1;
    cudaEvent_t e0, e1;
    RGX_CUDA(s, cudaEventCreate(&e0));
    RGX_CUDA(s, cudaEventCreate(&e1));
    float best_t = 1e30f;
    rgx_opts bo = *base;
    rgx_status r = RGX_OK;
    for (int ti = 0; ti < ntiles && !r; ti++)
        for (int ci = 0; ci < 7 && !r; ci++)
            for (int ni = 0; ni < nns && !r; ni++) {
                rgx_opts o = *base;
                if (ntiles > 1) { o.tile_w = tiles[ti][0]; o.tile_h = tiles[ti][1]; }
                o.hit_cap = caps[ci];
                if (tune_ns) o.n_s = nss[ni];
                r = run_once(s, cams, ncam, &o, with_backward, rgba, fwd_state, d_rgba, g, st);  // warm-up
                if (r) break;
                float tmin = 1e30f;
                for (int rep = 0; rep < 2 && !r; rep++) {
                    cudaEventRecord(e0, st);
                    r = run_once(s, cams, ncam, &o, with_backward, rgba, fwd_state, d_rgba, g, st);
                    cudaEventRecord(e1, st);
                    if (cudaEventSynchronize(e1) != cudaSuccess) { r = set_err(s, RGX_ERR_CUDA, "rgx_autotune: event"); break; }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < tmin) tmin = ms;
                }
                if (!r && tmin < best_t) { best_t = tmin; bo = o; }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r) return r;
    const rgx_status dev = rgx_sync_status(s, stream);
    if (dev) return dev;
    *best = bo;
    if (best_ms) *best_ms = best_t;
    return RGX_OK;
}
