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

// One candidate: a warm-up run (workspace growth, launch-configuration cache), then the
// best of two runs timed with CUDA events on the caller's stream.
static rgx_status time_candidate(rgx_scene* s, const rgx_camera* cams, int32_t ncam, const rgx_opts* o, int bwd,
                                 float* rgba, void* state, const float* d_rgba, float* const g[5], cudaStream_t st,
                                 cudaEvent_t e0, cudaEvent_t e1, float* out_ms) {
    rgx_status r = run_once(s, cams, ncam, o, bwd, rgba, state, d_rgba, g, st);
    if (r) return r;
    float tmin = 1e30f;
    for (int rep = 0; rep < 2; rep++) {
        RGX_CUDA(s, cudaEventRecord(e0, st));
        r = run_once(s, cams, ncam, o, bwd, rgba, state, d_rgba, g, st);
        if (r) return r;
        RGX_CUDA(s, cudaEventRecord(e1, st));
        RGX_CUDA(s, cudaEventSynchronize(e1));
        float ms = 0.f;
        RGX_CUDA(s, cudaEventElapsedTime(&ms, e0, e1));
        if (ms < tmin) tmin = ms;
    }
    *out_ms = tmin;
    return RGX_OK;
}

extern "C" rgx_status rgx_autotune(rgx_scene* s, const rgx_camera* cams, int32_t ncam, const rgx_opts* base,
                                   int32_t mode, int32_t with_backward, float* rgba, void* fwd_state,
                                   const float* d_rgba, float* d_means, float* d_scales, float* d_quats,
                                   float* d_dens, float* d_sh, rgx_opts* best, float* best_ms, void* stream) {
    if (!s || !base || !best || !rgba || !fwd_state) return set_err(s, RGX_ERR_INVALID_ARG, "rgx_autotune: null argument");
    if (with_backward && (!d_rgba || !d_means || !d_scales || !d_quats || !d_dens || !d_sh))
        return set_err(s, RGX_ERR_INVALID_ARG, "rgx_autotune: backward tuning needs d_rgba and gradient buffers");
    if (mode & ~(RGX_TUNE_NS | RGX_TUNE_EXHAUSTIVE)) return set_err(s, RGX_ERR_INVALID_ARG, "rgx_autotune: bad mode");
    cudaStream_t st = (cudaStream_t)stream;
    float* const g[5] = {d_means, d_scales, d_quats, d_dens, d_sh};
    const int tiles[4][2] = {{8, 4}, {4, 8}, {16, 2}, {32, 1}};
    const int ntiles = (base->flags & RGX_ZTILES) ? 4 : 1;
    const int caps[10] = {32, 64, 96, 128, 192, 256, 384, 512, 640, 768};
    const int ncaps = 10;
    const int nss[4] = {4, 8, 16, 32};
    const bool tune_ns = (mode & RGX_TUNE_NS) != 0;
    // knobs left at 0 in base start from the defaults (not from an earlier tuning)
    rgx_opts b0 = *base;
    if (b0.hit_cap == 0) b0.hit_cap = RGX_DEFAULT_HIT_CAP;
    if (b0.tile_w == 0 && b0.tile_h == 0) { b0.tile_w = RGX_DEFAULT_TILE_W; b0.tile_h = RGX_DEFAULT_TILE_H; }
    if (b0.n_s == 0) b0.n_s = RGX_DEFAULT_NS;
    cudaEvent_t e0, e1;
    RGX_CUDA(s, cudaEventCreate(&e0));
    RGX_CUDA(s, cudaEventCreate(&e1));
    float best_t = 1e30f;
    rgx_opts bo = b0;
    rgx_status r = RGX_OK;
    auto consider = [&](const rgx_opts& o) {
        if (r) return;
        float ms = 0.f;
        r = time_candidate(s, cams, ncam, &o, with_backward, rgba, fwd_state, d_rgba, g, st, e0, e1, &ms);
        if (!r && ms < best_t) { best_t = ms; bo = o; }
    };
    if (mode & RGX_TUNE_EXHAUSTIVE) {
        // every (tile shape, hit_cap[, N_S], first-window lowering) combination
        const int nlow = (base->flags & RGX_SKIP) ? 2 : 1;
        for (int ti = 0; ti < ntiles; ti++)
            for (int ci = 0; ci < ncaps; ci++)
                for (int ni = 0; ni < (tune_ns ? 4 : 1); ni++)
                    for (int li = 0; li < nlow; li++) {
                        rgx_opts o = b0;
                        if (ntiles > 1) { o.tile_w = tiles[ti][0]; o.tile_h = tiles[ti][1]; }
                        o.hit_cap = caps[ci];
                        if (tune_ns) o.n_s = nss[ni];
                        if (li) o.flags ^= RGX_LOWER_FIRST;
                        consider(o);
                    }
    } else {
        // coordinate descent: the tile shape at the base hit_cap and N_S, then hit_cap at the best
        // shape, then N_S at the best shape and hit_cap (each configuration timed once)
        for (int ti = 0; ti < ntiles; ti++) {
            rgx_opts o = b0;
            if (ntiles > 1) { o.tile_w = tiles[ti][0]; o.tile_h = tiles[ti][1]; }
            consider(o);
        }
        const rgx_opts t1 = bo;
        for (int ci = 0; ci < ncaps; ci++) {
            if (caps[ci] == t1.hit_cap) continue;
            rgx_opts o = t1;
            o.hit_cap = caps[ci];
            consider(o);
        }
        if (bo.hit_cap != t1.hit_cap) {
            // the best tile shape can change with the list capacity: the others again at the new one
            const rgx_opts t1b = bo;
            for (int ti = 0; ti < ntiles; ti++) {
                if (tiles[ti][0] == t1b.tile_w && tiles[ti][1] == t1b.tile_h) continue;
                rgx_opts o = t1b;
                o.tile_w = tiles[ti][0];
                o.tile_h = tiles[ti][1];
                consider(o);
            }
        }
        if (tune_ns) {
            const rgx_opts t2 = bo;
            for (int ni = 0; ni < 4; ni++) {
                if (nss[ni] == t2.n_s) continue;
                rgx_opts o = t2;
                o.n_s = nss[ni];
                consider(o);
            }
        }
        if (base->flags & RGX_SKIP) {
            // the first window lowered while it overflows, or the whole ray or nothing
            rgx_opts o = bo;
            o.flags ^= RGX_LOWER_FIRST;
            consider(o);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r) return r;
    const rgx_status dev = rgx_sync_status(s, stream);
    if (dev) return dev;
    *best = bo;
    if (best_ms) *best_ms = best_t;
    // what tuning knobs left at 0 select from now on
    s->has_tuned = 1;
    s->tuned_hit_cap = bo.hit_cap;
    s->tuned_tile_w = bo.tile_w;
    s->tuned_tile_h = bo.tile_h;
    s->tuned_n_s = bo.n_s;
    s->tuned_flags = bo.flags;
    return RGX_OK;
}
