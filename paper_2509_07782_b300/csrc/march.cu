// march.cu -- forward volume ray marching and its adjoint (Algorithm 1, Eq. 1-5).
//
// One thread marches one ray.  A warp owns a 32-ray tile popped from a
// persistent work counter shared by every camera of the launch (2D Z-order
// tiles with RGX_ZTILES, 32 consecutive scanline pixels otherwise).  Per
// segment [t_S, t_S + dS) the thread
//   1. collects the BVH leaves whose boxes overlap the segment, in ascending
//      leaf order, into its slice of shared memory (hit_cap entries; larger
//      lists are processed in chunks by restarting the traversal after the last
//      leaf taken, so no hit is ever dropped);
//   2. for every collected Gaussian solves its exact ellipsoid chord; those
//      whose chord overlaps the segment are the segment's hit set (Algorithm 1's
//      BVHTraversal, with segments wholly inside an ellipsoid included);
//   3. adds each hit's density sigma~ exp(-q/2) (hard-truncated at Q_eps) and
//      density-weighted SH colour to the N_S per-sample accumulators in
//      registers (Eq. 1), hits outer / samples inner;
//   4. composites the N_S samples front to back (Eq. 3).
// An empty hit set advances by dS, or with RGX_SKIP jumps to ClosestHit (Eq. 4).
//
// The adjoint kernel replays exactly the same arithmetic (same hit order, same
// explicitly rounded operations), so it reproduces T and the schedule bit for
// bit without storing any sample.  Using the residual C_final - C_<=i it
// forms dL/dsigma_i and dL/dc_i per sample, then per hit accumulates over the
// samples three scalars (sum w, sum w u, sum w u^2, w = dL/dg * g, u the
// sample offset from the chord centre) and dL/dc_l; these give the local-frame
// moments A0, V = sum w y, P = sum w y y^T that are atomically added per
// Gaussian.  k_grad_finalize chains them to mu, s, q, sigma~ (and scatters SH
// gradients) once per Gaussian.
#include <stdio.h>
#include "common.cuh"

#define FULLMASK 0xffffffffu
#define LEAF_BIT 0x80000000u
#define DONE 0xffffffffu
#define NEG_HALF_LOG2E (-0.72134752044448170368f)   // -1 / (2 ln 2)

struct MarchParams {
    const float4* __restrict__ geom;
    const float4* __restrict__ shc;
    const int32_t* __restrict__ perm;
    const float4* __restrict__ nodes;
    const float* __restrict__ root;
    const rgx_camera* __restrict__ cams;
    int64_t n;
    int morton;
    int ncam;
    int flags;
    float dt, dt_min, dt_max, beta, t_eps;
    float bg0, bg1, bg2;
    int tile_w, tile_h, hit_cap, max_segments;
    float4* rgba;
    float4* state;
    const float4* d_rgba;
    float4* grad;
    float2* sched;
    int sched_cap;
    int32_t* sched_n;
    unsigned int* queue;
    unsigned int* status;
    unsigned long long* counters;
};

struct Ray {
    float ox, oy, oz, dx, dy, dz;
    float ix, iy, iz;        // 1/d
};

struct Counters {
    unsigned segs, hits, evals, visits, chq, skips;
};

// Slab test of box [lo, hi] against the ray over [ta, tb].  Empty boxes are
// stored inverted (lo = +inf, hi = -inf) and always miss.
__device__ __forceinline__ bool box_overlap(float4 lo, float4 hi, const Ray& r, float ta, float tb, float& tentry) {
    float nx = r.ix >= 0.0f ? lo.x : hi.x, fx = r.ix >= 0.0f ? hi.x : lo.x;
    float ny = r.iy >= 0.0f ? lo.y : hi.y, fy = r.iy >= 0.0f ? hi.y : lo.y;
    float nz = r.iz >= 0.0f ? lo.z : hi.z, fz = r.iz >= 0.0f ? hi.z : lo.z;
    float t0 = fmaxf(fmaxf((nx - r.ox) * r.ix, (ny - r.oy) * r.iy), fmaxf((nz - r.oz) * r.iz, ta));
    float t1 = fminf(fminf((fx - r.ox) * r.ix, (fy - r.oy) * r.iy), fminf((fz - r.oz) * r.iz, tb));
    tentry = t0;
    return t0 <= t1;
}

// Exact chord of the Q_eps ellipsoid of Gaussian p: q(t) = qmin + a (t - tc)^2.
struct Chord {
    float tc, a, qmin, Qe, L;      // L = log2 sigma~
    float tin, tout;
    bool ok;
};

__device__ __forceinline__ Chord chord_of(const float4* __restrict__ geom, int64_t p, const Ray& r,
                                          float4& g1, float4& g2, float4& g3, float4& g0) {
    g0 = __ldg(&geom[4 * p + 0]);
    g1 = __ldg(&geom[4 * p + 1]);
    g2 = __ldg(&geom[4 * p + 2]);
    g3 = __ldg(&geom[4 * p + 3]);
    Chord c;
    const float ex = r.ox - g0.x, ey = r.oy - g0.y, ez = r.oz - g0.z;
    const float y0x = g1.x * ex + g1.y * ey + g1.z * ez;
    const float y0y = g2.x * ex + g2.y * ey + g2.z * ez;
    const float y0z = g3.x * ex + g3.y * ey + g3.z * ez;
    const float ydx = g1.x * r.dx + g1.y * r.dy + g1.z * r.dz;
    const float ydy = g2.x * r.dx + g2.y * r.dy + g2.z * r.dz;
    const float ydz = g3.x * r.dx + g3.y * r.dy + g3.z * r.dz;
    c.a = ydx * ydx + ydy * ydy + ydz * ydz;
    c.tc = -(y0x * ydx + y0y * ydy + y0z * ydz) / c.a;
    const float ycx = y0x + c.tc * ydx, ycy = y0y + c.tc * ydy, ycz = y0z + c.tc * ydz;
    c.qmin = ycx * ycx + ycy * ycy + ycz * ycz;
    c.Qe = g0.w;
    c.L = g1.w;
    const float rem = c.Qe - c.qmin;
    c.ok = (c.Qe > 0.0f) && (rem > 0.0f) && (c.a > 0.0f);
    const float h = c.ok ? sqrtf(rem / c.a) : 0.0f;
    c.tin = c.tc - h;
    c.tout = c.tc + h;
    return c;
}

// Local-frame quantities the adjoint needs: y_c = y(tc) and yd = M d.
__device__ __forceinline__ void local_frame(float4 g0, float4 g1, float4 g2, float4 g3, const Ray& r, float tc,
                                            float yc[3], float yd[3]) {
    const float ex = r.ox - g0.x, ey = r.oy - g0.y, ez = r.oz - g0.z;
    yd[0] = g1.x * r.dx + g1.y * r.dy + g1.z * r.dz;
    yd[1] = g2.x * r.dx + g2.y * r.dy + g2.z * r.dz;
    yd[2] = g3.x * r.dx + g3.y * r.dy + g3.z * r.dz;
    yc[0] = g1.x * ex + g1.y * ey + g1.z * ez + tc * yd[0];
    yc[1] = g2.x * ex + g2.y * ey + g2.z * ez + tc * yd[1];
    yc[2] = g3.x * ex + g3.y * ey + g3.z * ez + tc * yd[2];
}

// Left-first DFS over the radix tree collecting leaves >= cursor whose boxes
// overlap [ta, tb].  Returns the number collected; cursor becomes the first
// leaf not yet taken (DONE when the traversal finished).
__device__ int collect(const MarchParams& P, const Ray& r, float ta, float tb, uint32_t* __restrict__ hl,
                       int cap, uint32_t& cursor, uint32_t* __restrict__ stk, Counters& cnt) {
    const uint32_t start = cursor;
    int count = 0, sp = 0;
    uint32_t ref = 0;  // root (internal node 0)
    float te;
    while (true) {
        if (ref & LEAF_BIT) {
            const uint32_t leaf = ref & ~LEAF_BIT;
            if (count == cap) { cursor = leaf; return count; }
            hl[count * RGX_BLOCK] = leaf;
            count++;
        } else {
            cnt.visits++;
            const float4* nd = P.nodes + 4 * (size_t)ref;
            const float4 a0 = __ldg(nd), a1 = __ldg(nd + 1), a2 = __ldg(nd + 2), a3 = __ldg(nd + 3);
            const uint32_t first = __float_as_uint(a0.w), split = __float_as_uint(a1.w), last = __float_as_uint(a2.w);
            const bool hl_ = (split >= start) && box_overlap(a0, a1, r, ta, tb, te);
            const bool hr_ = (last >= start) && box_overlap(a2, a3, r, ta, tb, te);
            const uint32_t rl = (first == split) ? (split | LEAF_BIT) : split;
            const uint32_t rr = (split + 1 == last) ? ((split + 1) | LEAF_BIT) : (split + 1);
            if (hl_ && hr_) {
                if (sp < RGX_STACK) stk[sp++] = rr; else atomicOr(P.status, (unsigned)RGX_ERR_STACK_OVERFLOW);
                ref = rl;
                continue;
            }
            if (hl_) { ref = rl; continue; }
            if (hr_) { ref = rr; continue; }
        }
        if (sp == 0) { cursor = DONE; return count; }
        ref = stk[--sp];
    }
}

// ClosestHit(ta) = min over Gaussians whose chord has t_out > ta and
// t_in < tf of max(t_in, ta); tf if there is none (Algorithm 1, Eq. 4).
// Nearest-first traversal pruned by the best value found so far.
__device__ float closest_hit(const MarchParams& P, const Ray& r, float ta, float tf, uint32_t* __restrict__ stk,
                             float* __restrict__ tstk, Counters& cnt) {
    cnt.chq++;
    float best = tf;
    int sp = 0;
    uint32_t ref = 0;
    while (true) {
        if (!(ref & LEAF_BIT)) {
            cnt.visits++;
            const float4* nd = P.nodes + 4 * (size_t)ref;
            const float4 a0 = __ldg(nd), a1 = __ldg(nd + 1), a2 = __ldg(nd + 2), a3 = __ldg(nd + 3);
            const uint32_t first = __float_as_uint(a0.w), split = __float_as_uint(a1.w), last = __float_as_uint(a2.w);
            float tl, tr;
            bool hl_ = box_overlap(a0, a1, r, ta, best, tl);
            bool hr_ = box_overlap(a2, a3, r, ta, best, tr);
            uint32_t rl = (first == split) ? (split | LEAF_BIT) : split;
            uint32_t rr = (split + 1 == last) ? ((split + 1) | LEAF_BIT) : (split + 1);
            // leaves are resolved at once
            for (int side = 0; side < 2; side++) {
                const bool h = side ? hr_ : hl_;
                const uint32_t rf = side ? rr : rl;
                if (h && (rf & LEAF_BIT)) {
                    const uint32_t leaf = rf & ~LEAF_BIT;
                    const int64_t p = P.morton ? (int64_t)leaf : (int64_t)P.perm[leaf];
                    float4 g0, g1, g2, g3;
                    const Chord c = chord_of(P.geom, p, r, g1, g2, g3, g0);
                    if (c.ok && c.tout > ta && c.tin < tf) {
                        const float t = fmaxf(c.tin, ta);
                        if (t < best) best = t;
                    }
                    if (side) hr_ = false; else hl_ = false;
                }
            }
            if (best <= ta) return ta;
            if (hl_ && tl >= best) hl_ = false;
            if (hr_ && tr >= best) hr_ = false;
            if (hl_ && hr_) {
                const bool lfirst = tl <= tr;
                if (sp < RGX_STACK) { stk[sp] = lfirst ? rr : rl; tstk[sp] = lfirst ? tr : tl; sp++; }
                else atomicOr(P.status, (unsigned)RGX_ERR_STACK_OVERFLOW);
                ref = lfirst ? rl : rr;
                continue;
            }
            if (hl_) { ref = rl; continue; }
            if (hr_) { ref = rr; continue; }
        }
        bool found = false;
        while (sp > 0) {
            --sp;
            if (tstk[sp] < best) { ref = stk[sp]; found = true; break; }
        }
        if (!found) return best;
    }
}

// SH colour c_l(d) = max(0, 1/2 + sum_k Y_k(d) K_k); `pre` keeps the argument.
__device__ __forceinline__ void sh_colour(const float4* __restrict__ shc, int64_t p, const float Y[16], float c[3],
                                          float pre[3]) {
    const float4* s = shc + 12 * p;
    float r = 0.5f, g = 0.5f, b = 0.5f;
#pragma unroll
    for (int j = 0; j < 12; j++) {
        const float4 v = __ldg(&s[j]);
        // coefficient index 4j..4j+3 in (k, channel) order
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int idx = 4 * j + e;
            const int k = idx / 3, ch = idx % 3;
            const float t = Y[k] * vv[e];
            if (ch == 0) r += t; else if (ch == 1) g += t; else b += t;
        }
    }
    pre[0] = r; pre[1] = g; pre[2] = b;
    c[0] = fmaxf(r, 0.0f); c[1] = fmaxf(g, 0.0f); c[2] = fmaxf(b, 0.0f);
}

// Per-sample evaluation of one hit over the N_S samples of a segment.
template <int NS>
__device__ __forceinline__ void eval_hit(const Chord& c, float u0, float dtk, const float col[3], float sig[NS],
                                         float S[NS][3]) {
#pragma unroll
    for (int k = 0; k < NS; k++) {
        const float u = __fmaf_rn((float)k, dtk, u0);
        const float q = __fmaf_rn(__fmul_rn(c.a, u), u, c.qmin);
        if (q <= c.Qe) {
            const float g = exp2f(__fmaf_rn(q, NEG_HALF_LOG2E, c.L));
            sig[k] = __fadd_rn(sig[k], g);
            S[k][0] = __fmaf_rn(g, col[0], S[k][0]);
            S[k][1] = __fmaf_rn(g, col[1], S[k][1]);
            S[k][2] = __fmaf_rn(g, col[2], S[k][2]);
        }
    }
}

__device__ __forceinline__ void red_add4(float4* addr, float a, float b, float c, float d) {
    atomicAdd(addr, make_float4(a, b, c, d));
}

template <int NS, bool BWD>
__device__ void march_ray(const MarchParams& P, int64_t ray, int cam, int px, int py, uint32_t* __restrict__ hl,
                          uint32_t* __restrict__ stk, float* __restrict__ tstk, Counters& cnt) {
    const rgx_camera& C = P.cams[cam];
    // ---- ray (pinhole, OpenCV convention)
    Ray r;
    {
        const float ux = ((float)px + 0.5f - C.cx) / C.fx;
        const float vy = ((float)py + 0.5f - C.cy) / C.fy;
        float dx = C.c2w[0] * ux + C.c2w[1] * vy + C.c2w[2];
        float dy = C.c2w[4] * ux + C.c2w[5] * vy + C.c2w[6];
        float dz = C.c2w[8] * ux + C.c2w[9] * vy + C.c2w[10];
        const float inv = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
        r.dx = dx * inv; r.dy = dy * inv; r.dz = dz * inv;
        r.ox = C.c2w[3]; r.oy = C.c2w[7]; r.oz = C.c2w[11];
        const float tiny = 1e-20f;
        r.ix = 1.0f / (fabsf(r.dx) > tiny ? r.dx : copysignf(tiny, r.dx));
        r.iy = 1.0f / (fabsf(r.dy) > tiny ? r.dy : copysignf(tiny, r.dy));
        r.iz = 1.0f / (fabsf(r.dz) > tiny ? r.dz : copysignf(tiny, r.dz));
    }
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, bA = 0.f, Cf0 = 0.f, Cf1 = 0.f, Cf2 = 0.f, Tf = 1.f, dTcoef = 0.f;
    if (BWD) {
        const float4 up = P.d_rgba[ray];
        if (up.x == 0.0f && up.y == 0.0f && up.z == 0.0f && up.w == 0.0f) return;
        a0 = up.x; a1 = up.y; a2 = up.z; bA = up.w;
        const float4 st = P.state[ray];
        Cf0 = st.x; Cf1 = st.y; Cf2 = st.z; Tf = st.w;
        dTcoef = (a0 * P.bg0 + a1 * P.bg1 + a2 * P.bg2 - bA) * Tf;
    }
    // ---- bounds: t_n, and t_f = camera t_far or the exit of the scene box
    const float tn = C.t_near;
    float tf = C.t_far;
    if (!(tf > 0.0f)) {
        const float4 lo = make_float4(P.root[0], P.root[1], P.root[2], 0.f);
        const float4 hi = make_float4(P.root[3], P.root[4], P.root[5], 0.f);
        float tentry;
        const bool in = box_overlap(lo, hi, r, -INFINITY, INFINITY, tentry);
        float fx = r.ix >= 0.0f ? hi.x : lo.x, fy = r.iy >= 0.0f ? hi.y : lo.y, fz = r.iz >= 0.0f ? hi.z : lo.z;
        const float texit = fminf(fminf((fx - r.ox) * r.ix, (fy - r.oy) * r.iy), (fz - r.oz) * r.iz);
        tf = (in && texit > tn) ? texit : tn;
    }
    float Y[16];
    sh_basis16(r.dx, r.dy, r.dz, Y);

    const bool skip = (P.flags & RGX_SKIP) != 0;
    const bool uniform = (P.flags & RGX_ADAPTIVE) == 0;
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    float tS = tn;
    int j = 0;  // lattice index in uniform mode
    int nrec = 0;
    if (P.n > 0 && tf > tn && skip) {
        const float th = closest_hit(P, r, tn, tf, stk, tstk, cnt);
        if (uniform) {
            const int jj = (int)floorf((th - tn) / P.dt) - 1;
            j = jj > 0 ? jj : 0;
            tS = __fmaf_rn((float)j, P.dt, tn);
        } else {
            tS = th;
        }
    }
    const float minstep = uniform ? P.dt : (float)NS * fminf(P.dt_min, P.dt_max);
    const int iter_cap = P.max_segments > 0 ? P.max_segments
                                            : (int)fminf((tf - tn) / minstep, 2.0e9f) + 8;
    int iters = 0;
    while (P.n > 0 && tS < tf && T > P.t_eps) {
        if (iters >= iter_cap) { atomicOr(P.status, (unsigned)RGX_ERR_ITER_LIMIT); break; }
        iters++;
        // ---- segment size: uniform dt, or Eq. 5
        float dtk;
        if (uniform) {
            dtk = P.dt;
        } else {
            float base = fmaxf(__fdiv_rn(tS, P.beta), P.dt_min);
            dtk = fminf(__fmul_rn(base, rcbrtf(T)), P.dt_max);
        }
        const float te = uniform ? __fmaf_rn((float)(j + NS), P.dt, tn) : __fadd_rn(tS, __fmul_rn((float)NS, dtk));
        const float tcut = fminf(te, tf);
        float sig[NS], S[NS][3];
#pragma unroll
        for (int k = 0; k < NS; k++) { sig[k] = 0.f; S[k][0] = S[k][1] = S[k][2] = 0.f; }
        // ---- hit collection + per-sample accumulation (chunked)
        int nexact = 0;
        int nchunk = 0;
        int first_count = 0;
        uint32_t cursor = 0;
        do {
            const int nh = collect(P, r, tS, tcut, hl, P.hit_cap, cursor, stk, cnt);
            if (nchunk == 0) first_count = nh;
            nchunk++;
            for (int h = 0; h < nh; h++) {
                const uint32_t leaf = hl[h * RGX_BLOCK];
                const int64_t p = P.morton ? (int64_t)leaf : (int64_t)P.perm[leaf];
                float4 g0, g1, g2, g3;
                const Chord c = chord_of(P.geom, p, r, g1, g2, g3, g0);
                if (!(c.ok && c.tin < tcut && c.tout > tS)) continue;
                nexact++;
                float col[3], pre[3];
                sh_colour(P.shc, p, Y, col, pre);
                const float u0 = __fadd_rn(__fsub_rn(tS, c.tc), __fmul_rn(0.5f, dtk));
                eval_hit<NS>(c, u0, dtk, col, sig, S);
            }
        } while (cursor != DONE);
        (void)first_count;
        if (nexact == 0) {
            cnt.skips++;
            if (skip) {
                const float th = closest_hit(P, r, te, tf, stk, tstk, cnt);
                if (th >= tf) break;
                if (uniform) {
                    const int jj = (int)floorf((th - tn) / P.dt) - 1;
                    j = jj > j + 1 ? jj : j + 1;
                    tS = __fmaf_rn((float)j, P.dt, tn);
                } else {
                    tS = th;
                }
            } else {
                if (uniform) { j += NS; tS = __fmaf_rn((float)j, P.dt, tn); } else tS = te;
            }
            continue;
        }
        cnt.segs++;
        cnt.hits += nexact;
        cnt.evals += nexact * NS;
        if (!BWD && P.sched) {
            if (nrec < P.sched_cap) P.sched[ray * P.sched_cap + nrec] = make_float2(tS, dtk);
        }
        nrec++;
        // ---- front-to-back compositing of the N_S samples (Eq. 3)
        const float t0 = __fadd_rn(tS, __fmul_rn(0.5f, dtk));
        if (!BWD) {
#pragma unroll
            for (int k = 0; k < NS; k++) {
                const float tk = __fmaf_rn((float)k, dtk, t0);
                if (tk < tf && sig[k] > 0.0f) {
                    const float x = __fmul_rn(sig[k], dtk);
                    const float e = expf(-x);
                    const float alpha = -expm1f(-x);
                    const float w = __fmul_rn(T, alpha);
                    const float inv = __fdiv_rn(1.0f, sig[k]);
                    C0 = __fmaf_rn(w, __fmul_rn(S[k][0], inv), C0);
                    C1 = __fmaf_rn(w, __fmul_rn(S[k][1], inv), C1);
                    C2 = __fmaf_rn(w, __fmul_rn(S[k][2], inv), C2);
                    T = __fmul_rn(T, e);
                }
            }
        } else {
            // replay compositing, turning (sig, S) into (beta, gamma):
            //   dL/dg_l = beta_k + gamma_k . c_l,   dL/dc_l += gamma_k g_l
#pragma unroll
            for (int k = 0; k < NS; k++) {
                const float tk = __fmaf_rn((float)k, dtk, t0);
                if (tk < tf && sig[k] > 0.0f) {
                    const float x = __fmul_rn(sig[k], dtk);
                    const float e = expf(-x);
                    const float alpha = -expm1f(-x);
                    const float w = __fmul_rn(T, alpha);
                    const float inv = __fdiv_rn(1.0f, sig[k]);
                    const float c0 = __fmul_rn(S[k][0], inv), c1 = __fmul_rn(S[k][1], inv), c2 = __fmul_rn(S[k][2], inv);
                    C0 = __fmaf_rn(w, c0, C0);
                    C1 = __fmaf_rn(w, c1, C1);
                    C2 = __fmaf_rn(w, c2, C2);
                    const float Tn = __fmul_rn(T, e);
                    float ds = a0 * (Tn * c0 - (Cf0 - C0)) + a1 * (Tn * c1 - (Cf1 - C1)) + a2 * (Tn * c2 - (Cf2 - C2));
                    ds = dtk * (ds - dTcoef);
                    const float g0 = a0 * w * inv, g1_ = a1 * w * inv, g2_ = a2 * w * inv;
                    sig[k] = ds - (g0 * c0 + g1_ * c1 + g2_ * c2);
                    S[k][0] = g0; S[k][1] = g1_; S[k][2] = g2_;
                    T = Tn;
                } else {
                    sig[k] = 0.0f; S[k][0] = S[k][1] = S[k][2] = 0.0f;
                }
            }
            // second pass over the same hits: per-Gaussian moments and atomics
            uint32_t cur2 = 0;
            const bool reuse = (nchunk == 1);
            do {
                int nh;
                if (reuse) { nh = first_count; cur2 = DONE; }
                else nh = collect(P, r, tS, tcut, hl, P.hit_cap, cur2, stk, cnt);
                for (int h = 0; h < nh; h++) {
                    const uint32_t leaf = hl[h * RGX_BLOCK];
                    const int64_t p = P.morton ? (int64_t)leaf : (int64_t)P.perm[leaf];
                    float4 q0, q1, q2, q3;
                    const Chord c = chord_of(P.geom, p, r, q1, q2, q3, q0);
                    if (!(c.ok && c.tin < tcut && c.tout > tS)) continue;
                    float col[3], pre[3];
                    sh_colour(P.shc, p, Y, col, pre);
                    const float u0 = __fadd_rn(__fsub_rn(tS, c.tc), __fmul_rn(0.5f, dtk));
                    float A0 = 0.f, A1 = 0.f, A2 = 0.f, dc0 = 0.f, dc1 = 0.f, dc2 = 0.f;
#pragma unroll
                    for (int k = 0; k < NS; k++) {
                        const float u = __fmaf_rn((float)k, dtk, u0);
                        const float q = __fmaf_rn(__fmul_rn(c.a, u), u, c.qmin);
                        if (q <= c.Qe) {
                            const float g = exp2f(__fmaf_rn(q, NEG_HALF_LOG2E, c.L));
                            const float gp = sig[k] + S[k][0] * col[0] + S[k][1] * col[1] + S[k][2] * col[2];
                            const float wv = gp * g;
                            A0 += wv;
                            A1 += wv * u;
                            A2 += wv * u * u;
                            dc0 += S[k][0] * g; dc1 += S[k][1] * g; dc2 += S[k][2] * g;
                        }
                    }
                    float yc[3], yd[3];
                    local_frame(q0, q1, q2, q3, r, c.tc, yc, yd);
                    const float V0 = A0 * yc[0] + A1 * yd[0], V1 = A0 * yc[1] + A1 * yd[1], V2 = A0 * yc[2] + A1 * yd[2];
                    float Pm[6];
                    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
                    for (int m = 0; m < 6; m++) {
                        const int x = ia[m], y = ib[m];
                        Pm[m] = A0 * yc[x] * yc[y] + A1 * (yc[x] * yd[y] + yd[x] * yc[y]) + A2 * yd[x] * yd[y];
                    }
                    float4* gp = P.grad + 16 * p;
                    red_add4(gp + 0, A0, V0, V1, V2);
                    red_add4(gp + 1, Pm[0], Pm[1], Pm[2], Pm[3]);
                    red_add4(gp + 2, Pm[4], Pm[5], 0.f, 0.f);
                    const float m0 = pre[0] > 0.f ? dc0 : 0.f, m1 = pre[1] > 0.f ? dc1 : 0.f, m2 = pre[2] > 0.f ? dc2 : 0.f;
#pragma unroll
                    for (int jx = 0; jx < 12; jx++) {
                        float v[4];
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            const int idx = 4 * jx + e, k = idx / 3, ch = idx % 3;
                            v[e] = Y[k] * (ch == 0 ? m0 : (ch == 1 ? m1 : m2));
                        }
                        red_add4(gp + 4 + jx, v[0], v[1], v[2], v[3]);
                    }
                }
            } while (cur2 != DONE);
        }
        if (uniform) { j += NS; tS = __fmaf_rn((float)j, P.dt, tn); } else tS = te;
    }
    if (!BWD) {
        P.rgba[ray] = make_float4(C0 + T * P.bg0, C1 + T * P.bg1, C2 + T * P.bg2, 1.0f - T);
        if (P.state) P.state[ray] = make_float4(C0, C1, C2, T);
        if (P.sched_n) P.sched_n[ray] = nrec;
    } else {
        if (T != Tf) atomicOr(P.status, (unsigned)RGX_ERR_REPLAY);
    }
}

// ------------------------------------------------------------------ kernel
__device__ __forceinline__ uint32_t tiles_of(const rgx_camera& c, bool ztiles, int tw, int th) {
    if (!ztiles) return (uint32_t)(((int64_t)c.width * c.height + 31) / 32);
    const uint32_t ntx = (c.width + tw - 1) / tw, nty = (c.height + th - 1) / th;
    return ((ntx + 7) / 8) * ((nty + 7) / 8) * 64u;
}

template <int NS, bool BWD>
__global__ void __launch_bounds__(RGX_BLOCK) k_march(MarchParams P) {
    extern __shared__ uint32_t smem[];
    uint32_t* s_tiles = smem;                 // [ncam+1] tile prefix
    uint32_t* s_pix = smem + (P.ncam + 1);    // [ncam+1] pixel prefix
    const int off = ((2 * (P.ncam + 1)) + 3) & ~3;
    uint32_t* s_hits = smem + off;
    const bool zt = (P.flags & RGX_ZTILES) != 0;
    if (threadIdx.x == 0) {
        uint32_t tsum = 0, psum = 0;
        for (int c = 0; c < P.ncam; c++) {
            s_tiles[c] = tsum; s_pix[c] = psum;
            tsum += tiles_of(P.cams[c], zt, P.tile_w, P.tile_h);
            psum += (uint32_t)(P.cams[c].width * P.cams[c].height);
        }
        s_tiles[P.ncam] = tsum; s_pix[P.ncam] = psum;
    }
    __syncthreads();
    const uint32_t total = s_tiles[P.ncam];
    const int lane = threadIdx.x & 31;
    uint32_t* hl = s_hits + threadIdx.x;
    uint32_t stk[RGX_STACK];
    float tstk[RGX_STACK];
    while (true) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(P.queue, 1u);
        t = __shfl_sync(FULLMASK, t, 0);
        if (t >= total) break;
        int lo = 0, hi = P.ncam;  // find camera: s_tiles[c] <= t < s_tiles[c+1]
        while (hi - lo > 1) { int mid = (lo + hi) >> 1; if (s_tiles[mid] <= t) lo = mid; else hi = mid; }
        const int c = lo;
        const rgx_camera& cam = P.cams[c];
        const uint32_t lt = t - s_tiles[c];
        int px, py;
        bool valid;
        if (!zt) {
            const int64_t pix = (int64_t)lt * 32 + lane;
            valid = pix < (int64_t)cam.width * cam.height;
            px = (int)(pix % cam.width); py = (int)(pix / cam.width);
        } else {
            const uint32_t ntx = (cam.width + P.tile_w - 1) / P.tile_w;
            const uint32_t nsx = (ntx + 7) / 8;
            const uint32_t sblk = lt >> 6, w = lt & 63u;
            const uint32_t wx = (w & 1u) | ((w >> 1) & 2u) | ((w >> 2) & 4u);
            const uint32_t wy = ((w >> 1) & 1u) | ((w >> 2) & 2u) | ((w >> 3) & 4u);
            const uint32_t tx = (sblk % nsx) * 8 + wx, ty = (sblk / nsx) * 8 + wy;
            px = (int)(tx * P.tile_w + lane % P.tile_w);
            py = (int)(ty * P.tile_h + lane / P.tile_w);
            valid = px < cam.width && py < cam.height;
        }
        Counters cnt = {0, 0, 0, 0, 0, 0};
        if (valid) {
            const int64_t ray = (int64_t)s_pix[c] + (int64_t)py * cam.width + px;
            march_ray<NS, BWD>(P, ray, c, px, py, hl, stk, tstk, cnt);
        }
        if (P.counters) {
            const unsigned v[7] = {valid ? 1u : 0u, cnt.segs, cnt.hits, cnt.evals, cnt.visits, cnt.chq, cnt.skips};
#pragma unroll
            for (int i = 0; i < 7; i++) {
                const unsigned s = __reduce_add_sync(FULLMASK, v[i]);
                if (lane == 0 && s) atomicAdd(&P.counters[i == 6 ? 6 : i], (unsigned long long)s);
            }
        }
    }
}

// Per-Gaussian chain of the accumulated local-frame moments to the caller's
// parameters (packed index p -> caller index l):
//   dsigma~ = A0 / sigma~,  dmu = M^T V,  ds_j = P_jj / s_j,
//   dR = -R S P S^-1 (from dM = -P M^-T with M = S^-1 R^T), dq via R(q^) and the
//   normalisation q^ = q/|q|.
__global__ void k_grad_finalize(int64_t n, int morton, int nk, const float4* __restrict__ grad,
                                const float4* __restrict__ geom, const float4* __restrict__ aux,
                                const int32_t* __restrict__ perm, float* d_means, float* d_scales, float* d_quats,
                                float* d_dens, float* d_sh) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = morton ? (int64_t)perm[p] : p;
        const float4* gp = grad + 16 * p;
        const float4 v0 = gp[0], v1 = gp[1], v2 = gp[2];
        const float A0 = v0.x, V[3] = {v0.y, v0.z, v0.w};
        const float Ps[3][3] = {{v1.x, v1.y, v1.z}, {v1.y, v1.w, v2.x}, {v1.z, v2.x, v2.y}};
        const float4 g0 = geom[4 * p], g1 = geom[4 * p + 1], g2 = geom[4 * p + 2], g3 = geom[4 * p + 3];
        const float M[3][3] = {{g1.x, g1.y, g1.z}, {g2.x, g2.y, g2.z}, {g3.x, g3.y, g3.z}};
        (void)g0;
        const float sig = g2.w;
        const float4 qa = aux[2 * p], sa = aux[2 * p + 1];
        const float s[3] = {sa.x, sa.y, sa.z};
        if (sig > 0.0f) d_dens[l] += A0 / sig;
        for (int k = 0; k < 3; k++) d_means[3 * l + k] += M[0][k] * V[0] + M[1][k] * V[1] + M[2][k] * V[2];
        for (int jx = 0; jx < 3; jx++) d_scales[3 * l + jx] += Ps[jx][jx] / s[jx];
        const float qn = sqrtf(qa.x * qa.x + qa.y * qa.y + qa.z * qa.z + qa.w * qa.w);
        const float w = qa.x / qn, x = qa.y / qn, y = qa.z / qn, z = qa.w / qn;
        const float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                               {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                               {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
        float dR[3][3];
        for (int k = 0; k < 3; k++)
            for (int jx = 0; jx < 3; jx++) {
                float acc = 0.f;
                for (int m = 0; m < 3; m++) acc += R[k][m] * s[m] * Ps[m][jx];
                dR[k][jx] = -acc / s[jx];
            }
        const float dw = dR[0][1] * (-2 * z) + dR[0][2] * (2 * y) + dR[1][0] * (2 * z) + dR[1][2] * (-2 * x) +
                         dR[2][0] * (-2 * y) + dR[2][1] * (2 * x);
        const float dx = dR[0][1] * (2 * y) + dR[0][2] * (2 * z) + dR[1][0] * (2 * y) + dR[1][1] * (-4 * x) +
                         dR[1][2] * (-2 * w) + dR[2][0] * (2 * z) + dR[2][1] * (2 * w) + dR[2][2] * (-4 * x);
        const float dy = dR[0][0] * (-4 * y) + dR[0][1] * (2 * x) + dR[0][2] * (2 * w) + dR[1][0] * (2 * x) +
                         dR[1][2] * (2 * z) + dR[2][0] * (-2 * w) + dR[2][1] * (2 * z) + dR[2][2] * (-4 * y);
        const float dz = dR[0][0] * (-4 * z) + dR[0][1] * (-2 * w) + dR[0][2] * (2 * x) + dR[1][0] * (2 * w) +
                         dR[1][1] * (-4 * z) + dR[1][2] * (2 * y) + dR[2][0] * (2 * x) + dR[2][1] * (2 * y);
        const float dot = w * dw + x * dx + y * dy + z * dz;
        d_quats[4 * l + 0] += (dw - w * dot) / qn;
        d_quats[4 * l + 1] += (dx - x * dot) / qn;
        d_quats[4 * l + 2] += (dy - y * dot) / qn;
        d_quats[4 * l + 3] += (dz - z * dot) / qn;
        const float* gs = (const float*)(gp + 4);
        for (int i = 0; i < 3 * nk; i++) d_sh[(int64_t)l * 3 * nk + i] += gs[i];
    }
}

// ------------------------------------------------------------------ host side
template <int NS, bool BWD>
static void* kernel_ptr() { return (void*)k_march<NS, BWD>; }

static void* pick_kernel(int ns, bool bwd) {
    switch (ns) {
        case 4: return bwd ? kernel_ptr<4, true>() : kernel_ptr<4, false>();
        case 8: return bwd ? kernel_ptr<8, true>() : kernel_ptr<8, false>();
        case 16: return bwd ? kernel_ptr<16, true>() : kernel_ptr<16, false>();
        case 32: return bwd ? kernel_ptr<32, true>() : kernel_ptr<32, false>();
    }
    return nullptr;
}

static rgx_status check_opts(rgx_scene* s, const rgx_opts* o) {
    if (!o) return set_err(s, RGX_ERR_INVALID_ARG, "null opts");
    if (o->n_s != 4 && o->n_s != 8 && o->n_s != 16 && o->n_s != 32)
        return set_err(s, RGX_ERR_INVALID_ARG, "n_s must be 4, 8, 16 or 32");
    if (o->flags & RGX_ADAPTIVE) {
        if (!(o->dt_min > 0.0f) || !(o->dt_max >= o->dt_min) || !(o->beta > 0.0f))
            return set_err(s, RGX_ERR_INVALID_ARG, "adaptive mode needs 0 < dt_min <= dt_max and beta > 0");
    } else if (!(o->dt > 0.0f)) {
        return set_err(s, RGX_ERR_INVALID_ARG, "dt must be > 0");
    }
    if (o->hit_cap < 8 || o->hit_cap > 256) return set_err(s, RGX_ERR_INVALID_ARG, "hit_cap must be in [8, 256]");
    if ((o->flags & RGX_ZTILES) && (o->tile_w <= 0 || o->tile_h <= 0 || o->tile_w * o->tile_h != 32))
        return set_err(s, RGX_ERR_INVALID_ARG, "tile_w * tile_h must be 32");
    if (!(o->t_eps >= 0.0f)) return set_err(s, RGX_ERR_INVALID_ARG, "t_eps must be >= 0");
    return RGX_OK;
}

static rgx_status check_cams(rgx_scene* s, const rgx_camera* cams, int32_t ncam, int64_t* rays) {
    if (!cams || ncam <= 0 || ncam > RGX_MAX_CAMS) return set_err(s, RGX_ERR_INVALID_ARG, "need 1..1024 cameras");
    int64_t R = 0;
    for (int i = 0; i < ncam; i++) {
        const rgx_camera& c = cams[i];
        if (c.width <= 0 || c.height <= 0) return set_err(s, RGX_ERR_INVALID_ARG, "camera with zero size");
        if (!(c.fx != 0.0f) || !(c.fy != 0.0f)) return set_err(s, RGX_ERR_INVALID_ARG, "camera with zero focal");
        R += (int64_t)c.width * c.height;
    }
    if (R >= (int64_t)0xffffffffu) return set_err(s, RGX_ERR_INVALID_ARG, "too many rays in one call");
    *rays = R;
    return RGX_OK;
}

static rgx_status launch_march(rgx_scene* s, const rgx_camera* cams, int32_t ncam, const rgx_opts* o, bool bwd,
                               float* rgba, void* state, const float* d_rgba, float* sched, int sched_cap,
                               int32_t* sched_n, cudaStream_t st) {
    MarchParams P;
    memset(&P, 0, sizeof P);
    P.geom = s->geom; P.shc = s->shc; P.perm = s->perm; P.nodes = s->nodes; P.root = s->root;
    P.n = s->n; P.morton = s->morton;
    P.cams = s->cams; P.ncam = ncam;
    P.flags = o->flags;
    P.dt = o->dt; P.dt_min = o->dt_min; P.dt_max = o->dt_max; P.beta = o->beta; P.t_eps = o->t_eps;
    P.bg0 = o->bg[0]; P.bg1 = o->bg[1]; P.bg2 = o->bg[2];
    P.tile_w = o->tile_w > 0 ? o->tile_w : 8; P.tile_h = o->tile_h > 0 ? o->tile_h : 4;
    P.hit_cap = o->hit_cap; P.max_segments = o->max_segments;
    P.rgba = (float4*)rgba; P.state = (float4*)state;
    P.d_rgba = (const float4*)d_rgba; P.grad = s->grad;
    P.sched = (float2*)sched; P.sched_cap = sched_cap; P.sched_n = sched_n;
    P.queue = s->queue; P.status = s->status; P.counters = s->counters;
    RGX_CUDA(s, cudaMemcpyAsync(s->cams, cams, sizeof(rgx_camera) * ncam, cudaMemcpyHostToDevice, st));
    RGX_CUDA(s, cudaMemsetAsync(s->queue, 0, sizeof(unsigned), st));
    RGX_CUDA(s, cudaMemsetAsync(s->counters, 0, 8 * sizeof(unsigned long long), st));
    void* k = pick_kernel(o->n_s, bwd);
    const size_t smem = (size_t)((((2 * (ncam + 1)) + 3) & ~3) + o->hit_cap * RGX_BLOCK) * sizeof(uint32_t);
    RGX_CUDA(s, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    RGX_CUDA(s, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, RGX_BLOCK, smem));
    if (occ < 1) occ = 1;
    const int grid = s->num_sms * occ;
    void* args[] = {&P};
    RGX_CUDA(s, cudaLaunchKernel(k, dim3(grid), dim3(RGX_BLOCK), args, smem, st));
    return RGX_OK;
}

static rgx_status ensure_cams(rgx_scene* s, int ncam) {
    if (ncam <= s->cams_cap) return RGX_OK;
    if (s->cams) cudaFree(s->cams);
    s->cams = nullptr;
    if (cudaMalloc(&s->cams, sizeof(rgx_camera) * RGX_MAX_CAMS) != cudaSuccess)
        return set_err(s, RGX_ERR_WORKSPACE, "camera buffer allocation failed");
    s->cams_cap = RGX_MAX_CAMS;
    return RGX_OK;
}

static rgx_status forward_common(rgx_scene* s, const rgx_camera* cams, int32_t ncam, const rgx_opts* o, float* rgba,
                                 void* state, float* sched, int32_t sched_cap, int32_t* sched_n, void* stream) {
    if (!s) return set_err(s, RGX_ERR_INVALID_ARG, "null scene");
    if (!s->built) return set_err(s, RGX_ERR_NOT_BUILT, "rgx_render_forward before rgx_build_bvh");
    rgx_status r = check_opts(s, o);
    if (r) return r;
    int64_t R = 0;
    r = check_cams(s, cams, ncam, &R);
    if (r) return r;
    if (!rgba) return set_err(s, RGX_ERR_INVALID_ARG, "null rgba");
    if (sched && (sched_cap <= 0 || !sched_n)) return set_err(s, RGX_ERR_INVALID_ARG, "bad schedule buffers");
    RGX_CUDA(s, cudaSetDevice(s->device));
    r = ensure_cams(s, ncam);
    if (r) return r;
    return launch_march(s, cams, ncam, o, false, rgba, state, nullptr, sched, sched_cap, sched_n,
                        (cudaStream_t)stream);
}

extern "C" rgx_status rgx_render_forward(rgx_scene* s, const rgx_camera* cams, int32_t ncam, const rgx_opts* o,
                                         float* rgba, void* fwd_state, void* stream) {
    return forward_common(s, cams, ncam, o, rgba, fwd_state, nullptr, 0, nullptr, stream);
}

extern "C" rgx_status rgx_render_forward_sched(rgx_scene* s, const rgx_camera* cams, int32_t ncam, const rgx_opts* o,
                                               float* rgba, void* fwd_state, float* sched, int32_t sched_cap,
                                               int32_t* sched_n, void* stream) {
    if (!sched) return set_err(s, RGX_ERR_INVALID_ARG, "null schedule buffer");
    return forward_common(s, cams, ncam, o, rgba, fwd_state, sched, sched_cap, sched_n, stream);
}

extern "C" rgx_status rgx_render_backward(rgx_scene* s, const rgx_camera* cams, int32_t ncam, const rgx_opts* o,
                                          const void* fwd_state, const float* d_rgba, float* d_means,
                                          float* d_scales, float* d_quats, float* d_dens, float* d_sh, void* stream) {
    if (!s) return set_err(s, RGX_ERR_INVALID_ARG, "null scene");
    if (!s->built) return set_err(s, RGX_ERR_NOT_BUILT, "rgx_render_backward before rgx_build_bvh");
    rgx_status r = check_opts(s, o);
    if (r) return r;
    int64_t R = 0;
    r = check_cams(s, cams, ncam, &R);
    if (r) return r;
    if (!fwd_state || !d_rgba) return set_err(s, RGX_ERR_INVALID_ARG, "null fwd_state or d_rgba");
    if (s->n > 0 && (!d_means || !d_scales || !d_quats || !d_dens || !d_sh))
        return set_err(s, RGX_ERR_INVALID_ARG, "null gradient array");
    cudaStream_t st = (cudaStream_t)stream;
    RGX_CUDA(s, cudaSetDevice(s->device));
    r = ensure_cams(s, ncam);
    if (r) return r;
    if (s->n == 0) return RGX_OK;
    if (s->grad_cap < s->n) {
        if (s->grad) cudaFree(s->grad);
        s->grad = nullptr;
        if (cudaMalloc(&s->grad, (size_t)16 * sizeof(float4) * s->cap_n) != cudaSuccess)
            return set_err(s, RGX_ERR_WORKSPACE, "gradient accumulator allocation failed");
        s->grad_cap = s->cap_n;
    }
    RGX_CUDA(s, cudaMemsetAsync(s->grad, 0, (size_t)16 * sizeof(float4) * s->n, st));
    r = launch_march(s, cams, ncam, o, true, nullptr, (void*)fwd_state, d_rgba, nullptr, 0, nullptr, st);
    if (r) return r;
    const int nk = (s->sh_degree + 1) * (s->sh_degree + 1);
    int64_t b = (s->n + 255) / 256;
    if (b > (int64_t)s->num_sms * 16) b = (int64_t)s->num_sms * 16;
    k_grad_finalize<<<(int)b, 256, 0, st>>>(s->n, s->morton, nk, s->grad, s->geom, s->aux, s->perm, d_means,
                                            d_scales, d_quats, d_dens, d_sh);
    RGX_CUDA(s, cudaGetLastError());
    return RGX_OK;
}
