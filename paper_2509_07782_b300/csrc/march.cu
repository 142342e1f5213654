// march.cu -- forward volume ray marching and its adjoint (Algorithm 1, Eq. 1-5).
//
// Warp-per-ray design.  A warp pops a 32-ray tile from a persistent work
// counter shared by every camera of the launch (2D Z-order tiles with
// RGX_ZTILES, 32 consecutive scanline pixels otherwise) and marches the tile's
// rays one after another with all 32 lanes, so the control flow of a ray never
// diverges across lanes.  For a ray the warp
//   1. collects, by a cooperative BVH traversal (up to 32 nodes per step, a
//      shared-memory stack), the exact ellipsoid chords [t_in, t_out] of every
//      Gaussian overlapping a *window* [t_S, t_S + W) that spans one or more
//      segments, together with the per-(ray, Gaussian) quadratic
//      q(t) = q_min + a (t - t_c)^2 and SH colour c_l(d) -- once per window
//      instead of once per segment.  W adapts to the list capacity (hit_cap);
//      a single segment whose hits exceed it is processed in chunks, so no
//      hit is ever dropped;
//   2. takes, per segment [t_S, t_S + dS), the chords overlapping it: that is
//      the segment's hit set of Algorithm 1 (BVHTraversal), including segments
//      wholly inside an ellipsoid;
//   3. evaluates lane-parallel over samples (lane = sample k; 32/N_S lane groups
//      split the hits) sigma_k = sum_l sigma~_l exp(-q_l/2) (hard truncation at
//      Q_eps) and S_k = sum_l g_l c_l (Eq. 1), then composites the N_S samples
//      with a multiplicative warp scan for T_k (Eq. 3);
//   4. an empty hit set advances by dS, or with RGX_SKIP jumps to ClosestHit
//      (Eq. 4): from the window's chords when they decide it, else by a
//      cooperative nearest-hit traversal (at a ray's start first limited to a
//      little beyond the previous ray's first hit, which prunes it from the start).
// A segment whose hits overflow the list marks the ray as in a dense stretch:
// its following segments are collected in chunks straight away, and so is the
// first segment of the work item's next ray (the flag is kept in the ray's
// state, so the adjoint takes the same path) -- instead of first trying windows
// that would overflow again.
//
// The adjoint kernel replays exactly the same decisions and arithmetic, so it
// reproduces T and the schedule bit for bit without storing any sample.  Per
// segment it forms beta_k = dL/dsigma_k - gamma_k.c_k and gamma_k = dL/dc_k /
// sigma_k from the residual C_final - C_<=k, then hit-parallel sums per
// (ray, Gaussian) over the segment's samples w, w u, w u^2 (w = dL/dg g,
// u = t - t_c) and dL/dc_l; these give the local-frame moments A0, V = sum w y,
// P = sum w y y^T that are added atomically per Gaussian right away.
// k_grad_finalize chains them to mu, s, q, sigma~ once per Gaussian.
#include <stdio.h>
#include <cuda_fp16.h>
#include "common.cuh"

// Version of the march kernels: changed whenever their code changes, so that
// profiler counters taken on an older version are not attributed to this one.
#define RGX_MARCH_VERSION "m2-16"
#define FULLMASK 0xffffffffu
#define LEAF_BIT 0x80000000u
#define NEG_HALF_LOG2E (-0.72134752044448170368f)   // -1 / (2 ln 2)
#define WARPS (RGX_BLOCK / 32)
// Per-warp traversal stack.  A dense window's frontier fills it: with 320 entries the
// room above the depth-first reserve let a step pop only 21 of its 32 nodes on average
// on a 1M-Gaussian scene, with 448-1,024 about 31 (forward 17 % faster there).  448 is
// the most that still lets eight adjoint warps of hit_cap 512 share an SM's shared memory.
#define STK 448
#define STK_RES 152                                 // depth-first reserve: 3 x (4-wide depth bound 48) + 4
#define SURV 160                                    // leaves awaiting their exact chord (< 32 left + 128 new)
#define CUT 32                                      // child records of a tile's BVH cut
#ifndef RGX_LEAN_REGS
#define RGX_LEAN_REGS 168                           // registers per thread of the lean march kernel (12 warps/SM)
#endif
#ifndef SPILL_CAP
#define SPILL_CAP 4096                              // adjoint: chunk entries kept per warp in global scratch
#endif

#define TAPE_CHUNK 2048                             // tape entries a warp reserves at a time
#define TAPE_FULL 0xffffffffu                       // a warp's tape_base once a reservation has failed
#define RGX_CSUM_SLOTS 32                           // chunked-segment sums records per ray
#define PTAPE_BLOCK 65536                           // index-tape entries a warp reserves at a time
#define PTAPE_MIN_FREE 4096                         // a chunked segment starts a new block below this much room
#define RGX_CSUM_BUDGET (16ull << 30)               // bytes for those records
#define RGX_PTAPE_MAX (3000000000ull)               // entries of the index tape at most (48 GB with their colours)

struct MarchParams {
    const float4* __restrict__ geom;
    const float4* __restrict__ shc;
    const float4* __restrict__ sgp;  // spherical-Gaussian lobes (n_sg > 0)
    int n_sg;
    float4* gsg;                     // adjoint: lobe gradient accumulators (NULL: not requested)
    const int32_t* __restrict__ perm;
    const float4* __restrict__ nodes;
    const uint4* __restrict__ nodew;
    const float* __restrict__ root;
    const rgx_camera* __restrict__ cams;
    int64_t n;
    int morton;
    int ncam;
    int flags;
    float dt, dt_min, dt_max, beta, t_eps;
    float bg0, bg1, bg2;
    int tile_w, tile_h, hit_cap, max_segments;
    uint32_t min_items;  // small views are split until they have this many work items (16 per SM)
    float4* rgba;
    float4* state;
    const float4* d_rgba;
    float4* grad;
    float4* vgrad;  // adjoint with the densification statistic: per (packed Gaussian, camera) V moment
    float4* spill;  // adjoint: [grid][SPILL_CAP][3] chunk entries (q, c, pid) of an overflowing segment
    float4* tape;        // taped first-window lists, three planes of tape_cap entries: (t_c, a, q_min, Q_eps),
                         // (log2 sigma~, colour), (t_in, t_out, packed index bits, 0); forward writes, adjoint reads
    uint32_t* tape_n;    // forward: entries used so far
    uint32_t tape_cap;   // capacity in entries (0: no tape)
    uint32_t tape_tag;   // identifies the forward call whose lists the tape (and the sums records) hold
    float4* csums;       // per (ray, chunked segment ordinal < csum_slots): N_S + 1 float4 -- the segment's
                         // per-sample sums (sigma, S) as composited, then (hit count bits, 0, 0, 0)
    uint32_t csum_slots; // records per ray (0: none)
    uint4* ptape;        // recorded chunked segments' chords in the order the forward met them: (packed index,
                         // colour R, G, B bits) -- the colour as the forward evaluated it
    uint32_t* ptape_n;   // forward: entries reserved so far (per-warp blocks of PTAPE_BLOCK)
    uint32_t ptape_cap;  // capacity in entries (0: none)
    float2* sched;
    int sched_cap;
    int32_t* sched_n;
    unsigned int* queue;
    unsigned int* status;
    unsigned long long* counters;
};

struct Ray {
    float ox, oy, oz, dx, dy, dz;
    float ix, iy, iz;  // 1/d
};

struct Counters {
    unsigned segs, hits, evals, visits, chq, skips, windows;
};

// ------------------------------------------------------------------ per-warp shared memory
struct WS {
    float4* q;      // [cap] (t_c, a, q_min, Q_eps)
    float4* c;      // [cap] (log2 sigma~, c0, c1, c2)
    float2* tio;    // [cap] (t_in, t_out)
    float4* bg;     // [32]  (beta, gamma0..2)     adjoint only
    uint32_t* pid;  // [cap] packed index
    uint32_t* seg;  // [max(cap, STK)] entries of the current segment
    uint32_t* stk;  // [STK] node refs
    float* stkt;    // [STK] entry distance (nearest-hit traversal); aliases seg, which
                    // is dead whenever a traversal runs
    uint32_t* surv; // [SURV] leaves whose box meets the ray, awaiting the exact chord
    float* Y;       // [16] SH basis of the current ray direction
    uint4* cut;     // [CUT] the tile's BVH cut: compressed child records (box, ref)
    int* ncut;      // [1]   its size
};

__host__ __device__ inline size_t warp_bytes(int cap, bool bwd) {
    size_t b = (size_t)cap * (16 + 16 + 8 + 4) + (size_t)(cap > STK ? cap : STK) * 4 + (size_t)STK * 4 + SURV * 4 +
               CUT * 16 + 16 * 4 + 16;
    if (bwd) b += 32 * 16;
    return (b + 15) & ~(size_t)15;
}

__device__ inline WS carve(char* base, int cap, bool bwd) {
    WS w;
    char* p = base;
    w.q = (float4*)p; p += (size_t)cap * 16;
    w.c = (float4*)p; p += (size_t)cap * 16;
    w.cut = (uint4*)p; p += CUT * 16;
    if (bwd) { w.bg = (float4*)p; p += 32 * 16; } else w.bg = nullptr;
    w.tio = (float2*)p; p += (size_t)cap * 8;
    w.pid = (uint32_t*)p; p += (size_t)cap * 4;
    w.seg = (uint32_t*)p; p += (size_t)(cap > STK ? cap : STK) * 4;
    w.stkt = (float*)w.seg;
    w.stk = (uint32_t*)p; p += (size_t)STK * 4;
    w.surv = (uint32_t*)p; p += SURV * 4;
    w.Y = (float*)p; p += 16 * 4;
    w.ncut = (int*)p;
    return w;
}

// ------------------------------------------------------------------ geometry
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

// One child of a compressed node: its box (halves -> floats) and its ref.
__device__ __forceinline__ void child_of(uint4 v, float4& lo, float4& hi) {
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
    const float2 c = __half22float2(*reinterpret_cast<const __half2*>(&v.z));
    lo = make_float4(a.x, a.y, b.x, 0.0f);
    hi = make_float4(b.y, c.x, c.y, 0.0f);
}

// Exact chord of the Q_eps ellipsoid of Gaussian p: q(t) = qmin + a (t - tc)^2.
// a.b in three explicitly rounded steps (a fused multiply-add chain)
__device__ __forceinline__ float dot3_rn(float a0, float a1, float a2, float b0, float b1, float b2) {
    return __fmaf_rn(a0, b0, __fmaf_rn(a1, b1, __fmul_rn(a2, b2)));
}

struct Chord {
    float tc, a, qmin, Qe, L;
    float tin, tout;
    bool ok;
};

__device__ __forceinline__ Chord chord_of(const float4* __restrict__ geom, int64_t p, const Ray& r) {
    const float4 g0 = __ldg(&geom[4 * p + 0]);
    const float4 g1 = __ldg(&geom[4 * p + 1]);
    const float4 g2 = __ldg(&geom[4 * p + 2]);
    const float4 g3 = __ldg(&geom[4 * p + 3]);
    // every operation rounded explicitly: the adjoint kernel recomputes chords in
    // other contexts and must get the same bits (no compiler contraction choices)
    Chord c;
    const float ex = __fsub_rn(r.ox, g0.x), ey = __fsub_rn(r.oy, g0.y), ez = __fsub_rn(r.oz, g0.z);
    const float y0x = dot3_rn(g1.x, g1.y, g1.z, ex, ey, ez);
    const float y0y = dot3_rn(g2.x, g2.y, g2.z, ex, ey, ez);
    const float y0z = dot3_rn(g3.x, g3.y, g3.z, ex, ey, ez);
    const float ydx = dot3_rn(g1.x, g1.y, g1.z, r.dx, r.dy, r.dz);
    const float ydy = dot3_rn(g2.x, g2.y, g2.z, r.dx, r.dy, r.dz);
    const float ydz = dot3_rn(g3.x, g3.y, g3.z, r.dx, r.dy, r.dz);
    c.a = dot3_rn(ydx, ydy, ydz, ydx, ydy, ydz);
    const float inv_a = __frcp_rn(c.a);
    c.tc = __fmul_rn(-dot3_rn(y0x, y0y, y0z, ydx, ydy, ydz), inv_a);
    const float ycx = __fmaf_rn(c.tc, ydx, y0x), ycy = __fmaf_rn(c.tc, ydy, y0y), ycz = __fmaf_rn(c.tc, ydz, y0z);
    c.qmin = dot3_rn(ycx, ycy, ycz, ycx, ycy, ycz);
    c.Qe = g0.w;
    c.L = g1.w;
    const float rem = __fsub_rn(c.Qe, c.qmin);
    c.ok = (c.Qe > 0.0f) && (rem > 0.0f) && (c.a > 0.0f);
    const float h = c.ok ? __fsqrt_rn(__fmul_rn(rem, inv_a)) : 0.0f;
    c.tin = __fsub_rn(c.tc, h);
    c.tout = __fadd_rn(c.tc, h);
    return c;
}

// y_c = M (o + t_c d - mu) and yd = M d of Gaussian p.
__device__ __forceinline__ void local_frame(const float4* __restrict__ geom, int64_t p, const Ray& r, float tc,
                                            float yc[3], float yd[3]) {
    const float4 g0 = __ldg(&geom[4 * p + 0]);
    const float4 g1 = __ldg(&geom[4 * p + 1]);
    const float4 g2 = __ldg(&geom[4 * p + 2]);
    const float4 g3 = __ldg(&geom[4 * p + 3]);
    const float ex = __fsub_rn(r.ox, g0.x), ey = __fsub_rn(r.oy, g0.y), ez = __fsub_rn(r.oz, g0.z);
    yd[0] = dot3_rn(g1.x, g1.y, g1.z, r.dx, r.dy, r.dz);
    yd[1] = dot3_rn(g2.x, g2.y, g2.z, r.dx, r.dy, r.dz);
    yd[2] = dot3_rn(g3.x, g3.y, g3.z, r.dx, r.dy, r.dz);
    yc[0] = __fmaf_rn(tc, yd[0], dot3_rn(g1.x, g1.y, g1.z, ex, ey, ez));
    yc[1] = __fmaf_rn(tc, yd[1], dot3_rn(g2.x, g2.y, g2.z, ex, ey, ez));
    yc[2] = __fmaf_rn(tc, yd[2], dot3_rn(g3.x, g3.y, g3.z, ex, ey, ez));
}

// Colour c_l(d) = max(0, 1/2 + sum_k Y_k(d) K_k + sum_j a_j exp(lambda_j (mu_j . d - 1))):
// SH (Y in shared memory) plus the Gaussian's spherical-Gaussian lobes, if any.
__device__ __forceinline__ void sh_colour(const float4* __restrict__ shc, const float4* __restrict__ sgp, int n_sg,
                                          int64_t p, const float* Y, const Ray& ray, float c[3]) {
    const float4* s = shc + 12 * p;
    // two partial sums per channel (even / odd SH index) shorten the dependency chains
    float r = 0.5f, g = 0.5f, b = 0.5f, r2 = 0.0f, g2 = 0.0f, b2 = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        // coefficients 12j .. 12j+11 = SH indices 4j .. 4j+3, three channels each
        const float4 v0 = __ldg(&s[3 * j]), v1 = __ldg(&s[3 * j + 1]), v2 = __ldg(&s[3 * j + 2]);
        const float4 y = *reinterpret_cast<const float4*>(Y + 4 * j);
        r = __fmaf_rn(y.x, v0.x, r); g = __fmaf_rn(y.x, v0.y, g); b = __fmaf_rn(y.x, v0.z, b);
        r2 = __fmaf_rn(y.y, v0.w, r2); g2 = __fmaf_rn(y.y, v1.x, g2); b2 = __fmaf_rn(y.y, v1.y, b2);
        r = __fmaf_rn(y.z, v1.z, r); g = __fmaf_rn(y.z, v1.w, g); b = __fmaf_rn(y.z, v2.x, b);
        r2 = __fmaf_rn(y.w, v2.y, r2); g2 = __fmaf_rn(y.w, v2.z, g2); b2 = __fmaf_rn(y.w, v2.w, b2);
    }
    for (int j = 0; j < n_sg; j++) {
        const float4 ax = __ldg(&sgp[2 * (p * n_sg + j)]), am = __ldg(&sgp[2 * (p * n_sg + j) + 1]);
        const float e = expf(__fmul_rn(ax.w, __fsub_rn(dot3_rn(ax.x, ax.y, ax.z, ray.dx, ray.dy, ray.dz), 1.0f)));
        r2 = __fmaf_rn(am.x, e, r2); g2 = __fmaf_rn(am.y, e, g2); b2 = __fmaf_rn(am.z, e, b2);
    }
    c[0] = fmaxf(__fadd_rn(r, r2), 0.0f); c[1] = fmaxf(__fadd_rn(g, g2), 0.0f); c[2] = fmaxf(__fadd_rn(b, b2), 0.0f);
}

// Minimum over the warp in one reduction: floats mapped to order-preserving
// unsigned keys (no NaN reaches here).
__device__ __forceinline__ float warp_min(float v) {
    return ord2f(__reduce_min_sync(FULLMASK, f2ord(v)));
}

__device__ __forceinline__ uint32_t lanemask_lt() { return (1u << (threadIdx.x & 31)) - 1u; }

// ------------------------------------------------------------------ traversals
struct NoChunk {
    __device__ void operator()(int) const {}
};

// Test of one 4-wide child record (a box for internal and leaf children alike)
// against the ray over [ta, tb); te = entry distance.
__device__ __forceinline__ bool record_hit(uint4 v, const Ray& r, float ta, float tb, float& te) {
    float4 lo, hi;
    child_of(v, lo, hi);
    return box_overlap(lo, hi, r, ta, tb, te);
}

// Exclusive prefix sum over the warp; `total` receives the sum over all lanes.
__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t v, uint32_t& total) {
    const int lane = threadIdx.x & 31;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(FULLMASK, x, d);
        if (lane >= d) x += t;
    }
    total = __shfl_sync(FULLMASK, x, 31);
    return x - v;
}

// Nodes to pop in one traversal step: up to 32 while the stack keeps room for
// their (up to 4) children each above the depth-first reserve, then one at a
// time; 0 when even that no longer fits (stack overflow).
__device__ __forceinline__ int pop_count(int sp) {
    if (STK - sp < 4) return 0;
    return min(min(sp, 32), max((STK - STK_RES - sp) / 4, 1));
}

// Colours of list entries [from, to), computed once the list is final.
__device__ __forceinline__ void colour_entries(const MarchParams& P, const WS& W, const Ray& r, int from, int to) {
    const int lane = threadIdx.x & 31;
    for (int e = from + lane; e < to; e += 32) {
        float col[3];
        sh_colour(P.shc, P.sgp, P.n_sg, W.pid[e], W.Y, r, col);
        W.c[e] = make_float4(W.c[e].x, col[0], col[1], col[2]);
    }
    __syncwarp();
}

// Ascending bitonic sort of one float per lane across the warp.
__device__ __forceinline__ float warp_sort_asc(float v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const float o = __shfl_xor_sync(FULLMASK, v, j);
            const bool up = (lane & k) == 0, lower = (lane & j) == 0;
            v = (lower == up) ? fminf(v, o) : fmaxf(v, o);
        }
    }
    return v;
}

// Smaller window end for a list that overflows: about the median chord entry of
// the list (from 32 evenly spaced entries), but above tb_floor.
__device__ __forceinline__ float shrink_bound(const WS& W, int nL, float tb_floor) {
    const int lane = threadIdx.x & 31;
    const float v = warp_sort_asc(W.tio[(lane * nL) >> 5].x);
    const float med = __shfl_sync(FULLMASK, v, 16);
    return fmaxf(med, nextafterf(tb_floor, INFINITY));
}

// Keep, in order, the list entries whose chord starts before tb; returns their number.
__device__ __forceinline__ int compact_below(const WS& W, int nL, float tb) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    int out = 0;
    for (int b = 0; b < nL; b += 32) {
        const int e = b + lane;
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f), c = q;
        float2 io = make_float2(0.f, 0.f);
        uint32_t pid = 0;
        const bool k = e < nL && W.tio[e].x < tb;
        if (k) { q = W.q[e]; c = W.c[e]; io = W.tio[e]; pid = W.pid[e]; }
        const uint32_t bb = __ballot_sync(FULLMASK, k);
        __syncwarp();
        if (k) {
            const int d = out + __popc(bb & lt);
            W.q[d] = q; W.c[d] = c; W.tio[d] = io; W.pid[d] = pid;
        }
        out += __popc(bb);
        __syncwarp();
    }
    return out;
}

// Collect into the list every Gaussian whose exact chord overlaps [ta, tb).
// Each traversal step pops up to 32 4-wide nodes (one per lane; a lane tests
// the node's four child boxes).  Leaves whose box meets the ray are queued and
// their exact chords solved in full 32-lane rounds; SH colours are computed
// afterwards for the kept entries only.
//   Window mode (chunked = false): when the chords would overflow the list,
// the window end tb is lowered -- to about the median chord entry of the list,
// never to tb_floor or below -- the list keeps the chords that start before
// it and the same traversal goes on against the smaller window (popped nodes
// and queued leaves are tested against the current tb).  On return the list
// holds exactly the chords overlapping [ta, tb) for the final tb.  Returns 0
// when complete, 1 when even a window ending just above tb_floor overflows
// (pass tb_floor >= tb to forbid lowering tb), 2 on a traversal-stack overflow.
//   Chunked mode: tb stays; a full list is handed to `on_full(m)` and reset.
template <bool BWD, class OnFull>
__device__ int w_collect(const MarchParams& P, const WS& W, const Ray& r, float ta, float& tb, float tb_floor,
                         int cap, int& nL, bool chunked, OnFull on_full, Counters& cnt, float min_extent = 0.0f) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    int sp = 0, nsurv = 0, ncol = nL;  // entries [ncol, nL) still need their colour
    // first step: the tile's cut (at most 32 records in shared memory) instead of the root
    {
        const int ncut = *W.ncut;
        bool h = false;
        uint32_t rf = 0;
        if (lane < ncut) {
            const uint4 v = W.cut[lane];
            float te;
            h = record_hit(v, r, ta, tb, te);
            rf = v.w;
        }
        const bool leaf = (rf & LEAF_BIT) != 0;
        const bool pi = h && !leaf, pl = h && leaf;
        const uint32_t bi = __ballot_sync(FULLMASK, pi), bl = __ballot_sync(FULLMASK, pl);
        if (pi) W.stk[__popc(bi & lt)] = rf;
        if (pl) W.surv[__popc(bl & lt)] = rf & ~LEAF_BIT;
        sp = __popc(bi);
        nsurv = __popc(bl);
        __syncwarp();
    }
    while (sp > 0 || nsurv > 0) {
        if (sp > 0) {
            const int take = pop_count(sp);
            if (take <= 0) {
                if (lane == 0) atomicOr(P.status, (unsigned)RGX_ERR_STACK_OVERFLOW);
                return 2;
            }
            const int base = sp - take;
            const uint32_t ref = lane < take ? W.stk[base + lane] : 0u;
            __syncwarp();
            sp = base;
            uint32_t rf[4];
            bool hit[4];
#pragma unroll
            for (int j = 0; j < 4; j++) { rf[j] = 0u; hit[j] = false; }
            if (lane < take) {
                cnt.visits++;
                const uint4* nw = P.nodew + 4 * (size_t)ref;
                uint4 v[4];
#pragma unroll
                for (int j = 0; j < 4; j++) v[j] = __ldg(nw + j);
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    float te;
                    rf[j] = v[j].w;
                    hit[j] = record_hit(v[j], r, ta, tb, te);
                }
            }
            // slot-major compaction: internal children onto the stack, leaves into the queue
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const bool leaf = (rf[j] & LEAF_BIT) != 0;
                const uint32_t bi = __ballot_sync(FULLMASK, hit[j] && !leaf);
                const uint32_t bl = __ballot_sync(FULLMASK, hit[j] && leaf);
                if (hit[j] && !leaf) W.stk[sp + __popc(bi & lt)] = rf[j];
                if (hit[j] && leaf) W.surv[nsurv + __popc(bl & lt)] = rf[j] & ~LEAF_BIT;
                sp += __popc(bi);
                nsurv += __popc(bl);
            }
            __syncwarp();
        }
        // exact chords of the queued leaves, 32 at a time (all of them once the
        // traversal has finished)
        while (nsurv >= 32 || (sp == 0 && nsurv > 0)) {
            const int m = min(nsurv, 32);
            const bool h2 = lane < m;
            Chord ch;
            ch.ok = false;
            uint32_t q = 0;
            if (h2) {
                q = W.surv[nsurv - m + lane];
                ch = chord_of(P.geom, q, r);
            }
            bool keep = h2 && ch.ok && ch.tout > ta && ch.tin < tb;
            uint32_t bk = __ballot_sync(FULLMASK, keep);
            int nk = __popc(bk);
            if (nL + nk > cap) {
                if (chunked) {
                    colour_entries(P, W, r, ncol, nL);
                    on_full(nL);
                    nL = 0;
                    ncol = 0;
                } else {
                    // lower the window end until the list and this round fit; with min_extent > 0
                    // the window must keep that much beyond its earliest chord entry
                    while (nL + nk > cap) {
                        float fl = tb_floor;
                        if (min_extent > 0.0f) {
                            float m = INFINITY;
                            for (int e = lane; e < nL; e += 32) m = fminf(m, fmaxf(W.tio[e].x, ta));
                            if (keep) m = fminf(m, fmaxf(ch.tin, ta));
                            fl = fmaxf(fl, __fadd_rn(warp_min(m), min_extent));
                        }
                        const float tb2 = nL > 0 ? shrink_bound(W, nL, fl) : nextafterf(fl, INFINITY);
                        if (!(tb2 < tb)) return 1;
                        nL = compact_below(W, nL, tb2);
                        tb = tb2;
                        keep = keep && ch.tin < tb;
                        bk = __ballot_sync(FULLMASK, keep);
                        nk = __popc(bk);
                    }
                    ncol = min(ncol, nL);
                }
            }
            if (keep) {
                const int slot = nL + __popc(bk & lt);
                W.q[slot] = make_float4(ch.tc, ch.a, ch.qmin, ch.Qe);
                W.c[slot] = make_float4(ch.L, 0.f, 0.f, 0.f);
                W.tio[slot] = make_float2(ch.tin, ch.tout);
                W.pid[slot] = q;
            }
            nL += nk;
            nsurv -= m;
            __syncwarp();
        }
    }
    colour_entries(P, W, r, ncol, nL);
    return 0;
}

// ClosestHit(ta) = min over Gaussians whose chord has t_out > ta and t_in < tf of
// max(t_in, ta); tf if there is none (Algorithm 1, Eq. 4).  Cooperative 4-wide
// traversal pruned by the warp's best value: a lane pushes its node's internal
// children far to near (so the nearest is popped first) and queues leaves whose
// box starts before the best value; after every step the queued leaves' exact
// chords are solved 32 at a time and lower the best value.  Called with tf
// replaced by a smaller limit it returns the same minimum if one lies below the
// limit, else the limit itself.
__device__ __forceinline__ void cswap_desc(float& ta_, uint32_t& ra, float& tb_, uint32_t& rb) {
    if (ta_ < tb_) {
        const float t = ta_; ta_ = tb_; tb_ = t;
        const uint32_t x = ra; ra = rb; rb = x;
    }
}

__device__ float w_closest(const MarchParams& P, const WS& W, const Ray& r, float ta, float tf, Counters& cnt) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    if (lane == 0) cnt.chq++;
    int sp = 0, nq = 0;
    float best = tf;
    // first step: the tile's cut (at most 32 records in shared memory) instead of the root
    {
        const int ncut = *W.ncut;
        bool h = false;
        uint32_t rf = 0;
        float te = INFINITY;
        if (lane < ncut) {
            const uint4 v = W.cut[lane];
            h = record_hit(v, r, ta, tf, te);
            rf = v.w;
        }
        const bool leaf = (rf & LEAF_BIT) != 0;
        const bool pi = h && !leaf, pl = h && leaf;
        const uint32_t bi = __ballot_sync(FULLMASK, pi), bl = __ballot_sync(FULLMASK, pl);
        if (pi) {
            W.stk[__popc(bi & lt)] = rf;
            W.stkt[__popc(bi & lt)] = te;
        }
        if (pl) W.surv[__popc(bl & lt)] = rf & ~LEAF_BIT;
        sp = __popc(bi);
        nq = __popc(bl);
        __syncwarp();
    }
    while (true) {
        // exact chords of the queued leaves
        while (nq > 0) {
            const int m = min(nq, 32);
            float cand = INFINITY;
            if (lane < m) {
                const Chord c = chord_of(P.geom, W.surv[nq - m + lane], r);
                if (c.ok && c.tout > ta && c.tin < tf) cand = fmaxf(c.tin, ta);
            }
            best = fminf(best, warp_min(cand));
            nq -= m;
        }
        if (best <= ta) return ta;
        if (sp == 0) break;
        const int take = pop_count(sp);
        if (take <= 0) {
            if (lane == 0) atomicOr(P.status, (unsigned)RGX_ERR_STACK_OVERFLOW);
            return best;
        }
        const int base = sp - take;
        const uint32_t ref = lane < take ? W.stk[base + lane] : 0u;
        const float tent = lane < take ? W.stkt[base + lane] : INFINITY;
        __syncwarp();
        sp = base;
        float tt[4];
        uint32_t rr[4];
        uint32_t ni = 0, nl = 0, lmask = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) { tt[j] = -INFINITY; rr[j] = 0u; }
        if (lane < take && tent < best) {
            cnt.visits++;
            const uint4* nw = P.nodew + 4 * (size_t)ref;
            uint4 v[4];
#pragma unroll
            for (int j = 0; j < 4; j++) v[j] = __ldg(nw + j);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                float te;
                if (record_hit(v[j], r, ta, best, te)) {
                    rr[j] = v[j].w;
                    if (v[j].w & LEAF_BIT) { lmask |= 1u << j; nl++; }
                    else { tt[j] = te; ni++; }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const bool q = (lmask >> j) & 1u;
            const uint32_t bl = __ballot_sync(FULLMASK, q);
            if (q) W.surv[nq + __popc(bl & lt)] = rr[j] & ~LEAF_BIT;
            nq += __popc(bl);
        }
        // internal children, far to near
        cswap_desc(tt[0], rr[0], tt[1], rr[1]);
        cswap_desc(tt[2], rr[2], tt[3], rr[3]);
        cswap_desc(tt[0], rr[0], tt[2], rr[2]);
        cswap_desc(tt[1], rr[1], tt[3], rr[3]);
        cswap_desc(tt[1], rr[1], tt[2], rr[2]);
        // slot-major: every lane's farthest child first, so the nearest ones end on top
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const bool pu = j < (int)ni;
            const uint32_t bi = __ballot_sync(FULLMASK, pu);
            if (pu) {
                const int o = sp + __popc(bi & lt);
                W.stk[o] = rr[j];
                W.stkt[o] = tt[j];
            }
            sp += __popc(bi);
        }
        __syncwarp();
    }
    return best;
}

// ClosestHit(ta) with a guess: the query is first limited to [ta, lim) with lim a
// little beyond the guess (a neighbouring ray's first hit), which prunes from the
// first step; when nothing starts below lim the rest [lim, tf) is searched.  The
// result is the same minimum either way (the limited query returns lim exactly
// when no chord with t_in < lim ends after ta).
__device__ __forceinline__ float w_closest_guess(const MarchParams& P, const WS& W, const Ray& r, float ta, float tf,
                                                 float guess, Counters& cnt) {
    float hi = tf;
    if (guess > ta && guess < tf) {
        const float lim = fminf(__fadd_rn(guess, __fmul_rn(0.02f, __fsub_rn(guess, ta))), tf);
        if (lim > ta && lim < tf) hi = lim;
    }
    // one call site, two passes at most: [ta, lim), then [lim, tf) when nothing starts below lim
    float lo = ta, t;
    while (true) {
        t = w_closest(P, W, r, lo, hi, cnt);
        if (t < hi || hi >= tf) break;
        lo = hi;
        hi = tf;
    }
    return t;
}

// ------------------------------------------------------------------ per-segment work
// Lane-parallel sample evaluation: lane = (sample k, group grp); the group's
// lanes take every G-th hit.  Entry indices come from W.seg (idx) or 0..m-1.
// Only lanes whose sample lies in the current piece of the segment (act) add.
template <int NS>
__device__ __forceinline__ void eval_entries(const WS& W, bool idx, int m, float tS, float dtk, bool act,
                                             float& sig, float& S0, float& S1, float& S2) {
    constexpr int G = 32 / NS;
    const int lane = threadIdx.x & 31;
    const int k = lane % NS, grp = lane / NS;
    const float half = __fmul_rn(0.5f, dtk);
    if (!act) return;
    // four hits per iteration, all shared-memory loads issued before the math
    int h = grp;
    for (; h + 3 * G < m; h += 4 * G) {
        uint32_t e[4];
#pragma unroll
        for (int i = 0; i < 4; i++) e[i] = idx ? W.seg[h + i * G] : (uint32_t)(h + i * G);
        float4 q4[4], c4[4];
#pragma unroll
        for (int i = 0; i < 4; i++) { q4[i] = W.q[e[i]]; c4[i] = W.c[e[i]]; }
        float g[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const float u = __fmaf_rn((float)k, dtk, __fadd_rn(__fsub_rn(tS, q4[i].x), half));
            const float q = __fmaf_rn(__fmul_rn(q4[i].y, u), u, q4[i].z);
            g[i] = q <= q4[i].w ? exp2f(__fmaf_rn(q, NEG_HALF_LOG2E, c4[i].x)) : 0.0f;
        }
        // pairwise sums: two independent chains per accumulator
        sig = __fadd_rn(sig, __fadd_rn(__fadd_rn(g[0], g[1]), __fadd_rn(g[2], g[3])));
        S0 = __fadd_rn(S0, __fmaf_rn(g[0], c4[0].y, __fmaf_rn(g[1], c4[1].y, __fmaf_rn(g[2], c4[2].y, __fmul_rn(g[3], c4[3].y)))));
        S1 = __fadd_rn(S1, __fmaf_rn(g[0], c4[0].z, __fmaf_rn(g[1], c4[1].z, __fmaf_rn(g[2], c4[2].z, __fmul_rn(g[3], c4[3].z)))));
        S2 = __fadd_rn(S2, __fmaf_rn(g[0], c4[0].w, __fmaf_rn(g[1], c4[1].w, __fmaf_rn(g[2], c4[2].w, __fmul_rn(g[3], c4[3].w)))));
    }
    for (; h < m; h += G) {
        const uint32_t e = idx ? W.seg[h] : (uint32_t)h;
        const float4 q4 = W.q[e];
        const float u = __fmaf_rn((float)k, dtk, __fadd_rn(__fsub_rn(tS, q4.x), half));
        const float q = __fmaf_rn(__fmul_rn(q4.y, u), u, q4.z);
        if (q <= q4.w) {
            const float4 c4 = W.c[e];
            const float g = exp2f(__fmaf_rn(q, NEG_HALF_LOG2E, c4.x));
            sig = __fadd_rn(sig, g);
            S0 = __fmaf_rn(g, c4.y, S0);
            S1 = __fmaf_rn(g, c4.z, S1);
            S2 = __fmaf_rn(g, c4.w, S2);
        }
    }
}

__device__ __forceinline__ void red_add4(float4* addr, float a, float b, float c, float d) {
    atomicAdd(addr, make_float4(a, b, c, d));
}

// Adjoint, hit-parallel, one piece of a segment: per entry (lane = entry) the sums
// over the piece's samples k in [ka, kb) of w, w u, w u^2 (w = (beta_k + gamma_k . c_l) g,
// u = t - t_c) and of dL/dc_l, turned at once into the local-frame moments A0,
// V = sum w y, P = sum w y y^T and the SH gradients, which are added to the
// Gaussian's accumulator (15 float4 atomics).  Nothing is kept per entry between pieces.
template <int NS>
__device__ __forceinline__ void adjoint_flush(const MarchParams& P, const WS& W, const Ray& r, bool idx, int m,
                                              float tS, float dtk, int ka, int kb, int cam) {
    const int lane = threadIdx.x & 31;
    const float half = __fmul_rn(0.5f, dtk);
    for (int h = lane; h < m; h += 32) {
        const uint32_t e = idx ? W.seg[h] : (uint32_t)h;
        const float4 q4 = W.q[e], c4 = W.c[e];
        const float u0 = __fadd_rn(__fsub_rn(tS, q4.x), half);
        float A0 = 0.f, A1 = 0.f, A2 = 0.f, d0 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll 4
        for (int k = ka; k < kb; k++) {
            const float u = __fmaf_rn((float)k, dtk, u0);
            const float q = __fmaf_rn(__fmul_rn(q4.y, u), u, q4.z);
            if (q <= q4.w) {
                const float4 b = W.bg[k];
                const float g = exp2f(__fmaf_rn(q, NEG_HALF_LOG2E, c4.x));
                const float gp = b.x + b.y * c4.y + b.z * c4.z + b.w * c4.w;
                const float w = gp * g;
                A0 += w;
                A1 += w * u;
                A2 += w * u * u;
                d0 += b.y * g; d1 += b.z * g; d2 += b.w * g;
            }
        }
        if (A0 == 0.f && A1 == 0.f && A2 == 0.f && d0 == 0.f && d1 == 0.f && d2 == 0.f) continue;
        const int64_t p = W.pid[e];
        float yc[3], yd[3];
        local_frame(P.geom, p, r, q4.x, yc, yd);
        const float V0 = A0 * yc[0] + A1 * yd[0], V1 = A0 * yc[1] + A1 * yd[1], V2 = A0 * yc[2] + A1 * yd[2];
        float Pm[6];
        const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
        for (int t = 0; t < 6; t++) {
            const int x = ia[t], y = ib[t];
            Pm[t] = A0 * yc[x] * yc[y] + A1 * (yc[x] * yd[y] + yd[x] * yc[y]) + A2 * yd[x] * yd[y];
        }
        float4* gp = P.grad + 16 * p;
        red_add4(gp + 0, A0, V0, V1, V2);
        red_add4(gp + 1, Pm[0], Pm[1], Pm[2], Pm[3]);
        red_add4(gp + 2, Pm[4], Pm[5], 0.f, 0.f);
        // this camera's share of V, for its own mean gradient M^T V (Eq. 11)
        if (P.vgrad) red_add4(P.vgrad + (size_t)p * P.ncam + cam, V0, V1, V2, 0.f);
        // SH: dL/dK_k = Y_k dL/dc_l where the colour is not clamped
        const float m0 = c4.y > 0.f ? d0 : 0.f, m1 = c4.z > 0.f ? d1 : 0.f, m2 = c4.w > 0.f ? d2 : 0.f;
        const float* Y = W.Y;
#pragma unroll
        for (int jx = 0; jx < 12; jx++) {
            float v[4];
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const int ix = 4 * jx + t, k = ix / 3, ch = ix % 3;
                v[t] = Y[k] * (ch == 0 ? m0 : (ch == 1 ? m1 : m2));
            }
            red_add4(gp + 4 + jx, v[0], v[1], v[2], v[3]);
        }
        if (P.gsg) {
            // lobe j: dc/da = e_j, dc/dlambda = a e_j (mu.d - 1), dc/dmu = a e_j lambda d (unit axis;
            // the projection onto the raw axis happens once per Gaussian)
            for (int jl = 0; jl < P.n_sg; jl++) {
                const float4 ax = __ldg(&P.sgp[2 * (p * P.n_sg + jl)]);
                const float4 am = __ldg(&P.sgp[2 * (p * P.n_sg + jl) + 1]);
                const float cosv = ax.x * r.dx + ax.y * r.dy + ax.z * r.dz;
                const float e = expf(ax.w * (cosv - 1.0f));
                const float sa = (m0 * am.x + m1 * am.y + m2 * am.z) * e;
                const float sl = sa * ax.w;
                float4* gs = P.gsg + 2 * (p * P.n_sg + jl);
                red_add4(gs, sl * r.dx, sl * r.dy, sl * r.dz, sa * (cosv - 1.0f));
                red_add4(gs + 1, m0 * e, m1 * e, m2 * e, 0.f);
            }
        }
    }
    __syncwarp();
}

// ------------------------------------------------------------------ one ray, one warp
// Ray through the centre of pixel (px, py) (pinhole, OpenCV convention); every
// lane holds the same values.
__device__ __forceinline__ Ray make_ray(const rgx_camera& C, int px, int py) {
    Ray r;  // explicitly rounded: both the forward and the adjoint kernel build it
    const float ux = __fdiv_rn(__fsub_rn(__fadd_rn((float)px, 0.5f), C.cx), C.fx);
    const float vy = __fdiv_rn(__fsub_rn(__fadd_rn((float)py, 0.5f), C.cy), C.fy);
    const float dx = __fmaf_rn(C.c2w[0], ux, __fmaf_rn(C.c2w[1], vy, C.c2w[2]));
    const float dy = __fmaf_rn(C.c2w[4], ux, __fmaf_rn(C.c2w[5], vy, C.c2w[6]));
    const float dz = __fmaf_rn(C.c2w[8], ux, __fmaf_rn(C.c2w[9], vy, C.c2w[10]));
    const float inv = __frcp_rn(__fsqrt_rn(dot3_rn(dx, dy, dz, dx, dy, dz)));
    r.dx = __fmul_rn(dx, inv); r.dy = __fmul_rn(dy, inv); r.dz = __fmul_rn(dz, inv);
    r.ox = C.c2w[3]; r.oy = C.c2w[7]; r.oz = C.c2w[11];
    const float tiny = 1e-20f;
    r.ix = __frcp_rn(fabsf(r.dx) > tiny ? r.dx : copysignf(tiny, r.dx));
    r.iy = __frcp_rn(fabsf(r.dy) > tiny ? r.dy : copysignf(tiny, r.dy));
    r.iz = __frcp_rn(fabsf(r.dz) > tiny ? r.dz : copysignf(tiny, r.dz));
    return r;
}

// t_f: the camera's t_far, or (t_far <= 0) the exit of the scene box (t_n when
// the ray misses the box).
__device__ __forceinline__ float far_bound(const float4& lo, const float4& hi, const rgx_camera& C, const Ray& r) {
    const float tn = C.t_near;
    float tf = C.t_far;
    if (!(tf > 0.0f)) {
        float tentry;
        const bool in = box_overlap(lo, hi, r, -INFINITY, INFINITY, tentry);
        const float fx = r.ix >= 0.0f ? hi.x : lo.x, fy = r.iy >= 0.0f ? hi.y : lo.y, fz = r.iz >= 0.0f ? hi.z : lo.z;
        const float texit = fminf(fminf((fx - r.ox) * r.ix, (fy - r.oy) * r.iy), (fz - r.oz) * r.iz);
        tf = (in && texit > tn) ? texit : tn;
    }
    return tf;
}

template <int NS, bool BWD>
__device__ void march_ray(const MarchParams& P, const WS& W, int64_t ray, int cam, const rgx_camera& C, int px, int py,
                          const float4& root_lo, const float4& root_hi, const float4& up, const float4& st,
                          const uint4& st2, Counters& cnt, bool& whole, uint32_t& tape_base,
                          uint32_t& tape_left, uint32_t& pt_base, uint32_t& pt_left, float4& o_rgba,
                          float4& o_state, uint4& o_tape, int& o_nrec, float& th_guess, bool& carry_dense) {
    const int lane = threadIdx.x & 31;
    const int k = lane % NS;
    const int cap = P.hit_cap;
    const Ray r = make_ray(C, px, py);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, Cf0 = 0.f, Cf1 = 0.f, Cf2 = 0.f, Tf = 1.f, dTcoef = 0.f;
    bool fwd_whole = false;  // adjoint: the forward marched this ray with a whole-ray first window
    if (BWD) {
        if (up.x == 0.0f && up.y == 0.0f && up.z == 0.0f && up.w == 0.0f) return;
        a0 = up.x; a1 = up.y; a2 = up.z;
        Cf0 = st.x; Cf1 = st.y; Cf2 = st.z; Tf = fabsf(st.w);
        fwd_whole = signbit(st.w);
        dTcoef = (a0 * P.bg0 + a1 * P.bg1 + a2 * P.bg2 - up.w) * Tf;
    }
    // ---- bounds: t_n, and t_f = camera t_far or the exit of the scene box
    const float tn = C.t_near;
    const float tf = far_bound(root_lo, root_hi, C, r);
    {
        float Y[16];
        sh_basis16(r.dx, r.dy, r.dz, Y);
        __syncwarp();
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < 16; i++) W.Y[i] = Y[i];
        }
        __syncwarp();
    }

    const bool skip = (P.flags & RGX_SKIP) != 0;
    const bool uniform = (P.flags & RGX_ADAPTIVE) == 0;
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    float tS = tn;
    int j = 0;  // lattice index in uniform mode
    int nrec = 0;
    int nL = 0;
    float w_lo = 1.0f, w_hi = 0.0f;  // current window (empty)
    bool used_whole = false;  // the ray used a first window (recorded in the sign bit of its state)
    float first_hi = 0.0f;    // that window's end (recorded for the adjoint's taped replay)
    bool dense = false;  // the last evaluated segment overflowed the list: go straight to chunks
    int kseg = 0;        // chunked segments so far (their sums records are kept in this order)
    // adjoint: the forward of this state recorded the sums of its chunked segments
    const bool csum_ok = BWD && P.csums != nullptr && P.csum_slots > 0 && st2.z == P.tape_tag;
    uint32_t tape_off = 0;
    int tape_cnt = -1;  // forward: where this ray's first-window list went on the tape (-1: not taped)
    float th_start = 0.0f;  // ClosestHit(t_n) of a ray without a whole-ray window (kept in its state)
    bool query = false;     // ClosestHit(t_n) still to be found by a nearest-hit traversal
    float wlen = 4.0f * (float)NS * (uniform ? P.dt : P.dt_max);
    if (P.n > 0 && tf > tn && skip) {
        // One window over the whole ray [t_n, t_f): when every chord fits in the
        // list, ClosestHit(t_n) is its smallest max(t_in, t_n) (a chord outside the
        // window would start later) and every later segment reuses the window.
        // After an overflow the work item's remaining rays use the nearest-hit
        // traversal.
        float th = tf;
        bool have = false;
        // adjoint: the forward's list of this window, from the tape when it is there
        const bool taped = BWD && fwd_whole && P.tape_cap > 0 && st2.z == P.tape_tag && (int)st2.y >= 0 &&
                           (int)st2.y <= cap;
        if (taped) {
            nL = (int)st2.y;
            if (lane == 0) cnt.windows++;
            const float4* tq = P.tape + st2.x;
            const float4* tc = tq + P.tape_cap;
            const float4* tx = tc + P.tape_cap;
            for (int e = lane; e < nL; e += 32) {
                const float4 x = tx[e];
                W.q[e] = tq[e];
                W.c[e] = tc[e];
                W.tio[e] = make_float2(x.x, x.y);
                W.pid[e] = __float_as_uint(x.z);
            }
            __syncwarp();
            have = true;
            used_whole = true;
            w_lo = tn;
            w_hi = __uint_as_float(st2.w);
        } else if (BWD ? fwd_whole : whole) {
            nL = 0;
            if (lane == 0) cnt.windows++;
            // with RGX_LOWER_FIRST the window's end is lowered while its chords overflow the list, as
            // long as it keeps one segment of the smallest size past its first chord (else the first
            // segment is chunked anyway and a nearest-hit query is cheaper)
            float tb = tf;
            const float seg_min = __fmul_rn((float)NS, uniform ? P.dt : fminf(P.dt_min, P.dt_max));
            const bool lower = (P.flags & RGX_LOWER_FIRST) != 0;  // else the whole ray or nothing
            if (w_collect<BWD>(P, W, r, tn, tb, lower ? tn : tf, cap, nL, false, NoChunk(), cnt, lower ? seg_min : 0.0f) == 0) {
                have = true;
                used_whole = true;
                w_lo = tn;
                w_hi = tb;
                if (!BWD && P.tape_cap > 0) {
                    // tape the finished list (entries in list order) for the adjoint, in the
                    // warp's current chunk of the tape (a new chunk when it is used up)
                    if ((uint32_t)nL > tape_left && tape_base != TAPE_FULL) {
                        // A warp stops reserving once one reservation has failed, and never adds to a
                        // counter already at the capacity: the counter then stays below
                        // tape_cap + (resident warps) x TAPE_CHUNK < 2^32 (tape_cap < 2^31), so it
                        // cannot wrap round and hand out a chunk that another ray's list occupies.
                        const uint32_t want = max((uint32_t)TAPE_CHUNK, (uint32_t)nL);
                        uint32_t base = TAPE_FULL;
                        if (lane == 0 && *(volatile uint32_t*)P.tape_n < P.tape_cap) base = atomicAdd(P.tape_n, want);
                        base = __shfl_sync(FULLMASK, base, 0);
                        if (base != TAPE_FULL && (uint64_t)base + want <= (uint64_t)P.tape_cap) {
                            tape_base = base;
                            tape_left = want;
                        } else {
                            tape_base = TAPE_FULL;
                            tape_left = 0;
                        }
                    }
                    if ((uint32_t)nL <= tape_left) {
                        float4* tq = P.tape + tape_base;
                        float4* tc = tq + P.tape_cap;
                        float4* tx = tc + P.tape_cap;
                        for (int e = lane; e < nL; e += 32) {
                            const float2 io = W.tio[e];
                            tq[e] = W.q[e];
                            tc[e] = W.c[e];
                            tx[e] = make_float4(io.x, io.y, __uint_as_float(W.pid[e]), 0.f);
                        }
                        tape_off = tape_base;
                        tape_cnt = nL;
                        tape_base += (uint32_t)nL;
                        tape_left -= (uint32_t)nL;
                    }
                }
            } else {
                whole = false;
                nL = 0;
            }
        }
        if (have) {
            first_hi = w_hi;
            float m = INFINITY;
            for (int e = lane; e < nL; e += 32) m = fminf(m, fmaxf(W.tio[e].x, tn));
            m = warp_min(m);
            // no chord starts inside a window that had to be lowered: look beyond it
            if (m < INFINITY) th = fminf(m, tf);
            else if (w_hi >= tf) th = tf;
            else query = true;
        } else if (BWD && st2.y == 0xffffffffu) {
            // the forward's ClosestHit(t_n) of this ray, kept in its state: no query again
            th = __uint_as_float(st2.x);
        } else {
            query = true;
        }
        if (query) th = w_closest_guess(P, W, r, tn, tf, th_guess, cnt);  // the one call site at a ray's start
        if (!have) th_start = th;
        if (th < tf) th_guess = th;
        if (uniform) {
            const int jj = (int)floorf((th - tn) / P.dt) - 1;
            j = jj > 0 ? jj : 0;
            tS = __fmaf_rn((float)j, P.dt, tn);
        } else {
            tS = th;
        }
    }
    // A ray that does not start with a whole-ray window starts in chunked mode when the
    // previous ray of its work item ended in a dense stretch (the forward records this in
    // the ray's state, so that the adjoint starts the same way)
    const bool start_dense = !used_whole && (BWD ? (!fwd_whole && st2.w == 1u) : carry_dense);
    dense = start_dense;
    const float minstep = uniform ? P.dt : (float)NS * fminf(P.dt_min, P.dt_max);
    // max_segments = 0: the ray's own bound, (t_f - t_n) / minstep + 8, but never above
    // RGX_SEGMENT_CEILING, so that a scene box vast next to the step cannot keep a warp busy
    // for minutes; a ray stopped there sets RGX_ERR_ITER_LIMIT like one stopped by max_segments
    const int iter_cap = P.max_segments > 0
        ? P.max_segments
        : (int)fminf((tf - tn) / minstep + 8.0f, (float)RGX_SEGMENT_CEILING);
    int iters = 0;
    while (P.n > 0 && tS < tf && T > P.t_eps) {
        if (iters >= iter_cap) {
            if (lane == 0) atomicOr(P.status, (unsigned)RGX_ERR_ITER_LIMIT);
            break;
        }
        iters++;
        // ---- segment size: uniform dt, or Eq. 5
        float dtk;
        if (uniform) {
            dtk = P.dt;
        } else {
            const float base = fmaxf(__fdiv_rn(tS, P.beta), P.dt_min);
            dtk = fminf(__fmul_rn(base, rcbrtf(T)), P.dt_max);
        }
        const float te = uniform ? __fmaf_rn((float)(j + NS), P.dt, tn) : __fadd_rn(tS, __fmul_rn((float)NS, dtk));
        const float tcut = fminf(te, tf);
        // ---- window of chords covering [tS, tcut)
        bool chunked = false;
        bool spill_ok = BWD && P.spill != nullptr;  // adjoint: chunks kept in this warp's scratch
        float4* wspill = BWD && P.spill
            ? P.spill + ((size_t)blockIdx.x * WARPS + (threadIdx.x >> 5)) * SPILL_CAP * 3 : nullptr;
        if (!(tS >= w_lo && tcut <= w_hi) && dense) {
            // dense stretch: a window would overflow again, collect this segment in chunks
            chunked = true;
            nL = 0; w_lo = 1.0f; w_hi = 0.0f;
        } else if (!(tS >= w_lo && tcut <= w_hi)) {
            const float need = te - tS;
            float len = fmaxf(wlen, need);
            while (true) {
                float hi = (len <= need) ? tcut : fminf(tS + len, tf);
                hi = fmaxf(hi, tcut);
                nL = 0;
                if (lane == 0) cnt.windows++;
                const int rc = w_collect<BWD>(P, W, r, tS, hi, hi, cap, nL, false, NoChunk(), cnt);
                if (rc == 0) {
                    w_lo = tS; w_hi = hi;
                    wlen = (nL * 4 <= cap) ? 2.0f * len : len;
                    break;
                }
                if (len <= need || rc == 2) { chunked = true; break; }
                len = fmaxf(0.25f * len, need);
                wlen = len;
            }
            if (chunked) { nL = 0; w_lo = 1.0f; w_hi = 0.0f; }
        }
        // ---- the segment's hits and per-sample sums
        float sig = 0.f, S0 = 0.f, S1 = 0.f, S2 = 0.f;
        int nexact = 0;
        float4* seg_rec = nullptr;  // this chunked segment's sums record
        uint32_t pid_off = TAPE_FULL;  // adjoint: where the segment's chord indices start on the index tape
        if (!chunked) {
            const uint32_t lt = lanemask_lt();
            // four 32-entry slices per step: all loads before the ballots
            for (int b = 0; b < nL; b += 128) {
                bool in[4];
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const int e = b + 32 * i + lane;
                    in[i] = false;
                    if (e < nL) { const float2 io = W.tio[e]; in[i] = io.x < tcut && io.y > tS; }
                }
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const uint32_t bb = __ballot_sync(FULLMASK, in[i]);
                    if (in[i]) W.seg[nexact + __popc(bb & lt)] = (uint32_t)(b + 32 * i + lane);
                    nexact += __popc(bb);
                }
            }
            __syncwarp();
            if (nexact) eval_entries<NS>(W, true, nexact, tS, dtk, true, sig, S0, S1, S2);
        } else if (csum_ok && (uint32_t)kseg < P.csum_slots) {
            // adjoint: the forward's sums of this chunked segment, as it composited them -- group 0
            // holds them and the other lane groups zero, so the butterfly below reproduces them
            // exactly -- instead of a traversal and every sample evaluated a second time; the
            // gradients' pass traverses the segment once
            const float4* rec = P.csums + ((size_t)ray * P.csum_slots + kseg) * (NS + 1);
            const float4 v = lane < NS ? rec[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
            sig = v.x; S0 = v.y; S1 = v.z; S2 = v.w;
            const float4 hd = rec[NS];
            nexact = __float_as_int(hd.x);
            // the segment's chords by index, when the forward could tape them
            if (P.ptape && __float_as_uint(hd.z) != 0u) pid_off = __float_as_uint(hd.y);
            spill_ok = false;
            nL = 0;
            kseg++;
        } else {
            if (!BWD && P.csums && (uint32_t)kseg < P.csum_slots)
                seg_rec = P.csums + ((size_t)ray * P.csum_slots + kseg) * (NS + 1);
            kseg++;
            // forward: the chords of a recorded segment also go to the index tape, contiguously in
            // this warp's block (a new block when little room is left; none when the tape is full)
            bool pt_ok = false;
            if (!BWD && seg_rec && P.ptape) {
                if (pt_left < PTAPE_MIN_FREE && pt_base != TAPE_FULL) {
                    uint32_t base = TAPE_FULL;
                    if (lane == 0 && *(volatile uint32_t*)P.ptape_n < P.ptape_cap)
                        base = atomicAdd(P.ptape_n, (uint32_t)PTAPE_BLOCK);
                    base = __shfl_sync(FULLMASK, base, 0);
                    if (base != TAPE_FULL && (uint64_t)base + PTAPE_BLOCK <= (uint64_t)P.ptape_cap) {
                        pt_base = base;
                        pt_left = PTAPE_BLOCK;
                    } else {
                        pt_base = TAPE_FULL;
                        pt_left = 0;
                    }
                }
                pt_ok = pt_base != TAPE_FULL && pt_left > 0;
            }
            int tot = 0;
            auto onfull = [&](int m) {
                eval_entries<NS>(W, false, m, tS, dtk, true, sig, S0, S1, S2);
                if (!BWD && pt_ok) {
                    if ((uint32_t)(tot + m) <= pt_left) {
                        for (int e = lane; e < m; e += 32) {
                            const float4 c = W.c[e];
                            P.ptape[(size_t)pt_base + (uint32_t)tot + e] =
                                make_uint4(W.pid[e], __float_as_uint(c.y), __float_as_uint(c.z), __float_as_uint(c.w));
                        }
                    } else {
                        pt_ok = false;
                    }
                }
                if (BWD && spill_ok) {
                    // keep the chunk for the adjoint pass (no second traversal)
                    if (tot + m <= SPILL_CAP) {
                        for (int e = lane; e < m; e += 32) {
                            float4* d = wspill + 3 * (size_t)(tot + e);
                            d[0] = W.q[e];
                            d[1] = W.c[e];
                            d[2] = make_float4(__uint_as_float(W.pid[e]), 0.f, 0.f, 0.f);
                        }
                    } else {
                        spill_ok = false;
                    }
                }
                tot += m;
                __syncwarp();
            };
            nL = 0;
            float tb_c = tcut;
            w_collect<BWD>(P, W, r, tS, tb_c, tcut, cap, nL, true, onfull, cnt);
            if (nL) onfull(nL);
            nexact = tot;
            nL = 0;
            if (seg_rec && lane == 0)
                seg_rec[NS] = make_float4(__int_as_float(tot), __uint_as_float(pt_ok ? pt_base : 0u),
                                          __uint_as_float(pt_ok ? 1u : 0u), 0.f);
            if (!BWD && pt_ok) {
                pt_base += (uint32_t)tot;
                pt_left -= (uint32_t)tot;
            }
        }
        // chunks stay in use while segments keep more than half a list of hits
        dense = chunked && 2 * nexact > cap;
        if (nexact == 0) {
            if (lane == 0) cnt.skips++;
            if (skip) {
                float cand = INFINITY;
                for (int e = lane; e < nL; e += 32) {
                    const float2 io = W.tio[e];
                    if (io.y > te && io.x < tf) cand = fminf(cand, fmaxf(io.x, te));
                }
                cand = warp_min(cand);
                float th;
                if (cand < INFINITY) th = cand;
                else if (w_hi >= tf && w_lo <= w_hi) th = tf;
                else th = w_closest(P, W, r, te, tf, cnt);
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
        if (lane == 0) {
            cnt.segs++;
            cnt.hits += nexact;
            cnt.evals += nexact * NS;
            if (!BWD && P.sched && nrec < P.sched_cap) P.sched[ray * P.sched_cap + nrec] = make_float2(tS, dtk);
        }
        nrec++;
        // ---- combine the lane groups (butterfly: every lane ends with the same sums)
#pragma unroll
        for (int off = NS; off < 32; off <<= 1) {
            sig = __fadd_rn(sig, __shfl_xor_sync(FULLMASK, sig, off));
            S0 = __fadd_rn(S0, __shfl_xor_sync(FULLMASK, S0, off));
            S1 = __fadd_rn(S1, __shfl_xor_sync(FULLMASK, S1, off));
            S2 = __fadd_rn(S2, __shfl_xor_sync(FULLMASK, S2, off));
        }
        if (!BWD && seg_rec && lane < NS) seg_rec[lane] = make_float4(sig, S0, S1, S2);
        // ---- front-to-back compositing of the N_S samples (Eq. 3)
        const float t0 = __fadd_rn(tS, __fmul_rn(0.5f, dtk));
        const float tk = __fmaf_rn((float)k, dtk, t0);
        const bool valid = tk < tf && sig > 0.0f;
        const float x = valid ? __fmul_rn(sig, dtk) : 0.0f;
        const float e = valid ? expf(-x) : 1.0f;
        const float alpha = valid ? -expm1f(-x) : 0.0f;
        const float inv = valid ? __fdiv_rn(1.0f, sig) : 0.0f;
        const float c0 = __fmul_rn(S0, inv), c1 = __fmul_rn(S1, inv), c2 = __fmul_rn(S2, inv);
        float pinc = e;  // inclusive product of e over samples 0..k
#pragma unroll
        for (int d = 1; d < NS; d <<= 1) {
            const float v = __shfl_up_sync(FULLMASK, pinc, d, NS);
            if (k >= d) pinc = __fmul_rn(pinc, v);
        }
        float pexc = __shfl_up_sync(FULLMASK, pinc, 1, NS);
        if (k == 0) pexc = 1.0f;
        const float Tk = __fmul_rn(T, pexc);
        const float w = __fmul_rn(Tk, alpha);
        const float k0 = __fmul_rn(w, c0), k1 = __fmul_rn(w, c1), k2 = __fmul_rn(w, c2);
        float s0 = k0, s1 = k1, s2 = k2;
#pragma unroll
        for (int d = NS / 2; d >= 1; d >>= 1) {
            s0 = __fadd_rn(s0, __shfl_xor_sync(FULLMASK, s0, d, NS));
            s1 = __fadd_rn(s1, __shfl_xor_sync(FULLMASK, s1, d, NS));
            s2 = __fadd_rn(s2, __shfl_xor_sync(FULLMASK, s2, d, NS));
        }
        const float Tend = __fmul_rn(T, __shfl_sync(FULLMASK, pinc, NS - 1, NS));
        if (BWD) {
            // C_<=k = C + inclusive prefix of the contributions; T_{k+1} = T_k e_k
            float p0 = k0, p1 = k1, p2 = k2;
#pragma unroll
            for (int d = 1; d < NS; d <<= 1) {
                const float v0 = __shfl_up_sync(FULLMASK, p0, d, NS);
                const float v1 = __shfl_up_sync(FULLMASK, p1, d, NS);
                const float v2 = __shfl_up_sync(FULLMASK, p2, d, NS);
                if (k >= d) { p0 += v0; p1 += v1; p2 += v2; }
            }
            const float Tn = Tk * e;
            float ds = a0 * (Tn * c0 - (Cf0 - (C0 + p0))) + a1 * (Tn * c1 - (Cf1 - (C1 + p1))) +
                       a2 * (Tn * c2 - (Cf2 - (C2 + p2)));
            ds = dtk * (ds - dTcoef);
            const float g0 = a0 * w * inv, g1 = a1 * w * inv, g2 = a2 * w * inv;
            const float beta = ds - (g0 * c0 + g1 * c1 + g2 * c2);
            if (lane < NS) W.bg[k] = valid ? make_float4(beta, g0, g1, g2) : make_float4(0.f, 0.f, 0.f, 0.f);
            __syncwarp();
            if (!chunked) {
                adjoint_flush<NS>(P, W, r, true, nexact, tS, dtk, 0, NS, cam);
                __syncwarp();
            } else if (spill_ok) {
                // the segment's chunks, kept by the first pass, in the same order
                for (int b = 0; b < nexact; b += cap) {
                    const int m = min(cap, nexact - b);
                    for (int e = lane; e < m; e += 32) {
                        const float4* d = wspill + 3 * (size_t)(b + e);
                        W.q[e] = d[0];
                        W.c[e] = d[1];
                        W.pid[e] = __float_as_uint(d[2].x);
                    }
                    __syncwarp();
                    adjoint_flush<NS>(P, W, r, false, m, tS, dtk, 0, NS, cam);
                }
            } else if (pid_off != TAPE_FULL) {
                // the chords the forward taped by index, in its order: solved and coloured again
                // (the same rounded arithmetic) without a traversal
                for (int b = 0; b < nexact; b += cap) {
                    const int m = min(cap, nexact - b);
                    for (int e = lane; e < m; e += 32) {
                        // the index and the forward's colour bits: no SH record gathered again
                        const uint4 x = P.ptape[(size_t)pid_off + (uint32_t)(b + e)];
                        const Chord ch = chord_of(P.geom, x.x, r);
                        W.q[e] = make_float4(ch.tc, ch.a, ch.qmin, ch.Qe);
                        W.c[e] = make_float4(ch.L, __uint_as_float(x.y), __uint_as_float(x.z), __uint_as_float(x.w));
                        W.pid[e] = x.x;
                    }
                    __syncwarp();
                    adjoint_flush<NS>(P, W, r, false, m, tS, dtk, 0, NS, cam);
                }
            } else {
                auto onfull2 = [&](int m) {
                    adjoint_flush<NS>(P, W, r, false, m, tS, dtk, 0, NS, cam);
                };
                nL = 0;
                float tb_c2 = tcut;
                w_collect<BWD>(P, W, r, tS, tb_c2, tcut, cap, nL, true, onfull2, cnt);
                if (nL) onfull2(nL);
                nL = 0;
            }
        }
        C0 = __fadd_rn(C0, s0);
        C1 = __fadd_rn(C1, s1);
        C2 = __fadd_rn(C2, s2);
        T = Tend;
        if (uniform) { j += NS; tS = __fmaf_rn((float)j, P.dt, tn); } else tS = te;
    }
    if (BWD) {
        if (lane == 0 && T != Tf) atomicOr(P.status, (unsigned)RGX_ERR_REPLAY);
    } else {
        o_rgba = make_float4(C0 + T * P.bg0, C1 + T * P.bg1, C2 + T * P.bg2, 1.0f - T);
        // the sign bit of T (>= 0) records the first-window path for the adjoint's replay
        o_state = make_float4(C0, C1, C2, used_whole ? -T : T);
        // a ray with a whole-ray window keeps where its list is on the tape and the window's end; one
        // without keeps its ClosestHit(t_n) and whether it started in a dense stretch
        o_tape = make_uint4(used_whole ? tape_off : __float_as_uint(th_start), (uint32_t)tape_cnt, P.tape_tag,
                            used_whole ? __float_as_uint(first_hi) : (start_dense ? 1u : 0u));
        carry_dense = dense;
        o_nrec = nrec;
    }
}

// ------------------------------------------------------------------ kernel
__device__ __forceinline__ uint32_t tiles_of(const rgx_camera& c, bool ztiles, int tw, int th) {
    if (!ztiles) return (uint32_t)(((int64_t)c.width * c.height + 31) / 32);
    const uint32_t ntx = (c.width + tw - 1) / tw, nty = (c.height + th - 1) / th;
    return ((ntx + 7) / 8) * ((nty + 7) / 8) * 64u;
}

// Pixel of lane `l` of local tile `lt` of camera `cam`.
__device__ __forceinline__ bool tile_pixel(const rgx_camera& cam, uint32_t lt, int l, bool zt, int tw, int th,
                                           int& px, int& py) {
    if (!zt) {
        const int64_t pix = (int64_t)lt * 32 + l;
        px = (int)(pix % cam.width);
        py = (int)(pix / cam.width);
        return pix < (int64_t)cam.width * cam.height;
    }
    const uint32_t ntx = (cam.width + tw - 1) / tw;
    const uint32_t nsx = (ntx + 7) / 8;
    const uint32_t sblk = lt >> 6, w = lt & 63u;
    const uint32_t wx = (w & 1u) | ((w >> 1) & 2u) | ((w >> 2) & 4u);
    const uint32_t wy = ((w >> 1) & 1u) | ((w >> 2) & 2u) | ((w >> 3) & 4u);
    const uint32_t tx = (sblk % nsx) * 8 + wx, ty = (sblk / nsx) * 8 + wy;
    px = (int)(tx * tw + l % tw);
    py = (int)(ty * th + l / tw);
    return px < cam.width && py < cam.height;
}

// ------------------------------------------------------------------ tile cut
// Conservative view cone of the pixel rectangle [pxa, pxb] x [pya, pyb]: four
// planes through the camera centre, each spanned by two corner rays of the
// rectangle's outer pixel boundaries (half a pixel beyond the outermost ray),
// oriented so that the centre ray is inside.  Any invertible c2w rotation part.
struct Frustum {
    float4 pl[4];  // (n, -n.o): a point x is inside a plane when n.x - n.o >= 0
};

__device__ __forceinline__ float3 cam_dir(const rgx_camera& C, float u, float v) {
    return make_float3(__fmaf_rn(C.c2w[0], u, __fmaf_rn(C.c2w[1], v, C.c2w[2])),
                       __fmaf_rn(C.c2w[4], u, __fmaf_rn(C.c2w[5], v, C.c2w[6])),
                       __fmaf_rn(C.c2w[8], u, __fmaf_rn(C.c2w[9], v, C.c2w[10])));
}

__device__ Frustum tile_frustum(const rgx_camera& C, int pxa, int pya, int pxb, int pyb) {
    // explicitly rounded: both the forward and the adjoint kernel build the tile's cut from it
    const float u0 = __fdiv_rn(__fsub_rn((float)pxa, C.cx), C.fx);
    const float u1 = __fdiv_rn(__fsub_rn(__fadd_rn((float)pxb, 1.0f), C.cx), C.fx);
    const float v0 = __fdiv_rn(__fsub_rn((float)pya, C.cy), C.fy);
    const float v1 = __fdiv_rn(__fsub_rn(__fadd_rn((float)pyb, 1.0f), C.cy), C.fy);
    const float3 d00 = cam_dir(C, u0, v0), d10 = cam_dir(C, u1, v0), d01 = cam_dir(C, u0, v1),
                 d11 = cam_dir(C, u1, v1);
    const float3 dc = cam_dir(C, __fmul_rn(0.5f, __fadd_rn(u0, u1)), __fmul_rn(0.5f, __fadd_rn(v0, v1)));
    const float ox = C.c2w[3], oy = C.c2w[7], oz = C.c2w[11];
    const float3 ea[4] = {d00, d10, d00, d01}, eb[4] = {d01, d11, d10, d11};
    Frustum F;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float nx = __fmaf_rn(ea[i].y, eb[i].z, -__fmul_rn(ea[i].z, eb[i].y));
        float ny = __fmaf_rn(ea[i].z, eb[i].x, -__fmul_rn(ea[i].x, eb[i].z));
        float nz = __fmaf_rn(ea[i].x, eb[i].y, -__fmul_rn(ea[i].y, eb[i].x));
        if (dot3_rn(nx, ny, nz, dc.x, dc.y, dc.z) < 0.0f) { nx = -nx; ny = -ny; nz = -nz; }
        F.pl[i] = make_float4(nx, ny, nz, -dot3_rn(nx, ny, nz, ox, oy, oz));
    }
    return F;
}

// Box entirely on the outer side of one plane (beyond a rounding allowance).
// Empty (inverted) boxes give inf / NaN sums and are kept; the ray test drops them.
__device__ __forceinline__ bool box_outside(const Frustum& F, float4 lo, float4 hi) {
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const float4 p = F.pl[i];
        const float x = p.x > 0.0f ? hi.x : lo.x, y = p.y > 0.0f ? hi.y : lo.y, z = p.z > 0.0f ? hi.z : lo.z;
        const float v = __fadd_rn(dot3_rn(p.x, p.y, p.z, x, y, z), p.w);
        const float mag = __fadd_rn(__fadd_rn(fabsf(__fmul_rn(p.x, x)), fabsf(__fmul_rn(p.y, y))),
                                    __fadd_rn(fabsf(__fmul_rn(p.z, z)), fabsf(p.w)));
        if (v < -1e-5f * mag) return true;
    }
    return false;
}

// A 4-wide child record whose box lies entirely outside the view cone.
__device__ __forceinline__ bool record_outside(const Frustum& F, uint4 v) {
    float4 lo, hi;
    child_of(v, lo, hi);
    return box_outside(F, lo, hi);
}

// The tile's BVH cut: a set of at most CUT (= 32, one per lane) child records
// whose subtrees hold every leaf whose bounds meet the view cone.  Starts from
// the root's 4-wide record and replaces internal records by their children
// inside the cone, level by level, while the set stays within CUT; records
// outside the cone are dropped.  Every traversal of the tile's rays starts from it.
#define CUT_LEVELS 48
static_assert(CUT == 32, "one cut record per lane");
__device__ void build_cut(const MarchParams& P, const WS& W, const Frustum& F, Counters& cnt) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    {
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        bool keep = false;
        if (lane < 4) {
            v = __ldg(P.nodew + lane);
            keep = !record_outside(F, v);
        }
        const uint32_t b = __ballot_sync(FULLMASK, keep);
        if (keep) W.cut[__popc(b & lt)] = v;
        if (lane == 0) *W.ncut = __popc(b);
        __syncwarp();
    }
    int nc = *W.ncut;
    for (int it = 0; it < CUT_LEVELS; it++) {
        const bool have = lane < nc;
        const uint4 mine = have ? W.cut[lane] : make_uint4(0u, 0u, 0u, LEAF_BIT);
        const bool internal = have && !(mine.w & LEAF_BIT);
        uint4 c[4];
        bool k[4];
        int kept = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) { c[j] = make_uint4(0u, 0u, 0u, 0u); k[j] = false; }
        if (internal) {
            cnt.visits++;
#pragma unroll
            for (int j = 0; j < 4; j++) c[j] = __ldg(P.nodew + 4 * (size_t)mine.w + j);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                k[j] = !record_outside(F, c[j]);
                kept += k[j] ? 1 : 0;
            }
        }
        // a record grows the set by add = (children kept) - 1; shrinking ones always
        // expand, growing ones while the running total of growth (in record order) fits
        const int add = internal ? kept - 1 : 0;
        uint32_t gsum;
        const int pre = (int)warp_excl_scan(add > 0 ? (uint32_t)add : 0u, gsum) + (add > 0 ? add : 0);
        const bool expand = internal && (add <= 0 || nc + pre <= CUT);
        if (!__any_sync(FULLMASK, expand)) break;
        const int mcount = expand ? kept : (have ? 1 : 0);
        uint32_t total;
        int off = (int)warp_excl_scan((uint32_t)mcount, total);
        __syncwarp();
        if (expand) {
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (k[j]) W.cut[off++] = c[j];
        } else if (have) {
            W.cut[off] = mine;
        }
        nc = (int)total;
        __syncwarp();
    }
    if (lane == 0) *W.ncut = nc;
    __syncwarp();
}

template <int NS, bool BWD>
__device__ __forceinline__ void march_kernel(const MarchParams& P) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* s_tiles = (uint32_t*)smem;         // [ncam+1] work-item prefix
    uint32_t* s_pix = s_tiles + (P.ncam + 1);    // [ncam+1] pixel prefix
    uint32_t* s_shift = s_pix + (P.ncam + 1);    // [ncam+1] per camera: a work item is 32 >> shift rays
    const size_t head = ((size_t)(3 * (P.ncam + 1)) * 4 + 15) & ~(size_t)15;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const WS W = carve((char*)smem + head + (size_t)warp * warp_bytes(P.hit_cap, BWD), P.hit_cap, BWD);
    const bool zt = (P.flags & RGX_ZTILES) != 0;
    if (threadIdx.x == 0) {
        uint32_t tsum = 0, psum = 0;
        for (int c = 0; c < P.ncam; c++) {
            // a small view is split into smaller work items until it has 16 per SM (about
            // two per resident warp); the split depends on the view and the device alone,
            // so a view renders the same in any batch
            const uint32_t rays = (uint32_t)(P.cams[c].width * P.cams[c].height);
            uint32_t sh = 0;
            while (sh < 5 && rays / (32u >> sh) < P.min_items) sh++;
            s_shift[c] = sh;
            s_tiles[c] = tsum; s_pix[c] = psum;
            tsum += tiles_of(P.cams[c], zt, P.tile_w, P.tile_h) << sh;
            psum += rays;
        }
        s_tiles[P.ncam] = tsum; s_pix[P.ncam] = psum;
    }
    __syncthreads();
    const uint32_t total = s_tiles[P.ncam];
    // the scene box (t_f of every ray), in registers for the whole launch
    const float4 root_lo = make_float4(P.root[0], P.root[1], P.root[2], 0.f);
    const float4 root_hi = make_float4(P.root[3], P.root[4], P.root[5], 0.f);
    uint32_t tape_base = 0, tape_left = 0;  // forward: this warp's current chunk of the tape
    uint32_t pt_base = 0, pt_left = 0;      // forward: this warp's current block of the index tape
    while (true) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(P.queue, 1u);
        t = __shfl_sync(FULLMASK, t, 0);
        if (t >= total) break;
        int lo = 0, hi = P.ncam;
        while (hi - lo > 1) { const int mid = (lo + hi) >> 1; if (s_tiles[mid] <= t) lo = mid; else hi = mid; }
        const int c = lo;
        const rgx_camera cam = P.cams[c];  // in registers for the tile's 32 rays
        const uint32_t item = t - s_tiles[c], sh = s_shift[c];
        const uint32_t lt = item >> sh;                        // the tile
        const int l0 = (int)(item & ((1u << sh) - 1u)) << (5 - sh);
        const int l1 = l0 + (32 >> sh);                        // its rays [l0, l1)
        const bool mine = lane >= l0 && lane < l1;
        Counters cnt = {0, 0, 0, 0, 0, 0, 0};
        float4 my_rgba = make_float4(0.f, 0.f, 0.f, 0.f), my_state = my_rgba;
        uint4 my_tape = make_uint4(0u, 0xffffffffu, 0u, 0u);
        int my_nrec = 0;
        bool work = P.n > 0;
        // adjoint: lane l holds the upstream gradient and forward state of the tile's ray l
        float4 my_up = make_float4(0.f, 0.f, 0.f, 0.f), my_st = my_up;
        uint4 my_st2 = make_uint4(0u, 0xffffffffu, 0u, 0u);
        if (BWD && work) {
            // the adjoint skips tiles whose rays all have a zero upstream gradient
            int px, py;
            bool nz = false;
            if (mine && tile_pixel(cam, lt, lane, zt, P.tile_w, P.tile_h, px, py)) {
                const int64_t ray = (int64_t)s_pix[c] + (int64_t)py * cam.width + px;
                my_up = P.d_rgba[ray];
                my_st = P.state[2 * ray];
                my_st2 = reinterpret_cast<const uint4*>(P.state)[2 * ray + 1];
                nz = my_up.x != 0.0f || my_up.y != 0.0f || my_up.z != 0.0f || my_up.w != 0.0f;
            }
            work = __any_sync(FULLMASK, nz);
        }
        if (work) {
            int pxa, pya, pxb, pyb;
            if (zt) {
                tile_pixel(cam, lt, 0, zt, P.tile_w, P.tile_h, pxa, pya);
                pxb = pxa + P.tile_w - 1;
                pyb = pya + P.tile_h - 1;
            } else {
                const int64_t p0 = (int64_t)lt * 32, p1 = p0 + 31;
                pya = (int)(p0 / cam.width);
                pyb = (int)(p1 / cam.width);
                if (pya == pyb) { pxa = (int)(p0 % cam.width); pxb = (int)(p1 % cam.width); }
                else { pxa = 0; pxb = cam.width - 1; }
            }
            build_cut(P, W, tile_frustum(cam, pxa, pya, pxb, pyb), cnt);
        }
        bool whole = true;  // whole-ray first windows, until one overflows in this work item
        float th_guess = -1.0f;  // the last ray's first hit in this work item (none yet)
        bool carry_dense = false;  // the last ray of this work item ended in a dense stretch
        for (int l = l0; l < l1; l++) {
            int px, py;
            if (!tile_pixel(cam, lt, l, zt, P.tile_w, P.tile_h, px, py)) continue;
            const int64_t ray = (int64_t)s_pix[c] + (int64_t)py * cam.width + px;
            float4 o_rgba, o_state;
            uint4 o_tape = make_uint4(0u, 0xffffffffu, 0u, 0u);
            int o_nrec = 0;
            float4 up_l = make_float4(0.f, 0.f, 0.f, 0.f), st_l = up_l;
            uint4 st2_l = make_uint4(0u, 0xffffffffu, 0u, 0u);
            if (BWD) {
                up_l = make_float4(__shfl_sync(FULLMASK, my_up.x, l), __shfl_sync(FULLMASK, my_up.y, l),
                                   __shfl_sync(FULLMASK, my_up.z, l), __shfl_sync(FULLMASK, my_up.w, l));
                st_l = make_float4(__shfl_sync(FULLMASK, my_st.x, l), __shfl_sync(FULLMASK, my_st.y, l),
                                   __shfl_sync(FULLMASK, my_st.z, l), __shfl_sync(FULLMASK, my_st.w, l));
                st2_l = make_uint4(__shfl_sync(FULLMASK, my_st2.x, l), __shfl_sync(FULLMASK, my_st2.y, l),
                                   __shfl_sync(FULLMASK, my_st2.z, l), __shfl_sync(FULLMASK, my_st2.w, l));
            }
            march_ray<NS, BWD>(P, W, ray, c, cam, px, py, root_lo, root_hi, up_l, st_l, st2_l, cnt, whole, tape_base,
                               tape_left, pt_base, pt_left, o_rgba, o_state, o_tape, o_nrec, th_guess, carry_dense);
            if (!BWD && lane == l) { my_rgba = o_rgba; my_state = o_state; my_tape = o_tape; my_nrec = o_nrec; }
        }
        if (!BWD) {
            int px, py;
            if (mine && tile_pixel(cam, lt, lane, zt, P.tile_w, P.tile_h, px, py)) {
                const int64_t ray = (int64_t)s_pix[c] + (int64_t)py * cam.width + px;
                P.rgba[ray] = my_rgba;
                if (P.state) {
                    P.state[2 * ray] = my_state;
                    reinterpret_cast<uint4*>(P.state)[2 * ray + 1] = my_tape;
                }
                if (P.sched_n) P.sched_n[ray] = my_nrec;
            }
        }
        if (P.counters) {
            int nvalid = 0;
            {
                int px, py;
                nvalid = mine && tile_pixel(cam, lt, lane, zt, P.tile_w, P.tile_h, px, py) ? 1 : 0;
            }
            const unsigned v[8] = {(unsigned)nvalid, cnt.segs, cnt.hits, cnt.evals, cnt.visits, cnt.chq, cnt.skips,
                                   cnt.windows};
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const unsigned s = __reduce_add_sync(FULLMASK, v[i]);
                if (lane == 0 && s) atomicAdd(&P.counters[i], (unsigned long long)s);
            }
        }
    }
}

// The march kernel in two register budgets.  Without a cap the compiler takes up to ~240
// registers per thread, so registers allow 8 one-warp blocks per SM -- as many as the shared
// memory of a large chord list (hit_cap 512) does.  With short lists (dense scenes) shared
// memory would allow more: k_march_lean is capped at RGX_LEAN_REGS registers (12 warps per SM,
// with a few bytes of spills), and the host picks it when it really gets more warps.
template <int NS, bool BWD>
__global__ void __launch_bounds__(RGX_BLOCK, 1) k_march(MarchParams P) {
    march_kernel<NS, BWD>(P);
}

template <int NS, bool BWD>
__global__ void __maxnreg__(RGX_LEAN_REGS) k_march_lean(MarchParams P) {
    march_kernel<NS, BWD>(P);
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
static void* kernel_ptr(bool lean) { return lean ? (void*)k_march_lean<NS, BWD> : (void*)k_march<NS, BWD>; }

static void* pick_kernel(int ns, bool bwd, bool lean) {
    switch (ns) {
        case 4: return bwd ? kernel_ptr<4, true>(lean) : kernel_ptr<4, false>(lean);
        case 8: return bwd ? kernel_ptr<8, true>(lean) : kernel_ptr<8, false>(lean);
        case 16: return bwd ? kernel_ptr<16, true>(lean) : kernel_ptr<16, false>(lean);
        case 32: return bwd ? kernel_ptr<32, true>(lean) : kernel_ptr<32, false>(lean);
    }
    return nullptr;
}

// Fills the tuning knobs left at 0 -- hit_cap, the tile shape (both 0), N_S -- with the
// scene's last rgx_autotune result, else the defaults, then checks the options.
static rgx_status check_opts(rgx_scene* s, const rgx_opts* in, rgx_opts* o) {
    if (!in) return set_err(s, RGX_ERR_INVALID_ARG, "null opts");
    *o = *in;
    const bool tuned = s && s->has_tuned;
    if (o->hit_cap == 0) {
        o->hit_cap = tuned ? s->tuned_hit_cap : RGX_DEFAULT_HIT_CAP;
        // the tuned choice of first-window lowering comes with the tuned list capacity
        if (tuned) o->flags = (o->flags & ~RGX_LOWER_FIRST) | (s->tuned_flags & RGX_LOWER_FIRST);
    }
    if (o->tile_w == 0 && o->tile_h == 0) {
        o->tile_w = tuned ? s->tuned_tile_w : RGX_DEFAULT_TILE_W;
        o->tile_h = tuned ? s->tuned_tile_h : RGX_DEFAULT_TILE_H;
    }
    if (o->n_s == 0) o->n_s = tuned ? s->tuned_n_s : RGX_DEFAULT_NS;
    if (o->n_s != 4 && o->n_s != 8 && o->n_s != 16 && o->n_s != 32)
        return set_err(s, RGX_ERR_INVALID_ARG, "n_s must be 0, 4, 8, 16 or 32");
    if (o->flags & RGX_ADAPTIVE) {
        if (!(o->dt_min > 0.0f) || !(o->dt_max >= o->dt_min) || !(o->beta > 0.0f))
            return set_err(s, RGX_ERR_INVALID_ARG, "adaptive mode needs 0 < dt_min <= dt_max and beta > 0");
    } else if (!(o->dt > 0.0f)) {
        return set_err(s, RGX_ERR_INVALID_ARG, "dt must be > 0");
    }
    if (o->hit_cap < 32 || o->hit_cap > 1024 || (o->hit_cap & 31))
        return set_err(s, RGX_ERR_INVALID_ARG, "hit_cap must be 0 or a multiple of 32 in [32, 1024]");
    if ((o->flags & RGX_ZTILES) && (o->tile_w <= 0 || o->tile_h <= 0 || o->tile_w * o->tile_h != 32))
        return set_err(s, RGX_ERR_INVALID_ARG, "tile_w * tile_h must be 32 (or both 0)");
    if (!(o->t_eps >= 0.0f)) return set_err(s, RGX_ERR_INVALID_ARG, "t_eps must be >= 0");
    if (o->max_segments < 0) return set_err(s, RGX_ERR_INVALID_ARG, "max_segments must be >= 0");
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
                               int32_t* sched_n, cudaStream_t st, float4* vgrad = nullptr, float4* gsg = nullptr) {
    MarchParams P;
    memset(&P, 0, sizeof P);
    P.geom = s->geom; P.shc = s->shc; P.perm = s->perm;
    P.sgp = s->sgp; P.n_sg = s->n_sg; P.nodes = s->nodes; P.nodew = s->nodew; P.root = s->root;
    P.n = s->n; P.morton = s->morton;
    P.cams = s->cams; P.ncam = ncam;
    P.flags = o->flags;
    P.dt = o->dt; P.dt_min = o->dt_min; P.dt_max = o->dt_max; P.beta = o->beta; P.t_eps = o->t_eps;
    P.bg0 = o->bg[0]; P.bg1 = o->bg[1]; P.bg2 = o->bg[2];
    P.tile_w = o->tile_w > 0 ? o->tile_w : RGX_DEFAULT_TILE_W; P.tile_h = o->tile_h > 0 ? o->tile_h : RGX_DEFAULT_TILE_H;
    P.hit_cap = o->hit_cap; P.max_segments = o->max_segments;
    P.rgba = (float4*)rgba; P.state = (float4*)state;
    P.d_rgba = (const float4*)d_rgba; P.grad = s->grad; P.vgrad = vgrad; P.gsg = gsg;
    P.sched = (float2*)sched; P.sched_cap = sched_cap; P.sched_n = sched_n;
    P.queue = s->queue; P.status = s->status; P.counters = s->counters;
    P.min_items = 16u * (uint32_t)s->num_sms;
    RGX_CUDA(s, cudaMemcpyAsync(s->cams, cams, sizeof(rgx_camera) * ncam, cudaMemcpyHostToDevice, st));
    RGX_CUDA(s, cudaMemsetAsync(s->queue, 0, sizeof(unsigned), st));
    // first-window tape and chunked-segment sums: the forward (with a state to hand on) fills
    // them under a new tag, the adjoint reads them for states carrying that tag
    if (!bwd && state) {
        s->tape_gen++;
        uint32_t tag = (uint32_t)(((uintptr_t)s >> 6) * 0x9E3779B1u) ^ (s->tape_gen * 0x85EBCA77u);
        s->tape_tag = tag ? tag : 1u;
        P.tape_tag = s->tape_tag;
        if (s->tape_cap > 0) {
            RGX_CUDA(s, cudaMemsetAsync(s->queue + 1, 0, sizeof(unsigned), st));
            P.tape = s->tape; P.tape_n = s->queue + 1; P.tape_cap = (uint32_t)s->tape_cap;
        }
        s->csum_slots_last = s->csum_slots;
        s->csum_ns_last = o->n_s;
        if (s->csum_slots > 0) { P.csums = s->csums; P.csum_slots = (uint32_t)s->csum_slots; }
        s->ptape_cap_last = 0;
        if (s->csum_slots > 0 && s->ptape_cap > 0) {
            RGX_CUDA(s, cudaMemsetAsync(s->queue + 2, 0, sizeof(unsigned), st));
            P.ptape = s->ptape; P.ptape_n = s->queue + 2; P.ptape_cap = (uint32_t)s->ptape_cap;
            s->ptape_cap_last = s->ptape_cap;
        }
    } else if (bwd && s->tape_tag != 0) {
        P.tape_tag = s->tape_tag;
        if (s->tape_cap > 0) { P.tape = s->tape; P.tape_cap = (uint32_t)s->tape_cap; }
        if (s->csum_slots_last > 0 && s->csum_ns_last == o->n_s) {
            P.csums = s->csums;
            P.csum_slots = (uint32_t)s->csum_slots_last;
            if (s->ptape_cap_last > 0) { P.ptape = s->ptape; P.ptape_cap = (uint32_t)s->ptape_cap_last; }
        }
    }
    RGX_CUDA(s, cudaMemsetAsync(s->counters, 0, 8 * sizeof(unsigned long long), st));
    const size_t head = ((size_t)(3 * (ncam + 1)) * 4 + 15) & ~(size_t)15;
    const size_t smem = head + (size_t)WARPS * warp_bytes(o->hit_cap, bwd);
    // resident blocks per SM of a kernel at this shared-memory size (cached: no attribute query
    // inside a CUDA-graph capture once a configuration has been seen)
    auto occupancy = [&](void* kk, int* occ_out) -> rgx_status {
        int occ = 0;
        for (int i = 0; i < s->ncfg; i++)
            if (s->cfg[i].k == kk && s->cfg[i].smem == smem) occ = s->cfg[i].occ;
        if (occ == 0) {
            RGX_CUDA(s, cudaFuncSetAttribute(kk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            RGX_CUDA(s, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kk, RGX_BLOCK, smem));
            if (occ < 1) occ = 1;
            const int slot = s->ncfg < 64 ? s->ncfg++ : 63;
            s->cfg[slot] = {kk, smem, occ};
        }
        *occ_out = occ;
        return RGX_OK;
    };
    void* k = pick_kernel(o->n_s, bwd, false);
    void* kl = pick_kernel(o->n_s, bwd, true);
    int occ = 0, occl = 0;
    rgx_status rs = occupancy(k, &occ);
    if (rs) return rs;
    rs = occupancy(kl, &occl);
    if (rs) return rs;
    // the lean kernel only where it gains at least two warps per SM (its spills cost a little)
    if (occl >= occ + 2) { k = kl; occ = occl; }
    if (occ < 1) occ = 1;
    const int grid = s->num_sms * occ;

    if (bwd) {
        // scratch for the chunks of overflowing segments (one region per resident
        // warp); without it the adjoint re-traverses such segments
        const size_t need = (size_t)grid * WARPS * SPILL_CAP * 3;
        if (s->spill_cap < need) {
            if (s->spill) cudaFree(s->spill);
            s->spill = nullptr;
            s->spill_cap = 0;
            if (cudaMalloc(&s->spill, need * sizeof(float4)) == cudaSuccess) s->spill_cap = need;
            else { s->spill = nullptr; cudaGetLastError(); }
        }
        P.spill = s->spill;
    }
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

static rgx_status forward_common(rgx_scene* s, const rgx_camera* cams, int32_t ncam, const rgx_opts* in,
                                 float* rgba, void* state, float* sched, int32_t sched_cap, int32_t* sched_n,
                                 void* stream) {
    if (!s) return set_err(s, RGX_ERR_INVALID_ARG, "null scene");
    if (!s->built) return set_err(s, RGX_ERR_NOT_BUILT, "rgx_render_forward before rgx_build_bvh");
    rgx_opts ro;
    const rgx_opts* o = &ro;
    rgx_status r = check_opts(s, in, &ro);
    if (r) return r;
    int64_t R = 0;
    r = check_cams(s, cams, ncam, &R);
    if (r) return r;
    if (!rgba) return set_err(s, RGX_ERR_INVALID_ARG, "null rgba");
    if (sched && (sched_cap <= 0 || !sched_n)) return set_err(s, RGX_ERR_INVALID_ARG, "bad schedule buffers");
    RGX_CUDA(s, cudaSetDevice(s->device));
    r = ensure_cams(s, ncam);
    if (r) return r;
    if (state) {
        // room on the tape for hit_cap / 6 entries of 48 B per ray on average (or the caller's
        // limit); a ray that finds no room is simply not taped (its adjoint collects the window
        // itself).  tape_cap is the capacity this forward uses: the stride of the three planes.
        size_t need = (size_t)R * (size_t)(o->hit_cap / 6);
        if (need > (size_t)0x7fffffff) need = (size_t)0x7fffffff;
        if (s->tape_limit >= 0 && need > (size_t)s->tape_limit) need = (size_t)s->tape_limit;
        if (s->tape_alloc < need) {
            if (s->tape) cudaFree(s->tape);
            s->tape = nullptr;
            s->tape_alloc = 0;
            if (cudaMalloc(&s->tape, 3 * need * sizeof(float4)) == cudaSuccess) s->tape_alloc = need;
            else { s->tape = nullptr; cudaGetLastError(); }
        }
        s->tape_cap = s->tape_alloc < need ? s->tape_alloc : need;
        // sums records of chunked segments: up to RGX_CSUM_SLOTS per ray within RGX_CSUM_BUDGET bytes
        // (none when the tape is disabled); rays with more chunked segments re-evaluate the rest
        const size_t per_slot = (size_t)(o->n_s + 1) * sizeof(float4);
        size_t slots = s->tape_limit == 0 ? 0 : (size_t)RGX_CSUM_BUDGET / ((size_t)R * per_slot + 1);
        if (slots > RGX_CSUM_SLOTS) slots = RGX_CSUM_SLOTS;
        const size_t cneed = slots * (size_t)R * (size_t)(o->n_s + 1);
        if (slots > 0 && s->csum_alloc < cneed) {
            if (s->csums) cudaFree(s->csums);
            s->csums = nullptr;
            s->csum_alloc = 0;
            if (cudaMalloc(&s->csums, cneed * sizeof(float4)) == cudaSuccess) s->csum_alloc = cneed;
            else { s->csums = nullptr; cudaGetLastError(); }
        }
        s->csum_slots = (s->csums && s->csum_alloc >= cneed) ? (int)slots : 0;
        // the index tape of the recorded segments' chords, each with its colour (16 B an entry): up to
        // 2,048 per ray within its budget
        size_t pneed = s->csum_slots > 0 ? (size_t)R * 2048 : 0;
        if (pneed > (size_t)RGX_PTAPE_MAX) pneed = (size_t)RGX_PTAPE_MAX;
        if (pneed > 0 && s->ptape_alloc < pneed) {
            if (s->ptape) cudaFree(s->ptape);
            s->ptape = nullptr;
            s->ptape_alloc = 0;
            if (cudaMalloc(&s->ptape, pneed * sizeof(uint4)) == cudaSuccess) s->ptape_alloc = pneed;
            else { s->ptape = nullptr; cudaGetLastError(); }
        }
        s->ptape_cap = (s->ptape && s->ptape_alloc >= pneed) ? pneed : 0;
    }
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

// Eq. 11 for every camera of a batched adjoint: camera c's own mean gradient of Gaussian
// (packed index) p is M^T V_c, V_c the first moment the camera's rays added; a Gaussian
// with a non-zero one adds |mu - o_c| / f_c |M^T V_c| to its statistic and 1 to its count.
__global__ void k_densify_views(int64_t n, int morton, int ncam, const float4* __restrict__ vgrad,
                                const float4* __restrict__ geom, const int32_t* __restrict__ perm,
                                const rgx_camera* __restrict__ cams, float* stat, int32_t* count) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = morton ? (int64_t)perm[p] : p;
        const float4 g0 = geom[4 * p], g1 = geom[4 * p + 1], g2 = geom[4 * p + 2], g3 = geom[4 * p + 3];
        float acc = 0.0f;
        int cnt = 0;
        for (int c = 0; c < ncam; c++) {
            const float4 v = vgrad[(size_t)p * ncam + c];
            const float dx = g1.x * v.x + g2.x * v.y + g3.x * v.z;
            const float dy = g1.y * v.x + g2.y * v.y + g3.y * v.z;
            const float dz = g1.z * v.x + g2.z * v.y + g3.z * v.z;
            const float gn = sqrtf(dx * dx + dy * dy + dz * dz);
            if (gn > 0.0f) {
                const rgx_camera& C = cams[c];
                const float ex = g0.x - C.c2w[3], ey = g0.y - C.c2w[7], ez = g0.z - C.c2w[11];
                acc += sqrtf(ex * ex + ey * ey + ez * ez) / C.fx * gn;
                cnt++;
            }
        }
        if (cnt) {
            stat[l] += acc;
            count[l] += cnt;
        }
    }
}

// Lobe gradients in the caller's order: the unit-axis gradient projected onto the raw axis
// u (mu = u / |u|: du = (dmu - mu (mu . dmu)) / |u|), sharpness and amplitude as accumulated.
__global__ void k_grad_finalize_sg(int64_t n, int n_sg, int morton, const float4* __restrict__ gsg,
                                   const float4* __restrict__ sgp, const int32_t* __restrict__ perm, float* d_sg) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = morton ? (int64_t)perm[p] : p;
        for (int j = 0; j < n_sg; j++) {
            const float4 g0 = gsg[2 * (p * n_sg + j)], g1 = gsg[2 * (p * n_sg + j) + 1];
            const float4 ax = sgp[2 * (p * n_sg + j)], am = sgp[2 * (p * n_sg + j) + 1];
            const float md = ax.x * g0.x + ax.y * g0.y + ax.z * g0.z;
            float* o = d_sg + (l * n_sg + j) * 7;
            o[0] += (g0.x - ax.x * md) * am.w;
            o[1] += (g0.y - ax.y * md) * am.w;
            o[2] += (g0.z - ax.z * md) * am.w;
            o[3] += g0.w;
            o[4] += g1.x;
            o[5] += g1.y;
            o[6] += g1.z;
        }
    }
}

static rgx_status backward_common(rgx_scene* s, const rgx_camera* cams, int32_t ncam, const rgx_opts* in,
                                  const void* fwd_state, const float* d_rgba, float* d_means, float* d_scales,
                                  float* d_quats, float* d_dens, float* d_sh, float* d_sg, float* dstat,
                                  int32_t* dcount, void* stream) {
    if (!s) return set_err(s, RGX_ERR_INVALID_ARG, "null scene");
    if (!s->built) return set_err(s, RGX_ERR_NOT_BUILT, "rgx_render_backward before rgx_build_bvh");
    rgx_opts ro;
    const rgx_opts* o = &ro;
    rgx_status r = check_opts(s, in, &ro);
    if (r) return r;
    int64_t R = 0;
    r = check_cams(s, cams, ncam, &R);
    if (r) return r;
    if (!fwd_state || !d_rgba) return set_err(s, RGX_ERR_INVALID_ARG, "null fwd_state or d_rgba");
    if (s->n > 0 && (!d_means || !d_scales || !d_quats || !d_dens || !d_sh))
        return set_err(s, RGX_ERR_INVALID_ARG, "null gradient array");
    const bool densify = dstat != nullptr || dcount != nullptr;
    if (densify && (!dstat || !dcount)) return set_err(s, RGX_ERR_INVALID_ARG, "densification needs stat and count");
    if (densify) {
        for (int i = 0; i < ncam; i++)
            if (!(cams[i].fx > 0.0f)) return set_err(s, RGX_ERR_INVALID_ARG, "densification needs fx > 0");
    }
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
    float4* vgrad = nullptr;
    if (densify) {
        const size_t need = (size_t)s->n * (size_t)ncam;
        if (s->vgrad_cap < need) {
            if (s->vgrad) cudaFree(s->vgrad);
            s->vgrad = nullptr;
            s->vgrad_cap = 0;
            if (cudaMalloc(&s->vgrad, need * sizeof(float4)) != cudaSuccess)
                return set_err(s, RGX_ERR_WORKSPACE, "per-camera moment allocation failed");
            s->vgrad_cap = need;
        }
        vgrad = s->vgrad;
        RGX_CUDA(s, cudaMemsetAsync(vgrad, 0, need * sizeof(float4), st));
    }
    float4* gsg = nullptr;
    if (d_sg && s->n_sg > 0) {
        const size_t need = (size_t)s->n * s->n_sg * 2;
        if (s->gsg_cap < need) {
            if (s->gsg) cudaFree(s->gsg);
            s->gsg = nullptr;
            s->gsg_cap = 0;
            if (cudaMalloc(&s->gsg, need * sizeof(float4)) != cudaSuccess)
                return set_err(s, RGX_ERR_WORKSPACE, "lobe gradient allocation failed");
            s->gsg_cap = need;
        }
        gsg = s->gsg;
        RGX_CUDA(s, cudaMemsetAsync(gsg, 0, need * sizeof(float4), st));
    }
    RGX_CUDA(s, cudaMemsetAsync(s->grad, 0, (size_t)16 * sizeof(float4) * s->n, st));
    r = launch_march(s, cams, ncam, o, true, nullptr, (void*)fwd_state, d_rgba, nullptr, 0, nullptr, st, vgrad, gsg);
    if (r) return r;
    const int nk = (s->sh_degree + 1) * (s->sh_degree + 1);
    int64_t b = (s->n + 255) / 256;
    if (b > (int64_t)s->num_sms * 16) b = (int64_t)s->num_sms * 16;
    k_grad_finalize<<<(int)b, 256, 0, st>>>(s->n, s->morton, nk, s->grad, s->geom, s->aux, s->perm, d_means,
                                            d_scales, d_quats, d_dens, d_sh);
    RGX_CUDA(s, cudaGetLastError());
    if (gsg) {
        k_grad_finalize_sg<<<(int)b, 256, 0, st>>>(s->n, s->n_sg, s->morton, gsg, s->sgp, s->perm, d_sg);
        RGX_CUDA(s, cudaGetLastError());
    }
    if (densify) {
        k_densify_views<<<(int)b, 256, 0, st>>>(s->n, s->morton, ncam, vgrad, s->geom, s->perm, s->cams, dstat,
                                                dcount);
        RGX_CUDA(s, cudaGetLastError());
    }
    return RGX_OK;
}

extern "C" rgx_status rgx_render_backward(rgx_scene* s, const rgx_camera* cams, int32_t ncam, const rgx_opts* o,
                                          const void* fwd_state, const float* d_rgba, float* d_means,
                                          float* d_scales, float* d_quats, float* d_dens, float* d_sh, void* stream) {
    return backward_common(s, cams, ncam, o, fwd_state, d_rgba, d_means, d_scales, d_quats, d_dens, d_sh, nullptr,
                           nullptr, nullptr, stream);
}

extern "C" rgx_status rgx_render_backward_ex(rgx_scene* s, const rgx_camera* cams, int32_t ncam, const rgx_opts* o,
                                             const void* fwd_state, const float* d_rgba, float* d_means,
                                             float* d_scales, float* d_quats, float* d_dens, float* d_sh,
                                             float* d_sg, float* stat, int32_t* count, void* stream) {
    if (s && s->n_sg > 0 && s->n > 0 && !d_sg)
        return set_err(s, RGX_ERR_INVALID_ARG, "rgx_render_backward_ex: the scene has lobes: d_sg is required");
    return backward_common(s, cams, ncam, o, fwd_state, d_rgba, d_means, d_scales, d_quats, d_dens, d_sh, d_sg,
                           stat, count, stream);
}

extern "C" rgx_status rgx_set_tape_limit(rgx_scene* s, int64_t max_entries) {
    if (!s) return set_err(s, RGX_ERR_INVALID_ARG, "rgx_set_tape_limit: null scene");
    s->tape_limit = max_entries < 0 ? -1 : max_entries;
    return RGX_OK;
}
