// common.cuh -- internal declarations of librgx (not part of the ABI).
//
// Packed per-Gaussian record (packed index p; Z-order position with
// RGX_MORTON, caller index otherwise):
//   geom[4p+0] = (mu.x, mu.y, mu.z, Q_eps)       Q_eps = 2 ln(sigma~/sigma_eps)
//   geom[4p+1] = (M00, M01, M02, log2 sigma~)    M = S^-1 R^T (whitening)
//   geom[4p+2] = (M10, M11, M12, sigma~)
//   geom[4p+3] = (M20, M21, M22, 0)
//   shc [12p..12p+11] = 48 SH coefficients, (k, channel) channel fastest
//   aux [2p+0] = raw quaternion (w,x,y,z), aux[2p+1] = (s0, s1, s2, 0)
// so that q(x) = |M (x - mu)|^2 and sigma_l(x) = sigma~ exp(-q/2) (Supp. Sec. 2.1).
//
// Internal BVH node i (0 <= i < n-1), 4 x float4 = 64 B, both children's
// boxes stored in the parent so one fetch tests both:
//   node[4i+0] = (left.lo xyz,  first)   first/split/last: int32 bit patterns
//   node[4i+1] = (left.hi xyz,  split)   left child  = split   (leaf iff first == split)
//   node[4i+2] = (right.lo xyz, last)    right child = split+1 (leaf iff split+1 == last)
//   node[4i+3] = (right.hi xyz, 0)
//
// 4-wide copy read by the traversals: nodew[4i .. 4i+3] = the (up to) four
// grandchildren of internal node i (a child itself where it is a leaf), 16 B each:
// the child's box as 6 halves rounded outward (so it stays conservative) and a ref
// = internal node id, or packed index | 0x80000000 for a leaf.  Unused slots hold
// an inverted (empty) box.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include "../../include/rgx.h"

#define RGX_STACK 96          // >= depth of a radix tree over (63-bit code, 32-bit index) keys
#define RGX_MAX_CAMS 1024
#define RGX_MAX_SG 7          // spherical-Gaussian lobes per Gaussian (Supp. Sec. 6.1 uses seven)
// defaults of the tuning knobs left at 0 before a scene has been autotuned (the values
// rgx_autotune picked on a 100k-Gaussian object view at 800x800)
#define RGX_DEFAULT_HIT_CAP 512
#define RGX_DEFAULT_TILE_W 32
#define RGX_DEFAULT_TILE_H 1
#define RGX_DEFAULT_NS 16
#define RGX_SEGMENT_CEILING (1 << 20)  // per-ray segment bound when max_segments = 0
#define RGX_BLOCK 32          // threads per block of the march kernels (one warp: finest shared-memory granularity)

// ---------------------------------------------------------------- scene
struct rgx_scene {
    int device = 0;
    int num_sms = 0;
    // current build
    int64_t n = 0;
    int sh_degree = 0;
    int built = 0;
    int morton = 0;           // packed order is Z-order
    // capacity-managed device buffers
    int64_t cap_n = 0;
    uint64_t* keys[2] = {nullptr, nullptr};
    uint32_t* vals[2] = {nullptr, nullptr};
    int sorted_buf = 0;       // which of keys/vals holds the sorted result
    uint32_t* hist = nullptr; size_t hist_cap = 0;
    float4* nodes = nullptr;
    uint4* nodew = nullptr;        // [4 (n-1)] 4-wide traversal records
    int32_t* parent = nullptr;     // [2n]: parent of leaf i at [i], of internal j at [n+j]
    int32_t* visit = nullptr;      // [n] refit arrival counters
    float4* geom = nullptr;
    float4* shc = nullptr;
    float4* aux = nullptr;
    int32_t* perm = nullptr;       // sorted position -> caller index
    float4* leafbox = nullptr;     // [2n] leaf boxes in sorted order (lo, hi)
    unsigned int* bounds = nullptr;// [8] ordered-int min/max of the means
    float* root = nullptr;         // [8] scene box
    float4* grad = nullptr;        // [16n] backward accumulators (packed order)
    int64_t grad_cap = 0;
    int n_sg = 0;                  // spherical-Gaussian lobes per Gaussian (0..7)
    float4* sgp = nullptr;         // [n][n_sg][2] lobes: (unit axis, sharpness), (RGB amplitude, 1/|raw axis|)
    size_t sgp_cap = 0;            // in float4
    float4* gsg = nullptr;         // [n][n_sg][2] adjoint accumulators: (d unit axis, d sharpness), (d amplitude)
    size_t gsg_cap = 0;            // in float4
    float4* vgrad = nullptr;       // [n][ncam] per-camera V moments (densification statistic)
    void* loss_ws = nullptr;       // image-loss scratch (24 floats per pixel, 2 doubles per view)
    size_t loss_cap = 0;           // in bytes
    int ssim_w_set = 0;            // SSIM window taps uploaded to this device
    void* plan_ws = nullptr;       // densification plan: scan block sums and the total
    size_t plan_cap = 0;           // in bytes
    size_t vgrad_cap = 0;          // in float4
    float4* spill = nullptr;       // adjoint scratch: chunk entries of overflowing segments, per resident warp
    size_t spill_cap = 0;          // in float4
    float4* tape = nullptr;        // the last forward's first-window lists: 3 planes of tape_cap float4
    size_t tape_cap = 0;           // entries the last forward with a state could use (the planes' stride)
    size_t tape_alloc = 0;         // entries allocated
    uint32_t tape_gen = 0, tape_tag = 0;  // tag of the forward call whose lists the tape holds
    int64_t tape_limit = -1;       // caller's cap on tape entries (< 0: hit_cap / 6 per ray)
    float4* csums = nullptr;       // sums records of chunked segments (see MarchParams::csums)
    size_t csum_alloc = 0;         // in float4
    int csum_slots = 0;            // records per ray the next forward with a state uses
    int csum_slots_last = 0, csum_ns_last = 0;  // layout of the last forward's records
    uint4* ptape = nullptr;        // chords of recorded chunked segments: (packed index, colour bits)
    size_t ptape_alloc = 0, ptape_cap = 0, ptape_cap_last = 0;  // entries: allocated / next forward / last forward
    // the last rgx_autotune result: what tuning knobs left at 0 select
    int has_tuned = 0;
    int tuned_hit_cap = 0, tuned_tile_w = 0, tuned_tile_h = 0, tuned_n_s = 0, tuned_flags = 0;
    // render
    rgx_camera* cams = nullptr; int cams_cap = 0;
    unsigned int* queue = nullptr; // [4] persistent work counters
    unsigned int* status = nullptr;
    unsigned long long* counters = nullptr; // [8]
    // launch-configuration cache: (kernel, dynamic smem) -> resident blocks/SM,
    // so that calls inside a CUDA-graph capture make no attribute queries
    struct LaunchCfg { const void* k; size_t smem; int occ; };
    LaunchCfg cfg[64];
    int ncfg = 0;
    char last_error[256] = {0};
};

// ordered mapping float <-> uint so that atomicMin/Max on uint orders floats
__device__ __forceinline__ unsigned int f2ord(float f) {
    unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned int u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// ---------------------------------------------------------------- SH
// Real spherical harmonics up to degree 3 as polynomials in the unit
// direction (x, y, z), Condon-Shortley phase, index k = l^2 + l + m.
// Constants are K_l^m-normalisation values written out:
//   1/(2 sqrt(pi)); sqrt(3/(4pi)); sqrt(15/(4pi)), sqrt(5/(16pi)), sqrt(15/(16pi));
//   sqrt(35/(32pi)), sqrt(105/(4pi)), sqrt(21/(32pi)), sqrt(7/(16pi)), sqrt(105/(16pi)).
__device__ __forceinline__ void sh_basis16(float x, float y, float z, float Y[16]) {
    // explicitly rounded: the forward and the adjoint kernel must get the same bits
    const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    Y[0] = 0.28209479177387814f;
    Y[1] = __fmul_rn(-0.48860251190291992f, y);
    Y[2] = __fmul_rn(0.48860251190291992f, z);
    Y[3] = __fmul_rn(-0.48860251190291992f, x);
    Y[4] = __fmul_rn(__fmul_rn(1.0925484305920792f, x), y);
    Y[5] = __fmul_rn(__fmul_rn(-1.0925484305920792f, y), z);
    Y[6] = __fmul_rn(0.31539156525252005f, __fmaf_rn(3.0f, zz, -1.0f));
    Y[7] = __fmul_rn(__fmul_rn(-1.0925484305920792f, x), z);
    Y[8] = __fmul_rn(0.54627421529603959f, __fsub_rn(xx, yy));
    Y[9] = __fmul_rn(__fmul_rn(-0.59004358992664352f, y), __fmaf_rn(3.0f, xx, -yy));
    Y[10] = __fmul_rn(__fmul_rn(__fmul_rn(2.8906114426405538f, x), y), z);
    Y[11] = __fmul_rn(__fmul_rn(-0.45704579946446572f, y), __fmaf_rn(5.0f, zz, -1.0f));
    Y[12] = __fmul_rn(__fmul_rn(0.37317633259011540f, z), __fmaf_rn(5.0f, zz, -3.0f));
    Y[13] = __fmul_rn(__fmul_rn(-0.45704579946446572f, x), __fmaf_rn(5.0f, zz, -1.0f));
    Y[14] = __fmul_rn(__fmul_rn(1.4453057213202769f, z), __fsub_rn(xx, yy));
    Y[15] = __fmul_rn(__fmul_rn(-0.59004358992664352f, x), __fmaf_rn(-3.0f, yy, xx));
}

// ---------------------------------------------------------------- host helpers
static inline rgx_status set_err(rgx_scene* s, rgx_status st, const char* msg) {
    extern char g_rgx_last_error[256];
    if (s) { strncpy(s->last_error, msg, sizeof(s->last_error) - 1); }
    strncpy(g_rgx_last_error, msg, 255);
    return st;
}

#define RGX_CUDA(s, call)                                                         \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            char m_[256];                                                         \
            snprintf(m_, sizeof m_, "%s: %s", #call, cudaGetErrorString(e_));     \
            return set_err((s), RGX_ERR_CUDA, m_);                                \
        }                                                                         \
    } while (0)

// internal entry points shared between translation units
rgx_status rgx_internal_reserve(rgx_scene* s, int64_t n);
