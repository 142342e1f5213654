// build.cu -- per-iteration acceleration-structure build (rgx_build_bvh).
//
// Sec. 3.2 of RayGaussX rebuilds the BVH over the Gaussians' AABBs at every
// optimisation step; Sec. 3.3 re-indexes the Gaussians along a Z-order curve
// of their means.  On B300 both are one pipeline of bandwidth-bound kernels:
//
//   k_bounds    per-axis min/max of the means (ordered-int atomics), input check
//   k_morton    30-bit (10/axis) or 63-bit (21/axis) Z-order code of each mean
//   k_rs_*      stable LSD radix sort of (code, index), 8-bit digits
//   k_pack      Z-order gather of the parameters into float4 records with the
//               whitening matrix M = S^-1 R^T, Q_eps and the minimal AABB of the
//               sigma_eps ellipsoid (Supp. Sec. 2.2: L_i = sqrt(sum_j r_ij^2 s~_j^2))
//   k_karras    binary radix tree over the sorted codes (Karras 2012), one thread
//               per internal node, ties broken by sorted position
//   k_refit     bottom-up AABB union with per-node arrival counters
//   k_widen     4-wide traversal records: per internal node its (up to) four
//               grandchildren as half-precision boxes, rounded outward
#include <stdio.h>
#include <cuda_fp16.h>
#include <atomic>
#include "common.cuh"

#define FULLMASK 0xffffffffu
#define RS_THREADS 256
#define RS_ITEMS 16
#define RS_TILE (RS_THREADS * RS_ITEMS)

char g_rgx_last_error[256] = "";

// ------------------------------------------------------------------ bounds
__global__ void k_bounds(int64_t n, const float* __restrict__ means, const float* __restrict__ scales,
                         const float* __restrict__ quats, const float* __restrict__ dens,
                         unsigned int* __restrict__ bounds, unsigned int* __restrict__ status) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        for (int a = 0; a < 3; a++) {
            float m = means[3 * l + a];
            float s = scales[3 * l + a];
            bad |= !isfinite(m) || !isfinite(s) || !(s > 0.0f);
            lo[a] = fminf(lo[a], m);
            hi[a] = fmaxf(hi[a], m);
        }
        float q2 = 0.0f;
        for (int a = 0; a < 4; a++) { float q = quats[4 * l + a]; bad |= !isfinite(q); q2 += q * q; }
        bad |= !(q2 > 0.0f);
        float d = dens[l];
        bad |= !isfinite(d) || d < 0.0f;
    }
    for (int a = 0; a < 3; a++) {
        for (int off = 16; off > 0; off >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(FULLMASK, lo[a], off));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(FULLMASK, hi[a], off));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        for (int a = 0; a < 3; a++) {
            atomicMin(&bounds[a], f2ord(lo[a]));
            atomicMax(&bounds[3 + a], f2ord(hi[a]));
        }
    }
    if (__any_sync(FULLMASK, bad) && (threadIdx.x & 31) == 0) atomicOr(status, (unsigned)RGX_ERR_BAD_PARAMS);
}

// ------------------------------------------------------------------ Morton
// Cell of one coordinate, every operation rounded to nearest in float32 with
// no contraction:  cell = min(trunc(fl(fl(m - lo) * fl(B / (hi - lo)))), B-1).
__device__ __forceinline__ uint32_t quant_cell(float m, float lo, float hi, float B, uint32_t bmax) {
    float ext = __fsub_rn(hi, lo);
    float scale = ext > 0.0f ? __fdiv_rn(B, ext) : 0.0f;
    float v = __fmul_rn(__fsub_rn(m, lo), scale);
    uint32_t c = (v > 0.0f) ? (uint32_t)v : 0u;
    return c < bmax ? c : bmax;
}

__global__ void k_morton(int64_t n, const float* __restrict__ means, const unsigned int* __restrict__ bounds,
                         int wide, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int bits = wide ? 21 : 10;
    const float B = wide ? 2097152.0f : 1024.0f;
    const uint32_t bmax = (1u << bits) - 1u;
    float lo[3], hi[3];
    for (int a = 0; a < 3; a++) { lo[a] = ord2f(bounds[a]); hi[a] = ord2f(bounds[3 + a]); }
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c[3];
        for (int a = 0; a < 3; a++) {
            float m = means[3 * l + a];
            c[a] = isfinite(m) ? quant_cell(m, lo[a], hi[a], B, bmax) : 0u;
        }
        uint64_t code = 0;
        for (int i = 0; i < bits; i++) {
            code |= (uint64_t)((c[0] >> i) & 1u) << (3 * i + 2);
            code |= (uint64_t)((c[1] >> i) & 1u) << (3 * i + 1);
            code |= (uint64_t)((c[2] >> i) & 1u) << (3 * i);
        }
        keys[l] = code;
        vals[l] = (uint32_t)l;
    }
}

// ------------------------------------------------------------------ radix sort
// One 8-bit digit per pass; the per-block digit histogram is stored digit-major
// so that one exclusive scan yields every block's scatter base.
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                                                        uint32_t* __restrict__ hist, int nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int it = 0; it < RS_ITEMS; it++) {
        int64_t idx = base + it * RS_THREADS + threadIdx.x;
        if (idx < n) atomicAdd(&h[(uint32_t)(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t* __restrict__ hist, int total) {
    __shared__ uint32_t s[1024];
    const int chunk = (total + 1023) / 1024;
    const int beg = threadIdx.x * chunk;
    const int end = min(beg + chunk, total);
    uint32_t sum = 0;
    for (int i = beg; i < end; i++) sum += hist[i];
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t v = threadIdx.x >= off ? s[threadIdx.x - off] : 0u;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = threadIdx.x ? s[threadIdx.x - 1] : 0u;
    for (int i = beg; i < end; i++) { uint32_t v = hist[i]; hist[i] = run; run += v; }
}

// Stable scatter: keys are taken in 256-wide rounds in input order; inside a
// round, a key's position is its block base + keys of the same digit in
// earlier warps + its rank among same-digit lanes of its own warp.
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                           uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                           int64_t n, int shift, const uint32_t* __restrict__ hist,
                                                           int nblocks) {
    __shared__ uint32_t base[256];
    __shared__ uint32_t wc[RS_THREADS / 32][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    base[threadIdx.x] = hist[(size_t)threadIdx.x * nblocks + blockIdx.x];
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
    for (int it = 0; it < RS_ITEMS; it++) {
        const int64_t idx = tile0 + it * RS_THREADS + threadIdx.x;
        const bool valid = idx < n;
        uint64_t k = valid ? kin[idx] : 0ull;
        uint32_t v = valid ? vin[idx] : 0u;
        uint32_t d = valid ? ((uint32_t)(k >> shift) & 255u) : 0xffffffffu;
        uint32_t peers = __match_any_sync(FULLMASK, d);
        uint32_t rank = __popc(peers & lt);
        for (int j = threadIdx.x; j < (RS_THREADS / 32) * 256; j += RS_THREADS) (&wc[0][0])[j] = 0u;
        __syncthreads();
        if (valid && rank == 0) wc[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t off = base[d];
            for (int w = 0; w < warp; w++) off += wc[w][d];
            off += rank;
            kout[off] = k;
            vout[off] = v;
        }
        __syncthreads();
        uint32_t acc = 0;
        for (int w = 0; w < RS_THREADS / 32; w++) acc += wc[w][threadIdx.x];
        base[threadIdx.x] += acc;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ pack
__global__ void k_pack(int64_t n, int sh_degree, float sigma_eps, int morton,
                       const float* __restrict__ means, const float* __restrict__ scales,
                       const float* __restrict__ quats, const float* __restrict__ dens,
                       const float* __restrict__ sh, const uint32_t* __restrict__ sorted_idx,
                       int32_t* __restrict__ perm, float4* __restrict__ geom, float4* __restrict__ shc,
                       float4* __restrict__ aux, float4* __restrict__ leafbox,
                       unsigned int* __restrict__ status) {
    const int nk = (sh_degree + 1) * (sh_degree + 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t l = sorted_idx[i];
        perm[i] = (int32_t)l;
        const int64_t p = morton ? i : (int64_t)l;
        float mu[3] = {means[3 * l], means[3 * l + 1], means[3 * l + 2]};
        float s[3] = {scales[3 * l], scales[3 * l + 1], scales[3 * l + 2]};
        float qw = quats[4 * l], qx = quats[4 * l + 1], qy = quats[4 * l + 2], qz = quats[4 * l + 3];
        float sig = dens[l];
        float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        bool ok = isfinite(mu[0]) && isfinite(mu[1]) && isfinite(mu[2]) && s[0] > 0.0f && s[1] > 0.0f &&
                  s[2] > 0.0f && isfinite(s[0] + s[1] + s[2]) && qn > 0.0f && isfinite(qn) && isfinite(sig) &&
                  sig >= 0.0f;
        // copy SH (zero-padded to 16 coefficients)
        float c[48];
        bool shok = true;
        for (int j = 0; j < 48; j++) {
            float v = (j < 3 * nk) ? sh[(int64_t)l * 3 * nk + j] : 0.0f;
            shok &= isfinite(v);
            c[j] = v;
        }
        ok &= shok;
        if (!ok) atomicOr(status, (unsigned)RGX_ERR_BAD_PARAMS);
        if (!ok) { qw = 1.0f; qx = qy = qz = 0.0f; qn = 1.0f; s[0] = s[1] = s[2] = 1.0f; sig = 0.0f; }
        float w = qw / qn, x = qx / qn, y = qy / qn, z = qz / qn;
        float R[9] = {1.0f - 2.0f * (y * y + z * z), 2.0f * (x * y - w * z), 2.0f * (x * z + w * y),
                      2.0f * (x * y + w * z), 1.0f - 2.0f * (x * x + z * z), 2.0f * (y * z - w * x),
                      2.0f * (x * z - w * y), 2.0f * (y * z + w * x), 1.0f - 2.0f * (x * x + y * y)};
        float Qe = (sig > sigma_eps) ? 2.0f * logf(sig / sigma_eps) : 0.0f;
        float M[9];
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++) M[3 * j + k] = R[3 * k + j] / s[j];
        geom[4 * p + 0] = make_float4(mu[0], mu[1], mu[2], Qe);
        geom[4 * p + 1] = make_float4(M[0], M[1], M[2], sig > 0.0f ? log2f(sig) : -INFINITY);
        geom[4 * p + 2] = make_float4(M[3], M[4], M[5], sig);
        geom[4 * p + 3] = make_float4(M[6], M[7], M[8], 0.0f);
        for (int j = 0; j < 12; j++) shc[12 * p + j] = make_float4(c[4 * j], c[4 * j + 1], c[4 * j + 2], c[4 * j + 3]);
        aux[2 * p + 0] = make_float4(qw, qx, qy, qz);
        aux[2 * p + 1] = make_float4(s[0], s[1], s[2], 0.0f);
        // minimal AABB of the Q_eps ellipsoid, padded so float32 rounding never shrinks it
        float4 lo, hi;
        if (Qe > 0.0f) {
            float rq = sqrtf(Qe);
            float L[3];
            for (int a = 0; a < 3; a++) {
                float acc = 0.0f;
                for (int j = 0; j < 3; j++) { float t = R[3 * a + j] * s[j]; acc += t * t; }
                float h = rq * sqrtf(acc);
                L[a] = h * 1.0001f + 1e-6f * (fabsf(mu[a]) + h);
            }
            lo = make_float4(mu[0] - L[0], mu[1] - L[1], mu[2] - L[2], 0.0f);
            hi = make_float4(mu[0] + L[0], mu[1] + L[1], mu[2] + L[2], 0.0f);
        } else {
            lo = make_float4(INFINITY, INFINITY, INFINITY, 0.0f);
            hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.0f);
        }
        leafbox[2 * i] = lo;
        leafbox[2 * i + 1] = hi;
    }
}

// ------------------------------------------------------------------ Karras
__device__ __forceinline__ int delta(const uint64_t* __restrict__ k, int64_t n, int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    uint64_t a = k[i], b = k[j];
    if (a == b) return 64 + __clz((uint32_t)(i ^ j));
    return __clzll(a ^ b);
}

__global__ void k_karras(int64_t n, const uint64_t* __restrict__ keys, float4* __restrict__ nodes,
                         int32_t* __restrict__ parent) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n - 1; i += (int64_t)gridDim.x * blockDim.x) {
        const int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
        const int dmin = delta(keys, n, i, i - d);
        int64_t lmax = 2;
        while (delta(keys, n, i, i + lmax * d) > dmin) lmax *= 2;
        int64_t l = 0;
        for (int64_t t = lmax / 2; t >= 1; t /= 2)
            if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
        const int64_t j = i + l * d;
        const int dnode = delta(keys, n, i, j);
        int64_t s = 0;
        for (int64_t div = 2;; div *= 2) {
            int64_t t = (l + div - 1) / div;
            if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
            if (t <= 1) break;
        }
        const int64_t g = i + s * d + (d < 0 ? -1 : 0);
        const int64_t first = d > 0 ? i : j, last = d > 0 ? j : i;
        nodes[4 * i + 0].w = __int_as_float((int)first);
        nodes[4 * i + 1].w = __int_as_float((int)g);
        nodes[4 * i + 2].w = __int_as_float((int)last);
        nodes[4 * i + 3].w = 0.0f;
        // parents: leaves at [0, n), internal nodes at [n, 2n-1)
        if (first == g) parent[g] = (int)i; else parent[n + g] = (int)i;
        if (last == g + 1) parent[g + 1] = (int)i; else parent[n + g + 1] = (int)i;
    }
}

// Leaf i walks up; the second thread to reach a node unions its two child boxes.
__global__ void k_refit(int64_t n, const float4* __restrict__ leafbox, float4* nodes,
                        const int32_t* __restrict__ parent, int32_t* visit, float* root) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float4 lo = leafbox[2 * i], hi = leafbox[2 * i + 1];
        int64_t child = i;
        int node = parent[i];
        while (true) {
            const int split = __float_as_int(__ldcg(&nodes[4 * node + 1].w));
            // the left child of `node` is `split` (leaf or internal), the right child split+1
            const bool left = (child == split);
            float4* slo = &nodes[4 * node + (left ? 0 : 2)];
            float4* shi = &nodes[4 * node + (left ? 1 : 3)];
            slo->x = lo.x; slo->y = lo.y; slo->z = lo.z;
            shi->x = hi.x; shi->y = hi.y; shi->z = hi.z;
            __threadfence();
            if (atomicAdd(&visit[node], 1) == 0) break;
            __threadfence();
            float4 a0 = __ldcg(&nodes[4 * node + 0]), a1 = __ldcg(&nodes[4 * node + 1]);
            float4 a2 = __ldcg(&nodes[4 * node + 2]), a3 = __ldcg(&nodes[4 * node + 3]);
            lo = make_float4(fminf(a0.x, a2.x), fminf(a0.y, a2.y), fminf(a0.z, a2.z), 0.0f);
            hi = make_float4(fmaxf(a1.x, a3.x), fmaxf(a1.y, a3.y), fmaxf(a1.z, a3.z), 0.0f);
            if (node == 0) {
                root[0] = lo.x; root[1] = lo.y; root[2] = lo.z;
                root[3] = hi.x; root[4] = hi.y; root[5] = hi.z;
                break;
            }
            child = node;
            node = parent[n + node];
        }
    }
}

// n == 1: one node whose left child is leaf 0 and whose right child (leaf 1)
// has an empty box; the root box is leaf 0's box.
__global__ void k_single(const float4* __restrict__ leafbox, float4* nodes, float* root) {
    float4 lo = leafbox[0], hi = leafbox[1];
    nodes[0] = make_float4(lo.x, lo.y, lo.z, __int_as_float(0));
    nodes[1] = make_float4(hi.x, hi.y, hi.z, __int_as_float(0));
    nodes[2] = make_float4(INFINITY, INFINITY, INFINITY, __int_as_float(1));
    nodes[3] = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.0f);
    root[0] = lo.x; root[1] = lo.y; root[2] = lo.z; root[3] = hi.x; root[4] = hi.y; root[5] = hi.z;
}

// 4-wide traversal nodes.  Every internal node i of the binary radix tree gets a
// record of (up to) four children: its grandchildren, or a child itself where that
// child is a leaf.  A traversal that pushes the internal ids found in a record and
// later reads their records visits the binary tree two levels per fetch.  Each
// child is 16 B: its box (the refitted box, or a leaf's minimal AABB) as 6 halves
// rounded outward (lo down, hi up) and a ref = binary node id for an internal
// child, packed index | 0x80000000 for a leaf.  Unused slots, and empty Gaussians,
// hold an inverted box (lo = +inf, hi = -inf) that every ray misses.
__device__ __forceinline__ uint32_t pack_h2(__half a, __half b) {
    return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

__device__ __forceinline__ uint4 box_record(float4 lo, float4 hi, uint32_t ref) {
    return make_uint4(pack_h2(__float2half_rd(lo.x), __float2half_rd(lo.y)),
                      pack_h2(__float2half_rd(lo.z), __float2half_ru(hi.x)),
                      pack_h2(__float2half_ru(hi.y), __float2half_ru(hi.z)), ref);
}

__device__ __forceinline__ uint4 child_record(int64_t n, int morton, const int32_t* __restrict__ perm, float4 lo,
                                              float4 hi, bool leaf, int64_t c) {
    if (!leaf) return box_record(lo, hi, (uint32_t)c);
    if (c >= n)  // the missing second leaf of a 1-Gaussian tree
        return box_record(make_float4(INFINITY, INFINITY, INFINITY, 0.f), make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f),
                          0xffffffffu);
    const uint32_t p = morton ? (uint32_t)c : (uint32_t)perm[c];
    return box_record(lo, hi, p | 0x80000000u);
}

__global__ void k_widen(int64_t n_internal, int64_t n, int morton, const float4* __restrict__ nodes,
                        const int32_t* __restrict__ perm, uint4* __restrict__ nodew) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_internal; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a0 = nodes[4 * i], a1 = nodes[4 * i + 1], a2 = nodes[4 * i + 2], a3 = nodes[4 * i + 3];
        const int first = __float_as_int(a0.w), split = __float_as_int(a1.w), last = __float_as_int(a2.w);
        uint4 rec[4];
        int k = 0;
#pragma unroll
        for (int side = 0; side < 2; side++) {
            const int c = split + side;
            const bool leaf = side ? (c == last) : (first == c);
            if (leaf) {
                rec[k++] = side ? child_record(n, morton, perm, a2, a3, true, c)
                                : child_record(n, morton, perm, a0, a1, true, c);
            } else {
                const float4 c0 = nodes[4 * (int64_t)c], c1 = nodes[4 * (int64_t)c + 1];
                const float4 c2 = nodes[4 * (int64_t)c + 2], c3 = nodes[4 * (int64_t)c + 3];
                const int cf = __float_as_int(c0.w), cs = __float_as_int(c1.w), cl = __float_as_int(c2.w);
                rec[k++] = child_record(n, morton, perm, c0, c1, cf == cs, cs);
                rec[k++] = child_record(n, morton, perm, c2, c3, cs + 1 == cl, cs + 1);
            }
        }
        for (int j = k; j < 4; j++)
            rec[j] = box_record(make_float4(INFINITY, INFINITY, INFINITY, 0.f),
                                make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f), 0xffffffffu);
#pragma unroll
        for (int j = 0; j < 4; j++) nodew[4 * i + j] = rec[j];
    }
}

__global__ void k_empty_root(float* root) {
    root[0] = root[1] = root[2] = INFINITY;
    root[3] = root[4] = root[5] = -INFINITY;
}

// ------------------------------------------------------------------ host
static int grid_for(int64_t n, int threads, int num_sms) {
    int64_t b = (n + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

template <typename T>
static cudaError_t grow(T** p, size_t count) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    return cudaMalloc((void**)p, count * sizeof(T) + 256);
}

rgx_status rgx_internal_reserve(rgx_scene* s, int64_t n) {
    if (n <= s->cap_n && s->keys[0]) return RGX_OK;
    int64_t c = n < 1024 ? 1024 : n;
    cudaError_t e = cudaSuccess;
    e = e ? e : grow(&s->keys[0], c); e = e ? e : grow(&s->keys[1], c);
    e = e ? e : grow(&s->vals[0], c); e = e ? e : grow(&s->vals[1], c);
    e = e ? e : grow(&s->nodes, 4 * (size_t)c);
    e = e ? e : grow(&s->nodew, 4 * (size_t)c);
    e = e ? e : grow(&s->parent, 2 * (size_t)c);
    e = e ? e : grow(&s->visit, (size_t)c);
    e = e ? e : grow(&s->geom, 4 * (size_t)c);
    e = e ? e : grow(&s->shc, 12 * (size_t)c);
    e = e ? e : grow(&s->aux, 2 * (size_t)c);
    e = e ? e : grow(&s->perm, (size_t)c);
    e = e ? e : grow(&s->leafbox, 2 * (size_t)c);
    size_t hb = (size_t)256 * ((c + RS_TILE - 1) / RS_TILE);
    e = e ? e : grow(&s->hist, hb);
    if (e != cudaSuccess) {
        s->cap_n = 0;
        return set_err(s, RGX_ERR_WORKSPACE, "rgx_build_bvh: device allocation failed");
    }
    s->hist_cap = hb;
    s->cap_n = c;
    return RGX_OK;
}

// Spherical-Gaussian lobes in packed order: per lobe (u / |u|, lambda) and (a_rgb, 1 / |u|)
// from the caller's raw (u_x, u_y, u_z, lambda, a_r, a_g, a_b).  A lobe with a non-finite
// value, a zero axis or lambda < 0 is flagged and packed as zero.
__global__ void k_pack_sg(int64_t n, int n_sg, int morton, const float* __restrict__ sg,
                          const uint32_t* __restrict__ sorted_idx, float4* __restrict__ sgp,
                          unsigned int* __restrict__ status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t l = sorted_idx[i];
        const int64_t p = morton ? i : (int64_t)l;
        for (int j = 0; j < n_sg; j++) {
            const float* r = sg + ((int64_t)l * n_sg + j) * 7;
            const float ux = r[0], uy = r[1], uz = r[2], lam = r[3];
            const float nu = sqrtf(ux * ux + uy * uy + uz * uz);
            const bool ok = nu > 0.0f && isfinite(nu) && isfinite(lam) && lam >= 0.0f && isfinite(r[4]) &&
                            isfinite(r[5]) && isfinite(r[6]);
            if (!ok) atomicOr(status, (unsigned)RGX_ERR_BAD_PARAMS);
            const float inv = ok ? 1.0f / nu : 0.0f;
            sgp[2 * (p * n_sg + j) + 0] = ok ? make_float4(ux * inv, uy * inv, uz * inv, lam)
                                             : make_float4(0.f, 0.f, 1.f, 0.f);
            sgp[2 * (p * n_sg + j) + 1] = ok ? make_float4(r[4], r[5], r[6], inv) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

static rgx_status build_common(rgx_scene* s, int64_t n, int32_t sh_degree, const float* means,
                               const float* scales, const float* quats, const float* densities,
                               const float* sh, int32_t n_sg, const float* sg, const rgx_opts* opts,
                               void* stream_);

extern "C" rgx_status rgx_build_bvh(rgx_scene* s, int64_t n, int32_t sh_degree, const float* means,
                                    const float* scales, const float* quats, const float* densities,
                                    const float* sh, const rgx_opts* opts, void* stream_) {
    return build_common(s, n, sh_degree, means, scales, quats, densities, sh, 0, nullptr, opts, stream_);
}

extern "C" rgx_status rgx_build_bvh_sg(rgx_scene* s, int64_t n, int32_t sh_degree, const float* means,
                                       const float* scales, const float* quats, const float* densities,
                                       const float* sh, int32_t n_sg, const float* sg, const rgx_opts* opts,
                                       void* stream_) {
    if (n_sg < 0 || n_sg > RGX_MAX_SG) return set_err(s, RGX_ERR_INVALID_ARG, "rgx_build_bvh_sg: n_sg not in 0..7");
    if (n_sg > 0 && n > 0 && !sg) return set_err(s, RGX_ERR_INVALID_ARG, "rgx_build_bvh_sg: null sg");
    return build_common(s, n, sh_degree, means, scales, quats, densities, sh, n_sg, sg, opts, stream_);
}

static rgx_status build_common(rgx_scene* s, int64_t n, int32_t sh_degree, const float* means,
                               const float* scales, const float* quats, const float* densities,
                               const float* sh, int32_t n_sg, const float* sg, const rgx_opts* opts,
                               void* stream_) {
    if (!s || !opts) return set_err(s, RGX_ERR_INVALID_ARG, "rgx_build_bvh: null scene or opts");
    if (n < 0 || n >= (int64_t)0x7fffffff) return set_err(s, RGX_ERR_INVALID_ARG, "rgx_build_bvh: n out of range");
    if (sh_degree < 0 || sh_degree > 3) return set_err(s, RGX_ERR_INVALID_ARG, "rgx_build_bvh: sh_degree not in 0..3");
    if (n > 0 && (!means || !scales || !quats || !densities || !sh))
        return set_err(s, RGX_ERR_INVALID_ARG, "rgx_build_bvh: null parameter array");
    if (!(opts->sigma_eps > 0.0f)) return set_err(s, RGX_ERR_INVALID_ARG, "rgx_build_bvh: sigma_eps must be > 0");
    cudaStream_t st = (cudaStream_t)stream_;
    RGX_CUDA(s, cudaSetDevice(s->device));
    rgx_status r = rgx_internal_reserve(s, n);
    if (r != RGX_OK) return r;
    if (n_sg > 0 && s->sgp_cap < (size_t)n * n_sg * 2) {
        if (s->sgp) cudaFree(s->sgp);
        s->sgp = nullptr;
        s->sgp_cap = 0;
        if (cudaMalloc(&s->sgp, (size_t)n * n_sg * 2 * sizeof(float4)) != cudaSuccess)
            return set_err(s, RGX_ERR_WORKSPACE, "rgx_build_bvh_sg: lobe buffer allocation failed");
        s->sgp_cap = (size_t)n * n_sg * 2;
    }
    s->n = n;
    s->sh_degree = sh_degree;
    s->n_sg = n_sg;
    s->morton = (opts->flags & RGX_MORTON) ? 1 : 0;
    s->built = 1;
    if (n == 0) {
        k_empty_root<<<1, 1, 0, st>>>(s->root);
        RGX_CUDA(s, cudaGetLastError());
        return RGX_OK;
    }
    const int wide = (opts->flags & RGX_MORTON63) ? 1 : 0;
    const int T = 256;
    const int g = grid_for(n, T, s->num_sms);
    RGX_CUDA(s, cudaMemsetAsync(s->bounds, 0xff, 3 * sizeof(unsigned), st));
    RGX_CUDA(s, cudaMemsetAsync(s->bounds + 3, 0x00, 3 * sizeof(unsigned), st));
    k_bounds<<<g, T, 0, st>>>(n, means, scales, quats, densities, s->bounds, s->status);
    k_morton<<<g, T, 0, st>>>(n, means, s->bounds, wide, s->keys[0], s->vals[0]);
    // radix sort: 4 passes (30-bit codes) or 8 passes (63-bit)
    const int passes = wide ? 8 : 4;
    const int nb = (int)((n + RS_TILE - 1) / RS_TILE);
    int cur = 0;
    for (int p = 0; p < passes; p++) {
        const int shift = 8 * p;
        k_rs_hist<<<nb, RS_THREADS, 0, st>>>(s->keys[cur], n, shift, s->hist, nb);
        k_rs_scan<<<1, 1024, 0, st>>>(s->hist, 256 * nb);
        k_rs_scatter<<<nb, RS_THREADS, 0, st>>>(s->keys[cur], s->vals[cur], s->keys[cur ^ 1], s->vals[cur ^ 1], n,
                                                shift, s->hist, nb);
        cur ^= 1;
    }
    s->sorted_buf = cur;
    k_pack<<<g, T, 0, st>>>(n, sh_degree, opts->sigma_eps, s->morton, means, scales, quats, densities, sh,
                            s->vals[cur], s->perm, s->geom, s->shc, s->aux, s->leafbox, s->status);
    if (n_sg > 0) k_pack_sg<<<g, T, 0, st>>>(n, n_sg, s->morton, sg, s->vals[cur], s->sgp, s->status);
    if (n == 1) {
        k_single<<<1, 1, 0, st>>>(s->leafbox, s->nodes, s->root);
    } else {
        k_karras<<<grid_for(n - 1, T, s->num_sms), T, 0, st>>>(n, s->keys[cur], s->nodes, s->parent);
        RGX_CUDA(s, cudaMemsetAsync(s->visit, 0, (size_t)(n - 1) * sizeof(int32_t), st));
        k_refit<<<g, T, 0, st>>>(n, s->leafbox, s->nodes, s->parent, s->visit, s->root);
    }
    const int64_t ni = n > 1 ? n - 1 : 1;
    k_widen<<<grid_for(ni, T, s->num_sms), T, 0, st>>>(ni, n, s->morton, s->nodes, s->perm, s->nodew);
    RGX_CUDA(s, cudaGetLastError());
    return RGX_OK;
}

// ------------------------------------------------------------------ allocation-free variant
// rgx_morton_sort_noalloc runs the same bounds -> Morton code -> radix sort
// pipeline as rgx_build_bvh, but its scratch (two key/value ping-pong buffers,
// the digit histogram and the bounds) lives in the file-scope array below
// instead of a scene workspace, so the call allocates nothing.  The array is
// RGX_NOALLOC_BYTES (about 6.3 MB) on every GPU that loads the library, for
// the life of the process.
#define RGX_NOALLOC_MAX_N (1 << 18)
#define RGX_NOALLOC_NB ((RGX_NOALLOC_MAX_N + RS_TILE - 1) / RS_TILE)
#define RGX_NOALLOC_BYTES ((size_t)RGX_NOALLOC_MAX_N * (2 * 8 + 2 * 4) + (size_t)256 * RGX_NOALLOC_NB * 4 + 256)
static __device__ __align__(256) unsigned char g_noalloc_scratch[RGX_NOALLOC_BYTES];

#define RGX_MAX_DEVICES 64
// per device: the array's device address, looked up by the first call on that device;
// atomic, since two host threads may make that first call at the same time
static std::atomic<void*> g_noalloc_addr[RGX_MAX_DEVICES];

// per-axis min/max of the means only (no other parameter is read here)
__global__ void k_bounds_means(int64_t n, const float* __restrict__ means, unsigned int* __restrict__ bounds) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        for (int a = 0; a < 3; a++) {
            const float m = means[3 * l + a];
            lo[a] = fminf(lo[a], m);
            hi[a] = fmaxf(hi[a], m);
        }
    }
    for (int a = 0; a < 3; a++) {
        for (int off = 16; off > 0; off >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(FULLMASK, lo[a], off));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(FULLMASK, hi[a], off));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        for (int a = 0; a < 3; a++) {
            atomicMin(&bounds[a], f2ord(lo[a]));
            atomicMax(&bounds[3 + a], f2ord(hi[a]));
        }
    }
}

extern "C" rgx_status rgx_morton_sort_noalloc(int64_t n, const float* means, int32_t wide, uint64_t* codes,
                                              int32_t* perm, void* stream_) {
    if (n < 0 || n > RGX_NOALLOC_MAX_N)
        return set_err(nullptr, RGX_ERR_INVALID_ARG,
                       "rgx_morton_sort_noalloc: n must be in [0, 262144] (the size of its static scratch)");
    if (n > 0 && (!means || !codes || !perm))
        return set_err(nullptr, RGX_ERR_INVALID_ARG, "rgx_morton_sort_noalloc: null pointer");
    if (n == 0) return RGX_OK;
    int dev = 0;
    RGX_CUDA(nullptr, cudaGetDevice(&dev));
    if (dev < 0 || dev >= RGX_MAX_DEVICES)
        return set_err(nullptr, RGX_ERR_INVALID_ARG, "rgx_morton_sort_noalloc: device index too large");
    void* addr = g_noalloc_addr[dev].load(std::memory_order_relaxed);
    if (!addr) {
        // first call on this device: the host-side name of the array is not a
        // device address; ask the runtime for it (with this device current)
        RGX_CUDA(nullptr, cudaGetSymbolAddress(&addr, g_noalloc_scratch));
        g_noalloc_addr[dev].store(addr, std::memory_order_relaxed);
    }
    unsigned char* base = (unsigned char*)addr;
    uint64_t* keys[2] = {(uint64_t*)base, (uint64_t*)base + RGX_NOALLOC_MAX_N};
    uint32_t* vals0 = (uint32_t*)(base + (size_t)RGX_NOALLOC_MAX_N * 16);
    uint32_t* vals[2] = {vals0, vals0 + RGX_NOALLOC_MAX_N};
    uint32_t* hist = vals0 + 2 * (size_t)RGX_NOALLOC_MAX_N;
    unsigned int* bounds = (unsigned int*)(hist + (size_t)256 * RGX_NOALLOC_NB);
    cudaStream_t st = (cudaStream_t)stream_;
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int T = 256;
    const int g = grid_for(n, T, nsm);
    // the array keeps the previous call's contents: the bounds must restart
    RGX_CUDA(nullptr, cudaMemsetAsync(bounds, 0xff, 3 * sizeof(unsigned), st));
    RGX_CUDA(nullptr, cudaMemsetAsync(bounds + 3, 0x00, 3 * sizeof(unsigned), st));
    k_bounds_means<<<g, T, 0, st>>>(n, means, bounds);
    k_morton<<<g, T, 0, st>>>(n, means, bounds, wide ? 1 : 0, keys[0], vals[0]);
    const int passes = wide ? 8 : 4;
    const int nb = (int)((n + RS_TILE - 1) / RS_TILE);
    int cur = 0;
    for (int p = 0; p < passes; p++) {
        k_rs_hist<<<nb, RS_THREADS, 0, st>>>(keys[cur], n, 8 * p, hist, nb);
        k_rs_scan<<<1, 1024, 0, st>>>(hist, 256 * nb);
        k_rs_scatter<<<nb, RS_THREADS, 0, st>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n, 8 * p, hist, nb);
        cur ^= 1;
    }
    RGX_CUDA(nullptr, cudaMemcpyAsync(codes, keys[cur], (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    RGX_CUDA(nullptr, cudaMemcpyAsync(perm, vals[cur], (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    RGX_CUDA(nullptr, cudaGetLastError());
    return RGX_OK;
}
