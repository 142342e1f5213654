// loss.cu -- per-Gaussian training terms around the march.
//
// rgx_isotropic_loss (Sec. 3.4, Eqs. 6-8): L_s = 1/N sum_l max(r_max,l - r0, 0)
// with r_max = 2/(pi sqrt 3) |s|^3 / (s1 s2 s3), the rotation-independent bound
// of the AABB / ellipsoid volume ratio (Supp. Sec. 2.3); its gradient with
// respect to the linear scales is r_max (3 s_j / |s|^2 - 1 / s_j) where active.
//
// rgx_densify_accumulate (Sec. 3.5, Eq. 11): after the adjoint of one view i,
// every Gaussian with a non-zero mean gradient adds |mu - o_i| / f_i * |grad mu|
// to its statistic and one to its view count.
#include <stdio.h>
#include "common.cuh"

#define ISO_K 0.36755259694786136f  // 2 / (pi sqrt 3)

__global__ void k_isotropic(int64_t n, const float* __restrict__ s, float r0, float w_over_n,
                            float* __restrict__ loss, float* __restrict__ ds) {
    float acc = 0.0f;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const float a = s[3 * l], b = s[3 * l + 1], c = s[3 * l + 2];
        const float ss = a * a + b * b + c * c;
        const float r = ISO_K * ss * sqrtf(ss) / (a * b * c);
        if (r > r0) {
            acc += r - r0;
            const float k3 = 3.0f / ss;
            ds[3 * l + 0] += w_over_n * r * (k3 * a - 1.0f / a);
            ds[3 * l + 1] += w_over_n * r * (k3 * b - 1.0f / b);
            ds[3 * l + 2] += w_over_n * r * (k3 * c - 1.0f / c);
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0 && v != 0.0f) atomicAdd(loss, w_over_n * v);
    }
}

__global__ void k_densify(int64_t n, const float* __restrict__ mu, const float* __restrict__ g, float ox, float oy,
                          float oz, float inv_f, float* __restrict__ stat, int32_t* __restrict__ count) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const float gx = g[3 * l], gy = g[3 * l + 1], gz = g[3 * l + 2];
        const float gn = sqrtf(gx * gx + gy * gy + gz * gz);
        if (gn > 0.0f) {
            const float dx = mu[3 * l] - ox, dy = mu[3 * l + 1] - oy, dz = mu[3 * l + 2] - oz;
            stat[l] += sqrtf(dx * dx + dy * dy + dz * dz) * inv_f * gn;
            count[l] += 1;
        }
    }
}

static int grid_of(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    return (int)(b < 1 ? 1 : b);
}

extern "C" rgx_status rgx_isotropic_loss(int64_t n, const float* scales, float r0, float weight, float* loss,
                                         float* d_scales, void* stream) {
    if (n < 0 || (n > 0 && (!scales || !loss || !d_scales)))
        return set_err(nullptr, RGX_ERR_INVALID_ARG, "rgx_isotropic_loss: bad arguments");
    if (n == 0) return RGX_OK;
    k_isotropic<<<grid_of(n), 256, 0, (cudaStream_t)stream>>>(n, scales, r0, weight / (float)n, loss, d_scales);
    RGX_CUDA(nullptr, cudaGetLastError());
    return RGX_OK;
}

extern "C" rgx_status rgx_densify_accumulate(int64_t n, const float* means, const float* d_means,
                                             const rgx_camera* cam, float* stat, int32_t* count, void* stream) {
    if (n < 0 || !cam || (n > 0 && (!means || !d_means || !stat || !count)))
        return set_err(nullptr, RGX_ERR_INVALID_ARG, "rgx_densify_accumulate: bad arguments");
    if (!(cam->fx > 0.0f)) return set_err(nullptr, RGX_ERR_INVALID_ARG, "rgx_densify_accumulate: fx must be > 0");
    if (n == 0) return RGX_OK;
    k_densify<<<grid_of(n), 256, 0, (cudaStream_t)stream>>>(n, means, d_means, cam->c2w[3], cam->c2w[7],
                                                           cam->c2w[11], 1.0f / cam->fx, stat, count);
    RGX_CUDA(nullptr, cudaGetLastError());
    return RGX_OK;
}
