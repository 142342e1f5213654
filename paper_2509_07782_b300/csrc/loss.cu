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

// ------------------------------------------------------------------ image loss of the training step
// Sec. 3.4: L = (1 - lambda) L1 + lambda DSSIM per view, on the composited RGB.  Readings:
// DSSIM = 1 - SSIM; SSIM with an 11 x 11 Gaussian window (standard deviation 1.5),
// C1 = 0.01^2, C2 = 0.03^2, zero padding outside the image, averaged over pixels and
// channels, like L1.  The window is separable, so every 2-D window sum is a row pass
// then a column pass.  The gradient of mean SSIM with respect to pixel p is
//   (1/n) sum_q w(q - p) [dS/dmu_x + 2 x_p dS/dE[x^2] + y_p dS/dE[xy]]_q,
// i.e. the same window applied to three per-pixel maps.  All views of a batch run in
// one launch per pass; scratch (24 floats per pixel) is scene workspace.
#define SSIM_R 5

__constant__ float c_ssim_w[2 * SSIM_R + 1];

struct LossViews {
    int ncam;
    uint32_t pix0[RGX_MAX_CAMS + 1];  // pixel prefix
    int w[RGX_MAX_CAMS], h[RGX_MAX_CAMS];
};

__device__ __forceinline__ int view_of(const LossViews& V, uint32_t i) {
    int lo = 0, hi = V.ncam;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (V.pix0[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// pass 1: row sums of x, y, x^2, y^2, xy per channel -> h [15][R]
__global__ void k_ssim_rows5(const __grid_constant__ LossViews V, const float4* __restrict__ rgba,
                             const float* __restrict__ tgt, float* __restrict__ h, uint32_t R) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < R; i += gridDim.x * blockDim.x) {
        const int c = view_of(V, i);
        const uint32_t base = V.pix0[c], loc = i - base;
        const int W = V.w[c], x = (int)(loc % (uint32_t)W);
        float acc[15];
#pragma unroll
        for (int k = 0; k < 15; k++) acc[k] = 0.f;
        for (int d = -SSIM_R; d <= SSIM_R; d++) {
            const int xx = x + d;
            if (xx < 0 || xx >= W) continue;
            const uint32_t j = i + d;
            const float wk = c_ssim_w[d + SSIM_R];
            const float4 pv = rgba[j];
            const float pa[3] = {pv.x, pv.y, pv.z};
#pragma unroll
            for (int ch = 0; ch < 3; ch++) {
                const float a = pa[ch], b = tgt[3 * (size_t)j + ch];
                acc[5 * ch + 0] += wk * a;
                acc[5 * ch + 1] += wk * b;
                acc[5 * ch + 2] += wk * a * a;
                acc[5 * ch + 3] += wk * b * b;
                acc[5 * ch + 4] += wk * a * b;
            }
        }
#pragma unroll
        for (int k = 0; k < 15; k++) h[(size_t)k * R + i] = acc[k];
    }
}

// pass 2: column sums -> local statistics -> SSIM and its three partials per channel
// (abc [9][R]); per-view sums of SSIM and |x - y| into sums[2 * ncam] (double)
__global__ void k_ssim_cols5(const __grid_constant__ LossViews V, const float4* __restrict__ rgba,
                             const float* __restrict__ tgt, const float* __restrict__ h, float* __restrict__ abc,
                             double* __restrict__ sums, uint32_t R) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < R; i += gridDim.x * blockDim.x) {
        const int c = view_of(V, i);
        const uint32_t base = V.pix0[c], loc = i - base;
        const int W = V.w[c], H = V.h[c], y = (int)(loc / (uint32_t)W);
        float m[15];
#pragma unroll
        for (int k = 0; k < 15; k++) m[k] = 0.f;
        for (int d = -SSIM_R; d <= SSIM_R; d++) {
            const int yy = y + d;
            if (yy < 0 || yy >= H) continue;
            const uint32_t j = (uint32_t)((int64_t)i + (int64_t)d * W);
            const float wk = c_ssim_w[d + SSIM_R];
#pragma unroll
            for (int k = 0; k < 15; k++) m[k] += wk * h[(size_t)k * R + j];
        }
        const float4 pv = rgba[i];
        const float pa[3] = {pv.x, pv.y, pv.z};
        float s_sum = 0.f, l1 = 0.f;
#pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            const float mx = m[5 * ch], my = m[5 * ch + 1], exx = m[5 * ch + 2], eyy = m[5 * ch + 3],
                        exy = m[5 * ch + 4];
            const float vx = exx - mx * mx, vy = eyy - my * my, cxy = exy - mx * my;
            const float A1 = 2.f * mx * my + 1e-4f, A2 = 2.f * cxy + 9e-4f;
            const float B1 = mx * mx + my * my + 1e-4f, B2 = vx + vy + 9e-4f;
            const float S = A1 * A2 / (B1 * B2);
            abc[(size_t)(3 * ch + 0) * R + i] = S * (2.f * my / A1 - 2.f * my / A2 - 2.f * mx / B1 + 2.f * mx / B2);
            abc[(size_t)(3 * ch + 1) * R + i] = -S / B2;
            abc[(size_t)(3 * ch + 2) * R + i] = 2.f * S / A2;
            s_sum += S;
            l1 += fabsf(pa[ch] - tgt[3 * (size_t)i + ch]);
        }
        atomicAdd(&sums[2 * c], (double)s_sum);
        atomicAdd(&sums[2 * c + 1], (double)l1);
    }
}

// pass 3: row sums of the nine partial maps -> h [9][R]
__global__ void k_ssim_rows3(const __grid_constant__ LossViews V, const float* __restrict__ abc,
                             float* __restrict__ h, uint32_t R) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < R; i += gridDim.x * blockDim.x) {
        const int c = view_of(V, i);
        const uint32_t loc = i - V.pix0[c];
        const int W = V.w[c], x = (int)(loc % (uint32_t)W);
        float acc[9];
#pragma unroll
        for (int k = 0; k < 9; k++) acc[k] = 0.f;
        for (int d = -SSIM_R; d <= SSIM_R; d++) {
            const int xx = x + d;
            if (xx < 0 || xx >= W) continue;
            const float wk = c_ssim_w[d + SSIM_R];
#pragma unroll
            for (int k = 0; k < 9; k++) acc[k] += wk * abc[(size_t)k * R + i + d];
        }
#pragma unroll
        for (int k = 0; k < 9; k++) h[(size_t)k * R + i] = acc[k];
    }
}

// pass 4: column sums of the partial maps -> dL/d rgba (opacity gets 0)
__global__ void k_ssim_grad(const __grid_constant__ LossViews V, const float4* __restrict__ rgba,
                            const float* __restrict__ tgt, const float* __restrict__ h, float lam,
                            float4* __restrict__ d_rgba, uint32_t R) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < R; i += gridDim.x * blockDim.x) {
        const int c = view_of(V, i);
        const uint32_t loc = i - V.pix0[c];
        const int W = V.w[c], H = V.h[c], y = (int)(loc / (uint32_t)W);
        float m[9];
#pragma unroll
        for (int k = 0; k < 9; k++) m[k] = 0.f;
        for (int d = -SSIM_R; d <= SSIM_R; d++) {
            const int yy = y + d;
            if (yy < 0 || yy >= H) continue;
            const uint32_t j = (uint32_t)((int64_t)i + (int64_t)d * W);
            const float wk = c_ssim_w[d + SSIM_R];
#pragma unroll
            for (int k = 0; k < 9; k++) m[k] += wk * h[(size_t)k * R + j];
        }
        const float inv_n = 1.0f / (3.0f * (float)W * (float)H);
        const float4 pv = rgba[i];
        const float pa[3] = {pv.x, pv.y, pv.z};
        float g[3];
#pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            const float x = pa[ch], t = tgt[3 * (size_t)i + ch];
            const float sgn = (float)((x > t) - (x < t));
            const float dS = (m[3 * ch] + 2.f * x * m[3 * ch + 1] + t * m[3 * ch + 2]) * inv_n;
            g[ch] = (1.f - lam) * sgn * inv_n - lam * dS;
        }
        d_rgba[i] = make_float4(g[0], g[1], g[2], 0.f);
    }
}

// per view: loss[c] += (1 - lam) L1_c + lam (1 - SSIM_c)
__global__ void k_image_loss_total(const __grid_constant__ LossViews V, const double* __restrict__ sums, float lam,
                                   float* __restrict__ loss) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= V.ncam) return;
    const double n = 3.0 * (double)V.w[c] * (double)V.h[c];
    loss[c] += (float)((1.0 - lam) * sums[2 * c + 1] / n + lam * (1.0 - sums[2 * c] / n));
}

extern "C" rgx_status rgx_image_loss(rgx_scene* s, const rgx_camera* cams, int32_t ncam, const float* rgba,
                                     const float* target, float lambda, float* loss, float* d_rgba, void* stream) {
    if (!s || !cams || ncam <= 0 || ncam > RGX_MAX_CAMS || !rgba || !target || !loss || !d_rgba)
        return set_err(s, RGX_ERR_INVALID_ARG, "rgx_image_loss: bad arguments");
    if (!(lambda >= 0.0f && lambda <= 1.0f)) return set_err(s, RGX_ERR_INVALID_ARG, "rgx_image_loss: lambda not in [0,1]");
    LossViews V;
    V.ncam = ncam;
    uint64_t R = 0;
    for (int c = 0; c < ncam; c++) {
        if (cams[c].width <= 0 || cams[c].height <= 0)
            return set_err(s, RGX_ERR_INVALID_ARG, "rgx_image_loss: camera with zero size");
        V.pix0[c] = (uint32_t)R;
        V.w[c] = cams[c].width;
        V.h[c] = cams[c].height;
        R += (uint64_t)cams[c].width * cams[c].height;
    }
    if (R >= 0x7fffffffull) return set_err(s, RGX_ERR_INVALID_ARG, "rgx_image_loss: too many pixels");
    V.pix0[ncam] = (uint32_t)R;
    RGX_CUDA(s, cudaSetDevice(s->device));
    cudaStream_t st = (cudaStream_t)stream;
    // scratch: 15 + 9 floats per pixel, and 2 doubles per view
    const size_t need = (size_t)R * 24 * sizeof(float) + (size_t)2 * RGX_MAX_CAMS * sizeof(double);
    if (s->loss_cap < need) {
        if (s->loss_ws) cudaFree(s->loss_ws);
        s->loss_ws = nullptr;
        s->loss_cap = 0;
        if (cudaMalloc(&s->loss_ws, need) != cudaSuccess)
            return set_err(s, RGX_ERR_WORKSPACE, "rgx_image_loss: scratch allocation failed");
        s->loss_cap = need;
    }
    if (!s->ssim_w_set) {
        float w[2 * SSIM_R + 1], tot = 0.f;
        for (int k = -SSIM_R; k <= SSIM_R; k++) tot += (w[k + SSIM_R] = expf(-(float)(k * k) / (2.0f * 1.5f * 1.5f)));
        for (int k = 0; k < 2 * SSIM_R + 1; k++) w[k] /= tot;
        RGX_CUDA(s, cudaMemcpyToSymbol(c_ssim_w, w, sizeof w));
        s->ssim_w_set = 1;
    }
    float* h = (float*)s->loss_ws;
    float* abc = h + (size_t)R * 15;
    double* sums = (double*)(abc + (size_t)R * 9);
    const uint32_t RR = (uint32_t)R;
    int grid = (int)((R + 255) / 256);
    if (grid > s->num_sms * 32) grid = s->num_sms * 32;
    RGX_CUDA(s, cudaMemsetAsync(sums, 0, 2 * (size_t)ncam * sizeof(double), st));
    k_ssim_rows5<<<grid, 256, 0, st>>>(V, (const float4*)rgba, target, h, RR);
    k_ssim_cols5<<<grid, 256, 0, st>>>(V, (const float4*)rgba, target, h, abc, sums, RR);
    k_ssim_rows3<<<grid, 256, 0, st>>>(V, abc, h, RR);
    k_ssim_grad<<<grid, 256, 0, st>>>(V, (const float4*)rgba, target, h, lambda, (float4*)d_rgba, RR);
    k_image_loss_total<<<(ncam + 127) / 128, 128, 0, st>>>(V, sums, lambda, loss);
    RGX_CUDA(s, cudaGetLastError());
    return RGX_OK;
}
