// train.cu -- optimiser and adaptive density control of the training step.
//
// rgx_adam_step: one Adam step (Kingma & Ba 2015) on one parameter tensor, with the
// exponential parameterisation of scales and densities folded in: the optimiser's
// variable is log(value), the gradient given is d/d value, so the variable's gradient
// is grad * exp(param), and the new exp(param) is written for the next BVH build.
//
// rgx_densify_plan / rgx_densify_apply: adaptive density control driven by the
// criterion of Sec. 3.5, Eq. 11 (stat / count > tau, Sec. 4.2: tau = 1.5e-4).  The
// paper keeps the clone/split heuristic of the methods it builds on; the reading
// taken: a Gaussian over the threshold is cloned (kept, plus an identical copy) when
// its largest scale is at most size_threshold, else split into two children drawn
// from it -- mean mu + R(q) (s * z_k) with z_k ~ N(0, I) supplied by the caller,
// scales s / 1.6, rotation, density and colour unchanged -- which replace it.
#include <stdio.h>
#include "common.cuh"

__global__ void k_adam(int64_t n, float* __restrict__ param, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                       int exp_param, float* __restrict__ activated) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float p = param[i];
        float g = grad[i];
        if (exp_param) g *= expf(p);
        const float mi = b1 * m[i] + (1.0f - b1) * g;
        const float vi = b2 * v[i] + (1.0f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        p -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        param[i] = p;
        if (activated) activated[i] = exp_param ? expf(p) : p;
    }
}

static int grid_n(int64_t n, int sms) {
    int64_t b = (n + 255) / 256;
    if (b > (int64_t)sms * 16) b = (int64_t)sms * 16;
    return (int)(b < 1 ? 1 : b);
}

extern "C" rgx_status rgx_adam_step(int64_t n, float* param, const float* grad, float* m, float* v, float lr,
                                    float beta1, float beta2, float eps, int32_t step, int32_t exp_param,
                                    float* activated, void* stream) {
    if (n < 0 || (n > 0 && (!param || !grad || !m || !v)) || step < 1 || !(beta1 >= 0.f && beta1 < 1.f) ||
        !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return set_err(nullptr, RGX_ERR_INVALID_ARG, "rgx_adam_step: bad arguments");
    if (n == 0) return RGX_OK;
    const float c1 = (float)(1.0 - pow((double)beta1, (double)step));
    const float c2 = (float)(1.0 - pow((double)beta2, (double)step));
    int sms = 148;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_adam<<<grid_n(n, sms), 256, 0, (cudaStream_t)stream>>>(n, param, grad, m, v, lr, beta1, beta2, eps, c1, c2,
                                                             exp_param, activated);
    RGX_CUDA(nullptr, cudaGetLastError());
    return RGX_OK;
}

// ------------------------------------------------------------------ densification
// action: 0 keep, 1 clone, 2 split; outputs per Gaussian: 1, 2, 2
__global__ void k_densify_action(int64_t n, const float* __restrict__ stat, const int32_t* __restrict__ count,
                                 const float* __restrict__ scales, float tau, float size_thr,
                                 int32_t* __restrict__ action, int32_t* __restrict__ nout) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        int a = 0;
        const int c = count[l];
        if (c > 0 && stat[l] / (float)c > tau) {
            const float smax = fmaxf(fmaxf(scales[3 * l], scales[3 * l + 1]), scales[3 * l + 2]);
            a = smax <= size_thr ? 1 : 2;
        }
        action[l] = a;
        nout[l] = a == 0 ? 1 : 2;
    }
}

// Exclusive scan, three steps: per block of 1024 elements (in place), the block sums,
// then the block offsets added back.
__global__ void k_scan_blocks(int64_t n, int32_t* __restrict__ x, int32_t* __restrict__ bsum) {
    __shared__ int32_t wsum[32];
    const int64_t i = blockIdx.x * (int64_t)1024 + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int32_t v = i < n ? x[i] : 0;
    int32_t s = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, s, d);
        if (lane >= d) s += t;
    }
    if (lane == 31) wsum[wid] = s;
    __syncthreads();
    if (wid == 0) {
        int32_t w = wsum[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += t;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    const int32_t before = wid > 0 ? wsum[wid - 1] : 0;
    if (i < n) x[i] = before + s - v;
    if (threadIdx.x == 1023) bsum[blockIdx.x] = before + s;
}

__global__ void k_scan_sums(int64_t nb, int32_t* __restrict__ bsum, int64_t* __restrict__ total) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t acc = 0;
    for (int64_t b = 0; b < nb; b++) {
        const int32_t v = bsum[b];
        bsum[b] = (int32_t)acc;
        acc += v;
    }
    *total = acc;
}

__global__ void k_scan_add(int64_t n, int32_t* __restrict__ x, const int32_t* __restrict__ bsum) {
    const int64_t i = blockIdx.x * (int64_t)1024 + threadIdx.x;
    if (i < n) x[i] += bsum[blockIdx.x];
}

extern "C" rgx_status rgx_densify_plan(rgx_scene* s, int64_t n, const float* stat, const int32_t* count,
                                       const float* scales, float tau, float size_threshold, int32_t* action,
                                       int32_t* offset, int64_t* n_out, void* stream) {
    if (!s || n < 0 || n >= (int64_t)0x3fffffff || !n_out ||
        (n > 0 && (!stat || !count || !scales || !action || !offset)))
        return set_err(s, RGX_ERR_INVALID_ARG, "rgx_densify_plan: bad arguments");
    *n_out = 0;
    if (n == 0) return RGX_OK;
    cudaStream_t st = (cudaStream_t)stream;
    RGX_CUDA(s, cudaSetDevice(s->device));
    const int64_t nb = (n + 1023) / 1024;
    const size_t need = (size_t)nb * sizeof(int32_t) + sizeof(int64_t);
    if (s->plan_cap < need) {
        if (s->plan_ws) cudaFree(s->plan_ws);
        s->plan_ws = nullptr;
        s->plan_cap = 0;
        if (cudaMalloc(&s->plan_ws, need) != cudaSuccess)
            return set_err(s, RGX_ERR_WORKSPACE, "rgx_densify_plan: scratch allocation failed");
        s->plan_cap = need;
    }
    int64_t* total = (int64_t*)s->plan_ws;
    int32_t* bsum = (int32_t*)(total + 1);
    k_densify_action<<<grid_n(n, s->num_sms), 256, 0, st>>>(n, stat, count, scales, tau, size_threshold, action,
                                                            offset);
    k_scan_blocks<<<(int)nb, 1024, 0, st>>>(n, offset, bsum);
    k_scan_sums<<<1, 32, 0, st>>>(nb, bsum, total);
    k_scan_add<<<(int)nb, 1024, 0, st>>>(n, offset, bsum);
    RGX_CUDA(s, cudaGetLastError());
    int64_t h = 0;
    RGX_CUDA(s, cudaMemcpyAsync(&h, total, sizeof h, cudaMemcpyDeviceToHost, st));
    RGX_CUDA(s, cudaStreamSynchronize(st));
    *n_out = h;
    return RGX_OK;
}

__global__ void k_densify_apply(int64_t n, const int32_t* __restrict__ action, const int32_t* __restrict__ offset,
                                const float* __restrict__ normals, const float* __restrict__ means,
                                const float* __restrict__ scales, const float* __restrict__ quats,
                                const float* __restrict__ dens, const float* __restrict__ sh, int nsh,
                                const float* __restrict__ sg, int nsg, float* __restrict__ om,
                                float* __restrict__ os, float* __restrict__ oq, float* __restrict__ od,
                                float* __restrict__ osh, float* __restrict__ osg, int32_t* __restrict__ osrc) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const int a = action[l];
        const int64_t o = offset[l];
        const int k_out = a == 0 ? 1 : 2;
        const float qw = quats[4 * l], qx = quats[4 * l + 1], qy = quats[4 * l + 2], qz = quats[4 * l + 3];
        const float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        const float w = qw / qn, x = qx / qn, y = qy / qn, z = qz / qn;
        const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                            2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                            2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
        for (int k = 0; k < k_out; k++) {
            const int64_t d = o + k;
            float mu[3] = {means[3 * l], means[3 * l + 1], means[3 * l + 2]};
            float sc[3] = {scales[3 * l], scales[3 * l + 1], scales[3 * l + 2]};
            if (a == 2) {
                const float* zk = normals + 6 * l + 3 * k;
                const float t0 = sc[0] * zk[0], t1 = sc[1] * zk[1], t2 = sc[2] * zk[2];
                for (int r = 0; r < 3; r++) mu[r] += R[3 * r] * t0 + R[3 * r + 1] * t1 + R[3 * r + 2] * t2;
                for (int r = 0; r < 3; r++) sc[r] = sc[r] / 1.6f;
            }
            for (int r = 0; r < 3; r++) { om[3 * d + r] = mu[r]; os[3 * d + r] = sc[r]; }
            for (int r = 0; r < 4; r++) oq[4 * d + r] = quats[4 * l + r];
            od[d] = dens[l];
            for (int r = 0; r < nsh; r++) osh[d * nsh + r] = sh[l * nsh + r];
            for (int r = 0; r < nsg; r++) osg[d * nsg + r] = sg[l * nsg + r];
            if (osrc) osrc[d] = (int32_t)l;
        }
    }
}

extern "C" rgx_status rgx_densify_apply(int64_t n, const int32_t* action, const int32_t* offset, const float* normals,
                                        const float* means, const float* scales, const float* quats,
                                        const float* densities, const float* sh, int32_t sh_floats, const float* sg,
                                        int32_t sg_floats, float* out_means, float* out_scales, float* out_quats,
                                        float* out_densities, float* out_sh, float* out_sg, int32_t* out_src,
                                        void* stream) {
    if (n < 0 || sh_floats < 0 || sh_floats > 48 || sg_floats < 0 || sg_floats > 7 * RGX_MAX_SG ||
        (n > 0 && (!action || !offset || !normals || !means || !scales || !quats || !densities ||
                   (sh_floats && (!sh || !out_sh)) || (sg_floats && (!sg || !out_sg)) || !out_means ||
                   !out_scales || !out_quats || !out_densities)))
        return set_err(nullptr, RGX_ERR_INVALID_ARG, "rgx_densify_apply: bad arguments");
    if (n == 0) return RGX_OK;
    int sms = 148, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_densify_apply<<<grid_n(n, sms), 256, 0, (cudaStream_t)stream>>>(
        n, action, offset, normals, means, scales, quats, densities, sh, sh_floats, sg, sg_floats, out_means,
        out_scales, out_quats, out_densities, out_sh, out_sg, out_src);
    RGX_CUDA(nullptr, cudaGetLastError());
    return RGX_OK;
}
