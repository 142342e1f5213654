// api.cu -- scene lifecycle, status word and introspection entry points.
#include <stdio.h>
#include "common.cuh"

extern char g_rgx_last_error[256];

extern "C" rgx_status rgx_scene_create(rgx_scene** out, int32_t device) {
    if (!out) return set_err(nullptr, RGX_ERR_INVALID_ARG, "rgx_scene_create: null out");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return set_err(nullptr, RGX_ERR_INVALID_ARG, "rgx_scene_create: no such CUDA device");
    rgx_scene* s = new rgx_scene();
    s->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&s->bounds, 8 * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&s->root, 8 * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&s->queue, 4 * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&s->status, sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&s->counters, 8 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(s->status, 0, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(s->counters, 0, 8 * sizeof(unsigned long long)) != cudaSuccess) {
        rgx_scene_destroy(s);
        return set_err(nullptr, RGX_ERR_WORKSPACE, "rgx_scene_create: device allocation failed");
    }
    *out = s;
    return RGX_OK;
}

extern "C" rgx_status rgx_scene_destroy(rgx_scene* s) {
    if (!s) return RGX_OK;
    cudaSetDevice(s->device);
    void* ptrs[] = {s->keys[0], s->keys[1], s->vals[0], s->vals[1], s->hist, s->nodes, s->nodew, s->parent, s->visit,
                    s->geom, s->shc, s->aux, s->perm, s->leafbox, s->bounds, s->root, s->grad, s->cams,
                    s->queue, s->status, s->counters, s->spill, s->tape, s->vgrad, s->sgp, s->gsg, s->loss_ws, s->plan_ws, s->csums, s->ptape};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete s;
    return RGX_OK;
}

extern "C" rgx_status rgx_sync_status(rgx_scene* s, void* stream) {
    if (!s) return set_err(nullptr, RGX_ERR_INVALID_ARG, "rgx_sync_status: null scene");
    cudaStream_t st = (cudaStream_t)stream;
    RGX_CUDA(s, cudaSetDevice(s->device));
    unsigned v = 0;
    RGX_CUDA(s, cudaMemcpyAsync(&v, s->status, sizeof v, cudaMemcpyDeviceToHost, st));
    RGX_CUDA(s, cudaMemsetAsync(s->status, 0, sizeof v, st));
    RGX_CUDA(s, cudaStreamSynchronize(st));
    if (v) {
        char m[128];
        snprintf(m, sizeof m, "device status 0x%x", v);
        set_err(s, (rgx_status)v, m);
    }
    return (rgx_status)v;
}

extern "C" size_t rgx_fwd_state_bytes(void) { return 32; }

extern "C" const char* rgx_last_error(const rgx_scene* s) { return s ? s->last_error : g_rgx_last_error; }

extern "C" rgx_status rgx_get_bvh(rgx_scene* s, uint64_t* codes, int32_t* perm, float* nodes, float* root,
                                  void* stream) {
    if (!s) return set_err(nullptr, RGX_ERR_INVALID_ARG, "rgx_get_bvh: null scene");
    if (!s->built) return set_err(s, RGX_ERR_NOT_BUILT, "rgx_get_bvh before rgx_build_bvh");
    cudaStream_t st = (cudaStream_t)stream;
    RGX_CUDA(s, cudaSetDevice(s->device));
    const int64_t n = s->n;
    if (codes && n > 0)
        RGX_CUDA(s, cudaMemcpyAsync(codes, s->keys[s->sorted_buf], n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    if (perm && n > 0) RGX_CUDA(s, cudaMemcpyAsync(perm, s->perm, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    if (nodes && n > 0) {
        const int64_t nn = n > 1 ? n - 1 : 1;
        RGX_CUDA(s, cudaMemcpyAsync(nodes, s->nodes, nn * 4 * sizeof(float4), cudaMemcpyDeviceToDevice, st));
    }
    if (root) RGX_CUDA(s, cudaMemcpyAsync(root, s->root, 6 * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return RGX_OK;
}

extern "C" rgx_status rgx_get_counters(rgx_scene* s, uint64_t* out8, void* stream) {
    if (!s || !out8) return set_err(s, RGX_ERR_INVALID_ARG, "rgx_get_counters: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    RGX_CUDA(s, cudaSetDevice(s->device));
    unsigned long long v[8];
    RGX_CUDA(s, cudaMemcpyAsync(v, s->counters, sizeof v, cudaMemcpyDeviceToHost, st));
    RGX_CUDA(s, cudaStreamSynchronize(st));
    for (int i = 0; i < 8; i++) out8[i] = v[i];
    return RGX_OK;
}
