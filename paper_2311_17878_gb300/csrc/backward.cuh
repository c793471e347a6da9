// Shared by the two backward paths of render_rays: the FP32 SIMT one that walks
// both networks a tile of samples at a time (backward.cu) and the layer-major
// one whose layers are GEMMs over a chunk of samples on the tensor cores
// (backward_gemm.cu).  Not part of the C ABI.
#pragma once
#include "common.cuh"

namespace tsdfs {

// per-sample adjoints produced by the compositing backward: of f, of grad f, of the colour
struct __align__(16) SampleAdj {
    float gf, ggx, ggy, ggz;
    float gr, gg, gb, pad;
};

// id of the calling thread's current CUDA context (abi.cu)
unsigned long long current_context_id();

// compositing backward (one thread per ray): per-sample records -> per-sample adjoints
int launch_comp_bwd(const SampleRec* rec, const int32_t* offsets, const uint8_t* status, const float* ray_d,
                    int64_t n_rays, const tsdfs_mlp* mlp, const float* d_rgb, const float* d_depth,
                    const float* d_eik, SampleAdj* adj, cudaStream_t st);

// samples per chunk of the layer-major path set by tsdfs_set_backward_chunk (0: sized
// by the path's default chunk bytes)
int64_t backward_chunk_setting();

// the layer-major path (backward_gemm.cu); arguments checked by render_rays_backward
size_t gemm_backward_workspace(const tsdfs_mlp* mlp, int64_t max_samples);
int64_t gemm_backward_chunk(const tsdfs_mlp* mlp, int64_t max_samples);
// kept: from the records and activations a gemm_train_forward call left in ws
int gemm_backward(const tsdfs_mlp* mlp, const float* ray_o, const float* ray_d, const float* t_n, const float* t_f,
                  const int32_t* offsets, const uint8_t* status, int64_t n_rays, int64_t max_samples,
                  const float* d_rgb, const float* d_depth, const float* d_eik, float* d_sdf_w, float* d_rgb_w,
                  void* ws, size_t ws_bytes, cudaStream_t st, bool kept);
// render_rays through the layer-major forward, keeping records and activations in ws
int gemm_train_forward(const tsdfs_mlp* mlp, const float* ray_o, const float* ray_d, const float* t_n,
                       const float* t_f, const int32_t* offsets, const uint8_t* status, int64_t n_rays,
                       int64_t max_samples, float* rgb, float* depth, float* wsum, float* normal, float* eik, void* ws,
                       size_t ws_bytes, cudaStream_t st);

}  // namespace tsdfs
