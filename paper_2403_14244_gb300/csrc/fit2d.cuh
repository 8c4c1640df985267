// Launchers of the 2D image-fitting path (fit2d.cu). Internal to libigs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>

namespace igs {

struct Fit2dAdam {
    float lr[8];  // per particle slot
    float b1, b2, omb1, omb2, eps;
    double b1d, b2d;
};

cudaError_t launch_fit2d_render(const float* particles, int k, float D, int width, int height, float* img,
                                cudaStream_t s);
cudaError_t launch_fit2d_backward(const float* particles, int k, float D, int width, int height, const float* dL,
                                  float* d_particles, cudaStream_t s);
cudaError_t launch_fit2d_adam(float* particles, const float* d_particles, float* m, float* v, int k,
                              const Fit2dAdam& a, int32_t* state, cudaStream_t s);
// Densify / prune: the accumulated position-gradient norm, and one pass that
// deletes, divides and keeps particles into new buffers (count to *count).
cudaError_t launch_fit2d_grad_accum(const float* d_particles, int k, float* accum, cudaStream_t s);
cudaError_t launch_fit2d_densify(const float* particles, const float* m, const float* v, const float* accum, int k,
                                 float thr, float tau_a, float log_sigma_min, int capacity, float* out, float* out_m,
                                 float* out_v, int32_t* count, cudaStream_t s);
// QuadTree initialisation: scratch size and the chain of launches.
size_t quadtree_work_bytes(int side, int min_cell);
cudaError_t launch_quadtree_init(const float* img, int side, int k_max, int min_cell, float* particles,
                                 int32_t* count, void* work, cudaStream_t s);

}  // namespace igs
