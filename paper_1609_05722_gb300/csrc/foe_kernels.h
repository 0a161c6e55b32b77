// Host-side launchers of the FoE kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include "foe_common.cuh"

namespace foe {

// Plain FP32 fused tile kernel (foe_f32.cu).
int f32_tile();
size_t f32_smem_bytes();
cudaError_t f32_setup();
cudaError_t f32_launch(const LaunchArgs &a, int mode, cudaStream_t s);

// Tensor-core (tcgen05, BF16) fused tile kernel (foe_tc.cu).
int tc_tile_h();
int tc_tile_w();
size_t tc_smem_bytes();
cudaError_t tc_setup();
cudaError_t tc_launch(const LaunchArgs &a, int mode, int *d_status, cudaStream_t s);

cudaError_t launch_init(const float *y, int H, int W, int yld, int ld, int model, float zero_c, float *d, float *uh,
                        float *ul, float *delta, cudaStream_t s);
cudaError_t launch_output(const float *uh, const float *ul, int H, int W, int ld, int xld, int model, float *x,
                          cudaStream_t s);
cudaError_t launch_anscombe(const float *y, float *v, long n, cudaStream_t s);
cudaError_t launch_inverse(const float *z, float *x, long n, cudaStream_t s);
cudaError_t launch_reduce(const double *p, int n, double *out, cudaStream_t s);

}  // namespace foe
