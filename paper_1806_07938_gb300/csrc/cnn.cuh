// Internal interface of the warm-start network kernels (cnn.cu).
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace tomo {

// valid slopes [B][NP][n_vs] <-> grids [B][NP][n][n] (scaled; zero off the valid set)
// (the grid has ctot >= NP channels; all are cleared, the first NP receive s)
cudaError_t cnn_scatter(const Launch& L, int B, int NP, int n, int n_vs, const int* rowcol, const float* s,
                        float scale, float* grid, int ctot);
cudaError_t cnn_scatter_planes(const Launch& L, int B, int c0, int ctot, int np, int n, int n_vs, const int* rowcol,
                               const float* s, float scale, float* grid);
cudaError_t axpy_f32(const Launch& L, size_t total, float a, const float* x, float* y);
cudaError_t cnn_gather(const Launch& L, int B, int NP, int n, int n_vs, const int* rowcol, const float* grid,
                       float scale, float* out);
// y = relu?(conv3x3(x, W) + b) with Wt = W as [Cin][9][Cout]; x [B][Cin][n][n], y [B][Cout][n][n]
cudaError_t conv_fwd(const Launch& L, int B, int Cin, int Cout, int n, const float* x, const float* Wt,
                     const float* bias, float* y, bool relu);
// W [Cout][Cin][3][3] -> Wt [Cin][9][Cout] and (if Wb) Wb [Cout][9][Cin] flipped: dX = conv(dY, Wb)
cudaError_t weight_layouts(const Launch& L, int Cin, int Cout, const float* W, float* Wt, float* Wb);
cudaError_t relu_bwd(const Launch& L, size_t total, const float* yact, float* dy);
// dW [Cout][Cin][3][3] followed by db [Cout], through per-block partials (part: conv_wgrad_parts floats)
size_t conv_wgrad_parts(int B, int Cin, int Cout, int n);
cudaError_t conv_wgrad(const Launch& L, int B, int Cin, int Cout, int n, const float* x, const float* dy,
                       float* part, float* dW_db);
// loss = |z - t|^2 / |t|^2 over `total` entries; g = dloss/dz; sums: 512 doubles of scratch
cudaError_t loss_grad(const Launch& L, size_t total, const float* z, const float* t, double* sums, float* g,
                      double* loss);
cudaError_t adam(const Launch& L, int np, float* w, const float* g, float* m, float* v, float lr, int step);

}  // namespace tomo
