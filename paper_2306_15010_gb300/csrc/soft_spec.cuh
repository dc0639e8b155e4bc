// Soft-VQ heatmap: the cell grid, workspace layout and entry points (soft.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace vqnnf {

constexpr int kSoftMaxK = 128;     // centroids
constexpr int kSoftMaxG = 4;       // grid side (F = G * G filters)
constexpr int kSoftSlices = 256;   // pixel slices of the centroid-gradient reduction

// A cell [y0, y1) x [x0, x1) of the template window; s = its size class (index into the
// at most four (height, width) pairs of the grid).
struct SoftCell {
    int y0, y1, x0, x1, s;
};

struct SoftGrid {
    int G, F;
    int nw, nh, ns;                 // distinct cell widths, heights, (height, width) pairs
    int wid[2], hgt[2];
    int size_w[4], size_h[4];       // size class -> width index, height index
    SoftCell cell[kSoftMaxG * kSoftMaxG];
};

struct SoftWs {
    float *P;      // B x k x H x W     query soft assignment (planar), kept for the backward
    float *RW;     // nw x B x k x H x W row sums of each cell width
    float *BX;     // B x ns x k x H x W box sums of each cell size (the query soft counts)
    float *Pt;     // k x th x tw       template soft assignment, kept for the backward
    float *T;      // F x k             template soft counts
    float *L1;     // B x F x HO x WO   per-filter L1 distances
    float *R2;     // ns x B x k x H x W gradient gather + adjoint row pass of each cell size
    float *G;      // B x k x H x W     dL/dp of the query pixels (planar)
    float *A;      // B x H x W x k     dL/dd of the query pixels (pixel-major)
    float *At;     // th x tw x k       dL/dd of the template pixels
    float *dT;     // F x k             dL/dT
    float *part;   // 2 kSoftSlices x (k D + k) partial centroid gradients (query, template)
    uint8_t *ct;   // C^T hi/lo image of the tensor-core gradient kernel (soft_tc.cu)
};

bool soft_grid(int th, int tw, int G, SoftGrid &sg);

// Tensor-core gradient contractions (soft_tc.cu): dX = 2 (sum_j a_j) x - 2 A C and the per-CTA
// partials Y_j = sum_u a_j(u) x_u, S_j = sum_u a_j(u) in part[slice][j D + d], part[slice][k D + j]
// (slices = CTAs launched, written to *slices).  Supported when k <= 64 and the operands fit in
// shared memory (soft_tc_supported); dX may be null.
bool soft_tc_supported(int D, int k);
size_t soft_ct_image_bytes(int D);
cudaError_t launch_soft_ct_image(const float *C, int k, int D, uint8_t *img, cudaStream_t s);
cudaError_t launch_soft_grad_tc(const float *X, long long n, long long npi, int D, int k, float tau,
                                const float *P, const float *G, const uint8_t *ct_img, float *dX, float *part,
                                int max_slices, int *slices, cudaStream_t s);
cudaError_t read_and_clear_soft_error(int *out);
size_t soft_workspace_bytes(int B, int H, int W, int D, int k, int th, int tw, const SoftGrid &sg);
SoftWs carve_soft(WsCursor &c, int B, int H, int W, int D, int k, int th, int tw, const SoftGrid &sg);
cudaError_t soft_forward(const float *Qf, int B, int H, int W, const float *Tf, int th, int tw, int D,
                         const float *C, int k, float tau, const SoftGrid &sg, const float *wf, float *heat,
                         SoftWs &w, cudaStream_t s);
cudaError_t soft_backward(const float *Qf, int B, int H, int W, const float *Tf, int th, int tw, int D,
                          const float *C, int k, float tau, const SoftGrid &sg, const float *wf,
                          const float *dheat, float *dQf, float *dC, float *dwf, SoftWs &w, cudaStream_t s);

}  // namespace vqnnf
