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
    float *R2;     // B x k x H x W     gradient gather + adjoint row pass of one cell size
    float *G;      // B x k x H x W     dL/dp of the query pixels (planar)
    float *A;      // B x H x W x k     dL/dd of the query pixels (pixel-major)
    float *At;     // th x tw x k       dL/dd of the template pixels
    float *dT;     // F x k             dL/dT
    float *part;   // 2 kSoftSlices x (k D + k) partial centroid gradients (query, template)
};

bool soft_grid(int th, int tw, int G, SoftGrid &sg);
size_t soft_workspace_bytes(int B, int H, int W, int D, int k, int th, int tw, const SoftGrid &sg);
SoftWs carve_soft(WsCursor &c, int B, int H, int W, int D, int k, int th, int tw, const SoftGrid &sg);
cudaError_t soft_forward(const float *Qf, int B, int H, int W, const float *Tf, int th, int tw, int D,
                         const float *C, int k, float tau, const SoftGrid &sg, const float *wf, float *heat,
                         SoftWs &w, cudaStream_t s);
cudaError_t soft_backward(const float *Qf, int B, int H, int W, const float *Tf, int th, int tw, int D,
                          const float *C, int k, float tau, const SoftGrid &sg, const float *wf,
                          const float *dheat, float *dQf, float *dC, float *dwf, SoftWs &w, cudaStream_t s);

}  // namespace vqnnf
