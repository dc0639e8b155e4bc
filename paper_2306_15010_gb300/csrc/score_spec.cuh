// Filter-bank descriptions passed to the score kernels by value (kernel parameters).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vqnnf {

constexpr int kMaxFilters = 32;
constexpr int kMaxRects = 192;
constexpr int kMaxRows = 2 * kMaxRects;

// One weighted half-open rectangle; ry0 / ry1 index the bank's distinct row offsets.
struct RectSpec {
    int x0, y0, x1, y1, weight;
    int ry0, ry1;
};

// Any bank: F filters, rectangles of filter f are rect[rect_begin[f] .. rect_begin[f+1]).
struct BankSpec {
    int F;
    int nrow;                     // distinct row offsets staged per window row
    int ncol;                     // staged columns per row (256 windows + template width)
    int roff[kMaxRows];           // the distinct row offsets, ascending
    int rect_begin[kMaxFilters + 1];
    RectSpec rect[kMaxRects];
    float coef[kMaxFilters];      // w_f / A_f
};

// Grid bank: the window cut by column boundaries bx[0..G] and row boundaries by[0..G]
// into G x G cells (slot r * G + c), optionally with the full window (slot G * G).  Every
// filter is one cell or the full window with weight 1.
struct GridSpec {
    int G;                        // 0 = not a grid bank
    int full;
    int F;
    int ncol;
    int bx[5];
    int by[5];
    int slot_filter[17];          // slot -> filter index
    int slot_area[17];            // pixels in the slot's rectangle
    float slot_coef[17];          // w_f / A_f of the slot's filter
    int filter_slot[kMaxFilters]; // filter index -> slot
    float coef[kMaxFilters];
};

// Weighted-grid bank: every filter is an integer weighting of the 3 x 3 cells of one of up to
// four grids (cells cut by column boundaries bx[g][0..3] and row boundaries by[g][0..3]; a
// boundary may repeat, giving empty cells), at most five filters per grid.  The coarse
// Gaussian / Haar filters of the paper at sub-scales have this form.
constexpr int kMaxWGrids = 4;
constexpr int kMaxWFilters = 5;
struct WGridSpec {
    int NG;                                   // 0 = not a weighted-grid bank
    int ncol;
    int nf[kMaxWGrids];
    int bx[kMaxWGrids][4];
    int by[kMaxWGrids][4];
    int w[kMaxWGrids][kMaxWFilters][9];       // cell weights, cell r * 3 + c
    int filt[kMaxWGrids][kMaxWFilters];       // bank index of the filter
    float coef[kMaxWGrids][kMaxWFilters];     // w_f / A_f
};

size_t score_smem_bytes_for(size_t elem, const BankSpec &bs, const GridSpec &gs, int k);
size_t score_wgrid_smem_bytes(size_t elem, const WGridSpec &ws, int k);
bool sat_is_u16(int th, int tw);
int sat_pitch(int W);
int sat_strips(int W);
int sat_bands(int H);
int score_ncol(int tw);
bool score_grid_fits(int ncol);   // the grid kernel stages at most TXW + 256 columns
size_t sat_slack_elems(int tw);
cudaError_t launch_sat(const uint8_t *lab, int H, int W, int k, bool u16, int *carry, int *bandsum,
                       void *S, cudaStream_t s);
cudaError_t launch_filter_responses(const uint8_t *lab, int h, int w, int k, const BankSpec &bs,
                                    int32_t *counts, cudaStream_t s);
cudaError_t launch_score(const void *S, bool u16, int W, int k, int HO, int WO, const BankSpec &bs,
                         const GridSpec &gs, const WGridSpec &ws, const int32_t *tc, float *heat,
                         unsigned long long *amax, int32_t *argmax_yx, cudaStream_t s);
cudaError_t read_and_clear_score_error(int *out);
// One-thread kernel whose mbarrier wait gives up after limit_cycles (self-test of the bounded
// waits; sets the error word that read_and_clear_score_error returns).
cudaError_t launch_wait_selftest(long long limit_cycles, cudaStream_t s);

}  // namespace vqnnf
