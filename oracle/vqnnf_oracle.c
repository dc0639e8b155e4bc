/*
 * VQ-NNF oracle: a plain, slow, obviously correct CPU implementation of the
 * template-matching hot path of "Efficient High-Resolution Template Matching with
 * Vector Quantized Nearest Neighbour Fields" (Gupta & Sintorn).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU baseline
 * leg of the benchmark load this file.  It shares no code, header, table or helper with
 * the CUDA library; it is built by its own gcc command and reached through its own
 * ctypes wrapper (oracle/__init__.py).
 *
 * Arithmetic: FP64 for every floating-point step, int64 for every count.  No blocking,
 * no fusion, no summed-area tables: every quantity is computed from its definition.
 *
 * Readings of points the paper leaves open (each is listed in the design notes):
 *   - distance: squared L2, summed in dimension order (Sec. 4.2 "exact NN ... L2").
 *   - ties: the lowest centroid index wins; the heatmap maximum takes the lowest
 *     row-major (y, then x) window.
 *   - k-means: the paper only names a library (Sec. 4.2).  Here: k distinct initial
 *     pixel indices from a partial Fisher-Yates shuffle driven by SplitMix64, then
 *     exactly `iters` Lloyd steps; an empty cluster keeps its centroid; each mean is
 *     accumulated in FP64 in pixel order and rounded to FP32.
 *   - filters: a filter is a list of weighted half-open rectangles [x0,x1) x [y0,y1)
 *     relative to the window's top-left; its response for cluster j is the weighted
 *     count of pixels labelled j inside the rectangles (Eq. 1 without the 1/area
 *     factor, which the score applies as w_f / A_f).
 *   - score: Eq. 2 with |.| read as the L1 norm over the k clusters:
 *       H(y,x) = - sum_f (w_f / A_f) * sum_j | t_f[j] - q_f(y,x)[j] |
 *     over valid windows only ((H-th+1) x (W-tw+1)), indexed by the top-left corner.
 *
 * Parity pins: every function here is checked by tests/test_oracle_pins.py against
 * exact rational brute force on tiny inputs, closed forms and invariants.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number           */
/* generators", OOPSLA 2014): state advances by the golden gamma, output is the     */
/* state passed through the variant-13 64-bit finaliser.                           */
/* ------------------------------------------------------------------------------ */
uint64_t oracle_splitmix64_next(uint64_t *state)
{
    uint64_t z;
    *state += 0x9E3779B97F4A7C15ULL;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* k distinct indices in [0, l): the first k slots of a Fisher-Yates shuffle of
 * 0..l-1 in which slot i swaps with slot i + (r mod (l - i)), r = next output.
 * Returns 0, or -1 when k > l or on allocation failure. */
int oracle_kmeans_init(int64_t l, int k, uint64_t seed, int64_t *idx_out)
{
    int64_t *perm;
    uint64_t state = seed;
    int i;
    if (k < 1 || (int64_t)k > l)
        return -1;
    perm = (int64_t *)malloc((size_t)l * sizeof(int64_t));
    if (!perm)
        return -1;
    for (int64_t p = 0; p < l; ++p)
        perm[p] = p;
    for (i = 0; i < k; ++i) {
        uint64_t r = oracle_splitmix64_next(&state);
        int64_t j = (int64_t)i + (int64_t)(r % (uint64_t)(l - i));
        int64_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
        idx_out[i] = perm[i];
    }
    free(perm);
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* Nearest-neighbour field (Algorithm 1): for every pixel, the index of the nearest   */
/* codebook vector under the squared L2 distance.                                  */
/* ------------------------------------------------------------------------------ */
static double sqdist(const float *x, const float *c, int D)
{
    double s = 0.0;
    for (int i = 0; i < D; ++i) {
        double d = (double)x[i] - (double)c[i];
        s += d * d;
    }
    return s;
}

/* X: n x D (row-major), C: k x D.  Writes labels[n]; d1/d2 (may be NULL) get the
 * smallest and second-smallest distance (d2 == d1 when two centroids tie; d2 = +inf
 * when k == 1). */
void oracle_assign(const float *X, int64_t n, int D, const float *C, int k,
                   int32_t *labels, double *d1, double *d2)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; ++p) {
        const float *x = X + p * (int64_t)D;
        double best = INFINITY, second = INFINITY;
        int32_t arg = 0;
        for (int j = 0; j < k; ++j) {
            double d = sqdist(x, C + (int64_t)j * D, D);
            if (d < best) {
                second = best;
                best = d;
                arg = j;
            } else if (d < second) {
                second = d;
            }
        }
        labels[p] = arg;
        if (d1)
            d1[p] = best;
        if (d2)
            d2[p] = second;
    }
}

/* ------------------------------------------------------------------------------ */
/* k-means codebook (Sec. 3.1): seeded init, then `iters` Lloyd steps.              */
/* ------------------------------------------------------------------------------ */
/* T: l x D template features.  C_out: k x D.  Returns 0 or -1. */
int oracle_fit_codebook(const float *T, int64_t l, int D, int k, int iters, uint64_t seed,
                        float *C_out)
{
    int64_t *init = (int64_t *)malloc((size_t)k * sizeof(int64_t));
    int32_t *lab = (int32_t *)malloc((size_t)l * sizeof(int32_t));
    double *sum = (double *)malloc((size_t)k * (size_t)D * sizeof(double));
    int64_t *cnt = (int64_t *)malloc((size_t)k * sizeof(int64_t));
    int rc = -1;
    if (!init || !lab || !sum || !cnt)
        goto done;
    if (oracle_kmeans_init(l, k, seed, init) != 0)
        goto done;
    for (int j = 0; j < k; ++j)
        memcpy(C_out + (int64_t)j * D, T + init[j] * D, (size_t)D * sizeof(float));
    for (int it = 0; it < iters; ++it) {
        oracle_assign(T, l, D, C_out, k, lab, NULL, NULL);
        memset(sum, 0, (size_t)k * (size_t)D * sizeof(double));
        memset(cnt, 0, (size_t)k * sizeof(int64_t));
        for (int64_t p = 0; p < l; ++p) {          /* pixel order */
            double *s = sum + (int64_t)lab[p] * D;
            const float *x = T + p * D;
            for (int i = 0; i < D; ++i)
                s[i] += (double)x[i];
            cnt[lab[p]] += 1;
        }
        for (int j = 0; j < k; ++j) {
            if (cnt[j] == 0)
                continue;                           /* empty cluster keeps its centroid */
            for (int i = 0; i < D; ++i)
                C_out[(int64_t)j * D + i] = (float)(sum[(int64_t)j * D + i] / (double)cnt[j]);
        }
    }
    rc = 0;
done:
    free(init);
    free(lab);
    free(sum);
    free(cnt);
    return rc;
}

/* Sum over pixels of the squared distance to the assigned centroid (k-means objective). */
double oracle_kmeans_objective(const float *T, int64_t l, int D, const float *C, int k)
{
    int32_t *lab = (int32_t *)malloc((size_t)l * sizeof(int32_t));
    double *d1 = (double *)malloc((size_t)l * sizeof(double));
    double s = 0.0;
    if (!lab || !d1) {
        free(lab);
        free(d1);
        return NAN;
    }
    oracle_assign(T, l, D, C, k, lab, d1, NULL);
    for (int64_t p = 0; p < l; ++p)
        s += d1[p];
    free(lab);
    free(d1);
    return s;
}

/* ------------------------------------------------------------------------------ */
/* Filter responses by direct counting (no integral image).                        */
/* A filter bank is passed flat:                                                    */
/*   n_rects[F]        rectangles per filter                                        */
/*   rects[R * 5]      (x0, y0, x1, y1, weight) for all filters, filter by filter    */
/* ------------------------------------------------------------------------------ */
static void window_counts(const int32_t *labels, int W, int k, int wy, int wx,
                          int F, const int32_t *n_rects, const int32_t *rects,
                          int64_t *out /* F x k */)
{
    const int32_t *r = rects;
    memset(out, 0, (size_t)F * (size_t)k * sizeof(int64_t));
    for (int f = 0; f < F; ++f) {
        int64_t *o = out + (int64_t)f * k;
        for (int q = 0; q < n_rects[f]; ++q, r += 5) {
            int x0 = r[0], y0 = r[1], x1 = r[2], y1 = r[3], wgt = r[4];
            for (int y = wy + y0; y < wy + y1; ++y)
                for (int x = wx + x0; x < wx + x1; ++x)
                    o[labels[(int64_t)y * W + x]] += wgt;
        }
    }
}

/* Template representation vectors: the bank applied to the whole h x w template NNF. */
void oracle_filter_counts(const int32_t *labels, int h, int w, int k,
                          int F, const int32_t *n_rects, const int32_t *rects,
                          int64_t *counts /* F x k */)
{
    (void)h;
    window_counts(labels, w, k, 0, 0, F, n_rects, rects, counts);
}

/* Counts of one query window (for invariant checks). */
void oracle_window_counts(const int32_t *labels, int H, int W, int k, int wy, int wx,
                          int F, const int32_t *n_rects, const int32_t *rects,
                          int64_t *counts /* F x k */)
{
    (void)H;
    window_counts(labels, W, k, wy, wx, F, n_rects, rects, counts);
}

static double window_score(const int32_t *q_labels, int W, int k, int wy, int wx, int F,
                           const int32_t *n_rects, const int32_t *rects,
                           const double *w_f, const double *area,
                           const int64_t *t_counts, int64_t *scratch)
{
    double acc = 0.0;
    window_counts(q_labels, W, k, wy, wx, F, n_rects, rects, scratch);
    for (int f = 0; f < F; ++f) {
        int64_t l1 = 0;
        for (int j = 0; j < k; ++j) {
            int64_t d = t_counts[(int64_t)f * k + j] - scratch[(int64_t)f * k + j];
            l1 += d < 0 ? -d : d;
        }
        acc += (w_f[f] / area[f]) * (double)l1;
    }
    return -acc;
}

/* Eq. 2 heatmap over every valid window, plus its maximum (lowest row-major index on
 * ties).  heat: (H-th+1) x (W-tw+1).  argmax_yx may be NULL.  Returns 0 or -1. */
int oracle_score(const int32_t *q_labels, int H, int W, int k, int th, int tw,
                 int F, const int32_t *n_rects, const int32_t *rects,
                 const double *w_f, const double *area, const int64_t *t_counts,
                 double *heat, int32_t *argmax_yx)
{
    int HO = H - th + 1, WO = W - tw + 1;
    if (HO < 1 || WO < 1)
        return -1;
#pragma omp parallel
    {
        int64_t *scratch = (int64_t *)malloc((size_t)F * (size_t)k * sizeof(int64_t));
#pragma omp for schedule(dynamic, 1)
        for (int y = 0; y < HO; ++y)
            for (int x = 0; x < WO; ++x)
                heat[(int64_t)y * WO + x] = window_score(q_labels, W, k, y, x, F, n_rects,
                                                         rects, w_f, area, t_counts, scratch);
        free(scratch);
    }
    if (argmax_yx) {
        int64_t best = 0;
        for (int64_t i = 1; i < (int64_t)HO * WO; ++i)
            if (heat[i] > heat[best])
                best = i;
        argmax_yx[0] = (int32_t)(best / WO);
        argmax_yx[1] = (int32_t)(best % WO);
    }
    return 0;
}

/* Eq. 2 at a list of windows (top-left (y, x) pairs): for sampled checks at sizes where
 * the full heatmap is too slow. */
void oracle_score_at(const int32_t *q_labels, int H, int W, int k,
                     int F, const int32_t *n_rects, const int32_t *rects,
                     const double *w_f, const double *area, const int64_t *t_counts,
                     int64_t n_win, const int32_t *win_yx, double *out)
{
    (void)H;
#pragma omp parallel
    {
        int64_t *scratch = (int64_t *)malloc((size_t)F * (size_t)k * sizeof(int64_t));
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < n_win; ++i)
            out[i] = window_score(q_labels, W, k, win_yx[2 * i], win_yx[2 * i + 1], F, n_rects,
                                  rects, w_f, area, t_counts, scratch);
        free(scratch);
    }
}

/* ------------------------------------------------------------------------------ */
/* Algorithm 2: a coarse filter f_i of r_w x r_h bin weights (each weight repeated   */
/* over a d_x x d_y bin) becomes an (r_w+1) x (r_h+1) dilation filter f_d on the      */
/* integral image by adding f_i(i, j) * [[1, -1], [-1, 1]] onto f_d at (i..i+1,        */
/* j..j+1).  Arrays are indexed [i][j] with i along x (r_w) and j along y (r_h).      */
/* The 2x2 multiplier's sign pattern matches the exclusive-prefix box sum            */
/*   box = S(x1, y1) - S(x0, y1) - S(x1, y0) + S(x0, y0):                            */
/* f_d(i, j) += +f (top-left corner (x0, y0)), f_d(i+1, j) -= f, f_d(i, j+1) -= f,     */
/* f_d(i+1, j+1) += f.                                                               */
/* ------------------------------------------------------------------------------ */
void oracle_coarse_to_dilation(const double *f_i, int r_w, int r_h, double *f_d)
{
    memset(f_d, 0, (size_t)(r_w + 1) * (size_t)(r_h + 1) * sizeof(double));
    for (int i = 0; i < r_w; ++i) {
        for (int j = 0; j < r_h; ++j) {
            double a = f_i[(int64_t)i * r_h + j];
            f_d[(int64_t)i * (r_h + 1) + j] += a;
            f_d[(int64_t)(i + 1) * (r_h + 1) + j] -= a;
            f_d[(int64_t)i * (r_h + 1) + (j + 1)] -= a;
            f_d[(int64_t)(i + 1) * (r_h + 1) + (j + 1)] += a;
        }
    }
}

/* Direct weighted count of a coarse filter over one window of the label image:
 * sum over bins (i, j) of f_i(i, j) * #{pixels labelled `cls` in bin (i, j)}, bin (i, j)
 * covering x in [wx + i*d_x, wx + (i+1)*d_x), y in [wy + j*d_y, wy + (j+1)*d_y). */
double oracle_coarse_direct(const int32_t *labels, int W, int wy, int wx, int cls,
                            const double *f_i, int r_w, int r_h, int d_x, int d_y)
{
    double s = 0.0;
    for (int i = 0; i < r_w; ++i)
        for (int j = 0; j < r_h; ++j) {
            int64_t c = 0;
            for (int y = wy + j * d_y; y < wy + (j + 1) * d_y; ++y)
                for (int x = wx + i * d_x; x < wx + (i + 1) * d_x; ++x)
                    c += labels[(int64_t)y * W + x] == cls;
            s += f_i[(int64_t)i * r_h + j] * (double)c;
        }
    return s;
}

/* Threads of the parallel loops above, for timing only: every loop computes independent
 * elements, so the results do not depend on it.  n >= 1 sets the count; returns the count in
 * effect before the call. */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    const int prev = omp_get_max_threads();
    if (n >= 1) omp_set_num_threads(n);
    return prev;
#else
    (void)n;
    return 1;
#endif
}
