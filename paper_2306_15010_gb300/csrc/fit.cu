// k-means codebook of the template (Sec. 3.1): seeded initial centroids, then Lloyd
// steps whose assignment is the exact nearest-neighbour field of assign_fp32.cu /
// assign_tc.cu and whose update sums every cluster's members in FP64 in pixel order.
//
// Determinism: the members of each cluster are listed in pixel order by a stable counting
// sort, and thread (j, i) adds member features one after another in that order, so every
// FP64 sum is the same sequence of additions as a plain loop over pixels -- the centroids
// do not depend on scheduling.
#include "common.cuh"

namespace vqnnf {

namespace {

__global__ void gather_init_kernel(const float *__restrict__ T, int D, int k, InitIdx ii,
                                   float *__restrict__ C)
{
    const int j = blockIdx.x;
    const float *src = T + (size_t)ii.idx[j] * D;
    for (int i = threadIdx.x; i < D; i += blockDim.x) C[(size_t)j * D + i] = src[i];
}

// Stable counting sort of the labels by cluster (one block of 1024 threads).
//   cnt[k], off[k+1], members[l] (pixel indices in increasing order within a cluster)
__global__ void __launch_bounds__(1024) stable_sort_kernel(const uint8_t *__restrict__ lab,
                                                           int l, int k, int *cnt, int *off,
                                                           int *members)
{
    __shared__ int hist[kMaxK];
    __shared__ int base[kMaxK];
    __shared__ int wc[32][kMaxK];   // per-warp counts of the current chunk
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (int j = t; j < k; j += blockDim.x) hist[j] = 0;
    __syncthreads();
    for (int p = t; p < l; p += blockDim.x) atomicAdd(&hist[lab[p]], 1);
    __syncthreads();
    if (t == 0) {
        int s = 0;
        for (int j = 0; j < k; ++j) {
            base[j] = s;
            off[j] = s;
            cnt[j] = hist[j];
            s += hist[j];
        }
        off[k] = s;
    }
    __syncthreads();
    for (int c0 = 0; c0 < l; c0 += blockDim.x) {
        for (int q = t; q < 32 * kMaxK; q += blockDim.x)
            if ((q & (kMaxK - 1)) < k) (&wc[0][0])[q] = 0;
        __syncthreads();
        const int p = c0 + t;
        const bool ok = p < l;
        const int l0 = (int)lab[ok ? p : l - 1];          // clamped address
        const int lb = ok ? l0 : -1 - lane;               // unique dummies never match
        const unsigned same = __match_any_sync(0xffffffffu, lb);
        const int rank = __popc(same & ((1u << lane) - 1u));
        if (ok && rank == 0) wc[w][lb] = __popc(same);
        __syncthreads();
        // exclusive prefix over warps for every cluster; base advances by the chunk total
        for (int j = t; j < k; j += blockDim.x) {
            int s = base[j];
            for (int q = 0; q < 32; ++q) {
                const int c = wc[q][j];
                wc[q][j] = s;
                s += c;
            }
            base[j] = s;
        }
        __syncthreads();
        if (ok) members[wc[w][lb] + rank] = p;
        __syncthreads();
    }
}

// c_j[i] = fl32( (sum over members, pixel order, FP64) / count ); empty clusters keep c_j.
// One warp per (cluster, 32 dimensions).  Each lane streams its own column of the member
// rows through a shared-memory ring (cp.async, UR rows ahead), so the in-order FP64
// additions are not serialised behind scattered-row load latency.
constexpr int UR = 64;       // ring depth (member rows in flight per lane)
constexpr int UIDX = 1024;   // member indices staged per block

__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__global__ void __launch_bounds__(32) update_kernel(const float *__restrict__ T, int D, int k,
                                                    const int *__restrict__ cnt, const int *__restrict__ off,
                                                    const int *__restrict__ members, float *__restrict__ C)
{
    __shared__ float ring[UR][32];
    __shared__ int idx[UIDX];
    const int j = blockIdx.y;
    const int lane = threadIdx.x;
    const int i = blockIdx.x * 32 + lane;
    const int c = cnt[j];
    if (c == 0) return;
    const int *m = members + off[j];
    const int ic = i < D ? i : D - 1;           // clamped column (every address in bounds)
    double s = 0.0;
    for (int q0 = 0; q0 < c; q0 += UIDX) {
        const int nq = min(UIDX, c - q0);
        __syncwarp();
        for (int t = lane; t < nq; t += 32) idx[t] = m[q0 + t];
        __syncwarp();
        int qi = 0;                              // next row to issue
        for (; qi < nq && qi < UR; ++qi) {
            cp_async4(&ring[qi % UR][lane], T + (size_t)idx[qi] * D + ic);
            cp_commit();
        }
        for (int q = 0; q < nq; ++q) {
            if (qi - q == UR) cp_wait<UR - 1>();
            else cp_wait<0>();
            s += (double)ring[q % UR][lane];     // strictly in member (pixel) order
            if (qi < nq) {
                cp_async4(&ring[qi % UR][lane], T + (size_t)idx[qi] * D + ic);
                cp_commit();
                ++qi;
            }
        }
    }
    if (i < D) C[(size_t)j * D + i] = (float)(s / (double)c);
}

}  // namespace

cudaError_t launch_gather_init(const float *T, int D, int k, const InitIdx &ii, float *C,
                               cudaStream_t s)
{
    gather_init_kernel<<<k, 128, 0, s>>>(T, D, k, ii, C);
    return cudaGetLastError();
}

cudaError_t launch_lloyd_update(const float *T, int l, int D, int k, const uint8_t *lab, int *cnt,
                                int *off, int *members, float *C, cudaStream_t s)
{
    stable_sort_kernel<<<1, 1024, 0, s>>>(lab, l, k, cnt, off, members);
    // one warp per (32 dimensions, cluster): a large cluster's in-order FP64 chains spread
    // over many SMs (FP64 throughput per SM is small)
    dim3 g((D + 31) / 32, k);
    update_kernel<<<g, 32, 0, s>>>(T, D, k, cnt, off, members, C);
    return cudaGetLastError();
}

}  // namespace vqnnf
