// Tensor-core (tcgen05) BF16 distance contraction -- placeholder until the kernel lands.
#include "common.cuh"

namespace vqnnf {

namespace {
__device__ int g_tc_error = 0;
}

cudaError_t launch_assign_bf16(const float *, long long, int, int, const CodebookPrep &,
                               uint8_t *, FlagList, cudaStream_t)
{
    return cudaErrorNotSupported;
}

cudaError_t read_and_clear_tc_error(int *out)
{
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(out, g_tc_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int));
    return e;
}

}  // namespace vqnnf
