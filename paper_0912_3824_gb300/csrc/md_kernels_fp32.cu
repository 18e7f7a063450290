// Kernels of the FP32 precision mode (see md_kernels.cuh).
#include "md_kernels.cuh"

namespace mdk {

const KernelSet &kernels_fp32()
{
    static const KernelSet k = make_kernel_set<FP32>();
    return k;
}

}  // namespace mdk
