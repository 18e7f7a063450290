// Kernels of the FP64 precision mode (see md_kernels.cuh).
#include "md_kernels.cuh"

namespace mdk {

const KernelSet &kernels_fp64()
{
    static const KernelSet k = make_kernel_set<FP64>();
    return k;
}

}  // namespace mdk
