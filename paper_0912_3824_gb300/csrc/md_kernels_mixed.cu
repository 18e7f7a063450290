// Kernels of the MIXED precision mode (see md_kernels.cuh).
#include "md_kernels.cuh"

namespace mdk {

const KernelSet &kernels_mixed()
{
    static const KernelSet k = make_kernel_set<MIXED>();
    return k;
}

}  // namespace mdk
