// inst_bf16.cu -- kernels and launchers for the StoreBF16 population format
#include "lbm_kernels.cuh"

namespace lbm {
const Dispatch& dispatch_bf16()
{
    static const Dispatch d = make_dispatch<StoreBF16>();
    return d;
}
}  // namespace lbm
