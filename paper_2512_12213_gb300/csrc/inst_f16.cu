// inst_f16.cu -- kernels and launchers for the StoreF16 population format
#include "lbm_kernels.cuh"

namespace lbm {
const Dispatch& dispatch_f16()
{
    static const Dispatch d = make_dispatch<StoreF16>();
    return d;
}
}  // namespace lbm
