// inst_f64.cu -- kernels and launchers for the StoreF64 population format
#include "lbm_kernels.cuh"

namespace lbm {
const Dispatch& dispatch_f64()
{
    static const Dispatch d = make_dispatch<StoreF64>();
    return d;
}
}  // namespace lbm
