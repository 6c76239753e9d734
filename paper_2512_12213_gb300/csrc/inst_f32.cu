// inst_f32.cu -- kernels and launchers for the StoreF32 population format
#include "lbm_kernels.cuh"

namespace lbm {
const Dispatch& dispatch_f32()
{
    static const Dispatch d = make_dispatch<StoreF32>();
    return d;
}
}  // namespace lbm
