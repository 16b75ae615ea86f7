// sweep_f32.cu -- kernel instantiations for float population storage.
#include "kernels.cuh"

namespace lbm {
LBM_INSTANTIATE(float)
}  // namespace lbm
