// sweep_f16.cu -- kernel instantiations for __half population storage.
#include "kernels.cuh"

namespace lbm {
LBM_INSTANTIATE(__half)
}  // namespace lbm
