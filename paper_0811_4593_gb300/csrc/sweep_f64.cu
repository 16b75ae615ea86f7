// sweep_f64.cu -- kernel instantiations for double population storage.
#include "kernels.cuh"

namespace lbm {
LBM_INSTANTIATE(double)
}  // namespace lbm
