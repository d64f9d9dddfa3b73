// Temporal blocking of the FP32/BF16 update (several steps per HBM pass).
#include "common.cuh"
#include "kernels.cuh"

namespace fdtd {

int blocked_max_depth() { return 1; }
int auto_depth(int, int) { return 1; }

}  // namespace fdtd
