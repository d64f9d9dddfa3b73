// Batched persistent driver: many lattices advance in one launch.
#include "common.cuh"
#include "kernels.cuh"

namespace fdtd {

size_t batched_workspace_bytes(const fdtd_lattice_desc*, int) { return 0; }

}  // namespace fdtd
