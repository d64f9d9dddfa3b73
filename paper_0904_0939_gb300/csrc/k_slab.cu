// Reduction of a z-slab's partial sums and its renormalisation (Sec. V: each
// process sums over its own planes; the partial sums are then reduced over
// the processes, and the common factor 1/sqrt(S0 a^3) is applied by every
// process to its own planes).  The slab field has n x n x nzbuf sites, own
// planes [zbase, zbase + nzo), and halo planes around them that hold the
// neighbouring slabs' planes (zero beyond the lattice's faces).
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace fdtd {

namespace {

// out4 = the partials summed in block order (one thread: fixed order)
__global__ void k_slab_reduce(const double* __restrict__ partials, int np, double* __restrict__ out4) {
  double acc[4] = {0, 0, 0, 0};
  for (int i = 0; i < np; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += partials[(size_t)i * 4 + q];
#pragma unroll
  for (int q = 0; q < 4; ++q) out4[q] = acc[q];
}

// out = factor * P(in) on the own planes; P the x and y symmetry operators
// of Sec. IV (mask bits 0-3), with the FP32 rounding of the one-lattice
// renormalisation (the factor rounded to FP32, one product per site).
__global__ void __launch_bounds__(256) k_slab_scale(const float* __restrict__ in, float* __restrict__ out, int n,
                                                    int nzo, int zbase, int mask, float factor) {
  const int x0 = blockIdx.x * 32 + threadIdx.x, y0 = blockIdx.y * 8 + threadIdx.y, zl = zbase + blockIdx.z;
  if (x0 >= n || y0 >= n) return;
  int c[2] = {x0, y0};
  bool neg = false, zero = false;
  for (int ax = 0; ax < 2; ++ax) {
    const int mode = (mask >> (2 * ax)) & 3;
    if (mode == 0) continue;
    const int mm = n - 1 - c[ax];
    if (c[ax] > mm) {
      c[ax] = mm;
      neg ^= (mode == 2);
    } else if (c[ax] == mm && mode == 2) {
      zero = true;
    }
  }
  const float v = in[((size_t)zl * n + c[1]) * n + c[0]];
  out[((size_t)zl * n + y0) * n + x0] = scale_site(v, factor, neg, zero);
}

}  // namespace

void launch_slab_reduce(const double* partials, int nparts, double* out4, cudaStream_t st) {
  k_slab_reduce<<<1, 1, 0, st>>>(partials, nparts, out4);
}

void launch_slab_scale(const float* in, float* out, int n, int nzo, int zbase, int mask_xy, double factor,
                       cudaStream_t st) {
  dim3 grid((n + 31) / 32, (n + 7) / 8, nzo);
  k_slab_scale<<<grid, dim3(32, 8), 0, st>>>(in, out, n, nzo, zbase, mask_xy, (float)factor);
}

}  // namespace fdtd
