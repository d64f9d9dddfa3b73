// Sums and renormalisation of a z-slab of an FP32 lattice (Sec. V: each
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

constexpr int kSlabThreads = 256;

// S0 = sum psi^2, SH = sum psi (-Lap psi / (2 m a^2) + V psi), Sr = sum r^2
// psi^2, SV = sum V psi^2 (Eq. energysum, sign of Sec. II's H) over the own
// planes; block b takes rows b, b + nb, ... of the own planes in order,
// FP64 accumulation, fixed-order block reduction.
__global__ void __launch_bounds__(kSlabThreads) k_slab_sums(const float* __restrict__ psi, const float* __restrict__ v,
                                                            int n, int nzo, int zbase, int z_first, double a,
                                                            double kfac, double* __restrict__ partials) {
  __shared__ double red[4][kSlabThreads];
  double acc[4] = {0, 0, 0, 0};
  const size_t nn = (size_t)n * n;
  const double half = 0.5 * (double)(n - 1);
  for (int r = blockIdx.x; r < n * nzo; r += gridDim.x) {
    const int y = r % n, zl = zbase + r / n;
    const double py = ((double)y - half) * a, pz = ((double)(z_first + r / n) - half) * a;
    for (int x = threadIdx.x; x < n; x += kSlabThreads) {
      const size_t i = ((size_t)zl * n + y) * n + x;
      const double c = psi[i];
      const double xm = x > 0 ? psi[i - 1] : 0.0, xp = x < n - 1 ? psi[i + 1] : 0.0;
      const double ym = y > 0 ? psi[i - n] : 0.0, yp = y < n - 1 ? psi[i + n] : 0.0;
      const double zm = psi[i - nn], zp = psi[i + nn];  // own or halo planes
      const double lap = (((xm + xp) + (ym + yp)) + (zm + zp)) - 6.0 * c;
      const double vv = v[i];
      const double px = ((double)x - half) * a;
      acc[0] += c * c;
      acc[1] += c * (-kfac * lap + vv * c);
      acc[2] += (px * px + py * py + pz * pz) * c * c;
      acc[3] += vv * c * c;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = kSlabThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) partials[(size_t)blockIdx.x * 4 + threadIdx.x] = red[threadIdx.x][0];
}

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

int slab_sums_blocks(int n, int nzo) { return (int)std::min<long long>((long long)n * nzo, 152 * 8); }

int launch_slab_sums(const float* psi, const float* v, const Params& p, int nzo, int zbase, int z_first,
                     double* partials, cudaStream_t st) {
  const int nb = slab_sums_blocks(p.n, nzo);
  k_slab_sums<<<nb, kSlabThreads, 0, st>>>(psi, v, p.n, nzo, zbase, z_first, p.a, 1.0 / (2.0 * p.mass * p.a * p.a),
                                           partials);
  return nb;
}

void launch_slab_reduce(const double* partials, int nparts, double* out4, cudaStream_t st) {
  k_slab_reduce<<<1, 1, 0, st>>>(partials, nparts, out4);
}

void launch_slab_scale(const float* in, float* out, int n, int nzo, int zbase, int mask_xy, double factor,
                       cudaStream_t st) {
  dim3 grid((n + 31) / 32, (n + 7) / 8, nzo);
  k_slab_scale<<<grid, dim3(32, 8), 0, st>>>(in, out, n, nzo, zbase, mask_xy, (float)factor);
}

}  // namespace fdtd
