// Adjoint kernels for gradients with respect to the potential V through the
// unrolled update of Eq. updateeq.
//
// The step is linear in psi, psi' = M psi with
//   M = diag(A) + c diag(B) Adj - 6c diag(B),   Adj = sum of the 6 neighbours,
// and Adj is symmetric under the zero boundary, so
//   M^T lam = A lam + c [ Adj(B lam) - 6 B lam ].
// Differentiating (1 + h) psi' = (1 - h) psi + c (Adj - 6) psi, h = dtau V/2,
// at one site gives  d psi'(s)/d V(s) = -(dtau/2) B(s) (psi'(s) + psi(s)),
// with psi' the step's raw output (before any check).
//
// An FP64 adjoint step is split in two passes: a pointwise pass (u = B lam
// and the g_V accumulation, one thread per site) and a z-marching stencil
// pass over u (launch_adjoint_stencil in k_core.cu); an FP32 step is one
// fused z-marching pass (launch_adjoint_step_f32 in k_core.cu).  The seed and
// the transpose of the checks are one thread per site.
#include "common.cuh"
#include "kernels.cuh"

namespace fdtd {

static int grid_1d(size_t total) {
  size_t b = (total + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

// neighbour value: zero beyond the lattice, or wrapped with periodic boundaries
template <typename T>
__device__ __forceinline__ double ldz(const T* p, int x, int y, int z, int n, int periodic) {
  if (periodic) {
    x = x < 0 ? x + n : (x >= n ? x - n : x);
    y = y < 0 ? y + n : (y >= n ? y - n : y);
    z = z < 0 ? z + n : (z >= n ? z - n : z);
  }
  if ((unsigned)x < (unsigned)n && (unsigned)y < (unsigned)n && (unsigned)z < (unsigned)n)
    return (double)Store<T>::to(p[site_index(x, y, z, n)]);
  return 0.0;
}

// B at a site: FP64 lattices from the stored c B, FP32 from V as the forward does.
template <typename T>
__device__ __forceinline__ double b_at(const void* v, const double* coefCB, size_t i, const Params& p) {
  if constexpr (sizeof(T) == 8) {
    return coefCB[i] / p.c;
  } else {
    return (double)coef_f32(((const float*)v)[i], p.half_dtau_f, p.one_m6c_f).b;
  }
}

// Pointwise half of the adjoint step from psi_prev to psi_next (the raw
// output of that step):  u = B lam  and
//   g_V += lam * d psi_next / dV = lam * (-(dtau/2) B (psi_next + psi_prev)),
// which is the derivative of (1 + h) psi' = (1 - h) psi + c Lap psi at one site.
template <typename T>
__global__ void k_adjoint_pointwise(const T* __restrict__ lam, const T* __restrict__ psi_prev,
                                    const T* __restrict__ psi_next, const void* __restrict__ v,
                                    const double* __restrict__ coefCB, T* __restrict__ u, double* __restrict__ gv,
                                    Params p) {
  const size_t total = (size_t)p.n * p.n * p.n;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const double b = b_at<T>(v, coefCB, i, p);
    const double l = (double)Store<T>::to(lam[i]);
    const double sum = (double)Store<T>::to(psi_next[i]) + (double)Store<T>::to(psi_prev[i]);
    gv[i] += l * (-0.5 * p.dtau * b * sum);
    if constexpr (sizeof(T) == 8)
      u[i] = b * l;
    else
      u[i] = Store<T>::from((float)(b * l));
  }
}
template <typename T>
void launch_adjoint_pointwise(const T* lam, const T* psi_prev, const T* psi_next, const void* v, const double* coefCB,
                              T* u, double* gv, const Params& p, cudaStream_t st) {
  size_t total = (size_t)p.n * p.n * p.n;
  k_adjoint_pointwise<T><<<grid_1d(total), 256, 0, st>>>(lam, psi_prev, psi_next, v, coefCB, u, gv, p);
}
template void launch_adjoint_pointwise<double>(const double*, const double*, const double*, const void*, const double*,
                                               double*, double*, const Params&, cudaStream_t);
template void launch_adjoint_pointwise<float>(const float*, const float*, const float*, const void*, const double*,
                                              float*, double*, const Params&, cudaStream_t);

// Seed at T:  lam = w_e 2 (H psi - E psi) / S0 + w_r 2 (r^2 - <r^2>) psi / S0,
// and the direct term gv = w_e psi^2 / S0 (E depends on V explicitly).
template <typename T>
__global__ void k_adjoint_seed(const T* __restrict__ psi, const void* __restrict__ v, const LatState* __restrict__ s,
                               double w_e, double w_r, T* __restrict__ lam, double* __restrict__ gv, Params p) {
  const int n = p.n;
  const size_t total = (size_t)n * n * n;
  const double s0 = s->s0, e = s->energy, r2m = s->r2;
  const double kfac = 1.0 / (2.0 * p.mass * p.a * p.a);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((size_t)n * n));
    double c = (double)Store<T>::to(psi[i]);
    const int pr = p.periodic;
    double nb = ldz(psi, x - 1, y, z, n, pr) + ldz(psi, x + 1, y, z, n, pr) + ldz(psi, x, y - 1, z, n, pr) +
                ldz(psi, x, y + 1, z, n, pr) + ldz(psi, x, y, z - 1, n, pr) + ldz(psi, x, y, z + 1, n, pr);
    double vv = (sizeof(T) == 8) ? ((const double*)v)[i] : (double)((const float*)v)[i];
    double hpsi = -kfac * (nb - 6.0 * c) + vv * c;
    double px = coord_f64(x, n, p.a), py = coord_f64(y, n, p.a), pz = coord_f64(z, n, p.a);
    double r2 = px * px + py * py + pz * pz;
    double l = w_e * 2.0 * (hpsi - e * c) / s0 + w_r * 2.0 * (r2 - r2m) * c / s0;
    gv[i] = w_e * c * c / s0;
    if constexpr (sizeof(T) == 8)
      lam[i] = l;
    else
      lam[i] = Store<T>::from((float)l);
  }
}
template <typename T>
void launch_adjoint_seed(const T* psi, const void* v, const LatState* s, double w_e, double w_r, T* lam, double* gv,
                         const Params& p, cudaStream_t st) {
  size_t total = (size_t)p.n * p.n * p.n;
  k_adjoint_seed<T><<<grid_1d(total), 256, 0, st>>>(psi, v, s, w_e, w_r, lam, gv, p);
}
template void launch_adjoint_seed<double>(const double*, const void*, const LatState*, double, double, double*,
                                          double*, const Params&, cudaStream_t);
template void launch_adjoint_seed<float>(const float*, const void*, const LatState*, double, double, float*,
                                         double*, const Params&, cudaStream_t);

// Transpose of the check  psi <- P(s psi):  lam <- s P^T lam.
// P sends the value at a source site q (lower half along every masked axis,
// or the central plane of an S_i axis) to q and to each of its mirror images
// o with sign sg(o); P^T gathers sum_o sg(o) lam(o) back onto q and leaves 0
// on every non-source site.  In place: every site is read only by the
// thread of its own source.
template <typename T>
__global__ void k_parity_adjoint_scale(T* __restrict__ lam, int n, int mask, const double* __restrict__ scale) {
  const double s = scale ? *scale : 1.0;
  const size_t total = (size_t)n * n * n;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    int c[3] = {(int)(i % n), (int)((i / n) % n), (int)(i / ((size_t)n * n))};
    bool source = true;
    int img_axes = 0;  // axes along which q has a distinct mirror image
    double sgn_ax[3] = {1.0, 1.0, 1.0};
    for (int ax = 0; ax < 3; ++ax) {
      int mode = (mask >> (2 * ax)) & 3;
      if (mode == 0) continue;
      int mm = n - 1 - c[ax];
      if (c[ax] > mm || (c[ax] == mm && mode == 2)) source = false;
      if (c[ax] < mm) img_axes |= 1 << ax;
      sgn_ax[ax] = (mode == 2) ? -1.0 : 1.0;
    }
    if (!source) continue;  // zeroed below by its own source thread
    double acc = 0.0;
    for (int sub = 0; sub < 8; ++sub) {
      if (sub & ~img_axes) continue;
      int o[3] = {c[0], c[1], c[2]};
      double sg = 1.0;
      for (int ax = 0; ax < 3; ++ax)
        if (sub & (1 << ax)) {
          o[ax] = n - 1 - c[ax];
          sg *= sgn_ax[ax];
        }
      size_t j = site_index(o[0], o[1], o[2], n);
      acc += sg * (double)Store<T>::to(lam[j]);
      if (sub) lam[j] = Store<T>::from(0.0f);
    }
    // non-source sites that are not a mirror image of any source (central
    // planes of A_i axes) are zeroed here as well
    double val = s * acc;
    if constexpr (sizeof(T) == 8)
      lam[i] = val;
    else
      lam[i] = Store<T>::from((float)val);
  }
}

template <typename T>
__global__ void k_zero_central_planes(T* __restrict__ lam, int n, int mask) {
  const size_t total = (size_t)n * n * n;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    int c[3] = {(int)(i % n), (int)((i / n) % n), (int)(i / ((size_t)n * n))};
    for (int ax = 0; ax < 3; ++ax) {
      int mode = (mask >> (2 * ax)) & 3;
      if (mode == 2 && c[ax] == n - 1 - c[ax]) lam[i] = Store<T>::from(0.0f);
    }
  }
}

template <typename T>
void launch_parity_adjoint_scale(T* lam, int n, int mask, const double* scale, cudaStream_t st) {
  size_t total = (size_t)n * n * n;
  if (mask && (n & 1)) k_zero_central_planes<T><<<grid_1d(total), 256, 0, st>>>(lam, n, mask);
  k_parity_adjoint_scale<T><<<grid_1d(total), 256, 0, st>>>(lam, n, mask, scale);
}
template void launch_parity_adjoint_scale<double>(double*, int, int, const double*, cudaStream_t);
template void launch_parity_adjoint_scale<float>(float*, int, int, const double*, cudaStream_t);

__global__ void k_store_scale(const LatState* s, double* dst) { *dst = s->scale; }
void launch_store_scale(const LatState* s, double* dst, cudaStream_t st) { k_store_scale<<<1, 1, 0, st>>>(s, dst); }

// Recompute pass of the checkpointed forward: out = P(scale * in) with the
// factor saved by the first forward pass, rounded as the forward check
// rounds it (scale_site), one site per thread on an (x, y, z) grid.
template <typename T>
__global__ void __launch_bounds__(256) k_scale_parity_from(const T* __restrict__ in, T* __restrict__ out, int n,
                                                           int mask, const double* __restrict__ scale) {
  using S = typename ScaleT<T>::S;
  const S s = (S)*scale;
  const int x0 = blockIdx.x * 32 + threadIdx.x, y0 = blockIdx.y * 8 + threadIdx.y, z0 = blockIdx.z;
  if (x0 >= n || y0 >= n) return;
  int c[3] = {x0, y0, z0};
  bool neg = false, zero = false;
  for (int ax = 0; ax < 3; ++ax) {
    int mode = (mask >> (2 * ax)) & 3;
    if (mode == 0) continue;
    int mm = n - 1 - c[ax];
    if (c[ax] > mm) {
      c[ax] = mm;
      neg ^= (mode == 2);
    } else if (c[ax] == mm && mode == 2) {
      zero = true;
    }
  }
  const S v = (S)Store<T>::to(in[site_index(c[0], c[1], c[2], n)]);
  out[site_index(x0, y0, z0, n)] = Store<T>::from(scale_site(v, s, neg, zero));
}
template <typename T>
void launch_scale_parity_from(const T* in, T* out, int n, int mask, const double* scale, cudaStream_t st) {
  k_scale_parity_from<T><<<dim3((n + 31) / 32, (n + 7) / 8, n), dim3(32, 8), 0, st>>>(in, out, n, mask, scale);
}
template void launch_scale_parity_from<double>(const double*, double*, int, int, const double*, cudaStream_t);
template void launch_scale_parity_from<float>(const float*, float*, int, int, const double*, cudaStream_t);

}  // namespace fdtd
