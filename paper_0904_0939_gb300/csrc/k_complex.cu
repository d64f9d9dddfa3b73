// Complex potentials (the paper's outlook, Sec. VIII): V = V_R + i V_I and a
// complex wavefunction, stored as interleaved (re, im) pairs of T (double for
// FDTD_C64 lattices, float for FDTD_C32).  The update keeps the form of
// Eq. updateeq with complex coefficients,
//     psi' = A psi + c B (S - 6 psi),  A = (1 - h)/(1 + h),  B = 1/(1 + h),
//     h = dtau V / 2,  c = dtau / (2 m a^2),  S = sum of the six neighbours,
// with A and cB formed once per site in FP64 when V is set.  The sums use
// the Hermitian inner product: S0 = sum |psi|^2, SH = sum conj(psi) H psi,
// Sr = sum r^2 |psi|^2, SV = sum V |psi|^2 (SH, SV complex), accumulated in
// FP64 in a fixed order.  Renormalisation, the symmetry masks of Sec. IV and
// the multi-resolution transfer of Sec. VI act on both parts alike.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace fdtd {

template <typename T>
struct Cx;
template <>
struct Cx<double> {
  using V = double2;
};
template <>
struct Cx<float> {
  using V = float2;
};

namespace {

size_t grid1(size_t total, int block) {
  size_t g = (total + block - 1) / block;
  return g < 152 * 32 ? (g < 1 ? 1 : g) : 152 * 32;
}

// ---------------------------------------------------------------- potential
// V (dense, x fastest; interleaved pairs if `cplx`, else real) -> V, A, cB of
// the lattice.  flags[0] |= 1: a value is not finite; |= 2: Re(1 + h) <= 0.
template <typename Ti, typename T>
__global__ void k_cset_potential(const Ti* __restrict__ in, int cplx, size_t count, size_t off,
                                 typename Cx<T>::V* __restrict__ v2, typename Cx<T>::V* __restrict__ a2,
                                 typename Cx<T>::V* __restrict__ cb2, double half_dtau, double c, int32_t* flags) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const double vr = (double)in[cplx ? 2 * i : i], vi = cplx ? (double)in[2 * i + 1] : 0.0;
    if (!isfinite(vr) || !isfinite(vi)) atomicOr(flags, 1);
    const double hr = half_dtau * vr, hi = half_dtau * vi;
    const double qr = 1.0 + hr;
    if (!(qr > 0.0)) atomicOr(flags, 2);
    // B = 1 / q = conj(q) / |q|^2,  A = (1 - h) B
    const double den = qr * qr + hi * hi;
    const double br = qr / den, bi = -hi / den;
    const double pr = 1.0 - hr, pi = -hi;
    const double ar = pr * br - pi * bi, ai = pr * bi + pi * br;
    const size_t j = off + i;
    v2[j].x = (T)vr;
    v2[j].y = (T)vi;
    a2[j].x = (T)ar;
    a2[j].y = (T)ai;
    cb2[j].x = (T)(c * br);
    cb2[j].y = (T)(c * bi);
  }
}

// ---------------------------------------------------------------- update
// One site per thread: 128 threads along x, one block row per (y, z).
template <typename T>
__global__ void __launch_bounds__(128) k_cstep(const typename Cx<T>::V* __restrict__ in, typename Cx<T>::V* __restrict__ out,
                                               const typename Cx<T>::V* __restrict__ a2,
                                               const typename Cx<T>::V* __restrict__ cb2, int n,
                                               const int32_t* __restrict__ active) {
  using V = typename Cx<T>::V;
  if (active && *active == 0) return;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= n) return;
  const size_t i = site_index(x, y, z, n);
  const size_t nn = (size_t)n * n;
  const V zero = {T(0), T(0)};
  const V c = in[i];
  const V xm = x > 0 ? in[i - 1] : zero, xp = x < n - 1 ? in[i + 1] : zero;
  const V ym = y > 0 ? in[i - n] : zero, yp = y < n - 1 ? in[i + n] : zero;
  const V zm = z > 0 ? in[i - nn] : zero, zp = z < n - 1 ? in[i + nn] : zero;
  // S = ((xm + xp) + (ym + yp)) + (zm + zp), each part on its own
  const T sr = ((xm.x + xp.x) + (ym.x + yp.x)) + (zm.x + zp.x);
  const T si = ((xm.y + xp.y) + (ym.y + yp.y)) + (zm.y + zp.y);
  const T lr = sr - T(6) * c.x, li = si - T(6) * c.y;
  const V A = a2[i], cB = cb2[i];
  V o;
  o.x = (A.x * c.x - A.y * c.y) + (cB.x * lr - cB.y * li);
  o.y = (A.x * c.y + A.y * c.x) + (cB.x * li + cB.y * lr);
  out[i] = o;
}

// ---------------------------------------------------------------- sums
constexpr int kCSumThreads = 256;

// Block b takes the (y, z) rows b, b + nb, ... in order, threads along x;
// six FP64 partials per block in a fixed-order block reduction.
template <typename T>
__global__ void __launch_bounds__(kCSumThreads) k_csums(const typename Cx<T>::V* __restrict__ psi,
                                                       const typename Cx<T>::V* __restrict__ v2, int n, double a,
                                                       double kfac, double* __restrict__ partials,
                                                       const int32_t* __restrict__ active) {
  using V = typename Cx<T>::V;
  if (active && *active == 0) return;
  __shared__ double red[6][kCSumThreads];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const size_t nn = (size_t)n * n;
  const double half = 0.5 * (double)(n - 1);
  for (int r = blockIdx.x; r < n * n; r += gridDim.x) {
    const int y = r % n, z = r / n;
    const double py = ((double)y - half) * a, pz = ((double)z - half) * a;
    for (int x = threadIdx.x; x < n; x += kCSumThreads) {
      const size_t i = site_index(x, y, z, n);
      auto at = [&](bool inside, size_t j) {
        const V q = inside ? psi[j] : V{T(0), T(0)};
        return make_double2((double)q.x, (double)q.y);
      };
      const double2 c = at(true, i);
      const double2 xm = at(x > 0, i - 1), xp = at(x < n - 1, i + 1);
      const double2 ym = at(y > 0, i - n), yp = at(y < n - 1, i + n);
      const double2 zm = at(z > 0, i - nn), zp = at(z < n - 1, i + nn);
      const double lr = (((xm.x + xp.x) + (ym.x + yp.x)) + (zm.x + zp.x)) - 6.0 * c.x;
      const double li = (((xm.y + xp.y) + (ym.y + yp.y)) + (zm.y + zp.y)) - 6.0 * c.y;
      const V vv = v2[i];
      const double vr = (double)vv.x, vi = (double)vv.y;
      // H psi = -kfac (S - 6 psi) + V psi
      const double hr = -kfac * lr + (vr * c.x - vi * c.y);
      const double hi = -kfac * li + (vr * c.y + vi * c.x);
      const double m2 = c.x * c.x + c.y * c.y;
      const double px = ((double)x - half) * a;
      acc[0] += m2;
      acc[1] += c.x * hr + c.y * hi;  // Re conj(psi) H psi
      acc[2] += c.x * hi - c.y * hr;  // Im conj(psi) H psi
      acc[3] += (px * px + py * py + pz * pz) * m2;
      acc[4] += vr * m2;
      acc[5] += vi * m2;
    }
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = kCSumThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < 6; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 6) partials[(size_t)blockIdx.x * 6 + threadIdx.x] = red[threadIdx.x][0];
}

// ---------------------------------------------------------------- renormalise + symmetry
// out(site) = sign * scale * in(source) on both parts (Secs. III, IV), with
// the factor and its gating of k_scale_parity: FP64 lattices multiply in
// FP64, FP32 ones by the factor rounded to FP32.
template <typename T>
__global__ void __launch_bounds__(256) k_cscale_parity(const typename Cx<T>::V* __restrict__ in,
                                                       typename Cx<T>::V* __restrict__ out, int n, int mask,
                                                       const LatState* __restrict__ s, int check_id, int out_idx,
                                                       LatState* sw) {
  T scale = T(1);
  if (s) {
    if (check_id < 0 ? s->post != 1 : s->scale_seq != check_id) return;
    scale = (T)s->scale;
  }
  const int x0 = blockIdx.x * 32 + threadIdx.x, y0 = blockIdx.y * 8 + threadIdx.y, z0 = blockIdx.z;
  if (sw && (x0 | y0 | z0) == 0) sw->cur = out_idx;
  if (x0 >= n || y0 >= n) return;
  int c[3] = {x0, y0, z0};
  bool neg = false, zero = false;
  for (int ax = 0; ax < 3; ++ax) {
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
  const typename Cx<T>::V v = in[site_index(c[0], c[1], c[2], n)];
  typename Cx<T>::V o;
  o.x = zero ? T(0) : (neg ? -(v.x * scale) : v.x * scale);
  o.y = zero ? T(0) : (neg ? -(v.y * scale) : v.y * scale);
  out[site_index(x0, y0, z0, n)] = o;
}

// ---------------------------------------------------------------- random start
// The real part takes the draws of the real lattices (k_init_random), the
// imaginary part starts at zero (the evolution builds it from V_I).
template <typename T>
__global__ void k_cinit_random(typename Cx<T>::V* __restrict__ out, int n, uint64_t seed, uint64_t lat, int dist) {
  const size_t total = (size_t)n * n * n;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    double val;
    if (dist == 1) {
      uint64_t d = (lat << 42) + 2ull * i;
      double u1 = unit_interval(sm64(seed, d)), u2 = unit_interval(sm64(seed, d + 1));
      val = sqrt(-2.0 * log(1.0 - u1)) * cos(2.0 * 3.14159265358979323846 * u2);  // Box-Muller
    } else {
      val = 2.0 * unit_interval(sm64(seed, (lat << 42) + i)) - 1.0;
    }
    out[i].x = (T)val;
    out[i].y = T(0);
  }
}

// ---------------------------------------------------------------- transfer
// The cell-centred trilinear map of k_upsample (Sec. VI), both parts, summed
// in FP64 (fine site x between coarse x/2 - 1 and x/2 for even x, (x-1)/2 and
// (x+1)/2 for odd x, weights 1/4 and 3/4; zero outside the coarse box).
template <typename Ti, typename To>
__global__ void k_cupsample(const typename Cx<Ti>::V* __restrict__ in, int nc, typename Cx<To>::V* __restrict__ out) {
  const int nf = 2 * nc;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= nf) return;
  int lo[3];
  double w[3][2];
  const int f[3] = {x, y, z};
  for (int ax = 0; ax < 3; ++ax) {
    if (f[ax] & 1) {
      lo[ax] = (f[ax] - 1) >> 1;
      w[ax][0] = 0.75;
      w[ax][1] = 0.25;
    } else {
      lo[ax] = (f[ax] >> 1) - 1;
      w[ax][0] = 0.25;
      w[ax][1] = 0.75;
    }
  }
  double ar = 0.0, ai = 0.0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const int cx = lo[0] + dx, cy = lo[1] + dy, cz = lo[2] + dz;
        if ((unsigned)cx >= (unsigned)nc || (unsigned)cy >= (unsigned)nc || (unsigned)cz >= (unsigned)nc) continue;
        const double wt = w[0][dx] * w[1][dy] * w[2][dz];
        const typename Cx<Ti>::V q = in[site_index(cx, cy, cz, nc)];
        ar += wt * (double)q.x;
        ai += wt * (double)q.y;
      }
  out[((size_t)z * nf + y) * nf + x].x = (To)ar;
  out[((size_t)z * nf + y) * nf + x].y = (To)ai;
}

}  // namespace

int csums_blocks(int n) { return (int)std::min<long long>((long long)n * n, 152 * 8); }

template <typename T>
void launch_cset_potential(const void* in, int in_f64, int in_complex, size_t count, size_t off, T* v2, T* a2, T* cb2,
                           const Params& p, int32_t* flags, cudaStream_t st) {
  using V = typename Cx<T>::V;
  const size_t g = grid1(count, 256);
  if (in_f64)
    k_cset_potential<double, T><<<g, 256, 0, st>>>((const double*)in, in_complex, count, off, (V*)v2, (V*)a2,
                                                    (V*)cb2, 0.5 * p.dtau, p.c, flags);
  else
    k_cset_potential<float, T><<<g, 256, 0, st>>>((const float*)in, in_complex, count, off, (V*)v2, (V*)a2, (V*)cb2,
                                                   0.5 * p.dtau, p.c, flags);
}

template <typename T>
void launch_cstep(const T* in, T* out, const T* a2, const T* cb2, const Params& p, const int32_t* active,
                  cudaStream_t st) {
  using V = typename Cx<T>::V;
  dim3 grid((p.n + 127) / 128, p.n, p.n);
  k_cstep<T><<<grid, 128, 0, st>>>((const V*)in, (V*)out, (const V*)a2, (const V*)cb2, p.n, active);
}

template <typename T>
int launch_csums(const T* psi, const T* v2, const Params& p, double* partials, const int32_t* active, cudaStream_t st) {
  using V = typename Cx<T>::V;
  const int nb = csums_blocks(p.n);
  k_csums<T><<<nb, kCSumThreads, 0, st>>>((const V*)psi, (const V*)v2, p.n, p.a, 1.0 / (2.0 * p.mass * p.a * p.a),
                                          partials, active);
  return nb;
}

template <typename T>
void launch_cscale_parity(const T* in, T* out, int n, int mask, const LatState* s, int check_id, int out_idx,
                          LatState* sw, cudaStream_t st) {
  using V = typename Cx<T>::V;
  dim3 grid((n + 31) / 32, (n + 7) / 8, n);
  k_cscale_parity<T><<<grid, dim3(32, 8), 0, st>>>((const V*)in, (V*)out, n, mask, s, check_id, out_idx, sw);
}

template <typename T>
void launch_cinit_random(T* out, int n, uint64_t seed, uint64_t lat, int dist, cudaStream_t st) {
  using V = typename Cx<T>::V;
  const size_t total = (size_t)n * n * n;
  k_cinit_random<T><<<grid1(total, 256), 256, 0, st>>>((V*)out, n, seed, lat, dist);
}

template <typename Ti, typename To>
void launch_cupsample(const Ti* in, int nc, To* out, cudaStream_t st) {
  dim3 grid((2 * nc + 127) / 128, 2 * nc, 2 * nc);
  k_cupsample<Ti, To><<<grid, 128, 0, st>>>((const typename Cx<Ti>::V*)in, nc, (typename Cx<To>::V*)out);
}

#define INST_C(T)                                                                                                \
  template void launch_cset_potential<T>(const void*, int, int, size_t, size_t, T*, T*, T*, const Params&,       \
                                         int32_t*, cudaStream_t);                                                \
  template void launch_cstep<T>(const T*, T*, const T*, const T*, const Params&, const int32_t*, cudaStream_t);   \
  template int launch_csums<T>(const T*, const T*, const Params&, double*, const int32_t*, cudaStream_t);         \
  template void launch_cscale_parity<T>(const T*, T*, int, int, const LatState*, int, int, LatState*,             \
                                        cudaStream_t);                                                           \
  template void launch_cinit_random<T>(T*, int, uint64_t, uint64_t, int, cudaStream_t);
INST_C(double)
INST_C(float)
template void launch_cupsample<double, double>(const double*, int, double*, cudaStream_t);
template void launch_cupsample<double, float>(const double*, int, float*, cudaStream_t);
template void launch_cupsample<float, double>(const float*, int, double*, cudaStream_t);
template void launch_cupsample<float, float>(const float*, int, float*, cudaStream_t);

}  // namespace fdtd
