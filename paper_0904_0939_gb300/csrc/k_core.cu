// Core FDTD kernels for sm_103a: the one-step 7-point update (Eq. updateeq),
// the fused lattice sums of Eq. energysum, the check finaliser, the
// renormalisation + symmetry pass (Secs. III-IV), the random start, the
// multi-resolution transfer (Sec. VI) and the potential loader.
//
// The stencil and the sums share one traversal: a block of 32 x 8 threads
// owns a 32 x 8 column of sites and walks `zc` consecutive z-planes.  Each
// thread keeps psi(z-1), psi(z), psi(z+1) of its own column in registers
// (the z-neighbours), exchanges x-neighbours by warp shuffles (a warp is one
// x-row of the tile) and reads y-neighbours from a double-buffered shared
// row tile; only the tile's rim is loaded twice.  Loads for plane z+1 are
// issued one iteration ahead.  HBM traffic is the ideal one-read-one-write
// of psi plus one read of V per site.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace fdtd {

constexpr int TX = 32, TY = 8;

Tiling tiling_for(int n, int min_blocks) {
  Tiling t;
  int bx = (n + TX - 1) / TX, by = (n + TY - 1) / TY;
  int zc = n;
  while (zc > 8 && (long long)bx * by * ((n + zc - 1) / zc) < min_blocks) zc = (zc + 1) / 2;
  t.zc = zc;
  t.grid = dim3(bx, by, (n + zc - 1) / zc);
  return t;
}

template <typename C>
struct RowTile {
  C r[2][TY + 2][TX];
};

// P: periodic boundaries (every load wraps modulo n, so the tile's rim and
// the z-neighbours of the first and last planes come from the opposite side);
// otherwise sites beyond the lattice read as zero.  The marched field is
// get(i) at the site of linear index i: a stored field, or one computed from
// stored fields as it is loaded.
template <typename C, bool P, typename Get, typename Body>
__device__ __forceinline__ void zmarch_fn(int n, int zc, RowTile<C>& tile, Get&& get, Body&& body) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x = blockIdx.x * TX + tx, y = blockIdx.y * TY + ty;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, n);
  const bool act = (x < n) && (y < n);
  auto ld = [&](int xx, int yy, int zz) -> C {
    if constexpr (P) {
      auto wrap = [n](int q) {
        q %= n;
        return q < 0 ? q + n : q;
      };
      return get(site_index(wrap(xx), wrap(yy), wrap(zz), n));
    } else {
      if ((unsigned)xx < (unsigned)n && (unsigned)yy < (unsigned)n && (unsigned)zz < (unsigned)n)
        return get(site_index(xx, yy, zz, n));
      return C(0);
    }
  };
  const bool hy_lo = (ty == 0), hy_hi = (ty == TY - 1), hx_lo = (tx == 0), hx_hi = (tx == TX - 1);
  const int hy = hy_lo ? y - 1 : y + 1;
  C zm = ld(x, y, z0 - 1), c = ld(x, y, z0), zp = ld(x, y, z0 + 1);
  C hyv = (hy_lo || hy_hi) ? ld(x, hy, z0) : C(0);
  C hxm = hx_lo ? ld(x - 1, y, z0) : C(0);
  C hxp = hx_hi ? ld(x + 1, y, z0) : C(0);
  for (int z = z0; z < z1; ++z) {
    C zpp = ld(x, y, z + 2);
    C hyv_n = (hy_lo || hy_hi) ? ld(x, hy, z + 1) : C(0);
    C hxm_n = hx_lo ? ld(x - 1, y, z + 1) : C(0);
    C hxp_n = hx_hi ? ld(x + 1, y, z + 1) : C(0);
    const int b = (z - z0) & 1;
    tile.r[b][ty + 1][tx] = c;
    if (hy_lo) tile.r[b][0][tx] = hyv;
    if (hy_hi) tile.r[b][TY + 1][tx] = hyv;
    C xm = __shfl_up_sync(0xffffffffu, c, 1);
    C xp = __shfl_down_sync(0xffffffffu, c, 1);
    if (hx_lo) xm = hxm;
    if (hx_hi) xp = hxp;
    __syncthreads();
    C ym = tile.r[b][ty][tx], yp = tile.r[b][ty + 2][tx];
    body(x, y, z, act, c, xm, xp, ym, yp, zm, zp);
    zm = c;
    c = zp;
    zp = zpp;
    hyv = hyv_n;
    hxm = hxm_n;
    hxp = hxp_n;
  }
}

template <typename T, bool P, typename Body>
__device__ __forceinline__ void zmarch(const T* __restrict__ in, int n, int zc, RowTile<typename Store<T>::C>& tile,
                                       Body&& body) {
  zmarch_fn<typename Store<T>::C, P>(
      n, zc, tile, [in](size_t i) { return Store<T>::ld(in + i); }, body);
}

// ------------------------------------------------------------------ update
template <bool P>
__global__ void __launch_bounds__(TX* TY) k_step_f64(const double* __restrict__ in, double* __restrict__ out,
                                                     const double* __restrict__ coefA,
                                                     const double* __restrict__ coefCB, int n, int zc,
                                                     const int32_t* __restrict__ active) {
  pdl_wait();
  pdl_trigger();
  if (active && *active == 0) return;
  __shared__ RowTile<double> tile;
  zmarch<double, P>(in, n, zc, tile,
                    [&](int x, int y, int z, bool act, double c, double xm, double xp, double ym, double yp, double zm,
                        double zp) {
                   if (!act) return;
                   size_t i = site_index(x, y, z, n);
                   double s = nbr_sum(xm, xp, ym, yp, zm, zp);
                   out[i] = update_f64(c, s, __ldg(coefA + i), __ldg(coefCB + i));
                 });
}

template <typename T, bool P>
__global__ void __launch_bounds__(TX* TY) k_step_f32(const T* __restrict__ in, T* __restrict__ out,
                                                     const float* __restrict__ v, int n, int zc, float half_dtau,
                                                     float one_m6c, float cc, const int32_t* __restrict__ active) {
  pdl_wait();
  pdl_trigger();
  if (active && *active == 0) return;
  __shared__ RowTile<float> tile;
  zmarch<T, P>(in, n, zc, tile,
            [&](int x, int y, int z, bool act, float c, float xm, float xp, float ym, float yp, float zm, float zp) {
              if (!act) return;
              size_t i = site_index(x, y, z, n);
              CoefF k = coef_f32(__ldg(v + i), half_dtau, one_m6c);
              float s = nbr_sum(xm, xp, ym, yp, zm, zp);
              out[i] = Store<T>::from(update_f32(c, s, k, cc));
            });
}

void launch_step_f64(const double* in, double* out, const double* coefA, const double* coefCB, const Params& p,
                     const int32_t* active, cudaStream_t st) {
  Tiling t = tiling_for(p.n, 1216);
  launch_pdl(p.periodic ? k_step_f64<true> : k_step_f64<false>, t.grid, dim3(TX, TY), 0, st, in, out, coefA, coefCB,
             p.n, t.zc, active);
}

template <typename T>
void launch_step_f32(const T* in, T* out, const float* v, const Params& p, const int32_t* active, cudaStream_t st) {
  Tiling t = tiling_for(p.n, 1216);
  launch_pdl(p.periodic ? k_step_f32<T, true> : k_step_f32<T, false>, t.grid, dim3(TX, TY), 0, st, in, out, v, p.n,
             t.zc, p.half_dtau_f, p.one_m6c_f, p.c_f, active);
}
template void launch_step_f32<float>(const float*, float*, const float*, const Params&, const int32_t*, cudaStream_t);
template void launch_step_f32<__nv_bfloat16>(const __nv_bfloat16*, __nv_bfloat16*, const float*, const Params&,
                                             const int32_t*, cudaStream_t);

// ------------------------------------------------------------------ direct stencil
// One thread per four consecutive x sites (n % 4 == 0) and every neighbour an
// independent load instead of a z-march: on lattices too small to give a
// z-marching grid many planes per block, each thread's loads no longer wait
// on one another plane by plane.  FP32 or BF16 storage (four BF16 sites are
// one 8-byte load); the per-site arithmetic and the rounding of the stored
// value are k_step_f32's (same bits).
template <typename T>
struct Quad;
template <>
struct Quad<float> {
  __device__ __forceinline__ static float4 ld(const float* base, size_t q) {
    return __ldg(reinterpret_cast<const float4*>(base) + q);
  }
  __device__ __forceinline__ static void st(float* base, size_t q, float4 o) {
    reinterpret_cast<float4*>(base)[q] = o;
  }
};
template <>
struct Quad<__nv_bfloat16> {
  __device__ __forceinline__ static float4 ld(const __nv_bfloat16* base, size_t q) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(base) + q);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
  }
  __device__ __forceinline__ static void st(__nv_bfloat16* base, size_t q, float4 o) {
    __nv_bfloat162 a, b;
    a.x = Store<__nv_bfloat16>::from(o.x);
    a.y = Store<__nv_bfloat16>::from(o.y);
    b.x = Store<__nv_bfloat16>::from(o.z);
    b.y = Store<__nv_bfloat16>::from(o.w);
    uint2 u;
    u.x = *reinterpret_cast<const unsigned*>(&a);
    u.y = *reinterpret_cast<const unsigned*>(&b);
    reinterpret_cast<uint2*>(base)[q] = u;
  }
};

template <typename T, bool P>
__global__ void __launch_bounds__(256) k_direct(const T* __restrict__ in, T* __restrict__ out,
                                                const float* __restrict__ v, int n, float half_dtau, float one_m6c,
                                                float cc, const int32_t* __restrict__ active) {
  pdl_wait();
  pdl_trigger();
  if (active && *active == 0) return;
  const int n4 = n >> 2;
  const size_t total = (size_t)n4 * n * n;
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  auto wrap = [n](int q) { return q < 0 ? q + n : (q >= n ? q - n : q); };
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int x4 = (int)(q % n4);
    const size_t row = q / n4;  // z n + y
    const int y = (int)(row % n), z = (int)(row / n);
    auto at = [&](int yy, int zz) -> float4 {
      if constexpr (P) {
        yy = wrap(yy);
        zz = wrap(zz);
      } else if ((unsigned)yy >= (unsigned)n || (unsigned)zz >= (unsigned)n) {
        return zero4;
      }
      return Quad<T>::ld(in, ((size_t)zz * n + yy) * n4 + x4);
    };
    const float4 c = Quad<T>::ld(in, q);
    const float4 ym = at(y - 1, z), yp = at(y + 1, z), zm = at(y, z - 1), zp = at(y, z + 1);
    const T* rp = in + row * n;
    float xl, xr;
    if constexpr (P) {
      xl = Store<T>::ld(rp + (x4 == 0 ? n - 1 : 4 * x4 - 1));
      xr = Store<T>::ld(rp + (x4 == n4 - 1 ? 0 : 4 * x4 + 4));
    } else {
      xl = x4 > 0 ? Store<T>::ld(rp + 4 * x4 - 1) : 0.f;
      xr = x4 < n4 - 1 ? Store<T>::ld(rp + 4 * x4 + 4) : 0.f;
    }
    const float4 vv = __ldg(reinterpret_cast<const float4*>(v) + q);
    auto site = [&](float cv, float s, float vs) { return update_f32(cv, s, coef_f32(vs, half_dtau, one_m6c), cc); };
    float4 o;
    o.x = site(c.x, nbr_sum(xl, c.y, ym.x, yp.x, zm.x, zp.x), vv.x);
    o.y = site(c.y, nbr_sum(c.x, c.z, ym.y, yp.y, zm.y, zp.y), vv.y);
    o.z = site(c.z, nbr_sum(c.y, c.w, ym.z, yp.z, zm.z, zp.z), vv.z);
    o.w = site(c.w, nbr_sum(c.z, xr, ym.w, yp.w, zm.w, zp.w), vv.w);
    Quad<T>::st(out, q, o);
  }
}

static int grid_f4(int n) {
  const size_t total = (size_t)(n >> 2) * n * n;
  const size_t b = (total + 255) / 256;
  return (int)std::max<size_t>(1, std::min<size_t>(b, 152 * 64));
}

template <typename T>
void launch_direct(const T* in, T* out, const float* v, const Params& p, const int32_t* active, cudaStream_t st) {
  launch_pdl(p.periodic ? k_direct<T, true> : k_direct<T, false>, dim3(grid_f4(p.n)), dim3(256), 0, st, in, out, v,
             p.n, p.half_dtau_f, p.one_m6c_f, p.c_f, active);
}
template void launch_direct<float>(const float*, float*, const float*, const Params&, const int32_t*, cudaStream_t);
template void launch_direct<__nv_bfloat16>(const __nv_bfloat16*, __nv_bfloat16*, const float*, const Params&,
                                           const int32_t*, cudaStream_t);

void launch_direct_f32(const float* in, float* out, const float* v, const Params& p, const int32_t* active,
                       cudaStream_t st) {
  launch_direct<float>(in, out, v, p, active, st);
}

// One whole FP32 adjoint step, four x sites per thread (n % 4 == 0), no
// z-march: with u = B lam formed as each value is loaded (B from V as the
// forward computes it),
//   lam_out = c Adj(u) + alpha u   and   g_V += -(dtau/2) u (psi_next + psi_prev),
// the transpose of psi' = B (c Adj + alpha) psi and its site derivative.
// The rounding is that of k_adjoint_step_f32 (same bits); u at the six
// neighbours is recomputed (5.5 reciprocals per site) instead of stored.
template <bool P>
__global__ void __launch_bounds__(256) k_adjoint_direct_f32(const float* __restrict__ lam,
                                                            const float* __restrict__ psi_prev,
                                                            const float* __restrict__ psi_next,
                                                            const float* __restrict__ v, float* __restrict__ lam_out,
                                                            double* __restrict__ gv, int n, float half_dtau,
                                                            float one_m6c, float cc) {
  pdl_wait();
  pdl_trigger();
  const int n4 = n >> 2;
  const size_t total = (size_t)n4 * n * n;
  const float4* l4 = reinterpret_cast<const float4*>(lam);
  const float4* v4 = reinterpret_cast<const float4*>(v);
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  auto wrap = [n](int q) { return q < 0 ? q + n : (q >= n ? q - n : q); };
  auto b = [&](float vs) { return coef_f32(vs, half_dtau, one_m6c).b; };
  auto u1 = [&](size_t i) { return __fmul_rn(b(__ldg(v + i)), __ldg(lam + i)); };
  auto u4 = [&](size_t i4) {
    const float4 l = __ldg(l4 + i4), vv = __ldg(v4 + i4);
    return make_float4(__fmul_rn(b(vv.x), l.x), __fmul_rn(b(vv.y), l.y), __fmul_rn(b(vv.z), l.z),
                       __fmul_rn(b(vv.w), l.w));
  };
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int x4 = (int)(q % n4);
    const size_t row = q / n4;  // z n + y
    const int y = (int)(row % n), z = (int)(row / n);
    auto at = [&](int yy, int zz) -> float4 {
      if constexpr (P) {
        yy = wrap(yy);
        zz = wrap(zz);
      } else if ((unsigned)yy >= (unsigned)n || (unsigned)zz >= (unsigned)n) {
        return zero4;
      }
      return u4(((size_t)zz * n + yy) * n4 + x4);
    };
    const float4 vv = __ldg(v4 + q), l = __ldg(l4 + q);
    const float4 c = make_float4(__fmul_rn(b(vv.x), l.x), __fmul_rn(b(vv.y), l.y), __fmul_rn(b(vv.z), l.z),
                                 __fmul_rn(b(vv.w), l.w));
    const float4 ym = at(y - 1, z), yp = at(y + 1, z), zm = at(y, z - 1), zp = at(y, z + 1);
    const size_t r0 = row * n;
    float xl, xr;
    if constexpr (P) {
      xl = u1(r0 + (x4 == 0 ? n - 1 : 4 * x4 - 1));
      xr = u1(r0 + (x4 == n4 - 1 ? 0 : 4 * x4 + 4));
    } else {
      xl = x4 > 0 ? u1(r0 + 4 * x4 - 1) : 0.f;
      xr = x4 < n4 - 1 ? u1(r0 + 4 * x4 + 4) : 0.f;
    }
    const float4 pp = __ldg(reinterpret_cast<const float4*>(psi_prev) + q);
    const float4 pn = __ldg(reinterpret_cast<const float4*>(psi_next) + q);
    auto out = [&](float cu, float s, float vs) {
      const float alpha = __fsub_rn(one_m6c, __fmul_rn(half_dtau, vs));
      return __fmaf_rn(cc, s, __fmul_rn(alpha, cu));
    };
    float4 o;
    o.x = out(c.x, nbr_sum(xl, c.y, ym.x, yp.x, zm.x, zp.x), vv.x);
    o.y = out(c.y, nbr_sum(c.x, c.z, ym.y, yp.y, zm.y, zp.y), vv.y);
    o.z = out(c.z, nbr_sum(c.y, c.w, ym.z, yp.z, zm.z, zp.z), vv.z);
    o.w = out(c.w, nbr_sum(c.z, xr, ym.w, yp.w, zm.w, zp.w), vv.w);
    reinterpret_cast<float4*>(lam_out)[q] = o;
    double2* g2 = reinterpret_cast<double2*>(gv) + 2 * q;
    double2 g0 = g2[0], g1 = g2[1];
    auto dg = [&](float cu, float a, float bb) {
      return (double)__fmul_rn(__fmul_rn(-half_dtau, cu), __fadd_rn(bb, a));
    };
    g0.x = __dadd_rn(g0.x, dg(c.x, pp.x, pn.x));
    g0.y = __dadd_rn(g0.y, dg(c.y, pp.y, pn.y));
    g1.x = __dadd_rn(g1.x, dg(c.z, pp.z, pn.z));
    g1.y = __dadd_rn(g1.y, dg(c.w, pp.w, pn.w));
    g2[0] = g0;
    g2[1] = g1;
  }
}

void launch_adjoint_direct_f32(const float* lam, const float* psi_prev, const float* psi_next, const float* v,
                               float* lam_out, double* gv, const Params& p, cudaStream_t st) {
  launch_pdl(p.periodic ? k_adjoint_direct_f32<true> : k_adjoint_direct_f32<false>, dim3(grid_f4(p.n)), dim3(256), 0,
             st, lam, psi_prev, psi_next, v, lam_out, gv, p.n, p.half_dtau_f, p.one_m6c_f, p.c_f);
}

// ------------------------------------------------------------------ adjoint stencil
// lam_out = A lam + c (sum of the 6 neighbours of u - 6 u), u = B lam given;
// the transpose of the update with the symmetric lattice Laplacian.
template <typename T, bool P>
__global__ void __launch_bounds__(TX* TY) k_adjoint_stencil(const T* __restrict__ u, const T* __restrict__ lam,
                                                            T* __restrict__ lam_out, const void* __restrict__ v,
                                                            const double* __restrict__ coefA, int n, int zc,
                                                            float half_dtau, float one_m6c, float cc, double c64) {
  using C = typename Store<T>::C;
  __shared__ RowTile<C> tile;
  zmarch<T, P>(u, n, zc, tile, [&](int x, int y, int z, bool act, C cu, C xm, C xp, C ym, C yp, C zm, C zp) {
    if (!act) return;
    size_t i = site_index(x, y, z, n);
    if constexpr (sizeof(T) == 8) {
      double s = nbr_sum(xm, xp, ym, yp, zm, zp);
      lam_out[i] = __fma_rn(c64, __fma_rn(-6.0, cu, s), __dmul_rn(coefA[i], (double)lam[i]));
    } else {
      CoefF k = coef_f32(__ldg((const float*)v + i), half_dtau, one_m6c);
      float A = k.b * (k.alpha + 6.0f * cc);
      float s = nbr_sum(xm, xp, ym, yp, zm, zp);
      lam_out[i] = Store<T>::from(__fmaf_rn(cc, __fmaf_rn(-6.0f, cu, s), A * Store<T>::to(lam[i])));
    }
  });
}

template <typename T>
void launch_adjoint_stencil(const T* u, const T* lam, T* lam_out, const void* v, const double* coefA, const Params& p,
                            cudaStream_t st) {
  Tiling t = tiling_for(p.n, 1216);
  auto k = p.periodic ? k_adjoint_stencil<T, true> : k_adjoint_stencil<T, false>;
  k<<<t.grid, dim3(TX, TY), 0, st>>>(u, lam, lam_out, v, coefA, p.n, t.zc, p.half_dtau_f, p.one_m6c_f, p.c_f, p.c);
}
template void launch_adjoint_stencil<double>(const double*, const double*, double*, const void*, const double*,
                                             const Params&, cudaStream_t);
template void launch_adjoint_stencil<float>(const float*, const float*, float*, const void*, const double*,
                                            const Params&, cudaStream_t);

// One whole FP32 adjoint step in one pass.  The FP32 update is
// psi' = B (c Adj psi + alpha psi), i.e. M = diag(B) (c Adj + diag(alpha)),
// so with u = B lam
//   M^T lam = c Adj(u) + alpha u,
// and the site derivative d psi'(s)/dV(s) = -(dtau/2) B (psi' + psi) gives
//   g_V += -(dtau/2) u (psi_next + psi_prev).
// u is formed as the z-march loads it (B from V as the forward computes it),
// the per-site terms are FP32 and g_V accumulates in FP64.
template <bool P>
__global__ void __launch_bounds__(TX* TY) k_adjoint_step_f32(const float* __restrict__ lam,
                                                             const float* __restrict__ psi_prev,
                                                             const float* __restrict__ psi_next,
                                                             const float* __restrict__ v, float* __restrict__ lam_out,
                                                             double* __restrict__ gv, int n, int zc, float half_dtau,
                                                             float one_m6c, float cc) {
  pdl_wait();
  pdl_trigger();
  __shared__ RowTile<float> tile;
  zmarch_fn<float, P>(
      n, zc, tile,
      [&](size_t i) { return __fmul_rn(coef_f32(__ldg(v + i), half_dtau, one_m6c).b, __ldg(lam + i)); },
      [&](int x, int y, int z, bool act, float cu, float xm, float xp, float ym, float yp, float zm, float zp) {
        if (!act) return;
        const size_t i = site_index(x, y, z, n);
        const float alpha = __fsub_rn(one_m6c, __fmul_rn(half_dtau, __ldg(v + i)));
        lam_out[i] = __fmaf_rn(cc, nbr_sum(xm, xp, ym, yp, zm, zp), __fmul_rn(alpha, cu));
        const float d = __fmul_rn(__fmul_rn(-half_dtau, cu), __fadd_rn(__ldg(psi_next + i), __ldg(psi_prev + i)));
        gv[i] = __dadd_rn(gv[i], (double)d);
      });
}

void launch_adjoint_step_f32(const float* lam, const float* psi_prev, const float* psi_next, const float* v,
                             float* lam_out, double* gv, const Params& p, cudaStream_t st) {
  Tiling t = tiling_for(p.n, 1216);
  launch_pdl(p.periodic ? k_adjoint_step_f32<true> : k_adjoint_step_f32<false>, t.grid, dim3(TX, TY), 0, st, lam,
             psi_prev, psi_next, v, lam_out, gv, p.n, t.zc, p.half_dtau_f, p.one_m6c_f, p.c_f);
}

// ------------------------------------------------------------------ sums
__device__ __forceinline__ void block_sum4_store(double v0, double v1, double v2, double v3, double* dst) {
  __shared__ double red[TY][4];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v0 += __shfl_down_sync(0xffffffffu, v0, off);
    v1 += __shfl_down_sync(0xffffffffu, v1, off);
    v2 += __shfl_down_sync(0xffffffffu, v2, off);
    v3 += __shfl_down_sync(0xffffffffu, v3, off);
  }
  if (threadIdx.x == 0) {
    red[threadIdx.y][0] = v0;
    red[threadIdx.y][1] = v1;
    red[threadIdx.y][2] = v2;
    red[threadIdx.y][3] = v3;
  }
  __syncthreads();
  if (threadIdx.y == 0 && threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < TY; ++w) s += red[w][threadIdx.x];
    size_t b = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    dst[b * 4 + threadIdx.x] = s;
  }
}

// FP64: every term and sum in FP64.
template <bool P>
__global__ void __launch_bounds__(TX* TY) k_sums_f64(const double* __restrict__ psi, const double* __restrict__ v,
                                                     int n, int zc, double a, double kfac, double* partials,
                                                     const int32_t* __restrict__ active) {
  pdl_wait();
  pdl_trigger();
  if (active && *active == 0) return;
  __shared__ RowTile<double> tile;
  double s0 = 0, sh = 0, sr = 0, sv = 0;
  zmarch<double, P>(psi, n, zc, tile,
                 [&](int x, int y, int z, bool act, double c, double xm, double xp, double ym, double yp, double zm,
                     double zp) {
                   if (!act) return;
                   size_t i = site_index(x, y, z, n);
                   double vv = __ldg(v + i);
                   double lap = __fma_rn(-6.0, c, nbr_sum(xm, xp, ym, yp, zm, zp));
                   double px = coord_f64(x, n, a), py = coord_f64(y, n, a), pz = coord_f64(z, n, a);
                   double c2 = c * c;
                   s0 += c2;
                   sh += c * (-kfac * lap + vv * c);
                   sr += (px * px + py * py + pz * pz) * c2;
                   sv += vv * c2;
                 });
  block_sum4_store(s0, sh, sr, sv, partials);
}

// FP32 / BF16 storage: per-site terms in FP32, Kahan-compensated FP32 runs
// per thread, FP64 across threads and blocks.
template <typename T, bool P>
__global__ void __launch_bounds__(TX* TY) k_sums_f32(const T* __restrict__ psi, const float* __restrict__ v, int n,
                                                     int zc, float a, float kfac, double* partials,
                                                     const int32_t* __restrict__ active) {
  pdl_wait();
  pdl_trigger();
  if (active && *active == 0) return;
  __shared__ RowTile<float> tile;
  Kahan s0, sh, sr, sv;
  zmarch<T, P>(psi, n, zc, tile,
            [&](int x, int y, int z, bool act, float c, float xm, float xp, float ym, float yp, float zm, float zp) {
              if (!act) return;
              size_t i = site_index(x, y, z, n);
              float vv = __ldg(v + i);
              // sum of neighbour differences: each difference is exact when
              // the neighbours are within a factor 2 of psi (Sterbenz), so the
              // kinetic term loses far less to cancellation than S - 6 psi
              float lap = ((__fsub_rn(xm, c) + __fsub_rn(xp, c)) + (__fsub_rn(ym, c) + __fsub_rn(yp, c))) +
                          (__fsub_rn(zm, c) + __fsub_rn(zp, c));
              float px = coord_f32(x, n, a), py = coord_f32(y, n, a), pz = coord_f32(z, n, a);
              float c2 = c * c;
              s0.add(c2);
              sh.add(c * (-kfac * lap + vv * c));
              sr.add((px * px + py * py + pz * pz) * c2);
              sv.add(vv * c2);
            });
  block_sum4_store(s0.value(), sh.value(), sr.value(), sv.value(), partials);
}

static Tiling sums_tiling(int n) { return tiling_for(n, 1216); }
int sums_blocks(int n) {
  Tiling t = sums_tiling(n);
  return (int)(t.grid.x * t.grid.y * t.grid.z);
}

template <>
int launch_sums<double>(const double* psi, const void* v, const Params& p, double* partials, const int32_t* active,
                        cudaStream_t st) {
  Tiling t = sums_tiling(p.n);
  launch_pdl(p.periodic ? k_sums_f64<true> : k_sums_f64<false>, t.grid, dim3(TX, TY), 0, st, psi, (const double*)v,
             p.n, t.zc, p.a,
             1.0 / (2.0 * p.mass * p.a * p.a), partials, active);
  return (int)(t.grid.x * t.grid.y * t.grid.z);
}
template <typename T>
int launch_sums(const T* psi, const void* v, const Params& p, double* partials, const int32_t* active,
                cudaStream_t st) {
  Tiling t = sums_tiling(p.n);
  launch_pdl(p.periodic ? k_sums_f32<T, true> : k_sums_f32<T, false>, t.grid, dim3(TX, TY), 0, st, psi,
             (const float*)v, p.n, t.zc, (float)p.a,
             (float)(1.0 / (2.0 * p.mass * p.a * p.a)), partials, active);
  return (int)(t.grid.x * t.grid.y * t.grid.z);
}
template int launch_sums<float>(const float*, const void*, const Params&, double*, const int32_t*, cudaStream_t);
template int launch_sums<__nv_bfloat16>(const __nv_bfloat16*, const void*, const Params&, double*, const int32_t*,
                                        cudaStream_t);

// ------------------------------------------------------------------ check
// One block: deterministic reduction of the partials, then the check of
// Secs. III-V on thread 0.
// NS = 4: real lattices (S0, SH, Sr, SV per block); NS = 6: complex lattices
// (S0, Re SH, Im SH, Sr, Re SV, Im SV), whose E and <V> get imaginary parts
// and whose convergence test takes the complex modulus of the change of E_b.
template <int NS>
__global__ void __launch_bounds__(256) k_finalize(LatState* s, const double* __restrict__ parts, int np, int check_id,
                                                  int64_t t, double a3, double v_inf, double tol, int tol_rel,
                                                  int record, int seq_ce, cudaGraphConditionalHandle cond,
                                                  const int32_t* err, double* hist) {
  pdl_wait();
  pdl_trigger();
  const bool seq = seq_ce > 0;
  if (record && s->active == 0) {
    if (seq && threadIdx.x == 0) {
      s->post = 0;
      cudaGraphSetConditional(cond, 0u);
    }
    return;
  }
  __shared__ double sm[NS][256];
  double acc[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) acc[q] = 0.0;
  for (int i = threadIdx.x; i < np; i += 256)
#pragma unroll
    for (int q = 0; q < NS; ++q) acc[q] += parts[(size_t)i * NS + q];
#pragma unroll
  for (int q = 0; q < NS; ++q) sm[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < NS; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  if (seq) {
    check_id = s->checks;
    t = (int64_t)check_id * seq_ce;
  }
  const double s0 = sm[0][0];
  const double sh = sm[1][0], shi = NS == 6 ? sm[2][0] : 0.0;
  const double sr = sm[NS == 6 ? 3 : 2][0];
  const double sv = sm[NS == 6 ? 4 : 3][0], svi = NS == 6 ? sm[5][0] : 0.0;
  if (!(s0 > 0.0) || !isfinite(s0) || !isfinite(sh) || !isfinite(sr) || !isfinite(sv) || !isfinite(shi) ||
      !isfinite(svi)) {
    s->status = STATUS_NONFINITE;
    s->active = 0;
    s->scale_seq = -1;
    if (seq) {
      s->post = 0;
      cudaGraphSetConditional(cond, 0u);
    }
    return;
  }
  s->scale = 1.0 / sqrt(s0 * a3);
  s->scale_seq = check_id;
  if (seq) s->post = 1;
  if (!record) return;
  double e = sh / s0, eb = e - v_inf, ei = shi / s0;
  s->s0 = s0;
  s->sh = sh;
  s->sr = sr;
  s->sv = sv;
  s->energy = e;
  s->energy_im = ei;
  s->ebind = eb;
  s->r2 = sr / s0;
  s->vexp = sv / s0;
  s->vexp_im = svi / s0;
  s->step = t;
  s->checks += 1;
  double d = -1.0;
  if (s->has_prev) {
    d = NS == 6 ? hypot(eb - s->e_prev, ei - s->e_prev_im) : fabs(eb - s->e_prev);
    double thr = tol * (tol_rel ? (NS == 6 ? hypot(eb, ei) : fabs(eb)) : 1.0);
    if (tol > 0.0 && d <= thr) {
      s->converged = 1;
      s->active = 0;
    }
  }
  s->delta_e = d;
  s->e_prev = eb;
  s->e_prev_im = ei;
  s->has_prev = 1;
  if (hist) {
    double* h = hist + (size_t)((s->checks - 1) % kHistCap) * kHistFields;
    h[0] = (double)t;
    h[1] = e;
    h[2] = eb;
    h[3] = s0 * a3;
    h[4] = sr / s0;
    h[5] = sv / s0;
    h[6] = d;
    h[7] = s0;
  }
  if (seq) {
    const bool more = s->active && check_id + 1 < s->seq_limit && *(volatile const int32_t*)err == 0;
    cudaGraphSetConditional(cond, more ? 1u : 0u);
  }
}

void launch_finalize(LatState* s, const double* partials, int nparts, int check_id, int64_t t, const Params& p,
                     double v_inf, double tol, int tol_rel, int record, cudaStream_t st, int seq_ce,
                     cudaGraphConditionalHandle cond, const int32_t* err, double* hist, int nsum) {
  if (nsum == 6)
    launch_pdl(k_finalize<6>, dim3(1), dim3(256), 0, st, s, partials, nparts, check_id, t, p.a * p.a * p.a, v_inf,
               tol, tol_rel, record, seq_ce, cond, err, hist);
  else
    launch_pdl(k_finalize<4>, dim3(1), dim3(256), 0, st, s, partials, nparts, check_id, t, p.a * p.a * p.a, v_inf,
               tol, tol_rel, record, seq_ce, cond, err, hist);
}

__global__ void k_state_reset(LatState* s, int mode, int seq_limit) {
  if (mode == 2) {
    s->post = 0;
    s->seq_limit = seq_limit;
    return;
  }
  if (mode == 1) {
    *s = LatState{};
    s->scale_seq = -1;
    s->delta_e = -1.0;
    return;
  }
  s->post = 0;
  s->seq_limit = seq_limit;
  s->has_prev = 0;
  s->active = 1;
  s->converged = 0;
  s->status = STATUS_OK;
  s->checks = 0;
  s->scale_seq = -1;
  s->step = 0;
  s->delta_e = -1.0;
}
void launch_state_reset(LatState* s, int mode, cudaStream_t st, int seq_limit) {
  k_state_reset<<<1, 1, 0, st>>>(s, mode, seq_limit);
}

// ------------------------------------------------------------------ renormalise + symmetry
// out(site) = sign * scale * in(source): for each masked axis the upper half
// (index above its mirror n-1-index) takes the mirrored lower-half value
// (sign -1 for A_i), the central plane of odd n is zeroed by A_i, the rest is
// scaled in place of itself (Sec. IV; renormalisation of Sec. III).
template <typename T>
__device__ __forceinline__ void parity_source(int& x, int& y, int& z, int n, int mask, double& sign, bool& zero) {
  int* cs[3] = {&x, &y, &z};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    int mode = (mask >> (2 * ax)) & 3;
    if (mode == 0) continue;
    int m = *cs[ax], mm = n - 1 - m;
    if (m > mm) {
      *cs[ax] = mm;
      if (mode == 2) sign = -sign;
    } else if (m == mm && mode == 2) {
      zero = true;
    }
  }
}

// psi_out = P(scale psi_in) (Secs. III, IV), one site per thread on an
// (x, y, z) grid of 32 x 8 blocks; with s given, only if this check's factor
// was posted (s->scale_seq == check_id).
template <typename T>
__global__ void __launch_bounds__(256) k_scale_parity(const T* __restrict__ in, T* __restrict__ out, int n, int mask,
                                                      const LatState* __restrict__ s, int check_id, int out_idx,
                                                      LatState* sw) {
  pdl_wait();
  pdl_trigger();
  using S = typename ScaleT<T>::S;
  S scale = S(1);
  if (s) {
    if (check_id < 0 ? s->post != 1 : s->scale_seq != check_id) return;
    scale = (S)s->scale;
  }
  const int x0 = blockIdx.x * 32 + threadIdx.x, y0 = blockIdx.y * 8 + threadIdx.y, z0 = blockIdx.z;
  if (sw && (x0 | y0 | z0) == 0) sw->cur = out_idx;
  if (x0 >= n || y0 >= n) return;
  int x = x0, y = y0, z = z0;
  double sign = 1.0;
  bool zero = false;
  if (mask) parity_source<T>(x, y, z, n, mask, sign, zero);
  const S v = (S)Store<T>::to(in[site_index(x, y, z, n)]);
  out[site_index(x0, y0, z0, n)] = Store<T>::from(scale_site(v, scale, sign < 0.0, zero));
}

// FP32, n % 4 == 0: one float4 per thread (x over float4 columns).  The
// mirror of an aligned float4 along x is the aligned float4 ending at
// n-1-4i, read reversed; each site gets exactly the expression of
// k_scale_parity, so the two agree bit for bit.
__global__ void __launch_bounds__(256) k_scale_parity_f4(const float* __restrict__ in, float* __restrict__ out, int n,
                                                         int mask, const LatState* __restrict__ s, int check_id,
                                                         int out_idx, LatState* sw) {
  pdl_wait();
  pdl_trigger();
  float scale = 1.0f;
  if (s) {
    if (check_id < 0 ? s->post != 1 : s->scale_seq != check_id) return;
    scale = (float)s->scale;
  }
  const int x4 = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
  if (sw && (x4 | y | z) == 0) sw->cur = out_idx;
  if (x4 >= (n >> 2) || y >= n) return;
  scale_parity_f4_at(in, out, n, mask, scale, x4, y, z);
}

static int grid_for(size_t total, int threads) {
  size_t b = (total + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

template <typename T>
void launch_scale_parity(const T* in, T* out, int n, int mask, const LatState* s, int check_id, int out_idx,
                         LatState* s_w, cudaStream_t st) {
  if constexpr (std::is_same_v<T, float>) {
    if (n % 4 == 0) {
      launch_pdl(k_scale_parity_f4, dim3((n / 4 + 31) / 32, (n + 7) / 8, n), dim3(32, 8), 0, st, in, out, n, mask, s,
                 check_id, out_idx, s_w);
      return;
    }
  }
  launch_pdl(k_scale_parity<T>, dim3((n + 31) / 32, (n + 7) / 8, n), dim3(32, 8), 0, st, in, out, n, mask, s, check_id,
             out_idx, s_w);
}
template void launch_scale_parity<double>(const double*, double*, int, int, const LatState*, int, int, LatState*,
                                          cudaStream_t);
template void launch_scale_parity<float>(const float*, float*, int, int, const LatState*, int, int, LatState*,
                                         cudaStream_t);
template void launch_scale_parity<__nv_bfloat16>(const __nv_bfloat16*, __nv_bfloat16*, int, int, const LatState*,
                                                 int, int, LatState*, cudaStream_t);

// ------------------------------------------------------------------ random start
template <typename T>
__global__ void k_init_random(T* __restrict__ out, int n, uint64_t seed, uint64_t lat, int dist) {
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
    if constexpr (sizeof(T) == 8)
      out[i] = val;
    else
      out[i] = Store<T>::from((float)val);
  }
}
template <typename T>
void launch_init_random(T* out, int n, uint64_t seed, uint64_t lat, int dist, cudaStream_t st) {
  size_t total = (size_t)n * n * n;
  k_init_random<T><<<grid_for(total, 256), 256, 0, st>>>(out, n, seed, lat, dist);
}
template void launch_init_random<double>(double*, int, uint64_t, uint64_t, int, cudaStream_t);
template void launch_init_random<float>(float*, int, uint64_t, uint64_t, int, cudaStream_t);
template void launch_init_random<__nv_bfloat16>(__nv_bfloat16*, int, uint64_t, uint64_t, int, cudaStream_t);

// ------------------------------------------------------------------ multi-resolution transfer
// Fine site x (0-based) of a 2 nc lattice lies at coarse index position
// x/2 - 1/4 (0-based, cell-centred boxes of equal length): between coarse
// sites x/2 - 1 (weight 1/4) and x/2 (3/4) for even x, (x-1)/2 (3/4) and
// (x+1)/2 (1/4) for odd x; coarse sites outside the box hold 0.
__device__ __forceinline__ void interp_axis(int x, int& lo, double& wlo, double& whi) {
  if (x & 1) {
    lo = (x - 1) >> 1;
    wlo = 0.75;
    whi = 0.25;
  } else {
    lo = (x >> 1) - 1;
    wlo = 0.25;
    whi = 0.75;
  }
}

// One fine site per thread on an (x, y, z) grid.  With an FP64 side the
// eight weighted coarse values are summed in FP64; FP32 / BF16 lattices
// interpolate separably in FP32 (x, then y, then z): the weights 1/4 and 3/4
// are exact, so the result differs from the FP64 sum only by the rounding of
// the seven FP32 operations.
template <typename Ti, typename To>
__global__ void k_upsample(const Ti* __restrict__ in, int nc, To* __restrict__ out, int periodic) {
  const int nf = 2 * nc;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= nf) return;
  const size_t i = ((size_t)z * nf + y) * nf + x;
  int lx, ly, lz;
  double wx[2], wy[2], wz[2];
  interp_axis(x, lx, wx[0], wx[1]);
  interp_axis(y, ly, wy[0], wy[1]);
  interp_axis(z, lz, wz[0], wz[1]);
  auto at = [&](int dx, int dy, int dz) {
    int cx = lx + dx, cy = ly + dy, cz = lz + dz;
    if (periodic) {  // coarse index -1 is nc-1 and nc is 0
      cx = cx < 0 ? cx + nc : (cx >= nc ? cx - nc : cx);
      cy = cy < 0 ? cy + nc : (cy >= nc ? cy - nc : cy);
      cz = cz < 0 ? cz + nc : (cz >= nc ? cz - nc : cz);
    }
    return ((unsigned)cx < (unsigned)nc && (unsigned)cy < (unsigned)nc && (unsigned)cz < (unsigned)nc)
               ? in[site_index(cx, cy, cz, nc)]
               : Store<Ti>::from(0.0f);
  };
  if constexpr (sizeof(Ti) == 8 || sizeof(To) == 8) {
    double acc = 0.0;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) acc += (wx[dx] * wy[dy] * wz[dz]) * (double)Store<Ti>::to(at(dx, dy, dz));
    if constexpr (sizeof(To) == 8)
      out[i] = acc;
    else
      out[i] = Store<To>::from((float)acc);
  } else {
    const float fx0 = (float)wx[0], fx1 = (float)wx[1], fy0 = (float)wy[0], fy1 = (float)wy[1];
    float row[2][2];
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        row[dz][dy] = __fadd_rn(__fmul_rn(fx0, Store<Ti>::to(at(0, dy, dz))), __fmul_rn(fx1, Store<Ti>::to(at(1, dy, dz))));
    const float p0 = __fadd_rn(__fmul_rn(fy0, row[0][0]), __fmul_rn(fy1, row[0][1]));
    const float p1 = __fadd_rn(__fmul_rn(fy0, row[1][0]), __fmul_rn(fy1, row[1][1]));
    out[i] = Store<To>::from(__fadd_rn(__fmul_rn((float)wz[0], p0), __fmul_rn((float)wz[1], p1)));
  }
}
template <typename Ti, typename To>
void launch_upsample(const Ti* in, int nc, To* out, int periodic, cudaStream_t st) {
  const int nf = 2 * nc;
  dim3 grid((nf + 127) / 128, nf, nf);
  k_upsample<Ti, To><<<grid, 128, 0, st>>>(in, nc, out, periodic);
}
#define INST_UP(Ti, To) template void launch_upsample<Ti, To>(const Ti*, int, To*, int, cudaStream_t);
INST_UP(double, double)
INST_UP(double, float)
INST_UP(double, __nv_bfloat16)
INST_UP(float, double)
INST_UP(float, float)
INST_UP(float, __nv_bfloat16)
INST_UP(__nv_bfloat16, double)
INST_UP(__nv_bfloat16, float)
INST_UP(__nv_bfloat16, __nv_bfloat16)

// ------------------------------------------------------------------ snapshot algebra
constexpr int kDotBlocks = 152 * 8;

template <typename T>
__global__ void __launch_bounds__(256) k_dot2(const T* __restrict__ phi, const T* __restrict__ psi, size_t count,
                                              double* __restrict__ partials) {
  double a = 0.0, b = 0.0;
  if constexpr (sizeof(T) == 8) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
      const double f = phi[i];
      a += f * (double)psi[i];
      b += f * f;
    }
  } else {
    Kahan ka, kb;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
      const float f = Store<T>::to(phi[i]);
      ka.add(f * Store<T>::to(psi[i]));
      kb.add(f * f);
    }
    a = ka.value();
    b = kb.value();
  }
  __shared__ double red[8][2];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, off);
    b += __shfl_down_sync(0xffffffffu, b, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = a;
    red[threadIdx.x >> 5][1] = b;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
    partials[2 * blockIdx.x + threadIdx.x] = s;
  }
}
template <typename T>
int launch_dot2(const T* phi, const T* psi, size_t count, double* partials, cudaStream_t st) {
  int blocks = (int)std::min<size_t>(kDotBlocks, (count + 255) / 256);
  k_dot2<T><<<blocks, 256, 0, st>>>(phi, psi, count, partials);
  return blocks;
}
template int launch_dot2<double>(const double*, const double*, size_t, double*, cudaStream_t);
template int launch_dot2<float>(const float*, const float*, size_t, double*, cudaStream_t);
template int launch_dot2<__nv_bfloat16>(const __nv_bfloat16*, const __nv_bfloat16*, size_t, double*, cudaStream_t);

// coef[0] = <phi|psi> / <phi|phi> (0 for a vanishing phi), fixed-order sum.
__global__ void k_ratio(const double* __restrict__ partials, int np, double* coef) {
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < np; ++i) {
    a += partials[2 * i];
    b += partials[2 * i + 1];
  }
  coef[0] = b > 0.0 ? a / b : 0.0;
}
void launch_ratio(const double* partials, int nparts, double* coef, cudaStream_t st) {
  k_ratio<<<1, 32, 0, st>>>(partials, nparts, coef);
}

template <typename T>
__global__ void k_axpy(T* __restrict__ psi, const T* __restrict__ phi, const double* __restrict__ coef, double sign,
                       double alpha, size_t count) {
  const double w = coef ? sign * coef[0] : alpha;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const double val = (double)Store<T>::to(psi[i]) + w * (double)Store<T>::to(phi[i]);
    if constexpr (sizeof(T) == 8)
      psi[i] = val;
    else
      psi[i] = Store<T>::from((float)val);
  }
}
template <typename T>
void launch_axpy(T* psi, const T* phi, const double* coef, double sign, double alpha, size_t count, cudaStream_t st) {
  int blocks = (int)std::min<size_t>(152 * 32, (count + 255) / 256);
  k_axpy<T><<<blocks, 256, 0, st>>>(psi, phi, coef, sign, alpha, count);
}
template void launch_axpy<double>(double*, const double*, const double*, double, double, size_t, cudaStream_t);
template void launch_axpy<float>(float*, const float*, const double*, double, double, size_t, cudaStream_t);
template void launch_axpy<__nv_bfloat16>(__nv_bfloat16*, const __nv_bfloat16*, const double*, double, double, size_t,
                                         cudaStream_t);

// ------------------------------------------------------------------ conversions
template <typename Ti, typename To>
__global__ void k_convert(const Ti* __restrict__ in, To* __restrict__ out, size_t count) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    double val = (double)Store<Ti>::to(in[i]);
    if constexpr (sizeof(To) == 8)
      out[i] = val;
    else
      out[i] = Store<To>::from((float)val);
  }
}
template <typename Ti, typename To>
void launch_convert(const Ti* in, To* out, size_t count, cudaStream_t st) {
  k_convert<Ti, To><<<grid_for(count, 256), 256, 0, st>>>(in, out, count);
}
#define INST_CV(Ti, To) template void launch_convert<Ti, To>(const Ti*, To*, size_t, cudaStream_t);
INST_CV(double, double)
INST_CV(double, float)
INST_CV(double, __nv_bfloat16)
INST_CV(float, double)
INST_CV(float, float)
INST_CV(float, __nv_bfloat16)
INST_CV(__nv_bfloat16, double)
INST_CV(__nv_bfloat16, float)

// ------------------------------------------------------------------ potential
template <typename Ti>
__global__ void k_set_potential(const Ti* __restrict__ in, size_t count, size_t offset, float* vf, double* vd,
                                double* coefA, double* coefCB, double half_dtau, double c, int32_t* flags) {
  int bad = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    double v = (double)in[i];
    size_t o = offset + i;
    if (!isfinite(v)) bad |= 1;
    double onep = 1.0 + half_dtau * v;
    if (!(onep > 0.0)) bad |= 2;
    if (vd) {
      vd[o] = v;
      coefA[o] = (1.0 - half_dtau * v) / onep;
      coefCB[o] = c / onep;
    } else {
      float vv = (float)v;
      vf[o] = vv;
      if (!(1.0f + (float)half_dtau * vv > 0.0f)) bad |= 2;
    }
  }
  if (bad) atomicOr(flags, bad);
}
template <typename Ti>
void launch_set_potential(const Ti* in, size_t count, size_t offset, float* vf, double* vd, double* coefA,
                          double* coefCB, const Params& p, int32_t* flags, cudaStream_t st) {
  k_set_potential<Ti><<<grid_for(count, 256), 256, 0, st>>>(in, count, offset, vf, vd, coefA, coefCB, 0.5 * p.dtau,
                                                           p.c, flags);
}
// The checks of k_set_potential on an FP32 potential already in place (copied
// straight from the caller's buffer): non-finite values (flag 1) and
// 1 + dtau V / 2 <= 0 in FP64 or FP32 (flag 2).
__global__ void k_guard_potential_f32(const float* __restrict__ vf, size_t count, double half_dtau, int32_t* flags) {
  int bad = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const float vv = vf[i];
    const double v = (double)vv;
    if (!isfinite(v)) bad |= 1;
    if (!(1.0 + half_dtau * v > 0.0)) bad |= 2;
    if (!(1.0f + (float)half_dtau * vv > 0.0f)) bad |= 2;
  }
  if (bad) atomicOr(flags, bad);
}
void launch_guard_potential_f32(const float* vf, size_t count, const Params& p, int32_t* flags, cudaStream_t st) {
  k_guard_potential_f32<<<grid_for(count, 256), 256, 0, st>>>(vf, count, 0.5 * p.dtau, flags);
}

template void launch_set_potential<double>(const double*, size_t, size_t, float*, double*, double*, double*,
                                           const Params&, int32_t*, cudaStream_t);
template void launch_set_potential<float>(const float*, size_t, size_t, float*, double*, double*, double*,
                                          const Params&, int32_t*, cudaStream_t);

}  // namespace fdtd
