// Device-side helpers shared by the FDTD kernels (sm_103a).
//
// Field layout in HBM: dense N^3, x fastest, no padding; sites outside
// [0, N) along any axis read as 0 (Dirichlet wall of Sec. III / Sec. V).
// Indices in this file are 0-based: site (x, y, z) sits at physical
// coordinate (x - (N-1)/2) a, the centred convention of Sec. VII.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fdtd {

// ---------------------------------------------------------------- storage
template <typename T> struct Store;
template <> struct Store<double> {
  using C = double;  // arithmetic type
  __device__ __forceinline__ static double ld(const double* p) { return __ldg(p); }
  __device__ __forceinline__ static double to(double v) { return v; }
  __device__ __forceinline__ static double from(double v) { return v; }
};
template <> struct Store<float> {
  using C = float;
  __device__ __forceinline__ static float ld(const float* p) { return __ldg(p); }
  __device__ __forceinline__ static float to(float v) { return v; }
  __device__ __forceinline__ static float from(float v) { return v; }
};
template <> struct Store<__nv_bfloat16> {
  using C = float;
  __device__ __forceinline__ static float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  __device__ __forceinline__ static float to(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ __forceinline__ static __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
};

// ---------------------------------------------------------------- launch overlap
// Programmatic dependent launch: a kernel launched with launch_pdl may be
// scheduled while its predecessor on the stream is still running.  Every
// such kernel calls pdl_wait() before it touches memory (it returns once the
// predecessor has completed and its writes are visible) and pdl_trigger()
// to let its own successor be scheduled early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------- renormalisation
// One site of psi <- P(s psi) (Secs. III, IV): FP64 lattices multiply in
// FP64; FP32 / BF16 lattices multiply the FP32 value by s rounded to FP32
// (ScaleT), so every kernel that renormalises an FP32 lattice rounds alike.
template <typename T>
struct ScaleT {
  using S = float;
};
template <>
struct ScaleT<double> {
  using S = double;
};
__device__ __forceinline__ float scale_site(float v, float s, bool neg, bool zero) {
  const float r = __fmul_rn(v, s);
  return zero ? 0.0f : (neg ? -r : r);
}
__device__ __forceinline__ double scale_site(double v, double s, bool neg, bool zero) {
  const double r = __dmul_rn(v, s);
  return zero ? 0.0 : (neg ? -r : r);
}

// ---------------------------------------------------------------- coefficients
// Eq. updateeq with h = dtau V / 2:
//   psi' = A psi + (B dtau / 2m) sum_i (D . PsiHat)_i,
//   A = (1 - h)/(1 + h),  B = 1/(1 + h),  D = [1, -2, 1] / a^2.
// With c = dtau / (2 m a^2) and S = sum of the 6 neighbours this is
//   psi' = B [ (1 - h - 6c) psi + c S ],
// the form the FP32 kernels evaluate (one reciprocal per site, the rest
// FMAs).  The neighbour sum is always taken as ((xm + xp) + (ym + yp)) +
// (zm + zp): commutative pairs keep an odd/even field exactly odd/even.
// B uses the hardware reciprocal approximation (rcp.approx, max 1 ulp): every
// FP32 kernel (single step, temporally blocked, adjoint) takes B from this
// one function, so they agree bit for bit.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
struct CoefF {
  float b;      // 1 / (1 + h)
  float alpha;  // 1 - h - 6c
};
// Every operation rounds on its own (no contraction), so kernels that
// evaluate the update with packed two-lane instructions (k_step_tma) agree
// with the one-site kernels bit for bit.
__device__ __forceinline__ CoefF coef_f32(float v, float half_dtau, float one_minus_6c) {
  const float h = __fmul_rn(half_dtau, v);
  CoefF k;
  k.b = rcp_approx(__fadd_rn(1.0f, h));
  k.alpha = __fsub_rn(one_minus_6c, h);
  return k;
}
__device__ __forceinline__ float nbr_sum(float xm, float xp, float ym, float yp, float zm, float zp) {
  return __fadd_rn(__fadd_rn(__fadd_rn(xm, xp), __fadd_rn(ym, yp)), __fadd_rn(zm, zp));
}
__device__ __forceinline__ float update_f32(float c, float s, CoefF k, float cc) {
  return __fmul_rn(k.b, __fmaf_rn(cc, s, __fmul_rn(k.alpha, c)));
}

// FP64 ("plain") form: the per-site A and c B are precomputed once from V
// and stored, psi' = A psi + cB (S - 6 psi).
__device__ __forceinline__ double nbr_sum(double xm, double xp, double ym, double yp, double zm, double zp) {
  return __dadd_rn(__dadd_rn(__dadd_rn(xm, xp), __dadd_rn(ym, yp)), __dadd_rn(zm, zp));
}
__device__ __forceinline__ double update_f64(double c, double s, double A, double cB) {
  return __fma_rn(cB, __fma_rn(-6.0, c, s), __dmul_rn(A, c));
}

// ---------------------------------------------------------------- geometry
__device__ __forceinline__ float coord_f32(int i, int n, float a) { return ((float)i - 0.5f * (float)(n - 1)) * a; }
__device__ __forceinline__ double coord_f64(int i, int n, double a) { return ((double)i - 0.5 * (double)(n - 1)) * a; }

// ---------------------------------------------------------------- RNG
// SplitMix64 (Steele, Lea & Flood 2014): output d of the stream seeded with
// s is fin(s + (d + 1) * 0x9E3779B97F4A7C15), fin = the 30/27/31 xor-shift
// multiply finaliser.  Lattice `lat` owns draws lat * 2^42 .. (lat+1) * 2^42 - 1.
__device__ __forceinline__ uint64_t sm64(uint64_t seed, uint64_t d) {
  uint64_t z = seed + (d + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double unit_interval(uint64_t bits) {
  return (double)(bits >> 11) * 0x1.0p-53;  // [0, 1)
}

// ---------------------------------------------------------------- misc
__device__ __forceinline__ size_t site_index(int x, int y, int z, int n) {
  return ((size_t)z * (size_t)n + (size_t)y) * (size_t)n + (size_t)x;
}

// Kahan-compensated FP32 accumulator (Kahan 1965): sum - comp carries the
// running total to ~2^-48 relative, enough to hand over to FP64.
// out = scale * P(in) on the float4 of sites 4 x4 .. 4 x4 + 3 of row (y, z)
// of an n^3 FP32 field with n % 4 == 0; P the symmetry operators of the mask
// (Sec. IV).  The mirror of an aligned float4 along x is the aligned float4
// ending at n - 1 - 4 x4, read reversed; each site gets scale_site, the
// expression of the one-site renormalisation, so every caller agrees bit
// for bit.
__device__ __forceinline__ void scale_parity_f4_at(const float* __restrict__ in, float* __restrict__ out, int n,
                                                   int mask, float scale, int x4, int y, int z) {
  const int mx = mask & 3, my = (mask >> 2) & 3, mz = (mask >> 4) & 3;
  int ys = y, zs = z;
  bool neg = false, zero = false;
  if (my) {
    const int mm = n - 1 - y;
    if (y > mm) {
      ys = mm;
      neg ^= (my == 2);
    } else if (y == mm && my == 2) {
      zero = true;
    }
  }
  if (mz) {
    const int mm = n - 1 - z;
    if (z > mm) {
      zs = mm;
      neg ^= (mz == 2);
    } else if (z == mm && mz == 2) {
      zero = true;
    }
  }
  const float* row = in + ((size_t)zs * n + ys) * n;
  const float4 a = *reinterpret_cast<const float4*>(row + 4 * x4);
  float av[4] = {a.x, a.y, a.z, a.w}, mv[4] = {0.f, 0.f, 0.f, 0.f};
  if (mx) {
    const float4 b = *reinterpret_cast<const float4*>(row + (n - 4 - 4 * x4));
    mv[0] = b.w;  // mirror of site 4 x4 + 0 is n - 1 - 4 x4
    mv[1] = b.z;
    mv[2] = b.y;
    mv[3] = b.x;
  }
  float o[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int x = 4 * x4 + c, mm = n - 1 - x;
    bool ng = neg, zc = zero;
    float src = av[c];
    if (mx) {
      if (x > mm) {
        src = mv[c];
        ng ^= (mx == 2);
      } else if (x == mm && mx == 2) {
        zc = true;
      }
    }
    o[c] = scale_site(src, scale, ng, zc);
  }
  *reinterpret_cast<float4*>(out + ((size_t)z * n + y) * n + 4 * x4) = make_float4(o[0], o[1], o[2], o[3]);
}

struct Kahan {
  float sum = 0.f, comp = 0.f;
  __device__ __forceinline__ void add(float v) {
    float y = __fsub_rn(v, comp);
    float t = __fadd_rn(sum, y);
    comp = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
  }
  __device__ __forceinline__ double value() const { return (double)sum - (double)comp; }
};

}  // namespace fdtd
