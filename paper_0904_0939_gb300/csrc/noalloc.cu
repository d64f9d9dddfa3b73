// fdtd_observables_noalloc: the lattice sums of a caller-held field with no
// allocation of any kind.
//
// Why it exists: some callers cannot allocate device memory at the point
// where they need the energy of a field -- code running inside a memory
// pool or arena that must not grow, callers in a process where another
// framework owns every allocation, or plug-ins that are handed raw device
// pointers and a stream but no allocator.  fdtd_create needs a workspace
// from the caller; this entry point needs none.  The per-block partial sums
// live in a file-scope __device__ array instead (kMaxBlocks x 4 doubles =
// 128 KiB, plus one error word), which every GPU that loads this library
// holds until the process exits.
//
// The array's name in host code is only a host-side stand-in, never a
// device address, so the host looks the address up with
// cudaGetSymbolAddress once per device (with that device current) and
// passes the pointer to the kernels; the first call on each device does
// that set-up, so it should come before any stream capture on that device.
//
// All calls share the one array.  Every partial is written by the sums
// kernel of the same call before the finishing kernel reads it; the one word
// that must start at zero -- the flag a bounded wait sets if it expires --
// is cleared by each call before its kernels run.  Two calls whose kernels
// overlap on the GPU (for example on two streams) race on the array and may
// return wrong sums.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "common.cuh"
#include "fdtd.h"
#include "kernels.cuh"

namespace fdtd {
void set_detached_error(const std::string& msg);
}

namespace {

constexpr int kMaxBlocks = 4096;  // block partials of the sums for n <= 1024
constexpr int kMaxN = 1024;
constexpr int kMaxDevices = 128;

// block partials, then (at kMaxBlocks * 4) the error word and the wait budget of the bounded waits
__device__ __align__(256) double g_noalloc_partials[kMaxBlocks * 4 + 32];

std::mutex g_mu;
double* g_partials_addr[kMaxDevices] = {};

// Same deterministic reduction as the check finaliser: strided per-thread
// sums in a fixed order, then a fixed tree.
__global__ void __launch_bounds__(256) k_noalloc_finish(const double* __restrict__ parts, int np, double a3,
                                                        const int32_t* __restrict__ err, double* __restrict__ out) {
  __shared__ double sm[4][256];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < np; i += 256)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += parts[(size_t)i * 4 + q];
#pragma unroll
  for (int q = 0; q < 4; ++q) sm[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < 4; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  double s0 = sm[0][0], sh = sm[1][0], sr = sm[2][0], sv = sm[3][0];
  if (*err != 0) s0 = sh = sr = sv = nan("");  // a bounded wait expired: report NaN
  out[0] = sh / s0;  // E
  out[1] = sr / s0;  // <r^2>
  out[2] = sv / s0;  // <V>
  out[3] = s0 * a3;  // sum psi^2 a^3
  out[4] = s0;
  out[5] = sh;
  out[6] = sr;
  out[7] = sv;
}

int fail(int code, const char* msg) {
  fdtd::set_detached_error(msg);
  return code;
}

}  // namespace

extern "C" FDTD_API int fdtd_observables_noalloc(const void* psi, const void* v, int dtype, int n, double length,
                                                 double mass, double* out, void* stream) {
  using namespace fdtd;
  if (!psi || !v || !out) return fail(FDTD_ERR_INVALID_ARG, "observables_noalloc: null pointer");
  if (dtype != FDTD_F64 && dtype != FDTD_F32)
    return fail(FDTD_ERR_INVALID_ARG, "observables_noalloc: dtype must be FDTD_F64 or FDTD_F32");
  if (!(length > 0.0) || !std::isfinite(length) || !(mass > 0.0) || !std::isfinite(mass))
    return fail(FDTD_ERR_INVALID_ARG, "observables_noalloc: length and mass must be positive and finite");
  if (n < 1 || n > kMaxN)
    return fail(FDTD_ERR_SHAPE,
                "observables_noalloc: n must be in [1, 1024]; its static scratch holds the partial sums of at "
                "most 4096 blocks (128 KiB)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fail(FDTD_ERR_CUDA, "observables_noalloc: no current CUDA device");
  }
  double* parts = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_partials_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(FDTD_ERR_CUDA, (std::string("observables_noalloc: cudaGetSymbolAddress failed: ") +
                                    cudaGetErrorString(e)).c_str());
      }
      g_partials_addr[dev] = (double*)p;
    }
    parts = g_partials_addr[dev];
  }
  Params p{};
  p.n = n;
  p.a = length / n;
  p.mass = mass;
  p.dtau = p.a * p.a / 4.0;
  p.c = p.dtau / (2.0 * mass * p.a * p.a);
  int nb = sums_blocks(n);
  if (nb > kMaxBlocks) return fail(FDTD_ERR_SHAPE, "observables_noalloc: lattice needs more partials than the scratch holds");
  cudaStream_t st = (cudaStream_t)stream;
  // FP32 lattices with n % 4 == 0 take the same TMA-fed sums as
  // fdtd_observables (tensor maps are encoded on the host stack; nothing is
  // allocated), so the two agree bit for bit; other cases take the plain
  // sums kernel, as fdtd_observables does.
  CUtensorMap mpsi, mv;
  int bw = 0, bh = 0;
  tma_box(1, 64, &bw, &bh);
  const bool tma = dtype == FDTD_F32 && tma_supported(n, FDTD_F32) && tma_sums_blocks(n) <= kMaxBlocks &&
                   encode_field_map(&mpsi, (const float*)psi, n, bw, bh) == 0 &&
                   encode_field_map(&mv, (const float*)v, n, bw, bh) == 0;
  int32_t* err = (int32_t*)(parts + (size_t)kMaxBlocks * 4);  // error flag, then the wait budget (0 = default)
  cudaMemsetAsync(err, 0, 2 * sizeof(int32_t), st);
  if (tma)
    nb = launch_sums_tma(mpsi, mv, p, parts, nullptr, err, st);
  else if (dtype == FDTD_F64)
    nb = launch_sums<double>((const double*)psi, v, p, parts, nullptr, st);
  else
    nb = launch_sums<float>((const float*)psi, v, p, parts, nullptr, st);
  k_noalloc_finish<<<1, 256, 0, st>>>(parts, nb, p.a * p.a * p.a, err, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(FDTD_ERR_CUDA, (std::string("observables_noalloc: ") + cudaGetErrorString(e)).c_str());
  return FDTD_OK;
}
