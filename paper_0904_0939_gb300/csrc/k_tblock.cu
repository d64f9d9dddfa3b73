// One-lattice launches of the TMA-streamed tile pipelines (tma_item.cuh):
// the temporally blocked FP32 update (K = 1..3 steps per pass over HBM,
// tile width 64 or 128) and the fused lattice sums of Eq. energysum.
// Algorithmic HBM traffic of a stencil launch: psi in + psi out + V in,
// 12 B per site for K steps; of a sums launch: psi + V, 8 B per site.
#include <map>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "tma_item.cuh"

namespace fdtd {

namespace tb {

template <int K, int TXT>
__global__ void __launch_bounds__(Geo<K, TXT>::THREADS) k_step_tma(const __grid_constant__ CUtensorMap map_psi,
                                                                    const __grid_constant__ CUtensorMap map_v,
                                                                    float* __restrict__ out, int n, int zc,
                                                                    float half_dtau, float one_m6c, float cc,
                                                                    const int32_t* __restrict__ active,
                                                                    int32_t* __restrict__ err) {
  if (active && *active == 0) return;
  if (*(volatile const int32_t*)err != 0) return;  // an earlier wait expired: do nothing
  extern __shared__ __align__(128) char smem_raw[];
  char* smem = aligned_smem(smem_raw);
  const int z0 = blockIdx.z * zc;
  tma_step_item<K, TXT>(smem, &map_psi, &map_v, out, n, blockIdx.x * TXT, blockIdx.y * TY, z0, min(z0 + zc, n),
                        half_dtau, one_m6c, cc, err);
}

constexpr int kSumsTX = 64;

__global__ void __launch_bounds__(Geo<1, kSumsTX>::THREADS) k_sums_tma(const __grid_constant__ CUtensorMap map_psi,
                                                                       const __grid_constant__ CUtensorMap map_v,
                                                                       int n, float a, float kfac,
                                                                       double* __restrict__ partials,
                                                                       const int32_t* __restrict__ active,
                                                                       int32_t* __restrict__ err) {
  if (active && *active == 0) return;
  if (*(volatile const int32_t*)err != 0) return;
  extern __shared__ __align__(128) char smem_raw[];
  char* smem = aligned_smem(smem_raw);
  const int item = blockIdx.y * gridDim.x + blockIdx.x;
  tma_sums_item<kSumsTX>(smem, &map_psi, &map_v, n, blockIdx.x * kSumsTX, blockIdx.y * TY, 0, n, a, kfac,
                         partials + (size_t)item * 4, err);
}

// Opt each kernel in to its dynamic shared memory once per device.
std::mutex g_smem_mu;
std::map<const void*, unsigned long long> g_smem_done;  // kernel -> device bitmask

template <typename Kern>
void set_smem(Kern k, size_t bytes) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_smem_mu);
  unsigned long long& done = g_smem_done[(const void*)k];
  if (dev >= 64 || !(done & (1ull << dev))) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (dev < 64) done |= 1ull << dev;
  }
}

template <int K, int TXT>
void launch_k(const CUtensorMap& mpsi, const CUtensorMap& mv, float* out, const Params& p, int zc,
              const int32_t* active, int32_t* err, cudaStream_t st) {
  using G = Geo<K, TXT>;
  set_smem(k_step_tma<K, TXT>, G::SMEM);
  dim3 grid((p.n + TXT - 1) / TXT, (p.n + TY - 1) / TY, (p.n + zc - 1) / zc);
  k_step_tma<K, TXT><<<grid, G::THREADS, G::SMEM, st>>>(mpsi, mv, out, p.n, zc, p.half_dtau_f, p.one_m6c_f, p.c_f,
                                                         active, err);
}

}  // namespace tb

int blocked_max_depth() { return 3; }

bool tma_supported(int n, int precision) { return precision == FDTD_F32 && n % 4 == 0 && n >= 8; }

int auto_depth(int n, int precision) {
  if (!tma_supported(n, precision)) return 1;
  return n >= 96 ? 3 : 2;
}

int tma_zchunk(int n, int depth, int tx) {
  // enough blocks for several waves over the 152 SMs, chunks not much
  // shorter than the 2(K-1) planes of warm-up they repeat
  int tiles = ((n + tx - 1) / tx) * ((n + tb::TY - 1) / tb::TY);
  int zc = n;
  while (zc > 16 * depth && (long long)tiles * ((n + zc - 1) / zc) < 4 * 152) zc = (zc + 1) / 2;
  return zc;
}

void launch_step_tma(const CUtensorMap& map_psi_in, const CUtensorMap& map_v, float* out, const Params& p, int depth,
                     int tx, int zc, const int32_t* active, int32_t* err, cudaStream_t st) {
  if (zc <= 0) zc = tma_zchunk(p.n, depth, tx);
  if (tx == 64) {
    if (depth == 1)
      tb::launch_k<1, 64>(map_psi_in, map_v, out, p, zc, active, err, st);
    else if (depth == 2)
      tb::launch_k<2, 64>(map_psi_in, map_v, out, p, zc, active, err, st);
    else
      tb::launch_k<3, 64>(map_psi_in, map_v, out, p, zc, active, err, st);
  } else {
    if (depth == 1)
      tb::launch_k<1, 128>(map_psi_in, map_v, out, p, zc, active, err, st);
    else if (depth == 2)
      tb::launch_k<2, 128>(map_psi_in, map_v, out, p, zc, active, err, st);
    else
      tb::launch_k<3, 128>(map_psi_in, map_v, out, p, zc, active, err, st);
  }
}

int tma_sums_blocks(int n) { return ((n + tb::kSumsTX - 1) / tb::kSumsTX) * ((n + tb::TY - 1) / tb::TY); }

int launch_sums_tma(const CUtensorMap& map_psi, const CUtensorMap& map_v, const Params& p, double* partials,
                    const int32_t* active, int32_t* err, cudaStream_t st) {
  using G = tb::Geo<1, tb::kSumsTX>;
  tb::set_smem(tb::k_sums_tma, G::SMEM);
  dim3 grid((p.n + tb::kSumsTX - 1) / tb::kSumsTX, (p.n + tb::TY - 1) / tb::TY, 1);
  tb::k_sums_tma<<<grid, G::THREADS, G::SMEM, st>>>(map_psi, map_v, p.n, (float)p.a,
                                                     (float)(1.0 / (2.0 * p.mass * p.a * p.a)), partials, active,
                                                     err);
  return (int)(grid.x * grid.y);
}

void tma_box(int depth, int tx, int* box_w, int* box_h) {
  *box_w = tx + 2 * tb::HX;
  *box_h = tb::TY + 2 * depth;
}

// Tensor map of a dense n^3 FP32 field for box loads of box_w x box_h x 1.
int encode_field_map(CUtensorMap* map, const float* base, int n, int box_w, int box_h) {
  static void* fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      fn = nullptr;
      return -1;
    }
  }
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)n};
  cuuint64_t strides[2] = {(cuuint64_t)n * 4, (cuuint64_t)n * n * 4};
  cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = ((Encode)fn)(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -2;
}

}  // namespace fdtd
