// Temporally blocked FP32 update (Eq. updateeq applied K times per HBM pass)
// with TMA-fed plane streaming, for lattices with n % 4 == 0.
//
// A block owns an output tile of TX x TY sites in x-y and a chunk of ZC
// z-planes.  It streams the input planes of a (TX + 2 HX) x (TY + 2K) box
// -- psi and V -- through a ring of R shared-memory slots with
// cp.async.bulk.tensor (one thread issues, an mbarrier per slot counts the
// bytes); sites outside the lattice arrive as zeros, which is the Dirichlet
// wall of Sec. III.  Each thread owns one float4 column of the box and walks
// z: level 1 (the first update) reads psi from the ring; level l > 1 keeps
// the three z-planes of level l-1 of its column in registers and reads the
// x/y neighbours of level l-1 from a double-buffered shared plane.  Level l
// trails level l-1 by one plane, so one barrier per z-step orders
// everything.  Level K writes the tile interior to HBM.  Algorithmic HBM
// traffic per launch: psi in + psi out + V in, 12 B per site for K steps.
//
// The per-site arithmetic is exactly that of k_step_f32 (same neighbour
// order, same coefficient function), so K fused steps reproduce K single
// steps bit for bit.  Outer box sites compute garbage at levels < K (their
// own neighbours are missing); the garbage moves inward one site per level
// and the x margin HX >= K and y margin K keep it out of the output.
//
// Every wait on an mbarrier is bounded; on expiry the block records
// FDTD timeout in *err, waits (bounded) for its own copies in flight and
// leaves -- all threads together, after a block-wide vote.
#include <cuda.h>

#include "common.cuh"
#include "kernels.cuh"

namespace fdtd {

namespace tb {

constexpr int TX = 128;  // interior tile width (sites)
constexpr int TY = 16;   // interior tile height
constexpr int HX = 4;    // x margin of the box: >= K and a multiple of 4 (TMA: x * 4 B % 16 == 0)
constexpr int BW = TX + 2 * HX;
constexpr int C4 = BW / 4;  // float4 columns per box row
constexpr int D = 2;        // planes prefetched beyond the newest one in use
constexpr int LW = BW + 8;  // level-plane row pitch: 4-float guards on both sides
constexpr unsigned long long kWaitLimitNs = 200ull * 1000 * 1000;  // 0.2 s per wait

template <int K>
struct Geo {
  static constexpr int BH = TY + 2 * K;
  static constexpr int USED = C4 * BH;                      // threads that own a box column
  static constexpr int THREADS = (USED + 31) / 32 * 32;     // whole warps
  static constexpr int R = D + 2 + (K > 1 ? K - 1 : 1);     // ring slots
  static constexpr int PLANE = ((BW * BH * 4 + 127) / 128) * 128 / 4;  // floats per ring box, 128 B multiple
  static constexpr int LPLANE = LW * BH;
  static constexpr size_t RING_OFF = 128;                   // guard before the ring
  static constexpr size_t SLOT_BYTES = 2 * (size_t)PLANE * 4;
  static constexpr unsigned TX_BYTES = 2u * BW * BH * 4;    // bytes the two box loads of a plane deliver
  static constexpr size_t LEVEL_OFF = RING_OFF + R * SLOT_BYTES + 128;
  static constexpr size_t BAR_OFF = LEVEL_OFF + (size_t)(K > 1 ? K - 1 : 0) * 2 * LPLANE * 4;
  static constexpr size_t SMEM = BAR_OFF + 8 * R + 128;     // + room to align the base to 128 B
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Wait bounded in wall-clock time (kWaitLimitNs); gives up early when any
// block has already reported an expired wait in *err.  Returns false if
// it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, const int32_t* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0) {
      if (*(volatile const int32_t*)err != 0) return false;
      if (global_ns() - t0 > kWaitLimitNs) return false;
    }
  }
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// slot of plane j + d given the slot sj of plane j, for -R < d < R
template <int R>
__device__ __forceinline__ int slot_add(int sj, int d) {
  int s = sj + d;
  s -= (s >= R) ? R : 0;
  s += (s < 0) ? R : 0;
  return s;
}

template <int K>
__device__ __forceinline__ void issue_plane(char* smem, const CUtensorMap* mpsi, const CUtensorMap* mv, int q, int s,
                                            int x0, int y0) {
  using G = Geo<K>;
  float* box = (float*)(smem + G::RING_OFF + s * G::SLOT_BYTES);
  uint64_t* bar = (uint64_t*)(smem + G::BAR_OFF) + s;
  mbar_expect_tx(bar, G::TX_BYTES);
  tma_load_3d(box, mpsi, x0 - HX, y0 - K, q, bar);
  tma_load_3d(box + G::PLANE, mv, x0 - HX, y0 - K, q, bar);
}

__device__ __forceinline__ float4 f4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// One float4 of site updates: c at x..x+3, xl = site x-1, xr = site x+4.
__device__ __forceinline__ float4 update4(float4 c, float xl, float xr, float4 ym, float4 yp, float4 zm, float4 zp,
                                          float4 v, float hd, float om6c, float cc) {
  float4 o;
  o.x = update_f32(c.x, nbr_sum(xl, c.y, ym.x, yp.x, zm.x, zp.x), coef_f32(v.x, hd, om6c), cc);
  o.y = update_f32(c.y, nbr_sum(c.x, c.z, ym.y, yp.y, zm.y, zp.y), coef_f32(v.y, hd, om6c), cc);
  o.z = update_f32(c.z, nbr_sum(c.y, c.w, ym.z, yp.z, zm.z, zp.z), coef_f32(v.z, hd, om6c), cc);
  o.w = update_f32(c.w, nbr_sum(c.z, xr, ym.w, yp.w, zm.w, zp.w), coef_f32(v.w, hd, om6c), cc);
  return o;
}

template <int K>
__global__ void __launch_bounds__(Geo<K>::THREADS) k_step_tma(const __grid_constant__ CUtensorMap map_psi,
                                                               const __grid_constant__ CUtensorMap map_v,
                                                               float* __restrict__ out, int n, int zc,
                                                               float half_dtau, float one_m6c, float cc,
                                                               const int32_t* __restrict__ active,
                                                               int32_t* __restrict__ err) {
  using G = Geo<K>;
  constexpr int R = G::R;
  if (active && *active == 0) return;
  if (*(volatile const int32_t*)err != 0) return;  // an earlier wait expired: do nothing
  extern __shared__ __align__(128) char smem_raw[];
  // TMA destinations need 128-byte aligned shared addresses
  char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const bool owner = tid < G::USED;          // threads beyond the box only join barriers and shuffles
  const int row = owner ? tid / C4 : 0, col = owner ? tid % C4 : 0;  // box row, float4 column
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, n);
  const int xg = x0 - HX + 4 * col;  // lattice x of this thread's first site
  const int yg = y0 - K + row;
  const bool inside = owner && (xg >= 0) && (xg < n) && (yg >= 0) && (yg < n);
  const bool interior_col = (col >= HX / 4) && (col < HX / 4 + TX / 4);
  const bool interior_row = owner && (row >= K) && (row < K + TY);
  // x-neighbours come from the adjacent lanes; only lanes 0 and 31 read them
  // from shared memory (row ends take the neighbouring row's value, which
  // only ever reaches margin sites)
  const bool fix_l = owner && lane == 0 && col > 0;
  const bool fix_r = owner && lane == 31 && col < C4 - 1;
  const int j0 = z0 - K + 1, j1 = z1 + K - 2;
  uint64_t* bars = (uint64_t*)(smem + G::BAR_OFF);
  float* ring = (float*)(smem + G::RING_OFF);
  float* lev = (float*)(smem + G::LEVEL_OFF);
  const int ro = row * BW + 4 * col;        // offset of this column in a ring box
  const int lo = row * LW + 4 + 4 * col;    // offset of this column in a level plane
  float* const out_col = out + (size_t)yg * n + xg;

  // zero the level planes (guards included) and set up the barriers
  for (int i = tid; i < (K > 1 ? (K - 1) * 2 * G::LPLANE : 0); i += G::THREADS) lev[i] = 0.f;
  if (tid == 0) {
    for (int s = 0; s < R; ++s) mbar_init(bars + s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // planes j0-1 .. j0+D go to consecutive slots starting at slot 0
  const int sj0 = 1;  // slot of plane j0
  unsigned outstanding = 0;  // (thread 0) slots with a copy issued and not yet waited for
  if (tid == 0) {
    int s = 0;
    for (int q = j0 - 1; q <= min(j0 + D, j1 + 1); ++q, s = slot_add<R>(s, 1)) {
      issue_plane<K>(smem, &map_psi, &map_v, q, s, x0, y0);
      outstanding |= 1u << s;
    }
  }
  unsigned phase = 0;  // bit s: parity of the next wait on slot s (toggled on success only)
  int timeout = 0;
  auto wait_slot = [&](int s) {
    if (mbar_wait_bounded(bars + s, (phase >> s) & 1u, err)) {
      phase ^= 1u << s;
      outstanding &= ~(1u << s);
    } else {
      timeout = 1;
    }
  };
  wait_slot(0);
  wait_slot(1);

  // register windows of levels 1..K-1: planes (p-1, p, p+1) of this column
  constexpr int NW = K > 1 ? K - 1 : 1;
  float4 wm[NW], wc[NW], wp[NW];
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int l = 0; l < NW; ++l) {
    wm[l] = zero4;
    wc[l] = zero4;
    wp[l] = zero4;
  }

  int sj = sj0;  // slot of plane j
  for (int j = j0; j <= j1; ++j) {
    if (tid == 0 && j + 1 + D <= j1 + 1) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const int s = slot_add<R>(sj, 1 + D);
      issue_plane<K>(smem, &map_psi, &map_v, j + 1 + D, s, x0, y0);
      outstanding |= 1u << s;
    }
    wait_slot(slot_add<R>(sj, 1));

    // ---- level 1: plane j from the ring
    {
      const float* b0 = ring + sj * (G::SLOT_BYTES / 4);
      const float* bm = ring + slot_add<R>(sj, -1) * (G::SLOT_BYTES / 4);
      const float* bp = ring + slot_add<R>(sj, 1) * (G::SLOT_BYTES / 4);
      const int p = j;
      const bool need = owner && (row >= 1 && row < G::BH - 1) && (K > 1 || interior_col);
      float4 c = owner ? f4(b0 + ro) : zero4;
      float xl = __shfl_up_sync(0xffffffffu, c.w, 1);
      float xr = __shfl_down_sync(0xffffffffu, c.x, 1);
      if (fix_l) xl = b0[ro - 1];
      if (fix_r) xr = b0[ro + 4];
      if (need) {
        float4 r = update4(c, xl, xr, f4(b0 + ro - BW), f4(b0 + ro + BW), f4(bm + ro), f4(bp + ro),
                           f4(b0 + G::PLANE + ro), half_dtau, one_m6c, cc);
        if (!inside || p < 0 || p >= n) r = zero4;
        if constexpr (K == 1) {
          if (interior_row && inside && p >= z0 && p < z1)
            *reinterpret_cast<float4*>(out_col + (size_t)p * n * n) = r;
        } else {
          *reinterpret_cast<float4*>(lev + (p & 1) * G::LPLANE + lo) = r;
          wm[0] = wc[0];
          wc[0] = wp[0];
          wp[0] = r;
        }
      }
    }
    // ---- levels 2..K: plane j - l + 1 from level l-1
#pragma unroll
    for (int l = 2; l <= K; ++l) {
      const int p = j - l + 1;
      const bool need = owner && (row >= l && row < G::BH - l) && (l < K || interior_col);
      const float* lp = lev + ((l - 2) * 2 + (p & 1)) * G::LPLANE;  // level l-1, plane p
      const float4 c = wc[l - 2];
      float xl = __shfl_up_sync(0xffffffffu, c.w, 1);
      float xr = __shfl_down_sync(0xffffffffu, c.x, 1);
      if (fix_l) xl = lp[lo - 1];
      if (fix_r) xr = lp[lo + 4];
      if (need) {
        const float4 v = f4(ring + slot_add<R>(sj, 1 - l) * (G::SLOT_BYTES / 4) + G::PLANE + ro);
        float4 r = update4(c, xl, xr, f4(lp + lo - LW), f4(lp + lo + LW), wm[l - 2], wp[l - 2], v, half_dtau,
                           one_m6c, cc);
        if (!inside || p < 0 || p >= n) r = zero4;
        if (l == K) {
          if (interior_row && inside && p >= z0 && p < z1)
            *reinterpret_cast<float4*>(out_col + (size_t)p * n * n) = r;
        } else {
          *reinterpret_cast<float4*>(lev + ((l - 1) * 2 + (p & 1)) * G::LPLANE + lo) = r;
          wm[l - 1] = wc[l - 1];
          wc[l - 1] = wp[l - 1];
          wp[l - 1] = r;
        }
      }
    }
    if (__syncthreads_or(timeout)) {
      if (tid == 0) {
        atomicOr(err, 1);
        // the copies still in flight target this block's shared memory:
        // wait for them (each wait bounded in time) before leaving
        for (int s = 0; s < R; ++s) {
          if (!(outstanding & (1u << s))) continue;
          const unsigned long long t0 = global_ns();
          while (!mbar_try_wait(bars + s, (phase >> s) & 1u) && global_ns() - t0 < kWaitLimitNs) {
          }
        }
      }
      return;
    }
    sj = slot_add<R>(sj, 1);
  }
}

template <int K>
void launch_k(const CUtensorMap& mpsi, const CUtensorMap& mv, float* out, const Params& p, int zc,
              const int32_t* active, int32_t* err, cudaStream_t st) {
  using G = Geo<K>;
  static unsigned long long attr_set = 0;  // one bit per device ordinal
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 64 || !(attr_set & (1ull << dev))) {
    cudaFuncSetAttribute(k_step_tma<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    if (dev < 64) attr_set |= 1ull << dev;
  }
  dim3 grid((p.n + TX - 1) / TX, (p.n + TY - 1) / TY, (p.n + zc - 1) / zc);
  k_step_tma<K><<<grid, G::THREADS, G::SMEM, st>>>(mpsi, mv, out, p.n, zc, p.half_dtau_f, p.one_m6c_f, p.c_f,
                                                    active, err);
}

}  // namespace tb

int blocked_max_depth() { return 3; }

bool tma_supported(int n, int precision) { return precision == FDTD_F32 && n % 4 == 0 && n >= 8; }

int auto_depth(int n, int precision) {
  if (!tma_supported(n, precision)) return 1;
  return n >= 96 ? 3 : 2;
}

int tma_zchunk(int n, int depth) {
  // enough blocks for several waves over the 152 SMs, chunks not much
  // shorter than the 2(K-1) planes of warm-up they repeat
  int tiles = ((n + tb::TX - 1) / tb::TX) * ((n + tb::TY - 1) / tb::TY);
  int zc = n;
  while (zc > 16 * depth && (long long)tiles * ((n + zc - 1) / zc) < 4 * 152) zc = (zc + 1) / 2;
  return zc;
}

size_t tma_smem_bytes(int depth) {
  return depth == 1 ? tb::Geo<1>::SMEM : depth == 2 ? tb::Geo<2>::SMEM : tb::Geo<3>::SMEM;
}

void launch_step_tma(const CUtensorMap& map_psi_in, const CUtensorMap& map_v, float* out, const Params& p,
                     int depth, int zc, const int32_t* active, int32_t* err, cudaStream_t st) {
  if (zc <= 0) zc = tma_zchunk(p.n, depth);
  if (depth == 1)
    tb::launch_k<1>(map_psi_in, map_v, out, p, zc, active, err, st);
  else if (depth == 2)
    tb::launch_k<2>(map_psi_in, map_v, out, p, zc, active, err, st);
  else
    tb::launch_k<3>(map_psi_in, map_v, out, p, zc, active, err, st);
}

// Tensor map of a dense n^3 FP32 field for the box loads above.
int encode_field_map(CUtensorMap* map, const float* base, int n, int depth) {
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
  cuuint32_t box[3] = {(cuuint32_t)tb::BW, (cuuint32_t)(tb::TY + 2 * depth), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = ((Encode)fn)(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -2;
}

}  // namespace fdtd
