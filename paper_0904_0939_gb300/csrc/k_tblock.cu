// One-lattice launches of the TMA-streamed tile pipelines (tma_item.cuh):
// the temporally blocked FP32 update (K = 1..3 steps per pass over HBM,
// tile width 64 or 128) and the fused lattice sums of Eq. energysum.
// Algorithmic HBM traffic of a stencil launch: psi in + psi out + V in,
// 12 B per site for K steps; of a sums launch: psi + V, 8 B per site.
#include <algorithm>
#include <map>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "tma_item.cuh"

namespace fdtd {

namespace tb {

// The tile columns (TXT x TY sites in x-y, all n planes in z) are laid end
// to end, column-major with z fastest, into ntiles * n "tile planes"; block
// b updates the `span` consecutive tile planes from b * span on, split into
// one item per column it touches.  A span that divides n is a plain z-chunk
// grid; a span of ceil(ntiles * n / resident blocks) gives every SM the
// same work in one wave whatever the lattice size.
//
// span <= 0 selects the balanced partition: every item costs its planes plus
// wcost = 2(K - 1) warm-up and drain steps, so a block whose equal span runs
// into the next column (two items) is the slowest of the wave.  Instead each
// tile column counts n + wcost cost units (the item start first), the grid
// splits the cost line into equal parts, and a cost coordinate u maps to the
// tile plane  c n + clamp(u - c (n + wcost) - wcost, 0, n),  c = u / (n + wcost):
// monotone, from 0 to ntiles * n, so the blocks' ranges cover every tile
// plane once.
//
// span == -2 selects the columns-first partition (for grids with more
// blocks than tile columns): block b < C (C = ntiles) takes planes
// [0, zsplit) of column b, and the other blocks cut the column tops
// [zsplit, n), laid end to end, into equal parts.  The first C blocks move
// through z in step, so a tile's y-neighbours are read at about the same z
// and the halo rows of its box come from L2 instead of HBM.
__device__ __forceinline__ long long balanced_plane(long long u, int n, int wcost) {
  const long long unit = n + wcost, c = u / unit;
  long long o = u - c * unit - wcost;
  o = o < 0 ? 0 : (o > n ? n : o);
  return c * n + o;
}
// One pipeline item.  The 128-wide depth-3 items (768 threads, at most 80
// registers each) run out of line, so that the partition's state does not
// compete with the pipeline for registers (it is saved once per item); the
// others, with registers to spare, stay inline.
template <int K, int TXT, typename PT = float>
__device__ __noinline__ bool step_item_ool(char* smem, const CUtensorMap* map_psi, const CUtensorMap* map_v, PT* out,
                                           int n, int x0, int y0, int z0, int z1, float half_dtau, float one_m6c,
                                           float cc, int32_t* err, int nz, int zlo, int zhi) {
  return tma_step_item<K, TXT, TY, PT>(smem, map_psi, map_v, out, n, x0, y0, z0, z1, half_dtau, one_m6c, cc, err, nz,
                                       zlo, zhi);
}
template <int K, int TXT, typename PT = float>
__device__ __forceinline__ bool step_item(char* smem, const CUtensorMap* map_psi, const CUtensorMap* map_v, PT* out,
                                          int n, int x0, int y0, int z0, int z1, float half_dtau, float one_m6c,
                                          float cc, int32_t* err, int nz = -1, int zlo = 0, int zhi = -1) {
  if constexpr (TXT == 128 && K == 3)
    return step_item_ool<K, TXT, PT>(smem, map_psi, map_v, out, n, x0, y0, z0, z1, half_dtau, one_m6c, cc, err, nz,
                                     zlo, zhi);
  else
    return tma_step_item<K, TXT, TY, PT>(smem, map_psi, map_v, out, n, x0, y0, z0, z1, half_dtau, one_m6c, cc, err,
                                         nz, zlo, zhi);
}

template <int K, int TXT, typename PT = float>
__global__ void __launch_bounds__(Geo<K, TXT>::THREADS) k_step_tma(const __grid_constant__ CUtensorMap map_psi,
                                                                    const __grid_constant__ CUtensorMap map_v,
                                                                    PT* __restrict__ out, int n, int ntx,
                                                                    long long total, int span, int wcost,
                                                                    int zsplit, float half_dtau,
                                                                    float one_m6c, float cc,
                                                                    const int32_t* __restrict__ active,
                                                                    int32_t* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  if (active && *active == 0) return;
  if (*(volatile const int32_t*)err != 0) return;  // an earlier wait expired: do nothing
  extern __shared__ __align__(128) char smem_raw[];
  char* smem = aligned_smem(smem_raw);
  // the block's items: the range [r, rend) of a sequence of columns of
  // `top` planes each, starting at plane `base` of every column
  long long r, rend;
  int top = n, base = 0;
  if (span == -2) {
    const int C = (int)(total / n);
    if ((int)blockIdx.x < C) {
      top = zsplit;
      r = (long long)blockIdx.x * top;
      rend = r + top;
    } else {
      const int rb = gridDim.x - C;
      top = n - zsplit;
      base = zsplit;
      const long long rest = (long long)C * top;
      r = rest * (blockIdx.x - C) / rb;
      rend = rest * (blockIdx.x - C + 1) / rb;
    }
  } else if (span > 0) {
    r = (long long)blockIdx.x * span;
    rend = min(r + span, total);
  } else {
    const long long ctot = (total / n) * (n + wcost);
    r = balanced_plane(ctot * blockIdx.x / gridDim.x, n, wcost);
    rend = balanced_plane(ctot * (blockIdx.x + 1) / gridDim.x, n, wcost);
  }
  while (r < rend) {
    const int t = (int)(r / top), z0 = (int)(r - (long long)t * top);
    const int z1 = (int)min((long long)top, z0 + (rend - r));
    if (!step_item<K, TXT, PT>(smem, &map_psi, &map_v, out, n, (t % ntx) * TXT, (t / ntx) * TY, base + z0,
                               base + z1, half_dtau, one_m6c, cc, err))
      return;
    r += z1 - z0;
  }
}

// K update steps on a z-slab of the lattice (Sec. V): a field of n x n x
// nzbuf sites whose planes [zbase, zbase + nzo) are this slab's own and
// whose `zbase` planes below and above are halo copies of the neighbouring
// slabs' planes (planes outside [zlo, zhi) lie beyond the lattice's faces and
// stay zero).  The own planes of every tile column are dealt to the blocks
// by the balanced partition of k_step_tma.
template <int K, int TXT>
__global__ void __launch_bounds__(Geo<K, TXT>::THREADS) k_step_slab(const __grid_constant__ CUtensorMap map_psi,
                                                                     const __grid_constant__ CUtensorMap map_v,
                                                                     float* __restrict__ out, int n, int ntx,
                                                                     int ncol, int nzo, int zbase, int nzbuf,
                                                                     int zlo, int zhi, float half_dtau,
                                                                     float one_m6c, float cc,
                                                                     int32_t* __restrict__ err) {
  if (*(volatile const int32_t*)err != 0) return;
  extern __shared__ __align__(128) char smem_raw[];
  char* smem = aligned_smem(smem_raw);
  const int wcost = 2 * (K - 1);
  const long long ctot = (long long)ncol * (nzo + wcost);
  long long r = balanced_plane(ctot * blockIdx.x / gridDim.x, nzo, wcost);
  const long long rend = balanced_plane(ctot * (blockIdx.x + 1) / gridDim.x, nzo, wcost);
  while (r < rend) {
    const int t = (int)(r / nzo), z0 = (int)(r - (long long)t * nzo);
    const int z1 = (int)min((long long)nzo, z0 + (rend - r));
    if (!step_item<K, TXT>(smem, &map_psi, &map_v, out, n, (t % ntx) * TXT, (t / ntx) * TY, zbase + z0,
                           zbase + z1, half_dtau, one_m6c, cc, err, nzbuf, zlo, zhi))
      return;
    r += z1 - z0;
  }
}

// The check step: one update step from map_psi's field into `out` and the
// lattice sums of the result, over the lattice sums' items (grid and
// partial index as k_sums_tma), so that the partials equal those of a
// separate k_sums_tma on `out` bit for bit.
__global__ void __launch_bounds__(Geo<2, kSumsTX>::THREADS) k_step_sums_tma(const __grid_constant__ CUtensorMap map_psi,
                                                                            const __grid_constant__ CUtensorMap map_v,
                                                                            float* __restrict__ out, int n,
                                                                            float half_dtau, float one_m6c, float cc,
                                                                            float a, float kfac,
                                                                            double* __restrict__ partials,
                                                                            const int32_t* __restrict__ active,
                                                                            int32_t* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  if (active && *active == 0) return;
  if (*(volatile const int32_t*)err != 0) return;
  extern __shared__ __align__(128) char smem_raw[];
  char* smem = aligned_smem(smem_raw);
  const int item = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  const int zc = sums_zchunk(n), z0 = blockIdx.z * zc;
  tma_step_sums_item<kSumsTX>(smem, &map_psi, &map_v, out, n, blockIdx.x * kSumsTX, blockIdx.y * TY, z0,
                              min(z0 + zc, n), half_dtau, one_m6c, cc, a, kfac, partials + (size_t)item * 4, err);
}

// Partial sums of a z-slab's own planes [zbase, zbase + nzo) (Sec. V: each
// process sums its own planes), cut like the lattice sums; plane zbase is
// the lattice's plane z_first.
__global__ void __launch_bounds__(Geo<1, kSumsTX>::THREADS) k_slab_sums_tma(const __grid_constant__ CUtensorMap map_psi,
                                                                            const __grid_constant__ CUtensorMap map_v,
                                                                            int n, int nzo, int zbase, int z_first,
                                                                            float a, float kfac,
                                                                            double* __restrict__ partials,
                                                                            int32_t* __restrict__ err) {
  if (*(volatile const int32_t*)err != 0) return;
  extern __shared__ __align__(128) char smem_raw[];
  char* smem = aligned_smem(smem_raw);
  const int item = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  const int zc = sums_zchunk_of(n, nzo), z0 = blockIdx.z * zc;
  tma_sums_item<kSumsTX>(smem, &map_psi, &map_v, n, blockIdx.x * kSumsTX, blockIdx.y * TY, zbase + z0,
                         zbase + min(z0 + zc, nzo), a, kfac, partials + (size_t)item * 4, err, z_first - zbase);
}

__global__ void __launch_bounds__(Geo<1, kSumsTX>::THREADS) k_sums_tma(const __grid_constant__ CUtensorMap map_psi,
                                                                       const __grid_constant__ CUtensorMap map_v,
                                                                       int n, float a, float kfac,
                                                                       double* __restrict__ partials,
                                                                       const int32_t* __restrict__ active,
                                                                       int32_t* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  if (active && *active == 0) return;
  if (*(volatile const int32_t*)err != 0) return;
  extern __shared__ __align__(128) char smem_raw[];
  char* smem = aligned_smem(smem_raw);
  const int item = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  const int zc = sums_zchunk(n), z0 = blockIdx.z * zc;
  tma_sums_item<kSumsTX>(smem, &map_psi, &map_v, n, blockIdx.x * kSumsTX, blockIdx.y * TY, z0, min(z0 + zc, n), a,
                         kfac, partials + (size_t)item * 4, err);
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
long long tile_planes(int n) {
  return (long long)((n + TXT - 1) / TXT) * ((n + TY - 1) / TY) * n;
}

template <int K, int TXT, typename PT = float>
int resident_blocks();

// span > 0: equal spans; span == -2: columns first; other span <= 0: the balanced
// partition over one wave
template <int K, int TXT, typename PT = float>
void launch_k(const CUtensorMap& mpsi, const CUtensorMap& mv, PT* out, const Params& p, int span,
              const int32_t* active, int32_t* err, cudaStream_t st) {
  using G = Geo<K, TXT, TY, PT>;
  set_smem(k_step_tma<K, TXT, PT>, G::SMEM);
  const long long total = tile_planes<K, TXT>(p.n);
  const unsigned blocks = span > 0 ? (unsigned)((total + span - 1) / span)
                                   : (unsigned)std::min<long long>(resident_blocks<K, TXT, PT>(), total);
  const int w = 2 * (K - 1);
  int zsplit = 0;
  if (span == -2) {
    // columns first needs more blocks than columns; zsplit = C (n + w) / blocks
    // gives both groups the same planes plus warm-up steps
    const long long C = total / p.n;
    zsplit = (int)std::min<long long>(p.n, C * (p.n + w) / std::max(1u, blocks));
    if ((long long)blocks <= C || zsplit < 1 || zsplit >= p.n) span = -1;
  }
  launch_pdl(k_step_tma<K, TXT, PT>, dim3(blocks), dim3(G::THREADS), G::SMEM, st, mpsi, mv, out, p.n,
             (p.n + TXT - 1) / TXT, total, span > 0 ? span : (span == -2 ? -2 : 0), w, zsplit, p.half_dtau_f,
             p.one_m6c_f, p.c_f, active, err);
}

// Blocks of k_step_tma<K, TXT> resident on the whole device at once
// (queried once per device).
template <int K, int TXT, typename PT>
int resident_blocks() {
  using G = Geo<K, TXT, TY, PT>;
  static int cache[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && cache[dev] > 0) return cache[dev];
  set_smem(k_step_tma<K, TXT, PT>, G::SMEM);
  int sms = 0, occ = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step_tma<K, TXT, PT>, G::THREADS, G::SMEM);
  const int r = std::max(1, sms) * std::max(1, occ);
  if (dev < 64) cache[dev] = r;
  return r;
}

}  // namespace tb

int blocked_max_depth() { return 3; }

bool tma_supported(int n, int precision) { return precision == FDTD_F32 && n % 4 == 0 && n >= 8; }

int auto_depth(int n, int precision) {
  if (!tma_supported(n, precision)) return 1;
  return n >= 96 ? 3 : 2;
}

long long tma_tile_planes(int n, int tx) {
  return tx == 64 ? tb::tile_planes<1, 64>(n) : tb::tile_planes<1, 128>(n);
}

namespace {
template <typename PT>
int resident_of(int depth, int tx) {
  if (tx == 64)
    return depth == 1 ? tb::resident_blocks<1, 64, PT>()
                      : depth == 2 ? tb::resident_blocks<2, 64, PT>() : tb::resident_blocks<3, 64, PT>();
  return depth == 1 ? tb::resident_blocks<1, 128, PT>()
                    : depth == 2 ? tb::resident_blocks<2, 128, PT>() : tb::resident_blocks<3, 128, PT>();
}
template <typename PT>
void launch_step_any(const CUtensorMap& map_psi_in, const CUtensorMap& map_v, PT* out, const Params& p, int depth,
                     int tx, int zc, const int32_t* active, int32_t* err, cudaStream_t st) {
  if (zc == 0) zc = tma_zchunk(p.n, depth, tx, sizeof(PT) == 2);  // zc -2: columns first, other zc < 0: balanced
  if (tx == 64) {
    if (depth == 1)
      tb::launch_k<1, 64, PT>(map_psi_in, map_v, out, p, zc, active, err, st);
    else if (depth == 2)
      tb::launch_k<2, 64, PT>(map_psi_in, map_v, out, p, zc, active, err, st);
    else
      tb::launch_k<3, 64, PT>(map_psi_in, map_v, out, p, zc, active, err, st);
  } else {
    if (depth == 1)
      tb::launch_k<1, 128, PT>(map_psi_in, map_v, out, p, zc, active, err, st);
    else if (depth == 2)
      tb::launch_k<2, 128, PT>(map_psi_in, map_v, out, p, zc, active, err, st);
    else
      tb::launch_k<3, 128, PT>(map_psi_in, map_v, out, p, zc, active, err, st);
  }
}
}  // namespace

int tma_resident_blocks(int depth, int tx, bool bf16) {
  return bf16 ? resident_of<__nv_bfloat16>(depth, tx) : resident_of<float>(depth, tx);
}

int tma_zchunk(int n, int depth, int tx, bool bf16) {
  // one wave of equal spans over the resident blocks
  const long long total = tma_tile_planes(n, tx), slots = tma_resident_blocks(depth, tx, bf16);
  return (int)std::max(1LL, (total + slots - 1) / slots);
}

void launch_step_tma(const CUtensorMap& map_psi_in, const CUtensorMap& map_v, float* out, const Params& p, int depth,
                     int tx, int zc, const int32_t* active, int32_t* err, cudaStream_t st) {
  launch_step_any<float>(map_psi_in, map_v, out, p, depth, tx, zc, active, err, st);
}

void launch_step_tma(const CUtensorMap& map_psi_in, const CUtensorMap& map_v, __nv_bfloat16* out, const Params& p,
                     int depth, int tx, int zc, const int32_t* active, int32_t* err, cudaStream_t st) {
  launch_step_any<__nv_bfloat16>(map_psi_in, map_v, out, p, depth, tx, zc, active, err, st);
}

namespace tb {
template <int K>
void launch_slab_k(const CUtensorMap& mpsi, const CUtensorMap& mv, float* out, const Params& p, int nzo, int zbase,
                   int nzbuf, int zlo, int zhi, int32_t* err, cudaStream_t st) {
  using G = Geo<K, 128>;
  set_smem(k_step_slab<K, 128>, G::SMEM);
  const int ntx = (p.n + 127) / 128, ncol = ntx * ((p.n + TY - 1) / TY);
  const long long planes = (long long)ncol * nzo;
  const unsigned blocks = (unsigned)std::max<long long>(1, std::min<long long>(resident_blocks<K, 128>(), planes));
  k_step_slab<K, 128><<<blocks, G::THREADS, G::SMEM, st>>>(mpsi, mv, out, p.n, ntx, ncol, nzo, zbase, nzbuf, zlo, zhi,
                                                           p.half_dtau_f, p.one_m6c_f, p.c_f, err);
}
}  // namespace tb

void launch_step_slab(const CUtensorMap& map_psi_in, const CUtensorMap& map_v, float* out, const Params& p, int depth,
                      int nzo, int zbase, int nzbuf, int zlo, int zhi, int32_t* err, cudaStream_t st) {
  if (depth == 1)
    tb::launch_slab_k<1>(map_psi_in, map_v, out, p, nzo, zbase, nzbuf, zlo, zhi, err, st);
  else if (depth == 2)
    tb::launch_slab_k<2>(map_psi_in, map_v, out, p, nzo, zbase, nzbuf, zlo, zhi, err, st);
  else
    tb::launch_slab_k<3>(map_psi_in, map_v, out, p, nzo, zbase, nzbuf, zlo, zhi, err, st);
}

int tma_sums_blocks(int n) { return tb::sums_items(n); }

int launch_step_sums_tma(const CUtensorMap& map_psi, const CUtensorMap& map_v, float* out, const Params& p,
                         double* partials, const int32_t* active, int32_t* err, cudaStream_t st) {
  using G = tb::Geo<2, tb::kSumsTX>;
  tb::set_smem(tb::k_step_sums_tma, G::SMEM);
  const int zc = tb::sums_zchunk(p.n);
  dim3 grid((p.n + tb::kSumsTX - 1) / tb::kSumsTX, (p.n + tb::TY - 1) / tb::TY, (p.n + zc - 1) / zc);
  launch_pdl(tb::k_step_sums_tma, grid, dim3(G::THREADS), G::SMEM, st, map_psi, map_v, out, p.n, p.half_dtau_f,
             p.one_m6c_f, p.c_f, (float)p.a, (float)(1.0 / (2.0 * p.mass * p.a * p.a)), partials, active, err);
  return (int)(grid.x * grid.y * grid.z);
}
int slab_sums_blocks(int n, int nzo) { return tb::sums_items_of(n, nzo); }

int launch_slab_sums(const CUtensorMap& map_psi, const CUtensorMap& map_v, const Params& p, int nzo, int zbase,
                     int z_first, double* partials, int32_t* err, cudaStream_t st) {
  using G = tb::Geo<1, tb::kSumsTX>;
  tb::set_smem(tb::k_slab_sums_tma, G::SMEM);
  const int zc = tb::sums_zchunk_of(p.n, nzo);
  dim3 grid((p.n + tb::kSumsTX - 1) / tb::kSumsTX, (p.n + tb::TY - 1) / tb::TY, (nzo + zc - 1) / zc);
  tb::k_slab_sums_tma<<<grid, G::THREADS, G::SMEM, st>>>(map_psi, map_v, p.n, nzo, zbase, z_first, (float)p.a,
                                                        (float)(1.0 / (2.0 * p.mass * p.a * p.a)), partials, err);
  return (int)(grid.x * grid.y * grid.z);
}

int launch_sums_tma(const CUtensorMap& map_psi, const CUtensorMap& map_v, const Params& p, double* partials,
                    const int32_t* active, int32_t* err, cudaStream_t st) {
  using G = tb::Geo<1, tb::kSumsTX>;
  tb::set_smem(tb::k_sums_tma, G::SMEM);
  const int zc = tb::sums_zchunk(p.n);
  dim3 grid((p.n + tb::kSumsTX - 1) / tb::kSumsTX, (p.n + tb::TY - 1) / tb::TY, (p.n + zc - 1) / zc);
  launch_pdl(tb::k_sums_tma, grid, dim3(G::THREADS), G::SMEM, st, map_psi, map_v, p.n, (float)p.a,
             (float)(1.0 / (2.0 * p.mass * p.a * p.a)), partials, active, err);
  return (int)(grid.x * grid.y * grid.z);
}

void tma_box(int depth, int tx, int* box_w, int* box_h, int ty) {
  *box_w = tx + 2 * tb::HX;
  *box_h = ty + 2 * depth;
}

int encode_field_map(CUtensorMap* map, const float* base, int n, int box_w, int box_h) {
  return encode_field_map_nz(map, base, n, n, box_w, box_h);
}

namespace {
// Tensor map of a dense n x n x nz field of `esize`-byte elements for box
// loads of box_w x box_h x 1 (zero fill outside the field).
int encode_map(CUtensorMap* map, CUtensorMapDataType dtype, int esize, const void* base, int n, int nz, int box_w,
               int box_h) {
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
  cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)nz};
  cuuint64_t strides[2] = {(cuuint64_t)n * esize, (cuuint64_t)n * n * esize};
  cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  // 64 B L2 promotion: a box row (tx + 8 floats) starts 16 B before a tile
  // boundary, and wider promotion fetches up to twice the row from HBM
  CUresult r = ((Encode)fn)(map, dtype, 3, (void*)base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_64B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -2;
}
}  // namespace

// Tensor map of a dense n x n x nz FP32 field for box loads of box_w x box_h x 1.
int encode_field_map_nz(CUtensorMap* map, const float* base, int n, int nz, int box_w, int box_h) {
  return encode_map(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, n, nz, box_w, box_h);
}

// The same for a BF16 field (n % 8 == 0, so that rows are 16-byte multiples).
int encode_field_map_bf16(CUtensorMap* map, const __nv_bfloat16* base, int n, int box_w, int box_h) {
  return encode_map(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, n, n, box_w, box_h);
}

// TMA box of a BF16 psi field for a tile item: (tx + 16) x (ty + 2 depth).
void tma_box_bf16(int depth, int tx, int* box_w, int* box_h, int ty) {
  *box_w = tx + 16;
  *box_h = ty + 2 * depth;
}

}  // namespace fdtd
