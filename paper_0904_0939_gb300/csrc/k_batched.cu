// Batched persistent driver: every lattice of a handle advances in ONE
// cooperative launch that runs the whole evolution -- checks (sums of
// Eq. energysum, renormalisation, symmetry re-imposition, convergence test
// on the binding energy, Secs. III-V) and update steps (Eq. updateeq) --
// until every lattice has converged or max_steps is reached.
//
// Work is split into phases separated by a grid-wide barrier:
//   SUMS      the lattice-sums items of every active lattice (the one-lattice
//             partition: 64 x 16 tile columns cut into z-chunks), dealt to
//             the blocks in equal runs of consecutive items, so that a block
//             streams several chunks of one column in one pipeline run;
//   FINALIZE  one lattice per block;
//   SCALE     renormalise + symmetry, out of place, float4 sites of every
//             checked lattice dealt grid-wide;
//   STEP      K update steps through the TMA pipeline of tma_item.cuh: the
//             tile columns of the active lattices are laid end to end, each
//             costing n + 2(K - 1) z-steps, and the cost line is cut into one
//             equal range per block (the balanced partition of the one-lattice
//             stencil, across lattices), so a block runs few, long items.
// Converged lattices drop out of every phase.  The per-site arithmetic and
// the reduction order are those of the one-lattice path, so every lattice
// ends bit-identical to a separate fdtd_evolve of the same lattice.
//
// A tuning mode runs a given number of STEP phases from the current fields
// into the spare ones without advancing the state, so that candidates
// (depth, tile width) can be timed on the same work.
//
// The grid barrier is a sense-reversing counter in global memory; every wait
// on it is bounded in wall-clock time, after which the block sets the error
// flag and leaves (the others then give up at their next wait).
#include <cooperative_groups.h>

#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"
#include "tma_item.cuh"

namespace fdtd {

namespace {

constexpr int kSumsTXB = tb::kSumsTX;  // tile width of the sums items (the one-lattice partition)
constexpr int kMaxLat = 256;           // lattices per batched handle

}  // namespace

// Device table entry of one lattice (written by the host before the launch).
struct alignas(128) BatchLat {
  CUtensorMap step_map[3][3][3];  // [tile 64x16, 128x16, 64x32][depth-1][psi0, psi1, V]
  CUtensorMap sums_map[3];        // [psi0, psi1, V], the sums box
  float* psi[2];
  double* partials;
  LatState* state;
  double* hist;  // check history ring (kHistCap records)
  int n, mask, cur, pad0;
  float hd, om6c, cc, a_f, kfac_f;
  int pad1;
  double a3, v_inf;
};

struct BatchRun {
  int64_t max_steps, t_start, t_end;
  double tol;
  int check_every, tol_rel, reimpose, depth, nlat, skip_first, check0, tune_passes;
  unsigned bar_count, bar_gen;
  int64_t steps_done;
};

size_t batched_workspace_bytes(const fdtd_lattice_desc*, int count) {
  return (size_t)count * sizeof(BatchLat) + sizeof(BatchRun) + 256;
}

namespace {

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Sense-reversing grid barrier, bounded in wall-clock time.  Returns false
// in every thread of the block if the wait expired (or another block
// already reported an error).
__device__ bool grid_barrier(BatchRun* run, int32_t* err) {
  __shared__ int bad;
  // psi written by plain stores in this phase is read by TMA (the async
  // proxy) in the next one, from other blocks
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    bad = 0;
    const unsigned gen = ld_acquire(&run->bar_gen);
    __threadfence();
    const unsigned arrived = atomicAdd(&run->bar_count, 1u) + 1u;
    if (arrived == gridDim.x) {
      run->bar_count = 0;
      __threadfence();
      atomicAdd(&run->bar_gen, 1u);
    } else {
      // budget: the word after the error flag (0 = 2 s, > 0 = microseconds,
      // < 0 = none: give up unless the barrier has already opened)
      const int us = *(volatile const int32_t*)(err + 1);
      const unsigned long long budget = us == 0 ? 2000ull * 1000 * 1000 : (us > 0 ? 1000ull * us : 0ull);
      const unsigned long long t0 = tb::global_ns();
      unsigned it = 0;
      while (ld_acquire(&run->bar_gen) == gen) {
        if (us < 0 || (++it & 63u) == 0) {
          if (us < 0 || *(volatile int32_t*)err != 0 || tb::global_ns() - t0 > budget) {
            atomicOr(err, 1);
            bad = 1;
            break;
          }
        }
      }
    }
    __threadfence();
    asm volatile("fence.proxy.async.global;" ::: "memory");
  }
  __syncthreads();
  return bad == 0;
}

// the lattice whose range [pre[l], pre[l + 1]) holds u: the largest l with
// pre[l] <= u (lattices with empty ranges are skipped that way)
template <typename T>
__device__ __forceinline__ int find_lattice(const T* pre, int nlat, T u) {
  int lo = 0, hi = nlat - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= u)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// tile plane c n + clamp(u - c (n + w) - w, 0, n), c = u / (n + w): the
// balanced partition's map from cost to tile planes of one lattice
__device__ __forceinline__ long long cost_to_plane(long long u, int n, int w) {
  const long long unit = n + w, c = u / unit;
  long long o = u - c * unit - w;
  o = o < 0 ? 0 : (o > n ? n : o);
  return c * n + o;
}

// Check of Secs. III-V on the block's lattice, same order as k_finalize;
// red: 1024 doubles of scratch (the block's dynamic shared memory).
__device__ void finalize_lattice(const BatchLat& L, int nparts, int check_id, int64_t t, const BatchRun& run,
                                 double* red) {
  double (*sm)[256] = reinterpret_cast<double (*)[256]>(red);
  LatState* s = L.state;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < nparts; i += 256)
    if (threadIdx.x < 256)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += L.partials[(size_t)i * 4 + q];
  if (threadIdx.x < 256)
#pragma unroll
    for (int q = 0; q < 4; ++q) sm[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < 4; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double s0 = sm[0][0], sh = sm[1][0], sr = sm[2][0], sv = sm[3][0];
    if (!(s0 > 0.0) || !isfinite(s0) || !isfinite(sh) || !isfinite(sr) || !isfinite(sv)) {
      s->status = STATUS_NONFINITE;
      s->active = 0;
      s->scale_seq = -1;
    } else {
      s->scale = 1.0 / sqrt(s0 * L.a3);
      s->scale_seq = check_id;
      double e = sh / s0, eb = e - L.v_inf;
      s->s0 = s0;
      s->sh = sh;
      s->sr = sr;
      s->sv = sv;
      s->energy = e;
      s->ebind = eb;
      s->r2 = sr / s0;
      s->vexp = sv / s0;
      s->step = t;
      s->checks += 1;
      double d = -1.0;
      if (s->has_prev) {
        d = fabs(eb - s->e_prev);
        double thr = run.tol * (run.tol_rel ? fabs(eb) : 1.0);
        if (run.tol > 0.0 && d <= thr) {
          s->converged = 1;
          s->active = 0;
        }
      }
      s->delta_e = d;
      s->e_prev = eb;
      s->has_prev = 1;
      if (L.hist) {
        double* h = L.hist + (size_t)((s->checks - 1) % kHistCap) * kHistFields;
        h[0] = (double)t;
        h[1] = e;
        h[2] = eb;
        h[3] = s0 * L.a3;
        h[4] = sr / s0;
        h[5] = sv / s0;
        h[6] = d;
        h[7] = s0;
      }
    }
  }
  __syncthreads();
}

// Per-block views of the lattices, rebuilt by thread 0 whenever the active
// set changes: prefix sums of the sums items and of the STEP costs of the
// active lattices.
struct Views {
  int pre_sums[kMaxLat + 1];
  long long pre_cost[kMaxLat + 1];
  long long pre_scale[kMaxLat + 1];
  int cur[kMaxLat], act[kMaxLat];
  float scale[kMaxLat];
};

template <int TXT, int TYT>
__device__ void build_prefixes(Views& v, const BatchLat* __restrict__ lats, int nlat, int w) {
  int a = 0;
  long long b = 0;
  for (int l = 0; l < nlat; ++l) {
    v.pre_sums[l] = a;
    v.pre_cost[l] = b;
    if (!v.act[l]) continue;
    const int n = lats[l].n;
    a += tb::sums_items(n);
    b += (long long)((n + TXT - 1) / TXT) * ((n + TYT - 1) / TYT) * (n + w);
  }
  v.pre_sums[nlat] = a;
  v.pre_cost[nlat] = b;
}

// One update item, kept out of line so that the phase loop's state does not
// compete with the pipeline for registers (it is saved once per item).
template <int K, int TXT, int TYT>
__device__ __noinline__ bool step_item(char* smem, const CUtensorMap* map_psi, const CUtensorMap* map_v, float* out,
                                       int n, int x0, int y0, int z0, int z1, float hd, float om6c, float cc,
                                       int32_t* err) {
  return tb::tma_step_item<K, TXT, TYT>(smem, map_psi, map_v, out, n, x0, y0, z0, z1, hd, om6c, cc, err);
}

// A run of consecutive sums items of one tile column, out of line like the
// update items.
__device__ __noinline__ bool sums_run(char* smem, const CUtensorMap* map_psi, const CUtensorMap* map_v, int n, int x0,
                                      int y0, int z0, int z1, float a, float kfac, double* dst, int32_t* err, int zc,
                                      long long stride) {
  return tb::tma_sums_item<kSumsTXB>(smem, map_psi, map_v, n, x0, y0, z0, z1, a, kfac, dst, err, 0, zc, stride);
}

// One STEP phase: k (<= KMAX) steps of every active lattice, from field
// cur[l] into the other, over the block's range of the cost line.
template <int KMAX, int TXT, int TYT>
__device__ bool step_phase(char* smem, const Views& v, const BatchLat* __restrict__ lats, int nlat, int k, int w,
                           int32_t* err) {
  const long long U = v.pre_cost[nlat];
  const long long u0 = U * blockIdx.x / gridDim.x, u1 = U * (blockIdx.x + 1) / gridDim.x;
  if (u0 >= u1) return true;
  constexpr int TI = TXT == 128 ? 1 : (TYT == 32 ? 2 : 0);
  bool ok = true;
  for (int l = find_lattice(v.pre_cost, nlat, u0); l < nlat && v.pre_cost[l] < u1 && ok; ++l) {
    if (!v.act[l]) continue;
    const BatchLat& L = lats[l];
    const int n = L.n, gx = (n + TXT - 1) / TXT;
    const long long base = v.pre_cost[l];
    const long long lo = (u0 > base ? u0 : base) - base;
    const long long hi = (u1 < v.pre_cost[l + 1] ? u1 : v.pre_cost[l + 1]) - base;
    long long r = cost_to_plane(lo, n, w);
    const long long rend = cost_to_plane(hi, n, w);
    const int cur = v.cur[l];
    while (r < rend && ok) {
      const int t = (int)(r / n), z0 = (int)(r - (long long)t * n);
      const int z1 = (int)((long long)n < z0 + (rend - r) ? (long long)n : z0 + (rend - r));
      const int x0 = (t % gx) * TXT, y0 = (t / gx) * TYT;
      if (k == 1)
        ok = step_item<1, TXT, TYT>(smem, &L.step_map[TI][0][cur], &L.step_map[TI][0][2], L.psi[cur ^ 1], n, x0,
                                       y0, z0, z1, L.hd, L.om6c, L.cc, err);
      else if (k == 2 || KMAX == 2)
        ok = step_item<(KMAX >= 2 ? 2 : 1), TXT, TYT>(smem, &L.step_map[TI][1][cur], &L.step_map[TI][1][2],
                                                         L.psi[cur ^ 1], n, x0, y0, z0, z1, L.hd, L.om6c, L.cc, err);
      else
        ok = step_item<KMAX, TXT, TYT>(smem, &L.step_map[TI][KMAX - 1][cur], &L.step_map[TI][KMAX - 1][2],
                                          L.psi[cur ^ 1], n, x0, y0, z0, z1, L.hd, L.om6c, L.cc, err);
      r += z1 - z0;
    }
  }
  return ok;
}

template <int KMAX, int TXT, int TYT>
__global__ void __launch_bounds__(tb::Geo<KMAX, TXT, TYT>::THREADS) k_batched(const BatchLat* __restrict__ lats,
                                                                         BatchRun* run, int32_t* err) {
  extern __shared__ __align__(128) char smem_raw[];
  char* smem = tb::aligned_smem(smem_raw);
  __shared__ Views v;
  const int nlat = run->nlat;
  const int64_t max_steps = run->max_steps;
  const int ce = run->check_every;
  const int w = 2 * (KMAX - 1);
  if (threadIdx.x == 0) {
    for (int l = 0; l < nlat; ++l) {
      v.cur[l] = lats[l].cur;
      v.act[l] = lats[l].state->active;  // a lattice that converged in an earlier launch stays retired
    }
    build_prefixes<TXT, TYT>(v, lats, nlat, w);
  }
  __syncthreads();
  const int64_t t_start = run->t_start, t_end = run->t_end;
  if (run->tune_passes > 0) {  // timing: STEP phases into the spare fields, state unchanged
    for (int p = 0; p < run->tune_passes; ++p)
      if (!step_phase<KMAX, TXT, TYT>(smem, v, lats, nlat, KMAX, w, err) || !grid_barrier(run, err)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) run->steps_done = t_start;
    return;
  }
  int64_t t = t_start;
  int check_id = run->check0;
  for (;;) {
    if ((t % ce == 0 || t == max_steps) && !(run->skip_first && t == t_start)) {
      // ---- SUMS: equal runs of consecutive sums items (chunks of one column stream as one run)
      {
        const int C = v.pre_sums[nlat];
        const int c0 = (int)((long long)C * blockIdx.x / gridDim.x);
        const int c1 = (int)((long long)C * (blockIdx.x + 1) / gridDim.x);
        bool ok = true;
        for (int it = c0; it < c1 && ok;) {
          const int l = find_lattice(v.pre_sums, nlat, it);
          const BatchLat& L = lats[l];
          const int n = L.n, gx = (n + kSumsTXB - 1) / kSumsTXB, gy = (n + tb::TY - 1) / tb::TY;
          const int zc = tb::sums_zchunk(n), nch = (n + zc - 1) / zc;
          const int q = it - v.pre_sums[l], col = q / nch, ch0 = q - col * nch;
          const int ch1 = min(nch, ch0 + (c1 - it));
          const int tx = col % gx, ty = col / gx;
          ok = sums_run(smem, &L.sums_map[v.cur[l]], &L.sums_map[2], n, tx * kSumsTXB, ty * tb::TY, ch0 * zc,
                        min(ch1 * zc, n), L.a_f, L.kfac_f,
                        L.partials + ((size_t)ch0 * gy * gx + (size_t)ty * gx + tx) * 4, err, zc,
                        (long long)gx * gy * 4);
          it += ch1 - ch0;
        }
        if (!ok || !grid_barrier(run, err)) return;
      }
      // ---- FINALIZE
      for (int l = blockIdx.x; l < nlat; l += gridDim.x) {
        if (!v.act[l]) continue;
        finalize_lattice(lats[l], tb::sums_items(lats[l].n), check_id, t, *run, (double*)smem);
      }
      if (!grid_barrier(run, err)) return;
      // ---- SCALE: out = P(scale * in) for the lattices checked now, float4 sites dealt grid-wide
      if (threadIdx.x == 0) {
        long long a = 0;
        for (int l = 0; l < nlat; ++l) {
          v.pre_scale[l] = a;
          const LatState* st = lats[l].state;
          if (v.act[l] && *(volatile const int32_t*)&st->scale_seq == check_id) {
            v.scale[l] = (float)*(volatile const double*)&st->scale;
            a += (long long)lats[l].n * lats[l].n * (lats[l].n >> 2);
          }
        }
        v.pre_scale[nlat] = a;
      }
      __syncthreads();
      {
        const long long T4 = v.pre_scale[nlat];
        const long long stride = (long long)gridDim.x * blockDim.x;
        for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < T4; g += stride) {
          const int l = find_lattice(v.pre_scale, nlat, g);
          const BatchLat& L = lats[l];
          const int n = L.n, n4 = n >> 2;
          const long long i4 = g - v.pre_scale[l];
          const long long row = i4 / n4;
          const int x4 = (int)(i4 - row * n4), y = (int)(row % n), z = (int)(row / n);
          scale_parity_f4_at(L.psi[v.cur[l]], L.psi[v.cur[l] ^ 1], n, run->reimpose ? L.mask : 0, v.scale[l], x4, y, z);
        }
      }
      if (!grid_barrier(run, err)) return;
      // every block updates its view of the lattices identically
      if (threadIdx.x == 0) {
        for (int l = 0; l < nlat; ++l) {
          if (!v.act[l]) continue;
          const LatState* st = lats[l].state;
          if (*(volatile const int32_t*)&st->scale_seq == check_id) v.cur[l] ^= 1;
          v.act[l] = *(volatile const int32_t*)&st->active;
          if (blockIdx.x == 0) lats[l].state->cur = v.cur[l];
        }
        build_prefixes<TXT, TYT>(v, lats, nlat, w);
      }
      __syncthreads();
      ++check_id;
      if (t >= t_end || v.pre_sums[nlat] == 0) break;
    }
    // ---- STEP: up to the next check, KMAX steps per phase
    const int64_t nc = (t / ce + 1) * ce;
    const int64_t next = nc < t_end ? nc : t_end;
    while (t < next) {
      const int k = (int)((next - t) < KMAX ? (next - t) : KMAX);
      if (!step_phase<KMAX, TXT, TYT>(smem, v, lats, nlat, k, w, err) || !grid_barrier(run, err)) return;
      if (threadIdx.x == 0)
        for (int l = 0; l < nlat; ++l)
          if (v.act[l]) v.cur[l] ^= 1;
      __syncthreads();
      t += k;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    run->steps_done = t;
    for (int l = 0; l < nlat; ++l) lats[l].state->cur = v.cur[l];
  }
}

template <int KMAX, int TXT, int TYT>
size_t batched_smem() {
  size_t a = tb::Geo<KMAX, TXT, TYT>::SMEM;
  size_t b = tb::Geo<1, kSumsTXB>::SMEM + 8 * 4 * (tb::Geo<KMAX, TXT, TYT>::THREADS / 32);  // sums item + reduction
  return a > b ? a : b;
}

}  // namespace

// Host side: fill the device table and launch the persistent kernel once
// (cooperative, so every block is resident and the grid barrier can complete).
int batched_max_lattices() { return kMaxLat; }

int batched_fill(void* host_entry, const float* psi0, const float* psi1, const float* v, double* partials,
                 LatState* state, double* hist, const Params& p, int mask, int cur, double v_inf) {
  BatchLat& B = *(BatchLat*)host_entry;
  int bw, bh;
  const float* bufs[3] = {psi0, psi1, v};
  for (int kind = 0; kind < kBatchedTileKinds; ++kind)
    for (int k = 1; k <= 3; ++k) {
      tma_box(k, batched_tile_x(kind), &bw, &bh, batched_tile_y(kind));
      for (int b = 0; b < 3; ++b)
        if (encode_field_map(&B.step_map[kind][k - 1][b], bufs[b], p.n, bw, bh)) return -1;
    }
  tma_box(1, kSumsTXB, &bw, &bh);
  for (int b = 0; b < 3; ++b)
    if (encode_field_map(&B.sums_map[b], bufs[b], p.n, bw, bh)) return -1;
  B.psi[0] = (float*)psi0;
  B.psi[1] = (float*)psi1;
  B.partials = partials;
  B.state = state;
  B.hist = hist;
  B.n = p.n;
  B.mask = mask;
  B.cur = cur;
  B.hd = p.half_dtau_f;
  B.om6c = p.one_m6c_f;
  B.cc = p.c_f;
  B.a_f = (float)p.a;
  B.kfac_f = (float)(1.0 / (2.0 * p.mass * p.a * p.a));
  B.a3 = p.a * p.a * p.a;
  B.v_inf = v_inf;
  return 0;
}

void batched_patch(void* host_entry, int mask, int cur) {
  BatchLat& B = *(BatchLat*)host_entry;
  B.mask = mask;
  B.cur = cur;
}

size_t batched_entry_bytes() { return sizeof(BatchLat); }
size_t batched_run_offset(int count) { return (size_t)count * sizeof(BatchLat); }

void BatchedGraphs::release() {
  for (int t = 0; t < kBatchedTileKinds; ++t)
    for (int d = 0; d < 4; ++d) {
      if (exec[t][d]) cudaGraphExecDestroy(exec[t][d]);
      exec[t][d] = nullptr;
      grid[t][d] = 0;
    }
}

int batched_prepare(void* dev_table, int count, int depth, int kind, int32_t* err, BatchedGraphs* graphs) {
  depth = depth < 1 ? 1 : (depth > 3 ? 3 : depth);
  const int ti = kind < 0 || kind >= kBatchedTileKinds ? 0 : kind;
  if (graphs->exec[ti][depth]) return 0;
  // capture the cooperative launch once: grid = resident blocks of the whole device
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const BatchLat* tab = (const BatchLat*)dev_table;
  BatchRun* drun = (BatchRun*)((char*)dev_table + batched_run_offset(count));
  void* args[3] = {(void*)&tab, (void*)&drun, (void*)&err};
  auto capture = [&](auto kern, int threads, size_t smem) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = per_sm * sms;
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t el = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(threads), args, smem, cs);
      e = cudaStreamEndCapture(cs, &g);
      if (e == cudaSuccess) e = el;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&graphs->exec[ti][depth], g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      graphs->exec[ti][depth] = nullptr;
      return e;
    }
    graphs->grid[ti][depth] = grid;
    return cudaSuccess;
  };
  auto by_depth = [&](auto tx_c, auto ty_c) {
    constexpr int TXT = decltype(tx_c)::value, TYT = decltype(ty_c)::value;
    if (depth == 1) return capture(k_batched<1, TXT, TYT>, tb::Geo<1, TXT, TYT>::THREADS, batched_smem<1, TXT, TYT>());
    if (depth == 2) return capture(k_batched<2, TXT, TYT>, tb::Geo<2, TXT, TYT>::THREADS, batched_smem<2, TXT, TYT>());
    return capture(k_batched<3, TXT, TYT>, tb::Geo<3, TXT, TYT>::THREADS, batched_smem<3, TXT, TYT>());
  };
  cudaError_t e;
  if (ti == 0)
    e = by_depth(std::integral_constant<int, 64>{}, std::integral_constant<int, 16>{});
  else if (ti == 1)
    e = by_depth(std::integral_constant<int, 128>{}, std::integral_constant<int, 16>{});
  else
    e = by_depth(std::integral_constant<int, 64>{}, std::integral_constant<int, 32>{});
  if (e != cudaSuccess) {
    cudaGetLastError();
    return (int)e;
  }
  return 0;
}

int batched_launch(void* dev_table, int count, int64_t max_steps, int64_t t_start, int64_t t_end, int skip_first,
                   int check0, int check_every, double tol, int tol_rel, int reimpose, int depth, int kind,
                   int tune_passes, int32_t* err, cudaStream_t st, BatchedGraphs* graphs, int64_t* steps_done,
                   int* grid_out) {
  BatchRun run{};
  run.max_steps = max_steps;
  run.t_start = t_start;
  run.t_end = t_end;
  run.skip_first = skip_first;
  run.check0 = check0;
  run.tol = tol;
  run.check_every = check_every;
  run.tol_rel = tol_rel;
  run.reimpose = reimpose;
  run.depth = depth;
  run.nlat = count;
  run.tune_passes = tune_passes;
  BatchRun* drun = (BatchRun*)((char*)dev_table + batched_run_offset(count));
  cudaMemcpyAsync(drun, &run, sizeof(run), cudaMemcpyHostToDevice, st);
  int e = batched_prepare(dev_table, count, depth, kind, err, graphs);
  if (e) return e;
  depth = depth < 1 ? 1 : (depth > 3 ? 3 : depth);
  const int ti = kind < 0 || kind >= kBatchedTileKinds ? 0 : kind;
  *grid_out = graphs->grid[ti][depth];
  cudaError_t ce = cudaGraphLaunch(graphs->exec[ti][depth], st);
  if (ce != cudaSuccess) return (int)ce;
  cudaMemcpyAsync(steps_done, &drun->steps_done, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  return 0;
}

}  // namespace fdtd
