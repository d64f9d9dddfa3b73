// Batched persistent driver: every lattice of a handle advances in ONE
// cooperative launch that runs the whole evolution -- checks (sums of
// Eq. energysum, renormalisation, symmetry re-imposition, convergence test
// on the binding energy, Secs. III-V) and update steps (Eq. updateeq) --
// until every lattice has converged or max_steps is reached.
//
// Work is split into phases separated by a grid-wide barrier: SUMS (one item
// per 64 x 16 tile column of each active lattice), FINALIZE (one lattice per
// block), SCALE (renormalise + symmetry, out of place), and STEP (one item
// per tile x z-chunk, K update steps through the TMA pipeline of
// tma_item.cuh).  Items are dealt to blocks round-robin over the active
// lattices; converged lattices drop out.  The per-site arithmetic and the
// reduction order are those of the one-lattice path, so every lattice ends
// bit-identical to a separate fdtd_evolve of the same lattice.
//
// The grid barrier is a sense-reversing counter in global memory; every wait
// on it is bounded in wall-clock time, after which the block sets the error
// flag and leaves (the others then give up at their next wait).
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tma_item.cuh"

namespace fdtd {

namespace {

constexpr int kTXB = 64;      // tile width of the batched stencil items
static_assert(kTXB == tb::kSumsTX, "the batched sums use the one-lattice sums partition");
constexpr int kMaxLat = 256;  // lattices per batched handle

}  // namespace

// Device table entry of one lattice (written by the host before the launch).
struct alignas(64) BatchLat {
  CUtensorMap step_map[3][3];  // [depth-1][psi0, psi1, V], tile width kTXB
  CUtensorMap sums_map[3];     // [psi0, psi1, V]
  float* psi[2];
  double* partials;
  LatState* state;
  double* hist;  // check history ring (kHistCap records)
  int n, mask, step_zc, cur;
  float hd, om6c, cc, a_f, kfac_f;
  int pad;
  double a3, v_inf;
};

struct BatchRun {
  int64_t max_steps, t_start, t_end;
  double tol;
  int check_every, tol_rel, reimpose, depth, nlat, skip_first, check0, pad;
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

// lattice of a global item index (prefix[] has nlat + 1 entries)
__device__ __forceinline__ int find_lattice(const int* prefix, int nlat, int item) {
  int lo = 0, hi = nlat - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Check of Secs. III-V on the block's lattice, same order as k_finalize.
__device__ void finalize_lattice(const BatchLat& L, int nparts, int check_id, int64_t t, const BatchRun& run) {
  __shared__ double sm[4][256];
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

template <int K>
__device__ __forceinline__ void step_item(char* smem, const BatchLat& L, int cur, int local, int32_t* err, bool& ok) {
  const int gx = (L.n + kTXB - 1) / kTXB, gy = (L.n + tb::TY - 1) / tb::TY;
  const int bx = local % gx, by = (local / gx) % gy, bz = local / (gx * gy);
  const int z0 = bz * L.step_zc;
  ok = tb::tma_step_item<K, kTXB>(smem, &L.step_map[K - 1][cur], &L.step_map[K - 1][2], L.psi[cur ^ 1], L.n,
                                  bx * kTXB, by * tb::TY, z0, min(z0 + L.step_zc, L.n), L.hd, L.om6c, L.cc, err) &&
       ok;
}

template <int KMAX>
__global__ void __launch_bounds__(tb::Geo<KMAX, kTXB>::THREADS) k_batched(const BatchLat* __restrict__ lats,
                                                                          BatchRun* run, int32_t* err) {
  extern __shared__ __align__(128) char smem_raw[];
  char* smem = tb::aligned_smem(smem_raw);
  __shared__ int pre_sums[kMaxLat + 1], pre_step[kMaxLat + 1], s_cur[kMaxLat], s_act[kMaxLat];
  const int nlat = run->nlat;
  const int64_t max_steps = run->max_steps;
  const int ce = run->check_every;
  if (threadIdx.x == 0) {
    int a = 0, b = 0;
    for (int l = 0; l < nlat; ++l) {
      pre_sums[l] = a;
      pre_step[l] = b;
      const int n = lats[l].n;
      const int tiles64 = ((n + kTXB - 1) / kTXB) * ((n + tb::TY - 1) / tb::TY);
      a += tb::sums_items(n);
      b += tiles64 * ((n + lats[l].step_zc - 1) / lats[l].step_zc);
      s_cur[l] = lats[l].cur;
      s_act[l] = lats[l].state->active;  // a lattice that converged in an earlier slice stays retired
    }
    pre_sums[nlat] = a;
    pre_step[nlat] = b;
  }
  __syncthreads();
  bool ok = true;
  const int64_t t_start = run->t_start, t_end = run->t_end;
  int64_t t = t_start;
  int check_id = run->check0;
  for (;;) {
    if ((t % ce == 0 || t == max_steps) && !(run->skip_first && t == t_start)) {
      // ---- SUMS
      for (int it = blockIdx.x; it < pre_sums[nlat] && ok; it += gridDim.x) {
        const int l = find_lattice(pre_sums, nlat, it);
        if (!s_act[l]) continue;
        const BatchLat& L = lats[l];
        const int local = it - pre_sums[l];
        const int gx = (L.n + kTXB - 1) / kTXB, gy = (L.n + tb::TY - 1) / tb::TY;
        const int zc = tb::sums_zchunk(L.n), z0 = (local / (gx * gy)) * zc;
        ok = tb::tma_sums_item<kTXB>(smem, &L.sums_map[s_cur[l]], &L.sums_map[2], L.n, (local % gx) * kTXB,
                                     ((local / gx) % gy) * tb::TY, z0, min(z0 + zc, L.n), L.a_f, L.kfac_f,
                                     L.partials + (size_t)local * 4, err);
      }
      if (!ok || !grid_barrier(run, err)) return;
      // ---- FINALIZE
      for (int l = blockIdx.x; l < nlat; l += gridDim.x) {
        if (!s_act[l]) continue;
        const int n = lats[l].n;
        finalize_lattice(lats[l], tb::sums_items(n), check_id, t, *run);
      }
      if (!grid_barrier(run, err)) return;
      // ---- SCALE: out = P(scale * in) for lattices checked now (sites dealt grid-wide)
      for (int l = 0; l < nlat; ++l) {
        if (!s_act[l]) continue;
        const BatchLat& L = lats[l];
        const LatState* st = L.state;
        if (*(volatile const int32_t*)&st->scale_seq != check_id) continue;
        const float scale = (float)*(volatile const double*)&st->scale;
        const int mask = run->reimpose ? L.mask : 0;
        const int n = L.n;
        const float* in = L.psi[s_cur[l]];
        float* out = L.psi[s_cur[l] ^ 1];
        // rows (y, z) dealt to the grid's warps, x along the lanes
        const int lane = threadIdx.x & 31, nwarps = (gridDim.x * blockDim.x) >> 5;
        for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n * n; r += nwarps) {
          const int y0 = r % n, z0 = r / n;
          for (int x0 = lane; x0 < n; x0 += 32) {
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
            out[((size_t)z0 * n + y0) * n + x0] = scale_site(in[site_index(c[0], c[1], c[2], n)], scale, neg, zero);
          }
        }
      }
      if (!grid_barrier(run, err)) return;
      // every block updates its view of the lattices identically
      if (threadIdx.x == 0) {
        for (int l = 0; l < nlat; ++l) {
          if (!s_act[l]) continue;
          const LatState* st = lats[l].state;
          if (*(volatile const int32_t*)&st->scale_seq == check_id) s_cur[l] ^= 1;
          s_act[l] = *(volatile const int32_t*)&st->active;
          if (blockIdx.x == 0) lats[l].state->cur = s_cur[l];
        }
      }
      __syncthreads();
      ++check_id;
      int any = 0;
      for (int l = 0; l < nlat; ++l) any |= s_act[l];
      if (t >= t_end || !any) break;
    }
    // ---- STEP: up to the next check, KMAX steps per phase
    const int64_t nc = (t / ce + 1) * ce;
    const int64_t next = nc < t_end ? nc : t_end;
    while (t < next) {
      const int k = (int)((next - t) < KMAX ? (next - t) : KMAX);
      for (int it = blockIdx.x; it < pre_step[nlat] && ok; it += gridDim.x) {
        const int l = find_lattice(pre_step, nlat, it);
        if (!s_act[l]) continue;
        const int local = it - pre_step[l];
        if (k == 1)
          step_item<1>(smem, lats[l], s_cur[l], local, err, ok);
        else if (k == 2)
          step_item<(KMAX >= 2 ? 2 : 1)>(smem, lats[l], s_cur[l], local, err, ok);
        else
          step_item<KMAX>(smem, lats[l], s_cur[l], local, err, ok);
      }
      if (!ok || !grid_barrier(run, err)) return;
      if (threadIdx.x == 0)
        for (int l = 0; l < nlat; ++l)
          if (s_act[l]) s_cur[l] ^= 1;
      __syncthreads();
      t += k;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    run->steps_done = t;
    for (int l = 0; l < nlat; ++l) lats[l].state->cur = s_cur[l];
  }
}

template <int KMAX>
size_t batched_smem() {
  size_t a = tb::Geo<KMAX, kTXB>::SMEM;
  size_t b = tb::Geo<1, kTXB>::SMEM + 8 * 4 * (tb::Geo<KMAX, kTXB>::THREADS / 32);  // sums item + reduction
  return a > b ? a : b;
}

}  // namespace

// Host side: fill the device table and launch the persistent kernel once
// (cooperative, so every block is resident and the grid barrier can complete).
int batched_max_lattices() { return kMaxLat; }

int batched_fill(void* host_entry, const float* psi0, const float* psi1, const float* v, double* partials,
                 LatState* state, double* hist, const Params& p, int mask, int cur, double v_inf, int zc) {
  BatchLat& B = *(BatchLat*)host_entry;
  int bw, bh;
  const float* bufs[3] = {psi0, psi1, v};
  for (int k = 1; k <= 3; ++k) {
    tma_box(k, kTXB, &bw, &bh);
    for (int b = 0; b < 3; ++b)
      if (encode_field_map(&B.step_map[k - 1][b], bufs[b], p.n, bw, bh)) return -1;
  }
  tma_box(1, kTXB, &bw, &bh);
  for (int b = 0; b < 3; ++b)
    if (encode_field_map(&B.sums_map[b], bufs[b], p.n, bw, bh)) return -1;
  B.psi[0] = (float*)psi0;
  B.psi[1] = (float*)psi1;
  B.partials = partials;
  B.state = state;
  B.hist = hist;
  B.n = p.n;
  B.mask = mask;
  B.step_zc = zc < p.n ? zc : p.n;
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

size_t batched_entry_bytes() { return sizeof(BatchLat); }
size_t batched_run_offset(int count) { return (size_t)count * sizeof(BatchLat); }

void BatchedGraphs::release() {
  for (int d = 0; d < 4; ++d) {
    if (exec[d]) cudaGraphExecDestroy(exec[d]);
    exec[d] = nullptr;
    grid[d] = 0;
  }
}

int batched_launch(void* dev_table, int count, int64_t max_steps, int64_t t_start, int64_t t_end, int skip_first,
                   int check0, int check_every, double tol, int tol_rel, int reimpose, int depth, int32_t* err,
                   cudaStream_t st, BatchedGraphs* graphs, int64_t* steps_done, int* grid_out) {
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
  BatchRun* drun = (BatchRun*)((char*)dev_table + batched_run_offset(count));
  cudaMemcpyAsync(drun, &run, sizeof(run), cudaMemcpyHostToDevice, st);
  depth = depth < 1 ? 1 : (depth > 3 ? 3 : depth);
  if (!graphs->exec[depth]) {
    // capture the cooperative launch once: grid = resident blocks of the whole device
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const BatchLat* tab = (const BatchLat*)dev_table;
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
      if (e == cudaSuccess) e = cudaGraphInstantiate(&graphs->exec[depth], g, 0);
      if (g) cudaGraphDestroy(g);
      cudaStreamDestroy(cs);
      if (e != cudaSuccess) {
        graphs->exec[depth] = nullptr;
        return e;
      }
      graphs->grid[depth] = grid;
      return cudaSuccess;
    };
    cudaError_t e;
    if (depth == 1)
      e = capture(k_batched<1>, tb::Geo<1, kTXB>::THREADS, batched_smem<1>());
    else if (depth == 2)
      e = capture(k_batched<2>, tb::Geo<2, kTXB>::THREADS, batched_smem<2>());
    else
      e = capture(k_batched<3>, tb::Geo<3, kTXB>::THREADS, batched_smem<3>());
    if (e != cudaSuccess) {
      cudaGetLastError();
      return (int)e;
    }
  }
  *grid_out = graphs->grid[depth];
  cudaError_t e = cudaGraphLaunch(graphs->exec[depth], st);
  if (e != cudaSuccess) return (int)e;
  cudaMemcpyAsync(steps_done, &drun->steps_done, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  return 0;
}

}  // namespace fdtd
