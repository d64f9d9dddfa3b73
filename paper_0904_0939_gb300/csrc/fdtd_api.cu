// C ABI of the FDTD solver (declared in include/fdtd.h): argument checks,
// workspace carving, and the host-side drivers that enqueue the kernels of
// k_core.cu / k_tblock.cu / k_adjoint.cu / k_batched.cu on the caller's stream.
//
// The library never allocates device memory: every buffer is a slice of the
// caller's workspace.  Per lattice the workspace holds two psi fields
// (ping-pong), V (plus A and cB for FP64 lattices), the block partials of
// the lattice sums, two state records, and -- when backward storage was
// requested -- the start field, the sqrt(T) checkpoint pool, one segment of
// recomputed fields, two adjoint fields and the FP64 gradient accumulator.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fdtd.h"
#include "kernels.cuh"

using namespace fdtd;

namespace {

thread_local std::string g_create_err;

constexpr size_t kStagingBytes = 8u << 20;

size_t elem_bytes(int prec) { return prec == FDTD_F64 ? 8 : (prec == FDTD_F32 ? 4 : 2); }

struct Lat {
  fdtd_lattice_desc d{};
  Params p{};
  size_t n3 = 0;
  int es = 0;
  void* psi[2] = {nullptr, nullptr};
  int cur = 0;
  void* v = nullptr;
  double* coefA = nullptr;
  double* coefCB = nullptr;
  double* partials = nullptr;
  int nparts = 0;
  LatState* state = nullptr;    // [0] evolve record, [1] scratch
  double* hist = nullptr;       // check history ring of the evolve (kHistCap records)
  int mask = 0;
  bool has_v = false, has_psi = false, has_psi0 = false;
  // backward storage
  void* psi0 = nullptr;
  int64_t bw_T = 0;
  int bw_K = 0;
  int64_t bw_npool = 0;
  void* pool = nullptr;
  void* seg = nullptr;
  void* lam[2] = {nullptr, nullptr};
  void* bw_u = nullptr;    // B lam of the split adjoint step
  void* bw_raw = nullptr;  // step outputs before a check (and the segment's last output)
  int bw_nraw = 0;
  double* gv = nullptr;
  double* scales = nullptr;
  // snapshots (Sec. III) and the scratch of the snapshot algebra
  void* snaps = nullptr;
  int nsnap = 0;
  double* dot_parts = nullptr;
  double* coef = nullptr;
  // last evolve
  int64_t last_steps = 0;
  LatState host_state{};
  // TMA descriptors of psi[0], psi[1], V: stencil boxes per tile width
  // (64, 128) and depth 1..3, and the sums boxes
  bool tma_ok = false;
  CUtensorMap maps[2][3][3];
  CUtensorMap sums_maps[3];
  // stencil configuration: depth, tile width, z-planes per block (0 = not chosen yet);
  // plain = the one-step z-marching kernel (bit-identical) was timed fastest
  int depth = 0, tx = 128, zc = 0;
  bool plain = false;
  // evolve graphs: a while loop over pairs of (check, check_every steps),
  // one per start buffer (an evolve ends on either), each built for a mask,
  // stencil configuration and cadence
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
  int64_t graph_key[2][6] = {{-1, -1, -1, -1, -1, -1}, {-1, -1, -1, -1, -1, -1}};
  int64_t graph_kernels = 0;  // kernels per loop iteration
};

void release_graph(Lat& L, int b) {
  if (L.graph_exec[b]) cudaGraphExecDestroy(L.graph_exec[b]);
  if (L.graph[b]) cudaGraphDestroy(L.graph[b]);
  L.graph_exec[b] = nullptr;
  L.graph[b] = nullptr;
  L.graph_key[b][0] = -1;
}
void release_graph(Lat& L) {
  release_graph(L, 0);
  release_graph(L, 1);
}

struct Carve {
  char* base = nullptr;
  size_t off = 0;
  void* take(size_t bytes) {
    off = (off + 255) & ~size_t(255);
    void* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  }
};

int check_desc(const fdtd_lattice_desc& d, std::string& err) {
  if (d.n < 1 || d.n > 2048) {
    err = "lattice n must be in [1, 2048]";
    return FDTD_ERR_INVALID_ARG;
  }
  if (d.precision != FDTD_F64 && d.precision != FDTD_F32 && d.precision != FDTD_BF16) {
    err = "unknown precision";
    return FDTD_ERR_INVALID_ARG;
  }
  if (!(d.length > 0.0) || !std::isfinite(d.length) || !(d.mass > 0.0) || !std::isfinite(d.mass) ||
      !(d.dtau >= 0.0) || !std::isfinite(d.dtau) || !std::isfinite(d.v_inf)) {
    err = "length and mass must be positive and finite, dtau >= 0";
    return FDTD_ERR_INVALID_ARG;
  }
  double a = d.length / d.n;
  double dt = d.dtau > 0.0 ? d.dtau : a * a / 4.0;
  if (!(dt < d.mass * a * a / 3.0)) {
    err = "dtau violates the von Neumann bound dtau < m a^2 / 3";
    return FDTD_ERR_UNSTABLE_DT;
  }
  return FDTD_OK;
}

int check_options(const fdtd_options& o, std::string& err) {
  if (o.check_every < 1) {
    err = "check_every must be >= 1";
    return FDTD_ERR_INVALID_ARG;
  }
  if (o.temporal_depth < 0 || o.temporal_depth > blocked_max_depth()) {
    err = "temporal_depth out of range";
    return FDTD_ERR_INVALID_ARG;
  }
  if (o.zchunk < 0) {
    err = "zchunk must be >= 0";
    return FDTD_ERR_INVALID_ARG;
  }
  if (o.autotune < 0 || o.autotune > 1) {
    err = "autotune must be 0 or 1";
    return FDTD_ERR_INVALID_ARG;
  }
  if (o.stencil_kernel < 0 || o.stencil_kernel > 1) {
    err = "stencil_kernel must be 0 or 1";
    return FDTD_ERR_INVALID_ARG;
  }
  if (o.snapshots < 0 || o.snapshots > 1024) {
    err = "snapshots must be in [0, 1024]";
    return FDTD_ERR_INVALID_ARG;
  }
  if (o.graphs != 0 && o.graphs != 1) {
    err = "graphs must be 0 or 1";
    return FDTD_ERR_INVALID_ARG;
  }
  if (o.boundary != 0 && o.boundary != 1) {
    err = "boundary must be 0 (zero) or 1 (periodic)";
    return FDTD_ERR_INVALID_ARG;
  }
  if (o.boundary == 1 && o.batched) {
    err = "batched mode needs zero boundaries";
    return FDTD_ERR_INVALID_ARG;
  }
  if (o.backward_steps < 0 || !std::isfinite(o.tol)) {
    err = "backward_steps must be >= 0 and tol finite";
    return FDTD_ERR_INVALID_ARG;
  }
  return FDTD_OK;
}

Params make_params(const fdtd_lattice_desc& d, int periodic) {
  Params p{};
  p.periodic = periodic ? 1 : 0;
  p.n = d.n;
  p.a = d.length / d.n;
  p.dtau = d.dtau > 0.0 ? d.dtau : p.a * p.a / 4.0;
  p.mass = d.mass;
  p.c = p.dtau / (2.0 * p.mass * p.a * p.a);
  p.half_dtau_f = (float)(0.5 * p.dtau);
  p.c_f = (float)p.c;
  p.one_m6c_f = (float)(1.0 - 6.0 * p.c);
  return p;
}

// Carve (or, with base == nullptr, measure) the workspace of every lattice.
void layout(const fdtd_lattice_desc* d, int count, const fdtd_options& o, Carve& cv, std::vector<Lat>* lats,
            void** staging, int32_t** flags, void** batch_ws, size_t* batch_bytes) {
  *staging = cv.take(kStagingBytes);
  *flags = (int32_t*)cv.take(256);
  for (int l = 0; l < count; ++l) {
    Lat L;
    L.d = d[l];
    L.p = make_params(d[l], o.boundary);
    L.n3 = (size_t)d[l].n * d[l].n * d[l].n;
    L.es = (int)elem_bytes(d[l].precision);
    L.psi[0] = cv.take(L.n3 * L.es);
    L.psi[1] = cv.take(L.n3 * L.es);
    if (d[l].precision == FDTD_F64) {
      L.v = cv.take(L.n3 * 8);
      L.coefA = (double*)cv.take(L.n3 * 8);
      L.coefCB = (double*)cv.take(L.n3 * 8);
    } else {
      L.v = cv.take(L.n3 * 4);
    }
    L.nparts = std::max(sums_blocks(d[l].n), tma_sums_blocks(d[l].n));
    L.partials = (double*)cv.take((size_t)L.nparts * 4 * sizeof(double));
    L.state = (LatState*)cv.take(2 * sizeof(LatState));
    L.hist = (double*)cv.take((size_t)kHistCap * kHistFields * sizeof(double));
    if (o.backward_steps > 0 && d[l].precision != FDTD_BF16) {
      L.bw_T = o.backward_steps;
      L.bw_K = (int)std::ceil(std::sqrt((double)o.backward_steps));
      L.bw_npool = (L.bw_T + L.bw_K - 1) / L.bw_K;
      L.psi0 = cv.take(L.n3 * L.es);
      L.pool = cv.take((size_t)L.bw_npool * L.n3 * L.es);
      L.seg = cv.take((size_t)L.bw_K * L.n3 * L.es);
      L.lam[0] = cv.take(L.n3 * L.es);
      L.lam[1] = cv.take(L.n3 * L.es);
      L.bw_u = cv.take(L.n3 * L.es);
      L.bw_nraw = (L.bw_K - 1) / o.check_every + 2;  // check steps inside a segment + its last step
      L.bw_raw = cv.take((size_t)L.bw_nraw * L.n3 * L.es);
      L.gv = (double*)cv.take(L.n3 * 8);
      L.scales = (double*)cv.take((size_t)(L.bw_T / o.check_every + 2) * sizeof(double));
    }
    if (o.snapshots > 0) {
      L.nsnap = o.snapshots;
      L.snaps = cv.take((size_t)L.nsnap * L.n3 * L.es);
    }
    L.dot_parts = (double*)cv.take((size_t)152 * 8 * 2 * sizeof(double));
    L.coef = (double*)cv.take(8 * sizeof(double));
    if (lats) lats->push_back(L);
  }
  *batch_bytes = o.batched ? batched_workspace_bytes(d, count) : 0;
  *batch_ws = o.batched ? cv.take(*batch_bytes) : nullptr;
}

}  // namespace

namespace fdtd {
// Message for fdtd_last_error(NULL) from entry points that take no handle.
void set_detached_error(const std::string& msg) { g_create_err = msg; }
}  // namespace fdtd

struct fdtd_context {
  std::vector<Lat> lats;
  fdtd_options o{};
  cudaStream_t st = nullptr;
  int device = 0;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  void* staging = nullptr;
  int32_t* flags = nullptr;
  void* batch_ws = nullptr;
  size_t batch_bytes = 0;
  std::string err;
  fdtd_stats stats{};
  bool profiling = false;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  int check_seq = 0;
  BatchedGraphs batch_graphs;     // graphs of the batched persistent launch
  int batch_depth = 0, batch_zc = 0;  // configuration of the last batched evolve
  cudaStream_t cap_st = nullptr;  // private stream the evolve graphs are captured and launched on
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;  // order cap_st after / before the handle's stream
  // stencil launches not yet credited to the stats: a launch enqueued past
  // the check at which its lattice converged runs as a no-op and is dropped
  struct Pending {
    int64_t t_start, updates;
    double bytes;
    long ev;  // index of its start event, or -1
  };
  std::vector<Pending> pending;
};

namespace {

// NVTX range for profilers (header-only NVTX3: no cost without a tool attached)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

int fail(fdtd_context* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_check(fdtd_context* c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, FDTD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return FDTD_OK;
}

int lat_check(fdtd_context* c, int lat) {
  if (!c) return FDTD_ERR_INVALID_ARG;
  if (lat < 0 || lat >= (int)c->lats.size()) return fail(c, FDTD_ERR_INVALID_ARG, "lattice index out of range");
  return FDTD_OK;
}

// ---- profiling of the stencil launches --------------------------------------
long prof_begin(fdtd_context* c) {
  if (!c->profiling) return -1;
  while (c->ev.size() < c->ev_used + 2) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->ev.push_back(e);
  }
  cudaEventRecord(c->ev[c->ev_used], c->st);
  return (long)c->ev_used;
}
void prof_end(fdtd_context* c) {
  if (!c->profiling) return;
  cudaEventRecord(c->ev[c->ev_used + 1], c->st);
  c->ev_used += 2;
}
// Credit the pending stencil launches that started before step `cutoff`
// (call after a stream synchronisation).
void flush_pending(fdtd_context* c, int64_t cutoff) {
  for (const auto& p : c->pending) {
    if (p.t_start >= cutoff) continue;
    c->stats.stencil_launches += 1;
    c->stats.stencil_site_updates += p.updates;
    c->stats.stencil_bytes += p.bytes;
    float ms = 0.f;
    if (p.ev >= 0 && cudaEventElapsedTime(&ms, c->ev[p.ev], c->ev[p.ev + 1]) == cudaSuccess) {
      c->stats.stencil_ms += ms;
      c->stats.stencil_timed_launches += 1;
    }
  }
  c->pending.clear();
  c->ev_used = 0;
}
void prof_collect(fdtd_context* c) { flush_pending(c, INT64_MAX); }

// ---- typed dispatch helpers ---------------------------------------------------
template <typename F>
void with_type(int prec, F&& f) {
  if (prec == FDTD_F64)
    f((double*)nullptr);
  else if (prec == FDTD_F32)
    f((float*)nullptr);
  else
    f((__nv_bfloat16*)nullptr);
}

// ---- autotuning of the stencil configuration ---------------------------------
// Fastest (depth, z-chunk) per (n, precision, device), shared by all handles.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, std::tuple<int, int, int, bool>> g_tune;

void choose_config(fdtd_context* c, Lat& L) {
  if (L.depth) return;
  const bool tma = L.tma_ok && c->o.stencil_kernel == 0;
  L.plain = false;
  if (!tma) {
    L.depth = 1;
    L.tx = 128;
    L.zc = 0;
    L.plain = true;
    return;
  }
  if (c->o.temporal_depth > 0 || !c->o.autotune) {
    L.depth = c->o.temporal_depth > 0 ? c->o.temporal_depth : auto_depth(L.d.n, L.d.precision);
    L.tx = L.d.n > 64 ? 128 : 64;
    L.zc = c->o.zchunk > 0 ? c->o.zchunk : tma_zchunk(L.d.n, L.depth, L.tx);
    return;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  auto key = std::make_tuple(L.d.n, L.d.precision, dev);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      std::tie(L.depth, L.tx, L.zc, L.plain) = it->second;
      return;
    }
  }
  Range r("stencil autotune");
  // time each candidate (every one of them is bit-identical):
  // psi[cur] -> psi[1-cur], psi[cur] is only read
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int n = L.d.n;
  double best = 0.0;
  int bd = auto_depth(n, L.d.precision), bt = n > 64 ? 128 : 64, bz = tma_zchunk(n, bd, bt);
  bool bp = false;
  auto time_it = [&](auto&& launch, int depth) {
    launch();
    const int reps = 3;
    cudaEventRecord(e0, c->st);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1, c->st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    c->stats.launches += reps + 1;
    return (double)L.n3 * depth * reps / (ms > 0.f ? ms : 1e-6);
  };
  // the plain one-step kernel
  {
    double rate = time_it(
        [&]() {
          launch_step_f32<float>((const float*)L.psi[L.cur], (float*)L.psi[1 - L.cur], (const float*)L.v, L.p,
                                 nullptr, c->st);
        },
        1);
    best = rate;
    bd = 1;
    bp = true;
  }
  for (int ti = 0; ti < 2; ++ti) {
    const int tx = ti ? 128 : 64;
    if (tx == 128 && n <= 64) continue;
    for (int d = 1; d <= blocked_max_depth(); ++d) {
      // spans: z-chunks n / 2^i (depth 1 repeats no planes, deeper levels
      // repeat 2(d-1) per item, so short chunks only for depth 1) and the
      // spans that fill the resident blocks in one, two or three waves
      std::vector<int> spans;
      for (int div = 1; div <= 128; div *= 2) {
        const int zc = (n + div - 1) / div;
        if (zc >= (d == 1 ? 2 : std::max(8, 4 * d))) spans.push_back(zc);
      }
      const long long total = tma_tile_planes(n, tx), slots = tma_resident_blocks(d, tx);
      for (int m = 1; m <= 3; ++m) spans.push_back((int)std::max(1LL, (total + m * slots - 1) / (m * slots)));
      std::sort(spans.begin(), spans.end());
      spans.erase(std::unique(spans.begin(), spans.end()), spans.end());
      for (int zc : spans) {
        double rate = time_it(
            [&]() {
              launch_step_tma(L.maps[ti][d - 1][L.cur], L.maps[ti][d - 1][2], (float*)L.psi[1 - L.cur], L.p, d, tx,
                              zc, nullptr, c->flags + 1, c->st);
            },
            d);
        if (rate > best) {
          best = rate;
          bd = d;
          bt = tx;
          bz = zc;
          bp = false;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int32_t err = 0;
  cudaMemcpy(&err, c->flags + 1, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (err) {  // the timed launches did no work: keep the heuristic, cache nothing
    L.depth = auto_depth(n, L.d.precision);
    L.tx = n > 64 ? 128 : 64;
    L.zc = tma_zchunk(n, L.depth, L.tx);
    return;
  }
  L.depth = bd;
  L.tx = bt;
  L.zc = bz;
  L.plain = bp;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = std::make_tuple(bd, bt, bz, bp);
}

// Enqueue `count` update steps of lattice L (psi[cur] -> ... ; cur follows),
// the first of them being step t0 of the current evolve.
void run_steps(fdtd_context* c, Lat& L, int64_t count, const int32_t* active, int64_t t0 = 0) {
  const int prec = L.d.precision;
  choose_config(c, L);
  const bool tma = L.tma_ok && c->o.stencil_kernel == 0 && !L.plain;
  const int depth = tma ? L.depth : 1;
  while (count > 0) {
    int k = (int)std::min<int64_t>(count, depth);
    const long ev = prof_begin(c);
    if (prec == FDTD_F64) {
      launch_step_f64((const double*)L.psi[L.cur], (double*)L.psi[1 - L.cur], L.coefA, L.coefCB, L.p, active, c->st);
    } else if (prec == FDTD_F32) {
      if (tma)
        launch_step_tma(L.maps[L.tx == 128][k - 1][L.cur], L.maps[L.tx == 128][k - 1][2], (float*)L.psi[1 - L.cur],
                        L.p, k, L.tx, k == depth ? L.zc : 0, active, c->flags + 1, c->st);
      else
        launch_step_f32<float>((const float*)L.psi[L.cur], (float*)L.psi[1 - L.cur], (const float*)L.v, L.p, active,
                               c->st);
    } else {
      launch_step_f32<__nv_bfloat16>((const __nv_bfloat16*)L.psi[L.cur], (__nv_bfloat16*)L.psi[1 - L.cur],
                                     (const float*)L.v, L.p, active, c->st);
    }
    prof_end(c);
    c->stats.launches += 1;
    // algorithmic bytes: psi read + psi write + V (FP64: A and cB) read once per launch
    c->pending.push_back({t0, (int64_t)L.n3 * k, (double)L.n3 * (2.0 * L.es + (prec == FDTD_F64 ? 16.0 : 4.0)), ev});
    L.cur ^= 1;
    count -= k;
    t0 += k;
  }
}

int launch_sums_any(fdtd_context* c, Lat& L, const void* psi, const int32_t* active) {
  int np = 0;
  if (L.tma_ok && (psi == L.psi[0] || psi == L.psi[1])) {
    np = launch_sums_tma(L.sums_maps[psi == L.psi[1]], L.sums_maps[2], L.p, L.partials, active, c->flags + 1, c->st);
    c->stats.launches += 1;
    return np;
  }
  with_type(L.d.precision, [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    np = launch_sums<T>((const T*)psi, L.v, L.p, L.partials, active, c->st);
  });
  c->stats.launches += 1;
  return np;
}

void scale_parity_any(fdtd_context* c, Lat& L, const void* in, void* out, int mask, const LatState* s, int id,
                      int out_idx, LatState* sw) {
  with_type(L.d.precision, [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    launch_scale_parity<T>((const T*)in, (T*)out, L.d.n, mask, s, id, out_idx, sw, c->st);
  });
  c->stats.launches += 1;
}

// One check of Secs. III-V on psi[cur]: sums, finalize, renormalise + mask.
void enqueue_check(fdtd_context* c, Lat& L, int check_id, int64_t t) {
  int np = launch_sums_any(c, L, L.psi[L.cur], &L.state[0].active);
  launch_finalize(&L.state[0], L.partials, np, check_id, t, L.p, L.d.v_inf, c->o.tol, c->o.tol_relative, 1, c->st, 0,
                  0, nullptr, L.hist);
  c->stats.launches += 1;
  int mask = c->o.reimpose_parity ? L.mask : 0;
  scale_parity_any(c, L, L.psi[L.cur], L.psi[1 - L.cur], mask, &L.state[0], check_id, 1 - L.cur, &L.state[0]);
  L.cur ^= 1;
}

int read_state(fdtd_context* c, Lat& L) {
  int32_t err = 0;
  cudaMemcpyAsync(&L.host_state, &L.state[0], sizeof(LatState), cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(&err, c->flags + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st);
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return fail(c, FDTD_ERR_CUDA, std::string("evolve: ") + cudaGetErrorString(e));
  flush_pending(c, L.host_state.converged ? L.host_state.step : INT64_MAX);
  if (err) return fail(c, FDTD_ERR_TIMEOUT, "evolve: a bounded device-side wait expired in the stencil kernel");
  return FDTD_OK;
}

// The check of enqueue_check in device-sequenced form (inside the graph).
void enqueue_check_seq(fdtd_context* c, Lat& L, int64_t ce, cudaGraphConditionalHandle cond) {
  int np = launch_sums_any(c, L, L.psi[L.cur], &L.state[0].active);
  launch_finalize(&L.state[0], L.partials, np, 0, 0, L.p, L.d.v_inf, c->o.tol, c->o.tol_relative, 1, c->st, (int)ce,
                  cond, c->flags + 1, L.hist);
  c->stats.launches += 1;
  int mask = c->o.reimpose_parity ? L.mask : 0;
  scale_parity_any(c, L, L.psi[L.cur], L.psi[1 - L.cur], mask, &L.state[0], -1, 1 - L.cur, &L.state[0]);
  L.cur ^= 1;
}

// Stencil launches and algorithmic bytes of one check_every-step segment.
void segment_work(fdtd_context* c, const Lat& L, int64_t ce, int64_t* launches, double* bytes) {
  const bool tma = L.tma_ok && c->o.stencil_kernel == 0 && !L.plain;
  const int depth = tma ? L.depth : 1;
  *launches = (ce + depth - 1) / depth;
  *bytes = (double)*launches * L.n3 * (2.0 * L.es + (L.d.precision == FDTD_F64 ? 16.0 : 4.0));
}

// Build (or reuse) the evolve graph of lattice L for its current start
// buffer: a while node whose body is two (check, segment) pairs -- a segment
// flips the ping-pong buffers an odd number of times, a pair an even number,
// so the body is the same at every iteration.  Returns false if the graph
// cannot be made (the caller then uses the stream).
bool ensure_graph(fdtd_context* c, Lat& L, int64_t ce) {
  choose_config(c, L);  // autotuning synchronises: never inside a capture
  const int mask = c->o.reimpose_parity ? L.mask : 0;
  const int b = L.cur;
  const int64_t key[6] = {L.cur, mask, L.depth, L.zc, L.plain, ce};
  if (L.graph_exec[b] && std::equal(key, key + 6, L.graph_key[b])) return true;
  release_graph(L, b);
  Range r("evolve graph build");
  if (L.tma_ok && c->o.stencil_kernel == 0 && !L.plain && ce % L.depth)
    (void)tma_zchunk(L.d.n, (int)(ce % L.depth), L.tx);  // occupancy query outside the capture
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return false;
  cudaGraphConditionalHandle cond;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  cudaGraphNode_t node;
  if (cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    return false;
  }
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    return false;
  }
  cudaGraph_t body = np.conditional.phGraph_out[0];
  const int cur0 = L.cur;
  const int64_t launches0 = c->stats.launches;
  const size_t pending0 = c->pending.size();
  // capture on the private stream (the handle's stream may be the legacy
  // one, which cannot be captured); the graph is launched on the handle's
  if (!c->cap_st && cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
    c->cap_st = nullptr;
    cudaGraphDestroy(g);
    cudaGetLastError();
    return false;
  }
  cudaStream_t user_st = c->st;
  c->st = c->cap_st;
  bool ok = cudaStreamBeginCaptureToGraph(c->st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
            cudaSuccess;
  if (ok) {
    for (int rep = 0; rep < 2; ++rep) {
      enqueue_check_seq(c, L, ce, cond);
      run_steps(c, L, ce, &L.state[0].active, 0);
    }
    cudaGraph_t captured = nullptr;
    ok = cudaStreamEndCapture(c->st, &captured) == cudaSuccess && L.cur == cur0;
  }
  c->st = user_st;
  L.graph_kernels = c->stats.launches - launches0;
  c->stats.launches = launches0;
  c->pending.resize(pending0);
  L.cur = cur0;
  cudaGraphExec_t exec = nullptr;
  if (ok) ok = cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
  if (ok && !c->ev_in) {
    ok = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) == cudaSuccess;
  }
  if (ok) ok = cudaGraphUpload(exec, c->cap_st) == cudaSuccess;
  if (!ok) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    return false;
  }
  L.graph[b] = g;
  L.graph_exec[b] = exec;
  std::copy(key, key + 6, L.graph_key[b]);
  return true;
}

int evolve_one(fdtd_context* c, Lat& L, int64_t max_steps) {
  cudaMemsetAsync(c->flags + 1, 0, sizeof(int32_t), c->st);
  launch_state_reset(&L.state[0], 0, c->st);
  c->stats.launches += 1;
  const int64_t ce = c->o.check_every;
  int64_t t = 0;
  int check_id = 0;
  int groups = 2;
  bool done = false;
  if (c->o.graphs && c->profiling) {
    // the timed sample: two segments through the stream, every stencil
    // launch between CUDA events (a graph loop body cannot hold events)
    for (int i = 0; i < 2 && t + ce <= max_steps; ++i) {
      enqueue_check(c, L, check_id++, t);
      run_steps(c, L, ce, &L.state[0].active, t);
      t += ce;
    }
    int rc = cuda_check(c, "evolve launch");
    if (rc) return rc;
    if ((rc = read_state(c, L))) return rc;
    if (!L.host_state.active) done = true;
  }
  // full pairs of segments in one graph launch, the convergence check
  // ending the loop on the device
  const int64_t pairs = (!done && c->o.graphs) ? std::min<int64_t>((max_steps - t) / (2 * ce), 1 << 28) : 0;
  if (pairs > 0 && ensure_graph(c, L, ce)) {
    const int64_t t_end = t + 2 * pairs * ce;
    launch_state_reset(&L.state[0], 2, c->st, check_id + (int)(2 * pairs));
    c->stats.launches += 1;
    // launched on the private stream, ordered after and before the handle's
    // stream by events (a graph launched into the legacy stream paid about
    // half a millisecond per launch)
    cudaEventRecord(c->ev_in, c->st);
    cudaStreamWaitEvent(c->cap_st, c->ev_in, 0);
    cudaGraphLaunch(L.graph_exec[L.cur], c->cap_st);
    cudaEventRecord(c->ev_out, c->cap_st);
    cudaStreamWaitEvent(c->st, c->ev_out, 0);
    c->stats.graph_launches += 1;
    int rc = cuda_check(c, "evolve graph launch");
    if (rc) return rc;
    if ((rc = read_state(c, L))) return rc;
    const LatState& hs = L.host_state;
    c->stats.launches += (int64_t)((hs.checks - check_id + 1) / 2) * L.graph_kernels;
    const int64_t advanced = std::max<int64_t>(0, (hs.active ? t_end : hs.step) - t);  // steps taken while active
    int64_t seg_l;
    double seg_b;
    segment_work(c, L, ce, &seg_l, &seg_b);
    c->stats.stencil_launches += advanced / ce * seg_l;
    c->stats.stencil_site_updates += advanced * (int64_t)L.n3;
    c->stats.stencil_bytes += (double)(advanced / ce) * seg_b;
    if (!hs.active) {
      done = true;
    } else {
      t = t_end;
      check_id = hs.checks;
    }
  }
  int prev_checks = 0;
  double prev_delta = -1.0;
  while (!done) {
    for (int g = 0; g < groups && !done; ++g) {
      enqueue_check(c, L, check_id++, t);
      if (t >= max_steps) {
        done = true;
        break;
      }
      int64_t nst = std::min<int64_t>(ce, max_steps - t);
      run_steps(c, L, nst, &L.state[0].active, t);
      t += nst;
    }
    int rc = cuda_check(c, "evolve launch");
    if (rc) return rc;
    rc = read_state(c, L);
    if (rc) return rc;
    if (!L.host_state.active) done = true;
    // segments to enqueue before the next look: predicted from the decay of
    // |dE_b| per check, so that little work is queued past convergence
    const LatState& hs = L.host_state;
    int next = std::min(groups * 2, 32);
    if (c->o.tol > 0.0 && hs.delta_e > 0.0 && prev_delta > 0.0 && hs.checks > prev_checks) {
      const double rate = std::pow(hs.delta_e / prev_delta, 1.0 / (hs.checks - prev_checks));
      const double thr = c->o.tol * (c->o.tol_relative ? std::fabs(hs.ebind) : 1.0);
      if (rate < 0.999 && thr > 0.0) {
        double m = std::log(thr / hs.delta_e) / std::log(rate);
        next = (int)std::max(1.0, std::min(32.0, std::ceil(m)));
      }
    }
    prev_checks = hs.checks;
    prev_delta = hs.delta_e;
    groups = next;
  }
  if (L.host_state.status == STATUS_NONFINITE)
    return fail(c, FDTD_ERR_NONFINITE, "non-finite or vanishing norm during evolve");
  L.cur = L.host_state.cur;
  L.last_steps = L.host_state.converged ? L.host_state.step : max_steps;
  return FDTD_OK;
}

void fill_obs(const Lat& L, const LatState& s, fdtd_obs* out) {
  std::memset(out, 0, sizeof(*out));
  out->energy = s.energy;
  out->binding_energy = s.ebind;
  out->norm = s.s0 * L.p.a * L.p.a * L.p.a;
  out->r2 = s.r2;
  out->r_rms = std::sqrt(std::max(0.0, s.r2));
  out->v_expect = s.vexp;
  out->delta_e = s.delta_e;
}

// Copy n3 elements of dtype `dt` from user memory into a typed device
// buffer of lattice precision `prec` (through the staging buffer for host
// memory).
int import_field(fdtd_context* c, const void* src, int dt, int mem, void* dst, int prec, size_t n3) {
  const size_t isz = dt == FDTD_F64 ? 8 : 4;
  auto convert = [&](const void* s, size_t count, size_t off) {
    with_type(prec, [&](auto* tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      if (dt == FDTD_F64)
        launch_convert<double, T>((const double*)s, (T*)dst + off, count, c->st);
      else
        launch_convert<float, T>((const float*)s, (T*)dst + off, count, c->st);
    });
    c->stats.launches += 1;
  };
  if (mem == FDTD_MEM_DEVICE) {
    convert(src, n3, 0);
  } else {
    const size_t chunk = kStagingBytes / isz;
    for (size_t off = 0; off < n3; off += chunk) {
      size_t cnt = std::min(chunk, n3 - off);
      cudaMemcpyAsync(c->staging, (const char*)src + off * isz, cnt * isz, cudaMemcpyHostToDevice, c->st);
      convert(c->staging, cnt, off);
    }
  }
  return cuda_check(c, "import");
}

int export_field(fdtd_context* c, const void* src, int prec, void* dst, int dt, int mem, size_t n3) {
  const size_t osz = dt == FDTD_F64 ? 8 : 4;
  auto convert = [&](void* d, size_t count, size_t off) {
    with_type(prec, [&](auto* tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      if (dt == FDTD_F64)
        launch_convert<T, double>((const T*)src + off, (double*)d, count, c->st);
      else
        launch_convert<T, float>((const T*)src + off, (float*)d, count, c->st);
    });
    c->stats.launches += 1;
  };
  if (mem == FDTD_MEM_DEVICE) {
    convert(dst, n3, 0);
  } else {
    const size_t chunk = kStagingBytes / osz;
    for (size_t off = 0; off < n3; off += chunk) {
      size_t cnt = std::min(chunk, n3 - off);
      convert(c->staging, cnt, off);
      cudaMemcpyAsync((char*)dst + off * osz, c->staging, cnt * osz, cudaMemcpyDeviceToHost, c->st);
    }
  }
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return fail(c, FDTD_ERR_CUDA, std::string("export: ") + cudaGetErrorString(e));
  return cuda_check(c, "export");
}

// Batched configurations already chosen, by device and lattice sizes.
std::mutex g_btune_mu;
std::map<std::pair<int, std::vector<int>>, std::pair<int, int>> g_btune;

// All lattices of the handle in persistent launches.  With autotuning on
// (and no depth given) the first launches of a new set of lattice sizes are
// slices of 2 x check_every steps, one per (depth 1..3, z-chunk 16/32/64)
// candidate, timed with CUDA events; the fastest runs the rest in one
// launch.  Every candidate computes the same bits, so tuning costs no extra
// work, only launch boundaries.
int evolve_batched(fdtd_context* c, int64_t max_steps) {
  const int count = (int)c->lats.size();
  if (count > batched_max_lattices()) return fail(c, FDTD_ERR_INVALID_ARG, "evolve: too many lattices for batched mode");
  for (auto& L : c->lats)
    if (!L.tma_ok) return fail(c, FDTD_ERR_INVALID_ARG, "evolve: batched mode needs FP32 lattices with n % 4 == 0");
  const int64_t ce = c->o.check_every;
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<int> sizes;
  for (auto& L : c->lats) sizes.push_back(L.d.n);
  const auto key = std::make_pair(dev, sizes);
  std::vector<std::pair<int, int>> cands;  // (depth, z-chunk)
  if (c->o.temporal_depth > 0 || !c->o.autotune) {
    cands.push_back({c->o.temporal_depth > 0 ? c->o.temporal_depth : 2, c->o.zchunk > 0 ? c->o.zchunk : 32});
  } else {
    std::lock_guard<std::mutex> lock(g_btune_mu);
    auto it = g_btune.find(key);
    if (it != g_btune.end()) {
      cands.push_back(it->second);
    } else {
      for (int d = 1; d <= 3; ++d)
        for (int zc : {16, 32, 64}) cands.push_back({d, zc});
    }
  }
  const bool tuning = cands.size() > 1;
  for (auto& L : c->lats) {
    launch_state_reset(&L.state[0], 0, c->st);
    c->stats.launches += 1;
  }
  cudaMemsetAsync(c->flags + 1, 0, sizeof(int32_t), c->st);
  std::vector<char> table(batched_entry_bytes() * count + 64);
  char* base = table.data() + ((64 - ((uintptr_t)table.data() & 63)) & 63);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int64_t t = 0, steps = 0, slices = 0;
  double best_rate = -1.0;
  std::pair<int, int> best = cands[0];
  std::vector<int64_t> step_at(count, 0);  // steps each lattice advanced while active
  int rc = FDTD_OK;
  auto slice = [&](std::pair<int, int> cd, int64_t t_end) -> int {
    for (int l = 0; l < count; ++l) {
      Lat& L = c->lats[l];
      if (batched_fill(base + l * batched_entry_bytes(), (const float*)L.psi[0], (const float*)L.psi[1],
                       (const float*)L.v, L.partials, &L.state[0], L.hist, L.p, L.mask, L.cur, L.d.v_inf,
                       cd.second))
        return fail(c, FDTD_ERR_CUDA, "evolve: could not encode the batched tensor maps");
    }
    cudaMemcpyAsync(c->batch_ws, base, batched_entry_bytes() * count, cudaMemcpyHostToDevice, c->st);
    int grid = 0;
    cudaEventRecord(e0, c->st);
    int e = batched_launch(c->batch_ws, count, max_steps, t, t_end, t > 0, 0, (int)ce, c->o.tol, c->o.tol_relative,
                           c->o.reimpose_parity, cd.first, c->flags + 1, c->st, &c->batch_graphs, &steps, &grid);
    cudaEventRecord(e1, c->st);
    if (e) return fail(c, FDTD_ERR_CUDA, std::string("evolve (batched): ") + cudaGetErrorString((cudaError_t)e));
    c->stats.launches += 1;
    c->stats.graph_launches += 1;
    ++slices;
    int r = cuda_check(c, "evolve (batched)");
    if (r) return r;
    double upd = 0.0;
    for (int l = 0; l < count; ++l) {
      Lat& L = c->lats[l];
      const bool was_active = L.host_state.active || t == 0;
      if ((r = read_state(c, L))) return r;
      if (L.host_state.status == STATUS_NONFINITE)
        return fail(c, FDTD_ERR_NONFINITE, "non-finite or vanishing norm during evolve");
      L.cur = L.host_state.cur;
      if (was_active) {
        const int64_t upto = L.host_state.active ? steps : L.host_state.step;
        upd += (double)L.n3 * (double)std::max<int64_t>(0, upto - t);
        step_at[l] = std::max(step_at[l], upto);
      }
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (c->profiling) c->stats.stencil_ms += ms;
    const double rate = ms > 0.f ? upd / ms : 0.0;
    if (rate > best_rate) {
      best_rate = rate;
      best = cd;
    }
    t = steps;
    return FDTD_OK;
  };
  bool any = true;
  for (size_t i = 0; tuning && i < cands.size() && any && t < max_steps; ++i) {
    if ((rc = slice(cands[i], std::min<int64_t>(max_steps, t + 2 * ce)))) break;
    any = false;
    for (auto& L : c->lats) any |= L.host_state.active != 0;
  }
  if (!rc && tuning && best_rate > 0.0) {
    std::lock_guard<std::mutex> lock(g_btune_mu);
    g_btune[key] = best;
  }
  if (!rc && any && t < max_steps) rc = slice(best, max_steps);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  // the persistent launches are the stencil launches of a batched evolve
  for (int l = 0; l < count; ++l) {
    Lat& L = c->lats[l];
    L.last_steps = L.host_state.converged ? L.host_state.step : max_steps;
    c->stats.stencil_site_updates += (int64_t)L.n3 * step_at[l];
    c->stats.stencil_bytes += (double)L.n3 * 12.0 * ((step_at[l] + best.first - 1) / best.first);
  }
  c->stats.stencil_launches += slices;
  if (c->profiling) c->stats.stencil_timed_launches += slices;
  c->batch_depth = best.first;
  c->batch_zc = best.second;
  return FDTD_OK;
}

int valid_mask(int mask) {
  if (mask < 0 || mask >= 64) return 0;
  for (int ax = 0; ax < 3; ++ax)
    if (((mask >> (2 * ax)) & 3) == 3) return 0;
  return 1;
}

// ---- checkpoint files ---------------------------------------------------------
// 64-byte little-endian header followed by n^3 values (x fastest) of dtype.
struct PsiFileHeader {
  char magic[8];       // "FDTDPSI1"
  uint32_t version;    // 1
  int32_t n;
  int32_t dtype;       // FDTD_F64 or FDTD_F32
  int32_t mask;        // symmetry mask of the field
  double length, mass, dtau;
  int64_t step;        // steps of the evolve that produced it
  uint64_t checksum;   // FNV-1a (64 bit) of the data bytes
};
static_assert(sizeof(PsiFileHeader) == 64, "checkpoint header layout");
constexpr char kPsiMagic[8] = {'F', 'D', 'T', 'D', 'P', 'S', 'I', '1'};

// FNV-1a, 64-bit: offset basis 14695981039346656037, prime 1099511628211.
uint64_t fnv1a64(const unsigned char* p, size_t len) {
  uint64_t h = 14695981039346656037ull;
  for (size_t i = 0; i < len; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

void record_start(fdtd_context* c, Lat& L) {
  if (L.psi0) {
    cudaMemcpyAsync(L.psi0, L.psi[L.cur], L.n3 * L.es, cudaMemcpyDeviceToDevice, c->st);
    L.has_psi0 = true;
  }
}

}  // namespace

// =============================================================================
extern "C" {

int fdtd_default_options(fdtd_options* o) {
  if (!o) return FDTD_ERR_INVALID_ARG;
  std::memset(o, 0, sizeof(*o));
  o->check_every = 100;
  o->tol = 1e-6;
  o->tol_relative = 1;
  o->temporal_depth = 0;
  o->backward_steps = 0;
  o->batched = 0;
  o->reimpose_parity = 1;
  o->stencil_kernel = 0;
  o->autotune = 1;
  o->graphs = 1;
  return FDTD_OK;
}

int fdtd_workspace_size(const fdtd_lattice_desc* d, int count, const fdtd_options* o, size_t* bytes) {
  if (!d || count < 1 || !bytes) {
    g_create_err = "workspace_size: null descriptor/out or count < 1";
    return FDTD_ERR_INVALID_ARG;
  }
  fdtd_options oo;
  if (o)
    oo = *o;
  else
    fdtd_default_options(&oo);
  std::string err;
  int rc = check_options(oo, err);
  for (int l = 0; rc == FDTD_OK && l < count; ++l) rc = check_desc(d[l], err);
  if (rc) {
    g_create_err = err;
    return rc;
  }
  Carve cv;
  void* s;
  int32_t* f;
  void* bw;
  size_t bb;
  layout(d, count, oo, cv, nullptr, &s, &f, &bw, &bb);
  *bytes = cv.off + 256;
  return FDTD_OK;
}

int fdtd_create(const fdtd_lattice_desc* d, int count, const fdtd_options* o, void* ws, size_t ws_bytes,
                void* stream, fdtd_handle* out) {
  if (!out) {
    g_create_err = "create: null output handle";
    return FDTD_ERR_INVALID_ARG;
  }
  *out = nullptr;
  size_t need = 0;
  int rc = fdtd_workspace_size(d, count, o, &need);
  if (rc) return rc;
  if (!ws || ((uintptr_t)ws & 255) || ws_bytes < need) {
    g_create_err = "workspace null, not 256-byte aligned, or smaller than fdtd_workspace_size()";
    return FDTD_ERR_WORKSPACE;
  }
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, ws) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    g_create_err = "workspace is not device memory";
    return FDTD_ERR_WORKSPACE;
  }
  fdtd_context* c = new fdtd_context();
  if (o)
    c->o = *o;
  else
    fdtd_default_options(&c->o);
  c->st = (cudaStream_t)stream;
  c->ws = (char*)ws;
  c->ws_bytes = ws_bytes;
  cudaGetDevice(&c->device);
  Carve cv;
  cv.base = c->ws;
  layout(d, count, c->o, cv, &c->lats, &c->staging, &c->flags, &c->batch_ws, &c->batch_bytes);
  cudaMemsetAsync(c->flags, 0, 256, c->st);
  // flags[1]: error flag of the bounded device waits; flags[2]: their budget
  cudaMemcpyAsync(c->flags + 2, &c->o.wait_limit_us, sizeof(int32_t), cudaMemcpyHostToDevice, c->st);
  for (auto& L : c->lats) {
    launch_state_reset(&L.state[0], 1, c->st);
    launch_state_reset(&L.state[1], 1, c->st);
    c->stats.launches += 2;
    if (tma_supported(L.d.n, L.d.precision) && !L.p.periodic) {  // TMA boxes zero-fill
      const float* bufs[3] = {(const float*)L.psi[0], (const float*)L.psi[1], (const float*)L.v};
      bool ok = true;
      int bw, bh;
      for (int ti = 0; ti < 2; ++ti)
        for (int k = 1; k <= blocked_max_depth(); ++k) {
          tma_box(k, ti ? 128 : 64, &bw, &bh);
          for (int b = 0; b < 3; ++b) ok = ok && encode_field_map(&L.maps[ti][k - 1][b], bufs[b], L.d.n, bw, bh) == 0;
        }
      tma_box(1, 64, &bw, &bh);
      for (int b = 0; b < 3; ++b) ok = ok && encode_field_map(&L.sums_maps[b], bufs[b], L.d.n, bw, bh) == 0;
      L.tma_ok = ok;
    }
  }
  if (cuda_check(c, "create")) {
    g_create_err = c->err;
    delete c;
    return FDTD_ERR_CUDA;
  }
  *out = c;
  return FDTD_OK;
}

int fdtd_destroy(fdtd_handle h) {
  if (!h) return FDTD_ERR_INVALID_ARG;
  cudaStreamSynchronize(h->st);
  for (auto& L : h->lats) release_graph(L);
  h->batch_graphs.release();
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  for (auto e : h->ev) cudaEventDestroy(e);
  delete h;
  return FDTD_OK;
}

int fdtd_last_error(fdtd_handle h, char* buf, size_t n) {
  const std::string& m = h ? h->err : g_create_err;
  if (buf && n > 0) {
    const size_t k = std::min(n - 1, m.size());
    std::memcpy(buf, m.data(), k);
    buf[k] = '\0';
  }
  return (int)std::min<size_t>(m.size(), 0x7fffffff);
}

int fdtd_set_potential(fdtd_handle h, int lat, const void* v, int dtype, int mem_kind) {
  int rc = lat_check(h, lat);
  if (rc) return rc;
  if (!v || (dtype != FDTD_F64 && dtype != FDTD_F32) || (mem_kind != FDTD_MEM_HOST && mem_kind != FDTD_MEM_DEVICE))
    return fail(h, FDTD_ERR_INVALID_ARG, "set_potential: null pointer, bad dtype or mem_kind");
  Lat& L = h->lats[lat];
  cudaMemsetAsync(h->flags, 0, sizeof(int32_t), h->st);
  const size_t isz = dtype == FDTD_F64 ? 8 : 4;
  float* vf = L.d.precision == FDTD_F64 ? nullptr : (float*)L.v;
  double* vd = L.d.precision == FDTD_F64 ? (double*)L.v : nullptr;
  auto conv = [&](const void* src, size_t cnt, size_t off) {
    if (dtype == FDTD_F64)
      launch_set_potential<double>((const double*)src, cnt, off, vf, vd, L.coefA, L.coefCB, L.p, h->flags, h->st);
    else
      launch_set_potential<float>((const float*)src, cnt, off, vf, vd, L.coefA, L.coefCB, L.p, h->flags, h->st);
    h->stats.launches += 1;
  };
  if (mem_kind == FDTD_MEM_DEVICE) {
    conv(v, L.n3, 0);
  } else {
    const size_t chunk = kStagingBytes / isz;
    for (size_t off = 0; off < L.n3; off += chunk) {
      size_t cnt = std::min(chunk, L.n3 - off);
      cudaMemcpyAsync(h->staging, (const char*)v + off * isz, cnt * isz, cudaMemcpyHostToDevice, h->st);
      conv(h->staging, cnt, off);
    }
  }
  int32_t flags = 0;
  cudaMemcpyAsync(&flags, h->flags, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st);
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return fail(h, FDTD_ERR_CUDA, std::string("set_potential: ") + cudaGetErrorString(e));
  if ((rc = cuda_check(h, "set_potential"))) return rc;
  if (flags & 1) return fail(h, FDTD_ERR_NONFINITE, "set_potential: NaN or Inf in V");
  if (flags & 2) return fail(h, FDTD_ERR_UNSTABLE_DT, "set_potential: 1 + dtau V / 2 <= 0 at some site");
  L.has_v = true;
  return FDTD_OK;
}

int fdtd_init_symmetric(fdtd_handle h, int lat, uint64_t seed, int parity_mask, int dist) {
  int rc = lat_check(h, lat);
  if (rc) return rc;
  if (!valid_mask(parity_mask) || (dist != FDTD_DIST_UNIFORM && dist != FDTD_DIST_GAUSSIAN))
    return fail(h, FDTD_ERR_INVALID_ARG, "init_symmetric: bad parity mask or distribution");
  Lat& L = h->lats[lat];
  with_type(L.d.precision, [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    launch_init_random<T>((T*)L.psi[0], L.d.n, seed, (uint64_t)lat, dist, h->st);
  });
  h->stats.launches += 1;
  L.cur = 0;
  if (parity_mask) {
    scale_parity_any(h, L, L.psi[0], L.psi[1], parity_mask, nullptr, 0, 1, nullptr);
    L.cur = 1;
  }
  L.mask = parity_mask;
  L.has_psi = true;
  record_start(h, L);
  return cuda_check(h, "init_symmetric");
}

int fdtd_set_psi(fdtd_handle h, int lat, const void* psi, int dtype, int mem_kind, int parity_mask) {
  int rc = lat_check(h, lat);
  if (rc) return rc;
  if (!psi || (dtype != FDTD_F64 && dtype != FDTD_F32) ||
      (mem_kind != FDTD_MEM_HOST && mem_kind != FDTD_MEM_DEVICE) || !valid_mask(parity_mask))
    return fail(h, FDTD_ERR_INVALID_ARG, "set_psi: null pointer, bad dtype, mem_kind or mask");
  Lat& L = h->lats[lat];
  if ((rc = import_field(h, psi, dtype, mem_kind, L.psi[L.cur], L.d.precision, L.n3))) return rc;
  L.mask = parity_mask;
  L.has_psi = true;
  record_start(h, L);
  return cuda_check(h, "set_psi");
}

int fdtd_get_psi(fdtd_handle h, int lat, void* psi, int dtype, int mem_kind) {
  int rc = lat_check(h, lat);
  if (rc) return rc;
  if (!psi || (dtype != FDTD_F64 && dtype != FDTD_F32) || (mem_kind != FDTD_MEM_HOST && mem_kind != FDTD_MEM_DEVICE))
    return fail(h, FDTD_ERR_INVALID_ARG, "get_psi: null pointer, bad dtype or mem_kind");
  Lat& L = h->lats[lat];
  if (!L.has_psi) return fail(h, FDTD_ERR_STATE, "get_psi: no wavefunction yet");
  return export_field(h, L.psi[L.cur], L.d.precision, psi, dtype, mem_kind, L.n3);
}

int fdtd_save_psi(fdtd_handle h, int lat, const char* path) {
  Range r("fdtd_save_psi");
  int rc = lat_check(h, lat);
  if (rc) return rc;
  if (!path) return fail(h, FDTD_ERR_INVALID_ARG, "save_psi: null path");
  Lat& L = h->lats[lat];
  if (!L.has_psi) return fail(h, FDTD_ERR_STATE, "save_psi: no wavefunction yet");
  PsiFileHeader hd{};
  std::memcpy(hd.magic, kPsiMagic, 8);
  hd.version = 1;
  hd.n = L.d.n;
  hd.dtype = L.d.precision == FDTD_F64 ? FDTD_F64 : FDTD_F32;
  hd.mask = L.mask;
  hd.length = L.d.length;
  hd.mass = L.p.mass;
  hd.dtau = L.p.dtau;
  hd.step = L.last_steps;
  const size_t bytes = L.n3 * (hd.dtype == FDTD_F64 ? 8 : 4);
  std::vector<unsigned char> data(bytes);
  if ((rc = export_field(h, L.psi[L.cur], L.d.precision, data.data(), hd.dtype, FDTD_MEM_HOST, L.n3))) return rc;
  hd.checksum = fnv1a64(data.data(), bytes);
  std::FILE* f = std::fopen(path, "wb");
  if (!f) return fail(h, FDTD_ERR_IO, std::string("save_psi: cannot open ") + path);
  const bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 && std::fwrite(data.data(), 1, bytes, f) == bytes;
  const bool closed = std::fclose(f) == 0;
  if (!ok || !closed) return fail(h, FDTD_ERR_IO, std::string("save_psi: write failed for ") + path);
  return FDTD_OK;
}

int fdtd_load_psi(fdtd_handle h, int lat, const char* path) {
  Range r("fdtd_load_psi");
  int rc = lat_check(h, lat);
  if (rc) return rc;
  if (!path) return fail(h, FDTD_ERR_INVALID_ARG, "load_psi: null path");
  Lat& L = h->lats[lat];
  std::FILE* f = std::fopen(path, "rb");
  if (!f) return fail(h, FDTD_ERR_IO, std::string("load_psi: cannot open ") + path);
  PsiFileHeader hd{};
  std::vector<unsigned char> data;
  std::string why;
  if (std::fread(&hd, sizeof(hd), 1, f) != 1) {
    why = "shorter than its header";
  } else if (std::memcmp(hd.magic, kPsiMagic, 8) != 0 || hd.version != 1) {
    why = "not a wavefunction file of this format";
  } else if (hd.n < 1 || hd.n > 2048 || (hd.dtype != FDTD_F64 && hd.dtype != FDTD_F32) || !valid_mask(hd.mask) ||
             !(hd.length > 0.0) || !std::isfinite(hd.length)) {
    why = "header fields out of range";
  } else {
    const size_t bytes = (size_t)hd.n * hd.n * hd.n * (hd.dtype == FDTD_F64 ? 8 : 4);
    data.resize(bytes + 1);
    const size_t got = std::fread(data.data(), 1, bytes + 1, f);
    if (got != bytes)
      why = got < bytes ? "truncated" : "longer than its header says";
    else if (fnv1a64(data.data(), bytes) != hd.checksum)
      why = "checksum mismatch (corrupted data)";
    data.resize(bytes);
  }
  std::fclose(f);
  if (!why.empty()) return fail(h, FDTD_ERR_IO, std::string("load_psi: ") + path + ": " + why);
  if (std::fabs(hd.length - L.d.length) > 1e-12 * L.d.length)
    return fail(h, FDTD_ERR_SHAPE, "load_psi: the file's box length differs from the lattice's");
  int levels = 0;
  while ((hd.n << levels) < L.d.n) ++levels;
  if ((hd.n << levels) != L.d.n)
    return fail(h, FDTD_ERR_SHAPE, "load_psi: the lattice must have the file's n times a power of two");
  if (levels == 0) {  // same resolution: as fdtd_set_psi
    if ((rc = import_field(h, data.data(), hd.dtype, FDTD_MEM_HOST, L.psi[L.cur], L.d.precision, L.n3))) return rc;
  } else {
    // Sec. VII.G: the saved field is the start at a finer resolution.  Stage
    // it and every intermediate level in the spare buffer, transfer level by
    // level (the last into psi[cur]), then renormalise and re-impose its
    // symmetry as fdtd_upsample does.
    char* spare = (char*)L.psi[1 - L.cur];
    size_t off = 0;
    int nc = hd.n;
    const size_t n3c = (size_t)nc * nc * nc;
    if ((rc = import_field(h, data.data(), hd.dtype, FDTD_MEM_HOST, spare, L.d.precision, n3c))) return rc;
    for (int k = 0; k < levels; ++k) {
      const size_t in_off = off;
      const bool last = k == levels - 1;
      const size_t out_off = in_off + (size_t)nc * nc * nc;
      with_type(L.d.precision, [&](auto* tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        T* out = last ? (T*)L.psi[L.cur] : (T*)(spare + out_off * L.es);
        launch_upsample<T, T>((const T*)(spare + in_off * L.es), nc, out, L.p.periodic, h->st);
      });
      h->stats.launches += 1;
      off = out_off;
      nc *= 2;
    }
    const int id = 1000000 + (h->check_seq++);
    const int np = launch_sums_any(h, L, L.psi[L.cur], nullptr);
    launch_state_reset(&L.state[1], 0, h->st);
    launch_finalize(&L.state[1], L.partials, np, id, 0, L.p, L.d.v_inf, 0.0, 0, 0, h->st);
    scale_parity_any(h, L, L.psi[L.cur], L.psi[1 - L.cur], h->o.reimpose_parity ? hd.mask : 0, &L.state[1], id,
                     1 - L.cur, nullptr);
    h->stats.launches += 2;
    L.cur ^= 1;
    LatState st;
    cudaMemcpyAsync(&st, &L.state[1], sizeof(LatState), cudaMemcpyDeviceToHost, h->st);
    cudaError_t e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return fail(h, FDTD_ERR_CUDA, std::string("load_psi: ") + cudaGetErrorString(e));
    if (st.status == STATUS_NONFINITE) return fail(h, FDTD_ERR_NONFINITE, "load_psi: non-finite or zero norm");
  }
  L.mask = hd.mask;
  L.has_psi = true;
  record_start(h, L);
  return cuda_check(h, "load_psi");
}

int fdtd_evolve(fdtd_handle h, int64_t max_steps, int64_t* steps_done) {
  Range r("fdtd_evolve");
  if (!h) return FDTD_ERR_INVALID_ARG;
  if (max_steps < 0) return fail(h, FDTD_ERR_INVALID_ARG, "evolve: max_steps < 0");
  for (auto& L : h->lats)
    if (!L.has_v || !L.has_psi) return fail(h, FDTD_ERR_STATE, "evolve: set_potential and init/set_psi first");
  int rc = FDTD_OK;
  if (h->o.batched) {
    rc = evolve_batched(h, max_steps);
  } else {
    for (auto& L : h->lats) {
      rc = evolve_one(h, L, max_steps);
      if (rc) return rc;
    }
  }
  if (rc) return rc;
  int64_t mx = 0;
  bool all_conv = true;
  for (auto& L : h->lats) {
    mx = std::max(mx, L.last_steps);
    all_conv = all_conv && L.host_state.converged;
  }
  if (steps_done) *steps_done = mx;
  return (h->o.tol > 0.0 && !all_conv) ? FDTD_NOT_CONVERGED : FDTD_OK;
}

int fdtd_last_check(fdtd_handle h, int lat, fdtd_obs* out) {
  int rc = lat_check(h, lat);
  if (rc) return rc;
  if (!out) return fail(h, FDTD_ERR_INVALID_ARG, "last_check: null output");
  Lat& L = h->lats[lat];
  cudaMemcpyAsync(&L.host_state, &L.state[0], sizeof(LatState), cudaMemcpyDeviceToHost, h->st);
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return fail(h, FDTD_ERR_CUDA, std::string("last_check: ") + cudaGetErrorString(e));
  fill_obs(L, L.host_state, out);
  out->steps = L.last_steps;
  out->converged = L.host_state.converged;
  out->checks = L.host_state.checks;
  return FDTD_OK;
}

int fdtd_bounds_violations(fdtd_handle h, int64_t* count) {
  if (!h || !count) return FDTD_ERR_INVALID_ARG;
#ifdef FDTD_CHECK_BOUNDS
  int32_t v = 0;
  cudaMemcpyAsync(&v, h->flags + 3, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st);
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return fail(h, FDTD_ERR_CUDA, std::string("bounds_violations: ") + cudaGetErrorString(e));
  *count = v;
  return FDTD_OK;
#else
  *count = 0;
  return fail(h, FDTD_ERR_STATE, "bounds_violations: not a bounds-checking build (-DFDTD_CHECK_BOUNDS)");
#endif
}

int fdtd_check_history(fdtd_handle h, int lat, double* out, int cap, int* count) {
  int rc = lat_check(h, lat);
  if (rc) return rc;
  if (!count || cap < 0 || (cap > 0 && !out)) return fail(h, FDTD_ERR_INVALID_ARG, "check_history: bad output");
  Lat& L = h->lats[lat];
  cudaMemcpyAsync(&L.host_state, &L.state[0], sizeof(LatState), cudaMemcpyDeviceToHost, h->st);
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return fail(h, FDTD_ERR_CUDA, std::string("check_history: ") + cudaGetErrorString(e));
  const int total = L.host_state.checks;
  *count = total;
  // the most recent min(total, kHistCap, cap) records, oldest first
  const int keep = std::min(std::min(total, kHistCap), cap);
  const size_t rec = (size_t)kHistFields * sizeof(double);
  for (int q = 0; q < keep; ++q) {
    const int k = total - keep + q;  // check number, 0-based
    cudaMemcpyAsync(out + (size_t)q * kHistFields, L.hist + (size_t)(k % kHistCap) * kHistFields, rec,
                    cudaMemcpyDeviceToHost, h->st);
  }
  e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return fail(h, FDTD_ERR_CUDA, std::string("check_history: ") + cudaGetErrorString(e));
  return FDTD_OK;
}

int fdtd_observables(fdtd_handle h, int lat, fdtd_obs* out) {
  Range r("fdtd_observables");
  int rc = lat_check(h, lat);
  if (rc) return rc;
  if (!out) return fail(h, FDTD_ERR_INVALID_ARG, "observables: null output");
  Lat& L = h->lats[lat];
  if (!L.has_v || !L.has_psi) return fail(h, FDTD_ERR_STATE, "observables: set_potential and init/set_psi first");
  int np = launch_sums_any(h, L, L.psi[L.cur], nullptr);
  launch_state_reset(&L.state[1], 0, h->st);
  launch_finalize(&L.state[1], L.partials, np, 0, 0, L.p, L.d.v_inf, 0.0, 0, 1, h->st);
  h->stats.launches += 2;
  LatState s;
  cudaMemcpyAsync(&s, &L.state[1], sizeof(LatState), cudaMemcpyDeviceToHost, h->st);
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return fail(h, FDTD_ERR_CUDA, std::string("observables: ") + cudaGetErrorString(e));
  if ((rc = cuda_check(h, "observables"))) return rc;
  if (s.status == STATUS_NONFINITE) return fail(h, FDTD_ERR_NONFINITE, "observables: non-finite or zero norm");
  fill_obs(L, s, out);
  out->steps = L.last_steps;
  out->converged = L.host_state.converged;
  out->checks = L.host_state.checks;
  return FDTD_OK;
}

int fdtd_upsample(fdtd_handle src, int lat_src, fdtd_handle dst, int lat_dst) {
  Range r("fdtd_upsample");
  int rc = lat_check(src, lat_src);
  if (rc) return rc;
  if ((rc = lat_check(dst, lat_dst))) return rc;
  Lat& S = src->lats[lat_src];
  Lat& D = dst->lats[lat_dst];
  if (D.d.n != 2 * S.d.n || std::fabs(D.d.length - S.d.length) > 1e-12 * S.d.length)
    return fail(dst, FDTD_ERR_SHAPE, "upsample: need n_dst = 2 n_src and equal box lengths");
  if (!S.has_psi) return fail(dst, FDTD_ERR_STATE, "upsample: source has no wavefunction");
  if (S.p.periodic != D.p.periodic) return fail(dst, FDTD_ERR_INVALID_ARG, "upsample: boundaries differ");
  if (!D.has_v) return fail(dst, FDTD_ERR_STATE, "upsample: set the destination potential first");
  if (src->st != dst->st) {
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, src->st);
    cudaStreamWaitEvent(dst->st, ev, 0);
    cudaEventDestroy(ev);
  }
  void* tmp = D.psi[1 - D.cur];
  with_type(S.d.precision, [&](auto* tin) {
    using Ti = std::remove_pointer_t<decltype(tin)>;
    with_type(D.d.precision, [&](auto* tout) {
      using To = std::remove_pointer_t<decltype(tout)>;
      launch_upsample<Ti, To>((const Ti*)S.psi[S.cur], S.d.n, (To*)tmp, D.p.periodic, dst->st);
    });
  });
  dst->stats.launches += 1;
  // renormalise and give the field the source's symmetry (Sec. VI)
  int id = 1000000 + (dst->check_seq++);
  int np = launch_sums_any(dst, D, tmp, nullptr);
  launch_state_reset(&D.state[1], 0, dst->st);
  launch_finalize(&D.state[1], D.partials, np, id, 0, D.p, D.d.v_inf, 0.0, 0, 0, dst->st);
  scale_parity_any(dst, D, tmp, D.psi[D.cur], S.mask, &D.state[1], id, D.cur, nullptr);
  dst->stats.launches += 2;
  D.mask = S.mask;
  D.has_psi = true;
  record_start(dst, D);
  LatState s;
  cudaMemcpyAsync(&s, &D.state[1], sizeof(LatState), cudaMemcpyDeviceToHost, dst->st);
  cudaError_t e = cudaStreamSynchronize(dst->st);
  if (e != cudaSuccess) return fail(dst, FDTD_ERR_CUDA, std::string("upsample: ") + cudaGetErrorString(e));
  if (s.status == STATUS_NONFINITE) return fail(dst, FDTD_ERR_NONFINITE, "upsample: non-finite or zero norm");
  return cuda_check(dst, "upsample");
}

int fdtd_backward(fdtd_handle h, int lat, int64_t T, double w_e, double w_r, void* gv_out, int dtype, int mem_kind,
                  fdtd_obs* obs) {
  Range r("fdtd_backward");
  int rc = lat_check(h, lat);
  if (rc) return rc;
  Lat& L = h->lats[lat];
  if (!gv_out || (dtype != FDTD_F64 && dtype != FDTD_F32) ||
      (mem_kind != FDTD_MEM_HOST && mem_kind != FDTD_MEM_DEVICE) || T < 1 || !std::isfinite(w_e) ||
      !std::isfinite(w_r))
    return fail(h, FDTD_ERR_INVALID_ARG, "backward: bad pointer, dtype, mem_kind, T or weights");
  if (L.d.precision == FDTD_BF16) return fail(h, FDTD_ERR_INVALID_ARG, "backward: not available for BF16 storage");
  if (!L.psi0 || T > L.bw_T)
    return fail(h, FDTD_ERR_WORKSPACE, "backward: T exceeds options.backward_steps given at create");
  if (!L.has_v || !L.has_psi0) return fail(h, FDTD_ERR_STATE, "backward: set_potential and init/set_psi first");
  const int64_t ce = h->o.check_every;
  const int K = L.bw_K;
  const int mask = h->o.reimpose_parity ? L.mask : 0;
  const size_t fb = L.n3 * L.es;
  auto field = [&](void* base, int64_t i) { return (void*)((char*)base + (size_t)i * fb); };
  LatState* scratch = &L.state[1];
  launch_state_reset(scratch, 0, h->st);
  h->stats.launches += 1;

  // forward pass from the recorded start, saving every K-th field
  L.cur = 0;
  cudaMemcpyAsync(L.psi[0], L.psi0, fb, cudaMemcpyDeviceToDevice, h->st);
  for (int64_t t = 0; t < T; ++t) {
    if (t % ce == 0) {
      int id = 2000000 + (h->check_seq++);
      int np = launch_sums_any(h, L, L.psi[L.cur], nullptr);
      launch_finalize(scratch, L.partials, np, id, t, L.p, 0.0, 0.0, 0, 0, h->st);
      launch_store_scale(scratch, L.scales + t / ce, h->st);
      scale_parity_any(h, L, L.psi[L.cur], L.psi[1 - L.cur], mask, scratch, id, 1 - L.cur, nullptr);
      h->stats.launches += 2;
      L.cur ^= 1;
    }
    if (t % K == 0)
      cudaMemcpyAsync(field(L.pool, t / K), L.psi[L.cur], fb, cudaMemcpyDeviceToDevice, h->st);
    run_steps(h, L, 1, nullptr);
  }
  // seed the adjoint with the derivative of the loss at psi_T
  int np = launch_sums_any(h, L, L.psi[L.cur], nullptr);
  launch_finalize(scratch, L.partials, np, 0, T, L.p, 0.0, 0.0, 0, 1, h->st);
  h->stats.launches += 1;
  int lc = 0;
  with_type(L.d.precision, [&](auto* tag) {
    using T_ = std::remove_pointer_t<decltype(tag)>;
    if constexpr (!std::is_same_v<T_, __nv_bfloat16>)
      launch_adjoint_seed<T_>((const T_*)L.psi[L.cur], L.v, scratch, w_e, w_r, (T_*)L.lam[0], L.gv, L.p, h->st);
  });
  h->stats.launches += 1;
  // psi[cur] keeps psi_T
  for (int64_t sgi = (T - 1) / K; sgi >= 0; --sgi) {
    const int64_t t0 = sgi * K, t1 = std::min<int64_t>(t0 + K, T);
    // raw output of the step ending at t (t0 < t <= t1): the segment's last
    // one and those of check steps go to bw_raw, the others are the seg fields
    auto raw_slot = [&](int64_t t) -> void* {
      if (t == t1) return field(L.bw_raw, 0);
      return field(L.bw_raw, 1 + (t - (t0 / ce + 1) * ce) / ce);
    };
    auto raw_of = [&](int64_t t) -> void* { return (t == t1 || t % ce == 0) ? raw_slot(t) : field(L.seg, t - t0); };
    cudaMemcpyAsync(field(L.seg, 0), field(L.pool, sgi), fb, cudaMemcpyDeviceToDevice, h->st);
    for (int64_t t = t0; t < t1; ++t) {
      with_type(L.d.precision, [&](auto* tag) {
        using T_ = std::remove_pointer_t<decltype(tag)>;
        void* nxt = raw_of(t + 1);
        if constexpr (std::is_same_v<T_, double>)
          launch_step_f64((const double*)field(L.seg, t - t0), (double*)nxt, L.coefA, L.coefCB, L.p, nullptr, h->st);
        else if constexpr (std::is_same_v<T_, float>)
          launch_step_f32<float>((const float*)field(L.seg, t - t0), (float*)nxt, (const float*)L.v, L.p, nullptr,
                                 h->st);
        if constexpr (!std::is_same_v<T_, __nv_bfloat16>)
          if ((t + 1) % ce == 0 && t + 1 < t1)
            launch_scale_parity_from<T_>((const T_*)nxt, (T_*)field(L.seg, t + 1 - t0), L.d.n, mask,
                                         L.scales + (t + 1) / ce, h->st);
      });
      h->stats.launches += ((t + 1) % ce == 0 && t + 1 < t1) ? 2 : 1;
    }
    for (int64_t t = t1; t > t0; --t) {
      with_type(L.d.precision, [&](auto* tag) {
        using T_ = std::remove_pointer_t<decltype(tag)>;
        if constexpr (!std::is_same_v<T_, __nv_bfloat16>) {
          launch_adjoint_pointwise<T_>((const T_*)L.lam[lc], (const T_*)field(L.seg, t - 1 - t0), (const T_*)raw_of(t),
                                       L.v, L.coefCB, (T_*)L.bw_u, L.gv, L.p, h->st);
          launch_adjoint_stencil<T_>((const T_*)L.bw_u, (const T_*)L.lam[lc], (T_*)L.lam[1 - lc], L.v, L.coefA, L.p,
                                     h->st);
          if ((t - 1) % ce == 0)
            launch_parity_adjoint_scale<T_>((T_*)L.lam[1 - lc], L.d.n, mask, L.scales + (t - 1) / ce, h->st);
        }
      });
      h->stats.launches += ((t - 1) % ce == 0) ? 3 : 2;
      lc ^= 1;
    }
  }
  if ((rc = cuda_check(h, "backward"))) return rc;
  if (obs) {
    LatState s;
    cudaMemcpyAsync(&s, scratch, sizeof(LatState), cudaMemcpyDeviceToHost, h->st);
    cudaStreamSynchronize(h->st);
    fill_obs(L, s, obs);
    obs->steps = T;
  }
  return export_field(h, L.gv, FDTD_F64, gv_out, dtype, mem_kind, L.n3);
}

namespace {

void* snap_field(Lat& L, int slot) { return (char*)L.snaps + (size_t)slot * L.n3 * L.es; }

int snap_check(fdtd_context* h, int lat, int slot) {
  int rc = lat_check(h, lat);
  if (rc) return rc;
  if (slot < 0 || slot >= h->lats[lat].nsnap)
    return fail(h, FDTD_ERR_INVALID_ARG, "snapshot slot out of range (options.snapshots)");
  return FDTD_OK;
}

// psi[cur] <- s psi[cur] with sum psi^2 a^3 = 1 (no symmetry pass).
int renormalise(fdtd_context* c, Lat& L) {
  const int id = 3000000 + (c->check_seq++);
  int np = launch_sums_any(c, L, L.psi[L.cur], nullptr);
  launch_state_reset(&L.state[1], 0, c->st);
  launch_finalize(&L.state[1], L.partials, np, id, 0, L.p, L.d.v_inf, 0.0, 0, 0, c->st);
  scale_parity_any(c, L, L.psi[L.cur], L.psi[1 - L.cur], 0, &L.state[1], id, 1 - L.cur, nullptr);
  c->stats.launches += 2;
  LatState s;
  cudaMemcpyAsync(&s, &L.state[1], sizeof(LatState), cudaMemcpyDeviceToHost, c->st);
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return fail(c, FDTD_ERR_CUDA, std::string("renormalise: ") + cudaGetErrorString(e));
  if (s.status == STATUS_NONFINITE) return fail(c, FDTD_ERR_NONFINITE, "the field vanished or is not finite");
  L.cur ^= 1;
  return cuda_check(c, "renormalise");
}

}  // namespace

int fdtd_snapshot_save(fdtd_handle h, int lat, int slot) {
  int rc = snap_check(h, lat, slot);
  if (rc) return rc;
  Lat& L = h->lats[lat];
  if (!L.has_psi) return fail(h, FDTD_ERR_STATE, "snapshot_save: no wavefunction yet");
  cudaMemcpyAsync(snap_field(L, slot), L.psi[L.cur], L.n3 * L.es, cudaMemcpyDeviceToDevice, h->st);
  return cuda_check(h, "snapshot_save");
}

int fdtd_snapshot_load(fdtd_handle h, int lat, int slot) {
  int rc = snap_check(h, lat, slot);
  if (rc) return rc;
  Lat& L = h->lats[lat];
  cudaMemcpyAsync(L.psi[L.cur], snap_field(L, slot), L.n3 * L.es, cudaMemcpyDeviceToDevice, h->st);
  L.has_psi = true;
  record_start(h, L);
  return cuda_check(h, "snapshot_load");
}

int fdtd_project_out(fdtd_handle h, int lat, const int* slots, int count) {
  int rc = lat_check(h, lat);
  if (rc) return rc;
  if (count < 0 || (count > 0 && !slots)) return fail(h, FDTD_ERR_INVALID_ARG, "project_out: bad slot list");
  Lat& L = h->lats[lat];
  if (!L.has_psi || !L.has_v) return fail(h, FDTD_ERR_STATE, "project_out: set_potential and a wavefunction first");
  for (int k = 0; k < count; ++k)
    if ((rc = snap_check(h, lat, slots[k]))) return rc;
  for (int k = 0; k < count; ++k) {
    with_type(L.d.precision, [&](auto* tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      const T* phi = (const T*)snap_field(L, slots[k]);
      int np = launch_dot2<T>(phi, (const T*)L.psi[L.cur], L.n3, L.dot_parts, h->st);
      launch_ratio(L.dot_parts, np, L.coef, h->st);
      launch_axpy<T>((T*)L.psi[L.cur], phi, L.coef, -1.0, 0.0, L.n3, h->st);
    });
    h->stats.launches += 3;
  }
  return renormalise(h, L);
}

int fdtd_combine(fdtd_handle h, int lat, const int* slots, const double* weights, int count) {
  int rc = lat_check(h, lat);
  if (rc) return rc;
  if (count < 1 || !slots || !weights) return fail(h, FDTD_ERR_INVALID_ARG, "combine: bad slot or weight list");
  Lat& L = h->lats[lat];
  if (!L.has_v) return fail(h, FDTD_ERR_STATE, "combine: set_potential first");
  for (int k = 0; k < count; ++k) {
    if ((rc = snap_check(h, lat, slots[k]))) return rc;
    if (!std::isfinite(weights[k])) return fail(h, FDTD_ERR_INVALID_ARG, "combine: weights must be finite");
  }
  cudaMemsetAsync(L.psi[L.cur], 0, L.n3 * L.es, h->st);
  for (int k = 0; k < count; ++k) {
    with_type(L.d.precision, [&](auto* tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      launch_axpy<T>((T*)L.psi[L.cur], (const T*)snap_field(L, slots[k]), nullptr, 0.0, weights[k], L.n3, h->st);
    });
    h->stats.launches += 1;
  }
  L.has_psi = true;
  if ((rc = renormalise(h, L))) return rc;
  record_start(h, L);
  return FDTD_OK;
}

int fdtd_tuned_config(fdtd_handle h, int lat, int* depth, int* zchunk) {
  int rc = lat_check(h, lat);
  if (rc) return rc;
  if (!depth || !zchunk) return fail(h, FDTD_ERR_INVALID_ARG, "tuned_config: null output");
  Lat& L = h->lats[lat];
  if (h->o.batched && h->batch_depth) {  // the persistent launch's choice
    *depth = h->batch_depth;
    *zchunk = h->batch_zc;
    return FDTD_OK;
  }
  if (L.has_v && L.has_psi) choose_config(h, L);
  *depth = L.depth;
  *zchunk = L.plain ? 0 : L.zc;
  return cuda_check(h, "tuned_config");
}

int fdtd_get_stats(fdtd_handle h, fdtd_stats* out) {
  if (!h || !out) return FDTD_ERR_INVALID_ARG;
  cudaStreamSynchronize(h->st);
  prof_collect(h);
  *out = h->stats;
  return FDTD_OK;
}

int fdtd_reset_stats(fdtd_handle h) {
  if (!h) return FDTD_ERR_INVALID_ARG;
  cudaStreamSynchronize(h->st);
  h->ev_used = 0;
  std::memset(&h->stats, 0, sizeof(h->stats));
  return FDTD_OK;
}

int fdtd_set_profiling(fdtd_handle h, int on) {
  if (!h) return FDTD_ERR_INVALID_ARG;
  cudaStreamSynchronize(h->st);
  prof_collect(h);
  h->profiling = on != 0;
  return FDTD_OK;
}

}  // extern "C"
