// Evolution (Secs. III-V): the stencil autotuner, the steps and checks of one
// lattice on the stream or as a CUDA graph with a device-side loop, and the
// batched persistent driver.
#include "api_internal.cuh"

using namespace fdtd;
using namespace fdtd::api;

namespace fdtd {
namespace api {

// ---- autotuning of the stencil configuration ---------------------------------
// Fastest (depth, tile width, span, one-step kernel, direct four-site
// one-step kernel) per (n, precision, device, periodic, TMA kernel usable),
// shared by all handles.  The last key member keeps a lattice whose tensor
// maps could not be encoded (timed on the one-step kernels only) from
// handing its choice to lattices of the same size that can use the TMA
// kernel.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, std::tuple<int, int, int, bool, bool>> g_tune;

// depth of the blocked stencil when none is timed or forced
int blocked_depth(int n) { return n >= 96 ? 3 : 2; }

// One launch of the TMA stencil, psi[cur] -> psi[1 - cur] (FP32 or BF16 psi)
void launch_step_tma_any(const Lat& L, int ti, int d, int tx, int zc, const int32_t* active, int32_t* err,
                         cudaStream_t st) {
  if (L.tma16)
    launch_step_tma(L.maps[ti][d - 1][L.cur], L.maps[ti][d - 1][2], (__nv_bfloat16*)L.psi[1 - L.cur], L.p, d, tx, zc,
                    active, err, st);
  else
    launch_step_tma(L.maps[ti][d - 1][L.cur], L.maps[ti][d - 1][2], (float*)L.psi[1 - L.cur], L.p, d, tx, zc, active,
                    err, st);
}

void choose_config(fdtd_context* c, Lat& L) {
  if (L.depth) return;
  const bool tma = (L.tma_ok || L.tma16) && c->o.stencil_kernel == 0;
  // the direct kernel applies (FP32 or BF16 storage, n % 4 == 0)
  const bool f4 = (L.d.precision == FDTD_F32 || L.d.precision == FDTD_BF16) && L.d.n % 4 == 0;
  const bool bf16 = L.d.precision == FDTD_BF16;
  L.plain = false;
  L.direct = false;
  if (!tma) {
    L.depth = 1;
    L.tx = 128;
    L.zc = 0;
    L.plain = true;
    L.direct = c->o.stencil_kernel == 2 && f4;
    // a lattice the TMA kernel does not take (periodic, or n < 8) still
    // times the two one-step kernels when none is forced
    if (!(c->o.stencil_kernel == 0 && c->o.autotune && f4)) return;
  } else if (c->o.temporal_depth > 0 || !c->o.autotune) {
    L.depth = c->o.temporal_depth > 0 ? c->o.temporal_depth : blocked_depth(L.d.n);
    L.tx = c->o.tile_x ? c->o.tile_x : (L.d.n > 64 ? 128 : 64);
    L.zc = c->o.zchunk != 0 ? c->o.zchunk : tma_zchunk(L.d.n, L.depth, L.tx, bf16);
    return;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  auto key = std::make_tuple(L.d.n, L.d.precision, dev, L.p.periodic, (int)tma);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      std::tie(L.depth, L.tx, L.zc, L.plain, L.direct) = it->second;
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
  int bd = tma ? blocked_depth(n) : 1, bt = n > 64 ? 128 : 64, bz = tma ? tma_zchunk(n, bd, bt, bf16) : 0;
  bool bp = !tma, bdir = false;
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
          if (bf16)
            launch_step_f32<__nv_bfloat16>((const __nv_bfloat16*)L.psi[L.cur], (__nv_bfloat16*)L.psi[1 - L.cur],
                                           (const float*)L.v, L.p, nullptr, c->st);
          else
            launch_step_f32<float>((const float*)L.psi[L.cur], (float*)L.psi[1 - L.cur], (const float*)L.v, L.p,
                                   nullptr, c->st);
        },
        1);
    best = rate;
    bd = 1;
    bp = true;
  }
  // the direct four-site one-step kernel (n % 4 == 0 wherever the TMA kernel applies)
  {
    double rate = time_it(
        [&]() {
          if (bf16)
            launch_direct<__nv_bfloat16>((const __nv_bfloat16*)L.psi[L.cur], (__nv_bfloat16*)L.psi[1 - L.cur],
                                         (const float*)L.v, L.p, nullptr, c->st);
          else
            launch_direct<float>((const float*)L.psi[L.cur], (float*)L.psi[1 - L.cur], (const float*)L.v, L.p,
                                 nullptr, c->st);
        },
        1);
    if (rate > best) {
      best = rate;
      bd = 1;
      bp = true;
      bdir = true;
    }
  }
  for (int ti = 0; ti < (tma ? 2 : 0); ++ti) {
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
      const long long total = tma_tile_planes(n, tx), slots = tma_resident_blocks(d, tx, bf16);
      for (int m = 1; m <= 3; ++m) spans.push_back((int)std::max(1LL, (total + m * slots - 1) / (m * slots)));
      spans.push_back(-1);  // the balanced one-wave partition
      spans.push_back(-2);  // columns first (neighbouring tiles in step)
      std::sort(spans.begin(), spans.end());
      spans.erase(std::unique(spans.begin(), spans.end()), spans.end());
      for (int zc : spans) {
        double rate = time_it(
            [&]() {
              launch_step_tma_any(L, ti, d, tx, zc, nullptr, c->flags + 1, c->st);
            },
            d);
        if (rate > best) {
          best = rate;
          bd = d;
          bt = tx;
          bz = zc;
          bp = false;
          bdir = false;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int32_t err = 0;
  cudaMemcpy(&err, c->flags + 1, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (err) {  // the timed launches did no work: keep the heuristic, cache nothing
    if (tma) {
      L.depth = blocked_depth(n);
      L.tx = n > 64 ? 128 : 64;
      L.zc = tma_zchunk(n, L.depth, L.tx, bf16);
    }
    return;
  }
  L.depth = bd;
  L.tx = bt;
  L.zc = bz;
  L.plain = bp;
  L.direct = bdir;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = std::make_tuple(bd, bt, bz, bp, bdir);
}

// The last step before a check runs as the check step (update + sums of
// its result in one pass, the sums item's partials): FP32 lattices on the
// TMA stencil.
bool check_step_fused(const fdtd_context* c, const Lat& L) {
  return L.tma_ok && c->o.stencil_kernel == 0 && !L.plain;
}

// Enqueue `count` update steps of lattice L (psi[cur] -> ... ; cur follows),
// the first of them being step t0 of the current evolve.  With
// before_check, a check follows: the last step is the check step, which
// leaves the check's partial sums in L.partials (L.sums_ready).
void run_steps(fdtd_context* c, Lat& L, int64_t count, const int32_t* active, int64_t t0, bool before_check) {
  const int prec = L.d.precision;
  choose_config(c, L);
  const bool tma = (L.tma_ok || L.tma16) && c->o.stencil_kernel == 0 && !L.plain;
  const int depth = tma ? L.depth : 1;
  const bool fuse = before_check && count > 0 && check_step_fused(c, L);
  if (count > 0) L.sums_ready = false;
  if (fuse) --count;
  // the launches go to the profiling record in runs of one depth: one pair
  // of events around each run (an event between two launches would cost
  // the second its early launch), credited per launch
  fdtd_context::Pending run{};
  int run_k = 0;
  auto close_run = [&]() {
    if (!run.launches) return;
    prof_end(c);
    c->pending.push_back(run);
    run = fdtd_context::Pending{};
  };
  while (count > 0) {
    int k = (int)std::min<int64_t>(count, depth);
    if (run.launches && k != run_k) close_run();
    if (!run.launches) {
      run.ev = prof_begin(c);
      run.t_start = t0;
      run_k = k;
    }
    if (is_complex(prec)) {
      with_ctype(prec, [&](auto* tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        launch_cstep<T>((const T*)L.psi[L.cur], (T*)L.psi[1 - L.cur], (const T*)L.coefA, (const T*)L.coefCB, L.p,
                        active, c->st);
      });
    } else if (prec == FDTD_F64) {
      launch_step_f64((const double*)L.psi[L.cur], (double*)L.psi[1 - L.cur], L.coefA, L.coefCB, L.p, active, c->st);
    } else if (prec == FDTD_F32) {
      if (tma)
        launch_step_tma(L.maps[L.tx == 128][k - 1][L.cur], L.maps[L.tx == 128][k - 1][2], (float*)L.psi[1 - L.cur],
                        L.p, k, L.tx, k == depth ? L.zc : 0, active, c->flags + 1, c->st);
      else if (L.direct)
        launch_direct_f32((const float*)L.psi[L.cur], (float*)L.psi[1 - L.cur], (const float*)L.v, L.p, active,
                          c->st);
      else
        launch_step_f32<float>((const float*)L.psi[L.cur], (float*)L.psi[1 - L.cur], (const float*)L.v, L.p, active,
                               c->st);
    } else if (tma) {
      launch_step_tma(L.maps[L.tx == 128][k - 1][L.cur], L.maps[L.tx == 128][k - 1][2],
                      (__nv_bfloat16*)L.psi[1 - L.cur], L.p, k, L.tx, k == depth ? L.zc : 0, active, c->flags + 1,
                      c->st);
    } else if (L.direct) {
      launch_direct<__nv_bfloat16>((const __nv_bfloat16*)L.psi[L.cur], (__nv_bfloat16*)L.psi[1 - L.cur],
                                   (const float*)L.v, L.p, active, c->st);
    } else {
      launch_step_f32<__nv_bfloat16>((const __nv_bfloat16*)L.psi[L.cur], (__nv_bfloat16*)L.psi[1 - L.cur],
                                     (const float*)L.v, L.p, active, c->st);
    }
    c->stats.launches += 1;
    // algorithmic bytes: psi read + psi write + V (FP64: A and cB; complex: A and cB pairs) read once per launch
    run.launches += 1;
    run.updates += (int64_t)L.n3 * k;
    run.bytes += (double)L.n3 * (2.0 * L.es + coef_bytes(prec));
    L.cur ^= 1;
    count -= k;
    t0 += k;
  }
  close_run();
  if (fuse) {
    launch_step_sums_tma(L.maps[0][1][L.cur], L.maps[0][1][2], (float*)L.psi[1 - L.cur], L.p, L.partials, active,
                         c->flags + 1, c->st);
    c->stats.launches += 1;
    L.cur ^= 1;
    L.sums_ready = true;
  }
}

int launch_sums_any(fdtd_context* c, Lat& L, const void* psi, const int32_t* active) {
  int np = 0;
  if (is_complex(L.d.precision)) {
    with_ctype(L.d.precision, [&](auto* tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      np = launch_csums<T>((const T*)psi, (const T*)L.v, L.p, L.partials, active, c->st);
    });
    c->stats.launches += 1;
    return np;
  }
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
  if (is_complex(L.d.precision)) {
    with_ctype(L.d.precision, [&](auto* tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      launch_cscale_parity<T>((const T*)in, (T*)out, L.d.n, mask, s, id, out_idx, sw, c->st);
    });
    c->stats.launches += 1;
    return;
  }
  with_type(L.d.precision, [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    launch_scale_parity<T>((const T*)in, (T*)out, L.d.n, mask, s, id, out_idx, sw, c->st);
  });
  c->stats.launches += 1;
}

// The partial sums of psi[cur]: those the check step left, or a sums pass.
int check_sums(fdtd_context* c, Lat& L) {
  if (L.sums_ready) {
    L.sums_ready = false;
    return tma_sums_blocks(L.d.n);
  }
  return launch_sums_any(c, L, L.psi[L.cur], &L.state[0].active);
}

// One check of Secs. III-V on psi[cur]: sums, finalize, renormalise + mask.
void enqueue_check(fdtd_context* c, Lat& L, int check_id, int64_t t) {
  int np = check_sums(c, L);
  launch_finalize(&L.state[0], L.partials, np, check_id, t, L.p, L.d.v_inf, c->o.tol, c->o.tol_relative, 1, c->st, 0,
                  0, nullptr, L.hist, sums_per_block(L.d.precision));
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
  int np = check_sums(c, L);
  launch_finalize(&L.state[0], L.partials, np, 0, 0, L.p, L.d.v_inf, c->o.tol, c->o.tol_relative, 1, c->st, (int)ce,
                  cond, c->flags + 1, L.hist, sums_per_block(L.d.precision));
  c->stats.launches += 1;
  int mask = c->o.reimpose_parity ? L.mask : 0;
  scale_parity_any(c, L, L.psi[L.cur], L.psi[1 - L.cur], mask, &L.state[0], -1, 1 - L.cur, &L.state[0]);
  L.cur ^= 1;
}

// Stencil launches and algorithmic bytes of one check_every-step segment.
// (The check step, the last of a segment on a fused lattice, is not counted:
// it is the check's sums pass as well.)
void segment_work(fdtd_context* c, const Lat& L, int64_t ce, int64_t* launches, double* bytes, int64_t* updates) {
  const bool tma = (L.tma_ok || L.tma16) && c->o.stencil_kernel == 0 && !L.plain;
  const int depth = tma ? L.depth : 1;
  const int64_t steps = check_step_fused(c, L) ? ce - 1 : ce;
  *launches = (steps + depth - 1) / depth;
  *bytes = (double)*launches * L.n3 * (2.0 * L.es + coef_bytes(L.d.precision));
  *updates = steps * (int64_t)L.n3;
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
  const int64_t key[6] = {L.cur, mask, L.depth, L.zc, L.plain + 2 * L.direct, ce};
  if (L.graph_exec[b] && std::equal(key, key + 6, L.graph_key[b])) return true;
  release_graph(L, b);
  Range r("evolve graph build");
  if ((L.tma_ok || L.tma16) && c->o.stencil_kernel == 0 && !L.plain && ce % L.depth)
    (void)tma_zchunk(L.d.n, (int)(ce % L.depth), L.tx, L.tma16);  // occupancy query outside the capture
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
  // one, which cannot be captured); the graph runs on the lattice's own
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
  const bool ready0 = L.sums_ready;
  // the body starts with the sums of its start field in place: the last
  // check step of the previous iteration, or the sums pass before the launch
  L.sums_ready = check_step_fused(c, L);
  if (ok) {
    for (int rep = 0; rep < 2; ++rep) {
      enqueue_check_seq(c, L, ce, cond);
      run_steps(c, L, ce, &L.state[0].active, 0, true);
    }
    cudaGraph_t captured = nullptr;
    ok = cudaStreamEndCapture(c->st, &captured) == cudaSuccess && L.cur == cur0;
  }
  c->st = user_st;
  L.sums_ready = ready0;
  L.graph_kernels = c->stats.launches - launches0;
  c->stats.launches = launches0;
  c->pending.resize(pending0);
  L.cur = cur0;
  cudaGraphExec_t exec = nullptr;
  if (ok) ok = cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
  if (ok && !L.run_st) {
    ok = cudaStreamCreateWithFlags(&L.run_st, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) L.run_st = nullptr;
  }
  if (ok) ok = cudaGraphUpload(exec, L.run_st) == cudaSuccess;
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

// One lattice's evolve in stages, so that the graph loops of several
// lattices of a handle can run at the same time: begin (state reset and,
// with profiling on, the timed sample), the graph loop over full pairs of
// segments, and the stream-driven tail (what the graph did not cover).
struct EvolveRun {
  int64_t t = 0, t_end = 0, pairs = 0;
  int check_id = 0;
  bool done = false, graph = false;
};

int evolve_begin(fdtd_context* c, Lat& L, int64_t max_steps, EvolveRun& r) {
  launch_state_reset(&L.state[0], 0, c->st);
  c->stats.launches += 1;
  L.sums_ready = false;
  const int64_t ce = c->o.check_every;
  if (c->o.graphs && c->profiling) {
    // the timed sample: two segments through the stream, every stencil
    // launch between CUDA events (a graph loop body cannot hold events)
    for (int i = 0; i < 2 && r.t + ce <= max_steps; ++i) {
      enqueue_check(c, L, r.check_id++, r.t);
      run_steps(c, L, ce, &L.state[0].active, r.t, true);
      r.t += ce;
    }
    int rc = cuda_check(c, "evolve launch");
    if (rc) return rc;
    if ((rc = read_state(c, L))) return rc;
    if (!L.host_state.active) r.done = true;
  }
  // full pairs of segments in one graph launch, the convergence check
  // ending the loop on the device
  r.pairs = (!r.done && c->o.graphs) ? std::min<int64_t>((max_steps - r.t) / (2 * ce), 1 << 28) : 0;
  r.graph = r.pairs > 0 && ensure_graph(c, L, ce);
  if (r.graph) {
    // the graph's first check takes the sums of its start field as ready
    if (check_step_fused(c, L) && !L.sums_ready) {
      launch_sums_any(c, L, L.psi[L.cur], &L.state[0].active);
      L.sums_ready = true;
    }
    r.t_end = r.t + 2 * r.pairs * ce;
    launch_state_reset(&L.state[0], 2, c->st, r.check_id + (int)(2 * r.pairs));
    c->stats.launches += 1;
  }
  return FDTD_OK;
}

// Launch the graph loop on the lattice's own stream, ordered after the
// handle's stream up to `ready` and before whatever the handle's stream
// takes next.  (A graph launched into the legacy stream paid about half a
// millisecond per launch, hence private non-blocking streams.)
int evolve_graph_launch(fdtd_context* c, Lat& L, cudaEvent_t ready) {
  if (!L.run_st && cudaStreamCreateWithFlags(&L.run_st, cudaStreamNonBlocking) != cudaSuccess) {
    L.run_st = nullptr;
    return cuda_check(c, "evolve stream");
  }
  if (!L.run_ev && cudaEventCreateWithFlags(&L.run_ev, cudaEventDisableTiming) != cudaSuccess) {
    L.run_ev = nullptr;
    return cuda_check(c, "evolve event");
  }
  cudaStreamWaitEvent(L.run_st, ready, 0);
  cudaGraphLaunch(L.graph_exec[L.cur], L.run_st);
  cudaEventRecord(L.run_ev, L.run_st);
  cudaStreamWaitEvent(c->st, L.run_ev, 0);
  c->stats.graph_launches += 1;
  return cuda_check(c, "evolve graph launch");
}

int evolve_graph_finish(fdtd_context* c, Lat& L, EvolveRun& r) {
  int rc = read_state(c, L);
  if (rc) return rc;
  const int64_t ce = c->o.check_every;
  const LatState& hs = L.host_state;
  c->stats.launches += (int64_t)((hs.checks - r.check_id + 1) / 2) * L.graph_kernels;
  const int64_t advanced = std::max<int64_t>(0, (hs.active ? r.t_end : hs.step) - r.t);  // steps taken while active
  int64_t seg_l, seg_u;
  double seg_b;
  segment_work(c, L, ce, &seg_l, &seg_b, &seg_u);
  c->stats.stencil_launches += advanced / ce * seg_l;
  c->stats.stencil_site_updates += advanced / ce * seg_u;
  c->stats.stencil_bytes += (double)(advanced / ce) * seg_b;
  L.sums_ready = check_step_fused(c, L);  // the body ends with a check step
  if (!hs.active) {
    r.done = true;
  } else {
    r.t = r.t_end;
    r.check_id = hs.checks;
  }
  return FDTD_OK;
}

int evolve_tail(fdtd_context* c, Lat& L, int64_t max_steps, EvolveRun& r) {
  const int64_t ce = c->o.check_every;
  int groups = 2;
  int prev_checks = 0;
  double prev_delta = -1.0;
  while (!r.done) {
    for (int g = 0; g < groups && !r.done; ++g) {
      enqueue_check(c, L, r.check_id++, r.t);
      if (r.t >= max_steps) {
        r.done = true;
        break;
      }
      int64_t nst = std::min<int64_t>(ce, max_steps - r.t);
      run_steps(c, L, nst, &L.state[0].active, r.t, true);
      r.t += nst;
    }
    int rc = cuda_check(c, "evolve launch");
    if (rc) return rc;
    rc = read_state(c, L);
    if (rc) return rc;
    if (!L.host_state.active) r.done = true;
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

// Every lattice of a (non-batched) handle.  The graph loops of all lattices
// are launched together, each on its own stream, so independent lattices
// share the GPU (the small ones leave most of it idle on their own); every
// lattice computes the same bits as when evolved alone.
int evolve_lattices(fdtd_context* c, int64_t max_steps) {
  cudaMemsetAsync(c->flags + 1, 0, sizeof(int32_t), c->st);
  std::vector<EvolveRun> runs(c->lats.size());
  int rc = FDTD_OK;
  // every capture and autotuning pass (which times launches) before any loop runs
  for (size_t i = 0; i < c->lats.size(); ++i)
    if ((rc = evolve_begin(c, c->lats[i], max_steps, runs[i]))) return rc;
  bool any = false;
  for (const auto& r : runs) any = any || r.graph;
  if (any) {
    if (!c->ev_in && cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess) {
      c->ev_in = nullptr;
      return cuda_check(c, "evolve event");
    }
    cudaEventRecord(c->ev_in, c->st);
    for (size_t i = 0; i < c->lats.size(); ++i)
      if (runs[i].graph && (rc = evolve_graph_launch(c, c->lats[i], c->ev_in))) return rc;
    for (size_t i = 0; i < c->lats.size(); ++i)
      if (runs[i].graph && (rc = evolve_graph_finish(c, c->lats[i], runs[i]))) return rc;
  }
  for (size_t i = 0; i < c->lats.size(); ++i)
    if ((rc = evolve_tail(c, c->lats[i], max_steps, runs[i]))) return rc;
  return FDTD_OK;
}

// Batched configurations already chosen, by device and lattice sizes.
std::mutex g_btune_mu;
std::map<std::pair<int, std::vector<int>>, std::pair<int, int>> g_btune;

// All lattices of the handle in one persistent launch.  With autotuning on
// (and no depth given) the first evolve of a new set of lattice sizes times
// every (depth 1..3, tile 64x16 / 128x16 / 64x32) candidate on update passes that
// write the spare fields (the state does not advance, so every candidate
// does the same work), caches the fastest and runs the evolve with it.
// Every candidate computes the same bits.
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
  std::vector<std::pair<int, int>> cands;  // (depth, tile kind: 64x16, 128x16, 64x32)
  if (c->o.temporal_depth > 0 || !c->o.autotune) {
    int kind;
    if (c->o.tile_y == 32) {
      kind = 2;
    } else if (c->o.tile_x) {
      kind = c->o.tile_x == 128 ? 1 : 0;
    } else {  // 128 wide if most sites lie in lattices of 96 or more sites per axis
      double big = 0.0, all = 0.0;
      for (auto& L : c->lats) {
        all += (double)L.n3;
        if (L.d.n >= 96) big += (double)L.n3;
      }
      kind = 2.0 * big > all ? 1 : 0;
    }
    cands.push_back({c->o.temporal_depth > 0 ? c->o.temporal_depth : 2, kind});
  } else {
    std::lock_guard<std::mutex> lock(g_btune_mu);
    auto it = g_btune.find(key);
    if (it != g_btune.end()) {
      cands.push_back(it->second);
    } else {
      for (int kind = 0; kind < kBatchedTileKinds; ++kind)
        for (int d = 1; d <= 3; ++d) cands.push_back({d, kind});
    }
  }
  for (auto& L : c->lats) {
    launch_state_reset(&L.state[0], 0, c->st);
    c->stats.launches += 1;
  }
  cudaMemsetAsync(c->flags + 1, 0, sizeof(int32_t), c->st);
  // the table: tensor maps encoded once per handle, mask and field index patched per evolve
  const size_t eb = batched_entry_bytes();
  if (c->batch_table.size() != eb * count + 64) {
    c->batch_table.assign(eb * count + 64, 0);
    char* base = c->batch_table.data() + ((64 - ((uintptr_t)c->batch_table.data() & 63)) & 63);
    for (int l = 0; l < count; ++l) {
      Lat& L = c->lats[l];
      if (batched_fill(base + l * eb, (const float*)L.psi[0], (const float*)L.psi[1], (const float*)L.v, L.partials,
                       &L.state[0], L.hist, L.p, L.mask, L.cur, L.d.v_inf)) {
        c->batch_table.clear();
        return fail(c, FDTD_ERR_CUDA, "evolve: could not encode the batched tensor maps");
      }
    }
  }
  char* base = c->batch_table.data() + ((64 - ((uintptr_t)c->batch_table.data() & 63)) & 63);
  for (int l = 0; l < count; ++l) batched_patch(base + l * eb, c->lats[l].mask, c->lats[l].cur);
  cudaMemcpyAsync(c->batch_ws, base, eb * count, cudaMemcpyHostToDevice, c->st);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int64_t steps = 0;
  int grid = 0;
  int rc = FDTD_OK;
  auto launch = [&](std::pair<int, int> cd, int tune_passes) -> int {
    int e = batched_launch(c->batch_ws, count, max_steps, 0, max_steps, 0, 0, (int)ce, c->o.tol, c->o.tol_relative,
                           c->o.reimpose_parity, cd.first, cd.second, tune_passes, c->flags + 1, c->st,
                           &c->batch_graphs, &steps, &grid);
    if (e) return fail(c, FDTD_ERR_CUDA, std::string("evolve (batched): ") + cudaGetErrorString((cudaError_t)e));
    c->stats.launches += 1;
    c->stats.graph_launches += 1;
    return FDTD_OK;
  };
  std::pair<int, int> best = cands[0];
  if (cands.size() > 1) {
    Range r("batched autotune");
    double best_rate = -1.0;
    double sites = 0.0;
    for (auto& L : c->lats) sites += (double)L.n3;
    constexpr int kPasses = 4;
    for (auto cd : cands) {
      int e = batched_prepare(c->batch_ws, count, cd.first, cd.second, c->flags + 1, &c->batch_graphs);
      if (e) {
        cudaGetLastError();
        continue;  // a configuration that cannot be made resident is skipped
      }
      if ((rc = launch(cd, 1))) break;  // first launch of the graph: not timed
      cudaEventRecord(e0, c->st);
      if ((rc = launch(cd, kPasses))) break;
      cudaEventRecord(e1, c->st);
      cudaEventSynchronize(e1);
      if ((rc = cuda_check(c, "evolve (batched autotune)"))) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double rate = ms > 0.f ? sites * cd.first * kPasses / ms : 0.0;
      if (rate > best_rate) {
        best_rate = rate;
        best = cd;
      }
    }
    int32_t expired = 0;  // timings of launches whose waits expired are not kept
    if (!rc) {
      cudaMemcpyAsync(&expired, c->flags + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st);
      cudaStreamSynchronize(c->st);
    }
    if (!rc && !expired && best_rate > 0.0) {
      std::lock_guard<std::mutex> lock(g_btune_mu);
      g_btune[key] = best;
    }
  }
  if (!rc) {
    cudaEventRecord(e0, c->st);
    rc = launch(best, 0);
    cudaEventRecord(e1, c->st);
  }
  if (!rc) rc = cuda_check(c, "evolve (batched)");
  std::vector<int64_t> step_at(count, 0);  // steps each lattice advanced while active
  for (int l = 0; !rc && l < count; ++l) {
    Lat& L = c->lats[l];
    if ((rc = read_state(c, L))) break;
    if (L.host_state.status == STATUS_NONFINITE) {
      rc = fail(c, FDTD_ERR_NONFINITE, "non-finite or vanishing norm during evolve");
      break;
    }
    L.cur = L.host_state.cur;
    step_at[l] = L.host_state.active ? steps : L.host_state.step;
  }
  if (!rc && c->profiling) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    c->stats.stencil_ms += ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  // the persistent launch is the stencil launch of a batched evolve
  for (int l = 0; l < count; ++l) {
    Lat& L = c->lats[l];
    L.last_steps = L.host_state.converged ? L.host_state.step : max_steps;
    c->stats.stencil_site_updates += (int64_t)L.n3 * step_at[l];
    c->stats.stencil_bytes += (double)L.n3 * 12.0 * ((step_at[l] + best.first - 1) / best.first);
  }
  c->stats.stencil_launches += 1;
  if (c->profiling) c->stats.stencil_timed_launches += 1;
  c->batch_depth = best.first;
  c->batch_kind = best.second;
  return FDTD_OK;
}

}  // namespace api
}  // namespace fdtd

extern "C" {

int fdtd_evolve(fdtd_handle h, int64_t max_steps, int64_t* steps_done) {
  Range r("fdtd_evolve");
  if (!h) return FDTD_ERR_INVALID_ARG;
  if (max_steps < 0) return fail(h, FDTD_ERR_INVALID_ARG, "evolve: max_steps < 0");
  int rc = resolve_potentials(h);
  if (rc) return rc;
  for (auto& L : h->lats)
    if (!L.has_v || !L.has_psi) return fail(h, FDTD_ERR_STATE, "evolve: set_potential and init/set_psi first");
  if (h->o.batched) {
    rc = evolve_batched(h, max_steps);
  } else {
    rc = evolve_lattices(h, max_steps);
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

}  // extern "C"
