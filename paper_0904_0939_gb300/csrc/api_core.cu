// C ABI entry points of the solver (include/fdtd.h): options, workspace
// carving and handle creation, potentials and fields, checks and
// observables, the multi-resolution transfer, statistics.
#include "api_internal.cuh"

using namespace fdtd;
using namespace fdtd::api;

namespace fdtd {
namespace api {

thread_local std::string g_create_err;

}  // namespace api

// Message for fdtd_last_error(NULL) from entry points that take no handle.
void set_detached_error(const std::string& msg) { api::g_create_err = msg; }

}  // namespace fdtd

namespace {

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
  if (d.precision != FDTD_F64 && d.precision != FDTD_F32 && d.precision != FDTD_BF16 && d.precision != FDTD_C64 &&
      d.precision != FDTD_C32) {
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
  if (o.zchunk < -2) {
    err = "zchunk must be >= -2";
    return FDTD_ERR_INVALID_ARG;
  }
  if (o.autotune < 0 || o.autotune > 1) {
    err = "autotune must be 0 or 1";
    return FDTD_ERR_INVALID_ARG;
  }
  if (o.tile_x != 0 && o.tile_x != 64 && o.tile_x != 128) {
    err = "tile_x must be 0, 64 or 128";
    return FDTD_ERR_INVALID_ARG;
  }
  if ((o.tile_y != 0 && o.tile_y != 16 && o.tile_y != 32) || (o.tile_y == 32 && o.tile_x == 128)) {
    err = "tile_y must be 0, 16 or 32 (32 with 64-wide tiles only)";
    return FDTD_ERR_INVALID_ARG;
  }
  if (o.stencil_kernel < 0 || o.stencil_kernel > 2) {
    err = "stencil_kernel must be 0, 1 or 2";
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
    const bool cplx = is_complex(d[l].precision);
    if (d[l].precision == FDTD_F64 || cplx) {
      // FP64: V, A, cB as doubles; complex: V, A, cB as (re, im) pairs of the lattice's scalar
      L.v = cv.take(L.n3 * L.es);
      L.coefA = (double*)cv.take(L.n3 * L.es);
      L.coefCB = (double*)cv.take(L.n3 * L.es);
    } else {
      L.v = cv.take(L.n3 * 4);
    }
    L.nparts = cplx ? csums_blocks(d[l].n) : std::max(sums_blocks(d[l].n), tma_sums_blocks(d[l].n));
    L.partials = (double*)cv.take((size_t)L.nparts * sums_per_block(d[l].precision) * sizeof(double));
    L.state = (LatState*)cv.take(2 * sizeof(LatState));
    L.hist = (double*)cv.take((size_t)kHistCap * kHistFields * sizeof(double));
    if (o.backward_steps > 0 && d[l].precision != FDTD_BF16 && !cplx) {
      L.bw_T = o.backward_steps;
      L.bw_K = (int)std::ceil(std::sqrt((double)o.backward_steps));
      L.bw_npool = (L.bw_T + L.bw_K - 1) / L.bw_K;
      L.psi0 = cv.take(L.n3 * L.es);
      L.pool = cv.take((size_t)L.bw_npool * L.n3 * L.es);
      L.seg = cv.take((size_t)L.bw_K * L.n3 * L.es);
      L.lam[0] = cv.take(L.n3 * L.es);
      L.lam[1] = cv.take(L.n3 * L.es);
      if (d[l].precision == FDTD_F64) L.bw_u = cv.take(L.n3 * L.es);  // FP32: one adjoint pass per step
      L.bw_nraw = (L.bw_K - 1) / o.check_every + 2;  // check steps inside a segment + its last step
      L.bw_raw = cv.take((size_t)L.bw_nraw * L.n3 * L.es);
      L.gv = (double*)cv.take(L.n3 * 8);
      L.scales = (double*)cv.take((size_t)(L.bw_T / o.check_every + 2) * sizeof(double));
    }
    if (o.snapshots > 0 && !cplx) {
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
namespace api {

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
// Credit the pending runs of stencil launches that started before step
// `cutoff` (call after a stream synchronisation).
void flush_pending(fdtd_context* c, int64_t cutoff) {
  for (const auto& p : c->pending) {
    if (p.t_start >= cutoff) continue;
    c->stats.stencil_launches += p.launches;
    c->stats.stencil_site_updates += p.updates;
    c->stats.stencil_bytes += p.bytes;
    float ms = 0.f;
    if (p.ev >= 0 && cudaEventElapsedTime(&ms, c->ev[p.ev], c->ev[p.ev + 1]) == cudaSuccess) {
      c->stats.stencil_ms += ms;
      c->stats.stencil_timed_launches += p.launches;
    }
  }
  c->pending.clear();
  c->ev_used = 0;
}
void prof_collect(fdtd_context* c) { flush_pending(c, INT64_MAX); }

void fill_obs(const Lat& L, const LatState& s, fdtd_obs* out) {
  std::memset(out, 0, sizeof(*out));
  out->energy = s.energy;
  out->binding_energy = s.ebind;
  out->norm = s.s0 * L.p.a * L.p.a * L.p.a;
  out->r2 = s.r2;
  out->r_rms = std::sqrt(std::max(0.0, s.r2));
  out->v_expect = s.vexp;
  out->delta_e = s.delta_e;
  out->energy_imag = s.energy_im;
}

// Copy n3 elements of dtype `dt` from user memory into a typed device
// buffer of lattice precision `prec` (through the staging buffer for host
// memory).
int import_field(fdtd_context* c, const void* src, int dt, int mem, void* dst, int prec, size_t n3) {
  if (is_complex(prec)) {  // a complex field is 2 n3 interleaved scalars
    n3 *= 2;
    dt = dt == FDTD_C64 ? FDTD_F64 : FDTD_F32;
    prec = prec == FDTD_C64 ? FDTD_F64 : FDTD_F32;
  }
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
    // a host input is borrowed for the call only: from pinned memory the
    // copies above are asynchronous, so wait until they have read it
    cudaStreamSynchronize(c->st);
  }
  return cuda_check(c, "import");
}

int export_field(fdtd_context* c, const void* src, int prec, void* dst, int dt, int mem, size_t n3) {
  if (is_complex(prec)) {  // a complex field is 2 n3 interleaved scalars
    n3 *= 2;
    dt = dt == FDTD_C64 ? FDTD_F64 : FDTD_F32;
    prec = prec == FDTD_C64 ? FDTD_F64 : FDTD_F32;
  }
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

int valid_mask(int mask) {
  if (mask < 0 || mask >= 64) return 0;
  for (int ax = 0; ax < 3; ++ax)
    if (((mask >> (2 * ax)) & 3) == 3) return 0;
  return 1;
}

void record_start(fdtd_context* c, Lat& L) {
  if (L.psi0) {
    cudaMemcpyAsync(L.psi0, L.psi[L.cur], L.n3 * L.es, cudaMemcpyDeviceToDevice, c->st);
    L.has_psi0 = true;
  }
}

}  // namespace api
}  // namespace fdtd

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
  {
    fdtd_options oo;
    if (o)
      oo = *o;
    else
      fdtd_default_options(&oo);
    for (int l = 0; l < count; ++l)
      if (is_complex(d[l].precision) && (oo.boundary != 0 || oo.batched)) {
        g_create_err = "complex lattices need zero boundaries and a non-batched handle";
        return FDTD_ERR_INVALID_ARG;
      }
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
    } else if (L.d.precision == FDTD_BF16 && L.d.n % 8 == 0 && L.d.n >= 8 && !L.p.periodic) {
      // BF16 storage: the temporally blocked stencil with BF16 psi boxes
      // (x start a multiple of 8 sites) and FP32 V boxes
      bool ok = true;
      int bw, bh;
      for (int ti = 0; ti < 2; ++ti)
        for (int k = 1; k <= blocked_max_depth(); ++k) {
          tma_box_bf16(k, ti ? 128 : 64, &bw, &bh);
          for (int b = 0; b < 2; ++b)
            ok = ok && encode_field_map_bf16(&L.maps[ti][k - 1][b], (const __nv_bfloat16*)L.psi[b], L.d.n, bw, bh) == 0;
          tma_box(k, ti ? 128 : 64, &bw, &bh);
          ok = ok && encode_field_map(&L.maps[ti][k - 1][2], (const float*)L.v, L.d.n, bw, bh) == 0;
        }
      L.tma16 = ok;
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
  for (auto& L : h->lats) {
    release_graph(L);
    if (L.run_st) {
      cudaStreamSynchronize(L.run_st);
      cudaStreamDestroy(L.run_st);
    }
    if (L.run_ev) cudaEventDestroy(L.run_ev);
  }
  h->batch_graphs.release();
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
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

}  // extern "C"

namespace fdtd {
namespace api {
namespace {
// Enqueue V's conversion (or copy) and its checks on the handle's stream;
// the check bits accumulate in flags[0] until resolve_potentials reads them.
int enqueue_potential(fdtd_handle h, int lat, const void* v, int dtype, int mem_kind) {
  int rc = lat_check(h, lat);
  if (rc) return rc;
  const bool cplx_in = dtype == FDTD_C64 || dtype == FDTD_C32;
  if (!v || (dtype != FDTD_F64 && dtype != FDTD_F32 && !cplx_in) ||
      (mem_kind != FDTD_MEM_HOST && mem_kind != FDTD_MEM_DEVICE))
    return fail(h, FDTD_ERR_INVALID_ARG, "set_potential: null pointer, bad dtype or mem_kind");
  Lat& L = h->lats[lat];
  if (cplx_in && !is_complex(L.d.precision))
    return fail(h, FDTD_ERR_INVALID_ARG, "set_potential: a complex potential needs a complex lattice (FDTD_C64/C32)");
  bool pending = false;
  for (const Lat& o : h->lats) pending = pending || o.v_pending;
  if (!pending) cudaMemsetAsync(h->flags, 0, sizeof(int32_t), h->st);
  L.has_v = false;
  L.v_pending = true;
  if (is_complex(L.d.precision)) {
    // V, A and cB of a complex lattice (real input: V_I = 0)
    const bool in64 = dtype == FDTD_F64 || dtype == FDTD_C64;
    const size_t isz = (in64 ? 8 : 4) * (cplx_in ? 2 : 1);
    auto cconv = [&](const void* src, size_t cnt, size_t off) {
      with_ctype(L.d.precision, [&](auto* tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        launch_cset_potential<T>(src, in64, cplx_in, cnt, off, (T*)L.v, (T*)L.coefA, (T*)L.coefCB, L.p, h->flags,
                                 h->st);
      });
      h->stats.launches += 1;
    };
    if (mem_kind == FDTD_MEM_DEVICE) {
      cconv(v, L.n3, 0);
    } else {
      const size_t chunk = kStagingBytes / isz;
      for (size_t off = 0; off < L.n3; off += chunk) {
        size_t cnt = std::min(chunk, L.n3 - off);
        cudaMemcpyAsync(h->staging, (const char*)v + off * isz, cnt * isz, cudaMemcpyHostToDevice, h->st);
        cconv(h->staging, cnt, off);
      }
    }
  }
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
  if (is_complex(L.d.precision)) {
    // done above
  } else if (mem_kind == FDTD_MEM_DEVICE) {
    conv(v, L.n3, 0);
  } else if (vf && dtype == FDTD_F32) {
    // FP32 into an FP32/BF16 lattice's FP32 V: one copy straight into place
    // (full host-link bandwidth from pinned memory), then the checks
    cudaMemcpyAsync(vf, v, L.n3 * sizeof(float), cudaMemcpyHostToDevice, h->st);
    launch_guard_potential_f32(vf, L.n3, L.p, h->flags, h->st);
    h->stats.launches += 1;
  } else {
    const size_t chunk = kStagingBytes / isz;
    for (size_t off = 0; off < L.n3; off += chunk) {
      size_t cnt = std::min(chunk, L.n3 - off);
      cudaMemcpyAsync(h->staging, (const char*)v + off * isz, cnt * isz, cudaMemcpyHostToDevice, h->st);
      conv(h->staging, cnt, off);
    }
  }
  return cuda_check(h, "set_potential");
}
}  // namespace

int resolve_potentials(fdtd_context* c) {
  bool pending = false;
  for (const Lat& o : c->lats) pending = pending || o.v_pending;
  if (!pending) return FDTD_OK;
  int32_t flags = 0;
  cudaMemcpyAsync(&flags, c->flags, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st);
  cudaError_t e = cudaStreamSynchronize(c->st);
  for (Lat& o : c->lats) {
    if (!o.v_pending) continue;
    o.v_pending = false;
    o.has_v = e == cudaSuccess && (flags & 3) == 0;
  }
  if (e != cudaSuccess) return fail(c, FDTD_ERR_CUDA, std::string("set_potential: ") + cudaGetErrorString(e));
  if (flags & 1) return fail(c, FDTD_ERR_NONFINITE, "set_potential: NaN or Inf in V");
  if (flags & 2) return fail(c, FDTD_ERR_UNSTABLE_DT, "set_potential: 1 + dtau Re V / 2 <= 0 at some site");
  return FDTD_OK;
}

}  // namespace api
}  // namespace fdtd

extern "C" {

int fdtd_set_potential(fdtd_handle h, int lat, const void* v, int dtype, int mem_kind) {
  int rc = fdtd::api::enqueue_potential(h, lat, v, dtype, mem_kind);
  if (rc) return rc;
  return fdtd::api::resolve_potentials(h);
}

int fdtd_set_potential_async(fdtd_handle h, int lat, const void* v, int dtype, int mem_kind) {
  return fdtd::api::enqueue_potential(h, lat, v, dtype, mem_kind);
}

int fdtd_init_symmetric(fdtd_handle h, int lat, uint64_t seed, int parity_mask, int dist) {
  int rc = lat_check(h, lat);
  if (rc) return rc;
  if (!valid_mask(parity_mask) || (dist != FDTD_DIST_UNIFORM && dist != FDTD_DIST_GAUSSIAN))
    return fail(h, FDTD_ERR_INVALID_ARG, "init_symmetric: bad parity mask or distribution");
  Lat& L = h->lats[lat];
  if (is_complex(L.d.precision)) {
    with_ctype(L.d.precision, [&](auto* tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      launch_cinit_random<T>((T*)L.psi[0], L.d.n, seed, (uint64_t)lat, dist, h->st);
    });
  } else {
    with_type(L.d.precision, [&](auto* tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      launch_init_random<T>((T*)L.psi[0], L.d.n, seed, (uint64_t)lat, dist, h->st);
    });
  }
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
  if (!psi || (dtype != FDTD_F64 && dtype != FDTD_F32 && dtype != FDTD_C64 && dtype != FDTD_C32) ||
      (mem_kind != FDTD_MEM_HOST && mem_kind != FDTD_MEM_DEVICE) || !valid_mask(parity_mask))
    return fail(h, FDTD_ERR_INVALID_ARG, "set_psi: null pointer, bad dtype, mem_kind or mask");
  Lat& L = h->lats[lat];
  if (is_complex(dtype) != is_complex(L.d.precision))
    return fail(h, FDTD_ERR_INVALID_ARG, "set_psi: complex lattices take complex fields (FDTD_C64/C32), real ones real");
  if ((rc = import_field(h, psi, dtype, mem_kind, L.psi[L.cur], L.d.precision, L.n3))) return rc;
  L.mask = parity_mask;
  L.has_psi = true;
  record_start(h, L);
  return cuda_check(h, "set_psi");
}

int fdtd_get_psi(fdtd_handle h, int lat, void* psi, int dtype, int mem_kind) {
  int rc = lat_check(h, lat);
  if (rc) return rc;
  if (!psi || (dtype != FDTD_F64 && dtype != FDTD_F32 && dtype != FDTD_C64 && dtype != FDTD_C32) ||
      (mem_kind != FDTD_MEM_HOST && mem_kind != FDTD_MEM_DEVICE))
    return fail(h, FDTD_ERR_INVALID_ARG, "get_psi: null pointer, bad dtype or mem_kind");
  Lat& L = h->lats[lat];
  if (is_complex(dtype) != is_complex(L.d.precision))
    return fail(h, FDTD_ERR_INVALID_ARG, "get_psi: complex lattices give complex fields (FDTD_C64/C32), real ones real");
  if (!L.has_psi) return fail(h, FDTD_ERR_STATE, "get_psi: no wavefunction yet");
  return export_field(h, L.psi[L.cur], L.d.precision, psi, dtype, mem_kind, L.n3);
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
  if ((rc = resolve_potentials(h))) return rc;
  if (!L.has_v || !L.has_psi) return fail(h, FDTD_ERR_STATE, "observables: set_potential and init/set_psi first");
  int np = launch_sums_any(h, L, L.psi[L.cur], nullptr);
  launch_state_reset(&L.state[1], 0, h->st);
  launch_finalize(&L.state[1], L.partials, np, 0, 0, L.p, L.d.v_inf, 0.0, 0, 1, h->st, 0, 0, nullptr, nullptr,
                  sums_per_block(L.d.precision));
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
  if ((rc = resolve_potentials(dst))) return rc;
  if (!D.has_v) return fail(dst, FDTD_ERR_STATE, "upsample: set the destination potential first");
  if (is_complex(S.d.precision) != is_complex(D.d.precision))
    return fail(dst, FDTD_ERR_INVALID_ARG, "upsample: both lattices complex or both real");
  if (src->st != dst->st) {
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, src->st);
    cudaStreamWaitEvent(dst->st, ev, 0);
    cudaEventDestroy(ev);
  }
  void* tmp = D.psi[1 - D.cur];
  if (is_complex(S.d.precision)) {
    with_ctype(S.d.precision, [&](auto* tin) {
      using Ti = std::remove_pointer_t<decltype(tin)>;
      with_ctype(D.d.precision, [&](auto* tout) {
        using To = std::remove_pointer_t<decltype(tout)>;
        launch_cupsample<Ti, To>((const Ti*)S.psi[S.cur], S.d.n, (To*)tmp, dst->st);
      });
    });
  } else {
    with_type(S.d.precision, [&](auto* tin) {
      using Ti = std::remove_pointer_t<decltype(tin)>;
      with_type(D.d.precision, [&](auto* tout) {
        using To = std::remove_pointer_t<decltype(tout)>;
        launch_upsample<Ti, To>((const Ti*)S.psi[S.cur], S.d.n, (To*)tmp, D.p.periodic, dst->st);
      });
    });
  }
  dst->stats.launches += 1;
  // renormalise and give the field the source's symmetry (Sec. VI)
  int id = 1000000 + (dst->check_seq++);
  int np = launch_sums_any(dst, D, tmp, nullptr);
  launch_state_reset(&D.state[1], 0, dst->st);
  launch_finalize(&D.state[1], D.partials, np, id, 0, D.p, D.d.v_inf, 0.0, 0, 0, dst->st, 0, 0, nullptr, nullptr,
                  sums_per_block(D.d.precision));
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

int fdtd_tuned_config(fdtd_handle h, int lat, int* depth, int* zchunk) {
  int rc = lat_check(h, lat);
  if (rc) return rc;
  if (!depth || !zchunk) return fail(h, FDTD_ERR_INVALID_ARG, "tuned_config: null output");
  Lat& L = h->lats[lat];
  if (h->o.batched && h->batch_depth) {  // the persistent launch's choice (balanced partition)
    *depth = h->batch_depth;
    *zchunk = -1;
    return FDTD_OK;
  }
  if ((rc = resolve_potentials(h))) return rc;
  if (L.has_v && L.has_psi) choose_config(h, L);
  *depth = L.depth;
  *zchunk = L.plain ? 0 : L.zc;
  return cuda_check(h, "tuned_config");
}

int fdtd_tuned_kernel(fdtd_handle h, int lat, int* tile_x, int* tile_y) {
  int rc = lat_check(h, lat);
  if (rc) return rc;
  if (!tile_x || !tile_y) return fail(h, FDTD_ERR_INVALID_ARG, "tuned_kernel: null output");
  Lat& L = h->lats[lat];
  *tile_x = *tile_y = 0;
  if (h->o.batched) {
    if (h->batch_depth) {
      *tile_x = batched_tile_x(h->batch_kind);
      *tile_y = batched_tile_y(h->batch_kind);
    }
    return FDTD_OK;
  }
  if ((rc = resolve_potentials(h))) return rc;
  if (L.has_v && L.has_psi) choose_config(h, L);
  if ((L.tma_ok || L.tma16) && h->o.stencil_kernel == 0 && !L.plain && L.depth > 0) {
    int bw = 0, bh = 0;
    tma_box(L.depth, L.tx, &bw, &bh);
    *tile_x = L.tx;
    *tile_y = bh - 2 * L.depth;
  }
  return cuda_check(h, "tuned_kernel");
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
