// Internal interface of the C ABI implementation (api_*.cu): the per-handle
// context, the per-lattice view of the caller's workspace, and the host-side
// helpers the entry points share.  Not installed; include/fdtd.h is the
// public interface.
//
// The library never allocates device memory: every buffer is a slice of the
// caller's workspace.  Per lattice the workspace holds two psi fields
// (ping-pong), V (plus A and cB for FP64 lattices), the block partials of
// the lattice sums, two state records, the check history, and -- when
// backward storage was requested -- the start field, the sqrt(T) checkpoint
// pool, one segment of recomputed fields, two adjoint fields and the FP64
// gradient accumulator; snapshot slots when requested.
#pragma once
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


namespace fdtd {
namespace api {

extern thread_local std::string g_create_err;  // message of a call that has no handle

constexpr size_t kStagingBytes = 8u << 20;

inline bool is_complex(int prec) { return prec == FDTD_C64 || prec == FDTD_C32; }
// bytes of one site of a field of precision prec (complex: an (re, im) pair)
inline size_t elem_bytes(int prec) {
  switch (prec) {
    case FDTD_F64: return 8;
    case FDTD_F32: return 4;
    case FDTD_C64: return 16;
    case FDTD_C32: return 8;
    default: return 2;
  }
}
// bytes per site of the coefficients a step reads besides psi: V (FP32, BF16
// storage), A and cB (FP64: two doubles; complex: two pairs)
inline double coef_bytes(int prec) {
  return prec == FDTD_F64 ? 16.0 : (is_complex(prec) ? 2.0 * (double)elem_bytes(prec) : 4.0);
}
// sums per block of the lattice's partials (S0, SH, Sr, SV; complex: SH and SV with imaginary parts)
inline int sums_per_block(int prec) { return is_complex(prec) ? 6 : 4; }

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
  bool v_pending = false;  // V enqueued by fdtd_set_potential_async, its checks not yet read
  // backward storage
  void* psi0 = nullptr;
  int64_t bw_T = 0;
  int bw_K = 0;
  int64_t bw_npool = 0;
  void* pool = nullptr;
  void* seg = nullptr;
  void* lam[2] = {nullptr, nullptr};
  void* bw_u = nullptr;    // B lam of the split FP64 adjoint step
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
  bool tma_ok = false;   // FP32 lattice with TMA maps (stencil, sums, batched)
  bool tma16 = false;    // BF16 lattice with TMA stencil maps (BF16 psi boxes, FP32 V boxes)
  bool sums_ready = false;  // partials hold the sums of psi[cur] (written by the last check step)
  CUtensorMap maps[2][3][3];
  CUtensorMap sums_maps[3];
  // stencil configuration: depth, tile width, z-planes per block (0 = not chosen yet);
  // plain = a one-step kernel (bit-identical) was timed fastest: the
  // z-marching one, or the direct four-site one when direct is set
  int depth = 0, tx = 128, zc = 0;
  bool plain = false, direct = false;
  // evolve graphs: a while loop over pairs of (check, check_every steps),
  // one per start buffer (an evolve ends on either), each built for a mask,
  // stencil configuration and cadence
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
  int64_t graph_key[2][6] = {{-1, -1, -1, -1, -1, -1}, {-1, -1, -1, -1, -1, -1}};
  int64_t graph_kernels = 0;  // kernels per loop iteration
  // the lattice's own stream for its graph loop (lattices of a handle run
  // concurrently) and the event that orders the handle's stream after it
  cudaStream_t run_st = nullptr;
  cudaEvent_t run_ev = nullptr;
};

void release_graph(Lat& L, int b);
void release_graph(Lat& L);
// Read the checks of every potential enqueued without waiting
// (fdtd_set_potential_async) on handle c: one stream synchronisation; the
// lattices become usable (has_v) or the error is returned.  No-op when none
// is pending.
int resolve_potentials(fdtd_context* c);

}  // namespace api
}  // namespace fdtd

struct fdtd_context {
  std::vector<fdtd::api::Lat> lats;
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
  fdtd::BatchedGraphs batch_graphs;     // graphs of the batched persistent launch
  int batch_depth = 0, batch_kind = 0;  // configuration of the last batched evolve (depth, tile kind)
  std::vector<char> batch_table;      // host copy of the batched driver's table (maps encoded once)
  cudaStream_t cap_st = nullptr;  // private stream the evolve graphs are captured on
  cudaEvent_t ev_in = nullptr;    // orders the lattices' graph loops after the handle's stream
  // stencil launches not yet credited to the stats: a launch enqueued past
  // the check at which its lattice converged runs as a no-op and is dropped
  struct Pending {  // a run of consecutive stencil launches of one depth
    int64_t t_start, updates;
    double bytes;
    long ev;  // index of the run's start event, or -1
    int64_t launches;
  };
  std::vector<Pending> pending;
};

namespace fdtd {
namespace api {

// NVTX range for profilers (header-only NVTX3: no cost without a tool attached)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

int fail(fdtd_context* c, int code, const std::string& msg);
int cuda_check(fdtd_context* c, const char* where);
int lat_check(fdtd_context* c, int lat);

// profiling of the stencil launches (CUDA events around each, when on)
long prof_begin(fdtd_context* c);
void prof_end(fdtd_context* c);
void flush_pending(fdtd_context* c, int64_t cutoff);
void prof_collect(fdtd_context* c);

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
// the scalar type of a complex lattice's (re, im) pairs
template <typename F>
void with_ctype(int prec, F&& f) {
  if (prec == FDTD_C64)
    f((double*)nullptr);
  else
    f((float*)nullptr);
}

// stencil configuration, steps, checks and evolves (api_evolve.cu)
void choose_config(fdtd_context* c, Lat& L);
void run_steps(fdtd_context* c, Lat& L, int64_t count, const int32_t* active, int64_t t0 = 0,
               bool before_check = false);
int launch_sums_any(fdtd_context* c, Lat& L, const void* psi, const int32_t* active);
void scale_parity_any(fdtd_context* c, Lat& L, const void* in, void* out, int mask, const LatState* s, int id,
                      int out_idx, LatState* sw);
int read_state(fdtd_context* c, Lat& L);
int evolve_lattices(fdtd_context* c, int64_t max_steps);
int evolve_batched(fdtd_context* c, int64_t max_steps);

// fields and records (api_core.cu)
void fill_obs(const Lat& L, const LatState& s, fdtd_obs* out);
int import_field(fdtd_context* c, const void* src, int dt, int mem, void* dst, int prec, size_t n3);
int export_field(fdtd_context* c, const void* src, int prec, void* dst, int dt, int mem, size_t n3);
int valid_mask(int mask);
void record_start(fdtd_context* c, Lat& L);

}  // namespace api
}  // namespace fdtd
