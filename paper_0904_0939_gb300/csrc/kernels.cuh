// Internal launch interface between the C ABI (api_*.cu) and the kernels.
#pragma once
#include <utility>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fdtd.h"

namespace fdtd {

// Per-lattice state kept in device memory: the check record of the last
// evolve, the pending renormalisation factor and the run flags.
struct LatState {
  double e_prev;    // binding energy of the previous check
  double s0, sh, sr, sv;
  double energy, ebind, r2, vexp, delta_e;
  double energy_im, vexp_im, e_prev_im;  // imaginary parts (complex lattices; 0 otherwise)
  double scale;     // 1 / sqrt(S0 a^3) of the last check
  int64_t step;     // t of the last check
  int32_t has_prev, active, converged, status;
  int32_t checks, scale_seq, cur;
  int32_t post;       // device-sequenced checks: 1 if the last finalize posted a factor
  int32_t seq_limit;  // device-sequenced checks: stop the loop before check seq_limit
  int32_t pad;
};

enum : int32_t { STATUS_OK = 0, STATUS_NONFINITE = 1 };

// Physical parameters a kernel needs, precomputed on the host.
struct Params {
  int n;
  double a, dtau, mass;
  double c;            // dtau / (2 m a^2)
  float half_dtau_f;   // dtau / 2 (FP32)
  float one_m6c_f;     // 1 - 6c (FP32)
  float c_f;           // c (FP32)
  int periodic;        // 1: periodic boundaries, 0: psi = 0 beyond the lattice
};

// Tiling of the z-marching kernels: 32 x 8 threads per block, one site per
// thread in x-y, each block walks `zc` planes.
struct Tiling {
  dim3 grid;
  int zc;
};
Tiling tiling_for(int n, int min_blocks);

// Launch with programmatic stream serialisation (the kernel must start with
// pdl_wait(), see common.cuh).
template <typename... Exp, typename... Act>
void launch_pdl(void (*k)(Exp...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Act&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, std::forward<Act>(args)...);
}

// ---- launchers (all asynchronous on `st`) -----------------------------------
// One update step psi_out = M psi_in (Eq. updateeq).
void launch_step_f64(const double* in, double* out, const double* coefA, const double* coefCB, const Params& p,
                     const int32_t* active, cudaStream_t st);
template <typename T>
void launch_step_f32(const T* in, T* out, const float* v, const Params& p, const int32_t* active, cudaStream_t st);

// TMA-streamed tile pipelines (k_tblock.cu / tma_item.cuh), FP32 lattices
// with n % 4 == 0: `depth` update steps per pass over HBM (tile width tx =
// 64 or 128), bit-identical to `depth` calls of launch_step_f32; and the
// lattice sums with one partial per 64 x 16 tile column.  *err |= 1 if a
// bounded wait expired.  A stencil launch gives each block `zc` consecutive
// tile planes of the column-major sequence of tma_tile_planes(n, tx) (a
// block's span may run on into the next tile column); tma_zchunk is the
// span that fills the device's resident blocks in one wave, and zc = 0
// takes it; zc < 0 is the balanced partition over one wave (each item's
// warm-up and drain steps counted, so that a block spanning two columns
// gets fewer planes).
bool tma_supported(int n, int precision);
int blocked_max_depth();
int auto_depth(int n, int precision);
long long tma_tile_planes(int n, int tx);
int tma_resident_blocks(int depth, int tx, bool bf16 = false);
int tma_zchunk(int n, int depth, int tx, bool bf16 = false);
// TMA box of a tile item: (tx + 8) x (ty + 2 depth) sites.
void tma_box(int depth, int tx, int* box_w, int* box_h, int ty = 16);
int encode_field_map(CUtensorMap* map, const float* base, int n, int box_w, int box_h);
int encode_field_map_nz(CUtensorMap* map, const float* base, int n, int nz, int box_w, int box_h);
// BF16 psi fields (n % 8 == 0): the box is (tx + 16) x (ty + 2 depth), its x
// start a multiple of 8 sites
int encode_field_map_bf16(CUtensorMap* map, const __nv_bfloat16* base, int n, int box_w, int box_h);
void tma_box_bf16(int depth, int tx, int* box_w, int* box_h, int ty = 16);
// `depth` steps on a z-slab field of n x n x nzbuf sites: own planes
// [zbase, zbase + nzo), halo planes around them, planes outside [zlo, zhi)
// beyond the lattice (tile width 128).
void launch_step_slab(const CUtensorMap& map_psi_in, const CUtensorMap& map_v, float* out, const Params& p, int depth,
                      int nzo, int zbase, int nzbuf, int zlo, int zhi, int32_t* err, cudaStream_t st);
// slab sums (k_tblock.cu): partials of S0, SH, Sr, SV over the own planes
// (the lattice sums' per-site arithmetic and partition), z measured from the
// lattice centre with own plane zbase at lattice plane z_first; maps with the
// 64-wide sums box.  Reduction and renormalisation (k_slab.cu): out4 = the
// partials added in order; out = factor * P_xy(in) on the own planes.
int slab_sums_blocks(int n, int nzo);
int launch_slab_sums(const CUtensorMap& map_psi, const CUtensorMap& map_v, const Params& p, int nzo, int zbase,
                     int z_first, double* partials, int32_t* err, cudaStream_t st);
void launch_slab_reduce(const double* partials, int nparts, double* out4, cudaStream_t st);
void launch_slab_scale(const float* in, float* out, int n, int nzo, int zbase, int mask_xy, double factor,
                       cudaStream_t st);
void launch_step_tma(const CUtensorMap& map_psi_in, const CUtensorMap& map_v, float* out, const Params& p, int depth,
                     int tx, int zc, const int32_t* active, int32_t* err, cudaStream_t st);
void launch_step_tma(const CUtensorMap& map_psi_in, const CUtensorMap& map_v, __nv_bfloat16* out, const Params& p,
                     int depth, int tx, int zc, const int32_t* active, int32_t* err, cudaStream_t st);
int tma_sums_blocks(int n);
// The check step (FP32, TMA lattices): one update step psi -> out (depth-2,
// 64-wide maps of the input field and V) and the partial sums of `out` as
// launch_sums_tma would write them (the same partials, bit for bit).
// Returns the number of partials.
int launch_step_sums_tma(const CUtensorMap& map_psi, const CUtensorMap& map_v, float* out, const Params& p,
                         double* partials, const int32_t* active, int32_t* err, cudaStream_t st);
int launch_sums_tma(const CUtensorMap& map_psi, const CUtensorMap& map_v, const Params& p, double* partials,
                    const int32_t* active, int32_t* err, cudaStream_t st);

// ---- batched persistent driver (k_batched.cu) ---------------------------------
// Device table of the batched driver for `count` lattices.
size_t batched_workspace_bytes(const fdtd_lattice_desc* d, int count);
int batched_max_lattices();
size_t batched_entry_bytes();
// Encodes the lattice's tensor maps (both tile widths, every depth, the
// sums box) into its table entry; batched_patch updates the fields that
// change between launches.
int batched_fill(void* host_entry, const float* psi0, const float* psi1, const float* v, double* partials,
                 LatState* state, double* hist, const Params& p, int mask, int cur, double v_inf);
void batched_patch(void* host_entry, int mask, int cur);
// Tile kinds of the batched update items: 64 x 16, 128 x 16, 64 x 32 sites.
constexpr int kBatchedTileKinds = 3;
inline int batched_tile_x(int kind) { return kind == 1 ? 128 : 64; }
inline int batched_tile_y(int kind) { return kind == 2 ? 32 : 16; }
// Instantiated CUDA graphs of the persistent launch, one per (tile kind,
// depth), owned by the handle (the kernel's arguments are the fixed table,
// run record and error flag, so a graph is reused by every evolve).
struct BatchedGraphs {
  cudaGraphExec_t exec[kBatchedTileKinds][4] = {};
  int grid[kBatchedTileKinds][4] = {};
  void release();
};
// Capture and instantiate the graph of (depth, tile kind) if not done yet.
int batched_prepare(void* dev_table, int count, int depth, int kind, int32_t* err, BatchedGraphs* graphs);
// One cooperative launch (through the cached graph) that runs every check
// and step of every lattice from step t_start to t_end (a multiple of
// check_every, or max_steps): the check at t_start is made unless
// skip_first, the one at t_end always; checks are numbered from check0.
// With tune_passes > 0 it instead runs that many update passes of `depth`
// steps from the current fields into the spare ones (the state does not
// advance).  Returns 0 or a cudaError_t value.  *steps_done is written
// asynchronously.
int batched_launch(void* dev_table, int count, int64_t max_steps, int64_t t_start, int64_t t_end, int skip_first,
                   int check0, int check_every, double tol, int tol_rel, int reimpose, int depth, int kind,
                   int tune_passes, int32_t* err, cudaStream_t st, BatchedGraphs* graphs, int64_t* steps_done,
                   int* grid_out);

// Lattice sums S0, SH, Sr, SV into per-block partials; returns block count.
template <typename T>
int launch_sums(const T* psi, const void* v, const Params& p, double* partials, const int32_t* active,
                cudaStream_t st);
int sums_blocks(int n);

// Reduce partials, compute E, E_b, <r^2>, the renormalisation factor and
// the convergence decision.  record = 0: only the scale (for upsample).
// Device-sequenced mode (seq_ce > 0, inside the evolve graph): the check
// number is s->checks and its step s->checks * seq_ce, s->post tells the
// following scale whether a factor was posted, and the graph's while
// condition `cond` is set to continue only while the lattice is active, no
// device-side wait has expired (*err == 0) and check + 1 < s->seq_limit.
// With hist, a recording check also writes its record {t, E, E_b, norm,
// <r^2>, <V>, |dE_b|, S0} to slot (checks - 1) % kHistCap of the lattice's
// history ring.
constexpr int kHistCap = 4096;
constexpr int kHistFields = 8;
// nsum = 4 for real lattices (S0, SH, Sr, SV per block), 6 for complex ones
// (S0, Re SH, Im SH, Sr, Re SV, Im SV): E and <V> then get imaginary parts
// and the convergence test uses the complex modulus of the change of E_b.
void launch_finalize(LatState* s, const double* partials, int nparts, int check_id, int64_t t, const Params& p,
                     double v_inf, double tol, int tol_rel, int record, cudaStream_t st, int seq_ce = 0,
                     cudaGraphConditionalHandle cond = 0, const int32_t* err = nullptr, double* hist = nullptr,
                     int nsum = 4);

// out = P(scale * in): renormalisation and symmetry re-imposition.  With
// s == nullptr the factor is 1 and the call is unconditional; otherwise it
// applies if s->scale_seq == check_id, or, for check_id < 0 (device-
// sequenced checks), if s->post == 1.
template <typename T>
void launch_scale_parity(const T* in, T* out, int n, int mask, const LatState* s, int check_id, int out_idx,
                         LatState* s_w, cudaStream_t st);

template <typename T>
void launch_init_random(T* out, int n, uint64_t seed, uint64_t lat, int dist, cudaStream_t st);

template <typename Ti, typename To>
void launch_upsample(const Ti* in, int nc, To* out, int periodic, cudaStream_t st);

template <typename Ti, typename To>
void launch_convert(const Ti* in, To* out, size_t count, cudaStream_t st);

// V (FP64 or FP32 input) -> lattice storage; flags[0] |= 1 nonfinite,
// flags[0] |= 2 unstable (1 + dtau V / 2 <= 0).  For FP64 lattices also
// A = (1-h)/(1+h) and cB = c / (1+h).
// checks of an FP32 potential copied into place (flags as launch_set_potential)
void launch_guard_potential_f32(const float* vf, size_t count, const Params& p, int32_t* flags, cudaStream_t st);
template <typename Ti>
void launch_set_potential(const Ti* in, size_t count, size_t offset, float* vf, double* vd, double* coefA,
                          double* coefCB, const Params& p, int32_t* flags, cudaStream_t st);

// mode 1: clear everything; mode 0: start of an evolve (keeps the scale);
// mode 2: only set seq_limit for device-sequenced checks.
void launch_state_reset(LatState* s, int mode, cudaStream_t st, int seq_limit = 0);

// Snapshot algebra (Sec. III / Sec. VI): block partials of <phi|psi> and
// <phi|phi> (returns the block count), the ratio on the device, and
// psi += (sign * coef[0] or alpha) * phi.
template <typename T>
int launch_dot2(const T* phi, const T* psi, size_t count, double* partials, cudaStream_t st);
void launch_ratio(const double* partials, int nparts, double* coef, cudaStream_t st);
template <typename T>
void launch_axpy(T* psi, const T* phi, const double* coef, double sign, double alpha, size_t count, cudaStream_t st);

// ---- complex potentials (k_complex.cu) ------------------------------------------
// Fields of complex lattices are interleaved (re, im) pairs of T (double or
// float); A and cB are formed once per site in FP64 from V.
int csums_blocks(int n);
template <typename T>
void launch_cset_potential(const void* in, int in_f64, int in_complex, size_t count, size_t off, T* v2, T* a2, T* cb2,
                           const Params& p, int32_t* flags, cudaStream_t st);
template <typename T>
void launch_cstep(const T* in, T* out, const T* a2, const T* cb2, const Params& p, const int32_t* active,
                  cudaStream_t st);
template <typename T>
int launch_csums(const T* psi, const T* v2, const Params& p, double* partials, const int32_t* active, cudaStream_t st);
template <typename T>
void launch_cscale_parity(const T* in, T* out, int n, int mask, const LatState* s, int check_id, int out_idx,
                          LatState* sw, cudaStream_t st);
template <typename T>
void launch_cinit_random(T* out, int n, uint64_t seed, uint64_t lat, int dist, cudaStream_t st);
template <typename Ti, typename To>
void launch_cupsample(const Ti* in, int nc, To* out, cudaStream_t st);

// ---- adjoint (k_adjoint.cu) ---------------------------------------------------
// Split adjoint step: u = B lam with the g_V accumulation (pointwise), then
// lam_out = A lam + c (Adj u - 6 u) (z-marching stencil over u).
template <typename T>
void launch_adjoint_pointwise(const T* lam, const T* psi_prev, const T* psi_next, const void* v, const double* coefCB,
                              T* u, double* gv, const Params& p, cudaStream_t st);
template <typename T>
void launch_adjoint_stencil(const T* u, const T* lam, T* lam_out, const void* v, const double* coefA, const Params& p,
                            cudaStream_t st);
// FP32 one-step stencil without z-march, four x sites per thread
// (n % 4 == 0): launch_step_f32's step, same bits
template <typename T>
void launch_direct(const T* in, T* out, const float* v, const Params& p, const int32_t* active, cudaStream_t st);
void launch_direct_f32(const float* in, float* out, const float* v, const Params& p, const int32_t* active,
                       cudaStream_t st);
// one whole FP32 adjoint step the same way (n % 4 == 0): u = B lam on load,
// lam_out = c Adj(u) + alpha u, g_V accumulation; same bits as
// launch_adjoint_step_f32
void launch_adjoint_direct_f32(const float* lam, const float* psi_prev, const float* psi_next, const float* v,
                               float* lam_out, double* gv, const Params& p, cudaStream_t st);
// one fused FP32 adjoint step (u = B lam, g_V accumulation, lam_out = M^T lam)
void launch_adjoint_step_f32(const float* lam, const float* psi_prev, const float* psi_next, const float* v,
                             float* lam_out, double* gv, const Params& p, cudaStream_t st);
template <typename T>
void launch_adjoint_seed(const T* psi, const void* v, const LatState* s, double w_e, double w_r, T* lam, double* gv,
                         const Params& p, cudaStream_t st);
template <typename T>
void launch_parity_adjoint_scale(T* lam, int n, int mask, const double* scale, cudaStream_t st);
void launch_store_scale(const LatState* s, double* dst, cudaStream_t st);
template <typename T>
void launch_scale_parity_from(const T* in, T* out, int n, int mask, const double* scale, cudaStream_t st);

}  // namespace fdtd
