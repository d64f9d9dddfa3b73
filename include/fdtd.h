/*
 * fdtd.h -- C ABI of the GB300 imaginary-time FDTD solver for the 3-D
 * Schroedinger equation (Strickland & Yager-Elorriaga, "A Parallel Algorithm
 * for Solving the 3d Schroedinger Equation", arXiv:0904.0939).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Units: hbar = 1; the mass m is a lattice parameter (Sec. II).
 * - Lattice: N sites per axis, spacing a = L / N (Sec. III), site (i, j, k),
 *   1 <= i, j, k <= N, at x = (i - (N+1)/2) a (likewise y, z), so the box is
 *   centred on the origin and r is measured from its centre (Sec. VII).
 *   Dirichlet boundary: psi = 0 outside the N^3 sites (Sec. III, Sec. V).
 * - Field layout across the ABI: dense N^3 arrays, x fastest, then y, then z
 *   (element (i, j, k) at offset ((k-1) N + (j-1)) N + (i-1)).  No padding.
 * - Sizes: every field pointer must address n^3 elements of the stated
 *   dtype; the library cannot check the length of a raw buffer.
 * - Memory: every pointer argument is paired with a mem_kind (FDTD_MEM_HOST
 *   or FDTD_MEM_DEVICE).  Inputs are borrowed for the duration of the call
 *   only: the library copies them into its own layout.  A host input has
 *   been read completely when the call returns (pinned or pageable); a
 *   device input is read in stream order on the handle's stream, so the
 *   caller may overwrite it with later work on that stream (or after
 *   synchronising it).  Outputs are written into caller-owned buffers.
 * - Ownership: the caller allocates ONE device workspace of at least
 *   fdtd_workspace_size() bytes (256-byte aligned) and keeps it alive until
 *   fdtd_destroy(); the library never allocates device memory itself.  The
 *   host-side context is allocated by fdtd_create and freed by fdtd_destroy.
 * - Streams: all device work of a handle is issued on the cudaStream_t given
 *   to fdtd_create (passed as void*; NULL = legacy default stream).  Calls
 *   that return results to host memory synchronise that stream.
 * - Errors: every call returns an int status (FDTD_OK = 0; negative = error;
 *   FDTD_NOT_CONVERGED is a positive, soft status).  Nothing aborts, exits or
 *   throws across the ABI.  fdtd_last_error() copies a message for the last
 *   failure on a handle.
 * - Threads: a handle must not be used by two host threads at once.
 */
#ifndef FDTD_H_
#define FDTD_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FDTD_API __attribute__((visibility("default")))
#else
#define FDTD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define FDTD_OK 0
#define FDTD_NOT_CONVERGED 1       /* soft: max_steps reached with tol > 0 */
#define FDTD_ERR_INVALID_ARG (-1)  /* bad pointer, size, enum or index */
#define FDTD_ERR_UNSTABLE_DT (-2)  /* dtau >= m a^2 / 3, or 1 + dtau V / 2 <= 0 */
#define FDTD_ERR_NONFINITE (-3)    /* NaN/Inf in an input or in the norm */
#define FDTD_ERR_CUDA (-4)         /* a CUDA runtime call failed */
#define FDTD_ERR_TIMEOUT (-5)      /* a bounded device-side wait gave up */
#define FDTD_ERR_SHAPE (-6)        /* lattice sizes or boxes do not match */
#define FDTD_ERR_WORKSPACE (-7)    /* workspace missing, misaligned or too small */
#define FDTD_ERR_STATE (-8)        /* call out of order (e.g. evolve before set_potential) */
#define FDTD_ERR_IO (-9)           /* a file cannot be opened, read or written, or is malformed */

/* ---- enums ---------------------------------------------------------------- */
#define FDTD_F64 0   /* psi and V in FP64 ("plain FP64 form") */
#define FDTD_F32 1   /* psi and V in FP32, sums in FP64 / compensated FP32 */
#define FDTD_BF16 2  /* psi stored as BF16, V and arithmetic in FP32 (coarse levels) */
/* Complex potentials V = V_R + i V_I (the paper's outlook, Sec. VIII): a
 * complex wavefunction, fields stored as interleaved (re, im) pairs.  As a
 * lattice precision: psi, V and the per-site A, cB of Eq. updateeq as FP64
 * (C64) or FP32 (C32) pairs, A and cB formed in FP64.  As a dtype of a field
 * passed across the ABI: n^3 interleaved pairs of doubles (C64) or floats
 * (C32).  Complex lattices take the one-step z-parallel kernel, zero
 * boundaries, and evolve / observables / upsample (complex to complex);
 * backward, snapshots, checkpoint files and batched mode are for real
 * lattices only (FDTD_ERR_INVALID_ARG). */
#define FDTD_C64 3
#define FDTD_C32 4

#define FDTD_MEM_HOST 0
#define FDTD_MEM_DEVICE 1

#define FDTD_DIST_UNIFORM 0   /* U[-1, 1) */
#define FDTD_DIST_GAUSSIAN 1  /* N(0, 1), Box-Muller (Sec. III) */

/* Symmetry mask for fdtd_init_symmetric (Sec. IV): two bits per axis,
 * x in bits 0-1, y in bits 2-3, z in bits 4-5; per axis 0 = none,
 * 1 = S_i (copy), 2 = A_i (copy with sign flip). */
#define FDTD_PARITY_NONE 0
#define FDTD_PARITY_S 1
#define FDTD_PARITY_A 2
#define FDTD_PARITY_MASK(px, py, pz) ((px) | ((py) << 2) | ((pz) << 4))

/* ---- descriptors ------------------------------------------------------------ */
typedef struct {
  int32_t n;          /* sites per axis, 1 <= n <= 2048 */
  int32_t precision;  /* FDTD_F64 / FDTD_F32 / FDTD_BF16 */
  double length;      /* box length L = n a (> 0) */
  double mass;        /* particle mass m (> 0) */
  double dtau;        /* imaginary time step; 0 selects a^2 / 4 (Sec. VII) */
  double v_inf;       /* V at infinity for the binding energy (Eq. bindingenergy) */
} fdtd_lattice_desc;

typedef struct {
  int32_t check_every;    /* steps between checks (Sec. V; default 100) */
  int32_t tol_relative;   /* 1: converged when |dE_b| <= tol |E_b|; 0: |dE_b| <= tol */
  double tol;             /* convergence tolerance; <= 0 never converges */
  int32_t temporal_depth; /* FP32/BF16 steps fused per stencil launch; 0 = auto */
  int32_t backward_steps; /* largest T that fdtd_backward may be asked for; 0 = none */
  int32_t batched;        /* 1: all lattices of the handle advance in one persistent launch (a
                             cooperative kernel in a CUDA graph; the update items of all
                             active lattices are cut into one equal range per block); with
                             autotune and no temporal_depth, the first evolve of a set of
                             lattice sizes times (depth 1..3) x (tiles 64x16, 128x16, 64x32) on
                             update passes that write the spare fields without advancing the
                             state, then runs the whole evolve in one launch with the
                             fastest (cached; identical results for every choice) */
  int32_t reimpose_parity;/* 1 (default): re-impose the symmetry mask at every check (Sec. IV) */
  int32_t stencil_kernel; /* 0 (default): TMA-streamed, temporally blocked kernel where it applies
                             (FP32, n % 4 == 0); 1: the plain one-step z-marching kernel
                             everywhere; 2: the one-step kernel with four x sites per thread
                             and no z-march where it applies (FP32, n % 4 == 0), else 1.
                             Results are identical for all. */
  int32_t autotune;       /* 1 (default): time every (depth, tile width, span) candidate and the
                             two one-step kernels on first use of a lattice size and keep the
                             fastest (results are identical for all); FP32 lattices the TMA
                             kernel does not take (periodic, n < 8) with n % 4 == 0 time the
                             two one-step kernels */
  int32_t zchunk;         /* span of the TMA stencil when temporal_depth > 0: consecutive tile
                             planes per block, the x-y tile columns laid end to end with z
                             fastest (a span that divides n is a z-chunk; a longer or ragged
                             one runs on into the next column); 0 = one equal span per
                             resident block; -1 = one wave with each block's planes cut so
                             that blocks whose range starts a second column (its warm-up
                             and drain steps counted) get fewer; -2 = columns first: one
                             block per tile column from plane 0, the other resident blocks
                             share the column tops (falls back to -1 when there are no
                             more resident blocks than columns) */
  int32_t wait_limit_us;  /* bound on every device-side wait: 0 = default (0.2 s per pipeline
                             wait, 2 s per grid barrier), > 0 = microseconds, < 0 = none (a wait
                             that is not already complete expires at once; for testing the
                             FDTD_ERR_TIMEOUT path) */
  int32_t snapshots;      /* snapshot slots per lattice (Sec. III excited states); 0 = none */
  int32_t graphs;         /* 1 (default): fdtd_evolve runs each lattice's full pairs of
                             check_every-step segments as one CUDA graph whose while loop is
                             ended on the device by the convergence check (no host round trip
                             per segment); the loops of a handle's lattices run at the same
                             time, each on its own stream.  The rest, and the first two
                             segments of a run with profiling on, go through the handle's
                             stream.  Results are identical either way. */
  int32_t boundary;       /* 0 (default): psi = 0 beyond the lattice (Sec. III); 1: periodic
                             (neighbour index -1 is N-1 and N is 0 along every axis; the
                             paper notes that other boundary conditions are easily
                             implemented).  Periodic lattices use the z-marching kernels
                             (the TMA boxes zero-fill), not batched mode and not
                             fdtd_observables_noalloc */
  int32_t tile_x;         /* tile width of the TMA stencil (64 or 128) when temporal_depth > 0
                             or autotune is off; 0 = 128 for n > 64, else 64 (batched: 128 if
                             most sites lie in lattices with n >= 96, else 64) */
  int32_t tile_y;         /* batched mode, with temporal_depth > 0 or autotune off: 32 selects
                             64 x 32 tiles (tile_x 0 or 64); 0 or 16: tiles 16 high */
} fdtd_options;

typedef struct {
  double energy;          /* E = sum psi H psi / sum psi^2 (Eq. energysum, sign of Sec. II's H) */
  double binding_energy;  /* E - v_inf (Eq. bindingenergy) */
  double norm;            /* sum psi^2 a^3 of the field the sums were taken on */
  double r2;              /* <r^2> = sum r^2 psi^2 / sum psi^2 */
  double r_rms;           /* sqrt(<r^2>) */
  double v_expect;        /* <V> = sum V psi^2 / sum psi^2 */
  double delta_e;         /* |E_b - E_b(previous check)|, -1 if none (complex lattices: the modulus) */
  double energy_imag;     /* Im E = <V_I> for complex lattices (Hermitian Rayleigh quotient), 0 otherwise */
  int64_t steps;          /* steps taken by the last fdtd_evolve on this lattice */
  int32_t converged;      /* 1 if the last fdtd_evolve met the tolerance */
  int32_t checks;         /* checks made by the last fdtd_evolve */
} fdtd_obs;

typedef struct {
  int64_t launches;       /* kernels launched by this handle since creation/reset */
  int64_t stencil_launches;
  double stencil_ms;      /* summed device time of stencil launches (profiling on) */
  int64_t stencil_site_updates;
  double stencil_bytes;   /* algorithmic HBM bytes of those launches */
  int64_t graph_launches; /* evolve graphs launched (options.graphs) */
  int64_t stencil_timed_launches; /* stencil launches stencil_ms covers (profiling on: the
                             launches of the first two segments of each evolve, or all of
                             them with options.graphs = 0) */
} fdtd_stats;

typedef struct fdtd_context* fdtd_handle;

/* ---- calls ------------------------------------------------------------------ */

/* Fill *o with the defaults: check_every 100, tol 1e-6 relative, auto depth,
 * no backward storage, not batched, parity re-imposed at every check. */
FDTD_API int fdtd_default_options(fdtd_options* o);

/* Bytes of device workspace that fdtd_create needs for `count` lattices.
 * o may be NULL (defaults). */
FDTD_API int fdtd_workspace_size(const fdtd_lattice_desc* d, int count, const fdtd_options* o, size_t* bytes);

/* Create a handle for `count` lattices on the current CUDA device.
 * Validates every descriptor: n, L, m > 0; the von Neumann bound
 * dtau < m a^2 / 3 (Sec. III) else FDTD_ERR_UNSTABLE_DT.  ws must be a
 * device pointer, 256-byte aligned, of ws_bytes >= fdtd_workspace_size().
 * stream is a cudaStream_t (or NULL).  On success *out owns no device memory. */
FDTD_API int fdtd_create(const fdtd_lattice_desc* d, int count, const fdtd_options* o, void* ws, size_t ws_bytes,
                void* stream, fdtd_handle* out);

/* Release the host-side context (the caller frees the workspace). */
FDTD_API int fdtd_destroy(fdtd_handle h);

/* Message for the last error on h (or on handle creation and the
 * handle-free calls when h is NULL), copied into the caller's buf of n bytes
 * (truncated, always NUL-terminated when n > 0; buf may be NULL when n is 0).
 * Returns the full length of the message, so a caller can size buf; never
 * negative. */
FDTD_API int fdtd_last_error(fdtd_handle h, char* buf, size_t n);

/* Load V (n^3 values, dense x-fastest, dtype FDTD_F64 or FDTD_F32) for
 * lattice `lat` (Sec. II: static real potential).  The coefficients
 * A = (1 - dtau V/2)/(1 + dtau V/2) and B = 1/(1 + dtau V/2) of
 * Eq. updateeq are derived from it on the device.  Returns
 * FDTD_ERR_NONFINITE for NaN/Inf and FDTD_ERR_UNSTABLE_DT where
 * 1 + dtau V/2 <= 0 (the update would divide by zero or flip sign). */
FDTD_API int fdtd_set_potential(fdtd_handle h, int lat, const void* v, int dtype, int mem_kind);
/* fdtd_set_potential without waiting: the copy (or conversion) of V and its
 * checks are enqueued on the handle's stream and the call returns; argument
 * errors are reported at once.  The caller keeps v valid and unchanged until
 * the handle's stream has passed the copy (for host memory, page-locked
 * memory makes the copy asynchronous; from pageable memory the CUDA runtime
 * may copy before returning).  The next call of the handle that uses V
 * (fdtd_evolve, fdtd_observables, fdtd_upsample into it, fdtd_backward,
 * fdtd_project_out, fdtd_combine, fdtd_tuned_config/kernel) or a
 * fdtd_set_potential first waits for the stream and reports the checks'
 * result (FDTD_ERR_NONFINITE / FDTD_ERR_UNSTABLE_DT as above; with several
 * potentials pending, every one of them is then unset).  A handle on its own
 * stream can so upload one level's potential while another handle computes. */
FDTD_API int fdtd_set_potential_async(fdtd_handle h, int lat, const void* v, int dtype, int mem_kind);

/* Random initial wavefunction (Sec. III) followed by the symmetry mask
 * (Sec. IV).  Site value = draw number lat_id * 2^42 + n (uniform) or
 * draws 2n, 2n+1 (Gaussian) of the SplitMix64 stream seeded with `seed`,
 * n = dense site index.  The mask is remembered and re-imposed at every
 * check of fdtd_evolve.  The field becomes the start of fdtd_backward. */
FDTD_API int fdtd_init_symmetric(fdtd_handle h, int lat, uint64_t seed, int parity_mask, int dist);

/* Replace / read psi (n^3 values, dense x-fastest, dtype FDTD_F64/F32) --
 * the save/restore of Sec. VII.G.  set_psi also records the field as the
 * start of fdtd_backward and sets the symmetry mask to `parity_mask`. */
FDTD_API int fdtd_set_psi(fdtd_handle h, int lat, const void* psi, int dtype, int mem_kind, int parity_mask);
FDTD_API int fdtd_get_psi(fdtd_handle h, int lat, void* psi, int dtype, int mem_kind);

/* Imaginary-time evolution of every lattice of the handle (Eq. updateeq),
 * with a check at step t = 0, check_every, 2 check_every, ... and at
 * t = max_steps: the sums of Eq. energysum on psi_t, renormalisation to
 * sum psi^2 a^3 = 1 (Sec. III), re-imposition of the symmetry mask
 * (Sec. IV), and the convergence test on the binding energy (Sec. V).
 * A lattice stops at the first check whose |dE_b| meets the tolerance.
 * The lattices of a non-batched handle are independent: with
 * options.graphs their evolve loops run at the same time, each on its own
 * stream, and every lattice ends bit-identical to an evolve of it alone.
 * *steps_done (may be NULL) receives the largest step count over lattices.
 * Returns FDTD_OK, FDTD_NOT_CONVERGED (tol > 0 and some lattice reached
 * max_steps), FDTD_ERR_NONFINITE, FDTD_ERR_TIMEOUT or another error. */
FDTD_API int fdtd_evolve(fdtd_handle h, int64_t max_steps, int64_t* steps_done);

/* Observables recorded at the last check of the last fdtd_evolve. */
FDTD_API int fdtd_last_check(fdtd_handle h, int lat, fdtd_obs* out);

/* Observables of the current psi (Eq. energysum, <r^2>, <V>, norm);
 * the field is not modified.  steps/converged/checks echo the last evolve. */
FDTD_API int fdtd_observables(fdtd_handle h, int lat, fdtd_obs* out);

/* Multi-resolution transfer (Sec. VI, Sec. VII.G): psi of (dst, lat_dst)
 * becomes the trilinear interpolation of psi of (src, lat_src), then is
 * renormalised and given the source's symmetry mask.  Requires
 * n_dst = 2 n_src and equal box lengths (else FDTD_ERR_SHAPE).  Storage
 * precisions may differ (e.g. BF16 coarse -> FP32 fine).  Both handles must
 * use the same device; the work runs on dst's stream after src's work. */
FDTD_API int fdtd_upsample(fdtd_handle src, int lat_src, fdtd_handle dst, int lat_dst);

/* Gradient of  w_e E[psi_T] + w_r <r^2>[psi_T]  with respect to V at every
 * site, through T unrolled update steps started from the recorded initial
 * field (the last init_symmetric / set_psi), with the same checks as
 * fdtd_evolve with tol = 0 (renormalisation factors held constant; the
 * symmetry projection differentiated exactly).  sqrt(T) checkpointing:
 * the forward pass stores psi every ceil(sqrt T) steps and recomputes each
 * segment.  Needs T <= options.backward_steps.  gv receives n^3 values of
 * dtype FDTD_F64 or FDTD_F32.  obs (may be NULL) receives E, <r^2> at T.
 * Leaves psi of the lattice equal to psi_T. */
FDTD_API int fdtd_backward(fdtd_handle h, int lat, int64_t T, double w_e, double w_r, void* gv, int dtype,
                  int mem_kind, fdtd_obs* obs);

/* Stencil configuration in use for lattice `lat` (after autotuning, if on):
 * temporal depth (steps per launch) and the span (tile planes per block,
 * options.zchunk; -1 = the balanced one-wave partition, -2 = columns first) of
 * the TMA kernel;
 * zchunk = 0 (depth 1) when the one-step
 * z-marching kernel is in use.  For a batched handle after an evolve: the
 * depth of its persistent launch and zchunk = -1 (the balanced partition). */
FDTD_API int fdtd_tuned_config(fdtd_handle h, int lat, int* depth, int* zchunk);

/* The tile of that TMA stencil: tile_x x tile_y output sites of one z-plane
 * per block and step (tile_x 64 or 128, tile_y 16; a batched handle after
 * an evolve: its persistent launch's tile, also 64 x 32).  Both are 0 when
 * the one-step kernel is in use (FP64, BF16, periodic lattices,
 * stencil_kernel 1 or 2, or the autotuner's choice). */
FDTD_API int fdtd_tuned_kernel(fdtd_handle h, int lat, int* tile_x, int* tile_y);

/* Checkpoint files (Sec. VII.G: a run saves its wavefunction, and a later
 * run reads it back as its initial condition, adjusting the resolution).
 * File layout, little-endian: a 64-byte header {char magic[8] = "FDTDPSI1";
 * uint32 version = 1; int32 n; int32 dtype (FDTD_F64 for FP64 lattices,
 * FDTD_F32 otherwise); int32 symmetry mask; double box length, mass, dtau;
 * int64 steps of the last evolve; uint64 FNV-1a hash of the data bytes}
 * followed by the n^3 values, x fastest.
 * fdtd_save_psi writes psi of lattice `lat` (FDTD_ERR_STATE before any
 * psi, FDTD_ERR_IO if the file cannot be written).
 * fdtd_load_psi reads it into lattice `lat`: the box length must match
 * (FDTD_ERR_SHAPE) and the lattice's n must be the file's n times 2^k.  For
 * k = 0 psi is taken as stored (as fdtd_set_psi); for k > 0 it is
 * transferred k times by the trilinear map of fdtd_upsample, then
 * renormalised and given the file's symmetry mask.  A file that is
 * truncated, too long, of another format or whose data do not match the
 * stored hash is rejected with FDTD_ERR_IO before the lattice is touched. */
FDTD_API int fdtd_save_psi(fdtd_handle h, int lat, const char* path);
FDTD_API int fdtd_load_psi(fdtd_handle h, int lat, const char* path);

/* Bounds-checking builds (compiled with -DFDTD_CHECK_BOUNDS, e.g.
 * `python paper_0904_0939_gb300/_build.py --checked`): the number of
 * shared-memory and output accesses of the TMA tile pipelines that fell
 * outside their allocation since the handle was created (each was skipped,
 * not performed).  Other builds return FDTD_ERR_STATE. */
FDTD_API int fdtd_bounds_violations(fdtd_handle h, int64_t* count);

/* Per-check record of the last fdtd_evolve on lattice `lat` (Secs. III-V):
 * 8 doubles per check {t, E, E_b, norm = sum psi^2 a^3 before the
 * renormalisation, <r^2>, <V>, |dE_b| (-1 at the first check), S0}, oldest
 * first.  The device keeps the last 4096 checks of an evolve; the most
 * recent min(checks, 4096, cap) are copied to the host array out (cap
 * records of 8 doubles) and *count receives the number of checks made. */
FDTD_API int fdtd_check_history(fdtd_handle h, int lat, double* out, int cap, int* count);

/* Snapshots (Sec. III): full copies of psi kept in the workspace, in
 * options.snapshots slots per lattice.  save: psi -> slot; load: slot -> psi
 * (also recorded as the start of fdtd_backward; the symmetry mask is kept). */
FDTD_API int fdtd_snapshot_save(fdtd_handle h, int lat, int slot);
FDTD_API int fdtd_snapshot_load(fdtd_handle h, int lat, int slot);

/* Projection of Sec. III: psi <- psi - phi <phi|psi> / <phi|phi> for each
 * snapshot slot listed, one after another (Gram-Schmidt order), then
 * renormalised to sum psi^2 a^3 = 1.  With psi a snapshot taken at tau_snap
 * >> 1/(E2 - E1) and the slots holding the lower states, the result
 * approximates the next excited state (fdtd_observables gives its energy).
 * Sums in FP64 (FP64 lattices) or compensated FP32. */
FDTD_API int fdtd_project_out(fdtd_handle h, int lat, const int* slots, int count);

/* Linear combination as an initial condition (Sec. VI): psi <- sum_k
 * weights[k] * slot_k, renormalised; the field becomes the start of
 * fdtd_backward.  FDTD_ERR_NONFINITE if the combination vanishes. */
FDTD_API int fdtd_combine(fdtd_handle h, int lat, const int* slots, const double* weights, int count);

/* Launch counters and (when profiling is on) summed stencil device time. */
FDTD_API int fdtd_get_stats(fdtd_handle h, fdtd_stats* out);
FDTD_API int fdtd_reset_stats(fdtd_handle h);
/* on = 1: bracket stencil launches issued through the stream with CUDA events
 * on the handle's stream, one pair around each run of consecutive launches of
 * one temporal depth (with options.graphs = 1, fdtd_evolve issues its first
 * two segments through the stream for this and the rest as a graph). */
FDTD_API int fdtd_set_profiling(fdtd_handle h, int on);

/* Allocation-free observables of a caller-held field (no counterpart in
 * the paper; it serves callers that cannot allocate device memory, e.g.
 * code running inside a fixed memory pool or handed only raw device
 * pointers and a stream).  psi and v are DEVICE pointers to n^3 values
 * (dense, x fastest), both FDTD_F64 or both FDTD_F32; out is a DEVICE
 * pointer to 8 doubles that receive E, <r^2>, <V>, sum psi^2 a^3, and the
 * raw sums S0, SH, Sr, SV, with the same arithmetic as fdtd_observables
 * for that precision.  The work is enqueued on `stream` (cudaStream_t or
 * NULL) and the call returns without synchronising.
 * Nothing is allocated: the block partials live in a static 128 KiB device
 * array (plus one error word, cleared by every call) that every GPU loading
 * the library keeps until exit, so n is limited to 1 <= n <= 1024
 * (FDTD_ERR_SHAPE beyond).  A bounded device-side wait that expires
 * yields NaN in out.  The first call on a
 * device looks the array's address up (make it before any stream capture
 * on that device).  All calls share the array: calls whose kernels overlap
 * on the GPU race and may return wrong sums.  A zero or non-finite field
 * yields NaN/Inf in out (there is no status for it).  Errors are reported
 * through fdtd_last_error(NULL). */
FDTD_API int fdtd_observables_noalloc(const void* psi, const void* v, int dtype, int n, double length, double mass,
                                      double* out, void* stream);

/* ---- z-slab decomposition (Sec. V) -------------------------------------------
 * The paper partitions the lattice into slabs along z, one per process; each
 * process updates its own planes, exchanges boundary planes with its
 * neighbours, and the processes reduce their partial sums at every check.
 * These calls are one process's side of that scheme on its GPU: the caller
 * moves the halo planes between processes (e.g. NCCL send/recv through
 * torch.distributed) and reduces the partial sums (an all-reduce of four
 * doubles); the library allocates nothing.
 *
 * A slab of an N^3 FP32 lattice (N % 4 == 0, 8 <= N <= 2048) owns the nz_own
 * global planes z_first .. z_first + nz_own - 1 (0-based, z the slowest
 * index).  Its two fields psi0, psi1 and its potential v are caller-owned
 * DEVICE buffers of N x N x (nz_own + 2 halo) floats, x fastest, plane k
 * holding global plane z_first - halo + k: `halo` planes below and above
 * the own planes.  V must be set on every plane that lies inside the
 * lattice, with 1 + dtau V / 2 > 0 (not checked here); halo planes beyond the lattice's faces are never read for psi
 * (treated as the zero boundary of Sec. III) and must hold psi = 0.  The
 * buffers must be 16-byte aligned and stay alive until fdtd_slab_destroy.
 * Errors are reported through fdtd_last_error(NULL). */
typedef struct fdtd_slab_ctx* fdtd_slab;

/* Bytes of device workspace (partial sums, flags) a slab of nz_own planes needs. */
FDTD_API int fdtd_slab_workspace_size(int n, int nz_own, size_t* bytes);

/* Create the slab: 1 <= halo <= min(3, nz_own) (the deepest temporal block it will run),
 * box length L, mass m, dtau (0 selects a^2/4; the von Neumann bound of
 * Sec. III applies, else FDTD_ERR_UNSTABLE_DT), ws a 256-byte aligned device
 * workspace of fdtd_slab_workspace_size() bytes, stream a cudaStream_t. */
FDTD_API int fdtd_slab_create(int n, int z_first, int nz_own, int halo, double length, double mass, double dtau,
                              float* psi0, float* psi1, const float* v, void* ws, size_t ws_bytes, void* stream,
                              fdtd_slab* out);
FDTD_API int fdtd_slab_destroy(fdtd_slab s);

/* `depth` (1 <= depth <= halo) update steps of Eq. updateeq from field `src`
 * (0 or 1) into the other field's own planes, with the same arithmetic as
 * fdtd_evolve's FP32 stencil (bit for bit).  The src field's `depth` halo
 * planes on each side must hold the neighbouring slabs' current planes; the
 * destination's halo planes are not written (the caller refreshes them by
 * the exchange).  Asynchronous on the slab's stream. */
FDTD_API int fdtd_slab_steps(fdtd_slab s, int src, int depth);

/* The same steps for own planes z_begin .. z_end - 1 only (0-based within
 * the own planes; 0 <= z_begin <= z_end <= nz_own).  The paper's inside-out
 * order (Sec. V): update the planes the neighbours need first, start their
 * exchange, then update the interior while the messages are in flight.  The
 * result equals fdtd_slab_steps over any cover of the own planes by
 * disjoint ranges. */
FDTD_API int fdtd_slab_steps_range(fdtd_slab s, int src, int depth, int z_begin, int z_end);

/* Partial sums of Eq. energysum over the own planes of field `src`:
 * sums4 = {S0, SH, Sr, SV} with r measured from the lattice centre (the
 * halo planes adjacent to the own planes must be current), formed with the
 * per-site arithmetic of the FP32 lattice sums of fdtd_observables.  mem_kind
 * FDTD_MEM_HOST: written to host memory after synchronising the stream;
 * FDTD_MEM_DEVICE: four doubles of device memory, in stream order.  Returns
 * FDTD_ERR_TIMEOUT if a bounded wait of an earlier step expired. */
FDTD_API int fdtd_slab_sums(fdtd_slab s, int src, double* sums4, int mem_kind);

/* Own planes of field dst = factor * P(own planes of field src): the
 * renormalisation of Sec. III with the x and y symmetry operators of Sec. IV
 * (mask bits 0-3; a z operator would need the mirror slab's planes and is
 * refused).  src may equal dst only with mask 0 (a mirrored site is read
 * by another thread than the one writing it). */
FDTD_API int fdtd_slab_scale(fdtd_slab s, int src, int dst, double factor, int mask);

/* Host arithmetic of a check from the lattice-wide sums {S0, SH, Sr, SV}
 * (the sum over all slabs): out = {E, E_b = E - v_inf, <r^2>, <V>,
 * sum psi^2 a^3, 1 / sqrt(S0 a^3)} for an N^3 lattice of box length L. */
FDTD_API int fdtd_check_sums(const double* sums4, double length, int n, double v_inf, double* out);

#ifdef __cplusplus
}
#endif
#endif /* FDTD_H_ */
