// z-slab decomposition (Sec. V): the C ABI of one process's slab -- the
// temporally blocked update of its own planes from its own and its halo
// planes, its partial sums, its renormalisation -- and the host-side check
// arithmetic that turns the summed partial sums of all slabs into E, <r^2>,
// <V> and the common renormalisation factor.  Moving the halo planes
// between processes and reducing the partial sums is the caller's (e.g.
// torch.distributed over NCCL); the library allocates nothing.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "fdtd.h"
#include "kernels.cuh"

namespace fdtd {
void set_detached_error(const std::string& msg);
}

using namespace fdtd;

struct fdtd_slab_ctx {
  int n = 0, z_first = 0, nzo = 0, halo = 0, nzbuf = 0;
  Params p{};
  float* psi[2] = {nullptr, nullptr};
  const float* v = nullptr;
  cudaStream_t st = nullptr;
  int32_t* flags = nullptr;  // [0] unused, [1] expired-wait flag, [2] wait budget
  double* partials = nullptr;
  double* sums = nullptr;
  int nparts = 0;
  CUtensorMap maps[3][3];  // [depth - 1][psi0, psi1, V], stencil boxes
  CUtensorMap smaps[3];    // psi0, psi1, V with the sums box
};

namespace {

size_t slab_ws_bytes(int n, int nzo) {
  const size_t parts = (size_t)slab_sums_blocks(n, nzo) * 4 * sizeof(double);
  return 256 + ((parts + 255) & ~size_t(255)) + 256;
}

int slab_fail(const std::string& msg, int code = FDTD_ERR_INVALID_ARG) {
  set_detached_error(msg);
  return code;
}

int slab_cuda(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return slab_fail(std::string(where) + ": " + cudaGetErrorString(e), FDTD_ERR_CUDA);
  return FDTD_OK;
}

}  // namespace

extern "C" {

int fdtd_slab_workspace_size(int n, int nz_own, size_t* bytes) {
  if (!bytes || n < 8 || n % 4 || nz_own < 1 || nz_own > n) return slab_fail("slab_workspace_size: bad n or nz_own");
  *bytes = slab_ws_bytes(n, nz_own);
  return FDTD_OK;
}

int fdtd_slab_create(int n, int z_first, int nz_own, int halo, double length, double mass, double dtau, float* psi0,
                     float* psi1, const float* v, void* ws, size_t ws_bytes, void* stream, fdtd_slab* out) {
  if (!out) return slab_fail("slab_create: null output");
  *out = nullptr;
  if (n < 8 || n % 4 || n > 2048 || nz_own < 1 || z_first < 0 || z_first + nz_own > n || halo < 1 ||
      halo > blocked_max_depth() || nz_own < halo)
    return slab_fail("slab_create: need n % 4 == 0, 8 <= n <= 2048, 0 <= z_first, z_first + nz_own <= n, "
                     "1 <= halo <= 3 and halo <= nz_own (a neighbour's halo is taken from the own planes)");
  if (!psi0 || !psi1 || !v || psi0 == psi1) return slab_fail("slab_create: null or aliased field pointers");
  if (!(length > 0.0) || !(mass > 0.0) || !(dtau >= 0.0) || !std::isfinite(length + mass + dtau))
    return slab_fail("slab_create: length and mass must be positive, dtau >= 0");
  const double a = length / n, dt = dtau > 0.0 ? dtau : a * a / 4.0;
  if (!(dt < mass * a * a / 3.0))
    return slab_fail("slab_create: dtau violates the von Neumann bound dtau < m a^2 / 3", FDTD_ERR_UNSTABLE_DT);
  if (!ws || ((uintptr_t)ws & 255) || ws_bytes < slab_ws_bytes(n, nz_own))
    return slab_fail("slab_create: workspace null, not 256-byte aligned, or smaller than fdtd_slab_workspace_size()",
                     FDTD_ERR_WORKSPACE);
  fdtd_slab_ctx* s = new fdtd_slab_ctx();
  s->n = n;
  s->z_first = z_first;
  s->nzo = nz_own;
  s->halo = halo;
  s->nzbuf = nz_own + 2 * halo;
  s->p.n = n;
  s->p.a = a;
  s->p.dtau = dt;
  s->p.mass = mass;
  s->p.c = dt / (2.0 * mass * a * a);
  s->p.half_dtau_f = (float)(0.5 * dt);
  s->p.c_f = (float)s->p.c;
  s->p.one_m6c_f = (float)(1.0 - 6.0 * s->p.c);
  s->psi[0] = psi0;
  s->psi[1] = psi1;
  s->v = v;
  s->st = (cudaStream_t)stream;
  char* base = (char*)ws;
  s->flags = (int32_t*)base;
  s->partials = (double*)(base + 256);
  s->nparts = slab_sums_blocks(n, nz_own);
  s->sums = (double*)(base + slab_ws_bytes(n, nz_own) - 256);
  cudaMemsetAsync(s->flags, 0, 256, s->st);
  const float* bufs[3] = {psi0, psi1, v};
  bool ok = true;
  for (int k = 1; k <= blocked_max_depth(); ++k) {
    int bw, bh;
    tma_box(k, 128, &bw, &bh);
    for (int b = 0; b < 3; ++b) ok = ok && encode_field_map_nz(&s->maps[k - 1][b], bufs[b], n, s->nzbuf, bw, bh) == 0;
  }
  {
    int bw, bh;
    tma_box(1, 64, &bw, &bh);
    for (int b = 0; b < 3; ++b) ok = ok && encode_field_map_nz(&s->smaps[b], bufs[b], n, s->nzbuf, bw, bh) == 0;
  }
  if (!ok) {
    delete s;
    return slab_fail("slab_create: tensor maps could not be encoded (fields must be 16-byte aligned)", FDTD_ERR_CUDA);
  }
  int rc = slab_cuda("slab_create");
  if (rc) {
    delete s;
    return rc;
  }
  *out = s;
  return FDTD_OK;
}

int fdtd_slab_destroy(fdtd_slab s) {
  if (!s) return FDTD_ERR_INVALID_ARG;
  cudaStreamSynchronize(s->st);
  delete s;
  return FDTD_OK;
}

int fdtd_slab_steps_range(fdtd_slab s, int src, int depth, int z_begin, int z_end) {
  if (!s || (src != 0 && src != 1) || depth < 1 || depth > s->halo)
    return slab_fail("slab_steps: bad handle, source index or depth (1 <= depth <= halo)");
  if (z_begin < 0 || z_end > s->nzo || z_begin > z_end)
    return slab_fail("slab_steps_range: need 0 <= z_begin <= z_end <= nz_own");
  if (z_begin == z_end) return FDTD_OK;
  // planes below the lattice's bottom face and above its top face stay zero
  const int zlo = s->z_first == 0 ? s->halo : 0;
  const int zhi = s->z_first + s->nzo == s->n ? s->halo + s->nzo : s->nzbuf;
  launch_step_slab(s->maps[depth - 1][src], s->maps[depth - 1][2], s->psi[1 - src], s->p, depth, z_end - z_begin,
                   s->halo + z_begin, s->nzbuf, zlo, zhi, s->flags + 1, s->st);
  return slab_cuda("slab_steps");
}

int fdtd_slab_steps(fdtd_slab s, int src, int depth) {
  if (!s) return slab_fail("slab_steps: null handle");
  return fdtd_slab_steps_range(s, src, depth, 0, s->nzo);
}

int fdtd_slab_sums(fdtd_slab s, int src, double* sums4, int mem_kind) {
  if (!s || (src != 0 && src != 1) || !sums4 || (mem_kind != FDTD_MEM_HOST && mem_kind != FDTD_MEM_DEVICE))
    return slab_fail("slab_sums: bad handle, source index, output or mem_kind");
  const int np =
      launch_slab_sums(s->smaps[src], s->smaps[2], s->p, s->nzo, s->halo, s->z_first, s->partials, s->flags + 1, s->st);
  launch_slab_reduce(s->partials, np, mem_kind == FDTD_MEM_DEVICE ? sums4 : s->sums, s->st);
  int rc = slab_cuda("slab_sums");
  if (rc) return rc;
  int32_t err = 0;
  cudaMemcpyAsync(&err, s->flags + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s->st);
  if (mem_kind == FDTD_MEM_HOST) cudaMemcpyAsync(sums4, s->sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, s->st);
  cudaError_t e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) return slab_fail(std::string("slab_sums: ") + cudaGetErrorString(e), FDTD_ERR_CUDA);
  if (err) return slab_fail("slab: a bounded device-side wait expired in the stencil kernel", FDTD_ERR_TIMEOUT);
  return FDTD_OK;
}

int fdtd_slab_scale(fdtd_slab s, int src, int dst, double factor, int mask) {
  if (!s || (src != 0 && src != 1) || (dst != 0 && dst != 1) || !std::isfinite(factor) || mask < 0 || mask >= 16 ||
      (mask & 3) == 3 || ((mask >> 2) & 3) == 3 || (mask && src == dst))
    return slab_fail("slab_scale: bad handle, index, factor or mask (x and y symmetry only, src != dst with a mask)");
  launch_slab_scale(s->psi[src], s->psi[dst], s->n, s->nzo, s->halo, mask, factor, s->st);
  return slab_cuda("slab_scale");
}

int fdtd_check_sums(const double* sums4, double length, int n, double v_inf, double* out) {
  if (!sums4 || !out || n < 1 || !(length > 0.0)) return slab_fail("check_sums: bad arguments");
  const double a = length / n, a3 = a * a * a;
  const double s0 = sums4[0], sh = sums4[1], sr = sums4[2], sv = sums4[3];
  if (!(s0 > 0.0) || !std::isfinite(s0) || !std::isfinite(sh) || !std::isfinite(sr) || !std::isfinite(sv))
    return slab_fail("check_sums: non-finite or zero norm", FDTD_ERR_NONFINITE);
  out[0] = sh / s0;            // E
  out[1] = sh / s0 - v_inf;    // E_b
  out[2] = sr / s0;            // <r^2>
  out[3] = sv / s0;            // <V>
  out[4] = s0 * a3;            // sum psi^2 a^3
  out[5] = 1.0 / std::sqrt(s0 * a3);  // renormalisation factor
  return FDTD_OK;
}

}  // extern "C"
