// States beyond the field in use: checkpoint files (Sec. VII.G), snapshot
// slots, the projection of lower states (Sec. III) and linear combinations
// (Sec. VI).
#include "api_internal.cuh"

using namespace fdtd;
using namespace fdtd::api;

namespace {

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

}  // namespace

extern "C" {

int fdtd_save_psi(fdtd_handle h, int lat, const char* path) {
  Range r("fdtd_save_psi");
  int rc = lat_check(h, lat);
  if (rc) return rc;
  if (!path) return fail(h, FDTD_ERR_INVALID_ARG, "save_psi: null path");
  Lat& L = h->lats[lat];
  if (is_complex(L.d.precision))
    return fail(h, FDTD_ERR_INVALID_ARG, "save_psi: not available for complex lattices");
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
  if (is_complex(L.d.precision))
    return fail(h, FDTD_ERR_INVALID_ARG, "load_psi: not available for complex lattices");
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
  if (is_complex(L.d.precision))
    return fail(h, FDTD_ERR_INVALID_ARG, "snapshot_save: not available for complex lattices");
  if (!L.has_psi) return fail(h, FDTD_ERR_STATE, "snapshot_save: no wavefunction yet");
  cudaMemcpyAsync(snap_field(L, slot), L.psi[L.cur], L.n3 * L.es, cudaMemcpyDeviceToDevice, h->st);
  return cuda_check(h, "snapshot_save");
}

int fdtd_snapshot_load(fdtd_handle h, int lat, int slot) {
  int rc = snap_check(h, lat, slot);
  if (rc) return rc;
  Lat& L = h->lats[lat];
  if (is_complex(L.d.precision))
    return fail(h, FDTD_ERR_INVALID_ARG, "snapshot_load: not available for complex lattices");
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
  if (is_complex(L.d.precision))
    return fail(h, FDTD_ERR_INVALID_ARG, "project_out: not available for complex lattices");
  if ((rc = resolve_potentials(h))) return rc;
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
  if (is_complex(L.d.precision))
    return fail(h, FDTD_ERR_INVALID_ARG, "combine: not available for complex lattices");
  if ((rc = resolve_potentials(h))) return rc;
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

}  // extern "C"
