// Gradients through the unrolled evolution: fdtd_backward (sqrt(T)
// checkpoints, segment recompute, the adjoint step: one pass for FP32
// lattices -- four x sites per thread when n % 4 == 0, else z-marching --
// and a pointwise and a stencil pass for FP64).
#include "api_internal.cuh"

using namespace fdtd;
using namespace fdtd::api;

extern "C" {

int fdtd_backward(fdtd_handle h, int lat, int64_t T, double w_e, double w_r, void* gv_out, int dtype, int mem_kind,
                  fdtd_obs* obs) {
  Range r("fdtd_backward");
  int rc = lat_check(h, lat);
  if (rc) return rc;
  Lat& L = h->lats[lat];
  if (is_complex(L.d.precision))
    return fail(h, FDTD_ERR_INVALID_ARG, "backward: not available for complex lattices");
  if (!gv_out || (dtype != FDTD_F64 && dtype != FDTD_F32) ||
      (mem_kind != FDTD_MEM_HOST && mem_kind != FDTD_MEM_DEVICE) || T < 1 || !std::isfinite(w_e) ||
      !std::isfinite(w_r))
    return fail(h, FDTD_ERR_INVALID_ARG, "backward: bad pointer, dtype, mem_kind, T or weights");
  if (L.d.precision == FDTD_BF16) return fail(h, FDTD_ERR_INVALID_ARG, "backward: not available for BF16 storage");
  if (!L.psi0 || T > L.bw_T)
    return fail(h, FDTD_ERR_WORKSPACE, "backward: T exceeds options.backward_steps given at create");
  if ((rc = resolve_potentials(h))) return rc;
  if (!L.has_v || !L.has_psi0) return fail(h, FDTD_ERR_STATE, "backward: set_potential and init/set_psi first");
  const int64_t ce = h->o.check_every;
  const int K = L.bw_K;
  const int mask = h->o.reimpose_parity ? L.mask : 0;
  const size_t fb = L.n3 * L.es;
  const bool f4 = L.d.precision == FDTD_F32 && L.d.n % 4 == 0;  // the direct four-site kernels
  auto field = [&](void* base, int64_t i) { return (void*)((char*)base + (size_t)i * fb); };
  LatState* scratch = &L.state[1];
  launch_state_reset(scratch, 0, h->st);
  h->stats.launches += 1;

  // forward pass from the recorded start, saving every K-th field
  L.cur = 0;
  cudaMemcpyAsync(L.psi[0], L.psi0, fb, cudaMemcpyDeviceToDevice, h->st);
  for (int64_t t = 0; t < T;) {
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
    // the steps up to the next check or checkpoint, temporally blocked
    const int64_t next = std::min(std::min((t / ce + 1) * ce, (t / K + 1) * K), T);
    run_steps(h, L, next - t, nullptr, t);
    t = next;
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
        else if constexpr (std::is_same_v<T_, float>) {
          if (f4)
            launch_direct_f32((const float*)field(L.seg, t - t0), (float*)nxt, (const float*)L.v, L.p, nullptr, h->st);
          else
            launch_step_f32<float>((const float*)field(L.seg, t - t0), (float*)nxt, (const float*)L.v, L.p, nullptr,
                                   h->st);
        }
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
        if constexpr (std::is_same_v<T_, float>) {
          if (f4) {
            launch_adjoint_direct_f32((const float*)L.lam[lc], (const float*)field(L.seg, t - 1 - t0),
                                      (const float*)raw_of(t), (const float*)L.v, (float*)L.lam[1 - lc], L.gv, L.p,
                                      h->st);
          } else {
            launch_adjoint_step_f32((const float*)L.lam[lc], (const float*)field(L.seg, t - 1 - t0),
                                    (const float*)raw_of(t), (const float*)L.v, (float*)L.lam[1 - lc], L.gv, L.p,
                                    h->st);
          }
        } else if constexpr (std::is_same_v<T_, double>) {
          launch_adjoint_pointwise<T_>((const T_*)L.lam[lc], (const T_*)field(L.seg, t - 1 - t0), (const T_*)raw_of(t),
                                       L.v, L.coefCB, (T_*)L.bw_u, L.gv, L.p, h->st);
          launch_adjoint_stencil<T_>((const T_*)L.bw_u, (const T_*)L.lam[lc], (T_*)L.lam[1 - lc], L.v, L.coefA, L.p,
                                     h->st);
        }
        if constexpr (!std::is_same_v<T_, __nv_bfloat16>) {
          if ((t - 1) % ce == 0)
            launch_parity_adjoint_scale<T_>((T_*)L.lam[1 - lc], L.d.n, mask, L.scales + (t - 1) / ce, h->st);
        }
      });
      h->stats.launches += ((t - 1) % ce == 0 ? 1 : 0) + (L.d.precision == FDTD_F64 ? 2 : 1);
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

}  // extern "C"
