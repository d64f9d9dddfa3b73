// TMA-streamed tile pipelines shared by the one-lattice kernels
// (k_tblock.cu) and the batched persistent kernel (k_batched.cu).
//
// A tile item covers TXT x TY sites in x-y and the z-planes [z0, z1) of one
// FP32 lattice with n % 4 == 0.  Input planes of a (TXT + 2 HX) x (TY + 2K)
// box -- psi and V -- stream through a ring of R shared-memory slots with
// cp.async.bulk.tensor; one thread issues, an mbarrier per slot counts the
// bytes; sites outside the lattice arrive as zeros (the Dirichlet wall of
// Sec. III).  Each thread owns one float4 column of the box.
//
// tma_step_item applies the update of Eq. updateeq K times: level 1 reads
// the ring, level l > 1 keeps three z-planes of level l-1 of its column in
// registers and takes the y-neighbours from a double-buffered shared plane
// and the x-neighbours from the adjacent lanes.  Level l trails level l-1 by
// one plane, so one barrier per z-step orders everything.  Level K writes
// the tile interior.  The per-site arithmetic is that of the one-step
// kernel, so K fused steps equal K single steps bit for bit; box sites
// outside the tile compute garbage at levels < K that moves inward one site
// per level and never reaches the interior (x margin HX >= K, y margin K).
//
// tma_sums_item accumulates S0 = sum psi^2, SH = sum psi(-Lap psi/(2 m a^2)
// + V psi), Sr = sum r^2 psi^2, SV = sum V psi^2 (Eq. energysum) over the
// tile interior with Kahan-compensated FP32 per thread and a fixed-order
// FP64 block reduction.
//
// Every mbarrier wait is bounded in wall-clock time; on expiry the item
// sets *err, waits (bounded) for its copies in flight and returns false in
// every thread (a shared flag read by all after the z-step's barrier).
#pragma once
#include <cuda.h>

#include <type_traits>

#include "common.cuh"

namespace fdtd {
namespace tb {

constexpr int TY = 16;   // interior tile height
constexpr int HX = 4;    // x margin of the box: >= K and a multiple of 4 (TMA x * 4 B % 16 == 0)
constexpr int RING = 6;  // ring slots: a multiple of 2 and 3, so a six-step group sees every slot at a fixed place
constexpr unsigned long long kWaitLimitNs = 200ull * 1000 * 1000;  // 0.2 s per wait

// Shared-memory layout of a tile item with K update levels.  The ring
// holds psi and V of RING planes: the three planes level 1 reads, the V of
// the K - 1 older planes the deeper levels need, and D planes prefetched.
// Level 1's planes are triple-buffered (a thread writes the next one before
// the other threads have finished reading the previous step's), the planes
// of levels 2..K-1 double-buffered (written after the step's wait).
template <int K, int TXT, int TYT = TY, typename PT = float>
struct Geo {
  static constexpr int TX = TXT;
  static constexpr int BW = TX + 2 * HX;
  static constexpr int C4 = BW / 4;                          // float4 columns per box row
  static constexpr int LW = BW + 8;                          // level-plane pitch: 4-float guards
  static constexpr int BH = TYT + 2 * K;
  static constexpr int USED = C4 * BH;                       // threads that own a box column
  static constexpr int THREADS = (USED + 31) / 32 * 32;      // whole warps
  static constexpr int R = RING;                             // ring slots
  static constexpr int D = R - 2 - (K > 1 ? K - 1 : 1);      // planes prefetched beyond the newest in use
  static_assert(D >= 1, "the ring must prefetch at least one plane");
  static constexpr int PLANE = ((BW * BH * 4 + 127) / 128) * 128 / 4;  // floats per box, 128 B multiple
  static constexpr int LPLANE = LW * BH;
  static constexpr int NLEV = K > 1 ? 3 + 2 * (K - 2) : 0;  // level planes
  static constexpr size_t RING_OFF = 128;                    // guard before the ring
  // psi box: FP32 like V, or BF16 with an 8-site x margin (a TMA box must
  // start at an x whose byte offset is a multiple of 16); the threads'
  // columns sit XOFF sites into it
  static constexpr int PS = (int)sizeof(PT);
  static constexpr int HXP = PS == 4 ? HX : 8;
  static constexpr int BWP = TX + 2 * HXP;
  static constexpr int XOFF = HXP - HX;
  static constexpr size_t PSI_BYTES = ((size_t)BWP * BH * PS + 127) / 128 * 128;
  static constexpr size_t SLOT_BYTES = PSI_BYTES + (size_t)PLANE * 4;  // psi box, then the V box
  static constexpr unsigned TX_BYTES = (unsigned)(BWP * BH * PS + BW * BH * 4);  // bytes the two box loads deliver
  static constexpr size_t LEVEL_OFF = RING_OFF + R * SLOT_BYTES + 128;
  static constexpr size_t BAR_OFF = LEVEL_OFF + (size_t)NLEV * LPLANE * 4;
  static constexpr size_t CBAR_OFF = BAR_OFF + 8 * R;        // the step barrier of the block
  static constexpr size_t FLAG_OFF = CBAR_OFF + 8;           // "a wait expired" word of the item
  static constexpr size_t RED_OFF = FLAG_OFF + 8;            // block reduction scratch (sums)
  static constexpr size_t SMEM = RED_OFF + 8 * 4 * (THREADS / 32) + 128;  // + base alignment slack
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory base aligned to 128 B (TMA destinations)
__device__ __forceinline__ char* aligned_smem(char* raw) {
  return raw + ((128u - (smem_u32(raw) & 127u)) & 127u);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Invalidate a barrier whose phases are all complete, so that its shared
// memory can be reused (the next item's barriers or another item's data).
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// try_wait that may suspend the thread until the phase completes or about
// suspend_ns have passed, instead of returning at once: a waiting warp then
// takes no issue slots from the warps that are working.
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t* bar, unsigned parity, unsigned suspend_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(suspend_ns)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Wait budget in ns from the word after the error flag: 0 = default,
// > 0 = that many microseconds, < 0 = none (a wait that is not already
// complete gives up at once -- the mode the timeout test uses).
__device__ __forceinline__ long long wait_budget_ns(const int32_t* err) {
  const int us = *(volatile const int32_t*)(err + 1);
  return us == 0 ? (long long)kWaitLimitNs : (us > 0 ? 1000ll * us : -1);
}
// Wait bounded in wall-clock time (budget from wait_budget_ns, read once per
// item so that the wait itself touches no global memory on its fast path);
// gives up early once any block has reported an expired wait in *err.
// After a first plain try_wait the thread waits suspended, at most
// kSuspendNs per try, and checks the flag and the clock between tries.
// Returns false if it gave up.
constexpr unsigned kSuspendNs = 100000;  // 0.1 ms, well inside every budget
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, const int32_t* err,
                                                  long long budget) {
  if (budget < 0) return mbar_test_wait(bar, parity);
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait_suspend(bar, parity, kSuspendNs)) return true;
    if (*(volatile const int32_t*)err != 0) return false;
    if (global_ns() - t0 > (unsigned long long)budget) return false;
  }
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// slot of plane j + d given the slot sj of plane j, for -R < d < R
template <int R>
__device__ __forceinline__ int slot_add(int sj, int d) {
  int s = sj + d;
  s -= (s >= R) ? R : 0;
  s += (s < 0) ? R : 0;
  return s;
}

__device__ __forceinline__ float4 f4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// Bounds-checking build (nvcc -DFDTD_CHECK_BOUNDS): every shared-memory
// load and store of the tile pipelines and every store to the output field
// goes through Chk, which tests the address against its allocation; an
// access outside is not performed (a load reads the allocation's first
// element and gives 0, a store is dropped) and counted per thread, and the
// count is added to *bad (the word after the wait budget) when the item
// ends (flush), so a debug run reports index errors without faulting the
// GPU.  The checks add no branch around an access.  In the normal build
// Chk is empty and the accessors are plain loads and stores.
struct Chk {
#ifdef FDTD_CHECK_BOUNDS
  const char* lo = nullptr;
  const char* hi = nullptr;
  int32_t* bad = nullptr;
  int miss = 0;
  __device__ __forceinline__ bool ok(const void* p, int bytes) {
    const char* q = (const char*)p;
    const bool good = q >= lo && q + bytes <= hi;
    miss += good ? 0 : 1;
    return good;
  }
#endif
  __device__ __forceinline__ void set(const void* l, const void* h, int32_t* err) {
#ifdef FDTD_CHECK_BOUNDS
    lo = (const char*)l;
    hi = (const char*)h;
    bad = err + 2;
    miss = 0;
#else
    (void)l, (void)h, (void)err;
#endif
  }
  __device__ __forceinline__ float4 ld4(const float* p) {
#ifdef FDTD_CHECK_BOUNDS
    const bool good = ok(p, 16);
    const float4 v = f4(good ? p : (const float*)lo);
    return good ? v : make_float4(0.f, 0.f, 0.f, 0.f);
#else
    return f4(p);
#endif
  }
  __device__ __forceinline__ float ld1(const float* p) {
#ifdef FDTD_CHECK_BOUNDS
    const bool good = ok(p, 4);
    const float v = *(good ? p : (const float*)lo);
    return good ? v : 0.f;
#else
    return *p;
#endif
  }
  __device__ __forceinline__ void st4(float* p, float4 v) {
#ifdef FDTD_CHECK_BOUNDS
    if (!ok(p, 16)) return;
#endif
    *reinterpret_cast<float4*>(p) = v;
  }
  // BF16 storage: four sites (8 bytes) widened to FP32, one site, and four
  // FP32 values rounded to BF16 and stored
  __device__ __forceinline__ float4 ld4(const __nv_bfloat16* p) {
#ifdef FDTD_CHECK_BOUNDS
    const bool good = ok(p, 8);
    const uint2 u = *reinterpret_cast<const uint2*>(good ? (const char*)p : lo);
#else
    const uint2 u = *reinterpret_cast<const uint2*>(p);
#endif
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
#ifdef FDTD_CHECK_BOUNDS
    if (!good) return make_float4(0.f, 0.f, 0.f, 0.f);
#endif
    return make_float4(a.x, a.y, b.x, b.y);
  }
  __device__ __forceinline__ float ld1(const __nv_bfloat16* p) {
#ifdef FDTD_CHECK_BOUNDS
    const bool good = ok(p, 2);
    const float v = __bfloat162float(*(good ? p : (const __nv_bfloat16*)lo));
    return good ? v : 0.f;
#else
    return __bfloat162float(*p);
#endif
  }
  __device__ __forceinline__ void st4(__nv_bfloat16* p, float4 v) {
#ifdef FDTD_CHECK_BOUNDS
    if (!ok(p, 8)) return;
#endif
    __nv_bfloat162 a, b;
    a.x = __float2bfloat16_rn(v.x);
    a.y = __float2bfloat16_rn(v.y);
    b.x = __float2bfloat16_rn(v.z);
    b.y = __float2bfloat16_rn(v.w);
    uint2 u;
    u.x = *reinterpret_cast<const unsigned*>(&a);
    u.y = *reinterpret_cast<const unsigned*>(&b);
    *reinterpret_cast<uint2*>(p) = u;
  }
  // add this thread's count of accesses outside the allocation to *bad
  __device__ __forceinline__ void flush() {
#ifdef FDTD_CHECK_BOUNDS
    if (miss) atomicAdd(bad, miss);
    miss = 0;
#endif
  }
};

// One float4 of site updates: c at x..x+3, xl = site x-1, xr = site x+4.
// The arithmetic of coef_f32 / nbr_sum / update_f32, evaluated on the site
// pairs (x, x+1) and (x+2, x+3) with packed two-lane FP32 instructions (each
// lane rounds exactly as the scalar _rn operation); om6c - h is taken as
// fma(h, -1, om6c), which is the same single rounding.
__device__ __forceinline__ float2 pr(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float4 update4(float4 c, float xl, float xr, float4 ym, float4 yp, float4 zm, float4 zp,
                                          float4 v, float hd, float om6c, float cc) {
  const float2 hd2 = pr(hd, hd), one2 = pr(1.0f, 1.0f), m1 = pr(-1.0f, -1.0f), om2 = pr(om6c, om6c), cc2 = pr(cc, cc);
  const float2 c0 = pr(c.x, c.y), c1 = pr(c.z, c.w);
  // ((xm + xp) + (ym + yp)) + (zm + zp) per site
  const float2 s0 = __fadd2_rn(__fadd2_rn(__fadd2_rn(pr(xl, c.x), pr(c.y, c.z)), __fadd2_rn(pr(ym.x, ym.y), pr(yp.x, yp.y))),
                               __fadd2_rn(pr(zm.x, zm.y), pr(zp.x, zp.y)));
  const float2 s1 = __fadd2_rn(__fadd2_rn(__fadd2_rn(pr(c.y, c.z), pr(c.w, xr)), __fadd2_rn(pr(ym.z, ym.w), pr(yp.z, yp.w))),
                               __fadd2_rn(pr(zm.z, zm.w), pr(zp.z, zp.w)));
  // h = hd V, b = 1 / (1 + h), alpha = (1 - 6c) - h
  const float2 h0 = __fmul2_rn(hd2, pr(v.x, v.y)), h1 = __fmul2_rn(hd2, pr(v.z, v.w));
  const float2 q0 = __fadd2_rn(one2, h0), q1 = __fadd2_rn(one2, h1);
  const float2 b0 = pr(rcp_approx(q0.x), rcp_approx(q0.y)), b1 = pr(rcp_approx(q1.x), rcp_approx(q1.y));
  const float2 a0 = __ffma2_rn(h0, m1, om2), a1 = __ffma2_rn(h1, m1, om2);
  // psi' = b (c S + alpha psi)
  const float2 o0 = __fmul2_rn(b0, __ffma2_rn(cc2, s0, __fmul2_rn(a0, c0)));
  const float2 o1 = __fmul2_rn(b1, __ffma2_rn(cc2, s1, __fmul2_rn(a1, c1)));
  return make_float4(o0.x, o0.y, o1.x, o1.y);
}

// The ring pipeline: barriers, prologue, and the bounded waits.  Step items
// also use the block's step barrier (an mbarrier counting every thread):
// a thread arrives after its last level-plane store of a z-step and waits
// for that phase in the middle of the next z-step.
template <int K, int TXT, int TYT = TY, typename PT = float>
struct Pipe {
  using G = Geo<K, TXT, TYT, PT>;
  static constexpr int R = G::R;
  static constexpr int D = G::D;
  char* smem;
  const CUtensorMap* mpsi;
  const CUtensorMap* mv;
  int x0, y0;
  const int32_t* err;
  long long budget = 0;  // wall-clock wait budget in ns (< 0: do not wait)
  uint64_t* bars;
  uint64_t* cbar;
  int* flag;  // shared: set by any thread whose wait expired, read by all after a barrier
  float* ring;
  unsigned phase = 0;        // bit s: parity of the next wait on slot s (toggled on success)
  unsigned outstanding = 0;  // (thread 0) slots with a copy in flight
  int timeout = 0;

  __device__ __forceinline__ void issue(int q, int s) {
    char* box = (char*)ring + s * G::SLOT_BYTES;
    uint64_t* bar = bars + s;
    mbar_expect_tx(bar, G::TX_BYTES);
    tma_load_3d(box, mpsi, x0 - G::HXP, y0 - K, q, bar);
    tma_load_3d(box + G::PSI_BYTES, mv, x0 - HX, y0 - K, q, bar);
    outstanding |= 1u << s;
  }
  __device__ __forceinline__ void wait(int s) {
    if (mbar_wait_bounded(bars + s, (phase >> s) & 1u, err, budget)) {
      phase ^= 1u << s;
      outstanding &= ~(1u << s);
    } else {
      timeout = 1;
    }
  }
  // Set up barriers and issue planes j0-1 .. min(j0+D, jlast) into slots 0, 1, ...;
  // with `step`, also the step barrier and its first phase (the item start).
  __device__ __forceinline__ void begin(int j0, int jlast, bool step = false) {
    bars = (uint64_t*)(smem + G::BAR_OFF);
    cbar = (uint64_t*)(smem + G::CBAR_OFF);
    flag = (int*)(smem + G::FLAG_OFF);
    ring = (float*)(smem + G::RING_OFF);
    budget = wait_budget_ns(err);
    if (threadIdx.x == 0) {
      *(volatile int*)flag = 0;
      for (int s = 0; s < R; ++s) mbar_init(bars + s, 1);
      // every thread of the block arrives (a batched launch runs shallower
      // items with the deepest item's block size)
      if (step) mbar_init(cbar, blockDim.x);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      int s = 0;
      for (int q = j0 - 1; q <= min(j0 + D, jlast); ++q, s = slot_add<R>(s, 1)) issue(q, s);
    }
    wait(0);
    wait(1);
    if (step) cta_arrive();
  }
  // Issue plane j + 1 + D into the slot of plane j + 1 + D - R (thread 0;
  // no new copy after an expired wait).
  __device__ __forceinline__ void refill(int j, int sj, int jlast) {
    if (threadIdx.x == 0 && !timeout && j + 1 + D <= jlast) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(j + 1 + D, slot_add<R>(sj, 1 + D));
    }
  }
  // Start of iteration j (slot sj): prefetch plane j+1+D, wait for plane j+1.
  __device__ __forceinline__ void advance(int j, int sj, int jlast) {
    refill(j, sj, jlast);
    wait(slot_add<R>(sj, 1));
  }
  // End of a z-step of a sums item: a thread whose wait expired marks the
  // shared flag and the barrier publishes it.
  __device__ __forceinline__ void end_step() {
    if (timeout) *(volatile int*)flag = 1;
    __syncthreads();
  }
  // The step barrier: arrive (after marking the flag if a wait expired) and
  // wait for a phase, bounded like every wait.
  __device__ __forceinline__ void cta_arrive() {
    if (timeout) *(volatile int*)flag = 1;
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(cbar)) : "memory");
  }
  __device__ __forceinline__ void cta_wait(unsigned parity) {
    if (!mbar_wait_bounded(cbar, parity, err, budget)) timeout = 1;
  }
  // After a barrier: every thread reads the same flag; on a timeout drain
  // and report.
  __device__ __forceinline__ bool ok(int32_t* err_w) {
    if (*(volatile const int*)flag) {
      if (threadIdx.x == 0) {
        atomicOr(err_w, 1);
        for (int s = 0; s < R; ++s) {
          if (!(outstanding & (1u << s))) continue;
          const unsigned long long t0 = global_ns();
          while (!mbar_try_wait(bars + s, (phase >> s) & 1u) && global_ns() - t0 < kWaitLimitNs) {
          }
        }
      }
      return false;
    }
    return true;
  }
  __device__ __forceinline__ const float* box(int s) const { return ring + s * (G::SLOT_BYTES / 4); }
  // End of an item, after its last barrier and ok(): the barriers are
  // invalidated (thread 0) before the next item initialises barriers or
  // stores data in the same shared memory (a barrier's memory may be reused
  // only after mbarrier.inval; without it, blocks that ran several items
  // gave up waits in some builds).
  __device__ __forceinline__ void finish(bool step) {
    if (threadIdx.x == 0) {
      for (int s = 0; s < R; ++s) mbar_inval(bars + s);
      if (step) mbar_inval(cbar);
    }
  }
};

// The lattice sums' contribution of four sites c (x .. x + 3) with their
// neighbours (xl = site x - 1, xr = site x + 4) and potential: S0 += c^2,
// SH += c (-kfac Lap c + V c), Sr += r^2 c^2, SV += V c^2 (Eq. energysum),
// every operation rounding on its own, Kahan-compensated per accumulator.
// The sums item and the check step's fused sums both use it, so their
// partial sums agree bit for bit.
__device__ __forceinline__ void sums_site4(Kahan& s0, Kahan& sh, Kahan& sr, Kahan& sv, float4 c, float xl, float xr,
                                           float4 ym, float4 yp, float4 zm, float4 zp, float4 v, const float (&px)[4],
                                           float py, float pz, float kfac) {
  const float cs[4] = {c.x, c.y, c.z, c.w};
  const float xls[4] = {xl, c.x, c.y, c.z};
  const float xrs[4] = {c.y, c.z, c.w, xr};
  const float yms[4] = {ym.x, ym.y, ym.z, ym.w}, yps[4] = {yp.x, yp.y, yp.z, yp.w};
  const float zms[4] = {zm.x, zm.y, zm.z, zm.w}, zps[4] = {zp.x, zp.y, zp.z, zp.w};
  const float vs[4] = {v.x, v.y, v.z, v.w};
  const float r2yz = __fadd_rn(__fmul_rn(py, py), __fmul_rn(pz, pz));
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float ci = cs[i];
    // sum of neighbour differences (exact for neighbours within a factor 2)
    const float lap = __fadd_rn(__fadd_rn(__fadd_rn(__fsub_rn(xls[i], ci), __fsub_rn(xrs[i], ci)),
                                          __fadd_rn(__fsub_rn(yms[i], ci), __fsub_rn(yps[i], ci))),
                                __fadd_rn(__fsub_rn(zms[i], ci), __fsub_rn(zps[i], ci)));
    const float c2 = __fmul_rn(ci, ci);
    s0.add(c2);
    sh.add(__fmul_rn(ci, __fadd_rn(__fmul_rn(-kfac, lap), __fmul_rn(vs[i], ci))));
    sr.add(__fmul_rn(__fadd_rn(__fmul_rn(px[i], px[i]), r2yz), c2));
    sv.add(__fmul_rn(vs[i], c2));
  }
}

// The value a BF16 field stores for each of four FP32 results (FP32 storage:
// the results themselves), so that a temporally blocked BF16 item rounds
// every level as a one-step kernel rounds every stored step.
template <typename PT>
__device__ __forceinline__ float4 stored4(float4 r) {
  if constexpr (sizeof(PT) == 4) {
    return r;
  } else {
    return make_float4(__bfloat162float(__float2bfloat16_rn(r.x)), __bfloat162float(__float2bfloat16_rn(r.y)),
                       __bfloat162float(__float2bfloat16_rn(r.z)), __bfloat162float(__float2bfloat16_rn(r.w)));
  }
}

// Per-thread constants of a step item: the shared-memory bases every access
// adds a compile-time offset to, the output column, and which levels this
// thread's column computes.
template <int K, int TXT, int TYT = TY, typename PT = float>
struct StepCtx {
  using G = Geo<K, TXT, TYT, PT>;
  const float* rb;   // ring + this thread's offset in a box (FP32 psi: the psi box, V at + PLANE;
                     // BF16 psi: the V box)
  const PT* rp;      // BF16 psi: ring + this thread's offset in the psi box
  float* lb;         // level planes + this thread's offset in a level plane
  PT* out;           // the output field
  long long ooff;    // offset of this thread's output column at the plane level K writes this
                     // z-step (negative before the lattice: only planes in [z0, z1) are stored)
  size_t plane;      // n * n
  int z0, z1;       // output planes of the item
  int zlo, zhi;      // planes of the field inside the lattice (outside: zero at every level)
  bool owner, fix_l, fix_r, interior_row;
  bool need[K + 1];  // level l computes this column (without the z tests)
  float hd, om6c, cc;
  Chk sm, gl;        // shared memory of the item, the output field
  // check step (level 1 the update, level 2 the sums of its output): the
  // column is inside the tile, the coordinates of its sites, the sums
  bool interior_col;
  int n;
  float a, kfac, py;
  float px[4];
  Kahan s0, sh, sr, sv;
};

// One z-step of a step item.  U = (j - j0) mod 6 makes every ring slot, the
// register-window rotation and the level-plane buffers compile-time
// constants: plane q sits in ring slot (q - j0 + 1) mod 6; level 1's plane p
// in buffer (p - j0) mod 3; level l's (1 < l < K) in buffer (p - j0) mod 2;
// the three window registers of each level rotate by renaming (after level l
// computes its new plane into w[l][U mod 3] the window reads zm = w[(U+1)%3],
// c = w[(U+2)%3], zp = w[U%3]).
//
// Level 1 needs only ring data, so it runs before the step barrier (the
// wait for every thread's stores of the previous z-step); the ring refill,
// which overwrites a plane last read in the previous z-step, and levels
// 2..K follow it; the thread arrives after its last store.  STEADY: every
// level's plane lies inside the lattice and level K's inside [z0, z1), so
// no z tests are needed.
//
// Sites outside the lattice must read as zero at every level.  The level
// planes and windows start each item at zero, so a site is simply never
// written when it lies outside the lattice in x or y (the thread does not
// compute) or below it in z (p < 0 comes first in an item); above it
// (p >= n, block-uniform) zeros are written.  The last level computes only
// the planes it stores.
template <int K, int TXT, int TYT, typename PT, int U, bool STEADY, bool SUMS = false>
__device__ __forceinline__ void step_iteration(StepCtx<K, TXT, TYT, PT>& x, Pipe<K, TXT, TYT, PT>& pp, int j, int jlast,
                                               float4 (&w)[K > 1 ? K - 1 : 1][3]) {
  using G = Geo<K, TXT, TYT, PT>;
  constexpr int R = G::R;
  static_assert(R == 6, "the step assumes a six-slot ring");
  constexpr int SJ = (U + 1) % R;  // slot of plane j
  constexpr int I0 = U % 3, I1 = (U + 1) % 3, I2 = (U + 2) % 3;
  constexpr int SL = G::SLOT_BYTES / 4;
  constexpr int BW = G::BW, LW = G::LW;
  // psi in the ring: slot stride and row pitch in PT elements; V at VOFF
  // floats from x.rb in every slot
  constexpr int SLP = (int)(G::SLOT_BYTES / G::PS), PW = G::PS == 4 ? BW : G::BWP;
  constexpr int VOFF = G::PS == 4 ? G::PLANE : 0;
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  pp.wait((SJ + 1) % R);  // plane j + 1
  // ---- level 1: plane j from the ring
  {
    const int p = j;
    constexpr int S0 = SJ, SM = (SJ + R - 1) % R, SP = (SJ + 1) % R;
    const PT* pr0;
    if constexpr (G::PS == 4)
      pr0 = x.rb;
    else
      pr0 = x.rp;
    const PT* b0 = pr0 + S0 * SLP;
    float4 c = x.owner ? x.sm.ld4(b0) : zero4;
    float xl = __shfl_up_sync(0xffffffffu, c.w, 1);
    float xr = __shfl_down_sync(0xffffffffu, c.x, 1);
    // lanes 0 and 31 read their outer neighbour from shared memory (at a row
    // end the neighbouring row's value is taken, which only reaches margins)
    if (x.fix_l) xl = x.sm.ld1(b0 - 1);
    if (x.fix_r) xr = x.sm.ld1(b0 + 4);
    auto upd = [&]() {
      return update4(c, xl, xr, x.sm.ld4(b0 - PW), x.sm.ld4(b0 + PW), x.sm.ld4(pr0 + SM * SLP),
                     x.sm.ld4(pr0 + SP * SLP), x.sm.ld4(x.rb + S0 * SL + VOFF), x.hd, x.om6c, x.cc);
    };
    if constexpr (K == 1) {
      if (x.need[1] && x.interior_row && (STEADY || (p >= x.z0 && p < x.z1))) x.gl.st4(x.out + x.ooff, upd());
    } else {
      float* dst = x.lb + (U % 3) * G::LPLANE;
      if constexpr (STEADY) {
        if (x.need[1]) {
          const float4 r = stored4<PT>(upd());
          x.sm.st4(dst, r);
          w[0][I0] = r;
          // the check step: level 1 is the output (plane j, one after level K's)
          if constexpr (SUMS)
            if (x.interior_row && x.interior_col && p >= x.z0 && p < x.z1) x.gl.st4(x.out + x.ooff + x.plane, r);
        }
      } else if (p >= x.zhi) {
        if (x.need[1]) {
          x.sm.st4(dst, zero4);
          w[0][I0] = zero4;
        }
      } else if (p >= x.zlo && x.need[1]) {
        const float4 r = stored4<PT>(upd());
        x.sm.st4(dst, r);
        w[0][I0] = r;
        if constexpr (SUMS)
          if (x.interior_row && x.interior_col && p >= x.z0 && p < x.z1) x.gl.st4(x.out + x.ooff + x.plane, r);
      }
    }
  }
  pp.cta_wait(U & 1);  // every thread's stores of z-step j - 1
  pp.refill(j, SJ, jlast);
  // ---- levels 2..K: plane j - l + 1 from level l-1
#pragma unroll
  for (int l = 2; l <= K; ++l) {
    const int p = j - l + 1;
    const float* lp = l == 2 ? x.lb + ((U + 5) % 3) * G::LPLANE                         // level 1, plane j - 1
                             : x.lb + (3 + 2 * (l - 3) + ((U - l + 7) & 1)) * G::LPLANE;  // level l-1, plane p
    const float4 c = w[l - 2][I2];
    float xl = __shfl_up_sync(0xffffffffu, c.w, 1);
    float xr = __shfl_down_sync(0xffffffffu, c.x, 1);
    if (x.fix_l) xl = x.sm.ld1(lp - 1);
    if (x.fix_r) xr = x.sm.ld1(lp + 4);
    auto upd = [&]() {
      return update4(c, xl, xr, x.sm.ld4(lp - LW), x.sm.ld4(lp + LW), w[l - 2][I1], w[l - 2][I0],
                     x.sm.ld4(x.rb + ((SJ - l + 1 + 2 * R) % R) * SL + VOFF), x.hd, x.om6c, x.cc);
    };
    if (l == K) {
      if constexpr (SUMS) {  // the sums of level K-1's output (the update) at plane p
        if (x.need[K] && x.interior_row && (STEADY || (p >= x.z0 && p < x.z1)))
          sums_site4(x.s0, x.sh, x.sr, x.sv, c, xl, xr, x.sm.ld4(lp - LW), x.sm.ld4(lp + LW), w[l - 2][I1],
                     w[l - 2][I0], x.sm.ld4(x.rb + ((SJ - l + 1 + 2 * R) % R) * SL + VOFF), x.px, x.py,
                     coord_f32(p, x.n, x.a), x.kfac);
      } else {
        if (x.need[K] && x.interior_row && (STEADY || (p >= x.z0 && p < x.z1))) x.gl.st4(x.out + x.ooff, upd());
      }
    } else {
      float* dst = x.lb + (3 + 2 * (l - 2) + ((U - l + 7) & 1)) * G::LPLANE;
      if constexpr (STEADY) {
        if (x.need[l]) {
          const float4 r = stored4<PT>(upd());
          x.sm.st4(dst, r);
          w[l - 1][I0] = r;
        }
      } else if (p >= x.zhi) {
        if (x.need[l]) {
          x.sm.st4(dst, zero4);
          w[l - 1][I0] = zero4;
        }
      } else if (p >= x.zlo && x.need[l]) {
        const float4 r = stored4<PT>(upd());
        x.sm.st4(dst, r);
        w[l - 1][I0] = r;
      }
    }
  }
  pp.cta_arrive();
  x.ooff += (long long)x.plane;
}

// Six z-steps from j (j - j0 a multiple of 6); a partial group stops after
// step j1.
template <int K, int TXT, int TYT, typename PT, bool STEADY, bool SUMS = false>
__device__ __forceinline__ void step_group(StepCtx<K, TXT, TYT, PT>& x, Pipe<K, TXT, TYT, PT>& pp, int& j, int j1,
                                           float4 (&w)[K > 1 ? K - 1 : 1][3]) {
  const int jl = j1 + 1;
  step_iteration<K, TXT, TYT, PT, 0, STEADY, SUMS>(x, pp, j, jl, w);
  if (!STEADY && j + 1 > j1) { j += 1; return; }
  step_iteration<K, TXT, TYT, PT, 1, STEADY, SUMS>(x, pp, j + 1, jl, w);
  if (!STEADY && j + 2 > j1) { j += 2; return; }
  step_iteration<K, TXT, TYT, PT, 2, STEADY, SUMS>(x, pp, j + 2, jl, w);
  if (!STEADY && j + 3 > j1) { j += 3; return; }
  step_iteration<K, TXT, TYT, PT, 3, STEADY, SUMS>(x, pp, j + 3, jl, w);
  if (!STEADY && j + 4 > j1) { j += 4; return; }
  step_iteration<K, TXT, TYT, PT, 4, STEADY, SUMS>(x, pp, j + 4, jl, w);
  if (!STEADY && j + 5 > j1) { j += 5; return; }
  step_iteration<K, TXT, TYT, PT, 5, STEADY, SUMS>(x, pp, j + 5, jl, w);
  j += 6;
}

// K update steps on one tile item: output planes [z0, z1) of a field of
// n x n x nz sites (nz = n: a whole lattice).  Planes outside [zlo, zhi) are
// outside the lattice and stay zero at every level (a whole lattice: [0, n);
// a z-slab with K-plane halos: the halo planes beyond the lattice's faces);
// the planes beyond the field read as zero (TMA fill).  Returns false (in
// every thread) if a bounded wait expired.
template <int K, int TXT, int TYT = TY, typename PT = float>
__device__ bool tma_step_item(char* smem, const CUtensorMap* map_psi, const CUtensorMap* map_v,
                              PT* __restrict__ out, int n, int x0, int y0, int z0, int z1, float half_dtau,
                              float one_m6c, float cc, int32_t* err, int nz = -1, int zlo = 0, int zhi = -1) {
  if (nz < 0) nz = n;
  if (zhi < 0) zhi = nz;
  using G = Geo<K, TXT, TYT, PT>;
  constexpr int C4 = G::C4;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  StepCtx<K, TXT, TYT, PT> x;
  x.owner = tid < G::USED;
  const int row = x.owner ? tid / C4 : 0;
  const int col = x.owner ? tid % C4 : 0;
  const int xg = x0 - HX + 4 * col;
  const int yg = y0 - K + row;
  const bool inside = x.owner && (xg >= 0) && (xg < n) && (yg >= 0) && (yg < n);
  const bool interior_col = (col >= HX / 4) && (col < HX / 4 + G::TX / 4);
  x.interior_row = x.owner && (row >= K) && (row < K + TYT);
  x.fix_l = x.owner && lane == 0 && col > 0;
  x.fix_r = x.owner && lane == 31 && col < C4 - 1;
#pragma unroll
  for (int l = 1; l <= K; ++l) x.need[l] = inside && (row >= l && row < G::BH - l) && (l < K || interior_col);
  x.z0 = z0;
  x.z1 = z1;
  x.zlo = zlo;
  x.zhi = zhi;
  x.hd = half_dtau;
  x.om6c = one_m6c;
  x.cc = cc;
  float* lev = (float*)(smem + G::LEVEL_OFF);
  x.lb = lev + row * G::LW + 4 + 4 * col;
  if constexpr (G::PS == 4) {
    x.rb = (const float*)(smem + G::RING_OFF) + row * G::BW + 4 * col;
  } else {
    x.rb = (const float*)(smem + G::RING_OFF + G::PSI_BYTES) + row * G::BW + 4 * col;
    x.rp = (const PT*)(smem + G::RING_OFF) + row * G::BWP + G::XOFF + 4 * col;
  }
  x.plane = (size_t)n * n;
  x.sm.set(smem, smem + (G::SMEM - 128), err);
  x.gl.set(out, out + (size_t)n * n * nz, err);
  const int j0 = z0 - K + 1, j1 = z1 + K - 2;
  // level K writes plane j - K + 1 at z-step j (only planes in [z0, z1) are
  // stored, so the offset is never dereferenced while negative)
  x.out = out;
  x.ooff = (long long)yg * n + xg + (long long)(j0 - K + 1) * (long long)x.plane;

  for (int i = tid; i < G::NLEV * G::LPLANE; i += blockDim.x) lev[i] = 0.f;
  Pipe<K, TXT, TYT, PT> pp;
  pp.smem = smem;
  pp.mpsi = map_psi;
  pp.mv = map_v;
  pp.x0 = x0;
  pp.y0 = y0;
  pp.err = err;
  pp.begin(j0, j1 + 1, true);

  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 w[K > 1 ? K - 1 : 1][3];
#pragma unroll
  for (int l = 0; l < (K > 1 ? K - 1 : 1); ++l) w[l][0] = w[l][1] = w[l][2] = zero4;
  // steady z-steps: level K's plane j - K + 1 in [z0, z1) and level 1's
  // plane j in [0, n)
  const int ss = z0 + K - 1, se = min(z1 + K - 2, zhi - 1);
  int j = j0;
  while (j <= j1) {
    if (j >= ss && j + 5 <= se)
      step_group<K, TXT, TYT, PT, true>(x, pp, j, j1, w);
    else
      step_group<K, TXT, TYT, PT, false>(x, pp, j, j1, w);
    // an expired wait seen early ends the loop; the decision that counts is
    // taken below, after a barrier, the same in every thread
    if (*(volatile const int*)pp.flag) break;
  }
  // every thread's last z-step is complete before the caller's next item
  // reinitialises the shared memory
  pp.cta_wait((unsigned)((j - j0) & 1));
  x.sm.flush();
  x.gl.flush();
  __syncthreads();
  const bool good = pp.ok(err);
  pp.finish(true);
  return good;
}

// The check step: one update step on a 64 x TY tile item, planes [z0, z1),
// whose result is also summed (S0, SH, Sr, SV of Eq. energysum) -- the
// depth-2 item with level 2 replaced by the sums of level 1's output.  The
// item is one of the lattice sums' items (the same tile, z-chunk and
// partial index), and its partial sums are bit-identical to that item's:
// the same per-site arithmetic (sums_site4) in the same order per site
// column, and each thread's totals moved to the thread that holds the same
// column in the sums item before the same fixed-order block reduction.
// Writes psi_t to out and the four totals to dst[0..3]; false if a bounded
// wait expired.
template <int TXT>
__device__ bool tma_step_sums_item(char* smem, const CUtensorMap* map_psi, const CUtensorMap* map_v,
                                   float* __restrict__ out, int n, int x0, int y0, int z0, int z1, float half_dtau,
                                   float one_m6c, float cc, float a, float kfac, double* __restrict__ dst,
                                   int32_t* err) {
  constexpr int K = 2;
  using G = Geo<K, TXT>;
  using GS = Geo<1, TXT>;  // the sums item's layout
  static_assert(G::C4 == GS::C4, "the sums layout differs from the step layout by whole rows");
  constexpr int C4 = G::C4;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  StepCtx<K, TXT> x;
  x.owner = tid < G::USED;
  const int row = x.owner ? tid / C4 : 0;
  const int col = x.owner ? tid % C4 : 0;
  const int xg = x0 - HX + 4 * col;
  const int yg = y0 - K + row;
  const bool inside = x.owner && (xg >= 0) && (xg < n) && (yg >= 0) && (yg < n);
  x.interior_col = (col >= HX / 4) && (col < HX / 4 + G::TX / 4);
  x.interior_row = x.owner && (row >= K) && (row < K + TY);
  x.fix_l = x.owner && lane == 0 && col > 0;
  x.fix_r = x.owner && lane == 31 && col < C4 - 1;
#pragma unroll
  for (int l = 1; l <= K; ++l) x.need[l] = inside && (row >= l && row < G::BH - l) && (l < K || x.interior_col);
  x.z0 = z0;
  x.z1 = z1;
  x.zlo = 0;
  x.zhi = n;
  x.hd = half_dtau;
  x.om6c = one_m6c;
  x.cc = cc;
  x.n = n;
  x.a = a;
  x.kfac = kfac;
  x.py = coord_f32(yg, n, a);
#pragma unroll
  for (int i = 0; i < 4; ++i) x.px[i] = coord_f32(xg + i, n, a);
  float* lev = (float*)(smem + G::LEVEL_OFF);
  x.lb = lev + row * G::LW + 4 + 4 * col;
  x.rb = (const float*)(smem + G::RING_OFF) + row * G::BW + 4 * col;
  x.plane = (size_t)n * n;
  x.sm.set(smem, smem + (G::SMEM - 128), err);
  x.gl.set(out, out + (size_t)n * n * n, err);
  const int j0 = z0 - K + 1, j1 = z1 + K - 2;
  x.out = out;
  x.ooff = (long long)yg * n + xg + (long long)(j0 - K + 1) * (long long)x.plane;

  for (int i = tid; i < G::NLEV * G::LPLANE; i += blockDim.x) lev[i] = 0.f;
  Pipe<K, TXT> pp;
  pp.smem = smem;
  pp.mpsi = map_psi;
  pp.mv = map_v;
  pp.x0 = x0;
  pp.y0 = y0;
  pp.err = err;
  pp.begin(j0, j1 + 1, true);

  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 w[K - 1][3];
  w[0][0] = w[0][1] = w[0][2] = zero4;
  const int ss = z0 + K - 1, se = min(z1 + K - 2, n - 1);
  int j = j0;
  while (j <= j1) {
    if (j >= ss && j + 5 <= se)
      step_group<K, TXT, TY, float, true, true>(x, pp, j, j1, w);
    else
      step_group<K, TXT, TY, float, false, true>(x, pp, j, j1, w);
    if (*(volatile const int*)pp.flag) break;
  }
  pp.cta_wait((unsigned)((j - j0) & 1));
  x.sm.flush();
  x.gl.flush();
  __syncthreads();
  const bool good = pp.ok(err);
  pp.finish(true);
  if (!good) return false;
  // each thread's totals to the sums item's thread of the same site column
  // (K - 1 rows earlier: row r here is row r - 1 there), then that item's
  // reduction over its warps
  double* slot = (double*)(smem + G::LEVEL_OFF);  // the level planes are free now
  constexpr int SHIFT = (K - 1) * C4;
  for (int i = tid; i < GS::THREADS * 4; i += blockDim.x) slot[i] = 0.0;
  __syncthreads();
  if (tid >= SHIFT && tid - SHIFT < GS::THREADS) {
    double* d = slot + (size_t)(tid - SHIFT) * 4;
    d[0] = x.s0.value();
    d[1] = x.sh.value();
    d[2] = x.sr.value();
    d[3] = x.sv.value();
  }
  __syncthreads();
  double v4[4] = {0.0, 0.0, 0.0, 0.0};
  if (tid < GS::THREADS)
#pragma unroll
    for (int q = 0; q < 4; ++q) v4[q] = slot[(size_t)tid * 4 + q];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v4[q] += __shfl_down_sync(0xffffffffu, v4[q], off);
  double* red = (double*)(smem + G::RED_OFF);
  if (lane == 0 && tid < GS::THREADS)
#pragma unroll
    for (int q = 0; q < 4; ++q) red[(tid >> 5) * 4 + q] = v4[q];
  __syncthreads();
  if (tid < 4) {
    double acc = 0.0;
    for (int wi = 0; wi < GS::THREADS / 32; ++wi) acc += red[wi * 4 + tid];
    dst[tid] = acc;
  }
  __syncthreads();
  return true;
}

// Partition of the lattice sums: 64 x TY tile columns cut along z into
// chunks of sums_zchunk(n) planes, item (chunk, ty, tx) at index
// (chunk * gy + ty) * gx + tx.  A function of n only, so every kernel that
// sums a lattice (one lattice, batched, allocation-free) adds the same
// partials in the same order: about four items per SM of a 152-SM device,
// chunks of at least 16 planes, at most 4096 items.
// A z-slab of nz planes of an n x n cross-section is cut the same way.
constexpr int kSumsTX = 64;
__host__ __device__ inline int sums_zchunk_of(int n, int nz) {
  const int tiles = ((n + kSumsTX - 1) / kSumsTX) * ((n + TY - 1) / TY);
  int zs = (608 + tiles - 1) / tiles;
  const int by_planes = nz / 16 > 1 ? nz / 16 : 1, by_count = 4096 / tiles > 1 ? 4096 / tiles : 1;
  zs = zs < by_planes ? zs : by_planes;
  zs = zs < by_count ? zs : by_count;
  return (nz + zs - 1) / zs;
}
__host__ __device__ inline int sums_zchunk(int n) { return sums_zchunk_of(n, n); }
__host__ __device__ inline int sums_items_of(int n, int nz) {
  const int zc = sums_zchunk_of(n, nz);
  return ((n + kSumsTX - 1) / kSumsTX) * ((n + TY - 1) / TY) * ((nz + zc - 1) / zc);
}
__host__ __device__ inline int sums_items(int n) { return sums_items_of(n, n); }

// Lattice sums over the tile interior, planes [z0, z1) of the mapped field,
// whose plane j is the lattice's plane j + zoff (zoff != 0 for a z-slab with
// halo planes); the block's four totals (FP64) go to dst[0..3].  With
// zc > 0 the planes are cut at the multiples of zc (z0 must be one) and
// each piece's totals go to dst + c * dst_stride (c = 0, 1, ... in z order):
// several consecutive sums items of one tile column in one pipeline run,
// each piece's totals equal to those of a separate item over it.  Returns
// false if a bounded wait expired.
template <int TXT>
__device__ bool tma_sums_item(char* smem, const CUtensorMap* map_psi, const CUtensorMap* map_v, int n, int x0,
                              int y0, int z0, int z1, float a, float kfac, double* __restrict__ dst, int32_t* err,
                              int zoff = 0, int zc = 0, long long dst_stride = 0) {
  using G = Geo<1, TXT>;
  constexpr int R = G::R;
  constexpr int C4 = G::C4, BW = G::BW;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const bool owner = tid < G::USED;
  const int row = owner ? tid / C4 : 0, col = owner ? tid % C4 : 0;
  const int xg = x0 - HX + 4 * col;
  const int yg = y0 - 1 + row;
  const bool use = owner && (xg >= 0) && (xg < n) && (yg >= 0) && (yg < n) && row >= 1 && row < 1 + TY &&
                   col >= HX / 4 && col < HX / 4 + G::TX / 4;
  const bool fix_l = owner && lane == 0 && col > 0;
  const bool fix_r = owner && lane == 31 && col < C4 - 1;
  const int ro = row * BW + 4 * col;
  Chk sm;
  sm.set(smem, smem + (G::SMEM - 128), err);
  const float py = coord_f32(yg, n, a);
  float px[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) px[i] = coord_f32(xg + i, n, a);
  Kahan s0, sh, sr, sv;
  // fixed-order block reduction of the four accumulators into d[0..3]
  // (every thread; the caller's last barrier separates it from the
  // previous reduction's reads)
  double* red = (double*)(smem + G::RED_OFF);
  auto reduce_to = [&](double* d) {
    double v4[4] = {s0.value(), sh.value(), sr.value(), sv.value()};
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v4[q] += __shfl_down_sync(0xffffffffu, v4[q], off);
    if (lane == 0 && tid < G::THREADS)
#pragma unroll
      for (int q = 0; q < 4; ++q) red[(tid >> 5) * 4 + q] = v4[q];
    __syncthreads();
    if (tid < 4) {
      double acc = 0.0;
      for (int w = 0; w < G::THREADS / 32; ++w) acc += red[w * 4 + tid];
      d[tid] = acc;
    }
  };
  Pipe<1, TXT> pp;
  pp.smem = smem;
  pp.mpsi = map_psi;
  pp.mv = map_v;
  pp.x0 = x0;
  pp.y0 = y0;
  pp.err = err;
  const int j0 = z0, j1 = z1 - 1;
  pp.begin(j0, j1 + 1);
  int sj = 1;
  for (int j = j0; j <= j1; ++j) {
    pp.advance(j, sj, j1 + 1);
    const float* b0 = pp.box(sj);
    const float* bm = pp.box(slot_add<R>(sj, -1));
    const float* bp = pp.box(slot_add<R>(sj, 1));
    float4 c = owner ? sm.ld4(b0 + ro) : make_float4(0.f, 0.f, 0.f, 0.f);
    float xl = __shfl_up_sync(0xffffffffu, c.w, 1);
    float xr = __shfl_down_sync(0xffffffffu, c.x, 1);
    if (fix_l) xl = sm.ld1(b0 + ro - 1);
    if (fix_r) xr = sm.ld1(b0 + ro + 4);
    if (use) {
      const float4 ym = sm.ld4(b0 + ro - BW), yp = sm.ld4(b0 + ro + BW), zm = sm.ld4(bm + ro), zp = sm.ld4(bp + ro);
      const float4 v = sm.ld4(b0 + G::PLANE + ro);
      sums_site4(s0, sh, sr, sv, c, xl, xr, ym, yp, zm, zp, v, px, py, coord_f32(j + zoff, n, a), kfac);
    }
    pp.end_step();
    if (!pp.ok(err)) {
      sm.flush();
      pp.finish(false);
      return false;
    }
    sj = slot_add<R>(sj, 1);
    if (zc > 0 && j < j1 && (j + 1) % zc == 0) {  // a piece ends inside the run
      reduce_to(dst);
      dst += dst_stride;
      s0 = Kahan{};
      sh = Kahan{};
      sr = Kahan{};
      sv = Kahan{};
    }
  }
  sm.flush();
  reduce_to(dst);
  pp.finish(false);
  __syncthreads();
  return true;
}

}  // namespace tb
}  // namespace fdtd
