// sweep.cu -- staged block triangular solves of the Block-Jacobi apply
// (Sec. 2.3: z = M^{-1} r with M = blockdiag(L_b L_b^T) or blockdiag(L_b U_b)).
//
// One CTA per diagonal block (all blocks are independent work of one launch).
// The block's rows are grouped by level (Sec. 2.2, level scheduling); the
// rows of one level are packed into 32-lane tiles, a row taking V lanes.
// Each tile is a contiguous byte record in HBM (format in precond.cu,
// k_vt_fill):
//   [16 B header: nr, ne, level, tiles of the two levels below]
//   [32 lane records, 8 B each][inverse diagonals, nr]
//   [block-local columns, ne x u16][values, ne]            (16-byte aligned parts)
// A row's entries are split into "near" ones (columns one level below the
// row, read by the row's leader lane) and "far" ones (two or more levels
// below, dealt round-robin to the row's lanes).
// Warp w of the CTA takes the block's tiles w, w+W, ... in order; its lanes
// keep cp.async copies of the next SLOTS-1 tiles in flight into the warp's
// shared-memory ring while the warp solves the current tile.  y lives in
// shared memory, initialised to a signalling-NaN sentinel; a tile polls
// (warp-uniformly, bounded) until every value it reads is no longer the
// sentinel, so no barrier separates the levels.
#include <cuda_bf16.h>

#include <type_traits>

#include "pcg_common.cuh"

namespace sdsl {

namespace {

constexpr int kSweepWarps = 16;
constexpr int kNear = 4;  // near entries per lane and round of the staged sweeps

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__host__ __device__ inline size_t align128(size_t x) { return (x + 127) & ~(size_t)127; }

// Sum within aligned lane groups of size V (a power of two, per lane): every
// lane takes part in every shuffle; a lane adds only partners of its group.
// Vmax is the warp's largest group (warp-uniform): wider offsets are skipped.
template <typename T>
__device__ __forceinline__ T segmented_sum(T v, int V, int Vmax) {
  for (int o = Vmax >> 1; o > 0; o >>= 1) {
    const T w = __shfl_xor_sync(0xffffffffu, v, o);
    if (o < V) v += w;
  }
  return v;
}

// ---- float-float arithmetic of the FP32-factor apply (apply_prec 48)
// A value is an unevaluated sum h + l of two floats (|l| <= ulp(h)/2 after
// renormalisation): about 48 significant bits on the FP32 pipes.  The
// building blocks are the error-free transformations TwoSum (Knuth) and
// TwoProd via a fused multiply-add (Dekker 1971), and the compensated dot
// product Dot2 of Ogita, Rump and Oishi (2005): every product's and every
// addition's rounding error is carried in a second accumulator.  The
// explicit _rn intrinsics keep the compiler from contracting or
// reassociating them.  With this arithmetic the apply of the FP32-stored
// factors is one fixed linear operator to ~1e-14 relative, as PCG assumes.
struct ff_tag {};
constexpr unsigned long long kFFSentinel = 0x7FA5A5A57FA5A5A5ull;  // hi word: the FP32 sentinel

__device__ __forceinline__ unsigned long long ff_pack(float h, float l) {
  return ((unsigned long long)__float_as_uint(h) << 32) | (unsigned long long)__float_as_uint(l);
}
__device__ __forceinline__ float ff_hi(unsigned long long v) { return __uint_as_float((unsigned)(v >> 32)); }
__device__ __forceinline__ float ff_lo(unsigned long long v) { return __uint_as_float((unsigned)v); }
// s + e = a + b exactly, s = fl(a + b)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (h, l) += (bh, bl), renormalised
__device__ __forceinline__ void ff_add(float& h, float& l, float bh, float bl) {
  float s, e;
  two_sum(h, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(l, bl));
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}
// Dot2 step: (s, c) += v * (xh + xl); s is the running sum, c collects the
// rounding errors of every product and sum.
__device__ __forceinline__ void dot2_step(float v, float xh, float xl, float& s, float& c) {
  const float p = __fmul_rn(v, xh);
  float pe = __fmaf_rn(v, xh, -p);  // exact: v*xh - p
  pe = __fmaf_rn(v, xl, pe);
  float t, e;
  two_sum(s, p, t, e);
  s = t;
  c = __fadd_rn(c, __fadd_rn(e, pe));
}
// (h, l) = split of a double into two floats, h + l = d to ~2^-48
__device__ __forceinline__ unsigned long long ff_from_double(double d) {
  const float h = __double2float_rn(d);
  const float l = __double2float_rn(d - (double)h);
  return ff_pack(h, l);
}
__device__ __forceinline__ double ff_to_double(unsigned long long v) { return (double)ff_hi(v) + (double)ff_lo(v); }

// Arithmetic of one sweep: the type X of a solved value in shared memory,
// the type VV of a factor value in registers, and a lane's accumulator.  A
// row's sum starts at -(right-hand side) in its leader lane, so that
// y = -(sum) * dinv at the end; the far entries feed two chains alternately
// (instruction-level parallelism; the slot order is fixed, so results are
// deterministic); the lanes' far sums are added into the leader before the
// row waits for its near entries, which the leader then adds one by one.
template <typename TS, typename TC, bool FF>
struct SweepArith {  // plain: TC = float or double
  using TSt = TS;
  using X = TC;
  using VV = TC;
  using D = TC;
  struct Acc {
    TC a0, a1;
  };
  static __device__ __forceinline__ X sent() { return sentinel(TC(0)); }
  static __device__ __forceinline__ bool is_sent(X x) { return is_sentinel(x); }
  static __device__ __forceinline__ VV val(TS v) {
    if constexpr (std::is_same<TS, __nv_bfloat16>::value) return (TC)__bfloat162float(v);
    else return (TC)v;
  }
  static __device__ __forceinline__ void init(Acc& a, X minus_in_of) { a.a0 = -minus_in_of; a.a1 = TC(0); }
  static __device__ __forceinline__ void add(Acc& a, int k, VV v, X x) {  // k: unrolled slot
    if (k & 1) a.a1 = fma(v, x, a.a1);
    else a.a0 = fma(v, x, a.a0);
  }
  // far sum of the row's lane group, valid in every lane of the group
  static __device__ __forceinline__ void gather(Acc& a, int V, int Vmax) {
    a.a0 = segmented_sum(a.a0 + a.a1, V, Vmax);
    a.a1 = TC(0);
  }
  static __device__ __forceinline__ void add_near(Acc& a, VV v, X x) { a.a0 = fma(v, x, a.a0); }
  static __device__ __forceinline__ X finish(const Acc& a, D d) { return -a.a0 * d; }
};

template <typename TS, typename TC>
struct SweepArith<TS, TC, true> {  // float-float (TS = float or BF16)
  using TSt = TS;
  using X = unsigned long long;
  using VV = float;
  using D = float;
  struct Acc {
    float s0, c0, s1, c1;
  };
  static __device__ __forceinline__ X sent() { return kFFSentinel; }
  static __device__ __forceinline__ bool is_sent(X x) { return x == kFFSentinel; }
  static __device__ __forceinline__ VV val(TS v) {
    if constexpr (std::is_same<TS, __nv_bfloat16>::value) return __bfloat162float(v);
    else return (float)v;
  }
  static __device__ __forceinline__ void init(Acc& a, X in) {
    a.s0 = -ff_hi(in);
    a.c0 = -ff_lo(in);
    a.s1 = a.c1 = 0.f;
  }
  static __device__ __forceinline__ void add(Acc& a, int k, VV v, X x) {
    if (k & 1) dot2_step(v, ff_hi(x), ff_lo(x), a.s1, a.c1);
    else dot2_step(v, ff_hi(x), ff_lo(x), a.s0, a.c0);
  }
  static __device__ __forceinline__ void gather(Acc& a, int V, int Vmax) {
    float h, l;
    two_sum(a.s0, a.s1, h, l);
    l = __fadd_rn(l, __fadd_rn(a.c0, a.c1));
    {
      const float hh = __fadd_rn(h, l);
      l = __fsub_rn(l, __fsub_rn(hh, h));
      h = hh;
    }
    for (int o = Vmax >> 1; o > 0; o >>= 1) {
      const float ph = __shfl_xor_sync(0xffffffffu, h, o);
      const float pl = __shfl_xor_sync(0xffffffffu, l, o);
      if (o < V) ff_add(h, l, ph, pl);
    }
    a.s0 = h;
    a.c0 = l;
    a.s1 = a.c1 = 0.f;
  }
  static __device__ __forceinline__ void add_near(Acc& a, VV v, X x) { dot2_step(v, ff_hi(x), ff_lo(x), a.s0, a.c0); }
  // y = -(s0 + c0) * d in float-float
  static __device__ __forceinline__ X finish(const Acc& a, D d) {
    float h, l;
    two_sum(a.s0, a.c0, h, l);  // |c0| can exceed |s0| after cancellation
    const float p = __fmul_rn(h, d);
    float pe = __fmaf_rn(h, d, -p);
    pe = __fmaf_rn(l, d, pe);
    const float yh = __fadd_rn(p, pe);
    const float yl = __fsub_rn(pe, __fsub_rn(yh, p));
    return ff_pack(-yh, -yl);
  }
};

// Per-level completion barriers (mbarrier objects in shared memory, one per
// level of the sweep, expecting one arrival per tile of that level).  A
// waiting warp parks in mbarrier.try_wait, which suspends it in hardware
// until the phase completes or a short time window passes, instead of
// spinning: waiting warps leave the issue slots to the warps that compute.
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// One arrival with release semantics: the arriving thread's earlier writes
// (and, through the warp's __syncwarp, its lanes' stores) are visible to a
// thread whose wait on the completed phase returns.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait until level `wl` is complete (every tile of it arrived: the
// barrier's first phase).  Gives up after `limit` try_waits or about a second
// (2^31 clocks), sets *timeout and returns.
__device__ __forceinline__ void wait_level(uint64_t* bars, int wl, int limit, int* timeout) {
  uint64_t* bar = bars + wl;
  if (mbar_try_wait(bar, 0u)) return;
  const long long deadline = clock64() + (1ll << 31);
  for (int spins = 1;; ++spins) {
    if (mbar_try_wait(bar, 0u)) return;
    if (spins > limit || clock64() > deadline) { *timeout = 1; return; }
  }
}

// Loads out[jj[k]] for KR slots (jj < 0: none) and polls, warp-uniformly and
// bounded, until no loaded value is the sentinel.  A value that is not the
// sentinel is final: it is written once per sweep.
template <typename AR, int KR>
__device__ __forceinline__ void load_ready(const int (&jj)[KR], typename AR::X (&xv)[KR],
                                           volatile typename AR::X* out, unsigned backoff, int limit, int* timeout) {
  using X = typename AR::X;
  bool ready = true;
#pragma unroll
  for (int k = 0; k < KR; ++k) {
    xv[k] = jj[k] >= 0 ? out[jj[k]] : X(0);
    if (AR::is_sent(xv[k])) ready = false;
  }
  int spins = 0;
  while (!__all_sync(0xffffffffu, ready)) {
    if (backoff) __nanosleep(backoff);
    ready = true;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      if (jj[k] >= 0 && AR::is_sent(xv[k])) xv[k] = out[jj[k]];
      if (AR::is_sent(xv[k])) ready = false;
    }
    if (++spins > limit) {
      *timeout = 1;
      ready = true;
#pragma unroll
      for (int k = 0; k < KR; ++k)
        if (AR::is_sent(xv[k])) xv[k] = X(0);
    }
  }
}

// One tile of a sweep: the rows of one level in one warp.  The lanes' far
// entries are summed (after wait_far, which may park the warp until the far
// levels are complete), added into each row's leader, then the leader adds
// its near entries, polling their values until final (after wait_near), and
// stores the row's value.  Returns the tile's level.
template <typename AR, int KREG, int KNEAR, typename WaitFar, typename WaitNear>
__device__ __forceinline__ int solve_tile(const unsigned char* base, int lane, volatile typename AR::X* in,
                                          volatile typename AR::X* out, bool unit, unsigned backoff, int limit,
                                          int* timeout, WaitFar wait_far, WaitNear wait_near) {
  using X = typename AR::X;
  using VV = typename AR::VV;
  using D = typename AR::D;
  using TS = typename AR::TSt;
  const int nr = reinterpret_cast<const int32_t*>(base)[0];
  const int ne = reinterpret_cast<const int32_t*>(base)[1];
  const int level = reinterpret_cast<const int32_t*>(base)[2];
  const uint2 rec = reinterpret_cast<const uint2*>(base + 16)[lane];  // this lane's role, one load
  const int row = (int)(rec.x & 0xFFFFu);
  const int first = (int)(rec.x >> 16);
  const int nfar = (int)(rec.y & 0xFFu);
  const int V = 1 << ((rec.y >> 8) & 0xFFu);
  const int r = (int)((rec.y >> 16) & 0x7Fu);
  const bool leader = ((rec.y >> 23) & 1u) != 0;
  const int nnear = (int)(rec.y >> 24);
  const int Vmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)V);
  const TS* dv = reinterpret_cast<const TS*>(base + 16 + 256);
  const uint16_t* cols = reinterpret_cast<const uint16_t*>(base + 16 + 256 + ((nr * (int)sizeof(TS) + 15) & ~15));
  const TS* vals = reinterpret_cast<const TS*>(reinterpret_cast<const unsigned char*>(cols) + ((2 * ne + 15) & ~15));
  // The right-hand side and the inverse diagonal are final before the
  // sweep starts: read them first, off the critical path.
  const X inr = leader ? in[row] : X(0);
  const D dvr = leader && !unit ? (D)AR::val(dv[r]) : D(1);
  typename AR::Acc acc;
  AR::init(acc, inr);
  // far entries of the lane, KREG per warp-uniform round
  const int rfar = __reduce_max_sync(0xffffffffu, (unsigned)((nfar + KREG - 1) / KREG));
  if (rfar > 0) wait_far(level);
  for (int c = 0; c < rfar; ++c) {
    int jj[KREG];
    VV vv[KREG];
    X xv[KREG];
#pragma unroll
    for (int k2 = 0; k2 < KREG; ++k2) {
      const int idx = c * KREG + k2;
      const bool ok = idx < nfar;
      const int e = first + idx * V;
      jj[k2] = ok ? (int)cols[e] : -1;
      vv[k2] = ok ? AR::val(vals[e]) : VV(0);
    }
    load_ready<AR, KREG>(jj, xv, out, backoff, limit, timeout);
#pragma unroll
    for (int k2 = 0; k2 < KREG; ++k2) AR::add(acc, k2, vv[k2], xv[k2]);
  }
  AR::gather(acc, V, Vmax);
  wait_near(level);
  // near entries (leader lanes), KNEAR per round
  const int near0 = first - nnear;
  const int rnear = __reduce_max_sync(0xffffffffu, (unsigned)((nnear + KNEAR - 1) / KNEAR));
  for (int c = 0; c < rnear; ++c) {
    int jj[KNEAR];
    VV vv[KNEAR];
    X xv[KNEAR];
#pragma unroll
    for (int k2 = 0; k2 < KNEAR; ++k2) {
      const int idx = c * KNEAR + k2;
      const bool ok = idx < nnear;
      jj[k2] = ok ? (int)cols[near0 + idx] : -1;
      vv[k2] = ok ? AR::val(vals[near0 + idx]) : VV(0);
    }
    load_ready<AR, KNEAR>(jj, xv, out, backoff, limit, timeout);
#pragma unroll
    for (int k2 = 0; k2 < KNEAR; ++k2)
      if (jj[k2] >= 0) AR::add_near(acc, vv[k2], xv[k2]);
  }
  if (leader) out[row] = AR::finish(acc, dvr);
  return level;
}

// One sweep of a block.  `in` holds the right-hand side, `out` the solution
// (sentinel until solved; an aligned store publishes value and readiness at
// once).  Only warps w < W take tiles.  A tile's rows are at one level L.
// Each lane first sums its "far" entries (columns at levels <= L - gap) --
// with per-level barriers (`done`) the warp first waits, suspended, until
// level L - gap is complete (a tile arrives only after its values are stored
// and its own level below is complete, so this means every level <= L - gap
// is solved) -- and the lanes' far sums are added into the row's leader.  Only then does the leader load its "near"
// entries (levels L - gap + 1 .. L - 1), polling the values themselves: one
// or two per row, the only arithmetic left between a value's store and the
// next level's.  The gap lets the barriers, whose completions trail the
// values, gate the far part without delaying it.  Readiness
// is always confirmed on the values, so a value is never used before it is
// final; the barriers spare the waiting warps the value polls.
template <typename TS, typename TC, bool FF, int SLOTS, int KREG, int KNEAR>
__device__ __forceinline__ void sweep_staged(const unsigned char* __restrict__ stream, const int64_t* toff_s,
                                             int ntile, unsigned char* ring, int slot_bytes,
                                             volatile typename SweepArith<TS, TC, FF>::X* in,
                                             volatile typename SweepArith<TS, TC, FF>::X* out, bool unit,
                                             int* timeout, int W, unsigned backoff, uint64_t* done, int limit,
                                             int pad, int gap) {
  using AR = SweepArith<TS, TC, FF>;
  const int lane = lane_id(), w = threadIdx.x >> 5;
  if (w >= W) return;
  const int nk = ntile > w ? (ntile - w + W - 1) / W : 0;  // tiles of this warp
  if (nk == 0) return;
  // Every lane copies 16-byte chunks of a tile; one commit group per tile
  // (empty groups keep the count uniform).  Tiles 0..SLOTS-2 are issued up
  // front and tile k+SLOTS-1 right after tile k is solved, so at tile k
  // wait_group<SLOTS-2> means "tile k has landed" for this lane; __syncwarp
  // then publishes all lanes' chunks to the warp.
  auto issue = [&](int k) {
    if (k < nk) {
      const int t = w + k * W;
      const int64_t a = toff_s[t];
      const int n16 = (int)((toff_s[t + 1] - a) >> 4);
      if (n16 * 16 <= slot_bytes) {
        unsigned char* dst = ring + (k % SLOTS) * slot_bytes;
        const unsigned char* src = stream + a;
        for (int c = lane; c < n16; c += 32) cp_async16(dst + 16 * c, src + 16 * c);
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int d = 0; d < SLOTS - 1; ++d) issue(d);
  // far part: park until level L - gap is complete; near part: under the
  // timeout-path test the tile first waits for level L - 1, whose barrier
  // then expects one arrival more than it gets
  auto wait_far = [&](int level) {
    if (done && level >= gap) wait_level(done, level - gap, limit, timeout);
  };
  auto wait_near = [&](int level) {
    if (pad && done && level >= 1) wait_level(done, level - 1, limit, timeout);
  };
  for (int k = 0; k < nk; ++k) {
    const int t = w + k * W;
    const int64_t a = toff_s[t];
    const int bytes = (int)(toff_s[t + 1] - a);
    cp_async_wait<SLOTS - 2>();
    __syncwarp();
    // A tile larger than a slot (one very long row) is read in place.  The
    // two calls keep the usual path's pointers in the shared window.
    const int level =
        bytes <= slot_bytes
            ? solve_tile<AR, KREG, KNEAR>(ring + (k % SLOTS) * slot_bytes, lane, in, out, unit, backoff, limit,
                                          timeout, wait_far, wait_near)
            : solve_tile<AR, KREG, KNEAR>(stream + a, lane, in, out, unit, backoff, limit, timeout, wait_far,
                                          wait_near);
    __syncwarp();  // the slot of tile k-1 is free: refill it with tile k+SLOTS-1
    if (done) {
      // The tile arrives on level L's barrier once its values are stored and
      // level L - 1 is complete, so a complete level L means every level
      // <= L is solved.  The next level's rows read this tile's values
      // directly, so neither wait nor arrival is on their path.
      if (level >= 1) wait_level(done, level - 1, limit, timeout);
      if (lane == 0) mbar_arrive(done + level);
    }
    issue(k + SLOTS - 1);
  }
  cp_async_wait<0>();
}

// Level-synchronous sweep of a block: the W sweeping warps step through the
// block's nlev levels together, one named barrier (bar.sync 1, W warps) per
// level, which also makes the level's stored values visible to all of them.
// Every entry of a level-L tile lies at a level below L and is final when
// the tile starts, so no wait sits inside a level and nothing spins: a level
// costs its slowest tile plus one barrier.  Tiles are staged as in
// sweep_staged; lend[l] (shared memory) ends level l's tiles, so a warp
// knows which of its tiles belong to a level without waiting for their
// bytes.  Each warp passes exactly nlev barriers.
template <typename TS, typename TC, bool FF, int SLOTS, int KREG, int KNEAR>
__device__ __forceinline__ void sweep_levels(const unsigned char* __restrict__ stream, const int64_t* toff_s,
                                             int ntile, const int32_t* lend, int nlev, unsigned char* ring,
                                             int slot_bytes,
                                             volatile typename SweepArith<TS, TC, FF>::X* in,
                                             volatile typename SweepArith<TS, TC, FF>::X* out, bool unit,
                                             int* timeout, int W, int limit) {
  using AR = SweepArith<TS, TC, FF>;
  const int lane = lane_id(), w = threadIdx.x >> 5;
  if (w >= W) return;
  const int nk = ntile > w ? (ntile - w + W - 1) / W : 0;  // tiles of this warp
  auto issue = [&](int k) {
    if (k < nk) {
      const int t = w + k * W;
      const int64_t a = toff_s[t];
      const int n16 = (int)((toff_s[t + 1] - a) >> 4);
      if (n16 * 16 <= slot_bytes) {
        unsigned char* dst = ring + (k % SLOTS) * slot_bytes;
        const unsigned char* src = stream + a;
        for (int c = lane; c < n16; c += 32) cp_async16(dst + 16 * c, src + 16 * c);
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int d = 0; d < SLOTS - 1; ++d) issue(d);
  auto none = [](int) {};
  int k = 0;
  for (int level = 0; level < nlev; ++level) {
    const int tend = lend[level];
    for (; k < nk && w + k * W < tend; ++k) {
      const int t = w + k * W;
      const int64_t a = toff_s[t];
      const int bytes = (int)(toff_s[t + 1] - a);
      cp_async_wait<SLOTS - 2>();
      __syncwarp();
      if (bytes <= slot_bytes)
        solve_tile<AR, KREG, KNEAR>(ring + (k % SLOTS) * slot_bytes, lane, in, out, unit, 0u, limit, timeout, none,
                                    none);
      else
        solve_tile<AR, KREG, KNEAR>(stream + a, lane, in, out, unit, 0u, limit, timeout, none, none);
      __syncwarp();
      issue(k + SLOTS - 1);
    }
    asm volatile("bar.sync 1, %0;" ::"r"(W * 32) : "memory");
  }
  cp_async_wait<0>();
}

// mode 0: x += alpha p, r -= alpha q, ||r||^2, z = M^{-1} r, r^T z, z^T q;
// mode 1: z = M^{-1} r only, then rho = r^T z and p = z (start or restart);
// mode 2: z = M^{-1} r only; mode 3: mode 2, skipped once the solve has stopped.
// Block b of one request (the whole CTA): the body of the single-request
// kernel below and of the batched one (batch.cu's persistent launches walk a
// table of (request, block) items through the same code).
template <typename TS, typename TC, int SLOTS, int KREG>
__device__ __forceinline__ void update_staged_body(const TriSolve& M, const double* __restrict__ p,
                                                   const double* __restrict__ q, double* __restrict__ x,
                                                   double* __restrict__ r, double* __restrict__ z,
                                                   double* __restrict__ pp, double* __restrict__ part,
                                                   PcgState* __restrict__ s, int mode, int b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double sh[32];
  __shared__ int timeout;
  const int64_t s0 = M.bp[b], e0 = M.bp[b + 1];
  constexpr bool FF = std::is_same<TC, ff_tag>::value;
  using TY = typename std::conditional<FF, unsigned long long, TC>::type;  // y storage in shared memory
  const size_t ybytes = align128((size_t)M.max_block * sizeof(TY));
  volatile TY* yb = reinterpret_cast<volatile TY*>(smem_raw);
  volatile TY* yf = reinterpret_cast<volatile TY*>(smem_raw + ybytes);
  TY S;
  if constexpr (FF) S = kFFSentinel;
  else S = sentinel(TC(0));
  const int w = threadIdx.x >> 5;
  const int W = blockDim.x >> 5;
  unsigned char* rings = smem_raw + 2 * ybytes;
  unsigned char* ring = rings + (size_t)w * SLOTS * M.slot_bytes;
  // this block's tile offsets of both directions, staged once
  int64_t* toff_f = reinterpret_cast<int64_t*>(rings + (size_t)W * SLOTS * M.slot_bytes);
  const int64_t tf0 = M.fwd_tile[b];
  const int ntf = (int)(M.fwd_tile[b + 1] - tf0);
  const int64_t tb0 = M.bwd_tile[b];
  const int ntb = (int)(M.bwd_tile[b + 1] - tb0);
  int64_t* toff_b = toff_f + ntf + 1;
  uint64_t* done = M.level_wait == 1 ? reinterpret_cast<uint64_t*>(toff_f + M.max_tiles + 2) : nullptr;
  const bool lsync = M.level_wait == 2;
  int32_t* lend = reinterpret_cast<int32_t*>(toff_f + M.max_tiles + 2);  // level-synchronous: tile ends per level
  const int lf0 = M.lev_off_lo[b], nlf = M.lev_off_lo[b + 1] - lf0;  // levels of this block, forward
  const int lb0 = M.lev_off_up[b], nlb = M.lev_off_up[b + 1] - lb0;  // and backward
  for (int t = threadIdx.x; t <= ntf; t += blockDim.x) toff_f[t] = M.fwd_toff[tf0 + t];
  for (int t = threadIdx.x; t <= ntb; t += blockDim.x) toff_b[t] = M.bwd_toff[tb0 + t];
  if (done)
    for (int t = threadIdx.x; t < nlf; t += blockDim.x)
      mbar_init(done + t, (unsigned)(M.fwd_ltiles[lf0 + t] + M.wait_pad));
  if (lsync)
    for (int t = threadIdx.x; t < nlf; t += blockDim.x) lend[t] = M.fwd_lend[lf0 + t];
  if (threadIdx.x == 0) timeout = 0;
  double rr = 0.0;
  if (mode == 0) {
    const double a = s->alpha;
    for (int64_t i = s0 + threadIdx.x; i < e0; i += blockDim.x) {
      const double ri = __fma_rn(-a, q[i], r[i]);
      x[i] = __fma_rn(a, p[i], x[i]);
      r[i] = ri;
      rr = __fma_rn(ri, ri, rr);
      if constexpr (FF) yb[i - s0] = ff_from_double(ri);
      else yb[i - s0] = (TC)ri;
      yf[i - s0] = S;
    }
  } else {
    for (int64_t i = s0 + threadIdx.x; i < e0; i += blockDim.x) {
      const double ri = r[i];
      rr = __fma_rn(ri, ri, rr);
      if constexpr (FF) yb[i - s0] = ff_from_double(ri);
      else yb[i - s0] = (TC)ri;
      yf[i - s0] = S;
    }
  }
  const double rrb = block_sum(rr, sh);
  __syncthreads();
  if (lsync)
    sweep_levels<TS, TC, FF, SLOTS, KREG, kNear>(M.fwd_stream, toff_f, ntf, lend, nlf, ring, M.slot_bytes, yb, yf,
                                                 M.unit_lower != 0, &timeout, M.sweep_warps, M.wait_limit);
  else
    sweep_staged<TS, TC, FF, SLOTS, KREG, kNear>(M.fwd_stream, toff_f, ntf, ring, M.slot_bytes, yb, yf,
                                                 M.unit_lower != 0, &timeout, M.sweep_warps, (unsigned)M.backoff_ns,
                                                 done, M.wait_limit, M.wait_pad, M.far_gap);
  __syncthreads();
  for (int64_t i = threadIdx.x; i < e0 - s0; i += blockDim.x) yb[i] = S;
  if (done) {
    for (int t = threadIdx.x; t < nlf; t += blockDim.x) mbar_inval(done + t);
    __syncthreads();
    for (int t = threadIdx.x; t < nlb; t += blockDim.x)
      mbar_init(done + t, (unsigned)(M.bwd_ltiles[lb0 + t] + M.wait_pad));
  }
  if (lsync)
    for (int t = threadIdx.x; t < nlb; t += blockDim.x) lend[t] = M.bwd_lend[lb0 + t];
  __syncthreads();
  if (lsync)
    sweep_levels<TS, TC, FF, SLOTS, KREG, kNear>(M.bwd_stream, toff_b, ntb, lend, nlb, ring, M.slot_bytes, yf, yb,
                                                 false, &timeout, M.sweep_warps, M.wait_limit);
  else
    sweep_staged<TS, TC, FF, SLOTS, KREG, kNear>(M.bwd_stream, toff_b, ntb, ring, M.slot_bytes, yf, yb, false,
                                                 &timeout, M.sweep_warps, (unsigned)M.backoff_ns, done, M.wait_limit,
                                                 M.wait_pad, M.far_gap);
  __syncthreads();
  double rz = 0.0, zq = 0.0;
  for (int64_t i = s0 + threadIdx.x; i < e0; i += blockDim.x) {
    double zi;
    if constexpr (FF) zi = ff_to_double(yb[i - s0]);
    else zi = (double)yb[i - s0];
    z[i] = zi;
    if (mode == 1) pp[i] = zi;
    rz = __fma_rn(r[i], zi, rz);
    if (mode == 0) zq = __fma_rn(zi, q[i], zq);
  }
  const double rzb = block_sum(rz, sh);
  const double zqb = block_sum(zq, sh);
  update_epilogue(M, rrb, rzb, zqb, part, s, mode, timeout != 0, b);
  if (done) {  // the shared memory may hold another block's barriers next
    __syncthreads();
    for (int t = threadIdx.x; t < nlb; t += blockDim.x) mbar_inval(done + t);
    __syncthreads();
  }
}

template <typename TS, typename TC, int SLOTS, int KREG>
__global__ void __launch_bounds__(kSweepWarps * 32) k_pcg_update_staged(TriSolve M, const double* __restrict__ p,
                                                                        const double* __restrict__ q,
                                                                        double* __restrict__ x, double* __restrict__ r,
                                                                        double* __restrict__ z, double* __restrict__ pp,
                                                                        double* __restrict__ part,
                                                                        PcgState* __restrict__ s, int mode) {
  if ((mode == 0 || mode == 3) && s->done) return;
  update_staged_body<TS, TC, SLOTS, KREG>(M, p, q, x, r, z, pp, part, s, mode, (int)blockIdx.x);
}

// One PCG update + apply over the blocks of several requests in one
// persistent launch: CTA c takes items c, c + gridDim.x, ... of the table;
// an item is (request, block).  Requests whose solve has stopped are skipped
// (the decision is read once per item and shared by the CTA).
template <typename TS, typename TC, int SLOTS, int KREG>
__global__ void __launch_bounds__(kSweepWarps * 32) k_batch_update_staged(const BatchReq* __restrict__ reqs,
                                                                          const BatchItem* __restrict__ items,
                                                                          int nitems) {
  __shared__ int skip;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BatchItem I = items[it];
    const BatchReq& R = reqs[I.req];
    __syncthreads();
    if (threadIdx.x == 0) skip = R.s->done;
    __syncthreads();
    if (skip) continue;
    update_staged_body<TS, TC, SLOTS, KREG>(R.M, R.p, R.q, R.x, R.r, R.z, nullptr, R.part_blk, R.s, 0, I.vb);
  }
}

template <typename TS, typename TC, int SLOTS, int KREG>
cudaError_t launch_staged(const TriSolve& M, const double* p, const double* q, double* x, double* r, double* z,
                          double* pp, double* part, PcgState* s, int mode, cudaStream_t st) {
  constexpr size_t kTY = std::is_same<TC, ff_tag>::value ? 8 : sizeof(TC);
  const size_t need = staged_smem_bytes(M.max_block, kTY, kSweepWarps, M.slot_bytes, M.slots, M.max_tiles,
                                        M.level_wait != 0 ? M.max_levels : 0);
  auto kern = k_pcg_update_staged<TS, TC, SLOTS, KREG>;
  SDSL_CUDA_TRY((allow_max_dynamic_smem<k_pcg_update_staged<TS, TC, SLOTS, KREG>>()));
  kern<<<(unsigned)M.nblocks, kSweepWarps * 32, need, st>>>(M, p, q, x, r, z, pp, part, s, mode); count_launch();
  return cudaGetLastError();
}

template <typename TS, typename TC>
cudaError_t launch_shape(const TriSolve& M, const double* p, const double* q, double* x, double* r, double* z,
                         double* pp, double* part, PcgState* s, int mode, cudaStream_t st) {
  const bool wide = M.kreg > 8;
  switch (M.slots) {
    case 2:
      return wide ? launch_staged<TS, TC, 2, 16>(M, p, q, x, r, z, pp, part, s, mode, st)
                  : launch_staged<TS, TC, 2, 8>(M, p, q, x, r, z, pp, part, s, mode, st);
    case 3:
      return wide ? launch_staged<TS, TC, 3, 16>(M, p, q, x, r, z, pp, part, s, mode, st)
                  : launch_staged<TS, TC, 3, 8>(M, p, q, x, r, z, pp, part, s, mode, st);
    default:
      return wide ? launch_staged<TS, TC, 4, 16>(M, p, q, x, r, z, pp, part, s, mode, st)
                  : launch_staged<TS, TC, 4, 8>(M, p, q, x, r, z, pp, part, s, mode, st);
  }
}

template <typename TS, typename TC, int SLOTS, int KREG>
cudaError_t launch_batch_staged(const BatchReq* reqs, const BatchItem* items, int nitems, int grid, size_t smem,
                                cudaStream_t st) {
  SDSL_CUDA_TRY((allow_max_dynamic_smem<k_batch_update_staged<TS, TC, SLOTS, KREG>>()));
  k_batch_update_staged<TS, TC, SLOTS, KREG><<<(unsigned)grid, kSweepWarps * 32, smem, st>>>(reqs, items, nitems);
  count_launch();
  return cudaGetLastError();
}

template <typename TS, typename TC>
cudaError_t batch_shape(const TriSolve& M, const BatchReq* reqs, const BatchItem* items, int nitems, int grid,
                        size_t smem, cudaStream_t st) {
  const bool wide = M.kreg > 8;
  switch (M.slots) {
    case 2:
      return wide ? launch_batch_staged<TS, TC, 2, 16>(reqs, items, nitems, grid, smem, st)
                  : launch_batch_staged<TS, TC, 2, 8>(reqs, items, nitems, grid, smem, st);
    case 3:
      return wide ? launch_batch_staged<TS, TC, 3, 16>(reqs, items, nitems, grid, smem, st)
                  : launch_batch_staged<TS, TC, 3, 8>(reqs, items, nitems, grid, smem, st);
    default:
      return wide ? launch_batch_staged<TS, TC, 4, 16>(reqs, items, nitems, grid, smem, st)
                  : launch_batch_staged<TS, TC, 4, 8>(reqs, items, nitems, grid, smem, st);
  }
}

}  // namespace

cudaError_t batch_update(const TriSolve& M0, const BatchReq* reqs, const BatchItem* items, int nitems, int grid,
                         size_t smem, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  if (M0.prec == 16) {
    if (M0.apply_prec == 32) return batch_shape<__nv_bfloat16, float>(M0, reqs, items, nitems, grid, smem, st);
    return batch_shape<__nv_bfloat16, ff_tag>(M0, reqs, items, nitems, grid, smem, st);
  }
  if (M0.prec == 64) return batch_shape<double, double>(M0, reqs, items, nitems, grid, smem, st);
  if (M0.apply_prec == 64) return batch_shape<float, double>(M0, reqs, items, nitems, grid, smem, st);
  if (M0.apply_prec == 48) return batch_shape<float, ff_tag>(M0, reqs, items, nitems, grid, smem, st);
  return batch_shape<float, float>(M0, reqs, items, nitems, grid, smem, st);
}

size_t staged_smem_bytes_of(const TriSolve& M) {
  const size_t tc = M.apply_prec == 32 ? 4 : 8;
  return staged_smem_bytes(M.max_block, tc, kSweepWarps, M.slot_bytes, M.slots, M.max_tiles,
                           M.level_wait != 0 ? M.max_levels : 0);
}

size_t staged_smem_bytes(int64_t max_block, size_t tc_size, int warps, int slot_bytes, int slots, int64_t max_tiles,
                         int64_t max_levels) {
  return 2 * align128((size_t)max_block * tc_size) + (size_t)warps * slots * (size_t)slot_bytes +
         (size_t)(max_tiles + 2) * sizeof(int64_t) + (size_t)max_levels * sizeof(uint64_t);
}

cudaError_t update_staged(const TriSolve& M, const double* p, const double* q, double* x, double* r, double* z,
                          double* pp, double* part, PcgState* s, int mode, cudaStream_t st) {
  if (M.prec == 16) {
    if (M.apply_prec == 32) return launch_shape<__nv_bfloat16, float>(M, p, q, x, r, z, pp, part, s, mode, st);
    return launch_shape<__nv_bfloat16, ff_tag>(M, p, q, x, r, z, pp, part, s, mode, st);
  }
  if (M.prec == 64) return launch_shape<double, double>(M, p, q, x, r, z, pp, part, s, mode, st);
  if (M.apply_prec == 64) return launch_shape<float, double>(M, p, q, x, r, z, pp, part, s, mode, st);
  if (M.apply_prec == 48) return launch_shape<float, ff_tag>(M, p, q, x, r, z, pp, part, s, mode, st);
  return launch_shape<float, float>(M, p, q, x, r, z, pp, part, s, mode, st);
}

}  // namespace sdsl
