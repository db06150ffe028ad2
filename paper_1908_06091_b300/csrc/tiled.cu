// tiled.cu -- shared-memory staged nabla kernels for sm_103a.
//
// A persistent grid walks the tiles of a TilePlan (consecutive Hilbert-
// ordered nodes whose own columns plus halo columns fit one stage).  A
// producer warp fills each stage with TMA copies completing on an mbarrier:
// one bulk copy (cp.async.bulk) of the tile's contiguous column block, bulk
// copies of the tile's CSR weights, staged offsets and row pointers, and the
// halo columns four at a time with tile::gather4 tensor copies (the copy
// engine's cost is per copy, so scattered halo columns are gathered in
// fours).  Two stages alternate, so tile k+1 is copied while tile k is
// computed.  Eleven or twelve consumer warps take (node, 4-level group)
// items, read the node's and its neighbours' columns from shared memory
// with 16-byte loads and accumulate with packed FP32x2 compensated sums;
// pole tiles (the first and last grid rows cut into at most one tile per
// CTA, walked first) run in FP64.  Every mbarrier wait is bounded:
// on timeout the kernel records NB_ETIMEOUT in a device status word, waits
// (bounded) for its own copies and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>

#include "kernels_common.cuh"

namespace nb {

// device status word: 0 = ok, otherwise an NB_* code (first error wins)
__device__ int g_device_status = 0;

int launch_tiled(nb_method *m, int op, const nb_field *in, const nb_field *out, const nb_field *out2,
                 cudaStream_t st, bool *handled, int comp = -1);

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// Fire-and-forget prefetch of a global range into L2 (16-byte aligned
// address, size a multiple of 16).
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// Four rows (y0..y3) of a 2-D tensor, one box row each, into consecutive
// shared memory at `dst` (128-byte aligned).
__device__ __forceinline__ void gather4_g2s(uint32_t dst, const CUtensorMap *map, int32_t y0, int32_t y1,
                                           int32_t y2, int32_t y3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(y0), "r"(y1), "r"(y2), "r"(y3), "r"(bar)
      : "memory");
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Non-blocking test of the phase (never suspends the thread).
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for `parity` on the barrier for at most ~`limit_ns`; false on timeout.
// A limit of 0 tests the phase once without suspending.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  if (limit_ns == 0) return mbar_test_wait(bar, parity);
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0 && globaltimer() - t0 > limit_ns) return false;
  }
}

// packed FP32x2 arithmetic (two lanes per register pair, IEEE round-to-nearest)
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t pk(float a, float b) {
  f2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk(f2_t r, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f2_t fma2(f2_t a, f2_t b, f2_t c) {
  f2_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2_t add2(f2_t a, f2_t b) {
  f2_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t sub2(f2_t a, f2_t b) {
  f2_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// Kahan accumulation of two independent sums at once.  nc holds the
// negated running correction.  One term w*d costs one fma2 and three
// add/sub2: y = w*d + nc; t = s + y; nc = y - (t - s); s = t.  A pair of
// edge terms is summed as one summand, y = w1*d1 + (w0*d0 + nc) by two
// fma2, then compensated into s: 2.5 operations per term.  (Each product is
// rounded once without compensation in either form; the compensation keeps
// the running sum's rounding out of the result.)
template <bool COMP>
struct Kahan2 {
  f2_t s = 0ull, nc = 0ull;
  __device__ __forceinline__ void add_prod(f2_t w, f2_t d) {
    if (COMP) {
      const f2_t y = fma2(w, d, nc);
      const f2_t t = add2(s, y);
      nc = sub2(y, sub2(t, s));
      s = t;
    } else {
      s = fma2(w, d, s);
    }
  }
  __device__ __forceinline__ void add_pair(f2_t w0, f2_t d0, f2_t w1, f2_t d1) {
    if (COMP) {
      const f2_t y = fma2(w1, d1, fma2(w0, d0, nc));
      const f2_t t = add2(s, y);
      nc = sub2(y, sub2(t, s));
      s = t;
    } else {
      s = fma2(w1, d1, fma2(w0, d0, s));
    }
  }
  // three edge terms as one summand (the six-neighbour path: two per node)
  __device__ __forceinline__ void add_triple(f2_t w0, f2_t d0, f2_t w1, f2_t d1, f2_t w2, f2_t d2) {
    if (COMP) {
      const f2_t y = fma2(w2, d2, fma2(w1, d1, fma2(w0, d0, nc)));
      const f2_t t = add2(s, y);
      nc = sub2(y, sub2(t, s));
      s = t;
    } else {
      s = fma2(w2, d2, fma2(w1, d1, fma2(w0, d0, s)));
    }
  }
  __device__ __forceinline__ f2_t value() const { return COMP ? add2(s, nc) : s; }
};

// ------------------------------------------------------------- kernel

struct TiledArgs {
  int ntiles, ntiles_main;
  const int32_t *tile_node0;
  const int32_t *halo_ptr;
  const int32_t *halo;
  const uint32_t *loff;
  const int32_t *row_ptr;
  const float2 *w32;
  const double2 *w64;
  const float2 *s32;
  const double2 *s64;
  const float4 *w4;     // fused div+curl: (du, dv, cu, cv) per CSR entry (else unused)
  const double2 *w64b;  // fused div+curl: FP64 curl weights and self weights (pole rows)
  const float4 *s4;     // fused div+curl: (su, sv, tu, tv) per node
  const double2 *s64b;
  float *out2;          // fused div+curl: the curl output (same strides as out)
  const char *in;
  uint32_t row_bytes;  // bytes of one own column (in_stride * 4)
  int64_t in_stride;   // elements
  float *out;
  int64_t out_stride;  // elements
  int nlev;
  int G;               // items per node (4 levels each)
  uint64_t g_magic;    // item / G == (item * g_magic) >> g_shift, exact for items < 2^24
  uint32_t g_shift;
  uint32_t copy_bytes; // bytes copied per column: the real data rounded up to 16
  uint32_t gpitch;     // shared-memory pitch of a group of four halo columns
  uint32_t off_w, off_l, off_r;  // stage offsets of the staged weights, offsets, row pointers
  uint32_t off_s;      // stage offset of the tile's self weights (div / curl; 0 = not staged)
  int rec16;           // fused div+curl: weights and self weights staged as 16-byte records
  uint32_t off_h;      // stage offset of the tile header: first and end node
  uint32_t stage_bytes;
  int nstages;
  int *status;
  uint64_t timeout_ns;  // limit of every pipeline wait (the method's wait limit)
};

// Limit of the producer's drain after a failed wait.  The copies it waits for
// were issued already and complete without any other warp, so this wait
// does not depend on the (possibly tiny) pipeline limit.
constexpr uint64_t kDrainLimitNs = 4000000000ull;
// Pipeline wait limit when the method sets none.
constexpr uint64_t kDefaultWaitNs = 2000000000ull;

// Issue the copies of tile t into the stage at `stage` (one whole warp).
__device__ __forceinline__ void issue_tile(const TiledArgs &a, const CUtensorMap *map, int t,
                                           uint32_t stage, uint32_t bar, int lane) {
  const int32_t n0 = __ldg(a.tile_node0 + t), n1 = __ldg(a.tile_node0 + t + 1);
  const int32_t h0 = __ldg(a.halo_ptr + t), h1 = __ldg(a.halo_ptr + t + 1);
  const int32_t pa = __ldg(a.row_ptr + n0), pb = __ldg(a.row_ptr + n1);
  const uint32_t n = (uint32_t)(n1 - n0), H = (uint32_t)(h1 - h0);
  // 8-byte weights are copied from an even entry; 16-byte records as they are
  const int32_t wa = a.rec16 ? pa : (pa & ~1), wb = a.rec16 ? pb : ((pb + 1) & ~1);
  const int32_t la = pa & ~3, lb = (pb + 3) & ~3;
  const int32_t ra = n0 & ~3, rb = (n1 + 4) & ~3;
  const uint32_t body = (n - 1) * a.row_bytes + a.copy_bytes;
  const uint32_t wbytes = (uint32_t)(wb - wa) * (a.rec16 ? 16u : 8u), lbytes = (uint32_t)(lb - la) * 4u,
                 rbytes = (uint32_t)(rb - ra) * 4u;
  const uint32_t groups = (H + 3u) >> 2;
  const uint32_t hbase = (n * a.row_bytes + 127u) & ~127u;
  const int32_t sa = a.rec16 ? n0 : (n0 & ~1), sb = a.rec16 ? n1 : ((n1 + 1) & ~1);
  const uint32_t sbytes = a.off_s ? (uint32_t)(sb - sa) * (a.rec16 ? 16u : 8u) : 0u;
  if (lane == 0) {
    // header for the consumers, published by the arrive below
    asm volatile("st.shared.v2.s32 [%0], {%1, %2};" ::"r"(stage + a.off_h), "r"(n0), "r"(n1) : "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (lane == 0)
    mbar_expect_tx(bar, body + wbytes + lbytes + rbytes + sbytes + groups * 4u * a.copy_bytes);
  __syncwarp();
  if (lane == 0) bulk_g2s(stage, a.in + (int64_t)n0 * a.in_stride * 4, body, bar);
  if (lane == 1) {
    if (a.rec16) bulk_g2s(stage + a.off_w, a.w4 + wa, wbytes, bar);
    else bulk_g2s(stage + a.off_w, a.w32 + wa, wbytes, bar);
  }
  if (lane == 2) bulk_g2s(stage + a.off_l, a.loff + la, lbytes, bar);
  if (lane == 3) bulk_g2s(stage + a.off_r, a.row_ptr + ra, rbytes, bar);
  if (lane == 4 && sbytes) {
    if (a.rec16) bulk_g2s(stage + a.off_s, a.s4 + sa, sbytes, bar);
    else bulk_g2s(stage + a.off_s, a.s32 + sa, sbytes, bar);
  }
  for (uint32_t g = lane; g < groups; g += 32) {
    // a short last group repeats its last node (the copy fills the group's slots)
    const int32_t *hp = a.halo + h0;
    const uint32_t k = 4u * g, last = H - 1u;
    gather4_g2s(stage + hbase + g * a.gpitch, map, __ldg(hp + k), __ldg(hp + min(k + 1u, last)),
                __ldg(hp + min(k + 2u, last)), __ldg(hp + min(k + 3u, last)), bar);
  }
}

// Shared-memory loads by 32-bit address (volatile: they must stay after the
// mbarrier wait that makes the staged data visible).
__device__ __forceinline__ float4 lds128(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a));
  return v;
}
__device__ __forceinline__ float2 lds64(uint32_t a) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
  return v;
}
// 16 bytes as two packed FP32x2 registers, 8 bytes as one (no repacking moves)
__device__ __forceinline__ void lds2x64(uint32_t a, unsigned long long &lo, unsigned long long &hi) {
  asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(lo), "=l"(hi) : "r"(a));
}
__device__ __forceinline__ unsigned long long lds_b64(uint32_t a) {
  unsigned long long v;
  asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ int32_t lds_s32(uint32_t a) {
  int32_t v;
  asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}

// 32-bit shared addresses of one staged tile: entry p's weight is at
// w + 8 p, its staged byte offset at l + 4 p, node i's row pointer at r + 4 i
// (wrap-around arithmetic; the sums land inside the stage).
struct TileView {
  int32_t n0, n1;
  uint32_t rows, w, l, r, s;
  __device__ __forceinline__ TileView(const TiledArgs &a, int t, uint32_t stage) {
    n0 = lds_s32(stage + a.off_h);
    n1 = lds_s32(stage + a.off_h + 4u);
    rows = stage;
    s = a.rec16 ? stage + a.off_s - 16u * (uint32_t)n0 : stage + a.off_s - 8u * (uint32_t)(n0 & ~1);
    const int32_t ra = n0 & ~3;
    r = stage + a.off_r - 4u * (uint32_t)ra;
    pa = lds_s32(r + 4u * (uint32_t)n0);
    w = a.rec16 ? stage + a.off_w - 16u * (uint32_t)pa : stage + a.off_w - 8u * (uint32_t)(pa & ~1);
    l = stage + a.off_l - 4u * (uint32_t)(pa & ~3);
  }
  int32_t pa;  // CSR index of the tile's first entry
};

// Consumer side.  A warp takes items [i0, i1) of tile t, one per lane,
// stride 32.  All but a handful of nodes of an octahedral mesh have six
// neighbours: for them the neighbour loop is fully unrolled, so every
// accumulator and address stays in fixed registers and no loop bookkeeping
// is issued; other degrees take a loop over neighbour pairs.  Staged data
// is loaded straight into packed FP32x2 registers.
//
// div / curl.  A staged (u, v) column is a sequence of 16-byte units of two
// levels each; item c of a node takes units c and c + G, so that every
// shared-memory load of a warp reads consecutive 16-byte words.  FUSED
// evaluates div and curl of the same wind in one pass: the staged columns,
// offsets and differences are shared, each operator keeps its own weights
// and accumulators, and each output gets exactly the arithmetic of its
// single-operator pass.
template <bool COMP, bool FUSED>
__device__ __forceinline__ void divcurl_tile(const TiledArgs &a, int t, uint32_t stage, int part,
                                             int nparts) {
  const TileView v(a, t, stage);
  const uint32_t items = (uint32_t)(v.n1 - v.n0) * a.G;
  const uint32_t i0 = (uint32_t)(((uint64_t)items * part) / nparts);
  const uint32_t i1 = (uint32_t)(((uint64_t)items * (part + 1)) / nparts);
  const bool pole = t >= a.ntiles_main;
  const int units = (a.nlev + 1) / 2;
  const uint32_t rb = a.row_bytes;
  const uint32_t g16 = 16u * (uint32_t)a.G;
  for (uint32_t item = i0 + (threadIdx.x & 31); item < i1; item += 32) {
    const uint32_t il = (uint32_t)(((uint64_t)item * a.g_magic) >> a.g_shift);
    const uint32_t c = item - il * a.G;
    const int u0 = (int)c, u1 = (int)c + a.G;
    const bool has1 = u1 < units;
    const int32_t node = v.n0 + (int32_t)il;
    const int32_t p0 = lds_s32(v.r + 4u * (uint32_t)node), p1 = lds_s32(v.r + 4u * (uint32_t)node + 4u);
    const uint32_t colA = v.rows + (uint32_t)u0 * 16u;
    const uint32_t colB = colA + (has1 ? g16 : 0u);
    float r[4], z[4];
    if (!pole) {
      f2_t i0p, i1p, i2p, i3p;
      lds2x64(colA + il * rb, i0p, i1p);
      lds2x64(colB + il * rb, i2p, i3p);
      Kahan2<COMP> k0, k1, k2, k3, q0, q1, q2, q3;
      // weights of entry e: single pass, 8-byte (w.x, w.y) at pw + 8 e; fused,
      // 16-byte (div, curl) records at pw + 16 e
      const uint32_t pw = v.w + (FUSED ? 16u : 8u) * (uint32_t)p0;
      auto weights = [&](uint32_t e, f2_t &wd, f2_t &wc) {
        if (FUSED) lds2x64(pw + 16u * e, wd, wc);
        else wd = lds_b64(pw + 8u * e);
      };
      const uint32_t pl = v.l + 4u * (uint32_t)p0;
      // differences of neighbour entry e: units (c, c + G) minus the node's own
      auto diffs = [&](uint32_t e, f2_t (&d)[4]) {
        const uint32_t off = lds_u32(pl + 4u * e);
        f2_t x0, x1, y0, y1;
        lds2x64(colA + off, x0, x1);
        lds2x64(colB + off, y0, y1);
        d[0] = sub2(x0, i0p);
        d[1] = sub2(x1, i1p);
        d[2] = sub2(y0, i2p);
        d[3] = sub2(y1, i3p);
      };
      auto triple = [&](uint32_t e) {
        f2_t d0[4], d1[4], d2[4];
        diffs(e, d0);
        diffs(e + 1u, d1);
        diffs(e + 2u, d2);
        f2_t w0, w1, w2, x0 = 0ull, x1 = 0ull, x2 = 0ull;
        weights(e, w0, x0);
        weights(e + 1u, w1, x1);
        weights(e + 2u, w2, x2);
        k0.add_triple(w0, d0[0], w1, d1[0], w2, d2[0]);
        k1.add_triple(w0, d0[1], w1, d1[1], w2, d2[1]);
        k2.add_triple(w0, d0[2], w1, d1[2], w2, d2[2]);
        k3.add_triple(w0, d0[3], w1, d1[3], w2, d2[3]);
        if (FUSED) {
          q0.add_triple(x0, d0[0], x1, d1[0], x2, d2[0]);
          q1.add_triple(x0, d0[1], x1, d1[1], x2, d2[1]);
          q2.add_triple(x0, d0[2], x1, d1[2], x2, d2[2]);
          q3.add_triple(x0, d0[3], x1, d1[3], x2, d2[3]);
        }
      };
      auto pair = [&](uint32_t e) {
        f2_t d0[4], d1[4];
        diffs(e, d0);
        diffs(e + 1u, d1);
        f2_t w0, w1, x0 = 0ull, x1 = 0ull;
        weights(e, w0, x0);
        weights(e + 1u, w1, x1);
        k0.add_pair(w0, d0[0], w1, d1[0]);
        k1.add_pair(w0, d0[1], w1, d1[1]);
        k2.add_pair(w0, d0[2], w1, d1[2]);
        k3.add_pair(w0, d0[3], w1, d1[3]);
        if (FUSED) {
          q0.add_pair(x0, d0[0], x1, d1[0]);
          q1.add_pair(x0, d0[1], x1, d1[1]);
          q2.add_pair(x0, d0[2], x1, d1[2]);
          q3.add_pair(x0, d0[3], x1, d1[3]);
        }
      };
      auto single = [&](uint32_t e) {
        f2_t d0[4];
        diffs(e, d0);
        f2_t w0, x0 = 0ull;
        weights(e, w0, x0);
        k0.add_prod(w0, d0[0]);
        k1.add_prod(w0, d0[1]);
        k2.add_prod(w0, d0[2]);
        k3.add_prod(w0, d0[3]);
        if (FUSED) {
          q0.add_prod(x0, d0[0]);
          q1.add_prod(x0, d0[1]);
          q2.add_prod(x0, d0[2]);
          q3.add_prod(x0, d0[3]);
        }
      };
      const int deg = p1 - p0;
      if (deg == 6) {
        triple(0);
        triple(3);
      } else {
        int e = 0;
        for (; e + 1 < deg; e += 2) pair((uint32_t)e);
        if (e < deg) single((uint32_t)e);
      }
      const f2_t self[4] = {i0p, i1p, i2p, i3p};
      f2_t sw_div, sw_curl = 0ull;
      if (FUSED) lds2x64(v.s + 16u * (uint32_t)node, sw_div, sw_curl);
      else sw_div = lds_b64(v.s + 8u * (uint32_t)node);
      {
        const f2_t sw = sw_div;
        const f2_t vals[4] = {k0.value(), k1.value(), k2.value(), k3.value()};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          float x, y;
          upk(fma2(sw, self[k], vals[k]), x, y);
          r[k] = __fadd_rn(x, y);
        }
      }
      if (FUSED) {
        const f2_t sw = sw_curl;
        const f2_t vals[4] = {q0.value(), q1.value(), q2.value(), q3.value()};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          float x, y;
          upk(fma2(sw, self[k], vals[k]), x, y);
          z[k] = __fadd_rn(x, y);
        }
      }
    } else {
      const float4 A = lds128(colA + il * rb);
      const float4 B = lds128(colB + il * rb);
      const float iu[4] = {A.x, A.z, B.x, B.z}, iv[4] = {A.y, A.w, B.y, B.w};
      double sacc[4] = {0, 0, 0, 0}, zacc[4] = {0, 0, 0, 0};
      for (int32_t p = p0; p < p1; ++p) {
        const double2 w = __ldg(a.w64 + p);
        const double2 x = FUSED ? __ldg(a.w64b + p) : w;
        const uint32_t r0 = lds_u32(v.l + 4u * (uint32_t)p);
        const float4 C = lds128(colA + r0);
        const float4 D = lds128(colB + r0);
        const float ju[4] = {C.x, C.z, D.x, D.z}, jv[4] = {C.y, C.w, D.y, D.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const double du = (double)ju[k] - (double)iu[k], dv = (double)jv[k] - (double)iv[k];
          sacc[k] = fma(w.y, dv, fma(w.x, du, sacc[k]));
          if (FUSED) zacc[k] = fma(x.y, dv, fma(x.x, du, zacc[k]));
        }
      }
      const double2 sw = __ldg(a.s64 + node);
      const double2 sx = FUSED ? __ldg(a.s64b + node) : sw;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        r[k] = (float)fma(sw.y, (double)iv[k], fma(sw.x, (double)iu[k], sacc[k]));
        if (FUSED) z[k] = (float)fma(sx.y, (double)iv[k], fma(sx.x, (double)iu[k], zacc[k]));
      }
    }
    // levels 2 u0, 2 u0 + 1 from r[0..1], levels 2 u1, 2 u1 + 1 from r[2..3]
    auto put = [&](float *oo, const float (&o)[4]) {
      const int la0 = 2 * u0, la1 = 2 * u1;
      if (la0 + 1 < a.nlev) __stcs(reinterpret_cast<float2 *>(oo + la0), make_float2(o[0], o[1]));
      else oo[la0] = o[0];
      if (has1) {
        if (la1 + 1 < a.nlev) __stcs(reinterpret_cast<float2 *>(oo + la1), make_float2(o[2], o[3]));
        else oo[la1] = o[2];
      }
    };
    put(a.out + (int64_t)node * a.out_stride, r);
    if (FUSED) put(a.out2 + (int64_t)node * a.out_stride, z);
  }
}

// grad.  Item c of a node takes the 4-level unit c of its scalar column;
// each weight is broadcast to both lanes of a packed register.
template <bool COMP>
__device__ __forceinline__ void grad_tile(const TiledArgs &a, int t, uint32_t stage, int part,
                                          int nparts) {
  const TileView v(a, t, stage);
  const uint32_t items = (uint32_t)(v.n1 - v.n0) * a.G;
  const uint32_t i0 = (uint32_t)(((uint64_t)items * part) / nparts);
  const uint32_t i1 = (uint32_t)(((uint64_t)items * (part + 1)) / nparts);
  const bool pole = t >= a.ntiles_main;
  const uint32_t rb = a.row_bytes;
  for (uint32_t item = i0 + (threadIdx.x & 31); item < i1; item += 32) {
    const uint32_t il = (uint32_t)(((uint64_t)item * a.g_magic) >> a.g_shift);
    const uint32_t c = item - il * a.G;
    const int l0 = 4 * (int)c;
    const int32_t node = v.n0 + (int32_t)il;
    const int32_t p0 = lds_s32(v.r + 4u * (uint32_t)node), p1 = lds_s32(v.r + 4u * (uint32_t)node + 4u);
    const uint32_t col = v.rows + c * 16u;
    float gx[4], gy[4];
    if (!pole) {
      f2_t fi01, fi23;
      lds2x64(col + il * rb, fi01, fi23);
      Kahan2<COMP> ax01, ax23, ay01, ay23;
      const uint32_t pw = v.w + 8u * (uint32_t)p0, pl = v.l + 4u * (uint32_t)p0;
      auto pair = [&](uint32_t q) {
        const float2 w0 = lds64(pw + 8u * q), w1 = lds64(pw + 8u * q + 8u);
        const uint32_t r0 = lds_u32(pl + 4u * q), r1 = lds_u32(pl + 4u * q + 4u);
        f2_t f001, f023, f101, f123;
        lds2x64(col + r0, f001, f023);
        lds2x64(col + r1, f101, f123);
        const f2_t a01 = sub2(f001, fi01), a23 = sub2(f023, fi23);
        const f2_t b01 = sub2(f101, fi01), b23 = sub2(f123, fi23);
        const f2_t wx0 = pk(w0.x, w0.x), wy0 = pk(w0.y, w0.y);
        const f2_t wx1 = pk(w1.x, w1.x), wy1 = pk(w1.y, w1.y);
        ax01.add_pair(wx0, a01, wx1, b01);
        ax23.add_pair(wx0, a23, wx1, b23);
        ay01.add_pair(wy0, a01, wy1, b01);
        ay23.add_pair(wy0, a23, wy1, b23);
      };
      auto triple = [&](uint32_t q) {
        const float2 w0 = lds64(pw + 8u * q), w1 = lds64(pw + 8u * q + 8u), w2 = lds64(pw + 8u * q + 16u);
        const uint32_t r0 = lds_u32(pl + 4u * q), r1 = lds_u32(pl + 4u * q + 4u), r2 = lds_u32(pl + 4u * q + 8u);
        f2_t f001, f023, f101, f123, f201, f223;
        lds2x64(col + r0, f001, f023);
        lds2x64(col + r1, f101, f123);
        lds2x64(col + r2, f201, f223);
        const f2_t a01 = sub2(f001, fi01), a23 = sub2(f023, fi23);
        const f2_t b01 = sub2(f101, fi01), b23 = sub2(f123, fi23);
        const f2_t e01 = sub2(f201, fi01), e23 = sub2(f223, fi23);
        const f2_t wx0 = pk(w0.x, w0.x), wy0 = pk(w0.y, w0.y);
        const f2_t wx1 = pk(w1.x, w1.x), wy1 = pk(w1.y, w1.y);
        const f2_t wx2 = pk(w2.x, w2.x), wy2 = pk(w2.y, w2.y);
        ax01.add_triple(wx0, a01, wx1, b01, wx2, e01);
        ax23.add_triple(wx0, a23, wx1, b23, wx2, e23);
        ay01.add_triple(wy0, a01, wy1, b01, wy2, e01);
        ay23.add_triple(wy0, a23, wy1, b23, wy2, e23);
      };
      auto single = [&](uint32_t q) {
        const float2 w = lds64(pw + 8u * q);
        f2_t f001, f023;
        lds2x64(col + lds_u32(pl + 4u * q), f001, f023);
        const f2_t d01 = sub2(f001, fi01), d23 = sub2(f023, fi23);
        const f2_t wx = pk(w.x, w.x), wy = pk(w.y, w.y);
        ax01.add_prod(wx, d01);
        ax23.add_prod(wx, d23);
        ay01.add_prod(wy, d01);
        ay23.add_prod(wy, d23);
      };
      const int deg = p1 - p0;
      if (deg == 6) {
        triple(0);
        triple(3);
      } else {
        int q = 0;
        for (; q + 1 < deg; q += 2) pair((uint32_t)q);
        if (q < deg) single((uint32_t)q);
      }
      upk(ax01.value(), gx[0], gx[1]);
      upk(ax23.value(), gx[2], gx[3]);
      upk(ay01.value(), gy[0], gy[1]);
      upk(ay23.value(), gy[2], gy[3]);
    } else {
      const float4 fi = lds128(col + il * rb);
      double sx[4] = {0, 0, 0, 0}, sy[4] = {0, 0, 0, 0};
      const float fiv[4] = {fi.x, fi.y, fi.z, fi.w};
      for (int32_t p = p0; p < p1; ++p) {
        const double2 w = __ldg(a.w64 + p);
        const float4 fj = lds128(col + lds_u32(v.l + 4u * (uint32_t)p));
        const float fjv[4] = {fj.x, fj.y, fj.z, fj.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const double d = (double)fjv[k] - (double)fiv[k];
          sx[k] = fma(w.x, d, sx[k]);
          sy[k] = fma(w.y, d, sy[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        gx[k] = (float)sx[k];
        gy[k] = (float)sy[k];
      }
    }
    float *go = a.out + (int64_t)node * a.out_stride + 2 * l0;
    if (l0 + 4 <= a.nlev) {
      __stcs(reinterpret_cast<float4 *>(go), make_float4(gx[0], gy[0], gx[1], gy[1]));
      __stcs(reinterpret_cast<float4 *>(go) + 1, make_float4(gx[2], gy[2], gx[3], gy[3]));
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (l0 + k < a.nlev) {
          go[2 * k] = gx[k];
          go[2 * k + 1] = gy[k];
        }
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Consumer warps per operator.  Fewer warps than the SM could hold: timed on
// B300 at O1280 x 137 levels, 11-12 consumer warps beat 16 by 1-7 % (more
// warps only queue more shared-memory requests behind the same pipeline),
// and a block of at most 4 warps per scheduler leaves up to 128 registers a
// thread.
// The producer also prefetches into L2 the column block of the tile
// `ahead` steps further along the CTA's walk, so that its stage copy reads
// L2 instead of HBM (timed: 1-3 % per launch; 1 step for the single
// operators, 2 for the fused pass).
template <int OP>
struct StagedShape {
  static constexpr int warps = OP == 0 ? 12 : 11;
  static constexpr int threads = 32 * (warps + 1);
  static constexpr int ahead = OP == 2 ? 2 : 1;
};

// Tile of the i-th position in the walk: the pole tiles first (FP64 and
// slow, at most one per CTA), so that they overlap the main tiles on other
// CTAs instead of running alone at the end of the launch.
__device__ __forceinline__ int tile_at(const TiledArgs &a, int i) {
  const int npole = a.ntiles - a.ntiles_main;
  return i < npole ? a.ntiles_main + i : i - npole;
}

// Warp-specialised pipeline.  The last warp (warp W) is the producer: for
// iteration k it waits until stage k % NS has been released by every
// consumer warp ("empty" barrier), then issues the copies of the k-th tile
// of this CTA's walk into it ("full" barrier, transaction count).  Each of
// the W consumer warps waits for "full", computes its 1/W share of the
// tile's items and releases the stage; no block-wide barrier is used.
template <int OP, bool COMP>
__global__ void __launch_bounds__(StagedShape<OP>::threads, 1)
    staged_f32(const TiledArgs a, const __grid_constant__ CUtensorMap map) {
  constexpr int W = StagedShape<OP>::warps;
  extern __shared__ __align__(128) unsigned char smem[];
  const int NS = a.nstages;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)NS * a.stage_bytes);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8u * NS;
  const uint32_t stage0 = smem_u32(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, W);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int G = gridDim.x;
  if (warp == W) {
    // producer
    int k = 0;
    bool failed = false;
    for (int i = blockIdx.x; i < a.ntiles; i += G, ++k) {
      const int t = tile_at(a, i);
      const int s = k % NS;
      if (k >= NS && !mbar_wait_bounded(empty0 + 8 * s, (uint32_t)(k / NS - 1) & 1u, a.timeout_ns)) {
        failed = true;
        break;
      }
      issue_tile(a, &map, t, stage0 + s * a.stage_bytes, full0 + 8 * s, lane);
      // L2 prefetch of the column block of a later tile of this walk
      constexpr int D = StagedShape<OP>::ahead;
      if (lane == 0 && i + D * G < a.ntiles) {
        const int tp = tile_at(a, i + D * G);
        const int32_t p0 = __ldg(a.tile_node0 + tp), p1 = __ldg(a.tile_node0 + tp + 1);
        bulk_prefetch_l2(a.in + (int64_t)p0 * a.in_stride * 4, (uint32_t)(p1 - p0 - 1) * a.row_bytes + a.copy_bytes);
      }
    }
    if (failed) {
      if (lane == 0) atomicCAS(a.status, 0, (int)NB_ETIMEOUT);
      // copies already issued (iterations k-NS .. k-1) land before exit (bounded)
      for (int j = (k >= NS ? k - NS : 0); j < k; ++j)
        if (!mbar_wait_bounded(full0 + 8 * (j % NS), (uint32_t)(j / NS) & 1u, kDrainLimitNs)) break;
    }
    return;
  }
  // consumers
  int k = 0;
  for (int i = blockIdx.x; i < a.ntiles; i += G, ++k) {
    const int t = tile_at(a, i);
    const int s = k % NS;
    if (!mbar_wait_bounded(full0 + 8 * s, (uint32_t)(k / NS) & 1u, a.timeout_ns)) {
      if (lane == 0) atomicCAS(a.status, 0, (int)NB_ETIMEOUT);
      break;
    }
    const uint32_t rows = stage0 + (uint32_t)s * a.stage_bytes;
    if (OP == 0) grad_tile<COMP>(a, t, rows, warp, W);
    else if (OP == 1) divcurl_tile<COMP, false>(a, t, rows, warp, W);
    else divcurl_tile<COMP, true>(a, t, rows, warp, W);
    __syncwarp();
    if (lane == 0) mbar_arrive(empty0 + 8 * s);
  }
}

// --------------------------------------------------------------- host

static int plan_upload(TilePlan *tp, nb_method *m) {
  const nb_mesh *mesh = m->mesh;
  std::vector<int32_t> node0, hptr, halo;
  std::vector<uint32_t> loff;
  build_tile_plan_bytes(mesh, tp->area, tp->row_bytes, tp->copy_bytes, tp->nmax, tp->ecap, tp->pole_cap, node0, hptr,
                        halo, loff, tp->max_halo, tp->max_entries, tp->ntiles_main);
  loff.resize(loff.size() + 8, 0);  // slack for 16-byte bounding copies
  if (halo.empty()) halo.push_back(0);
  tp->ntiles = (int)node0.size() - 1;
  auto up = [&](void **dst, const void *src, size_t bytes) -> int {
    const size_t nb = std::max<size_t>(bytes, 16);
    const int st = dev_alloc(m->alloc, dst, nb, "tile plan upload");
    if (st != NB_OK) return st;
    m->blocks.push_back({*dst, nb});
    if (bytes) NB_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    tp->bytes += (int64_t)bytes;
    return NB_OK;
  };
  int st;
  if ((st = up((void **)&tp->d_tile_node0, node0.data(), node0.size() * 4))) return st;
  if ((st = up((void **)&tp->d_halo_ptr, hptr.data(), hptr.size() * 4))) return st;
  if ((st = up((void **)&tp->d_halo, halo.data(), halo.size() * 4))) return st;
  if ((st = up((void **)&tp->d_loff, loff.data(), loff.size() * 4))) return st;
  return NB_OK;
}

// Pole-row tiles: the pole rows take the FP64 path, far slower per node on
// B300 than the FP32 one.  They are cut into at most one tile per CTA of the
// persistent grid (one node each for the 20-point rows of O<N>; ~70 for the
// 5,120-point rows of F1280), and the walk takes them first.
static TilePlan *get_plan(nb_method *m, int64_t area, int64_t row_bytes, int64_t copy_bytes, int nmax,
                          int ecap, int nctas, int *status) {
  const int64_t npole = m->mesh->V - m->mesh->cap_begin;
  const int pole_cap = (int)std::max<int64_t>(1, (npole + nctas - 1) / std::max(1, nctas));
  std::lock_guard<std::mutex> lk(m->plan_mu);
  auto key = std::make_tuple(area, row_bytes, copy_bytes, nmax, ecap, pole_cap);
  auto it = m->plans.find(key);
  if (it != m->plans.end()) return it->second.get();
  auto tp = std::make_unique<TilePlan>();
  tp->area = area;
  tp->row_bytes = row_bytes;
  tp->copy_bytes = copy_bytes;
  tp->nmax = nmax;
  tp->ecap = ecap;
  tp->pole_cap = pole_cap;
  *status = plan_upload(tp.get(), m);
  if (*status != NB_OK) return nullptr;
  TilePlan *raw = tp.get();
  m->plans[key] = std::move(tp);
  return raw;
}

// cuTensorMapEncodeTiled from the driver, looked up once.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// Division by a run-time constant d: x / d == (x * m) >> k with k = 32 + s,
// s = ceil(log2 d), m = ceil(2^k / d).  The error of x * m / 2^k against
// x / d is below x / 2^k <= 1 / d for x < 2^32, so the floor is exact; for
// x < 2^24 (at most 1024 nodes x 16384 groups per tile) and m < 2^33 the
// product fits in 64 bits.
static void magic_div(uint32_t d, uint64_t &magic, uint32_t &shift) {
  uint32_t s = 0;
  while ((1u << s) < d) ++s;
  shift = 32 + s;
  magic = ((1ull << shift) + d - 1) / d;
}

template <int OP, bool COMP>
static int launch_staged_t(const TiledArgs &a, const CUtensorMap &map, int grid, size_t smem,
                           cudaStream_t st) {
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [&] {
    attr_err = cudaFuncSetAttribute(staged_f32<OP, COMP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    227 * 1024);
  });
  NB_CUDA(attr_err);
  staged_f32<OP, COMP><<<grid, StagedShape<OP>::threads, smem, st>>>(a, map);
  count_launch(1);
  NB_CUDA(cudaGetLastError());
  return NB_OK;
}

static int g_sm_count = 0;

// Device address of the status word on the current device (looked up once
// per device).
static int status_word(int **out) {
  static std::mutex mu;
  static int *addr[64] = {};
  int dev = 0;
  NB_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 0 || dev >= 64) return NB_EINVAL;
  if (!addr[dev]) {
    void *p = nullptr;
    NB_CUDA(cudaGetSymbolAddress(&p, g_device_status));
    addr[dev] = static_cast<int *>(p);
  }
  *out = addr[dev];
  return NB_OK;
}

// out2 != nullptr (op == NB_OP_DIV): fused pass writing div to out and curl
// to out2.  comp: compensated accumulation (1), plain (0), or the method's
// setting (-1).
int launch_tiled(nb_method *m, int op, const nb_field *in, const nb_field *out, const nb_field *out2,
                 cudaStream_t st, bool *handled, int comp_mode) {
  *handled = false;
  if (in->dtype != NB_F32) return NB_OK;
  const bool fused = out2 != nullptr;
  if (fused && (op != NB_OP_DIV || out2->node_stride != out->node_stride || out2->dtype != NB_F32))
    return NB_OK;
  const uintptr_t addr_bits = (uintptr_t)in->data | (uintptr_t)out->data | (fused ? (uintptr_t)out2->data : 0u);
  const bool aligned = (addr_bits & 15u) == 0 && in->node_stride % 4 == 0 && out->node_stride % 4 == 0;
  // short columns leave most staged items idle: the direct kernels do better
  if (!aligned || in->nlev < 16) return NB_OK;
  const uint32_t row_bytes = (uint32_t)(in->node_stride * 4);
  const int G = (in->nlev + 3) / 4;
  const int nvar = in->nvar;
  // each 4-level group must lie inside the staged column
  if ((uint64_t)G * 16u * nvar > row_bytes) return NB_OK;
  const uint32_t copy_bytes = (uint32_t)(((int64_t)in->nlev * nvar * 4 + 15) / 16 * 16);
  // halo columns are gathered as tensor rows of 4-byte (scalar) or 8-byte
  // (vector) elements; a box row holds at most 256 elements
  const uint32_t esz = nvar == 2 ? 8u : 4u;
  if (copy_bytes / esz > 256u || encode_fn() == nullptr) return NB_OK;
  // nstages stages of stage_kb KB, one CTA per SM.  A stage holds the staged
  // columns, then the tile's weights, offsets and row pointers (bounding
  // ranges, 16-byte aligned).
  const int nstages = m->nstages > 0 ? m->nstages : 2;
  const int stage_kb = m->stage_kb > 0 ? m->stage_kb : 112;
  // Metadata reservation: a tile holds at most area / row_bytes own nodes;
  // the plan caps its CSR entries at 7 per such node (tiles are cut earlier
  // otherwise), so the reservation follows the columns that fit.
  auto up16 = [](uint32_t x) { return (x + 15u) & ~15u; };
  const uint32_t stage_target = (uint32_t)stage_kb * 1024u;
  const int nmax_req = m->tile_nodes > 0 ? m->tile_nodes : 256;
  const int fit_nodes = (int)(stage_target / row_bytes) + 1;
  const int nmax = std::max(1, std::min(nmax_req, fit_nodes));
  const int ecap = 7 * nmax + 16;
  const uint32_t rec = fused ? 16u : 8u;  // bytes per weight record and per self-weight record
  const uint32_t wsz = up16((uint32_t)(ecap + 2) * rec), lsz = up16((uint32_t)(ecap + 8) * 4u),
                 rsz = up16((uint32_t)(nmax + 8) * 4u);
  const uint32_t ssz = op == NB_OP_GRAD ? 0u : up16((uint32_t)(nmax + 2) * rec), hsz = 16u;
  const uint32_t meta = wsz + lsz + rsz + ssz + hsz;
  if (stage_target <= meta + 4096u) return NB_OK;
  const uint32_t area = ((stage_target - meta) / 128u) * 128u;
  if (area < 24u * row_bytes) return NB_OK;  // columns too tall to stage a useful tile
  if (g_sm_count == 0) {
    int dev = 0;
    NB_CUDA(cudaGetDevice(&dev));
    NB_CUDA(cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev));
  }
  int status = NB_OK;
  TilePlan *tp = get_plan(m, area, row_bytes, copy_bytes, nmax, ecap, g_sm_count, &status);
  if (!tp) return status;
  // tensor map over the input columns: rows = nodes (pitch row_bytes), the
  // first copy_bytes of each row
  CUtensorMap map;
  const cuuint64_t gdim[2] = {copy_bytes / esz, (cuuint64_t)in->nnodes};
  const cuuint64_t gstride[1] = {row_bytes};
  const cuuint32_t box[2] = {copy_bytes / esz, 1};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult cr = encode_fn()(&map, esz == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                  2, const_cast<void *>(in->data), gdim, gstride, box, estr,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) {
    set_error("staged kernel: cuTensorMapEncodeTiled failed (" + std::to_string((int)cr) + ")");
    return NB_ECUDA;
  }
  TiledArgs a;
  a.ntiles = tp->ntiles;
  a.ntiles_main = tp->ntiles_main;
  a.tile_node0 = tp->d_tile_node0;
  a.halo_ptr = tp->d_halo_ptr;
  a.halo = tp->d_halo;
  a.loff = tp->d_loff;
  a.row_ptr = m->d_row_ptr;
  const bool g = op == NB_OP_GRAD;
  a.w32 = reinterpret_cast<const float2 *>(g ? m->d_wgrad32 : op == NB_OP_DIV ? m->d_wdiv32 : m->d_wcurl32);
  a.w64 = reinterpret_cast<const double2 *>(g ? m->d_wgrad64 : op == NB_OP_DIV ? m->d_wdiv64 : m->d_wcurl64);
  a.s32 = reinterpret_cast<const float2 *>(op == NB_OP_CURL ? m->d_scurl32 : m->d_sdiv32);
  a.s64 = reinterpret_cast<const double2 *>(op == NB_OP_CURL ? m->d_scurl64 : m->d_sdiv64);
  a.w4 = fused ? reinterpret_cast<const float4 *>(m->d_wdc32) : nullptr;
  a.w64b = fused ? reinterpret_cast<const double2 *>(m->d_wcurl64) : nullptr;
  a.s4 = fused ? reinterpret_cast<const float4 *>(m->d_sdc32) : nullptr;
  a.s64b = fused ? reinterpret_cast<const double2 *>(m->d_scurl64) : nullptr;
  a.rec16 = fused ? 1 : 0;
  a.out2 = fused ? static_cast<float *>(out2->data) : nullptr;
  a.in = static_cast<const char *>(in->data);
  a.row_bytes = row_bytes;
  a.in_stride = in->node_stride;
  a.out = static_cast<float *>(out->data);
  a.out_stride = out->node_stride;
  a.nlev = in->nlev;
  a.G = G;
  magic_div((uint32_t)a.G, a.g_magic, a.g_shift);
  a.copy_bytes = copy_bytes;
  a.gpitch = (4u * copy_bytes + 127u) & ~127u;
  a.off_w = area;
  a.off_l = a.off_w + wsz;
  a.off_r = a.off_l + lsz;
  a.off_s = ssz ? a.off_r + rsz : 0u;
  a.off_h = a.off_r + rsz + ssz;
  a.stage_bytes = (a.off_h + hsz + 127u) & ~127u;
  a.nstages = nstages;
  a.status = nullptr;
  if (const int rc = status_word(&a.status)) return rc;
  a.timeout_ns = m->wait_limit_ns >= 0 ? (uint64_t)m->wait_limit_ns : kDefaultWaitNs;
  const size_t smem = (size_t)nstages * a.stage_bytes + 16 * (size_t)nstages;
  if (smem > 227 * 1024) {
    set_error("staged kernel: nstages * stage size exceeds 227 KB of shared memory");
    return NB_EINVAL;
  }
  const int grid = std::min(tp->ntiles, g_sm_count);
  *handled = true;
  const bool comp = comp_mode < 0 ? m->compensated != 0 : comp_mode != 0;
  if (g) return comp ? launch_staged_t<0, true>(a, map, grid, smem, st) : launch_staged_t<0, false>(a, map, grid, smem, st);
  if (fused)
    return comp ? launch_staged_t<2, true>(a, map, grid, smem, st) : launch_staged_t<2, false>(a, map, grid, smem, st);
  return comp ? launch_staged_t<1, true>(a, map, grid, smem, st) : launch_staged_t<1, false>(a, map, grid, smem, st);
}

int device_status(int clear, int *code) {
  NB_CUDA(cudaMemcpyFromSymbol(code, g_device_status, sizeof(int)));
  if (clear) {
    const int zero = 0;
    NB_CUDA(cudaMemcpyToSymbol(g_device_status, &zero, sizeof(int)));
  }
  return NB_OK;
}

}  // namespace nb
