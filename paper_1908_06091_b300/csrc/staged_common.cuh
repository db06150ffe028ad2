// staged_common.cuh -- device helpers of the shared-memory staged kernels
// (tiled.cu, fusedlap.cu): PTX wrappers for mbarriers, bulk and tensor
// copies and shared-memory loads, packed FP32x2 arithmetic, the compensated
// grouped sum, and the bounded waits with their limits.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "kernels_common.cuh"

namespace nb {

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

// Packed FP32x2 arithmetic: two independent FP32 lanes per value, each
// operation IEEE round-to-nearest (the CUDA float2 intrinsics of sm_100 and
// later; a difference is the sum with the negated operand, which is exact).
typedef float2 f2_t;
__device__ __forceinline__ f2_t pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ void upk(f2_t r, float &a, float &b) {
  a = r.x;
  b = r.y;
}
__device__ __forceinline__ f2_t fma2(f2_t a, f2_t b, f2_t c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2_t add2(f2_t a, f2_t b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2_t sub2(f2_t a, f2_t b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ f2_t mul2(f2_t a, f2_t b) { return __fmul2_rn(a, b); }

// Compensated per-node sum of edge terms, two independent lanes at once (a
// packed FP32x2 register).  In the difference form every term w (x_j - x_i)
// is of the size of the result, so terms are summed in groups by FMA chains
// (three per group for a six-neighbour node, two otherwise); each group sum
// y joins the node's sum s by a Fast2Sum step, t = s + y, whose rounding
// error y - (t - s) collects in e, and e is added last: after the self term
// of div and curl, where the flux form's cancellation happens, so that the
// correction survives it.  The first group initialises s (adding it to an
// empty sum is exact, so it costs no compensation).  COMP = false sums the
// same groups without the correction.
template <bool COMP>
struct GroupSum {
  f2_t s, y, e;
  __device__ __forceinline__ void start(f2_t w, f2_t d) { y = mul2(w, d); }
  __device__ __forceinline__ void term(f2_t w, f2_t d) { y = fma2(w, d, y); }
  __device__ __forceinline__ void close_first() {
    s = y;
    e = make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ void close() {
    const f2_t t = add2(s, y);
    if (COMP) e = add2(e, sub2(y, sub2(t, s)));
    s = t;
  }
  // the second of exactly two groups: its error is the whole correction
  __device__ __forceinline__ void close_second() {
    const f2_t t = add2(s, y);
    if (COMP) e = sub2(y, sub2(t, s));
    s = t;
  }
  __device__ __forceinline__ f2_t finish() const { return COMP ? add2(s, e) : s; }
  // s + a b, then the correction
  __device__ __forceinline__ f2_t finish(f2_t a, f2_t b) const {
    const f2_t r = fma2(a, b, s);
    return COMP ? add2(r, e) : r;
  }
};

// Limit of the producer's drain after a failed wait.  The copies it waits for
// were issued already and complete without any other warp, so this wait
// does not depend on the (possibly tiny) pipeline limit.
constexpr uint64_t kDrainLimitNs = 4000000000ull;
// Pipeline wait limit when the method sets none.
constexpr uint64_t kDefaultWaitNs = 2000000000ull;

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
// 16 bytes as two packed FP32x2 values, 8 bytes as one
__device__ __forceinline__ void lds2x64(uint32_t a, f2_t &lo, f2_t &hi) {
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(lo.x), "=f"(lo.y), "=f"(hi.x), "=f"(hi.y) : "r"(a));
}
__device__ __forceinline__ f2_t lds_b64(uint32_t a) {
  f2_t v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
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

// Items [i0, i1) of a tile's `items` for consumer warp `part` of `nparts`:
// shares start on multiples of 8 items, so that with G a multiple of 8 no
// quarter-warp spans two nodes.
__device__ __forceinline__ void warp_share(uint32_t items, int part, int nparts, uint32_t &i0, uint32_t &i1) {
  const uint32_t oct = (items + 7u) >> 3;
  i0 = (uint32_t)(((uint64_t)oct * part) / nparts) << 3;
  i1 = min(items, (uint32_t)(((uint64_t)oct * (part + 1)) / nparts) << 3);
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// 32-bit shared addresses of one staged tile, biased so that global indices
// address them: node i's row pointer at r + 4 i, CSR entry p's weight at
// w + 8 p (16 p for 16-byte records), its staged byte offset at l + 4 p,
// node i's self weights at s + 8 i (16 i); own node k's column at rows + k
// times the column pitch (wrap-around arithmetic; the sums land inside the
// stage).  The tile's own nodes are [n0, n1).
struct TileView {
  int32_t n0, n1;
  uint32_t rows, w, l, r, s;
  // slot list (div / curl, 0 = none): slot q = own node li | node lj << 16;
  // the first npairs slots are node pairs (li, lj), the rest single nodes
  uint32_t p;
  int32_t npairs;
};

// Consumer side.  A warp takes items [i0, i1) of tile t, one per lane,
// stride 32.  All but a handful of nodes of an octahedral mesh have six
// neighbours: for them the neighbour loop is fully unrolled into two groups
// of three, so every accumulator and address stays in fixed registers;
// other degrees take groups of two.  Staged data is loaded straight into
// packed FP32x2 registers.
//
// div / curl.  A staged (u, v) column is a sequence of 16-byte units of two
// levels each.  Item c of a slot takes the KU units c, c + G, c + 2G, ...
// (G items per slot).  With G a multiple of 8 and warp shares starting on
// multiples of 8 items, the 8 lanes of every quarter-warp read 8 consecutive
// units of one column, 128 contiguous bytes: no shared-memory bank
// conflicts.  More units per item spread each item's row pointers, offsets
// and weights (loaded once per item) over more levels.  FUSED evaluates div
// and curl of the same wind in one pass: the staged columns, offsets and
// differences are shared, each operator keeps its own weights and sums, and
// each output gets exactly the arithmetic of its single-operator pass.
//
// Slots.  Without a slot list a slot is one own node, in node order.  With
// one, the first npairs slots are node pairs (i, j): adjacent six-neighbour
// nodes whose rows both start with their two shared neighbours A, B and
// then the partner.  A pair item reads the columns of i, j, A and B once,
// forms the first group of both nodes (A, B and the partner, whose
// difference x_i - x_j is the exact negation of x_j - x_i), then each
// node's other three neighbours: 10 column reads for two nodes instead of
// 14, and each node's sum takes the same terms in the same order as on the
// single-node path, so the bits are the same.
//
// A supplies G, g_magic32, nlev, the FP64 weights of the pole path
// (w64, w64b, s64, s64b), the outputs (out, out2, out_stride), and for the
// bounds-checked build status and col_area (staged column offsets lie below
// it); v locates the tile's columns (own node k at v.rows + k rb), staged
// metadata and slot list; pole tiles run in FP64 (they hold no pairs).
// PAIRS = false compiles the consumer without the slot list and pair path.
// GC > 0 fixes G at compile time (it must equal a.G): each unit's offset in
// a column is then a constant the shared-memory loads take as an immediate,
// instead of an integer add per neighbour and unit.
template <bool COMP, bool FUSED, int KU, bool PAIRS, int GC, class A>
__device__ __forceinline__ void divcurl_tile(const A &a, const TileView &v, bool pole, uint32_t rb, int part,
                                             int nparts) {
  const uint32_t n = (uint32_t)(v.n1 - v.n0);
  const uint32_t npairs = (PAIRS && v.p) ? (uint32_t)v.npairs : 0u;
  uint32_t i0, i1;
  warp_share((n - npairs) * (uint32_t)a.G, part, nparts, i0, i1);
  const uint32_t units = (uint32_t)(a.nlev + 1) >> 1;
  const uint32_t G = GC > 0 ? (uint32_t)GC : (uint32_t)a.G;
  const uint32_t rs = FUSED ? 16u : 8u;  // bytes of a weight record (and of a self-weight record)
  // weights of staged record `at`: div, and curl when fused
  auto weights = [&](uint32_t at, f2_t &wd, f2_t &wc) {
    if (FUSED) lds2x64(at, wd, wc);
    else {
      wd = lds_b64(at);
      wc = make_float2(0.f, 0.f);
    }
  };
  // a neighbour's staged column offset (relative to v.rows)
  auto column = [&](uint32_t at) { return (uint32_t)NB_IDX(lds_u32(at), 0, a.col_area, a.status); };
  // unit k holds levels 2u, 2u + 1 (u = c + k G)
  const uint32_t nfull = (uint32_t)a.nlev >> 1;  // units holding two valid levels
  auto put = [&](float *oo, const float (&o)[2 * KU], uint32_t c, const bool (&has)[KU]) {
    float *ob = oo + 2 * c;
#pragma unroll
    for (int k = 0; k < KU; ++k) {
      if (!has[k]) continue;
      float *p = ob + 2 * (uint32_t)k * G;
      // with G compiled in (more than (KU - 1) G units), every unit but the
      // last of an item exists and holds two levels
      if ((GC > 0 && k < KU - 1) || c + (uint32_t)k * G < nfull)
        __stcs(reinterpret_cast<float2 *>(p), make_float2(o[2 * k], o[2 * k + 1]));
      else p[0] = o[2 * k];
    }
  };
  // self terms (su, sv) . (u_i, v_i) of `node`, then the (u, v) halves
  auto finish_node = [&](int32_t node, const f2_t (&x)[KU][2], const GroupSum<COMP> (&sd)[KU][2],
                         const GroupSum<COMP> (&sc)[KU][2], float (&r)[2 * KU], float (&z)[2 * KU]) {
    f2_t sw_div, sw_curl;
    weights(v.s + rs * (uint32_t)node, sw_div, sw_curl);
#pragma unroll
    for (int k = 0; k < KU; ++k)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float x0, y0;
        upk(sd[k][h].finish(sw_div, x[k][h]), x0, y0);
        r[2 * k + h] = __fadd_rn(x0, y0);
        if (FUSED) {
          upk(sc[k][h].finish(sw_curl, x[k][h]), x0, y0);
          z[2 * k + h] = __fadd_rn(x0, y0);
        }
      }
  };
  auto close_all = [&](GroupSum<COMP> (&sd)[KU][2], GroupSum<COMP> (&sc)[KU][2], int which) {
#pragma unroll
    for (int k = 0; k < KU; ++k)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (which == 0) sd[k][h].close_first();
        else if (which == 1) sd[k][h].close_second();
        else sd[k][h].close();
        if (FUSED) {
          if (which == 0) sc[k][h].close_first();
          else if (which == 1) sc[k][h].close_second();
          else sc[k][h].close();
        }
      }
  };
  // the item loop, compiled once for main tiles and once for the pole tiles
  // (FP64, never pairs); the flag is uniform per tile
  auto walk = [&](auto pole_tag) {
    constexpr bool POLE = decltype(pole_tag)::value;
    for (uint32_t item = i0 + (threadIdx.x & 31); item < i1; item += 32) {
      const uint32_t q = GC > 0 ? item / (uint32_t)GC : __umulhi(item, a.g_magic32);
      const uint32_t c = item - q * G;
      if (GC == 0 && c >= units) continue;  // G * KU may exceed the column's units
      uint32_t il = q, jl = 0;
      if (PAIRS && v.p) {
        const uint32_t sl = lds_u32(v.p + 4u * q);
        il = (uint32_t)NB_IDX(sl & 0xffffu, 0, n, a.status);
        jl = (uint32_t)NB_IDX(sl >> 16, 0, n, a.status);
      }
      // byte offset of each unit in a column; a unit past the column reads
      // unit c again and is not stored
      uint32_t uo[KU];
      bool has[KU];
  #pragma unroll
      for (int k = 0; k < KU; ++k) {
        const uint32_t u = c + (uint32_t)k * G;
        has[k] = (GC > 0 && k < KU - 1) || u < units;
        uo[k] = 16u * (has[k] ? u : c);
      }
      const int32_t node = v.n0 + (int32_t)il;
      // unit c of a column at (column offset) + cb; unit k at + rel[k]
      const uint32_t cb = v.rows + 16u * c;
      uint32_t rel[KU];
#pragma unroll
      for (int k = 0; k < KU; ++k) rel[k] = uo[k] - 16u * c;
      const uint32_t own = cb + il * rb;
      // terms of the staged neighbour column `col` for a node with own values x
      auto accumulate = [&](GroupSum<COMP> (&sd)[KU][2], GroupSum<COMP> (&sc)[KU][2], const f2_t (&x)[KU][2],
                            uint32_t col, f2_t wd, f2_t wc, bool first) {
  #pragma unroll
        for (int k = 0; k < KU; ++k) {
          f2_t n0, n1;
          lds2x64(col + rel[k], n0, n1);
          const f2_t d0 = sub2(n0, x[k][0]), d1 = sub2(n1, x[k][1]);
          if (first) {
            sd[k][0].start(wd, d0);
            sd[k][1].start(wd, d1);
            if (FUSED) {
              sc[k][0].start(wc, d0);
              sc[k][1].start(wc, d1);
            }
          } else {
            sd[k][0].term(wd, d0);
            sd[k][1].term(wd, d1);
            if (FUSED) {
              sc[k][0].term(wc, d0);
              sc[k][1].term(wc, d1);
            }
          }
        }
      };
      if (!POLE && PAIRS && q < npairs) {
        // node pair (il, jl): rows (A, B, partner, three others)
        const int32_t nodej = v.n0 + (int32_t)jl;
        const uint32_t pi = (uint32_t)lds_s32(v.r + 4u * (uint32_t)node);
        const uint32_t pj = (uint32_t)lds_s32(v.r + 4u * (uint32_t)nodej);
        const uint32_t ownj = cb + jl * rb;
        f2_t xi[KU][2], xj[KU][2];
  #pragma unroll
        for (int k = 0; k < KU; ++k) {
          lds2x64(own + rel[k], xi[k][0], xi[k][1]);
          lds2x64(ownj + rel[k], xj[k][0], xj[k][1]);
        }
        GroupSum<COMP> sdi[KU][2], sci[KU][2], sdj[KU][2], scj[KU][2];
        const uint32_t wi = v.w + rs * pi, wj = v.w + rs * pj;
        const uint32_t li = v.l + 4u * pi, lj = v.l + 4u * pj;
        // first group of both nodes: the shared neighbours A and B ...
  #pragma unroll
        for (int e = 0; e < 2; ++e) {
          const uint32_t col = cb + column(li + 4u * e);
          f2_t wdi, wci, wdj, wcj;
          weights(wi + rs * e, wdi, wci);
          weights(wj + rs * e, wdj, wcj);
  #pragma unroll
          for (int k = 0; k < KU; ++k) {
            f2_t n0, n1;
            lds2x64(col + rel[k], n0, n1);
            const f2_t n[2] = {n0, n1};
  #pragma unroll
            for (int h = 0; h < 2; ++h) {
              const f2_t di = sub2(n[h], xi[k][h]), dj = sub2(n[h], xj[k][h]);
              if (e == 0) {
                sdi[k][h].start(wdi, di);
                sdj[k][h].start(wdj, dj);
                if (FUSED) {
                  sci[k][h].start(wci, di);
                  scj[k][h].start(wcj, dj);
                }
              } else {
                sdi[k][h].term(wdi, di);
                sdj[k][h].term(wdj, dj);
                if (FUSED) {
                  sci[k][h].term(wci, di);
                  scj[k][h].term(wcj, dj);
                }
              }
            }
          }
        }
        // ... and the partner
        {
          f2_t wdi, wci, wdj, wcj;
          weights(wi + 2u * rs, wdi, wci);
          weights(wj + 2u * rs, wdj, wcj);
  #pragma unroll
          for (int k = 0; k < KU; ++k)
  #pragma unroll
            for (int h = 0; h < 2; ++h) {
              const f2_t d = sub2(xj[k][h], xi[k][h]), nd = make_float2(-d.x, -d.y);
              sdi[k][h].term(wdi, d);
              sdj[k][h].term(wdj, nd);
              if (FUSED) {
                sci[k][h].term(wci, d);
                scj[k][h].term(wcj, nd);
              }
            }
        }
        close_all(sdi, sci, 0);
        close_all(sdj, scj, 0);
        // second group of node i, then of node j
  #pragma unroll
        for (int e = 3; e < 6; ++e) {
          f2_t wd, wc;
          weights(wi + rs * e, wd, wc);
          accumulate(sdi, sci, xi, cb + column(li + 4u * e), wd, wc, e == 3);
        }
        close_all(sdi, sci, 1);
        {
          float r[2 * KU], z[2 * KU];
          finish_node(node, xi, sdi, sci, r, z);
          put(a.out + (int64_t)node * a.out_stride, r, c, has);
          if (FUSED) put(a.out2 + (int64_t)node * a.out_stride, z, c, has);
        }
  #pragma unroll
        for (int e = 3; e < 6; ++e) {
          f2_t wd, wc;
          weights(wj + rs * e, wd, wc);
          accumulate(sdj, scj, xj, cb + column(lj + 4u * e), wd, wc, e == 3);
        }
        close_all(sdj, scj, 1);
        {
          float r[2 * KU], z[2 * KU];
          finish_node(nodej, xj, sdj, scj, r, z);
          put(a.out + (int64_t)nodej * a.out_stride, r, c, has);
          if (FUSED) put(a.out2 + (int64_t)nodej * a.out_stride, z, c, has);
        }
        continue;
      }
      const int32_t p0 = lds_s32(v.r + 4u * (uint32_t)node), p1 = lds_s32(v.r + 4u * (uint32_t)node + 4u);
      float r[2 * KU], z[2 * KU];
      if constexpr (!POLE) {
        f2_t x[KU][2];  // own (u, v) at levels 2u and 2u + 1 of each unit
  #pragma unroll
        for (int k = 0; k < KU; ++k) lds2x64(own + rel[k], x[k][0], x[k][1]);
        GroupSum<COMP> sd[KU][2], sc[KU][2];
        // weights of entry e: single pass, 8-byte (w.x, w.y) at pw + 8 e; fused,
        // 16-byte (div, curl) records at pw + 16 e
        const uint32_t pw = v.w + rs * (uint32_t)p0;
        const uint32_t pl = v.l + 4u * (uint32_t)p0;
        // neighbour entry e: its units minus the node's own, times the weights
        auto nbr = [&](uint32_t e, bool first) {
          const uint32_t col = cb + column(pl + 4u * e);
          f2_t wd, wc;
          weights(pw + rs * e, wd, wc);
          accumulate(sd, sc, x, col, wd, wc, first);
        };
        const int deg = p1 - p0;
        if (deg == 6) {
          nbr(0, true), nbr(1, false), nbr(2, false);
          close_all(sd, sc, 0);
          nbr(3, true), nbr(4, false), nbr(5, false);
          close_all(sd, sc, 1);
        } else {
          int e = 0;
          for (; e + 1 < deg; e += 2) {
            nbr((uint32_t)e, true), nbr((uint32_t)e + 1, false);
            close_all(sd, sc, e == 0 ? 0 : 2);
          }
          if (e < deg) {
            nbr((uint32_t)e, true);
            close_all(sd, sc, e == 0 ? 0 : 2);
          }
        }
        finish_node(node, x, sd, sc, r, z);
      } else {
        float iu[2 * KU], iv[2 * KU];
  #pragma unroll
        for (int k = 0; k < KU; ++k) {
          const float4 x4 = lds128(own + rel[k]);
          iu[2 * k] = x4.x, iv[2 * k] = x4.y, iu[2 * k + 1] = x4.z, iv[2 * k + 1] = x4.w;
        }
        double sacc[2 * KU], zacc[2 * KU];
  #pragma unroll
        for (int j = 0; j < 2 * KU; ++j) sacc[j] = zacc[j] = 0.0;
        for (int32_t p = p0; p < p1; ++p) {
          const double2 w = __ldg(a.w64 + p);
          const double2 qw = FUSED ? __ldg(a.w64b + p) : w;
          const uint32_t col = cb + column(v.l + 4u * (uint32_t)p);
  #pragma unroll
          for (int k = 0; k < KU; ++k) {
            const float4 C = lds128(col + rel[k]);
            const float ju[2] = {C.x, C.z}, jv[2] = {C.y, C.w};
  #pragma unroll
            for (int h = 0; h < 2; ++h) {
              const double du = (double)ju[h] - (double)iu[2 * k + h];
              const double dv = (double)jv[h] - (double)iv[2 * k + h];
              sacc[2 * k + h] = fma(w.y, dv, fma(w.x, du, sacc[2 * k + h]));
              if (FUSED) zacc[2 * k + h] = fma(qw.y, dv, fma(qw.x, du, zacc[2 * k + h]));
            }
          }
        }
        const double2 sw = __ldg(a.s64 + node);
        const double2 sx = FUSED ? __ldg(a.s64b + node) : sw;
  #pragma unroll
        for (int j = 0; j < 2 * KU; ++j) {
          r[j] = (float)fma(sw.y, (double)iv[j], fma(sw.x, (double)iu[j], sacc[j]));
          if (FUSED) z[j] = (float)fma(sx.y, (double)iv[j], fma(sx.x, (double)iu[j], zacc[j]));
        }
      }
      put(a.out + (int64_t)node * a.out_stride, r, c, has);
      if (FUSED) put(a.out2 + (int64_t)node * a.out_stride, z, c, has);
    }
  };
  if (pole) walk(std::true_type{});
  else walk(std::false_type{});
}

// Host helpers of the staged kernels (tiled.cu).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn();  // cuTensorMapEncodeTiled from the driver (NULL if missing)
// x / d == (x * magic) >> shift for x < 2^24
void magic_div(uint32_t d, uint64_t &magic, uint32_t &shift);
// x / d == __umulhi(x, magic32(d)) for 2 <= d and x < 2^32 / d
uint32_t magic32(uint32_t d);
int sm_count(int *out);
// item shape of the div / curl consumers (KU units per item, G items per node)
void item_shape(int units_req, int align_req, int units, int &KU, int &G);

}  // namespace nb
