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
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "kernels_common.cuh"
#include "staged_common.cuh"

namespace nb {

// device status word: 0 = ok, otherwise an NB_* code (first error wins)
__device__ int g_device_status = 0;

int launch_tiled(nb_method *m, int op, const nb_field *in, const nb_field *out, const nb_field *out2,
                 cudaStream_t st, bool *handled, int comp = -1);

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
  uint32_t g_magic32;  // item / G == umulhi(item, g_magic32) for item < 2^32 / G (magic32)
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
  int32_t nnodes;       // nodes of the mesh (index checks)
  uint32_t col_area;    // staged column offsets lie below this (index checks)
  // node pairs (div / curl): tile t's slot list is slots[slot_ptr[t] ..
  // slot_ptr[t + 1]), its first npairs[t] slots pairs; off_p = 0: no pairs
  const int32_t *slot_ptr;
  const int32_t *npairs;
  const uint32_t *slots;
  uint32_t off_p;       // stage offset of the slot list
};

// What the producer reads from global memory to issue a tile's copies: its
// node and halo ranges, its CSR range, and this lane's first group of four
// halo nodes.  Loaded one iteration ahead, while the producer waits for the
// stage to be released, so that a release is followed at once by the copies.
struct TilePrep {
  int32_t n0, n1, h0, h1, pa, pb;
  int32_t qa, qb, np;  // slot list range and pair count (node pairs only)
  int32_t y[4];  // halo nodes of group `lane` (when the tile has that group)
};

__device__ __forceinline__ TilePrep prepare_tile(const TiledArgs &a, int t, int lane) {
  TilePrep p;
  p.n0 = __ldg(a.tile_node0 + t);
  p.n1 = __ldg(a.tile_node0 + t + 1);
  p.h0 = __ldg(a.halo_ptr + t);
  p.h1 = __ldg(a.halo_ptr + t + 1);
  p.pa = __ldg(a.row_ptr + p.n0);
  p.pb = __ldg(a.row_ptr + p.n1);
  p.qa = p.qb = p.np = 0;
  if (a.off_p) {
    p.qa = __ldg(a.slot_ptr + t);
    p.qb = __ldg(a.slot_ptr + t + 1);
    p.np = __ldg(a.npairs + t);
  }
  const uint32_t H = (uint32_t)(p.h1 - p.h0);
  if ((uint32_t)lane < ((H + 3u) >> 2)) {
    // a short last group repeats its last node (the copy fills the group's slots)
    const int32_t *hp = a.halo + p.h0;
    const uint32_t k = 4u * (uint32_t)lane, last = H - 1u;
#pragma unroll
    for (int q = 0; q < 4; ++q) p.y[q] = (int32_t)NB_IDX(__ldg(hp + min(k + (uint32_t)q, last)), 0, a.nnodes, a.status);
  }
  return p;
}

// Issue the copies of a prepared tile into the stage at `stage` (one whole
// warp).
__device__ __forceinline__ void issue_tile(const TiledArgs &a, const CUtensorMap *map, const TilePrep &p,
                                           uint32_t stage, uint32_t bar, int lane) {
  const int32_t n0 = p.n0, n1 = p.n1, h0 = p.h0, h1 = p.h1, pa = p.pa, pb = p.pb;
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
  const uint32_t pbytes = (uint32_t)(p.qb - p.qa) * 4u;  // a multiple of 16 (lists padded to 4 slots)
#ifdef NB_BOUNDS_CHECK
  // a tile whose copies would leave their stage regions is not copied: it is
  // published empty and NB_EINVAL is recorded
  {
    const uint32_t send = a.off_s ? a.off_s : a.off_p ? a.off_p : a.off_h;
    const uint32_t pend = a.off_p ? a.off_p : a.off_h;
    const bool bad = n1 <= n0 || n1 > a.nnodes || h1 < h0 || hbase + groups * a.gpitch > a.off_w ||
                     a.off_w + wbytes > a.off_l || a.off_l + lbytes > a.off_r || a.off_r + rbytes > send ||
                     (a.off_s && a.off_s + sbytes > pend) || (a.off_p && a.off_p + pbytes > a.off_h) ||
                     p.np < 0 || 2 * p.np > (int32_t)n || (a.off_p && 4u * (n - (uint32_t)p.np) > pbytes);
    if (bad) {
      if (lane == 0) {
        atomicCAS(a.status, 0, (int)NB_EINVAL);
        asm volatile("st.shared.v4.s32 [%0], {%1, %1, %2, %2};" ::"r"(stage + a.off_h), "r"(n0), "r"(0) : "memory");
        mbar_expect_tx(bar, 0);
      }
      __syncwarp();
      return;
    }
  }
#endif
  if (lane == 0) {
    // header for the consumers, published by the arrive below
    asm volatile("st.shared.v4.s32 [%0], {%1, %2, %3, %4};" ::"r"(stage + a.off_h), "r"(n0), "r"(n1), "r"(p.np),
                 "r"(0)
                 : "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (lane == 0)
    mbar_expect_tx(bar, body + wbytes + lbytes + rbytes + sbytes + pbytes + groups * 4u * a.copy_bytes);
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
  if (lane == 5 && pbytes) bulk_g2s(stage + a.off_p, a.slots + p.qa, pbytes, bar);
  if ((uint32_t)lane < groups)
    gather4_g2s(stage + hbase + (uint32_t)lane * a.gpitch, map, p.y[0], p.y[1], p.y[2], p.y[3], bar);
  for (uint32_t g = (uint32_t)lane + 32u; g < groups; g += 32) {
    // groups past the 32nd (rare): halo nodes loaded here
    const int32_t *hp = a.halo + h0;
    const uint32_t k = 4u * g, last = H - 1u;
    auto hid = [&](uint32_t q) { return (int32_t)NB_IDX(__ldg(hp + q), 0, a.nnodes, a.status); };
    gather4_g2s(stage + hbase + g * a.gpitch, map, hid(k), hid(min(k + 1u, last)), hid(min(k + 2u, last)),
                hid(min(k + 3u, last)), bar);
  }
}

// The view of one staged tile of the single-operator and fused passes.
__device__ __forceinline__ TileView staged_view(const TiledArgs &a, uint32_t stage) {
  TileView v;
  v.n0 = lds_s32(stage + a.off_h);
  v.n1 = lds_s32(stage + a.off_h + 4u);
  v.rows = stage;
  v.s = a.rec16 ? stage + a.off_s - 16u * (uint32_t)v.n0 : stage + a.off_s - 8u * (uint32_t)(v.n0 & ~1);
  const int32_t ra = v.n0 & ~3;
  v.r = stage + a.off_r - 4u * (uint32_t)ra;
  const int32_t pa = lds_s32(v.r + 4u * (uint32_t)v.n0);
  v.w = a.rec16 ? stage + a.off_w - 16u * (uint32_t)pa : stage + a.off_w - 8u * (uint32_t)(pa & ~1);
  v.l = stage + a.off_l - 4u * (uint32_t)(pa & ~3);
  v.p = a.off_p ? stage + a.off_p : 0u;
  v.npairs = lds_s32(stage + a.off_h + 8u);
  return v;
}

// grad.  Item c of a slot takes the 4-level unit c of its scalar column;
// each weight is broadcast to both lanes of a packed register.  A node pair
// slot (see divcurl_tile) evaluates both nodes from 10 staged columns: the
// shared neighbours A and B and the partner first, then each node's other
// three, every node's terms in its row order as on the single-node path.
// PAIRS = false compiles it without the slot list and pair path.
template <bool COMP, bool PAIRS>
__device__ __forceinline__ void grad_tile(const TiledArgs &a, int t, uint32_t stage, int part,
                                          int nparts) {
  const TileView v = staged_view(a, stage);
  const uint32_t n = (uint32_t)(v.n1 - v.n0);
  const uint32_t npairs = (PAIRS && v.p) ? (uint32_t)v.npairs : 0u;
  const uint32_t items = (n - npairs) * a.G;
  const uint32_t i0 = (uint32_t)(((uint64_t)items * part) / nparts);
  const uint32_t i1 = (uint32_t)(((uint64_t)items * (part + 1)) / nparts);
  const bool pole = t >= a.ntiles_main;
  const uint32_t rb = a.row_bytes;
  struct Acc {
    GroupSum<COMP> x01, x23, y01, y23;
  };
  // terms w (f_j - f_i) of one neighbour, four levels
  auto term = [](Acc &s, float2 w, f2_t d01, f2_t d23, bool first) {
    const f2_t wx = pk(w.x, w.x), wy = pk(w.y, w.y);
    if (first) {
      s.x01.start(wx, d01), s.x23.start(wx, d23), s.y01.start(wy, d01), s.y23.start(wy, d23);
    } else {
      s.x01.term(wx, d01), s.x23.term(wx, d23), s.y01.term(wy, d01), s.y23.term(wy, d23);
    }
  };
  auto close = [](Acc &s, int which) {  // 0: first group, 1: second of two, 2: later
    GroupSum<COMP> *acc[4] = {&s.x01, &s.x23, &s.y01, &s.y23};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (which == 0) acc[j]->close_first();
      else if (which == 1) acc[j]->close_second();
      else acc[j]->close();
    }
  };
  auto store = [&](int32_t node, int l0, const float (&gx)[4], const float (&gy)[4]) {
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
  };
  auto finish = [&](int32_t node, int l0, const Acc &s) {
    float gx[4], gy[4];
    upk(s.x01.finish(), gx[0], gx[1]);
    upk(s.x23.finish(), gx[2], gx[3]);
    upk(s.y01.finish(), gy[0], gy[1]);
    upk(s.y23.finish(), gy[2], gy[3]);
    store(node, l0, gx, gy);
  };
  // the item loop, compiled once for main tiles and once for the pole tiles
  // (FP64, never pairs); the flag is uniform per tile
  auto walk = [&](auto pole_tag) {
    constexpr bool POLE = decltype(pole_tag)::value;
    for (uint32_t item = i0 + (threadIdx.x & 31); item < i1; item += 32) {
      const uint32_t q = __umulhi(item, a.g_magic32);
      const uint32_t c = item - q * a.G;
      const int l0 = 4 * (int)c;
      uint32_t il = q, jl = 0;
      if (PAIRS && v.p) {
        const uint32_t sl = lds_u32(v.p + 4u * q);
        il = (uint32_t)NB_IDX(sl & 0xffffu, 0, n, a.status);
        jl = (uint32_t)NB_IDX(sl >> 16, 0, n, a.status);
      }
      const int32_t node = v.n0 + (int32_t)il;
      const uint32_t col = v.rows + c * 16u;
      auto column = [&](uint32_t at) { return col + (uint32_t)NB_IDX(lds_u32(at), 0, a.col_area, a.status); };
      if (!POLE && PAIRS && q < npairs) {
        // node pair (il, jl): rows (A, B, partner, three others)
        const int32_t nodej = v.n0 + (int32_t)jl;
        const uint32_t pi = (uint32_t)lds_s32(v.r + 4u * (uint32_t)node);
        const uint32_t pj = (uint32_t)lds_s32(v.r + 4u * (uint32_t)nodej);
        f2_t xi01, xi23, xj01, xj23;
        lds2x64(col + il * rb, xi01, xi23);
        lds2x64(col + jl * rb, xj01, xj23);
        Acc si, sj;
        const uint32_t wi = v.w + 8u * pi, wj = v.w + 8u * pj, li = v.l + 4u * pi, lj = v.l + 4u * pj;
  #pragma unroll
        for (int e = 0; e < 2; ++e) {
          f2_t f01, f23;
          lds2x64(column(li + 4u * e), f01, f23);
          term(si, lds64(wi + 8u * e), sub2(f01, xi01), sub2(f23, xi23), e == 0);
          term(sj, lds64(wj + 8u * e), sub2(f01, xj01), sub2(f23, xj23), e == 0);
        }
        {
          const f2_t d01 = sub2(xj01, xi01), d23 = sub2(xj23, xi23);
          term(si, lds64(wi + 16u), d01, d23, false);
          term(sj, lds64(wj + 16u), make_float2(-d01.x, -d01.y), make_float2(-d23.x, -d23.y), false);
        }
        close(si, 0);
        close(sj, 0);
  #pragma unroll
        for (int e = 3; e < 6; ++e) {
          f2_t f01, f23;
          lds2x64(column(li + 4u * e), f01, f23);
          term(si, lds64(wi + 8u * e), sub2(f01, xi01), sub2(f23, xi23), e == 3);
        }
        close(si, 1);
        finish(node, l0, si);
  #pragma unroll
        for (int e = 3; e < 6; ++e) {
          f2_t f01, f23;
          lds2x64(column(lj + 4u * e), f01, f23);
          term(sj, lds64(wj + 8u * e), sub2(f01, xj01), sub2(f23, xj23), e == 3);
        }
        close(sj, 1);
        finish(nodej, l0, sj);
        continue;
      }
      const int32_t p0 = lds_s32(v.r + 4u * (uint32_t)node), p1 = lds_s32(v.r + 4u * (uint32_t)node + 4u);
      if constexpr (!POLE) {
        f2_t fi01, fi23;
        lds2x64(col + il * rb, fi01, fi23);
        Acc s;
        const uint32_t pw = v.w + 8u * (uint32_t)p0, pl = v.l + 4u * (uint32_t)p0;
        auto nbr = [&](uint32_t e, bool first) {
          const float2 w = lds64(pw + 8u * e);
          f2_t f01, f23;
          lds2x64(column(pl + 4u * e), f01, f23);
          term(s, w, sub2(f01, fi01), sub2(f23, fi23), first);
        };
        const int deg = p1 - p0;
        if (deg == 6) {
          nbr(0, true), nbr(1, false), nbr(2, false);
          close(s, 0);
          nbr(3, true), nbr(4, false), nbr(5, false);
          close(s, 1);
        } else {
          int e = 0;
          for (; e + 1 < deg; e += 2) {
            nbr((uint32_t)e, true), nbr((uint32_t)e + 1, false);
            close(s, e == 0 ? 0 : 2);
          }
          if (e < deg) {
            nbr((uint32_t)e, true);
            close(s, e == 0 ? 0 : 2);
          }
        }
        finish(node, l0, s);
      } else {
        const float4 fi = lds128(col + il * rb);
        double sx[4] = {0, 0, 0, 0}, sy[4] = {0, 0, 0, 0};
        const float fiv[4] = {fi.x, fi.y, fi.z, fi.w};
        for (int32_t p = p0; p < p1; ++p) {
          const double2 w = __ldg(a.w64 + p);
          const float4 fj = lds128(column(v.l + 4u * (uint32_t)p));
          const float fjv[4] = {fj.x, fj.y, fj.z, fj.w};
  #pragma unroll
          for (int k = 0; k < 4; ++k) {
            const double d = (double)fjv[k] - (double)fiv[k];
            sx[k] = fma(w.x, d, sx[k]);
            sy[k] = fma(w.y, d, sy[k]);
          }
        }
        float gx[4], gy[4];
  #pragma unroll
        for (int k = 0; k < 4; ++k) {
          gx[k] = (float)sx[k];
          gy[k] = (float)sy[k];
        }
        store(node, l0, gx, gy);
      }
    }
  };
  if (pole) walk(std::true_type{});
  else walk(std::false_type{});
}


// Consumer warps per operator.  Fewer warps than the SM could hold: timed on
// B300 at O1280 x 137 levels, 11-12 consumer warps beat 16 by 1-7 % (more
// warps only queue more shared-memory requests behind the same pipeline),
// and a block of at most 4 warps per scheduler leaves up to 128 registers a
// thread.
// The producer also prefetches into L2 the column block of the tile
// `ahead` steps further along the CTA's walk, so that its stage copy reads
// L2 instead of HBM (timed: 1-3 % per launch for the single operators).
// The fused pass used 2 steps until its tiles grew; at O1280 x 137 it then
// timed 3.10 ms with 1 step or none against 3.22 with 2 and 3.33 with 3.
#ifndef NB_GRAD_WARPS
#define NB_GRAD_WARPS 12
#endif
#ifndef NB_DIV_WARPS
#define NB_DIV_WARPS 11
#endif
#ifndef NB_DIVCURL_WARPS
#define NB_DIVCURL_WARPS 11
#endif
template <int OP>
struct StagedShape {
  static constexpr int warps = OP == 0 ? NB_GRAD_WARPS : OP == 1 ? NB_DIV_WARPS : NB_DIVCURL_WARPS;
  static constexpr int threads = 32 * (warps + 1);
  static constexpr int ahead = 1;
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
template <int OP, bool COMP, int KU, bool PAIRS, int GC>
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
    // producer: tile i+G's global metadata is loaded before waiting for the
    // stage tile i goes to
    int k = 0;
    bool failed = false;
    TilePrep next{};
    if ((int)blockIdx.x < a.ntiles) next = prepare_tile(a, tile_at(a, blockIdx.x), lane);
    for (int i = blockIdx.x; i < a.ntiles; i += G, ++k) {
      const TilePrep cur = next;
      if (i + G < a.ntiles) next = prepare_tile(a, tile_at(a, i + G), lane);
      const int s = k % NS;
      if (k >= NS && !mbar_wait_bounded(empty0 + 8 * s, (uint32_t)(k / NS - 1) & 1u, a.timeout_ns)) {
        failed = true;
        break;
      }
      issue_tile(a, &map, cur, stage0 + s * a.stage_bytes, full0 + 8 * s, lane);
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
    if (OP == 0) grad_tile<COMP, PAIRS>(a, t, rows, warp, W);
    else if (OP == 1)
      divcurl_tile<COMP, false, KU, PAIRS, GC>(a, staged_view(a, rows), t >= a.ntiles_main, a.row_bytes, warp, W);
    else divcurl_tile<COMP, true, KU, PAIRS, GC>(a, staged_view(a, rows), t >= a.ntiles_main, a.row_bytes, warp, W);
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
  {
    // every staged offset must decode to the column of its neighbour
    const int64_t rb = tp->row_bytes, cb = tp->copy_bytes, gp = (4 * cb + 127) / 128 * 128;
    auto slot = [&](int64_t p, int, int64_t n) -> int64_t {
      const int64_t off = loff[p], hb = (n * rb + 127) / 128 * 128;
      if (off < n * rb) return off % rb == 0 ? off / rb : -1;
      if (off < hb) return -1;
      const int64_t r = (off - hb) % gp;
      return (r % cb == 0 && r / cb < 4) ? n + 4 * ((off - hb) / gp) + r / cb : -1;
    };
    std::string why;
    if (!check_tile_plan(mesh, (int)node0.size() - 1, node0.data(), hptr.data(), halo.data(), slot, why)) {
      set_error("staged kernel: invalid tile plan (" + why + ")");
      return NB_EINVAL;
    }
  }
  loff.resize(loff.size() + 8, 0);  // slack for 16-byte bounding copies
  if (halo.empty()) halo.push_back(0);
  tp->ntiles = (int)node0.size() - 1;
  // slot lists: the tile's node pairs (both nodes own nodes of the tile),
  // then its other nodes, each list padded to a multiple of 4 slots
  std::vector<int32_t> sptr(tp->ntiles + 1, 0), npairs(tp->ntiles, 0);
  std::vector<uint32_t> slots;
  slots.reserve(mesh->V + 4 * (size_t)tp->ntiles);
  for (int t = 0; t < tp->ntiles; ++t) {
    const int32_t a = node0[t], b = node0[t + 1];
    sptr[t] = (int32_t)slots.size();
    for (int32_t k = a; k < b; ++k) {
      const int32_t j = mesh->mate[k];
      if (j > k && j < b) slots.push_back((uint32_t)(k - a) | (uint32_t)(j - a) << 16);
    }
    npairs[t] = (int32_t)slots.size() - sptr[t];
    tp->paired_nodes += 2 * npairs[t];
    for (int32_t k = a; k < b; ++k) {
      const int32_t j = mesh->mate[k];
      if (!(j >= a && j < b)) slots.push_back((uint32_t)(k - a) * 0x10001u);
    }
    while (slots.size() % 4) slots.push_back(0);
  }
  sptr[tp->ntiles] = (int32_t)slots.size();
  {
    std::string why;
    if (!check_slot_lists(mesh, tp->ntiles, node0.data(), sptr.data(), npairs.data(), slots.data(), why)) {
      set_error("staged kernel: invalid slot list (" + why + ")");
      return NB_EINVAL;
    }
  }
  log_msg(1, "staged plan: %d tiles (%d pole-row), column pitch %lld B, stage area %lld B, largest halo %d, "
          "%zu halo columns in all", tp->ntiles, tp->ntiles - tp->ntiles_main, (long long)tp->row_bytes,
          (long long)tp->area, tp->max_halo, halo.size());
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
  if ((st = up((void **)&tp->d_slot_ptr, sptr.data(), sptr.size() * 4))) return st;
  if ((st = up((void **)&tp->d_npairs, npairs.data(), npairs.size() * 4))) return st;
  if ((st = up((void **)&tp->d_slots, slots.data(), slots.size() * 4))) return st;
  log_msg(1, "staged plan: %lld of %lld nodes in pair slots", (long long)tp->paired_nodes, (long long)mesh->V);
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
EncodeTiledFn encode_fn() {
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
void magic_div(uint32_t d, uint64_t &magic, uint32_t &shift) {
  uint32_t s = 0;
  while ((1u << s) < d) ++s;
  shift = 32 + s;
  magic = ((1ull << shift) + d - 1) / d;
}

// x / d == umulhi(x, m) with m = ceil(2^32 / d), for 2 <= d and x < 2^32 / d:
// m = 2^32 / d + e with 0 <= e < 1, so x m / 2^32 = x / d + x e / 2^32, and
// the excess x e / 2^32 < 1 / d cannot reach the next multiple of 1 / d
// above x / d.  The staged kernels' items per tile (at most 1024 nodes x
// d items) stay far below 2^32 / d.
uint32_t magic32(uint32_t d) { return (uint32_t)(((1ull << 32) + d - 1) / d); }

template <int OP, bool COMP, int KU, bool PAIRS, int GC>
static int launch_staged_t(const TiledArgs &a, const CUtensorMap &map, int grid, size_t smem,
                           cudaStream_t st) {
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [&] {
    attr_err = cudaFuncSetAttribute(staged_f32<OP, COMP, KU, PAIRS, GC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    227 * 1024);
  });
  NB_CUDA(attr_err);
  staged_f32<OP, COMP, KU, PAIRS, GC><<<grid, StagedShape<OP>::threads, smem, st>>>(a, map);
  count_launch(1);
  NB_CUDA(cudaGetLastError());
  return NB_OK;
}

template <int OP, int KU, int GC = 0>
static int launch_staged_sel(bool comp, bool pairs, const TiledArgs &a, const CUtensorMap &map, int grid,
                             size_t smem, cudaStream_t st) {
  if (comp)
    return pairs ? launch_staged_t<OP, true, KU, true, GC>(a, map, grid, smem, st)
                 : launch_staged_t<OP, true, KU, false, GC>(a, map, grid, smem, st);
  return pairs ? launch_staged_t<OP, false, KU, true, GC>(a, map, grid, smem, st)
               : launch_staged_t<OP, false, KU, false, GC>(a, map, grid, smem, st);
}

// Items per slot compiled in: 24 is the aligned count of three-unit items
// for columns of 129 to 144 levels (137 in the benchmark configuration).
constexpr int kFixedG = 24;

static int g_sm_count = 0;

int sm_count(int *out) {
  if (g_sm_count == 0) {
    int dev = 0;
    NB_CUDA(cudaGetDevice(&dev));
    NB_CUDA(cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev));
  }
  *out = g_sm_count;
  return NB_OK;
}

// Item shape of the div / curl consumers for a column of `units` 16-byte
// units: KU units per item, G items per node.  units_req 2 or 3 fixes KU,
// align_req 1 (0) asks for G rounded up to a multiple of 8 (not rounded).
// Left to the library (0 / -1), the shape with the fewest shared-memory
// wavefronts per node is taken, (G / 32) (22 + 28 KU f): per warp-wide item
// ~22 for its row pointers, offsets and weights, 28 per unit for its seven
// 16-byte column loads, and f = 1.25 when quarter-warps can span two nodes
// (bank-conflict replays), else 1.  At 137 levels that is KU = 3, G = 24,
// timed on B300 at O1280 x 137: div 2.60 against 2.82 ms with KU = 2,
// G = 35, and div+curl 3.67 against 3.69 ms.
void item_shape(int units_req, int align_req, int units, int &KU, int &G) {
  double best = 1e30;
  for (int ku = 2; ku <= 3; ++ku) {
    if (units_req && units_req != ku) continue;
    for (int al = 0; al <= 1; ++al) {
      if (align_req >= 0 && align_req != al) continue;
      const int g = al ? ((units + ku - 1) / ku + 7) / 8 * 8 : (units + ku - 1) / ku;
      const double f = (g % 8 == 0) ? 1.0 : 1.25;
      const double cost = g * (22.0 + 28.0 * ku * f);
      if (cost < best) {
        best = cost;
        KU = ku;
        G = g;
      }
    }
  }
}

// Device address of the status word on the current device (looked up once
// per device).
int status_word(int **out) {
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
  const int nvar = in->nvar;
  // items per node: grad, one 4-level unit per item; div / curl, KU 2-level
  // units per item (item_shape)
  int KU = 1, G = (in->nlev + 3) / 4;
  if (nvar == 2) item_shape(m->item_units, m->item_align, (in->nlev + 1) / 2, KU, G);
  if (G < 2) return NB_OK;  // magic32 needs a divisor of at least 2 (nlev >= 16 gives G >= 3)
  // each 16-byte unit must lie inside the staged column
  if ((uint64_t)(nvar == 2 ? (in->nlev + 1) / 2 : G) * 16u > row_bytes) return NB_OK;
  const uint32_t copy_bytes = (uint32_t)(((int64_t)in->nlev * nvar * 4 + 15) / 16 * 16);
  // halo columns are gathered as tensor rows of 4-byte (scalar) or 8-byte
  // (vector) elements; a box row holds at most 256 elements
  const uint32_t esz = nvar == 2 ? 8u : 4u;
  if (copy_bytes / esz > 256u || encode_fn() == nullptr) return NB_OK;
  // nstages stages of stage_kb KB, one CTA per SM.  A stage holds the staged
  // columns, then the tile's weights, offsets and row pointers (bounding
  // ranges, 16-byte aligned).
  const int nstages = m->nstages > 0 ? m->nstages : 2;
  // two stages of 113 KB and their 32 bytes of barriers fill the 227 KB a CTA
  // may hold (timed at O1280 x 137 against 112 KB: grad 2.00 -> 1.98,
  // div+curl 3.25 -> 3.23 ms)
  const int stage_kb = m->stage_kb > 0 ? m->stage_kb : 113;
  // Metadata reservation: the plan caps a tile's own nodes at nmax and its
  // CSR entries at 7 per own node (tiles are cut earlier otherwise), and the
  // stage reserves that much metadata after the column area.
  auto up16 = [](uint32_t x) { return (x + 15u) & ~15u; };
  const uint32_t stage_target = (uint32_t)stage_kb * 1024u;
  const int nmax_req = m->tile_nodes > 0 ? m->tile_nodes : 256;
  const uint32_t rec = fused ? 16u : 8u;  // bytes per weight record and per self-weight record
  // slot list of the node pairs: at most nmax slots plus padding.  By
  // default (-1) every pass but the fused div+curl evaluates node pairs:
  // timed at O1280 x 137, pairs took grad from 2.14 to 2.03 ms and div from
  // 2.67 to 2.39 ms, while the fused pass, whose two sets of sums leave
  // fewer registers for a second node (157-168 a thread), ran 3.78 ms with
  // pairs against 3.66 ms without.
  const bool pairs = m->node_pairs > 0 || (m->node_pairs < 0 && !fused);
  // metadata bytes of a stage for at most nn own nodes
  auto meta_bytes = [&](int nn) {
    const int ec = 7 * nn + 16;
    return up16((uint32_t)(ec + 2) * rec) + up16((uint32_t)(ec + 8) * 4u) + up16((uint32_t)(nn + 8) * 4u) +
           (op == NB_OP_GRAD ? 0u : up16((uint32_t)(nn + 2) * rec)) + (pairs ? up16((uint32_t)(nn + 4) * 4u) : 0u) +
           16u;
  };
  // Own nodes a tile can reach: a tile of C staged columns has about
  // 6 sqrt(n) halo columns around its n own nodes (Hilbert tiles of
  // octahedral meshes; O1280: 45.8 own + 40.1 halo at 87 columns, ~130 +
  // ~69 at ~200), so n + 6 sqrt(n) = C.  The metadata is reserved for a cap
  // 25 % above that (a tile reaching it is cut there), C taken from the
  // column area left by a first reservation, rather than for a stage of own
  // nodes only: more of the stage holds columns.  Timed at O1280 x 137 for
  // the vector columns of div and div+curl: 2.26 -> 2.24 and 3.37 -> 3.29 ms;
  // the scalar columns of grad keep a stage of own nodes (the cap made its
  // tiles smaller: 2.00 -> 2.02 ms).
  auto own_cap = [&](double ccols) {
    const double rn = (-6.0 + std::sqrt(36.0 + 4.0 * ccols)) / 2.0;
    return std::max(1, std::min((int)(1.25 * rn * rn) + 8, (int)ccols + 1));
  };
  int nmax = std::min(nmax_req, (int)(stage_target / row_bytes) + 1);
  if (nvar == 2) {
    nmax = std::min(nmax_req, own_cap((double)stage_target / row_bytes));
    if (stage_target > meta_bytes(nmax))
      nmax = std::min(nmax_req, own_cap((double)(stage_target - meta_bytes(nmax)) / row_bytes));
  }
  const int ecap = 7 * nmax + 16;
  const uint32_t wsz = up16((uint32_t)(ecap + 2) * rec), lsz = up16((uint32_t)(ecap + 8) * 4u),
                 rsz = up16((uint32_t)(nmax + 8) * 4u);
  const uint32_t ssz = op == NB_OP_GRAD ? 0u : up16((uint32_t)(nmax + 2) * rec), hsz = 16u;
  const uint32_t psz = pairs ? up16((uint32_t)(nmax + 4) * 4u) : 0u;
  const uint32_t meta = wsz + lsz + rsz + ssz + psz + hsz;
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
  a.g_magic32 = magic32((uint32_t)a.G);
  a.copy_bytes = copy_bytes;
  a.gpitch = (4u * copy_bytes + 127u) & ~127u;
  a.off_w = area;
  a.off_l = a.off_w + wsz;
  a.off_r = a.off_l + lsz;
  a.off_s = ssz ? a.off_r + rsz : 0u;
  a.off_p = psz ? a.off_r + rsz + ssz : 0u;
  a.off_h = a.off_r + rsz + ssz + psz;
  a.slot_ptr = tp->d_slot_ptr;
  a.npairs = tp->d_npairs;
  a.slots = tp->d_slots;
  a.stage_bytes = (a.off_h + hsz + 127u) & ~127u;
  a.nstages = nstages;
  a.status = nullptr;
  if (const int rc = status_word(&a.status)) return rc;
  a.timeout_ns = m->wait_limit_ns >= 0 ? (uint64_t)m->wait_limit_ns : kDefaultWaitNs;
  a.nnodes = (int32_t)in->nnodes;
  a.col_area = area;
  const size_t smem = (size_t)nstages * a.stage_bytes + 16 * (size_t)nstages;
  if (smem > 227 * 1024) {
    set_error("staged kernel: nstages * stage size exceeds 227 KB of shared memory");
    return NB_EINVAL;
  }
  const int grid = std::min(tp->ntiles, g_sm_count);
  log_msg(2, "staged launch: op %d%s, %d levels x %d vars, %d units per item, %d items per slot, %d tiles, "
          "grid %d, %zu B shared, node pairs %s", op, fused ? " (div+curl)" : "", in->nlev, nvar, KU, G, tp->ntiles,
          grid, smem, pairs ? "on" : "off");
  *handled = true;
  const bool comp = comp_mode < 0 ? m->compensated != 0 : comp_mode != 0;
  if (g) return launch_staged_sel<0, 1>(comp, pairs, a, map, grid, smem, st);
  // compiled-in G: the consumers then skip the checks of an item's first
  // KU - 1 units, which needs more than (KU - 1) G units in a column
  const bool fixed = KU == 3 && G == kFixedG && (in->nlev + 1) / 2 > (KU - 1) * kFixedG;
  if (fused) {
    if (fixed) return launch_staged_sel<2, 3, kFixedG>(comp, pairs, a, map, grid, smem, st);
    return KU == 3 ? launch_staged_sel<2, 3>(comp, pairs, a, map, grid, smem, st)
                   : launch_staged_sel<2, 2>(comp, pairs, a, map, grid, smem, st);
  }
  if (fixed) return launch_staged_sel<1, 3, kFixedG>(comp, pairs, a, map, grid, smem, st);
  return KU == 3 ? launch_staged_sel<1, 3>(comp, pairs, a, map, grid, smem, st)
                 : launch_staged_sel<1, 2>(comp, pairs, a, map, grid, smem, st);
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
