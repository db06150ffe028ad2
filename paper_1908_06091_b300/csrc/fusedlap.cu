// fusedlap.cu -- single-pass Laplacian, L = div(grad f) (Sec. 4.7, Fig. 33:
// the Laplacian beside grad and div in one Nabla), for FP32 fields.
//
// The two-pass route writes the gradient g to HBM and reads it back (24
// bytes per node-level).  Here a tile's gradient never leaves shared
// memory: a persistent grid walks the tiles of a LapPlan; a producer warp
// stages f on the tile's own nodes (one bulk copy of their contiguous
// columns) and on its two rings of neighbours (tile::gather4 tensor copies),
// with the tile's metadata, in two alternating stages.  Twelve consumer
// warps then
//   1. compute g on the own and ring-1 nodes (the "g-nodes") into a
//      shared-memory g buffer, with the gradient kernel's arithmetic (FP64
//      for pole-row nodes), optionally also writing own nodes' g to HBM;
//   2. after all warps have written g (a consumer mbarrier), compute the
//      divergence of g on the own nodes with the divergence kernel's
//      consumer (divcurl_tile), reading g from the buffer;
//   3. release the stage, and before the next tile's g phase wait until
//      every warp has finished reading the buffer (a second mbarrier).
// Each output has exactly the arithmetic of the two-pass route, so the
// results are bit-identical to it.  f is read once from HBM and lap written
// once (8 bytes per node-level), at the price of recomputing g on ring 1
// and staging two rings of f columns: shared-memory traffic, not HBM, bounds
// this kernel.  Every wait is bounded; on timeout the kernel records
// NB_ETIMEOUT, drains its own copies and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "kernels_common.cuh"
#include "staged_common.cuh"

namespace nb {

struct LapArgs {
  int ntiles, ntiles_main;
  const int32_t *tile_node0, *halo_ptr, *halo, *r1_count, *gn_ptr, *rec_ptr;
  const uint32_t *gn;     // per g-node: record start relative to the tile | pole-row flag
  const float4 *rec;      // g-phase records (gx weight, gy weight, staged f offset, CSR index)
  const uint32_t *goff;   // per CSR entry of an own node: g-buffer byte offset of the neighbour
  const int32_t *row_ptr;
  const float2 *wd32, *sd32;   // divergence weights and self weights (FP32)
  const double2 *wg64;         // gradient weights (FP64, pole-row g-nodes)
  // divergence consumer (divcurl_tile): FP64 pole weights, outputs, item shape
  const double2 *w64, *s64, *w64b, *s64b;
  float *out, *out2;
  int64_t out_stride;
  int nlev;
  int G;
  uint32_t g_magic32;
  // gradient phase
  int Gg;
  uint64_t gg_magic;
  uint32_t gg_shift;
  float *gout;       // own nodes' gradient to HBM (nullptr: not written)
  int64_t g_stride;
  const char *in;
  uint32_t row_bytes;  // pitch of own f columns (= global pitch)
  int64_t in_stride;
  uint32_t copy_bytes, gpitch;  // ring columns: bytes each, pitch of a group of four
  uint32_t g_pitch;             // g-buffer column pitch
  uint32_t off_rec, off_gn, off_wd, off_go, off_rp, off_sd, off_h, stage_bytes, off_g;
  int nstages;
  int *status;
  uint64_t timeout_ns;
  int32_t nnodes;      // nodes of the mesh (index checks)
  uint32_t col_area;   // g-buffer bytes: the divergence phase's column offsets lie below (index checks)
};

constexpr int kLapWarps = 12;
constexpr int kLapThreads = 32 * (kLapWarps + 1);

// A tile's global metadata and this lane's first group of four ring nodes,
// loaded one iteration ahead while the producer waits for the stage.
struct LapPrep {
  int32_t n0, n1, h0, h1, g0, g1, q0, q1, pa, pb, H1;
  int32_t y[4];
};

__device__ __forceinline__ LapPrep prepare_lap_tile(const LapArgs &a, int t, int lane) {
  LapPrep p;
  p.n0 = __ldg(a.tile_node0 + t);
  p.n1 = __ldg(a.tile_node0 + t + 1);
  p.h0 = __ldg(a.halo_ptr + t);
  p.h1 = __ldg(a.halo_ptr + t + 1);
  p.g0 = __ldg(a.gn_ptr + t);
  p.g1 = __ldg(a.gn_ptr + t + 1);
  p.q0 = __ldg(a.rec_ptr + t);
  p.q1 = __ldg(a.rec_ptr + t + 1);
  p.pa = __ldg(a.row_ptr + p.n0);
  p.pb = __ldg(a.row_ptr + p.n1);
  p.H1 = __ldg(a.r1_count + t);
  const uint32_t H = (uint32_t)(p.h1 - p.h0);
  if ((uint32_t)lane < ((H + 3u) >> 2)) {
    const int32_t *hp = a.halo + p.h0;
    const uint32_t k = 4u * (uint32_t)lane, last = H - 1u;
#pragma unroll
    for (int q = 0; q < 4; ++q) p.y[q] = (int32_t)NB_IDX(__ldg(hp + min(k + (uint32_t)q, last)), 0, a.nnodes, a.status);
  }
  return p;
}

__device__ __forceinline__ void issue_lap_tile(const LapArgs &a, const CUtensorMap *map, const LapPrep &p,
                                               uint32_t stage, uint32_t bar, int lane) {
  const int32_t n0 = p.n0, n1 = p.n1, h0 = p.h0, h1 = p.h1, g0 = p.g0, g1 = p.g1, q0 = p.q0, q1 = p.q1;
  const int32_t pa = p.pa, pb = p.pb, H1 = p.H1;
  const uint32_t n = (uint32_t)(n1 - n0), H = (uint32_t)(h1 - h0);
  // 16-byte bounding ranges of the metadata arrays
  const int32_t ga = g0 & ~3, gb = (g1 + 3) & ~3;
  const int32_t wa = pa & ~1, wb = (pb + 1) & ~1;
  const int32_t la = pa & ~3, lb = (pb + 3) & ~3;
  const int32_t ra = n0 & ~3, rb = (n1 + 4) & ~3;
  const int32_t sa = n0 & ~1, sb = (n1 + 1) & ~1;
  const uint32_t body = (n - 1) * a.row_bytes + a.copy_bytes;
  const uint32_t recb = (uint32_t)(q1 - q0) * 16u, gnb = (uint32_t)(gb - ga) * 4u;
  const uint32_t wdb = (uint32_t)(wb - wa) * 8u, gob = (uint32_t)(lb - la) * 4u;
  const uint32_t rpb = (uint32_t)(rb - ra) * 4u, sdb = (uint32_t)(sb - sa) * 8u;
  const uint32_t groups = (H + 3u) >> 2;
  const uint32_t hbase = (n * a.row_bytes + 127u) & ~127u;
#ifdef NB_BOUNDS_CHECK
  // a tile whose copies would leave their stage regions is published empty
  {
    const bool bad = n1 <= n0 || n1 > a.nnodes || H1 < 0 || (uint32_t)H1 > H ||
                     hbase + groups * a.gpitch > a.off_rec || a.off_rec + recb > a.off_gn ||
                     a.off_gn + gnb > a.off_wd || a.off_wd + wdb > a.off_go || a.off_go + gob > a.off_rp ||
                     a.off_rp + rpb > a.off_sd || a.off_sd + sdb > a.off_h ||
                     (n + (uint32_t)H1) * a.g_pitch > a.col_area;
    if (bad) {
      if (lane == 0) {
        atomicCAS(a.status, 0, (int)NB_EINVAL);
        asm volatile("st.shared.v4.s32 [%0], {%1, %1, %2, %3};" ::"r"(stage + a.off_h), "r"(n0), "r"(0), "r"(g0)
                     : "memory");
        mbar_expect_tx(bar, 0);
      }
      __syncwarp();
      return;
    }
  }
#endif
  if (lane == 0) {
    asm volatile("st.shared.v4.s32 [%0], {%1, %2, %3, %4};" ::"r"(stage + a.off_h), "r"(n0), "r"(n1), "r"(H1),
                 "r"(g0)
                 : "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (lane == 0) mbar_expect_tx(bar, body + recb + gnb + wdb + gob + rpb + sdb + groups * 4u * a.copy_bytes);
  __syncwarp();
  if (lane == 0) bulk_g2s(stage, a.in + (int64_t)n0 * a.in_stride * 4, body, bar);
  if (lane == 1) bulk_g2s(stage + a.off_rec, a.rec + q0, recb, bar);
  if (lane == 2) bulk_g2s(stage + a.off_gn, a.gn + ga, gnb, bar);
  if (lane == 3) bulk_g2s(stage + a.off_wd, a.wd32 + wa, wdb, bar);
  if (lane == 4) bulk_g2s(stage + a.off_go, a.goff + la, gob, bar);
  if (lane == 5) bulk_g2s(stage + a.off_rp, a.row_ptr + ra, rpb, bar);
  if (lane == 6) bulk_g2s(stage + a.off_sd, a.sd32 + sa, sdb, bar);
  if ((uint32_t)lane < groups)
    gather4_g2s(stage + hbase + (uint32_t)lane * a.gpitch, map, p.y[0], p.y[1], p.y[2], p.y[3], bar);
  for (uint32_t g = (uint32_t)lane + 32u; g < groups; g += 32) {
    const int32_t *hp = a.halo + h0;
    const uint32_t k = 4u * g, last = H - 1u;
    auto hid = [&](uint32_t q) { return (int32_t)NB_IDX(__ldg(hp + q), 0, a.nnodes, a.status); };
    gather4_g2s(stage + hbase + g * a.gpitch, map, hid(k), hid(min(k + 1u, last)), hid(min(k + 2u, last)),
                hid(min(k + 3u, last)), bar);
  }
}

// Gradient phase: items (g-node k, 4-level unit c) of the tile's n + H1
// g-nodes, warp shares as in the other consumers.  The arithmetic of each
// g-node is that of the gradient kernel (grad_tile): two groups of three
// for six neighbours, groups of two otherwise, FP64 for pole-row nodes.
template <bool COMP>
__device__ __forceinline__ void lap_grad_phase(const LapArgs &a, uint32_t stage, uint32_t gbuf, int32_t n0,
                                               uint32_t n, uint32_t H1, int32_t g0, int part, int nparts) {
  uint32_t i0, i1;
  warp_share((n + H1) * (uint32_t)a.Gg, part, nparts, i0, i1);
  const uint32_t hbase = (n * a.row_bytes + 127u) & ~127u;
  const uint32_t gnb = stage + a.off_gn + 4u * (uint32_t)(g0 & 3);
  const uint32_t recb = stage + a.off_rec;
  for (uint32_t item = i0 + (threadIdx.x & 31); item < i1; item += 32) {
    const uint32_t k = (uint32_t)(((uint64_t)item * a.gg_magic) >> a.gg_shift);
    const uint32_t c = item - k * (uint32_t)a.Gg;
    const uint32_t gw = lds_u32(gnb + 4u * k);
    uint32_t rs = gw & 0x7fffffffu, re = lds_u32(gnb + 4u * k + 4u) & 0x7fffffffu;
#ifdef NB_BOUNDS_CHECK
    // the node's records must lie inside the staged record region
    if (re < rs || 16u * re > a.off_gn - a.off_rec) {
      atomicCAS(a.status, 0, (int)NB_EINVAL);
      rs = re = 0;
    }
#endif
    const bool pole = (gw >> 31) != 0;
    const uint32_t h = k - n;
    const uint32_t fo = k < n ? k * a.row_bytes : hbase + (h >> 2) * a.gpitch + (h & 3u) * a.copy_bytes;
    const uint32_t col = stage + c * 16u;
    float gx[4], gy[4];
    if (!pole) {
      f2_t fi01, fi23;
      lds2x64(col + fo, fi01, fi23);
      GroupSum<COMP> ax01, ax23, ay01, ay23;
      const uint32_t pr = recb + 16u * rs;
      auto nbr = [&](uint32_t q, bool first) {
        const float4 r = lds128(pr + 16u * q);
        f2_t f01, f23;
        lds2x64(col + (uint32_t)NB_IDX(__float_as_uint(r.z), 0, a.off_rec, a.status), f01, f23);
        const f2_t a01 = sub2(f01, fi01), a23 = sub2(f23, fi23);
        const f2_t wx = pk(r.x, r.x), wy = pk(r.y, r.y);
        if (first) {
          ax01.start(wx, a01), ax23.start(wx, a23), ay01.start(wy, a01), ay23.start(wy, a23);
        } else {
          ax01.term(wx, a01), ax23.term(wx, a23), ay01.term(wy, a01), ay23.term(wy, a23);
        }
      };
      auto close = [&](int which) {
        GroupSum<COMP> *acc[4] = {&ax01, &ax23, &ay01, &ay23};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (which == 0) acc[j]->close_first();
          else if (which == 1) acc[j]->close_second();
          else acc[j]->close();
        }
      };
      const int deg = (int)(re - rs);
      if (deg == 6) {
        nbr(0, true), nbr(1, false), nbr(2, false);
        close(0);
        nbr(3, true), nbr(4, false), nbr(5, false);
        close(1);
      } else {
        int q = 0;
        for (; q + 1 < deg; q += 2) {
          nbr((uint32_t)q, true), nbr((uint32_t)q + 1, false);
          close(q == 0 ? 0 : 2);
        }
        if (q < deg) {
          nbr((uint32_t)q, true);
          close(q == 0 ? 0 : 2);
        }
      }
      upk(ax01.finish(), gx[0], gx[1]);
      upk(ax23.finish(), gx[2], gx[3]);
      upk(ay01.finish(), gy[0], gy[1]);
      upk(ay23.finish(), gy[2], gy[3]);
    } else {
      const float4 fi = lds128(col + fo);
      double sx[4] = {0, 0, 0, 0}, sy[4] = {0, 0, 0, 0};
      const float fiv[4] = {fi.x, fi.y, fi.z, fi.w};
      for (uint32_t q = rs; q < re; ++q) {
        const float4 r = lds128(recb + 16u * q);
        const double2 w = __ldg(a.wg64 + __float_as_int(r.w));
        const float4 fj = lds128(col + (uint32_t)NB_IDX(__float_as_uint(r.z), 0, a.off_rec, a.status));
        const float fjv[4] = {fj.x, fj.y, fj.z, fj.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const double d = (double)fjv[j] - (double)fiv[j];
          sx[j] = fma(w.x, d, sx[j]);
          sy[j] = fma(w.y, d, sy[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        gx[j] = (float)sx[j];
        gy[j] = (float)sy[j];
      }
    }
    // g buffer: levels 4c .. 4c + 3 as (gx, gy) pairs, 32 bytes (the pitch
    // holds all Gg units; levels past the column are never read back)
    const uint32_t go = gbuf + k * a.g_pitch + 32u * c;
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(go), "f"(gx[0]), "f"(gy[0]), "f"(gx[1]),
                 "f"(gy[1])
                 : "memory");
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(go + 16u), "f"(gx[2]), "f"(gy[2]), "f"(gx[3]),
                 "f"(gy[3])
                 : "memory");
    if (a.gout != nullptr && k < n) {
      const int l0 = 4 * (int)c;
      float *o = a.gout + (int64_t)(n0 + (int32_t)k) * a.g_stride + 2 * l0;
      if (l0 + 4 <= a.nlev) {
        __stcs(reinterpret_cast<float4 *>(o), make_float4(gx[0], gy[0], gx[1], gy[1]));
        __stcs(reinterpret_cast<float4 *>(o) + 1, make_float4(gx[2], gy[2], gx[3], gy[3]));
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (l0 + j < a.nlev) {
            o[2 * j] = gx[j];
            o[2 * j + 1] = gy[j];
          }
      }
    }
  }
}

__device__ __forceinline__ int lap_tile_at(const LapArgs &a, int i) {
  const int npole = a.ntiles - a.ntiles_main;
  return i < npole ? a.ntiles_main + i : i - npole;
}

template <bool COMP, int KU>
__global__ void __launch_bounds__(kLapThreads, 1)
    staged_lap(const LapArgs a, const __grid_constant__ CUtensorMap map) {
  constexpr int W = kLapWarps;
  extern __shared__ __align__(128) unsigned char smem[];
  const int NS = a.nstages;
  // shared memory: the stages, then the barriers (full[NS], empty[NS], g
  // written, g read), then the g buffer at off_g
  const uint32_t stage0 = smem_u32(smem);
  const uint32_t barb = stage0 + (uint32_t)NS * a.stage_bytes;
  const uint32_t fullb = barb, emptyb = barb + 8u * NS, gdone = barb + 16u * NS, ddone = gdone + 8u;
  const uint32_t gbuf = stage0 + a.off_g;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(fullb + 8 * s, 1);
      mbar_init(emptyb + 8 * s, W);
    }
    mbar_init(gdone, W);
    mbar_init(ddone, W);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int GR = gridDim.x;
  if (warp == W) {
    int k = 0;
    bool failed = false;
    LapPrep next{};
    if ((int)blockIdx.x < a.ntiles) next = prepare_lap_tile(a, lap_tile_at(a, blockIdx.x), lane);
    for (int i = blockIdx.x; i < a.ntiles; i += GR, ++k) {
      const LapPrep cur = next;
      if (i + GR < a.ntiles) next = prepare_lap_tile(a, lap_tile_at(a, i + GR), lane);
      const int s = k % NS;
      if (k >= NS && !mbar_wait_bounded(emptyb + 8 * s, (uint32_t)(k / NS - 1) & 1u, a.timeout_ns)) {
        failed = true;
        break;
      }
      issue_lap_tile(a, &map, cur, stage0 + s * a.stage_bytes, fullb + 8 * s, lane);
      if (lane == 0 && i + GR < a.ntiles) {
        const int tp = lap_tile_at(a, i + GR);
        const int32_t p0 = __ldg(a.tile_node0 + tp), p1 = __ldg(a.tile_node0 + tp + 1);
        bulk_prefetch_l2(a.in + (int64_t)p0 * a.in_stride * 4, (uint32_t)(p1 - p0 - 1) * a.row_bytes + a.copy_bytes);
      }
    }
    if (failed) {
      if (lane == 0) atomicCAS(a.status, 0, (int)NB_ETIMEOUT);
      for (int j = (k >= NS ? k - NS : 0); j < k; ++j)
        if (!mbar_wait_bounded(fullb + 8 * (j % NS), (uint32_t)(j / NS) & 1u, kDrainLimitNs)) break;
    }
    return;
  }
  int k = 0;
  for (int i = blockIdx.x; i < a.ntiles; i += GR, ++k) {
    const int t = lap_tile_at(a, i);
    const int s = k % NS;
    const uint32_t stage = stage0 + (uint32_t)s * a.stage_bytes;
    bool ok = mbar_wait_bounded(fullb + 8 * s, (uint32_t)(k / NS) & 1u, a.timeout_ns);
    // every warp has read the previous tile's g buffer
    if (ok && k > 0) ok = mbar_wait_bounded(ddone, (uint32_t)(k - 1) & 1u, a.timeout_ns);
    if (!ok) {
      if (lane == 0) atomicCAS(a.status, 0, (int)NB_ETIMEOUT);
      break;
    }
    const int32_t n0 = lds_s32(stage + a.off_h), n1 = lds_s32(stage + a.off_h + 4u);
    const uint32_t H1 = (uint32_t)lds_s32(stage + a.off_h + 8u);
    const int32_t g0 = lds_s32(stage + a.off_h + 12u);
    lap_grad_phase<COMP>(a, stage, gbuf, n0, (uint32_t)(n1 - n0), H1, g0, warp, W);
    __syncwarp();
    if (lane == 0) mbar_arrive(gdone);
    if (!mbar_wait_bounded(gdone, (uint32_t)k & 1u, a.timeout_ns)) {
      if (lane == 0) atomicCAS(a.status, 0, (int)NB_ETIMEOUT);
      break;
    }
    TileView v;
    v.n0 = n0;
    v.n1 = n1;
    v.rows = gbuf;
    v.r = stage + a.off_rp - 4u * (uint32_t)(n0 & ~3);
    const int32_t pa = lds_s32(v.r + 4u * (uint32_t)n0);
    v.w = stage + a.off_wd - 8u * (uint32_t)(pa & ~1);
    v.l = stage + a.off_go - 4u * (uint32_t)(pa & ~3);
    v.s = stage + a.off_sd - 8u * (uint32_t)(n0 & ~1);
    v.p = 0u;  // every node alone
    v.npairs = 0;
    divcurl_tile<COMP, false, KU, false, 0>(a, v, t >= a.ntiles_main, a.g_pitch, warp, W);
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(emptyb + 8 * s);
      mbar_arrive(ddone);
    }
  }
}

// ------------------------------------------------------------------ host

// Byte sizes of the parts of a stage and of the g buffer.
struct LapSizes {
  int Gg = 0;  // 4-level units of a column
  int64_t rec = 0, gn = 0, wd = 0, go = 0, rp = 0, sd = 0, hdr = 0, stage = 0, gbytes = 0;
};

// Layout of the fused kernel's shared memory for one column shape: two
// stages (f columns and metadata) and the g buffer, within 227 KB.
static LapLayout lap_layout(int nlev, int64_t row_bytes, int nmax, LapSizes &z) {
  LapLayout L;
  L.row_bytes = row_bytes;
  L.copy_bytes = ((int64_t)nlev * 4 + 15) / 16 * 16;
  L.gpitch = (4 * L.copy_bytes + 127) / 128 * 128;
  z.Gg = (nlev + 3) / 4;
  L.g_pitch = 32 * (int64_t)z.Gg;
  const int64_t total = 227 * 1024;
  const int64_t bars = 64;  // full[2], empty[2], g written, g read
  // g buffer for ~72 KB of g-nodes (at most 2.5 nmax: an own node brings
  // ~1.2 ring-1 nodes in the tiles of 137-level columns), the rest split
  // into two stages
  L.gcap = std::max<int64_t>(8, std::min<int64_t>((72 * 1024) / L.g_pitch, 5 * (int64_t)nmax / 2));
  const int64_t gbytes = L.gcap * L.g_pitch;
  const int64_t stage = ((total - bars - gbytes) / 2) / 128 * 128;
  L.nmax = nmax;
  L.ecap = 7 * (int64_t)nmax + 16;
  L.rcap = 7 * L.gcap + 16;
  auto up16 = [](int64_t x) { return (x + 15) / 16 * 16; };
  z.rec = up16(16 * L.rcap);
  z.gn = up16(4 * (L.gcap + 8));
  z.wd = up16(8 * (L.ecap + 2));
  z.go = up16(4 * (L.ecap + 8));
  z.rp = up16(4 * (nmax + 8));
  z.sd = up16(8 * (nmax + 2));
  z.hdr = 16;
  const int64_t meta = z.rec + z.gn + z.wd + z.go + z.rp + z.sd + z.hdr;
  L.farea = (stage - meta) / 128 * 128;
  z.stage = stage;
  z.gbytes = gbytes;
  return L;
}

__global__ void lap_records_kernel(int64_t n, const int32_t *__restrict__ p, const uint32_t *__restrict__ foff,
                                   const float2 *__restrict__ wg32, float4 *__restrict__ rec) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t q = p[i];
  const float2 w = wg32[q];
  rec[i] = make_float4(w.x, w.y, __uint_as_float(foff[i]), __int_as_float(q));
}

// Structural check of a single-pass Laplacian plan before it is used: the
// tiles, their rings and the own nodes' g-buffer offsets (each must decode to
// the g slot of its neighbour).
static bool check_lap_plan(const nb_mesh *mesh, const LapLayout &L, const LapPlanHost &h, std::string &why) {
  const int64_t gp = L.g_pitch;
  auto slot = [&](int64_t p, int t, int64_t n) -> int64_t {
    const int64_t off = h.goff[p];
    return (off % gp == 0 && off / gp < n + h.r1_count[t]) ? off / gp : -1;
  };
  return check_tile_plan(mesh, (int)h.node0.size() - 1, h.node0.data(), h.halo_ptr.data(), h.halo.data(), slot,
                         why);
}

static int lap_plan_upload(LapPlan *lp, nb_method *m, const LapLayout &L, int nmax, int pole_cap) {
  LapPlanHost h;
  build_lap_plan(m->mesh, L, nmax, pole_cap, h);
  if (!h.fits) {
    set_error("fused Laplacian: a tile of the plan does not fit its shared-memory layout");
    return NB_EINVAL;
  }
  {
    std::string why;
    if (!check_lap_plan(m->mesh, L, h, why)) {
      set_error("fused Laplacian: invalid tile plan (" + why + ")");
      return NB_EINVAL;
    }
  }
  lp->ntiles = (int)h.node0.size() - 1;
  log_msg(1, "single-pass Laplacian plan: %d tiles (%d pole-row), at most %d g-nodes and %d records a tile, "
          "%zu ring columns in all", lp->ntiles, lp->ntiles - h.ntiles_main, h.max_gnodes, h.max_recs,
          h.halo.size());
  lp->ntiles_main = h.ntiles_main;
  lp->max_gnodes = h.max_gnodes;
  h.gn.resize(h.gn.size() + 8, 0);        // slack for 16-byte bounding copies
  h.goff.resize(h.goff.size() + 8, 0);
  if (h.halo.empty()) h.halo.push_back(0);
  auto up = [&](void **dst, const void *src, size_t bytes) -> int {
    const size_t nb = std::max<size_t>(bytes, 16);
    const int st = dev_alloc(m->alloc, dst, nb, "Laplacian tile plan upload");
    if (st != NB_OK) return st;
    m->blocks.push_back({*dst, nb});
    if (bytes && src) NB_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    lp->bytes += (int64_t)bytes;
    return NB_OK;
  };
  int st;
  if ((st = up((void **)&lp->d_tile_node0, h.node0.data(), h.node0.size() * 4))) return st;
  if ((st = up((void **)&lp->d_halo_ptr, h.halo_ptr.data(), h.halo_ptr.size() * 4))) return st;
  if ((st = up((void **)&lp->d_halo, h.halo.data(), h.halo.size() * 4))) return st;
  if ((st = up((void **)&lp->d_r1_count, h.r1_count.data(), h.r1_count.size() * 4))) return st;
  if ((st = up((void **)&lp->d_gn_ptr, h.gn_ptr.data(), h.gn_ptr.size() * 4))) return st;
  if ((st = up((void **)&lp->d_gn, h.gn.data(), h.gn.size() * 4))) return st;
  if ((st = up((void **)&lp->d_rec_ptr, h.rec_ptr.data(), h.rec_ptr.size() * 4))) return st;
  if ((st = up((void **)&lp->d_goff, h.goff.data(), h.goff.size() * 4))) return st;
  const int64_t nrec = (int64_t)h.rec_p.size();
  if ((st = up((void **)&lp->d_rec, nullptr, (size_t)std::max<int64_t>(nrec, 1) * 16))) return st;
  if (nrec > 0) {
    // records: the FP32 gradient weights of each entry, gathered on the device
    void *dp = nullptr, *df = nullptr;
    if ((st = dev_alloc(m->alloc, &dp, (size_t)nrec * 4, "Laplacian plan records"))) return st;
    if ((st = dev_alloc(m->alloc, &df, (size_t)nrec * 4, "Laplacian plan records"))) {
      dev_free(m->alloc, dp, (size_t)nrec * 4);
      return st;
    }
    cudaError_t e = cudaMemcpy(dp, h.rec_p.data(), (size_t)nrec * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(df, h.rec_foff.data(), (size_t)nrec * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      lap_records_kernel<<<(unsigned)((nrec + 255) / 256), 256>>>(
          nrec, static_cast<const int32_t *>(dp), static_cast<const uint32_t *>(df),
          reinterpret_cast<const float2 *>(m->d_wgrad32), static_cast<float4 *>(lp->d_rec));
      count_launch(1);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    dev_free(m->alloc, dp, (size_t)nrec * 4);
    dev_free(m->alloc, df, (size_t)nrec * 4);
    NB_CUDA(e);
  }
  return NB_OK;
}

static LapPlan *get_lap_plan(nb_method *m, const LapLayout &L, int nmax, int pole_cap, int *status) {
  std::lock_guard<std::mutex> lk(m->plan_mu);
  const auto key = std::make_tuple(L.row_bytes, L.copy_bytes, L.g_pitch, L.farea, L.gcap, nmax, pole_cap);
  auto it = m->lap_plans.find(key);
  if (it != m->lap_plans.end()) return it->second.get();
  auto lp = std::make_unique<LapPlan>();
  *status = lap_plan_upload(lp.get(), m, L, nmax, pole_cap);
  if (*status != NB_OK) return nullptr;
  LapPlan *raw = lp.get();
  m->lap_plans[key] = std::move(lp);
  return raw;
}

template <bool COMP, int KU>
static int launch_lap_t(const LapArgs &a, const CUtensorMap &map, int grid, size_t smem, cudaStream_t st) {
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [&] {
    attr_err = cudaFuncSetAttribute(staged_lap<COMP, KU>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  NB_CUDA(attr_err);
  staged_lap<COMP, KU><<<grid, kLapThreads, smem, st>>>(a, map);
  count_launch(1);
  NB_CUDA(cudaGetLastError());
  return NB_OK;
}

// Single-pass Laplacian of f into lap (and f's gradient into g when g is
// not NULL).  *handled = false when the field's shape is not one this
// kernel takes (FP64, unaligned, fewer than 16 levels): the caller then
// uses the two-pass route.
int launch_fused_lap(nb_method *m, const nb_field *f, const nb_field *lap, const nb_field *g, cudaStream_t st,
                     bool *handled) {
  *handled = false;
  if (f->dtype != NB_F32 || f->nvar != 1) return NB_OK;
  const uintptr_t bits = (uintptr_t)f->data | (uintptr_t)lap->data | (g ? (uintptr_t)g->data : 0u);
  if ((bits & 15u) != 0 || f->node_stride % 4 != 0 || lap->node_stride % 4 != 0 ||
      (g && g->node_stride % 4 != 0) || f->nlev < 16)
    return NB_OK;
  if (encode_fn() == nullptr) return NB_OK;
  const uint32_t copy_elems = (uint32_t)(((int64_t)f->nlev * 4 + 15) / 16 * 4);
  if (copy_elems > 256u) return NB_OK;  // a tensor box row holds at most 256 elements
  const int nmax = 64;
  LapSizes z;
  const LapLayout L = lap_layout(f->nlev, f->node_stride * 4, nmax, z);
  if (L.farea < 16 * L.row_bytes || L.gcap < 16) return NB_OK;
  int sms = 0;
  if (const int rc = sm_count(&sms)) return rc;
  const int64_t npole = m->mesh->V - m->mesh->cap_begin;
  const int pole_cap = (int)std::max<int64_t>(1, (npole + sms - 1) / std::max(1, sms));
  int status = NB_OK;
  LapPlan *lp = get_lap_plan(m, L, nmax, pole_cap, &status);
  if (!lp) return status;
  CUtensorMap map;
  const cuuint64_t gdim[2] = {copy_elems, (cuuint64_t)f->nnodes};
  const cuuint64_t gstride[1] = {(cuuint64_t)(f->node_stride * 4)};
  const cuuint32_t box[2] = {copy_elems, 1};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult cr = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(f->data), gdim,
                                  gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) {
    set_error("fused Laplacian: cuTensorMapEncodeTiled failed (" + std::to_string((int)cr) + ")");
    return NB_ECUDA;
  }
  LapArgs a{};
  a.ntiles = lp->ntiles;
  a.ntiles_main = lp->ntiles_main;
  a.tile_node0 = lp->d_tile_node0;
  a.halo_ptr = lp->d_halo_ptr;
  a.halo = lp->d_halo;
  a.r1_count = lp->d_r1_count;
  a.gn_ptr = lp->d_gn_ptr;
  a.rec_ptr = lp->d_rec_ptr;
  a.gn = lp->d_gn;
  a.rec = static_cast<const float4 *>(lp->d_rec);
  a.goff = lp->d_goff;
  a.row_ptr = m->d_row_ptr;
  a.wd32 = reinterpret_cast<const float2 *>(m->d_wdiv32);
  a.sd32 = reinterpret_cast<const float2 *>(m->d_sdiv32);
  a.wg64 = reinterpret_cast<const double2 *>(m->d_wgrad64);
  a.w64 = reinterpret_cast<const double2 *>(m->d_wdiv64);
  a.s64 = reinterpret_cast<const double2 *>(m->d_sdiv64);
  a.w64b = nullptr;
  a.s64b = nullptr;
  a.out = static_cast<float *>(lap->data);
  a.out2 = nullptr;
  a.out_stride = lap->node_stride;
  a.nlev = f->nlev;
  int KU = 2, G = 0;
  item_shape(m->item_units, m->item_align, (f->nlev + 1) / 2, KU, G);
  a.G = G;
  a.g_magic32 = magic32((uint32_t)G);
  a.Gg = z.Gg;
  magic_div((uint32_t)z.Gg, a.gg_magic, a.gg_shift);
  a.gout = g ? static_cast<float *>(g->data) : nullptr;
  a.g_stride = g ? g->node_stride : 0;
  a.in = static_cast<const char *>(f->data);
  a.row_bytes = (uint32_t)L.row_bytes;
  a.in_stride = f->node_stride;
  a.copy_bytes = (uint32_t)L.copy_bytes;
  a.gpitch = (uint32_t)L.gpitch;
  a.g_pitch = (uint32_t)L.g_pitch;
  a.off_rec = (uint32_t)L.farea;
  a.off_gn = a.off_rec + (uint32_t)z.rec;
  a.off_wd = a.off_gn + (uint32_t)z.gn;
  a.off_go = a.off_wd + (uint32_t)z.wd;
  a.off_rp = a.off_go + (uint32_t)z.go;
  a.off_sd = a.off_rp + (uint32_t)z.rp;
  a.off_h = a.off_sd + (uint32_t)z.sd;
  a.stage_bytes = (uint32_t)z.stage;
  a.nstages = 2;
  a.off_g = 2u * a.stage_bytes + 64u;  // the g buffer after the stages and the barriers
  if (a.off_h + 16u > a.stage_bytes) {
    set_error("fused Laplacian: stage layout does not fit");
    return NB_EINVAL;
  }
  a.status = nullptr;
  if (const int rc = status_word(&a.status)) return rc;
  a.timeout_ns = m->wait_limit_ns >= 0 ? (uint64_t)m->wait_limit_ns : kDefaultWaitNs;
  a.nnodes = (int32_t)f->nnodes;
  a.col_area = (uint32_t)z.gbytes;
  const size_t smem = (size_t)a.off_g + (size_t)z.gbytes;
  if (smem > 227 * 1024) {
    set_error("fused Laplacian: shared memory layout exceeds 227 KB");
    return NB_EINVAL;
  }
  const int grid = std::min(lp->ntiles, sms);
  log_msg(2, "single-pass Laplacian launch: %d levels, %d tiles, grid %d, %zu B shared%s", f->nlev, lp->ntiles,
          grid, smem, g ? ", gradient written" : "");
  *handled = true;
  const bool comp = m->compensated != 0;
  if (KU == 3) return comp ? launch_lap_t<true, 3>(a, map, grid, smem, st) : launch_lap_t<false, 3>(a, map, grid, smem, st);
  return comp ? launch_lap_t<true, 2>(a, map, grid, smem, st) : launch_lap_t<false, 2>(a, map, grid, smem, st);
}

// Host-side plan statistics (tests): the plan the fused kernel would use
// for FP32 columns of nlev levels at the functionspace's padded stride.
int lap_plan_info(const nb_mesh *mesh, int nlev, int32_t *ntiles, int32_t *ntiles_main, int32_t *max_gnodes,
                  int32_t *fits) {
  const int64_t lp = ((int64_t)nlev + 3) / 4 * 4;
  LapSizes z;
  const LapLayout L = lap_layout(nlev, 4 * lp, 64, z);
  LapPlanHost h;
  build_lap_plan(mesh, L, 64, 1, h);
  *ntiles = (int32_t)h.node0.size() - 1;
  *ntiles_main = h.ntiles_main;
  *max_gnodes = h.max_gnodes;
  std::string why;
  *fits = (h.fits && check_lap_plan(mesh, L, h, why)) ? 1 : 0;
  return NB_OK;
}

}  // namespace nb
