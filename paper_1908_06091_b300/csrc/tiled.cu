// tiled.cu -- shared-memory staged nabla kernels for sm_103a.
//
// A persistent grid walks the tiles of a TilePlan (consecutive Hilbert-
// ordered nodes whose own columns plus halo columns fit one stage).  For
// each tile one warp issues 1-D TMA bulk copies (cp.async.bulk) of the
// tile's contiguous column block and of every halo column into a
// shared-memory stage, completing on an mbarrier; two stages alternate, so
// the copies of tile k+1 run under the arithmetic of tile k.  Threads then
// take (node, 4-level group) items: the node's own column and its
// neighbours' columns are read from shared memory with 16-byte loads, the
// edge weights through L1, and the per-node gather is accumulated with
// packed FP32x2 Kahan arithmetic.  Pole tiles (the first and last grid
// rows) are evaluated in FP64.  Every mbarrier wait is bounded: on timeout
// the kernel records NB_ETIMEOUT in a device status word, waits (bounded)
// for its own copies and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>

#include "kernels_common.cuh"

namespace nb {

// device status word: 0 = ok, otherwise an NB_* code (first error wins)
__device__ int g_device_status = 0;

int launch_tiled(nb_method *m, int op, const nb_field *in, const nb_field *out, cudaStream_t st,
                 bool *handled);

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
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for `parity` on the barrier for at most ~`limit_ns`; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
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
// negated running correction, so each term w * d costs one fma2 and three
// add/sub2: y = w*d + nc; t = s + y; nc = y - (t - s); s = t.
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
  __device__ __forceinline__ f2_t value() const { return COMP ? add2(s, nc) : s; }
};

// ------------------------------------------------------------- kernel

struct TiledArgs {
  int ntiles, ntiles_main;
  const int32_t *tile_node0;
  const int32_t *halo_ptr;
  const int32_t *halo;
  const uint16_t *hrun;
  const int32_t *nruns;
  const uint16_t *lnbr;
  const int32_t *row_ptr;
  const float2 *w32;
  const double2 *w64;
  const float2 *s32;
  const double2 *s64;
  const char *in;
  uint32_t row_bytes;  // bytes of one staged column (in_stride * 4)
  int64_t in_stride;   // elements
  float *out;
  int64_t out_stride;  // elements
  int nlev;
  int G;               // items per node (4 levels each)
  uint64_t g_magic;    // item / G == (item * g_magic) >> g_shift, exact for items < 2^24
  uint32_t g_shift;
  uint32_t copy_bytes; // bytes copied per column: the real data rounded up to 16
  uint32_t off_w, off_l, off_r;  // stage offsets of the staged weights, rows, row pointers
  uint32_t stage_bytes;
  int nstages;
  int *status;
  uint64_t timeout_ns;
};

// Issue the copies of tile t into the stage at `stage` (one whole warp): the
// tile's contiguous column block, its halo columns (one bulk copy per run of
// consecutive node ids), and 16-byte aligned bounding ranges of the tile's
// CSR weights, staged-row indices and row pointers, all as TMA bulk copies
// completing on the stage's "full" barrier.  The copy engine's cost is per
// copy rather than per byte, so copies are kept few and large.
__device__ __forceinline__ void issue_tile(const TiledArgs &a, int t, uint32_t stage, uint32_t bar,
                                           int lane) {
  const int32_t n0 = __ldg(a.tile_node0 + t), n1 = __ldg(a.tile_node0 + t + 1);
  const int32_t h0 = __ldg(a.halo_ptr + t), h1 = __ldg(a.halo_ptr + t + 1);
  const int32_t pa = __ldg(a.row_ptr + n0), pb = __ldg(a.row_ptr + n1);
  const uint32_t n = (uint32_t)(n1 - n0), H = (uint32_t)(h1 - h0);
  const int32_t wa = pa & ~1, wb = (pb + 1) & ~1;
  const int32_t la = pa & ~7, lb = (pb + 7) & ~7;
  const int32_t ra = n0 & ~3, rb = (n1 + 4) & ~3;
  const uint32_t body = (n - 1) * a.row_bytes + a.copy_bytes;
  const uint32_t wbytes = (uint32_t)(wb - wa) * 8u, lbytes = (uint32_t)(lb - la) * 2u,
                 rbytes = (uint32_t)(rb - ra) * 4u;
  // a run of L halo columns is one copy of (L - 1) full columns + one column
  const uint32_t runs = (uint32_t)__ldg(a.nruns + t);
  const uint32_t hbytes = H * a.copy_bytes + (H - runs) * (a.row_bytes - a.copy_bytes);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (lane == 0) mbar_expect_tx(bar, body + hbytes + wbytes + lbytes + rbytes);
  __syncwarp();
  if (lane == 0) bulk_g2s(stage, a.in + (int64_t)n0 * a.in_stride * 4, body, bar);
  if (lane == 1) bulk_g2s(stage + a.off_w, a.w32 + wa, wbytes, bar);
  if (lane == 2) bulk_g2s(stage + a.off_l, a.lnbr + la, lbytes, bar);
  if (lane == 3) bulk_g2s(stage + a.off_r, a.row_ptr + ra, rbytes, bar);
  for (uint32_t h = lane; h < H; h += 32) {
    const uint32_t L = __ldg(a.hrun + h0 + h);
    if (L == 0) continue;
    const int32_t node = __ldg(a.halo + h0 + h);
    bulk_g2s(stage + (n + h) * a.row_bytes, a.in + (int64_t)node * a.in_stride * 4,
             (L - 1) * a.row_bytes + a.copy_bytes, bar);
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
__device__ __forceinline__ uint32_t lds_u16(uint32_t a) {
  uint16_t v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ int32_t lds_s32(uint32_t a) {
  int32_t v;
  asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}

// 32-bit shared addresses of one staged tile: entry p's weight is at
// w + 8 p, its staged-row index at l + 2 p, node i's row pointer at r + 4 i
// (wrap-around arithmetic; the sums land inside the stage).
struct TileView {
  int32_t n0, n1;
  uint32_t rows, w, l, r;
  __device__ __forceinline__ TileView(const TiledArgs &a, int t, uint32_t stage) {
    n0 = __ldg(a.tile_node0 + t);
    n1 = __ldg(a.tile_node0 + t + 1);
    rows = stage;
    const int32_t ra = n0 & ~3;
    r = stage + a.off_r - 4u * (uint32_t)ra;
    const int32_t pa = lds_s32(r + 4u * (uint32_t)n0);
    w = stage + a.off_w - 8u * (uint32_t)(pa & ~1);
    l = stage + a.off_l - 2u * (uint32_t)(pa & ~7);
  }
};

// Items [i0, i1) of tile t for the calling warp, one per lane, stride 32.
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
    const float4 fi = lds128(col + il * rb);
    float gx[4], gy[4];
    if (!pole) {
      const f2_t fi01 = pk(fi.x, fi.y), fi23 = pk(fi.z, fi.w);
      Kahan2<COMP> ax01, ax23, ay01, ay23;
      auto body = [&](const float2 w, const float4 fj) {
        const f2_t d01 = sub2(pk(fj.x, fj.y), fi01), d23 = sub2(pk(fj.z, fj.w), fi23);
        const f2_t wx = pk(w.x, w.x), wy = pk(w.y, w.y);
        ax01.add_prod(wx, d01);
        ax23.add_prod(wx, d23);
        ay01.add_prod(wy, d01);
        ay23.add_prod(wy, d23);
      };
      uint32_t pw = v.w + 8u * (uint32_t)p0, pl = v.l + 2u * (uint32_t)p0;
      int32_t p = p0;
      for (; p + 1 < p1; p += 2, pw += 16u, pl += 4u) {
        const float2 w0 = lds64(pw), w1 = lds64(pw + 8u);
        const uint32_t r0 = lds_u16(pl), r1 = lds_u16(pl + 2u);
        const float4 f0 = lds128(col + r0 * rb);
        const float4 f1 = lds128(col + r1 * rb);
        body(w0, f0);
        body(w1, f1);
      }
      if (p < p1) body(lds64(pw), lds128(col + lds_u16(pl) * rb));
      upk(ax01.value(), gx[0], gx[1]);
      upk(ax23.value(), gx[2], gx[3]);
      upk(ay01.value(), gy[0], gy[1]);
      upk(ay23.value(), gy[2], gy[3]);
    } else {
      double sx[4] = {0, 0, 0, 0}, sy[4] = {0, 0, 0, 0};
      const float fiv[4] = {fi.x, fi.y, fi.z, fi.w};
      for (int32_t p = p0; p < p1; ++p) {
        const double2 w = __ldg(a.w64 + p);
        const float4 fj = lds128(col + lds_u16(v.l + 2u * (uint32_t)p) * rb);
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

// div / curl.  A staged (u, v) column is a sequence of 16-byte units of two
// levels each; item c of a node takes units c and c + G, so that every
// shared-memory load of a warp reads consecutive 16-byte words.
template <bool COMP>
__device__ __forceinline__ void divcurl_tile(const TiledArgs &a, int t, uint32_t stage, int part,
                                             int nparts) {
  const TileView v(a, t, stage);
  const uint32_t items = (uint32_t)(v.n1 - v.n0) * a.G;
  const uint32_t i0 = (uint32_t)(((uint64_t)items * part) / nparts);
  const uint32_t i1 = (uint32_t)(((uint64_t)items * (part + 1)) / nparts);
  const bool pole = t >= a.ntiles_main;
  const int units = (a.nlev + 1) / 2;
  const uint32_t rb = a.row_bytes;
  for (uint32_t item = i0 + (threadIdx.x & 31); item < i1; item += 32) {
    const uint32_t il = (uint32_t)(((uint64_t)item * a.g_magic) >> a.g_shift);
    const uint32_t c = item - il * a.G;
    const int u0 = (int)c, u1 = (int)c + a.G;
    const bool has1 = u1 < units;
    const int32_t node = v.n0 + (int32_t)il;
    const int32_t p0 = lds_s32(v.r + 4u * (uint32_t)node), p1 = lds_s32(v.r + 4u * (uint32_t)node + 4u);
    const uint32_t colA = v.rows + (uint32_t)u0 * 16u;
    const uint32_t colB = v.rows + (uint32_t)(has1 ? u1 : u0) * 16u;
    const float4 A = lds128(colA + il * rb);
    const float4 B = lds128(colB + il * rb);
    float r[4];
    if (!pole) {
      // pair accumulators (sum of w.x du, sum of w.y dv) per level
      const f2_t i0p = pk(A.x, A.y), i1p = pk(A.z, A.w), i2p = pk(B.x, B.y), i3p = pk(B.z, B.w);
      Kahan2<COMP> k0, k1, k2, k3;
      auto body = [&](const float2 w, const float4 C, const float4 D) {
        const f2_t w2 = pk(w.x, w.y);
        k0.add_prod(w2, sub2(pk(C.x, C.y), i0p));
        k1.add_prod(w2, sub2(pk(C.z, C.w), i1p));
        k2.add_prod(w2, sub2(pk(D.x, D.y), i2p));
        k3.add_prod(w2, sub2(pk(D.z, D.w), i3p));
      };
      uint32_t pw = v.w + 8u * (uint32_t)p0, pl = v.l + 2u * (uint32_t)p0;
      int32_t p = p0;
      for (; p + 1 < p1; p += 2, pw += 16u, pl += 4u) {
        const float2 w0 = lds64(pw), w1 = lds64(pw + 8u);
        const uint32_t r0 = lds_u16(pl) * rb, r1 = lds_u16(pl + 2u) * rb;
        const float4 C0 = lds128(colA + r0), D0 = lds128(colB + r0);
        const float4 C1 = lds128(colA + r1), D1 = lds128(colB + r1);
        body(w0, C0, D0);
        body(w1, C1, D1);
      }
      if (p < p1) {
        const uint32_t r0 = lds_u16(pl) * rb;
        body(lds64(pw), lds128(colA + r0), lds128(colB + r0));
      }
      const float2 sw = __ldg(a.s32 + node);
      const f2_t sw2 = pk(sw.x, sw.y);
      const f2_t vals[4] = {k0.value(), k1.value(), k2.value(), k3.value()};
      const f2_t self[4] = {i0p, i1p, i2p, i3p};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const f2_t q = fma2(sw2, self[k], vals[k]);
        float x, y;
        upk(q, x, y);
        r[k] = __fadd_rn(x, y);
      }
    } else {
      const float iu[4] = {A.x, A.z, B.x, B.z}, iv[4] = {A.y, A.w, B.y, B.w};
      double sacc[4] = {0, 0, 0, 0};
      for (int32_t p = p0; p < p1; ++p) {
        const double2 w = __ldg(a.w64 + p);
        const uint32_t r0 = lds_u16(v.l + 2u * (uint32_t)p) * rb;
        const float4 C = lds128(colA + r0);
        const float4 D = lds128(colB + r0);
        const float ju[4] = {C.x, C.z, D.x, D.z}, jv[4] = {C.y, C.w, D.y, D.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          sacc[k] = fma(w.x, (double)ju[k] - (double)iu[k], sacc[k]);
          sacc[k] = fma(w.y, (double)jv[k] - (double)iv[k], sacc[k]);
        }
      }
      const double2 sw = __ldg(a.s64 + node);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        sacc[k] = fma(sw.x, (double)iu[k], sacc[k]);
        sacc[k] = fma(sw.y, (double)iv[k], sacc[k]);
        r[k] = (float)sacc[k];
      }
    }
    // levels 2 u0, 2 u0 + 1 from r[0..1], levels 2 u1, 2 u1 + 1 from r[2..3]
    float *oo = a.out + (int64_t)node * a.out_stride;
    const int la0 = 2 * u0, la1 = 2 * u1;
    if (la0 + 1 < a.nlev) __stcs(reinterpret_cast<float2 *>(oo + la0), make_float2(r[0], r[1]));
    else oo[la0] = r[0];
    if (has1) {
      if (la1 + 1 < a.nlev) __stcs(reinterpret_cast<float2 *>(oo + la1), make_float2(r[2], r[3]));
      else oo[la1] = r[2];
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

constexpr int kConsumerWarps = 16;
constexpr int kStagedThreads = 32 * (kConsumerWarps + 1);

// Warp-specialised pipeline.  Warp kConsumerWarps is the producer: for
// iteration k it waits until stage k % NS has been released by every
// consumer warp ("empty" barrier), then issues the copies of tile
// blockIdx.x + k * gridDim.x into it ("full" barrier, transaction count).
// Each consumer warp waits for "full", computes its 1/16 share of the
// tile's items and releases the stage; no block-wide barrier is used.
template <int OP, bool COMP>
__global__ void __launch_bounds__(kStagedThreads, 1) staged_f32(TiledArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int NS = a.nstages;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)NS * a.stage_bytes);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8u * NS;
  const uint32_t stage0 = smem_u32(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int G = gridDim.x;
  if (warp == kConsumerWarps) {
    // producer
    int k = 0;
    bool failed = false;
    for (int t = blockIdx.x; t < a.ntiles; t += G, ++k) {
      const int s = k % NS;
      if (k >= NS && !mbar_wait_bounded(empty0 + 8 * s, (uint32_t)(k / NS - 1) & 1u, a.timeout_ns)) {
        failed = true;
        break;
      }
      issue_tile(a, t, stage0 + s * a.stage_bytes, full0 + 8 * s, lane);
    }
    if (failed) {
      if (lane == 0) atomicCAS(a.status, 0, (int)NB_ETIMEOUT);
      // copies already issued (iterations k-NS .. k-1) land before exit (bounded)
      for (int j = (k >= NS ? k - NS : 0); j < k; ++j)
        if (!mbar_wait_bounded(full0 + 8 * (j % NS), (uint32_t)(j / NS) & 1u, a.timeout_ns)) break;
    }
    return;
  }
  // consumers
  int k = 0;
  for (int t = blockIdx.x; t < a.ntiles; t += G, ++k) {
    const int s = k % NS;
    if (!mbar_wait_bounded(full0 + 8 * s, (uint32_t)(k / NS) & 1u, a.timeout_ns)) {
      if (lane == 0) atomicCAS(a.status, 0, (int)NB_ETIMEOUT);
      break;
    }
    const uint32_t rows = stage0 + (uint32_t)s * a.stage_bytes;
    if (OP == 0) grad_tile<COMP>(a, t, rows, warp, kConsumerWarps);
    else divcurl_tile<COMP>(a, t, rows, warp, kConsumerWarps);
    __syncwarp();
    if (lane == 0) mbar_arrive(empty0 + 8 * s);
  }
}

// --------------------------------------------------------------- host

static int plan_upload(TilePlan *tp, const nb_mesh *mesh) {
  std::vector<int32_t> node0, hptr, halo;
  std::vector<uint16_t> lnbr;
  build_tile_plan_host(mesh, tp->rcap, tp->nmax, tp->ecap, node0, hptr, halo, lnbr, tp->max_halo,
                       tp->max_entries, tp->ntiles_main);
  lnbr.resize(lnbr.size() + 16, 0);  // slack for 16-byte bounding copies
  tp->ntiles = (int)node0.size() - 1;
  auto up = [&](void **dst, const void *src, size_t bytes) -> int {
    NB_CUDA(cudaMalloc(dst, std::max<size_t>(bytes, 16)));
    if (bytes) NB_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    tp->bytes += (int64_t)bytes;
    return NB_OK;
  };
  int st;
  if ((st = up((void **)&tp->d_tile_node0, node0.data(), node0.size() * 4))) return st;
  if ((st = up((void **)&tp->d_halo_ptr, hptr.data(), hptr.size() * 4))) return st;
  if ((st = up((void **)&tp->d_halo, halo.data(), halo.size() * 4))) return st;
  if ((st = up((void **)&tp->d_lnbr, lnbr.data(), lnbr.size() * 2))) return st;
  // runs of consecutive node ids inside each tile's sorted halo
  std::vector<uint16_t> hrun(halo.size(), 0);
  std::vector<int32_t> nruns(tp->ntiles, 0);
  for (int t = 0; t < tp->ntiles; ++t) {
    int32_t i = hptr[t];
    while (i < hptr[t + 1]) {
      int32_t j = i + 1;
      while (j < hptr[t + 1] && halo[j] == halo[j - 1] + 1 && j - i < 65535) ++j;
      hrun[i] = (uint16_t)(j - i);
      ++nruns[t];
      i = j;
    }
  }
  if ((st = up((void **)&tp->d_hrun, hrun.data(), hrun.size() * 2))) return st;
  if ((st = up((void **)&tp->d_nruns, nruns.data(), nruns.size() * 4))) return st;
  return NB_OK;
}

static TilePlan *get_plan(nb_method *m, int rcap, int nmax, int ecap, int *status) {
  std::lock_guard<std::mutex> lk(m->plan_mu);
  auto key = std::make_tuple(rcap, nmax, ecap);
  auto it = m->plans.find(key);
  if (it != m->plans.end()) return it->second.get();
  auto tp = std::make_unique<TilePlan>();
  tp->rcap = rcap;
  tp->nmax = nmax;
  tp->ecap = ecap;
  *status = plan_upload(tp.get(), m->mesh);
  if (*status != NB_OK) return nullptr;
  TilePlan *raw = tp.get();
  m->plans[key] = std::move(tp);
  return raw;
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
static int launch_staged_t(const TiledArgs &a, int grid, size_t smem, cudaStream_t st) {
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [&] {
    attr_err = cudaFuncSetAttribute(staged_f32<OP, COMP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    227 * 1024);
  });
  NB_CUDA(attr_err);
  staged_f32<OP, COMP><<<grid, kStagedThreads, smem, st>>>(a);
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

int launch_tiled(nb_method *m, int op, const nb_field *in, const nb_field *out, cudaStream_t st,
                 bool *handled) {
  *handled = false;
  if (in->dtype != NB_F32) return NB_OK;
  const bool aligned = (((uintptr_t)in->data | (uintptr_t)out->data) & 15u) == 0 &&
                       in->node_stride % 4 == 0 && out->node_stride % 4 == 0;
  // short columns leave most staged items idle: the direct kernels do better
  if (!aligned || in->nlev < 16) return NB_OK;
  const uint32_t row_bytes = (uint32_t)(in->node_stride * 4);
  const int G = (in->nlev + 3) / 4;
  const int nvar = in->nvar;
  // each 4-level group must lie inside the staged column
  if ((uint64_t)G * 16u * nvar > row_bytes) return NB_OK;
  // nstages stages of stage_kb KB, one 512-thread CTA per SM.  A stage holds
  // the staged columns, then the tile's weights, staged-row indices and
  // row pointers (bounding ranges, 16-byte aligned).
  const int nstages = m->nstages > 0 ? m->nstages : 2;
  const int stage_kb = m->stage_kb > 0 ? m->stage_kb : 112;
  const int nmax = m->tile_nodes > 0 ? m->tile_nodes : 256;
  const int ecap = 10 * nmax;
  const uint32_t meta_bytes = (uint32_t)((ecap + 2) * 8 + 16) + (uint32_t)((ecap + 16) * 2 + 16) +
                              (uint32_t)((nmax + 8) * 4 + 16);
  const uint32_t stage_target = (uint32_t)stage_kb * 1024u;
  if (stage_target <= meta_bytes) return NB_OK;
  const int rcap = (int)((stage_target - meta_bytes) / row_bytes);
  if (rcap < 24) return NB_OK;  // columns too tall to stage a useful tile
  int status = NB_OK;
  TilePlan *tp = get_plan(m, rcap, nmax, ecap, &status);
  if (!tp) return status;
  if (g_sm_count == 0) {
    int dev = 0;
    NB_CUDA(cudaGetDevice(&dev));
    NB_CUDA(cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev));
  }
  TiledArgs a;
  a.ntiles = tp->ntiles;
  a.ntiles_main = tp->ntiles_main;
  a.tile_node0 = tp->d_tile_node0;
  a.halo_ptr = tp->d_halo_ptr;
  a.halo = tp->d_halo;
  a.hrun = tp->d_hrun;
  a.nruns = tp->d_nruns;
  a.lnbr = tp->d_lnbr;
  a.row_ptr = m->d_row_ptr;
  const bool g = op == NB_OP_GRAD;
  a.w32 = reinterpret_cast<const float2 *>(g ? m->d_wgrad32 : op == NB_OP_DIV ? m->d_wdiv32 : m->d_wcurl32);
  a.w64 = reinterpret_cast<const double2 *>(g ? m->d_wgrad64 : op == NB_OP_DIV ? m->d_wdiv64 : m->d_wcurl64);
  a.s32 = reinterpret_cast<const float2 *>(op == NB_OP_CURL ? m->d_scurl32 : m->d_sdiv32);
  a.s64 = reinterpret_cast<const double2 *>(op == NB_OP_CURL ? m->d_scurl64 : m->d_sdiv64);
  a.in = static_cast<const char *>(in->data);
  a.row_bytes = row_bytes;
  a.in_stride = in->node_stride;
  a.out = static_cast<float *>(out->data);
  a.out_stride = out->node_stride;
  a.nlev = in->nlev;
  a.G = G;
  magic_div((uint32_t)a.G, a.g_magic, a.g_shift);
  a.copy_bytes = (uint32_t)(((int64_t)in->nlev * nvar * 4 + 15) / 16 * 16);
  auto up16 = [](uint32_t x) { return (x + 15u) & ~15u; };
  a.off_w = up16((uint32_t)rcap * row_bytes);
  a.off_l = a.off_w + up16((uint32_t)(ecap + 2) * 8u);
  a.off_r = a.off_l + up16((uint32_t)(ecap + 16) * 2u);
  a.stage_bytes = (a.off_r + up16((uint32_t)(nmax + 8) * 4u) + 127u) & ~127u;
  a.nstages = nstages;
  a.status = nullptr;
  if (const int rc = status_word(&a.status)) return rc;
  a.timeout_ns = 2000000000ull;
  const size_t smem = (size_t)nstages * a.stage_bytes + 16 * (size_t)nstages;
  if (smem > 227 * 1024) {
    set_error("staged kernel: nstages * stage size exceeds 227 KB of shared memory");
    return NB_EINVAL;
  }
  const int grid = std::min(tp->ntiles, g_sm_count);
  *handled = true;
  const bool comp = m->compensated != 0;
  if (g) return comp ? launch_staged_t<0, true>(a, grid, smem, st) : launch_staged_t<0, false>(a, grid, smem, st);
  return comp ? launch_staged_t<1, true>(a, grid, smem, st) : launch_staged_t<1, false>(a, grid, smem, st);
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
