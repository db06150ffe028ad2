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
  int G;               // 4-level groups per column
  uint64_t g_magic;    // item / G == (item * g_magic) >> g_shift, exact for items < 2^24
  uint32_t g_shift;
  uint32_t copy_bytes; // bytes copied per column: the real data rounded up to 16
  uint32_t stage_bytes;
  int *status;
  uint64_t timeout_ns;
};

// Issue the copies of tile t into the stage at `rows` (warp 0 only).
__device__ __forceinline__ void issue_tile(const TiledArgs &a, int t, uint32_t rows, uint32_t bar,
                                           int lane) {
  const int32_t n0 = __ldg(a.tile_node0 + t), n1 = __ldg(a.tile_node0 + t + 1);
  const int32_t h0 = __ldg(a.halo_ptr + t), h1 = __ldg(a.halo_ptr + t + 1);
  const uint32_t n = (uint32_t)(n1 - n0), H = (uint32_t)(h1 - h0);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const uint32_t body = (n - 1) * a.row_bytes + a.copy_bytes;
  if (lane == 0) mbar_expect_tx(bar, body + H * a.copy_bytes);
  __syncwarp();
  if (lane == 0) bulk_g2s(rows, a.in + (int64_t)n0 * a.in_stride * 4, body, bar);
  for (uint32_t h = lane; h < H; h += 32) {
    const int32_t node = __ldg(a.halo + h0 + h);
    bulk_g2s(rows + (n + h) * a.row_bytes, a.in + (int64_t)node * a.in_stride * 4, a.copy_bytes, bar);
  }
}

template <bool COMP>
__device__ __forceinline__ void grad_tile(const TiledArgs &a, int t, const char *rows) {
  const int32_t n0 = __ldg(a.tile_node0 + t), n1 = __ldg(a.tile_node0 + t + 1);
  const uint32_t items = (uint32_t)(n1 - n0) * a.G;
  const bool pole = t >= a.ntiles_main;
  for (uint32_t item = threadIdx.x; item < items; item += blockDim.x) {
    const uint32_t il = (uint32_t)(((uint64_t)item * a.g_magic) >> a.g_shift);
    const uint32_t c = item - il * a.G;
    const int l0 = 4 * (int)c;
    const int64_t node = n0 + il;
    const int32_t p0 = __ldg(a.row_ptr + node), p1 = __ldg(a.row_ptr + node + 1);
    const char *col = rows + c * 16;
    const float4 fi = *reinterpret_cast<const float4 *>(col + il * a.row_bytes);
    float gx[4], gy[4];
    if (!pole) {
      const f2_t fi01 = pk(fi.x, fi.y), fi23 = pk(fi.z, fi.w);
      Kahan2<COMP> ax01, ax23, ay01, ay23;
      for (int32_t p = p0; p < p1; ++p) {
        const uint32_t lr = __ldg(a.lnbr + p);
        const float2 w = __ldg(a.w32 + p);
        const float4 fj = *reinterpret_cast<const float4 *>(col + lr * a.row_bytes);
        const f2_t d01 = sub2(pk(fj.x, fj.y), fi01), d23 = sub2(pk(fj.z, fj.w), fi23);
        const f2_t wx = pk(w.x, w.x), wy = pk(w.y, w.y);
        ax01.add_prod(wx, d01);
        ax23.add_prod(wx, d23);
        ay01.add_prod(wy, d01);
        ay23.add_prod(wy, d23);
      }
      upk(ax01.value(), gx[0], gx[1]);
      upk(ax23.value(), gx[2], gx[3]);
      upk(ay01.value(), gy[0], gy[1]);
      upk(ay23.value(), gy[2], gy[3]);
    } else {
      double sx[4] = {0, 0, 0, 0}, sy[4] = {0, 0, 0, 0};
      const float fiv[4] = {fi.x, fi.y, fi.z, fi.w};
      for (int32_t p = p0; p < p1; ++p) {
        const uint32_t lr = __ldg(a.lnbr + p);
        const double2 w = __ldg(a.w64 + p);
        const float4 fj = *reinterpret_cast<const float4 *>(col + lr * a.row_bytes);
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
    float *go = a.out + node * a.out_stride + 2 * l0;
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

// div / curl: the (u, v) columns are interleaved, a 4-level group is 32 bytes.
template <bool COMP>
__device__ __forceinline__ void divcurl_tile(const TiledArgs &a, int t, const char *rows) {
  const int32_t n0 = __ldg(a.tile_node0 + t), n1 = __ldg(a.tile_node0 + t + 1);
  const uint32_t items = (uint32_t)(n1 - n0) * a.G;
  const bool pole = t >= a.ntiles_main;
  for (uint32_t item = threadIdx.x; item < items; item += blockDim.x) {
    const uint32_t il = (uint32_t)(((uint64_t)item * a.g_magic) >> a.g_shift);
    const uint32_t c = item - il * a.G;
    const int l0 = 4 * (int)c;
    const int64_t node = n0 + il;
    const int32_t p0 = __ldg(a.row_ptr + node), p1 = __ldg(a.row_ptr + node + 1);
    const char *col = rows + c * 32;
    const float4 A = *reinterpret_cast<const float4 *>(col + il * a.row_bytes);
    const float4 B = *reinterpret_cast<const float4 *>(col + il * a.row_bytes + 16);
    float r[4];
    if (!pole) {
      // pair accumulators (sum of w.x du, sum of w.y dv) per level
      const f2_t i0 = pk(A.x, A.y), i1 = pk(A.z, A.w), i2 = pk(B.x, B.y), i3 = pk(B.z, B.w);
      Kahan2<COMP> k0, k1, k2, k3;
      for (int32_t p = p0; p < p1; ++p) {
        const uint32_t lr = __ldg(a.lnbr + p);
        const float2 w = __ldg(a.w32 + p);
        const char *cj = col + lr * a.row_bytes;
        const float4 C = *reinterpret_cast<const float4 *>(cj);
        const float4 D = *reinterpret_cast<const float4 *>(cj + 16);
        const f2_t w2 = pk(w.x, w.y);
        k0.add_prod(w2, sub2(pk(C.x, C.y), i0));
        k1.add_prod(w2, sub2(pk(C.z, C.w), i1));
        k2.add_prod(w2, sub2(pk(D.x, D.y), i2));
        k3.add_prod(w2, sub2(pk(D.z, D.w), i3));
      }
      const float2 sw = __ldg(a.s32 + node);
      const f2_t sw2 = pk(sw.x, sw.y);
      // self term joins each pair before the two halves are added
      f2_t v[4] = {k0.value(), k1.value(), k2.value(), k3.value()};
      const f2_t self[4] = {i0, i1, i2, i3};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const f2_t q = fma2(sw2, self[k], v[k]);
        float x, y;
        upk(q, x, y);
        r[k] = __fadd_rn(x, y);
      }
    } else {
      const float iu[4] = {A.x, A.z, B.x, B.z}, iv[4] = {A.y, A.w, B.y, B.w};
      double s[4] = {0, 0, 0, 0};
      for (int32_t p = p0; p < p1; ++p) {
        const uint32_t lr = __ldg(a.lnbr + p);
        const double2 w = __ldg(a.w64 + p);
        const char *cj = col + lr * a.row_bytes;
        const float4 C = *reinterpret_cast<const float4 *>(cj);
        const float4 D = *reinterpret_cast<const float4 *>(cj + 16);
        const float ju[4] = {C.x, C.z, D.x, D.z}, jv[4] = {C.y, C.w, D.y, D.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          s[k] = fma(w.x, (double)ju[k] - (double)iu[k], s[k]);
          s[k] = fma(w.y, (double)jv[k] - (double)iv[k], s[k]);
        }
      }
      const double2 sw = __ldg(a.s64 + node);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        s[k] = fma(sw.x, (double)iu[k], s[k]);
        s[k] = fma(sw.y, (double)iv[k], s[k]);
        r[k] = (float)s[k];
      }
    }
    float *oo = a.out + node * a.out_stride + l0;
    if (l0 + 4 <= a.nlev) {
      __stcs(reinterpret_cast<float4 *>(oo), make_float4(r[0], r[1], r[2], r[3]));
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (l0 + k < a.nlev) oo[k] = r[k];
    }
  }
}

template <int OP, bool COMP>
__global__ void __launch_bounds__(512, 1) staged_f32(TiledArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + 2 * (size_t)a.stage_bytes);
  const uint32_t bar0 = smem_u32(&bars[0]), bar1 = smem_u32(&bars[1]);
  const uint32_t stage0 = smem_u32(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int t = blockIdx.x;
  // copies issued into / consumed from stage 0 and stage 1 so far
  uint32_t issued0 = 0, issued1 = 0, done0 = 0, done1 = 0;
  if (t < a.ntiles) {
    if (warp == 0) issue_tile(a, t, stage0, bar0, lane);
    issued0 = 1;
  }
  bool failed = false;
  for (int k = 0; t < a.ntiles; t += gridDim.x, ++k) {
    const int s = k & 1;
    const int tn = t + gridDim.x;
    if (tn < a.ntiles) {
      if (warp == 0) issue_tile(a, tn, stage0 + (s ^ 1) * a.stage_bytes, s ? bar0 : bar1, lane);
      if (s) ++issued0;
      else ++issued1;
    }
    if (!mbar_wait_bounded(s ? bar1 : bar0, (s ? done1 : done0) & 1, a.timeout_ns)) {
      failed = true;
      break;
    }
    if (s) ++done1;
    else ++done0;
    const char *rows = reinterpret_cast<const char *>(smem) + s * a.stage_bytes;
    if (OP == 0) grad_tile<COMP>(a, t, rows);
    else divcurl_tile<COMP>(a, t, rows);
    __syncthreads();
  }
  if (failed) {
    if (threadIdx.x == 0) atomicCAS(a.status, 0, (int)NB_ETIMEOUT);
    // let this CTA's own copies land (bounded) before its shared memory is released
    for (uint32_t u = done0; u < issued0; ++u)
      if (!mbar_wait_bounded(bar0, u & 1, a.timeout_ns)) break;
    for (uint32_t u = done1; u < issued1; ++u)
      if (!mbar_wait_bounded(bar1, u & 1, a.timeout_ns)) break;
  }
}

// --------------------------------------------------------------- host

static int plan_upload(TilePlan *tp, const nb_mesh *mesh) {
  std::vector<int32_t> node0, hptr, halo;
  std::vector<uint16_t> lnbr;
  build_tile_plan_host(mesh, tp->rcap, tp->nmax, node0, hptr, halo, lnbr, tp->max_halo,
                       tp->max_entries, tp->ntiles_main);
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
  return NB_OK;
}

static TilePlan *get_plan(nb_method *m, int rcap, int nmax, int *status) {
  std::lock_guard<std::mutex> lk(m->plan_mu);
  auto key = std::make_pair(rcap, nmax);
  auto it = m->plans.find(key);
  if (it != m->plans.end()) return it->second.get();
  auto tp = std::make_unique<TilePlan>();
  tp->rcap = rcap;
  tp->nmax = nmax;
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
  staged_f32<OP, COMP><<<grid, 512, smem, st>>>(a);
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
  if (!aligned || in->nlev < 4) return NB_OK;
  const uint32_t row_bytes = (uint32_t)(in->node_stride * 4);
  const int G = (in->nlev + 3) / 4;
  const int nvar = in->nvar;
  // each 4-level group must lie inside the staged column
  if ((uint64_t)G * 16u * nvar > row_bytes) return NB_OK;
  // two stages of ~96 KB, one 512-thread CTA per SM
  const uint32_t stage_target = 96 * 1024;
  const int rcap = (int)(stage_target / row_bytes);
  if (rcap < 72) return NB_OK;  // columns too tall to stage a useful tile
  const int nmax = m->tile_nodes > 0 ? m->tile_nodes : 256;
  int status = NB_OK;
  TilePlan *tp = get_plan(m, rcap, nmax, &status);
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
  a.stage_bytes = (uint32_t)rcap * row_bytes;
  a.stage_bytes = (a.stage_bytes + 127u) & ~127u;
  a.status = nullptr;
  if (const int rc = status_word(&a.status)) return rc;
  a.timeout_ns = 2000000000ull;
  const size_t smem = 2 * (size_t)a.stage_bytes + 64;
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
