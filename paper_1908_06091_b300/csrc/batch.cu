// batch.cu -- many nabla operations on fields of different meshes and level
// counts in one persistent launch, captured in a CUDA graph.
//
// Each item (op, method, in, out) is cut into work units of `npw * 8 * rounds`
// nodes x `lpb` levels.  A persistent grid of 256-thread CTAs takes units from
// an atomic counter (dynamic load balancing across uneven items); inside a
// unit, warp w takes `npw` nodes per round and each node's 32 / npw lanes take
// consecutive levels, so a neighbour's column is read as contiguous words.
// The per-(node, level) arithmetic is exactly the direct kernels' (same weights,
// same neighbour order, same compensated accumulation, FP64 for pole-row
// nodes), so a batched result equals the same operation run alone on the
// direct kernels bit for bit.  Laplacian items run their gradient pass in
// phase 1 (into batch-owned scratch) and their divergence pass in phase 2.
// Large FP32 items instead take the shared-memory staged kernels (one launch,
// two for a Laplacian), exactly as when run alone.  The counter resets, the
// two persistent launches and the staged launches form one CUDA graph.  The
// route and, for the persistent kernel, `levels per block` and `nodes per
// warp` are chosen per item class (op, dtype, grid, levels) by an autotuner
// that times the candidates on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "kernels_common.cuh"

namespace nb {

struct BItem {
  int32_t op;     // 0 grad, 1 div, 2 curl (the Laplacian is split into 0 then 1)
  int32_t f64;
  int32_t vec;    // FP32 with 16-byte columns: lanes take groups of 4 levels
  int32_t nlev, lpb, npw, rounds;
  int32_t nchunk_lev;
  int64_t V, cap_begin;
  int64_t unit_begin;  // first unit of this item in its phase
  const int32_t *row_ptr, *nbr;
  const void *w32, *w64, *s32, *s64;
  const void *in;
  void *out;
  int64_t in_stride, out_stride;
  int *status;  // device status word (index checks of the bounds-checked build)
};

constexpr int kBatchThreads = 256;
constexpr int kBatchWarps = kBatchThreads / 32;

// ----------------------------------------------------------- device part

// One (node, level) of grad / div / curl with the direct kernels' arithmetic.
__device__ __forceinline__ void unit_point_f32(const BItem &it, int64_t i, int l, bool comp) {
  const int32_t p0 = __ldg(it.row_ptr + i), p1 = __ldg(it.row_ptr + i + 1);
  if (it.op == 0) {
    const float *f = static_cast<const float *>(it.in);
    const float fi = __ldg(f + i * it.in_stride + l);
    float gx, gy;
    if (i < it.cap_begin) {
      const float2 *w = static_cast<const float2 *>(it.w32);
      KahanAcc ax, ay;
      PlainAcc px, py;
      for (int32_t p = p0; p < p1; ++p) {
        const int32_t j = (int32_t)NB_IDX(__ldg(it.nbr + p), 0, it.V, it.status);
        const float2 wp = __ldg(w + p);
        const float d = __fsub_rn(__ldg(f + (int64_t)j * it.in_stride + l), fi);
        if (comp) {
          ax.add_prod(wp.x, d);
          ay.add_prod(wp.y, d);
        } else {
          px.add_prod(wp.x, d);
          py.add_prod(wp.y, d);
        }
      }
      gx = comp ? ax.value() : px.value();
      gy = comp ? ay.value() : py.value();
    } else {
      const double2 *w = static_cast<const double2 *>(it.w64);
      double sx = 0, sy = 0;
      for (int32_t p = p0; p < p1; ++p) {
        const int32_t j = (int32_t)NB_IDX(__ldg(it.nbr + p), 0, it.V, it.status);
        const double2 wp = __ldg(w + p);
        const double d = (double)__ldg(f + (int64_t)j * it.in_stride + l) - (double)fi;
        sx = fma(wp.x, d, sx);
        sy = fma(wp.y, d, sy);
      }
      gx = (float)sx;
      gy = (float)sy;
    }
    float *g = static_cast<float *>(it.out) + i * it.out_stride + 2 * l;
    g[0] = gx;
    g[1] = gy;
  } else {
    const float *uv = static_cast<const float *>(it.in);
    const float ui = __ldg(uv + i * it.in_stride + 2 * l), vi = __ldg(uv + i * it.in_stride + 2 * l + 1);
    float r;
    if (i < it.cap_begin) {
      const float2 *w = static_cast<const float2 *>(it.w32);
      const float2 sw = __ldg(static_cast<const float2 *>(it.s32) + i);
      KahanAcc acc;
      PlainAcc pacc;
      for (int32_t p = p0; p < p1; ++p) {
        const int32_t j = (int32_t)NB_IDX(__ldg(it.nbr + p), 0, it.V, it.status);
        const float2 wp = __ldg(w + p);
        const float *cj = uv + (int64_t)j * it.in_stride + 2 * l;
        const float du = __fsub_rn(__ldg(cj), ui), dv = __fsub_rn(__ldg(cj + 1), vi);
        const float term = __fmaf_rn(wp.x, du, __fmul_rn(wp.y, dv));
        if (comp) acc.add(term);
        else pacc.add(term);
      }
      const float self = __fmaf_rn(sw.x, ui, __fmul_rn(sw.y, vi));
      if (comp) {
        acc.add(self);
        r = acc.value();
      } else {
        pacc.add(self);
        r = pacc.value();
      }
    } else {
      const double2 *w = static_cast<const double2 *>(it.w64);
      const double2 sw = __ldg(static_cast<const double2 *>(it.s64) + i);
      double s = 0;
      for (int32_t p = p0; p < p1; ++p) {
        const int32_t j = (int32_t)NB_IDX(__ldg(it.nbr + p), 0, it.V, it.status);
        const double2 wp = __ldg(w + p);
        const float *cj = uv + (int64_t)j * it.in_stride + 2 * l;
        s = fma(wp.x, (double)__ldg(cj) - (double)ui, s);
        s = fma(wp.y, (double)__ldg(cj + 1) - (double)vi, s);
      }
      s = fma(sw.x, (double)ui, s);
      s = fma(sw.y, (double)vi, s);
      r = (float)s;
    }
    static_cast<float *>(it.out)[i * it.out_stride + l] = r;
  }
}

// Levels l0 .. l0+3 of one node with the direct kernels' 4-level arithmetic
// (16-byte loads of the column and of each neighbour's column).
__device__ __forceinline__ void unit_group4_f32(const BItem &it, int64_t i, int l0, bool comp) {
  const int32_t p0 = __ldg(it.row_ptr + i), p1 = __ldg(it.row_ptr + i + 1);
  if (it.op == 0) {
    const float *f = static_cast<const float *>(it.in);
    float fi[4], gx[4], gy[4];
    load_scalar_f32<4>(f + i * it.in_stride, l0, it.nlev, fi);
    if (i < it.cap_begin) {
      const float2 *w = static_cast<const float2 *>(it.w32);
      KahanAcc ax[4], ay[4];
      PlainAcc px[4], py[4];
      for (int32_t p = p0; p < p1; ++p) {
        const int32_t j = (int32_t)NB_IDX(__ldg(it.nbr + p), 0, it.V, it.status);
        const float2 wp = __ldg(w + p);
        float fj[4];
        load_scalar_f32<4>(f + (int64_t)j * it.in_stride, l0, it.nlev, fj);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float d = __fsub_rn(fj[k], fi[k]);
          if (comp) {
            ax[k].add_prod(wp.x, d);
            ay[k].add_prod(wp.y, d);
          } else {
            px[k].add_prod(wp.x, d);
            py[k].add_prod(wp.y, d);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        gx[k] = comp ? ax[k].value() : px[k].value();
        gy[k] = comp ? ay[k].value() : py[k].value();
      }
    } else {
      const double2 *w = static_cast<const double2 *>(it.w64);
      double sx[4] = {0, 0, 0, 0}, sy[4] = {0, 0, 0, 0};
      for (int32_t p = p0; p < p1; ++p) {
        const int32_t j = (int32_t)NB_IDX(__ldg(it.nbr + p), 0, it.V, it.status);
        const double2 wp = __ldg(w + p);
        float fj[4];
        load_scalar_f32<4>(f + (int64_t)j * it.in_stride, l0, it.nlev, fj);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const double d = (double)fj[k] - (double)fi[k];
          sx[k] = fma(wp.x, d, sx[k]);
          sy[k] = fma(wp.y, d, sy[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        gx[k] = (float)sx[k];
        gy[k] = (float)sy[k];
      }
    }
    float *go = static_cast<float *>(it.out) + i * it.out_stride + 2 * l0;
    if (l0 + 4 <= it.nlev) {
      reinterpret_cast<float4 *>(go)[0] = make_float4(gx[0], gy[0], gx[1], gy[1]);
      reinterpret_cast<float4 *>(go)[1] = make_float4(gx[2], gy[2], gx[3], gy[3]);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (l0 + k < it.nlev) {
          go[2 * k] = gx[k];
          go[2 * k + 1] = gy[k];
        }
    }
  } else {
    const float *uv = static_cast<const float *>(it.in);
    float ui[4], vi[4], r[4];
    load_vector_f32<4>(uv + i * it.in_stride, l0, it.nlev, ui, vi);
    if (i < it.cap_begin) {
      const float2 *w = static_cast<const float2 *>(it.w32);
      const float2 sw = __ldg(static_cast<const float2 *>(it.s32) + i);
      KahanAcc acc[4];
      PlainAcc pacc[4];
      for (int32_t p = p0; p < p1; ++p) {
        const int32_t j = (int32_t)NB_IDX(__ldg(it.nbr + p), 0, it.V, it.status);
        const float2 wp = __ldg(w + p);
        float uj[4], vj[4];
        load_vector_f32<4>(uv + (int64_t)j * it.in_stride, l0, it.nlev, uj, vj);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float du = __fsub_rn(uj[k], ui[k]), dv = __fsub_rn(vj[k], vi[k]);
          const float term = __fmaf_rn(wp.x, du, __fmul_rn(wp.y, dv));
          if (comp) acc[k].add(term);
          else pacc[k].add(term);
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float self = __fmaf_rn(sw.x, ui[k], __fmul_rn(sw.y, vi[k]));
        if (comp) {
          acc[k].add(self);
          r[k] = acc[k].value();
        } else {
          pacc[k].add(self);
          r[k] = pacc[k].value();
        }
      }
    } else {
      const double2 *w = static_cast<const double2 *>(it.w64);
      const double2 sw = __ldg(static_cast<const double2 *>(it.s64) + i);
      double sacc[4] = {0, 0, 0, 0};
      for (int32_t p = p0; p < p1; ++p) {
        const int32_t j = (int32_t)NB_IDX(__ldg(it.nbr + p), 0, it.V, it.status);
        const double2 wp = __ldg(w + p);
        float uj[4], vj[4];
        load_vector_f32<4>(uv + (int64_t)j * it.in_stride, l0, it.nlev, uj, vj);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          sacc[k] = fma(wp.x, (double)uj[k] - (double)ui[k], sacc[k]);
          sacc[k] = fma(wp.y, (double)vj[k] - (double)vi[k], sacc[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        sacc[k] = fma(sw.x, (double)ui[k], sacc[k]);
        sacc[k] = fma(sw.y, (double)vi[k], sacc[k]);
        r[k] = (float)sacc[k];
      }
    }
    float *oo = static_cast<float *>(it.out) + i * it.out_stride + l0;
    if (l0 + 4 <= it.nlev) {
      *reinterpret_cast<float4 *>(oo) = make_float4(r[0], r[1], r[2], r[3]);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (l0 + k < it.nlev) oo[k] = r[k];
    }
  }
}

__device__ __forceinline__ void unit_point_f64(const BItem &it, int64_t i, int l) {
  const int32_t p0 = __ldg(it.row_ptr + i), p1 = __ldg(it.row_ptr + i + 1);
  const double2 *w = static_cast<const double2 *>(it.w64);
  if (it.op == 0) {
    const double *f = static_cast<const double *>(it.in);
    const double fi = __ldg(f + i * it.in_stride + l);
    double sx = 0, sy = 0;
    for (int32_t p = p0; p < p1; ++p) {
      const int32_t j = (int32_t)NB_IDX(__ldg(it.nbr + p), 0, it.V, it.status);
      const double2 wp = __ldg(w + p);
      const double d = __ldg(f + (int64_t)j * it.in_stride + l) - fi;
      sx = fma(wp.x, d, sx);
      sy = fma(wp.y, d, sy);
    }
    double *g = static_cast<double *>(it.out) + i * it.out_stride + 2 * l;
    g[0] = sx;
    g[1] = sy;
  } else {
    const double *uv = static_cast<const double *>(it.in);
    const double ui = __ldg(uv + i * it.in_stride + 2 * l), vi = __ldg(uv + i * it.in_stride + 2 * l + 1);
    const double2 sw = __ldg(static_cast<const double2 *>(it.s64) + i);
    double s = 0;
    for (int32_t p = p0; p < p1; ++p) {
      const int32_t j = (int32_t)NB_IDX(__ldg(it.nbr + p), 0, it.V, it.status);
      const double2 wp = __ldg(w + p);
      const double *cj = uv + (int64_t)j * it.in_stride + 2 * l;
      s = fma(wp.x, __ldg(cj) - ui, s);
      s = fma(wp.y, __ldg(cj + 1) - vi, s);
    }
    s = fma(sw.x, ui, s);
    s = fma(sw.y, vi, s);
    static_cast<double *>(it.out)[i * it.out_stride + l] = s;
  }
}

// Persistent batch kernel for one phase: CTAs take units from `counter`.
__global__ void __launch_bounds__(kBatchThreads) batch_kernel(const BItem *__restrict__ items,
                                                              int nitems, int64_t nunits,
                                                              unsigned long long *counter, int comp) {
  __shared__ long long s_unit;
  __shared__ int s_item;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long u = (long long)atomicAdd(counter, 1ull);
      s_unit = u;
      int it = -1;
      if (u < nunits) {  // binary search: last item with unit_begin <= u
        int lo = 0, hi = nitems - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (items[mid].unit_begin <= u) lo = mid;
          else hi = mid - 1;
        }
        it = lo;
      }
      s_item = it;
    }
    __syncthreads();
    const long long u = s_unit;
    const int ii = s_item;
    __syncthreads();
    if (u >= nunits) return;
    const BItem &it = items[ii];
    const int64_t k = u - it.unit_begin;
    const int64_t nchunk = k / it.nchunk_lev, lchunk = k - nchunk * it.nchunk_lev;
    const int npw = it.npw, sub = 32 / npw;
    const int l0 = (int)lchunk * it.lpb;
    const int l1 = min(it.nlev, l0 + it.lpb);
    const int64_t nodes_per_unit = (int64_t)npw * kBatchWarps * it.rounds;
    const int64_t n_begin = nchunk * nodes_per_unit;
    for (int r = 0; r < it.rounds; ++r) {
      const int64_t i = n_begin + ((int64_t)r * kBatchWarps + warp) * npw + lane / sub;
      if (i >= it.V) continue;
      if (it.vec) {
        for (int l = l0 + 4 * (lane % sub); l < l1; l += 4 * sub) unit_group4_f32(it, i, l, comp != 0);
      } else {
        for (int l = l0 + lane % sub; l < l1; l += sub) {
          if (it.f64) unit_point_f64(it, i, l);
          else unit_point_f32(it, i, l, comp != 0);
        }
      }
    }
  }
}

// ------------------------------------------------------------- host part

// Item class: op, dtype, grid size (nodes) and levels.
struct TuneKey {
  int op, f64;
  int64_t V;
  int nlev;
  bool operator<(const TuneKey &o) const {
    return std::tie(op, f64, V, nlev) < std::tie(o.op, o.f64, o.V, o.nlev);
  }
};

static std::mutex g_tune_mu;
static std::map<std::string, std::map<TuneKey, std::pair<int, int>>> g_tune;  // gpu -> key -> (lpb, npw)

static std::string gpu_name() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  return p.name;
}

// Autotune cache file: NB_TUNE_CACHE (if set), lines "gpu|op|f64|V|nlev|lpb|npw".
static void load_tune_cache() {
  const char *path = std::getenv("NB_TUNE_CACHE");
  if (!path) return;
  std::ifstream in(path);
  std::string line;
  while (std::getline(in, line)) {
    std::vector<std::string> f;
    std::stringstream ss(line);
    std::string tok;
    while (std::getline(ss, tok, '|')) f.push_back(tok);
    if (f.size() != 7) continue;
    try {
      TuneKey k{std::stoi(f[1]), std::stoi(f[2]), (int64_t)std::stoll(f[3]), std::stoi(f[4])};
      g_tune[f[0]][k] = {std::stoi(f[5]), std::stoi(f[6])};
    } catch (...) {
    }
  }
}
static void save_tune_cache() {
  const char *path = std::getenv("NB_TUNE_CACHE");
  if (!path) return;
  std::ofstream out(path, std::ios::trunc);
  for (auto &g : g_tune)
    for (auto &kv : g.second)
      out << g.first << '|' << kv.first.op << '|' << kv.first.f64 << '|' << kv.first.V << '|'
          << kv.first.nlev << '|' << kv.second.first << '|' << kv.second.second << '\n';
}

// Size heuristic when no tuned entry exists: short columns -> many nodes per
// warp; tall columns -> one node per warp with 32 levels per lane group.
static std::pair<int, int> default_shape(int nlev) {
  if (nlev <= 2) return {nlev, 32};
  if (nlev <= 8) return {8, 4};
  if (nlev <= 40) return {32, 1};
  return {64, 1};
}

// Shape {0, 0} routes an item to the staged kernels.
static const std::pair<int, int> kStagedRoute{0, 0};
static bool staged_route(const std::pair<int, int> &shp) { return shp.first == 0; }

// FP32 items with 16-byte aligned columns of at least 16 levels can take the
// staged kernels (which still fall back to the direct ones when a column does
// not fit a stage).
static bool staged_candidate(const nb_field &in, const nb_field &out) {
  return in.dtype == NB_F32 && in.nlev >= 16 &&
         ((((uintptr_t)in.data) | ((uintptr_t)out.data)) & 15u) == 0 && in.node_stride % 4 == 0 &&
         out.node_stride % 4 == 0;
}

// Default route: the staged kernels for large candidates (about two million
// node-levels and up), the persistent kernel otherwise.
static std::pair<int, int> default_route(const nb_field &in, const nb_field &out) {
  if (staged_candidate(in, out) && in.nnodes * (int64_t)in.nlev >= (int64_t)1 << 21) return kStagedRoute;
  return default_shape(in.nlev);
}

}  // namespace nb

struct nb_batch : nb::RefCounted {
  struct Src {
    int op;
    nb_method *method;
    nb_field in, out;
  };
  std::vector<Src> src;
  std::vector<nb::TuneKey> keys;  // per source item
  std::vector<std::pair<int, int>> shape;  // per source item (lpb, npw)
  std::vector<void *> scratch;  // per source item (Laplacian only)
  std::vector<size_t> scratch_bytes;
  nb::DevAlloc alloc;  // allocator current at creation
  nb::BItem *d_items[2] = {nullptr, nullptr};
  size_t items_bytes[2] = {0, 0};
  int nitems[2] = {0, 0};
  int64_t nunits[2] = {0, 0};
  unsigned long long *d_counter = nullptr;  // 2 counters
  int64_t node_levels = 0;
  int staged_launches = 0;  // launches of the staged route per run
  int comp = 1;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t graph_nodes = 0, graph_kernels = 0;  // of the captured graph
  int grid = 0;
  ~nb_batch() override {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (d_counter || d_items[0] || d_items[1]) cudaDeviceSynchronize();
    for (int ph = 0; ph < 2; ++ph) nb::dev_free(alloc, d_items[ph], items_bytes[ph]);
    nb::dev_free(alloc, d_counter, 2 * sizeof(unsigned long long));
    for (size_t k = 0; k < scratch.size(); ++k) nb::dev_free(alloc, scratch[k], scratch_bytes[k]);
    for (auto &s : src) nb::release(s.method);
  }
};

namespace nb {

int validate_op(const nb_method *m, int op, const nb_field *in, const nb_field *out,
                const nb_field *scratch);

static BItem make_item(const nb_method *m, int op, const nb_field &in, const nb_field &out,
                       std::pair<int, int> shp) {
  BItem b{};
  b.op = op;
  b.f64 = in.dtype == NB_F64;
  b.vec = !b.f64 && in.nlev >= 4 && ((((uintptr_t)in.data) | ((uintptr_t)out.data)) & 15u) == 0 &&
          in.node_stride % 4 == 0 && out.node_stride % 4 == 0;
  b.nlev = in.nlev;
  b.lpb = std::max(1, std::min(shp.first, in.nlev));
  if (b.vec) b.lpb = (b.lpb + 3) / 4 * 4;  // level chunks start on 4-level groups
  b.npw = shp.second;
  const int sub = 32 / b.npw;
  // rounds: about 2048 point evaluations per unit
  const int per_round = b.npw * kBatchWarps * std::min(b.lpb, b.vec ? 4 * sub : sub);
  b.rounds = std::max(1, 2048 / std::max(1, per_round));
  b.nchunk_lev = (in.nlev + b.lpb - 1) / b.lpb;
  b.V = m->mesh->V;
  b.cap_begin = m->mesh->cap_begin;
  b.row_ptr = m->d_row_ptr;
  b.nbr = m->d_nbr;
  b.w32 = op == 0 ? (const void *)m->d_wgrad32 : op == 1 ? (const void *)m->d_wdiv32 : (const void *)m->d_wcurl32;
  b.w64 = op == 0 ? (const void *)m->d_wgrad64 : op == 1 ? (const void *)m->d_wdiv64 : (const void *)m->d_wcurl64;
  b.s32 = op == 2 ? (const void *)m->d_scurl32 : (const void *)m->d_sdiv32;
  b.s64 = op == 2 ? (const void *)m->d_scurl64 : (const void *)m->d_sdiv64;
  b.in = in.data;
  b.out = out.data;
  b.in_stride = in.node_stride;
  b.out_stride = out.node_stride;
  b.status = nullptr;
#ifdef NB_BOUNDS_CHECK
  status_word(&b.status);  // NULL on failure: the checks still clamp, unrecorded
#endif
  return b;
}

static int64_t item_units(const BItem &b) {
  const int64_t nodes_per_unit = (int64_t)b.npw * kBatchWarps * b.rounds;
  return ((b.V + nodes_per_unit - 1) / nodes_per_unit) * b.nchunk_lev;
}

// (Re)build the device work tables of both phases from the current shapes.
static int batch_build_tables(nb_batch *bt) {
  std::vector<BItem> ph[2];
  bt->staged_launches = 0;
  for (size_t k = 0; k < bt->src.size(); ++k) {
    const auto &s = bt->src[k];
    if (staged_route(bt->shape[k])) {
      bt->staged_launches += s.op == NB_OP_LAP ? 2 : 1;
      continue;
    }
    if (s.op == NB_OP_LAP) {
      nb_field tmp = s.in;
      tmp.data = bt->scratch[k];
      tmp.nvar = 2;
      const int q = s.in.dtype == NB_F64 ? 2 : 4;
      tmp.node_stride = 2 * (int64_t)((s.in.nlev + q - 1) / q) * q;
      tmp.lev_stride = 2;
      ph[0].push_back(make_item(s.method, 0, s.in, tmp, bt->shape[k]));
      ph[1].push_back(make_item(s.method, 1, tmp, s.out, bt->shape[k]));
    } else {
      ph[0].push_back(make_item(s.method, s.op, s.in, s.out, bt->shape[k]));
    }
  }
  for (int p = 0; p < 2; ++p) {
    int64_t u = 0;
    for (auto &b : ph[p]) {
      b.unit_begin = u;
      u += item_units(b);
    }
    bt->nunits[p] = u;
    bt->nitems[p] = (int)ph[p].size();
    if (bt->d_items[p]) {
      cudaDeviceSynchronize();
      dev_free(bt->alloc, bt->d_items[p], bt->items_bytes[p]);
      bt->d_items[p] = nullptr;
      bt->items_bytes[p] = 0;
    }
    if (!ph[p].empty()) {
      const int st = dev_alloc(bt->alloc, (void **)&bt->d_items[p], ph[p].size() * sizeof(BItem),
                               "batch work table");
      if (st != NB_OK) return st;
      bt->items_bytes[p] = ph[p].size() * sizeof(BItem);
      NB_CUDA(cudaMemcpy(bt->d_items[p], ph[p].data(), ph[p].size() * sizeof(BItem),
                         cudaMemcpyHostToDevice));
    }
  }
  log_msg(1, "batch: %zu items; persistent route %d + %d items in %lld + %lld units; staged route %d launches",
          bt->src.size(), bt->nitems[0], bt->nitems[1], (long long)bt->nunits[0], (long long)bt->nunits[1],
          bt->staged_launches);
  return NB_OK;
}

int launch_tiled(nb_method *m, int op, const nb_field *in, const nb_field *out, const nb_field *out2,
                 cudaStream_t st, bool *handled, int comp);

// One operation of a staged-route item: the staged kernel, or the direct one
// where a column does not fit a stage.
static int staged_or_direct(nb_method *m, int op, const nb_field &in, const nb_field &out, int comp,
                            cudaStream_t st) {
  bool handled = false;
  const int rc = launch_tiled(m, op, &in, &out, nullptr, st, &handled, comp);
  if (handled || rc != NB_OK) return rc;
  return launch_direct(m, op, &in, &out, st);
}

// Branches of the batch's launch graph: the staged-route items are spread
// over the main stream and kBatchBranches - 1 side streams, forked from and
// joined back to the main stream with events, so that a small item's launch
// (fewer tiles than SMs) runs beside others and each launch's ramp and tail
// overlap its neighbours'.  No CTA of these kernels waits on another, so
// they complete in any overlap.
#ifndef NB_BATCH_BRANCHES
#define NB_BATCH_BRANCHES 4
#endif
constexpr int kBatchBranches = NB_BATCH_BRANCHES;

// One staged-route item (both passes of a Laplacian) on stream st.
static int staged_item(nb_batch *bt, size_t k, cudaStream_t st) {
  const auto &s = bt->src[k];
  if (s.op == NB_OP_LAP) {
    nb_field tmp = s.in;
    tmp.data = bt->scratch[k];
    tmp.nvar = 2;
    tmp.node_stride = 2 * (int64_t)((s.in.nlev + 3) / 4) * 4;
    tmp.lev_stride = 2;
    int rc = staged_or_direct(s.method, NB_OP_GRAD, s.in, tmp, bt->comp, st);
    if (rc == NB_OK) rc = staged_or_direct(s.method, NB_OP_DIV, tmp, s.out, bt->comp, st);
    return rc;
  }
  return staged_or_direct(s.method, s.op, s.in, s.out, bt->comp, st);
}

// Launch the phases on stream st and its side streams (used for capture and
// for tuning): the persistent phases on st, then the staged-route items
// spread over st and the side streams, largest first onto the least-loaded
// branch (st's load counts the persistent items).  Errors after the fork
// still join every branch, so a capture ends with no branch left open.
static int batch_launch(nb_batch *bt, cudaStream_t st, cudaStream_t *side = nullptr, int nside = 0) {
  const int nb = 1 + std::min(nside, kBatchBranches - 1);
  cudaStream_t lanes[kBatchBranches] = {st};
  for (int b = 1; b < nb; ++b) lanes[b] = side[b - 1];
  cudaEvent_t ev[2 * kBatchBranches] = {};
  int nev = 0;
  // the persistent phases first, on st alone: run beside the large staged
  // launches they compete for SMs (timed: 4.74 against 4.63 ms on the
  // 64-field batch)
  NB_CUDA(cudaMemsetAsync(bt->d_counter, 0, 2 * sizeof(unsigned long long), st));
  for (int p = 0; p < 2; ++p) {
    if (bt->nunits[p] == 0) continue;
    batch_kernel<<<bt->grid, kBatchThreads, 0, st>>>(bt->d_items[p], bt->nitems[p], bt->nunits[p],
                                                     bt->d_counter + p, bt->comp);
    count_launch(1);
    NB_CUDA(cudaGetLastError());
  }
  int rc = NB_OK;
  if (nb > 1) {  // fork: the side streams follow st
    cudaEvent_t fork = nullptr;
    NB_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    ev[nev++] = fork;
    if (cudaEventRecord(fork, st) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "batch fork");
    for (int b = 1; b < nb && rc == NB_OK; ++b)
      if (cudaStreamWaitEvent(lanes[b], fork, 0) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "batch fork");
  }
  double load[kBatchBranches] = {};
  for (size_t k = 0; k < bt->src.size(); ++k)
    if (!staged_route(bt->shape[k])) load[0] += (double)bt->src[k].in.nnodes * bt->src[k].in.nlev;
  std::vector<size_t> order;
  for (size_t k = 0; k < bt->src.size(); ++k)
    if (staged_route(bt->shape[k])) order.push_back(k);
  auto work = [&](size_t k) {
    const auto &s = bt->src[k];
    return (double)s.in.nnodes * s.in.nlev * (s.op == NB_OP_LAP ? 2.0 : 1.0);
  };
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return work(x) > work(y); });
  for (size_t k : order) {
    if (rc != NB_OK) break;
    int b = 0;
    for (int c = 1; c < nb; ++c)
      if (load[c] < load[b]) b = c;
    load[b] += work(k);
    rc = staged_item(bt, k, lanes[b]);
  }
  for (int b = 1; b < nb; ++b) {  // join: st waits for every side stream
    cudaEvent_t join = nullptr;
    if (cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) {
      if (rc == NB_OK) rc = cuda_fail(cudaGetLastError(), "batch join");
      continue;
    }
    ev[nev++] = join;
    if (cudaEventRecord(join, lanes[b]) != cudaSuccess || cudaStreamWaitEvent(st, join, 0) != cudaSuccess)
      if (rc == NB_OK) rc = cuda_fail(cudaGetLastError(), "batch join");
  }
  for (int e = 0; e < nev; ++e) cudaEventDestroy(ev[e]);
  return rc;
}

static void drop_graph(nb_batch *bt) {
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  bt->exec = nullptr;
  bt->graph = nullptr;
}

static int batch_capture(nb_batch *bt) {
  drop_graph(bt);
  cudaStream_t cs, side[kBatchBranches - 1] = {};
  NB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  int nside = 0;
  for (; nside < kBatchBranches - 1; ++nside)
    if (cudaStreamCreateWithFlags(&side[nside], cudaStreamNonBlocking) != cudaSuccess) break;
  auto destroy = [&] {
    cudaStreamDestroy(cs);
    for (int b = 0; b < nside; ++b) cudaStreamDestroy(side[b]);
  };
  // one eager run first: staged launches build their tile plans (host and
  // device allocations) on first use, which a capture must not contain
  int rc = batch_launch(bt, cs, side, nside);
  if (rc == NB_OK && cudaStreamSynchronize(cs) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "batch warm-up");
  if (rc != NB_OK) {
    destroy();
    return rc;
  }
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    destroy();
    set_error("nb_batch: stream capture failed to start");
    return NB_ECUDA;
  }
  rc = batch_launch(bt, cs, side, nside);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &g);
  destroy();
  if (rc != NB_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  bt->graph = g;
  size_t nn = 0;
  NB_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) NB_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
  bt->graph_nodes = (int64_t)nn;
  bt->graph_kernels = 0;
  for (cudaGraphNode_t node : nodes) {
    cudaGraphNodeType ty;
    NB_CUDA(cudaGraphNodeGetType(node, &ty));
    bt->graph_kernels += ty == cudaGraphNodeTypeKernel;
  }
  NB_CUDA(cudaGraphInstantiate(&bt->exec, g, 0));
  return NB_OK;
}

}  // namespace nb

extern "C" {

int nb_batch_create(const nb_batch_item *items, int n, nb_batch **out) {
  if (!out || (!items && n > 0) || n < 0) {
    nb::set_error("nb_batch_create: NULL argument or negative count");
    return NB_EINVAL;
  }
  try {
    auto *bt = new nb_batch();
    bt->alloc = nb::current_allocator();
    std::lock_guard<std::mutex> lk(nb::g_tune_mu);
    static bool loaded = false;
    if (!loaded) {
      nb::load_tune_cache();
      loaded = true;
    }
    const std::string gpu = nb::gpu_name();
    for (int k = 0; k < n; ++k) {
      const nb_batch_item &it = items[k];
      int st = nb::validate_op(it.method, it.op, &it.in, &it.out, nullptr);
      if (st != NB_OK) {
        nb::release(bt);
        return st;
      }
      nb_batch::Src s{it.op, nb::retain(const_cast<nb_method *>(it.method)), it.in, it.out};
      bt->src.push_back(s);
      nb::TuneKey key{it.op, it.in.dtype == NB_F64, it.method->mesh->V, it.in.nlev};
      bt->keys.push_back(key);
      auto g = nb::g_tune.find(gpu);
      auto hit = (g != nb::g_tune.end()) ? g->second.find(key) : std::map<nb::TuneKey, std::pair<int, int>>::iterator();
      auto shp = (g != nb::g_tune.end() && hit != g->second.end()) ? hit->second
                                                                   : nb::default_route(it.in, it.out);
      if (nb::staged_route(shp) && !nb::staged_candidate(it.in, it.out)) shp = nb::default_shape(it.in.nlev);
      bt->shape.push_back(shp);
      void *scr = nullptr;
      size_t scr_bytes = 0;
      if (it.op == NB_OP_LAP) {
        const int64_t elem = it.in.dtype == NB_F64 ? 8 : 4;
        const int q = it.in.dtype == NB_F64 ? 2 : 4;
        const int64_t stride = 2 * (int64_t)((it.in.nlev + q - 1) / q) * q;
        scr_bytes = (size_t)(stride * it.in.nnodes * elem);
        const int sa = nb::dev_alloc(bt->alloc, &scr, scr_bytes, "nb_batch_create: Laplacian scratch");
        if (sa != NB_OK) {
          nb::release(bt);
          return sa;
        }
      }
      bt->scratch.push_back(scr);
      bt->scratch_bytes.push_back(scr_bytes);
      bt->node_levels += it.in.nnodes * (int64_t)it.in.nlev;
    }
    {
      const int ca = nb::dev_alloc(bt->alloc, (void **)&bt->d_counter, 2 * sizeof(unsigned long long),
                                   "nb_batch_create: counters");
      if (ca != NB_OK) {
        nb::release(bt);
        return ca;
      }
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, nb::batch_kernel, nb::kBatchThreads, 0);
    bt->grid = std::max(1, sms * std::max(1, per_sm));
    int st = nb::batch_build_tables(bt);
    if (st != NB_OK) {
      nb::release(bt);
      return st;
    }
    *out = bt;
    return NB_OK;
  } catch (...) {
    nb::set_error("nb_batch_create: host allocation failed");
    return NB_EOOM;
  }
}

int nb_batch_release(nb_batch *b) {
  nb::release(b);
  return NB_OK;
}

int nb_batch_set_compensated(nb_batch *b, int on) {
  if (!b) {
    nb::set_error("nb_batch_set_compensated: NULL batch");
    return NB_EINVAL;
  }
  b->comp = on ? 1 : 0;
  nb::drop_graph(b);
  return NB_OK;
}

int nb_batch_run(nb_batch *b, void *stream) {
  if (!b) {
    nb::set_error("nb_batch_run: NULL batch");
    return NB_EINVAL;
  }
  if (!b->exec) {
    const int st = nb::batch_capture(b);
    if (st != NB_OK) return st;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cudaError_t e = cudaGraphLaunch(b->exec, s);
  if (e != cudaSuccess) return nb::cuda_fail(e, "cudaGraphLaunch");
  nb::count_launch((b->nunits[0] > 0) + (b->nunits[1] > 0) + b->staged_launches);
  return NB_OK;
}

int nb_batch_info(const nb_batch *b, int64_t *units, int64_t *node_levels, int32_t *nodes_per_warp,
                  int32_t *levels_per_block) {
  if (!b) {
    nb::set_error("nb_batch_info: NULL batch");
    return NB_EINVAL;
  }
  if (units) *units = b->nunits[0] + b->nunits[1];
  if (node_levels) *node_levels = b->node_levels;
  for (size_t k = 0; k < b->src.size(); ++k) {
    if (nodes_per_warp) nodes_per_warp[k] = b->shape[k].second;
    if (levels_per_block) levels_per_block[k] = b->shape[k].first;
  }
  return NB_OK;
}

int nb_batch_graph_nodes(const nb_batch *b, int64_t *nodes, int64_t *kernels) {
  if (!b || !nodes || !kernels) {
    nb::set_error("nb_batch_graph_nodes: NULL argument");
    return NB_EINVAL;
  }
  *nodes = b->graph_nodes;
  *kernels = b->graph_kernels;
  return NB_OK;
}

int nb_batch_tune(nb_batch *b, void *stream) {
  if (!b) {
    nb::set_error("nb_batch_tune: NULL batch");
    return NB_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int lpbs[] = {4, 8, 16, 32, 64};
  const int npws[] = {1, 2, 4, 8, 16, 32};
  const std::string gpu = nb::gpu_name();
  cudaEvent_t e0, e1;
  NB_CUDA(cudaEventCreate(&e0));
  NB_CUDA(cudaEventCreate(&e1));
  // tune each item class once, timing a batch that holds only that item
  std::map<nb::TuneKey, std::pair<int, int>> best;
  int rc = NB_OK;
  for (size_t k = 0; k < b->src.size() && rc == NB_OK; ++k) {
    if (best.count(b->keys[k])) continue;
    nb_batch one;
    one.src.push_back(b->src[k]);
    nb::retain(b->src[k].method);
    one.scratch.push_back(b->scratch[k]);
    one.scratch_bytes.push_back(b->scratch_bytes[k]);
    one.alloc = b->alloc;
    one.grid = b->grid;
    one.comp = b->comp;
    one.shape.push_back({0, 0});
    if ((rc = nb::dev_alloc(one.alloc, (void **)&one.d_counter, 2 * sizeof(unsigned long long),
                            "nb_batch_tune: counters")) != NB_OK) {
      one.scratch[0] = nullptr;
      break;
    }
    float best_ms = 1e30f;
    std::pair<int, int> best_shape = nb::default_shape(b->src[k].in.nlev);
    if (nb::staged_candidate(b->src[k].in, b->src[k].out)) {
      one.shape[0] = nb::kStagedRoute;
      if ((rc = nb::batch_build_tables(&one)) != NB_OK) break;
      for (int w = 0; w < 2 && rc == NB_OK; ++w) rc = nb::batch_launch(&one, st);
      cudaEventRecord(e0, st);
      for (int r = 0; r < 5 && rc == NB_OK; ++r) rc = nb::batch_launch(&one, st);
      cudaEventRecord(e1, st);
      if (rc != NB_OK) break;
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      best_ms = ms;
      best_shape = nb::kStagedRoute;
    }
    for (int lpb : lpbs) {
      if (lpb > 2 * b->src[k].in.nlev && lpb != 4) continue;
      for (int npw : npws) {
        one.shape[0] = {lpb, npw};
        if ((rc = nb::batch_build_tables(&one)) != NB_OK) break;
        for (int w = 0; w < 2 && rc == NB_OK; ++w) rc = nb::batch_launch(&one, st);
        cudaEventRecord(e0, st);
        for (int r = 0; r < 5 && rc == NB_OK; ++r) rc = nb::batch_launch(&one, st);
        cudaEventRecord(e1, st);
        if (rc != NB_OK) break;
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
          best_ms = ms;
          best_shape = {lpb, npw};
        }
      }
      if (rc != NB_OK) break;
    }
    one.scratch[0] = nullptr;  // owned by the outer batch
    best[b->keys[k]] = best_shape;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != NB_OK) return rc;
  {
    std::lock_guard<std::mutex> lk(nb::g_tune_mu);
    for (auto &kv : best) nb::g_tune[gpu][kv.first] = kv.second;
    nb::save_tune_cache();
  }
  for (size_t k = 0; k < b->src.size(); ++k) b->shape[k] = best[b->keys[k]];
  nb::drop_graph(b);
  return nb::batch_build_tables(b);
}

}  // extern "C"
