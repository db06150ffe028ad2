// nabla_kernels.cu -- sm_103a kernels of the edge-based median-dual nabla
// operators (Sec. 4.7, Fig. 33, Listing 12) and the device side of the
// fvm::Method (geometry upload and FP64 weight setup).
//
// Discretisation (one level; sums over the edges e = (i, j) at node i, with
// S_e^(i), T_e^(i) the face normal / tangent integrals seen from i and V_i
// the dual volume):
//   grad  G_i = (1/V_i) sum 1/2 (f_j - f_i) S_e^(i)      -> (G.e_i, G.n_i)
//   div   D_i = (1/V_i) sum 1/2 (W_i + W_j) . S_e^(i)    W = u e + v n
//   curl  Z_i = (1/V_i) sum 1/2 (W_i + W_j) . T_e^(i)
//   lap   L_i = div(grad f)_i
// The weights are projected once per method in FP64 on the device:
//   grad  (gx, gy)_p = 1/2 S.(e_i, n_i) / V_i
//   div   (du, dv)_p = 1/2 S.(e_j, n_j) / V_i,
//         self (su, sv)_i = sum_p 1/2 S.(e_i + e_j, n_i + n_j) / V_i
//   curl  the same with T,
// so that div and curl are evaluated in difference form,
//   D_i = sum_p du_p (u_j - u_i) + dv_p (v_j - v_i) + su_i u_i + sv_i v_i,
// algebraically the flux form, but with every FP32 term of the size of the
// result (no cancellation between large edge fluxes).  Pole-row nodes, whose
// cap chords join nodes with nearly opposite local frames, are evaluated in
// FP64 inside the FP32 kernels.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>

#include "internal.h"
#include "kernels_common.cuh"

namespace nb {

static std::atomic<int64_t> g_launches{0};
int64_t launch_count() { return g_launches.load(); }
void count_launch(int n) { g_launches.fetch_add(n); }

int cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return NB_ECUDA;
}

// ------------------------------------------------------------ weight setup

// One thread per node: project the FP64 face integrals onto the local frames
// and divide by the dual volume (all in FP64), then round to FP32.
__global__ void __launch_bounds__(256) setup_weights_kernel(
    int64_t V, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ nbr,
    const int32_t *__restrict__ nbr_edge, const double *__restrict__ vol,
    const double *__restrict__ S, const double *__restrict__ T, const double *__restrict__ east,
    const double *__restrict__ north, double2 *wgrad64, double2 *wdiv64, double2 *wcurl64,
    double2 *sdiv64, double2 *scurl64, float2 *wgrad32, float2 *wdiv32, float2 *wcurl32,
    float2 *sdiv32, float2 *scurl32, float4 *wdc32, float4 *sdc32) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  const double h = 0.5 / vol[i];
  const double ei[3] = {east[3 * i], east[3 * i + 1], east[3 * i + 2]};
  const double ni[3] = {north[3 * i], north[3 * i + 1], north[3 * i + 2]};
  double su = 0, sv = 0, tu = 0, tv = 0;
  for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
    const int32_t j = nbr[p], e = nbr_edge[p];
    const double sg = (i < j) ? h : -h;  // S_e, T_e are stored as seen from the lower id
    const double s[3] = {sg * S[3 * e], sg * S[3 * e + 1], sg * S[3 * e + 2]};
    const double t[3] = {sg * T[3 * e], sg * T[3 * e + 1], sg * T[3 * e + 2]};
    const double ej[3] = {east[3 * j], east[3 * j + 1], east[3 * j + 2]};
    const double nj[3] = {north[3 * j], north[3 * j + 1], north[3 * j + 2]};
    auto dot = [](const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
    const double gx = dot(s, ei), gy = dot(s, ni);
    const double du = dot(s, ej), dv = dot(s, nj);
    const double cu = dot(t, ej), cv = dot(t, nj);
    su += du + gx;
    sv += dv + gy;
    tu += cu + dot(t, ei);
    tv += cv + dot(t, ni);
    wgrad64[p] = make_double2(gx, gy);
    wdiv64[p] = make_double2(du, dv);
    wcurl64[p] = make_double2(cu, cv);
    wgrad32[p] = make_float2((float)gx, (float)gy);
    wdiv32[p] = make_float2((float)du, (float)dv);
    wcurl32[p] = make_float2((float)cu, (float)cv);
    wdc32[p] = make_float4((float)du, (float)dv, (float)cu, (float)cv);
  }
  sdiv64[i] = make_double2(su, sv);
  scurl64[i] = make_double2(tu, tv);
  sdiv32[i] = make_float2((float)su, (float)sv);
  scurl32[i] = make_float2((float)tu, (float)tv);
  sdc32[i] = make_float4((float)su, (float)sv, (float)tu, (float)tv);
}

template <class T>
static int dev_upload(nb_method *m, T **dst, const void *src, size_t n) {
  const int st = dev_alloc(m->alloc, (void **)dst, n * sizeof(T), "method upload");
  if (st != NB_OK) return st;
  m->blocks.push_back({*dst, n * sizeof(T)});
  m->device_bytes += (int64_t)(n * sizeof(T));
  if (src) NB_CUDA(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
  return NB_OK;
}

int method_upload(nb_method *m) {
  const nb_mesh *mesh = m->mesh;
  const int64_t V = mesh->V, E = mesh->E, P = 2 * E;
  NB_CUDA(cudaGetDevice(&m->device));
  // row_ptr is padded with 8 copies of its last entry so that 16-byte
  // aligned bounding copies of any node range stay inside the allocation
  std::vector<int32_t> rp(V + 1 + 8);
  for (int64_t i = 0; i <= V; ++i) rp[i] = (int32_t)mesh->row_ptr[i];
  for (int64_t i = V + 1; i < V + 9; ++i) rp[i] = (int32_t)mesh->row_ptr[V];
  int st;
#define UP(dst, src, n) \
  if ((st = dev_upload(m, &(dst), (src), (n))) != NB_OK) return st;
  UP(m->d_row_ptr, rp.data(), V + 9);
  UP(m->d_nbr, mesh->nbr.data(), P);
  UP(m->d_nbr_edge, mesh->nbr_edge.data(), P);
  UP(m->d_edge, mesh->edge.data(), 2 * E);
  UP(m->d_vol, m->vol.data(), V);
  UP(m->d_S, m->S.data(), 3 * E);
  UP(m->d_T, m->T.data(), 3 * E);
  UP(m->d_east, m->east.data(), 3 * V);
  UP(m->d_north, m->north.data(), 3 * V);
  UP(m->d_wgrad64, nullptr, 2 * P);
  UP(m->d_wdiv64, nullptr, 2 * P);
  UP(m->d_wcurl64, nullptr, 2 * P);
  UP(m->d_sdiv64, nullptr, 2 * V);
  UP(m->d_scurl64, nullptr, 2 * V);
  UP(m->d_wgrad32, nullptr, 2 * P);
  UP(m->d_wdiv32, nullptr, 2 * P);
  UP(m->d_wcurl32, nullptr, 2 * P);
  // self weights are staged in even-aligned node pairs: one spare node
  UP(m->d_sdiv32, nullptr, 2 * V + 4);
  UP(m->d_scurl32, nullptr, 2 * V + 4);
  // fused div+curl records: (du, dv, cu, cv) per CSR entry, (su, sv, tu, tv) per node
  UP(m->d_wdc32, nullptr, 4 * P);
  UP(m->d_sdc32, nullptr, 4 * V + 4);
#undef UP
  const int threads = 256;
  const int64_t blocks = (V + threads - 1) / threads;
  setup_weights_kernel<<<(unsigned)blocks, threads>>>(
      V, m->d_row_ptr, m->d_nbr, m->d_nbr_edge, m->d_vol, m->d_S, m->d_T, m->d_east, m->d_north,
      (double2 *)m->d_wgrad64, (double2 *)m->d_wdiv64, (double2 *)m->d_wcurl64,
      (double2 *)m->d_sdiv64, (double2 *)m->d_scurl64, (float2 *)m->d_wgrad32,
      (float2 *)m->d_wdiv32, (float2 *)m->d_wcurl32, (float2 *)m->d_sdiv32,
      (float2 *)m->d_scurl32, (float4 *)m->d_wdc32, (float4 *)m->d_sdc32);
  count_launch(1);
  NB_CUDA(cudaGetLastError());
  NB_CUDA(cudaDeviceSynchronize());
  return NB_OK;
}

void method_free_device(nb_method *m) {
  // every block of the method and of its tile plans, through the allocator
  // that made it (plans are created under plan_mu and recorded there too)
  if (!m->blocks.empty()) cudaDeviceSynchronize();
  for (const DevBlock &b : m->blocks) dev_free(m->alloc, b.ptr, b.bytes);
  m->blocks.clear();
  m->plans.clear();
}

// ------------------------------------------------------------- direct kernels
//
// One thread per (node, group of LPT levels).  Consecutive threads take
// consecutive level groups of one node, so a node's column and each
// neighbour's column are read as contiguous 16-byte vectors.  Neighbour
// columns are gathered through L1/L2 (the tiled kernels stage them in shared
// memory instead).

struct DirectArgs {
  int64_t V;
  int64_t cap_begin;
  int nlev;
  int ngroups;  // level groups per node
  const int32_t *row_ptr;
  const int32_t *nbr;
  const void *w32;  // float2 per CSR entry (op weights)
  const void *w64;  // double2 per CSR entry
  const void *s32;  // float2 per node (div / curl self weights)
  const void *s64;  // double2 per node
  const void *in;
  int64_t in_stride;
  void *out;
  int64_t out_stride;
  // edge variant: per-edge differences q[e] = x[b] - x[a] (edges a < b), row
  // stride q_stride; a node i takes +q for a neighbour j > i and -q otherwise
  // (the same value x_j - x_i rounds to: IEEE subtraction is antisymmetric)
  const void *q;
  int64_t q_stride;
  const int32_t *nbr_edge;
  int64_t E;
  int *status;  // device status word (index checks of the bounds-checked build)
};

// op 0: grad.  FP32 arithmetic, compensated or plain accumulation.  EDGE:
// neighbour differences come from the per-edge array (non-pole nodes; the
// FP64 pole rows keep their FP64 differences).
template <int LPT, class Acc, bool EDGE = false>
__global__ void __launch_bounds__(256) grad_direct_f32(DirectArgs a) {
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = item / a.ngroups;
  if (i >= a.V) return;
  const int l0 = (int)(item - i * a.ngroups) * LPT;
  const float *f = static_cast<const float *>(a.in);
  float *g = static_cast<float *>(a.out);
  const int32_t p0 = __ldg(a.row_ptr + i), p1 = __ldg(a.row_ptr + i + 1);
  float gx[LPT], gy[LPT], fi[LPT];
  load_scalar_f32<LPT>(f + i * a.in_stride, l0, a.nlev, fi);
  if (i < a.cap_begin) {
    Acc ax[LPT], ay[LPT];
    const float2 *w = static_cast<const float2 *>(a.w32);
    for (int32_t p = p0; p < p1; ++p) {
      const int32_t j = (int32_t)NB_IDX(__ldg(a.nbr + p), 0, a.V, a.status);
      const float2 wp = __ldg(w + p);
      float dj[LPT];
      if (EDGE) {
        load_scalar_f32<LPT>(static_cast<const float *>(a.q) + NB_IDX(__ldg(a.nbr_edge + p), 0, a.E, a.status) * a.q_stride, l0,
                             a.nlev, dj);
        if (j < i)
#pragma unroll
          for (int k = 0; k < LPT; ++k) dj[k] = -dj[k];
      } else {
        float fj[LPT];
        load_scalar_f32<LPT>(f + (int64_t)j * a.in_stride, l0, a.nlev, fj);
#pragma unroll
        for (int k = 0; k < LPT; ++k) dj[k] = __fsub_rn(fj[k], fi[k]);
      }
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        ax[k].add_prod(wp.x, dj[k]);
        ay[k].add_prod(wp.y, dj[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      gx[k] = ax[k].value();
      gy[k] = ay[k].value();
    }
  } else {
    // pole-row node: FP64 weights and FP64 accumulation
    const double2 *w = static_cast<const double2 *>(a.w64);
    double sx[LPT] = {}, sy[LPT] = {};
    for (int32_t p = p0; p < p1; ++p) {
      const int32_t j = (int32_t)NB_IDX(__ldg(a.nbr + p), 0, a.V, a.status);
      const double2 wp = __ldg(w + p);
      float fj[LPT];
      load_scalar_f32<LPT>(f + (int64_t)j * a.in_stride, l0, a.nlev, fj);
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const double d = (double)fj[k] - (double)fi[k];
        sx[k] = fma(wp.x, d, sx[k]);
        sy[k] = fma(wp.y, d, sy[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      gx[k] = (float)sx[k];
      gy[k] = (float)sy[k];
    }
  }
  float *go = g + i * a.out_stride + 2 * l0;
  if (LPT == 4 && l0 + 4 <= a.nlev) {
    reinterpret_cast<float4 *>(go)[0] = make_float4(gx[0], gy[0], gx[1], gy[1]);
    reinterpret_cast<float4 *>(go)[1] = make_float4(gx[2], gy[2], gx[3], gy[3]);
  } else {
#pragma unroll
    for (int k = 0; k < LPT; ++k)
      if (l0 + k < a.nlev) {
        go[2 * k] = gx[k];
        go[2 * k + 1] = gy[k];
      }
  }
}

// op 1 / 2: div or curl (same stencil, different weights).
template <int LPT, class Acc, bool EDGE = false>
__global__ void __launch_bounds__(256) divcurl_direct_f32(DirectArgs a) {
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = item / a.ngroups;
  if (i >= a.V) return;
  const int l0 = (int)(item - i * a.ngroups) * LPT;
  const float *uv = static_cast<const float *>(a.in);
  float *o = static_cast<float *>(a.out);
  const int32_t p0 = __ldg(a.row_ptr + i), p1 = __ldg(a.row_ptr + i + 1);
  float ui[LPT], vi[LPT], r[LPT];
  load_vector_f32<LPT>(uv + i * a.in_stride, l0, a.nlev, ui, vi);
  if (i < a.cap_begin) {
    const float2 *w = static_cast<const float2 *>(a.w32);
    const float2 sw = __ldg(static_cast<const float2 *>(a.s32) + i);
    Acc acc[LPT];
    for (int32_t p = p0; p < p1; ++p) {
      const int32_t j = (int32_t)NB_IDX(__ldg(a.nbr + p), 0, a.V, a.status);
      const float2 wp = __ldg(w + p);
      float du[LPT], dv[LPT];
      if (EDGE) {
        load_vector_f32<LPT>(static_cast<const float *>(a.q) + NB_IDX(__ldg(a.nbr_edge + p), 0, a.E, a.status) * a.q_stride, l0,
                             a.nlev, du, dv);
        if (j < i)
#pragma unroll
          for (int k = 0; k < LPT; ++k) {
            du[k] = -du[k];
            dv[k] = -dv[k];
          }
      } else {
        float uj[LPT], vj[LPT];
        load_vector_f32<LPT>(uv + (int64_t)j * a.in_stride, l0, a.nlev, uj, vj);
#pragma unroll
        for (int k = 0; k < LPT; ++k) {
          du[k] = __fsub_rn(uj[k], ui[k]);
          dv[k] = __fsub_rn(vj[k], vi[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < LPT; ++k) acc[k].add(__fmaf_rn(wp.x, du[k], __fmul_rn(wp.y, dv[k])));
    }
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      acc[k].add(__fmaf_rn(sw.x, ui[k], __fmul_rn(sw.y, vi[k])));
      r[k] = acc[k].value();
    }
  } else {
    const double2 *w = static_cast<const double2 *>(a.w64);
    const double2 sw = __ldg(static_cast<const double2 *>(a.s64) + i);
    double s[LPT] = {};
    for (int32_t p = p0; p < p1; ++p) {
      const int32_t j = (int32_t)NB_IDX(__ldg(a.nbr + p), 0, a.V, a.status);
      const double2 wp = __ldg(w + p);
      float uj[LPT], vj[LPT];
      load_vector_f32<LPT>(uv + (int64_t)j * a.in_stride, l0, a.nlev, uj, vj);
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        s[k] = fma(wp.x, (double)uj[k] - (double)ui[k], s[k]);
        s[k] = fma(wp.y, (double)vj[k] - (double)vi[k], s[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      s[k] = fma(sw.x, (double)ui[k], s[k]);
      s[k] = fma(sw.y, (double)vi[k], s[k]);
      r[k] = (float)s[k];
    }
  }
  float *oo = o + i * a.out_stride + l0;
  if (LPT == 4 && l0 + 4 <= a.nlev) {
    *reinterpret_cast<float4 *>(oo) = make_float4(r[0], r[1], r[2], r[3]);
  } else {
#pragma unroll
    for (int k = 0; k < LPT; ++k)
      if (l0 + k < a.nlev) oo[k] = r[k];
  }
}

// FP64 path: plain FP64 arithmetic everywhere (the reference GPU path).
template <int LPT, bool EDGE = false>
__global__ void __launch_bounds__(256) grad_direct_f64(DirectArgs a) {
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = item / a.ngroups;
  if (i >= a.V) return;
  const int l0 = (int)(item - i * a.ngroups) * LPT;
  const double *f = static_cast<const double *>(a.in);
  double *g = static_cast<double *>(a.out);
  const double2 *w = static_cast<const double2 *>(a.w64);
  const int32_t p0 = __ldg(a.row_ptr + i), p1 = __ldg(a.row_ptr + i + 1);
  double fi[LPT], sx[LPT] = {}, sy[LPT] = {};
  const double *ci = f + i * a.in_stride;
#pragma unroll
  for (int k = 0; k < LPT; ++k) fi[k] = (l0 + k < a.nlev) ? __ldg(ci + l0 + k) : 0.0;
  for (int32_t p = p0; p < p1; ++p) {
    const int32_t j = (int32_t)NB_IDX(__ldg(a.nbr + p), 0, a.V, a.status);
    const double2 wp = __ldg(w + p);
    const double *cj = EDGE ? static_cast<const double *>(a.q) + NB_IDX(__ldg(a.nbr_edge + p), 0, a.E, a.status) * a.q_stride
                            : f + (int64_t)j * a.in_stride;
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const double x = (l0 + k < a.nlev) ? __ldg(cj + l0 + k) : 0.0;
      const double d = EDGE ? (j < i ? -x : x) : x - fi[k];
      sx[k] = fma(wp.x, d, sx[k]);
      sy[k] = fma(wp.y, d, sy[k]);
    }
  }
  double *go = g + i * a.out_stride + 2 * l0;
#pragma unroll
  for (int k = 0; k < LPT; ++k)
    if (l0 + k < a.nlev) {
      go[2 * k] = sx[k];
      go[2 * k + 1] = sy[k];
    }
}

template <int LPT, bool EDGE = false>
__global__ void __launch_bounds__(256) divcurl_direct_f64(DirectArgs a) {
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = item / a.ngroups;
  if (i >= a.V) return;
  const int l0 = (int)(item - i * a.ngroups) * LPT;
  const double *uv = static_cast<const double *>(a.in);
  double *o = static_cast<double *>(a.out);
  const double2 *w = static_cast<const double2 *>(a.w64);
  const double2 sw = __ldg(static_cast<const double2 *>(a.s64) + i);
  const int32_t p0 = __ldg(a.row_ptr + i), p1 = __ldg(a.row_ptr + i + 1);
  double ui[LPT], vi[LPT], s[LPT] = {};
  const double *ci = uv + i * a.in_stride;
#pragma unroll
  for (int k = 0; k < LPT; ++k) {
    const bool ok = l0 + k < a.nlev;
    ui[k] = ok ? __ldg(ci + 2 * (l0 + k)) : 0.0;
    vi[k] = ok ? __ldg(ci + 2 * (l0 + k) + 1) : 0.0;
  }
  for (int32_t p = p0; p < p1; ++p) {
    const int32_t j = (int32_t)NB_IDX(__ldg(a.nbr + p), 0, a.V, a.status);
    const double2 wp = __ldg(w + p);
    const double *cj = EDGE ? static_cast<const double *>(a.q) + NB_IDX(__ldg(a.nbr_edge + p), 0, a.E, a.status) * a.q_stride
                            : uv + (int64_t)j * a.in_stride;
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const bool ok = l0 + k < a.nlev;
      const double xu = ok ? __ldg(cj + 2 * (l0 + k)) : 0.0;
      const double xv = ok ? __ldg(cj + 2 * (l0 + k) + 1) : 0.0;
      const double du = EDGE ? (j < i ? -xu : xu) : xu - ui[k];
      const double dv = EDGE ? (j < i ? -xv : xv) : xv - vi[k];
      s[k] = fma(wp.x, du, s[k]);
      s[k] = fma(wp.y, dv, s[k]);
    }
  }
  double *oo = o + i * a.out_stride + l0;
#pragma unroll
  for (int k = 0; k < LPT; ++k) {
    s[k] = fma(sw.x, ui[k], s[k]);
    s[k] = fma(sw.y, vi[k], s[k]);
    if (l0 + k < a.nlev) oo[k] = s[k];
  }
}

// Edge pass of the edge variant: q[e][k] = x[b][k] - x[a][k] for the nvals
// values (levels x components) of every edge (a, b), a < b.  VEC: 16-byte
// groups (rows 16-byte aligned), else one value per thread.
template <class T, bool VEC>
__global__ void __launch_bounds__(256) edge_diff_kernel(int64_t E, const int32_t *__restrict__ edge,
                                                        const T *__restrict__ x, int64_t x_stride, int nvals,
                                                        T *__restrict__ q, int64_t q_stride) {
  constexpr int W = VEC ? 16 / (int)sizeof(T) : 1;
  const int per = (nvals + W - 1) / W;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t e = t / per;
  if (e >= E) return;
  const int k = (int)(t - e * per) * W;
  const int64_t a = __ldg(edge + 2 * e), b = __ldg(edge + 2 * e + 1);
  if (VEC) {
    const float4 xa = __ldg(reinterpret_cast<const float4 *>(x + a * x_stride + k));
    const float4 xb = __ldg(reinterpret_cast<const float4 *>(x + b * x_stride + k));
    if constexpr (sizeof(T) == 4) {
      *reinterpret_cast<float4 *>(q + e * q_stride + k) =
          make_float4(__fsub_rn(xb.x, xa.x), __fsub_rn(xb.y, xa.y), __fsub_rn(xb.z, xa.z), __fsub_rn(xb.w, xa.w));
    }
  } else {
    q[e * q_stride + k] = x[b * x_stride + k] - x[a * x_stride + k];
  }
}

// ------------------------------------------------------------------ launch

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Launch one op (0 grad, 1 div, 2 curl) with the direct kernels; with q
// (edge variant) the neighbour differences come from the per-edge array.
int launch_direct(const nb_method *m, int op, const nb_field *in, const nb_field *out,
                  cudaStream_t st, const void *q, int64_t q_stride) {
  const nb_mesh *mesh = m->mesh;
  const bool f64 = in->dtype == NB_F64;
  DirectArgs a;
  a.V = mesh->V;
  a.cap_begin = mesh->cap_begin;
  a.nlev = in->nlev;
  a.row_ptr = m->d_row_ptr;
  a.nbr = m->d_nbr;
  a.w32 = op == 0 ? (const void *)m->d_wgrad32 : op == 1 ? (const void *)m->d_wdiv32 : (const void *)m->d_wcurl32;
  a.w64 = op == 0 ? (const void *)m->d_wgrad64 : op == 1 ? (const void *)m->d_wdiv64 : (const void *)m->d_wcurl64;
  a.s32 = op == 2 ? (const void *)m->d_scurl32 : (const void *)m->d_sdiv32;
  a.s64 = op == 2 ? (const void *)m->d_scurl64 : (const void *)m->d_sdiv64;
  a.in = in->data;
  a.in_stride = in->node_stride;
  a.out = out->data;
  a.out_stride = out->node_stride;
  a.q = q;
  a.q_stride = q_stride;
  a.nbr_edge = m->d_nbr_edge;
  a.E = mesh->E;
  a.status = nullptr;
#ifdef NB_BOUNDS_CHECK
  if (const int rc = status_word(&a.status)) return rc;
#endif
  const bool edge = q != nullptr;
  // 16-byte vectors need aligned bases and strides that are multiples of 4 floats
  const bool vec = !f64 && in->nlev >= 4 && aligned16(in->data) && aligned16(out->data) &&
                   in->node_stride % 4 == 0 && out->node_stride % 4 == 0 && (!edge || q_stride % 4 == 0);
  const int LPT = f64 ? 2 : (vec ? 4 : 1);
  a.ngroups = (in->nlev + LPT - 1) / LPT;
  const int threads = 256;
  const int64_t items = a.V * a.ngroups;
  const int64_t blocks = (items + threads - 1) / threads;
  if (blocks > 0x7fffffff) {
    set_error("launch: problem too large for one grid");
    return NB_EINVAL;
  }
  const bool comp = m->compensated != 0;
  const unsigned nb = (unsigned)blocks;
  if (edge) {
    if (f64) {
      if (op == 0) grad_direct_f64<2, true><<<nb, threads, 0, st>>>(a);
      else divcurl_direct_f64<2, true><<<nb, threads, 0, st>>>(a);
    } else if (vec) {
      if (op == 0) {
        if (comp) grad_direct_f32<4, KahanAcc, true><<<nb, threads, 0, st>>>(a);
        else grad_direct_f32<4, PlainAcc, true><<<nb, threads, 0, st>>>(a);
      } else {
        if (comp) divcurl_direct_f32<4, KahanAcc, true><<<nb, threads, 0, st>>>(a);
        else divcurl_direct_f32<4, PlainAcc, true><<<nb, threads, 0, st>>>(a);
      }
    } else {
      if (op == 0) {
        if (comp) grad_direct_f32<1, KahanAcc, true><<<nb, threads, 0, st>>>(a);
        else grad_direct_f32<1, PlainAcc, true><<<nb, threads, 0, st>>>(a);
      } else {
        if (comp) divcurl_direct_f32<1, KahanAcc, true><<<nb, threads, 0, st>>>(a);
        else divcurl_direct_f32<1, PlainAcc, true><<<nb, threads, 0, st>>>(a);
      }
    }
  } else if (f64) {
    if (op == 0) grad_direct_f64<2><<<nb, threads, 0, st>>>(a);
    else divcurl_direct_f64<2><<<nb, threads, 0, st>>>(a);
  } else if (vec) {
    if (op == 0) {
      if (comp) grad_direct_f32<4, KahanAcc><<<nb, threads, 0, st>>>(a);
      else grad_direct_f32<4, PlainAcc><<<nb, threads, 0, st>>>(a);
    } else {
      if (comp) divcurl_direct_f32<4, KahanAcc><<<nb, threads, 0, st>>>(a);
      else divcurl_direct_f32<4, PlainAcc><<<nb, threads, 0, st>>>(a);
    }
  } else {
    if (op == 0) {
      if (comp) grad_direct_f32<1, KahanAcc><<<nb, threads, 0, st>>>(a);
      else grad_direct_f32<1, PlainAcc><<<nb, threads, 0, st>>>(a);
    } else {
      if (comp) divcurl_direct_f32<1, KahanAcc><<<nb, threads, 0, st>>>(a);
      else divcurl_direct_f32<1, PlainAcc><<<nb, threads, 0, st>>>(a);
    }
  }
  count_launch(1);
  NB_CUDA(cudaGetLastError());
  return NB_OK;
}

// Edge variant (the EdgeColumns pattern, Sec. 4.5): materialise the
// difference of every edge's end columns, q[e] = x[b] - x[a] (E x nlev x
// nvar values, stream-ordered scratch), then reduce per node from q through
// the node -> edge connectivity.  Results equal the direct kernels' bit for
// bit; the point of the variant is the cost of the extra pass and traffic.
int launch_edge(nb_method *m, int op, const nb_field *in, const nb_field *out, cudaStream_t st) {
  const bool f64 = in->dtype == NB_F64;
  const int64_t elem = f64 ? 8 : 4;
  const int q4 = f64 ? 2 : 4;
  const int64_t lq = (int64_t)((in->nlev + q4 - 1) / q4) * q4;
  const int64_t q_stride = lq * in->nvar;
  const int64_t E = m->mesh->E;
  const size_t bytes = (size_t)(E * q_stride * elem);
  void *q = nullptr;
  const DevAlloc alloc = current_allocator();
  int rc = dev_alloc_async(alloc, &q, bytes, st, "edge variant scratch");
  if (rc != NB_OK) return rc;
  const int nvals = in->nlev * in->nvar;
  const bool vec = !f64 && aligned16(in->data) && in->node_stride % 4 == 0;
  const int per = vec ? (nvals + 3) / 4 : nvals;
  const int64_t blocks = (E * per + 255) / 256;
  if (blocks > 0x7fffffff) {
    dev_free_async(alloc, q, bytes, st);
    set_error("edge variant: problem too large for one grid");
    return NB_EINVAL;
  }
  if (f64)
    edge_diff_kernel<double, false><<<(unsigned)blocks, 256, 0, st>>>(
        E, m->d_edge, static_cast<const double *>(in->data), in->node_stride, nvals, static_cast<double *>(q),
        q_stride);
  else if (vec)
    edge_diff_kernel<float, true><<<(unsigned)blocks, 256, 0, st>>>(
        E, m->d_edge, static_cast<const float *>(in->data), in->node_stride, nvals, static_cast<float *>(q),
        q_stride);
  else
    edge_diff_kernel<float, false><<<(unsigned)blocks, 256, 0, st>>>(
        E, m->d_edge, static_cast<const float *>(in->data), in->node_stride, nvals, static_cast<float *>(q),
        q_stride);
  count_launch(1);
  if ((rc = cudaGetLastError()) != cudaSuccess) {
    dev_free_async(alloc, q, bytes, st);
    return cuda_fail((cudaError_t)rc, "edge_diff_kernel");
  }
  rc = launch_direct(m, op, in, out, st, q, q_stride);
  const int rf = dev_free_async(alloc, q, bytes, st);
  return rc != NB_OK ? rc : rf;
}

}  // namespace nb
