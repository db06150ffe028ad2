// server.cu -- continuous-batching request server for derived fields.
//
// A request asks for one nabla operator on 1..8 fields of a resident grid
// with a given number of levels.  A request's fields are packed side by
// side along the level axis into column blocks ([node][field][level]) of at
// most kBlockLevels levels, so one synthesis launch and one operator launch
// (two for a Laplacian) serve all fields of a block; the operators act on
// each level independently, so every field's result is the one it gets
// alone.  A worker thread admits arriving requests in
// arrival order while the device-memory budget and the in-flight limit allow,
// takes stream-ordered memory for the request's fields from the CUDA memory
// pool, synthesises the input fields on the device from the grid's resident
// spherical-harmonic bases (per-level mixing weights drawn from the request
// seed with SplitMix64, mixed in FP32), launches the operator on one of several streams and
// records a completion event.  Finished requests (event polled) release their
// memory and budget immediately, so requests that arrive while others are on
// the GPU are admitted as memory frees up and their work overlaps on the
// device.  The same engine with one stream, one request in flight and FP64
// fields gives the sequential plain-FP64 baseline.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "kernels_common.cuh"

namespace nb {

int validate_op(const nb_method *m, int op, const nb_field *in, const nb_field *out,
                const nb_field *scratch);

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the output function of a
// 64-bit counter-based generator.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Mixing weight of basis b at level k of field f: uniform in [-1, 1) scaled
// by 1 + k / nlev.
__device__ __forceinline__ double mix_weight(uint64_t seed, int f, int k, int b, int nlev) {
  const uint64_t z = splitmix64(seed ^ ((uint64_t)f << 40) ^ ((uint64_t)k << 8) ^ (uint64_t)b);
  const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
  return (2.0 * u - 1.0) * (1.0 + (double)k / nlev);
}

// Mixing weights of all fields of a request: w[f][k][b], drawn once.
__global__ void __launch_bounds__(256) synth_weights_kernel(uint64_t seed, int nfields, int nlev,
                                                            float *w) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nfields * nlev * 8) return;
  const int f = t / (nlev * 8), r = t - f * nlev * 8;
  w[t] = (float)mix_weight(seed, f, r >> 3, r & 7, nlev);
}

// in[node][k][c] = sum_b w[k][b] basis[node][b][c]  (c < nvar), in FP32
// arithmetic from an FP32 copy of the basis (these are request inputs, not
// operator arithmetic).  A CTA takes kSynthNodes consecutive nodes: it
// stages the block's mixing weights (transposed, [b][level], zero past nlev)
// and its nodes' basis values in shared memory.  A lane owns one level of a
// 32-level chunk (its 8 weights in registers, each duplicated into a packed
// pair) and a warp walks the nodes, so stores are contiguous and basis loads
// are broadcasts.  Packed FMAs (__ffma2_rn) carry two sums at once: a wind's
// (u, v), whose basis values sit side by side; for a scalar, the same level
// of two consecutive nodes, whose basis values are staged interleaved.
// Each sum still runs b = 0..7 in order with one rounding per FMA, so the
// values are those of scalar FMAs.  Levels from nlev up to the padded
// stride get 0.
constexpr int kSynthNodes = 64;
constexpr int kSynthThreads = 256;
template <class T>
__global__ void __launch_bounds__(kSynthThreads) synth_fields_kernel(const float *__restrict__ basis, int nvar,
                                                                     int64_t V, int nlev, int64_t stride,
                                                                     const float *__restrict__ wts, T *out) {
  extern __shared__ __align__(16) float sm[];
  const int lb = (int)(stride / nvar);           // padded levels of the column block
  float *wT = sm;                                // [8][lb]
  float *bs = sm + 8 * lb;                       // wind [node][8][2]; scalar [node pair][8][2]
  const int64_t n0 = (int64_t)blockIdx.x * kSynthNodes;
  const int nn = (int)min((int64_t)kSynthNodes, V - n0);
  for (int t = threadIdx.x; t < 8 * lb; t += blockDim.x) {
    const int b = t / lb, k = t - b * lb;
    wT[t] = k < nlev ? __ldg(wts + 8 * k + b) : 0.f;
  }
  if (nvar == 2) {
    for (int t = threadIdx.x; t < nn * 16; t += blockDim.x) bs[t] = __ldg(basis + n0 * 16 + t);
  } else {
    // node i's basis b at (i / 2) * 16 + 2 b + (i & 1); a missing odd node gets 0
    const int np = (nn + 1) >> 1;
    for (int t = threadIdx.x; t < np * 16; t += blockDim.x) {
      const int pr = t >> 4, b = (t >> 1) & 7, i = 2 * pr + (t & 1);
      bs[t] = i < nn ? __ldg(basis + (n0 + i) * 8 + b) : 0.f;
    }
  }
  __syncthreads();
  // lane = level within a 32-level chunk (weights held in registers), warp
  // = a stride over the CTA's nodes (scalar: node pairs)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int k = lane; k - lane < lb; k += 32) {
    if (k >= lb) continue;
    float2 w[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const float x = wT[b * lb + k];
      w[b] = make_float2(x, x);
    }
    if (nvar == 2) {
      for (int il = warp; il < nn; il += nwarps) {
        // the node's (u, v) of bases 2h and 2h + 1: 16-byte broadcast loads
        const float4 *bi = reinterpret_cast<const float4 *>(bs + il * 16);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const float4 p = bi[h];
          acc = __ffma2_rn(w[2 * h], make_float2(p.x, p.y), acc);
          acc = __ffma2_rn(w[2 * h + 1], make_float2(p.z, p.w), acc);
        }
        T *o = out + (n0 + il) * stride + (int64_t)k * 2;
        if constexpr (sizeof(T) == 4) *reinterpret_cast<float2 *>(o) = acc;
        else *reinterpret_cast<double2 *>(o) = make_double2((double)acc.x, (double)acc.y);
      }
    } else {
      for (int ip = warp; 2 * ip < nn; ip += nwarps) {
        // bases b, b + 1 of nodes 2 ip and 2 ip + 1, interleaved
        const float4 *bi = reinterpret_cast<const float4 *>(bs + ip * 16);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const float4 p = bi[h];
          acc = __ffma2_rn(w[2 * h], make_float2(p.x, p.y), acc);
          acc = __ffma2_rn(w[2 * h + 1], make_float2(p.z, p.w), acc);
        }
        const int64_t i = n0 + 2 * ip;
        out[i * stride + k] = (T)acc.x;
        if (2 * ip + 1 < nn) out[(i + 1) * stride + k] = (T)acc.y;
      }
    }
  }
}

struct SrvGrid {
  nb_method *method = nullptr;
  float *d_scalar = nullptr;  // [V][8]
  float *d_wind = nullptr;    // [V][8][2]
};

struct SrvReq {
  uint64_t ticket = 0;
  nb_request r{};
  double arrival = 0, admit = -1, done = -1;
  int status = NB_OK;
  int64_t bytes = 0, node_levels = 0;
  int stream = -1;
  cudaEvent_t ev = nullptr;
  std::vector<void *> bufs;
  void *wts = nullptr;         // mixing weights of the request's fields
  std::vector<char> host_out;  // kept outputs (tests)
  std::vector<char> host_in;   // kept inputs (keep_output == 2)
  int fail_at = -1;            // injected failure: index of the refused allocation
  int nalloc = 0;              // device allocations made so far
};

// One device allocation of a request from the stream-ordered pool.  The
// allocation the fault injector marks (nb_server_inject_failure) is refused
// as a full pool would refuse it.
static int req_alloc(SrvReq *q, void **p, size_t bytes, cudaStream_t st) {
  if (q->nalloc++ == q->fail_at) {
    set_error("server request: device allocation refused (injected failure)");
    return NB_EOOM;
  }
  NB_CUDA(cudaMallocAsync(p, bytes, st));
  return NB_OK;
}

}  // namespace nb

struct nb_server : nb::RefCounted {
  int device = 0;
  int64_t budget = 0;
  int max_inflight = 0;
  std::vector<cudaStream_t> streams;
  std::map<int, nb::SrvGrid> grids;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<nb::SrvReq *> pending;  // arrived, not admitted
  std::vector<nb::SrvReq *> inflight;
  std::map<uint64_t, nb::SrvReq *> all;
  std::map<uint64_t, int> inject;  // request seed -> index of the allocation to refuse
  std::atomic<uint64_t> next_ticket{1};
  int64_t used = 0, peak_used = 0;
  int rr = 0;
  bool stop = false;
  std::thread worker;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  ~nb_server() override;
};

namespace nb {

// Column blocks: fields per block, and the level stride of a block of nf
// fields (padded so that columns start on 16 bytes).  Blocks stay within the
// column heights the staged kernels handle well.
constexpr int kBlockLevels = 144;
static int fields_per_block(const nb_request &r) {
  return std::max(1, std::min(r.nfields, kBlockLevels / std::max(1, r.nlev)));
}
static int64_t block_stride(const nb_request &r, int nf) {
  const int q = r.dtype == NB_F64 ? 2 : 4;
  return ((int64_t)nf * r.nlev + q - 1) / q * q;
}

static int64_t req_bytes(const nb_server *s, const nb_request &r, int64_t V) {
  const int64_t elem = r.dtype == NB_F64 ? 8 : 4;
  const int in_var = (r.op == NB_OP_DIV || r.op == NB_OP_CURL) ? 2 : 1;
  const int out_var = r.op == NB_OP_GRAD ? 2 : 1;
  const int scr_var = r.op == NB_OP_LAP ? 2 : 0;
  (void)s;
  const int fpb = fields_per_block(r);
  int64_t levels = 0;
  for (int f0 = 0; f0 < r.nfields; f0 += fpb) levels += block_stride(r, std::min(fpb, r.nfields - f0));
  return V * levels * elem * (in_var + out_var + scr_var);
}

// Enqueue one admitted request on its stream (caller holds no lock).
static int launch_request(nb_server *s, SrvReq *q) {
  const nb_request &r = q->r;
  SrvGrid &g = s->grids[r.N];
  nb_method *m = g.method;
  const int64_t V = m->mesh->V;
  cudaStream_t st = s->streams[q->stream];
  const int64_t elem = r.dtype == NB_F64 ? 8 : 4;
  const int in_var = (r.op == NB_OP_DIV || r.op == NB_OP_CURL) ? 2 : 1;
  const int out_var = r.op == NB_OP_GRAD ? 2 : 1;
  float *wts = nullptr;
  const int nw = r.nfields * r.nlev * 8;
  if (const int rc = req_alloc(q, (void **)&wts, (size_t)nw * sizeof(float), st)) return rc;
  q->wts = wts;
  synth_weights_kernel<<<(nw + 255) / 256, 256, 0, st>>>(r.seed, r.nfields, r.nlev, wts);
  count_launch(1);
  NB_CUDA(cudaGetLastError());
  const float *basis = in_var == 2 ? g.d_wind : g.d_scalar;
  const int fpb = fields_per_block(r);
  for (int f0 = 0; f0 < r.nfields; f0 += fpb) {
    const int nf = std::min(fpb, r.nfields - f0);
    const int nl = nf * r.nlev;  // levels of the block in use
    const int64_t lb = block_stride(r, nf);
    void *din = nullptr, *dout = nullptr, *dscr = nullptr;
    if (const int rc = req_alloc(q, &din, (size_t)(V * lb * in_var * elem), st)) return rc;
    q->bufs.push_back(din);
    if (const int rc = req_alloc(q, &dout, (size_t)(V * lb * out_var * elem), st)) return rc;
    q->bufs.push_back(dout);
    if (r.op == NB_OP_LAP) {
      if (const int rc = req_alloc(q, &dscr, (size_t)(V * lb * 2 * elem), st)) return rc;
      q->bufs.push_back(dscr);
    }
    // weights are [field][level][basis]: the block's are contiguous
    const float *wb = wts + (size_t)f0 * r.nlev * 8;
    const unsigned blocks = (unsigned)((V + kSynthNodes - 1) / kSynthNodes);
    const size_t smem = sizeof(float) * (size_t)(8 * lb + kSynthNodes * 8 * in_var);
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
      // columns of up to 4096 levels: 8 x 4096 weights + the nodes' bases
      const int bytes = (int)(sizeof(float) * (8 * 4096 + kSynthNodes * 16));
      attr_err = cudaFuncSetAttribute(synth_fields_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      if (attr_err == cudaSuccess)
        attr_err = cudaFuncSetAttribute(synth_fields_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    });
    NB_CUDA(attr_err);
    if (r.dtype == NB_F64)
      synth_fields_kernel<double><<<blocks, kSynthThreads, smem, st>>>(basis, in_var, V, nl, lb * in_var, wb,
                                                                       static_cast<double *>(din));
    else
      synth_fields_kernel<float><<<blocks, kSynthThreads, smem, st>>>(basis, in_var, V, nl, lb * in_var, wb,
                                                                      static_cast<float *>(din));
    count_launch(1);
    NB_CUDA(cudaGetLastError());
    nb_field fi{din, r.dtype, in_var, V, nl, 0, lb * in_var, in_var};
    nb_field fo{dout, r.dtype, out_var, V, nl, 0, lb * out_var, out_var};
    nb_field fsc{dscr, r.dtype, 2, V, nl, 0, lb * 2, 2};
    const int rc = launch_op(m, r.op, &fi, &fo, r.op == NB_OP_LAP ? &fsc : nullptr, st);
    if (rc != NB_OK) return rc;
  }
  NB_CUDA(cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming));
  NB_CUDA(cudaEventRecord(q->ev, st));
  return NB_OK;
}

// Copy field j of a column block (level stride lb) to host memory laid out
// as [V][lp][nvar] at `host` (padding levels left as they are).
static void copy_field_out(char *host, const void *dev, int64_t V, int64_t lb, int64_t lp, int nlev,
                           int nvar, int64_t elem, int j) {
  const size_t dpitch = (size_t)(lp * nvar * elem), spitch = (size_t)(lb * nvar * elem);
  cudaMemcpy2D(host, dpitch, static_cast<const char *>(dev) + (size_t)j * nlev * nvar * elem, spitch,
               (size_t)(nlev * nvar * elem), (size_t)V, cudaMemcpyDeviceToHost);
}

static void finish_request(nb_server *s, SrvReq *q) {
  cudaStream_t st = s->streams[q->stream];
  if (q->r.keep_output && q->status == NB_OK) {
    // per block: the input block, the output block (and the Laplacian scratch)
    const nb_request &r = q->r;
    const int per = r.op == NB_OP_LAP ? 3 : 2;
    const int64_t V = s->grids[r.N].method->mesh->V;
    const int64_t elem = r.dtype == NB_F64 ? 8 : 4;
    const int qq = r.dtype == NB_F64 ? 2 : 4;
    const int64_t lp = (int64_t)((r.nlev + qq - 1) / qq) * qq;
    const int in_var = (r.op == NB_OP_DIV || r.op == NB_OP_CURL) ? 2 : 1;
    const int out_var = r.op == NB_OP_GRAD ? 2 : 1;
    const int64_t one = V * lp * out_var * elem, ione = V * lp * in_var * elem;
    q->host_out.assign((size_t)(one * r.nfields), 0);
    if (r.keep_output == 2) q->host_in.assign((size_t)(ione * r.nfields), 0);
    const int fpb = fields_per_block(r);
    for (int f = 0; f < r.nfields; ++f) {
      const int blk = f / fpb, j = f - blk * fpb;
      const int64_t lb = block_stride(r, std::min(fpb, r.nfields - blk * fpb));
      copy_field_out(q->host_out.data() + f * one, q->bufs[blk * per + 1], V, lb, lp, r.nlev, out_var, elem, j);
      if (r.keep_output == 2)
        copy_field_out(q->host_in.data() + f * ione, q->bufs[blk * per], V, lb, lp, r.nlev, in_var, elem, j);
    }
  }
  for (void *p : q->bufs) cudaFreeAsync(p, st);
  q->bufs.clear();
  if (q->wts) cudaFreeAsync(q->wts, st);
  q->wts = nullptr;
  if (q->ev) cudaEventDestroy(q->ev);
  q->ev = nullptr;
}

static void worker_loop(nb_server *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    // retire finished requests
    for (size_t k = 0; k < s->inflight.size();) {
      SrvReq *q = s->inflight[k];
      const cudaError_t e = cudaEventQuery(q->ev);
      if (e == cudaErrorNotReady) {
        ++k;
        continue;
      }
      if (e != cudaSuccess) q->status = NB_ECUDA;
      // the result is published (done >= 0) only once its outputs are kept
      const double t_done = s->now();
      lk.unlock();
      finish_request(s, q);
      lk.lock();
      q->done = t_done;
      s->used -= q->bytes;
      s->inflight.erase(s->inflight.begin() + (long)k);
      s->cv.notify_all();
    }
    // admit in arrival order while budget and slots allow
    while (!s->pending.empty() && (int)s->inflight.size() < s->max_inflight) {
      SrvReq *q = s->pending.front();
      if (s->used + q->bytes > s->budget) break;
      s->pending.pop_front();
      s->used += q->bytes;
      s->peak_used = std::max(s->peak_used, s->used);
      q->admit = s->now();
      // least-loaded stream: the one with the fewest in-flight requests
      std::vector<int> load(s->streams.size(), 0);
      for (SrvReq *o : s->inflight) load[o->stream]++;
      q->stream = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      s->inflight.push_back(q);
      lk.unlock();
      const int rc = launch_request(s, q);
      lk.lock();
      if (rc != NB_OK) {
        log_msg(1, "server: request %llu (op %d, O%d, %d levels, %d fields) failed with status %d",
                (unsigned long long)q->ticket, q->r.op, q->r.N, q->r.nlev, q->r.nfields, rc);
        q->status = rc;
        if (!q->ev) {  // nothing to wait for: retire now
          const double t_done = s->now();
          lk.unlock();
          finish_request(s, q);
          lk.lock();
          q->done = t_done;
          s->used -= q->bytes;
          s->inflight.erase(std::find(s->inflight.begin(), s->inflight.end(), q));
          s->cv.notify_all();
        }
      }
    }
    if (s->stop && s->pending.empty() && s->inflight.empty()) return;
    if (s->inflight.empty())
      s->cv.wait_for(lk, std::chrono::milliseconds(2));
    else {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    }
  }
}

}  // namespace nb

nb_server::~nb_server() {
  {
    std::lock_guard<std::mutex> lk(mu);
    stop = true;
  }
  cv.notify_all();
  if (worker.joinable()) worker.join();
  for (auto &kv : all) delete kv.second;
  for (auto &kv : grids) {
    if (kv.second.d_scalar) cudaFree(kv.second.d_scalar);
    if (kv.second.d_wind) cudaFree(kv.second.d_wind);
    nb::release(kv.second.method);
  }
  for (cudaStream_t st : streams) cudaStreamDestroy(st);
}

extern "C" {

int nb_server_create(int64_t hbm_budget, int nstreams, int max_inflight, nb_server **out) {
  if (!out || hbm_budget <= 0 || nstreams < 1 || nstreams > 64 || max_inflight < 1) {
    nb::set_error("nb_server_create: need out, budget > 0, 1 <= nstreams <= 64, max_inflight >= 1");
    return NB_EINVAL;
  }
  try {
    auto *s = new nb_server();
    s->budget = hbm_budget;
    s->max_inflight = max_inflight;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
      delete s;
      nb::set_error("nb_server_create: no CUDA device");
      return NB_ECUDA;
    }
    for (int k = 0; k < nstreams; ++k) {
      cudaStream_t st;
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        nb::set_error("nb_server_create: stream creation failed");
        return NB_ECUDA;
      }
      s->streams.push_back(st);
    }
    // keep freed request memory in the pool instead of returning it
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    s->worker = std::thread(nb::worker_loop, s);
    *out = s;
    return NB_OK;
  } catch (...) {
    nb::set_error("nb_server_create: host allocation failed");
    return NB_EOOM;
  }
}

int nb_server_release(nb_server *s) {
  nb::release(s);
  return NB_OK;
}

int nb_server_add_grid(nb_server *s, const nb_method *m, const double *scalar_basis,
                       const double *wind_basis) {
  if (!s || !m || !scalar_basis || !wind_basis) {
    nb::set_error("nb_server_add_grid: NULL argument");
    return NB_EINVAL;
  }
  const int N = m->mesh->grid->N;
  const int64_t V = m->mesh->V;
  nb::SrvGrid g;
  g.method = nb::retain(const_cast<nb_method *>(m));
  std::vector<float> sb((size_t)(V * 8)), wb((size_t)(V * 16));
  for (size_t k = 0; k < sb.size(); ++k) sb[k] = (float)scalar_basis[k];
  for (size_t k = 0; k < wb.size(); ++k) wb[k] = (float)wind_basis[k];
  if (cudaMalloc(&g.d_scalar, sb.size() * 4) != cudaSuccess ||
      cudaMalloc(&g.d_wind, wb.size() * 4) != cudaSuccess ||
      cudaMemcpy(g.d_scalar, sb.data(), sb.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(g.d_wind, wb.data(), wb.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
    if (g.d_scalar) cudaFree(g.d_scalar);
    if (g.d_wind) cudaFree(g.d_wind);
    nb::release(g.method);
    nb::set_error("nb_server_add_grid: device allocation or copy failed");
    return NB_EOOM;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->grids.find(N);
  if (it != s->grids.end()) {
    cudaFree(it->second.d_scalar);
    cudaFree(it->second.d_wind);
    nb::release(it->second.method);
  }
  s->grids[N] = g;
  return NB_OK;
}

int nb_server_submit(nb_server *s, const nb_request *r, uint64_t *ticket) {
  if (!s || !r || !ticket) {
    nb::set_error("nb_server_submit: NULL argument");
    return NB_EINVAL;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto g = s->grids.find(r->N);
  if (g == s->grids.end()) {
    nb::set_error("nb_server_submit: grid O" + std::to_string(r->N) + " is not resident");
    return NB_EINVAL;
  }
  if (r->op < NB_OP_GRAD || r->op > NB_OP_LAP || r->nlev < 1 || r->nlev > 4096 || r->nfields < 1 ||
      r->nfields > 64 || (r->dtype != NB_F32 && r->dtype != NB_F64)) {
    nb::set_error("nb_server_submit: bad op, nlev, nfields or dtype");
    return NB_EINVAL;
  }
  auto *q = new nb::SrvReq();
  q->r = *r;
  {
    auto fi = s->inject.find(r->seed);
    if (fi != s->inject.end()) q->fail_at = fi->second;
  }
  q->bytes = nb::req_bytes(s, *r, g->second.method->mesh->V);
  if (q->bytes > s->budget) {
    delete q;
    nb::set_error("nb_server_submit: request needs more memory than the whole budget");
    return NB_EBUDGET;
  }
  q->node_levels = (int64_t)r->nfields * g->second.method->mesh->V * r->nlev;
  q->ticket = s->next_ticket.fetch_add(1);
  q->arrival = s->now();
  s->all[q->ticket] = q;
  s->pending.push_back(q);
  *ticket = q->ticket;
  lk.unlock();
  s->cv.notify_all();
  return NB_OK;
}

int nb_server_inject_failure(nb_server *s, uint64_t seed, int32_t alloc_index) {
  if (!s || alloc_index < -1) {
    nb::set_error("nb_server_inject_failure: NULL server or alloc_index < -1");
    return NB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (alloc_index < 0) s->inject.erase(seed);
  else s->inject[seed] = alloc_index;
  return NB_OK;
}

// NB_OK with the result when the request has finished; NB_ETIMEOUT if it is
// still queued or running after waiting up to timeout_ms (0 = just look).
int nb_server_wait(nb_server *s, uint64_t ticket, double timeout_ms, nb_result *res) {
  if (!s || !res) {
    nb::set_error("nb_server_wait: NULL argument");
    return NB_EINVAL;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) {
    nb::set_error("nb_server_wait: unknown ticket");
    return NB_EINVAL;
  }
  nb::SrvReq *q = it->second;
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::microseconds((int64_t)(timeout_ms * 1000.0));
  while (q->done < 0) {
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout && q->done < 0) return NB_ETIMEOUT;
  }
  res->ticket = q->ticket;
  res->status = q->status;
  res->reserved = 0;
  res->arrival_s = q->arrival;
  res->admit_s = q->admit;
  res->done_s = q->done;
  res->node_levels = q->node_levels;
  res->bytes = q->bytes;
  return NB_OK;
}

int nb_server_poll(nb_server *s, uint64_t ticket, int32_t *done, nb_result *res) {
  if (!s || !done || !res) {
    nb::set_error("nb_server_poll: NULL argument");
    return NB_EINVAL;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) {
      nb::set_error("nb_server_poll: unknown ticket");
      return NB_EINVAL;
    }
    if (it->second->done < 0) {
      *done = 0;
      return NB_OK;
    }
  }
  *done = 1;
  return nb_server_wait(s, ticket, 0.0, res);
}

int nb_server_output(nb_server *s, uint64_t ticket, void *host_out, int64_t bytes) {
  if (!s || !host_out) {
    nb::set_error("nb_server_output: NULL argument");
    return NB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end() || it->second->done < 0 || !it->second->r.keep_output) {
    nb::set_error("nb_server_output: unknown, unfinished or output not kept");
    return NB_EINVAL;
  }
  if ((int64_t)it->second->host_out.size() != bytes) {
    nb::set_error("nb_server_output: size mismatch");
    return NB_ESHAPE;
  }
  std::memcpy(host_out, it->second->host_out.data(), (size_t)bytes);
  return NB_OK;
}

int nb_server_input(nb_server *s, uint64_t ticket, void *host_in, int64_t bytes) {
  if (!s || !host_in) {
    nb::set_error("nb_server_input: NULL argument");
    return NB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end() || it->second->done < 0 || it->second->r.keep_output != 2) {
    nb::set_error("nb_server_input: unknown, unfinished or inputs not kept");
    return NB_EINVAL;
  }
  if ((int64_t)it->second->host_in.size() != bytes) {
    nb::set_error("nb_server_input: size mismatch");
    return NB_ESHAPE;
  }
  std::memcpy(host_in, it->second->host_in.data(), (size_t)bytes);
  return NB_OK;
}

int nb_server_stats(nb_server *s, int64_t *used, int64_t *peak_used, int32_t *pending,
                    int32_t *inflight) {
  if (!s) {
    nb::set_error("nb_server_stats: NULL server");
    return NB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (used) *used = s->used;
  if (peak_used) *peak_used = s->peak_used;
  if (pending) *pending = (int32_t)s->pending.size();
  if (inflight) *inflight = (int32_t)s->inflight.size();
  return NB_OK;
}

// Replay a trace: request k is submitted at arrival_s[k] seconds after the
// call starts (host clock, sleeping between arrivals), then the call waits
// for all of them and fills results[k] (times relative to the call start).
int nb_server_run_trace(nb_server *s, const nb_request *reqs, const double *arrival_s, int n,
                        nb_result *results) {
  if (!s || (n > 0 && (!reqs || !arrival_s || !results)) || n < 0) {
    nb::set_error("nb_server_run_trace: NULL argument");
    return NB_EINVAL;
  }
  std::vector<uint64_t> tickets(n, 0);
  const double base = s->now();
  for (int k = 0; k < n; ++k) {
    for (;;) {
      const double wait = base + arrival_s[k] - s->now();
      if (wait <= 0) break;
      if (wait > 2e-3) std::this_thread::sleep_for(std::chrono::microseconds((int64_t)((wait - 1e-3) * 1e6)));
    }
    const int rc = nb_server_submit(s, &reqs[k], &tickets[k]);
    if (rc != NB_OK) return rc;
  }
  for (int k = 0; k < n; ++k) {
    const int rc = nb_server_wait(s, tickets[k], 3.6e6, &results[k]);
    if (rc != NB_OK) return rc;
    results[k].arrival_s -= base;
    results[k].admit_s -= base;
    results[k].done_s -= base;
  }
  return NB_OK;
}

}  // extern "C"
