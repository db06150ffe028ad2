// internal.h -- library-private types shared by the host builder, the CUDA
// kernels and the C ABI implementation.
#pragma once

#include <atomic>
#include <functional>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/nabla_b300.h"

namespace nb {

void set_error(const std::string &msg);
// stderr logging when NB_DEBUG >= level (capi.cu)
int log_level();
void log_msg(int level, const char *fmt, ...);

// Source of library-owned device memory: the caller's nb_allocator, or the
// CUDA runtime when user.alloc is NULL (capi.cu).
struct DevAlloc {
  nb_allocator user{};
};
struct DevBlock {
  void *ptr;
  size_t bytes;
};
DevAlloc current_allocator();
// Long-lived blocks (stream NULL): cudaMalloc/cudaFree or the callbacks.
int dev_alloc(const DevAlloc &a, void **ptr, size_t bytes, const char *what);
void dev_free(const DevAlloc &a, void *ptr, size_t bytes);
// Stream-ordered scratch: cudaMallocAsync/cudaFreeAsync or the callbacks.
int dev_alloc_async(const DevAlloc &a, void **ptr, size_t bytes, void *stream, const char *what);
int dev_free_async(const DevAlloc &a, void *ptr, size_t bytes, void *stream);

// Intrusive reference count shared by every handle type.
struct RefCounted {
  std::atomic<int> refs{1};
  virtual ~RefCounted() = default;
};
template <class T>
inline T *retain(T *p) {
  if (p) p->refs.fetch_add(1);
  return p;
}
template <class T>
inline void release(T *p) {
  if (p && p->refs.fetch_sub(1) == 1) delete p;
}

}  // namespace nb

// Reduced Gaussian grid (Sec. 4.2.3.7): octahedral O<N>, regular F<N>, or
// any PL array.
struct nb_grid : nb::RefCounted {
  int N = 0;
  int64_t V = 0;
  std::vector<int32_t> nx;       // points per row, 2N rows north to south
  std::vector<int64_t> row_off;  // first grid index of each row, 2N+1
  std::vector<double> mu;        // sin(latitude) of each row (Legendre roots)
};

// Triangulated mesh in functionspace numbering.
struct nb_mesh : nb::RefCounted {
  nb_grid *grid = nullptr;
  int64_t V = 0, E = 0, F = 0;
  int64_t cap_begin = 0;             // nodes [cap_begin, V) are pole-row nodes
  std::vector<int32_t> perm;         // new -> old (grid index)
  std::vector<int32_t> iperm;        // old -> new
  std::vector<double> xyz;           // [V][3] unit position, new order
  std::vector<double> lat, lon;      // per node, new order
  std::vector<int32_t> tri;          // [F][3] CCW, new numbering
  // node -> neighbour CSR, neighbours ascending except in the rows of
  // paired nodes: (shared A, shared B, partner, the other three ascending)
  std::vector<int64_t> row_ptr;      // V+1
  std::vector<int32_t> nbr;          // 2E neighbour node
  std::vector<int32_t> nbr_edge;     // 2E edge id
  std::vector<int32_t> nbr_left;     // 2E triangle left of (i -> j)
  std::vector<int32_t> nbr_right;    // 2E triangle right of (i -> j)
  std::vector<int32_t> edge;         // [E][2] a < b
  std::vector<int32_t> edge_tri;     // [E][2] (left, right) of a -> b
  std::vector<int32_t> mate;         // [V] partner of a paired node, -1 if unpaired (pair_nodes)
  ~nb_mesh() override { nb::release(grid); }
};

// Per-tile halo plan of the staged kernels for one stage layout.
struct TilePlan {
  int64_t area = 0;      // stage bytes for columns
  int64_t row_bytes = 0; // column pitch of the tile's own nodes
  int64_t copy_bytes = 0;// bytes copied per column (halo pitch)
  int nmax = 0;          // nodes per tile at most
  int ecap = 0;          // CSR entries per tile at most
  int pole_cap = 1;      // nodes per pole-row tile at most
  int ntiles = 0;
  int ntiles_main = 0;               // tiles before the pole block
  int max_halo = 0;
  int max_entries = 0;
  int64_t bytes = 0;
  int32_t *d_tile_node0 = nullptr;   // ntiles+1: tile t = [node0[t], node0[t+1])
  int32_t *d_halo_ptr = nullptr;     // ntiles+1
  int32_t *d_halo = nullptr;         // halo node ids
  uint32_t *d_loff = nullptr;        // 2E (+4): stage byte offset of each CSR neighbour
  // node pairs: tile t's slots d_slots[d_slot_ptr[t] .. d_slot_ptr[t + 1])
  // (padded to a multiple of 4), own node li | partner lj << 16, the first
  // d_npairs[t] of them pairs, then single nodes (li | li << 16)
  int32_t *d_slot_ptr = nullptr;     // ntiles+1
  int32_t *d_npairs = nullptr;       // ntiles
  uint32_t *d_slots = nullptr;
  int64_t paired_nodes = 0;          // own nodes that fall in a pair slot
};

// Device side of a single-pass Laplacian plan (fusedlap.cu).
struct LapPlan {
  int ntiles = 0, ntiles_main = 0, max_gnodes = 0;
  int64_t bytes = 0;
  int32_t *d_tile_node0 = nullptr, *d_halo_ptr = nullptr, *d_halo = nullptr, *d_r1_count = nullptr;
  int32_t *d_gn_ptr = nullptr, *d_rec_ptr = nullptr;
  uint32_t *d_gn = nullptr, *d_goff = nullptr;
  void *d_rec = nullptr;  // float4 records
};

// fvm::Method: geometry and operator weights resident on one device.
struct nb_method : nb::RefCounted {
  nb_mesh *mesh = nullptr;
  double R = 0;
  int device = 0;
  std::vector<double> vol;          // [V]
  double area = 0;                  // sum of vol (4 pi R^2 to rounding)
  std::vector<double> S, T;         // [E][3]
  std::vector<double> east, north;  // [V][3]
  // device: connectivity
  int32_t *d_row_ptr = nullptr;     // V+1 (2E < 2^31 for N <= 8000)
  int32_t *d_nbr = nullptr;         // 2E
  int32_t *d_nbr_edge = nullptr;    // 2E
  int32_t *d_edge = nullptr;        // [E][2] a < b
  // device: FP64 raw geometry
  double *d_vol = nullptr, *d_S = nullptr, *d_T = nullptr, *d_east = nullptr, *d_north = nullptr;
  // device: per CSR entry operator weights (FP64 and FP32 rounding)
  //   grad: (gx, gy); div: (du, dv); curl: (cu, cv); per node self (su, sv), (tu, tv)
  double *d_wgrad64 = nullptr, *d_wdiv64 = nullptr, *d_wcurl64 = nullptr;
  double *d_sdiv64 = nullptr, *d_scurl64 = nullptr;
  float *d_wgrad32 = nullptr, *d_wdiv32 = nullptr, *d_wcurl32 = nullptr;
  float *d_sdiv32 = nullptr, *d_scurl32 = nullptr;
  float *d_wdc32 = nullptr, *d_sdc32 = nullptr;  // fused div+curl: float4 records
  int64_t device_bytes = 0;
  nb::DevAlloc alloc;                // allocator current at creation
  std::vector<nb::DevBlock> blocks;  // every device block of the method and its plans
  // kernel control
  int kernel_variant = 0;  // NB_KERNEL_*
  int tile_nodes = 0;   // staged kernels: nodes per tile at most (0 = 256)
  int nstages = 0;      // staged kernels: pipeline stages (0 = default)
  int stage_kb = 0;     // staged kernels: KB per stage (0 = default)
  int compensated = 1;
  int64_t wait_limit_ns = -1;  // staged kernels' pipeline wait limit (-1 = default)
  int item_units = 0;   // staged div / curl: 2-level units per item (0 = chosen per column)
  int item_align = -1;  // staged div / curl: items per node a multiple of 8 (1), not (0), chosen (-1)
  int node_pairs = -1;  // staged kernels: node pairs always (1), never (0), all but the fused pass (-1)
  std::mutex plan_mu;
  std::map<std::tuple<int64_t, int64_t, int64_t, int, int, int>, std::unique_ptr<TilePlan>> plans;
  std::map<std::tuple<int64_t, int64_t, int64_t, int64_t, int64_t, int, int>, std::unique_ptr<LapPlan>> lap_plans;
  int lap_route = 0;    // Laplacian: 0 two passes, 1 single fused pass (FP32 staged)
  ~nb_method() override;
};

struct nb_fs : nb::RefCounted {
  nb_method *method = nullptr;
  int nlev = 0;
  nb_dtype dtype = NB_F32;
  int64_t lp = 0;
  ~nb_fs() override { nb::release(method); }
};

namespace nb {

// partitions (partition.cpp)
std::vector<int> eq_zone_counts(int nparts);
void equal_regions(const nb_grid *g, int nparts, std::vector<int32_t> &part);
void partition_halo(const nb_mesh *m, const int32_t *part, int p, std::vector<int32_t> &owned,
                    std::vector<int32_t> &halo);

// host builders (host_mesh.cpp)
nb_grid *build_grid(int N);                                   // O<N>
nb_grid *build_grid_pl(int N, const std::vector<int32_t> &nx);  // any PL array of 2N rows
nb_mesh *build_mesh(nb_grid *grid, int reorder);
void build_geometry(const nb_mesh *m, double R, std::vector<double> &vol, std::vector<double> &S,
                    std::vector<double> &T, std::vector<double> &east, std::vector<double> &north);
// host side of a tile plan: node0[ntiles+1], halo_ptr[ntiles+1], halo[], lnbr[2E]
void build_tile_plan_host(const nb_mesh *m, int rcap, int nmax, int ecap, std::vector<int32_t> &node0,
                          std::vector<int32_t> &halo_ptr, std::vector<int32_t> &halo,
                          std::vector<uint16_t> &lnbr, int &max_halo, int &max_entries,
                          int &ntiles_main);

// pole_cap: nodes per pole-row tile at most
void build_tile_plan_bytes(const nb_mesh *m, int64_t area, int64_t row_bytes, int64_t copy_bytes,
                           int nmax, int ecap, int pole_cap, std::vector<int32_t> &node0,
                           std::vector<int32_t> &halo_ptr, std::vector<int32_t> &halo,
                           std::vector<uint32_t> &loff, int &max_halo, int &max_entries,
                           int &ntiles_main);

// Stage layout of the single-pass Laplacian (sizes in bytes): f columns of
// own nodes at row_bytes pitch, of ring nodes in groups of four at gpitch
// (copy_bytes each), within farea; g columns at g_pitch for at most gcap
// g-nodes; at most nmax own nodes, ecap own CSR entries, rcap g-phase
// records (the CSR entries of own and ring-1 nodes).
struct LapLayout {
  int64_t row_bytes = 0, copy_bytes = 0, gpitch = 0, farea = 0, g_pitch = 0;
  int64_t nmax = 0, gcap = 0, ecap = 0, rcap = 0;
};
struct LapPlanHost {
  std::vector<int32_t> node0;     // ntiles + 1
  int ntiles_main = 0;
  std::vector<int32_t> halo_ptr;  // ntiles + 1: ring 1 then ring 2 of each tile, each sorted
  std::vector<int32_t> r1_count;  // ntiles
  std::vector<int32_t> halo;
  std::vector<int32_t> gn_ptr;    // ntiles + 1: g-node entries of each tile (own, ring 1, end)
  std::vector<uint32_t> gn;       // record start relative to the tile | 0x80000000 for pole-row nodes
  std::vector<int32_t> rec_ptr;   // ntiles + 1
  std::vector<int32_t> rec_p;     // per record: CSR index of the entry
  std::vector<uint32_t> rec_foff; // per record: staged byte offset of the entry's neighbour's f column
  std::vector<uint32_t> loff;     // per CSR entry of an own node: staged f byte offset of the neighbour
  std::vector<uint32_t> goff;     // per CSR entry of an own node: g byte offset of the neighbour
  int max_gnodes = 0, max_recs = 0;
  bool fits = false;  // every tile, rings counted exactly, fits the layout
};
void build_lap_plan(const nb_mesh *m, const LapLayout &layout, int nmax, int pole_cap, LapPlanHost &out);
bool check_tile_plan(const nb_mesh *m, int ntiles, const int32_t *node0, const int32_t *halo_ptr,
                     const int32_t *halo, const std::function<int64_t(int64_t, int, int64_t)> &slot,
                     std::string &why);
bool check_slot_lists(const nb_mesh *m, int ntiles, const int32_t *node0, const int32_t *slot_ptr,
                      const int32_t *npairs, const uint32_t *slots, std::string &why);

// device side (nabla_kernels.cu)
int method_upload(nb_method *m);            // returns NB_* status
void method_free_device(nb_method *m);
int launch_op(nb_method *m, int op, const nb_field *in, const nb_field *out,
              const nb_field *scratch, void *stream);
int64_t launch_count();

}  // namespace nb
