// capi.cu -- extern "C" boundary of the library (declared in
// include/nabla_b300.h): handle lifetimes, argument validation and the
// dispatch of each nabla operator to its kernels.  No C++ exception crosses
// this file's functions.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <cstdio>
#include <cstdarg>
#include <chrono>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>

#include "internal.h"
#include "kernels_common.cuh"

namespace nb {

static thread_local std::string t_last_error;
void set_error(const std::string &msg) { t_last_error = msg; }

// NB_DEBUG=1 (or 2) logs the library's setup steps to stderr: mesh and method
// builds, tile plans, kernel shapes; 2 adds one line per operator launch.
// Read once per process.
int log_level() {
  static const int level = [] {
    const char *v = std::getenv("NB_DEBUG");
    return v ? std::max(0, std::atoi(v)) : 0;
  }();
  return level;
}

void log_msg(int level, const char *fmt, ...) {
  if (log_level() < level) return;
  static std::mutex mu;
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  std::lock_guard<std::mutex> lk(mu);
  std::fprintf(stderr, "[nabla_b300] %s\n", buf);
}

static std::mutex g_alloc_mu;
static DevAlloc g_alloc;

DevAlloc current_allocator() {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  return g_alloc;
}

int dev_alloc(const DevAlloc &a, void **ptr, size_t bytes, const char *what) {
  *ptr = nullptr;
  if (!a.user.alloc) {
    const cudaError_t e = cudaMalloc(ptr, bytes);
    if (e == cudaSuccess) return NB_OK;
    *ptr = nullptr;
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      set_error(std::string(what) + ": cudaMalloc of " + std::to_string(bytes) + " bytes failed");
      return NB_EOOM;
    }
    return cuda_fail(e, what);
  }
  *ptr = a.user.alloc(a.user.ctx, (int64_t)bytes, nullptr);
  if (*ptr) return NB_OK;
  set_error(std::string(what) + ": allocator callback returned NULL for " + std::to_string(bytes) +
            " bytes");
  return NB_EOOM;
}

void dev_free(const DevAlloc &a, void *ptr, size_t bytes) {
  if (!ptr) return;
  if (a.user.release)
    a.user.release(a.user.ctx, ptr, (int64_t)bytes, nullptr);
  else
    cudaFree(ptr);
}

int dev_alloc_async(const DevAlloc &a, void **ptr, size_t bytes, void *stream, const char *what) {
  *ptr = nullptr;
  if (!a.user.alloc) {
    const cudaError_t e = cudaMallocAsync(ptr, bytes, static_cast<cudaStream_t>(stream));
    if (e == cudaSuccess) return NB_OK;
    *ptr = nullptr;
    return cuda_fail(e, what);
  }
  *ptr = a.user.alloc(a.user.ctx, (int64_t)bytes, stream);
  if (*ptr) return NB_OK;
  set_error(std::string(what) + ": allocator callback returned NULL for " + std::to_string(bytes) +
            " bytes");
  return NB_EOOM;
}

int dev_free_async(const DevAlloc &a, void *ptr, size_t bytes, void *stream) {
  if (!ptr) return NB_OK;
  if (a.user.release) {
    a.user.release(a.user.ctx, ptr, (int64_t)bytes, stream);
    return NB_OK;
  }
  const cudaError_t e = cudaFreeAsync(ptr, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? NB_OK : cuda_fail(e, "cudaFreeAsync");
}

int launch_fused_lap(nb_method *m, const nb_field *f, const nb_field *lap, const nb_field *g, cudaStream_t st,
                     bool *handled);
int lap_plan_info(const nb_mesh *mesh, int nlev, int32_t *ntiles, int32_t *ntiles_main, int32_t *max_gnodes,
                  int32_t *fits);
int launch_tiled(nb_method *m, int op, const nb_field *in, const nb_field *out, const nb_field *out2,
                 cudaStream_t st, bool *handled, int comp = -1);
int device_status(int clear, int *code);

}  // namespace nb

nb_method::~nb_method() {
  nb::method_free_device(this);
  nb::release(mesh);
}

using nb::set_error;

#define NB_GUARD_BEGIN try {
#define NB_GUARD_END                                      \
  }                                                       \
  catch (const std::bad_alloc &) {                        \
    set_error("host allocation failed");                  \
    return NB_EOOM;                                       \
  }                                                       \
  catch (const std::exception &ex) {                      \
    set_error(ex.what());                                 \
    return NB_EINVAL;                                     \
  }                                                       \
  catch (...) {                                           \
    set_error("unknown C++ exception");                   \
    return NB_EINVAL;                                     \
  }

#define NB_REQUIRE(cond, code, msg) \
  do {                              \
    if (!(cond)) {                  \
      set_error(msg);               \
      return code;                  \
    }                               \
  } while (0)

extern "C" {

#ifdef NB_BOUNDS_CHECK
const char *nb_version(void) { return "nabla_b300 0.1.0 sm_103a bounds-checked"; }
#else
const char *nb_version(void) { return "nabla_b300 0.1.0 sm_103a"; }
#endif

const char *nb_last_error(void) { return nb::t_last_error.c_str(); }

int nb_set_allocator(const nb_allocator *a) {
  NB_REQUIRE(!a || (a->alloc && a->release), NB_EINVAL,
             "nb_set_allocator: alloc and release must both be set");
  std::lock_guard<std::mutex> lk(nb::g_alloc_mu);
  nb::g_alloc.user = a ? *a : nb_allocator{};
  return NB_OK;
}

int nb_launch_count(int64_t *count) {
  NB_REQUIRE(count, NB_EINVAL, "nb_launch_count: NULL");
  *count = nb::launch_count();
  return NB_OK;
}

int nb_device_status(int clear, int32_t *code) {
  NB_REQUIRE(code, NB_EINVAL, "nb_device_status: NULL");
  int c = 0;
  const int st = nb::device_status(clear, &c);
  *code = c;
  return st;
}

// ------------------------------------------------------------------ grid

int nb_grid_create_octahedral(int N, nb_grid **out) {
  NB_REQUIRE(out, NB_EINVAL, "nb_grid_create_octahedral: out is NULL");
  NB_REQUIRE(N >= 1 && N <= 8000, NB_EINVAL, "nb_grid_create_octahedral: N must be in [1, 8000]");
  NB_GUARD_BEGIN
  *out = nb::build_grid(N);
  return NB_OK;
  NB_GUARD_END
}

int nb_grid_create_regular(int N, nb_grid **out) {
  NB_REQUIRE(out, NB_EINVAL, "nb_grid_create_regular: out is NULL");
  NB_REQUIRE(N >= 1 && N <= 8000, NB_EINVAL, "nb_grid_create_regular: N must be in [1, 8000]");
  NB_GUARD_BEGIN
  *out = nb::build_grid_pl(N, std::vector<int32_t>(2 * N, 4 * N));
  return NB_OK;
  NB_GUARD_END
}

int nb_grid_create_reduced(int nrows, const int32_t *pl, nb_grid **out) {
  NB_REQUIRE(out && pl, NB_EINVAL, "nb_grid_create_reduced: NULL argument");
  NB_REQUIRE(nrows >= 2 && nrows % 2 == 0 && nrows <= 16000, NB_EINVAL,
             "nb_grid_create_reduced: nrows must be even, in [2, 16000]");
  int64_t V = 0;
  for (int j = 0; j < nrows; ++j) {
    NB_REQUIRE(pl[j] >= 3, NB_EINVAL, "nb_grid_create_reduced: every row needs at least 3 points");
    V += pl[j];
  }
  NB_REQUIRE(V <= INT32_MAX, NB_EINVAL, "nb_grid_create_reduced: more than 2^31 - 1 points");
  NB_GUARD_BEGIN
  *out = nb::build_grid_pl(nrows / 2, std::vector<int32_t>(pl, pl + nrows));
  return NB_OK;
  NB_GUARD_END
}

int nb_grid_create_named(const char *name, nb_grid **out) {
  NB_REQUIRE(name && out, NB_EINVAL, "nb_grid_create_named: NULL argument");
  const char family = name[0];
  char *end = nullptr;
  const long N = std::strtol(name + 1, &end, 10);
  NB_REQUIRE(name[1] >= '0' && name[1] <= '9' && end && *end == '\0', NB_EINVAL,
             "nb_grid_create_named: expected O<N> or F<N>");
  NB_REQUIRE(family != 'N', NB_EINVAL,
             "nb_grid_create_named: classic N<N> grids need their tabulated PL array "
             "(nb_grid_create_reduced)");
  NB_REQUIRE(N >= 1 && N <= 8000, NB_EINVAL, "nb_grid_create_named: N must be in [1, 8000]");
  if (family == 'O') return nb_grid_create_octahedral((int)N, out);
  if (family == 'F') return nb_grid_create_regular((int)N, out);
  set_error("nb_grid_create_named: expected O<N> or F<N>");
  return NB_EINVAL;
}

int nb_grid_release(nb_grid *g) {
  nb::release(g);
  return NB_OK;
}

int nb_grid_pl(const nb_grid *g, int32_t *pl) {
  NB_REQUIRE(g && pl, NB_EINVAL, "nb_grid_pl: NULL argument");
  std::memcpy(pl, g->nx.data(), sizeof(int32_t) * g->nx.size());
  return NB_OK;
}

int nb_grid_size(const nb_grid *g, int64_t *nodes) {
  NB_REQUIRE(g && nodes, NB_EINVAL, "nb_grid_size: NULL argument");
  *nodes = g->V;
  return NB_OK;
}

int nb_grid_gaussian_number(const nb_grid *g, int *N) {
  NB_REQUIRE(g && N, NB_EINVAL, "nb_grid_gaussian_number: NULL argument");
  *N = g->N;
  return NB_OK;
}

int nb_grid_lonlat(const nb_grid *g, double *lonlat) {
  NB_REQUIRE(g && lonlat, NB_EINVAL, "nb_grid_lonlat: NULL argument");
  const double pi = 3.14159265358979323846;
  for (int j = 0; j < 2 * g->N; ++j) {
    const double phi = std::asin(g->mu[j]);
    for (int i = 0; i < g->nx[j]; ++i) {
      const int64_t id = g->row_off[j] + i;
      lonlat[2 * id] = 2.0 * pi * (double)i / (double)g->nx[j];
      lonlat[2 * id + 1] = phi;
    }
  }
  return NB_OK;
}

// ------------------------------------------------------------------ mesh

int nb_mesh_create(const nb_grid *g, int reorder, nb_mesh **out) {
  NB_REQUIRE(g && out, NB_EINVAL, "nb_mesh_create: NULL argument");
  NB_REQUIRE(reorder == 0 || reorder == 1, NB_EINVAL, "nb_mesh_create: reorder must be 0 or 1");
  NB_GUARD_BEGIN
  const auto t0 = std::chrono::steady_clock::now();
  *out = nb::build_mesh(const_cast<nb_grid *>(g), reorder);
  nb::log_msg(1, "mesh: %lld nodes, %lld edges, %lld triangles, %s order, built in %.3f s", (long long)(*out)->V,
              (long long)(*out)->E, (long long)(*out)->F, reorder ? "Hilbert" : "grid",
              std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
  return NB_OK;
  NB_GUARD_END
}

int nb_mesh_release(nb_mesh *m) {
  nb::release(m);
  return NB_OK;
}

int nb_mesh_sizes(const nb_mesh *m, int64_t *nodes, int64_t *edges, int64_t *tris) {
  NB_REQUIRE(m, NB_EINVAL, "nb_mesh_sizes: NULL mesh");
  if (nodes) *nodes = m->V;
  if (edges) *edges = m->E;
  if (tris) *tris = m->F;
  return NB_OK;
}

int nb_mesh_permutation(const nb_mesh *m, int32_t *perm) {
  NB_REQUIRE(m && perm, NB_EINVAL, "nb_mesh_permutation: NULL argument");
  std::memcpy(perm, m->perm.data(), sizeof(int32_t) * m->V);
  return NB_OK;
}

int nb_mesh_triangles(const nb_mesh *m, int32_t *tri) {
  NB_REQUIRE(m && tri, NB_EINVAL, "nb_mesh_triangles: NULL argument");
  std::memcpy(tri, m->tri.data(), sizeof(int32_t) * 3 * m->F);
  return NB_OK;
}

int nb_mesh_edges(const nb_mesh *m, int32_t *edge) {
  NB_REQUIRE(m && edge, NB_EINVAL, "nb_mesh_edges: NULL argument");
  std::memcpy(edge, m->edge.data(), sizeof(int32_t) * 2 * m->E);
  return NB_OK;
}

int nb_mesh_csr(const nb_mesh *m, int64_t *row_ptr, int32_t *nbr) {
  NB_REQUIRE(m && row_ptr && nbr, NB_EINVAL, "nb_mesh_csr: NULL argument");
  std::memcpy(row_ptr, m->row_ptr.data(), sizeof(int64_t) * (m->V + 1));
  std::memcpy(nbr, m->nbr.data(), sizeof(int32_t) * m->nbr.size());
  return NB_OK;
}

int nb_mesh_node_pairs(const nb_mesh *m, int32_t *mate) {
  NB_REQUIRE(m && mate, NB_EINVAL, "nb_mesh_node_pairs: NULL argument");
  std::memcpy(mate, m->mate.data(), sizeof(int32_t) * m->V);
  return NB_OK;
}

int nb_mesh_tile_plan(const nb_mesh *m, int rcap, int nmax, int32_t *ntiles, int32_t *ntiles_main,
                      int64_t *nhalo, int32_t *node0, int32_t *halo_ptr, int32_t *halo,
                      uint16_t *lnbr) {
  NB_REQUIRE(m && ntiles && ntiles_main && nhalo, NB_EINVAL, "nb_mesh_tile_plan: NULL argument");
  NB_REQUIRE(rcap >= 1 && rcap <= 65535 && nmax >= 1 && nmax <= 1024, NB_EINVAL,
             "nb_mesh_tile_plan: rcap in [1, 65535], nmax in [1, 1024]");
  NB_GUARD_BEGIN
  std::vector<int32_t> n0, hp, h;
  std::vector<uint16_t> ln;
  int mh = 0, me = 0, nm = 0;
  nb::build_tile_plan_host(m, rcap, nmax, 1 << 20, n0, hp, h, ln, mh, me, nm);
  *ntiles = (int32_t)n0.size() - 1;
  *ntiles_main = nm;
  *nhalo = (int64_t)h.size();
  if (node0) std::memcpy(node0, n0.data(), sizeof(int32_t) * n0.size());
  if (halo_ptr) std::memcpy(halo_ptr, hp.data(), sizeof(int32_t) * hp.size());
  if (halo) std::memcpy(halo, h.data(), sizeof(int32_t) * h.size());
  if (lnbr) std::memcpy(lnbr, ln.data(), sizeof(uint16_t) * ln.size());
  return NB_OK;
  NB_GUARD_END
}

int nb_check_tile_plan(const nb_mesh *m, int32_t ntiles, const int32_t *node0, const int32_t *halo_ptr,
                       const int32_t *halo, const uint16_t *lnbr) {
  NB_REQUIRE(m && node0 && halo_ptr && halo && lnbr, NB_EINVAL, "nb_check_tile_plan: NULL argument");
  NB_GUARD_BEGIN
  std::string why;
  const bool ok = nb::check_tile_plan(m, ntiles, node0, halo_ptr, halo,
                                      [&](int64_t p, int, int64_t) { return (int64_t)lnbr[p]; }, why);
  NB_REQUIRE(ok, NB_EINVAL, "nb_check_tile_plan: " + why);
  return NB_OK;
  NB_GUARD_END
}

int nb_check_slot_lists(const nb_mesh *m, int32_t ntiles, const int32_t *node0, const int32_t *slot_ptr,
                        const int32_t *npairs, const uint32_t *slots, int64_t nslots) {
  NB_REQUIRE(m && node0 && slot_ptr && npairs && slots && ntiles >= 1, NB_EINVAL,
             "nb_check_slot_lists: NULL argument or no tiles");
  NB_GUARD_BEGIN
  std::string why;
  NB_REQUIRE(node0[0] == 0 && node0[ntiles] == m->V, NB_EINVAL, "nb_check_slot_lists: tiles do not cover the nodes");
  for (int32_t t = 0; t < ntiles; ++t)
    NB_REQUIRE(node0[t + 1] > node0[t], NB_EINVAL, "nb_check_slot_lists: tiles out of order");
  // slot ranges inside the caller's array before any slot is read
  NB_REQUIRE(slot_ptr[0] >= 0 && (int64_t)slot_ptr[ntiles] <= nslots, NB_EINVAL,
             "nb_check_slot_lists: slot ranges leave the slot array");
  for (int32_t t = 0; t < ntiles; ++t)
    NB_REQUIRE(slot_ptr[t + 1] >= slot_ptr[t], NB_EINVAL, "nb_check_slot_lists: slot ranges out of order");
  const bool ok = nb::check_slot_lists(m, ntiles, node0, slot_ptr, npairs, slots, why);
  NB_REQUIRE(ok, NB_EINVAL, "nb_check_slot_lists: " + why);
  return NB_OK;
  NB_GUARD_END
}

int nb_mesh_lap_plan(const nb_mesh *m, int nlev, int32_t *ntiles, int32_t *ntiles_main, int32_t *max_gnodes,
                     int32_t *fits) {
  NB_REQUIRE(m && ntiles && ntiles_main && max_gnodes && fits, NB_EINVAL, "nb_mesh_lap_plan: NULL argument");
  NB_REQUIRE(nlev >= 16 && nlev <= 1020, NB_EINVAL, "nb_mesh_lap_plan: nlev in [16, 1020]");
  NB_GUARD_BEGIN
  return nb::lap_plan_info(m, nlev, ntiles, ntiles_main, max_gnodes, fits);
  NB_GUARD_END
}

int nb_mesh_cap_begin(const nb_mesh *m, int64_t *cap_begin) {
  NB_REQUIRE(m && cap_begin, NB_EINVAL, "nb_mesh_cap_begin: NULL argument");
  *cap_begin = m->cap_begin;
  return NB_OK;
}

// ------------------------------------------------------------ partitions

int nb_partition_equal_regions(const nb_grid *g, int nparts, int32_t *part, int32_t *zones,
                               int32_t *nzones) {
  NB_REQUIRE(g && (part || nzones), NB_EINVAL, "nb_partition_equal_regions: NULL argument");
  NB_REQUIRE(nparts >= 1 && nparts <= g->V, NB_EINVAL, "nb_partition_equal_regions: nparts out of range");
  NB_GUARD_BEGIN
  const std::vector<int> z = nb::eq_zone_counts(nparts);
  if (nzones) *nzones = (int32_t)z.size();
  if (zones)
    for (size_t k = 0; k < z.size(); ++k) zones[k] = z[k];
  if (part) {
    std::vector<int32_t> p;
    nb::equal_regions(g, nparts, p);
    std::memcpy(part, p.data(), sizeof(int32_t) * p.size());
  }
  return NB_OK;
  NB_GUARD_END
}

int nb_partition_halo(const nb_mesh *m, const int32_t *part, int p, int64_t *nowned, int32_t *owned,
                      int64_t *nhalo, int32_t *halo) {
  NB_REQUIRE(m && part && nowned && nhalo, NB_EINVAL, "nb_partition_halo: NULL argument");
  NB_GUARD_BEGIN
  std::vector<int32_t> o, h;
  nb::partition_halo(m, part, p, o, h);
  *nowned = (int64_t)o.size();
  *nhalo = (int64_t)h.size();
  if (owned) std::memcpy(owned, o.data(), sizeof(int32_t) * o.size());
  if (halo) std::memcpy(halo, h.data(), sizeof(int32_t) * h.size());
  return NB_OK;
  NB_GUARD_END
}

// ---------------------------------------------------------------- method

int nb_method_create(const nb_mesh *mesh, double radius_m, nb_method **out) {
  NB_REQUIRE(mesh && out, NB_EINVAL, "nb_method_create: NULL argument");
  NB_GUARD_BEGIN
  auto *m = new nb_method();
  m->mesh = nb::retain(const_cast<nb_mesh *>(mesh));
  m->R = radius_m > 0 ? radius_m : 6.37122e6;
  m->alloc = nb::current_allocator();
  nb::build_geometry(mesh, m->R, m->vol, m->S, m->T, m->east, m->north);
  for (double v : m->vol) m->area += v;
  const int st = nb::method_upload(m);
  if (st != NB_OK) {
    nb::release(m);
    return st;
  }
  nb::log_msg(1, "method: R = %.6g m, dual area / (4 pi R^2) - 1 = %.3g, %.1f MB on device %d", m->R,
              m->area / (4.0 * 3.14159265358979323846 * m->R * m->R) - 1.0, m->device_bytes / 1e6, m->device);
  *out = m;
  return NB_OK;
  NB_GUARD_END
}

int nb_method_release(nb_method *m) {
  nb::release(m);
  return NB_OK;
}

int nb_method_dual_volumes(const nb_method *m, double *host_out) {
  NB_REQUIRE(m && host_out, NB_EINVAL, "nb_method_dual_volumes: NULL argument");
  std::memcpy(host_out, m->vol.data(), sizeof(double) * m->vol.size());
  return NB_OK;
}

int nb_method_device_bytes(const nb_method *m, int64_t *bytes) {
  NB_REQUIRE(m && bytes, NB_EINVAL, "nb_method_device_bytes: NULL argument");
  int64_t b = m->device_bytes;
  for (auto &kv : m->plans) b += kv.second->bytes;
  *bytes = b;
  return NB_OK;
}

int nb_method_set_kernel(nb_method *m, int variant, int tile_nodes) {
  NB_REQUIRE(m, NB_EINVAL, "nb_method_set_kernel: NULL method");
  NB_REQUIRE(variant >= NB_KERNEL_AUTO && variant <= NB_KERNEL_EDGE, NB_EINVAL,
             "nb_method_set_kernel: unknown variant");
  NB_REQUIRE(tile_nodes == 0 || (tile_nodes >= 8 && tile_nodes <= 1024), NB_EINVAL,
             "nb_method_set_kernel: tile_nodes must be 0 or in [8, 1024]");
  m->kernel_variant = variant;
  m->tile_nodes = tile_nodes;
  return NB_OK;
}

int nb_method_set_staging(nb_method *m, int nstages, int stage_kb) {
  NB_REQUIRE(m, NB_EINVAL, "nb_method_set_staging: NULL method");
  NB_REQUIRE((nstages == 0 && stage_kb == 0) ||
                 (nstages >= 2 && nstages <= 8 && stage_kb >= 8 && nstages * stage_kb <= 226),
             NB_EINVAL, "nb_method_set_staging: need 2 <= nstages <= 8, stage_kb >= 8, product <= 226");
  m->nstages = nstages;
  m->stage_kb = stage_kb;
  return NB_OK;
}

int nb_method_set_compensated(nb_method *m, int on) {
  NB_REQUIRE(m, NB_EINVAL, "nb_method_set_compensated: NULL method");
  m->compensated = on ? 1 : 0;
  return NB_OK;
}

int nb_method_set_laplacian_route(nb_method *m, int route) {
  NB_REQUIRE(m, NB_EINVAL, "nb_method_set_laplacian_route: NULL method");
  NB_REQUIRE(route == NB_LAP_TWO_PASS || route == NB_LAP_FUSED, NB_EINVAL,
             "nb_method_set_laplacian_route: route must be NB_LAP_TWO_PASS or NB_LAP_FUSED");
  m->lap_route = route;
  return NB_OK;
}

int nb_method_set_item_shape(nb_method *m, int units, int aligned) {
  NB_REQUIRE(m, NB_EINVAL, "nb_method_set_item_shape: NULL method");
  NB_REQUIRE(units == 0 || units == 2 || units == 3, NB_EINVAL,
             "nb_method_set_item_shape: units must be 0 (chosen), 2 or 3");
  NB_REQUIRE(aligned >= -1 && aligned <= 1, NB_EINVAL, "nb_method_set_item_shape: aligned must be -1, 0 or 1");
  m->item_units = units;
  m->item_align = aligned;
  return NB_OK;
}

int nb_method_set_node_pairs(nb_method *m, int mode) {
  NB_REQUIRE(m, NB_EINVAL, "nb_method_set_node_pairs: NULL method");
  NB_REQUIRE(mode >= -1 && mode <= 1, NB_EINVAL, "nb_method_set_node_pairs: mode must be -1, 0 or 1");
  m->node_pairs = mode;
  nb::log_msg(1, "method: node pairs %s", mode > 0 ? "on" : mode == 0 ? "off" : "on except in the fused pass");
  return NB_OK;
}

int nb_method_set_wait_limit(nb_method *m, int64_t limit_ns) {
  NB_REQUIRE(m, NB_EINVAL, "nb_method_set_wait_limit: NULL method");
  NB_REQUIRE(limit_ns >= -1 && limit_ns <= 60000000000ll, NB_EINVAL,
             "nb_method_set_wait_limit: limit_ns must be -1 (default) or in [0, 60 s]");
  m->wait_limit_ns = limit_ns;
  return NB_OK;
}

// --------------------------------------------------------- functionspace

int nb_fs_nodecolumns(const nb_method *m, int nlev, nb_dtype dtype, nb_fs **out) {
  NB_REQUIRE(m && out, NB_EINVAL, "nb_fs_nodecolumns: NULL argument");
  NB_REQUIRE(nlev >= 1 && nlev <= 65536, NB_EINVAL, "nb_fs_nodecolumns: nlev must be in [1, 65536]");
  NB_REQUIRE(dtype == NB_F32 || dtype == NB_F64, NB_EDTYPE, "nb_fs_nodecolumns: dtype must be NB_F32 or NB_F64");
  NB_GUARD_BEGIN
  auto *fs = new nb_fs();
  fs->method = nb::retain(const_cast<nb_method *>(m));
  fs->nlev = nlev;
  fs->dtype = dtype;
  const int q = dtype == NB_F32 ? 4 : 2;
  fs->lp = (int64_t)((nlev + q - 1) / q) * q;
  *out = fs;
  return NB_OK;
  NB_GUARD_END
}

int nb_fs_release(nb_fs *fs) {
  nb::release(fs);
  return NB_OK;
}

int nb_fs_level_stride(const nb_fs *fs, int64_t *lp) {
  NB_REQUIRE(fs && lp, NB_EINVAL, "nb_fs_level_stride: NULL argument");
  *lp = fs->lp;
  return NB_OK;
}

int nb_field_view(const nb_fs *fs, void *dev_ptr, int nvar, int64_t node_stride,
                  int64_t lev_stride, nb_field *out) {
  NB_REQUIRE(fs && out, NB_EINVAL, "nb_field_view: NULL argument");
  NB_REQUIRE(dev_ptr || fs->method->mesh->V == 0, NB_EINVAL, "nb_field_view: NULL data");
  NB_REQUIRE(nvar == 1 || nvar == 2, NB_EINVAL, "nb_field_view: nvar must be 1 or 2");
  NB_REQUIRE(lev_stride == nvar, NB_ESHAPE, "nb_field_view: lev_stride must equal nvar");
  NB_REQUIRE(node_stride >= (int64_t)fs->nlev * nvar, NB_ESHAPE,
             "nb_field_view: node_stride < nlev * nvar");
  out->data = dev_ptr;
  out->dtype = fs->dtype;
  out->nvar = nvar;
  out->nnodes = fs->method->mesh->V;
  out->nlev = fs->nlev;
  out->reserved = 0;
  out->node_stride = node_stride;
  out->lev_stride = lev_stride;
  return NB_OK;
}

}  // extern "C"

// ------------------------------------------------------------- operators

namespace nb {

static int check_field(const nb_method *m, const nb_field *f, int nvar, const char *what) {
  if (!f) {
    set_error(std::string(what) + ": field is NULL");
    return NB_EINVAL;
  }
  if (!f->data && m->mesh->V > 0) {
    set_error(std::string(what) + ": field data is NULL");
    return NB_EINVAL;
  }
  if (f->dtype != NB_F32 && f->dtype != NB_F64) {
    set_error(std::string(what) + ": unknown dtype");
    return NB_EDTYPE;
  }
  if (f->nvar != nvar) {
    set_error(std::string(what) + ": expected nvar = " + std::to_string(nvar));
    return NB_ESHAPE;
  }
  if (f->nnodes != m->mesh->V) {
    set_error(std::string(what) + ": node count differs from the mesh");
    return NB_ESHAPE;
  }
  if (f->nlev < 1 || f->lev_stride != nvar || f->node_stride < (int64_t)f->nlev * nvar) {
    set_error(std::string(what) + ": bad level count or strides");
    return NB_ESHAPE;
  }
  const int64_t elem = f->dtype == NB_F64 ? 8 : 4;
  if (((uintptr_t)f->data) % elem) {
    set_error(std::string(what) + ": data not aligned to its element size");
    return NB_ESHAPE;
  }
  return NB_OK;
}

static int validate(const nb_method *m, int op, const nb_field *in, const nb_field *out,
                    const nb_field *scratch) {
  if (!m) {
    set_error("nabla: method is NULL");
    return NB_EINVAL;
  }
  if (op < NB_OP_GRAD || op > NB_OP_LAP) {
    set_error("nabla: unknown op");
    return NB_EINVAL;
  }
  const int nin = (op == NB_OP_DIV || op == NB_OP_CURL) ? 2 : 1;
  const int nout = op == NB_OP_GRAD ? 2 : 1;
  int st = check_field(m, in, nin, "nabla input");
  if (st) return st;
  if ((st = check_field(m, out, nout, "nabla output"))) return st;
  if (in->dtype != out->dtype) {
    set_error("nabla: input and output dtypes differ");
    return NB_EDTYPE;
  }
  if (in->nlev != out->nlev) {
    set_error("nabla: input and output level counts differ");
    return NB_ESHAPE;
  }
  const int64_t elem = in->dtype == NB_F64 ? 8 : 4;
  auto span = [&](const nb_field *f) {
    const char *b = static_cast<const char *>(f->data);
    return std::make_pair(b, b + ((f->nnodes - 1) * f->node_stride + (int64_t)f->nlev * f->nvar) * elem);
  };
  auto overlap = [&](const nb_field *a, const nb_field *b) {
    auto x = span(a), y = span(b);
    return x.first < y.second && y.first < x.second;
  };
  if (m->mesh->V > 0 && overlap(in, out)) {
    set_error("nabla: output aliases input");
    return NB_EINVAL;
  }
  if (op == NB_OP_LAP && scratch) {
    if ((st = check_field(m, scratch, 2, "laplacian scratch"))) return st;
    if (scratch->dtype != in->dtype || scratch->nlev != in->nlev) {
      set_error("laplacian scratch: dtype or level count differs from input");
      return NB_ESHAPE;
    }
    if (overlap(scratch, in) || overlap(scratch, out)) {
      set_error("laplacian scratch aliases input or output");
      return NB_EINVAL;
    }
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != m->device) {
    set_error("nabla: current CUDA device differs from the method's device");
    return NB_EINVAL;
  }
  return NB_OK;
}

// Argument checks shared with the allocation-free entry point.
int validate_op(const nb_method *m, int op, const nb_field *in, const nb_field *out,
                const nb_field *scratch) {
  return validate(m, op, in, out, scratch);
}

// One of grad, div, curl on the chosen kernel variant.
static int launch_single(nb_method *m, int op, const nb_field *in, const nb_field *out,
                         cudaStream_t st) {
  if (m->kernel_variant == NB_KERNEL_EDGE) return launch_edge(m, op, in, out, st);
  if (m->kernel_variant != NB_KERNEL_DIRECT) {
    bool handled = false;
    const int rc = launch_tiled(m, op, in, out, nullptr, st, &handled);
    if (handled || rc != NB_OK) return rc;
  }
  return launch_direct(m, op, in, out, st);
}

int launch_op(nb_method *m, int op, const nb_field *in, const nb_field *out,
              const nb_field *scratch, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (m->mesh->V == 0) return NB_OK;
  if (op != NB_OP_LAP) return launch_single(m, op, in, out, st);
  if (m->lap_route == NB_LAP_FUSED &&
      (m->kernel_variant == NB_KERNEL_AUTO || m->kernel_variant == NB_KERNEL_TILED)) {
    bool handled = false;
    const int rc = launch_fused_lap(m, in, out, nullptr, st, &handled);
    if (handled || rc != NB_OK) return rc;
  }
  // Laplacian: gradient into scratch, then the divergence of it
  nb_field tmp;
  void *owned = nullptr;
  size_t owned_bytes = 0;
  const DevAlloc alloc = current_allocator();
  if (scratch) {
    tmp = *scratch;
  } else {
    const int64_t elem = in->dtype == NB_F64 ? 8 : 4;
    const int q = in->dtype == NB_F64 ? 2 : 4;
    const int64_t stride = 2 * (int64_t)((in->nlev + q - 1) / q) * q;
    owned_bytes = (size_t)(stride * in->nnodes * elem);
    const int ra = dev_alloc_async(alloc, &owned, owned_bytes, stream, "Laplacian scratch");
    if (ra != NB_OK) return ra;
    tmp = *in;
    tmp.data = owned;
    tmp.nvar = 2;
    tmp.node_stride = stride;
    tmp.lev_stride = 2;
  }
  int rc = launch_single(m, NB_OP_GRAD, in, &tmp, st);
  if (rc == NB_OK) rc = launch_single(m, NB_OP_DIV, &tmp, out, st);
  if (owned) {
    const int rf = dev_free_async(alloc, owned, owned_bytes, stream);
    if (rc == NB_OK) rc = rf;
  }
  return rc;
}

}  // namespace nb

extern "C" {

int nb_nabla_apply(const nb_method *m, int op, const nb_field *in, const nb_field *out,
                   const nb_field *scratch, void *stream) {
  const int st = nb::validate(m, op, in, out, scratch);
  if (st != NB_OK) return st;
  NB_GUARD_BEGIN
  return nb::launch_op(const_cast<nb_method *>(m), op, in, out, scratch, stream);
  NB_GUARD_END
}

int nb_nabla_gradient(const nb_method *m, const nb_field *f, const nb_field *g, void *stream) {
  return nb_nabla_apply(m, NB_OP_GRAD, f, g, nullptr, stream);
}

int nb_nabla_divergence(const nb_method *m, const nb_field *uv, const nb_field *d, void *stream) {
  return nb_nabla_apply(m, NB_OP_DIV, uv, d, nullptr, stream);
}

int nb_nabla_curl(const nb_method *m, const nb_field *uv, const nb_field *z, void *stream) {
  return nb_nabla_apply(m, NB_OP_CURL, uv, z, nullptr, stream);
}

int nb_nabla_divcurl(const nb_method *m, const nb_field *uv, const nb_field *d, const nb_field *z,
                     void *stream) {
  int st = nb::validate(m, NB_OP_DIV, uv, d, nullptr);
  if (st != NB_OK) return st;
  if ((st = nb::validate(m, NB_OP_CURL, uv, z, nullptr)) != NB_OK) return st;
  NB_REQUIRE(d->node_stride == z->node_stride && d->lev_stride == z->lev_stride, NB_ESHAPE,
             "nb_nabla_divcurl: d and z must have the same layout");
  {
    const int64_t elem = d->dtype == NB_F64 ? 8 : 4;
    const char *d0 = static_cast<const char *>(d->data), *z0 = static_cast<const char *>(z->data);
    const int64_t span = (d->nnodes - 1) * d->node_stride * elem + (int64_t)d->nlev * elem;
    NB_REQUIRE(d->nnodes == 0 || d0 + span <= z0 || z0 + span <= d0, NB_ESHAPE,
               "nb_nabla_divcurl: d and z overlap");
  }
  NB_GUARD_BEGIN
  nb_method *mm = const_cast<nb_method *>(m);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (mm->mesh->V == 0) return NB_OK;
  if (mm->kernel_variant == NB_KERNEL_AUTO || mm->kernel_variant == NB_KERNEL_TILED) {
    bool handled = false;
    const int rc = nb::launch_tiled(mm, NB_OP_DIV, uv, d, z, s, &handled);
    if (handled || rc != NB_OK) return rc;
  }
  st = nb::launch_op(mm, NB_OP_DIV, uv, d, nullptr, stream);
  if (st == NB_OK) st = nb::launch_op(mm, NB_OP_CURL, uv, z, nullptr, stream);
  return st;
  NB_GUARD_END
}

int nb_nabla_gradlap(const nb_method *m, const nb_field *f, const nb_field *g, const nb_field *lap,
                     void *stream) {
  int st = nb::validate(m, NB_OP_GRAD, f, g, nullptr);
  if (st != NB_OK) return st;
  // g also serves as the Laplacian's scratch: same checks (no aliasing)
  if ((st = nb::validate(m, NB_OP_LAP, f, lap, g)) != NB_OK) return st;
  NB_GUARD_BEGIN
  nb_method *mm = const_cast<nb_method *>(m);
  if (mm->mesh->V == 0) return NB_OK;
  if (mm->lap_route == NB_LAP_FUSED &&
      (mm->kernel_variant == NB_KERNEL_AUTO || mm->kernel_variant == NB_KERNEL_TILED)) {
    bool handled = false;
    const int rc = nb::launch_fused_lap(mm, f, lap, g, static_cast<cudaStream_t>(stream), &handled);
    if (handled || rc != NB_OK) return rc;
  }
  // the Laplacian's gradient pass is g: its divergence pass reads it
  st = nb::launch_op(const_cast<nb_method *>(m), NB_OP_GRAD, f, g, nullptr, stream);
  if (st == NB_OK) st = nb::launch_op(const_cast<nb_method *>(m), NB_OP_DIV, g, lap, nullptr, stream);
  return st;
  NB_GUARD_END
}

int nb_nabla_laplacian(const nb_method *m, const nb_field *f, const nb_field *lap,
                       const nb_field *scratch, void *stream) {
  return nb_nabla_apply(m, NB_OP_LAP, f, lap, scratch, stream);
}

static int field_copy(void *dst, const void *src, const nb_field *f, cudaMemcpyKind kind, void *stream,
                      const char *who) {
  NB_REQUIRE(f && dst && src, NB_EINVAL, std::string(who) + ": NULL argument");
  NB_REQUIRE(f->dtype == NB_F32 || f->dtype == NB_F64, NB_EDTYPE, std::string(who) + ": unknown dtype");
  NB_REQUIRE(f->nnodes >= 0 && f->node_stride >= 0, NB_EINVAL, std::string(who) + ": negative size");
  const size_t bytes = (size_t)(f->nnodes * f->node_stride * (f->dtype == NB_F64 ? 8 : 4));
  if (bytes == 0) return NB_OK;
  NB_CUDA(cudaMemcpyAsync(dst, src, bytes, kind, static_cast<cudaStream_t>(stream)));
  return NB_OK;
}

int nb_field_upload(const nb_field *dev, const void *host, void *stream) {
  return field_copy(dev ? dev->data : nullptr, host, dev, cudaMemcpyHostToDevice, stream, "nb_field_upload");
}

int nb_field_download(void *host, const nb_field *dev, void *stream) {
  return field_copy(host, dev ? dev->data : nullptr, dev, cudaMemcpyDeviceToHost, stream, "nb_field_download");
}

int nb_nabla_apply_host(const nb_method *m, int op, const void *host_in, void *host_out,
                        const nb_field *dev_in, const nb_field *dev_out,
                        const nb_field *scratch, void *stream) {
  NB_REQUIRE(host_in && host_out, NB_EINVAL, "nb_nabla_apply_host: NULL host buffer");
  int st = nb::validate(m, op, dev_in, dev_out, scratch);
  if (st != NB_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t elem = dev_in->dtype == NB_F64 ? 8 : 4;
  const size_t bin = (size_t)(dev_in->nnodes * dev_in->node_stride * elem);
  const size_t bout = (size_t)(dev_out->nnodes * dev_out->node_stride * elem);
  NB_CUDA(cudaMemcpyAsync(dev_in->data, host_in, bin, cudaMemcpyHostToDevice, s));
  NB_GUARD_BEGIN
  st = nb::launch_op(const_cast<nb_method *>(m), op, dev_in, dev_out, scratch, stream);
  NB_GUARD_END
  if (st != NB_OK) return st;
  NB_CUDA(cudaMemcpyAsync(host_out, dev_out->data, bout, cudaMemcpyDeviceToHost, s));
  NB_CUDA(cudaStreamSynchronize(s));
  return NB_OK;
}

}  // extern "C"
