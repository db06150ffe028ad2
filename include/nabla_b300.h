/*
 * nabla_b300.h -- C ABI of the B300 (sm_103a) library for edge-based
 * median-dual finite-volume nabla operators on octahedral reduced Gaussian
 * grids.
 *
 * The calls follow the paper's concept chain (Sec. 1 Fig. 1-2, Sec. 4.7
 * Listing 12): grid -> mesh -> method (median-dual geometry) ->
 * functionspace (NodeColumns) -> field -> nabla operator.  Every C++ object
 * sits behind a C function, as the paper's Fortran interface does
 * (Sec. 4.1, Fig. 3).
 *
 * Conventions
 *   - Every function returns an int status (NB_OK on success).  No C++
 *     exception crosses this interface.  nb_last_error() returns a
 *     thread-local, human-readable message for the last failing call of the
 *     calling thread.
 *   - Handles are opaque and reference counted.  A mesh keeps its grid alive,
 *     a method its mesh, a functionspace its method.  *_release drops the
 *     caller's reference; passing NULL is a no-op.
 *   - The library owns mesh and geometry memory (host and device).  Field
 *     memory is NEVER owned: an nb_field is a view of caller memory (for
 *     example a torch tensor).  Outputs are preallocated by the caller.
 *   - Operators are asynchronous on the caller's CUDA stream, passed as
 *     `void *stream` (a cudaStream_t; NULL = the legacy default stream).
 *     The first call for a method and column layout builds tile plans
 *     (host work and synchronous uploads); after it, the same calls can be
 *     captured into a CUDA graph (library scratch is stream-ordered).
 *   - Node order of fields is the functionspace (reordered) order, see
 *     nb_mesh_permutation.  Layout is [node][level][var]: a vertical column
 *     is contiguous (Sec. 4.5, Fig. 31) and vector fields carry their local
 *     (east, north) components innermost (Listing 12: variables(2)).
 *   - Sizes and strides are in elements, not bytes.
 */
#ifndef NABLA_B300_H
#define NABLA_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
enum {
  NB_OK = 0,
  NB_EINVAL = 1,   /* bad handle, NULL pointer or out-of-range argument */
  NB_ESHAPE = 2,   /* field shape, stride or alignment does not fit */
  NB_EDTYPE = 3,   /* field dtype does not match the functionspace/op */
  NB_EOOM = 4,     /* host or device allocation failed */
  NB_ECUDA = 5,    /* a CUDA runtime call failed (message has the name) */
  NB_ETIMEOUT = 6, /* a bounded device wait ran out */
  NB_EBUDGET = 7   /* request exceeds the server's HBM budget */
};

typedef enum { NB_F32 = 0, NB_F64 = 1 } nb_dtype;

typedef enum {
  NB_OP_GRAD = 0, /* gradient:   scalar [V][L]    -> vector [V][L][2] */
  NB_OP_DIV = 1,  /* divergence: vector [V][L][2] -> scalar [V][L]    */
  NB_OP_CURL = 2, /* curl:       vector [V][L][2] -> scalar [V][L]    */
  NB_OP_LAP = 3   /* Laplacian:  scalar [V][L]    -> scalar [V][L]    */
} nb_op;

typedef struct nb_grid nb_grid;
typedef struct nb_mesh nb_mesh;
typedef struct nb_method nb_method;
typedef struct nb_fs nb_fs;
typedef struct nb_batch nb_batch;
typedef struct nb_server nb_server;

/* A non-owning view of a field in device memory (Sec. 4.6, Fig. 32). */
typedef struct nb_field {
  void *data;          /* device pointer, caller owned */
  int32_t dtype;       /* nb_dtype */
  int32_t nvar;        /* 1 = scalar, 2 = (east, north) vector */
  int64_t nnodes;      /* number of mesh nodes */
  int32_t nlev;        /* number of vertical levels */
  int32_t reserved;    /* zero */
  int64_t node_stride; /* elements from one node's column to the next */
  int64_t lev_stride;  /* elements from one level to the next; == nvar */
} nb_field;

/* Library version string, e.g. "nabla_b300 0.1.0 sm_103a". */
const char *nb_version(void);

/* Message of the last failing call on this thread ("" if none). */
const char *nb_last_error(void);

/* ------------------------------------------------------ device memory
 *
 * Where the device memory the library owns comes from: method geometry and
 * weights, tile plans, batch tables and batch scratch, and the Laplacian's
 * intermediate gradient when the caller passes no scratch.  (The paper
 * leaves memory to its Array/storage layer, Sec. 5.1-5.2; this hook lets a
 * caller's caching allocator, e.g. torch's, serve these buffers.)
 *
 *   alloc(ctx, bytes, stream) returns at least `bytes` bytes of device
 *     memory on the current device, usable in stream order on `stream`
 *     (NULL = the legacy default stream; used for buffers that live as long
 *     as their object), or NULL on failure -- the library call then fails
 *     with NB_EOOM;
 *   release(ctx, ptr, bytes, stream) gives a block back, with the size and
 *     stream it was allocated with.
 *
 * Both are called on the thread that called into the library, never from
 * a library-owned thread.  An object keeps the allocator that was current
 * when it was created and releases its blocks through it.  The request
 * server (nb_server_*) always uses its own stream-ordered CUDA pool. */
typedef struct nb_allocator {
  void *ctx;
  void *(*alloc)(void *ctx, int64_t bytes, void *stream);
  void (*release)(void *ctx, void *ptr, int64_t bytes, void *stream);
} nb_allocator;

/* Install a copy of *allocator for objects created and calls made from now
 * on, process-wide.  NULL restores the CUDA runtime (cudaMalloc/cudaFree
 * for objects, cudaMallocAsync/cudaFreeAsync on the call's stream for the
 * Laplacian scratch).  Errors: NB_EINVAL if alloc or release is NULL. */
int nb_set_allocator(const nb_allocator *allocator);

/* ------------------------------------------------------------------ grid */

/* Octahedral reduced Gaussian grid O<N> (Sec. 4.2.3.7, Listing 6): 2N
 * latitude rows on the roots of the Legendre polynomial of degree 2N
 * (Sec. 4.2.3.5), row j holding 20 + 4j points counted from the nearer pole,
 * the first point of every row at longitude 0.  N in [1, 8000].
 * Errors: NB_EINVAL (N out of range or out == NULL), NB_EOOM. */
int nb_grid_create_octahedral(int N, nb_grid **out);

/* Regular Gaussian grid F<N> (Sec. 4.2.3.6): 4N points on each of the 2N
 * Gaussian latitude rows.  N in [1, 8000].  Errors as above. */
int nb_grid_create_regular(int N, nb_grid **out);

/* Reduced Gaussian grid from its PL array (Sec. 4.2.3.7): pl[j] points on
 * Gaussian row j (north to south) of nrows = 2N rows.  nrows even and >= 2,
 * every pl[j] >= 3 (a pole ring needs a triangle), at most 2^31 - 1 points in
 * all.  Classic N<N> grids are built this way from their tabulated PL arrays.
 * pl: caller-owned host array, copied.  Errors: NB_EINVAL, NB_EOOM. */
int nb_grid_create_reduced(int nrows, const int32_t *pl, nb_grid **out);

/* Grid by name (Sec. 4.2.3): "O<N>" octahedral, "F<N>" regular.  "N<N>"
 * (classic) needs the tabulated PL array: use nb_grid_create_reduced.
 * Errors: NB_EINVAL (unknown or unsupported name), NB_EOOM. */
int nb_grid_create_named(const char *name, nb_grid **out);
int nb_grid_release(nb_grid *grid);

/* Number of grid points V (4N^2 + 36N for O<N>, 8N^2 for F<N>, the sum of
 * the PL array otherwise). */
int nb_grid_size(const nb_grid *grid, int64_t *nodes);

/* The grid's PL array: points per row, north to south (host int32[2N]). */
int nb_grid_pl(const nb_grid *grid, int32_t *pl);

/* Gaussian number N of the grid. */
int nb_grid_gaussian_number(const nb_grid *grid, int *N);

/* Longitude and latitude in radians of every point, original grid order
 * (rows north to south, points west to east; Sec. 4.2.3, Listing 5).
 * lonlat: caller-owned host array [V][2] = (lon, lat). */
int nb_grid_lonlat(const nb_grid *grid, double *lonlat);

/* ------------------------------------------------------------------ mesh */

/* Triangulate the grid (structured mesh generator, Sec. 4.3, Listing 7,
 * Fig. 25b): row strips joined by an exact integer longitude merge, pole
 * caps closed with no extra node (an odd ring by one last triangle), so
 * F = 2V - 4 and E = 3V - 6.
 * reorder: 0 keeps grid order, 1 renumbers nodes along a 3-D Hilbert curve
 * for memory locality; in both the nodes of the first and last row come
 * last (see nb_mesh_cap_begin).  Runs on the host, multi-threaded.
 * Errors: NB_EINVAL, NB_EOOM. */
int nb_mesh_create(const nb_grid *grid, int reorder, nb_mesh **out);
int nb_mesh_release(nb_mesh *mesh);

int nb_mesh_sizes(const nb_mesh *mesh, int64_t *nodes, int64_t *edges, int64_t *triangles);

/* perm[new] = old: the grid index (global_index, Sec. 4.4) of every node in
 * functionspace order.  perm: caller-owned host int32[V]. */
int nb_mesh_permutation(const nb_mesh *mesh, int32_t *perm);

/* Counter-clockwise triangles [F][3] in functionspace numbering (host). */
int nb_mesh_triangles(const nb_mesh *mesh, int32_t *tri);

/* Edges [E][2] (a < b, functionspace numbering) (host). */
int nb_mesh_edges(const nb_mesh *mesh, int32_t *edge);

/* Node -> neighbour CSR in functionspace numbering (host): row_ptr[V+1],
 * nbr[2E].  Each node's neighbours are ascending, except in the rows of
 * paired nodes (nb_mesh_node_pairs), which start with the two neighbours
 * the pair shares, ascending, then the partner, then the other three
 * ascending.  Every operator sums a node's edge terms in this row order. */
int nb_mesh_csr(const nb_mesh *mesh, int64_t *row_ptr, int32_t *nbr);

/* Node pairs of the FP32 staged kernels (host): mate[V] is the
 * partner of each paired node, -1 for an unpaired one.  A pair is two
 * adjacent six-neighbour nodes outside the pole rows, at most 16 places
 * apart in functionspace order, with exactly two common neighbours,
 * matched greedily along the node order.  When both nodes of a pair are
 * own nodes of one staged tile, one consumer thread evaluates both from
 * the 10 columns they span instead of 14 (the shared neighbours and the
 * partner's own column are read once); results are the same bits as the
 * single-node evaluation (nb_method_set_node_pairs).
 * mate: caller-owned host int32[V].  Errors: NB_EINVAL. */
int nb_mesh_node_pairs(const nb_mesh *mesh, int32_t *mate);

/* Tile plan of the shared-memory staged kernels (host, for inspection):
 * tiles of consecutive nodes, grown while own nodes + halo nodes <= rcap and
 * nodes <= nmax.  Call with NULL arrays to get *ntiles and *nhalo; then pass
 * node0[ntiles+1], halo_ptr[ntiles+1], halo[nhalo] and lnbr[2E] (staged row
 * of every CSR neighbour: k < n is the tile's node k, n + h its halo node h).
 * *ntiles_main counts the tiles before the pole block; here the pole block is
 * one node per tile (the staged kernels cut it into at most one tile per
 * CTA of their persistent grid). */
int nb_mesh_tile_plan(const nb_mesh *mesh, int rcap, int nmax, int32_t *ntiles,
                      int32_t *ntiles_main, int64_t *nhalo, int32_t *node0, int32_t *halo_ptr,
                      int32_t *halo, uint16_t *lnbr);

/* Host-side check of a tile plan in the format nb_mesh_tile_plan returns
 * (ntiles tiles; node0[ntiles + 1], halo_ptr[ntiles + 1], halo[], lnbr[2E]):
 * the tiles cover the nodes in order, each halo entry is a valid node
 * outside its tile, and lnbr maps every CSR neighbour of a tile's node to
 * the staged row holding it (own node k: row k; halo entry h: n + h).  The
 * library runs the same check on each plan of its staged kernels before
 * uploading it, so a corrupted plan is refused before any launch.
 * Errors: NB_EINVAL with the first violation in nb_last_error. */
int nb_check_tile_plan(const nb_mesh *mesh, int32_t ntiles, const int32_t *node0, const int32_t *halo_ptr,
                       const int32_t *halo, const uint16_t *lnbr);

/* Host-side check of the slot lists of a staged plan (ntiles tiles over
 * node0[ntiles + 1]; tile t's slots are slots[slot_ptr[t] ..
 * slot_ptr[t + 1]), its first npairs[t] of them node pairs): each slot is
 * own node li | lj << 16 (li == lj for a single node), every own node of a
 * tile is in exactly one of the tile's first n - npairs[t] slots, slot_ptr
 * entries are multiples of 4, and each pair holds two mates
 * (nb_mesh_node_pairs) whose rows have six entries, the same two shared
 * neighbours first and the partner third.  The library runs the same check
 * on each staged plan before uploading it.  nslots is the length of the
 * slots array; the slot ranges are checked against it before any slot is
 * read.  Host only.  Errors: NB_EINVAL with the first violation in
 * nb_last_error. */
int nb_check_slot_lists(const nb_mesh *mesh, int32_t ntiles, const int32_t *node0, const int32_t *slot_ptr,
                        const int32_t *npairs, const uint32_t *slots, int64_t nslots);

/* Host-side statistics of the tile plan the single-pass Laplacian
 * (NB_LAP_FUSED) builds for FP32 columns of nlev levels at the padded
 * stride: tiles, tiles before the pole-row tiles, the largest number of
 * g-nodes (own plus first-ring nodes) of a tile, and fits = 1 when every
 * tile, its rings counted exactly, fits the kernel's shared-memory layout
 * (the library refuses to launch a plan that does not).  Runs on the host
 * only (for tests).  Errors: NB_EINVAL (nlev outside [16, 1020]). */
int nb_mesh_lap_plan(const nb_mesh *mesh, int nlev, int32_t *ntiles, int32_t *ntiles_main,
                     int32_t *max_gnodes, int32_t *fits);

/* First node of the pole-row block: nodes [cap_begin, V) are the nodes of
 * the first and last grid rows, which the FP32 kernels treat in FP64. */
int nb_mesh_cap_begin(const nb_mesh *mesh, int64_t *cap_begin);

/* ---------------------------------------------------------- partitions
 * Host-side building blocks of a horizontally partitioned (multi-GPU) run;
 * the operators themselves run on one device here. */

/* EqualRegions partition (Sec. 4.2.4.2) of the grid's points into nparts
 * regions: the zonal equal-area partition of the sphere (two polar caps and
 * collars, regions per collar rounded with carry) gives the bands north to
 * south; the points, taken north to south, are dealt to the bands in
 * proportion to their region counts and, within a band ordered by
 * longitude, into its regions, so every region holds V / nparts points
 * (+-1).  part: caller-owned host int32[V] in grid order, part ids
 * 0..nparts-1 numbered north to south (may be NULL to query the zones).
 * zones (may be NULL): regions per band, north to south, *nzones of them.
 * Errors: NB_EINVAL (nparts < 1 or > V). */
int nb_partition_equal_regions(const nb_grid *grid, int nparts, int32_t *part, int32_t *zones,
                               int32_t *nzones);

/* Owned nodes and halo of partition p (Sec. 4.4): part is a host int32[V]
 * in functionspace (mesh) order; owned = nodes with part == p, halo = the
 * nodes owned elsewhere that neighbour an owned node (what a one-ring
 * stencil needs), both ascending.  Pass owned/halo NULL to get the counts
 * first.  Errors: NB_EINVAL. */
int nb_partition_halo(const nb_mesh *mesh, const int32_t *part, int p, int64_t *nowned, int32_t *owned,
                      int64_t *nhalo, int32_t *halo);

/* -------------------------------------------------------------- method */

/* fvm::Method (Sec. 4.7): build the median-dual geometry of the mesh on a
 * sphere of radius radius_m (FP64, host), upload it once to the current
 * CUDA device and derive the per-edge operator weights there in FP64 (plus
 * their FP32 roundings).  radius_m <= 0 selects 6.37122e6 m.
 * Errors: NB_EINVAL, NB_EOOM, NB_ECUDA. */
int nb_method_create(const nb_mesh *mesh, double radius_m, nb_method **out);
int nb_method_release(nb_method *method);

/* Dual volumes V_i (m^2), functionspace order, host double[V]. */
int nb_method_dual_volumes(const nb_method *method, double *host_out);

/* Device bytes held by the method (geometry, weights, tile plans). */
int nb_method_device_bytes(const nb_method *method, int64_t *bytes);

/* ------------------------------------------------------- functionspace */

/* NodeColumns function space (Sec. 4.5): nlev levels of dtype.  Reports the
 * padded level stride Lp that fields should use: nlev rounded up to a
 * multiple of 4 (FP32) or 2 (FP64), so that every column starts on a
 * 16-byte boundary.  Errors: NB_EINVAL (nlev < 1), NB_EDTYPE. */
int nb_fs_nodecolumns(const nb_method *method, int nlev, nb_dtype dtype, nb_fs **out);
int nb_fs_release(nb_fs *fs);
int nb_fs_level_stride(const nb_fs *fs, int64_t *lp);

/* Fill an nb_field view of caller memory for this functionspace.
 * nvar 1 or 2.  node_stride >= nlev * nvar, lev_stride == nvar.
 * Errors: NB_EINVAL, NB_ESHAPE. */
int nb_field_view(const nb_fs *fs, void *dev_ptr, int nvar, int64_t node_stride,
                  int64_t lev_stride, nb_field *out);

/* --------------------------------------------------------- operators
 * fvm::Nabla (Sec. 4.7, Fig. 33, Listing 12).  In and out must have the
 * same dtype, node count and level count; out must not alias in.  FP64
 * fields run the FP64 kernels; FP32 fields run FP32 arithmetic with
 * compensated per-node accumulation and FP64 for the pole-row nodes.
 * Errors (before any launch): NB_EINVAL, NB_ESHAPE, NB_EDTYPE;
 * NB_ECUDA if the launch fails. */

/* Gradient, horizontal components only (Listing 12): f [V][L] -> g [V][L][2]
 * in 1/m times f's unit, (east, north). */
int nb_nabla_gradient(const nb_method *method, const nb_field *f, const nb_field *g, void *stream);

/* Divergence of a (east, north) vector field: uv [V][L][2] -> d [V][L]. */
int nb_nabla_divergence(const nb_method *method, const nb_field *uv, const nb_field *d,
                        void *stream);

/* Vertical curl (vorticity, positive counter-clockwise seen from outside):
 * uv [V][L][2] -> z [V][L]. */
int nb_nabla_curl(const nb_method *method, const nb_field *uv, const nb_field *z, void *stream);

/* Divergence and curl of the same wind in one pass: uv [V][L][2] -> d [V][L]
 * and z [V][L] (Fig. 33 puts both in the one Nabla operator of a Method).
 * Each output equals, bit for bit, what nb_nabla_divergence and
 * nb_nabla_curl write for the same input; the fused FP32 pass reads the wind
 * and the neighbour structure once for both.  d and z must have the same
 * layout.  Errors as for nb_nabla_divergence, plus NB_ESHAPE if d and z
 * differ in layout or overlap the wind. */
int nb_nabla_divcurl(const nb_method *method, const nb_field *uv, const nb_field *d,
                     const nb_field *z, void *stream);

/* Gradient and Laplacian of the same scalar field: f [V][L] -> g [V][L][2]
 * and lap [V][L].  The Laplacian is the divergence of the gradient (Fig. 33),
 * so its first pass is g itself: two launches instead of three.  Each output
 * equals, bit for bit, what nb_nabla_gradient and nb_nabla_laplacian write
 * for the same input.  Errors as for those calls (g is checked as the
 * Laplacian's scratch: it must not overlap f or lap). */
int nb_nabla_gradlap(const nb_method *method, const nb_field *f, const nb_field *g,
                     const nb_field *lap, void *stream);

/* Laplacian = divergence of the gradient: f [V][L] -> lap [V][L].
 * scratch: a [V][L][2] field of f's dtype receiving the intermediate
 * gradient, or NULL to let the library take stream-ordered memory from the
 * CUDA default pool for the call. */
int nb_nabla_laplacian(const nb_method *method, const nb_field *f, const nb_field *lap,
                       const nb_field *scratch, void *stream);

/* Laplacian that allocates nothing.  The paper has no counterpart: this call
 * serves callers that cannot allocate device memory while they run, such as
 * a component embedded in a larger model with a device-memory budget fixed at
 * start-up, or a latency-critical loop in which cudaMalloc/cudaFree (which can
 * synchronise the whole device) are not allowed.  The intermediate gradient
 * lives in a fixed array of NB_NOALLOC_SCRATCH_BYTES inside the library; it
 * fits [V][Lq][2] values of f's dtype with Lq = nlev rounded up to a multiple
 * of 4 (FP32) or 2 (FP64), and larger problems get NB_ESHAPE (use
 * nb_nabla_laplacian with a scratch field).  The CUDA runtime loads the
 * library's device code lazily (its default): the array's device memory is
 * taken on a device when this call first runs there, which also looks up
 * the array's device address and may synchronise the device.  So make the
 * first call on each device at start-up, inside the caller's memory budget
 * and before any stream capture; from then on the array stays on that
 * device until the process exits and no call allocates.  (A process started
 * with CUDA_MODULE_LOADING=EAGER takes the memory when the library loads.)
 * All calls share the one array and it keeps the last call's
 * contents (nothing in it needs to start at zero); calls whose work overlaps
 * on the GPU, on any stream, race on it, so serialise them.  Same argument
 * rules and errors as nb_nabla_laplacian. */
#define NB_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
int nb_nabla_laplacian_noalloc(const nb_method *method, const nb_field *f, const nb_field *lap,
                               void *stream);

/* Generic entry: op is an nb_op; for NB_OP_LAP scratch may be NULL. */
int nb_nabla_apply(const nb_method *method, int op, const nb_field *in, const nb_field *out,
                   const nb_field *scratch, void *stream);

/* Copy a whole field between host memory laid out exactly like it (node
 * stride included: nnodes x node_stride elements) and the device, enqueued
 * on `stream` without waiting.  Pinned host memory makes the copy
 * asynchronous and gives full link bandwidth; uploads and downloads on
 * different streams use the two copy directions at once, and overlap
 * operators running on a third stream (order them with CUDA events).
 * Errors: NB_EINVAL (NULL), NB_EDTYPE, NB_ECUDA. */
int nb_field_upload(const nb_field *dev, const void *host, void *stream);
int nb_field_download(void *host, const nb_field *dev, void *stream);

/* NodeColumns reductions (Sec. 4.5: global minimum, maximum and mean values
 * of a field), per level and component: host_out[l * nvar + c] for l < nlev,
 * c < nvar, in FP64.  NB_REDUCE_SUM is the plain sum over the nodes;
 * NB_REDUCE_AREA_MEAN the dual-volume weighted mean sum(V_i x_i) / sum(V_i);
 * NB_REDUCE_AREA_RMS sqrt(sum(V_i x_i^2) / sum(V_i)), the area-weighted
 * norm used for error measures.  Deterministic (fixed reduction order); runs
 * on `stream` and waits for it.  Errors: NB_EINVAL, NB_EDTYPE, NB_ESHAPE
 * (field not on the method's mesh), NB_EOOM, NB_ECUDA. */
enum { NB_REDUCE_MIN = 0, NB_REDUCE_MAX = 1, NB_REDUCE_SUM = 2, NB_REDUCE_AREA_MEAN = 3, NB_REDUCE_AREA_RMS = 4 };
int nb_field_reduce(const nb_method *method, const nb_field *field, int kind, double *host_out, void *stream);

/* End-to-end call on HOST buffers: copy host_in (laid out exactly like
 * dev_in, node_stride included) to dev_in, apply op, copy dev_out back to
 * host_out and wait for the stream.  Pinned host memory gives full link
 * bandwidth.  dev_in/dev_out are caller-owned device fields. */
int nb_nabla_apply_host(const nb_method *method, int op, const void *host_in, void *host_out,
                        const nb_field *dev_in, const nb_field *dev_out,
                        const nb_field *scratch, void *stream);

/* --------------------------------------------------------------- batching
 * Many operations on fields of different grids and level counts in one
 * CUDA graph, captured once and replayed (the batching pattern named for
 * this hot path; the paper groups all operators in one Nabla, Sec. 4.7
 * Fig. 33).  Each item takes one of two routes:
 *   - the persistent kernel: the item is cut into work units of (nodes per
 *     warp x 8 warps x rounds) nodes by (levels per block) levels and one
 *     persistent launch per phase takes units of all such items from an
 *     atomic counter.  Its per-(node, level) arithmetic equals the direct
 *     kernels', so the result is bitwise equal to the operation run alone
 *     with nb_method_set_kernel(m, NB_KERNEL_DIRECT, 0);
 *   - the staged route (FP32, 16-byte aligned columns of >= 16 levels): the
 *     item gets its own shared-memory staged launch(es) inside the graph, so
 *     the result is bitwise equal to the operation run alone with the default
 *     kernel choice.
 * Laplacian items use batch-owned scratch (a second phase on the persistent
 * route).  Field memory stays caller-owned and must outlive the batch. */
typedef struct nb_batch_item {
  int32_t op;              /* nb_op */
  int32_t reserved;        /* zero */
  const nb_method *method; /* retained by the batch */
  nb_field in;             /* input field (as for nb_nabla_apply) */
  nb_field out;            /* output field */
} nb_batch_item;

/* Validate the items (same rules as nb_nabla_apply), allocate the work tables
 * and Laplacian scratch on the current device, take each item's route and
 * shape from the tuned table, else a size heuristic (the staged route for
 * candidates of 2^21 node-levels and more).
 * Errors: NB_EINVAL, NB_ESHAPE, NB_EDTYPE, NB_EOOM. */
int nb_batch_create(const nb_batch_item *items, int n, nb_batch **out);
int nb_batch_release(nb_batch *batch);

/* Autotune per item class (op, dtype, grid nodes V, levels) by timing single-item
 * launches on `stream`: the staged route (where possible) against the
 * persistent kernel with levels-per-block in {4,8,16,32,64} x nodes-per-warp
 * in {1,2,4,8,16,32}.  Results are kept per GPU name for later batches and,
 * if the environment variable NB_TUNE_CACHE names a file, saved there
 * ("gpu|op|f64|V|nlev|lpb|npw" lines, lpb = npw = 0 for the staged route)
 * and read back by later processes. */
int nb_batch_tune(nb_batch *batch, void *stream);

/* Run the batch: the first call (and the first after tuning) captures the
 * launches into a CUDA graph; every call replays it on `stream`. */
int nb_batch_run(nb_batch *batch, void *stream);

/* Compensated (1, default) or plain (0) FP32 accumulation for the batch. */
int nb_batch_set_compensated(nb_batch *batch, int on);

/* Work units of the persistent route, node-levels (sum over items of
 * V x nlev), and per item the chosen nodes-per-warp and levels-per-block
 * (arrays of n, may be NULL; both 0 for an item on the staged route). */
int nb_batch_info(const nb_batch *batch, int64_t *units, int64_t *node_levels,
                  int32_t *nodes_per_warp, int32_t *levels_per_block);

/* Nodes of the batch's captured CUDA graph, and how many of them are kernel
 * launches (the rest: the counter reset and the events that fork and join
 * the staged branches); both 0 before the first nb_batch_run or
 * nb_batch_tune captures it.  Host only.  Errors: NB_EINVAL. */
int nb_batch_graph_nodes(const nb_batch *batch, int64_t *nodes, int64_t *kernels);

/* ---------------------------------------------------------------- serving
 * Continuous-batching server for derived-field requests (the serving pattern
 * named for this hot path; the paper has no server).  Grids are registered
 * once and stay resident with two spherical-harmonic bases used to
 * synthesise request inputs on the device.  A worker thread admits arrived
 * requests in arrival order while the device-memory budget and the in-flight
 * limit allow, takes the request's field memory from the CUDA memory pool
 * (stream ordered), synthesises its inputs, runs the operator on the least
 * loaded of `nstreams` streams (a request's fields packed side by side
 * along the level axis into column blocks of at most 144 levels, one launch
 * per operator pass and block) and frees everything when the request's
 * completion event has fired, so requests overlap on the device.  A result is
 * computed by the same kernels whether the request runs alone or among
 * others, so it is bitwise the same. */
typedef struct nb_request {
  int32_t op;          /* nb_op */
  int32_t N;           /* Gaussian number of a registered grid */
  int32_t nlev;        /* levels, 1..4096 */
  int32_t nfields;     /* fields, 1..64; each gets the operator */
  int32_t dtype;       /* NB_F32 or NB_F64 */
  int32_t keep_output; /* 1: copy outputs to the host on completion;
                          2: outputs and inputs (tests) */
  uint64_t seed;       /* input synthesis seed */
} nb_request;

typedef struct nb_result {
  uint64_t ticket;
  int32_t status;      /* NB_OK or the error of this request */
  int32_t reserved;
  double arrival_s, admit_s, done_s; /* seconds, server clock (trace: from its start) */
  int64_t node_levels; /* nfields x V x nlev */
  int64_t bytes;       /* device memory the request held */
} nb_result;

/* Server on the current device with a device-memory budget in bytes for
 * request fields, nstreams streams (1..64) and at most max_inflight requests
 * on the device at once.  Sets the device's default memory pool to keep freed
 * memory cached.  Errors: NB_EINVAL, NB_ECUDA, NB_EOOM. */
int nb_server_create(int64_t hbm_budget, int nstreams, int max_inflight, nb_server **out);
int nb_server_release(nb_server *server);

/* Make the method's grid resident for requests with N = its Gaussian number.
 * scalar_basis: host double [V][8]; wind_basis: host double [V][8][2] (east,
 * north), both in functionspace node order; kept on the device as FP32.
 * Request inputs are per-level mixtures of these 8 fields, computed in FP32,
 * with weights drawn from the request seed (SplitMix64), rounded to the
 * request's dtype. */
int nb_server_add_grid(nb_server *server, const nb_method *method, const double *scalar_basis,
                       const double *wind_basis);

/* Queue a request now; returns its ticket.  Errors: NB_EINVAL (grid not
 * resident, bad fields), NB_EBUDGET (needs more than the whole budget). */
int nb_server_submit(nb_server *server, const nb_request *request, uint64_t *ticket);

/* Wait up to timeout_ms for a request; NB_ETIMEOUT if it is still queued or
 * running, NB_OK with its result otherwise. */
int nb_server_wait(nb_server *server, uint64_t ticket, double timeout_ms, nb_result *result);

/* Non-blocking query of a request: *done = 1 and *result filled if it has
 * finished (result->status holds its own error), *done = 0 if it is still
 * queued or running.  Errors: NB_EINVAL (NULL argument, unknown ticket). */
int nb_server_poll(nb_server *server, uint64_t ticket, int32_t *done, nb_result *result);

/* Copy a finished request's kept outputs (nfields x [V][Lp][nvar] of its
 * dtype, Lp the padded level stride) to host memory of exactly `bytes`. */
int nb_server_output(nb_server *server, uint64_t ticket, void *host_out, int64_t bytes);

/* Copy a finished request's kept inputs (keep_output == 2): nfields x
 * [V][Lp][nvar_in] of its dtype, to host memory of exactly `bytes`. */
int nb_server_input(nb_server *server, uint64_t ticket, void *host_in, int64_t bytes);

/* Fault injection for tests of the serving loop.  Every request submitted
 * afterwards whose seed is `seed` has its alloc_index-th device allocation
 * refused, as a pool with no memory left would refuse it (index 0 is the
 * request's mixing weights, then per column block of its fields the input,
 * the output and, for a Laplacian, the scratch field).  Such a request is
 * retired at once with status NB_EOOM and returns its share of the budget;
 * the work it had already enqueued still runs on its stream, and its device
 * memory goes back to the pool in stream order after that work.  Requests in
 * flight beside it are not touched.  alloc_index = -1 removes the injection
 * for `seed`.  Host-side only: no device fault is involved.  (No counterpart
 * in the paper.)  Errors: NB_EINVAL. */
int nb_server_inject_failure(nb_server *server, uint64_t seed, int32_t alloc_index);

/* Budget in use, its peak, queued and in-flight request counts. */
int nb_server_stats(nb_server *server, int64_t *used, int64_t *peak_used, int32_t *pending,
                    int32_t *inflight);

/* Replay a trace: submit request k at arrival_s[k] seconds after the call
 * starts, wait for all, fill results[k] (times relative to the call start). */
int nb_server_run_trace(nb_server *server, const nb_request *requests, const double *arrival_s,
                        int n, nb_result *results);

/* ------------------------------------------------------ kernel control */

/* Kernel variant used for a call: NB_KERNEL_AUTO lets the library choose
 * (tuned table, else a size heuristic). */
enum { NB_KERNEL_AUTO = 0, NB_KERNEL_DIRECT = 1, NB_KERNEL_TILED = 2, NB_KERNEL_EDGE = 3 };
/* NB_KERNEL_EDGE: the edge-based variant (the EdgeColumns pattern, Sec.
 * 4.5), kept as a baseline: every call first materialises the difference of
 * each edge's end columns (E x nlev x nvar values of stream-ordered scratch
 * from the current allocator), then reduces per node through the node ->
 * edge connectivity.  Results equal NB_KERNEL_DIRECT's bit for bit; the
 * extra pass and traffic are its cost. */

/* Force a kernel variant for subsequent calls on this method (tests and
 * tuning).  tile_nodes is the tiled variant's nodes per tile (0 = default). */
int nb_method_set_kernel(nb_method *method, int variant, int tile_nodes);

/* Pipeline shape of the shared-memory staged kernels: nstages stages of
 * stage_kb KB each (nstages * stage_kb <= 226; 0 = defaults 2 x 113 KB).
 * Tile plans are sized so that a tile's own columns plus its halo columns
 * fill one stage. */
int nb_method_set_staging(nb_method *method, int nstages, int stage_kb);

/* Accumulation mode of the FP32 path: 1 = compensated (default): per node
 * the edge terms are summed in groups by FMA chains, the group sums are
 * combined by error-free Fast2Sum steps and their rounding error is added
 * last (after the self term of div and curl); 0 = the same sums without the
 * correction (for accuracy/throughput comparison). */
int nb_method_set_compensated(nb_method *method, int on);

/* Route of the Laplacian (nb_nabla_laplacian, nb_nabla_apply with
 * NB_OP_LAP, nb_nabla_gradlap) for FP32 fields the staged kernels take
 * (16-byte aligned columns of at least 16 levels, kernel variant AUTO or
 * TILED); other fields always take two passes.
 *   NB_LAP_TWO_PASS (default): a gradient pass into scratch (or g) and a
 *     divergence pass of it; the gradient goes through HBM.
 *   NB_LAP_FUSED: one pass (Sec. 4.7, Fig. 33: the Laplacian is one Nabla
 *     operator): each tile stages f on its nodes and two rings of
 *     neighbours, computes the gradient on its nodes and the first ring in
 *     shared memory and the divergence of it on its nodes; the gradient
 *     reaches HBM only when nb_nabla_gradlap asks for it.  Bit-identical to
 *     the two-pass route.
 * Errors: NB_EINVAL. */
enum { NB_LAP_TWO_PASS = 0, NB_LAP_FUSED = 1 };
int nb_method_set_laplacian_route(nb_method *method, int route);

/* Item shape of the staged FP32 div / curl kernels (and the fused pass):
 * each consumer thread takes `units` 16-byte units (two levels of (u, v))
 * of one node's column per item, spread G units apart, G items per node.
 * aligned = 1 rounds G up to a multiple of 8, so that no quarter-warp reads
 * two nodes' columns (no shared-memory bank conflicts) at the price of idle
 * items; 0 does not round.  units = 0 / aligned = -1 let the library choose
 * per level count.  Results do not depend on the shape (each level's
 * arithmetic is the same).  For tuning and tests; errors: NB_EINVAL. */
int nb_method_set_item_shape(nb_method *method, int units, int aligned);

/* Node pairs in the staged FP32 kernels (grad, div, curl, fused div+curl).
 * With pairs, one consumer thread evaluates both nodes of a pair
 * (nb_mesh_node_pairs) whose nodes are own nodes of the same staged tile,
 * reading the 10 columns they span once instead of 14 times; without,
 * every node alone.  Both give the same bits (each node's terms are summed
 * in its row order either way).  mode = 1: pairs in every staged pass;
 * 0: in none; -1 (the default): in all but the fused div+curl pass, whose
 * two sets of sums leave too few registers for a second node.  For tuning
 * and tests; errors: NB_EINVAL. */
int nb_method_set_node_pairs(nb_method *method, int mode);

/* Limit of every wait inside the staged kernels' copy pipeline (a warp
 * waiting for a stage's copies to land, or for the consumer warps to release
 * a stage), in nanoseconds of the GPU's global timer.
 *   limit_ns = -1: the default, 2 s.  limit_ns = 0: every wait tests its
 *   barrier once, without suspending, and gives up at once if the phase is
 *   not complete.  Otherwise 1 ns .. 60 s.
 * A wait that runs out makes the kernel record NB_ETIMEOUT in the device
 * status word (nb_device_status) and return early, its outputs incomplete;
 * a CTA first waits (up to a fixed 4 s, independent of this limit) for the
 * copies it has already issued, so that none is in flight when it exits.
 * The GPU context stays usable.  Used to test failure detection: a short
 * limit makes the waits run out without any fault.  Returns NB_EINVAL for
 * other values.  (No counterpart in the paper.) */
int nb_method_set_wait_limit(nb_method *method, int64_t limit_ns);

/* Measured FP64 FMA rate of the current device, the roofline of the FP64
 * operator path (which B300's FP64 units bound, not HBM): one launch of
 * independent FMA chains (8 per thread, `iters` steps, 4 CTAs of 256
 * threads per SM) timed with CUDA events on `stream` after a warm-up
 * launch; *tflops = 2 x FMAs / time, *ms the launch time.  Waits for the
 * stream.  ~40000 iters take ~0.1 s on a B300.  (No counterpart in the
 * paper.)  Errors: NB_EINVAL, NB_ECUDA. */
int nb_probe_fp64_rate(int64_t iters, void *stream, double *tflops, double *ms);

/* Number of this library's kernel launches since load (all devices). */
int nb_launch_count(int64_t *count);

/* Device status word of the current device: 0 if every kernel so far ran
 * normally, else the NB_* code a kernel recorded (NB_ETIMEOUT when a bounded
 * wait inside a kernel ran out; the kernel then returned early and its
 * outputs are incomplete).  Synchronises the device.  clear != 0 resets the
 * word to 0 after reading it. */
int nb_device_status(int clear, int32_t *code);

#ifdef __cplusplus
}
#endif

#endif /* NABLA_B300_H */
