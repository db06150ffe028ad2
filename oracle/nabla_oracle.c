/*
 * nabla_oracle.c -- plain, slow, obviously correct CPU reference ("the
 * oracle") for the edge-based median-dual finite-volume nabla operators on an
 * octahedral reduced Gaussian grid.  All floating point is IEEE double.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or table with the CUDA
 * path.
 *
 * What the paper fixes and what is a reading (the paper prints no formula for
 * the operators; it names them and says they are "edge-based finite volume"):
 *   - grid: points per row, Listing 6 (Sec. 4.2.3.7); rows on the roots of the
 *     Legendre polynomial of degree 2N, first point of every row at 0 degrees
 *     longitude, Sec. 4.2.3.5; N parallels per hemisphere, Sec. 4.2.
 *   - mesh: grid points become mesh nodes, elements join them (Sec. 4.3,
 *     Listing 7, Fig. 25b shows closed pole caps).  The strip rule and the
 *     cap rule below are readings.
 *   - operators: gradient, divergence, curl and Laplacian on a node-centred
 *     ("NodeColumns", Sec. 4.5) field, built by fvm::Method / fvm::Nabla
 *     (Sec. 4.7, Fig. 33, Listing 12).  Median-dual control volumes on the
 *     sphere, difference-form gradient, flux-form divergence and curl, and
 *     Laplacian = div(grad) are readings.
 *
 * Every array is in the ORIGINAL grid order: rows north to south, points
 * west to east inside a row (Sec. 4.2.3, Listing 5 iterates the grid in this
 * order).  Fields are laid out [node][level] (a column is contiguous,
 * Sec. 4.5 Fig. 31); vector fields [node][level][2] with the local east and
 * north components innermost.
 *
 * A single global "mutation" switch lets the test suite plant a known mistake
 * in this oracle and check that its pins catch it.  It is zero (off) unless a
 * test sets it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* Planted-mistake switch, read only where a mistake is planted. */
static int g_mutation = 0;
void or_set_mutation(int m) { g_mutation = m; }
int or_get_mutation(void) { return g_mutation; }

/* ------------------------------------------------------------------ grid */

/* Number of points on row j of O<N>: 20 + 4j counting from either pole
 * (Listing 6, Sec. 4.2.3.7). */
static int row_nx(int N, int j) {
  int jj = (j < N) ? j : (2 * N - 1 - j);
  return 20 + 4 * jj;
}

long or_num_nodes(int N) {
  long v = 0;
  for (int j = 0; j < 2 * N; ++j) v += row_nx(N, j);
  return v;
}

void or_row_nx(int N, int *nx) {
  for (int j = 0; j < 2 * N; ++j) nx[j] = row_nx(N, j);
}

/* Any reduced Gaussian grid is given by its points per parallel, the "PL"
 * array nx[0..rows) from north to south (Sec. 4.2.3.7); the regular F<N>
 * grid has nx = 4N on all 2N rows (Sec. 4.2.3.6), the octahedral O<N> grid
 * the row lengths above.  The _pl functions take such an array. */
long or_num_nodes_pl(int rows, const int *nx) {
  long v = 0;
  for (int j = 0; j < rows; ++j) v += nx[j];
  return v;
}

/* Legendre polynomial P_n(x) and its derivative, from the three-term
 * recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}, in extended
 * precision (long double). */
static void legendre(int n, long double x, long double *pn, long double *dpn) {
  long double pm1 = 1.0L, p = x;
  for (int k = 1; k < n; ++k) {
    long double pp1 = ((2.0L * k + 1.0L) * x * p - k * pm1) / (k + 1.0L);
    pm1 = p;
    p = pp1;
  }
  *pn = p;
  *dpn = n * (x * p - pm1) / (x * x - 1.0L);
}

/* Gaussian latitudes: the 2N roots mu_j of P_{2N}, ordered from north to
 * south (Sec. 4.2.3.5), with their Gauss-Legendre weights.  Newton's method
 * from the classical first guess cos(pi (j + 3/4) / (2N + 1/2)), carried out
 * in extended precision and rounded once, so that each root is the double
 * nearest to the true root.  (The median-dual geometry is sensitive to node
 * positions at the last bit, so a correctly rounded grid matters.) */
void or_gaussian_rows(int N, double *mu, double *weight) {
  int n = 2 * N;
  for (int j = 0; j < N; ++j) {
    long double x = cosl(3.14159265358979323846264338327950288L * (j + 0.75L) / (n + 0.5L));
    long double p, dp;
    for (int it = 0; it < 100; ++it) {
      legendre(n, x, &p, &dp);
      long double dx = p / dp;
      x -= dx;
      if (fabsl(dx) < 1e-19L) break;
    }
    legendre(n, x, &p, &dp);
    mu[j] = (double)x;
    mu[n - 1 - j] = -(double)x;
    double w = (double)(2.0L / ((1.0L - x * x) * dp * dp));
    weight[j] = w;
    weight[n - 1 - j] = w;
  }
}

/* Latitude and longitude (radians) of every node, original order.  The first
 * point of each row is at longitude 0 and the points of a row are equispaced
 * (Sec. 4.2, Sec. 4.2.3.5). */
void or_grid_lonlat_pl(int rows, const int *nx, double *lat, double *lon) {
  int N = rows / 2;
  double *mu = (double *)malloc(sizeof(double) * 2 * N);
  double *w = (double *)malloc(sizeof(double) * 2 * N);
  or_gaussian_rows(N, mu, w);
  long id = 0;
  for (int j = 0; j < 2 * N; ++j) {
    double phi = asin(mu[j]);
    /* planted: equally spaced latitudes instead of the Gaussian rows */
    if (g_mutation == 12) phi = 0.5 * OR_PI - OR_PI * (j + 0.5) / (2.0 * N);
    for (int i = 0; i < nx[j]; ++i) {
      lat[id] = phi;
      lon[id] = 2.0 * OR_PI * (double)i / (double)nx[j];
      /* planted: rows start half a spacing east of longitude 0 */
      if (g_mutation == 13) lon[id] = 2.0 * OR_PI * ((double)i + 0.5) / (double)nx[j];
      ++id;
    }
  }
  free(mu);
  free(w);
}

void or_grid_lonlat(int N, double *lat, double *lon) {
  int *nx = (int *)malloc(sizeof(int) * 2 * N);
  or_row_nx(N, nx);
  or_grid_lonlat_pl(2 * N, nx, lat, lon);
  free(nx);
}

/* ---------------------------------------------------------- triangulation */

long or_num_triangles(int N) { return 2 * or_num_nodes(N) - 4; }

/* Structured triangulation (reading of Sec. 4.3, Listing 7, Fig. 25b).
 *
 * Strip between row j (n points, first node id a0) and row j+1 (n2 points,
 * first id b0): walk both rings from longitude 0 and always advance the ring
 * whose next point comes first in longitude; the comparison
 * (a+1)/n  vs  (b+1)/n2  is done exactly in integers.  On a tie advance the
 * ring with fewer points, and the northern ring if both have the same count.
 * Advancing the northern ring emits (A_a, B_b, A_{a+1}); advancing the
 * southern ring emits (A_a, B_b, B_{b+1}).  Both are counter-clockwise seen
 * from outside the sphere.  A strip holds n + n2 triangles.
 *
 * Pole caps: the polygon of the first (last) row is closed with no extra
 * node by the parallel chords (k, n-1-k); the quad (k, k+1, n-2-k, n-1-k) is
 * split along (k+1, n-1-k).  An odd ring leaves the triangle
 * (m, m+1, n-1-m), m = n/2 - 1 (integer division), after the last quad.
 * n - 2 triangles per cap, so F = 2V - 4.
 *
 * Output order: north cap, strips north to south, south cap. */
void or_triangulate_pl(int rows, const int *nx, int32_t *tri) {
  long *off = (long *)malloc(sizeof(long) * (rows + 1));
  off[0] = 0;
  for (int j = 0; j < rows; ++j) off[j + 1] = off[j] + nx[j];
  long t = 0;

  /* north cap: ring increases counter-clockwise seen from above the pole */
  {
    int n = nx[0];
    long b = off[0];
    int k = 0;
    for (; k + 1 < n / 2; ++k) {
      tri[3 * t + 0] = (int32_t)(b + k);
      tri[3 * t + 1] = (int32_t)(b + k + 1);
      tri[3 * t + 2] = (int32_t)(b + n - 1 - k);
      ++t;
      tri[3 * t + 0] = (int32_t)(b + k + 1);
      tri[3 * t + 1] = (int32_t)(b + n - 2 - k);
      tri[3 * t + 2] = (int32_t)(b + n - 1 - k);
      ++t;
    }
    if (n % 2 == 1) {
      tri[3 * t + 0] = (int32_t)(b + k);
      tri[3 * t + 1] = (int32_t)(b + k + 1);
      tri[3 * t + 2] = (int32_t)(b + n - 1 - k);
      ++t;
    }
  }

  for (int j = 0; j + 1 < rows; ++j) {
    long n = nx[j], n2 = nx[j + 1];
    long a0 = off[j], b0 = off[j + 1];
    long a = 0, b = 0;
    while (a < n || b < n2) {
      long lhs = (a + 1) * n2; /* next northern longitude, scaled by n*n2 */
      long rhs = (b + 1) * n;  /* next southern longitude, scaled */
      int advance_north;
      if (a >= n) advance_north = 0;
      else if (b >= n2) advance_north = 1;
      else if (lhs < rhs) advance_north = 1;
      else if (lhs > rhs) advance_north = 0;
      else advance_north = (n <= n2); /* tie: fewer points, north if equal */
      int32_t A = (int32_t)(a0 + (a % n)), B = (int32_t)(b0 + (b % n2));
      if (advance_north) {
        tri[3 * t + 0] = A;
        tri[3 * t + 1] = B;
        tri[3 * t + 2] = (int32_t)(a0 + ((a + 1) % n));
        ++a;
      } else {
        tri[3 * t + 0] = A;
        tri[3 * t + 1] = B;
        tri[3 * t + 2] = (int32_t)(b0 + ((b + 1) % n2));
        ++b;
      }
      ++t;
    }
  }

  /* south cap: the same chords, reversed so that the triangles are
   * counter-clockwise seen from below the south pole */
  {
    int n = nx[rows - 1];
    long b = off[rows - 1];
    int k = 0;
    for (; k + 1 < n / 2; ++k) {
      tri[3 * t + 0] = (int32_t)(b + k);
      tri[3 * t + 1] = (int32_t)(b + n - 1 - k);
      tri[3 * t + 2] = (int32_t)(b + k + 1);
      ++t;
      tri[3 * t + 0] = (int32_t)(b + k + 1);
      tri[3 * t + 1] = (int32_t)(b + n - 1 - k);
      tri[3 * t + 2] = (int32_t)(b + n - 2 - k);
      ++t;
    }
    if (n % 2 == 1) {
      tri[3 * t + 0] = (int32_t)(b + k);
      tri[3 * t + 1] = (int32_t)(b + n - 1 - k);
      tri[3 * t + 2] = (int32_t)(b + k + 1);
      ++t;
    }
  }
  free(off);
}

void or_triangulate(int N, int32_t *tri) {
  int *nx = (int *)malloc(sizeof(int) * 2 * N);
  or_row_nx(N, nx);
  or_triangulate_pl(2 * N, nx, tri);
  free(nx);
}

/* ------------------------------------------------------------------ edges */

/* Node -> incident triangles, as counts and a flat list (CSR). */
static void node_triangles(long V, long F, const int32_t *tri, long **ptr_out,
                           long **list_out) {
  long *ptr = (long *)calloc(V + 1, sizeof(long));
  for (long t = 0; t < F; ++t)
    for (int c = 0; c < 3; ++c) ptr[tri[3 * t + c] + 1]++;
  for (long i = 0; i < V; ++i) ptr[i + 1] += ptr[i];
  long *fill = (long *)malloc(sizeof(long) * V);
  memcpy(fill, ptr, sizeof(long) * V);
  long *list = (long *)malloc(sizeof(long) * ptr[V]);
  for (long t = 0; t < F; ++t)
    for (int c = 0; c < 3; ++c) list[fill[tri[3 * t + c]]++] = t;
  free(fill);
  *ptr_out = ptr;
  *list_out = list;
}

/* Does triangle t contain the directed edge p -> q? */
static int has_directed(const int32_t *tri, long t, int32_t p, int32_t q) {
  for (int c = 0; c < 3; ++c)
    if (tri[3 * t + c] == p && tri[3 * t + (c + 1) % 3] == q) return 1;
  return 0;
}

/* Edges of the mesh.  Every undirected edge {a, b} with a < b appears as the
 * directed edge a -> b in exactly one counter-clockwise triangle, which lies
 * to its LEFT seen from outside; the triangle holding b -> a lies to its
 * RIGHT.  Edges are listed in the order the scan of triangles meets them.
 * edge[e] = (a, b), etri[e] = (left, right).  Returns the number of edges,
 * or -1 if the mesh is not a closed oriented surface. */
long or_edges(long V, long F, const int32_t *tri, int32_t *edge, int32_t *etri) {
  long *ptr, *list;
  node_triangles(V, F, tri, &ptr, &list);
  long e = 0;
  for (long t = 0; t < F; ++t) {
    for (int c = 0; c < 3; ++c) {
      int32_t a = tri[3 * t + c], b = tri[3 * t + (c + 1) % 3];
      if (a >= b) continue;
      long right = -1;
      for (long k = ptr[a]; k < ptr[a + 1]; ++k)
        if (has_directed(tri, list[k], b, a)) right = list[k];
      if (right < 0) { free(ptr); free(list); return -1; }
      edge[2 * e + 0] = a;
      edge[2 * e + 1] = b;
      etri[2 * e + 0] = (int32_t)t;
      etri[2 * e + 1] = (int32_t)right;
      ++e;
    }
  }
  free(ptr);
  free(list);
  return e;
}

/* Node -> incident edges (CSR), edges in increasing edge id. */
void or_node_edges(long V, long E, const int32_t *edge, int64_t *ptr, int32_t *list) {
  for (long i = 0; i <= V; ++i) ptr[i] = 0;
  for (long e = 0; e < E; ++e) {
    ptr[edge[2 * e] + 1]++;
    ptr[edge[2 * e + 1] + 1]++;
  }
  for (long i = 0; i < V; ++i) ptr[i + 1] += ptr[i];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * V);
  for (long i = 0; i < V; ++i) fill[i] = ptr[i];
  for (long e = 0; e < E; ++e) {
    list[fill[edge[2 * e]]++] = (int32_t)e;
    list[fill[edge[2 * e + 1]]++] = (int32_t)e;
  }
  free(fill);
}

/* --------------------------------------------------------------- geometry */

static void unit_xyz(double lat, double lon, double x[3]) {
  x[0] = cos(lat) * cos(lon);
  x[1] = cos(lat) * sin(lon);
  x[2] = sin(lat);
}
static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }
static void normalize3(double a[3]) {
  double n = norm3(a);
  a[0] /= n; a[1] /= n; a[2] /= n;
}

/* Local frame at a node: unit east and unit north vectors. */
void or_frames(long V, const double *lat, const double *lon, double *east, double *north) {
  for (long i = 0; i < V; ++i) {
    double sl = sin(lon[i]), cl = cos(lon[i]), sp = sin(lat[i]), cp = cos(lat[i]);
    east[3 * i + 0] = -sl;
    east[3 * i + 1] = cl;
    east[3 * i + 2] = 0.0;
    north[3 * i + 0] = -sp * cl;
    north[3 * i + 1] = -sp * sl;
    north[3 * i + 2] = cp;
  }
}

/* Spherical excess of the geodesic triangle (A, B, C) on the unit sphere,
 * from tan(E/2) = |A.(BxC)| / (1 + A.B + B.C + C.A) (Van Oosterom and
 * Strackee, 1983). */
static double spherical_excess(const double A[3], const double B[3], const double C[3]) {
  double bc[3];
  cross3(B, C, bc);
  double num = fabs(dot3(A, bc));
  double den = 1.0 + dot3(A, B) + dot3(B, C) + dot3(C, A);
  return 2.0 * atan2(num, den);
}

/* Centroid direction of a triangle: the normalised sum of its vertices. */
static void tri_centroid(const double *xyz, const int32_t *tri, long t, double c[3]) {
  for (int d = 0; d < 3; ++d)
    c[d] = xyz[3 * tri[3 * t] + d] + xyz[3 * tri[3 * t + 1] + d] + xyz[3 * tri[3 * t + 2] + d];
  if (g_mutation == 10) { /* planted: planar centroid, not projected to the sphere */
    for (int d = 0; d < 3; ++d) c[d] /= 3.0;
    return;
  }
  normalize3(c);
}

/* Integral of the unit conormal over the great-circle arc p -> q on the unit
 * sphere: the conormal is the pole of the arc's great circle, constant along
 * the arc, so the integral is theta * (p x q)/|p x q| up to sign.  The sign
 * is chosen so that the result points from node a towards node b. */
static void arc_conormal(const double p[3], const double q[3], const double ab[3], double out[3]) {
  double c[3];
  cross3(p, q, c);
  double s = norm3(c);
  double theta = atan2(s, dot3(p, q));
  double sgn = (dot3(c, ab) >= 0.0) ? 1.0 : -1.0;
  if (g_mutation == 2) sgn = 1.0; /* planted: conormal sign not oriented */
  for (int d = 0; d < 3; ++d) out[d] = sgn * theta * c[d] / s;
}

/* Median-dual geometry on the sphere of radius R (reading of the edge-based
 * finite-volume method of Sec. 4.7).
 *
 * For edge e = (a, b) with left triangle L and right triangle R:
 *   m  = normalise(x_a + x_b)           (edge midpoint)
 *   cT = normalise(x_p + x_q + x_r)     (triangle centroid)
 *   the dual face of e is the pair of great-circle arcs cR -> m -> cL;
 *   S_e = R * (conormal integral of both arcs), pointing from a to b
 *         (= the integral of the outward unit normal n ds seen from a);
 *   T_e = R * (cL - cR)
 *         (= the integral of the unit tangent t ds along the face,
 *          counter-clockwise around a).
 * Seen from b both change sign.
 *
 * Dual volume of node i: for every incident triangle with centroid c and the
 * midpoints m1, m2 of the two triangle edges at i, the two geodesic
 * triangles (x_i, m1, c) and (x_i, c, m2); area R^2 * spherical excess.
 * The dual cells tile the sphere, so sum(vol) = 4 pi R^2. */
void or_geometry(long V, long F, long E, const double *lat, const double *lon,
                 const int32_t *tri, const int32_t *edge, const int32_t *etri,
                 double R, double *vol, double *S, double *T) {
  double *xyz = (double *)malloc(sizeof(double) * 3 * V);
  for (long i = 0; i < V; ++i) unit_xyz(lat[i], lon[i], xyz + 3 * i);

  for (long e = 0; e < E; ++e) {
    int32_t a = edge[2 * e], b = edge[2 * e + 1];
    double m[3], cL[3], cR[3], ab[3], s1[3], s2[3];
    for (int d = 0; d < 3; ++d) {
      m[d] = xyz[3 * a + d] + xyz[3 * b + d];
      ab[d] = xyz[3 * b + d] - xyz[3 * a + d];
    }
    normalize3(m);
    tri_centroid(xyz, tri, etri[2 * e + 0], cL);
    tri_centroid(xyz, tri, etri[2 * e + 1], cR);
    arc_conormal(cR, m, ab, s1);
    arc_conormal(m, cL, ab, s2);
    for (int d = 0; d < 3; ++d) {
      S[3 * e + d] = R * (s1[d] + s2[d]);
      T[3 * e + d] = R * (cL[d] - cR[d]);
    }
    if (g_mutation == 3)
      for (int d = 0; d < 3; ++d) T[3 * e + d] = R * (cR[d] - cL[d]); /* planted */
  }

  for (long i = 0; i < V; ++i) vol[i] = 0.0;
  for (long t = 0; t < F; ++t) {
    double c[3];
    tri_centroid(xyz, tri, t, c);
    for (int k = 0; k < 3; ++k) {
      int32_t i = tri[3 * t + k];
      int32_t nxt = tri[3 * t + (k + 1) % 3];
      int32_t prv = tri[3 * t + (k + 2) % 3];
      double m1[3], m2[3];
      for (int d = 0; d < 3; ++d) {
        m1[d] = xyz[3 * i + d] + xyz[3 * nxt + d];
        m2[d] = xyz[3 * i + d] + xyz[3 * prv + d];
      }
      normalize3(m1);
      normalize3(m2);
      double area = spherical_excess(xyz + 3 * i, m1, c);
      if (g_mutation != 5) area += spherical_excess(xyz + 3 * i, c, m2);
      vol[i] += R * R * area;
    }
  }
  free(xyz);
}

/* -------------------------------------------------------------- operators */

/* Sign of edge e seen from node i: +1 if i is its first node, else -1. */
static double side(const int32_t *edge, long e, long i) {
  return (edge[2 * e] == i) ? 1.0 : -1.0;
}
static long other(const int32_t *edge, long e, long i) {
  return (edge[2 * e] == i) ? edge[2 * e + 1] : edge[2 * e];
}

/* Gradient (Sec. 4.7, Listing 12: horizontal components only).
 * Reading: g_i = (1/V_i) sum_{e at i} 1/2 (f_j - f_i) S_e^(i), a 3-D vector,
 * returned as its components on the local east and north unit vectors.
 * f is [V][L], out is [V][L][2]. */
void or_grad(long V, const int64_t *nptr, const int32_t *nlist, const int32_t *edge,
             const double *S, const double *vol, const double *east, const double *north,
             long L, const double *f, double *out) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < V; ++i) {
    for (long k = 0; k < L; ++k) {
      double g[3] = {0.0, 0.0, 0.0};
      for (long p = nptr[i]; p < nptr[i + 1]; ++p) {
        long e = nlist[p];
        long j = other(edge, e, i);
        double s = side(edge, e, i);
        double half_df = 0.5 * (f[j * L + k] - f[i * L + k]);
        if (g_mutation == 1) half_df = 0.5 * (f[j * L + k] + f[i * L + k]); /* planted */
        for (int d = 0; d < 3; ++d) g[d] += half_df * s * S[3 * e + d];
      }
      /* planted: normalised by the first neighbour's dual volume */
      const double vi = g_mutation == 9 ? vol[other(edge, nlist[nptr[i]], i)] : vol[i];
      for (int d = 0; d < 3; ++d) g[d] /= vi;
      out[(i * L + k) * 2 + 0] = dot3(g, east + 3 * i);
      out[(i * L + k) * 2 + 1] = dot3(g, north + 3 * i);
      if (g_mutation == 6) { /* planted: east and north swapped */
        out[(i * L + k) * 2 + 0] = dot3(g, north + 3 * i);
        out[(i * L + k) * 2 + 1] = dot3(g, east + 3 * i);
      }
    }
  }
}

/* 3-D vector of the local (east, north) components at node i. */
static void wind3(const double *east, const double *north, long i, double u, double v, double w[3]) {
  for (int d = 0; d < 3; ++d) w[d] = u * east[3 * i + d] + v * north[3 * i + d];
}

/* Divergence (Sec. 4.7, Fig. 33).  Reading, flux form:
 * D_i = (1/V_i) sum_{e at i} 1/2 (W_i + W_j) . S_e^(i),  W = u east + v north.
 * uv is [V][L][2], out is [V][L]. */
void or_div(long V, const int64_t *nptr, const int32_t *nlist, const int32_t *edge,
            const double *S, const double *vol, const double *east, const double *north,
            long L, const double *uv, double *out) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < V; ++i) {
    for (long k = 0; k < L; ++k) {
      double wi[3], acc = 0.0;
      wind3(east, north, i, uv[(i * L + k) * 2], uv[(i * L + k) * 2 + 1], wi);
      for (long p = nptr[i]; p < nptr[i + 1]; ++p) {
        long e = nlist[p];
        long j = other(edge, e, i);
        double s = side(edge, e, i), wj[3], wf[3];
        wind3(east, north, j, uv[(j * L + k) * 2], uv[(j * L + k) * 2 + 1], wj);
        for (int d = 0; d < 3; ++d) wf[d] = 0.5 * (wi[d] + wj[d]);
        if (g_mutation == 7) /* planted: the node's own wind dropped from the edge average */
          for (int d = 0; d < 3; ++d) wf[d] = 0.5 * wj[d];
        acc += s * dot3(wf, S + 3 * e);
      }
      out[i * L + k] = acc / vol[i];
    }
  }
}

/* Curl, vertical component, positive counter-clockwise seen from outside
 * (Sec. 4.7, Fig. 33).  Reading, flux form:
 * Z_i = (1/V_i) sum_{e at i} 1/2 (W_i + W_j) . T_e^(i). */
void or_curl(long V, const int64_t *nptr, const int32_t *nlist, const int32_t *edge,
             const double *T, const double *vol, const double *east, const double *north,
             long L, const double *uv, double *out) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < V; ++i) {
    for (long k = 0; k < L; ++k) {
      double wi[3], acc = 0.0;
      wind3(east, north, i, uv[(i * L + k) * 2], uv[(i * L + k) * 2 + 1], wi);
      for (long p = nptr[i]; p < nptr[i + 1]; ++p) {
        long e = nlist[p];
        long j = other(edge, e, i);
        double s = side(edge, e, i), wj[3], wf[3];
        wind3(east, north, j, uv[(j * L + k) * 2], uv[(j * L + k) * 2 + 1], wj);
        for (int d = 0; d < 3; ++d) wf[d] = 0.5 * (wi[d] + wj[d]);
        if (g_mutation == 8) s = 1.0; /* planted: tangent not negated for the edge's second node */
        acc += s * dot3(wf, T + 3 * e);
      }
      out[i * L + k] = acc / vol[i];
    }
  }
}

/* Laplacian (Sec. 4.7, Fig. 33).  Reading: the divergence of the gradient,
 * the gradient's local components re-expanded as a 3-D vector.  tmp is a
 * caller-owned [V][L][2] buffer that receives the gradient. */
void or_lap(long V, const int64_t *nptr, const int32_t *nlist, const int32_t *edge,
            const double *S, const double *vol, const double *east, const double *north,
            long L, const double *f, double *tmp, double *out) {
  or_grad(V, nptr, nlist, edge, S, vol, east, north, L, f, tmp);
  if (g_mutation == 14) /* planted: gradient components swapped before the divergence */
    for (long q = 0; q < V * L; ++q) {
      const double x = tmp[2 * q];
      tmp[2 * q] = tmp[2 * q + 1];
      tmp[2 * q + 1] = x;
    }
  or_div(V, nptr, nlist, edge, S, vol, east, north, L, tmp, out);
}

/* --------------------------------------------------- brute-force dual walk */

/* Independent per-node check of the assembled operators: walk the boundary
 * of node i's dual cell triangle by triangle and integrate over each arc
 * directly, with no edge list and no per-edge sign.  Inside an incident
 * counter-clockwise triangle (i, j, k) the dual boundary runs
 * m_ij -> c -> m_ik, counter-clockwise around i; on an arc p -> q traversed
 * counter-clockwise the outward conormal integral is theta (q x p)/|q x p|,
 * and the tangent integral is q - p.  Values on the arc belonging to edge
 * (i, j) are the edge averages 1/2 (value_i + value_j).
 * op: 0 grad (out[2]), 1 div (out[1]), 2 curl (out[1]); one level, f or uv
 * given per node (uv as [V][2]).  Also returns the dual volume. */
void or_bruteforce_node(long V, long F, const double *lat, const double *lon,
                        const int32_t *tri, double R, long i, int op,
                        const double *f, const double *uv, double *out, double *vol_out) {
  double xi[3];
  unit_xyz(lat[i], lon[i], xi);
  double acc3[3] = {0, 0, 0}, acc = 0.0, vol = 0.0;
  double ei[3] = {-sin(lon[i]), cos(lon[i]), 0.0};
  double ni[3] = {-sin(lat[i]) * cos(lon[i]), -sin(lat[i]) * sin(lon[i]), cos(lat[i])};
  for (long t = 0; t < F; ++t) {
    int c;
    for (c = 0; c < 3; ++c)
      if (tri[3 * t + c] == i) break;
    if (c == 3) continue;
    long j = tri[3 * t + (c + 1) % 3], k = tri[3 * t + (c + 2) % 3];
    double xj[3], xk[3], mij[3], mik[3], ct[3];
    unit_xyz(lat[j], lon[j], xj);
    unit_xyz(lat[k], lon[k], xk);
    for (int d = 0; d < 3; ++d) {
      mij[d] = xi[d] + xj[d];
      mik[d] = xi[d] + xk[d];
      ct[d] = xi[d] + xj[d] + xk[d];
    }
    normalize3(mij);
    normalize3(mik);
    normalize3(ct);
    vol += R * R * (spherical_excess(xi, mij, ct) + spherical_excess(xi, ct, mik));
    /* two arcs: (mij -> ct) belongs to edge (i,j); (ct -> mik) to edge (i,k) */
    const double *P[2] = {mij, ct}, *Q[2] = {ct, mik};
    long nb[2] = {j, k};
    for (int s = 0; s < 2; ++s) {
      double qp[3];
      cross3(Q[s], P[s], qp);
      double sn = norm3(qp), th = atan2(sn, dot3(P[s], Q[s]));
      double nu[3], tg[3];
      for (int d = 0; d < 3; ++d) {
        nu[d] = R * th * qp[d] / sn;
        tg[d] = R * (Q[s][d] - P[s][d]);
      }
      long jj = nb[s];
      if (op == 0) {
        double h = 0.5 * (f[jj] - f[i]);
        for (int d = 0; d < 3; ++d) acc3[d] += h * nu[d];
      } else {
        double wa[3], wb[3];
        double ej[3] = {-sin(lon[jj]), cos(lon[jj]), 0.0};
        double nj[3] = {-sin(lat[jj]) * cos(lon[jj]), -sin(lat[jj]) * sin(lon[jj]), cos(lat[jj])};
        for (int d = 0; d < 3; ++d) {
          wa[d] = uv[2 * i] * ei[d] + uv[2 * i + 1] * ni[d];
          wb[d] = uv[2 * jj] * ej[d] + uv[2 * jj + 1] * nj[d];
        }
        double wf[3] = {0.5 * (wa[0] + wb[0]), 0.5 * (wa[1] + wb[1]), 0.5 * (wa[2] + wb[2])};
        acc += dot3(wf, op == 1 ? nu : tg);
      }
    }
  }
  if (op == 0) {
    out[0] = dot3(acc3, ei) / vol;
    out[1] = dot3(acc3, ni) / vol;
  } else {
    out[0] = acc / vol;
  }
  *vol_out = vol;
}
