// host_mesh.cpp -- multi-threaded host builder: octahedral grid, structured
// triangulation, space-filling-curve node order, node->edge CSR, FP64
// median-dual geometry on the sphere, and per-tile halo plans.
//
// Grid: Sec. 4.2.3.5 (Gaussian latitudes), Sec. 4.2.3.7 + Listing 6 (row
// lengths).  Mesh: Sec. 4.3, Listing 7, Fig. 25b (row strips, closed caps).
// Geometry: the dual mesh of the edge-based finite-volume method, Sec. 4.7.
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <stdexcept>

#include "internal.h"

namespace nb {

static constexpr double kPi = 3.14159265358979323846;

// ----------------------------------------------------------------- grid

// Points on row j of O<N>: 20 + 4 * (distance in rows from the nearer pole).
static inline int32_t octa_nx(int N, int j) { return 20 + 4 * std::min(j, 2 * N - 1 - j); }

// Positive roots of P_n (n = 2N), northernmost first: Newton on the Legendre
// recurrence in double from Tricomi's asymptotic first guess, then polished
// by Newton steps in extended precision and rounded once, so each root is
// the double nearest the true root.  The median-dual geometry reacts to
// node positions at the last bit (a one-ulp shift of the latitudes moves
// O640 dual volumes by ~1e-12), so the rows are computed correctly rounded.
template <class F>
static F legendre_newton_step(int n, F x) {
  F p0 = 1, p1 = x;
  for (int l = 2; l <= n; ++l) {
    const F p2 = ((F)(2 * l - 1) * x * p1 - (F)(l - 1) * p0) / (F)l;
    p0 = p1;
    p1 = p2;
  }
  const F dp = (F)n * (p0 - x * p1) / ((F)1 - x * x);
  return p1 / dp;
}

static void legendre_roots(int N, std::vector<double> &mu) {
  const int n = 2 * N;
  mu.assign(n, 0.0);
#pragma omp parallel for schedule(dynamic, 16)
  for (int k = 0; k < N; ++k) {
    const double th = kPi * (4.0 * (k + 1) - 1.0) / (4.0 * n + 2.0);
    double x = (1.0 - (n - 1.0) / (8.0 * n * (double)n * n)) * std::cos(th);
    for (int it = 0; it < 50; ++it) {
      const double step = legendre_newton_step<double>(n, x);
      x -= step;
      if (std::fabs(step) <= 1e-15) break;
    }
    long double xl = x;
    for (int it = 0; it < 3; ++it) xl -= legendre_newton_step<long double>(n, xl);
    mu[k] = (double)xl;
    mu[n - 1 - k] = -(double)xl;
  }
}

nb_grid *build_grid_pl(int N, const std::vector<int32_t> &nx) {
  auto *g = new nb_grid();
  g->N = N;
  g->nx = nx;
  g->row_off.resize(2 * N + 1);
  g->row_off[0] = 0;
  for (int j = 0; j < 2 * N; ++j) g->row_off[j + 1] = g->row_off[j] + g->nx[j];
  g->V = g->row_off[2 * N];
  legendre_roots(N, g->mu);
  return g;
}

nb_grid *build_grid(int N) {
  std::vector<int32_t> nx(2 * N);
  for (int j = 0; j < 2 * N; ++j) nx[j] = octa_nx(N, j);
  return build_grid_pl(N, nx);
}

// --------------------------------------------------- triangulation (grid ids)

// Row strips and caps as the structured generator defines them: advance the
// ring whose next point comes first in longitude ((a+1)/n vs (b+1)/n2
// compared in integers); ties advance the ring with fewer points, the
// northern one if equal; caps by the chords (k, n-1-k) split along
// (k+1, n-1-k), and an odd ring's last three points (m, m+1, n-1-m),
// m = n/2 - 1, as one more triangle.  Triangles counter-clockwise seen from
// outside.
static void triangulate_grid_ids(const nb_grid *g, std::vector<int32_t> &tri) {
  const int rows = 2 * g->N;
  const int64_t F = 2 * g->V - 4;
  tri.assign(3 * F, 0);
  std::vector<int64_t> start(rows);
  start[0] = g->nx[0] - 2;  // strip j begins at start[j]; the north cap comes first
  for (int j = 0; j + 1 < rows - 1; ++j) start[j + 1] = start[j] + g->nx[j] + g->nx[j + 1];
  const int64_t south_cap = start[rows - 2] + g->nx[rows - 2] + g->nx[rows - 1];
  auto cap = [&](int row, int64_t t, bool north) {
    const int n = g->nx[row];
    const int32_t b = (int32_t)g->row_off[row];
    for (int k = 0; k + 1 < n / 2; ++k) {
      const int32_t A = b + k, B = b + k + 1, C = b + n - 2 - k, D = b + n - 1 - k;
      int32_t *o = &tri[3 * t];
      if (north) {
        o[0] = A; o[1] = B; o[2] = D;
        o[3] = B; o[4] = C; o[5] = D;
      } else {
        o[0] = A; o[1] = D; o[2] = B;
        o[3] = B; o[4] = D; o[5] = C;
      }
      t += 2;
    }
    if (n & 1) {
      const int m = n / 2 - 1;
      const int32_t A = b + m, B = b + m + 1, D = b + n - 1 - m;
      int32_t *o = &tri[3 * t];
      if (north) {
        o[0] = A; o[1] = B; o[2] = D;
      } else {
        o[0] = A; o[1] = D; o[2] = B;
      }
    }
  };
  cap(0, 0, true);
  cap(rows - 1, south_cap, false);
#pragma omp parallel for schedule(dynamic, 4)
  for (int j = 0; j < rows - 1; ++j) {
    const int64_t n = g->nx[j], n2 = g->nx[j + 1];
    const int64_t a0 = g->row_off[j], b0 = g->row_off[j + 1];
    int64_t t = start[j];
    int64_t a = 0, b = 0;
    const bool north_on_tie = n <= n2;
    while (a < n || b < n2) {
      bool north;
      if (a == n) north = false;
      else if (b == n2) north = true;
      else {
        const int64_t ln = (a + 1) * n2, ls = (b + 1) * n;
        north = (ln == ls) ? north_on_tie : (ln < ls);
      }
      int32_t *o = &tri[3 * t++];
      o[0] = (int32_t)(a0 + a % n);
      o[1] = (int32_t)(b0 + b % n2);
      if (north) {
        o[2] = (int32_t)(a0 + (a + 1) % n);
        ++a;
      } else {
        o[2] = (int32_t)(b0 + (b + 1) % n2);
        ++b;
      }
    }
  }
}

// ------------------------------------------------------------ node order

// 3-D Hilbert index of integer coordinates with `bits` bits each: Skilling's
// transpose algorithm ("Programming the Hilbert curve", AIP Conf. Proc. 707,
// 2004), followed by bit interleaving of the transposed coordinates.
static uint64_t hilbert3(uint32_t x0, uint32_t x1, uint32_t x2, int bits) {
  uint32_t X[3] = {x0, x1, x2};
  const uint32_t M = 1u << (bits - 1);
  for (uint32_t Q = M; Q > 1; Q >>= 1) {
    const uint32_t P = Q - 1;
    for (int i = 0; i < 3; ++i) {
      if (X[i] & Q) {
        X[0] ^= P;
      } else {
        const uint32_t t = (X[0] ^ X[i]) & P;
        X[0] ^= t;
        X[i] ^= t;
      }
    }
  }
  for (int i = 1; i < 3; ++i) X[i] ^= X[i - 1];
  uint32_t t = 0;
  for (uint32_t Q = M; Q > 1; Q >>= 1)
    if (X[2] & Q) t ^= Q - 1;
  for (int i = 0; i < 3; ++i) X[i] ^= t;
  uint64_t key = 0;
  for (int q = bits - 1; q >= 0; --q)
    for (int i = 0; i < 3; ++i) key = (key << 1) | ((X[i] >> q) & 1u);
  return key;
}

// perm[new] = old.  Pole-row nodes (first and last row) go last, in grid
// order; the rest follow the Hilbert curve (reorder = 1) or grid order.
static void node_order(const nb_grid *g, const std::vector<double> &xyz, int reorder,
                       std::vector<int32_t> &perm, int64_t &cap_begin) {
  const int64_t V = g->V;
  const int64_t n0 = g->nx[0], nl = g->nx[2 * g->N - 1];
  std::vector<int32_t> inner;
  inner.reserve(V - n0 - nl);
  for (int64_t i = n0; i < V - nl; ++i) inner.push_back((int32_t)i);
  if (reorder == 1) {
    const int bits = 20;
    const double top = (double)((1u << bits) - 1);
    std::vector<uint64_t> key(V);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < V; ++i) {
      uint32_t c[3];
      for (int d = 0; d < 3; ++d) {
        double v = (xyz[3 * i + d] + 1.0) * 0.5 * top;
        v = std::min(std::max(v, 0.0), top);
        c[d] = (uint32_t)std::llround(v);
      }
      key[i] = hilbert3(c[0], c[1], c[2], bits);
    }
    std::sort(inner.begin(), inner.end(), [&](int32_t a, int32_t b) {
      return key[a] != key[b] ? key[a] < key[b] : a < b;
    });
  }
  perm = std::move(inner);
  cap_begin = (int64_t)perm.size();
  for (int64_t i = 0; i < n0; ++i) perm.push_back((int32_t)i);
  for (int64_t i = V - nl; i < V; ++i) perm.push_back((int32_t)i);
}

// ------------------------------------------------------------------ mesh

nb_mesh *build_mesh(nb_grid *g, int reorder) {
  auto *m = new nb_mesh();
  m->grid = retain(g);
  const int64_t V = g->V, F = 2 * V - 4, E = 3 * V - 6;
  m->V = V;
  m->F = F;
  m->E = E;

  // positions in grid order
  std::vector<double> xyz_g(3 * V), lat_g(V), lon_g(V);
#pragma omp parallel for schedule(dynamic, 8)
  for (int j = 0; j < 2 * g->N; ++j) {
    const double phi = std::asin(g->mu[j]);
    const double cphi = std::cos(phi), sphi = std::sin(phi);
    for (int i = 0; i < g->nx[j]; ++i) {
      const int64_t id = g->row_off[j] + i;
      const double lam = 2.0 * kPi * (double)i / (double)g->nx[j];
      lat_g[id] = phi;
      lon_g[id] = lam;
      xyz_g[3 * id + 0] = cphi * std::cos(lam);
      xyz_g[3 * id + 1] = cphi * std::sin(lam);
      xyz_g[3 * id + 2] = sphi;
    }
  }

  node_order(g, xyz_g, reorder, m->perm, m->cap_begin);
  m->iperm.assign(V, 0);
  for (int64_t i = 0; i < V; ++i) m->iperm[m->perm[i]] = (int32_t)i;
  m->xyz.resize(3 * V);
  m->lat.resize(V);
  m->lon.resize(V);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < V; ++i) {
    const int64_t o = m->perm[i];
    for (int d = 0; d < 3; ++d) m->xyz[3 * i + d] = xyz_g[3 * o + d];
    m->lat[i] = lat_g[o];
    m->lon[i] = lon_g[o];
  }

  // triangles, renumbered
  triangulate_grid_ids(g, m->tri);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < 3 * F; ++k) m->tri[k] = m->iperm[m->tri[k]];

  // node -> incident triangles (ascending triangle id)
  std::vector<int64_t> tptr(V + 1, 0);
  for (int64_t k = 0; k < 3 * F; ++k) tptr[m->tri[k] + 1]++;
  for (int64_t i = 0; i < V; ++i) tptr[i + 1] += tptr[i];
  std::vector<int32_t> tlist(3 * F);
  {
    std::vector<int64_t> fill(tptr.begin(), tptr.end() - 1);
    for (int64_t t = 0; t < F; ++t)
      for (int c = 0; c < 3; ++c) tlist[fill[m->tri[3 * t + c]]++] = (int32_t)t;
  }

  // CSR: on a closed triangulated surface a node has as many neighbours as
  // incident triangles.  Each neighbour j is the "next" vertex of exactly one
  // incident triangle (left of i -> j) and the "previous" vertex of one
  // (right of i -> j).
  m->row_ptr = tptr;
  if (m->row_ptr[V] != 2 * E) throw std::runtime_error("mesh: degree sum != 2E");
  m->nbr.assign(2 * E, 0);
  m->nbr_left.assign(2 * E, -1);
  m->nbr_right.assign(2 * E, -1);
  m->nbr_edge.assign(2 * E, -1);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : bad)
  for (int64_t i = 0; i < V; ++i) {
    const int64_t p0 = tptr[i], deg = tptr[i + 1] - tptr[i];
    struct Ent {
      int32_t j, left, right;
    };
    Ent ent[64];
    if (deg > 64) {
      ++bad;
      continue;
    }
    int n = 0;
    for (int64_t q = p0; q < p0 + deg; ++q) {
      const int32_t t = tlist[q];
      const int32_t *v = &m->tri[3 * t];
      const int c = (v[0] == i) ? 0 : (v[1] == i) ? 1 : 2;
      const int32_t jn = v[(c + 1) % 3];
      int k = 0;
      while (k < n && ent[k].j != jn) ++k;
      if (k == n) ent[n++] = {jn, -1, -1};
      ent[k].left = t;
    }
    for (int64_t q = p0; q < p0 + deg; ++q) {
      const int32_t t = tlist[q];
      const int32_t *v = &m->tri[3 * t];
      const int c = (v[0] == i) ? 0 : (v[1] == i) ? 1 : 2;
      const int32_t jp = v[(c + 2) % 3];
      int k = 0;
      while (k < n && ent[k].j != jp) ++k;
      if (k == n) {
        ++bad;
        break;
      }
      ent[k].right = t;
    }
    if (n != deg) {
      ++bad;
      continue;
    }
    std::sort(ent, ent + n, [](const Ent &a, const Ent &b) { return a.j < b.j; });
    for (int k = 0; k < n; ++k) {
      if (ent[k].left < 0 || ent[k].right < 0) ++bad;
      m->nbr[p0 + k] = ent[k].j;
      m->nbr_left[p0 + k] = ent[k].left;
      m->nbr_right[p0 + k] = ent[k].right;
    }
  }
  if (bad) throw std::runtime_error("mesh: triangulation is not a closed oriented surface");

  // edge ids: (a, b) with a < b numbered in CSR order of a
  std::vector<int64_t> ebase(V + 1, 0);
  for (int64_t i = 0; i < V; ++i) {
    int64_t c = 0;
    for (int64_t p = m->row_ptr[i]; p < m->row_ptr[i + 1]; ++p) c += (m->nbr[p] > i);
    ebase[i + 1] = ebase[i] + c;
  }
  if (ebase[V] != E) throw std::runtime_error("mesh: edge count != 3V - 6");
  m->edge.assign(2 * E, 0);
  m->edge_tri.assign(2 * E, 0);
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < V; ++i) {
    int64_t e = ebase[i];
    for (int64_t p = m->row_ptr[i]; p < m->row_ptr[i + 1]; ++p) {
      if (m->nbr[p] > i) {
        m->nbr_edge[p] = (int32_t)e;
        m->edge[2 * e] = (int32_t)i;
        m->edge[2 * e + 1] = m->nbr[p];
        m->edge_tri[2 * e] = m->nbr_left[p];
        m->edge_tri[2 * e + 1] = m->nbr_right[p];
        ++e;
      }
    }
  }
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < V; ++i) {
    for (int64_t p = m->row_ptr[i]; p < m->row_ptr[i + 1]; ++p) {
      const int32_t j = m->nbr[p];
      if (j > i) continue;
      const int32_t *b = m->nbr.data() + m->row_ptr[j];
      const int32_t *e = m->nbr.data() + m->row_ptr[j + 1];
      const int32_t *it = std::lower_bound(b, e, (int32_t)i);
      m->nbr_edge[p] = m->nbr_edge[m->row_ptr[j] + (it - b)];
    }
  }
  return m;
}

// --------------------------------------------------------------- geometry

static inline void cross(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double dot(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static inline void unit(double *a) {
  const double n = std::sqrt(dot(a, a));
  a[0] /= n;
  a[1] /= n;
  a[2] /= n;
}
// Area of the geodesic triangle (A, B, C) on the unit sphere: spherical
// excess from tan(E/2) = |A.(BxC)| / (1 + A.B + B.C + C.A)
// (Van Oosterom and Strackee, IEEE Trans. Biomed. Eng. 30, 1983).
static inline double excess(const double *A, const double *B, const double *C) {
  double bc[3];
  cross(B, C, bc);
  return 2.0 * std::atan2(std::fabs(dot(A, bc)), 1.0 + dot(A, B) + dot(B, C) + dot(C, A));
}
// Accumulate the integral of the unit conormal of the great-circle arc
// p -> q, oriented along `dir`: the arc length times the pole of the arc.
static inline void add_arc_conormal(const double *p, const double *q, const double *dir, double *acc) {
  double c[3];
  cross(p, q, c);
  const double s = std::sqrt(dot(c, c));
  const double th = std::atan2(s, dot(p, q));
  const double k = (dot(c, dir) < 0.0 ? -th : th) / s;
  acc[0] += k * c[0];
  acc[1] += k * c[1];
  acc[2] += k * c[2];
}

void build_geometry(const nb_mesh *m, double R, std::vector<double> &vol, std::vector<double> &S,
                    std::vector<double> &T, std::vector<double> &east, std::vector<double> &north) {
  const int64_t V = m->V, E = m->E, F = m->F;
  const double *x = m->xyz.data();
  std::vector<double> cen(3 * F);
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < F; ++t) {
    const int32_t *v = &m->tri[3 * t];
    double c[3];
    for (int d = 0; d < 3; ++d) c[d] = x[3 * v[0] + d] + x[3 * v[1] + d] + x[3 * v[2] + d];
    unit(c);
    for (int d = 0; d < 3; ++d) cen[3 * t + d] = c[d];
  }
  // face integrals per edge: dual face = arcs c_right -> mid -> c_left
  S.assign(3 * E, 0.0);
  T.assign(3 * E, 0.0);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < E; ++e) {
    const int32_t a = m->edge[2 * e], b = m->edge[2 * e + 1];
    const double *cl = &cen[3 * m->edge_tri[2 * e]];
    const double *cr = &cen[3 * m->edge_tri[2 * e + 1]];
    double mid[3], dir[3], acc[3] = {0, 0, 0};
    for (int d = 0; d < 3; ++d) {
      mid[d] = x[3 * a + d] + x[3 * b + d];
      dir[d] = x[3 * b + d] - x[3 * a + d];
    }
    unit(mid);
    add_arc_conormal(cr, mid, dir, acc);
    add_arc_conormal(mid, cl, dir, acc);
    for (int d = 0; d < 3; ++d) {
      S[3 * e + d] = R * acc[d];
      T[3 * e + d] = R * (cl[d] - cr[d]);
    }
  }
  // dual volumes: per triangle corner, then summed per node
  std::vector<double> corner(3 * F);
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < F; ++t) {
    const int32_t *v = &m->tri[3 * t];
    const double *c = &cen[3 * t];
    for (int k = 0; k < 3; ++k) {
      const double *xi = &x[3 * v[k]], *xn = &x[3 * v[(k + 1) % 3]], *xp = &x[3 * v[(k + 2) % 3]];
      double m1[3], m2[3];
      for (int d = 0; d < 3; ++d) {
        m1[d] = xi[d] + xn[d];
        m2[d] = xi[d] + xp[d];
      }
      unit(m1);
      unit(m2);
      corner[3 * t + k] = R * R * (excess(xi, m1, c) + excess(xi, c, m2));
    }
  }
  std::vector<int64_t> tptr(V + 1, 0);
  for (int64_t k = 0; k < 3 * F; ++k) tptr[m->tri[k] + 1]++;
  for (int64_t i = 0; i < V; ++i) tptr[i + 1] += tptr[i];
  std::vector<double> cl(3 * F);
  {
    std::vector<int64_t> fill(tptr.begin(), tptr.end() - 1);
    for (int64_t t = 0; t < F; ++t)
      for (int k = 0; k < 3; ++k) cl[fill[m->tri[3 * t + k]]++] = corner[3 * t + k];
  }
  vol.assign(V, 0.0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < V; ++i) {
    double s = 0.0;
    for (int64_t q = tptr[i]; q < tptr[i + 1]; ++q) s += cl[q];
    vol[i] = s;
  }
  east.resize(3 * V);
  north.resize(3 * V);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < V; ++i) {
    const double sl = std::sin(m->lon[i]), cln = std::cos(m->lon[i]);
    const double sp = std::sin(m->lat[i]), cp = std::cos(m->lat[i]);
    east[3 * i + 0] = -sl;
    east[3 * i + 1] = cln;
    east[3 * i + 2] = 0.0;
    north[3 * i + 0] = -sp * cln;
    north[3 * i + 1] = -sp * sl;
    north[3 * i + 2] = cp;
  }
}

// ------------------------------------------------------------- tile plans

// Tiles of consecutive nodes for the shared-memory staged kernels, grown
// greedily along the node order while fits(n, H) holds for the tile's n own
// nodes and H halo nodes (neighbours outside it), with at most nmax nodes and
// ecap CSR entries.  Main tiles cover [0, cap_begin), pole tiles
// [cap_begin, V) with at most pole_cap nodes each.  halo[t] lists the sorted
// halo nodes of tile t.
template <class Fits>
static void plan_tiles(const nb_mesh *m, Fits fits, int nmax, int ecap, int pole_cap, std::vector<int32_t> &node0,
                       std::vector<int32_t> &halo_ptr, std::vector<int32_t> &halo, int &max_halo,
                       int &max_entries, int &ntiles_main) {
  const int64_t V = m->V;
  std::vector<int32_t> mark(V, -1);
  node0.clear();
  int32_t stamp = 0;
  auto cover = [&](int64_t a, int64_t b, int64_t cap) {
    int64_t n0 = a;
    while (n0 < b) {
      ++stamp;
      int64_t n1 = n0, H = 0;
      while (n1 < b && n1 - n0 < cap) {
        const int64_t v = n1;
        if (n1 > n0 && m->row_ptr[v + 1] - m->row_ptr[n0] > ecap) break;
        int64_t add = 0;
        for (int64_t p = m->row_ptr[v]; p < m->row_ptr[v + 1]; ++p) {
          const int32_t j = m->nbr[p];
          if ((j < n0 || j > v) && mark[j] != stamp) ++add;
        }
        const int64_t inhalo = (mark[v] == stamp) ? 1 : 0;
        const int64_t newH = H + add - inhalo;
        if (n1 > n0 && !fits(n1 - n0 + 1, newH)) break;
        for (int64_t p = m->row_ptr[v]; p < m->row_ptr[v + 1]; ++p) {
          const int32_t j = m->nbr[p];
          if (j < n0 || j > v) mark[j] = stamp;
        }
        mark[v] = -2;  // inside the tile now
        H = newH;
        ++n1;
      }
      node0.push_back((int32_t)n0);
      n0 = n1;
    }
  };
  cover(0, m->cap_begin, nmax);
  ntiles_main = (int)node0.size();
  cover(m->cap_begin, V, std::max(1, std::min(pole_cap, nmax)));
  node0.push_back((int32_t)V);
  const int nt = (int)node0.size() - 1;
  std::vector<std::vector<int32_t>> hal(nt);
  std::vector<int> hmax(nt, 0), emax(nt, 0);
#pragma omp parallel for schedule(dynamic, 64)
  for (int t = 0; t < nt; ++t) {
    const int32_t a = node0[t], b = node0[t + 1];
    std::vector<int32_t> &h = hal[t];
    for (int64_t p = m->row_ptr[a]; p < m->row_ptr[b]; ++p) {
      const int32_t j = m->nbr[p];
      if (j < a || j >= b) h.push_back(j);
    }
    std::sort(h.begin(), h.end());
    h.erase(std::unique(h.begin(), h.end()), h.end());
    hmax[t] = (int)h.size();
    emax[t] = (int)(m->row_ptr[b] - m->row_ptr[a]);
  }
  max_halo = 0;
  max_entries = 0;
  halo_ptr.assign(nt + 1, 0);
  for (int t = 0; t < nt; ++t) {
    halo_ptr[t + 1] = halo_ptr[t] + (int32_t)hal[t].size();
    max_halo = std::max(max_halo, hmax[t]);
    max_entries = std::max(max_entries, emax[t]);
  }
  halo.resize(halo_ptr[nt]);
  for (int t = 0; t < nt; ++t) std::copy(hal[t].begin(), hal[t].end(), halo.begin() + halo_ptr[t]);
}

// Position of CSR neighbour p of a node of tile t among the staged columns:
// k < n for the tile's own node k, n + h for halo node h.
template <class Out>
static void staged_index(const nb_mesh *m, const std::vector<int32_t> &node0,
                         const std::vector<int32_t> &halo_ptr, const std::vector<int32_t> &halo,
                         Out out) {
  const int nt = (int)node0.size() - 1;
#pragma omp parallel for schedule(dynamic, 64)
  for (int t = 0; t < nt; ++t) {
    const int32_t a = node0[t], b = node0[t + 1];
    const int32_t *h0 = halo.data() + halo_ptr[t], *h1 = halo.data() + halo_ptr[t + 1];
    for (int64_t p = m->row_ptr[a]; p < m->row_ptr[b]; ++p) {
      const int32_t j = m->nbr[p];
      const int64_t k = (j >= a && j < b) ? (j - a) : (b - a) + (std::lower_bound(h0, h1, j) - h0);
      out(p, t, (int64_t)(b - a), k);
    }
  }
}

// Plan with a staged-row capacity: own nodes + halo nodes <= rcap; lnbr[p]
// is the staged row of CSR neighbour p.
void build_tile_plan_host(const nb_mesh *m, int rcap, int nmax, int ecap, std::vector<int32_t> &node0,
                          std::vector<int32_t> &halo_ptr, std::vector<int32_t> &halo,
                          std::vector<uint16_t> &lnbr, int &max_halo, int &max_entries,
                          int &ntiles_main) {
  plan_tiles(m, [&](int64_t n, int64_t H) { return n + H <= rcap; }, nmax, ecap, 1, node0, halo_ptr, halo,
             max_halo, max_entries, ntiles_main);
  lnbr.assign(m->row_ptr[m->V], 0);
  staged_index(m, node0, halo_ptr, halo,
               [&](int64_t p, int, int64_t, int64_t k) { lnbr[p] = (uint16_t)k; });
}

// Plan in bytes for the gather-staged layout: the tile's own columns at
// `row_bytes` pitch from offset 0, then halo columns in groups of four at
// `copy_bytes` pitch, each group starting on a 128-byte boundary
// (group pitch = 4 copy_bytes rounded up to 128).  Tiles grow while the
// layout fits `area` bytes; loff[p] is the byte offset of CSR neighbour p.
void build_tile_plan_bytes(const nb_mesh *m, int64_t area, int64_t row_bytes, int64_t copy_bytes,
                           int nmax, int ecap, int pole_cap, std::vector<int32_t> &node0,
                           std::vector<int32_t> &halo_ptr, std::vector<int32_t> &halo,
                           std::vector<uint32_t> &loff, int &max_halo, int &max_entries,
                           int &ntiles_main) {
  const int64_t gpitch = (4 * copy_bytes + 127) / 128 * 128;
  auto hbase = [&](int64_t n) { return (n * row_bytes + 127) / 128 * 128; };
  plan_tiles(m, [&](int64_t n, int64_t H) { return hbase(n) + (H + 3) / 4 * gpitch <= area; }, nmax,
             ecap, pole_cap, node0, halo_ptr, halo, max_halo, max_entries, ntiles_main);
  loff.assign(m->row_ptr[m->V], 0);
  staged_index(m, node0, halo_ptr, halo, [&](int64_t p, int, int64_t n, int64_t k) {
    loff[p] = (uint32_t)(k < n ? k * row_bytes : hbase(n) + ((k - n) >> 2) * gpitch + ((k - n) & 3) * copy_bytes);
  });
}

}  // namespace nb
