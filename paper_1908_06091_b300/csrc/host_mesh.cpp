// host_mesh.cpp -- multi-threaded host builder: octahedral grid, structured
// triangulation, space-filling-curve node order, node->edge CSR, FP64
// median-dual geometry on the sphere, and per-tile halo plans.
//
// Grid: Sec. 4.2.3.5 (Gaussian latitudes), Sec. 4.2.3.7 + Listing 6 (row
// lengths).  Mesh: Sec. 4.3, Listing 7, Fig. 25b (row strips, closed caps).
// Geometry: the dual mesh of the edge-based finite-volume method, Sec. 4.7.
#include <omp.h>

#include <algorithm>
#include <functional>
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

// Node pairs of the staged kernels.  Two adjacent six-neighbour
// nodes i < j outside the pole rows, j at most kPairWindow places after i in
// the node order, that share exactly two neighbours A < B, are matched
// greedily along the node order (i takes its smallest such unmatched j).
// Both rows are then reordered to (A, B, partner, the other three
// ascending).  The kernels sum a six-neighbour node's terms in row order in
// two groups of three, so one consumer can evaluate both nodes of a pair
// from 10 staged columns (the two own, A, B, three others each) instead of
// 14, with exactly the arithmetic of the single-node path.  On octahedral
// grids in Hilbert order ~95 % of the nodes are paired.
static constexpr int64_t kPairWindow = 16;

static void pair_nodes(nb_mesh *m) {
  const int64_t V = m->V;
  const int64_t *rp = m->row_ptr.data();
  int32_t *nb = m->nbr.data();
  m->mate.assign(V, -1);
  auto deg = [&](int64_t i) { return rp[i + 1] - rp[i]; };
  // common neighbours of i and j (rows still ascending), up to 3
  auto common = [&](int64_t i, int64_t j, int32_t *c) {
    int n = 0;
    int64_t p = rp[i], q = rp[j];
    while (p < rp[i + 1] && q < rp[j + 1]) {
      if (nb[p] < nb[q]) ++p;
      else if (nb[q] < nb[p]) ++q;
      else {
        if (n < 3) c[n] = nb[p];
        ++n, ++p, ++q;
      }
    }
    return n;
  };
  for (int64_t i = 0; i < m->cap_begin; ++i) {
    if (m->mate[i] >= 0 || deg(i) != 6) continue;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int64_t j = nb[p];
      if (j <= i || j > i + kPairWindow || j >= m->cap_begin || m->mate[j] >= 0 || deg(j) != 6) continue;
      int32_t c[3];
      if (common(i, j, c) != 2) continue;
      m->mate[i] = (int32_t)j;
      m->mate[j] = (int32_t)i;
      break;
    }
  }
  // reorder the rows of paired nodes; the per-entry arrays move together
  std::vector<int32_t> cm(2 * V, -1);
  for (int64_t i = 0; i < V; ++i) {
    const int64_t j = m->mate[i];
    if (j > i) common(i, j, &cm[2 * i]);
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < V; ++i) {
    const int64_t j = m->mate[i];
    if (j < 0) continue;
    const int32_t *c = &cm[2 * std::min(i, j)];
    const int32_t head[3] = {c[0], c[1], (int32_t)j};
    const int64_t p0 = rp[i];
    int32_t on[6], oe[6], ol[6], orr[6];
    for (int k = 0; k < 6; ++k) {
      on[k] = nb[p0 + k];
      oe[k] = m->nbr_edge[p0 + k];
      ol[k] = m->nbr_left[p0 + k];
      orr[k] = m->nbr_right[p0 + k];
    }
    int order[6], n = 0;
    for (int h = 0; h < 3; ++h)
      for (int k = 0; k < 6; ++k)
        if (on[k] == head[h]) order[n++] = k;
    for (int k = 0; k < 6; ++k)
      if (on[k] != head[0] && on[k] != head[1] && on[k] != head[2]) order[n++] = k;
    for (int k = 0; k < 6; ++k) {
      nb[p0 + k] = on[order[k]];
      m->nbr_edge[p0 + k] = oe[order[k]];
      m->nbr_left[p0 + k] = ol[order[k]];
      m->nbr_right[p0 + k] = orr[order[k]];
    }
  }
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
  pair_nodes(m);
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

namespace nb {

// ------------------------------------------------ fused Laplacian plans

// Tiles of the single-pass Laplacian.  A tile's own nodes are a run of
// consecutive nodes; ring 1 = the neighbours of own nodes outside the tile,
// ring 2 = the neighbours of ring-1 nodes outside own and ring 1.  The
// kernel stages f on own, ring-1 and ring-2 nodes, computes the gradient on
// own and ring-1 nodes (the "g-nodes"), then the divergence of it on own
// nodes.  Tiles grow along the node order while fits(n, H1, H2, own entries,
// ring-1 entries) holds; the rings are tracked incrementally (a node that
// joins the tile turns its neighbours into ring 1 and theirs into ring 2;
// no node ever leaves a ring except by joining the tile), with an undo log
// for the node that no longer fits.
template <class Fits>
static void plan_lap_tiles(const nb_mesh *m, Fits fits, int nmax, int pole_cap, std::vector<int32_t> &node0,
                           int &ntiles_main) {
  const int64_t V = m->V;
  std::vector<int32_t> stamp(V, -1);
  std::vector<uint8_t> state(V, 0);  // valid when stamp == tile: 1 own, 2 ring 1, 3 ring 2
  auto deg = [&](int64_t x) { return (int64_t)(m->row_ptr[x + 1] - m->row_ptr[x]); };
  int32_t tile = 0;
  node0.clear();
  struct Undo {
    int32_t node;
    int32_t stamp;
    uint8_t state;
  };
  std::vector<Undo> undo;
  auto cover = [&](int64_t a, int64_t b, int64_t cap) {
    int64_t n0 = a;
    while (n0 < b) {
      ++tile;
      int64_t n = 0, H1 = 0, H2 = 0, Eo = 0, E1 = 0;
      auto st = [&](int64_t x) -> uint8_t { return stamp[x] == tile ? state[x] : 0; };
      auto set = [&](int64_t x, uint8_t s) {
        undo.push_back({(int32_t)x, stamp[x], state[x]});
        stamp[x] = tile;
        state[x] = s;
      };
      int64_t n1 = n0;
      while (n1 < b && n < cap) {
        undo.clear();
        const int64_t v = n1;
        const int64_t sn = n, s1 = H1, s2 = H2, so = Eo, se = E1;
        const uint8_t old = st(v);
        if (old == 2) --H1, E1 -= deg(v);
        if (old == 3) --H2;
        set(v, 1);
        ++n;
        Eo += deg(v);
        for (int64_t p = m->row_ptr[v]; p < m->row_ptr[v + 1]; ++p) {
          const int32_t j = m->nbr[p];
          const uint8_t sj = st(j);
          if (sj == 1 || sj == 2) continue;
          if (sj == 3) --H2;
          set(j, 2);
          ++H1;
          E1 += deg(j);
        }
        // ring 2: neighbours of ring-1 nodes that are in no ring yet (only
        // the neighbours of v's neighbours can have changed)
        for (int64_t p = m->row_ptr[v]; p < m->row_ptr[v + 1]; ++p) {
          const int32_t j = m->nbr[p];
          if (st(j) != 2) continue;
          for (int64_t q = m->row_ptr[j]; q < m->row_ptr[j + 1]; ++q) {
            const int32_t k = m->nbr[q];
            if (st(k) == 0) {
              set(k, 3);
              ++H2;
            }
          }
        }
        if (n > 1 && !fits(n, H1, H2, Eo, E1)) {
          for (auto it = undo.rbegin(); it != undo.rend(); ++it) {
            stamp[it->node] = it->stamp;
            state[it->node] = it->state;
          }
          n = sn, H1 = s1, H2 = s2, Eo = so, E1 = se;
          break;
        }
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
}

void build_lap_plan(const nb_mesh *m, const LapLayout &L, int nmax, int pole_cap, LapPlanHost &out) {
  const int64_t hb_unit = 128;
  auto hbase = [&](int64_t n) { return (n * L.row_bytes + hb_unit - 1) / hb_unit * hb_unit; };
  auto fits = [&](int64_t n, int64_t H1, int64_t H2, int64_t Eo, int64_t E1) {
    if (n > L.nmax || n + H1 > L.gcap || Eo > L.ecap || Eo + E1 > L.rcap) return false;
    return hbase(n) + (H1 + H2 + 3) / 4 * L.gpitch <= L.farea;
  };
  plan_lap_tiles(m, fits, nmax, pole_cap, out.node0, out.ntiles_main);
  const int nt = (int)out.node0.size() - 1;
  // per tile: rings (each sorted), then the offsets and g-phase records
  std::vector<std::vector<int32_t>> r1(nt), r2(nt);
#pragma omp parallel for schedule(dynamic, 64)
  for (int t = 0; t < nt; ++t) {
    const int32_t a = out.node0[t], b = out.node0[t + 1];
    std::vector<int32_t> &h1 = r1[t], &h2 = r2[t];
    for (int64_t p = m->row_ptr[a]; p < m->row_ptr[b]; ++p) {
      const int32_t j = m->nbr[p];
      if (j < a || j >= b) h1.push_back(j);
    }
    std::sort(h1.begin(), h1.end());
    h1.erase(std::unique(h1.begin(), h1.end()), h1.end());
    for (int32_t j : h1)
      for (int64_t q = m->row_ptr[j]; q < m->row_ptr[j + 1]; ++q) {
        const int32_t k = m->nbr[q];
        if ((k < a || k >= b) && !std::binary_search(h1.begin(), h1.end(), k)) h2.push_back(k);
      }
    std::sort(h2.begin(), h2.end());
    h2.erase(std::unique(h2.begin(), h2.end()), h2.end());
  }
  out.halo_ptr.assign(nt + 1, 0);
  out.r1_count.assign(nt, 0);
  out.gn_ptr.assign(nt + 1, 0);
  out.rec_ptr.assign(nt + 1, 0);
  for (int t = 0; t < nt; ++t) {
    const int32_t a = out.node0[t], b = out.node0[t + 1];
    out.r1_count[t] = (int32_t)r1[t].size();
    out.halo_ptr[t + 1] = out.halo_ptr[t] + (int32_t)(r1[t].size() + r2[t].size());
    // g-node entries: one per own and ring-1 node, plus the end
    out.gn_ptr[t + 1] = out.gn_ptr[t] + (int32_t)((b - a) + r1[t].size() + 1);
    int64_t recs = m->row_ptr[b] - m->row_ptr[a];
    for (int32_t j : r1[t]) recs += m->row_ptr[j + 1] - m->row_ptr[j];
    out.rec_ptr[t + 1] = out.rec_ptr[t] + (int32_t)recs;
  }
  out.halo.resize(out.halo_ptr[nt]);
  out.gn.resize(out.gn_ptr[nt]);
  out.rec_p.resize(out.rec_ptr[nt]);
  out.rec_foff.resize(out.rec_ptr[nt]);
  out.loff.assign(m->row_ptr[m->V], 0);
  out.goff.assign(m->row_ptr[m->V], 0);
  int mg = 0, mr = 0;
  out.fits = true;
  for (int t = 0; t < nt; ++t) {
    mg = std::max(mg, out.gn_ptr[t + 1] - out.gn_ptr[t] - 1);
    mr = std::max(mr, out.rec_ptr[t + 1] - out.rec_ptr[t]);
    // every tile, with its exact rings, must fit the layout the kernel uses
    const int64_t n = out.node0[t + 1] - out.node0[t];
    const int64_t Eo = m->row_ptr[out.node0[t + 1]] - m->row_ptr[out.node0[t]];
    const int64_t E1 = (out.rec_ptr[t + 1] - out.rec_ptr[t]) - Eo;
    if (n < 1 || !fits(n, (int64_t)r1[t].size(), (int64_t)r2[t].size(), Eo, E1)) out.fits = false;
  }
  out.max_gnodes = mg;
  out.max_recs = mr;
#pragma omp parallel for schedule(dynamic, 64)
  for (int t = 0; t < nt; ++t) {
    const int32_t a = out.node0[t], b = out.node0[t + 1];
    const int64_t n = b - a;
    const std::vector<int32_t> &h1 = r1[t], &h2 = r2[t];
    std::copy(h1.begin(), h1.end(), out.halo.begin() + out.halo_ptr[t]);
    std::copy(h2.begin(), h2.end(), out.halo.begin() + out.halo_ptr[t] + h1.size());
    // staged slot of node x: own k -> k, ring 1 r -> n + r, ring 2 s -> n + H1 + s
    auto slot = [&](int32_t x) -> int64_t {
      if (x >= a && x < b) return x - a;
      auto it = std::lower_bound(h1.begin(), h1.end(), x);
      if (it != h1.end() && *it == x) return n + (it - h1.begin());
      return n + (int64_t)h1.size() + (std::lower_bound(h2.begin(), h2.end(), x) - h2.begin());
    };
    auto fbyte = [&](int64_t k) -> uint32_t {
      return (uint32_t)(k < n ? k * L.row_bytes : hbase(n) + ((k - n) >> 2) * L.gpitch + ((k - n) & 3) * L.copy_bytes);
    };
    for (int64_t p = m->row_ptr[a]; p < m->row_ptr[b]; ++p) {
      const int64_t k = slot(m->nbr[p]);
      out.loff[p] = fbyte(k);
      out.goff[p] = (uint32_t)(k * L.g_pitch);  // own or ring 1: k < n + H1
    }
    // g-phase records: own nodes then ring-1 nodes, each node's entries in
    // CSR order; gn = record start relative to the tile | pole-row flag
    int64_t r = out.rec_ptr[t], g = out.gn_ptr[t];
    auto add_gnode = [&](int32_t x) {
      out.gn[g++] = (uint32_t)(r - out.rec_ptr[t]) | (x >= m->cap_begin ? 0x80000000u : 0u);
      for (int64_t p = m->row_ptr[x]; p < m->row_ptr[x + 1]; ++p) {
        out.rec_p[r] = (int32_t)p;
        out.rec_foff[r] = fbyte(slot(m->nbr[p]));
        ++r;
      }
    };
    for (int32_t x = a; x < b; ++x) add_gnode(x);
    for (int32_t x : h1) add_gnode(x);
    out.gn[g] = (uint32_t)(r - out.rec_ptr[t]);
  }
}

}  // namespace nb

namespace nb {

// ------------------------------------------------------ plan validation

// A tile plan is valid when its tiles cover [0, V) in order, each halo
// list holds valid nodes outside its tile, and every CSR neighbour of
// a tile's node maps (slot(p, t, n)) to the staged slot that holds it: own
// node k at slot k, halo entry h at slot n + h.  slot returns -1 for an
// entry it cannot decode.  Run on every plan before it is uploaded, so a
// corrupted plan is refused before any launch.
bool check_tile_plan(const nb_mesh *m, int ntiles, const int32_t *node0, const int32_t *halo_ptr,
                     const int32_t *halo, const std::function<int64_t(int64_t, int, int64_t)> &slot,
                     std::string &why) {
  if (ntiles < 0 || (ntiles == 0 && m->V > 0)) {
    why = "no tiles";
    return false;
  }
  if (node0[0] != 0 || node0[ntiles] != m->V || halo_ptr[0] != 0) {
    why = "tiles do not cover the nodes";
    return false;
  }
  for (int t = 0; t < ntiles; ++t) {
    const int32_t a = node0[t], b = node0[t + 1];
    if (b <= a) {
      why = "tile " + std::to_string(t) + " is empty or out of order";
      return false;
    }
    const int32_t h0 = halo_ptr[t], h1 = halo_ptr[t + 1];
    if (h1 < h0) {
      why = "halo range of tile " + std::to_string(t) + " is reversed";
      return false;
    }
    for (int32_t h = h0; h < h1; ++h) {
      const int32_t x = halo[h];
      if (x < 0 || x >= m->V || (x >= a && x < b)) {
        why = "halo entry " + std::to_string(h) + " of tile " + std::to_string(t) + " is invalid";
        return false;
      }
    }
    const int64_t n = b - a;
    for (int64_t p = m->row_ptr[a]; p < m->row_ptr[b]; ++p) {
      const int32_t j = m->nbr[p];
      const int64_t k = slot(p, t, n);
      const bool ok = (k >= 0 && k < n) ? (a + k == j)
                                        : (k >= n && k - n < h1 - h0 && halo[h0 + (k - n)] == j);
      if (!ok) {
        why = "CSR entry " + std::to_string(p) + " of tile " + std::to_string(t) + " maps to the wrong staged column";
        return false;
      }
    }
  }
  return true;
}

// A slot list is valid when every own node of a tile appears in exactly one
// slot, each of the tile's first npairs[t] slots holds two own nodes that
// are each other's mates, and both rows of such a pair have six entries,
// the same two shared neighbours first and the partner third (the layout
// the pair path of the div / curl consumers reads); the rest are single
// nodes (li == lj).  Run on every plan before it is uploaded.
bool check_slot_lists(const nb_mesh *m, int ntiles, const int32_t *node0, const int32_t *slot_ptr,
                      const int32_t *npairs, const uint32_t *slots, std::string &why) {
  std::vector<uint8_t> seen;
  for (int t = 0; t < ntiles; ++t) {
    const int32_t a = node0[t], b = node0[t + 1], n = b - a;
    const int32_t q0 = slot_ptr[t], q1 = slot_ptr[t + 1], np = npairs[t];
    const std::string tile = " of tile " + std::to_string(t);
    if (q0 % 4 || q1 < q0 || np < 0 || 2 * np > n || q1 - q0 < n - np) {
      why = "slot range" + tile + " is invalid";
      return false;
    }
    seen.assign(n, 0);
    for (int32_t q = 0; q < n - np; ++q) {
      const uint32_t li = slots[q0 + q] & 0xffffu, lj = slots[q0 + q] >> 16;
      if ((int32_t)li >= n || (int32_t)lj >= n || (q < np) == (li == lj) || seen[li] || (li != lj && seen[lj])) {
        why = "slot " + std::to_string(q) + tile + " is invalid";
        return false;
      }
      seen[li] = seen[lj] = 1;
      if (li == lj) continue;
      const int64_t i = a + li, j = a + lj;
      const int64_t pi = m->row_ptr[i], pj = m->row_ptr[j];
      if (m->mate[i] != j || m->mate[j] != i || m->row_ptr[i + 1] - pi != 6 || m->row_ptr[j + 1] - pj != 6 ||
          m->nbr[pi] != m->nbr[pj] || m->nbr[pi + 1] != m->nbr[pj + 1] || m->nbr[pi + 2] != j ||
          m->nbr[pj + 2] != i) {
        why = "pair slot " + std::to_string(q) + tile + " does not hold a reordered node pair";
        return false;
      }
    }
    for (int32_t k = 0; k < n; ++k)
      if (!seen[k]) {
        why = "node " + std::to_string(a + k) + " has no slot";
        return false;
      }
  }
  return true;
}

}  // namespace nb
