// partition.cpp -- EqualRegions partition of a grid's points (Sec. 4.2.4.2)
// and the halo of a partition of the mesh (Sec. 4.4), host side.
//
// The sphere is cut into nparts regions of equal area by the recursive
// zonal equal-area construction (Leopardi, 2006): two polar caps of area
// 4 pi / nparts and collars in between, the number of regions per collar
// rounded with carry from its ideal value.  Grid points, taken north to
// south (row order; within a row by longitude), are dealt to the bands in
// proportion to the bands' region counts, and within a band, ordered by
// longitude, into that band's regions -- so every region gets V / nparts
// points (+-1), as the paper describes for reduced grids.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "internal.h"

namespace nb {

// Regions per zone, north to south: 1 (cap), collars..., 1 (cap).
std::vector<int> eq_zone_counts(int n) {
  if (n == 1) return {1};
  if (n == 2) return {1, 1};
  const double pi = 3.14159265358979323846;
  const double area = 4.0 * pi / n;
  const double theta_c = 2.0 * std::asin(std::sqrt(1.0 / n));  // polar cap colatitude
  const double delta_ideal = std::sqrt(area);
  const int collars = std::max(1, (int)std::lround((pi - 2.0 * theta_c) / delta_ideal));
  const double delta = (pi - 2.0 * theta_c) / collars;
  std::vector<int> z{1};
  double carry = 0.0;
  for (int i = 1; i <= collars; ++i) {
    const double t0 = theta_c + (i - 1) * delta, t1 = theta_c + i * delta;
    const double ideal = 2.0 * pi * (std::cos(t0) - std::cos(t1)) / area;
    const int m = (int)std::lround(ideal + carry);
    carry += ideal - m;
    z.push_back(m);
  }
  z.push_back(1);
  return z;
}

void equal_regions(const nb_grid *g, int nparts, std::vector<int32_t> &part) {
  const int64_t V = g->V;
  part.assign(V, 0);
  const std::vector<int> zones = eq_zone_counts(nparts);
  const double pi = 3.14159265358979323846;
  // points in grid order: rows north to south, longitude ascending in a row
  std::vector<int64_t> order(V);
  std::iota(order.begin(), order.end(), 0);
  int64_t taken = 0;
  int regions_before = 0;
  for (int zone : zones) {
    const int64_t end = (int64_t)std::llround((double)V * (regions_before + zone) / nparts);
    // the band's points, ordered by longitude (ties: north first)
    std::vector<int64_t> band(order.begin() + taken, order.begin() + end);
    auto lon = [&](int64_t id) {
      const int64_t j = std::upper_bound(g->row_off.begin(), g->row_off.end(), id) - g->row_off.begin() - 1;
      return 2.0 * pi * (double)(id - g->row_off[j]) / (double)g->nx[j];
    };
    std::stable_sort(band.begin(), band.end(), [&](int64_t a, int64_t b) { return lon(a) < lon(b); });
    const int64_t nb = (int64_t)band.size();
    for (int r = 0; r < zone; ++r) {
      const int64_t b0 = (int64_t)std::llround((double)nb * r / zone);
      const int64_t b1 = (int64_t)std::llround((double)nb * (r + 1) / zone);
      for (int64_t k = b0; k < b1; ++k) part[band[k]] = regions_before + r;
    }
    taken = end;
    regions_before += zone;
  }
}

void partition_halo(const nb_mesh *m, const int32_t *part, int p, std::vector<int32_t> &owned,
                    std::vector<int32_t> &halo) {
  owned.clear();
  halo.clear();
  std::vector<char> in_halo(m->V, 0);
  for (int64_t i = 0; i < m->V; ++i) {
    if (part[i] != p) continue;
    owned.push_back((int32_t)i);
    for (int64_t q = m->row_ptr[i]; q < m->row_ptr[i + 1]; ++q) {
      const int32_t j = m->nbr[q];
      if (part[j] != p && !in_halo[j]) {
        in_halo[j] = 1;
        halo.push_back(j);
      }
    }
  }
  std::sort(halo.begin(), halo.end());
}

}  // namespace nb
