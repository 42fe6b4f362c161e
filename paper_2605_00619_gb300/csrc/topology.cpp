// Host-side mesh topology of the AFE scheme (see topology.hpp).
#include "topology.hpp"

#include <algorithm>
#include <array>
#include <tuple>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <thread>
#include <unordered_map>

namespace afe {
namespace {

struct VKey {  // a sub-tet vertex in the frame of its cell: global id + periodic image
  int64_t id;
  int8_t s[3];
  bool operator<(const VKey& o) const {
    if (id != o.id) return id < o.id;
    for (int c = 0; c < 3; ++c)
      if (s[c] != o.s[c]) return s[c] < o.s[c];
    return false;
  }
  bool operator==(const VKey& o) const { return id == o.id && s[0] == o.s[0] && s[1] == o.s[1] && s[2] == o.s[2]; }
};

struct TriKey {  // canonical translate of a triangle: sorted (id, shift - ref shift)
  VKey v[3];
  bool operator==(const TriKey& o) const { return v[0] == o.v[0] && v[1] == o.v[1] && v[2] == o.v[2]; }
};

struct TriKeyHash {
  size_t operator()(const TriKey& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < 3; ++i) {
      h ^= (uint64_t)k.v[i].id + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
      for (int c = 0; c < 3; ++c) h = (h ^ (uint8_t)k.v[i].s[c]) * 1099511628211ull;
    }
    return (size_t)h;
  }
};

struct SlotTmp {
  uint16_t sub;
  uint8_t loc[kMaxNf];
  uint16_t node[kMaxNf];
  double normal[3];
  double area;
  TriKey key;
  int8_t ref[3];  // image shift of the reference vertex in this cell's frame
};

struct CellOut {
  int err = 0;
  std::string msg;
  int Ni = 0, S = 0;
  std::vector<uint16_t> A;
  std::vector<double> geo;
  std::vector<double> xyz;
  std::vector<int32_t> inc_cnt;
  std::vector<uint32_t> inc;
  std::vector<SlotTmp> slots;
  double vol = 0;
  double hsub = 1e300;  // smallest 6 |T_k| / |dT_k| over the cell's sub-tets
  double diam = 0;      // largest distance between two vertices of the cell
};

inline uint64_t pack_node(int n, const int* lv, const int* al) {
  // sorted (local vertex, weight) pairs with weight > 0: 12-bit vertex, 3-bit weight (N <= 4),
  // after the count in the low 4 bits
  int idx[4], m = 0;
  for (int k = 0; k < n; ++k)
    if (al[k] > 0) idx[m++] = k;
  for (int a = 1; a < m; ++a)
    for (int b = a; b > 0 && lv[idx[b]] < lv[idx[b - 1]]; --b) std::swap(idx[b], idx[b - 1]);
  uint64_t key = (uint64_t)m;
  for (int k = 0; k < m; ++k) key |= (uint64_t)(((lv[idx[k]] & 0xfff) << 3) | (al[idx[k]] & 7)) << (4 + 15 * k);
  return key;
}

void process_cell(const RefData& R, const double* xyz, const int64_t* vtx, const int8_t* shift,
                  const double period[3], int64_t k0, int64_t k1, int64_t n_vertices, CellOut* out) {
  const int N = R.N, Np = R.Np, Nf = R.Nf;
  const int S = (int)(k1 - k0);
  out->S = S;
  if (S <= 0 || S > 65535) {
    out->err = 2;
    out->msg = "cell with no sub-tets or more than 65535 sub-tets";
    return;
  }
  std::vector<VKey> lverts;  // local vertex table
  std::vector<double> lxyz;  // its coordinates (periodic images applied)
  std::vector<std::array<int, 4>> sub_lv(S);
  std::vector<std::array<double, 12>> X(S);
  out->geo.resize((size_t)S * 10);
  out->A.resize((size_t)S * Np);
  for (int k = 0; k < S; ++k) {
    VKey vk[4];
    double P[4][3];
    for (int m = 0; m < 4; ++m) {
      int64_t id = vtx[(k0 + k) * 4 + m];
      if (id < 0 || id >= n_vertices) {
        out->err = 1;
        out->msg = "sub-tet vertex id out of range";
        return;
      }
      vk[m].id = id;
      for (int c = 0; c < 3; ++c) {
        vk[m].s[c] = shift ? shift[((k0 + k) * 4 + m) * 3 + c] : 0;
        P[m][c] = xyz[id * 3 + c] + (double)vk[m].s[c] * period[c];
      }
    }
    auto detJ = [&](double Q[4][3]) {
      double a[3], b[3], c[3];
      for (int d = 0; d < 3; ++d) {
        a[d] = Q[1][d] - Q[0][d];
        b[d] = Q[2][d] - Q[0][d];
        c[d] = Q[3][d] - Q[0][d];
      }
      return a[0] * (b[1] * c[2] - b[2] * c[1]) - b[0] * (a[1] * c[2] - a[2] * c[1]) + c[0] * (a[1] * b[2] - a[2] * b[1]);
    };
    double det = detJ(P);
    if (det < 0) {  // reorient by exchanging the first two vertices
      std::swap(vk[0], vk[1]);
      for (int d = 0; d < 3; ++d) std::swap(P[0][d], P[1][d]);
      det = -det;
    }
    if (!(det > 0) || !std::isfinite(det)) {
      out->err = 2;
      out->msg = "sub-tet with zero or non-finite volume";
      return;
    }
    // J columns: P1-P0, P2-P0, P3-P0; adj(J) = det(J) J^-1 (cofactor transpose)
    double J[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) J[r][c] = P[c + 1][r] - P[0][r];
    double* g = &out->geo[(size_t)k * 10];
    g[0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    g[1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    g[2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    g[3] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    g[4] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    g[5] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    g[6] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    g[7] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    g[8] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    g[9] = det;
    out->vol += det / 6.0;
    {
      auto tri = [&](int a, int b, int c) {  // area of the sub-tet face (a, b, c)
        double u[3], v[3];
        for (int d = 0; d < 3; ++d) {
          u[d] = P[b][d] - P[a][d];
          v[d] = P[c][d] - P[a][d];
        }
        const double x = u[1] * v[2] - u[2] * v[1], y = u[2] * v[0] - u[0] * v[2], z = u[0] * v[1] - u[1] * v[0];
        return 0.5 * std::sqrt(x * x + y * y + z * z);
      };
      const double area = tri(0, 1, 2) + tri(0, 1, 3) + tri(0, 2, 3) + tri(1, 2, 3);
      out->hsub = std::min(out->hsub, det / area);  // 6 (det / 6) / area
    }
    for (int m = 0; m < 4; ++m) {
      int found = -1;
      for (size_t q = 0; q < lverts.size(); ++q)
        if (lverts[q] == vk[m]) {
          found = (int)q;
          break;
        }
      if (found < 0) {
        found = (int)lverts.size();
        lverts.push_back(vk[m]);
        lxyz.push_back(P[m][0]);
        lxyz.push_back(P[m][1]);
        lxyz.push_back(P[m][2]);
      }
      sub_lv[k][m] = found;
      for (int d = 0; d < 3; ++d) X[k][m * 3 + d] = P[m][d];
    }
  }
  if (lverts.size() > 0xfff) {
    out->err = 2;
    out->msg = "cell with too many vertices";
    return;
  }
  for (size_t a = 0; a < lverts.size(); ++a)
    for (size_t b = a + 1; b < lverts.size(); ++b) {
      double d2 = 0;
      for (int d = 0; d < 3; ++d) {
        const double e = lxyz[a * 3 + d] - lxyz[b * 3 + d];
        d2 += e * e;
      }
      out->diam = std::max(out->diam, d2);
    }
  out->diam = std::sqrt(out->diam);

  // AFE nodes: the union without repetition of the sub-tets' P_N nodes (Sec. 4.1)
  std::unordered_map<uint64_t, int> nodes;
  nodes.reserve((size_t)S * Np);
  for (int k = 0; k < S; ++k)
    for (int j = 0; j < Np; ++j) {
      uint64_t key = pack_node(4, sub_lv[k].data(), R.alpha[j]);
      auto it = nodes.find(key);
      int id;
      if (it == nodes.end()) {
        id = (int)nodes.size();
        nodes.emplace(key, id);
        for (int d = 0; d < 3; ++d) {
          double x = 0;
          for (int m = 0; m < 4; ++m) x += (double)R.alpha[j][m] / N * X[k][m * 3 + d];
          out->xyz.push_back(x);
        }
      } else {
        id = it->second;
      }
      out->A[(size_t)k * Np + j] = (uint16_t)id;
    }
  const int Ni = (int)nodes.size();
  if (Ni > 65535) {
    out->err = 2;
    out->msg = "cell with more than 65535 nodes";
    return;
  }
  out->Ni = Ni;

  // sub-tet incidences of every node, in (k, j) order
  out->inc_cnt.assign(Ni, 0);
  for (int k = 0; k < S; ++k)
    for (int j = 0; j < Np; ++j) out->inc_cnt[out->A[(size_t)k * Np + j]]++;
  std::vector<int> off(Ni + 1, 0);
  for (int n = 0; n < Ni; ++n) off[n + 1] = off[n] + out->inc_cnt[n];
  out->inc.resize(off[Ni]);
  {
    std::vector<int> fill(off.begin(), off.end() - 1);
    for (int k = 0; k < S; ++k)
      for (int j = 0; j < Np; ++j) out->inc[fill[out->A[(size_t)k * Np + j]]++] = ((uint32_t)k << 6) | (uint32_t)j;
  }

  // triangles of the subgrid: interior ones appear twice, cell-boundary ones once
  std::map<std::array<int, 3>, std::vector<std::pair<int, int>>> tris;
  std::map<std::array<int, 2>, int> edges;
  for (int k = 0; k < S; ++k) {
    for (int o = 0; o < 4; ++o) {
      std::array<int, 3> t;
      int c = 0;
      for (int m = 0; m < 4; ++m)
        if (m != o) t[c++] = sub_lv[k][m];
      std::sort(t.begin(), t.end());
      tris[t].push_back({k, o});
    }
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b) {
        std::array<int, 2> e = {std::min(sub_lv[k][a], sub_lv[k][b]), std::max(sub_lv[k][a], sub_lv[k][b])};
        edges[e] = 1;
      }
  }
  long chi = (long)lverts.size() - (long)edges.size() + (long)tris.size() - S;
  std::map<std::array<int, 2>, int> bedges;
  for (auto& kv : tris) {
    if (kv.second.size() > 2) {
      out->err = 2;
      out->msg = "non-conforming subgrid: a triangle shared by more than two sub-tets of one cell";
      return;
    }
    if (kv.second.size() != 1) continue;
    const auto& t = kv.first;
    bedges[{t[0], t[1]}]++;
    bedges[{t[0], t[2]}]++;
    bedges[{t[1], t[2]}]++;
  }
  for (auto& kv : bedges)
    if (kv.second != 2) {
      out->err = 2;
      out->msg = "cell boundary is not a closed 2-manifold";
      return;
    }
  if (chi != 1) {
    out->err = 2;
    out->msg = "cell subgrid is not a topological ball (Euler characteristic != 1)";
    return;
  }

  // face slots
  for (auto& kv : tris) {
    if (kv.second.size() != 1) continue;
    int k = kv.second[0].first, o = kv.second[0].second;
    int ms[3], c = 0;
    for (int m = 0; m < 4; ++m)
      if (m != o) ms[c++] = m;
    VKey v[3];
    for (int q = 0; q < 3; ++q) v[q] = lverts[sub_lv[k][ms[q]]];
    VKey ref = std::min({v[0], v[1], v[2]});
    SlotTmp sl;
    std::memset(&sl, 0, sizeof(sl));
    for (int q = 0; q < 3; ++q) {
      v[q].id = v[q].id;
      for (int d = 0; d < 3; ++d) v[q].s[d] = (int8_t)(v[q].s[d] - ref.s[d]);
    }
    for (int d = 0; d < 3; ++d) sl.ref[d] = ref.s[d];
    int order[3] = {0, 1, 2};
    std::sort(order, order + 3, [&](int a, int b) { return v[a] < v[b]; });
    for (int q = 0; q < 3; ++q) sl.key.v[q] = v[order[q]];
    sl.sub = (uint16_t)k;
    for (int f = 0; f < Nf; ++f) {
      int al[4] = {0, 0, 0, 0};
      for (int q = 0; q < 3; ++q) al[ms[order[q]]] = R.beta[f][q];
      int j = ref_node_index(R, al);
      sl.loc[f] = (uint8_t)j;
      sl.node[f] = out->A[(size_t)k * Np + j];
    }
    const double* P = X[k].data();
    int a = ms[order[0]], b = ms[order[1]], cc = ms[order[2]];
    double e1[3], e2[3], nrm[3], to[3];
    for (int d = 0; d < 3; ++d) {
      e1[d] = P[b * 3 + d] - P[a * 3 + d];
      e2[d] = P[cc * 3 + d] - P[a * 3 + d];
      to[d] = P[o * 3 + d] - P[a * 3 + d];
    }
    nrm[0] = e1[1] * e2[2] - e1[2] * e2[1];
    nrm[1] = e1[2] * e2[0] - e1[0] * e2[2];
    nrm[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double len = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
    double sgn = (nrm[0] * to[0] + nrm[1] * to[1] + nrm[2] * to[2]) > 0 ? -1.0 : 1.0;
    if (!(len > 0)) {
      out->err = 2;
      out->msg = "zero-area cell-boundary triangle";
      return;
    }
    for (int d = 0; d < 3; ++d) sl.normal[d] = sgn * nrm[d] / len;
    sl.area = 0.5 * len;
    out->slots.push_back(sl);
  }
  if (out->slots.size() > 65535) {
    out->err = 2;
    out->msg = "cell with more than 65535 boundary triangles";
  }
}

}  // namespace

int build_topology(const RefData& R, int64_t n_vertices, const double* xyz, int64_t n_cells,
                   const int64_t* ptr, const int64_t* vtx, const int8_t* shift, const double period[3],
                   bool periodic, Topology* out, std::string* err) {
  Topology& T = *out;
  T.N = R.N;
  T.Np = R.Np;
  T.Nt = R.Nt;
  T.Nf = R.Nf;
  T.C = n_cells;
  if (n_cells <= 0 || ptr[0] != 0) {
    *err = "empty mesh or cell_subtet_ptr[0] != 0";
    return 1;
  }
  for (int64_t c = 0; c < n_cells; ++c)
    if (ptr[c + 1] <= ptr[c]) {
      *err = "cell_subtet_ptr must be strictly increasing";
      return 1;
    }
  if (n_cells > 0x7fffffffLL) {
    *err = "too many cells";
    return 1;
  }
  T.T = ptr[n_cells];

  std::vector<CellOut> cells(n_cells);
  unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::atomic<int64_t> next(0);
  auto worker = [&]() {
    for (;;) {
      int64_t c0 = next.fetch_add(64);
      if (c0 >= n_cells) break;
      int64_t c1 = std::min(n_cells, c0 + 64);
      for (int64_t c = c0; c < c1; ++c) process_cell(R, xyz, vtx, shift, period, ptr[c], ptr[c + 1], n_vertices, &cells[c]);
    }
  };
  std::vector<std::thread> pool;
  for (unsigned t = 0; t < nth; ++t) pool.emplace_back(worker);
  for (auto& th : pool) th.join();
  for (int64_t c = 0; c < n_cells; ++c)
    if (cells[c].err) {
      *err = "cell " + std::to_string(c) + ": " + cells[c].msg;
      return cells[c].err;
    }

  // offsets
  T.node_ptr.assign(n_cells + 1, 0);
  T.sub_ptr.assign(n_cells + 1, 0);
  T.slot_ptr.assign(n_cells + 1, 0);
  T.minv_ptr.assign(n_cells + 1, 0);
  for (int64_t c = 0; c < n_cells; ++c) {
    T.node_ptr[c + 1] = T.node_ptr[c] + cells[c].Ni;
    T.sub_ptr[c + 1] = T.sub_ptr[c] + cells[c].S;
    T.slot_ptr[c + 1] = T.slot_ptr[c] + (int64_t)cells[c].slots.size();
    // rows padded to minv_ld words, blocks to a multiple of 32 words (128 bytes)
    const int64_t ld = minv_ld(cells[c].Ni);
    T.minv_ptr[c + 1] = T.minv_ptr[c] + ((int64_t)cells[c].Ni * ld + 31) / 32 * 32;
    T.Nmax = std::max(T.Nmax, cells[c].Ni);
    T.Smax = std::max(T.Smax, cells[c].S);
    T.slots_max = std::max(T.slots_max, (int)cells[c].slots.size());
  }
  T.n_nodes = T.node_ptr[n_cells];
  T.n_slots = T.slot_ptr[n_cells];
  const int Np = R.Np, Nf = R.Nf;
  T.A.resize((size_t)T.T * Np);
  T.geo.resize((size_t)T.T * 10);
  T.node_xyz.resize((size_t)T.n_nodes * 3);
  T.inc_ptr.assign(T.n_nodes + 1, 0);
  T.finc_ptr.assign(T.n_nodes + 1, 0);
  T.slot_cell.resize(T.n_slots);
  T.slot_sub.resize(T.n_slots);
  T.slot_loc.resize((size_t)T.n_slots * Nf);
  T.slot_node.resize((size_t)T.n_slots * Nf);
  T.slot_geo.resize((size_t)T.n_slots * 4);
  T.slot_partner.assign(T.n_slots, -1);
  T.slot_nbr.assign(T.n_slots, -1);
  T.cell_vol.resize(n_cells);
  T.cell_h.resize(n_cells);
  T.cell_hsub.resize(n_cells);
  T.cell_diam.resize(n_cells);

  for (int64_t c = 0; c < n_cells; ++c) {
    const CellOut& co = cells[c];
    std::copy(co.A.begin(), co.A.end(), T.A.begin() + T.sub_ptr[c] * Np);
    std::copy(co.geo.begin(), co.geo.end(), T.geo.begin() + T.sub_ptr[c] * 10);
    std::copy(co.xyz.begin(), co.xyz.end(), T.node_xyz.begin() + T.node_ptr[c] * 3);
    for (int n = 0; n < co.Ni; ++n) T.inc_ptr[T.node_ptr[c] + n + 1] = co.inc_cnt[n];
    T.cell_vol[c] = co.vol;
    T.cell_hsub[c] = co.hsub;
    T.cell_diam[c] = co.diam;
    for (size_t s = 0; s < co.slots.size(); ++s) {
      int64_t g = T.slot_ptr[c] + (int64_t)s;
      const SlotTmp& sl = co.slots[s];
      T.slot_cell[g] = (int32_t)c;
      T.slot_sub[g] = sl.sub;
      for (int f = 0; f < Nf; ++f) {
        T.slot_loc[g * Nf + f] = sl.loc[f];
        T.slot_node[g * Nf + f] = sl.node[f];
        T.finc_ptr[T.node_ptr[c] + sl.node[f] + 1]++;
      }
      for (int d = 0; d < 3; ++d) T.slot_geo[g * 4 + d] = sl.normal[d];
      T.slot_geo[g * 4 + 3] = sl.area;
    }
  }
  for (int64_t n = 0; n < T.n_nodes; ++n) {
    T.inc_ptr[n + 1] += T.inc_ptr[n];
    T.finc_ptr[n + 1] += T.finc_ptr[n];
  }
  T.inc.resize(T.inc_ptr[T.n_nodes]);
  T.finc.resize(T.finc_ptr[T.n_nodes]);
  for (int64_t c = 0; c < n_cells; ++c) {
    const CellOut& co = cells[c];
    // cell-local incidence lists were built in node order already
    int64_t base = T.inc_ptr[T.node_ptr[c]];
    std::copy(co.inc.begin(), co.inc.end(), T.inc.begin() + base);
    std::vector<int64_t> fill(co.Ni);
    for (int n = 0; n < co.Ni; ++n) fill[n] = T.finc_ptr[T.node_ptr[c] + n];
    for (size_t s = 0; s < co.slots.size(); ++s)
      for (int f = 0; f < Nf; ++f) T.finc[fill[co.slots[s].node[f]]++] = ((uint32_t)s << 4) | (uint32_t)f;
  }

  // match cell-boundary triangles across cells
  std::unordered_map<TriKey, int64_t, TriKeyHash> table;
  table.reserve((size_t)T.n_slots);
  for (int64_t c = 0; c < n_cells; ++c)
    for (size_t s = 0; s < cells[c].slots.size(); ++s) {
      int64_t g = T.slot_ptr[c] + (int64_t)s;
      const SlotTmp& sl = cells[c].slots[s];
      auto it = table.find(sl.key);
      if (it == table.end()) {
        table.emplace(sl.key, g);
        continue;
      }
      int64_t h = it->second;
      if (h < 0) {
        *err = "a cell-boundary triangle is shared by more than two cells";
        return 2;
      }
      T.slot_partner[g] = h;
      T.slot_partner[h] = g;
      T.slot_nbr[g] = T.slot_cell[h];
      T.slot_nbr[h] = (int32_t)c;
      // one geometry per pair: the first slot's normal and area, negated normal on the other side
      for (int d = 0; d < 3; ++d) T.slot_geo[g * 4 + d] = -T.slot_geo[h * 4 + d];
      T.slot_geo[g * 4 + 3] = T.slot_geo[h * 4 + 3];
      it->second = -1;
    }
  if (periodic)
    for (int64_t g = 0; g < T.n_slots; ++g)
      if (T.slot_partner[g] < 0) {
        *err = "unmatched cell-boundary triangle on a periodic mesh (cell " + std::to_string(T.slot_cell[g]) + ")";
        return 2;
      }

  // characteristic lengths
  T.h_min = 1e300;
  for (int64_t c = 0; c < n_cells; ++c) {
    double area = 0;
    for (int64_t g = T.slot_ptr[c]; g < T.slot_ptr[c + 1]; ++g) area += T.slot_geo[g * 4 + 3];
    T.cell_h[c] = 6.0 * T.cell_vol[c] / area;
    T.h_min = std::min(T.h_min, T.cell_h[c]);
  }

  // polygonal faces: group each cell's slots by (neighbour, image offset); keep the group
  // from one side of each pair only
  T.group_ptr.assign(1, 0);
  T.group_slot.clear();
  for (int64_t c = 0; c < n_cells; ++c) {
    std::map<std::array<int64_t, 4>, std::vector<int64_t>> groups;
    std::vector<int64_t> order;
    for (int64_t g = T.slot_ptr[c]; g < T.slot_ptr[c + 1]; ++g) {
      int64_t p = T.slot_partner[g];
      if (p < 0) {
        T.group_slot.push_back(g);
        T.group_ptr.push_back((int64_t)T.group_slot.size());
        continue;
      }
      int64_t nb = T.slot_nbr[g];
      const SlotTmp& a = cells[c].slots[g - T.slot_ptr[c]];
      const SlotTmp& b = cells[nb].slots[p - T.slot_ptr[nb]];
      std::array<int64_t, 4> key = {nb, a.ref[0] - b.ref[0], a.ref[1] - b.ref[1], a.ref[2] - b.ref[2]};
      bool canon = nb > c;
      if (nb == c) canon = std::make_tuple(key[1], key[2], key[3]) > std::make_tuple(0LL, 0LL, 0LL);
      if (!canon) continue;
      groups[key].push_back(g);
    }
    for (auto& kv : groups) {
      for (int64_t g : kv.second) T.group_slot.push_back(g);
      T.group_ptr.push_back((int64_t)T.group_slot.size());
    }
  }
  T.n_groups = (int64_t)T.group_ptr.size() - 1;
  return 0;
}

}  // namespace afe
