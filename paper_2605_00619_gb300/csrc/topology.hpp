// Host-side mesh topology of the AFE scheme (Sec. 4.1, 4.4): cell nodes, sub-tet gather
// maps, per-sub-tet affine geometry, cell-boundary sub-triangles ("face slots") and their
// matching across cells.  Everything here is integer bookkeeping plus FP64 geometry; the
// mass matrices are assembled and inverted on the GPU.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "refelem.hpp"

namespace afe {

// Leading dimension of a cell's M_i^-1 block: N_i rounded up to a multiple of 16, plus 8.
// Rows start on 16-byte boundaries (bulk copies of whole rows), every 16-row tile of the
// tensor-core apply stays inside a row, and LD = 8 (mod 16) makes the fragment loads of
// four consecutive rows hit 32 different shared-memory banks.
inline constexpr int minv_ld(int n) { return (n + 15) / 16 * 16 + 8; }

struct Topology {
  int N = 0, Np = 0, Nt = 0, Nf = 0;
  int64_t C = 0, T = 0, n_nodes = 0, n_slots = 0, n_groups = 0;
  int Nmax = 0, Smax = 0, slots_max = 0;

  std::vector<int64_t> node_ptr;   // [C+1] global node offset of each cell
  std::vector<int64_t> sub_ptr;    // [C+1] sub-tet offset of each cell
  std::vector<int64_t> slot_ptr;   // [C+1] face-slot offset of each cell
  std::vector<int64_t> minv_ptr;   // [C+1] offset of the dense N_i x minv_ld(N_i) block of each cell

  std::vector<uint16_t> A;         // [T*Np] cell-local node of sub-tet node j
  std::vector<double> geo;         // [T*10] adj(J) row-major (adj = det(J) J^-1), det(J)
  std::vector<double> node_xyz;    // [n_nodes*3]

  // node -> (sub-tet, local node) incidences, cell-local sub-tet index, fixed order
  std::vector<int64_t> inc_ptr;    // [n_nodes+1]
  std::vector<uint32_t> inc;       // (k_local << 5) | j

  // face slots: one per cell-boundary sub-triangle, grouped by cell
  std::vector<int32_t> slot_cell;  // [n_slots]
  std::vector<uint16_t> slot_sub;  // [n_slots] cell-local sub-tet owning the triangle
  std::vector<uint8_t> slot_loc;   // [n_slots*Nf] sub-tet-local node of each face node
  std::vector<uint16_t> slot_node; // [n_slots*Nf] cell-local node of each face node
  std::vector<double> slot_geo;    // [n_slots*4] outward unit normal (3), area
  std::vector<int64_t> slot_partner; // [n_slots] matched slot of the neighbour, or -1
  std::vector<int32_t> slot_nbr;   // [n_slots] neighbour cell, or -1 on the domain boundary

  // node -> (slot, face node) incidences for the corrector's face term
  std::vector<int64_t> finc_ptr;   // [n_nodes+1]
  std::vector<uint32_t> finc;      // (slot_local << 4) | a

  // polygonal faces: slots of one cell shared with one neighbour image, listed once per pair
  std::vector<int64_t> group_ptr;  // [n_groups+1]
  std::vector<int64_t> group_slot; // own-side slots

  std::vector<double> cell_vol;    // |P_i|
  std::vector<double> cell_h;      // 6 |P_i| / |dP_i|
  std::vector<double> cell_hsub;   // min over the cell's sub-tets of 6 |T_k| / |dT_k|
  std::vector<double> cell_diam;   // largest distance between two vertices of the cell
  double h_min = 0;
};

// Builds the topology; returns 0 on success, 2 (AFE_EMESH) or 1 (AFE_EINVAL) with a message.
int build_topology(const RefData& ref, int64_t n_vertices, const double* xyz, int64_t n_cells,
                   const int64_t* cell_subtet_ptr, const int64_t* subtet_vtx,
                   const int8_t* subtet_shift, const double period[3], bool periodic,
                   Topology* out, std::string* err);

}  // namespace afe
