// Universal (mesh-independent) matrices of the AFE scheme for degree N = 1..4.
//
// Reference tetrahedron {(r,s,t) >= 0, r+s+t <= 1} with the equispaced P_N node lattice
// of App. A; Lagrange basis from the nodal property phi_j(x_m) = delta_jm (Sec. 4.1);
// quadrature-free matrices as exact polynomial integrals over the reference element
// (Sec. 4.3, 4.4); time basis = Lagrange polynomials through the N+1 Gauss-Legendre
// points of [0,1] (Sec. 4.3).
#pragma once

namespace afe {

constexpr int kMaxN = 4;
constexpr int kMaxNp = 35;  // (N+1)(N+2)(N+3)/6 at N = 4
constexpr int kMaxNt = 5;   // N+1
constexpr int kMaxNf = 15;  // (N+1)(N+2)/2

struct RefData {
  int N, Np, Nt, Nf;
  int alpha[kMaxNp][4];                 // barycentric multi-index of node j (sum N), vertex order 0..3
  double xi[kMaxNp][3];                 // node coordinates on the reference tet
  double M[kMaxNp][kMaxNp];             // int phi_m phi_l
  double S[3][kMaxNp][kMaxNp];          // int phi_m d/dxi_d phi_l
  double D[3][kMaxNp][kMaxNp];          // D[d][j][l] = d/dxi_d phi_l at node j
  int beta[kMaxNf][3];                  // triangle lattice multi-indices
  double Z[kMaxNf][kMaxNf];             // face mass on the unit right triangle (area 1/2)
  double tau[kMaxNt], w[kMaxNt];        // Gauss-Legendre points and weights on [0,1]
  double psi0[kMaxNt], psi1[kMaxNt];    // psi_t(0), psi_t(1)
  double K1t[kMaxNt][kMaxNt];           // psi_s(1)psi_t(1) - int psi_s' psi_t
  double K1tinv[kMaxNt][kMaxNt];
};

// Fills `out` for degree N (1..4); returns false on an unsupported N.
bool build_ref(int N, RefData* out);

// Index of the node with multi-index a[4], or -1.
int ref_node_index(const RefData& r, const int a[4]);

// Index of the triangle-lattice node with multi-index b[3], or -1.
int ref_tri_index(const RefData& r, const int b[3]);

}  // namespace afe
