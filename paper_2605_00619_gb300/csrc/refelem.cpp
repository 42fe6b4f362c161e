// Universal matrices of the AFE scheme (see refelem.hpp).
//
// The Lagrange basis is obtained by inverting the monomial Vandermonde matrix of the
// node lattice in long double; every integral of a product of monomials over the
// reference tetrahedron is exact, int r^a s^b t^c = a! b! c! / (a+b+c+3)!, and over the
// unit right triangle int u^a v^b = a! b! / (a+b+2)!.
#include "refelem.hpp"

#include <cmath>
#include <cstring>
#include <vector>

namespace afe {
namespace {

typedef long double ld;

ld fact(int n) {
  ld f = 1;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

// Solve A X = I in place (Gauss-Jordan with partial pivoting); A is n x n row-major.
bool invert(std::vector<ld>& A, int n) {
  std::vector<ld> X(n * n, 0);
  for (int i = 0; i < n; ++i) X[i * n + i] = 1;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(A[r * n + c]) > fabsl(A[p * n + c])) p = r;
    if (A[p * n + c] == 0) return false;
    if (p != c)
      for (int k = 0; k < n; ++k) {
        std::swap(A[p * n + k], A[c * n + k]);
        std::swap(X[p * n + k], X[c * n + k]);
      }
    ld piv = A[c * n + c];
    for (int k = 0; k < n; ++k) {
      A[c * n + k] /= piv;
      X[c * n + k] /= piv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      ld f = A[r * n + c];
      if (f == 0) continue;
      for (int k = 0; k < n; ++k) {
        A[r * n + k] -= f * A[c * n + k];
        X[r * n + k] -= f * X[c * n + k];
      }
    }
  }
  A = X;
  return true;
}

struct Mono3 {
  int e[3];
};

}  // namespace

int ref_node_index(const RefData& r, const int a[4]) {
  for (int j = 0; j < r.Np; ++j)
    if (r.alpha[j][0] == a[0] && r.alpha[j][1] == a[1] && r.alpha[j][2] == a[2] && r.alpha[j][3] == a[3])
      return j;
  return -1;
}

int ref_tri_index(const RefData& r, const int b[3]) {
  for (int j = 0; j < r.Nf; ++j)
    if (r.beta[j][0] == b[0] && r.beta[j][1] == b[1] && r.beta[j][2] == b[2]) return j;
  return -1;
}

bool build_ref(int N, RefData* out) {
  if (N < 1 || N > kMaxN) return false;
  RefData& R = *out;
  std::memset(&R, 0, sizeof(R));
  R.N = N;
  R.Nt = N + 1;

  // Node lattice, vertices first, then edge, face and interior nodes (by the number of
  // non-zero barycentric weights), lexicographic in the multi-index within each class.
  int np = 0;
  for (int nz = 1; nz <= 4; ++nz)
    for (int a0 = N; a0 >= 0; --a0)
      for (int a1 = N - a0; a1 >= 0; --a1)
        for (int a2 = N - a0 - a1; a2 >= 0; --a2) {
          int a3 = N - a0 - a1 - a2;
          int cnt = (a0 > 0) + (a1 > 0) + (a2 > 0) + (a3 > 0);
          if (cnt != nz) continue;
          R.alpha[np][0] = a0;
          R.alpha[np][1] = a1;
          R.alpha[np][2] = a2;
          R.alpha[np][3] = a3;
          // vertex 0 at the origin, vertices 1, 2, 3 on the r, s, t axes
          R.xi[np][0] = double(a1) / N;
          R.xi[np][1] = double(a2) / N;
          R.xi[np][2] = double(a3) / N;
          ++np;
        }
  R.Np = np;

  // Monomials r^a s^b t^c with a+b+c <= N.
  std::vector<Mono3> mono;
  for (int d = 0; d <= N; ++d)
    for (int a = d; a >= 0; --a)
      for (int b = d - a; b >= 0; --b) mono.push_back({{a, b, d - a - b}});
  if ((int)mono.size() != np) return false;

  auto powl_i = [](ld x, int e) {
    ld v = 1;
    for (int i = 0; i < e; ++i) v *= x;
    return v;
  };
  std::vector<ld> V(np * np);
  for (int i = 0; i < np; ++i)
    for (int m = 0; m < np; ++m) {
      ld r = (ld)R.alpha[i][1] / N, s = (ld)R.alpha[i][2] / N, t = (ld)R.alpha[i][3] / N;
      V[i * np + m] = powl_i(r, mono[m].e[0]) * powl_i(s, mono[m].e[1]) * powl_i(t, mono[m].e[2]);
    }
  if (!invert(V, np)) return false;  // V now holds C with phi_j = sum_m C[m][j] mono_m
  auto C = [&](int m, int j) { return V[m * np + j]; };

  auto int_tet = [&](int a, int b, int c) { return fact(a) * fact(b) * fact(c) / fact(a + b + c + 3); };
  for (int m = 0; m < np; ++m)
    for (int l = 0; l < np; ++l) {
      ld acc = 0, sd[3] = {0, 0, 0};
      for (int p = 0; p < np; ++p)
        for (int q = 0; q < np; ++q) {
          ld cp = C(p, m), cq = C(q, l);
          if (cp == 0 || cq == 0) continue;
          const int* ep = mono[p].e;
          const int* eq = mono[q].e;
          acc += cp * cq * int_tet(ep[0] + eq[0], ep[1] + eq[1], ep[2] + eq[2]);
          for (int d = 0; d < 3; ++d) {
            if (eq[d] == 0) continue;
            int e2[3] = {ep[0] + eq[0], ep[1] + eq[1], ep[2] + eq[2]};
            e2[d] -= 1;
            sd[d] += cp * cq * eq[d] * int_tet(e2[0], e2[1], e2[2]);
          }
        }
      R.M[m][l] = (double)acc;
      for (int d = 0; d < 3; ++d) R.S[d][m][l] = (double)sd[d];
    }
  // nodal derivative matrices
  for (int d = 0; d < 3; ++d)
    for (int j = 0; j < np; ++j)
      for (int l = 0; l < np; ++l) {
        ld x[3] = {(ld)R.alpha[j][1] / N, (ld)R.alpha[j][2] / N, (ld)R.alpha[j][3] / N};
        ld acc = 0;
        for (int p = 0; p < np; ++p) {
          const int* e = mono[p].e;
          if (e[d] == 0) continue;
          ld v = C(p, l) * e[d];
          for (int c = 0; c < 3; ++c) v *= powl_i(x[c], e[c] - (c == d ? 1 : 0));
          acc += v;
        }
        R.D[d][j][l] = (double)acc;
      }

  // Triangle lattice and face mass on the unit right triangle (u, v): vertex 0 at the
  // origin, vertex 1 at u = 1, vertex 2 at v = 1.
  int nf = 0;
  for (int b0 = N; b0 >= 0; --b0)
    for (int b1 = N - b0; b1 >= 0; --b1) {
      R.beta[nf][0] = b0;
      R.beta[nf][1] = b1;
      R.beta[nf][2] = N - b0 - b1;
      ++nf;
    }
  R.Nf = nf;
  std::vector<int> m2a, m2b;
  for (int d = 0; d <= N; ++d)
    for (int a = d; a >= 0; --a) {
      m2a.push_back(a);
      m2b.push_back(d - a);
    }
  std::vector<ld> V2(nf * nf);
  for (int i = 0; i < nf; ++i)
    for (int m = 0; m < nf; ++m) {
      ld u = (ld)R.beta[i][1] / N, v = (ld)R.beta[i][2] / N;
      V2[i * nf + m] = powl_i(u, m2a[m]) * powl_i(v, m2b[m]);
    }
  if (!invert(V2, nf)) return false;
  for (int a = 0; a < nf; ++a)
    for (int b = 0; b < nf; ++b) {
      ld acc = 0;
      for (int p = 0; p < nf; ++p)
        for (int q = 0; q < nf; ++q) {
          int ea = m2a[p] + m2a[q], eb = m2b[p] + m2b[q];
          acc += V2[p * nf + a] * V2[q * nf + b] * fact(ea) * fact(eb) / fact(ea + eb + 2);
        }
      R.Z[a][b] = (double)acc;
    }

  // Gauss-Legendre points of [-1, 1] by Newton iteration on P_{Nt}, mapped to [0, 1].
  const int nt = R.Nt;
  for (int i = 0; i < nt; ++i) {
    ld x = cosl(3.14159265358979323846264338327950288L * (i + 0.75L) / (nt + 0.5L));
    ld dp = 0;
    for (int it = 0; it < 100; ++it) {
      ld p0 = 1, p1 = x;
      for (int k = 2; k <= nt; ++k) {
        ld p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      ld pn = (nt == 1) ? x : p1, pnm1 = (nt == 1) ? 1 : p0;
      dp = nt * (x * pn - pnm1) / (x * x - 1);
      ld dx = pn / dp;
      x -= dx;
      if (fabsl(dx) < 1e-30L) break;
    }
    // recompute derivative at the converged point for the weight
    ld p0 = 1, p1 = x;
    for (int k = 2; k <= nt; ++k) {
      ld p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    ld pn = (nt == 1) ? x : p1, pnm1 = (nt == 1) ? 1 : p0;
    dp = nt * (x * pn - pnm1) / (x * x - 1);
    ld wgt = 2 / ((1 - x * x) * dp * dp);
    R.tau[nt - 1 - i] = (double)((x + 1) / 2);   // ascending order
    R.w[nt - 1 - i] = (double)(wgt / 2);
  }
  // Lagrange basis through tau: values at 0 and 1, derivative at the nodes
  auto psi = [&](int s, ld x) {
    ld v = 1;
    for (int r = 0; r < nt; ++r)
      if (r != s) v *= (x - (ld)R.tau[r]) / ((ld)R.tau[s] - (ld)R.tau[r]);
    return v;
  };
  auto dpsi = [&](int s, ld x) {
    ld tot = 0;
    for (int q = 0; q < nt; ++q) {
      if (q == s) continue;
      ld v = 1 / ((ld)R.tau[s] - (ld)R.tau[q]);
      for (int r = 0; r < nt; ++r)
        if (r != s && r != q) v *= (x - (ld)R.tau[r]) / ((ld)R.tau[s] - (ld)R.tau[r]);
      tot += v;
    }
    return tot;
  };
  std::vector<ld> K(nt * nt);
  for (int s = 0; s < nt; ++s) {
    R.psi0[s] = (double)psi(s, 0);
    R.psi1[s] = (double)psi(s, 1);
    for (int t = 0; t < nt; ++t) {
      // the Gauss rule is exact for int psi_s' psi_t (degree 2N-1)
      K[s * nt + t] = psi(s, 1) * psi(t, 1) - (ld)R.w[t] * dpsi(s, (ld)R.tau[t]);
      R.K1t[s][t] = (double)K[s * nt + t];
    }
  }
  if (!invert(K, nt)) return false;
  for (int s = 0; s < nt; ++s)
    for (int t = 0; t < nt; ++t) R.K1tinv[s][t] = (double)K[s * nt + t];
  return true;
}

}  // namespace afe
