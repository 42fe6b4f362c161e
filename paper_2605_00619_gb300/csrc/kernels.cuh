// Device kernels of the ADER-AFE-DG step (sm_103a).  Included by afe.cu only.
//
// Layouts (all in HBM, resident for the life of a mesh handle):
//   u        [n_nodes][5] FP64 master state, node-major, contiguous per cell
//   minv     per cell a dense N_i x N_i block (symmetric), FP64 or FP32 copy
//   A        [T][Np] cell-local node of every sub-tet node (uint16)
//   geo      [T][10] adj(J_ik) (row-major, = det J J^-1) and det J_ik (FP64)
//   slot_*   one entry per cell-boundary sub-triangle ("face slot"), cell-major
// Per-step intermediates (Real = double or float):
//   vol      [n_nodes][5]            volume term of the corrector
//   slot_q   [n_slots][Nf][5]        time-integrated predictor at the face nodes
//   slot_fn  [n_slots][Nf][5]        time-integrated flux . (own outward normal)
//   slot_G   [n_slots][Nf][5]        Rusanov flux, own-side orientation
#pragma once

#include <cstdint>

#include "refelem.hpp"
#include "topology.hpp"

namespace afe {

constexpr int np_of(int N) { return (N + 1) * (N + 2) * (N + 3) / 6; }
constexpr int nf_of(int N) { return (N + 1) * (N + 2) / 2; }

enum FlagIndex { F_NONCONV = 0, F_NONFINITE = 1, F_TROUBLED = 2, F_ITERSUM = 3, F_TIMEOUT = 4, F_COUNT = 8 };

struct DevMesh {
  int N;
  int64_t C, n_nodes, n_slots, n_groups;
  int Nmax, Smax;
  const int64_t* node_ptr;
  const int64_t* sub_ptr;
  const int64_t* slot_ptr;
  const int64_t* minv_ptr;
  const uint16_t* A;
  const double* geo;
  unsigned char* sub32;  // packed FP32 sub-tet records, reduced-precision path only
  const int64_t* inc_ptr;
  const uint32_t* inc;
  const int32_t* slot_cell;
  const uint16_t* slot_sub;
  const uint8_t* slot_loc;
  const uint16_t* slot_node;
  const double* slot_geo;
  const int64_t* slot_partner;
  const int32_t* slot_nbr;
  const int64_t* finc_ptr;
  const uint32_t* finc;
  const int64_t* group_ptr;
  const int64_t* group_slot;
  const double* cell_vol;
  const double* cell_h;
  const double* cell_hv;  // length in the viscous term of the time step (cell_h or the sub-tet length)
  double* wvec;
  double* minv64;
  float* minv32;
  double* u;
  void* vol;
  void* slot_q;
  void* slot_fn;
  void* slot_G;
  int32_t* iters;
  double* beta;
  double* mu;     // per-cell dynamic viscosity mu_i (physical + artificial)
  double* means;  // [C][5] cell means
  double* dt;     // device scalar: time step of the current step
  double* tacc;   // device scalar: accumulated time
  unsigned long long* maxbits;
  int* flags;
  int* work;      // work counter of the persistent predictor
  double* qbar_diag;
  // physics
  double gamma, Rgas, cv, cfl, m1, mu0, Pr, kappa0, tol, h_min;
  int picard_max, limiter, eq;
  int first_wait_polls;  // poll limit of the FP32 predictor's first bounded wait per cell
};

// A set of meshes stepped by one launch per stage (one mesh is a batch of one).  The whole
// table travels as one __grid_constant__ kernel parameter (about 31 KB, below the 32 KB
// parameter limit), so every field read stays a constant-bank load as with a single DevMesh
// passed by value, and a captured graph node carries its own copy of the table.
constexpr int kMaxBatch = 64;
struct Batch {
  int nh;                        // members in use
  int Nmax, Smax;                // maxima over the members (shared-memory layout)
  int ring_cap;                  // FP32 predictor: most M_i^-1 ring stages (0: as many as fit)
  int narrow;                    // FP32 predictor: 1 = narrow right-hand-side chunks everywhere
  int pad;
  int* work;                     // work counter of the persistent predictor
  const int32_t* order;          // global cells in the order the predictor takes them (NULL: index order)
  int64_t cpre[kMaxBatch + 1];   // prefix sums of the members' cells
  int64_t gpre[kMaxBatch + 1];   // prefix sums of the members' polygonal faces
  DevMesh tab[kMaxBatch];
};

// Member holding global item x of a prefix-sum array (largest h with pre[h] <= x).
__device__ __forceinline__ int batch_find(const int64_t* __restrict__ pre, int nh, int64_t x) {
  int lo = 0, hi = nh - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ double cell_kappa(const DevMesh& m, double mu_i) {
  return m.kappa0 >= 0.0 ? m.kappa0 : mu_i * m.gamma * m.cv / m.Pr;
}

// Physical flux F_e(Q, grad Q) of Sec. 2: F[e][var].  gq[e][var] = dQ_var/dx_e (only read
// when visc).  sigma = (p + 2/3 mu div v) I - mu (grad v + grad v^T); energy flux
// v . (rho E I + sigma) - kappa grad T, T = p / (rho R).
template <typename Real>
__device__ __forceinline__ void phys_flux(const Real* Q, const Real (*gq)[5], bool visc, Real mu, Real kap,
                                          Real gam, Real Rg, Real F[3][5]) {
  const Real rho = Q[0];
  const Real ir = Real(1) / rho;
  const Real v[3] = {Q[1] * ir, Q[2] * ir, Q[3] * ir};
  const Real vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  const Real p = (gam - Real(1)) * (Q[4] - Real(0.5) * rho * vv);
  Real sig[3][3] = {{p, 0, 0}, {0, p, 0}, {0, 0, p}};
  Real heat[3] = {0, 0, 0};
  if (visc) {
    Real dv[3][3];  // dv[e][a] = d v_a / d x_e
#pragma unroll
    for (int e = 0; e < 3; ++e)
#pragma unroll
      for (int a = 0; a < 3; ++a) dv[e][a] = (gq[e][1 + a] - v[a] * gq[e][0]) * ir;
    const Real div = dv[0][0] + dv[1][1] + dv[2][2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int e = 0; e < 3; ++e) sig[a][e] -= mu * (dv[e][a] + dv[a][e]);
      sig[a][a] += Real(2.0 / 3.0) * mu * div;
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const Real dp = (gam - Real(1)) *
                      (gq[e][4] - Real(0.5) * vv * gq[e][0] - rho * (v[0] * dv[e][0] + v[1] * dv[e][1] + v[2] * dv[e][2]));
      const Real dT = (dp * ir - p * gq[e][0] * ir * ir) / Rg;
      heat[e] = kap * dT;
    }
  }
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    F[e][0] = Q[1 + e];
#pragma unroll
    for (int a = 0; a < 3; ++a) F[e][1 + a] = Q[1 + a] * v[e] + sig[a][e];
    F[e][4] = Q[4] * v[e] + v[0] * sig[0][e] + v[1] * sig[1][e] + v[2] * sig[2][e] - heat[e];
  }
}

// Block-wide max of two values (blockDim.x a multiple of 32, <= 1024).
__device__ __forceinline__ void block_max2(double& a, double& b, double* sh /* >= 64 */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) {
    sh[w] = a;
    sh[32 + w] = b;
  }
  __syncthreads();
  a = l < nw ? sh[l] : 0.0;
  b = l < nw ? sh[32 + l] : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
}

// ----------------------------------------------------------------------------------------
// Set-up (FP64): cell mass matrices M_i = sum_k |J_ik| A_k^T M^ A_k (Sec. 4.4), written
// into the per-cell dense blocks, and w_i = M_i 1.  One block per cell; sub-tets are added
// in order (within one sub-tet the gather A_k is injective, so there is no write conflict).
__global__ void assemble_mass_kernel(DevMesh m, const RefData* __restrict__ ref) {
  const int Np = ref->Np;
  for (int64_t c = blockIdx.x; c < m.C; c += gridDim.x) {
    const int64_t n0 = m.node_ptr[c];
    const int Ni = (int)(m.node_ptr[c + 1] - n0);
    double* M = m.minv64 + m.minv_ptr[c];
    const int LD = minv_ld(Ni);
    for (int64_t e = threadIdx.x; e < m.minv_ptr[c + 1] - m.minv_ptr[c]; e += blockDim.x) M[e] = 0.0;
    __syncthreads();
    for (int64_t k = m.sub_ptr[c]; k < m.sub_ptr[c + 1]; ++k) {
      const double det = m.geo[k * 10 + 9];
      const uint16_t* Ak = m.A + k * Np;
      for (int e = threadIdx.x; e < Np * Np; e += blockDim.x) {
        const int j = e / Np, l = e % Np;
        M[(int64_t)Ak[j] * LD + Ak[l]] += det * ref->M[j][l];
      }
      __syncthreads();
    }
    for (int n = threadIdx.x; n < Ni; n += blockDim.x) {
      double s = 0.0;
      for (int l = 0; l < Ni; ++l) s += M[(int64_t)n * LD + l];
      m.wvec[n0 + n] = s;
    }
    __syncthreads();
  }
}

// In-place inverse of each cell's SPD mass matrix by tiled Gauss-Jordan elimination in FP64
// (no pivoting is needed for SPD matrices; every pivot block is a Schur complement of an
// SPD matrix).  One block of 256 threads per cell, 32 x 32 tiles staged in shared memory.
// A non-positive pivot raises flags[F_NONFINITE].
__global__ void __launch_bounds__(256) invert_spd_kernel(DevMesh m) {
  constexpr int B = 32;
  __shared__ double sD[B][B + 1];
  __shared__ double sX[B][B + 1];
  __shared__ double sY[B][B + 1];
  __shared__ double sPiv;
  const int tid = threadIdx.x;
  for (int64_t c = blockIdx.x; c < m.C; c += gridDim.x) {
    const int n = (int)(m.node_ptr[c + 1] - m.node_ptr[c]);
    const int LD = minv_ld(n);
    double* A = m.minv64 + m.minv_ptr[c];
    const int T = (n + B - 1) / B;
    auto load = [&](double (*dst)[B + 1], int ib, int jb, bool ident) {
      for (int e = tid; e < B * B; e += blockDim.x) {
        const int r = e / B, q = e % B;
        const int gr = ib * B + r, gq = jb * B + q;
        double v = (ident && r == q) ? 1.0 : 0.0;
        if (gr < n && gq < n) v = A[(int64_t)gr * LD + gq];
        dst[r][q] = v;
      }
    };
    auto store = [&](double (*src)[B + 1], int ib, int jb) {
      for (int e = tid; e < B * B; e += blockDim.x) {
        const int r = e / B, q = e % B;
        const int gr = ib * B + r, gq = jb * B + q;
        if (gr < n && gq < n) A[(int64_t)gr * LD + gq] = src[r][q];
      }
    };
    for (int kb = 0; kb < T; ++kb) {
      // 1. invert the diagonal tile (padding rows/cols act as identity)
      load(sD, kb, kb, true);
      __syncthreads();
      for (int p = 0; p < B; ++p) {
        if (tid == 0) {
          const double piv = sD[p][p];
          if (!(piv > 0.0)) atomicOr(&m.flags[F_NONFINITE], 2);
          sPiv = 1.0 / piv;
        }
        __syncthreads();
        const double ip = sPiv;
        // row p scaled; other rows eliminated (classic in-place sweep).  Every thread reads
        // the pivot row and column entries it needs before any entry is overwritten.
        double colp[4], rowp[4];
        int cnt = 0;
        for (int e = tid; e < B * B; e += blockDim.x, ++cnt) {
          colp[cnt] = sD[e / B][p];
          rowp[cnt] = sD[p][e % B];
        }
        __syncthreads();
        cnt = 0;
        for (int e = tid; e < B * B; e += blockDim.x, ++cnt) {
          const int r = e / B, q = e % B;
          const double arp = colp[cnt], apq = rowp[cnt];
          if (r == p) {
            sD[r][q] = (q == p) ? ip : apq * ip;
          } else {
            // new a_rq = a_rq - a_rp a_pq / a_pp ; new a_rp = -a_rp / a_pp
            sD[r][q] = (q == p) ? -arp * ip : sD[r][q] - arp * apq * ip;
          }
        }
        __syncthreads();
      }
      // 2. row panel: A[K, J] <- Dinv A[K, J]
      for (int jb = 0; jb < T; ++jb) {
        if (jb == kb) continue;
        load(sX, kb, jb, false);
        __syncthreads();
        for (int e = tid; e < B * B; e += blockDim.x) {
          const int r = e / B, q = e % B;
          double s = 0.0;
#pragma unroll 8
          for (int k = 0; k < B; ++k) s += sD[r][k] * sX[k][q];
          sY[r][q] = s;
        }
        __syncthreads();
        store(sY, kb, jb);
        __syncthreads();
      }
      // 3. trailing update: A[I, J] -= A[I, K] A[K, J]
      for (int ib = 0; ib < T; ++ib) {
        if (ib == kb) continue;
        load(sY, ib, kb, false);  // A[I, K] (not yet updated)
        for (int jb = 0; jb < T; ++jb) {
          if (jb == kb) continue;
          load(sX, kb, jb, false);  // updated row panel
          __syncthreads();
          for (int e = tid; e < B * B; e += blockDim.x) {
            const int r = e / B, q = e % B;
            const int gr = ib * B + r, gq = jb * B + q;
            if (gr < n && gq < n) {
              double s = 0.0;
#pragma unroll 8
              for (int k = 0; k < B; ++k) s += sY[r][k] * sX[k][q];
              A[(int64_t)gr * LD + gq] -= s;
            }
          }
          __syncthreads();
        }
        // 4. column panel: A[I, K] <- -A[I, K] Dinv
        for (int e = tid; e < B * B; e += blockDim.x) {
          const int r = e / B, q = e % B;
          const int gr = ib * B + r, gq = kb * B + q;
          if (gr < n && gq < n) {
            double s = 0.0;
#pragma unroll 8
            for (int k = 0; k < B; ++k) s += sY[r][k] * sD[k][q];
            A[(int64_t)gr * LD + gq] = -s;
          }
        }
        __syncthreads();
      }
      // 5. diagonal tile
      store(sD, kb, kb);
      __syncthreads();
    }
  }
}

// Symmetrise in FP64 and keep the FP32 copy used by the reduced-precision path.
__global__ void symmetrize_kernel(DevMesh m, int make32) {
  for (int64_t c = blockIdx.x; c < m.C; c += gridDim.x) {
    const int n = (int)(m.node_ptr[c + 1] - m.node_ptr[c]);
    const int LD = minv_ld(n);
    double* A = m.minv64 + m.minv_ptr[c];
    for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
      const int r = (int)(e / n), q = (int)(e % n);
      if (q < r) continue;
      const double v = 0.5 * (A[(int64_t)r * LD + q] + A[(int64_t)q * LD + r]);
      A[(int64_t)r * LD + q] = v;
      A[(int64_t)q * LD + r] = v;
    }
    __syncthreads();
    if (make32)  // padding (columns >= n, rows >= n) written as zeros
      for (int64_t e = threadIdx.x; e < m.minv_ptr[c + 1] - m.minv_ptr[c]; e += blockDim.x) {
        const int64_t r = e / LD, q = e % LD;
        m.minv32[m.minv_ptr[c] + e] = (r < n && q < n) ? (float)A[e] : 0.f;
      }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------------------
// Per-step kernels over a batch of meshes (one mesh is a batch of one).
//
// Start of a series of steps: clear every member's status flags (they then accumulate over
// the steps until the host reads them).
__global__ void flags_clear_kernel(const __grid_constant__ Batch bt) {
  for (int h = threadIdx.x; h < bt.nh; h += blockDim.x) {
#pragma unroll
    for (int f = 0; f < F_COUNT; ++f) bt.tab[h].flags[f] = 0;
  }
}

// Start of a step: clear every member's CFL maximum and the shared work counter of the
// persistent predictor.
__global__ void step_begin_kernel(const __grid_constant__ Batch bt) {
  for (int h = threadIdx.x; h < bt.nh; h += blockDim.x) *bt.tab[h].maxbits = 0ull;
  if (threadIdx.x == 0) *bt.work = 0;
}

// Sec. 4.5: cell means u_bar_i = w_i . u_i / |P_i|  (w_i = M_i 1), one block per cell at a time.
__global__ void cell_means_kernel(const __grid_constant__ Batch bt) {
  __shared__ double sh[5][256];
  const int64_t total = bt.cpre[bt.nh];
  for (int64_t gc = blockIdx.x; gc < total; gc += gridDim.x) {
    const int hh = batch_find(bt.cpre, bt.nh, gc);
    const DevMesh& m = bt.tab[hh];
    if (!m.limiter) continue;  // block-uniform
    const int64_t c = gc - bt.cpre[hh];
    const int64_t n0 = m.node_ptr[c], n1 = m.node_ptr[c + 1];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
      const double w = m.wvec[n];
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v] += w * m.u[n * 5 + v];
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) sh[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s)
#pragma unroll
        for (int v = 0; v < 5; ++v) sh[v][threadIdx.x] += sh[v][threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x < 5) m.means[c * 5 + threadIdx.x] = sh[threadIdx.x][0] / m.cell_vol[c];
    __syncthreads();
  }
}

// Artificial-viscosity limiter (Sec. 4.5, Eq. beta3D): beta_i from the discrete velocity
// divergence of the cell means over the faces of P_i, mu_i = mu + beta_i rho_i lambda_i h_i/(2N+1).
__global__ void limiter_kernel(const __grid_constant__ Batch bt) {
  const int64_t gc = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gc >= bt.cpre[bt.nh]) return;
  const int hh = batch_find(bt.cpre, bt.nh, gc);
  const DevMesh& m = bt.tab[hh];
  if (!m.limiter) return;  // a batch member without the limiter keeps beta = 0, mu_i = mu
  const int64_t c = gc - bt.cpre[hh];
  auto prim = [&](int64_t i, double v[3], double& rho, double& cs) {
    const double* q = m.means + i * 5;
    rho = q[0];
    for (int d = 0; d < 3; ++d) v[d] = q[1 + d] / rho;
    const double p = (m.gamma - 1.0) * (q[4] - 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
    cs = sqrt(m.gamma * p / rho);
  };
  double vi[3], rhoi, ci;
  prim(c, vi, rhoi, ci);
  double div = 0.0, cmin = ci;
  for (int64_t s = m.slot_ptr[c]; s < m.slot_ptr[c + 1]; ++s) {
    const int32_t nb = m.slot_nbr[s];
    if (nb < 0) continue;
    double vj[3], rj, cj;
    prim(nb, vj, rj, cj);
    const double* g = m.slot_geo + s * 4;
    div += g[3] * ((vj[0] - vi[0]) * g[0] + (vj[1] - vi[1]) * g[1] + (vj[2] - vi[2]) * g[2]);
    cmin = fmin(cmin, cj);
  }
  div /= m.cell_vol[c];
  const double b = fmin(1.0, fmax(0.0, -(div + m.m1 * cmin) / (m.m1 * cmin)));
  m.beta[c] = b;
  const double lam = sqrt(vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]) + ci;
  m.mu[c] = m.mu0 + b * rhoi * lam * m.cell_h[c] / (2 * m.N + 1);
  if (b > 0.0) atomicAdd(&m.flags[F_TROUBLED], 1);
}

// CFL bound (Sec. 4.6): max over nodes of lambda + 2 lambda_v (2N+1)/h_i, one warp per cell,
// folded into the member's maximum by an integer atomicMax on the bits of a non-negative
// double (order-independent, hence deterministic).
__global__ void cfl_kernel(const __grid_constant__ Batch bt) {
  const int64_t gc = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gc >= bt.cpre[bt.nh]) return;
  const int hh = batch_find(bt.cpre, bt.nh, gc);
  const DevMesh& m = bt.tab[hh];
  const int64_t c = gc - bt.cpre[hh];
  const double mu_i = m.mu[c], kap = cell_kappa(m, mu_i), h = m.cell_hv[c];
  // per cell: lambda_v = max(4 mu / 3, kappa / c_v) / rho, weighted by 2 (2N+1) / h
  const double gam = m.gamma, visc = fmax(4.0 * mu_i / 3.0, kap / m.cv) * (2.0 * (2 * m.N + 1) / h);
  double best = 0.0;
  bool bad = false;
  for (int64_t n = m.node_ptr[c] + lane; n < m.node_ptr[c + 1]; n += 32) {
    const double* q = m.u + n * 5;
    const double rho = q[0], ir = 1.0 / rho;  // one division per node
    const double m2 = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    const double p = (gam - 1.0) * (q[4] - 0.5 * m2 * ir);
    double br = sqrt(m2) * ir + sqrt(gam * p * ir) + visc * ir;
    if (!(rho > 0.0) || !(br >= 0.0) || !isfinite(br)) {  // inadmissible state: report, keep dt finite
      bad = true;
      br = 0.0;
    }
    best = fmax(best, br);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&m.flags[F_NONFINITE], 1);
  if (lane == 0) atomicMax(m.maxbits, (unsigned long long)__double_as_longlong(best));
}

// dt = CFL h_min / ((2N+1) max_bound) per member (Sec. 4.6)
__global__ void dt_finalize_kernel(const __grid_constant__ Batch bt) {
  for (int h = threadIdx.x; h < bt.nh; h += blockDim.x) {
    const DevMesh& m = bt.tab[h];
    const double mx = __longlong_as_double((long long)*m.maxbits);
    double dt = mx > 0.0 ? m.cfl * m.h_min / ((2 * m.N + 1) * mx) : 0.0;
    if (!(dt > 0.0)) atomicOr(&m.flags[F_NONFINITE], 4);
    *m.dt = dt;
  }
}

__global__ void set_dt_kernel(const __grid_constant__ Batch bt, double dt) {
  for (int h = threadIdx.x; h < bt.nh; h += blockDim.x) *bt.tab[h].dt = dt;
}

__global__ void advance_time_kernel(const __grid_constant__ Batch bt) {
  for (int h = threadIdx.x; h < bt.nh; h += blockDim.x) *bt.tab[h].tacc += *bt.tab[h].dt;
}

// ----------------------------------------------------------------------------------------
// Space-time predictor (Sec. 4.3).  Persistent: each block takes cells from a work
// counter.  Per cell, with q [N_i][Nt][5] the space-time nodal coefficients:
//   q^0 = u^  at every time node;
//   repeat:  B_{k,t}  = dt adj(J_ik) . F(q at the nodes of T_ik, time t)          (f*, g*, h*)
//            R_{k,t}  = w_t sum_d S^_d B_{k,t,d}                                     (K_d terms)
//            RHS_t    = sum_k A_k^T R_{k,t}           (fixed-order gather: deterministic)
//            Y        = M_i^-1 RHS                    (all Nt*5 columns at once)
//            q^{r+1}[n,s] = u^[n] - sum_t K1t^-1[s,t] Y[n,t]        (K_1,i^-1 = M_i^-1 (x) K1t^-1,
//                                                                      K1t^-1 psi(0) = 1)
//   until max|q^{r+1}-q^r| <= tol max(1, max|q^r|) or picard_max.
// Epilogue (Eq. TAvectors and the corrector's volume term of Sec. 4.4):
//   vol[n]     = sum_k A_k^T sum_d S^_d^T adj(J_ik) F_bar_k,  F_bar = dt sum_t w_t F(q_t)
//   slot_q     = dt sum_t w_t q_t at the face nodes
//   slot_fn    = F_bar . n at the face nodes (flux of the sub-tet owning the triangle)
// Per-block scratch in global memory (L2-resident): q, RHS, Y, B, R.
template <int N, typename Real>
__global__ void __launch_bounds__(256) predictor_kernel(DevMesh m, const RefData* __restrict__ ref, Real* scratch,
                                                        int64_t scratch_stride, int diag) {
  constexpr int NP = np_of(N), NT = N + 1, NF = nf_of(N);
  // the nodal derivative matrices stay in global memory (L1-cached) when both reference
  // matrices would not fit the static shared-memory limit (FP64 at N = 4)
  constexpr bool kDShared = 2 * 3 * NP * NP * sizeof(Real) <= 44 * 1024;
  constexpr int DS = kDShared ? NP : 1;
  __shared__ Real sS[3][NP][NP];
  __shared__ Real sD[3][DS][DS];
  __shared__ Real sK[NT][NT];
  __shared__ Real sW[NT];
  __shared__ double sred[64];
  __shared__ int64_t sCell;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int e = tid; e < 3 * NP * NP; e += nthr) {
    const int d = e / (NP * NP), r = (e / NP) % NP, q = e % NP;
    sS[d][r][q] = (Real)ref->S[d][r][q];
    if constexpr (kDShared) sD[d][r % DS][q % DS] = (Real)ref->D[d][r][q];
  }
  auto Dv = [&](int d, int j, int l) -> Real {
    if constexpr (kDShared) return sD[d][j % DS][l % DS];
    else return (Real)ref->D[d][j][l];
  };
  if (tid < NT * NT) sK[tid / NT][tid % NT] = (Real)ref->K1tinv[tid / NT][tid % NT];
  if (tid < NT) sW[tid] = (Real)ref->w[tid];
  const int Nmax = m.Nmax, Smax = m.Smax;
  Real* q = scratch + blockIdx.x * scratch_stride;
  Real* RHS = q + (int64_t)Nmax * NT * 5;
  Real* Y = RHS + (int64_t)Nmax * NT * 5;
  Real* Bf = Y + (int64_t)Nmax * NT * 5;        // [Smax][NT][3][NP][5]
  Real* Rb = Bf + (int64_t)Smax * NT * 3 * NP * 5;  // [Smax][NT][NP][5]
  const double dt = *m.dt;
  const Real gam = (Real)m.gamma, Rg = (Real)m.Rgas;
  const Real* minv = nullptr;
  __syncthreads();
  for (;;) {
    if (tid == 0) sCell = atomicAdd(m.work, 1);
    __syncthreads();
    const int64_t c = sCell;
    __syncthreads();
    if (c >= m.C) break;
    const int64_t n0 = m.node_ptr[c];
    const int Ni = (int)(m.node_ptr[c + 1] - n0);
    const int64_t k0 = m.sub_ptr[c];
    const int S = (int)(m.sub_ptr[c + 1] - k0);
    const double mu_d = m.mu[c];
    const double kap_d = cell_kappa(m, mu_d);
    const bool visc = (mu_d != 0.0) || (kap_d != 0.0);
    const Real mu = (Real)mu_d, kap = (Real)kap_d;
    if constexpr (sizeof(Real) == 8) minv = (const Real*)(m.minv64 + m.minv_ptr[c]);
    else minv = (const Real*)(m.minv32 + m.minv_ptr[c]);
    const double* uh = m.u + n0 * 5;
    for (int e = tid; e < Ni * NT * 5; e += nthr) {
      const int n = e / (NT * 5), v = e % 5;
      q[e] = (Real)uh[n * 5 + v];
    }
    __syncthreads();

    // flux pre-contraction at one (sub-tet k, time t, local node j): out[d][v] = sum_e G[d][e] F_e[v]
    auto flux_item = [&](int k, int t, int j, Real out[3][5], bool scale_dt) {
      const int64_t kg = k0 + k;
      const uint16_t* Ak = m.A + kg * NP;
      const double* g = m.geo + kg * 10;
      Real Q[5];
      const int node = Ak[j];
#pragma unroll
      for (int v = 0; v < 5; ++v) Q[v] = q[(node * NT + t) * 5 + v];
      Real gq[3][5];
      if (visc) {
        Real gx[3][5];
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int v = 0; v < 5; ++v) gx[d][v] = 0;
        for (int l = 0; l < NP; ++l) {
          const Real* ql = q + (Ak[l] * NT + t) * 5;
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const Real dd = Dv(d, j, l);
#pragma unroll
            for (int v = 0; v < 5; ++v) gx[d][v] += dd * ql[v];
          }
        }
        // grad_x = J^-T grad_xi, J^-1 = adj / det
        const Real idet = Real(1) / (Real)g[9];
#pragma unroll
        for (int e = 0; e < 3; ++e)
#pragma unroll
          for (int v = 0; v < 5; ++v)
            gq[e][v] = ((Real)g[0 * 3 + e] * gx[0][v] + (Real)g[1 * 3 + e] * gx[1][v] + (Real)g[2 * 3 + e] * gx[2][v]) * idet;
      }
      Real F[3][5];
      phys_flux<Real>(Q, gq, visc, mu, kap, gam, Rg, F);
      const Real sc = scale_dt ? (Real)dt : Real(1);
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < 5; ++v)
          out[d][v] = sc * ((Real)g[d * 3 + 0] * F[0][v] + (Real)g[d * 3 + 1] * F[1][v] + (Real)g[d * 3 + 2] * F[2][v]);
    };

    int it = 0;
    bool conv = false;
    while (!conv && it < m.picard_max) {
      ++it;
      // A: B[k][t][d][j][v]
      for (int e = tid; e < S * NT * NP; e += nthr) {
        const int k = e / (NT * NP), t = (e / NP) % NT, j = e % NP;
        Real out[3][5];
        flux_item(k, t, j, out, true);
        Real* dst = Bf + ((int64_t)(k * NT + t) * 3) * NP * 5 + j * 5;
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int v = 0; v < 5; ++v) dst[d * NP * 5 + v] = out[d][v];
      }
      __syncthreads();
      // B: R[k][t][m][v] = w_t sum_d sum_j S[d][m][j] B[k][t][d][j][v]
      for (int e = tid; e < S * NT * NP * 5; e += nthr) {
        const int k = e / (NT * NP * 5), t = (e / (NP * 5)) % NT, mm = (e / 5) % NP, v = e % 5;
        const Real* src = Bf + ((int64_t)(k * NT + t) * 3) * NP * 5 + v;
        Real acc = 0;
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int j = 0; j < NP; ++j) acc += sS[d][mm][j] * src[(d * NP + j) * 5];
        Rb[e] = sW[t] * acc;
      }
      __syncthreads();
      // C: RHS[n][t][v] = sum over incidences (k, j) of node n
      for (int e = tid; e < Ni * NT * 5; e += nthr) {
        const int n = e / (NT * 5), t = (e / 5) % NT, v = e % 5;
        Real acc = 0;
        for (int64_t p = m.inc_ptr[n0 + n]; p < m.inc_ptr[n0 + n + 1]; ++p) {
          const uint32_t w = m.inc[p];
          const int k = (int)(w >> 6), j = (int)(w & 63);
          acc += Rb[((int64_t)(k * NT + t) * NP + j) * 5 + v];
        }
        RHS[e] = acc;
      }
      __syncthreads();
      // D: Y = M_i^-1 RHS (M_i^-1 symmetric: row n read as column n, coalesced)
      for (int n = tid; n < Ni; n += nthr) {
        Real acc[NT * 5];
#pragma unroll
        for (int c2 = 0; c2 < NT * 5; ++c2) acc[c2] = 0;
        const int LD = minv_ld(Ni);
        for (int l = 0; l < Ni; ++l) {
          const Real a = minv[(int64_t)l * LD + n];
          const Real* r = RHS + l * NT * 5;
#pragma unroll
          for (int c2 = 0; c2 < NT * 5; ++c2) acc[c2] += a * r[c2];
        }
#pragma unroll
        for (int c2 = 0; c2 < NT * 5; ++c2) Y[n * NT * 5 + c2] = acc[c2];
      }
      __syncthreads();
      // E: update and residual
      double res = 0.0, qmax = 0.0;
      for (int e = tid; e < Ni * NT * 5; e += nthr) {
        const int n = e / (NT * 5), s = (e / 5) % NT, v = e % 5;
        Real acc = (Real)uh[n * 5 + v];
#pragma unroll
        for (int t = 0; t < NT; ++t) acc -= sK[s][t] * Y[(n * NT + t) * 5 + v];
        const Real old = q[e];
        res = fmax(res, (double)fabs(acc - old));
        qmax = fmax(qmax, (double)fabs(old));
        q[e] = acc;
      }
      block_max2(res, qmax, sred);
      conv = res <= m.tol * fmax(1.0, qmax);
      __syncthreads();
    }
    if (tid == 0) {
      m.iters[c] = it;
      if (!conv) atomicAdd(&m.flags[F_NONCONV], 1);
    }

    // epilogue: B_bar[k][d][j][v] = sum_t w_t dt adj F(q_t) = adj F_bar  (stored in Bf)
    for (int e = tid; e < S * NP; e += nthr) {
      const int k = e / NP, j = e % NP;
      Real accb[3][5];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < 5; ++v) accb[d][v] = 0;
      for (int t = 0; t < NT; ++t) {
        Real out[3][5];
        flux_item(k, t, j, out, true);
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int v = 0; v < 5; ++v) accb[d][v] += sW[t] * out[d][v];
      }
      Real* dst = Bf + ((int64_t)k * 3) * NP * 5 + j * 5;
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < 5; ++v) dst[d * NP * 5 + v] = accb[d][v];
    }
    __syncthreads();
    // R_bar[k][mm][v] = sum_d sum_j S[d][j][mm] B_bar[k][d][j][v]   (V_d = S^_d^T)
    for (int e = tid; e < S * NP * 5; e += nthr) {
      const int k = e / (NP * 5), mm = (e / 5) % NP, v = e % 5;
      const Real* src = Bf + ((int64_t)k * 3) * NP * 5 + v;
      Real acc = 0;
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int j = 0; j < NP; ++j) acc += sS[d][j][mm] * src[(d * NP + j) * 5];
      Rb[e] = acc;
    }
    __syncthreads();
    Real* vol = (Real*)m.vol;
    for (int e = tid; e < Ni * 5; e += nthr) {
      const int n = e / 5, v = e % 5;
      Real acc = 0;
      for (int64_t p = m.inc_ptr[n0 + n]; p < m.inc_ptr[n0 + n + 1]; ++p) {
        const uint32_t w = m.inc[p];
        acc += Rb[((int64_t)(w >> 6) * NP + (w & 63)) * 5 + v];
      }
      vol[(n0 + n) * 5 + v] = acc;
    }
    // face slots: q_bar and F_bar . n at every face node
    const int64_t s0 = m.slot_ptr[c];
    const int ns = (int)(m.slot_ptr[c + 1] - s0);
    Real* sq = (Real*)m.slot_q;
    Real* sfn = (Real*)m.slot_fn;
    for (int e = tid; e < ns * NF; e += nthr) {
      const int s = e / NF, a = e % NF;
      const int64_t sg = s0 + s;
      const int k = m.slot_sub[sg];
      const int j = m.slot_loc[sg * NF + a];
      const int node = m.slot_node[sg * NF + a];
      const double* g = m.slot_geo + sg * 4;
      Real qb[5] = {0, 0, 0, 0, 0}, fb[5] = {0, 0, 0, 0, 0};
      // F . n from the owning sub-tet: reuse flux_item with unit geometry is not possible,
      // so evaluate the physical flux directly.
      const int64_t kg = k0 + k;
      const uint16_t* Ak = m.A + kg * NP;
      const double* gk = m.geo + kg * 10;
      for (int t = 0; t < NT; ++t) {
        Real Q[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) Q[v] = q[(node * NT + t) * 5 + v];
        Real gq[3][5];
        if (visc) {
          Real gx[3][5];
#pragma unroll
          for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int v = 0; v < 5; ++v) gx[d][v] = 0;
          for (int l = 0; l < NP; ++l) {
            const Real* ql = q + (Ak[l] * NT + t) * 5;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              const Real dd = Dv(d, j, l);
#pragma unroll
              for (int v = 0; v < 5; ++v) gx[d][v] += dd * ql[v];
            }
          }
          const Real idet = Real(1) / (Real)gk[9];
#pragma unroll
          for (int e2 = 0; e2 < 3; ++e2)
#pragma unroll
            for (int v = 0; v < 5; ++v)
              gq[e2][v] = ((Real)gk[0 * 3 + e2] * gx[0][v] + (Real)gk[1 * 3 + e2] * gx[1][v] + (Real)gk[2 * 3 + e2] * gx[2][v]) * idet;
        }
        Real F[3][5];
        phys_flux<Real>(Q, gq, visc, mu, kap, gam, Rg, F);
        const Real wt = sW[t] * (Real)dt;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          qb[v] += wt * Q[v];
          fb[v] += wt * ((Real)g[0] * F[0][v] + (Real)g[1] * F[1][v] + (Real)g[2] * F[2][v]);
        }
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        sq[(sg * NF + a) * 5 + v] = qb[v];
        sfn[(sg * NF + a) * 5 + v] = fb[v];
      }
    }
    if (diag && m.qbar_diag) {
      for (int e = tid; e < Ni * 5; e += nthr) {
        const int n = e / 5, v = e % 5;
        double acc = 0.0;
        for (int t = 0; t < NT; ++t) acc += (double)sW[t] * (double)q[(n * NT + t) * 5 + v];
        m.qbar_diag[(n0 + n) * 5 + v] = dt * acc;
      }
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------------------
// Rusanov fluxes (Eq. 3.33) on the face nodes; one warp per polygonal face (all its
// sub-triangles, both sides).  The wave speeds are reduced over the face with warp
// shuffles; G is written for the own side and, negated, for the matched side.
template <int N, typename Real>
__global__ void face_kernel(const __grid_constant__ Batch bt) {
  constexpr int NF = nf_of(N);
  const int64_t ggw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (ggw >= bt.gpre[bt.nh]) return;
  const int h = batch_find(bt.gpre, bt.nh, ggw);
  const DevMesh& m = bt.tab[h];
  const int64_t gw = ggw - bt.gpre[h];
  const int64_t g0 = m.group_ptr[gw], g1 = m.group_ptr[gw + 1];
  const int nitems = (int)(g1 - g0) * NF;
  const Real* sq = (const Real*)m.slot_q;
  const Real* sfn = (const Real*)m.slot_fn;
  Real* sG = (Real*)m.slot_G;
  const double dt = *m.dt;
  const Real idt = Real(1.0 / dt);
  const Real gam = (Real)m.gamma;
  const int64_t s_first = m.group_slot[g0];
  const int32_t ci = m.slot_cell[s_first];
  const int32_t cj = m.slot_nbr[s_first];
  const double mu_i = m.mu[ci], kap_i = cell_kappa(m, mu_i);
  const double mu_j = cj >= 0 ? m.mu[cj] : mu_i, kap_j = cell_kappa(m, mu_j);
  const double h_i = m.cell_h[ci], h_j = cj >= 0 ? m.cell_h[cj] : h_i;
  // |lambda_v| = max(4 mu / 3, kappa / c_v) / rho: the coefficient once per side, then one
  // reciprocal per face node (1 / rho = dt / q_bar_rho)
  const Real cvis_i = (Real)fmax(4.0 * mu_i / 3.0, kap_i / m.cv), cvis_j = (Real)fmax(4.0 * mu_j / 3.0, kap_j / m.cv);
  const Real rdt = (Real)dt;
  Real smax = 0, vmax = 0;
  for (int e = lane; e < nitems; e += 32) {
    const int64_t s = m.group_slot[g0 + e / NF];
    const int a = e % NF;
    const int64_t ps = m.slot_partner[s];
    const double* g = m.slot_geo + s * 4;
    for (int side = 0; side < 2; ++side) {
      const int64_t ss = side == 0 ? s : ps;
      if (ss < 0) continue;
      const Real* Q = sq + (ss * NF + a) * 5;
      const Real rho = Q[0] * idt;
      const Real ir = Real(1) / Q[0];
      const Real v0 = Q[1] * ir, v1 = Q[2] * ir, v2 = Q[3] * ir;  // q_bar / dt ratios
      const Real p = (gam - 1) * (Q[4] * idt - Real(0.5) * rho * (v0 * v0 + v1 * v1 + v2 * v2));
      const Real vn = fabs(v0 * (Real)g[0] + v1 * (Real)g[1] + v2 * (Real)g[2]);
      const Real irho = ir * rdt;  // 1 / rho
      smax = fmax(smax, vn + sqrt(gam * p * irho));
      vmax = fmax(vmax, (side == 0 ? cvis_i : cvis_j) * irho);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  }
  const Real eps = (Real)((2 * N + 1) / ((h_i + h_j) * sqrt(3.14159265358979323846 / 2.0)));
  const Real diss = Real(0.5) * (smax + Real(2) * eps * vmax);
  for (int e = lane; e < nitems * 5; e += 32) {
    const int item = e / 5, v = e % 5;
    const int64_t s = m.group_slot[g0 + item / NF];
    const int a = item % NF;
    const int64_t ps = m.slot_partner[s];
    const int64_t io = (s * NF + a) * 5 + v;
    if (ps < 0) {  // transmissive boundary: q+ = q-, F+ = F-
      sG[io] = sfn[io];
      continue;
    }
    const int64_t ip = (ps * NF + a) * 5 + v;
    // the matched side stores F_bar . (its own normal) = -F_bar+ . n
    const Real G = Real(0.5) * (sfn[io] - sfn[ip]) - diss * (sq[ip] - sq[io]);
    sG[io] = G;
    sG[ip] = -G;
  }
}

// ----------------------------------------------------------------------------------------
// Corrector (Sec. 4.4): r = vol - sum_slots 2 area Z^ G (fixed-order gather), then
// u^{n+1} = u^n + M_i^-1 r.  FP64 path: everything in FP64.  FP32 path: r and the apply in
// FP32, then an FP64 correction adds a constant to du so that w_i . du equals sum(r)
// exactly in FP64 (the conserved totals of the cell: 1^T M_i du = 1^T r).
template <int N, typename Real>
__global__ void __launch_bounds__(256) corrector_kernel(DevMesh m, const RefData* __restrict__ ref) {
  constexpr int NF = nf_of(N);
  extern __shared__ double smem_dbl[];
  Real* r = (Real*)smem_dbl;                       // [Nmax][5]
  double* du = smem_dbl + ((m.Nmax * 5 * sizeof(Real) + 7) / 8);  // [Nmax][5], FP32 path only
  __shared__ Real sZ[NF][NF];
  __shared__ double sfix[2][5][sizeof(Real) == 4 ? 256 : 1];
  const int tid = threadIdx.x;
  for (int e = tid; e < NF * NF; e += blockDim.x) sZ[e / NF][e % NF] = (Real)ref->Z[e / NF][e % NF];
  __syncthreads();
  const Real* vol = (const Real*)m.vol;
  const Real* sG = (const Real*)m.slot_G;
  for (int64_t c = blockIdx.x; c < m.C; c += gridDim.x) {
    const int64_t n0 = m.node_ptr[c];
    const int Ni = (int)(m.node_ptr[c + 1] - n0);
    const int64_t s0 = m.slot_ptr[c];
    double tot[5] = {0, 0, 0, 0, 0};
    for (int e = tid; e < Ni * 5; e += blockDim.x) {
      const int n = e / 5, v = e % 5;
      Real acc = vol[(n0 + n) * 5 + v];
      for (int64_t p = m.finc_ptr[n0 + n]; p < m.finc_ptr[n0 + n + 1]; ++p) {
        const uint32_t w = m.finc[p];
        const int64_t s = s0 + (w >> 4);
        const int a = w & 15;
        const Real twoA = Real(2) * (Real)m.slot_geo[s * 4 + 3];
        Real f = 0;
#pragma unroll
        for (int b = 0; b < NF; ++b) f += sZ[a][b] * sG[(s * NF + b) * 5 + v];
        acc -= twoA * f;
      }
      r[e] = acc;
    }
    if constexpr (sizeof(Real) == 4) {
      // exact cell total of the update in FP64: sum_m vol[m] = int grad(sum phi_m) . F = 0,
      // so 1^T r = -sum_slots 2 area sum_b (sum_a Z^[a][b]) G[b]; matched slots cancel.
      const int ns = (int)(m.slot_ptr[c + 1] - s0);
      for (int e = tid; e < ns * NF * 5; e += blockDim.x) {
        const int sl = e / (NF * 5), b = (e / 5) % NF, v = e % 5;
        const int64_t s = s0 + sl;
        double zs = 0.0;
#pragma unroll
        for (int a = 0; a < NF; ++a) zs += ref->Z[a][b];
        tot[v] -= 2.0 * m.slot_geo[s * 4 + 3] * zs * (double)sG[(s * NF + b) * 5 + v];
      }
    }
    __syncthreads();
    const Real* minv;
    if constexpr (sizeof(Real) == 8) minv = (const Real*)(m.minv64 + m.minv_ptr[c]);
    else minv = (const Real*)(m.minv32 + m.minv_ptr[c]);
    double wdu[5] = {0, 0, 0, 0, 0};
    for (int n = tid; n < Ni; n += blockDim.x) {
      Real acc[5] = {0, 0, 0, 0, 0};
      const int LD = minv_ld(Ni);
      for (int l = 0; l < Ni; ++l) {
        const Real a = minv[(int64_t)l * LD + n];
#pragma unroll
        for (int v = 0; v < 5; ++v) acc[v] += a * r[l * 5 + v];
      }
      if constexpr (sizeof(Real) == 8) {
        bool bad = false;
        double* un = m.u + (n0 + n) * 5;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          un[v] += (double)acc[v];
          bad |= !isfinite(un[v]);
        }
        const double rho = un[0];
        const double p = (m.gamma - 1.0) * (un[4] - 0.5 * (un[1] * un[1] + un[2] * un[2] + un[3] * un[3]) / rho);
        if (bad || !(rho > 0.0) || !(p > 0.0)) atomicOr(&m.flags[F_NONFINITE], 8);
      } else {
        const double w = m.wvec[n0 + n];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          wdu[v] += w * (double)acc[v];
          du[n * 5 + v] = (double)acc[v];
        }
      }
    }
    if constexpr (sizeof(Real) == 4) {
      // FP64 totals (target and w . du), block-reduced in a fixed order
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        sfix[0][v][tid] = tot[v];
        sfix[1][v][tid] = wdu[v];
      }
      __syncthreads();
      for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (tid < st)
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            sfix[0][v][tid] += sfix[0][v][tid + st];
            sfix[1][v][tid] += sfix[1][v][tid + st];
          }
        __syncthreads();
      }
      double corr[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) corr[v] = (sfix[0][v][0] - sfix[1][v][0]) / m.cell_vol[c];
      for (int n = tid; n < Ni; n += blockDim.x) {
        double* un = m.u + (n0 + n) * 5;
        bool bad = false;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          un[v] += du[n * 5 + v] + corr[v];
          bad |= !isfinite(un[v]);
        }
        const double rho = un[0];
        const double p = (m.gamma - 1.0) * (un[4] - 0.5 * (un[1] * un[1] + un[2] * un[2] + un[3] * un[3]) / rho);
        if (bad || !(rho > 0.0) || !(p > 0.0)) atomicOr(&m.flags[F_NONFINITE], 8);
      }
    }
    __syncthreads();
  }
}

// FP64 conserved totals sum_i w_i . u_i: per-block partials over a fixed cell partition,
// then a single block sums the partials in order (bitwise reproducible).
__global__ void totals_partial_kernel(DevMesh m, double* partial) {
  __shared__ double sh[5][256];
  double acc[5] = {0, 0, 0, 0, 0};
  const int64_t per = (m.n_nodes + gridDim.x - 1) / gridDim.x;
  const int64_t a = blockIdx.x * per, b = min(m.n_nodes, a + per);
  for (int64_t n = a + threadIdx.x; n < b; n += blockDim.x) {
    const double w = m.wvec[n];
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] += w * m.u[n * 5 + v];
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) sh[v][threadIdx.x] = acc[v];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int v = 0; v < 5; ++v) sh[v][threadIdx.x] += sh[v][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 5) partial[blockIdx.x * 5 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void totals_final_kernel(const double* partial, int nblk, double* out) {
  if (threadIdx.x < 5) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[b * 5 + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

}  // namespace afe
