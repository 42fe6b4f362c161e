// FP32 space-time predictor for sm_103a (Sec. 4.3, Eqs. ADER-localCauchy, ader4, TAvectors).
//
// One block of 512 threads per cell (persistent: blocks take cells from a work counter).
// The cell's working set stays in shared memory for the whole fixed-point iteration:
//   sq   [N_i][Nt*5]  space-time nodal coefficients q (node-major)
//   srhs [N_i][Nt*5]  right-hand side sum_k A_k^T R_k (zeroed and gathered every iteration)
//   sR   [CH][Nt][Np][5]  per-chunk sub-tet results R_{k,t} (deterministic gather buffer)
//   sB   [warps][3][Np][5]  per-warp flux pre-contraction of one (sub-tet, time)
//   sM   [NSTAGE][rows][LD] pipelined stages of M_i^-1
// Per iteration:
//   1. for chunks of CH sub-tets: every warp takes (sub-tet k, time t) pairs; lanes j < Np
//      evaluate the flux at node j and pre-contract it with dt adj(J_k) (f*, g*, h*); lanes
//      m < Np then form R[m][v] = w_t sum_d sum_j S^_d[m][j] B_d[j][v]; after the chunk each
//      thread adds, for the nodes it owns, the chunk's incidences in (k, j) order (fixed
//      order: the sum is bitwise reproducible and has no atomics);
//   2. Y = M_i^-1 RHS with M_i^-1 streamed through shared memory in stages of `rows` rows by
//      cp.async.bulk (TMA bulk copies, completion on an mbarrier), each thread owning up to two
//      rows of Y (M_i^-1 is symmetric: row l of the stage serves column l);
//      q^{r+1}[n,s] = u^[n] - sum_t K1t^-1[s,t] Y[n,t] and the residual, in registers.
// Epilogue: vol = sum_k A_k^T sum_d S^_d^T adj(J_k) F_bar_k, and q_bar, F_bar . n on the face
// slots, as the FP64 kernel.  Every mbarrier wait is bounded; a wait that runs out sets
// flags[F_TIMEOUT], drains the copies in flight (bounded again) and the block returns.
#pragma once

#include "kernels.cuh"

namespace afe {

constexpr int kF32Threads = 512;
constexpr int kF32Warps = kF32Threads / 32;
constexpr int kF32Chunk = 8;     // sub-tets per gather chunk
constexpr int kF32Stages = 3;    // M_i^-1 pipeline depth

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase: false if it did not complete within the limit.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (int i = 0; i < (1 << 20); ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Bulk (TMA) copy of `bytes` (multiple of 16, both addresses 16-byte aligned) global -> shared,
// completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Bytes of dynamic shared memory the FP32 predictor needs for a mesh.
inline size_t predictor_f32_smem(int N, int Nmax, int rows) {
  const int Np = (N + 1) * (N + 2) * (N + 3) / 6, NC = (N + 1) * 5;
  auto up = [](size_t x) { return (x + 127) / 128 * 128; };
  size_t b = 0;
  b += up((size_t)Nmax * NC * 4);                                 // sq
  b += up((size_t)Nmax * NC * 4);                                 // srhs
  b += up((size_t)kF32Stages * rows * minv_ld(Nmax) * 4);         // sM
  b += up((size_t)kF32Chunk * (N + 1) * Np * 5 * 4);              // sR
  b += up((size_t)kF32Warps * 3 * Np * 5 * 4);                    // sB
  return b;
}

// flux pre-contraction at one (sub-tet, time, local node j): out[d][v] = sum_e G[d][e] F_e[v]
// with G = scale * adj(J); gradients (viscous only) from the sub-tet's own polynomial
template <int N>
__device__ __forceinline__ void f32_flux_contract(const float* __restrict__ sq, const uint16_t* __restrict__ Ak,
                                                  const float* __restrict__ g, int j, int t, bool visc, float mu,
                                                  float kap, float gam, float Rg, float scale,
                                                  const float (*sD)[np_of(N)][np_of(N)], float out[3][5]) {
  constexpr int NP = np_of(N), NC = (N + 1) * 5;
  float Q[5];
  const float* qn = sq + Ak[j] * NC + t * 5;
#pragma unroll
  for (int v = 0; v < 5; ++v) Q[v] = qn[v];
  float gq[3][5];
  if (visc) {
    float gx[3][5];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int v = 0; v < 5; ++v) gx[d][v] = 0.f;
    for (int l = 0; l < NP; ++l) {
      const float* ql = sq + Ak[l] * NC + t * 5;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float dd = sD[d][j][l];
#pragma unroll
        for (int v = 0; v < 5; ++v) gx[d][v] += dd * ql[v];
      }
    }
    const float idet = 1.f / g[9];
#pragma unroll
    for (int e = 0; e < 3; ++e)
#pragma unroll
      for (int v = 0; v < 5; ++v) gq[e][v] = (g[0 * 3 + e] * gx[0][v] + g[1 * 3 + e] * gx[1][v] + g[2 * 3 + e] * gx[2][v]) * idet;
  }
  float F[3][5];
  phys_flux<float>(Q, gq, visc, mu, kap, gam, Rg, F);
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int v = 0; v < 5; ++v) out[d][v] = scale * (g[d * 3 + 0] * F[0][v] + g[d * 3 + 1] * F[1][v] + g[d * 3 + 2] * F[2][v]);
}

template <int N>
__global__ void __launch_bounds__(kF32Threads, 1) predictor_f32_kernel(DevMesh m, const RefData* __restrict__ ref,
                                                                        int rows, int diag) {
  constexpr int NP = np_of(N), NT = N + 1, NF = nf_of(N), NC = NT * 5;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ float sSt[3][NP][NP];   // sSt[d][j][m] = S^_d[m][j]  (iteration contraction, lane = m)
  __shared__ float sSo[3][NP][NP];   // sSo[d][j][m] = S^_d[j][m]  (volume term, lane = m)
  __shared__ float sD[3][NP][NP];    // nodal derivative matrices (viscous fluxes)
  __shared__ float sK[NT][NT];
  __shared__ float sW[NT];
  __shared__ __align__(8) uint64_t sbar[kF32Stages];
  __shared__ float sred[2][kF32Warps];
  __shared__ int64_t sCell;
  __shared__ int sAbort;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Nmax = m.Nmax;
  const int LDmax = minv_ld(Nmax);
  auto up = [](size_t x) { return (x + 127) / 128 * 128; };
  unsigned char* p = smem_raw;
  float* sq = (float*)p;
  p += up((size_t)Nmax * NC * 4);
  float* srhs = (float*)p;
  p += up((size_t)Nmax * NC * 4);
  float* sM = (float*)p;
  p += up((size_t)kF32Stages * rows * LDmax * 4);
  float* sR = (float*)p;
  p += up((size_t)kF32Chunk * NT * NP * 5 * 4);
  float* sB = (float*)p + warp * 3 * NP * 5;

  for (int e = tid; e < 3 * NP * NP; e += kF32Threads) {
    const int d = e / (NP * NP), r = (e / NP) % NP, c = e % NP;
    sSt[d][c][r] = (float)ref->S[d][r][c];
    sSo[d][r][c] = (float)ref->S[d][r][c];
    sD[d][r][c] = (float)ref->D[d][r][c];
  }
  if (tid < NT * NT) sK[tid / NT][tid % NT] = (float)ref->K1tinv[tid / NT][tid % NT];
  if (tid < NT) sW[tid] = (float)ref->w[tid];
  if (tid == 0) {
    for (int s = 0; s < kF32Stages; ++s) mbar_init(&sbar[s], 1);
    sAbort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t phase = 0;  // bit s: parity of the next completion of stage s (same in every thread)
  const float dt = (float)*m.dt;
  const float gam = (float)m.gamma, Rg = (float)m.Rgas;
  const float tol = (float)m.tol;

  for (;;) {
    if (tid == 0) sCell = atomicAdd(m.work, 1);
    __syncthreads();
    const int64_t c = sCell;
    if (c >= m.C) break;
    const int64_t n0 = m.node_ptr[c];
    const int Ni = (int)(m.node_ptr[c + 1] - n0);
    const int LD = minv_ld(Ni);
    const int64_t kbase = m.sub_ptr[c];
    const int S = (int)(m.sub_ptr[c + 1] - kbase);
    const float mu = (float)m.mu[c];
    const float kap = (float)cell_kappa(m, m.mu[c]);
    const bool visc = (mu != 0.f) || (kap != 0.f);
    const float* minv = m.minv32 + m.minv_ptr[c];
    const int nblk = (Ni + rows - 1) / rows;

    // rows owned by this thread (n = tid, tid + 512) and their u^ in registers
    float uh[2][5];
    int cur[2], cend[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int n = tid + r * kF32Threads;
      cur[r] = cend[r] = 0;
      if (n < Ni) {
        const double* un = m.u + (n0 + n) * 5;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          uh[r][v] = (float)un[v];
#pragma unroll
          for (int t = 0; t < NT; ++t) sq[n * NC + t * 5 + v] = uh[r][v];
        }
      } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) uh[r][v] = 0.f;
      }
    }
    __syncthreads();

    int it = 0;
    bool conv = false;
    while (!conv && it < m.picard_max) {
      ++it;
      // prefetch the first stages of M_i^-1 while the right-hand side is formed
      if (tid == 0) {
        for (int b = 0; b < kF32Stages && b < nblk; ++b) {
          const int rb = min(rows, Ni - b * rows);
          mbar_expect_tx(&sbar[b], (uint32_t)(rb * LD * 4));
          bulk_g2s(sM + (size_t)b * rows * LDmax, minv + (size_t)b * rows * LD, (uint32_t)(rb * LD * 4), &sbar[b]);
        }
      }
      // ---- 1. right-hand side
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int n = tid + r * kF32Threads;
        if (n < Ni) {
#pragma unroll
          for (int e = 0; e < NC; ++e) srhs[n * NC + e] = 0.f;
          cur[r] = (int)(m.inc_ptr[n0 + n] - m.inc_ptr[n0]);
          cend[r] = (int)(m.inc_ptr[n0 + n + 1] - m.inc_ptr[n0]);
        }
      }
      const uint32_t* inc = m.inc + m.inc_ptr[n0];
      for (int kc = 0; kc < S; kc += kF32Chunk) {
        const int nk = min(kF32Chunk, S - kc);
        for (int pr = warp; pr < nk * NT; pr += kF32Warps) {
          const int kl = pr / NT, t = pr % NT;
          const int64_t kg = kbase + kc + kl;
          const uint16_t* Ak = m.A + kg * NP;
          const float* g = m.geo32 + kg * 12;
          if (lane < NP) {
            float out[3][5];
            f32_flux_contract<N>(sq, Ak, g, lane, t, visc, mu, kap, gam, Rg, dt, sD, out);
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
              for (int v = 0; v < 5; ++v) sB[(d * NP + lane) * 5 + v] = out[d][v];
          }
          __syncwarp();
          if (lane < NP) {
            float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll 4
              for (int j = 0; j < NP; ++j) {
                const float s = sSt[d][j][lane];
                const float* b = sB + (d * NP + j) * 5;
#pragma unroll
                for (int v = 0; v < 5; ++v) acc[v] += s * b[v];
              }
            float* dst = sR + ((kl * NT + t) * NP + lane) * 5;
#pragma unroll
            for (int v = 0; v < 5; ++v) dst[v] = sW[t] * acc[v];
          }
          __syncwarp();
        }
        __syncthreads();
        // gather this chunk's incidences, in (k, j) order, into the owned rows
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int n = tid + r * kF32Threads;
          if (n >= Ni) continue;
          while (cur[r] < cend[r]) {
            const uint32_t w = inc[cur[r]];
            const int k = (int)(w >> 5) - kc;
            if (k >= nk) break;
            const int j = (int)(w & 31);
#pragma unroll
            for (int t = 0; t < NT; ++t)
#pragma unroll
              for (int v = 0; v < 5; ++v) srhs[n * NC + t * 5 + v] += sR[((k * NT + t) * NP + j) * 5 + v];
            ++cur[r];
          }
        }
        __syncthreads();
      }
      // ---- 2. Y = M_i^-1 RHS (streamed), update and residual
      float acc[2][NC];
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int e = 0; e < NC; ++e) acc[r][e] = 0.f;
      const int na = tid, nb = tid + kF32Threads;
      for (int b = 0; b < nblk; ++b) {
        const int s = b % kF32Stages;
        if (!mbar_wait_bounded(&sbar[s], (phase >> s) & 1u)) {
          atomicOr(&m.flags[F_TIMEOUT], 1);
          sAbort = 1;
        }
        phase ^= (1u << s);
        const float* stage = sM + (size_t)s * rows * LDmax;
        const int l0 = b * rows, rb = min(rows, Ni - l0);
        for (int lr = 0; lr < rb; ++lr) {
          const float* rhs = srhs + (l0 + lr) * NC;
          const float a0 = na < Ni ? stage[lr * LD + na] : 0.f;
          const float a1 = nb < Ni ? stage[lr * LD + nb] : 0.f;
#pragma unroll
          for (int e = 0; e < NC; ++e) {
            const float x = rhs[e];
            acc[0][e] += a0 * x;
            acc[1][e] += a1 * x;
          }
        }
        __syncthreads();  // every thread is done with stage s
        if (sAbort) break;
        if (tid == 0 && b + kF32Stages < nblk) {
          const int bn = b + kF32Stages;
          const int rbn = min(rows, Ni - bn * rows);
          mbar_expect_tx(&sbar[s], (uint32_t)(rbn * LD * 4));
          bulk_g2s(sM + (size_t)s * rows * LDmax, minv + (size_t)bn * rows * LD, (uint32_t)(rbn * LD * 4), &sbar[s]);
        }
      }
      if (sAbort) break;
      float res = 0.f, qmax = 0.f;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int n = tid + r * kF32Threads;
        if (n >= Ni) continue;
#pragma unroll
        for (int s2 = 0; s2 < NT; ++s2)
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            float x = uh[r][v];
#pragma unroll
            for (int t = 0; t < NT; ++t) x -= sK[s2][t] * acc[r][t * 5 + v];
            const float old = sq[n * NC + s2 * 5 + v];
            res = fmaxf(res, fabsf(x - old));
            qmax = fmaxf(qmax, fabsf(old));
            sq[n * NC + s2 * 5 + v] = x;
          }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        res = fmaxf(res, __shfl_xor_sync(0xffffffffu, res, o));
        qmax = fmaxf(qmax, __shfl_xor_sync(0xffffffffu, qmax, o));
      }
      if (lane == 0) {
        sred[0][warp] = res;
        sred[1][warp] = qmax;
      }
      __syncthreads();
      res = 0.f;
      qmax = 0.f;
#pragma unroll
      for (int w = 0; w < kF32Warps; ++w) {
        res = fmaxf(res, sred[0][w]);
        qmax = fmaxf(qmax, sred[1][w]);
      }
      conv = res <= tol * fmaxf(1.f, qmax);
      __syncthreads();
    }
    if (sAbort) {
      // drain: wait (bounded) for every stage still in flight, then leave
      if (tid == 0)
        for (int s = 0; s < kF32Stages; ++s) (void)mbar_wait_bounded(&sbar[s], (phase >> s) & 1u);
      __syncthreads();
      return;
    }
    if (tid == 0) {
      m.iters[c] = it;
      if (!conv) atomicAdd(&m.flags[F_NONCONV], 1);
    }

    // ---- epilogue: volume term (gathered into srhs[n][0..4])
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int n = tid + r * kF32Threads;
      if (n < Ni) {
#pragma unroll
        for (int v = 0; v < 5; ++v) srhs[n * NC + v] = 0.f;
        cur[r] = (int)(m.inc_ptr[n0 + n] - m.inc_ptr[n0]);
        cend[r] = (int)(m.inc_ptr[n0 + n + 1] - m.inc_ptr[n0]);
      }
    }
    const uint32_t* inc = m.inc + m.inc_ptr[n0];
    const int CHV = kF32Chunk * NT;  // sub-tets per volume chunk (sR holds CH*NT slices)
    for (int kc = 0; kc < S; kc += CHV) {
      const int nk = min(CHV, S - kc);
      for (int kl = warp; kl < nk; kl += kF32Warps) {
        const int64_t kg = kbase + kc + kl;
        const uint16_t* Ak = m.A + kg * NP;
        const float* g = m.geo32 + kg * 12;
        if (lane < NP) {
          float accb[3][5];
#pragma unroll
          for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int v = 0; v < 5; ++v) accb[d][v] = 0.f;
          for (int t = 0; t < NT; ++t) {
            float out[3][5];
            f32_flux_contract<N>(sq, Ak, g, lane, t, visc, mu, kap, gam, Rg, dt * sW[t], sD, out);
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
              for (int v = 0; v < 5; ++v) accb[d][v] += out[d][v];
          }
#pragma unroll
          for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int v = 0; v < 5; ++v) sB[(d * NP + lane) * 5 + v] = accb[d][v];
        }
        __syncwarp();
        if (lane < NP) {
          float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int d = 0; d < 3; ++d)
#pragma unroll 4
            for (int j = 0; j < NP; ++j) {
              const float s = sSo[d][j][lane];
              const float* b = sB + (d * NP + j) * 5;
#pragma unroll
              for (int v = 0; v < 5; ++v) acc[v] += s * b[v];
            }
          float* dst = sR + (kl * NP + lane) * 5;
#pragma unroll
          for (int v = 0; v < 5; ++v) dst[v] = acc[v];
        }
        __syncwarp();
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int n = tid + r * kF32Threads;
        if (n >= Ni) continue;
        while (cur[r] < cend[r]) {
          const uint32_t w = inc[cur[r]];
          const int k = (int)(w >> 5) - kc;
          if (k >= nk) break;
          const int j = (int)(w & 31);
#pragma unroll
          for (int v = 0; v < 5; ++v) srhs[n * NC + v] += sR[(k * NP + j) * 5 + v];
          ++cur[r];
        }
      }
      __syncthreads();
    }
    float* vol = (float*)m.vol;
    for (int e = tid; e < Ni * 5; e += kF32Threads) vol[(n0 + e / 5) * 5 + e % 5] = srhs[(e / 5) * NC + e % 5];

    // face slots: q_bar and F_bar . n at every face node (flux of the owning sub-tet)
    const int64_t s0 = m.slot_ptr[c];
    const int ns = (int)(m.slot_ptr[c + 1] - s0);
    float* sqo = (float*)m.slot_q;
    float* sfn = (float*)m.slot_fn;
    for (int e = tid; e < ns * NF; e += kF32Threads) {
      const int sl = e / NF, a = e % NF;
      const int64_t sg = s0 + sl;
      const int64_t kg = kbase + m.slot_sub[sg];
      const int j = m.slot_loc[sg * NF + a];
      const uint16_t* Ak = m.A + kg * NP;
      const float* g = m.geo32 + kg * 12;
      const double* gs = m.slot_geo + sg * 4;
      const float nx = (float)gs[0], ny = (float)gs[1], nz = (float)gs[2];
      float qb[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, fb[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      for (int t = 0; t < NT; ++t) {
        // physical flux (unit geometry): contract with the identity instead of adj(J)
        float Q[5];
        const float* qn = sq + Ak[j] * NC + t * 5;
#pragma unroll
        for (int v = 0; v < 5; ++v) Q[v] = qn[v];
        float gq[3][5];
        if (visc) {
          float gx[3][5];
#pragma unroll
          for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int v = 0; v < 5; ++v) gx[d][v] = 0.f;
          for (int l = 0; l < NP; ++l) {
            const float* ql = sq + Ak[l] * NC + t * 5;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              const float dd = sD[d][j][l];
#pragma unroll
              for (int v = 0; v < 5; ++v) gx[d][v] += dd * ql[v];
            }
          }
          const float idet = 1.f / g[9];
#pragma unroll
          for (int e2 = 0; e2 < 3; ++e2)
#pragma unroll
            for (int v = 0; v < 5; ++v)
              gq[e2][v] = (g[0 * 3 + e2] * gx[0][v] + g[1 * 3 + e2] * gx[1][v] + g[2 * 3 + e2] * gx[2][v]) * idet;
        }
        float F[3][5];
        phys_flux<float>(Q, gq, visc, mu, kap, gam, Rg, F);
        const float wt = sW[t] * dt;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          qb[v] += wt * Q[v];
          fb[v] += wt * (nx * F[0][v] + ny * F[1][v] + nz * F[2][v]);
        }
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        sqo[(sg * NF + a) * 5 + v] = qb[v];
        sfn[(sg * NF + a) * 5 + v] = fb[v];
      }
    }
    if (diag && m.qbar_diag)
      for (int e = tid; e < Ni * 5; e += kF32Threads) {
        const int n = e / 5, v = e % 5;
        float acc = 0.f;
        for (int t = 0; t < NT; ++t) acc += sW[t] * sq[n * NC + t * 5 + v];
        m.qbar_diag[(n0 + n) * 5 + v] = (double)dt * (double)acc;
      }
    __syncthreads();
  }
}

// FP32 copy of the sub-tet geometry: [T][12] = adj(J) row-major (9), det J, padding.
__global__ void geo32_kernel(DevMesh m, int64_t T) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= T) return;
#pragma unroll
  for (int i = 0; i < 10; ++i) m.geo32[k * 12 + i] = (float)m.geo[k * 10 + i];
  m.geo32[k * 12 + 10] = 0.f;
  m.geo32[k * 12 + 11] = 0.f;
}

}  // namespace afe
