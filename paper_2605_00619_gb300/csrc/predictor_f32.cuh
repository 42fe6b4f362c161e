// FP32 space-time predictor for sm_103a (Sec. 4.3, Eqs. ADER-localCauchy, ader4, TAvectors).
//
// One block of 512 threads per cell (persistent: blocks take cells from a work counter).
// The cell's working set stays in shared memory for the whole fixed-point iteration:
//   srec [S][REC]       the cell's packed sub-tet records
//   sq   [N_i][Nt*5|1]  space-time nodal coefficients q (node-major, odd row stride)
//   srhs [N_i][24]      right-hand side sum_k A_k^T R_k, then Y, [5][NTP] per row (time
//                       slices padded to a vector width NTP, columns padded to 24)
// followed by one region used by the two phases in turn:
//   phase 1: sR  [CH][Nt][Np][5]     per-chunk sub-tet results R_{k,t} (gather buffer)
//            sBt [CH Nt 5][KKS]      pre-contracted fluxes of the chunk, one column (k, t, v)
//                                    of the 3 Np values (d, j) per row
//   phase 2: ring [NSTAGE][rows][LD]  pipelined stages of M_i^-1 (as many as fit), at the top
//                                     of the region: its first slot above the phase-1 buffers
//                                     when there is room, filled while phase 1 runs
// Per iteration:
//   1. for chunks of CH sub-tets (twice as many when the cell leaves room): every thread
//      takes (sub-tet k, node j, time t) items, evaluates the flux and pre-contracts it with
//      adj(J_k) (f*, g*, h*) into B^T; then every thread takes one column (k, t, v) and forms
//      R[t][m][v] = w_t dt sum_d sum_j S^_d[m][j] B_d[j][v][t] for all Np rows m in registers,
//      with the universal S^ entries as instruction immediates (gen_sref.cpp writes the
//      multiply-adds out at build time, zero entries skipped); after the chunk each thread
//      adds, in registers for the nodes it owns, the chunk's incidences in (k, j) order (fixed
//      order: the sum is bitwise reproducible and has no atomics);
//      The first iteration starts from q^0 = u^, the same at every time node: one flux per
//      (k, j) and one column per (k, v) serve all time slices (R_{k,t} = w_t R_k) and the apply
//      takes the 5 time-independent columns (Y_t = w_t Y_0);
//   2. Y = M_i^-1 RHS with M_i^-1 streamed through shared memory in stages of `rows` rows by
//      cp.async.bulk (TMA bulk copies, completion on an mbarrier), on the tensor cores:
//      mma.sync m16n8k8 TF32 with each FP32 operand split into a TF32 head and tail (bit
//      truncation) and the three leading products accumulated in FP32 (3xTF32: FP32-level
//      accuracy); warp w
//      owns the 16-row tiles w, w+15, w+30 of Y (M_i^-1 is symmetric: row l of the stage
//      serves column l);
//      q^{r+1}[n,s] = u^[n] - sum_t K1t^-1[s,t] Y[n,t] and the residual, in registers.
// Epilogue: vol = sum_k A_k^T sum_d S^_d^T adj(J_k) F_bar_k (the same column-per-thread
// contraction with S^ transposed), and q_bar, F_bar . n on the face slots, as the FP64 kernel.
// Every mbarrier wait is bounded; a wait that runs out sets flags[F_TIMEOUT], drains the
// copies in flight (bounded again) and the block returns.
#pragma once

#include <algorithm>
#include <type_traits>

#include "kernels.cuh"
#include "sref_gen.cuh"  // generated at build time by gen_sref.cpp

namespace afe {

constexpr int kF32Threads = 512;
constexpr int kF32Warps = kF32Threads / 32;
constexpr int kF32Rows = 32;     // rows of M_i^-1 per pipeline stage
constexpr int kF32MaxStages = 8;
constexpr int kF32Consumers = kF32Warps - 1;  // warps that apply M_i^-1 (the last one loads it)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One test of an mbarrier phase.  The waiting thread may be suspended until the phase
// completes or a time limit passes: the hardware's own, or about kWaitHintNs nanoseconds when
// that is set (a hint of 32 or 1000 ns measured no different from none on these kernels).
#ifndef AFE_WAIT_HINT_NS
#define AFE_WAIT_HINT_NS 0
#endif
constexpr uint32_t kWaitHintNs = AFE_WAIT_HINT_NS;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  if constexpr (kWaitHintNs == 0) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kWaitHintNs)
        : "memory");
  }
  return ok != 0;
}

// Bounded wait on an mbarrier phase: false if it did not complete within `polls` polls.
constexpr int kWaitPolls = 1 << 20;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int polls = kWaitPolls) {
  for (int i = 0; i < polls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// x = hi + lo + e with hi, lo TF32 (the low 13 bits cleared: truncation) and
// |e| <= 2^-21 |x|; hi + lo and the products of 3xTF32 carry FP32-level accuracy.
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = __float_as_uint(x) & 0xffffe000u;
  lo = __float_as_uint(x - __uint_as_float(hi)) & 0xffffe000u;
}
// D += A B, m16n8k8, A row-major TF32 (4 regs), B column-major TF32 (2 regs), D FP32.
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// acc[v] += rows[(k - kc) row of incidence][v] over the incidences inc[cur .. end) whose
// sub-tet k lies in [kc, kc + nk), in list order (the list is sorted by k).  Four incidences
// are fetched per round so that their shared-memory loads overlap; the additions keep the
// list order, so the sum is the same as one incidence at a time.
template <typename RowOf>
__device__ __forceinline__ void gather_in_order(const uint32_t* __restrict__ inc, int& cur, int end, int kc,
                                                int nk, RowOf row_of, float (&acc)[5]) {
  while (cur < end) {
    bool ok[4];
    const float* src[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ok[q] = cur + q < end;
      const uint32_t w = ok[q] ? inc[cur + q] : 0u;
      const int k = (int)(w >> 6) - kc;
      ok[q] = ok[q] && k < nk;  // a prefix of the four (the list is sorted by k)
      src[q] = row_of(ok[q] ? k : 0, (int)(w & 63));
    }
    float val[4][5];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int v = 0; v < 5; ++v) val[q][v] = ok[q] ? src[q][v] : 0.f;
    int adv = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (ok[q]) {
#pragma unroll
        for (int v = 0; v < 5; ++v) acc[v] += val[q][v];
        ++adv;
      }
    cur += adv;
    if (adv < 4) break;
  }
}

// Bulk (TMA) copy of `bytes` (multiple of 16, both addresses 16-byte aligned) global -> shared,
// completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ---- 5th-generation tensor cores (tcgen05) and tensor memory (TMEM).
// Ordering between thread-synchronising operations and tcgen05 work.
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Whole warp: allocate `cols` columns (a power of two >= 32) of this SM's tensor memory; the
// address is written to *dst in shared memory.  The block holds it until tmem_dealloc.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}
// Shared-memory matrix descriptor of a K-major operand without swizzle: 8-row x 16-byte
// core matrices, `lbo` bytes between K-adjacent ones, `sbo` bytes between row-adjacent ones.
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B (both K-major), M = 128.
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
// D[128 x N] (+)= A[128 x 8] * B[N x 8]^T, A in tensor memory (lane = row, column = k), B in
// shared memory.  The tensor core reads each FP32 operand as TF32 by dropping its 13 low
// mantissa bits (truncation).  Issued by one thread; completion is tracked by tc_commit.
__device__ __forceinline__ void tc_mma_tmem_a(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
      "r"(a), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
// Arrive once on `bar` when every tcgen05.mma this thread issued before has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// Warp-wide stores to / loads from tensor memory, shape 32x32b: lane l of the warp writes
// (reads) lane (quarter * 32 + l) of the addressed rows, consecutive columns.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}
__device__ __forceinline__ void tmem_st8v(uint32_t taddr, float a0, float a1, float a2, float a3, float a4, float a5,
                                          float a6, float a7) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr), "f"(a0),
               "f"(a1), "f"(a2), "f"(a3), "f"(a4), "f"(a5), "f"(a6), "f"(a7)
               : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// 16 consecutive columns, waiting for the load in the same statement (the registers are
// valid only after the wait)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n\ttcgen05.wait::ld.sync.aligned;"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]), "=f"(v[8]),
        "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
      : "r"(taddr)
      : "memory");
}
// FP32 -> TF32 by truncation (the value the tensor core reads) and the remainder.
__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xffffe000u); }

// Largest cell (nodes) the FP32 predictor handles: up to kF32Items (node, time slice) gather
// items and two 4-row groups of the M_i^-1 apply per thread.
constexpr int kF32MaxNodes = 640;
constexpr int kF32Items = 5;  // ceil(640 * 4 / 512)
inline int predictor_f32_max_nodes(int N) {
  const int by_items = kF32Items * kF32Threads / (N + 1);
  const int by_rows = 3 * 16 * kF32Consumers;  // three 16-row tiles per consumer warp
  (void)N;
  return std::min(kF32MaxNodes, std::min(by_items, by_rows));
}

// Row stride (floats) of q in shared memory: Nt*5 made odd, so that one thread per row
// touches 32 different banks.
constexpr int f32_row_stride(int N) { return ((N + 1) * 5) | 1; }
// Time slices of RHS / Y padded to a vector width, and their row stride [5][NTP].
constexpr int f32_ntp(int N) { return N == 1 ? 2 : 4; }
// Row stride of RHS / Y: 24 floats (5 NTP used, the rest zero), a multiple of 8 columns for
// the tensor-core tiles, and 24 = 8 (mod 16) for conflict-free fragment loads.
constexpr int f32_rhs_stride(int N) { return (void)N, 24; }
// Sub-tets per (narrow) chunk of the right-hand side; wide chunks take twice as many.
constexpr int f32_chunk(int N) { return f32_ntp(N) == 4 ? 8 : 16; }

// Packed FP32 sub-tet record: adj(J) row-major (9 floats), det J, then the Np cell-local node
// ids (uint16); padded to 16 bytes so that a cell's records are one bulk copy.
constexpr int f32_rec_bytes(int N) { return (40 + 2 * np_of(N) + 15) / 16 * 16; }

// Dynamic shared memory of the FP32 predictor: a fixed part (chunk results, per-warp staging,
// sub-tet records) and, per cell, q and RHS rows followed by a ring of M_i^-1 stages that
// takes whatever is left.  Returns the bytes needed for the largest cell with one stage.
// Byte sizes of the fixed parts; the kernel carves its shared memory with the same functions.
__host__ __device__ constexpr size_t f32_up128(size_t x) { return (x + 127) / 128 * 128; }
__host__ __device__ constexpr size_t f32_sR_bytes(int N, int ch) {
  return f32_up128((size_t)ch * (N + 1) * np_of(N) * 5 * 4);
}
// Column stride (floats) of the pre-contracted fluxes B^T[(k, t, v)][(d, j)] in shared memory:
// 3 Np values padded to a multiple of 4 floats with an odd number of 16-byte groups (16-byte
// rows for vector loads; the eight lanes of a quarter warp that load consecutive columns hit
// eight different bank groups).  gen_sref.cpp emits the same stride as SrefFP32<N>::KKS.
__host__ __device__ constexpr int f32_kks(int N) {
  return 4 * (((3 * np_of(N) + 3) / 4) % 2 == 0 ? (3 * np_of(N) + 3) / 4 + 1 : (3 * np_of(N) + 3) / 4);
}
__host__ __device__ constexpr size_t f32_sB_bytes(int N, int ch) {
  return f32_up128((size_t)ch * (N + 1) * 5 * f32_kks(N) * 4);
}
__host__ __device__ constexpr size_t f32_sR_bytes(int N) { return f32_sR_bytes(N, f32_chunk(N)); }
__host__ __device__ constexpr size_t f32_sB_bytes(int N) { return f32_sB_bytes(N, f32_chunk(N)); }
// Bytes needed for the largest cell with one stage of M_i^-1.
// The cell's node -> (sub-tet, local node) incidences (one per sub-tet node) and their row
// offsets, staged in shared memory for the gathers.
__host__ __device__ constexpr size_t f32_inc_bytes(int N, int Smax) {
  return f32_up128((size_t)Smax * np_of(N) * 4) + f32_up128((size_t)(kF32MaxNodes + 1) * 4);
}
// Per-cell plan of the predictor's shared memory: whether the right-hand side takes chunks
// of 2 CH sub-tets (4-time contraction tiles) and how many M_i^-1 stages the ring holds.
// The kernel and the host-side plan report use this one function.
struct F32CellPlan {
  bool wide;
  int nstage;
};
__host__ __device__ inline F32CellPlan f32_cell_plan(int N, size_t smem_bytes, int Smax, int Ni) {
  const int SR = f32_row_stride(N), SRN = f32_rhs_stride(N), CH = f32_chunk(N);
  const size_t fixed = f32_up128((size_t)Smax * f32_rec_bytes(N)) + f32_inc_bytes(N, Smax) +
                       f32_up128((size_t)Ni * SR * 4) + f32_up128((size_t)Ni * SRN * 4);
  const size_t region = smem_bytes > fixed ? smem_bytes - fixed : 0;
  F32CellPlan P;
  P.wide = f32_ntp(N) == 4 && region >= f32_sR_bytes(N, 2 * CH) + f32_sB_bytes(N, 2 * CH);
  const size_t stage = (size_t)kF32Rows * minv_ld(Ni) * 4;
  const size_t ns = region / stage;
  P.nstage = (int)(ns < (size_t)kF32MaxStages ? ns : (size_t)kF32MaxStages);
  return P;
}

// Tensor-memory form of the M_i^-1 apply: per 128-row tile of Y one accumulator in tensor
// memory, D[128 x 2 NB] = (A_hi + A_lo) [B_hi | B_lo] with A = the tile's rows of M_i^-1
// (staged into tensor memory, split into the TF32 value and its remainder) and B = the
// right-hand side split the same way, stored in shared memory as one K-major operand of
// 2 NB rows (NB = 5 NTP rounded up to 8).  Y = D[:, 0:NB] + D[:, NB:2 NB] (3xTF32 plus the
// negligible lo * lo product).
constexpr int tc_nb(int N) { return (5 * f32_ntp(N) + 7) / 8 * 8; }
constexpr int kTcMaxTiles = 5;      // 128-row tiles: cells of up to 640 nodes
constexpr int kTcGroups = 3;        // groups of 4 warps that stage M_i^-1 and read Y
constexpr int kTcStagers = 4 * kTcGroups;
constexpr int kTcDCols = 48;        // tensor-memory columns per accumulator (2 NB <= 48)
constexpr int kTcBufs = 3;          // most A staging buffers per tile
constexpr int kTcCols = 512;
// A staging buffers per tile for a cell of `ntiles` tiles: as many as the 512 columns hold
// after the accumulators (32 columns each: TF32 value and remainder of 16 rows)
__host__ __device__ constexpr int tc_nbuf(int ntiles) { return ntiles <= 3 ? 3 : (ntiles == 4 ? 2 : 1); }
// Bytes of the right-hand-side operand: 2 NB rows x Kp (N_i rounded up to 16) TF32 words.
__host__ __device__ inline size_t tc_bop_bytes(int N, int Ni) {
  const size_t Kp = (size_t)(Ni + 15) / 16 * 16;
  return (size_t)(2 * tc_nb(N)) * Kp * 4;
}
struct TcCellPlan {
  bool ok;      // the cell fits this form
  bool wide;    // right-hand side in chunks of 2 CH sub-tets
  int rows;     // rows of M_i^-1 per ring stage (32, 16 or 8)
  int slice;    // rows (= K columns) staged into tensor memory at a time: min(16, rows)
  int nstage;   // stages the ring holds
  int ntiles;   // 128-row tiles of Y
};
__host__ __device__ inline TcCellPlan tc_cell_plan(int N, size_t smem_bytes, int Smax, int Ni) {
  const int SR = f32_row_stride(N), CH = f32_chunk(N);
  const size_t fixed = f32_up128((size_t)Smax * f32_rec_bytes(N)) + f32_inc_bytes(N, Smax) +
                       f32_up128((size_t)Ni * SR * 4);
  const size_t region = smem_bytes > fixed ? smem_bytes - fixed : 0;
  TcCellPlan P{};
  P.wide = f32_ntp(N) == 4 && region >= f32_sR_bytes(N, 2 * CH) + f32_sB_bytes(N, 2 * CH);
  const bool narrow_ok = region >= f32_sR_bytes(N, CH) + f32_sB_bytes(N, CH);
  const size_t bop = f32_up128(tc_bop_bytes(N, Ni));
  const size_t room = region > bop ? region - bop : 0;
  int best = 0, best_ns = 0;
  for (int R = 32; R >= 8; R /= 2) {  // the tallest stage of which two fit, else of which one fits
    const size_t ns = room / ((size_t)R * minv_ld(Ni) * 4);
    if (ns >= 2) {
      best = R;
      best_ns = (int)(ns < (size_t)kF32MaxStages ? ns : (size_t)kF32MaxStages);
      break;
    }
    if (ns == 1 && best == 0) {
      best = R;
      best_ns = 1;
    }
  }
  P.rows = best;
  P.nstage = best_ns;
  P.slice = best < 16 ? best : 16;
  P.ntiles = (Ni + 127) / 128;
  P.ok = narrow_ok && best > 0 && P.ntiles <= kTcMaxTiles && Ni <= kF32MaxNodes;
  return P;
}

inline size_t predictor_f32_smem(int N, int Nmax, int Smax) {
  const size_t phase1 = f32_sR_bytes(N) + f32_sB_bytes(N);
  const size_t stage = (size_t)kF32Rows * minv_ld(Nmax) * 4;
  return f32_up128((size_t)Smax * f32_rec_bytes(N)) + f32_inc_bytes(N, Smax) +
         f32_up128((size_t)Nmax * f32_row_stride(N) * 4) + f32_up128((size_t)Nmax * f32_rhs_stride(N) * 4) +
         std::max(phase1, stage);
}

// physical flux F_e[v] at one (sub-tet, time, local node j); gradients (viscous only) from the
// sub-tet's own polynomial
template <int N>
__device__ __forceinline__ void f32_flux(const float* __restrict__ sq, const uint16_t* __restrict__ Ak,
                                         const float* __restrict__ g, int j, int t, bool visc, float mu, float kap,
                                         float gam, float Rg, const float (*sD)[np_of(N)][np_of(N)], float F[3][5]) {
  constexpr int NP = np_of(N), SQ = f32_row_stride(N);
  float Q[5];
  const float* qn = sq + Ak[j] * SQ + t * 5;
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
      const float* ql = sq + Ak[l] * SQ + t * 5;
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
  phys_flux<float>(Q, gq, visc, mu, kap, gam, Rg, F);
}
// flux pre-contraction: out[d][v] = scale sum_e adj(J)[d][e] F_e[v]
__device__ __forceinline__ void f32_contract_adj(const float* __restrict__ g, float scale, const float (&F)[3][5],
                                                 float out[3][5]) {
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int v = 0; v < 5; ++v) out[d][v] = scale * (g[d * 3 + 0] * F[0][v] + g[d * 3 + 1] * F[1][v] + g[d * 3 + 2] * F[2][v]);
}
template <int N>
__device__ __forceinline__ void f32_flux_contract(const float* __restrict__ sq, const uint16_t* __restrict__ Ak,
                                                  const float* __restrict__ g, int j, int t, bool visc, float mu,
                                                  float kap, float gam, float Rg, float scale,
                                                  const float (*sD)[np_of(N)][np_of(N)], float out[3][5]) {
  float F[3][5];
  f32_flux<N>(sq, Ak, g, j, t, visc, mu, kap, gam, Rg, sD, F);
  f32_contract_adj(g, scale, F, out);
}

// Inputs of the tensor-memory apply's streaming loops (one cell-iteration).
struct TcStreamArgs {
  int warp, lane, Ni, LD, srows, stage_floats, nstage, nblk, SL, spr, nsl, ntl, nbuf;
  float* ring;
  const float* minv;
  uint32_t tmem, bsh, sbo;
  uint64_t *sfull, *sempty, *safull, *saempty, *sdfull;
  int* abortp;
  int* flags;
};
// Barrier parities and counts the streaming loops carry from one cell-iteration to the next.
struct TcStreamState {
  uint32_t fpar, epar, ipar, issued, afp, acnt, aever;
};
// The producer, staging and issuing loops of the tensor-memory M_i^-1 apply, kept out of line:
// the kernel's long-lived per-cell values are saved once around the call instead of being
// spilled and reloaded (from L2: the 216 KB of shared memory leave L1 almost nothing) inside
// these loops.
template <int N>
__device__ __noinline__ TcStreamState tc_stream(const TcStreamArgs a, TcStreamState st) {
  constexpr int NB = tc_nb(N), NM = 2 * NB;
  constexpr uint32_t IDESC = tc_idesc_tf32(NM);
  const int warp = a.warp, lane = a.lane, Ni = a.Ni, LD = a.LD, srows = a.srows, stage_floats = a.stage_floats;
  const int nstage = a.nstage, nblk = a.nblk, SL = a.SL, spr = a.spr, nsl = a.nsl, ntl = a.ntl, nbuf = a.nbuf;
  float* const ring = a.ring;
  const float* const minv = a.minv;
  const uint32_t tmem = a.tmem, bsh = a.bsh, sbo = a.sbo;
  uint64_t* const sfull = a.sfull;
  uint64_t* const sempty = a.sempty;
  uint64_t* const safull = a.safull;
  uint64_t* const saempty = a.saempty;
  uint64_t* const sdfull = a.sdfull;
  int* const abortp = a.abortp;
  int* const flags = a.flags;
  uint32_t fpar = st.fpar, epar = st.epar, ipar = st.ipar, issued = st.issued, afp = st.afp, acnt = st.acnt,
           aever = st.aever;
  auto acol = [&](int T, int b) { return (uint32_t)(ntl * kTcDCols + (T * nbuf + b) * 32); };
  (void)LD;
    if (warp == kF32Warps - 1) {
      if (lane == 0) {
        for (int b = 0; b < nblk && !*(volatile int*)abortp; ++b) {
          const int s = b % nstage;
          if (b >= nstage) {
            if (!mbar_wait_bounded(&sempty[s], (epar >> s) & 1u)) {
              atomicOr(&flags[F_TIMEOUT], 1);
              *abortp = 1;
              break;
            }
            epar ^= 1u << s;
          }
          const int rb = min(srows, Ni - b * srows);
          mbar_expect_tx(&sfull[s], (uint32_t)(rb * LD * 4));
          bulk_g2s(ring + (size_t)s * stage_floats, minv + (size_t)b * stage_floats, (uint32_t)(rb * LD * 4),
                   &sfull[s]);
          issued |= 1u << s;
          ipar ^= 1u << s;
        }
        for (int b = max(0, nblk - nstage); b < nblk && !*(volatile int*)abortp; ++b) {
          const int s = b % nstage;
          if (!mbar_wait_bounded(&sempty[s], (epar >> s) & 1u)) {
            atomicOr(&flags[F_TIMEOUT], 1);
            *abortp = 1;
            break;
          }
          epar ^= 1u << s;
        }
      }
    } else if (warp < kTcStagers) {
      // staging warps: group g = warp / 4 owns tiles g, g + 3; warp quarter qq = warp % 4
      const int g = warp >> 2, qq = warp & 3;
      for (int s = 0; s < nsl; ++s) {
        if (*(volatile int*)abortp) break;
        const int b = s / spr, sl = s - b * spr, slot = b % nstage;
        const int rb = min(srows, Ni - b * srows);
        bool ok = true;
        if (sl == 0) {  // the stage has arrived
          if (lane == 0) ok = mbar_wait_bounded(&sfull[slot], (fpar >> slot) & 1u);
          ok = __shfl_sync(0xffffffffu, ok, 0);
          if (!ok) {
            if (lane == 0) {
              atomicOr(&flags[F_TIMEOUT], 1);
              *abortp = 1;
            }
            break;
          }
          __syncwarp();  // lane 0 observed the phase (acquire); the warp barrier orders the rest
          fpar ^= 1u << slot;
        }
        const float* stage = ring + (size_t)slot * stage_floats;
        const int buf = s % nbuf;
        for (int T = g; T < ntl; T += kTcGroups) {
          const int bi = T * kTcBufs + buf;
          if ((aever >> bi) & 1u) {  // the MMAs that last read this A buffer have completed
            if (lane == 0) ok = mbar_wait_bounded(&saempty[bi], ((acnt >> bi) & 1u) ^ 1u);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            __syncwarp();  // lane 0 observed the phase (acquire); the warp barrier orders the rest
            tc_fence_after();
          }
          const int mrow = T * 128 + qq * 32 + lane;
          const uint32_t ta = tmem + ((uint32_t)(qq * 32) << 16) + acol(T, buf);
          // the slice's columns k of this thread's row of M_i^-1: every shared-memory load
          // first, then the tensor-memory stores (a load issued behind a store waits for it)
          const int kend = (mrow < Ni) ? min(SL, rb - sl * SL) : 0;
          const float* src = stage + (size_t)(sl * SL) * LD + mrow;
          float x[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) x[i] = (i < kend) ? src[i * LD] : 0.f;
          tmem_st8v(ta, x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7]);
          tmem_st8v(ta + 16, x[0] - tf32_trunc(x[0]), x[1] - tf32_trunc(x[1]), x[2] - tf32_trunc(x[2]),
                    x[3] - tf32_trunc(x[3]), x[4] - tf32_trunc(x[4]), x[5] - tf32_trunc(x[5]),
                    x[6] - tf32_trunc(x[6]), x[7] - tf32_trunc(x[7]));
          if (SL == 16) {
            tmem_st8v(ta + 8, x[8], x[9], x[10], x[11], x[12], x[13], x[14], x[15]);
            tmem_st8v(ta + 24, x[8] - tf32_trunc(x[8]), x[9] - tf32_trunc(x[9]), x[10] - tf32_trunc(x[10]),
                      x[11] - tf32_trunc(x[11]), x[12] - tf32_trunc(x[12]), x[13] - tf32_trunc(x[13]),
                      x[14] - tf32_trunc(x[14]), x[15] - tf32_trunc(x[15]));
          }
          acnt ^= 1u << bi;  // the issuer commits once per tile and slice
          aever |= 1u << bi;
        }
        if (!ok) {
          if (lane == 0) {
            atomicOr(&flags[F_TIMEOUT], 1);
            *abortp = 1;
          }
          break;
        }
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          for (int T = g; T < ntl; T += kTcGroups) mbar_arrive(&safull[T * kTcBufs + buf]);
          if (sl == spr - 1 || s == nsl - 1) mbar_arrive(&sempty[slot]);  // stage read
        }
      }
    } else if (warp < kTcStagers + kTcGroups && lane == 0) {
      // issuing thread of group g: per slice and tile, once the four staging warps have
      // filled the A buffer, D_T += A_hi [B_hi | B_lo] + A_lo [B_hi | B_lo] per 8 columns
      const int g = warp - kTcStagers;
      for (int s = 0; s < nsl; ++s) {
        if (*(volatile int*)abortp) break;
        const int buf = s % nbuf;
        bool ok = true;
        for (int T = g; T < ntl; T += kTcGroups) {
          const int bi = T * kTcBufs + buf;
          if (!mbar_wait_bounded(&safull[bi], (afp >> bi) & 1u)) {
            ok = false;
            break;
          }
          afp ^= 1u << bi;
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(T * kTcDCols);
          const uint32_t a = tmem + acol(T, buf);
          for (int j = 0; j < SL / 8; ++j) {
            const int k0 = s * SL + 8 * j;
            const uint64_t bd = tc_sdesc(bsh + (uint32_t)k0 * 32u, 128u, sbo);
            tc_mma_tmem_a(d, a + 8 * j, bd, IDESC, (s | j) != 0 ? 1u : 0u);
            tc_mma_tmem_a(d, a + 16 + 8 * j, bd, IDESC, 1u);
          }
          tc_commit(&saempty[bi]);
        }
        if (!ok) {
          atomicOr(&flags[F_TIMEOUT], 1);
          *abortp = 1;
          break;
        }
      }
      if (!*(volatile int*)abortp)
        for (int T = g; T < ntl; T += kTcGroups) tc_commit(&sdfull[T]);
    }
  return TcStreamState{fpar, epar, ipar, issued, afp, acnt, aever};
}

// TC = true: the M_i^-1 apply on the 5th-generation tensor cores with tensor memory (tcgen05);
// TC = false: the same product with mma.sync on the per-warp tensor-core path.
template <int N, bool TC>
__global__ void __launch_bounds__(kF32Threads, 1) predictor_f32_kernel(const __grid_constant__ Batch bt,
                                                                        const RefData* __restrict__ ref,
                                                                        int diag, int smem_bytes) {
  constexpr int NP = np_of(N), NT = N + 1, NF = nf_of(N), SR = f32_row_stride(N);
  constexpr int NTP = f32_ntp(N), SRN = f32_rhs_stride(N), CH = f32_chunk(N);
  constexpr int KKS = f32_kks(N);  // column stride of B^T
  static_assert(KKS == SrefFP32<N>::KKS && SrefFP32<N>::KK == 3 * NP, "generated contraction and layout disagree");
  constexpr int REC = f32_rec_bytes(N);  // bytes per sub-tet record
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ float sD[3][NP][NP];    // nodal derivative matrices (viscous fluxes)
  __shared__ float sK[NT][NT];
  __shared__ float sW[NT];
  __shared__ __align__(8) uint64_t sbar;
  __shared__ __align__(8) uint64_t sfull[kF32MaxStages];
  __shared__ __align__(8) uint64_t sempty[kF32MaxStages];
  __shared__ int sAbort;
  __shared__ float sred[2][kF32Warps];
  __shared__ int64_t sCell;
  // tensor-memory form: per (tile, buffer) "A staged" and "MMAs done reading A", per tile
  // "accumulator complete", per staging group a drain barrier; the tensor-memory address
  __shared__ __align__(8) uint64_t safull[TC ? kTcBufs * kTcMaxTiles : 1];
  __shared__ __align__(8) uint64_t saempty[TC ? kTcBufs * kTcMaxTiles : 1];
  __shared__ __align__(8) uint64_t sdfull[TC ? kTcMaxTiles : 1];
  __shared__ __align__(8) uint64_t sdrain[TC ? kTcGroups : 1];
  __shared__ uint32_t stmem;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Nmax = bt.Nmax;
  auto up = [](size_t x) { return (x + 127) / 128 * 128; };
  unsigned char* p = smem_raw;
  unsigned char* srec = p;  // [S][REC] sub-tet records of the current cell
  p += f32_up128((size_t)bt.Smax * REC);
  uint32_t* sinc = reinterpret_cast<uint32_t*>(p);  // [incidences] (k << 6) | j of the cell's nodes
  int* sincp = reinterpret_cast<int*>(p + f32_up128((size_t)bt.Smax * NP * 4));  // [N_i + 1] row offsets
  p += f32_inc_bytes(N, bt.Smax);
  unsigned char* const cell_base = p;  // per cell: sq, srhs, then {sR, sB | M_i^-1 ring}
  (void)Nmax;

  for (int e = tid; e < 3 * NP * NP; e += kF32Threads) {
    const int d = e / (NP * NP), r = (e / NP) % NP, c = e % NP;
    sD[d][r][c] = (float)ref->D[d][r][c];
  }
  if (tid < NT * NT) sK[tid / NT][tid % NT] = (float)ref->K1tinv[tid / NT][tid % NT];
  if (tid < NT) sW[tid] = (float)ref->w[tid];
  if (tid == 0) {
    mbar_init(&sbar, 1);
    for (int i = 0; i < kF32MaxStages; ++i) {
      mbar_init(&sfull[i], 1);
      mbar_init(&sempty[i], TC ? kTcStagers : kF32Consumers);
    }
    if constexpr (TC) {
      for (int i = 0; i < kTcBufs * kTcMaxTiles; ++i) {
        mbar_init(&safull[i], 4);
        mbar_init(&saempty[i], 1);
      }
      for (int i = 0; i < kTcMaxTiles; ++i) mbar_init(&sdfull[i], 1);
      for (int i = 0; i < kTcGroups; ++i) mbar_init(&sdrain[i], 1);
    }
    sAbort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if constexpr (TC) {
    if (warp == 0) tmem_alloc(&stmem, kTcCols);  // one block per SM: all 512 columns
    tc_fence_before();
  }
  __syncthreads();
  if constexpr (TC) tc_fence_after();
  const uint32_t tmem = TC ? stmem : 0u;
  // tensor-memory form: parities / counts of the barriers this thread waits on or tracks
  uint32_t afp = 0;     // issuer: parity of the next completion of safull[i]
  uint32_t acnt = 0;    // staging group: parity of the commits issued into saempty[i] so far
  uint32_t aever = 0;   // staging group: saempty[i] has received a commit
  uint32_t dpar = 0;    // staging group: parity of the next completion of sdfull[T]
  (void)afp; (void)acnt; (void)aever; (void)dpar; (void)tmem;
  uint32_t phase = 0;
  uint32_t fpar = 0, epar = 0;  // parities of the next completion of sfull[s] / sempty[s]
  // producer lane: parity of the phase of sfull[s] its next copy into slot s completes, and
  // the slots that have received a copy (to drain exactly the copies issued)
  uint32_t ipar = 0, issued = 0;
  const int64_t total = bt.cpre[bt.nh];
  auto rec_g = [&](int k) { return reinterpret_cast<const float*>(srec + (size_t)k * REC); };
  auto rec_a = [&](int k) { return reinterpret_cast<const uint16_t*>(srec + (size_t)k * REC + 40); };

  for (;;) {
    if (tid == 0) {  // next cell of the work queue (index order, or the schedule's cost order)
      const int w = atomicAdd(bt.work, 1);
      sCell = (bt.order != nullptr && (int64_t)w < total) ? (int64_t)bt.order[w] : (int64_t)w;
    }
    __syncthreads();
    const int64_t gc = sCell;
    if (gc >= total) break;
    const int h = batch_find(bt.cpre, bt.nh, gc);
    const DevMesh& m = bt.tab[h];
    const int64_t c = gc - bt.cpre[h];
    const float dt = (float)*m.dt;
    const float gam = (float)m.gamma, Rg = (float)m.Rgas;
    const float tol = (float)m.tol;
    const int64_t n0 = m.node_ptr[c];
    const int Ni = (int)(m.node_ptr[c + 1] - n0);
    const int LD = minv_ld(Ni);
    const int64_t kbase = m.sub_ptr[c];
    const int S = (int)(m.sub_ptr[c + 1] - kbase);
    const float mu = (float)m.mu[c];
    const float kap = (float)cell_kappa(m, m.mu[c]);
    const bool visc = (mu != 0.f) || (kap != 0.f);
    const float* minv = m.minv32 + m.minv_ptr[c];
    const uint32_t* inc = sinc;  // the cell's incidences, staged in shared memory below
    float* sq = reinterpret_cast<float*>(cell_base);
    // mma.sync form: RHS / Y rows [N_i][SRN] after q; tensor-memory form: none (the
    // right-hand side operand lives in the shared region, Y in tensor memory)
    float* srhs = reinterpret_cast<float*>(cell_base + up((size_t)Ni * SR * 4));
    unsigned char* const shared_region = cell_base + up((size_t)Ni * SR * 4) + (TC ? 0 : up((size_t)Ni * SRN * 4));
    // chunks of 2 CH sub-tets (4-time contraction tiles) when the cell leaves room for them;
    // the M_i^-1 ring takes as many stages as fit (the same plans the host reports)
    const F32CellPlan plan = f32_cell_plan(N, (size_t)smem_bytes, bt.Smax, Ni);
    const TcCellPlan tplan = tc_cell_plan(N, (size_t)smem_bytes, bt.Smax, Ni);
    const bool wide = (TC ? tplan.wide : plan.wide) && !bt.narrow;
    const int CHc = wide ? 2 * CH : CH;
    float* sR = reinterpret_cast<float*>(shared_region);                          // phase 1, epilogue
    float* sBc = reinterpret_cast<float*>(shared_region + f32_sR_bytes(N, CHc));  // [CHc NT 5][KKS]
    // phase 2: the ring of M_i^-1 stages (after the right-hand-side operand in the TC form)
    float* bop = reinterpret_cast<float*>(shared_region);
    float* ring = reinterpret_cast<float*>(shared_region + (TC ? f32_up128(tc_bop_bytes(N, Ni)) : 0));
    const int srows = TC ? tplan.rows : kF32Rows;  // rows of M_i^-1 per stage
    const int stage_floats = srows * LD;
    const int nstage = min(TC ? tplan.nstage : plan.nstage, bt.ring_cap > 0 ? bt.ring_cap : kF32MaxStages);
    const int nblk = (Ni + srows - 1) / srows;
    // mma.sync form: the ring sits at the top of the shared region, slot s at top - (s + 1)
    // stages, so that slot 0 lies above the phase-1 buffers whenever the region leaves room
    // for a stage there; then the first stage of M_i^-1 is loaded while phase 1 runs (npre).
    const size_t region_top =
        ((size_t)smem_bytes - (size_t)(shared_region - smem_raw)) / 128 * 128;  // bytes of the region
    float* const ring_top = reinterpret_cast<float*>(shared_region + region_top);
    auto slot_ptr = [&](int sl) -> float* {
      return TC ? ring + (size_t)sl * stage_floats : ring_top - (size_t)(sl + 1) * stage_floats;
    };
    const int npre = (!TC && nblk > 0 && nstage > 0 &&
                      region_top >= f32_sR_bytes(N, CHc) + f32_sB_bytes(N, CHc) + (size_t)stage_floats * 4)
                         ? 1 : 0;

    // the cell's sub-tet records arrive by one bulk copy while the state is loaded
    if (tid == 0) {
      mbar_expect_tx(&sbar, (uint32_t)(S * REC));
      bulk_g2s(srec, m.sub32 + (size_t)kbase * REC, (uint32_t)(S * REC), &sbar);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int n = tid + r * kF32Threads;
      if (n < Ni) {
        const double* un = m.u + (n0 + n) * 5;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const float uv = (float)un[v];
#pragma unroll
          for (int t = 0; t < NT; ++t) sq[n * SR + t * 5 + v] = uv;
        }
      }
    }
    // the padded columns of RHS stay zero (so do those of Y)
    if constexpr (!TC)
      for (int e = tid; e < Ni * SRN; e += kF32Threads) srhs[e] = 0.f;
    {
      const int64_t ib = m.inc_ptr[n0];
      const int ninc = (int)(m.inc_ptr[n0 + Ni] - ib);  // <= S * NP
      for (int e = tid; e < ninc; e += kF32Threads) sinc[e] = m.inc[ib + e];
      for (int e = tid; e <= Ni; e += kF32Threads) sincp[e] = (int)(m.inc_ptr[n0 + e] - ib);
    }
    if (tid == 0 && !mbar_wait_bounded(&sbar, phase & 1u, m.first_wait_polls)) {
      atomicOr(&m.flags[F_TIMEOUT], 1);
      sAbort = 1;
    }
    __syncthreads();
    if (sAbort) {
      // a bulk copy that never completed: wait once more (bounded) for it, then leave
      if (tid == 0) (void)mbar_wait_bounded(&sbar, phase & 1u);
      goto kernel_exit;
    }
    // thread 0 observed the copy's completion (acquire); the barrier above orders the records
    // for every thread (a wait by all 512 threads would be 512 serialised barrier tests)
    phase ^= 1u;
    // the first stage's bulk copy may overwrite memory that earlier generic accesses (the
    // last cell's buffers) used: order them first (every thread, then the barrier)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();

    constexpr int NNT = (5 * NTP + 7) / 8;  // 8-column tiles of Y
    const bool consumer = warp < kF32Consumers;
    const int gq = lane >> 2, tq = lane & 3;  // mma fragment coordinates
    const int nmt = (Ni + 15) / 16;           // 16-row tiles of Y

    int it = 0;
    bool conv = false;
    while (!conv && it < m.picard_max) {
      ++it;
      // the first stage of M_i^-1 for this iteration's apply, into slot 0 above the phase-1
      // buffers (the ring was drained at the end of the last apply)
      if (npre && warp == kF32Warps - 1 && lane == 0) {
        const int rb = min(kF32Rows, Ni);
        mbar_expect_tx(&sfull[0], (uint32_t)(rb * LD * 4));
        bulk_g2s(slot_ptr(0), minv, (uint32_t)(rb * LD * 4), &sfull[0]);
        issued |= 1u;
        ipar ^= 1u;
      }
      // ---- 1. right-hand side RHS[n][t] = sum over incidences (k, j) of R_{k,t}[j]
      // First iteration of the mma.sync form: q^0 = u^ at every time node (the initial guess),
      // so the fluxes at the N+1 time nodes are equal and R_{k,t} = w_t R_k with R_k the
      // contraction of the time-independent flux; the right-hand side is RHS[n][t] = w_t r[n]
      // with r[n] = sum_{(k, j) at n} R_k[j], and Y[n][t] = w_t (M_i^-1 r)[n].  The same code
      // then runs with one time slice (NTe = 1, weight 1) on chunks (N+1) times as wide, and
      // the apply takes the 5 columns of r (one 8-column tile) instead of 5 (N+1).
      const bool first_const = !TC && it == 1;
      const int NTe = first_const ? 1 : NT;
      // gather items of this thread: (node, time slice) = (i / NTe, i % NTe), i = tid + 512 r
      int inode[kF32Items], cur[kF32Items], cend[kF32Items];
      float racc[kF32Items][5];
#pragma unroll
      for (int r = 0; r < kF32Items; ++r) {
        const int i = tid + r * kF32Threads;
        inode[r] = i < Ni * NTe ? (first_const ? i : i / NT) : -1;
        cur[r] = cend[r] = 0;
#pragma unroll
        for (int v = 0; v < 5; ++v) racc[r][v] = 0.f;
        if (inode[r] >= 0) {
          cur[r] = sincp[inode[r]];
          cend[r] = sincp[inode[r] + 1];
        }
      }
      // chunks of CHT sub-tets (a runtime value: one copy of the code for every width)
      const int CHT = first_const ? CHc * NT : CHc;
      for (int kc = 0; kc < S; kc += CHT) {
        const int nk = min(CHT, S - kc);
        // (a) fluxes: items (k, j, t), t fastest; the 15 values of an item go to the columns
        // (k, t, v) of B^T at rows (d, j)
        for (int e = tid; e < nk * NP * NTe; e += kF32Threads) {
          const int et = first_const ? e : e / NT, t = first_const ? 0 : e - et * NT;
          const int j = et % NP, kl = et / NP;
          float out[3][5];
          f32_flux_contract<N>(sq, rec_a(kc + kl), rec_g(kc + kl), j, t, visc, mu, kap, gam, Rg, 1.f, sD, out);
          float* dst = sBc + (size_t)((kl * NTe + t) * 5) * KKS + j;
#pragma unroll
          for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int v = 0; v < 5; ++v) dst[v * KKS + d * NP] = out[d][v];
        }
        __syncthreads();
        // (b) R[k][t][m][v] = w_t dt sum_{d,j} S^_d[m][j] B^T[(k, t, v)][d j]: one column per
        // thread, all Np rows m in registers, S^ as instruction immediates (zero entries skipped)
        for (int c = tid; c < nk * NTe * 5; c += kF32Threads) {
          float acc[NP];
#pragma unroll
          for (int i = 0; i < NP; ++i) acc[i] = 0.f;
          SrefFP32<N>::contract(sBc + (size_t)c * KKS, acc);
          const int kt = c / 5, v = c - kt * 5;  // kt = kl NTe + t
          const float wt = first_const ? 1.f : sW[kt % NT] * dt;  // time weight and dt, once per column
          float* dst = sR + kt * NP * 5 + v;
#pragma unroll
          for (int i = 0; i < NP; ++i) dst[5 * i] = wt * acc[i];
        }
        __syncthreads();
        // gather this chunk's incidences, in (k, j) order, into the items' registers
#pragma unroll
        for (int r = 0; r < kF32Items; ++r) {
          if (inode[r] < 0) continue;
          const int t = first_const ? 0 : (tid + r * kF32Threads) % NT;
          gather_in_order(inc, cur[r], cend[r], kc, nk,
                          [&](int k, int j) { return sR + ((k * NTe + t) * NP + j) * 5; }, racc[r]);
        }
        // no barrier here: the next chunk's flux items write only sB, and its contraction,
        // which overwrites sR, starts after the barrier that follows those items
      }
      if constexpr (!TC) {
        if (first_const) {
          // r in columns 0..4 (columns 5..7 of the tile are still zero from the cell's start)
#pragma unroll
          for (int r = 0; r < kF32Items; ++r) {
            if (inode[r] < 0) continue;
#pragma unroll
            for (int v = 0; v < 5; ++v) srhs[inode[r] * SRN + v] = dt * racc[r][v];
          }
        } else {
#pragma unroll
          for (int r = 0; r < kF32Items; ++r) {
            if (inode[r] < 0) continue;
            const int t = (tid + r * kF32Threads) % NT;
#pragma unroll
            for (int v = 0; v < 5; ++v) srhs[inode[r] * SRN + v * NTP + t] = racc[r][v];
          }
        }
      } else {
        // the right-hand-side operand B = [RHS | RHS - tf32(RHS)] (2 NB rows, K = the cell's
        // nodes) aliases the last chunk's buffers: every thread has finished its gathers first
        __syncthreads();
        constexpr int NB = tc_nb(N);
        const int Kp = (Ni + 15) / 16 * 16;
        auto bidx = [&](int n, int k) { return (n >> 3) * (Kp * 8) + (k >> 2) * 32 + (n & 7) * 4 + (k & 3); };
#pragma unroll
        for (int r = 0; r < kF32Items; ++r) {
          if (inode[r] < 0) continue;
          const int t = (tid + r * kF32Threads) % NT;
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            const float x = racc[r][v];
            bop[bidx(v * NTP + t, inode[r])] = x;
            bop[bidx(NB + v * NTP + t, inode[r])] = x - tf32_trunc(x);
          }
        }
        // rows without data (time slices past N+1, padding to NB) and columns past N_i: zero
        constexpr int NPAD = NB - 5 * NT;  // such rows per half
        constexpr int TP = NTP - NT > 0 ? NTP - NT : 1;  // padded time slices per variable (divisor)
        for (int e = tid; e < 2 * NPAD * Ni; e += kF32Threads) {
          const int k = e % Ni, pr = e / Ni, half = pr / NPAD;
          int nh = pr % NPAD;  // the nh-th row of a half that holds no data
          nh = nh < 5 * (NTP - NT) ? (nh / TP) * NTP + NT + nh % TP : 5 * NTP + (nh - 5 * (NTP - NT));
          bop[bidx(half * NB + nh, k)] = 0.f;
        }
        for (int e = tid; e < 2 * NB * (Kp - Ni); e += kF32Threads)
          bop[bidx(e / (Kp - Ni), Ni + e % (Kp - Ni))] = 0.f;
      }
      // the ring reuses the phase-1 buffers: order this thread's generic-proxy accesses to
      // them before the bulk copies (async proxy) that overwrite them; the tensor cores read
      // the right-hand-side operand through the async proxy too
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      float res = 0.f, qmax = 0.f;
      // q^{r+1}[n, s] = u^[n] - sum_t K1t^-1[s, t] Y[n, t], the residual and max |q^r|
      auto update_node = [&](int n, const float (&y)[NT][5]) {
        float uh[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) uh[v] = (float)m.u[(n0 + n) * 5 + v];  // u^ (L2-resident)
#pragma unroll
        for (int s2 = 0; s2 < NT; ++s2)
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            float x = uh[v];
#pragma unroll
            for (int t = 0; t < NT; ++t) x -= sK[s2][t] * y[t][v];
            const float old = sq[n * SR + s2 * 5 + v];
            res = fmaxf(res, fabsf(x - old));
            qmax = fmaxf(qmax, fabsf(old));
            sq[n * SR + s2 * 5 + v] = x;
          }
      };
      if constexpr (TC) {
        // ---- 2. Y = M_i^-1 RHS on the tensor cores with tensor memory.  The last warp streams
        // M_i^-1 through the ring of `srows`-row stages (as in the mma.sync form).  Three groups
        // of four warps (one warp per 32-lane quarter of tensor memory) own the 128-row tiles
        // T = g, g + 3 of Y: per slice of `SL` rows of a stage (= SL columns of M_i^-1 by
        // symmetry) each thread moves its row's SL values into the tile's A buffer in tensor
        // memory as TF32 value and remainder (up to three buffers per tile in turn); a
        // dedicated issuing warp per group (warps 12 - 14) then issues
        // D_T += A_hi [B_hi | B_lo] + A_lo [B_hi | B_lo] per 8 columns and commits.  Several
        // issuing warps keep the tensor core busy despite the narrow N.
        constexpr int NB = tc_nb(N), NM = 2 * NB;
        constexpr uint32_t IDESC = tc_idesc_tf32(NM);
        const int SL = tplan.slice, spr = srows / SL, nsl = (Ni + SL - 1) / SL;
        const int ntl = tplan.ntiles, nbuf = tc_nbuf(ntl);
        const uint32_t sbo = (uint32_t)((Ni + 15) / 16 * 16) * 32u;
        const uint32_t bsh = smem_u32(bop);
        // tensor-memory columns: accumulators T * 48, then the A buffers (32 columns each)
        auto acol = [&](int T, int b) { return (uint32_t)(ntl * kTcDCols + (T * nbuf + b) * 32); };
        {
          TcStreamArgs ta;
          ta.warp = warp;
          ta.lane = lane;
          ta.Ni = Ni;
          ta.LD = LD;
          ta.srows = srows;
          ta.stage_floats = stage_floats;
          ta.nstage = nstage;
          ta.nblk = nblk;
          ta.SL = SL;
          ta.spr = spr;
          ta.nsl = nsl;
          ta.ntl = ntl;
          ta.nbuf = nbuf;
          ta.ring = ring;
          ta.minv = minv;
          ta.tmem = tmem;
          ta.bsh = bsh;
          ta.sbo = sbo;
          ta.sfull = sfull;
          ta.sempty = sempty;
          ta.safull = safull;
          ta.saempty = saempty;
          ta.sdfull = sdfull;
          ta.abortp = &sAbort;
          ta.flags = m.flags;
          const TcStreamState ts = tc_stream<N>(ta, TcStreamState{fpar, epar, ipar, issued, afp, acnt, aever});
          fpar = ts.fpar;
          epar = ts.epar;
          ipar = ts.ipar;
          issued = ts.issued;
          afp = ts.afp;
          acnt = ts.acnt;
          aever = ts.aever;
        }
        __syncthreads();
        if (sAbort) {
          // a bounded wait ran out: wait (bounded) for the ring's copies in flight and for every
          // issuer's MMAs, then leave
          if (warp == kF32Warps - 1 && lane == 0)
            for (int s2 = 0; s2 < kF32MaxStages; ++s2)
              if ((issued >> s2) & 1u) (void)mbar_wait_bounded(&sfull[s2], ((ipar >> s2) & 1u) ^ 1u);
          if (warp >= kTcStagers && warp < kTcStagers + kTcGroups && lane == 0) {
            tc_commit(&sdrain[warp - kTcStagers]);
            (void)mbar_wait_bounded(&sdrain[warp - kTcStagers], 0u);
          }
          __syncthreads();
          goto kernel_exit;
        }
        // Y from the accumulators: thread (group g, quarter qq, lane) holds node T*128 + qq*32 + lane
        if (warp < kTcStagers) {
          const int g = warp >> 2, qq = warp & 3;
          for (int T = g; T < ntl; T += kTcGroups) {
            bool ok = true;
            if (lane == 0) ok = mbar_wait_bounded(&sdfull[T], (dpar >> T) & 1u);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
              if (lane == 0) {
                atomicOr(&m.flags[F_TIMEOUT], 1);
                sAbort = 1;
              }
              break;
            }
            __syncwarp();  // lane 0 observed the phase (acquire); the warp barrier orders the rest
            dpar ^= 1u << T;
            tc_fence_after();
            const uint32_t ta = tmem + ((uint32_t)(qq * 32) << 16) + (uint32_t)(T * kTcDCols);
            // Y column c = v NTP + t is D[:, c] + D[:, NB + c]; eight columns at a time
            float yf[NB];
#pragma unroll
            for (int c = 0; c < NB; c += 8) {
              float hi[8], lo[8];
              tmem_ld8(ta + c, hi);
              tmem_ld8(ta + NB + c, lo);
#pragma unroll
              for (int i = 0; i < 8; ++i) yf[c + i] = hi[i] + lo[i];
            }
            const int n = T * 128 + qq * 32 + lane;
            if (n < Ni) {
              float y[NT][5];
#pragma unroll
              for (int v = 0; v < 5; ++v)
#pragma unroll
                for (int t = 0; t < NT; ++t) y[t][v] = yf[v * NTP + t];
              update_node(n, y);
            }
          }
          tc_fence_before();
        }
      } else {
        // ---- 2. Y = M_i^-1 RHS.  The last warp streams M_i^-1 through a ring of shared-memory
        // stages (cp.async.bulk, full/empty mbarriers); the other warps never wait for each
        // other inside the apply.  Consumer warp w accumulates the 16 x 8 tiles (mt, nt) of Y
        // for mt = w, w + 15, w + 30 with 3xTF32 mma.sync; per 8-row k-step of a stage it loads
        // the B fragments (RHS rows) once for all column tiles and the A fragments (M_i^-1
        // rows = columns) once per row tile.
        // the consumer loops and Y's write-out for NT1 8-column tiles of RHS / Y: one in the
        // first iteration (the 5 time-independent columns), 5 (N+1) / 8 rounded up otherwise
        auto apply = [&](auto nt_tag) {
          constexpr int NT1 = decltype(nt_tag)::value;
          float cacc[3][NT1][4];
#pragma unroll
          for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int nt = 0; nt < NT1; ++nt)
#pragma unroll
              for (int i = 0; i < 4; ++i) cacc[r][nt][i] = 0.f;
          if (!consumer) {
            if (lane == 0) {
              for (int b = npre; b < nblk && !sAbort; ++b) {
                const int s = b % nstage;
                if (b >= nstage) {
                  if (!mbar_wait_bounded(&sempty[s], (epar >> s) & 1u)) {
                    atomicOr(&m.flags[F_TIMEOUT], 1);
                    sAbort = 1;
                    break;
                  }
                  epar ^= 1u << s;
                }
                const int rb = min(srows, Ni - b * srows);
                mbar_expect_tx(&sfull[s], (uint32_t)(rb * LD * 4));
                bulk_g2s(slot_ptr(s), minv + (size_t)b * stage_floats, (uint32_t)(rb * LD * 4), &sfull[s]);
                issued |= 1u << s;
                ipar ^= 1u << s;
              }
              // every stage released by the consumers before the ring is reused
              for (int b = max(0, nblk - nstage); b < nblk && !sAbort; ++b) {
                const int s = b % nstage;
                if (!mbar_wait_bounded(&sempty[s], (epar >> s) & 1u)) {
                  atomicOr(&m.flags[F_TIMEOUT], 1);
                  sAbort = 1;
                  break;
                }
                epar ^= 1u << s;
              }
            }
          } else {
            for (int b = 0; b < nblk; ++b) {
              const int s = b % nstage;
              // lane 0 waits (bounded); the warp follows its verdict, so that no lane leaves the
              // loop alone
              bool ok = true;
              if (lane == 0) ok = mbar_wait_bounded(&sfull[s], (fpar >> s) & 1u);
              ok = __shfl_sync(0xffffffffu, ok, 0);
              if (!ok) {
                if (lane == 0) {
                  atomicOr(&m.flags[F_TIMEOUT], 1);
                  sAbort = 1;
                }
                break;
              }
              __syncwarp();  // lane 0 observed the phase (acquire); the warp barrier orders the rest
              fpar ^= 1u << s;
              const float* stage = slot_ptr(s);
              const int l0 = b * kF32Rows, rb = min(kF32Rows, Ni - l0);
              // one 8-row k-step: B fragments (RHS rows) for every column tile, then per row tile the
              // A fragments (M_i^-1 rows) and three rounds of MMAs over the column tiles
              auto kstep = [&](int ks, bool full) {
                const int k0 = ks * 8 + tq, k1 = k0 + 4;  // stage rows of this lane's fragments
                const bool v0 = full || k0 < rb, v1 = full || k1 < rb;  // rows past N_i give zero
                uint32_t bh[NT1][2], bl[NT1][2];
#pragma unroll
                for (int nt = 0; nt < NT1; ++nt) {
                  const float x0 = v0 ? srhs[(l0 + k0) * SRN + nt * 8 + gq] : 0.f;
                  const float x1 = v1 ? srhs[(l0 + k1) * SRN + nt * 8 + gq] : 0.f;
                  tf32_split(x0, bh[nt][0], bl[nt][0]);
                  tf32_split(x1, bh[nt][1], bl[nt][1]);
                }
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                  const int mt = warp + r * kF32Consumers;
                  if (mt >= nmt) break;
                  const float* arow0 = stage + k0 * LD + mt * 16 + gq;
                  const float* arow1 = stage + k1 * LD + mt * 16 + gq;
                  uint32_t ah[4], al[4];
                  tf32_split(v0 ? arow0[0] : 0.f, ah[0], al[0]);
                  tf32_split(v0 ? arow0[8] : 0.f, ah[1], al[1]);
                  tf32_split(v1 ? arow1[0] : 0.f, ah[2], al[2]);
                  tf32_split(v1 ? arow1[8] : 0.f, ah[3], al[3]);
#pragma unroll
                  for (int nt = 0; nt < NT1; ++nt)
                    mma_tf32(cacc[r][nt], al, bh[nt][0], bh[nt][1]);
#pragma unroll
                  for (int nt = 0; nt < NT1; ++nt)
                    mma_tf32(cacc[r][nt], ah, bl[nt][0], bl[nt][1]);
#pragma unroll
                  for (int nt = 0; nt < NT1; ++nt)
                    mma_tf32(cacc[r][nt], ah, bh[nt][0], bh[nt][1]);
                }
              };
              if (rb == kF32Rows) {  // full stage: no row masks
#pragma unroll
                for (int ks = 0; ks < kF32Rows / 8; ++ks) kstep(ks, true);
              } else {
#pragma unroll
                for (int ks = 0; ks < kF32Rows / 8; ++ks) kstep(ks, false);
              }
              __syncwarp();
              if (lane == 0) mbar_arrive(&sempty[s]);
            }
          }
          __syncthreads();  // every thread has finished reading RHS and the ring is drained
          if (sAbort) return;
          if (consumer)
#pragma unroll
            for (int r = 0; r < 3; ++r) {
              const int mt = warp + r * kF32Consumers;
              if (mt >= nmt) break;
              const int n0r = mt * 16 + gq, n1r = n0r + 8;
#pragma unroll
              for (int nt = 0; nt < NT1; ++nt) {
                const int col = nt * 8 + 2 * tq;
                if (n0r < Ni) {
                  srhs[n0r * SRN + col] = cacc[r][nt][0];
                  srhs[n0r * SRN + col + 1] = cacc[r][nt][1];
                }
                if (n1r < Ni) {
                  srhs[n1r * SRN + col] = cacc[r][nt][2];
                  srhs[n1r * SRN + col + 1] = cacc[r][nt][3];
                }
              }
            }
        };
        if (first_const) apply(std::integral_constant<int, 1>{});
        else apply(std::integral_constant<int, NNT>{});
        if (sAbort) {
          // a bounded wait ran out (flags[F_TIMEOUT] is set): wait (bounded) for the last copy
          // issued into every slot (the phase its completion ends), then leave
          if (!consumer && lane == 0)
            for (int s2 = 0; s2 < kF32MaxStages; ++s2)
              if ((issued >> s2) & 1u) (void)mbar_wait_bounded(&sfull[s2], ((ipar >> s2) & 1u) ^ 1u);
          __syncthreads();
          goto kernel_exit;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int n = tid + r * kF32Threads;
          if (n >= Ni) continue;
          float y[NT][5];
          if (first_const) {
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              const float y0 = srhs[n * SRN + v];
#pragma unroll
              for (int t = 0; t < NT; ++t) y[t][v] = sW[t] * y0;
            }
            update_node(n, y);
            continue;
          }
#pragma unroll
          for (int v = 0; v < 5; ++v) {  // one vector load per variable
            float yv[NTP];
            if constexpr (NTP == 4) {
              const float4 w = *reinterpret_cast<const float4*>(srhs + n * SRN + v * 4);
              yv[0] = w.x; yv[1] = w.y; yv[2] = w.z; yv[3] = w.w;
            } else {
              const float2 w = *reinterpret_cast<const float2*>(srhs + n * SRN + v * 2);
              yv[0] = w.x; yv[1] = w.y;
            }
#pragma unroll
            for (int t = 0; t < NT; ++t) y[t][v] = yv[t];
          }
          update_node(n, y);
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
      if constexpr (TC) {
        if (sAbort) {  // an accumulator never completed: drain every issuer's MMAs and leave
          if (warp >= kTcStagers && warp < kTcStagers + kTcGroups && lane == 0) {
            tc_commit(&sdrain[warp - kTcStagers]);
            (void)mbar_wait_bounded(&sdrain[warp - kTcStagers], 0u);
          }
          __syncthreads();
          goto kernel_exit;
        }
      }
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
    if (tid == 0) {
      m.iters[c] = it;
      if (!conv) atomicAdd(&m.flags[F_NONCONV], 1);
    }

    // ---- epilogue: volume term vol = sum_k A_k^T sum_d S^_d^T adj(J_k) F_bar_k
    float vacc[2][5];
    int vcur[2], vend[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int n = tid + r * kF32Threads;
#pragma unroll
      for (int v = 0; v < 5; ++v) vacc[r][v] = 0.f;
      vcur[r] = vend[r] = 0;
      if (n < Ni) {
        vcur[r] = sincp[n];
        vend[r] = sincp[n + 1];
      }
    }
    const int CHV = CHc * NT;  // sub-tets per volume chunk (sR holds CHc*NT slices)
    float* sBv = sBc;          // [CHV 5][KKS] time-integrated pre-contracted fluxes (fits in sB)
    for (int kc = 0; kc < S; kc += CHV) {
      const int nk = min(CHV, S - kc);
      // (a) items (k, j): B_bar[k][d j][v] = sum_t w_t dt adj(J_k) F(q_t) at node j
      for (int e = tid; e < nk * NP; e += kF32Threads) {
        const int kl = e / NP, j = e % NP;
        // F_bar = sum_t w_t F(q_t), then dt adj(J) F_bar once
        float fbar[3][5];
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int v = 0; v < 5; ++v) fbar[d][v] = 0.f;
        for (int t = 0; t < NT; ++t) {
          float F[3][5];
          f32_flux<N>(sq, rec_a(kc + kl), rec_g(kc + kl), j, t, visc, mu, kap, gam, Rg, sD, F);
          const float wt = sW[t];
#pragma unroll
          for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int v = 0; v < 5; ++v) fbar[d][v] += wt * F[d][v];
        }
        float accb[3][5];
        f32_contract_adj(rec_g(kc + kl), dt, fbar, accb);
        float* dst = sBv + (size_t)(kl * 5) * KKS + j;  // columns (k, v), rows (d, j)
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int v = 0; v < 5; ++v) dst[v * KKS + d * NP] = accb[d][v];
      }
      __syncthreads();
      // (b) R_bar[k][m][v] = sum_{d,j} S^_d[j][m] B_bar^T[(k, v)][d j]: one column per thread, all
      // Np rows in registers, S^ as instruction immediates
      for (int c = tid; c < nk * 5; c += kF32Threads) {
        float acc[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) acc[i] = 0.f;
        SrefFP32<N>::contract_t(sBv + (size_t)c * KKS, acc);
        const int kl = c / 5, v = c - kl * 5;
        float* dst = sR + kl * NP * 5 + v;
#pragma unroll
        for (int i = 0; i < NP; ++i) dst[5 * i] = acc[i];
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        gather_in_order(inc, vcur[r], vend[r], kc, nk, [&](int k, int j) { return sR + (k * NP + j) * 5; },
                        vacc[r]);
      }
      // no barrier here: the next chunk's items write only B_bar, and its tiles, which
      // overwrite sR, start after the barrier that follows those items
    }
    __syncthreads();
    float* vol = (float*)m.vol;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int n = tid + r * kF32Threads;
      if (n < Ni)
#pragma unroll
        for (int v = 0; v < 5; ++v) vol[(n0 + n) * 5 + v] = vacc[r][v];
    }

    // face slots: q_bar and F_bar . n at every face node (flux of the owning sub-tet)
    const int64_t s0 = m.slot_ptr[c];
    const int ns = (int)(m.slot_ptr[c + 1] - s0);
    float* sqo = (float*)m.slot_q;
    float* sfn = (float*)m.slot_fn;
    for (int e = tid; e < ns * NF; e += kF32Threads) {
      const int sl = e / NF, a = e % NF;
      const int64_t sg = s0 + sl;
      const int kl = m.slot_sub[sg];
      const int j = m.slot_loc[sg * NF + a];
      const uint16_t* Ak = rec_a(kl);
      const float* g = rec_g(kl);
      const double* gs = m.slot_geo + sg * 4;
      const float nx = (float)gs[0], ny = (float)gs[1], nz = (float)gs[2];
      float qb[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, fb[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      for (int t = 0; t < NT; ++t) {
        float Q[5];
        const float* qn = sq + Ak[j] * SR + t * 5;
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
            const float* ql = sq + Ak[l] * SR + t * 5;
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
        for (int t = 0; t < NT; ++t) acc += sW[t] * sq[n * SR + t * 5 + v];
        m.qbar_diag[(n0 + n) * 5 + v] = (double)dt * (double)acc;
      }
    __syncthreads();
  }
kernel_exit:
  if constexpr (TC) {  // every path out of the cell loop ends here: release the tensor memory
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTcCols);
  }
}

// Packed FP32 sub-tet records (see f32_rec_bytes): adj(J) and det J as floats, node ids.
template <int N>
__global__ void sub32_kernel(DevMesh m, int64_t T) {
  constexpr int NP = np_of(N), REC = f32_rec_bytes(N);
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= T) return;
  float* g = reinterpret_cast<float*>(m.sub32 + k * REC);
#pragma unroll
  for (int i = 0; i < 10; ++i) g[i] = (float)m.geo[k * 10 + i];
  uint16_t* a = reinterpret_cast<uint16_t*>(m.sub32 + k * REC + 40);
  for (int j = 0; j < NP; ++j) a[j] = m.A[k * NP + j];
  for (int j = NP; j < (REC - 40) / 2; ++j) a[j] = 0;
}

}  // namespace afe

namespace afe {

// FP32 corrector (Sec. 4.4): one block of 128 threads per cell, six blocks per SM (the
// register cap that lets six fit keeps more of M_i^-1 in flight per SM; du waits in shared
// memory, not registers, until the FP64 correction is known).
//   r = vol - sum_slots 2 area Z^ G          (fixed-order gather, FP32)
//   du = M_i^-1 r                            (thread g: 4-row tiles 4g..4g+3, g + 128, ...;
//                                             M_i^-1 streamed by 16-byte loads, eight rows in
//                                             flight)
//   u += du + (T - w_i . du) / |P_i|         (FP64: T = exact cell total of r, see below)
// The FP64 correction makes the cell's conserved totals change by exactly
// T = 1^T r = -sum_slots 2 area sum_b (sum_a Z^[a][b]) G[b] (the volume term sums to zero:
// sum_m grad phi_m = 0), so the matched slots of neighbouring cells cancel in FP64.
constexpr int kCorrThreads = 128;

template <int N>
__global__ void __launch_bounds__(kCorrThreads, 6) corrector_f32_kernel(const __grid_constant__ Batch bt,
                                                                        const RefData* __restrict__ ref) {
  constexpr int NF = nf_of(N);
  extern __shared__ __align__(16) float sr[];  // [Nmax][5] r, then [Nmax][5] du
  __shared__ float sZ[NF][NF];
  __shared__ double szs[NF];
  __shared__ double sred[2][5][kCorrThreads];
  const int tid = threadIdx.x;
  for (int e = tid; e < NF * NF; e += kCorrThreads) sZ[e / NF][e % NF] = (float)ref->Z[e / NF][e % NF];
  if (tid < NF) {
    double z = 0.0;
    for (int a = 0; a < NF; ++a) z += ref->Z[a][tid];
    szs[tid] = z;
  }
  __syncthreads();
  const int64_t gc = blockIdx.x;
  if (gc >= bt.cpre[bt.nh]) return;
  const int h = batch_find(bt.cpre, bt.nh, gc);
  const DevMesh& m = bt.tab[h];
  const int64_t c = gc - bt.cpre[h];
  const int64_t n0 = m.node_ptr[c];
  const int Ni = (int)(m.node_ptr[c + 1] - n0);
  const int LD = minv_ld(Ni);
  const int64_t s0 = m.slot_ptr[c];
  const int ns = (int)(m.slot_ptr[c + 1] - s0);
  const float* vol = (const float*)m.vol;
  const float* sG = (const float*)m.slot_G;
  // r = vol - face term
  for (int n = tid; n < Ni; n += kCorrThreads) {
    float acc[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] = vol[(n0 + n) * 5 + v];
    for (int64_t p = m.finc_ptr[n0 + n]; p < m.finc_ptr[n0 + n + 1]; ++p) {
      const uint32_t w = m.finc[p];
      const int64_t s = s0 + (w >> 4);
      const int a = w & 15;
      const float twoA = 2.f * (float)m.slot_geo[s * 4 + 3];
      const float* g = sG + s * NF * 5;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        float f = 0.f;
#pragma unroll
        for (int b = 0; b < NF; ++b) f += sZ[a][b] * g[b * 5 + v];
        acc[v] -= twoA * f;
      }
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) sr[n * 5 + v] = acc[v];
  }
  // exact FP64 cell total of the update
  double tot[5] = {0, 0, 0, 0, 0};
  for (int e = tid; e < ns * NF; e += kCorrThreads) {
    const int64_t s = s0 + e / NF;
    const int b = e % NF;
    const double twoA = 2.0 * m.slot_geo[s * 4 + 3];
#pragma unroll
    for (int v = 0; v < 5; ++v) tot[v] -= twoA * szs[b] * (double)sG[(s * NF + b) * 5 + v];
  }
  __syncthreads();
  // du = M_i^-1 r, thread tid owns the column groups g = tid, tid + 128, ... (rows 4g..4g+3)
  const float* minv = m.minv32 + m.minv_ptr[c];
  double wdu[5] = {0, 0, 0, 0, 0};
  float* sdu = sr + (size_t)bt.Nmax * 5;  // du rows, kept in shared memory until corr is known
  for (int g = tid; 4 * g < Ni; g += kCorrThreads) {
    float du[1][4][5];  // one column group at a time
    constexpr int r = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int v = 0; v < 5; ++v) du[r][i][v] = 0.f;
    const float* col = minv + 4 * g;
    for (int l0 = 0; l0 < Ni; l0 += 8) {
      float4 a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        a[u] = l0 + u < Ni ? __ldcs(reinterpret_cast<const float4*>(col + (size_t)(l0 + u) * LD))
                           : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (l0 + u >= Ni) break;
        const float* x = sr + (l0 + u) * 5;
        const float av[4] = {a[u].x, a[u].y, a[u].z, a[u].w};
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const float xv = x[v];
#pragma unroll
          for (int i = 0; i < 4; ++i) du[r][i][v] += av[i] * xv;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int n = 4 * g + i;
      if (n >= Ni) break;
      const double w = m.wvec[n0 + n];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        wdu[v] += w * (double)du[r][i][v];
        sdu[n * 5 + v] = du[r][i][v];
      }
    }
  }
  // fixed-order block reductions of T and w . du
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    sred[0][v][tid] = tot[v];
    sred[1][v][tid] = wdu[v];
  }
  __syncthreads();
  for (int st = kCorrThreads / 2; st > 0; st >>= 1) {
    if (tid < st)
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        sred[0][v][tid] += sred[0][v][tid + st];
        sred[1][v][tid] += sred[1][v][tid + st];
      }
    __syncthreads();
  }
  double corr[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) corr[v] = (sred[0][v][0] - sred[1][v][0]) / m.cell_vol[c];
  for (int g = tid; 4 * g < Ni; g += kCorrThreads) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int n = 4 * g + i;
      if (n >= Ni) break;
      double* un = m.u + (n0 + n) * 5;
      bool bad = false;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        un[v] += (double)sdu[n * 5 + v] + corr[v];
        bad |= !isfinite(un[v]);
      }
      // rho > 0 and p > 0, with p > 0 tested as rho E > |rho u|^2 / 2 (no division)
      const double rho = un[0];
      const double pr = rho * un[4] - 0.5 * (un[1] * un[1] + un[2] * un[2] + un[3] * un[3]);
      if (bad || !(rho > 0.0) || !(pr > 0.0)) atomicOr(&m.flags[F_NONFINITE], 8);
    }
  }
}

}  // namespace afe
