// Build-time generator of the FP32 predictor's reference-stiffness contractions (Sec. 4.3,
// Eq. ader4: R_{k,t} = sum_d S^_d (dt adj(J_k) F)_d; Eq. TAvectors: the volume term with
// S^_d transposed).
//
// The stiffness matrices S^_d[m][l] = int phi_m d/dxi_d phi_l of the reference tetrahedron are
// universal, so the contraction of one column b[(d, j)] (the 3 Np pre-contracted flux values of
// one sub-tet, variable and time slice) with them can be written out with the matrix entries
// as instruction immediates: every multiply-add reads its coefficient from the instruction
// stream (no shared-memory or constant-cache traffic for S^) and the entries that vanish are
// not multiplied at all.  The entries are those of build_ref() (the values the library uploads
// for its other kernels), rounded to FP32 as the FP32 form uses them.  Entries that vanish in
// exact arithmetic come out of build_ref()'s extended-precision solve at the 1e-19 level; those
// below 1e-13 of the largest entry are taken as the zeros they are.  The accumulation runs over
// (d, j) in increasing order for every m, as a dense loop would.
//
// Usage: gen_sref <output header>
#include <cmath>
#include <cstdio>
#include <string>

#include "refelem.hpp"

namespace {

// Row stride (floats) of a column in shared memory: a multiple of 4 floats (16-byte rows for
// vector loads) with an odd number of 16-byte groups, so that the eight lanes of a quarter
// warp that load consecutive columns hit eight different bank groups.
int column_stride(int kk) {
  int g = (kk + 3) / 4;
  if (g % 2 == 0) ++g;
  return 4 * g;
}

std::string lit(float x) {
  char buf[64];
  std::snprintf(buf, sizeof buf, "%af", (double)x);
  return buf;
}

// acc[m] += sum_{kk < KK} C(m, kk) b[kk], kk = d Np + j, in increasing kk for every m.
template <typename Coef>
void emit_body(FILE* f, int np, Coef coef) {
  const int kk_n = 3 * np;
  const int groups = (kk_n + 3) / 4;
  for (int q = 0; q < groups; ++q) {
    std::fprintf(f, "    {\n      const float4 x = *reinterpret_cast<const float4*>(b + %d);\n", 4 * q);
    static const char* comp[4] = {"x.x", "x.y", "x.z", "x.w"};
    for (int i = 0; i < 4; ++i) {
      const int kk = 4 * q + i;
      if (kk >= kk_n) break;
      for (int m = 0; m < np; ++m) {
        const float c = coef(m, kk);
        if (c == 0.0f) continue;
        std::fprintf(f, "      acc[%d] = fmaf(%s, %s, acc[%d]);\n", m, lit(c).c_str(), comp[i], m);
      }
    }
    std::fprintf(f, "    }\n");
  }
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 2) {
    std::fprintf(stderr, "usage: %s <output header>\n", argv[0]);
    return 2;
  }
  FILE* f = std::fopen(argv[1], "w");
  if (!f) {
    std::perror(argv[1]);
    return 1;
  }
  std::fprintf(f,
               "// Generated at build time by gen_sref.cpp from build_ref(): the FP32 predictor's\n"
               "// reference-stiffness contractions with S^ as immediates.  Do not edit.\n"
               "#pragma once\n\nnamespace afe {\n\n"
               "template <int N>\nstruct SrefFP32;\n\n");
  for (int N = 1; N <= 3; ++N) {
    static afe::RefData r;
    if (!afe::build_ref(N, &r)) {
      std::fprintf(stderr, "build_ref(%d) failed\n", N);
      return 1;
    }
    const int np = r.Np, kk_n = 3 * np;
    double smax = 0.0;
    for (int d = 0; d < 3; ++d)
      for (int m = 0; m < np; ++m)
        for (int j = 0; j < np; ++j) smax = std::fmax(smax, std::fabs(r.S[d][m][j]));
    for (int d = 0; d < 3; ++d)
      for (int m = 0; m < np; ++m)
        for (int j = 0; j < np; ++j)
          if (std::fabs(r.S[d][m][j]) < 1e-13 * smax) r.S[d][m][j] = 0.0;
    int nz_p = 0, nz_v = 0;
    for (int d = 0; d < 3; ++d)
      for (int m = 0; m < np; ++m)
        for (int j = 0; j < np; ++j) {
          nz_p += (float)r.S[d][m][j] != 0.0f;
          nz_v += (float)r.S[d][j][m] != 0.0f;
        }
    std::fprintf(f, "// node order j = 0 .. Np-1 (barycentric multi-indices alpha_0 alpha_1 alpha_2 alpha_3):");
    for (int j = 0; j < np; ++j)
      std::fprintf(f, "%s %d%d%d%d", j % 10 == 0 ? "\n//" : "", r.alpha[j][0], r.alpha[j][1], r.alpha[j][2], r.alpha[j][3]);
    std::fprintf(f, "\ntemplate <>\nstruct SrefFP32<%d> {\n", N);
    std::fprintf(f, "  static constexpr int KK = %d;   // 3 Np pre-contracted values per column\n", kk_n);
    std::fprintf(f, "  static constexpr int KKS = %d;  // column stride in shared memory (floats)\n",
                 column_stride(kk_n));
    std::fprintf(f, "  static constexpr int kTerms = %d, kTermsT = %d;  // non-zero entries used\n", nz_p, nz_v);
    std::fprintf(f,
                 "  // acc[m] += sum_{d,j} S^_d[m][j] b[d Np + j]: the reference-stiffness contraction of\n"
                 "  // the predictor's right-hand side\n"
                 "  static __device__ __forceinline__ void contract(const float* __restrict__ b, float (&acc)[%d]) {\n",
                 np);
    emit_body(f, np, [&](int m, int kk) { return (float)r.S[kk / np][m][kk % np]; });
    std::fprintf(f, "  }\n");
    std::fprintf(f,
                 "  // acc[m] += sum_{d,j} S^_d[j][m] b[d Np + j]: the volume term's contraction\n"
                 "  static __device__ __forceinline__ void contract_t(const float* __restrict__ b, float (&acc)[%d]) {\n",
                 np);
    emit_body(f, np, [&](int m, int kk) { return (float)r.S[kk / np][kk % np][m]; });
    std::fprintf(f, "  }\n};\n\n");
  }
  std::fprintf(f, "}  // namespace afe\n");
  std::fclose(f);
  return 0;
}
