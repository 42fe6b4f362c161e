// C-ABI implementation (include/afe.h): mesh set-up, the step driver and host plumbing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "afe.h"
#include "kernels.cuh"
#include "predictor_f32.cuh"
#include "refelem.hpp"
#include "topology.hpp"

namespace {

thread_local std::string g_err;

// Named NVTX range around the host-side enqueue of a stage (visible to Nsight Systems and
// other NVTX tools, which correlate it with the kernels it launches; a no-op without a tool).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

afe_status fail(afe_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define AFE_CUDA(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return fail(AFE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

struct afe_mesh {
  afe_params p{};
  int bc = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int n_sm = 0;
  afe::RefData ref{};
  afe::Topology topo;
  afe::DevMesh dm{};
  afe::RefData* d_ref = nullptr;
  afe::Batch self{};  // this mesh as a batch of one (its DevMesh record is kept in step with dm)
  std::vector<void*> allocs;
  int64_t bytes = 0;
  void* scratch = nullptr;
  int64_t scratch_stride = 0;
  int pred_grid = 0;
  int f32_ok = 0;        // the shared-memory FP32 predictor is used
  int f32_tc = 0;        // ... with its M_i^-1 apply on tcgen05 / tensor memory (else mma.sync)
  int f32_tc_fits = 0;   // every cell fits the tensor-memory plan
  int variant = 0;       // 0: mma.sync apply, 1: tcgen05 / tensor memory where the cells fit
  afe_schedule sched{};  // predictor schedule (cost order, ring cap, narrow chunks; variant above)
  int32_t* d_order = nullptr;  // the cells in decreasing cost (allocated when first asked for)
  size_t f32_smem = 0;
  double* d_totals_partial = nullptr;
  double* d_totals = nullptr;
  int totals_blocks = 256;
  int diag = 0;
  int pending = 0;  // accumulated status of asynchronous steps
  int profiling = 0;
  int64_t launches = 0;
  std::vector<cudaEvent_t> ev;  // 5 events per profiled step
  size_t ev_used = 0;
  double t_host = 0;
  int64_t steps = 0;
  double last_dt = 0;

  template <typename T>
  afe_status alloc(T** ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) count = 1;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) return fail(AFE_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    allocs.push_back(p);
    bytes += (int64_t)(count * sizeof(T));
    *ptr = (T*)p;
    return AFE_OK;
  }
  template <typename T>
  afe_status upload(T** ptr, const std::vector<T>& v) {
    afe_status s = alloc(ptr, v.size());
    if (s != AFE_OK) return s;
    if (!v.empty()) AFE_CUDA(cudaMemcpy(*ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return AFE_OK;
  }
  ~afe_mesh() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (void* p : allocs) cudaFree(p);
  }
};

namespace {

#define AFE_TRY(x)                   \
  do {                               \
    afe_status s_ = (x);             \
    if (s_ != AFE_OK) return s_;     \
  } while (0)

// One launch sequence: the batch table plus what the launches need besides it.  A single
// mesh runs as a batch of one; the FP64 kernels (and the FP32 fall-backs for cells too large
// for shared memory) take the single mesh's record directly.
struct StepPlan {
  const afe::Batch* b = nullptr;
  cudaStream_t st = nullptr;
  int order = 1, fp32 = 0, limiter = 0, n_sm = 1, diag = 0;
  int f32_ok = 0, f32_tc = 0;
  size_t f32_smem = 0;
  const afe::RefData* d_ref = nullptr;
  afe_mesh* single = nullptr;  // nullptr for a batch (FP32 shared-memory kernels only)
  afe_mesh* prof = nullptr;    // stage events are recorded on this mesh when profiling
};

StepPlan plan_of(afe_mesh* m) {
  StepPlan P;
  P.b = &m->self;
  P.st = m->stream;
  P.order = m->p.order;
  P.fp32 = m->p.precision == AFE_FP32;
  P.limiter = m->p.limiter;
  P.n_sm = m->n_sm;
  P.diag = m->diag;
  P.f32_ok = m->f32_ok;
  P.f32_tc = m->f32_tc;
  P.f32_smem = m->f32_smem;
  P.d_ref = m->d_ref;
  P.single = m;
  P.prof = m;
  return P;
}

bool corrector_f32_fits(int Nmax) { return Nmax <= 2 * 4 * afe::kCorrThreads; }

template <int N, typename Real>
void launch_predictor(const StepPlan& P) {
  if constexpr (N <= 3) {  // the shared-memory FP32 predictor exists for N <= 3 (cells up to 640 nodes)
    if (sizeof(Real) == 4 && P.f32_ok) {
      if (P.f32_tc)
        afe::predictor_f32_kernel<N, true><<<P.n_sm, afe::kF32Threads, P.f32_smem, P.st>>>(*P.b, P.d_ref, P.diag,
                                                                                         (int)P.f32_smem);
      else
        afe::predictor_f32_kernel<N, false><<<P.n_sm, afe::kF32Threads, P.f32_smem, P.st>>>(*P.b, P.d_ref, P.diag,
                                                                                          (int)P.f32_smem);
      return;
    }
  }
  afe_mesh* m = P.single;
  afe::predictor_kernel<N, Real><<<m->pred_grid, 256, 0, P.st>>>(m->dm, m->d_ref, (Real*)m->scratch,
                                                                 m->scratch_stride, P.diag);
}

// Shared-memory plan of the FP32 predictor; cells too large for it use the global-scratch kernel.
// The M_i^-1 apply runs on mma.sync unless the handle asks for the tcgen05 / tensor-memory
// form and every cell fits that plan.
template <int N>
afe_status plan_f32(afe_mesh* m) {
  cudaFuncAttributes fa, fb;
  AFE_CUDA(cudaFuncGetAttributes(&fa, afe::predictor_f32_kernel<N, false>));
  AFE_CUDA(cudaFuncGetAttributes(&fb, afe::predictor_f32_kernel<N, true>));
  int optin = 0;
  AFE_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device));
  const size_t limit = (size_t)optin - std::max(fa.sharedSizeBytes, fb.sharedSizeBytes) - 1024;
  m->f32_ok = 0;
  m->f32_tc = 0;
  m->f32_tc_fits = 0;
  if (m->dm.Nmax > afe::predictor_f32_max_nodes(N)) return AFE_OK;
  const size_t need = afe::predictor_f32_smem(N, m->dm.Nmax, m->dm.Smax);
  if (need > limit) return AFE_OK;
  // all the shared memory the block may have: smaller cells get a deeper M_i^-1 ring
  const size_t b = limit / 128 * 128;
  m->f32_ok = 1;
  m->f32_smem = b;
  m->f32_tc_fits = afe::tc_cell_plan(N, b, m->dm.Smax, m->dm.Nmax).ok ? 1 : 0;
  m->f32_tc = (m->f32_tc_fits && m->variant == 1) ? 1 : 0;
  AFE_CUDA(cudaFuncSetAttribute(afe::predictor_f32_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)b));
  AFE_CUDA(cudaFuncSetAttribute(afe::predictor_f32_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)b));
  return AFE_OK;
}

template <int N, typename Real>
void launch_face(const StepPlan& P) {
  const int64_t threads = P.b->gpre[P.b->nh] * 32;
  const int blocks = (int)((threads + 255) / 256);
  if (blocks > 0) afe::face_kernel<N, Real><<<blocks, 256, 0, P.st>>>(*P.b);
}

template <int N, typename Real>
afe_status launch_corrector(const StepPlan& P) {
  if (sizeof(Real) == 4 && corrector_f32_fits(P.b->Nmax)) {
    const size_t smem = (size_t)P.b->Nmax * 10 * sizeof(float);
    if (smem > 48 * 1024)
      AFE_CUDA(cudaFuncSetAttribute(afe::corrector_f32_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    afe::corrector_f32_kernel<N><<<(unsigned)P.b->cpre[P.b->nh], afe::kCorrThreads, smem, P.st>>>(*P.b, P.d_ref);
    return AFE_OK;
  }
  afe_mesh* m = P.single;
  size_t smem = ((size_t)m->dm.Nmax * 5 * sizeof(Real) + 7) / 8 * 8;
  if (sizeof(Real) == 4) smem += (size_t)m->dm.Nmax * 5 * sizeof(double);
  // static + dynamic shared memory may exceed the 48 KB default: opt in to the size used
  AFE_CUDA(cudaFuncSetAttribute(afe::corrector_kernel<N, Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = (int)std::min<int64_t>(m->dm.C, (int64_t)m->n_sm * 4);
  afe::corrector_kernel<N, Real><<<grid, 256, smem, P.st>>>(m->dm, m->d_ref);
  return AFE_OK;
}

template <typename Real>
afe_status dispatch_stage(const StepPlan& P, int stage) {
  switch (P.order) {
    case 1:
      if (stage == 0) launch_predictor<1, Real>(P);
      else if (stage == 1) launch_face<1, Real>(P);
      else return launch_corrector<1, Real>(P);
      break;
    case 2:
      if (stage == 0) launch_predictor<2, Real>(P);
      else if (stage == 1) launch_face<2, Real>(P);
      else return launch_corrector<2, Real>(P);
      break;
    case 3:
      if (stage == 0) launch_predictor<3, Real>(P);
      else if (stage == 1) launch_face<3, Real>(P);
      else return launch_corrector<3, Real>(P);
      break;
    case 4:
      if (stage == 0) launch_predictor<4, Real>(P);
      else if (stage == 1) launch_face<4, Real>(P);
      else return launch_corrector<4, Real>(P);
      break;
    default:
      return fail(AFE_EINVAL, "order must be 1, 2, 3 or 4");
  }
  return AFE_OK;
}

afe_status stage(const StepPlan& P, int s) { return P.fp32 ? dispatch_stage<float>(P, s) : dispatch_stage<double>(P, s); }

// limiter (if on) and the time step, all on the device
afe_status enqueue_dt(const StepPlan& P, double dt) {
  const int64_t C = P.b->cpre[P.b->nh];
  if (P.limiter) {
    const int cgrid = (int)std::min<int64_t>(C, (int64_t)P.n_sm * 8);
    afe::cell_means_kernel<<<cgrid, 256, 0, P.st>>>(*P.b);
    afe::limiter_kernel<<<(int)((C + 127) / 128), 128, 0, P.st>>>(*P.b);
  }
  if (dt > 0) {
    afe::set_dt_kernel<<<1, 64, 0, P.st>>>(*P.b, dt);
  } else {
    afe::cfl_kernel<<<(int)((C * 32 + 255) / 256), 256, 0, P.st>>>(*P.b);
    afe::dt_finalize_kernel<<<1, 64, 0, P.st>>>(*P.b);
  }
  return AFE_OK;
}

afe_status record(const StepPlan& P) {
  afe_mesh* m = P.prof;
  if (!m || !m->profiling) return AFE_OK;
  if (m->ev_used >= m->ev.size()) {
    cudaEvent_t e;
    AFE_CUDA(cudaEventCreate(&e));
    m->ev.push_back(e);
  }
  AFE_CUDA(cudaEventRecord(m->ev[m->ev_used++], P.st));
  return AFE_OK;
}

// kernels per step: begin + [means + limiter] + (set_dt | cfl + finalize) + predictor + face
// + corrector + clock
int launches_per_step(const StepPlan& P, double dt) { return 1 + (P.limiter ? 2 : 0) + (dt > 0 ? 1 : 2) + 3 + 1; }

afe_status enqueue_step(const StepPlan& P, double dt) {
  NvtxRange step_range("afe step");
  afe::step_begin_kernel<<<1, 64, 0, P.st>>>(*P.b);
  AFE_TRY(record(P));
  {
    NvtxRange r("afe limiter + time step");
    AFE_TRY(enqueue_dt(P, dt));
  }
  AFE_TRY(record(P));
  {
    NvtxRange r("afe predictor");
    AFE_TRY(stage(P, 0));
  }
  AFE_TRY(record(P));
  {
    NvtxRange r("afe face fluxes");
    AFE_TRY(stage(P, 1));
  }
  AFE_TRY(record(P));
  {
    NvtxRange r("afe corrector");
    AFE_TRY(stage(P, 2));
  }
  AFE_TRY(record(P));
  afe::advance_time_kernel<<<1, 64, 0, P.st>>>(*P.b);
  AFE_CUDA(cudaGetLastError());
  return AFE_OK;
}

afe_status enqueue_step(afe_mesh* m, double dt) {
  const StepPlan P = plan_of(m);
  m->launches += launches_per_step(P, dt);
  return enqueue_step(P, dt);
}

afe_status read_flags(afe_mesh* m, int* flags) {
  AFE_CUDA(cudaMemcpyAsync(flags, m->dm.flags, afe::F_COUNT * sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  AFE_CUDA(cudaStreamSynchronize(m->stream));
  return AFE_OK;
}

afe_status status_of(const int* flags) {
  if (flags[afe::F_TIMEOUT]) return fail(AFE_ETIMEOUT, "a bounded wait on an asynchronous copy gave up");
  if (flags[afe::F_NONFINITE]) return fail(AFE_ENONFINITE, "non-finite or inadmissible state (flags " +
                                                               std::to_string(flags[afe::F_NONFINITE]) + ")");
  if (flags[afe::F_NONCONV])
    return fail(AFE_ENOCONV, std::to_string(flags[afe::F_NONCONV]) + " cells hit picard_max");
  return AFE_OK;
}

// Refreshes the batch-of-one record read by the batch-aware kernels.
void sync_self(afe_mesh* m) {
  afe::Batch& b = m->self;
  b.ring_cap = m->sched.ring_cap;
  b.narrow = m->sched.narrow;
  b.order = m->sched.cost_order ? m->d_order : nullptr;
  b.nh = 1;
  b.Nmax = m->topo.Nmax;
  b.Smax = m->topo.Smax;
  b.work = m->dm.work;
  b.cpre[0] = 0;
  b.cpre[1] = m->topo.C;
  b.gpre[0] = 0;
  b.gpre[1] = m->topo.n_groups;
  b.tab[0] = m->dm;
}

afe_status check_params(const afe_params* p) {
  if (!p) return fail(AFE_EINVAL, "params is NULL");
  if (p->order < 1 || p->order > 4) return fail(AFE_EINVAL, "order must be 1, 2, 3 or 4");
  if (p->precision != AFE_FP64 && p->precision != AFE_FP32) return fail(AFE_EINVAL, "unknown precision");
  if (p->equations != AFE_EULER && p->equations != AFE_NAVIER_STOKES) return fail(AFE_EINVAL, "unknown equations");
  if (!(p->gamma > 1.0) || !(p->R > 0.0) || !(p->cfl > 0.0) || !(p->picard_tol > 0.0) || p->picard_max < 1)
    return fail(AFE_EINVAL, "gamma > 1, R > 0, cfl > 0, picard_tol > 0 and picard_max >= 1 are required");
  if (p->mu < 0.0) return fail(AFE_EINVAL, "mu must be >= 0");
  if (p->visc_dt_subtet != 0 && p->visc_dt_subtet != 1) return fail(AFE_EINVAL, "visc_dt_subtet must be 0 or 1");
  if (p->h_diameter != 0 && p->h_diameter != 1) return fail(AFE_EINVAL, "h_diameter must be 0 or 1");
  if (p->kappa < 0.0 && !(p->Pr > 0.0)) return fail(AFE_EINVAL, "Pr > 0 is required when kappa < 0");
  return AFE_OK;
}

afe_status check_schedule(const afe_schedule* s) {
  if (!s) return fail(AFE_EINVAL, "schedule is NULL");
  if ((s->cost_order != 0 && s->cost_order != 1) || (s->variant != 0 && s->variant != 1) ||
      (s->narrow != 0 && s->narrow != 1) || s->ring_cap < 0 || s->ring_cap > afe::kF32MaxStages)
    return fail(AFE_EINVAL, "schedule: cost_order, variant and narrow are 0 or 1, ring_cap 0..8");
  return AFE_OK;
}

// Estimated flops of one fixed-point iteration of a cell (the stiffness contraction and the
// M_i^-1 apply dominate).
double cell_cost(int N, int64_t Ni, int64_t S) {
  const double Np = (N + 1) * (N + 2) * (N + 3) / 6, Nt = N + 1;
  return (double)S * Nt * Np * (155.0 + 30.0 * Np) + 10.0 * Nt * (double)Ni * (double)Ni;
}

// Global cells of the given topologies (concatenated in order) sorted by decreasing cost;
// equal costs keep index order.
std::vector<int32_t> cost_order(const std::vector<const afe::Topology*>& tops, int N) {
  std::vector<std::pair<double, int32_t>> v;
  int64_t base = 0;
  for (const afe::Topology* t : tops) {
    for (int64_t c = 0; c < t->C; ++c)
      v.push_back({cell_cost(N, t->node_ptr[c + 1] - t->node_ptr[c], t->sub_ptr[c + 1] - t->sub_ptr[c]),
                   (int32_t)(base + c)});
    base += t->C;
  }
  std::stable_sort(v.begin(), v.end(), [](const std::pair<double, int32_t>& a, const std::pair<double, int32_t>& b) {
    return a.first > b.first;
  });
  std::vector<int32_t> out(v.size());
  for (size_t i = 0; i < v.size(); ++i) out[i] = v[i].second;
  return out;
}

// Signature of a set of meshes for the autotuner's memory: order, and per mesh its cell count
// and an FNV-1a hash of the cells' node and sub-tet counts.
std::string mesh_signature(const std::vector<const afe::Topology*>& tops, int N) {
  std::string sig = "N" + std::to_string(N);
  for (const afe::Topology* t : tops) {
    uint64_t h = 1469598103934665603ull;
    for (int64_t c = 0; c < t->C; ++c) {
      const uint64_t a = (uint64_t)(t->node_ptr[c + 1] - t->node_ptr[c]), b = (uint64_t)(t->sub_ptr[c + 1] - t->sub_ptr[c]);
      h = (h ^ a) * 1099511628211ull;
      h = (h ^ b) * 1099511628211ull;
    }
    sig += "|" + std::to_string(t->C) + ":" + std::to_string(h);
  }
  return sig;
}

std::mutex g_tune_mutex;
std::map<std::string, afe_schedule> g_tune_cache;

}  // namespace

extern "C" {

const char* afe_last_error(void) { return g_err.c_str(); }

afe_status afe_default_params(afe_params* p, int order) {
  if (!p) return fail(AFE_EINVAL, "params is NULL");
  std::memset(p, 0, sizeof(*p));
  p->order = order;
  p->equations = AFE_EULER;
  p->precision = AFE_FP64;
  p->gamma = 1.4;
  p->R = 1.0;
  p->mu = 0.0;
  p->Pr = 0.71;
  p->kappa = 0.0;
  p->cfl = 0.3;
  p->limiter = 0;
  p->m1 = 0.1;
  p->picard_tol = 1e-12;
  p->picard_max = 64;
  p->period[0] = p->period[1] = p->period[2] = 1.0;
  return (order >= 1 && order <= 4) ? AFE_OK : fail(AFE_EINVAL, "order must be 1, 2, 3 or 4");
}

afe_status afe_mesh_create(const afe_params* p, int64_t n_vertices, const double* xyz, int64_t n_cells,
                           const int64_t* cell_subtet_ptr, const int64_t* subtet_vtx, const int8_t* subtet_shift,
                           int boundary, void* cuda_stream, afe_mesh** out) {
  if (!out) return fail(AFE_EINVAL, "out is NULL");
  *out = nullptr;
  AFE_TRY(check_params(p));
  if (!xyz || !cell_subtet_ptr || !subtet_vtx || n_vertices <= 0 || n_cells <= 0)
    return fail(AFE_EINVAL, "mesh arrays must be non-NULL and non-empty");
  if (boundary != AFE_BC_PERIODIC && boundary != AFE_BC_TRANSMISSIVE) return fail(AFE_EINVAL, "unknown boundary");
  if (boundary == AFE_BC_PERIODIC && subtet_shift)
    for (int d = 0; d < 3; ++d)
      if (!(p->period[d] > 0.0)) return fail(AFE_EINVAL, "period must be > 0 with image shifts");

  std::unique_ptr<afe_mesh> m(new afe_mesh());
  m->p = *p;
  m->bc = boundary;
  m->stream = (cudaStream_t)cuda_stream;
  if (!afe::build_ref(p->order, &m->ref)) return fail(AFE_EINVAL, "reference element build failed");
  {
    std::string err;
    double period[3] = {p->period[0], p->period[1], p->period[2]};
    if (!subtet_shift) period[0] = period[1] = period[2] = 0.0;
    int rc = afe::build_topology(m->ref, n_vertices, xyz, n_cells, cell_subtet_ptr, subtet_vtx, subtet_shift, period,
                                 boundary == AFE_BC_PERIODIC, &m->topo, &err);
    if (rc) return fail(rc == 2 ? AFE_EMESH : AFE_EINVAL, err);
  }

  // ---- GPU part
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(AFE_ECUDA, "no CUDA device");
  AFE_CUDA(cudaGetDevice(&m->device));
  AFE_CUDA(cudaDeviceGetAttribute(&m->n_sm, cudaDevAttrMultiProcessorCount, m->device));
  const afe::Topology& T = m->topo;
  afe::DevMesh& d = m->dm;
  d.N = p->order;
  d.C = T.C;
  d.n_nodes = T.n_nodes;
  d.n_slots = T.n_slots;
  d.n_groups = T.n_groups;
  d.Nmax = T.Nmax;
  d.Smax = T.Smax;
  d.gamma = p->gamma;
  d.Rgas = p->R;
  d.cv = p->R / (p->gamma - 1.0);
  d.cfl = p->cfl;
  d.m1 = p->m1;
  d.mu0 = (p->equations == AFE_NAVIER_STOKES) ? p->mu : 0.0;
  d.Pr = p->Pr;
  d.kappa0 = (p->equations == AFE_NAVIER_STOKES) ? p->kappa : (p->kappa < 0 ? 0.0 : p->kappa);
  d.tol = p->picard_tol;
  // the characteristic length h_i (Sec. 4.2): insphere-equivalent diameter or the diameter
  const std::vector<double>& hcell = p->h_diameter ? T.cell_diam : T.cell_h;
  d.h_min = p->h_diameter ? *std::min_element(hcell.begin(), hcell.end()) : T.h_min;
  d.picard_max = p->picard_max;
  d.limiter = p->limiter;
  d.eq = p->equations;
  d.first_wait_polls = afe::kWaitPolls;
  afe_mesh* M = m.get();
  AFE_TRY(M->upload((int64_t**)&d.node_ptr, T.node_ptr));
  AFE_TRY(M->upload((int64_t**)&d.sub_ptr, T.sub_ptr));
  AFE_TRY(M->upload((int64_t**)&d.slot_ptr, T.slot_ptr));
  AFE_TRY(M->upload((int64_t**)&d.minv_ptr, T.minv_ptr));
  AFE_TRY(M->upload((uint16_t**)&d.A, T.A));
  AFE_TRY(M->upload((double**)&d.geo, T.geo));
  AFE_TRY(M->upload((int64_t**)&d.inc_ptr, T.inc_ptr));
  AFE_TRY(M->upload((uint32_t**)&d.inc, T.inc));
  AFE_TRY(M->upload((int32_t**)&d.slot_cell, T.slot_cell));
  AFE_TRY(M->upload((uint16_t**)&d.slot_sub, T.slot_sub));
  AFE_TRY(M->upload((uint8_t**)&d.slot_loc, T.slot_loc));
  AFE_TRY(M->upload((uint16_t**)&d.slot_node, T.slot_node));
  AFE_TRY(M->upload((double**)&d.slot_geo, T.slot_geo));
  AFE_TRY(M->upload((int64_t**)&d.slot_partner, T.slot_partner));
  AFE_TRY(M->upload((int32_t**)&d.slot_nbr, T.slot_nbr));
  AFE_TRY(M->upload((int64_t**)&d.finc_ptr, T.finc_ptr));
  AFE_TRY(M->upload((uint32_t**)&d.finc, T.finc));
  AFE_TRY(M->upload((int64_t**)&d.group_ptr, T.group_ptr));
  AFE_TRY(M->upload((int64_t**)&d.group_slot, T.group_slot));
  AFE_TRY(M->upload((double**)&d.cell_vol, T.cell_vol));
  AFE_TRY(M->upload((double**)&d.cell_h, hcell));
  if (p->visc_dt_subtet) AFE_TRY(M->upload((double**)&d.cell_hv, T.cell_hsub));
  else d.cell_hv = d.cell_h;
  AFE_TRY(M->alloc(&d.wvec, T.n_nodes));
  const int64_t nminv = T.minv_ptr[T.C];
  AFE_TRY(M->alloc(&d.minv64, nminv));
  if (p->precision == AFE_FP32) AFE_TRY(M->alloc(&d.minv32, nminv));
  AFE_TRY(M->alloc(&d.u, T.n_nodes * 5));
  const size_t rb = p->precision == AFE_FP32 ? 4 : 8;
  {
    void* v;
    AFE_TRY(M->alloc((char**)&v, T.n_nodes * 5 * rb));
    d.vol = v;
    AFE_TRY(M->alloc((char**)&v, T.n_slots * T.Nf * 5 * rb));
    d.slot_q = v;
    AFE_TRY(M->alloc((char**)&v, T.n_slots * T.Nf * 5 * rb));
    d.slot_fn = v;
    AFE_TRY(M->alloc((char**)&v, T.n_slots * T.Nf * 5 * rb));
    d.slot_G = v;
  }
  AFE_TRY(M->alloc(&d.iters, T.C));
  AFE_TRY(M->alloc(&d.beta, T.C));
  AFE_TRY(M->alloc(&d.mu, T.C));
  AFE_TRY(M->alloc(&d.means, T.C * 5));
  AFE_TRY(M->alloc(&d.dt, 1));
  AFE_TRY(M->alloc(&d.tacc, 1));
  AFE_TRY(M->alloc(&d.maxbits, 1));
  AFE_TRY(M->alloc(&d.flags, afe::F_COUNT));
  AFE_TRY(M->alloc(&d.work, 1));
  AFE_TRY(M->alloc(&M->d_ref, 1));

  AFE_TRY(M->alloc(&M->d_totals_partial, (size_t)M->totals_blocks * 5));
  AFE_TRY(M->alloc(&M->d_totals, 5));
  AFE_CUDA(cudaMemcpy(M->d_ref, &M->ref, sizeof(afe::RefData), cudaMemcpyHostToDevice));
  AFE_CUDA(cudaMemset(d.u, 0, T.n_nodes * 5 * sizeof(double)));
  AFE_CUDA(cudaMemset(d.beta, 0, T.C * sizeof(double)));
  AFE_CUDA(cudaMemset(d.tacc, 0, sizeof(double)));
  AFE_CUDA(cudaMemset(d.iters, 0, T.C * sizeof(int32_t)));
  {
    std::vector<double> mu0(T.C, d.mu0);
    AFE_CUDA(cudaMemcpy(d.mu, mu0.data(), T.C * sizeof(double), cudaMemcpyHostToDevice));
  }
  if (p->precision == AFE_FP32) {
    const int blocks = (int)((T.T + 255) / 256);
    switch (p->order) {
      case 1:
        AFE_TRY(M->alloc(&d.sub32, (size_t)T.T * afe::f32_rec_bytes(1)));
        afe::sub32_kernel<1><<<blocks, 256, 0, M->stream>>>(d, T.T);
        AFE_TRY(plan_f32<1>(M));
        break;
      case 2:
        AFE_TRY(M->alloc(&d.sub32, (size_t)T.T * afe::f32_rec_bytes(2)));
        afe::sub32_kernel<2><<<blocks, 256, 0, M->stream>>>(d, T.T);
        AFE_TRY(plan_f32<2>(M));
        break;
      case 3:
        AFE_TRY(M->alloc(&d.sub32, (size_t)T.T * afe::f32_rec_bytes(3)));
        afe::sub32_kernel<3><<<blocks, 256, 0, M->stream>>>(d, T.T);
        AFE_TRY(plan_f32<3>(M));
        break;
      default:  // N = 4: the cells (about 1,100 nodes) exceed the shared-memory plan: the
        break;  // global-scratch FP32 kernels run, which need no packed records
    }
  }
  // predictor scratch (persistent grid, one slice per block)
  {
    const int64_t per = (int64_t)T.Nmax * T.Nt * 5 * 3 + (int64_t)T.Smax * T.Nt * T.Np * 5 * 4;
    M->scratch_stride = (per + 31) / 32 * 32;
    M->pred_grid = (int)std::min<int64_t>(T.C, (int64_t)M->n_sm * 2);
    if (!(p->precision == AFE_FP32 && M->f32_ok)) {  // the shared-memory FP32 kernel needs none
      void* s;
      AFE_TRY(M->alloc((char**)&s, (size_t)M->scratch_stride * M->pred_grid * rb));
      M->scratch = s;
    }
  }
  // FP64 set-up on the GPU: mass matrices, w_i, inverses
  NvtxRange setup_range("afe set-up: mass matrices and inverses");
  AFE_CUDA(cudaMemsetAsync(d.flags, 0, afe::F_COUNT * sizeof(int), M->stream));
  const int sgrid = (int)std::min<int64_t>(T.C, (int64_t)M->n_sm * 4);
  afe::assemble_mass_kernel<<<sgrid, 256, 0, M->stream>>>(d, M->d_ref);
  afe::invert_spd_kernel<<<(int)std::min<int64_t>(T.C, (int64_t)M->n_sm * 4), 256, 0, M->stream>>>(d);
  afe::symmetrize_kernel<<<sgrid, 256, 0, M->stream>>>(d, p->precision == AFE_FP32);
  AFE_CUDA(cudaGetLastError());
  int flags[afe::F_COUNT];
  AFE_TRY(read_flags(M, flags));
  if (flags[afe::F_NONFINITE]) return fail(AFE_EMESH, "a cell mass matrix is not positive definite");
  if (p->precision == AFE_FP32) {
    // only the FP32 copy is used by the reduced-precision step
    for (size_t i = 0; i < M->allocs.size(); ++i)
      if (M->allocs[i] == d.minv64) {
        cudaFree(d.minv64);
        M->allocs.erase(M->allocs.begin() + i);
        M->bytes -= nminv * 8;
        d.minv64 = nullptr;
        break;
      }
  }
  sync_self(M);
  *out = m.release();
  return AFE_OK;
}

afe_status afe_mesh_validate(const afe_params* p, int64_t n_vertices, const double* xyz, int64_t n_cells,
                             const int64_t* cell_subtet_ptr, const int64_t* subtet_vtx, const int8_t* subtet_shift,
                             int boundary, int64_t* n_nodes, int64_t* n_face_tris) {
  AFE_TRY(check_params(p));
  if (!xyz || !cell_subtet_ptr || !subtet_vtx || n_vertices <= 0 || n_cells <= 0)
    return fail(AFE_EINVAL, "mesh arrays must be non-NULL and non-empty");
  if (boundary != AFE_BC_PERIODIC && boundary != AFE_BC_TRANSMISSIVE) return fail(AFE_EINVAL, "unknown boundary");
  afe::RefData ref;
  if (!afe::build_ref(p->order, &ref)) return fail(AFE_EINVAL, "reference element build failed");
  afe::Topology topo;
  std::string err;
  double period[3] = {p->period[0], p->period[1], p->period[2]};
  if (!subtet_shift) period[0] = period[1] = period[2] = 0.0;
  int rc = afe::build_topology(ref, n_vertices, xyz, n_cells, cell_subtet_ptr, subtet_vtx, subtet_shift, period,
                               boundary == AFE_BC_PERIODIC, &topo, &err);
  if (rc) return fail(rc == 2 ? AFE_EMESH : AFE_EINVAL, err);
  if (n_nodes) *n_nodes = topo.n_nodes;
  if (n_face_tris) *n_face_tris = topo.n_slots;
  return AFE_OK;
}

void afe_mesh_destroy(afe_mesh* m) {
  if (!m) return;
  if (m->stream) cudaStreamSynchronize(m->stream);
  else cudaDeviceSynchronize();
  delete m;
}

afe_status afe_num_nodes(const afe_mesh* m, int64_t* n_nodes, int64_t* node_ptr) {
  if (!m || !n_nodes) return fail(AFE_EINVAL, "NULL argument");
  *n_nodes = m->topo.n_nodes;
  if (node_ptr) std::memcpy(node_ptr, m->topo.node_ptr.data(), (m->topo.C + 1) * sizeof(int64_t));
  return AFE_OK;
}

afe_status afe_get_node_coords(const afe_mesh* m, double* xyz) {
  if (!m || !xyz) return fail(AFE_EINVAL, "NULL argument");
  std::memcpy(xyz, m->topo.node_xyz.data(), m->topo.node_xyz.size() * sizeof(double));
  return AFE_OK;
}

afe_status afe_set_stream(afe_mesh* m, void* s) {
  if (!m) return fail(AFE_EINVAL, "NULL mesh");
  m->stream = (cudaStream_t)s;
  return AFE_OK;
}

afe_status afe_set_state(afe_mesh* m, const double* q) {
  if (!m || !q) return fail(AFE_EINVAL, "NULL argument");
  AFE_CUDA(cudaStreamSynchronize(m->stream));
  AFE_CUDA(cudaMemcpy(m->dm.u, q, m->topo.n_nodes * 5 * sizeof(double), cudaMemcpyHostToDevice));
  return AFE_OK;
}

afe_status afe_set_state_device(afe_mesh* m, const double* dq, void* s) {
  if (!m || !dq) return fail(AFE_EINVAL, "NULL argument");
  cudaStream_t st = s ? (cudaStream_t)s : m->stream;
  AFE_CUDA(cudaMemcpyAsync(m->dm.u, dq, m->topo.n_nodes * 5 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (st != m->stream) AFE_CUDA(cudaStreamSynchronize(st));
  return AFE_OK;
}

afe_status afe_get_state(const afe_mesh* m, double* q) {
  if (!m || !q) return fail(AFE_EINVAL, "NULL argument");
  AFE_CUDA(cudaStreamSynchronize(m->stream));
  AFE_CUDA(cudaMemcpy(q, m->dm.u, m->topo.n_nodes * 5 * sizeof(double), cudaMemcpyDeviceToHost));
  return AFE_OK;
}

afe_status afe_get_state_device(const afe_mesh* m, double* dq) {
  if (!m || !dq) return fail(AFE_EINVAL, "NULL argument");
  AFE_CUDA(cudaMemcpyAsync(dq, m->dm.u, m->topo.n_nodes * 5 * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
  return AFE_OK;
}

afe_status afe_compute_dt(afe_mesh* m, double* dt) {
  if (!m || !dt) return fail(AFE_EINVAL, "NULL argument");
  const StepPlan P = plan_of(m);
  afe::flags_clear_kernel<<<1, 64, 0, P.st>>>(*P.b);
  afe::step_begin_kernel<<<1, 64, 0, P.st>>>(*P.b);
  AFE_TRY(enqueue_dt(P, -1.0));
  AFE_CUDA(cudaMemcpyAsync(dt, m->dm.dt, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  int flags[afe::F_COUNT];
  AFE_TRY(read_flags(m, flags));
  return status_of(flags);
}

afe_status afe_cfl_pieces(afe_mesh* m, int64_t n_cells, double* bracket_max, double* h_min) {
  if (!m || !bracket_max || !h_min) return fail(AFE_EINVAL, "NULL argument");
  if (n_cells < 1 || n_cells > m->topo.C) return fail(AFE_EINVAL, "n_cells must be in 1..cells of the handle");
  const StepPlan P = plan_of(m);
  afe::flags_clear_kernel<<<1, 64, 0, P.st>>>(*P.b);
  afe::step_begin_kernel<<<1, 64, 0, P.st>>>(*P.b);
  if (P.limiter) {  // the viscosity of every cell of the handle
    const int64_t C = m->topo.C;
    afe::cell_means_kernel<<<(int)std::min<int64_t>(C, (int64_t)P.n_sm * 8), 256, 0, P.st>>>(*P.b);
    afe::limiter_kernel<<<(int)((C + 127) / 128), 128, 0, P.st>>>(*P.b);
  }
  afe::Batch sub = m->self;  // the bracket over the first n_cells cells only
  sub.cpre[1] = n_cells;
  afe::cfl_kernel<<<(int)((n_cells * 32 + 255) / 256), 256, 0, P.st>>>(sub);
  AFE_CUDA(cudaGetLastError());
  unsigned long long bits = 0;
  AFE_CUDA(cudaMemcpyAsync(&bits, m->dm.maxbits, sizeof(bits), cudaMemcpyDeviceToHost, m->stream));
  int flags[afe::F_COUNT];
  AFE_TRY(read_flags(m, flags));
  double bm;
  std::memcpy(&bm, &bits, sizeof(bm));
  *bracket_max = bm;
  const std::vector<double>& hc = m->p.h_diameter ? m->topo.cell_diam : m->topo.cell_h;
  *h_min = *std::min_element(hc.begin(), hc.begin() + n_cells);
  return status_of(flags);
}

afe_status afe_step(afe_mesh* m, double dt) {
  if (!m) return fail(AFE_EINVAL, "NULL mesh");
  afe::flags_clear_kernel<<<1, 64, 0, m->stream>>>(m->self);
  m->launches += 1;
  AFE_TRY(enqueue_step(m, dt));
  int flags[afe::F_COUNT];
  double hdt = 0;
  AFE_CUDA(cudaMemcpyAsync(&hdt, m->dm.dt, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  AFE_TRY(read_flags(m, flags));
  m->last_dt = hdt;
  m->t_host += hdt;
  m->steps += 1;
  return status_of(flags);
}

afe_status afe_step_async(afe_mesh* m, double dt, int nsteps) {
  if (!m || nsteps < 0) return fail(AFE_EINVAL, "bad argument");
  if (m->pending == 0 && nsteps > 0) {  // a new series: its status starts clean
    afe::flags_clear_kernel<<<1, 64, 0, m->stream>>>(m->self);
    m->launches += 1;
  }
  for (int i = 0; i < nsteps; ++i) {
    AFE_TRY(enqueue_step(m, dt));
    // fold this step's flags into the pending status without a host round trip
    m->steps += 1;
  }
  m->pending += nsteps;
  return AFE_OK;
}

afe_status afe_sync(afe_mesh* m) {
  if (!m) return fail(AFE_EINVAL, "NULL mesh");
  int flags[afe::F_COUNT];
  double hdt = 0, ht = 0;
  AFE_CUDA(cudaMemcpyAsync(&hdt, m->dm.dt, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  AFE_CUDA(cudaMemcpyAsync(&ht, m->dm.tacc, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  AFE_TRY(read_flags(m, flags));
  m->last_dt = hdt;
  m->t_host = ht;
  m->pending = 0;
  return status_of(flags);
}

afe_status afe_get_stats(const afe_mesh* mc, afe_stats* s) {
  afe_mesh* m = const_cast<afe_mesh*>(mc);
  if (!m || !s) return fail(AFE_EINVAL, "NULL argument");
  std::memset(s, 0, sizeof(*s));
  std::vector<int32_t> it(m->topo.C);
  int flags[afe::F_COUNT];
  afe::totals_partial_kernel<<<m->totals_blocks, 256, 0, m->stream>>>(m->dm, m->d_totals_partial);
  afe::totals_final_kernel<<<1, 32, 0, m->stream>>>(m->d_totals_partial, m->totals_blocks, m->d_totals);
  AFE_CUDA(cudaGetLastError());
  AFE_CUDA(cudaMemcpyAsync(it.data(), m->dm.iters, m->topo.C * sizeof(int32_t), cudaMemcpyDeviceToHost, m->stream));
  AFE_CUDA(cudaMemcpyAsync(s->totals, m->d_totals, 5 * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  double ht = 0;
  AFE_CUDA(cudaMemcpyAsync(&ht, m->dm.tacc, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  AFE_CUDA(cudaMemcpyAsync(&s->dt, m->dm.dt, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  AFE_TRY(read_flags(m, flags));
  s->t = ht;
  s->steps = m->steps;
  int64_t sum = 0;
  int32_t mx = 0;
  for (int32_t v : it) {
    sum += v;
    mx = std::max(mx, v);
  }
  s->picard_mean = (double)sum / (double)m->topo.C;
  s->picard_max = mx;
  s->nonconverged = flags[afe::F_NONCONV];
  s->troubled = flags[afe::F_TROUBLED];
  s->kernel_launches = m->launches;
  return AFE_OK;
}

afe_status afe_set_diagnostics(afe_mesh* m, int on) {
  if (!m) return fail(AFE_EINVAL, "NULL mesh");
  if (on && !m->dm.qbar_diag) {
    AFE_CUDA(cudaStreamSynchronize(m->stream));
    AFE_TRY(m->alloc(&m->dm.qbar_diag, m->topo.n_nodes * 5));
    sync_self(m);
  }
  m->diag = on ? 1 : 0;
  return AFE_OK;
}

afe_status afe_get_diagnostics(const afe_mesh* m, double* qbar, int32_t* iterations, double* beta, double* mu) {
  if (!m) return fail(AFE_EINVAL, "NULL mesh");
  AFE_CUDA(cudaStreamSynchronize(m->stream));
  if (qbar) {
    if (!m->dm.qbar_diag) return fail(AFE_EINVAL, "diagnostics were not enabled");
    AFE_CUDA(cudaMemcpy(qbar, m->dm.qbar_diag, m->topo.n_nodes * 5 * sizeof(double), cudaMemcpyDeviceToHost));
  }
  if (iterations) AFE_CUDA(cudaMemcpy(iterations, m->dm.iters, m->topo.C * sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (beta) AFE_CUDA(cudaMemcpy(beta, m->dm.beta, m->topo.C * sizeof(double), cudaMemcpyDeviceToHost));
  if (mu) AFE_CUDA(cudaMemcpy(mu, m->dm.mu, m->topo.C * sizeof(double), cudaMemcpyDeviceToHost));
  return AFE_OK;
}

afe_status afe_set_profiling(afe_mesh* m, int on) {
  if (!m) return fail(AFE_EINVAL, "NULL mesh");
  m->profiling = on ? 1 : 0;
  return AFE_OK;
}

afe_status afe_stage_times(afe_mesh* m, double* ms, int64_t* nsteps, int reset) {
  if (!m || !ms) return fail(AFE_EINVAL, "NULL argument");
  AFE_CUDA(cudaStreamSynchronize(m->stream));
  for (int s = 0; s < 4; ++s) ms[s] = 0.0;
  const size_t n = m->ev_used / 5;
  for (size_t i = 0; i < n; ++i)
    for (int s = 0; s < 4; ++s) {
      float t = 0.f;
      AFE_CUDA(cudaEventElapsedTime(&t, m->ev[i * 5 + s], m->ev[i * 5 + s + 1]));
      ms[s] += t;
    }
  if (nsteps) *nsteps = (int64_t)n;
  if (reset) m->ev_used = 0;
  return AFE_OK;
}

afe_status afe_plan_info(const afe_mesh* m, afe_plan* out) {
  if (!m || !out) return fail(AFE_EINVAL, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  const afe::Topology& T = m->topo;
  const int N = m->p.order;
  const bool fp32 = m->p.precision == AFE_FP32;
  out->max_nodes = T.Nmax;
  out->max_subtets = T.Smax;
  out->fp32_shared = (fp32 && m->f32_ok) ? 1 : 0;
  out->corrector_block = (fp32 && corrector_f32_fits(T.Nmax)) ? 1 : 0;
  if (!out->fp32_shared) return AFE_OK;
  out->smem_bytes = (int64_t)m->f32_smem;
  out->tcgen05 = m->f32_tc;
  int rmin = afe::kF32MaxStages, rmax = 0, hmin = afe::kF32Rows;
  for (int64_t c = 0; c < T.C; ++c) {
    const int Ni = (int)(T.node_ptr[c + 1] - T.node_ptr[c]);
    bool wide;
    int ns, rows;
    if (m->f32_tc) {
      const afe::TcCellPlan P = afe::tc_cell_plan(N, m->f32_smem, T.Smax, Ni);
      wide = P.wide;
      ns = P.nstage;
      rows = P.rows;
    } else {
      const afe::F32CellPlan P = afe::f32_cell_plan(N, m->f32_smem, T.Smax, Ni);
      wide = P.wide;
      ns = P.nstage;
      rows = afe::kF32Rows;
    }
    rmin = std::min(rmin, ns);
    rmax = std::max(rmax, ns);
    hmin = std::min(hmin, rows);
    if (afe::f32_ntp(N) == 4 && !wide) out->narrow_cells += 1;
    if (Ni % rows) out->masked_cells += 1;
  }
  out->ring_min = rmin;
  out->ring_max = rmax;
  out->stage_rows_min = hmin;
  return AFE_OK;
}

afe_status afe_set_schedule(afe_mesh* m, const afe_schedule* s) {
  if (!m) return fail(AFE_EINVAL, "NULL mesh");
  AFE_TRY(check_schedule(s));
  if (s->variant == 1 && m->p.precision == AFE_FP32 && !(m->f32_ok && m->f32_tc_fits))
    return fail(AFE_EINVAL, "the cells do not fit the tensor-memory plan of the FP32 predictor");
  AFE_CUDA(cudaStreamSynchronize(m->stream));
  if (s->cost_order && !m->d_order) {
    const std::vector<int32_t> ord = cost_order({&m->topo}, m->p.order);
    AFE_TRY(m->upload(&m->d_order, ord));
  }
  m->sched = *s;
  m->variant = s->variant;
  m->f32_tc = (m->f32_ok && m->f32_tc_fits && s->variant == 1) ? 1 : 0;
  sync_self(m);
  return AFE_OK;
}

afe_status afe_get_schedule(const afe_mesh* m, afe_schedule* s) {
  if (!m || !s) return fail(AFE_EINVAL, "NULL argument");
  *s = m->sched;
  s->variant = m->variant;
  return AFE_OK;
}

afe_status afe_set_predictor_variant(afe_mesh* m, int32_t variant) {
  if (!m) return fail(AFE_EINVAL, "NULL mesh");
  if (variant != 0 && variant != 1) return fail(AFE_EINVAL, "variant must be 0 (mma.sync) or 1 (tcgen05)");
  if (variant == 1 && m->p.precision == AFE_FP32 && !(m->f32_ok && m->f32_tc_fits))
    return fail(AFE_EINVAL, "the cells do not fit the tensor-memory plan of the FP32 predictor");
  m->variant = variant;
  m->sched.variant = variant;
  m->f32_tc = (m->f32_ok && m->f32_tc_fits && variant == 1) ? 1 : 0;
  return AFE_OK;
}

afe_status afe_set_wait_limit(afe_mesh* m, int32_t polls) {
  if (!m) return fail(AFE_EINVAL, "NULL mesh");
  if (polls < 0) return fail(AFE_EINVAL, "polls must be >= 0");
  AFE_CUDA(cudaStreamSynchronize(m->stream));
  m->dm.first_wait_polls = polls;
  sync_self(m);
  return AFE_OK;
}

afe_status afe_device_bytes(const afe_mesh* m, int64_t* bytes) {
  if (!m || !bytes) return fail(AFE_EINVAL, "NULL argument");
  *bytes = m->bytes;
  return AFE_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------------------
// Batches: several handles advanced by one launch per stage (afe_batch_*).

struct afe_batch {
  std::vector<afe_mesh*> mem;
  afe::Batch bt{};
  int* d_work = nullptr;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  StepPlan plan;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  double graph_dt = 0.0;
  bool have_graph = false;
  int pending = 0;
  int64_t launches = 0, graph_launches = 0;
  afe_schedule sched{};
  int32_t* d_order = nullptr;
  int tc_fits = 0;  // the members' cells fit the tensor-memory plan together
  ~afe_batch() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (d_order) cudaFree(d_order);
    if (d_work) cudaFree(d_work);
    if (own_stream && st) cudaStreamDestroy(st);
  }
};

namespace {

size_t f32_need(int order, int Nmax, int Smax) { return afe::predictor_f32_smem(order, Nmax, Smax); }

afe_status batch_capture(afe_batch* b, double dt) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  b->have_graph = false;
  AFE_CUDA(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
  afe_status s = enqueue_step(b->plan, dt);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->st, &g);
  if (s != AFE_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return fail(AFE_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  b->graph = g;
  AFE_CUDA(cudaGraphInstantiate(&b->gexec, g, 0));
  b->graph_dt = dt;
  b->have_graph = true;
  return AFE_OK;
}

}  // namespace

extern "C" {

afe_status afe_batch_create(afe_mesh* const* members, int n_members, void* cuda_stream, afe_batch** out) {
  if (!out) return fail(AFE_EINVAL, "out is NULL");
  *out = nullptr;
  if (!members || n_members < 1 || n_members > AFE_MAX_BATCH)
    return fail(AFE_EINVAL, "a batch holds 1 to " + std::to_string(AFE_MAX_BATCH) + " members");
  static_assert(AFE_MAX_BATCH <= afe::kMaxBatch, "batch table too small");
  std::unique_ptr<afe_batch> b(new afe_batch());
  int64_t C = 0, G = 0;
  int Nmax = 0, Smax = 0;
  for (int h = 0; h < n_members; ++h) {
    afe_mesh* m = members[h];
    if (!m) return fail(AFE_EINVAL, "member " + std::to_string(h) + " is NULL");
    for (int k = 0; k < h; ++k)
      if (members[k] == m) return fail(AFE_EINVAL, "a handle appears twice in the batch");
    if (m->p.precision != AFE_FP32) return fail(AFE_EINVAL, "batch members must use AFE_FP32");
    if (m->p.order != members[0]->p.order) return fail(AFE_EINVAL, "batch members must share the order N");
    if (m->device != members[0]->device) return fail(AFE_EINVAL, "batch members must live on one device");
    if (!m->f32_ok || !corrector_f32_fits(m->topo.Nmax))
      return fail(AFE_EINVAL, "member " + std::to_string(h) + " has cells too large for the batched kernels");
    AFE_CUDA(cudaStreamSynchronize(m->stream));
    b->bt.cpre[h] = C;
    b->bt.gpre[h] = G;
    b->bt.tab[h] = m->dm;
    C += m->topo.C;
    G += m->topo.n_groups;
    Nmax = std::max(Nmax, m->topo.Nmax);
    Smax = std::max(Smax, m->topo.Smax);
  }
  b->bt.cpre[n_members] = C;
  b->bt.gpre[n_members] = G;
  b->bt.nh = n_members;
  b->bt.Nmax = Nmax;
  b->bt.Smax = Smax;
  afe_mesh* m0 = members[0];
  if (f32_need(m0->p.order, Nmax, Smax) > m0->f32_smem)
    return fail(AFE_EINVAL, "the members' largest cells do not fit the shared-memory plan together");
  if (C > (int64_t)INT32_MAX) return fail(AFE_EINVAL, "too many cells in one batch");
  int dev = -1;
  AFE_CUDA(cudaGetDevice(&dev));
  if (dev != m0->device) return fail(AFE_EINVAL, "the current device is not the members' device");
  {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, sizeof(int));
    if (e != cudaSuccess) return fail(AFE_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    b->d_work = (int*)p;
  }
  b->bt.work = b->d_work;
  if (cuda_stream) {
    b->st = (cudaStream_t)cuda_stream;
  } else {
    AFE_CUDA(cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking));
    b->own_stream = true;
  }
  b->mem.assign(members, members + n_members);
  StepPlan& P = b->plan;
  P.b = &b->bt;
  P.st = b->st;
  P.order = m0->p.order;
  P.fp32 = 1;
  P.limiter = 0;
  for (afe_mesh* m : b->mem) P.limiter |= m->p.limiter ? 1 : 0;
  P.n_sm = m0->n_sm;
  P.diag = 0;
  P.f32_ok = 1;
  P.f32_smem = m0->f32_smem;
  b->tc_fits = afe::tc_cell_plan(P.order, P.f32_smem, Smax, Nmax).ok ? 1 : 0;
  P.f32_tc = b->tc_fits;
  for (afe_mesh* m : b->mem)
    if (m->variant != 1) P.f32_tc = 0;
  b->sched.variant = P.f32_tc;
  P.d_ref = m0->d_ref;
  P.single = nullptr;
  P.prof = nullptr;
  *out = b.release();
  return AFE_OK;
}

afe_status afe_batch_step_async(afe_batch* b, double dt, int nsteps, int use_graph) {
  if (!b || nsteps < 0) return fail(AFE_EINVAL, "bad argument");
  if (nsteps == 0) return AFE_OK;
  if (b->pending == 0) {
    afe::flags_clear_kernel<<<1, 64, 0, b->st>>>(b->bt);
    AFE_CUDA(cudaGetLastError());
    b->launches += 1;
  }
  const int per = launches_per_step(b->plan, dt);
  if (use_graph) {
    if (!b->have_graph || b->graph_dt != dt) AFE_TRY(batch_capture(b, dt));
    for (int i = 0; i < nsteps; ++i) AFE_CUDA(cudaGraphLaunch(b->gexec, b->st));
    b->graph_launches += nsteps;
  } else {
    for (int i = 0; i < nsteps; ++i) AFE_TRY(enqueue_step(b->plan, dt));
  }
  b->launches += (int64_t)per * nsteps;
  b->pending += nsteps;
  return AFE_OK;
}

afe_status afe_batch_sync(afe_batch* b, int* member_status) {
  if (!b) return fail(AFE_EINVAL, "NULL batch");
  const int nh = b->bt.nh;
  std::vector<int> flags((size_t)nh * afe::F_COUNT);
  std::vector<double> dts(nh), ts(nh);
  for (int h = 0; h < nh; ++h) {
    const afe::DevMesh& d = b->bt.tab[h];
    AFE_CUDA(cudaMemcpyAsync(&flags[(size_t)h * afe::F_COUNT], d.flags, afe::F_COUNT * sizeof(int),
                             cudaMemcpyDeviceToHost, b->st));
    AFE_CUDA(cudaMemcpyAsync(&dts[h], d.dt, sizeof(double), cudaMemcpyDeviceToHost, b->st));
    AFE_CUDA(cudaMemcpyAsync(&ts[h], d.tacc, sizeof(double), cudaMemcpyDeviceToHost, b->st));
  }
  AFE_CUDA(cudaStreamSynchronize(b->st));
  afe_status worst = AFE_OK;
  std::string first_msg;
  for (int h = 0; h < nh; ++h) {
    afe_mesh* m = b->mem[h];
    m->last_dt = dts[h];
    m->t_host = ts[h];
    m->steps += b->pending;
    m->pending = 0;
    const afe_status s = status_of(&flags[(size_t)h * afe::F_COUNT]);
    if (member_status) member_status[h] = (int)s;
    if (s != AFE_OK && (worst == AFE_OK || (int)s > (int)worst)) {
      worst = s;
      first_msg = "member " + std::to_string(h) + ": " + g_err;
    }
  }
  b->pending = 0;
  if (worst != AFE_OK) return fail(worst, first_msg);
  return AFE_OK;
}

afe_status afe_batch_set_schedule(afe_batch* b, const afe_schedule* s) {
  if (!b) return fail(AFE_EINVAL, "NULL batch");
  AFE_TRY(check_schedule(s));
  if (s->variant == 1 && !b->tc_fits)
    return fail(AFE_EINVAL, "the members' cells do not fit the tensor-memory plan together");
  AFE_CUDA(cudaStreamSynchronize(b->st));
  if (s->cost_order && !b->d_order) {
    std::vector<const afe::Topology*> tops;
    for (afe_mesh* m : b->mem) tops.push_back(&m->topo);
    const std::vector<int32_t> ord = cost_order(tops, b->plan.order);
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, ord.size() * sizeof(int32_t));
    if (e != cudaSuccess) return fail(AFE_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    b->d_order = (int32_t*)p;
    AFE_CUDA(cudaMemcpy(b->d_order, ord.data(), ord.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  }
  b->sched = *s;
  b->bt.ring_cap = s->ring_cap;
  b->bt.narrow = s->narrow;
  b->bt.order = s->cost_order ? b->d_order : nullptr;
  b->plan.f32_tc = s->variant;
  b->have_graph = false;  // the captured graph holds the old table
  return AFE_OK;
}

}  // extern "C"

namespace {

// Times `trials` launches of the predictor alone for every candidate schedule (after computing
// the time step of the current state) and sets the fastest.  `set` applies a schedule, `plan`
// returns the launch plan under the schedule last applied.
template <typename SetFn, typename PlanFn>
afe_status autotune_impl(const std::string& sig, int order, bool tc_fits, int* work, cudaStream_t st, int trials,
                         SetFn set, PlanFn plan, afe_schedule* best, double* best_ms, double* default_ms) {
  if (trials < 1 || trials > 64) return fail(AFE_EINVAL, "trials must be in 1..64");
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(sig);
    if (it != g_tune_cache.end()) {
      AFE_TRY(set(it->second));
      if (best) *best = it->second;
      if (best_ms) *best_ms = -1.0;
      if (default_ms) *default_ms = -1.0;
      return AFE_OK;
    }
  }
  {
    const StepPlan P = plan();
    afe::flags_clear_kernel<<<1, 64, 0, st>>>(*P.b);
    afe::step_begin_kernel<<<1, 64, 0, st>>>(*P.b);
    AFE_TRY(enqueue_dt(P, -1.0));
  }
  cudaEvent_t e0, e1;
  AFE_CUDA(cudaEventCreate(&e0));
  AFE_CUDA(cudaEventCreate(&e1));
  std::vector<afe_schedule> cand;
  for (int co = 0; co < 2; ++co)
    for (int va = 0; va < (tc_fits ? 2 : 1); ++va)
      for (int rc : {0, 2})
        for (int na = 0; na < (afe::f32_ntp(order) == 4 ? 2 : 1); ++na) cand.push_back(afe_schedule{co, va, rc, na});
  double tbest = 1e300, tdef = -1.0;
  afe_schedule sbest = cand[0];
  afe_status status = AFE_OK;
  for (const afe_schedule& c : cand) {
    status = set(c);
    if (status != AFE_OK) break;
    const StepPlan P = plan();
    float ms = 0.f;
    for (int r = 0; r <= trials && status == AFE_OK; ++r) {
      if (r == 1) cudaEventRecord(e0, st);
      cudaMemsetAsync(work, 0, sizeof(int), st);
      status = stage(P, 0);
    }
    if (status != AFE_OK) break;
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      status = fail(AFE_ECUDA, "autotune: event timing failed");
      break;
    }
    const double t = ms / trials;
    if (c.cost_order == 0 && c.variant == 0 && c.ring_cap == 0 && c.narrow == 0) tdef = t;
    if (t < tbest) {
      tbest = t;
      sbest = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != AFE_OK) return status;
  AFE_TRY(set(sbest));
  {  // the tuning launches' status flags (iteration cap) are not a step's
    const StepPlan P = plan();
    afe::flags_clear_kernel<<<1, 64, 0, st>>>(*P.b);
    AFE_CUDA(cudaStreamSynchronize(st));
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[sig] = sbest;
  }
  if (best) *best = sbest;
  if (best_ms) *best_ms = tbest;
  if (default_ms) *default_ms = tdef;
  return AFE_OK;
}

}  // namespace

extern "C" {

afe_status afe_autotune(afe_mesh* m, int trials, afe_schedule* best, double* best_ms, double* default_ms) {
  if (!m) return fail(AFE_EINVAL, "NULL mesh");
  if (m->p.precision != AFE_FP32 || !m->f32_ok)
    return fail(AFE_EINVAL, "autotune: the handle does not use the FP32 shared-memory predictor");
  AFE_CUDA(cudaStreamSynchronize(m->stream));
  return autotune_impl(
      "mesh:" + mesh_signature({&m->topo}, m->p.order), m->p.order, m->f32_tc_fits != 0, m->dm.work, m->stream,
      trials, [&](const afe_schedule& c) { return afe_set_schedule(m, &c); }, [&]() { return plan_of(m); }, best,
      best_ms, default_ms);
}

afe_status afe_batch_autotune(afe_batch* b, int trials, afe_schedule* best, double* best_ms, double* default_ms) {
  if (!b) return fail(AFE_EINVAL, "NULL batch");
  AFE_CUDA(cudaStreamSynchronize(b->st));
  std::vector<const afe::Topology*> tops;
  for (afe_mesh* m : b->mem) tops.push_back(&m->topo);
  return autotune_impl(
      "batch:" + mesh_signature(tops, b->plan.order), b->plan.order, b->tc_fits != 0, b->d_work, b->st, trials,
      [&](const afe_schedule& c) { return afe_batch_set_schedule(b, &c); }, [&]() { return b->plan; }, best, best_ms,
      default_ms);
}

afe_status afe_batch_info(const afe_batch* b, int64_t* n_cells, int64_t* n_nodes, int64_t* launches,
                          int64_t* graph_launches) {
  if (!b) return fail(AFE_EINVAL, "NULL batch");
  if (n_cells) *n_cells = b->bt.cpre[b->bt.nh];
  if (n_nodes) {
    int64_t n = 0;
    for (afe_mesh* m : b->mem) n += m->topo.n_nodes;
    *n_nodes = n;
  }
  if (launches) *launches = b->launches;
  if (graph_launches) *graph_launches = b->graph_launches;
  return AFE_OK;
}

void afe_batch_destroy(afe_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->st);
  delete b;
}

}  // extern "C"

// ----------------------------------------------------------------------------------------
// Conserved totals without device allocation (afe_conserved_totals_noalloc).  The partial
// sums go to a fixed file-scope device array instead of memory from cudaMalloc.

namespace {

__device__ __align__(256) double g_noalloc_partials[AFE_NOALLOC_MAX_PARTIALS * 5];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kNoallocMaxDevices] = {nullptr};

// Block b sums w . u over nodes [b*CHUNK, min(n, (b+1)*CHUNK)) in a fixed order.
__global__ void noalloc_partial_kernel(const double* __restrict__ w, const double* __restrict__ u, int64_t n,
                                       double* partials) {
  __shared__ double sh[5][256];
  const int64_t a = (int64_t)blockIdx.x * AFE_NOALLOC_CHUNK;
  const int64_t b = min(n, a + (int64_t)AFE_NOALLOC_CHUNK);
  double acc[5] = {0, 0, 0, 0, 0};
  for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
    const double wi = w[i];
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] += wi * u[i * 5 + v];
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
  if (threadIdx.x < 5) partials[blockIdx.x * 5 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void noalloc_final_kernel(const double* partials, int np, double* out) {
  if (threadIdx.x < 5) {
    double s = 0.0;
    for (int b = 0; b < np; ++b) s += partials[b * 5 + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

}  // namespace

extern "C" afe_status afe_conserved_totals_noalloc(const afe_mesh* m, const double* dq, double* dtotals,
                                                   void* cuda_stream) {
  if (!m || !dq || !dtotals) return fail(AFE_EINVAL, "NULL argument");
  const int64_t n = m->topo.n_nodes;  // >= 1 for every handle afe_mesh_create returns
  if (n > AFE_NOALLOC_MAX_NODES)
    return fail(AFE_EINVAL, "afe_conserved_totals_noalloc: " + std::to_string(n) +
                                " nodes exceed the fixed scratch limit of " + std::to_string(AFE_NOALLOC_MAX_NODES) +
                                " nodes (" + std::to_string(AFE_NOALLOC_MAX_PARTIALS) + " partials of " +
                                std::to_string(AFE_NOALLOC_CHUNK) + ")");
  if (m->device < 0 || m->device >= kNoallocMaxDevices) return fail(AFE_EINVAL, "device index out of range");
  int prev = -1;
  AFE_CUDA(cudaGetDevice(&prev));
  if (prev != m->device) AFE_CUDA(cudaSetDevice(m->device));
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : m->stream;
  double* scratch = nullptr;
  {
    // one-time set-up per device, with that device current: the host-side symbol is only a
    // stand-in, the kernels need the array's device address
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[m->device]) {
      // the look-up must not happen inside a stream capture: refuse with a clear message
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      const cudaError_t ce = cudaStreamIsCapturing(st, &cs);
      if (ce != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        if (prev != m->device) cudaSetDevice(prev);
        return fail(AFE_EINVAL, "afe_conserved_totals_noalloc: the first call on a device must come before any "
                                "stream capture (it looks up the scratch array's device address)");
      }
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
      if (e != cudaSuccess) {
        if (prev != m->device) cudaSetDevice(prev);
        return fail(AFE_ECUDA, std::string("cudaGetSymbolAddress(g_noalloc_partials): ") + cudaGetErrorString(e));
      }
      g_noalloc_ptr[m->device] = (double*)p;
    }
    scratch = g_noalloc_ptr[m->device];
  }
  const int np = (int)((n + AFE_NOALLOC_CHUNK - 1) / AFE_NOALLOC_CHUNK);
  if (np > 0) noalloc_partial_kernel<<<np, 256, 0, st>>>(m->dm.wvec, dq, n, scratch);
  noalloc_final_kernel<<<1, 32, 0, st>>>(scratch, np, dtotals);  // np = 0 writes zeros
  cudaError_t e = cudaGetLastError();
  if (prev != m->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return fail(AFE_ECUDA, std::string("afe_conserved_totals_noalloc launch: ") + cudaGetErrorString(e));
  return AFE_OK;
}
