// C-ABI and device orchestration of the KFBI Stokes solver (see include/kfbim.h).
//
// Interface solve (Sec. 4, Alg. 1 step 2), all on the GPU:
//   jumps (k_jumps) -> RHS f~ + corrections (k_rhs_fill, k_corrections)
//   -> Schur RHS b = g + (1/mu) sum_c G_c^T (-Delta_c)^{-1} f^(c)
//   -> CG on (S + gamma gamma^T / alpha) p = b with
//      S = (1/mu) sum_c B_c^{-1} Lambda_c B_c
//   -> u^(c) = (1/mu) (-Delta_c)^{-1} (f^(c) - G_c p).
// S is applied spectrally: G_c maps the cell basis cos(pi a (i+1/2)/N) to the
// face basis -(2/h) sin(pi a / 2N) sin(pi a i / N), so each term
// G_c^T (-Delta_c)^{-1} G_c is diagonal in B_c = DCT-II along axis c times
// DST-II across, with eigenvalue sin^2(a_c) / sum_b sin^2(a_b).  This is the
// same operator as the paper's (up to rounding) with only length-N transforms.
// MIXED precision runs the transforms and CG in FP32 inside FP64 iterative
// refinement of the corrected MAC system.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels.cuh"
#include "transforms.cuh"
#include "transforms2.cuh"
#include "pass2.h"
#include "tc_pass.cuh"
#include "slab.h"

using namespace kfbim;

struct kfbim_ctx {
  kfbim_options opt{};
  std::string err;
  HostTables host;
  // device memory through the caller's allocator (kfbim_setup_ex), if any
  kfbim_allocator allocator{};
  bool custom_alloc = false;
  std::vector<size_t> alloc_bytes;   // sizes of `allocs`, for the caller's free
  int N = 0, lg = 0;   // lg = log2 N, or -1 when N is not a power of two (96)
  GridIx gix() const { return GridIx{N, lg}; }
  int64_t N3 = 0, n_all = 0, n_prim = 0, n_corr_rows = 0;
  double h = 0, mu = 1;
  bool navier = false;
  double cpen = 0.0;   // c = 1/(lambda + mu) of the Navier continuity row, 0 for Stokes
  std::vector<void*> allocs;
  // tables
  int32_t *d_comp = nullptr, *d_pid = nullptr, *d_fit_col = nullptr, *d_tr_comp = nullptr,
          *d_tr_node = nullptr;
  int64_t *d_corr_row = nullptr, *d_corr_ptr = nullptr,
          *d_corr_src = nullptr, *d_prim_of = nullptr;
  // surface fit, interleaved by groups of 32 rows (k_jumps): entry i of row r
  // at fit_off[r / 32] + 32 i + r % 32, rows padded to their group's longest
  // with zero weights; fit_pos maps a CSR entry to its interleaved position
  int64_t* d_fit_off = nullptr;
  int64_t fit_ell = 0;
  std::vector<int32_t> fit_pos;
  double *d_fit_w = nullptr, *d_jmap = nullptr, *d_corr_coef = nullptr, *d_tr_w = nullptr,
         *d_tr_cj = nullptr, *d_s2 = nullptr;
  uint8_t* d_side[4] = {nullptr, nullptr, nullptr, nullptr};
  C2<double>* d_tw64 = nullptr;
  C2<double>* d_q64 = nullptr;
  C2<float>* d_tw32 = nullptr;
  C2<float>* d_q32 = nullptr;
  C2<double>* d_twc64 = nullptr;  // full-circle twiddles exp(-2 pi i t / 2N), t < 2N
  C2<float>* d_twc32 = nullptr;
  float* d_s2f = nullptr;         // FP32 copy of the eigenvalue table
  double* d_xyz = nullptr;        // control point coordinates (3 per point)
  // tensor-core passes (N = 128, MIXED): transform matrices [type 1..6][hi|lo][n][m],
  // the kernels' timeout flag, and the kernel chosen per stage kind (0 FFT, 1 GEMM)
  float* d_tc_mats = nullptr;
  int* d_tc_err = nullptr;
  int xf_plain = 0, xf_fused = 0;
  // MIXED Schur CG as the three-kernel z-pencil / xy-slab iteration (slab.cuh)
  bool slab = false;
  // MIXED refinement tolerance of the next grid solve: opt.refine_tol, or
  // looser inside GMRES once its residual is small (opt.relax > 0)
  double refine_tol_now = 0.0;
  double relax = 0.0;
  // precision requested at setup (FP32 and MIXED_TF32 run as MIXED internally:
  // FP32 without the FP64 refinement sweeps, MIXED_TF32 on tensor-core passes)
  int precision_requested = KFBIM_FP64;
  bool fp32_only = false;
  // stream of the setup's device work (kfbim_setup_async; null: legacy stream)
  cudaStream_t setup_stream = nullptr;
  int num_sms = 152;
  float tune_ms[4] = {0, 0, 0, 0};   // plain FFT, plain GEMM, fused FFT, fused GEMM (ms per stage)
  // FP64 workspace
  double *J = nullptr, *rhs = nullptr, *u = nullptr, *p = nullptr, *t1 = nullptr, *t2 = nullptr;
  double *cr = nullptr, *cd = nullptr, *cq = nullptr, *rres = nullptr, *zero_phi = nullptr;
  double *partial = nullptr, *scal = nullptr;   // reduction partials, scalars
  CGScalars* cgs = nullptr;
  // FP32 workspace (mixed)
  float *f1 = nullptr, *f2 = nullptr, *fx = nullptr, *fr = nullptr, *fd = nullptr, *fq = nullptr,
        *fu = nullptr;
  // second and third component outputs of the Schur apply, six stage temporaries
  double *q2 = nullptr, *q3 = nullptr, *T6 = nullptr;
  float *fq2 = nullptr, *fq3 = nullptr, *fT6 = nullptr;
  // GMRES
  int gm_max = 0;
  double *V = nullptr, *gw = nullptr, *gh = nullptr, *grhs = nullptr, *gy = nullptr;
  double* pinned = nullptr;  // host scalars
  // staging buffers of kfbim_solve_host (allocated on first use)
  double *hs_g = nullptr, *hs_phi = nullptr, *hs_fp = nullptr, *hs_fg = nullptr, *hs_u = nullptr,
         *hs_p = nullptr;
  bool device = false;        // false for kfbim_setup_host contexts
  int dev_id = -1;            // CUDA device holding the context's memory, streams and graphs (-1: none)
  // CUDA graphs of kCgGraphIters CG iterations (index 0: FP64, 1: FP32)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t cg_exec[2] = {nullptr, nullptr};
  int64_t cg_graph_kernels[2] = {0, 0};
  // the batched slab CG of all bcap slots as one device-side while loop
  // (captured once per batch allocation; null where conditional nodes are
  // not available) and its kernels per trip
  cudaGraphExec_t bcg_exec = nullptr;
  int64_t bcg_kernels = 0;
  bool bcg_tried = false;
  // whether cg_exec[slot] is the device-side while loop (conditional node)
  // or kCgGraphIters iterations in a row
  bool cg_loop[2] = {false, false};
  bool use_graphs = true;
  // optional per-kernel timing (kfbim_profile, kfbim_profile_kernels): CUDA
  // events around launches, totals per kernel class (kfbim_kernel_class)
  bool prof = false;
  std::vector<cudaEvent_t> prof_ev;    // pairs (start, stop)
  int prof_used = 0;
  double prof_ms[KFBIM_KCLASS_COUNT] = {};
  int64_t prof_count[KFBIM_KCLASS_COUNT] = {};
  std::vector<int> prof_tag;           // kernel class of each event pair
  double prof_bytes[KFBIM_KCLASS_COUNT] = {};   // algorithmic bytes moved by those launches
  int64_t fit_nnz = 0, corr_nnz = 0;
  // batch of instances on this geometry (kfbim_solve_batch), allocated on demand
  struct Slot {
    double *J, *rhs, *u, *p, *res, *grhs, *V, *gw, *gh, *gy;
    float *x, *r, *d, *q, *q2, *q3, *T6, *fu;
  };
  std::vector<Slot> bs;
  CGScalars* bcgs = nullptr;   // one per slot, contiguous
  double* bscal = nullptr;     // 8 per slot, contiguous
  double* bgh = nullptr;       // (bm + 1) per slot, contiguous (slot.gh points into it)
  double* bpartial = nullptr;  // kRunPartials reduction partials per slot (batched CG kernels)
  void* bpinned = nullptr;     // host staging of bcgs / bscal / bgh
  int bcap = 0, bm = 0;
  std::vector<int> b_cg, b_sweeps, b_isolves;   // per-slot counters of the current call
  std::vector<double> b_refine_tol;              // per-slot refine_tol_now of a batched call
  // adjoint: transposed trace (by node), corrections (by jump slot) and fit
  // (by primary column) tables, built at setup; Jbar, Dbar work arrays
  bool adj_ready = false;
  int64_t ta_n = 0, ca_n = 0;
  int64_t *d_ta_key = nullptr, *d_ta_ptr = nullptr, *d_ca_key = nullptr, *d_ca_ptr = nullptr,
          *d_ca_row = nullptr, *d_fa_ptr = nullptr;
  int32_t *d_ta_q = nullptr, *d_fa_q = nullptr, *d_fa_rr = nullptr;
  double *d_ta_w = nullptr, *d_ca_coef = nullptr, *d_Jbar = nullptr, *d_Dbar = nullptr;
  // counters of the current call
  int cg_iters = 0, refine_sweeps = 0, interface_solves = 0;
};

// Raise, never lower, the dynamic shared-memory limit of a kernel on the
// current device.  The attribute belongs to the device, so the limit already
// set is tracked per (kernel, device); a kernel launched with several sizes
// (the runtime-N pass) keeps the largest, since setting a small size would
// also lower it below the 48 KiB default for every later launch of that
// kernel, from any path of this library.  Safe to call from several threads.
cudaError_t kfbim::raise_dynamic_smem(const void* kern, size_t bytes) {
  struct Limit {
    const void* kern;
    int dev;
    size_t bytes;
  };
  static std::mutex m;
  static std::vector<Limit> limit;
  int dev = 0;
  const cudaError_t ge = cudaGetDevice(&dev);
  if (ge != cudaSuccess) return ge;
  std::lock_guard<std::mutex> lock(m);
  size_t* cur = nullptr;
  for (auto& e : limit)
    if (e.kern == kern && e.dev == dev) cur = &e.bytes;
  if (!cur) {
    limit.push_back({kern, dev, (size_t)48 * 1024});
    cur = &limit.back().bytes;
  }
  if (bytes <= *cur) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) *cur = bytes;
  return e;
}

namespace {

struct CudaError {
  std::string msg;
  int code = KFBIM_E_CUDA;
};

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) throw CudaError{std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

// Device memory of the context: from the caller's allocator when setup was
// given one (kfbim_setup_ex; at least 256-byte aligned), else cudaMalloc.
template <typename T>
T* dalloc(kfbim_ctx* c, size_t count) {
  void* p = nullptr;
  if (count == 0) count = 1;
  const size_t bytes = count * sizeof(T);
  if (c->custom_alloc) {
    p = c->allocator.alloc(bytes, c->allocator.user);
    if (!p) throw CudaError{"allocator callback: out of memory", KFBIM_E_OOM};
    if (reinterpret_cast<uintptr_t>(p) % 256 != 0) {
      c->allocator.free(p, bytes, c->allocator.user);
      throw CudaError{"allocator callback: memory not 256-byte aligned", KFBIM_E_INVALID};
    }
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) throw CudaError{std::string("cudaMalloc: ") + cudaGetErrorString(e)};
  }
  c->allocs.push_back(p);
  c->alloc_bytes.push_back(bytes);
  return static_cast<T*>(p);
}

// Copies a host table to new device memory, ordered on the setup stream
// (the caller's stream for kfbim_setup_async); setup synchronises that stream
// before the host tables are released.
template <typename T>
T* upload(kfbim_ctx* c, const std::vector<T>& v) {
  T* d = dalloc<T>(c, v.size());
  if (!v.empty())
    CK(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->setup_stream));
  return d;
}

inline int grid_for(int64_t n, int threads = 256) {
  int64_t b = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

// Kernel launches issued through this library by the calling host thread: an
// entry point reports the difference across its own call, so calls running on
// other threads (other contexts) do not enter its count.
thread_local int64_t g_launches = 0;

inline void check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw CudaError{std::string("kernel launch: ") + cudaGetErrorString(e)};
}


// ------------------------------------------------------------ transforms
template <typename T>
struct Tw;
template <>
struct Tw<double> {
  static const C2<double>* tw(kfbim_ctx* c) { return c->d_tw64; }
  static const C2<double>* q(kfbim_ctx* c) { return c->d_q64; }
  static const C2<double>* twc(kfbim_ctx* c) { return c->d_twc64; }
  static const double* s2(kfbim_ctx* c) { return c->d_s2; }
};
template <>
struct Tw<float> {
  static const C2<float>* tw(kfbim_ctx* c) { return c->d_tw32; }
  static const C2<float>* q(kfbim_ctx* c) { return c->d_q32; }
  static const C2<float>* twc(kfbim_ctx* c) { return c->d_twc32; }
  static const float* s2(kfbim_ctx* c) { return c->d_s2f; }
};

// Reduction partials per batch slot: RED_BLOCKS for the staged CG kernels,
// four per block of the slab iteration's k_cg_zinv (4 x 512 at N = 128).
constexpr int kRunPartials = 2 * RED_BLOCKS;
constexpr int kMaxJobs = kPass2BatchJobs;   // jobs per batched launch: 3 per instance, 16 instances

template <typename Tin, typename T, typename Tout, int N, int MAXJ>
void launch_pass2(kfbim_ctx* c, const PassJobs<Tin, Tout, MAXJ>& jobs, int njobs, cudaStream_t s) {
  CK((pass2_launch<N, Tin, T, Tout, MAXJ>(jobs, njobs, Tw<T>::twc(c), Tw<T>::q(c), Tw<T>::s2(c), s)));
}

// One transform pass of a stage: input, output, axis, first transform,
// second transform, spectral weight, weight component, accumulate flag, and
// the done flag of the CG run the pass belongs to (nullable).
struct Job {
  const void* in;
  void* out;
  int axis, t0, t1, wmode, wc, acc;
  const int* skip = nullptr;
};

void prof_collect(kfbim_ctx* c);

template <typename Tin, typename Tout>
PassJob<Tin, Tout> make_job(kfbim_ctx* c, const Job& j, const int* skip) {
  PassArgs a{};  // value-initialised: every field, skip included, starts at zero
  a.N = c->N;
  a.axis = j.axis;
  a.type0 = j.t0;
  a.type1 = j.t1;
  a.wmode = j.wmode;
  a.wc = j.wc;
  for (int b = 0; b < 3; ++b) a.kind[b] = (b == j.wc) ? 0 : 1;
  a.mu = c->mu;
  a.h = c->h;
  a.accumulate = j.acc;
  a.scale = 1.0;
  a.skip = j.skip ? j.skip : skip;
  return {static_cast<const Tin*>(j.in), static_cast<Tout*>(j.out), a};
}

template <typename Tin, typename T, typename Tout, int MAXJ>
void launch_jobs(kfbim_ctx* c, const Job* list, int nj, cudaStream_t s, const int* skip) {
  PassJobs<Tin, Tout, MAXJ> jobs{};
  for (int k = 0; k < nj; ++k) jobs.j[k] = make_job<Tin, Tout>(c, list[k], skip);
  if (c->N == 128) launch_pass2<Tin, T, Tout, 128, MAXJ>(c, jobs, nj, s);
  else if (c->N == 256) launch_pass2<Tin, T, Tout, 256, MAXJ>(c, jobs, nj, s);
  else if (c->N == 96) launch_pass2<Tin, T, Tout, 96, MAXJ>(c, jobs, nj, s);
  else if (c->N == 64) launch_pass2<Tin, T, Tout, 64, MAXJ>(c, jobs, nj, s);
  else launch_pass2<Tin, T, Tout, 32, MAXJ>(c, jobs, nj, s);
  ++g_launches;
}

// Launch a list of independent passes: up to 3 jobs per launch on the
// compile-time-N kernel (48 for longer, batched lists), one launch per job on
// the runtime-N kernel.
// Tensor-core passes of one stage: all jobs share the first transform; a
// fused job (second transform) becomes a weighted pass into its output and an
// in-place pass of the second transform.  Returns the kernel launches.
int tc_passes(kfbim_ctx* c, const std::vector<Job>& list, cudaStream_t s, const int* skip, double* bytes) {
  const int nj = (int)list.size();
  auto launch = [&](const Job* jl, int n) {
    const int type = jl[0].t0;
    PassJobs<float, float, TC_MAXJ> jobs{};
    for (int k = 0; k < n; ++k) {
      Job j = jl[k];
      j.t1 = X_NONE;
      jobs.j[k] = make_job<float, float>(c, j, skip);
      *bytes += (double)c->N3 * sizeof(float) * (j.acc ? 3 : 2);
    }
    const int grid = std::min(c->num_sms, n * TC_TILES_PER_JOB);
    CK(raise_dynamic_smem(reinterpret_cast<const void*>(k_tc_pass), TC_SMEM));
    k_tc_pass<<<grid, TC_THREADS, TC_SMEM, s>>>(jobs, n, c->d_tc_mats + (size_t)(type - 1) * 2 * TC_N * TC_N,
                                                c->d_s2f, c->d_tc_err);
    ++g_launches;
  };
  int launches = 0;
  for (int k0 = 0; k0 < nj; k0 += TC_MAXJ) {
    launch(list.data() + k0, std::min(TC_MAXJ, nj - k0));
    ++launches;
  }
  if (list[0].t1 != X_NONE) {
    std::vector<Job> second;
    for (const Job& j : list) second.push_back({j.out, j.out, j.axis, j.t1, X_NONE, W_NONE, j.wc, j.acc, j.skip});
    for (int k0 = 0; k0 < nj; k0 += TC_MAXJ) {
      launch(second.data() + k0, std::min(TC_MAXJ, nj - k0));
      ++launches;
    }
  }
  check_launch();
  return launches;
}

// Whether a stage of FP32 passes goes to the tensor-core kernel (FP32 input
// and output; FP64-input stages stay on the FFT kernel).
template <typename Tin, typename T, typename Tout>
bool use_tc(const kfbim_ctx* c, const std::vector<Job>& list) {
  if (!std::is_same<Tin, float>::value || !std::is_same<T, float>::value || !std::is_same<Tout, float>::value)
    return false;
  if (!c->d_tc_mats || list.empty()) return false;
  const bool fused = list[0].t1 != X_NONE;
  if (!(fused ? c->xf_fused : c->xf_plain)) return false;
  for (const Job& j : list) {
    if (j.t0 != list[0].t0 || j.t1 != list[0].t1) return false;
    if (fused && j.acc) return false;   // the split passes cannot accumulate through a temporary
  }
  return true;
}

template <typename Tin, typename T, typename Tout>
void stage_list(kfbim_ctx* c, const std::vector<Job>& list, cudaStream_t s, const int* skip = nullptr) {
  double bytes = 0.0;
  const bool prof = c->prof && c->prof_used + 2 <= (int)c->prof_ev.size();
  if (prof) CK(cudaEventRecord(c->prof_ev[c->prof_used], s));
  const int nj = (int)list.size();
  int launches = 1;
  if (use_tc<Tin, T, Tout>(c, list)) {
    launches = tc_passes(c, list, s, skip, &bytes);
  } else if (c->N == 256 || c->N == 128 || c->N == 96 || c->N == 64 || c->N == 32) {
    for (const Job& j : list) bytes += (double)c->N3 * (sizeof(Tin) + sizeof(Tout) * (j.acc ? 2 : 1));
    if (nj <= 3) {
      launch_jobs<Tin, T, Tout, 3>(c, list.data(), nj, s, skip);
    } else {
      for (int k0 = 0; k0 < nj; k0 += kMaxJobs)
        launch_jobs<Tin, T, Tout, kMaxJobs>(c, list.data() + k0, std::min(kMaxJobs, nj - k0), s, skip);
    }
    launches = nj <= 3 ? 1 : (nj + kMaxJobs - 1) / kMaxJobs;
  } else {
    const size_t smem = pass_smem_bytes(c->N, sizeof(T));
    auto kern = k_axis_pass<Tin, T, Tout>;
    CK(raise_dynamic_smem((const void*)kern, smem));
    const int blocks = (int)((int64_t)c->N * c->N / LPC);
    for (const Job& j : list) {
      bytes += (double)c->N3 * (sizeof(Tin) + sizeof(Tout) * (j.acc ? 2 : 1));
      const PassJob<Tin, Tout> pj = make_job<Tin, Tout>(c, j, skip);
      kern<<<blocks, PASS_THREADS, smem, s>>>(pj.in, pj.out, pj.a, Tw<T>::tw(c), Tw<T>::q(c), c->d_s2);
      ++g_launches;
    }
    launches = nj;
  }
  check_launch();
  if (prof) {
    CK(cudaEventRecord(c->prof_ev[c->prof_used + 1], s));
    const int slot = sizeof(T) == 8 ? KFBIM_KCLASS_TRANSFORM_FP64 : KFBIM_KCLASS_TRANSFORM_FP32;
    c->prof_tag[c->prof_used / 2] = slot;
    c->prof_used += 2;
    c->prof_count[slot] += launches;
    c->prof_bytes[slot] += bytes;
  }
}

template <typename Tin, typename T, typename Tout>
void stage(kfbim_ctx* c, std::initializer_list<Job> list, cudaStream_t s, const int* skip = nullptr) {
  stage_list<Tin, T, Tout>(c, std::vector<Job>(list), s, skip);
}

// Timing of one launch group of a kernel class: prof_begin records the start
// event (returns -1 when profiling is off or the event pool is full),
// prof_end the stop event and the group's launches and algorithmic bytes.
int prof_begin(kfbim_ctx* c, cudaStream_t s) {
  if (!c->prof || c->prof_used + 2 > (int)c->prof_ev.size()) return -1;
  CK(cudaEventRecord(c->prof_ev[c->prof_used], s));
  return c->prof_used;
}

void prof_end(kfbim_ctx* c, cudaStream_t s, int at, int cls, int launches, double bytes) {
  if (at < 0) return;
  CK(cudaEventRecord(c->prof_ev[at + 1], s));
  c->prof_tag[at / 2] = cls;
  c->prof_used = at + 2;
  c->prof_count[cls] += launches;
  c->prof_bytes[cls] += bytes;
}

// Fold recorded event pairs into the totals (the stream must be idle).
void prof_collect(kfbim_ctx* c) {
  for (int e = 0; e + 1 < c->prof_used; e += 2) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->prof_ev[e], c->prof_ev[e + 1]));
    c->prof_ms[c->prof_tag[e / 2]] += ms;
  }
  c->prof_used = 0;
}

inline void others(int cax, int& o1, int& o2) {
  o1 = (cax == 0) ? 1 : 0;
  o2 = (cax == 2) ? 1 : 2;
}

// Stage tables.  Component c (axis cax = c - 1) is transformed along its two
// other axes (o1 < o2) with DST-II, and along cax with DCT-II (cell basis) or
// DST-I (face basis); the middle pass along cax is fused with the weight.

// u = (1/mu) (-Delta_c)^{-1} r on face grid c (single component)
template <typename Tin, typename T, typename Tout>
void face_poisson(kfbim_ctx* c, int cax, const Tin* r, Tout* u, T* t1, T* t2, cudaStream_t s) {
  int o1, o2;
  others(cax, o1, o2);
  stage<Tin, T, T>(c, {{r, t1, o2, X_DST2F, X_NONE, W_NONE, cax, 0}}, s);
  stage<T, T, T>(c, {{t1, t2, o1, X_DST2F, X_NONE, W_NONE, cax, 0}}, s);
  stage<T, T, T>(c, {{t2, t1, cax, X_DST1F, X_DST1I, W_POISSON, cax, 0}}, s);
  stage<T, T, T>(c, {{t1, t2, o1, X_DST2I, X_NONE, W_NONE, cax, 0}}, s);
  stage<T, T, Tout>(c, {{t2, u, o2, X_DST2I, X_NONE, W_NONE, cax, 0}}, s);
}

// u^(c) = (1/mu) (-Delta_c)^{-1} r^(c) for c = 1..3 (r, u: 3 N^3, may alias);
// T6 = six N^3 temporaries.
template <typename T>
void face_poisson3(kfbim_ctx* c, const T* r, T* u, T* T6, cudaStream_t s) {
  const int64_t n = c->N3;
  const T *r1 = r, *r2 = r + n, *r3 = r + 2 * n;
  T *u1 = u, *u2 = u + n, *u3 = u + 2 * n;
  T *A = T6, *B = T6 + n, *C = T6 + 2 * n, *D = T6 + 3 * n, *E = T6 + 4 * n, *F = T6 + 5 * n;
  stage<T, T, T>(c, {{r1, A, 2, X_DST2F, X_NONE, W_NONE, 0, 0}, {r2, B, 2, X_DST2F, X_NONE, W_NONE, 1, 0},
                     {r3, C, 1, X_DST2F, X_NONE, W_NONE, 2, 0}}, s);
  stage<T, T, T>(c, {{A, D, 1, X_DST2F, X_NONE, W_NONE, 0, 0}, {B, E, 0, X_DST2F, X_NONE, W_NONE, 1, 0},
                     {C, F, 0, X_DST2F, X_NONE, W_NONE, 2, 0}}, s);
  stage<T, T, T>(c, {{D, A, 0, X_DST1F, X_DST1I, W_POISSON, 0, 0}, {E, B, 1, X_DST1F, X_DST1I, W_POISSON, 1, 0},
                     {F, C, 2, X_DST1F, X_DST1I, W_POISSON, 2, 0}}, s);
  stage<T, T, T>(c, {{A, D, 1, X_DST2I, X_NONE, W_NONE, 0, 0}, {B, E, 0, X_DST2I, X_NONE, W_NONE, 1, 0},
                     {C, F, 0, X_DST2I, X_NONE, W_NONE, 2, 0}}, s);
  stage<T, T, T>(c, {{D, u1, 2, X_DST2I, X_NONE, W_NONE, 0, 0}, {E, u2, 2, X_DST2I, X_NONE, W_NONE, 1, 0},
                     {F, u3, 1, X_DST2I, X_NONE, W_NONE, 2, 0}}, s);
}

// b_c = (1/mu) G_c^T (-Delta_c)^{-1} f^(c) for c = 1..3 into b1, b2, b3
// (f: 3 N^3 of type Tin); the caller adds g.
template <typename Tin, typename T>
void schur_rhs3(kfbim_ctx* c, const Tin* f, T* b1, T* b2, T* b3, T* T6, cudaStream_t s) {
  const int64_t n = c->N3;
  const Tin *f1 = f, *f2 = f + n, *f3 = f + 2 * n;
  T *A = T6, *B = T6 + n, *C = T6 + 2 * n, *D = T6 + 3 * n, *E = T6 + 4 * n, *F = T6 + 5 * n;
  stage<Tin, T, T>(c, {{f1, A, 2, X_DST2F, X_NONE, W_NONE, 0, 0}, {f2, B, 2, X_DST2F, X_NONE, W_NONE, 1, 0},
                       {f3, C, 1, X_DST2F, X_NONE, W_NONE, 2, 0}}, s);
  stage<T, T, T>(c, {{A, D, 1, X_DST2F, X_NONE, W_NONE, 0, 0}, {B, E, 0, X_DST2F, X_NONE, W_NONE, 1, 0},
                     {C, F, 0, X_DST2F, X_NONE, W_NONE, 2, 0}}, s);
  stage<T, T, T>(c, {{D, A, 0, X_DST1F, X_DCT2I, W_RHS, 0, 0}, {E, B, 1, X_DST1F, X_DCT2I, W_RHS, 1, 0},
                     {F, C, 2, X_DST1F, X_DCT2I, W_RHS, 2, 0}}, s);
  stage<T, T, T>(c, {{A, D, 1, X_DST2I, X_NONE, W_NONE, 0, 0}, {B, E, 0, X_DST2I, X_NONE, W_NONE, 1, 0},
                     {C, F, 0, X_DST2I, X_NONE, W_NONE, 2, 0}}, s);
  stage<T, T, T>(c, {{D, b1, 2, X_DST2I, X_NONE, W_NONE, 0, 0}, {E, b2, 2, X_DST2I, X_NONE, W_NONE, 1, 0},
                     {F, b3, 1, X_DST2I, X_NONE, W_NONE, 2, 0}}, s);
}

// q_c = (1/mu) G_c^T (-Delta_c)^{-1} G_c d into q, q2, q3 (the CG kernel sums
// them); the c = 1 and c = 2 terms share their first transform (DST-II along z).
template <typename T>
void schur_apply3(kfbim_ctx* c, const T* d, T* q, T* q2, T* q3, T* T6, cudaStream_t s,
                  const int* skip = nullptr) {
  const int64_t n = c->N3;
  T *A = T6, *B = T6 + n, *C = T6 + 2 * n, *D = T6 + 3 * n, *E = T6 + 4 * n, *F = T6 + 5 * n;
  stage<T, T, T>(c, {{d, A, 2, X_DST2F, X_NONE, W_NONE, 0, 0}, {d, B, 1, X_DST2F, X_NONE, W_NONE, 2, 0}},
                 s, skip);
  stage<T, T, T>(c, {{A, C, 1, X_DST2F, X_NONE, W_NONE, 0, 0}, {A, D, 0, X_DST2F, X_NONE, W_NONE, 1, 0},
                     {B, E, 0, X_DST2F, X_NONE, W_NONE, 2, 0}}, s, skip);
  stage<T, T, T>(c, {{C, A, 0, X_DCT2F, X_DCT2I, W_SCHUR, 0, 0}, {D, B, 1, X_DCT2F, X_DCT2I, W_SCHUR, 1, 0},
                     {E, F, 2, X_DCT2F, X_DCT2I, W_SCHUR, 2, 0}}, s, skip);
  stage<T, T, T>(c, {{A, C, 1, X_DST2I, X_NONE, W_NONE, 0, 0}, {B, D, 0, X_DST2I, X_NONE, W_NONE, 1, 0},
                     {F, E, 0, X_DST2I, X_NONE, W_NONE, 2, 0}}, s, skip);
  stage<T, T, T>(c, {{C, q, 2, X_DST2I, X_NONE, W_NONE, 0, 0}, {D, q2, 2, X_DST2I, X_NONE, W_NONE, 1, 0},
                     {E, q3, 1, X_DST2I, X_NONE, W_NONE, 2, 0}}, s, skip);
}

double read_scalar(kfbim_ctx* c, const double* dptr, cudaStream_t s) {
  CK(cudaMemcpyAsync(c->pinned, dptr, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (c->prof_used) prof_collect(c);
  return c->pinned[0];
}

template <typename Ta, typename Tb>
void dot(kfbim_ctx* c, const Ta* x, const Tb* y, int64_t n, double* out, double scale, cudaStream_t s) {
  k_dot_partial<Ta, Tb><<<RED_BLOCKS, RED_THREADS, 0, s>>>(x, y, n, c->partial); ++g_launches;
  check_launch();
  k_sum_partials<<<1, RED_THREADS, 0, s>>>(c->partial, RED_BLOCKS, scale, out); ++g_launches;
  check_launch();
}

// |x|^2 of an FP64 field for the refinement's stopping test (about 1e-7
// relative; compensated FP32 sums of the values rounded to FP32).
void norm2_fast(kfbim_ctx* c, const double* x, int64_t n, double* out, cudaStream_t s) {
  float2* part = reinterpret_cast<float2*>(c->partial);
  k_norm2_partial<<<RED_BLOCKS, RED_THREADS, 0, s>>>(x, n, part); ++g_launches;
  k_merge_partials<<<1, RED_THREADS, 0, s>>>(part, RED_BLOCKS, 1.0, out); ++g_launches;
  check_launch();
}

constexpr int kCgGraphIters = 4;

// CG vectors and stage temporaries of one precision (fixed workspace buffers).
template <typename T>
struct CgWs {
  T *x, *r, *d, *q, *q2, *q3, *T6;
};

CgWs<double> ws64(kfbim_ctx* c) { return {c->p, c->rres, c->cd, c->cq, c->q2, c->q3, c->T6}; }
CgWs<float> ws32(kfbim_ctx* c) { return {c->fx, c->fr, c->fd, c->fq, c->fq2, c->fq3, c->fT6}; }

// The slab CG of a single run on the FP32 workspace.
SlabCg slab_run(kfbim_ctx* c, const CgWs<float>& w) {
  const int64_t n = c->N3;
  return {c->N, w.x, w.r, w.d, w.q, w.T6, w.T6 + n, c->d_twc32, c->d_q32, c->d_s2f, (float)(1.0 / c->mu),
          c->cgs, c->partial};
}

// One CG iteration: q = S d (5 staged launches), then the three fused
// scalar/vector kernels; or the three slab kernels.  All of it is a no-op
// once cgs->done is set.
template <typename T>
void cg_iteration(kfbim_ctx* c, const CgWs<T>& w, cudaStream_t s) {
  const int64_t n = c->N3;
  if constexpr (std::is_same<T, float>::value) {
    if (c->slab) {
      // the previous iteration's update, d = r + beta d and the z transforms;
      // the xy planes; the inverse z transforms with d.q, r.q, q.q (slab.cuh)
      const SlabCg a = slab_run(c, w);
      if (c->prof) {
        for (int k = 0; k < 3; ++k) {
          const int at = prof_begin(c, s);
          g_launches += slab_launch(k, a, s);
          prof_end(c, s, at, KFBIM_KCLASS_CG_ZFWD + k, 1, (double)kSlabValues[k] * n * sizeof(float));
        }
      } else {
        g_launches += slab_cg_iteration(a, s);
      }
      check_launch();
      return;
    }
  }
  schur_apply3<T>(c, w.d, w.q, w.q2, w.q3, w.T6, s, &c->cgs->done);
  const int at = prof_begin(c, s);
  k_cg_alpha<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(w.d, w.q, w.q2, w.q3, n, c->cgs, c->partial); ++g_launches;
  k_cg_update<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(w.x, w.r, w.d, w.q, n, c->cgs, c->partial); ++g_launches;
  k_cg_direction<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(w.d, w.r, n, c->cgs, c->partial); ++g_launches;
  // values moved: alpha 5 N^3 (d, q, q2, q3 read, q written), update 6, direction 3
  prof_end(c, s, at, KFBIM_KCLASS_CG_VECTOR, 3, 14.0 * n * sizeof(T));
  check_launch();
}

template <typename T>
struct Slot;
template <>
struct Slot<double> { static constexpr int v = 0; };
template <>
struct Slot<float> { static constexpr int v = 1; };

// Device side of the CG loop of a conditional graph: counts the trip and
// keeps the loop going while the run is neither converged (done) nor at its
// iteration cap, so the loop always ends after at most maxit trips.
__global__ void k_cg_cond(cudaGraphConditionalHandle h, CGScalars* s, int maxit) {
  const int t = ++s->trips;
  cudaGraphSetConditional(h, (!s->done && t < maxit) ? 1u : 0u);
}

// The CG graph of this precision, captured once per context (every pointer
// it uses is a fixed workspace buffer): a conditional while node whose body is
// one CG iteration and k_cg_cond, so that a whole CG run is one graph launch
// and one read of the scalars; where conditional nodes are not available,
// kCgGraphIters iterations in a row, launched until the run is done.
template <typename T>
cudaGraphExec_t cg_graph(kfbim_ctx* c, const CgWs<T>& w) {
  const int slot = Slot<T>::v;
  if (c->cg_exec[slot]) return c->cg_exec[slot];
  // kernel attributes are set outside the capture: one iteration on the idle
  // capture stream with the done flag raised does nothing but configure them
  const int one = 1;
  CK(cudaMemcpyAsync(&c->cgs->done, &one, sizeof(int), cudaMemcpyHostToDevice, c->cap_stream));
  const int64_t before = g_launches;
  cg_iteration<T>(c, w, c->cap_stream);
  CK(cudaStreamSynchronize(c->cap_stream));
  const int64_t per_iter = g_launches - before;
  g_launches = before;
  cudaGraph_t graph = nullptr;
  CK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle h{};
  bool loop = cudaGraphConditionalHandleCreate(&h, graph, 1u, cudaGraphCondAssignDefault) == cudaSuccess;
  if (loop) {
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    loop = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np) == cudaSuccess;
    if (loop) {
      cudaGraph_t body = np.conditional.phGraph_out[0];
      CK(cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal));
      cg_iteration<T>(c, w, c->cap_stream);
      k_cg_cond<<<1, 1, 0, c->cap_stream>>>(h, c->cgs, std::max(1, c->opt.cg_max));
      CK(cudaStreamEndCapture(c->cap_stream, &body));
    }
  }
  if (!loop) {
    (void)cudaGetLastError();   // a refused conditional node is not an error of this call
    CK(cudaGraphDestroy(graph));
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int it = 0; it < kCgGraphIters; ++it) cg_iteration<T>(c, w, c->cap_stream);
    CK(cudaStreamEndCapture(c->cap_stream, &graph));
  }
  g_launches = before;
  CK(cudaGraphInstantiate(&c->cg_exec[slot], graph, 0));
  CK(cudaGraphDestroy(graph));
  c->cg_loop[slot] = loop;
  c->cg_graph_kernels[slot] = loop ? per_iter + 1 : per_iter * kCgGraphIters;
  return c->cg_exec[slot];
}

// CG on (S + 1 1^T / (mu N^3)) x = b from x = 0, vectors of type T, FP64
// scalars.  With a loop graph the host reads the scalars once per run; else
// once per kCgGraphIters iterations.
template <typename T>
int cg_loop(kfbim_ctx* c, const T* b, const CgWs<T>& w, double tol, int maxit, cudaStream_t s, int* iters) {
  const int64_t n = c->N3;
  const bool graphs = c->use_graphs && !c->prof;
  cudaGraphExec_t exec = graphs ? cg_graph<T>(c, w) : nullptr;
  CK(cudaMemsetAsync(c->cgs, 0, sizeof(CGScalars), s));
  CK(cudaMemsetAsync(w.x, 0, n * sizeof(T), s));
  CK(cudaMemcpyAsync(w.r, b, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(w.d, b, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
  const double rank1 = c->navier ? 0.0 : 1.0 / (c->mu * (double)n);
  k_cg_init<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(b, n, c->cgs, tol * tol, rank1, c->cpen,
                                                   c->partial);
  ++g_launches;
  check_launch();
  const bool loop = graphs && c->cg_loop[Slot<T>::v];
  if (loop) CK(cudaGraphLaunch(exec, s));
  int launched = 0;
  while (true) {
    CK(cudaMemcpyAsync(c->pinned, c->cgs, sizeof(CGScalars), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (c->prof_used) prof_collect(c);
    CGScalars h;
    std::memcpy(&h, c->pinned, sizeof(CGScalars));
    *iters = h.iters;
    if (loop) g_launches += (int64_t)h.trips * c->cg_graph_kernels[Slot<T>::v];
    if (!std::isfinite(h.rr)) return KFBIM_E_NONFINITE;
    if (h.done) return KFBIM_OK;
    if (loop || launched >= maxit) return KFBIM_E_NOCONV;
    if (graphs) {
      CK(cudaGraphLaunch(exec, s));
      g_launches += c->cg_graph_kernels[Slot<T>::v];
    } else {
      for (int it = 0; it < kCgGraphIters; ++it) cg_iteration<T>(c, w, s);
    }
    launched += kCgGraphIters;
  }
}

// The CG run, and for the slab iteration the update it left pending.
template <typename T>
int cg(kfbim_ctx* c, const T* b, const CgWs<T>& w, double tol, int maxit, cudaStream_t s, int* iters) {
  const int st = cg_loop<T>(c, b, w, tol, maxit, s, iters);
  if constexpr (std::is_same<T, float>::value) {
    if (c->slab) {
      const int at = prof_begin(c, s);
      g_launches += slab_cg_finish(slab_run(c, w), s);
      prof_end(c, s, at, KFBIM_KCLASS_CG_UPDATE, 1, (double)kSlabValues[3] * c->N3 * sizeof(float));
      check_launch();
    }
  }
  return st;
}

// Solve the corrected MAC system for rhs = [f1|f2|f3|g] (FP64) -> u, p (FP64).
int grid_solve_fp64(kfbim_ctx* c, cudaStream_t s) {
  const int64_t N3 = c->N3;
  double* f = c->rhs;
  double* g = c->rhs + 3 * N3;
  double* b = c->cr;   // Schur RHS; CG copies it into its residual
  const CgWs<double> w = ws64(c);
  schur_rhs3<double, double>(c, f, w.q, w.q2, w.q3, w.T6, s);
  k_sum4<double, double><<<grid_for(N3), 256, 0, s>>>(g, w.q, w.q2, w.q3, b, N3); ++g_launches;
  check_launch();
  int it = 0;
  int st = cg<double>(c, b, w, c->opt.cg_tol, c->opt.cg_max, s, &it);
  c->cg_iters += it;
  if (st != KFBIM_OK && st != KFBIM_E_NOCONV) return st;
  // u^(c) = (1/mu)(-Delta)^{-1} (f^(c) - G_c p)
  k_f_minus_gp<double, double><<<grid_for(3 * N3), 256, 0, s>>>(f, c->p, c->gix(), c->h, c->u); ++g_launches;
  check_launch();
  face_poisson3<double>(c, c->u, c->u, w.T6, s);
  return st;
}

double relaxed_inner_tol(const kfbim_ctx* c, double tol);

// MIXED: FP32 transforms and CG inside FP64 iterative refinement.
int grid_solve_mixed(kfbim_ctx* c, cudaStream_t s) {
  const int64_t N3 = c->N3;
  double* f = c->rhs;
  double* g = c->rhs + 3 * N3;
  double* resf = c->t1;            // FP64 residual [rf (3 fields) | rg]
  double* resg = c->t1 + 3 * N3;
  double* gmean = c->scal + 4;
  double* sc = c->scal + 5;
  CK(cudaMemsetAsync(c->u, 0, 3 * N3 * sizeof(double), s));
  CK(cudaMemsetAsync(c->p, 0, N3 * sizeof(double), s));
  if (c->navier) CK(cudaMemsetAsync(gmean, 0, sizeof(double), s));
  else dot(c, g, (const double*)nullptr, N3, gmean, 1.0 / (double)N3, s);
  // u = p = 0: the first residual is [f; g - mean g] (no stencil needed)
  CK(cudaMemcpyAsync(resf, f, 3 * N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(resg, g, N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  k_shift<<<grid_for(N3), 256, 0, s>>>(resg, gmean, -1.0, N3); ++g_launches;
  check_launch();
  norm2_fast(c, resf, 4 * N3, sc, s);
  const double ref2 = read_scalar(c, sc, s);
  if (!std::isfinite(ref2)) return KFBIM_E_NONFINITE;
  int status = KFBIM_OK;
  for (int sweep = 0;; ++sweep) {
    if (sweep > 0) {
      if (c->fp32_only) break;   // FP32: one correction solve, no FP64 residual
      const int at = prof_begin(c, s);
      k_mac_residual<<<grid_for(4 * N3), 256, 0, s>>>(f, g, gmean, c->u, c->p, c->gix(), c->h, c->mu, c->cpen, resf, resg); ++g_launches;
      // reads f, g, u, p (8 N^3 doubles), writes rf, rg (4 N^3)
      prof_end(c, s, at, KFBIM_KCLASS_MAC_RESIDUAL, 1, 12.0 * N3 * sizeof(double));
      check_launch();
      norm2_fast(c, resf, 4 * N3, sc, s);
      const double r2 = read_scalar(c, sc, s);
      if (!std::isfinite(r2)) return KFBIM_E_NONFINITE;
      if (r2 <= c->refine_tol_now * c->refine_tol_now * ref2 || ref2 == 0.0) break;
      if (sweep >= c->opt.refine_max) { status = KFBIM_E_NOCONV; break; }
    }
    ++c->refine_sweeps;
    // FP32 correction solve: b = rg + (1/mu) sum G^T (-Delta)^{-1} rf
    const CgWs<float> w = ws32(c);
    float* b32 = c->fu;  // N3 floats (fu holds 3*N3)
    schur_rhs3<double, float>(c, resf, w.q, w.q2, w.q3, w.T6, s);
    k_sum4<double, float><<<grid_for(N3), 256, 0, s>>>(resg, w.q, w.q2, w.q3, b32, N3); ++g_launches;
    check_launch();
    int it = 0;
    int st = cg<float>(c, b32, w, relaxed_inner_tol(c, c->refine_tol_now), c->opt.cg_max, s, &it);
    c->cg_iters += it;
    if (st == KFBIM_E_NONFINITE) return st;
    // p += dp; u += (1/mu)(-Delta)^{-1}(rf - G dp)
    k_add_to<float><<<grid_for(N3), 256, 0, s>>>(w.x, c->p, N3); ++g_launches;
    k_f_minus_gp<float, float><<<grid_for(3 * N3), 256, 0, s>>>(resf, w.x, c->gix(), c->h, c->fu); ++g_launches;
    check_launch();
    face_poisson3<float>(c, c->fu, c->fu, w.T6, s);
    k_add_to<float><<<grid_for(3 * N3), 256, 0, s>>>(c->fu, c->u, 3 * N3); ++g_launches;
    check_launch();
  }
  if (c->navier) return status;
  // gauge: mean(p) = mu * mean(g)  (the lambda_h system with gamma = 1, alpha = mu N^3)
  dot(c, c->p, (const double*)nullptr, N3, sc, 1.0 / (double)N3, s);
  k_shift<<<grid_for(N3), 256, 0, s>>>(c->p, sc, -1.0, N3); ++g_launches;
  k_shift<<<grid_for(N3), 256, 0, s>>>(c->p, gmean, c->mu, N3); ++g_launches;
  check_launch();
  return status;
}

// Full interface solve: jumps -> RHS -> grid solve.  Leaves J, u, p in ctx.
int interface_solve(kfbim_ctx* c, const double* phi, const double* fpts, const double* fgrid,
                    cudaStream_t s) {
  const int64_t n = c->n_all;
  const int at = prof_begin(c, s);
  k_jumps<<<(unsigned)((n + JB - 1) / JB), 3 * JB, 0, s>>>(
      phi, fpts, n, c->d_comp, c->d_pid, c->d_fit_off, c->d_fit_col, c->d_fit_w, c->fit_ell, c->d_jmap,
      c->J); ++g_launches;
  // fit rows (column index, six weights, the density value), the 11 x 18 jump
  // map, the forcing and the twelve jump slots per point
  prof_end(c, s, at, KFBIM_KCLASS_JUMPS, 1,
           (double)c->fit_ell * (4 + 6 * 8 + 8) + (double)n * 8 * (11 * 18 + 3 * (fpts ? 1 : 0) + 12));
  check_launch();
  k_rhs_fill<<<grid_for(4 * c->N3), 256, 0, s>>>(fgrid, c->d_side[1], c->d_side[2], c->d_side[3],
                                                  c->gix(), c->rhs); ++g_launches;
  check_launch();
  if (c->n_corr_rows > 0) {
    k_corrections<<<grid_for(c->n_corr_rows), 256, 0, s>>>(c->d_corr_row, c->d_corr_ptr, c->d_corr_src,
                                                            c->d_corr_coef, c->n_corr_rows, c->J, c->rhs); ++g_launches;
    check_launch();
  }
  ++c->interface_solves;
  return c->opt.precision == KFBIM_MIXED ? grid_solve_mixed(c, s) : grid_solve_fp64(c, s);
}

void trace(kfbim_ctx* c, const double* u, const double* J, double* out, cudaStream_t s) {
  k_trace<<<grid_for(c->n_prim), 256, 0, s>>>(u, J, c->n_all, c->n_prim, c->d_prim_of, c->N,
                                               c->d_tr_comp, c->d_tr_node, c->d_tr_w, c->d_tr_cj, out); ++g_launches;
  check_launch();
}

int apply_impl(kfbim_ctx* c, const double* phi, double* out, cudaStream_t s) {
  int st = interface_solve(c, phi, nullptr, nullptr, s);
  if (st != KFBIM_OK && st != KFBIM_E_NOCONV) return st;
  trace(c, c->u, c->J, out, s);
  return st;
}

// GMRES (Alg. 1 step 3): unrestarted, CGS2 on the device, Givens on the host;
// with `adjoint`, GMRES on the transposed matvec.
int adjoint_apply(kfbim_ctx* c, const double* lam, double* out, cudaStream_t s);

// Inexact GMRES (relaxation of the matvec accuracy as the residual falls):
// the grid solve of the matvec that extends the Krylov basis from a relative
// residual res need only be accurate to relax * gmres_tol / res, because its
// error enters the solution through a coefficient of size about res, so the
// product stays about relax * gmres_tol however loose the matvec gets.  The
// MIXED refinement stops at that relative residual (never above kRelaxCap,
// never below refine_tol); relax = 0 keeps refine_tol throughout.
constexpr double kRelaxCap = 1e-4;

double relaxed_refine_tol(const kfbim_ctx* c, double res) {
  if (!(c->relax > 0.0) || !(res > 0.0)) return c->opt.refine_tol;
  return std::max(c->opt.refine_tol, std::min(kRelaxCap, c->relax * c->opt.gmres_tol / res));
}

// The FP32 CG tolerance of a grid solve refined to relative residual `tol`:
// inner_tol, or looser with the relaxed refinement tolerance, 0.3 of it (a
// refinement stopping at 1e-5 has no use for an inner solve to 3e-6).
constexpr double kInnerRelaxFactor = 0.3;
constexpr double kInnerRelaxCap = 1e-4;
double relaxed_inner_tol(const kfbim_ctx* c, double tol) {
  if (!(tol > c->opt.refine_tol)) return c->opt.inner_tol;
  return std::max(c->opt.inner_tol, std::min(kInnerRelaxCap, kInnerRelaxFactor * tol));
}

int gmres(kfbim_ctx* c, const double* rhs, double* x, cudaStream_t s, int* iters, double* res_out,
          bool adjoint = false) {
  const int64_t n = c->n_prim;
  const int m = c->gm_max;
  const int64_t ld = n;
  double* sc = c->scal;
  dot(c, rhs, rhs, n, sc, 1.0, s);
  const double beta = std::sqrt(read_scalar(c, sc, s));
  if (!std::isfinite(beta)) return KFBIM_E_NONFINITE;
  if (beta == 0.0) {
    CK(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    *iters = 0;
    *res_out = 0.0;
    return KFBIM_OK;
  }
  k_scale_copy<<<grid_for(n), 256, 0, s>>>(rhs, 1.0 / beta, nullptr, c->V, n); ++g_launches;
  check_launch();
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), gvec(m + 1, 0.0), hcol(m + 1);
  gvec[0] = beta;
  int k = 0;
  int status = KFBIM_E_NOCONV;
  double res = 1.0;
  const int nb = 64;
  struct ResetTol {
    kfbim_ctx* c;
    ~ResetTol() { c->refine_tol_now = c->opt.refine_tol; }
  } reset_tol{c};
  for (k = 1; k <= m; ++k) {
    c->refine_tol_now = relaxed_refine_tol(c, res);
    int st = adjoint ? adjoint_apply(c, c->V + (int64_t)(k - 1) * ld, c->gw, s)
                     : apply_impl(c, c->V + (int64_t)(k - 1) * ld, c->gw, s);
    if (st != KFBIM_OK && st != KFBIM_E_NOCONV) return st;
    std::fill(hcol.begin(), hcol.end(), 0.0);
    for (int pass2 = 0; pass2 < 2; ++pass2) {
      dim3 grid(nb, k);
      k_multidot_partial<<<grid, RED_THREADS, 0, s>>>(c->V, ld, c->gw, n, c->partial); ++g_launches;
      k_sum_partials<<<k, RED_THREADS, 0, s>>>(c->partial, nb, 1.0, c->gh); ++g_launches;
      k_multi_axpy<<<grid_for(n), 256, 0, s>>>(c->V, ld, c->gh, k, c->gw, n, 0); ++g_launches;
      check_launch();
      CK(cudaMemcpyAsync(c->pinned, c->gh, k * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int j = 0; j < k; ++j) hcol[j] += c->pinned[j];
    }
    dot(c, c->gw, c->gw, n, sc, 1.0, s);
    const double hn = std::sqrt(read_scalar(c, sc, s));
    if (!std::isfinite(hn)) return KFBIM_E_NONFINITE;
    hcol[k] = hn;
    for (int j = 0; j < k - 1; ++j) {
      const double a = hcol[j], b = hcol[j + 1];
      hcol[j] = cs[j] * a + sn[j] * b;
      hcol[j + 1] = -sn[j] * a + cs[j] * b;
    }
    const double a = hcol[k - 1], b = hcol[k];
    const double r = std::hypot(a, b);
    cs[k - 1] = (r == 0.0) ? 1.0 : a / r;
    sn[k - 1] = (r == 0.0) ? 0.0 : b / r;
    hcol[k - 1] = r;
    hcol[k] = 0.0;
    gvec[k] = -sn[k - 1] * gvec[k - 1];
    gvec[k - 1] = cs[k - 1] * gvec[k - 1];
    for (int j = 0; j < k; ++j) H[(size_t)j * m + (k - 1)] = hcol[j];
    res = std::fabs(gvec[k]) / beta;
    if (res < c->opt.gmres_tol || hn == 0.0) {
      status = KFBIM_OK;
      break;
    }
    if (k < m) {
      k_scale_copy<<<grid_for(n), 256, 0, s>>>(c->gw, 1.0 / hn, nullptr, c->V + (int64_t)k * ld, n); ++g_launches;
      check_launch();
    }
  }
  const int kk = std::min(k, m);
  std::vector<double> y(kk, 0.0);
  for (int i = kk - 1; i >= 0; --i) {
    double acc = gvec[i];
    for (int j = i + 1; j < kk; ++j) acc -= H[(size_t)i * m + j] * y[j];
    y[i] = acc / H[(size_t)i * m + i];
  }
  CK(cudaMemcpyAsync(c->gy, y.data(), kk * sizeof(double), cudaMemcpyHostToDevice, s));
  k_multi_axpy<<<grid_for(n), 256, 0, s>>>(c->V, ld, c->gy, kk, x, n, 1); ++g_launches;
  check_launch();
  CK(cudaStreamSynchronize(s));
  *iters = kk;
  *res_out = res;
  return status;
}

// ------------------------------------------------------------ adjoint
// A phi = T_u K^-1 C J(phi) + T_J J(phi) (trace of the interface solve), so
// A^T lam = J^T (C^T K^-T (T_u^T lam, 0) + T_J^T lam).  K is the corrected MAC
// operator [mu L, G; D, c I] with D = -G^T (c = 0, plus the lambda_h
// projection and gauge, for Stokes): with S = diag(I, -I), K^T = S K S, so
// K^-T (w, 0) = (u', -p') where (u', p') is the forward grid solve of (w, 0).
template <typename V>
void csr_by_key(std::vector<std::pair<int64_t, V>>& e, std::vector<int64_t>& key, std::vector<int64_t>& ptr,
                std::vector<V>& val) {
  std::stable_sort(e.begin(), e.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  ptr.assign(1, 0);
  for (size_t k = 0; k < e.size(); ++k) {
    if (k == 0 || e[k].first != e[k - 1].first) {
      if (k > 0) ptr.push_back((int64_t)k);
      key.push_back(e[k].first);
    }
    val.push_back(e[k].second);
  }
  ptr.push_back((int64_t)e.size());
}

void adjoint_tables(kfbim_ctx* c) {
  if (c->adj_ready) return;
  const HostTables& t = c->host;
  const int64_t N3 = c->N3;
  {  // trace rows by face-grid node
    std::vector<std::pair<int64_t, std::pair<int32_t, double>>> e;
    for (int64_t q = 0; q < t.n_prim; ++q)
      for (int i = 0; i < kStencil; ++i)
        e.push_back({(int64_t)(t.tr_comp[q] - 1) * N3 + t.tr_node[kStencil * q + i],
                     {(int32_t)q, t.tr_w[kStencil * q + i]}});
    std::vector<int64_t> key, ptr;
    std::vector<std::pair<int32_t, double>> val;
    csr_by_key(e, key, ptr, val);
    std::vector<int32_t> qv;
    std::vector<double> wv;
    for (const auto& v : val) {
      qv.push_back(v.first);
      wv.push_back(v.second);
    }
    c->ta_n = (int64_t)key.size();
    c->d_ta_key = upload(c, key);
    c->d_ta_ptr = upload(c, ptr);
    c->d_ta_q = upload(c, qv);
    c->d_ta_w = upload(c, wv);
  }
  {  // correction rows by jump slot
    std::vector<std::pair<int64_t, std::pair<int64_t, double>>> e;
    for (size_t r = 0; r + 1 < t.corr_ptr.size(); ++r)
      for (int64_t k = t.corr_ptr[r]; k < t.corr_ptr[r + 1]; ++k)
        e.push_back({t.corr_src[k], {t.corr_row[r], t.corr_coef[k]}});
    std::vector<int64_t> key, ptr;
    std::vector<std::pair<int64_t, double>> val;
    csr_by_key(e, key, ptr, val);
    std::vector<int64_t> row;
    std::vector<double> coef;
    for (const auto& v : val) {
      row.push_back(v.first);
      coef.push_back(v.second);
    }
    c->ca_n = (int64_t)key.size();
    c->d_ca_key = upload(c, key);
    c->d_ca_ptr = upload(c, ptr);
    c->d_ca_row = upload(c, row);
    c->d_ca_coef = upload(c, coef);
  }
  {  // fit entries by primary column
    std::vector<std::vector<std::pair<int64_t, int64_t>>> bycol(std::max<int64_t>(1, t.n_prim));
    for (int64_t rr = 0; rr + 1 < (int64_t)t.fit_ptr.size(); ++rr)
      for (int64_t q = t.fit_ptr[rr]; q < t.fit_ptr[rr + 1]; ++q) bycol[t.fit_col[q]].emplace_back(q, rr);
    std::vector<int64_t> ptr{0};
    std::vector<int32_t> qv, rv;
    for (int64_t col = 0; col < t.n_prim; ++col) {
      for (const auto& pr : bycol[col]) {
        qv.push_back(c->fit_pos[pr.first]);
        rv.push_back((int32_t)pr.second);
      }
      ptr.push_back((int64_t)qv.size());
    }
    c->d_fa_ptr = upload(c, ptr);
    c->d_fa_q = upload(c, qv);
    c->d_fa_rr = upload(c, rv);
  }
  c->d_Jbar = dalloc<double>(c, kSlots * c->n_all);
  c->d_Dbar = dalloc<double>(c, 18 * c->n_all);
  c->adj_ready = true;
}

// rhs = [ubar | 0] and Jbar hold the adjoint inputs of the interface solve:
// out = J^T (C^T K^-T rhs + Jbar).
int adjoint_tail(kfbim_ctx* c, double* out, cudaStream_t s) {
  const int64_t N3 = c->N3, n = c->n_all;
  ++c->interface_solves;
  int st = c->opt.precision == KFBIM_MIXED ? grid_solve_mixed(c, s) : grid_solve_fp64(c, s);
  if (st != KFBIM_OK && st != KFBIM_E_NOCONV) return st;
  double* rbar = c->t1;   // [u' | -p'] (4 N^3)
  CK(cudaMemcpyAsync(rbar, c->u, 3 * N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  k_scale_copy<<<grid_for(N3), 256, 0, s>>>(c->p, -1.0, nullptr, rbar + 3 * N3, N3); ++g_launches;
  if (c->ca_n > 0) {
    k_corrections_T<<<grid_for(c->ca_n), 256, 0, s>>>(c->d_ca_key, c->d_ca_ptr, c->d_ca_row, c->d_ca_coef, c->ca_n,
                                                       rbar, c->d_Jbar); ++g_launches;
  }
  k_jumps_T<<<grid_for(n), 256, 0, s>>>(c->d_Jbar, n, c->d_comp, c->d_pid, c->d_jmap, c->d_Dbar); ++g_launches;
  k_fit_T<<<grid_for(c->n_prim), 256, 0, s>>>(c->d_fa_ptr, c->d_fa_q, c->d_fa_rr, c->d_fit_w, c->fit_ell, c->d_Dbar,
                                               c->d_Jbar, c->d_prim_of, c->n_prim, out); ++g_launches;
  check_launch();
  return st;
}

// out = A^T lam (primary points).
int adjoint_apply(kfbim_ctx* c, const double* lam, double* out, cudaStream_t s) {
  adjoint_tables(c);
  const int64_t N3 = c->N3;
  CK(cudaMemsetAsync(c->rhs, 0, 4 * N3 * sizeof(double), s));
  CK(cudaMemsetAsync(c->d_Jbar, 0, kSlots * c->n_all * sizeof(double), s));
  if (c->ta_n > 0) {
    k_trace_T_u<<<grid_for(c->ta_n), 256, 0, s>>>(c->d_ta_key, c->d_ta_ptr, c->d_ta_q, c->d_ta_w, c->ta_n, lam,
                                                   c->rhs); ++g_launches;
  }
  k_trace_T_J<<<grid_for(c->n_prim), 256, 0, s>>>(lam, c->n_all, c->n_prim, c->d_prim_of, c->d_tr_cj, c->d_Jbar);
  ++g_launches;
  check_launch();
  return adjoint_tail(c, out, s);
}

// out = U^T ubar, U: phi -> interface-solve velocity (3 face fields).
int adjoint_from_u(kfbim_ctx* c, const double* ubar, double* out, cudaStream_t s) {
  adjoint_tables(c);
  k_adjoint_rhs<<<grid_for(4 * c->N3), 256, 0, s>>>(ubar, c->gix(), c->rhs); ++g_launches;
  CK(cudaMemsetAsync(c->d_Jbar, 0, kSlots * c->n_all * sizeof(double), s));
  check_launch();
  return adjoint_tail(c, out, s);
}

// Transform matrices of the tensor-core passes, M[a][n] (output a, input n),
// for the six transforms of transforms.cuh at N = 128, split into TF32 hi/lo
// parts and stored column-major ([type][hi|lo][n][a]) so that lane a of a warp
// reads row a.  TF32 rounding: round to nearest, ties away from zero, on the
// 13 low mantissa bits.
std::vector<float> tc_matrices(int N) {
  auto tf32 = [](float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
  };
  std::vector<float> out((size_t)6 * 2 * N * N);
  const double pi = M_PI;
  for (int type = 1; type <= 6; ++type) {
    for (int a = 0; a < N; ++a)
      for (int n = 0; n < N; ++n) {
        double m = 0.0;
        switch (type) {
          case X_DCT2F: m = std::cos(pi * a * (n + 0.5) / N); break;
          case X_DCT2I: m = (n == 0 ? 1.0 : 2.0) / N * std::cos(pi * n * (a + 0.5) / N); break;
          case X_DST2F: m = std::sin(pi * (a + 1) * (n + 0.5) / N); break;
          case X_DST2I: m = (n == N - 1 ? 1.0 : 2.0) / N * std::sin(pi * (n + 1) * (a + 0.5) / N); break;
          case X_DST1F: m = (a > 0 && n > 0) ? std::sin(pi * (double)a * n / N) : 0.0; break;
          case X_DST1I: m = (a > 0 && n > 0) ? 2.0 / N * std::sin(pi * (double)a * n / N) : 0.0; break;
        }
        const float hi = tf32((float)m);
        const float lo = tf32((float)(m - (double)hi));
        const size_t base = (size_t)(type - 1) * 2 * N * N;
        out[base + (size_t)n * N + a] = hi;
        out[base + (size_t)N * N + (size_t)n * N + a] = lo;
      }
  }
  return out;
}

void check_tc(kfbim_ctx* c, cudaStream_t s) {
  if (!c->d_tc_err) return;
  int e = 0;
  CK(cudaMemcpyAsync(&e, c->d_tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (e) throw CudaError{"tensor-core transform pass: an mbarrier wait timed out"};
}

// Autotuner of the FP32 axis passes (N = 128): times a plain three-job stage
// (DST-II along z/z/y) and a fused three-job stage (DCT-II, Schur weight,
// DCT-III along each component's axis) with the FFT kernel and with the
// tensor-core kernel on the FP32 stage temporaries, and keeps the faster
// kernel for each stage kind.  The tensor-core passes are less accurate (TF32
// products accumulate in the tensor core's FP32 adder, about 2e-6 relative
// against about 2e-7 for the FFT), which costs the MIXED refinement a third
// sweep per interface solve: on star128 the Schur CG iterations per solve grew
// from 1642 to 2489.  A tensor-core stage is therefore chosen only when it is
// faster than the FFT stage by that factor.
constexpr float kTcIterationFactor = 1.5f;
void autotune(kfbim_ctx* c) {
  const int64_t n = c->N3;
  float* X = c->fT6;
  cudaStream_t s = c->cap_stream;
  CK(cudaMemsetAsync(X, 0, 6 * n * sizeof(float), s));
  const std::vector<Job> plain = {{X, X + 3 * n, 2, X_DST2F, X_NONE, W_NONE, 0, 0},
                                  {X + n, X + 4 * n, 2, X_DST2F, X_NONE, W_NONE, 1, 0},
                                  {X + 2 * n, X + 5 * n, 1, X_DST2F, X_NONE, W_NONE, 2, 0}};
  const std::vector<Job> fused = {{X + 3 * n, X, 0, X_DCT2F, X_DCT2I, W_SCHUR, 0, 0},
                                  {X + 4 * n, X + n, 1, X_DCT2F, X_DCT2I, W_SCHUR, 1, 0},
                                  {X + 5 * n, X + 2 * n, 2, X_DCT2F, X_DCT2I, W_SCHUR, 2, 0}};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int64_t launches0 = g_launches;
  auto time_stage = [&](const std::vector<Job>& list) {
    for (int w = 0; w < 2; ++w) stage_list<float, float, float>(c, list, s);
    const int reps = 10;
    CK(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) stage_list<float, float, float>(c, list, s);
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    return ms / reps;
  };
  c->xf_plain = 0;
  c->tune_ms[0] = time_stage(plain);
  c->xf_plain = 1;
  c->tune_ms[1] = time_stage(plain);
  c->xf_fused = 0;
  c->tune_ms[2] = time_stage(fused);
  c->xf_fused = 1;
  c->tune_ms[3] = time_stage(fused);
  CK(cudaEventDestroy(e0));
  CK(cudaEventDestroy(e1));
  g_launches = launches0;
  check_tc(c, s);
  c->xf_plain = c->tune_ms[1] * kTcIterationFactor < c->tune_ms[0];
  c->xf_fused = c->tune_ms[3] * kTcIterationFactor < c->tune_ms[2];
}

void fill_tables(kfbim_ctx* c) {
  HostTables& t = c->host;
  const int N = c->N;
  c->d_comp = upload(c, t.comp);
  c->d_pid = upload(c, t.pid);
  {
    // the fit rows interleaved by groups of 32 (a warp of k_jumps reads one
    // entry of each of its 32 rows with one coalesced load per array), the
    // weights weight-major within that layout; input-major jump maps
    const int64_t rows = (int64_t)t.fit_ptr.size() - 1;
    const int64_t groups = (rows + 31) / 32;
    std::vector<int64_t> off(groups + 1, 0);
    for (int64_t g = 0; g < groups; ++g) {
      int64_t len = 0;
      for (int64_t r = 32 * g; r < std::min(rows, 32 * g + 32); ++r)
        len = std::max(len, t.fit_ptr[r + 1] - t.fit_ptr[r]);
      off[g + 1] = off[g] + 32 * len;
    }
    const int64_t E = off[groups];
    if (E > INT32_MAX) throw CudaError{"surface fit table too large", KFBIM_E_INVALID};
    std::vector<int32_t> col(std::max<int64_t>(E, 1), 0);
    std::vector<double> fw((size_t)kFitW * std::max<int64_t>(E, 1), 0.0);
    c->fit_pos.assign(t.fit_col.size(), 0);
    for (int64_t r = 0; r < rows; ++r)
      for (int64_t q = t.fit_ptr[r]; q < t.fit_ptr[r + 1]; ++q) {
        const int64_t pos = off[r / 32] + 32 * (q - t.fit_ptr[r]) + (r % 32);
        col[pos] = t.fit_col[q];
        for (int k = 0; k < kFitW; ++k) fw[(size_t)k * E + pos] = t.fit_w[kFitW * q + k];
        c->fit_pos[q] = (int32_t)pos;
      }
    c->fit_ell = E;
    c->d_fit_off = upload(c, off);
    c->d_fit_col = upload(c, col);
    c->d_fit_w = upload(c, fw);
    std::vector<double> jm(t.jmap.size());
    for (int64_t y = 0; y < t.n_all; ++y)
      for (int r = 0; r < kMapOut; ++r)
        for (int q = 0; q < kMapIn; ++q)
          jm[((size_t)y * kMapIn + q) * kMapOut + r] = t.jmap[((size_t)y * kMapOut + r) * kMapIn + q];
    c->d_jmap = upload(c, jm);
  }
  c->d_corr_row = upload(c, t.corr_row);
  c->d_corr_ptr = upload(c, t.corr_ptr);
  c->d_corr_src = upload(c, t.corr_src);
  c->d_corr_coef = upload(c, t.corr_coef);
  c->n_corr_rows = (int64_t)t.corr_row.size();
  c->d_tr_comp = upload(c, t.tr_comp);
  c->d_tr_node = upload(c, t.tr_node);
  c->d_tr_w = upload(c, t.tr_w);
  c->d_tr_cj = upload(c, t.tr_cj);
  std::vector<int64_t> prim_of;
  for (int64_t y = 0; y < t.n_all; ++y)
    if (t.primary[y]) prim_of.push_back(y);
  c->d_prim_of = upload(c, prim_of);
  c->d_xyz = upload(c, t.xyz);
  for (int g = 0; g < 4; ++g) c->d_side[g] = upload(c, t.side[g]);
  // twiddles exp(-2 pi i t / 2N), t < N; post twiddles exp(-i pi k / 2N), k < N
  std::vector<C2<double>> tw(N), q(N);
  std::vector<C2<float>> tw32(N), q32(N);
  for (int k = 0; k < N; ++k) {
    const double a = M_PI * (double)k / (double)N;
    tw[k] = {std::cos(a), -std::sin(a)};
    const double b = 0.5 * a;
    q[k] = {std::cos(b), -std::sin(b)};
    tw32[k] = {(float)tw[k].x, (float)tw[k].y};
    q32[k] = {(float)q[k].x, (float)q[k].y};
  }
  std::vector<C2<double>> twc(2 * N);
  std::vector<C2<float>> twc32(2 * N);
  for (int k = 0; k < 2 * N; ++k) {
    const double a = M_PI * (double)k / (double)N;
    twc[k] = {std::cos(a), -std::sin(a)};
    twc32[k] = {(float)twc[k].x, (float)twc[k].y};
  }
  c->d_twc64 = upload(c, twc);
  c->d_twc32 = upload(c, twc32);
  c->d_tw64 = upload(c, tw);
  c->d_q64 = upload(c, q);
  c->d_tw32 = upload(c, tw32);
  c->d_q32 = upload(c, q32);
  std::vector<double> s2(2 * N);
  for (int i = 0; i < N; ++i) {
    const double a = std::sin(M_PI * i / (2.0 * N)), b = std::sin(M_PI * (i + 1) / (2.0 * N));
    s2[i] = 4.0 * a * a;
    s2[N + i] = 4.0 * b * b;
  }
  c->d_s2 = upload(c, s2);
  std::vector<float> s2f(s2.begin(), s2.end());
  c->d_s2f = upload(c, s2f);
  // workspace
  const int64_t N3 = c->N3;
  c->J = dalloc<double>(c, kSlots * t.n_all);
  c->rhs = dalloc<double>(c, 4 * N3);
  c->u = dalloc<double>(c, 3 * N3);
  c->p = dalloc<double>(c, N3);
  c->t1 = dalloc<double>(c, 4 * N3);   // also the FP64 residual [rf | rg] of MIXED
  c->t2 = dalloc<double>(c, N3);
  c->cr = dalloc<double>(c, N3);
  c->cd = dalloc<double>(c, N3);
  c->cq = dalloc<double>(c, N3);
  c->rres = dalloc<double>(c, N3);
  c->zero_phi = dalloc<double>(c, std::max<int64_t>(1, t.n_prim));
  CK(cudaMemsetAsync(c->zero_phi, 0, std::max<int64_t>(1, t.n_prim) * sizeof(double), c->setup_stream));
  c->partial = dalloc<double>(c, (size_t)RED_BLOCKS * 256);
  c->scal = dalloc<double>(c, 64);
  c->cgs = dalloc<CGScalars>(c, 1);
  c->q2 = dalloc<double>(c, N3);
  c->q3 = dalloc<double>(c, N3);
  c->T6 = dalloc<double>(c, 6 * N3);
  if (c->opt.precision == KFBIM_MIXED) {
    c->fq2 = dalloc<float>(c, N3);
    c->fq3 = dalloc<float>(c, N3);
    c->fT6 = dalloc<float>(c, 6 * N3);
    c->f1 = dalloc<float>(c, N3);
    c->f2 = dalloc<float>(c, N3);
    c->fx = dalloc<float>(c, N3);
    c->fr = dalloc<float>(c, N3);
    c->fd = dalloc<float>(c, N3);
    c->fq = dalloc<float>(c, N3);
    c->fu = dalloc<float>(c, 3 * N3);
  }
  c->gm_max = c->opt.gmres_max;
  c->V = dalloc<double>(c, (size_t)(c->gm_max + 1) * std::max<int64_t>(1, t.n_prim));
  c->gw = dalloc<double>(c, std::max<int64_t>(1, t.n_prim));
  c->gh = dalloc<double>(c, c->gm_max + 1);
  c->grhs = dalloc<double>(c, std::max<int64_t>(1, t.n_prim));
  c->gy = dalloc<double>(c, c->gm_max + 1);
  CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  void* ph = nullptr;
  CK(cudaMallocHost(&ph, sizeof(double) * 256));
  c->pinned = static_cast<double*>(ph);
  if (c->opt.precision == KFBIM_MIXED && slab_supported(N) && c->opt.transforms != KFBIM_XF_TENSOR &&
      c->opt.transforms != KFBIM_XF_STAGED) {
    CK(slab_prepare(N));
    c->slab = true;
  }
  // the autotuner below runs on the capture stream: the uploads come first
  CK(cudaStreamSynchronize(c->setup_stream));
  if (c->opt.precision == KFBIM_MIXED && N == TC_N &&
      (c->opt.transforms == KFBIM_XF_AUTO || c->opt.transforms == KFBIM_XF_TENSOR)) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev));
    c->d_tc_mats = upload(c, tc_matrices(N));
    c->d_tc_err = dalloc<int>(c, 1);
    CK(cudaMemsetAsync(c->d_tc_err, 0, sizeof(int), c->setup_stream));
    if (c->opt.transforms == KFBIM_XF_TENSOR) {
      c->xf_plain = c->xf_fused = 1;
    } else {
      autotune(c);
    }
  }
}

int fail(kfbim_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

// Makes a context's device current for the duration of a call and gives the
// calling thread its own current device back afterwards: the context's
// memory, streams and graphs belong to the device it was set up on.  A
// negative device (host-only context) makes no CUDA call.
class DeviceScope {
 public:
  explicit DeviceScope(int dev) {
    if (dev < 0) return;
    st_ = cudaGetDevice(&prev_);
    if (st_ == cudaSuccess && prev_ != dev) {
      st_ = cudaSetDevice(dev);
      switched_ = st_ == cudaSuccess;
    }
  }
  ~DeviceScope() {
    if (switched_) cudaSetDevice(prev_);
  }
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;
  cudaError_t status() const { return st_; }

 private:
  int prev_ = 0;
  bool switched_ = false;
  cudaError_t st_ = cudaSuccess;
};

// Runs one entry point on a device context: on its device, with every C++
// exception turned into a status (none crosses the C ABI).
template <typename F>
int guarded(kfbim_ctx* c, F&& f) {
  if (!c) return KFBIM_E_INVALID;
  if (!c->device) return fail(c, KFBIM_E_INVALID, "host-only context");
  const DeviceScope scope(c->dev_id);
  if (scope.status() != cudaSuccess)
    return fail(c, KFBIM_E_CUDA, std::string("selecting the context's device: ") + cudaGetErrorString(scope.status()));
  try {
    return f();
  } catch (const CudaError& e) {
    return fail(c, e.code, e.msg);
  } catch (const std::bad_alloc&) {
    return fail(c, KFBIM_E_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(c, KFBIM_E_INVALID, std::string("internal error: ") + e.what());
  }
}

void reset_counters(kfbim_ctx* c) {
  c->cg_iters = 0;
  c->refine_sweeps = 0;
  c->interface_solves = 0;
}

}  // namespace

// ------------------------------------------------ allocation-free Poisson
// kfbim_poisson_noalloc runs the same five transform passes as kfbim_poisson
// without a context: its two scratch fields and its twiddle and eigenvalue
// tables live in the file-scope device arrays below, sized for N <= 64.
// In host code these names are only stand-ins for the device symbols; the
// device addresses are fetched with cudaGetSymbolAddress once per device.
namespace {
constexpr int kNoAllocMaxN = 64;
static __device__ __align__(256) double g_na_scratch[2 * kNoAllocMaxN * kNoAllocMaxN * kNoAllocMaxN];
static __device__ __align__(256) C2<double> g_na_tw[kNoAllocMaxN];
static __device__ __align__(256) C2<double> g_na_q[kNoAllocMaxN];
static __device__ __align__(256) double g_na_s2[2 * kNoAllocMaxN];

struct NoAllocSymbols {
  bool ready = false;
  double* scratch = nullptr;
  C2<double>* tw = nullptr;
  C2<double>* q = nullptr;
  double* s2 = nullptr;
};
constexpr int kMaxDevices = 64;
NoAllocSymbols g_na_dev[kMaxDevices];
std::mutex g_na_mutex;

// Twiddles exp(-2 pi i t / 2N), post-twiddles exp(-i pi k / 2N) and the
// one-dimensional Laplacian eigenvalues 4 sin^2 for length N (rewritten on
// every call, so consecutive calls with different N are consistent).
__global__ void k_na_tables(int N, C2<double>* tw, C2<double>* q, double* s2) {
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    double sn, cs;
    sincospi((double)k / (double)N, &sn, &cs);
    tw[k] = {cs, -sn};
    sincospi(0.5 * (double)k / (double)N, &sn, &cs);
    q[k] = {cs, -sn};
    const double a = sinpi(0.5 * (double)k / (double)N), b = sinpi(0.5 * (double)(k + 1) / (double)N);
    s2[k] = 4.0 * a * a;
    s2[N + k] = 4.0 * b * b;
  }
}

// The device addresses of the static arrays on the current device.  Outside
// a stream capture they are looked up on every call (a lookup, no
// allocation), so a context torn down by cudaDeviceReset never leaves stale
// addresses behind; inside a capture, where the lookup may have to load the
// module and is not allowed, the addresses of the last call on this device
// are used, and a first call under capture is rejected.
int noalloc_symbols(cudaStream_t s, NoAllocSymbols** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return KFBIM_E_CUDA;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return KFBIM_E_CUDA;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  NoAllocSymbols& d = g_na_dev[dev];
  if (cap != cudaStreamCaptureStatusNone) {
    if (!d.ready) {
      std::fprintf(stderr, "kfbim_poisson_noalloc: the first call on a device must come before any "
                           "stream capture\n");
      return KFBIM_E_INVALID;
    }
    *out = &d;
    return KFBIM_OK;
  }
  NoAllocSymbols f;
  cudaError_t e = cudaGetSymbolAddress((void**)&f.scratch, g_na_scratch);
  if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&f.tw, g_na_tw);
  if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&f.q, g_na_q);
  if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&f.s2, g_na_s2);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "kfbim_poisson_noalloc: resolving the static scratch failed: %s\n",
                 cudaGetErrorString(e));
    return KFBIM_E_CUDA;
  }
  f.ready = true;
  d = f;
  *out = &d;
  return KFBIM_OK;
}

// One pass of the allocation-free Poisson solve; returns the launch's own
// status (cudaLaunchKernel reports it directly, so an error left behind by
// unrelated earlier work is neither reported as this call's nor cleared).
cudaError_t noalloc_pass(const NoAllocSymbols& d, int N, double h, const double* in, double* out, int axis,
                         int t0, int t1, int wmode, int wc, cudaStream_t s) {
  PassArgs a{};  // value-initialised: every field, skip included, starts at zero
  a.N = N;
  a.axis = axis;
  a.type0 = t0;
  a.type1 = t1;
  a.wmode = wmode;
  a.wc = wc;
  for (int b = 0; b < 3; ++b) a.kind[b] = (b == wc) ? 0 : 1;
  a.mu = 1.0;
  a.h = h;
  a.accumulate = 0;
  a.scale = 1.0;
  a.skip = nullptr;
  // N <= 64 in FP64 needs at most 40 KiB of dynamic shared memory, within the
  // 48 KiB default; the kernel's limit may only have been raised by other
  // paths of this library (raise_dynamic_smem never lowers it)
  const size_t smem = pass_smem_bytes(N, sizeof(double));
  const C2<double>* tw = d.tw;
  const C2<double>* q = d.q;
  const double* s2 = d.s2;
  void* args[] = {(void*)&in, (void*)&out, (void*)&a, (void*)&tw, (void*)&q, (void*)&s2};
  return cudaLaunchKernel((const void*)k_axis_pass<double, double, double>, dim3((unsigned)(N * N / LPC)),
                          dim3(PASS_THREADS), args, smem, s);
}
}  // namespace

// ------------------------------------------------------------------ batch
// Several boundary-data instances on one geometry (MIXED precision), solved in
// lockstep: every transform stage is one launch for all active instances (three
// jobs per instance, each with its instance's CG done flag), the CG and
// refinement loops stop per instance, and GMRES advances all unconverged
// instances with one batched matvec per iteration.
namespace {

void batch_alloc(kfbim_ctx* c, int B) {
  if (B <= c->bcap) return;
  if (c->bcg_exec) CK(cudaGraphExecDestroy(c->bcg_exec));   // it holds the old slot scalars
  c->bcg_exec = nullptr;
  c->bcg_tried = false;
  const int64_t N3 = c->N3, np = std::max<int64_t>(1, c->n_prim);
  c->bm = c->opt.gmres_max;
  c->bgh = dalloc<double>(c, (size_t)B * (c->bm + 1));
  for (int b = 0; b < c->bcap; ++b) c->bs[b].gh = c->bgh + (size_t)b * (c->bm + 1);
  for (int b = c->bcap; b < B; ++b) {
    kfbim_ctx::Slot sl{};
    sl.J = dalloc<double>(c, kSlots * c->n_all);
    sl.rhs = dalloc<double>(c, 4 * N3);
    sl.u = dalloc<double>(c, 3 * N3);
    sl.p = dalloc<double>(c, N3);
    sl.res = dalloc<double>(c, 4 * N3);
    sl.grhs = dalloc<double>(c, np);
    sl.V = dalloc<double>(c, (size_t)(c->bm + 1) * np);
    sl.gw = dalloc<double>(c, np);
    sl.gh = c->bgh + (size_t)b * (c->bm + 1);
    sl.gy = dalloc<double>(c, c->bm + 1);
    sl.x = dalloc<float>(c, N3);
    sl.r = dalloc<float>(c, N3);
    sl.d = dalloc<float>(c, N3);
    sl.q = dalloc<float>(c, N3);
    sl.q2 = dalloc<float>(c, N3);
    sl.q3 = dalloc<float>(c, N3);
    sl.T6 = dalloc<float>(c, 6 * N3);
    sl.fu = dalloc<float>(c, 3 * N3);
    c->bs.push_back(sl);
  }
  c->bcgs = dalloc<CGScalars>(c, B);
  c->bscal = dalloc<double>(c, 8 * (size_t)B);
  c->bpartial = dalloc<double>(c, (size_t)kRunPartials * B);
  if (c->bpinned) CK(cudaFreeHost(c->bpinned));
  c->bpinned = nullptr;
  const size_t pin = std::max({sizeof(CGScalars) * B, sizeof(double) * 8 * B,
                               sizeof(double) * (size_t)B * (c->bm + 1)});
  CK(cudaMallocHost(&c->bpinned, pin));
  c->bcap = B;
}

// Stage lists for the instances in `act` (3 jobs each, skip = instance done flag).
void schur_apply_batch(kfbim_ctx* c, const std::vector<int>& act, cudaStream_t s) {
  const int64_t n = c->N3;
  std::vector<Job> L[5];
  for (int b : act) {
    const kfbim_ctx::Slot& w = c->bs[b];
    const int* sk = &c->bcgs[b].done;
    float *A = w.T6, *B = w.T6 + n, *C = w.T6 + 2 * n, *D = w.T6 + 3 * n, *E = w.T6 + 4 * n,
          *F = w.T6 + 5 * n;
    L[0].push_back({w.d, A, 2, X_DST2F, X_NONE, W_NONE, 0, 0, sk});
    L[0].push_back({w.d, B, 1, X_DST2F, X_NONE, W_NONE, 2, 0, sk});
    L[1].push_back({A, C, 1, X_DST2F, X_NONE, W_NONE, 0, 0, sk});
    L[1].push_back({A, D, 0, X_DST2F, X_NONE, W_NONE, 1, 0, sk});
    L[1].push_back({B, E, 0, X_DST2F, X_NONE, W_NONE, 2, 0, sk});
    L[2].push_back({C, A, 0, X_DCT2F, X_DCT2I, W_SCHUR, 0, 0, sk});
    L[2].push_back({D, B, 1, X_DCT2F, X_DCT2I, W_SCHUR, 1, 0, sk});
    L[2].push_back({E, F, 2, X_DCT2F, X_DCT2I, W_SCHUR, 2, 0, sk});
    L[3].push_back({A, C, 1, X_DST2I, X_NONE, W_NONE, 0, 0, sk});
    L[3].push_back({B, D, 0, X_DST2I, X_NONE, W_NONE, 1, 0, sk});
    L[3].push_back({F, E, 0, X_DST2I, X_NONE, W_NONE, 2, 0, sk});
    L[4].push_back({C, w.q, 2, X_DST2I, X_NONE, W_NONE, 0, 0, sk});
    L[4].push_back({D, w.q2, 2, X_DST2I, X_NONE, W_NONE, 1, 0, sk});
    L[4].push_back({E, w.q3, 1, X_DST2I, X_NONE, W_NONE, 2, 0, sk});
  }
  for (int k = 0; k < 5; ++k) stage_list<float, float, float>(c, L[k], s);
}

// face-to-cell (W_RHS) or face-to-face (W_POISSON) transform of three face
// fields per instance: src(b) -> dst(b) (component outputs at stride N^3)
template <typename Tin>
void face3_batch(kfbim_ctx* c, const std::vector<int>& act, const std::vector<const Tin*>& src,
                 const std::vector<float*>& dst1, const std::vector<float*>& dst2,
                 const std::vector<float*>& dst3, int wmode, cudaStream_t s) {
  const int64_t n = c->N3;
  const int t1 = wmode == W_RHS ? X_DCT2I : X_DST1I;
  std::vector<Job> L[5];
  for (size_t q = 0; q < act.size(); ++q) {
    const kfbim_ctx::Slot& w = c->bs[act[q]];
    const Tin* f = src[q];
    float *A = w.T6, *B = w.T6 + n, *C = w.T6 + 2 * n, *D = w.T6 + 3 * n, *E = w.T6 + 4 * n,
          *F = w.T6 + 5 * n;
    L[0].push_back({f, A, 2, X_DST2F, X_NONE, W_NONE, 0, 0});
    L[0].push_back({f + n, B, 2, X_DST2F, X_NONE, W_NONE, 1, 0});
    L[0].push_back({f + 2 * n, C, 1, X_DST2F, X_NONE, W_NONE, 2, 0});
    L[1].push_back({A, D, 1, X_DST2F, X_NONE, W_NONE, 0, 0});
    L[1].push_back({B, E, 0, X_DST2F, X_NONE, W_NONE, 1, 0});
    L[1].push_back({C, F, 0, X_DST2F, X_NONE, W_NONE, 2, 0});
    L[2].push_back({D, A, 0, X_DST1F, t1, wmode, 0, 0});
    L[2].push_back({E, B, 1, X_DST1F, t1, wmode, 1, 0});
    L[2].push_back({F, C, 2, X_DST1F, t1, wmode, 2, 0});
    L[3].push_back({A, D, 1, X_DST2I, X_NONE, W_NONE, 0, 0});
    L[3].push_back({B, E, 0, X_DST2I, X_NONE, W_NONE, 1, 0});
    L[3].push_back({C, F, 0, X_DST2I, X_NONE, W_NONE, 2, 0});
    L[4].push_back({D, dst1[q], 2, X_DST2I, X_NONE, W_NONE, 0, 0});
    L[4].push_back({E, dst2[q], 2, X_DST2I, X_NONE, W_NONE, 1, 0});
    L[4].push_back({F, dst3[q], 1, X_DST2I, X_NONE, W_NONE, 2, 0});
  }
  stage_list<Tin, float, float>(c, L[0], s);
  for (int k = 1; k < 5; ++k) stage_list<float, float, float>(c, L[k], s);
}

// The slab CG runs of batch slots `slots`.
std::vector<SlabCg> slab_batch_runs(kfbim_ctx* c, const std::vector<int>& slots) {
  const int64_t n = c->N3;
  std::vector<SlabCg> runs;
  for (int b : slots) {
    const kfbim_ctx::Slot& w = c->bs[b];
    runs.push_back({c->N, w.x, w.r, w.d, w.q, w.T6, w.T6 + n, c->d_twc32, c->d_q32, c->d_s2f,
                    (float)(1.0 / c->mu), &c->bcgs[b], c->bpartial + (size_t)kRunPartials * b});
  }
  return runs;
}

// Slots not in the run are marked done, so that the batched kernels of all
// slots skip them.
__global__ void k_cg_mark_idle(CGScalars* s, int nslot, unsigned long long active) {
  const int b = threadIdx.x;
  if (b < nslot && !((active >> b) & 1ull)) s[b].done = 1;
}

// Device side of the batched CG loop: counts the trip (in every slot) and
// keeps the loop going while any slot is running and the cap is not reached.
__global__ void k_cg_cond_batch(cudaGraphConditionalHandle h, CGScalars* s, int nslot, int maxit) {
  bool any = false;
  int t = 0;
  for (int b = 0; b < nslot; ++b) {
    t = ++s[b].trips;
    any = any || !s[b].done;
  }
  cudaGraphSetConditional(h, (any && t < maxit) ? 1u : 0u);
}

// The batched slab CG of all bcap slots as a conditional while loop: one
// graph launch runs every slot's CG to its end (slots already done return
// at once).  Captured on first use after the slot scalars are reset with
// every slot marked done, after one untimed iteration (which then does
// nothing but load the kernels).  Null where conditional nodes are refused.
cudaGraphExec_t cg_batch_graph(kfbim_ctx* c, const std::vector<SlabCg>& all) {
  if (c->bcg_tried) return c->bcg_exec;
  c->bcg_tried = true;
  CK(cudaStreamSynchronize(c->cap_stream));
  const int64_t before = g_launches;
  slab_cg_iteration_batch(all.data(), (int)all.size(), c->cap_stream);
  CK(cudaStreamSynchronize(c->cap_stream));
  const int64_t per_iter = g_launches - before;
  g_launches = before;
  cudaGraph_t graph = nullptr;
  CK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle h{};
  bool ok = cudaGraphConditionalHandleCreate(&h, graph, 1u, cudaGraphCondAssignDefault) == cudaSuccess;
  cudaGraphNodeParams np{};
  if (ok) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    ok = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np) == cudaSuccess;
  }
  if (!ok) {
    (void)cudaGetLastError();   // a refused conditional node is not an error of this call
    CK(cudaGraphDestroy(graph));
    return nullptr;
  }
  cudaGraph_t body = np.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  slab_cg_iteration_batch(all.data(), (int)all.size(), c->cap_stream);
  k_cg_cond_batch<<<1, 1, 0, c->cap_stream>>>(h, c->bcgs, (int)all.size(), std::max(1, c->opt.cg_max));
  CK(cudaStreamEndCapture(c->cap_stream, &body));
  g_launches = before;
  CK(cudaGraphInstantiate(&c->bcg_exec, graph, 0));
  CK(cudaGraphDestroy(graph));
  c->bcg_kernels = per_iter + 1;
  return c->bcg_exec;
}

// Lockstep FP32 CG of the instances in `act` on (S + ...) x = b (b in fu[0:N3]).
void cg_batch(kfbim_ctx* c, const std::vector<int>& act, double tol, cudaStream_t s) {
  const int64_t n = c->N3;
  const double rank1 = c->navier ? 0.0 : 1.0 / (c->mu * (double)n);
  std::vector<int> slots(c->bcap);
  for (int b = 0; b < c->bcap; ++b) slots[b] = b;
  const std::vector<SlabCg> all = c->slab ? slab_batch_runs(c, slots) : std::vector<SlabCg>();
  const bool graphs = c->slab && c->use_graphs && !c->prof;
  if (graphs && !c->bcg_tried) {
    // the capture stream's warm-up iteration must see every slot done
    CK(cudaMemsetAsync(c->bcgs, 0, sizeof(CGScalars) * c->bcap, s));
    k_cg_mark_idle<<<1, 64, 0, s>>>(c->bcgs, c->bcap, 0ull);
    ++g_launches;
    check_launch();
    CK(cudaStreamSynchronize(s));
    cg_batch_graph(c, all);
  }
  cudaGraphExec_t exec = graphs ? c->bcg_exec : nullptr;
  unsigned long long mask = 0ull;
  for (int b : act) mask |= 1ull << b;
  CK(cudaMemsetAsync(c->bcgs, 0, sizeof(CGScalars) * c->bcap, s));
  k_cg_mark_idle<<<1, 64, 0, s>>>(c->bcgs, c->bcap, mask);
  ++g_launches;
  for (int b : act) {
    const kfbim_ctx::Slot& w = c->bs[b];
    CK(cudaMemsetAsync(w.x, 0, n * sizeof(float), s));
    CK(cudaMemcpyAsync(w.r, w.fu, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(w.d, w.fu, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    // the slot's tolerance, relaxed with its refinement tolerance as in grid_solve_mixed
    const double tb = std::max(tol, relaxed_inner_tol(c, c->b_refine_tol[b]));
    k_cg_init<float><<<RED_BLOCKS, RED_THREADS, 0, s>>>(w.fu, n, &c->bcgs[b], tb * tb, rank1, c->cpen,
                                                         c->partial);
    ++g_launches;
  }
  check_launch();
  std::vector<CGScalars> h(c->bcap);
  int launched = 0;
  if (exec) {
    // one graph launch: every slot's CG runs to done or to the cap
    CK(cudaGraphLaunch(exec, s));
    launched = c->opt.cg_max;
  }
  while (true) {
    CK(cudaMemcpyAsync(c->bpinned, c->bcgs, sizeof(CGScalars) * c->bcap, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (c->prof_used) prof_collect(c);
    std::memcpy(h.data(), c->bpinned, sizeof(CGScalars) * c->bcap);
    if (exec) g_launches += (int64_t)h[0].trips * c->bcg_kernels;
    std::vector<int> run;
    for (int b : act) {
      if (!std::isfinite(h[b].rr)) throw CudaError{"non-finite CG residual in a batched solve", KFBIM_E_NONFINITE};
      if (!h[b].done) run.push_back(b);
    }
    if (run.empty() || launched >= c->opt.cg_max) break;
    // the CG vector updates of every running instance in one launch per step,
    // RED_BLOCKS blocks per instance (the single-run reduction order)
    CgBatchArgs<float> A{};
    for (size_t k = 0; k < run.size(); ++k) {
      const kfbim_ctx::Slot& w = c->bs[run[k]];
      A.x[k] = w.x;
      A.r[k] = w.r;
      A.d[k] = w.d;
      A.q[k] = w.q;
      A.q2[k] = w.q2;
      A.q3[k] = w.q3;
      A.s[k] = &c->bcgs[run[k]];
      A.partial[k] = c->bpartial + (size_t)kRunPartials * run[k];
    }
    const dim3 grid(RED_BLOCKS, (unsigned)run.size());
    if (c->slab) {
      // the three slab kernels of all running instances, one launch each per
      // iteration (blockIdx.y = instance; the single-run arithmetic)
      const std::vector<SlabCg> runs = slab_batch_runs(c, run);
      for (int it = 0; it < kCgGraphIters; ++it) {
        g_launches += slab_cg_iteration_batch(runs.data(), (int)runs.size(), s);
        check_launch();
      }
    } else {
      for (int it = 0; it < kCgGraphIters; ++it) {
        schur_apply_batch(c, run, s);
        k_cg_alpha_b<float><<<grid, RED_THREADS, 0, s>>>(A, n);
        k_cg_update_b<float><<<grid, RED_THREADS, 0, s>>>(A, n);
        k_cg_direction_b<float><<<grid, RED_THREADS, 0, s>>>(A, n);
        g_launches += 3;
        check_launch();
      }
    }
    launched += kCgGraphIters;
  }
  if (c->slab && !act.empty()) {
    // the update each run left pending when it stopped
    const std::vector<SlabCg> runs = slab_batch_runs(c, act);
    g_launches += slab_cg_finish_batch(runs.data(), (int)runs.size(), s);
    check_launch();
  }
  for (int b : act) {
    c->cg_iters += h[b].iters;
    c->b_cg[b] += h[b].iters;
  }
}

// Read one double per slot of `act` from bscal[8 b + k].
std::vector<double> read_slots(kfbim_ctx* c, const std::vector<int>& act, int k, cudaStream_t s) {
  CK(cudaMemcpyAsync(c->bpinned, c->bscal, sizeof(double) * 8 * c->bcap, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (c->prof_used) prof_collect(c);
  const double* h = static_cast<const double*>(c->bpinned);
  std::vector<double> v;
  for (int b : act) {
    if (!std::isfinite(h[8 * b + k])) throw CudaError{"non-finite residual in a batched solve", KFBIM_E_NONFINITE};
    v.push_back(h[8 * b + k]);
  }
  return v;
}

// MIXED grid solve of the instances in `act` (rhs in slot.rhs -> slot.u, slot.p).
void grid_solve_batch(kfbim_ctx* c, const std::vector<int>& act, cudaStream_t s) {
  const int64_t N3 = c->N3;
  for (int b : act) {
    const kfbim_ctx::Slot& w = c->bs[b];
    double* g = w.rhs + 3 * N3;
    double* gmean = c->bscal + 8 * b;
    CK(cudaMemsetAsync(w.u, 0, 3 * N3 * sizeof(double), s));
    CK(cudaMemsetAsync(w.p, 0, N3 * sizeof(double), s));
    if (c->navier) CK(cudaMemsetAsync(gmean, 0, sizeof(double), s));
    else dot(c, g, (const double*)nullptr, N3, gmean, 1.0 / (double)N3, s);
    CK(cudaMemcpyAsync(w.res, w.rhs, 4 * N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    k_shift<<<grid_for(N3), 256, 0, s>>>(w.res + 3 * N3, gmean, -1.0, N3); ++g_launches;
    norm2_fast(c, w.res, 4 * N3, c->bscal + 8 * b + 1, s);
  }
  const std::vector<double> ref2 = read_slots(c, act, 1, s);
  std::vector<int> live;
  for (size_t q = 0; q < act.size(); ++q)
    if (ref2[q] > 0.0) live.push_back(act[q]);
  for (int sweep = 0; !live.empty(); ++sweep) {
    if (sweep > 0) {
      if (c->fp32_only) break;   // FP32: one correction solve, no FP64 residual
      for (int b : live) {
        const kfbim_ctx::Slot& w = c->bs[b];
        k_mac_residual<<<grid_for(4 * N3), 256, 0, s>>>(w.rhs, w.rhs + 3 * N3, c->bscal + 8 * b, w.u, w.p,
                                                        c->gix(), c->h, c->mu, c->cpen, w.res, w.res + 3 * N3);
        ++g_launches;
        norm2_fast(c, w.res, 4 * N3, c->bscal + 8 * b + 2, s);
      }
      check_launch();
      const std::vector<double> r2 = read_slots(c, live, 2, s);
      std::vector<int> keep;
      for (size_t q = 0; q < live.size(); ++q) {
        const double ref = ref2[std::find(act.begin(), act.end(), live[q]) - act.begin()];
        const double tol = c->b_refine_tol[live[q]];
        if (!(r2[q] <= tol * tol * ref)) keep.push_back(live[q]);
      }
      live.swap(keep);
      if (live.empty() || sweep >= c->opt.refine_max) break;
    }
    c->refine_sweeps += (int)live.size();
    for (int b : live) ++c->b_sweeps[b];
    std::vector<const double*> src;
    std::vector<float*> d1, d2, d3;
    for (int b : live) {
      const kfbim_ctx::Slot& w = c->bs[b];
      src.push_back(w.res);
      d1.push_back(w.q);
      d2.push_back(w.q2);
      d3.push_back(w.q3);
    }
    face3_batch<double>(c, live, src, d1, d2, d3, W_RHS, s);
    for (int b : live) {
      const kfbim_ctx::Slot& w = c->bs[b];
      k_sum4<double, float><<<grid_for(N3), 256, 0, s>>>(w.res + 3 * N3, w.q, w.q2, w.q3, w.fu, N3);
      ++g_launches;
    }
    check_launch();
    cg_batch(c, live, c->opt.inner_tol, s);
    std::vector<const float*> fsrc;
    std::vector<float*> u1, u2, u3;
    for (int b : live) {
      const kfbim_ctx::Slot& w = c->bs[b];
      k_add_to<float><<<grid_for(N3), 256, 0, s>>>(w.x, w.p, N3);
      k_f_minus_gp<float, float><<<grid_for(3 * N3), 256, 0, s>>>(w.res, w.x, c->gix(), c->h, w.fu);
      g_launches += 2;
      fsrc.push_back(w.fu);
      u1.push_back(w.fu);
      u2.push_back(w.fu + N3);
      u3.push_back(w.fu + 2 * N3);
    }
    check_launch();
    face3_batch<float>(c, live, fsrc, u1, u2, u3, W_POISSON, s);
    for (int b : live) {
      const kfbim_ctx::Slot& w = c->bs[b];
      k_add_to<float><<<grid_for(3 * N3), 256, 0, s>>>(w.fu, w.u, 3 * N3);
      ++g_launches;
    }
    check_launch();
  }
  if (c->navier) return;
  for (int b : act) {   // gauge mean(p) = mu mean(g)
    const kfbim_ctx::Slot& w = c->bs[b];
    double* sc = c->bscal + 8 * b + 3;
    dot(c, w.p, (const double*)nullptr, N3, sc, 1.0 / (double)N3, s);
    k_shift<<<grid_for(N3), 256, 0, s>>>(w.p, sc, -1.0, N3);
    k_shift<<<grid_for(N3), 256, 0, s>>>(w.p, c->bscal + 8 * b, c->mu, N3);
    g_launches += 2;
  }
  check_launch();
}

// Jumps, RHS and grid solve for the instances in `act`; phi/fpts/fgrid per instance.
void interface_batch(kfbim_ctx* c, const std::vector<int>& act, const std::vector<const double*>& phi,
                     const std::vector<const double*>& fpts, const std::vector<const double*>& fgrid,
                     cudaStream_t s) {
  const int64_t n = c->n_all;
  for (size_t q = 0; q < act.size(); ++q) {
    const kfbim_ctx::Slot& w = c->bs[act[q]];
    k_jumps<<<(unsigned)((n + JB - 1) / JB), 3 * JB, 0, s>>>(
        phi[q], fpts[q], n, c->d_comp, c->d_pid, c->d_fit_off, c->d_fit_col, c->d_fit_w, c->fit_ell,
        c->d_jmap, w.J);
    k_rhs_fill<<<grid_for(4 * c->N3), 256, 0, s>>>(fgrid[q], c->d_side[1], c->d_side[2], c->d_side[3],
                                                    c->gix(), w.rhs);
    g_launches += 2;
    if (c->n_corr_rows > 0) {
      k_corrections<<<grid_for(c->n_corr_rows), 256, 0, s>>>(c->d_corr_row, c->d_corr_ptr, c->d_corr_src,
                                                              c->d_corr_coef, c->n_corr_rows, w.J, w.rhs);
      ++g_launches;
    }
  }
  check_launch();
  c->interface_solves += (int)act.size();
  for (int b : act) ++c->b_isolves[b];
  grid_solve_batch(c, act, s);
}

// Lockstep GMRES (Alg. 1 step 3) of the instances in `act` with right-hand
// sides slot.grhs; solutions to x[b].  Per instance the arithmetic is the
// single-instance GMRES; the batch shares the matvec launches and the host
// reads (three per iteration for the whole batch).
void gmres_batch(kfbim_ctx* c, const std::vector<int>& act, const std::vector<double*>& x,
                 std::vector<int>& iters, std::vector<double>& resid, std::vector<int>& status,
                 cudaStream_t s) {
  const int64_t n = c->n_prim, ld = n;
  const int m = c->bm, nb = 64;
  const int B = c->bcap;
  for (int b : act) dot(c, c->bs[b].grhs, c->bs[b].grhs, n, c->bscal + 8 * b + 4, 1.0, s);
  const std::vector<double> b2 = read_slots(c, act, 4, s);
  struct Gm {
    std::vector<double> H, cs, sn, g;
    double beta = 0.0;
  };
  std::vector<Gm> G(B);
  std::vector<int> live;
  for (size_t q = 0; q < act.size(); ++q) {
    const int b = act[q];
    Gm& z = G[b];
    z.beta = std::sqrt(b2[q]);
    iters[b] = 0;
    resid[b] = 0.0;
    status[b] = KFBIM_OK;
    if (z.beta == 0.0) {
      CK(cudaMemsetAsync(x[b], 0, n * sizeof(double), s));
      continue;
    }
    z.H.assign((size_t)(m + 1) * m, 0.0);
    z.cs.assign(m, 0.0);
    z.sn.assign(m, 0.0);
    z.g.assign(m + 1, 0.0);
    z.g[0] = z.beta;
    status[b] = KFBIM_E_NOCONV;
    resid[b] = 1.0;
    k_scale_copy<<<grid_for(n), 256, 0, s>>>(c->bs[b].grhs, 1.0 / z.beta, nullptr, c->bs[b].V, n);
    ++g_launches;
    live.push_back(b);
  }
  check_launch();
  std::vector<int> done_at(B, 0);
  const double* hp = static_cast<const double*>(c->bpinned);
  struct ResetTols {
    kfbim_ctx* c;
    ~ResetTols() { std::fill(c->b_refine_tol.begin(), c->b_refine_tol.end(), c->opt.refine_tol); }
  } reset_tols{c};
  for (int k = 1; k <= m && !live.empty(); ++k) {
    std::vector<const double*> phi, nul(live.size(), nullptr);
    for (int b : live) {
      phi.push_back(c->bs[b].V + (int64_t)(k - 1) * ld);
      c->b_refine_tol[b] = relaxed_refine_tol(c, resid[b]);
    }
    interface_batch(c, live, phi, nul, nul, s);
    for (int b : live) {
      const kfbim_ctx::Slot& w = c->bs[b];
      k_trace<<<grid_for(c->n_prim), 256, 0, s>>>(w.u, w.J, c->n_all, c->n_prim, c->d_prim_of, c->N,
                                                   c->d_tr_comp, c->d_tr_node, c->d_tr_w, c->d_tr_cj, w.gw);
      ++g_launches;
    }
    check_launch();
    std::vector<std::vector<double>> hcol(B);
    for (int b : live) hcol[b].assign(m + 1, 0.0);
    for (int pass2 = 0; pass2 < 2; ++pass2) {
      for (int b : live) {
        const kfbim_ctx::Slot& w = c->bs[b];
        k_multidot_partial<<<dim3(nb, k), RED_THREADS, 0, s>>>(w.V, ld, w.gw, n, c->partial);
        k_sum_partials<<<k, RED_THREADS, 0, s>>>(c->partial, nb, 1.0, w.gh);
        k_multi_axpy<<<grid_for(n), 256, 0, s>>>(w.V, ld, w.gh, k, w.gw, n, 0);
        g_launches += 3;
      }
      check_launch();
      CK(cudaMemcpyAsync(c->bpinned, c->bgh, sizeof(double) * (size_t)B * (m + 1), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int b : live)
        for (int j = 0; j < k; ++j) hcol[b][j] += hp[(size_t)b * (m + 1) + j];
    }
    for (int b : live) dot(c, c->bs[b].gw, c->bs[b].gw, n, c->bscal + 8 * b + 5, 1.0, s);
    const std::vector<double> hn2 = read_slots(c, live, 5, s);
    std::vector<int> keep;
    for (size_t q = 0; q < live.size(); ++q) {
      const int b = live[q];
      Gm& z = G[b];
      std::vector<double>& h = hcol[b];
      const double hn = std::sqrt(hn2[q]);
      h[k] = hn;
      for (int j = 0; j < k - 1; ++j) {
        const double a = h[j], bb = h[j + 1];
        h[j] = z.cs[j] * a + z.sn[j] * bb;
        h[j + 1] = -z.sn[j] * a + z.cs[j] * bb;
      }
      const double a = h[k - 1], bb = h[k];
      const double r = std::hypot(a, bb);
      z.cs[k - 1] = (r == 0.0) ? 1.0 : a / r;
      z.sn[k - 1] = (r == 0.0) ? 0.0 : bb / r;
      h[k - 1] = r;
      h[k] = 0.0;
      z.g[k] = -z.sn[k - 1] * z.g[k - 1];
      z.g[k - 1] = z.cs[k - 1] * z.g[k - 1];
      for (int j = 0; j < k; ++j) z.H[(size_t)j * m + (k - 1)] = h[j];
      resid[b] = std::fabs(z.g[k]) / z.beta;
      done_at[b] = k;
      if (resid[b] < c->opt.gmres_tol || hn == 0.0) {
        status[b] = KFBIM_OK;
        continue;
      }
      if (k < m) {
        k_scale_copy<<<grid_for(n), 256, 0, s>>>(c->bs[b].gw, 1.0 / hn, nullptr, c->bs[b].V + (int64_t)k * ld, n);
        ++g_launches;
      }
      keep.push_back(b);
    }
    check_launch();
    live.swap(keep);
  }
  for (int b : act) {
    Gm& z = G[b];
    if (z.beta == 0.0) continue;
    const int kk = done_at[b];
    std::vector<double> y(kk, 0.0);
    for (int i = kk - 1; i >= 0; --i) {
      double acc = z.g[i];
      for (int j = i + 1; j < kk; ++j) acc -= z.H[(size_t)i * m + j] * y[j];
      y[i] = acc / z.H[(size_t)i * m + i];
    }
    CK(cudaMemcpyAsync(c->bs[b].gy, y.data(), kk * sizeof(double), cudaMemcpyHostToDevice, s));
    k_multi_axpy<<<grid_for(n), 256, 0, s>>>(c->bs[b].V, ld, c->bs[b].gy, kk, x[b], n, 1);
    ++g_launches;
    CK(cudaStreamSynchronize(s));   // y lives on the host stack
    iters[b] = kk;
  }
  check_launch();
}

}  // namespace

// =================================================================== C ABI
extern "C" {

void kfbim_default_options(kfbim_options* o) {
  if (!o) return;
  o->mu = 1.0;
  o->precision = KFBIM_FP64;
  o->gmres_tol = 1e-10;
  o->gmres_max = 200;
  o->cg_tol = 1e-14;
  o->cg_max = 2000;
  o->refine_tol = 1e-11;
  o->refine_max = 8;
  o->inner_tol = 3e-6;
  o->pde = KFBIM_STOKES;
  o->lambda = 0.0;
  o->transforms = KFBIM_XF_AUTO;
  o->relax = 0.1;
}

static int setup_common(const kfbim_geometry* geom, const kfbim_grid* grid, const kfbim_options* opt,
                        kfbim_ctx** out, bool device, cudaStream_t stream = nullptr,
                        const kfbim_allocator* alloc = nullptr) {
  if (!out) return KFBIM_E_INVALID;
  *out = nullptr;
  if (!geom || !grid || !opt) return KFBIM_E_INVALID;
  const int N = grid->N;
  if (N < 16 || N > 256 || ((N & (N - 1)) != 0 && N != 96) || !(grid->hi > grid->lo)) return KFBIM_E_INVALID;
  if (!(opt->mu > 0) || opt->gmres_max < 1 || opt->gmres_max > 200 || opt->cg_max < 1 ||
      opt->precision < KFBIM_FP64 || opt->precision > KFBIM_MIXED_TF32)
    return KFBIM_E_INVALID;
  if (opt->precision == KFBIM_MIXED_TF32 && N != TC_N) return KFBIM_E_INVALID;
  if (!(opt->relax >= 0.0)) return KFBIM_E_INVALID;
  if (alloc && (!alloc->alloc || !alloc->free)) return KFBIM_E_INVALID;
  if (geom->kind < KFBIM_SPHERE || geom->kind > KFBIM_CALLBACK) return KFBIM_E_INVALID;
  if (geom->kind == KFBIM_CALLBACK && (!geom->F || !geom->derivs)) return KFBIM_E_INVALID;
  if (geom->kind == KFBIM_TORUS && !(geom->params[0] > 0.0 && geom->params[1] > geom->params[0]))
    return KFBIM_E_INVALID;
  if (opt->pde != KFBIM_STOKES && opt->pde != KFBIM_NAVIER) return KFBIM_E_INVALID;
  if (opt->transforms < KFBIM_XF_AUTO || opt->transforms > KFBIM_XF_STAGED) return KFBIM_E_INVALID;
  if (opt->pde == KFBIM_NAVIER && !(opt->lambda >= 0.0 && opt->lambda + opt->mu > 0.0))
    return KFBIM_E_INVALID;
  std::unique_ptr<kfbim_ctx> c(new (std::nothrow) kfbim_ctx());
  if (!c) return KFBIM_E_OOM;
  c->opt = *opt;
  c->precision_requested = opt->precision;
  if (opt->precision == KFBIM_FP32) {
    c->opt.precision = KFBIM_MIXED;
    c->fp32_only = true;
  } else if (opt->precision == KFBIM_MIXED_TF32) {
    c->opt.precision = KFBIM_MIXED;
    c->opt.transforms = KFBIM_XF_TENSOR;
  }
  c->setup_stream = stream;
  // KFBIM_CUDA_GRAPHS=0 launches the CG kernels one by one (kernel profilers
  // cannot look inside graphs with conditional nodes)
  if (const char* g = std::getenv("KFBIM_CUDA_GRAPHS")) c->use_graphs = std::strcmp(g, "0") != 0;
  c->refine_tol_now = c->opt.refine_tol;
  c->relax = c->opt.relax;
  if (alloc) {
    c->allocator = *alloc;
    c->custom_alloc = true;
  }
  c->N = N;
  while ((1 << c->lg) < N) ++c->lg;
  if ((1 << c->lg) != N) c->lg = -1;
  c->N3 = (int64_t)N * N * N;
  c->h = (grid->hi - grid->lo) / N;
  c->mu = opt->mu;
  c->navier = opt->pde == KFBIM_NAVIER;
  c->cpen = c->navier ? 1.0 / (opt->lambda + opt->mu) : 0.0;
  std::string err;
  int st;
  try {
    st = build_tables(*geom, *grid, opt->mu, c->navier ? opt->lambda : -1.0, c->host, err);
  } catch (const std::bad_alloc&) {
    return KFBIM_E_OOM;
  }
  if (st != KFBIM_OK) {
    std::fprintf(stderr, "kfbim_setup: %s\n", err.c_str());
    return st;
  }
  c->n_all = c->host.n_all;
  c->n_prim = c->host.n_prim;
  c->fit_nnz = (int64_t)c->host.fit_col.size();
  c->corr_nnz = (int64_t)c->host.corr_src.size();
  c->n_corr_rows = (int64_t)c->host.corr_row.size();
  if (device) {
    const cudaError_t ge = cudaGetDevice(&c->dev_id);
    if (ge != cudaSuccess) {
      std::fprintf(stderr, "kfbim_setup: cudaGetDevice: %s\n", cudaGetErrorString(ge));
      return KFBIM_E_CUDA;
    }
    try {
      fill_tables(c.get());
      adjoint_tables(c.get());   // before the host fit and correction tables are released
      CK(cudaStreamSynchronize(stream));   // every upload has left the host tables
    } catch (const CudaError& e) {
      std::fprintf(stderr, "kfbim_setup: %s\n", e.msg.c_str());
      // releases whatever was created so far (memory, pinned buffers, stream, graphs)
      kfbim_destroy(c.release());
      if (e.code != KFBIM_E_CUDA) return e.code;
      return e.msg.find("out of memory") != std::string::npos ? KFBIM_E_OOM : KFBIM_E_CUDA;
    }
    c->device = true;
  }
  // the host tables are on the device now; keep only point data
  HostTables& t = c->host;
  std::vector<int64_t>().swap(t.fit_ptr);
  std::vector<int32_t>().swap(t.fit_col);
  std::vector<int32_t>().swap(c->fit_pos);
  std::vector<double>().swap(t.fit_w);
  std::vector<double>().swap(t.jmap);
  std::vector<int64_t>().swap(t.corr_row);
  std::vector<int64_t>().swap(t.corr_ptr);
  std::vector<int64_t>().swap(t.corr_src);
  std::vector<double>().swap(t.corr_coef);
  *out = c.release();
  return KFBIM_OK;
}

int kfbim_setup(const kfbim_geometry* geom, const kfbim_grid* grid, const kfbim_options* opt,
                kfbim_ctx** out) {
  return setup_common(geom, grid, opt, out, true);
}

int kfbim_setup_host(const kfbim_geometry* geom, const kfbim_grid* grid, const kfbim_options* opt,
                     kfbim_ctx** out) {
  return setup_common(geom, grid, opt, out, false);
}

int kfbim_setup_async(const kfbim_geometry* geom, const kfbim_grid* grid, const kfbim_options* opt,
                      void* stream, kfbim_ctx** out) {
  return setup_common(geom, grid, opt, out, true, (cudaStream_t)stream);
}

int kfbim_setup_ex(const kfbim_geometry* geom, const kfbim_grid* grid, const kfbim_options* opt, void* stream,
                   const kfbim_allocator* alloc, kfbim_ctx** out) {
  return setup_common(geom, grid, opt, out, true, (cudaStream_t)stream, alloc);
}

int kfbim_control_points(const kfbim_ctx* c, int comp, int64_t* n, double* xyz, double* normal) {
  if (!c || !n || comp < 1 || comp > 3) return KFBIM_E_INVALID;
  const HostTables& t = c->host;
  int64_t k = 0;
  for (int64_t y = 0; y < t.n_all; ++y) {
    if (!t.primary[y] || t.comp[y] != comp) continue;
    for (int a = 0; a < 3; ++a) {
      if (xyz) xyz[3 * k + a] = t.xyz[3 * y + a];
      if (normal) normal[3 * k + a] = t.normal[3 * y + a];
    }
    ++k;
  }
  *n = k;
  return KFBIM_OK;
}

int kfbim_jump_points(const kfbim_ctx* c, int64_t* n, double* xyz) {
  if (!c || !n) return KFBIM_E_INVALID;
  const HostTables& t = c->host;
  *n = t.n_all;
  if (xyz) std::memcpy(xyz, t.xyz.data(), (size_t)t.n_all * 3 * sizeof(double));
  return KFBIM_OK;
}

int kfbim_table_sizes(const kfbim_ctx* c, int64_t* fit_nnz, int64_t* corr_rows, int64_t* corr_nnz) {
  if (!c) return KFBIM_E_INVALID;
  if (fit_nnz) *fit_nnz = c->fit_nnz;
  if (corr_rows) *corr_rows = c->n_corr_rows;
  if (corr_nnz) *corr_nnz = c->corr_nnz;
  return KFBIM_OK;
}

int kfbim_destroy(kfbim_ctx* c) {
  if (!c) return KFBIM_E_INVALID;
  // a context whose setup failed part-way has device resources (dev_id >= 0)
  // but device == false; a host-only context has dev_id < 0 and no CUDA state
  const DeviceScope scope(c->dev_id);
  if (c->device) cudaDeviceSynchronize();
  for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
  for (auto& e : c->cg_exec)
    if (e) cudaGraphExecDestroy(e);
  if (c->bcg_exec) cudaGraphExecDestroy(c->bcg_exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (size_t k = 0; k < c->allocs.size(); ++k) {
    if (c->custom_alloc) c->allocator.free(c->allocs[k], c->alloc_bytes[k], c->allocator.user);
    else cudaFree(c->allocs[k]);
  }
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->bpinned) cudaFreeHost(c->bpinned);
  delete c;
  return KFBIM_OK;
}

const char* kfbim_last_error(const kfbim_ctx* c) { return c ? c->err.c_str() : "null context"; }

int kfbim_sizes(const kfbim_ctx* c, int64_t* n_points, int64_t* n_primary, int* N) {
  if (!c) return KFBIM_E_INVALID;
  if (n_points) *n_points = c->n_all;
  if (n_primary) *n_primary = c->n_prim;
  if (N) *N = c->N;
  return KFBIM_OK;
}

int kfbim_points(const kfbim_ctx* c, double* xyz, int32_t* comp, int32_t* axis, int32_t* primary) {
  if (!c) return KFBIM_E_INVALID;
  const HostTables& t = c->host;
  if (xyz) std::memcpy(xyz, t.xyz.data(), sizeof(double) * 3 * t.n_all);
  if (comp) std::memcpy(comp, t.comp.data(), sizeof(int32_t) * t.n_all);
  if (axis) std::memcpy(axis, t.axis.data(), sizeof(int32_t) * t.n_all);
  if (primary) std::memcpy(primary, t.primary.data(), sizeof(int32_t) * t.n_all);
  return KFBIM_OK;
}

int kfbim_normals(const kfbim_ctx* c, double* normal) {
  if (!c || !normal) return KFBIM_E_INVALID;
  std::memcpy(normal, c->host.normal.data(), sizeof(double) * 3 * c->host.n_all);
  return KFBIM_OK;
}

int kfbim_sides(const kfbim_ctx* c, int g, uint8_t* side) {
  if (!c || g < 0 || g > 3 || !side) return KFBIM_E_INVALID;
  std::memcpy(side, c->host.side[g].data(), c->N3);
  return KFBIM_OK;
}

int kfbim_apply(kfbim_ctx* c, const double* phi, double* out, void* stream) {
  return guarded(c, [&]() -> int {
    if (!phi || !out || phi == out) return fail(c, KFBIM_E_INVALID, "kfbim_apply: bad pointers");
    reset_counters(c);
    cudaStream_t s = (cudaStream_t)stream;
    int st = apply_impl(c, phi, out, s);
    check_tc(c, s);
    if (st == KFBIM_E_NOCONV) c->err = "inner CG reached its iteration cap";
    return st;
  });
}

int kfbim_jumps(kfbim_ctx* c, const double* phi, const double* fpts, double* Jout, void* stream) {
  return guarded(c, [&]() -> int {
    if (!phi || !Jout) return fail(c, KFBIM_E_INVALID, "kfbim_jumps: bad pointers");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = c->n_all;
    k_jumps<<<(unsigned)((n + JB - 1) / JB), 3 * JB, 0, s>>>(
        phi, fpts, n, c->d_comp, c->d_pid, c->d_fit_off, c->d_fit_col, c->d_fit_w, c->fit_ell, c->d_jmap,
        Jout); ++g_launches;
    check_launch();
    return KFBIM_OK;
  });
}

int kfbim_interface(kfbim_ctx* c, const double* phi, const double* fpts, const double* fgrid,
                    double* u, double* p, void* stream) {
  return guarded(c, [&]() -> int {
    if (!phi || !u || !p) return fail(c, KFBIM_E_INVALID, "kfbim_interface: bad pointers");
    reset_counters(c);
    cudaStream_t s = (cudaStream_t)stream;
    int st = interface_solve(c, phi, fpts, fgrid, s);
    CK(cudaMemcpyAsync(u, c->u, 3 * c->N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(p, c->p, c->N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    check_tc(c, s);
    return st;
  });
}

int kfbim_trace(kfbim_ctx* c, const double* u, const double* J, double* out, void* stream) {
  return guarded(c, [&]() -> int {
    if (!u || !J || !out) return fail(c, KFBIM_E_INVALID, "kfbim_trace: bad pointers");
    trace(c, u, J, out, (cudaStream_t)stream);
    return KFBIM_OK;
  });
}

int kfbim_pressure_trace(kfbim_ctx* c, const double* p, const double* J, double* out, void* stream) {
  return guarded(c, [&]() -> int {
    if (!p || !J || !out) return fail(c, KFBIM_E_INVALID, "kfbim_pressure_trace: bad pointers");
    cudaStream_t s = (cudaStream_t)stream;
    k_pressure_trace<<<grid_for(c->n_all), 256, 0, s>>>(p, J, c->d_xyz, c->n_all, c->N, c->host.lo, c->h,
                                                         c->d_side[0], out); ++g_launches;
    check_launch();
    return KFBIM_OK;
  });
}

int kfbim_transform_f32(kfbim_ctx* c, int type, int axis, int wmode, int wc, const float* in, float* out,
                        int backend, void* stream) {
  return guarded(c, [&]() -> int {
    if (type < X_DCT2F || type > X_DST1I || axis < 0 || axis > 2 || wmode < W_NONE || wmode > W_RHS || wc < 0 ||
        wc > 2 || !in || !out || (backend != KFBIM_XF_FFT && backend != KFBIM_XF_TENSOR))
      return fail(c, KFBIM_E_INVALID, "kfbim_transform_f32: bad arguments");
    if (c->opt.precision != KFBIM_MIXED) return fail(c, KFBIM_E_INVALID, "kfbim_transform_f32: needs a MIXED context");
    if (backend == KFBIM_XF_TENSOR && !c->d_tc_mats)
      return fail(c, KFBIM_E_INVALID, "kfbim_transform_f32: tensor-core passes need N = 128 and transforms != FFT");
    cudaStream_t s = (cudaStream_t)stream;
    const int keep = c->xf_plain;
    c->xf_plain = backend == KFBIM_XF_TENSOR;
    try {
      stage<float, float, float>(c, {{in, out, axis, type, X_NONE, wmode, wc, 0}}, s);
    } catch (...) {
      c->xf_plain = keep;
      throw;
    }
    c->xf_plain = keep;
    check_tc(c, s);
    return KFBIM_OK;
  });
}

int kfbim_transforms_info(const kfbim_ctx* c, int* plain, int* fused, float* tune_ms4) {
  if (!c) return KFBIM_E_INVALID;
  if (plain) *plain = c->xf_plain;
  if (fused) *fused = c->xf_fused;
  if (tune_ms4)
    for (int k = 0; k < 4; ++k) tune_ms4[k] = c->tune_ms[k];
  return KFBIM_OK;
}

int kfbim_poisson(kfbim_ctx* c, int comp, const double* r, double* u, void* stream) {
  return guarded(c, [&]() -> int {
    if (comp < 1 || comp > 3 || !r || !u) return fail(c, KFBIM_E_INVALID, "kfbim_poisson: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    // (1/mu) scaling is part of the weight: undo it so this is (-Delta_h)^{-1}
    face_poisson<double, double, double>(c, comp - 1, r, c->cr, c->t1, c->t2, s);
    k_scale_copy<<<grid_for(c->N3), 256, 0, s>>>(c->cr, c->mu, nullptr, u, c->N3); ++g_launches;
    check_launch();
    return KFBIM_OK;
  });
}

int kfbim_schur_apply_f32(kfbim_ctx* c, const float* d, float* q, void* stream) {
  return guarded(c, [&]() -> int {
    if (!d || !q || d == q) return fail(c, KFBIM_E_INVALID, "kfbim_schur_apply_f32: bad pointers");
    if (!c->slab) return fail(c, KFBIM_E_INVALID, "kfbim_schur_apply_f32: no slab CG on this context");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = c->N3;
    const CgWs<float> w = ws32(c);
    // scalars of a fresh run: beta = 0 (so d = r), not done, the Navier c p block
    CGScalars h{};
    h.cdiag = c->cpen;
    std::memcpy(c->pinned, &h, sizeof(CGScalars));
    CK(cudaMemcpyAsync(c->cgs, c->pinned, sizeof(CGScalars), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(w.r, d, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(w.d, 0, n * sizeof(float), s));
    SlabCg a{c->N, w.x, w.r, w.d, q, w.T6, w.T6 + n, c->d_twc32, c->d_q32, c->d_s2f, (float)(1.0 / c->mu),
             c->cgs, c->partial};
    g_launches += slab_schur_apply(a, s);
    check_launch();
    CK(cudaStreamSynchronize(s));   // the pinned scalars are reused by the next call
    return KFBIM_OK;
  });
}

int kfbim_schur_apply(kfbim_ctx* c, const double* d, double* q, void* stream) {
  return guarded(c, [&]() -> int {
    if (!d || !q || d == q) return fail(c, KFBIM_E_INVALID, "kfbim_schur_apply: bad pointers");
    cudaStream_t s = (cudaStream_t)stream;
    const CgWs<double> w = ws64(c);
    schur_apply3<double>(c, d, w.q, w.q2, w.q3, w.T6, s);
    k_sum3<double><<<grid_for(c->N3), 256, 0, s>>>(w.q, w.q2, w.q3, q, c->N3);
    ++g_launches;
    if (c->navier) {
      k_axpy<<<grid_for(c->N3), 256, 0, s>>>(d, c->cpen, q, c->N3);
      ++g_launches;
      check_launch();
      return KFBIM_OK;
    }
    dot(c, d, (const double*)nullptr, c->N3, c->scal, 1.0 / (c->mu * (double)c->N3), s);
    k_shift<<<grid_for(c->N3), 256, 0, s>>>(q, c->scal, 1.0, c->N3); ++g_launches;
    check_launch();
    return KFBIM_OK;
  });
}

int kfbim_solve(kfbim_ctx* c, const double* g, const double* fpts, const double* fgrid, double* phi,
                double* u, double* p, kfbim_stats* stats, void* stream) {
  return guarded(c, [&]() -> int {
    if (!g || !phi) return fail(c, KFBIM_E_INVALID, "kfbim_solve: bad pointers");
    reset_counters(c);
    const int64_t launches0 = g_launches;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = c->n_prim;
    CK(cudaMemcpyAsync(c->grhs, g, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (fpts || fgrid) {
      int st = interface_solve(c, c->zero_phi, fpts, fgrid, s);
      if (st != KFBIM_OK && st != KFBIM_E_NOCONV) return st;
      trace(c, c->u, c->J, c->gw, s);
      k_scale_copy<<<grid_for(n), 256, 0, s>>>(c->gw, -1.0, nullptr, c->gw, n); ++g_launches;
      k_add_to<double><<<grid_for(n), 256, 0, s>>>(c->gw, c->grhs, n); ++g_launches;
      check_launch();
    }
    int its = 0;
    double res = 0.0;
    int st = gmres(c, c->grhs, phi, s, &its, &res);
    if (st != KFBIM_OK && st != KFBIM_E_NOCONV) return st;
    int st2 = interface_solve(c, phi, fpts, fgrid, s);
    if (u) CK(cudaMemcpyAsync(u, c->u, 3 * c->N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (p) CK(cudaMemcpyAsync(p, c->p, c->N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    check_tc(c, s);
    if (stats) {
      stats->gmres_iters = its;
      stats->interface_solves = c->interface_solves;
      stats->cg_iters = c->cg_iters;
      stats->refine_sweeps = c->refine_sweeps;
      stats->gmres_residual = res;
      stats->kernel_launches = g_launches - launches0;
    }
    if (st == KFBIM_E_NOCONV) {
      c->err = "GMRES reached its iteration cap";
      return st;
    }
    if (st2 == KFBIM_E_NOCONV) {
      c->err = "inner CG or refinement reached its iteration cap";
      return st2;
    }
    return st2;
  });
}

int kfbim_solve_batch(kfbim_ctx* c, int B, const double* g, const double* fpts, const double* fgrid,
                      double* phi, double* u, double* p, kfbim_stats* stats, void* stream) {
  return guarded(c, [&]() -> int {
    if (B < 1 || B > KFBIM_BATCH_MAX || !g || !phi)
      return fail(c, KFBIM_E_INVALID, "kfbim_solve_batch: bad batch size or pointers");
    const int64_t n = c->n_prim, N3 = c->N3, na = c->n_all;
    if (c->opt.precision != KFBIM_MIXED) {
      // FP64 contexts solve the instances one after another
      int worst = KFBIM_OK;
      for (int b = 0; b < B; ++b) {
        int st = kfbim_solve(c, g + b * n, fpts ? fpts + b * 3 * na : nullptr,
                             fgrid ? fgrid + b * 3 * N3 : nullptr, phi + b * n, u ? u + b * 3 * N3 : nullptr,
                             p ? p + b * N3 : nullptr, stats ? stats + b : nullptr, stream);
        if (st != KFBIM_OK && st != KFBIM_E_NOCONV) return st;
        if (st != KFBIM_OK) worst = st;
      }
      return worst;
    }
    batch_alloc(c, B);
    reset_counters(c);
    c->b_cg.assign(c->bcap, 0);
    c->b_sweeps.assign(c->bcap, 0);
    c->b_isolves.assign(c->bcap, 0);
    c->b_refine_tol.assign(c->bcap, c->opt.refine_tol);
    const int64_t launches0 = g_launches;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int> all(B);
    std::vector<const double*> fp(B, nullptr), fg(B, nullptr), zero(B, c->zero_phi), ph(B);
    std::vector<double*> x(c->bcap, nullptr);
    for (int b = 0; b < B; ++b) {
      all[b] = b;
      if (fpts) fp[b] = fpts + b * 3 * na;
      if (fgrid) fg[b] = fgrid + b * 3 * N3;
      ph[b] = phi + b * n;
      x[b] = phi + b * n;
      CK(cudaMemcpyAsync(c->bs[b].grhs, g + b * n, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    if (fpts || fgrid) {
      // g - G_v f: the interface solve with zero density and the forcing
      interface_batch(c, all, zero, fp, fg, s);
      for (int b = 0; b < B; ++b) {
        const kfbim_ctx::Slot& w = c->bs[b];
        k_trace<<<grid_for(n), 256, 0, s>>>(w.u, w.J, na, n, c->d_prim_of, c->N, c->d_tr_comp, c->d_tr_node,
                                            c->d_tr_w, c->d_tr_cj, w.gw);
        k_scale_copy<<<grid_for(n), 256, 0, s>>>(w.gw, -1.0, nullptr, w.gw, n);
        k_add_to<double><<<grid_for(n), 256, 0, s>>>(w.gw, w.grhs, n);
        g_launches += 3;
      }
      check_launch();
    }
    std::vector<int> its(c->bcap, 0), st(c->bcap, KFBIM_OK);
    std::vector<double> res(c->bcap, 0.0);
    gmres_batch(c, all, x, its, res, st, s);
    interface_batch(c, all, ph, fp, fg, s);
    for (int b = 0; b < B; ++b) {
      const kfbim_ctx::Slot& w = c->bs[b];
      if (u) CK(cudaMemcpyAsync(u + b * 3 * N3, w.u, 3 * N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
      if (p) CK(cudaMemcpyAsync(p + b * N3, w.p, N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaStreamSynchronize(s));
    check_tc(c, s);
    int worst = KFBIM_OK;
    for (int b = 0; b < B; ++b) {
      if (st[b] != KFBIM_OK) worst = st[b];
      if (stats) {
        stats[b].gmres_iters = its[b];
        stats[b].interface_solves = c->b_isolves[b];
        stats[b].cg_iters = c->b_cg[b];
        stats[b].refine_sweeps = c->b_sweeps[b];
        stats[b].gmres_residual = res[b];
        stats[b].kernel_launches = g_launches - launches0;
      }
    }
    if (worst == KFBIM_E_NOCONV) c->err = "GMRES reached its iteration cap for an instance of the batch";
    return worst;
  });
}

int kfbim_apply_adjoint(kfbim_ctx* c, const double* lam, double* out, void* stream) {
  return guarded(c, [&]() -> int {
    if (!lam || !out || lam == out) return fail(c, KFBIM_E_INVALID, "kfbim_apply_adjoint: bad pointers");
    reset_counters(c);
    cudaStream_t s = (cudaStream_t)stream;
    int st = adjoint_apply(c, lam, out, s);
    CK(cudaStreamSynchronize(s));
    check_tc(c, s);
    if (st == KFBIM_E_NOCONV) c->err = "inner CG reached its iteration cap";
    return st;
  });
}

int kfbim_solve_adjoint(kfbim_ctx* c, const double* ubar, double* gbar, kfbim_stats* stats, void* stream) {
  return guarded(c, [&]() -> int {
    if (!ubar || !gbar) return fail(c, KFBIM_E_INVALID, "kfbim_solve_adjoint: bad pointers");
    reset_counters(c);
    const int64_t launches0 = g_launches;
    cudaStream_t s = (cudaStream_t)stream;
    int st0 = adjoint_from_u(c, ubar, c->grhs, s);
    if (st0 != KFBIM_OK && st0 != KFBIM_E_NOCONV) return st0;
    int its = 0;
    double res = 0.0;
    int st = gmres(c, c->grhs, gbar, s, &its, &res, true);
    CK(cudaStreamSynchronize(s));
    check_tc(c, s);
    if (stats) {
      stats->gmres_iters = its;
      stats->interface_solves = c->interface_solves;
      stats->cg_iters = c->cg_iters;
      stats->refine_sweeps = c->refine_sweeps;
      stats->gmres_residual = res;
      stats->kernel_launches = g_launches - launches0;
    }
    if (st == KFBIM_E_NOCONV) c->err = "adjoint GMRES reached its iteration cap";
    return st;
  });
}

int kfbim_profile(kfbim_ctx* c, int enable, double* ms64, int64_t* launches64, double* bytes64,
                  double* ms32, int64_t* launches32, double* bytes32) {
  return guarded(c, [&]() -> int {
    if (enable >= 0) {
      if (enable && c->prof_ev.empty()) {
        c->prof_ev.resize(8192);
        c->prof_tag.resize(4096);
        for (auto& e : c->prof_ev) CK(cudaEventCreate(&e));
      }
      c->prof = enable != 0;
      c->prof_used = 0;
      for (int k = 0; k < KFBIM_KCLASS_COUNT; ++k) {
        c->prof_ms[k] = c->prof_bytes[k] = 0;
        c->prof_count[k] = 0;
      }
      return KFBIM_OK;
    }
    CK(cudaDeviceSynchronize());
    if (c->prof_used) prof_collect(c);
    if (ms64) *ms64 = c->prof_ms[0];
    if (launches64) *launches64 = c->prof_count[0];
    if (bytes64) *bytes64 = c->prof_bytes[0];
    if (ms32) *ms32 = c->prof_ms[1];
    if (launches32) *launches32 = c->prof_count[1];
    if (bytes32) *bytes32 = c->prof_bytes[1];
    return KFBIM_OK;
  });
}

int kfbim_profile_kernels(kfbim_ctx* c, int n, double* ms, int64_t* launches, double* bytes) {
  return guarded(c, [&]() -> int {
    if (n < 0) return fail(c, KFBIM_E_INVALID, "kfbim_profile_kernels: negative count");
    CK(cudaDeviceSynchronize());
    if (c->prof_used) prof_collect(c);
    for (int k = 0; k < n; ++k) {
      const bool in = k < KFBIM_KCLASS_COUNT;
      if (ms) ms[k] = in ? c->prof_ms[k] : 0.0;
      if (launches) launches[k] = in ? c->prof_count[k] : 0;
      if (bytes) bytes[k] = in ? c->prof_bytes[k] : 0.0;
    }
    return KFBIM_OK;
  });
}

int kfbim_poisson_noalloc(int c, int N, double lo, double hi, const double* r, double* u,
                          void* stream) {
  if (c < 1 || c > 3 || !r || !u || r == u || !(hi > lo) || N < 16 || (N & (N - 1)) != 0)
    return KFBIM_E_INVALID;
  if (N > kNoAllocMaxN) {
    std::fprintf(stderr, "kfbim_poisson_noalloc: N = %d exceeds the static scratch limit N <= %d\n",
                 N, kNoAllocMaxN);
    return KFBIM_E_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  NoAllocSymbols* d = nullptr;
  int st = noalloc_symbols(s, &d);
  if (st != KFBIM_OK) return st;
  const double h = (hi - lo) / N;
  const int64_t N3 = (int64_t)N * N * N;
  double* t1 = d->scratch;
  double* t2 = d->scratch + N3;
  const int cax = c - 1;
  int o1, o2;
  others(cax, o1, o2);
  const cudaError_t pending = cudaPeekAtLastError();
  int Nv = N;
  C2<double>* tw = d->tw;
  C2<double>* q = d->q;
  double* s2 = d->s2;
  void* targs[] = {(void*)&Nv, (void*)&tw, (void*)&q, (void*)&s2};
  cudaError_t e = cudaLaunchKernel((const void*)k_na_tables, dim3(1), dim3(64), targs, 0, s);
  if (e == cudaSuccess) e = noalloc_pass(*d, N, h, r, t1, o2, X_DST2F, X_NONE, W_NONE, cax, s);
  if (e == cudaSuccess) e = noalloc_pass(*d, N, h, t1, t2, o1, X_DST2F, X_NONE, W_NONE, cax, s);
  if (e == cudaSuccess) e = noalloc_pass(*d, N, h, t2, t1, cax, X_DST1F, X_DST1I, W_POISSON, cax, s);
  if (e == cudaSuccess) e = noalloc_pass(*d, N, h, t1, t2, o1, X_DST2I, X_NONE, W_NONE, cax, s);
  if (e == cudaSuccess) e = noalloc_pass(*d, N, h, t2, u, o2, X_DST2I, X_NONE, W_NONE, cax, s);
  if (e != cudaSuccess) {
    // clear this call's own launch error from the thread's last-error state,
    // unless an earlier, unrelated error was already pending there
    if (pending == cudaSuccess) (void)cudaGetLastError();
    std::fprintf(stderr, "kfbim_poisson_noalloc: launch failed: %s\n", cudaGetErrorString(e));
    return KFBIM_E_CUDA;
  }
  return KFBIM_OK;
}

int kfbim_solve_host(kfbim_ctx* c, const double* g, const double* fpts, const double* fgrid,
                     double* phi, double* u, double* p, kfbim_stats* stats, void* stream) {
  return guarded(c, [&]() -> int {
    if (!g || !phi) return fail(c, KFBIM_E_INVALID, "kfbim_solve_host: bad pointers");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = c->n_prim, N3 = c->N3;
    if (!c->hs_g) {
      c->hs_g = dalloc<double>(c, n);
      c->hs_phi = dalloc<double>(c, n);
      c->hs_fp = dalloc<double>(c, 3 * c->n_all);
      c->hs_fg = dalloc<double>(c, 3 * N3);
      c->hs_u = dalloc<double>(c, 3 * N3);
      c->hs_p = dalloc<double>(c, N3);
    }
    CK(cudaMemcpyAsync(c->hs_g, g, n * sizeof(double), cudaMemcpyHostToDevice, s));
    if (fpts) CK(cudaMemcpyAsync(c->hs_fp, fpts, 3 * c->n_all * sizeof(double), cudaMemcpyHostToDevice, s));
    if (fgrid) CK(cudaMemcpyAsync(c->hs_fg, fgrid, 3 * N3 * sizeof(double), cudaMemcpyHostToDevice, s));
    int st = kfbim_solve(c, c->hs_g, fpts ? c->hs_fp : nullptr, fgrid ? c->hs_fg : nullptr, c->hs_phi,
                         u ? c->hs_u : nullptr, p ? c->hs_p : nullptr, stats, stream);
    CK(cudaMemcpyAsync(phi, c->hs_phi, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (u) CK(cudaMemcpyAsync(u, c->hs_u, 3 * N3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (p) CK(cudaMemcpyAsync(p, c->hs_p, N3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return st;
  });
}

}  // extern "C"
