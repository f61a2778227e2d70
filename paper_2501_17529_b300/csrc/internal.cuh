// Internal declarations shared by the dcflow translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dcflow.h"

namespace dcf {

constexpr int kNB = 64;          // dense FP64 block size (factor and solves)
constexpr int kRMax = 16;        // largest rank r = effective splits + outages
constexpr int kEntMax = 256;     // moved + outaged branches per topology
constexpr int kTMaxPass = 32;    // timesteps handled by one N-1 pass

void set_error(const std::string& msg);

#define DCF_CUDA(call)                                                          \
  do {                                                                          \
    cudaError_t e__ = (call);                                                   \
    if (e__ != cudaSuccess) {                                                   \
      ::dcf::set_error(std::string(#call) + ": " + cudaGetErrorString(e__));    \
      return DCFLOW_ERR_CUDA;                                                   \
    }                                                                           \
  } while (0)

#define DCF_CHECK_LAUNCH()                                                      \
  do {                                                                          \
    cudaError_t e__ = cudaGetLastError();                                       \
    if (e__ != cudaSuccess) {                                                   \
      ::dcf::set_error(std::string("kernel launch: ") + cudaGetErrorString(e__)); \
      return DCFLOW_ERR_CUDA;                                                   \
    }                                                                           \
  } while (0)

// Device buffer that grows on demand and is freed with the context.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  int ensure(size_t need);  // 0 or DCFLOW_ERR_OOM
  void release();
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// Per-chunk scratch of dcflow_solve_batch; two sets alternate so that one
// chunk's preparation overlaps the previous chunk's N-1 kernel.
struct ChunkBufs {
  DevBuf ent_n, ent_s, ent_w, mod_ptr, q_info;
  DevBuf Kinv, alpha, Vt64, VtR, Zs, Zbf, ptil, meta, s, valid, nisl;
  DevBuf pmax, parg, povl, cmr, p2max, tile;
  // injection candidates: per (timestep, candidate) operands and screening maxima,
  // the chosen candidate per timestep and its operands
  DevBuf ptv, svv, pmaxv, pargv, povlv, bestu, ptb, sb;
  // learned screener: selected-contingency bit masks, fallback flags, the
  // selected lists and their counts, the N-1 work list and its length
  DevBuf selmask, sfb, csel, nsel, work, nwork;
  // multi-outage sets: per (topology, set) K^{-1}-weighted columns, weights, flags
  DevBuf mvt, mw, mflag;
  // injection topologies: Z[c, :] / den_c, eligible injections and their split rows, their count
  DevBuf zcd, tiel, tirow, nel;
  void release_all() {
    DevBuf* b[] = {&ent_n, &ent_s, &ent_w, &mod_ptr, &q_info, &Kinv, &alpha, &Vt64, &VtR, &Zs, &Zbf, &ptil, &meta,
                   &s, &valid, &nisl, &pmax, &parg, &povl, &cmr, &p2max, &tile, &ptv, &svv, &pmaxv, &pargv, &povlv, &bestu, &ptb, &sb,
                   &selmask, &sfb, &csel, &nsel, &work, &nwork, &mvt, &mw, &mflag, &zcd, &tiel, &tirow, &nel};
    for (auto* x : b) x->release();
  }
};

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// multi-outage sets of a study: four per block of the per-set preparation, whose
// grid y extent is at most 65,535
constexpr int kMaxMultiSets = 4 * 65535;

// float copy of a double array (grid-stride)
static __global__ void k_to_float(const double* __restrict__ x, float* __restrict__ y, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

// Raise a kernel's dynamic shared-memory limit once per device (a function
// attribute lives in each device's context); `done` holds one bit per device.
template <class K>
inline cudaError_t smem_attr_once(K kernel, int bytes, uint64_t& done) {
  int d = 0;
  cudaError_t e = cudaGetDevice(&d);
  if (e != cudaSuccess) return e;
  if (d < 64 && ((done >> d) & 1ull)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && d < 64) done |= 1ull << d;
  return e;
}

// Makes `dev` the current device for the lifetime of the guard and puts the
// caller's device back afterwards: an entry point runs on its context's
// device whichever device the calling thread has current.
struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
    else prev = -1;  // nothing to restore
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// The schedule of dcflow_solve_batch: how the topologies are grouped by rank
// and chunked, and which N-1 variant runs.  The autotuner searches over these.
struct SchedPlan {
  int budget_mb = 8192;           // scratch per buffer set (two sets alternate); sets the chunk size
  int bounds[3] = {4, 8, 16};     // rank classes: ascending upper bounds, the last 16; unused 0
  int compact = 0;                // FP32 forms: N-1 over each topology's compacted valid contingencies
  int remainder = 1;              // a short contingency remainder goes to the final pass
};
inline bool operator==(const SchedPlan& a, const SchedPlan& b) {
  return a.budget_mb == b.budget_mb && a.bounds[0] == b.bounds[0] && a.bounds[1] == b.bounds[1] &&
         a.bounds[2] == b.bounds[2] && a.compact == b.compact && a.remainder == b.remainder;
}

// What a tuned schedule is keyed on: the shape of a batch as far as it changes
// the work per topology (timesteps, candidates, the extra outputs).
struct ShapeKey {
  int T = 0, U = 0, ti = 0, top_k = 0, gen = 0, multi = 0, mode = 0;
  bool operator==(const ShapeKey& o) const {
    return T == o.T && U == o.U && ti == o.ti && top_k == o.top_k && gen == o.gen && multi == o.multi &&
           mode == o.mode;
  }
};

}  // namespace dcf

struct dcflow_ctx {
  dcflow_options opt{};
  int dev = 0;
  // grid
  int V = 0, E = 0, slack = 0;
  int n = 0, npad = 0;  // reduced size V-1 and its padding to the block size
  std::vector<int> hf, ht;
  std::vector<double> hb;
  std::vector<int> h_inc_ptr, h_inc_list;
  dcf::DevBuf f, t, b, inc_ptr, inc_list, rid, L, info;
  // study
  bool has_study = false;
  int M = 0, C = 0, NN = 0;  // monitored, contingencies, needed rows
  std::vector<int> h_mon, h_cont, h_N, h_nidx;
  dcf::DevBuf nidx;        // int[E]: branch -> needed-row index or -1
  dcf::DevBuf split_ok;    // uint8[V]
  dcf::DevBuf out_ok;      // uint8[E]: outage candidates of the study
  dcf::DevBuf monN, contN; // int[M], int[C]: needed-row index of mon / cont
  dcf::DevBuf cpos_of_mon; // int[M]: position in cont of the same branch or -1
  dcf::DevBuf mpos_of_cont;// int[C]: position in mon of the same branch or -1
  dcf::DevBuf inv_lim;     // double[M]
  dcf::DevBuf bN;          // double[NN]: susceptance of the needed branches
  dcf::DevBuf PhiN;        // double[NN*NN] base branch-to-branch factors
  dcf::DevBuf PhiNf, bNf;  // FP32 form: float copies of PhiN and bN (the monitored rows' Z, no conversions)
  dcf::DevBuf PtdfN;       // double[NN*V] base PTDF rows of the needed branches
  dcf::DevBuf PhiMC;       // Real[M*ldc] Phi[mon, cont] / limit[mon], row stride ldc
  int ldc = 0;             // round_up(C, 4): 16-byte row pitch for the tensor-memory accelerator
  std::vector<uint8_t> h_split_ok;  // split-capable buses of the study
  // Internal contingency order: the contingencies that are not bridges of the
  // base grid first (in the caller's order), then the bridges.  A split or an
  // outage only removes paths, so a base-grid bridge islands every topology:
  // the N-1 kernels cover the first C_eff only.
  int C_eff = 0;
  std::vector<int> h_cont_pos;  // internal index -> caller's position
  dcf::DevBuf cont_pos, cont_inv;  // int[C]: internal -> caller position, caller position -> internal
  // multi-outage N-1 sets (Def. 4): CSR over entries, each entry's needed-row
  // index and monitored position, and Phi[mon, entry] / limit transposed [entries][Mpad]
  int n_multi = 0, n_multi_ent = 0;
  dcf::DevBuf multi_ptr, multiN, multi_mpos, PhiMO;
  dcf::DevBuf PhiCM;       // Real[C*Mpad] the same factors transposed (final pass, screened N-1; first solve builds it)
  bool phicm_ready = false;
  dcf::DevBuf Y;           // solve workspace
  // batch scratch
  dcf::DevBuf p0;          // double[NN*(T+R)]: base flows, then R pool columns
  dcf::DevBuf p0f;         // FP32 form: float copy of p0
  dcf::DevBuf pool, var_k;  // candidate pool buses; pool index of every candidate entry
  dcf::DevBuf dp;          // double[NN*U] base flow change of each candidate
  dcf::DevBuf rank, status, perm, hist, hist_host;
  dcf::DevBuf cm_scratch;  // float[N*T*C] per-contingency maxima for the top-k pass when not requested
  // output-first candidates: per (topology, timestep x candidate) the per-contingency maxima
  // float[N*T*U*C] and the top-k cases int, int, float [N*T*U*k] of every candidate
  dcf::DevBuf of_cmax, of_top;
  dcf::DevBuf gen_cols;    // Real[G*M] PTDF[mon, gen_bus] / limit of the batch's generators
  dcf::ChunkBufs bufs[2];
  cudaStream_t side = nullptr;           // preparation stream (created on first use)
  cudaEvent_t ev_ready = nullptr, ev_prep[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
  dcf::DevBuf err;         // int: set by a kernel whose bounded wait expired
  int64_t launches = 0;
  int64_t chunk_cap = 0;
  // schedule: fixed by dcflow_set_schedule, else tuned per batch shape
  // (dcflow_autotune, or automatically with opt.autotune), else the defaults
  bool sched_fixed = false;
  dcf::SchedPlan sched;
  std::vector<std::pair<dcf::ShapeKey, dcf::SchedPlan>> tuned;
  bool tuning = false;  // inside the autotuner: the plan below is forced
  dcf::SchedPlan tune_plan;
  dcf::SchedPlan last_plan;  // the schedule of the last solve
  int last_uc = 0;           // candidates per (topology, timestep) of the last solve
  // kernel timing (dcflow_profile)
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;  // pairs (start, stop) per timed launch
  std::vector<int> prof_kind;        // DCFLOW_PROF_* of each pair
  size_t prof_used = 0;
  // start a timed launch of `kind` on `st` (returns the pair, or -1 when not profiling)
  int prof_begin(cudaStream_t st) {
    if (!prof_on) return -1;
    while (prof_ev.size() < prof_used + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      prof_ev.push_back(e);
    }
    const int p = (int)prof_used;
    prof_used += 2;
    prof_kind.resize(prof_used / 2);
    prof_kind[p / 2] = -1;  // completed by prof_end
    return cudaEventRecord(prof_ev[p], st) == cudaSuccess ? p : -1;
  }
  void prof_end(int p, int kind, cudaStream_t st) {
    if (p < 0) return;
    prof_kind[p / 2] = kind;
    cudaEventRecord(prof_ev[p + 1], st);
  }
};
