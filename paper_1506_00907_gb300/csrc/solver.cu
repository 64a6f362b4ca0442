// Host engine and C ABI: uploads the discretisation, schedules the fused step kernel per step of
// the finest level (Algorithm 1), and drives one RTM shot (Sec. 2, Sec. 4.3).
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <array>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <utility>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <vector>

#include "ridg.h"
#include "dispatch.hpp"
#include "data_scale.hpp"
#include "energy_noalloc.hpp"
#include "exchange.hpp"
#include "setup.hpp"
#include "step_kernel_tc.cuh"

namespace ridg {

static thread_local std::string g_last_error;

static void set_error(const std::string& s) { g_last_error = s; }

#define RIDG_CUDA(call)                                                                                   \
  do {                                                                                                    \
    cudaError_t e_ = (call);                                                                              \
    if (e_ != cudaSuccess) throw Error{RIDG_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

template <typename F>
static auto dispatch_order(int N, F&& f) {
  switch (N) {
    case 1: return f(std::integral_constant<int, 1>{});
    case 2: return f(std::integral_constant<int, 2>{});
    case 3: return f(std::integral_constant<int, 3>{});
    case 4: return f(std::integral_constant<int, 4>{});
    case 5: return f(std::integral_constant<int, 5>{});
    default: return f(std::integral_constant<int, 6>{});
  }
}

// ---- host-side fault injection (tests): one armed failure point fires once, after a number of
// passes, through the same error path as the failure it stands for; nothing touches the GPU.
// Armed by RIDG_FAULT=<point>[:<passes before it fires>] in the environment (read when the library
// loads) or by ridg_inject_fault.
enum FaultPoint { kFaultNone = 0, kFaultAlloc, kFaultArena, kFaultAdmission, kFaultExchange };
struct FaultState {
  std::atomic<int> point{kFaultNone};
  std::atomic<int64_t> after{0};
};
static FaultState g_fault;

static int fault_point_of(const std::string& name) {
  if (name == "alloc") return kFaultAlloc;
  if (name == "arena") return kFaultArena;
  if (name == "admission") return kFaultAdmission;
  if (name == "exchange") return kFaultExchange;
  if (name == "none") return kFaultNone;
  return -1;
}

// true once, when the armed point k is passed for the (after + 1)-th time; then disarmed
static bool fault_fires(int k) {
  if (g_fault.point.load() != k) return false;
  if (g_fault.after.fetch_sub(1) > 0) return false;
  int expected = k;
  return g_fault.point.compare_exchange_strong(expected, kFaultNone);
}

static const bool g_fault_from_env = [] {
  const char* v = std::getenv("RIDG_FAULT");
  if (!v) return false;
  std::string spec(v), name = spec;
  int64_t after = 0;
  const size_t colon = spec.find(':');
  if (colon != std::string::npos) {
    name = spec.substr(0, colon);
    after = std::atoll(spec.c_str() + colon + 1);
  }
  const int k = fault_point_of(name);
  if (k <= 0) return false;
  g_fault.after.store(after);
  g_fault.point.store(k);
  return true;
}();

// NVTX range for the lifetime of the object (shot phases, fine steps by their first active level):
// seen by ncu's --nvtx filters and by timeline tools, a few tens of nanoseconds without one.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Environment switches read when a solver is created: RIDG_PROFILE=<every> turns on the CUDA-event
// profiling of ridg_set_profiling; RIDG_DEBUG=1 checks the solver's tables on the host before they
// are uploaded (a failed check is RIDG_E_INTERNAL, naming the entry).
static int env_int(const char* name, int fallback) {
  const char* v = std::getenv(name);
  if (!v || !*v) return fallback;
  char* end = nullptr;
  long x = std::strtol(v, &end, 10);
  return (end && *end == '\0') ? int(x) : fallback;
}

// Owning device allocation.
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  // at least n bytes, keeping a larger allocation (resident buffers reused across shots)
  void reserve(size_t n) {
    if (p && bytes >= n) return;
    alloc(n);
  }
  void alloc(size_t n) {
    if (n == bytes && p) return;
    release();
    if (n == 0) return;
    if (fault_fires(kFaultAlloc))
      throw Error{RIDG_E_OOM, "cudaMalloc of " + std::to_string(n) + " bytes failed (injected failure)"};
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      throw Error{RIDG_E_OOM, "cudaMalloc of " + std::to_string(n) + " bytes failed: " + cudaGetErrorString(e)};
    }
    bytes = n;
  }
};

// Owning pinned host allocation (grow-only), for boundary-trace records kept in host memory.
struct HBuf {
  void* p = nullptr;
  size_t bytes = 0;
  HBuf() = default;
  HBuf(const HBuf&) = delete;
  HBuf& operator=(const HBuf&) = delete;
  ~HBuf() { release(); }
  void release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
  }
  void reserve(size_t n) {
    if (p && bytes >= n) return;
    release();
    if (fault_fires(kFaultAlloc))
      throw Error{RIDG_E_OOM, "cudaHostAlloc of " + std::to_string(n) + " bytes failed (injected failure)"};
    cudaError_t e = cudaHostAlloc(&p, n, cudaHostAllocDefault);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      throw Error{RIDG_E_OOM, "cudaHostAlloc of " + std::to_string(n) + " bytes failed: " + cudaGetErrorString(e)};
    }
    bytes = n;
  }
};

template <typename T>
static T* dptr(const DBuf& b) {
  return static_cast<T*>(b.p);
}

template <typename T>
static void upload(DBuf& b, const std::vector<T>& v, cudaStream_t st) {
  // grow-only: a shot's tables change size with its receivers, and freeing device memory would
  // synchronise the whole device (and so stall the shots of other streams)
  b.reserve(v.size() * sizeof(T));
  if (!v.empty()) RIDG_CUDA(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
}

// Boundary-trace records of a shot beyond a device budget (Sec. 4.3: the paper moves them from the
// device to a host deque).  The records of consecutive fine steps form chunks of at most half the
// budget.  The forward run fills one half of the device buffer while a copy stream moves the chunk
// before it to pinned host memory; the backward run reads the chunks in reverse order, one half
// while the copy stream brings the next chunk back into the other.  The last two chunks never leave
// the device (a tiered shot has at least three: two chunks of half the budget would hold every
// record).  Events order the compute and copy streams; no kernel waits on a copy.
class TraceTier {
 public:
  TraceTier() = default;
  TraceTier(const TraceTier&) = delete;
  TraceTier& operator=(const TraceTier&) = delete;
  ~TraceTier() {
    if (cs_) cudaStreamSynchronize(cs_);
    for (cudaEvent_t e : ev_)
      if (e) cudaEventDestroy(e);
    if (cs_) cudaStreamDestroy(cs_);
  }
  // rec_base[t] is the first record of step t (t = 0 .. n_steps, the last entry the total), each
  // record rec_bytes long.  Returns false when the budget is 0 or holds every record (no tier);
  // throws when half the budget cannot hold the records of the largest step.
  bool plan(const std::vector<int64_t>& rec_base, size_t rec_bytes, size_t budget) {
    const int64_t n_steps = int64_t(rec_base.size()) - 1;
    const int64_t total = rec_base.back();
    active_ = false;
    if (budget == 0 || size_t(total) * rec_bytes <= budget) return false;
    const int64_t cap = int64_t(budget / 2 / rec_bytes);
    int64_t largest = 0;
    for (int64_t t = 0; t < n_steps; ++t) largest = std::max(largest, rec_base[t + 1] - rec_base[t]);
    if (largest > cap)
      throw Error{RIDG_E_INVALID_ARG, "boundary-trace budget of " + std::to_string(budget) +
                                          " bytes is below twice the records of one step (" +
                                          std::to_string(2 * largest * int64_t(rec_bytes)) + " bytes)"};
    rec_bytes_ = rec_bytes;
    cap_ = cap;
    first_step_.assign(1, 0);
    chunk_of_.assign(size_t(n_steps), 0);
    for (int64_t t = 0; t < n_steps; ++t) {
      if (rec_base[t + 1] - rec_base[first_step_.back()] > cap) first_step_.push_back(t);
      chunk_of_[size_t(t)] = int(first_step_.size()) - 1;
    }
    first_step_.push_back(n_steps);
    first_rec_.resize(first_step_.size());
    for (size_t k = 0; k < first_step_.size(); ++k) first_rec_[k] = rec_base[size_t(first_step_[k])];
    if (!cs_) {
      RIDG_CUDA(cudaStreamCreateWithFlags(&cs_, cudaStreamNonBlocking));
      for (cudaEvent_t& e : ev_) RIDG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    active_ = true;
    return true;
  }
  bool active() const { return active_; }
  int n_chunks() const { return int(first_step_.size()) - 1; }
  size_t device_bytes() const { return size_t(2 * cap_) * rec_bytes_; }
  int chunk_of(int64_t t) const { return chunk_of_[size_t(t)]; }
  int64_t first_record(int k) const { return first_rec_[size_t(k)]; }
  int64_t host_bytes() const { return host_bytes_; }

  // before the forward run: the copy stream's earlier work (a previous shot) is done first
  void begin_forward(cudaStream_t st) {
    after_copies(st);
    cur_ = -1;
    drained_[0] = drained_[1] = false;
    host_bytes_ = 0;
  }
  // device address of chunk k for a forward step that records into it (chunks in ascending order)
  char* forward_chunk(int k, char* dev, char* host, cudaStream_t st) {
    if (k != cur_) {
      if (cur_ >= 0 && cur_ < n_chunks() - 2) {  // the last two chunks stay on the device
        const size_t n = size_t(first_rec_[cur_ + 1] - first_rec_[cur_]) * rec_bytes_;
        RIDG_CUDA(cudaEventRecord(ev_[kFilled], st));
        RIDG_CUDA(cudaStreamWaitEvent(cs_, ev_[kFilled], 0));
        RIDG_CUDA(cudaMemcpyAsync(host + size_t(first_rec_[cur_]) * rec_bytes_, half(dev, cur_), n,
                                  cudaMemcpyDeviceToHost, cs_));
        RIDG_CUDA(cudaEventRecord(ev_[kDrained + (cur_ & 1)], cs_));
        drained_[cur_ & 1] = true;
        host_bytes_ += int64_t(n);
      }
      if (drained_[k & 1]) RIDG_CUDA(cudaStreamWaitEvent(st, ev_[kDrained + (k & 1)], 0));
      drained_[k & 1] = false;
      cur_ = k;
    }
    return half(dev, k);
  }
  // before the backward run, which reads the steps down to lowest_step
  void begin_backward(int64_t lowest_step) {
    cur_ = n_chunks();
    const int64_t last = int64_t(chunk_of_.size()) - 1;
    lowest_ = chunk_of(std::min(std::max<int64_t>(lowest_step, 0), last));
  }
  // device address of chunk k for a backward step that reads it (chunks in descending order)
  char* backward_chunk(int k, char* dev, char* host, cudaStream_t st) {
    if (k != cur_) {
      const int K = n_chunks();
      if (k < K - 2) RIDG_CUDA(cudaStreamWaitEvent(st, ev_[kReady + (k & 1)], 0));
      const int next = k - 1;
      if (next >= lowest_ && next < K - 2) {
        // into the other half, whose chunk (k + 1) the steps launched so far have read
        const size_t n = size_t(first_rec_[next + 1] - first_rec_[next]) * rec_bytes_;
        RIDG_CUDA(cudaEventRecord(ev_[kUsed], st));
        RIDG_CUDA(cudaStreamWaitEvent(cs_, ev_[kUsed], 0));
        RIDG_CUDA(cudaMemcpyAsync(half(dev, next), host + size_t(first_rec_[next]) * rec_bytes_, n,
                                  cudaMemcpyHostToDevice, cs_));
        RIDG_CUDA(cudaEventRecord(ev_[kReady + (next & 1)], cs_));
      }
      cur_ = k;
    }
    return half(dev, k);
  }
  // the compute stream waits for every copy issued so far
  void after_copies(cudaStream_t st) {
    if (!cs_) return;
    RIDG_CUDA(cudaEventRecord(ev_[kTail], cs_));
    RIDG_CUDA(cudaStreamWaitEvent(st, ev_[kTail], 0));
  }

 private:
  enum { kFilled = 0, kDrained = 1, kReady = 3, kUsed = 5, kTail = 6, kEvents = 7 };
  char* half(char* dev, int k) const { return dev + size_t(k & 1) * size_t(cap_) * rec_bytes_; }
  bool active_ = false;
  size_t rec_bytes_ = 0;
  int64_t cap_ = 0;
  std::vector<int64_t> first_step_, first_rec_;
  std::vector<int> chunk_of_;
  int cur_ = -1, lowest_ = 0;
  bool drained_[2] = {false, false};
  int64_t host_bytes_ = 0;
  cudaStream_t cs_ = nullptr;
  cudaEvent_t ev_[kEvents] = {};
};

static int mod3(int64_t x) { return int(((x % 3) + 3) % 3); }

static double ricker(double t, double f0, double tp, double amp) {
  double a = M_PI * f0 * (t - tp);
  a *= a;
  return amp * (1.0 - 2.0 * a) * std::exp(-a);
}

// Source wavelet of a ridg_source (a copy: sampled wavelets keep their own samples).
struct Wavelet {
  int kind = RIDG_SRC_RICKER;
  double f0 = 0.0, tp = 0.0, amp = 1.0, dt = 0.0;
  std::vector<double> samples;
  static Wavelet of(const ridg_source& s) {
    Wavelet w;
    w.kind = s.kind;
    w.f0 = s.f0;
    w.tp = s.t_peak;
    w.amp = s.amplitude;
    if (s.kind == RIDG_SRC_SAMPLED) {
      if (!(s.sample_dt > 0.0) || s.n_samples < 1 || !s.samples)
        throw Error{RIDG_E_INVALID_ARG, "sampled source needs sample_dt > 0, n_samples >= 1 and samples"};
      w.dt = s.sample_dt;
      w.samples.assign(s.samples, s.samples + s.n_samples);
    } else if (s.kind != RIDG_SRC_RICKER) {
      throw Error{RIDG_E_INVALID_ARG, "unknown source kind"};
    }
    return w;
  }
  // f(t): the Ricker pulse, or the 4-point Lagrange interpolant of the samples on the nodes
  // n_lo - 1 .. n_lo + 2 around t / dt (zero outside the samples)
  double operator()(double t) const {
    if (kind == RIDG_SRC_RICKER) return ricker(t, f0, tp, amp);
    const double u = t / dt, n_lo = std::floor(u), x = u - n_lo;
    const double xs[4] = {-1.0, 0.0, 1.0, 2.0};
    double acc = 0.0;
    for (int i = 0; i < 4; ++i) {
      const double n = n_lo - 1.0 + i;
      if (n < 0.0 || n >= double(samples.size())) continue;
      double li = 1.0;
      for (int j = 0; j < 4; ++j)
        if (j != i) li *= (x - xs[j]) / (xs[i] - xs[j]);
      acc += li * samples[size_t(n)];
    }
    return amp * acc;
  }
};

}  // namespace ridg

struct ridg_mesh {
  ridg::MeshData m;
  std::unique_ptr<ridg::PointLocator> loc;  // built on the first ridg_mesh_locate
};

struct ridg_solver {
  virtual ~ridg_solver() = default;
  virtual void info(ridg_info* out) const = 0;
  virtual void levels(int32_t* out) const = 0;
  virtual void nodes(double* out) const = 0;
  virtual void set_state(const double* q) = 0;
  virtual void set_history(const double* r1, const double* r2) = 0;
  virtual void eval_rhs(const double* q, double* out) = 0;
  virtual void step(int64_t n) = 0;
  virtual void get_state(double* q) = 0;
  virtual double energy() = 0;
  virtual void energy_noalloc(double* out_dev) = 0;
  virtual int64_t trace_len(double t_final) const = 0;
  virtual void shot(const ridg_source& src, const double* rec, int64_t nrec, double t_final, double t_i,
                    const double* obs_dev, double* traces_dev, double* imgp_dev, double* imgq_dev,
                    const double* e_up) = 0;
  // n shots in lockstep, device buffers (ridg_rtm_shots_device)
  virtual void shots(int32_t n, const ridg_shot_io* io, double t_final, double t_i, const double* e_up) = 0;
  virtual cudaStream_t stream() const = 0;
  virtual const ridg_shot_stats& stats() = 0;
  virtual void set_profiling(int every) = 0;
  virtual void set_trace_budget(int64_t device_bytes) = 0;
  // CUDA-graph replay of repeated shots with the same launch arguments (ridg_set_graph_replay)
  virtual void set_graph_replay(bool on) = 0;
  // device bytes a shot of this record length would still allocate (arena growth, first-shot buffers)
  virtual size_t shot_extra_device_bytes(double t_final) const = 0;
  // the same for a batch of n shots in lockstep
  virtual size_t shots_extra_device_bytes(double t_final, int32_t n) const = 0;
  // frees the device buffers only a shot uses (the next shot allocates them again); returns their bytes
  virtual size_t release_shot_buffers() = 0;
  virtual void forward(const ridg_source& src, const double* rec, int64_t nrec, double t_final,
                       double* traces_dev) = 0;
  virtual void set_state_device(const double* q_dev) = 0;
  virtual void get_state_device(double* q_dev) = 0;
  // velocity gradient (single rate level): see ridg_set_velocity / ridg_misfit_forward / _backward
  virtual void set_velocity(const double* c) = 0;
  virtual void eval_adjoint_rhs(const double* lam, double* out) = 0;
  virtual double misfit_forward(const ridg_source& src, const double* rec, int64_t nrec, double t_final,
                                const double* observed, int n_ckpt, double* traces_host) = 0;
  virtual void misfit_backward(double* grad) = 0;
};

// A shot on a partitioned mesh, one solver per part (ridg_group_*).
struct ridg_group {
  virtual ~ridg_group() = default;
  virtual void shot(const ridg_source& src, const double* rec, int64_t nrec, double t_final, double t_i,
                    const double* observed, double* traces_out, double* image_p, double* image_q,
                    const double* e_up) = 0;
  virtual void info(ridg_group_info* out) const = 0;
  virtual int64_t trace_len(double t_final, int32_t* np_out) const = 0;
};

namespace ridg {

template <typename real>
struct Wave {
  DBuf q, ring, trace;
  DBuf inj_range, inj_w, inj_row;
};

// What a solver for one part of a partitioned mesh (Sec. 4.2) asks of the group that drives the
// parts: after each fine step (and after the traces are initialised) the interface traces its
// elements pushed into their ghosts' inboxes go to the parts that own those ghosts, and the data
// scale of the receiver run is taken over the data of every part.
template <typename real>
class Engine;
template <typename real>
struct PartHook {
  virtual ~PartHook() = default;
  // pushers: levels >= first_level pushed traces at this step; waves: bit w = wavefield w
  virtual void exchange(Engine<real>& e, int first_level, int waves) = 0;
  // work: the engine's data-scale work buffer, holding this part's max |data| bits
  virtual void combine_data_scale(Engine<real>& e, void* work) = 0;
};

template <typename real>
class Group;

template <typename real>
class Engine final : public ridg_solver {
  template <typename R>
  friend class Group;

 public:
  Engine(const MeshData& mesh, int N, const double* c, const double* rho, const ridg_options& opt, cudaStream_t st,
         const int32_t* part = nullptr, int32_t rank = 0)
      : mesh_(mesh), N_(N), st_(st) {
    {
      // the device numbers the element's nodes so that face-node gathers spread over the banks;
      // every array that crosses the C ABI stays in the reference numbering
      RefElem r0 = build_reference(N);
      std::vector<int> order = bank_spread_order(r0);
      ref_ = permute_nodes(r0, order);
      pos_of_.assign(order.size(), 0);
      for (int p = 0; p < int(order.size()); ++p) pos_of_[order[p]] = p;
    }
    Np_ = ref_.Np;
    Nfp_ = ref_.Nfp;
    NFPP_ = Nfp_ <= 16 ? 16 : 32;
    NPa_ = 2 * ((Np_ + 1) / 2);
    geo_ = build_geometry(mesh_);
    loc_ = build_locator(mesh_);
    c_.assign(c, c + mesh_.K);
    c_ref_ = c_;
    rho_.assign(rho, rho + mesh_.K);
    for (int64_t k = 0; k < mesh_.K; ++k)
      if (!(rho_[k] > 0.0) || !(c_[k] > 0.0) || !std::isfinite(rho_[k]) || !std::isfinite(c_[k]))
        throw Error{RIDG_E_INVALID_ARG, "c and rho must be positive and finite"};
    double cfl = opt.cfl > 0 ? opt.cfl : 0.15;
    cfl_ = cfl;
    int nlm = opt.n_levels_max > 0 ? opt.n_levels_max : 3;
    tau_scale_ = opt.tau_scale > 0 ? opt.tau_scale : 1.0;
    if (opt.contraction != RIDG_CONTRACT_TENSOR && opt.contraction != RIDG_CONTRACT_CUDA_CORES &&
        opt.contraction != RIDG_CONTRACT_TENSOR_BF16 && opt.contraction != RIDG_CONTRACT_TENSOR_FP16 &&
        opt.contraction != RIDG_CONTRACT_TENSOR_TF32)
      throw Error{RIDG_E_INVALID_ARG,
                  "contraction must be one of RIDG_CONTRACT_TENSOR, _CUDA_CORES, _TENSOR_BF16, _TENSOR_FP16, _TENSOR_TF32"};
    // RIDG_CONTRACT_TENSOR: the TF32 split up to N = 4, the FP16 split with column scales from N = 5
    // (measured faster there, and more accurate at every order)
    contraction_ = std::is_same<real, float>::value ? opt.contraction : RIDG_CONTRACT_CUDA_CORES;
    if (contraction_ == RIDG_CONTRACT_TENSOR && N >= 5) contraction_ = RIDG_CONTRACT_TENSOR_FP16;
    if (contraction_ == RIDG_CONTRACT_TENSOR_TF32) contraction_ = RIDG_CONTRACT_TENSOR;
    image_mode_ = ((opt.image_mask & RIDG_IMAGE_P) || !(opt.image_mask & 3) ? kModeImageP : 0) |
                  ((opt.image_mask & RIDG_IMAGE_Q) || !(opt.image_mask & 3) ? kModeImageQ : 0);
    if (nlm > kMaxLevels) throw Error{RIDG_E_INVALID_ARG, "n_levels_max too large"};
    lv_ = assign_levels(mesh_, geo_, N, c_.data(), cfl, nlm);
    if (part) {
      part_.assign(part, part + mesh_.K);
      rank_ = rank;
    }
    ord_ = part ? build_part_ordering(lv_, mesh_, part, rank) : build_ordering(lv_, mesh_.K);
    n_slots_ = ord_.n_slots;
    L_ = lv_.n_levels;
    NL_ = int64_t(1) << (L_ - 1);
    check_shared_memory();
    build_nodes();
    check_face_nodes();
    debug_ = env_int("RIDG_DEBUG", 0) > 0;
    prof_every_ = std::max(0, env_int("RIDG_PROFILE", 0));
    build_tables();
    alloc_wave(w_[0]);
    reset_time();
    RIDG_CUDA(cudaStreamSynchronize(st_));
  }

  cudaStream_t stream() const override { return st_; }
  const ridg_shot_stats& stats() override {
    RIDG_CUDA(cudaStreamSynchronize(st_));
    double fw = 0.0, bw = 0.0;
    int64_t nf = 0, nb = 0;
    for (size_t i = 0; i < prof_used_; ++i) {
      float ms = 0.f;
      RIDG_CUDA(cudaEventElapsedTime(&ms, prof_ev_[2 * i], prof_ev_[2 * i + 1]));
      if (prof_w_[i] == 1) {
        fw += ms;
        ++nf;
      } else {
        bw += ms;
        ++nb;
      }
    }
    stats_.prof_forward_ms = fw;
    stats_.prof_backward_ms = bw;
    stats_.prof_forward_launches = nf;
    stats_.prof_backward_launches = nb;
    return stats_;
  }
  void set_profiling(int every) override { prof_every_ = std::max(0, every); }
  void set_trace_budget(int64_t device_bytes) override {
    if (device_bytes < 0) throw Error{RIDG_E_INVALID_ARG, "boundary-trace budget must be >= 0"};
    trace_budget_ = size_t(device_bytes);
  }

  ~Engine() override {
    for (auto e : prof_ev_) cudaEventDestroy(e);
    drop_graph();
  }
  void set_graph_replay(bool on) override {
    RIDG_CUDA(cudaStreamSynchronize(st_));
    graph_on_ = on;
    drop_graph();
  }

  void info(ridg_info* out) const override {
    std::memset(out, 0, sizeof(*out));
    out->N = N_;
    out->Np = Np_;
    out->Nfp = Nfp_;
    out->n_levels = L_;
    out->K = mesh_.K;
    out->dt_local = lv_.dt_local;
    out->dt_global = lv_.dt_local * double(NL_);
    for (int l = 1; l <= L_ && l <= 8; ++l)
      out->level_count[l - 1] = std::count(lv_.level.begin(), lv_.level.end(), l);
    out->n_boundary_faces = n_bfaces_;
    out->device_bytes = int64_t(device_bytes());
    out->n_half_step = n_half_;
  }
  void levels(int32_t* out) const override {
    for (int64_t k = 0; k < mesh_.K; ++k) out[k] = lv_.level[k];
  }
  void nodes(double* out) const override {
    for (int64_t k = 0; k < mesh_.K; ++k)
      for (int n = 0; n < Np_; ++n)
        for (int d = 0; d < 3; ++d) out[(k * Np_ + n) * 3 + d] = xnodes_[(k * Np_ + pos_of_[n]) * 3 + d];
  }

  // ------------------------------------------------------------------ state
  void set_state(const double* q) override {
    std::vector<real> h = to_slots(q);
    RIDG_CUDA(cudaMemcpyAsync(w_[0].q.p, h.data(), h.size() * sizeof(real), cudaMemcpyHostToDevice, st_));
    RIDG_CUDA(cudaMemsetAsync(w_[0].ring.p, 0, w_[0].ring.bytes, st_));
    reset_time();
    init_traces(w_[0], mod3(tau_));
    RIDG_CUDA(cudaStreamSynchronize(st_));
  }
  void set_history(const double* r1, const double* r2) override {
    size_t qb = qsize() * sizeof(real);
    // with every level counter at 0 the two older ring slots are 2 (one step back) and 1
    const double* src[2] = {r1, r2};
    const int slot[2] = {2, 1};
    for (int i = 0; i < 2; ++i) {
      char* dst = static_cast<char*>(w_[0].ring.p) + slot[i] * qb;
      if (!src[i]) {
        RIDG_CUDA(cudaMemsetAsync(dst, 0, qb, st_));
      } else {
        std::vector<real> h = to_slots(src[i]);
        RIDG_CUDA(cudaMemcpyAsync(dst, h.data(), qb, cudaMemcpyHostToDevice, st_));
      }
    }
    std::fill(ring_count_.begin(), ring_count_.end(), 0);
    RIDG_CUDA(cudaStreamSynchronize(st_));
  }
  void eval_rhs(const double* q, double* out) override {
    Wave<real> tmp;
    tmp.q.alloc(qsize() * sizeof(real));
    tmp.trace.alloc(trace_slot_elems() * sizeof(real));
    DBuf rout;
    rout.alloc(qsize() * sizeof(real));
    RIDG_CUDA(cudaMemsetAsync(rout.p, 0, rout.bytes, st_));
    std::vector<real> h = to_slots(q);
    RIDG_CUDA(cudaMemcpyAsync(tmp.q.p, h.data(), h.size() * sizeof(real), cudaMemcpyHostToDevice, st_));
    init_traces_into(dptr<real>(tmp.q), dptr<real>(tmp.trace), 0);
    StepArgs<real> a = base_args();
    a.wave[0] = wave_args(tmp);
    a.wave[0].amp_mode = 0;
    a.slot_lo = 0;
    a.slot_hi = ord_.owned_end;
    a.trace_read = 0;
    a.tau_sign = real(1);
    a.mode = kModeRhsOnly;
    a.rhs_out = dptr<real>(rout);
    launch(a, 1);
    std::vector<real> r(qsize());
    RIDG_CUDA(cudaMemcpyAsync(r.data(), rout.p, rout.bytes, cudaMemcpyDeviceToHost, st_));
    RIDG_CUDA(cudaStreamSynchronize(st_));
    from_slots(r, out);
  }
  void step(int64_t n) override {
    if (n < 0) throw Error{RIDG_E_INVALID_ARG, "n_global must be >= 0"};
    for (int64_t g = 0; g < n; ++g)
      for (int64_t s = 0; s < NL_; ++s) {
        StepArgs<real> a = fine_args(+1, 1, 0);
        a.wave[0] = wave_args(w_[0]);
        a.wave[0].amp_mode = 0;
        launch_fine(a, +1, 1);
      }
    RIDG_CUDA(cudaGetLastError());
  }
  void get_state(double* q) override {
    std::vector<real> h(qsize());
    RIDG_CUDA(cudaMemcpyAsync(h.data(), w_[0].q.p, h.size() * sizeof(real), cudaMemcpyDeviceToHost, st_));
    RIDG_CUDA(cudaStreamSynchronize(st_));
    from_slots(h, q);
  }
  double energy() override { return energy_of(dptr<real>(w_[0].q)); }
  void energy_noalloc(double* out_dev) override {
    if (n_slots_ > ridg::energy_noalloc_max_slots())
      throw Error{RIDG_E_INVALID_ARG, "ridg_energy_noalloc: " + std::to_string(n_slots_) +
                                          " element slots exceed the fixed scratch limit of " +
                                          std::to_string(ridg::energy_noalloc_max_slots())};
    cudaError_t e = ridg::energy_noalloc(N_, std::is_same<real, double>::value, w_[0].q.p, n_slots_,
                                         dptr<const double>(J_d_), mat_d_.p, dptr<const int>(meta_d_),
                                         dptr<const double>(M_d_), out_dev, st_);
    if (e != cudaSuccess) throw Error{RIDG_E_CUDA, std::string("ridg_energy_noalloc: ") + cudaGetErrorString(e)};
  }
  void set_state_device(const double* q_dev) override {
    if (!q_dev) throw Error{RIDG_E_INVALID_ARG, "q_dev is null"};
    state_io(true, q_dev, nullptr);
    RIDG_CUDA(cudaMemsetAsync(w_[0].ring.p, 0, w_[0].ring.bytes, st_));
    reset_time();
    init_traces(w_[0], mod3(tau_));
  }
  void get_state_device(double* q_dev) override {
    if (!q_dev) throw Error{RIDG_E_INVALID_ARG, "q_dev is null"};
    state_io(false, nullptr, q_dev);
  }
  void state_io(bool to_slots, const double* in, double* out) {
    cudaError_t e = dispatch_order(N_, [&](auto NC) {
      return Launch<decltype(NC)::value, real>::state_io(to_slots, in, out, dptr<real>(w_[0].q),
                                                          dptr<const int64_t>(slot_of_d_), dptr<const int>(pos_d_),
                                                          mesh_.K, st_);
    });
    if (e != cudaSuccess) throw Error{RIDG_E_CUDA, cudaGetErrorString(e)};
    ++stats_.kernel_launches;
  }

  // Forward modelling: the forward source run of a shot alone (Sec. 2), receiver pressures
  // sampled at every global step into traces_dev [nrec][n_t].
  void forward(const ridg_source& src, const double* rec, int64_t nrec, double t_final,
               double* traces_dev) override {
    NvtxRange nv("ridg forward");
    if (!(t_final > 0.0)) throw Error{RIDG_E_INVALID_ARG, "t_final must be > 0"};
    if (nrec < 0 || (nrec > 0 && (!rec || !traces_dev))) throw Error{RIDG_E_INVALID_ARG, "bad receiver list"};
    const Wavelet wav = Wavelet::of(src);
    std::memset(&stats_, 0, sizeof(stats_));
    prof_used_ = 0;
    const double dtl = lv_.dt_local, dtg = dtl * double(NL_);
    const int64_t n_global = int64_t(std::ceil(t_final / dtg - 1e-9));
    const int64_t n_t = n_global + 1;
    stats_.n_global = n_global;
    double rst[3];
    const int64_t ks = locate_point(mesh_, loc_, src.xyz, rst);
    if (ks < 0) throw Error{RIDG_E_NOT_FOUND, "source lies outside the mesh"};
    {
      std::vector<int2> range(n_slots_, make_int2(0, 0));
      if (owned(ks)) range[ord_.slot_of[ks]] = make_int2(0, 1);
      upload(w_[0].inj_range, range, st_);
      upload(w_[0].inj_w, projected_dirac(ks, rst), st_);
      upload(w_[0].inj_row, std::vector<int>{0}, st_);
    }
    std::vector<int64_t> rslot(std::max<int64_t>(nrec, 1), 0);
    std::vector<real> rrow(std::max<int64_t>(nrec, 1) * Np_, real(0));
    for (int64_t r = 0; r < nrec; ++r) {
      const int64_t kr = locate_point(mesh_, loc_, rec + 3 * r, rst);
      if (kr < 0) throw Error{RIDG_E_NOT_FOUND, "receiver " + std::to_string(r) + " lies outside the mesh"};
      rslot[r] = owned(kr) ? ord_.slot_of[kr] : -1;
      std::vector<double> l = ref_.lagrange_at({rst[0], rst[1], rst[2]});
      for (int m = 0; m < Np_; ++m) rrow[r * Np_ + m] = real(l[m]);
    }
    upload(rec_slot_, rslot, st_);
    upload(rec_row_, rrow, st_);
    zero_wave(w_[0]);
    reset_time();
    if (nrec > 0) RIDG_CUDA(cudaMemsetAsync(traces_dev, 0, size_t(nrec) * n_t * sizeof(double), st_));
    sample(traces_dev, n_t, 0, nrec);
    for (int64_t g = 0; g < n_global; ++g) {
      for (int64_t sub = 0; sub < NL_; ++sub) {
        StepArgs<real> a = fine_args(+1, 1, 0);
        a.wave[0] = wave_args(w_[0]);
        a.wave[0].amp_mode = 1;
        a.wave[0].amp = real(wav(double(tau_) * dtl));
        launch_fine(a, +1, 1);
      }
      sample(traces_dev, n_t, g + 1, nrec);
    }
    stats_.dof_updates_forward = dof_;
    RIDG_CUDA(cudaGetLastError());
  }

  // ------------------------------------------------------------------ velocity gradient
  void set_velocity(const double* c) override {
    if (!c) throw Error{RIDG_E_INVALID_ARG, "c is null"};
    for (int64_t k = 0; k < mesh_.K; ++k)
      if (!(c[k] > 0.0) || !std::isfinite(c[k])) throw Error{RIDG_E_INVALID_ARG, "c must be positive and finite"};
    // the time step and levels stay those of the creation model: an element may speed up only while
    // its Courant number on its level's step stays within kVelocityCflMargin x the solver's CFL
    // constant (AB3 with this step rule measured stable to C = 0.22, unstable at 0.25)
    for (int64_t k = 0; k < mesh_.K; ++k) {
      const double dt_l = lv_.dt_local * double(int64_t(1) << (L_ - lv_.level[k]));
      const double courant = dt_l * (N_ + 1.0) * (N_ + 1.0) * c[k] / geo_.lmin[k];
      if (courant > kVelocityCflMargin * cfl_ * (1.0 + 1e-12))
        throw Error{RIDG_E_INVALID_ARG, "velocity of element " + std::to_string(k) + " (" + std::to_string(c[k]) +
                                            " m/s) exceeds the stability bound of its frozen time step: Courant " +
                                            std::to_string(courant) + " > " +
                                            std::to_string(kVelocityCflMargin * cfl_)};
    }
    c_.assign(c, c + mesh_.K);
    upload_material();
    adj_.ready = false;
    RIDG_CUDA(cudaStreamSynchronize(st_));
  }

  // out = A^T lam; adjt: scratch for the adjoint traces and their inboxes (2 trace slots).  With s1,
  // lam += h (a1 out + a2 s1 + a3 s2) in the same pass (the adjoint Adams-Bashforth update).
  void adjoint_rhs_into(real* lam, real* out, real* adjt, const real* s1 = nullptr, const real* s2 = nullptr,
                        double h = 0.0) {
    cudaError_t e = dispatch_order(N_, [&](auto NC) {
      return Launch<decltype(NC)::value, real>::adj_rhs(
          lam, adjt, adjt + trace_slot_elems(), out, n_slots_, dptr<const double>(geo_d_), dptr<const real>(mat_d_),
          dptr<const int>(meta_d_), dptr<const real>(Dt4_d_), dptr<const real>(Lt_d_), NPa_, dptr<const int>(fmask_d_),
          dptr<const int>(nbr_d_), dptr<const uint8_t>(finfo_d_), dptr<const int>(perm_d_), s1, s2, h, st_);
    });
    if (e != cudaSuccess) throw Error{RIDG_E_CUDA, cudaGetErrorString(e)};
  }

  void eval_adjoint_rhs(const double* lam, double* out) override {
    if (!lam || !out) throw Error{RIDG_E_INVALID_ARG, "null lam or out"};
    DBuf l, o, t;
    l.alloc(qsize() * sizeof(real));
    o.alloc(qsize() * sizeof(real));
    t.alloc(2 * trace_slot_elems() * sizeof(real));
    std::vector<real> h = to_slots(lam);
    RIDG_CUDA(cudaMemcpyAsync(l.p, h.data(), h.size() * sizeof(real), cudaMemcpyHostToDevice, st_));
    adjoint_rhs_into(dptr<real>(l), dptr<real>(o), dptr<real>(t));
    std::vector<real> r(qsize());
    RIDG_CUDA(cudaMemcpyAsync(r.data(), o.p, o.bytes, cudaMemcpyDeviceToHost, st_));
    RIDG_CUDA(cudaStreamSynchronize(st_));
    from_slots(r, out);
  }

  void misfit_step(const Wavelet& wav) {
    StepArgs<real> a = fine_args(+1, 1, 0);
    a.wave[0] = wave_args(w_[0]);
    a.wave[0].amp_mode = 1;
    a.wave[0].amp = real(wav(double(tau_) * lv_.dt_local));
    launch_fine(a, +1, 1);
  }

  double misfit_forward(const ridg_source& src, const double* rec, int64_t nrec, double t_final,
                        const double* observed, int n_ckpt, double* traces_host) override {
    NvtxRange nv("ridg misfit forward");
    if (!(t_final > 0.0)) throw Error{RIDG_E_INVALID_ARG, "t_final must be > 0"};
    if (nrec < 1 || !rec || !observed) throw Error{RIDG_E_INVALID_ARG, "receivers and observed traces are required"};
    adj_.ready = false;
    adj_.wav = Wavelet::of(src);
    const double dtl = lv_.dt_local, dt = dtl * double(NL_);  // fine and global step
    const int64_t n_global = int64_t(std::ceil(t_final / dt - 1e-9)), n_t = n_global + 1;
    const int64_t n_ck_max = n_ckpt > 0 ? n_ckpt : 16;
    adj_.n_global = n_global;
    adj_.seg = std::max<int64_t>(1, (n_global + n_ck_max - 1) / n_ck_max);
    adj_.n_ck = (n_global + adj_.seg - 1) / adj_.seg;
    adj_.nrec = nrec;
    double rst[3];
    const int64_t ks = locate_point(mesh_, loc_, src.xyz, rst);
    if (ks < 0) throw Error{RIDG_E_NOT_FOUND, "source lies outside the mesh"};
    adj_.src_slot = ord_.slot_of[ks];
    const std::vector<real> w_src = projected_dirac(ks, rst);
    {
      std::vector<int2> range(n_slots_, make_int2(0, 0));
      range[adj_.src_slot] = make_int2(0, 1);
      upload(w_[0].inj_range, range, st_);
      upload(w_[0].inj_w, w_src, st_);
      upload(w_[0].inj_row, std::vector<int>{0}, st_);
      upload(adj_w_, w_src, st_);
    }
    std::vector<int64_t> rslot(nrec, 0);
    std::vector<real> rrow(nrec * Np_, real(0));
    for (int64_t r = 0; r < nrec; ++r) {
      const int64_t kr = locate_point(mesh_, loc_, rec + 3 * r, rst);
      if (kr < 0) throw Error{RIDG_E_NOT_FOUND, "receiver " + std::to_string(r) + " lies outside the mesh"};
      rslot[r] = owned(kr) ? ord_.slot_of[kr] : -1;
      std::vector<double> l = ref_.lagrange_at({rst[0], rst[1], rst[2]});
      for (int m = 0; m < Np_; ++m) rrow[r * Np_ + m] = real(l[m]);
    }
    upload(rec_slot_, rslot, st_);
    upload(rec_row_, rrow, st_);
    upload(adj_rec_slot_, rslot, st_);
    upload(adj_rec_row_, rrow, st_);
    {
      // receivers grouped by element slot (stable: each group keeps the receivers' order)
      std::vector<int> order(nrec);
      for (int64_t r = 0; r < nrec; ++r) order[r] = int(r);
      std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return rslot[x] < rslot[y]; });
      std::vector<int> grp{0};
      for (int64_t i = 1; i < nrec; ++i)
        if (rslot[order[i]] != rslot[order[i - 1]]) grp.push_back(int(i));
      grp.push_back(int(nrec));
      adj_.n_groups = int64_t(grp.size()) - 1;
      upload(adj_grp_, grp, st_);
      upload(adj_rec_sorted_, order, st_);
    }
    // the wavelet at every fine step, as the step kernel injects it
    adj_.amp.assign(n_global * NL_ + 1, 0.0);
    for (int64_t n = 0; n <= n_global * NL_; ++n) adj_.amp[n] = double(real(adj_.wav(double(n) * dtl)));
    const size_t qb = qsize() * sizeof(real), tb = 3 * trace_slot_elems() * sizeof(real);
    ck_q_.reserve(size_t(adj_.n_ck) * qb);
    ck_ring_.reserve(size_t(adj_.n_ck) * 3 * qb);
    ck_trace_.reserve(size_t(adj_.n_ck) * tb);
    adj_.ck_tau.assign(adj_.n_ck, 0);
    adj_.ck_count.assign(size_t(adj_.n_ck) * L_, 0);
    DBuf y;
    y.alloc(size_t(nrec) * n_t * sizeof(double));
    zero_wave(w_[0]);
    reset_time();
    std::memset(&stats_, 0, sizeof(stats_));
    stats_.n_global = n_global;
    sample(dptr<double>(y), n_t, 0, nrec);
    for (int64_t g = 0; g < n_global; ++g) {
      if (g % adj_.seg == 0) {
        const int64_t j = g / adj_.seg;
        char* cq = static_cast<char*>(ck_q_.p) + size_t(j) * qb;
        char* cr = static_cast<char*>(ck_ring_.p) + size_t(j) * 3 * qb;
        char* ct = static_cast<char*>(ck_trace_.p) + size_t(j) * tb;
        RIDG_CUDA(cudaMemcpyAsync(cq, w_[0].q.p, qb, cudaMemcpyDeviceToDevice, st_));
        RIDG_CUDA(cudaMemcpyAsync(cr, w_[0].ring.p, 3 * qb, cudaMemcpyDeviceToDevice, st_));
        RIDG_CUDA(cudaMemcpyAsync(ct, w_[0].trace.p, tb, cudaMemcpyDeviceToDevice, st_));
        adj_.ck_tau[j] = tau_;
        for (int l = 0; l < L_; ++l) adj_.ck_count[size_t(j) * L_ + l] = ring_count_[l];
      }
      for (int64_t sub = 0; sub < NL_; ++sub) misfit_step(adj_.wav);
      sample(dptr<double>(y), n_t, g + 1, nrec);
    }
    stats_.dof_updates_forward = dof_;
    std::vector<double> yh(size_t(nrec) * n_t);
    RIDG_CUDA(cudaMemcpyAsync(yh.data(), y.p, yh.size() * sizeof(double), cudaMemcpyDeviceToHost, st_));
    RIDG_CUDA(cudaStreamSynchronize(st_));
    double J = 0.0;
    for (size_t i = 0; i < yh.size(); ++i) {
      const double r = yh[i] - observed[i];
      J += r * r;
      yh[i] = r;
    }
    J *= 0.5 * dt;
    if (traces_host)
      for (size_t i = 0; i < yh.size(); ++i) traces_host[i] = yh[i] + observed[i];
    upload(adj_res_, yh, st_);
    RIDG_CUDA(cudaStreamSynchronize(st_));
    if (!std::isfinite(J)) throw Error{RIDG_E_UNSTABLE, "non-finite misfit"};
    adj_.ready = true;
    return J;
  }

  void misfit_backward(double* grad) override {
    NvtxRange nv("ridg misfit backward");
    if (!adj_.ready) throw Error{RIDG_E_INVALID_ARG, "no misfit forward run to differentiate (or the velocity changed)"};
    if (!grad) throw Error{RIDG_E_INVALID_ARG, "grad is null"};
    if (L_ > 1) return misfit_backward_levels(grad);
    const double h = lv_.dt_local;
    const size_t qn = qsize(), qb = qn * sizeof(real), tb = 3 * trace_slot_elems() * sizeof(real);
    const int64_t n_t = adj_.n_global + 1;
    DBuf lam, sring, adjt, seg, acc;
    lam.alloc(qb);
    sring.alloc(3 * qb);
    adjt.alloc(2 * trace_slot_elems() * sizeof(real));
    seg.alloc(size_t(adj_.seg + 1) * qb);
    acc.alloc(size_t(n_slots_) * sizeof(double));  // per element slot
    RIDG_CUDA(cudaMemsetAsync(lam.p, 0, lam.bytes, st_));
    RIDG_CUDA(cudaMemsetAsync(sring.p, 0, sring.bytes, st_));
    RIDG_CUDA(cudaMemsetAsync(acc.p, 0, acc.bytes, st_));
    real* L = dptr<real>(lam);
    auto sr = [&](int64_t j) { return dptr<real>(sring) + size_t(j % 3) * qn; };
    auto sg = [&](int64_t i) { return dptr<real>(seg) + size_t(i) * qn; };
    const double a[3] = {AB::a1, AB::a2, AB::a3};
    for (int64_t j = adj_.n_ck - 1; j >= 0; --j) {
      const int64_t a0 = j * adj_.seg, b0 = std::min(a0 + adj_.seg, adj_.n_global);
      // recompute the forward states q^a0 .. q^b0 from the checkpoint
      RIDG_CUDA(cudaMemcpyAsync(w_[0].q.p, static_cast<char*>(ck_q_.p) + size_t(j) * qb, qb, cudaMemcpyDeviceToDevice,
                                st_));
      RIDG_CUDA(cudaMemcpyAsync(w_[0].ring.p, static_cast<char*>(ck_ring_.p) + size_t(j) * 3 * qb, 3 * qb,
                                cudaMemcpyDeviceToDevice, st_));
      RIDG_CUDA(cudaMemcpyAsync(w_[0].trace.p, static_cast<char*>(ck_trace_.p) + size_t(j) * tb, tb,
                                cudaMemcpyDeviceToDevice, st_));
      tau_ = adj_.ck_tau[j];
      ring_count_[0] = int(adj_.ck_count[size_t(j)]);
      RIDG_CUDA(cudaMemcpyAsync(sg(0), w_[0].q.p, qb, cudaMemcpyDeviceToDevice, st_));
      for (int64_t n = a0; n < b0; ++n) {
        misfit_step(adj_.wav);
        RIDG_CUDA(cudaMemcpyAsync(sg(n + 1 - a0), w_[0].q.p, qb, cudaMemcpyDeviceToDevice, st_));
      }
      // adjoint steps m = b0 .. a0 + 1: lambda^m = lambda^{m+1} + h sum_s a_s A^T lambda^{m+1+s} - g^m
      for (int64_t m = b0; m > a0; --m) {
        // A^T lambda^{m+1} into the ring and the update of lambda with it, in one pass
        adjoint_rhs_into(L, sr(m + 1), dptr<real>(adjt), sr(m + 2), sr(m + 3), h);
        double F = 0.0;  // source part of q^m - q^{m-1}
        for (int s = 0; s < 3; ++s)
          if (m - 1 - s >= 0) F += h * a[s] * adj_.amp[m - 1 - s];
        cudaError_t e = dispatch_order(N_, [&](auto NC) {
          using LN = Launch<decltype(NC)::value, real>;
          cudaError_t e2 = LN::adj_inject(L, dptr<const int>(adj_grp_), dptr<const int>(adj_rec_sorted_), int(adj_.n_groups),
                                dptr<const int64_t>(adj_rec_slot_), dptr<const real>(adj_rec_row_),
                                dptr<const double>(adj_res_), n_t, m, h, st_);
          if (e2 == cudaSuccess)
            e2 = LN::adj_grad(L, sg(m - a0), sg(m - 1 - a0), n_slots_, adj_.src_slot, dptr<const real>(adj_w_), F,
                              dptr<double>(acc), st_);
          return e2;
        });
        if (e != cudaSuccess) throw Error{RIDG_E_CUDA, cudaGetErrorString(e)};
      }
    }
    std::vector<double> per_slot(static_cast<size_t>(n_slots_));
    RIDG_CUDA(cudaMemcpyAsync(per_slot.data(), acc.p, acc.bytes, cudaMemcpyDeviceToHost, st_));
    RIDG_CUDA(cudaStreamSynchronize(st_));
    for (int64_t k = 0; k < mesh_.K; ++k) grad[k] = -2.0 / c_[k] * per_slot[ord_.slot_of[k]];
    for (int64_t k = 0; k < mesh_.K; ++k)
      if (!std::isfinite(grad[k])) throw Error{RIDG_E_UNSTABLE, "non-finite gradient"};
  }

  // The gradient on several rate levels: reverse accumulation over the fine steps of the library's
  // multi-rate scheme (adjoint_mr_kernels.cuh), segment by segment from the checkpoints.  Each
  // segment is recomputed first, keeping every fine step's new right-hand sides; then its fine
  // steps are reversed, the receiver residuals entering at the global steps.
  void misfit_backward_levels(double* grad) {
    const size_t qn = qsize(), qb = qn * sizeof(real), tsz = trace_slot_elems();
    const size_t tb = 3 * tsz * sizeof(real);
    const int64_t n_t = adj_.n_global + 1;
    const double dtl = lv_.dt_local, dtg = dtl * double(NL_);
    const int64_t fseg = adj_.seg * NL_;  // fine steps per segment
    DBuf mu, mring, min, own, rsav, acc;
    mu.alloc(qb);
    mring.alloc(3 * qb);
    min.alloc(3 * tsz * sizeof(real));
    own.alloc(tsz * sizeof(real));
    rsav.alloc(size_t(fseg) * qb);
    acc.alloc(size_t(n_slots_) * sizeof(double));
    for (DBuf* b : {&mu, &mring, &min, &own, &rsav, &acc}) RIDG_CUDA(cudaMemsetAsync(b->p, 0, b->bytes, st_));
    AdjMrArgs<real> a{};
    a.mu = dptr<real>(mu);
    a.mu_ring = dptr<real>(mring);
    a.mu_in = dptr<real>(min);
    a.own = dptr<real>(own);
    a.n_slots = n_slots_;
    a.n_levels = L_;
    for (int l = 0; l <= L_; ++l) a.level_begin[l] = ord_.level_begin[l];
    a.geo = dptr<const double>(geo_d_);
    a.mat = dptr<const real>(mat_d_);
    a.meta = dptr<const int>(meta_d_);
    a.Dt4 = dptr<const real>(Dt4_d_);
    a.Lt = dptr<const real>(Lt_d_);
    a.NPa = NPa_;
    a.fmask = dptr<const int>(fmask_d_);
    a.inv_fmask = dptr<const int>(inv_fmask_d_);
    a.nbr = dptr<const int>(nbr_d_);
    a.finfo = dptr<const uint8_t>(finfo_d_);
    a.perm = dptr<const int>(perm_d_);
    a.src_slot = adj_.src_slot;
    a.w_src = dptr<const real>(adj_w_);
    a.acc = dptr<double>(acc);
    std::vector<int> cnt(size_t(fseg) * L_);  // each level's ring count before each fine step
    for (int64_t j = adj_.n_ck - 1; j >= 0; --j) {
      const int64_t g0 = j * adj_.seg, g1 = std::min(g0 + adj_.seg, adj_.n_global);
      const int64_t t0 = g0 * NL_, t1 = g1 * NL_;
      RIDG_CUDA(cudaMemcpyAsync(w_[0].q.p, static_cast<char*>(ck_q_.p) + size_t(j) * qb, qb, cudaMemcpyDeviceToDevice,
                                st_));
      RIDG_CUDA(cudaMemcpyAsync(w_[0].ring.p, static_cast<char*>(ck_ring_.p) + size_t(j) * 3 * qb, 3 * qb,
                                cudaMemcpyDeviceToDevice, st_));
      RIDG_CUDA(cudaMemcpyAsync(w_[0].trace.p, static_cast<char*>(ck_trace_.p) + size_t(j) * tb, tb,
                                cudaMemcpyDeviceToDevice, st_));
      tau_ = adj_.ck_tau[j];
      for (int l = 0; l < L_; ++l) ring_count_[l] = int(adj_.ck_count[size_t(j) * L_ + l]);
      for (int64_t t = t0; t < t1; ++t) {
        const int l0 = first_active_level(t);
        for (int l = 0; l < L_; ++l) cnt[size_t(t - t0) * L_ + l] = ring_count_[l];
        misfit_step(adj_.wav);
        for (int l = l0; l <= L_; ++l) {  // the new right-hand sides of the active levels
          const int64_t b0 = ord_.level_begin[l - 1] / 32, b1 = ord_.level_begin[l] / 32;
          if (b1 <= b0) continue;
          const size_t off = size_t(b0) * 4 * Np_ * 32, len = size_t(b1 - b0) * 4 * Np_ * 32;
          const int rn = cnt[size_t(t - t0) * L_ + (l - 1)] % 3;
          RIDG_CUDA(cudaMemcpyAsync(dptr<real>(rsav) + size_t(t - t0) * qn + off, dptr<real>(w_[0].ring) + rn * qn + off,
                                    len * sizeof(real), cudaMemcpyDeviceToDevice, st_));
        }
      }
      for (int64_t t = t1 - 1; t >= t0; --t) {
        cudaError_t e = dispatch_order(N_, [&](auto NC) {
          using LN = Launch<decltype(NC)::value, real>;
          cudaError_t e2 = cudaSuccess;
          if ((t + 1) % NL_ == 0)  // mu_q += Dt (y - d) l(x_r) at the global step t + 1
            e2 = LN::adj_inject(dptr<real>(mu), dptr<const int>(adj_grp_), dptr<const int>(adj_rec_sorted_),
                                int(adj_.n_groups), dptr<const int64_t>(adj_rec_slot_), dptr<const real>(adj_rec_row_),
                                dptr<const double>(adj_res_), n_t, (t + 1) / NL_, -dtg, st_);
          if (e2 != cudaSuccess) return e2;
          a.slot_lo = ord_.level_begin[first_active_level(t) - 1];
          a.slot_read = mod3(t);
          for (int l = 1; l <= L_; ++l) {
            const int64_t d = int64_t(1) << (L_ - l);
            const int c = cnt[size_t(t - t0) * L_ + (l - 1)];
            a.ring_new[l - 1] = c % 3;
            a.ring_old1[l - 1] = (c + 2) % 3;
            a.ring_old2[l - 1] = (c + 1) % 3;
            a.h[l - 1] = real(double(d) * dtl);
            a.slot_full[l - 1] = mod3(t + d);
            a.slot_half[l - 1] = d >= 2 ? mod3(t + d / 2) : mod3(t + 2);
          }
          a.rsaved = dptr<const real>(rsav) + size_t(t - t0) * qn;
          a.F = real(adj_.amp[t]);
          return LN::adjml_step(a, st_);
        });
        if (e != cudaSuccess) throw Error{RIDG_E_CUDA, cudaGetErrorString(e)};
      }
    }
    std::vector<double> per_slot(static_cast<size_t>(n_slots_));
    RIDG_CUDA(cudaMemcpyAsync(per_slot.data(), acc.p, acc.bytes, cudaMemcpyDeviceToHost, st_));
    RIDG_CUDA(cudaStreamSynchronize(st_));
    for (int64_t k = 0; k < mesh_.K; ++k) grad[k] = 2.0 / c_[k] * per_slot[ord_.slot_of[k]];
    for (int64_t k = 0; k < mesh_.K; ++k)
      if (!std::isfinite(grad[k])) throw Error{RIDG_E_UNSTABLE, "non-finite gradient"};
  }

  size_t shot_extra_device_bytes(double t_final) const override {
    if (!(t_final > 0.0)) return 0;
    const double dtg = lv_.dt_local * double(NL_);
    const int64_t tau_f = int64_t(std::ceil(t_final / dtg - 1e-9)) * NL_;
    int64_t recs = 0;
    for (int64_t t = 0; t <= tau_f; ++t) recs += n_bfaces_ - bface_first(slot_lo(t));
    size_t arena = std::max<size_t>(size_t(recs) * 2 * NFPP_ * sizeof(real), 16);
    if (trace_budget_ > 0 && arena > trace_budget_) arena = trace_budget_;  // at most the budget (TraceTier)
    size_t extra = arena > arena_.bytes ? arena - arena_.bytes : 0;
    if (!q_snap_.p) extra += 4 * qsize() * sizeof(real) + 2 * size_t(n_slots_) * Np_ * sizeof(double);
    if (!w_[1].q.p) extra += 4 * qsize() * sizeof(real) + 3 * trace_slot_elems() * sizeof(real);
    return extra;
  }
  size_t shots_extra_device_bytes(double t_final, int32_t n) const override {
    size_t extra = shot_extra_device_bytes(t_final);
    if (n <= 1 || !(t_final > 0.0)) return extra;
    // shots 1.. of the batch: their own arena, snapshots, images and two wavefields
    const double dtg = lv_.dt_local * double(NL_);
    const int64_t tau_f = int64_t(std::ceil(t_final / dtg - 1e-9)) * NL_;
    int64_t recs = 0;
    for (int64_t t = 0; t <= tau_f; ++t) recs += n_bfaces_ - bface_first(slot_lo(t));
    const size_t arena = std::max<size_t>(size_t(recs) * 2 * NFPP_ * sizeof(real), 16);
    const size_t wave = 4 * qsize() * sizeof(real) + 3 * trace_slot_elems() * sizeof(real);
    const size_t per = arena + 4 * qsize() * sizeof(real) + 2 * size_t(n_slots_) * Np_ * sizeof(double) + 2 * wave;
    for (int32_t b = 1; b < n; ++b) {
      const ShotState* x = size_t(b - 1) < extra_shots_.size() ? extra_shots_[size_t(b - 1)].get() : nullptr;
      size_t have = 0;
      if (x) {
        have = x->arena.bytes + x->q_snap.bytes + x->ring_snap.bytes + x->img_p.bytes + x->img_q.bytes;
        for (const Wave<real>& w : x->w) have += w.q.bytes + w.ring.bytes + w.trace.bytes;
      }
      extra += per > have ? per - have : 0;
    }
    return extra;
  }
  size_t release_shot_buffers() override {
    RIDG_CUDA(cudaStreamSynchronize(st_));
    size_t bytes = 0;
    for (DBuf* d : {&arena_, &q_snap_, &ring_snap_, &img_p_, &img_q_, &traces_tmp_, &w_[1].q, &w_[1].ring, &w_[1].trace,
                    &w_[1].inj_range, &w_[1].inj_w, &w_[1].inj_row}) {
      bytes += d->bytes;
      d->release();
    }
    for (auto& x : extra_shots_) {
      for (DBuf* d : {&x->rec_slot, &x->rec_row, &x->traces_tmp, &x->arena, &x->q_snap, &x->ring_snap, &x->img_p,
                      &x->img_q, &x->scale})
        bytes += d->bytes;
      for (Wave<real>& w : x->w)
        for (DBuf* d : {&w.q, &w.ring, &w.trace, &w.inj_range, &w.inj_w, &w.inj_row}) bytes += d->bytes;
    }
    extra_shots_.clear();
    return bytes;
  }
  int64_t trace_len(double t_final) const override {
    double dtg = lv_.dt_local * double(NL_);
    return int64_t(std::ceil(t_final / dtg - 1e-9)) + 1;
  }

  // ------------------------------------------------------------------ RTM shots
  void shot(const ridg_source& src, const double* rec, int64_t nrec, double t_final, double t_i, const double* obs_dev,
            double* traces_dev, double* imgp_dev, double* imgq_dev, const double* e_up) override {
    ridg_shot_io io{};
    io.source = src;
    io.rec_xyz = rec;
    io.nrec = nrec;
    io.observed = obs_dev;
    io.traces_out = traces_dev;
    io.image_p = imgp_dev;
    io.image_q = imgq_dev;
    shots(1, &io, t_final, t_i, e_up);
  }

  // n shots of this solver's model in lockstep (one record length and image window): every fine step
  // is one merged launch over the active slots of all of them (FP32 tensor-core contractions; the
  // other kernels step the shots one after the other).  Shot 0 keeps its device state in the
  // solver's own buffers, shots 1.. in extra_shots_.
  void shots(int32_t n, const ridg_shot_io* io, double t_final, double t_i, const double* e_up) override {
    NvtxRange nv_shot(n == 1 ? "ridg shot" : "ridg merged shots");
    if (n < 1 || n > kMaxBatch || !io)
      throw Error{RIDG_E_INVALID_ARG, "a batch holds 1 to " + std::to_string(kMaxBatch) + " shots"};
    if (n > 1 && hook_) throw Error{RIDG_E_INVALID_ARG, "the parts of a group run one shot at a time"};
    if (n > 1 && trace_budget_ > 0)
      throw Error{RIDG_E_INVALID_ARG, "a batch of shots keeps its boundary records on the device (no trace budget)"};
    if (!(t_final > 0.0) || !(t_i >= 0.0) || t_i > t_final + lv_.dt_local * double(NL_))
      throw Error{RIDG_E_INVALID_ARG, "bad time span"};
    for (int b = 0; b < n; ++b)
      if (io[b].nrec < 0 || (io[b].nrec > 0 && !io[b].rec_xyz))
        throw Error{RIDG_E_INVALID_ARG, "bad receiver list of shot " + std::to_string(b)};
    while (int(extra_shots_.size()) < n - 1) extra_shots_.push_back(std::make_unique<ShotState>());
    std::memset(&stats_, 0, sizeof(stats_));
    prof_used_ = 0;
    const double dtl = lv_.dt_local, dtg = dtl * double(NL_);
    const int64_t n_global = int64_t(std::ceil(t_final / dtg - 1e-9));
    const int64_t n_t = n_global + 1;
    int64_t n_i = int64_t(std::floor(t_i / dtg + 1e-9));
    n_i = std::min(n_i, n_global);
    const int64_t tau_f = n_global * NL_, tau_i = n_i * NL_;
    stats_.n_global = n_global;
    std::vector<ShotRef> S(n);
    for (int b = 0; b < n; ++b) S[b] = shot_ref(b);
    // ---- sources and receivers of every shot
    std::vector<Wavelet> wav(n);
    for (int b = 0; b < n; ++b) {
      const ridg_source& src = io[b].source;
      const int64_t nrec = io[b].nrec;
      const double* rec = io[b].rec_xyz;
      double rst[3];
      int64_t ks = locate_point(mesh_, loc_, src.xyz, rst);
      if (ks < 0) throw Error{RIDG_E_NOT_FOUND, "source lies outside the mesh"};
      std::vector<real> w_src = projected_dirac(ks, rst);
      wav[b] = Wavelet::of(src);
      const bool src_here = owned(ks);
      struct Rec {
        int64_t slot;
        std::vector<real> row, w;
        int idx;
      };
      std::vector<Rec> recs(nrec);
      for (int64_t r = 0; r < nrec; ++r) {
        int64_t kr = locate_point(mesh_, loc_, rec + 3 * r, rst);
        if (kr < 0) throw Error{RIDG_E_NOT_FOUND, "receiver " + std::to_string(r) + " lies outside the mesh"};
        recs[r].slot = owned(kr) ? ord_.slot_of[kr] : -1;  // -1: another part samples and injects it
        std::array<double, 3> p = {rst[0], rst[1], rst[2]};
        std::vector<double> l = ref_.lagrange_at(p);
        recs[r].row.assign(l.begin(), l.end());
        recs[r].w = projected_dirac(kr, rst);
        recs[r].idx = int(r);
      }
      Wave<real>* w = S[b].w;
      alloc_wave(w[0]);
      // source injection table (wavefield 0)
      {
        std::vector<int2> range(n_slots_, make_int2(0, 0));
        if (src_here) range[ord_.slot_of[ks]] = make_int2(0, 1);
        upload(w[0].inj_range, range, st_);
        upload(w[0].inj_w, w_src, st_);
        upload(w[0].inj_row, std::vector<int>{0}, st_);
      }
      alloc_wave(w[1]);
      {
        // receiver injections grouped by slot (wavefield 1)
        std::vector<Rec> sorted;
        for (const Rec& r : recs)
          if (r.slot >= 0) sorted.push_back(r);
        std::stable_sort(sorted.begin(), sorted.end(), [](const Rec& a, const Rec& c) { return a.slot < c.slot; });
        std::vector<int2> range(n_slots_, make_int2(0, 0));
        std::vector<real> wv;
        std::vector<int> rows;
        for (size_t i = 0; i < sorted.size(); ++i) {
          int2& rg = range[sorted[i].slot];
          if (rg.y == 0) rg.x = int(i);
          rg.y += 1;
          wv.insert(wv.end(), sorted[i].w.begin(), sorted[i].w.end());
          rows.push_back(sorted[i].idx);
        }
        if (rows.empty()) {
          rows.push_back(0);
          wv.assign(Np_, real(0));
        }
        upload(w[1].inj_range, range, st_);
        upload(w[1].inj_w, wv, st_);
        upload(w[1].inj_row, rows, st_);
        std::vector<int64_t> rslot(std::max<int64_t>(nrec, 1), 0);
        std::vector<real> rrow(std::max<int64_t>(nrec, 1) * Np_, real(0));
        for (int64_t r = 0; r < nrec; ++r) {
          rslot[r] = recs[r].slot;
          for (int m = 0; m < Np_; ++m) rrow[r * Np_ + m] = recs[r].row[m];
        }
        upload(*S[b].rec_slot, rslot, st_);
        upload(*S[b].rec_row, rrow, st_);
      }
    }
    std::vector<double*> traces(n);
    for (int b = 0; b < n; ++b) {
      traces[b] = io[b].traces_out;
      if (!traces[b]) {
        S[b].traces_tmp->alloc(size_t(std::max<int64_t>(io[b].nrec, 1)) * n_t * sizeof(double));
        traces[b] = dptr<double>(*S[b].traces_tmp);
      }
    }
    // ---- boundary-trace arenas: one record per boundary face of every active element per step
    std::vector<int64_t> arena_base(tau_f + 2, 0);
    for (int64_t t = 0; t <= tau_f; ++t) arena_base[t + 1] = arena_base[t] + (n_bfaces_ - bface_first(slot_lo(t)));
    const size_t rec_bytes = 2 * NFPP_ * sizeof(real);
    size_t arena_bytes = size_t(arena_base[tau_f + 1]) * rec_bytes;
    if (fault_fires(kFaultArena))
      throw Error{RIDG_E_OOM, "boundary-trace arena of " + std::to_string(arena_bytes) + " bytes (injected failure)"};
    // beyond the device budget the records go to pinned host memory in chunks (TraceTier; one shot)
    const bool tiered = tier_.plan(arena_base, rec_bytes, trace_budget_);
    for (int b = 0; b < n; ++b) S[b].arena->reserve(std::max<size_t>(tiered ? tier_.device_bytes() : arena_bytes, 16));
    if (tiered && tier_.n_chunks() > 2) host_arena_.reserve(arena_bytes);
    stats_.boundary_trace_bytes = int64_t(arena_bytes) * n;
    stats_.trace_chunks = tiered ? tier_.n_chunks() : 1;
    // device address and record offset of step t's records (the first record of its chunk at the start)
    auto arena_at = [&](int b, int64_t t, int sigma, int64_t slot_lo) {
      char* base = static_cast<char*>(S[b].arena->p);
      int64_t first = 0;
      if (tiered) {
        const int k = tier_.chunk_of(t);
        char* host = static_cast<char*>(host_arena_.p);
        base = sigma > 0 ? tier_.forward_chunk(k, base, host, st_) : tier_.backward_chunk(k, base, host, st_);
        first = tier_.first_record(k);
      }
      return std::make_pair(reinterpret_cast<real*>(base), arena_base[t] - first - bface_first(slot_lo));
    };
    for (int b = 0; b < n; ++b) {
      S[b].q_snap->alloc(qsize() * sizeof(real));
      S[b].ring_snap->alloc(3 * qsize() * sizeof(real));
      S[b].img_p->alloc(size_t(n_slots_) * Np_ * sizeof(double));
      S[b].img_q->alloc(size_t(n_slots_) * Np_ * sizeof(double));
    }
    for (int b = 0; b < n; ++b)
      if (io[b].nrec > 0) S[b].scale->reserve(kDataScaleWorkBytes);
    BatchArgs<real> batch{};
    const bool merged = n > 1;
    double eu[3] = {0.0, 0.0, -1.0};
    if (e_up) std::memcpy(eu, e_up, sizeof(eu));

    // the time stepping: only work enqueued on the solver's stream (capturable as a CUDA graph)
    auto steps = [&] {
      // ---- forward source runs
      for (int b = 0; b < n; ++b) zero_wave(S[b].w[0]);
      reset_time();
      for (int b = 0; b < n; ++b) {
        RIDG_CUDA(cudaMemsetAsync(traces[b], 0, size_t(std::max<int64_t>(io[b].nrec, 1)) * n_t * sizeof(double), st_));
        sample(S[b], traces[b], n_t, 0, io[b].nrec);
      }
      auto forward_step = [&](int mode) {
        StepArgs<real> a = fine_args(+1, 1, mode);
        const int64_t t_rec = std::min<int64_t>(tau_, tau_f);
        for (int b = 0; b < n; ++b) {
          ShotArgs<real>& sa = batch.shot[b];
          sa = ShotArgs<real>{};
          sa.wave[0] = wave_args(S[b].w[0]);
          sa.wave[0].amp_mode = 1;
          sa.wave[0].amp = real(wav[b](double(tau_) * dtl));
          std::tie(sa.arena_write, a.arena_offset) = arena_at(b, t_rec, +1, a.slot_lo);
        }
        a.wave[0] = batch.shot[0].wave[0];
        a.arena_write = batch.shot[0].arena_write;
        launch_fine(a, +1, 1, merged ? &batch : nullptr, n);
      };
      if (tiered) tier_.begin_forward(st_);
      {
        NvtxRange nv("forward source run");
        for (int64_t g = 0; g < n_global; ++g) {
          for (int64_t s = 0; s < NL_; ++s) forward_step(kModeRecord);
          for (int b = 0; b < n; ++b) sample(S[b], traces[b], n_t, g + 1, io[b].nrec);
        }
      }
      stats_.dof_updates_forward = dof_;
      for (int b = 0; b < n; ++b)
        RIDG_CUDA(cudaMemcpyAsync(S[b].q_snap->p, S[b].w[0].q.p, qsize() * sizeof(real), cudaMemcpyDeviceToDevice,
                                  st_));
      // two more global steps (and the first right-hand side of a third) give, per level l, the
      // right-hand sides at t_f + Delta t_l and t_f + 2 Delta t_l that start the backward run
      for (int64_t i = 0; i <= 2 * NL_; ++i) {
        int64_t t_now = tau_;
        std::vector<int> before = ring_count_;
        forward_step(t_now == tau_f ? kModeRecord : 0);
        for (int l = 1; l <= L_; ++l) {
          int64_t d = int64_t(1) << (L_ - l);
          if (t_now == tau_f + 2 * d)
            for (int b = 0; b < n; ++b) snapshot_history(S[b], l, before[l - 1]);
        }
      }
      // ---- backward: source (replayed boundary) and receiver wavefields in lockstep
      for (int b = 0; b < n; ++b) {
        RIDG_CUDA(cudaMemcpyAsync(S[b].w[0].q.p, S[b].q_snap->p, qsize() * sizeof(real), cudaMemcpyDeviceToDevice,
                                  st_));
        RIDG_CUDA(cudaMemcpyAsync(S[b].w[0].ring.p, S[b].ring_snap->p, 3 * qsize() * sizeof(real),
                                  cudaMemcpyDeviceToDevice, st_));
        zero_wave(S[b].w[1]);
        RIDG_CUDA(cudaMemsetAsync(S[b].img_p->p, 0, S[b].img_p->bytes, st_));
        RIDG_CUDA(cudaMemsetAsync(S[b].img_q->p, 0, S[b].img_q->bytes, st_));
      }
      std::fill(ring_count_.begin(), ring_count_.end(), 0);
      tau_ = tau_f;
      for (int b = 0; b < n; ++b) {
        RIDG_CUDA(cudaMemsetAsync(S[b].w[0].trace.p, 0, S[b].w[0].trace.bytes, st_));
        init_traces(S[b].w[0], mod3(tau_));
      }
      if (hook_) hook_->exchange(*this, 1, 1);
      // the receiver run injects the data times a power of two that brings max |data| into [1, 2), so
      // that the image products of small-amplitude shots stay inside the FP32 range; the images are
      // divided by it on the way out (both steps exact)
      std::vector<const double*> data(n), dscale(n, nullptr), dscale_inv(n, nullptr);
      for (int b = 0; b < n; ++b) {
        data[b] = io[b].observed ? io[b].observed : traces[b];
        const int64_t nrec = io[b].nrec;
        if (nrec > 0) {
          cudaError_t e = data_scale(data[b], nrec * n_t, S[b].scale->p, st_);
          if (e != cudaSuccess) throw Error{RIDG_E_CUDA, std::string("data scale: ") + cudaGetErrorString(e)};
          if (hook_) hook_->combine_data_scale(*this, S[b].scale->p);
          stats_.kernel_launches += 2;
          dscale[b] = dptr<const double>(*S[b].scale) + 1;
          dscale_inv[b] = dptr<const double>(*S[b].scale) + 2;
        }
      }
      int64_t dof_before = dof_;
      if (tiered) tier_.begin_backward(tau_i + 1);
      NvtxRange nv_back("backward source and receiver runs");
      while (tau_ > tau_i) {
        StepArgs<real> a = fine_args(-1, 2, kModeReplay | image_mode_);
        int64_t n_lo = tau_ / NL_;
        double u = double(tau_ - n_lo * NL_) / double(NL_);
        a.interp_n0 = int(n_lo - 1);
        const double xs[4] = {-1.0, 0.0, 1.0, 2.0};
        for (int i = 0; i < 4; ++i) {
          double li = 1.0;
          for (int j = 0; j < 4; ++j)
            if (j != i) li *= (u - xs[j]) / (xs[i] - xs[j]);
          a.interp_w[i] = li;
        }
        for (int d = 0; d < 3; ++d) a.e_up[d] = real(eu[d]);
        for (int b = 0; b < n; ++b) {
          ShotArgs<real>& sa = batch.shot[b];
          sa = ShotArgs<real>{};
          sa.wave[0] = wave_args(S[b].w[0]);
          sa.wave[0].amp_mode = 1;
          sa.wave[0].amp = real(wav[b](double(tau_) * dtl));
          sa.wave[1] = wave_args(S[b].w[1]);
          sa.wave[1].amp_mode = io[b].nrec > 0 ? 2 : 0;
          sa.wave[1].data = data[b];
          sa.wave[1].data_scale = dscale[b];
          sa.wave[1].n_time = int(n_t);
          std::tie(sa.arena_read, a.arena_offset) = arena_at(b, tau_, -1, a.slot_lo);
          sa.image_p = dptr<double>(*S[b].img_p);
          sa.image_q = dptr<double>(*S[b].img_q);
        }
        a.wave[0] = batch.shot[0].wave[0];
        a.wave[1] = batch.shot[0].wave[1];
        a.arena_read = batch.shot[0].arena_read;
        a.image_p = batch.shot[0].image_p;
        a.image_q = batch.shot[0].image_q;
        launch_fine(a, -1, 2, merged ? &batch : nullptr, n);
      }
      stats_.dof_updates_backward = dof_ - dof_before;
      if (tiered) {
        tier_.after_copies(st_);
        stats_.host_trace_bytes = tier_.host_bytes();
      } else {
        stats_.host_trace_bytes = 0;
      }
      for (int b = 0; b < n; ++b) {
        if (io[b].image_p) image_out(dptr<double>(*S[b].img_p), dscale_inv[b], io[b].image_p);
        if (io[b].image_q) image_out(dptr<double>(*S[b].img_q), dscale_inv[b], io[b].image_q);
      }
    };
    // (the legacy default stream cannot be captured)
    if (!graph_on_ || tiered || hook_ || prof_every_ > 0 || st_ == nullptr || st_ == cudaStreamLegacy) {
      steps();
    } else {
      run_graphed(steps, graph_key(n, io, t_final, t_i, eu, S, traces));
    }
    RIDG_CUDA(cudaGetLastError());
  }

 private:
  // ------------------------------------------------------------------ helpers
  // the device buffers of shot b of a batch
  struct ShotRef {
    Wave<real>* w;
    DBuf *rec_slot, *rec_row, *traces_tmp, *arena, *q_snap, *ring_snap, *img_p, *img_q, *scale;
  };
  ShotRef shot_ref(int b) {
    if (b == 0)
      return ShotRef{w_, &rec_slot_, &rec_row_, &traces_tmp_, &arena_, &q_snap_, &ring_snap_, &img_p_, &img_q_,
                     &scale_d_};
    ShotState& x = *extra_shots_[size_t(b - 1)];
    return ShotRef{x.w,      &x.rec_slot,  &x.rec_row, &x.traces_tmp, &x.arena,
                   &x.q_snap, &x.ring_snap, &x.img_p,   &x.img_q,      &x.scale};
  }
  // ---- CUDA-graph replay of a batch's time stepping
  // Every argument the time stepping bakes into its launches: the batch's time span, e_up and image
  // mode, per shot the wavelet (its values at every step are kernel arguments), the receiver count
  // and the device address of every buffer it touches.  Source and receiver positions and the data
  // values are read from device memory, uploaded before the stepping, so they may differ.
  std::vector<uint64_t> graph_key(int32_t n, const ridg_shot_io* io, double t_final, double t_i, const double* eu,
                                  const std::vector<ShotRef>& S, const std::vector<double*>& traces) const {
    std::vector<uint64_t> k;
    auto bits = [](double x) {
      uint64_t u;
      std::memcpy(&u, &x, sizeof(u));
      return u;
    };
    auto ptr = [](const void* p) { return uint64_t(reinterpret_cast<uintptr_t>(p)); };
    k.push_back(uint64_t(n));
    k.push_back(bits(t_final));
    k.push_back(bits(t_i));
    for (int d = 0; d < 3; ++d) k.push_back(bits(eu[d]));
    k.push_back(uint64_t(image_mode_));
    k.push_back(uint64_t(contraction_));
    const DBuf* tables[] = {&geo_d_, &mat_d_, &nbr_d_, &finfo_d_, &bface_d_, &meta_d_, &Dt_d_, &Lt_d_, &fmask_d_,
                            &perm_d_, &afrag_d_, &gtab_d_[0], &gtab_d_[1], &slot_of_d_, &pos_d_};
    for (const DBuf* d : tables) k.push_back(ptr(d->p));
    for (int b = 0; b < n; ++b) {
      const ridg_source& src = io[b].source;
      k.push_back(uint64_t(src.kind));
      for (double x : {src.f0, src.t_peak, src.amplitude, src.sample_dt}) k.push_back(bits(x));
      k.push_back(uint64_t(src.n_samples));
      uint64_t h = 1469598103934665603ull;  // FNV-1a over the samples
      if (src.kind == RIDG_SRC_SAMPLED && src.samples)
        for (int64_t i = 0; i < src.n_samples; ++i) {
          const uint64_t u = bits(src.samples[i]);
          for (int byte = 0; byte < 8; ++byte) h = (h ^ ((u >> (8 * byte)) & 0xffu)) * 1099511628211ull;
        }
      k.push_back(h);
      k.push_back(uint64_t(io[b].nrec));
      for (const void* p : {static_cast<const void*>(io[b].observed), static_cast<const void*>(traces[b]),
                            static_cast<const void*>(io[b].image_p), static_cast<const void*>(io[b].image_q)})
        k.push_back(ptr(p));
      for (int w = 0; w < 2; ++w) {
        const Wave<real>& wv = S[b].w[w];
        const DBuf* wbufs[] = {&wv.q, &wv.ring, &wv.trace, &wv.inj_range, &wv.inj_w, &wv.inj_row};
        for (const DBuf* d : wbufs) k.push_back(ptr(d->p));
      }
      const DBuf* sbufs[] = {S[b].rec_slot, S[b].rec_row, S[b].arena, S[b].q_snap,
                             S[b].ring_snap, S[b].img_p, S[b].img_q, S[b].scale};
      for (const DBuf* d : sbufs) k.push_back(ptr(d->p));
    }
    return k;
  }

  // The first run of a key runs directly; the second captures its stream work into a graph, which
  // later runs of the same key launch instead of the individual kernels (with the host-side counters
  // and time state of the captured run restored).
  template <typename F>
  void run_graphed(F&& steps, std::vector<uint64_t> key) {
    if (graph_exec_ && key == graph_exec_key_) {
      RIDG_CUDA(cudaGraphLaunch(graph_exec_, st_));
      stats_ = graph_stats_;
      tau_ = graph_tau_;
      dof_ = graph_dof_;
      ring_count_ = graph_ring_;
      stats_.graph_replay = 1;
      return;
    }
    if (!(graph_seen_ && key == graph_key_)) {
      steps();
      graph_key_ = std::move(key);
      graph_seen_ = true;
      return;
    }
    drop_graph();
    RIDG_CUDA(cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal));
    cudaGraph_t g = nullptr;
    try {
      steps();
    } catch (...) {
      cudaStreamEndCapture(st_, &g);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      throw;
    }
    RIDG_CUDA(cudaStreamEndCapture(st_, &g));
    cudaGraphExec_t ex = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) throw Error{RIDG_E_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(e)};
    graph_exec_ = ex;
    graph_exec_key_ = std::move(key);
    graph_stats_ = stats_;
    graph_tau_ = tau_;
    graph_dof_ = dof_;
    graph_ring_ = ring_count_;
    RIDG_CUDA(cudaGraphLaunch(graph_exec_, st_));
    stats_.graph_replay = 1;
  }
  void drop_graph() {
    if (graph_exec_) cudaGraphExecDestroy(graph_exec_);
    graph_exec_ = nullptr;
    graph_exec_key_.clear();
    graph_key_.clear();
    graph_seen_ = false;
  }

  size_t qsize() const { return size_t(n_slots_) * 4 * Np_; }
  size_t trace_slot_elems() const { return size_t(n_slots_) * 8 * NFPP_; }
  size_t device_bytes() const {
    size_t b = 0;
    const DBuf* all[] = {&geo_d_, &J_d_, &mat_d_, &nbr_d_, &finfo_d_, &bface_d_, &meta_d_, &Dt_d_, &Dt4_d_, &Lt_d_,
                         &fmask_d_, &perm_d_, &M_d_, &slot_of_d_, &q_snap_, &ring_snap_, &img_p_, &img_q_, &arena_,
                         &afrag_d_, &gtab_d_[0], &gtab_d_[1]};
    for (auto* x : all) b += x->bytes;
    for (auto& w : w_) b += w.q.bytes + w.ring.bytes + w.trace.bytes;
    for (const auto& x : extra_shots_) {
      b += x->arena.bytes + x->q_snap.bytes + x->ring_snap.bytes + x->img_p.bytes + x->img_q.bytes;
      for (const Wave<real>& w : x->w) b += w.q.bytes + w.ring.bytes + w.trace.bytes;
    }
    return b;
  }
  int64_t bface_first(int64_t slot) const { return slot >= n_slots_ ? n_bfaces_ : bface_host_[slot]; }
  int first_active_level(int64_t tau) const {
    // level l (1..L) is active iff tau is a multiple of 2^(L-l); the active set is a suffix
    for (int l = 1; l <= L_; ++l)
      if (tau % (int64_t(1) << (L_ - l)) == 0) return l;
    return L_;
  }
  int64_t slot_lo(int64_t tau) const { return ord_.level_begin[first_active_level(tau) - 1]; }

  void reset_time() {
    tau_ = 0;
    ring_count_.assign(L_, 0);
    dof_ = 0;
  }

  std::vector<real> to_slots(const double* q) const {
    std::vector<real> h(qsize(), real(0));
    for (int64_t k = 0; k < mesh_.K; ++k) {
      int64_t s = ord_.slot_of[k];
      if (!owned(k)) continue;
      for (int f = 0; f < 4; ++f)
        for (int n = 0; n < Np_; ++n)
          h[(((s >> 5) * 4 + f) * Np_ + pos_of_[n]) * 32 + (s & 31)] = real(q[(k * 4 + f) * Np_ + n]);
    }
    return h;
  }
  void from_slots(const std::vector<real>& h, double* q) const {
    for (int64_t k = 0; k < mesh_.K; ++k) {
      int64_t s = ord_.slot_of[k];
      for (int f = 0; f < 4; ++f)
        for (int n = 0; n < Np_; ++n)
          q[(k * 4 + f) * Np_ + n] = owned(k) ? double(h[(((s >> 5) * 4 + f) * Np_ + pos_of_[n]) * 32 + (s & 31)]) : 0.0;
    }
  }

  void check_shared_memory() const {
    int dev = 0, optin = 0;
    RIDG_CUDA(cudaGetDevice(&dev));
    RIDG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    size_t need = dispatch_order(N_, [&](auto NC) {
      constexpr int NN = decltype(NC)::value;
      if constexpr (std::is_same<real, float>::value)
        if (contraction_ != RIDG_CONTRACT_CUDA_CORES)
          return std::max(SmemTc<NN, 1, kSplitFp16>::bytes, SmemTc<NN, 2, kSplitFp16>::bytes);
      return std::max(step_smem_bytes<NN, real, 1>(), step_smem_bytes<NN, real, 2>());
    });
    if (need > size_t(optin))
      throw Error{RIDG_E_INVALID_ARG, "order " + std::to_string(N_) + " in this precision needs " +
                                          std::to_string(need) + " bytes of shared memory per block (device allows " +
                                          std::to_string(optin) + ")"};
  }

  void build_nodes() {
    xnodes_.assign(size_t(mesh_.K) * Np_ * 3, 0.0);
    for (int64_t k = 0; k < mesh_.K; ++k)
      for (int n = 0; n < Np_; ++n) {
        const auto& r = ref_.rst[n];
        double lam[4] = {-(1 + r[0] + r[1] + r[2]) / 2, (1 + r[0]) / 2, (1 + r[1]) / 2, (1 + r[2]) / 2};
        for (int v = 0; v < 4; ++v)
          for (int d = 0; d < 3; ++d) xnodes_[(k * Np_ + n) * 3 + d] += lam[v] * mesh_.xyz[3 * mesh_.tet[4 * k + v] + d];
      }
  }

  void check_face_nodes() {
    for (int64_t k = 0; k < mesh_.K; ++k)
      for (int f = 0; f < 4; ++f) {
        int64_t k2 = mesh_.nbr[4 * k + f];
        if (k2 < 0) continue;
        int f2 = mesh_.nbr_face[4 * k + f], code = mesh_.perm_code[4 * k + f];
        double tol = 1e-8 * std::max(geo_.lmin[k], 1e-300);
        for (int j = 0; j < Nfp_; ++j) {
          const double* xa = &xnodes_[(k * Np_ + ref_.fmask[f][j]) * 3];
          const double* xb = &xnodes_[(k2 * Np_ + ref_.fmask[f2][ref_.perm[code][j]]) * 3];
          double d = std::fabs(xa[0] - xb[0]) + std::fabs(xa[1] - xb[1]) + std::fabs(xa[2] - xb[2]);
          if (d > tol) throw Error{RIDG_E_BAD_MESH, "face nodes of neighbouring elements do not coincide"};
        }
        // traces are pushed with the writer's correspondence and read without one: the two sides'
        // correspondences must be mutually inverse
        int code2 = mesh_.perm_code[4 * k2 + f2];
        for (int j = 0; j < Nfp_; ++j)
          if (ref_.perm[code2][ref_.perm[code][j]] != j)
            throw Error{RIDG_E_BAD_MESH, "face-node correspondences of a shared face are not mutually inverse"};
      }
  }

  void build_tables() {
    const int64_t S = n_slots_;
    std::vector<double> geo(S * kGeo, 0.0), J(S, 0.0);
    std::vector<int> nbr(S * 4, -1), bface(S, 0), meta(S, 0);
    std::vector<uint8_t> finfo(S * 4, 0);
    int64_t nb = 0;
    for (int64_t s = 0; s < S; ++s) {
      bface[s] = int(nb);
      int64_t k = ord_.elem_of[s];
      if (k < 0 || s >= ord_.owned_end) continue;  // padding, or a ghost of another part
      meta[s] = kMetaValid;
      for (int i = 0; i < 9; ++i) geo[s * kGeo + i] = geo_.rx[9 * k + i];
      for (int i = 0; i < 12; ++i) geo[s * kGeo + 9 + i] = geo_.normal[12 * k + i];
      for (int f = 0; f < 4; ++f) geo[s * kGeo + 21 + f] = geo_.fscale[4 * k + f];
      J[s] = geo_.J[k];
      for (int f = 0; f < 4; ++f) {
        int64_t k2 = mesh_.nbr[4 * k + f];
        int bc = k2 >= 0 ? 0 : mesh_.bc[4 * k + f];
        int nf = k2 >= 0 ? mesh_.nbr_face[4 * k + f] : 0;
        int pc = k2 >= 0 ? mesh_.perm_code[4 * k + f] : 0;
        finfo[s * 4 + f] = uint8_t(nf | (pc << 2) | (bc << 5));
        nbr[s * 4 + f] = k2 >= 0 ? int(ord_.slot_of[k2]) : -1;
        if (k2 < 0) ++nb;
        if (k2 >= 0 && lv_.level[k2] > lv_.level[k]) meta[s] |= kMetaHalf;
      }
      if (meta[s] & kMetaHalf) ++n_half_;
    }
    n_bfaces_ = nb;
    bface_host_ = bface;
    if (debug_) check_tables(nbr, finfo, bface, meta);
    upload(geo_d_, geo, st_);
    upload(J_d_, J, st_);
    upload_material();
    upload(nbr_d_, nbr, st_);
    upload(finfo_d_, finfo, st_);
    upload(bface_d_, bface, st_);
    upload(meta_d_, meta, st_);
    std::vector<real> Dt(3 * Np_ * NPa_, real(0)), Lt(4 * Nfp_ * NPa_, real(0));
    for (int j = 0; j < 3; ++j)
      for (int m = 0; m < Np_; ++m)
        for (int n = 0; n < Np_; ++n) Dt[(j * Np_ + m) * NPa_ + n] = real(ref_.D[j](n, m));
    for (int fm = 0; fm < 4 * Nfp_; ++fm)
      for (int n = 0; n < Np_; ++n) Lt[fm * NPa_ + n] = real(ref_.LIFT(n, fm));
    std::vector<real> Dt4(size_t(Np_) * Np_ * 4, real(0));  // (D_0, D_1, D_2, 0)[n][m] at (m, n)
    for (int m = 0; m < Np_; ++m)
      for (int n = 0; n < Np_; ++n)
        for (int j = 0; j < 3; ++j) Dt4[(size_t(m) * Np_ + n) * 4 + j] = real(ref_.D[j](n, m));
    upload(Dt_d_, Dt, st_);
    upload(Dt4_d_, Dt4, st_);
    upload(Lt_d_, Lt, st_);
    if (contraction_ != RIDG_CONTRACT_CUDA_CORES)
      upload(afrag_d_, operator_fragments(contraction_), st_);
    std::vector<int> fm(128, 0), pm(192, 0);
    for (int f = 0; f < 4; ++f)
      for (int j = 0; j < Nfp_; ++j) fm[f * 32 + j] = ref_.fmask[f][j];
    for (int c = 0; c < 6; ++c)
      for (int j = 0; j < Nfp_; ++j) pm[c * 32 + j] = ref_.perm[c][j];
    upload(fmask_d_, fm, st_);
    {
      // the face nodes (f * 32 + jf, in (f, jf) order) that are node m, three at most, -1 after them
      std::vector<int> inv(size_t(Np_) * 3, -1);
      for (int m = 0; m < Np_; ++m) {
        int cnt = 0;
        for (int f = 0; f < 4; ++f)
          for (int j = 0; j < Nfp_; ++j)
            if (ref_.fmask[f][j] == m && cnt < 3) inv[m * 3 + cnt++] = f * 32 + j;
      }
      upload(inv_fmask_d_, inv, st_);
    }
    upload(perm_d_, pm, st_);
    upload(M_d_, ref_.M.a, st_);
    upload(pos_d_, pos_of_, st_);
    upload(slot_of_d_, ord_.slot_of, st_);
    level_count_.assign(L_, 0);
    for (int64_t k = 0; k < mesh_.K; ++k)
      if (owned(k)) level_count_[lv_.level[k] - 1]++;
  }

  // RIDG_DEBUG: every index the kernels follow stays in its array and the connectivity is symmetric
  // (a face's neighbour names it back through the recorded face), the slot maps are inverse to each
  // other, the boundary-face numbering counts the boundary faces in slot order, and the face-node
  // tables are permutations of the face's nodes.
  void check_tables(const std::vector<int>& nbr, const std::vector<uint8_t>& finfo, const std::vector<int>& bface,
                    const std::vector<int>& meta) const {
    auto fail = [](const std::string& what) { throw Error{RIDG_E_INTERNAL, "table check: " + what}; };
    const int64_t S = n_slots_;
    for (int64_t k = 0; k < mesh_.K; ++k) {
      const int64_t s = ord_.slot_of[k];
      if (s >= S || (s >= 0 && ord_.elem_of[s] != k)) fail("slot_of/elem_of of element " + std::to_string(k));
    }
    int64_t nb = 0;
    for (int64_t s = 0; s < S; ++s) {
      if (bface[s] != nb) fail("boundary-face start of slot " + std::to_string(s));
      if (!(meta[s] & kMetaValid)) continue;
      for (int f = 0; f < 4; ++f) {
        const int n2 = nbr[s * 4 + f];
        const int nf = finfo_face(finfo[s * 4 + f]), pc = finfo_perm(finfo[s * 4 + f]);
        const int bc = finfo_bc(finfo[s * 4 + f]);
        const std::string at = "slot " + std::to_string(s) + " face " + std::to_string(f);
        if (n2 < -1 || n2 >= S) fail("neighbour slot out of range at " + at);
        if ((n2 < 0) != (bc != 0)) fail("boundary code and neighbour disagree at " + at);
        if (pc > 5 || bc > 3) fail("face code out of range at " + at);
        if (n2 < 0) {
          ++nb;
          continue;
        }
        if ((meta[n2] & kMetaValid) && nbr[int64_t(n2) * 4 + nf] != int(s)) fail("asymmetric neighbours at " + at);
      }
    }
    if (nb != n_bfaces_) fail("boundary-face count");
    for (int c = 0; c < 6; ++c) {
      std::vector<int> seen(Nfp_, 0);
      for (int j = 0; j < Nfp_; ++j) {
        const int q = ref_.perm[c][j];
        if (q < 0 || q >= Nfp_ || seen[q]++) fail("face-node permutation " + std::to_string(c));
      }
    }
    for (int f = 0; f < 4; ++f)
      for (int j = 0; j < Nfp_; ++j)
        if (ref_.fmask[f][j] < 0 || ref_.fmask[f][j] >= Np_) fail("face node " + std::to_string(j) + " of face " + std::to_string(f));
  }

  // Per-element coefficients of the FP32 tensor-core kernel for penalty sign `sigma` (Eq. penaltyFlux
  // with tau negated in backward runs), [n_slots][kGtab]: -rho c^2 rx_ij (volume p equation,
  // Eq. dgLocalSchemeP), rho c, -rx_ij / rho (volume v equation, Eq. dgLocalSchemeU), the outward
  // normals, and per face the coefficients of t = A [n.v] + B [p] and s = C [p] + D [n.v] with the
  // surface Jacobian and the 1/2 of the weak form folded in.
  // Per-element material factors: rho c^2 with the current velocity; the impedance (penalty
  // parameters, characteristics of I_Q) with the velocity the solver was created with.
  void upload_material() {
    const int64_t S = n_slots_;
    std::vector<real> mat(S * kMat, real(0));
    for (int64_t s = 0; s < S; ++s) {
      int64_t k = ord_.elem_of[s];
      if (k < 0) continue;
      const double Zk = rho_[k] * c_ref_[k];
      mat[s * kMat + 0] = real(rho_[k] * c_[k] * c_[k]);
      mat[s * kMat + 1] = real(1.0 / rho_[k]);
      mat[s * kMat + 2] = real(Zk);
      for (int f = 0; f < 4; ++f) {
        int64_t k2 = mesh_.nbr[4 * k + f];
        double Zb = k2 >= 0 ? 0.5 * (Zk + rho_[k2] * c_ref_[k2]) : Zk;
        mat[s * kMat + 3 + f] = real(tau_scale_ / Zb);
        mat[s * kMat + 7 + f] = real(tau_scale_ * Zb);
      }
    }
    upload(mat_d_, mat, st_);
    if (std::is_same<real, float>::value) {
      upload(gtab_d_[0], coefficient_table(+1), st_);
      upload(gtab_d_[1], coefficient_table(-1), st_);
    }
  }

  std::vector<float> coefficient_table(int sigma) const {
    const int64_t S = n_slots_;
    std::vector<float> g(size_t(S) * kGtab, 0.f);
    for (int64_t s = 0; s < S; ++s) {
      int64_t k = ord_.elem_of[s];
      if (k < 0) continue;
      float* at = &g[size_t(s) * kGtab];
      const double rho = rho_[k], c = c_[k], rc2 = rho * c * c, irho = 1.0 / rho, Zk = rho * c_ref_[k];
      for (int i = 0; i < 9; ++i) {
        at[kGtU + i] = float(-rc2 * geo_.rx[9 * k + i]);
        at[kGtV + i] = float(-irho * geo_.rx[9 * k + i]);
      }
      at[kGtZ] = float(Zk);
      for (int f = 0; f < 4; ++f) {
        for (int d = 0; d < 3; ++d) at[kGtN + 4 * f + d] = float(geo_.normal[12 * k + 3 * f + d]);
        int64_t k2 = mesh_.nbr[4 * k + f];
        double Zb = k2 >= 0 ? 0.5 * (Zk + rho_[k2] * c_ref_[k2]) : Zk;
        double fs = geo_.fscale[4 * k + f], taup = sigma * tau_scale_ / Zb, tauv = sigma * tau_scale_ * Zb;
        at[kGtP + 4 * f + 0] = float(-0.5 * fs * rc2);
        at[kGtP + 4 * f + 1] = float(0.5 * fs * rc2 * taup);
        at[kGtP + 4 * f + 2] = float(0.5 * fs * irho);
        at[kGtP + 4 * f + 3] = float(-0.5 * fs * irho * tauv);
      }
    }
    return g;
  }

  // TF32 rounding (round to nearest, ties away from zero) of an FP32 value
  static uint32_t tf32_bits(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return u;
    u += 0x1000u;
    return u & 0xffffe000u;
  }
  // Operator fragments of mma.m16n8k8 (A: 16 x 8 row major; lane (g, t) holds rows g, g+8 and
  // columns t, t+4) for D_r, D_s, D_t and the four LIFT blocks, tiles of 16 nodes x 8 nodes,
  // each value split into TF32 hi and lo (hi + lo = the FP64 operator to ~2^-22).  One stream
  // per node tile mt, in the order the kernel consumes them: D_jd k-steps, then LIFT blocks.
  // BF16 rounding (round to nearest even) of an FP32 value, as the 16 high bits
  static uint32_t bf16_bits(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return u >> 16;
    u += 0x7fffu + ((u >> 16) & 1u);
    return u >> 16;
  }
  // Operator fragments for the tensor-core products, one stream per node tile mt, in the order the
  // kernel consumes them: D_jd k-steps, then LIFT blocks; each value split into hi and lo
  // (hi + lo = the FP64 operator to ~2^-22 in TF32, ~2^-16 in BF16).
  //  TF32 (mma.m16n8k8, A 16 x 8 row major): lane (g, t) holds rows g, g+8 and columns t, t+4.
  //  BF16 (mma.m16n8k16, A 16 x 16 row major): lane (g, t) holds rows g, g+8 and fragment columns
  //  2t, 2t+1 (register 0/1) and 2t+8, 2t+9 (register 2/3), two values per register, lower column
  //  in the low half; fragment columns 2t, 2t+1, 2t+8, 2t+9 are the step's nodes t, t+4, t+8, t+12
  //  (the kernel loads B in the same order).
  // FP16 rounding (round to nearest even) of an FP32 value, as its 16 bits
  static uint32_t fp16_bits(float x) {
    const __half_raw r = __half(__float2half_rn(x));
    return r.x;
  }
  static float fp16_value(uint32_t bits) {
    __half_raw r;
    r.x = uint16_t(bits);
    return __half2float(__half(r));
  }

  std::vector<uint32_t> operator_fragments(int contraction) const {
    const bool bf16 = contraction != RIDG_CONTRACT_TENSOR;  // a 16-bit split: BF16 or FP16
    const bool fp16 = contraction == RIDG_CONTRACT_TENSOR_FP16;
    const int KS = bf16 ? 16 : 8;
    const int MT = (Np_ + 15) / 16, KSD = (Np_ + KS - 1) / KS, KSF = (Nfp_ + KS - 1) / KS;
    const int NSTEP = 3 * KSD + 4 * KSF;
    std::vector<uint32_t> out(size_t(MT * NSTEP) * 256, 0u);
    // op(r, c): the operator value of row r, column c of step (matrix, k-step kb)
    auto tile = [&](size_t step, int mt, int kb, int ncol, auto&& op) {
      for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, t = lane & 3;
        auto val = [&](int r, int c) { return (r < Np_ && c < ncol) ? op(r, c) : 0.0; };
        for (int q = 0; q < 4; ++q) {
          const int r = mt * 16 + g + 8 * (q & 1);
          uint32_t hi, lo;
          if (!bf16) {
            const int c = kb * 8 + t + 4 * (q >> 1);
            const double v = val(r, c);
            hi = tf32_bits(float(v));
            float hv;
            std::memcpy(&hv, &hi, 4);
            lo = tf32_bits(float(v - double(hv)));
          } else {
            const int c0 = kb * 16 + t + 8 * (q >> 1), c1 = c0 + 4;  // fragment columns 2t(+8), 2t+1(+8)
            uint32_t h2[2], l2[2];
            const double v2[2] = {val(r, c0), val(r, c1)};
            for (int i = 0; i < 2; ++i) {
              if (fp16) {
                h2[i] = fp16_bits(float(v2[i]));
                l2[i] = fp16_bits(float(v2[i] - double(fp16_value(h2[i]))));
                continue;
              }
              h2[i] = bf16_bits(float(v2[i]));
              const uint32_t hb = h2[i] << 16;
              float hv;
              std::memcpy(&hv, &hb, 4);
              l2[i] = bf16_bits(float(v2[i] - double(hv)));
            }
            hi = h2[0] | (h2[1] << 16);
            lo = l2[0] | (l2[1] << 16);
          }
          out[step * 256 + lane * 8 + q] = hi;
          out[step * 256 + lane * 8 + 4 + q] = lo;
        }
      }
    };
    for (int mt = 0; mt < MT; ++mt) {
      for (int jd = 0; jd < 3; ++jd)
        for (int kb = 0; kb < KSD; ++kb)
          tile(size_t(mt * NSTEP + jd * KSD + kb), mt, kb, Np_, [&](int r, int c) { return ref_.D[jd](r, c); });
      for (int f = 0; f < 4; ++f)
        for (int kb = 0; kb < KSF; ++kb)
          tile(size_t(mt * NSTEP + 3 * KSD + f * KSF + kb), mt, kb, Nfp_,
               [&](int r, int c) { return ref_.LIFT(r, f * Nfp_ + c); });
    }
    return out;
  }


  void alloc_wave(Wave<real>& w) {
    if (w.q.p) return;
    w.q.alloc(qsize() * sizeof(real));
    w.ring.alloc(3 * qsize() * sizeof(real));
    w.trace.alloc(3 * trace_slot_elems() * sizeof(real));
    zero_wave(w);
    if (!w.inj_range.p) {
      upload(w.inj_range, std::vector<int2>(n_slots_, make_int2(0, 0)), st_);
      upload(w.inj_w, std::vector<real>(Np_, real(0)), st_);
      upload(w.inj_row, std::vector<int>{0}, st_);
    }
  }
  void zero_wave(Wave<real>& w) {
    RIDG_CUDA(cudaMemsetAsync(w.q.p, 0, w.q.bytes, st_));
    RIDG_CUDA(cudaMemsetAsync(w.ring.p, 0, w.ring.bytes, st_));
    RIDG_CUDA(cudaMemsetAsync(w.trace.p, 0, w.trace.bytes, st_));
  }

  std::vector<real> projected_dirac(int64_t k, const double rst[3]) const {
    // Eq. sourceTerm: M_k w = l(x0), M_k = J_k M
    std::array<double, 3> p = {rst[0], rst[1], rst[2]};
    std::vector<double> l = ref_.lagrange_at(p);
    std::vector<real> w(Np_, real(0));
    for (int i = 0; i < Np_; ++i) {
      double acc = 0.0;
      for (int j = 0; j < Np_; ++j) acc += ref_.Minv(i, j) * l[j];
      w[i] = real(acc / geo_.J[k]);
    }
    return w;
  }

  WaveArgs<real> wave_args(Wave<real>& w) {
    WaveArgs<real> a{};
    a.q = dptr<real>(w.q);
    a.ring = dptr<real>(w.ring);
    a.trace = dptr<real>(w.trace);
    a.inj_range = dptr<const int2>(w.inj_range);
    a.inj_w = dptr<const real>(w.inj_w);
    a.inj_row = dptr<const int>(w.inj_row);
    return a;
  }

  StepArgs<real> base_args() const {
    StepArgs<real> a{};
    a.n_slots = n_slots_;
    a.n_levels = L_;
    for (int l = 0; l <= L_; ++l) a.level_begin[l] = ord_.level_begin[l];
    for (int l = L_ + 1; l <= kMaxLevels; ++l) a.level_begin[l] = n_slots_;
    a.geo = dptr<const double>(geo_d_);
    a.mat = dptr<const real>(mat_d_);
    a.nbr = dptr<const int>(nbr_d_);
    a.finfo = dptr<const uint8_t>(finfo_d_);
    a.bface = dptr<const int>(bface_d_);
    a.meta = dptr<const int>(meta_d_);
    a.Dt = dptr<const real>(Dt_d_);
    a.Lt = dptr<const real>(Lt_d_);
    a.fmask = dptr<const int>(fmask_d_);
    a.perm = dptr<const int>(perm_d_);
    a.afrag = dptr<const uint32_t>(afrag_d_);
    a.contraction = contraction_;
    a.e_up[2] = real(-1);
    return a;
  }

  // arguments of one step of the finest level at the current time tau_ (direction sigma)
  StepArgs<real> fine_args(int sigma, int W, int mode) const {
    (void)W;
    StepArgs<real> a = base_args();
    int l0 = first_active_level(tau_);
    a.slot_lo = ord_.level_begin[l0 - 1];
    a.slot_hi = ord_.owned_end;
    a.trace_read = mod3(tau_);
    for (int l = 1; l <= L_; ++l) {
      int64_t d = int64_t(1) << (L_ - l);
      int c = ring_count_[l - 1];
      a.ring_new[l - 1] = c % 3;
      a.ring_old1[l - 1] = (c + 2) % 3;
      a.ring_old2[l - 1] = (c + 1) % 3;
      a.h[l - 1] = real(double(sigma) * double(d) * lv_.dt_local);
      a.trace_write[l - 1] = mod3(tau_ + sigma * d);
      a.trace_half[l - 1] = d >= 2 ? mod3(tau_ + sigma * (d / 2)) : mod3(tau_ + 2 * sigma);
    }
    a.tau_sign = real(sigma);
    a.mode = mode;
    return a;
  }

  // batch != null: n shots in lockstep, one merged launch where the kernel supports it (FP32 tensor-core
  // contractions), else one launch per shot with its arguments in the step's own
  void launch(const StepArgs<real>& a0, int W, const BatchArgs<real>* batch = nullptr, int n = 1) {
    StepArgs<real> a = a0;
    a.gtab = dptr<const float>(gtab_d_[a.tau_sign > real(0) ? 0 : 1]);
    const bool merges = std::is_same<real, float>::value && contraction_ != RIDG_CONTRACT_CUDA_CORES;
    auto one = [&](const StepArgs<real>& x, const BatchArgs<real>* bt) {
      cudaError_t e = dispatch_order(N_, [&](auto NC) {
        return Launch<decltype(NC)::value, real>::step(x, W, st_, bt, bt ? n : 1);
      });
      if (e != cudaSuccess) throw Error{RIDG_E_CUDA, std::string("step kernel launch: ") + cudaGetErrorString(e)};
      ++stats_.kernel_launches;
      ++stats_.fused_launches;
    };
    if (!batch) return one(a, nullptr);
    if (merges) {
      BatchArgs<real> bt = *batch;
      bt.shot_blocks = int((a.slot_hi - a.slot_lo) / (32 / W));
      return one(a, &bt);
    }
    for (int b = 0; b < n; ++b) {
      StepArgs<real> x = a;
      const ShotArgs<real>& sa = batch->shot[b];
      x.wave[0] = sa.wave[0];
      x.wave[1] = sa.wave[1];
      x.arena_write = sa.arena_write;
      x.arena_read = sa.arena_read;
      x.image_p = sa.image_p;
      x.image_q = sa.image_q;
      one(x, nullptr);
    }
  }

  void launch_fine(const StepArgs<real>& a, int sigma, int W, const BatchArgs<real>* batch = nullptr, int n = 1) {
    int l0 = first_active_level(tau_);
    static const char* const kStepNames[kMaxLevels] = {
        "fine step, levels 1+", "fine step, levels 2+", "fine step, levels 3+", "fine step, levels 4+",
        "fine step, levels 5+", "fine step, levels 6+", "fine step, levels 7+", "fine step, levels 8+"};
    NvtxRange nv(kStepNames[std::min(std::max(l0, 1), kMaxLevels) - 1]);
    bool prof = prof_every_ > 0 && l0 == 1 && ((tau_ / NL_) % prof_every_) == 0;
    if (prof) {
      if (prof_used_ >= prof_w_.size()) {
        cudaEvent_t e0, e1;
        RIDG_CUDA(cudaEventCreate(&e0));
        RIDG_CUDA(cudaEventCreate(&e1));
        prof_ev_.push_back(e0);
        prof_ev_.push_back(e1);
        prof_w_.push_back(0);
      }
      prof_w_[prof_used_] = W;
      RIDG_CUDA(cudaEventRecord(prof_ev_[2 * prof_used_], st_));
    }
    launch(a, W, batch, n);
    if (prof) {
      RIDG_CUDA(cudaEventRecord(prof_ev_[2 * prof_used_ + 1], st_));
      ++prof_used_;
    }
    if (hook_) hook_->exchange(*this, l0, W == 2 ? 3 : 1);
    for (int l = l0; l <= L_; ++l) {
      ring_count_[l - 1] += 1;
      dof_ += level_count_[l - 1] * 4 * Np_ * W * (batch ? n : 1);
    }
    tau_ += sigma;
  }

  void init_traces_into(const real* q, real* trace, int slot) {
    cudaError_t e = dispatch_order(N_, [&](auto NC) {
      return Launch<decltype(NC)::value, real>::init_traces(
          q, trace, slot, n_slots_, dptr<const double>(geo_d_), dptr<const int>(meta_d_), dptr<const int>(fmask_d_),
          dptr<const int>(nbr_d_), dptr<const uint8_t>(finfo_d_), dptr<const int>(perm_d_), st_);
    });
    if (e != cudaSuccess) throw Error{RIDG_E_CUDA, cudaGetErrorString(e)};
    ++stats_.kernel_launches;
  }
  void init_traces(Wave<real>& w, int slot) { init_traces_into(dptr<real>(w.q), dptr<real>(w.trace), slot); }

  void sample(double* traces, int64_t n_t, int64_t col, int64_t nrec) { sample(shot_ref(0), traces, n_t, col, nrec); }
  // receiver traces of shot S's source wavefield at column col
  void sample(const ShotRef& S, double* traces, int64_t n_t, int64_t col, int64_t nrec) {
    if (nrec <= 0) return;
    cudaError_t e = dispatch_order(N_, [&](auto NC) {
      return Launch<decltype(NC)::value, real>::sample(dptr<real>(S.w[0].q), dptr<const int64_t>(*S.rec_slot),
                                                        dptr<const real>(*S.rec_row), int(nrec), traces, n_t, col, st_);
    });
    if (e != cudaSuccess) throw Error{RIDG_E_CUDA, cudaGetErrorString(e)};
    ++stats_.kernel_launches;
  }

  void snapshot_history(const ShotRef& S, int l, int count_before) {
    // the step that just ran wrote r(t_f + 2 dt_l) into ring slot count_before % 3; the one before
    // it, r(t_f + dt_l), sits in (count_before + 2) % 3.  The backward run starts with counter 0,
    // whose older slots are 2 (one step back: t_f + dt_l) and 1 (two steps back: t_f + 2 dt_l).
    size_t per = 4 * size_t(Np_) * 32;
    size_t off = size_t(ord_.level_begin[l - 1] / 32) * per;
    size_t len = size_t((ord_.level_begin[l] - ord_.level_begin[l - 1]) / 32) * per * sizeof(real);
    if (len == 0) return;
    const char* ring = static_cast<const char*>(S.w[0].ring.p);
    char* snap = static_cast<char*>(S.ring_snap->p);
    size_t qb = qsize() * sizeof(real);
    int newest = count_before % 3, prev = (count_before + 2) % 3;
    RIDG_CUDA(cudaMemcpyAsync(snap + 1 * qb + off * sizeof(real), ring + newest * qb + off * sizeof(real), len,
                              cudaMemcpyDeviceToDevice, st_));
    RIDG_CUDA(cudaMemcpyAsync(snap + 2 * qb + off * sizeof(real), ring + prev * qb + off * sizeof(real), len,
                              cudaMemcpyDeviceToDevice, st_));
  }

  void image_out(const double* img, const double* inv_scale, double* out) {
    cudaError_t e = dispatch_order(N_, [&](auto NC) {
      return Launch<decltype(NC)::value, real>::image_out(img, dptr<const int64_t>(slot_of_d_), dptr<const int>(pos_d_),
                                                           mesh_.K, inv_scale, out, st_);
    });
    if (e != cudaSuccess) throw Error{RIDG_E_CUDA, cudaGetErrorString(e)};
    ++stats_.kernel_launches;
  }

  double energy_of(const real* q) {
    DBuf out;
    out.alloc(sizeof(double));
    RIDG_CUDA(cudaMemsetAsync(out.p, 0, sizeof(double), st_));
    cudaError_t e = dispatch_order(N_, [&](auto NC) {
      return Launch<decltype(NC)::value, real>::energy(q, n_slots_, dptr<const double>(J_d_), dptr<const real>(mat_d_),
                                                        dptr<const int>(meta_d_), dptr<const double>(M_d_),
                                                        dptr<double>(out), st_);
    });
    if (e != cudaSuccess) throw Error{RIDG_E_CUDA, cudaGetErrorString(e)};
    double v = 0.0;
    RIDG_CUDA(cudaMemcpyAsync(&v, out.p, sizeof(double), cudaMemcpyDeviceToHost, st_));
    RIDG_CUDA(cudaStreamSynchronize(st_));
    return v;
  }

  // this solver advances element k (the whole mesh, or its part of a partitioned mesh)
  bool owned(int64_t k) const { return ord_.slot_of[k] >= 0 && ord_.slot_of[k] < ord_.owned_end; }

  MeshData mesh_;
  std::vector<int32_t> part_;  // part per element of a partitioned mesh (empty: the whole mesh)
  int32_t rank_ = 0;
  PartHook<real>* hook_ = nullptr;
  int N_, Np_ = 0, Nfp_ = 0, NFPP_ = 16, NPa_ = 0;
  cudaStream_t st_;
  RefElem ref_;
  Geometry geo_;
  PointLocator loc_;
  Levels lv_;
  Ordering ord_;
  std::vector<double> c_, c_ref_, rho_, xnodes_;
  // misfit gradient: the last misfit forward run (checkpoints of the single-level state)
  struct AdjointRun {
    bool ready = false;
    Wavelet wav;
    int64_t n_global = 0, seg = 1, n_ck = 0, nrec = 0, src_slot = 0, n_groups = 0;
    std::vector<int64_t> ck_tau, ck_count;
    std::vector<double> amp;
  } adj_;
  DBuf ck_q_, ck_ring_, ck_trace_, adj_res_, adj_w_, adj_rec_slot_, adj_rec_row_, adj_grp_, adj_rec_sorted_;
  int64_t n_slots_ = 0, NL_ = 1, n_bfaces_ = 0;
  int L_ = 1;
  std::vector<int> bface_host_;
  std::vector<int64_t> level_count_;
  DBuf geo_d_, J_d_, mat_d_, nbr_d_, finfo_d_, bface_d_, meta_d_, Dt_d_, Dt4_d_, Lt_d_, fmask_d_, perm_d_, M_d_, slot_of_d_;
  DBuf afrag_d_, gtab_d_[2], pos_d_, inv_fmask_d_;
  double tau_scale_ = 1.0;
  double cfl_ = 0.15;
  static constexpr double kVelocityCflMargin = 4.0 / 3.0;
  int contraction_ = RIDG_CONTRACT_TENSOR;  // how the FP32 element products run (FP64: CUDA cores)
  int image_mode_ = kModeImage;
  std::vector<int> pos_of_;  // device position of each reference node
  DBuf q_snap_, ring_snap_, img_p_, img_q_, arena_, rec_slot_, rec_row_, traces_tmp_, scale_d_;
  HBuf host_arena_;
  bool debug_ = false;       // RIDG_DEBUG: host checks of the tables
  size_t trace_budget_ = 0;  // device bytes for boundary-trace records (0: no limit)
  TraceTier tier_;           // after the buffers it copies between: destroyed (and drained) first
  Wave<real> w_[2];
  // device state of shots 1.. of a merged batch (shot 0 uses the buffers above)
  struct ShotState {
    Wave<real> w[2];
    DBuf rec_slot, rec_row, traces_tmp, arena, q_snap, ring_snap, img_p, img_q, scale;
  };
  std::vector<std::unique_ptr<ShotState>> extra_shots_;
  // CUDA-graph replay (ridg_set_graph_replay): the key of the last direct run and the captured graph
  bool graph_on_ = false, graph_seen_ = false;
  std::vector<uint64_t> graph_key_, graph_exec_key_;
  cudaGraphExec_t graph_exec_ = nullptr;
  ridg_shot_stats graph_stats_{};
  int64_t graph_tau_ = 0, graph_dof_ = 0;
  std::vector<int> graph_ring_;
  int64_t tau_ = 0, dof_ = 0;
  std::vector<int> ring_count_;
  ridg_shot_stats stats_{};
  int prof_every_ = 0;
  size_t prof_used_ = 0;
  std::vector<cudaEvent_t> prof_ev_;
  std::vector<int> prof_w_;
  int64_t n_half_ = 0;
};


// ------------------------------------------------------------------ domain decomposition (Sec. 4.2)
// A host barrier for the threads that drive the parts of a group; a part that fails releases the
// others (their wait then throws) so that no thread waits for a part that will not arrive.
class PartBarrier {
 public:
  void reset(int n) {
    std::lock_guard<std::mutex> l(m_);
    n_ = n;
    count_ = 0;
    aborted_ = false;
  }
  void wait() {
    std::unique_lock<std::mutex> l(m_);
    if (aborted_) throw Error{RIDG_E_CUDA, "another part of the group failed"};
    const int64_t gen = gen_;
    if (++count_ == n_) {
      count_ = 0;
      ++gen_;
      cv_.notify_all();
      return;
    }
    cv_.wait(l, [&] { return gen_ != gen || aborted_; });
    if (gen_ == gen) throw Error{RIDG_E_CUDA, "another part of the group failed"};
  }
  void abort() {
    std::lock_guard<std::mutex> l(m_);
    aborted_ = true;
    cv_.notify_all();
  }

 private:
  std::mutex m_;
  std::condition_variable cv_;
  int n_ = 1, count_ = 0;
  int64_t gen_ = 0;
  bool aborted_ = false;
};

// One solver per part.  Part p's elements push their traces across an interface face into the inbox
// of p's ghost copy of the neighbour (an element of part q); after a fine step those rows (all three
// time slots) go to q, into the inbox of q's own element: gathered on p's stream into a send buffer
// (two, used in turn), copied on q's stream once p's gather has run, and scattered.  A send buffer
// is gathered into again only after q's copy from it two transfers earlier has run.  The rows of
// one ordered pair of parts are sorted by the level of the pushing element, finest first, so the
// rows pushed at a step whose coarsest advanced level is l0 are a prefix.  Each part's thread runs
// the unchanged single-solver shot; the solver calls exchange() after every fine step.
template <typename real>
class Group final : public ridg_group, public PartHook<real> {
  struct Pair {
    int from = 0, to = 0;
    int64_t n = 0;
    std::vector<int64_t> prefix;  // [L + 2]: rows pushed by levels >= l0
    DBuf src_rows, dst_rows;      // on from's and to's device
    DBuf send[2], recv;           // [2 wavefields][n][3][row_len]
    cudaEvent_t copied[2] = {nullptr, nullptr};  // recorded on to's stream after each copy
  };
  struct Part {
    int dev = 0;
    cudaStream_t st = nullptr;
    std::unique_ptr<Engine<real>> e;
    cudaEvent_t packed[2] = {nullptr, nullptr};
    int64_t parity = 0, transfer_steps = 0, silent_steps = 0, bytes = 0;
    unsigned long long max_bits = 0, global_bits = 0;
    std::vector<int> out_pairs, in_pairs;
    DBuf traces, obs, img_p, img_q;
  };

 public:
  Group(const MeshData& mesh, int N, const double* c, const double* rho, const ridg_options& opt,
        const int32_t* part, int32_t n_parts, const int32_t* devices)
      : K_(mesh.K), parts_(checked_parts(n_parts)) {
    std::vector<int64_t> count(n_parts, 0);
    for (int64_t k = 0; k < mesh.K; ++k) {
      if (part[k] < 0 || part[k] >= n_parts) throw Error{RIDG_E_INVALID_ARG, "part index out of range"};
      ++count[part[k]];
    }
    for (int p = 0; p < n_parts; ++p)
      if (count[p] == 0) throw Error{RIDG_E_INVALID_ARG, "part " + std::to_string(p) + " has no elements"};
    int dev0 = 0;
    RIDG_CUDA(cudaGetDevice(&dev0));
    for (int p = 0; p < n_parts; ++p) {
      Part& P = parts_[p];
      P.dev = devices ? devices[p] : dev0;
      RIDG_CUDA(cudaSetDevice(P.dev));
      RIDG_CUDA(cudaStreamCreateWithFlags(&P.st, cudaStreamNonBlocking));
      P.e.reset(new Engine<real>(mesh, N, c, rho, opt, P.st, part, p));
      P.e->hook_ = this;
      for (int i = 0; i < 2; ++i) RIDG_CUDA(cudaEventCreateWithFlags(&P.packed[i], cudaEventDisableTiming));
    }
    const Engine<real>& e0 = *parts_[0].e;
    L_ = e0.L_;
    row_len_ = 2 * e0.NFPP_;
    // interface rows of every ordered pair of parts
    std::map<std::pair<int, int>, std::vector<std::array<int64_t, 5>>> rows;  // (-level, g, f, src, dst)
    for (int p = 0; p < n_parts; ++p) {
      const Engine<real>& ep = *parts_[p].e;
      for (int64_t sl = ep.ord_.owned_end; sl < ep.ord_.n_slots; ++sl) {
        const int64_t g = ep.ord_.elem_of[sl];
        if (g < 0) continue;
        const int q = part[g];
        for (int f = 0; f < 4; ++f) {
          const int64_t el = mesh.nbr[4 * g + f];
          if (el < 0 || part[el] != p) continue;
          const int64_t dst = parts_[q].e->ord_.slot_of[g];
          rows[{p, q}].push_back({-int64_t(e0.lv_.level[el]), g, f, sl * 4 + f, dst * 4 + f});
        }
      }
    }
    for (auto& kv : rows) {
      auto& v = kv.second;
      std::sort(v.begin(), v.end());
      auto pr = std::make_unique<Pair>();
      pr->from = kv.first.first;
      pr->to = kv.first.second;
      pr->n = int64_t(v.size());
      pr->prefix.assign(L_ + 2, 0);
      for (int l0 = 1; l0 <= L_; ++l0)
        for (const auto& r : v)
          if (-r[0] >= l0) ++pr->prefix[l0];
      std::vector<int64_t> src(v.size()), dst(v.size());
      for (size_t i = 0; i < v.size(); ++i) {
        src[i] = v[i][3];
        dst[i] = v[i][4];
      }
      const size_t buf = size_t(2) * pr->n * 3 * row_len_ * sizeof(real);
      Part& F = parts_[pr->from];
      Part& T = parts_[pr->to];
      RIDG_CUDA(cudaSetDevice(F.dev));
      upload(pr->src_rows, src, F.st);
      pr->send[0].alloc(buf);
      pr->send[1].alloc(buf);
      RIDG_CUDA(cudaStreamSynchronize(F.st));
      RIDG_CUDA(cudaSetDevice(T.dev));
      upload(pr->dst_rows, dst, T.st);
      pr->recv.alloc(buf);
      for (int i = 0; i < 2; ++i) RIDG_CUDA(cudaEventCreateWithFlags(&pr->copied[i], cudaEventDisableTiming));
      RIDG_CUDA(cudaStreamSynchronize(T.st));
      F.out_pairs.push_back(int(pairs_.size()));
      T.in_pairs.push_back(int(pairs_.size()));
      pairs_.push_back(std::move(pr));
    }
    any_.assign(L_ + 2, false);
    for (int l0 = 1; l0 <= L_; ++l0)
      for (const auto& pr : pairs_) any_[l0] = any_[l0] || pr->prefix[l0] > 0;
    RIDG_CUDA(cudaSetDevice(dev0));
  }

  ~Group() override {
    for (auto& pr : pairs_) {
      cudaSetDevice(parts_[pr->to].dev);
      for (auto ev : pr->copied)
        if (ev) cudaEventDestroy(ev);
    }
    pairs_.clear();
    for (auto& P : parts_) {
      cudaSetDevice(P.dev);
      if (P.st) cudaStreamSynchronize(P.st);
      P.e.reset();
      P.traces.release();
      P.obs.release();
      P.img_p.release();
      P.img_q.release();
      for (auto ev : P.packed)
        if (ev) cudaEventDestroy(ev);
      if (P.st) cudaStreamDestroy(P.st);
    }
  }

  // ---- PartHook (called from the part's own thread, its device current)
  void exchange(Engine<real>& e, int l0, int waves) override {
    Part& P = parts_[e.rank_];
    if (fault_fires(kFaultExchange)) throw Error{RIDG_E_CUDA, "interface transfer failed (injected failure)"};
    if (!any_[l0]) {
      ++P.silent_steps;  // nothing pushed across an interface (finest level only, lumping held)
      return;
    }
    ++P.transfer_steps;
    const int par = int(P.parity++ & 1);
    for (int i : P.out_pairs) {
      Pair& pr = *pairs_[i];
      const int64_t n = pr.prefix[l0];
      if (n == 0) continue;
      RIDG_CUDA(cudaStreamWaitEvent(P.st, pr.copied[par], 0));  // the copy out of this buffer two transfers ago
      for (int w = 0; w < 2; ++w)
        if (waves & (1 << w)) check(pack_face_rows<real>(dptr<const real>(e.w_[w].trace), e.n_slots_, row_len_,
                                                         dptr<const int64_t>(pr.src_rows), n,
                                                         dptr<real>(pr.send[par]) + size_t(w) * pr.n * 3 * row_len_, P.st));
    }
    RIDG_CUDA(cudaEventRecord(P.packed[par], P.st));
    barrier_.wait();
    for (int i : P.in_pairs) {
      Pair& pr = *pairs_[i];
      const int64_t n = pr.prefix[l0];
      if (n == 0) continue;
      const Part& F = parts_[pr.from];
      RIDG_CUDA(cudaStreamWaitEvent(P.st, F.packed[par], 0));
      for (int w = 0; w < 2; ++w)
        if (waves & (1 << w)) {
          const size_t off = size_t(w) * pr.n * 3 * row_len_, bytes = size_t(n) * 3 * row_len_ * sizeof(real);
          RIDG_CUDA(cudaMemcpyPeerAsync(dptr<real>(pr.recv) + off, P.dev, dptr<const real>(pr.send[par]) + off, F.dev,
                                        bytes, P.st));
          P.bytes += int64_t(bytes);
        }
      RIDG_CUDA(cudaEventRecord(pr.copied[par], P.st));
      for (int w = 0; w < 2; ++w)
        if (waves & (1 << w)) check(unpack_face_rows<real>(dptr<real>(e.w_[w].trace), e.n_slots_, row_len_,
                                                           dptr<const int64_t>(pr.dst_rows), n,
                                                           dptr<const real>(pr.recv) + size_t(w) * pr.n * 3 * row_len_, P.st));
    }
  }

  void combine_data_scale(Engine<real>& e, void* work) override {
    Part& P = parts_[e.rank_];
    RIDG_CUDA(cudaMemcpyAsync(&P.max_bits, work, sizeof(P.max_bits), cudaMemcpyDeviceToHost, P.st));
    RIDG_CUDA(cudaStreamSynchronize(P.st));
    barrier_.wait();
    P.global_bits = 0;
    for (const Part& Q : parts_) P.global_bits = std::max(P.global_bits, Q.max_bits);
    barrier_.wait();
    RIDG_CUDA(cudaMemcpyAsync(work, &P.global_bits, sizeof(P.global_bits), cudaMemcpyHostToDevice, P.st));
    check(data_scale_finish(work, P.st));
    RIDG_CUDA(cudaStreamSynchronize(P.st));
  }

  // ---- the shot
  void shot(const ridg_source& src, const double* rec, int64_t nrec, double t_final, double t_i, const double* observed,
            double* traces_out, double* image_p, double* image_q, const double* e_up) override {
    if (nrec < 0 || (nrec > 0 && !rec)) throw Error{RIDG_E_INVALID_ARG, "bad receiver list"};
    const int64_t n_t = parts_[0].e->trace_len(t_final);
    const int Np = parts_[0].e->Np_;
    const size_t tb = size_t(std::max<int64_t>(nrec, 1)) * n_t * sizeof(double), ib = size_t(K_) * Np * sizeof(double);
    for (Part& P : parts_) {
      RIDG_CUDA(cudaSetDevice(P.dev));
      P.traces.reserve(tb);
      P.img_p.reserve(ib);
      P.img_q.reserve(ib);
      if (observed) {
        P.obs.reserve(tb);
        RIDG_CUDA(cudaMemcpyAsync(P.obs.p, observed, size_t(nrec) * n_t * sizeof(double), cudaMemcpyHostToDevice, P.st));
      }
      P.parity = P.transfer_steps = P.silent_steps = P.bytes = 0;
    }
    barrier_.reset(int(parts_.size()));
    std::vector<std::string> err(parts_.size());
    std::vector<int> code(parts_.size(), 0);
    std::vector<std::thread> th;
    for (size_t p = 0; p < parts_.size(); ++p)
      th.emplace_back([&, p] {
        Part& P = parts_[p];
        try {
          RIDG_CUDA(cudaSetDevice(P.dev));
          P.e->shot(src, rec, nrec, t_final, t_i, observed ? dptr<const double>(P.obs) : nullptr, dptr<double>(P.traces),
                    dptr<double>(P.img_p), dptr<double>(P.img_q), e_up);
          RIDG_CUDA(cudaStreamSynchronize(P.st));
        } catch (const Error& x) {
          code[p] = x.code;
          err[p] = x.msg;
          barrier_.abort();
        } catch (const std::exception& x) {
          code[p] = RIDG_E_CUDA;
          err[p] = x.what();
          barrier_.abort();
        }
      });
    for (auto& t : th) t.join();
    // the first failure that is not another part's release
    for (size_t p = 0; p < parts_.size(); ++p)
      if (code[p] != 0 && err[p] != "another part of the group failed")
        throw Error{code[p], "part " + std::to_string(p) + ": " + err[p]};
    for (size_t p = 0; p < parts_.size(); ++p)
      if (code[p] != 0) throw Error{code[p], "part " + std::to_string(p) + ": " + err[p]};
    // the union of the parts: traces and images of the other parts read zero in each
    std::vector<double> buf;
    auto gather = [&](DBuf Part::*member, double* out, size_t n) {
      if (!out) return;
      std::fill(out, out + n, 0.0);
      buf.resize(n);
      for (Part& P : parts_) {
        RIDG_CUDA(cudaSetDevice(P.dev));
        RIDG_CUDA(cudaMemcpy(buf.data(), (P.*member).p, n * sizeof(double), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i) out[i] += buf[i];
      }
    };
    gather(&Part::traces, traces_out, size_t(nrec) * n_t);
    gather(&Part::img_p, image_p, size_t(K_) * Np);
    gather(&Part::img_q, image_q, size_t(K_) * Np);
    dof_ = 0;
    for (Part& P : parts_) {
      RIDG_CUDA(cudaSetDevice(P.dev));
      const ridg_shot_stats& st = P.e->stats();
      dof_ += st.dof_updates_forward + st.dof_updates_backward;
    }
  }

  int64_t trace_len(double t_final, int32_t* np_out) const override {
    if (np_out) *np_out = parts_[0].e->Np_;
    return parts_[0].e->trace_len(t_final);
  }

  void info(ridg_group_info* out) const override {
    std::memset(out, 0, sizeof(*out));
    out->n_parts = int32_t(parts_.size());
    for (size_t p = 0; p < parts_.size(); ++p) {
      const Engine<real>& e = *parts_[p].e;
      out->elements[p] = std::count_if(e.ord_.elem_of.begin(), e.ord_.elem_of.begin() + e.ord_.owned_end,
                                       [](int64_t k) { return k >= 0; });
      out->ghosts[p] = std::count_if(e.ord_.elem_of.begin() + e.ord_.owned_end, e.ord_.elem_of.end(),
                                     [](int64_t k) { return k >= 0; });
      for (int i : parts_[p].out_pairs) out->interface_faces[p] += pairs_[i]->n;
      out->transfer_bytes += parts_[p].bytes;
    }
    out->dof_updates = dof_;
    out->transfer_steps = parts_[0].transfer_steps;
    out->silent_steps = parts_[0].silent_steps;
  }

 private:
  static void check(cudaError_t e) {
    if (e != cudaSuccess) throw Error{RIDG_E_CUDA, std::string("interface transfer: ") + cudaGetErrorString(e)};
  }
  static size_t checked_parts(int32_t n) {
    if (n < 1 || n > RIDG_MAX_PARTS) throw Error{RIDG_E_INVALID_ARG, "n_parts must be in 1..64"};
    return size_t(n);
  }

  int64_t K_ = 0, dof_ = 0;
  int L_ = 1, row_len_ = 32;
  std::vector<Part> parts_;
  std::vector<std::unique_ptr<Pair>> pairs_;
  std::vector<bool> any_;
  PartBarrier barrier_;
};

}  // namespace ridg

// ==================================================================== C ABI
using ridg::Error;

template <typename F>
static int guarded(F&& f) {
  try {
    f();
    ridg::g_last_error.clear();
    return RIDG_OK;
  } catch (const Error& e) {
    ridg::set_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    ridg::set_error("host allocation failed");
    return RIDG_E_OOM;
  } catch (const std::exception& e) {
    ridg::set_error(e.what());
    return RIDG_E_INVALID_ARG;
  } catch (...) {
    ridg::set_error("unknown error");
    return RIDG_E_INVALID_ARG;
  }
}

namespace ridg {

// Device buffers of a shot with host inputs and outputs (kept by a server between shots).
struct HostShotBuffers {
  DBuf obs, tr, ip, iq;
};

// One shot with host buffers: copies the observed traces in, runs the shot on the solver's stream,
// copies traces and images out and waits for them.
static void run_host_shot(ridg_solver* s, const ridg_source& src, const double* rec_xyz, int64_t nrec, double t_final,
                          double t_image_start, const double* observed, double* traces_out, double* image_p,
                          double* image_q, const double* e_up, HostShotBuffers& b) {
  ridg_info inf;
  s->info(&inf);
  int64_t n_t = s->trace_len(t_final);
  size_t tb = size_t(std::max<int64_t>(nrec, 1)) * n_t * sizeof(double);
  size_t ib = size_t(inf.K) * inf.Np * sizeof(double);
  cudaStream_t st = s->stream();
  if (observed) {
    b.obs.reserve(tb);
    RIDG_CUDA(cudaMemcpyAsync(b.obs.p, observed, size_t(nrec) * n_t * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  b.tr.reserve(tb);
  if (image_p) b.ip.reserve(ib);
  if (image_q) b.iq.reserve(ib);
  s->shot(src, rec_xyz, nrec, t_final, t_image_start, observed ? dptr<double>(b.obs) : nullptr, dptr<double>(b.tr),
          image_p ? dptr<double>(b.ip) : nullptr, image_q ? dptr<double>(b.iq) : nullptr, e_up);
  if (traces_out && nrec > 0)
    RIDG_CUDA(cudaMemcpyAsync(traces_out, b.tr.p, size_t(nrec) * n_t * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (image_p) RIDG_CUDA(cudaMemcpyAsync(image_p, b.ip.p, ib, cudaMemcpyDeviceToHost, st));
  if (image_q) RIDG_CUDA(cudaMemcpyAsync(image_q, b.iq.p, ib, cudaMemcpyDeviceToHost, st));
  RIDG_CUDA(cudaStreamSynchronize(st));
  if (image_p)
    for (size_t i = 0; i < ib / sizeof(double); ++i)
      if (!std::isfinite(image_p[i])) throw Error{RIDG_E_UNSTABLE, "non-finite image value"};
}

// n shots in lockstep with host buffers: the observed traces of each in, the batch on the solver's
// stream, every shot's traces and images out, then one wait.
static void run_host_shots(ridg_solver* s, int32_t n, const ridg_shot_io* io, double t_final, double t_image_start,
                           const double* e_up, HostShotBuffers* b) {
  if (n < 1 || n > kMaxBatch || !io) throw Error{RIDG_E_INVALID_ARG, "a batch holds 1 to " + std::to_string(kMaxBatch) + " shots"};
  ridg_info inf;
  s->info(&inf);
  const int64_t n_t = s->trace_len(t_final);
  const size_t ib = size_t(inf.K) * inf.Np * sizeof(double);
  cudaStream_t st = s->stream();
  std::vector<ridg_shot_io> dev(io, io + n);
  for (int i = 0; i < n; ++i) {
    const int64_t nrec = io[i].nrec;
    if (nrec < 0) throw Error{RIDG_E_INVALID_ARG, "bad receiver list of shot " + std::to_string(i)};
    const size_t tb = size_t(std::max<int64_t>(nrec, 1)) * n_t * sizeof(double);
    if (io[i].observed) {
      b[i].obs.reserve(tb);
      RIDG_CUDA(cudaMemcpyAsync(b[i].obs.p, io[i].observed, size_t(nrec) * n_t * sizeof(double), cudaMemcpyHostToDevice, st));
      dev[i].observed = dptr<double>(b[i].obs);
    }
    b[i].tr.reserve(tb);
    dev[i].traces_out = dptr<double>(b[i].tr);
    if (io[i].image_p) b[i].ip.reserve(ib);
    if (io[i].image_q) b[i].iq.reserve(ib);
    dev[i].image_p = io[i].image_p ? dptr<double>(b[i].ip) : nullptr;
    dev[i].image_q = io[i].image_q ? dptr<double>(b[i].iq) : nullptr;
  }
  s->shots(n, dev.data(), t_final, t_image_start, e_up);
  for (int i = 0; i < n; ++i) {
    const int64_t nrec = io[i].nrec;
    if (io[i].traces_out && nrec > 0)
      RIDG_CUDA(cudaMemcpyAsync(io[i].traces_out, b[i].tr.p, size_t(nrec) * n_t * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (io[i].image_p) RIDG_CUDA(cudaMemcpyAsync(io[i].image_p, b[i].ip.p, ib, cudaMemcpyDeviceToHost, st));
    if (io[i].image_q) RIDG_CUDA(cudaMemcpyAsync(io[i].image_q, b[i].iq.p, ib, cudaMemcpyDeviceToHost, st));
  }
  RIDG_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < n; ++i)
    if (io[i].image_p)
      for (size_t k = 0; k < ib / sizeof(double); ++k)
        if (!std::isfinite(io[i].image_p[k])) throw Error{RIDG_E_UNSTABLE, "non-finite image value"};
}

static_assert(kMaxBatch == RIDG_MAX_BATCH, "the merged launch holds as many shots as the ABI allows");

}  // namespace ridg

// Shot server: requests queued in arrival order, served by slots (one solver and one worker thread
// each); an idle slot takes the oldest request of its model.
struct ridg_server {
  using clock = std::chrono::steady_clock;
  struct Request {
    ridg_shot_request r{};
    std::vector<double> rec, obs, eup, samples;
    clock::time_point submitted, started, finished;
    int64_t slot = -1;
    bool done = false;
    int status = RIDG_OK;
    std::string error;
  };
  struct Slot {
    ridg_solver* solver = nullptr;
    int32_t model = 0;
    bool busy = false;     // running a request, or its buffers being released
    bool waiting = false;  // its request waits for device memory (counts as not running)
    std::thread worker;
    ridg::HostShotBuffers buffers[ridg::kMaxBatch];  // one per shot of a lockstep batch
  };
  std::vector<std::unique_ptr<Slot>> slots;
  int device = 0;
  int64_t max_queued = 1;
  int32_t max_batch = 1;  // waiting requests a slot starts together as one lockstep batch
  clock::time_point created = clock::now();
  std::mutex mu;
  std::condition_variable work_cv, done_cv;
  std::deque<int64_t> queue;
  std::map<int64_t, std::unique_ptr<Request>> requests;
  int64_t next_ticket = 1;
  int64_t finished_shots = 0;
  bool memory_wait = false;  // a request waits for device memory: idle slots start nothing new
  bool stop = false;

  bool serves(int32_t model) const {
    for (const auto& s : slots)
      if (s->model == model) return true;
    return false;
  }
  // oldest queued request of a model (queue.end() if none); mu held
  std::deque<int64_t>::iterator next_of(int32_t model) {
    for (auto it = queue.begin(); it != queue.end(); ++it)
      if (requests[*it]->r.model == model) return it;
    return queue.end();
  }

  // Device memory for the shot slot s is about to run: free it from idle slots, or wait for
  // running ones, or give up with RIDG_E_OOM.
  void admit(Slot* s, const Request* q, int32_t n_shots) {
    const size_t margin = size_t(256) << 20;
    struct Done {
      ridg_server* sv;
      Slot* s;
      ~Done() {
        std::lock_guard<std::mutex> lk(sv->mu);
        s->waiting = false;
        bool any = false;
        for (auto& o : sv->slots) any = any || o->waiting;
        sv->memory_wait = any;
      }
    } done{this, s};
    for (;;) {
      const size_t need = s->solver->shots_extra_device_bytes(q->r.t_final, n_shots);
      if (ridg::fault_fires(ridg::kFaultAdmission))
        throw Error{RIDG_E_OOM, "shot needs " + std::to_string(need) + " more device bytes (injected admission refusal)"};
      size_t free_b = 0, total_b = 0;
      RIDG_CUDA(cudaMemGetInfo(&free_b, &total_b));
      if (need + margin <= free_b) return;
      std::vector<Slot*> idle;
      bool running = false;
      int64_t seen = 0;
      {
        std::lock_guard<std::mutex> lk(mu);
        memory_wait = true;
        s->waiting = true;
        seen = finished_shots;
        for (auto& o : slots) {
          if (o.get() == s) continue;
          if (o->busy) {
            running = running || !o->waiting;
          } else {
            o->busy = true;
            idle.push_back(o.get());
          }
        }
      }
      size_t released = 0;
      for (Slot* o : idle) {
        released += o->solver->release_shot_buffers();
        for (ridg::HostShotBuffers& hb : o->buffers)
          for (ridg::DBuf* d : {&hb.obs, &hb.tr, &hb.ip, &hb.iq}) {
            released += d->bytes;
            d->release();
          }
      }
      released += [&] {
        // this slot's own host-shot buffers are re-reserved by the shot
        size_t b = 0;
        for (ridg::HostShotBuffers& hb : s->buffers)
          for (ridg::DBuf* d : {&hb.obs, &hb.tr, &hb.ip, &hb.iq}) {
            b += d->bytes;
            d->release();
          }
        return b;
      }();
      {
        std::unique_lock<std::mutex> lk(mu);
        for (Slot* o : idle) o->busy = false;
        if (released > 0) continue;
        if (!running)
          throw Error{RIDG_E_OOM, "shot needs " + std::to_string(need) + " more device bytes, " +
                                      std::to_string(free_b) + " free"};
        done_cv.wait(lk, [&] { return stop || finished_shots != seen; });
        if (stop) throw Error{RIDG_E_INVALID_ARG, "server stopped while the request waited for device memory"};
      }
    }
  }

  // a waiting request r may join q's lockstep batch: same record length, image window and e_up
  static bool joins(const Request* q, const Request* r) {
    return r->r.model == q->r.model && r->r.t_final == q->r.t_final && r->r.t_image_start == q->r.t_image_start &&
           r->eup == q->eup;
  }

  void run(Slot* s, int64_t index) {
    cudaSetDevice(device);
    for (;;) {
      std::vector<Request*> batch;
      {
        std::unique_lock<std::mutex> lk(mu);
        work_cv.wait(lk, [&] { return stop || (!memory_wait && !s->busy && next_of(s->model) != queue.end()); });
        if (stop) return;
        auto it = next_of(s->model);
        batch.push_back(requests[*it].get());
        queue.erase(it);
        // later requests of the model that share the time span join it, up to max_batch shots
        for (auto jt = queue.begin(); jt != queue.end() && int32_t(batch.size()) < max_batch;) {
          Request* r = requests[*jt].get();
          if (joins(batch[0], r)) {
            batch.push_back(r);
            jt = queue.erase(jt);
          } else {
            ++jt;
          }
        }
        s->busy = true;
        const auto now = clock::now();
        for (Request* r : batch) {
          r->started = now;
          r->slot = index;
        }
      }
      Request* q = batch[0];
      const int32_t n = int32_t(batch.size());
      // runs fn, recording its error as the status of the requests it served
      auto attempt = [](auto&& fn, int& status, std::string& error) {
        status = RIDG_OK;
        error.clear();
        try {
          fn();
        } catch (const Error& e) {
          status = e.code;
          error = e.msg;
        } catch (const std::bad_alloc&) {
          status = RIDG_E_OOM;
          error = "host allocation failed";
        } catch (const std::exception& e) {
          status = RIDG_E_INVALID_ARG;
          error = e.what();
        }
      };
      auto alone = [&](Request* r) {
        ridg::run_host_shot(s->solver, r->r.source, r->rec.empty() ? nullptr : r->rec.data(), r->r.nrec,
                            r->r.t_final, r->r.t_image_start, r->obs.empty() ? nullptr : r->obs.data(),
                            r->r.traces_out, r->r.image_p, r->r.image_q, r->eup.empty() ? nullptr : r->eup.data(),
                            s->buffers[0]);
      };
      std::vector<int> status(static_cast<size_t>(n), RIDG_OK);
      std::vector<std::string> error(static_cast<size_t>(n));
      auto admitted = [&](Request* r, int32_t shots) {
        admit(s, r, shots);
        work_cv.notify_all();
      };
      if (n == 1) {
        attempt([&] {
          admitted(q, 1);
          alone(q);
        }, status[0], error[0]);
      } else {
        std::vector<ridg_shot_io> io(static_cast<size_t>(n));
        for (int32_t i = 0; i < n; ++i) {
          const Request* r = batch[size_t(i)];
          io[size_t(i)] = ridg_shot_io{r->r.source, r->rec.empty() ? nullptr : r->rec.data(), r->r.nrec,
                                       r->obs.empty() ? nullptr : r->obs.data(), r->r.traces_out, r->r.image_p,
                                       r->r.image_q};
        }
        attempt([&] {
          admitted(q, n);
          ridg::run_host_shots(s->solver, n, io.data(), q->r.t_final, q->r.t_image_start,
                               q->eup.empty() ? nullptr : q->eup.data(), s->buffers);
        }, status[0], error[0]);
        // a batch that failed (one bad request, or too little memory for all of them) runs its requests
        // one by one, so that each gets its own result and status
        if (status[0] != RIDG_OK)
          for (int32_t i = 0; i < n; ++i)
            attempt([&] {
              admitted(batch[size_t(i)], 1);
              alone(batch[size_t(i)]);
            }, status[size_t(i)], error[size_t(i)]);
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        const auto now = clock::now();
        for (int32_t i = 0; i < n; ++i) {
          Request* r = batch[size_t(i)];
          r->status = status[size_t(i)];
          r->error = error[size_t(i)];
          r->finished = now;
          r->done = true;
        }
        s->busy = false;
        finished_shots += n;
      }
      done_cv.notify_all();
      work_cv.notify_all();
    }
  }

  void start(int64_t max_q) {
    max_queued = max_q;
    RIDG_CUDA(cudaGetDevice(&device));
    for (size_t i = 0; i < slots.size(); ++i) {
      Slot* s = slots[i].get();
      s->worker = std::thread([this, s, i] { run(s, int64_t(i)); });
    }
  }
};

extern "C" {

const char* ridg_last_error(void) { return ridg::g_last_error.c_str(); }
const char* ridg_version(void) { return "ridg-gb300 0.1 (sm_103a)"; }

int ridg_mesh_create(const double* xyz, int64_t n_vert, const int64_t* tet, int64_t K, const int8_t* face_bc,
                     int8_t default_bc, ridg_mesh** out) {
  return guarded([&] {
    if (!out) throw Error{RIDG_E_INVALID_ARG, "out is null"};
    *out = nullptr;
    auto m = std::make_unique<ridg_mesh>();
    m->m = ridg::build_mesh(xyz, n_vert, tet, K, face_bc, default_bc);
    // reject inverted or degenerate elements here already
    ridg::build_geometry(m->m);
    *out = m.release();
  });
}

void ridg_mesh_destroy(ridg_mesh* mesh) { delete mesh; }

int ridg_mesh_counts(const ridg_mesh* mesh, int64_t* nb, int64_t* ni) {
  return guarded([&] {
    if (!mesh) throw Error{RIDG_E_INVALID_ARG, "mesh is null"};
    if (nb) *nb = mesh->m.n_boundary;
    if (ni) *ni = mesh->m.n_interior;
  });
}

int ridg_mesh_locate(ridg_mesh* mesh, const double* xyz, int64_t n, int64_t* elem_out, double* rst_out) {
  return guarded([&] {
    if (!mesh || (n > 0 && (!xyz || !elem_out))) throw Error{RIDG_E_INVALID_ARG, "null argument"};
    if (n < 0) throw Error{RIDG_E_INVALID_ARG, "n must be >= 0"};
    if (!mesh->loc) mesh->loc = std::make_unique<ridg::PointLocator>(ridg::build_locator(mesh->m));
    for (int64_t i = 0; i < n; ++i) {
      double rst[3] = {0, 0, 0};
      elem_out[i] = ridg::locate_point(mesh->m, *mesh->loc, xyz + 3 * i, rst);
      if (rst_out)
        for (int d = 0; d < 3; ++d) rst_out[3 * i + d] = rst[d];
    }
  });
}

int ridg_reference_operators(int N, double* rst, double* D, double* M, double* LIFT, int32_t* fmask) {
  return guarded([&] {
    ridg::RefElem re = ridg::build_reference(N);
    int Np = re.Np, Nfp = re.Nfp;
    if (rst)
      for (int n = 0; n < Np; ++n)
        for (int d = 0; d < 3; ++d) rst[3 * n + d] = re.rst[n][d];
    if (D)
      for (int j = 0; j < 3; ++j)
        for (int a = 0; a < Np; ++a)
          for (int b = 0; b < Np; ++b) D[(j * Np + a) * Np + b] = re.D[j](a, b);
    if (M) std::memcpy(M, re.M.a.data(), sizeof(double) * Np * Np);
    if (LIFT) std::memcpy(LIFT, re.LIFT.a.data(), sizeof(double) * Np * 4 * Nfp);
    if (fmask)
      for (int f = 0; f < 4; ++f)
        for (int j = 0; j < Nfp; ++j) fmask[f * Nfp + j] = re.fmask[f][j];
  });
}

int ridg_solver_create(const ridg_mesh* mesh, int N, const double* c, const double* rho, const ridg_options* opt,
                       uintptr_t cuda_stream, ridg_solver** out) {
  return guarded([&] {
    if (!out) throw Error{RIDG_E_INVALID_ARG, "out is null"};
    *out = nullptr;
    if (!mesh || !c || !rho) throw Error{RIDG_E_INVALID_ARG, "null mesh, c or rho"};
    ridg_options o{};
    if (opt) o = *opt;
    if (o.dtype != RIDG_F32 && o.dtype != RIDG_F64) throw Error{RIDG_E_INVALID_ARG, "dtype must be RIDG_F32 or RIDG_F64"};
    if (N < 1 || N > 6) throw Error{RIDG_E_INVALID_ARG, "order N must be in 1..6"};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) throw Error{RIDG_E_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e)};
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    if (o.dtype == RIDG_F32)
      *out = new ridg::Engine<float>(mesh->m, N, c, rho, o, st);
    else
      *out = new ridg::Engine<double>(mesh->m, N, c, rho, o, st);
  });
}

void ridg_solver_destroy(ridg_solver* s) {
  if (s) {
    cudaStreamSynchronize(s->stream());
    delete s;
  }
}

#define RIDG_NEED(s)                                                      \
  if (!(s)) throw Error{RIDG_E_INVALID_ARG, "solver handle is null"};

int ridg_solver_info(const ridg_solver* s, ridg_info* info) {
  return guarded([&] {
    RIDG_NEED(s);
    if (!info) throw Error{RIDG_E_INVALID_ARG, "info is null"};
    s->info(info);
  });
}
int ridg_solver_levels(const ridg_solver* s, int32_t* levels) {
  return guarded([&] {
    RIDG_NEED(s);
    if (!levels) throw Error{RIDG_E_INVALID_ARG, "levels is null"};
    s->levels(levels);
  });
}
int ridg_solver_nodes(const ridg_solver* s, double* xyz) {
  return guarded([&] {
    RIDG_NEED(s);
    if (!xyz) throw Error{RIDG_E_INVALID_ARG, "xyz is null"};
    s->nodes(xyz);
  });
}
int ridg_set_state(ridg_solver* s, const double* q) {
  return guarded([&] {
    RIDG_NEED(s);
    if (!q) throw Error{RIDG_E_INVALID_ARG, "q is null"};
    s->set_state(q);
  });
}
int ridg_set_history(ridg_solver* s, const double* r1, const double* r2) {
  return guarded([&] {
    RIDG_NEED(s);
    s->set_history(r1, r2);
  });
}
int ridg_eval_rhs(ridg_solver* s, const double* q, double* out) {
  return guarded([&] {
    RIDG_NEED(s);
    if (!q || !out) throw Error{RIDG_E_INVALID_ARG, "null buffer"};
    s->eval_rhs(q, out);
  });
}
int ridg_step(ridg_solver* s, int64_t n) {
  return guarded([&] {
    RIDG_NEED(s);
    s->step(n);
  });
}
int ridg_get_state(ridg_solver* s, double* q) {
  return guarded([&] {
    RIDG_NEED(s);
    if (!q) throw Error{RIDG_E_INVALID_ARG, "q is null"};
    s->get_state(q);
  });
}
int ridg_energy(ridg_solver* s, double* e) {
  return guarded([&] {
    RIDG_NEED(s);
    if (!e) throw Error{RIDG_E_INVALID_ARG, "energy is null"};
    *e = s->energy();
  });
}
int ridg_energy_noalloc(ridg_solver* s, double* energy_dev) {
  return guarded([&] {
    RIDG_NEED(s);
    if (!energy_dev) throw Error{RIDG_E_INVALID_ARG, "energy_dev is null"};
    s->energy_noalloc(energy_dev);
  });
}

int64_t ridg_trace_len(const ridg_solver* s, double t_final) {
  if (!s || !(t_final > 0.0)) return 0;
  return s->trace_len(t_final);
}

int ridg_rtm_shot_device(ridg_solver* s, const ridg_source* src, const double* rec_xyz, int64_t nrec, double t_final,
                         double t_image_start, const double* observed_dev, double* traces_dev, double* image_p_dev,
                         double* image_q_dev, const double* e_up) {
  return guarded([&] {
    RIDG_NEED(s);
    if (!src) throw Error{RIDG_E_INVALID_ARG, "source is null"};
    s->shot(*src, rec_xyz, nrec, t_final, t_image_start, observed_dev, traces_dev, image_p_dev, image_q_dev, e_up);
  });
}

int ridg_rtm_shot(ridg_solver* s, const ridg_source* src, const double* rec_xyz, int64_t nrec, double t_final,
                  double t_image_start, const double* observed, double* traces_out, double* image_p, double* image_q,
                  const double* e_up) {
  return guarded([&] {
    RIDG_NEED(s);
    if (!src) throw Error{RIDG_E_INVALID_ARG, "source is null"};
    ridg::HostShotBuffers b;
    ridg::run_host_shot(s, *src, rec_xyz, nrec, t_final, t_image_start, observed, traces_out, image_p, image_q, e_up,
                        b);
  });
}

int ridg_rtm_shots_device(ridg_solver* s, int32_t n_shots, const ridg_shot_io* shots, double t_final,
                          double t_image_start, const double* e_up) {
  return guarded([&] {
    RIDG_NEED(s);
    if (n_shots < 1 || n_shots > RIDG_MAX_BATCH || !shots)
      throw Error{RIDG_E_INVALID_ARG, "n_shots must be in 1.." + std::to_string(RIDG_MAX_BATCH)};
    s->shots(n_shots, shots, t_final, t_image_start, e_up);
  });
}

int ridg_rtm_shots(ridg_solver* s, int32_t n_shots, const ridg_shot_io* shots, double t_final, double t_image_start,
                   const double* e_up) {
  return guarded([&] {
    RIDG_NEED(s);
    if (n_shots < 1 || n_shots > RIDG_MAX_BATCH || !shots)
      throw Error{RIDG_E_INVALID_ARG, "n_shots must be in 1.." + std::to_string(RIDG_MAX_BATCH)};
    std::vector<ridg::HostShotBuffers> b(static_cast<size_t>(n_shots));
    ridg::run_host_shots(s, n_shots, shots, t_final, t_image_start, e_up, b.data());
  });
}

int ridg_last_shot_stats(const ridg_solver* s, ridg_shot_stats* stats) {
  return guarded([&] {
    RIDG_NEED(s);
    if (!stats) throw Error{RIDG_E_INVALID_ARG, "stats is null"};
    *stats = const_cast<ridg_solver*>(s)->stats();
  });
}

int ridg_set_graph_replay(ridg_solver* s, int32_t on) {
  return guarded([&] {
    RIDG_NEED(s);
    s->set_graph_replay(on != 0);
  });
}

int ridg_set_profiling(ridg_solver* s, int32_t every) {
  return guarded([&] {
    RIDG_NEED(s);
    s->set_profiling(every);
  });
}

int ridg_set_trace_budget(ridg_solver* s, int64_t device_bytes) {
  return guarded([&] {
    RIDG_NEED(s);
    s->set_trace_budget(device_bytes);
  });
}

int ridg_forward(ridg_solver* s, const ridg_source* src, const double* rec_xyz, int64_t nrec, double t_final,
                 double* traces_out) {
  return guarded([&] {
    RIDG_NEED(s);
    if (!src) throw Error{RIDG_E_INVALID_ARG, "source is null"};
    const int64_t n_t = s->trace_len(t_final);
    ridg::DBuf tr;
    tr.alloc(size_t(std::max<int64_t>(nrec, 1)) * n_t * sizeof(double));
    s->forward(*src, rec_xyz, nrec, t_final, ridg::dptr<double>(tr));
    if (traces_out && nrec > 0)
      RIDG_CUDA(cudaMemcpyAsync(traces_out, tr.p, size_t(nrec) * n_t * sizeof(double), cudaMemcpyDeviceToHost,
                                s->stream()));
    RIDG_CUDA(cudaStreamSynchronize(s->stream()));
  });
}

int ridg_set_state_device(ridg_solver* s, const double* q_dev) {
  return guarded([&] {
    RIDG_NEED(s);
    s->set_state_device(q_dev);
  });
}

int ridg_get_state_device(ridg_solver* s, double* q_dev) {
  return guarded([&] {
    RIDG_NEED(s);
    s->get_state_device(q_dev);
  });
}

int ridg_set_velocity(ridg_solver* s, const double* c) {
  return guarded([&] {
    RIDG_NEED(s);
    s->set_velocity(c);
  });
}

int ridg_eval_adjoint_rhs(ridg_solver* s, const double* lam, double* out) {
  return guarded([&] {
    RIDG_NEED(s);
    s->eval_adjoint_rhs(lam, out);
  });
}

int ridg_misfit_forward(ridg_solver* s, const ridg_source* src, const double* rec_xyz, int64_t nrec, double t_final,
                        const double* observed, int32_t n_checkpoints, double* misfit, double* traces_out) {
  return guarded([&] {
    RIDG_NEED(s);
    if (!src || !misfit) throw Error{RIDG_E_INVALID_ARG, "null source or misfit"};
    *misfit = s->misfit_forward(*src, rec_xyz, nrec, t_final, observed, n_checkpoints, traces_out);
  });
}

int ridg_misfit_backward(ridg_solver* s, double* grad) {
  return guarded([&] {
    RIDG_NEED(s);
    s->misfit_backward(grad);
  });
}

int ridg_server_create(ridg_solver* s, int64_t max_queued, ridg_server** out) {
  return ridg_server_create_slots(&s, nullptr, 1, max_queued, out);
}

int ridg_server_create_slots(ridg_solver* const* solvers, const int32_t* models, int64_t n_slots, int64_t max_queued,
                             ridg_server** out) {
  return guarded([&] {
    if (!out) throw Error{RIDG_E_INVALID_ARG, "out is null"};
    *out = nullptr;
    if (!solvers || n_slots < 1) throw Error{RIDG_E_INVALID_ARG, "a server needs at least one solver"};
    if (max_queued < 1) throw Error{RIDG_E_INVALID_ARG, "max_queued must be >= 1"};
    auto sv = std::make_unique<ridg_server>();
    std::map<int32_t, ridg_info> model_info;
    for (int64_t i = 0; i < n_slots; ++i) {
      ridg_solver* s = solvers[i];
      RIDG_NEED(s);
      const int32_t m = models ? models[i] : 0;
      if (m < 0) throw Error{RIDG_E_INVALID_ARG, "model numbers must be >= 0"};
      for (int64_t j = 0; j < i; ++j)
        if (solvers[j] == s) throw Error{RIDG_E_INVALID_ARG, "a solver appears twice among the slots"};
      ridg_info inf;
      s->info(&inf);
      auto it = model_info.find(m);
      if (it == model_info.end()) {
        model_info[m] = inf;
      } else if (it->second.K != inf.K || it->second.N != inf.N || it->second.n_levels != inf.n_levels ||
                 it->second.dt_local != inf.dt_local) {
        throw Error{RIDG_E_INVALID_ARG, "solvers of model " + std::to_string(m) + " differ in K, N or time step"};
      }
      auto slot = std::make_unique<ridg_server::Slot>();
      slot->solver = s;
      slot->model = m;
      sv->slots.push_back(std::move(slot));
    }
    sv->start(max_queued);
    *out = sv.release();
  });
}

int ridg_server_submit(ridg_server* sv, const ridg_shot_request* req, int64_t* ticket) {
  return guarded([&] {
    if (!sv || !req || !ticket) throw Error{RIDG_E_INVALID_ARG, "null argument"};
    if (!(req->t_final > 0.0) || !(req->t_image_start >= 0.0)) throw Error{RIDG_E_INVALID_ARG, "bad time span"};
    if (req->nrec < 0 || (req->nrec > 0 && !req->rec_xyz)) throw Error{RIDG_E_INVALID_ARG, "bad receiver list"};
    if (!sv->serves(req->model)) throw Error{RIDG_E_INVALID_ARG, "no slot serves model " + std::to_string(req->model)};
    ridg_solver* model_solver = nullptr;
    for (const auto& sl : sv->slots)
      if (sl->model == req->model) model_solver = sl->solver;
    auto q = std::make_unique<ridg_server::Request>();
    q->r = *req;
    q->rec.assign(req->rec_xyz, req->rec_xyz + 3 * req->nrec);
    if (req->observed) {
      const int64_t n_t = model_solver->trace_len(req->t_final);
      q->obs.assign(req->observed, req->observed + req->nrec * n_t);
    }
    if (req->e_up) q->eup.assign(req->e_up, req->e_up + 3);
    if (req->source.kind == RIDG_SRC_SAMPLED && req->source.samples && req->source.n_samples > 0) {
      q->samples.assign(req->source.samples, req->source.samples + req->source.n_samples);
      q->r.source.samples = q->samples.data();
    }
    q->submitted = ridg_server::clock::now();
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      if (int64_t(sv->queue.size()) >= sv->max_queued)
        throw Error{RIDG_E_BUSY, "server queue full (" + std::to_string(sv->max_queued) + " waiting)"};
      const int64_t t = sv->next_ticket++;
      sv->requests[t] = std::move(q);
      sv->queue.push_back(t);
      *ticket = t;
    }
    sv->work_cv.notify_all();
  });
}

int ridg_server_set_batch(ridg_server* sv, int32_t max_batch) {
  return guarded([&] {
    if (!sv) throw Error{RIDG_E_INVALID_ARG, "server handle is null"};
    if (max_batch < 1 || max_batch > RIDG_MAX_BATCH)
      throw Error{RIDG_E_INVALID_ARG, "max_batch must be in 1.." + std::to_string(RIDG_MAX_BATCH)};
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->max_batch = max_batch;
    }
    sv->work_cv.notify_all();
  });
}

int ridg_server_wait(ridg_server* sv, int64_t ticket, double timeout_s, ridg_request_timing* timing) {
  int status = RIDG_OK;
  std::string error;
  int rc = guarded([&] {
    if (!sv) throw Error{RIDG_E_INVALID_ARG, "server handle is null"};
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->requests.find(ticket);
    if (it == sv->requests.end()) throw Error{RIDG_E_INVALID_ARG, "unknown ticket " + std::to_string(ticket)};
    ridg_server::Request* q = it->second.get();
    auto ready = [&] { return q->done; };
    if (timeout_s < 0) {
      sv->done_cv.wait(lk, ready);
    } else if (!sv->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
      throw Error{RIDG_E_TIMEOUT, "request " + std::to_string(ticket) + " has not completed"};
    }
    if (timing) {
      using sec = std::chrono::duration<double>;
      timing->queued_s = sec(q->started - q->submitted).count();
      timing->run_s = sec(q->finished - q->started).count();
      timing->total_s = sec(q->finished - q->submitted).count();
      timing->start_s = sec(q->started - sv->created).count();
      timing->end_s = sec(q->finished - sv->created).count();
      timing->slot = q->slot;
    }
    status = q->status;
    error = q->error;
    sv->requests.erase(it);
  });
  if (rc != RIDG_OK) return rc;
  if (status != RIDG_OK) ridg::set_error(error);
  return status;
}

int ridg_server_destroy(ridg_server* sv) {
  return guarded([&] {
    if (!sv) throw Error{RIDG_E_INVALID_ARG, "server handle is null"};
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->stop = true;
      sv->queue.clear();
    }
    sv->work_cv.notify_all();
    sv->done_cv.notify_all();
    for (auto& sl : sv->slots)
      if (sl->worker.joinable()) sl->worker.join();
    delete sv;
  });
}


int ridg_partition(const ridg_mesh* mesh, int N, const double* c, const ridg_options* opt, int32_t n_parts,
                   int32_t* part_out) {
  return guarded([&] {
    if (!mesh || !c || !part_out) throw Error{RIDG_E_INVALID_ARG, "null mesh, c or part_out"};
    if (N < 1 || N > 6) throw Error{RIDG_E_INVALID_ARG, "order N must be in 1..6"};
    if (n_parts < 1 || n_parts > RIDG_MAX_PARTS) throw Error{RIDG_E_INVALID_ARG, "n_parts must be in 1..64"};
    for (int64_t k = 0; k < mesh->m.K; ++k)
      if (!(c[k] > 0.0) || !std::isfinite(c[k])) throw Error{RIDG_E_INVALID_ARG, "c must be positive and finite"};
    ridg_options o{};
    if (opt) o = *opt;
    const double cfl = o.cfl > 0 ? o.cfl : 0.15;
    const int nlm = o.n_levels_max > 0 ? o.n_levels_max : 3;
    if (nlm > ridg::kMaxLevels) throw Error{RIDG_E_INVALID_ARG, "n_levels_max too large"};
    const ridg::Geometry geo = ridg::build_geometry(mesh->m);
    const ridg::Levels lv = ridg::assign_levels(mesh->m, geo, N, c, cfl, nlm);
    const std::vector<int32_t> part = ridg::partition_mesh(mesh->m, lv, n_parts);
    std::copy(part.begin(), part.end(), part_out);
  });
}

int ridg_group_create(const ridg_mesh* mesh, int N, const double* c, const double* rho, const ridg_options* opt,
                      const int32_t* part, int32_t n_parts, const int32_t* devices, ridg_group** out) {
  return guarded([&] {
    if (!out) throw Error{RIDG_E_INVALID_ARG, "out is null"};
    *out = nullptr;
    if (!mesh || !c || !rho || !part) throw Error{RIDG_E_INVALID_ARG, "null mesh, c, rho or part"};
    ridg_options o{};
    if (opt) o = *opt;
    if (o.dtype != RIDG_F32 && o.dtype != RIDG_F64) throw Error{RIDG_E_INVALID_ARG, "dtype must be RIDG_F32 or RIDG_F64"};
    if (N < 1 || N > 6) throw Error{RIDG_E_INVALID_ARG, "order N must be in 1..6"};
    if (o.dtype == RIDG_F32)
      *out = new ridg::Group<float>(mesh->m, N, c, rho, o, part, n_parts, devices);
    else
      *out = new ridg::Group<double>(mesh->m, N, c, rho, o, part, n_parts, devices);
  });
}

int ridg_group_rtm_shot(ridg_group* g, const ridg_source* src, const double* rec_xyz, int64_t nrec, double t_final,
                        double t_image_start, const double* observed, double* traces_out, double* image_p,
                        double* image_q, const double* e_up) {
  return guarded([&] {
    if (!g || !src) throw Error{RIDG_E_INVALID_ARG, "null group or source"};
    g->shot(*src, rec_xyz, nrec, t_final, t_image_start, observed, traces_out, image_p, image_q, e_up);
  });
}

int ridg_group_info_get(const ridg_group* g, ridg_group_info* out) {
  return guarded([&] {
    if (!g || !out) throw Error{RIDG_E_INVALID_ARG, "null group or out"};
    g->info(out);
  });
}

int64_t ridg_group_trace_len(const ridg_group* g, double t_final, int32_t* np_out) {
  return g ? g->trace_len(t_final, np_out) : -1;
}

void ridg_group_destroy(ridg_group* g) { delete g; }

int ridg_inject_fault(const char* point, int64_t after) {
  return guarded([&] {
    const int k = point ? ridg::fault_point_of(point) : -1;
    if (k < 0) throw Error{RIDG_E_INVALID_ARG, "unknown failure point"};
    if (after < 0) throw Error{RIDG_E_INVALID_ARG, "after must be >= 0"};
    ridg::g_fault.point.store(ridg::kFaultNone);
    ridg::g_fault.after.store(after);
    ridg::g_fault.point.store(k);
  });
}

int ridg_fault_armed(void) { return ridg::g_fault.point.load(); }

}  // extern "C"
