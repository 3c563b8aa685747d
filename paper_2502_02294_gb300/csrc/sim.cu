// Simulation handle: one time step of the coupled DM + gas + subgrid system, checkpointed
// runs and their reverse-mode derivative (arXiv 2502.02294, Secs. 2.1-2.4 and 2.3.5).
//
// Step i (a_i -> a_{i+1}), the same kick-drift-kick for DM and gas:
//   1 half kick with g(a_i) (K1) and DM drift (dtau)        [kick_drift, gas_kick]
//   2 three relaxing-TVD sweeps in the Strang order (i mod 6) [sweep x3]
//   3 subgrid at a_{i+1} with the Philox draws of step i      [subgrid]
//   4 CIC deposit + spectral Poisson -> g(a_{i+1})             [deposit, fix, r2c, green, c2r]
//   5 half kick with g(a_{i+1}) (K2)                           [kick_drift, gas_kick]
// The reverse pass recomputes each checkpoint segment forward, recording the inputs of
// every stage (the tape), then applies the hand-written adjoint of each stage in reverse
// order. The adjoint of g(a_i) seen by the first kick of step i is carried into step i-1,
// whose force stage produced it, so each force adjoint runs once per step. Scalar
// parameter partials are reduced per step on the device and chained through the FP64
// schedule derivatives by a small device kernel, so neither pass synchronises the host.
//
// With graphs enabled (sim_set_graphs), sim_run and sim_run_adjoint are captured once per
// argument set into CUDA graphs on a private stream and replayed on the caller's stream;
// the handle's host-side bookkeeping (step counter, ping-pong buffers, checkpoint list) is
// restored to what the captured call produced.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "closure.cuh"
#include "diag.cuh"
#include "fli.cuh"
#include "ics.cuh"
#include "pm.cuh"
#include "schedule.h"
#include "subgrid.cuh"

namespace dh {

// ------------------------------------------------------------------ errors
static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

const char* get_error() { return g_err; }

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// kick_g (may be NULL): the sweep first applies the gravity half kick K of force kick_g to
// every cell it loads (only where sweep_takes_kick says the form can)
sim_status launch_sweep(int axis, const float* uin, float* uout, int n, SArg nu, double gam,
                        double eps, int B, int variant, cudaStream_t st,
                        const float* kick_g = nullptr, SArg kick_K = SArg{0.0f, nullptr});
bool sweep_takes_kick(int axis, int n, int variant, const float* uin, const float* uout);
sim_status launch_sweep_adjoint(int axis, const float* uin, const float* lout, float* lin,
                                int n, SArg nu, double gam, double eps, DPart dnu,
                                float* scratch, int B, int variant, cudaStream_t st);
sim_status prepare_sweep_kernels();

static const char* kOrders[6] = {"xyz", "zyx", "zxy", "yxz", "yzx", "xzy"};

// per-step partial sums of the reverse pass (doubles on the device), and the chain-rule
// coefficient of each with respect to Omega_m
// SL_DKM: the merged kick K2_{i-1} + K1_i that opens step i inside a checkpoint segment
enum { SL_DK1 = 0, SL_DK2, SL_DNU, SL_DDTAU, SL_DPREF, SL_DCM, SL_DFB, SL_DKM, SL_N = 8 };
// extra global partials after the SIM_NPARAMS subgrid ones (per instance: NG doubles)
enum { GX_DRP = 0, GX_DFB_IC = 1, GX_LAMC = 2, GX_N = 8 };
constexpr int NG = SIM_NPARAMS + GX_N;
// per-step float constants of every instance (device table [n_steps][SC_N][B])
enum { SC_K1 = 0, SC_K2, SC_DTAU, SC_NU, SC_PN1, SC_KM, SC_N };
// per-instance chain-rule constants of the parameter derivatives (device [B][PCH_N])
enum { PCH_CCM0 = 0, PCH_DLNC, PCH_DRP, PCH_DFB, PCH_INVS8, PCH_N };

// Host constants of one instance (Sec. 2.1 ICs, Sec. 2.2 mass split).
struct InstConst {
  double fb, cm, dfb_dom, C, dlnC_dom, rp, drp_dom, a2e0;
};

// One recorded step: inputs of every stage (pointers into the tape allocation).
struct TapeSlot {
  float *U0, *Uk1, *Us1, *Us2, *Us3, *Usg;  // 5 n^3 each
  float *s0, *p0, *g0, *s1, *g1;            // 3 n^3 each
  float* gd;                                 // n^3: the step's Gumbel difference g0 - g1
};
constexpr int kTapeFloatsPerCell = 6 * 5 + 5 * 3 + 1;

// Host-side state that a call changes; a replayed graph must start from and end in the
// same values as the captured call.
struct HostState {
  int step, init_step, prev_step, ckpt_count, tape_first, tape_end;
  bool ics_valid;
  bool taped;  // a tape to record on exists (read, not restored: a run records only then)
  float *gas, *gas2, *w_gas, *w_gas2, *lam_gas, *lam_tmp, *lamG0, *lamG1;
  std::vector<int> ckpt_step;
  bool operator==(const HostState& o) const {
    return step == o.step && init_step == o.init_step && prev_step == o.prev_step &&
           ckpt_count == o.ckpt_count && tape_first == o.tape_first &&
           tape_end == o.tape_end && ics_valid == o.ics_valid && taped == o.taped && gas == o.gas &&
           gas2 == o.gas2 && w_gas == o.w_gas && w_gas2 == o.w_gas2 && lam_gas == o.lam_gas &&
           lam_tmp == o.lam_tmp && lamG0 == o.lamG0 && lamG1 == o.lamG1 &&
           std::vector<int>(ckpt_step.begin(), ckpt_step.begin() + ckpt_count) ==
               std::vector<int>(o.ckpt_step.begin(), o.ckpt_step.begin() + o.ckpt_count);
  }
};

struct GraphEntry {
  int kind = 0;
  std::vector<uintptr_t> key;
  HostState before, after;
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;
};

}  // namespace dh

using namespace dh;

struct sim_s {
  sim_params prm;                // instance 0; the fields shared by all instances
  std::vector<sim_params> prms;  // per instance
  int B = 1;
  int n = 0;
  long long N3 = 0, NC = 0;
  cudaStream_t st = 0;
  double dx = 0, inv_dx = 0;
  std::vector<StepFactors> sched;               // instance 0 (the a_i are shared)
  std::vector<std::vector<StepFactors>> scheds;  // per instance
  std::vector<InstConst> inst;                   // per instance
  FFTPlans plans;   // batch B: the step's transforms
  FFTPlans plans1;  // batch 1: initial conditions (created when B > 1)
  // device tables of the per-instance constants (uploaded once by sim_init)
  float* d_sc = nullptr;            // [n_steps][SC_N][B]
  std::vector<float> h_sc, h_pn;    // host copies (a single instance passes values)
  std::vector<SubgridConst> h_sub;
  float* d_pn = nullptr;            // [n_steps + 1][B] Poisson factor / n^3 at a_i
  float* d_cm = nullptr;            // [B] DM mass per particle (1 - f_b)
  SubgridConst* d_sub = nullptr;    // [n_steps][B]
  double* d_pch = nullptr;          // [B][PCH_N] chain-rule constants of the parameters
  double* d_cpref = nullptr;        // [n_steps + 1][B] chain coefficient of a flush slot
  sim_closure_t* closure = nullptr;  // learned correction after every step (not owned)
  uint64_t closure_gen = 0;
  int fwd_var[3] = {SIM_SWEEP_DEFAULT, SIM_SWEEP_DEFAULT, SIM_SWEEP_DEFAULT};
  int adj_var[3] = {SIM_SWEEP_DEFAULT, SIM_SWEEP_DEFAULT, SIM_SWEEP_DEFAULT};
  // state (B instances one after another in every buffer)
  float *gas = nullptr, *gas2 = nullptr, *s = nullptr, *p = nullptr, *g = nullptr;
  float *star = nullptr, *aux = nullptr, *zhat = nullptr, *delta = nullptr;
  uint32_t* events = nullptr;
  unsigned long long* acc = nullptr;
  cufftComplex* ck = nullptr;  // max(4 B, 5) NC complex scratch
  float *noise = nullptr, *f4 = nullptr;
  float *init_gas = nullptr, *init_part = nullptr;
  float *prev_gas = nullptr, *prev_part = nullptr;
  int prev_step = -1;
  bool ics_valid = false;
  int init_step = 0;
  int step = 0;
  // checkpoints: a pool of buffers (11 n^3 floats per instance) allocated on first use
  std::vector<float*> ckpt_pool;
  std::vector<int> ckpt_step;
  int ckpt_count = 0;
  // tape and adjoint scratch (allocated on first use)
  float* tape = nullptr;
  int tape_cap = 0;
  // steps [tape_first, tape_end) of the last run, recorded on the tape by the run itself
  // (its last checkpoint segment), or -1: the reverse pass then needs no recompute of it
  int tape_first = -1, tape_end = -1;
  // checkpoint segments a run records at its end (sim_set_tape_recording; -1: all of them)
  int tape_segments = 1;
  float *w_gas = nullptr, *w_gas2 = nullptr, *w_s = nullptr, *w_p = nullptr, *w_g = nullptr;
  float *lam_gas = nullptr, *lam_tmp = nullptr, *lam_s = nullptr, *lam_p = nullptr;
  float *lamG0 = nullptr, *lamG1 = nullptr, *lam_delta = nullptr, *lam4 = nullptr;
  float* lam_scr = nullptr;  // 20 n^3 per instance, scratch of the marching sweep adjoints
  double* dslots = nullptr;  // [n_steps + 2][B][SL_N]
  double* dcoef = nullptr;   // [n_steps][B][SL_N] chain-rule coefficients
  double* dglob = nullptr;   // [B][NG]
  // per-step diagnostics: records [n_steps + 1][B] (allocated by sim_set_diagnostics)
  bool diag_on = false;
  double* d_diag_sums = nullptr;  // [n_steps + 1][B][DG_NSUM]
  int* d_diag_mins = nullptr;     // [n_steps + 1][B][2]
  std::vector<char> diag_recorded;
  // field-level inference (allocated on the first sim_fli_step)
  float *fli_g = nullptr, *fli_dL = nullptr;  // B n^3 data-term gradient; B 5 n^3 dL/dgas
  double* fli_dpar = nullptr;                 // B x SIM_NPARAMS
  unsigned int* speed_bits = nullptr;  // [B]
  // optional per-class kernel timing: event pairs around each timed launch (eager runs only)
  bool kt_on = false;
  std::vector<cudaEvent_t> kt_ev;  // 2 per recorded launch
  std::vector<int> kt_cls;
  size_t kt_used = 0;
  long long kt_dropped = 0;
  // graphs
  bool graphs = false;
  cudaStream_t cap_stream = nullptr;
  std::vector<GraphEntry> graph_cache;
  std::vector<void*> allocs;
  std::string err;
};

namespace dh {

static sim_status fail(sim_t* h, sim_status s) {
  if (h && s != SIM_OK) h->err = get_error();
  return s;
}

static sim_status dalloc(sim_t* h, void** ptr, size_t bytes) {
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    set_error("cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    return SIM_ENOMEM;
  }
  h->allocs.push_back(*ptr);
  return SIM_OK;
}

template <class T>
static sim_status dalloc_t(sim_t* h, T** ptr, size_t count) {
  return dalloc(h, (void**)ptr, count * sizeof(T));
}

static sim_status dcopy(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  DH_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st));
  return SIM_OK;
}

static sim_status dzero(void* dst, size_t bytes, cudaStream_t st) {
  DH_CUDA_TRY(cudaMemsetAsync(dst, 0, bytes, st));
  return SIM_OK;
}

static HostState snapshot(const sim_t* h) {
  HostState s;
  s.step = h->step;
  s.init_step = h->init_step;
  s.prev_step = h->prev_step;
  s.ckpt_count = h->ckpt_count;
  s.tape_first = h->tape_first;
  s.tape_end = h->tape_end;
  s.ics_valid = h->ics_valid;
  s.taped = h->tape != nullptr;
  s.gas = h->gas;
  s.gas2 = h->gas2;
  s.w_gas = h->w_gas;
  s.w_gas2 = h->w_gas2;
  s.lam_gas = h->lam_gas;
  s.lam_tmp = h->lam_tmp;
  s.lamG0 = h->lamG0;
  s.lamG1 = h->lamG1;
  s.ckpt_step = h->ckpt_step;
  return s;
}

static void restore(sim_t* h, const HostState& s) {
  h->step = s.step;
  h->init_step = s.init_step;
  h->prev_step = s.prev_step;
  h->ckpt_count = s.ckpt_count;
  h->tape_first = s.tape_first;
  h->tape_end = s.tape_end;
  h->ics_valid = s.ics_valid;
  h->gas = s.gas;
  h->gas2 = s.gas2;
  h->w_gas = s.w_gas;
  h->w_gas2 = s.w_gas2;
  h->lam_gas = s.lam_gas;
  h->lam_tmp = s.lam_tmp;
  h->lamG0 = s.lamG0;
  h->lamG1 = s.lamG1;
  h->ckpt_step = s.ckpt_step;
}

// Run `body` directly, or (graphs on) replay the graph captured for (kind, key) from the
// same host state, capturing it first if there is none.
template <class Body>
static sim_status run_maybe_graph(sim_t* h, int kind, const std::vector<uintptr_t>& key,
                                  Body body) {
  if (!h->graphs || h->kt_on) return body();
  const HostState before = snapshot(h);
  for (GraphEntry& e : h->graph_cache) {
    if (e.kind == kind && e.key == key && e.before == before) {
      DH_CUDA_TRY(cudaGraphLaunch(e.exec, h->st));
      restore(h, e.after);
      g_launches.fetch_add(e.launches, std::memory_order_relaxed);
      return SIM_OK;
    }
  }
  // capture on the private stream, ordered after the caller's stream
  cudaEvent_t ev;
  DH_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaStream_t user = h->st;
  cudaError_t ce = cudaEventRecord(ev, user);
  if (ce == cudaSuccess) ce = cudaStreamWaitEvent(h->cap_stream, ev, 0);
  cudaEventDestroy(ev);
  if (ce != cudaSuccess) {
    set_error("graph capture setup failed: %s", cudaGetErrorString(ce));
    return SIM_ECUDA;
  }
  DH_CUDA_TRY(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  h->st = h->cap_stream;
  const long long l0 = g_launches.load();
  sim_status r = body();
  h->st = user;
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(h->cap_stream, &graph);
  if (r != SIM_OK || ee != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    restore(h, before);
    if (r == SIM_OK) set_error("graph capture failed: %s", cudaGetErrorString(ee));
    return r != SIM_OK ? r : SIM_ECUDA;
  }
  GraphEntry e;
  e.kind = kind;
  e.key = key;
  e.before = before;
  e.after = snapshot(h);
  e.launches = g_launches.load() - l0;
  ce = cudaGraphInstantiate(&e.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    restore(h, before);
    set_error("cudaGraphInstantiate failed: %s", cudaGetErrorString(ce));
    return SIM_ECUDA;
  }
  // the captured call's work has not run yet: run it now
  ce = cudaGraphLaunch(e.exec, h->st);
  if (ce != cudaSuccess) {
    cudaGraphExecDestroy(e.exec);
    restore(h, before);
    set_error("cudaGraphLaunch failed: %s", cudaGetErrorString(ce));
    return SIM_ECUDA;
  }
  h->graph_cache.push_back(std::move(e));
  return SIM_OK;
}

static void clear_graphs(sim_t* h) {
  for (GraphEntry& e : h->graph_cache)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  h->graph_cache.clear();
}

// Launch through `launch`; with kernel timing on, bracket it with two events on the
// handle's stream (class `cls`). At most kKtMax launches are recorded between resets.
static constexpr size_t kKtMax = 8192;
template <class Launch>
static sim_status timed(sim_t* h, int cls, Launch launch) {
  if (!h->kt_on) return launch();
  if (h->kt_used >= kKtMax) {
    ++h->kt_dropped;
    return launch();
  }
  if (2 * h->kt_used + 2 > h->kt_ev.size()) {
    for (int k = 0; k < 2; ++k) {
      cudaEvent_t e;
      DH_CUDA_TRY(cudaEventCreate(&e));
      h->kt_ev.push_back(e);
    }
    h->kt_cls.push_back(cls);
  }
  h->kt_cls[h->kt_used] = cls;
  DH_CUDA_TRY(cudaEventRecord(h->kt_ev[2 * h->kt_used], h->st));
  DH_TRY(launch());
  DH_CUDA_TRY(cudaEventRecord(h->kt_ev[2 * h->kt_used + 1], h->st));
  ++h->kt_used;
  return SIM_OK;
}

static sim_status validate(const sim_params* p) {
  if (!p) {
    set_error("null parameter block");
    return SIM_EINVAL;
  }
  if (p->n < 4 || p->n > 1024) {
    set_error("n must be in [4, 1024] (got %d)", p->n);
    return SIM_EINVAL;
  }
  if (p->n_steps < 1 || p->ckpt_every < 1) {
    set_error("n_steps and ckpt_every must be >= 1");
    return SIM_EINVAL;
  }
  if (!(p->box > 0) || !(p->omega_m > 0 && p->omega_m <= 1) || !(p->omega_b > 0) ||
      !(p->omega_b < p->omega_m) || !(p->gamma > 1) || !(p->mu > 0) || !(p->T_init > 0) ||
      !(p->a_start > 0) || !(p->a_end > p->a_start) || !(p->sigma8 > 0) ||
      !(p->rms_ref >= 0) || !(p->a_ref > 0) || !(p->sigma8_ref > 0) ||
      !(p->omega_m_ref > 0 && p->omega_m_ref <= 1) || !(p->kc_frac > 0) ||
      !(p->limiter_eps > 0)) {
    set_error("invalid cosmology, gas or IC parameters");
    return SIM_EINVAL;
  }
  if (p->subgrid_on && (!(p->Pi0 > 0 && p->Pi0 < 1) || !(p->tau > 0) || !(p->w_delta > 0) ||
                        !(p->w_T > 0) || !(p->T0_uv >= 0))) {
    set_error("invalid subgrid parameters (0 < Pi0 < 1, tau > 0, widths > 0, T0_uv >= 0)");
    return SIM_EINVAL;
  }
  if (p->kdk_mode != 0 && p->kdk_mode != 1) {
    set_error("kdk_mode must be 0 (FastPM) or 1 (plain)");
    return SIM_EINVAL;
  }
  return SIM_OK;
}

static double a_of_step(const sim_t* h, int i) {
  return i == 0 ? h->prm.a_start : h->sched[i - 1].a1;
}

// per-instance scalars of step i, read by the kernels from the device tables
// (one instance: the value itself, so that the kernels need no table load)
static SArg sc(const sim_t* h, int i, int field) {
  const size_t o = ((size_t)i * SC_N + field) * h->B;
  return h->B == 1 ? sarg(h->h_sc[o]) : sarg(h->d_sc + o);
}
static SArg pn_at(const sim_t* h, int i) {
  const size_t o = (size_t)i * h->B;
  return h->B == 1 ? sarg(h->h_pn[o]) : sarg(h->d_pn + o);
}
static SubArg sub_at(const sim_t* h, int i) {
  const size_t o = (size_t)i * h->B;
  return h->B == 1 ? subarg(h->h_sub[o]) : subarg(h->d_sub + o);
}
static DPart slot_part(double* slot, int field) { return dpart(slot + field, SL_N); }
static FFTPlans& ic_plans(sim_t* h) { return h->B == 1 ? h->plans : h->plans1; }

// Particle arrays: the API holds B x [s (3 n^3), p (3 n^3)]; the handle keeps s and p apart.
static sim_status part_join(float* dst6, const float* s, const float* p, const sim_t* h,
                            cudaStream_t st) {
  const size_t w = 3 * h->N3 * sizeof(float);
  DH_CUDA_TRY(cudaMemcpy2DAsync(dst6, 2 * w, s, w, w, h->B, cudaMemcpyDeviceToDevice, st));
  DH_CUDA_TRY(cudaMemcpy2DAsync((char*)dst6 + w, 2 * w, p, w, w, h->B,
                                cudaMemcpyDeviceToDevice, st));
  return SIM_OK;
}

static sim_status part_split(float* s, float* p, const float* src6, const sim_t* h,
                             cudaStream_t st) {
  const size_t w = 3 * h->N3 * sizeof(float);
  DH_CUDA_TRY(cudaMemcpy2DAsync(s, w, src6, 2 * w, w, h->B, cudaMemcpyDeviceToDevice, st));
  DH_CUDA_TRY(cudaMemcpy2DAsync(p, w, (const char*)src6 + w, 2 * w, w, h->B,
                                cudaMemcpyDeviceToDevice, st));
  return SIM_OK;
}

// total matter contrast from particles and gas, then the force field g (3 n^3)
static sim_status compute_force(sim_t* h, const float* s, const float* gas, SArg pn, float* g) {
  const int B = h->B;
  if (!h->prm.gravity_on) return dzero(g, 3 * B * h->N3 * sizeof(float), h->st);
  DH_TRY(timed(h, SIM_KT_DEPOSIT, [&] {
    // the accumulator cleared by a memset ahead of the deposit, not by the conversion
    DH_TRY(dzero(h->acc, (size_t)B * h->N3 * sizeof(unsigned long long), h->st));
    DH_TRY(launch_deposit(s, nullptr, h->n, (float)h->inv_dx, h->acc, B, h->st));
    return launch_fix_to_float(h->acc, sarg(h->d_cm), gas, (int)(5 * h->N3), -1.0f, h->delta,
                               h->n, B, h->st, false);
  }));
  return timed(h, SIM_KT_POISSON, [&] {
    return launch_gravity(h->delta, g, h->ck, h->ck + B * h->NC, h->n, h->prm.box, pn, B,
                          h->plans, h->st);
  });
}

// Diagnostics record `idx` (the state after step idx - 1; idx 0 is the initial state).
static sim_status record_diag(sim_t* h, int idx, const float* gas, const float* p,
                              const float* zhat, const uint32_t* events) {
  if (idx < 0 || idx > h->prm.n_steps) return SIM_OK;
  const size_t r = (size_t)idx * h->B;
  h->diag_recorded[idx] = 1;
  return launch_diag(gas, p, zhat, events, h->N3, (float)h->prm.gamma, sarg(h->d_cm), h->B,
                     h->d_diag_sums + r * DG_NSUM, h->d_diag_mins + r * 2, h->st);
}

// One forward step in place on (gas/gas_tmp ping-pong, s, p, g). With tape != nullptr the
// inputs of every stage are recorded; diagnostics (star, aux, events) only without tape.
// merged_in: the step opens with the merged kick K2_{i-1} + K1_i (the previous step ran
// without its closing kick), which also does the previous step's star readout;
// kick_out: the step ends with its closing half kick K2_i.
// T: the step's tape slot (stage inputs recorded, outputs out of place) or NULL. primary:
// a step of the run itself (star readout, star field, events, diagnostics), as every step
// without a tape is; a recompute for the reverse pass (T set, primary false) has none of
// these side effects.
// Tnext (with T, when the next step records into the chained slot after T): the slot whose
// p0 takes this step's kicked momenta.
static sim_status forward_step(sim_t* h, int i, float** gas, float** gas_tmp, float* s, float* p,
                               float* g, const TapeSlot* T, bool merged_in = false,
                               bool kick_out = true, bool primary = false,
                               const TapeSlot* Tnext = nullptr) {
  const sim_params& P = h->prm;
  const int B = h->B;
  cudaStream_t st = h->st;
  const size_t gb = 5 * B * h->N3 * sizeof(float), vb = 3 * B * h->N3 * sizeof(float);
  const SArg K1 = sc(h, i, merged_in ? SC_KM : SC_K1), K2 = sc(h, i, SC_K2);
  const bool fwd = !T || primary;
  float* zh_prev = (merged_in && P.subgrid_on && fwd) ? h->zhat : nullptr;
  // With a tape every stage reads and writes the step's slot: the working gas, positions,
  // momenta and force are read only by the first step of a recorded run of steps and
  // written back only for the closing kick. A step with a merged opening kick records into
  // a chained slot (tape_slot): its input state, positions and force are the previous
  // slot's outputs, and its input momenta were written into its p0 by the previous step.
  const bool chained = T && merged_in;
  if (T && !chained) {
    DH_TRY(dcopy(T->U0, *gas, gb, st));
    DH_TRY(dcopy(T->s0, s, vb, st));
    DH_TRY(dcopy(T->p0, p, vb, st));
    DH_TRY(dcopy(T->g0, g, vb, st));
  }
  // 1. half kick + drift (with a tape: from s0, p0, g0 into s1 and the next slot's p0, or p)
  DH_TRY(timed(h, SIM_KT_KICK, [&] {
    if (T)
      return launch_kick_drift(T->s0, T->s1, T->p0, Tnext ? Tnext->p0 : p, T->g0, K1,
                               sc(h, i, SC_DTAU), zh_prev, zh_prev ? h->aux : nullptr, h->n,
                               (float)h->inv_dx, B, st);
    return launch_kick_drift(s, s, p, p, g, K1, sc(h, i, SC_DTAU), zh_prev,
                             zh_prev ? h->aux : nullptr, h->n, (float)h->inv_dx, B, st);
  }));
  float* cur = *gas;
  if (T) {
    // the gas kick out of place from the recorded input state into the slot's Uk1
    if (P.gravity_on)
      DH_TRY(timed(h, SIM_KT_KICK, [&] { return launch_gas_kick(T->U0, T->Uk1, T->g0, K1, h->n, B, st); }));
    else
      DH_TRY(dcopy(T->Uk1, T->U0, gb, st));
    cur = T->Uk1;
  }
  // without a tape the gas kick rides in the first sweep, which kicks every cell it loads
  // (the kicked state is never stored), where that sweep's form can
  const int first_axis = kOrders[i % 6][0] - 'x';
  const bool kick_in_sweep = !T && P.gravity_on && P.hydro_on &&
                             sweep_takes_kick(first_axis, h->n, h->fwd_var[first_axis], cur,
                                              cur == *gas ? *gas_tmp : *gas);
  if (!T && P.gravity_on && !kick_in_sweep)
    DH_TRY(timed(h, SIM_KT_KICK, [&] { return launch_gas_kick(cur, cur, g, K1, h->n, B, st); }));
  // 2. sweeps
  if (P.hydro_on) {
    const char* order = kOrders[i % 6];
    const SArg nu = sc(h, i, SC_NU);
    float* outs_tape[3] = {T ? T->Us1 : nullptr, T ? T->Us2 : nullptr, T ? T->Us3 : nullptr};
    for (int k = 0; k < 3; ++k) {
      float* out = T ? outs_tape[k] : (cur == *gas ? *gas_tmp : *gas);
      const int axis = order[k] - 'x';
      const bool kick = k == 0 && kick_in_sweep;
      DH_TRY(timed(h, SIM_KT_SWEEP, [&] {
        return launch_sweep(axis, cur, out, h->n, nu, P.gamma, P.limiter_eps, B,
                            h->fwd_var[axis], st, kick ? g : nullptr, K1);
      }));
      cur = out;
    }
  } else if (T) {
    DH_TRY(dcopy(T->Us3, cur, gb, st));
    cur = T->Us3;
  }
  // 3. subgrid
  float* zh = nullptr;
  if (P.subgrid_on) {
    float* out = T ? T->Usg : cur;
    zh = fwd ? h->zhat : nullptr;
    DH_TRY(timed(h, SIM_KT_SUBGRID, [&] {
      return launch_subgrid(cur, out, sub_at(h, i), zh, fwd ? h->events : nullptr, h->N3, B, st,
                            T ? T->gd : nullptr, zh ? h->star : nullptr);
    }));
    cur = out;
  } else if (T) {
    DH_TRY(dcopy(T->Usg, cur, gb, st));
    cur = T->Usg;
  }
  // 4. force at a_{i+1}
  DH_TRY(compute_force(h, T ? T->s1 : s, cur, sc(h, i, SC_PN1), T ? T->g1 : g));
  if (T) {
    // the working state takes the step's result only for the closing kick (the end of a
    // run of recorded steps, or every step when kicks are not merged); the momenta are
    // already in p then (no next slot)
    if (kick_out) {
      DH_TRY(dcopy(*gas, cur, gb, st));
      DH_TRY(dcopy(s, T->s1, vb, st));
      DH_TRY(dcopy(g, T->g1, vb, st));
      cur = *gas;
    }
  } else if (cur != *gas) {
    float* t = *gas;
    *gas = *gas_tmp;
    *gas_tmp = t;
  }
  // 5. half kick (+ star readout on the particles); deferred into the next step's opening
  //    kick when that one is merged
  if (kick_out) {
    DH_TRY(timed(h, SIM_KT_KICK, [&] {
      return launch_kick_drift(s, s, p, p, g, K2, sarg(0.0f), zh, zh ? h->aux : nullptr, h->n,
                               (float)h->inv_dx, B, st);
    }));
    if (P.gravity_on)
      DH_TRY(timed(h, SIM_KT_KICK, [&] { return launch_gas_kick(*gas, *gas, g, K2, h->n, B, st); }));
  }
  // 6. learned correction of the gas fields (solver in the loop, Sec. 4)
  if (h->closure) DH_TRY(closure_apply(h->closure, *gas, h->n, B, st));
  // 7. diagnostics of the state after the step (steps of the run, not the recompute)
  if (h->diag_on && fwd)
    DH_TRY(record_diag(h, i + 1, *gas, p, zh, P.subgrid_on ? h->events : nullptr));
  return SIM_OK;
}

static sim_status ensure_adjoint_buffers(sim_t* h, int tape_steps) {
  const long long N3 = h->N3 * h->B;  // cells of all instances
  if (!h->lam_gas) {
    DH_TRY(dalloc_t(h, &h->w_gas, 5 * N3));
    DH_TRY(dalloc_t(h, &h->w_gas2, 5 * N3));
    DH_TRY(dalloc_t(h, &h->w_s, 3 * N3));
    DH_TRY(dalloc_t(h, &h->w_p, 3 * N3));
    DH_TRY(dalloc_t(h, &h->w_g, 3 * N3));
    DH_TRY(dalloc_t(h, &h->lam_gas, 5 * N3));
    DH_TRY(dalloc_t(h, &h->lam_tmp, 5 * N3));
    DH_TRY(dalloc_t(h, &h->lam_s, 3 * N3));
    DH_TRY(dalloc_t(h, &h->lam_p, 3 * N3));
    DH_TRY(dalloc_t(h, &h->lamG0, 4 * N3));  // node-interleaved (x, y, z, 0)
    DH_TRY(dalloc_t(h, &h->lamG1, 4 * N3));
    DH_TRY(dalloc_t(h, &h->lam_delta, N3));
    DH_TRY(dalloc_t(h, &h->lam4, 4 * h->N3));  // one instance at a time
    DH_TRY(dalloc_t(h, &h->lam_scr, 20 * N3));
    DH_TRY(dalloc_t(h, &h->dglob, (size_t)h->B * NG));
    DH_TRY(dalloc_t(h, &h->dslots, (size_t)(h->prm.n_steps + 2) * h->B * SL_N));
  }
  if (h->tape_cap < tape_steps) {
    if (h->tape) {
      DH_CUDA_TRY(cudaStreamSynchronize(h->st));
      clear_graphs(h);
      cudaFree(h->tape);
      for (auto& a : h->allocs)
        if (a == h->tape) a = nullptr;
    }
    h->tape = nullptr;
    h->tape_first = h->tape_end = -1;
    DH_TRY(dalloc_t(h, &h->tape, (size_t)tape_steps * kTapeFloatsPerCell * N3));
    h->tape_cap = tape_steps;
  }
  return SIM_OK;
}

// Slot k of the tape. A chained slot (a step with merged kicks, i.e. not the first of its
// checkpoint segment, recorded right after the slot before it) takes its input gas state,
// positions and force from that slot: they are the previous step's Usg, s1 and g1.
static TapeSlot tape_slot(sim_t* h, int k, bool chained = false) {
  const long long N3 = h->N3 * h->B;
  float* b = h->tape + (size_t)k * kTapeFloatsPerCell * N3;
  TapeSlot t;
  t.U0 = b;
  t.Uk1 = b + 5 * N3;
  t.Us1 = b + 10 * N3;
  t.Us2 = b + 15 * N3;
  t.Us3 = b + 20 * N3;
  t.Usg = b + 25 * N3;
  t.s0 = b + 30 * N3;
  t.p0 = b + 33 * N3;
  t.g0 = b + 36 * N3;
  t.s1 = b + 39 * N3;
  t.g1 = b + 42 * N3;
  t.gd = b + 45 * N3;
  if (chained && k > 0) {
    const float* p = b - (size_t)kTapeFloatsPerCell * N3;
    t.U0 = const_cast<float*>(p + 25 * N3);  // previous Usg
    t.s0 = const_cast<float*>(p + 39 * N3);  // previous s1
    t.g0 = const_cast<float*>(p + 42 * N3);  // previous g1
  }
  return t;
}

static inline float4* lam_g4(float* p) { return reinterpret_cast<float4*>(p); }

// Adjoint of the force field g = G(s, rho) at one state: lam_G (n^3 float4 (x, y, z, 0),
// consumed) -> lam_rho += ..., lam_s += ...; slot[SL_DPREF] += lam_G . g,
// slot[SL_DCM] += d/d(1 - f_b). The three components go to lam_scr for the transforms.
static sim_status force_adjoint(sim_t* h, const float* s, const float* g, SArg pn,
                                float* lamG, double* slot) {
  if (!h->prm.gravity_on) return SIM_OK;
  const int B = h->B;
  cudaStream_t st = h->st;
  DH_TRY(timed(h, SIM_KT_POISSON_ADJOINT, [&] {
    DH_TRY(launch_unpack_dot(reinterpret_cast<const float4*>(lamG), g, h->lam_scr,
                             slot_part(slot, SL_DPREF), h->n, B, st));
    return launch_gravity_adjoint(h->lam_scr, h->lam_delta, h->ck, h->ck + 3 * B * h->NC, h->n,
                                  h->prm.box, pn, B, h->plans, st);
  }));
  return timed(h, SIM_KT_DEPOSIT_ADJOINT, [&] {
    // with lam_rho += lam_delta (d delta / d rho_gas = 1) for each particle's own cell
    return launch_deposit_adjoint(s, h->lam_delta, sarg(h->d_cm), h->lam_s,
                                  slot_part(slot, SL_DCM), h->n, (float)h->inv_dx, B, st,
                                  h->lam_gas, 5 * h->N3);
  });
}

// Reverse of forward_step for step i with tape T. In: lam_gas / lam_s / lam_p of the state
// after the step, lamG1 = adjoint of g(a_{i+1}) carried from step i+1. Out: the same
// buffers for the state before the step, lamG1 = adjoint of g(a_i) (to carry).
// slot: the step's partials, [B][SL_N].
static sim_status reverse_step(sim_t* h, int i, const TapeSlot& T, double* slot,
                               bool merged_in = false, bool kick_out = true) {
  const sim_params& P = h->prm;
  const int B = h->B;
  cudaStream_t st = h->st;
  const SArg K1 = sc(h, i, merged_in ? SC_KM : SC_K1), K2 = sc(h, i, SC_K2);
  const int slot_in = merged_in ? SL_DKM : SL_DK1;
  // 5. second half kick (when the step ran it; otherwise the next step's merged opening kick
  //    has already put its adjoint of g(a_{i+1}) into lamG1)
  if (P.gravity_on && kick_out) {
    DH_TRY(timed(h, SIM_KT_KICK_ADJOINT, [&] {
      return launch_kick_drift_adjoint(T.s1, nullptr, T.g1, K2, sarg(0.0f), h->lam_s, h->lam_p,
                                       lam_g4(h->lamG1), slot_part(slot, SL_DK2), dpart(nullptr),
                                       T.Usg, h->lam_gas, h->n, (float)h->inv_dx, B, st);
    }));
  }
  // 4. force at a_{i+1}
  if (P.gravity_on) DH_TRY(force_adjoint(h, T.s1, T.g1, sc(h, i, SC_PN1), h->lamG1, slot));
  // 3. subgrid
  if (P.subgrid_on)
    DH_TRY(timed(h, SIM_KT_SUBGRID_ADJOINT, [&] {
      return launch_subgrid_adjoint(T.Us3, h->lam_gas, sub_at(h, i), dpart(h->dglob, NG),
                                    slot_part(slot, SL_DFB), h->N3, B, st, T.gd);
    }));
  // 2. sweeps in reverse
  if (P.hydro_on) {
    const char* order = kOrders[i % 6];
    const SArg nu = sc(h, i, SC_NU);
    const float* ins[3] = {T.Uk1, T.Us1, T.Us2};
    for (int k = 2; k >= 0; --k) {
      const int axis = order[k] - 'x';
      DH_TRY(timed(h, SIM_KT_SWEEP_ADJOINT, [&] {
        return launch_sweep_adjoint(axis, ins[k], h->lam_gas, h->lam_tmp, h->n, nu, P.gamma,
                                    P.limiter_eps, slot_part(slot, SL_DNU), h->lam_scr, B,
                                    h->adj_var[axis], st);
      }));
      float* t = h->lam_gas;
      h->lam_gas = h->lam_tmp;
      h->lam_tmp = t;
    }
  }
  // 1. first half kick and drift
  DH_TRY(dzero(h->lamG0, 4 * B * h->N3 * sizeof(float), st));
  DH_TRY(timed(h, SIM_KT_KICK_ADJOINT, [&] {
    return launch_kick_drift_adjoint(T.s0, T.p0, T.g0, K1, sc(h, i, SC_DTAU), h->lam_s, h->lam_p,
                                     lam_g4(h->lamG0), slot_part(slot, slot_in), slot_part(slot, SL_DDTAU),
                                     P.gravity_on ? T.U0 : nullptr, P.gravity_on ? h->lam_gas : nullptr,
                                     h->n, (float)h->inv_dx, B, st);
  }));
  float* t = h->lamG0;
  h->lamG0 = h->lamG1;
  h->lamG1 = t;  // carry: lamG1 now holds the adjoint of g(a_i)
  return SIM_OK;
}

// dL/dparams of instance b = blockIdx.x from the device partials: d/dOmega_m = sum over
// step slots of slot * coef (schedule derivatives, host FP64, uploaded once) + the flush
// slot (force at the start of the differentiated span) + the IC terms; sigma8 from the IC
// amplitude; the subgrid parameters pass through. out is overwritten, or accumulated.
__global__ void param_chain_kernel(const double* __restrict__ slots,
                                   const double* __restrict__ coef, int nsteps, int B,
                                   const double* __restrict__ flush,
                                   const double* __restrict__ cpref,
                                   const double* __restrict__ pch,
                                   const double* __restrict__ glob, int ics, int accumulate,
                                   double* __restrict__ out) {
  pdl_enter();
  __shared__ double red[256];
  const int b = blockIdx.x;
  double acc = 0.0;
  for (int idx = threadIdx.x; idx < nsteps * SL_N; idx += blockDim.x) {
    const int i = idx / SL_N, k = idx - i * SL_N;
    const size_t o = ((size_t)i * B + b) * SL_N + k;
    acc += slots[o] * coef[o];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double* fl = flush + (size_t)b * SL_N;
    const double* pc = pch + (size_t)b * PCH_N;
    const double* gl = glob + (size_t)b * NG;
    double dom = red[0] + fl[SL_DPREF] * cpref[b] + fl[SL_DCM] * pc[PCH_CCM0];
    double ds8 = 0.0;
    if (ics) {
      const double* gx = gl + SIM_NPARAMS;
      dom += gx[GX_LAMC] * pc[PCH_DLNC] + gx[GX_DRP] * pc[PCH_DRP] + gx[GX_DFB_IC] * pc[PCH_DFB];
      ds8 = gx[GX_LAMC] * pc[PCH_INVS8];
    }
    double v[SIM_NPARAMS];
    v[SIM_P_OMEGA_M] = dom;
    v[SIM_P_SIGMA8] = ds8;
    for (int k = SIM_P_DELTA_C; k < SIM_NPARAMS; ++k) v[k] = gl[k];
    double* o = out + (size_t)b * SIM_NPARAMS;
    for (int k = 0; k < SIM_NPARAMS; ++k) o[k] = accumulate ? o[k] + v[k] : v[k];
  }
}

// steps [first, last) with slots starting at slots_first; the flush slot belongs to the
// force at a_{flush_step}
static sim_status launch_param_chain(sim_t* h, int first, int last, const double* flush,
                                     int flush_step, bool ics, bool accumulate, double* out,
                                     const double* slots_first) {
  const int B = h->B;
  DH_CUDA_TRY((launch_pdl(param_chain_kernel, B, 256, 0, h->st, slots_first, h->dcoef + (size_t)first * B * SL_N,
                                           last - first, B, flush,
                                           h->d_cpref + (size_t)flush_step * B, h->d_pch,
                                           h->dglob, ics ? 1 : 0, accumulate ? 1 : 0, out)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

// Host constants of every instance and their device tables.
static sim_status setup_instances(sim_t* h) {
  const int B = h->B, n = h->n, ns = h->prm.n_steps;
  h->scheds.resize(B);
  h->inst.resize(B);
  std::vector<float> sctab((size_t)ns * SC_N * B), pn((size_t)(ns + 1) * B), cm(B);
  std::vector<SubgridConst> sub((size_t)ns * B);
  std::vector<double> pch((size_t)B * PCH_N), cpref((size_t)(ns + 1) * B);
  std::vector<double> coef((size_t)ns * B * SL_N, 0.0);
  for (int b = 0; b < B; ++b) {
    const sim_params& p = h->prms[b];
    InstConst& c = h->inst[b];
    h->scheds[b] = make_schedule(p.a_start, p.a_end, p.n_steps, p.omega_m, p.kdk_mode);
    const std::vector<StepFactors>& sch = h->scheds[b];
    c.fb = p.omega_b / p.omega_m;
    c.cm = 1.0 - c.fb;
    c.dfb_dom = -c.fb / p.omega_m;
    // IC constants (Sec. 2.1): C = rms_target sqrt(n^3 / sum_k P(k))
    const double kf = 2.0 * M_PI / p.box, kc = p.kc_frac * M_PI * n / p.box;
    double total = 0.0;
    for (int z = 0; z < n; ++z)
      for (int y = 0; y < n; ++y)
        for (int x = 0; x <= n / 2; ++x) {
          const int kz = z > n / 2 ? z - n : z, ky = y > n / 2 ? y - n : y;
          const double k2 = kf * kf * ((double)x * x + (double)ky * ky + (double)kz * kz);
          if (k2 <= 0) continue;
          const double w = (x == 0 || (n % 2 == 0 && x == n / 2)) ? 1.0 : 2.0;
          total += w * std::exp(-k2 / (kc * kc)) / k2;
        }
    const double Di = growth_D(p.a_start, p.omega_m);
    const double rms =
        p.rms_ref * (p.sigma8 / p.sigma8_ref) * Di / growth_D(p.a_ref, p.omega_m_ref);
    c.C = rms * std::sqrt((double)n * n * n / total);
    const double hh = 1e-5 * p.omega_m;
    c.dlnC_dom =
        (growth_D(p.a_start, p.omega_m + hh) - growth_D(p.a_start, p.omega_m - hh)) / (2 * hh) / Di;
    auto rpf = [&](double om) { return growth_gp(p.a_start, om) / growth_D(p.a_start, om); };
    c.rp = rpf(p.omega_m);
    c.drp_dom = (rpf(p.omega_m + hh) - rpf(p.omega_m - hh)) / (2 * hh);
    c.a2e0 = p.a_start * p.a_start * (p.T_init / temperature_per_energy(p.gamma, p.mu));
    // step tables
    for (int i = 0; i < ns; ++i) {
      const StepFactors& f = sch[i];
      float* row = sctab.data() + (size_t)i * SC_N * B;
      row[SC_K1 * B + b] = p.gravity_on ? (float)f.K1 : 0.0f;
      row[SC_K2 * B + b] = p.gravity_on ? (float)f.K2 : 0.0f;
      // the closing half kick of step i - 1 and the opening one of step i see the same force
      // at the same positions: inside a segment they are one kick of K2_{i-1} + K1_i
      const double km = f.K1 + (i > 0 ? sch[i - 1].K2 : 0.0);
      row[SC_KM * B + b] = p.gravity_on ? (float)km : 0.0f;
      row[SC_DTAU * B + b] = (float)f.dtau;
      row[SC_NU * B + b] = (float)(f.dtau * h->inv_dx);
      row[SC_PN1 * B + b] = gravity_pref_norm(f.pref1, n);
      sub[(size_t)i * B + b] = make_subgrid_const(p, f.a1, i);
      double* cf = coef.data() + ((size_t)i * B + b) * SL_N;
      cf[SL_DK1] = f.dK1;
      cf[SL_DK2] = f.dK2;
      cf[SL_DKM] = f.dK1 + (i > 0 ? sch[i - 1].dK2 : 0.0);
      cf[SL_DNU] = f.ddtau * h->inv_dx;
      cf[SL_DDTAU] = f.ddtau;
      cf[SL_DPREF] = f.dpref1 / f.pref1;
      cf[SL_DCM] = -c.dfb_dom;
      cf[SL_DFB] = c.dfb_dom;
    }
    for (int i = 0; i <= ns; ++i) {
      const double a = i == 0 ? p.a_start : sch[i - 1].a1;
      const double pref = 1.5 * p.omega_m / a;
      pn[(size_t)i * B + b] = gravity_pref_norm(pref, n);
      cpref[(size_t)i * B + b] = (1.5 / a) / pref;
    }
    cm[b] = (float)c.cm;
    double* pc = pch.data() + (size_t)b * PCH_N;
    pc[PCH_CCM0] = -c.dfb_dom;
    pc[PCH_DLNC] = c.dlnC_dom;
    pc[PCH_DRP] = c.drp_dom;
    pc[PCH_DFB] = c.dfb_dom;
    pc[PCH_INVS8] = 1.0 / p.sigma8;
  }
  h->sched = h->scheds[0];
  h->h_sc = sctab;
  h->h_pn = pn;
  h->h_sub = sub;
  // the tables keep their size for a handle's life (sim_set_params refills them in place)
  if (!h->d_sc) {
    DH_TRY(dalloc_t(h, &h->d_sc, sctab.size()));
    DH_TRY(dalloc_t(h, &h->d_pn, pn.size()));
    DH_TRY(dalloc_t(h, &h->d_cm, cm.size()));
    DH_TRY(dalloc_t(h, &h->d_sub, sub.size()));
    DH_TRY(dalloc_t(h, &h->d_pch, pch.size()));
    DH_TRY(dalloc_t(h, &h->d_cpref, cpref.size()));
    DH_TRY(dalloc_t(h, &h->dcoef, coef.size()));
  }
  auto up = [](void* d, const void* s, size_t bytes) -> sim_status {
    DH_CUDA_TRY(cudaMemcpy(d, s, bytes, cudaMemcpyHostToDevice));
    return SIM_OK;
  };
  DH_TRY(up(h->d_sc, sctab.data(), sctab.size() * sizeof(float)));
  DH_TRY(up(h->d_pn, pn.data(), pn.size() * sizeof(float)));
  DH_TRY(up(h->d_cm, cm.data(), cm.size() * sizeof(float)));
  DH_TRY(up(h->d_sub, sub.data(), sub.size() * sizeof(SubgridConst)));
  DH_TRY(up(h->d_pch, pch.data(), pch.size() * sizeof(double)));
  DH_TRY(up(h->d_cpref, cpref.data(), cpref.size() * sizeof(double)));
  DH_TRY(up(h->dcoef, coef.data(), coef.size() * sizeof(double)));
  return SIM_OK;
}

static sim_status alloc_state(sim_t* h) {
  const long long N3 = h->N3 * h->B, NC = h->NC;
  const long long words = (h->N3 + 31) / 32 * h->B;
  DH_TRY(dalloc_t(h, &h->gas, 5 * N3));
  DH_TRY(dalloc_t(h, &h->gas2, 5 * N3));
  DH_TRY(dalloc_t(h, &h->s, 3 * N3));
  DH_TRY(dalloc_t(h, &h->p, 3 * N3));
  DH_TRY(dalloc_t(h, &h->g, 3 * N3));
  DH_TRY(dalloc_t(h, &h->star, N3));
  DH_TRY(dalloc_t(h, &h->aux, N3));
  DH_TRY(dalloc_t(h, &h->zhat, N3));
  DH_TRY(dalloc_t(h, &h->delta, N3));
  DH_TRY(dalloc_t(h, &h->events, words));
  DH_TRY(dalloc_t(h, &h->acc, N3));
  DH_TRY(dalloc_t(h, &h->ck, (size_t)(4 * h->B > 5 ? 4 * h->B : 5) * NC));
  DH_TRY(dalloc_t(h, &h->noise, N3));
  DH_TRY(dalloc_t(h, &h->f4, 4 * N3));
  DH_TRY(dalloc_t(h, &h->init_gas, 5 * N3));
  DH_TRY(dalloc_t(h, &h->init_part, 6 * N3));
  DH_TRY(dalloc_t(h, &h->prev_gas, 5 * N3));
  DH_TRY(dalloc_t(h, &h->prev_part, 6 * N3));
  DH_TRY(dalloc_t(h, &h->speed_bits, h->B));
  DH_TRY(dzero(h->acc, N3 * sizeof(unsigned long long), h->st));
  DH_TRY(dzero(h->events, words * sizeof(uint32_t), h->st));
  return SIM_OK;
}

// Initial conditions of every instance from its noise (already in h->noise), into
// init_gas / init_part (Sec. 2.1).
static sim_status make_ics(sim_t* h) {
  const long long N3 = h->N3;
  cudaStream_t st = h->st;
  for (int b = 0; b < h->B; ++b) {
    const sim_params& p = h->prms[b];
    const InstConst& c = h->inst[b];
    float* f4 = h->f4 + (size_t)b * 4 * N3;
    float* part = h->init_part + (size_t)b * 6 * N3;
    DH_TRY(launch_linear_field(h->noise + (size_t)b * N3, f4, h->ck, h->n, p.box, p.kc_frac, c.C,
                               ic_plans(h), st));
    DH_TRY(launch_place(f4, h->init_gas + (size_t)b * 5 * N3, part, part + 3 * N3, c.rp, c.fb,
                        c.a2e0, N3, st));
  }
  return SIM_OK;
}

static sim_status load_noise(sim_t* h, const float* noise) {
  if (noise) return dcopy(h->noise, noise, h->B * h->N3 * sizeof(float), h->st);
  for (int b = 0; b < h->B; ++b)
    DH_TRY(launch_noise(h->prms[b].seed, h->prms[b].instance, h->noise + (size_t)b * h->N3,
                        h->N3, h->st));
  return SIM_OK;
}

static void clear_checkpoints(sim_t* h) {
  h->ckpt_count = 0;
  h->tape_first = h->tape_end = -1;
}

static sim_status ensure_ckpt_pool(sim_t* h, int count) {
  while ((int)h->ckpt_pool.size() < count) {
    float* c = nullptr;
    DH_TRY(dalloc_t(h, &c, 11 * h->N3 * h->B));
    h->ckpt_pool.push_back(c);
    h->ckpt_step.push_back(0);
  }
  return SIM_OK;
}

static sim_status reset_to_init(sim_t* h) {
  const long long N3 = h->N3 * h->B;
  cudaStream_t st = h->st;
  DH_TRY(dcopy(h->gas, h->init_gas, 5 * N3 * sizeof(float), st));
  DH_TRY(part_split(h->s, h->p, h->init_part, h, st));
  DH_TRY(dzero(h->star, N3 * sizeof(float), st));
  DH_TRY(dzero(h->aux, N3 * sizeof(float), st));
  h->step = h->init_step;
  DH_TRY(compute_force(h, h->s, h->gas, pn_at(h, h->init_step), h->g));
  clear_checkpoints(h);
  h->prev_step = -1;
  return SIM_OK;
}

// checkpoint layout: gas (B 5 n^3) | s (B 3 n^3) | p (B 3 n^3)
static sim_status store_checkpoint(sim_t* h) {
  const long long N3 = h->N3 * h->B;
  if (h->ckpt_count >= (int)h->ckpt_pool.size()) {
    set_error("internal: checkpoint pool exhausted");
    return SIM_EINVAL;
  }
  float* c = h->ckpt_pool[h->ckpt_count];
  h->ckpt_step[h->ckpt_count] = h->step;
  h->ckpt_count += 1;
  DH_TRY(dcopy(c, h->gas, 5 * N3 * sizeof(float), h->st));
  DH_TRY(dcopy(c + 5 * N3, h->s, 3 * N3 * sizeof(float), h->st));
  return dcopy(c + 8 * N3, h->p, 3 * N3 * sizeof(float), h->st);
}

static sim_status validate_batch(const sim_params* p, int B) {
  if (!p || B < 1) {
    set_error("null parameter block or B < 1");
    return SIM_EINVAL;
  }
  for (int b = 0; b < B; ++b) DH_TRY(validate(p + b));
  const sim_params& a = p[0];
  for (int b = 1; b < B; ++b) {
    const sim_params& q = p[b];
    const bool same = q.n == a.n && q.box == a.box && q.n_steps == a.n_steps &&
                      q.a_start == a.a_start && q.a_end == a.a_end &&
                      q.ckpt_every == a.ckpt_every && q.subgrid_on == a.subgrid_on &&
                      q.gravity_on == a.gravity_on && q.hydro_on == a.hydro_on &&
                      q.kdk_mode == a.kdk_mode && q.gamma == a.gamma && q.mu == a.mu &&
                      q.h == a.h && q.rms_ref == a.rms_ref && q.a_ref == a.a_ref &&
                      q.sigma8_ref == a.sigma8_ref && q.omega_m_ref == a.omega_m_ref &&
                      q.kc_frac == a.kc_frac && q.limiter_eps == a.limiter_eps &&
                      q.cfl_max == a.cfl_max;
    if (!same) {
      set_error("sim_init_batch: instance %d differs from instance 0 in a shared field (n, "
                "box, schedule, switches, gamma, mu, h, IC normalisation, limiter, cfl_max)", b);
      return SIM_EINVAL;
    }
  }
  const long long zlim = (long long)a.n * B;
  if (zlim > 65535) {
    set_error("sim_init_batch: n * B = %lld exceeds the launch grid limit 65535", zlim);
    return SIM_EINVAL;
  }
  return SIM_OK;
}

static sim_status cfl_now(sim_t* h, double* cfl_out);

// The closure's workspace for this handle's grid; graphs that captured an older workspace
// are dropped.
static sim_status closure_ready(sim_t* h) {
  if (!h->closure) return SIM_OK;
  DH_TRY(closure_prepare(h->closure, h->n, h->B, false));
  const uint64_t g = closure_generation(h->closure);
  if (g != h->closure_gen) {
    clear_graphs(h);
    h->closure_gen = g;
  }
  return SIM_OK;
}

// Whether sim_run keeps each step's closing half kick apart from the next step's opening
// one (the reverse pass recomputes segments the same way).
static bool kicks_apart(const sim_t* h) {
  return h->closure || h->prm.cfl_max > 0 || h->diag_on;
}

// Checks and allocations of sim_run (never inside a capture).
static sim_status run_prepare(sim_t* h, int n_steps) {
  if (h->step != h->init_step || h->ckpt_count != 0) {
    set_error("sim_run: the handle must be at its initial state (sim_init / sim_reset)");
    return SIM_EINVAL;
  }
  if (n_steps < 0 || h->step + n_steps > h->prm.n_steps) {
    set_error("sim_run: n_steps out of range");
    return SIM_EINVAL;
  }
  DH_TRY(closure_ready(h));
  return ensure_ckpt_pool(h, (n_steps + h->prm.ckpt_every - 1) / h->prm.ckpt_every);
}

// Checkpoint segments the handle records at the end of a run, at least min_segments.
static int recorded_segments(const sim_t* h, int min_segments) {
  const int all = (h->prm.n_steps + h->prm.ckpt_every - 1) / h->prm.ckpt_every;
  const int k = h->tape_segments < 0 ? all : h->tape_segments;
  return std::min(all, std::max(k, min_segments));
}

// Tape steps the reverse pass of a run needs: one segment to recompute into, or the
// segments the runs record.
static int tape_steps_wanted(const sim_t* h) {
  return h->prm.ckpt_every * std::max(1, recorded_segments(h, 0));
}

// n_steps forward steps with a checkpoint every ckpt_every steps (Sec. 2.3.5).
static sim_status run_body(sim_t* h, int n_steps, int min_segments = 0) {
  const int last = h->step + n_steps;
  const int every = h->prm.ckpt_every, init = h->init_step;
  // Once the handle holds a tape (it has run a reverse pass), the run records its last
  // checkpoint segments as it goes (as many as asked for and as the tape holds, from a
  // segment start not before this call's first step), so the next reverse pass recomputes
  // none of them.
  const int segs = recorded_segments(h, min_segments);
  int rec_first = 0;
  bool record = false;
  if (n_steps > 0 && segs > 0 && h->tape && !h->closure) {
    const int last_seg = init + (last - 1 - init) / every * every;
    rec_first = last_seg - (segs - 1) * every;
    const int fit = last - h->tape_cap;                        // earliest step with a slot
    if (rec_first < fit) rec_first = init + (fit - init + every - 1) / every * every;
    const int call_seg = init + (h->step - init + every - 1) / every * every;
    if (rec_first < call_seg) rec_first = call_seg;
    record = rec_first <= last_seg;
  }
  h->tape_first = h->tape_end = -1;
  if (h->diag_on && n_steps > 0)
    DH_TRY(record_diag(h, h->step, h->gas, h->p, nullptr, nullptr));
  for (int k = 0; k < n_steps; ++k) {
    const int rel = h->step - h->init_step;
    if (rel % every == 0) DH_TRY(store_checkpoint(h));
    // kicks merge inside a checkpoint segment (not with a closure, which acts on the state
    // after the closing kick, nor with the CFL watchdog or the diagnostics, which read every
    // step's state)
    const bool plain = kicks_apart(h);
    const bool merged_in = !plain && rel % every != 0;
    const bool kick_out = plain || h->step + 1 == last || (rel + 1) % every == 0;
    const bool rec = record && h->step >= rec_first;
    const TapeSlot T = rec ? tape_slot(h, h->step - rec_first, merged_in) : TapeSlot{};
    // the next step records into the chained slot after T unless this one closes its kick
    const TapeSlot Tn = rec && !kick_out ? tape_slot(h, h->step + 1 - rec_first, true) : TapeSlot{};
    DH_TRY(forward_step(h, h->step, &h->gas, &h->gas2, h->s, h->p, h->g, rec ? &T : nullptr,
                        merged_in, kick_out, true, rec && !kick_out ? &Tn : nullptr));
    h->step += 1;
    if (h->prm.cfl_max > 0 && h->step < h->prm.n_steps) {
      double c = 0;
      DH_TRY(cfl_now(h, &c));
      if (!(c <= h->prm.cfl_max)) {
        set_error("sim_run: CFL number %.4g above cfl_max %.4g after step %d", c,
                  h->prm.cfl_max, h->step);
        return std::isfinite(c) ? SIM_ECFL : SIM_ENAN;
      }
    }
  }
  h->prev_step = -1;
  if (record) {
    h->tape_first = rec_first;
    h->tape_end = last;
  }
  return SIM_OK;
}

static sim_status run_adjoint_prepare(sim_t* h, const float* dL_dnoise, const double* dL_dparams) {
  if (h->closure) {
    set_error("sim_run_adjoint: not available while a learned closure is set");
    return SIM_ENOTIMPL;
  }
  if (!dL_dparams) {
    set_error("sim_run_adjoint: null arguments");
    return SIM_EINVAL;
  }
  if (h->ckpt_count == 0) {
    set_error("sim_run_adjoint: no sim_run to differentiate");
    return SIM_EINVAL;
  }
  if (!h->ics_valid && dL_dnoise) {
    set_error("sim_run_adjoint: the run did not start from initial conditions");
    return SIM_EINVAL;
  }
  return ensure_adjoint_buffers(h, tape_steps_wanted(h));
}

// Reverse pass over the checkpointed run: every segment recomputed forward with the tape,
// then reversed step by step; the initial force and the ICs last.
static sim_status run_adjoint_body(sim_t* h, const float* dL_dgas, const float* dL_dpart,
                                   float* dL_dnoise, double* dL_dparams) {
  const long long N3 = h->N3 * h->B;
  const int B = h->B;
  const int nseg = h->ckpt_count;
  const int last = h->step;
  cudaStream_t st = h->st;
  DH_TRY(dzero(h->dslots, (size_t)(h->prm.n_steps + 2) * B * SL_N * sizeof(double), st));
  DH_TRY(dzero(h->dglob, (size_t)B * NG * sizeof(double), st));
  if (dL_dgas)
    DH_TRY(dcopy(h->lam_gas, dL_dgas, 5 * N3 * sizeof(float), st));
  else
    DH_TRY(dzero(h->lam_gas, 5 * N3 * sizeof(float), st));
  if (dL_dpart) {
    DH_TRY(part_split(h->lam_s, h->lam_p, dL_dpart, h, st));
  } else {
    DH_TRY(dzero(h->lam_s, 3 * N3 * sizeof(float), st));
    DH_TRY(dzero(h->lam_p, 3 * N3 * sizeof(float), st));
  }
  DH_TRY(dzero(h->lamG1, 4 * N3 * sizeof(float), st));
  // the segments the run recorded on the tape need no recompute (reversed first, from their
  // slots); the recompute of the other segments overwrites the tape from slot 0
  const int taped_first = h->tape_first, taped_end = h->tape_end;
  h->tape_first = h->tape_end = -1;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int first = h->ckpt_step[seg];
    const int end = seg + 1 < nseg ? h->ckpt_step[seg + 1] : last;
    // the same kick merging as the forward run: opening kicks merged after the segment's
    // first step, the closing kick only at the segment's end
    const bool plain = kicks_apart(h);
    const bool taped = taped_first >= 0 && first >= taped_first && end <= taped_end;
    const int base = taped ? taped_first : first;  // step of tape slot 0
    if (!taped) {
      const float* c = h->ckpt_pool[seg];
      DH_TRY(dcopy(h->w_gas, c, 5 * N3 * sizeof(float), st));
      DH_TRY(dcopy(h->w_s, c + 5 * N3, 3 * N3 * sizeof(float), st));
      DH_TRY(dcopy(h->w_p, c + 8 * N3, 3 * N3 * sizeof(float), st));
      DH_TRY(compute_force(h, h->w_s, h->w_gas, pn_at(h, first), h->w_g));
      for (int i = first; i < end; ++i) {
        const bool out = plain || i == end - 1;
        const TapeSlot T = tape_slot(h, i - first, !plain && i != first);
        const TapeSlot Tn = out ? TapeSlot{} : tape_slot(h, i + 1 - first, true);
        DH_TRY(forward_step(h, i, &h->w_gas, &h->w_gas2, h->w_s, h->w_p, h->w_g, &T,
                            !plain && i != first, out, false, out ? nullptr : &Tn));
      }
    }
    for (int i = end - 1; i >= first; --i)
      DH_TRY(reverse_step(h, i, tape_slot(h, i - base, !plain && i != first),
                          h->dslots + (size_t)i * B * SL_N,
                          !plain && i != first, plain || i == end - 1));
  }
  // g at the start of the run is a function of the initial state
  const TapeSlot T0 = tape_slot(h, 0);
  const int s0 = h->ckpt_step[0];
  double* slot0 = h->dslots + (size_t)h->prm.n_steps * B * SL_N;
  DH_TRY(force_adjoint(h, T0.s0, T0.g0, pn_at(h, s0), h->lamG1, slot0));
  // through the initial conditions to the white noise, one instance at a time
  if (h->ics_valid) {
    const long long n3 = h->N3;
    for (int b = 0; b < B; ++b) {
      const InstConst& c = h->inst[b];
      double* gx = h->dglob + (size_t)b * NG + SIM_NPARAMS;
      const float* f4 = h->f4 + (size_t)b * 4 * n3;
      DH_TRY(launch_ic_adjoint(f4, h->lam_gas + (size_t)b * 5 * n3, h->lam_s + (size_t)b * 3 * n3,
                               h->lam_p + (size_t)b * 3 * n3, h->lam4,
                               dL_dnoise ? dL_dnoise + (size_t)b * n3 : nullptr, h->ck, h->n,
                               h->prm.box, h->prm.kc_frac, c.C, c.rp, c.fb, c.a2e0,
                               gx + GX_DRP, gx + GX_DFB_IC, ic_plans(h), st));
      DH_TRY(launch_dot(h->lam4, f4, 4 * n3, dpart(gx + GX_LAMC), 1, st));
    }
  }
  return launch_param_chain(h, s0, last, slot0, s0, h->ics_valid, false, dL_dparams,
                            h->dslots + (size_t)s0 * B * SL_N);
}

}  // namespace dh

// ===================================================================== C ABI
extern "C" {

int64_t sim_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

sim_status sim_params_default(sim_params* p) {
  if (!p) return SIM_EINVAL;
  memset(p, 0, sizeof(*p));
  p->n = 32;
  p->n_steps = 20;
  p->ckpt_every = 6;
  p->subgrid_on = 0;
  p->gravity_on = 1;
  p->hydro_on = 1;
  p->kdk_mode = 0;
  p->instance = 0;
  p->seed = 1;
  p->box = 32.0;
  p->omega_m = 0.3;
  p->omega_b = 0.049;
  p->h = 0.7;
  p->sigma8 = 0.8;
  p->gamma = 5.0 / 3.0;
  p->mu = 0.6;
  p->T_init = 1.0e4;
  p->a_start = 0.1;
  p->a_end = 0.5;
  p->delta_c = 100.0;
  p->Pi0 = 0.05;
  p->E0 = 0.03;
  p->T_c = 3.0e4;
  p->w_delta = 5.0;
  p->w_T = 1500.0;
  p->tau = 0.1;
  p->T0_uv = 0.0;
  p->gamma_uv = 1.4;
  p->rms_ref = 0.05;
  p->a_ref = 0.1;
  p->sigma8_ref = 0.8;
  p->omega_m_ref = 0.3;
  p->kc_frac = 0.5;
  p->limiter_eps = 1e-30;
  p->cfl_max = 0.0;
  return SIM_OK;
}

const char* sim_last_error(const sim_t* h) { return h ? h->err.c_str() : get_error(); }


sim_status sim_init_batch(const sim_params* p, int32_t B, const float* noise, void* stream,
                          sim_t** out) {
  if (!out) {
    set_error("sim_init: out is NULL");
    return SIM_EINVAL;
  }
  *out = nullptr;
  DH_TRY(validate_batch(p, B));
  sim_t* h = new sim_t();
  h->prm = p[0];
  h->prms.assign(p, p + B);
  h->B = B;
  h->n = p->n;
  h->N3 = (long long)p->n * p->n * p->n;
  h->NC = (long long)p->n * p->n * (p->n / 2 + 1);
  h->st = (cudaStream_t)stream;
  h->dx = p->box / p->n;
  h->inv_dx = p->n / p->box;
  sim_status r = prepare_sweep_kernels();
  if (r == SIM_OK) r = setup_instances(h);
  if (r == SIM_OK) r = h->plans.create(p->n, B);
  if (r == SIM_OK && B > 1) r = h->plans1.create(p->n, 1);
  if (r == SIM_OK) r = alloc_state(h);
  if (r == SIM_OK && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    set_error("cudaStreamCreate failed");
    r = SIM_ECUDA;
  }
  if (r == SIM_OK) r = load_noise(h, noise);
  if (r == SIM_OK) r = make_ics(h);
  if (r == SIM_OK) {
    h->ics_valid = true;
    h->init_step = 0;
    r = reset_to_init(h);
  }
  if (r != SIM_OK) {
    sim_destroy(h);
    return r;
  }
  *out = h;
  return SIM_OK;
}

sim_status sim_set_params(sim_t* h, const sim_params* p) {
  if (!h) return SIM_EINVAL;
  sim_status r = validate_batch(p, h->B);
  if (r != SIM_OK) return fail(h, r);
  const sim_params& a = h->prm;
  const sim_params& q = p[0];
  const bool same = q.n == a.n && q.box == a.box && q.n_steps == a.n_steps &&
                    q.a_start == a.a_start && q.a_end == a.a_end && q.ckpt_every == a.ckpt_every &&
                    q.subgrid_on == a.subgrid_on && q.gravity_on == a.gravity_on &&
                    q.hydro_on == a.hydro_on && q.kdk_mode == a.kdk_mode && q.gamma == a.gamma &&
                    q.mu == a.mu && q.limiter_eps == a.limiter_eps && q.cfl_max == a.cfl_max;
  if (!same) {
    set_error("sim_set_params: n, box, schedule, switches, gamma, mu, limiter_eps and cfl_max "
              "must stay as at sim_init");
    return fail(h, SIM_EINVAL);
  }
  // the tables are read by captured graphs in place, but one instance passes its scalars by
  // value: drop the graphs
  DH_CUDA_TRY(cudaStreamSynchronize(h->st));
  clear_graphs(h);
  h->prms.assign(p, p + h->B);
  h->prm = p[0];
  r = setup_instances(h);
  if (r == SIM_OK && h->ics_valid) r = make_ics(h);
  if (r == SIM_OK) r = reset_to_init(h);
  return fail(h, r);
}

sim_status sim_init(const sim_params* p, const float* noise, void* stream, sim_t** out) {
  return sim_init_batch(p, 1, noise, stream, out);
}

int32_t sim_batch_size(const sim_t* h) { return h ? h->B : 0; }

void sim_destroy(sim_t* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  if (h->cap_stream) cudaStreamSynchronize(h->cap_stream);
  clear_graphs(h);
  for (cudaEvent_t e : h->kt_ev) cudaEventDestroy(e);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  h->plans.destroy();
  h->plans1.destroy();
  for (void* a : h->allocs)
    if (a) cudaFree(a);
  delete h;
}

sim_status sim_set_graphs(sim_t* h, int32_t on) {
  if (!h) return SIM_EINVAL;
  if (!on) clear_graphs(h);
  h->graphs = on != 0;
  return SIM_OK;
}

sim_status sim_kernel_timing(sim_t* h, int32_t enable) {
  if (!h) return SIM_EINVAL;
  h->kt_on = enable != 0;
  return SIM_OK;
}

sim_status sim_kernel_times(sim_t* h, double* ms, int64_t* count, int32_t reset) {
  if (!h || !ms || !count) {
    set_error("sim_kernel_times: null argument");
    return SIM_EINVAL;
  }
  for (int c = 0; c < SIM_KT_N; ++c) {
    ms[c] = 0.0;
    count[c] = 0;
  }
  if (h->kt_used) DH_CUDA_TRY(cudaEventSynchronize(h->kt_ev[2 * h->kt_used - 1]));
  for (size_t i = 0; i < h->kt_used; ++i) {
    float t = 0.0f;
    DH_CUDA_TRY(cudaEventElapsedTime(&t, h->kt_ev[2 * i], h->kt_ev[2 * i + 1]));
    ms[h->kt_cls[i]] += t;
    count[h->kt_cls[i]] += 1;
  }
  if (reset) {
    h->kt_used = 0;
    h->kt_dropped = 0;
  }
  return SIM_OK;
}

sim_status sim_set_sweep_variants(sim_t* h, const int32_t* fwd, const int32_t* adj) {
  if (!h) return SIM_EINVAL;
  for (int a = 0; a < 3; ++a) {
    const int vals[2] = {fwd ? fwd[a] : 0, adj ? adj[a] : 0};
    for (int v : vals)
      if (v < SIM_SWEEP_DEFAULT || v > SIM_SWEEP_PAIR) {
        set_error("sim_set_sweep_variants: unknown variant %d", v);
        return fail(h, SIM_EINVAL);
      }
  }
  clear_graphs(h);
  for (int a = 0; a < 3; ++a) {
    if (fwd) h->fwd_var[a] = fwd[a];
    if (adj) h->adj_var[a] = adj[a];
  }
  return SIM_OK;
}

sim_status sim_autotune(sim_t* h, int32_t reps, int32_t* fwd_out, int32_t* adj_out) {
  if (!h || reps < 1) {
    set_error("sim_autotune: null handle or reps < 1");
    return fail(h, SIM_EINVAL);
  }
  sim_status r = ensure_adjoint_buffers(h, 0);
  if (r != SIM_OK) return fail(h, r);
  clear_graphs(h);
  cudaStream_t st = h->st;
  cudaEvent_t e0, e1;
  DH_CUDA_TRY(cudaEventCreate(&e0));
  DH_CUDA_TRY(cudaEventCreate(&e1));
  const int i = h->step < h->prm.n_steps ? h->step : h->prm.n_steps - 1;
  const SArg nu = sc(h, i, SC_NU);
  const int cand[5] = {SIM_SWEEP_TILE, SIM_SWEEP_MARCH32, SIM_SWEEP_MARCH16, SIM_SWEEP_MARCH_FIT,
                       SIM_SWEEP_PAIR};
  auto time_it = [&](auto launch, float* ms) -> sim_status {
    DH_TRY(launch());  // warm-up
    float best = 1e30f;
    for (int k = 0; k < reps; ++k) {
      DH_CUDA_TRY(cudaEventRecord(e0, st));
      DH_TRY(launch());
      DH_CUDA_TRY(cudaEventRecord(e1, st));
      DH_CUDA_TRY(cudaEventSynchronize(e1));
      float t = 0.0f;
      DH_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
      best = t < best ? t : best;
    }
    *ms = best;
    return SIM_OK;
  };
  auto body = [&]() -> sim_status {
    for (int axis = 0; axis < 3; ++axis) {
      float bf = 1e30f, ba = 1e30f;
      for (int c = 0; c < 5; ++c) {
        float t = 0.0f;
        // forward x: the tile only; the paired form needs an even n
        if ((axis != 0 || c == 0) && (cand[c] != SIM_SWEEP_PAIR || h->n % 2 == 0)) {
          DH_TRY(time_it([&] { return launch_sweep(axis, h->gas, h->w_gas2, h->n, nu,
                                                   h->prm.gamma, h->prm.limiter_eps, h->B,
                                                   cand[c], st); }, &t));
          if (t < bf) {
            bf = t;
            h->fwd_var[axis] = cand[c];
          }
        }
        if (cand[c] == SIM_SWEEP_PAIR) continue;  // forward only
        DH_TRY(time_it([&] { return launch_sweep_adjoint(axis, h->gas, h->gas, h->lam_tmp, h->n,
                                                         nu, h->prm.gamma, h->prm.limiter_eps,
                                                         dpart(h->dslots, SL_N), h->lam_scr,
                                                         h->B, cand[c], st); }, &t));
        if (t < ba) {
          ba = t;
          h->adj_var[axis] = cand[c];
        }
      }
      if (fwd_out) fwd_out[axis] = h->fwd_var[axis];
      if (adj_out) adj_out[axis] = h->adj_var[axis];
    }
    return SIM_OK;
  };
  r = body();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return fail(h, r);
}

sim_status sim_step(sim_t* h) {
  if (!h) return SIM_EINVAL;
  if (h->step >= h->prm.n_steps) {
    set_error("sim_step: already at the last step (%d)", h->prm.n_steps);
    return fail(h, SIM_EINVAL);
  }
  const long long N3 = h->N3 * h->B;
  sim_status r = closure_ready(h);
  if (r == SIM_OK && h->diag_on && h->step == h->init_step)
    r = record_diag(h, h->step, h->gas, h->p, nullptr, nullptr);
  if (r == SIM_OK) r = dcopy(h->prev_gas, h->gas, 5 * N3 * sizeof(float), h->st);
  if (r == SIM_OK) r = part_join(h->prev_part, h->s, h->p, h, h->st);
  if (r == SIM_OK) r = forward_step(h, h->step, &h->gas, &h->gas2, h->s, h->p, h->g, nullptr);
  if (r != SIM_OK) return fail(h, r);
  h->prev_step = h->step;
  h->step += 1;
  clear_checkpoints(h);
  return SIM_OK;
}

sim_status sim_step_adjoint(sim_t* h, float* adj_gas, float* adj_part, double* adj_params) {
  if (!h || !adj_gas || !adj_part) {
    set_error("sim_step_adjoint: null arguments");
    return fail(h, SIM_EINVAL);
  }
  if (h->prev_step < 0 || h->prev_step + 1 != h->step) {
    set_error("sim_step_adjoint: no sim_step to differentiate");
    return fail(h, SIM_EINVAL);
  }
  if (h->closure) {
    set_error("sim_step_adjoint: not available while a learned closure is set");
    return fail(h, SIM_ENOTIMPL);
  }
  const long long N3 = h->N3 * h->B;
  const int B = h->B;
  cudaStream_t st = h->st;
  const int i = h->prev_step;
  sim_status r = ensure_adjoint_buffers(h, 1);
  if (r != SIM_OK) return fail(h, r);
  const TapeSlot T = tape_slot(h, 0);
  h->tape_first = h->tape_end = -1;
  double* slot = h->dslots;
  auto run = [&]() -> sim_status {
    DH_TRY(dzero(h->dslots, 2 * (size_t)B * SL_N * sizeof(double), st));
    DH_TRY(dzero(h->dglob, (size_t)B * NG * sizeof(double), st));
    // recompute the step from its input with the tape
    DH_TRY(dcopy(h->w_gas, h->prev_gas, 5 * N3 * sizeof(float), st));
    DH_TRY(part_split(h->w_s, h->w_p, h->prev_part, h, st));
    DH_TRY(compute_force(h, h->w_s, h->w_gas, pn_at(h, i), h->w_g));
    DH_TRY(forward_step(h, i, &h->w_gas, &h->w_gas2, h->w_s, h->w_p, h->w_g, &T));
    // reverse
    DH_TRY(dcopy(h->lam_gas, adj_gas, 5 * N3 * sizeof(float), st));
    DH_TRY(part_split(h->lam_s, h->lam_p, adj_part, h, st));
    DH_TRY(dzero(h->lamG1, 4 * N3 * sizeof(float), st));
    DH_TRY(reverse_step(h, i, T, slot));
    // g(a_i) is a function of the input state: flush its adjoint now
    double* flush = slot + (size_t)B * SL_N;
    DH_TRY(force_adjoint(h, T.s0, T.g0, pn_at(h, i), h->lamG1, flush));
    DH_TRY(dcopy(adj_gas, h->lam_gas, 5 * N3 * sizeof(float), st));
    DH_TRY(part_join(adj_part, h->lam_s, h->lam_p, h, st));
    if (adj_params)
      DH_TRY(launch_param_chain(h, i, i + 1, flush, i, false, true, adj_params, slot));
    return SIM_OK;
  };
  return fail(h, run());
}

sim_status sim_set_tape_recording(sim_t* h, int32_t segments) {
  if (!h || segments < -1) {
    set_error("sim_set_tape_recording: null handle or segments < -1");
    return fail(h, SIM_EINVAL);
  }
  h->tape_segments = segments;
  return SIM_OK;
}

sim_status sim_run(sim_t* h, int32_t n_steps) {
  if (!h) return SIM_EINVAL;
  sim_status r = run_prepare(h, n_steps);
  if (r != SIM_OK) return fail(h, r);
  // the CFL watchdog reads back every step: never captured
  if (h->prm.cfl_max > 0) return fail(h, run_body(h, n_steps));
  return fail(h, run_maybe_graph(h, 1, {(uintptr_t)n_steps, (uintptr_t)recorded_segments(h, 0)},
                                 [&] { return run_body(h, n_steps); }));
}

sim_status sim_run_adjoint(sim_t* h, const float* dL_dgas, const float* dL_dpart,
                           float* dL_dnoise, double* dL_dparams) {
  if (!h) return SIM_EINVAL;
  sim_status r = run_adjoint_prepare(h, dL_dnoise, dL_dparams);
  if (r != SIM_OK) return fail(h, r);
  const std::vector<uintptr_t> key = {(uintptr_t)dL_dgas, (uintptr_t)dL_dpart,
                                      (uintptr_t)dL_dnoise, (uintptr_t)dL_dparams};
  return fail(h, run_maybe_graph(h, 2, key, [&] {
    return run_adjoint_body(h, dL_dgas, dL_dpart, dL_dnoise, dL_dparams);
  }));
}

sim_status sim_reset(sim_t* h) {
  if (!h) return SIM_EINVAL;
  return fail(h, reset_to_init(h));
}

sim_status sim_reinit(sim_t* h, const float* noise) {
  if (!h) return SIM_EINVAL;
  sim_status r = load_noise(h, noise);
  if (r == SIM_OK) r = make_ics(h);
  if (r == SIM_OK) {
    h->ics_valid = true;
    h->init_step = 0;
    r = reset_to_init(h);
  }
  return fail(h, r);
}

sim_status sim_loss_density(sim_t* h, const float* target, double c, float* dL_dgas,
                            double* loss) {
  if (!h || !target || !dL_dgas || !loss) {
    set_error("sim_loss_density: null arguments");
    return fail(h, SIM_EINVAL);
  }
  cudaStream_t st = h->st;
  sim_status r = dzero(dL_dgas, 5 * h->B * h->N3 * sizeof(float), st);
  if (r == SIM_OK) r = dzero(loss, h->B * sizeof(double), st);
  if (r == SIM_OK)
    r = launch_density_loss(h->gas, target, (float)c, dL_dgas, loss, h->N3, h->B, st);
  return fail(h, r);
}

}  // extern "C"

namespace dh {

// Loss of an observable of the current gas state against `target` (B n^3), c sum (o - t)^2,
// with dL/dgas (5 B n^3, fully written) and loss (B doubles, overwritten).
static sim_status field_loss(sim_t* h, int obs, const float* target, double c, float* dL_dgas,
                             double* loss) {
  cudaStream_t st = h->st;
  DH_TRY(dzero(loss, h->B * sizeof(double), st));
  if (obs == SIM_OBS_THERMAL)
    return launch_thermal_loss(h->gas, target, (float)c, dL_dgas, loss, h->N3, h->B, st);
  DH_TRY(dzero(dL_dgas, 5 * h->B * h->N3 * sizeof(float), st));
  return launch_density_loss(h->gas, target, (float)c, dL_dgas, loss, h->N3, h->B, st);
}

// The data term of the posterior of Sec. 3.2 at the amplitudes `noise`: ICs, the whole run,
// loss (B doubles) and its gradient with respect to the amplitudes in h->fli_g.
static sim_status posterior_data_term(sim_t* h, int obs, const float* noise, const float* data,
                                      double sigma_n, double* loss) {
  const long long N3 = h->N3 * h->B;
  if (!h->fli_g) {
    DH_TRY(dalloc_t(h, &h->fli_g, N3));
    DH_TRY(dalloc_t(h, &h->fli_dL, 5 * N3));
    DH_TRY(dalloc_t(h, &h->fli_dpar, (size_t)h->B * SIM_NPARAMS));
  }
  DH_TRY(load_noise(h, noise));
  DH_TRY(make_ics(h));
  h->ics_valid = true;
  h->init_step = 0;
  DH_TRY(reset_to_init(h));
  // the reverse-pass buffers first, so that the run records its last segment on the tape
  DH_TRY(ensure_adjoint_buffers(h, tape_steps_wanted(h)));
  DH_TRY(run_prepare(h, h->prm.n_steps));
  DH_TRY(run_maybe_graph(h, 1, {(uintptr_t)h->prm.n_steps, (uintptr_t)recorded_segments(h, 1)},
                         [&] { return run_body(h, h->prm.n_steps, 1); }));
  DH_TRY(field_loss(h, obs, data, 0.5 / (sigma_n * sigma_n), h->fli_dL, loss));
  DH_TRY(run_adjoint_prepare(h, h->fli_g, h->fli_dpar));
  const std::vector<uintptr_t> key = {(uintptr_t)h->fli_dL, (uintptr_t)0, (uintptr_t)h->fli_g,
                                      (uintptr_t)h->fli_dpar};
  return run_maybe_graph(h, 2, key, [&] {
    return run_adjoint_body(h, h->fli_dL, nullptr, h->fli_g, h->fli_dpar);
  });
}

static sim_status check_posterior_args(sim_t* h, int obs, const void* noise, const void* data,
                                       const void* loss, double sigma_n, const char* who) {
  if (!noise || !data || !loss || !(sigma_n > 0) || (obs != SIM_OBS_DENSITY && obs != SIM_OBS_THERMAL)) {
    set_error("%s: null arrays, sigma_n <= 0 or unknown observable", who);
    return SIM_EINVAL;
  }
  if (h->closure) {
    set_error("%s: not available while a learned closure is set", who);
    return SIM_ENOTIMPL;
  }
  if (h->prm.cfl_max > 0) {
    set_error("%s: needs cfl_max = 0 (the run is differentiated as a whole)", who);
    return SIM_EINVAL;
  }
  return SIM_OK;
}

}  // namespace dh

extern "C" {

sim_status sim_loss_field(sim_t* h, int32_t observable, const float* target, double c,
                          float* dL_dgas, double* loss) {
  if (!h || !target || !dL_dgas || !loss ||
      (observable != SIM_OBS_DENSITY && observable != SIM_OBS_THERMAL)) {
    set_error("sim_loss_field: null arguments or unknown observable");
    return fail(h, SIM_EINVAL);
  }
  return fail(h, field_loss(h, observable, target, c, dL_dgas, loss));
}

// One iteration of field-level inference (Sec. 3.2): the posterior at the amplitudes
// `noise`, its gradient through the whole checkpointed run, and an Adam step on the
// amplitudes. Every stage is a library kernel or cuFFT call on the handle's stream.
sim_status sim_fli_step(sim_t* h, int32_t observable, float* noise, float* m, float* v,
                        const float* data, double sigma_n, double lr, int32_t t, double* loss,
                        float* grad) {
  if (!h) return SIM_EINVAL;
  sim_status r = check_posterior_args(h, observable, noise, data, loss, sigma_n, "sim_fli_step");
  if (r == SIM_OK && (!m || !v || !(lr > 0) || t < 1)) {
    set_error("sim_fli_step: null moments, lr <= 0 or t < 1");
    r = SIM_EINVAL;
  }
  if (r == SIM_OK) r = posterior_data_term(h, observable, noise, data, sigma_n, loss);
  if (r == SIM_OK)
    r = launch_fli_adam(noise, h->fli_g, m, v, h->N3, h->B, lr, 0.9, 0.999, 1e-8, t, 1.0, grad,
                        loss, h->st);
  return fail(h, r);
}

sim_status sim_posterior(sim_t* h, int32_t observable, const float* noise, const float* data,
                         double sigma_n, double* loss, float* grad) {
  if (!h) return SIM_EINVAL;
  sim_status r = check_posterior_args(h, observable, noise, data, loss, sigma_n, "sim_posterior");
  if (r == SIM_OK && !grad) {
    set_error("sim_posterior: null gradient");
    r = SIM_EINVAL;
  }
  if (r == SIM_OK) r = posterior_data_term(h, observable, noise, data, sigma_n, loss);
  if (r == SIM_OK) r = launch_prior_grad(noise, h->fli_g, grad, h->N3, h->B, 1.0, loss, h->st);
  return fail(h, r);
}

sim_status sim_set_diagnostics(sim_t* h, int32_t on) {
  if (!h) return SIM_EINVAL;
  if (on && !h->d_diag_sums) {
    const size_t recs = (size_t)(h->prm.n_steps + 1) * h->B;
    sim_status r = dalloc_t(h, &h->d_diag_sums, recs * DG_NSUM);
    if (r == SIM_OK) r = dalloc_t(h, &h->d_diag_mins, recs * 2);
    if (r != SIM_OK) return fail(h, r);
    h->diag_recorded.assign(h->prm.n_steps + 1, 0);
  }
  if ((on != 0) != h->diag_on) clear_graphs(h);
  h->diag_on = on != 0;
  return SIM_OK;
}

sim_status sim_diagnostics(sim_t* h, int32_t step, double* out) {
  if (!h || !out || step < 0 || step > h->prm.n_steps) {
    set_error("sim_diagnostics: invalid arguments");
    return fail(h, SIM_EINVAL);
  }
  if (!h->d_diag_sums || !h->diag_recorded[step]) {
    set_error("sim_diagnostics: no record of step %d (diagnostics off when it ran?)", step);
    return fail(h, SIM_EINVAL);
  }
  const int B = h->B;
  std::vector<double> sums((size_t)B * DG_NSUM);
  std::vector<int> mins((size_t)B * 2);
  const size_t r = (size_t)step * B;
  DH_CUDA_TRY(cudaStreamSynchronize(h->st));
  DH_CUDA_TRY(cudaMemcpy(sums.data(), h->d_diag_sums + r * DG_NSUM, sums.size() * sizeof(double),
                         cudaMemcpyDeviceToHost));
  DH_CUDA_TRY(cudaMemcpy(mins.data(), h->d_diag_mins + r * 2, mins.size() * sizeof(int),
                         cudaMemcpyDeviceToHost));
  for (int b = 0; b < B; ++b) {
    double* o = out + (size_t)b * SIM_DG_N;
    const double* sb = sums.data() + (size_t)b * DG_NSUM;
    o[SIM_DG_A] = a_of_step(h, step);
    o[SIM_DG_MASS] = sb[DG_S_MASS];
    o[SIM_DG_MX] = sb[DG_S_MX];
    o[SIM_DG_MY] = sb[DG_S_MY];
    o[SIM_DG_MZ] = sb[DG_S_MZ];
    o[SIM_DG_ENERGY] = sb[DG_S_ENERGY];
    o[SIM_DG_PX] = sb[DG_S_PX];
    o[SIM_DG_PY] = sb[DG_S_PY];
    o[SIM_DG_PZ] = sb[DG_S_PZ];
    o[SIM_DG_STARS] = sb[DG_S_STARS];
    o[SIM_DG_EVENTS] = sb[DG_S_EVENTS];
    o[SIM_DG_NONFINITE] = sb[DG_S_NONFINITE];
    o[SIM_DG_RHO_MIN] = ordered_to_float(mins[2 * b]);
    o[SIM_DG_P_MIN] = ordered_to_float(mins[2 * b + 1]);
  }
  return SIM_OK;
}

sim_status sim_get_state(sim_t* h, float* gas, float* part, float* star, float* aux,
                         uint32_t* events, float* gravity, int32_t* step) {
  if (!h) return SIM_EINVAL;
  const long long N3 = h->N3 * h->B;
  const long long words = (h->N3 + 31) / 32 * h->B;
  cudaStream_t st = h->st;
  sim_status r = SIM_OK;
  if (gas && r == SIM_OK) r = dcopy(gas, h->gas, 5 * N3 * sizeof(float), st);
  if (part && r == SIM_OK) r = part_join(part, h->s, h->p, h, st);
  if (star && r == SIM_OK) r = dcopy(star, h->star, N3 * sizeof(float), st);
  if (aux && r == SIM_OK) r = dcopy(aux, h->aux, N3 * sizeof(float), st);
  if (events && r == SIM_OK) r = dcopy(events, h->events, words * sizeof(uint32_t), st);
  if (gravity && r == SIM_OK) r = dcopy(gravity, h->g, 3 * N3 * sizeof(float), st);
  if (step) *step = h->step;
  return fail(h, r);
}

sim_status sim_set_state(sim_t* h, const float* gas, const float* part, int32_t step) {
  if (!h || !gas || !part || step < 0 || step > h->prm.n_steps) {
    set_error("sim_set_state: invalid arguments");
    return fail(h, SIM_EINVAL);
  }
  const long long N3 = h->N3 * h->B;
  cudaStream_t st = h->st;
  sim_status r = dcopy(h->init_gas, gas, 5 * N3 * sizeof(float), st);
  if (r == SIM_OK) r = dcopy(h->init_part, part, 6 * N3 * sizeof(float), st);
  if (r == SIM_OK) {
    h->ics_valid = false;
    h->init_step = step;
    r = reset_to_init(h);
  }
  return fail(h, r);
}

sim_status sim_schedule(const sim_t* h, int32_t i, double* out6) {
  if (!h || !out6 || i < 0 || i >= h->prm.n_steps) {
    set_error("sim_schedule: invalid arguments");
    return SIM_EINVAL;
  }
  const StepFactors& f = h->sched[i];
  out6[0] = f.a0;
  out6[1] = f.a1;
  out6[2] = f.K1;
  out6[3] = f.dtau;
  out6[4] = f.K2;
  out6[5] = f.pref1;
  return SIM_OK;
}

sim_status sim_set_closure(sim_t* h, sim_closure_t* c) {
  if (!h) return SIM_EINVAL;
  clear_graphs(h);
  h->closure = c;
  h->closure_gen = 0;
  if (c) {
    sim_status r = closure_prepare(c, h->n, h->B, false);
    if (r != SIM_OK) {
      h->closure = nullptr;
      return fail(h, r);
    }
    h->closure_gen = closure_generation(c);
  }
  return SIM_OK;
}

sim_status sim_ic_amplitude(const sim_t* h, int32_t b, double* C) {
  if (!h || !C || b < 0 || b >= h->B) {
    set_error("sim_ic_amplitude: invalid arguments");
    return SIM_EINVAL;
  }
  *C = h->inst[b].C;
  return SIM_OK;
}

sim_status sim_cfl(sim_t* h, double* cfl_out) {
  if (!h || !cfl_out) return SIM_EINVAL;
  return fail(h, cfl_now(h, cfl_out));
}

}  // extern "C"

namespace dh {

// Largest CFL number over the instances for the next step (reads back, synchronises).
static sim_status cfl_now(sim_t* h, double* cfl_out) {
  cudaStream_t st = h->st;
  std::vector<unsigned int> bits(h->B, 0u);
  DH_TRY(dzero(h->speed_bits, h->B * sizeof(unsigned int), st));
  DH_TRY(launch_signal_speed(h->gas, (float)h->prm.gamma, h->N3, h->speed_bits, h->B, st));
  if (cudaMemcpyAsync(bits.data(), h->speed_bits, h->B * sizeof(unsigned int),
                      cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    set_error("sim_cfl: readback failed");
    return SIM_ECUDA;
  }
  const int i = h->step < h->prm.n_steps ? h->step : h->prm.n_steps - 1;
  double c = 0.0;
  for (int b = 0; b < h->B; ++b) {
    float v;
    memcpy(&v, &bits[b], sizeof(v));
    const double cb = (double)v * h->scheds[b][i].dtau * h->inv_dx;
    if (std::isnan(cb) || (!std::isnan(c) && cb > c)) c = cb;  // a NaN of any instance wins
  }
  *cfl_out = c;
  return SIM_OK;
}

}  // namespace dh

// ===================================================================== groups of handles
// Batches on grids of different sizes: one batched handle per size, captured together.
// The group's graph forks one branch per member from a private capture stream, runs the
// member's body on its branch stream, and joins the branches again, so the members' kernels
// may overlap on the GPU; one graph launch replays the whole call.
struct GroupEntry {
  int kind = 0;
  std::vector<uintptr_t> key;
  std::vector<HostState> before, after;
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;
};

struct sim_group_s {
  std::vector<sim_t*> m;
  cudaStream_t st = 0, cap = nullptr;
  std::vector<cudaStream_t> br;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr, order = nullptr;
  std::vector<GroupEntry> cache;
};

namespace dh {

static void group_free(sim_group_t* g) {
  for (GroupEntry& e : g->cache)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  for (cudaStream_t s : g->br)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : g->join)
    if (e) cudaEventDestroy(e);
  if (g->fork) cudaEventDestroy(g->fork);
  if (g->order) cudaEventDestroy(g->order);
  if (g->cap) cudaStreamDestroy(g->cap);
  delete g;
}

// Replay the group's graph for (kind, key) from the members' current host states, or
// capture it: body(k) enqueues member k's work on m[k]->st.
template <class Body>
static sim_status group_graph(sim_group_t* g, int kind, const std::vector<uintptr_t>& key,
                              Body body) {
  const size_t K = g->m.size();
  std::vector<HostState> before;
  for (sim_t* h : g->m) before.push_back(snapshot(h));
  for (GroupEntry& e : g->cache) {
    if (e.kind == kind && e.key == key && e.before == before) {
      DH_CUDA_TRY(cudaGraphLaunch(e.exec, g->st));
      for (size_t k = 0; k < K; ++k) restore(g->m[k], e.after[k]);
      g_launches.fetch_add(e.launches, std::memory_order_relaxed);
      return SIM_OK;
    }
  }
  DH_CUDA_TRY(cudaEventRecord(g->order, g->st));
  DH_CUDA_TRY(cudaStreamWaitEvent(g->cap, g->order, 0));
  DH_CUDA_TRY(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
  const long long l0 = g_launches.load();
  sim_status r = SIM_OK;
  cudaError_t ce = cudaEventRecord(g->fork, g->cap);
  for (size_t k = 0; k < K && ce == cudaSuccess; ++k) {
    ce = cudaStreamWaitEvent(g->br[k], g->fork, 0);
    if (ce != cudaSuccess) break;
    cudaStream_t saved = g->m[k]->st;
    g->m[k]->st = g->br[k];
    if (r == SIM_OK) r = body(k);
    g->m[k]->st = saved;
    // every forked branch is joined back, also after a failure, so the capture can end
    ce = cudaEventRecord(g->join[k], g->br[k]);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(g->cap, g->join[k], 0);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(g->cap, &graph);
  if (r != SIM_OK || ce != cudaSuccess || ee != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    for (size_t k = 0; k < K; ++k) restore(g->m[k], before[k]);
    if (r == SIM_OK)
      set_error("group capture failed: %s",
                cudaGetErrorString(ce != cudaSuccess ? ce : ee));
    return r != SIM_OK ? r : SIM_ECUDA;
  }
  GroupEntry e;
  e.kind = kind;
  e.key = key;
  e.before = before;
  for (sim_t* h : g->m) e.after.push_back(snapshot(h));
  e.launches = g_launches.load() - l0;
  ce = cudaGraphInstantiate(&e.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce == cudaSuccess) ce = cudaGraphLaunch(e.exec, g->st);
  if (ce != cudaSuccess) {
    if (e.exec) cudaGraphExecDestroy(e.exec);
    for (size_t k = 0; k < K; ++k) restore(g->m[k], before[k]);
    set_error("group graph instantiate/launch failed: %s", cudaGetErrorString(ce));
    return SIM_ECUDA;
  }
  g->cache.push_back(std::move(e));
  return SIM_OK;
}

}  // namespace dh

extern "C" {

sim_status sim_group_create(sim_t* const* members, int32_t count, void* stream,
                            sim_group_t** out) {
  if (!out || !members || count < 1) {
    set_error("sim_group_create: invalid arguments");
    return SIM_EINVAL;
  }
  *out = nullptr;
  for (int k = 0; k < count; ++k)
    for (int j = 0; j < k; ++j)
      if (!members[k] || members[k] == members[j]) {
        set_error("sim_group_create: null or repeated member %d", k);
        return SIM_EINVAL;
      }
  sim_group_t* g = new sim_group_t();
  g->m.assign(members, members + count);
  g->st = (cudaStream_t)stream;
  bool ok = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->order, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < count && ok; ++k) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) g->br.push_back(s);
    ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (ok) g->join.push_back(e);
  }
  if (!ok) {
    set_error("sim_group_create: stream or event creation failed");
    group_free(g);
    return SIM_ECUDA;
  }
  *out = g;
  return SIM_OK;
}

void sim_group_destroy(sim_group_t* g) {
  if (!g) return;
  cudaStreamSynchronize(g->st);
  group_free(g);
}

sim_status sim_group_run(sim_group_t* g) {
  if (!g) return SIM_EINVAL;
  for (sim_t* h : g->m) {
    if (h->prm.cfl_max > 0) {
      set_error("sim_group_run: members with cfl_max > 0 read back every step");
      return fail(h, SIM_EINVAL);
    }
    if (h->closure) {
      set_error("sim_group_run: members with a learned closure are run on their own");
      return fail(h, SIM_ENOTIMPL);
    }
    DH_TRY(fail(h, run_prepare(h, h->prm.n_steps - h->step)));
  }
  std::vector<uintptr_t> key;
  for (sim_t* h : g->m) {
    key.push_back((uintptr_t)(h->prm.n_steps - h->step));
    key.push_back((uintptr_t)recorded_segments(h, 0));
  }
  return group_graph(g, 1, key, [&](size_t k) {
    sim_t* h = g->m[k];
    return fail(h, run_body(h, h->prm.n_steps - h->step));
  });
}

sim_status sim_group_run_adjoint(sim_group_t* g, const float* const* dL_dgas,
                                 double* const* dL_dparams) {
  if (!g || !dL_dparams) {
    set_error("sim_group_run_adjoint: null arguments");
    return SIM_EINVAL;
  }
  const size_t K = g->m.size();
  for (size_t k = 0; k < K; ++k)
    DH_TRY(fail(g->m[k], run_adjoint_prepare(g->m[k], nullptr, dL_dparams[k])));
  std::vector<uintptr_t> key;
  for (size_t k = 0; k < K; ++k) {
    key.push_back((uintptr_t)(dL_dgas ? dL_dgas[k] : nullptr));
    key.push_back((uintptr_t)dL_dparams[k]);
  }
  return group_graph(g, 2, key, [&](size_t k) {
    sim_t* h = g->m[k];
    return fail(h, run_adjoint_body(h, dL_dgas ? dL_dgas[k] : nullptr, nullptr, nullptr,
                                    dL_dparams[k]));
  });
}

sim_status sim_group_reset(sim_group_t* g) {
  if (!g) return SIM_EINVAL;
  for (sim_t* h : g->m) DH_TRY(sim_reset(h));
  return SIM_OK;
}

}  // extern "C"
