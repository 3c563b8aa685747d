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

sim_status launch_sweep(int axis, const float* uin, float* uout, int n, double nu, double gam,
                        double eps, cudaStream_t st);
sim_status launch_sweep_adjoint(int axis, const float* uin, const float* lout, float* lin,
                                int n, double nu, double gam, double eps, double* dnu,
                                float* scratch, cudaStream_t st);
sim_status prepare_sweep_kernels();

static const char* kOrders[6] = {"xyz", "zyx", "zxy", "yxz", "yzx", "xzy"};

// per-step partial sums of the reverse pass (doubles on the device), and the chain-rule
// coefficient of each with respect to Omega_m
enum { SL_DK1 = 0, SL_DK2, SL_DNU, SL_DDTAU, SL_DPREF, SL_DCM, SL_DFB, SL_N = 8 };
// extra global partials after the SIM_NPARAMS subgrid ones
enum { GX_DRP = 0, GX_DFB_IC = 1, GX_LAMC = 2, GX_N = 8 };

// One recorded step: inputs of every stage (pointers into the tape allocation).
struct TapeSlot {
  float *U0, *Uk1, *Us1, *Us2, *Us3, *Usg;  // 5 n^3 each
  float *s0, *p0, *g0, *s1, *g1;            // 3 n^3 each
};
constexpr int kTapeFloatsPerCell = 6 * 5 + 5 * 3;

// Host-side state that a call changes; a replayed graph must start from and end in the
// same values as the captured call.
struct HostState {
  int step, init_step, prev_step, ckpt_count;
  bool ics_valid;
  float *gas, *gas2, *w_gas, *w_gas2, *lam_gas, *lam_tmp, *lamG0, *lamG1;
  std::vector<int> ckpt_step;
  bool operator==(const HostState& o) const {
    return step == o.step && init_step == o.init_step && prev_step == o.prev_step &&
           ckpt_count == o.ckpt_count && ics_valid == o.ics_valid && gas == o.gas &&
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
  sim_params prm;
  int n = 0;
  long long N3 = 0, NC = 0;
  cudaStream_t st = 0;
  double dx = 0, inv_dx = 0, fb = 0, cm = 0, dfb_dom = 0;
  std::vector<StepFactors> sched;
  // ICs constants
  double C = 0, dlnC_dom = 0, rp = 0, drp_dom = 0, a2e0 = 0;
  FFTPlans plans;
  // state
  float *gas = nullptr, *gas2 = nullptr, *s = nullptr, *p = nullptr, *g = nullptr;
  float *star = nullptr, *aux = nullptr, *zhat = nullptr, *delta = nullptr;
  uint32_t* events = nullptr;
  unsigned long long* acc = nullptr;
  cufftComplex* ck = nullptr;  // 5 NC complex scratch
  float *noise = nullptr, *f4 = nullptr;
  float *init_gas = nullptr, *init_part = nullptr;
  float *prev_gas = nullptr, *prev_part = nullptr;
  int prev_step = -1;
  bool ics_valid = false;
  int init_step = 0;
  int step = 0;
  // checkpoints: a pool of buffers (11 n^3 floats each) allocated on first use
  std::vector<float*> ckpt_pool;
  std::vector<int> ckpt_step;
  int ckpt_count = 0;
  // tape and adjoint scratch (allocated on first use)
  float* tape = nullptr;
  int tape_cap = 0;
  float *w_gas = nullptr, *w_gas2 = nullptr, *w_s = nullptr, *w_p = nullptr, *w_g = nullptr;
  float *lam_gas = nullptr, *lam_tmp = nullptr, *lam_s = nullptr, *lam_p = nullptr;
  float *lamG0 = nullptr, *lamG1 = nullptr, *lam_delta = nullptr, *lam4 = nullptr;
  float* lam_scr = nullptr;  // 5 n^3 scratch of the marching sweep adjoint
  double* dslots = nullptr;  // (n_steps + 2) x SL_N
  double* dcoef = nullptr;   // (n_steps) x SL_N chain-rule coefficients
  double* dglob = nullptr;   // SIM_NPARAMS + GX_N
  unsigned int* speed_bits = nullptr;
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
  s.ics_valid = h->ics_valid;
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

// total matter contrast from particles and gas, then the force field g (3 n^3)
static sim_status compute_force(sim_t* h, const float* s, const float* gas, double pref,
                                float* g) {
  if (!h->prm.gravity_on) return dzero(g, 3 * h->N3 * sizeof(float), h->st);
  DH_TRY(launch_deposit(s, nullptr, h->n, (float)h->inv_dx, h->acc, h->st));
  DH_TRY(launch_fix_to_float(h->acc, (float)h->cm, gas, -1.0f, h->delta, h->n, h->st));
  return launch_gravity(h->delta, g, h->ck, h->ck + h->NC, h->n, h->prm.box, pref, h->plans,
                        h->st);
}

// One forward step in place on (gas/gas_tmp ping-pong, s, p, g). With tape != nullptr the
// inputs of every stage are recorded; diagnostics (star, aux, events) only without tape.
static sim_status forward_step(sim_t* h, int i, float** gas, float** gas_tmp, float* s, float* p,
                               float* g, const TapeSlot* T) {
  const StepFactors& f = h->sched[i];
  const sim_params& P = h->prm;
  cudaStream_t st = h->st;
  const size_t gb = 5 * h->N3 * sizeof(float), vb = 3 * h->N3 * sizeof(float);
  const float K1 = P.gravity_on ? (float)f.K1 : 0.0f;
  const float K2 = P.gravity_on ? (float)f.K2 : 0.0f;
  if (T) {
    DH_TRY(dcopy(T->U0, *gas, gb, st));
    DH_TRY(dcopy(T->s0, s, vb, st));
    DH_TRY(dcopy(T->p0, p, vb, st));
    DH_TRY(dcopy(T->g0, g, vb, st));
  }
  // 1. half kick + drift
  DH_TRY(launch_kick_drift(s, p, g, K1, (float)f.dtau, nullptr, nullptr, h->n,
                           (float)h->inv_dx, st));
  float* cur = *gas;
  if (T) {
    DH_TRY(dcopy(T->Uk1, cur, gb, st));
    cur = T->Uk1;
  }
  if (P.gravity_on) DH_TRY(launch_gas_kick(cur, g, K1, h->n, st));
  // 2. sweeps
  if (P.hydro_on) {
    const char* order = kOrders[i % 6];
    const double nu = f.dtau * h->inv_dx;
    float* outs_tape[3] = {T ? T->Us1 : nullptr, T ? T->Us2 : nullptr, T ? T->Us3 : nullptr};
    for (int k = 0; k < 3; ++k) {
      float* out = T ? outs_tape[k] : (cur == *gas ? *gas_tmp : *gas);
      DH_TRY(timed(h, SIM_KT_SWEEP, [&] {
        return launch_sweep(order[k] - 'x', cur, out, h->n, nu, P.gamma, P.limiter_eps, st);
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
    const SubgridConst c = make_subgrid_const(P, f.a1, i);
    float* out = T ? T->Usg : cur;
    zh = T ? nullptr : h->zhat;
    DH_TRY(launch_subgrid(cur, out, c, zh, T ? nullptr : h->events, h->N3, st));
    cur = out;
  } else if (T) {
    DH_TRY(dcopy(T->Usg, cur, gb, st));
    cur = T->Usg;
  }
  // 4. force at a_{i+1}
  DH_TRY(compute_force(h, s, cur, f.pref1, g));
  if (T) {
    DH_TRY(dcopy(T->s1, s, vb, st));
    DH_TRY(dcopy(T->g1, g, vb, st));
    DH_TRY(dcopy(*gas, cur, gb, st));
    cur = *gas;
  } else if (cur != *gas) {
    float* t = *gas;
    *gas = *gas_tmp;
    *gas_tmp = t;
  }
  // 5. half kick (+ star readout on the particles)
  DH_TRY(launch_kick_drift(s, p, g, K2, 0.0f, zh, zh ? h->aux : nullptr, h->n,
                           (float)h->inv_dx, st));
  if (P.gravity_on) DH_TRY(launch_gas_kick(*gas, g, K2, h->n, st));
  if (zh) DH_TRY(launch_axpy(1.0f, zh, h->star, h->N3, st));
  return SIM_OK;
}

static sim_status ensure_adjoint_buffers(sim_t* h, int tape_steps) {
  const long long N3 = h->N3;
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
    DH_TRY(dalloc_t(h, &h->lamG0, 3 * N3));
    DH_TRY(dalloc_t(h, &h->lamG1, 3 * N3));
    DH_TRY(dalloc_t(h, &h->lam_delta, N3));
    DH_TRY(dalloc_t(h, &h->lam4, 4 * N3));
    DH_TRY(dalloc_t(h, &h->lam_scr, 5 * N3));
    DH_TRY(dalloc_t(h, &h->dglob, SIM_NPARAMS + GX_N));
    DH_TRY(dalloc_t(h, &h->dslots, (size_t)(h->prm.n_steps + 2) * SL_N));
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
    DH_TRY(dalloc_t(h, &h->tape, (size_t)tape_steps * kTapeFloatsPerCell * N3));
    h->tape_cap = tape_steps;
  }
  return SIM_OK;
}

static TapeSlot tape_slot(sim_t* h, int k) {
  const long long N3 = h->N3;
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
  return t;
}

// Adjoint of the force field g = G(s, rho) at one state: lam_G (3 n^3, consumed) ->
// lam_rho += ..., lam_s += ...; slot[SL_DPREF] += lam_G . g, slot[SL_DCM] += d/d(1 - f_b).
static sim_status force_adjoint(sim_t* h, const float* s, const float* g, double pref,
                                float* lamG, double* slot) {
  if (!h->prm.gravity_on) return SIM_OK;
  cudaStream_t st = h->st;
  DH_TRY(launch_dot(lamG, g, 3 * h->N3, slot + SL_DPREF, st));
  DH_TRY(launch_gravity_adjoint(lamG, h->lam_delta, h->ck, h->ck + 3 * h->NC, h->n,
                                h->prm.box, pref, h->plans, st));
  DH_TRY(launch_axpy(1.0f, h->lam_delta, h->lam_gas, h->N3, st));
  return launch_deposit_adjoint(s, h->lam_delta, (float)h->cm, h->lam_s, slot + SL_DCM, h->n,
                                (float)h->inv_dx, st);
}

// Reverse of forward_step for step i with tape T. In: lam_gas / lam_s / lam_p of the state
// after the step, lamG1 = adjoint of g(a_{i+1}) carried from step i+1. Out: the same
// buffers for the state before the step, lamG1 = adjoint of g(a_i) (to carry).
static sim_status reverse_step(sim_t* h, int i, const TapeSlot& T, double* slot) {
  const StepFactors& f = h->sched[i];
  const sim_params& P = h->prm;
  cudaStream_t st = h->st;
  const float K1 = P.gravity_on ? (float)f.K1 : 0.0f;
  const float K2 = P.gravity_on ? (float)f.K2 : 0.0f;
  // 5. second half kick
  if (P.gravity_on) {
    DH_TRY(launch_gas_kick_adjoint(T.Usg, T.g1, K2, h->lam_gas, h->lamG1, slot + SL_DK2, h->n, st));
    DH_TRY(launch_kick_drift_adjoint(T.s1, nullptr, T.g1, K2, 0.0f, h->lam_s, h->lam_p, h->lamG1,
                                     slot + SL_DK2, nullptr, h->n, (float)h->inv_dx, st));
    // 4. force at a_{i+1}
    DH_TRY(force_adjoint(h, T.s1, T.g1, f.pref1, h->lamG1, slot));
  }
  // 3. subgrid
  if (P.subgrid_on) {
    const SubgridConst c = make_subgrid_const(P, f.a1, i);
    DH_TRY(launch_subgrid_adjoint(T.Us3, h->lam_gas, c, h->dglob, slot + SL_DFB, h->N3, st));
  }
  // 2. sweeps in reverse
  if (P.hydro_on) {
    const char* order = kOrders[i % 6];
    const double nu = f.dtau * h->inv_dx;
    const float* ins[3] = {T.Uk1, T.Us1, T.Us2};
    for (int k = 2; k >= 0; --k) {
      DH_TRY(timed(h, SIM_KT_SWEEP_ADJOINT, [&] {
        return launch_sweep_adjoint(order[k] - 'x', ins[k], h->lam_gas, h->lam_tmp, h->n, nu,
                                    P.gamma, P.limiter_eps, slot + SL_DNU, h->lam_scr, st);
      }));
      float* t = h->lam_gas;
      h->lam_gas = h->lam_tmp;
      h->lam_tmp = t;
    }
  }
  // 1. first half kick and drift
  DH_TRY(dzero(h->lamG0, 3 * h->N3 * sizeof(float), st));
  if (P.gravity_on)
    DH_TRY(launch_gas_kick_adjoint(T.U0, T.g0, K1, h->lam_gas, h->lamG0, slot + SL_DK1, h->n, st));
  DH_TRY(launch_kick_drift_adjoint(T.s0, T.p0, T.g0, K1, (float)f.dtau, h->lam_s, h->lam_p,
                                   h->lamG0, slot + SL_DK1, slot + SL_DDTAU, h->n,
                                   (float)h->inv_dx, st));
  float* t = h->lamG0;
  h->lamG0 = h->lamG1;
  h->lamG1 = t;  // carry: lamG1 now holds the adjoint of g(a_i)
  return SIM_OK;
}

// dL/dparams from the device partials: d/dOmega_m = sum over step slots of slot * coef
// (schedule derivatives, host FP64, uploaded once) + the flush slot (force at the start of
// the differentiated span) + the IC terms; sigma8 from the IC amplitude; the subgrid
// parameters pass through. out is overwritten, or accumulated when `accumulate`.
__global__ void param_chain_kernel(const double* __restrict__ slots,
                                   const double* __restrict__ coef, int nvals,
                                   const double* __restrict__ flush, double c_pref0,
                                   double c_cm0, const double* __restrict__ glob,
                                   double dlnC, double drp, double dfb, double inv_s8, int ics,
                                   int accumulate, double* __restrict__ out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nvals; i += blockDim.x) acc += slots[i] * coef[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double dom = red[0] + flush[SL_DPREF] * c_pref0 + flush[SL_DCM] * c_cm0;
    double ds8 = 0.0;
    if (ics) {
      const double* gx = glob + SIM_NPARAMS;
      dom += gx[GX_LAMC] * dlnC + gx[GX_DRP] * drp + gx[GX_DFB_IC] * dfb;
      ds8 = gx[GX_LAMC] * inv_s8;
    }
    double v[SIM_NPARAMS];
    v[SIM_P_OMEGA_M] = dom;
    v[SIM_P_SIGMA8] = ds8;
    for (int k = SIM_P_DELTA_C; k < SIM_NPARAMS; ++k) v[k] = glob[k];
    for (int k = 0; k < SIM_NPARAMS; ++k) out[k] = accumulate ? out[k] + v[k] : v[k];
  }
}

static sim_status launch_param_chain(sim_t* h, int first, int last, const double* flush,
                                     double a_flush, bool ics, bool accumulate, double* out,
                                     const double* slots_first) {
  const int nvals = (last - first) * SL_N;
  const double pref0 = 1.5 * h->prm.omega_m / a_flush;
  const double c_pref0 = (1.5 / a_flush) / pref0;
  param_chain_kernel<<<1, 256, 0, h->st>>>(slots_first, h->dcoef + (size_t)first * SL_N, nvals,
                                           flush, c_pref0, -h->dfb_dom, h->dglob, h->dlnC_dom,
                                           h->drp_dom, h->dfb_dom, 1.0 / h->prm.sigma8, ics ? 1 : 0,
                                           accumulate ? 1 : 0, out);
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

static sim_status alloc_state(sim_t* h) {
  const long long N3 = h->N3, NC = h->NC;
  DH_TRY(dalloc_t(h, &h->gas, 5 * N3));
  DH_TRY(dalloc_t(h, &h->gas2, 5 * N3));
  DH_TRY(dalloc_t(h, &h->s, 3 * N3));
  DH_TRY(dalloc_t(h, &h->p, 3 * N3));
  DH_TRY(dalloc_t(h, &h->g, 3 * N3));
  DH_TRY(dalloc_t(h, &h->star, N3));
  DH_TRY(dalloc_t(h, &h->aux, N3));
  DH_TRY(dalloc_t(h, &h->zhat, N3));
  DH_TRY(dalloc_t(h, &h->delta, N3));
  DH_TRY(dalloc_t(h, &h->events, (N3 + 31) / 32));
  DH_TRY(dalloc_t(h, &h->acc, N3));
  DH_TRY(dalloc_t(h, &h->ck, 5 * NC));
  DH_TRY(dalloc_t(h, &h->noise, N3));
  DH_TRY(dalloc_t(h, &h->f4, 4 * N3));
  DH_TRY(dalloc_t(h, &h->init_gas, 5 * N3));
  DH_TRY(dalloc_t(h, &h->init_part, 6 * N3));
  DH_TRY(dalloc_t(h, &h->prev_gas, 5 * N3));
  DH_TRY(dalloc_t(h, &h->prev_part, 6 * N3));
  DH_TRY(dalloc_t(h, &h->speed_bits, 1));
  DH_TRY(dalloc_t(h, &h->dcoef, (size_t)h->prm.n_steps * SL_N));
  DH_TRY(dzero(h->acc, N3 * sizeof(unsigned long long), h->st));
  DH_TRY(dzero(h->events, ((N3 + 31) / 32) * sizeof(uint32_t), h->st));
  // chain-rule coefficients of the per-step partials with respect to Omega_m
  std::vector<double> coef((size_t)h->prm.n_steps * SL_N, 0.0);
  for (int i = 0; i < h->prm.n_steps; ++i) {
    const StepFactors& f = h->sched[i];
    double* c = coef.data() + (size_t)i * SL_N;
    c[SL_DK1] = f.dK1;
    c[SL_DK2] = f.dK2;
    c[SL_DNU] = f.ddtau * h->inv_dx;
    c[SL_DDTAU] = f.ddtau;
    c[SL_DPREF] = f.dpref1 / f.pref1;
    c[SL_DCM] = -h->dfb_dom;
    c[SL_DFB] = h->dfb_dom;
  }
  DH_CUDA_TRY(cudaMemcpy(h->dcoef, coef.data(), coef.size() * sizeof(double),
                         cudaMemcpyHostToDevice));
  return SIM_OK;
}

static void clear_checkpoints(sim_t* h) { h->ckpt_count = 0; }

static sim_status ensure_ckpt_pool(sim_t* h, int count) {
  while ((int)h->ckpt_pool.size() < count) {
    float* c = nullptr;
    DH_TRY(dalloc_t(h, &c, 11 * h->N3));
    h->ckpt_pool.push_back(c);
    h->ckpt_step.push_back(0);
  }
  return SIM_OK;
}

static sim_status reset_to_init(sim_t* h) {
  const long long N3 = h->N3;
  cudaStream_t st = h->st;
  DH_TRY(dcopy(h->gas, h->init_gas, 5 * N3 * sizeof(float), st));
  DH_TRY(dcopy(h->s, h->init_part, 3 * N3 * sizeof(float), st));
  DH_TRY(dcopy(h->p, h->init_part + 3 * N3, 3 * N3 * sizeof(float), st));
  DH_TRY(dzero(h->star, N3 * sizeof(float), st));
  DH_TRY(dzero(h->aux, N3 * sizeof(float), st));
  h->step = h->init_step;
  DH_TRY(compute_force(h, h->s, h->gas, 1.5 * h->prm.omega_m / a_of_step(h, h->init_step), h->g));
  clear_checkpoints(h);
  h->prev_step = -1;
  return SIM_OK;
}

static sim_status store_checkpoint(sim_t* h) {
  const long long N3 = h->N3;
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

sim_status sim_init(const sim_params* p, const float* noise, void* stream, sim_t** out) {
  if (!out) {
    set_error("sim_init: out is NULL");
    return SIM_EINVAL;
  }
  *out = nullptr;
  DH_TRY(validate(p));
  sim_t* h = new sim_t();
  h->prm = *p;
  h->n = p->n;
  h->N3 = (long long)p->n * p->n * p->n;
  h->NC = (long long)p->n * p->n * (p->n / 2 + 1);
  h->st = (cudaStream_t)stream;
  h->dx = p->box / p->n;
  h->inv_dx = p->n / p->box;
  h->fb = p->omega_b / p->omega_m;
  h->cm = 1.0 - h->fb;
  h->dfb_dom = -h->fb / p->omega_m;
  h->sched = make_schedule(p->a_start, p->a_end, p->n_steps, p->omega_m, p->kdk_mode);
  // IC constants (Sec. 2.1): C = rms_target sqrt(n^3 / sum_k P(k))
  {
    const int n = p->n;
    const double kf = 2.0 * M_PI / p->box, kc = p->kc_frac * M_PI * n / p->box;
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
    const double Di = growth_D(p->a_start, p->omega_m);
    const double rms = p->rms_ref * (p->sigma8 / p->sigma8_ref) * Di /
                       growth_D(p->a_ref, p->omega_m_ref);
    h->C = rms * std::sqrt((double)n * n * n / total);
    const double hh = 1e-5 * p->omega_m;
    h->dlnC_dom = (growth_D(p->a_start, p->omega_m + hh) - growth_D(p->a_start, p->omega_m - hh)) /
                  (2 * hh) / Di;
    auto rpf = [&](double om) { return growth_gp(p->a_start, om) / growth_D(p->a_start, om); };
    h->rp = rpf(p->omega_m);
    h->drp_dom = (rpf(p->omega_m + hh) - rpf(p->omega_m - hh)) / (2 * hh);
    const double e0 = p->T_init / temperature_per_energy(p->gamma, p->mu);
    h->a2e0 = p->a_start * p->a_start * e0;
  }
  sim_status r = prepare_sweep_kernels();
  if (r == SIM_OK) r = h->plans.create(p->n);
  if (r == SIM_OK) r = alloc_state(h);
  if (r == SIM_OK && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    set_error("cudaStreamCreate failed");
    r = SIM_ECUDA;
  }
  cudaStream_t st = h->st;
  if (r == SIM_OK) {
    if (noise)
      r = dcopy(h->noise, noise, h->N3 * sizeof(float), st);
    else
      r = launch_noise(p->seed, p->instance, h->noise, h->N3, st);
  }
  if (r == SIM_OK)
    r = launch_linear_field(h->noise, h->f4, h->ck, p->n, p->box, p->kc_frac, h->C, h->plans, st);
  if (r == SIM_OK) r = launch_place(h->f4, h->gas, h->s, h->p, h->rp, h->fb, h->a2e0, h->N3, st);
  if (r == SIM_OK) r = dcopy(h->init_gas, h->gas, 5 * h->N3 * sizeof(float), st);
  if (r == SIM_OK) r = dcopy(h->init_part, h->s, 3 * h->N3 * sizeof(float), st);
  if (r == SIM_OK) r = dcopy(h->init_part + 3 * h->N3, h->p, 3 * h->N3 * sizeof(float), st);
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

void sim_destroy(sim_t* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  if (h->cap_stream) cudaStreamSynchronize(h->cap_stream);
  clear_graphs(h);
  for (cudaEvent_t e : h->kt_ev) cudaEventDestroy(e);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  h->plans.destroy();
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

sim_status sim_step(sim_t* h) {
  if (!h) return SIM_EINVAL;
  if (h->step >= h->prm.n_steps) {
    set_error("sim_step: already at the last step (%d)", h->prm.n_steps);
    return fail(h, SIM_EINVAL);
  }
  const long long N3 = h->N3;
  sim_status r = dcopy(h->prev_gas, h->gas, 5 * N3 * sizeof(float), h->st);
  if (r == SIM_OK) r = dcopy(h->prev_part, h->s, 3 * N3 * sizeof(float), h->st);
  if (r == SIM_OK) r = dcopy(h->prev_part + 3 * N3, h->p, 3 * N3 * sizeof(float), h->st);
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
  const long long N3 = h->N3;
  cudaStream_t st = h->st;
  const int i = h->prev_step;
  sim_status r = ensure_adjoint_buffers(h, 1);
  if (r != SIM_OK) return fail(h, r);
  const TapeSlot T = tape_slot(h, 0);
  double* slot = h->dslots;
  const double a0 = h->sched[i].a0;
  auto run = [&]() -> sim_status {
    DH_TRY(dzero(h->dslots, 2 * SL_N * sizeof(double), st));
    DH_TRY(dzero(h->dglob, (SIM_NPARAMS + GX_N) * sizeof(double), st));
    // recompute the step from its input with the tape
    DH_TRY(dcopy(h->w_gas, h->prev_gas, 5 * N3 * sizeof(float), st));
    DH_TRY(dcopy(h->w_s, h->prev_part, 3 * N3 * sizeof(float), st));
    DH_TRY(dcopy(h->w_p, h->prev_part + 3 * N3, 3 * N3 * sizeof(float), st));
    DH_TRY(compute_force(h, h->w_s, h->w_gas, 1.5 * h->prm.omega_m / a0, h->w_g));
    DH_TRY(forward_step(h, i, &h->w_gas, &h->w_gas2, h->w_s, h->w_p, h->w_g, &T));
    // reverse
    DH_TRY(dcopy(h->lam_gas, adj_gas, 5 * N3 * sizeof(float), st));
    DH_TRY(dcopy(h->lam_s, adj_part, 3 * N3 * sizeof(float), st));
    DH_TRY(dcopy(h->lam_p, adj_part + 3 * N3, 3 * N3 * sizeof(float), st));
    DH_TRY(dzero(h->lamG1, 3 * N3 * sizeof(float), st));
    DH_TRY(reverse_step(h, i, T, slot));
    // g(a_i) is a function of the input state: flush its adjoint now
    DH_TRY(force_adjoint(h, T.s0, T.g0, 1.5 * h->prm.omega_m / a0, h->lamG1, slot + SL_N));
    DH_TRY(dcopy(adj_gas, h->lam_gas, 5 * N3 * sizeof(float), st));
    DH_TRY(dcopy(adj_part, h->lam_s, 3 * N3 * sizeof(float), st));
    DH_TRY(dcopy(adj_part + 3 * N3, h->lam_p, 3 * N3 * sizeof(float), st));
    if (adj_params)
      DH_TRY(launch_param_chain(h, i, i + 1, slot + SL_N, a0, false, true, adj_params, slot));
    return SIM_OK;
  };
  return fail(h, run());
}

sim_status sim_run(sim_t* h, int32_t n_steps) {
  if (!h) return SIM_EINVAL;
  if (h->step != h->init_step || h->ckpt_count != 0) {
    set_error("sim_run: the handle must be at its initial state (sim_init / sim_reset)");
    return fail(h, SIM_EINVAL);
  }
  if (n_steps < 0 || h->step + n_steps > h->prm.n_steps) {
    set_error("sim_run: n_steps out of range");
    return fail(h, SIM_EINVAL);
  }
  sim_status r = ensure_ckpt_pool(h, (n_steps + h->prm.ckpt_every - 1) / h->prm.ckpt_every);
  if (r != SIM_OK) return fail(h, r);
  auto body = [&]() -> sim_status {
    for (int k = 0; k < n_steps; ++k) {
      if ((h->step - h->init_step) % h->prm.ckpt_every == 0) DH_TRY(store_checkpoint(h));
      DH_TRY(forward_step(h, h->step, &h->gas, &h->gas2, h->s, h->p, h->g, nullptr));
      h->step += 1;
      if (h->prm.cfl_max > 0 && h->step < h->prm.n_steps) {
        double c = 0;
        DH_TRY(sim_cfl(h, &c));
        if (!(c <= h->prm.cfl_max)) {
          set_error("sim_run: CFL number %.4g above cfl_max %.4g after step %d", c,
                    h->prm.cfl_max, h->step);
          return std::isfinite(c) ? SIM_ECFL : SIM_ENAN;
        }
      }
    }
    h->prev_step = -1;
    return SIM_OK;
  };
  // the CFL watchdog reads back every step: never captured
  if (h->prm.cfl_max > 0) return fail(h, body());
  return fail(h, run_maybe_graph(h, 1, {(uintptr_t)n_steps}, body));
}

sim_status sim_run_adjoint(sim_t* h, const float* dL_dgas, const float* dL_dpart,
                           float* dL_dnoise, double* dL_dparams) {
  if (!h || !dL_dparams) {
    set_error("sim_run_adjoint: null arguments");
    return fail(h, SIM_EINVAL);
  }
  if (h->ckpt_count == 0) {
    set_error("sim_run_adjoint: no sim_run to differentiate");
    return fail(h, SIM_EINVAL);
  }
  if (!h->ics_valid && dL_dnoise) {
    set_error("sim_run_adjoint: the run did not start from initial conditions");
    return fail(h, SIM_EINVAL);
  }
  const long long N3 = h->N3;
  sim_status r = ensure_adjoint_buffers(h, h->prm.ckpt_every);
  if (r != SIM_OK) return fail(h, r);
  const int nseg = h->ckpt_count;
  const int last = h->step;
  auto body = [&]() -> sim_status {
    cudaStream_t st = h->st;
    DH_TRY(dzero(h->dslots, (size_t)(h->prm.n_steps + 2) * SL_N * sizeof(double), st));
    DH_TRY(dzero(h->dglob, (SIM_NPARAMS + GX_N) * sizeof(double), st));
    if (dL_dgas)
      DH_TRY(dcopy(h->lam_gas, dL_dgas, 5 * N3 * sizeof(float), st));
    else
      DH_TRY(dzero(h->lam_gas, 5 * N3 * sizeof(float), st));
    if (dL_dpart) {
      DH_TRY(dcopy(h->lam_s, dL_dpart, 3 * N3 * sizeof(float), st));
      DH_TRY(dcopy(h->lam_p, dL_dpart + 3 * N3, 3 * N3 * sizeof(float), st));
    } else {
      DH_TRY(dzero(h->lam_s, 3 * N3 * sizeof(float), st));
      DH_TRY(dzero(h->lam_p, 3 * N3 * sizeof(float), st));
    }
    DH_TRY(dzero(h->lamG1, 3 * N3 * sizeof(float), st));
    for (int seg = nseg - 1; seg >= 0; --seg) {
      const int first = h->ckpt_step[seg];
      const int end = seg + 1 < nseg ? h->ckpt_step[seg + 1] : last;
      const float* c = h->ckpt_pool[seg];
      DH_TRY(dcopy(h->w_gas, c, 5 * N3 * sizeof(float), st));
      DH_TRY(dcopy(h->w_s, c + 5 * N3, 3 * N3 * sizeof(float), st));
      DH_TRY(dcopy(h->w_p, c + 8 * N3, 3 * N3 * sizeof(float), st));
      DH_TRY(compute_force(h, h->w_s, h->w_gas, 1.5 * h->prm.omega_m / a_of_step(h, first), h->w_g));
      for (int i = first; i < end; ++i) {
        const TapeSlot T = tape_slot(h, i - first);
        DH_TRY(forward_step(h, i, &h->w_gas, &h->w_gas2, h->w_s, h->w_p, h->w_g, &T));
      }
      for (int i = end - 1; i >= first; --i)
        DH_TRY(reverse_step(h, i, tape_slot(h, i - first), h->dslots + (size_t)i * SL_N));
    }
    // g at the start of the run is a function of the initial state
    const TapeSlot T0 = tape_slot(h, 0);
    const int s0 = h->ckpt_step[0];
    const double a0 = a_of_step(h, s0);
    double* slot0 = h->dslots + (size_t)h->prm.n_steps * SL_N;
    DH_TRY(force_adjoint(h, T0.s0, T0.g0, 1.5 * h->prm.omega_m / a0, h->lamG1, slot0));
    // through the initial conditions to the white noise
    if (h->ics_valid) {
      double* gx = h->dglob + SIM_NPARAMS;
      DH_TRY(launch_ic_adjoint(h->f4, h->lam_gas, h->lam_s, h->lam_p, h->lam4, dL_dnoise, h->ck,
                               h->n, h->prm.box, h->prm.kc_frac, h->C, h->rp, h->fb, h->a2e0,
                               gx + GX_DRP, gx + GX_DFB_IC, h->plans, st));
      DH_TRY(launch_dot(h->lam4, h->f4, 4 * N3, gx + GX_LAMC, st));
    }
    return launch_param_chain(h, s0, last, slot0, a0, h->ics_valid, false, dL_dparams,
                              h->dslots + (size_t)s0 * SL_N);
  };
  const std::vector<uintptr_t> key = {(uintptr_t)dL_dgas, (uintptr_t)dL_dpart,
                                      (uintptr_t)dL_dnoise, (uintptr_t)dL_dparams};
  return fail(h, run_maybe_graph(h, 2, key, body));
}

sim_status sim_reset(sim_t* h) {
  if (!h) return SIM_EINVAL;
  return fail(h, reset_to_init(h));
}

sim_status sim_reinit(sim_t* h, const float* noise) {
  if (!h) return SIM_EINVAL;
  cudaStream_t st = h->st;
  const long long N3 = h->N3;
  sim_status r = noise ? dcopy(h->noise, noise, N3 * sizeof(float), st)
                       : launch_noise(h->prm.seed, h->prm.instance, h->noise, N3, st);
  if (r == SIM_OK)
    r = launch_linear_field(h->noise, h->f4, h->ck, h->n, h->prm.box, h->prm.kc_frac, h->C,
                            h->plans, st);
  if (r == SIM_OK)
    r = launch_place(h->f4, h->init_gas, h->init_part, h->init_part + 3 * N3, h->rp, h->fb,
                     h->a2e0, N3, st);
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
  sim_status r = dzero(dL_dgas + h->N3, 4 * h->N3 * sizeof(float), st);
  if (r == SIM_OK) r = dzero(loss, sizeof(double), st);
  if (r == SIM_OK) r = launch_density_loss(h->gas, target, (float)c, dL_dgas, loss, h->N3, st);
  return fail(h, r);
}

sim_status sim_get_state(sim_t* h, float* gas, float* part, float* star, float* aux,
                         uint32_t* events, float* gravity, int32_t* step) {
  if (!h) return SIM_EINVAL;
  const long long N3 = h->N3;
  cudaStream_t st = h->st;
  sim_status r = SIM_OK;
  if (gas && r == SIM_OK) r = dcopy(gas, h->gas, 5 * N3 * sizeof(float), st);
  if (part && r == SIM_OK) r = dcopy(part, h->s, 3 * N3 * sizeof(float), st);
  if (part && r == SIM_OK) r = dcopy(part + 3 * N3, h->p, 3 * N3 * sizeof(float), st);
  if (star && r == SIM_OK) r = dcopy(star, h->star, N3 * sizeof(float), st);
  if (aux && r == SIM_OK) r = dcopy(aux, h->aux, N3 * sizeof(float), st);
  if (events && r == SIM_OK) r = dcopy(events, h->events, ((N3 + 31) / 32) * sizeof(uint32_t), st);
  if (gravity && r == SIM_OK) r = dcopy(gravity, h->g, 3 * N3 * sizeof(float), st);
  if (step) *step = h->step;
  return fail(h, r);
}

sim_status sim_set_state(sim_t* h, const float* gas, const float* part, int32_t step) {
  if (!h || !gas || !part || step < 0 || step > h->prm.n_steps) {
    set_error("sim_set_state: invalid arguments");
    return fail(h, SIM_EINVAL);
  }
  const long long N3 = h->N3;
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

sim_status sim_cfl(sim_t* h, double* cfl_out) {
  if (!h || !cfl_out) return SIM_EINVAL;
  cudaStream_t st = h->st;
  unsigned int bits = 0;
  sim_status r = dzero(h->speed_bits, sizeof(unsigned int), st);
  if (r == SIM_OK) r = launch_signal_speed(h->gas, (float)h->prm.gamma, h->N3, h->speed_bits, st);
  if (r == SIM_OK && (cudaMemcpyAsync(&bits, h->speed_bits, sizeof(unsigned int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                      cudaStreamSynchronize(st) != cudaSuccess)) {
    set_error("sim_cfl: readback failed");
    r = SIM_ECUDA;
  }
  if (r != SIM_OK) return fail(h, r);
  float v;
  memcpy(&v, &bits, sizeof(v));
  const int i = h->step < h->prm.n_steps ? h->step : h->prm.n_steps - 1;
  *cfl_out = (double)v * h->sched[i].dtau * h->inv_dx;
  return SIM_OK;
}

}  // extern "C"
