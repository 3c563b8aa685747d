/*
 * diffhydro.h -- C ABI of the GB300 (sm_103a) differentiable cosmological hydro step.
 *
 * Method: arXiv 2502.02294 (Horowitz & Lukic, "Differentiable Cosmological Hydrodynamics",
 * diffHydro). One time step couples
 *   - the comoving Euler equations (Sec. 2.3, Eqs. cont / momentum / ev / conservation)
 *     solved with the relaxing TVD scheme (Sec. 2.3.1-2.3.2, Eqs. TVD_halfstep and
 *     TVD_fullstep, van Leer limiter, Strang-split sweeps),
 *   - dark matter particles under particle-mesh gravity with FastPM kick-drift-kick factors
 *     (Sec. 2.2, Eq. dm_hamil),
 *   - a stochastic subgrid star-formation step differentiated with Gumbel-softmax
 *     (Sec. 2.4, Eqs. reparam / gumbelsoftmax and pi_0(rho, T)),
 * and its reverse-mode derivative (Sec. 2.3.5), with checkpoints every few steps.
 *
 * Conventions for every entry point
 *   - Array arguments are DEVICE pointers owned by the caller unless a comment says "host".
 *     The library never frees them and never keeps them past the call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). Work is
 *     enqueued on it and the call returns without synchronising, except where stated.
 *   - Grids are n^3 float32 in C order [z][y][x] (x fastest). The gas state is 5 such
 *     fields back to back: rho, m_x, m_y, m_z, eps (structure of arrays, 5 n^3 floats).
 *     Particle arrays are [3][n^3] (x, y, z components) in Lagrangian order, particle
 *     index (qz n + qy) n + qx for lattice site q = (qx, qy, qz) dx; positions are stored
 *     as displacements s from the lattice site (x = q + s, periodic), momenta as p = a^2 dx/dt.
 *   - Units: length Mpc/h (comoving), velocity 100 km/s, time 1/H0 (so H0 = 1). Densities
 *     in units of the mean total matter density; the mean gas density is f_b = Omega_b/Omega_m.
 *     Gas variables: m = a rho U (U peculiar velocity), eps = a^2 rho (e + U^2/2).
 *   - Errors are returned as sim_status codes; nothing aborts or traps. sim_last_error()
 *     gives a message. Invalid arguments are rejected before any work is enqueued.
 *   - The library is not thread safe for one handle; distinct handles may be used from
 *     distinct threads.
 */
#ifndef DIFFHYDRO_H
#define DIFFHYDRO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SIM_OK = 0,
  SIM_EINVAL = 1,   /* invalid argument or state                          */
  SIM_ENOMEM = 2,   /* device allocation failed                           */
  SIM_ECUDA = 3,    /* a CUDA runtime or cuFFT call failed                */
  SIM_ECFL = 4,     /* CFL number above the configured limit (sim_run)   */
  SIM_ENAN = 5,     /* non-finite value detected in the state            */
  SIM_ETIMEOUT = 6, /* a bounded device wait gave up                      */
  SIM_ENOTIMPL = 7  /* option not implemented                             */
} sim_status;

/* Parameter block. sim_params_default() fills the values quoted beside each field. */
typedef struct {
  int32_t n;            /* grid cells per side = particles per side (32)                 */
  int32_t n_steps;      /* steps from a_start to a_end, uniform in a (20)  Sec. 2.3.3   */
  int32_t ckpt_every;   /* checkpoint interval of sim_run, steps (6)       Sec. 2.3.5   */
  int32_t subgrid_on;   /* 1: star formation + UV floor each step (0)      Sec. 2.4     */
  int32_t gravity_on;   /* 1: PM gravity and kicks (1)                                   */
  int32_t hydro_on;     /* 1: gas sweeps (1)                                             */
  int32_t kdk_mode;     /* 0: FastPM factors, 1: plain int dt factors (0)  Sec. 2.2     */
  int32_t instance;     /* Philox counter word 2 (0)                                     */
  uint64_t seed;        /* Philox key (1)                                                */
  double box;           /* box side, Mpc/h (32)                                          */
  double omega_m;       /* (0.3) */
  double omega_b;       /* (0.049): f_b = omega_b / omega_m                              */
  double h;             /* (0.7), does not enter in these units                          */
  double sigma8;        /* (0.8): scales the initial amplitude linearly                  */
  double gamma;         /* adiabatic index (5/3)                                         */
  double mu;            /* mean molecular weight (0.6)                                   */
  double T_init;        /* initial gas temperature, K (1e4)                              */
  double a_start;       /* (0.1) */
  double a_end;         /* (0.5) */
  double delta_c;       /* star-formation overdensity threshold (100)      Sec. 2.4.2  */
  double Pi0;           /* star-formation probability scale (0.05)                      */
  double E0;            /* injected specific energy, (100 km/s)^2 (0.03)                */
  double T_c;           /* star-formation temperature threshold, K (3e4)                */
  double w_delta;       /* sigmoid width in delta (5)                                    */
  double w_T;           /* sigmoid width in T, K (1500)                                  */
  double tau;           /* Gumbel-softmax temperature (0.1)                Sec. 2.4.2  */
  double T0_uv;         /* UV-background floor temperature at mean density, K; 0 = off (0) */
  double gamma_uv;      /* floor slope: T_floor = T0 (rho/f_b)^(gamma_uv - 1) (1.4)      */
  double rms_ref;       /* rms of the linear contrast at a_ref for sigma8_ref (0.05)     */
  double a_ref;         /* (0.1) */
  double sigma8_ref;    /* (0.8) */
  double omega_m_ref;   /* (0.3) */
  double kc_frac;       /* spectrum cutoff k_c as a fraction of Nyquist (0.5)            */
  double limiter_eps;   /* van Leer epsilon (1e-30)                                      */
  double cfl_max;       /* sim_run returns SIM_ECFL above this CFL number; 0 = no check (0) */
} sim_params;

/* Order of the parameter-gradient vector of sim_run_adjoint / sim_step_adjoint. */
enum {
  SIM_P_OMEGA_M = 0,
  SIM_P_SIGMA8 = 1,
  SIM_P_DELTA_C = 2,
  SIM_P_PI0 = 3,
  SIM_P_E0 = 4,
  SIM_P_T0_UV = 5,
  SIM_P_GAMMA_UV = 6,
  SIM_NPARAMS = 7
};

typedef struct sim_s sim_t;

/* Fill *p with the defaults above. Host pointer. */
sim_status sim_params_default(sim_params* p);

/* Last error message of this handle, or of the calling thread when h is NULL. */
const char* sim_last_error(const sim_t* h);

/* Number of CUDA kernels this library has launched in this process so far (all devices,
 * all threads; cuFFT's own kernels are not counted). Host-only, never fails. */
int64_t sim_kernel_launches(void);

/* ------------------------------------------------------------------ whole path */

/* Create a simulation and set up its initial conditions (Sec. 2.1): white noise w
 * (noise: device n^3 floats, or NULL to draw it from Philox with tag 0), shaped by the
 * synthetic spectrum P(k) = A k^-2 exp(-(k/k_c)^2) normalised to rms_ref (sigma8/sigma8_ref)
 * D(a_start)/D(a_ref), displaced with the Zel'dovich approximation for DM and gas, then
 * the initial force. Allocates all working memory on the current device (the handle owns
 * it). The noise buffer is read before the call returns to the stream order only; the
 * caller may reuse it after the stream reaches this point. */
sim_status sim_init(const sim_params* p, const float* noise, void* stream, sim_t** out);

/* Free the handle and its device memory (synchronises its stream). NULL is ignored. */
void sim_destroy(sim_t* h);

/* ------------------------------------------------------------------ batched instances
 * Parameter sampling (Sec. 3: many simulations differing in cosmology, subgrid parameters
 * and random seed) as one handle holding B instances on grids of the same size, stepped
 * together: every kernel of the step runs all B instances in one launch and the FFTs are
 * batched. p is a HOST array of B parameter sets that agree in n, box, n_steps, a_start,
 * a_end, ckpt_every, subgrid_on, gravity_on, hydro_on, kdk_mode, gamma, mu, h, rms_ref,
 * a_ref, sigma8_ref, omega_m_ref, kc_frac, limiter_eps and cfl_max (SIM_EINVAL
 * otherwise); omega_m, omega_b, sigma8, T_init, the subgrid parameters, seed and instance
 * may differ. noise: device B n^3 floats (instance b at b n^3) or NULL (Philox per
 * instance). With B = 1 this is sim_init.
 *
 * Every whole-path entry below then takes arrays of all B instances one after another:
 * gas B x 5 n^3, part B x 6 n^3, star / aux / noise / target B x n^3, events B x
 * ceil(n^3/32) words, gravity B x 3 n^3, parameter derivatives B x SIM_NPARAMS and the
 * loss of sim_loss_density B doubles. Instance b of a batch evolves bit for bit as a
 * B = 1 handle with the same parameters (same kernels, same order of operations), except
 * where cuFFT's batched transforms round differently from single ones. */
sim_status sim_init_batch(const sim_params* p, int32_t B, const float* noise, void* stream,
                          sim_t** out);

/* Replace the parameters of every instance (host array of B sets) keeping the handle's
 * allocations: n, box, the schedule (n_steps, a_start, a_end, ckpt_every), the switches,
 * gamma, mu, limiter_eps and cfl_max must equal those at creation (SIM_EINVAL otherwise);
 * cosmology (omega_m, omega_b, sigma8), T_init, the IC normalisation, the subgrid
 * parameters and the seeds may change. The schedules and per-instance tables are
 * recomputed, the initial conditions are rebuilt from the current white noise (or stay
 * invalid after sim_set_state), the handle is rewound to its initial state and captured
 * graphs are dropped. Synchronises the handle's stream. This is the entry of parameter
 * inference (Sec. 3.1): one handle evaluated at many parameter points. */
sim_status sim_set_params(sim_t* h, const sim_params* p);

/* Number of instances of the handle (1 for sim_init). */
int32_t sim_batch_size(const sim_t* h);

/* Hydro sweep kernel variants (Sec. 2.3.1 sweeps; the paper has no counterpart: these are
 * GB300 launch shapes). DEFAULT: the built-in choice for the grid size; TILE: shared-memory
 * tile; MARCH32 / MARCH16: one thread marches a line segment of 32 / 16 cells; MARCH_FIT:
 * the same with the segment length that fits the launch to whole waves of resident blocks
 * (forward: y and z only, the forward x sweep then uses the tile; adjoint: every axis,
 * x on x <-> y transposed copies, two passes through a 5-field scratch); PAIR: below. */
enum {
  SIM_SWEEP_DEFAULT = 0,
  SIM_SWEEP_TILE = 1,
  SIM_SWEEP_MARCH32 = 2,
  SIM_SWEEP_MARCH16 = 3,
  SIM_SWEEP_MARCH_FIT = 4,
  SIM_SWEEP_PAIR = 5  /* forward y / z sweeps with even n: the fitted marching form on two
                         adjacent x columns per thread in packed FP32x2 arithmetic (the
                         tile for x and for odd n); adjoint: as MARCH_FIT                 */
};

/* Set the variant of the forward (fwd[3], per axis) and adjoint (adj[3]) sweeps of the
 * handle. Host arrays; NULL leaves that set unchanged. Drops captured graphs. */
sim_status sim_set_sweep_variants(sim_t* h, const int32_t* fwd, const int32_t* adj);

/* ------------------------------------------------------------------ groups of handles
 * Batches on grids of different sizes (e.g. 32 instances each at 32^3, 48^3 and 64^3): one
 * batched handle per size, run as a group. The group captures its members' runs into one
 * CUDA graph with one concurrent branch per member and replays it with a single graph
 * launch on `stream` (members are used on their branches during the call and must not be
 * used concurrently elsewhere; create them on the same stream). The paper has no
 * counterpart: this is the launch structure of many-sample parameter studies (Sec. 3). */
typedef struct sim_group_s sim_group_t;

/* members: host array of `count` distinct handles (not owned). */
sim_status sim_group_create(sim_t* const* members, int32_t count, void* stream,
                            sim_group_t** out);

/* sim_run of every member from its initial state to its last step (cfl_max must be 0). */
sim_status sim_group_run(sim_group_t* g);

/* sim_run_adjoint of every member: dL_dgas[k] is member k's loss derivative at the final
 * gas state (device, B_k x 5 n_k^3; the host array or an entry may be NULL = 0) and
 * dL_dparams[k] receives its B_k x SIM_NPARAMS parameter derivatives (device, overwritten).
 * No noise gradient. */
sim_status sim_group_run_adjoint(sim_group_t* g, const float* const* dL_dgas,
                                 double* const* dL_dparams);

/* sim_reset of every member. */
sim_status sim_group_reset(sim_group_t* g);

/* Free the group (not its members); synchronises its stream. NULL is ignored. */
void sim_group_destroy(sim_group_t* g);

/* Autotuner: times every variant of each forward and adjoint sweep on the handle's current
 * state (all B instances, CUDA events, `reps` launches each, best of them), keeps the
 * fastest per axis, and writes the choice to fwd_out[3] / adj_out[3] (host, may be NULL).
 * The state is not modified. Synchronises the stream; drops captured graphs. */
sim_status sim_autotune(sim_t* h, int32_t reps, int32_t* fwd_out, int32_t* adj_out);

/* on != 0: sim_run and sim_run_adjoint are captured into CUDA graphs the first time they
 * are called with a given argument set from a given handle state, and replayed afterwards
 * (launch overhead of the ~50 kernels per step removed). Capture happens on a private
 * stream ordered after the handle's stream; replays run on the handle's stream. Graphs
 * keep the argument pointers they were captured with. Not used when cfl_max > 0.
 * on == 0 drops all graphs. Default off. */
sim_status sim_set_graphs(sim_t* h, int32_t on);

/* Kernel classes timed by sim_kernel_timing. The paper has no counterpart: these exist to
 * measure the stages of the step (Secs. 2.2-2.4) and their adjoints inside a real run. */
enum {
  SIM_KT_SWEEP = 0,            /* forward sweeps, including the reverse pass's recompute */
  SIM_KT_SWEEP_ADJOINT = 1,    /* adjoint sweeps */
  SIM_KT_KICK = 2,             /* particle kick + drift, gas kick */
  SIM_KT_KICK_ADJOINT = 3,     /* their adjoints */
  SIM_KT_DEPOSIT = 4,          /* CIC deposit and fixed-point conversion */
  SIM_KT_DEPOSIT_ADJOINT = 5,  /* deposit adjoint (CIC gradient readout) */
  SIM_KT_POISSON = 6,          /* r2c, Green's function, 3 c2r */
  SIM_KT_POISSON_ADJOINT = 7,  /* its adjoint, with the force dot product */
  SIM_KT_SUBGRID = 8,          /* subgrid step */
  SIM_KT_SUBGRID_ADJOINT = 9,  /* its adjoint */
  SIM_KT_N = 10
};

/* enable != 0: later sim_step / sim_run / sim_step_adjoint / sim_run_adjoint calls run
 * eagerly (no graph replay) and bracket every launch of a timed class with two CUDA events
 * on the handle's stream; up to 8192 launches are recorded between resets, later ones run
 * untimed. enable == 0 stops recording. Default off. */
sim_status sim_kernel_timing(sim_t* h, int32_t enable);

/* Host arrays ms[SIM_KT_N] and count[SIM_KT_N] receive the summed device time (ms) and the
 * number of recorded launches per class; waits for the last recorded event. reset != 0
 * clears the records afterwards. SIM_EINVAL on a NULL argument. */
sim_status sim_kernel_times(sim_t* h, double* ms, int64_t* count, int32_t reset);

/* Advance one step a_n -> a_{n+1}: half kick (DM + gas), DM drift, three Strang-ordered
 * hydro sweeps (order XYZ, ZYX, ZXY, YXZ, YZX, XZY by n mod 6, Sec. 2.3.2), subgrid,
 * CIC deposit + Poisson (Sec. 2.2), half kick. Keeps a copy of the step's input state
 * so that sim_step_adjoint can back-propagate through it. */
sim_status sim_step(sim_t* h);

/* Reverse-mode derivative of the most recent sim_step. On entry adj_gas (5 n^3) and
 * adj_part (6 n^3: d/ds then d/dp) hold dL/d(state after the step); on return they hold
 * dL/d(state before the step). adj_params (device, SIM_NPARAMS doubles) is ACCUMULATED
 * with the step's direct dependence on the parameters. The step's gravity at its start is
 * a function of the state before it, and is differentiated as such. */
sim_status sim_step_adjoint(sim_t* h, float* adj_gas, float* adj_part, double* adj_params);

/* Advance n_steps steps from the initial state (the handle must be fresh from sim_init or
 * sim_reset), storing a checkpoint of the state every ckpt_every steps for
 * sim_run_adjoint (Sec. 2.3.5: checkpoints every 6 steps in the paper). Once the handle
 * holds the reverse pass's tape (after its first sim_run_adjoint), the run also records its
 * last checkpoint segment(s) on the tape (sim_set_tape_recording), so that the next
 * sim_run_adjoint does not recompute them; the results are the same either way. */
sim_status sim_run(sim_t* h, int32_t n_steps);

/* Checkpoint segments (ckpt_every steps each) that sim_run records on the tape at the end of
 * a run once the handle holds one: 1 (the default) records the segment after the last
 * checkpoint, k > 1 the last k segments, -1 all of them (the reverse pass then recomputes
 * nothing: at 128^3, 46 floats per cell per step, 3.9 GB per 10-step segment), 0 nothing
 * (for handles that mostly run forward). Each recorded step costs a few device copies; each
 * recorded segment is one segment less for the next sim_run_adjoint to recompute. The tape
 * for k segments is allocated by the next sim_run_adjoint (or sim_fli_step /
 * sim_posterior, which record at least one segment). Results are the same for every k.
 * SIM_EINVAL on a NULL handle or segments < -1. */
sim_status sim_set_tape_recording(sim_t* h, int32_t segments);

/* Gradient of a scalar loss through the whole run made by sim_run and through the
 * initial conditions. dL_dgas (5 n^3) and dL_dpart (6 n^3: d/ds then d/dp) are the
 * loss derivatives at the final state (either may be NULL = 0). Outputs: dL_dnoise
 * (n^3, may be NULL) and dL_dparams (device, SIM_NPARAMS doubles, overwritten). Each
 * segment between checkpoints is recomputed forward once. */
sim_status sim_run_adjoint(sim_t* h, const float* dL_dgas, const float* dL_dpart,
                           float* dL_dnoise, double* dL_dparams);

/* Rewind the handle to its initial state (keeps allocations; clears checkpoints). */
sim_status sim_reset(sim_t* h);

/* Recompute the initial conditions from new white noise (device n^3; NULL = Philox draw
 * of the handle's seed) and rewind to step 0, keeping all allocations. This is the
 * per-iteration entry of field-level inference (Sec. 3.2): the noise is the variable. */
sim_status sim_reinit(sim_t* h, const float* noise);

/* Density loss of the current state (Sec. 3.1-3.2): L = c sum_cells (rho - target)^2,
 * c = 1/n^3 gives the mean squared error, c = 1/(2 sigma^2) the Gaussian pixel likelihood
 * of field-level inference. Writes dL/d(gas) (5 n^3: 2 c (rho - target) in the density
 * field, 0 elsewhere) and stores L in *loss (device double, overwritten). */
sim_status sim_loss_density(sim_t* h, const float* target, double c, float* dL_dgas,
                            double* loss);

/* ------------------------------------------------------------------ field-level inference
 * Sec. 3.2: the initial conditions are inferred from a final observed field d by minimising
 * the negative log posterior of the white-noise amplitudes s,
 *   L(s) = 1/2 [ sum_cells (d - O(s))^2 / sigma_n^2 + sum_cells s^2 ],
 * O(s) an observable of the final gas state of the handle's whole run (sim_init
 * parameters) from initial conditions made of s (Sec. 2.1). Observables: */
enum {
  SIM_OBS_DENSITY = 0,  /* gas density rho                                              */
  SIM_OBS_THERMAL = 1   /* internal energy density eps - |m|^2/(2 rho) = a^2 rho e, which is
                           proportional to the gas-mass-weighted temperature rho T (the
                           delta_b T probe of Sec. 3.2)                                   */
};

/* Loss of an observable of the current state: L = c sum_cells (O - target)^2 per instance
 * (loss: B device doubles, overwritten) and dL/d(gas) (5 B n^3, overwritten). */
sim_status sim_loss_field(sim_t* h, int32_t observable, const float* target, double c,
                          float* dL_dgas, double* loss);

/* Posterior and its gradient at the amplitudes `noise` (B n^3, device, read only): ICs from
 * noise (sim_reinit), sim_run of all n_steps (checkpoints every ckpt_every), the checkpointed
 * reverse pass, plus the prior. loss (B device doubles): L; grad (B n^3): dL/ds. The
 * handle's state is the run from `noise` afterwards. Requires cfl_max = 0; SIM_ENOTIMPL
 * while a learned closure is set. */
sim_status sim_posterior(sim_t* h, int32_t observable, const float* noise, const float* data,
                         double sigma_n, double* loss, float* grad);

/* One Adam iteration: sim_posterior at the input amplitudes, then one Adam step (Kingma &
 * Ba 2015; beta1 0.9, beta2 0.999, eps 1e-8, bias corrected with step t >= 1) on them with
 * learning rate lr. noise (B n^3, in: s, out: the updated s), m and v (B n^3, Adam moments,
 * in/out; at t = 1 their contents are ignored and the moments start from zero), data
 * (B n^3). loss (B doubles: L at the input s), grad
 * (B n^3 or NULL: dL/ds at the input s). Stream-ordered, no synchronisation. SIM_EINVAL for
 * NULL arrays, sigma_n <= 0, lr <= 0, t < 1 or an unknown observable. */
sim_status sim_fli_step(sim_t* h, int32_t observable, float* noise, float* m, float* v,
                        const float* data, double sigma_n, double lr, int32_t t, double* loss,
                        float* grad);

/* Vector kernels for host-driven optimisers (L-BFGS two-loop recursion, line searches) on
 * device vectors of `count` floats: sim_dot writes sum a_i b_i to *out (one device double,
 * overwritten); sim_axpby sets y = alpha x + beta y. The paper has no counterpart. */
sim_status sim_dot(const float* a, const float* b, int64_t count, double* out, void* stream);
sim_status sim_axpby(double alpha, const float* x, double beta, float* y, int64_t count,
                     void* stream);

/* Adam step on a device vector (Kingma & Ba 2015, Algorithm 1, bias corrected with step
 * t >= 1) with the gradient g + prior_w x, the gradient of a data term plus that of the
 * Gaussian prior prior_w |x|^2 / 2 (prior_w = 1 for the white-noise amplitudes of Sec. 3.2,
 * 0 for plain Adam). x, m, v (count floats, in/out; at t = 1 the moments start from zero
 * and their contents are not read), g (count floats). grad_out (count
 * floats or NULL) receives g + prior_w x; prior (one device double or NULL) is ACCUMULATED
 * with prior_w / 2 |x|^2 at the input x. SIM_EINVAL for NULL arrays, count < 1, t < 1,
 * lr <= 0, beta outside [0, 1) or eps <= 0. */
sim_status sim_adam(float* x, const float* g, float* m, float* v, int64_t count, double lr,
                    double beta1, double beta2, double eps, int32_t t, double prior_w,
                    float* grad_out, double* prior, void* stream);

/* Adjoint of sim_power_spectrum (auto spectrum): dL_da (n^3, overwritten) = sum over bins b
 * of dL_dpk[b] dP_b/da, for dL_dpk device doubles of length nbins, same binning. Uses cuFFT.
 * With it a likelihood of the binned spectrum is differentiated back to the density field
 * and, through sim_run_adjoint, to the parameters (Sec. 3.1). */
sim_status sim_power_spectrum_adjoint(const float* a, int32_t n, double box, int32_t nbins,
                                      const double* dL_dpk, float* dL_da, void* stream);

/* Cross-correlation coefficient r_c(k) = P_ab / sqrt(P_aa P_bb) (Sec. 3.2) of two n^3 fields,
 * binned as sim_power_spectrum (width 2 pi / box, index round(|k| box / 2 pi), bins
 * 1..nbins): k (mode-weighted mean |k|), rc (0 where a power is 0), nmodes; device doubles
 * of length nbins (1 <= nbins <= 1024). Uses cuFFT. */
sim_status sim_cross_correlation(const float* a, const float* b, int32_t n, double box,
                                 int32_t nbins, double* k, double* rc, double* nmodes,
                                 void* stream);

/* ------------------------------------------------------------------ diagnostics
 * Per-step record of a run, for time-step control (Eq. dt) and for conservation checks of
 * the finite-volume scheme (Sec. 2.3): after every step of sim_step / sim_run (and for the
 * initial state at the start of a run) one kernel sums the state into a device record.
 * Entries of a record (doubles), per instance: */
enum {
  SIM_DG_A = 0,       /* scale factor of the recorded state                      */
  SIM_DG_MASS,        /* sum over cells of rho (gas mass / cell volume)         */
  SIM_DG_MX,          /* sums of the gas momentum density m_x, m_y, m_z          */
  SIM_DG_MY,
  SIM_DG_MZ,
  SIM_DG_ENERGY,      /* sum of eps                                              */
  SIM_DG_PX,          /* DM momentum: particle mass x sum of p_x, p_y, p_z       */
  SIM_DG_PY,
  SIM_DG_PZ,
  SIM_DG_STARS,       /* sum of the step's relaxed star field zhat (Sec. 2.4.2)  */
  SIM_DG_EVENTS,      /* number of hard star-formation events of the step        */
  SIM_DG_NONFINITE,   /* cells with a non-finite field or pressure (left out of
                         the sums and minima above)                             */
  SIM_DG_RHO_MIN,     /* smallest density (NaN if no finite cell)                */
  SIM_DG_P_MIN,       /* smallest pressure P = (gamma-1)(eps - |m|^2/2rho)       */
  SIM_DG_N
};

/* on != 0: record every later step (allocates (n_steps + 1) x B records on the first call;
 * never call it inside a stream capture). While on, sim_run keeps each step's closing half
 * kick apart from the next opening one so that every record holds a whole step's end
 * state; keep the setting unchanged between a sim_run and its sim_run_adjoint. Drops
 * captured graphs when the setting changes. The paper has no counterpart. */
sim_status sim_set_diagnostics(sim_t* h, int32_t on);

/* Record of the state after step `step` (0 = the run's initial state): host out[B][SIM_DG_N].
 * Synchronises the handle's stream. SIM_EINVAL if that step was not recorded. */
sim_status sim_diagnostics(sim_t* h, int32_t step, double* out);

/* Copy the current state out (device pointers; any may be NULL):
 * gas 5 n^3, part 6 n^3 (s then p), star n^3 (accumulated relaxed star field),
 * aux n^3 (per-particle star readout, Sec. 2.4.1), events n^3/32 uint32 words (bit i of
 * word j: cell 32 j + i formed a star in the last step's hard Gumbel-max draw),
 * gravity 3 n^3 (current force field on the mesh). Also returns the step index. */
sim_status sim_get_state(sim_t* h, float* gas, float* part, float* star, float* aux,
                         uint32_t* events, float* gravity, int32_t* step);

/* Overwrite the state (gas 5 n^3, part 6 n^3) at step index `step` and recompute the
 * force field. Star, aux and checkpoints are cleared. */
sim_status sim_set_state(sim_t* h, const float* gas, const float* part, int32_t step);

/* Host FP64 step factors of step i: out[0..5] = a_i, a_{i+1}, K1, dtau, K2,
 * 3 Omega_m / (2 a_{i+1}) (FastPM or plain, Sec. 2.2). Host pointer. */
sim_status sim_schedule(const sim_t* h, int32_t i, double* out6);

/* Largest CFL number max(|v_d| + c_s) dtau / dx over cells and directions for the
 * current state and the next step's dtau (Eq. dt). Synchronises the stream. A non-finite
 * value anywhere in the gas state makes the result NaN (sim_run with cfl_max > 0 then
 * returns SIM_ENAN). */
sim_status sim_cfl(sim_t* h, double* cfl_out);

/* ------------------------------------------------------------------ learned closure
 * Solver-in-the-loop refinement (Sec. 4 lists it among the uses of a differentiable
 * solver): after every step the five gas fields get a residual correction
 *   u <- u + s * NN((u - mu) / sigma)        (mu, sigma, s: one value per field)
 * from a network of four periodic 3x3x3 convolutions 5 -> 16 -> 16 -> 16 -> 5 with GELU
 * between them, bfloat16 weights and activations, float32 accumulation on the tensor
 * cores. conv(h, W)[v, co] = sum over taps t and input channels ci of
 * h[v + off(t), ci] W[t, ci, co], tap t = 9 (dz + 1) + 3 (dy + 1) + (dx + 1).
 * Weight vector (host float32, SIM_CLOSURE_NWEIGHTS values): for layers (Cin, Cout) =
 * (5, 16), (16, 16), (16, 16), (16, 5): W[t][ci][co] (co fastest), then b[co].
 * Gas arrays are B x 5 n^3 as everywhere else. */
#define SIM_CLOSURE_NWEIGHTS 18197

typedef struct sim_closure_s sim_closure_t;

/* weights: host vector or NULL (all zero: the correction is the identity). */
sim_status sim_closure_create(const float* weights, void* stream, sim_closure_t** out);
void sim_closure_destroy(sim_closure_t* c);

/* Per-field normalisation: host arrays of 5 (sigma, scale > 0). Default 0 / 1 / 1. */
sim_status sim_closure_set_norm(sim_closure_t* c, const float* mu, const float* sigma,
                                const float* scale);

/* Copy the weights out / in (host vectors). Setting them clears the optimiser state;
 * both synchronise the closure's stream. */
sim_status sim_closure_get_weights(sim_closure_t* c, float* host_out);
sim_status sim_closure_set_weights(sim_closure_t* c, const float* host_in);

/* y = NN((gas - mu) / sigma) (device, B x 5 n^3, normalised units; gas unchanged). */
sim_status sim_closure_forward(sim_closure_t* c, const float* gas, int32_t n, int32_t B,
                               float* y);

/* gas += s * NN((gas - mu) / sigma) in place. */
sim_status sim_closure_apply(sim_closure_t* c, float* gas, int32_t n, int32_t B);

/* Loss L = mean over fields, cells and instances of (y - (target - gas) / s)^2 and its
 * gradient with respect to the weights (host vector, SIM_CLOSURE_NWEIGHTS), for the
 * training pair (gas before the correction, target state). Synchronises. */
sim_status sim_closure_gradient(sim_closure_t* c, const float* gas, const float* target,
                                int32_t n, int32_t B, double* loss_host, float* grad_host);

/* One training step on that loss: gradient, then Adam (beta 0.9 / 0.999, eps 1e-8, bias
 * corrected) with learning rate lr. loss_out (device double, may be NULL) receives the
 * loss before the update. Stream-ordered, no synchronisation. */
sim_status sim_closure_train_step(sim_closure_t* c, const float* gas, const float* target,
                                  int32_t n, int32_t B, double lr, double* loss_out);

/* Synchronise and report a timed-out tensor-core wait of an earlier call (SIM_ETIMEOUT),
 * then clear the report: a later call returns SIM_OK unless a wait timed out again. The
 * outputs of a call whose wait timed out are undefined. */
sim_status sim_closure_status(sim_closure_t* c);

/* Time limit of each wait inside the closure's tensor-core kernels (a stage waiting for an
 * input plane, for its MMAs, or for a free accumulator slot), in nanoseconds of the GPU's
 * global timer (a wait gives up within 20 us after it); default 1e9 (1 s). A wait that
 * runs out records SIM_ETIMEOUT for
 * sim_closure_status and its kernel stops early, after waiting (up to 4 s) for the copies
 * and MMAs it has already issued, so the context stays usable. ns = 0 allows a single
 * non-blocking check per wait (which makes the first waits of a launch give up: the way to
 * exercise this path). Applies to later launches; graphs captured earlier keep the limit
 * they were captured with. The paper has no counterpart. SIM_EINVAL if ns < 0. */
sim_status sim_closure_set_wait_limit(sim_closure_t* c, int64_t ns);

/* Apply `c` at the end of every step of the handle (sim_step, sim_run, groups), on the
 * handle's stream; NULL removes it (the plain solver). Prepares the closure's workspace for
 * the handle's grid. While a closure is set the adjoint entry points return SIM_ENOTIMPL.
 * The closure must outlive its use by the handle. */
sim_status sim_set_closure(sim_t* h, sim_closure_t* c);

/* Training pairs of the closure: coarse runs against runs twice as fine.
 * sim_refine_noise: w_f (n_f^3) = scale * band-limited interpolation of w_c (n_c^3): the
 *   coarse Fourier modes, with an even n_c's Nyquist modes split equally between +k and
 *   -k, the finer modes zero. With scale = C_coarse / C_fine (sim_ic_amplitude) and the
 *   fine handle's kc_frac halved, the fine run's linear field equals the coarse one.
 * sim_restrict_gas: coarse cell j = tent-weighted (1/4, 1/2, 1/4 per axis) mean of the
 *   fine cells around fine cell 2j; B x 5 fields.
 * sim_restrict_particles: the fine particle at lattice site 2q is coarse particle q;
 *   B x 6 n^3 (s then p). */
sim_status sim_refine_noise(const float* w_c, int32_t n_c, float* w_f, int32_t n_f,
                            double scale, void* stream);
sim_status sim_restrict_gas(const float* gas_f, int32_t n_f, float* gas_c, int32_t B,
                            void* stream);
sim_status sim_restrict_particles(const float* part_f, int32_t n_f, float* part_c, int32_t B,
                                  void* stream);

/* Amplitude C of instance b's initial conditions (delta_k = C sqrt(P(k)) w_k / n^3), host. */
sim_status sim_ic_amplitude(const sim_t* h, int32_t b, double* C);

/* ------------------------------------------------------------------ single kernels */

/* One relaxing-TVD sweep along axis (0 = x, 1 = y, 2 = z) with nu = dtau/dx:
 * half step with first-order upwind relaxed fluxes (Eq. TVD_halfstep), full step with
 * limited second-order fluxes on the half-step state (Eq. TVD_fullstep). u_in, u_out:
 * 5 n^3 each, must not alias. variant: SIM_SWEEP_* kernel form (SIM_SWEEP_DEFAULT = the
 * built-in choice for the axis and n; every form gives the same result up to float32
 * rounding order), other values SIM_EINVAL. */
sim_status sim_sweep(const float* u_in, float* u_out, int32_t n, int32_t axis, double nu,
                     double gamma, double limiter_eps, int32_t variant, void* stream);

/* Largest signal speed max over cells of max(|v_x|, |v_y|, |v_z|) + c_s of a gas state
 * (5 n^3), written to *out (one device float); NaN if any cell is not finite. With a step
 * dt the CFL number of Eq. dt is *out dt / dx. */
sim_status sim_max_signal_speed(const float* gas, int32_t n, double gamma, float* out,
                                void* stream);

/* Adjoint of sim_sweep at u_in: lam_in = (d u_out / d u_in)^T lam_out (5 n^3 each, no
 * aliasing). If dnu (device double) is not NULL, adds lam_out . d u_out / d nu to it.
 * variant as for sim_sweep. */
sim_status sim_sweep_adjoint(const float* u_in, const float* lam_out, float* lam_in,
                             int32_t n, int32_t axis, double nu, double gamma,
                             double limiter_eps, double* dnu, int32_t variant, void* stream);

/* Cloud-in-cell deposit (Sec. 2.2): grid[node] += sum_p value_p W(x_p - node) with
 * W the CIC weights, cell decision floor(s/dx) taken in float32. values may be NULL (=1).
 * Particles: np = n^3 in Lagrangian order of an n^3 lattice, s: 3 n^3. grid: n^3,
 * ACCUMULATED. Deterministic (64-bit fixed-point accumulation). */
sim_status sim_deposit_cic(const float* s, const float* values, int32_t n, double box,
                           float* grid, void* stream);

/* Same result as sim_deposit_cic, for callers that cannot allocate device memory: those
 * running while a framework's caching allocator holds the device memory (a direct
 * allocation may then fail), those that must keep a fixed device footprint after start-up,
 * and latency-critical loops that cannot take cudaFree's implicit synchronisation. The
 * paper has no counterpart; this is a deployment variant of the deposit above.
 * It calls no allocating routine: its fixed-point accumulator is a library-owned static
 * device array of SIM_DEPOSIT_STATIC_MAX_CELLS 64-bit words (16 MiB), which every GPU
 * that loads the library holds until the process exits. Requires n^3 <= that maximum
 * (n <= 128), else SIM_EINVAL. The first call on each device looks up the array's device
 * address with that device current; make that first call before any stream capture.
 * All calls on one device share its array, which keeps the last call's contents; each call
 * clears the part it uses on entry. Calls on the same device that can overlap on the GPU
 * (for instance on two streams without ordering between them) race. */
#define SIM_DEPOSIT_STATIC_MAX_CELLS 2097152
sim_status sim_deposit_cic_static(const float* s, const float* values, int32_t n, double box,
                                  float* grid, void* stream);

/* CIC readout of `nf` fields (grid: nf n^3) at the particles: out[f][p] (nf n^3). */
sim_status sim_interp_cic(const float* grid, int32_t nf, int32_t n, double box,
                          const float* s, float* out, void* stream);

/* Spectral Poisson force g = -grad(phi), del^2 phi = pref * delta (Sec. 2.2):
 * g_k = i k pref delta_k / k^2, k = 0 removed, Nyquist gradient factor zeroed.
 * delta: n^3, g: 3 n^3 (x, y, z). Uses cuFFT. */
sim_status sim_gravity(const float* delta, int32_t n, double box, double pref, float* g,
                       void* stream);

/* Adjoint of sim_gravity: lam_delta = (d g / d delta)^T lam_g (lam_g 3 n^3, lam_delta n^3). */
sim_status sim_gravity_adjoint(const float* lam_g, int32_t n, double box, double pref,
                               float* lam_delta, void* stream);

/* Subgrid update of a gas state in place at scale factor a with Philox draws of
 * (seed, step, instance): pi_0(rho, T), Gumbel-softmax zhat (Eq. gumbelsoftmax), energy
 * injection E0 zhat, UV floor. zhat (n^3) and events (n^3/32 words) may be NULL.
 * `gas` 5 n^3. Parameters from *p (gamma, mu, omega_b/omega_m, subgrid fields). */
sim_status sim_subgrid(float* gas, int32_t n, double a, const sim_params* p, int32_t step,
                       float* zhat, uint32_t* events, void* stream);

/* Adjoint of sim_subgrid at gas_in (the state before the update): lam (5 n^3) is
 * overwritten with the adjoint of the input; dparams (device doubles, SIM_NPARAMS) is
 * accumulated for delta_c, Pi0, E0, T0_uv, gamma_uv; dfb (device double, may be NULL)
 * accumulates the derivative with respect to f_b. */
sim_status sim_subgrid_adjoint(const float* gas_in, float* lam, int32_t n, double a,
                               const sim_params* p, int32_t step, double* dparams,
                               double* dfb, void* stream);

/* Philox4x32-10 words for counters (i, step, instance, tag), i = 0..count-1, key from
 * seed: out[4*i + j] = word j. */
sim_status sim_philox(uint64_t seed, uint32_t step, uint32_t instance, uint32_t tag,
                      int64_t count, uint32_t* out, void* stream);

/* Binned power spectrum (Sec. 3.1; cross spectrum if b != NULL) of n^3 fields a, b with
 * bins of width k_f = 2 pi / box, bin index round(|k|/k_f), bins 1..nbins reported:
 * k (mode-weighted mean |k|), pk = box^3 <Re(a_k conj(b_k))> / n^6, nmodes. Outputs are
 * device doubles of length nbins (1 <= nbins <= 2048). Uses cuFFT. */
sim_status sim_power_spectrum(const float* a, const float* b, int32_t n, double box,
                              int32_t nbins, double* k, double* pk, double* nmodes,
                              void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DIFFHYDRO_H */
